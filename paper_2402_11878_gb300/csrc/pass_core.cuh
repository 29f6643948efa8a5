// Device core of the ansatz tile passes, shared by the grid kernels
// (k_layers.cu) and the persistent batched kernel (k_batch.cu).
//
// A tile holds 2^k amplitudes of the state.  Its tile bits map to global
// index bits as [0, m) -> [0, m) and [m, k) -> [a, a + k - m); `gbase` carries
// the fixed global bits of the tile.  The pass program (see vqe_internal.h)
// moves the amplitudes between shared memory and registers in "rounds": in a
// round, each thread holds 2^R amplitudes whose tile indices differ in the R
// bits [chunk, chunk + R) and applies the RY butterflies of those bits in
// registers.  Between rounds the tile goes through shared memory in a padded
// layout (pad_of below).
//
// The Env policy supplies the per-state data:
//   RotCoef<T> coef(int slot, int tile_bit)    RY coefficient of a gated bit
//   C diag(int slot, uint32_t e)               diagonal table entry of tile element e
//   static constexpr bool kDiagRow  true: the slot's table is stored in full and
//        const C *diag_row(int slot, uint32_t e0) points at entry e0 (entry e0 + j at [j])
//   void grad(int slot, int tile_bit, int comp, double v)   (backward) block total of
//        a gradient partial: comp 0 = theta (RY), 1 = phi (RZ); called by thread 0
//   static constexpr int kLoad    where the first round reads the tile:
//        0 = `buf`/`lbuf` in plain order, 1 = the state in global memory
//        (members P, L and init_zero: start from |0...0>), 2 = `buf`/`lbuf` in
//        the padded layout of the first round's chunk (a prefetched tile)
//   static constexpr int kStore   where the last round writes the tile:
//        0 = `buf`/`lbuf` in plain order, 1 = the state in global memory (P, L)
#pragma once

#include <type_traits>

#include "csum.cuh"
#include "vqe_internal.h"

namespace vqe {

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

template <int P> struct ChunkC { static constexpr int value = P; };

__device__ __forceinline__ uint32_t elem_of(uint32_t t, uint32_t r, int p, int R) {
    const uint32_t lo = t & ((1u << p) - 1u);
    return lo | (r << p) | ((t >> p) << (p + R));
}

// Shared-memory slot of tile element e between register rounds: one pad
// element after every bank row of 128 bytes (2^S elements, S = 4 for 8-byte
// and 3 for 16-byte elements).  A round at chunk P accesses elements
// e0 + (r << P) with disjoint bits, and since the low S bits of e0 and of
// r << P are disjoint, pad(e0 + (r << P)) = pad(e0) + pad(r << P): the
// register part is a compile-time offset.  For the register counts of the
// default plans (16 amplitudes per thread in FP32, 8 in FP64) the 16 (FP32) or
// 8 (FP64) lanes of one shared-memory wavefront fall on distinct bank groups
// at every chunk position.
template <typename T> struct PadShift;
template <> struct PadShift<float> { static constexpr int value = 4; };
template <> struct PadShift<double> { static constexpr int value = 3; };
template <typename T> __host__ __device__ constexpr uint32_t pad_of(uint32_t e) {
    return e + (e >> PadShift<T>::value);
}

// A chunk known only at run time, with the same `value` member as ChunkC: code
// written against `pc.value` compiles for both (constant-folded for ChunkC).
struct RtChunk {
    int value;
};

// Calls f(std::integral_constant<int, P>) for the runtime chunk p, P in [0, 14 - R].
template <int R, class F>
__device__ __forceinline__ void with_chunk(int p, F &&f) {
    switch (p) {
#define VQE_CHUNK_CASE(PP) \
    case PP:               \
        if constexpr (PP + R <= kMaxTileBits) f(ChunkC<PP>{}); \
        break;
        VQE_CHUNK_CASE(0) VQE_CHUNK_CASE(1) VQE_CHUNK_CASE(2) VQE_CHUNK_CASE(3)
        VQE_CHUNK_CASE(4) VQE_CHUNK_CASE(5) VQE_CHUNK_CASE(6) VQE_CHUNK_CASE(7)
        VQE_CHUNK_CASE(8) VQE_CHUNK_CASE(9) VQE_CHUNK_CASE(10) VQE_CHUNK_CASE(11)
        VQE_CHUNK_CASE(12) VQE_CHUNK_CASE(13)
#undef VQE_CHUNK_CASE
        default:
            break;
    }
}

__device__ __forceinline__ double flip_sign(double v, uint32_t s) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)s << 63));
}
__device__ __forceinline__ float flip_sign(float v, uint32_t s) {
    return __int_as_float(__float_as_int(v) ^ (int)(s << 31));
}

// Truth table of bit j of the register index r over r = 0..31 (bit r of the
// result is bit j of r).
__host__ __device__ constexpr uint32_t reg_bit_table(int j) {
    return j == 0 ? 0xAAAAAAAAu : j == 1 ? 0xCCCCCCCCu : j == 2 ? 0xF0F0F0F0u
         : j == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}

// a * x + y on both components of a complex value: FP32 issues one packed
// f32x2 FMA (sm_100 and later), FP64 two DFMA.
__device__ __forceinline__ float2 caxpy(float a, float2 x, float2 y) {
    return __ffma2_rn(make_float2(a, a), x, y);
}
__device__ __forceinline__ double2 caxpy(double a, double2 x, double2 y) {
    return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

template <typename C>
__device__ __forceinline__ C cmul(C x, C d) {
    C r;
    r.x = fma(x.x, d.x, -x.y * d.y);
    r.y = fma(x.x, d.y, x.y * d.x);
    return r;
}
template <typename C>
__device__ __forceinline__ C cmul_conj(C x, C d) {   // x * conj(d)
    C r;
    r.x = fma(x.x, d.x, x.y * d.y);
    r.y = fma(x.y, d.x, -x.x * d.y);
    return r;
}

// Scratch a backward tile program needs besides the tile buffers:
// nwarps * k * 2 doubles.
__host__ __device__ inline size_t tile_grad_scratch_bytes(int threads, int k) {
    return size_t((threads + 31) / 32) * k * 2 * sizeof(double);
}

// Runs the program `ops[0..n_ops)` of pass `d` on the tile in `buf` (and
// `lbuf` when backward).  All threads of the block must call it; threads
// t >= 2^(k-R) take part only in the barriers.  `gsh` is the backward
// scratch of tile_grad_scratch_bytes(blockDim.x, k) bytes.
template <typename T, int R, bool BWD, class Env>
__device__ __forceinline__ void run_tile(const PassDesc &d, const PassOp *ops, int n_ops,
                                         uint64_t gbase, typename V2<T>::type *buf,
                                         typename V2<T>::type *lbuf, double *gsh, Env &env) {
    using C = typename V2<T>::type;
    constexpr int NR = 1 << R;
    const int k = d.k, m = d.m, a = d.a;
    const uint32_t nthr = 1u << (k - R);
    const uint32_t t = threadIdx.x;
    const bool active = t < nthr;
    const int nwarps = (int)((blockDim.x + 31) >> 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned wmask = nthr >= 32 ? 0xffffffffu : ((1u << nthr) - 1u);
    const int wlanes = nthr >= 32 ? 32 : (int)nthr;
    const uint32_t lowmask = (1u << m) - 1u;
    auto g32 = [&](uint32_t e) -> uint32_t {
        return (uint32_t)(gbase | (uint64_t)(e & lowmask) | ((uint64_t)(e >> m) << a));
    };

    C v[NR];
    C w[NR];

    // Global loads (first round) and stores (last round) at compile-time
    // chunk P: register r holds global index g0 + off_r, off_r the sum of the
    // global strides of the set bits of r (tile bit b sits at global position
    // b below m and a + b - m above).  When the chunk lies in the low
    // contiguous part the offsets are compile-time constants.
    auto reg_offset = [&](auto pc, int r, const uint32_t (&gst)[R]) -> uint32_t {
        constexpr int P = decltype(pc)::value;
        uint32_t off = 0;
#pragma unroll
        for (int j = 0; j < R; ++j)
            if ((r >> j) & 1) off += (P + R <= m) ? (1u << (P + j)) : gst[j];
        return off;
    };
    auto global_strides = [&](auto pc, uint32_t (&gst)[R]) {
        constexpr int P = decltype(pc)::value;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int bt = P + j;
            gst[j] = bt < m ? (1u << bt) : (1u << (a + bt - m));
        }
    };
    auto direct_load = [&](auto pc) {
        if constexpr (Env::kLoad == 1) {
            constexpr int P = decltype(pc)::value;
            const uint32_t g0 = g32(elem_of(t, 0, P, R));
            uint32_t gst[R];
            global_strides(pc, gst);
            const C *Pb = env.P + g0;
            const C *Lb = BWD ? env.L + g0 : nullptr;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t off = reg_offset(pc, r, gst);
                if (env.init_zero) {
                    v[r].x = (g0 + off == 0u) ? T(1) : T(0);
                    v[r].y = T(0);
                } else {
                    v[r] = Pb[off];
                }
                if (BWD) w[r] = Lb[off];
            }
        }
    };
    auto direct_store = [&](auto pc) {
        if constexpr (Env::kStore == 1) {
            constexpr int P = decltype(pc)::value;
            const uint32_t g0 = g32(elem_of(t, 0, P, R));
            uint32_t gst[R];
            global_strides(pc, gst);
            C *Pb = env.P + g0;
            C *Lb = BWD ? env.L + g0 : nullptr;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t off = reg_offset(pc, r, gst);
                Pb[off] = v[r];
                if (BWD) Lb[off] = w[r];
            }
        }
    };

    int chunk = -1;
    for (int oi = 0; oi < n_ops; ++oi) {
        const PassOp op = ops[oi];
        if (op.kind == OP_ROUND) {
            const int p = op.chunk;
            if (chunk < 0) {
                if (active) {
                    auto first_round = [&](auto pc) {
                        if constexpr (Env::kLoad == 1) {
                            direct_load(pc);
                        } else if constexpr (Env::kLoad == 2) {
                            constexpr int P = decltype(pc)::value;
                            const uint32_t sb = pad_of<T>(elem_of(t, 0, P, R));
#pragma unroll
                            for (int r = 0; r < NR; ++r) {
                                v[r] = buf[sb + pad_of<T>((uint32_t)r << P)];
                                if (BWD) w[r] = lbuf[sb + pad_of<T>((uint32_t)r << P)];
                            }
                        }
                    };
                    if constexpr (Env::kLoad == 0) {   // plain order: one runtime instance
                        const uint32_t e0 = elem_of(t, 0, p, R);
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            v[r] = buf[e0 + ((uint32_t)r << p)];
                            if (BWD) w[r] = lbuf[e0 + ((uint32_t)r << p)];
                        }
                    } else {
                        with_chunk<R>(p, first_round);
                    }
                }
            } else {
                __syncthreads();
                if (active) {
                    with_chunk<R>(chunk, [&](auto pc) {
                        constexpr int P = decltype(pc)::value;
                        const uint32_t sb = pad_of<T>(elem_of(t, 0, P, R));
                        C *bp = buf + sb;
                        C *lp = BWD ? lbuf + sb : nullptr;
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            bp[pad_of<T>((uint32_t)r << P)] = v[r];
                            if (BWD) lp[pad_of<T>((uint32_t)r << P)] = w[r];
                        }
                    });
                }
                __syncthreads();
                if (active) {
                    with_chunk<R>(p, [&](auto pc) {
                        constexpr int P = decltype(pc)::value;
                        const uint32_t sb = pad_of<T>(elem_of(t, 0, P, R));
                        const C *bp = buf + sb;
                        const C *lp = BWD ? lbuf + sb : nullptr;
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            v[r] = bp[pad_of<T>((uint32_t)r << P)];
                            if (BWD) w[r] = lp[pad_of<T>((uint32_t)r << P)];
                        }
                    });
                }
            }
            chunk = p;
        } else if (op.kind == OP_BF) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (!((op.mask >> j) & 1)) continue;
                const RotCoef<T> rc = env.coef(op.slot, chunk + j);
                const T cv = rc.v;
                if (BWD) {
                    // dE/dtheta = Im<l|Y|p>; per pair Re(conj(l1) p0) - Re(conj(l0) p1)
                    T gt = T(0);
                    if (active) {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r & (1 << j)) continue;
                            const C p0 = v[r], p1 = v[r | (1 << j)];
                            const C l0 = w[r], l1 = w[r | (1 << j)];
                            gt = fma(l1.x, p0.x, gt);
                            gt = fma(l1.y, p0.y, gt);
                            gt = fma(-l0.x, p1.x, gt);
                            gt = fma(-l0.y, p1.y, gt);
                        }
                        // warp sum: FP64, or compensated FP32 pairs (FP64 adds
                        // are scarce on this GPU), then FP64 per warp
                        double dgt;
                        if constexpr (sizeof(T) == 4) {
                            dgt = f32c_value(f32c_warp_sum(F32c{gt * rc.gs, 0.f}, wmask, wlanes));
                        } else {
                            T wgt = gt * rc.gs;
                            for (int o = wlanes >> 1; o > 0; o >>= 1)
                                wgt += __shfl_xor_sync(wmask, wgt, o);
                            dgt = (double)wgt;
                        }
                        if (lane == 0) gsh[(warp * k + chunk + j) * 2 + 0] = dgt;
                    }
                }
                if (!active) continue;
                // FP64: both butterfly forms share one shape once the operands
                // are chosen by the mode: with (P, Q) = (x, y) in tan mode and
                // (y, x) in cot mode,
                //   forward  [[1,-t],[t,1]] / [[u,-1],[1,u]]:
                //     y' = fma(c, P, Q),  x' = s * fma(-c, Q, P)
                //   backward (transposes):
                //     x' = fma(c, Q, P),  y' = s * fma(-c, P, Q)
                // with s = -1 in cot mode (an integer sign flip).  Selecting
                // operands keeps every DFMA useful on the slow FP64 pipe.  FP32
                // branches on the (block-uniform) mode around the whole register
                // loop instead: no selects on the busier integer pipe.
                const uint32_t md = (uint32_t)rc.mode;
                if constexpr (sizeof(T) == 8) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (r & (1 << j)) continue;
                        const int r1 = r | (1 << j);
#pragma unroll
                        for (int bufi = 0; bufi < (BWD ? 2 : 1); ++bufi) {
                            C *u = bufi ? w : v;
                            const C x = u[r], y = u[r1];
                            C P, Q;
                            P.x = md ? y.x : x.x;  P.y = md ? y.y : x.y;
                            Q.x = md ? x.x : y.x;  Q.y = md ? x.y : y.y;
                            if (!BWD) {
                                u[r1].x = fma(cv, P.x, Q.x);
                                u[r1].y = fma(cv, P.y, Q.y);
                                u[r].x = flip_sign(fma(-cv, Q.x, P.x), md);
                                u[r].y = flip_sign(fma(-cv, Q.y, P.y), md);
                            } else {
                                u[r].x = fma(cv, Q.x, P.x);
                                u[r].y = fma(cv, Q.y, P.y);
                                u[r1].x = flip_sign(fma(-cv, P.x, Q.x), md);
                                u[r1].y = flip_sign(fma(-cv, P.y, Q.y), md);
                            }
                        }
                    }
                } else if (md == 0) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (r & (1 << j)) continue;
                        const int r1 = r | (1 << j);
#pragma unroll
                        for (int bufi = 0; bufi < (BWD ? 2 : 1); ++bufi) {
                            C *u = bufi ? w : v;
                            const C x = u[r], y = u[r1];
                            if (!BWD) {   // [[1,-t],[t,1]]
                                u[r].x = fma(-cv, y.x, x.x);  u[r].y = fma(-cv, y.y, x.y);
                                u[r1].x = fma(cv, x.x, y.x);  u[r1].y = fma(cv, x.y, y.y);
                            } else {      // transpose: [[1,t],[-t,1]], packed f32x2
                                u[r] = caxpy(cv, y, x);
                                u[r1] = caxpy(-cv, x, y);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (r & (1 << j)) continue;
                        const int r1 = r | (1 << j);
#pragma unroll
                        for (int bufi = 0; bufi < (BWD ? 2 : 1); ++bufi) {
                            C *u = bufi ? w : v;
                            const C x = u[r], y = u[r1];
                            if (!BWD) {   // [[u,-1],[1,u]]
                                u[r].x = fma(cv, x.x, -y.x);  u[r].y = fma(cv, x.y, -y.y);
                                u[r1].x = fma(cv, y.x, x.x);  u[r1].y = fma(cv, y.y, x.y);
                            } else {      // transpose: [[u,1],[-1,u]]
                                u[r] = caxpy(cv, x, y);
                                // u y - x as two scalar FMAs (a negated addend is
                                // free there, not in the packed form)
                                u[r1].x = fma(cv, y.x, -x.x);
                                u[r1].y = fma(cv, y.y, -x.y);
                            }
                        }
                    }
                }
            }
        } else if (op.kind == OP_DIAG) {
            const uint32_t cz = d.slot_czmask[op.slot];
            if (BWD && active) {
                // dE/dphi_q = Im<l|Z_q|p> = sum_i u_i (-1)^{bit_q(i)}, u = Im(conj(l) p),
                // for every gated bit q of the slot, taken before the diagonal is
                // undone (where the buffers hold the exact states).
                T u[NR];
                T tot = T(0);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    u[r] = fma(w[r].x, v[r].y, -w[r].y * v[r].x);
                    tot += u[r];
                }
                const uint32_t gated = d.slot_gated[op.slot];
                const uint32_t e0 = elem_of(t, 0, chunk, R);
                for (int q = 0; q < k; ++q) {
                    if (!((gated >> q) & 1u)) continue;
                    T gq;
                    if (q >= chunk && q < chunk + R) {
                        gq = T(0);
#pragma unroll
                        for (int r = 0; r < NR; ++r) gq += ((r >> (q - chunk)) & 1) ? -u[r] : u[r];
                    } else {
                        gq = ((e0 >> q) & 1u) ? -tot : tot;
                    }
                    double dg;
                    if constexpr (sizeof(T) == 4) {
                        dg = f32c_value(f32c_warp_sum(F32c{gq, 0.f}, wmask, wlanes));
                    } else {
                        for (int o = wlanes >> 1; o > 0; o >>= 1) gq += __shfl_xor_sync(wmask, gq, o);
                        dg = (double)gq;
                    }
                    if (lane == 0) gsh[(warp * k + q) * 2 + 1] = dg;
                }
            }
            if (active) {
                // compile-time chunk (constant register offsets) only where the
                // diagonal is read as full table rows; else one runtime instance
                auto diag_body = [&](auto pc) {
                    const int P = pc.value;
                    const uint32_t e0 = elem_of(t, 0, P, R);
                    const uint32_t g0 = g32(e0);
                    // CZ signs of all NR registers as one mask (bit r = register r).
                    // Register r holds global index g = g0 ^ L_r, L_r the global
                    // image of r << P, and the CZ chain sign is Q(g) =
                    // parity(g & (g >> 1) & cz).  Q is quadratic over GF(2):
                    //   Q(g0 ^ L) = Q(g0) ^ Q(L) ^ parity(L & W),
                    //   W = ((g0 & cz) << 1) ^ ((g0 >> 1) & cz),
                    // where parity(L_r & W) is linear in the bits of r (the bits of
                    // W at the chunk's global positions) and Q(L_r) comes from the
                    // CZ pairs that join two adjacent bits of the chunk.
                    uint32_t sm;
                    {
                        constexpr uint32_t kFull = NR >= 32 ? 0xffffffffu : ((1u << NR) - 1u);
                        const uint32_t W = ((g0 & cz) << 1) ^ ((g0 >> 1) & cz);
                        const int lo_cnt = min(max(m - P, 0), R);
                        uint32_t wv = (W >> P) & ((1u << lo_cnt) - 1u);
                        if (lo_cnt < R)
                            wv |= ((W >> (a + max(P - m, 0))) & ((1u << (R - lo_cnt)) - 1u)) << lo_cnt;
                        // tile bits b whose qubits b, b+1 are adjacent and CZ-coupled
                        uint32_t czt = 0u;
                        if (m >= 1) {
                            czt = cz & ((1u << (m - 1)) - 1u);
                            if (a == m && k > m) czt |= cz & (1u << (m - 1));
                        }
                        if (k - m >= 2) czt |= ((cz >> a) & ((1u << (k - m - 1)) - 1u)) << m;
                        const uint32_t adj = czt >> P;
                        sm = (__popc(g0 & (g0 >> 1) & cz) & 1u) ? kFull : 0u;
    #pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if ((wv >> j) & 1u) sm ^= reg_bit_table(j);
                            if (j + 1 < R && ((adj >> j) & 1u)) sm ^= reg_bit_table(j) & reg_bit_table(j + 1);
                        }
                        sm &= kFull;
                    }
                        // diagonal entries e0 + (r << P): with a full table, one row
                    // pointer and constant offsets
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const uint32_t sgn = (sm >> r) & 1u;
                        C dv;
                        if constexpr (Env::kDiagRow) dv = env.diag_row(op.slot, e0)[(uint32_t)r << P];
                        else dv = env.diag(op.slot, e0 + ((uint32_t)r << P));
                        if (!BWD) {
                            C y = cmul(v[r], dv);
                            y.x = flip_sign(y.x, sgn);
                            y.y = flip_sign(y.y, sgn);
                            v[r] = y;
                        } else {
                            C y = cmul_conj(v[r], dv);
                            y.x = flip_sign(y.x, sgn);
                            y.y = flip_sign(y.y, sgn);
                            v[r] = y;
                            C z = cmul_conj(w[r], dv);
                            z.x = flip_sign(z.x, sgn);
                            z.y = flip_sign(z.y, sgn);
                            w[r] = z;
                        }
                    }
                };
                if constexpr (Env::kDiagRow) with_chunk<R>(chunk, diag_body);
                else diag_body(RtChunk{chunk});
            }
        } else if (BWD && op.kind == OP_FLUSH) {
            __syncthreads();
            const uint32_t gated = d.slot_gated[op.slot];
            const int used_warps = (int)((nthr + 31) >> 5);
            if (threadIdx.x == 0) {
                for (int idx = 0; idx < 2 * k; ++idx) {
                    if (!((gated >> (idx >> 1)) & 1u)) continue;
                    double s = 0.0;
                    for (int wi = 0; wi < used_warps; ++wi) s += gsh[wi * 2 * k + idx];
                    env.grad(op.slot, idx >> 1, idx & 1, s);
                }
            }
            __syncthreads();
        }
    }
    if constexpr (Env::kStore == 1) {
        if (active) with_chunk<R>(chunk, [&](auto pc) { direct_store(pc); });
    } else {
        // back to plain order in shared memory
        __syncthreads();
        if (active) {
            const uint32_t e0 = elem_of(t, 0, chunk, R);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                buf[e0 + ((uint32_t)r << chunk)] = v[r];
                if (BWD) lbuf[e0 + ((uint32_t)r << chunk)] = w[r];
            }
        }
        __syncthreads();
    }
    (void)nwarps;
}

// ---------------------------------------------------------------- fixed programs
//
// The forward pass programs of the default plans come in a handful of shapes:
// the same sequence of op kinds and round chunks, differing only in masks and
// slots.  For a known shape (the template pack, one code per op) the program
// runs fully unrolled: every chunk is a compile-time constant, the op list is
// read at constant indices, and no value has to return to a fixed register
// at an interpreter back-edge.  Forward only, for environments that read and
// write the state directly (kLoad == 1, kStore == 1) with full diagonal rows.

constexpr int prog_round(int chunk) { return 256 | chunk; }
constexpr int kProgBF = 512, kProgDiag = 768, kProgFlush = 1024;

template <int I>
struct IdxC {
    static constexpr int value = I;
};

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(IdxC<I>{});
        static_for<I + 1, N>(f);
    }
}

// Chunk of the round in effect at op i of the program (-1 before the first).
template <int... Codes>
__host__ __device__ constexpr int prog_chunk_at(int i) {
    constexpr int code[] = {Codes...};
    for (int j = i; j >= 0; --j)
        if ((code[j] >> 8) == 1) return code[j] & 255;
    return -1;
}

// Largest round chunk of a program: the tile has this many bits plus R.
template <int... Codes>
__host__ __device__ constexpr int prog_top_chunk() {
    constexpr int code[] = {Codes...};
    int top = 0;
    for (int c : code)
        if ((c >> 8) == 1 && (c & 255) > top) top = c & 255;
    return top;
}

template <typename T, int R, bool BWD, class Env, int... Codes>
__device__ __forceinline__ void run_tile_fixed(const PassDesc &d, const PassOp *ops, uint64_t gbase,
                                               typename V2<T>::type *buf,
                                               typename V2<T>::type *lbuf, double *gsh,
                                               Env &env) {
    static_assert(Env::kLoad == 1 && Env::kStore == 1 && Env::kDiagRow, "direct environment");
    static_assert(!(BWD && sizeof(T) == 8) || R == 3, "FP64 gradient rows are sized for R = 3");
    static_assert(!(BWD && sizeof(T) == 4) || R == 4, "FP32 gradient rows are sized for R = 4");
    using C = typename V2<T>::type;
    constexpr int NR = 1 << R;
    constexpr int N = sizeof...(Codes);
    constexpr int code[] = {Codes...};
    const int k = d.k, m = d.m, a = d.a;
    const uint32_t t = threadIdx.x;
    const uint32_t nthr = 1u << (k - R);   // == blockDim.x for these kernels
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lowmask = (1u << m) - 1u;
    auto g32 = [&](uint32_t e) -> uint32_t {
        return (uint32_t)(gbase | (uint64_t)(e & lowmask) | ((uint64_t)(e >> m) << a));
    };
    // global strides of the R register bits of chunk P, and register offsets
    auto strides = [&](auto pc, uint32_t (&gst)[R]) {
        constexpr int P = decltype(pc)::value;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int bt = P + j;
            gst[j] = bt < m ? (1u << bt) : (1u << (a + bt - m));
        }
    };
    auto offset = [&](auto pc, int r, const uint32_t (&gst)[R]) -> uint32_t {
        constexpr int P = decltype(pc)::value;
        uint32_t off = 0;
#pragma unroll
        for (int j = 0; j < R; ++j)
            if ((r >> j) & 1) off += (P + R <= m) ? (1u << (P + j)) : gst[j];
        return off;
    };
    C v[NR];
    C w[NR];
    int diag_chunk = 0;   // chunk of the last diagonal op (backward flush)
    static_for<0, N>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int kind = code[i] >> 8;
        constexpr int P = prog_chunk_at<Codes...>(i);
        using PC = ChunkC<P < 0 ? 0 : P>;
        if constexpr (kind == 1 && i == 0) {   // first round: load from global memory
            const uint32_t g0 = g32(elem_of(t, 0, P, R));
            uint32_t gst[R];
            strides(PC{}, gst);
            const C *Pb = env.P + g0;
            const C *Lb = BWD ? env.L + g0 : nullptr;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t off = offset(PC{}, r, gst);
                if (env.init_zero) {
                    v[r].x = (g0 + off == 0u) ? T(1) : T(0);
                    v[r].y = T(0);
                } else {
                    v[r] = Pb[off];
                }
                if (BWD) w[r] = Lb[off];
            }
        } else if constexpr (kind == 1) {       // round change through shared memory
            constexpr int PO = prog_chunk_at<Codes...>(i - 1);
            __syncthreads();
            {
                C *bp = buf + pad_of<T>(elem_of(t, 0, PO, R));
                C *lp = BWD ? lbuf + pad_of<T>(elem_of(t, 0, PO, R)) : nullptr;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    bp[pad_of<T>((uint32_t)r << PO)] = v[r];
                    if (BWD) lp[pad_of<T>((uint32_t)r << PO)] = w[r];
                }
            }
            __syncthreads();
            {
                const C *bp = buf + pad_of<T>(elem_of(t, 0, P, R));
                const C *lp = BWD ? lbuf + pad_of<T>(elem_of(t, 0, P, R)) : nullptr;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    v[r] = bp[pad_of<T>((uint32_t)r << P)];
                    if (BWD) w[r] = lp[pad_of<T>((uint32_t)r << P)];
                }
            }
        } else if constexpr (kind == 2) {       // RY butterflies of the chunk's gated bits
            const PassOp op = ops[i];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (!((op.mask >> j) & 1)) continue;
                const RotCoef<T> rc = env.coef(op.slot, P + j);
                const T cv = rc.v;
                const uint32_t md = (uint32_t)rc.mode;
                if constexpr (BWD) {
                    // dE/dtheta = Im<l|Y|p>; per pair Re(conj(l1) p0) - Re(conj(l0) p1)
                    T gt = T(0);
                    if constexpr (sizeof(T) == 4) {
                        // packed: both components in f32x2 accumulators, the two
                        // orientations apart (no negation per pair)
                        float2 gp = make_float2(0.f, 0.f), gn = make_float2(0.f, 0.f);
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r & (1 << j)) continue;
                            gp = __ffma2_rn(w[r | (1 << j)], v[r], gp);
                            gn = __ffma2_rn(w[r], v[r | (1 << j)], gn);
                        }
                        gt = (gp.x + gp.y) - (gn.x + gn.y);
                    } else {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r & (1 << j)) continue;
                            const C p0 = v[r], p1 = v[r | (1 << j)];
                            const C l0 = w[r], l1 = w[r | (1 << j)];
                            gt = fma(l1.x, p0.x, gt);
                            gt = fma(l1.y, p0.y, gt);
                            gt = fma(-l0.x, p1.x, gt);
                            gt = fma(-l0.y, p1.y, gt);
                        }
                    }
                    if constexpr (sizeof(T) == 4) {
                        // FP32: row P + j, already scaled by gs, summed at the flush
                        reinterpret_cast<float *>(gsh)[(P + j) * nthr + t] = gt * rc.gs;
                    } else {
                        // FP64: row P + j of per-thread partials, summed (and scaled by gs)
                        // at the flush: no shuffle tree per bit on the scarce FP64 pipe
                        gsh[(P + j) * nthr + t] = gt;
                    }
                }
#pragma unroll
                for (int bufi = 0; bufi < (BWD ? 2 : 1); ++bufi) {
                    C *u = bufi ? w : v;
                    if constexpr (sizeof(T) == 8) {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r & (1 << j)) continue;
                            const int r1 = r | (1 << j);
                            const C x = u[r], y = u[r1];
                            C Pp, Q;
                            Pp.x = md ? y.x : x.x;  Pp.y = md ? y.y : x.y;
                            Q.x = md ? x.x : y.x;   Q.y = md ? x.y : y.y;
                            if (!BWD) {
                                u[r1].x = fma(cv, Pp.x, Q.x);
                                u[r1].y = fma(cv, Pp.y, Q.y);
                                u[r].x = flip_sign(fma(-cv, Q.x, Pp.x), md);
                                u[r].y = flip_sign(fma(-cv, Q.y, Pp.y), md);
                            } else {
                                u[r].x = fma(cv, Q.x, Pp.x);
                                u[r].y = fma(cv, Q.y, Pp.y);
                                u[r1].x = flip_sign(fma(-cv, Pp.x, Q.x), md);
                                u[r1].y = flip_sign(fma(-cv, Pp.y, Q.y), md);
                            }
                        }
                    } else if (md == 0) {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r & (1 << j)) continue;
                            const int r1 = r | (1 << j);
                            const C x = u[r], y = u[r1];
                            if (!BWD) {   // [[1,-t],[t,1]]
                                u[r].x = fma(-cv, y.x, x.x);  u[r].y = fma(-cv, y.y, x.y);
                                u[r1].x = fma(cv, x.x, y.x);  u[r1].y = fma(cv, x.y, y.y);
                            } else {      // transpose: [[1,t],[-t,1]], packed f32x2
                                u[r] = caxpy(cv, y, x);
                                u[r1] = caxpy(-cv, x, y);
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r & (1 << j)) continue;
                            const int r1 = r | (1 << j);
                            const C x = u[r], y = u[r1];
                            if (!BWD) {   // [[u,-1],[1,u]]
                                u[r].x = fma(cv, x.x, -y.x);  u[r].y = fma(cv, x.y, -y.y);
                                u[r1].x = fma(cv, y.x, x.x);  u[r1].y = fma(cv, y.y, x.y);
                            } else {      // transpose: [[u,1],[-1,u]]
                                u[r] = caxpy(cv, x, y);
                                // u y - x as two scalar FMAs (a negated addend is
                                // free there, not in the packed form)
                                u[r1].x = fma(cv, y.x, -x.x);
                                u[r1].y = fma(cv, y.y, -x.y);
                            }
                        }
                    }
                }
            }
        } else if constexpr (kind == 3) {       // RZ phases, scales and CZ signs
            const PassOp op = ops[i];
            const uint32_t cz = d.slot_czmask[op.slot];
            const uint32_t e0 = elem_of(t, 0, P, R);
            if constexpr (BWD) {
                // dE/dphi_q = Im<l|Z_q|p> = sum_i u_i (-1)^{bit_q(i)}, u = Im(conj(l) p),
                // taken before the diagonal is undone.  Each thread stores its
                // total (row k) and its signed sums over the chunk's own bits
                // (rows k + 1 + j); the flush sums the rows, taking the sign of a
                // bit outside the chunk from the thread's element base.  The
                // total and the R signed sums come from one butterfly over the
                // register bits (level j pairs the partial sums that differ in
                // bit j): 2^(R+1) + R - 4 adds instead of (R + 1) 2^R.
                T a[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) a[r] = fma(w[r].x, v[r].y, -w[r].y * v[r].x);
                const uint32_t gated = d.slot_gated[op.slot];
                T *rows = reinterpret_cast<T *>(gsh);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    constexpr int kHalfMax = NR / 2;
                    const int half = NR >> (j + 1);
                    T dsum = T(0);
#pragma unroll
                    for (int c = 0; c < kHalfMax; ++c) {
                        if (c >= half) break;
                        const T x0 = a[2 * c], x1 = a[2 * c + 1];
                        dsum = c == 0 ? x0 - x1 : dsum + (x0 - x1);
                        a[c] = x0 + x1;
                    }
                    if ((gated >> (P + j)) & 1u) rows[(k + 1 + j) * nthr + t] = dsum;
                }
                rows[k * nthr + t] = a[0];
                diag_chunk = P;
            }
            const uint32_t g0 = g32(e0);
            // CZ signs of the NR registers as one mask (see run_tile)
            constexpr uint32_t kFull = NR >= 32 ? 0xffffffffu : ((1u << NR) - 1u);
            const uint32_t W = ((g0 & cz) << 1) ^ ((g0 >> 1) & cz);
            const int lo_cnt = min(max(m - P, 0), R);
            uint32_t wv = (W >> P) & ((1u << lo_cnt) - 1u);
            if (lo_cnt < R) wv |= ((W >> (a + max(P - m, 0))) & ((1u << (R - lo_cnt)) - 1u)) << lo_cnt;
            uint32_t czt = 0u;
            if (m >= 1) {
                czt = cz & ((1u << (m - 1)) - 1u);
                if (a == m && k > m) czt |= cz & (1u << (m - 1));
            }
            if (k - m >= 2) czt |= ((cz >> a) & ((1u << (k - m - 1)) - 1u)) << m;
            const uint32_t adj = czt >> P;
            uint32_t sm = (__popc(g0 & (g0 >> 1) & cz) & 1u) ? kFull : 0u;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if ((wv >> j) & 1u) sm ^= reg_bit_table(j);
                if (j + 1 < R && ((adj >> j) & 1u)) sm ^= reg_bit_table(j) & reg_bit_table(j + 1);
            }
            sm &= kFull;
            const C *drow = env.diag_row(op.slot, e0);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t sgn = (sm >> r) & 1u;
                const C dv = drow[(uint32_t)r << P];
                C y = BWD ? cmul_conj(v[r], dv) : cmul(v[r], dv);
                y.x = flip_sign(y.x, sgn);
                y.y = flip_sign(y.y, sgn);
                v[r] = y;
                if (BWD) {
                    C z = cmul_conj(w[r], dv);
                    z.x = flip_sign(z.x, sgn);
                    z.y = flip_sign(z.y, sgn);
                    w[r] = z;
                }
            }
        } else if constexpr (kind == 4) {       // block totals of a slot's gradient partials
            // The tile shape is fixed by the program: k = top chunk + R bits,
            // NT = 2^(k - R) threads, NW warps.  Two stages, both in a fixed
            // order (bitwise reproducible):
            //  1. warp w takes rows w, w + NW, ... (RPW of them); each lane adds
            //     its strided part of each row (NT / 32 values);
            //  2. the lane partials go to shared memory (the psi tile buffer,
            //     row stride 33: the lanes of stage 2 read different banks) and
            //     lane r of warp 0 adds the 32 partials of row r, all rows at
            //     once, in place of a shuffle tree per row (5 adds per lane and
            //     row, with lanes that carry no needed value).
            // Rows: 2q = theta of tile bit q, 2q + 1 = phi of bit q (from the
            // chunk rows, or from the total row with the sign of the element's
            // bit q); 2k <= 28 rows fit the lanes of one warp.
            constexpr int KT = prog_top_chunk<Codes...>() + R;
            constexpr int NT = 1 << (KT - R);
            constexpr int NW = NT / 32;
            [[maybe_unused]] constexpr int RPW = (2 * KT + NW - 1) / NW;
            static_assert(NT >= 32, "fixed programs run whole warps");
            static_assert(2 * KT <= 32, "one lane per row in the second stage");
            if constexpr (BWD) {
                using A = typename std::conditional<sizeof(T) == 4, F32c, double>::type;
                // stage-2 partials go to the psi tile buffer, free between rounds
                // (the tile is in registers; the next round exchange starts
                // with a barrier): 2 KT rows of 33
                static_assert(2 * KT * 33 * sizeof(A) <= (1u << KT) * sizeof(typename V2<T>::type),
                              "partials fit the tile buffer");
                const PassOp op = ops[i];
                __syncthreads();
                const uint32_t gated = d.slot_gated[op.slot];
                const int dp = diag_chunk;
                const T *rows = reinterpret_cast<const T *>(gsh);
                A *sp2 = reinterpret_cast<A *>(buf);
                auto stage1 = [&](int r) {
                    const int idx = warp + r * NW;
                    const int q = idx >> 1, comp = idx & 1;
                    if (idx < 2 * KT && ((gated >> q) & 1u)) {
                        const bool in_chunk = q >= dp && q < dp + R;
                        const T *src = rows + (comp == 0 ? q : (in_chunk ? k + 1 + q - dp : k)) * NT;
                        const bool signed_total = comp == 1 && !in_chunk;
                        auto term = [&](uint32_t tt) {
                            const T v = src[tt];
                            return signed_total ? flip_sign(v, (elem_of(tt, 0, dp, R) >> q) & 1u) : v;
                        };
                        A part;
                        if constexpr (sizeof(T) == 4) {
                            part = F32c{term(lane), 0.f};
#pragma unroll
                            for (int c = 1; c < NT / 32; ++c) f32c_add(part, term(lane + 32 * c));
                        } else {
                            part = term(lane);
#pragma unroll
                            for (int c = 1; c < NT / 32; ++c) part += term(lane + 32 * c);
                        }
                        sp2[idx * 33 + lane] = part;
                    }
                };
                if constexpr (sizeof(T) == 4) {
                    // one row at a time (its NT / 32 loads together): the
                    // tile's registers stay live across the flush
#pragma unroll 1
                    for (int r = 0; r < RPW; ++r) stage1(r);
                } else {
#pragma unroll
                    for (int r = 0; r < RPW; ++r) stage1(r);
                }
                __syncthreads();
                if (warp == 0) {
                    const int idx = lane, q = idx >> 1, comp = idx & 1;
                    if (idx < 2 * KT && ((gated >> q) & 1u)) {
                        // four interleaved chains (lanes l = m mod 4), then
                        // (0 + 1) + (2 + 3): a fixed order, a quarter of the latency
                        const A *row = sp2 + idx * 33;
                        A ch[4] = {row[0], row[1], row[2], row[3]};
#pragma unroll
                        for (int l = 4; l < 32; l += 4) {
#pragma unroll
                            for (int m = 0; m < 4; ++m) {
                                if constexpr (sizeof(T) == 4) ch[m] = f32c_add_lazy(ch[m], row[l + m]);
                                else ch[m] += row[l + m];
                            }
                        }
                        A tot;
                        if constexpr (sizeof(T) == 4)
                            tot = f32c_add_lazy(f32c_add_lazy(ch[0], ch[1]), f32c_add_lazy(ch[2], ch[3]));
                        else
                            tot = (ch[0] + ch[1]) + (ch[2] + ch[3]);
                        if constexpr (sizeof(T) == 4) {
                            // theta rows came scaled by gs
                            env.grad(op.slot, q, comp, f32c_value(tot));
                        } else {
                            env.grad(op.slot, q, comp, comp == 0 ? tot * (double)env.coef(op.slot, q).gs : tot);
                        }
                    }
                }
                __syncthreads();
            }
        }
    });
    {   // last round: store to global memory
        constexpr int P = prog_chunk_at<Codes...>(N - 1);
        using PC = ChunkC<P>;
        const uint32_t g0 = g32(elem_of(t, 0, P, R));
        uint32_t gst[R];
        strides(PC{}, gst);
        C *Pb = env.P + g0;
        C *Lb = BWD ? env.L + g0 : nullptr;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const uint32_t off = offset(PC{}, r, gst);
            Pb[off] = v[r];
            if (BWD) Lb[off] = w[r];
        }
    }
}

}  // namespace vqe
