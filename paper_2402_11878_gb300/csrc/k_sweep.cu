// lambda = H psi by bit-ordered sweeps over the state (Sec. II-B, Eqs. 2-4
// and 7: the adjoint gradient needs lambda = H psi, and <psi|lambda> is the
// energy).  The layout and the pattern form of the terms are described with
// SweepDesc in vqe_internal.h.
//
// Blocks take chunks of kSweepChunk consecutive counter values from a
// per-state atomic counter, in increasing order, so the states in flight
// span a few blocks of the sweep's fast bits whatever the blocks' relative
// speed: a block's amplitudes come from DRAM once and the gathers
// psi_{i^x} of its groups are served by L2.  lambda accumulates in
// registers over the sweep's groups and is written once per sweep (read
// back by the next sweep).  <psi|lambda> and <psi|psi> are summed per chunk
// (FP64 per thread in the FP64 kernel, compensated FP32 (csum.cuh) in the
// complex64 kernel, then a fixed-order block tree) and the chunk partials
// in chunk order: bitwise reproducible although chunks go to blocks in
// varying order.
#include <algorithm>

#include "csum.cuh"
#include "vqe_internal.h"

namespace vqe {
namespace {

template <typename T> struct SV2;
template <> struct SV2<float> { using type = float2; };
template <> struct SV2<double> { using type = double2; };

__device__ __forceinline__ double sw_sign(double v, uint32_t s) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)s << 63));
}
__device__ __forceinline__ float sw_sign(float v, uint32_t s) {
    return __int_as_float(__float_as_int(v) ^ (int)(s << 31));
}

__device__ __forceinline__ bool nonzero(double v) { return (__double_as_longlong(v) << 1) != 0; }
__device__ __forceinline__ bool nonzero(float v) { return (__float_as_uint(v) << 1) != 0u; }

__device__ __forceinline__ void sweep_block_sum(double &a, double &b, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[2 * warp] = a;
        sh[2 * warp + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sa += sh[2 * w];
            sb += sh[2 * w + 1];
        }
        a = sa;
        b = sb;
    }
}

__device__ __forceinline__ void sweep_block_sum_c(F32c a, F32c b, float *sh, double &ra, double &rb) {
    a = f32c_warp_sum(a, 0xffffffffu, 32);
    b = f32c_warp_sum(b, 0xffffffffu, 32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[4 * warp] = a.hi;
        sh[4 * warp + 1] = a.lo;
        sh[4 * warp + 2] = b.hi;
        sh[4 * warp + 3] = b.lo;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        a = lane < nw ? F32c{sh[4 * lane], sh[4 * lane + 1]} : f32c_zero();
        b = lane < nw ? F32c{sh[4 * lane + 2], sh[4 * lane + 3]} : f32c_zero();
        a = f32c_warp_sum(a, 0xffffffffu, 32);
        b = f32c_warp_sum(b, 0xffffffffu, 32);
        ra = f32c_value(a);
        rb = f32c_value(b);
    }
}

// FP64: three blocks of 256 threads per SM (<= 85 registers), FP32 four.
template <typename T>
__global__ void __launch_bounds__(kSweepThreads, sizeof(T) == 8 ? 3 : 4)
k_apply_h_sweep(SweepDesc W, const uint32_t *__restrict__ order, const SGroup *__restrict__ groups,
                const uint32_t *__restrict__ pat, const uint32_t *__restrict__ tz,
                const T *__restrict__ ca, const T *__restrict__ cb, const T *__restrict__ hdiag,
                int n, const typename SV2<T>::type *__restrict__ psi,
                typename SV2<T>::type *__restrict__ lam, size_t stride, int first, int last,
                unsigned long long *__restrict__ ctr, double *__restrict__ cpart) {
    using C = typename SV2<T>::type;
    constexpr int J = kSweepJ;
    constexpr uint32_t kIter = kSweepThreads * J;   // counter values per block iteration
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(sizeof(SGroup) == 16, "a sweep group is one 16-byte shared-memory load");
    const int ng = W.g_end - W.g_begin;
    uint32_t *sord = reinterpret_cast<uint32_t *>(smem_raw);       // [1024] bit-order bytes
    SGroup *sg = reinterpret_cast<SGroup *>(sord + 1024);            // [ng], 16-byte aligned
    T *sca = reinterpret_cast<T *>(sg + ng);                         // [t_count]
    T *scb = sca + W.t_count;                                        // [t_count]
    uint32_t *sz = reinterpret_cast<uint32_t *>(scb + W.t_count);    // [t_count]
    uint32_t *spat = sz + W.t_count;                                 // [n_pat]
    __shared__ double sh[2 * (kSweepThreads / 32)];
    __shared__ unsigned long long chunk_sh;

    for (int i = threadIdx.x; i < 1024; i += blockDim.x) sord[i] = order[i];
    for (int i = threadIdx.x; i < W.t_count; i += blockDim.x) {
        sca[i] = ca[W.t_begin + i];
        scb[i] = cb[W.t_begin + i];
        sz[i] = tz[W.t_begin + i];
    }
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(groups + W.g_begin);
        uint32_t *dst = reinterpret_cast<uint32_t *>(sg);
        for (int i = threadIdx.x; i < ng * (int)(sizeof(SGroup) / 4); i += blockDim.x) dst[i] = src[i];
    }
    for (int i = threadIdx.x; i < W.n_pat; i += blockDim.x) spat[i] = pat[W.p_begin + i];

    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    C *L = lam + (size_t)b * stride;
    const uint64_t dim = 1ull << n;
    const uint64_t nchunks = (dim + kSweepChunk - 1) / kSweepChunk;
    const bool with_diag = W.diag && hdiag != nullptr;
    // Chunks of kSweepChunk counter values are taken in increasing order
    // from a per-state counter: the chunks in flight are always the latest
    // ones handed out, whatever the relative speed of the blocks, so the
    // states being processed stay within a few blocks of the fast bits.
    for (;;) {
        __syncthreads();   // tables staged; the previous chunk's reads of chunk_sh done
        if (threadIdx.x == 0) chunk_sh = atomicAdd(ctr + b, 1ull);
        __syncthreads();
        const uint64_t chunk = chunk_sh;
        if (chunk >= nchunks) break;
        double dacc = 0.0, dnrm = 0.0;
        F32c facc = f32c_zero(), fnrm = f32c_zero();
        for (uint32_t it = 0; it < kSweepChunk / kIter; ++it) {
            const uint64_t s0 = chunk * kSweepChunk + (uint64_t)it * kIter + threadIdx.x;
            uint32_t a[J];
            bool ok[J];
            C lv[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const uint64_t s = s0 + (uint64_t)j * kSweepThreads;
                ok[j] = s < dim;
                const uint32_t ss = (uint32_t)(ok[j] ? s : 0u);
                a[j] = sord[ss & 255u] | sord[256 + ((ss >> 8) & 255u)] |
                       sord[512 + ((ss >> 16) & 255u)] | sord[768 + (ss >> 24)];
            }
#pragma unroll
            for (int j = 0; j < J; ++j) lv[j] = first ? C{T(0), T(0)} : L[a[j]];
            if (with_diag) {
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const C p = P[a[j]];
                    const T dv = __ldg(hdiag + a[j]);
                    lv[j].x = fma(p.x, dv, lv[j].x);
                    lv[j].y = fma(p.y, dv, lv[j].y);
                }
            }
            for (int g = 0; g < ng; ++g) {
                const uint4 gw = reinterpret_cast<const uint4 *>(sg)[g];
                const uint32_t x = gw.x, xbits = gw.z, flags = gw.w;
                const uint32_t nxb = flags & 255u;
                const bool has_b = (flags >> 8) & 1u, multi = (flags >> 9) & 1u;
                T fa[J], fb[J];
                bool nz[J];
                if ((flags >> 10) & 1u) {
                    // parity form: one term, taken where popc(i & x) has parity p
                    const uint32_t pk = (flags >> 11) & 1u;
                    const uint32_t t = (uint32_t)gw.y;
                    const uint32_t z = sz[t];
                    const T c_a = sca[t];
                    const T c_b = has_b ? scb[t] : T(0);
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        nz[j] = ((__popc(a[j] & x) ^ pk) & 1u) == 0u;
                        const uint32_t par = __popc(a[j] & z) & 1u;
                        fa[j] = sw_sign(c_a, par);
                        fb[j] = sw_sign(c_b, par);
                    }
                } else {
                    // pattern of each state at the group's X bits (group-uniform
                    // branch on their number; pattern bit 1 taken with one shift
                    // since the X bits are increasing)
                    uint32_t pv[J];
                    const uint32_t s0b = xbits & 31u, s1b = ((xbits >> 5) & 31u) - 1u;
                    if (nxb == 2u) {
#pragma unroll
                        for (int j = 0; j < J; ++j) pv[j] = ((a[j] >> s0b) & 1u) | ((a[j] >> s1b) & 2u);
                    } else if (nxb == 1u) {
#pragma unroll
                        for (int j = 0; j < J; ++j) pv[j] = (a[j] >> s0b) & 1u;
                    } else if (nxb == 0u) {
#pragma unroll
                        for (int j = 0; j < J; ++j) pv[j] = 0u;
                    } else {
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            uint32_t v = 0u;
                            for (uint32_t k = 0; k < nxb; ++k) v |= ((a[j] >> ((xbits >> (5 * k)) & 31u)) & 1u) << k;
                            pv[j] = v;
                        }
                    }
                    if (!multi) {
                        // the pattern's term slot (a zero term for an empty pattern)
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const uint32_t t = (uint32_t)gw.y + pv[j];
                            const uint32_t par = __popc(a[j] & sz[t]) & 1u;
                            const T c_a = sca[t];
                            const T c_b = has_b ? scb[t] : T(0);
                            nz[j] = nonzero(c_a) || nonzero(c_b);   // integer test, off the FP64 pipe
                            fa[j] = sw_sign(c_a, par);
                            fb[j] = sw_sign(c_b, par);
                        }
                    } else {
                        const uint32_t *gp = spat + gw.y;
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const uint32_t e = gp[pv[j]];
                            const uint32_t r0 = e & 0xffffu, cnt = e >> 16;
                            nz[j] = cnt != 0u;
                            fa[j] = T(0);
                            fb[j] = T(0);
                            for (uint32_t r = r0; r < r0 + cnt; ++r) {
                                const uint32_t pr = __popc(a[j] & sz[r]) & 1u;
                                fa[j] += sw_sign(sca[r], pr);
                                if (has_b) fb[j] += sw_sign(scb[r], pr);
                            }
                        }
                    }
                }
                if constexpr (sizeof(T) == 8) {
                    // FP64 (bound by the FP64 pipe): the gather and the
                    // multiply-adds of a state inside a warp-uniform branch.
                    // The patterns of X bits above the lanes' bits are
                    // warp-uniform, so warps of the zero half of such a group
                    // skip their DFMAs (24 qubits: 49 DFMA per state in a
                    // 34-group sweep, 64.8 when the gathers were issued
                    // before the vote and the compiler made it a select).
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        if (__any_sync(0xffffffffu, nz[j])) {
                            const C pj = nz[j] ? P[a[j] ^ x] : C{T(0), T(0)};
                            if (has_b) {
                                lv[j].x = fma(pj.x, fa[j], fma(pj.y, fb[j], lv[j].x));
                                lv[j].y = fma(pj.y, fa[j], fma(-pj.x, fb[j], lv[j].y));
                            } else {
                                lv[j].x = fma(pj.x, fa[j], lv[j].x);
                                lv[j].y = fma(pj.y, fa[j], lv[j].y);
                            }
                        }
                    }
                } else {
                    C p[J];
#pragma unroll
                    for (int j = 0; j < J; ++j) p[j] = nz[j] ? P[a[j] ^ x] : C{T(0), T(0)};
                    // complex64 (issue-bound): the gathers of the J states
                    // issued together, the multiply-adds after a warp vote
                    // (which the compiler may turn into a select)
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        if (!__any_sync(0xffffffffu, nz[j])) continue;
                        if (has_b) {
                            // (px + i py)(fa - i fb)
                            lv[j].x = fma(p[j].x, fa[j], fma(p[j].y, fb[j], lv[j].x));
                            lv[j].y = fma(p[j].y, fa[j], fma(-p[j].x, fb[j], lv[j].y));
                        } else {
                            lv[j].x = fma(p[j].x, fa[j], lv[j].x);
                            lv[j].y = fma(p[j].y, fa[j], lv[j].y);
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (!ok[j]) continue;
                L[a[j]] = lv[j];
                if (last) {
                    const C x = P[a[j]];
                    const T e = fma(x.x, lv[j].x, x.y * lv[j].y);
                    const T q = fma(x.x, x.x, x.y * x.y);
                    if constexpr (sizeof(T) == 4) {
                        f32c_add(facc, e);
                        f32c_add(fnrm, q);
                    } else {
                        dacc += e;
                        dnrm += q;
                    }
                }
            }
        }
        if (last) {   // uniform over the launch: the chunk's partials, fixed order
            if constexpr (sizeof(T) == 4)
                sweep_block_sum_c(facc, fnrm, reinterpret_cast<float *>(sh), dacc, dnrm);
            else
                sweep_block_sum(dacc, dnrm, sh);
            if (threadIdx.x == 0) {
                double *o = cpart + ((size_t)b * nchunks + chunk) * 3;
                o[0] = dacc;
                o[1] = dnrm;
                o[2] = 0.0;
            }
        }
    }
}

}  // namespace

size_t sweep_smem_bytes(const SweepDesc &W, size_t real_bytes) {
    const size_t ng = size_t(W.g_end - W.g_begin);
    return 1024 * 4 + size_t(W.t_count) * (2 * real_bytes + 4) + ng * sizeof(SGroup) +
           size_t(W.n_pat) * 4 + 16;
}

// Resident blocks per SM of the sweep kernel with `smem` bytes of dynamic
// shared memory: the grid must be resident at once, so that all threads of
// a state traverse the counter together.
int sweep_blocks_per_sm(int elem_bytes, size_t smem) {
    int occ = 0;
    if (smem > 48 * 1024) {
        cudaError_t e = elem_bytes == 16
            ? cudaFuncSetAttribute(k_apply_h_sweep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(k_apply_h_sweep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
    }
    cudaError_t e = elem_bytes == 16
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_h_sweep<double>, kSweepThreads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_h_sweep<float>, kSweepThreads, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return occ < 1 ? 1 : occ;
}

template <typename T>
cudaError_t launch_apply_h_sweep(const SweepDesc &W, const uint32_t *order, const SGroup *groups,
                                 const uint32_t *pat, const uint32_t *tz, const void *ca,
                                 const void *cb, const void *hdiag, int n_qubits, int batch,
                                 const void *psi, void *lam, size_t state_stride, int first,
                                 int last, unsigned long long *ctr, double *cpart, int blocks,
                                 cudaStream_t s) {
    using C = typename SV2<T>::type;
    if (W.t_count > kSweepMaxTerms || W.g_end - W.g_begin > kSweepMaxGroups || W.n_pat > kSweepMaxPat)
        return cudaErrorInvalidValue;
    const size_t smem = sweep_smem_bytes(W, sizeof(T));
    auto kern = k_apply_h_sweep<T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)blocks, batch);
    kern<<<grid, kSweepThreads, smem, s>>>(W, order, groups, pat, tz, static_cast<const T *>(ca),
                                           static_cast<const T *>(cb), static_cast<const T *>(hdiag),
                                           n_qubits, static_cast<const C *>(psi), static_cast<C *>(lam),
                                           state_stride, first, last, ctr, cpart);
    return cudaGetLastError();
}

template cudaError_t launch_apply_h_sweep<float>(const SweepDesc &, const uint32_t *, const SGroup *,
                                                 const uint32_t *, const uint32_t *, const void *,
                                                 const void *, const void *, int, int, const void *,
                                                 void *, size_t, int, int, unsigned long long *,
                                                 double *, int, cudaStream_t);
template cudaError_t launch_apply_h_sweep<double>(const SweepDesc &, const uint32_t *, const SGroup *,
                                                  const uint32_t *, const uint32_t *, const void *,
                                                  const void *, const void *, int, int, const void *,
                                                  void *, size_t, int, int, unsigned long long *,
                                                  double *, int, cudaStream_t);

}  // namespace vqe
