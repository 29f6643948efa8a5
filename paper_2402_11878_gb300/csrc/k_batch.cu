// Batched driver: many independent VQE problems of uneven size in one
// persistent launch (the single-GPU counterpart of the paper's distributed
// processing of independent circuit evaluations, Sec. II-C).
//
// Each CTA takes whole instances from an atomic queue ordered largest first.
// For an instance it stages the RY coefficients and the diagonal tables of
// every slot into shared memory (the diagonal as two half tables whose
// product is the entry), runs the forward passes, lambda = H psi with the
// energy, and the adjoint backward passes, accumulating the gradient in
// shared memory in a fixed order.  An instance whose state fits one tile
// (all passes span all qubits) never leaves shared memory; larger ones go
// tile by tile through a per-CTA slice of global memory.
#include "batch_internal.h"
#include "pass_core.cuh"

namespace vqe {

namespace {

template <typename T>
struct BatchEnv {
    using C = typename V2<T>::type;
    static constexpr int kLoad = 0, kStore = 0;   // the tile is in shared memory, plain order
    const PassDesc *d;
    const RotCoef<T> *coef_s;   // shared: all slots of the instance (plan's coef offsets)
    const C *lo_s;              // shared: per plan slot, 2^kl low half-table entries
    const C *hi_s;              // shared: per plan slot, 2^(k-kl) high half-table entries
    const int *slot_base;       // shared: plan slot index of pass slot s
    int kl, lo_stride, hi_stride;
    double *gacc;               // shared: gradient accumulators (2 n D)
    int n;
    int a, m;
    __device__ RotCoef<T> coef(int slot, int bit) const { return coef_s[d->slot_coef_off[slot] + bit]; }
    __device__ C diag(int slot, uint32_t e) const {
        const int ps = slot_base[slot];
        const C l = lo_s[ps * lo_stride + (e & ((1u << kl) - 1u))];
        const C h = hi_s[ps * hi_stride + (e >> kl)];
        return cmul(l, h);
    }
    static constexpr bool kDiagRow = false;   // half tables
    __device__ void grad(int slot, int bit, int comp, double v) const {
        const int q = bit < m ? bit : a + (bit - m);
        gacc[(d->slot_layer[slot] * n + q) * 2 + comp] += v;
    }
};

template <typename T>
__device__ __forceinline__ T bsign_sum(uint32_t i, const uint32_t *__restrict__ tz,
                                       const T *__restrict__ tc, int t0, int t1) {
    T f = T(0);
    for (int t = t0; t < t1; ++t) f += (__popc(i & tz[t]) & 1u) ? -tc[t] : tc[t];
    return f;
}

// The tile program for the instance's register bits.  Kernels are split by
// R4 (R = 4 alone, or R <= 3): one kernel holding all four bodies spills
// heavily, each half does not.
template <typename T, bool BWD, bool R4, class Env>
__device__ __forceinline__ void run_tile_any(int R, const PassDesc &d, uint64_t gbase,
                                             typename V2<T>::type *sp, typename V2<T>::type *sl,
                                             double *gsh, Env &env) {
    if constexpr (R4) {
        (void)R;
        run_tile<T, 4, BWD>(d, d.ops, d.n_ops, gbase, sp, sl, gsh, env);
    } else {
        switch (R) {
            case 1: run_tile<T, 1, BWD>(d, d.ops, d.n_ops, gbase, sp, sl, gsh, env); break;
            case 2: run_tile<T, 2, BWD>(d, d.ops, d.n_ops, gbase, sp, sl, gsh, env); break;
            default: run_tile<T, 3, BWD>(d, d.ops, d.n_ops, gbase, sp, sl, gsh, env); break;
        }
    }
}

}  // namespace

template <typename T, bool R4>
__global__ void __launch_bounds__(kBatchThreads, 1)
k_batch(BatchArgs args) {
    using C = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const BatchLayout &Ly = args.layout;
    C *sp = reinterpret_cast<C *>(smem + Ly.off_psi);
    C *sl = reinterpret_cast<C *>(smem + Ly.off_lam);
    double *gsh = reinterpret_cast<double *>(smem + Ly.off_gsh);
    RotCoef<T> *coef_s = reinterpret_cast<RotCoef<T> *>(smem + Ly.off_coef);
    C *lo_s = reinterpret_cast<C *>(smem + Ly.off_lo);
    C *hi_s = reinterpret_cast<C *>(smem + Ly.off_hi);
    double *gacc = reinterpret_cast<double *>(smem + Ly.off_gacc);
    double *red = reinterpret_cast<double *>(smem + Ly.off_red);
    int *slot_base = reinterpret_cast<int *>(smem + Ly.off_slotbase);
    __shared__ int s_item;

    C *gpsi = reinterpret_cast<C *>(args.scratch) + (size_t)blockIdx.x * 2 * args.scratch_elems;
    C *glam = gpsi + args.scratch_elems;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(args.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= args.count) break;
        const BatchInst I = args.inst[args.order[item]];
        const BatchPlan &PL = args.plans[I.plan];
        const int n = I.n;
        const int np = 2 * n * I.depth;
        const double *prm = args.params + I.params_off;

        // ---- stage every slot of the plan into shared memory
        double *phc = reinterpret_cast<double *>(smem + Ly.off_phc);   // [slot][bit] cos(phi/2)
        double *phs = reinterpret_cast<double *>(smem + Ly.off_phs);   // [slot][bit] sin(phi/2)
        double *scl = reinterpret_cast<double *>(smem + Ly.off_scl);   // [slot][bit] RY scale
        double *sig = reinterpret_cast<double *>(smem + Ly.off_sigma); // [slot] product of scales
        for (int i = threadIdx.x; i < np; i += blockDim.x) gacc[i] = 0.0;
        for (int w = threadIdx.x; w < PL.n_stage * kMaxTileBits; w += blockDim.x) {
            const int si = w / kMaxTileBits, j = w % kMaxTileBits;
            const StageSlot &S = args.stage[PL.stage_off + si];
            if (j >= S.n_gated) continue;
            const size_t pi = ((size_t)S.layer * n + S.qubit[j]) * 2;
            double s, c;
            sincos(0.5 * prm[pi], &s, &c);
            RotCoef<T> rc;
            if (fabs(c) >= fabs(s)) { rc.v = (T)(s / c); rc.mode = 0; scl[w] = c; }
            else                    { rc.v = (T)(c / s); rc.mode = 1; scl[w] = s; }
            rc.gs = T(0);
            coef_s[S.coef_off + S.tile_bit[j]] = rc;
            sincos(0.5 * prm[pi + 1], &s, &c);
            phc[w] = c;
            phs[w] = s;
        }
        __syncthreads();
        for (int si = threadIdx.x; si < PL.n_stage; si += blockDim.x) {
            const StageSlot &S = args.stage[PL.stage_off + si];
            double p = 1.0;
            for (int j = 0; j < S.n_gated; ++j) p *= scl[si * kMaxTileBits + j];
            sig[si] = p;
        }
        __syncthreads();
        for (int w = threadIdx.x; w < PL.n_stage * kMaxTileBits; w += blockDim.x) {
            const int si = w / kMaxTileBits, j = w % kMaxTileBits;
            const StageSlot &S = args.stage[PL.stage_off + si];
            if (j >= S.n_gated) continue;
            double pb = 1.0;
            for (int u = 0; u < S.n_gated; ++u)
                if ((S.before[j] >> S.tile_bit[u]) & 1u) pb *= scl[si * kMaxTileBits + u];
            const double f = sig[si] / pb;
            coef_s[S.coef_off + S.tile_bit[j]].gs = (T)(1.0 / (f * f));
        }
        // half tables: lo[v] = sigma * prod_{gated bits < kl} phase, hi[v] = prod_{gated bits >= kl}
        const int kl = PL.kl;
        const int per_slot = PL.lo_stride + PL.hi_stride;
        for (int w = threadIdx.x; w < PL.n_stage * per_slot; w += blockDim.x) {
            const int si = w / per_slot, e = w % per_slot;
            const StageSlot &S = args.stage[PL.stage_off + si];
            const bool low = e < PL.lo_stride;
            const uint32_t v = low ? e : e - PL.lo_stride;
            if (!low && v >= (1u << (S.k - kl))) continue;
            double re = low ? sig[si] : 1.0, im = 0.0;
            for (int j = 0; j < S.n_gated; ++j) {
                const int tb = S.tile_bit[j];
                if ((tb < kl) != low) continue;
                const int pos = low ? tb : tb - kl;
                const double c = phc[si * kMaxTileBits + j];
                const double sn = ((v >> pos) & 1u) ? phs[si * kMaxTileBits + j] : -phs[si * kMaxTileBits + j];
                const double nr = re * c - im * sn;
                im = re * sn + im * c;
                re = nr;
            }
            C out;
            out.x = (T)re;
            out.y = (T)im;
            if (low) lo_s[si * PL.lo_stride + v] = out;
            else hi_s[si * PL.hi_stride + v] = out;
        }
        __syncthreads();

        const uint64_t dim = 1ull << n;
        const bool in_smem = PL.whole_tile != 0;
        // ---- forward passes
        if (in_smem) {
            for (uint32_t e = threadIdx.x; e < dim; e += blockDim.x) {
                C z;
                z.x = (e == 0) ? T(1) : T(0);
                z.y = T(0);
                sp[e] = z;
            }
            __syncthreads();
        }
        for (int p = 0; p < PL.n_passes; ++p) {
            const PassDesc &d = args.fwd[PL.pass_off + p];
            for (int s = threadIdx.x; s < d.n_slots; s += blockDim.x)
                slot_base[s] = PL.slot_first[p] + s;
            __syncthreads();
            BatchEnv<T> env{&d, coef_s, lo_s, hi_s, slot_base, PL.kl, PL.lo_stride, PL.hi_stride,
                            gacc, n, d.a, d.m};
            const int k = d.k, m = d.m, a = d.a, mid = a - m;
            const uint64_t tiles = 1ull << (n - k);
            for (uint64_t tile = 0; tile < tiles; ++tile) {
                const uint64_t base = ((tile & ((1ull << mid) - 1ull)) << m) | ((tile >> mid) << (a + (k - m)));
                if (!in_smem) {
                    for (uint32_t e = threadIdx.x; e < (1u << k); e += blockDim.x) {
                        const uint64_t g = base | (e & ((1u << m) - 1u)) | ((uint64_t)(e >> m) << a);
                        if (p == 0) {
                            C z;
                            z.x = (g == 0) ? T(1) : T(0);
                            z.y = T(0);
                            sp[e] = z;
                        } else {
                            sp[e] = gpsi[g];
                        }
                    }
                    __syncthreads();
                }
                run_tile_any<T, false, R4>(d.R, d, base, sp, nullptr, gsh, env);
                if (!in_smem) {
                    for (uint32_t e = threadIdx.x; e < (1u << k); e += blockDim.x) {
                        const uint64_t g = base | (e & ((1u << m) - 1u)) | ((uint64_t)(e >> m) << a);
                        gpsi[g] = sp[e];
                    }
                    __syncthreads();
                }
            }
        }

        // ---- lambda = H psi and the energy
        {
            const C *P = in_smem ? sp : gpsi;
            C *L = in_smem ? sl : glam;
            double acc = 0.0, nrm = 0.0;
            const GroupDesc *G0 = args.groups + I.groups_off;
            const uint32_t *tz = args.tz + I.terms_off;
            const T *tc = reinterpret_cast<const T *>(args.tc) + I.terms_off;
            for (uint64_t ii = threadIdx.x; ii < dim; ii += blockDim.x) {
                const uint32_t i = (uint32_t)ii;
                T lr = T(0), li = T(0);
                for (int g = 0; g < I.n_groups; ++g) {
                    const GroupDesc G = G0[g];
                    const C pj = P[i ^ G.x];
                    const T fa = bsign_sum<T>(i, tz, tc, G.t_begin, G.t_mid);
                    const T fb = bsign_sum<T>(i, tz, tc, G.t_mid, G.t_end);
                    lr = fma(pj.x, fa, fma(pj.y, fb, lr));
                    li = fma(pj.y, fa, fma(-pj.x, fb, li));
                }
                C out;
                out.x = lr;
                out.y = li;
                L[i] = out;
                const C x = P[i];
                acc += (double)fma(x.x, lr, x.y * li);
                nrm += (double)fma(x.x, x.x, x.y * x.y);
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(0xffffffffu, acc, o);
                nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            }
            if ((threadIdx.x & 31) == 0) {
                red[2 * (threadIdx.x >> 5)] = acc;
                red[2 * (threadIdx.x >> 5) + 1] = nrm;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double e = 0.0, nn = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    e += red[2 * w];
                    nn += red[2 * w + 1];
                }
                args.energies[I.index] = e / nn;
            }
            __syncthreads();
        }

        // ---- adjoint backward passes
        for (int p = PL.n_passes - 1; p >= 0; --p) {
            const PassDesc &d = args.bwd[PL.pass_off + p];
            for (int s = threadIdx.x; s < d.n_slots; s += blockDim.x)
                slot_base[s] = PL.slot_first[p] + s;
            __syncthreads();
            BatchEnv<T> env{&d, coef_s, lo_s, hi_s, slot_base, PL.kl, PL.lo_stride, PL.hi_stride,
                            gacc, n, d.a, d.m};
            const int k = d.k, m = d.m, a = d.a, mid = a - m;
            const uint64_t tiles = 1ull << (n - k);
            for (uint64_t tile = 0; tile < tiles; ++tile) {
                const uint64_t base = ((tile & ((1ull << mid) - 1ull)) << m) | ((tile >> mid) << (a + (k - m)));
                if (!in_smem) {
                    for (uint32_t e = threadIdx.x; e < (1u << k); e += blockDim.x) {
                        const uint64_t g = base | (e & ((1u << m) - 1u)) | ((uint64_t)(e >> m) << a);
                        sp[e] = gpsi[g];
                        sl[e] = glam[g];
                    }
                    __syncthreads();
                }
                run_tile_any<T, true, R4>(d.R, d, base, sp, sl, gsh, env);
                if (!in_smem) {
                    for (uint32_t e = threadIdx.x; e < (1u << k); e += blockDim.x) {
                        const uint64_t g = base | (e & ((1u << m) - 1u)) | ((uint64_t)(e >> m) << a);
                        gpsi[g] = sp[e];
                        glam[g] = sl[e];
                    }
                    __syncthreads();
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < np; i += blockDim.x) args.grads[I.params_off + i] = gacc[i];
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_batch(const BatchArgs &args, bool r4, int grid, size_t smem, cudaStream_t s) {
    auto kern = k_batch<T, false>;
    if constexpr (sizeof(T) == 4) {
        if (r4) kern = k_batch<T, true>;
    } else if (r4) {
        return cudaErrorInvalidValue;   // FP64 plans keep R <= 3 (tiles of at most 2^12)
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBatchThreads, smem, s>>>(args);
    return cudaGetLastError();
}

template cudaError_t launch_batch<float>(const BatchArgs &, bool, int, size_t, cudaStream_t);
template cudaError_t launch_batch<double>(const BatchArgs &, bool, int, size_t, cudaStream_t);

}  // namespace vqe
