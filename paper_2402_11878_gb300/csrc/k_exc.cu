// Kernels of the particle-conserving ansatz (Sec. II-B, Eqs. 5-6):
// psi(theta) = U(theta) psi_HF with U a product of fermionic excitation gates
// exp(theta (T - T^dag)), T = a_p^dag a_r (single) or a_p^dag a_q^dag a_r a_s
// (double), under the Jordan-Wigner mapping.
//
// A gate pairs each basis state j whose annihilated modes are occupied and
// created modes empty with j' = j ^ (amask | cmask); on the pair it is the
// rotation
//     psi_j  <- cos t psi_j  - sgn sin t psi_j'
//     psi_j' <- cos t psi_j' + sgn sin t psi_j,   sgn = (-1)^(sign0 + popc(j & smask)),
// and leaves every other amplitude alone.  A pass stages a tile of 2^k
// amplitudes in shared memory (its low m bits are a contiguous run of the
// state, its other k - m bits the modes of its gates) and applies a run of
// consecutive gates whose modes lie in the tile, one barrier per gate, with
// one HBM read and write of the state per pass.  The sign factors into a
// per-tile part (the sign mask's bits outside the tile, fixed by the tile's
// base) and a per-element parity over the tile bits.
//
// The backward (adjoint) pass un-applies the gates in reverse on psi and
// lambda = H psi and, before un-applying gate g, takes
//     dE/dtheta_g = 2 Re <lambda| G_g |psi>,  G_g = T_g - T_g^dag,
// per pair sgn * (Re conj(lambda_j') psi_j - Re conj(lambda_j) psi_j').
#include "csum.cuh"
#include "vqe_internal.h"

namespace vqe {

template <typename T> struct XV2;
template <> struct XV2<float> { using type = float2; };
template <> struct XV2<double> { using type = double2; };

constexpr int kExcMaxHigh = 8;   // k - m <= 8: 256 high-part offsets per pass

template <typename T>
__global__ void k_exc_stage(const double *__restrict__ params, int total, T *__restrict__ cs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    double s, c;
    sincos(params[i], &s, &c);
    cs[2 * i] = (T)c;
    cs[2 * i + 1] = (T)s;
}

template <typename T>
cudaError_t launch_exc_stage(const double *params, int n_exc, int batch, T *cs, cudaStream_t s) {
    const int total = n_exc * batch;
    if (total == 0) return cudaSuccess;
    k_exc_stage<T><<<(total + 255) / 256, 256, 0, s>>>(params, total, cs);
    return cudaGetLastError();
}

// f with a zero bit inserted at each tile position fixed[0..nf) (increasing).
__device__ __forceinline__ uint32_t spread_fixed(uint32_t f, const uint8_t *fixed, int nf) {
    for (int i = 0; i < nf; ++i) {
        const int b = fixed[i];
        f = ((f >> b) << (b + 1)) | (f & ((1u << b) - 1u));
    }
    return f;
}

__device__ __forceinline__ double xflip(double v, uint32_t s) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)s << 63));
}
__device__ __forceinline__ float xflip(float v, uint32_t s) {
    return __int_as_float(__float_as_int(v) ^ (int)(s << 31));
}

template <typename T, bool BWD>
__global__ void __launch_bounds__(kExcThreads)
k_exc_pass(ExcPass P, const ExcGate *__restrict__ gates, const uint32_t *__restrict__ hoff,
           typename XV2<T>::type *__restrict__ psi, typename XV2<T>::type *__restrict__ lam,
           size_t stride, const T *__restrict__ cs, int n_exc, double *__restrict__ gpart,
           size_t grad_stride, int init_hf, uint64_t hf) {
    using C = typename XV2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ExcGate sg[kExcMaxGates];
    __shared__ T scs[2 * kExcMaxGates];
    __shared__ uint32_t shoff[1 << kExcMaxHigh];
    const int k = P.k, m = P.m, ng = P.n_gates;
    const uint32_t size = 1u << k;
    const uint32_t tid = threadIdx.x;
    C *sp = reinterpret_cast<C *>(smem_raw);
    C *sl = BWD ? sp + size : nullptr;
    // backward: per-thread gradient partials, one row of kExcThreads per gate
    // (FP64 values, or compensated FP32 pairs in the FP32 kernel)
    unsigned char *rows = reinterpret_cast<unsigned char *>(sp + (BWD ? 2 * size : size));
    const int b = blockIdx.y;
    C *Pp = psi + (size_t)b * stride;
    C *Lp = BWD ? lam + (size_t)b * stride : nullptr;
    uint64_t base = 0;
    {
        uint32_t bm = P.bmask;
        uint64_t tn = blockIdx.x;
        while (bm) {
            const int bit = __ffs(bm) - 1;
            base |= (tn & 1ull) << bit;
            tn >>= 1;
            bm &= bm - 1u;
        }
    }
    // tiles outside the support of the state (see ExcPass): block-uniform
    if (!BWD && (base & P.zmask) != P.zval) {
        if (init_hf) {   // the first pass writes the whole state
            const uint32_t lowmask = (1u << m) - 1u;
            for (uint32_t e = tid; e < size; e += blockDim.x)
                Pp[base | (e & lowmask) | hoff[P.hoff + (e >> m)]] = C{};
        }
        return;
    }
    if (BWD && (base & P.bzmask) != P.bzval) {
        double *out = gpart + (size_t)b * grad_stride + P.grad_off + (size_t)blockIdx.x * ng;
        for (int i = tid; i < ng; i += blockDim.x) out[i] = 0.0;
        return;
    }
    for (int i = tid; i < ng; i += blockDim.x) {
        sg[i] = gates[P.g_begin + i];
        const int prm = gates[P.g_begin + i].param;
        scs[2 * i] = cs[((size_t)b * n_exc + prm) * 2];
        scs[2 * i + 1] = cs[((size_t)b * n_exc + prm) * 2 + 1];
    }
    const uint32_t nh = 1u << (k - m);
    for (uint32_t i = tid; i < nh; i += blockDim.x) shoff[i] = hoff[P.hoff + i];
    __syncthreads();
    const uint32_t lowmask = (1u << m) - 1u;
    // a thread's loads of the tile in flight together (kLoadBatch per
    // buffer), then their shared-memory stores
    constexpr int kLoadBatch = 8;
    for (uint32_t e0 = tid; e0 < size; e0 += kLoadBatch * blockDim.x) {
        C x[kLoadBatch], l[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const uint32_t e = e0 + u * blockDim.x;
            if (e >= size) break;
            const uint64_t g = base | (e & lowmask) | shoff[e >> m];
            if (init_hf) {
                x[u].x = (g == hf) ? T(1) : T(0);
                x[u].y = T(0);
            } else {
                x[u] = Pp[g];
            }
            if (BWD) l[u] = Lp[g];
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const uint32_t e = e0 + u * blockDim.x;
            if (e >= size) break;
            sp[e] = x[u];
            if (BWD) sl[e] = l[u];
        }
    }
    __syncthreads();
    for (int ii = 0; ii < ng; ++ii) {
        const int i = BWD ? ng - 1 - ii : ii;
        const ExcGate &G = sg[i];
        const T c = scs[2 * i], s = scs[2 * i + 1];
        const uint32_t sb = (uint32_t)((__popcll(base & (uint64_t)G.smask_g) + G.sign0) & 1);
        const uint32_t npairs = size >> G.n_fixed;
        const uint32_t flip = G.amask | G.cmask;
        double gd = 0.0;
        F32c gf = f32c_zero();
        for (uint32_t f = tid; f < npairs; f += blockDim.x) {
            const uint32_t e = spread_fixed(f, G.fixed, G.n_fixed) | G.amask;
            const uint32_t e2 = e ^ flip;
            const uint32_t par = sb ^ (__popc(e & G.smask_t) & 1u);
            const T ss = xflip(s, par);
            const C x = sp[e], y = sp[e2];
            C nx, ny;
            if (!BWD) {
                nx.x = fma(c, x.x, -ss * y.x);
                nx.y = fma(c, x.y, -ss * y.y);
                ny.x = fma(c, y.x, ss * x.x);
                ny.y = fma(c, y.y, ss * x.y);
            } else {
                const C lx = sl[e], ly = sl[e2];
                const T dg = xflip(fma(ly.x, x.x, fma(ly.y, x.y, -fma(lx.x, y.x, lx.y * y.y))), par);
                if constexpr (sizeof(T) == 8) gd += dg;
                else f32c_add(gf, dg);
                nx.x = fma(c, x.x, ss * y.x);
                nx.y = fma(c, x.y, ss * y.y);
                ny.x = fma(c, y.x, -ss * x.x);
                ny.y = fma(c, y.y, -ss * x.y);
                C mx, my;
                mx.x = fma(c, lx.x, ss * ly.x);
                mx.y = fma(c, lx.y, ss * ly.y);
                my.x = fma(c, ly.x, -ss * lx.x);
                my.y = fma(c, ly.y, -ss * lx.y);
                sl[e] = mx;
                sl[e2] = my;
            }
            sp[e] = nx;
            sp[e2] = ny;
        }
        if constexpr (BWD) {
            if constexpr (sizeof(T) == 8) reinterpret_cast<double *>(rows)[i * kExcThreads + tid] = gd;
            else reinterpret_cast<F32c *>(rows)[i * kExcThreads + tid] = gf;
        }
        __syncthreads();   // the next gate's pairs touch other threads' elements
    }
    for (uint32_t e = tid; e < size; e += blockDim.x) {
        const uint64_t g = base | (e & lowmask) | shoff[e >> m];
        Pp[g] = sp[e];
        if (BWD) Lp[g] = sl[e];
    }
    if constexpr (BWD) {
        // each warp sums whole rows in a fixed order (bitwise reproducible)
        const int warp = tid >> 5, lane = tid & 31;
        const int nw = kExcThreads / 32;
        double *out = gpart + (size_t)b * grad_stride + P.grad_off + (size_t)blockIdx.x * ng;
        for (int i = warp; i < ng; i += nw) {
            if constexpr (sizeof(T) == 8) {
                const double *r = reinterpret_cast<const double *>(rows) + i * kExcThreads;
                double sum = 0.0;
                for (int t = lane; t < kExcThreads; t += 32) sum += r[t];
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0) out[i] = 2.0 * sum;
            } else {
                const F32c *r = reinterpret_cast<const F32c *>(rows) + i * kExcThreads;
                F32c sum = f32c_zero();
                for (int t = lane; t < kExcThreads; t += 32) sum = f32c_add(sum, r[t]);
                sum = f32c_warp_sum(sum, 0xffffffffu, 32);
                if (lane == 0) out[i] = 2.0 * f32c_value(sum);
            }
        }
    }
}

template <typename T>
cudaError_t launch_exc_pass(const ExcPass &P, const ExcGate *gates_dev, const uint32_t *hoff_dev,
                            int n_qubits, int batch, void *psi, void *lam, size_t state_stride,
                            const T *cs, int n_exc, double *gpart, size_t grad_stride,
                            bool backward, int init_hf, uint64_t hf_index, cudaStream_t s) {
    using C = typename XV2<T>::type;
    if (P.k - P.m > kExcMaxHigh || P.n_gates > kExcMaxGates || P.n_gates < 1 || P.k > n_qubits)
        return cudaErrorInvalidValue;
    const size_t tile = (size_t(1) << P.k) * sizeof(C);
    const size_t row = sizeof(T) == 8 ? sizeof(double) : sizeof(F32c);
    const size_t smem = backward ? 2 * tile + size_t(P.n_gates) * kExcThreads * row : tile;
    dim3 grid((unsigned)(1ull << (n_qubits - P.k)), batch);
    if (backward) {
        auto kern = k_exc_pass<T, true>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, kExcThreads, smem, s>>>(P, gates_dev, hoff_dev, static_cast<C *>(psi),
                                             static_cast<C *>(lam), state_stride, cs, n_exc, gpart,
                                             grad_stride, 0, hf_index);
    } else {
        auto kern = k_exc_pass<T, false>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, kExcThreads, smem, s>>>(P, gates_dev, hoff_dev, static_cast<C *>(psi), nullptr,
                                             state_stride, cs, n_exc, nullptr, 0, init_hf, hf_index);
    }
    return cudaGetLastError();
}

template cudaError_t launch_exc_stage<float>(const double *, int, int, float *, cudaStream_t);
template cudaError_t launch_exc_stage<double>(const double *, int, int, double *, cudaStream_t);
template cudaError_t launch_exc_pass<float>(const ExcPass &, const ExcGate *, const uint32_t *, int,
                                            int, void *, void *, size_t, const float *, int,
                                            double *, size_t, bool, int, uint64_t, cudaStream_t);
template cudaError_t launch_exc_pass<double>(const ExcPass &, const ExcGate *, const uint32_t *, int,
                                             int, void *, void *, size_t, const double *, int,
                                             double *, size_t, bool, int, uint64_t, cudaStream_t);

}  // namespace vqe
