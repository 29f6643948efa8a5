// Expectation-value kernels: <psi|H|psi> and <psi|psi> (Sec. II-B, Eq. 7)
// for H = sum_i w_i P_i (Eqs. 2-4), and lambda = H psi for the adjoint
// gradient.
//
// The paper evaluates the terms one at a time, which makes the time
// proportional to the number of terms (Sec. III-D).  Here terms are grouped
// by their X mask x: P(x, z) psi at index i reads the same partner amplitude
// psi_{i^x} for every z of the group, so one sweep per group computes
//     sum_i conj(psi_i) psi_{i^x} * sum_z c'_z (-1)^{popc(i & z)},
// with the Pauli phase (-i)^{popc(x&z)} folded into the sign and real/imag
// split of c' on the host.  Each unordered pair (i, i^x) is visited once: the
// two orientations contribute equal real parts.  Accumulation is FP64 per
// thread; reductions go through fixed-order warp shuffles, a block partial
// per CTA, and a fixed-order final sum, so results are bitwise reproducible.
#include "vqe_internal.h"

namespace vqe {

template <typename T> struct EV2;
template <> struct EV2<float> { using type = float2; };
template <> struct EV2<double> { using type = double2; };

__device__ __forceinline__ double sgn_flip(double v, uint32_t s) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)s << 63));
}
__device__ __forceinline__ float sgn_flip(float v, uint32_t s) {
    return __int_as_float(__float_as_int(v) ^ (int)(s << 31));
}

// sum over terms [t0, t1) of c_t * (-1)^{popc(i & z_t)}
template <typename T>
__device__ __forceinline__ T sign_sum(uint32_t i, const uint32_t *__restrict__ tz,
                                      const T *__restrict__ tc, int t0, int t1) {
    T f = T(0);
    for (int t = t0; t < t1; ++t) {
        const uint32_t par = __popc(i & __ldg(tz + t)) & 1u;
        f += sgn_flip(__ldg(tc + t), par);
    }
    return f;
}

__device__ __forceinline__ void block_reduce2(double &a, double &b, double *sh) {
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
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; ++w) {
            sa += sh[2 * w];
            sb += sh[2 * w + 1];
        }
        a = sa;
        b = sb;
    }
}

template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
k_energy(const GroupDesc *__restrict__ groups, int n_groups, const uint32_t *__restrict__ tz,
         const T *__restrict__ tc, int n, const typename EV2<T>::type *__restrict__ psi,
         size_t stride, double *__restrict__ partials) {
    using C = typename EV2<T>::type;
    __shared__ double sh[2 * (kEnergyThreads / 32)];
    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    const uint64_t npairs = 1ull << (n - 1);
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0, nrm = 0.0;
    for (int g = 0; g < n_groups; ++g) {
        const GroupDesc G = groups[g];
        T part = T(0), pn = T(0);
        if (G.x == 0u) {
            for (uint64_t p = tid; p < npairs; p += nthr) {
                const uint32_t i0 = (uint32_t)(2 * p), i1 = i0 | 1u;
                const C x0 = P[i0], x1 = P[i1];
                const T a0 = fma(x0.x, x0.x, x0.y * x0.y);
                const T a1 = fma(x1.x, x1.x, x1.y * x1.y);
                const T f0 = sign_sum<T>(i0, tz, tc, G.t_begin, G.t_mid);
                const T f1 = sign_sum<T>(i1, tz, tc, G.t_begin, G.t_mid);
                part = fma(a0, f0, fma(a1, f1, part));
                pn += a0 + a1;
            }
            nrm += (double)pn;
        } else {
            const int h = G.h;
            const uint64_t lowm = (1ull << h) - 1ull;
            for (uint64_t p = tid; p < npairs; p += nthr) {
                const uint32_t i0 = (uint32_t)(((p >> h) << (h + 1)) | (p & lowm));
                const uint32_t i1 = i0 ^ G.x;
                const C x0 = P[i0], x1 = P[i1];
                // conj(x0) * x1 = ar + i ai
                const T ar = fma(x0.x, x1.x, x0.y * x1.y);
                const T ai = fma(x0.x, x1.y, -x0.y * x1.x);
                const T fa = sign_sum<T>(i0, tz, tc, G.t_begin, G.t_mid);
                const T fb = sign_sum<T>(i0, tz, tc, G.t_mid, G.t_end);
                part = fma(ar, fa, fma(ai, fb, part));
            }
            part *= T(2);
        }
        acc += (double)part;
    }
    block_reduce2(acc, nrm, sh);
    if (threadIdx.x == 0) {
        double *o = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = acc;
        o[1] = nrm;
        o[2] = 0.0;
    }
}

// lambda_i = sum_groups psi_{i^x} (FA(i) - i FB(i)); fused E = Re<psi|lambda>.
template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
k_apply_h(const GroupDesc *__restrict__ groups, int n_groups, const uint32_t *__restrict__ tz,
          const T *__restrict__ tc, int n, const typename EV2<T>::type *__restrict__ psi,
          typename EV2<T>::type *__restrict__ lam, size_t stride, double *__restrict__ partials) {
    using C = typename EV2<T>::type;
    __shared__ double sh[2 * (kEnergyThreads / 32)];
    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    C *L = lam + (size_t)b * stride;
    const uint64_t dim = 1ull << n;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0, nrm = 0.0;
    for (uint64_t ii = tid; ii < dim; ii += nthr) {
        const uint32_t i = (uint32_t)ii;
        T lr = T(0), li = T(0);
        for (int g = 0; g < n_groups; ++g) {
            const GroupDesc G = groups[g];
            const C pj = P[i ^ G.x];
            const T fa = sign_sum<T>(i, tz, tc, G.t_begin, G.t_mid);
            const T fb = sign_sum<T>(i, tz, tc, G.t_mid, G.t_end);
            // (pr + i pi)(fa - i fb)
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
    block_reduce2(acc, nrm, sh);
    if (threadIdx.x == 0) {
        double *o = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = acc;
        o[1] = nrm;
        o[2] = 0.0;
    }
}

// One thread per state; partials summed in block order.
__global__ void k_energy_finish(const double *__restrict__ partials, int bps, int batch,
                                double *energies, double *norms, double *unnorm) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double *p = partials + (size_t)b * bps * 3;
    double e = 0.0, nn = 0.0;
    for (int i = 0; i < bps; ++i) {
        e += p[3 * i];
        nn += p[3 * i + 1];
    }
    if (energies) energies[b] = e / nn;
    if (norms) norms[b] = nn;
    if (unnorm) unnorm[b] = e;
}

// One block per (state, parameter): threads sum strided partials, then a
// fixed-order tree over the block (bitwise reproducible).
constexpr int kGradThreads = 128;
__global__ void __launch_bounds__(kGradThreads)
k_grad_finish(const double *__restrict__ part, size_t part_stride, const int *__restrict__ off,
              const int *__restrict__ count, const int *__restrict__ step, int n_params,
              double *grads) {
    __shared__ double sh[kGradThreads];
    const int p = blockIdx.x, b = blockIdx.y;
    const double *src = part + (size_t)b * part_stride + off[p];
    const int c = count[p], s = step[p];
    double acc = 0.0;
    for (int j = threadIdx.x; j < c; j += kGradThreads) acc += src[(size_t)j * s];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kGradThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) grads[(size_t)b * n_params + p] = sh[0];
}

template <typename T>
cudaError_t launch_energy(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                          const double *tc, int n_qubits, int batch, const void *psi,
                          size_t state_stride, double *partials, int bps, cudaStream_t s) {
    using C = typename EV2<T>::type;
    dim3 grid(bps, batch);
    k_energy<T><<<grid, kEnergyThreads, 0, s>>>(groups, n_groups, tz,
                                                reinterpret_cast<const T *>(tc), n_qubits,
                                                static_cast<const C *>(psi), state_stride,
                                                partials);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_h(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                           const double *tc, int n_qubits, int batch, const void *psi, void *lam,
                           size_t state_stride, double *partials, int bps, cudaStream_t s) {
    using C = typename EV2<T>::type;
    dim3 grid(bps, batch);
    k_apply_h<T><<<grid, kEnergyThreads, 0, s>>>(groups, n_groups, tz,
                                                 reinterpret_cast<const T *>(tc), n_qubits,
                                                 static_cast<const C *>(psi),
                                                 static_cast<C *>(lam), state_stride, partials);
    return cudaGetLastError();
}

cudaError_t launch_energy_finish(const double *partials, int bps, int batch, double *energies,
                                 double *norms, double *unnorm, cudaStream_t s) {
    k_energy_finish<<<(batch + 127) / 128, 128, 0, s>>>(partials, bps, batch, energies, norms,
                                                        unnorm);
    return cudaGetLastError();
}

cudaError_t launch_grad_finish(const double *part, size_t part_stride, const int *off,
                               const int *count, const int *step, int n_params, int batch,
                               double *grads, cudaStream_t s) {
    dim3 grid(n_params, batch);
    k_grad_finish<<<grid, kGradThreads, 0, s>>>(part, part_stride, off, count, step, n_params,
                                                grads);
    return cudaGetLastError();
}

template cudaError_t launch_energy<float>(const GroupDesc *, int, const uint32_t *, const double *,
                                          int, int, const void *, size_t, double *, int,
                                          cudaStream_t);
template cudaError_t launch_energy<double>(const GroupDesc *, int, const uint32_t *,
                                           const double *, int, int, const void *, size_t,
                                           double *, int, cudaStream_t);
template cudaError_t launch_apply_h<float>(const GroupDesc *, int, const uint32_t *,
                                           const double *, int, int, const void *, void *, size_t,
                                           double *, int, cudaStream_t);
template cudaError_t launch_apply_h<double>(const GroupDesc *, int, const uint32_t *,
                                            const double *, int, int, const void *, void *,
                                            size_t, double *, int, cudaStream_t);

}  // namespace vqe
