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
#include <algorithm>

#include "csum.cuh"
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

// f[j] += sum over terms [t0, t1) of c_t (-1)^{popc(i[j] & z_t)}, one load of
// each term for all J indices.
template <typename T, int J>
__device__ __forceinline__ void sign_sums(const uint32_t (&i)[J], T (&f)[J],
                                          const uint32_t *__restrict__ tz,
                                          const T *__restrict__ tc, int t0, int t1) {
    for (int t = t0; t < t1; ++t) {
        const uint32_t z = __ldg(tz + t);
        const T c = __ldg(tc + t);
#pragma unroll
        for (int j = 0; j < J; ++j) f[j] += sgn_flip(c, __popc(i[j] & z) & 1u);
    }
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

// Block sum of two per-thread compensated FP32 values (the complex64 window
// kernels): a fixed-order butterfly of compensated adds within each warp,
// then one warp over the warp totals; thread 0 receives both totals widened
// to FP64 for the fixed-order reduction across blocks.  Every add is an FP32
// TwoSum, so the block total keeps about 48 bits without FP64 instructions.
__device__ __forceinline__ void block_reduce2_c(F32c a, F32c b, float *sh, double &ra, double &rb) {
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
        const int nw = blockDim.x >> 5;
        a = lane < nw ? F32c{sh[4 * lane], sh[4 * lane + 1]} : f32c_zero();
        b = lane < nw ? F32c{sh[4 * lane + 2], sh[4 * lane + 3]} : f32c_zero();
        a = f32c_warp_sum(a, 0xffffffffu, 32);
        b = f32c_warp_sum(b, 0xffffffffu, 32);
        ra = f32c_value(a);
        rb = f32c_value(b);
    }
}

template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
k_energy_cols(const GroupDesc *__restrict__ groups, int n_groups, const uint32_t *__restrict__ tz,
              const T *__restrict__ tc, const T *__restrict__ hdiag, int n,
              const typename EV2<T>::type *__restrict__ psi, size_t stride,
              double *__restrict__ partials, int block_off, int bps_total) {
    using C = typename EV2<T>::type;
    constexpr int J = 4;   // pairs per thread and iteration: one load of each term serves J pairs
    __shared__ double sh[2 * (kEnergyThreads / 32)];
    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    const uint64_t npairs = 1ull << (n - 1);
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0, nrm = 0.0;
    for (int g = 0; g < n_groups; ++g) {
        const GroupDesc G = groups[g];
        // a thread's sums over its pairs of the group: FP64, or compensated
        // FP32 pairs in the FP32 kernel (one add per iteration of J pairs)
        T part = T(0), pn = T(0);
        F32c cpart = f32c_zero(), cpn = f32c_zero();
        const int h = G.x ? G.h : 0;
        const uint64_t lowm = (1ull << h) - 1ull;
        const bool has_b = G.t_end > G.t_mid;
        for (uint64_t p0 = tid; p0 < npairs; p0 += nthr * J) {
            uint32_t i0[J], i1[J];
            bool ok[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const uint64_t p = p0 + (uint64_t)j * nthr;
                ok[j] = p < npairs;
                const uint64_t pp = ok[j] ? p : p0;
                if (G.x == 0u) {
                    i0[j] = (uint32_t)(2 * pp);
                    i1[j] = i0[j] | 1u;
                } else {
                    i0[j] = (uint32_t)(((pp >> h) << (h + 1)) | (pp & lowm));
                    i1[j] = i0[j] ^ G.x;
                }
            }
            if (G.x == 0u) {
                T a0[J], a1[J], f0[J], f1[J];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const C x0 = P[i0[j]], x1 = P[i1[j]];
                    a0[j] = ok[j] ? fma(x0.x, x0.x, x0.y * x0.y) : T(0);
                    a1[j] = ok[j] ? fma(x1.x, x1.x, x1.y * x1.y) : T(0);
                    f0[j] = T(0);
                    f1[j] = T(0);
                }
                if (hdiag) {
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        f0[j] = __ldg(hdiag + i0[j]);
                        f1[j] = __ldg(hdiag + i1[j]);
                    }
                } else {
                    sign_sums<T, J>(i0, f0, tz, tc, G.t_begin, G.t_mid);
                    sign_sums<T, J>(i1, f1, tz, tc, G.t_begin, G.t_mid);
                }
                T it = T(0), itn = T(0);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    it = fma(a0[j], f0[j], fma(a1[j], f1[j], it));
                    itn += a0[j] + a1[j];
                }
                if constexpr (sizeof(T) == 4) {
                    f32c_add(cpart, it);
                    f32c_add(cpn, itn);
                } else {
                    part += it;
                    pn += itn;
                }
            } else {
                T ar[J], ai[J], fa[J], fb[J];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const C x0 = P[i0[j]], x1 = P[i1[j]];
                    // conj(x0) * x1 = ar + i ai; the imaginary part only matters for B terms
                    ar[j] = ok[j] ? fma(x0.x, x1.x, x0.y * x1.y) : T(0);
                    ai[j] = ok[j] ? fma(x0.x, x1.y, -x0.y * x1.x) : T(0);
                    fa[j] = T(0);
                    fb[j] = T(0);
                }
                sign_sums<T, J>(i0, fa, tz, tc, G.t_begin, G.t_mid);
                if (has_b) sign_sums<T, J>(i0, fb, tz, tc, G.t_mid, G.t_end);
                T it = T(0);
#pragma unroll
                for (int j = 0; j < J; ++j) it = fma(ar[j], fa[j], has_b ? fma(ai[j], fb[j], it) : it);
                if constexpr (sizeof(T) == 4) f32c_add(cpart, it);
                else part += it;
            }
        }
        double dpart = sizeof(T) == 4 ? f32c_value(cpart) : (double)part;
        if (G.x == 0u) nrm += sizeof(T) == 4 ? f32c_value(cpn) : (double)pn;
        else dpart *= 2.0;
        acc += dpart;
    }
    block_reduce2(acc, nrm, sh);
    if (threadIdx.x == 0) {
        double *o = partials + ((size_t)b * bps_total + block_off + blockIdx.x) * 3;
        o[0] = acc;
        o[1] = nrm;
        o[2] = 0.0;
    }
}

// lambda_i = sum_groups psi_{i^x} (FA(i) - i FB(i)); fused E = Re<psi|lambda>.
template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
k_apply_h(const GroupDesc *__restrict__ groups, int n_groups, const uint32_t *__restrict__ tz,
          const T *__restrict__ tc, const T *__restrict__ hdiag, int n,
          const typename EV2<T>::type *__restrict__ psi, typename EV2<T>::type *__restrict__ lam,
          size_t stride, double *__restrict__ partials) {
    using C = typename EV2<T>::type;
    constexpr int J = 4;
    __shared__ double sh[2 * (kEnergyThreads / 32)];
    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    C *L = lam + (size_t)b * stride;
    const uint64_t dim = 1ull << n;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0, nrm = 0.0;
    for (uint64_t i00 = tid; i00 < dim; i00 += nthr * J) {
        uint32_t i[J];
        bool ok[J];
        T lr[J], li[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const uint64_t ii = i00 + (uint64_t)j * nthr;
            ok[j] = ii < dim;
            i[j] = (uint32_t)(ok[j] ? ii : i00);
            lr[j] = T(0);
            li[j] = T(0);
        }
        for (int g = 0; g < n_groups; ++g) {
            const GroupDesc G = groups[g];
            T fa[J], fb[J];
            C pj[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                pj[j] = P[i[j] ^ G.x];
                fa[j] = T(0);
                fb[j] = T(0);
            }
            if (G.x == 0u && hdiag) {
#pragma unroll
                for (int j = 0; j < J; ++j) fa[j] = __ldg(hdiag + i[j]);
            } else {
                sign_sums<T, J>(i, fa, tz, tc, G.t_begin, G.t_mid);
            }
            if (G.t_end > G.t_mid) sign_sums<T, J>(i, fb, tz, tc, G.t_mid, G.t_end);
            if (G.t_end > G.t_mid) {
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    // (pr + i pi)(fa - i fb)
                    lr[j] = fma(pj[j].x, fa[j], fma(pj[j].y, fb[j], lr[j]));
                    li[j] = fma(pj[j].y, fa[j], fma(-pj[j].x, fb[j], li[j]));
                }
            } else {   // no class-B term: fb = 0
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    lr[j] = fma(pj[j].x, fa[j], lr[j]);
                    li[j] = fma(pj[j].y, fa[j], li[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (!ok[j]) continue;
            C out;
            out.x = lr[j];
            out.y = li[j];
            L[i[j]] = out;
            const C x = P[i[j]];
            acc += (double)fma(x.x, lr[j], x.y * li[j]);
            nrm += (double)fma(x.x, x.x, x.y * x.y);
        }
    }
    block_reduce2(acc, nrm, sh);
    if (threadIdx.x == 0) {
        double *o = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = acc;
        o[1] = nrm;
        o[2] = 0.0;
    }
}

// Diagonal of H: D_i = sum over the terms of the x = 0 group of
// c_t (-1)^{popc(i & z_t)}, summed in FP64 in term order and stored in T.
// Built once per Hamiltonian (and cutoff); the expectation and apply-H
// kernels then read D_i instead of evaluating every Z string per amplitude.
template <typename T>
__global__ void k_build_hdiag(const uint32_t *__restrict__ z, const double *__restrict__ c,
                              int n_terms, int n, T *__restrict__ D) {
    const uint64_t dim = 1ull << n;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        double f = 0.0;
        for (int t = 0; t < n_terms; ++t)
            f += sgn_flip(__ldg(c + t), __popc((uint32_t)i & __ldg(z + t)) & 1u);
        D[i] = (T)f;
    }
}

template <typename T>
cudaError_t launch_build_hdiag(const uint32_t *z, const double *c, int n_terms, int n_qubits,
                               void *D, int sms, cudaStream_t s) {
    const uint64_t dim = 1ull << n_qubits;
    const uint64_t want = (dim + 255) / 256;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)sms * 16);
    k_build_hdiag<T><<<blocks, 256, 0, s>>>(z, c, n_terms, n_qubits, static_cast<T *>(D));
    return cudaGetLastError();
}
template cudaError_t launch_build_hdiag<float>(const uint32_t *, const double *, int, int, void *,
                                               int, cudaStream_t);
template cudaError_t launch_build_hdiag<double>(const uint32_t *, const double *, int, int,
                                                void *, int, cudaStream_t);

// One block per state: each thread sums a strided subset of the block
// partials, then a fixed-order tree over the block (bitwise reproducible).
constexpr int kFinishThreads = 256;
__global__ void __launch_bounds__(kFinishThreads)
k_energy_finish(const double *__restrict__ partials, int bps, int batch, double *energies,
                double *norms, double *unnorm) {
    __shared__ double se[kFinishThreads], sn[kFinishThreads];
    const int b = blockIdx.x;
    const double *p = partials + (size_t)b * bps * 3;
    double e = 0.0, nn = 0.0;
    for (int i = threadIdx.x; i < bps; i += kFinishThreads) {
        e += p[3 * (size_t)i];
        nn += p[3 * (size_t)i + 1];
    }
    se[threadIdx.x] = e;
    sn[threadIdx.x] = nn;
    __syncthreads();
    for (int w = kFinishThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            se[threadIdx.x] += se[threadIdx.x + w];
            sn[threadIdx.x] += sn[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (energies) energies[b] = se[0] / sn[0];
        if (norms) norms[b] = sn[0];
        if (unnorm) unnorm[b] = se[0];
    }
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
                          const double *tc, const void *hdiag, int n_qubits, int batch,
                          const void *psi, size_t state_stride, double *partials, int bps,
                          cudaStream_t s) {
    using C = typename EV2<T>::type;
    dim3 grid(bps, batch);
    k_energy_cols<T><<<grid, kEnergyThreads, 0, s>>>(groups, n_groups, tz,
                                                     reinterpret_cast<const T *>(tc),
                                                     static_cast<const T *>(hdiag), n_qubits,
                                                     static_cast<const C *>(psi), state_stride,
                                                     partials, 0, bps);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_h(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                           const double *tc, const void *hdiag, int n_qubits, int batch,
                           const void *psi, void *lam, size_t state_stride, double *partials,
                           int bps, cudaStream_t s) {
    using C = typename EV2<T>::type;
    dim3 grid(bps, batch);
    k_apply_h<T><<<grid, kEnergyThreads, 0, s>>>(groups, n_groups, tz,
                                                 reinterpret_cast<const T *>(tc),
                                                 static_cast<const T *>(hdiag), n_qubits,
                                                 static_cast<const C *>(psi),
                                                 static_cast<C *>(lam), state_stride, partials);
    return cudaGetLastError();
}

cudaError_t launch_energy_finish(const double *partials, int bps, int batch, double *energies,
                                 double *norms, double *unnorm, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    k_energy_finish<<<batch, kFinishThreads, 0, s>>>(partials, bps, batch, energies, norms,
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
                                          const void *, int, int, const void *, size_t, double *,
                                          int, cudaStream_t);
template cudaError_t launch_energy<double>(const GroupDesc *, int, const uint32_t *,
                                           const double *, const void *, int, int, const void *,
                                           size_t, double *, int, cudaStream_t);
template cudaError_t launch_apply_h<float>(const GroupDesc *, int, const uint32_t *,
                                           const double *, const void *, int, int, const void *,
                                           void *, size_t, double *, int, cudaStream_t);
template cudaError_t launch_apply_h<double>(const GroupDesc *, int, const uint32_t *,
                                            const double *, const void *, int, int, const void *,
                                            void *, size_t, double *, int, cudaStream_t);

}  // namespace vqe

// ---------------------------------------------------------------- windowed expectation
//
// Groups whose X mask lies inside one tile "window" are evaluated from the
// window's tile staged in shared memory: the state is read once per window
// instead of once per group.  A window is the low run of m global bits plus
// k - m further global bits at any positions (a per-window offset table places
// them); the low window (m = k) also yields <psi|psi>.
//
// Signs.  For a term with Z mask z and a tile with global base `base`,
// (-1)^{popc(g & z)} = (-1)^{popc(base & zout)} * (-1)^{popc(e & zt)}: the
// first factor is folded into the coefficient once per tile, the second uses
// the element's tile index e.  A thread handles the pairs p = tid + j * 512
// (zero inserted at the group's top bit hl), i.e. e_j = e_0 | D_j with D_j
// linear in the bits of j, so (-1)^{popc(e_j & zt)} = (-1)^{popc(e_0 & zt)} *
// (-1)^{parity(j & v)} with v the term's "register pattern".  The host sorts a
// group's terms by v; the thread sums each run once with the sign of e_0,
//     F[v] = sum_{t in run v} c_t (-1)^{popc(e_0 & zt_t)},
// and a Walsh-Hadamard transform over v gives the sign sums of all its pairs,
//     f(j) = sum_v F[v] (-1)^{parity(j & v)},
// so a term costs one sign evaluation per thread instead of one per pair.

namespace vqe {

template <int N, typename T>
__device__ __forceinline__ void wht_inplace(T (&F)[N]) {
#pragma unroll
    for (int h = 1; h < N; h <<= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i & h) continue;
            const T x = F[i], y = F[i | h];
            F[i] = x + y;
            F[i | h] = x - y;
        }
    }
}

// F[v] += sum over the terms of run v of sc_t (-1)^{popc(e0 & zt_t)}.
template <int NV, typename T>
__device__ __forceinline__ void run_sums(T (&F)[NV], const uint16_t *run, int begin,
                                         const T *sc, const uint32_t *szt, uint32_t e0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        T f = T(0);
        const int t1 = begin + run[v + 1];
        for (int t = begin + run[v]; t < t1; ++t) f += sgn_flip(sc[t], __popc(e0 & szt[t]) & 1u);
        F[v] = f;
    }
}

// Shared-memory slot of tile element e in the window kernels: one pad
// element per 128-byte row, so that pair reads whose indices skip fixed bits
// (strides of 2..16 elements) spread over the banks.
template <typename C>
__host__ __device__ constexpr uint32_t wpad(uint32_t e) {
    return e + (e >> (sizeof(C) == 16 ? 3 : 4));
}

template <typename T, int K, bool RUNS>
__global__ void __launch_bounds__(kEnergyWinThreads, 2)
k_energy_win(WinDesc W, const WinGroup *__restrict__ wgroups, const WinTerm *__restrict__ wterms,
             const uint32_t *__restrict__ hoff, const T *__restrict__ hdiag,
             const typename EV2<T>::type *__restrict__ psi, size_t stride,
             double *__restrict__ partials, int bps_total) {
    using C = typename EV2<T>::type;
    static_assert(kEnergyWinThreads == 512, "pair layout assumes 512 threads");
    constexpr uint32_t size = 1u << K;
    constexpr int EPT = size / kEnergyWinThreads;   // tile elements per thread
    constexpr int PPT = EPT / 2;                    // pairs per thread and group
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sp = reinterpret_cast<C *>(smem_raw);                      // [wpad(size)] the tile (padded)
    T *sc = reinterpret_cast<T *>(sp + wpad<C>(size));           // [t_count] coefficients, base sign folded
    uint32_t *szt = reinterpret_cast<uint32_t *>(sc + W.t_count); // [t_count] tile Z bits
    uint32_t *soff = szt + W.t_count;                             // [2^(K-m)] high-part offsets
    __shared__ double sh[2 * (kEnergyWinThreads / 32)];
    __shared__ WinGroup sg[kWinMaxGroups];                         // the window's groups
    const int m = W.m;
    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    const uint32_t tid = threadIdx.x;
    // tile number -> the global bits of bmask, in increasing order
    uint32_t base = 0;
    {
        uint32_t bm = W.bmask, tn = blockIdx.x;
        while (bm) {
            const int bit = __ffs(bm) - 1;
            base |= (tn & 1u) << bit;
            tn >>= 1;
            bm &= bm - 1u;
        }
    }
    const uint32_t nh = 1u << (K - m);
    for (uint32_t i = tid; i < nh; i += blockDim.x) soff[i] = hoff[W.hoff + i];
    {
        const int ng = W.g_end - W.g_begin;
        const uint32_t *src = reinterpret_cast<const uint32_t *>(wgroups + W.g_begin);
        uint32_t *dst = reinterpret_cast<uint32_t *>(sg);
        for (int i = tid; i < ng * (int)(sizeof(WinGroup) / 4); i += blockDim.x) dst[i] = src[i];
    }
    for (int t = tid; t < W.t_count; t += blockDim.x) {
        const WinTerm wt = wterms[W.t_begin + t];
        sc[t] = (T)sgn_flip(wt.c, __popc(base & wt.zout) & 1u);
        szt[t] = wt.zt;
    }
    __syncthreads();
    const uint32_t lowmask = (1u << m) - 1u;
    {
        // all of a thread's loads in flight at once, then the stores
        C x[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = tid + j * kEnergyWinThreads;
            x[j] = P[(size_t)(base | (e & lowmask) | soff[e >> m])];
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) sp[wpad<C>(tid + j * kEnergyWinThreads)] = x[j];
    }
    __syncthreads();
    // Accumulators: FP64 in the FP64 kernels; in the FP32 kernels compensated
    // FP32 pairs (csum.cuh), into which every group total is added.
    double acc = 0.0, nrm = 0.0;
    F32c cacc = f32c_zero(), cnrm = f32c_zero();
    if (W.with_norm) {
        T pn = T(0);
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const C x = sp[wpad<C>(tid + j * kEnergyWinThreads)];
            pn += fma(x.x, x.x, x.y * x.y);
        }
        if constexpr (sizeof(T) == 4) cnrm.hi = pn;
        else nrm = (double)pn;
    }
    for (int gi = 0; gi < W.g_end - W.g_begin; ++gi) {
        const WinGroup &G = sg[gi];
        T part = T(0);
        if (G.xl == 0u) {
            if (!RUNS || hdiag) {   // the low window: global index = base | e
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const uint32_t e = tid + j * kEnergyWinThreads;
                    const C x = sp[wpad<C>(e)];
                    part = fma(fma(x.x, x.x, x.y * x.y), __ldg(hdiag + (size_t)(base | e)), part);
                }
            } else {
                if constexpr (RUNS) {
                T F[EPT];
                run_sums<EPT>(F, G.arun, G.a_begin, sc, szt, tid);
                wht_inplace<EPT>(F);
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const C x = sp[wpad<C>(tid + j * kEnergyWinThreads)];
                    part = fma(fma(x.x, x.x, x.y * x.y), F[j], part);
                }
                }
            }
        } else {
            // pair P = tid + 512 s of pattern u = P >> plog has lower element
            // i0 = spread(P mod 2^plog) | fval[u]: e0 spreads the thread's
            // bits below 9, D[s] the bits of s below plog - 9
            const uint32_t xl = G.xl;
            const int plog = G.plog;
            const uint32_t t0 = tid & (plog >= 9 ? 511u : ((1u << plog) - 1u));
            const uint32_t e0 = (t0 & G.smask[0]) | ((t0 & G.smask[1]) << 1) | ((t0 & G.smask[2]) << 2) |
                                ((t0 & G.smask[3]) << 3) | ((t0 & G.smask[4]) << 4);
            uint32_t D[PPT];
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                uint32_t d = 0;
#pragma unroll
                for (int bb = 0; (1 << bb) < PPT; ++bb)
                    if ((j >> bb) & 1) d |= G.dj[bb];
                D[j] = d;
            }
            const bool has_b = G.b_end > G.b_begin;
            if (!RUNS || G.direct) {
                // terms listed per pattern (at most kWinDirectMax per class),
                // one sign evaluation per term and pair.  FP32 holds a
                // pattern's terms in registers while the slots stay on it;
                // FP64 (fewer registers per value) reads them per slot.
                const uint32_t npat = (uint32_t)G.npat;
                T ca[kWinDirectMax], cb[kWinDirectMax];
                uint32_t za[kWinDirectMax], zb[kWinDirectMax];
                int na = 0, nb = 0;
                uint32_t ucur = ~0u;
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const uint32_t u = (tid + ((uint32_t)j << 9)) >> plog;   // warp-uniform
                    if (u >= npat) break;
                    const uint32_t il = e0 | D[j] | G.fval[u];
                    const C x0 = sp[wpad<C>(il)], x1 = sp[wpad<C>(il ^ xl)];
                    const T ar = fma(x0.x, x1.x, x0.y * x1.y);   // Re conj(x0) x1
                    const T ai = has_b ? fma(x0.x, x1.y, -x0.y * x1.x) : T(0);   // Im conj(x0) x1
                    if constexpr (sizeof(T) == 8) {
                        const int a1 = G.a_begin + G.arun[u + 1];
                        for (int t = G.a_begin + G.arun[u]; t < a1; ++t)
                            part = fma(ar, sgn_flip(sc[t], __popc(il & szt[t]) & 1u), part);
                        if (has_b) {
                            const int b1 = G.b_begin + G.brun[u + 1];
                            for (int t = G.b_begin + G.brun[u]; t < b1; ++t)
                                part = fma(ai, sgn_flip(sc[t], __popc(il & szt[t]) & 1u), part);
                        }
                    } else {
                        if (u != ucur) {
                            ucur = u;
                            const int a0 = G.a_begin + G.arun[u], b0 = G.b_begin + G.brun[u];
                            na = G.arun[u + 1] - G.arun[u];
                            nb = G.brun[u + 1] - G.brun[u];
#pragma unroll
                            for (int w = 0; w < kWinDirectMax; ++w) {
                                ca[w] = w < na ? sc[a0 + w] : T(0);
                                za[w] = w < na ? szt[a0 + w] : 0u;
                                cb[w] = w < nb ? sc[b0 + w] : T(0);
                                zb[w] = w < nb ? szt[b0 + w] : 0u;
                            }
                        }
#pragma unroll
                        for (int w = 0; w < kWinDirectMax; ++w)
                            if (w < na) part = fma(ar, sgn_flip(ca[w], __popc(il & za[w]) & 1u), part);
                        if (has_b) {
#pragma unroll
                            for (int w = 0; w < kWinDirectMax; ++w)
                                if (w < nb) part = fma(ai, sgn_flip(cb[w], __popc(il & zb[w]) & 1u), part);
                        }
                    }
                }
            } else if constexpr (RUNS) {
                // a whole group (one pattern, plog = K - 1: every slot valid)
                T ar[PPT], ai[PPT];
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const uint32_t il = e0 | D[j];
                    const C x0 = sp[wpad<C>(il)], x1 = sp[wpad<C>(il ^ xl)];
                    ar[j] = fma(x0.x, x1.x, x0.y * x1.y);
                    ai[j] = fma(x0.x, x1.y, -x0.y * x1.x);
                }
                T F[PPT];
                run_sums<PPT>(F, G.arun, G.a_begin, sc, szt, e0);
                wht_inplace<PPT>(F);
#pragma unroll
                for (int j = 0; j < PPT; ++j) part = fma(ar[j], F[j], part);
                if (has_b) {
                    run_sums<PPT>(F, G.brun, G.b_begin, sc, szt, e0);
                    wht_inplace<PPT>(F);
#pragma unroll
                    for (int j = 0; j < PPT; ++j) part = fma(ai[j], F[j], part);
                }
            }
            part *= T(2);
        }
        if constexpr (sizeof(T) == 4) f32c_add(cacc, part);
        else acc += (double)part;
    }
    if constexpr (sizeof(T) == 4) block_reduce2_c(cacc, cnrm, reinterpret_cast<float *>(sh), acc, nrm);
    else block_reduce2(acc, nrm, sh);
    if (threadIdx.x == 0) {
        double *o = partials + ((size_t)b * bps_total + W.block_off + blockIdx.x) * 3;
        o[0] = acc;
        o[1] = nrm;
        o[2] = 0.0;
    }
}

size_t win_smem_bytes(const WinDesc &W, size_t elem_bytes) {
    const size_t real = elem_bytes / 2;
    const size_t tile = (size_t(1) << W.k) + ((size_t(1) << W.k) >> (elem_bytes == 16 ? 3 : 4));   // padded
    return tile * elem_bytes + size_t(W.t_count) * (real + 4) +
           (size_t(1) << (W.k - W.m)) * 4;
}

// Windowed apply-H (the adjoint's lambda = H psi) over the expectation's
// windows and pair groups.  A tile of lambda is held in shared memory beside
// the tile of psi; the first window starts it from zero, the others from the
// lambda written by the previous window (a fixed order); the last window also
// yields the block partials of Re<psi|lambda> and <psi|psi>.  For a pair
// (i0, i1 = i0 ^ xl) of a group with sign sums FA, FB at i0 (the terms' signs
// at i1 are those at i0 times (-1)^{popc(x & z)}: +1 on class A, -1 on B),
//     lambda_i0 += psi_i1 (FA - i FB),   lambda_i1 += psi_i0 (FA + i FB).
// One thread owns a pair; a group's pairs are disjoint, so a barrier between
// groups orders the read-modify-writes of shared lambda.
template <typename T, int K, bool RUNS>
__global__ void __launch_bounds__(kEnergyWinThreads, 1)
k_apply_h_win(WinDesc W, const WinGroup *__restrict__ wgroups, const WinTerm *__restrict__ wterms,
              const uint32_t *__restrict__ hoff, const T *__restrict__ hdiag,
              const typename EV2<T>::type *__restrict__ psi, typename EV2<T>::type *__restrict__ lam,
              size_t stride, int first, int last, double *__restrict__ partials) {
    using C = typename EV2<T>::type;
    static_assert(kEnergyWinThreads == 512, "pair layout assumes 512 threads");
    constexpr uint32_t size = 1u << K;
    constexpr int EPT = size / kEnergyWinThreads;
    constexpr int PPT = EPT / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sp = reinterpret_cast<C *>(smem_raw);                      // [size] psi tile
    C *sl = sp + wpad<C>(size);                                   // [wpad(size)] lambda tile
    T *sc = reinterpret_cast<T *>(sl + wpad<C>(size));
    uint32_t *szt = reinterpret_cast<uint32_t *>(sc + W.t_count);
    uint32_t *soff = szt + W.t_count;
    __shared__ double sh[2 * (kEnergyWinThreads / 32)];
    __shared__ WinGroup sg[kWinMaxGroups];
    const int m = W.m;
    const int b = blockIdx.y;
    const C *P = psi + (size_t)b * stride;
    C *L = lam + (size_t)b * stride;
    const uint32_t tid = threadIdx.x;
    uint32_t base = 0;
    {
        uint32_t bm = W.bmask, tn = blockIdx.x;
        while (bm) {
            const int bit = __ffs(bm) - 1;
            base |= (tn & 1u) << bit;
            tn >>= 1;
            bm &= bm - 1u;
        }
    }
    const uint32_t nh = 1u << (K - m);
    for (uint32_t i = tid; i < nh; i += blockDim.x) soff[i] = hoff[W.hoff + i];
    {
        const int ng = W.g_end - W.g_begin;
        const uint32_t *src = reinterpret_cast<const uint32_t *>(wgroups + W.g_begin);
        uint32_t *dst = reinterpret_cast<uint32_t *>(sg);
        for (int i = tid; i < ng * (int)(sizeof(WinGroup) / 4); i += blockDim.x) dst[i] = src[i];
    }
    for (int t = tid; t < W.t_count; t += blockDim.x) {
        const WinTerm wt = wterms[W.t_begin + t];
        sc[t] = (T)sgn_flip(wt.c, __popc(base & wt.zout) & 1u);
        szt[t] = wt.zt;
    }
    __syncthreads();
    const uint32_t lowmask = (1u << m) - 1u;
    auto gidx = [&](uint32_t e) -> size_t { return (size_t)(base | (e & lowmask) | soff[e >> m]); };
    {
        // all of a thread's loads in flight at once, then the stores
        C x[EPT], l[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const size_t g = gidx(tid + j * kEnergyWinThreads);
            x[j] = P[g];
            l[j] = first ? C{} : L[g];
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            sp[wpad<C>(tid + j * kEnergyWinThreads)] = x[j];
            sl[wpad<C>(tid + j * kEnergyWinThreads)] = l[j];
        }
    }
    __syncthreads();
    // lambda_i0 += x1 (fa - i fb), lambda_i1 += x0 (fa + i fb); groups with
    // no class-B term (fb = 0, e.g. every hopping term XX + YY) take the real
    // form, half the multiply-adds
    auto pair_update = [&](uint32_t i0, uint32_t i1, C x0, C x1, T fa, T fb, bool with_b) {
        C l0 = sl[wpad<C>(i0)], l1 = sl[wpad<C>(i1)];
        if (with_b) {
            l0.x = fma(x1.x, fa, fma(x1.y, fb, l0.x));
            l0.y = fma(x1.y, fa, fma(-x1.x, fb, l0.y));
            l1.x = fma(x0.x, fa, fma(-x0.y, fb, l1.x));
            l1.y = fma(x0.y, fa, fma(x0.x, fb, l1.y));
        } else {
            l0.x = fma(x1.x, fa, l0.x);
            l0.y = fma(x1.y, fa, l0.y);
            l1.x = fma(x0.x, fa, l1.x);
            l1.y = fma(x0.y, fa, l1.y);
        }
        sl[wpad<C>(i0)] = l0;
        sl[wpad<C>(i1)] = l1;
    };
    const int ng = W.g_end - W.g_begin;
    for (int gi = 0; gi < ng; ++gi) {
        const WinGroup &G = sg[gi];
        const uint32_t xl = G.xl;
        const bool has_b = G.b_end > G.b_begin;
        if (xl == 0u) {
            T F[EPT];
            if (!RUNS || hdiag) {
#pragma unroll
                for (int j = 0; j < EPT; ++j) F[j] = __ldg(hdiag + gidx(tid + j * kEnergyWinThreads));
            } else if constexpr (RUNS) {
                run_sums<EPT>(F, G.arun, G.a_begin, sc, szt, tid);
                wht_inplace<EPT>(F);
            }
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const uint32_t e = tid + j * kEnergyWinThreads;
                const C y = sp[wpad<C>(e)];
                C l = sl[wpad<C>(e)];
                l.x = fma(y.x, F[j], l.x);
                l.y = fma(y.y, F[j], l.y);
                sl[wpad<C>(e)] = l;
            }
        } else {
            // pairs as in the expectation: pair P = tid + 512 s of pattern
            // u = P >> plog has i0 = spread(P mod 2^plog) | fval[u]
            const int plog = G.plog;
            const uint32_t t0 = tid & (plog >= 9 ? 511u : ((1u << plog) - 1u));
            const uint32_t e0 = (t0 & G.smask[0]) | ((t0 & G.smask[1]) << 1) | ((t0 & G.smask[2]) << 2) |
                                ((t0 & G.smask[3]) << 3) | ((t0 & G.smask[4]) << 4);
            uint32_t D[PPT];
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                uint32_t d = 0;
#pragma unroll
                for (int bb = 0; (1 << bb) < PPT; ++bb)
                    if ((j >> bb) & 1) d |= G.dj[bb];
                D[j] = d;
            }
            if (!RUNS || G.direct) {
                const uint32_t npat = (uint32_t)G.npat;
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const uint32_t u = (tid + ((uint32_t)j << 9)) >> plog;   // warp-uniform
                    if (u >= npat) break;
                    const uint32_t il = e0 | D[j] | G.fval[u];
                    // sign sums of the pattern's terms, started from the first
                    // term (a kept pattern has at least one; most hold exactly
                    // one after the merge, so no add is spent on a zero)
                    const int a0 = G.a_begin + G.arun[u], a1 = G.a_begin + G.arun[u + 1];
                    T fa = a1 > a0 ? sgn_flip(sc[a0], __popc(il & szt[a0]) & 1u) : T(0);
                    for (int t = a0 + 1; t < a1; ++t) fa += sgn_flip(sc[t], __popc(il & szt[t]) & 1u);
                    T fb = T(0);
                    if (has_b) {
                        const int b0 = G.b_begin + G.brun[u], b1 = G.b_begin + G.brun[u + 1];
                        fb = b1 > b0 ? sgn_flip(sc[b0], __popc(il & szt[b0]) & 1u) : T(0);
                        for (int t = b0 + 1; t < b1; ++t) fb += sgn_flip(sc[t], __popc(il & szt[t]) & 1u);
                    }
                    pair_update(il, il ^ xl, sp[wpad<C>(il)], sp[wpad<C>(il ^ xl)], fa, fb, has_b);
                }
            } else if constexpr (RUNS) {
                // a whole group (one pattern, plog = K - 1: every slot valid)
                T FA[PPT], FB[PPT];
                run_sums<PPT>(FA, G.arun, G.a_begin, sc, szt, e0);
                wht_inplace<PPT>(FA);
                if (has_b) {
                    run_sums<PPT>(FB, G.brun, G.b_begin, sc, szt, e0);
                    wht_inplace<PPT>(FB);
                } else {
#pragma unroll
                    for (int j = 0; j < PPT; ++j) FB[j] = T(0);
                }
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const uint32_t il = e0 | D[j];
                    pair_update(il, il ^ xl, sp[wpad<C>(il)], sp[wpad<C>(il ^ xl)], FA[j], FB[j], has_b);
                }
            }
        }
        __syncthreads();   // the next group's pairs touch other threads' elements
    }
    double acc = 0.0, nrm = 0.0;
    {
        T pa = T(0), pn = T(0);
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = tid + j * kEnergyWinThreads;
            const C l = sl[wpad<C>(e)];
            L[gidx(e)] = l;
            if (last) {
                const C x = sp[wpad<C>(e)];
                pa = fma(x.x, l.x, fma(x.y, l.y, pa));
                pn = fma(x.x, x.x, fma(x.y, x.y, pn));
            }
        }
        acc = (double)pa;
        nrm = (double)pn;
    }
    if (last) {   // uniform over the launch
        if constexpr (sizeof(T) == 4)
            block_reduce2_c(F32c{(float)acc, 0.f}, F32c{(float)nrm, 0.f}, reinterpret_cast<float *>(sh),
                            acc, nrm);
        else
            block_reduce2(acc, nrm, sh);
        if (threadIdx.x == 0) {
            double *o = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
            o[0] = acc;
            o[1] = nrm;
            o[2] = 0.0;
        }
    }
}

template <typename T>
cudaError_t launch_apply_h_win(const WinDesc &W, const WinGroup *wgroups, const WinTerm *wterms,
                               const uint32_t *hoff, const void *hdiag, int n_qubits, int batch,
                               const void *psi, void *lam, size_t state_stride, int first,
                               int last, double *partials, cudaStream_t s) {
    using C = typename EV2<T>::type;
    const size_t smem = win_smem_bytes(W, sizeof(C)) +
                        size_t(wpad<C>(1u << W.k)) * sizeof(C);   // + lambda tile (padded)
    auto kern = W.any_runs
        ? (W.k == 13 ? k_apply_h_win<T, 13, true> : (W.k == 12 ? k_apply_h_win<T, 12, true> : nullptr))
        : (W.k == 13 ? k_apply_h_win<T, 13, false> : (W.k == 12 ? k_apply_h_win<T, 12, false> : nullptr));
    if (!kern || W.t_count > kWinMaxTerms || W.g_end - W.g_begin > kWinMaxGroups)
        return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(1ull << (n_qubits - W.k)), batch);
    kern<<<grid, kEnergyWinThreads, smem, s>>>(W, wgroups, wterms, hoff, static_cast<const T *>(hdiag),
                                               static_cast<const C *>(psi), static_cast<C *>(lam),
                                               state_stride, first, last, partials);
    return cudaGetLastError();
}


template <typename T>
cudaError_t launch_energy_win(const WinDesc &W, const WinGroup *wgroups, const WinTerm *wterms,
                              const uint32_t *hoff, const void *hdiag, int n_qubits, int batch,
                              const void *psi, size_t state_stride, double *partials,
                              int bps_total, cudaStream_t s) {
    using C = typename EV2<T>::type;
    const size_t smem = win_smem_bytes(W, sizeof(C));
    auto kern = W.any_runs
        ? (W.k == 13 ? k_energy_win<T, 13, true> : (W.k == 12 ? k_energy_win<T, 12, true> : nullptr))
        : (W.k == 13 ? k_energy_win<T, 13, false> : (W.k == 12 ? k_energy_win<T, 12, false> : nullptr));
    if (!kern || W.t_count > kWinMaxTerms || W.g_end - W.g_begin > kWinMaxGroups)
        return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(1ull << (n_qubits - W.k)), batch);
    kern<<<grid, kEnergyWinThreads, smem, s>>>(W, wgroups, wterms, hoff,
                                               static_cast<const T *>(hdiag),
                                               static_cast<const C *>(psi), state_stride,
                                               partials, bps_total);
    return cudaGetLastError();
}

// Global-sweep expectation for a subset of groups, writing its block partials
// at column `block_off` of a layout with `bps_total` columns per state.
template <typename T>
cudaError_t launch_energy_sub(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                              const double *tc, int n_qubits, int batch, const void *psi,
                              size_t state_stride, double *partials, int bps, int block_off,
                              int bps_total, cudaStream_t s) {
    using C = typename EV2<T>::type;
    dim3 grid(bps, batch);
    k_energy_cols<T><<<grid, kEnergyThreads, 0, s>>>(groups, n_groups, tz,
                                                     reinterpret_cast<const T *>(tc), nullptr,
                                                     n_qubits, static_cast<const C *>(psi),
                                                     state_stride, partials, block_off, bps_total);
    return cudaGetLastError();
}

template cudaError_t launch_apply_h_win<float>(const WinDesc &, const WinGroup *, const WinTerm *,
                                               const uint32_t *, const void *, int, int,
                                               const void *, void *, size_t, int, int, double *,
                                               cudaStream_t);
template cudaError_t launch_apply_h_win<double>(const WinDesc &, const WinGroup *, const WinTerm *,
                                                const uint32_t *, const void *, int, int,
                                                const void *, void *, size_t, int, int, double *,
                                                cudaStream_t);
template cudaError_t launch_energy_win<float>(const WinDesc &, const WinGroup *, const WinTerm *,
                                              const uint32_t *, const void *, int, int,
                                              const void *, size_t, double *, int, cudaStream_t);
template cudaError_t launch_energy_win<double>(const WinDesc &, const WinGroup *, const WinTerm *,
                                               const uint32_t *, const void *, int, int,
                                               const void *, size_t, double *, int, cudaStream_t);
template cudaError_t launch_energy_sub<float>(const GroupDesc *, int, const uint32_t *,
                                              const double *, int, int, const void *, size_t,
                                              double *, int, int, int, cudaStream_t);
template cudaError_t launch_energy_sub<double>(const GroupDesc *, int, const uint32_t *,
                                               const double *, int, int, const void *, size_t,
                                               double *, int, int, int, cudaStream_t);

}  // namespace vqe
