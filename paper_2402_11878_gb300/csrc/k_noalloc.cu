// vqe_energy_noalloc: the energy kernel in a form that allocates no device
// memory, for callers that cannot call cudaMalloc.
//
// Typical such callers: code whose device memory is owned entirely by
// another allocator (a framework's caching allocator or a pre-reserved pool
// that must not be exceeded), loops that keep other streams busy and cannot
// afford the device-wide synchronisation that cudaMalloc/cudaFree imply, and
// plug-ins that are handed raw device pointers by a host application and are
// not allowed to allocate on their own.
//
// The caller passes the state, the Pauli terms and the outputs in device
// memory.  The only scratch is the per-block partial sums, which live in the
// fixed file-scope array below; every GPU that loads this library holds it
// (64 KiB) until the process exits.
#include "vqe.h"
#include "vqe_internal.h"

#include <algorithm>
#include <mutex>

namespace {

constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;
// two doubles (energy, norm) per block; VQE_NOALLOC_MAX_BATCH states share
// them; one more slot holds the "invalid term" flag of the last call.
constexpr int kPartials = VQE_NOALLOC_MAX_BATCH;
constexpr int kFlagSlot = 2 * kPartials;

static __device__ __align__(256) double g_noalloc_scratch[2 * kPartials + 32];

double *g_scratch_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices] = {};

template <typename T> struct NV2;
template <> struct NV2<float> { using type = float2; };
template <> struct NV2<double> { using type = double2; };

__device__ __forceinline__ double na_flip(double v, uint32_t s) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)s << 63));
}

// One Pauli term at a time (the paper's per-term evaluation): for term
// (x, z, c) with kappa = popc(x & z), each pair (i, i^x) with the top bit of
// x clear contributes 2 Re[(-i)^kappa c (-1)^{popc(i&z)} conj(psi_i) psi_{i^x}],
// and x = 0 terms contribute c (-1)^{popc(i&z)} |psi_i|^2.  Block b of state s
// writes its partial (energy, norm) to scratch[2 * (s * bps + b)].
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_energy_terms(const typename NV2<T>::type *__restrict__ psi, int n,
               const uint64_t *__restrict__ xs, const uint64_t *__restrict__ zs,
               const double *__restrict__ cs, int n_terms, double *__restrict__ scratch) {
    using C = typename NV2<T>::type;
    __shared__ double sh[2 * (kThreads / 32)];
    const int s = blockIdx.y;
    const C *P = psi + ((size_t)s << n);
    const uint64_t dim = 1ull << n;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0, nrm = 0.0;
    const uint64_t over = ~((dim << 0) - 1ull);   // mask bits at or above n
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        // written by every call, so the flag never carries over between calls
        double bad = 0.0;
        for (int t = 0; t < n_terms; ++t)
            if ((xs[t] | zs[t]) & over || !isfinite(cs[t])) bad = 1.0;
        scratch[kFlagSlot] = bad;
    }
    for (uint64_t i = tid; i < dim; i += nthr) {
        const C v = P[i];
        nrm += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int t = 0; t < n_terms; ++t) {
        if ((xs[t] | zs[t]) & over) continue;     // reported through the flag
        const uint32_t x = (uint32_t)xs[t], z = (uint32_t)zs[t];
        const int kappa = __popc(x & z);
        const double c = cs[t];
        if (x == 0u) {
            for (uint64_t i = tid; i < dim; i += nthr) {
                const C v = P[i];
                const double a = (double)v.x * v.x + (double)v.y * v.y;
                acc += a * na_flip(c, __popc((uint32_t)i & z) & 1u);
            }
        } else {
            const int h = 31 - __clz(x);
            const uint64_t lowm = (1ull << h) - 1ull;
            // (-i)^kappa: kappa even -> real part with sign (-1)^{kappa/2},
            // kappa odd -> imaginary part with sign (-1)^{(kappa-1)/2}
            const double cc = ((kappa >> 1) & 1) ? -c : c;
            const bool imag = kappa & 1;
            for (uint64_t p = tid; p < (dim >> 1); p += nthr) {
                const uint32_t i0 = (uint32_t)(((p >> h) << (h + 1)) | (p & lowm));
                const C a = P[i0], b = P[i0 ^ x];
                const double re = (double)a.x * b.x + (double)a.y * b.y;
                const double im = (double)a.x * b.y - (double)a.y * b.x;
                acc += 2.0 * (imag ? im : re) * na_flip(cc, __popc(i0 & z) & 1u);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[2 * warp] = acc;
        sh[2 * warp + 1] = nrm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ea = 0.0, na = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ea += sh[2 * w];
            na += sh[2 * w + 1];
        }
        double *o = scratch + 2 * ((size_t)s * gridDim.x + blockIdx.x);
        o[0] = ea;
        o[1] = na;
    }
}

__global__ void k_energy_terms_finish(const double *__restrict__ scratch, int bps, int batch,
                                      double *energies, double *norms) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    const double *p = scratch + 2 * (size_t)s * bps;
    double e = 0.0, nn = 0.0;
    for (int b = 0; b < bps; ++b) {
        e += p[2 * b];
        nn += p[2 * b + 1];
    }
    const bool bad = scratch[kFlagSlot] != 0.0;
    energies[s] = bad ? __longlong_as_double(0x7ff8000000000000ll) : e / nn;
    if (norms) norms[s] = nn;
}

// Device address of the scratch array on `dev` and the device's SM count,
// looked up once per device with that device current.
cudaError_t scratch_address(int dev, double **out, int *sms) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_scratch_once[dev], [dev]() {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        int n_sm = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) cudaGetLastError();
        g_scratch_err[dev] = e;
        g_scratch_addr[dev] = (e == cudaSuccess) ? static_cast<double *>(p) : nullptr;
        g_sms[dev] = (e == cudaSuccess && n_sm > 0) ? n_sm : 1;
    });
    *out = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return g_scratch_err[dev];
}

}  // namespace

extern "C" vqe_status vqe_energy_noalloc(int n_qubits, vqe_precision precision,
                                         const void *psi_dev, int batch,
                                         const uint64_t *x_masks_dev,
                                         const uint64_t *z_masks_dev, const double *coeffs_dev,
                                         size_t n_terms, double *energies_dev,
                                         double *norms_dev, void *cuda_stream) {
    if (n_qubits < 1 || n_qubits > 32) return VQE_ERR_ARG;
    if (precision != VQE_C64 && precision != VQE_C128) return VQE_ERR_ARG;
    if (batch < 1 || batch > VQE_NOALLOC_MAX_BATCH) return VQE_ERR_ARG;
    if (n_terms > 0x7fffffff) return VQE_ERR_ARG;
    if (!psi_dev || !energies_dev) return VQE_ERR_ARG;
    if (n_terms > 0 && (!x_masks_dev || !z_masks_dev || !coeffs_dev)) return VQE_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VQE_ERR_CUDA;
    }
    double *scratch = nullptr;
    int sms = 1;
    if (scratch_address(dev, &scratch, &sms) != cudaSuccess || !scratch) return VQE_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // blocks per state: about 4 per SM over the whole batch, all partials in scratch
    const uint64_t work = (uint64_t(1) << n_qubits) / kThreads;
    int bps = (sms * 4 + batch - 1) / batch;
    bps = std::min(bps, kPartials / batch);
    if (uint64_t(bps) > work) bps = int(std::max<uint64_t>(work, 1));
    bps = std::max(bps, 1);
    dim3 grid(bps, batch);
    if (precision == VQE_C128)
        k_energy_terms<double><<<grid, kThreads, 0, s>>>(
            static_cast<const double2 *>(psi_dev), n_qubits, x_masks_dev, z_masks_dev,
            coeffs_dev, int(n_terms), scratch);
    else
        k_energy_terms<float><<<grid, kThreads, 0, s>>>(
            static_cast<const float2 *>(psi_dev), n_qubits, x_masks_dev, z_masks_dev,
            coeffs_dev, int(n_terms), scratch);
    if (cudaGetLastError() != cudaSuccess) return VQE_ERR_CUDA;
    k_energy_terms_finish<<<(batch + 127) / 128, 128, 0, s>>>(scratch, bps, batch, energies_dev,
                                                              norms_dev);
    if (cudaGetLastError() != cudaSuccess) return VQE_ERR_CUDA;
    return VQE_OK;
}
