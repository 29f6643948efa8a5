// Software-pipelined tile pass.  Persistent CTAs walk the (state, tile) work
// list with a grid stride.  While a CTA runs the pass program on one tile, the
// first-round elements of its next tile are already on their way from global
// memory into a second shared-memory buffer (cp.async), so global latency
// overlaps the arithmetic and shared-memory rounds of the current tile.  The
// last round stores straight from registers.  Same program, same results as
// the one-CTA-per-tile kernel of k_layers.cu; the first pass of a forward
// sweep (which starts from |0...0> and loads nothing) stays with that kernel.
#include <algorithm>

#include "pass_core.cuh"

namespace vqe {

namespace {

constexpr int kSpMaxThreads = 512;

template <typename T>
struct SpEnv {
    using C = typename V2<T>::type;
    static constexpr int kLoad = 2, kStore = 1;   // prefetched padded tile in, global out
    const PassDesc *d;
    const RotCoef<T> *cf;   // shared-memory coefficient rows of the pass's slots
    const C *dt;
    double *gout;
    uint64_t tile;
    C *P, *L;
    __device__ RotCoef<T> coef(int slot, int bit) const { return cf[slot * d->k + bit]; }
    __device__ C diag(int slot, uint32_t e) const { return dt[d->slot_dtab_off[slot] + e]; }
    static constexpr bool kDiagRow = true;
    __device__ const C *diag_row(int slot, uint32_t e0) const { return dt + d->slot_dtab_off[slot] + e0; }
    __device__ void grad(int slot, int bit, int comp, double v) const {
        gout[d->slot_grad_off[slot] + tile * (uint64_t)(2 * d->k) + bit * 2 + comp] = v;
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copy of one amplitude (8 or 16 bytes).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Thread t copies the 2^R elements it reads in the first round (chunk p0) of
// the tile with global base `gbase` into the padded slots run_tile reads them
// from (kLoad == 2).
template <typename T, int R, bool BWD>
__device__ __forceinline__ void prefetch_tile(const PassDesc &d, int p0, uint64_t gbase,
                                              const typename V2<T>::type *P,
                                              const typename V2<T>::type *L,
                                              typename V2<T>::type *buf,
                                              typename V2<T>::type *lbuf) {
    using C = typename V2<T>::type;
    constexpr int NR = 1 << R;
    const int k = d.k, m = d.m, a = d.a;
    const uint32_t t = threadIdx.x;
    if (t >= (1u << (k - R))) return;
    const uint32_t lowmask = (1u << m) - 1u;
    with_chunk<R>(p0, [&](auto pc) {
        constexpr int PP = decltype(pc)::value;
        const uint32_t e0 = elem_of(t, 0, PP, R);
        const uint32_t g0 =
            (uint32_t)(gbase | (uint64_t)(e0 & lowmask) | ((uint64_t)(e0 >> m) << a));
        uint32_t gst[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int bt = PP + j;
            gst[j] = bt < m ? (1u << bt) : (1u << (a + bt - m));
        }
        const uint32_t sb = pad_of<T>(e0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            uint32_t off = 0;
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((r >> j) & 1) off += gst[j];
            const uint32_t slot = sb + pad_of<T>((uint32_t)r << PP);
            cp_async<sizeof(C)>(buf + slot, P + g0 + off);
            if (BWD) cp_async<sizeof(C)>(lbuf + slot, L + g0 + off);
        }
    });
}

template <typename T, int R, bool BWD>
__global__ void __launch_bounds__(kSpMaxThreads, (BWD || R > 4) ? 1 : 2)
k_pass_sp(const PassDesc *__restrict__ desc, int n_qubits, int batch,
          typename V2<T>::type *__restrict__ psi, typename V2<T>::type *__restrict__ lam,
          size_t stride, const RotCoef<T> *__restrict__ coefs, size_t coef_stride,
          const typename V2<T>::type *__restrict__ dtab, size_t dtab_stride,
          double *__restrict__ gpart, size_t grad_stride) {
    using C = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PassDesc sd;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(desc);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sd);
        for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const PassDesc &d = sd;
    const int k = d.k, m = d.m, a = d.a, mid = a - m;
    constexpr int kBufs = BWD ? 2 : 1;                   // psi (and lambda) per stage
    const uint32_t bs = tile_buf_elems(k, (int)sizeof(C));
    C *bufs = reinterpret_cast<C *>(smem_raw);           // [2 stages][kBufs][bs]
    double *gsh = reinterpret_cast<double *>(bufs + (size_t)2 * kBufs * bs);
    RotCoef<T> *scf = reinterpret_cast<RotCoef<T> *>(
        reinterpret_cast<unsigned char *>(gsh) +
        (BWD ? tile_grad_scratch_bytes((int)blockDim.x, k) : 0));
    auto pbuf = [&](int s) { return bufs + (size_t)s * kBufs * bs; };
    auto lbuf = [&](int s) { return BWD ? bufs + ((size_t)s * kBufs + 1) * bs : nullptr; };
    auto tile_base = [&](uint64_t tile) -> uint64_t {
        return ((tile & ((1ull << mid) - 1ull)) << m) | ((tile >> mid) << (a + (k - m)));
    };

    const uint64_t n_tiles = 1ull << (n_qubits - k);
    const uint64_t total = n_tiles * (uint64_t)batch;
    uint64_t it = blockIdx.x;
    if (it >= total) return;   // whole block, before any further barrier
    const int p0 = d.ops[0].chunk;
    auto issue = [&](uint64_t w, int s) {
        const uint64_t b = w / n_tiles, tile = w % n_tiles;
        prefetch_tile<T, R, BWD>(d, p0, tile_base(tile), psi + b * stride,
                                 BWD ? lam + b * stride : nullptr, pbuf(s), lbuf(s));
    };
    issue(it, 0);
    cp_async_commit();
    int64_t cur_b = -1;
    for (int i = 0; it < total; ++i) {
        const int s = i & 1;
        const uint64_t nxt = it + gridDim.x;
        if (nxt < total) issue(nxt, s ^ 1);   // buffer s^1 was released by the last barrier
        cp_async_commit();                    // (possibly empty) group of the next tile
        cp_async_wait<1>();                   // this tile's group has landed
        const uint64_t b = it / n_tiles, tile = it % n_tiles;
        if ((int64_t)b != cur_b) {            // coefficient rows of this state
            const RotCoef<T> *cf = coefs + b * coef_stride;
            for (int j = threadIdx.x; j < d.n_slots * k; j += blockDim.x)
                scf[j] = cf[d.slot_coef_off[j / k] + (j % k)];
            cur_b = (int64_t)b;
        }
        __syncthreads();
        SpEnv<T> env{&sd, scf, dtab + b * dtab_stride, BWD ? gpart + b * grad_stride : nullptr,
                     tile, psi + b * stride, BWD ? lam + b * stride : nullptr};
        run_tile<T, R, BWD>(d, d.ops, d.n_ops, tile_base(tile), pbuf(s), lbuf(s), gsh, env);
        __syncthreads();                      // buffer s is free for the copies of tile i + 2
        it = nxt;
    }
    cp_async_wait<0>();
}

}  // namespace

size_t sp_smem_bytes(const PassDesc &d, bool backward, size_t elem_bytes) {
    const size_t tiles = size_t(tile_buf_elems(d.k, (int)elem_bytes)) * elem_bytes * 2 *
                         (backward ? 2 : 1);
    const size_t threads = size_t(1) << (d.k - d.R);
    const size_t gsh = backward ? tile_grad_scratch_bytes((int)threads, d.k) : 0;
    const size_t coef = elem_bytes == 16 ? sizeof(RotCoef<double>) : sizeof(RotCoef<float>);
    return tiles + gsh + size_t(d.n_slots) * d.k * coef;
}

template <typename T, int R, bool BWD>
static cudaError_t launch_sp_r(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits,
                               int batch, void *psi, void *lam, size_t stride,
                               const RotCoef<T> *coefs, size_t coef_stride, const void *dtab,
                               size_t dtab_stride, double *gpart, size_t grad_stride, int sms,
                               cudaStream_t s) {
    using C = typename V2<T>::type;
    const int threads = 1 << (dh.k - dh.R);
    if (threads > kSpMaxThreads) return cudaErrorInvalidConfiguration;
    const size_t smem = sp_smem_bytes(dh, BWD, sizeof(C));
    auto kern = k_pass_sp<T, R, BWD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t total = (1ull << (n_qubits - dh.k)) * (uint64_t)batch;
    const uint64_t grid = std::min<uint64_t>(total, (uint64_t)per_sm * sms);
    kern<<<(unsigned)grid, threads, smem, s>>>(desc_dev, n_qubits, batch, static_cast<C *>(psi),
                                               static_cast<C *>(lam), stride, coefs, coef_stride,
                                               static_cast<const C *>(dtab), dtab_stride, gpart,
                                               grad_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass_sp(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits, int batch,
                           void *psi, void *lam, size_t stride, const RotCoef<T> *coefs,
                           size_t coef_stride, const void *dtab, size_t dtab_stride,
                           double *gpart, size_t grad_stride, bool backward, int sms,
                           cudaStream_t s) {
#define VQE_SP_CASE(RR)                                                                          \
    case RR:                                                                                     \
        return backward ? launch_sp_r<T, RR, true>(desc_dev, dh, n_qubits, batch, psi, lam,      \
                                                   stride, coefs, coef_stride, dtab, dtab_stride, \
                                                   gpart, grad_stride, sms, s)                    \
                        : launch_sp_r<T, RR, false>(desc_dev, dh, n_qubits, batch, psi, nullptr, \
                                                    stride, coefs, coef_stride, dtab,            \
                                                    dtab_stride, gpart, grad_stride, sms, s);
    switch (dh.R) {
        VQE_SP_CASE(1)
        VQE_SP_CASE(2)
        VQE_SP_CASE(3)
        VQE_SP_CASE(4)
        default:
            return cudaErrorInvalidValue;
    }
#undef VQE_SP_CASE
}

template cudaError_t launch_pass_sp<float>(const PassDesc *, const PassDesc &, int, int, void *,
                                           void *, size_t, const RotCoef<float> *, size_t,
                                           const void *, size_t, double *, size_t, bool, int,
                                           cudaStream_t);
template cudaError_t launch_pass_sp<double>(const PassDesc *, const PassDesc &, int, int, void *,
                                            void *, size_t, const RotCoef<double> *, size_t,
                                            const void *, size_t, double *, size_t, bool, int,
                                            cudaStream_t);

}  // namespace vqe
