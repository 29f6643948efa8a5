// Persistent, bulk-copy-pipelined tile passes.
//
// Same pass programs as k_pass (pass_core.cuh), but each CTA stays resident
// and walks a contiguous range of (state, tile) items with two shared-memory
// tile buffers: while the tile of item i is computed in one buffer, the bulk
// copy engine (cp.async.bulk, completion on an mbarrier) fetches item i+1 into
// the other, and the result of item i leaves through a bulk store.  A tile is
// one contiguous run (low-qubit passes) or 2^(k-m) runs of 2^m amplitudes
// (high-qubit passes), one bulk copy per run.  Coefficient rows are staged in
// shared memory once per state.  Every mbarrier wait is bounded: on timeout
// the CTA records an error in *err, drains its copies and returns.
#include "pass_core.cuh"

namespace vqe {

namespace {

__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *mb, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(mb)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mb, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(su32(mb)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *mb) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            su32(dst_smem)),
        "l"(src), "r"(bytes), "r"(su32(mb))
        : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(su32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// mbarrier waits give up after this many polls (each poll may suspend the
// thread for a while); a healthy copy completes within a few thousand.
constexpr uint32_t kMaxPolls = 1u << 22;

template <typename T>
struct PipeEnv {
    using C = typename V2<T>::type;
    static constexpr int kLoad = 0, kStore = 0;   // the tile is in shared memory, plain order
    const PassDesc *d;
    const RotCoef<T> *cf;
    const C *dt;
    double *gout;
    uint64_t tile;
    __device__ RotCoef<T> coef(int slot, int bit) const { return cf[slot * d->k + bit]; }
    __device__ C diag(int slot, uint32_t e) const { return dt[d->slot_dtab_off[slot] + e]; }
    static constexpr bool kDiagRow = true;
    __device__ const C *diag_row(int slot, uint32_t e0) const { return dt + d->slot_dtab_off[slot] + e0; }
    __device__ void grad(int slot, int bit, int comp, double v) const {
        gout[d->slot_grad_off[slot] + tile * (uint64_t)(2 * d->k) + bit * 2 + comp] = v;
    }
};

}  // namespace

template <typename T, int R, bool BWD>
__global__ void __launch_bounds__(512, 1)
k_pass_pipe(const PassDesc *__restrict__ desc, int init_zero, int n_qubits, int batch,
            typename V2<T>::type *__restrict__ psi, typename V2<T>::type *__restrict__ lam,
            size_t stride, const RotCoef<T> *__restrict__ coefs, size_t coef_stride,
            const typename V2<T>::type *__restrict__ dtab, size_t dtab_stride,
            double *__restrict__ gpart, size_t grad_stride, int *__restrict__ err) {
    using C = typename V2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ PassDesc sd;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ int s_fail;

    {   // descriptor -> shared memory
        const uint32_t *src = reinterpret_cast<const uint32_t *>(desc);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sd);
        for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / 4); i += blockDim.x) dst[i] = src[i];
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const PassDesc &d = sd;
    const int k = d.k, m = d.m, a = d.a, mid = a - m;
    const uint32_t size = 1u << k;
    const uint32_t bstride = tile_buf_elems(k, (int)sizeof(C));   // padded buffer stride
    const int nbuf = BWD ? 4 : 2;   // psi[0], psi[1] (, lam[0], lam[1])
    C *tiles = reinterpret_cast<C *>(smem_raw);
    double *gsh = reinterpret_cast<double *>(tiles + (size_t)nbuf * bstride);
    RotCoef<T> *scf = reinterpret_cast<RotCoef<T> *>(
        reinterpret_cast<unsigned char *>(gsh) + (BWD ? tile_grad_scratch_bytes((int)blockDim.x, k) : 0));

    const uint64_t n_tiles = 1ull << (n_qubits - k);
    const uint64_t total = n_tiles * (uint64_t)batch;
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t it0 = (uint64_t)blockIdx.x * per;
    const uint64_t it1 = it0 + per < total ? it0 + per : total;
    if (it0 >= it1) return;

    const uint32_t runs = 1u << (k - m);                   // contiguous runs per tile
    const uint32_t run_bytes = (1u << m) * (uint32_t)sizeof(C);
    const uint32_t tile_bytes = size * (uint32_t)sizeof(C);
    auto tile_base = [&](uint64_t tile) -> uint64_t {
        return ((tile & ((1ull << mid) - 1ull)) << m) | ((tile >> mid) << (a + (k - m)));
    };
    // Bulk copies are issued by warp 0; each lane commits and waits its own groups.
    const unsigned w0mask = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
    auto issue_load = [&](uint64_t it, int s) {
        if (threadIdx.x >= 32) return;
        const uint64_t b = it / n_tiles, tile = it % n_tiles, base = tile_base(tile);
        bulk_wait_read();      // the buffer's previous contents have left through a store
        __syncwarp(w0mask);
        if (threadIdx.x == 0) mbar_expect_tx(&mbar[s], tile_bytes * (BWD ? 2u : 1u));
        __syncwarp(w0mask);
        C *dp = tiles + (size_t)s * bstride;
        C *dl = tiles + (size_t)(2 + s) * bstride;
        const C *P = psi + b * stride;
        const C *L = BWD ? lam + b * stride : nullptr;
        for (uint32_t r = threadIdx.x; r < runs; r += 32) {
            const uint64_t g = base | ((uint64_t)r << a);
            bulk_load(dp + ((size_t)r << m), P + g, run_bytes, &mbar[s]);
            if (BWD) bulk_load(dl + ((size_t)r << m), L + g, run_bytes, &mbar[s]);
        }
    };
    auto issue_store = [&](uint64_t it, int s) {
        if (threadIdx.x >= 32) return;
        const uint64_t b = it / n_tiles, tile = it % n_tiles, base = tile_base(tile);
        C *dp = tiles + (size_t)s * bstride;
        C *dl = tiles + (size_t)(2 + s) * bstride;
        C *P = psi + b * stride;
        C *L = BWD ? lam + b * stride : nullptr;
        for (uint32_t r = threadIdx.x; r < runs; r += 32) {
            const uint64_t g = base | ((uint64_t)r << a);
            bulk_store(P + g, dp + ((size_t)r << m), run_bytes);
            if (BWD) bulk_store(L + g, dl + ((size_t)r << m), run_bytes);
        }
        bulk_commit();
    };

    uint32_t phase[2] = {0u, 0u};
    if (!init_zero) issue_load(it0, 0);
    int64_t cur_b = -1;
    bool failed = false;
    for (uint64_t it = it0; it < it1; ++it) {
        const int s = (int)((it - it0) & 1);
        if (!init_zero && it + 1 < it1) issue_load(it + 1, s ^ 1);
        C *sp = tiles + (size_t)s * bstride;
        C *sl = tiles + (size_t)(2 + s) * bstride;
        const uint64_t b = it / n_tiles, tile = it % n_tiles, base = tile_base(tile);
        if (init_zero) {
            // the first pass starts from |0...0>: no load
            if (threadIdx.x < 32) bulk_wait_read();
            __syncthreads();
            for (uint32_t e = threadIdx.x; e < size; e += blockDim.x) {
                C z;
                z.x = (base == 0 && e == 0) ? T(1) : T(0);
                z.y = T(0);
                sp[e] = z;
            }
        } else {
            uint32_t polls = 0;
            while (!mbar_try_wait(&mbar[s], phase[s]) && ++polls < kMaxPolls) {
            }
            if (polls >= kMaxPolls) s_fail = 1;
            phase[s] ^= 1u;
        }
        if ((int64_t)b != cur_b) {     // coefficient rows of this state
            __syncthreads();
            const RotCoef<T> *cf = coefs + b * coef_stride;
            for (int i = threadIdx.x; i < d.n_slots * k; i += blockDim.x)
                scf[i] = cf[d.slot_coef_off[i / k] + (i % k)];
            cur_b = (int64_t)b;
        }
        __syncthreads();
        if (s_fail) {
            failed = true;
            break;
        }
        PipeEnv<T> env{&d, scf, dtab + b * dtab_stride, BWD ? gpart + b * grad_stride : nullptr, tile};
        run_tile<T, R, BWD>(d, d.ops, d.n_ops, base, sp, sl, gsh, env);
        fence_async_smem();      // generic writes of the tile -> visible to the bulk store
        __syncthreads();
        issue_store(it, s);
    }
    if (failed) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // let the loads still in flight land before the block's shared memory goes away
        for (int s = 0; s < 2; ++s) {
            uint32_t polls = 0;
            while (!mbar_try_wait(&mbar[s], phase[s]) && ++polls < kMaxPolls) {
            }
        }
    }
    if (threadIdx.x < 32) bulk_wait_all();
}

size_t pipe_smem_bytes(const PassDesc &d, bool backward, size_t elem_bytes) {
    const size_t tiles = size_t(tile_buf_elems(d.k, (int)elem_bytes)) * elem_bytes * (backward ? 4 : 2);
    const size_t gsh = backward ? tile_grad_scratch_bytes(1 << (d.k - d.R), d.k) : 0;
    const size_t coef = elem_bytes == 16 ? sizeof(RotCoef<double>) : sizeof(RotCoef<float>);
    return tiles + gsh + size_t(d.n_slots) * d.k * coef;
}

template <typename T, int R, bool BWD>
static cudaError_t launch_pipe_r(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits,
                                 int batch, void *psi, void *lam, size_t stride,
                                 const RotCoef<T> *coefs, size_t coef_stride, const void *dtab,
                                 size_t dtab_stride, double *gpart, size_t grad_stride,
                                 int init_zero, int *err, int sms, cudaStream_t s) {
    using C = typename V2<T>::type;
    const int threads = 1 << (dh.k - dh.R);
    const size_t smem = pipe_smem_bytes(dh, BWD, sizeof(C));
    auto kern = k_pass_pipe<T, R, BWD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    const uint64_t total = (1ull << (n_qubits - dh.k)) * (uint64_t)batch;
    uint64_t grid = (uint64_t)sms * per_sm;
    if (grid > total) grid = total;
    kern<<<(unsigned)grid, threads, smem, s>>>(desc_dev, init_zero, n_qubits, batch,
                                                 static_cast<C *>(psi), static_cast<C *>(lam),
                                                 stride, coefs, coef_stride,
                                                 static_cast<const C *>(dtab), dtab_stride, gpart,
                                                 grad_stride, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass_pipe(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits,
                             int batch, void *psi, void *lam, size_t stride,
                             const RotCoef<T> *coefs, size_t coef_stride, const void *dtab,
                             size_t dtab_stride, double *gpart, size_t grad_stride, bool backward,
                             int init_zero, int *err, int sms, cudaStream_t s) {
#define VQE_PIPE_CASE(RR)                                                                       \
    case RR:                                                                                    \
        return backward ? launch_pipe_r<T, RR, true>(desc_dev, dh, n_qubits, batch, psi, lam,   \
                                                     stride, coefs, coef_stride, dtab,          \
                                                     dtab_stride, gpart, grad_stride, 0, err,   \
                                                     sms, s)                                    \
                        : launch_pipe_r<T, RR, false>(desc_dev, dh, n_qubits, batch, psi,       \
                                                      nullptr, stride, coefs, coef_stride,      \
                                                      dtab, dtab_stride, gpart, grad_stride,    \
                                                      init_zero, err, sms, s);
    switch (dh.R) {
        VQE_PIPE_CASE(1)
        VQE_PIPE_CASE(2)
        VQE_PIPE_CASE(3)
        VQE_PIPE_CASE(4)
        default:
            return cudaErrorInvalidValue;
    }
#undef VQE_PIPE_CASE
}

template cudaError_t launch_pass_pipe<float>(const PassDesc *, const PassDesc &, int, int, void *,
                                             void *, size_t, const RotCoef<float> *, size_t,
                                             const void *, size_t, double *, size_t, bool, int,
                                             int *, int, cudaStream_t);
template cudaError_t launch_pass_pipe<double>(const PassDesc *, const PassDesc &, int, int, void *,
                                              void *, size_t, const RotCoef<double> *, size_t,
                                              const void *, size_t, double *, size_t, bool, int,
                                              int *, int, cudaStream_t);

}  // namespace vqe
