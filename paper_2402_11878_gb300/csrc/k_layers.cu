// Ansatz kernels: parameter staging, fused tile passes (forward and adjoint
// backward), and the one-gate-per-pass reference kernels.
//
// Method: the hardware-efficient ansatz (Sec. II-B names the class) applied
// to a 2^n state vector, psi(theta) = U(theta)|0...0> (Eq. 6).  Layer l is
//     CZ_chain * prod_q RZ(phi_{l,q}) * prod_q RY(theta_{l,q}),
// because gates on different qubits commute.  A pass stages a tile of 2^k
// amplitudes spanning one qubit group in shared memory and applies all gates
// of one or more layers on those qubits; RY(theta) is applied as scale * B
// with B = [[1,-t],[t,1]] (t = tan theta/2) or [[u,-1],[1,u]] (u = cot),
// one FMA per real output, and the scale is folded with the RZ phases into a
// per-slot diagonal table.  CZ signs are integer sign flips.
//
// The backward pass is the adjoint method: it un-applies the same slots in
// reverse on psi and lambda = H psi, and for each gated qubit q accumulates
//     dE/dtheta = Im <lambda| Y_q |psi>,   dE/dphi = Im <lambda| Z_q |psi>
// at a point of the sweep where both are valid (after the slot's diagonal is
// undone and before q's own rotation is undone).
#include <algorithm>
#include <vector>

#include "pass_core.cuh"

namespace vqe {

// ---------------------------------------------------------------- staging

template <typename T>
__global__ void k_stage(const StageSlot *__restrict__ slots, int n, int depth,
                        const double *__restrict__ params, RotCoef<T> *__restrict__ coefs,
                        size_t coef_stride, typename V2<T>::type *__restrict__ dtab,
                        size_t dtab_stride) {
    using C = typename V2<T>::type;
    __shared__ double ph_c[kMaxTileBits], ph_s[kMaxTileBits], scl[kMaxTileBits], ph_v[kMaxTileBits];
    __shared__ int ph_m[kMaxTileBits];
    __shared__ double sigma;
    const StageSlot S = slots[blockIdx.x];
    const int b = blockIdx.y;
    const double *pr = params + (size_t)b * (2 * (size_t)n * depth);
    if (threadIdx.x < (unsigned)S.n_gated) {
        const int j = threadIdx.x;
        const int q = S.qubit[j];
        const double th = pr[((size_t)S.layer * n + q) * 2];
        const double phi = pr[((size_t)S.layer * n + q) * 2 + 1];
        double s, c;
        sincos(0.5 * th, &s, &c);
        if (fabs(c) >= fabs(s)) { ph_v[j] = s / c; ph_m[j] = 0; scl[j] = c; }
        else                    { ph_v[j] = c / s; ph_m[j] = 1; scl[j] = s; }
        double sp, cp;
        sincos(0.5 * phi, &sp, &cp);
        ph_c[j] = cp;
        ph_s[j] = sp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double p = 1.0;
        for (int u = 0; u < S.n_gated; ++u) p *= scl[u];
        sigma = p;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)S.n_gated) {
        const int j = threadIdx.x;
        double pb = 1.0;
        for (int u = 0; u < S.n_gated; ++u)
            if ((S.before[j] >> S.tile_bit[u]) & 1u) pb *= scl[u];
        const double f = sigma / pb;
        RotCoef<T> rc;
        rc.v = (T)ph_v[j];
        rc.gs = (T)(1.0 / (f * f));
        rc.mode = ph_m[j];
        coefs[(size_t)b * coef_stride + S.coef_off + S.tile_bit[j]] = rc;
    }
    // table[e] = sigma * prod_j (bit_j(e) ? e^{+i phi_j/2} : e^{-i phi_j/2})
    C *tab = dtab + (size_t)b * dtab_stride + S.dtab_off;
    const uint32_t size = 1u << S.k;
    const double sg = sigma;
    for (uint32_t e = threadIdx.x; e < size; e += blockDim.x) {
        double re = sg, im = 0.0;
        for (int j = 0; j < S.n_gated; ++j) {
            const double c = ph_c[j];
            const double s = ((e >> S.tile_bit[j]) & 1u) ? ph_s[j] : -ph_s[j];
            const double nr = re * c - im * s;
            const double ni = re * s + im * c;
            re = nr;
            im = ni;
        }
        C d;
        d.x = (T)re;
        d.y = (T)im;
        tab[e] = d;
    }
}

template <typename T>
cudaError_t launch_stage(const StageSlot *slots_dev, int n_slots, int n_qubits, int depth,
                         const double *params, int batch, RotCoef<T> *coefs, size_t coef_stride,
                         void *dtab, size_t dtab_stride, cudaStream_t s) {
    if (n_slots == 0 || batch == 0) return cudaSuccess;
    dim3 grid(n_slots, batch);
    k_stage<T><<<grid, 256, 0, s>>>(slots_dev, n_qubits, depth, params, coefs, coef_stride,
                                    static_cast<typename V2<T>::type *>(dtab), dtab_stride);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- tile pass

// Plans keep k - R <= 9, so a pass block has at most 512 threads.
constexpr int kPassMaxThreads = 512;

template <typename T>
struct GridEnv {
    using C = typename V2<T>::type;
    // first/last round straight from/to global memory: run_tile reads P, L
    // (this state's psi and lambda) and init_zero (start from |0...0>)
    static constexpr int kLoad = 1, kStore = 1;
    const PassDesc *d;          // shared-memory copy of the pass descriptor
    const RotCoef<T> *cf;       // shared-memory copy: coefficient rows of the pass's slots
    const C *dt;
    double *gout;   // this state's gradient partials
    uint64_t tile;
    C *P, *L;
    uint64_t base;
    uint32_t lowmask;
    int m, a;
    int init_zero;
    __device__ RotCoef<T> coef(int slot, int bit) const { return cf[slot * d->k + bit]; }
    __device__ C diag(int slot, uint32_t e) const { return dt[d->slot_dtab_off[slot] + e]; }
    static constexpr bool kDiagRow = true;
    __device__ const C *diag_row(int slot, uint32_t e0) const { return dt + d->slot_dtab_off[slot] + e0; }
    __device__ void grad(int slot, int bit, int comp, double v) const {
        gout[d->slot_grad_off[slot] + tile * (uint64_t)(2 * d->k) + bit * 2 + comp] = v;
    }
};

// Copies the pass descriptor and the pass's coefficient rows into shared
// memory, so the op interpreter reads them with shared-memory loads.
template <typename T>
__device__ __forceinline__ void stage_pass(const PassDesc *__restrict__ desc,
                                           const RotCoef<T> *__restrict__ cf, PassDesc *sd,
                                           RotCoef<T> *scf) {
    static_assert(sizeof(PassDesc) % 4 == 0, "descriptor copied in words");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(desc);
    uint32_t *dst = reinterpret_cast<uint32_t *>(sd);
    for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    const int k = sd->k;
    for (int i = threadIdx.x; i < sd->n_slots * k; i += blockDim.x)
        scf[i] = cf[sd->slot_coef_off[i / k] + (i % k)];
    __syncthreads();
}

// A backward tile outside the support of psi (its base has a bit of the
// backward zmask): psi is zero there, so its gradient partials are zero and
// its lambda is never read again; only the partials are written.
__device__ __forceinline__ void write_zero_partials(const PassDesc &d, double *gout, uint64_t tile) {
    const int k = d.k;
    for (int i = threadIdx.x; i < d.n_slots * 2 * k; i += blockDim.x) {
        const int slot = i / (2 * k), j = i % (2 * k);
        gout[d.slot_grad_off[slot] + tile * (uint64_t)(2 * k) + j] = 0.0;
    }
}

// A forward tile known to be zero (its base has a bit of zmask set): the
// pass maps it to zero, so it is written without being read or transformed.
template <typename C>
__device__ __forceinline__ void write_zero_tile(C *P, uint64_t base, uint32_t lowmask, int m, int a, int k) {
    const C z{};
    for (uint32_t e = threadIdx.x; e < (1u << k); e += blockDim.x)
        P[base | (e & lowmask) | ((uint64_t)(e >> m) << a)] = z;
}

// The first forward pass when it holds one slot: its only nonzero tile (base
// 0) starts as |0...0>, so the slot's scaled butterflies give each element
// the product of one factor per tile bit (|0> -> (1, v) in tan form, (v, 1)
// in cot form; an ungated bit stays 0), and the slot's diagonal (table entry
// and CZ sign) follows.  Written straight to global memory, no tile rounds.
template <typename T>
__device__ __forceinline__ void write_product_tile(const PassDesc &d, const RotCoef<T> *cf,
                                                   const typename V2<T>::type *dt,
                                                   typename V2<T>::type *P, uint64_t base,
                                                   uint32_t lowmask, int m, int a, int k) {
    using C = typename V2<T>::type;
    const uint32_t gated = d.slot_gated[0], cz = d.slot_czmask[0];
    const C *tab = dt + d.slot_dtab_off[0];
    for (uint32_t e = threadIdx.x; e < (1u << k); e += blockDim.x) {
        const uint64_t g = base | (e & lowmask) | ((uint64_t)(e >> m) << a);
        T f = T(1);
        for (int j = 0; j < k; ++j) {
            const uint32_t bit = (e >> j) & 1u;
            if (!((gated >> j) & 1u)) {
                if (bit) f = T(0);
                continue;
            }
            const RotCoef<T> rc = cf[j];
            if (bit ^ (uint32_t)rc.mode) f *= rc.v;
        }
        C y = tab[e];
        const uint32_t s = __popc((uint32_t)g & ((uint32_t)g >> 1) & cz) & 1u;
        y.x = flip_sign(y.x * f, s);
        y.y = flip_sign(y.y * f, s);
        P[g] = y;
    }
}

// One CTA per (tile, state): global -> shared (plain order), the pass
// program, shared -> global.
// Forward passes hold one buffer per thread: two blocks of 512 threads fit an
// SM (<= 64 registers); backward passes hold two.
template <typename T, int R, bool BWD>
__global__ void __launch_bounds__(kPassMaxThreads, (BWD || R > 4) ? 1 : 2)
k_pass(const PassDesc *__restrict__ desc, int init_zero, typename V2<T>::type *__restrict__ psi,
       typename V2<T>::type *__restrict__ lam, size_t stride, const RotCoef<T> *__restrict__ coefs,
       size_t coef_stride, const typename V2<T>::type *__restrict__ dtab, size_t dtab_stride,
       double *__restrict__ gpart, size_t grad_stride) {
    using C = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PassDesc sd;
    const int b = blockIdx.y;
    // dynamic shared memory: tile(s) | gradient scratch (backward) | coefficient rows
    const int kk = desc->k;
    const uint32_t size = tile_buf_elems(kk, (int)sizeof(C));   // padded tile buffer
    C *sp = reinterpret_cast<C *>(smem_raw);
    C *sl = sp + (BWD ? size : 0u);
    double *gsh = reinterpret_cast<double *>(sp + (BWD ? 2 * size : size));
    RotCoef<T> *scf = reinterpret_cast<RotCoef<T> *>(
        reinterpret_cast<unsigned char *>(gsh) +
        (BWD ? tile_grad_scratch_bytes((int)blockDim.x, kk) : 0));
    stage_pass<T>(desc, coefs + (size_t)b * coef_stride, &sd, scf);
    const PassDesc &d = sd;
    const int k = d.k, m = d.m, a = d.a;
    const int mid = a - m;
    const uint32_t lowmask = (1u << m) - 1u;
    C *P = psi + (size_t)b * stride;
    C *L = BWD ? lam + (size_t)b * stride : nullptr;
    const uint64_t tile = blockIdx.x;
    const uint64_t base = ((tile & ((1ull << mid) - 1ull)) << m) | ((tile >> mid) << (a + (k - m)));
    if (base & d.zmask) {   // block-uniform
        if (BWD) write_zero_partials(d, gpart + (size_t)b * grad_stride, tile);
        else write_zero_tile(P, base, lowmask, m, a, k);
        return;
    }
    if (!BWD && init_zero && d.n_slots == 1) {   // the tile at base 0
        write_product_tile<T>(d, scf, dtab + (size_t)b * dtab_stride, P, base, lowmask, m, a, k);
        return;
    }
    GridEnv<T> env{&sd, scf, dtab + (size_t)b * dtab_stride,
                   BWD ? gpart + (size_t)b * grad_stride : nullptr, tile, P, L, base, lowmask,
                   m, a, init_zero};
    run_tile<T, R, BWD>(d, d.ops, d.n_ops, base, sp, sl, gsh, env);
}

// Gradient scratch of a fixed-shape backward pass, rows of per-thread
// partials summed at the flush: one theta row per tile bit, the phi total row
// and one row per register bit.
template <typename T, int R>
__host__ __device__ inline size_t fixed_grad_scratch_bytes(int threads, int k) {
    return size_t(threads) * (k + 1 + R) * sizeof(T);
}

// Pass with a program shape fixed at compile time (run_tile_fixed); same
// staging and environment as k_pass, the gradient scratch as above.
template <typename T, int R, bool BWD, int... Codes>
__global__ void __launch_bounds__(kPassMaxThreads, (BWD || R > 4) ? 1 : 2)
k_pass_fixed(const PassDesc *__restrict__ desc, int init_zero, typename V2<T>::type *__restrict__ psi,
             typename V2<T>::type *__restrict__ lam, size_t stride,
             const RotCoef<T> *__restrict__ coefs, size_t coef_stride,
             const typename V2<T>::type *__restrict__ dtab, size_t dtab_stride,
             double *__restrict__ gpart, size_t grad_stride) {
    using C = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PassDesc sd;
    const int b = blockIdx.y;
    const int kk = desc->k;
    const uint32_t size = tile_buf_elems(kk, (int)sizeof(C));
    C *sp = reinterpret_cast<C *>(smem_raw);
    C *sl = sp + (BWD ? size : 0u);
    double *gsh = reinterpret_cast<double *>(sp + (BWD ? 2 * size : size));
    RotCoef<T> *scf = reinterpret_cast<RotCoef<T> *>(
        reinterpret_cast<unsigned char *>(gsh) +
        (BWD ? fixed_grad_scratch_bytes<T, R>((int)blockDim.x, kk) : 0));
    stage_pass<T>(desc, coefs + (size_t)b * coef_stride, &sd, scf);
    const PassDesc &d = sd;
    const int k = d.k, m = d.m, a = d.a;
    const uint64_t tile = blockIdx.x;
    const int mid = a - m;
    const uint64_t base = ((tile & ((1ull << mid) - 1ull)) << m) | ((tile >> mid) << (a + (k - m)));
    const uint32_t lowmask = (1u << m) - 1u;
    if (base & d.zmask) {   // block-uniform
        if (BWD) write_zero_partials(d, gpart + (size_t)b * grad_stride, tile);
        else write_zero_tile(psi + (size_t)b * stride, base, lowmask, m, a, k);
        return;
    }
    if (!BWD && init_zero && d.n_slots == 1) {   // the tile at base 0
        write_product_tile<T>(d, scf, dtab + (size_t)b * dtab_stride, psi + (size_t)b * stride, base,
                              lowmask, m, a, k);
        return;
    }
    GridEnv<T> env{&sd, scf, dtab + (size_t)b * dtab_stride,
                   BWD ? gpart + (size_t)b * grad_stride : nullptr, tile, psi + (size_t)b * stride,
                   BWD ? lam + (size_t)b * stride : nullptr, base, lowmask, m, a, init_zero};
    run_tile_fixed<T, R, BWD, GridEnv<T>, Codes...>(d, d.ops, base, sp, sl, gsh, env);
}

namespace {

using FixedLaunch = cudaError_t (*)(const PassDesc *, const PassDesc &, int, int, void *, void *,
                                    size_t, const void *, size_t, const void *, size_t, double *,
                                    size_t, int, cudaStream_t);

template <typename T, int R, bool BWD, int... Codes>
cudaError_t launch_fixed(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits, int batch,
                         void *psi, void *lam, size_t stride, const void *coefs,
                         size_t coef_stride, const void *dtab, size_t dtab_stride, double *gpart,
                         size_t grad_stride, int init_zero, cudaStream_t s) {
    using C = typename V2<T>::type;
    const int threads = 1 << (dh.k - dh.R);
    size_t smem = pass_smem_bytes(dh, BWD, sizeof(C));
    if (BWD) smem += fixed_grad_scratch_bytes<T, R>(threads, dh.k) - tile_grad_scratch_bytes(threads, dh.k);
    auto kern = k_pass_fixed<T, R, BWD, Codes...>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(1ull << (n_qubits - dh.k)), batch);
    kern<<<grid, threads, smem, s>>>(desc_dev, init_zero, static_cast<C *>(psi),
                                     static_cast<C *>(lam), stride,
                                     static_cast<const RotCoef<T> *>(coefs), coef_stride,
                                     static_cast<const C *>(dtab), dtab_stride, gpart, grad_stride);
    return cudaGetLastError();
}

struct FixedEntry {
    int elem_bytes, R;
    bool backward;
    std::vector<int> codes;
    FixedLaunch fn;
};

#define VQE_RD(c) prog_round(c)
#define VQE_B kProgBF
#define VQE_D kProgDiag
#define VQE_F kProgFlush
#define VQE_FWD(TT, RR, ...) \
    FixedEntry{int(2 * sizeof(TT)), RR, false, std::vector<int>{__VA_ARGS__}, &launch_fixed<TT, RR, false, __VA_ARGS__>}
#define VQE_BWD(TT, RR, ...) \
    FixedEntry{int(2 * sizeof(TT)), RR, true, std::vector<int>{__VA_ARGS__}, &launch_fixed<TT, RR, true, __VA_ARGS__>}

// The pass program shapes of the default plans (tiles of 2^11; FP32 with 16
// amplitudes per thread: chunks 0, 4, 7; FP64 with 8: chunks 0, 3, 6, 8),
// forward and backward, and of FP64 plans with 2^12 tiles (chunks 0, 3, 6, 9)
// as the 32-qubit plan uses them.
const std::vector<FixedEntry> &fixed_programs() {
    static const std::vector<FixedEntry> table = {
        VQE_FWD(float, 4, VQE_RD(7), VQE_B, VQE_RD(4), VQE_B, VQE_D, VQE_RD(7)),
        VQE_FWD(float, 4, VQE_RD(7), VQE_B, VQE_RD(4), VQE_B, VQE_RD(0), VQE_B, VQE_D, VQE_RD(7)),
        VQE_FWD(float, 4, VQE_RD(7), VQE_B, VQE_RD(4), VQE_B, VQE_RD(0), VQE_B, VQE_D, VQE_B,
                VQE_RD(4), VQE_B, VQE_RD(7), VQE_B, VQE_D),
        VQE_FWD(float, 4, VQE_RD(7), VQE_B, VQE_RD(4), VQE_B, VQE_D, VQE_B, VQE_RD(7), VQE_B, VQE_D),
        VQE_FWD(float, 4, VQE_RD(7), VQE_B, VQE_D, VQE_B, VQE_D),
        VQE_FWD(float, 4, VQE_RD(7), VQE_B, VQE_D),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_D, VQE_RD(8)),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_RD(0), VQE_B,
                VQE_D, VQE_RD(8)),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_RD(0), VQE_B,
                VQE_D, VQE_B, VQE_RD(3), VQE_B, VQE_RD(6), VQE_B, VQE_RD(8), VQE_B, VQE_D),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_D, VQE_B,
                VQE_RD(6), VQE_B, VQE_RD(8), VQE_B, VQE_D),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_RD(6), VQE_B, VQE_D, VQE_B, VQE_RD(8), VQE_B, VQE_D),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_RD(6), VQE_B, VQE_D, VQE_RD(8)),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_D, VQE_B, VQE_D),
        VQE_FWD(double, 3, VQE_RD(8), VQE_B, VQE_D),
        VQE_BWD(float, 4, VQE_RD(7), VQE_RD(4), VQE_D, VQE_B, VQE_RD(7), VQE_B, VQE_F),
        VQE_BWD(float, 4, VQE_RD(7), VQE_RD(0), VQE_D, VQE_B, VQE_RD(4), VQE_B, VQE_RD(7), VQE_B, VQE_F),
        VQE_BWD(float, 4, VQE_RD(7), VQE_D, VQE_B, VQE_RD(4), VQE_B, VQE_RD(0), VQE_B, VQE_F, VQE_D,
                VQE_B, VQE_RD(4), VQE_B, VQE_RD(7), VQE_B, VQE_F),
        VQE_BWD(float, 4, VQE_RD(7), VQE_D, VQE_B, VQE_RD(4), VQE_B, VQE_F, VQE_D, VQE_B, VQE_RD(7),
                VQE_B, VQE_F),
        VQE_BWD(float, 4, VQE_RD(7), VQE_D, VQE_B, VQE_F, VQE_D, VQE_B, VQE_F),
        VQE_BWD(float, 4, VQE_RD(7), VQE_D, VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_RD(3), VQE_D, VQE_B, VQE_RD(6), VQE_B, VQE_RD(8), VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_RD(0), VQE_D, VQE_B, VQE_RD(3), VQE_B, VQE_RD(6), VQE_B,
                VQE_RD(8), VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_D, VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_RD(0),
                VQE_B, VQE_F, VQE_D, VQE_B, VQE_RD(3), VQE_B, VQE_RD(6), VQE_B, VQE_RD(8), VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_D, VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_F, VQE_D,
                VQE_B, VQE_RD(6), VQE_B, VQE_RD(8), VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_D, VQE_B, VQE_RD(6), VQE_B, VQE_F, VQE_D, VQE_B, VQE_RD(8),
                VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_RD(6), VQE_D, VQE_B, VQE_RD(8), VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_D, VQE_B, VQE_F, VQE_D, VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(8), VQE_D, VQE_B, VQE_F),
        // FP64 with 2^12-amplitude tiles (512 threads): three qubit groups
        // instead of four at 32 qubits, so fewer slots (diagonal ops) per layer
        VQE_FWD(double, 3, VQE_RD(9), VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_RD(0), VQE_B,
                VQE_D, VQE_B, VQE_RD(3), VQE_B, VQE_RD(6), VQE_B, VQE_RD(9), VQE_B, VQE_D),
        VQE_FWD(double, 3, VQE_RD(9), VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_RD(0), VQE_B,
                VQE_D, VQE_RD(9)),
        VQE_BWD(double, 3, VQE_RD(9), VQE_D, VQE_B, VQE_RD(6), VQE_B, VQE_RD(3), VQE_B, VQE_RD(0),
                VQE_B, VQE_F, VQE_D, VQE_B, VQE_RD(3), VQE_B, VQE_RD(6), VQE_B, VQE_RD(9), VQE_B, VQE_F),
        VQE_BWD(double, 3, VQE_RD(9), VQE_RD(0), VQE_D, VQE_B, VQE_RD(3), VQE_B, VQE_RD(6), VQE_B,
                VQE_RD(9), VQE_B, VQE_F),
    };
    return table;
}
#undef VQE_FWD
#undef VQE_BWD
#undef VQE_RD
#undef VQE_B
#undef VQE_D
#undef VQE_F

// The fixed-shape launcher of a pass program, or null.
FixedLaunch find_fixed(const PassDesc &dh, size_t elem_bytes, bool backward) {
    std::vector<int> codes;
    codes.reserve(dh.n_ops);
    for (int i = 0; i < dh.n_ops; ++i) {
        const PassOp &op = dh.ops[i];
        if (op.kind == OP_ROUND) codes.push_back(prog_round(op.chunk));
        else if (op.kind == OP_BF) codes.push_back(kProgBF);
        else if (op.kind == OP_DIAG) codes.push_back(kProgDiag);
        else if (op.kind == OP_FLUSH) codes.push_back(kProgFlush);
        else return nullptr;
    }
    for (const FixedEntry &f : fixed_programs())
        if (f.elem_bytes == int(elem_bytes) && f.R == dh.R && f.backward == backward && f.codes == codes)
            return f.fn;
    return nullptr;
}

}  // namespace

int pass_threads(const PassDesc &d) { return 1 << (d.k - d.R); }

size_t pass_smem_bytes(const PassDesc &d, bool backward, size_t elem_bytes) {
    size_t tiles = size_t(tile_buf_elems(d.k, (int)elem_bytes)) * elem_bytes * (backward ? 2 : 1);
    size_t gsh = backward ? tile_grad_scratch_bytes(pass_threads(d), d.k) : 0;
    const size_t coef = elem_bytes == 16 ? sizeof(RotCoef<double>) : sizeof(RotCoef<float>);
    return tiles + gsh + size_t(d.n_slots) * d.k * coef;
}

template <typename T, int R, bool BWD>
static cudaError_t launch_pass_r(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits,
                                 int batch, void *psi, void *lam, size_t stride,
                                 const RotCoef<T> *coefs, size_t coef_stride, const void *dtab,
                                 size_t dtab_stride, double *gpart, size_t grad_stride,
                                 int init_zero, cudaStream_t s) {
    using C = typename V2<T>::type;
    const int threads = pass_threads(dh);
    if (threads > kPassMaxThreads) return cudaErrorInvalidConfiguration;
    const size_t smem = pass_smem_bytes(dh, BWD, sizeof(C));
    auto kern = k_pass<T, R, BWD>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(1ull << (n_qubits - dh.k)), batch);
    kern<<<grid, threads, smem, s>>>(desc_dev, init_zero, static_cast<C *>(psi),
                                     static_cast<C *>(lam), stride, coefs, coef_stride,
                                     static_cast<const C *>(dtab), dtab_stride, gpart, grad_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass(const PassDesc *desc_dev, const PassDesc &dh, int n_qubits, int batch,
                        void *psi, void *lam, size_t stride, const RotCoef<T> *coefs,
                        size_t coef_stride, const void *dtab, size_t dtab_stride,
                        double *gpart, size_t grad_stride, bool backward, int init_zero,
                        cudaStream_t s) {
    // a program of a known shape runs unrolled
    if (FixedLaunch f = find_fixed(dh, 2 * sizeof(T), backward))
        return f(desc_dev, dh, n_qubits, batch, psi, backward ? lam : nullptr, stride, coefs,
                 coef_stride, dtab, dtab_stride, gpart, grad_stride, init_zero, s);
#define VQE_PASS_CASE(RR)                                                                       \
    case RR:                                                                                    \
        return backward ? launch_pass_r<T, RR, true>(desc_dev, dh, n_qubits, batch, psi, lam,   \
                                                     stride, coefs, coef_stride, dtab,          \
                                                     dtab_stride, gpart, grad_stride, 0, s)     \
                        : launch_pass_r<T, RR, false>(desc_dev, dh, n_qubits, batch, psi,       \
                                                      nullptr, stride, coefs, coef_stride,      \
                                                      dtab, dtab_stride, gpart, grad_stride,    \
                                                      init_zero, s);
    switch (dh.R) {
        VQE_PASS_CASE(1)
        VQE_PASS_CASE(2)
        VQE_PASS_CASE(3)
        VQE_PASS_CASE(4)
        case 5:   // forward only (the backward buffers would not fit in registers)
            if (backward) return cudaErrorInvalidValue;
            return launch_pass_r<T, 5, false>(desc_dev, dh, n_qubits, batch, psi, nullptr, stride,
                                             coefs, coef_stride, dtab, dtab_stride, gpart,
                                             grad_stride, init_zero, s);
        default:
            return cudaErrorInvalidValue;
    }
#undef VQE_PASS_CASE
}

// ---------------------------------------------------------------- one gate per pass

template <typename T>
__global__ void k_gate_ry(typename V2<T>::type *psi, size_t stride, int n, int q,
                          const double *params, int pidx, int pstride) {
    using C = typename V2<T>::type;
    __shared__ T cs[2];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) {
        double s, c;
        sincos(0.5 * params[(size_t)b * pstride + pidx], &s, &c);
        cs[0] = (T)c;
        cs[1] = (T)s;
    }
    __syncthreads();
    const T c = cs[0], s = cs[1];
    C *P = psi + (size_t)b * stride;
    const uint64_t half = 1ull << (n - 1);
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < half;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i0 = ((p >> q) << (q + 1)) | (p & ((1ull << q) - 1));
        const uint64_t i1 = i0 | (1ull << q);
        const C x = P[i0], y = P[i1];
        C nx, ny;
        nx.x = c * x.x - s * y.x;  nx.y = c * x.y - s * y.y;
        ny.x = s * x.x + c * y.x;  ny.y = s * x.y + c * y.y;
        P[i0] = nx;
        P[i1] = ny;
    }
}

template <typename T>
__global__ void k_gate_rz(typename V2<T>::type *psi, size_t stride, int n, int q,
                          const double *params, int pidx, int pstride) {
    using C = typename V2<T>::type;
    __shared__ T cs[2];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) {
        double s, c;
        sincos(0.5 * params[(size_t)b * pstride + pidx], &s, &c);
        cs[0] = (T)c;
        cs[1] = (T)s;
    }
    __syncthreads();
    const T c = cs[0], s0 = cs[1];
    C *P = psi + (size_t)b * stride;
    const uint64_t dim = 1ull << n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const T s = ((i >> q) & 1) ? s0 : -s0;   // e^{+-i phi/2}
        const C x = P[i];
        C y;
        y.x = x.x * c - x.y * s;
        y.y = x.x * s + x.y * c;
        P[i] = y;
    }
}

template <typename T>
__global__ void k_gate_cz(typename V2<T>::type *psi, size_t stride, int n, int q) {
    using C = typename V2<T>::type;
    C *P = psi + (size_t)blockIdx.y * stride;
    const uint64_t dim = 1ull << n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (((i >> q) & 3ull) == 3ull) {
            C x = P[i];
            x.x = -x.x;
            x.y = -x.y;
            P[i] = x;
        }
    }
}

template <typename T>
__global__ void k_zero_state(typename V2<T>::type *psi, size_t stride, int n) {
    using C = typename V2<T>::type;
    C *P = psi + (size_t)blockIdx.y * stride;
    const uint64_t dim = 1ull << n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        C x;
        x.x = (i == 0) ? T(1) : T(0);
        x.y = T(0);
        P[i] = x;
    }
}

// Grid of a grid-stride kernel: one thread per work item, at most 16 blocks
// per SM of the current device.
static unsigned grid_for(uint64_t work, int threads) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    uint64_t g = (work + threads - 1) / threads;
    if (g > uint64_t(sms) * 16) g = uint64_t(sms) * 16;
    if (g == 0) g = 1;
    return (unsigned)g;
}

template <typename T>
cudaError_t launch_gate_ry(void *psi, size_t stride, int n, int batch, int q, const double *params,
                           int pidx, int pstride, cudaStream_t s) {
    dim3 grid(grid_for(1ull << (n - 1), 256), batch);
    k_gate_ry<T><<<grid, 256, 0, s>>>(static_cast<typename V2<T>::type *>(psi), stride, n, q,
                                      params, pidx, pstride);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gate_rz(void *psi, size_t stride, int n, int batch, int q, const double *params,
                           int pidx, int pstride, cudaStream_t s) {
    dim3 grid(grid_for(1ull << n, 256), batch);
    k_gate_rz<T><<<grid, 256, 0, s>>>(static_cast<typename V2<T>::type *>(psi), stride, n, q,
                                      params, pidx, pstride);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gate_cz(void *psi, size_t stride, int n, int batch, int q, cudaStream_t s) {
    dim3 grid(grid_for(1ull << n, 256), batch);
    k_gate_cz<T><<<grid, 256, 0, s>>>(static_cast<typename V2<T>::type *>(psi), stride, n, q);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_init_zero_state(void *psi, size_t stride, int n, int batch, cudaStream_t s) {
    dim3 grid(grid_for(1ull << n, 256), batch);
    k_zero_state<T><<<grid, 256, 0, s>>>(static_cast<typename V2<T>::type *>(psi), stride, n);
    return cudaGetLastError();
}

#define VQE_INSTANTIATE(T)                                                                      \
    template cudaError_t launch_stage<T>(const StageSlot *, int, int, int, const double *, int, \
                                         RotCoef<T> *, size_t, void *, size_t, cudaStream_t);   \
    template cudaError_t launch_pass<T>(const PassDesc *, const PassDesc &, int, int, void *,   \
                                        void *, size_t, const RotCoef<T> *, size_t,             \
                                        const void *, size_t, double *, size_t, bool, int,      \
                                        cudaStream_t);                                          \
    template cudaError_t launch_gate_ry<T>(void *, size_t, int, int, int, const double *, int,  \
                                           int, cudaStream_t);                                  \
    template cudaError_t launch_gate_rz<T>(void *, size_t, int, int, int, const double *, int,  \
                                           int, cudaStream_t);                                  \
    template cudaError_t launch_gate_cz<T>(void *, size_t, int, int, int, cudaStream_t);        \
    template cudaError_t launch_init_zero_state<T>(void *, size_t, int, int, cudaStream_t);

VQE_INSTANTIATE(float)
VQE_INSTANTIATE(double)

}  // namespace vqe
