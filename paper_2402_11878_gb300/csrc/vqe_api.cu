// Host side of libvqe_gb300: the C ABI of include/vqe.h, Hamiltonian
// canonicalisation and cutoff, term grouping, the tile-pass planner, device
// buffers and the evaluation pipelines.  All numerical work runs in the
// kernels of k_layers.cu and k_energy.cu; this file only plans and launches.
#include "vqe.h"
#include "vqe_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

using namespace vqe;

namespace {

struct Group {        // one qubit group = the tile bits of one kind of pass
    int k, m, a;      // tile bits, low run bits, start of the high range
    uint32_t gated;   // tile bits that carry this group's qubits
    int qubit_of(int j) const { return j < m ? j : a + (j - m); }
};

struct PlanOptions {
    int tile_bits_max = 0;  // 0: default (11 for C128 and C64)
    int run_bits = 0;       // 0: default (2 for C128, 3 for C64)
    int reg_bits = 0;       // 0: default (3 for C128, 4 for C64)
};

struct PassPlan {
    int group;
    std::vector<int> layers;  // one slot per layer
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void swap(DevBuf &o) {
        std::swap(p, o.p);
        std::swap(bytes, o.bytes);
    }
};

// The device form of one Hamiltonian plan.  vqe_set_hamiltonian and
// vqe_slim build a new one beside the handle's and swap it in only when every
// step has succeeded, so a failure leaves the previous plan in use.
struct HamDev {
    DevBuf d_groups, d_tz, d_tc;
    int n_groups = 0;
    uint64_t n_groups_nonempty = 0;
    // windowed expectation: tile windows, their group lists, groups too wide for any window
    std::vector<WinDesc> wins;
    DevBuf d_wgroups, d_wterms, d_whoff, d_wide;
    int n_wide = 0;
    // lambda = H psi: form 0 = one global sweep gathering psi_{i^x} per
    // group; 1 = over the windows above (possible when every group fits a
    // window); 2 = bit-ordered sweeps (SweepDesc; possible when every group's
    // merged terms fit a sweep).  apply_default is the form of mode -1;
    // apply_form the one in use.
    bool win_possible = false, sweep_possible = false;
    int apply_default = 0, apply_form = 0;
    int win_tiles = 0;   // columns of all windows per state
    std::vector<SweepDesc> sweeps;
    DevBuf d_sorder, d_sgroups, d_spat, d_stz, d_sta, d_stb;
    // diagonal of H (one T per basis state), built when it fits in a quarter
    // of the free device memory; null: the x = 0 terms are evaluated inline
    DevBuf d_hdiag, d_hdiag_z, d_hdiag_c;
    bool hdiag_ok = false;
    const void *hdiag() const { return hdiag_ok ? d_hdiag.p : nullptr; }
    void release() {
        for (DevBuf *b : {&d_groups, &d_tz, &d_tc, &d_wgroups, &d_wterms, &d_whoff, &d_wide,
                          &d_hdiag, &d_hdiag_z, &d_hdiag_c, &d_sorder, &d_sgroups, &d_spat, &d_stz,
                          &d_sta, &d_stb})
            b->release();
    }
};

// Form of apply-H for vqe_set_apply_mode's mode: -1 the plan's default; a
// form the Hamiltonian cannot use falls back to the global sweep.
int resolve_apply_form(int mode, const HamDev &d) {
    if (mode < 0) return d.apply_default;
    if (mode == 1 && d.win_possible) return 1;
    if (mode == 2 && d.sweep_possible) return 2;
    return 0;
}

}  // namespace

struct vqe_ctx {
    int n = 0, depth = 0;
    vqe_precision prec = VQE_C64;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;

    // Hamiltonian (host)
    std::vector<uint64_t> cx, cz;  // canonical terms
    std::vector<double> cc;
    std::vector<uint8_t> keep;
    bool ham_set = false;
    bool state_valid = false;
    vqe_stats stats{};

    // Hamiltonian plan (device); built into a temporary and swapped in whole
    HamDev hd;

    // ansatz plans: [0] energy evaluations (forward only), [1] gradients (forward + backward)
    struct DevPlan {
        PlanOptions opts;
        std::vector<Group> groups;
        std::vector<PassDesc> fwd, bwd;
        DevBuf d_fwd, d_bwd, d_stage, d_goff, d_gcnt, d_gstep;
        int n_stage = 0;
        size_t coef_stride = 0, dtab_stride = 0, grad_stride = 0;
        void release() {
            for (DevBuf *b : {&d_fwd, &d_bwd, &d_stage, &d_goff, &d_gcnt, &d_gstep}) b->release();
        }
    } plan[2];
    int n_params = 0;

    // workspace and scratch
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    DevBuf ws_own;
    DevBuf d_params, d_coefs, d_dtab, d_gpart, d_epart, d_out;
    DevBuf d_sctr;   // chunk counters of the sweep form of apply-H
    DevBuf hb_params, hb_e, hb_n, hb_g;   // device copies for the host-buffer batch calls
    int scratch_batch = 0;

    // particle-conserving ansatz (vqe_create_pc); ansatz 0 = hardware-efficient
    int ansatz = 0;
    int n_elec = 0;
    uint64_t hf_index = 0;
    std::vector<int> exc;                // 4 per excitation, in the order of application
    std::vector<ExcPass> pc_passes;
    DevBuf d_pc_gates, d_pc_hoff;
    int pc_k = 0;

    // apply-H form: -1 automatic, 0 one global sweep, 1 windowed (where possible)
    int apply_mode = -1;
    int sms = 0;

    // event timing (vqe_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Mark { int group; int launches; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    size_t ev_used = 0;
    vqe_kernel_times times{};

    size_t elem_bytes() const { return prec == VQE_C128 ? 16 : 8; }
    size_t state_elems() const { return size_t(1) << n; }
    size_t state_bytes() const { return state_elems() * elem_bytes(); }
};

namespace {

vqe_status fail(vqe_ctx *h, vqe_status st, const std::string &msg) {
    if (h) h->err = msg;
    return st;
}

vqe_status cuda_fail(vqe_ctx *h, cudaError_t e, const char *where) {
    return fail(h, VQE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define VQE_CUDA(h, call)                                            \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);     \
    } while (0)

// Allocation failures injected by vqe_testing_fail_allocations: -1 = none,
// else the number of allocations that still succeed before every later one
// fails.
std::atomic<int> g_alloc_budget{-1};

bool injected_alloc_failure() {
    int b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return true;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return false;
    }
    return false;
}

// Grows b to at least `bytes`.  The new buffer is allocated before the old
// one is released, so a failed allocation leaves b as it was.
vqe_status ensure(vqe_ctx *h, DevBuf &b, size_t bytes, const char *what) {
    if (b.bytes >= bytes && b.p) return VQE_OK;
    if (bytes == 0) return VQE_OK;
    if (injected_alloc_failure())
        return fail(h, VQE_ERR_OOM, std::string("injected allocation failure for ") + what);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, VQE_ERR_OOM, std::string("cudaMalloc failed for ") + what);
    }
    b.release();
    b.p = p;
    b.bytes = bytes;
    return VQE_OK;
}

template <typename V>
vqe_status upload(vqe_ctx *h, DevBuf &b, const std::vector<V> &v, const char *what) {
    vqe_status st = ensure(h, b, std::max<size_t>(v.size() * sizeof(V), 16), what);
    if (st != VQE_OK) return st;
    if (!v.empty())
        VQE_CUDA(h, cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice,
                                    h->stream));
    VQE_CUDA(h, cudaStreamSynchronize(h->stream));
    return VQE_OK;
}

// ---------------------------------------------------------------- event timing

cudaEvent_t next_event(vqe_ctx *h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

// Opens a timed interval for kernel group g; returns the mark index or -1.
int prof_begin(vqe_ctx *h, int g) {
    if (!h->prof) return -1;
    cudaEvent_t a = next_event(h), b = next_event(h);
    if (!a || !b) return -1;
    cudaEventRecord(a, h->stream);
    h->marks.push_back({g, 0, a, b});
    return int(h->marks.size()) - 1;
}

void prof_end(vqe_ctx *h, int mark, int launches) {
    if (mark < 0) return;
    h->marks[mark].launches = launches;
    cudaEventRecord(h->marks[mark].b, h->stream);
}

vqe_status prof_collect(vqe_ctx *h) {
    if (h->marks.empty()) return VQE_OK;
    VQE_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto &m : h->marks) {
        float ms = 0.f;
        VQE_CUDA(h, cudaEventElapsedTime(&ms, m.a, m.b));
        h->times.ms[m.group] += ms;
        h->times.launches[m.group] += uint64_t(m.launches);
        h->times.chunks[m.group] += 1;
    }
    h->marks.clear();
    h->ev_used = 0;
    return VQE_OK;
}

// ---------------------------------------------------------------- planner

// Qubit groups: the low kmax qubits, then high groups of at most kmax - mrun
// qubits (balanced).  Every high tile is filled up to kmax bits with low
// qubits, so its contiguous runs hold 2^(kmax - h) >= 2^mrun amplitudes.
std::vector<Group> plan_groups(int n, int kmax, int mrun) {
    std::vector<Group> gs;
    if (n <= kmax) {
        gs.push_back({n, n, n, (n >= 32 ? 0xffffffffu : ((1u << n) - 1u))});
        return gs;
    }
    gs.push_back({kmax, kmax, kmax, (1u << kmax) - 1u});
    const int rest = n - kmax, hmax = kmax - mrun;
    const int ng = (rest + hmax - 1) / hmax;
    int a = kmax;
    for (int j = 0; j < ng; ++j) {
        const int hj = rest / ng + (j < rest % ng ? 1 : 0);
        const int m = kmax - hj;
        gs.push_back({kmax, m, a, ((1u << kmax) - 1u) & ~((1u << m) - 1u)});
        a += hj;
    }
    return gs;
}


struct Round {
    int chunk;
    std::vector<PassOp> ops;
};

// Zero fields take the defaults, the fastest plans measured on GB300 for the
// forward and the adjoint passes: tiles of 2^11 amplitudes; FP64 with runs of
// at least 4 amplitudes and 8 amplitudes per thread (256 threads), FP32 with
// runs of at least 8 and 16 per thread (128 threads).  Plans with fewer
// passes (larger tiles, or 32 amplitudes per thread) measured slower.
PlanOptions resolve(const PlanOptions &o, vqe_precision prec) {
    PlanOptions r;
    r.tile_bits_max = o.tile_bits_max ? o.tile_bits_max : 11;
    r.run_bits = o.run_bits ? o.run_bits : (prec == VQE_C128 ? 2 : 3);
    r.reg_bits = o.reg_bits ? o.reg_bits : (prec == VQE_C128 ? 3 : 4);
    return r;
}

bool options_valid(const PlanOptions &o, vqe_precision prec, std::string &err) {
    const PlanOptions r = resolve(o, prec);
    if (r.tile_bits_max < 1 || r.tile_bits_max > kMaxTileBits) err = "tile_bits_max out of 1..14";
    else if (r.reg_bits < 1 || r.reg_bits > 5) err = "reg_bits out of 1..5";
    else if (r.tile_bits_max - r.reg_bits > 9) err = "tile_bits_max - reg_bits must be <= 9 (512 threads)";
    else if (r.run_bits < 1 || r.run_bits >= r.tile_bits_max) err = "run_bits out of 1..tile_bits_max-1";
    else {
        const size_t elem = prec == VQE_C128 ? 16 : 8;
        const size_t warps = ((size_t(1) << (r.tile_bits_max - std::min(r.reg_bits, r.tile_bits_max))) + 31) / 32;
        const size_t bufs = r.reg_bits > 4 ? 1 : 2;   // 32-amplitude plans are forward only
        const size_t smem = bufs * tile_buf_elems(r.tile_bits_max, int(elem)) * elem +
                            warps * r.tile_bits_max * 16;
        if (smem > 227 * 1024) err = "tile does not fit in shared memory";
    }
    return err.empty();
}

struct HostPlan {
    std::vector<Group> groups;
    std::vector<PassDesc> fwd, bwd;
    std::vector<int> pass_tiles_log2;
    std::vector<StageSlot> stage;
    std::vector<int> goff, gcnt, gstep;
    size_t coef_stride = 0, dtab_stride = 0, grad_stride = 0;
    int n_params = 0;
};

// Rounds of one pass: per slot, the gated tile bits are covered by register
// chunks; chunk order alternates between slots so that consecutive slots
// share the chunk at their boundary (the diagonal sits there).
std::vector<Round> make_rounds(int k, int R, const std::vector<uint32_t> &slot_gated) {
    std::vector<int> chunks;
    for (int c = 0; c < k; c += R) chunks.push_back(std::min(c, k - R));
    const int top = chunks.back();
    std::vector<Round> rounds;
    for (size_t s = 0; s < slot_gated.size(); ++s) {
        std::vector<uint8_t> cmask(chunks.size(), 0);
        uint32_t left = slot_gated[s];
        for (size_t ci = 0; ci < chunks.size(); ++ci) {
            for (int j = 0; j < R; ++j) {
                const int bit = chunks[ci] + j;
                if ((left >> bit) & 1u) {
                    cmask[ci] |= uint8_t(1u << j);
                    left &= ~(1u << bit);
                }
            }
        }
        std::vector<size_t> order;
        for (size_t ci = 0; ci < chunks.size(); ++ci)
            if (cmask[ci]) order.push_back(ci);
        if (s % 2 == 0) std::reverse(order.begin(), order.end());
        for (size_t ci : order) {
            if (rounds.empty() || rounds.back().chunk != chunks[ci]) rounds.push_back({chunks[ci], {}});
            rounds.back().ops.push_back({OP_BF, 0, cmask[ci], uint8_t(s)});
        }
        rounds.back().ops.push_back({OP_DIAG, 0, 0, uint8_t(s)});
    }
    if (rounds.back().chunk != top) rounds.push_back({top, {}});
    return rounds;
}

int count_ops(const std::vector<Round> &rs) {
    int c = 0;
    for (auto &r : rs) c += 1 + int(r.ops.size());
    return c;
}

void emit_forward(PassDesc &d, const std::vector<Round> &rs) {
    int k = 0;
    for (auto &r : rs) {
        d.ops[k++] = {OP_ROUND, uint8_t(r.chunk), 0, 0};
        for (auto &o : r.ops) d.ops[k++] = o;
    }
    d.n_ops = k;
}

void emit_backward(PassDesc &d, const std::vector<Round> &rs, int n_slots) {
    std::vector<int> bf_left(n_slots, 0);
    for (auto &r : rs)
        for (auto &o : r.ops)
            if (o.kind == OP_BF) bf_left[o.slot]++;
    int k = 0;
    for (auto it = rs.rbegin(); it != rs.rend(); ++it) {
        d.ops[k++] = {OP_ROUND, uint8_t(it->chunk), 0, 0};
        for (auto o = it->ops.rbegin(); o != it->ops.rend(); ++o) {
            d.ops[k++] = *o;
            if (o->kind == OP_BF && --bf_left[o->slot] == 0)
                d.ops[k++] = {OP_FLUSH, 0, 0, o->slot};
        }
    }
    d.n_ops = k;
}

bool make_plan(int n, int D, vqe_precision prec, const PlanOptions &opt, HostPlan &hp,
               std::string &err) {
    hp = HostPlan{};
    if (!options_valid(opt, prec, err)) return false;
    const PlanOptions o = resolve(opt, prec);
    hp.groups = plan_groups(n, o.tile_bits_max, o.run_bits);
    const int ng = int(hp.groups.size());
    const int Rdef = o.reg_bits;

    // Layer events in zigzag order; consecutive events of one group merge.
    std::vector<PassPlan> plans;
    for (int l = 0; l < D; ++l) {
        for (int jj = 0; jj < ng; ++jj) {
            const int g = (l % 2 == 0) ? jj : ng - 1 - jj;
            if (!plans.empty() && plans.back().group == g) plans.back().layers.push_back(l);
            else plans.push_back({g, {l}});
        }
    }
    // Split passes whose program would not fit.
    std::vector<PassPlan> split;
    for (auto &p : plans) {
        const Group &G = hp.groups[p.group];
        const int R = std::min(Rdef, G.k);
        PassPlan cur{p.group, {}};
        for (int l : p.layers) {
            cur.layers.push_back(l);
            std::vector<uint32_t> gm(cur.layers.size(), G.gated);
            const int nb = count_ops(make_rounds(G.k, R, gm)) + int(cur.layers.size());
            if (int(cur.layers.size()) > kMaxSlots || nb > kMaxOps) {
                cur.layers.pop_back();
                split.push_back(cur);
                cur.layers = {l};
            }
        }
        split.push_back(cur);
    }
    plans.swap(split);

    const int np = int(plans.size());
    hp.fwd.assign(np, PassDesc{});
    hp.bwd.assign(np, PassDesc{});
    hp.pass_tiles_log2.assign(np, 0);
    // slot ids in global order and where RY_l(q) lives
    std::vector<std::vector<int>> slot_of(D, std::vector<int>(n, -1));
    std::vector<std::pair<int, int>> slot_pos;   // global slot id -> (pass, slot)
    for (int p = 0; p < np; ++p) {
        const Group &G = hp.groups[plans[p].group];
        for (size_t s = 0; s < plans[p].layers.size(); ++s) {
            const int gid = int(slot_pos.size());
            slot_pos.push_back({p, int(s)});
            for (int j = 0; j < G.k; ++j)
                if ((G.gated >> j) & 1u) slot_of[plans[p].layers[s]][G.qubit_of(j)] = gid;
        }
    }
    for (int l = 0; l < D; ++l)
        for (int q = 0; q < n; ++q)
            if (slot_of[l][q] < 0) {
                err = "planner left a qubit uncovered";
                return false;
            }

    std::vector<StageSlot> stage;
    size_t coef_off = 0, dtab_off = 0, grad_off = 0;
    std::vector<size_t> slot_grad_off(slot_pos.size());
    for (int p = 0; p < np; ++p) {
        const Group &G = hp.groups[plans[p].group];
        const int R = std::min(Rdef, G.k);
        PassDesc &d = hp.fwd[p];
        d.k = G.k;
        d.m = G.m;
        d.a = G.a;
        d.R = R;
        d.n_slots = int(plans[p].layers.size());
        hp.pass_tiles_log2[p] = n - G.k;
        std::vector<uint32_t> gm(d.n_slots, G.gated);
        for (int s = 0; s < d.n_slots; ++s) {
            const int l = plans[p].layers[s];
            d.slot_layer[s] = l;
            d.slot_gated[s] = G.gated;
            d.slot_czmask[s] = 0;
            if (coef_off > 0x7fffffff || dtab_off > 0x7fffffff || grad_off > 0x7fffffff) {
                err = "plan tables exceed 2^31 entries";
                return false;
            }
            d.slot_coef_off[s] = int(coef_off);
            d.slot_dtab_off[s] = int(dtab_off);
            d.slot_grad_off[s] = int(grad_off);
            StageSlot ss{};
            ss.k = G.k;
            ss.layer = l;
            ss.coef_off = int(coef_off);
            ss.dtab_off = int(dtab_off);
            for (int j = 0; j < G.k; ++j) {
                if (!((G.gated >> j) & 1u)) continue;
                ss.tile_bit[ss.n_gated] = uint8_t(j);
                ss.qubit[ss.n_gated] = uint8_t(G.qubit_of(j));
                ss.n_gated++;
            }
            stage.push_back(ss);
            slot_grad_off[stage.size() - 1] = grad_off;
            coef_off += G.k;
            dtab_off += size_t(1) << G.k;
            grad_off += (size_t(1) << (n - G.k)) * 2 * G.k;
        }
        const auto rounds = make_rounds(G.k, R, gm);
        emit_forward(d, rounds);
        hp.bwd[p] = d;
        emit_backward(hp.bwd[p], rounds, d.n_slots);
        // order in which the backward program un-rotates each slot's bits
        std::vector<uint32_t> done(d.n_slots, 0);
        std::vector<std::vector<uint16_t>> before(d.n_slots, std::vector<uint16_t>(G.k, 0));
        int chunk = -1;
        const PassDesc &bd = hp.bwd[p];
        for (int oi = 0; oi < bd.n_ops; ++oi) {
            const PassOp &o = bd.ops[oi];
            if (o.kind == OP_ROUND) chunk = o.chunk;
            if (o.kind != OP_BF) continue;
            for (int j = 0; j < R; ++j) {
                if (!((o.mask >> j) & 1)) continue;
                before[o.slot][chunk + j] = uint16_t(done[o.slot]);
                done[o.slot] |= 1u << (chunk + j);
            }
        }
        const size_t first_stage = stage.size() - d.n_slots;
        for (int s = 0; s < d.n_slots; ++s) {
            StageSlot &ss = stage[first_stage + s];
            for (int u = 0; u < ss.n_gated; ++u) ss.before[u] = before[s][ss.tile_bit[u]];
        }
    }
    // Support of the state before each forward pass (it starts from |0...0>):
    // bits of qubits no earlier pass has rotated are 0.  The backward pass p
    // skips the tiles outside the support of the state after forward pass p
    // (the forward zmask of pass p + 1): there psi is zero, so the gradient
    // terms vanish, and passes p' <= p never mix those indices with the
    // support (they rotate no qubit of that mask), so their lambda is never
    // read again.
    {
        uint32_t rotated = 0;
        const uint32_t nmask = n >= 32 ? ~0u : ((1u << n) - 1u);
        for (int p = 0; p < np; ++p) {
            hp.fwd[p].zmask = nmask & ~rotated;
            const Group &G = hp.groups[plans[p].group];
            for (int j = 0; j < G.k; ++j)
                if ((G.gated >> j) & 1u) rotated |= 1u << G.qubit_of(j);
        }
        for (int p = 0; p < np; ++p) hp.bwd[p].zmask = p + 1 < np ? hp.fwd[p + 1].zmask : 0u;
    }
    // CZ(q, q+1) of layer l goes to the later of the slots holding RY_l(q), RY_l(q+1).
    for (int l = 0; l < D; ++l) {
        for (int q = 0; q + 1 < n; ++q) {
            const int gid = std::max(slot_of[l][q], slot_of[l][q + 1]);
            const auto ps = slot_pos[gid];
            hp.fwd[ps.first].slot_czmask[ps.second] |= (1u << q);
            hp.bwd[ps.first].slot_czmask[ps.second] |= (1u << q);
        }
    }
    // Gradient reduction map: param (l, q, comp) -> partial column.
    const int NP = 2 * n * D;
    std::vector<int> goff(NP), gcnt(NP), gstep(NP);
    for (int l = 0; l < D; ++l) {
        for (int q = 0; q < n; ++q) {
            const int gid = slot_of[l][q];
            const auto ps = slot_pos[gid];
            const PassDesc &d = hp.fwd[ps.first];
            const Group &G = hp.groups[plans[ps.first].group];
            int j = -1;
            for (int jj = 0; jj < G.k; ++jj)
                if (((G.gated >> jj) & 1u) && G.qubit_of(jj) == q) j = jj;
            for (int comp = 0; comp < 2; ++comp) {
                const int pidx = (l * n + q) * 2 + comp;
                goff[pidx] = int(slot_grad_off[gid]) + j * 2 + comp;
                gcnt[pidx] = 1 << (n - d.k);
                gstep[pidx] = 2 * d.k;
            }
        }
    }
    hp.coef_stride = coef_off;
    hp.dtab_stride = dtab_off;
    hp.grad_stride = grad_off;
    hp.stage = stage;
    hp.goff = goff;
    hp.gcnt = gcnt;
    hp.gstep = gstep;
    hp.n_params = NP;
    return true;
}

// Default plan options: the energy plan may use 32 amplitudes per thread
// (forward only); the gradient plan keeps at most 16 (both buffers in registers).

vqe_status build_one_plan(vqe_ctx *h, int which) {
    vqe_ctx::DevPlan &P = h->plan[which];
    HostPlan hp;
    std::string err;
    if (!make_plan(h->n, h->depth, h->prec, P.opts, hp, err)) return fail(h, VQE_ERR_ARG, err);
    P.groups = hp.groups;
    P.fwd = hp.fwd;
    P.bwd = hp.bwd;
    P.coef_stride = hp.coef_stride;
    P.dtab_stride = hp.dtab_stride;
    P.grad_stride = hp.grad_stride;
    P.n_stage = int(hp.stage.size());
    h->n_params = hp.n_params;
    vqe_status st;
    if ((st = upload(h, P.d_fwd, P.fwd, "pass plan")) != VQE_OK) return st;
    if (which == 1) {
        if ((st = upload(h, P.d_bwd, P.bwd, "pass plan")) != VQE_OK) return st;
        if ((st = upload(h, P.d_goff, hp.goff, "grad map")) != VQE_OK) return st;
        if ((st = upload(h, P.d_gcnt, hp.gcnt, "grad map")) != VQE_OK) return st;
        if ((st = upload(h, P.d_gstep, hp.gstep, "grad map")) != VQE_OK) return st;
    }
    if ((st = upload(h, P.d_stage, hp.stage, "stage plan")) != VQE_OK) return st;
    return VQE_OK;
}

// ---------------------------------------------------------------- particle-conserving plan

struct PcHostPlan {
    std::vector<ExcPass> passes;
    std::vector<ExcGate> gates;
    std::vector<uint32_t> hoff;
    std::vector<int> goff, gcnt, gstep;
    size_t grad_stride = 0;
    int k = 0;
};

// Passes of the excitation sequence: runs of consecutive gates (at most
// kExcMaxGates) whose modes outside the low run [0, m) fit the k - m further
// tile bits.  Tiles hold 2^k amplitudes: 2^11 (32 KiB) in FP64, 2^12 in FP32,
// with contiguous runs of 2^m = 256 bytes.
bool make_pc_plan(int n, vqe_precision prec, const std::vector<int> &exc, uint64_t hf_index,
                  PcHostPlan &pp, std::string &err) {
    pp = PcHostPlan{};
    int k = prec == VQE_C128 ? 11 : 12;
    int m = prec == VQE_C128 ? 4 : 5;
    if (n <= k) {
        k = n;
        m = n;
    }
    const int hi = k - m;
    pp.k = k;
    const int K = int(exc.size() / 4);
    auto high_bits = [&](int j) {
        uint32_t b = 0;
        for (int u = 0; u < 4; ++u) {
            const int md = exc[4 * j + u];
            if (md >= m) b |= 1u << md;
        }
        return b;
    };
    std::vector<std::pair<int, int>> runs;   // (first gate, count)
    uint32_t cur = 0;
    int first = 0;
    for (int j = 0; j < K; ++j) {
        const uint32_t hb = high_bits(j);
        const int cnt = j - first;
        if (cnt > 0 && (__builtin_popcount(cur | hb) > hi || cnt >= kExcMaxGates)) {
            runs.push_back({first, cnt});
            first = j;
            cur = 0;
        }
        cur |= hb;
        if (__builtin_popcount(cur) > hi) {
            err = "an excitation spans more modes than a tile holds";
            return false;
        }
    }
    if (K > first) runs.push_back({first, K - first});
    const uint64_t tiles = uint64_t(1) << (n - k);
    const uint32_t hf = uint32_t(hf_index);
    uint32_t touched = 0;   // modes of the gates of earlier passes
    size_t goff = 0;
    pp.goff.assign(K, 0);
    pp.gcnt.assign(K, 0);
    pp.gstep.assign(K, 0);
    for (const auto &r : runs) {
        uint32_t S = 0;
        for (int j = r.first; j < r.first + r.second; ++j) S |= high_bits(j);
        for (int b = m; b < n && __builtin_popcount(S) < hi; ++b) S |= 1u << b;   // fill with low bits
        std::vector<int> pos;
        for (int b = 0; b < n; ++b)
            if ((S >> b) & 1u) pos.push_back(b);
        const uint32_t nmask = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
        const uint32_t tile_global = ((1u << m) - 1u) | S;
        auto to_tile = [&](uint32_t g) {   // global mask restricted to tile bits -> tile coordinates
            uint32_t t = g & ((1u << m) - 1u);
            for (size_t j = 0; j < pos.size(); ++j)
                if ((g >> pos[j]) & 1u) t |= 1u << (m + int(j));
            return t;
        };
        ExcPass P{};
        P.k = k;
        P.m = m;
        P.g_begin = int(pp.gates.size());
        P.n_gates = r.second;
        P.hoff = int(pp.hoff.size());
        P.bmask = nmask & ~tile_global;
        if (goff > 0x7fffffff) {
            err = "gradient partials exceed 2^31 entries";
            return false;
        }
        P.grad_off = int(goff);
        P.zmask = P.bmask & ~touched;
        P.zval = hf & P.zmask;
        for (int j = r.first; j < r.first + r.second; ++j)
            for (int u = 0; u < 4; ++u)
                if (exc[4 * j + u] >= 0) touched |= 1u << exc[4 * j + u];
        P.bzmask = P.bmask & ~touched;
        P.bzval = hf & P.bzmask;
        for (uint32_t hh = 0; hh < (1u << hi); ++hh) {
            uint32_t g = 0;
            for (int j = 0; j < hi; ++j)
                if ((hh >> j) & 1u) g |= 1u << pos[j];
            pp.hoff.push_back(g);
        }
        for (int j = r.first; j < r.first + r.second; ++j) {
            const int p = exc[4 * j], q = exc[4 * j + 1], rr = exc[4 * j + 2], ss = exc[4 * j + 3];
            const bool dbl = q >= 0;
            auto below = [](int md) { return md >= 32 ? 0xffffffffu : ((1u << md) - 1u); };
            uint32_t amask_g = 1u << rr, cmask_g = 1u << p;
            uint32_t smask = below(p) ^ below(rr);
            uint32_t sign0;
            if (dbl) {
                amask_g |= 1u << ss;
                cmask_g |= 1u << q;
                smask ^= below(q) ^ below(ss);
                sign0 = uint32_t((ss < rr) + (ss < q) + (rr < q) + (ss < p) + (rr < p) + (q < p)) & 1u;
            } else {
                sign0 = uint32_t(rr < p);
            }
            ExcGate G{};
            G.amask = to_tile(amask_g);
            G.cmask = to_tile(cmask_g);
            G.smask_t = to_tile(smask & tile_global);
            G.smask_g = smask & ~tile_global;
            G.sign0 = sign0;
            const uint32_t fixed = G.amask | G.cmask;
            G.n_fixed = __builtin_popcount(fixed);
            int u = 0;
            for (int b = 0; b < k; ++b)
                if ((fixed >> b) & 1u) G.fixed[u++] = uint8_t(b);
            G.param = j;
            pp.gates.push_back(G);
            pp.goff[j] = int(goff) + (j - r.first);
            pp.gcnt[j] = int(tiles);
            pp.gstep[j] = r.second;
        }
        pp.passes.push_back(P);
        goff += size_t(tiles) * r.second;
    }
    pp.grad_stride = goff;
    return true;
}

vqe_status build_pc_plan(vqe_ctx *h) {
    PcHostPlan pp;
    std::string err;
    if (!make_pc_plan(h->n, h->prec, h->exc, h->hf_index, pp, err)) return fail(h, VQE_ERR_ARG, err);
    vqe_status st;
    if ((st = upload(h, h->d_pc_gates, pp.gates, "excitation gates")) != VQE_OK) return st;
    if ((st = upload(h, h->d_pc_hoff, pp.hoff, "excitation tiles")) != VQE_OK) return st;
    vqe_ctx::DevPlan &P = h->plan[1];
    if ((st = upload(h, P.d_goff, pp.goff, "grad map")) != VQE_OK) return st;
    if ((st = upload(h, P.d_gcnt, pp.gcnt, "grad map")) != VQE_OK) return st;
    if ((st = upload(h, P.d_gstep, pp.gstep, "grad map")) != VQE_OK) return st;
    h->pc_passes = pp.passes;
    h->pc_k = pp.k;
    for (int w = 0; w < 2; ++w) {
        h->plan[w].fwd.clear();
        h->plan[w].bwd.clear();
        h->plan[w].groups.clear();
        h->plan[w].coef_stride = h->exc.size() / 4;   // (cos, sin) per excitation
        h->plan[w].dtab_stride = 0;
        h->plan[w].grad_stride = pp.grad_stride;
        h->plan[w].n_stage = 0;
    }
    h->n_params = int(h->exc.size() / 4);
    h->stats.ansatz_passes = uint32_t(pp.passes.size());
    h->stats.tile_bits_max = uint32_t(pp.k);
    return VQE_OK;
}

vqe_status build_plan(vqe_ctx *h) {
    if (h->ansatz == 1) return build_pc_plan(h);
    for (int w = 0; w < 2; ++w) {
        vqe_status st = build_one_plan(h, w);
        if (st != VQE_OK) return st;
    }
    h->stats.ansatz_passes = uint32_t(h->plan[0].fwd.size());
    int kmax = 0;
    for (auto &g : h->plan[0].groups) kmax = std::max(kmax, g.k);
    h->stats.tile_bits_max = uint32_t(kmax);
    return VQE_OK;
}

// ---------------------------------------------------------------- Hamiltonian

struct HamPlan {
    std::vector<GroupDesc> groups;
    std::vector<uint32_t> tz;
    std::vector<double> tc;
    uint64_t n_groups_nonempty = 0;
};

// Groups of kept terms by x mask (the x = 0 group always first, since it
// also yields <psi|psi>); within a group A terms (kappa even) precede B
// terms (kappa odd); the coefficient carries the sign (-1)^{floor(kappa/2)}.
void make_ham_plan(const std::vector<uint64_t> &cx, const std::vector<uint64_t> &cz,
                   const std::vector<double> &cc, const std::vector<uint8_t> &keep, HamPlan &hp) {
    struct T3 { uint32_t x, z; int cls; double c; };
    std::vector<T3> terms;
    for (size_t t = 0; t < cc.size(); ++t) {
        if (!keep[t]) continue;
        const uint32_t x = uint32_t(cx[t]), z = uint32_t(cz[t]);
        const int kappa = __builtin_popcount(x & z);
        const double sign = ((kappa >> 1) & 1) ? -1.0 : 1.0;
        terms.push_back({x, z, kappa & 1, cc[t] * sign});
    }
    std::stable_sort(terms.begin(), terms.end(), [](const T3 &p, const T3 &q) {
        if (p.x != q.x) return p.x < q.x;
        if (p.cls != q.cls) return p.cls < q.cls;
        return p.z < q.z;
    });
    hp = HamPlan{};
    auto open_group = [&](uint32_t x) {
        GroupDesc g{};
        g.x = x;
        g.h = x ? 31 - __builtin_clz(x) : 0;
        g.t_begin = int(hp.tz.size());
        g.t_mid = g.t_begin;
        g.t_end = g.t_begin;
        hp.groups.push_back(g);
    };
    open_group(0);
    for (size_t t = 0; t < terms.size(); ++t) {
        if (terms[t].x != hp.groups.back().x) open_group(terms[t].x);
        hp.tz.push_back(terms[t].z);
        hp.tc.push_back(terms[t].c);
        GroupDesc &g = hp.groups.back();
        g.t_end = int(hp.tz.size());
        if (terms[t].cls == 0) g.t_mid = g.t_end;
    }
    for (auto &g : hp.groups)
        if (g.t_end > g.t_begin) hp.n_groups_nonempty++;
}

// Canonical form: equal strings merged (coefficients summed in input
// order), exact zeros removed, sorted by (x, z).
void canonicalise(const uint64_t *x, const uint64_t *z, const double *c, size_t n_terms,
                  std::vector<uint64_t> &cx, std::vector<uint64_t> &cz, std::vector<double> &cc) {
    std::vector<size_t> idx(n_terms);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t p, size_t q) {
        if (x[p] != x[q]) return x[p] < x[q];
        return z[p] < z[q];
    });
    cx.clear();
    cz.clear();
    cc.clear();
    for (size_t i = 0; i < n_terms;) {
        size_t j = i;
        double s = 0.0;
        while (j < n_terms && x[idx[j]] == x[idx[i]] && z[idx[j]] == z[idx[i]]) s += c[idx[j++]];
        if (s != 0.0) {
            cx.push_back(x[idx[i]]);
            cz.push_back(z[idx[i]]);
            cc.push_back(s);
        }
        i = j;
    }
}

// Cutoff (Sec. II-D, III-D): keep |c| >= threshold; returns sum |c| dropped.
double slim_keep(const std::vector<double> &cc, double threshold, std::vector<uint8_t> &keep,
                 size_t &kept) {
    keep.assign(cc.size(), 0);
    kept = 0;
    double dropped = 0.0;
    for (size_t t = 0; t < cc.size(); ++t) {
        if (std::fabs(cc[t]) >= threshold) {
            keep[t] = 1;
            ++kept;
        } else {
            dropped += std::fabs(cc[t]);
        }
    }
    return dropped;
}

// Energy windows (see k_energy_win): window 0 = the low kE bits (and the
// x = 0 group); a group whose X mask above the low `mrun` bits spans at most
// kE - mrun bits joins (or opens) a window [0, mrun) + [a, a + kE - mrun);
// wider groups are swept over the whole state.
struct WinPlan {
    std::vector<WinDesc> wins;
    std::vector<WinGroup> groups;
    std::vector<WinTerm> terms;
    std::vector<uint32_t> hoff;
    std::vector<GroupDesc> wide;   // groups that fit no window: global sweeps
    int win_tiles = 0;
};

// Tile coordinates of global mask g for a window with low run m and high
// positions pos (increasing): bits [0, m) stay, bit pos[j] -> tile bit m + j.
uint32_t win_gather(uint32_t g, int m, const std::vector<int> &pos) {
    uint32_t t = g & ((1u << m) - 1u);
    for (size_t j = 0; j < pos.size(); ++j)
        if ((g >> pos[j]) & 1u) t |= 1u << (m + int(j));
    return t;
}

// bit i of v -> the i-th set bit of mask (a software bit deposit)
uint32_t deposit_bits(uint32_t v, uint32_t mask) {
    uint32_t out = 0;
    int i = 0;
    for (int q = 0; q < 32; ++q)
        if ((mask >> q) & 1u) {
            if ((v >> i) & 1u) out |= 1u << q;
            ++i;
        }
    return out;
}

// p with a zero inserted at every set bit of mask (ascending): the tile index
// of free-index p when the bits of mask are fixed
uint32_t spread_bits(uint32_t p, uint32_t mask) {
    for (int q = 0; q < 32; ++q)
        if ((mask >> q) & 1u) p = ((p >> q) << (q + 1)) | (p & ((1u << q) - 1u));
    return p;
}

// A group of the expectation split per pattern b of its X bits below the top
// one (global coordinates).  For the lower element i0 of a pair (top X bit 0)
// with those bits equal to b, (-1)^{popc(i0 & z)} = (-1)^{popc(i0 & (z & ~x))}
// * (-1)^{popc(b & z)}: terms sharing the Z bits outside x merge into one
// coefficient per pattern, and patterns whose merged coefficients all vanish
// (the pairs the group does not connect, e.g. |00> <-> |11> for a hop) are
// left out.  With more than 3 such bits the group stays whole.
struct VTerm {
    uint32_t z;
    double c;
};
struct VGroup {
    uint32_t fix_mask, fix_val;
    std::vector<VTerm> a, b;
};

std::vector<VGroup> split_group(const GroupDesc &G, const HamPlan &hp) {
    std::vector<VGroup> out;
    const uint32_t x = G.x;
    const int h = 31 - __builtin_clz(x);
    const uint32_t xp = x & ~(1u << h);
    const int rp = __builtin_popcount(xp);
    if (rp > 3) {
        VGroup v{1u << h, 0u, {}, {}};
        for (int t = G.t_begin; t < G.t_mid; ++t) v.a.push_back({hp.tz[t], hp.tc[t]});
        for (int t = G.t_mid; t < G.t_end; ++t) v.b.push_back({hp.tz[t], hp.tc[t]});
        out.push_back(v);
        return out;
    }
    const int np = 1 << rp;
    auto classes = [&](int t0, int t1, std::vector<uint32_t> &keys, std::vector<std::vector<double>> &tab) {
        for (int t = t0; t < t1; ++t) {
            const uint32_t z = hp.tz[t], zc = z & ~x;
            size_t ci = 0;
            while (ci < keys.size() && keys[ci] != zc) ++ci;
            if (ci == keys.size()) {
                keys.push_back(zc);
                tab.emplace_back(np, 0.0);
            }
            for (int bb = 0; bb < np; ++bb)
                tab[ci][bb] += (__builtin_popcount(deposit_bits(bb, xp) & z) & 1) ? -hp.tc[t] : hp.tc[t];
        }
    };
    std::vector<uint32_t> ka, kb;
    std::vector<std::vector<double>> ta, tb;
    classes(G.t_begin, G.t_mid, ka, ta);
    classes(G.t_mid, G.t_end, kb, tb);
    for (int bb = 0; bb < np; ++bb) {
        VGroup v{(1u << h) | xp, deposit_bits(bb, xp), {}, {}};
        for (size_t c = 0; c < ka.size(); ++c)
            if (ta[c][bb] != 0.0) v.a.push_back({ka[c], ta[c][bb]});
        for (size_t c = 0; c < kb.size(); ++c)
            if (tb[c][bb] != 0.0) v.b.push_back({kb[c], tb[c][bb]});
        if (!v.a.empty() || !v.b.empty()) out.push_back(std::move(v));
    }
    return out;
}

// Windows of the windowed expectation (Sec. II-B Eq. 7 evaluated per X-mask
// group) and of the windowed apply-H, which walks the same pairs: the low
// tile (with <psi|psi> and the diagonal group), then windows
// of mrun low bits plus kE - mrun further bits chosen greedily so that every
// group's X mask lies inside one window (a greedy cover of the groups' high
// bits), each window holding at most kWinMaxTerms terms.  Groups with more
// high bits than a window has go to the global sweep.  `diag_terms`: store
// the diagonal group's terms (false when the diagonal of H is precomputed).
void plan_windows(int n, vqe_precision prec, const HamPlan &hp, bool diag_terms, WinPlan &wp) {
    wp = WinPlan{};
    const bool c128 = prec == VQE_C128;
    const int kE = win_tile_bits(c128);
    const int mrun = c128 ? 3 : 4;
    if (n <= kE) return;
    const int hw = kE - mrun;
    const int lt = 9;                      // log2 of the kernel's 512 threads
    const int EPT = 1 << (kE - lt), PPT = EPT / 2;
    // the fixed bits of i0 in tile coordinates, and from them the spread of a
    // pair's free index: smask by shift, dj for the bits at and above lt
    auto set_fixed = [&](WinGroup &wg, uint32_t fmask) {
        wg.fmask = fmask;
        wg.plog = kE - __builtin_popcount(fmask);
        for (int i = 0; i < wg.plog; ++i) {
            const uint32_t o = spread_bits(1u << i, fmask);
            wg.smask[(31 - __builtin_clz(o)) - i] |= 1u << i;
        }
        for (int bb = 0; bb < 4; ++bb)
            wg.dj[bb] = (lt + bb < wg.plog) ? spread_bits(1u << (lt + bb), fmask) : 0u;
    };

    struct Cand {
        int m;
        uint32_t S;                        // high positions (bits >= m) of the window
        std::vector<int> groups;
        int terms = 0;
        bool norm = false;
        int ngroups = 0;                   // window groups after splitting
    };
    std::vector<Cand> cands;
    // expectation layout: a pair group is split by the patterns of its X bits
    // below the top one when every kept pattern has few terms (one sign
    // evaluation per term and pair); otherwise it stays whole
    const int split_max = c128 ? 3 : 2;
    std::vector<std::vector<VGroup>> vgs(hp.groups.size());
    std::vector<char> is_split(hp.groups.size(), 0), vanishes(hp.groups.size(), 0);
    for (size_t g = 0; g < hp.groups.size(); ++g) {
        const GroupDesc &G = hp.groups[g];
        if (G.x == 0u) continue;
        std::vector<VGroup> v = split_group(G, hp);
        if (v.empty()) {
            vanishes[g] = 1;
            continue;
        }
        bool ok = v[0].fix_mask != (1u << (31 - __builtin_clz(G.x)));
        for (const VGroup &vg : v)
            ok = ok && int(vg.a.size()) <= kWinDirectMax && int(vg.b.size()) <= kWinDirectMax &&
                 int(vg.a.size() + vg.b.size()) <= split_max;
        if (ok) {
            vgs[g] = std::move(v);
            is_split[g] = 1;
        }
    }
    auto group_terms = [&](int g) {
        const GroupDesc &G = hp.groups[g];
        if (G.x == 0u && !diag_terms) return 0;
        if (is_split[g]) {
            int t = 0;
            for (const VGroup &v : vgs[g]) t += int(v.a.size() + v.b.size());
            return t;
        }
        return G.t_end - G.t_begin;
    };
    auto group_count = [&](int g) { return vanishes[g] ? 0 : 1; };
    // the low tile: every group whose X mask lies in bits [0, kE); split when
    // the term cap is reached (only the first part yields the norm)
    cands.push_back({kE, 0u, {}, 0, true});
    std::vector<int> rest;
    for (size_t g = 0; g < hp.groups.size(); ++g) {
        const uint32_t x = hp.groups[g].x;
        if (x < (1u << kE)) {
            const int tg = group_terms(int(g));
            if (tg > kWinMaxTerms) {                 // too many terms for any window
                wp.wide.push_back(hp.groups[g]);
                if (x == 0u) cands[0].norm = false;  // the sweep of the diagonal group yields the norm
                continue;
            }
            const int gc = group_count(int(g));
            if (gc == 0) continue;                   // every pair of the group vanishes
            if (cands.back().m != kE || cands.back().terms + tg > kWinMaxTerms ||
                cands.back().ngroups + gc > kWinMaxGroups)
                cands.push_back({kE, 0u, {}, 0, false});
            cands.back().groups.push_back(int(g));
            cands.back().terms += tg;
            cands.back().ngroups += gc;
        } else {
            rest.push_back(int(g));
        }
    }
    // other groups: greedy cover in decreasing X mask order, so that masks
    // sharing their top bits meet in the same windows (the synthetic
    // molecular Hamiltonian at 24 qubits: 108 windows, against 246 when the
    // groups went by decreasing number of high bits)
    const uint32_t lowm = (1u << mrun) - 1u;
    std::stable_sort(rest.begin(), rest.end(),
                     [&](int p, int q) { return hp.groups[p].x > hp.groups[q].x; });
    const size_t first_free = cands.size();
    for (int g : rest) {
        const uint32_t H = hp.groups[g].x & ~lowm;
        const int tg = group_terms(g);
        const int gc = group_count(g);
        if (gc == 0) continue;
        if (__builtin_popcount(H) > hw || tg > kWinMaxTerms || gc > kWinMaxGroups) {
            wp.wide.push_back(hp.groups[g]);
            continue;
        }
        int best = -1, best_add = 1 << 30;
        for (size_t c = first_free; c < cands.size(); ++c) {
            const uint32_t U = cands[c].S | H;
            const int sz = __builtin_popcount(U);
            if (sz > hw || cands[c].terms + tg > kWinMaxTerms || cands[c].ngroups + gc > kWinMaxGroups)
                continue;
            const int add = sz - __builtin_popcount(cands[c].S);
            if (add < best_add) {
                best_add = add;
                best = int(c);
            }
        }
        if (best < 0) {
            cands.push_back({mrun, H, {}, 0, false});
            best = int(cands.size()) - 1;
        }
        cands[best].S |= H;
        cands[best].groups.push_back(g);
        cands[best].terms += tg;
        cands[best].ngroups += gc;
    }
    const uint32_t nmask = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    for (Cand &c : cands) {
        if (c.groups.empty() && !c.norm) continue;
        // fill the high positions up to kE - m with the lowest free bits
        for (int b = c.m; __builtin_popcount(c.S) < kE - c.m && b < n; ++b) c.S |= 1u << b;
        std::vector<int> pos;
        for (int b = 0; b < n; ++b)
            if ((c.S >> b) & 1u) pos.push_back(b);
        WinDesc W{};
        W.k = kE;
        W.m = c.m;
        W.bmask = nmask & ~((1u << c.m) - 1u) & ~c.S;
        W.hoff = int(wp.hoff.size());
        for (uint32_t hh = 0; hh < (1u << (kE - c.m)); ++hh) {
            uint32_t off = 0;
            for (size_t j = 0; j < pos.size(); ++j)
                if ((hh >> j) & 1u) off |= 1u << pos[j];
            wp.hoff.push_back(off);
        }
        W.g_begin = int(wp.groups.size());
        W.t_begin = int(wp.terms.size());
        for (int g : c.groups) {
            const GroupDesc &G = hp.groups[g];
            if (is_split[g]) {
                WinGroup wg{};
                wg.xl = win_gather(G.x, c.m, pos);
                wg.hl = 31 - __builtin_clz(wg.xl);
                wg.direct = 1;
                set_fixed(wg, win_gather(vgs[g][0].fix_mask, c.m, pos));
                wg.npat = int(vgs[g].size());
                for (int u = 0; u < wg.npat; ++u) wg.fval[u] = win_gather(vgs[g][u].fix_val, c.m, pos);
                auto emit_p = [&](bool cls_b, uint16_t *run, int &begin) {
                    begin = int(wp.terms.size()) - W.t_begin;
                    for (int u = 0; u < wg.npat; ++u) {
                        run[u] = uint16_t(int(wp.terms.size()) - W.t_begin - begin);
                        for (const VTerm &vt : cls_b ? vgs[g][u].b : vgs[g][u].a) {
                            WinTerm wt{};
                            wt.zt = win_gather(vt.z, c.m, pos);
                            wt.zout = vt.z & W.bmask;
                            wt.c = vt.c;
                            wp.terms.push_back(wt);
                        }
                    }
                    run[wg.npat] = uint16_t(int(wp.terms.size()) - W.t_begin - begin);
                };
                emit_p(false, wg.arun, wg.a_begin);
                emit_p(true, wg.brun, wg.b_begin);
                wg.b_end = int(wp.terms.size()) - W.t_begin;
                wp.groups.push_back(wg);
                continue;
            }
            if (vanishes[g]) continue;
            WinGroup wg{};
            wg.xl = win_gather(G.x, c.m, pos);
            wg.hl = wg.xl ? 31 - __builtin_clz(wg.xl) : 0;
            const int NV = wg.xl ? PPT : EPT;
            // few terms: per-pair sign sums beat the transform over the
            // register patterns and its per-run loop (FP64: up to 3 terms,
            // FP32: up to 2)
            const int n_t = (G.x != 0u || diag_terms) ? G.t_end - G.t_begin : 0;
            wg.direct = (wg.xl != 0u && n_t <= std::min(kWinDirectMax, c128 ? 3 : 2)) ? 1 : 0;
            // tile bit of register-pattern bit b: element bit lt + b of a
            // thread's elements (diagonal group), or of its pairs after the
            // zero inserted at hl
            auto pattern = [&](uint32_t zt) {
                uint32_t v = 0;
                for (int bb = 0; (1 << bb) < NV; ++bb) {
                    int q = lt + bb;
                    if (wg.xl && q >= wg.hl) q += 1;
                    v |= ((zt >> q) & 1u) << bb;
                }
                return v;
            };
            auto emit = [&](int t0, int t1, uint16_t *run, int &begin) {
                begin = int(wp.terms.size()) - W.t_begin;
                std::vector<std::pair<uint32_t, WinTerm>> ts;
                for (int t = t0; t < t1; ++t) {
                    WinTerm wt{};
                    wt.zt = win_gather(hp.tz[t], c.m, pos);
                    wt.zout = hp.tz[t] & W.bmask;
                    wt.c = hp.tc[t];
                    ts.push_back({pattern(wt.zt), wt});
                }
                if (!wg.direct)
                    std::stable_sort(ts.begin(), ts.end(),
                                     [](const auto &p, const auto &q) { return p.first < q.first; });
                else
                    for (auto &p : ts) p.first = 0;   // one run
                int at = 0;
                for (int v = 0; v <= NV; ++v) {
                    while (at < int(ts.size()) && int(ts[at].first) < v) ++at;
                    run[v] = uint16_t(at);
                }
                for (auto &p : ts) wp.terms.push_back(p.second);
            };
            if (wg.xl) {
                set_fixed(wg, 1u << wg.hl);
                wg.npat = 1;
            } else {
                wg.plog = kE;
            }
            const bool keep = G.x != 0u || diag_terms;
            emit(G.t_begin, keep ? G.t_mid : G.t_begin, wg.arun, wg.a_begin);
            emit(G.t_mid, keep ? G.t_end : G.t_mid, wg.brun, wg.b_begin);
            wg.b_end = int(wp.terms.size()) - W.t_begin;
            wp.groups.push_back(wg);
        }
        W.g_end = int(wp.groups.size());
        W.t_count = int(wp.terms.size()) - W.t_begin;
        W.any_runs = 0;
        for (int gi = W.g_begin; gi < W.g_end; ++gi) {
            const WinGroup &wg = wp.groups[gi];
            // transform path: a pair group that is not direct, or the diagonal
            // group with its terms (no precomputed diagonal)
            if ((wg.xl != 0u && !wg.direct) || (wg.xl == 0u && wg.b_end > wg.a_begin)) W.any_runs = 1;
        }
        W.block_off = wp.win_tiles;
        W.with_norm = c.norm ? 1 : 0;
        wp.win_tiles += 1 << (n - kE);
        wp.wins.push_back(W);
    }
}

// Sweeps of the sweep form of apply-H (see SweepDesc): the groups are
// assigned greedily, in decreasing X-mask order, to the sweep whose fast
// bits grow least by the group's X bits above the low run, while the fast
// bits stay within kSweepFastBits - mlo; groups with more such bits join the
// last sweep (their partners then come from DRAM).  The diagonal goes to the
// first sweep: D_i psi_i from the precomputed diagonal, or the x = 0 group's
// terms when `diag_terms`.
struct SweepPlan {
    std::vector<SweepDesc> sweeps;
    std::vector<SGroup> groups;
    std::vector<uint32_t> pat;
    std::vector<uint32_t> tz;
    std::vector<double> ta, tb;
    std::vector<uint32_t> order;   // 1024 per sweep
    bool ok = false;               // false: a group has more terms than a sweep holds
    bool all_parity = true;        // every group with an X mask in the parity form
};

void plan_sweeps(int n, vqe_precision prec, const HamPlan &hp, bool diag_terms, SweepPlan &sp) {
    sp = SweepPlan{};
    const int mlo = std::min(n, prec == VQE_C128 ? 4 : 5);   // runs of 256 bytes
    const int fmax = std::max(0, std::min(n, kSweepFastBits) - mlo);
    const uint32_t lowm = (1u << mlo) - 1u;
    // one group in pattern form: per pattern of its X bits, the terms merged
    // by z & ~x (A and B coefficients); a group with more X bits keeps its
    // terms (one pattern, z unmasked)
    struct MTerm { uint32_t z; double a, b; };
    struct MGroup {
        uint32_t x = 0;
        std::vector<int> xb;
        std::vector<std::vector<MTerm>> pats;
        bool has_b = false;
        int n_terms = 0;
    };
    auto merge = [&](const GroupDesc &G) {
        MGroup mg;
        mg.x = G.x;
        const int nx = __builtin_popcount(G.x);
        const bool pattern_form = nx <= kSweepMaxXBits;
        if (pattern_form)
            for (int q = 0; q < 32; ++q)
                if ((G.x >> q) & 1u) mg.xb.push_back(q);
        const int np = pattern_form ? 1 << nx : 1;
        mg.pats.resize(np);
        for (int pv = 0; pv < np; ++pv) {
            const uint32_t v = pattern_form ? deposit_bits(uint32_t(pv), G.x) : 0u;
            std::vector<MTerm> &ts = mg.pats[pv];
            for (int t = G.t_begin; t < G.t_end; ++t) {
                const bool cls_b = t >= G.t_mid;
                const uint32_t z = hp.tz[t];
                const uint32_t zk = pattern_form ? (z & ~G.x) : z;
                const double c = (__builtin_popcount(v & z) & 1) ? -hp.tc[t] : hp.tc[t];
                size_t k = 0;
                while (k < ts.size() && ts[k].z != zk) ++k;
                if (k == ts.size()) ts.push_back({zk, 0.0, 0.0});
                (cls_b ? ts[k].b : ts[k].a) += c;
            }
            std::vector<MTerm> kept;
            for (const MTerm &m : ts)
                if (m.a != 0.0 || m.b != 0.0) {
                    kept.push_back(m);
                    mg.has_b = mg.has_b || m.b != 0.0;
                }
            ts.swap(kept);
            mg.n_terms += int(ts.size());
        }
        return mg;
    };
    struct SC {
        uint32_t F = 0;                  // fast bits above the low run
        std::vector<MGroup> groups;
        int terms = 0, pats = 0;
    };
    std::vector<SC> sc(1);
    std::vector<MGroup> wide;
    // term slots and pattern entries a group takes: a group whose patterns
    // hold at most one term each takes one slot per pattern and no entry
    auto slots = [](const MGroup &mg) {
        bool multi = false;
        for (const auto &ts : mg.pats) multi = multi || ts.size() > 1;
        return multi ? std::make_pair(mg.n_terms, int(mg.pats.size())) : std::make_pair(int(mg.pats.size()), 0);
    };
    auto fits = [&](const SC &c, const MGroup &mg) {
        const auto sl = slots(mg);
        return int(c.groups.size()) + 1 <= kSweepMaxGroups && c.terms + sl.first <= kSweepMaxTerms &&
               c.pats + sl.second <= kSweepMaxPat;
    };
    auto add = [&](SC &c, MGroup &&mg) {
        const auto sl = slots(mg);
        c.terms += sl.first;
        c.pats += sl.second;
        c.groups.push_back(std::move(mg));
    };
    std::vector<int> order_g;
    for (size_t g = 0; g < hp.groups.size(); ++g) {
        if (hp.groups[g].x != 0u) {
            order_g.push_back(int(g));
        } else if (diag_terms) {                    // first, in the first sweep
            MGroup mg = merge(hp.groups[g]);
            if (mg.n_terms == 0) continue;
            if (!fits(sc[0], mg)) return;           // more terms than a sweep holds (sp.ok false)
            add(sc[0], std::move(mg));
        }
    }
    std::stable_sort(order_g.begin(), order_g.end(),
                     [&](int p, int q) { return hp.groups[p].x > hp.groups[q].x; });
    for (int g : order_g) {
        const GroupDesc &G = hp.groups[g];
        MGroup mg = merge(G);
        if (mg.n_terms == 0) continue;              // every term cancels
        if (!fits(SC{}, mg)) return;                // more terms than a sweep holds
        const uint32_t H = G.x & ~lowm;
        if (__builtin_popcount(H) > fmax) {
            wide.push_back(std::move(mg));
            continue;
        }
        int best = -1, best_add = 1 << 30;
        for (size_t c = 0; c < sc.size(); ++c) {
            const int sz = __builtin_popcount(sc[c].F | H);
            if (sz > fmax || !fits(sc[c], mg)) continue;
            const int add = sz - __builtin_popcount(sc[c].F);
            if (add < best_add) {
                best_add = add;
                best = int(c);
            }
        }
        if (best < 0) {
            sc.push_back(SC{});
            best = int(sc.size()) - 1;
        }
        sc[best].F |= H;
        add(sc[best], std::move(mg));
    }
    for (MGroup &mg : wide) {
        if (!fits(sc.back(), mg)) sc.push_back(SC{});
        add(sc.back(), std::move(mg));
    }
    for (size_t c = 0; c < sc.size(); ++c) {
        SweepDesc W{};
        W.g_begin = int(sp.groups.size());
        W.p_begin = int(sp.pat.size());
        W.t_begin = int(sp.tz.size());
        W.order = int(c);
        W.diag = c == 0 ? 1 : 0;
        W.fast = lowm | sc[c].F;
        for (const MGroup &mg : sc[c].groups) {
            SGroup sg{};
            sg.x = mg.x;
            bool multi = false;
            for (const auto &ts : mg.pats) multi = multi || ts.size() > 1;
            for (size_t k = 0; k < mg.xb.size(); ++k) sg.xbits |= uint32_t(mg.xb[k]) << (5 * k);
            // parity form: the nonempty patterns are exactly those of one
            // parity of the X bits and share one merged term (a hopping
            // XX + YY pair: the states whose two bits differ); the kernel
            // then tests popc(i & x) instead of indexing patterns
            int parity = -1;
            if (!multi && !mg.xb.empty()) {
                const MTerm *first = nullptr;
                bool same = true;
                int par_nonempty = -1;
                for (size_t pv = 0; pv < mg.pats.size() && same; ++pv) {
                    const int pp = __builtin_popcount(uint32_t(pv)) & 1;
                    const auto &ts = mg.pats[pv];
                    if (ts.empty()) {
                        if (par_nonempty == pp) same = false;
                        continue;
                    }
                    if (par_nonempty < 0) par_nonempty = pp;
                    if (par_nonempty != pp) same = false;
                    if (!first) first = &ts[0];
                    else same = same && ts[0].z == first->z && ts[0].a == first->a && ts[0].b == first->b;
                }
                // every pattern of that parity must be nonempty
                if (same && first && par_nonempty >= 0) {
                    for (size_t pv = 0; pv < mg.pats.size(); ++pv)
                        if ((__builtin_popcount(uint32_t(pv)) & 1) == par_nonempty && mg.pats[pv].empty()) same = false;
                }
                if (same && first) parity = par_nonempty;
                if (parity >= 0) {
                    sg.pat = int(sp.tz.size()) - W.t_begin;
                    sp.tz.push_back(first->z);
                    sp.ta.push_back(first->a);
                    sp.tb.push_back(first->b);
                }
            }
            if (parity >= 0) {
                // one term slot (above)
            } else if (!multi) {
                // one term slot per pattern, in pattern order (zero for an
                // empty pattern): the pattern indexes its term directly
                sg.pat = int(sp.tz.size()) - W.t_begin;
                for (const auto &ts : mg.pats) {
                    const MTerm m = ts.empty() ? MTerm{0u, 0.0, 0.0} : ts[0];
                    sp.tz.push_back(m.z);
                    sp.ta.push_back(m.a);
                    sp.tb.push_back(m.b);
                }
            } else {
                sg.pat = int(sp.pat.size()) - W.p_begin;
                for (const auto &ts : mg.pats) {
                    const uint32_t first = ts.empty() ? 0u : uint32_t(int(sp.tz.size()) - W.t_begin);
                    sp.pat.push_back(first | uint32_t(ts.size()) << 16);
                    for (const MTerm &m : ts) {
                        sp.tz.push_back(m.z);
                        sp.ta.push_back(m.a);
                        sp.tb.push_back(m.b);
                    }
                }
            }
            sg.flags = uint32_t(mg.xb.size()) | (mg.has_b ? 1u << 8 : 0u) | (multi ? 1u << 9 : 0u) |
                       (parity >= 0 ? 1u << 10 | uint32_t(parity) << 11 : 0u);
            if (mg.x != 0u && parity < 0) sp.all_parity = false;
            sp.groups.push_back(sg);
        }
        W.g_end = int(sp.groups.size());
        W.n_pat = int(sp.pat.size()) - W.p_begin;
        W.t_count = int(sp.tz.size()) - W.t_begin;
        // counter bit k -> global bit ord[k]: the low run, the fast bits, the rest
        std::vector<int> ord;
        for (int q = 0; q < mlo; ++q) ord.push_back(q);
        for (int q = mlo; q < n; ++q)
            if ((sc[c].F >> q) & 1u) ord.push_back(q);
        for (int q = mlo; q < n; ++q)
            if (!((sc[c].F >> q) & 1u)) ord.push_back(q);
        for (int byte = 0; byte < 4; ++byte)
            for (uint32_t v = 0; v < 256; ++v) {
                uint32_t a = 0;
                for (int t = 0; t < 8; ++t) {
                    const int k = 8 * byte + t;
                    if (k < n && ((v >> t) & 1u)) a |= 1u << ord[k];
                }
                sp.order.push_back(a);
            }
        sp.sweeps.push_back(W);
    }
    sp.ok = true;
}

// Builds the device plan of the kept terms into a new HamDev and swaps it
// into the handle only when every step has succeeded; on failure the
// handle keeps its previous plan.
vqe_status build_ham_plan(vqe_ctx *h) {
    HamPlan hp;
    make_ham_plan(h->cx, h->cz, h->cc, h->keep, hp);
    HamDev nd;
    nd.n_groups = int(hp.groups.size());
    nd.n_groups_nonempty = hp.n_groups_nonempty;
    vqe_status st = VQE_OK;
    auto bail = [&](vqe_status e) {
        nd.release();
        return e;
    };
    // The diagonal of H is optional: it is built when it fits in a quarter
    // of the free memory (or in the buffer of the previous plan, which is
    // then reused and written last, once nothing else can fail).
    const bool want_diag =
        !hp.groups.empty() && hp.groups[0].x == 0u && hp.groups[0].t_mid > hp.groups[0].t_begin;
    const size_t diag_bytes = h->state_elems() * (h->prec == VQE_C128 ? sizeof(double) : sizeof(float));
    bool reuse_diag = false;
    if (want_diag) {
        if (h->hd.d_hdiag.p && h->hd.d_hdiag.bytes >= diag_bytes) {
            reuse_diag = true;
            nd.hdiag_ok = true;
        } else {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
                cudaGetLastError();
                free_b = 0;
            }
            if (diag_bytes <= free_b / 4 && ensure(h, nd.d_hdiag, diag_bytes, "diagonal of H") == VQE_OK)
                nd.hdiag_ok = true;
            h->err.clear();
        }
    }
    std::vector<uint32_t> z0;
    std::vector<double> c0;
    if (nd.hdiag_ok) {
        const GroupDesc &G0 = hp.groups[0];
        z0.assign(hp.tz.begin() + G0.t_begin, hp.tz.begin() + G0.t_mid);
        c0.assign(hp.tc.begin() + G0.t_begin, hp.tc.begin() + G0.t_mid);
        if ((st = upload(h, nd.d_hdiag_z, z0, "diagonal terms")) != VQE_OK) return bail(st);
        if ((st = upload(h, nd.d_hdiag_c, c0, "diagonal terms")) != VQE_OK) return bail(st);
    }
    {
        WinPlan wp;
        plan_windows(h->n, h->prec, hp, !nd.hdiag_ok, wp);
        nd.wins = wp.wins;
        nd.win_tiles = wp.win_tiles;
        nd.n_wide = int(wp.wide.size());
        if ((st = upload(h, nd.d_wgroups, wp.groups, "window groups")) != VQE_OK) return bail(st);
        if ((st = upload(h, nd.d_wterms, wp.terms, "window terms")) != VQE_OK) return bail(st);
        if ((st = upload(h, nd.d_whoff, wp.hoff, "window offsets")) != VQE_OK) return bail(st);
        if ((st = upload(h, nd.d_wide, wp.wide, "wide groups")) != VQE_OK) return bail(st);
        // windowed apply-H (same windows and groups): psi is read and lambda
        // read and written once per window, against one gathered read of psi
        // per group in the global sweep.
        nd.win_possible = wp.wide.empty() && !wp.wins.empty();
    }
    bool sweep_all_parity = false;
    {
        // bit-ordered sweeps: psi read and lambda written once per sweep, the
        // gathers served by L2
        SweepPlan sp;
        plan_sweeps(h->n, h->prec, hp, !nd.hdiag_ok, sp);
        nd.sweep_possible = sp.ok && !sp.sweeps.empty();
        sweep_all_parity = sp.all_parity;
        if (nd.sweep_possible) {
            nd.sweeps = sp.sweeps;
            if ((st = upload(h, nd.d_sorder, sp.order, "sweep orders")) != VQE_OK) return bail(st);
            if ((st = upload(h, nd.d_sgroups, sp.groups, "sweep groups")) != VQE_OK) return bail(st);
            if ((st = upload(h, nd.d_spat, sp.pat, "sweep patterns")) != VQE_OK) return bail(st);
            if ((st = upload(h, nd.d_stz, sp.tz, "sweep terms")) != VQE_OK) return bail(st);
            if (h->prec == VQE_C128) {
                if ((st = upload(h, nd.d_sta, sp.ta, "sweep terms")) != VQE_OK) return bail(st);
                if ((st = upload(h, nd.d_stb, sp.tb, "sweep terms")) != VQE_OK) return bail(st);
            } else {
                std::vector<float> fa(sp.ta.begin(), sp.ta.end()), fb(sp.tb.begin(), sp.tb.end());
                if ((st = upload(h, nd.d_sta, fa, "sweep terms")) != VQE_OK) return bail(st);
                if ((st = upload(h, nd.d_stb, fb, "sweep terms")) != VQE_OK) return bail(st);
            }
        }
        // default form (mode -1): the bit-ordered sweeps when every group
        // takes their parity form (hopping Hamiltonians: at 32 qubits
        // complex64 269 ms against 342 for the windows and 393 for the
        // global sweep, FP64 671 / 898 / 2000 ms; at 24 qubits the sweeps
        // are fastest too), else the windows when they hold many groups each
        // (the synthetic molecular Hamiltonian at 24 qubits: windows 69 ms,
        // sweeps 229 ms, global 167 ms), else the global sweep.
        // vqe_set_apply_mode and the autotuner override the choice.
        nd.apply_default = nd.sweep_possible && sweep_all_parity ? 2
                         : (nd.win_possible && hp.groups.size() >= 10 * nd.wins.size() ? 1 : 0);
        nd.apply_form = resolve_apply_form(h->apply_mode, nd);
    }
    if ((st = upload(h, nd.d_groups, hp.groups, "groups")) != VQE_OK) return bail(st);
    if ((st = upload(h, nd.d_tz, hp.tz, "terms")) != VQE_OK) return bail(st);
    if (h->prec == VQE_C128) {
        if ((st = upload(h, nd.d_tc, hp.tc, "terms")) != VQE_OK) return bail(st);
    } else {
        std::vector<float> tcf(hp.tc.begin(), hp.tc.end());
        if ((st = upload(h, nd.d_tc, tcf, "terms")) != VQE_OK) return bail(st);
    }
    if (nd.hdiag_ok) {
        if (reuse_diag) nd.d_hdiag.swap(h->hd.d_hdiag);   // the old plan gives up its buffer
        cudaError_t e = h->prec == VQE_C128
            ? launch_build_hdiag<double>(static_cast<const uint32_t *>(nd.d_hdiag_z.p),
                                         static_cast<const double *>(nd.d_hdiag_c.p),
                                         int(z0.size()), h->n, nd.d_hdiag.p, h->sms, h->stream)
            : launch_build_hdiag<float>(static_cast<const uint32_t *>(nd.d_hdiag_z.p),
                                        static_cast<const double *>(nd.d_hdiag_c.p),
                                        int(z0.size()), h->n, nd.d_hdiag.p, h->sms, h->stream);
        if (e != cudaSuccess) {
            // the previous plan's diagonal may be overwritten: no plan is usable
            nd.release();
            h->hd.release();
            h->hd = HamDev{};
            h->ham_set = false;
            return cuda_fail(h, e, "launch_build_hdiag");
        }
        h->stats.kernel_launches++;
    }
    std::swap(h->hd, nd);
    nd.release();
    h->stats.n_groups = h->hd.n_groups_nonempty;
    return VQE_OK;
}

// ---------------------------------------------------------------- buffers

int capacity(const vqe_ctx *h, bool grad) {
    const size_t per = h->state_bytes() * (grad ? 2 : 1);
    if (!h->ws) return 0;
    return int(std::min<size_t>(h->ws_bytes / per, 65535));   // grid.y limit
}

// Library-owned workspace for `batch` states (chunked runs when fewer fit).
// A larger workspace is allocated before the old one is released; if it
// cannot be had, a workspace that already holds one state set is kept and
// the run goes in chunks, so a failure never loses the current workspace.
vqe_status ensure_workspace(vqe_ctx *h, int batch, bool grad) {
    const size_t one = h->state_bytes() * (grad ? 2 : 1);
    if (h->ws && !h->ws_owned) {
        if (capacity(h, grad) < 1)
            return fail(h, VQE_ERR_ARG, "bound workspace is smaller than one state set");
        return VQE_OK;
    }
    const size_t want = one * size_t(batch);
    if (h->ws && h->ws_bytes >= want) return VQE_OK;
    const bool usable = h->ws && h->ws_bytes >= one;
    size_t freeb = 0, total = 0;
    VQE_CUDA(h, cudaMemGetInfo(&freeb, &total));
    const size_t bytes = std::min(want, std::max(one, freeb / 10 * 9));
    if (bytes > freeb || (usable && bytes <= h->ws_bytes)) {
        if (usable) return VQE_OK;
        return fail(h, VQE_ERR_OOM, "state workspace does not fit in device memory");
    }
    DevBuf nb;
    vqe_status st = ensure(h, nb, bytes, "state workspace");
    if (st != VQE_OK) {
        if (usable) {
            h->err.clear();
            return VQE_OK;
        }
        return st;
    }
    h->ws_own.release();
    h->ws_own.swap(nb);
    h->ws = h->ws_own.p;
    h->ws_bytes = h->ws_own.bytes;
    h->ws_owned = true;
    return VQE_OK;
}

int blocks_per_state(const vqe_ctx *h, int batch) {
    const uint64_t work = uint64_t(1) << std::max(0, h->n - 1);
    int bps = (h->sms * 4 + batch - 1) / batch;
    const uint64_t cap = (work + kEnergyThreads - 1) / kEnergyThreads;
    if (uint64_t(bps) > cap) bps = int(cap);
    return std::max(1, bps);
}

vqe_status ensure_scratch(vqe_ctx *h, int batch) {
    const bool c128 = h->prec == VQE_C128;
    const size_t coef_b = c128 ? sizeof(RotCoef<double>) : sizeof(RotCoef<float>);
    vqe_status st;
    const size_t cs = std::max(h->plan[0].coef_stride, h->plan[1].coef_stride);
    const size_t ds = std::max(h->plan[0].dtab_stride, h->plan[1].dtab_stride);
    if ((st = ensure(h, h->d_coefs, coef_b * cs * batch + 16, "coefficients")) != VQE_OK)
        return st;
    if ((st = ensure(h, h->d_dtab, h->elem_bytes() * ds * batch + 16, "tables")) != VQE_OK)
        return st;
    // blocks_per_state(B) * B <= sms * 4 + B - 1 for every chunk size B <= batch
    if ((st = ensure(h, h->d_epart, sizeof(double) * 3 * (size_t(h->sms) * 4 + size_t(batch)) + 16,
                     "partials")) != VQE_OK)
        return st;
    if ((st = ensure(h, h->d_out, sizeof(double) * 4 * batch + 16, "results")) != VQE_OK) return st;
    if ((st = ensure(h, h->d_params, sizeof(double) * h->n_params * batch + 16, "params")) != VQE_OK)
        return st;
    return VQE_OK;
}

vqe_status ensure_grad_scratch(vqe_ctx *h, int batch) {
    return ensure(h, h->d_gpart, sizeof(double) * h->plan[1].grad_stride * batch + 16, "grad partials");
}

// ---------------------------------------------------------------- pipelines

template <typename T>
cudaError_t launch_any_pass(vqe_ctx *h, const vqe_ctx::DevPlan &P, const PassDesc *dd,
                            const PassDesc &dh, int B, void *psi, void *lam, RotCoef<T> *coefs,
                            double *gpart, bool backward, int init_zero) {
    return launch_pass<T>(dd, dh, h->n, B, psi, lam, h->state_elems(), coefs, P.coef_stride,
                          h->d_dtab.p, P.dtab_stride, gpart, P.grad_stride, backward, init_zero,
                          h->stream);
}

// Particle-conserving forward sweep: (cos, sin) of every excitation, then
// the passes in order, the first one starting from psi_HF.
template <typename T>
vqe_status run_forward_pc(vqe_ctx *h, const double *params_dev, int B, void *psi) {
    const int K = h->n_params;
    T *cs = static_cast<T *>(h->d_coefs.p);
    VQE_CUDA(h, launch_exc_stage<T>(params_dev, K, B, cs, h->stream));
    h->stats.kernel_launches++;
    const int mk = prof_begin(h, 0);
    for (size_t p = 0; p < h->pc_passes.size(); ++p) {
        VQE_CUDA(h, launch_exc_pass<T>(h->pc_passes[p], static_cast<const ExcGate *>(h->d_pc_gates.p),
                                       static_cast<const uint32_t *>(h->d_pc_hoff.p), h->n, B, psi,
                                       nullptr, h->state_elems(), cs, K, nullptr, 0, false,
                                       p == 0 ? 1 : 0, h->hf_index, h->stream));
        h->stats.kernel_launches++;
    }
    prof_end(h, mk, int(h->pc_passes.size()));
    return VQE_OK;
}

template <typename T>
vqe_status run_backward_pc(vqe_ctx *h, int B, void *psi, void *lam) {
    const int K = h->n_params;
    const T *cs = static_cast<const T *>(h->d_coefs.p);
    double *gpart = static_cast<double *>(h->d_gpart.p);
    const int mk = prof_begin(h, 3);
    for (int p = int(h->pc_passes.size()) - 1; p >= 0; --p) {
        VQE_CUDA(h, launch_exc_pass<T>(h->pc_passes[p], static_cast<const ExcGate *>(h->d_pc_gates.p),
                                       static_cast<const uint32_t *>(h->d_pc_hoff.p), h->n, B, psi,
                                       lam, h->state_elems(), cs, K, gpart, h->plan[1].grad_stride,
                                       true, 0, h->hf_index, h->stream));
        h->stats.kernel_launches++;
    }
    prof_end(h, mk, int(h->pc_passes.size()));
    return VQE_OK;
}

template <typename T>
vqe_status run_forward(vqe_ctx *h, int which, const double *params_dev, int B, void *psi) {
    if (h->ansatz == 1) return run_forward_pc<T>(h, params_dev, B, psi);
    cudaStream_t s = h->stream;
    const vqe_ctx::DevPlan &P = h->plan[which];
    auto *coefs = static_cast<RotCoef<T> *>(h->d_coefs.p);
    VQE_CUDA(h, launch_stage<T>(static_cast<const StageSlot *>(P.d_stage.p), P.n_stage, h->n,
                                h->depth, params_dev, B, coefs, P.coef_stride, h->d_dtab.p,
                                P.dtab_stride, s));
    h->stats.kernel_launches++;
    const PassDesc *dd = static_cast<const PassDesc *>(P.d_fwd.p);
    const int mk = prof_begin(h, 0);
    for (size_t p = 0; p < P.fwd.size(); ++p) {
        VQE_CUDA(h, launch_any_pass<T>(h, P, dd + p, P.fwd[p], B, psi, nullptr, coefs, nullptr,
                                       false, p == 0 ? 1 : 0));
        h->stats.kernel_launches++;
    }
    prof_end(h, mk, int(P.fwd.size()));
    return VQE_OK;
}

template <typename T>
vqe_status run_energy(vqe_ctx *h, int B, const void *psi, double *energies, double *norms,
                      double *unnorm) {
    if (!h->hd.wins.empty() && uint64_t(h->hd.win_tiles / int(h->hd.wins.size())) * B >= uint64_t(2 * h->sms)) {
        const int bps_wide = h->hd.n_wide ? blocks_per_state(h, B) : 0;
        const int bps_total = h->hd.win_tiles + bps_wide;
        vqe_status st = ensure(h, h->d_epart, sizeof(double) * 3 * size_t(bps_total) * B + 16, "partials");
        if (st != VQE_OK) return st;
        double *part = static_cast<double *>(h->d_epart.p);
        const int mk = prof_begin(h, 1);
        for (const WinDesc &W : h->hd.wins) {
            VQE_CUDA(h, launch_energy_win<T>(W, static_cast<const WinGroup *>(h->hd.d_wgroups.p),
                                             static_cast<const WinTerm *>(h->hd.d_wterms.p),
                                             static_cast<const uint32_t *>(h->hd.d_whoff.p),
                                             h->hd.hdiag(), h->n, B, psi, h->state_elems(), part,
                                             bps_total, h->stream));
            h->stats.kernel_launches++;
        }
        if (h->hd.n_wide) {
            VQE_CUDA(h, launch_energy_sub<T>(static_cast<const GroupDesc *>(h->hd.d_wide.p), h->hd.n_wide,
                                             static_cast<const uint32_t *>(h->hd.d_tz.p),
                                             static_cast<const double *>(h->hd.d_tc.p), h->n, B, psi,
                                             h->state_elems(), part, bps_wide, h->hd.win_tiles,
                                             bps_total, h->stream));
            h->stats.kernel_launches++;
        }
        prof_end(h, mk, int(h->hd.wins.size()) + (h->hd.n_wide ? 1 : 0));
        VQE_CUDA(h, launch_energy_finish(part, bps_total, B, energies, norms, unnorm, h->stream));
        h->stats.kernel_launches++;
        return VQE_OK;
    }
    const int bps = blocks_per_state(h, B);
    const int mk = prof_begin(h, 1);
    VQE_CUDA(h, launch_energy<T>(static_cast<const GroupDesc *>(h->hd.d_groups.p), h->hd.n_groups,
                                 static_cast<const uint32_t *>(h->hd.d_tz.p),
                                 static_cast<const double *>(h->hd.d_tc.p), h->hd.hdiag(), h->n, B, psi,
                                 h->state_elems(), static_cast<double *>(h->d_epart.p), bps,
                                 h->stream));
    prof_end(h, mk, 1);
    VQE_CUDA(h, launch_energy_finish(static_cast<double *>(h->d_epart.p), bps, B, energies, norms,
                                     unnorm, h->stream));
    h->stats.kernel_launches += 2;
    return VQE_OK;
}

template <typename T>
vqe_status energy_chunk(vqe_ctx *h, const double *params_dev, int B, double *E, double *nrm) {
    vqe_status st = run_forward<T>(h, 0, params_dev, B, h->ws);
    if (st != VQE_OK) return st;
    return run_energy<T>(h, B, h->ws, E, nrm, nullptr);
}

// lambda = H psi for B states with the fused energy E = Re<psi|lambda>/<psi|psi>.
template <typename T>
vqe_status run_apply_h(vqe_ctx *h, int B, void *psi, void *lam, double *E) {
    cudaStream_t s = h->stream;
    const size_t N = h->state_elems();
    const int mk_h = prof_begin(h, 2);
    const bool windows = h->hd.apply_form == 1;
    const uint64_t atiles = windows ? (uint64_t(1) << (h->n - h->hd.wins[0].k)) : 0;
    if (h->hd.apply_form == 2) {
        // bit-ordered sweeps: lambda accumulated sweep by sweep; the last
        // sweep writes the energy partials of its chunks (summed in chunk
        // order).  Blocks take chunks from one zeroed counter per sweep and
        // state; as many blocks as are resident at once.
        const int ns = int(h->hd.sweeps.size());
        const uint64_t nchunks = ((uint64_t(1) << h->n) + kSweepChunk - 1) / kSweepChunk;
        vqe_status st2 = ensure(h, h->d_sctr, sizeof(unsigned long long) * size_t(ns) * B, "sweep counters");
        if (st2 == VQE_OK)
            st2 = ensure(h, h->d_epart, sizeof(double) * 3 * size_t(nchunks) * B + 16, "partials");
        if (st2 != VQE_OK) return st2;
        VQE_CUDA(h, cudaMemsetAsync(h->d_sctr.p, 0, sizeof(unsigned long long) * size_t(ns) * B, s));
        size_t smem = 0;
        for (const SweepDesc &W : h->hd.sweeps)
            smem = std::max(smem, sweep_smem_bytes(W, h->prec == VQE_C128 ? 8 : 4));
        const int occ = sweep_blocks_per_sm(h->prec == VQE_C128 ? 16 : 8, smem);
        const int blocks = int(std::max<uint64_t>(1, std::min<uint64_t>(nchunks, uint64_t(h->sms) * occ / B)));
        auto *ctr = static_cast<unsigned long long *>(h->d_sctr.p);
        for (int w = 0; w < ns; ++w) {
            const SweepDesc &W = h->hd.sweeps[w];
            VQE_CUDA(h, launch_apply_h_sweep<T>(W, static_cast<const uint32_t *>(h->hd.d_sorder.p) + size_t(W.order) * 1024,
                                                static_cast<const SGroup *>(h->hd.d_sgroups.p),
                                                static_cast<const uint32_t *>(h->hd.d_spat.p),
                                                static_cast<const uint32_t *>(h->hd.d_stz.p),
                                                h->hd.d_sta.p, h->hd.d_stb.p, h->hd.hdiag(), h->n, B,
                                                psi, lam, N, w == 0 ? 1 : 0, w == ns - 1 ? 1 : 0,
                                                ctr + size_t(w) * B, static_cast<double *>(h->d_epart.p),
                                                blocks, s));
            h->stats.kernel_launches++;
        }
        prof_end(h, mk_h, ns);
        VQE_CUDA(h, launch_energy_finish(static_cast<double *>(h->d_epart.p), int(nchunks), B, E, nullptr,
                                         nullptr, s));
        h->stats.kernel_launches++;
    } else if (windows && atiles * B >= uint64_t(2 * h->sms)) {
        // windowed: lambda accumulated window by window; the last window's
        // blocks hold the partials of the energy
        const int bps_w = int(atiles);
        vqe_status st2 = ensure(h, h->d_epart, sizeof(double) * 3 * size_t(bps_w) * B + 16, "partials");
        if (st2 != VQE_OK) return st2;
        const int nw = int(h->hd.wins.size());
        for (int w = 0; w < nw; ++w) {
            VQE_CUDA(h, launch_apply_h_win<T>(h->hd.wins[w], static_cast<const WinGroup *>(h->hd.d_wgroups.p),
                                              static_cast<const WinTerm *>(h->hd.d_wterms.p),
                                              static_cast<const uint32_t *>(h->hd.d_whoff.p),
                                              h->hd.hdiag(), h->n, B, psi, lam, N, w == 0 ? 1 : 0,
                                              w == nw - 1 ? 1 : 0,
                                              static_cast<double *>(h->d_epart.p), s));
            h->stats.kernel_launches++;
        }
        prof_end(h, mk_h, nw);
        VQE_CUDA(h, launch_energy_finish(static_cast<double *>(h->d_epart.p), bps_w, B, E, nullptr,
                                         nullptr, s));
        h->stats.kernel_launches++;
    } else {
        const int bps = blocks_per_state(h, B);
        VQE_CUDA(h, launch_apply_h<T>(static_cast<const GroupDesc *>(h->hd.d_groups.p), h->hd.n_groups,
                                      static_cast<const uint32_t *>(h->hd.d_tz.p),
                                      static_cast<const double *>(h->hd.d_tc.p), h->hd.hdiag(), h->n, B,
                                      psi, lam, N, static_cast<double *>(h->d_epart.p), bps, s));
        prof_end(h, mk_h, 1);
        VQE_CUDA(h, launch_energy_finish(static_cast<double *>(h->d_epart.p), bps, B, E, nullptr,
                                         nullptr, s));
        h->stats.kernel_launches += 2;
    }
    return VQE_OK;
}

template <typename T>
vqe_status gradient_chunk(vqe_ctx *h, const double *params_dev, int B, double *grads,
                          double *E) {
    cudaStream_t s = h->stream;
    void *psi = h->ws;
    void *lam = static_cast<char *>(h->ws) + h->state_bytes() * size_t(B);
    vqe_status st = run_forward<T>(h, 1, params_dev, B, psi);
    if (st != VQE_OK) return st;
    if ((st = run_apply_h<T>(h, B, psi, lam, E)) != VQE_OK) return st;
    const vqe_ctx::DevPlan &P = h->plan[1];
    double *gpart = static_cast<double *>(h->d_gpart.p);
    if (h->ansatz == 1) {
        if ((st = run_backward_pc<T>(h, B, psi, lam)) != VQE_OK) return st;
    } else {
        auto *coefs = static_cast<RotCoef<T> *>(h->d_coefs.p);
        const PassDesc *dd = static_cast<const PassDesc *>(P.d_bwd.p);
        const int mk_b = prof_begin(h, 3);
        for (int p = int(P.bwd.size()) - 1; p >= 0; --p) {
            VQE_CUDA(h, launch_any_pass<T>(h, P, dd + p, P.bwd[p], B, psi, lam, coefs, gpart, true, 0));
            h->stats.kernel_launches++;
        }
        prof_end(h, mk_b, int(P.bwd.size()));
    }
    VQE_CUDA(h, launch_grad_finish(gpart, P.grad_stride, static_cast<const int *>(P.d_goff.p),
                                   static_cast<const int *>(P.d_gcnt.p),
                                   static_cast<const int *>(P.d_gstep.p), h->n_params, B, grads,
                                   s));
    h->stats.kernel_launches++;
    return VQE_OK;
}

template <typename T>
vqe_status pergate_chunk(vqe_ctx *h, const double *params_dev, int B, double *E, double *nrm) {
    cudaStream_t s = h->stream;
    const size_t N = h->state_elems();
    const int n = h->n, P = h->n_params;
    VQE_CUDA(h, launch_init_zero_state<T>(h->ws, N, n, B, s));
    h->stats.kernel_launches++;
    for (int l = 0; l < h->depth; ++l) {
        for (int q = 0; q < n; ++q) {
            VQE_CUDA(h, launch_gate_ry<T>(h->ws, N, n, B, q, params_dev, (l * n + q) * 2, P, s));
            VQE_CUDA(h, launch_gate_rz<T>(h->ws, N, n, B, q, params_dev, (l * n + q) * 2 + 1, P, s));
            h->stats.kernel_launches += 2;
        }
        for (int q = 0; q + 1 < n; ++q) {
            VQE_CUDA(h, launch_gate_cz<T>(h->ws, N, n, B, q, s));
            h->stats.kernel_launches++;
        }
    }
    return run_energy<T>(h, B, h->ws, E, nrm, nullptr);
}

enum class Job { Energy, Gradient, PerGate };

vqe_status run_batch(vqe_ctx *h, Job job, const double *params_dev, int batch, double *E,
                     double *nrm, double *grads) {
    if (!h->ham_set) return fail(h, VQE_ERR_STATE, "no Hamiltonian set");
    if (batch < 1) return fail(h, VQE_ERR_ARG, "batch must be >= 1");
    if (!params_dev) return fail(h, VQE_ERR_ARG, "params is NULL");
    const bool grad = job == Job::Gradient;
    vqe_status st = ensure_workspace(h, batch, grad);
    if (st != VQE_OK) return st;
    const int cap = std::max(1, std::min(batch, capacity(h, grad)));
    if ((st = ensure_scratch(h, cap)) != VQE_OK) return st;
    if (grad && (st = ensure_grad_scratch(h, cap)) != VQE_OK) return st;
    for (int b0 = 0; b0 < batch; b0 += cap) {
        const int B = std::min(cap, batch - b0);
        const double *pp = params_dev + size_t(b0) * h->n_params;
        double *e = E ? E + b0 : nullptr;
        double *nn = nrm ? nrm + b0 : nullptr;
        const bool c128 = h->prec == VQE_C128;
        switch (job) {
            case Job::Energy:
                st = c128 ? energy_chunk<double>(h, pp, B, e, nn) : energy_chunk<float>(h, pp, B, e, nn);
                break;
            case Job::PerGate:
                st = c128 ? pergate_chunk<double>(h, pp, B, e, nn) : pergate_chunk<float>(h, pp, B, e, nn);
                break;
            case Job::Gradient: {
                double *g = grads + size_t(b0) * h->n_params;
                st = c128 ? gradient_chunk<double>(h, pp, B, g, e) : gradient_chunk<float>(h, pp, B, g, e);
                break;
            }
        }
        if (st != VQE_OK) return st;
    }
    return VQE_OK;
}

bool finite_params(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

// ================================================================= C ABI

extern "C" {

const char *vqe_version(void) { return "vqe-gb300 0.1 (sm_103a)"; }

const char *vqe_last_error(vqe_handle h) { return h ? h->err.c_str() : "NULL handle"; }

vqe_status vqe_create(int n_qubits, int depth, vqe_precision precision, void *cuda_stream,
                      vqe_handle *out) {
    if (!out) return VQE_ERR_ARG;
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 32 || depth < 1 || depth > 4096) return VQE_ERR_ARG;
    if (precision != VQE_C64 && precision != VQE_C128) return VQE_ERR_ARG;
    vqe_ctx *h = new vqe_ctx();
    h->n = n_qubits;
    h->depth = depth;
    h->prec = precision;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return VQE_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return VQE_ERR_CUDA;
    }
    vqe_status st = build_plan(h);
    if (st != VQE_OK) {
        vqe_destroy(h);
        return st;
    }
    *out = h;
    return VQE_OK;
}

vqe_status vqe_create_pc(int n_qubits, int n_elec, int n_exc, const int *excitations,
                         vqe_precision precision, void *cuda_stream, vqe_handle *out) {
    if (!out) return VQE_ERR_ARG;
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 32 || n_elec < 0 || n_elec > n_qubits) return VQE_ERR_ARG;
    if (n_exc < 1 || n_exc > (1 << 20) || !excitations) return VQE_ERR_ARG;
    if (precision != VQE_C64 && precision != VQE_C128) return VQE_ERR_ARG;
    for (int j = 0; j < n_exc; ++j) {
        const int *e = excitations + 4 * j;
        const bool dbl = e[1] >= 0;
        const int cnt = dbl ? 4 : 2;
        const int modes[4] = {e[0], dbl ? e[1] : e[2], dbl ? e[2] : -1, dbl ? e[3] : -1};
        uint32_t seen = 0;
        for (int u = 0; u < cnt; ++u) {
            const int md = modes[u];
            if (md < 0 || md >= n_qubits || ((seen >> md) & 1u)) return VQE_ERR_ARG;
            seen |= 1u << md;
        }
        if (!dbl && (e[1] != -1 || e[3] != -1)) return VQE_ERR_ARG;
    }
    vqe_ctx *h = new vqe_ctx();
    h->n = n_qubits;
    h->depth = 1;
    h->prec = precision;
    h->ansatz = 1;
    h->n_elec = n_elec;
    h->hf_index = n_elec >= 64 ? ~uint64_t(0) : ((uint64_t(1) << n_elec) - 1);
    h->exc.assign(excitations, excitations + 4 * size_t(n_exc));
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return VQE_ERR_CUDA;
    }
    vqe_status st = build_plan(h);
    if (st != VQE_OK) {
        vqe_destroy(h);
        return st;
    }
    *out = h;
    return VQE_OK;
}

vqe_status vqe_destroy(vqe_handle h) {
    if (!h) return VQE_ERR_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->plan[0].release();
    h->plan[1].release();
    h->hd.release();
    h->d_pc_gates.release();
    h->d_pc_hoff.release();
    for (DevBuf *b : {&h->ws_own, &h->d_params, &h->d_coefs, &h->d_dtab, &h->d_gpart, &h->d_epart, &h->d_sctr,
                      &h->d_out, &h->hb_params, &h->hb_e, &h->hb_n, &h->hb_g})
        b->release();
    delete h;
    return VQE_OK;
}

vqe_status vqe_set_plan_options(vqe_handle h, int tile_bits_max, int run_bits, int reg_bits) {
    if (!h) return VQE_ERR_ARG;
    if (h->ansatz == 1)
        return fail(h, VQE_ERR_ARG, "plan options apply to the hardware-efficient ansatz");
    PlanOptions o;
    o.tile_bits_max = tile_bits_max;
    o.run_bits = run_bits;
    o.reg_bits = reg_bits;
    std::string err;
    if (!options_valid(o, h->prec, err)) return fail(h, VQE_ERR_ARG, err);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    // reg_bits 5 applies to the energy plan; the gradient plan holds two buffers per thread
    PlanOptions og = o;
    if (og.reg_bits > 4) og.reg_bits = 4;
    if (!options_valid(og, h->prec, err)) return fail(h, VQE_ERR_ARG, err);
    const PlanOptions old0 = h->plan[0].opts, old1 = h->plan[1].opts;
    h->plan[0].opts = o;
    h->plan[1].opts = og;
    vqe_status st = build_plan(h);
    if (st != VQE_OK) {
        h->plan[0].opts = old0;
        h->plan[1].opts = old1;
        build_plan(h);
        return st;
    }
    h->state_valid = false;
    return VQE_OK;
}

vqe_status vqe_set_apply_mode(vqe_handle h, int mode, int *form) {
    if (!h) return VQE_ERR_ARG;
    if (mode < -1 || mode > 2) return fail(h, VQE_ERR_ARG, "apply mode must be -1, 0, 1 or 2");
    h->apply_mode = mode;
    h->hd.apply_form = resolve_apply_form(mode, h->hd);
    if (form) *form = h->hd.apply_form;
    return VQE_OK;
}

vqe_status vqe_workspace_size(vqe_handle h, int batch, int want_gradient, size_t *bytes) {
    if (!h || !bytes || batch < 1) return fail(h, VQE_ERR_ARG, "bad argument");
    *bytes = h->state_bytes() * (want_gradient ? 2 : 1) * size_t(batch);
    return VQE_OK;
}

vqe_status vqe_bind_workspace(vqe_handle h, void *dev_ptr, size_t bytes) {
    if (!h) return VQE_ERR_ARG;
    if (dev_ptr == nullptr) {
        h->ws = nullptr;
        h->ws_bytes = 0;
        h->ws_owned = false;
        h->state_valid = false;
        return VQE_OK;
    }
    if (reinterpret_cast<uintptr_t>(dev_ptr) % 256 != 0)
        return fail(h, VQE_ERR_ARG, "workspace must be 256-byte aligned");
    if (bytes < h->state_bytes())
        return fail(h, VQE_ERR_ARG, "workspace smaller than one state");
    h->ws_own.release();
    h->ws = dev_ptr;
    h->ws_bytes = bytes;
    h->ws_owned = false;
    h->state_valid = false;
    return VQE_OK;
}

vqe_status vqe_set_hamiltonian(vqe_handle h, const uint64_t *x_masks, const uint64_t *z_masks,
                               const double *coeffs, size_t n_terms) {
    if (!h) return VQE_ERR_ARG;
    if (n_terms > 0 && (!x_masks || !z_masks || !coeffs))
        return fail(h, VQE_ERR_ARG, "NULL term array");
    if (n_terms > (size_t(1) << 30)) return fail(h, VQE_ERR_ARG, "too many terms");
    const uint64_t lim = h->n >= 64 ? ~0ull : ((uint64_t(1) << h->n) - 1);
    for (size_t t = 0; t < n_terms; ++t) {
        if ((x_masks[t] & ~lim) || (z_masks[t] & ~lim))
            return fail(h, VQE_ERR_ARG, "Pauli mask has a bit at or above n_qubits (term " +
                                            std::to_string(t) + ")");
        if (!std::isfinite(coeffs[t]))
            return fail(h, VQE_ERR_ARG, "non-finite coefficient (term " + std::to_string(t) + ")");
    }
    std::vector<uint64_t> cx, cz;
    std::vector<double> cc;
    canonicalise(x_masks, z_masks, coeffs, n_terms, cx, cz, cc);
    std::vector<uint8_t> keep(cc.size(), 1);
    h->cx.swap(cx);
    h->cz.swap(cz);
    h->cc.swap(cc);
    h->keep.swap(keep);
    vqe_status st = build_ham_plan(h);
    if (st != VQE_OK) {   // the previous terms and cutoff stay, with their plan
        h->cx.swap(cx);
        h->cz.swap(cz);
        h->cc.swap(cc);
        h->keep.swap(keep);
        return st;
    }
    h->ham_set = true;
    h->stats.n_terms_input = n_terms;
    h->stats.n_terms_canonical = h->cc.size();
    h->stats.n_terms_kept = h->cc.size();
    h->stats.sum_abs_dropped = 0.0;
    h->stats.threshold = 0.0;
    return VQE_OK;
}

vqe_status vqe_slim(vqe_handle h, double threshold, size_t *n_kept, double *sum_abs_dropped) {
    if (!h) return VQE_ERR_ARG;
    if (!h->ham_set) return fail(h, VQE_ERR_STATE, "no Hamiltonian set");
    if (!(threshold >= 0.0) || !std::isfinite(threshold))
        return fail(h, VQE_ERR_ARG, "threshold must be finite and >= 0");
    std::vector<uint8_t> old = h->keep;
    size_t kept = 0;
    const double dropped = slim_keep(h->cc, threshold, h->keep, kept);
    vqe_status st = build_ham_plan(h);
    if (st != VQE_OK) {
        h->keep.swap(old);
        return st;
    }
    h->stats.n_terms_kept = kept;
    h->stats.sum_abs_dropped = dropped;
    h->stats.threshold = threshold;
    if (n_kept) *n_kept = kept;
    if (sum_abs_dropped) *sum_abs_dropped = dropped;
    return VQE_OK;
}

vqe_status vqe_apply_ansatz(vqe_handle h, const double *params) {
    if (!h) return VQE_ERR_ARG;
    if (!params) return fail(h, VQE_ERR_ARG, "params is NULL");
    if (!finite_params(params, h->n_params)) return fail(h, VQE_ERR_ARG, "non-finite parameter");
    vqe_status st = ensure_workspace(h, 1, false);
    if (st != VQE_OK) return st;
    if ((st = ensure_scratch(h, 1)) != VQE_OK) return st;
    VQE_CUDA(h, cudaMemcpyAsync(h->d_params.p, params, sizeof(double) * h->n_params,
                                cudaMemcpyHostToDevice, h->stream));
    const double *pd = static_cast<const double *>(h->d_params.p);
    st = h->prec == VQE_C128 ? run_forward<double>(h, 0, pd, 1, h->ws)
                             : run_forward<float>(h, 0, pd, 1, h->ws);
    if (st != VQE_OK) return st;
    VQE_CUDA(h, cudaStreamSynchronize(h->stream));
    h->state_valid = true;
    return VQE_OK;
}

vqe_status vqe_energy(vqe_handle h, double *energy, double *norm) {
    if (!h) return VQE_ERR_ARG;
    if (!h->ham_set) return fail(h, VQE_ERR_STATE, "no Hamiltonian set");
    if (!h->state_valid) return fail(h, VQE_ERR_STATE, "no state: call vqe_apply_ansatz first");
    vqe_status st = ensure_scratch(h, 1);
    if (st != VQE_OK) return st;
    double *out = static_cast<double *>(h->d_out.p);
    st = h->prec == VQE_C128 ? run_energy<double>(h, 1, h->ws, out, out + 1, nullptr)
                             : run_energy<float>(h, 1, h->ws, out, out + 1, nullptr);
    if (st != VQE_OK) return st;
    double host[2];
    VQE_CUDA(h, cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, h->stream));
    VQE_CUDA(h, cudaStreamSynchronize(h->stream));
    if (energy) *energy = host[0];
    if (norm) *norm = host[1];
    return VQE_OK;
}

vqe_status vqe_get_state(vqe_handle h, void *host_out, size_t bytes) {
    if (!h) return VQE_ERR_ARG;
    if (!host_out || bytes != h->state_bytes()) return fail(h, VQE_ERR_ARG, "bad output buffer size");
    if (!h->state_valid) return fail(h, VQE_ERR_STATE, "no state: call vqe_apply_ansatz first");
    VQE_CUDA(h, cudaMemcpyAsync(host_out, h->ws, bytes, cudaMemcpyDeviceToHost, h->stream));
    VQE_CUDA(h, cudaStreamSynchronize(h->stream));
    return VQE_OK;
}

vqe_status vqe_gradient(vqe_handle h, const double *params, double *grad, double *energy) {
    if (!h) return VQE_ERR_ARG;
    if (!params || !grad) return fail(h, VQE_ERR_ARG, "NULL argument");
    return vqe_gradient_batch(h, params, 1, grad, energy);
}

vqe_status vqe_energy_batch_dev(vqe_handle h, const double *params_dev, int batch,
                                double *energies_dev, double *norms_dev) {
    if (!h) return VQE_ERR_ARG;
    if (!energies_dev) return fail(h, VQE_ERR_ARG, "energies is NULL");
    h->state_valid = false;
    return run_batch(h, Job::Energy, params_dev, batch, energies_dev, norms_dev, nullptr);
}

vqe_status vqe_gradient_batch_dev(vqe_handle h, const double *params_dev, int batch,
                                  double *grads_dev, double *energies_dev) {
    if (!h) return VQE_ERR_ARG;
    if (!grads_dev) return fail(h, VQE_ERR_ARG, "grads is NULL");
    h->state_valid = false;
    return run_batch(h, Job::Gradient, params_dev, batch, energies_dev, nullptr, grads_dev);
}

vqe_status vqe_energy_batch_pergate_dev(vqe_handle h, const double *params_dev, int batch,
                                        double *energies_dev, double *norms_dev) {
    if (!h) return VQE_ERR_ARG;
    if (h->ansatz == 1)
        return fail(h, VQE_ERR_ARG, "the one-gate-per-pass kernel is for the hardware-efficient ansatz");
    if (!energies_dev) return fail(h, VQE_ERR_ARG, "energies is NULL");
    h->state_valid = false;
    return run_batch(h, Job::PerGate, params_dev, batch, energies_dev, norms_dev, nullptr);
}

static vqe_status host_batch(vqe_handle h, Job job, const double *params, int batch, double *E,
                             double *nrm, double *grads) {
    if (!h) return VQE_ERR_ARG;
    if (!params || batch < 1) return fail(h, VQE_ERR_ARG, "bad params/batch");
    if (!finite_params(params, size_t(batch) * h->n_params))
        return fail(h, VQE_ERR_ARG, "non-finite parameter");
    const size_t P = size_t(h->n_params) * batch;
    DevBuf &dp = h->hb_params, &de = h->hb_e, &dn = h->hb_n, &dg = h->hb_g;
    vqe_status st = ensure(h, dp, P * sizeof(double), "params");
    if (st == VQE_OK) st = ensure(h, de, batch * sizeof(double), "energies");
    if (st == VQE_OK) st = ensure(h, dn, batch * sizeof(double), "norms");
    if (st == VQE_OK && job == Job::Gradient) st = ensure(h, dg, P * sizeof(double), "grads");
    if (st == VQE_OK) {
        cudaError_t e = cudaMemcpyAsync(dp.p, params, P * sizeof(double), cudaMemcpyHostToDevice,
                                        h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMemcpyAsync(params)");
    }
    if (st == VQE_OK) {
        h->state_valid = false;
        st = run_batch(h, job, static_cast<double *>(dp.p), batch, static_cast<double *>(de.p),
                       job == Job::Gradient ? nullptr : static_cast<double *>(dn.p),
                       static_cast<double *>(dg.p));
    }
    if (st == VQE_OK && E) {
        cudaError_t e = cudaMemcpyAsync(E, de.p, batch * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMemcpyAsync(energies)");
    }
    if (st == VQE_OK && nrm && job != Job::Gradient) {
        cudaError_t e = cudaMemcpyAsync(nrm, dn.p, batch * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMemcpyAsync(norms)");
    }
    if (st == VQE_OK && grads) {
        cudaError_t e = cudaMemcpyAsync(grads, dg.p, P * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMemcpyAsync(grads)");
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (st == VQE_OK && e != cudaSuccess) st = cuda_fail(h, e, "cudaStreamSynchronize");
    return st;
}

vqe_status vqe_energy_batch(vqe_handle h, const double *params, int batch, double *energies,
                            double *norms) {
    return host_batch(h, Job::Energy, params, batch, energies, norms, nullptr);
}

vqe_status vqe_gradient_batch(vqe_handle h, const double *params, int batch, double *grads,
                              double *energies) {
    if (!grads) return fail(h, VQE_ERR_ARG, "grads is NULL");
    return host_batch(h, Job::Gradient, params, batch, energies, nullptr, grads);
}

vqe_status vqe_profile(vqe_handle h, int enable) {
    if (!h) return VQE_ERR_ARG;
    vqe_status st = prof_collect(h);
    if (st != VQE_OK) return st;
    h->prof = enable != 0;
    h->times = vqe_kernel_times{};
    return VQE_OK;
}

vqe_status vqe_profile_read(vqe_handle h, vqe_kernel_times *out) {
    if (!h || !out) return VQE_ERR_ARG;
    vqe_status st = prof_collect(h);
    if (st != VQE_OK) return st;
    *out = h->times;
    return VQE_OK;
}

vqe_status vqe_get_stats(vqe_handle h, vqe_stats *out) {
    if (!h || !out) return VQE_ERR_ARG;
    *out = h->stats;
    return VQE_OK;
}

vqe_status vqe_autotune(vqe_handle h, const double *params_dev, int batch, int gradient,
                        double budget_ms, vqe_tuning *out) {
    if (!h) return VQE_ERR_ARG;
    if (!h->ham_set) return fail(h, VQE_ERR_STATE, "no Hamiltonian set");
    if (!params_dev || batch < 1) return fail(h, VQE_ERR_ARG, "bad params/batch");
    const Job job = gradient ? Job::Gradient : Job::Energy;
    vqe_status st;
    if ((st = ensure(h, h->hb_e, sizeof(double) * batch, "tuning energies")) != VQE_OK) return st;
    if (gradient && (st = ensure(h, h->hb_g, sizeof(double) * h->n_params * size_t(batch),
                                  "tuning gradients")) != VQE_OK)
        return st;
    double *E = static_cast<double *>(h->hb_e.p);
    double *G = gradient ? static_cast<double *>(h->hb_g.p) : nullptr;
    cudaEvent_t ea = nullptr, eb = nullptr;
    VQE_CUDA(h, cudaEventCreate(&ea));
    if (cudaEventCreate(&eb) != cudaSuccess) {
        cudaEventDestroy(ea);
        return cuda_fail(h, cudaGetLastError(), "cudaEventCreate");
    }
    auto timed = [&](auto &&fn, float &ms) -> vqe_status {
        cudaEventRecord(ea, h->stream);
        vqe_status s2 = fn();
        cudaEventRecord(eb, h->stream);
        cudaError_t e = cudaEventSynchronize(eb);
        if (s2 != VQE_OK) return s2;
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
        e = cudaEventElapsedTime(&ms, ea, eb);
        return e == cudaSuccess ? VQE_OK : cuda_fail(h, e, "cudaEventElapsedTime");
    };
    auto run_job = [&]() { return run_batch(h, job, params_dev, batch, E, nullptr, G); };
    // candidates: the default plan first, then other tile sizes, register
    // counts and run lengths ("fusion width": qubits per pass and the passes
    // per layer follow from the tile size)
    const bool c128 = h->prec == VQE_C128;
    std::vector<PlanOptions> cands;
    const int list128[][3] = {{0, 0, 0}, {10, 2, 3}, {12, 2, 3}, {11, 2, 2}, {11, 3, 3}, {9, 2, 2}};
    const int list64[][3] = {{0, 0, 0}, {12, 3, 4}, {10, 3, 4}, {11, 3, 3}, {12, 4, 4}, {13, 3, 4}};
    for (const auto &c : (c128 ? list128 : list64)) {
        PlanOptions o;
        o.tile_bits_max = c[0];
        o.run_bits = c[1];
        o.reg_bits = c[2];
        std::string err;
        if (options_valid(o, h->prec, err)) cands.push_back(o);
    }
    if (h->ansatz == 1) cands.resize(1);   // one tile plan for the excitation passes
    const PlanOptions old0 = h->plan[0].opts, old1 = h->plan[1].opts;
    float best_ms = 0.f, default_ms = 0.f;
    int best = -1, tried = 0;
    double spent = 0.0;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        if (ci > 0 && spent >= budget_ms) break;
        h->plan[0].opts = cands[ci];
        h->plan[1].opts = cands[ci];
        if (h->plan[1].opts.reg_bits > 4) h->plan[1].opts.reg_bits = 4;
        if (build_plan(h) != VQE_OK) continue;
        float ms = 0.f;
        if (ci == 0 || default_ms < 2000.f) {   // untimed run first (scratch, caches)
            if ((st = run_job()) != VQE_OK) break;
        }
        if ((st = timed(run_job, ms)) != VQE_OK) break;
        spent += ms;
        ++tried;
        if (ci == 0) default_ms = ms;
        if (best < 0 || ms < best_ms) {
            best = int(ci);
            best_ms = ms;
        }
    }
    if (best < 0 || st != VQE_OK) {
        h->plan[0].opts = old0;
        h->plan[1].opts = old1;
        build_plan(h);
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        h->state_valid = false;
        return st != VQE_OK ? st : fail(h, VQE_ERR_STATE, "no tuning candidate could run");
    }
    h->plan[0].opts = cands[best];
    h->plan[1].opts = cands[best];
    if (h->plan[1].opts.reg_bits > 4) h->plan[1].opts.reg_bits = 4;
    if ((st = build_plan(h)) != VQE_OK) {
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        return st;
    }
    // the apply-H form of gradient evaluations: every possible form on the same psi
    float ms_form[3] = {0.f, 0.f, 0.f};
    if (gradient && (h->hd.win_possible || h->hd.sweep_possible)) {
        const int keep = h->hd.apply_form;
        void *psi = h->ws;
        const int B = std::max(1, std::min(batch, capacity(h, true)));
        void *lam = static_cast<char *>(h->ws) + h->state_bytes() * size_t(B);
        st = c128 ? run_forward<double>(h, 1, params_dev, B, psi) : run_forward<float>(h, 1, params_dev, B, psi);
        int best_form = -1;
        for (int form = 0; form < 3 && st == VQE_OK; ++form) {
            if ((form == 1 && !h->hd.win_possible) || (form == 2 && !h->hd.sweep_possible)) continue;
            h->hd.apply_form = form;
            auto app = [&]() {
                return c128 ? run_apply_h<double>(h, B, psi, lam, E) : run_apply_h<float>(h, B, psi, lam, E);
            };
            if ((st = app()) != VQE_OK) break;
            if ((st = timed(app, ms_form[form])) != VQE_OK) break;
            if (best_form < 0 || ms_form[form] < ms_form[best_form]) best_form = form;
        }
        h->hd.apply_form = keep;
        if (st == VQE_OK && best_form >= 0) {
            h->apply_mode = best_form;
            h->hd.apply_form = best_form;
        }
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    h->state_valid = false;
    if (st != VQE_OK) return st;
    if (out) {
        const PlanOptions r = resolve(cands[best], h->prec);
        out->tile_bits_max = r.tile_bits_max;
        out->run_bits = r.run_bits;
        out->reg_bits = r.reg_bits;
        out->apply_form = h->hd.apply_form;
        out->candidates = tried;
        out->ms_default = default_ms / batch;
        out->ms_best = best_ms / batch;
        const double per = gradient ? std::max(1, std::min(batch, capacity(h, true))) : 1;
        out->apply_ms_global = ms_form[0] / per;
        out->apply_ms_windows = ms_form[1] / per;
        out->apply_ms_sweeps = ms_form[2] / per;
    }
    return VQE_OK;
}

}  // extern "C"

// ================================================================= test hooks

#include "vqe_testing.h"

extern "C" void vqe_testing_fail_allocations(int after) { g_alloc_budget.store(after < 0 ? -1 : after); }

// ================================================================= inspection (host only)

#include "vqe_inspect.h"

extern "C" {

size_t vqe_inspect_sizeof(int which) {
    switch (which) {
        case 0: return sizeof(PassDesc);
        case 1: return sizeof(StageSlot);
        case 2: return sizeof(GroupDesc);
        case 3: return sizeof(WinDesc);
        case 4: return sizeof(WinGroup);
        case 5: return sizeof(WinTerm);
        case 6: return sizeof(ExcPass);
        case 7: return sizeof(ExcGate);
        case 8: return sizeof(SweepDesc);
        case 9: return sizeof(SGroup);
        default: return 0;
    }
}

int vqe_inspect_plan(int n_qubits, int depth, int precision, const int options[3], void *fwd,
                     void *bwd, int max_passes, void *stage, int max_stage, int *grad_map,
                     int max_params, uint64_t strides[3], int counts[3]) {
    if (n_qubits < 1 || n_qubits > 32 || depth < 1 || (precision != 0 && precision != 1)) return -1;
    HostPlan hp;
    std::string err;
    PlanOptions opt;
    if (options) {
        opt.tile_bits_max = options[0];
        opt.run_bits = options[1];
        opt.reg_bits = options[2];
    }
    if (!make_plan(n_qubits, depth, vqe_precision(precision), opt, hp, err)) return -1;
    if (counts) {
        counts[0] = int(hp.fwd.size());
        counts[1] = int(hp.stage.size());
        counts[2] = hp.n_params;
    }
    if (strides) {
        strides[0] = hp.coef_stride;
        strides[1] = hp.dtab_stride;
        strides[2] = hp.grad_stride;
    }
    if (int(hp.fwd.size()) > max_passes || int(hp.stage.size()) > max_stage ||
        hp.n_params > max_params)
        return -1;
    if (fwd) std::memcpy(fwd, hp.fwd.data(), hp.fwd.size() * sizeof(PassDesc));
    if (bwd) std::memcpy(bwd, hp.bwd.data(), hp.bwd.size() * sizeof(PassDesc));
    if (stage) std::memcpy(stage, hp.stage.data(), hp.stage.size() * sizeof(StageSlot));
    if (grad_map)
        for (int p = 0; p < hp.n_params; ++p) {
            grad_map[3 * p] = hp.goff[p];
            grad_map[3 * p + 1] = hp.gcnt[p];
            grad_map[3 * p + 2] = hp.gstep[p];
        }
    return 0;
}

int vqe_inspect_pc_plan(int n_qubits, int n_elec, int precision, int n_exc, const int *excitations,
                        void *passes, int max_passes, void *gates, int max_gates, uint32_t *hoff,
                        int max_hoff, int counts[3]) {
    if (n_qubits < 1 || n_qubits > 32 || n_exc < 1 || !excitations) return -1;
    if (n_elec < 0 || n_elec > n_qubits) return -1;
    if (precision != VQE_C64 && precision != VQE_C128) return -1;
    std::vector<int> exc(excitations, excitations + 4 * size_t(n_exc));
    PcHostPlan pp;
    std::string err;
    const uint64_t hf = n_elec >= 64 ? ~uint64_t(0) : ((uint64_t(1) << n_elec) - 1);
    if (!make_pc_plan(n_qubits, vqe_precision(precision), exc, hf, pp, err)) return -1;
    if (counts) {
        counts[0] = int(pp.passes.size());
        counts[1] = int(pp.gates.size());
        counts[2] = int(pp.hoff.size());
    }
    if (int(pp.passes.size()) > max_passes || int(pp.gates.size()) > max_gates ||
        int(pp.hoff.size()) > max_hoff)
        return -1;
    if (passes) std::memcpy(passes, pp.passes.data(), pp.passes.size() * sizeof(ExcPass));
    if (gates) std::memcpy(gates, pp.gates.data(), pp.gates.size() * sizeof(ExcGate));
    if (hoff) std::memcpy(hoff, pp.hoff.data(), pp.hoff.size() * sizeof(uint32_t));
    return 0;
}

int vqe_inspect_hamiltonian(int n_qubits, const uint64_t *x_masks, const uint64_t *z_masks,
                            const double *coeffs, size_t n_terms, double threshold, void *groups,
                            int max_groups, uint32_t *tz, double *tc, int max_terms, int counts[2],
                            double *sum_abs_dropped, uint64_t *n_canonical) {
    if (n_qubits < 1 || n_qubits > 32) return -1;
    if (n_terms && (!x_masks || !z_masks || !coeffs)) return -1;
    if (!(threshold >= 0.0) || !std::isfinite(threshold)) return -1;
    const uint64_t lim = (uint64_t(1) << n_qubits) - 1;
    for (size_t t = 0; t < n_terms; ++t)
        if ((x_masks[t] & ~lim) || (z_masks[t] & ~lim) || !std::isfinite(coeffs[t])) return -1;
    std::vector<uint64_t> cx, cz;
    std::vector<double> cc;
    canonicalise(x_masks, z_masks, coeffs, n_terms, cx, cz, cc);
    std::vector<uint8_t> keep;
    size_t kept = 0;
    const double dropped = slim_keep(cc, threshold, keep, kept);
    HamPlan hp;
    make_ham_plan(cx, cz, cc, keep, hp);
    if (counts) {
        counts[0] = int(hp.groups.size());
        counts[1] = int(hp.tz.size());
    }
    if (sum_abs_dropped) *sum_abs_dropped = dropped;
    if (n_canonical) *n_canonical = cc.size();
    if (int(hp.groups.size()) > max_groups || int(hp.tz.size()) > max_terms) return -1;
    if (groups) std::memcpy(groups, hp.groups.data(), hp.groups.size() * sizeof(GroupDesc));
    if (tz) std::memcpy(tz, hp.tz.data(), hp.tz.size() * sizeof(uint32_t));
    if (tc) std::memcpy(tc, hp.tc.data(), hp.tc.size() * sizeof(double));
    return 0;
}

int vqe_inspect_sweeps(int n_qubits, int precision, const uint64_t *x_masks,
                       const uint64_t *z_masks, const double *coeffs, size_t n_terms,
                       double threshold, int diag_terms, void *sweeps, int max_sweeps,
                       void *groups, int max_groups, uint32_t *pat, int max_pat, uint32_t *tz,
                       double *ta, double *tb, int max_terms, uint32_t *order, int max_order,
                       int counts[4]) {
    if (n_qubits < 1 || n_qubits > 32 || (precision != 0 && precision != 1)) return -1;
    if (n_terms && (!x_masks || !z_masks || !coeffs)) return -1;
    const uint64_t lim = (uint64_t(1) << n_qubits) - 1;
    for (size_t t = 0; t < n_terms; ++t)
        if ((x_masks[t] & ~lim) || (z_masks[t] & ~lim) || !std::isfinite(coeffs[t])) return -1;
    std::vector<uint64_t> cx, cz;
    std::vector<double> cc;
    canonicalise(x_masks, z_masks, coeffs, n_terms, cx, cz, cc);
    std::vector<uint8_t> keep;
    size_t kept = 0;
    slim_keep(cc, threshold, keep, kept);
    HamPlan hp;
    make_ham_plan(cx, cz, cc, keep, hp);
    SweepPlan sp;
    plan_sweeps(n_qubits, vqe_precision(precision), hp, diag_terms != 0, sp);
    if (counts) {
        counts[0] = int(sp.sweeps.size());
        counts[1] = int(sp.groups.size());
        counts[2] = int(sp.pat.size());
        counts[3] = int(sp.tz.size());
    }
    if (!sp.ok) return -1;
    if (int(sp.sweeps.size()) > max_sweeps || int(sp.groups.size()) > max_groups ||
        int(sp.pat.size()) > max_pat || int(sp.tz.size()) > max_terms ||
        int(sp.order.size()) > max_order)
        return -1;
    if (sweeps) std::memcpy(sweeps, sp.sweeps.data(), sp.sweeps.size() * sizeof(SweepDesc));
    if (groups) std::memcpy(groups, sp.groups.data(), sp.groups.size() * sizeof(SGroup));
    if (pat) std::memcpy(pat, sp.pat.data(), sp.pat.size() * sizeof(uint32_t));
    if (tz) std::memcpy(tz, sp.tz.data(), sp.tz.size() * sizeof(uint32_t));
    if (ta) std::memcpy(ta, sp.ta.data(), sp.ta.size() * sizeof(double));
    if (tb) std::memcpy(tb, sp.tb.data(), sp.tb.size() * sizeof(double));
    if (order) std::memcpy(order, sp.order.data(), sp.order.size() * sizeof(uint32_t));
    return 0;
}

int vqe_inspect_windows(int n_qubits, int precision, const uint64_t *x_masks,
                        const uint64_t *z_masks, const double *coeffs, size_t n_terms,
                        double threshold, int diag_terms, void *windows,
                        int max_windows,
                        void *wgroups, int max_wgroups, void *wterms, int max_wterms,
                        uint32_t *hoff, int max_hoff, void *wide, int max_wide, int counts[5]) {
    if (n_qubits < 1 || n_qubits > 32 || (precision != 0 && precision != 1)) return -1;
    if (n_terms && (!x_masks || !z_masks || !coeffs)) return -1;
    const uint64_t lim = (uint64_t(1) << n_qubits) - 1;
    for (size_t t = 0; t < n_terms; ++t)
        if ((x_masks[t] & ~lim) || (z_masks[t] & ~lim) || !std::isfinite(coeffs[t])) return -1;
    std::vector<uint64_t> cx, cz;
    std::vector<double> cc;
    canonicalise(x_masks, z_masks, coeffs, n_terms, cx, cz, cc);
    std::vector<uint8_t> keep;
    size_t kept = 0;
    slim_keep(cc, threshold, keep, kept);
    HamPlan hp;
    make_ham_plan(cx, cz, cc, keep, hp);
    WinPlan wp;
    plan_windows(n_qubits, vqe_precision(precision), hp, diag_terms != 0, wp);
    if (counts) {
        counts[0] = int(wp.wins.size());
        counts[1] = int(wp.groups.size());
        counts[2] = int(wp.terms.size());
        counts[3] = int(wp.hoff.size());
        counts[4] = int(wp.wide.size());
    }
    if (int(wp.wins.size()) > max_windows || int(wp.groups.size()) > max_wgroups ||
        int(wp.terms.size()) > max_wterms || int(wp.hoff.size()) > max_hoff ||
        int(wp.wide.size()) > max_wide)
        return -1;
    if (windows) std::memcpy(windows, wp.wins.data(), wp.wins.size() * sizeof(WinDesc));
    if (wgroups) std::memcpy(wgroups, wp.groups.data(), wp.groups.size() * sizeof(WinGroup));
    if (wterms) std::memcpy(wterms, wp.terms.data(), wp.terms.size() * sizeof(WinTerm));
    if (hoff) std::memcpy(hoff, wp.hoff.data(), wp.hoff.size() * sizeof(uint32_t));
    if (wide) std::memcpy(wide, wp.wide.data(), wp.wide.size() * sizeof(GroupDesc));
    return 0;
}

}  // extern "C"

// ================================================================= batched driver

#include "batch_internal.h"

struct vqe_batch_ctx {
    int count = 0;
    vqe_precision prec = VQE_C64;
    cudaStream_t stream = nullptr;     // caller's stream (or an internal one)
    bool own_stream = false;
    int device = 0;
    int tile_bits = 0;                 // plan tile size for instances larger than one tile
    std::string err;
    std::vector<int> n, depth;
    std::vector<size_t> poff;          // parameter offsets (count + 1)
    std::vector<std::vector<uint64_t>> hx, hz;
    std::vector<std::vector<double>> hc;
    std::vector<uint8_t> ham_ok;
    bool ham_dirty = true, plan_dirty = true;
    // device
    DevBuf d_inst, d_order, d_counter, d_plans, d_fwd, d_bwd, d_stage, d_groups, d_tz, d_tc,
        d_scratch;
    DevBuf hb_p, hb_e, hb_g;   // device copies for vqe_batch_run (host buffers)
    BatchLayout layout{};
    int grid = 0;
    int count_r4 = 0;                  // instances of the R = 4 kernel (first in d_order)
    size_t scratch_elems = 0;
    std::vector<BatchInst> inst;
    // captured graph for the last pointer triple
    cudaGraphExec_t gexec = nullptr;
    const void *g_params = nullptr, *g_e = nullptr, *g_g = nullptr;
    uint64_t launches = 0;
};

namespace {

vqe_status bfail(vqe_batch_ctx *b, vqe_status st, const std::string &msg) {
    if (b) b->err = msg;
    return st;
}

#define VQE_BCUDA(b, call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return bfail((b), VQE_ERR_CUDA, std::string(#call) + ": " +       \
                                                                  cudaGetErrorString(e_));      \
    } while (0)

vqe_status bensure(vqe_batch_ctx *b, DevBuf &buf, size_t bytes, const char *what) {
    if (buf.bytes >= bytes && buf.p) return VQE_OK;
    buf.release();
    if (bytes == 0) return VQE_OK;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        buf.p = nullptr;
        return bfail(b, VQE_ERR_OOM, std::string("cudaMalloc failed for ") + what);
    }
    buf.bytes = bytes;
    return VQE_OK;
}

template <typename V>
vqe_status bupload(vqe_batch_ctx *b, DevBuf &buf, const std::vector<V> &v, const char *what) {
    vqe_status st = bensure(b, buf, std::max<size_t>(v.size() * sizeof(V), 16), what);
    if (st != VQE_OK) return st;
    if (!v.empty())
        VQE_BCUDA(b, cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice,
                                     b->stream));
    VQE_BCUDA(b, cudaStreamSynchronize(b->stream));
    return VQE_OK;
}

// Options that give every pass of an n-qubit instance exactly kBatchThreads
// threads: one tile for n <= tile bits, else a low group and one high group
// of equal tile size.
bool batch_options(int n, vqe_precision prec, int tile_bits, PlanOptions &o) {
    const int kmax = tile_bits;
    const int lg = 9;   // log2(kBatchThreads)
    if (n <= kmax) {
        o.tile_bits_max = std::max(n, 2);
        o.reg_bits = std::min(4, std::max(1, n - lg));
        o.run_bits = 1;
    } else {
        const int run = 2 * kmax - n;
        if (run < 1) return false;
        o.tile_bits_max = kmax;
        o.run_bits = run;
        o.reg_bits = kmax - lg;
    }
    (void)prec;
    return true;
}

vqe_status batch_build(vqe_batch_ctx *b) {
    const bool c128 = b->prec == VQE_C128;
    const size_t elem = c128 ? 16 : 8;
    const size_t coef_sz = c128 ? sizeof(RotCoef<double>) : sizeof(RotCoef<float>);
    std::vector<BatchPlan> plans;
    std::vector<PassDesc> fwd, bwd;
    std::vector<StageSlot> stage;
    std::vector<std::pair<int, int>> keys;   // (n, depth) -> plan index
    std::vector<char> plan_r4;               // plan runs in the R = 4 kernel
    b->inst.assign(b->count, BatchInst{});
    size_t max_tile = 0, max_coef = 0, max_lo = 0, max_hi = 0, max_np = 0, max_stage = 0;
    int max_multi_n = 0;
    for (int i = 0; i < b->count; ++i) {
        const std::pair<int, int> key{b->n[i], b->depth[i]};
        int pi = -1;
        for (size_t j = 0; j < keys.size(); ++j)
            if (keys[j] == key) pi = int(j);
        if (pi < 0) {
            PlanOptions o;
            if (!batch_options(key.first, b->prec, b->tile_bits, o))
                return bfail(b, VQE_ERR_ARG, "instance too large for the batched driver");
            HostPlan hp;
            std::string err;
            if (!make_plan(key.first, key.second, b->prec, o, hp, err))
                return bfail(b, VQE_ERR_ARG, "batch plan: " + err);
            if (int(hp.fwd.size()) > kBatchMaxPasses || int(hp.stage.size()) > kBatchMaxSlots)
                return bfail(b, VQE_ERR_ARG, "instance plan too deep for the batched driver");
            BatchPlan P{};
            P.n = key.first;
            P.depth = key.second;
            P.pass_off = int(fwd.size());
            P.n_passes = int(hp.fwd.size());
            P.stage_off = int(stage.size());
            P.n_stage = int(hp.stage.size());
            int slot = 0;
            int kk = 0;
            P.whole_tile = 1;
            for (int p = 1; p < P.n_passes; ++p)
                if (hp.fwd[p].R != hp.fwd[0].R)
                    return bfail(b, VQE_ERR_ARG, "batch plan: register bits differ between passes");
            plan_r4.push_back(hp.fwd[0].R == 4 ? 1 : 0);
            for (int p = 0; p < P.n_passes; ++p) {
                P.slot_first[p] = slot;
                slot += hp.fwd[p].n_slots;
                kk = std::max(kk, hp.fwd[p].k);
                if (hp.fwd[p].k != key.first) P.whole_tile = 0;
            }
            P.coef_entries = int(hp.coef_stride);
            P.kl = (kk + 1) / 2;
            P.lo_stride = 1 << P.kl;
            P.hi_stride = 1 << (kk - P.kl);
            fwd.insert(fwd.end(), hp.fwd.begin(), hp.fwd.end());
            bwd.insert(bwd.end(), hp.bwd.begin(), hp.bwd.end());
            stage.insert(stage.end(), hp.stage.begin(), hp.stage.end());
            max_tile = std::max(max_tile, size_t(tile_buf_elems(kk, int(elem))));   // padded
            max_coef = std::max(max_coef, hp.coef_stride);
            max_lo = std::max(max_lo, size_t(P.n_stage) * P.lo_stride);
            max_hi = std::max(max_hi, size_t(P.n_stage) * P.hi_stride);
            max_stage = std::max(max_stage, size_t(P.n_stage));
            if (!P.whole_tile) max_multi_n = std::max(max_multi_n, key.first);
            pi = int(plans.size());
            plans.push_back(P);
            keys.push_back(key);
        }
        BatchInst &I = b->inst[i];
        I.index = i;
        I.n = b->n[i];
        I.depth = b->depth[i];
        I.plan = pi;
        I.params_off = b->poff[i];
        max_np = std::max(max_np, size_t(2 * b->n[i] * b->depth[i]));
    }
    // shared-memory layout (16-byte aligned pieces)
    auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
    BatchLayout L{};
    size_t o = 0;
    L.off_psi = o; o = al(o + max_tile * elem);
    L.off_lam = o; o = al(o + max_tile * elem);
    L.off_gsh = o; o = al(o + size_t((kBatchThreads + 31) / 32) * kMaxTileBits * 2 * sizeof(double));
    L.off_coef = o; o = al(o + max_coef * coef_sz);
    L.off_lo = o; o = al(o + max_lo * elem);
    L.off_hi = o; o = al(o + max_hi * elem);
    L.off_gacc = o; o = al(o + max_np * sizeof(double));
    L.off_red = o; o = al(o + 2 * (kBatchThreads / 32) * sizeof(double));
    L.off_slotbase = o; o = al(o + kMaxSlots * sizeof(int));
    L.off_phc = o; o = al(o + max_stage * kMaxTileBits * sizeof(double));
    L.off_phs = o; o = al(o + max_stage * kMaxTileBits * sizeof(double));
    L.off_scl = o; o = al(o + max_stage * kMaxTileBits * sizeof(double));
    L.off_sigma = o; o = al(o + max_stage * sizeof(double));
    L.total = o;
    if (L.total > 227 * 1024) return bfail(b, VQE_ERR_ARG, "batched instance needs more than 227 KiB of shared memory");
    b->layout = L;
    vqe_status st;
    if ((st = bupload(b, b->d_plans, plans, "batch plans")) != VQE_OK) return st;
    if ((st = bupload(b, b->d_fwd, fwd, "batch passes")) != VQE_OK) return st;
    if ((st = bupload(b, b->d_bwd, bwd, "batch passes")) != VQE_OK) return st;
    if ((st = bupload(b, b->d_stage, stage, "batch stage")) != VQE_OK) return st;
    // the R = 4 kernel's instances, then the others; largest first in each
    std::vector<int> order(b->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
        const int rp = plan_r4[b->inst[p].plan], rq = plan_r4[b->inst[q].plan];
        if (rp != rq) return rp > rq;
        const double cp = double(size_t(1) << b->n[p]) * b->depth[p];
        const double cq = double(size_t(1) << b->n[q]) * b->depth[q];
        return cp > cq;
    });
    b->count_r4 = 0;
    for (int i = 0; i < b->count; ++i) b->count_r4 += plan_r4[b->inst[i].plan];
    if ((st = bupload(b, b->d_order, order, "batch order")) != VQE_OK) return st;
    int sms = 0;
    VQE_BCUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, std::min(sms, b->count));
    b->scratch_elems = max_multi_n ? (size_t(1) << max_multi_n) : 0;
    if ((st = bensure(b, b->d_scratch, std::max<size_t>(16, size_t(b->grid) * 2 * b->scratch_elems * elem),
                      "batch scratch")) != VQE_OK)
        return st;
    if ((st = bensure(b, b->d_counter, 16, "batch counter")) != VQE_OK) return st;
    b->plan_dirty = false;
    b->ham_dirty = true;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return VQE_OK;
}

vqe_status batch_upload_hams(vqe_batch_ctx *b) {
    std::vector<GroupDesc> groups;
    std::vector<uint32_t> tz;
    std::vector<double> tc;
    for (int i = 0; i < b->count; ++i) {
        if (!b->ham_ok[i]) return bfail(b, VQE_ERR_STATE, "instance " + std::to_string(i) + " has no Hamiltonian");
        std::vector<uint64_t> cx, cz;
        std::vector<double> cc;
        canonicalise(b->hx[i].data(), b->hz[i].data(), b->hc[i].data(), b->hc[i].size(), cx, cz, cc);
        std::vector<uint8_t> keep(cc.size(), 1);
        HamPlan hp;
        make_ham_plan(cx, cz, cc, keep, hp);
        BatchInst &I = b->inst[i];
        I.groups_off = int(groups.size());
        I.n_groups = int(hp.groups.size());
        I.terms_off = int(tz.size());
        for (auto g : hp.groups) {
            groups.push_back(g);
        }
        tz.insert(tz.end(), hp.tz.begin(), hp.tz.end());
        tc.insert(tc.end(), hp.tc.begin(), hp.tc.end());
    }
    vqe_status st;
    if ((st = bupload(b, b->d_inst, b->inst, "batch instances")) != VQE_OK) return st;
    if ((st = bupload(b, b->d_groups, groups, "batch groups")) != VQE_OK) return st;
    if ((st = bupload(b, b->d_tz, tz, "batch terms")) != VQE_OK) return st;
    if (b->prec == VQE_C128) {
        if ((st = bupload(b, b->d_tc, tc, "batch terms")) != VQE_OK) return st;
    } else {
        std::vector<float> tf(tc.begin(), tc.end());
        if ((st = bupload(b, b->d_tc, tf, "batch terms")) != VQE_OK) return st;
    }
    b->ham_dirty = false;
    return VQE_OK;
}

vqe_status batch_launch(vqe_batch_ctx *b, const double *params, double *energies, double *grads,
                        cudaStream_t s) {
    VQE_BCUDA(b, cudaMemsetAsync(b->d_counter.p, 0, 2 * sizeof(int), s));
    BatchArgs a{};
    a.inst = static_cast<const BatchInst *>(b->d_inst.p);
    a.order = static_cast<const int *>(b->d_order.p);
    a.count = b->count;
    a.counter = static_cast<int *>(b->d_counter.p);
    a.plans = static_cast<const BatchPlan *>(b->d_plans.p);
    a.fwd = static_cast<const PassDesc *>(b->d_fwd.p);
    a.bwd = static_cast<const PassDesc *>(b->d_bwd.p);
    a.stage = static_cast<const StageSlot *>(b->d_stage.p);
    a.groups = static_cast<const GroupDesc *>(b->d_groups.p);
    a.tz = static_cast<const uint32_t *>(b->d_tz.p);
    a.tc = b->d_tc.p;
    a.params = params;
    a.energies = energies;
    a.grads = grads;
    a.scratch = b->d_scratch.p;
    a.scratch_elems = b->scratch_elems;
    a.layout = b->layout;
    // two persistent launches: the R = 4 instances, then the rest
    for (int half = 0; half < 2; ++half) {
        const int first = half ? b->count_r4 : 0;
        const int cnt = half ? b->count - b->count_r4 : b->count_r4;
        if (cnt == 0) continue;
        BatchArgs h = a;
        h.order = a.order + first;
        h.count = cnt;
        h.counter = a.counter + half;
        const int grid = std::max(1, std::min(b->grid, cnt));
        cudaError_t e = b->prec == VQE_C128 ? launch_batch<double>(h, half == 0, grid, b->layout.total, s)
                                            : launch_batch<float>(h, half == 0, grid, b->layout.total, s);
        if (e != cudaSuccess) return bfail(b, VQE_ERR_CUDA, std::string("k_batch: ") + cudaGetErrorString(e));
    }
    return VQE_OK;
}

}  // namespace

extern "C" {

vqe_status vqe_batch_create(int count, const int *n_qubits, const int *depths,
                            vqe_precision precision, void *cuda_stream, vqe_batch *out) {
    if (!out) return VQE_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > (1 << 24) || !n_qubits || !depths) return VQE_ERR_ARG;
    if (precision != VQE_C64 && precision != VQE_C128) return VQE_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (n_qubits[i] < 1 || n_qubits[i] > 24 || depths[i] < 1 || depths[i] > 64) return VQE_ERR_ARG;
    vqe_batch_ctx *b = new vqe_batch_ctx();
    b->count = count;
    b->prec = precision;
    b->tile_bits = precision == VQE_C128 ? 12 : 13;
    b->n.assign(n_qubits, n_qubits + count);
    b->depth.assign(depths, depths + count);
    b->poff.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) b->poff[i + 1] = b->poff[i] + size_t(2 * b->n[i] * b->depth[i]);
    b->hx.resize(count);
    b->hz.resize(count);
    b->hc.resize(count);
    b->ham_ok.assign(count, 0);
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return VQE_ERR_CUDA;
    }
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return VQE_ERR_CUDA;
        }
        b->own_stream = true;
    }
    vqe_status st = batch_build(b);
    if (st != VQE_OK) {
        vqe_batch_destroy(b);
        return st;
    }
    *out = b;
    return VQE_OK;
}

vqe_status vqe_batch_destroy(vqe_batch b) {
    if (!b) return VQE_ERR_ARG;
    cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (DevBuf *d : {&b->d_inst, &b->d_order, &b->d_counter, &b->d_plans, &b->d_fwd, &b->d_bwd,
                      &b->d_stage, &b->d_groups, &b->d_tz, &b->d_tc, &b->d_scratch, &b->hb_p,
                      &b->hb_e, &b->hb_g})
        d->release();
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return VQE_OK;
}

const char *vqe_batch_last_error(vqe_batch b) { return b ? b->err.c_str() : "NULL batch"; }

vqe_status vqe_batch_param_offsets(vqe_batch b, size_t *offsets) {
    if (!b || !offsets) return VQE_ERR_ARG;
    std::memcpy(offsets, b->poff.data(), sizeof(size_t) * (b->count + 1));
    return VQE_OK;
}

vqe_status vqe_batch_set_hamiltonian(vqe_batch b, int instance, const uint64_t *x_masks,
                                     const uint64_t *z_masks, const double *coeffs,
                                     size_t n_terms) {
    if (!b) return VQE_ERR_ARG;
    if (instance < 0 || instance >= b->count) return bfail(b, VQE_ERR_ARG, "instance out of range");
    if (n_terms && (!x_masks || !z_masks || !coeffs)) return bfail(b, VQE_ERR_ARG, "NULL term array");
    const uint64_t lim = (uint64_t(1) << b->n[instance]) - 1;
    for (size_t t = 0; t < n_terms; ++t) {
        if ((x_masks[t] & ~lim) || (z_masks[t] & ~lim))
            return bfail(b, VQE_ERR_ARG, "Pauli mask has a bit at or above the instance's qubits");
        if (!std::isfinite(coeffs[t])) return bfail(b, VQE_ERR_ARG, "non-finite coefficient");
    }
    b->hx[instance].assign(x_masks, x_masks + n_terms);
    b->hz[instance].assign(z_masks, z_masks + n_terms);
    b->hc[instance].assign(coeffs, coeffs + n_terms);
    b->ham_ok[instance] = 1;
    b->ham_dirty = true;
    return VQE_OK;
}

vqe_status vqe_batch_run_dev(vqe_batch b, const double *params_dev, double *energies_dev,
                             double *grads_dev) {
    if (!b) return VQE_ERR_ARG;
    if (!params_dev || !energies_dev || !grads_dev) return bfail(b, VQE_ERR_ARG, "NULL buffer");
    vqe_status st;
    if (b->plan_dirty && (st = batch_build(b)) != VQE_OK) return st;
    if (b->ham_dirty) {
        if ((st = batch_upload_hams(b)) != VQE_OK) return st;
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
    }
    if (!b->gexec || b->g_params != params_dev || b->g_e != energies_dev || b->g_g != grads_dev) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        VQE_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        st = batch_launch(b, params_dev, energies_dev, grads_dev, b->stream);
        cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
        if (st != VQE_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ec != cudaSuccess) return bfail(b, VQE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) {
            b->gexec = nullptr;
            return bfail(b, VQE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
        }
        b->g_params = params_dev;
        b->g_e = energies_dev;
        b->g_g = grads_dev;
    }
    VQE_BCUDA(b, cudaGraphLaunch(b->gexec, b->stream));
    b->launches += 1;
    if (b->own_stream) VQE_BCUDA(b, cudaStreamSynchronize(b->stream));
    return VQE_OK;
}

vqe_status vqe_batch_run(vqe_batch b, const double *params, double *energies, double *grads) {
    if (!b) return VQE_ERR_ARG;
    if (!params || !energies || !grads) return bfail(b, VQE_ERR_ARG, "NULL buffer");
    const size_t P = b->poff[b->count];
    for (size_t i = 0; i < P; ++i)
        if (!std::isfinite(params[i])) return bfail(b, VQE_ERR_ARG, "non-finite parameter");
    DevBuf &dp = b->hb_p, &de = b->hb_e, &dg = b->hb_g;
    vqe_status st = bensure(b, dp, P * sizeof(double), "params");
    if (st == VQE_OK) st = bensure(b, de, b->count * sizeof(double), "energies");
    if (st == VQE_OK) st = bensure(b, dg, P * sizeof(double), "grads");
    if (st == VQE_OK && cudaMemcpyAsync(dp.p, params, P * sizeof(double), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        st = bfail(b, VQE_ERR_CUDA, "params upload failed");
    if (st == VQE_OK) st = vqe_batch_run_dev(b, static_cast<double *>(dp.p), static_cast<double *>(de.p), static_cast<double *>(dg.p));
    if (st == VQE_OK && cudaMemcpyAsync(energies, de.p, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        st = bfail(b, VQE_ERR_CUDA, "energies download failed");
    if (st == VQE_OK && cudaMemcpyAsync(grads, dg.p, P * sizeof(double), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        st = bfail(b, VQE_ERR_CUDA, "grads download failed");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && st == VQE_OK)
        st = bfail(b, VQE_ERR_CUDA, "stream synchronise failed");
    return st;
}

vqe_status vqe_batch_autotune(vqe_batch b, const double *params_dev, double *energies_dev,
                              double *grads_dev, int reps, int *tile_bits_out) {
    if (!b) return VQE_ERR_ARG;
    if (reps < 1) reps = 1;
    std::vector<int> cands = b->prec == VQE_C128 ? std::vector<int>{12, 11, 10}
                                                 : std::vector<int>{13, 12, 11};
    float best = 0.f;
    int best_k = b->tile_bits;
    cudaEvent_t e0, e1;
    VQE_BCUDA(b, cudaEventCreate(&e0));
    VQE_BCUDA(b, cudaEventCreate(&e1));
    for (int kb : cands) {
        b->tile_bits = kb;
        b->plan_dirty = true;
        vqe_status st = vqe_batch_run_dev(b, params_dev, energies_dev, grads_dev);   // builds + warms up
        if (st != VQE_OK) continue;
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && st == VQE_OK; ++r) st = vqe_batch_run_dev(b, params_dev, energies_dev, grads_dev);
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == VQE_OK && (best == 0.f || ms < best)) {
            best = ms;
            best_k = kb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile_bits = best_k;
    b->plan_dirty = true;
    vqe_status st = vqe_batch_run_dev(b, params_dev, energies_dev, grads_dev);
    if (tile_bits_out) *tile_bits_out = best_k;
    return st;
}

vqe_status vqe_batch_set_tile_bits(vqe_batch b, int tile_bits) {
    if (!b) return VQE_ERR_ARG;
    const int kmax = b->prec == VQE_C128 ? 12 : 13;
    if (tile_bits < 10 || tile_bits > kmax) return bfail(b, VQE_ERR_ARG, "tile_bits out of range");
    b->tile_bits = tile_bits;
    b->plan_dirty = true;
    return VQE_OK;
}

vqe_status vqe_batch_launch_count(vqe_batch b, uint64_t *graph_launches) {
    if (!b || !graph_launches) return VQE_ERR_ARG;
    *graph_launches = b->launches;
    return VQE_OK;
}

}  // extern "C"
