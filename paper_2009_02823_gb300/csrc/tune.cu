// Schedule autotuner of the fused sweeps (vqg_autotune).  The paper applies one gate at
// a time; this chooses how the tile-fused passes are cut: tile qubits K and the number
// of qubits held in registers per forward (Rf) and reverse (Rr) stage.  Whole
// energy-and-gradient evaluations of the circuit itself are timed per kernel family
// (CUDA events on the circuit's stream), so the choice reflects its gates, its
// Hamiltonian and the device it runs on.  Host code only: every candidate runs through
// the same planner and kernels as a normal call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/vqg.h"
#include "engine.h"
#include "plan.h"

namespace vqg {
namespace {

struct TuneKey {
    int n, dbl, G, P;
    uint64_t gates_hash, ham_hash;
    bool operator<(const TuneKey &o) const {
        return std::tie(n, dbl, G, P, gates_hash, ham_hash) < std::tie(o.n, o.dbl, o.G, o.P, o.gates_hash, o.ham_hash);
    }
};

// FNV-1a over the bytes of the structure (64-bit).
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

std::mutex g_mu;
std::map<TuneKey, vqg_tune_result> g_table;

TuneKey key_of(const Circuit &c) {
    Fnv fg, fh;
    for (const vqg_gate &g : c.gates) {
        const int32_t v[3] = {g.kind, g.q0, g.q1};
        fg.add(v, sizeof v);
    }
    for (const HamGroup &g : c.ham) {
        fh.add(&g.x, sizeof g.x);
        fh.add(&g.count, sizeof g.count);
    }
    for (const PauliTerm &t : c.host_terms) fh.add(&t.z, sizeof t.z);
    return {c.n, c.dbl ? (float_float(c.dbl, c.opt) ? 2 : 1) : 0, c.G, c.P, fg.h, fh.h};
}

struct FamTimes {
    double fwd = 0, ham = 0, rev = 0;
    double total() const { return fwd + ham + rev; }
};

}  // namespace

// Re-plan the fused sweeps for (K, Rf, Rr).  The circuit's checkpoints are re-placed
// at the new pass boundaries (buffers reused) and cached graphs dropped.
static int apply_schedule(Circuit &c, int K, int Rf, int Rr) {
    c.drop_plan();
    c.opt.tile_qubits = K;
    c.opt.fwd_reg_qubits = Rf;
    c.opt.rev_reg_qubits = Rr;
    c.invalidate_graphs();
    c.graph_warm = false;
    int st = c.build_plan();
    if (st) return st;
    if (!c.plan_ok) return set_error(VQG_ERR_UNSUPPORTED, "schedule K=%d Rf=%d Rr=%d has no fused plan", K, Rf, Rr);
    if ((st = c.rebuild_alt_plan())) return st;  // the stored anti-Hermitian part, if any
    return c.plan_checkpoints();
}

// One timed evaluation: per-family device time of the fused forward, Hamiltonian and
// reverse passes.  The caller's profiling counters are kept.
static int time_once(Circuit &c, const double *theta_dev, FamTimes &t) {
    c.prof_harvest();
    long saved_l[FAM_COUNT];
    double saved_ms[FAM_COUNT];
    std::memcpy(saved_l, c.fam_launches, sizeof saved_l);
    std::memcpy(saved_ms, c.fam_ms, sizeof saved_ms);
    const bool was = c.profiling;
    c.profiling = true;
    for (int f = 0; f < FAM_COUNT; ++f) c.fam_launches[f] = 0, c.fam_ms[f] = 0.0;
    int st = c.issue_gradient(theta_dev, c.d_out, c.d_out + 1);
    c.prof_harvest();
    t.fwd = c.fam_ms[FAM_FWD_FUSED];
    t.ham = c.fam_ms[FAM_HAM_FUSED] + c.fam_ms[FAM_HAM_DIAG] + c.fam_ms[FAM_HAM_GROUP];
    t.rev = c.fam_ms[FAM_ADJ_FUSED];
    c.profiling = was;
    std::memcpy(c.fam_launches, saved_l, sizeof saved_l);
    std::memcpy(c.fam_ms, saved_ms, sizeof saved_ms);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "autotune run: %s", cudaGetErrorString(e));
    return VQG_OK;
}

int Circuit::autotune(const double *theta_dev, vqg_tune_result *out) {
    vqg_tune_result r;
    std::memset(&r, 0, sizeof r);
    tuned = true;
    if (!has_ham) return set_error(VQG_ERR_STATE, "no Hamiltonian set");
    if (tile_explicit || !opt.fusion || !plan_ok) {  // nothing to choose
        if (out) *out = r;
        return VQG_OK;
    }
    const TuneKey key = key_of(*this);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_table.find(key);
        if (it != g_table.end()) {
            r = it->second;
            r.candidates = 0;
        }
    }
    int st;
    if (r.tile_qubits) {  // stored choice
        if (plan->K != r.tile_qubits || plan->Rf != r.fwd_reg_qubits || plan->Rr != r.rev_reg_qubits)
            if ((st = apply_schedule(*this, r.tile_qubits, r.fwd_reg_qubits, r.rev_reg_qubits))) return st;
        if (out) *out = r;
        return VQG_OK;
    }
    const int Kmax = std::min(n, dbl ? 12 : 13);
    const bool ff = float_float(dbl, opt);
    // (forward, reverse) register qubits; float-float has one compiled geometry
    const std::vector<std::pair<int, int>> reg_pairs =
        ff ? std::vector<std::pair<int, int>>{{3, 3}}
           : std::vector<std::pair<int, int>>{{dbl ? 4 : 5, dbl ? 3 : 4}, {dbl ? 3 : 4, dbl ? 2 : 3}};
    const int K0 = plan->K, Rf0 = plan->Rf, Rr0 = plan->Rr;
    double best = 1e300;
    int bK = K0, bRf = Rf0, bRr = Rr0;
    bool warm = false;
    const int Kmin = std::max(10, std::min(K0, Kmax - 2));  // the default is always a candidate
    for (int K = Kmax; K >= Kmin; --K) {
        double best_f = 1e300, best_r = 1e300, ham_t = 0, best_pair = 1e300;
        int kRf = 0, kRr = 0, pRf = 0, pRr = 0;
        for (const auto &rp : reg_pairs) {
            const int Rf = rp.first, Rr = rp.second;
            if (!fused_supported(dbl, K, Rf, Rr, ff)) continue;
            if ((st = apply_schedule(*this, K, Rf, Rr))) return st;
            FamTimes t;
            if (!warm) {  // first launch of the kernels: module load and attributes
                if ((st = time_once(*this, theta_dev, t))) return st;
                warm = true;
            }
            if ((st = time_once(*this, theta_dev, t))) return st;
            ++r.candidates;
            if (K == K0 && Rf == Rf0 && Rr == Rr0) r.default_ms = t.total();
            if (t.fwd < best_f) best_f = t.fwd, kRf = Rf;
            if (t.rev < best_r) best_r = t.rev, kRr = Rr;
            ham_t = t.ham;
            if (t.total() < best_pair) best_pair = t.total(), pRf = Rf, pRr = Rr;
        }
        if (!kRf) continue;
        double est = best_f + ham_t + best_r;
        if (!fused_supported(dbl, K, kRf, kRr, ff)) est = best_pair, kRf = pRf, kRr = pRr;  // mix not compiled
        if (est < best) best = est, bK = K, bRf = kRf, bRr = kRr;
    }
    if (plan->K != bK || plan->Rf != bRf || plan->Rr != bRr)
        if ((st = apply_schedule(*this, bK, bRf, bRr))) return st;
    r.tile_qubits = bK;
    r.fwd_reg_qubits = bRf;
    r.rev_reg_qubits = bRr;
    r.best_ms = best;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_table[key] = r;
    }
    if (out) *out = r;
    return VQG_OK;
}

}  // namespace vqg

using namespace vqg;

extern "C" int vqg_autotune(vqg_circuit *c, const double *theta, vqg_tune_result *out) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    if (cc->P) {
        if (theta) std::memcpy(cc->h_pinned, theta, sizeof(double) * cc->P);
        else std::memset(cc->h_pinned, 0, sizeof(double) * cc->P);
        cudaError_t e = cudaMemcpyAsync(cc->d_theta, cc->h_pinned, sizeof(double) * cc->P, cudaMemcpyHostToDevice,
                                        cc->stream);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "theta upload: %s", cudaGetErrorString(e));
    }
    return cc->autotune(cc->d_theta, out);
}

extern "C" void vqg_tune_table_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
}
