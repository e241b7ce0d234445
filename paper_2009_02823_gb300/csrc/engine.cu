// Execution planner: turns the gate list into tile passes and register stages, and
// the Pauli groups into Hamiltonian tile passes; issues the fused launch sequence.
//
// Scheduling rule (shared by passes and stages).  Gates are taken in circuit order;
// a gate is applied in the current pass/stage if every qubit it acts on
// non-diagonally lies in the chosen set S and no earlier gate left for later blocks
// it: an earlier deferred gate blocks a later one on a shared qubit unless both act
// diagonally there (RZ, CZ, and the control of CNOT are diagonal in the
// computational basis, so they commute).  The result is a reordering of the circuit
// that only swaps commuting gates, so U(theta) -- and with it E(theta) and every
// gradient entry -- is unchanged.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <map>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "fused.h"
#include "plan.h"

namespace vqg {

#define VQG_FWD_ARGS                                                                             \
    int K, int R, const void *src, void *dst, const FPass *passes, int pi, const FStage *st,      \
        const FOp *ops, const FDiag *dg, const FDItem *it, const void *mats, uint64_t n_tiles,    \
        int grid, cudaStream_t s
#define VQG_REV_ARGS                                                                             \
    int K, int R, const void *phi_src, void *phi_dst, void *lam, const FPass *passes, int pi,     \
        const FStage *st, const FOp *ops, const FDiag *dg, const FDItem *it, const int *slot_map, \
        const void *mats, uint64_t n_tiles, double *partials, int nb, int wmask, cudaStream_t s
bool launch_fused_fwd_c64(VQG_FWD_ARGS);
bool launch_fused_fwd_c128(VQG_FWD_ARGS);
bool launch_fused_rev_c64(VQG_REV_ARGS);
bool launch_fused_rev_c128(VQG_REV_ARGS);
bool launch_fused_fwd_df(VQG_FWD_ARGS);
bool launch_fused_rev_df(VQG_REV_ARGS);

// Compiled (tile qubits, register qubits) variants; every one fits shared memory.
// ff: complex128 in float-float arithmetic.
bool fused_supported(bool dbl, int K, int Rf, int Rr, bool ff) {
    if (!dbl) return K >= 10 && K <= 13 && (Rf == 4 || Rf == 5) && (Rr == 4 || (Rr == 3 && K <= 12));
    if (ff) return K >= 10 && K <= 12 && Rf == 3 && Rr == 3;
    return K >= 10 && K <= 12 && (Rf == 3 || Rf == 4) && (Rr == 3 || (Rr == 2 && K <= 11));
}
void launch_fused_ham(bool dbl, int K, const void *psi, void *lam, const HPass *hp, int pi,
                      const HGroup *groups, const HTerm *terms, uint64_t n_tiles, double *partials,
                      int nb, cudaStream_t s);
void launch_fused_ham_df(int K, const void *psi, void *lam, const HPass *hp, int pi, const HGroup *groups,
                         const HTerm *terms, uint64_t n_tiles, double *partials, int nb, cudaStream_t s);

bool float_float(bool dbl, const vqg_options &opt) { return dbl && opt.c128_arith == VQG_C128_FLOAT_FLOAT; }

// Forward tile pass in the circuit's arithmetic (complex64, complex128 FP64 or float-float).
bool launch_fused_fwd(bool dbl, bool ff, VQG_FWD_ARGS) {
    auto f = !dbl ? launch_fused_fwd_c64 : ff ? launch_fused_fwd_df : launch_fused_fwd_c128;
    return f(K, R, src, dst, passes, pi, st, ops, dg, it, mats, n_tiles, grid, s);
}

struct QUse {
    int q;
    bool diag;
};

// Qubit uses of a gate: a "diagonal" use (RZ, CZ, a control) commutes with every other
// diagonal use of that qubit; a non-diagonal use (a target) must sit in registers.
// PHASE and the targets of CRZ / CPHASE are diagonal too but are planned as targets
// (conservative: fewer reorderings, never a wrong one).
static int uses_of(const vqg_gate &g, QUse *u) {
    switch (g.kind) {
    case VQG_RX: case VQG_RY: case VQG_U3: case VQG_PHASE: u[0] = {g.q0, false}; return 1;
    case VQG_RZ: u[0] = {g.q0, true}; return 1;
    case VQG_CZ: u[0] = {g.q0, true}; u[1] = {g.q1, true}; return 2;
    case VQG_CNOT: case VQG_CRX: case VQG_CRY: case VQG_CRZ: case VQG_CPHASE:
        u[0] = {g.q0, true}; u[1] = {g.q1, false}; return 2;
    default: return 0;
    }
}

static bool has_control(int kind) { return kind == VQG_CNOT || is_controlled_param(kind); }

static int red_values(int kind) { return reduce_values_of(kind); }

// One greedy sweep over `order` with non-diagonal set `inS` (indexed by qubit).
// Applied gates go to `applied` (in order), the rest to `left`.  `cap_ops` /
// `cap_slots` bound the run (gates past the cap are deferred like blocked ones).
static void greedy(const std::vector<vqg_gate> &gates, const std::vector<int> &order,
                   const std::vector<char> &inS, int n, int cap_ops, int cap_slots,
                   std::vector<int> &applied, std::vector<int> &left) {
    std::vector<char> nd(n, 0), dg(n, 0);
    int slots = 0;
    applied.clear();
    left.clear();
    for (int i : order) {
        QUse u[2];
        const int nu = uses_of(gates[i], u);
        bool ok = (int)applied.size() < cap_ops && slots + red_values(gates[i].kind) <= cap_slots;
        for (int k = 0; k < nu && ok; ++k) {
            const int q = u[k].q;
            if (u[k].diag) ok = !nd[q];
            else ok = !nd[q] && !dg[q] && inS[q];
        }
        if (ok) {
            applied.push_back(i);
            slots += red_values(gates[i].kind);
        } else {
            left.push_back(i);
            for (int k = 0; k < nu; ++k) (u[k].diag ? dg : nd)[u[k].q] = 1;
        }
    }
}

// Tile layout of a pass: positions 0..L-1 are qubits 0..L-1, then `high` in its order
// (ascending, except where a Hamiltonian pass moves two qubits to its batch positions).
struct TileMap {
    int K, L;
    std::vector<int> pos_of;   // qubit -> tile position or -1
    std::vector<int> qubit_of; // tile position -> qubit
};

static TileMap make_tilemap(int n, int K, int L, const std::vector<int> &high) {
    TileMap t;
    t.K = K;
    t.L = L;
    t.pos_of.assign(n, -1);
    for (int q = 0; q < L; ++q) t.pos_of[q] = q, t.qubit_of.push_back(q);
    for (size_t i = 0; i < high.size(); ++i) t.pos_of[high[i]] = L + (int)i, t.qubit_of.push_back(high[i]);
    return t;
}

// Choose the K-L high qubits for the next pass: the first distinct qubits >= L used
// non-diagonally by the remaining gates, padded with the lowest unused qubits.
static std::vector<int> choose_high(const std::vector<vqg_gate> &gates, const std::vector<int> &rem,
                                    int n, int K, int L) {
    std::vector<int> high;
    std::vector<char> taken(n, 0);
    for (int i : rem) {
        QUse u[2];
        const int nu = uses_of(gates[i], u);
        for (int k = 0; k < nu; ++k)
            if (!u[k].diag && u[k].q >= L && !taken[u[k].q] && (int)high.size() < K - L)
                taken[u[k].q] = 1, high.push_back(u[k].q);
        if ((int)high.size() == K - L) break;
    }
    for (int q = L; q < n && (int)high.size() < K - L; ++q)
        if (!taken[q]) taken[q] = 1, high.push_back(q);
    std::sort(high.begin(), high.end());
    return high;
}

// Pass choice for a |0...0> start.  A pass computes only the tiles whose non-tile index
// bits lie inside the support (the qubits earlier gates acted on non-diagonally; see
// FPass::n_active), so gates applied while the support is small are cheap, and the order in
// which the tile sets visit the qubits decides how many gates run on sparse passes.  The
// planner therefore compares candidate tile sets -- choose_high's, and every window of K - L
// consecutive qubits above the row qubits -- by a cost model of the passes they lead to:
// a beam search over the next passes, each sequence completed with choose_high's passes, and
// the first tile set of the cheapest sequence taken (then searched again from the new state).
//
// Cost of one pass, forward plus reverse, in milliseconds of a 2^30-amplitude complex64 state
// on the measured kernels (only ratios matter): per-gate compute and per-pass memory
// traffic overlap (max), f = the share of tiles computed (skipped tiles are neither read nor
// written, FPass::zero_in).
static double pass_cost_model(int gates, double f) {
    const double fwd = std::max(f * 2.5, gates * f * 0.10) + 0.05;
    const double rev = std::max(f * 3.8, gates * f * 0.29) + 0.05;
    return fwd + rev;
}

namespace {
struct PassSearch {
    const std::vector<vqg_gate> &gates;
    int n, K, L, cap_ops;
    uint64_t support_of(uint64_t sup, const std::vector<int> &applied) const {
        for (int i : applied) {
            QUse u[2];
            const int nu = uses_of(gates[i], u);
            for (int k = 0; k < nu; ++k)
                if (!u[k].diag) sup |= 1ull << u[k].q;
        }
        return sup;
    }
    uint64_t tile_mask(const std::vector<int> &high) const {
        uint64_t m = (1ull << L) - 1ull;
        for (int q : high) m |= 1ull << q;
        return m;
    }
    // applies the pass with tile qubits `high` to (rem, sup); returns its cost
    double step(const std::vector<int> &high, std::vector<int> &rem, uint64_t &sup, std::vector<int> &applied) const {
        const uint64_t T = tile_mask(high);
        std::vector<char> inS(n, 0);
        for (int q = 0; q < n; ++q) inS[q] = (T >> q) & 1;
        std::vector<int> left;
        greedy(gates, rem, inS, n, cap_ops, kMaxPassSlots, applied, left);
        const int act = __builtin_popcountll(sup & ~T);
        const double c = pass_cost_model((int)applied.size(), std::ldexp(1.0, act - (n - K)));
        sup = support_of(sup, applied);
        rem.swap(left);
        return c;
    }
    double finish(std::vector<int> rem, uint64_t sup) const {
        double c = 0.0;
        std::vector<int> applied;
        while (!rem.empty()) {
            c += step(choose_high(gates, rem, n, K, L), rem, sup, applied);
            if (applied.empty()) return 1e30;  // no progress (cannot happen: the first gate fits)
        }
        return c;
    }
    std::vector<std::vector<int>> candidates(const std::vector<int> &rem) const {
        std::vector<std::vector<int>> out{choose_high(gates, rem, n, K, L)};
        for (int a = L; a + (K - L) <= n; ++a) {
            std::vector<int> h;
            for (int q = a; q < a + K - L; ++q) h.push_back(q);
            out.push_back(h);
        }
        return out;
    }
    std::vector<int> choose(const std::vector<int> &rem0, uint64_t sup0, int width, int depth) const {
        struct Node {
            double cost;
            std::vector<int> rem;
            uint64_t sup;
            int first;  // index of the first candidate on the way
        };
        const std::vector<std::vector<int>> first_cands = candidates(rem0);
        std::vector<Node> beam{{0.0, rem0, sup0, -1}};
        double best = 1e300;
        int best_first = 0;
        std::vector<int> applied;
        for (int d = 0; d < depth && !beam.empty(); ++d) {
            std::vector<std::pair<double, Node>> next;  // (cost with completion, node)
            for (const Node &nd : beam) {
                if (nd.rem.empty()) continue;
                const std::vector<std::vector<int>> cands = d == 0 ? first_cands : candidates(nd.rem);
                for (size_t c = 0; c < cands.size(); ++c) {
                    Node ch{nd.cost, nd.rem, nd.sup, nd.first < 0 ? (int)c : nd.first};
                    ch.cost += step(cands[c], ch.rem, ch.sup, applied);
                    if (applied.empty()) continue;
                    const double tot = ch.cost + finish(ch.rem, ch.sup);
                    if (tot < best) best = tot, best_first = ch.first;
                    next.push_back({tot, std::move(ch)});
                }
            }
            std::stable_sort(next.begin(), next.end(),
                             [](const std::pair<double, Node> &a, const std::pair<double, Node> &b) { return a.first < b.first; });
            beam.clear();
            for (auto &e : next) {
                bool dup = false;  // same remaining gates and support: keep the cheaper
                for (const Node &b : beam) dup = dup || (b.sup == e.second.sup && b.rem == e.second.rem);
                if (!dup) beam.push_back(std::move(e.second));
                if ((int)beam.size() >= width) break;
            }
        }
        return first_cands[best_first];
    }
};
}  // namespace

// Register stages of one pass over `seq` (gates in application order).  Emits stages,
// ops, diagonal blocks and their items into the plan; reverse stages carry reduction
// slots.  Within a stage, diagonal gates (RZ, CZ) are gathered into diagonal blocks:
// a diagonal gate joins the earliest block after the last op it does not commute
// with, and a non-diagonal gate is placed before a trailing run of blocks it commutes
// with.  Both moves only swap commuting gates.
struct StageItem {
    bool diag;
    uint64_t nd, dq;            // non-diagonal / diagonal qubit masks
    std::vector<int> gates;     // one gate, or the gates of a diagonal block
    int n_rz = 0, n_cz = 0;
};

static void build_stages(Plan &pl, const std::vector<vqg_gate> &gates, const std::vector<int> &slot_base,
                         int n, const TileMap &tm, const std::vector<int> &seq, int R, bool dbl,
                         bool reverse, int &n_lslots, int &stage0, int &n_stage, int &diag0, int &n_diag) {
    stage0 = (int)pl.stages.size();
    diag0 = (int)pl.diags.size();
    n_stage = 0;
    n_lslots = 0;
    const int K = tm.K;
    const int AB = dbl ? 16 : 8;
    std::vector<int> uns = seq, applied, left;
    while (!uns.empty()) {
        std::vector<int> regs;
        std::vector<char> isreg(K, 0);
        for (int i : uns) {
            QUse u[2];
            const int nu = uses_of(gates[i], u);
            for (int k = 0; k < nu; ++k) {
                if (u[k].diag) continue;
                const int p = tm.pos_of[u[k].q];
                if (!isreg[p] && (int)regs.size() < R) isreg[p] = 1, regs.push_back(p);
            }
            if ((int)regs.size() == R) break;
        }
        for (int p = K - 1; p >= 0 && (int)regs.size() < R; --p)
            if (!isreg[p]) isreg[p] = 1, regs.push_back(p);
        std::vector<char> inS(n, 0);
        for (int p : regs) inS[tm.qubit_of[p]] = 1;
        greedy(gates, uns, inS, n, kMaxPassOps, reverse ? kMaxStageValues : kMaxPassSlots, applied, left);
        const int NL = dbl ? 3 : 4, MOD = dbl ? 3 : 4;
        std::vector<int> thr;
        std::vector<char> used(K, 0);
        for (int r = 0; r < NL; ++r)
            for (int p = 0; p < K; ++p)
                if (!isreg[p] && !used[p] && p % MOD == r) {
                    used[p] = 1;
                    thr.push_back(p);
                    break;
                }
        for (int p = 0; p < K; ++p)
            if (!isreg[p] && !used[p]) used[p] = 1, thr.push_back(p);
        FStage st;
        std::memset(&st, 0, sizeof st);
        for (size_t b = 0; b < thr.size(); ++b) {
            st.thr_sw[b] = (uint16_t)(AB == 8 ? swz<8>(1u << thr[b]) : swz<16>(1u << thr[b]));
            st.thr_q[b] = (int8_t)tm.qubit_of[thr[b]];
        }
        for (int k = 0; k < R; ++k)
            st.reg_sw[k] = (uint16_t)(AB == 8 ? swz<8>(1u << regs[k]) : swz<16>(1u << regs[k]));
        auto regbit = [&](int q) -> int {
            const int p = tm.pos_of[q];
            if (p < 0) return -1;
            for (int k = 0; k < R; ++k)
                if (regs[k] == p) return k;
            return -1;
        };
        // order the stage's gates into single ops and diagonal blocks
        std::vector<StageItem> out;
        for (int i : applied) {
            const vqg_gate &g = gates[i];
            const bool is_diag = g.kind == VQG_RZ || g.kind == VQG_CZ;
            if (is_diag) {
                const uint64_t dq = (1ull << g.q0) | (g.kind == VQG_CZ ? 1ull << g.q1 : 0ull);
                int lim = -1;
                for (int idx = (int)out.size() - 1; idx >= 0; --idx)
                    if (!out[idx].diag && (out[idx].nd & dq)) { lim = idx; break; }
                bool placed = false;
                for (int idx = lim + 1; idx < (int)out.size() && !placed; ++idx) {
                    StageItem &b = out[idx];
                    if (!b.diag) continue;
                    if (g.kind == VQG_RZ ? b.n_rz >= kMaxDiagRz : b.n_cz >= kMaxDiagCz) continue;
                    b.gates.push_back(i);
                    b.dq |= dq;
                    (g.kind == VQG_RZ ? b.n_rz : b.n_cz)++;
                    placed = true;
                }
                if (!placed) {
                    StageItem b;
                    b.diag = true;
                    b.nd = 0;
                    b.dq = dq;
                    b.gates.push_back(i);
                    (g.kind == VQG_RZ ? b.n_rz : b.n_cz) = 1;
                    out.push_back(b);
                }
            } else {
                StageItem it;
                it.diag = false;
                it.nd = 1ull << (has_control(g.kind) ? g.q1 : g.q0);
                it.dq = has_control(g.kind) ? 1ull << g.q0 : 0ull;
                it.gates.push_back(i);
                size_t pos = out.size();
                while (pos > 0 && out[pos - 1].diag && !(out[pos - 1].dq & it.nd)) --pos;
                out.insert(out.begin() + pos, it);
            }
        }
        st.op0 = (int)pl.ops.size();
        // Reverse: the stash holds rowcap values per thread; when the next op's values do
        // not fit, a flush op reduces the rows written so far (their local slots are
        // contiguous from seg_first) and the rows restart at 0.
        const int rowcap = dbl ? kMaxStageRowsDbl : kMaxStageRows;
        int rows = 0, seg_first = n_lslots;
        for (const StageItem &it : out) {
            const int need = it.diag ? it.n_rz : red_values(gates[it.gates[0]].kind);
            if (reverse && need > 0 && rows + need > rowcap) {
                FOp f;
                std::memset(&f, 0, sizeof f);
                f.type = OP_FLUSH;
                f.gate = -1;
                f.cq = -1;
                f.diag = -1;
                f.lslot = (int16_t)seg_first;
                f.row = (int8_t)rows;
                pl.ops.push_back(f);
                seg_first = n_lslots;
                rows = 0;
            }
            FOp op;
            std::memset(&op, 0, sizeof op);
            op.lslot = -1;
            op.diag = -1;
            op.cq = -1;
            if (!it.diag) {
                const int i = it.gates[0];
                const vqg_gate &g = gates[i];
                op.gate = i;
                switch (g.kind) {
                case VQG_RY: op.type = OP_RY; op.k = (int8_t)regbit(g.q0); break;
                case VQG_RX: op.type = OP_RX; op.k = (int8_t)regbit(g.q0); break;
                case VQG_U3: op.type = OP_U3; op.k = (int8_t)regbit(g.q0); break;
                case VQG_CNOT:
                case VQG_CRX:
                case VQG_CRY:
                case VQG_CRZ:
                case VQG_CPHASE: {
                    const int kc = regbit(g.q0);
                    op.type = g.kind == VQG_CNOT ? OP_CNOT : g.kind == VQG_CRX ? OP_CRX : g.kind == VQG_CRY ? OP_CRY
                            : g.kind == VQG_CRZ ? OP_CRZ : OP_PH;
                    op.k = (int8_t)regbit(g.q1);
                    op.cq = -1;
                    if (kc >= 0) op.rm0 = 1u << kc; else op.cq = (int8_t)g.q0;
                    break;
                }
                case VQG_PHASE: op.type = OP_PH; op.k = (int8_t)regbit(g.q0); op.cq = -1; break;
                default: break;
                }
                if (reverse) {
                    const int nv = red_values(g.kind);
                    if (nv) {
                        op.lslot = (int16_t)n_lslots;
                        op.row = (int8_t)rows;
                        for (int v = 0; v < nv; ++v) {
                            pl.slot_map.push_back(slot_base[i] + v);
                            st.row_slot[rows++] = (int16_t)(n_lslots + v);
                        }
                        n_lslots += nv;
                    }
                }
            } else {
                op.type = OP_DIAG;
                op.gate = -1;
                op.cq = -1;
                op.row = (int8_t)rows;
                op.diag = (int16_t)((int)pl.diags.size() - diag0);
                FDiag d;
                std::memset(&d, 0, sizeof d);
                d.item0 = (int)pl.items.size();
                std::vector<FDItem> xs;
                for (int i : it.gates) {
                    const vqg_gate &g = gates[i];
                    FDItem x;
                    std::memset(&x, 0, sizeof x);
                    x.gate = i;
                    x.lslot = -1;
                    if (g.kind == VQG_RZ) {
                        const int k = regbit(g.q0);
                        if (k >= 0) x.type = DI_RZ_REG, x.k0 = (int16_t)k;
                        else x.type = DI_RZ_THR, x.g0 = 1ull << g.q0, st.has_phase = 1;
                    } else {
                        const int ka = regbit(g.q0), kb = regbit(g.q1);
                        if (ka >= 0 && kb >= 0) x.type = DI_CZ_RR, x.k0 = (int16_t)ka, x.k1 = (int16_t)kb;
                        else if (ka >= 0) x.type = DI_CZ_RT, x.k0 = (int16_t)ka, x.g0 = 1ull << g.q1;
                        else if (kb >= 0) x.type = DI_CZ_RT, x.k0 = (int16_t)kb, x.g0 = 1ull << g.q0;
                        else x.type = DI_CZ_TT, x.g0 = 1ull << g.q0, x.g1 = 1ull << g.q1, st.has_phase = 1;
                    }
                    xs.push_back(x);
                }
                // RZ_REG, RZ_THR, CZ_RT / CZ_TT, CZ_RR (stable: gate order within a class)
                auto cls = [](int t) { return t == DI_RZ_REG ? 0 : t == DI_RZ_THR ? 1 : t == DI_CZ_RR ? 3 : 2; };
                std::stable_sort(xs.begin(), xs.end(),
                                 [&](const FDItem &a, const FDItem &b) { return cls(a.type) < cls(b.type); });
                int thr0 = -1, n_thr = 0;
                for (size_t q = 0; q < xs.size(); ++q) {
                    FDItem &x = xs[q];
                    if (x.type == DI_RZ_REG || x.type == DI_RZ_THR) {
                        if (reverse) {  // reduction slots and stash rows follow the item order
                            x.lslot = n_lslots++;
                            pl.slot_map.push_back(slot_base[x.gate]);
                            st.row_slot[rows++] = (int16_t)x.lslot;
                        }
                        d.n_rz++;
                    }
                    if (x.type == DI_CZ_RT) d.has_rt = 1;
                    if (cls(x.type) == 1 || cls(x.type) == 2) {
                        if (thr0 < 0) thr0 = (int)q;
                        ++n_thr;
                    }
                    pl.items.push_back(x);
                }
                d.thr0 = (int16_t)(thr0 < 0 ? 0 : thr0);
                d.n_thr = (int16_t)n_thr;
                d.n_item = (int)pl.items.size() - d.item0;
                pl.diags.push_back(d);
            }
            pl.ops.push_back(op);
        }
        st.n_op = (int)pl.ops.size() - st.op0;
        st.n_rows = (int16_t)rows;
        pl.stages.push_back(st);
        std::array<int8_t, kMaxRegBits> rq{};
        for (int k = 0; k < R; ++k) rq[k] = (int8_t)tm.qubit_of[regs[k]];
        pl.stage_reg_q.push_back(rq);
        ++n_stage;
        uns.swap(left);
    }
    n_diag = (int)pl.diags.size() - diag0;
}

// Host-side check of every index a fused kernel derives from the plan: tile
// geometry, register/thread bit assignment (a permutation of the K tile positions),
// op fields, reduction slots and Hamiltonian masks.  Returns an empty string if valid.
std::string validate_plan(const Plan &pl, int n, int n_gslots, bool dbl) {
    char buf[256];
    const int K = pl.K, L = pl.L;
    const int rowcap = dbl ? kMaxStageRowsDbl : kMaxStageRows;
    auto fail = [&](const char *what, int a, int b) {
        snprintf(buf, sizeof buf, "plan check failed: %s (%d, %d)", what, a, b);
        return std::string(buf);
    };
    auto check_geom = [&](const int32_t *high, int n_high, const int32_t *nontile, int n_nt) -> std::string {
        if (n_high != K - L || n_nt != n - K) return fail("tile geometry", n_high, n_nt);
        std::vector<int> seen(n, 0);
        for (int q = 0; q < L; ++q) seen[q]++;
        for (int i = 0; i < n_high; ++i) {
            if (high[i] < L || high[i] >= n) return fail("high qubit", i, high[i]);
            seen[high[i]]++;
        }
        for (int i = 0; i < n_nt; ++i) {
            if (nontile[i] < 0 || nontile[i] >= n) return fail("non-tile qubit", i, nontile[i]);
            seen[nontile[i]]++;
        }
        for (int q = 0; q < n; ++q)
            if (seen[q] != 1) return fail("qubit coverage", q, seen[q]);
        return "";
    };
    for (size_t j = 0; j < pl.passes.size(); ++j) {
        const FPass &p = pl.passes[j];
        std::string e = check_geom(p.high, p.n_high, p.nontile, p.n_nontile);
        if (!e.empty()) return e;
        if (p.n_stage < 1 || p.n_stage > pl.caps.stages || p.n_rstage < 1 || p.n_rstage > pl.caps.stages)
            return fail("stage count", p.n_stage, p.n_rstage);
        if (p.n_lslots < 0 || p.n_lslots > kMaxPassSlots) return fail("slot count", (int)j, p.n_lslots);
        if (p.n_active < 0 || p.n_active > p.n_nontile || p.n_active_zero < 0 || p.n_active_zero > p.n_nontile)
            return fail("active non-tile qubits", (int)j, p.n_active);
        if (p.slotmap0 < 0 || p.slotmap0 + p.n_lslots > (int)pl.slot_map.size()) return fail("slot map", (int)j, p.slotmap0);
        for (int i = 0; i < p.n_lslots; ++i)
            if (pl.slot_map[p.slotmap0 + i] < 0 || pl.slot_map[p.slotmap0 + i] >= n_gslots)
                return fail("global slot", i, pl.slot_map[p.slotmap0 + i]);
        for (int dir = 0; dir < 2; ++dir) {
            const int s0 = dir ? p.rstage0 : p.stage0, ns = dir ? p.n_rstage : p.n_stage;
            const int R = dir ? pl.Rr : pl.Rf;
            if (s0 < 0 || s0 + ns > (int)pl.stages.size()) return fail("stage range", s0, ns);
            const int op_first = pl.stages[s0].op0;
            int op_total = 0;
            for (int s = s0; s < s0 + ns; ++s) {
                const FStage &st = pl.stages[s];
                if (st.op0 != op_first + op_total) return fail("op contiguity", s, st.op0);
                op_total += st.n_op;
                // swizzled masks of thread and register bits must span all 2^K slots
                uint32_t span = 0;
                std::vector<uint32_t> basis;
                for (int b = 0; b < K - R; ++b) basis.push_back(st.thr_sw[b]);
                for (int k = 0; k < R; ++k) basis.push_back(st.reg_sw[k]);
                // Gaussian elimination over GF(2)
                std::vector<uint32_t> rows;
                for (uint32_t v : basis) {
                    for (uint32_t r : rows) v = std::min(v, v ^ r);
                    if (!v) return fail("dependent tile bits", s, 0);
                    rows.push_back(v);
                    std::sort(rows.rbegin(), rows.rend());
                    span |= v;
                }
                for (uint32_t v : basis)
                    if (v >> K) return fail("swizzled mask range", s, (int)v);
                for (int k = 0; k < K - R; ++k)
                    if (st.thr_q[k] < 0 || st.thr_q[k] >= n) return fail("thread qubit", s, st.thr_q[k]);
                if (dir) {
                    if (st.n_rows < 0 || st.n_rows > rowcap) return fail("stage rows", s, st.n_rows);
                    for (int r = 0; r < st.n_rows; ++r)
                        if (st.row_slot[r] < 0 || st.row_slot[r] >= p.n_lslots || st.row_slot[r] != st.row_slot[0] + r)
                            return fail("row slot", s, st.row_slot[r]);
                }
                for (int o = st.op0; o < st.op0 + st.n_op; ++o) {
                    const FOp &op = pl.ops[o];
                    if (op.type < OP_RY || op.type > OP_LAST) return fail("op type", o, op.type);
                    if (op.type != OP_DIAG && (op.k < 0 || op.k >= R)) return fail("register bit", o, op.k);
                    if (op.rm0 >> R) return fail("register mask", o, (int)op.rm0);
                    const bool ctl_op = op.type == OP_CNOT || op.type >= OP_CRX;
                    if (ctl_op && op.rm0 == (1u << op.k)) return fail("control = target", o, op.k);
                    if (op.type == OP_CNOT && !op.rm0 && (op.cq < 0 || op.cq >= n)) return fail("control qubit", o, op.cq);
                    if (op.type >= OP_CRX && op.type <= OP_CRZ && !op.rm0 && (op.cq < 0 || op.cq >= n))
                        return fail("control qubit", o, op.cq);
                    if (op.type == OP_PH && !op.rm0 && (op.cq < -1 || op.cq >= n)) return fail("control qubit", o, op.cq);
                    if (!ctl_op && (op.rm0 || op.cq != -1)) return fail("stray control", o, op.cq);
                    if (op.type != OP_DIAG && op.type != OP_FLUSH && (op.gate < 0)) return fail("gate index", o, op.gate);
                    if (op.type == OP_FLUSH) {
                        if (!dir) return fail("flush in a forward stage", o, 0);
                        if (op.row < 1 || op.row > rowcap) return fail("flush rows", o, op.row);
                        if (op.lslot < 0 || op.lslot + op.row > p.n_lslots) return fail("flush slots", o, op.lslot);
                    }
                    // the stash segment this op writes into ends at the next flush or the stage end
                    int seg_rows = st.n_rows, seg_first = st.n_rows ? st.row_slot[0] : 0;
                    if (dir) {
                        for (int f = o; f < st.op0 + st.n_op; ++f)
                            if (f > o && pl.ops[f].type == OP_FLUSH) {
                                seg_rows = pl.ops[f].row;
                                seg_first = pl.ops[f].lslot;
                                break;
                            }
                    }
                    if (dir && op.lslot >= 0 && op.type != OP_FLUSH) {
                        const int nv = op.type == OP_U3 ? 8 : 1;
                        if (op.lslot + nv > p.n_lslots) return fail("local slot", o, op.lslot);
                        if (op.row < 0 || op.row + nv > seg_rows) return fail("stash row", o, op.row);
                        if (op.lslot != seg_first + op.row) return fail("slot of stash row", o, op.lslot);
                    }
                    if (dir && op.type == OP_DIAG) {
                        const FDiag &D = pl.diags[p.rdiag0 + op.diag];
                        if (op.row < 0 || op.row + D.n_rz > seg_rows) return fail("diag stash row", o, op.row);
                        for (int r = 0; r < D.n_rz; ++r)
                            if (pl.items[D.item0 + r].lslot != seg_first + op.row + r) return fail("slot of diag row", o, r);
                    }
                    if (op.type == OP_DIAG) {
                        const int d0 = dir ? p.rdiag0 : p.diag0, nd = dir ? p.n_rdiag : p.n_diag;
                        if (op.diag < 0 || op.diag >= nd) return fail("diagonal block", o, op.diag);
                        const FDiag &D = pl.diags[d0 + op.diag];
                        if (D.n_rz > kMaxDiagRz || D.n_rz > D.n_item) return fail("block RZ count", o, D.n_rz);
                        if (D.item0 < 0 || D.item0 + D.n_item > (int)pl.items.size()) return fail("item range", o, D.item0);
                        if (D.thr0 < 0 || D.n_thr < 0 || D.thr0 + D.n_thr > D.n_item) return fail("thread items", o, D.thr0);
                        for (int i = D.item0; i < D.item0 + D.n_item; ++i) {
                            const FDItem &x = pl.items[i];
                            const bool rz = x.type == DI_RZ_REG || x.type == DI_RZ_THR;
                            const bool thr = x.type == DI_RZ_THR || x.type == DI_CZ_RT || x.type == DI_CZ_TT;
                            const int rel = i - D.item0;
                            if (thr != (rel >= D.thr0 && rel < D.thr0 + D.n_thr)) return fail("thread item range", i, x.type);
                            if ((i - D.item0 < D.n_rz) != rz) return fail("item order", i, x.type);
                            if (x.type < DI_RZ_REG || x.type > DI_CZ_TT) return fail("item type", i, x.type);
                            const bool k0 = x.type == DI_RZ_REG || x.type == DI_CZ_RR || x.type == DI_CZ_RT;
                            if (k0 && (x.k0 < 0 || x.k0 >= R)) return fail("item bit", i, x.k0);
                            if (x.type == DI_CZ_RR && (x.k1 < 0 || x.k1 >= R || x.k1 == x.k0)) return fail("item bit 2", i, x.k1);
                            if (rz && (x.gate < 0)) return fail("item gate", i, x.gate);
                            if (dir && rz && (x.lslot < 0 || x.lslot >= p.n_lslots)) return fail("item slot", i, x.lslot);
                        }
                    }
                }
            }
            if (op_total > pl.caps.ops) return fail("ops per pass", (int)j, op_total);
        }
        for (int dir = 0; dir < 2; ++dir) {
            const int d0 = dir ? p.rdiag0 : p.diag0, nd = dir ? p.n_rdiag : p.n_diag;
            if (nd > pl.caps.diags) return fail("diagonal blocks per pass", (int)j, nd);
            if (nd) {
                if (d0 < 0 || d0 + nd > (int)pl.diags.size()) return fail("diagonal range", d0, nd);
                int it = pl.diags[d0].item0;
                for (int d = d0; d < d0 + nd; ++d) {
                    if (pl.diags[d].item0 != it) return fail("item contiguity", d, pl.diags[d].item0);
                    it += pl.diags[d].n_item;
                }
                if (it - pl.diags[d0].item0 > pl.caps.items) return fail("items per pass", (int)j, it);
            }
        }
    }
    for (size_t h = 0; h < pl.hp.size(); ++h) {
        const HPass &p = pl.hp[h];
        std::string e = check_geom(p.high, p.n_high, p.nontile, p.n_nontile);
        if (!e.empty()) return e;
        if (p.group0 < 0 || p.group0 + p.n_group > (int)pl.hg.size()) return fail("group range", (int)h, p.group0);
        if (p.n_group > kMaxHamGroups) return fail("groups per pass", (int)h, p.n_group);
        {
            int nt = 0;
            for (int g = p.group0; g < p.group0 + p.n_group; ++g) nt += pl.hg[g].n_term;
            if (nt > kMaxHamTerms) return fail("terms per pass", (int)h, nt);
            if (p.n_group && pl.hg[p.group0 + p.n_group - 1].term0 + pl.hg[p.group0 + p.n_group - 1].n_term -
                                 pl.hg[p.group0].term0 != nt)
                return fail("term contiguity", (int)h, nt);
        }
        for (int g = p.group0; g < p.group0 + p.n_group; ++g) {
            const HGroup &G0 = pl.hg[g];
            if (G0.xl >> K) return fail("tile flip mask", g, (int)G0.xl);
            if (G0.term0 < 0 || G0.term0 + G0.n_term > (int)pl.ht.size()) return fail("term range", g, G0.term0);
        }
    }
    return "";
}

// Built-in schedule table: the largest tile that still leaves 2^8 tiles for the SMs
// (n - 8), within the compiled range [10, 13] (complex64) / [10, 12] (complex128).
int default_tile_qubits(int n, bool dbl) {
    const int Kmax = dbl ? 12 : 13;
    return std::min(Kmax, std::max(10, n - 8));
}

static int occupancy_grid(int num_sms, int per_sm, uint64_t n_tiles) {
    const uint64_t g = (uint64_t)num_sms * (uint64_t)std::max(per_sm, 1);
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(g, n_tiles));
}

// Pure host planning of the gate passes (no device work).  Returns nullptr with an
// empty `err` when no fused schedule applies (n or the tile below 10 qubits, fusion
// off), nullptr with `err` set when the plan fails validation.
Plan *plan_gates(int n, const std::vector<vqg_gate> &gates, const std::vector<int> &slot_base,
                        int n_gslots, bool dbl, const vqg_options &opt, std::string &err, const PassCaps &caps,
                        bool single_kernels, bool zero_start) {
    err.clear();
    const int G = (int)gates.size();
    const bool ff = float_float(dbl, opt);
    int K = std::min(n, default_tile_qubits(n, dbl));
    if (opt.tile_qubits > 0) K = std::min(opt.tile_qubits, n);
    const int Rf = opt.fwd_reg_qubits > 0 ? opt.fwd_reg_qubits : (ff ? 3 : dbl ? 4 : 5);
    const int Rr = opt.rev_reg_qubits > 0 ? opt.rev_reg_qubits : (dbl ? 3 : 4);
    if (!opt.fusion || G == 0 || K < 10) return nullptr;
    if (single_kernels ? !fused_supported(dbl, K, Rf, Rr, ff)
                       : (Rf < 1 || Rr < 1 || Rf > kMaxRegBits || Rr > kMaxRegBits || K > 13 ||
                          K - Rf > kMaxThreadBits || K - Rr > kMaxThreadBits)) {
        err = "no compiled fused kernel for this tile / register-qubit choice";
        return nullptr;
    }
    Plan *pl = new Plan();
    pl->caps = caps;
    pl->K = K;
    pl->L = dbl ? 3 : 4;
    pl->Rf = Rf;
    pl->Rr = Rr;
    pl->n_tiles = 1ull << (n - K);
    const int L = pl->L;
    std::vector<int> rem(G), applied, left;
    for (int i = 0; i < G; ++i) rem[i] = i;
    uint64_t support = 0;  // qubits on which a |0...0> start may have a set bit before the pass
    // tile sets chosen for a |0...0> start (PassSearch) on plans with more than a few tiles;
    // the search's cost grows with gates x qubits, so large circuits search less, and the
    // batched launch (hundreds of circuits planned at once) searches narrowly
    const bool search = zero_start && n - K >= 2;
    const double work = (double)G * (double)n;
    const int width = !single_kernels ? 2 : work <= 4e4 ? 12 : work <= 2e5 ? 4 : 0;
    const int depth = !single_kernels ? 3 : width ? 8 : 0;
    const PassSearch ps{gates, n, K, L, caps.ops};
    while (!rem.empty()) {
        std::vector<int> high = search && width ? ps.choose(rem, support, width, depth) : choose_high(gates, rem, n, K, L);
        TileMap tm = make_tilemap(n, K, L, high);
        std::vector<char> inS(n, 0);
        for (int q = 0; q < n; ++q) inS[q] = tm.pos_of[q] >= 0;
        // a pass must fit the kernels' shared-memory program budget; shrink it if not
        for (int cap = caps.ops;; cap = std::max(1, cap / 2)) {
            greedy(gates, rem, inS, n, cap, kMaxPassSlots, applied, left);
            const size_t n_st = pl->stages.size(), n_op = pl->ops.size(), n_dg = pl->diags.size();
            const size_t n_it = pl->items.size(), n_sm = pl->slot_map.size();
            FPass p;
            std::memset(&p, 0, sizeof p);
            p.n_high = (int)high.size();
            for (size_t i = 0; i < high.size(); ++i) p.high[i] = high[i];
            // non-tile qubits that may carry a set bit come first (see FPass::n_active)
            for (int q = 0; q < n; ++q)
                if (tm.pos_of[q] < 0 && ((support >> q) & 1)) p.nontile[p.n_nontile++] = q;
            p.n_active_zero = p.n_active = p.n_nontile;
            p.zero_in = p.zero_in_zero = (n >= 64 ? ~0ull : (1ull << n) - 1ull) & ~support;
            for (int q = 0; q < n; ++q)
                if (tm.pos_of[q] < 0 && !((support >> q) & 1)) p.nontile[p.n_nontile++] = q;
            p.from_zero = pl->passes.empty() ? 1 : 0;
            p.n_gates = (int)applied.size();
            int nls;
            build_stages(*pl, gates, slot_base, n, tm, applied, pl->Rf, dbl, false, nls, p.stage0, p.n_stage,
                         p.diag0, p.n_diag);
            std::vector<int> rseq(applied.rbegin(), applied.rend());
            p.slotmap0 = (int)pl->slot_map.size();
            build_stages(*pl, gates, slot_base, n, tm, rseq, pl->Rr, dbl, true, p.n_lslots, p.rstage0,
                         p.n_rstage, p.rdiag0, p.n_rdiag);
            auto items_of = [&](int d0, int nd) {
                return nd ? pl->diags[d0 + nd - 1].item0 + pl->diags[d0 + nd - 1].n_item - pl->diags[d0].item0 : 0;
            };
            const bool fits = p.n_stage <= caps.stages && p.n_rstage <= caps.stages &&
                              p.n_diag <= caps.diags && p.n_rdiag <= caps.diags &&
                              items_of(p.diag0, p.n_diag) <= caps.items &&
                              items_of(p.rdiag0, p.n_rdiag) <= caps.items;
            if (fits || cap == 1) {
                pl->passes.push_back(p);
                pl->pass_gates.emplace_back(applied.begin(), applied.end());
                // amplitude can only move onto qubits that a gate acts on non-diagonally
                for (int i : applied) {
                    QUse u[2];
                    const int nu = uses_of(gates[i], u);
                    for (int k = 0; k < nu; ++k)
                        if (!u[k].diag) support |= 1ull << u[k].q;
                }
                break;
            }
            pl->stages.resize(n_st);
            pl->stage_reg_q.resize(n_st);
            pl->ops.resize(n_op);
            pl->diags.resize(n_dg);
            pl->items.resize(n_it);
            pl->slot_map.resize(n_sm);
        }
        rem.swap(left);
    }
    err = validate_plan(*pl, n, n_gslots, dbl);
    if (!err.empty()) {
        delete pl;
        return nullptr;
    }
    pl->ckpt_of_pass.assign(pl->passes.size(), -1);
    return pl;
}

// Device copies of a plan's pass tables (at least one element each: a valid pointer
// for empty tables; only what exists is copied).
int Circuit::upload_plan(Plan *pl) {
    auto up = [&](void **d, const auto &vec) -> int {
        const size_t elem = sizeof(vec[0]);
        int s2 = dalloc(d, elem * std::max<size_t>(vec.size(), 1));
        if (s2) return s2;
        if (!vec.empty() && h2d(*d, vec.data(), elem * vec.size()) != cudaSuccess)
            return set_error(VQG_ERR_CUDA, "plan upload failed");
        return VQG_OK;
    };
    int st;
    if ((st = up((void **)&pl->d_passes, pl->passes))) return st;
    if ((st = up((void **)&pl->d_stages, pl->stages))) return st;
    if ((st = up((void **)&pl->d_ops, pl->ops))) return st;
    if ((st = up((void **)&pl->d_slot_map, pl->slot_map))) return st;
    if ((st = up((void **)&pl->d_diags, pl->diags))) return st;
    if ((st = up((void **)&pl->d_items, pl->items))) return st;
    return VQG_OK;
}

// Release a plan with its device tables.
void Circuit::release_plan(Plan *pl) {
    if (!pl) return;
    for (void *p : {(void *)pl->d_passes, (void *)pl->d_stages, (void *)pl->d_ops, (void *)pl->d_diags,
                    (void *)pl->d_items, (void *)pl->d_slot_map, (void *)pl->d_hp, (void *)pl->d_hg,
                    (void *)pl->d_ht, (void *)pl->d_mats_f})
        dfree(p);
    delete pl;
}

int Circuit::build_plan() {
    // gate plan once; Hamiltonian plan whenever the Hamiltonian changes
    if (!plan) {
        plan_ok = false;
        std::string err;
        Plan *pl = plan_gates(n, gates, slot_base, n_gslots, dbl, opt, err);
        if (!pl) {
            if (!err.empty()) return set_error(VQG_ERR_UNSUPPORTED, "%s", err.c_str());
            return VQG_OK;  // no fused schedule for this size: one kernel per gate
        }
        pl->grid_fwd = occupancy_grid(num_sms, 2, pl->n_tiles);
        if (has_input) {  // pass 0 reads the input state; any tile may be non-zero
            pl->passes[0].from_zero = 0;
            for (FPass &p : pl->passes) p.n_active = p.n_nontile, p.zero_in = 0;
        }
        plan = pl;
        int st;
        if ((st = upload_plan(pl))) return st;
        if (!dbl && (st = dalloc((void **)&pl->d_mats_f, sizeof(float) * 8 * std::max(G, 1)))) return st;
        if (!dbl && opt.specialize && (st = spec_build(pl, opt.specialize >= 2))) return st;
        plan_ok = true;
        if (prod_active && (st = build_product_plans())) return st;  // same tile geometry
    }
    if (plan && has_ham) return build_ham_plan();
    return VQG_OK;
}

// Hamiltonian passes: greedy set cover of the groups' flip masks by tiles (the low L
// qubits are always inside; each pass adds the groups whose high flip bits fit).
// Returns false (nothing planned) when some group cannot live in one tile: its flip
// mask has more high bits than the tile has, or it has more terms than a pass holds.
// One greedy cover of the groups' high flip bits by tile high sets of at most K - L qubits:
// each pass adds the group that needs the fewest new qubits (ties: the one whose union covers
// most remaining groups), until none fits.  With rng, each pick is drawn from the (up to)
// three best-covering of the fewest-new-qubit candidates.  Returns each pass's high set and
// its groups (ascending).
using HamCover = std::vector<std::pair<uint64_t, std::vector<int>>>;
static HamCover cover_groups(const std::vector<HamGroup> &ham, int K, int L, uint64_t *rng) {
    const uint64_t lowmask = (1ull << L) - 1ull;
    auto high_of = [&](int g) { return ham[g].x & ~lowmask; };
    std::vector<int> rem;
    for (size_t g = 0; g < ham.size(); ++g) rem.push_back((int)g);
    HamCover out;
    while (!rem.empty()) {
        uint64_t S = 0;
        std::vector<char> chosen(ham.size(), 0);
        while (true) {
            std::vector<std::pair<int, int>> cands;  // (cov, group) of the fewest-new-qubit ones
            int best_new = 1 << 30;
            for (int g : rem) {
                if (chosen[g]) continue;
                const uint64_t h = high_of(g);
                if (__builtin_popcountll(S | h) > K - L) continue;
                const int nw = __builtin_popcountll(h & ~S);
                if (nw > best_new) continue;
                const uint64_t cand = S | h;
                int cov = 0;
                for (int g2 : rem) cov += ((high_of(g2) & ~cand) == 0);
                if (nw < best_new) best_new = nw, cands.clear();
                cands.push_back({cov, g});
            }
            if (cands.empty()) break;
            // highest coverage first; among equal coverage the lowest group index
            std::stable_sort(cands.begin(), cands.end(), [](const std::pair<int, int> &a, const std::pair<int, int> &b) {
                return a.first > b.first;
            });
            size_t pick = 0;
            if (rng) {
                *rng = *rng * 6364136223846793005ull + 1442695040888963407ull;  // LCG step
                pick = (size_t)((*rng >> 33) % std::min<size_t>(3, cands.size()));
            }
            const uint64_t S2 = S | high_of(cands[pick].second);
            int ng = 0, nt = 0;
            for (int g2 : rem)
                if ((high_of(g2) & ~S2) == 0) ++ng, nt += ham[g2].count;
            if (ng > kMaxHamGroups || nt > kMaxHamTerms) break;
            S = S2;
            for (int g2 : rem)
                if ((high_of(g2) & ~S) == 0) chosen[g2] = 1;
        }
        std::vector<int> mine, next;
        for (int g : rem) (chosen[g] ? mine : next).push_back(g);
        out.push_back({S, mine});
        rem.swap(next);
    }
    return out;
}

// Hamiltonian passes: greedy set cover of the groups' flip masks by tiles (the low L
// qubits are always inside; each pass adds the groups whose high flip bits fit).  The
// deterministic cover and a few randomised ones (fixed seed) are tried and the one with
// the fewest passes is kept: every pass streams psi and lambda once, so passes are the cost.
// Returns false (nothing planned) when some group cannot live in one tile: its flip
// mask has more high bits than the tile has, or it has more terms than a pass holds.
bool plan_hamiltonian(Plan *pl, int n, const std::vector<HamGroup> &ham,
                             const std::vector<PauliTerm> &host_terms) {
    pl->hp.clear();
    pl->hg.clear();
    pl->ht.clear();
    const int K = pl->K, L = pl->L;
    const uint64_t lowmask = (1ull << L) - 1ull;
    for (const HamGroup &g : ham)
        if (__builtin_popcountll(g.x & ~lowmask) > K - L || g.count > kMaxHamTerms) return false;
    HamCover cover = cover_groups(ham, K, L, nullptr);
    {
        // restarts while the work (groups^2 per pick) stays small
        const double work = (double)ham.size() * (double)ham.size() * (double)(K - L) * (double)cover.size();
        const int restarts = work > 0 ? (int)std::min(32.0, 4e8 / work) : 0;
        uint64_t rng = 0x9e3779b97f4a7c15ull;
        for (int r = 0; r < restarts && cover.size() > 1; ++r) {
            HamCover c = cover_groups(ham, K, L, &rng);
            if (c.size() < cover.size()) cover.swap(c);
        }
    }
    // The first pass writes lambda instead of adding to it (it reads 16 bytes per amplitude,
    // the others 24): lead with the pass with the fewest groups, whose time is the memory
    // traffic, rather than a shared-memory-bound one that would not get faster.
    if (!cover.empty()) {
        size_t lightest = 0;
        for (size_t i = 1; i < cover.size(); ++i)
            if (cover[i].second.size() < cover[lightest].second.size()) lightest = i;
        std::rotate(cover.begin(), cover.begin() + lightest, cover.begin() + lightest + 1);
    }
    bool first = true;
    for (const auto &pass : cover) {
        uint64_t S = pass.first;
        // fill the tile's high set: S's qubits, then the lowest others
        std::vector<int> high;
        for (int q = L; q < n; ++q)
            if ((S >> q) & 1) high.push_back(q);
        for (int q = L; q < n && (int)high.size() < K - L; ++q)
            if (!((S >> q) & 1)) high.push_back(q), S |= 1ull << q;
        std::sort(high.begin(), high.end());
        // complex64 batches of the Hamiltonian tile pass hold chunks that differ in tile
        // positions L+5 and L+6 (HamGeo): flip masks equal outside those two qubits and qubit
        // 0 share their partner loads, and one with no other bit needs none.  Put there the
        // pair of high qubits that leaves the fewest distinct other parts.
        if (L == 4 && (int)high.size() >= 7) {
            auto loads = [&](int a, int b) {
                const uint64_t m = 1ull | (1ull << a) | (1ull << b);
                std::vector<uint64_t> ys;
                for (int g : pass.second)
                    if (ham[g].x & ~m) ys.push_back(ham[g].x & ~m);
                std::sort(ys.begin(), ys.end());
                return (int)(std::unique(ys.begin(), ys.end()) - ys.begin());
            };
            int ba = high[5], bb = high[6], best = loads(ba, bb);
            for (size_t i = 0; i < high.size(); ++i)
                for (size_t j = i + 1; j < high.size(); ++j) {
                    const int c = loads(high[i], high[j]);
                    if (c < best) best = c, ba = high[i], bb = high[j];
                }
            std::vector<int> rest;
            for (int q : high)
                if (q != ba && q != bb) rest.push_back(q);
            rest.insert(rest.begin() + 5, {ba, bb});
            high.swap(rest);
        }
        TileMap tm = make_tilemap(n, K, L, high);
        HPass hp;
        std::memset(&hp, 0, sizeof hp);
        hp.n_high = (int)high.size();
        for (size_t i = 0; i < high.size(); ++i) hp.high[i] = high[i];
        for (int q = 0; q < n; ++q)
            if (tm.pos_of[q] < 0) hp.nontile[hp.n_nontile++] = q;
        hp.group0 = (int)pl->hg.size();
        hp.first = first ? 1 : 0;
        hp.eslot = (int)pl->hp.size();
        for (int g : pass.second) {
            const HamGroup &G0 = ham[g];
            HGroup hg;
            std::memset(&hg, 0, sizeof hg);
            hg.xg = G0.x;
            uint32_t xl = 0;
            for (int q = 0; q < n; ++q)
                if ((G0.x >> q) & 1) xl |= 1u << tm.pos_of[q];
            hg.xl = xl;
            hg.term0 = (int)pl->ht.size();
            hg.n_term = G0.count;
            for (int k = 0; k < G0.count; ++k) {
                const PauliTerm &t = host_terms[G0.first + k];
                HTerm h;
                std::memset(&h, 0, sizeof h);
                h.z = t.z;
                for (int q = 0; q < n; ++q) {
                    if (!((t.z >> q) & 1)) continue;
                    if (tm.pos_of[q] >= 0) h.zl |= 1u << tm.pos_of[q];
                    else h.znt |= 1ull << q;
                }
                const double sg = (__builtin_popcountll(G0.x & t.z) & 1) ? -1.0 : 1.0;
                h.wr = sg * t.wr;
                h.wi = sg * t.wi;
                h.fr = (float)h.wr;
                h.fi = (float)h.wi;
                pl->ht.push_back(h);
            }
            pl->hg.push_back(hg);
        }
        hp.n_group = (int)pl->hg.size() - hp.group0;
        pl->hp.push_back(hp);
        first = false;
    }
    if (pl->hp.empty()) {  // no terms at all: one pass that writes lambda = 0
        HPass hp;
        std::memset(&hp, 0, sizeof hp);
        std::vector<int> high;
        for (int q = L; q < n && (int)high.size() < K - L; ++q) high.push_back(q);
        TileMap tm = make_tilemap(n, K, L, high);
        hp.n_high = (int)high.size();
        for (size_t i = 0; i < high.size(); ++i) hp.high[i] = high[i];
        for (int q = 0; q < n; ++q)
            if (tm.pos_of[q] < 0) hp.nontile[hp.n_nontile++] = q;
        hp.first = 1;
        pl->hp.push_back(hp);
    }
    return true;
}

int Circuit::build_ham_plan() {
    Plan *pl = plan;
    ham_plan_ok = false;
    if (!plan_hamiltonian(pl, n, ham, host_terms)) return VQG_OK;  // one pass per group instead
    {
        const std::string err = validate_plan(*pl, n, n_gslots, dbl);
        if (!err.empty()) return set_error(VQG_ERR_UNSUPPORTED, "%s", err.c_str());
    }
    if ((int)pl->hp.size() > n_eslots) {
        n_eslots = (int)pl->hp.size();
        int st = ensure_partials();
        if (st) return st;
    }
    dfree(pl->d_hp);
    dfree(pl->d_hg);
    dfree(pl->d_ht);
    pl->d_hp = nullptr;
    pl->d_hg = nullptr;
    pl->d_ht = nullptr;
    int st;
    if ((st = dalloc((void **)&pl->d_hp, sizeof(HPass) * pl->hp.size()))) return st;
    if ((st = dalloc((void **)&pl->d_hg, sizeof(HGroup) * std::max<size_t>(pl->hg.size(), 1)))) return st;
    if ((st = dalloc((void **)&pl->d_ht, sizeof(HTerm) * std::max<size_t>(pl->ht.size(), 1)))) return st;
    h2d(pl->d_hp, pl->hp.data(), sizeof(HPass) * pl->hp.size());
    if (!pl->hg.empty()) h2d(pl->d_hg, pl->hg.data(), sizeof(HGroup) * pl->hg.size());
    if (!pl->ht.empty()) h2d(pl->d_ht, pl->ht.data(), sizeof(HTerm) * pl->ht.size());
    if (cudaGetLastError() != cudaSuccess) return set_error(VQG_ERR_CUDA, "Hamiltonian plan upload failed");
    ham_plan_ok = true;
    pl->spec_ham.clear();
    pl->spec_ham_for = nullptr;
    if (!dbl && opt.specialize && (st = spec_build_ham(pl))) return st;
    return VQG_OK;
}

void Circuit::free_plan() {
    delete plan;
    plan = nullptr;
}

// Release the plan with its device tables (the circuit's other buffers stay); plans
// derived from its geometry (tensor-product operators) go too.
void Circuit::drop_plan() {
    if (!plan) return;
    release_plan(plan);
    plan = nullptr;
    plan_ok = ham_plan_ok = false;
    drop_product_plans();
}

// Checkpoints of the fused schedule sit at pass boundaries: the output of pass j is
// stored when at least `interval` gates have passed since the previous one (never the
// last pass: its output is psi itself).
std::vector<int> Circuit::fused_checkpoint_passes(int interval) const {
    std::vector<int> want;
    int since = 0;
    for (size_t j = 0; j + 1 < plan->passes.size(); ++j) {
        since += plan->passes[j].n_gates;
        if (since >= interval) want.push_back((int)j), since = 0;
    }
    return want;
}

void Circuit::set_fused_checkpoint(int pass, int k) { plan->ckpt_of_pass[pass] = k; }

int Circuit::issue_forward_fused(bool with_ckpt) {
    Plan *pl = plan;
    const void *mats = dbl ? (const void *)d_mats : (const void *)pl->d_mats_f;
    const void *in = has_input ? d_input : psi;  // pass 0 synthesises |0...0> unless an input is set
    for (size_t j = 0; j < pl->passes.size(); ++j) {
        const int k = with_ckpt ? pl->ckpt_of_pass[j] : -1;
        void *out = k >= 0 ? ckpt_buf[k] : psi;
        // tiles the pass skips need zeros in its output only where a reader takes the whole
        // state: the last pass (psi) and, with diagnostics, every stored checkpoint; the next
        // pass does not read them (FPass::zero_in)
        const bool zero_fill = j + 1 == pl->passes.size() || diag_active;
        const uint64_t n_tiles = zero_fill ? pl->n_tiles : std::min<uint64_t>(pl->n_tiles, 1ull << pl->passes[j].n_active);
        prof_begin(FAM_FWD_FUSED);
        if (j < pl->spec_fwd.size())
            spec_launch_fwd(pl, (int)j, in, out, mats, n_tiles, stream);
        else
            launch_fused_fwd(dbl, float_float(dbl, opt), pl->K, pl->Rf, in, out, pl->d_passes, (int)j, pl->d_stages,
                             pl->d_ops, pl->d_diags, pl->d_items, mats, n_tiles, pl->grid_fwd, stream);
        prof_end();
        if (k >= 0)
            if (int st = diag_reduce(out, nullptr, DIAG_STORE, k)) return st;
        in = out;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "fused forward launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

int Circuit::issue_hamiltonian_fused() {
    Plan *pl = plan;
    for (size_t h = 0; h < pl->hp.size(); ++h) {
        prof_begin(FAM_HAM_FUSED);
        if (!dbl && h < pl->spec_ham.size() && pl->spec_ham_for == pl->d_hp)
            spec_launch_ham(pl, (int)h, psi, lam, d_partials, nb, stream);
        else if (float_float(dbl, opt))
            launch_fused_ham_df(pl->K, psi, lam, pl->d_hp, (int)h, pl->d_hg, pl->d_ht, pl->n_tiles, d_partials, nb,
                                stream);
        else
            launch_fused_ham(dbl, pl->K, psi, lam, pl->d_hp, (int)h, pl->d_hg, pl->d_ht, pl->n_tiles,
                             d_partials, nb, stream);
        prof_end();
    }
    e_used = (int)pl->hp.size();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "fused Hamiltonian launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

int Circuit::issue_reverse_fused() {
    Plan *pl = plan;
    const void *mats = dbl ? (const void *)d_mats : (const void *)pl->d_mats_f;
    double *gpart = d_partials + (size_t)n_eslots * nb;
    for (int j = (int)pl->passes.size() - 1; j >= 0; --j) {
        const int k = pl->ckpt_of_pass[j];
        const void *src = k >= 0 ? ckpt_buf[k] : psi;  // restart phi from the stored state
        if (k >= 0) {
            if (int st = diag_reduce(src, lam, DIAG_RESTART, k)) return st;
            if (int st = diag_reduce(psi, src, DIAG_UNAPPLIED, k)) return st;
        }
        // phi_j is read only if the next reverse pass does not restart from a checkpoint
        // (or diagnostics compare it with that checkpoint); nothing reads phi or lambda
        // after the last reverse pass
        const bool write_phi = j > 0 && (pl->ckpt_of_pass[j - 1] < 0 || diag_active), write_lam = j > 0;
        prof_begin(FAM_ADJ_FUSED);
        const int wmask = (write_phi ? 1 : 0) | (write_lam ? 2 : 0);
        // only the tiles that can hold amplitude (FPass::n_active); all of them when
        // diagnostics follow lambda's norm through the sweep
        const uint64_t n_tiles = diag_active ? pl->n_tiles : std::min<uint64_t>(pl->n_tiles, 1ull << pl->passes[j].n_active);
        if (j < (int)pl->spec_rev.size()) {
            spec_launch_rev(pl, j, src, psi, lam, mats, gpart, nb, wmask, n_tiles, stream);
        } else {
            auto rev = !dbl ? launch_fused_rev_c64 : float_float(dbl, opt) ? launch_fused_rev_df : launch_fused_rev_c128;
            if (!rev(pl->K, pl->Rr, src, psi, lam, pl->d_passes, j, pl->d_stages, pl->d_ops, pl->d_diags,
                     pl->d_items, pl->d_slot_map, mats, n_tiles, gpart, nb, wmask, stream))
                return set_error(VQG_ERR_UNSUPPORTED, "no reverse kernel for K=%d Rr=%d", pl->K, pl->Rr);
        }
        prof_end();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "fused reverse launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

float *Circuit::mats_f() const { return plan ? plan->d_mats_f : nullptr; }

void Circuit::fill_plan_info(vqg_plan_info *info) const {
    const bool fused = opt.fusion && plan_ok;
    info->forward_passes = fused ? (int)plan->passes.size() : G;
    info->hamiltonian_passes = (fused && ham_plan_ok) ? (int)plan->hp.size() : (int)ham.size();
    info->reverse_passes = fused ? (int)plan->passes.size() : G;
    int nck = 0;
    if (fused) {
        for (int k : plan->ckpt_of_pass) nck += k >= 0;
    } else {
        nck = (int)ckpt_pos.size();
    }
    info->checkpoints = nck;
    info->tile_qubits = fused ? plan->K : 0;
    info->specialized = !fused || plan->spec_fwd.empty() ? 0 : (plan->spec_rev.empty() ? 1 : 2);
    info->fwd_reg_qubits = fused ? plan->Rf : 0;
    info->rev_reg_qubits = fused ? plan->Rr : 0;
    info->hamiltonian_groups = (int)ham.size();
    info->launches_per_gradient = 1 + info->forward_passes + info->hamiltonian_passes + info->reverse_passes + 2 +
                                  (fused ? 0 : 1 + nck);
    info->dense_gates = G;
    if (fused) {
        info->dense_gates = 0;
        for (const FPass &p : plan->passes) info->dense_gates += p.n_active == p.n_nontile ? p.n_gates : 0;
    }
}

// Group Pauli terms by flip mask x (one pass over pairs (j, j^x) serves a group);
// each term keeps its z mask and w = coef * i^{popcount(x & z)}.  The diagonal group
// (x = 0) always exists and comes first.
int group_pauli_terms(int n, int n_terms, const uint64_t *x_mask, const uint64_t *z_mask,
                      const double *coef, std::vector<HamGroup> &ham, std::vector<PauliTerm> &flat) {
    if (n_terms < 0 || (n_terms > 0 && (!x_mask || !z_mask || !coef)))
        return set_error(VQG_ERR_INVALID, "bad Hamiltonian arrays");
    const uint64_t lim = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    std::map<uint64_t, std::vector<PauliTerm>> groups;
    groups[0];
    for (int t = 0; t < n_terms; ++t) {
        if ((x_mask[t] & ~lim) || (z_mask[t] & ~lim))
            return set_error(VQG_ERR_INVALID, "term %d: mask has bits >= n", t);
        if (!std::isfinite(coef[t])) return set_error(VQG_ERR_INVALID, "term %d: coefficient not finite", t);
        const int ny = __builtin_popcountll(x_mask[t] & z_mask[t]) & 3;
        PauliTerm p;
        p.z = z_mask[t];
        p.wr = (ny == 0) ? coef[t] : (ny == 2 ? -coef[t] : 0.0);
        p.wi = (ny == 1) ? coef[t] : (ny == 3 ? -coef[t] : 0.0);
        groups[x_mask[t]].push_back(p);
    }
    ham.clear();
    flat.clear();
    for (auto &kv : groups) {
        HamGroup g;
        g.x = kv.first;
        g.first = (int)flat.size();
        g.count = (int)kv.second.size();
        flat.insert(flat.end(), kv.second.begin(), kv.second.end());
        ham.push_back(g);
    }
    return VQG_OK;
}

}  // namespace vqg

// One fused pass of the schedule: gates, stages and computed tiles (include/vqg.h).
extern "C" int vqg_plan_pass(vqg_circuit *c, int pass, vqg_pass_info *info, int max_gates, int32_t *gates) {
    if (!c) return vqg::set_error(VQG_ERR_INVALID, "circuit is NULL");
    const vqg::Circuit *cc = reinterpret_cast<const vqg::Circuit *>(c);
    if (!info || max_gates < 0) return vqg::set_error(VQG_ERR_INVALID, "info is NULL or max_gates < 0");
    const vqg::Plan *pl = cc->plan;
    if (!pl || !cc->plan_ok) return vqg::set_error(VQG_ERR_STATE, "the circuit has no fused schedule");
    if (pass < 0 || pass >= (int)pl->passes.size())
        return vqg::set_error(VQG_ERR_INVALID, "pass %d outside 0..%d", pass, (int)pl->passes.size() - 1);
    const vqg::FPass &P = pl->passes[pass];
    std::memset(info, 0, sizeof *info);
    info->n_gates = P.n_gates;
    info->forward_stages = P.n_stage;
    info->reverse_stages = P.n_rstage;
    info->from_zero = P.from_zero;
    info->tiles = pl->n_tiles;
    info->active_tiles = std::min<uint64_t>(pl->n_tiles, 1ull << P.n_active);
    info->tile_mask = (1ull << pl->L) - 1ull;
    for (int i = 0; i < P.n_high; ++i) info->tile_mask |= 1ull << P.high[i];
    const std::vector<int32_t> &g = pl->pass_gates[pass];
    if (gates)
        for (int i = 0; i < std::min(max_gates, (int)g.size()); ++i) gates[i] = g[i];
    return VQG_OK;
}

// Host-only planning of a circuit and Hamiltonian: the same schedule a vqg_circuit
// would use, validated, without touching a GPU.
extern "C" int vqg_plan_dry_run(int n_qubits, const vqg_gate *gates, int n_gates, int n_params, int dtype,
                                const vqg_options *opt_in, int n_terms, const uint64_t *x_mask,
                                const uint64_t *z_mask, const double *coef, vqg_plan_info *info) {
    using namespace vqg;
    if (!info) return set_error(VQG_ERR_INVALID, "info is NULL");
    std::memset(info, 0, sizeof *info);
    int st = vqg_validate_circuit(n_qubits, gates, n_gates, n_params, dtype);
    if (st) return st;
    vqg_options opt;
    vqg_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.c128_arith != VQG_C128_FP64 && opt.c128_arith != VQG_C128_FLOAT_FLOAT)
        return set_error(VQG_ERR_INVALID, "c128_arith %d is not a vqg_c128_arith", opt.c128_arith);
    const bool dbl = dtype == VQG_C128;
    std::vector<vqg_gate> gv(gates, gates + n_gates);
    std::vector<int> slot_base(std::max(n_gates, 1), 0);
    int n_gslots = 0;
    for (int i = 0; i < n_gates; ++i) {
        slot_base[i] = n_gslots;
        n_gslots += red_values(gv[i].kind);
    }
    std::vector<HamGroup> ham;
    std::vector<PauliTerm> flat;
    if ((st = group_pauli_terms(n_qubits, n_terms, x_mask, z_mask, coef, ham, flat))) return st;
    std::string err;
    Plan *pl = plan_gates(n_qubits, gv, slot_base, n_gslots, dbl, opt, err);
    if (!pl) {
        if (!err.empty()) return set_error(VQG_ERR_UNSUPPORTED, "%s", err.c_str());
        info->forward_passes = n_gates;
        info->reverse_passes = n_gates;
        info->hamiltonian_passes = (int)ham.size();
        info->hamiltonian_groups = (int)ham.size();
        return VQG_OK;
    }
    const bool ham_fused = plan_hamiltonian(pl, n_qubits, ham, flat);
    err = validate_plan(*pl, n_qubits, n_gslots, dbl);
    if (!err.empty()) {
        delete pl;
        return set_error(VQG_ERR_UNSUPPORTED, "%s", err.c_str());
    }
    info->forward_passes = (int)pl->passes.size();
    info->reverse_passes = (int)pl->passes.size();
    info->hamiltonian_passes = ham_fused ? (int)pl->hp.size() : (int)ham.size();
    info->hamiltonian_groups = (int)ham.size();
    info->tile_qubits = pl->K;
    info->fwd_reg_qubits = pl->Rf;
    info->rev_reg_qubits = pl->Rr;
    int fs = 0, rs = 0, fd = 0, rd = 0;
    for (const FPass &p : pl->passes) fs += p.n_stage, rs += p.n_rstage, fd += p.n_diag, rd += p.n_rdiag;
    info->forward_stages = fs;
    info->reverse_stages = rs;
    info->stage_ops = (int)pl->ops.size();  // register-stage ops, both directions
    info->diag_blocks = fd + rd;            // diagonal blocks, both directions
    info->launches_per_gradient = 1 + 2 * info->forward_passes + info->hamiltonian_passes + 2;
    for (const FPass &p : pl->passes) info->dense_gates += p.n_active_zero == p.n_nontile ? p.n_gates : 0;
    delete pl;
    return VQG_OK;
}
