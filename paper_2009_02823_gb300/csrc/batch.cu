// Batched launch: many independent circuits (energy + full gradient each) in one
// persistent kernel.
//
// Every circuit is planned with the same tile geometry (complex64; K = 12 tile qubits
// with 4 register qubits, or K = 11 with 3, both 256 threads; vqg_batch_autotune times
// both), with a smaller shared-memory program than the single-circuit kernels so that
// two or three blocks stay resident per SM, and all plans are concatenated.  A task is
// (circuit, phase, chunk of tiles); the phases of a circuit are its forward passes,
// its Hamiltonian passes, its reverse passes (last pass first) and a finalize step.
// Tasks sit in one queue ordered by phase level, and resident blocks claim them with an
// atomic counter.  A task waits only for the earlier phases of its own circuit, whose
// tasks come earlier in the queue and were therefore claimed by running blocks; the
// wait is bounded (spin limit, then an error flag the host reads as VQG_ERR_TIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/vqg.h"
#include "fused_kernels.cuh"
#include "grad.cuh"
#include "plan.h"

namespace vqg {

constexpr int kBNT = 256;         // threads per block in every phase: 2^(K - R)
constexpr int kBatchMinQubits = 12;
// Compiled tile geometries (tile qubits K, register qubits R) of the batched kernel.
constexpr int kBatchGeom[2][2] = {{12, 4}, {11, 3}};

struct BCirc {
    uint64_t psi_off, lam_off;  // amplitude offsets into the state arena
    int32_t pass0, n_pass, hpass0, n_hpass;
    int32_t gate0, n_gates, param0, n_params;
    int32_t occ_ptr0, n_gslots, part0, chunks, tch;
    int32_t n_tiles, pad;
};

struct BTask {
    int32_t circ, phase, chunk, pad;
};

struct BatchArgs {
    float2 *arena;
    const BCirc *circs;
    const BTask *tasks;
    int n_tasks;
    int *head;
    unsigned long long *done;
    int *err;
    long long spin_limit;
    int stall_circ;
    const FPass *passes;
    const FStage *stages;
    const FOp *ops;
    const FDiag *diags;
    const FDItem *items;
    const int *slot_map;
    const HPass *hp;
    const HGroup *hg;
    const HTerm *ht;
    const float *mats;
    const double *theta;
    const DevGate *gates;
    const int *slot_base;
    const int *occ_ptr;
    const Occurrence *occ;
    double *partials;
    double *energy;
    double *grad;
};

template <typename T, int K, int R>
struct BatchCfg {
    using FC = FwdCfg<T, K, R, BatchCaps>;
    using RC = RevCfg<T, K, R, BatchCaps>;
    using HC = HamCfg<T, K>;
    static constexpr size_t smem() {
        size_t m = FC::smem();
        m = RC::smem() > m ? RC::smem() : m;
        m = HC::smem() > m ? HC::smem() : m;
        return m;
    }
};

// Bounded wait for a counter (done chunks of a circuit) to reach `need`.
VQG_DEV bool wait_count(const unsigned long long *cnt, unsigned long long need, long long limit) {
    long long spins = 0;
    while (*(volatile const unsigned long long *)cnt < need) {
        if (++spins > limit) return false;
        __nanosleep(200);
    }
    __threadfence();
    return true;
}

template <typename T, int K, int R>
__global__ void __launch_bounds__(kBNT) k_batch(BatchArgs a) {
    using A = amp_t<T>;
    using FC = typename BatchCfg<T, K, R>::FC;
    using RC = typename BatchCfg<T, K, R>::RC;
    using HC = HamCfg<T, K>;
    static_assert((1 << (K - R)) == kBNT, "one block size for every phase");
    constexpr int NW = kBNT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_task, s_ok;
    __shared__ double wsum[NW];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(a.head, 1);
            s_task = t;
            s_ok = 1;
            if (t < a.n_tasks) {
                const BTask tk = a.tasks[t];
                const BCirc C = a.circs[tk.circ];
                unsigned long long need = (unsigned long long)tk.phase * (unsigned long long)C.chunks;
                if (tk.circ == a.stall_circ && tk.phase >= 1) need = ULLONG_MAX;  // test hook: never met
                if (!wait_count(a.done + tk.circ, need, a.spin_limit)) {
                    atomicExch(a.err, 1);
                    s_ok = 0;
                }
            }
        }
        __syncthreads();
        const int t = s_task;
        const bool ok = s_ok != 0;
        if (t >= a.n_tasks) break;
        const BTask tk = a.tasks[t];
        const BCirc C = a.circs[tk.circ];
        A *psi = reinterpret_cast<A *>(a.arena) + C.psi_off;
        A *lam = reinterpret_cast<A *>(a.arena) + C.lam_off;
        const int F = C.n_pass, H = C.n_hpass;
        const int t0 = tk.chunk * C.tch, t1 = min(C.n_tiles, t0 + C.tch);
        double *part = a.partials + C.part0;
        if (ok && tk.phase < F) {  // forward pass
            const FPass &P = a.passes[C.pass0 + tk.phase];
            A *tile = reinterpret_cast<A *>(smem);
            uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + FC::o_row);
            Prog<T, R> pg;
            pg.template bind<BatchCaps>(smem + FC::o_prog);
            fill_row_offsets<T, K>(P.high, row_off, tid, kBNT);
            load_prog<T, R>(pg, P.stage0, P.n_stage, P.diag0, P.n_diag, a.stages, a.ops, a.diags, a.items,
                            a.mats, false, tid, kBNT);
            __syncthreads();
            // tiles a |0...0> start leaves at zero (FPass::n_active) are skipped; only the last
            // pass writes their zeros (the Hamiltonian reads the whole state), the others'
            // inputs are not read there (FPass::zero_in)
            const int n_act = (int)min((unsigned long long)C.n_tiles, 1ull << P.n_active);
            const bool last = tk.phase == F - 1;
            for (int ti = t0; ti < t1; ++ti) {
                if (ti >= n_act) {
                    if (last)
                        TileIO<T, K>::template store_zero<kBNT>(psi, tile_base(ti, P.nontile, P.n_nontile), row_off, tid);
                    continue;
                }
                if (ti + 1 < min(t1, n_act) && !P.from_zero)
                    TileIO<T, K>::template prefetch<kBNT>(psi, tile_base(ti + 1, P.nontile, P.n_nontile), row_off, tid,
                                                          P.zero_in);
                fwd_tile<T, K, R, true>(tile, row_off, pg, P.n_stage, tile_base(ti, P.nontile, P.n_nontile),
                                        P.from_zero != 0, psi, psi, tid, P.zero_in);
            }
        } else if (ok && tk.phase < F + H) {  // Hamiltonian pass
            const HPass &P = a.hp[C.hpass0 + tk.phase - F];
            A *tile = reinterpret_cast<A *>(smem);
            uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + HC::o_row);
            HamTab<T, K> tb;
            tb.bind(smem + HC::o_tab);
            fill_row_offsets<T, K>(P.high, row_off, tid, kBNT);
            using G = HamGeo<T, K>;
            tb.template load<G::D, G::SH, G::E0>(P, a.hg, a.ht, tid, kBNT);
            __syncthreads();
            double eacc = 0.0;
            for (int ti = t0; ti < t1; ++ti) {
                if (ti + 1 < t1) {
                    const uint64_t next = tile_base(ti + 1, P.nontile, P.n_nontile);
                    TileIO<T, K>::template prefetch<kBNT>(psi, next, row_off, tid);
                    if (!P.first) TileIO<T, K>::template prefetch<kBNT>(lam, next, row_off, tid);
                }
                const T run = ham_tile<T, K, true>(tile, row_off, tb, tile_base(ti, P.nontile, P.n_nontile),
                                                   P.first != 0, psi, lam, tid);
                eacc += (double)warp_tree<T>(run);
            }
            if ((tid & 31) == 0) wsum[warp] = eacc;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < NW; ++w) s += wsum[w];
                part[(size_t)(tk.phase - F) * C.chunks + tk.chunk] = s;
            }
        } else if (ok && tk.phase < 2 * F + H) {  // reverse pass, last pass first
            const FPass &P = a.passes[C.pass0 + (F - 1 - (tk.phase - F - H))];
            A *tphi = reinterpret_cast<A *>(smem);
            A *tlam = tphi + (1 << K);
            uint64_t *row_off = reinterpret_cast<uint64_t *>(smem + RC::o_row);
            Prog<T, R> pg;
            pg.template bind<BatchCaps>(smem + RC::o_prog);
            double *acc = reinterpret_cast<double *>(smem + RC::o_acc);
            T *stash = reinterpret_cast<T *>(smem + RC::o_stash);
            int *smap = reinterpret_cast<int *>(smem + RC::o_map);
            const int n_ls = P.n_lslots;
            fill_row_offsets<T, K>(P.high, row_off, tid, kBNT);
            for (int i = tid; i < n_ls; i += kBNT) acc[i] = 0.0, smap[i] = a.slot_map[P.slotmap0 + i];
            load_prog<T, R>(pg, P.rstage0, P.n_rstage, P.rdiag0, P.n_rdiag, a.stages, a.ops, a.diags, a.items,
                            a.mats, true, tid, kBNT);
            __syncthreads();
            // only the tiles that can hold amplitude (FPass::n_active)
            const int t1a = min(t1, (int)min((unsigned long long)C.n_tiles, 1ull << P.n_active));
            for (int ti = t0; ti < t1a; ++ti) {
                if (ti + 1 < t1a) {
                    const uint64_t next = tile_base(ti + 1, P.nontile, P.n_nontile);
                    TileIO<T, K>::template prefetch<kBNT>(psi, next, row_off, tid);
                    TileIO<T, K>::template prefetch<kBNT>(lam, next, row_off, tid);
                }
                rev_tile<T, K, R, true>(tphi, tlam, row_off, pg, P.n_rstage, tile_base(ti, P.nontile, P.n_nontile),
                                        psi, psi, lam, acc, stash, tid);
            }
            __syncthreads();
            for (int i = tid; i < n_ls; i += kBNT) part[(size_t)(H + smap[i]) * C.chunks + tk.chunk] = acc[i];
        } else if (ok) {  // finalize: E and the gradient of this circuit (fixed-order sums)
            if (tid == 0) {
                double e = 0.0;
                for (int h = 0; h < H; ++h)
                    for (int c = 0; c < C.chunks; ++c) e += __ldcg(part + (size_t)h * C.chunks + c);
                a.energy[tk.circ] = e;
            }
            for (int p = tid; p < C.n_params; p += kBNT) {
                double g = 0.0;
                const int *op = a.occ_ptr + C.occ_ptr0;
                for (int k = op[p]; k < op[p + 1]; ++k) {
                    const Occurrence o = a.occ[k];
                    const DevGate gt = a.gates[C.gate0 + o.gate];
                    const int sb = a.slot_base[C.gate0 + o.gate];
                    double v[8];
                    const int nv = gt.kind == K_U3 ? 8 : 1;
                    for (int x = 0; x < nv; ++x) {
                        double s = 0.0;
                        for (int c = 0; c < C.chunks; ++c) s += __ldcg(part + (size_t)(H + sb + x) * C.chunks + c);
                        v[x] = s;
                    }
                    if (gt.kind == K_U3) {
                        const double ang[3] = {a.theta[gt.p0], a.theta[gt.p1], a.theta[gt.p2]};
                        g += u3_slot_contribution(ang, o.slot, v);
                    } else {
                        g += v[0];
                    }
                }
                a.grad[C.param0 + p] = g;
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0 && ok) atomicAdd(a.done + tk.circ, 1ull);
    }
}

}  // namespace vqg

using namespace vqg;

struct BatchCircuit {
    int n = 0, P = 0;
    std::vector<vqg_gate> gates;
    std::vector<HamGroup> ham;
    std::vector<PauliTerm> terms;
    bool has_ham = false;
    std::vector<int> slot_base;
    int n_gslots = 0;
};

struct vqg_batch {
    int dtype = VQG_C64;
    std::vector<BatchCircuit> c;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1, grid = 1, n_tasks = 0, total_params = 0, total_gates = 0;
    int bk = kBatchGeom[0][0], br = kBatchGeom[0][1];  // tile geometry
    bool built = false;
    long long spin_limit = 1ll << 26;
    int stall_circ = -1;
    std::vector<void *> allocs;
    BatchArgs args{};
    double *d_theta = nullptr, *d_out = nullptr, *h_pinned = nullptr;
    DevGate *d_gates = nullptr;
    double *d_mats = nullptr;
    float *d_mats_f = nullptr;
    cudaGraphExec_t graph = nullptr;
    const void *graph_key[3] = {nullptr, nullptr, nullptr};
    bool graph_warm = false;
    size_t smem = 0;

    int dalloc(void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return set_error(VQG_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
        allocs.push_back(*p);
        return VQG_OK;
    }
    template <typename X>
    int upload(X **d, const std::vector<X> &h) {
        int st = dalloc((void **)d, sizeof(X) * std::max<size_t>(h.size(), 1));
        if (st) return st;
        if (!h.empty() && h2d(*d, h.data(), sizeof(X) * h.size()) != cudaSuccess)
            return set_error(VQG_ERR_CUDA, "batch upload failed");
        return VQG_OK;
    }
    // Release everything build() made (plans, tables, state arena, graph).
    void reset() {
        if (stream) cudaStreamSynchronize(stream);
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        graph_warm = false;
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        if (h_pinned) cudaFreeHost(h_pinned);
        h_pinned = nullptr;
        built = false;
    }
    ~vqg_batch() {
        reset();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
    int build();
    int autotune(const double *theta, vqg_tune_result *out);
    int issue(const double *theta_dev, double *energy_dev, double *grad_dev);
    int run(const double *theta_dev, double *energy_dev, double *grad_dev);
};

int vqg_batch::build() {
    if (built) return VQG_OK;
    vqg_options opt;
    vqg_default_options(&opt);
    opt.tile_qubits = bk;
    opt.fwd_reg_qubits = br;
    opt.rev_reg_qubits = br;
    std::vector<FPass> passes;
    std::vector<FStage> stages;
    std::vector<FOp> ops;
    std::vector<FDiag> diags;
    std::vector<FDItem> items;
    std::vector<int> slot_map, slot_base, occ_ptr;
    std::vector<Occurrence> occ;
    std::vector<HPass> hps;
    std::vector<HGroup> hgs;
    std::vector<HTerm> hts;
    std::vector<DevGate> dgates;
    std::vector<BCirc> circs(c.size());
    uint64_t arena = 0;
    size_t part = 0;
    int gate0 = 0, param0 = 0;
    std::vector<int> n_phase(c.size());
    for (size_t b = 0; b < c.size(); ++b) {
        BatchCircuit &bc = c[b];
        if (!bc.has_ham) return set_error(VQG_ERR_STATE, "circuit %zu of the batch has no Hamiltonian", b);
        std::string err;
        Plan *pl = plan_gates(bc.n, bc.gates, bc.slot_base, bc.n_gslots, false, opt, err, BatchCaps::value(), false);
        if (!pl) return set_error(VQG_ERR_UNSUPPORTED, "batch circuit %zu: %s", b, err.empty() ? "no fused plan" : err.c_str());
        if (!plan_hamiltonian(pl, bc.n, bc.ham, bc.terms)) {
            delete pl;
            return set_error(VQG_ERR_UNSUPPORTED, "batch circuit %zu: a Pauli group does not fit one tile", b);
        }
        err = validate_plan(*pl, bc.n, bc.n_gslots, false);
        if (!err.empty()) {
            delete pl;
            return set_error(VQG_ERR_UNSUPPORTED, "batch circuit %zu: %s", b, err.c_str());
        }
        BCirc C;
        std::memset(&C, 0, sizeof C);
        const int st0 = (int)stages.size(), op0 = (int)ops.size(), dg0 = (int)diags.size();
        const int it0 = (int)items.size(), sm0 = (int)slot_map.size(), hg0 = (int)hgs.size(), ht0 = (int)hts.size();
        C.pass0 = (int)passes.size();
        C.n_pass = (int)pl->passes.size();
        for (FPass p : pl->passes) {
            p.stage0 += st0;
            p.rstage0 += st0;
            p.diag0 += dg0;
            p.rdiag0 += dg0;
            p.slotmap0 += sm0;
            passes.push_back(p);
        }
        for (FStage s : pl->stages) s.op0 += op0, stages.push_back(s);
        for (FOp o : pl->ops) {
            if (o.gate >= 0) o.gate += gate0;
            ops.push_back(o);
        }
        for (FDiag d : pl->diags) d.item0 += it0, diags.push_back(d);
        for (FDItem x : pl->items) {
            if (x.type == DI_RZ_REG || x.type == DI_RZ_THR) x.gate += gate0;
            items.push_back(x);
        }
        slot_map.insert(slot_map.end(), pl->slot_map.begin(), pl->slot_map.end());
        C.hpass0 = (int)hps.size();
        C.n_hpass = (int)pl->hp.size();
        for (HPass h : pl->hp) h.group0 += hg0, hps.push_back(h);
        for (HGroup g : pl->hg) g.term0 += ht0, hgs.push_back(g);
        hts.insert(hts.end(), pl->ht.begin(), pl->ht.end());
        C.gate0 = gate0;
        C.n_gates = (int)bc.gates.size();
        C.param0 = param0;
        C.n_params = bc.P;
        for (const vqg_gate &g : bc.gates)
            dgates.push_back({g.kind, g.q0, g.q1, g.param[0] >= 0 ? g.param[0] + param0 : -1,
                              g.param[1] >= 0 ? g.param[1] + param0 : -1, g.param[2] >= 0 ? g.param[2] + param0 : -1});
        slot_base.insert(slot_base.end(), bc.slot_base.begin(), bc.slot_base.begin() + bc.gates.size());
        // occurrences (App. B.2 chain-rule sum), per circuit
        std::vector<std::vector<Occurrence>> by(bc.P);
        for (int i = 0; i < (int)bc.gates.size(); ++i) {
            const int k = params_of(bc.gates[i].kind);
            for (int j = 0; j < k; ++j) by[bc.gates[i].param[j]].push_back({i, j});
        }
        C.occ_ptr0 = (int)occ_ptr.size();
        for (int p = 0; p < bc.P; ++p) {
            occ_ptr.push_back((int)occ.size());
            occ.insert(occ.end(), by[p].begin(), by[p].end());
        }
        occ_ptr.push_back((int)occ.size());
        C.n_gslots = bc.n_gslots;
        C.n_tiles = 1 << (bc.n - bk);
        const int chunks = std::min(C.n_tiles, 32);
        C.tch = (C.n_tiles + chunks - 1) / chunks;
        C.chunks = (C.n_tiles + C.tch - 1) / C.tch;
        C.part0 = (int)part;
        part += (size_t)(C.n_hpass + C.n_gslots) * C.chunks;
        C.psi_off = arena;
        arena += 1ull << bc.n;
        C.lam_off = arena;
        arena += 1ull << bc.n;
        circs[b] = C;
        n_phase[b] = 2 * C.n_pass + C.n_hpass + 1;
        gate0 += (int)bc.gates.size();
        param0 += bc.P;
        delete pl;
    }
    total_gates = gate0;
    total_params = param0;
    // task queue: phase level by level, circuits with more work first inside a level
    std::vector<int> order(c.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const double wx = (double)(1ull << c[x].n) * c[x].gates.size(), wy = (double)(1ull << c[y].n) * c[y].gates.size();
        return wx > wy;
    });
    std::vector<BTask> tasks;
    const int max_phase = *std::max_element(n_phase.begin(), n_phase.end());
    for (int lv = 0; lv < max_phase; ++lv)
        for (int b : order) {
            if (lv >= n_phase[b]) continue;
            const int nchunk = lv == n_phase[b] - 1 ? 1 : circs[b].chunks;
            for (int ch = 0; ch < nchunk; ++ch) tasks.push_back({b, lv, ch, 0});
        }
    // a finalize task waits for all chunks of the earlier phases: phase * chunks counts them
    n_tasks = (int)tasks.size();
    int st;
    BatchArgs &A = args;
    std::memset(&A, 0, sizeof A);
    if ((st = dalloc((void **)&A.arena, sizeof(float2) * std::max<uint64_t>(arena, 1)))) return st;
    if ((st = upload((BCirc **)&A.circs, circs))) return st;
    if ((st = upload((BTask **)&A.tasks, tasks))) return st;
    A.n_tasks = n_tasks;
    if ((st = dalloc((void **)&A.head, sizeof(int)))) return st;
    if ((st = dalloc((void **)&A.done, sizeof(unsigned long long) * c.size()))) return st;
    if ((st = dalloc((void **)&A.err, sizeof(int)))) return st;
    if ((st = upload((FPass **)&A.passes, passes))) return st;
    if ((st = upload((FStage **)&A.stages, stages))) return st;
    if ((st = upload((FOp **)&A.ops, ops))) return st;
    if ((st = upload((FDiag **)&A.diags, diags))) return st;
    if ((st = upload((FDItem **)&A.items, items))) return st;
    if ((st = upload((int **)&A.slot_map, slot_map))) return st;
    if ((st = upload((HPass **)&A.hp, hps))) return st;
    if ((st = upload((HGroup **)&A.hg, hgs))) return st;
    if ((st = upload((HTerm **)&A.ht, hts))) return st;
    if ((st = upload(&d_gates, dgates))) return st;
    A.gates = d_gates;
    if ((st = upload((int **)&A.slot_base, slot_base))) return st;
    if ((st = upload((int **)&A.occ_ptr, occ_ptr))) return st;
    if ((st = upload((Occurrence **)&A.occ, occ))) return st;
    if ((st = dalloc((void **)&A.partials, sizeof(double) * std::max<size_t>(part, 1)))) return st;
    if ((st = dalloc((void **)&d_mats, sizeof(double) * 8 * std::max(gate0, 1)))) return st;
    if ((st = dalloc((void **)&d_mats_f, sizeof(float) * 8 * std::max(gate0, 1)))) return st;
    A.mats = d_mats_f;
    if ((st = dalloc((void **)&d_theta, sizeof(double) * std::max(param0, 1)))) return st;
    if ((st = dalloc((void **)&d_out, sizeof(double) * (c.size() + param0)))) return st;
    if (cudaMallocHost((void **)&h_pinned, sizeof(double) * (c.size() + 2 * (size_t)param0 + 1)) != cudaSuccess)
        return set_error(VQG_ERR_OOM, "pinned staging allocation failed");
    const bool g12 = bk == 12;
    smem = g12 ? BatchCfg<float, 12, 4>::smem() : BatchCfg<float, 11, 3>::smem();
    const void *fn = g12 ? (const void *)k_batch<float, 12, 4> : (const void *)k_batch<float, 11, 3>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBNT, smem);
    grid = num_sms * std::max(per_sm, 1);  // all blocks resident: waits only on running blocks
    built = true;
    return VQG_OK;
}

int vqg_batch::issue(const double *theta_dev, double *energy_dev, double *grad_dev) {
    BatchArgs A = args;
    A.theta = theta_dev;
    A.energy = energy_dev;
    A.grad = grad_dev;
    A.spin_limit = spin_limit;
    A.stall_circ = stall_circ;
    cudaMemsetAsync(A.head, 0, sizeof(int), stream);
    cudaMemsetAsync(A.done, 0, sizeof(unsigned long long) * c.size(), stream);
    cudaMemsetAsync(A.err, 0, sizeof(int), stream);
    launch_build_mats(theta_dev, d_gates, total_gates, d_mats, d_mats_f, -1, -1, 0.0, stream);
    if (bk == 12) k_batch<float, 12, 4><<<grid, kBNT, smem, stream>>>(A);
    else k_batch<float, 11, 3><<<grid, kBNT, smem, stream>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

// The launch sequence (flag resets, gate tables, the persistent kernel) is captured in a
// CUDA graph per set of argument pointers after one eager warm-up call.
int vqg_batch::run(const double *theta_dev, double *energy_dev, double *grad_dev) {
    int st = build();
    if (st) return st;
    const bool graphable = stream != nullptr && stream != cudaStreamLegacy && stall_circ < 0;
    if (!graphable) return issue(theta_dev, energy_dev, grad_dev);
    const void *key[3] = {theta_dev, energy_dev, grad_dev};
    if (graph && std::memcmp(key, graph_key, sizeof key) != 0) {
        cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
    if (!graph) {
        if (!graph_warm) {
            graph_warm = true;
            return issue(theta_dev, energy_dev, grad_dev);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
        st = issue(theta_dev, energy_dev, grad_dev);
        e = cudaStreamEndCapture(stream, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            graph = nullptr;
            return set_error(VQG_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
        }
        std::memcpy(graph_key, key, sizeof key);
    }
    cudaError_t e = cudaGraphLaunch(graph, stream);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "batch graph launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

// Time one evaluation of the whole batch under each compiled tile geometry and keep the
// fastest (the choice depends on the mix of circuit sizes and depths).
int vqg_batch::autotune(const double *theta, vqg_tune_result *out) {
    vqg_tune_result r;
    std::memset(&r, 0, sizeof r);
    double best = 1e300;
    int bi = 0;
    const int n_geom = (int)(sizeof kBatchGeom / sizeof kBatchGeom[0]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(VQG_ERR_CUDA, "batch autotune: event creation failed");
    int st = VQG_OK;
    for (int gi = 0; gi < n_geom && !st; ++gi) {
        reset();
        bk = kBatchGeom[gi][0];
        br = kBatchGeom[gi][1];
        if ((st = build())) break;
        const int P = total_params, nc = (int)c.size();
        if (theta) std::memcpy(h_pinned, theta, sizeof(double) * P);
        else std::memset(h_pinned, 0, sizeof(double) * P);
        cudaMemcpyAsync(d_theta, h_pinned, sizeof(double) * P, cudaMemcpyHostToDevice, stream);
        if ((st = issue(d_theta, d_out, d_out + nc))) break;  // warm-up
        cudaEventRecord(e0, stream);
        if ((st = issue(d_theta, d_out, d_out + nc))) break;
        cudaEventRecord(e1, stream);
        int errflag = 0;
        cudaMemcpyAsync(h_pinned + P, args.err, sizeof(int), cudaMemcpyDeviceToHost, stream);
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            st = set_error(VQG_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(e));
            break;
        }
        std::memcpy(&errflag, h_pinned + P, sizeof(int));
        if (errflag) {
            st = set_error(VQG_ERR_TIMEOUT, "a batched task gave up waiting for its circuit's previous phase");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ++r.candidates;
        if (gi == 0) r.default_ms = ms;
        if (ms < best) best = ms, bi = gi;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (bk != kBatchGeom[bi][0]) {
        reset();
        bk = kBatchGeom[bi][0];
        br = kBatchGeom[bi][1];
        if ((st = build())) return st;
    }
    r.tile_qubits = bk;
    r.fwd_reg_qubits = r.rev_reg_qubits = br;
    r.best_ms = best;
    if (out) *out = r;
    return VQG_OK;
}

extern "C" int vqg_batch_create(int n_circuits, const int *n_qubits, const vqg_gate *gates,
                                const int *gate_offsets, const int *n_params, int dtype, vqg_batch **out) {
    if (!out) return set_error(VQG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n_circuits < 1 || !n_qubits || !gate_offsets || !n_params)
        return set_error(VQG_ERR_INVALID, "bad batch arguments");
    if (dtype != VQG_C64) return set_error(VQG_ERR_UNSUPPORTED, "the batched launch runs complex64 circuits");
    if (gate_offsets[0] != 0) return set_error(VQG_ERR_INVALID, "gate_offsets[0] must be 0");
    for (int b = 0; b < n_circuits; ++b) {
        const int G = gate_offsets[b + 1] - gate_offsets[b];
        if (G < 1) return set_error(VQG_ERR_INVALID, "circuit %d: no gates", b);
        if (n_qubits[b] < kBatchMinQubits || n_qubits[b] > 30)
            return set_error(VQG_ERR_INVALID, "circuit %d: n_qubits=%d outside %d..30", b, n_qubits[b],
                             kBatchMinQubits);
        const int st = vqg_validate_circuit(n_qubits[b], gates + gate_offsets[b], G, n_params[b], dtype);
        if (st) return st;
    }
    vqg_batch *B = new (std::nothrow) vqg_batch();
    if (!B) return set_error(VQG_ERR_OOM, "host allocation failed");
    B->c.resize(n_circuits);
    for (int b = 0; b < n_circuits; ++b) {
        BatchCircuit &bc = B->c[b];
        bc.n = n_qubits[b];
        bc.P = n_params[b];
        bc.gates.assign(gates + gate_offsets[b], gates + gate_offsets[b + 1]);
        bc.slot_base.assign(bc.gates.size() + 1, 0);
        for (size_t i = 0; i < bc.gates.size(); ++i) {
            bc.slot_base[i] = bc.n_gslots;
            bc.n_gslots += reduce_values_of(bc.gates[i].kind);
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete B;
        return set_error(VQG_ERR_CUDA, "batch create: %s", cudaGetErrorString(e));
    }
    B->own_stream = true;
    *out = B;
    return VQG_OK;
}

extern "C" int vqg_batch_destroy(vqg_batch *b) {
    if (!b) return VQG_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    delete b;
    return VQG_OK;
}

extern "C" int vqg_batch_set_hamiltonian(vqg_batch *b, int circuit, int n_terms, const uint64_t *x_mask,
                                         const uint64_t *z_mask, const double *coef) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    if (circuit < 0 || circuit >= (int)b->c.size()) return set_error(VQG_ERR_INVALID, "circuit %d", circuit);
    if (b->built) return set_error(VQG_ERR_STATE, "Hamiltonians are fixed once the batch has run");
    BatchCircuit &bc = b->c[circuit];
    int st = group_pauli_terms(bc.n, n_terms, x_mask, z_mask, coef, bc.ham, bc.terms);
    if (st) return st;
    bc.has_ham = true;
    return VQG_OK;
}

extern "C" int vqg_batch_set_stream(vqg_batch *b, void *stream) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    if (stream) {
        if (b->own_stream) {
            cudaStreamSynchronize(b->stream);
            cudaStreamDestroy(b->stream);
        }
        b->stream = (cudaStream_t)stream;
        b->own_stream = false;
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return VQG_OK;
}

extern "C" int vqg_batch_set_wait_limit(vqg_batch *b, long long spins, int stall_circuit) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    if (spins < 1) return set_error(VQG_ERR_INVALID, "spins must be positive");
    b->spin_limit = spins;
    b->stall_circ = stall_circuit;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    return VQG_OK;
}

extern "C" int vqg_batch_energy_and_gradient_device(vqg_batch *b, const double *theta_dev,
                                                    double *energies_dev, double *grads_dev) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    if (!theta_dev || !energies_dev || !grads_dev) return set_error(VQG_ERR_INVALID, "null pointer");
    return b->run(theta_dev, energies_dev, grads_dev);
}

extern "C" int vqg_batch_energy_and_gradient(vqg_batch *b, const double *theta, double *energies,
                                             double *grads) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    if (!theta || !energies || !grads) return set_error(VQG_ERR_INVALID, "null pointer");
    int st = b->build();
    if (st) return st;
    const int nc = (int)b->c.size(), P = b->total_params;
    std::memcpy(b->h_pinned, theta, sizeof(double) * P);
    cudaError_t e = cudaMemcpyAsync(b->d_theta, b->h_pinned, sizeof(double) * P, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "batch theta upload: %s", cudaGetErrorString(e));
    if ((st = b->run(b->d_theta, b->d_out, b->d_out + nc))) return st;
    double *h = b->h_pinned + P;
    e = cudaMemcpyAsync(h, b->d_out, sizeof(double) * (nc + P), cudaMemcpyDeviceToHost, b->stream);
    int errflag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + nc + P, b->args.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "batch readback: %s", cudaGetErrorString(e));
    std::memcpy(&errflag, h + nc + P, sizeof(int));
    std::memcpy(energies, h, sizeof(double) * nc);
    std::memcpy(grads, h + nc, sizeof(double) * P);
    if (errflag) return set_error(VQG_ERR_TIMEOUT, "a batched task gave up waiting for its circuit's previous phase");
    return VQG_OK;
}

extern "C" int vqg_batch_info(vqg_batch *b, int *n_tasks, int *grid, int *total_params) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    int st = b->build();
    if (st) return st;
    if (n_tasks) *n_tasks = b->n_tasks;
    if (grid) *grid = b->grid;
    if (total_params) *total_params = b->total_params;
    return VQG_OK;
}

extern "C" int vqg_batch_autotune(vqg_batch *b, const double *theta, vqg_tune_result *out) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    for (const BatchCircuit &bc : b->c)
        if (!bc.has_ham) return set_error(VQG_ERR_STATE, "every circuit needs a Hamiltonian first");
    return b->autotune(theta, out);
}

extern "C" int vqg_batch_set_tile_qubits(vqg_batch *b, int tile_qubits) {
    if (!b) return set_error(VQG_ERR_INVALID, "batch is NULL");
    for (const auto &g : kBatchGeom)
        if (g[0] == tile_qubits) {
            if (b->bk != g[0]) {
                b->reset();
                b->bk = g[0];
                b->br = g[1];
            }
            return VQG_OK;
        }
    return set_error(VQG_ERR_UNSUPPORTED, "no batched kernel with %d tile qubits", tile_qubits);
}
