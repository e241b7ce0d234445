// C ABI of the library (include/vqg.h): circuit objects, Hamiltonian grouping, and
// the launch sequence of Algorithm 1 on one GPU.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/vqg.h"
#include "engine.h"

using namespace vqg;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

int vqg::set_error(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

cudaError_t vqg::h2d(void *dst, const void *src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cudaStreamLegacy);
    return e == cudaSuccess ? cudaStreamSynchronize(cudaStreamLegacy) : e;
}

extern "C" const char *vqg_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *vqg_status_string(int status) {
    switch (status) {
    case VQG_OK: return "ok";
    case VQG_ERR_INVALID: return "invalid argument";
    case VQG_ERR_OOM: return "out of device memory";
    case VQG_ERR_CUDA: return "CUDA error";
    case VQG_ERR_TIMEOUT: return "device wait timed out";
    case VQG_ERR_UNSUPPORTED: return "unsupported";
    case VQG_ERR_STATE: return "invalid call order";
    default: return "unknown status";
    }
}

extern "C" void vqg_default_options(vqg_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->fusion = 1;
    opt->checkpoint_interval = 0;
    opt->tile_qubits = 0;
    opt->use_graph = 0;
    opt->max_checkpoint_mib = 0;
}

static const char *kFamilyNames[] = {"init",      "table",     "fwd_gate",  "fwd_fused",
                                     "ham_diag",  "ham_group", "ham_fused", "adj_gate",
                                     "adj_fused", "reduce",    "ckpt_copy", "finalize",
                                     "batch"};

extern "C" const char *vqg_kernel_family_name(int id) {
    if (id < 0 || id >= FAM_COUNT) return "?";
    return kFamilyNames[id];
}

// ------------------------------------------------------------------ helpers
#define VQG_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_error(e_ == cudaErrorMemoryAllocation ? VQG_ERR_OOM : VQG_ERR_CUDA,     \
                             "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

static int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return VQG_OK;
}

void Circuit::prof_begin(int fam) {
    if (!profiling) return;
    if (ev_free.empty()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        ev_free.push_back({a, b});
    }
    pending.push_back({fam, ev_free.back().first, ev_free.back().second});
    ev_free.pop_back();
    cudaEventRecord(pending.back().start, stream);
}

void Circuit::prof_end() {
    if (!profiling || pending.empty()) return;
    cudaEventRecord(pending.back().stop, stream);
}

void Circuit::prof_harvest() {
    if (pending.empty()) return;
    cudaStreamSynchronize(stream);
    for (auto &p : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            fam_launches[p.fam] += 1;
            fam_ms[p.fam] += ms;
        }
        ev_free.push_back({p.start, p.stop});
    }
    pending.clear();
    cudaGetLastError();
}

Circuit::~Circuit() {
    free_alt();
    free_products();
    free_plan();
    if (graph_exec_grad) cudaGraphExecDestroy(graph_exec_grad);
    if (graph_exec_energy) cudaGraphExecDestroy(graph_exec_energy);
    for (void *p : dev_allocs) cudaFree(p);
    if (h_pinned) cudaFreeHost(h_pinned);
    for (auto &p : pending) ev_free.push_back({p.start, p.stop});
    for (auto &e : ev_free) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (own_stream && stream) cudaStreamDestroy(stream);
}

int Circuit::dalloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(VQG_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    dev_allocs.push_back(*p);
    return VQG_OK;
}

void Circuit::dfree(void *p) {
    if (!p) return;
    auto it = std::find(dev_allocs.begin(), dev_allocs.end(), p);
    if (it != dev_allocs.end()) dev_allocs.erase(it);
    cudaFree(p);
}

int Circuit::ensure_partials() {
    const int need = n_eslots + n_gslots;
    if (need <= partial_cap && d_partials) return VQG_OK;
    dfree(d_partials);
    dfree(d_red);
    d_partials = nullptr;
    d_red = nullptr;
    int st = dalloc((void **)&d_partials, sizeof(double) * (size_t)std::max(need, 1) * nb);
    if (st) return st;
    st = dalloc((void **)&d_red, sizeof(double) * (size_t)std::max(need, 1));
    if (st) return st;
    partial_cap = need;
    return VQG_OK;
}

// ------------------------------------------------------------------ create / destroy
static bool is_1q(int k) { return (k >= VQG_RX && k <= VQG_U3) || k == VQG_PHASE; }
static int nparams_of(int k) { return params_of(k); }

int vqg::vqg_validate_circuit(int n_qubits, const vqg_gate *gates, int n_gates, int n_params, int dtype) {
    if (n_qubits < 1 || n_qubits > 34) return set_error(VQG_ERR_INVALID, "n_qubits=%d outside 1..34", n_qubits);
    if (n_gates < 0 || (n_gates > 0 && !gates)) return set_error(VQG_ERR_INVALID, "bad gate list");
    if (n_params < 0) return set_error(VQG_ERR_INVALID, "n_params=%d < 0", n_params);
    if (dtype != VQG_C64 && dtype != VQG_C128) return set_error(VQG_ERR_INVALID, "dtype=%d", dtype);
    for (int i = 0; i < n_gates; ++i) {
        const vqg_gate &g = gates[i];
        if (g.kind < VQG_RX || g.kind > VQG_CPHASE) return set_error(VQG_ERR_INVALID, "gate %d: kind %d", i, g.kind);
        if (g.q0 < 0 || g.q0 >= n_qubits) return set_error(VQG_ERR_INVALID, "gate %d: qubit %d out of range", i, g.q0);
        if (!is_1q(g.kind)) {
            if (g.q1 < 0 || g.q1 >= n_qubits) return set_error(VQG_ERR_INVALID, "gate %d: qubit %d out of range", i, g.q1);
            if (g.q1 == g.q0) return set_error(VQG_ERR_INVALID, "gate %d: q0 == q1", i);
        }
        for (int j = 0; j < nparams_of(g.kind); ++j)
            if (g.param[j] < 0 || g.param[j] >= n_params)
                return set_error(VQG_ERR_INVALID, "gate %d: parameter index %d out of range", i, g.param[j]);
    }
    return VQG_OK;
}

extern "C" int vqg_circuit_create(int n_qubits, const vqg_gate *gates, int n_gates, int n_params,
                                  int dtype, const vqg_options *opt, vqg_circuit **out) {
    if (!out) return set_error(VQG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int vst = vqg_validate_circuit(n_qubits, gates, n_gates, n_params, dtype);
    if (vst) return vst;
    if (opt && opt->c128_arith != VQG_C128_FP64 && opt->c128_arith != VQG_C128_FLOAT_FLOAT)
        return set_error(VQG_ERR_INVALID, "c128_arith %d is not a vqg_c128_arith", opt->c128_arith);
    Circuit *c = new (std::nothrow) Circuit();
    if (!c) return set_error(VQG_ERR_OOM, "host allocation failed");
    int st = c->init(n_qubits, gates, n_gates, n_params, dtype, opt);
    if (st) {
        std::string msg = g_last_error;
        delete c;
        g_last_error = msg;
        return st;
    }
    *out = reinterpret_cast<vqg_circuit *>(c);
    return VQG_OK;
}

int Circuit::init(int n_, const vqg_gate *gates_, int G_, int P_, int dtype_, const vqg_options *opt_) {
    n = n_;
    G = G_;
    P = P_;
    dtype = dtype_;
    dbl = dtype == VQG_C128;
    amp_bytes = dbl ? 16 : 8;
    state_bytes = (size_t)amp_bytes << n;
    vqg_default_options(&opt);
    if (opt_) opt = *opt_;
    tile_explicit = opt.tile_qubits > 0;
    VQG_CUDA(cudaGetDevice(&device));
    VQG_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    VQG_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
    gates.assign(gates_, gates_ + G);
    // grid: persistent-style, up to 8 resident 256-thread blocks per SM
    {
        const uint64_t pairs = 1ull << (n - 1);
        const uint64_t want = (pairs + 1023) / 1024;
        nb = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms * 8));
    }
    // reverse-sweep reduction slots and occurrence lists (App. B.1 / B.2)
    slot_base.assign(std::max(G, 1), 0);
    n_gslots = 0;
    std::vector<std::vector<Occurrence>> by_param(P);
    for (int i = 0; i < G; ++i) {
        slot_base[i] = n_gslots;
        n_gslots += reduce_values_of(gates[i].kind);
        for (int j = 0; j < nparams_of(gates[i].kind); ++j) by_param[gates[i].param[j]].push_back({i, j});
    }
    std::vector<int> occ_ptr(P + 1, 0);
    std::vector<Occurrence> occ;
    for (int p = 0; p < P; ++p) {
        occ_ptr[p] = (int)occ.size();
        occ.insert(occ.end(), by_param[p].begin(), by_param[p].end());
    }
    occ_ptr[P] = (int)occ.size();

    int st;
    // small device tables
    std::vector<DevGate> dg(std::max(G, 1));
    for (int i = 0; i < G; ++i) dg[i] = {gates[i].kind, gates[i].q0, gates[i].q1, gates[i].param[0], gates[i].param[1], gates[i].param[2]};
    if ((st = dalloc((void **)&d_gates, sizeof(DevGate) * dg.size()))) return st;
    VQG_CUDA(h2d(d_gates, dg.data(), sizeof(DevGate) * dg.size()));
    if ((st = dalloc((void **)&d_mats, sizeof(double) * 8 * std::max(G, 1)))) return st;
    if ((st = dalloc((void **)&d_slot_base, sizeof(int) * slot_base.size()))) return st;
    VQG_CUDA(h2d(d_slot_base, slot_base.data(), sizeof(int) * slot_base.size()));
    if ((st = dalloc((void **)&d_occ_ptr, sizeof(int) * occ_ptr.size()))) return st;
    VQG_CUDA(h2d(d_occ_ptr, occ_ptr.data(), sizeof(int) * occ_ptr.size()));
    if ((st = dalloc((void **)&d_occ, sizeof(Occurrence) * std::max<size_t>(occ.size(), 1)))) return st;
    if (!occ.empty())
        VQG_CUDA(h2d(d_occ, occ.data(), sizeof(Occurrence) * occ.size()));
    if ((st = dalloc((void **)&d_theta, sizeof(double) * std::max(P, 1)))) return st;
    if ((st = dalloc((void **)&d_out, sizeof(double) * (P + 1)))) return st;
    VQG_CUDA(cudaMallocHost((void **)&h_pinned, sizeof(double) * (2 * (size_t)P + 2)));
    n_eslots = 1;
    if ((st = ensure_partials())) return st;
    // state vectors
    if ((st = dalloc(&psi, state_bytes))) return st;
    if ((st = dalloc(&lam, state_bytes))) return st;
    if ((st = build_plan())) return st;
    return plan_checkpoints();
}

// Forward states are stored every `interval` gates (per-gate schedule) or at the first
// pass boundary after every `interval` gates (fused schedule), as many as fit.  Buffers
// already held (from an earlier schedule of the same circuit) are reused; surplus ones
// are released.
int Circuit::plan_checkpoints() {
    const bool fused = opt.fusion && plan_ok;
    int interval = opt.checkpoint_interval;
    // automatic: complex64 stores the output of every fused pass (each reverse pass then
    // restarts phi from exact forward data, and no reverse pass has to store phi) or every
    // 64 gates unfused; complex128 stores none
    if (interval == 0) interval = dbl ? -1 : (fused ? 1 : 64);
    ckpt_pos.clear();
    std::vector<int> want;
    if (interval >= 0 && G >= 2) {
        if (fused) want = fused_checkpoint_passes(interval);
        else
            for (int c = interval; c < G; c += interval) want.push_back(c);
    }
    if (want.size() > ckpt_buf.size()) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const size_t headroom = (size_t)4 << 30;
        size_t budget = free_b > headroom ? free_b - headroom : 0;
        if (opt.max_checkpoint_mib > 0) {
            const size_t cap = (size_t)opt.max_checkpoint_mib << 20, held = ckpt_buf.size() * state_bytes;
            budget = std::min(budget, cap > held ? cap - held : 0);
        }
        const size_t fit = ckpt_buf.size() + budget / state_bytes;
        while (ckpt_buf.size() < std::min(fit, want.size())) {
            void *buf = nullptr;
            if (dalloc(&buf, state_bytes) != VQG_OK) break;  // fewer checkpoints, still correct
            ckpt_buf.push_back(buf);
        }
    }
    if (want.size() > ckpt_buf.size()) {  // keep evenly spread positions
        std::vector<int> keep;
        const size_t fit = ckpt_buf.size();
        for (size_t k = 0; k < fit; ++k) keep.push_back(want[(k + 1) * want.size() / (fit + 1)]);
        want.swap(keep);
    }
    while (ckpt_buf.size() > want.size()) {
        dfree(ckpt_buf.back());
        ckpt_buf.pop_back();
    }
    for (size_t k = 0; k < want.size(); ++k) {
        if (fused) set_fused_checkpoint(want[k], (int)k);
        else ckpt_pos.push_back(want[k]);
    }
    cudaGetLastError();
    g_last_error.clear();
    return VQG_OK;
}

extern "C" int vqg_circuit_destroy(vqg_circuit *c) {
    if (!c) return VQG_OK;
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    if (cc->stream) cudaStreamSynchronize(cc->stream);
    delete cc;
    return VQG_OK;
}

extern "C" int vqg_set_stream(vqg_circuit *c, void *stream) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    if (stream == nullptr) {
        if (!cc->own_stream) {
            VQG_CUDA(cudaStreamCreateWithFlags(&cc->stream, cudaStreamNonBlocking));
            cc->own_stream = true;
        }
    } else {
        if (cc->own_stream) {
            cudaStreamSynchronize(cc->stream);
            cudaStreamDestroy(cc->stream);
        }
        cc->stream = (cudaStream_t)stream;
        cc->own_stream = false;
    }
    cc->invalidate_graphs();
    return VQG_OK;
}

// ------------------------------------------------------------------ Hamiltonian
extern "C" int vqg_set_hamiltonian(vqg_circuit *c, int n_terms, const uint64_t *x_mask,
                                   const uint64_t *z_mask, const double *coef) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    std::vector<HamGroup> ham;
    std::vector<PauliTerm> flat;
    int st = group_pauli_terms(cc->n, n_terms, x_mask, z_mask, coef, ham, flat);
    if (st) return st;
    cc->free_alt();  // a Pauli Hamiltonian replaces a non-Hermitian or tensor-product operator
    cc->free_products();
    return cc->set_groups(ham, flat);
}

// ------------------------------------------------------------------ Pauli strings
// Character q of strings[t] is the Pauli letter on qubit q (I, X, Y or Z), so the
// string "XIZY" on 4 qubits is X_0 Z_2 Y_3.  X sets the x bit, Z the z bit, Y both
// (the mask form's convention: Y = i X Z).
extern "C" int vqg_pauli_strings_to_masks(int n_qubits, int n_terms, const char *const *strings,
                                          uint64_t *x_mask, uint64_t *z_mask) {
    if (n_qubits < 1 || n_qubits > 64) return set_error(VQG_ERR_INVALID, "n_qubits=%d outside 1..64", n_qubits);
    if (n_terms < 0) return set_error(VQG_ERR_INVALID, "n_terms=%d", n_terms);
    if (n_terms > 0 && (!strings || !x_mask || !z_mask)) return set_error(VQG_ERR_INVALID, "null pointer");
    for (int t = 0; t < n_terms; ++t) {
        const char *s = strings[t];
        if (!s) return set_error(VQG_ERR_INVALID, "string %d is NULL", t);
        uint64_t x = 0, z = 0;
        int q = 0;
        for (; s[q] != '\0'; ++q) {
            if (q >= n_qubits)
                return set_error(VQG_ERR_INVALID, "string %d is longer than %d qubits", t, n_qubits);
            const uint64_t b = 1ull << q;
            switch (s[q]) {
            case 'I': break;
            case 'X': x |= b; break;
            case 'Y': x |= b; z |= b; break;
            case 'Z': z |= b; break;
            default:
                return set_error(VQG_ERR_INVALID, "string %d: character %d is '%c', not one of I, X, Y, Z", t, q,
                                 s[q]);
            }
        }
        if (q != n_qubits)
            return set_error(VQG_ERR_INVALID, "string %d has %d characters for %d qubits", t, q, n_qubits);
        x_mask[t] = x;
        z_mask[t] = z;
    }
    return VQG_OK;
}

extern "C" int vqg_set_hamiltonian_strings(vqg_circuit *c, int n_terms, const char *const *strings,
                                           const double *coef) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    if (n_terms < 0) return set_error(VQG_ERR_INVALID, "n_terms=%d", n_terms);
    std::vector<uint64_t> x((size_t)std::max(n_terms, 1)), z((size_t)std::max(n_terms, 1));
    int st = vqg_pauli_strings_to_masks(cc->n, n_terms, strings, x.data(), z.data());
    if (st) return st;
    return vqg_set_hamiltonian(c, n_terms, x.data(), z.data(), coef);
}

int Circuit::set_groups(const std::vector<HamGroup> &groups, const std::vector<PauliTerm> &flat) {
    ham = groups;
    int st;
    dfree(d_terms);
    d_terms = nullptr;
    if ((st = dalloc((void **)&d_terms, sizeof(PauliTerm) * std::max<size_t>(flat.size(), 1)))) return st;
    if (!flat.empty())
        VQG_CUDA(h2d(d_terms, flat.data(), sizeof(PauliTerm) * flat.size()));
    n_terms = (int)flat.size();
    host_terms = flat;
    n_eslots = std::max(n_eslots, (int)ham.size());
    has_ham = true;
    tuned = false;
    if ((st = ensure_partials())) return st;
    invalidate_graphs();
    return build_plan();
}

// ------------------------------------------------------------------ launch sequences
int Circuit::issue_table(const double *theta_dev, int shift_gate, int shift_slot, double shift) {
    prof_begin(FAM_TABLE);
    launch_build_mats(theta_dev, d_gates, G, d_mats, mats_f(), shift_gate, shift_slot, shift, stream);
    prof_end();
    return check_launch("build_mats");
}

// NVTX range over the host-side issue of one phase (forward sweep, Hamiltonian, reverse
// sweep): a profiler that records NVTX (Nsight Systems, ncu --nvtx) attributes the phase's
// kernels to it; without one attached the calls do nothing.
namespace {
struct PhaseRange {
    explicit PhaseRange(const char *name) { nvtxRangePushA(name); }
    ~PhaseRange() { nvtxRangePop(); }
};
}  // namespace

int Circuit::issue_forward(bool with_ckpt) {
    PhaseRange range("vqg forward sweep");
    if (opt.fusion && plan_ok) return issue_forward_fused(with_ckpt);  // pass 0 starts from |in>
    prof_begin(FAM_INIT);
    if (has_input) VQG_CUDA(cudaMemcpyAsync(psi, d_input, state_bytes, cudaMemcpyDeviceToDevice, stream));
    else launch_init_zero(psi, n, dbl, nb, stream);
    prof_end();
    size_t k = 0;
    for (int i = 0; i < G; ++i) {
        const vqg_gate &g = gates[i];
        prof_begin(FAM_FWD_GATE);
        launch_fwd_gate(psi, n, dbl, g.kind, g.q0, g.q1, d_mats + 8 * (size_t)i, nb, stream);
        prof_end();
        if (with_ckpt && k < ckpt_pos.size() && ckpt_pos[k] == i + 1) {
            prof_begin(FAM_CKPT);
            VQG_CUDA(cudaMemcpyAsync(ckpt_buf[k], psi, state_bytes, cudaMemcpyDeviceToDevice, stream));
            prof_end();
            if (int st = diag_reduce(ckpt_buf[k], nullptr, DIAG_STORE, (int)k)) return st;
            ++k;
        }
    }
    return check_launch("forward");
}

int Circuit::issue_hamiltonian(bool write_lam) {
    PhaseRange range("vqg lambda = H psi");
    if (prod_active) return issue_hamiltonian_product();
    if (ham.empty()) {  // H = 0: lambda = 0, E = 0
        e_used = 0;
        if (write_lam) VQG_CUDA(cudaMemsetAsync(lam, 0, state_bytes, stream));
        return VQG_OK;
    }
    if (opt.fusion && plan_ok && ham_plan_ok) return issue_hamiltonian_fused();
    e_used = (int)ham.size();
    for (size_t g = 0; g < ham.size(); ++g) {
        const HamGroup &h = ham[g];
        double *part = d_partials + (size_t)g * nb;
        if (h.x == 0) {
            prof_begin(FAM_HAM_DIAG);
            launch_pauli_diag(psi, lam, n, dbl, d_terms + h.first, h.count, part, nb, write_lam, stream);
        } else {
            prof_begin(FAM_HAM_GROUP);
            launch_pauli_group(psi, lam, n, dbl, h.x, d_terms + h.first, h.count, part, nb, write_lam, stream);
        }
        prof_end();
    }
    return check_launch("hamiltonian");
}

int Circuit::issue_reverse() {
    PhaseRange range("vqg reverse sweep");
    if (opt.fusion && plan_ok) return issue_reverse_fused();
    double *gpart = d_partials + (size_t)n_eslots * nb;
    int k = (int)ckpt_pos.size() - 1;
    for (int i = G - 1; i >= 0; --i) {
        const vqg_gate &g = gates[i];
        const void *src = psi;
        while (k >= 0 && ckpt_pos[k] > i + 1) --k;
        if (k >= 0 && ckpt_pos[k] == i + 1) {  // restart phi from the stored state
            src = ckpt_buf[k];
            if (int st = diag_reduce(ckpt_buf[k], lam, DIAG_RESTART, k)) return st;
            if (int st = diag_reduce(psi, ckpt_buf[k], DIAG_UNAPPLIED, k)) return st;
        }
        prof_begin(FAM_ADJ_GATE);
        launch_adj_gate(src, psi, lam, n, dbl, g.kind, g.q0, g.q1, d_mats + 8 * (size_t)i,
                        gpart + (size_t)slot_base[i] * nb, nb, i > 0, i > 0, stream);
        prof_end();
    }
    return check_launch("reverse");
}

int Circuit::issue_finalize(double *energy_dev, double *grad_dev, const double *theta_dev) {
    prof_begin(FAM_REDUCE);
    launch_reduce_slots(d_partials, n_eslots + (grad_dev ? n_gslots : 0), nb, d_red, stream);
    prof_end();
    prof_begin(FAM_FINALIZE);
    launch_finalize(d_red, e_used, d_red + n_eslots, theta_dev, d_gates, d_slot_base, d_occ_ptr,
                    d_occ, grad_dev ? P : 0, energy_dev, grad_dev, stream);
    prof_end();
    return check_launch("finalize");
}

int Circuit::issue_gradient(const double *theta_dev, double *energy_dev, double *grad_dev) {
    int st;
    diag_active = false;
    if (diagnostics) {  // FP64 norms and inner products along the sweep (diag.cu)
        if ((st = diag_prepare())) return st;
        diag_active = true;
    }
    if (!(st = issue_table(theta_dev, -1, -1, 0.0)) && !(st = issue_forward(true)) && !(st = issue_hamiltonian(true)) &&
        !(st = diag_reduce(psi, lam, DIAG_FINAL, 0)) && !(st = issue_reverse()) &&
        !(st = issue_finalize(energy_dev, grad_dev, theta_dev)))
        st = diag_finish();
    diag_active = false;
    return st;
}

// With use_graph, the launch sequence of one call (it does not depend on theta: the
// gate matrices are rebuilt on the device from theta_dev) is captured once per set of
// argument pointers and replayed afterwards.  Profiling runs eagerly (it needs events
// between launches); the legacy default stream cannot be captured and also runs eagerly.
static int hermitian_only(const Circuit &c) {
    return c.op_complex ? set_error(VQG_ERR_STATE, "the operator is not Hermitian: use vqg_expectation_and_gradient")
                        : VQG_OK;
}

int Circuit::run_gradient(const double *theta_dev, double *energy_dev, double *grad_dev) {
    if (!has_ham) return set_error(VQG_ERR_STATE, "no Hamiltonian set");
    if (int st = hermitian_only(*this)) return st;
    if (opt.autotune && !tuned) {  // first evaluation picks the schedule (blocks once)
        int st = autotune(theta_dev, nullptr);
        if (st) return st;
    }
    const bool graphable =
        opt.use_graph && !profiling && !diagnostics && stream != cudaStreamLegacy && stream != nullptr;
    if (!graphable) return issue_gradient(theta_dev, energy_dev, grad_dev);
    const void *key[3] = {theta_dev, energy_dev, grad_dev};
    if (graph_exec_grad && std::memcmp(key, graph_key_grad, sizeof key) != 0) {
        cudaGraphExecDestroy(graph_exec_grad);
        graph_exec_grad = nullptr;
    }
    if (!graph_exec_grad) {
        if (!graph_warm) {  // first call eagerly: sets kernel attributes outside capture
            graph_warm = true;
            return issue_gradient(theta_dev, energy_dev, grad_dev);
        }
        cudaGraph_t g = nullptr;
        VQG_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        int st = issue_gradient(theta_dev, energy_dev, grad_dev);
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&graph_exec_grad, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            graph_exec_grad = nullptr;
            return set_error(VQG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        std::memcpy(graph_key_grad, key, sizeof key);
    }
    VQG_CUDA(cudaGraphLaunch(graph_exec_grad, stream));
    return VQG_OK;
}

int Circuit::run_energy(const double *theta_dev, double *energy_dev, int sg, int ss, double sh) {
    if (!has_ham) return set_error(VQG_ERR_STATE, "no Hamiltonian set");
    if (int st = hermitian_only(*this)) return st;
    int st;
    if ((st = issue_table(theta_dev, sg, ss, sh))) return st;
    if ((st = issue_forward(false))) return st;
    if ((st = issue_hamiltonian(false))) return st;
    return issue_finalize(energy_dev, nullptr, theta_dev);
}

// ------------------------------------------------------------------ public calls
static int get(vqg_circuit *c, Circuit **out) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    *out = reinterpret_cast<Circuit *>(c);
    return VQG_OK;
}

extern "C" int vqg_energy(vqg_circuit *c, const double *theta, double *energy) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    if ((!theta && cc->P > 0) || !energy) return set_error(VQG_ERR_INVALID, "null pointer");
    if (cc->P) {
        std::memcpy(cc->h_pinned, theta, sizeof(double) * cc->P);
        VQG_CUDA(cudaMemcpyAsync(cc->d_theta, cc->h_pinned, sizeof(double) * cc->P, cudaMemcpyHostToDevice, cc->stream));
    }
    if ((st = cc->run_energy(cc->d_theta, cc->d_out, -1, -1, 0.0))) return st;
    VQG_CUDA(cudaMemcpyAsync(cc->h_pinned + cc->P, cc->d_out, sizeof(double), cudaMemcpyDeviceToHost, cc->stream));
    VQG_CUDA(cudaStreamSynchronize(cc->stream));
    *energy = cc->h_pinned[cc->P];
    return VQG_OK;
}

extern "C" int vqg_energy_and_gradient(vqg_circuit *c, const double *theta, double *energy, double *grad) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    if ((!theta && cc->P > 0) || !energy || (!grad && cc->P > 0)) return set_error(VQG_ERR_INVALID, "null pointer");
    const int P = cc->P;
    if (P) {
        std::memcpy(cc->h_pinned, theta, sizeof(double) * P);
        VQG_CUDA(cudaMemcpyAsync(cc->d_theta, cc->h_pinned, sizeof(double) * P, cudaMemcpyHostToDevice, cc->stream));
    }
    if ((st = cc->run_gradient(cc->d_theta, cc->d_out, cc->d_out + 1))) return st;
    VQG_CUDA(cudaMemcpyAsync(cc->h_pinned + P, cc->d_out, sizeof(double) * (P + 1), cudaMemcpyDeviceToHost, cc->stream));
    VQG_CUDA(cudaStreamSynchronize(cc->stream));
    *energy = cc->h_pinned[P];
    if (P) std::memcpy(grad, cc->h_pinned + P + 1, sizeof(double) * P);
    return VQG_OK;
}

extern "C" int vqg_energy_device(vqg_circuit *c, const double *theta_dev, double *energy_dev) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    if ((!theta_dev && cc->P > 0) || !energy_dev) return set_error(VQG_ERR_INVALID, "null pointer");
    return cc->run_energy(theta_dev, energy_dev, -1, -1, 0.0);
}

extern "C" int vqg_energy_and_gradient_device(vqg_circuit *c, const double *theta_dev, double *energy_dev,
                                              double *grad_dev) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    if ((!theta_dev && cc->P > 0) || !energy_dev || (!grad_dev && cc->P > 0))
        return set_error(VQG_ERR_INVALID, "null pointer");
    return cc->run_gradient(theta_dev, energy_dev, grad_dev);
}

extern "C" int vqg_gradient_parameter_shift(vqg_circuit *c, const double *theta, int first_gate,
                                            int last_gate, double *grad) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    const int P = cc->P, G = cc->G;
    if ((!theta && P > 0) || (!grad && P > 0)) return set_error(VQG_ERR_INVALID, "null pointer");
    if (last_gate < 0 || last_gate > G) last_gate = G;
    if (first_gate < 0 || first_gate > last_gate) return set_error(VQG_ERR_INVALID, "bad gate range");
    // Shift rules: E as a function of one occurrence's angle has the frequencies of its
    // generator's eigenvalue differences.  Rotations, U3 slots and phase gates: {1}, so
    // dE/dt = [E(t + pi/2) - E(t - pi/2)] / 2.  Controlled rotations ((sigma/2) x
    // |1><1|): {1/2, 1}, so dE/dt = a1 [E(t + pi/2) - E(t - pi/2)] + a2 [E(t + 3pi/2) -
    // E(t - 3pi/2)] with a1 + a2 = 1/(2 sqrt 2), a1 - a2 = 1/2 (solving the two
    // frequencies' equations).
    struct Shift { int gate, slot, e0, n_e; };
    std::vector<Shift> occs;
    int n_e = 0;
    for (int i = first_gate; i < last_gate; ++i)
        for (int j = 0; j < nparams_of(cc->gates[i].kind); ++j) {
            const int k = cc->gates[i].kind;
            const int ne = (k >= VQG_CRX && k <= VQG_CRZ) ? 4 : 2;
            occs.push_back({i, j, n_e, ne});
            n_e += ne;
        }
    double *d_e = nullptr;
    if ((st = cc->dalloc((void **)&d_e, sizeof(double) * std::max(n_e, 1)))) return st;
    if (P) {
        std::memcpy(cc->h_pinned, theta, sizeof(double) * P);
        VQG_CUDA(cudaMemcpyAsync(cc->d_theta, cc->h_pinned, sizeof(double) * P, cudaMemcpyHostToDevice, cc->stream));
    }
    const double h = M_PI / 2.0;
    for (size_t k = 0; k < occs.size() && !st; ++k) {
        const Shift &o = occs[k];
        const double sh[4] = {+h, -h, +3.0 * h, -3.0 * h};
        for (int x = 0; x < o.n_e && !st; ++x) st = cc->run_energy(cc->d_theta, d_e + o.e0 + x, o.gate, o.slot, sh[x]);
    }
    std::vector<double> e(n_e);
    if (!st && !occs.empty()) {
        cudaError_t ce = cudaMemcpyAsync(e.data(), d_e, sizeof(double) * e.size(), cudaMemcpyDeviceToHost, cc->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(cc->stream);
        if (ce != cudaSuccess) st = set_error(VQG_ERR_CUDA, "parameter shift readback: %s", cudaGetErrorString(ce));
    } else {
        cudaStreamSynchronize(cc->stream);
    }
    cc->dfree(d_e);
    if (st) return st;
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    const double r2 = std::sqrt(2.0), a1 = (r2 + 1.0) / (4.0 * r2), a2 = -(r2 - 1.0) / (4.0 * r2);
    for (const Shift &o : occs) {
        const double *v = e.data() + o.e0;
        const double d = o.n_e == 4 ? a1 * (v[0] - v[1]) + a2 * (v[2] - v[3]) : 0.5 * (v[0] - v[1]);
        grad[cc->gates[o.gate].param[o.slot]] += d;
    }
    return VQG_OK;
}

extern "C" int vqg_get_state(vqg_circuit *c, void *out, size_t bytes) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    if (!out || bytes < cc->state_bytes) return set_error(VQG_ERR_INVALID, "output buffer too small");
    VQG_CUDA(cudaStreamSynchronize(cc->stream));
    VQG_CUDA(cudaMemcpy(out, cc->psi_forward(), cc->state_bytes, cudaMemcpyDeviceToHost));
    return VQG_OK;
}

extern "C" int vqg_set_profiling(vqg_circuit *c, int enable) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    cc->prof_harvest();
    cc->profiling = enable != 0;
    for (int f = 0; f < FAM_COUNT; ++f) cc->fam_launches[f] = 0, cc->fam_ms[f] = 0.0;
    return VQG_OK;
}

extern "C" int vqg_kernel_stats(vqg_circuit *c, int max_entries, int *name_id, int *launches, double *total_ms) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    cc->prof_harvest();
    int k = 0;
    for (int f = 0; f < FAM_COUNT && k < max_entries; ++f) {
        if (!cc->fam_launches[f]) continue;
        if (name_id) name_id[k] = f;
        if (launches) launches[k] = (int)cc->fam_launches[f];
        if (total_ms) total_ms[k] = cc->fam_ms[f];
        ++k;
    }
    return k;
}

extern "C" int vqg_plan(vqg_circuit *c, vqg_plan_info *info) {
    Circuit *cc;
    int st;
    if ((st = get(c, &cc))) return st;
    if (!info) return set_error(VQG_ERR_INVALID, "info is NULL");
    std::memset(info, 0, sizeof *info);
    cc->fill_plan_info(info);
    return VQG_OK;
}
