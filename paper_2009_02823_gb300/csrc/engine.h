// Circuit object and execution plan (host side).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <utility>
#include <vector>

#include "../../include/vqg.h"
#include "kernels.h"

namespace vqg {

struct Plan;
struct AltHam;
int set_error(int status, const char *fmt, ...);
// Host-to-device copy of a table that has landed when the call returns.  A plain cudaMemcpy
// from pageable memory may return before its DMA completes, and it runs on the legacy
// stream, which the library's non-blocking streams do not wait for.
cudaError_t h2d(void *dst, const void *src, size_t bytes);
int vqg_validate_circuit(int n_qubits, const vqg_gate *gates, int n_gates, int n_params, int dtype);

enum Family {
    FAM_INIT = 0, FAM_TABLE, FAM_FWD_GATE, FAM_FWD_FUSED, FAM_HAM_DIAG, FAM_HAM_GROUP,
    FAM_HAM_FUSED, FAM_ADJ_GATE, FAM_ADJ_FUSED, FAM_REDUCE, FAM_CKPT, FAM_FINALIZE, FAM_BATCH,
    FAM_COUNT
};

struct HamGroup {
    uint64_t x;
    int first, count;
};

int group_pauli_terms(int n, int n_terms, const uint64_t *x_mask, const uint64_t *z_mask,
                      const double *coef, std::vector<HamGroup> &ham, std::vector<PauliTerm> &flat);

// What a diagnostic reduction measured (diag.cu).
enum { DIAG_FINAL = 0, DIAG_STORE = 1, DIAG_RESTART = 2, DIAG_UNAPPLIED = 3 };

struct PendingEvent {
    int fam;
    cudaEvent_t start, stop;
};

struct Circuit {
    // problem
    int n = 0, G = 0, P = 0, dtype = 0;
    bool dbl = false;
    int amp_bytes = 8;
    size_t state_bytes = 0;
    vqg_options opt{};
    std::vector<vqg_gate> gates;
    std::vector<int> slot_base;
    int n_gslots = 0, n_eslots = 1;

    // device / stream
    int device = 0, num_sms = 1, nb = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // device buffers
    std::vector<void *> dev_allocs;
    void *psi = nullptr, *lam = nullptr;
    std::vector<int> ckpt_pos;
    std::vector<void *> ckpt_buf;
    DevGate *d_gates = nullptr;
    double *d_mats = nullptr, *d_theta = nullptr, *d_out = nullptr;
    double *d_partials = nullptr, *d_red = nullptr;
    int partial_cap = 0;
    int *d_slot_base = nullptr, *d_occ_ptr = nullptr;
    Occurrence *d_occ = nullptr;
    double *h_pinned = nullptr;

    // Hamiltonian
    bool has_ham = false;
    std::vector<HamGroup> ham;
    std::vector<PauliTerm> host_terms;
    PauliTerm *d_terms = nullptr;
    int n_terms = 0;
    int e_used = 1;  // energy partial slots written by the last Hamiltonian application

    // fused plan (engine.cu)
    bool plan_ok = false, ham_plan_ok = false;
    struct Plan *plan = nullptr;

    // non-Hermitian operator A = B + iC (operator.cu): the active Hamiltonian is B, `alt`
    // holds C; psi_saved keeps the forward result for the second part's run
    AltHam *alt = nullptr;
    bool op_complex = false;  // C has terms
    bool op_b_empty = false;  // B has no terms
    void *psi_saved = nullptr;
    double *d_op_out = nullptr, *d_op_res = nullptr;
    void swap_alt();
    void free_alt();
    int rebuild_alt_plan();
    int set_operator(int n_terms, const uint64_t *x, const uint64_t *z, const double *cr, const double *ci);
    int run_operator(const double *theta_dev, double *expect_dev, double *grad_dev);
    int ensure_op_scratch(double **out);

    // input state (product.cu): |in> replaces |0...0> when set
    bool has_input = false;
    void *d_input = nullptr;
    int set_input(const void *state, bool on_device);

    // tensor-product operators (product.cu): A = sum_k c_k (x)_q M_{k,q}, Hermitian factors
    bool prod_active = false;
    int n_products = 0;
    double *d_prod_mats = nullptr;  // 8 doubles per (product, qubit); c_k folded into qubit 0
    float *d_prod_mats_f = nullptr;
    void *d_prod_tmp = nullptr;
    std::vector<Plan *> prod_plans;
    int set_products(int n_products, const double *coef, const double *mats);
    int build_product_plans();
    int issue_hamiltonian_product();
    void drop_product_plans();
    void free_products();
    int upload_plan(Plan *pl);
    void release_plan(Plan *pl);

    // precision diagnostics (diag.cu): FP64 norms and inner products of the stored
    // checkpoints and of phi and lambda at every reverse restart, recorded by gradient
    // calls while enabled (those calls run eagerly, outside any graph)
    bool diagnostics = false;
    bool diag_active = false;          // set during a gradient call with diagnostics on
    double *d_diag_part = nullptr;     // [5 * reduction][nb] block partials (k_norm.cu)
    double *d_diag_red = nullptr;      // [5 * reduction] reduced values
    int diag_cap = 0;                  // reductions the buffers hold
    std::vector<int> diag_tag;         // kind and checkpoint of each queued reduction
    int diag_prepare();                // size the buffers for this circuit's checkpoints
    int diag_reduce(const void *a, const void *b, int kind, int ckpt);
    int diag_finish();

    // graphs
    cudaGraphExec_t graph_exec_grad = nullptr, graph_exec_energy = nullptr;
    const void *graph_key_grad[3] = {nullptr, nullptr, nullptr};
    bool graph_warm = false;

    // profiling
    bool profiling = false;
    std::vector<PendingEvent> pending;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
    long fam_launches[FAM_COUNT] = {};
    double fam_ms[FAM_COUNT] = {};

    ~Circuit();
    int init(int n, const vqg_gate *gates, int G, int P, int dtype, const vqg_options *opt);
    int dalloc(void **p, size_t bytes);
    void dfree(void *p);
    int ensure_partials();
    int plan_checkpoints();
    int set_groups(const std::vector<HamGroup> &groups, const std::vector<PauliTerm> &flat);

    int issue_table(const double *theta_dev, int shift_gate, int shift_slot, double shift);
    int issue_forward(bool with_ckpt);
    int issue_hamiltonian(bool write_lam);
    int issue_reverse();
    int issue_finalize(double *energy_dev, double *grad_dev, const double *theta_dev);
    int issue_gradient(const double *theta_dev, double *energy_dev, double *grad_dev);
    int run_gradient(const double *theta_dev, double *energy_dev, double *grad_dev);
    int run_energy(const double *theta_dev, double *energy_dev, int sg, int ss, double sh);

    // fused path (engine.cu)
    int build_plan();
    int build_ham_plan();
    void free_plan();
    void drop_plan();
    int autotune(const double *theta_dev, vqg_tune_result *out);
    bool tuned = false;          // autotune ran (or was found a no-op) for this circuit
    bool tile_explicit = false;  // the caller fixed tile_qubits: nothing to tune
    std::vector<int> fused_checkpoint_passes(int interval) const;
    void set_fused_checkpoint(int pass, int k);
    float *mats_f() const;
    int issue_forward_fused(bool with_ckpt);
    int issue_hamiltonian_fused();
    int issue_reverse_fused();
    void fill_plan_info(vqg_plan_info *info) const;
    const void *psi_forward() const { return psi; }
    void invalidate_graphs() {
        if (graph_exec_grad) cudaGraphExecDestroy(graph_exec_grad);
        if (graph_exec_energy) cudaGraphExecDestroy(graph_exec_energy);
        graph_exec_grad = graph_exec_energy = nullptr;
    }

    void prof_begin(int fam);
    void prof_end();
    void prof_harvest();
};

}  // namespace vqg
