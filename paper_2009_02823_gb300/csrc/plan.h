// Host-side execution plan of the fused sweeps (built by engine.cu, also used by the
// batched launch in batch.cu).
#pragma once

#include <string>
#include <array>
#include <vector>

#include "../../include/vqg.h"
#include "engine.h"
#include "fused.h"

namespace vqg {

struct Plan {
    int K = 0, L = 0, Rf = 0, Rr = 0;
    PassCaps caps = FullCaps::value();  // program budget of the kernels that run the passes
    uint64_t n_tiles = 0;
    int grid_fwd = 0;
    std::vector<FPass> passes;
    std::vector<FStage> stages;
    std::vector<std::vector<int32_t>> pass_gates;  // host only: gate indices of each pass, applied order
    std::vector<std::array<int8_t, kMaxRegBits>> stage_reg_q;  // host only: global qubit of each register bit
    std::vector<FOp> ops;
    std::vector<FDiag> diags;
    std::vector<FDItem> items;
    std::vector<int> slot_map;
    std::vector<int> ckpt_of_pass;  // checkpoint index storing the output of pass j, or -1
    std::vector<HPass> hp;
    std::vector<HGroup> hg;
    std::vector<HTerm> ht;
    FPass *d_passes = nullptr;
    FStage *d_stages = nullptr;
    FOp *d_ops = nullptr;
    FDiag *d_diags = nullptr;
    FDItem *d_items = nullptr;
    int *d_slot_map = nullptr;
    HPass *d_hp = nullptr;
    HGroup *d_hg = nullptr;
    HTerm *d_ht = nullptr;
    float *d_mats_f = nullptr;
    // specialised kernels of each pass (spec.cu; cudaKernel_t handles), empty when the
    // passes run on the interpreted kernels
    std::vector<void *> spec_fwd, spec_rev, spec_ham;
    size_t spec_smem_fwd = 0, spec_smem_ham = 0;
    std::vector<size_t> spec_smem_rev;  // per reverse pass
    const void *spec_ham_for = nullptr;  // the Hamiltonian tables (d_hp) spec_ham was built for
};

// Plan the gate passes of one circuit (host only; nullptr + empty err: no fused
// schedule applies; nullptr + err: the plan failed its checks).  single_kernels: the
// (K, Rf, Rr) choice must be one the single-circuit launchers compiled; the batched
// kernel passes false (it has its own instantiations).  zero_start: the sweep usually starts
// from |0...0>, so tile sets are chosen for the tiles that start leaves at zero (false for
// operators applied to a dense state).
Plan *plan_gates(int n, const std::vector<vqg_gate> &gates, const std::vector<int> &slot_base,
                 int n_gslots, bool dbl, const vqg_options &opt, std::string &err,
                 const PassCaps &caps = FullCaps::value(), bool single_kernels = true, bool zero_start = true);
// Hamiltonian tile passes of a plan; false if some group cannot live in one tile.
bool plan_hamiltonian(Plan *pl, int n, const std::vector<HamGroup> &ham, const std::vector<PauliTerm> &host_terms);
std::string validate_plan(const Plan &pl, int n, int n_gslots, bool dbl);
bool fused_supported(bool dbl, int K, int Rf, int Rr, bool ff);
// complex128 computed in float-float arithmetic (options.c128_arith)
bool float_float(bool dbl, const vqg_options &opt);
#define VQG_FWD_LAUNCH_ARGS                                                                      \
    int K, int R, const void *src, void *dst, const FPass *passes, int pi, const FStage *st,      \
        const FOp *ops, const FDiag *dg, const FDItem *it, const void *mats, uint64_t n_tiles,    \
        int grid, cudaStream_t s
bool launch_fused_fwd(bool dbl, bool ff, VQG_FWD_LAUNCH_ARGS);
int default_tile_qubits(int n, bool dbl);
// Per-pass specialised complex64 kernels (spec.cu): build them for every pass of a plan
// (generated, compiled, cached, loaded), and launch pass j of either direction.
int spec_compile(const Plan *pl, bool with_rev, std::vector<std::string> &cubins);
int spec_build(Plan *pl, bool with_rev);
int spec_build_ham(Plan *pl);
int spec_launch_ham(const Plan *pl, int h, const void *psi, void *lam, double *partials, int nb, cudaStream_t s);
int spec_launch_fwd(const Plan *pl, int j, const void *src, void *dst, const void *mats, uint64_t n_tiles,
                    cudaStream_t s);
int spec_launch_rev(const Plan *pl, int j, const void *phi_src, void *phi_dst, void *lam, const void *mats,
                    double *partials, int nb, int wmask, uint64_t n_tiles, cudaStream_t s);

}  // namespace vqg
