// Execution planner: turns the gate list into fused tile passes.
#include <cstring>

#include "engine.h"

namespace vqg {

int Circuit::build_plan() {
    plan_ok = false;
    ham_plan_ok = false;
    return VQG_OK;
}

void Circuit::free_plan() {}

int Circuit::issue_forward_fused(bool) { return set_error(VQG_ERR_UNSUPPORTED, "fused forward not built"); }
int Circuit::issue_hamiltonian_fused() { return set_error(VQG_ERR_UNSUPPORTED, "fused H not built"); }
int Circuit::issue_reverse_fused() { return set_error(VQG_ERR_UNSUPPORTED, "fused reverse not built"); }

void Circuit::fill_plan_info(vqg_plan_info *info) const {
    const bool fused = opt.fusion && plan_ok;
    info->forward_passes = fused ? 0 : G;
    info->hamiltonian_passes = (int)ham.size();
    info->reverse_passes = fused ? 0 : G;
    info->checkpoints = (int)ckpt_pos.size();
    info->tile_qubits = 0;
    info->hamiltonian_groups = (int)ham.size();
    info->launches_per_gradient = 1 + 1 + G + (int)ckpt_pos.size() + (int)ham.size() + G + 2;
}

}  // namespace vqg
