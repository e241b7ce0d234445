// Precision diagnostics of the reverse sweep (complex64 amplitudes with FP64 reductions
// and forward checkpoints): FP64 norms and inner products taken on the GPU while a
// gradient call runs, for the quantities Algorithm 1's recurrence keeps fixed (Sec. 2.3).
//
//   * after the Hamiltonian: ||psi||^2, E = Re <psi|lambda> and ||lambda||^2;
//   * when the forward sweep stores a checkpoint psi_c: ||psi_c||^2;
//   * where the reverse sweep restarts phi from psi_c: <lambda|psi_c> (= E, because phi
//     and lambda have been un-applied by the same unitaries) and ||lambda||^2 (constant);
//     and, against the phi that the sweep un-applied up to that point and that the restart
//     replaces, ||phi||^2 and ||phi - psi_c||^2 (the FP32 drift the restart removes).
//
// Off by default: enabling it adds one streaming reduction per checkpoint and two per
// restart, makes the reverse sweep keep its un-applied phi, and runs gradient calls
// eagerly (outside CUDA graphs).  Results are read with vqg_diagnostics.
#include <algorithm>
#include <cstring>
#include <vector>

#include "engine.h"
#include "kernels.h"

namespace vqg {

int Circuit::diag_prepare() {
    const int need = 1 + 3 * (int)std::max<size_t>(ckpt_buf.size(), ckpt_pos.size());
    diag_tag.clear();
    if (need <= diag_cap && d_diag_part) return VQG_OK;
    dfree(d_diag_part);
    dfree(d_diag_red);
    d_diag_part = d_diag_red = nullptr;
    diag_cap = 0;
    int st;
    if ((st = dalloc((void **)&d_diag_part, sizeof(double) * kNormValues * (size_t)need * nb))) return st;
    if ((st = dalloc((void **)&d_diag_red, sizeof(double) * kNormValues * (size_t)need))) return st;
    diag_cap = need;
    return VQG_OK;
}

// Queue one reduction of (a, b) (b = nullptr: a alone) into the next partial slots.
int Circuit::diag_reduce(const void *a, const void *b, int kind, int ckpt) {
    if (!diag_active) return VQG_OK;
    const int r = (int)diag_tag.size();
    if (r >= diag_cap) return set_error(VQG_ERR_STATE, "diagnostic reductions exceed their buffer (%d)", diag_cap);
    launch_norm_dot(a, b, n, dbl, d_diag_part + (size_t)kNormValues * r * nb, nb, stream);
    diag_tag.push_back(kind << 16 | (ckpt & 0xffff));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "norm/dot launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

int Circuit::diag_finish() {
    if (!diag_active) return VQG_OK;
    launch_reduce_slots(d_diag_part, kNormValues * (int)diag_tag.size(), nb, d_diag_red, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "diagnostic reduction: %s", cudaGetErrorString(e));
    return VQG_OK;
}

}  // namespace vqg

using namespace vqg;

extern "C" int vqg_set_diagnostics(vqg_circuit *c, int enable) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    cc->diagnostics = enable != 0;
    cc->diag_tag.clear();
    cc->invalidate_graphs();
    return VQG_OK;
}

extern "C" int vqg_diagnostics(vqg_circuit *c, vqg_diag_summary *summary, int max_entries,
                               vqg_checkpoint_diag *entries) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    if (max_entries < 0 || (max_entries > 0 && !entries)) return set_error(VQG_ERR_INVALID, "bad entries array");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    if (cc->diag_tag.empty()) return set_error(VQG_ERR_STATE, "no diagnostics recorded: enable them with "
                                                              "vqg_set_diagnostics, then run a gradient call");
    const size_t nr = cc->diag_tag.size();
    std::vector<double> v(kNormValues * nr);
    cudaError_t e = cudaStreamSynchronize(cc->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(v.data(), cc->d_diag_red, sizeof(double) * v.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "reading diagnostics: %s", cudaGetErrorString(e));
    int n_ck = 0;
    for (int t : cc->diag_tag) n_ck = std::max(n_ck, (t >> 16) != DIAG_FINAL ? (t & 0xffff) + 1 : 0);
    std::vector<vqg_checkpoint_diag> out((size_t)n_ck);
    for (int k = 0; k < n_ck; ++k) {
        std::memset(&out[k], 0, sizeof(vqg_checkpoint_diag));
        out[k].checkpoint = k;
    }
    if (summary) std::memset(summary, 0, sizeof(*summary));
    for (size_t r = 0; r < nr; ++r) {
        const double *x = v.data() + kNormValues * r;  // ||a||^2, Re <a|b>, Im <a|b>, ||b||^2, ||a-b||^2
        const int kind = cc->diag_tag[r] >> 16, k = cc->diag_tag[r] & 0xffff;
        if (kind == DIAG_FINAL) {
            if (summary) {
                summary->norm2_psi = x[0];
                summary->energy = x[1];
                summary->norm2_lambda = x[3];
            }
            continue;
        }
        vqg_checkpoint_diag &d = out[k];
        if (kind == DIAG_STORE) {
            d.stored = 1;
            d.norm2 = x[0];
        } else if (kind == DIAG_RESTART) {  // a = psi_c, b = lambda: <lambda|psi_c> = conj <psi_c|lambda>
            d.restarted = 1;
            d.lam_phi_re = x[1];
            d.lam_phi_im = -x[2];
            d.norm2_lambda = x[3];
        } else if (kind == DIAG_UNAPPLIED) {  // a = un-applied phi, b = psi_c
            d.norm2_unapplied = x[0];
            d.drift2 = x[4];
        }
    }
    if (summary) summary->checkpoints = n_ck;
    for (int k = 0; k < std::min(n_ck, max_entries); ++k) entries[k] = out[k];
    return n_ck;
}
