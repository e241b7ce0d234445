// Non-Hermitian cost operators (App. B.4): E = <psi|A|psi> and dE/dtheta, both complex,
// for a Pauli sum A = sum_k c_k P_k with complex c_k.
//
// The paper runs a modified Algorithm 1 twice (with A and with A^dagger).  Here A is
// split into its Hermitian and anti-Hermitian parts, A = B + iC with B = sum Re(c_k) P_k
// and C = sum Im(c_k) P_k (Pauli strings are Hermitian), so E = <B> + i<C> and
// dE = d<B> + i d<C>, each the ordinary real Algorithm-1 gradient.  The two runs share
// one forward sweep: the final state is saved, the B run consumes it (Hamiltonian
// application + reverse sweep), and the C run restarts from the saved copy.  Both
// parts keep their own Pauli groups and Hamiltonian tile passes on the device; the
// circuit's "active" Hamiltonian fields hold B and the fields below hold C, swapped in
// for the second run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/vqg.h"
#include "engine.h"
#include "fused.h"
#include "plan.h"

namespace vqg {

struct AltHam {
    std::vector<HamGroup> ham;
    std::vector<PauliTerm> host_terms;
    PauliTerm *d_terms = nullptr;
    int n_terms = 0;
    bool has_ham = false, ham_plan_ok = false;
    std::vector<HPass> hp;
    std::vector<HGroup> hg;
    std::vector<HTerm> ht;
    HPass *d_hp = nullptr;
    HGroup *d_hg = nullptr;
    HTerm *d_ht = nullptr;
};

__global__ void k_interleave(const double *__restrict__ re, const double *__restrict__ im, int count,
                             double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) {
        out[2 * k] = re ? re[k] : 0.0;
        out[2 * k + 1] = im ? im[k] : 0.0;
    }
}

static void launch_interleave(const double *re, const double *im, int count, double *out, cudaStream_t s) {
    if (count > 0) k_interleave<<<(count + 127) / 128, 128, 0, s>>>(re, im, count, out);
}

// Exchange the active Hamiltonian (fields of the circuit and its plan) with the stored one.
void Circuit::swap_alt() {
    AltHam &a = *alt;
    std::swap(ham, a.ham);
    std::swap(host_terms, a.host_terms);
    std::swap(d_terms, a.d_terms);
    std::swap(n_terms, a.n_terms);
    std::swap(has_ham, a.has_ham);
    std::swap(ham_plan_ok, a.ham_plan_ok);
    if (plan) {
        std::swap(plan->hp, a.hp);
        std::swap(plan->hg, a.hg);
        std::swap(plan->ht, a.ht);
        std::swap(plan->d_hp, a.d_hp);
        std::swap(plan->d_hg, a.d_hg);
        std::swap(plan->d_ht, a.d_ht);
    }
    invalidate_graphs();
}

void Circuit::free_alt() {
    if (!alt) return;
    for (void *p : {(void *)alt->d_terms, (void *)alt->d_hp, (void *)alt->d_hg, (void *)alt->d_ht}) dfree(p);
    delete alt;
    alt = nullptr;
    dfree(psi_saved);
    psi_saved = nullptr;
    op_complex = false;
    op_b_empty = false;
}

// Re-plan the stored part's Hamiltonian passes after the gate plan changed (autotuner).
int Circuit::rebuild_alt_plan() {
    if (!alt || !op_complex) return VQG_OK;
    for (void *p : {(void *)alt->d_hp, (void *)alt->d_hg, (void *)alt->d_ht}) dfree(p);
    alt->d_hp = nullptr;
    alt->d_hg = nullptr;
    alt->d_ht = nullptr;
    alt->hp.clear();
    alt->hg.clear();
    alt->ht.clear();
    alt->ham_plan_ok = false;
    swap_alt();
    int st = plan ? build_ham_plan() : VQG_OK;
    swap_alt();
    return st;
}

// Split the terms into B (real parts) and C (imaginary parts), plan C and store it, then
// make B the active Hamiltonian.  Terms with a zero part are left out of that part.
int Circuit::set_operator(int n_t, const uint64_t *x, const uint64_t *z, const double *cr, const double *ci) {
    if (n_t < 0 || (n_t > 0 && (!x || !z || !cr || !ci))) return set_error(VQG_ERR_INVALID, "bad operator arguments");
    std::vector<uint64_t> bx, bz, cx, cz;
    std::vector<double> bc, cc;
    for (int t = 0; t < n_t; ++t) {
        if (cr[t] != 0.0) bx.push_back(x[t]), bz.push_back(z[t]), bc.push_back(cr[t]);
        if (ci[t] != 0.0) cx.push_back(x[t]), cz.push_back(z[t]), cc.push_back(ci[t]);
    }
    std::vector<HamGroup> gb, gc;
    std::vector<PauliTerm> fb, fc;
    int st = group_pauli_terms(n, (int)bc.size(), bx.data(), bz.data(), bc.data(), gb, fb);
    if (!st) st = group_pauli_terms(n, (int)cc.size(), cx.data(), cz.data(), cc.data(), gc, fc);
    if (st) return st;
    free_alt();
    free_products();
    if (!cc.empty()) {
        alt = new AltHam();
        if ((st = dalloc(&psi_saved, state_bytes))) return st;
        if ((st = set_groups(gc, fc))) return st;  // plans C as the active part ...
        swap_alt();                               // ... and stores it
        op_complex = true;
    }
    op_b_empty = bc.empty();
    if ((st = set_groups(gb, fb))) return st;
    if (!d_op_out && (st = dalloc((void **)&d_op_out, sizeof(double) * 2 * (size_t)(P + 1)))) return st;
    return VQG_OK;
}

// E = <B> + i<C> and its gradient into expect_dev[2] and grad_dev[2P] (re, im pairs), on
// the circuit's stream.  One forward sweep; each part then applies its Hamiltonian to the
// final state and runs the reverse sweep (the C part from the saved copy).
int Circuit::run_operator(const double *theta_dev, double *expect_dev, double *grad_dev) {
    if (!has_ham && !op_complex && !op_b_empty) return set_error(VQG_ERR_STATE, "no operator set");
    if (!d_op_out) {
        int st = dalloc((void **)&d_op_out, sizeof(double) * 2 * (size_t)(P + 1));
        if (st) return st;
    }
    invalidate_graphs();
    double *out_b = d_op_out, *out_c = d_op_out + (P + 1);
    int st;
    if ((st = issue_table(theta_dev, -1, -1, 0.0))) return st;
    if ((st = issue_forward(true))) return st;
    if (op_complex) {
        cudaError_t e = cudaMemcpyAsync(psi_saved, psi, state_bytes, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "state copy: %s", cudaGetErrorString(e));
    }
    if (!op_b_empty) {
        if ((st = issue_hamiltonian(true))) return st;
        if ((st = issue_reverse())) return st;
        if ((st = issue_finalize(out_b, out_b + 1, theta_dev))) return st;
    }
    if (op_complex) {
        cudaError_t e = cudaMemcpyAsync(psi, psi_saved, state_bytes, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "state copy: %s", cudaGetErrorString(e));
        swap_alt();
        st = issue_hamiltonian(true);
        if (!st) st = issue_reverse();
        if (!st) st = issue_finalize(out_c, out_c + 1, theta_dev);
        swap_alt();
        if (st) return st;
    }
    const double *re = op_b_empty ? nullptr : out_b, *im = op_complex ? out_c : nullptr;
    launch_interleave(re, im, 1, expect_dev, stream);
    launch_interleave(re ? re + 1 : nullptr, im ? im + 1 : nullptr, P, grad_dev, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "interleave launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

}  // namespace vqg

using namespace vqg;

extern "C" int vqg_set_operator(vqg_circuit *c, int n_terms, const uint64_t *x_mask, const uint64_t *z_mask,
                                const double *coef_re, const double *coef_im) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    return reinterpret_cast<Circuit *>(c)->set_operator(n_terms, x_mask, z_mask, coef_re, coef_im);
}

extern "C" int vqg_expectation_and_gradient_device(vqg_circuit *c, const double *theta_dev, double *expect_dev,
                                                   double *grad_dev) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    if ((!theta_dev && cc->P > 0) || !expect_dev || (!grad_dev && cc->P > 0))
        return set_error(VQG_ERR_INVALID, "null pointer");
    return cc->run_operator(theta_dev, expect_dev, grad_dev);
}

extern "C" int vqg_expectation_and_gradient(vqg_circuit *c, const double *theta, double *expect, double *grad) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    Circuit *cc = reinterpret_cast<Circuit *>(c);
    const int P = cc->P;
    if ((!theta && P > 0) || !expect || (!grad && P > 0)) return set_error(VQG_ERR_INVALID, "null pointer");
    double *d_res = nullptr;  // 2 + 2P doubles: expectation then gradient, (re, im) pairs
    int st = cc->ensure_op_scratch(&d_res);
    if (st) return st;
    if (P) {
        std::memcpy(cc->h_pinned, theta, sizeof(double) * P);
        cudaError_t e = cudaMemcpyAsync(cc->d_theta, cc->h_pinned, sizeof(double) * P, cudaMemcpyHostToDevice, cc->stream);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "theta upload: %s", cudaGetErrorString(e));
    }
    if ((st = cc->run_operator(cc->d_theta, d_res, d_res + 2))) return st;
    std::vector<double> h(2 + 2 * (size_t)P);
    cudaError_t e = cudaMemcpyAsync(h.data(), d_res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, cc->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cc->stream);
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "readback: %s", cudaGetErrorString(e));
    expect[0] = h[0];
    expect[1] = h[1];
    if (P) std::memcpy(grad, h.data() + 2, sizeof(double) * 2 * P);
    return VQG_OK;
}

namespace vqg {
int Circuit::ensure_op_scratch(double **out) {
    if (!d_op_res) {
        int st = dalloc((void **)&d_op_res, sizeof(double) * (2 + 2 * (size_t)P));
        if (st) return st;
    }
    *out = d_op_res;
    return VQG_OK;
}
}  // namespace vqg
