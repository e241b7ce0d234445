// Tensor-product cost operators and user-supplied input states.
//
// A = sum_k c_k (x)_q M_{k,q} with Hermitian 2x2 factors (the paper's benchmark operator
// is Hadamard^{(x)N}, Sec. 3; Sec. 2.1 only asks that the simulator can apply the
// operator).  lambda = A psi is computed product by product: each product is a "circuit"
// of n one-qubit matrices, run through the same tile-fused forward kernels as the ansatz
// (a product over all n qubits takes ceil-ish n / K passes instead of n state sweeps),
// the coefficient c_k folded into its qubit-0 factor; products after the first go to a
// scratch state and are added into lambda.  E = Re <psi|lambda> is a separate FP64 dot
// product (the Pauli kernels fuse it instead).  The reverse sweep is unchanged.
//
// The input state |in> (Sec. 2.2's "fixed input state", |0...0> by default) is copied
// into a library-owned buffer; the forward sweep's first pass reads it instead of
// synthesising |0...0>.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vqg.h"
#include "engine.h"
#include "fused.h"
#include "plan.h"

namespace vqg {

// Re <psi|lambda> per block into partials[blockIdx.x] (FP64 per thread, deterministic tree).
template <typename T>
__global__ void __launch_bounds__(256) k_dot_re(const amp_t<T> *__restrict__ psi, const amp_t<T> *__restrict__ lam,
                                                uint64_t dim, double *__restrict__ partials, int nb) {
    double acc[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < dim; j += stride) {
        const amp_t<T> a = psi[j], b = lam[j];
        acc[0] += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
    }
    block_reduce_store<1>(acc, partials, nb);
}

// lam += tmp
template <typename T>
__global__ void __launch_bounds__(256) k_axpy(amp_t<T> *__restrict__ lam, const amp_t<T> *__restrict__ tmp,
                                              uint64_t dim) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < dim; j += stride) {
        const amp_t<T> a = lam[j], b = tmp[j];
        lam[j] = mk<T>(a.x + b.x, a.y + b.y);
    }
}

void Circuit::drop_product_plans() {
    for (Plan *pp : prod_plans) release_plan(pp);
    prod_plans.clear();
}

void Circuit::free_products() {
    drop_product_plans();
    dfree(d_prod_mats);
    dfree(d_prod_mats_f);
    dfree(d_prod_tmp);
    d_prod_mats = nullptr;
    d_prod_mats_f = nullptr;
    d_prod_tmp = nullptr;
    n_products = 0;
    prod_active = false;
}

// Fused plans of the products (same tile geometry as the ansatz plan): one U3-kind gate
// per qubit; the matrices come from the product's rows of the factor table.
int Circuit::build_product_plans() {
    drop_product_plans();
    if (!prod_active || !(opt.fusion && plan_ok)) return VQG_OK;
    std::vector<vqg_gate> pg(n);
    std::vector<int> sb(n);
    for (int q = 0; q < n; ++q) {
        pg[q] = vqg_gate{VQG_U3, q, -1, {0, 0, 0}};
        sb[q] = 8 * q;
    }
    vqg_options o = opt;
    o.tile_qubits = plan->K;
    o.fwd_reg_qubits = plan->Rf;
    o.rev_reg_qubits = plan->Rr;
    for (int k = 0; k < n_products; ++k) {
        std::string err;
        Plan *pp = plan_gates(n, pg, sb, 8 * n, dbl, o, err, FullCaps::value(), true, false);
        if (!pp) return set_error(VQG_ERR_UNSUPPORTED, "product operator plan: %s", err.empty() ? "none" : err.c_str());
        pp->grid_fwd = plan->grid_fwd;
        pp->passes[0].from_zero = 0;  // reads psi
        for (FPass &p : pp->passes) p.n_active = p.n_nontile, p.zero_in = 0;  // a dense input: every tile
        prod_plans.push_back(pp);
        int st = upload_plan(pp);
        if (st) return st;
    }
    return VQG_OK;
}

int Circuit::set_products(int np, const double *coef, const double *mats) {
    if (np < 1 || !coef || !mats) return set_error(VQG_ERR_INVALID, "bad product operator arguments");
    for (int k = 0; k < np; ++k)
        for (int q = 0; q < n; ++q) {
            const double *m = mats + 8 * ((size_t)k * n + q);
            double scale = 1.0;
            for (int e = 0; e < 8; ++e) scale = std::max(scale, std::fabs(m[e]));
            const double tol = 1e-12 * scale;
            // Hermitian: m00, m11 real, m01 = conj(m10)
            if (std::fabs(m[1]) > tol || std::fabs(m[7]) > tol || std::fabs(m[2] - m[4]) > tol ||
                std::fabs(m[3] + m[5]) > tol)
                return set_error(VQG_ERR_UNSUPPORTED, "product %d, qubit %d: factor is not Hermitian", k, q);
        }
    free_alt();
    free_products();
    std::vector<double> h(8 * (size_t)np * n);
    std::memcpy(h.data(), mats, sizeof(double) * h.size());
    for (int k = 0; k < np; ++k)  // c_k into the qubit-0 factor
        for (int e = 0; e < 8; ++e) h[8 * (size_t)k * n + e] *= coef[k];
    std::vector<float> hf(h.begin(), h.end());
    int st;
    if ((st = dalloc((void **)&d_prod_mats, sizeof(double) * h.size()))) return st;
    if ((st = dalloc((void **)&d_prod_mats_f, sizeof(float) * hf.size()))) return st;
    if (h2d(d_prod_mats, h.data(), sizeof(double) * h.size()) != cudaSuccess ||
        h2d(d_prod_mats_f, hf.data(), sizeof(float) * hf.size()) != cudaSuccess)
        return set_error(VQG_ERR_CUDA, "product operator upload failed");
    if (np > 1 && (st = dalloc(&d_prod_tmp, state_bytes))) return st;
    n_products = np;
    prod_active = true;
    has_ham = true;
    tuned = false;
    invalidate_graphs();
    return build_product_plans();
}

int Circuit::issue_hamiltonian_product() {
    const bool fused = opt.fusion && plan_ok && (int)prod_plans.size() == n_products;
    for (int k = 0; k < n_products; ++k) {
        void *dst = k == 0 ? lam : d_prod_tmp;
        prof_begin(fused ? FAM_FWD_FUSED : FAM_FWD_GATE);
        if (fused) {
            const Plan *pp = prod_plans[k];
            const void *m = dbl ? (const void *)(d_prod_mats + 8 * (size_t)k * n)
                                : (const void *)(d_prod_mats_f + 8 * (size_t)k * n);
            for (size_t j = 0; j < pp->passes.size(); ++j)
                launch_fused_fwd(dbl, float_float(dbl, opt), pp->K, pp->Rf, j == 0 ? psi : dst, dst, pp->d_passes,
                                 (int)j, pp->d_stages, pp->d_ops, pp->d_diags, pp->d_items, m, pp->n_tiles,
                                 pp->grid_fwd, stream);
        } else {
            cudaError_t e = cudaMemcpyAsync(dst, psi, state_bytes, cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "state copy: %s", cudaGetErrorString(e));
            for (int q = 0; q < n; ++q)
                launch_fwd_gate(dst, n, dbl, K_U3, q, -1, d_prod_mats + 8 * ((size_t)k * n + q), nb, stream);
        }
        prof_end();
        if (k > 0) {
            const uint64_t dim = 1ull << n;
            if (dbl) k_axpy<double><<<nb, 256, 0, stream>>>((double2 *)lam, (const double2 *)d_prod_tmp, dim);
            else k_axpy<float><<<nb, 256, 0, stream>>>((float2 *)lam, (const float2 *)d_prod_tmp, dim);
        }
    }
    const uint64_t dim = 1ull << n;
    prof_begin(FAM_HAM_DIAG);
    if (dbl) k_dot_re<double><<<nb, 256, 0, stream>>>((const double2 *)psi, (const double2 *)lam, dim, d_partials, nb);
    else k_dot_re<float><<<nb, 256, 0, stream>>>((const float2 *)psi, (const float2 *)lam, dim, d_partials, nb);
    prof_end();
    e_used = 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "product operator launch: %s", cudaGetErrorString(e));
    return VQG_OK;
}

int Circuit::set_input(const void *state, bool on_device) {
    if (!state) {
        has_input = false;
    } else {
        if (!d_input) {
            int st = dalloc(&d_input, state_bytes);
            if (st) return st;
        }
        cudaError_t e = cudaMemcpyAsync(d_input, state, state_bytes,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return set_error(VQG_ERR_CUDA, "input state copy: %s", cudaGetErrorString(e));
        has_input = true;
    }
    if (plan && !plan->passes.empty()) {  // pass 0: synthesise |0...0> or read the input
        plan->passes[0].from_zero = has_input ? 0 : 1;
        for (FPass &p : plan->passes) {
            p.n_active = has_input ? p.n_nontile : p.n_active_zero;
            p.zero_in = has_input ? 0 : p.zero_in_zero;
        }
        if (h2d(plan->d_passes, plan->passes.data(), sizeof(FPass) * plan->passes.size()) != cudaSuccess)
            return set_error(VQG_ERR_CUDA, "plan update failed");
    }
    invalidate_graphs();
    return VQG_OK;
}

}  // namespace vqg

using namespace vqg;

extern "C" int vqg_set_input_state(vqg_circuit *c, const void *state, int on_device) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    return reinterpret_cast<Circuit *>(c)->set_input(state, on_device != 0);
}

extern "C" int vqg_set_product_operator(vqg_circuit *c, int n_products, const double *coef, const double *mats) {
    if (!c) return set_error(VQG_ERR_INVALID, "circuit is NULL");
    return reinterpret_cast<Circuit *>(c)->set_products(n_products, coef, mats);
}
