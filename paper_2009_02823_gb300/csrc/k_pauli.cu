// Hamiltonian application |lambda> = H|psi> for a Pauli sum (Algorithm 1, before the reverse loop) with
// the energy E = Re <psi|lambda> fused in.
//
// A term coef * i^{popcount(x&z)} X^x Z^z maps psi to
//   (P psi)[j] = w * (-1)^{popcount((j^x) & z)} * psi[j^x],   w = coef * i^{popcount(x&z)}.
// Terms with the same flip mask x form a group; one pass over amplitude pairs
// (j, j^x) applies the whole group:
//   lambda[j]   += f(j^x) psi[j^x],   lambda[j^x] += f(j) psi[j],
//   f(i) = sum_k w_k (-1)^{popcount(i & z_k)}.
// The diagonal group (x = 0) writes lambda = f psi and runs first.
#include "kernels.h"

namespace vqg {

constexpr int kThreads = 256;
constexpr int kChunk = 16;

template <typename T>
VQG_DEV amp_t<T> fval(uint64_t i, const PauliTerm *__restrict__ terms, int count) {
    T re = 0, im = 0;
    for (int k = 0; k < count; ++k) {
        const PauliTerm t = terms[k];
        const T sg = (__popcll(i & t.z) & 1) ? (T)-1 : (T)1;
        re += sg * (T)t.wr;
        im += sg * (T)t.wi;
    }
    return mk<T>(re, im);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pauli_diag(const amp_t<T> *__restrict__ psi, amp_t<T> *__restrict__ lam,
                 const PauliTerm *__restrict__ terms, int count, uint64_t dim,
                 double *__restrict__ partials, int nb, int write_lam) {
    double acc[1] = {0.0};
    T run = 0;
    int in_run = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < dim; j += stride) {
        const amp_t<T> a = psi[j];
        const amp_t<T> f = fval<T>(j, terms, count);  // real for x = 0
        if (write_lam) lam[j] = mk<T>(f.x * a.x, f.x * a.y);
        run += f.x * (a.x * a.x + a.y * a.y);
        if (++in_run == kChunk) acc[0] += (double)run, run = 0, in_run = 0;
    }
    acc[0] += (double)run;
    block_reduce_store<1>(acc, partials, nb);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pauli_group(const amp_t<T> *__restrict__ psi, amp_t<T> *__restrict__ lam, uint64_t x, int h,
                  const PauliTerm *__restrict__ terms, int count, uint64_t units,
                  double *__restrict__ partials, int nb, int write_lam) {
    double acc[1] = {0.0};
    T run = 0;
    int in_run = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < units; p += stride) {
        const uint64_t j = insert0(p, h), jx = j ^ x;
        const amp_t<T> a = psi[j], b = psi[jx];
        const amp_t<T> fj = fval<T>(j, terms, count), fjx = fval<T>(jx, terms, count);
        const amp_t<T> tj = cmul<T>(fjx, b);   // contribution to lambda[j]
        const amp_t<T> tjx = cmul<T>(fj, a);   // contribution to lambda[j^x]
        if (write_lam) {
            lam[j] = cadd<T>(lam[j], tj);
            lam[jx] = cadd<T>(lam[jx], tjx);
        }
        run += (a.x * tj.x + a.y * tj.y) + (b.x * tjx.x + b.y * tjx.y);
        if (++in_run == kChunk) acc[0] += (double)run, run = 0, in_run = 0;
    }
    acc[0] += (double)run;
    block_reduce_store<1>(acc, partials, nb);
}

void launch_pauli_diag(const void *psi, void *lam, int n, bool dbl, const PauliTerm *terms,
                       int count, double *partials, int nb, bool write_lam, cudaStream_t s) {
    const uint64_t dim = 1ull << n;
    if (dbl)
        k_pauli_diag<double><<<nb, kThreads, 0, s>>>((const double2 *)psi, (double2 *)lam, terms,
                                                     count, dim, partials, nb, write_lam);
    else
        k_pauli_diag<float><<<nb, kThreads, 0, s>>>((const float2 *)psi, (float2 *)lam, terms,
                                                    count, dim, partials, nb, write_lam);
}

void launch_pauli_group(const void *psi, void *lam, int n, bool dbl, uint64_t x,
                        const PauliTerm *terms, int count, double *partials, int nb,
                        bool write_lam, cudaStream_t s) {
    const int h = 63 - __builtin_clzll(x);
    const uint64_t units = 1ull << (n - 1);
    if (dbl)
        k_pauli_group<double><<<nb, kThreads, 0, s>>>((const double2 *)psi, (double2 *)lam, x, h,
                                                      terms, count, units, partials, nb, write_lam);
    else
        k_pauli_group<float><<<nb, kThreads, 0, s>>>((const float2 *)psi, (float2 *)lam, x, h,
                                                     terms, count, units, partials, nb, write_lam);
}

}  // namespace vqg
