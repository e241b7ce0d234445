// Hamiltonian tile passes (complex64 and complex128 instantiations).
#include "fused_kernels.cuh"

namespace vqg {

template <typename Kern>
static void set_smem(Kern k, size_t bytes) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int K>
static void ham_t(const void *psi, void *lam, const HPass *hp, int pi, const HGroup *groups,
                  const HTerm *terms, uint64_t n_tiles, double *partials, int nb, cudaStream_t s) {
    constexpr size_t sm = HamCfg<T, K>::smem();
    static bool once = false;
    if (!once) set_smem(k_fused_ham<T, K>, sm), once = true;
    k_fused_ham<T, K><<<nb, 256, sm, s>>>((const amp_t<T> *)psi, (amp_t<T> *)lam, hp, pi, groups,
                                           terms, n_tiles, partials, nb);
}

void launch_fused_ham(bool dbl, int K, const void *psi, void *lam, const HPass *hp, int pi,
                      const HGroup *groups, const HTerm *terms, uint64_t n_tiles, double *partials,
                      int nb, cudaStream_t s) {
    if (!dbl) {
        switch (K) {
        case 10: ham_t<float, 10>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 11: ham_t<float, 11>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 12: ham_t<float, 12>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 13: ham_t<float, 13>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        default: break;
        }
    } else {
        switch (K) {
        case 10: ham_t<double, 10>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 11: ham_t<double, 11>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        case 12: ham_t<double, 12>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
        default: break;
        }
    }
}

}  // namespace vqg
