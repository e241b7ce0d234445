// Tile-fused forward and reverse passes, complex128 instantiations.
#include "fused_kernels.cuh"

namespace vqg {

template <typename Kern>
static void set_smem(Kern k, size_t bytes) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int K, int R>
static void fwd_t(const void *src, void *dst, const FPass *passes, int pi, const FStage *st,
                  const FOp *ops, const FDiag *dg, const FDItem *it, const void *mats, uint64_t n_tiles,
                  int grid, cudaStream_t s) {
    constexpr size_t sm = FwdCfg<T, K, R>::smem();
    static bool once = false;
    if (!once) set_smem(k_fused_fwd<T, K, R>, sm), once = true;
    k_fused_fwd<T, K, R><<<grid, FwdCfg<T, K, R>::NT, sm, s>>>(
        (const amp_t<T> *)src, (amp_t<T> *)dst, passes, pi, st, ops, dg, it, (const typename FT<T>::mat_t *)mats, n_tiles);
}

template <typename T, int K, int R>
static void rev_t(const void *phi_src, void *phi_dst, void *lam, const FPass *passes, int pi,
                  const FStage *st, const FOp *ops, const FDiag *dg, const FDItem *it,
                  const int *slot_map, const void *mats, uint64_t n_tiles, double *partials, int nb,
                  int wmask, cudaStream_t s) {
    constexpr size_t sm = RevCfg<T, K, R>::smem();
    static bool once = false;
    if (!once) set_smem(k_fused_rev<T, K, R>, sm), once = true;
    k_fused_rev<T, K, R><<<nb, RevCfg<T, K, R>::NT, sm, s>>>(
        (const amp_t<T> *)phi_src, (amp_t<T> *)phi_dst, (amp_t<T> *)lam, passes, pi, st, ops, dg, it,
        slot_map, (const typename FT<T>::mat_t *)mats, n_tiles, partials, nb, wmask);
}

// Returns false if (K, R) has no instantiation.
bool launch_fused_fwd_c128(int K, int R, const void *src, void *dst, const FPass *passes, int pi,
                      const FStage *st, const FOp *ops, const FDiag *dg, const FDItem *it,
                      const void *mats, uint64_t n_tiles, int grid, cudaStream_t s) {
#define VQG_FWD(KK, RR) \
    if (K == KK && R == RR) { fwd_t<double, KK, RR>(src, dst, passes, pi, st, ops, dg, it, mats, n_tiles, grid, s); return true; }
    VQG_FWD(10, 3)
    VQG_FWD(10, 4)
    VQG_FWD(11, 3)
    VQG_FWD(11, 4)
    VQG_FWD(12, 3)
    VQG_FWD(12, 4)
#undef VQG_FWD
    return false;
}

bool launch_fused_rev_c128(int K, int R, const void *phi_src, void *phi_dst, void *lam,
                      const FPass *passes, int pi, const FStage *st, const FOp *ops, const FDiag *dg,
                      const FDItem *it, const int *slot_map, const void *mats, uint64_t n_tiles,
                      double *partials, int nb, int wmask, cudaStream_t s) {
#define VQG_REV(KK, RR) \
    if (K == KK && R == RR) { \
        rev_t<double, KK, RR>(phi_src, phi_dst, lam, passes, pi, st, ops, dg, it, slot_map, mats, n_tiles, partials, nb, wmask, s); \
        return true; \
    }
    VQG_REV(10, 2)
    VQG_REV(10, 3)
    VQG_REV(11, 2)
    VQG_REV(11, 3)
    VQG_REV(12, 3)
#undef VQG_REV
    return false;
}

}  // namespace vqg
