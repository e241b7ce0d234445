// Float-float complex128 tile passes, K = 12 tile qubits, and the dispatch over K.
#define VQG_DF_DEFINE
#include "k_fused_df.cuh"

using namespace vqg;
VQG_DF_INSTANTIATE(12)

namespace vqg {

extern template void df_fwd<10>(const void *, void *, const FPass *, int, const FStage *, const FOp *,
                                const FDiag *, const FDItem *, const void *, uint64_t, int, cudaStream_t);
extern template void df_fwd<11>(const void *, void *, const FPass *, int, const FStage *, const FOp *,
                                const FDiag *, const FDItem *, const void *, uint64_t, int, cudaStream_t);
extern template void df_rev<10>(const void *, void *, void *, const FPass *, int, const FStage *, const FOp *,
                                const FDiag *, const FDItem *, const int *, const void *, uint64_t, double *,
                                int, int, cudaStream_t);
extern template void df_rev<11>(const void *, void *, void *, const FPass *, int, const FStage *, const FOp *,
                                const FDiag *, const FDItem *, const int *, const void *, uint64_t, double *,
                                int, int, cudaStream_t);
extern template void df_ham<10>(const void *, void *, const HPass *, int, const HGroup *, const HTerm *,
                                uint64_t, double *, int, cudaStream_t);
extern template void df_ham<11>(const void *, void *, const HPass *, int, const HGroup *, const HTerm *,
                                uint64_t, double *, int, cudaStream_t);

// Returns false if (K, R) has no float-float instantiation.
bool launch_fused_fwd_df(int K, int R, const void *src, void *dst, const FPass *passes, int pi, const FStage *st,
                         const FOp *ops, const FDiag *dg, const FDItem *it, const void *mats, uint64_t n_tiles,
                         int grid, cudaStream_t s) {
    if (R != kDfRegQubits) return false;
    switch (K) {
    case 10: df_fwd<10>(src, dst, passes, pi, st, ops, dg, it, mats, n_tiles, grid, s); return true;
    case 11: df_fwd<11>(src, dst, passes, pi, st, ops, dg, it, mats, n_tiles, grid, s); return true;
    case 12: df_fwd<12>(src, dst, passes, pi, st, ops, dg, it, mats, n_tiles, grid, s); return true;
    default: return false;
    }
}

bool launch_fused_rev_df(int K, int R, const void *phi_src, void *phi_dst, void *lam, const FPass *passes, int pi,
                         const FStage *st, const FOp *ops, const FDiag *dg, const FDItem *it, const int *slot_map,
                         const void *mats, uint64_t n_tiles, double *partials, int nb, int wmask, cudaStream_t s) {
    if (R != kDfRegQubits) return false;
    switch (K) {
    case 10: df_rev<10>(phi_src, phi_dst, lam, passes, pi, st, ops, dg, it, slot_map, mats, n_tiles, partials, nb, wmask, s); return true;
    case 11: df_rev<11>(phi_src, phi_dst, lam, passes, pi, st, ops, dg, it, slot_map, mats, n_tiles, partials, nb, wmask, s); return true;
    case 12: df_rev<12>(phi_src, phi_dst, lam, passes, pi, st, ops, dg, it, slot_map, mats, n_tiles, partials, nb, wmask, s); return true;
    default: return false;
    }
}

void launch_fused_ham_df(int K, const void *psi, void *lam, const HPass *hp, int pi, const HGroup *groups,
                         const HTerm *terms, uint64_t n_tiles, double *partials, int nb, cudaStream_t s) {
    switch (K) {
    case 10: df_ham<10>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
    case 11: df_ham<11>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
    case 12: df_ham<12>(psi, lam, hp, pi, groups, terms, n_tiles, partials, nb, s); break;
    default: break;
    }
}

}  // namespace vqg
