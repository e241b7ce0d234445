// Tile-fused forward, Hamiltonian and reverse passes for complex128 states computed in
// float-float arithmetic (df.cuh): amplitudes stay FP64 in HBM, the tile arithmetic runs
// on the FP32 pipe.  One register geometry (3 register qubits per stage, forward and
// reverse) for tile sizes K = 10..12; each K is its own translation unit so that the
// library builds in parallel.
#pragma once

#include "fused_kernels.cuh"

namespace vqg {

constexpr int kDfRegQubits = 3;

template <typename Kern>
static void df_set_smem(Kern k, size_t bytes) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int K>
void df_fwd(const void *src, void *dst, const FPass *passes, int pi, const FStage *st, const FOp *ops,
            const FDiag *dg, const FDItem *it, const void *mats, uint64_t n_tiles, int grid, cudaStream_t s)
#ifdef VQG_DF_DEFINE
{
    constexpr int R = kDfRegQubits;
    constexpr size_t sm = FwdCfg<df, K, R>::smem();
    static bool once = false;
    if (!once) df_set_smem(k_fused_fwd<df, K, R>, sm), once = true;
    k_fused_fwd<df, K, R><<<grid, FwdCfg<df, K, R>::NT, sm, s>>>(
        (const amp_t<df> *)src, (amp_t<df> *)dst, passes, pi, st, ops, dg, it, (const double *)mats, n_tiles);
}
#else
;
#endif

template <int K>
void df_rev(const void *phi_src, void *phi_dst, void *lam, const FPass *passes, int pi, const FStage *st,
            const FOp *ops, const FDiag *dg, const FDItem *it, const int *slot_map, const void *mats,
            uint64_t n_tiles, double *partials, int nb, int wmask, cudaStream_t s)
#ifdef VQG_DF_DEFINE
{
    constexpr int R = kDfRegQubits;
    constexpr size_t sm = RevCfg<df, K, R>::smem();
    static bool once = false;
    if (!once) df_set_smem(k_fused_rev<df, K, R>, sm), once = true;
    k_fused_rev<df, K, R><<<nb, RevCfg<df, K, R>::NT, sm, s>>>(
        (const amp_t<df> *)phi_src, (amp_t<df> *)phi_dst, (amp_t<df> *)lam, passes, pi, st, ops, dg, it,
        slot_map, (const double *)mats, n_tiles, partials, nb, wmask);
}
#else
;
#endif

template <int K>
void df_ham(const void *psi, void *lam, const HPass *hp, int pi, const HGroup *groups, const HTerm *terms,
            uint64_t n_tiles, double *partials, int nb, cudaStream_t s)
#ifdef VQG_DF_DEFINE
{
    constexpr size_t sm = HamCfg<df, K>::smem();
    static bool once = false;
    if (!once) df_set_smem(k_fused_ham<df, K>, sm), once = true;
    k_fused_ham<df, K><<<nb, 256, sm, s>>>((const amp_t<df> *)psi, (amp_t<df> *)lam, hp, pi, groups, terms,
                                            n_tiles, partials, nb);
}
#else
;
#endif

}  // namespace vqg

#define VQG_DF_INSTANTIATE(K)                                                                          \
    template void vqg::df_fwd<K>(const void *, void *, const FPass *, int, const FStage *, const FOp *,  \
                                 const FDiag *, const FDItem *, const void *, uint64_t, int, cudaStream_t); \
    template void vqg::df_rev<K>(const void *, void *, void *, const FPass *, int, const FStage *,       \
                                 const FOp *, const FDiag *, const FDItem *, const int *, const void *,  \
                                 uint64_t, double *, int, int, cudaStream_t);                            \
    template void vqg::df_ham<K>(const void *, void *, const HPass *, int, const HGroup *, const HTerm *, \
                                 uint64_t, double *, int, cudaStream_t);
