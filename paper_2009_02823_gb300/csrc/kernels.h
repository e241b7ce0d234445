// Host-side launch wrappers for the device kernels (C++ internal interface of the
// library; the public boundary is include/vqg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace vqg {

struct DevGate {
    int32_t kind, q0, q1, p0, p1, p2;
};

// One occurrence of a parameter: gate index and slot.
struct Occurrence {
    int32_t gate, slot;
};

// --- gate table and result assembly (k_table.cu)
// mats: FP64 table (8 doubles per gate); mats_f (nullable): the same rounded to FP32.
void launch_build_mats(const double *theta, const DevGate *gates, int G, double *mats,
                       float *mats_f, int shift_gate, int shift_slot, double shift, cudaStream_t s);
void launch_init_zero(void *psi, int n, bool dbl, int nb, cudaStream_t s);
void launch_reduce_slots(const double *partials, int n_slots, int nb, double *red, cudaStream_t s);
// E = sum red_e[0 .. e_count); grad[p] from the reduced reverse-sweep values
// red_g[slot_base[gate] ..] contracted per occurrence.
void launch_finalize(const double *red_e, int e_count, const double *red_g, const double *theta,
                     const DevGate *gates, const int *slot_base, const int *occ_ptr,
                     const Occurrence *occ, int P, double *out_energy, double *out_grad,
                     cudaStream_t s);

// --- FP64 norms and inner products (k_norm.cu): per-block partials of ||a||^2, Re <a|b>,
// Im <a|b>, ||b||^2, ||a - b||^2 into partials[v * nb + block], v = 0..4 (kNormValues);
// b = nullptr means b = a.
constexpr int kNormValues = 5;
void launch_norm_dot(const void *a, const void *b, int n, bool dbl, double *partials, int nb, cudaStream_t s);

// --- one kernel per gate (k_gate.cu)
void launch_fwd_gate(void *psi, int n, bool dbl, int kind, int q0, int q1, const double *mat,
                     int nb, cudaStream_t s);
void launch_adj_gate(const void *phi_src, void *phi_dst, void *lam, int n, bool dbl, int kind,
                     int q0, int q1, const double *mat, double *partials, int nb, bool write_phi,
                     bool write_lam, cudaStream_t s);

// --- Hamiltonian (k_pauli.cu)
// Diagonal group: lam = f(j) psi, E partial into partials[0 .. nb).
void launch_pauli_diag(const void *psi, void *lam, int n, bool dbl, const PauliTerm *terms,
                       int count, double *partials, int nb, bool write_lam, cudaStream_t s);
// Group with flip mask x != 0: lam[j] += f(j^x) psi[j^x] (write_lam), E partial.
void launch_pauli_group(const void *psi, void *lam, int n, bool dbl, uint64_t x,
                        const PauliTerm *terms, int count, double *partials, int nb,
                        bool write_lam, cudaStream_t s);

}  // namespace vqg
