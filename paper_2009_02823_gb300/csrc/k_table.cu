// Gate-table construction, state initialisation and the deterministic second-stage
// reductions that turn per-block partial sums into E and the gradient.
#include "grad.cuh"
#include "kernels.h"

namespace vqg {

// U_i(theta) for every gate with a parameter, FP64, row-major (re, im) x 4 (App. A gate
// set): R_sigma(t) = cos(t/2) I - i sin(t/2) sigma;  U3 per the ABI header; the phase
// gate diag(1, e^{it}); controlled kinds store the matrix applied to their target.
// shift_gate/shift_slot add `shift` to one parameter slot of one occurrence (the
// per-occurrence parameter-shift baseline).
__global__ void k_build_mats(const double *__restrict__ theta, const DevGate *__restrict__ gates,
                             int G, double *__restrict__ mats, float *__restrict__ mats_f,
                             int shift_gate, int shift_slot, double shift) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    DevGate g = gates[i];
    double a[3] = {0.0, 0.0, 0.0};
    if (has_matrix(g.kind)) {
        a[0] = theta[g.p0];
        if (g.kind == K_U3) {
            a[1] = theta[g.p1];
            a[2] = theta[g.p2];
        }
    }
    if (i == shift_gate && shift_slot >= 0) a[shift_slot] += shift;
    double s, c;
    sincos(0.5 * a[0], &s, &c);
    double *m = mats + 8 * (size_t)i;
    double r[8] = {1, 0, 0, 0, 0, 0, 1, 0};
    int kind = g.kind;
    if (kind >= K_CRX && kind <= K_CRZ) kind -= K_CRX - K_RX;  // target matrix of C[R_sigma]
    switch (kind) {
    case K_RX:  // [[c, -i s], [-i s, c]]
        r[0] = c; r[1] = 0; r[2] = 0; r[3] = -s; r[4] = 0; r[5] = -s; r[6] = c; r[7] = 0;
        break;
    case K_RY:  // [[c, -s], [s, c]]
        r[0] = c; r[1] = 0; r[2] = -s; r[3] = 0; r[4] = s; r[5] = 0; r[6] = c; r[7] = 0;
        break;
    case K_RZ:  // diag(e^{-it/2}, e^{it/2})
        r[0] = c; r[1] = -s; r[2] = 0; r[3] = 0; r[4] = 0; r[5] = 0; r[6] = c; r[7] = s;
        break;
    case K_U3: {  // [[c, -e^{il} s], [e^{if} s, e^{i(f+l)} c]]
        double sf, cf, sl, cl, sfl, cfl;
        sincos(a[1], &sf, &cf);
        sincos(a[2], &sl, &cl);
        sincos(a[1] + a[2], &sfl, &cfl);
        r[0] = c; r[1] = 0;
        r[2] = -cl * s; r[3] = -sl * s;
        r[4] = cf * s; r[5] = sf * s;
        r[6] = cfl * c; r[7] = sfl * c;
        break;
    }
    case K_PHASE:
    case K_CPHASE: {  // diag(1, e^{it})
        double st, ct;
        sincos(a[0], &st, &ct);
        r[0] = 1; r[1] = 0; r[2] = 0; r[3] = 0; r[4] = 0; r[5] = 0; r[6] = ct; r[7] = st;
        break;
    }
    default:
        break;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = r[k];
    if (mats_f) {
#pragma unroll
        for (int k = 0; k < 8; ++k) mats_f[8 * (size_t)i + k] = (float)r[k];
    }
}

void launch_build_mats(const double *theta, const DevGate *gates, int G, double *mats,
                       float *mats_f, int shift_gate, int shift_slot, double shift, cudaStream_t s) {
    if (G <= 0) return;
    k_build_mats<<<(G + 127) / 128, 128, 0, s>>>(theta, gates, G, mats, mats_f, shift_gate,
                                                 shift_slot, shift);
}

template <typename T>
__global__ void k_init_zero(amp_t<T> *__restrict__ psi, uint64_t dim) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < dim; j += stride)
        psi[j] = mk<T>(j == 0 ? (T)1 : (T)0, (T)0);
}

void launch_init_zero(void *psi, int n, bool dbl, int nb, cudaStream_t s) {
    const uint64_t dim = 1ull << n;
    if (dbl) k_init_zero<double><<<nb, 256, 0, s>>>((double2 *)psi, dim);
    else k_init_zero<float><<<nb, 256, 0, s>>>((float2 *)psi, dim);
}

// red[s] = sum_b partials[s * nb + b] in a fixed order (one warp per slot).
__global__ void k_reduce_slots(const double *__restrict__ partials, int n_slots, int nb,
                               double *__restrict__ red) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_slots) return;
    const double *p = partials + (size_t)warp * nb;
    double acc = 0.0;
    for (int b = lane; b < nb; b += 32) acc += p[b];
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
}

void launch_reduce_slots(const double *partials, int n_slots, int nb, double *red, cudaStream_t s) {
    if (n_slots <= 0) return;
    const int threads = 256, warps_per_block = threads / 32;
    k_reduce_slots<<<(n_slots + warps_per_block - 1) / warps_per_block, threads, 0, s>>>(
        partials, n_slots, nb, red);
}

__global__ void k_finalize(const double *__restrict__ red_e, int e_count,
                           const double *__restrict__ red_g, const double *__restrict__ theta, const DevGate *__restrict__ gates,
                           const int *__restrict__ slot_base, const int *__restrict__ occ_ptr,
                           const Occurrence *__restrict__ occ, int P, double *out_energy,
                           double *out_grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && out_energy) {
        double e = 0.0;
        for (int k = 0; k < e_count; ++k) e += red_e[k];
        *out_energy = e;
    }
    if (p >= P || !out_grad) return;
    double g = 0.0;
    for (int k = occ_ptr[p]; k < occ_ptr[p + 1]; ++k) {
        const Occurrence o = occ[k];
        const DevGate gt = gates[o.gate];
        const double *v = red_g + slot_base[o.gate];
        if (gt.kind == K_U3) {
            double a[3] = {theta[gt.p0], theta[gt.p1], theta[gt.p2]};
            g += u3_slot_contribution(a, o.slot, v);
        } else {
            g += v[0];  // Im <lambda|sigma|phi> = 2 Re <lambda|(-i/2) sigma U|phi_i>
        }
    }
    out_grad[p] = g;
}

void launch_finalize(const double *red_e, int e_count, const double *red_g, const double *theta,
                     const DevGate *gates, const int *slot_base, const int *occ_ptr,
                     const Occurrence *occ, int P, double *out_energy, double *out_grad,
                     cudaStream_t s) {
    const int n = P > 0 ? P : 1;
    k_finalize<<<(n + 127) / 128, 128, 0, s>>>(red_e, e_count, red_g, theta, gates, slot_base,
                                               occ_ptr, occ, P, out_energy, out_grad);
}

}  // namespace vqg
