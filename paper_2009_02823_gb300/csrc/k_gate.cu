// One kernel per gate: the unfused forward sweep (Algorithm 1's forward sweep, "apply gate")
// and the fused adjoint step (one step of Algorithm 1's reverse loop in one pass):
//   read phi_{i+1} and lambda_i once, reduce the gradient sums, write
//   phi_i = U_i^dag phi_{i+1} and lambda_{i-1} = U_i^dag lambda_i.
// mu = dU_i phi_i is never stored (App. A: dR/dt = -(i/2) sigma R, so
// <lambda_i| dU_i phi_i> = -(i/2) <lambda_i| sigma |phi_{i+1}>).
#include "kernels.h"

namespace vqg {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

// -------------------------------------------------------------------- forward
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads) k_fwd_1q(amp_t<T> *__restrict__ psi, int q,
                                                     const double *__restrict__ mat, uint64_t units) {
    const Mat2<T> u = load_mat<T>(mat);
    const uint64_t bit = 1ull << q;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; base < units;
         base += kUnroll * stride) {
        amp_t<T> a0[kUnroll], a1[kUnroll];
        uint64_t j0[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const uint64_t p = base + k * stride;
            j0[k] = insert0(p, q);
            if (p < units) {
                a0[k] = psi[j0[k]];
                a1[k] = psi[j0[k] | bit];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            if (base + k * stride >= units) continue;
            if (KIND == K_RZ || KIND == K_PHASE) {  // diagonal
                a0[k] = cmul<T>(u.m[0], a0[k]);
                a1[k] = cmul<T>(u.m[3], a1[k]);
            } else if (KIND == K_RY) {  // real matrix
                const T c = u.m[0].x, s = u.m[2].x;
                const amp_t<T> b0 = mk<T>(c * a0[k].x - s * a1[k].x, c * a0[k].y - s * a1[k].y);
                const amp_t<T> b1 = mk<T>(s * a0[k].x + c * a1[k].x, s * a0[k].y + c * a1[k].y);
                a0[k] = b0;
                a1[k] = b1;
            } else {
                apply2<T>(u, a0[k], a1[k]);
            }
            psi[j0[k]] = a0[k];
            psi[j0[k] | bit] = a1[k];
        }
    }
}

// CNOT(c -> t): swap the pair on t where c = 1.  units = 2^{n-2}.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fwd_cnot(amp_t<T> *__restrict__ psi, int c, int t,
                                                       uint64_t units) {
    const int lo = c < t ? c : t, hi = c < t ? t : c;
    const uint64_t cb = 1ull << c, tb = 1ull << t;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < units; u += stride) {
        const uint64_t j = insert00(u, lo, hi) | cb;
        const amp_t<T> a = psi[j], b = psi[j | tb];
        psi[j] = b;
        psi[j | tb] = a;
    }
}

// C_c[U]: the gate's 2x2 matrix on t where c = 1 (controlled rotations and the
// controlled phase gate, App. A).  units = 2^{n-2}.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fwd_c1q(amp_t<T> *__restrict__ psi, int c, int t,
                                                      const double *__restrict__ mat, uint64_t units) {
    const Mat2<T> u = load_mat<T>(mat);
    const int lo = c < t ? c : t, hi = c < t ? t : c;
    const uint64_t cb = 1ull << c, tb = 1ull << t;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < units; v += stride) {
        const uint64_t j = insert00(v, lo, hi) | cb;
        amp_t<T> a0 = psi[j], a1 = psi[j | tb];
        apply2<T>(u, a0, a1);
        psi[j] = a0;
        psi[j | tb] = a1;
    }
}

// CZ(a, b): negate amplitudes with both bits set.  units = 2^{n-2}.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fwd_cz(amp_t<T> *__restrict__ psi, int a, int b,
                                                     uint64_t units) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const uint64_t m = (1ull << a) | (1ull << b);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < units; u += stride) {
        const uint64_t j = insert00(u, lo, hi) | m;
        const amp_t<T> v = psi[j];
        psi[j] = mk<T>(-v.x, -v.y);
    }
}

template <typename T>
static void fwd_gate_t(void *psi, int n, int kind, int q0, int q1, const double *mat, int nb,
                       cudaStream_t s) {
    amp_t<T> *p = (amp_t<T> *)psi;
    const uint64_t pairs = 1ull << (n - 1);
    switch (kind) {
    case K_RX: k_fwd_1q<T, K_RX><<<nb, kThreads, 0, s>>>(p, q0, mat, pairs); break;
    case K_RY: k_fwd_1q<T, K_RY><<<nb, kThreads, 0, s>>>(p, q0, mat, pairs); break;
    case K_RZ: k_fwd_1q<T, K_RZ><<<nb, kThreads, 0, s>>>(p, q0, mat, pairs); break;
    case K_U3: k_fwd_1q<T, K_U3><<<nb, kThreads, 0, s>>>(p, q0, mat, pairs); break;
    case K_CNOT: k_fwd_cnot<T><<<nb, kThreads, 0, s>>>(p, q0, q1, pairs >> 1); break;
    case K_CZ: k_fwd_cz<T><<<nb, kThreads, 0, s>>>(p, q0, q1, pairs >> 1); break;
    case K_PHASE: k_fwd_1q<T, K_PHASE><<<nb, kThreads, 0, s>>>(p, q0, mat, pairs); break;
    case K_CRX:
    case K_CRY:
    case K_CRZ:
    case K_CPHASE: k_fwd_c1q<T><<<nb, kThreads, 0, s>>>(p, q0, q1, mat, pairs >> 1); break;
    default: break;
    }
}

void launch_fwd_gate(void *psi, int n, bool dbl, int kind, int q0, int q1, const double *mat,
                     int nb, cudaStream_t s) {
    if (dbl) fwd_gate_t<double>(psi, n, kind, q0, q1, mat, nb, s);
    else fwd_gate_t<float>(psi, n, kind, q0, q1, mat, nb, s);
}

// -------------------------------------------------------------------- adjoint
// Accumulator policy: products are formed in T; for complex64 they are summed in FP32
// over runs of at most kChunk pairs per thread, then promoted; every level above
// (thread run -> thread total -> warp -> block -> grid) is FP64.
constexpr int kChunk = 16;

template <typename T, int KIND> struct NV { static constexpr int value = reduce_values_of(KIND); };

// Reduction values of one pair (phi_{i+1}: a0, a1; lambda_i: l0, l1).
template <typename T, int KIND>
VQG_DEV void pair_values(const amp_t<T> &a0, const amp_t<T> &a1, const amp_t<T> &l0,
                         const amp_t<T> &l1, T *v) {
    if (KIND == K_RX || KIND == K_CRX) {  // Im(conj(l0) a1 + conj(l1) a0)
        v[0] = (l0.x * a1.y - l0.y * a1.x) + (l1.x * a0.y - l1.y * a0.x);
    } else if (KIND == K_RY || KIND == K_CRY) {  // Re(conj(l1) a0) - Re(conj(l0) a1)
        v[0] = (l1.x * a0.x + l1.y * a0.y) - (l0.x * a1.x + l0.y * a1.y);
    } else if (KIND == K_RZ || KIND == K_CRZ) {  // Im(conj(l0) a0) - Im(conj(l1) a1)
        v[0] = (l0.x * a0.y - l0.y * a0.x) - (l1.x * a1.y - l1.y * a1.x);
    } else if (KIND == K_PHASE || KIND == K_CPHASE) {
        // dP/dt = i e^{it}|1><1| (App. A): 2 Re<lambda| i |1><1| phi_{i+1}> = -2 Im(conj(l1) a1)
        v[0] = (T)-2 * (l1.x * a1.y - l1.y * a1.x);
    } else if (KIND == K_U3) {  // o_rc = conj(l_r) a_c, order 00, 01, 10, 11
        const amp_t<T> o00 = cconjmul<T>(l0, a0), o01 = cconjmul<T>(l0, a1);
        const amp_t<T> o10 = cconjmul<T>(l1, a0), o11 = cconjmul<T>(l1, a1);
        v[0] = o00.x; v[1] = o00.y; v[2] = o01.x; v[3] = o01.y;
        v[4] = o10.x; v[5] = o10.y; v[6] = o11.x; v[7] = o11.y;
    }
}

// Pairs on qubit q (for CNOT/CZ and the controlled kinds: on the target q1; q0 is the
// control / other qubit).  A controlled kind reduces and un-applies only the pairs whose
// control is 1: its derivative is projected onto control = 1 (App. A).
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads)
    k_adj(const amp_t<T> *__restrict__ phi_src, amp_t<T> *__restrict__ phi_dst,
          amp_t<T> *__restrict__ lam, int q0, int q1, const double *__restrict__ mat, uint64_t units,
          double *__restrict__ partials, int nb, int write_phi, int write_lam) {
    constexpr int NVAL = reduce_values_of(KIND);
    constexpr int NVA = NVAL > 0 ? NVAL : 1;
    constexpr bool CTRL = is_controlled_param(KIND);
    const int qp = (KIND == K_CNOT || KIND == K_CZ || CTRL) ? q1 : q0;
    const uint64_t bit = 1ull << qp;
    const uint64_t cbit = 1ull << q0;
    Mat2<T> ud;
    if (has_matrix(KIND)) ud = load_mat_dagger<T>(mat);
    double acc[NVA];
    T run[NVA];
#pragma unroll
    for (int v = 0; v < NVA; ++v) acc[v] = 0.0, run[v] = (T)0;
    int in_run = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; base < units;
         base += kUnroll * stride) {
        amp_t<T> a0[kUnroll], a1[kUnroll], l0[kUnroll], l1[kUnroll];
        uint64_t j0[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const uint64_t p = base + k * stride;
            j0[k] = insert0(p, qp);
            if (p < units) {
                a0[k] = phi_src[j0[k]];
                a1[k] = phi_src[j0[k] | bit];
                l0[k] = lam[j0[k]];
                l1[k] = lam[j0[k] | bit];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            if (base + k * stride >= units) continue;
            const bool active = !CTRL || (j0[k] & cbit) != 0;
            if (NVAL > 0 && active) {
                T v[NVA];
                pair_values<T, KIND>(a0[k], a1[k], l0[k], l1[k], v);
#pragma unroll
                for (int x = 0; x < NVA; ++x) run[x] += v[x];
                if (++in_run == kChunk) {
#pragma unroll
                    for (int x = 0; x < NVA; ++x) acc[x] += (double)run[x], run[x] = (T)0;
                    in_run = 0;
                }
            }
            if (KIND == K_CNOT) {
                if (j0[k] & cbit) {
                    amp_t<T> t = a0[k]; a0[k] = a1[k]; a1[k] = t;
                    t = l0[k]; l0[k] = l1[k]; l1[k] = t;
                }
            } else if (KIND == K_CZ) {
                if (j0[k] & cbit) {
                    a1[k] = mk<T>(-a1[k].x, -a1[k].y);
                    l1[k] = mk<T>(-l1[k].x, -l1[k].y);
                }
            } else if (KIND == K_RZ || KIND == K_PHASE) {
                a0[k] = cmul<T>(ud.m[0], a0[k]); a1[k] = cmul<T>(ud.m[3], a1[k]);
                l0[k] = cmul<T>(ud.m[0], l0[k]); l1[k] = cmul<T>(ud.m[3], l1[k]);
            } else if (CTRL) {
                if (active) {
                    apply2<T>(ud, a0[k], a1[k]);
                    apply2<T>(ud, l0[k], l1[k]);
                }
            } else if (KIND == K_RY) {
                const T c = ud.m[0].x, s = ud.m[2].x;  // U^dag = [[c, s], [-s, c]]
                amp_t<T> b0 = mk<T>(c * a0[k].x + ud.m[1].x * a1[k].x, c * a0[k].y + ud.m[1].x * a1[k].y);
                amp_t<T> b1 = mk<T>(s * a0[k].x + c * a1[k].x, s * a0[k].y + c * a1[k].y);
                a0[k] = b0; a1[k] = b1;
                b0 = mk<T>(c * l0[k].x + ud.m[1].x * l1[k].x, c * l0[k].y + ud.m[1].x * l1[k].y);
                b1 = mk<T>(s * l0[k].x + c * l1[k].x, s * l0[k].y + c * l1[k].y);
                l0[k] = b0; l1[k] = b1;
            } else {
                apply2<T>(ud, a0[k], a1[k]);
                apply2<T>(ud, l0[k], l1[k]);
            }
            if (write_phi) {
                phi_dst[j0[k]] = a0[k];
                phi_dst[j0[k] | bit] = a1[k];
            }
            if (write_lam) {
                lam[j0[k]] = l0[k];
                lam[j0[k] | bit] = l1[k];
            }
        }
    }
    if (NVAL > 0) {
#pragma unroll
        for (int x = 0; x < NVA; ++x) acc[x] += (double)run[x];
        block_reduce_store<NVA>(acc, partials, nb);
    }
}

template <typename T>
static void adj_gate_t(const void *phi_src, void *phi_dst, void *lam, int n, int kind, int q0,
                       int q1, const double *mat, double *partials, int nb, int wp, int wl,
                       cudaStream_t s) {
    const amp_t<T> *ps = (const amp_t<T> *)phi_src;
    amp_t<T> *pd = (amp_t<T> *)phi_dst, *l = (amp_t<T> *)lam;
    const uint64_t pairs = 1ull << (n - 1);
#define VQG_ADJ(K) k_adj<T, K><<<nb, kThreads, 0, s>>>(ps, pd, l, q0, q1, mat, pairs, partials, nb, wp, wl)
    switch (kind) {
    case K_RX: VQG_ADJ(K_RX); break;
    case K_RY: VQG_ADJ(K_RY); break;
    case K_RZ: VQG_ADJ(K_RZ); break;
    case K_U3: VQG_ADJ(K_U3); break;
    case K_CNOT: VQG_ADJ(K_CNOT); break;
    case K_CZ: VQG_ADJ(K_CZ); break;
    case K_CRX: VQG_ADJ(K_CRX); break;
    case K_CRY: VQG_ADJ(K_CRY); break;
    case K_CRZ: VQG_ADJ(K_CRZ); break;
    case K_PHASE: VQG_ADJ(K_PHASE); break;
    case K_CPHASE: VQG_ADJ(K_CPHASE); break;
    default: break;
    }
#undef VQG_ADJ
}

void launch_adj_gate(const void *phi_src, void *phi_dst, void *lam, int n, bool dbl, int kind,
                     int q0, int q1, const double *mat, double *partials, int nb, bool write_phi,
                     bool write_lam, cudaStream_t s) {
    if (dbl) adj_gate_t<double>(phi_src, phi_dst, lam, n, kind, q0, q1, mat, partials, nb, write_phi, write_lam, s);
    else adj_gate_t<float>(phi_src, phi_dst, lam, n, kind, q0, q1, mat, partials, nb, write_phi, write_lam, s);
}

}  // namespace vqg
