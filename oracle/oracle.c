/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct complex128 state-vector simulator used to check
 * the CUDA path.  Only tests/, the smoke check and bench.py's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Jones & Gacon, "Efficient calculation of gradients in classical
 * simulations of variational quantum algorithms"):
 *   - |psi(theta)> = U_G(theta) ... U_1(theta) |in>, |in> = |0...0>      (Sec. 2.2)
 *   - E = <psi|H|psi> for a Pauli sum H                                    (Sec. 2.2)
 *   - the gradient dE/dtheta_p by three independent routes:
 *       (a) per-occurrence parameter shift, the "faithful" O(P^2) emulation of the
 *           quantum evaluation (Sec. 1, Sec. 3);
 *       (b) Algorithm 2 (the reference gradient of Eq. reference_gradient): for every
 *           gate occurrence, rebuild the state with the gate replaced by its
 *           derivative matrix (App. A) and take 2 Re <lambda|mu>;
 *       (c) Algorithm 1 ("reverse mode") in the paper's own order with three
 *           working states lambda, phi, mu (Sec. 2.3; App. B.1 for multi-parameter
 *           gates; App. B.2's chain-rule sum for repeated parameters).
 *
 * Conventions (readings where the paper is silent):
 *   qubit q <-> bit q of the amplitude index (little endian);
 *   R_sigma(t) = exp(-i t sigma / 2), i.e. App. A's exp(alpha i t sigma) with alpha = -1/2;
 *   U3(t, f, l) = [[c, -e^{il} s], [e^{if} s, e^{i(f+l)} c]], c = cos(t/2), s = sin(t/2);
 *   CNOT(c -> t) flips t where c = 1; CZ(a, b) negates amplitudes with both bits 1;
 *   CRX/CRY/CRZ(c -> t, t) apply R_sigma(t) to qubit t where qubit c = 1 (App. A's
 *   C_c[U]); PHASE(t) = diag(1, e^{it}) (App. A); CPHASE(a, b, t) multiplies amplitudes
 *   with both bits 1 by e^{it} (= C_a[PHASE on b]);
 *   a Pauli term is coef * (tensor product of per-qubit letters), applied here letter
 *   by letter as 2x2 matrices (no bit-mask algebra).
 *
 * Gate record: 6 int32 per gate = kind, q0, q1, param0, param1, param2
 *   kind 0 RX, 1 RY, 2 RZ, 3 U3, 4 CNOT, 5 CZ, 6 CRX, 7 CRY, 8 CRZ, 9 PHASE, 10 CPHASE;
 *   controlled kinds: q0 = control, q1 = target; unused params are -1.
 * Hamiltonian: n_terms coefficients and an n_terms x n table of letters
 *   (0 = I, 1 = X, 2 = Y, 3 = Z), letters[t * n + q] acting on qubit q.  A non-Hermitian
 *   operator (App. B.4) has complex coefficients, given as separate real and imaginary
 *   arrays.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum {
    OR_RX = 0, OR_RY = 1, OR_RZ = 2, OR_U3 = 3, OR_CNOT = 4, OR_CZ = 5,
    OR_CRX = 6, OR_CRY = 7, OR_CRZ = 8, OR_PHASE = 9, OR_CPHASE = 10
};

#define PAR_FOR _Pragma("omp parallel for schedule(static) if (dim >= 16384)")

static int n_params_of(int kind) {
    if (kind == OR_U3) return 3;
    if (kind == OR_RX || kind == OR_RY || kind == OR_RZ) return 1;
    if (kind >= OR_CRX && kind <= OR_CPHASE) return 1;
    return 0;
}

/* Control qubit of a controlled parameterised gate (-1: none) and the qubit its 2x2
 * matrix acts on. */
static int control_of(const int32_t *g) {
    return (g[0] >= OR_CRX && g[0] <= OR_CRZ) || g[0] == OR_CPHASE ? g[1] : -1;
}
static int target_of(const int32_t *g) { return control_of(g) >= 0 ? g[2] : g[1]; }

int oracle_n_params_of_kind(int kind) { return n_params_of(kind); }

/* ---------------------------------------------------------------- gate matrices */

/* 2x2 matrix (row-major m[0]=m00, m[1]=m01, m[2]=m10, m[3]=m11) of a one-qubit gate
 * at angles a[0..2] (only a[0] for rotations); for a controlled kind, the matrix applied
 * to the target where the control is 1. */
void oracle_gate_matrix(int kind, const double *a, cplx *m) {
    double c = cos(a[0] / 2.0), s = sin(a[0] / 2.0);
    if (kind >= OR_CRX && kind <= OR_CRZ) kind -= OR_CRX - OR_RX;  /* same 2x2 as RX/RY/RZ */
    switch (kind) {
    case OR_RX: /* exp(-i t X / 2) = cos(t/2) I - i sin(t/2) X */
        m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case OR_RY: /* exp(-i t Y / 2) = cos(t/2) I - i sin(t/2) Y */
        m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    case OR_RZ: /* exp(-i t Z / 2) */
        m[0] = cexp(-I * a[0] / 2.0); m[1] = 0; m[2] = 0; m[3] = cexp(I * a[0] / 2.0); break;
    case OR_U3:
        m[0] = c;
        m[1] = -cexp(I * a[2]) * s;
        m[2] = cexp(I * a[1]) * s;
        m[3] = cexp(I * (a[1] + a[2])) * c;
        break;
    case OR_PHASE:
    case OR_CPHASE: /* diag(1, e^{it}) */
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * a[0]); break;
    default:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 1;
    }
}

/* Derivative of the gate matrix with respect to its slot-th parameter (App. A).
 * Rotations: d/dt exp(-i t s/2) = (-i/2) s exp(-i t s/2); U3 element-wise. */
void oracle_gate_derivative(int kind, int slot, const double *a, cplx *d) {
    double c = cos(a[0] / 2.0), s = sin(a[0] / 2.0);
    cplx m[4];
    if (kind >= OR_CRX && kind <= OR_CRZ) kind -= OR_CRX - OR_RX;  /* target part; App. A projects */
    switch (kind) {
    case OR_RX: /* (-i/2) X R */
        oracle_gate_matrix(kind, a, m);
        d[0] = -0.5 * I * m[2]; d[1] = -0.5 * I * m[3];
        d[2] = -0.5 * I * m[0]; d[3] = -0.5 * I * m[1];
        break;
    case OR_RY: /* (-i/2) Y R, Y = [[0,-i],[i,0]] */
        oracle_gate_matrix(kind, a, m);
        d[0] = -0.5 * I * (-I * m[2]); d[1] = -0.5 * I * (-I * m[3]);
        d[2] = -0.5 * I * (I * m[0]);  d[3] = -0.5 * I * (I * m[1]);
        break;
    case OR_RZ: /* (-i/2) Z R */
        oracle_gate_matrix(kind, a, m);
        d[0] = -0.5 * I * m[0]; d[1] = 0; d[2] = 0; d[3] = 0.5 * I * m[3];
        break;
    case OR_U3:
        if (slot == 0) {        /* d/d theta */
            d[0] = -0.5 * s;
            d[1] = -cexp(I * a[2]) * 0.5 * c;
            d[2] = cexp(I * a[1]) * 0.5 * c;
            d[3] = -cexp(I * (a[1] + a[2])) * 0.5 * s;
        } else if (slot == 1) { /* d/d phi */
            d[0] = 0; d[1] = 0;
            d[2] = I * cexp(I * a[1]) * s;
            d[3] = I * cexp(I * (a[1] + a[2])) * c;
        } else {                /* d/d lambda */
            d[0] = 0;
            d[1] = -I * cexp(I * a[2]) * s;
            d[2] = 0;
            d[3] = I * cexp(I * (a[1] + a[2])) * c;
        }
        break;
    case OR_PHASE:
    case OR_CPHASE: /* i e^{it} |1><1| (App. A) */
        d[0] = 0; d[1] = 0; d[2] = 0; d[3] = I * cexp(I * a[0]); break;
    default:
        d[0] = d[1] = d[2] = d[3] = 0;
    }
}

/* ------------------------------------------------------------- state primitives */

/* "apply gate": a 2x2 matrix (not necessarily unitary) on qubit q. */
void oracle_apply_matrix_1q(int n, cplx *psi, int q, const cplx *m) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
    PAR_FOR
    for (int64_t j = 0; j < dim; ++j) {
        if (j & bit) continue;
        cplx a0 = psi[j], a1 = psi[j | bit];
        psi[j] = m[0] * a0 + m[1] * a1;
        psi[j | bit] = m[2] * a0 + m[3] * a1;
    }
}

/* C_c[m]: the 2x2 matrix m on qubit t where qubit c is 1 (identity elsewhere). */
void oracle_apply_controlled_1q(int n, cplx *psi, int c, int t, const cplx *m) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t cb = (int64_t)1 << c, tb = (int64_t)1 << t;
    PAR_FOR
    for (int64_t j = 0; j < dim; ++j) {
        if ((j & tb) || !(j & cb)) continue;
        cplx a0 = psi[j], a1 = psi[j | tb];
        psi[j] = m[0] * a0 + m[1] * a1;
        psi[j | tb] = m[2] * a0 + m[3] * a1;
    }
}

/* The derivative of a controlled gate (App. A): d on qubit t, then the amplitudes whose
 * control qubit c is not 1 are overwritten with 0. */
void oracle_apply_projected_1q(int n, cplx *psi, int c, int t, const cplx *d) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t cb = (int64_t)1 << c;
    oracle_apply_matrix_1q(n, psi, t, d);
    PAR_FOR
    for (int64_t j = 0; j < dim; ++j)
        if (!(j & cb)) psi[j] = 0;
}

void oracle_apply_cnot(int n, cplx *psi, int control, int target) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t cb = (int64_t)1 << control, tb = (int64_t)1 << target;
    PAR_FOR
    for (int64_t j = 0; j < dim; ++j) {
        if ((j & cb) && !(j & tb)) {
            cplx t = psi[j];
            psi[j] = psi[j | tb];
            psi[j | tb] = t;
        }
    }
}

void oracle_apply_cz(int n, cplx *psi, int a, int b) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t ab = (int64_t)1 << a, bb = (int64_t)1 << b;
    PAR_FOR
    for (int64_t j = 0; j < dim; ++j)
        if ((j & ab) && (j & bb)) psi[j] = -psi[j];
}

static void gate_angles(const int32_t *g, const double *theta, double *a) {
    a[0] = a[1] = a[2] = 0.0;
    int k = n_params_of(g[0]);
    for (int j = 0; j < k; ++j) a[j] = theta[g[3 + j]];
}

/* Apply gate g, or its adjoint when dagger != 0.  shift_slot >= 0 adds `shift` to
 * that parameter slot of this gate only (per-occurrence parameter shift). */
static void apply_gate_ex(int n, cplx *psi, const int32_t *g, const double *theta, int dagger,
                          int shift_slot, double shift) {
    int kind = g[0];
    if (kind == OR_CNOT) { oracle_apply_cnot(n, psi, g[1], g[2]); return; }
    if (kind == OR_CZ) { oracle_apply_cz(n, psi, g[1], g[2]); return; }
    double a[3];
    gate_angles(g, theta, a);
    if (shift_slot >= 0) a[shift_slot] += shift;
    cplx m[4];
    oracle_gate_matrix(kind, a, m);
    if (dagger) {
        cplx t[4] = {conj(m[0]), conj(m[2]), conj(m[1]), conj(m[3])};
        m[0] = t[0]; m[1] = t[1]; m[2] = t[2]; m[3] = t[3];
    }
    if (control_of(g) >= 0) oracle_apply_controlled_1q(n, psi, control_of(g), target_of(g), m);
    else oracle_apply_matrix_1q(n, psi, target_of(g), m);
}

/* mu <- (dU_g / d slot) mu: the derivative matrix on the target, projected onto
 * control = 1 for controlled kinds (App. A). */
static void apply_gate_derivative(int n, cplx *mu, const int32_t *g, const double *theta, int slot) {
    double a[3];
    gate_angles(g, theta, a);
    cplx d[4];
    oracle_gate_derivative(g[0], slot, a, d);
    if (control_of(g) >= 0) oracle_apply_projected_1q(n, mu, control_of(g), target_of(g), d);
    else oracle_apply_matrix_1q(n, mu, target_of(g), d);
}

void oracle_apply_gate(int n, cplx *psi, const int32_t *g, const double *theta, int dagger) {
    apply_gate_ex(n, psi, g, theta, dagger, -1, 0.0);
}

void oracle_zero_state(int n, cplx *psi) {
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(cplx) * (size_t)dim);
    psi[0] = 1.0;
}

/* |psi> = U_{first..last-1} |psi> applied in gate order. */
void oracle_apply_gates(int n, cplx *psi, const int32_t *gates, int first, int last,
                        const double *theta) {
    for (int i = first; i < last; ++i) oracle_apply_gate(n, psi, gates + 6 * i, theta, 0);
}

/* |psi(theta)> = U_G ... U_1 |0...0>  (Sec. 2.2). */
void oracle_prepare_state(int n, const int32_t *gates, int n_gates, const double *theta,
                          cplx *psi) {
    oracle_zero_state(n, psi);
    oracle_apply_gates(n, psi, gates, 0, n_gates, theta);
}

/* "inner product" <a|b>. */
cplx oracle_inner(int n, const cplx *a, const cplx *b) {
    const int64_t dim = (int64_t)1 << n;
    double re = 0.0, im = 0.0;
    _Pragma("omp parallel for schedule(static) reduction(+:re,im) if (dim >= 16384)")
    for (int64_t j = 0; j < dim; ++j) {
        cplx v = conj(a[j]) * b[j];
        re += creal(v);
        im += cimag(v);
    }
    return re + I * im;
}

void oracle_inner_parts(int n, const cplx *a, const cplx *b, double *out2) {
    cplx v = oracle_inner(n, a, b);
    out2[0] = creal(v);
    out2[1] = cimag(v);
}

/* out = H psi with H = sum_t coef_t * (x)_q sigma_{t,q}: each term is applied to a
 * copy of psi one letter at a time as a plain 2x2 matrix, then accumulated. */
void oracle_apply_hamiltonian(int n, int n_terms, const double *coef, const uint8_t *letters,
                              const cplx *psi, cplx *out) {
    const int64_t dim = (int64_t)1 << n;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    static const cplx PX[4] = {0, 1, 1, 0};
    static const cplx PZ[4] = {1, 0, 0, -1};
    cplx PY[4] = {0, -I, I, 0};
    memset(out, 0, sizeof(cplx) * (size_t)dim);
    for (int t = 0; t < n_terms; ++t) {
        memcpy(tmp, psi, sizeof(cplx) * (size_t)dim);
        for (int q = 0; q < n; ++q) {
            int l = letters[(int64_t)t * n + q];
            if (l == 1) oracle_apply_matrix_1q(n, tmp, q, PX);
            else if (l == 2) oracle_apply_matrix_1q(n, tmp, q, PY);
            else if (l == 3) oracle_apply_matrix_1q(n, tmp, q, PZ);
        }
        const double c = coef[t];
        PAR_FOR
        for (int64_t j = 0; j < dim; ++j) out[j] += c * tmp[j];
    }
    free(tmp);
}

/* out = A psi for A = sum_k c_k (x)_q M_{k,q}, a sum of tensor products of 2x2 matrices
 * (the paper's benchmark operator Hadamard^{(x)N} is one product, Sec. 3): each product
 * applied to a copy of psi qubit by qubit, then accumulated.  mats holds the 2x2
 * matrices row-major, product k qubit q at mats + 4 (k n + q). */
void oracle_apply_product_operator(int n, int n_products, const double *coef, const cplx *mats,
                                   const cplx *psi, cplx *out) {
    const int64_t dim = (int64_t)1 << n;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    memset(out, 0, sizeof(cplx) * (size_t)dim);
    for (int k = 0; k < n_products; ++k) {
        memcpy(tmp, psi, sizeof(cplx) * (size_t)dim);
        for (int q = 0; q < n; ++q) oracle_apply_matrix_1q(n, tmp, q, mats + 4 * ((int64_t)k * n + q));
        const double c = coef[k];
        PAR_FOR
        for (int64_t j = 0; j < dim; ++j) out[j] += c * tmp[j];
    }
    free(tmp);
}

/* The cost operator of the energy and gradient routines: a Pauli sum (letters) or a sum
 * of tensor products (mats), both with real coefficients; and the input state |in>
 * (NULL: |0...0>, Sec. 2.2). */
typedef struct {
    int kind;  /* 0: Pauli sum, 1: tensor products */
    int n_terms;
    const double *coef;
    const uint8_t *letters;
    const cplx *mats;
    const cplx *in;
} Problem;

static void problem_apply(int n, const Problem *pb, const cplx *psi, cplx *out) {
    if (pb->kind == 1) oracle_apply_product_operator(n, pb->n_terms, pb->coef, pb->mats, psi, out);
    else oracle_apply_hamiltonian(n, pb->n_terms, pb->coef, pb->letters, psi, out);
}

static void problem_input(int n, const Problem *pb, cplx *psi) {
    if (pb->in) memcpy(psi, pb->in, sizeof(cplx) * ((size_t)1 << n));
    else oracle_zero_state(n, psi);
}

static double problem_expectation(int n, const Problem *pb, const cplx *psi) {
    const int64_t dim = (int64_t)1 << n;
    cplx *hp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    problem_apply(n, pb, psi, hp);
    double e = creal(oracle_inner(n, psi, hp));
    free(hp);
    return e;
}

/* E = <psi|H|psi> for a given state (real part; H is Hermitian for real coef). */
double oracle_expectation(int n, int n_terms, const double *coef, const uint8_t *letters,
                          const cplx *psi) {
    Problem pb = {0, n_terms, coef, letters, NULL, NULL};
    return problem_expectation(n, &pb, psi);
}

static double energy_shifted(int n, const int32_t *gates, int n_gates, const double *theta,
                             const Problem *pb, int shift_gate, int shift_slot, double shift, cplx *psi) {
    problem_input(n, pb, psi);
    for (int i = 0; i < n_gates; ++i)
        apply_gate_ex(n, psi, gates + 6 * i, theta, 0, i == shift_gate ? shift_slot : -1, shift);
    return problem_expectation(n, pb, psi);
}

/* E(theta) = <in|U^dagger H U|in>  (Sec. 2.2). */
static double energy_pb(int n, const int32_t *gates, int n_gates, const double *theta, const Problem *pb) {
    const int64_t dim = (int64_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    double e = energy_shifted(n, gates, n_gates, theta, pb, -1, -1, 0.0, psi);
    free(psi);
    return e;
}

/* (a) Faithful gradient by per-occurrence parameter-shift rules, occurrences of a shared
 * parameter adding by the chain rule (App. B.2).  As a function of one occurrence's angle
 * t, E is a trigonometric polynomial whose frequencies are the differences of the
 * generator's eigenvalues:
 *   - RX/RY/RZ, U3 (= e^{i(f+l)/2} RZ(f) RY(t) RZ(l), global phase), PHASE (= e^{it/2}
 *     RZ(t)) and CPHASE (generator |11><11|): eigenvalue differences {1}, so
 *     E = a + b cos t + c sin t and dE/dt = [E(t + pi/2) - E(t - pi/2)] / 2 exactly;
 *   - CRX/CRY/CRZ (generator (sigma/2) x |1><1|_c, eigenvalues 0, 0, +-1/2): frequencies
 *     {1/2, 1}.  With D(s) = E(t + s) - E(t - s) = 2 sum_w sin(w s) [w-th derivative
 *     term], requiring a1 D(pi/2) + a2 D(3pi/2) = dE/dt for w = 1/2 and w = 1 gives
 *     a1 + a2 = 1/(2 sqrt 2), a1 - a2 = 1/2, i.e. a1 = (sqrt2 + 1)/(4 sqrt2),
 *     a2 = -(sqrt2 - 1)/(4 sqrt2): a four-term rule, exact.
 * Optional: restrict to gate occurrences [g_first, g_last). */
static void ps_pb(int n, const int32_t *gates, int n_gates, const double *theta, int n_params,
                  const Problem *pb, double *grad, int g_first, int g_last) {
    const int64_t dim = (int64_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    const double h = M_PI / 2.0;
    for (int p = 0; p < n_params; ++p) grad[p] = 0.0;
    if (g_last < 0 || g_last > n_gates) g_last = n_gates;
    for (int i = g_first; i < g_last; ++i) {
        const int32_t *g = gates + 6 * i;
        for (int j = 0; j < n_params_of(g[0]); ++j) {
            double ep = energy_shifted(n, gates, n_gates, theta, pb, i, j, +h, psi);
            double em = energy_shifted(n, gates, n_gates, theta, pb, i, j, -h, psi);
            if (g[0] >= OR_CRX && g[0] <= OR_CRZ) {
                const double r2 = sqrt(2.0);
                const double a1 = (r2 + 1.0) / (4.0 * r2), a2 = -(r2 - 1.0) / (4.0 * r2);
                double ep3 = energy_shifted(n, gates, n_gates, theta, pb, i, j, +3.0 * h, psi);
                double em3 = energy_shifted(n, gates, n_gates, theta, pb, i, j, -3.0 * h, psi);
                grad[g[3 + j]] += a1 * (ep - em) + a2 * (ep3 - em3);
            } else {
                grad[g[3 + j]] += 0.5 * (ep - em);
            }
        }
    }
    free(psi);
}

/* (b) Algorithm 2 ("reference" gradient, Eq. reference_gradient):
 *   lambda = H U_{1:G}|in>;  for each occurrence i (and slot j of a multi-parameter gate):
 *   mu = |in>; mu <- U_{1:i-1} mu; mu <- dU_i/dphi_j mu; mu <- U_{i+1:G} mu;
 *   grad[param] += 2 Re <lambda|mu>. */
static void alg2_pb(int n, const int32_t *gates, int n_gates, const double *theta, int n_params,
                    const Problem *pb, double *grad) {
    const int64_t dim = (int64_t)1 << n;
    cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *mu = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    for (int p = 0; p < n_params; ++p) grad[p] = 0.0;
    problem_input(n, pb, mu);
    oracle_apply_gates(n, mu, gates, 0, n_gates, theta);
    problem_apply(n, pb, mu, lam);
    for (int i = 0; i < n_gates; ++i) {
        const int32_t *g = gates + 6 * i;
        for (int j = 0; j < n_params_of(g[0]); ++j) {
            problem_input(n, pb, mu);
            oracle_apply_gates(n, mu, gates, 0, i, theta);
            apply_gate_derivative(n, mu, g, theta, j);
            oracle_apply_gates(n, mu, gates, i + 1, n_gates, theta);
            grad[g[3 + j]] += 2.0 * creal(oracle_inner(n, lam, mu));
        }
    }
    free(lam);
    free(mu);
}

/* (c) Algorithm 1 ("reverse mode") in the paper's order, three working states:
 *   lambda := in; lambda <- U_{1:G} lambda; phi := lambda; lambda <- H lambda;
 *   for i = G..1: phi <- U_i^dag phi; for each slot j: mu := phi; mu <- dU_i/dphi_j mu;
 *                 grad[param] += 2 Re <lambda|mu>;  if i > 1: lambda <- U_i^dag lambda.
 * Also returns E = Re <phi_{G+1}|lambda_G> (= <psi|H|psi>) through *energy when non-null. */
static void alg1_pb(int n, const int32_t *gates, int n_gates, const double *theta, int n_params,
                    const Problem *pb, double *grad, double *energy) {
    const int64_t dim = (int64_t)1 << n;
    cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *phi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *mu = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    for (int p = 0; p < n_params; ++p) grad[p] = 0.0;
    problem_input(n, pb, lam);
    oracle_apply_gates(n, lam, gates, 0, n_gates, theta);
    memcpy(phi, lam, sizeof(cplx) * (size_t)dim);
    problem_apply(n, pb, phi, lam);
    if (energy) *energy = creal(oracle_inner(n, phi, lam));
    for (int i = n_gates - 1; i >= 0; --i) {
        const int32_t *g = gates + 6 * i;
        oracle_apply_gate(n, phi, g, theta, 1);
        for (int j = 0; j < n_params_of(g[0]); ++j) {
            memcpy(mu, phi, sizeof(cplx) * (size_t)dim);
            apply_gate_derivative(n, mu, g, theta, j);
            grad[g[3 + j]] += 2.0 * creal(oracle_inner(n, lam, mu));
        }
        if (i > 0) oracle_apply_gate(n, lam, g, theta, 1);
    }
    free(lam);
    free(phi);
    free(mu);
}

/* Pauli-sum operator, |in> = |0...0>. */
double oracle_energy(int n, const int32_t *gates, int n_gates, const double *theta, int n_terms,
                     const double *coef, const uint8_t *letters) {
    Problem pb = {0, n_terms, coef, letters, NULL, NULL};
    return energy_pb(n, gates, n_gates, theta, &pb);
}

void oracle_gradient_parameter_shift(int n, const int32_t *gates, int n_gates,
                                     const double *theta, int n_params, int n_terms,
                                     const double *coef, const uint8_t *letters, double *grad,
                                     int g_first, int g_last) {
    Problem pb = {0, n_terms, coef, letters, NULL, NULL};
    ps_pb(n, gates, n_gates, theta, n_params, &pb, grad, g_first, g_last);
}

void oracle_gradient_alg2(int n, const int32_t *gates, int n_gates, const double *theta,
                          int n_params, int n_terms, const double *coef, const uint8_t *letters,
                          double *grad) {
    Problem pb = {0, n_terms, coef, letters, NULL, NULL};
    alg2_pb(n, gates, n_gates, theta, n_params, &pb, grad);
}

void oracle_gradient_alg1(int n, const int32_t *gates, int n_gates, const double *theta,
                          int n_params, int n_terms, const double *coef, const uint8_t *letters,
                          double *grad, double *energy) {
    Problem pb = {0, n_terms, coef, letters, NULL, NULL};
    alg1_pb(n, gates, n_gates, theta, n_params, &pb, grad, energy);
}

/* General problem: op_kind 0 (Pauli sum: letters) or 1 (tensor products: mats), input
 * state in_state (NULL: |0...0>).  route 0: parameter shift, 1: Algorithm 2,
 * 2: Algorithm 1 (energy returned through *energy when non-null). */
void oracle_gradient_ex(int route, int n, const int32_t *gates, int n_gates, const double *theta,
                        int n_params, int op_kind, int n_terms, const double *coef,
                        const uint8_t *letters, const cplx *mats, const cplx *in_state,
                        double *grad, double *energy) {
    Problem pb = {op_kind, n_terms, coef, letters, mats, in_state};
    if (route == 0) ps_pb(n, gates, n_gates, theta, n_params, &pb, grad, 0, -1);
    else if (route == 1) alg2_pb(n, gates, n_gates, theta, n_params, &pb, grad);
    else alg1_pb(n, gates, n_gates, theta, n_params, &pb, grad, energy);
    if (energy && route != 2) *energy = energy_pb(n, gates, n_gates, theta, &pb);
}

/* ------------------------------------------------- non-Hermitian operators (App. B.4) */

/* out = A psi for A = sum_t (cr_t + i ci_t) (x)_q sigma_{t,q}: each term applied to a copy
 * of psi letter by letter as plain 2x2 matrices, then accumulated with its complex
 * coefficient. */
void oracle_apply_operator(int n, int n_terms, const double *cr, const double *ci,
                           const uint8_t *letters, const cplx *psi, cplx *out) {
    const int64_t dim = (int64_t)1 << n;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    static const cplx PX[4] = {0, 1, 1, 0};
    static const cplx PZ[4] = {1, 0, 0, -1};
    cplx PY[4] = {0, -I, I, 0};
    memset(out, 0, sizeof(cplx) * (size_t)dim);
    for (int t = 0; t < n_terms; ++t) {
        memcpy(tmp, psi, sizeof(cplx) * (size_t)dim);
        for (int q = 0; q < n; ++q) {
            int l = letters[(int64_t)t * n + q];
            if (l == 1) oracle_apply_matrix_1q(n, tmp, q, PX);
            else if (l == 2) oracle_apply_matrix_1q(n, tmp, q, PY);
            else if (l == 3) oracle_apply_matrix_1q(n, tmp, q, PZ);
        }
        const cplx c = cr[t] + I * ci[t];
        PAR_FOR
        for (int64_t j = 0; j < dim; ++j) out[j] += c * tmp[j];
    }
    free(tmp);
}

/* Algorithm 1 with App. B.4's change of the step value to <lambda|mu> (complex, no
 * 2 Re), for the operator with coefficients (cr, ci): g[p] += <lambda_i|mu_i>.
 * Returns <psi|lambda_G> = <psi|A|psi> through *ex when non-null. */
static void alg1_complex(int n, const int32_t *gates, int n_gates, const double *theta,
                         int n_params, int n_terms, const double *cr, const double *ci,
                         const uint8_t *letters, cplx *g, cplx *ex) {
    const int64_t dim = (int64_t)1 << n;
    cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *phi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *mu = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    for (int p = 0; p < n_params; ++p) g[p] = 0;
    oracle_prepare_state(n, gates, n_gates, theta, lam);
    memcpy(phi, lam, sizeof(cplx) * (size_t)dim);
    oracle_apply_operator(n, n_terms, cr, ci, letters, phi, lam);
    if (ex) *ex = oracle_inner(n, phi, lam);
    for (int i = n_gates - 1; i >= 0; --i) {
        const int32_t *gt = gates + 6 * i;
        oracle_apply_gate(n, phi, gt, theta, 1);
        for (int j = 0; j < n_params_of(gt[0]); ++j) {
            memcpy(mu, phi, sizeof(cplx) * (size_t)dim);
            apply_gate_derivative(n, mu, gt, theta, j);
            g[gt[3 + j]] += oracle_inner(n, lam, mu);
        }
        if (i > 0) oracle_apply_gate(n, lam, gt, theta, 1);
    }
    free(lam);
    free(phi);
    free(mu);
}

/* App. B.4: E = <psi|A|psi> and dE/dtheta for a non-Hermitian A (both complex), by two
 * runs of the modified Algorithm 1: one with A and one with A^dagger (the Pauli strings
 * are Hermitian, so A^dagger has the conjugate coefficients).  With <lambda|mu>
 * antilinear in lambda, the run with A yields conj(<d psi|A|psi>) and the run with
 * A^dagger yields <psi|A|d psi>, so dE = conj(run_A) + run_{A^dagger}.
 * grad2: 2 n_params doubles (re, im per parameter); expect2: 2 doubles. */
void oracle_gradient_alg1_operator(int n, const int32_t *gates, int n_gates, const double *theta,
                                   int n_params, int n_terms, const double *cr, const double *ci,
                                   const uint8_t *letters, double *grad2, double *expect2) {
    cplx *ga = (cplx *)malloc(sizeof(cplx) * (size_t)(n_params > 0 ? n_params : 1));
    cplx *gd = (cplx *)malloc(sizeof(cplx) * (size_t)(n_params > 0 ? n_params : 1));
    double *cin = (double *)malloc(sizeof(double) * (size_t)(n_terms > 0 ? n_terms : 1));
    for (int t = 0; t < n_terms; ++t) cin[t] = -ci[t];
    cplx ex = 0;
    alg1_complex(n, gates, n_gates, theta, n_params, n_terms, cr, ci, letters, ga, &ex);
    alg1_complex(n, gates, n_gates, theta, n_params, n_terms, cr, cin, letters, gd, NULL);
    for (int p = 0; p < n_params; ++p) {
        const cplx d = conj(ga[p]) + gd[p];
        grad2[2 * p] = creal(d);
        grad2[2 * p + 1] = cimag(d);
    }
    if (expect2) {
        expect2[0] = creal(ex);
        expect2[1] = cimag(ex);
    }
    free(ga);
    free(gd);
    free(cin);
}

int oracle_openmp_threads(void) {
    int t = 1;
#ifdef _OPENMP
    _Pragma("omp parallel")
    {
        _Pragma("omp single")
        t = omp_get_num_threads();
    }
#endif
    return t;
}
