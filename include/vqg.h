/*
 * vqg.h -- C ABI of the GB300 (sm_103a) reverse-mode gradient library.
 *
 * The library evaluates, for a variational circuit U(theta) = U_G ... U_1 acting on
 * |in> = |0...0> and a Pauli-sum Hamiltonian H,
 *     E(theta) = <psi|H|psi>,  |psi> = U(theta)|in>            (Sec. 2.2, problem statement)
 * and the full gradient dE/dtheta in O(G) gate passes by the "reverse mode" recurrence
 *     phi_i = U_i^dag phi_{i+1},  lambda_i = U_{i+1}^dag lambda_{i+1},
 *     dE/dtheta_i = 2 Re <lambda_i| dU_i/dtheta_i |phi_i>       (Sec. 2.2, Eq. recurrent_grad;
 *                                                               Algorithm 1)
 * with multi-parameter gates handled per App. B.1 (Algorithm 3) and repeated
 * parameters by the chain-rule sum of App. B.2 (Algorithm 4): each gate names the
 * parameter index of each of its slots, and gradient entries of all occurrences of
 * one index are added.
 *
 * Conventions: qubit q is bit q of the amplitude index.  State vectors are 2^n
 * complex amplitudes, interleaved (re, im), complex64 (8 B) or complex128 (16 B).
 *   RX/RY/RZ(t) = exp(-i t sigma / 2)    (App. A's exp(alpha i t sigma) with alpha = -1/2)
 *   U3(t, f, l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2, e^{i(f+l)} cos t/2]],
 *                 parameter slots (t, f, l) in that order
 *   CNOT(q0 -> q1): flips q1 where q0 = 1.   CZ(q0, q1): -1 where both are 1.
 *   CRX/CRY/CRZ(q0 -> q1, t): R_sigma(t) on q1 where q0 = 1 (App. A's C_c[U]; the
 *                 derivative is projected onto q0 = 1).
 *   PHASE(q0, t) = diag(1, e^{it}) (App. A; derivative i e^{it}|1><1|).
 *   CPHASE(q0, q1, t): e^{it} where both are 1 (= PHASE on q1 controlled by q0).
 *   Pauli term (x_mask, z_mask, coef): coef * i^{popcount(x & z)} X^x Z^z, i.e. the
 *   tensor product with X where only the x bit is set, Z where only the z bit is set,
 *   Y where both are set.
 *
 * Ownership: the library copies gates and Hamiltonian terms at create / set time and
 * owns all device buffers of a circuit (state vectors, checkpoints, reduction
 * scratch).  theta / energy / grad buffers are the caller's, read or written only
 * during the call.  Calls on one circuit are not thread-safe; different circuits
 * may be used from different threads.
 *
 * Errors: every entry point returns VQG_OK (0) or a negative vqg_status; nothing
 * throws across the ABI.  vqg_last_error() gives a thread-local message for the
 * last failing call on this thread.
 */
#ifndef VQG_H
#define VQG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vqg_status {
    VQG_OK = 0,
    VQG_ERR_INVALID = -1,     /* bad argument: qubit >= n, q0 == q1, param index out of range,
                                 mask bit >= n, n out of range, null pointer, ...          */
    VQG_ERR_OOM = -2,         /* device memory allocation failed                           */
    VQG_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed               */
    VQG_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up (status word set)      */
    VQG_ERR_UNSUPPORTED = -5, /* valid request this build does not implement               */
    VQG_ERR_STATE = -6        /* call order problem, e.g. energy before set_hamiltonian    */
} vqg_status;

typedef enum vqg_gate_kind {
    VQG_RX = 0, VQG_RY = 1, VQG_RZ = 2, VQG_U3 = 3, VQG_CNOT = 4, VQG_CZ = 5,
    VQG_CRX = 6, VQG_CRY = 7, VQG_CRZ = 8, VQG_PHASE = 9, VQG_CPHASE = 10
} vqg_gate_kind;

typedef enum vqg_dtype {
    VQG_C64 = 0,  /* complex64 amplitudes; FP64 reductions (energy, inner products) */
    VQG_C128 = 1  /* complex128 amplitudes and arithmetic                            */
} vqg_dtype;

/* One gate.  q1 = -1 for one-qubit gates (RX, RY, RZ, U3, PHASE); for CNOT and the
 * controlled kinds q0 is the control and q1 the target.  param[j] is the parameter
 * index of slot j (every parameterised kind uses slot 0, U3 slots 0..2); unused slots
 * are ignored (use -1). */
typedef struct vqg_gate {
    int32_t kind;
    int32_t q0;
    int32_t q1;
    int32_t param[3];
} vqg_gate;

/* Execution options (vqg_default_options fills the defaults). */
/* Arithmetic of the complex128 tile passes.  Amplitudes are FP64 in memory either way;
 * reductions (energy, gradient partials) are FP64 either way.
 *   VQG_C128_FP64:        gate arithmetic in FP64 (bounded by the GPU's FP64 rate).
 *   VQG_C128_FLOAT_FLOAT: gate arithmetic on pairs of FP32 numbers (hi + lo, about 48
 *                         significant bits; error-free TwoSum / FMA TwoProduct), rounded
 *                         to FP64 at every state store.  Absolute error per operation
 *                         below ~2^-46 (|a| + |b|) for a sum or a product-sum a*b + c
 *                         of amplitudes bounded by the state norm; tile passes only (3 register qubits per stage);
 *                         the one-kernel-per-gate route (fusion = 0, n < 10) stays FP64. */
typedef enum { VQG_C128_FP64 = 0, VQG_C128_FLOAT_FLOAT = 1 } vqg_c128_arith;

typedef struct vqg_options {
    int32_t fusion;              /* 1: apply runs of gates per tile pass (default);
                                    0: one kernel per gate                                  */
    int32_t checkpoint_interval; /* forward states stored every this many gates (fused: at
                                    the first pass boundary after that many gates) and used
                                    to restart phi in the reverse sweep; 0 = automatic
                                    (complex64: every fused pass boundary, or every 64 gates
                                    unfused; complex128: none), -1 = none; as many as fit
                                    in free device memory (see max_checkpoint_mib)         */
    int32_t tile_qubits;         /* qubits per fused tile; 0 = built-in table: n - 8 clamped
                                    to [10, 13] (complex64) or [10, 12] (complex128)        */
    int32_t use_graph;           /* 1: replay the launch sequence from a CUDA graph          */
    int32_t max_checkpoint_mib;  /* cap on checkpoint memory; 0 = fit in free memory         */
    int32_t fwd_reg_qubits;      /* qubits held in registers per forward stage; 0 = default  */
    int32_t rev_reg_qubits;      /* qubits held in registers per reverse stage; 0 = default  */
    int32_t autotune;            /* 1: time candidate schedules on the first evaluation and
                                    keep the fastest (see vqg_autotune)                     */
    int32_t c128_arith;          /* complex128 tile-pass arithmetic (vqg_c128_arith):
                                    VQG_C128_FP64 (default) or VQG_C128_FLOAT_FLOAT      */
    int32_t specialize;          /* complex64 tile passes run kernels generated for this
                                    circuit's passes (straight-line op sequences, compiled
                                    with nvcc when the schedule or Hamiltonian is set and
                                    cached on disk; needs nvcc and the library's headers
                                    at run time, VQG_ERR_UNSUPPORTED otherwise): 1 the
                                    forward and Hamiltonian passes, 2 the reverse passes
                                    too; results agree with the default kernels to
                                    rounding.  0 (default): the generic kernels only       */
    int32_t reserved[6];
} vqg_options;

typedef struct vqg_circuit vqg_circuit;

void vqg_default_options(vqg_options *opt);

/* Create the circuit U(theta) = U_G ... U_1 of Sec. 2.2 (gates[0] acts first; each
 * gate slot names the parameter it takes, App. B.1/B.2) on n_qubits (1..34) over
 * gates[0..n_gates) with n_params parameters.  gates: host array, copied.  dtype is a
 * vqg_dtype.  opt may be NULL (defaults).  Device buffers for two state vectors (and
 * checkpoints) are allocated here on the current CUDA device and owned by the circuit.
 * *out receives the handle.  Errors: VQG_ERR_INVALID for malformed gates (qubit out of
 * range, q0 == q1, parameter index outside 0..n_params-1, unknown kind), VQG_ERR_OOM
 * when buffers do not fit; *out is untouched on error. */
int vqg_circuit_create(int n_qubits, const vqg_gate *gates, int n_gates, int n_params,
                       int dtype, const vqg_options *opt, vqg_circuit **out);

/* Release a circuit of vqg_circuit_create and every device buffer it owns (the state
 * vectors of Sec. 2.2's |psi>, Algorithm 1's lambda and the checkpoints).  Waits for the
 * circuit's outstanding work first.  NULL is a no-op returning VQG_OK. */
int vqg_circuit_destroy(vqg_circuit *c);

/* Set (replace) the Hamiltonian: sum_t coef[t] * i^{popcount(x&z)} X^{x_mask[t]} Z^{z_mask[t]}.
 * Any representation is allowed by the method (Sec. 2.1, Algorithm 1 input); this one
 * groups terms by x_mask so that one pass over amplitude pairs (j, j^x) applies every
 * term of a group.  coef real (Hermitian H).  May be called between evaluations. */
int vqg_set_hamiltonian(vqg_circuit *c, int n_terms, const uint64_t *x_mask,
                        const uint64_t *z_mask, const double *coef);

/* The same Hamiltonian written as Pauli strings (Sec. 2.1 leaves the representation
 * open; Sec. 3's operators are tensor products of one-qubit Paulis):
 * strings[t] is a NUL-terminated string of exactly n_qubits characters, character q
 * the letter acting on qubit q, one of 'I', 'X', 'Y', 'Z' (so "XIZY" is X_0 Z_2 Y_3);
 * coef[t] its real coefficient.  Both arrays are host memory, read during the call.
 * Any other character, a NULL string, or a string of another length returns
 * VQG_ERR_INVALID and leaves the circuit's Hamiltonian unchanged.  Otherwise the call
 * behaves exactly as vqg_set_hamiltonian on the converted masks.
 * vqg_pauli_strings_to_masks does the conversion alone, on the host (no GPU, no
 * circuit): x_mask[t], z_mask[t] (host, n_terms each) receive term t's masks, with the
 * same checks and errors; n_qubits may be 1..64 there. */
int vqg_set_hamiltonian_strings(vqg_circuit *c, int n_terms, const char *const *strings,
                                const double *coef);
int vqg_pauli_strings_to_masks(int n_qubits, int n_terms, const char *const *strings,
                               uint64_t *x_mask, uint64_t *z_mask);

/* All work of this circuit is issued on `stream` (a cudaStream_t; NULL = the library's
 * own non-blocking stream; pass cudaStreamLegacy, (void *)0x1, for the legacy default
 * stream).  The caller keeps the stream alive while the circuit uses it. */
int vqg_set_stream(vqg_circuit *c, void *stream);

/* E(theta): forward sweep (Algorithm 1's forward sweep) then <psi|H|psi> with FP64 reduction.
 * theta: host array of n_params doubles.  energy: host double.  Blocks until done.
 * H is the Pauli sum or tensor-product operator set last; a non-Hermitian operator
 * (vqg_set_operator with imaginary coefficients) is refused with VQG_ERR_STATE; no
 * operator at all is VQG_ERR_STATE too.  The gradient calls below behave the same way;
 * with options.autotune the first of them blocks while candidate schedules are timed. */
int vqg_energy(vqg_circuit *c, const double *theta, double *energy);

/* E(theta) and dE/dtheta (Algorithm 1 with App. B.1/B.2): forward sweep, lambda = H psi
 * with E fused, then the fused reverse sweep.  theta: host, n_params doubles; energy:
 * host double; grad: host, n_params doubles (overwritten).  Blocks until done. */
int vqg_energy_and_gradient(vqg_circuit *c, const double *theta, double *energy, double *grad);

/* Same as above with device pointers (theta_dev: n_params doubles; energy_dev: 1 double;
 * grad_dev: n_params doubles).  Issued on the circuit's stream; does not synchronise. */
int vqg_energy_device(vqg_circuit *c, const double *theta_dev, double *energy_dev);
int vqg_energy_and_gradient_device(vqg_circuit *c, const double *theta_dev, double *energy_dev,
                                   double *grad_dev);

/* Faithful O(G^2) baseline on the GPU: per-occurrence parameter shift,
 * g_p += [E(theta_o + pi/2) - E(theta_o - pi/2)] / 2 over every parameter slot o of
 * gate occurrences [first_gate, last_gate) (last_gate < 0: all), each evaluation a
 * full forward sweep plus expectation (Sec. 1, Sec. 3).  Controlled rotations use the
 * exact four-term rule a1 [E(+pi/2) - E(-pi/2)] + a2 [E(+3pi/2) - E(-3pi/2)],
 * a1 = (sqrt2 + 1)/(4 sqrt2), a2 = -(sqrt2 - 1)/(4 sqrt2).  grad: host, n_params doubles,
 * overwritten (entries of parameters outside the range are 0).  Blocks until done. */
int vqg_gradient_parameter_shift(vqg_circuit *c, const double *theta, int first_gate,
                                 int last_gate, double *grad);

/* Copy the state buffer (complex64 or complex128 per dtype) into host memory `out` of
 * `bytes` >= 2^n * amplitude size.  Blocks until done.  After vqg_energy it holds
 * |psi> = U(theta)|in>; after a gradient call it holds reverse-sweep scratch (the reverse
 * sweep un-applies the gates in place), so call vqg_energy first to read |psi>. */
int vqg_get_state(vqg_circuit *c, void *out, size_t bytes);

/* Timing of the kernels of the last call, for measurement: fills up to max_entries
 * (name_id, launches, total_ms) rows per kernel family; returns the row count.  Only
 * populated when the circuit was created with profiling enabled via
 * vqg_set_profiling(c, 1).  Names are returned by vqg_kernel_family_name(). */
int vqg_set_profiling(vqg_circuit *c, int enable);
int vqg_kernel_stats(vqg_circuit *c, int max_entries, int *name_id, int *launches,
                     double *total_ms);
const char *vqg_kernel_family_name(int name_id);

/* Per-call details of the schedule: number of forward passes, reverse passes,
 * Hamiltonian passes, kernel launches per energy_and_gradient, checkpoints, and the
 * fused schedule's tile qubits and register qubits (0 when unfused).  The stage, op and
 * diagonal-block counts are filled by vqg_plan_dry_run only. */
typedef struct vqg_plan_info {
    int32_t forward_passes;
    int32_t hamiltonian_passes;
    int32_t reverse_passes;
    int32_t launches_per_gradient;
    int32_t checkpoints;
    int32_t tile_qubits;
    int32_t hamiltonian_groups;
    int32_t fwd_reg_qubits;
    int32_t rev_reg_qubits;
    int32_t forward_stages;
    int32_t reverse_stages;
    int32_t stage_ops;
    int32_t diag_blocks;
    int32_t specialized;  /* the specialize level in effect: 0 none, 1 forward (and
                             Hamiltonian), 2 also reverse */
    int32_t dense_gates;  /* gates applied by fused passes that compute every tile (the
                             others skip tiles left at zero, vqg_plan_pass); dry run: for a
                             |0...0> start */
    int32_t reserved[1];
} vqg_plan_info;
int vqg_plan(vqg_circuit *c, vqg_plan_info *info);

/* One fused tile pass of the schedule (forward order; vqg_plan's forward_passes of them):
 * the gates it applies and how many of the state's tiles it computes.  A sweep that starts
 * from |0...0> (Sec. 2.2's U(theta)|0>) leaves a tile at zero until some gate acts
 * non-diagonally on a qubit outside the tile on which the tile's index has a set bit: the
 * forward pass writes zeros to those tiles and the reverse pass skips them (phi is zero
 * there, so they add nothing to any gradient sum, and no earlier pass reads their lambda).
 * The results are those of computing every tile.  With an input state
 * (vqg_set_input_state), or while diagnostics are on (reverse passes), every tile is
 * computed. */
typedef struct vqg_pass_info {
    int32_t n_gates;         /* gates applied by the pass */
    int32_t forward_stages;  /* register stages of its forward pass */
    int32_t reverse_stages;  /* register stages of its reverse pass */
    int32_t from_zero;       /* 1: the pass synthesises |0...0> instead of reading a state */
    uint64_t tiles;          /* tiles of 2^tile_qubits amplitudes in the state */
    uint64_t active_tiles;   /* tiles the pass computes (the rest hold zeros) */
    uint64_t tile_mask;      /* bit q set: qubit q lies inside the pass's tiles */
    int32_t reserved[2];
} vqg_pass_info;

/* Fill *info for pass `pass` (0-based) and, when gates is not NULL, its first
 * min(max_gates, n_gates) gate indices (positions in the list given to
 * vqg_circuit_create) in the order the pass applies them.  Returns VQG_OK.  Errors:
 * VQG_ERR_INVALID for a NULL circuit or info, a negative max_gates, or a pass outside
 * 0..forward_passes-1; VQG_ERR_STATE when the circuit has no fused schedule (one kernel
 * per gate). */
int vqg_plan_pass(vqg_circuit *c, int pass, vqg_pass_info *info, int max_gates, int32_t *gates);

/* Precision diagnostics (complex64 amplitudes with FP64 reductions and forward
 * checkpoints; the invariants of Algorithm 1's recurrence, Sec. 2.3: phi and lambda are
 * un-applied by the same unitaries, so <lambda_i|phi_{i+1}> = E and ||lambda_i|| is
 * constant).  vqg_set_diagnostics(c, 1) makes every later gradient call of c also take,
 * in FP64 on the GPU: ||psi||^2, E and ||lambda||^2 after the Hamiltonian; ||psi_c||^2 of
 * every forward checkpoint when it is stored; and at every reverse restart from a
 * checkpoint, <lambda|psi_c>, ||lambda||^2, the norm of the phi the sweep had un-applied
 * up to there and its distance to psi_c (the drift the restart removes).  It costs one
 * streaming pass over one or two states per value set, makes the reverse sweep store
 * its un-applied phi, and runs the calls eagerly (no CUDA graph); 0 turns it off.
 * vqg_diagnostics reads the values of the last gradient call (blocking on the circuit's
 * stream): summary (nullable) and entries[0 .. min(count, max_entries)) (host memory),
 * one per checkpoint in forward order; returns the checkpoint count, or VQG_ERR_STATE when
 * no call recorded diagnostics.  Results are unchanged by diagnostics. */
typedef struct vqg_diag_summary {
    double energy;        /* Re <psi|lambda> of the final state                           */
    double norm2_psi;     /* ||psi||^2 of the final forward state                          */
    double norm2_lambda;  /* ||lambda||^2 = ||H psi||^2 as the reverse sweep starts        */
    int32_t checkpoints;  /* checkpoint entries recorded                                    */
    int32_t reserved;
} vqg_diag_summary;
typedef struct vqg_checkpoint_diag {
    int32_t checkpoint;      /* index, forward order                                        */
    int32_t stored;          /* 1: the forward sweep stored it in the last call             */
    int32_t restarted;       /* 1: the reverse sweep restarted phi from it                   */
    int32_t reserved;
    double norm2;            /* ||psi_c||^2 when stored                                      */
    double lam_phi_re;       /* Re <lambda|psi_c> at the restart (invariant: E)              */
    double lam_phi_im;       /* Im <lambda|psi_c> at the restart (invariant: 0)              */
    double norm2_lambda;     /* ||lambda||^2 at the restart (invariant: ||H psi||^2)         */
    double norm2_unapplied;  /* ||phi||^2 of the un-applied phi the restart replaces         */
    double drift2;           /* ||phi_unapplied - psi_c||^2                                  */
} vqg_checkpoint_diag;
int vqg_set_diagnostics(vqg_circuit *c, int enable);
int vqg_diagnostics(vqg_circuit *c, vqg_diag_summary *summary, int max_entries, vqg_checkpoint_diag *entries);

/* Plan a circuit and Hamiltonian on the host only (no GPU is touched): the same tile
 * passes, register stages and Hamiltonian passes a vqg_circuit with these options
 * would run, checked index by index, with the stage, op and diagonal-block counts
 * filled in.  Returns VQG_ERR_INVALID for malformed input and
 * VQG_ERR_UNSUPPORTED if the schedule fails its checks. */
int vqg_plan_dry_run(int n_qubits, const vqg_gate *gates, int n_gates, int n_params, int dtype,
                     const vqg_options *opt, int n_terms, const uint64_t *x_mask,
                     const uint64_t *z_mask, const double *coef, vqg_plan_info *info);

/* Specialised kernels (options.specialize): plan a complex64 circuit on the host exactly
 * as vqg_circuit_create would with these options and compile the per-pass kernels into
 * the on-disk cache (directory VQG_SPEC_CACHE, default $TMPDIR/vqg_spec_<uid>), so that a
 * later vqg_circuit_create with specialize = 1 only loads them.  No GPU is touched; needs
 * nvcc.  With n_terms > 0 the Hamiltonian passes of that Pauli sum (masks and coefficients
 * as vqg_set_hamiltonian) are compiled too.  gates, opt and the term arrays: host, read
 * during the call; *n_kernels (nullable) receives the
 * number of kernels (one per pass and specialised direction; 0 when unfused).  Errors:
 * VQG_ERR_INVALID for malformed gates, VQG_ERR_UNSUPPORTED when a kernel does not compile
 * (the message holds the compiler's output).  The paper has no counterpart: this is
 * the GB300 implementation's way to run a fixed circuit's gate sequence as compiled code
 * (Algorithm 1's primitives, Sec. 2.1, are otherwise interpreted per op). */
int vqg_specialize_prepare(int n_qubits, const vqg_gate *gates, int n_gates, int n_params,
                           const vqg_options *opt, int n_terms, const uint64_t *x_mask,
                           const uint64_t *z_mask, const double *coef, int *n_kernels);

/* Tensor-product cost operators (the paper's benchmark operator Hadamard^{(x)N}, Sec. 3;
 * Sec. 2.1 asks only that the operator can be applied to a state).
 * vqg_set_product_operator: A = sum_k coef[k] (x)_q M_{k,q}, n_products >= 1 products of
 *   one 2x2 matrix per qubit; mats: host, n_products * n_qubits * 8 doubles, product k
 *   qubit q at mats + 8 (k n + q), row-major (re, im) pairs (m00, m01, m10, m11).  Every
 *   factor must be Hermitian (VQG_ERR_UNSUPPORTED otherwise) so that E is real; the
 *   energy and gradient entry points then use A.  Replaces any Hamiltonian or operator;
 *   vqg_set_hamiltonian / vqg_set_operator replace it.  lambda = A psi runs each product
 *   through the fused forward passes (or one kernel per qubit below 10 qubits) and adds
 *   the products (one scratch state when n_products > 1). */
int vqg_set_product_operator(vqg_circuit *c, int n_products, const double *coef, const double *mats);

/* Input state (Sec. 2.2's fixed input state; default |0...0>).  state: 2^n amplitudes of
 * the circuit's dtype (complex64 or complex128, interleaved), host memory (on_device = 0)
 * or device memory (on_device = 1); copied into a library-owned buffer (one state), used
 * as given (not normalised).  NULL restores |0...0>.  Blocks until the copy is done.
 * A device source is read on the circuit's stream: the caller makes sure it has been
 * written (same stream, or synchronised) before the call. */
int vqg_set_input_state(vqg_circuit *c, const void *state, int on_device);

/* Non-Hermitian cost operators (App. B.4).  vqg_set_operator sets A = sum_k c_k P_k with
 * complex coefficients c_k = coef_re[k] + i coef_im[k] (masks as vqg_set_hamiltonian);
 * it replaces any Hamiltonian, and vqg_set_hamiltonian replaces it.  While the
 * operator has a non-zero imaginary coefficient, vqg_energy* refuse it
 * (VQG_ERR_STATE) and vqg_expectation_and_gradient* must be used.
 * vqg_expectation_and_gradient: E = <psi|A|psi> and dE/dtheta_p, both complex:
 *   expect: 2 doubles (re, im); grad: 2 n_params doubles, (re, im) per parameter; host
 *   buffers, blocks.  Works for Hermitian operators too (imaginary parts 0).
 * _device: the same with device pointers on the circuit's stream, no synchronisation.
 * Method: A = B + iC with B, C Hermitian (the real and imaginary coefficient parts), so
 * E = <B> + i<C> and dE = d<B> + i d<C>; one forward sweep, then the Hamiltonian
 * application and reverse sweep of Algorithm 1 once per part (the second from a saved
 * copy of the final state: one extra state vector of device memory). */
int vqg_set_operator(vqg_circuit *c, int n_terms, const uint64_t *x_mask, const uint64_t *z_mask,
                     const double *coef_re, const double *coef_im);
int vqg_expectation_and_gradient(vqg_circuit *c, const double *theta, double *expect, double *grad);
int vqg_expectation_and_gradient_device(vqg_circuit *c, const double *theta_dev, double *expect_dev,
                                        double *grad_dev);

/* Schedule autotuner (no counterpart in the paper, which applies one gate at a time;
 * it tunes the tile fusion of the sweeps).  Times whole energy-and-gradient
 * evaluations of THIS circuit and Hamiltonian under candidate schedules -- tile qubits
 * K, forward and reverse register-stage widths -- and keeps the fastest.  Candidates:
 * the compiled (K, Rf, Rr) combinations with K from Kmax = min(n, 13 complex64 / 12
 * complex128) down to Kmax - 2 or the built-in default, whichever is lower; each K
 * is run with two register choices, and per K the best forward and best reverse stage
 * widths (timed per kernel family) are combined.  Results are kept in a process-wide
 * table keyed by the circuit's structure (n, dtype, gates, Hamiltonian masks), so a
 * second circuit of the same structure takes the stored choice without timing.
 * theta: host, n_params doubles (NULL: all zeros).  out (nullable): the choice.
 * Needs a Hamiltonian; no-op (candidates = 0, tile_qubits = 0) when the circuit runs
 * unfused (n < 10 or fusion off) or was created with an explicit tile_qubits.
 * Blocks until done; the circuit's checkpoints and graphs are rebuilt for the choice.
 * Options.autotune = 1 runs this automatically on the first energy_and_gradient call. */
typedef struct vqg_tune_result {
    int32_t tile_qubits;
    int32_t fwd_reg_qubits;
    int32_t rev_reg_qubits;
    int32_t candidates;   /* schedules timed; 0 when taken from the table or a no-op   */
    double best_ms;       /* fused forward + Hamiltonian + reverse time of the choice   */
    double default_ms;    /* the same for the built-in default schedule (0 if untimed)  */
} vqg_tune_result;
int vqg_autotune(vqg_circuit *c, const double *theta, vqg_tune_result *out);
/* Drop every stored autotuner choice of this process. */
void vqg_tune_table_clear(void);

const char *vqg_last_error(void);
const char *vqg_status_string(int status);

/* ---------------------------------------------------------------- batched launch
 * Many independent circuits (each with its own parameters and Pauli-sum Hamiltonian),
 * every one evaluated by Algorithm 1 (energy and full gradient), in ONE persistent
 * kernel launch replayed from a CUDA graph.  complex64 amplitudes with FP64 reductions;
 * 12 <= n_qubits <= 30 per circuit.  Work is split into (circuit, phase, chunk of tiles)
 * tasks claimed from a device queue; a task waits (bounded) only for its own circuit's
 * earlier phases.
 *
 * vqg_batch_create: circuit b has n_qubits[b] qubits, gates gates[gate_offsets[b] ..
 *   gate_offsets[b+1]) (parameter indices local to the circuit) and n_params[b]
 *   parameters.  Arrays are host memory, copied.  dtype must be VQG_C64.
 * vqg_batch_set_hamiltonian: as vqg_set_hamiltonian for circuit `circuit`; all circuits
 *   need one before the first evaluation, after which they are fixed.
 * vqg_batch_energy_and_gradient: theta = the circuits' parameter vectors concatenated
 *   (host, sum n_params doubles); energies: n_circuits doubles; grads: concatenated like
 *   theta.  Blocks until done.  VQG_ERR_TIMEOUT if a task's bounded wait ran out (the
 *   context stays usable; results are then incomplete).
 * _device: the same with device pointers on the batch's stream, no synchronisation.
 * vqg_batch_set_wait_limit: spin limit of the dependency waits; stall_circuit >= 0 makes
 *   that circuit's later phases wait for a count that is never reached (a test hook for
 *   the timeout path); -1 disables it.
 * vqg_batch_info: task count, persistent grid size, total parameters.
 * vqg_batch_autotune: evaluates the whole batch once per compiled tile geometry (tile
 *   qubits 12 with 4 register qubits, the default, and 11 with 3), keeps the fastest and
 *   reports it in `out` (nullable; fwd_reg_qubits = rev_reg_qubits = the register
 *   qubits).  theta: host, concatenated like vqg_batch_energy_and_gradient (NULL: zeros).
 *   Every circuit needs its Hamiltonian first.  Blocks; rebuilds the batch's device
 *   buffers (device pointers of earlier outputs stay valid, a captured graph is redone).
 * vqg_batch_set_tile_qubits: select a compiled geometry by its tile qubits (12 or 11;
 *   VQG_ERR_UNSUPPORTED otherwise); the batch is rebuilt at its next evaluation. */
typedef struct vqg_batch vqg_batch;
int vqg_batch_create(int n_circuits, const int *n_qubits, const vqg_gate *gates,
                     const int *gate_offsets, const int *n_params, int dtype, vqg_batch **out);
int vqg_batch_set_hamiltonian(vqg_batch *b, int circuit, int n_terms, const uint64_t *x_mask,
                              const uint64_t *z_mask, const double *coef);
int vqg_batch_set_stream(vqg_batch *b, void *stream);
int vqg_batch_set_wait_limit(vqg_batch *b, long long spins, int stall_circuit);
int vqg_batch_energy_and_gradient(vqg_batch *b, const double *theta, double *energies,
                                  double *grads);
int vqg_batch_energy_and_gradient_device(vqg_batch *b, const double *theta_dev,
                                         double *energies_dev, double *grads_dev);
int vqg_batch_info(vqg_batch *b, int *n_tasks, int *grid, int *total_params);
int vqg_batch_autotune(vqg_batch *b, const double *theta, vqg_tune_result *out);
int vqg_batch_set_tile_qubits(vqg_batch *b, int tile_qubits);
int vqg_batch_destroy(vqg_batch *b);

/* ---------------------------------------------------------------- allocation-free step
 * The paper has no counterpart to this entry point; it exists for callers that must
 * not allocate device memory while they run: a process whose device memory is owned
 * by another allocator (for example a framework's caching pool that holds the whole
 * GPU), a service whose memory footprint is fixed at start-up, or a latency-critical
 * thread that may not enter cudaMalloc/cudaFree because those calls can synchronise
 * the device.  Every vqg_circuit allocates its state vectors at create time, so those
 * callers use this function on state vectors they already own.
 *
 * vqg_reverse_noalloc runs the reverse-sweep body (un-apply U^dagger to phi and lambda,
 * accumulate the gate's gradient contributions) for gates[n_gates-1] down to gates[0]:
 *   gates    : host array; kinds RX, RY, RZ, U3, CNOT and CZ (the controlled rotations
 *              and phase gates are refused with VQG_ERR_INVALID; use a vqg_circuit).
 *   phi, lam : device state vectors of 2^n_qubits amplitudes (dtype), both updated in
 *              place; on entry phi = U_{1:G}|in> restricted to the segment's end and lam
 *              the matching lambda, exactly as in Algorithm 1's loop.
 *   theta    : host array of n_params doubles; grad: device array of n_params doubles
 *              to which the contributions are ADDED (the caller zeroes it first).
 *   stream   : cudaStream_t (NULL = legacy default stream); work is asynchronous.
 * It calls no cudaMalloc, cudaFree or other allocating routine, and copies nothing from
 * host memory: the gate matrices travel as kernel parameters.  Its reduction scratch is
 * a file-scope static device array (1 MiB of per-block partial sums) that every GPU the
 * process uses holds until the process exits.  At most VQG_NOALLOC_MAX_GATES gates per
 * call; more returns VQG_ERR_INVALID (split a longer sweep into segments and call them
 * last segment first).  The first call on each device resolves the scratch array's
 * device address (cudaGetSymbolAddress) and keeps it for the process: make that first
 * call before any stream capture, and not across a cudaDeviceReset.  All calls share
 * the scratch: calls whose work overlaps on the GPU (different streams or host threads)
 * race and must be serialised by the caller.  Returns VQG_OK or a negative vqg_status. */
#define VQG_NOALLOC_MAX_GATES 32
#define VQG_NOALLOC_BLOCKS 512
int vqg_reverse_noalloc(int n_qubits, int dtype, const vqg_gate *gates, int n_gates,
                        const double *theta, int n_params, void *phi, void *lam, double *grad,
                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VQG_H */
