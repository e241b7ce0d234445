"""Thin ctypes binding over the C ABI in include/vqg.h (argument marshalling only;
every step of the computation runs in libvqg.so's CUDA kernels).

There is no CPU fallback: if libvqg.so cannot be built or loaded, or no CUDA device
is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

VQG_OK = 0
STATUS = {0: "VQG_OK", -1: "VQG_ERR_INVALID", -2: "VQG_ERR_OOM", -3: "VQG_ERR_CUDA",
          -4: "VQG_ERR_TIMEOUT", -5: "VQG_ERR_UNSUPPORTED", -6: "VQG_ERR_STATE"}
KIND = {"RX": 0, "RY": 1, "RZ": 2, "U3": 3, "CNOT": 4, "CZ": 5,
        "CRX": 6, "CRY": 7, "CRZ": 8, "PHASE": 9, "CPHASE": 10}
DTYPE = {"c64": 0, "complex64": 0, "c128": 1, "complex128": 1}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vqg.h")


class VqgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class vqg_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("param", ctypes.c_int32 * 3)]


class vqg_options(ctypes.Structure):
    _fields_ = [("fusion", ctypes.c_int32), ("checkpoint_interval", ctypes.c_int32),
                ("tile_qubits", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("max_checkpoint_mib", ctypes.c_int32), ("fwd_reg_qubits", ctypes.c_int32),
                ("rev_reg_qubits", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("c128_arith", ctypes.c_int32), ("specialize", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]

# vqg_c128_arith: arithmetic of the complex128 tile passes
C128_ARITH = {"fp64": 0, "float-float": 1}


class vqg_diag_summary(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("norm2_psi", ctypes.c_double), ("norm2_lambda", ctypes.c_double),
                ("checkpoints", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class vqg_checkpoint_diag(ctypes.Structure):
    _fields_ = [("checkpoint", ctypes.c_int32), ("stored", ctypes.c_int32), ("restarted", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("norm2", ctypes.c_double), ("lam_phi_re", ctypes.c_double),
                ("lam_phi_im", ctypes.c_double), ("norm2_lambda", ctypes.c_double),
                ("norm2_unapplied", ctypes.c_double), ("drift2", ctypes.c_double)]


class vqg_plan_info(ctypes.Structure):
    _fields_ = [("forward_passes", ctypes.c_int32), ("hamiltonian_passes", ctypes.c_int32),
                ("reverse_passes", ctypes.c_int32), ("launches_per_gradient", ctypes.c_int32),
                ("checkpoints", ctypes.c_int32), ("tile_qubits", ctypes.c_int32),
                ("hamiltonian_groups", ctypes.c_int32), ("fwd_reg_qubits", ctypes.c_int32),
                ("rev_reg_qubits", ctypes.c_int32), ("forward_stages", ctypes.c_int32),
                ("reverse_stages", ctypes.c_int32), ("stage_ops", ctypes.c_int32),
                ("diag_blocks", ctypes.c_int32), ("specialized", ctypes.c_int32),
                ("dense_gates", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class vqg_pass_info(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int32), ("forward_stages", ctypes.c_int32),
                ("reverse_stages", ctypes.c_int32), ("from_zero", ctypes.c_int32),
                ("tiles", ctypes.c_uint64), ("active_tiles", ctypes.c_uint64),
                ("tile_mask", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 2)]


class vqg_tune_result(ctypes.Structure):
    _fields_ = [("tile_qubits", ctypes.c_int32), ("fwd_reg_qubits", ctypes.c_int32),
                ("rev_reg_qubits", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


def declared_functions() -> list[str]:
    """Names of the functions include/vqg.h declares (for export checks)."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vqg_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libvqg.so (building it in-tree with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = ctypes.CDLL(path)
        p, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        pp = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "vqg_default_options": (None, [p]),
            "vqg_circuit_create": (i, [i, p, i, i, i, p, pp]),
            "vqg_circuit_destroy": (i, [p]),
            "vqg_set_hamiltonian": (i, [p, i, p, p, p]),
            "vqg_set_hamiltonian_strings": (i, [p, i, p, p]),
            "vqg_set_diagnostics": (i, [p, i]),
            "vqg_specialize_prepare": (i, [i, p, i, i, p, i, p, p, p, p]),
            "vqg_diagnostics": (i, [p, p, i, p]),
            "vqg_pauli_strings_to_masks": (i, [i, i, p, p, p]),
            "vqg_set_stream": (i, [p, p]),
            "vqg_energy": (i, [p, p, p]),
            "vqg_energy_and_gradient": (i, [p, p, p, p]),
            "vqg_energy_device": (i, [p, p, p]),
            "vqg_energy_and_gradient_device": (i, [p, p, p, p]),
            "vqg_gradient_parameter_shift": (i, [p, p, i, i, p]),
            "vqg_get_state": (i, [p, p, ctypes.c_size_t]),
            "vqg_set_profiling": (i, [p, i]),
            "vqg_kernel_stats": (i, [p, i, p, p, p]),
            "vqg_kernel_family_name": (ctypes.c_char_p, [i]),
            "vqg_plan": (i, [p, p]),
            "vqg_plan_pass": (i, [p, i, p, i, p]),
            "vqg_autotune": (i, [p, p, p]),
            "vqg_set_operator": (i, [p, i, p, p, p, p]),
            "vqg_set_product_operator": (i, [p, i, p, p]),
            "vqg_set_input_state": (i, [p, p, i]),
            "vqg_expectation_and_gradient": (i, [p, p, p, p]),
            "vqg_expectation_and_gradient_device": (i, [p, p, p, p]),
            "vqg_tune_table_clear": (None, []),
            "vqg_last_error": (ctypes.c_char_p, []),
            "vqg_status_string": (ctypes.c_char_p, [i]),
            "vqg_reverse_noalloc": (i, [i, i, p, i, p, i, p, p, p, p]),
            "vqg_plan_dry_run": (i, [i, p, i, i, i, p, i, p, p, p, p]),
            "vqg_batch_create": (i, [i, p, p, p, p, i, pp]),
            "vqg_batch_set_hamiltonian": (i, [p, i, i, p, p, p]),
            "vqg_batch_set_stream": (i, [p, p]),
            "vqg_batch_set_wait_limit": (i, [p, ctypes.c_longlong, i]),
            "vqg_batch_energy_and_gradient": (i, [p, p, p, p]),
            "vqg_batch_energy_and_gradient_device": (i, [p, p, p, p]),
            "vqg_batch_info": (i, [p, p, p, p]),
            "vqg_batch_autotune": (i, [p, p, p]),
            "vqg_batch_set_tile_qubits": (i, [p, i]),
            "vqg_batch_destroy": (i, [p]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _ = (d, u64)
        _lib = L
        return L


def _check(status: int):
    if status != VQG_OK:
        raise VqgError(status, lib().vqg_last_error().decode())


def _string_array(strings) -> ctypes.Array:
    arr = (ctypes.c_char_p * max(len(strings), 1))()
    for k, t in enumerate(strings):
        arr[k] = t.encode("ascii") if isinstance(t, str) else t
    return arr


def pauli_strings_to_masks(n_qubits: int, strings) -> tuple[np.ndarray, np.ndarray]:
    """Host-only conversion by the library (vqg_pauli_strings_to_masks): (x_mask, z_mask)."""
    arr = _string_array(strings)
    x = np.zeros(max(len(strings), 1), dtype=np.uint64)
    z = np.zeros(max(len(strings), 1), dtype=np.uint64)
    _check(lib().vqg_pauli_strings_to_masks(n_qubits, len(strings), ctypes.cast(arr, ctypes.c_void_p),
                                            _ptr(x), _ptr(z)))
    return x[:len(strings)], z[:len(strings)]


def specialize_prepare(n: int, gates, n_params: int, terms=None, **options) -> int:
    """Compile the specialised kernels of a complex64 circuit (and of its Hamiltonian's
    passes when terms are given) into the on-disk cache on the host
    (vqg_specialize_prepare); options as for Circuit.  Returns the kernel count."""
    opt = vqg_options()
    lib().vqg_default_options(ctypes.byref(opt))
    for k, v in options.items():
        setattr(opt, k, int(v))
    opt.specialize = int(options.get("specialize", 1))
    arr = gate_array(gates)
    nk = ctypes.c_int(0)
    if terms:
        x, z, c = pauli_masks(terms, n)
        x = np.ascontiguousarray(x, dtype=np.uint64)
        z = np.ascontiguousarray(z, dtype=np.uint64)
        c = np.ascontiguousarray(np.real(c), dtype=np.float64)
        _check(lib().vqg_specialize_prepare(n, arr, len(gates), n_params, ctypes.byref(opt), len(c), _ptr(x), _ptr(z),
                                            _ptr(c), ctypes.byref(nk)))
    else:
        _check(lib().vqg_specialize_prepare(n, arr, len(gates), n_params, ctypes.byref(opt), 0, None, None, None,
                                            ctypes.byref(nk)))
    return nk.value


def gate_array(gates) -> ctypes.Array:
    arr = (vqg_gate * max(len(gates), 1))()
    for k, (kind, q0, q1, ps) in enumerate(gates):
        arr[k].kind = KIND[kind] if isinstance(kind, str) else int(kind)
        arr[k].q0 = q0
        arr[k].q1 = q1
        for j in range(3):
            arr[k].param[j] = ps[j]
    return arr


def pauli_masks(terms, n: int):
    """Neutral Pauli terms -> (x_mask, z_mask, coef): X sets x, Z sets z, Y sets both."""
    x = np.zeros(len(terms), dtype=np.uint64)
    z = np.zeros(len(terms), dtype=np.uint64)
    c = np.zeros(len(terms), dtype=np.complex128 if any(isinstance(t[0], complex) for t in terms) else np.float64)
    for t, (coef, ops) in enumerate(terms):
        xm = zm = 0
        for q, l in ops:
            if not 0 <= q < 64:
                raise ValueError(f"qubit {q}")
            b = 1 << q
            if l in ("X", "Y"):
                xm |= b
            if l in ("Z", "Y"):
                zm |= b
        x[t], z[t], c[t] = xm, zm, coef
    return x, z, c


CUDA_STREAM_LEGACY = 0x1


def stream_handle(stream):
    """cudaStream_t value for the C ABI: None -> NULL (library's own stream); a torch
    stream or integer handle; handle 0 (the legacy default stream) -> cudaStreamLegacy."""
    if stream is None:
        return None
    raw = getattr(stream, "cuda_stream", stream)
    return CUDA_STREAM_LEGACY if int(raw) == 0 else int(raw)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Circuit:
    """One variational circuit on the current CUDA device (wraps vqg_circuit)."""

    def __init__(self, n: int, gates, n_params: int, dtype: str = "c64", *, fusion: bool = True,
                 checkpoint_interval: int = 0, tile_qubits: int = 0, use_graph: bool = False,
                 max_checkpoint_mib: int = 0, fwd_reg_qubits: int = 0, rev_reg_qubits: int = 0,
                 autotune: bool = False, c128_arith: str = "fp64", stream=None, specialize: int = 0):
        L = lib()
        self.n, self.n_params, self.n_gates = n, n_params, len(gates)
        self.dtype = dtype
        opt = vqg_options()
        L.vqg_default_options(ctypes.byref(opt))
        opt.fusion = int(fusion)
        opt.checkpoint_interval = checkpoint_interval
        opt.tile_qubits = tile_qubits
        opt.use_graph = int(use_graph)
        opt.max_checkpoint_mib = max_checkpoint_mib
        opt.fwd_reg_qubits = fwd_reg_qubits
        opt.rev_reg_qubits = rev_reg_qubits
        opt.autotune = int(autotune)
        opt.c128_arith = C128_ARITH[c128_arith]
        opt.specialize = int(specialize)
        self._gates = gate_array(gates)
        h = ctypes.c_void_p()
        _check(L.vqg_circuit_create(n, self._gates, len(gates), n_params, DTYPE[dtype],
                                    ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().vqg_circuit_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (the library's
        own stream).  A handle of 0 (torch's default stream) means the legacy default
        stream and is passed as cudaStreamLegacy."""
        _check(lib().vqg_set_stream(self._h, ctypes.c_void_p(stream_handle(stream))))

    def set_hamiltonian(self, terms):
        x, z, c = pauli_masks(terms, self.n)
        self.set_hamiltonian_masks(x, z, c)

    def set_hamiltonian_strings(self, strings, coef):
        """Pauli strings, character q acting on qubit q ("XIZY" = X_0 Z_2 Y_3), through
        vqg_set_hamiltonian_strings."""
        arr = _string_array(strings)
        c = np.ascontiguousarray(coef, dtype=np.float64)
        if len(c) != len(strings):
            raise ValueError("one coefficient per string")
        _check(lib().vqg_set_hamiltonian_strings(self._h, len(c), ctypes.cast(arr, ctypes.c_void_p), _ptr(c)))

    def set_hamiltonian_masks(self, x, z, coef):
        if np.iscomplexobj(coef):
            if np.any(np.imag(coef) != 0):
                raise ValueError("complex coefficients: use set_operator (non-Hermitian operator)")
            coef = np.real(coef)
        x = np.ascontiguousarray(x, dtype=np.uint64)
        z = np.ascontiguousarray(z, dtype=np.uint64)
        c = np.ascontiguousarray(coef, dtype=np.float64)
        _check(lib().vqg_set_hamiltonian(self._h, len(c), _ptr(x), _ptr(z), _ptr(c)))

    def set_operator(self, terms):
        """Non-Hermitian Pauli sum (complex coefficients), App. B.4."""
        x, z, c = pauli_masks(terms, self.n)
        c = np.asarray(c, dtype=np.complex128)
        cr = np.ascontiguousarray(c.real)
        ci = np.ascontiguousarray(c.imag)
        x = np.ascontiguousarray(x, dtype=np.uint64)
        z = np.ascontiguousarray(z, dtype=np.uint64)
        _check(lib().vqg_set_operator(self._h, len(c), _ptr(x), _ptr(z), _ptr(cr), _ptr(ci)))

    def set_product_operator(self, products):
        """A = sum_k c_k (x)_q M_{k,q}: products = [(c_k, [M_0, ..., M_{n-1}])], Hermitian 2x2
        factors (e.g. the Hadamard matrix on every qubit)."""
        coef = np.ascontiguousarray([float(c) for c, _ms in products], dtype=np.float64)
        mats = np.zeros((len(products), self.n, 8))
        for k, (_c, ms) in enumerate(products):
            if len(ms) != self.n:
                raise ValueError("one 2x2 matrix per qubit")
            for q, m in enumerate(ms):
                m = np.asarray(m, dtype=np.complex128).reshape(4)
                mats[k, q, 0::2], mats[k, q, 1::2] = m.real, m.imag
        mats = np.ascontiguousarray(mats)
        _check(lib().vqg_set_product_operator(self._h, len(products), _ptr(coef), _ptr(mats)))

    def set_input_state(self, state=None, device_ptr: int | None = None):
        """Input state |in> (host array of 2^n amplitudes, or a device pointer to them);
        no argument restores |0...0>."""
        if device_ptr is not None:
            _check(lib().vqg_set_input_state(self._h, ctypes.c_void_p(device_ptr), 1))
            return
        if state is None:
            _check(lib().vqg_set_input_state(self._h, None, 0))
            return
        dt = np.complex64 if DTYPE[self.dtype] == 0 else np.complex128
        st = np.ascontiguousarray(state, dtype=dt)
        if st.size != 1 << self.n:
            raise ValueError("input state must have 2^n amplitudes")
        _check(lib().vqg_set_input_state(self._h, _ptr(st), 0))

    def expectation_and_gradient(self, theta):
        """(E, dE/dtheta), complex, for the operator set by set_operator."""
        th = self._theta(theta)
        e = np.zeros(2)
        g = np.zeros(2 * max(self.n_params, 1))
        _check(lib().vqg_expectation_and_gradient(self._h, _ptr(th), _ptr(e), _ptr(g)))
        return complex(e[0], e[1]), (g[0::2] + 1j * g[1::2])[: self.n_params]

    def expectation_and_gradient_device(self, theta_ptr: int, expect_ptr: int, grad_ptr: int):
        _check(lib().vqg_expectation_and_gradient_device(self._h, ctypes.c_void_p(theta_ptr),
                                                         ctypes.c_void_p(expect_ptr),
                                                         ctypes.c_void_p(grad_ptr)))

    # -- evaluation (host buffers)
    def _theta(self, theta) -> np.ndarray:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if th.shape != (self.n_params,):
            raise ValueError(f"theta must have shape ({self.n_params},)")
        return th

    def energy(self, theta) -> float:
        th = self._theta(theta)
        e = np.zeros(1)
        _check(lib().vqg_energy(self._h, _ptr(th), _ptr(e)))
        return float(e[0])

    def energy_and_gradient(self, theta, out: np.ndarray | None = None):
        th = self._theta(theta)
        e = np.zeros(1)
        g = out if out is not None else np.zeros(max(self.n_params, 1))
        _check(lib().vqg_energy_and_gradient(self._h, _ptr(th), _ptr(e), _ptr(g)))
        return float(e[0]), g[: self.n_params]

    def gradient_parameter_shift(self, theta, first_gate: int = 0, last_gate: int = -1):
        th = self._theta(theta)
        g = np.zeros(max(self.n_params, 1))
        _check(lib().vqg_gradient_parameter_shift(self._h, _ptr(th), first_gate, last_gate, _ptr(g)))
        return g[: self.n_params]

    # -- evaluation (device pointers, e.g. torch CUDA tensors); no synchronisation
    def energy_device(self, theta_ptr: int, energy_ptr: int):
        _check(lib().vqg_energy_device(self._h, ctypes.c_void_p(theta_ptr), ctypes.c_void_p(energy_ptr)))

    def energy_and_gradient_device(self, theta_ptr: int, energy_ptr: int, grad_ptr: int):
        _check(lib().vqg_energy_and_gradient_device(self._h, ctypes.c_void_p(theta_ptr),
                                                    ctypes.c_void_p(energy_ptr),
                                                    ctypes.c_void_p(grad_ptr)))

    # -- inspection
    def get_state(self) -> np.ndarray:
        dt = np.complex64 if DTYPE[self.dtype] == 0 else np.complex128
        out = np.zeros(1 << self.n, dtype=dt)
        _check(lib().vqg_get_state(self._h, _ptr(out), out.nbytes))
        return out

    def plan(self) -> dict:
        info = vqg_plan_info()
        _check(lib().vqg_plan(self._h, ctypes.byref(info)))
        return {k: getattr(info, k) for k, _t in vqg_plan_info._fields_
                if k not in ("reserved", "forward_stages", "reverse_stages", "stage_ops", "diag_blocks")}

    def plan_passes(self) -> list:
        """The fused passes of the schedule (vqg_plan_pass): per pass its gate indices, stage
        counts, and how many of the state's tiles it computes (tiles that a |0...0> start
        leaves at zero are skipped)."""
        out = []
        for j in range(self.plan()["forward_passes"] if self.plan()["tile_qubits"] else 0):
            info = vqg_pass_info()
            _check(lib().vqg_plan_pass(self._h, j, ctypes.byref(info), 0, None))
            gates = (ctypes.c_int32 * max(info.n_gates, 1))()
            _check(lib().vqg_plan_pass(self._h, j, ctypes.byref(info), info.n_gates, gates))
            out.append({"gates": list(gates[:info.n_gates]), "forward_stages": info.forward_stages,
                        "reverse_stages": info.reverse_stages, "from_zero": info.from_zero,
                        "tiles": info.tiles, "active_tiles": info.active_tiles,
                        "tile_qubits": [q for q in range(self.n) if (info.tile_mask >> q) & 1]})
        return out

    def set_diagnostics(self, enable: bool = True):
        """Record FP64 norms and inner products along later gradient calls (vqg_set_diagnostics)."""
        _check(lib().vqg_set_diagnostics(self._h, 1 if enable else 0))

    def diagnostics(self) -> dict:
        """Values of the last gradient call with diagnostics on: the summary plus one dict
        per forward checkpoint (vqg_diagnostics)."""
        summ = vqg_diag_summary()
        cap = 64
        arr = (vqg_checkpoint_diag * cap)()
        n = lib().vqg_diagnostics(self._h, ctypes.byref(summ), cap, ctypes.cast(arr, ctypes.c_void_p))
        if n < 0:
            _check(n)
        out = {k: getattr(summ, k) for k, _t in vqg_diag_summary._fields_ if k != "reserved"}
        out["entries"] = [{k: getattr(arr[i], k) for k, _t in vqg_checkpoint_diag._fields_ if k != "reserved"}
                          for i in range(min(n, cap))]
        return out

    def autotune(self, theta=None) -> dict:
        """Time candidate fused schedules on this circuit and keep the fastest."""
        r = vqg_tune_result()
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        _check(lib().vqg_autotune(self._h, None if th is None else _ptr(th), ctypes.byref(r)))
        return {k: getattr(r, k) for k, _t in vqg_tune_result._fields_}

    def set_profiling(self, enable: bool = True):
        _check(lib().vqg_set_profiling(self._h, int(enable)))

    def kernel_stats(self) -> dict:
        n = 32
        ids = (ctypes.c_int * n)()
        launches = (ctypes.c_int * n)()
        ms = (ctypes.c_double * n)()
        k = lib().vqg_kernel_stats(self._h, n, ids, launches, ms)
        if k < 0:
            _check(k)
        return {lib().vqg_kernel_family_name(ids[i]).decode(): (launches[i], ms[i]) for i in range(k)}


NOALLOC_MAX_GATES = 32


def reverse_noalloc(n: int, dtype: str, gates, theta, n_params: int, phi_ptr: int, lam_ptr: int,
                    grad_ptr: int, stream=None):
    """vqg_reverse_noalloc: reverse-sweep steps over caller-owned device vectors, no
    device allocation (at most NOALLOC_MAX_GATES gates per call)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    arr = gate_array(gates)
    _check(lib().vqg_reverse_noalloc(n, DTYPE[dtype], arr, len(gates), _ptr(th), n_params,
                                     ctypes.c_void_p(phi_ptr), ctypes.c_void_p(lam_ptr),
                                     ctypes.c_void_p(grad_ptr), ctypes.c_void_p(stream_handle(stream))))


def plan_dry_run(n: int, gates, n_params: int, terms, dtype: str = "c64", *, fusion: bool = True,
                 tile_qubits: int = 0, checkpoint_interval: int = 0, fwd_reg_qubits: int = 0,
                 rev_reg_qubits: int = 0, c128_arith: str = "fp64") -> dict:
    """Host-only schedule of a circuit + Hamiltonian (vqg_plan_dry_run); no GPU needed."""
    L = lib()
    opt = vqg_options()
    L.vqg_default_options(ctypes.byref(opt))
    opt.fusion = int(fusion)
    opt.tile_qubits = tile_qubits
    opt.checkpoint_interval = checkpoint_interval
    opt.fwd_reg_qubits = fwd_reg_qubits
    opt.rev_reg_qubits = rev_reg_qubits
    opt.c128_arith = C128_ARITH[c128_arith]
    x, z, c = pauli_masks(terms, n)
    info = vqg_plan_info()
    arr = gate_array(gates)
    _check(L.vqg_plan_dry_run(n, arr, len(gates), n_params, DTYPE[dtype], ctypes.byref(opt), len(c),
                              _ptr(x), _ptr(z), _ptr(c), ctypes.byref(info)))
    out = {k: getattr(info, k) for k, _t in vqg_plan_info._fields_ if k != "reserved"}
    return out
