"""Batched launch (vqg_batch_*): many independent circuits, each with its own
parameters and Pauli-sum Hamiltonian, evaluated (energy + full reverse-mode gradient)
in one persistent kernel launch replayed from a CUDA graph."""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as B


class Batch:
    def __init__(self, workloads, dtype: str = "c64", stream=None):
        L = B.lib()
        self.n_circuits = len(workloads)
        self.n_params = [w.n_params for w in workloads]
        self.offsets = np.concatenate([[0], np.cumsum(self.n_params)]).astype(np.int64)
        gates = [g for w in workloads for g in w.gates]
        gate_off = np.concatenate([[0], np.cumsum([len(w.gates) for w in workloads])]).astype(np.int32)
        nq = np.array([w.n for w in workloads], dtype=np.int32)
        npar = np.array(self.n_params, dtype=np.int32)
        self._gates = B.gate_array(gates)
        h = ctypes.c_void_p()
        B._check(L.vqg_batch_create(self.n_circuits, B._ptr(nq), self._gates, B._ptr(gate_off),
                                    B._ptr(npar), B.DTYPE[dtype], ctypes.byref(h)))
        self._h = h
        for b, w in enumerate(workloads):
            x, z, c = B.pauli_masks(w.terms, w.n)
            B._check(L.vqg_batch_set_hamiltonian(self._h, b, len(c), B._ptr(x), B._ptr(z), B._ptr(c)))
        if stream is not None:
            B._check(L.vqg_batch_set_stream(self._h, ctypes.c_void_p(B.stream_handle(stream))))

    def close(self):
        if getattr(self, "_h", None):
            B.lib().vqg_batch_destroy(self._h)
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

    def energy_and_gradient(self, thetas):
        """thetas: list of per-circuit parameter arrays (or one concatenated array).
        Returns (energies[n_circuits], list of gradients)."""
        th = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).ravel() for t in thetas])
                                  if isinstance(thetas, (list, tuple)) else thetas, dtype=np.float64)
        e = np.zeros(self.n_circuits)
        g = np.zeros(max(th.size, 1))
        B._check(B.lib().vqg_batch_energy_and_gradient(self._h, B._ptr(th), B._ptr(e), B._ptr(g)))
        return e, [g[self.offsets[b]:self.offsets[b + 1]] for b in range(self.n_circuits)]

    def energy_and_gradient_device(self, theta_ptr: int, energies_ptr: int, grads_ptr: int):
        B._check(B.lib().vqg_batch_energy_and_gradient_device(self._h, ctypes.c_void_p(theta_ptr),
                                                              ctypes.c_void_p(energies_ptr),
                                                              ctypes.c_void_p(grads_ptr)))

    def set_wait_limit(self, spins: int, stall_circuit: int = -1):
        B._check(B.lib().vqg_batch_set_wait_limit(self._h, spins, stall_circuit))

    def info(self) -> dict:
        nt, grid, tp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        B._check(B.lib().vqg_batch_info(self._h, ctypes.byref(nt), ctypes.byref(grid), ctypes.byref(tp)))
        return {"tasks": nt.value, "grid": grid.value, "total_params": tp.value}

    def autotune(self, thetas=None) -> dict:
        """Time every compiled tile geometry on this batch and keep the fastest."""
        th = None
        if thetas is not None:
            th = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).ravel() for t in thetas])
                                      if isinstance(thetas, (list, tuple)) else thetas, dtype=np.float64)
        r = B.vqg_tune_result()
        B._check(B.lib().vqg_batch_autotune(self._h, None if th is None else B._ptr(th), ctypes.byref(r)))
        return {k: getattr(r, k) for k, _t in B.vqg_tune_result._fields_}

    def set_tile_qubits(self, tile_qubits: int):
        """Select a compiled tile geometry (12: 4 register qubits; 11: 3)."""
        B._check(B.lib().vqg_batch_set_tile_qubits(self._h, tile_qubits))
