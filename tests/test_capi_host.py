"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every function include/vqg.h declares, and rejects malformed input with
VQG_ERR_INVALID before touching the device."""
import ctypes

import numpy as np
import pytest

from paper_2009_02823_gb300 import binding as B


def test_library_exports_every_declared_symbol():
    L = B.lib()
    names = B.declared_functions()
    assert "vqg_energy_and_gradient" in names and "vqg_circuit_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    L = B.lib()
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert L.vqg_status_string(s)


def _create(n, gates, P, dtype=0):
    h = ctypes.c_void_p()
    arr = B.gate_array(gates)
    st = B.lib().vqg_circuit_create(n, arr, len(gates), P, dtype, None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("n,gates,P,dtype", [
    (0, [], 0, 0),                                        # n out of range
    (35, [], 0, 0),
    (3, [("RX", 3, -1, (0, -1, -1))], 1, 0),              # qubit >= n
    (3, [("RX", -1, -1, (0, -1, -1))], 1, 0),
    (3, [("CNOT", 1, 1, (-1, -1, -1))], 0, 0),            # q0 == q1
    (3, [("CZ", 0, 7, (-1, -1, -1))], 0, 0),
    (3, [("RY", 0, -1, (2, -1, -1))], 2, 0),              # parameter index >= P
    (3, [("U3", 0, -1, (0, 1, -1))], 2, 0),               # U3 needs three slots
    (3, [(11, 0, -1, (0, -1, -1))], 1, 0),                # unknown kind
    (3, [(-1, 0, -1, (0, -1, -1))], 1, 0),
    (3, [("CRX", 2, 2, (0, -1, -1))], 1, 0),              # control == target
    (3, [("CRY", 0, 3, (0, -1, -1))], 1, 0),              # target >= n
    (3, [("CPHASE", 0, -1, (0, -1, -1))], 1, 0),          # two-qubit kind without q1
    (3, [("PHASE", 1, -1, (1, -1, -1))], 1, 0),           # parameter index >= P
    (3, [], 0, 7),                                        # unknown dtype
])
def test_invalid_circuits_rejected(n, gates, P, dtype):
    st, h = _create(n, gates, P, dtype)
    assert st == -1, B.lib().vqg_last_error()
    assert not h.value
    assert B.lib().vqg_last_error()


def test_null_arguments():
    L = B.lib()
    assert L.vqg_circuit_create(2, None, 0, 0, 0, None, None) == -1
    assert L.vqg_energy(None, None, None) == -1
    assert L.vqg_set_hamiltonian(None, 0, None, None, None) == -1
    assert L.vqg_circuit_destroy(None) == 0


def test_masks_marshalling():
    x, z, c = B.pauli_masks([(0.5, ((0, "X"), (2, "Y"))), (-1.0, ((1, "Z"),))], 3)
    assert list(x) == [0b101, 0] and list(z) == [0b100, 0b010] and list(c) == [0.5, -1.0]


def test_no_gpu_means_loud_failure():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(B.VqgError) as ei:
        B.Circuit(2, [("RX", 0, -1, (0, -1, -1))], 1)
    assert ei.value.status in (-3, -2)
