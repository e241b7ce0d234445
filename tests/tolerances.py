"""Parity bars of the CUDA path against the FP64 oracle.

Norm-wise relative error (near-zero entries do not blow it up):
    grad: max_p |g_p - g_ref_p| / max(max_p |g_ref_p|, 1e-300)
    E:    |E - E_ref| / max(|E_ref|, 1)
complex128 path: <= 1e-10.  complex64 path (FP32 amplitudes, FP64 reductions): <= 1e-4.
"""
import numpy as np

TOL = {"c128": 1e-10, "c64": 1e-4}


def grad_err(g, ref) -> float:
    g, ref = np.asarray(g, float), np.asarray(ref, float)
    if g.size == 0:
        return 0.0
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))


def energy_err(e, ref) -> float:
    return abs(e - ref) / max(abs(ref), 1.0)


def assert_parity(dtype, e, g, e_ref, g_ref, what=""):
    tol = TOL[dtype]
    ee, ge = energy_err(e, e_ref), grad_err(g, g_ref)
    assert ee <= tol, f"{what} {dtype}: energy rel err {ee:.3e} > {tol:g} (E={e!r}, ref={e_ref!r})"
    assert ge <= tol, (f"{what} {dtype}: gradient rel err {ge:.3e} > {tol:g}; max abs "
                       f"{np.max(np.abs(np.asarray(g) - np.asarray(g_ref))):.3e}")
