"""The string form of Pauli-sum Hamiltonians (character q acts on qubit q, one of
I, X, Y, Z): the library's conversion against the mask form on the host, its
rejections, and on the GPU the energy and gradient against the CPU oracle (Algorithm 1,
Sec. 2.3) with the Hamiltonian given as strings."""
import numpy as np
import pytest

from paper_2009_02823_gb300 import binding as B
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, grad_err


def as_string(ops, n):
    """Neutral term ((qubit, letter), ...) -> the n-character string, qubit q at index q."""
    s = ["I"] * n
    for q, letter in ops:
        s[q] = letter
    return "".join(s)


def test_strings_match_mask_form():
    rng = np.random.default_rng(11)
    for n in (1, 4, 13, 30, 34, 64):
        terms = W.random_paulis(rng, n, 40, min(4, n))
        strings = [as_string(ops, n) for _c, ops in terms]
        x, z = B.pauli_strings_to_masks(n, strings)
        xr, zr, _c = B.pauli_masks(terms, n)
        assert np.array_equal(x, np.asarray(xr, dtype=np.uint64))
        assert np.array_equal(z, np.asarray(zr, dtype=np.uint64))


def test_string_letters_by_hand():
    # "XIZY": X on qubit 0, Z on qubit 2, Y (both bits) on qubit 3
    x, z = B.pauli_strings_to_masks(4, ["XIZY", "IIII", "YYYY", "ZIIX"])
    assert list(x) == [0b1001, 0, 0b1111, 0b1000]
    assert list(z) == [0b1100, 0, 0b1111, 0b0001]


@pytest.mark.parametrize("bad", ["XIZ", "XIZYI", "XIzY", "XI Y", "XIAY", ""])
def test_strings_rejected(bad):
    with pytest.raises(B.VqgError) as ei:
        B.pauli_strings_to_masks(4, ["IIII", bad])
    assert ei.value.status == -1  # VQG_ERR_INVALID


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,n", [("c128", 12), ("c64", 12), ("c128", 7)])
def test_string_hamiltonian_energy_and_gradient(dtype, n):
    import oracle

    w = W.config(3, n=n, layers=3)
    strings = [as_string(ops, n) for _c, ops in w.terms]
    coef = [c for c, _ops in w.terms]
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    with B.Circuit(w.n, w.gates, w.n_params, dtype) as c:
        c.set_hamiltonian_strings(strings, coef)
        e, g = c.energy_and_gradient(w.theta)
        # a rejected string leaves the Hamiltonian in place
        with pytest.raises(B.VqgError):
            c.set_hamiltonian_strings(["Q" * n], [1.0])
        e2, g2 = c.energy_and_gradient(w.theta)
    assert abs(e - e_ref) <= TOL[dtype] * max(1.0, abs(e_ref))
    assert grad_err(g, g_ref) <= TOL[dtype]
    assert e2 == e and np.array_equal(g2, g)
