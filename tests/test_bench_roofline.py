"""The roofline arithmetic bench.py reports, pinned on the CPU: algorithmic bytes per
launch (one state traversal = S bytes; Algorithm 1's cost unit), useful FP32 operations
per sweep, the FP32 lane-op peak and the amplitude-update rate, for the n=30 workload
(745 gates: 300 RY, 300 RZ, 145 CZ; 8 fused passes, 7 checkpoints)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2009_02823_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def w30():
    return W.config(3)


def test_gate_mix(w30):
    kinds = [g[0] for g in w30.gates]
    assert (kinds.count("RY"), kinds.count("RZ"), kinds.count("CZ"), len(kinds)) == (300, 300, 145, 745)


def test_algorithmic_bytes(w30):
    S = 8 << w30.n
    # forward pass: read + write psi
    assert bench.family_bytes("fwd_fused", w30, S, {}) == 2 * S
    # Hamiltonian pass: read psi, read + write lambda
    assert bench.family_bytes("ham_fused", w30, S, {}) == 3 * S
    # reverse passes, 8 of them with a checkpoint at every one of the 7 boundaries: every pass
    # reads phi and lambda, the first 7 write lambda, none writes phi
    per = bench.family_bytes("adj_fused", w30, S, {"reverse_passes": 8, "checkpoints": 7})
    assert per * 8 == (2 * 8 + 7) * S
    # no checkpoints: every pass but the last also writes phi
    per = bench.family_bytes("adj_fused", w30, S, {"reverse_passes": 8, "checkpoints": 0})
    assert per * 8 == (2 * 8 + 7 + 7) * S
    # one gate per launch: read + write one state forward, both states in reverse
    assert bench.family_bytes("fwd_gate", w30, S, {}) == 2 * S
    assert bench.family_bytes("adj_gate", w30, S, {}) == 4 * S


def test_useful_operation_counts(w30):
    amps = 1 << w30.n
    # forward: RY 4 and RZ 4 real operations per amplitude, CZ none
    assert bench.family_alu_ops("fwd_fused", w30) == amps * (300 * 4 + 300 * 4)
    # reverse: RY 10 (un-apply both states + Im<l|Y|p>), RZ 9
    assert bench.family_alu_ops("adj_fused", w30) == amps * (300 * 10 + 300 * 9)
    groups = len({tuple(sorted(q for q, l in ops if l in "XY")) for _c, ops in w30.terms})
    assert bench.family_alu_ops("ham_fused", w30) == amps * (2 * len(w30.terms) + 8 * groups)
    assert bench.family_alu_ops("reduce", w30) is None


def test_peak_and_update_rate(w30):
    peak, note = bench.alu_peak(2070.0)
    assert peak == pytest.approx(152 * 128 * 2.07)  # G lane-op/s
    assert "152 SM" in note
    S = 8 << w30.n
    r = bench.amplitude_updates(w30, S, 1.0, 6792.7)
    assert r["per_s"] == 3 * 745 * (1 << 30)
    assert r["unfused_hbm_roofline_per_s"] == pytest.approx(6792.7e9 / 16)
