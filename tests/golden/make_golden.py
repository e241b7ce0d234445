"""Writes the stored expected values for the full-size parity tests.

Calls only the CPU oracle (oracle/), never the CUDA path.  Each fixture records the
workload recipe, the oracle routine used and the paper passage it follows:
  * E and the full gradient by oracle.gradient_alg1 -- Algorithm 1 (reverse mode,
    Sec. 2.3) with App. B.1 for U3, itself pinned against the parameter-shift and
    Algorithm 2 routes and dense brute force in tests/test_oracle_pins.py;
  * E alone by oracle.energy (Sec. 2.2) where the gradient is out of reach on the CPU.

python tests/golden/make_golden.py cfg2 cfg5 cfg3e cfg3n29

cfg3n29 is the n=30 bench recipe (RY/RZ + CZ brickwork, 200 random Pauli strings) at
n=29: its full Algorithm 1 gradient needs four complex128 states (32 GiB) of host memory,
the largest size of that recipe that fits a 62 GB host.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_02823_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, payload):
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as fh:
        json.dump(payload, fh, indent=0)
    print("wrote", path, flush=True)


def grad_fixture(cfg, n=None):
    w = W.config(cfg, n=n)
    t0 = time.time()
    e, g = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    write(f"cfg{cfg}_n{w.n}", {
        "workload": w.name, "cfg": cfg, "n": w.n, "n_params": w.n_params, "n_gates": w.n_gates,
        "energy": e, "grad": [float(x) for x in g],
        "routine": "oracle.gradient_alg1 (complex128)",
        "follows": "Algorithm 1 (Sec. 2.3), App. B.1 for multi-parameter gates",
        "seconds": round(time.time() - t0, 1), "openmp_threads": oracle.threads()})


def energy_fixture(cfg):
    w = W.config(cfg)
    t0 = time.time()
    e = oracle.energy(w.n, w.gates, w.theta, w.terms)
    write(f"cfg{cfg}_n{w.n}_energy", {
        "workload": w.name, "cfg": cfg, "n": w.n, "energy": e,
        "routine": "oracle.energy (complex128)", "follows": "Sec. 2.2, E = <psi|H|psi>",
        "seconds": round(time.time() - t0, 1), "openmp_threads": oracle.threads()})


if __name__ == "__main__":
    for arg in sys.argv[1:] or ["cfg2", "cfg5", "cfg3e"]:
        if arg == "cfg3e":
            energy_fixture(3)
        elif arg == "cfg3n29":
            grad_fixture(3, n=29)
        else:
            grad_fixture(int(arg[3:]))
