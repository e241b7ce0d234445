"""Benchmark: adjoint (reverse-mode) energy gradients per second on the n=30, P=600
workload (10 layers of RY/RZ + CZ brickwork, 200 random Pauli strings), complex64
amplitudes with FP64 reductions, one gradient = one step of the whole hot path
(forward sweep, H|psi> with fused energy, fused reverse sweep with per-parameter
reductions).

python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--dtype c64|c128]

Prints one JSON line (rank 0).  N > 1 runs independent replicas (one circuit per
GPU, no collective on the data path) and reports the aggregate rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2009_02823_gb300.replicas import (circuit_cost, max_over_ranks, partition,  # noqa: E402
                                             replica_theta)

METRIC = "adjoint gradients/s at n=30,P=600"

# DRAM bytes (read + write) per launch per amplitude of the state, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of each complex64 pass kernel the bench
# runs, on the bench recipe at n=26 (0.5 GB per state, far larger than L2), of a pass that
# computes every tile and reads a whole input: specialised reverse 1.0838 + 0.4795 GB,
# specialised Hamiltonian 1.1488 + 0.4772 GB per launch.  Such launches stream whole states,
# so traffic scales with 2^n.  Reset an entry to None whenever its kernel changes until it is
# captured again (the forward kernel's last capture is of a pass whose input is mostly known
# zero and not read, so it gives no per-amplitude figure).
NCU_TRAFFIC_PER_AMP_C64 = {
    "adj_fused": (1.083791e9 + 0.479509504e9) / 2**26,
    "fwd_fused": None,
    "ham_fused": (1.148828e9 + 0.477248e9) / 2**26,
}
UNIT = "gradients/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _workload(args):
    from paper_2009_02823_gb300 import workloads as W
    w = W.config(args.cfg, n=args.n, layers=args.layers)
    return w


def _config(args, w, extra=None):
    cfg = {"workload": w.name, "n_qubits": w.n, "n_params": w.n_params, "n_gates": w.n_gates,
           "hamiltonian_terms": len(w.terms), "amplitudes": f"{args.dtype} (FP64 reductions)" if args.dtype == "c64" or args.c128_arith == "fp64"
           else "c128 storage, float-float tile arithmetic, FP64 reductions",
           "state_bytes": (8 if args.dtype == "c64" else 16) << w.n,
           "l2": "inputs larger than L2 (state vectors >> 129 MB)",
           "parallelism": "replicas" if args.gpus > 1 else "single GPU"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # raw samples go to $VQG_CLOCKS_DIR (default: the system temp directory)
        out_dir = os.environ.get("VQG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"vqg_clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                    power.append(float(f[3]))
                except ValueError:
                    continue
                for name, val in zip(names, f[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ---------------------------------------------------------------- algorithmic work
# Useful FP32 lane operations per amplitude (an FMA counts once) of each gate kind in the
# fused sweeps: forward U applied to psi; reverse U^dagger applied to phi and lambda plus
# the gradient products (Im<lambda|sigma|phi>: RY/RX 2, RZ 1; U3's four sums o_rc: 8).
FWD_OPS = {"RY": 4, "RX": 8, "U3": 8, "RZ": 4, "CZ": 0, "CNOT": 0}
REV_OPS = {"RY": 10, "RX": 18, "U3": 24, "RZ": 9, "CZ": 0, "CNOT": 0}


def family_alu_ops(fam: str, w, passes=None) -> float | None:
    """Useful FP32 operations of one whole sweep of a kernel family (all its launches in
    one gradient): per-amplitude counts x the amplitudes each gate's pass computes (2^n, or
    fewer where a fused pass skips tiles that a |0...0> start leaves at zero; passes: the
    schedule's vqg_plan_pass entries)."""
    amps = float(1 << w.n)

    def swept(table):
        if not passes:
            return amps * sum(table.get(g[0], 0) for g in w.gates)  # kinds not listed count 0
        return sum(amps * p["active_tiles"] / p["tiles"] * sum(table.get(w.gates[i][0], 0) for i in p["gates"])
                   for p in passes)
    if fam in ("fwd_fused", "fwd_gate"):
        return swept(FWD_OPS)
    if fam in ("adj_fused", "adj_gate"):
        return swept(REV_OPS)
    if fam in ("ham_fused", "ham_group", "ham_diag"):
        groups = len({tuple(sorted(q for q, l in ops if l in "XY")) for _c, ops in w.terms})
        return amps * (2 * len(w.terms) + 8 * groups)  # sign-weighted sums; complex MAC + energy
    return None


def alu_peak(sm_mhz: float | None, n_sm: int = 152) -> tuple[float, str]:
    """FP32 lane-op peak: SMs (read from the device) x 128 FP32 lanes x SM clock (sampled
    during the run)."""
    mhz = sm_mhz or 2070.0
    return n_sm * 128 * mhz * 1e6 / 1e9, f"{n_sm} SM x 128 FP32 lanes x {mhz:.0f} MHz (sampled)"


def family_bytes(fam: str, w, S: int, plan: dict, passes=None) -> float | None:
    """Algorithmic bytes per launch of a kernel family (one state traversal = S bytes
    read or written; Algorithm 1's cost unit, one gate primitive = O(2^n)).  Fused passes
    count the tiles they compute (passes: vqg_plan_pass entries); the last forward pass also
    writes the zeros of the tiles it skips."""
    if fam == "adj_gate":    # read phi, lambda; write phi, lambda
        return 4.0 * S
    if fam == "fwd_gate":    # read + write psi (CNOT/CZ touch part of it; counted whole)
        return 2.0 * S
    if fam == "adj_fused":
        # per reverse tile pass: read phi and lambda; write lambda except after the last
        # pass; write phi only when the next pass does not restart from a checkpoint
        P, C = plan.get("reverse_passes", 1), plan.get("checkpoints", 0)
        if not passes:
            return (2.0 * P + (P - 1) + max(P - 1 - C, 0)) * S / max(P, 1)
        w_phi = max(P - 1 - C, 0) / max(P - 1, 1)  # share of passes that write phi
        tot = 0.0
        for j, p in enumerate(passes):
            tot += p["active_tiles"] / p["tiles"] * S * (2.0 + ((1.0 + w_phi) if j > 0 else 0.0))
        return tot / len(passes)
    if fam == "fwd_fused":   # per forward tile pass: read + write psi
        if not passes:
            return 2.0 * S
        # computed tiles are read (at most: amplitudes known zero are skipped) and written;
        # the last pass also writes the zeros of the tiles it skips
        tot = 0.0
        for j, p in enumerate(passes):
            f = p["active_tiles"] / p["tiles"]
            tot += (0.0 if p["from_zero"] else f * S) + (S if j + 1 == len(passes) else f * S)
        return tot / len(passes)
    if fam == "ham_group":   # read psi, read + write lambda
        return 3.0 * S
    if fam == "ham_diag":    # read psi, write lambda
        return 2.0 * S
    if fam == "ham_fused":
        return 3.0 * S
    return None


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, dist):
    import torch

    from paper_2009_02823_gb300 import Circuit

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    w = _workload(args)
    S = (8 if args.dtype == "c64" else 16) << w.n
    stream = torch.cuda.Stream()  # every kernel of the step and both timing events go here
    spec = args.specialize if args.dtype == "c64" and args.fusion else 0
    t_make = time.perf_counter()  # includes compiling the specialised kernels (cached on disk)
    circ = Circuit(w.n, w.gates, w.n_params, args.dtype, stream=stream, c128_arith=args.c128_arith,
                   specialize=spec, fusion=bool(args.fusion))
    circ.set_hamiltonian(w.terms)
    t_make = time.perf_counter() - t_make
    theta_h = replica_theta(w.theta, rank)
    theta_d = torch.tensor(theta_h, dtype=torch.float64, device="cuda")
    e_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    g_d = torch.zeros(w.n_params, dtype=torch.float64, device="cuda")

    def step():
        circ.energy_and_gradient_device(theta_d.data_ptr(), e_d.data_ptr(), g_d.data_ptr())

    torch.cuda.synchronize()  # inputs were written on torch's default stream
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(dev)
    circ.set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    dev_ms = t0.elapsed_time(t1)
    stats = circ.kernel_stats()
    circ.set_profiling(False)
    ms_max = max_over_ranks(dev_ms, dist, "cuda")
    value = world * args.steps / (ms_max / 1e3)

    # end to end through the public host call: H2D theta, D2H energy + gradient per step
    e2e_steps = max(2, min(args.steps, 3))
    grad_h = np.zeros(w.n_params)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_e0 = time.perf_counter()
    for _ in range(e2e_steps):
        e_val, _g = circ.energy_and_gradient(theta_h, out=grad_h)
    t_e = max_over_ranks(time.perf_counter() - t_e0, dist, "cuda")
    e2e = {"value": world * e2e_steps / t_e, "unit": UNIT,
           "h2d_bytes_per_step": 8 * w.n_params, "d2h_bytes_per_step": 8 * (w.n_params + 1)}

    # roofline of the dominant kernel family (per-launch CUDA events inside the timed region)
    plan = circ.plan()
    passes = circ.plan_passes() if plan.get("tile_qubits") else None
    peak, peak_kind = _peaks()
    fam, (launches, tot_ms) = max(stats.items(), key=lambda kv: kv[1][1])
    roof = None
    per_family = {}
    total_ms = max(sum(v[1] for v in stats.values()), 1e-9)
    for f, (nl, ms) in stats.items():
        if not nl or ms <= 0:
            continue
        per = family_bytes(f, w, S, plan, passes)
        ops = family_alu_ops(f, w, passes)
        ent = {"launches": nl, "ms": round(ms, 3), "share": round(ms / total_ms, 4)}
        if per is not None:
            ent["hbm_gbs"] = round(per / (ms / nl / 1e3) / 1e9, 1)
            ent["hbm_frac"] = round(ent["hbm_gbs"] / peak, 4)
        if ops is not None:
            gops = ops * args.steps / (ms / 1e3) / 1e9
            ent["alu_gops"] = round(gops, 1)
            ent["alu_frac"] = round(gops / alu_peak(clk.get("sm_mhz"), n_sm)[0], 4)
        per_family[f] = ent
    if launches:
        avg_s = tot_ms / launches / 1e3
        per = family_bytes(fam, w, S, plan, passes)
        hbm = per / avg_s / 1e9 if per else None
        fused = fam.endswith("_fused")
        ops = family_alu_ops(fam, w, passes)
        if fused and ops:
            apk, apk_src = alu_peak(clk.get("sm_mhz"), n_sm)
            ach = ops * args.steps / (tot_ms / 1e3) / 1e9
            roof = {"bound": "alu", "kernel": fam, "achieved": round(ach, 1), "peak": round(apk, 1),
                    "unit": "GFLOP32-lane-op/s", "frac": round(ach / apk, 4), "peak_source": apk_src,
                    "ops_per_launch": ops / max(launches / args.steps, 1),
                    "hbm": {"achieved": round(hbm, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(hbm / peak, 4), "peak_source": peak_kind,
                            "bytes_per_launch": per},
                    "traffic": None, "launches": launches, "avg_launch_ms": round(tot_ms / launches, 4),
                    "share_of_step": round(tot_ms / total_ms, 4)}
        elif per is not None:
            roof = {"bound": "hbm", "kernel": fam, "achieved": round(hbm, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(hbm / peak, 4), "peak_source": peak_kind,
                    "traffic": None, "bytes_per_launch": per, "launches": launches,
                    "avg_launch_ms": round(tot_ms / launches, 4), "share_of_step": round(tot_ms / total_ms, 4)}
    if roof is not None:
        per_amp = NCU_TRAFFIC_PER_AMP_C64.get(fam) if args.dtype == "c64" else None
        if per_amp is not None:
            # the capture is of a pass that computes every tile; a launch moves that many
            # bytes per computed tile, so the average launch scales by the active share
            act = (sum(p["active_tiles"] / p["tiles"] for p in passes) / len(passes)
                   if passes and fam in ("adj_fused",) else 1.0)
            roof["traffic"] = round(per_amp * (1 << w.n) * act)
            roof["traffic_source"] = ("ncu dram__bytes_read+write per launch at n=26, scaled by 2^(n-26)"
                                      + (" x the mean share of computed tiles (%.4f)" % act if act < 1 else ""))
    gpu_launches = int(sum(v[0] for v in stats.values()))

    extra = {}
    if not args.no_batch:
        extra["batched"] = batched_rate(args, rank, world, dist)
    if rank == 0 and not args.no_extra and args.dtype == "c64":
        extra["c128_n%d" % w.n] = c128_rates(w, g_d, e_val, dev)
    if rank == 0 and not args.no_extra:
        extra["controlled"] = controlled_rate()
        extra["non_hermitian"] = non_hermitian_rate()
        extra["hadamard_product"] = product_rate()
        extra["p_scaling"] = p_scaling()
    if rank == 0 and not args.no_ps:
        extra["param_shift"] = param_shift_baseline(args, circ, w, theta_h, value / world)
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_sample(args, w, budget_s=args.cpu_budget, reps=3)
        if args.cpu_full_n > 0:
            cpu["full_gradient"] = cpu_full_gradient(args.cpu_full_n)
    else:
        cpu = None
    circ.close()
    if rank != 0:
        return None
    line = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128-float-float" if args.dtype == "c128" and args.c128_arith == "float-float" else args.dtype,
            "data": "synthetic (seeded; no dataset)",
            "config": _config(args, w, {"plan": plan, "specialize": spec, "setup_s": round(t_make, 2)}),
            "clocks": clk, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roof,
            "kernel_families": per_family, "energy": e_val,
            "amplitude_updates": amplitude_updates(w, S, value, peak, passes)}
    if cpu:
        line["cpu_baseline"] = cpu
    line.update(extra)
    return line


def amplitude_updates(w, S, grads_per_s, hbm_peak, passes=None):
    """Amplitude updates per second, (G + 2G) 2^n per gradient (G gate applications forward,
    two states un-applied per gate in reverse; a fused pass that skips tiles a |0...0> start
    leaves at zero counts only the tiles it computes), against the rate the HBM roofline
    allows a one-gate-per-pass schedule (each update reads and writes one amplitude)."""
    amp_bytes = S >> w.n
    applied = (sum(len(p["gates"]) * p["active_tiles"] / p["tiles"] for p in passes) if passes
               else w.n_gates)
    ups = 3 * applied * (1 << w.n) * grads_per_s
    roof = hbm_peak * 1e9 / (2 * amp_bytes)
    return {"per_s": ups, "unfused_hbm_roofline_per_s": roof, "ratio_to_unfused_roofline": round(ups / roof, 3)}


def c128_rates(w, g_c64_dev, e_c64, dev):
    """The same workload with complex128 amplitudes (the paper's double-precision state
    vector), timed on the GPU in both tile-pass arithmetics (FP64 and float-float): one
    untimed warm-up gradient, then one gradient timed with CUDA events on the circuit's
    stream, nvidia-smi clocks sampled meanwhile.  The FP64 gradient (the path that matches
    the oracle to 1e-10 in the parity tests) is also the reference for the complex64
    gradient of the timed run and for the float-float one: max-abs and norm-wise relative
    differences."""
    import torch

    from paper_2009_02823_gb300 import Circuit
    g64 = g_c64_dev.cpu().numpy()
    out, grads = {}, {}
    for arith in ("float-float", "fp64"):
        stream = torch.cuda.Stream()
        with Circuit(w.n, w.gates, w.n_params, "c128", stream=stream, c128_arith=arith) as c:
            c.set_hamiltonian(w.terms)
            th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
            e = torch.zeros(1, dtype=torch.float64, device="cuda")
            g = torch.zeros(w.n_params, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            c.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
            torch.cuda.synchronize()
            clocks = Clocks(dev)
            c.set_profiling(True)
            clocks.start()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            c.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
            t1.record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
            stats = c.kernel_stats()
            ms = t0.elapsed_time(t1)
            grads[arith] = (float(e.item()), g.cpu().numpy())
        out[arith] = {"ms_per_gradient": round(ms, 1), "gradients_per_s": round(1e3 / ms, 4),
                      "family_ms": {f: round(v[1], 1) for f, v in stats.items() if v[1] > 0.5},
                      "clocks": {"sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons")}}
    e128, g128 = grads["fp64"]
    scale = float(np.abs(g128).max())
    eff, gff = grads["float-float"]
    out["float-float"]["vs_fp64"] = {"max_abs_grad_err": float(np.abs(gff - g128).max()),
                                     "rel_grad_err": float(np.abs(gff - g128).max() / scale),
                                     "energy_err": abs(eff - e128)}
    out["c64_vs_fp64"] = {"max_abs_grad_err": float(np.abs(g64 - g128).max()),
                          "rel_grad_err": float(np.abs(g64 - g128).max() / scale),
                          "energy_err": abs(e_c64 - e128), "energy_c128": e128}
    out["timing"] = "one gradient each after one warm-up, CUDA events on the circuit's stream"
    return out


def batched_rate(args, rank=0, world=1, dist=None):
    """512-circuit batch (n 12..20, 4..16 layers, TFIM): circuit gradients per second
    through one persistent launch replayed from a CUDA graph (device buffers).  With
    several ranks the circuits are partitioned by cost and each rank runs its share;
    the rate divides all 512 circuits by the slowest rank's time."""
    import torch

    from paper_2009_02823_gb300 import workloads as W
    from paper_2009_02823_gb300.batch import Batch
    ws_all = W.batched()
    mine = partition([circuit_cost(w.n, w.n_gates, len(w.terms)) for w in ws_all], world)[rank]
    ws = [ws_all[b] for b in mine]
    stream = torch.cuda.Stream()
    b = Batch(ws, stream=stream)
    tune = b.autotune([w.theta for w in ws])  # picks the tile geometry (outside the timed region)
    th = torch.tensor(np.concatenate([w.theta for w in ws]), dtype=torch.float64, device="cuda")
    e = torch.zeros(len(ws), dtype=torch.float64, device="cuda")
    g = torch.zeros(th.numel(), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        b.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    t0.record(stream)
    for _ in range(reps):
        b.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1) / reps, dist, "cuda")
    info = b.info()
    b.close()
    seq = sequential_sample(ws, stream) if rank == 0 else None
    return {"workload": "512 circuits, n 12..20, 4..16 layers RY/RZ + CNOT ladder, TFIM h~U[0.5,1.5]",
            "ms_per_batch": round(ms, 3), "circuit_gradients_per_s": round(len(ws_all) / (ms / 1e3), 1),
            "circuits_per_rank": len(ws), "one_circuit_per_call": seq,
            "autotune": {"tile_qubits": tune["tile_qubits"], "reg_qubits": tune["fwd_reg_qubits"],
                         "candidates": tune["candidates"], "default_ms": round(tune["default_ms"], 3),
                         "best_ms": round(tune["best_ms"], 3)},
            "tasks": info["tasks"], "grid": info["grid"], "launches_per_batch": 2}


def sequential_sample(ws, stream, every=8):
    """The same circuits one per call (single-circuit device entry point, back to back on
    one stream): every `every`-th circuit timed, extrapolated to the whole list."""
    import torch

    from paper_2009_02823_gb300 import Circuit
    sample = ws[::every]
    circs, bufs = [], []
    for w in sample:
        c = Circuit(w.n, w.gates, w.n_params, "c64", stream=stream)
        c.set_hamiltonian(w.terms)
        th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        circs.append(c)
        bufs.append((th, torch.zeros(1, dtype=torch.float64, device="cuda"),
                     torch.zeros(w.n_params, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    for c, (th, e, g) in zip(circs, bufs):
        c.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for c, (th, e, g) in zip(circs, bufs):
        c.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) * len(ws) / len(sample)
    for c in circs:
        c.close()
    return {"circuits_timed": len(sample), "ms_extrapolated": round(ms, 3),
            "circuit_gradients_per_s": round(len(ws) / (ms / 1e3), 1)}


def workload_rate(w, dtype="c64", steps=3):
    """Gradients/s of one more workload through the same device entry point (CUDA events
    on a dedicated stream, one warm-up), with its per-family device times."""
    import torch

    from paper_2009_02823_gb300 import Circuit
    stream = torch.cuda.Stream()
    circ = Circuit(w.n, w.gates, w.n_params, dtype, stream=stream)
    circ.set_hamiltonian(w.terms)
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(w.n_params, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    circ.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        circ.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    circ.set_profiling(True)
    circ.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    stats = circ.kernel_stats()
    plan = circ.plan()
    circ.close()
    return {"workload": w.name, "n_qubits": w.n, "n_params": w.n_params, "n_gates": w.n_gates,
            "dtype": dtype, "ms_per_gradient": round(ms, 3), "gradients_per_s": round(1e3 / ms, 4),
            "family_ms": {f: round(v[1], 3) for f, v in stats.items() if v[1] > 0.01},
            "passes": {"forward": plan["forward_passes"], "hamiltonian": plan["hamiltonian_passes"],
                       "reverse": plan["reverse_passes"]}}


def controlled_rate():
    """Controlled-rotation ansatz (RX, RZ layers + CRX rings, App. A's controlled gates):
    n=30, 6 layers, P=540, TFIM."""
    from paper_2009_02823_gb300 import workloads as W
    gates, P = W.crx_ring(30, 6)
    rng = np.random.default_rng(W.SEED_BASE + 6)
    w = W.Workload("crx_ring_n30_L6_tfim", 30, gates, P, W.draw_theta(rng, P), W.tfim(30, 1.0))
    return workload_rate(w)


def non_hermitian_rate(steps=3):
    """Non-Hermitian operator (App. B.4): the bench circuit (n=30, 745 gates, P=600) with
    200 random Pauli strings whose coefficients are complex (real and imaginary parts
    N(0,1)): complex expectation + complex gradient per call."""
    import torch

    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300 import workloads as W
    w = W.config(3)
    rng = np.random.default_rng(W.SEED_BASE + 7)
    terms = [(complex(c, float(rng.normal())), ops) for c, ops in w.terms]
    stream = torch.cuda.Stream()
    circ = Circuit(w.n, w.gates, w.n_params, "c64", stream=stream)
    circ.set_operator(terms)
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    e = torch.zeros(2, dtype=torch.float64, device="cuda")
    g = torch.zeros(2 * w.n_params, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    circ.expectation_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        circ.expectation_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    circ.close()
    return {"workload": "hea_ry_rz_czbrick_n30_L10_rand200, complex coefficients", "dtype": "c64",
            "ms_per_gradient": round(ms, 3), "gradients_per_s": round(1e3 / ms, 4),
            "expectation": [float(e[0]), float(e[1])],
            "method": "A = B + iC: one forward sweep, Hamiltonian + reverse sweep per part"}


def product_rate(steps=3):
    """The paper's benchmark operator Hadamard^{(x)30} (Sec. 3) on the bench circuit (n=30,
    745 gates, P=600), from a random normalised input state generated on the device."""
    import torch

    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300 import workloads as W
    w = W.config(3)
    had = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    stream = torch.cuda.Stream()
    circ = Circuit(w.n, w.gates, w.n_params, "c64", stream=stream)
    circ.set_product_operator([(1.0, [had] * w.n)])
    gen = torch.Generator(device="cuda").manual_seed(W.SEED_BASE + 8)
    psi0 = torch.randn(1 << w.n, dtype=torch.complex64, device="cuda", generator=gen)
    psi0 /= torch.linalg.vector_norm(psi0)
    torch.cuda.synchronize()  # written on torch's stream; the library copies on its own
    circ.set_input_state(device_ptr=psi0.data_ptr())
    del psi0
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(w.n_params, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    circ.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        circ.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    circ.close()
    return {"workload": "hea_ry_rz_czbrick_n30_L10, operator Hadamard^(x)30, random input state",
            "dtype": "c64", "ms_per_gradient": round(ms, 3), "gradients_per_s": round(1e3 / ms, 4),
            "energy": float(e[0])}


def param_shift_baseline(args, circ, w, theta_h, adjoint_rate):
    """GPU parameter-shift gradient (2 energy evaluations per parameter occurrence)
    timed on a prefix of occurrences and extrapolated linearly: every shifted
    evaluation is the same work (a full forward sweep plus <H>)."""
    want = args.ps_evals // 2
    occ, last = 0, 0
    npar = {"RX": 1, "RY": 1, "RZ": 1, "U3": 3}
    for i, g in enumerate(w.gates):
        occ += npar.get(g[0], 0)
        last = i + 1
        if occ >= want:
            break
    total_occ = sum(npar.get(g[0], 0) for g in w.gates)
    circ.gradient_parameter_shift(theta_h, 0, 1)  # warm
    t0 = time.perf_counter()
    circ.gradient_parameter_shift(theta_h, 0, last)
    dt = time.perf_counter() - t0
    per_eval = dt / (2 * occ)
    full = per_eval * 2 * total_occ
    return {"evals_timed": 2 * occ, "s_per_energy_eval": round(per_eval, 5),
            "s_per_gradient_extrapolated": round(full, 3),
            "gradients_per_s": 1.0 / full,
            "adjoint_speedup": round(adjoint_rate * full, 2), "target_speedup": w.n_params / 4}


def p_scaling(n=20, layers=(4, 8, 16, 32)):
    """The paper's cost claim (Sec. 2.3, Fig. 2): a reverse-mode gradient costs O(P) gate
    applications, the faithful route (Algorithm 2 / parameter shift) O(P^2).  Adjoint
    gradients and complete GPU parameter-shift gradients (2 energies per parameter, each a
    whole forward sweep) on the RY/RZ + CZ brickwork at n=20 for growing depth; the slopes
    of log time against log P (the paper fits the same log-log lines)."""
    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300 import workloads as W
    rows = []
    for L in layers:
        w = W.config(3, n=n, layers=L)
        with Circuit(w.n, w.gates, w.n_params, "c64") as c:
            c.set_hamiltonian(w.terms)
            for _ in range(2):
                c.energy_and_gradient(w.theta)
            reps = 10
            t0 = time.perf_counter()
            for _ in range(reps):
                c.energy_and_gradient(w.theta)
            t_adj = (time.perf_counter() - t0) / reps
            c.gradient_parameter_shift(w.theta, 0, 1)
            t0 = time.perf_counter()
            c.gradient_parameter_shift(w.theta)
            t_ps = time.perf_counter() - t0
        rows.append({"layers": L, "P": w.n_params, "adjoint_ms": round(t_adj * 1e3, 3),
                     "param_shift_ms": round(t_ps * 1e3, 1), "ratio": round(t_ps / t_adj, 1)})
    lp = np.log([r["P"] for r in rows])
    slope = lambda key: round(float(np.polyfit(lp, np.log([r[key] for r in rows]), 1)[0]), 3)
    top = lambda key: round(float(np.log(rows[-1][key] / rows[-2][key]) / np.log(rows[-1]["P"] / rows[-2]["P"])), 3)
    return {"workload": f"hea_ry_rz_czbrick n={n}, layers {list(layers)}, 200 random Paulis, c64",
            "points": rows, "slope_adjoint": slope("adjoint_ms"), "slope_param_shift": slope("param_shift_ms"),
            "slope_ratio": slope("ratio"),
            "slope_top_pair": {"adjoint": top("adjoint_ms"), "param_shift": top("param_shift_ms")},
            "note": "costs independent of P (launches, host syncs, the Hamiltonian passes) flatten "
                    "both slopes at n=20; the asymptotic values are 1 and 2",
            "host_api": "energy_and_gradient (synchronous host calls)"}


# ---------------------------------------------------------------- CPU oracle baseline
def _primitive_total(L, oracle, w, psi, lam, gt, th, coef, let, budget_s, t_start):
    """One sample of the oracle's Algorithm-1 primitives at the workload's n, extrapolated
    to a whole gradient; returns (seconds per gradient, kinds timed, parameter slots)."""
    import ctypes
    n = w.n
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    kinds = {}
    for i, g in enumerate(w.gates):
        kinds.setdefault(g[0], i)
    per = {}
    # forward + adjoint application per kind (one call each; the work is data-independent)
    for kind, i in kinds.items():
        t0 = time.perf_counter()
        L.oracle_apply_gate(n, ptr(psi), ptr(gt[i]), ptr(th), 0)
        t1 = time.perf_counter()
        L.oracle_apply_gate(n, ptr(psi), ptr(gt[i]), ptr(th), 1)
        t2 = time.perf_counter()
        per[kind] = (t1 - t0, t2 - t1)
        if time.perf_counter() - t_start > budget_s:
            break
    # derivative step: clone + apply dU + inner product (Algorithm 1's derivative step)
    t0 = time.perf_counter()
    mu = psi.copy()
    d = oracle.gate_derivative("RY", 0, [0.3])
    L.oracle_apply_matrix_1q(n, ptr(mu), 0, ptr(np.ascontiguousarray(d.reshape(4))))
    out = np.zeros(2)
    L.oracle_inner_parts(n, ptr(lam), ptr(mu), ptr(out))
    t_deriv = time.perf_counter() - t0
    del mu
    # Hamiltonian: time a few terms, scale by the term count
    k_terms = max(1, min(3, len(w.terms)))
    t0 = time.perf_counter()
    L.oracle_apply_hamiltonian(n, k_terms, ptr(coef), ptr(let), ptr(psi), ptr(lam))
    t_h = (time.perf_counter() - t0) / k_terms * len(w.terms)
    # Algorithm 1 gradient: G forward + H + per gate (U^dag phi, U^dag lambda) + per slot deriv
    total = t_h
    n_slots = 0
    for g in w.gates:
        f, a = per.get(g[0], per.get("RY", (0.0, 0.0)))
        total += f + 2 * a
        n_slots += {"RX": 1, "RY": 1, "RZ": 1, "U3": 3}.get(g[0], 0)
    total += n_slots * t_deriv
    return total, sorted(per), n_slots, k_terms


def cpu_full_gradient(n=22):
    """One complete Algorithm-1 gradient of the oracle, timed in full, on the bench recipe
    at n qubits (same circuit structure and Hamiltonian recipe, smaller state)."""
    import oracle
    from paper_2009_02823_gb300 import workloads as W
    w = W.config(3, n=n)
    t0 = time.perf_counter()
    oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    dt = time.perf_counter() - t0
    return {"workload": w.name, "n_qubits": n, "n_params": w.n_params, "n_gates": w.n_gates,
            "s_per_gradient": round(dt, 2), "gradients_per_s": 1.0 / dt, "cores": oracle.threads(),
            "routine": "oracle.gradient_alg1 (complex128, Algorithm 1), timed in full"}


def cpu_baseline_sample(args, w, budget_s=20.0, reps=1):
    """The oracle as it stands, on the host cores, on a bounded sample of the same
    workload: its Algorithm-1 primitives (apply gate, apply adjoint gate, derivative
    matrix + clone + inner product, one Hamiltonian term) are timed at the workload's
    n on the workload's own gates/terms, and the full Algorithm-1 gradient time is
    extrapolated from the per-primitive times and the workload's gate and term counts.
    With reps > 1 the sample is repeated and the median extrapolation is reported with
    the spread of the samples."""
    import oracle
    L = oracle._load()
    n = w.n
    dim = 1 << n
    t_start = time.perf_counter()
    try:
        psi = np.zeros(dim, dtype=np.complex128)
        lam = np.zeros(dim, dtype=np.complex128)
    except MemoryError:
        return {"value": None, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                "sample": "host memory too small for the workload's state vectors"}
    psi[0] = 1.0
    lam[:] = psi
    gt = oracle.gate_table(w.gates)
    th = np.ascontiguousarray(w.theta)
    coef, let = oracle.letter_table(w.terms, n)
    totals = []
    for _ in range(max(1, reps)):
        total, kinds, n_slots, k_terms = _primitive_total(L, oracle, w, psi, lam, gt, th, coef, let,
                                                          budget_s * max(1, reps), t_start)
        totals.append(total)
    total = statistics.median(totals)
    sample_s = time.perf_counter() - t_start
    res = {"value": 1.0 / total, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
           "sample": (f"oracle primitives at n={n} (complex128): one forward and one adjoint "
                      f"application per gate kind {kinds}, one derivative+clone+inner "
                      f"product, {k_terms} of {len(w.terms)} Hamiltonian terms; Algorithm 1 "
                      f"time extrapolated over {w.n_gates} gates / {n_slots} parameter slots "
                      f"= {total:.1f} s per gradient (median of {len(totals)} samples); "
                      f"sample took {sample_s:.1f} s"),
           "extrapolated_s_per_gradient": round(total, 2)}
    if len(totals) > 1:
        res["samples_s_per_gradient"] = [round(t, 1) for t in totals]
        res["spread"] = round((max(totals) - min(totals)) / total, 4)
    return res


def run_reference(args, rank):
    if rank != 0:
        return None
    import oracle
    w = _workload(args)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline_sample(args, w, budget_s=args.cpu_budget)
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline_sample(args, w, budget_s=args.cpu_budget)
        if last["value"]:
            vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = statistics.median(vals) if vals else None
    cpu = dict(last or {})
    cpu["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall / max(args.steps, 1), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic (seeded; no dataset)",
            "config": _config(args, w, {"amplitudes": "c128 (CPU oracle, one gate at a time)",
                                        "parallelism": "host cores (rank 0 only)"}),
            "cpu_baseline": cpu, "cores": oracle.threads(),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--c128-arith", default="fp64", choices=["fp64", "float-float"],
                    help="arithmetic of the complex128 tile passes")
    ap.add_argument("--specialize", type=int, default=2,
                    help="complex64: kernels generated for the circuit's passes, compiled when the circuit is made "
                         "(outside the timed region): 1 forward and Hamiltonian passes, 2 (default) also the "
                         "reverse passes; 0 the generic kernels")
    ap.add_argument("--fusion", type=int, default=1,
                    help="0: one kernel per gate (the unfused passes, for their HBM figures)")
    ap.add_argument("--cfg", type=int, default=3)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--layers", type=int, default=None)
    ap.add_argument("--no-ps", action="store_true", help="skip the GPU parameter-shift baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-launch figure")
    ap.add_argument("--ps-evals", type=int, default=16)
    ap.add_argument("--no-extra", action="store_true", help="skip the extra-workload figures")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--cpu-full-n", type=int, default=22,
                    help="qubits of the complete CPU oracle gradient timed beside the sample (0: skip)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as tdist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            tdist.init_process_group("nccl")
            dist = tdist
        line = run_ours(args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
    if rank == 0 and line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
