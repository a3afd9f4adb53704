"""Benchmark: the 30-qubit gate benchmark on one GB300 (per rank).

Workload (one "step"): a 2^30-amplitude complex128 state holding i.i.d. Gaussian
amplitudes normalised to one; each of the gate types H, X, RZ, U3, CNOT, CZ, SWAP,
CU3 applied 30 times across targets 0..29 (two-qubit gates on (q, q+1 mod 30)), one
streaming kernel launch per gate: 240 gates per step.  Inputs (16 GiB) are far larger
than L2, so no flush is needed between iterations.

Prints ONE JSON line (rank 0): value = gates/s over all ranks (device-timed with CUDA
events on the launching stream), per-gate-type GB/s, the roofline of the dominant
kernel, clocks sampled during the timed region, the end-to-end rate through the C ABI
with host buffers, and the CPU oracle timed on a bounded sample.

``--impl reference`` times the CPU oracle instead (bounded sample per step).
Multi-GPU: one process per GPU under torchrun; ranks run independent replicas
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS = 30
GATE_TYPES = ("h", "x", "rz", "u3", "cnot", "cz", "swap", "cu3")
METRIC = "gates/sec (30-qubit gate benchmark, complex128, gate-by-gate)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--qubits", type=int, default=N_QUBITS)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-gates", type=int, default=2)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the context rows (planned circuits, the other dtype)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sweep_gates(n):
    from paper_2409_14697_gb300 import inputs
    return {name: inputs.gate_sweep(n, name, seed=2, count=30) for name in GATE_TYPES}


def alg_bytes_per_gate(name, q_list, n, B):
    """Algorithmic HBM bytes of one application (read + write of the amplitudes it
    changes; selecting bits inside a 32-byte sector count as full passes)."""
    full = 2.0 * B * (1 << n)
    sector_bits = 1 if B == 16 else 2
    if name in ("h", "x", "rz", "u3"):
        return full
    a, b = q_list
    if name == "cz":
        f = (a >= sector_bits) + (b >= sector_bits)
        return full / (4 if f == 2 else 2 if f == 1 else 1)
    if name == "swap":
        return full / 2 if (a >= sector_bits and b >= sector_bits) else full
    if name in ("cnot", "cu3"):
        return full / 2 if a >= sector_bits else full
    return full


def run_ours(args, rank, world, local):
    import torch
    from paper_2409_14697_gb300 import inputs, qs

    torch.cuda.set_device(local)
    n = args.qubits
    dt = qs.QS_C128 if args.dtype == "c128" else qs.QS_C64
    B = 16 if dt == qs.QS_C128 else 8
    npdt = np.complex128 if dt == qs.QS_C128 else np.complex64
    stream = torch.cuda.Stream()
    h = qs.qs_create(n, dt)
    qs.qs_set_stream(h, stream.cuda_stream)
    # pinned host copy of the initial state (also the e2e input buffer)
    host_in = torch.empty((1 << n) * 2, dtype=torch.float64 if B == 16 else torch.float32, pin_memory=True)
    hv = host_in.numpy().view(npdt)
    inputs.gaussian_state(n, seed=7, out=hv)
    qs.qs_set_amplitudes_from(h, 0, 1 << n, host_in.data_ptr())
    sweeps = sweep_gates(n)
    recs = {name: qs.gate_records(g) for name, g in sweeps.items()}
    opts = qs.options(mode=qs.QS_MODE_GATE)
    n_gates = sum(len(g) for g in sweeps.values())

    def step(events=None):
        for i, name in enumerate(GATE_TYPES):
            if events is not None:
                events[i].record(stream)
            qs.qs_apply_circuit(h, recs[name], opts)
        if events is not None:
            events[-1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(GATE_TYPES) + 1)] for _ in range(args.steps)]
    l0 = qs.qs_launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(args.steps):
            step(evs[s])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = qs.qs_launch_count() - l0
    per_type_ms = {name: 0.0 for name in GATE_TYPES}
    total_ms = 0.0
    for s in range(args.steps):
        for i, name in enumerate(GATE_TYPES):
            d = evs[s][i].elapsed_time(evs[s][i + 1])
            per_type_ms[name] += d
            total_ms += d
    ms_per_step = total_ms / args.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_per_step], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item())
    value = world * n_gates / (ms_per_step * 1e-3)

    peak, peak_kind = load_peaks()
    per_gate = {}
    for name in GATE_TYPES:
        launch_ms = per_type_ms[name] / (args.steps * len(sweeps[name]))
        byts = float(np.mean([alg_bytes_per_gate(name, g[1], n, B) for g in sweeps[name]]))
        per_gate[name] = {"ms": round(launch_ms, 4), "alg_bytes": byts,
                          "GBps": round(byts / (launch_ms * 1e-3) / 1e9, 1),
                          "frac_of_measured_hbm": round(byts / (launch_ms * 1e-3) / 1e9 / peak, 3),
                          "share": round(per_type_ms[name] / total_ms, 3)}
    dom = max(GATE_TYPES, key=lambda k: per_type_ms[k])
    traffic = load_traffic(dom, n, args.dtype)
    roof = {"kernel": f"k_stream[{dom}]", "bound": "hbm", "achieved": per_gate[dom]["GBps"],
            "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": round(per_gate[dom]["GBps"] / peak, 3), "traffic": traffic}
    all_bytes = sum(per_gate[k]["alg_bytes"] * len(sweeps[k]) for k in GATE_TYPES)
    agg_gbps = all_bytes / (ms_per_step * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(qs, h, host_in, recs, opts, n, B, n_gates, world)
    extra = {}
    if not args.no_extra:
        extra["planned"] = time_planned(qs, h, stream, recs, n, B)
    qs.qs_destroy(h)
    del host_in

    # correctness spot check of this run (norm preserved by the unitary sweep)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "gates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if B == 16 else "f32", "data": "synthetic (seeded Gaussian state, seeded angles)",
        "config": {"workload": f"{n}-qubit gate benchmark, {args.dtype}, 8 gate types x 30 targets, gate-by-gate",
                   "qubits": n, "state_bytes": B << n, "gates_per_step": n_gates,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
        "hbm_GBps_all_gates": round(agg_gbps, 1),
        "per_gate": per_gate,
        "roofline": roof,
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "wall_s_timed": round(wall, 3),
    }
    if e2e:
        out["e2e"] = e2e
    out.update(extra)
    return out


def time_planned(qs, h, stream, recs, n, B):
    """Context row: each gate type's 30 gates as ONE planned circuit (in-cache chunk
    passes, QS_MODE_AUTO).  Reports ms per 30 gates, passes, and effective gate GB/s
    (30 x a full pass of bytes / time: may exceed the roofline, that is what fusion buys)."""
    import torch
    out = {}
    opts = qs.options(mode=qs.QS_MODE_AUTO)
    for name in GATE_TYPES:
        qs.qs_apply_circuit(h, recs[name], opts)   # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            qs.qs_apply_circuit(h, recs[name], opts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        st = qs.qs_last_stats(h)
        out[name] = {"ms_per_30": round(ms, 3), "passes": int(st["passes"]),
                     "alg_GBps": round(st["bytes"] / (ms * 1e-3) / 1e9, 1),
                     "effective_gate_GBps": round(30 * 2 * B * (1 << n) / (ms * 1e-3) / 1e9, 1)}
    return out


def run_e2e(qs, h, host_in, recs, opts, n, B, n_gates, world):
    """Same metric through the C ABI with host buffers: each step copies the initial
    state from pinned host memory (H2D), applies the 240 gates, and copies the final
    state back to pinned host memory (D2H)."""
    import torch
    host_out = torch.empty_like(host_in, pin_memory=True)
    reps = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        qs.qs_set_amplitudes_from(h, 0, 1 << n, host_in.data_ptr())
        for name in GATE_TYPES:
            qs.qs_apply_circuit(h, recs[name], opts)
        qs.qs_amplitudes_into(h, 0, 1 << n, host_out.data_ptr())
    dt = (time.perf_counter() - t0) / reps
    rec_bytes = 72 * n_gates
    return {"value": round(world * n_gates / dt, 2), "unit": "gates/s",
            "h2d_bytes_per_step": (B << n) + rec_bytes, "d2h_bytes_per_step": B << n,
            "ms_per_step": round(dt * 1e3, 2), "steps": reps}


def load_traffic(kernel_gate, n, dtype):
    """Per-launch DRAM bytes from the committed ncu summary, if one matches."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        return t.get(f"{kernel_gate}:{n}:{dtype}")
    except Exception:
        return None


def cpu_baseline(args, n_gates_sample):
    """The CPU oracle, as it stands, on the first gate of the first types of the sweep
    at full size (same qubit count), timed on the host."""
    import oracle
    from paper_2409_14697_gb300 import inputs
    n = args.qubits
    sweeps = sweep_gates(n)
    sample = [sweeps[name][0] for name in GATE_TYPES[:n_gates_sample]]
    psi = oracle.zero_state(n)
    t0 = time.perf_counter()
    oracle.run(psi, n, sample)
    dt = time.perf_counter() - t0
    return {"value": round(len(sample) / dt, 4), "unit": "gates/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(sample)} gates ({', '.join(g[0] for g in sample)}) of the sweep on a "
                      f"{n}-qubit complex128 state, {dt:.1f} s"}


def run_reference(args, rank, world):
    import oracle
    n = args.qubits
    sweeps = sweep_gates(n)
    seq = [g for name in GATE_TYPES for g in sweeps[name][:1]]
    psi = oracle.zero_state(n)
    times = []
    for s in range(args.warmup + args.steps):
        g = seq[s % len(seq)]
        t0 = time.perf_counter()
        oracle.run(psi, n, [g])
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    v = len(times) / sum(times)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "gates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(times) / len(times), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{n}-qubit gate benchmark, c128, 8 gate types x 30 targets, gate-by-gate",
                       "qubits": n},
            "cpu_baseline": {"value": round(v, 4), "unit": "gates/s", "cores": 1, "kind": "oracle",
                             "sample": f"one gate per step, cycling {', '.join(GATE_TYPES)}, {n} qubits"},
            "e2e": {"value": round(v, 4), "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank == 0:
        if not args.no_cpu and world == 1:
            out["cpu_baseline"] = cpu_baseline(args, args.cpu_sample_gates)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
