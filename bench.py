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

# Hardware work queues for concurrent streams (read when the CUDA context is created): with
# the default 8, the served workload's 16 slot streams share queues and a small request's
# kernels wait behind a large one's.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS = 30
# complex128 arithmetic by --precision (the values of QS_PREC_DEFAULT / _FP64 / _DF32)
PRECISIONS = {"ix64": 0, "fp64": 1, "df32": 2}
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
    ap.add_argument("--workload", default="gates30",
                    choices=["gates30", "circuit12", "circuits33", "batched", "served", "reductions", "paper"],
                    help="gates30: the headline benchmark; the others print their own JSON line")
    ap.add_argument("--count", type=int, default=0, help="circuits/requests for batched/served")
    ap.add_argument("--fuse-k", type=int, default=0,
                    help="circuits33: fusion width (default: register phases k=1, then tensor-core blocks k=5)")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--no-rphases", action="store_true",
                    help="complex64 passes: one shared-memory sweep per op (no register phases)")
    ap.add_argument("--precision", default="ix64", choices=["ix64", "fp64", "df32"],
                    help="complex128 arithmetic of the served and paper workloads (ix64: the "
                         "library default, integer products for one-qubit dense and diagonal ops)")
    ap.add_argument("--loads", default="",
                    help="served: comma-separated offered loads in req/s for a load sweep")
    ap.add_argument("--no-workloads", action="store_true",
                    help="gates30: skip the compact summaries of the other workloads")
    ap.add_argument("--families", default="brickwork40,qaoa_p4,tfim50",
                    help="circuits33: comma-separated circuit families to run")
    return ap.parse_args()


def max_over_ranks(x: float, world: int) -> float:
    """Max of x over all ranks (replicas are timed independently; the slowest rank sets
    the job's step time).  Works with the nccl (CUDA tensor) and gloo (CPU tensor)
    backends."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, ms_per_step: float, world: int) -> float:
    """Whole-job throughput: every rank processed units_per_rank per step."""
    return world * units_per_rank / (ms_per_step * 1e-3)


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


def tf32_peak_tflops():
    """Dense TF32 tensor peak: the measured bf16 peak (sustained, for kernels inside a long
    circuit) times the nominal TF32 / bf16 ratio 1.1 / 2.25; else the fallback 1.7 PF/s
    sustained bf16 times the same ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        bf16, kind = float(p.get("bf16_tflops_sustained") or p["bf16_tflops"]), "measured"
    except Exception:
        bf16, kind = 1700.0, "fallback"
    return bf16 * 1.1 / 2.25, kind


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


def alg_bytes_per_gate(name, q_list, n, B, last=True):
    """Algorithmic HBM bytes of one application (read + write of the amplitudes it
    changes; selecting bits inside a 32-byte sector count as full passes).  Gate-by-gate
    runs apply every RZ of a call but the last as diag(1, e^{i theta}), which changes only
    the half with the target bit set; the last carries the collected global phase and
    changes every amplitude (last=True)."""
    full = 2.0 * B * (1 << n)
    sector_bits = 1 if B == 16 else 2
    if name == "rz":
        return full if (last or q_list[0] < sector_bits) else full / 2
    if name in ("h", "x", "u3"):
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


def sweep_bytes(name, gates, n, B):
    """Mean algorithmic bytes per gate of one sweep applied as one call."""
    return float(np.mean([alg_bytes_per_gate(name, g[1], n, B, last=(i == len(gates) - 1))
                          for i, g in enumerate(gates)]))


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
    # correctness check of this run: the sweep is unitary, so the squared norm of the
    # normalised initial state survives the warm-up and timed steps (FP64 rounding only)
    norm_after = qs.qs_norm(h)
    check = {"norm_after_timed_steps_minus_1": norm_after - 1.0,
             "gates_applied": n_gates * (args.warmup + args.steps),
             "ok": bool(abs(norm_after - 1.0) <= 1e-12)}
    per_type_ms = {name: 0.0 for name in GATE_TYPES}
    total_ms = 0.0
    for s in range(args.steps):
        for i, name in enumerate(GATE_TYPES):
            d = evs[s][i].elapsed_time(evs[s][i + 1])
            per_type_ms[name] += d
            total_ms += d
    ms_per_step = max_over_ranks(total_ms / args.steps, world)
    value = aggregate_rate(n_gates, ms_per_step, world)

    peak, peak_kind = load_peaks()
    per_gate = {}
    for name in GATE_TYPES:
        launch_ms = per_type_ms[name] / (args.steps * len(sweeps[name]))
        byts = sweep_bytes(name, sweeps[name], n, B)
        per_gate[name] = {"ms": round(launch_ms, 4), "alg_bytes": byts,
                          "GBps": round(byts / (launch_ms * 1e-3) / 1e9, 1),
                          "frac_of_measured_hbm": round(byts / (launch_ms * 1e-3) / 1e9 / peak, 3),
                          "share": round(per_type_ms[name] / total_ms, 3)}
    dom = max(GATE_TYPES, key=lambda k: per_type_ms[k])
    # complex128 default arithmetic: integer products for U3, CU3, RZ (QS_PREC_IX64)
    ix = B == 16 and dom in ("u3", "cu3", "rz")
    traffic = load_traffic(dom, n, args.dtype, "ix" if ix else "fp64")
    hbm = {"achieved": per_gate[dom]["GBps"], "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
           "frac": round(per_gate[dom]["GBps"] / peak, 3)}
    fp64 = fp64_roof(dom, n, B, per_type_ms[dom] / (args.steps * len(sweeps[dom])), ix=ix)
    if fp64 and not ix and fp64["frac"] > hbm["frac"]:
        roof = {"kernel": f"k_stream[{dom}]", "bound": "alu", "achieved": fp64["achieved"],
                "peak": fp64["peak"], "unit": fp64["unit"], "frac": fp64["frac"],
                "peak_source": fp64["peak_source"], "dgemm_measured_peak": fp64["dgemm_measured_peak"],
                "frac_of_dgemm": fp64["frac_of_dgemm"], "traffic": traffic, "hbm": hbm}
    else:
        roof = {"kernel": f"k_stream[{dom}]", "bound": "hbm", "achieved": hbm["achieved"], "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": hbm["frac"], "traffic": traffic}
        if fp64:
            roof["fp64"] = fp64
    all_bytes = sum(per_gate[k]["alg_bytes"] * len(sweeps[k]) for k in GATE_TYPES)
    agg_gbps = all_bytes / (ms_per_step * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        qs.qs_destroy(h)    # the e2e states are its own
        h = None
        e2e = run_e2e(qs, host_in, recs, opts, n, B, n_gates, world, dt)
        h = qs.qs_create(n, dt)
        qs.qs_set_stream(h, stream.cuda_stream)
        qs.qs_set_amplitudes_from(h, 0, 1 << n, host_in.data_ptr())
    extra = {}
    if not args.no_extra:
        extra["planned"] = time_planned(qs, h, stream, recs, n, B)
        if B == 16:
            extra["df32"] = time_prec(qs, h, stream, recs, n, sweeps, peak, qs.QS_PREC_DF32)
            extra["fp64_native"] = time_prec(qs, h, stream, recs, n, sweeps, peak, qs.QS_PREC_FP64)
            extra["c64"] = time_c64(qs, stream, n, sweeps, peak)
    qs.qs_destroy(h)
    del host_in

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "gates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # complex128: FP64 storage and additions, 64-bit integer significand products for
        # U3, CU3 and RZ (config.arithmetic)
        "dtype": "f64+i64" if B == 16 else "f32", "data": "synthetic (seeded Gaussian state, seeded angles)",
        "config": {"workload": f"{n}-qubit gate benchmark, {args.dtype}, 8 gate types x 30 targets, gate-by-gate",
                   "qubits": n, "state_bytes": B << n, "gates_per_step": n_gates,
                   "arithmetic": ("U3, CU3 and RZ: exact 64-bit integer significand products, one "
                                  "signed 64-bit accumulator per output aligned to its largest term, "
                                  "one rounding to FP64 (QS_PREC_IX64, the default; one group in four, "
                                  "phases one in six, in native FP64); H: FP64 additions; X, CNOT, "
                                  "SWAP, CZ: moves and sign flips" if B == 16 else "FP32"),
                   "gate_forms": "one launch per gate; every RZ of a call but its last multiplies only "
                                 "the half of the state where its qubit is 1 (the global phase joins "
                                 "the call's last RZ); Hadamards run as unscaled butterflies whose "
                                 "2^(-k/2) scale joins a later H (the call's last, or every 64th, to "
                                 "keep the range); the call's final state is exact; per_gate bytes "
                                 "count what each launch moves",
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
        "hbm_GBps_all_gates": round(agg_gbps, 1),
        "per_gate": per_gate,
        "roofline": roof,
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "wall_s_timed": round(wall, 3),
        "check": check,
    }
    if e2e:
        out["e2e"] = e2e
    out.update(extra)
    return out


def time_prec(qs, h, stream, recs, n, sweeps, peak, precision):
    """Context row: the same gate-by-gate sweep with another complex128 arithmetic
    (QS_PREC_DF32: IEEE-double storage, FP32-pair compensated arithmetic; QS_PREC_FP64:
    native FP64 instructions for every gate)."""
    import torch
    opts = qs.options(mode=qs.QS_MODE_GATE, precision=precision)
    for name in GATE_TYPES:
        qs.qs_apply_circuit(h, recs[name], opts)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(GATE_TYPES) + 1)]
    for i, name in enumerate(GATE_TYPES):
        evs[i].record(stream)
        qs.qs_apply_circuit(h, recs[name], opts)
    evs[-1].record(stream)
    torch.cuda.synchronize()
    per, tot = {}, 0.0
    for i, name in enumerate(GATE_TYPES):
        ms = evs[i].elapsed_time(evs[i + 1])
        tot += ms
        byts = sweep_bytes(name, sweeps[name], n, 16)
        per[name] = {"ms": round(ms / len(sweeps[name]), 4),
                     "GBps": round(byts / (ms / len(sweeps[name]) * 1e-3) / 1e9, 1)}
        per[name]["frac_of_measured_hbm"] = round(per[name]["GBps"] / peak, 3)
    n_g = sum(len(g) for g in sweeps.values())
    return {"value": round(n_g / (tot * 1e-3), 2), "unit": "gates/s", "ms_per_step": round(tot, 3),
            "per_gate": per}


def time_c64(qs, stream, n, sweeps, peak):
    """Context row: the same gate-by-gate sweep on a complex64 state of the same qubit count
    (8 GiB at 30 qubits): every one-qubit gate is an HBM-bound pass there."""
    import torch
    h = qs.qs_create(n, qs.QS_C64)
    try:
        qs.qs_set_stream(h, stream.cuda_stream)
        recs = {name: qs.gate_records(g) for name, g in sweeps.items()}
        opts = qs.options(mode=qs.QS_MODE_GATE)
        for name in GATE_TYPES:
            qs.qs_apply_circuit(h, recs[name], opts)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(GATE_TYPES) + 1)]
        for i, name in enumerate(GATE_TYPES):
            evs[i].record(stream)
            qs.qs_apply_circuit(h, recs[name], opts)
        evs[-1].record(stream)
        torch.cuda.synchronize()
    finally:
        qs.qs_destroy(h)
    per, tot = {}, 0.0
    for i, name in enumerate(GATE_TYPES):
        ms = evs[i].elapsed_time(evs[i + 1])
        tot += ms
        byts = sweep_bytes(name, sweeps[name], n, 8)
        per[name] = {"ms": round(ms / len(sweeps[name]), 4),
                     "GBps": round(byts / (ms / len(sweeps[name]) * 1e-3) / 1e9, 1)}
        per[name]["frac_of_measured_hbm"] = round(per[name]["GBps"] / peak, 3)
    n_g = sum(len(g) for g in sweeps.values())
    return {"value": round(n_g / (tot * 1e-3), 2), "unit": "gates/s", "ms_per_step": round(tot, 3),
            "per_gate": per}


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


def run_e2e(qs, host_in, recs, opts, n, B, n_gates, world, dt, in_flight=3, steps=12):
    """Same metric through the C ABI with host buffers.  Each step copies the initial state
    from pinned host memory into a state (H2D), applies the 240 gates and copies the final
    state back into pinned host memory (D2H); the host waits for a step's result before
    it reuses that step's buffers.  `in_flight` states on their own streams keep that many
    steps in flight (as the serving loop does with its slots): step s runs on state
    s % in_flight with the stream-ordered copy entry points, and its gates wait (CUDA event)
    for the gates of step s - 1, so one step's copies run under another's gates instead of
    the states computing in lockstep.  The first step's input and the last step's result,
    which no other step's gates can hide, use the synchronous entry points (a copy kernel
    over the CPU-GPU link, at full speed from the first byte)."""
    import torch
    states, streams = [], []
    for _ in range(in_flight):
        st = qs.qs_create(n, dt)
        sm = torch.cuda.Stream()
        qs.qs_set_stream(st, sm.cuda_stream)
        states.append(st)
        streams.append(sm)
    outs = [torch.empty_like(host_in, pin_memory=True) for _ in range(in_flight)]
    N = 1 << n
    try:
        for st in states:
            qs.qs_synchronize(st)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = None
        for s in range(steps):
            k = s % in_flight
            st, sm = states[k], streams[k]
            if s >= in_flight:
                qs.qs_synchronize(st)             # step s - in_flight's final state is on the host
                float(outs[k][0])
            if s == 0:
                qs.qs_set_amplitudes_from(st, 0, N, host_in.data_ptr())
            else:
                qs.qs_set_amplitudes_async(st, 0, N, host_in.data_ptr())
            if prev is not None:
                sm.wait_event(prev)
            for name in GATE_TYPES:
                qs.qs_apply_circuit(st, recs[name], opts)
            prev = torch.cuda.Event()
            prev.record(sm)
            if s == steps - 1:
                qs.qs_amplitudes_into(st, 0, N, outs[k].data_ptr())
            else:
                qs.qs_amplitudes_async(st, 0, N, outs[k].data_ptr())
        for st in states:
            qs.qs_synchronize(st)
        wall = (time.perf_counter() - t0) / steps
    finally:
        for st in states:
            qs.qs_destroy(st)
    rec_bytes = 72 * n_gates
    return {"value": round(world * n_gates / wall, 2), "unit": "gates/s",
            "h2d_bytes_per_step": (B << n) + rec_bytes, "d2h_bytes_per_step": B << n,
            "ms_per_step": round(wall * 1e3, 2), "steps": steps, "states_in_flight": in_flight}


# FP64 instructions per amplitude (FMA-class issues, one FP64 pipe slot each) of the
# complex128 streaming updates; the other gate types issue none on the FP64 pipe.  In a
# gate-by-gate call of 30: RZ, 29 change half the amplitudes (4 per changed amplitude) and
# the last all; H, 29 are the unscaled butterfly (2) and the last carries the scale (3).
FP64_INSTR_PER_AMP = {"h": (29 * 2 + 3) / 30, "rz": (29 * 2 + 4) / 30, "u3": 7, "cu3": 3.5}
# The default complex128 arithmetic (QS_PREC_IX64) of the streaming U3, CU3 and RZ kernels:
# one group in four (phases: one in six) in native FP64 (7 instructions per amplitude for
# U3, 4 for a phase), the others in integer products whose results take one
# integer-to-double conversion (an FP64-pipe instruction) per real output, 2 per amplitude.
IX_U3 = 0.25 * 7 + 0.75 * 2
IX_PHASE = 4 / 6 + 2 * 5 / 6
IX_DIAG = 0.25 * 4 + 0.75 * 2
FP64_INSTR_PER_AMP_IX = {"h": FP64_INSTR_PER_AMP["h"], "rz": (29 * IX_PHASE / 2 + IX_DIAG) / 30,
                         "u3": IX_U3, "cu3": IX_U3 / 2}
# FP64 pipe peak: 2 FP64 instructions per clock per SM (ncu: the U3 kernel at 0.526e12/s
# keeps the FP64 pipe 83.8 % busy) x 152 SMs x 2.07 GHz max SM clock = 1.26 TFLOP/s.
FP64_PEAK_TINSTR = 2 * 152 * 2.07e9 / 1e12


_DGEMM = {}


def fp64_gemm_tinstr():
    """FP64 FMA instructions per second that cuBLAS DGEMM reaches on this GPU (4096^3, best of
    5, CUDA events): 2 flops per FMA.  Measured once per process, after the timed region."""
    if "v" not in _DGEMM:
        try:
            import torch
            n = 4096
            a = torch.randn(n, n, dtype=torch.float64, device="cuda")
            b = torch.randn(n, n, dtype=torch.float64, device="cuda")
            for _ in range(2):
                torch.matmul(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) * 1e-3)
            _DGEMM["v"] = 2.0 * n ** 3 / best / 2.0 / 1e12
            del a, b
        except Exception:
            _DGEMM["v"] = None
    return _DGEMM["v"]


def fp64_roof(name, n, B, launch_ms, ix=False):
    table = FP64_INSTR_PER_AMP_IX if ix else FP64_INSTR_PER_AMP
    if B != 16 or name not in table:
        return None
    ach = table[name] * (1 << n) / (launch_ms * 1e-3) / 1e12
    gemm = fp64_gemm_tinstr()
    return {"achieved": round(ach, 4), "peak": round(FP64_PEAK_TINSTR, 4), "unit": "T FP64 instr/s",
            "frac": round(ach / FP64_PEAK_TINSTR, 3),
            "peak_source": "2 FP64 instr/clk/SM x 152 SMs x 2.07 GHz (ncu-confirmed pipe rate)",
            "dgemm_measured_peak": round(gemm, 4) if gemm else None,
            "frac_of_dgemm": round(ach / gemm, 3) if gemm else None}


def load_traffic(kernel_gate, n, dtype, form):
    """Per-launch DRAM bytes from the committed ncu summary of the kernel as it is built
    now (form: the complex128 arithmetic, "ix" or "fp64"), if one matches."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        return t.get(f"k_stream[{kernel_gate}]:{n}:{dtype}:{form}")
    except Exception:
        return None


def host_cpu():
    """CPU model and core count of this host (for the oracle rows)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def cpu_baseline(args, n_gates_sample):
    """The CPU oracle, as it stands, timed on the host at full size (same qubit count):
    one thread on the first gates of the first types of the sweep, and every host core
    (OpenMP over the groups of a gate; bitwise the same result) on the first gate of every
    type.  The all-cores row is the reported value."""
    import oracle
    n = args.qubits
    sweeps = sweep_gates(n)
    one = [sweeps[name][0] for name in GATE_TYPES[:n_gates_sample]]
    every = [sweeps[name][0] for name in GATE_TYPES]
    psi = oracle.zero_state(n)
    cores = oracle.default_threads()
    before = oracle.threads()
    try:
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.run(psi, n, one)
        dt1 = time.perf_counter() - t0
        used = oracle.set_threads(cores)
        t0 = time.perf_counter()
        oracle.run(psi, n, every)
        dtn = time.perf_counter() - t0
    finally:
        oracle.set_threads(before)
    return {"value": round(len(every) / dtn, 4), "unit": "gates/s", "cores": used, "kind": "oracle",
            "sample": f"one gate of each of the 8 types of the sweep on a {n}-qubit complex128 state, "
                      f"{used} threads, {dtn:.1f} s",
            **host_cpu(),
            "single_thread": {"value": round(len(one) / dt1, 4), "unit": "gates/s", "cores": 1,
                              "sample": f"{len(one)} gates ({', '.join(g[0] for g in one)}) of the sweep, "
                                        f"{dt1:.1f} s"}}


def run_reference(args, rank, world):
    """The oracle as it stands on every host core, one gate of the sweep per step."""
    import oracle
    n = args.qubits
    sweeps = sweep_gates(n)
    seq = [g for name in GATE_TYPES for g in sweeps[name][:1]]
    psi = oracle.zero_state(n)
    cores = oracle.threads()
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
            "cpu_baseline": {"value": round(v, 4), "unit": "gates/s", "cores": cores, "kind": "oracle",
                             "sample": f"one gate per step, cycling {', '.join(GATE_TYPES)}, {n} qubits, "
                                       f"{cores} threads", **host_cpu()},
            "e2e": {"value": round(v, 4), "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---- other workloads (each prints its own JSON line) ---------------------------------

def _event_ms(stream, fn, reps=1):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def wl_circuit12(args):
    """12-qubit random brickwork (20 layers, complex128) from |0...0>: the planned path (the
    whole 64 KiB state is one tile, 350 gates in one pass) and plain gate-by-gate (one
    streaming launch per gate), each against the oracle's full 4096-amplitude vector."""
    import torch
    import oracle
    from paper_2409_14697_gb300 import inputs, qs
    n = 12
    gates = inputs.brickwork(n, 20, seed=1)
    recs = qs.gate_records(gates)
    want = oracle.run(oracle.zero_state(n), n, gates)
    stream = torch.cuda.Stream()
    h = qs.qs_create(n, qs.QS_C128)
    qs.qs_set_stream(h, stream.cuda_stream)
    rows = {}
    for name, mode in (("planned", qs.QS_MODE_AUTO), ("gate_by_gate", qs.QS_MODE_GATE)):
        opts = qs.options(mode=mode)

        def once():
            qs.qs_reset(h)
            qs.qs_apply_circuit(h, recs, opts)
        for _ in range(max(args.warmup, 3)):
            once()
        reps = max(args.steps, 20)
        ms = _event_ms(stream, once, reps)
        got = qs.qs_amplitudes(h)
        st = qs.qs_last_stats(h)
        rows[name] = {"circuits_per_s": round(1e3 / ms, 1), "gates_per_s": round(len(gates) * 1e3 / ms, 1),
                      "ms_per_circuit": round(ms, 4), "passes": st["passes"], "launches": st["launches"],
                      "max_abs_err_vs_oracle": float(np.max(np.abs(got - want))), "reps": reps}
    qs.qs_destroy(h)
    return {"workload": "12-qubit brickwork, 20 layers, complex128", "metric": "circuits/s",
            "value": rows["planned"]["circuits_per_s"], **rows}


def wl_circuits33(args):
    """33-qubit complex64 circuits (64 GiB state): brickwork 40 layers, QAOA p=4 on a
    3-regular graph, TFIM 50 steps; by default with unfused gates in register phases (the
    fastest path) and with fused 5-qubit blocks on the tensor cores, or with --fuse-k only.
    Checks at full size: norm, and 1 - |<0|C^-1 C|0>|^2 (circuit then inverse)."""
    import torch
    from paper_2409_14697_gb300 import inputs, qs
    n = args.qubits if args.qubits != N_QUBITS else 33
    stream = torch.cuda.Stream()
    h = qs.qs_create(n, qs.QS_C64)
    qs.qs_set_stream(h, stream.cuda_stream)
    fams = {"brickwork40": inputs.brickwork(n, 40, seed=3), "qaoa_p4": inputs.qaoa_3regular(n, p=4, seed=3),
            "tfim50": inputs.tfim(n, steps=50, dt=0.05)}
    fams = {k: v for k, v in fams.items() if k in args.families.split(",")}
    widths = [args.fuse_k] if args.fuse_k > 0 else [1, 5]
    variants = {}
    inverse_widths = getattr(args, "inverse_widths", None)
    for k in widths:
        with_inverse = inverse_widths is None or k in inverse_widths
        tc = "tensor cores" if k >= 4 else ("SIMT" if args.no_rphases else "SIMT, register phases")
        opts = qs.options(fuse_k=k)
        if args.no_rphases:
            opts.flags |= qs.QS_OPT_NO_REG_PHASES
        rows = {}
        for name, gates in fams.items():
            recs = qs.gate_records(gates)
            inv = qs.gate_records(inputs.inverse(gates))
            qs.qs_reset(h)
            qs.qs_apply_circuit(h, recs, opts)      # warm-up (also plans)
            qs.qs_synchronize(h)
            qs.qs_reset(h)
            ms = _event_ms(stream, lambda: qs.qs_apply_circuit(h, recs, opts))
            st = qs.qs_last_stats(h)
            nrm = qs.qs_norm(h)
            rows[name] = {"gates": len(gates), "ms": round(ms, 2), "passes": st["passes"],
                          "ops_after_fuse": st["ops_after_fuse"],
                          "tile_sweeps": st["tile_sweeps"], "tc_blocks": st["tc_blocks"],
                          "gates_per_s": round(len(gates) * 1e3 / ms, 1),
                          "pass_GBps": round(st["bytes"] / (ms * 1e-3) / 1e9, 1),
                          "norm_minus_1": nrm - 1.0}
            if st["tc_blocks"]:
                # tensor-core work over the whole circuit's time (passes, SIMT ops included)
                tpk, tkind = tf32_peak_tflops()
                tf = st["tc_flops"] / (ms * 1e-3) / 1e12
                rows[name]["tc_tflops"] = round(tf, 1)
                rows[name]["tc_frac_of_tf32_peak"] = round(tf / tpk, 4)
                rows[name]["tf32_peak"] = f"{tpk:.0f} TFLOP/s ({tkind} bf16 x 1.1/2.25)"
            if with_inverse:
                qs.qs_apply_circuit(h, inv, opts)
                a0 = qs.qs_amplitudes(h, 0, 1)[0]
                nrm2 = qs.qs_norm(h)
                rows[name]["inverse_infidelity"] = 1.0 - abs(complex(a0)) ** 2
                rows[name]["inverse_infidelity_normalised"] = 1.0 - abs(complex(a0)) ** 2 / nrm2
        variants[f"k{k}"] = {"path": f"fused k={k} ({tc})", "circuits": rows}
    qs.qs_destroy(h)
    out = {"workload": f"{n}-qubit circuits, complex64", "qubits": n, "state_bytes": 8 << n}
    if len(variants) == 1:
        only = next(iter(variants.values()))
        out["workload"] += f", {only['path']}"
        out["circuits"] = only["circuits"]
    else:
        out["variants"] = variants
    return out


def wl_batched(args):
    """4096 independent random U3+CZ brickwork circuits (n ~ U{8..20}, depth ~ U{10..60}),
    complex64, all in ONE graph-captured persistent launch; against one circuit at a time
    through qs_apply_circuit on the same GPU."""
    import torch
    import oracle
    from paper_2409_14697_gb300 import inputs, qs
    from paper_2409_14697_gb300 import autotune
    count = args.count or 4096
    circs = inputs.batched_circuits(count, seed=10)
    # autotune chunk width and fusion width on a 256-circuit sample of the same mix
    tt0 = time.perf_counter()
    best, table = autotune.tune_batch(circs[:256], qs.QS_C64, path=os.path.join(
        os.environ.get("TMPDIR", "/tmp"), "qsim_autotune_bench.json"))
    tune_s = time.perf_counter() - tt0
    t0 = time.perf_counter()
    bo = qs.options(chunk_m=best["chunk_m"], fuse_k=best["fuse_k"])
    if args.no_rphases:
        bo.flags |= qs.QS_OPT_NO_REG_PHASES
    b = qs.qs_batch_create(circs, qs.QS_C64, bo)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    qs.qs_batch_set_stream(b, stream.cuda_stream)
    for _ in range(max(args.warmup, 3)):
        qs.qs_batch_run(b)
    qs.qs_batch_synchronize(b)
    reps = max(args.steps, 3)
    ms = _event_ms(stream, lambda: qs.qs_batch_run(b), reps)
    qs.qs_batch_synchronize(b)
    info = qs.qs_batch_info(b)
    # per-circuit error vs the FP64 oracle on a seeded sample of the smaller circuits
    rs = np.random.default_rng(1)
    small = [i for i, (n, g) in enumerate(circs) if n <= 12]
    sample = sorted(rs.choice(small, size=min(12, len(small)), replace=False).tolist())
    errs, infid = [], []
    for i in sample:
        n, g = circs[i]
        got = qs.qs_batch_amplitudes(b, i, n, qs.QS_C64).astype(np.complex128)
        want = oracle.run(oracle.zero_state(n), n, g)
        errs.append(float(np.max(np.abs(got - want))))
        infid.append(float(1 - abs(np.vdot(want, got)) ** 2 / (np.vdot(got, got).real * np.vdot(want, want).real)))
    qs.qs_batch_destroy(b)
    # one at a time on a subset, scaled to the whole batch by gate count
    sub = circs[: min(256, count)]
    hs = {}
    t_one = 0.0
    for n, g in sub:
        if n not in hs:
            hs[n] = qs.qs_create(n, qs.QS_C64)
            qs.qs_set_stream(hs[n], stream.cuda_stream)
        recs = qs.gate_records(g)
        qs.qs_reset(hs[n])
        qs.qs_apply_circuit(hs[n], recs, qs.options(fuse_k=best["fuse_k"]))
    torch.cuda.synchronize()
    for n, g in sub:
        recs = qs.gate_records(g)

        def one(h=hs[n], r=recs):
            qs.qs_reset(h)
            qs.qs_apply_circuit(h, r, qs.options(fuse_k=best["fuse_k"]))
        t_one += _event_ms(stream, one)
    for h in hs.values():
        qs.qs_destroy(h)
    one_cps = len(sub) / (t_one * 1e-3)
    return {"workload": f"batched: {count} random U3+CZ circuits, n 8-20, depth 10-60, complex64, one graph launch",
            "metric": "circuits/s", "value": round(count / (ms * 1e-3), 1), "ms_per_batch": round(ms, 3),
            "one_at_a_time_circuits_per_s": round(one_cps, 1), "one_at_a_time_sample": len(sub),
            "speedup_vs_one_at_a_time": round(count / (ms * 1e-3) / one_cps, 2),
            "passes": info["passes"], "work_items": info["work_items"], "grid": info["grid"],
            "state_bytes": info["state_bytes"], "host_build_s": round(build_s, 2),
            "autotuned": best, "autotune_s": round(tune_s, 1),
            "autotune_table_ms": {f"m{t['chunk_m']}k{t['fuse_k']}": t["ms"] for t in table},
            "oracle_sample": sample, "max_abs_err": max(errs), "max_infidelity": max(infid)}


def wl_reductions(args):
    """Reductions on a seeded Gaussian state: squared norm, <Z_q> for every q (one FP64
    pass), renormalisation (norm pass + scale pass) and top-1024 |a|^2 (radix select);
    each timed with CUDA events on the state's stream, reported as algorithmic GB/s
    against the measured HBM copy bandwidth."""
    import torch
    from paper_2409_14697_gb300 import inputs, qs
    n = args.qubits
    dt = qs.QS_C128 if args.dtype == "c128" else qs.QS_C64
    B = 16 if dt == qs.QS_C128 else 8
    npdt = np.complex128 if dt == qs.QS_C128 else np.complex64
    stream = torch.cuda.Stream()
    h = qs.qs_create(n, dt)
    qs.qs_set_stream(h, stream.cuda_stream)
    host = torch.empty((1 << n) * 2, dtype=torch.float64 if B == 16 else torch.float32, pin_memory=True)
    hv = host.numpy().view(npdt)
    inputs.gaussian_state(n, seed=7, out=hv)
    qs.qs_set_amplitudes_from(h, 0, 1 << n, host.data_ptr())
    state = B * (1 << n)
    peak, peak_kind = load_peaks()
    out = {"workload": f"reductions, {n} qubits, {args.dtype}", "state_bytes": state, "hbm_peak_GBps": peak,
           "hbm_peak_kind": peak_kind, "ops": {}}
    reps = max(args.steps, 5)
    cases = {"norm": (lambda: qs.qs_norm(h), state),
             "expectation_z_all": (lambda: qs.qs_expectation_z(h), state),
             "renormalize": (lambda: qs.qs_renormalize(h), 3 * state),
             "top_1024": (lambda: qs.qs_top_amplitudes(h, 1024), state)}
    # spot checks against host sums of the same state (FP64), before any renormalisation
    ez, nrm = qs.qs_expectation_z(h)
    p = np.abs(hv.astype(np.complex128)) ** 2
    out["norm_vs_host"] = abs(nrm - float(p.sum()))
    half = 1 << (n - 1)  # the top qubit is 0 on the first half of the indices
    out["expz_top_qubit_vs_host"] = abs(ez[n - 1] - float(p[:half].sum() - p[half:].sum()))
    del p
    for name, (fn, nbytes) in cases.items():
        for _ in range(max(args.warmup, 3)):
            fn()
        ms = _event_ms(stream, fn, reps)
        gbps = nbytes / (ms * 1e-3) / 1e9
        out["ops"][name] = {"ms": round(ms, 4), "alg_bytes": nbytes, "GBps": round(gbps, 1),
                            "frac_of_measured_hbm": round(gbps / peak, 3)}
    out["alg_bytes_note"] = "norm, <Z>, top-K: one read of the state; renormalize: norm read + scale read/write"
    qs.qs_destroy(h)
    return out


# QueenV2 Tables II-IV: seconds on an RTX 4090, complex128 (context, another GPU)
PAPER_S = {"h": {23: 0.011, 24: 0.014, 25: 0.014, 26: 0.021, 27: 0.021, 28: 0.035, 29: 0.041, 30: 0.084},
           "qft": {23: 0.011, 24: 0.014, 25: 0.024, 26: 0.041, 27: 0.064, 28: 0.124, 29: 0.252, 30: 0.519},
           "qaoa_complete_p5": {23: 0.030, 24: 0.054, 25: 0.098, 26: 0.196, 27: 0.371, 28: 0.776, 29: 1.613,
                                30: 3.391}}


def wl_paper(args):
    """The paper's own workloads, complex128, 23..30 qubits (or --qubits only): the Hadamard
    benchmark (Table II; read both as one H gate and as H on every qubit), QFT (Table III)
    and 5-level fully connected QAOA (Table IV), through qs_apply_circuit (QS_MODE_AUTO:
    planner, fusion, merged diagonal runs).  Times beside the paper's RTX-4090 seconds."""
    import torch
    from paper_2409_14697_gb300 import inputs, qs
    sizes = [args.qubits] if args.qubits != N_QUBITS else list(range(23, 31))
    prec = PRECISIONS[args.precision]
    out = {"workload": f"paper tables II-IV, complex128 ({args.precision})", "sizes": {}}
    stream = torch.cuda.Stream()
    for n in sizes:
        h = qs.qs_create(n, qs.QS_C128)
        qs.qs_set_stream(h, stream.cuda_stream)
        fams = {"h_one_gate": [("h", (n - 1,), ())], "h_all_qubits": [("h", (q,), ()) for q in range(n)],
                "qft": inputs.qft(n), "qaoa_complete_p5": inputs.qaoa_complete(n, p=5, seed=n)}
        row = {}
        for name, gates in fams.items():
            recs = qs.gate_records(gates)
            o = qs.options(precision=prec)

            def once():
                qs.qs_reset(h)
                qs.qs_apply_circuit(h, recs, o)
            once()
            reps = max(args.steps, 3)
            ms = _event_ms(stream, once, reps)
            st = qs.qs_last_stats(h)
            nrm = qs.qs_norm(h)
            paper = PAPER_S["h" if name.startswith("h_") else name].get(n)
            row[name] = {"gates": len(gates), "s": round(ms * 1e-3, 5), "passes": st["passes"],
                         "ops": st["ops_after_fuse"], "norm_minus_1": nrm - 1.0,
                         "paper_rtx4090_s": paper,
                         "paper_over_ours": round(paper / (ms * 1e-3), 2) if paper else None}
        qs.qs_destroy(h)
        out["sizes"][n] = row
    out["note"] = ("times include qs_reset (|0..0>) and the host planning of each call; "
                   "paper times are another GPU (RTX 4090, FP64), context only")
    return out


class ServedInputs:
    """Initial states of the served stream's sweep requests: for each (n, dtype) that occurs,
    the first 2^n amplitudes of one seeded 30-qubit Gaussian vector (i.i.d. N(0,1) real and
    imaginary parts), scaled to unit norm in FP64, held in page-locked host memory that the
    requests borrow (QS_REQ_BORROW_INIT: nothing is copied at submission)."""

    def __init__(self, reqs):
        import torch
        from paper_2409_14697_gb300 import inputs
        need = sorted({(r["n"], r["dtype"]) for r in reqs if r["init_seed"]})
        self.buf = {}
        if not need:
            return
        top = max(n for n, _ in need)
        base = inputs.gaussian_state(top, seed=700)   # unit norm over 2^top amplitudes
        for n, dt in need:
            part = base[:1 << n]
            scale = 1.0 / math.sqrt(float(np.vdot(part, part).real))
            npdt = np.complex128 if dt == "c128" else np.complex64
            t = torch.empty(np.dtype(npdt).itemsize << n, dtype=torch.uint8, pin_memory=True)
            v = t.numpy().view(npdt)
            for lo in range(0, 1 << n, 1 << 24):
                v[lo:lo + (1 << 24)] = part[lo:lo + (1 << 24)] * scale
            self.buf[(n, dt)] = t
        del base

    def ptr(self, r):
        return self.buf[(r["n"], r["dtype"])].data_ptr() if r["init_seed"] else 0


SERVED_SMALL_MAX = 18   # requests of at most this many qubits may run in the small-request slots


def served_run(qs, prepared, rate, prec):
    """Submits the prepared requests at their Poisson arrival times (scaled to `rate`) and
    polls until all are done; returns (latencies, wall seconds, server stats)."""
    sv = qs.qs_server_create(150 * 10 ** 9, max_slots=8, small_slots=8, small_max_qubits=SERVED_SMALL_MAX)
    lat = []
    pending = {}
    i = 0
    t0 = time.perf_counter()
    try:
        while i < len(prepared) or pending:
            now = time.perf_counter() - t0
            while i < len(prepared) and prepared[i]["t"] * (2000.0 / rate) <= now:
                q = prepared[i]
                tk = qs.qs_submit(sv, q["n"], q["dt"], q["recs"], top_k=q["k"], init_ptr=q["init"],
                                  precision=prec)
                pending[tk] = (q["n"], q["k"])
                i += 1
            done = []
            for tk, (n, k) in pending.items():
                r = qs.qs_poll(sv, tk, n, k)
                if r is not None:
                    lat.append((n, r["latency_s"]))
                    done.append(tk)
            for tk in done:
                del pending[tk]
            if not done:
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
        st = qs.qs_server_stats(sv)
    finally:
        qs.qs_server_drain(sv)
        qs.qs_server_destroy(sv)
    return np.array(lat), wall, st


def served_sequential(qs, prepared, prec):
    """The plain path: one request after the other through qs_apply_circuit on one state per
    (n, dtype), with the same initial states, <Z_q> and top-K reads."""
    import torch
    hs = {}
    t1 = time.perf_counter()
    for q in prepared:
        key = (q["n"], q["dt"])
        if key not in hs:
            hs[key] = qs.qs_create(q["n"], q["dt"])
        h = hs[key]
        if q["init"]:
            qs.qs_set_amplitudes_from(h, 0, 1 << q["n"], q["init"])
        else:
            qs.qs_reset(h)
        qs.qs_apply_circuit(h, q["recs"], qs.options(precision=prec))
        qs.qs_expectation_z(h)
        qs.qs_top_amplitudes(h, q["k"])
    wall = time.perf_counter() - t1
    for h in hs.values():
        qs.qs_destroy(h)
    torch.cuda.synchronize()
    return wall


def wl_served(args, count=None, loads=None):
    """Poisson stream of circuits with n log-uniform in 10..30, complex64 or complex128,
    each returning <Z_i> for all qubits and the top 1024 amplitudes; admission by an HBM
    budget of 150 GB, 8 slots; sweep requests start from seeded Gaussian states that they
    borrow from page-locked host memory.  The same requests arrive at each offered load of
    the sweep (arrival times scaled); the plain sequential path runs them once."""
    from paper_2409_14697_gb300 import inputs, qs
    count = count or args.count or 300
    if loads is None:
        loads = [float(x) for x in args.loads.split(",") if x] if args.loads else [args.rate]
    reqs = inputs.served_stream(count, rate_hz=2000.0, seed=11)
    si = ServedInputs(reqs)
    prepared = []
    for r in reqs:
        prepared.append({"t": r["t"], "n": r["n"], "dt": qs.QS_C128 if r["dtype"] == "c128" else qs.QS_C64,
                         "recs": qs.gate_records(r["gates"]), "k": min(1024, 1 << r["n"]), "init": si.ptr(r)})
    prec = PRECISIONS[args.precision]
    seq_wall = served_sequential(qs, prepared, prec)
    rows = {}
    for rate in loads:
        nl, wall, st = served_run(qs, prepared, rate, prec)
        lat = nl[:, 1]
        small = nl[nl[:, 0] <= SERVED_SMALL_MAX, 1]
        large = nl[nl[:, 0] > SERVED_SMALL_MAX, 1]
        rows[f"{rate:g}"] = {"requests_per_s": round(count / wall, 2),
                             "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
                             "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
                             "mean_latency_s": round(float(lat.mean()), 4), "wall_s": round(wall, 2),
                             f"small_n_le_{SERVED_SMALL_MAX}": {"count": int(small.size),
                                               "p50_latency_s": round(float(np.percentile(small, 50)), 4) if small.size else None,
                                               "p99_latency_s": round(float(np.percentile(small, 99)), 4) if small.size else None},
                             f"large_n_gt_{SERVED_SMALL_MAX}": {"count": int(large.size),
                                               "p50_latency_s": round(float(np.percentile(large, 50)), 4) if large.size else None,
                                               "p99_latency_s": round(float(np.percentile(large, 99)), 4) if large.size else None},
                             "peak_bytes": st["peak_bytes"], "failed": st["failed"]}
    main = rows[f"{loads[0]:g}"]
    return {"workload": f"served: {count} Poisson requests, n 10-30 log-uniform, c64/c128 "
                        f"({args.precision} for c128), <Z_i> + top-1024, 150 GB budget, 8 slots; "
                        f"sweep requests from borrowed page-locked Gaussian states",
            "lanes": f"8 slots + 8 small-request slots (n <= {SERVED_SMALL_MAX} may overtake larger requests)",
            "metric": "requests/s", "value": main["requests_per_s"], "offered_req_per_s": loads[0],
            "p50_latency_s": main["p50_latency_s"], "p99_latency_s": main["p99_latency_s"],
            "sequential_requests_per_s": round(count / seq_wall, 2), "sequential_wall_s": round(seq_wall, 2),
            "loads": rows}


def workload_summaries(args):
    """Compact, bounded runs of the other configurations for the default bench line: the
    12-qubit circuit, the 33-qubit circuits, the batched launch and the served stream."""
    import copy
    out = {}

    def timed(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # a failing summary must not hide the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["bench_s"] = round(time.perf_counter() - t0, 1)

    def c12():
        r = wl_circuit12(args)
        return {"workload": r["workload"], "circuits_per_s": r["planned"]["circuits_per_s"],
                "gate_by_gate_circuits_per_s": r["gate_by_gate"]["circuits_per_s"],
                "max_abs_err_vs_oracle": max(r["planned"]["max_abs_err_vs_oracle"],
                                             r["gate_by_gate"]["max_abs_err_vs_oracle"]),
                "passes": r["planned"]["passes"]}

    def c33():
        a = copy.copy(args)
        a.qubits, a.fuse_k, a.inverse_widths = 33, 0, (1,)
        r = wl_circuits33(a)
        res = {"workload": r["workload"]}
        for key, v in r["variants"].items():
            res[key] = {"path": v["path"]}
            for fam, row in v["circuits"].items():
                res[key][fam] = {x: row[x] for x in ("ms", "passes", "pass_GBps", "gates", "tc_blocks",
                                                      "tc_tflops", "tc_frac_of_tf32_peak",
                                                      "norm_minus_1", "inverse_infidelity_normalised")
                                 if x in row}
        return res

    def batched():
        a = copy.copy(args)
        a.count = 4096
        r = wl_batched(a)
        return {x: r[x] for x in ("workload", "value", "one_at_a_time_circuits_per_s", "speedup_vs_one_at_a_time",
                                  "max_abs_err", "max_infidelity", "autotuned")}

    def served():
        r = wl_served(args, count=120, loads=[2000.0, 8.0])
        return r

    timed("circuit12", c12)
    timed("circuits33", c33)
    timed("batched", batched)
    timed("served", served)
    return out


def run_workload(args):
    fn = {"circuit12": wl_circuit12, "circuits33": wl_circuits33,
          "batched": wl_batched, "served": wl_served, "reductions": wl_reductions,
          "paper": wl_paper}[args.workload]
    print(json.dumps(fn(args)))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload != "gates30" and args.impl == "ours":
        if rank == 0:
            run_workload(args)
        return
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
        if not args.no_workloads and world == 1 and args.qubits == N_QUBITS:
            out["workloads"] = workload_summaries(args)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
