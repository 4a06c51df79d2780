#!/usr/bin/env python
"""Time-to-solution of the OMM solve on GB300 (and of its oracle on the host cores).

One step = one whole solve of the Si512 DZP-like workload (m = 6656 basis
functions, n = 1024 Wannier functions): omm_create (shift, sliced tensor-core Cholesky
inverse of S + T/tau at preconditioner grade, operand splits) + omm_solve to max|G| < 1e-9
(certified with float64-class products) + the density matrix D. Inputs are
resident in HBM when the timed region starts; H, S, T (354 MB each) are larger
than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload si512_dzp] [--precision mixed|fp64]

The default line also carries two sub-records, each timed with CUDA events on its own
stream and with its own clock record: `batch64` (the 64 uneven instances in one batched
solve, create included) and `si4096_sequence` (the ten warm-started Si4096 Hamiltonians with
dE/dH each step, setup included). Their energies are compared with the exact minima stored
under tests/golden/ (written by tests/golden/make_exact_energies.py from the oracle).

Workloads (--workload): si64_sz, si512_dzp (default), water256_dzp (single solves), batch64
(64 independent instances in one batched solve), si8_kpoints (the 365 Hermitian problems of a
9x9x9 k grid in one batched solve), si4096_sequence (10 warm-started Hamiltonians).

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "OMM time-to-solution & GEMM TFLOP/s, mixed vs FP64 GPU at |ΔE|/|E|≤1e-9"
WORKLOADS = {
    "si64_sz": "si64_sz: Si 64-atom diamond, sp single-zeta, m=256, n=128, tau=5 Ha, eta=HOMO+0.1 Ha, |G|inf<1e-9",
    "si512_dzp": "si512_dzp: Si 512-atom diamond, DZP-like 13 orbitals/atom, m=6656, n=1024, tau=5 Ha, "
       "eta=HOMO+0.1 Ha, |G|inf<1e-9",
    "water256_dzp": "water256_dzp: 256 H2O at 1 g/cm3, DZP-like 23 orbitals/molecule, m=5888, n=1024, tau=5 Ha, "
       "eta=HOMO+0.1 Ha, |G|inf<1e-9",
    "batch64": "batch64: 64 independent Si / water instances (DZ, TZ, DZP, DZP+p / DZ+d, DZP, TZP bases), "
       "m ~ U[512,4096], n/m 0.125-0.25, one batched solve (grouped tensor-core launches in a CUDA graph), "
       "|G|inf<1e-9 each",
    "si8_kpoints": "si8_kpoints: bulk Si 8-atom cell, DZP-like (m=104, n=16 complex per k), 9x9x9 "
       "Monkhorst-Pack grid with k/-k merged (365 Hermitian problems), one batched solve, tau=5 Ha, "
       "|G|inf<1e-9 each",
    "si4096_sequence": "si4096_sz_warmstart: Si 4096-atom single-zeta, m=16384, n=8192, 10 Hamiltonians "
       "H_k = H_0 + k delta (on-site, sigma 0.01 Ha), each solve from the previous C, dE/dH each step",
}
GOLDEN = os.path.join(ROOT, "tests", "golden")
FP64_NOMINAL_TFLOPS = 1.25  # GB300 float64 FMA rate, nominal (context; the roofline uses the probe)


# DRAM bytes per launch of the four mixed line-search GEMMs of the Si512 workload (average of
# dram__bytes_read.sum + dram__bytes_write.sum over the P G, [HD; SD], projection and gradient
# launches of one ncu capture: profiles/traffic_si512_line_search.md). Valid only for the GEMM
# source it was measured on: reported as null once tc_gemm.cu has changed.
GEMM_TRAFFIC_BYTES = 299.1e6
GEMM_TRAFFIC_SOURCE_SHA256 = "a82f4112cd47d88477669b6c07d71553209b5c3cd8544153bf7443c62f1d46a0"


def gemm_traffic():
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1312_1549_gb300", "csrc", "tc_gemm.cu")
    try:
        with open(src, "rb") as fh:
            same = hashlib.sha256(fh.read()).hexdigest() == GEMM_TRAFFIC_SOURCE_SHA256
    except OSError:
        same = False
    return GEMM_TRAFFIC_BYTES if same else None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def golden(name):
    """Exact minima stored by tests/golden/make_exact_energies.py (oracle definition), or None."""
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if gpus > 1 and world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return rank, world, local, dist
    return rank, world, local, None


def max_over_ranks(value, dist, device):
    """The job's time: the largest of the ranks' values (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(count, rank, world):
    """Instances of rank `rank` when `count` independent instances are split over `world` ranks."""
    return list(range(rank, count, world))


def build_problem(workload):
    from synth import configs
    return configs.NAMED[workload]()


def cpu_oracle_solve(p):
    """The oracle (plain float64 numpy OMM) on the host cores, to max|G| < 1e-9: wall seconds."""
    from oracle import omm as oomm
    t0 = time.perf_counter()
    out = oomm.solve(p.H, p.S, p.T, p.eta, p.tau, p.C0, tol_grad=1e-9, want_matrices=False)
    return time.perf_counter() - t0, out


def cpu_oracle_setup(p):
    """A bounded oracle warm-up: preconditioner, initial state and certificate, no line search."""
    from oracle import omm as oomm
    oomm.solve(p.H, p.S, p.T, p.eta, p.tau, p.C0, tol_grad=0.0, max_iter=0, want_matrices=False)


def run_reference(args):
    """--impl reference: the oracle as it stands on the host cores.

    Single-problem workloads: every timed step is one whole oracle solve to max|G| < 1e-9 (a
    measurement, not an extrapolation); each warm-up step is the oracle's setup alone. The batch
    and the Si4096 sequence would take hours per step on the host and have no reference line.
    """
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload in ("batch64", "si4096_sequence"):
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the float64 numpy oracle takes hours per step on {args.workload}; the reference "
                          "lines are si64_sz, si512_dzp, water256_dzp and si8_kpoints"}), flush=True)
        return 0
    cores = os.cpu_count()
    if args.workload == "si8_kpoints":
        from synth.kpoints import silicon_mp_grid
        pk = silicon_mp_grid((9, 9, 9))
        times = [kpoint_oracle_sample(pk)[0] for _ in range(args.steps)]
        value = statistics.mean(times)
        dtype, sample = "c128", "per step: the complex oracle on every 16th k point, scaled to the grid"
    else:
        p = build_problem(args.workload)
        for _ in range(args.warmup):
            cpu_oracle_setup(p)
        times, iters = [], []
        for _ in range(args.steps):
            t, out = cpu_oracle_solve(p)
            times.append(t)
            iters.append(out["iters"])
        value = statistics.mean(times)
        dtype = "f64"
        sample = (f"per step: one whole oracle solve of this workload to max|G|<1e-9 ({iters[-1]} line searches, "
                  "setup and certificate included), timed; warm-up steps run the oracle's setup only")
    out = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOADS[args.workload], "l2": "inputs larger than L2"},
           "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _base_line(args, value_s, world=1):
    return {"metric": METRIC, "value": value_s, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value_s * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "precision": "mixed",
                       "l2": "inputs larger than L2", "parallelism": "1 GPU"}}


def fp64_peak_probe(device, seconds=3.0):
    """Float64 matmul rate of this GPU (torch, 4096^3), off the solver's path: the denominator of
    the float64 path's roofline. Best of 5 (burst) and a back-to-back loop (sustained)."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    c = torch.empty_like(a)
    flop = 2.0 * n ** 3
    torch.matmul(a, b, out=c)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(5):
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    reps = max(1, int(seconds * 1e3 / best))
    e0.record()
    for _ in range(reps):
        torch.matmul(a, b, out=c)
    e1.record()
    e1.synchronize()
    sustained = flop * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
    return {"burst_tflops": flop / (best * 1e-3) / 1e12, "sustained_tflops": sustained,
            "how": f"torch.matmul float64 {n}^3: best of 5 (burst) and {reps} back to back (sustained), CUDA events"}


# ------------------------------------------------------------------ batch of 64 uneven instances
def batch_record(args, probs, device, stream, with_fp64=True, profile_roofline=True):
    """One batched solve of the given instances per step (create + solve), CUDA-event timed.

    Returns the sub-record (time, line searches, grouped-GEMM roofline, error vs the stored exact
    minima) and the last infos."""
    import numpy as np
    import torch
    from paper_1312_1549_gb300 import solver as S
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    dev = [(t(p.H), t(p.S), t(p.T), p.n, p.eta, p.tau) for p in probs]
    C0 = [t(p.C0) for p in probs]
    phases = []

    def step(precision="mixed", subset=None, profile=False):
        idx = range(len(probs)) if subset is None else subset
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        with S.OMMBatch([dev[i] for i in idx], precision=precision, stream=stream, profile=profile,
                        native_certificate=args.native_certificate) as b:
            torch.cuda.synchronize(device)
            t1 = time.perf_counter()
            _, E, infos = b.solve([C0[i] for i in idx])
        phases.append((t1 - t0, time.perf_counter() - t1))
        return E, infos

    steps = args.batch_steps
    for _ in range(max(1, args.batch_warmup)):
        step()
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = S.launch_count()
    with ClockSampler(device.index or 0) as clk:
        e0.record(stream)
        for _ in range(steps):
            E, infos = step()
        e1.record(stream)
        torch.cuda.synchronize(device)
    launches = S.launch_count() - launches0
    ms = e0.elapsed_time(e1) / steps
    logical = sum(i["iterations"] * (6.0 * p.m * p.m * p.n + 16.0 * p.m * p.n * p.n) for i, p in zip(infos, probs))
    timed = phases[-steps:]
    rec = {"workload": WORKLOADS["batch64"], "value": ms * 1e-3, "unit": "s", "steps": steps,
           "warmup": max(1, args.batch_warmup), "instances": len(probs),
           "m_range": [min(p.m for p in probs), max(p.m for p in probs)],
           "status": sorted({i["status"] for i in infos}),
           "gmax_max": max(i["gmax"] for i in infos),
           "line_searches_max": max(i["iterations"] for i in infos),
           "line_searches_total": sum(i["iterations"] for i in infos),
           "gemm_tflops_logical": logical / (ms * 1e-3) / 1e12,
           "s_create_wall": statistics.mean(x[0] for x in timed),
           "s_solve_wall": statistics.mean(x[1] for x in timed),
           "ms_line_search_graphs": infos[0]["ms_iterate"],
           "ms_refresh_wall": infos[0]["ms_batch_refresh"],
           "ms_refresh_sum": sum(i["ms_refine"] - i["ms_certify"] for i in infos),
           "ms_certify_sum": sum(i["ms_certify"] for i in infos),
           "tile_width_autotuned": infos[0]["tile_width"], "gpu_launches": launches, "clocks": clk.summary()}
    gold = golden("batch64_exact.json")
    if gold is not None and len(probs) == 64:
        ref = gold["instances"]
        assert all(r["name"] == p.name for r, p in zip(ref, probs)), "golden batch energies do not match the inputs"
        rec["rel_err_E_vs_exact_max"] = max(abs(E[i] - r["E"]) / abs(r["E"]) for i, r in enumerate(ref))
        rec["exact"] = "E* of all 64 instances (tests/golden/batch64_exact.json, oracle eigenvalues)"
    if profile_roofline:
        # the grouped GEMMs timed with CUDA events in one more solve (launched eagerly, not timed)
        _, prof_infos = step(profile=True)
        b0 = prof_infos[0]
        achieved = (b0["main_gemm_flop"] / (b0["ms_main_gemm"] * 1e-3) / 1e12) if b0["ms_main_gemm"] > 0 else None
        peak = load_peaks()[0]["bf16_tflops_sustained"]
        rec["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": (achieved / peak) if achieved else None, "traffic": None,
                           "kernel": "gemm_pair_kernel / gemm_persistent_kernel (grouped over the batch, tcgen05; "
                                     "split form, single-pass P G; shapes as tile_width_autotuned)",
                           "peak_source": "bf16_tflops_sustained of measured MEASURED_PEAKS",
                           "launches": b0["main_gemm_launches"],
                           "avg_launch_ms": b0["ms_main_gemm"] / max(b0["main_gemm_launches"], 1),
                           "measured_in": "one extra profiled batched solve after the timed steps"}
    if with_fp64:
        # the float64 GPU path instance by instance on every 8th instance, scaled by flops
        sub = list(range(0, len(probs), 8))
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        step("fp64", sub)
        torch.cuda.synchronize(device)
        t_sub = time.perf_counter() - t0
        f = lambda ids: sum(6.0 * probs[i].m ** 2 * probs[i].n + 12.0 * probs[i].m * probs[i].n ** 2 for i in ids)
        est = t_sub * f(range(len(probs))) / f(sub)
        rec["fp64_gpu_loop"] = {"time_to_solution_s_estimate": est, "measured_instances": len(sub),
                                "measured_s": t_sub, "speedup_batched_mixed": est / (ms * 1e-3),
                                "note": "instances solved one by one on the float64 path; measured on every "
                                        "8th instance, scaled by per-line-search flops"}
    return rec, E, infos


# ------------------------------------------------------------------ Si4096 warm-start sequence
def sequence_record(args, p, device, stream):
    """The ten warm-started Hamiltonians H_k = H_0 + k delta in one timed region (setup, solves and
    dE/dH each step); one solve of H_0 beforehand warms the tile autotuner and the modules."""
    import numpy as np
    import torch
    from paper_1312_1549_gb300 import solver as S
    from synth import configs
    delta = configs.warm_start_delta(p, 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    H0, Sm, T, C0 = t(p.H), t(p.S), t(p.T), t(p.C0)
    dvec = t(delta)
    Hk = torch.empty_like(H0)
    dH = torch.empty_like(H0)
    K = args.sequence

    def run(K):
        infos = []
        with S.OMMSolver(H0, Sm, T, p.n, p.eta, p.tau, precision="mixed", stream=stream, profile=True,
                         native_certificate=args.native_certificate) as s:
            C = C0
            for k in range(K):
                if k > 0:
                    with torch.cuda.stream(stream):
                        Hk.copy_(H0)
                        Hk.diagonal().add_(k * dvec)
                    s.update_H(Hk)
                C, E, _, info = s.solve(C)
                s.backward(dEdH=dH, want_S=False)   # dE/dH = D each step
                infos.append((E, info))
        return infos

    run(1)  # warm-up: one solve of H_0
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = S.launch_count()
    with ClockSampler(device.index or 0) as clk:
        e0.record(stream)
        infos = run(K)
        e1.record(stream)
        torch.cuda.synchronize(device)
    launches = S.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    peak = load_peaks()[0]["bf16_tflops_sustained"]
    g_ms = sum(i["ms_main_gemm"] for _, i in infos)
    g_flop = sum(i["main_gemm_flop"] for _, i in infos)
    achieved = g_flop / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None
    rec = {"workload": WORKLOADS["si4096_sequence"], "value": ms * 1e-3, "unit": "s",
           "hamiltonians": K, "steps": 1, "warmup": 1,
           "line_searches": [i["iterations"] for _, i in infos], "E": [E for E, _ in infos],
           "gmax_max": max(i["gmax"] for _, i in infos), "status": [i["status"] for _, i in infos],
           "ms_setup": infos[0][1]["ms_setup"], "ms_precond": infos[0][1]["ms_precond"],
           "ms_iterate": [i["ms_iterate"] for _, i in infos], "ms_refine": [i["ms_refine"] for _, i in infos],
           "ms_outputs": [i["ms_outputs"] for _, i in infos],
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": (achieved / peak) if achieved else None, "traffic": None,
                        "kernel": "line-search GEMMs (tcgen05 on SM pairs or single SMs; split form, single-pass P G)",
                        "peak_source": "bf16_tflops_sustained of measured MEASURED_PEAKS",
                        "launches": sum(i["main_gemm_launches"] for _, i in infos)},
           "gpu_launches": launches, "clocks": clk.summary()}
    gold = golden("si4096_sequence_exact.json")
    if gold is not None:
        ref = {s["k"]: s["E"] for s in gold["steps"]}
        errs = {k: abs(E - ref[k]) / abs(ref[k]) for k, (E, _) in enumerate(infos) if k in ref}
        if errs:
            rec["rel_err_E_vs_exact_max"] = max(errs.values())
            rec["exact_steps"] = sorted(errs)
            rec["exact"] = "E* of H_k for the listed k (tests/golden/si4096_sequence_exact.json, oracle eigenvalues)"
    return rec


def kpoint_oracle_sample(p, stride=16):
    """The complex oracle to convergence on every stride-th k point (host cores), scaled to all."""
    from oracle import hermitian
    idx = list(range(0, len(p.H), stride))
    t0 = time.perf_counter()
    for i in idx:
        hermitian.solve(p.H[i], p.S[i], p.T[i], p.eta, p.tau, p.C0[i], tol_grad=1e-9, want_matrices=False)
    t = time.perf_counter() - t0
    return t * len(p.H) / len(idx), len(idx)


def run_batch(args):
    """--workload batch64: one batched solve of the instances (create + solve) per step."""
    import torch
    from paper_1312_1549_gb300 import build as _build
    _build.build()
    from synth import configs
    # instances are independent: ranks take disjoint shards, no collective on the data path
    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    probs = configs.batch_instances(shard(args.instances, rank, world))
    stream = torch.cuda.Stream(device=device)
    args.batch_steps, args.batch_warmup = args.steps, args.warmup
    rec, _, _ = batch_record(args, probs, device, stream, with_fp64=(not args.no_fp64_compare and world == 1),
                             profile_roofline=True)
    ms = max_over_ranks(rec["value"] * 1e3, dist, device)
    if dist is not None:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0
    out = _base_line(args, ms * 1e-3, world)
    if world > 1:
        out["scaling"] = "strong"
        out["config"]["parallelism"] = f"{args.instances} instances sharded over {world} GPUs (rank 0 shown)"
    out["config"]["certificate"] = "native float64" if args.native_certificate else "float64-class (sliced)"
    for k in ("workload", "value", "unit", "steps", "warmup"):
        rec.pop(k)
    out.update(rec)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_kpoints(args):
    """The k-point workload: every Hermitian problem of the grid in one batched solve per step."""
    import numpy as np
    import torch
    from paper_1312_1549_gb300 import build as _build
    _build.build()
    from paper_1312_1549_gb300 import solver as S
    from synth.kpoints import silicon_mp_grid
    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    p = silicon_mp_grid((9, 9, 9))
    mine = shard(len(p.H), rank, world)
    z = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()
    dev = [(z(p.H[i]), z(p.S[i]), z(p.T[i]), p.n, p.eta, p.tau) for i in mine]
    C0 = [z(p.C0[i]) for i in mine]
    stream = torch.cuda.Stream()
    phases = []

    def step(precision="mixed", subset=None, profile=False):
        idx = range(len(mine)) if subset is None else subset
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with S.OMMHermitianBatch([dev[i] for i in idx], precision=precision, stream=stream, profile=profile) as b:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, E, infos = b.solve([C0[i] for i in idx])
        phases.append((t1 - t0, time.perf_counter() - t1))
        return E, infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = S.launch_count()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            E, infos = step()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = S.launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, torch.device("cuda", local))
    if dist is not None:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0
    out = _base_line(args, ms * 1e-3, world)
    out["dtype"] = "bf16x3+f64 (complex as its real form)"
    if world > 1:
        out["scaling"] = "strong"
        out["config"]["parallelism"] = f"{len(p.H)} k points sharded over {world} GPUs (rank 0 shown)"
    w = np.array(p.meta["weights"])[mine]
    timed = phases[-args.steps:]
    _, prof_infos = step(profile=True)
    b0 = prof_infos[0]
    achieved = (b0["main_gemm_flop"] / (b0["ms_main_gemm"] * 1e-3) / 1e12) if b0["ms_main_gemm"] > 0 else None
    peak = load_peaks()[0]["bf16_tflops_sustained"]
    out.update({"k_points": len(p.H), "k_points_rank0": len(mine), "m": p.m, "n": p.n,
                "band_energy_per_cell": float(np.dot(w, E)) if world == 1 else None,
                "line_searches_max": max(i["iterations"] for i in infos),
                "line_searches_total": sum(i["iterations"] for i in infos),
                "s_create_wall": statistics.mean(t[0] for t in timed),
                "s_solve_wall": statistics.mean(t[1] for t in timed),
                "ms_line_search_graphs": infos[0]["ms_iterate"],
           "ms_refresh_wall": infos[0]["ms_batch_refresh"],
                "gpu_launches": launches, "clocks": clk.summary(),
                "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": (achieved / peak) if achieved else None, "traffic": None,
                             "kernel": "gemm_pair_kernel / gemm_persistent_kernel (grouped over the k points, tcgen05, fused 3-term "
                                       "split; real forms 2m x 2m, 2n)",
                             "peak_source": "bf16_tflops_sustained of measured MEASURED_PEAKS",
                             "launches": b0["main_gemm_launches"],
                             "avg_launch_ms": b0["ms_main_gemm"] / max(b0["main_gemm_launches"], 1),
                             "measured_in": "one extra profiled batched solve after the timed steps",
                             "note": "m = 104 per k: each launch is a few small tiles, latency-bound"}})
    if not args.no_exact_check:
        from oracle import hermitian
        out["rel_err_E_vs_exact_max"] = max(
            abs(E[j] - hermitian.exact_minimum(p.H[i], p.S[i], p.n)["E"]) / abs(E[j]) for j, i in enumerate(mine))
    if not args.no_fp64_compare and world == 1:
        sub = list(range(0, len(mine), 8))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step("fp64", sub)
        torch.cuda.synchronize()
        t_sub = time.perf_counter() - t0
        est = t_sub * len(mine) / len(sub)
        out["fp64_gpu_loop"] = {"time_to_solution_s_estimate": est, "measured_instances": len(sub),
                                "measured_s": t_sub, "speedup_batched_mixed": est / (ms * 1e-3),
                                "note": "k points solved one by one on the float64 path (every 8th, scaled)"}
    if not args.no_cpu_baseline and world == 1:
        t_cpu, n_cpu = kpoint_oracle_sample(p)
        out["cpu_baseline"] = {"value": t_cpu, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"complex oracle to |G|<1e-9 on {n_cpu} of the {len(p.H)} k points "
                                         "(every 16th), scaled to the grid"}
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_sequence(args):
    """--workload si4096_sequence: the warm-start sequence alone."""
    import torch
    from paper_1312_1549_gb300 import build as _build
    _build.build()
    from synth import configs
    device = torch.device("cuda", 0)
    p = configs.si4096_sz()
    rec = sequence_record(args, p, device, torch.cuda.Stream(device=device))
    out = _base_line(args, rec["value"])
    out["steps"], out["warmup"] = 1, 1
    out["config"]["certificate"] = "native float64" if args.native_certificate else "float64-class (sliced)"
    for k in ("workload", "value", "unit", "steps", "warmup"):
        rec.pop(k)
    out.update(rec)
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="si512_dzp", choices=list(WORKLOADS))
    ap.add_argument("--instances", type=int, default=64, help="batch64: instances in the batch")
    ap.add_argument("--sequence", type=int, default=10, help="si4096_sequence: Hamiltonians in the sequence")
    ap.add_argument("--batch-steps", type=int, default=1, help="timed steps of the batch64 sub-record")
    ap.add_argument("--batch-warmup", type=int, default=1, help="warm-up steps of the batch64 sub-record")
    ap.add_argument("--native-certificate", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-exact-check", action="store_true")
    ap.add_argument("--no-cholesky", action="store_true",
                    help="skip the extra solve in the Cholesky flavour (reduction to standard form)")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="skip the batch64 and si4096_sequence sub-records of the default line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "si4096_sequence":
        return run_sequence(args)
    if args.workload == "si8_kpoints":
        return run_kpoints(args)

    import numpy as np
    import torch
    from paper_1312_1549_gb300 import build as _build
    _build.build()
    from paper_1312_1549_gb300 import solver as S

    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = build_problem(args.workload)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    H, Sm, T, C0 = t(p.H), t(p.S), t(p.T), t(p.C0)
    stream = torch.cuda.Stream(device=dev)
    Cbuf = torch.empty_like(C0)
    Dbuf = torch.empty((p.m, p.m), dtype=torch.float64, device=dev)

    def step(precision=args.precision, profile=False):
        with S.OMMSolver(H, Sm, T, p.n, p.eta, p.tau, precision=precision, stream=stream,
                         profile=profile, native_certificate=args.native_certificate) as s:
            _, E, _, info = s.solve(C0, want_D=True, C_out=Cbuf, D_out=Dbuf)
        return E, info

    for _ in range(args.warmup):
        step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    energies = []
    launches0 = S.launch_count()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            E, info = step()
            infos.append(info)
            energies.append(E)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = S.launch_count() - launches0
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist, dev)
    if dist is not None:
        dist.barrier()
    if rank != 0:
        return 0

    # the kernels' own durations (CUDA events around every tensor-core GEMM launch on the solver's
    # stream, and around the sliced products) come from one more solve with profiling on, after the
    # timed steps, so that the timed region carries no event records
    _, prof_info = step(profile=True)
    peaks, peak_kind = load_peaks()
    main_ms = prof_info["ms_main_gemm"]
    main_flop = prof_info["main_gemm_flop"]
    main_launches = prof_info["main_gemm_launches"]
    iters = infos[-1]["iterations"]
    logical = statistics.mean(i["gemm_flop"] for i in infos)
    it_ms = statistics.mean(i["ms_iterate"] for i in infos)
    mixed = args.precision == "mixed"
    achieved = main_flop / (main_ms * 1e-3) / 1e12 if main_ms > 0 else None
    peak = peaks["bf16_tflops_sustained"] if mixed else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if (achieved and peak) else None,
                "traffic": gemm_traffic() if mixed else None,
                "traffic_source": ("bytes per launch, mean over the four line-search GEMMs of one ncu capture "
                                   "(dram__bytes_read.sum + dram__bytes_write.sum; algorithmic 277.5 MB); "
                                   "null once the GEMM source differs from the one measured") if mixed else None,
                "kernel": ("gemm_pair_kernel / gemm_persistent_kernel (tcgen05 on SM pairs or single SMs, "
                           "fused 3-term split; shapes as tile_width_autotuned)" if mixed
                           else "dgemm_kernel (DFMA)"),
                "peak_source": f"bf16_tflops_sustained of {peak_kind} MEASURED_PEAKS" if mixed else
                "float64 DFMA (see fp64_peak)",
                "launches": main_launches, "avg_launch_ms": main_ms / max(main_launches, 1),
                "measured_in": "one extra profiled solve after the timed steps (CUDA events on the solver's stream)"}
    if mixed and peak:
        # each line-search GEMM on its own: issued flops / summed launch time, against the same peak
        names = ["P G (single bf16 pass)", "[H D; S D] (split, block-sparse)", "projections (split)",
                 "gradient (split, MN-major B)"]
        roofline["per_gemm"] = []
        for k, name in enumerate(names):
            t, f = prof_info["ms_gemm_plan"][k], prof_info["flop_gemm_plan"][k]
            if t > 0:
                a = f / (t * 1e-3) / 1e12
                roofline["per_gemm"].append({"gemm": name, "shape": prof_info["tile_width"][k],
                                             "ms_per_solve": t, "achieved": a, "frac": a / peak})
    sl_ms = prof_info["ms_sliced_gemm"]
    sl_flop = prof_info["sliced_gemm_flop"]
    sl_n = prof_info["sliced_gemm_launches"]
    roofline_sliced = None
    if mixed and sl_ms > 0:
        a = sl_flop / (sl_ms * 1e-3) / 1e12
        roofline_sliced = {"bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                           "traffic": None, "kernel": "gemm_persistent_one_kernel (tcgen05, sliced products: "
                           "preconditioner inverse (3-term bf16 split), refreshes and certificate (10 slices), D (8))", "launches": sl_n,
                           "avg_launch_ms": sl_ms / max(sl_n, 1), "ms_per_solve": sl_ms}
    out = {"metric": METRIC, "value": ms * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16x3+f64" if mixed else "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "precision": args.precision,
                      "certificate": ("native float64" if args.native_certificate or not mixed
                                      else "float64-class (sliced)"),
                      "l2": "inputs larger than L2 (H, S, T are m*m*8 bytes each)",
                      "parallelism": "replicas only" if world > 1 else "1 GPU"},
           "line_searches": iters, "refinements": infos[-1]["refinements"],
           "E": energies[-1], "gmax": infos[-1]["gmax"],
           "ms_setup": statistics.mean(i["ms_setup"] for i in infos),
           "ms_precond": statistics.mean(i["ms_precond"] for i in infos),
           "tile_width_autotuned": infos[-1]["tile_width"],
           "ms_iterate": it_ms, "ms_per_line_search": it_ms / max(iters, 1),
           "ms_refine": statistics.mean(i["ms_refine"] for i in infos),
           "ms_certify": statistics.mean(i["ms_certify"] for i in infos),
           "ms_outputs": statistics.mean(i["ms_outputs"] for i in infos),
           "gemm_tflops_logical": logical / (ms * 1e-3) / 1e12,
           "gemm_tflops_logical_in_iterations": (infos[-1]["gemm_flop"] and
                                                 (iters * (6.0 * p.m * p.m * p.n + 12.0 * p.m * p.n * p.n))
                                                 / (it_ms * 1e-3) / 1e12),
           "roofline": roofline, "roofline_sliced": roofline_sliced, "gpu_launches": launches, "clocks": clocks}
    gold = golden("named_exact.json")
    ref = gold["workloads"].get(args.workload) if gold else None
    if not args.no_exact_check and ref is not None and ref["m"] == p.m and ref["n"] == p.n:
        out["rel_err_E_vs_exact"] = abs(energies[-1] - ref["E"]) / abs(ref["E"])
    if not args.no_e2e:
        Hh, Sh, Th, C0h = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (p.H, p.S, p.T, p.C0))
        Ch = torch.empty_like(C0h).pin_memory()
        Dh = torch.empty((p.m, p.m), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with S.OMMSolver(Hh, Sh, Th, p.n, p.eta, p.tau, precision=args.precision, stream=stream,
                         native_certificate=args.native_certificate) as s:
            _, Ee, _, _ = s.solve(C0h, want_D=True, C_out=Ch, D_out=Dh)
        te = time.perf_counter() - t0
        out["e2e"] = {"value": te, "unit": "s", "h2d_bytes_per_step": (3 * p.m * p.m + p.n * p.m) * 8,
                      "d2h_bytes_per_step": (p.n * p.m + p.m * p.m + 1) * 8,
                      "api": "omm_create + omm_solve with pinned host H, S, T, C0 and host C, D, E"}
        del Hh, Sh, Th, C0h, Ch, Dh
    subrecords = world == 1 and not args.no_subrecords and args.workload == "si512_dzp" and mixed
    gen = None
    if subrecords:
        # the sub-records' inputs are built by host worker processes (spawn) while the GPU runs the
        # comparisons below
        from concurrent.futures import ProcessPoolExecutor
        import multiprocessing as mp
        from synth import configs
        workers = max(1, min(8, (os.cpu_count() or 2) // 2))
        saved_env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "2"
        gen = ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
        seq_dir = tempfile.mkdtemp(prefix="omm_bench_")
        fut_seq = gen.submit(_build_sequence_inputs, seq_dir)
        fut_batch = [gen.submit(configs.batch_instance, i) for i in range(args.instances)]
        for k, v in saved_env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    if not args.no_fp64_compare and mixed:
        E64, i64 = step(precision="fp64", profile=True)
        probe = fp64_peak_probe(dev)
        out["fp64_peak"] = probe
        out["fp64_gpu"] = {"time_to_solution_s": (i64["ms_setup"] + i64["ms_iterate"] + i64["ms_refine"] +
                                                  i64["ms_outputs"]) * 1e-3,
                           "line_searches": i64["iterations"],
                           "dgemm_tflops": (i64["main_gemm_flop"] / (i64["ms_main_gemm"] * 1e-3) / 1e12
                                            if i64["ms_main_gemm"] > 0 else None),
                           "E": E64, "speedup_mixed_over_fp64": None}
        out["fp64_gpu"]["speedup_mixed_over_fp64"] = out["fp64_gpu"]["time_to_solution_s"] / (ms * 1e-3)
        dg = out["fp64_gpu"]["dgemm_tflops"]
        if dg:  # the float64 path is bound by the float64 FMA units (no tensor-core float64 here)
            pk = probe["sustained_tflops"]
            out["fp64_gpu"]["roofline"] = {"bound": "alu", "achieved": dg, "peak": pk, "unit": "TFLOP/s",
                                           "frac": dg / pk, "kernel": "dgemm_kernel (DFMA)",
                                           "peak_source": "measured: torch float64 matmul, sustained (fp64_peak)",
                                           "nominal_tflops": FP64_NOMINAL_TFLOPS}
    if not args.no_cholesky and args.workload != "si64_sz":
        # the paper's other flavour (Sec. 2.4): S = L L^T, H_r = L^-1 H L^-T, no preconditioner;
        # one warm-up solve (tile autotuning), then one timed create + solve
        def step_chol():
            with S.OMMSolver(H, Sm, None, p.n, p.eta, p.tau, precision=args.precision, stream=stream,
                             cholesky=True) as s:
                _, E, _, info = s.solve(C0, want_D=True, C_out=Cbuf, D_out=Dbuf)
            return E, info
        step_chol()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        Ec, ic = step_chol()
        c1.record(stream)
        torch.cuda.synchronize()
        out["cholesky"] = {"time_to_solution_s": c0.elapsed_time(c1) * 1e-3, "line_searches": ic["iterations"],
                           "ms_setup": ic["ms_setup"], "ms_reduce": ic["ms_precond"],
                           "ms_transform": ic["ms_transform"], "ms_iterate": ic["ms_iterate"],
                           "ms_refine": ic["ms_refine"], "ms_outputs": ic["ms_outputs"], "E": Ec,
                           "gmax_reduced": ic["gmax"],
                           "note": "reduction to standard form instead of the kinetic preconditioner; "
                                   "its line searches are those of P = S^-1"}
        if ref is not None and not args.no_exact_check:
            out["cholesky"]["rel_err_E_vs_exact"] = abs(Ec - ref["E"]) / abs(ref["E"])
    if subrecords:
        del H, Sm, T, C0, Cbuf, Dbuf
        torch.cuda.empty_cache()
        probs = [f.result() for f in fut_batch]
        rec, _, _ = batch_record(args, probs, dev, stream, with_fp64=not args.no_fp64_compare)
        del probs
        out["batch64"] = rec
        pseq = _load_sequence_inputs(fut_seq.result())
        gen.shutdown()
        torch.cuda.empty_cache()
        out["si4096_sequence"] = sequence_record(args, pseq, dev, stream)
        del pseq
        import shutil
        shutil.rmtree(seq_dir, ignore_errors=True)
    if not args.no_cpu_baseline and world == 1:
        t_cpu, ref_out = cpu_oracle_solve(p)
        out["cpu_baseline"] = {"value": t_cpu, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"one whole oracle solve of this workload to max|G|<1e-9 "
                                         f"({ref_out['iters']} line searches, setup and certificate included), "
                                         "timed on the host cores"}
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _build_sequence_inputs(folder):
    """Si4096 SZ inputs built in a worker process; its 2 GB matrices travel through files."""
    import numpy as np
    from synth import configs
    p = configs.si4096_sz()
    for name in ("H", "S", "T", "C0"):
        np.save(os.path.join(folder, name + ".npy"), getattr(p, name))
        setattr(p, name, None)
    return p, folder


def _load_sequence_inputs(result):
    import numpy as np
    p, folder = result
    for name in ("H", "S", "T", "C0"):
        setattr(p, name, np.load(os.path.join(folder, name + ".npy")))
    return p


if __name__ == "__main__":
    sys.exit(main())
