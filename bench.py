"""Benchmark: mu-solved density matrices per second on one GB300 (or N replicas).

One step = the whole hot path for one synthetic Hamiltonian: block filter and
symbolic analysis, then the mu bisection, each bisection step a full build
(gather, Gershgorin bound, Newton-Schulz sign iteration, scatter, trace and
energy).  The default workload is 1024 water-like molecules with 6x6 blocks
(N = 6144), filter 1e-5, bisection to trace(D) = 3072.

Prints one JSON line (rank 0).  Besides the headline it reports the FP64 plain
form, the learned bound's effect on an MD-like trajectory, and two FP64 forms
beside the hot path on 1024-molecule inputs: S^-1/2 of an overlap-like matrix
(``inv_sqrt_fp64``) and the mu-solved non-orthogonal density matrix of an
(H, S) pair (``nonorth_fp64``), each with a sampled check against the oracle
(``--no-functions`` skips them).  ``--impl reference`` times the FP64 CPU oracle
on the same workload instead (bounded column samples, extrapolated).
"""

from __future__ import annotations

import argparse
import contextlib
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_TEXT = {
    "water1024": "1024 water-like molecules on a jittered cubic lattice, 6x6 blocks (N=6144), cutoff 6 A, "
                 "decay 1.5 A, block filter 1e-5, bisection to trace(D)=3072 (tol 1e-2)",
    "water32": "32 water-like molecules, 6x6 blocks (N=192), cutoff 5 A, bisection to trace(D)=96",
    "water4096x23": "4096 molecules, 23x23 blocks (N=94208), cutoff 7 A, decay 2 A, filter 1e-6, mu = 0 fixed",
    "slab6000": "6000-molecule water/vacuum slab (50x50x200 A box, density ramp over two interfaces), 6x6 blocks, "
                "cutoff 15.3 A, decay 3 A, filter 1e-5, 20-step bisection to trace(D)=18000 (tol 1e-2)",
}
L2_FLUSH_BYTES = 256 << 20
FP64_PEAK_TFLOPS = 1.2  # DFMA throughput measured on this machine's GB300 (register-resident FMA loop)
METRIC = "density matrices/s (mu-solved), mixed precision vs FP64 plain at <=1e-5 error on D"


@contextlib.contextmanager
def no_gc():
    """Timed loops run with Python's cyclic garbage collector paused (as timeit does), so that a
    collection pause of the interpreter does not land inside a sub-millisecond step."""
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _profiled_traffic(workload: str, precision: str, gemms_per_launch: float):
    """DRAM bytes per launch of the Newton-Schulz kernel from the committed ncu record, or None
    when that record was taken on a different kernel source or workload.  A record captured on a
    column shard (a small case) is scaled to the launch by its number of GEMMs (two per step),
    which the traffic of the streamed form follows."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "ns_tc_traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["kernel_source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except Exception:
        return None, "no ncu record"
    if precision != "fp16x3":
        return None, "no ncu record for this precision"
    for r in rec["records"]:
        if r["workload"] == workload:
            if sha != r["sha256_16"]:  # each record names the kernel source it was captured on
                return None, "kernel changed since the ncu capture"
            t = r["dram_bytes_read"] + r["dram_bytes_write"]
            if "gemms" in r:
                return t * gemms_per_launch / r["gemms"], ("ncu dram__bytes_read+write of a 152-column launch, "
                                                           "scaled by the launch's GEMM count")
            return t, "ncu dram__bytes_read+write of one launch"
    return None, "no ncu record for this workload"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _oracle_sample(sysm, eps, mu, n_cols, workers, seed=0):
    """Oracle on a seeded sample of block columns; returns (seconds, columns, result)."""
    import oracle as O

    cp, ri, v, _ = O.filter_blocks(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, eps)
    rng = np.random.default_rng(seed)
    cols = sorted(rng.choice(sysm.n_blocks, size=min(n_cols, sysm.n_blocks), replace=False).tolist())
    t0 = time.perf_counter()
    res = O.density_submatrix(sysm.block_size, cp, ri, v, mu, workers=workers, columns=cols)
    dt = time.perf_counter() - t0
    return dt, cols, res, (cp, ri)


def learned_scaling(args, stream):
    """MD-like trajectory: train the bound model on the first snapshots, compare on the rest.

    The 1024-molecule system takes cumulative N(0, 0.05 A) position steps; one
    context holds the trajectory (the pair pattern of the first snapshot, the
    block filter prunes per snapshot).  Training snapshots: solve mu, then
    collect features and Lanczos labels at that mu.  Evaluation snapshots are
    timed (values already on the device) with the model off and on.
    """
    import torch

    import oracle as O
    from paper_2205_14741_gb300 import SubmatrixDensity
    from synth import WORKLOADS, md_trajectory

    w = WORKLOADS["md1024"]
    n_snap = args.learned_snapshots
    n_train = n_snap // 2
    t0 = time.perf_counter()
    snaps = list(md_trajectory(w["n_mol"], w["b"], w["r_c"], w["ell"], w["seed"], n_snap, fixed_pattern=True))
    t_gen = time.perf_counter() - t0
    ctx = SubmatrixDensity.from_system(snaps[0], stream=stream.cuda_stream)
    ctx.set_filter_threshold(w["eps"])
    ctx.set_precision(args.precision)
    ctx.set_electron_count(w["n_e"], max_steps=30, tol=1e-2)
    ctx.bound_model_init(w["seed"])
    t0 = time.perf_counter()
    for sysm in snaps[:n_train]:
        ctx.set_values(sysm.values)
        ctx.solve_mu()
        ctx.set_mu(ctx.get_trace()[2])
        ctx.bound_model_collect(48)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = ctx.bound_model_train(epochs=args.learned_epochs, batch=256, lr=2e-3)
    t_train = time.perf_counter() - t0
    vals = [torch.from_numpy(sysm.values).to("cuda") for sysm in snaps[n_train:]]

    def evaluate(model_on):
        ctx.set_bound_model(model_on)
        ctx.set_values(snaps[n_train - 1].values)
        ctx.solve_mu()
        torch.cuda.synchronize()
        ms, its, fb, ns_ms, builds = 0.0, [], 0, 0.0, 0
        for v in vals:
            ctx.reset_counters()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.set_values(v, on_device=True)
            ctx.solve_mu()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            st = ctx.get_stats()
            its.append(ctx.get_submatrix_info()[1].copy())
            fb += st["n_bound_fallback"]
            ns_ms += st["ns_ms_total"]
            builds += st["bisection_steps"]
        its = np.concatenate(its)
        return {"dm_per_s": len(vals) / (ms / 1e3), "ms_per_step": ms / len(vals), "ns_ms_per_step": ns_ms / len(vals),
                "iters_mean": float(its.mean()), "iters_max": int(its.max()),
                "fallback_rate": fb / its.shape[0], "builds_per_step": builds / len(vals)}, ctx.get_density()

    off, d_off = evaluate(False)
    on, d_on = evaluate(True)
    mu = ctx.get_trace()[2]
    last = snaps[-1]
    _, cols, res, _ = _oracle_sample(last, w["eps"], mu, 32, os.cpu_count() or 1)
    offs = O.block_value_offsets(last.block_size, last.col_ptr, last.row_idx)
    cp_f, ri_f, _, keep = O.filter_blocks(last.block_size, last.col_ptr, last.row_idx, last.values, w["eps"])
    off_f = O.block_value_offsets(last.block_size, cp_f, ri_f)
    kf = np.cumsum(keep) - 1
    err = 0.0
    for j in cols:  # compare the kept blocks of each sampled column (dropped blocks are zero on both sides)
        for k in range(last.col_ptr[j], last.col_ptr[j + 1]):
            a = d_on[offs[k]:offs[k + 1]]
            b = res.values[off_f[kf[k]]:off_f[kf[k] + 1]] if keep[k] else np.zeros_like(a)
            err = max(err, float(np.max(np.abs(a - b))))
    ctx.close()
    return {
        "workload": f"{w['n_mol']}-molecule trajectory, {n_snap} snapshots, cumulative N(0, 0.05 A) steps; "
                    f"model trained on the first {n_train} (features and 48-step Lanczos labels at the solved mu), "
                    f"evaluated on the last {n_snap - n_train}",
        "train_loss": loss, "train_samples": n_train * w["n_mol"], "epochs": args.learned_epochs,
        "seconds": {"generate": t_gen, "collect": t_collect, "train": t_train},
        "without_model": off, "with_model": on,
        "iters_saved_frac": 1.0 - on["iters_mean"] / off["iters_mean"],
        "speedup_with_model": on["dm_per_s"] / off["dm_per_s"],
        "d_max_abs_err_vs_oracle_last_snapshot": err, "oracle_columns": len(cols),
        "max_abs_diff_with_vs_without": float(np.max(np.abs(d_on - d_off))),
    }


def function_leg(args, stream, flush, check):
    """S^-1/2 of a 1024-molecule overlap-like matrix (6x6 blocks, cutoff 6 A) in FP64 through the
    same filter / gather / Newton-Schulz / scatter path (the coupled form of Eq. 12).  Timed per
    build with CUDA events, L2 flushed between builds; rate against the FP64 pipe; sampled columns
    against the oracle's eigendecomposition when ``check``."""
    import torch

    from paper_2205_14741_gb300 import SubmatrixDensity
    from synth import make_overlap_system

    s = make_overlap_system(1024, 6, 6.0, 1.5, 41)
    c = SubmatrixDensity.from_system(s, stream=stream.cuda_stream)
    try:
        c.set_precision("fp64")
        c.set_function("inv_sqrt")
        c.set_mu(0.0)
        for _ in range(args.warmup):
            c.build_density()
        torch.cuda.synchronize()
        c.reset_counters()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.function_steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            c.build_density()
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        st = c.get_stats()
        got = c.get_density()
        dims, iters, _ = c.get_submatrix_info()
    finally:
        c.close()
    tflops = 6.0 * st["ns_work_n3"] / (ms / 1e3) / 1e12  # work counter: sum over the timed builds
    out = {"value": args.function_steps / (ms / 1e3), "unit": "S^-1/2 per s", "ms_per_build": ms / args.function_steps,
           "workload": "1024 water-like molecules, overlap-like SPD matrix, 6x6 blocks (N=6144), cutoff 6 A, "
                       "decay 1.5 A, no filtering, mu = 0",
           "iters_mean": st["iters_mean"], "dims_mean": float(np.mean(dims)),
           "tflops": tflops, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
           "frac_of_fp64_peak": tflops / FP64_PEAK_TFLOPS,
           "note": "flops = sum over the timed builds of sum_j 6 n_j^3 iters_j (coupled iteration: three "
                   "products of n_j x n_j) over their summed event time; "
                   "FP64 peak = DFMA rate measured on this GB300 by a register-resident FMA loop"}
    if check:
        import oracle as O

        rng = np.random.default_rng(0)
        cols = sorted(set(np.argsort(dims)[-2:].tolist()) | set(rng.choice(s.n_blocks, 6, replace=False).tolist()))
        res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, "inv_sqrt", columns=cols)
        off = O.block_value_offsets(s.block_size, s.col_ptr, s.row_idx)
        err = max(float(np.max(np.abs(got[off[s.col_ptr[j]]:off[s.col_ptr[j + 1]]]
                                      - res.values[off[s.col_ptr[j]]:off[s.col_ptr[j + 1]]]))) for j in cols)
        out["max_abs_err_vs_oracle"] = err
        out["checked_columns"] = len(cols)
    return out


def nonorth_leg(args, stream, flush, check):
    """Eq. 14 with an overlap S != I (FP64): a 1024-molecule Kohn-Sham-like H and overlap-like S
    of one geometry (6x6 blocks, cutoff 6 A, filter 1e-5), mu bisected on tr(P S) = 3072.  A
    step = new values of H and S, setup (L_j = A_S^-1/2, M_j = L_j A_H L_j) and the bisection;
    a fixed-mu build on a ready setup is timed separately.  Sampled columns against the
    oracle at the solved mu when ``check``."""
    import torch

    from paper_2205_14741_gb300 import SubmatrixDensity
    from synth import make_nonorth_pair

    h, s = make_nonorth_pair(1024, 6, 6.0, 1.5, 16)
    eps, n_e = 1e-5, 3072.0
    h_dev = torch.from_numpy(h.values).to("cuda")
    s_dev = torch.from_numpy(s.values).to("cuda")
    c = SubmatrixDensity.from_system(h, stream=stream.cuda_stream)
    try:
        c.set_precision("fp64")
        c.set_filter_threshold(eps)
        c.set_electron_count(n_e, max_steps=40, tol=1e-2)

        def step():
            c.set_values(h_dev, on_device=True)
            c.set_overlap(s_dev, on_device=True)
            c.solve_mu()

        for _ in range(max(1, args.warmup // 2)):
            step()
        torch.cuda.synchronize()
        c.reset_counters()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.function_steps)]
        builds = []
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
            builds.append(c.get_stats()["bisection_steps"])
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        tr, en, mu = c.get_trace()
        p = c.get_density()
        dims, iters, _ = c.get_submatrix_info()
        # one build at the solved mu on the ready setup: the per-bisection-step cost
        c.set_mu(mu)
        c.build_density()
        torch.cuda.synchronize()
        c.reset_counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        c.build_density()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_build = e0.elapsed_time(e1)
        st_b = c.get_stats()
    finally:
        c.close()
    n_builds = float(np.mean(builds))
    out = {"value": args.function_steps / (ms / 1e3), "unit": "mu-solved non-orthogonal density matrices/s",
           "ms_per_step": ms / args.function_steps, "bisection_builds_per_step": n_builds,
           "ms_per_build_on_ready_setup": ms_build,
           "ms_setup_per_step_estimate": ms / args.function_steps - n_builds * ms_build,
           "build_tflops": 4.0 * st_b["ns_work_n3"] / (ms_build / 1e3) / 1e12,
           "fp64_peak_tflops": FP64_PEAK_TFLOPS,
           "workload": "1024 water-like molecules, H and S of one geometry, 6x6 blocks (N=6144), cutoff 6 A, "
                       "decay 1.5 A, block filter 1e-5 on H, bisection to tr(PS)=3072 (tol 1e-2)",
           "trace_ps": tr, "mu": mu, "iters_mean": float(np.mean(iters)), "dims_mean": float(np.mean(dims)),
           "note": "step = set_values(H) + set_overlap(S) + solve_mu, L2 flushed between steps; the setup "
                   "(A_S^-1/2 by the coupled iteration and M_j = L_j A_H L_j) runs once per step; build "
                   "flops = sum_j 4 n_j^3 iters_j over the build's event time"}
    if check:
        import oracle as O

        cp, ri, hv, keep = O.filter_blocks(h.block_size, h.col_ptr, h.row_idx, h.values, eps)
        sv = O.take_blocks(h.block_size, h.col_ptr, h.row_idx, s.values, keep)
        rng = np.random.default_rng(0)
        cols = sorted(set(np.argsort(dims)[-2:].tolist()) | set(rng.choice(h.n_blocks, 6, replace=False).tolist()))
        res = O.density_nonorth_submatrix(h.block_size, cp, ri, hv, sv, mu, columns=cols)
        if keep.all():  # the filter drops nothing here: the input and filtered layouts coincide
            off = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)
            out["max_abs_err_vs_oracle"] = max(
                float(np.max(np.abs(p[off[h.col_ptr[j]]:off[h.col_ptr[j + 1]]]
                                    - res.values[off[h.col_ptr[j]]:off[h.col_ptr[j + 1]]]))) for j in cols)
            out["checked_columns"] = len(cols)
    return out


def _dims_of(block_size, cp, ri):
    """n_j of every block column of a (filtered) block-CSC pattern (no method arithmetic)."""
    bs = np.asarray(block_size, dtype=np.int64)
    sizes = bs[np.asarray(ri, dtype=np.int64)]
    csum = np.concatenate([[0], np.cumsum(sizes)])
    return (csum[np.asarray(cp[1:])] - csum[np.asarray(cp[:-1])]).astype(np.int64)


def _work_scale(block_size, cp, ri, cols):
    """Factor from a column sample to the whole build: sum_j n_j^3 over all columns / over the sample."""
    d3 = _dims_of(block_size, cp, ri).astype(np.float64) ** 3
    return float(d3.sum() / d3[np.asarray(cols)].sum())


def _fixed_mu(w):
    return w.get("mu") is not None


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O
    from synth import WORKLOADS, make_workload

    w = WORKLOADS[args.workload]
    sysm = make_workload(args.workload)
    workers = os.cpu_count() or 1
    cp, ri, v, _ = O.filter_blocks(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, w["eps"])
    if _fixed_mu(w):
        mu, builds_per_step = float(w["mu"]), 1
    else:
        # one mu-solved density matrix = the builds of the bisection; water1024 settles on the
        # first midpoint of the bracket (one build), the slab's bisection takes all its steps
        lo, hi = O.global_gershgorin(sysm.block_size, cp, ri, v)
        mu = 0.5 * (lo + hi)
        builds_per_step = int(w.get("max_steps", 1))
    for _ in range(args.warmup):
        _oracle_sample(sysm, w["eps"], mu, 16, workers)
    times = []
    for k in range(args.steps):
        dt, cols, _, _ = _oracle_sample(sysm, w["eps"], mu, args.ref_columns, workers, seed=k)
        times.append(dt * _work_scale(sysm.block_size, cp, ri, cols) * builds_per_step)
    per = sum(times) / len(times)
    value = 1.0 / per
    out = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "density matrices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT.get(args.workload, args.workload)},
        "cpu_baseline": {"value": value, "unit": "density matrices/s", "cores": workers, "kind": "oracle",
                         "sample": f"{args.ref_columns} of {sysm.n_blocks} block columns per step (seeded), "
                                   f"time scaled by sum_j n_j^3 (all) / sum_j n_j^3 (sample)"
                                   + (f" x{builds_per_step} bisection builds" if builds_per_step > 1 else "")},
        "e2e": {"value": value, "unit": "density matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def train_heldout_model(args, w, stream):
    """Trains the learned bound on systems of the same generator with other seeds (held out: none
    of them is timed) and saves the parameters; returns (path, description)."""
    import tempfile

    from paper_2205_14741_gb300 import SubmatrixDensity
    from synth import make_workload

    path = os.path.join(tempfile.mkdtemp(prefix="smx_bound_"), "model.bin")
    seeds = [w["seed"] + 1000 * (k + 1) for k in range(args.model_systems)]
    t0 = time.perf_counter()
    samples = 0
    ctx = None
    for k, seed in enumerate(seeds):
        sysm = make_workload(args.workload, seed=seed)
        ctx = SubmatrixDensity.from_system(sysm, stream=stream.cuda_stream)
        ctx.set_filter_threshold(w["eps"])
        ctx.set_precision(args.precision)
        if k == 0:
            ctx.bound_model_init(w["seed"])
        else:
            ctx.bound_model_init(w["seed"])
            ctx.set_bound_model(False, path)  # continue from the parameters trained so far
        # two rounds per system: the second sees the previous-step feature of the first
        for _ in range(2):
            ctx.set_values(sysm.values)
            if _fixed_mu(w) or args.per_build:
                # fixed mu; for the per-build runs of the heavy bisection workloads the mid-gap
                # mu = 0 of these generators stands in for a full solve
                ctx.set_mu(float(w["mu"]) if _fixed_mu(w) else 0.0)
                ctx.build_density()
            else:
                ctx.set_electron_count(w["n_e"], max_steps=30, tol=1e-2)
                ctx.solve_mu()
                ctx.set_mu(ctx.get_trace()[2])
            ctx.bound_model_collect(48)
            samples += sysm.n_blocks
        loss = ctx.bound_model_train(epochs=args.model_epochs, batch=256, lr=2e-3)
        ctx.bound_model_save(path)
        ctx.close()
    return path, {"trained_on": f"{args.workload} generator, seeds {seeds} (held out: not timed)",
                  "samples": samples, "epochs_per_system": args.model_epochs, "train_loss": loss,
                  "seconds": time.perf_counter() - t0}


def shard_leg(args, w, sysm, stream, pg, world, rank):
    """One system split over the ranks by block-column ranges (balanced by sum n_j^3); each
    bisection step sums the 16-byte (trace, energy) over the ranks (NCCL all-reduce).  Returns
    (ms per mu-solved density matrix, max over ranks; final mu, trace)."""
    import torch

    from paper_2205_14741_gb300 import SubmatrixDensity
    from paper_2205_14741_gb300.shard import partition_columns, solve_mu_sharded

    ctx = SubmatrixDensity.from_system(sysm, stream=stream.cuda_stream)
    ctx.set_filter_threshold(w["eps"])
    ctx.set_precision(args.precision)
    ctx.set_mu(0.0)
    ctx.build_density()
    dims, _, _ = ctx.get_submatrix_info()
    j0, j1 = partition_columns(dims, world)[rank]
    ctx.set_column_range(j0, j1)
    h_dev = torch.from_numpy(sysm.values).to("cuda")
    red = torch.zeros(2, dtype=torch.float64, device="cuda")

    def allreduce(x):
        if pg is None:
            return x
        red.copy_(torch.from_numpy(x))
        pg.all_reduce(red)
        return red.cpu().numpy()

    def step():
        ctx.set_values(h_dev, on_device=True)
        if _fixed_mu(w):
            ctx.set_mu(float(w["mu"]))
            ctx.build_density()
            t, e, m = ctx.get_trace()
            t, e = allreduce(np.array([t, e]))
            return m, t, 1
        m, t, _, n = solve_mu_sharded(ctx, w["n_e"], allreduce, max_steps=w.get("max_steps", args.max_steps),
                                      tol=1e-2)
        return m, t, n

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    res = None
    for a, b in ev:
        a.record(stream)
        res = step()
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    if pg:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    ctx.close()
    return {"ms_per_step": ms, "value": 1e3 / ms, "unit": "density matrices/s", "ranks": world,
            "columns_this_rank": [int(j0), int(j1)], "mu": res[0], "trace": res[1], "builds_per_step": res[2],
            "scaling": "strong", "note": "one system; block-column shards balanced by sum n_j^3, 16-byte "
                                         "all-reduce of (trace, energy) per bisection step"}


def run_ours(args):
    import torch

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    from paper_2205_14741_gb300 import SubmatrixDensity
    from synth import WORKLOADS, make_workload

    w = WORKLOADS[args.workload]
    big = args.workload != "water1024" and w["n_mol"] * w["b"] > 20000
    sysm = make_workload(args.workload)
    stream = torch.cuda.current_stream()
    fixed = _fixed_mu(w)
    n_e = w.get("n_e")
    if n_e is None:
        n_e = float(sysm.n_occ)

    if args.shard:
        sh = shard_leg(args, w, sysm, stream, pg, world, rank)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": sh["value"], "unit": sh["unit"], "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": sh["ms_per_step"],
                              "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                              "dtype": args.precision, "data": "synthetic",
                              "config": {"workload": WORKLOAD_TEXT.get(args.workload, args.workload),
                                         "parallelism": f"{world} block-column shards"},
                              "shard": sh}))
        if pg:
            pg.destroy_process_group()
        return 0

    # learned bound trained on held-out systems of the same generator (before any timing)
    model_path, model_info = None, None
    if args.bound_mode != "off":
        model_path, model_info = train_heldout_model(args, w, stream)

    ctx = SubmatrixDensity.from_system(sysm, stream=stream.cuda_stream)
    ctx.set_filter_threshold(w["eps"])
    ctx.set_electron_count(n_e, max_steps=w.get("max_steps", args.max_steps), tol=1e-2)
    if args.columns:
        # a column shard only (a small case for profiling one launch); needs a fixed mu
        if not fixed:
            raise SystemExit("--columns needs a fixed-mu workload")
        ctx.set_column_range(0, args.columns)
    h_dev = torch.from_numpy(sysm.values).to("cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    if model_path:
        ctx.bound_model_init(0)

    # --per-build: a step is one build at the solved mu (a density matrix at a given mu); the full
    # bisection is timed once beside it
    mu_fixed = float(w["mu"]) if fixed else None
    solve_once = None
    if args.per_build and not fixed:
        ctx.set_precision(args.precision)
        if model_path:
            ctx.set_bound_model(args.bound_mode, model_path if args.bound_mode != "off" else None)
        ctx.set_values(h_dev, on_device=True)
        ctx.set_mu(0.0)
        ctx.build_density()  # warm (pattern analysis, workspace)
        torch.cuda.synchronize()
        ctx.set_values(h_dev, on_device=True)
        ctx.reset_counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve_mu()
        e1.record(stream)
        torch.cuda.synchronize()
        sst = ctx.get_stats()
        mu_fixed = ctx.get_trace()[2]
        solve_once = {"seconds": e0.elapsed_time(e1) / 1e3, "bisection_builds": sst["bisection_steps"],
                      "mu": mu_fixed, "trace": ctx.get_trace()[0], "iters_mean_last_build": sst["iters_mean"],
                      "host_reads": sst["bisection_steps"] + 1}
        if args.mu_device:
            # the same solve with the bisection's decisions on the device (one host read)
            ctx.set_values(h_dev, on_device=True)
            ctx.set_mu(0.0)
            ctx.build_density()  # the filter of the new values (not part of the solve)
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.solve_mu_device()
            e1.record(stream)
            torch.cuda.synchronize()
            solve_once["device_loop"] = {"seconds": e0.elapsed_time(e1) / 1e3,
                                         "bisection_builds": ctx.get_stats()["bisection_steps"],
                                         "mu": ctx.get_trace()[2], "same_mu": ctx.get_trace()[2] == mu_fixed,
                                         "host_reads": 1}

    def step():
        ctx.set_values(h_dev, on_device=True)
        if mu_fixed is not None:
            ctx.set_mu(mu_fixed)
            ctx.build_density()
        else:
            ctx.solve_mu()

    def timed(n_steps, prec, mode="off", warmup=None):
        ctx.set_precision(prec)
        if model_path:
            ctx.set_bound_model(mode, model_path if mode != "off" else None)
        for _ in range(args.warmup if warmup is None else warmup):
            step()
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        ctx.reset_counters()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        clocks = ClockSampler(local)
        clocks.start()
        with no_gc():
            for k in range(n_steps):
                flush.zero_()  # write > L2 between timed steps (outside the events)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        stats = ctx.get_stats()
        if pg:
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return ms, stats, clk

    def summary(ms, st, n_steps):
        return {"value": n_steps * world / (ms / 1e3), "ms_per_step": ms / n_steps,
                "ns_ms_per_step": st["ns_ms_total"] / n_steps, "iters_mean": st["iters_mean"],
                "iters_max": st["iters_max"], "fallbacks_per_step": st["n_bound_fallback"] / n_steps}

    # -- the other spectral-bound modes (same form, same workload) -----------------
    modes = {}
    if model_path and args.mode_steps > 0:
        for mode in ["off", "rho", "gap"]:
            if mode != args.bound_mode:
                m0, s0, _ = timed(args.mode_steps, args.precision, mode, warmup=1)
                modes[mode] = summary(m0, s0, args.mode_steps)

    # -- the headline --------------------------------------------------------------
    ms, st, clk = timed(args.steps, args.precision, args.bound_mode)
    modes[args.bound_mode] = summary(ms, st, args.steps)
    tr, en, mu = ctx.get_trace()
    d_gpu = ctx.get_density()
    dims_all, _, _ = ctx.get_submatrix_info()
    value = args.steps * world / (ms / 1e3)
    ns_flops = 4.0 * st["ns_work_n3"]
    ns_s = st["ns_ms_total"] / 1e3
    submatrix_tflops = ns_flops / (ms / 1e3) / 1e12
    achieved = ns_flops / ns_s / 1e12 if ns_s > 0 else None
    peaks, peak_kind = _peaks()
    passes = 3 if args.precision == "fp16x3" else 1
    peak = peaks["bf16_tflops"] / passes
    d3 = dims_all.astype(np.float64) ** 3
    onchip = float(d3[((dims_all + 31) // 32) * 32 <= 192].sum() / max(d3.sum(), 1.0))
    form = (f"on-chip form (kpad <= 192) for {100 * onchip:.0f}% of the n^3 work"
            if onchip >= 0.5 else f"streamed form (kpad > 192) for {100 * (1 - onchip):.0f}% of the n^3 work")
    roofline = {
        "bound": "tensor", "kernel": f"k_ns_tc<{args.precision}>, {form}", "achieved": achieved, "peak": peak,
        "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": None,
        "note": f"achieved = sum_j 4 n_j^3 iters_j (true n; the kernel multiplies only the tiles on and right "
                f"of the diagonal blocks of the symmetric products, the count stays 4 n^3) / summed NS-kernel "
                f"event time; peak = {peak_kind} dense bf16/fp16 burst peak {peaks['bf16_tflops']} TF/s"
                + (" / 3 (three fp16 products per multiply-add in the split form)" if passes == 3 else ""),
        "ns_share_of_step": (st["ns_ms_total"] / ms) if ms > 0 else None,
    }
    n_cols = int(dims_all.shape[0]) if not args.columns else args.columns
    builds_timed = args.steps * (1 if mu_fixed is not None else max(1, st["bisection_steps"]))
    launches_per_build = max(1.0, st["ns_launches"] / builds_timed)
    gemms = 2.0 * st["iters_mean"] * n_cols / launches_per_build  # two GEMMs per step
    roofline["traffic"], roofline["traffic_note"] = _profiled_traffic(args.workload, args.precision, gemms)
    gpu_launches = int(st["kernel_launches"])

    # -- e2e through the C ABI with host buffers -------------------------------
    h_host = torch.from_numpy(sysm.values.copy()).pin_memory()
    d_host = torch.empty(sysm.values.shape[0], dtype=torch.float64).pin_memory()
    h_np, d_np = h_host.numpy(), d_host.numpy()
    e2e_times = []
    bis_steps = []
    with no_gc():
        for k in range(args.warmup + args.e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_values(h_np)
            if mu_fixed is not None:
                ctx.set_mu(mu_fixed)
                ctx.build_density()
            else:
                ctx.solve_mu()
            ctx.get_density(d_np)
            ctx.get_trace()
            t1 = time.perf_counter()
            if k >= args.warmup:
                e2e_times.append(t1 - t0)
                bis_steps.append(ctx.get_stats()["bisection_steps"] if mu_fixed is None else 1)
    e2e_s = sum(e2e_times)
    if pg:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())
    nbytes = sysm.values.shape[0] * 8
    e2e = ({"value": args.e2e_steps * world / e2e_s, "unit": "density matrices/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes + 24 * int(np.mean(bis_steps)) + 16} if args.e2e_steps > 0 else None)

    # -- the plain FP64 form on the same workload ------------------------------
    fp64 = None
    if not args.no_fp64:
        if model_path:
            ctx.set_bound_model("off")  # the plain form: Gershgorin start
        if big:
            # FP64 on a column subset (one submatrix per SM), extrapolated by the work sum n_j^3
            sub = min(int(dims_all.shape[0]), 152)
            ctx.set_column_range(0, sub)
            ms64, st64, _ = timed(1, "fp64", warmup=1)
            ctx.set_column_range(0, int(dims_all.shape[0]))
            d3 = dims_all.astype(np.float64) ** 3
            scale = float(d3.sum() / d3[:sub].sum())
            fp64 = {"value": world / (ms64 * scale / 1e3), "unit": "density matrices/s",
                    "ms_per_step": ms64 * scale, "sample": f"block columns 0..{sub - 1} timed, x{scale:.1f} "
                                                          f"(sum n_j^3 all / sample)",
                    "submatrix_tflops": 4.0 * st64["ns_work_n3"] / (ms64 / 1e3) / 1e12}
        else:
            ms64, st64, _ = timed(args.fp64_steps, "fp64")
            d64 = ctx.get_density()
            fp64 = {"value": args.fp64_steps * world / (ms64 / 1e3), "unit": "density matrices/s",
                    "ms_per_step": ms64 / args.fp64_steps,
                    "submatrix_tflops": 4.0 * st64["ns_work_n3"] / (ms64 / 1e3) / 1e12,
                    "max_abs_diff_vs_mixed": float(np.max(np.abs(d64 - d_gpu)))}

    # -- function forms on the same machinery (FP64, 1024-molecule inputs) ----------
    funcs = None
    nonorth = None
    if not args.no_functions and args.workload == "water1024":
        funcs = function_leg(args, stream, flush, rank == 0 and not args.no_cpu)
        nonorth = nonorth_leg(args, stream, flush, rank == 0 and not args.no_cpu)

    # -- accuracy and CPU baseline (rank 0, oracle on a bounded sample) ---------
    cpu = None
    acc = None
    if rank == 0 and not args.no_cpu:
        import oracle as O

        workers = os.cpu_count() or 1
        n_cols = args.ref_columns if not big else min(args.ref_columns, 2 * workers)
        dt, cols, res, (cp_f, ri_f) = _oracle_sample(sysm, w["eps"], mu, n_cols, workers)
        off = O.block_value_offsets(sysm.block_size, sysm.col_ptr, sysm.row_idx)
        _, _, _, keep = O.filter_blocks(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, w["eps"])
        off_f = O.block_value_offsets(sysm.block_size, cp_f, ri_f)
        kf = np.cumsum(keep) - 1
        err = 0.0
        for j in cols:  # the kept blocks of each sampled column (dropped blocks are zero on both sides)
            for k in range(sysm.col_ptr[j], sysm.col_ptr[j + 1]):
                a = d_gpu[off[k]:off[k + 1]]
                b = res.values[off_f[kf[k]]:off_f[kf[k] + 1]] if keep[k] else np.zeros_like(a)
                err = max(err, float(np.max(np.abs(a - b))))
        # the asymmetry of D (the submatrix D is not symmetric; a diagnostic, not a check): block (i, j)
        # of a sampled column against the transpose of block (j, i)
        asym = 0.0
        bs = np.asarray(sysm.block_size, dtype=np.int64)
        for j in cols:
            for k in range(sysm.col_ptr[j], sysm.col_ptr[j + 1]):
                i = int(sysm.row_idx[k])
                kk = sysm.col_ptr[i] + int(np.searchsorted(sysm.row_idx[sysm.col_ptr[i]:sysm.col_ptr[i + 1]], j))
                a_ = d_gpu[off[k]:off[k + 1]].reshape(bs[j], bs[i])      # block (i, j), column-major
                b_ = d_gpu[off[kk]:off[kk + 1]].reshape(bs[i], bs[j])    # block (j, i), column-major
                asym = max(asym, float(np.max(np.abs(a_ - b_.T))))
        acc = {"d_max_abs_err_sampled_columns": err, "columns": len(cols), "trace": tr, "energy": en, "mu": mu,
               "d_asymmetry_max_sampled_columns": asym}
        builds = int(round(np.mean(bis_steps))) if bis_steps else 1
        scale = _work_scale(sysm.block_size, cp_f, ri_f, cols)
        per_dm = dt * scale * builds
        cpu = {"value": 1.0 / per_dm, "unit": "density matrices/s", "cores": workers, "kind": "oracle",
               "sample": f"{len(cols)} of {sysm.n_blocks} block columns at the GPU's final mu, "
                         f"time x{scale:.1f} (sum n_j^3 all / sample) x{builds} bisection build(s)"}

    # -- precision study: single-pass bulk forms and FP64 finishing steps, same mu, same columns --
    study = None
    if rank == 0 and cpu is not None and not args.no_study and not big:
        from paper_2205_14741_gb300 import SmxError

        study = []
        if model_path:
            ctx.set_bound_model("off")
        for prec, final in [("fp16x3", 0), ("fp16x3", 1), ("fp16", 0), ("fp16", 2), ("bf16", 0), ("bf16", 2)]:
            row = {"bulk": prec, "fp64_final_iters": final}
            try:
                ctx.set_precision(prec, final)
                ctx.set_mu(mu)
                for _ in range(2):
                    ctx.build_density()
                torch.cuda.synchronize()
                ctx.reset_counters()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(5):
                    ctx.build_density()
                e1.record(stream)
                torch.cuda.synchronize()
                sst = ctx.get_stats()
                dv = ctx.get_density()
                err = 0.0
                for j in cols:
                    for k in range(sysm.col_ptr[j], sysm.col_ptr[j + 1]):
                        a_ = dv[off[k]:off[k + 1]]
                        b_ = res.values[off_f[kf[k]]:off_f[kf[k] + 1]] if keep[k] else np.zeros_like(a_)
                        err = max(err, float(np.max(np.abs(a_ - b_))))
                row.update(ms_per_build=e0.elapsed_time(e1) / 5, iters_mean=sst["iters_mean"], d_max_abs_err=err)
            except SmxError as e:
                row["status"] = str(e)
            study.append(row)
        ctx.set_precision(args.precision)

    learned = None
    if rank == 0 and world == 1 and args.learned_snapshots > 0 and args.workload == "water1024":
        learned = learned_scaling(args, stream)

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value, "unit": "density matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT.get(args.workload, args.workload),
                       "precision": args.precision, "l2": "flushed between timed steps (256 MiB write)",
                       "spectral_bound": {"off": "a-posteriori Gershgorin start, plain steps",
                                          "rho": "learned rho_hat (held-out training), plain steps",
                                          "gap": "learned rho_hat and gap (held-out training), scaled steps"}[
                           args.bound_mode],
                       "mu": ("fixed" if fixed else "one build per step at the mu of a full bisection "
                              "(timed once: mu_solve)" if args.per_build else "bisection (tol 1e-2)"),
                       "bisection_builds_per_step": float(np.mean(bis_steps)) if bis_steps else None,
                       "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
            "submatrix_tflops": submatrix_tflops,
            "fp64_plain": fp64,
            "inv_sqrt_fp64": funcs,
            "nonorth_fp64": nonorth,
            "speedup_mixed_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "accuracy": acc,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": gpu_launches,
            "iters": {"min": st["iters_min"], "max": st["iters_max"], "mean": st["iters_mean"]},
            "dims": {"min": st["dim_min"], "max": st["dim_max"], "mean": st["dim_mean"]},
            "bound_model": ({"headline_mode": args.bound_mode, "training": model_info, "modes": modes,
                             "fallback_rate": st["n_bound_fallback"] / (sysm.n_blocks * args.steps
                                                                      * max(1.0, float(np.mean(bis_steps))))}
                            if model_path else None),
            "learned_scaling": learned,
            "mu_solve": solve_once,
            "precision_study": ({"note": "builds at the headline's mu, a-posteriori Gershgorin start, 5 builds "
                                         "timed after 2; D error on the CPU-baseline columns",
                                 "rows": study} if study else None),
        }
        print(json.dumps(out))
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water1024")
    ap.add_argument("--precision", default="fp16x3", choices=["fp16x3", "fp16", "bf16", "fp64"])
    ap.add_argument("--bound-mode", default="gap", choices=["off", "rho", "gap"],
                    help="spectral bound of the headline: off, learned rho_hat, or rho_hat and gap (scaled steps)")
    ap.add_argument("--model-systems", type=int, default=2, help="held-out systems the learned bound trains on")
    ap.add_argument("--model-epochs", type=int, default=100)
    ap.add_argument("--mode-steps", type=int, default=5, help="timed steps of each non-headline bound mode")
    ap.add_argument("--e2e-steps", type=int, default=None, help="end-to-end steps (default: --steps)")
    ap.add_argument("--max-steps", type=int, default=30, help="bisection steps at most")
    ap.add_argument("--mu-device", action="store_true",
                    help="with --per-build: also time the solve with the bisection's decisions on the device")
    ap.add_argument("--per-build", action="store_true",
                    help="a step is one build at the solved mu; the full bisection is timed once")
    ap.add_argument("--columns", type=int, default=0,
                    help="restrict the timed context to block columns [0, N) (a small case for profiling)")
    ap.add_argument("--shard", action="store_true",
                    help="one system split over the ranks by block columns (strong scaling)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--ref-columns", type=int, default=128)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-functions", action="store_true", help="skip the A^-1/2 and non-orthogonal (FP64) legs")
    ap.add_argument("--no-study", action="store_true", help="skip the precision study (single-pass, FP64 finish)")
    ap.add_argument("--function-steps", type=int, default=3)
    ap.add_argument("--learned-snapshots", type=int, default=200,
                    help="trajectory length of the learned-bound report (0 skips it)")
    ap.add_argument("--learned-epochs", type=int, default=40)
    args = ap.parse_args()
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
