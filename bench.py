#!/usr/bin/env python
"""Chebyshev-filter throughput of the PAW-FE R-ChFSI filter on GB300.

Metric: GDoF.vec/s = M * N * m / t_CF, one DoF.vec being one DoF of one vector
advanced one Chebyshev degree (Algorithm 2 over all N vectors in blocks of B).
Workload ``mid``: periodic 40 bohr box, 16^3 cells of degree 6 (96^3 = 884,736
DoFs), 64 atoms x 13 projectors, N = 512 vectors in blocks of 256, degree 30.
Inputs are seeded synthetic data, resident in HBM (3.6 GB per FP64 block set,
far above the 129 MB L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain restatement of the
paper's method) on the host cores, on a bounded sample of the same workload.
Multi-GPU: replicas only (independent problems per rank, no data exchange);
rank 0 prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402

METRIC = "Cheb-filter GDoF·vec/s, FP32/TF32 vs FP64 on GB300 at eigval err ≤1e-6 Ha"
UNIT = "GDoF*vec/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sus=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


def _n_sm():
    try:
        import torch
        return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        return 152


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x, ws):
    """The largest x over the ranks (the slowest replica's time); x itself at ws = 1."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_desc(name):
    """The workload as named in the config of both arms' JSON lines."""
    cfg = inputs.CONFIGS[name]
    sysd = inputs.make_system(name)
    M = (cfg["ncell"] * cfg["p"]) ** 3
    return (f"{name}: L={sysd['L']} bohr, {cfg['ncell']}^3 cells, p={cfg['p']}, M={M} DoFs, "
            f"{sysd['natoms']} atoms x {sysd['nproj']} projectors, N={cfg['nvec']} in blocks of {cfg['block']}, "
            f"degree {cfg['degree']}")


def whole_job_rate(units_per_step_per_rank, ws, ms_per_step):
    """GDoF.vec/s of the whole job: every replica processes units_per_step_per_rank per step
    and the step takes ms_per_step on the slowest one (weak scaling)."""
    return units_per_step_per_rank * ws / (ms_per_step / 1e3) / 1e9


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- CPU oracle timing
_ORACLE_OPS = {}


def oracle_sample(workload: str, ncols: int, m: int):
    """Time the oracle's Algorithm 2 on `ncols` columns and degree `m` (units, seconds).

    The oracle's operator set-up is built once per workload and not timed."""
    from oracle import cheb
    from oracle import ops as O
    if workload not in _ORACLE_OPS:
        _ORACLE_OPS[workload] = O.PawOperators(inputs.make_system(workload))
    op = _ORACLE_OPS[workload]
    X = inputs.start_columns(workload, range(ncols))
    lam = np.linspace(-0.3, 0.2, ncols)
    bounds = (-0.5, 0.25, 200.0)
    t0 = time.perf_counter()
    cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, X, lam, m, *bounds)
    dt = time.perf_counter() - t0
    return float(op.mesh.ndof) * ncols * m, dt


def _threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] or [os.cpu_count() or 1])
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_info():
    """CPU model, online core count and architecture of the host that runs the oracle."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    nproc = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": nproc,
            "arch": platform.machine(), "blas_threads": _threads()}


def _timed_cpu(fn):
    """(result, wall seconds, threads actually used = process CPU time / wall time)."""
    c0, t0 = time.process_time(), time.perf_counter()
    r = fn()
    dt = time.perf_counter() - t0
    return r, dt, (time.process_time() - c0) / max(dt, 1e-9)


def tiny_full_oracle():
    """Config 1 timed in full: the oracle's R-ChFSI on the tiny workload (16 vectors, Chebyshev
    degree 20, 10 iterations of Algorithm 2 + Rayleigh-Ritz), FP64 numpy/scipy."""
    from oracle import cheb, rr
    from oracle import ops as O
    cfg = inputs.CONFIGS["tiny"]
    op = O.PawOperators(inputs.make_system("tiny"))
    X0 = inputs.start_columns("tiny", range(cfg["nvec"]))
    tmin, bU = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)), op.apply_S, op.mesh.ndof)
    Psi, lam = rr.rayleigh_ritz(op, X0)
    t_cf = 0.0
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(cfg["iters"]):
        a = time.perf_counter()
        Xf = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, cfg["degree"],
                                min(lam[0], tmin), lam[-1], bU)
        t_cf += time.perf_counter() - a
        Psi, lam = rr.rayleigh_ritz(op, Xf)
    dt = time.perf_counter() - t0
    units = float(op.mesh.ndof) * cfg["nvec"] * cfg["degree"] * cfg["iters"]
    return {"value": units / t_cf / 1e9, "unit": UNIT, "filter_s": round(t_cf, 3), "rchfsi_s": round(dt, 3),
            "threads_used": round((time.process_time() - c0) / max(dt, 1e-9), 2),
            "workload": f"tiny in full: {op.mesh.ndof} DoFs, {cfg['nvec']} vectors, degree {cfg['degree']}, "
                        f"{cfg['iters']} R-ChFSI iterations (filter time only in value)"}


def cpu_baseline(workload, ncols=2, m=8):
    (units, dt), _, used = _timed_cpu(lambda: oracle_sample(workload, ncols, m))
    info = cpu_info()
    out = {"value": units / dt / 1e9, "unit": UNIT, "cores": round(used, 2), "kind": "oracle",
           "sample": f"{workload}: {ncols} vectors, Chebyshev degree {m} (Algorithm 2, FP64 numpy/scipy), "
                     f"{dt:.1f} s; operator set-up excluded; cores = process CPU time / wall time",
           **info}
    try:
        out["tiny_full"] = tiny_full_oracle()
    except Exception as ex:   # the sample above is the baseline; this is context
        out["tiny_full"] = {"error": str(ex)[:200]}
    return out


# ----------------------------------------------------------------------------- accuracy
def gap_index(lam, k0, gap_min=1e-4):
    """The state count nearest to k0 whose gap lam[k] - lam[k-1] exceeds gap_min (Ha), so
    that a (near-)degenerate level is never split between compared and uncompared states."""
    n = len(lam)
    for d in range(n):
        for k in (k0 - d, k0 + d):
            if 1 <= k < n and lam[k] - lam[k - 1] > gap_min:
                return k
    return n


def s_angles(fe, A, B):
    """Principal angles between span(A) and span(B) (S-orthonormal blocks) in the S inner
    product; angles below pi/4 from their sines, the others from their cosines."""
    import torch
    SB = fe.apply_S(B)
    C = A.T @ SB
    cos = torch.linalg.svdvals(C).clamp(0.0, 1.0).flip(0)          # ascending angles
    R = B - A @ C                                                   # part of span(B) S-orthogonal to span(A)
    G = R.T @ fe.apply_S(R)
    sin = torch.linalg.eigvalsh(0.5 * (G + G.T)).clamp(0.0, 1.0).sqrt()
    ang = torch.where(sin < 0.5 ** 0.5, torch.asin(sin), torch.acos(cos))
    return ang.cpu().numpy()


def accuracy_leg(fe, X0, lam0, tmin, bU, m, iters, prec, k_target):
    """R-ChFSI (Algorithm 1 with Algorithm 2 as the filter) from one S-orthonormal start, the
    same number of iterations with the mixed-precision filter and with the FP64 filter (both
    with the FP64 Rayleigh-Ritz step); the lowest k states compared.  The FP64 arm's filter
    calls are timed on the stream (CUDA events) and give the FP64 form's throughput."""
    import torch
    stream = torch.cuda.current_stream()
    runs = {}
    for arm in (prec, "fp64"):
        X = X0.clone()
        lam = lam0.copy()
        out = torch.empty_like(X)
        ms = []
        for _ in range(iters):
            bounds = (min(lam[0], tmin), float(lam[-1]), bU)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fe.cheb_filter(X, lam, m, bounds, prec=arm, out=out)
            e1.record(stream)
            X, out = out, X
            lam = fe.rayleigh_ritz(X)                  # synchronises
            fe.sync_status()
            ms.append(e0.elapsed_time(e1))
        del out
        runs[arm] = (X, lam, fe.residuals(X, lam), ms)
    (Xa, la, ra, msa), (Xb, lb, rb, msb) = runs[prec], runs["fp64"]
    k = gap_index(lb, k_target)
    ang = s_angles(fe, Xa[:, :k], Xb[:, :k])
    k2 = gap_index(lb, k_target // 2)
    ang2 = s_angles(fe, Xa[:, :k2], Xb[:, :k2])
    res = {"iterations": iters, "degree": m, "start": "Ritz vectors of the random block (FP64 Rayleigh-Ritz)",
           "states_compared": k, "k_target": k_target, "gap_after_k_ha": float(lb[k] - lb[k - 1]) if k < len(lb) else None,
           "eigval_err": float(np.abs(la[:k] - lb[:k]).max()), "max_angle": float(ang.max()),
           "max_residual": {prec: float(ra[:k].max()), "fp64": float(rb[:k].max())},
           "lowest_half": {"states": k2, "eigval_err": float(np.abs(la[:k2] - lb[:k2]).max()),
                           "max_angle": float(ang2.max())},
           "bounds": {"eigval_ha": 1e-6, "angle": 1e-5},
           "reference": "the same iteration with the FP64 filter on the GPU (checked against the FP64 oracle "
                        "at this size, tests/test_gpu_fullsize.py)",
           "filter_ms": {prec: round(statistics.median(msa[1:] or msa), 3), "fp64": round(statistics.median(msb[1:] or msb), 3)}}
    res["pass"] = bool(res["eigval_err"] <= 1e-6 and res["max_angle"] <= 1e-5)
    fp64_ms = msb[1:] or msb
    del runs, Xa, Xb
    return res, fp64_ms


# ----------------------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import torch
    import paper_2604_26037_gb300 as P

    torch.cuda.set_device(local)
    cfg = inputs.CONFIGS[args.workload]
    sysd = inputs.make_system(args.workload)
    kp = tuple(args.kpoint) if args.kpoint else None
    fe = P.PawFE.from_system(sysd, block=cfg["block"], y0_fp32=args.y0_fp32, kpoint=kp,
                             y0_pair32=args.y0_pair32, overlap=not args.no_overlap)
    M, N, m = fe.ndof, cfg["nvec"], cfg["degree"]
    # the library overlaps the blocks of a call for real vectors in a reduced precision
    overlapped = (not args.no_overlap and args.prec != "fp64" and N > cfg["block"])
    g = torch.Generator(device="cuda").manual_seed(1234 + rank)
    # at a Bloch wavevector k the vectors are complex (one complex vector = one vector of the metric)
    X = torch.randn((M, N), dtype=torch.complex128 if fe.complex else torch.float64, device="cuda", generator=g)
    tmin, bU = fe.lanczos_bounds(20, 7)
    if args.start == "ritz":
        lam = fe.rayleigh_ritz(X)                   # S-orthonormal Ritz vectors of the random block
    else:
        # random block with sorted estimates in the lower 30% of the spectrum: the same filter
        # work without the FP64 Rayleigh-Ritz set-up (minutes for thousands of vectors)
        lam = np.sort(np.random.default_rng(1234 + rank).uniform(tmin, tmin + 0.3 * (bU - tmin), N))
    bounds = (min(lam[0], tmin), float(lam[-1]), bU)
    out = torch.empty_like(X)
    stream = torch.cuda.current_stream()

    def timed(prec, steps, warmup, profile=False, h=None, dst=None):
        h = fe if h is None else h
        dst = out if dst is None else dst
        for _ in range(warmup):
            h.cheb_filter(X, lam, m, bounds, prec=prec, out=dst)
        torch.cuda.synchronize()
        _barrier(ws)
        if profile:
            h.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                h.cheb_filter(X, lam, m, bounds, prec=prec, out=dst)
            e1.record(stream)
            torch.cuda.synchronize()
        h.sync_status()                 # a kernel that gave up on a bounded wait fails the run
        prof = h.profile_read() if profile else None
        if profile:
            h.profile_enable(False)
        _barrier(ws)
        ms = e0.elapsed_time(e1) / steps
        return _max_over_ranks(ms, ws), prof, clk.summary()

    ms, prof, clocks = timed(args.prec, args.steps, args.warmup, profile=True)
    units_per_step = float(M) * N * m
    value = whole_job_rate(units_per_step, ws, ms)
    # With the overlapped block schedule a phase's wall time includes the SMs it shares with
    # the other stream.  The same kernels timed with the blocks one after another (a second
    # handle, a few calls right after the timed region) give each kernel's own rate.
    iso_run = None
    iso_skip = None
    if overlapped and args.iso_steps > 0:
        # a second handle holds as much device memory as the first (its workspaces included,
        # which the timed calls have grown to full size); leave it out where it does not fit
        free, _ = torch.cuda.mem_get_info()
        need = int(fe.info()["device_bytes"])
        if need > 0.9 * free:
            iso_skip = f"a second handle ({need / 1e9:.1f} GB) does not fit beside the first ({free / 1e9:.1f} GB free)"
    if overlapped and args.iso_steps > 0 and iso_skip is None:
        fe_s = P.PawFE.from_system(sysd, block=cfg["block"], y0_fp32=args.y0_fp32, y0_pair32=args.y0_pair32,
                                   kpoint=kp, overlap=False)
        iso_run = timed(args.prec, args.iso_steps, 1, profile=True, h=fe_s)
        fe_s.close()
        del fe_s
        torch.cuda.empty_cache()

    # accuracy at this size: R-ChFSI with the mixed filter vs with the FP64 filter
    acc = None
    fp64 = None
    if args.accuracy_iters > 0 and not kp and args.start == "ritz":
        acc, ms64s = accuracy_leg(fe, X, lam, tmin, bU, m, args.accuracy_iters, args.prec, N // 2)
        ms64 = _max_over_ranks(statistics.median(ms64s), ws)
        fp64 = {"value": whole_job_rate(units_per_step, ws, ms64), "ms_per_step": ms64, "steps": len(ms64s),
                "warmup": 1, "source": "FP64-filter calls of the accuracy leg (CUDA events on the stream)"}
        torch.cuda.empty_cache()

    # FP64 form of the same filter (the plain method), fewer steps: it is slow on GB300
    if fp64 is None and args.fp64_steps > 0:
        ms64, _, _ = timed("fp64", args.fp64_steps, 1)
        fp64 = {"value": whole_job_rate(units_per_step, ws, ms64), "ms_per_step": ms64,
                "steps": args.fp64_steps, "warmup": 1}

    # the same filter with step 2 in pair-of-FP32 arithmetic (FP64-class accuracy on the FP32 pipes)
    pair = None
    if args.pair_steps > 0 and not kp and not args.y0_pair32:
        fe_p = P.PawFE.from_system(sysd, block=cfg["block"], y0_fp32=args.y0_fp32, y0_pair32=True,
                                   overlap=not args.no_overlap)
        out_p = torch.empty_like(out)
        ms_p, prof_p, clk_p = timed(args.prec, args.pair_steps, 1, profile=True, h=fe_p, dst=out_p)
        # both handles filter the same input with the FP64 bracket: the outputs differ
        # by the step-2 rounding only
        fe.cheb_filter(X, lam, m, bounds, prec="fp64", out=out)
        fe_p.cheb_filter(X, lam, m, bounds, prec="fp64", out=out_p)
        diff64 = float((out_p - out).abs().max() / out.abs().max())
        ph = {k: round(v["ms"] / args.pair_steps, 3) for k, v in prof_p.items() if isinstance(v, dict)}
        ph64 = {k: v["ms"] / args.steps for k, v in prof.items() if isinstance(v, dict)}
        s2 = ph["residual_local"] + ph["residual_nonlocal"]
        s2_64 = ph64["residual_local"] + ph64["residual_nonlocal"]
        pair = {"value": round(whole_job_rate(units_per_step, ws, ms_p), 4), "ms_per_step": round(ms_p, 3),
                "steps": args.pair_steps, "warmup": 1, "phases_ms_per_step": ph,
                "step2_ms": round(s2, 3), "step2_speedup_vs_fp64": round(s2_64 / s2, 3),
                "fp64_bracket_output_rel_diff": diff64, "clocks": clk_p,
                "arithmetic": "step 2 with every product and sum on pairs of FP32 numbers (about 48 bits); "
                              "Y stored FP64; the rest of the call as the main measurement"}
        del out_p
        fe_p.close()

    # end to end through the public API with host buffers (pinned), copies inside the timed
    # region: every step copies the whole block in, filters it with one call and copies the
    # result out.  Consecutive steps are pipelined with three device buffer sets: the input of
    # step i + 2 is copied in (one copy stream, once step i - 1 has read its buffer) and the
    # output of step i out (another) while the filter calls run, each copy in 8 row chunks.  The
    # copy rate between pinned host memory and the GPU varies several-fold from run to run on
    # this machine (17 to 260 ms for the same 3.6 GB), so the inputs run two steps ahead.
    # Events around every copy and filter call give the per-step times.
    e2e = None
    if not args.no_e2e:
        del out
        torch.cuda.empty_cache()
        Xh = X.cpu().pin_memory()
        Oh = torch.empty_like(Xh).pin_memory()
        NB = 3
        Xd = [torch.empty_like(X) for _ in range(NB)]
        Od = [torch.empty_like(X) for _ in range(NB)]
        del X
        torch.cuda.empty_cache()
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        comp = torch.cuda.current_stream()
        nchunk = 8
        rows = (M + nchunk - 1) // nchunk
        tev = lambda: torch.cuda.Event(enable_timing=True)

        def e2e_run(n):
            ev_in, ev_f, ev_o = [None] * n, [None] * n, [None] * n
            spans = {"h2d": [], "filter": [], "d2h": []}
            t_first = tev()
            t_first.record(comp)

            def h2d(i):
                with torch.cuda.stream(s_in):
                    if i >= NB:
                        s_in.wait_event(ev_f[i - NB])         # the filter of step i - NB has read the buffer
                    a = tev()
                    a.record(s_in)
                    for r in range(0, M, rows):
                        Xd[i % NB][r:r + rows].copy_(Xh[r:r + rows], non_blocking=True)
                    ev_in[i] = tev()
                    ev_in[i].record(s_in)
                    spans["h2d"].append((a, ev_in[i]))

            for i in range(min(n, NB - 1)):
                h2d(i)
            for i in range(n):
                b = i % NB
                comp.wait_event(ev_in[i])
                if i >= NB:
                    comp.wait_event(ev_o[i - NB])             # Od[b] of step i - NB copied out
                f0 = tev()
                f0.record(comp)
                fe.cheb_filter(Xd[b], lam, m, bounds, prec=args.prec, out=Od[b])
                ev_f[i] = tev()
                ev_f[i].record(comp)
                spans["filter"].append((f0, ev_f[i]))
                if i + NB - 1 < n:
                    h2d(i + NB - 1)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_f[i])
                    o0 = tev()
                    o0.record(s_out)
                    for r in range(0, M, rows):
                        Oh[r:r + rows].copy_(Od[b][r:r + rows], non_blocking=True)
                    ev_o[i] = tev()
                    ev_o[i].record(s_out)
                    spans["d2h"].append((o0, ev_o[i]))
            torch.cuda.synchronize()
            return ({k: [a.elapsed_time(e) for a, e in v] for k, v in spans.items()},
                    {k: [t_first.elapsed_time(a) for a, _ in v] for k, v in spans.items()})

        e2e_run(2)                      # untimed: both buffer pairs and both copy directions
        _barrier(ws)
        t0 = time.perf_counter()
        spans, starts = e2e_run(args.steps)
        t_e2e = _max_over_ranks((time.perf_counter() - t0) / args.steps, ws)
        fe.sync_status()
        e2e = {"value": whole_job_rate(units_per_step, ws, t_e2e * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size() + N * 8),
               "d2h_bytes_per_step": int(Oh.numel() * Oh.element_size()),
               "ms_per_step": round(t_e2e * 1e3, 3),
               "step_ms": {k: [round(x, 2) for x in v] for k, v in spans.items()},
               "start_ms": {k: [round(x, 2) for x in v] for k, v in starts.items()},
               "overlap": "three device buffer sets: the H2D copy of step i+2 (one copy stream) and the D2H copy "
                          "of step i (another) run beside the filter calls, 8 row chunks each; the first input "
                          "and the last output copy are not overlapped"}
        out = Od[(args.steps - 1) % NB] if (args.rr or args.grad) else None   # a filtered block
        del Xd, Xh, Oh
        X = None

    # Rayleigh-Ritz on the filtered block: FP64 rotation vs the mixed-precision one (rr_mixed)
    rrm = None
    if args.rr:
        def rr_time(h, Xs):
            Xc = Xs.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam_r = h.rayleigh_ritz(Xc)             # synchronises (host eigenvalues)
            return time.perf_counter() - t0, lam_r, Xc
        rr_time(fe, out)                            # warm
        t64, lam64, X64 = rr_time(fe, out)
        fe_mx = P.PawFE.from_system(sysd, block=cfg["block"], y0_fp32=args.y0_fp32, rr_mixed=True)
        rr_time(fe_mx, out)
        tmx, lammx, Xmx = rr_time(fe_mx, out)
        sgn = torch.sign((X64 * Xmx).sum(0))
        rrm = {"vectors": N, "fp64_rotation_s": round(t64, 4), "mixed_rotation_s": round(tmx, 4),
               "speedup": round(t64 / tmx, 3), "max_ritz_value_diff": float(np.abs(lam64 - lammx).max()),
               "max_vector_diff_rel": float((X64 - Xmx * sgn).abs().max() / X64.abs().max()),
               "projection": "lower triangle (column blocks)"}
        fe_mx.close()
        del X64, Xmx

    # adjoint of E = tr(X^T H X) at the filtered block (the differentiation workload)
    gradm = None
    if args.grad:
        Xf = out.clone()
        X32 = Xf.float()
        fe.energy_grad(X32, "fp32")
        fe.energy_grad(Xf, "fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gV32, gD32 = fe.energy_grad(X32, "fp32")
        torch.cuda.synchronize()
        t32 = time.perf_counter() - t0
        t0 = time.perf_counter()
        gV, gD = fe.energy_grad(Xf, "fp64")
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        # E is linear in V and Delta_H: <dE/dV, d> = E(V = d) - E(V = 0) exactly (same for D)
        rng = np.random.default_rng(99)
        dV = torch.from_numpy(rng.standard_normal((fe.ncells, fe.quad_per_cell))).cuda()
        dD = rng.standard_normal((fe.natoms, fe.nproj, fe.nproj))
        dD = dD + dD.transpose(0, 2, 1)
        fe.set_veff(dV)
        e1 = fe.energy(Xf)
        fe.set_veff(torch.zeros_like(dV))
        e0 = fe.energy(Xf)
        fdV = e1 - e0
        fe.set_dij(dD)
        e1 = fe.energy(Xf)
        fe.set_dij(np.zeros_like(dD))
        e0 = fe.energy(Xf)
        fdD = e1 - e0
        lin_V = float((gV * dV).sum())
        lin_D = float((gD.cpu().numpy() * dD).sum())
        gradm = {"vectors": N, "quad_points": fe.ncells * fe.quad_per_cell, "d_entries": fe.natoms * fe.nproj ** 2,
                 "fp32_ms": round(t32 * 1e3, 3), "fp64_ms": round(t64 * 1e3, 3),
                 "fp32_vs_fp64_rel_V": float((gV32 - gV).norm() / gV.norm()),
                 "fp32_vs_fp64_rel_D": float((gD32 - gD).norm() / gD.norm()),
                 "fd_rel_V": abs(fdV - lin_V) / abs(fdV), "fd_rel_D": abs(fdD - lin_D) / abs(fdD)}

    # roofline of the dominant phase
    peaks = _peaks()
    phases = {k: v for k, v in prof.items() if isinstance(v, dict)}
    dom = max(phases, key=lambda k: phases[k]["ms"])
    roof = roofline(dom, phases[dom], fe, sysd, cfg, args.prec, peaks, clocks, args.workload)
    all_roof = {k: roofline(k, v, fe, sysd, cfg, args.prec, peaks, clocks, args.workload) for k, v in phases.items()}
    # each kernel's own rate (blocks one after another), beside the timed region's
    iso = None
    if iso_run is not None:
        ms_s, prof_s, clk_s = iso_run
        ph_s = {k: v for k, v in prof_s.items() if isinstance(v, dict)}
        iso = {k: roofline(k, v, fe, sysd, cfg, args.prec, peaks, clk_s, args.workload) for k, v in ph_s.items()}
        src = (f"the same kernels with the blocks one after another (options.no_overlap = 1), {args.iso_steps} "
               f"calls after the timed region: {ms_s:.1f} ms per call")
        roof["isolated"] = {kk: iso[dom][kk] for kk in ("achieved", "frac", "ms_per_launch") if kk in iso[dom]}
        roof["isolated"]["source"] = src
        if "peak_alt" in iso[dom]:
            roof["isolated"]["frac_alt"] = iso[dom]["peak_alt"]["frac"]
        roof["schedule"] = ("timed region: step 2 of block 0 alone, step 2 of block 1 beside the loop of block 0, "
                            "so the average launch duration includes the SMs shared with the loop")
        for k in all_roof:
            if k in iso:
                all_roof[k]["isolated_frac"] = iso[k]["frac"]
                all_roof[k]["isolated_ms_per_launch"] = iso[k]["ms_per_launch"]
        iso = {"ms_per_step": round(ms_s, 3), "steps": args.iso_steps, "warmup": 1, "clocks": clk_s,
               "phases_ms_per_step": {k: round(v["ms"] / args.iso_steps, 3) for k, v in ph_s.items()},
               "value": round(whole_job_rate(units_per_step, ws, ms_s), 4)}
    elif iso_skip is not None:
        iso = {"skipped": iso_skip}
    launches = prof["total_launches"] // args.steps

    res = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"tf32": "tf32", "fp32": "f32", "bf16": "bf16", "fp64": "f64"}[args.prec],
        "data": "synthetic (seeded), inputs resident in HBM and larger than L2",
        "config": {"workload": workload_desc(args.workload),
                   "precision": args.prec, "y0_storage": "fp32" if args.y0_fp32 else "fp64",
                   "step2_arithmetic": "pair-of-FP32" if args.y0_pair32 else "fp64",
                   **({"kpoint_per_bohr": list(kp), "vectors": "complex (real blocks of 2 B columns inside)"}
                      if kp else {}),
                   "start": args.start,
                   "block_schedule": ("step 2 of block j+1 overlaps the loop of block j (two internal streams)"
                                      if overlapped else "blocks one after another"),
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "phases_ms_per_step": {k: round(v["ms"] / args.steps, 3) for k, v in phases.items()},
        "phase_roofline": {k: {kk: v[kk] for kk in ("bound", "frac", "achieved", "unit", "ms_per_launch", "traffic",
                                                   "isolated_frac", "isolated_ms_per_launch")
                               if kk in v} for k, v in all_roof.items()},
        "serial_schedule": iso,
        "fp64_form": fp64,
        "speedup_vs_fp64": (round(value / fp64["value"], 3) if fp64 else None),
        "e2e": e2e,
        "bounds": [float(b) for b in bounds],
    }
    if acc is not None:
        res["accuracy"] = acc
    if pair is not None:
        res["step2_pair32"] = pair
    if rrm is not None:
        res["rayleigh_ritz"] = rrm
    if gradm is not None:
        res["gradient"] = gradm
    fe.close()
    return res


def fe_np1(nc):
    return int(round(nc ** (1.0 / 3.0)))


# kernels that make up each profiled phase of the filter (library phase brackets)
PHASE_KERNELS = {
    "residual_local": "k_local_sf (FP64 even/odd sum-factorised 1/2 K + V - lambda M)",
    "residual_nonlocal": "k_own_project64 + k_pair_reduce + k_own_couple + k_own_expand64 (FP64)",
    "recurrence": "k_exp_stream (tcgen05: fused Shat^-1 expansion + nonlocal H + recurrence update)",
    "projection": "k_tc_stream<ProjStream> + k_own_couple_sh (W_S and W_H from U)",
    "cell_products": "k_tc_stream<CellStream> (tcgen05 TF32/BF16) or k_cell_simt",
    "recovery": "Shat^-1 of R_m + FP64 combination",
}

# DRAM bytes per DoF.vector moved by the main kernel(s) of a phase, read off one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, a single pass) of a full-width launch with the
# kernels of this version, on the workload named in the entry; a launch of another size is scaled
# by its DoF.vectors (the traffic of these kernels grows in proportion to it).  Keyed by (phase,
# precision); None = the same kernels in every precision.  Summaries: profiles/.
MEASURED_TRAFFIC = {
    ("cell_products", "tf32"): (23.17, "k_tc_stream<CellStream>", "mid"),
    ("recurrence", "tf32"): (25.60, "k_exp_stream<2>", "mid"),
    ("projection", "tf32"): (5.584, "k_tc_stream<ProjStream>", "mid"),
    ("residual_local", None): (30.88, "k_local_sf<7,double>", "prof12"),
    ("residual_nonlocal", None): (32.33, "k_own_project64<16,double> + k_own_expand64<16,0,double>", "prof12"),
}


def measured_traffic(phase, prec, units, workload):
    """(bytes per launch, note) from MEASURED_TRAFFIC, or (None, None)."""
    hit = MEASURED_TRAFFIC.get((phase, None)) or MEASURED_TRAFFIC.get((phase, prec))
    if not hit:
        return None, None
    note = f"ncu capture of {hit[1]} on the {hit[2]} workload ({hit[0]} B per DoF.vector)"
    if workload != hit[2]:
        note += ", scaled by DoF.vectors"
    return round(hit[0] * units), note


def sf_flops_per_cell_vec(n1):
    """FP64 flops of the even/odd sum-factorised (1/2 K + V - lambda M) x per cell and vector
    (n1 nodes and n1 + 1 Gauss points per direction; FMA = 2 flops, add or multiply = 1)."""
    q1 = n1 + 1

    def eo(m, n):       # FMAs of one centro-symmetric m x n line product
        return ((m + 1) // 2) * ((n + 1) // 2) + (m // 2) * (n // 2)

    def split(n):       # adds forming the even/odd halves of a line
        return 2 * (n // 2)

    def outs(m):        # adds recombining the halves
        return m - (m & 1)

    lines = n1 * n1
    fl = 0
    fl += lines * (split(n1) + 2 * 2 * eo(n1, n1) + 2 * outs(n1))                  # P, Q
    fl += lines * (2 * split(n1) + 3 * 2 * eo(n1, n1) + 2 * n1 + 2 * outs(n1))  # S, R (R = kf T + c S on the halves)
    fl += n1 * n1 * (split(n1) + 2 * eo(q1, n1) + outs(q1))                      # U1
    fl += q1 * n1 * (split(n1) + 2 * eo(q1, n1) + outs(q1))                      # U2
    fl += q1 * q1 * (split(n1) + 2 * eo(q1, n1) + outs(q1) + q1)                 # U3 (times w V)
    fl += q1 * q1 * (split(q1) + 2 * eo(n1, q1) + outs(n1))                      # B2
    fl += q1 * n1 * (split(q1) + 2 * eo(n1, q1) + outs(n1))                      # B1
    # y: the last kinetic / mass and potential contractions in one accumulator per line
    fl += lines * (2 * split(n1) + split(q1) + 2 * 2 * eo(n1, n1) + 2 * eo(n1, q1) + outs(n1))
    return fl


def phase_model(phase, fe, cfg, prec):
    """Algorithmic (flops, bytes, compute kind) of one launch of a phase for one block.

    At a Bloch wavevector k a block of B complex vectors is processed as 2 B real
    columns; the extra cell products of the -i k.grad term (a shared cell matrix)
    are not in this model.
    """
    M, B = fe.ndof, cfg["block"] * (2 if fe.complex else 1)
    nc, ncells = fe.nodes_per_cell, fe.ncells
    n1 = fe_np1(nc)
    # algorithmic projector work: the nonzero entries of P^a on owned nodes
    # (no padding to 16 projectors, no all-zero projector of a pair)
    own, pairs, nnz = (n1 - 1) ** 3, fe.owner_pairs, fe.proj_nnz
    f32 = prec != "fp64"
    es = 4 if f32 else 8
    if phase == "cell_products":
        mat_es = {"bf16": 2, "tf32": 4, "fp32": 4, "fp64": 8}[prec]
        if prec == "fp64":   # sum-factorised local H in FP64
            return float(sf_flops_per_cell_vec(n1)) * ncells * B, M * B * 8 * 3, "fp64"
        kind = {"tf32": "tf32", "bf16": "bf16", "fp32": "fp32"}[prec]
        return 2.0 * ncells * nc * nc * B, ncells * nc * nc * mat_es + M * B * 4 * 3, kind
    if phase == "residual_local":
        return float(sf_flops_per_cell_vec(n1)) * ncells * B, M * B * 8 * 3, "fp64"
    pbytes = nnz * es
    if phase == "projection":
        return (2.0 * nnz * B, M * B * es + pbytes + 2 * pairs * fe.nproj * B * es, "fp32" if f32 else "fp64")
    if phase == "recurrence":
        # reads R_Y, R_X and Y (an FP32 hi/lo pair or FP64: 8 bytes), writes T and R_X
        return (4.0 * nnz * B, M * B * (es * 4 + 8) + pbytes, "fp32" if f32 else "fp64")
    if phase == "residual_nonlocal":
        return (4.0 * nnz * B, M * B * 8 * 3 + 2 * nnz * 8, "fp64")
    if phase == "recovery":
        return (4.0 * nnz * B, M * B * (es * 2 + 8 * 2), "fp32" if f32 else "fp64")
    return None, None, None


def compute_peak(kind, peaks, sm_mhz):
    """(TFLOP/s ceiling, bound, source) of a compute kind: tensor formats from the measured BF16
    burst (x the nominal dense ratio for TF32); plain ALU arithmetic from the unit counts and the
    SM clock sampled during the timed region."""
    nsm = _n_sm()
    if kind == "tf32":
        return (peaks["bf16"] * (1.1 / 2.25), "tensor",
                f"{peaks['src']} BF16 burst {peaks['bf16']} TFLOP/s x nominal TF32/BF16 ratio 1.1/2.25")
    if kind == "bf16":
        return peaks["bf16"], "tensor", f"{peaks['src']} BF16 burst"
    if kind == "fp64":
        # the FP64 pipe retires 2 FMA per SM per clock on GB300 (1.25 TFLOP/s nominal at 2070 MHz)
        return (nsm * 2 * 2 * sm_mhz * 1e6 / 1e12, "alu",
                f"derived: {nsm} SMs x 2 FP64 FMA/clk x 2 flop x {sm_mhz:.0f} MHz (median sampled SM clock)")
    return (nsm * 128 * 2 * sm_mhz * 1e6 / 1e12, "alu",
            f"derived: {nsm} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (median sampled SM clock)")


def roofline(phase, pinfo, fe, sysd, cfg, prec, peaks, clocks, workload=None):
    """Roofline of one phase of the filter, per launch, from algorithmic bytes/flops."""
    per_launch_ms = pinfo["ms"] / max(pinfo["intervals"], 1)
    flops, byts, kind = phase_model(phase, fe, cfg, prec)
    if flops is None or per_launch_ms <= 0:
        return {"bound": "hbm", "achieved": None, "peak": peaks["hbm"], "unit": "GB/s", "frac": None,
                "traffic": None, "kernel": phase, "peak_source": f"{peaks['src']} HBM copy bandwidth"}
    sec = per_launch_ms / 1e3
    gbs = byts / sec / 1e9
    traffic, tnote = (measured_traffic(phase, prec, float(fe.ndof) * cfg["block"], workload)
                      if not fe.complex else (None, None))
    tfs = flops / sec / 1e12
    hbm_frac = gbs / peaks["hbm"]
    sm_mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    cpk, cbound, csrc = compute_peak(kind, peaks, sm_mhz)
    c_frac = tfs / cpk
    common = {"traffic": traffic, "traffic_source": tnote, "kernel": phase, "kernels": PHASE_KERNELS.get(phase),
              "ms_per_launch": round(per_launch_ms, 4), "algorithmic_bytes_per_launch": byts,
              "algorithmic_flops_per_launch": flops}
    if c_frac >= hbm_frac:
        out = {"bound": cbound, "achieved": round(tfs, 3), "peak": round(cpk, 4), "unit": "TFLOP/s",
               "frac": round(c_frac, 4), "hbm_frac": round(hbm_frac, 4), "compute": kind, "peak_source": csrc,
               **common}
        if kind == "fp64":
            # the same kernel against the other admissible ceiling: the measured BF16 burst x the
            # nominal FP64/BF16 ratio (1.25 / 2250)
            alt = peaks["bf16"] * 1.25 / 2250.0
            out["peak_alt"] = {"peak": round(alt, 4), "frac": round(tfs / alt, 4),
                               "source": f"{peaks['src']} BF16 burst x nominal FP64/BF16 ratio 1.25/2250"}
        return out
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm"], "unit": "GB/s",
            "frac": round(hbm_frac, 4), "compute_frac": round(c_frac, 4), "compute": kind,
            "peak_source": f"{peaks['src']} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)", **common}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return None
    cfg = inputs.CONFIGS[args.workload]
    ncols, m = 1, 3
    vals, dts, used = [], [], []
    for _ in range(args.warmup):
        oracle_sample(args.workload, ncols, m)
    for _ in range(args.steps):
        (u, dt), _, th = _timed_cpu(lambda: oracle_sample(args.workload, ncols, m))
        vals.append(u / dt / 1e9)
        dts.append(dt)
        used.append(th)
    v = statistics.median(vals)
    cb = {"value": v, "unit": UNIT, "cores": round(statistics.median(used), 2), "kind": "oracle",
          "sample": f"{args.workload}: {ncols} vector, Chebyshev degree {m} per step (Algorithm 2, FP64 "
                    f"numpy/scipy); operator set-up excluded; cores = process CPU time / wall time",
          **cpu_info()}
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.median(dts) * 1e3, 3),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": workload_desc(args.workload), "precision": "fp64", "parallelism": "cpu"},
            "cpu_baseline": cb, "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- batched instances
def run_batch(args, ws, rank, local):
    """32 independent uneven instances (cells 4^3..12^3, degree 4-6, 8-64 atoms,
    block widths 32-512, Chebyshev degree 25) filtered by one CUDA-graph launch
    per step.  Throughput = sum_i M_i B_i m / t."""
    import torch
    import paper_2604_26037_gb300 as P

    torch.cuda.set_device(local)
    systems = inputs.batch_systems()
    fes, probs, units = [], [], 0.0
    for k, sd in enumerate(systems):
        fe = P.PawFE.from_system(sd, block=sd["block"], y0_fp32=args.y0_fp32)
        g = torch.Generator(device="cuda").manual_seed(4321 + 97 * k + rank)
        X = torch.randn((fe.ndof, sd["nvec"]), dtype=torch.float64, device="cuda", generator=g)
        lam = fe.rayleigh_ritz(X)
        tmin, bU = fe.lanczos_bounds(20, 7)
        probs.append((X, lam, sd["degree"], (min(lam[0], tmin), float(lam[-1]), bU), torch.empty_like(X)))
        units += float(fe.ndof) * sd["nvec"] * sd["degree"]
        fes.append(fe)
    stream = torch.cuda.current_stream()
    batch = P.PawBatch(fes, streams=4, autotune=True)
    for _ in range(args.warmup):
        batch.cheb_filter(probs, prec=args.prec)
    torch.cuda.synchronize()
    _barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            batch.cheb_filter(probs, prec=args.prec)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = _max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
    value = whole_job_rate(units, ws, ms)
    tun = [batch.tuning(i) for i in range(len(fes))]
    # the same instances one after another through paw_cheb_filter (no graph, no concurrency)
    for (X, lam, m, bd, out), fe in zip(probs, fes):
        fe.cheb_filter(X, lam, m, bd, prec=args.prec, out=out)
    torch.cuda.synchronize()
    e0.record(stream)
    for (X, lam, m, bd, out), fe in zip(probs, fes):
        fe.cheb_filter(X, lam, m, bd, prec=args.prec, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_serial = e0.elapsed_time(e1)
    # end to end: host (pinned) inputs and outputs of every instance, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hosts = [(X.cpu().pin_memory(), torch.empty_like(out, device="cpu").pin_memory()) for X, _, _, _, out in probs]
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for (Xh, _), (X, _, _, _, _) in zip(hosts, probs):
                X.copy_(Xh, non_blocking=True)
            batch.cheb_filter(probs, prec=args.prec)
            for (_, Oh), (_, _, _, _, out) in zip(hosts, probs):
                Oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e = _max_over_ranks((time.perf_counter() - t0) / args.steps, ws)
        e2e = {"value": whole_job_rate(units, ws, t_e2e * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(h[0].numel() * 8 for h in hosts)),
               "d2h_bytes_per_step": int(sum(h[1].numel() * 8 for h in hosts))}
    res = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"tf32": "tf32", "fp32": "f32", "bf16": "bf16", "fp64": "f64"}[args.prec],
        "data": "synthetic (seeded)",
        "config": {"workload": f"batch32: {len(fes)} independent instances, cells n^3 with n in 4..12 "
                               f"(h = 2.5 bohr), degree 4-6, 8-64 atoms x 13 projectors, block widths "
                               f"32-512, Chebyshev degree 25; one CUDA-graph launch per step",
                   "precision": args.prec, "parallelism": f"replicas x{ws}",
                   "dofs_vec_per_degree": units / 25.0},
        "gpu_launches": int(tun[0]["kernel_nodes"]),
        "graph": {"nodes": tun[0]["graph_nodes"], "kernel_nodes": tun[0]["kernel_nodes"],
                  "branches": tun[0]["branches"], "captures": tun[0]["captures"]},
        "tuning": {"persistent": sum(1 for t in tun if t["tc_variant"] == 0),
                   "one_cta_per_tile": sum(1 for t in tun if t["tc_variant"] == 1),
                   "grid_cap": tun[0]["grid_cap"]},
        "serial_calls_ms": round(ms_serial, 3),
        "speedup_vs_serial_calls": round(ms_serial / ms, 3),
        "clocks": clk.summary(),
        "roofline": None,
        "e2e": e2e,
    }
    batch.close()
    for fe in fes:
        fe.close()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid", choices=sorted(inputs.CONFIGS) + ["batch32"])
    ap.add_argument("--prec", default="tf32", choices=["tf32", "fp32", "bf16", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed FP64-filter calls when the accuracy leg does not run (it times them itself)")
    ap.add_argument("--accuracy-iters", type=int, default=16,
                    help="R-ChFSI iterations of the accuracy leg, mixed vs FP64 filter (0: skip)")
    ap.add_argument("--y0-fp32", action="store_true")
    ap.add_argument("--y0-pair32", action="store_true",
                    help="form step 2 (Y = H X - S X Lambda) in pair-of-FP32 arithmetic in the main measurement")
    ap.add_argument("--pair-steps", type=int, default=3,
                    help="timed calls of the filter with a pair-of-FP32 step 2, reported beside the FP64 one "
                         "(0: skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-overlap", action="store_true",
                    help="filter the blocks one after another (no overlap of step 2 with the previous block's loop)")
    ap.add_argument("--iso-steps", type=int, default=2,
                    help="calls timed with the blocks one after another after the (overlapped) timed region, "
                         "for each kernel's own roofline (0: skip)")
    ap.add_argument("--kpoint", type=float, nargs=3, default=None,
                    help="Bloch wavevector k (1/bohr): complex vectors, throughput per complex vector")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grad", action="store_true",
                    help="also time the adjoint (gradient of tr(X^T H X)) at the filtered block, with checks")
    ap.add_argument("--rr", action="store_true",
                    help="also time Rayleigh-Ritz on the filtered block, FP64 vs mixed-precision rotation")
    ap.add_argument("--start", default="ritz", choices=["ritz", "random"],
                    help="start block: Ritz vectors of a random block (default) or the random block itself")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if ws > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
    elif args.workload == "batch32":
        res = run_batch(args, ws, rank, local)
    else:
        res = run_ours(args, ws, rank, local)
        if rank == 0 and not args.no_cpu_baseline and not args.kpoint:
            res["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
