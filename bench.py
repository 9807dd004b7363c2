#!/usr/bin/env python
"""Benchmark: D-BiCGStab solves/s at relative residual 1e-10 on one GB300.

Workload (default): 16^4 periodic lattice, complex128, links exp(i*0.5*H),
kappa = 0.99 kappa_c.  One step is the whole method on one batch:
GMRES-DR(80,40) on a Z4 source to 1e-10 (giving V), the deflation space
(W = A V, LU of U^dagger A V with U = gamma5 V), and D-BiCGStab(40) on 10
further Z4 sources, all to a true relative residual of 1e-10.  value =
D-BiCGStab solves per second with the whole step in the denominator.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

For N > 1 launch under torchrun: every rank solves its own, independently
seeded batch on its own GPU (no collective on the data path: replicas,
weak scaling); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from inputs import lattice as L  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
KAPPA_TABLE = os.path.join(ROOT, "tests", "golden", "kappa_c.json")
ORACLE_COUNTS = os.path.join(ROOT, "tests", "golden", "oracle_counts_16x16x16x16.json")
# FP64 ALU peak derived from unit counts and clock: 2 DFMA (4 flops) per clock
# per SM on 152 SMs at the 2070 MHz maximum SM clock = 1.2586 TFLOP/s, the
# 1.25 TFLOP/s nominal figure; a DFMA throughput probe measured 1.188 TFLOP/s
# at 1995 MHz, i.e. the same 4 flops/clk/SM.
FP64_FLOPS_PER_CLK_PER_SM = 4
SMS = 152
SM_MAX_MHZ = 2070.0

DSLASH_FLOPS_PER_SITE = 1368      # 1320 hopping + 48 for 1 - kappa*D
DSLASH_BYTES_PER_SITE = 960       # 192 in + 192 out + 4 links x 144 (FP64)
# DRAM bytes (read + write) per site update of wilson_f64_kernel from one ncu
# capture of a 10-system launch at 16^4 (383.6 + 111.4 MB / 655,360 site
# updates); the bench scales it to a launch by the site updates it processed.
DSLASH_DRAM_BYTES_PER_SITE_UPDATE = 495.0e6 / 655360
METRIC = "D-BiCGStab solves/s at rel. residual 1e-10; dslash GB/s vs HBM roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="wilson_16x16x16x16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-growth", action="store_true",
                    help="skip the growth-row blocks (20^3x32 mixed, 24^3x48 shifts, 32^3x64 "
                         "forward+backward) of the default line")
    ap.add_argument("--storage", type=int, default=32, choices=[32, 16],
                    help="Krylov vector storage of the mixed workloads")
    ap.add_argument("--mixed-delta", type=float, default=None,
                    help="mixed solver: 0 = reliable updates every 50 iterations, delta in "
                         "(0, 1) = restarted refinement (default: 0 for the mixed Wilson "
                         "workload, 1e-3 for the twisted-mass shifts)")
    ap.add_argument("--mus", type=float, nargs="*", default=None,
                    help="twisted-mass shifts (default: the preset's)")
    ap.add_argument("--even-odd", action="store_true",
                    help="run the Wilson workload on the even-odd Schur system (Sec. 3)")
    ap.add_argument("--no-eo-variant", action="store_true",
                    help="skip the even-odd variant reported beside the default line")
    return ap.parse_args()


def load_json(path, default=None):
    if not os.path.exists(path):
        return default
    with open(path) as f:
        return json.load(f)


def kappa_for(cfg):
    table = load_json(KAPPA_TABLE, {})
    if cfg.name not in table:
        raise SystemExit(f"kappa_c of {cfg.name} missing: run tests/golden/make_kappa_c.py")
    return cfg.kappa_factor * table[cfg.name]["kappa_c"]


def rank_sources(cfg, rank, count):
    """Right-hand sides of this rank: independent seeds per rank."""
    out = []
    for j in range(count):
        seed = L.rhs_seed(cfg, j) + 100000 * rank
        if cfg.rhs_kind == "z4":
            out.append(L.z4_spinor(cfg.dims, seed))
        else:
            out.append(L.gaussian_spinor(cfg.dims, seed))
    return np.stack(out)


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest `value` over all ranks (the step time of the slowest GPU);
    the identity on one process."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("WD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle timing
#
# The oracle is timed on slices of its own step.  The step (the oracle's run
# of the workload, tests/golden/oracle_counts_*.json) is the Arnoldi sequence
# of GMRES-DR (j = 0..m-1 in the first cycle, j = k..m-1 in every later one:
# 400 Arnoldi+CGS2 steps at 16^4) and the BiCGStab iterations of the
# D-BiCGStab sources (2800 at 16^4).  Slice s of that step is one Arnoldi
# step at the j of the sequence position s and (iterations / sequence length)
# BiCGStab iterations, i.e. exactly 1/len(sequence) of the step, counted in
# solves as n_rhs / len(sequence).  The restart products, the deflation setup
# and the per-source projections (a few per cent of the oracle's step) are not
# in the slices.  Workers are spawned processes with one BLAS thread each,
# every one on its own source; a barrier before each slice makes the slices of
# all workers run together, and the wall time of a slice round is the time of
# the slowest worker.

THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def host_cores(bytes_per_worker=0):
    """Cores this process may use, capped so that `bytes_per_worker` each fit
    in half of the host's memory."""
    try:
        c = len(os.sched_getaffinity(0))
    except AttributeError:
        c = os.cpu_count() or 1
    if bytes_per_worker:
        try:
            mem = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
            c = max(1, min(c, int(mem // 2 // bytes_per_worker)))
        except (ValueError, OSError):
            pass
    return c


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(l.split(":", 1) for l in out.splitlines() if ":" in l)
        name = fields.get("Model name", "").strip()
        vendor = fields.get("Vendor ID", "").strip()
        if name:
            return f"{vendor} {name}".strip()
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    import platform
    return platform.processor() or platform.machine()


def slice_plan(cfg, counts):
    """(Arnoldi j sequence, BiCGStab iterations per slice) of the oracle's step."""
    js = list(range(cfg.m)) + list(range(cfg.k, cfg.m)) * (counts["gmresdr_cycles"] - 1)
    iters = sum(counts["dbicgstab_iters"])
    return js, max(1, round(iters / len(js)))


def worker_bytes(cfg):
    """Host memory of one slice worker: the Arnoldi basis plus a few vectors."""
    return (cfg.m + 12) * 12 * L.volume(cfg.dims) * 16


def spread_positions(count, total, offset=0.5):
    """`count` positions spread evenly over a sequence of length `total`."""
    return [min(total - 1, int((i + offset) * total / count)) for i in range(count)]


def _slice_worker(cfg_name, kappa, worker, js, bicg_per_slice, barrier, q):
    from oracle import dirac, krylov
    cfg = L.CONFIGS[cfg_name]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    A = lambda x: dirac.apply_A(U, x.reshape(v, 4, 3), cfg.dims, kappa).ravel()
    b = L.source(cfg, 1 + worker % cfg.n_rhs).ravel()
    n = b.size
    jmax = max(js)
    # an orthonormal-looking basis for the Gram-Schmidt passes (values do not
    # change the oracle's cost): shifted copies of the normalised source
    Vb = np.empty((jmax + 2, n), dtype=np.complex128)
    bn = b / np.linalg.norm(b)
    for i in range(jmax + 2):
        Vb[i] = np.roll(bn, 12 * i)
    times = []
    for j in js:
        barrier.wait()
        t = time.perf_counter()
        w = A(Vb[j])                         # Arnoldi step at j, CGS2 as the oracle's gmresdr
        h = Vb[: j + 1].conj() @ w
        w = w - Vb[: j + 1].T @ h
        h2 = Vb[: j + 1].conj() @ w
        w = w - Vb[: j + 1].T @ h2
        _ = np.sqrt(np.vdot(w, w).real)
        krylov.bicgstab(A, b, tol=1e-300, max_iter=bicg_per_slice, max_restarts=0)
        times.append(time.perf_counter() - t)
    q.put((worker, times))


def oracle_slices(cfg, kappa, counts, workers, positions):
    """Run the slices at `positions` of the oracle's step on `workers`
    concurrent processes.  Returns (wall seconds per slice round, details)."""
    js_all, bicg = slice_plan(cfg, counts)
    js = [js_all[p] for p in positions]
    saved = {var: os.environ.get(var) for var in THREAD_VARS}
    for var in THREAD_VARS:
        os.environ[var] = "1"
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        barrier = ctx.Barrier(workers, timeout=600)
        procs = [ctx.Process(target=_slice_worker,
                             args=(cfg.name, kappa, w, js, bicg, barrier, q))
                 for w in range(workers)]
        for p in procs:
            p.start()
        try:
            res = dict(q.get(timeout=1800) for _ in procs)
        finally:
            for p in procs:
                p.join(timeout=60)
                if p.is_alive():
                    p.terminate()
    finally:
        for var, val in saved.items():
            if val is None:
                os.environ.pop(var, None)
            else:
                os.environ[var] = val
    rounds = [max(res[w][i] for w in range(workers)) for i in range(len(js))]
    return rounds, {"js": js, "bicgstab_iters_per_slice": bicg,
                    "slices_per_step": len(js_all)}


def cpu_baseline_line(cfg, kappa, counts, slices=4):
    """The oracle on one host core and on all of them, `slices` slice rounds
    each (tens of seconds in all); solves/s of the workload."""
    js_all, bicg = slice_plan(cfg, counts)
    per_slice = cfg.n_rhs / len(js_all)
    pos = spread_positions(slices, len(js_all))
    r1, _ = oracle_slices(cfg, kappa, counts, 1, pos)
    cores = host_cores(worker_bytes(cfg))
    rp, _ = oracle_slices(cfg, kappa, counts, cores, pos)
    v1 = per_slice * len(r1) / sum(r1)
    vp = cores * per_slice * len(rp) / sum(rp)
    return {
        "value": round(vp, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
        "value_1_core": round(v1, 6), "cpu_model": cpu_model(), "nproc": os.cpu_count(),
        "sample": (f"the oracle (numpy FP64, 1 BLAS thread per process) on {slices} slices of its "
                   f"own {cfg.name} step, in 1 process ({sum(r1):.1f} s) and in {cores} concurrent "
                   f"processes, one source each ({sum(rp):.1f} s); a slice is 1/{len(js_all)} of "
                   f"the step: one Arnoldi+CGS2 step (j spread over the step's GMRES-DR "
                   f"sequence) and {bicg} BiCGStab iterations (the step's "
                   f"{sum(counts['dbicgstab_iters'])} / {len(js_all)}); restart products, "
                   f"deflation setup and projections left out"),
    }


# ------------------------------------------------------------------ GPU arm

def gpu_arm(args, cfg, rank, world, local_rank):
    import torch
    import paper_0710_1988_gb300 as wdl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    n = 12 * v
    src = rank_sources(cfg, rank, cfg.n_rhs + 1)
    b0 = torch.from_numpy(src[0].ravel()).to(dev)
    B = torch.from_numpy(src[1:].reshape(cfg.n_rhs, n)).to(dev)
    x0 = torch.zeros_like(b0)
    X = torch.zeros_like(B)
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device=dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step(b0_, x0_, B_, X_):
        x0_.zero_() if hasattr(x0_, "zero_") else x0_.fill(0)
        X_.zero_() if hasattr(X_, "zero_") else X_.fill(0)
        rc, st, _, theta = op.gmresdr(b0_, x0_, cfg.m, cfg.k, cfg.tol, 400000, V_out=V)
        defl = op.deflation(V, cfg.k)
        rc2, sts = op.dbicgstab(B_, X_, defl, tol=cfg.tol)
        defl.close()
        if rc != 0 or rc2 != 0 or not all(s["converged"] for s in sts):
            raise RuntimeError(f"solve did not converge: gmresdr rc={rc}, dbicgstab rc={rc2}")
        return st, sts, theta

    for _ in range(args.warmup):
        step(b0, x0, B, X)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs, dslash launches timed live
    clocks = ClockSampler(local_rank)
    clocks.start()
    op.profile(mask=0x1)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms_steps, last = [], None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step(b0, x0, B, X)
        e1.record(stream)
        e1.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    prof_live = op.profile_read()
    op.profile(mask=0)
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(ms_steps), dev)

    # ---- one more step with every kernel category timed: the breakdown
    op.profile(mask=0xF)
    step(b0, x0, B, X)
    prof_all = op.profile_read()
    op.profile(mask=0)

    # ---- the D-BiCGStab part alone, FP64 and mixed precision (same V, same B)
    mixed = None
    if not args.no_mixed:
        rc, st0, _, _ = op.gmresdr(b0, x0.zero_(), cfg.m, cfg.k, cfg.tol, 400000, V_out=V)
        defl = op.deflation(V, cfg.k)
        res = {}
        undeflated = lambda B_, X_, d_, tol: op.dbicgstab(B_, X_, None, tol=tol)
        for name, fn, bits in (("fp64", op.dbicgstab, 32), ("mixed", op.dbicgstab_mixed, 32),
                               ("mixed16", op.dbicgstab_mixed, 16),
                               ("fp64_undeflated", undeflated, 32)):
            op.set_mixed_storage(bits)
            X.zero_()
            fn(B, X, defl, tol=cfg.tol)            # warm
            ts = []
            for _ in range(2):
                X.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rc, ss = fn(B, X, defl, tol=cfg.tol)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
                if rc != 0 or not all(q["converged"] for q in ss):
                    raise RuntimeError(f"{name} D-BiCGStab did not converge")
            res[name] = (min(ts), ss)
        defl.close()
        op.set_mixed_storage(32)
        mixed = {
            "what": "solves/s as the workload defines it: D-BiCGStab(k) on the step's sources "
                    "after V and G are set up (the step's V), projection included; FP64 and the "
                    "mixed forms",
            "fp64_solves_per_s": round(cfg.n_rhs / (res["fp64"][0] * 1e-3), 3),
            "mixed_solves_per_s": round(cfg.n_rhs / (res["mixed"][0] * 1e-3), 3),
            "speedup": round(res["fp64"][0] / res["mixed"][0], 3),
            "fp64_iters": [q["iters"] for q in res["fp64"][1]],
            "mixed_iters": [q["iters"] for q in res["mixed"][1]],
            "mixed_max_true_rel_res": max(q["true_rel_res"] for q in res["mixed"][1]),
            "mixed16_solves_per_s": round(cfg.n_rhs / (res["mixed16"][0] * 1e-3), 3),
            "speedup16": round(res["fp64"][0] / res["mixed16"][0], 3),
            "mixed16_iters": [q["iters"] for q in res["mixed16"][1]],
            "mixed16_max_true_rel_res": max(q["true_rel_res"] for q in res["mixed16"][1]),
            "storage": {"mixed": "FP32 vectors and links", "mixed16": "FP16 p, v, t and links "
                        "(per-site norm), FP32 r, r_hat, x increment"},
            "reliable_every": 50,
        }
        mixed["sec2_deflation"] = {
            "what": "plain BiCGStab (FP64, no projection) on the same sources: the MVPs the "
                    "projection of Sec. 2 saves on this field",
            "fp64_undeflated_solves_per_s": round(cfg.n_rhs / (res["fp64_undeflated"][0] * 1e-3), 3),
            "mvp_deflated": [q["mvp"] for q in res["fp64"][1]],
            "mvp_undeflated": [q["mvp"] for q in res["fp64_undeflated"][1]],
        }

    gst, sts, theta = last
    th = np.sort(np.abs(np.asarray(theta)))
    counts = {"gmresdr_mvp": gst["mvp"], "gmresdr_cycles": gst["cycles"],
              "dbicgstab_mvp": [s["mvp"] for s in sts],
              "dbicgstab_iters": [s["iters"] for s in sts],
              "true_rel_res_max": max(s["true_rel_res"] for s in sts),
              "gmresdr_true_rel_res": gst["true_rel_res"],
              "harmonic_ritz_abs": {"min": float(th[0]), "median": float(th[len(th) // 2]),
                                    "max": float(th[-1])}}

    # ---- e2e: the same step through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        b0h = pin(src[0].ravel().copy())
        Bh = pin(src[1:].reshape(cfg.n_rhs, n).copy())
        x0h = pin(np.zeros(n, dtype=np.complex128))
        Xh = pin(np.zeros((cfg.n_rhs, n), dtype=np.complex128))
        step(b0h, x0h, Bh, Xh)  # warm the staging buffers
        if world > 1:
            torch.distributed.barrier()
        wall = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            step(b0h, x0h, Bh, Xh)
            torch.cuda.synchronize()
            wall.append(time.perf_counter() - t)
        tot = max_over_ranks(sum(wall), dev)
        h2d = (2 + 2 * cfg.n_rhs) * n * 16      # b0, x0, B, X0 staged in
        d2h = (1 + cfg.n_rhs) * n * 16          # x and X copied back
        e2e = {"value": cfg.n_rhs * args.steps * world / tot, "unit": "solves/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1000 * tot / args.steps}
    op.close()
    return {"total_ms": total_ms, "ms_steps": ms_steps, "prof_live": prof_live, "mixed": mixed,
            "prof_all": prof_all, "counts": counts, "clocks": clk, "e2e": e2e,
            "kappa": kappa, "n": n, "volume": v}


def measured_fp64_peak(local_rank, iters=1 << 15, reps=20):
    """FP64 FMA throughput measured live by the library's probe kernel
    (wd_probe_fp64_peak, CUDA events), with the SM clock sampled while it
    runs; the derived figure (unit count x clock) is kept beside it."""
    import paper_0710_1988_gb300 as wdl
    derived = FP64_FLOPS_PER_CLK_PER_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
    wdl.probe_fp64_peak(iters=iters, reps=2)             # warm
    clocks = ClockSampler(local_rank)
    clocks.start()
    tf, ms = wdl.probe_fp64_peak(iters=iters, reps=reps)
    clk = clocks.stop()
    return {"tflops": round(tf, 4), "ms_per_launch": round(ms, 3), "clocks": clk,
            "derived_tflops": round(derived, 4),
            "source": (f"measured live: wd_probe_fp64_peak (8 independent DFMA chains per "
                       f"thread, 4 x 256 threads per SM, {reps} launches of {ms:.1f} ms, CUDA "
                       f"events) at a median SM clock of {clk.get('sm_mhz')} MHz; "
                       f"profiles/fp64_peak_probe.md"),
            "derived_source": "4 FP64 flops/clk/SM x 152 SMs x 2070 MHz (= nominal 1.25 TFLOP/s)"}


def roofline(res, peaks, fp64_peak):
    live = res["prof_live"]
    launches = live["dslash"]["launches"]
    ms = live["dslash"]["ms"]
    sites = live["dslash_site_updates"]
    avg_ms = ms / max(1, launches)
    sites_per_launch = sites / max(1, launches)
    flops = DSLASH_FLOPS_PER_SITE * sites_per_launch
    tflops = flops / (avg_ms * 1e-3) / 1e12
    gbs = DSLASH_BYTES_PER_SITE * sites_per_launch / (avg_ms * 1e-3) / 1e9
    out = {
        "kernel": "wilson_f64_kernel (FP64 dslash)",
        "bound": "alu",
        "achieved": round(tflops, 4),
        "peak": fp64_peak["tflops"],
        "unit": "TFLOP/s",
        "frac": round(tflops / fp64_peak["tflops"], 4),
        "peak_source": fp64_peak["source"],
        "peak_derived": fp64_peak["derived_tflops"],
        "frac_of_derived": round(tflops / fp64_peak["derived_tflops"], 4),
        "peak_derived_source": fp64_peak["derived_source"],
        "traffic": round(DSLASH_DRAM_BYTES_PER_SITE_UPDATE * sites_per_launch),
        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 16^4 "
                          "10-system launch (755 B per site update), scaled to the average "
                          "launch by site updates",
        "algorithmic_flops_per_launch": flops,
        "avg_launch_ms": avg_ms,
        "launches": launches,
        "hbm_view": {"achieved_gbs": round(gbs, 1), "peak_gbs": peaks.get("hbm_gbs"),
                     "frac": round(gbs / peaks["hbm_gbs"], 4) if peaks.get("hbm_gbs") else None,
                     "algorithmic_bytes_per_launch": DSLASH_BYTES_PER_SITE * sites_per_launch},
    }
    return out


def headline_config(cfg, kappa, world):
    """The `config` of the headline line; the reference arm prints the same."""
    return {
        "workload": f"{cfg.name}: GMRES-DR({cfg.m},{cfg.k}) on 1 Z4 source + D-BiCGStab({cfg.k}) "
                    f"on {cfg.n_rhs} Z4 sources, tol {cfg.tol:g}, kappa = {cfg.kappa_factor} kappa_c",
        "lattice": list(cfg.dims), "kappa": kappa, "m": cfg.m, "k": cfg.k,
        "rhs_per_step": cfg.n_rhs, "parallelism": f"replicas x{world}",
        "l2": "256 MB L2 flush before every step; step working set (1.0 GB Krylov basis, "
              "0.9 GB BiCGStab batch) exceeds the 129 MB L2",
    }


def main():
    args = parse()
    cfg = L.CONFIGS[args.config]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, cfg, rank, world)

    import torch
    if world > 1:
        torch.distributed.init_process_group(backend="nccl")
    kind = workload_kind(cfg)
    if kind == "fp64" and args.even_odd:
        kind = "evenodd"
    if kind != "fp64":
        line = ROW_ARMS[kind](args, cfg, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    res = gpu_arm(args, cfg, rank, world, local_rank)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks = load_json(MEASURED_PEAKS, {}) or {}
    fp64_peak = measured_fp64_peak(local_rank)
    steps = args.steps
    value = cfg.n_rhs * steps * world / (res["total_ms"] * 1e-3)
    line = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": round(res["total_ms"] / steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic: SU(3) links exp(i*0.5*H) (seed 1001), Z4 sources; no dataset",
        "config": headline_config(cfg, res["kappa"], world),
        "gpu_launches": None,
        "roofline": roofline(res, peaks, fp64_peak),
        "clocks": res["clocks"],
        "e2e": res["e2e"],
        "counts": res["counts"],
        "dbicgstab_after_setup": res["mixed"],
        "kernel_breakdown_ms": {k: v for k, v in res["prof_all"].items() if isinstance(v, dict)},
    }
    pa = res["prof_all"]
    line["gpu_launches"] = int(sum(pa[c]["launches"] for c in ("dslash", "stream", "tall_skinny", "dense")) * steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = load_json(ORACLE_COUNTS)
        if counts is not None:
            line["cpu_baseline"] = cpu_baseline_line(cfg, res["kappa"], counts)
    if world == 1 and not args.no_eo_variant:
        # the same workload on the even-odd Schur system (the paper's system),
        # 1 warm-up and 1 timed step, reported beside the headline
        eo = evenodd_arm(argparse.Namespace(steps=1, warmup=1), cfg, rank, world, local_rank)
        line["even_odd_variant"] = {"value": eo["value"], "unit": eo["unit"],
                                    "ms_per_step": eo["ms_per_step"], "counts": eo["counts"],
                                    "dbicgstab_alone": eo["dbicgstab_alone"],
                                    "what": "same sources and tolerance, Schur complement on even "
                                            "sites, solutions reconstructed on the full lattice"}
    if world == 1 and not args.no_growth and cfg.name == "wilson_16x16x16x16":
        line["growth_rows"] = growth_rows(local_rank, peaks, fp64_peak)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ the other workloads
#
# The default workload above is the benchmark line.  The presets below are the
# workloads of the growth rows (mixed precision at 20^3x32, twisted-mass
# shifts at 24^3x48, differentiation at 32^3x64); `--config <preset>` runs one
# of them with the same timing rules (warm-up steps, L2 flush, CUDA events on
# the launching stream, clocks sampled, max over ranks) and prints its own
# JSON line.

# FP32 / FP16 bytes per site and system of the mixed solver's kernels
LOW_DSLASH_BYTES = {32: 3 * 96, 16: 52 + 52 + 96}   # in + out + (r_hat or r) per site update
LOW_LINK_BYTES = {32: 4 * 48, 16: 4 * 24}            # links (rows 0, 1), read once per launch
# even-odd Schur apply (FP32), per even site and system: v = A_hat p moves
# SCHUR1 in + tmp and SCHUR2 tmp + p + out + r_hat; t = A_hat (r - alpha v) moves
# SCHUR1 r + v + tmp and SCHUR2 tmp + r + v + out; the mean of the two applies
LOW_SCHUR_BYTES = {32: (2 * 96 + 4 * 96 + 3 * 96 + 4 * 96) / 2}
LOW_UPDATE_BYTES = {32: 4 * 96 + 8 * 96,             # p = r + beta (p - omega v); x, r update
                    16: (96 + 3 * 52) + (4 * 96 + 3 * 52 + 2 * 96)}


def workload_kind(cfg):
    if cfg.mus:
        return "twisted"
    if cfg.name.startswith("grad_"):
        return "grad"
    if cfg.name.endswith("_mixed"):
        return "mixed"
    return "fp64"


def timed_steps(args, step, op, flush, stream, world, dev, prof_mask=0):
    """W warm-up steps, then K steps timed with CUDA events on `stream` (L2
    flushed before each), clocks sampled; returns per-step ms, the last
    step's result, the profile of the timed region and the clock summary."""
    import torch
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    op.profile(mask=prof_mask)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms_steps, last = [], None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step()
        e1.record(stream)
        e1.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    prof = op.profile_read()
    op.profile(mask=0)
    return ms_steps, last, prof, clocks.stop()


def low_rooflines(prof, bits, V, peaks, iters_total, eo=False):
    """HBM rooflines of the mixed solver's FP32/FP16 kernels from a profiled
    step: the Wilson apply (site updates counted on the device) and the two
    per-iteration vector updates (one pass of each per system iteration).
    On the even-odd Schur system (eo) one profiled launch is a Schur apply: two
    half-lattice hop kernels, each reading every link, with V/2 counted site
    updates per system (LOW_SCHUR_BYTES each); the vector updates run over V/2
    sites."""
    hbm = peaks.get("hbm_gbs")
    out = {}
    d = prof["dslash_low"]
    if d["launches"]:
        if eo:
            byt = (LOW_SCHUR_BYTES[bits] * prof["dslash_low_site_updates"]
                   + 2 * LOW_LINK_BYTES[bits] * V * d["launches"])
        else:
            byt = (LOW_DSLASH_BYTES[bits] * prof["dslash_low_site_updates"]
                   + LOW_LINK_BYTES[bits] * V * d["launches"])
        gbs = byt / (d["ms"] * 1e-3) / 1e9
        name = "wilson_eo32_kernel x2 (one Schur apply)" if eo else f"wilson_f{bits}_kernel"
        out["dslash"] = {"kernel": name, "bound": "hbm", "achieved": round(gbs, 1),
                         "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4) if hbm else None,
                         "traffic": None, "avg_launch_ms": d["ms"] / d["launches"],
                         "launches": d["launches"],
                         "algorithmic_bytes_per_launch": byt / d["launches"]}
    u = prof["stream_low"]
    if u["launches"]:
        byt = LOW_UPDATE_BYTES[bits] * (V // 2 if eo else V) * iters_total
        gbs = byt / (u["ms"] * 1e-3) / 1e9
        out["updates"] = {"kernel": f"bicg{bits}_update_p + bicg{bits}_update_xr", "bound": "hbm",
                          "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                          "frac": round(gbs / hbm, 4) if hbm else None, "traffic": None,
                          "avg_launch_ms": u["ms"] / u["launches"], "launches": u["launches"],
                          "algorithmic_bytes_per_launch": byt / u["launches"]}
    return out


def _row_line(cfg, args, world, value, unit, total_ms, dtype, workload, extra):
    line = {"metric": METRIC if unit == "solves/s" else f"{unit} at rel. residual {cfg.tol:g}",
            "value": round(value, 4), "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": f"synthetic: SU(3) links exp(i*{cfg.eps}*H) (seed {L.link_seed(cfg)}), "
                    f"{cfg.rhs_kind} sources; no dataset",
            "config": {"workload": workload, "lattice": list(cfg.dims),
                       "parallelism": f"replicas x{world}",
                       "l2": "256 MB L2 flush before every step; vectors exceed the 129 MB L2"}}
    line.update(extra)
    return line


def mixed_arm(args, cfg, rank, world, local_rank):
    """20^3x32: GMRES-DR(80,60) (FP64) on one Z4 source, then D-BiCGStab(60)
    with the FP32 (or FP16) iteration and FP64 reliable updates every 50
    iterations on 12 Z4 sources, all to 1e-10 true residual."""
    import torch
    import paper_0710_1988_gb300 as wdl
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    n = 12 * v
    src = rank_sources(cfg, rank, cfg.n_rhs + 1)
    b0 = torch.from_numpy(src[0].ravel()).to(dev)
    B = torch.from_numpy(src[1:].reshape(cfg.n_rhs, n)).to(dev)
    x0 = torch.zeros_like(b0)
    X = torch.zeros_like(B)
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device=dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    op.set_mixed_storage(args.storage)
    delta = 0.0 if args.mixed_delta is None else args.mixed_delta
    op.set_mixed_restart(delta, 300)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        x0.zero_()
        X.zero_()
        rc, st, _, _ = op.gmresdr(b0, x0, cfg.m, cfg.k, cfg.tol, 400000, V_out=V)
        defl = op.deflation(V, cfg.k)
        rc2, sts = op.dbicgstab_mixed(B, X, defl, tol=cfg.tol, reliable_every=50)
        defl.close()
        if rc != 0 or rc2 != 0 or not all(q["converged"] for q in sts):
            raise RuntimeError(f"solve did not converge: gmresdr rc={rc}, mixed rc={rc2}")
        return st, sts

    ms_steps, last, _, clk = timed_steps(args, step, op, flush, stream, world, dev)
    total_ms = max_over_ranks(sum(ms_steps), dev)
    st, sts = last
    # one profiled step (graphs off while profiling): breakdown and rooflines
    op.profile(mask=0x3F)
    st_p, sts_p = step()
    prof = op.profile_read()
    op.profile(mask=0)
    peaks = load_json(MEASURED_PEAKS, {}) or {}
    roof = low_rooflines(prof, args.storage, v, peaks, sum(q["iters"] for q in sts_p))
    # D-BiCGStab alone: FP64 against FP32 and FP16 storage, same V and sources
    defl = op.deflation(V, cfg.k)
    comp = {}
    for name, bits, dl in (("fp64", None, 0.0), ("mixed32", 32, 0.0), ("mixed16", 16, 0.0),
                           ("mixed32_restarted", 32, 1e-3), ("mixed16_restarted", 16, 1e-3)):
        if bits:
            op.set_mixed_storage(bits)
            op.set_mixed_restart(dl, 300)
        fn = op.dbicgstab if bits is None else (
            lambda B_, X_, d_, tol: op.dbicgstab_mixed(B_, X_, d_, tol=tol, reliable_every=50))
        X.zero_()
        fn(B, X, defl, tol=cfg.tol)
        X.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, ss = fn(B, X, defl, tol=cfg.tol)
        e1.record(stream)
        e1.synchronize()
        if rc != 0 or not all(q["converged"] for q in ss):
            raise RuntimeError(f"{name} D-BiCGStab did not converge")
        comp[name] = {"solves_per_s": round(cfg.n_rhs / (e0.elapsed_time(e1) * 1e-3), 3),
                      "iters": [q["iters"] for q in ss],
                      "max_true_rel_res": max(q["true_rel_res"] for q in ss)}
    defl.close()
    op.set_mixed_storage(args.storage)
    op.set_mixed_restart(delta, 300)
    for name in comp:
        if name != "fp64":
            comp[name]["speedup_vs_fp64"] = round(comp[name]["solves_per_s"] / comp["fp64"]["solves_per_s"], 3)
    comp["strategies"] = {"mixed32/16": "reliable updates every 50 iterations",
                          "*_restarted": "restarted refinement, delta = 1e-3, a restart at least every 300 iterations"}
    op.close()
    extra = {
        "gpu_launches": None,
        "roofline": roof.get("updates"),
        "roofline_dslash": roof.get("dslash"),
        "clocks": clk,
        "e2e": None,
        "counts": {"gmresdr_mvp": st["mvp"], "gmresdr_cycles": st["cycles"],
                   "dbicgstab_iters": [q["iters"] for q in sts],
                   "true_rel_res_max": max(q["true_rel_res"] for q in sts)},
        "dbicgstab_alone": comp,
        "kernel_breakdown_ms": {k: v_ for k, v_ in prof.items() if isinstance(v_, dict)},
    }
    extra["gpu_launches"] = int(sum(c["launches"] for c in extra["kernel_breakdown_ms"].values()))
    return _row_line(cfg, args, world, cfg.n_rhs * args.steps * world / (total_ms * 1e-3),
                     "solves/s", total_ms, f"f{args.storage} iteration, f64 reliable updates",
                     f"{cfg.name}: GMRES-DR({cfg.m},{cfg.k}) FP64 on 1 Z4 source + D-BiCGStab("
                     f"{cfg.k}) mixed (FP{args.storage} storage, "
                     + ("FP64 reliable updates every 50" if delta == 0 else
                        f"restarted refinement delta {delta:g}, max 300 iterations per pass") + ") "
                     f"on {cfg.n_rhs} Z4 sources, tol {cfg.tol:g}, kappa = {cfg.kappa_factor} kappa_c",
                     extra)


def twisted_arm(args, cfg, rank, world, local_rank):
    """24^3x48 twisted mass at kappa_c: the Sec. 4 shifts heaviest first, each
    projected over the earlier solutions, 16 Gaussian sources per shift in one
    batch, mixed-precision BiCGStab."""
    import torch
    import paper_0710_1988_gb300 as wdl
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    n = 12 * v
    mus = sorted(args.mus if args.mus else cfg.mus, reverse=True)
    B = torch.from_numpy(rank_sources(cfg, rank, cfg.n_rhs).reshape(cfg.n_rhs, n)).to(dev)
    X = torch.zeros(len(mus) * cfg.n_rhs * n, dtype=torch.complex128, device=dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    op.set_mixed_storage(args.storage)
    if args.even_odd:  # each shift through its Schur system (Sec. 4 with even-odd)
        op.set_operator(True)
    delta = 1e-3 if args.mixed_delta is None else args.mixed_delta
    op.set_mixed_restart(delta, 300)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run(project):
        X.zero_()
        rc, sts = op.multishift(B, X, mus, tol=cfg.tol, project=project, mixed=True)
        if rc != 0 or not all(q["converged"] for row in sts for q in row):
            raise RuntimeError(f"twisted-mass shifts did not converge (status {rc})")
        return sts

    ms_steps, sts, _, clk = timed_steps(args, lambda: run(True), op, flush, stream, world, dev)
    total_ms = max_over_ranks(sum(ms_steps), dev)
    op.profile(mask=0x3F)
    sts_p = run(True)
    prof = op.profile_read()
    op.profile(mask=0)
    peaks = load_json(MEASURED_PEAKS, {}) or {}
    roof = low_rooflines(prof, args.storage, v, peaks, sum(q["iters"] for row in sts_p for q in row),
                         eo=args.even_odd)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sts_np = run(False)
    e1.record(stream)
    e1.synchronize()
    op.close()
    per_shift = []
    for i, mu in enumerate(mus):
        per_shift.append({"mu": mu,
                          "mvp_projected": [q["mvp"] + q["mvp_extra"] for q in sts[i]],
                          "mvp_unprojected": [q["mvp"] + q["mvp_extra"] for q in sts_np[i]],
                          "max_true_rel_res": max(q["true_rel_res"] for q in sts[i])})
    units = cfg.n_rhs * len(mus)
    extra = {
        "gpu_launches": None,
        "roofline": roof.get("updates"),
        "roofline_dslash": roof.get("dslash"),
        "clocks": clk,
        "e2e": None,
        "shifts": per_shift,
        "unprojected_solves_per_s": round(units / (e0.elapsed_time(e1) * 1e-3), 3),
        "kernel_breakdown_ms": {k: v_ for k, v_ in prof.items() if isinstance(v_, dict)},
    }
    extra["gpu_launches"] = int(sum(c["launches"] for c in extra["kernel_breakdown_ms"].values()))
    return _row_line(cfg, args, world, units * args.steps * world / (total_ms * 1e-3), "solves/s",
                     total_ms, f"f{args.storage} iteration, f64 reliable updates",
                     f"{cfg.name}: A_W + i mu gamma5 at kappa_c"
                     + (" on the even-odd Schur system" if args.even_odd else "")
                     + f", shifts {mus} heaviest first, each "
                     f"projected over the earlier solutions (Sec. 4), {cfg.n_rhs} Gaussian sources "
                     f"per shift batched, mixed BiCGStab (FP{args.storage}, "
                     + ("reliable updates every 50" if delta == 0 else
                        f"restarted refinement delta {delta:g}, max 300 iterations per pass")
                     + f") to {cfg.tol:g}; value counts (source, shift) pairs", extra)


def grad_arm(args, cfg, rank, world, local_rank):
    """Differentiation: x = A^-1 b forward (FP64 BiCGStab) and the backward of
    L = Re(eta^dagger x) through the autograd Function (adjoint solve via
    gamma5, dL/db, dL/dkappa and the link force), 1e-10."""
    import torch
    import paper_0710_1988_gb300 as wdl
    from paper_0710_1988_gb300.autograd import wilson_solve
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    src = rank_sources(cfg, rank, 2)
    b = torch.from_numpy(src[0].ravel()).to(dev)
    eta = torch.from_numpy(src[1].ravel()).to(dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(mixed=False):
        bt = b.clone().requires_grad_(True)
        kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
        om = torch.zeros((v, 4, 8), dtype=torch.float64, device=dev, requires_grad=True)
        x = wilson_solve(bt, kt, om, op, None, cfg.tol, mixed=mixed)
        loss = (eta.conj() * x).sum().real
        loss.backward()
        return float(kt.grad), float(om.grad.abs().max())

    ms_steps, last, prof_live, clk = timed_steps(args, step, op, flush, stream, world, dev,
                                                 prof_mask=0x1)
    total_ms = max_over_ranks(sum(ms_steps), dev)
    op.profile(mask=0x3F)
    step()
    prof = op.profile_read()
    op.profile(mask=0)
    # the same forward + backward with both solves in mixed precision (FP32
    # iteration, restarted refinement, FP64 true residual <= tol)
    op.set_mixed_restart(1e-3, 300)
    ms_mixed, last_m, _, _ = timed_steps(args, lambda: step(True), op, flush, stream, world, dev)
    mixed_ms = max_over_ranks(sum(ms_mixed), dev)
    op.close()
    peaks = load_json(MEASURED_PEAKS, {}) or {}
    fp64_peak = measured_fp64_peak(local_rank)
    r = roofline({"prof_live": prof_live}, peaks, fp64_peak)
    r["traffic"] = None
    r.pop("traffic_source", None)
    extra = {"gpu_launches": int(sum(c["launches"] for c in prof.values() if isinstance(c, dict))),
             "roofline": r, "clocks": clk, "e2e": None,
             "dkappa": last[0], "max_abs_force": last[1],
             "mixed_fp32": {"value": round(args.steps * world / (mixed_ms * 1e-3), 4),
                            "unit": "fwd+bwd solves/s",
                            "ms_per_step": round(mixed_ms / args.steps, 3),
                            "dkappa": last_m[0], "max_abs_force": last_m[1],
                            "what": "forward and adjoint solves with the FP32 iteration and "
                                    "restarted refinement (delta 1e-3), gradients in FP64"},
             "kernel_breakdown_ms": {k: v_ for k, v_ in prof.items() if isinstance(v_, dict)}}
    return _row_line(cfg, args, world, args.steps * world / (total_ms * 1e-3),
                     "fwd+bwd solves/s", total_ms, "f64",
                     f"{cfg.name}: x = A^-1 b (BiCGStab) and the backward of Re(eta^dagger x) "
                     f"(adjoint solve via gamma5, dL/db, dL/dkappa, link force), tol {cfg.tol:g}, "
                     f"kappa = {cfg.kappa_factor} kappa_c", extra)


def evenodd_arm(args, cfg, rank, world, local_rank):
    """The Wilson workload on the even-odd Schur complement (the paper's
    system, Sec. 3): b_hat = prepared sources, GMRES-DR(m,k) and D-BiCGStab(k)
    on even-site half vectors, solutions reconstructed on the full lattice."""
    import torch
    import paper_0710_1988_gb300 as wdl
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    n, nh = 12 * v, 6 * v
    src = rank_sources(cfg, rank, cfg.n_rhs + 1)
    b0 = torch.from_numpy(src[0].ravel()).to(dev)
    B = torch.from_numpy(src[1:].reshape(cfg.n_rhs, n)).to(dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    op.set_operator(True)
    bh0 = torch.empty(nh, dtype=torch.complex128, device=dev)
    Bh = torch.empty(cfg.n_rhs * nh, dtype=torch.complex128, device=dev)
    xe0 = torch.zeros(nh, dtype=torch.complex128, device=dev)
    Xe = torch.zeros(cfg.n_rhs * nh, dtype=torch.complex128, device=dev)
    X = torch.empty(cfg.n_rhs * n, dtype=torch.complex128, device=dev)
    V = torch.zeros(cfg.k * nh, dtype=torch.complex128, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        xe0.zero_()
        Xe.zero_()
        op.eo_prepare(b0, bh0)
        op.eo_prepare(B, Bh)
        rc, st, _, _ = op.gmresdr(bh0, xe0, cfg.m, cfg.k, cfg.tol, 400000, V_out=V)
        defl = op.deflation(V, cfg.k)
        rc2, sts = op.dbicgstab(Bh.view(cfg.n_rhs, nh), Xe, defl, tol=cfg.tol)
        defl.close()
        op.eo_reconstruct(B, Xe, X)
        if rc != 0 or rc2 != 0 or not all(q["converged"] for q in sts):
            raise RuntimeError(f"even-odd solve did not converge: gmresdr rc={rc}, dbicgstab rc={rc2}")
        return st, sts

    ms_steps, last, prof_live, clk = timed_steps(args, step, op, flush, stream, world, dev,
                                                 prof_mask=0x1)
    total_ms = max_over_ranks(sum(ms_steps), dev)
    st, sts = last
    # D-BiCGStab alone on the Schur system: FP64 against the FP32 Schur
    # iteration (restarted refinement), the step's deflation space
    defl = op.deflation(V, cfg.k)
    alone = {}
    op.set_mixed_restart(1e-3, 300)
    for name, fn in (("fp64", op.dbicgstab), ("mixed32_restarted", op.dbicgstab_mixed)):
        Xe.zero_()
        fn(Bh.view(cfg.n_rhs, nh), Xe, defl, tol=cfg.tol)   # warm
        Xe.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc_, ss = fn(Bh.view(cfg.n_rhs, nh), Xe, defl, tol=cfg.tol)
        e1.record(stream)
        e1.synchronize()
        if rc_ != 0 or not all(q["converged"] for q in ss):
            raise RuntimeError(f"{name} D-BiCGStab on the Schur system did not converge")
        alone[name] = {"solves_per_s": round(cfg.n_rhs / (e0.elapsed_time(e1) * 1e-3), 3),
                       "iters": [q["iters"] for q in ss]}
    alone["mixed32_restarted"]["speedup_vs_fp64"] = round(
        alone["mixed32_restarted"]["solves_per_s"] / alone["fp64"]["solves_per_s"], 3)
    defl.close()
    # full-system residuals of the reconstructed solutions, by the full operator
    op.set_operator(False)
    R = torch.empty_like(X)
    op.apply(X, R)
    R = B - R.view(cfg.n_rhs, n)
    full_rel = (torch.linalg.vector_norm(R, dim=1) / torch.linalg.vector_norm(B, dim=1)).max().item()
    op.close()
    extra = {"gpu_launches": None, "roofline": None, "clocks": clk, "e2e": None,
             "counts": {"gmresdr_schur_mvp": st["mvp"], "gmresdr_cycles": st["cycles"],
                        "dbicgstab_schur_mvp": [q["mvp"] for q in sts],
                        "dbicgstab_iters": [q["iters"] for q in sts],
                        "schur_true_rel_res_max": max(q["true_rel_res"] for q in sts),
                        "full_system_rel_res_max": full_rel},
             "note": "one Schur application = two half-lattice hops, the work of one full "
                     "Wilson application; tol is relative to ||b_hat||",
             "dbicgstab_alone": alone,
             "kernel_breakdown_ms": {"dslash": prof_live["dslash"]}}
    return _row_line(cfg, args, world, cfg.n_rhs * args.steps * world / (total_ms * 1e-3),
                     "solves/s", total_ms, "f64",
                     f"{cfg.name} on the even-odd Schur system: GMRES-DR({cfg.m},{cfg.k}) on 1 Z4 "
                     f"source + D-BiCGStab({cfg.k}) on {cfg.n_rhs} Z4 sources, tol {cfg.tol:g}, "
                     f"kappa = {cfg.kappa_factor} kappa_c", extra)


ROW_ARMS = {"mixed": mixed_arm, "twisted": twisted_arm, "grad": grad_arm, "evenodd": evenodd_arm}


# ------------------------------------------------------------------ growth rows in the headline line
#
# Short runs of the three growth-row workloads, nested in the default bench
# line: each block is one warm-up and one timed run (CUDA events on the
# launching stream, L2 flushed before, clocks sampled), with the roofline of
# its dominant kernel from one more, profiled run.  `--config <preset>` runs
# the full row arms above instead.

def _timed_once(fn, flush, stream, local_rank):
    """One L2-flushed run of fn timed by CUDA events, clocks sampled."""
    import torch
    clocks = ClockSampler(local_rank)
    clocks.start()
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out, clocks.stop()


def growth_mixed(local_rank, peaks):
    """20^3 x 32 at 0.995 kappa_c, k = 60 (m = 80): GMRES-DR in FP64 gives V
    (timed as setup), then D-BiCGStab(60) on the 12 Z4 sources in FP64 and in
    the mixed forms (FP32 and FP16 storage, restarted refinement with FP64
    true residuals), every solve to 1e-10."""
    import torch
    import paper_0710_1988_gb300 as wdl
    cfg = L.CONFIGS["wilson_20x20x20x32_mixed"]
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    n = 12 * v
    src = rank_sources(cfg, 0, cfg.n_rhs + 1)
    b0 = torch.from_numpy(src[0].ravel()).to(dev)
    B = torch.from_numpy(src[1:].reshape(cfg.n_rhs, n)).to(dev)
    X = torch.zeros_like(B)
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device=dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    ms_g, (rc, st, _, _), _ = _timed_once(
        lambda: op.gmresdr(b0, torch.zeros_like(b0), cfg.m, cfg.k, cfg.tol, 400000, V_out=V),
        flush, stream, local_rank)
    if rc != 0:
        raise RuntimeError(f"20^3x32 GMRES-DR status {rc}")
    defl = op.deflation(V, cfg.k)
    out = {}
    for name, bits in (("fp64", None), ("mixed32", 32), ("mixed16", 16)):
        if bits:
            op.set_mixed_storage(bits)
            op.set_mixed_restart(1e-3, 300)

        def solve():
            X.zero_()
            if bits is None:
                return op.dbicgstab(B, X, defl, tol=cfg.tol)
            return op.dbicgstab_mixed(B, X, defl, tol=cfg.tol)
        solve()                                            # warm-up (graphs, autotuner)
        ms, (rc, ss), clk = _timed_once(solve, flush, stream, local_rank)
        if rc != 0 or not all(q["converged"] for q in ss):
            raise RuntimeError(f"20^3x32 {name} D-BiCGStab status {rc}")
        out[name] = {"solves_per_s": round(cfg.n_rhs / (ms * 1e-3), 3), "ms": round(ms, 1),
                     "iters": [q["iters"] for q in ss],
                     "max_true_rel_res": max(q["true_rel_res"] for q in ss), "clocks": clk}
    # rooflines of the FP32 Wilson kernel and vector updates from one profiled solve
    op.set_mixed_storage(32)
    X.zero_()
    op.profile(mask=0x30)
    rc, ss = op.dbicgstab_mixed(B, X, defl, tol=cfg.tol)
    prof = op.profile_read()
    op.profile(mask=0)
    roof = low_rooflines(prof, 32, v, peaks, sum(q["iters"] for q in ss))
    defl.close()
    op.close()
    for name in ("mixed32", "mixed16"):
        out[name]["speedup_vs_fp64"] = round(out[name]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    return {"workload": f"{cfg.name}: D-BiCGStab({cfg.k}) on {cfg.n_rhs} Z4 sources after "
                        f"GMRES-DR({cfg.m},{cfg.k}) in FP64, tol {cfg.tol:g}, kappa = "
                        f"{cfg.kappa_factor} kappa_c; mixed = FP32 / FP16 storage, restarted "
                        f"refinement (delta 1e-3, at most 300 iterations per pass), FP64 true residual",
            "value": out["mixed32"]["solves_per_s"], "unit": "solves/s",
            "gmresdr_setup_ms": round(ms_g, 1), "gmresdr_mvp": st["mvp"],
            "gmresdr_cycles": st["cycles"], "dbicgstab": out,
            "roofline": roof.get("dslash"), "roofline_updates": roof.get("updates"),
            "timing": "1 warm-up + 1 timed solve of the batch each"}


def growth_twisted(local_rank, peaks, mus=(0.064, 0.032)):
    """24^3 x 48 twisted mass at kappa_c: the two heaviest shifts, 16 Gaussian
    sources each, the second projected over the first's solutions (Sec. 4),
    mixed BiCGStab (FP32, restarted refinement) on the even-odd Schur system,
    full-lattice solutions to 1e-10."""
    import torch
    import paper_0710_1988_gb300 as wdl
    cfg = L.CONFIGS["twisted_24x24x24x48"]
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    n = 12 * v
    B = torch.from_numpy(rank_sources(cfg, 0, cfg.n_rhs).reshape(cfg.n_rhs, n)).to(dev)
    X = torch.zeros(len(mus) * cfg.n_rhs * n, dtype=torch.complex128, device=dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    op.set_operator(True)
    op.set_mixed_storage(32)
    op.set_mixed_restart(1e-3, 300)

    def run(project=True):
        X.zero_()
        rc, sts = op.multishift(B, X, list(mus), tol=cfg.tol, project=project, mixed=True)
        if rc != 0 or not all(q["converged"] for row in sts for q in row):
            raise RuntimeError(f"24^3x48 shifts status {rc}")
        return sts
    run()
    ms, sts, clk = _timed_once(run, flush, stream, local_rank)
    ms_np, sts_np, _ = _timed_once(lambda: run(False), flush, stream, local_rank)
    op.profile(mask=0x30)
    sts_p = run()
    prof = op.profile_read()
    op.profile(mask=0)
    roof = low_rooflines(prof, 32, v, peaks, sum(q["iters"] for row in sts_p for q in row), eo=True)
    op.close()
    units = cfg.n_rhs * len(mus)
    return {"workload": f"{cfg.name}: A_W + i mu gamma5 at kappa_c, shifts {list(mus)} heaviest "
                        f"first, {cfg.n_rhs} Gaussian sources per shift batched, each shift "
                        f"projected over the earlier solutions (Sec. 4), solved on the even-odd "
                        f"Schur system by mixed BiCGStab (FP32, restarted refinement delta 1e-3), "
                        f"full-lattice true residual 1e-10; value counts (source, shift) pairs",
            "value": round(units / (ms * 1e-3), 3), "unit": "solves/s", "ms": round(ms, 1),
            "clocks": clk, "unprojected_solves_per_s": round(units / (ms_np * 1e-3), 3),
            "shifts": [{"mu": mu, "schur_mvp_projected": [q["mvp"] for q in sts[i]],
                        "schur_mvp_unprojected": [q["mvp"] for q in sts_np[i]],
                        "max_true_rel_res": max(q["true_rel_res"] for q in sts[i])}
                       for i, mu in enumerate(mus)],
            "roofline": roof.get("dslash"), "roofline_updates": roof.get("updates"),
            "timing": "1 warm-up + 1 timed run each (projected, unprojected)"}


def growth_grad(local_rank, fp64_peak):
    """32^3 x 64 at 0.99 kappa_c: x = A^-1 b and the backward of
    L = Re(eta^dagger x) (adjoint solve via gamma5, dL/db, dL/dkappa, link
    force), with both solves in FP64 and in mixed precision, to 1e-10."""
    import torch
    import paper_0710_1988_gb300 as wdl
    from paper_0710_1988_gb300.autograd import wilson_solve
    cfg = L.CONFIGS["grad_32x32x32x64"]
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    kappa = kappa_for(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    src = rank_sources(cfg, 0, 2)
    b = torch.from_numpy(src[0].ravel()).to(dev)
    eta = torch.from_numpy(src[1].ravel()).to(dev)
    op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).to(dev), kappa)
    op.set_mixed_restart(1e-3, 300)

    def step(mixed):
        bt = b.clone().requires_grad_(True)
        kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
        om = torch.zeros((v, 4, 8), dtype=torch.float64, device=dev, requires_grad=True)
        x = wilson_solve(bt, kt, om, op, None, cfg.tol, mixed=mixed)
        loss = (eta.conj() * x).sum().real
        loss.backward()
        return float(kt.grad), float(om.grad.abs().max())
    out = {}
    for name, mixed in (("fp64", False), ("mixed32", True)):
        step(mixed)
        if name == "fp64":
            op.profile(mask=0x1)
        ms, res, clk = _timed_once(lambda: step(mixed), flush, stream, local_rank)
        if name == "fp64":
            prof_live = op.profile_read()
            op.profile(mask=0)
        out[name] = {"value": round(1.0 / (ms * 1e-3), 4), "unit": "fwd+bwd solves/s",
                     "ms": round(ms, 1), "dkappa": res[0], "max_abs_force": res[1], "clocks": clk}
    op.close()
    r = roofline({"prof_live": prof_live}, {}, fp64_peak)
    r["traffic"] = None
    r.pop("traffic_source", None)
    r.pop("hbm_view", None)
    out["mixed32"]["speedup_vs_fp64"] = round(out["mixed32"]["value"] / out["fp64"]["value"], 3)
    out["mixed32"]["dkappa_rel_diff_vs_fp64"] = abs(out["mixed32"]["dkappa"] / out["fp64"]["dkappa"] - 1)
    return {"workload": f"{cfg.name}: x = A^-1 b (BiCGStab) and the backward of Re(eta^dagger x) "
                        f"(adjoint solve via gamma5, dL/db, dL/dkappa, link force), tol {cfg.tol:g}, "
                        f"kappa = {cfg.kappa_factor} kappa_c; FP64 and mixed (FP32 iteration, "
                        f"restarted refinement, FP64 gradients)",
            "value": out["fp64"]["value"], "unit": "fwd+bwd solves/s", "runs": out,
            "roofline": r, "timing": "1 warm-up + 1 timed forward+backward each"}


def growth_rows(local_rank, peaks, fp64_peak):
    rows = {}
    for key, fn in (("wilson_20x20x20x32_mixed", lambda: growth_mixed(local_rank, peaks)),
                    ("twisted_24x24x24x48", lambda: growth_twisted(local_rank, peaks)),
                    ("grad_32x32x32x64", lambda: growth_grad(local_rank, fp64_peak))):
        t = time.perf_counter()
        rows[key] = fn()
        rows[key]["wall_s"] = round(time.perf_counter() - t, 1)
    return rows


def reference_arm(args, cfg, rank, world):
    """The oracle on the host cores: same workload, metric and config.  Each
    step is one round of workload slices on every usable core (one process
    per core, each on its own source; see oracle_slices), so the step's wall
    time is measured, not extrapolated."""
    if rank != 0:
        return
    kappa = kappa_for(cfg)
    counts = load_json(ORACLE_COUNTS) if cfg.name == "wilson_16x16x16x16" else None
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"oracle step counts for {cfg.name} are not recorded"}))
        return
    js_all, bicg = slice_plan(cfg, counts)
    cores = host_cores(worker_bytes(cfg))
    # warm-up rounds, then timed rounds whose positions spread evenly over
    # the step's Arnoldi sequence
    order = (spread_positions(args.warmup, len(js_all), 0.25) if args.warmup else []) + \
        spread_positions(args.steps, len(js_all))
    rounds, _ = oracle_slices(cfg, kappa, counts, cores, order)
    timed = rounds[args.warmup:]
    t_total = sum(timed)
    per_step = cores * cfg.n_rhs / len(js_all)
    value = per_step * len(timed) / t_total
    line = {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * t_total / len(timed), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: SU(3) links exp(i*0.5*H) (seed 1001), Z4 sources; no dataset",
        "config": headline_config(cfg, kappa, world),
        "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores,
                         "kind": "oracle", "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                         "sample": (f"per step, {cores} concurrent oracle processes (numpy FP64, 1 "
                                    f"BLAS thread each, own source each) run one slice each: 1/"
                                    f"{len(js_all)} of the oracle's {cfg.name} step, one Arnoldi+"
                                    f"CGS2 step and {bicg} BiCGStab iterations; a step counts "
                                    f"{cores} x {cfg.n_rhs}/{len(js_all)} solves; restart products, "
                                    f"deflation setup and projections left out")},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
