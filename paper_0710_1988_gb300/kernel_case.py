"""Run one Wilson-operator kernel on its own, for profilers and timing.

    python -m paper_0710_1988_gb300.kernel_case --kernel f32 --lattice 20 20 20 32 --nrhs 12
    python -m paper_0710_1988_gb300.kernel_case --kernel f32 --even-odd --lattice 24 24 24 48 --nrhs 16
    python -m paper_0710_1988_gb300.kernel_case --kernel fp64-peak --reps 5
    python -m paper_0710_1988_gb300.kernel_case --kernel tsgemm --lattice 16 16 16 16 --kv 81 --ncol 41
    python -m paper_0710_1988_gb300.kernel_case --kernel gmresdr --workload wilson_16x16x16x16

Builds a seeded gauge field (U = exp(i 0.5 H)) and Gaussian spinors, then
applies the operator `--reps` times through the public binding (`apply`,
`apply_f32` or `apply_f16`) and prints the mean time per application from
the handle's own kernel timing.  The low-precision entry points also run
their conversion kernels; a profiler selects the Wilson kernel by name.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    import torch

    import paper_0710_1988_gb300 as wdl
    from inputs import lattice as L

    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=["f64", "f32", "f16", "mixed", "fp64-peak", "tsgemm",
                                         "gmresdr"],
                    default="f32",
                    help="a Wilson apply, 'mixed': --reps iterations of the FP32 mixed "
                         "BiCGStab on --nrhs sources (its vector updates and Wilson kernels), or "
                         "'fp64-peak': the library's DFMA throughput probe, 'tsgemm': the "
                         "restart product V_{m+1} P_{k+1} (--kv, --ncol) in both forms, "
                         "'gmresdr': one GMRES-DR(m,k) solve of a workload's first source "
                         "(--workload), its cycle-end kernels timed per restart")
    ap.add_argument("--workload", default="wilson_16x16x16x16",
                    help="a configuration of inputs.lattice (--kernel gmresdr)")
    ap.add_argument("--kappa-c", type=float, default=None,
                    help="kappa_c of the workload (default: the value stored with the tests)")
    ap.add_argument("--fp64-eig", action="store_true",
                    help="--kernel gmresdr: harmonic Ritz pairs by the FP64 QR iteration alone")
    ap.add_argument("--kv", type=int, default=81)
    ap.add_argument("--ncol", type=int, default=41)
    ap.add_argument("--lattice", type=int, nargs=4, default=[20, 20, 20, 32])
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--kappa", type=float, default=0.14)
    ap.add_argument("--storage", type=int, choices=[32, 16], default=32,
                    help="vector storage of the mixed solver (--kernel mixed)")
    ap.add_argument("--even-odd", action="store_true",
                    help="the even-odd Schur operator on even half vectors (f64 and f32 only)")
    args = ap.parse_args(argv)
    if args.kernel == "fp64-peak":
        for iters in (1 << 14, 1 << 15, 1 << 16):
            tf, ms = wdl.probe_fp64_peak(iters=iters, reps=args.reps)
            print(json.dumps({"kernel": "dfma_probe_kernel", "iters": iters, "reps": args.reps,
                              "tflops": tf, "ms_per_launch": ms}))
        for iters in (4096, 16384):
            tf, ms = wdl.probe_bf16_mma_peak(iters=iters, reps=args.reps)
            print(json.dumps({"kernel": "bf16_mma_probe_kernel", "iters": iters, "reps": args.reps,
                              "tflops": tf, "ms_per_launch": ms}))
        return
    if args.kernel == "gmresdr":
        cfg = L.CONFIGS[args.workload]
        kc = args.kappa_c
        if kc is None:
            import os
            path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "tests", "golden", "kappa_c.json")
            with open(path) as f:
                kc = json.load(f)[cfg.name]["kappa_c"]
        kappa = cfg.kappa_factor * kc
        U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
        b0 = torch.from_numpy(np.ascontiguousarray(L.source(cfg, 0)).reshape(-1)).cuda()
        op = wdl.WilsonOperator(cfg.dims, torch.from_numpy(U).cuda(), kappa)
        op.set_eigen_estimates(not args.fp64_eig)
        V = torch.zeros(cfg.k * b0.numel(), dtype=torch.complex128, device="cuda")
        res = []
        for rep in range(2):          # the first solve warms up
            x0 = torch.zeros_like(b0)
            op.profile(mask=0x08)     # category 3: LU and the GMRES-DR cycle end
            rc, st, _, theta = op.gmresdr(b0, x0, cfg.m, cfg.k, cfg.tol, 100000, V_out=V)
            p = op.profile_read()
            op.profile(mask=0)
            res.append((rc, st, p["dense"]))
        rc, st, dense = res[-1]
        restarts = st["cycles"]
        print(json.dumps({"kernel": "gmresdr_cycle_end", "workload": cfg.name, "m": cfg.m,
                          "k": cfg.k, "fp32_estimates": not args.fp64_eig, "status": rc,
                          "mvp": st["mvp"], "cycles": st["cycles"], "solve_ms": st["ms"],
                          "cycle_end_launches": dense["launches"], "cycle_end_ms": dense["ms"],
                          "ms_per_cycle_end": dense["ms"] / max(1, restarts)}))
        op.close()
        return
    dims = tuple(args.lattice)
    if args.kernel == "tsgemm":
        n = 12 * L.volume(dims)
        g = torch.Generator(device="cuda").manual_seed(5)
        V = torch.randn(args.kv * n, dtype=torch.complex128, device="cuda", generator=g)
        Y = torch.randn(args.kv * args.ncol, dtype=torch.complex128, device="cuda", generator=g)
        out = {}
        for tc in (True, False):
            W = torch.empty(args.ncol * n, dtype=torch.complex128, device="cuda")
            wdl.tsgemm(V, args.kv, Y, args.ncol, W, tensor_cores=tc)       # warm
            ts = []
            for _ in range(args.reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                wdl.tsgemm(V, args.kv, Y, args.ncol, W, tensor_cores=tc)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            out["tensor_cores" if tc else "fp64"] = {"ms": min(ts), "W": W}
        diff = (out["tensor_cores"]["W"] - out["fp64"]["W"]).abs().max().item()
        scale = out["fp64"]["W"].abs().max().item()
        print(json.dumps({"kernel": "tsgemm", "lattice": list(dims), "n": n, "kv": args.kv,
                          "ncol": args.ncol, "ms_tensor_cores": out["tensor_cores"]["ms"],
                          "ms_fp64": out["fp64"]["ms"], "max_abs_diff_over_max": diff / scale}))
        return
    U = L.gauge_field(dims, 0.5, 1002)
    psi = L.gaussian_spinor(dims, 2200, nrhs=args.nrhs)
    op = wdl.WilsonOperator(dims, torch.from_numpy(U).cuda(), args.kappa)
    if args.even_odd:
        op.set_operator(True)
        psi = psi.reshape(args.nrhs, -1)[:, : op.op_n]  # any values serve as even half vectors
    x = torch.from_numpy(np.ascontiguousarray(psi).reshape(-1)).cuda()
    y = torch.empty_like(x)
    if args.kernel == "mixed":
        op.set_mixed_storage(args.storage)
        y.zero_()
        op.dbicgstab_mixed(x, y, None, tol=1e-30, max_iter=3)  # warm-up (graphs, tuning)
        y.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, sts = op.dbicgstab_mixed(x, y, None, tol=1e-30, max_iter=args.reps)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel": "mixed", "lattice": list(dims), "nrhs": args.nrhs,
                          "even_odd": args.even_odd, "storage": args.storage,
                          "iters": [q["iters"] for q in sts][:4],
                          "ms": e0.elapsed_time(e1), "status": rc}))
        op.close()
        return
    fn = {"f64": op.apply, "f32": op.apply_f32, "f16": op.apply_f16}[args.kernel]
    fn(x, y)
    torch.cuda.synchronize()
    op.profile(mask=0x11)
    for _ in range(args.reps):
        fn(x, y)
    torch.cuda.synchronize()
    p = op.profile_read()
    op.profile(mask=0)
    cat = "dslash" if args.kernel == "f64" else "dslash_low"
    ms = p[cat]["ms"] / max(1, p[cat]["launches"])
    print(json.dumps({"kernel": args.kernel, "lattice": list(dims), "nrhs": args.nrhs,
                      "even_odd": args.even_odd, "ms_per_apply": ms, "finite": bool(np.isfinite(y.abs().max().item()))}))
    op.close()


if __name__ == "__main__":
    main()
