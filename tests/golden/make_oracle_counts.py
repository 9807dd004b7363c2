"""Write oracle_counts_<lattice>.json: the CPU oracle's own MVP, cycle and
iteration counts on the benchmark workload (GMRES-DR(80,40) on the first Z4
source, then D-BiCGStab(40) on 10 further Z4 sources, tol 1e-10, 16^4 at
kappa = 0.99 kappa_c).  Only oracle/ and inputs/ run here.

The counts serve two purposes: the full-size parity check of the GPU run
(the same cycle count, iteration counts within a few), and the
extrapolation of the timed CPU-oracle sample to whole solves.

    python tests/golden/make_oracle_counts.py [preset]      (about an hour of CPU)
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from inputs import lattice as L          # noqa: E402
from oracle import dirac, krylov         # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main(name="wilson_16x16x16x16"):
    cfg = L.CONFIGS[name]
    with open(os.path.join(HERE, "kappa_c.json")) as f:
        kappa = cfg.kappa_factor * json.load(f)[name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    A = lambda x: dirac.apply_A(U, x.reshape(v, 4, 3), cfg.dims, kappa).ravel()
    g5 = lambda x: dirac.gamma5(x.reshape(v, 4, 3)).ravel()
    t0 = time.time()
    gd = krylov.gmresdr(A, L.source(cfg, 0).ravel(), cfg.m, cfg.k, tol=cfg.tol)
    print(f"GMRES-DR: {gd.stats.mvp} MVPs, {gd.stats.cycles} cycles, "
          f"true rel res {gd.stats.true_rel_res:.3e} ({time.time() - t0:.0f} s)", flush=True)
    out = {"workload": name, "kappa": kappa, "m": cfg.m, "k": cfg.k, "tol": cfg.tol,
           "gmresdr_mvp": gd.stats.mvp, "gmresdr_cycles": gd.stats.cycles,
           "gmresdr_history": gd.stats.history,
           "theta": [[t.real, t.imag] for t in gd.theta],
           "dbicgstab_mvp": [], "dbicgstab_iters": [], "dbicgstab_true_rel_res": [],
           "bicgstab_first_source_mvp": None}
    for j in range(1, cfg.n_rhs + 1):
        b = L.source(cfg, j).ravel()
        x, st = krylov.dbicgstab(A, b, gd.V, tol=cfg.tol, gamma5=g5)
        out["dbicgstab_mvp"].append(st.mvp)
        out["dbicgstab_iters"].append(st.iters)
        out["dbicgstab_true_rel_res"].append(st.true_rel_res)
        print(f"rhs {j}: {st.mvp} MVPs, true rel res {st.true_rel_res:.3e} "
              f"({time.time() - t0:.0f} s)", flush=True)
    x, st = krylov.bicgstab(A, L.source(cfg, 1).ravel(), tol=cfg.tol)
    out["bicgstab_first_source_mvp"] = st.mvp
    with open(os.path.join(HERE, f"oracle_counts_{'x'.join(map(str, cfg.dims))}.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(*sys.argv[1:])
