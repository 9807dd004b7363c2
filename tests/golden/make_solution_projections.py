"""Write solution_projections_<lattice>.json: the oracle's solution of one
right-hand side of the benchmark workload, stored as 64 fixed random
projections <z_i, x> (the full vector is 12.6 MB).

The solution is A^-1 b itself, so the oracle reaches it with plain BiCGStab
to a relative residual of 1e-14 (which method gives x does not matter).  The
probes z_i are Gaussian spinors with the seeds recorded in the file (Re, Im
~ N(0, 1) per component); for such a probe E|<z, e>|^2 = 2 ||e||^2, so the
64 projections of the error of another solution estimate its norm (the full-size parity test's
solution-error check).  The same is recorded for the oracle's own 1e-10
solve, to show the error that tolerance leaves at this conditioning.
Only oracle/ and inputs/ run here.

    python tests/golden/make_solution_projections.py [preset] [rhs]   (minutes of CPU)
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from inputs import lattice as L          # noqa: E402
from oracle import dirac, krylov         # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
N_PROBES = 64
PROBE_SEED0 = 7000


def probes(dims):
    for i in range(N_PROBES):
        yield PROBE_SEED0 + i, L.gaussian_spinor(dims, PROBE_SEED0 + i).ravel()


def main(name="wilson_16x16x16x16", j="1"):
    j = int(j)
    cfg = L.CONFIGS[name]
    with open(os.path.join(HERE, "kappa_c.json")) as f:
        kappa = cfg.kappa_factor * json.load(f)[name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    A = lambda x: dirac.apply_A(U, x.reshape(v, 4, 3), cfg.dims, kappa).ravel()
    b = L.source(cfg, j).ravel()
    t0 = time.time()
    x, st = krylov.bicgstab(A, b, tol=1e-14, max_iter=20000)
    print(f"1e-14 solve: {st.mvp} MVPs, true rel res {st.true_rel_res:.3e} "
          f"({time.time() - t0:.0f} s)", flush=True)
    assert st.converged
    x10, st10 = krylov.bicgstab(A, b, tol=1e-10, max_iter=20000)
    print(f"1e-10 solve: {st10.mvp} MVPs ({time.time() - t0:.0f} s)", flush=True)
    seeds, proj, proj_err10 = [], [], []
    for seed, z in probes(cfg.dims):
        seeds.append(seed)
        p = np.vdot(z, x)
        proj.append([p.real, p.imag])
        proj_err10.append(abs(np.vdot(z, x10 - x)))
    xn = float(np.linalg.norm(x))
    out = {"workload": name, "rhs": j, "kappa": kappa, "tol": 1e-14,
           "true_rel_res": st.true_rel_res, "mvp": st.mvp,
           "x_norm": xn, "probe_kind": "gaussian_spinor", "probe_seeds": seeds,
           "projections": proj,
           "oracle_tol_1e-10": {
               "mvp": st10.mvp, "true_rel_res": st10.true_rel_res,
               "rel_error": float(np.linalg.norm(x10 - x)) / xn,
               "rel_error_from_probes": float(np.sqrt(np.mean(np.square(proj_err10)) / 2)) / xn}}
    path = os.path.join(HERE, f"solution_projections_{'x'.join(map(str, cfg.dims))}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["oracle_tol_1e-10"]))


if __name__ == "__main__":
    main(*sys.argv[1:])
