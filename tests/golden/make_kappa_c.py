"""Write kappa_c.json: the critical kappa of every preset gauge field.

kappa_c is computed by the CPU oracle only (rightmost eigenvalue of the
hopping matrix D, kappa_c = 1 / max Re lambda(D)); the CUDA path never
contributes to it.  Run from the repository root:

    python tests/golden/make_kappa_c.py [preset ...]
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from inputs import lattice as L          # noqa: E402
from oracle import kappa                 # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kappa_c.json")

# Presets whose Arnoldi basis would not fit in host memory (32^3 x 64: 403 MB
# per vector) take the kappa_c of a smaller field drawn with the same recipe
# (same eps and link seed); kappa_c of these fields varies with the volume by
# ~1e-4 (0.14753 at 8^3 x 16, 0.14762 at 16^4, 0.14770 at 20^3 x 32).
SUBSTITUTE = {"grad_32x32x32x64": "grad_8x8x8x16"}


def main(names):
    table = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            table = json.load(f)
    for name in names:
        cfg = L.CONFIGS[name]
        t0 = time.time()
        if name in SUBSTITUTE:
            src = SUBSTITUTE[name]
            if src not in table:
                main([src])
                with open(OUT) as f:
                    table = json.load(f)
            table[name] = {"dims": list(cfg.dims), "eps": cfg.eps, "link_seed": L.link_seed(cfg),
                           "kappa_c": table[src]["kappa_c"],
                           "method": f"kappa_c of {src} (same recipe; this field's Arnoldi basis "
                                     "exceeds host memory)"}
            print(f"{name}: kappa_c = {table[name]['kappa_c']!r} (from {src})", flush=True)
            with open(OUT, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            continue
        U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
        kc = kappa.kappa_c(U, cfg.dims)
        table[name] = {"dims": list(cfg.dims), "eps": cfg.eps,
                       "link_seed": L.link_seed(cfg), "kappa_c": kc,
                       "method": ("dense eig" if 12 * U.shape[0] <= 3072 else
                                  "Arnoldi (eigs LR, tol 1e-10)" if 12 * U.shape[0] <= 100_000
                                  else "300-step Arnoldi factorisation, rightmost Ritz value"
                                  if 12 * U.shape[0] <= 4_000_000
                                  else "200-step Arnoldi factorisation, rightmost Ritz value")}
        print(f"{name}: kappa_c = {kc!r}  ({time.time() - t0:.0f} s)", flush=True)
        with open(OUT, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(L.CONFIGS))
