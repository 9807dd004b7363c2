"""Host-side byte models behind the bench line's FP32 rooflines: the full
Wilson kernel, the two half-lattice launches of an even-odd Schur apply, and
the per-iteration vector updates (V sites, or V/2 on the Schur system)."""
import pytest

import bench


def _prof(site_updates, launches, ms, upd_launches, upd_ms):
    return {"dslash_low": {"launches": launches, "ms": ms},
            "stream_low": {"launches": upd_launches, "ms": upd_ms},
            "dslash_low_site_updates": site_updates}


def test_schur_bytes_per_even_site():
    # v = A_hat p: SCHUR1 reads p, writes tmp; SCHUR2 reads tmp and p, writes
    # v, reads r_hat.  t = A_hat s, s = r - alpha v: SCHUR1 reads r and v,
    # writes tmp; SCHUR2 reads tmp, r and v, writes t.  96 B per FP32 spinor.
    v_apply = (1 + 1) + (2 + 1 + 1)
    t_apply = (2 + 1) + (3 + 1)
    assert bench.LOW_SCHUR_BYTES[32] == 96 * (v_apply + t_apply) / 2


@pytest.mark.parametrize("eo", [False, True])
def test_low_rooflines(eo):
    V, nsys, applies, iters = 1000, 4, 10, 5
    counted = (V // 2 if eo else V) * nsys * applies  # the device's site counter
    prof = _prof(counted, applies, 2.0, 2 * iters, 1.0)
    out = bench.low_rooflines(prof, 32, V, {"hbm_gbs": 1000.0}, iters, eo=eo)
    d, u = out["dslash"], out["updates"]
    if eo:
        byt = bench.LOW_SCHUR_BYTES[32] * counted + 2 * bench.LOW_LINK_BYTES[32] * V * applies
        ubyt = bench.LOW_UPDATE_BYTES[32] * (V // 2) * iters
    else:
        byt = bench.LOW_DSLASH_BYTES[32] * counted + bench.LOW_LINK_BYTES[32] * V * applies
        ubyt = bench.LOW_UPDATE_BYTES[32] * V * iters
    assert d["algorithmic_bytes_per_launch"] == pytest.approx(byt / applies)
    assert d["achieved"] == pytest.approx(byt / 2.0e-3 / 1e9, abs=0.05)
    assert d["frac"] == pytest.approx(d["achieved"] / 1000.0, abs=1e-4)
    assert u["algorithmic_bytes_per_launch"] == pytest.approx(ubyt / (2 * iters))
    assert u["frac"] == pytest.approx(ubyt / 1.0e-3 / 1e9 / 1000.0, abs=1e-4)
    assert ("eo32" in d["kernel"]) == eo


def test_no_launches_no_lines():
    out = bench.low_rooflines(_prof(0, 0, 0.0, 0, 0.0), 32, 1000, {"hbm_gbs": 1.0}, 0)
    assert out == {}


def test_oracle_slices_partition_the_oracle_step():
    """The CPU baseline and the reference arm time slices that are exactly
    1/len(sequence) of the oracle's own step: the GMRES-DR Arnoldi sequence
    (m in the first cycle, m - k in each later one) and the BiCGStab
    iterations spread evenly over it."""
    import json
    import bench
    from inputs import lattice as L
    cfg = L.CONFIGS["wilson_16x16x16x16"]
    with open(bench.ORACLE_COUNTS) as f:
        counts = json.load(f)
    js, per = bench.slice_plan(cfg, counts)
    assert len(js) == cfg.m + (cfg.m - cfg.k) * (counts["gmresdr_cycles"] - 1) == counts["gmresdr_mvp"]
    assert per * len(js) == sum(counts["dbicgstab_iters"])
    pos = bench.spread_positions(20, len(js))
    assert len(set(pos)) == 20 and min(pos) >= 0 and max(pos) < len(js)


def test_oracle_slices_run_concurrently():
    import bench
    from inputs import lattice as L
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    counts = {"gmresdr_cycles": 2, "dbicgstab_iters": [10, 12, 8]}
    rounds, info = bench.oracle_slices(cfg, 0.12, counts, 2, [0, 3, 20])
    assert len(rounds) == 3 and all(t > 0 for t in rounds)
    assert info["js"] == [0, 3, 6] and info["slices_per_step"] == cfg.m + (cfg.m - cfg.k)
