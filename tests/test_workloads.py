"""The synthetic input recipe (seeded generators with no method arithmetic): the
properties the benchmarks and tests rely on."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import workloads


def test_poisson_disc_spacing_radius_and_seed():
    pts = workloads.poisson_disc(2000, 25.0, 0.5, seed=5)
    assert pts.shape == (2000, 2)
    assert np.all(np.hypot(pts[:, 0], pts[:, 1]) <= 25.0 + 1e-12)      # inside the disc
    d, _ = cKDTree(pts).query(pts, k=2)
    assert d[:, 1].min() >= 0.5 - 1e-12                                # minimum spacing
    assert np.array_equal(pts, workloads.poisson_disc(2000, 25.0, 0.5, seed=5))   # seeded
    assert not np.array_equal(pts, workloads.poisson_disc(2000, 25.0, 0.5, seed=6))


def test_bench_array_pair_distances_fit_the_fill_table():
    """The 10,000-element array's largest pair distance stays below the fill table's
    rho_max (121 lambda0) and its smallest above the minimum spacing."""
    pos, rot = workloads.irregular_array()
    assert pos.shape == (10000, 2) and set(np.unique(rot)) <= {0, 1}
    r = np.hypot(pos[:, 0], pos[:, 1])
    assert 2 * r.max() < 121.0
    assert 0.3 < rot.mean() < 0.7                                      # both rotations present


def test_sweep_items_sampling_rule_and_contours():
    items = workloads.sweep_items()
    assert len(items) == 512
    for it in items:
        step = it["beta_max"] / it["n"]
        kd = it["k0"] * math.sqrt(it["eps_r"])
        assert abs(it["beta_max"] - 5.0 * kd) < 1e-9 * it["beta_max"]  # 5 k_d
        assert 2 * math.pi / step >= 2.0 * 50.0 * 3.0                  # s period covers 2 rho_max 3x
        assert abs(it["beta_p"] / step - round(it["beta_p"] / step)) < 1e-9   # beta_p on a cell boundary
        assert abs(it["beta_p"] - 1.3 * kd) <= step                    # beyond every pole (< k_d)
        assert it["n"] % 256 == 0 and 2.0 <= it["eps_r"] <= 10.0 and 0.02 <= it["h"] <= 0.1
        # six node spacings, capped at height * rho_max = 3 (float32 growth exp(height * rho))
        assert it["height"] == pytest.approx(min(6.0 * step, 3.0 / 50.0), rel=1e-12)
        assert it["height"] * 50.0 <= 3.0 + 1e-12 and it["height"] >= 2.5 * step
    ns = {it["n"] for it in items}
    assert min(ns) >= 4096 and max(ns) <= 65536 and len(ns) > 1        # uneven contour lengths


def test_patch_element_and_table_workloads():
    el = workloads.patch_rooftops()
    assert el.q.shape == (200, 4) and el.n_mbf == 4
    assert np.sum(el.direction == 0) == 100 and np.sum(el.direction == 1) == 100
    wl = workloads.patch_m4()
    assert (wl.contour.n, wl.n_rho, wl.rho_max, wl.q_max) == (16384, 8192, 50.0, 16)
    c = wl.contour
    step = c.beta_max / c.n
    assert abs(c.height - 6.0 * step) < 1e-12 and c.beta_p < c.beta_max
