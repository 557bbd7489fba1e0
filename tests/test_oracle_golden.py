"""The golden fixture of the contour-height study (tests/golden/contour_study_strip.json)
is the oracle's own converged value: a harmonic recomputed here by the oracle's
adaptive quadrature matches the stored one, the stored reaction is the harmonic sum of
the stored harmonics, and the copy on a contour twice as high agrees (Cauchy: no pole
between the two contours)."""
import json
import math
import os

import numpy as np

import workloads
from oracle import reaction as orx, spectra as osp

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "contour_study_strip.json")


def _load():
    with open(GOLD) as f:
        return json.load(f)


def test_fixture_is_consistent():
    d = _load()
    meta = d["meta"]
    qs = np.arange(-meta["q_max"], meta["q_max"] + 1)
    for name in ("reference", "cauchy_check"):
        e = d[name]
        zq = np.array(e["zq_re"]) + 1j * np.array(e["zq_im"])
        z = orx.reaction_from_table(zq, qs, meta["phi"])
        assert abs(z - complex(e["z_re"], e["z_im"])) < 1e-14 * abs(z)
    zr = complex(d["reference"]["z_re"], d["reference"]["z_im"])
    zc = complex(d["cauchy_check"]["z_re"], d["cauchy_check"]["z_im"])
    assert abs(zr - zc) < 1e-10 * abs(zr)
    assert abs(meta["rho"] - math.hypot(meta["dx"], meta["dy"])) < 1e-12
    assert abs(meta["rho"] - 21.2) < 0.02      # the separation of the study (21.2 lambda0)


def test_fixture_reproduces_from_the_oracle():
    d = _load()
    meta = d["meta"]
    wl = workloads.strip_fp64(n=4096, q_max=meta["q_max"])
    s, el, c = wl.substrate, wl.element, wl.contour
    bs = osp.BasisSet("strip", np.ones((1, 1)), length=el.length, width=el.strip_width)
    q = 2
    z = orx.table_adaptive(bs, 0, 0, q, meta["rho"], c.beta_max, c.beta_p, d["reference"]["contour_height"],
                           128, s.eps_r, s.h, s.k0)
    i = q + meta["q_max"]
    stored = complex(d["reference"]["zq_re"][i], d["reference"]["zq_im"][i])
    assert abs(z - stored) < 1e-12 * max(abs(stored), 1e-300) + 1e-15
