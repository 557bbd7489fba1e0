"""Writes contour_study_strip.json: the converged reaction between two strip MBFs at
the diagonal separation of the paper's Table I study (Section IV, "On the Contour
height and Taylor's series order": d = sqrt(dx^2 + dy^2) = 21.2 lambda0), computed by
the oracle alone (adaptive Gauss-Kronrod along the contour, O1), for the GPU study
of error versus contour height and Taylor order (tests/test_gpu_contour_study.py).

Element and substrate: the strip workload (cosine strip L = 0.45, W = 0.02 lambda0;
eps_r = 2.2, h = 0.05 lambda0), harmonics |q| <= 4, Delta = (15, 15) lambda0.  The
same integral on a contour twice as high (Cauchy: no pole between them) is stored
beside it as the check of convergence.

Run: python tests/golden/make_contour_study.py   (about a minute on 16 cores)
"""
import json
import math
import os
import sys
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import reaction as orx, spectra as osp  # noqa: E402

DX, DY = 15.0, 15.0
Q_MAX = 4


def _zq(args):
    q, height = args
    wl = workloads.strip_fp64(n=4096, q_max=Q_MAX)
    s, el, c = wl.substrate, wl.element, wl.contour
    bs = osp.BasisSet("strip", np.ones((1, 1)), length=el.length, width=el.strip_width)
    rho = math.hypot(DX, DY)
    return orx.table_adaptive(bs, 0, 0, q, rho, c.beta_max, c.beta_p, height, 128, s.eps_r, s.h, s.k0)


def main():
    wl = workloads.strip_fp64(n=4096, q_max=Q_MAX)
    c = wl.contour
    qs = list(range(-Q_MAX, Q_MAX + 1))
    rho, phi = math.hypot(DX, DY), math.atan2(DY, DX)
    out = {}
    import multiprocessing as mp
    with ProcessPoolExecutor(max_workers=min(18, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        for name, height in (("reference", c.height), ("cauchy_check", 2.0 * c.height)):
            zq = np.array(list(ex.map(_zq, [(q, height) for q in qs])))
            z = orx.reaction_from_table(zq, qs, phi)
            out[name] = {"contour_height": height, "zq_re": zq.real.tolist(), "zq_im": zq.imag.tolist(),
                         "z_re": float(z.real), "z_im": float(z.imag)}
    zr = complex(out["reference"]["z_re"], out["reference"]["z_im"])
    zc = complex(out["cauchy_check"]["z_re"], out["cauchy_check"]["z_im"])
    out["meta"] = {"source": "oracle.reaction.table_adaptive (O1), strip workload, N-independent",
                   "dx": DX, "dy": DY, "rho": rho, "phi": phi, "q_max": Q_MAX,
                   "beta_max": c.beta_max, "beta_p": c.beta_p,
                   "cauchy_rel_diff": abs(zr - zc) / abs(zr)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "contour_study_strip.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, "Z' =", zr, "Cauchy rel diff %.2e" % out["meta"]["cauchy_rel_diff"])


if __name__ == "__main__":
    main()
