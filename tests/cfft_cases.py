"""Shared test plumbing: run a TableWorkload through the GPU library and through
the oracle, and compare.  Test infrastructure only (may import ``oracle``)."""
import numpy as np

import workloads
from oracle import contour as oc
from oracle import fill as ofill
from oracle import reaction as orx
from oracle import spectra as osp


def oracle_basis(el):
    if el.kind == "strip":
        return osp.BasisSet("strip", el.q, length=el.length, width=el.strip_width)
    return osp.BasisSet("rooftop", el.q, cx=el.cx, cy=el.cy, direction=el.direction,
                        half_len=el.half_len, width=el.width)


def oracle_n_alpha(wl):
    """A converged trapezoid size for the element (checked by the oracle pins)."""
    return 128


def oracle_workers():
    import os
    return max(1, min(32, os.cpu_count() or 1))


def oracle_harmonics(wl, classes=(0,)):
    c = wl.contour
    nodes = oc.contour_nodes(c.n, c.beta_max, c.beta_p, c.height)
    bs = oracle_basis(wl.element)
    s = wl.substrate
    out = {}
    for cls in classes:
        out[cls] = orx.harmonics(bs, nodes["beta_c"], wl.qs, oracle_n_alpha(wl), s.eps_r, s.h,
                                 s.k0, *orx.rotation_angles(cls), workers=oracle_workers())
    return nodes, out


def oracle_table(wl, classes=(0,), rho_index=None):
    """Z[cls][pair][q][r] (matched contour, Bessel sum) at rho_index (default: all)."""
    nodes, hq = oracle_harmonics(wl, classes)
    rho = wl.rho if rho_index is None else wl.rho[np.asarray(rho_index)]
    tabs = []
    for cls in classes:
        z = orx.table_bessel(hq[cls], wl.qs, nodes["beta_c"], nodes["weight"], rho)
        m = z.shape[0]
        tabs.append(z.reshape(m * m, len(wl.qs), len(rho)))
    return np.array(tabs), nodes, hq


def gpu_context(wl, device=0, options=None):
    from paper_1404_7357_gb300 import cfft
    ctx = cfft.Context(device)
    s = wl.substrate
    ctx.set_substrate(s.eps_r, s.h, s.k0)
    el = wl.element
    if el.kind == "strip":
        ctx.set_mbf_spectra_strip(el.length, el.strip_width)
    else:
        ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len, el.width, el.q)
    c = wl.contour
    ctx.build_contour(c.n, c.beta_max, c.beta_p, c.height, wl.extras.get("taylor", -1))
    for k, v in (options or {}).items():
        ctx.set_option(k, v)
    return ctx


def gpu_table(wl, device=0, options=None):
    from paper_1404_7357_gb300 import cfft
    ctx = gpu_context(wl, device, options)
    prec = cfft.CFFT_FP64 if wl.precision == "fp64" else cfft.CFFT_FP32_MIXED
    ctx.tabulate_reactions(wl.q_max, wl.rho_max, wl.n_rho, prec, wl.rotation_classes)
    return ctx, ctx.copy_table(host=True).numpy()


def rel_err_per_pair(got, ref):
    """max over (q, r) of |got - ref| / max |ref|, per (class, pair)."""
    got = np.asarray(got).astype(np.complex128)
    err = np.abs(got - ref).reshape(ref.shape[0], ref.shape[1], -1).max(-1)
    scale = np.abs(ref).reshape(ref.shape[0], ref.shape[1], -1).max(-1)
    return err / scale


def oracle_fill_entries(wl, hq_by_class, nodes, pos, rot, pairs):
    return ofill.entries(hq_by_class, wl.qs, nodes["beta_c"], nodes["weight"], pos, rot, pairs)


def small_patch(precision="fp32", n=2048, n_rho=384, rho_max=6.0, q_max=4, rotation_classes=1):
    return workloads.patch_m4(n=n, n_rho=n_rho, rho_max=rho_max, q_max=q_max, precision=precision,
                              rotation_classes=rotation_classes)
