"""Seeded synthetic inputs shared by the oracle-based tests and the GPU path.

This module only generates inputs: element geometry (basis-function meshes),
MBF coefficient matrices, array positions and rotations, substrate and grid
parameters.  It holds none of the C-FFT arithmetic, so that the oracle and
the CUDA path can both draw identical inputs without sharing any computation.

Lengths are in free-space wavelengths (k0 = 2 pi) unless a workload says
otherwise.  The paper's own antenna mesh and MBFs are not published, so every
workload here is synthetic, shaped like the paper's arrays (Section IV):
irregular arrays of identical printed elements and rooftop-meshed patches.
"""
from dataclasses import dataclass, field
import math

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass
class Substrate:
    eps_r: float
    h: float
    k0: float = TWO_PI

    @property
    def k_d(self):
        return self.k0 * math.sqrt(self.eps_r)


@dataclass
class ContourSpec:
    """Contour parameters: n samples on [0, beta_max]; parabola to beta_p of peak height."""
    n: int
    beta_max: float
    beta_p: float
    height: float

    @property
    def h(self):
        return self.beta_max / self.n


def default_contour(sub, n, height_in_steps=6.0, beta_max_factor=5.0, beta_p_factor=1.3):
    """beta_max = 5 k_d (Section III-A), beta_p ~ 1.3 k_d (beyond every surface-wave
    pole, which all lie in (k0, k_d)), peak height a few node spacings.  beta_p is
    moved to the nearest cell boundary m * beta_max / n so that the rectangle rule
    never straddles the corner where the parabola meets the real axis."""
    beta_max = beta_max_factor * sub.k_d
    step = beta_max / n
    beta_p = round(beta_p_factor * sub.k_d / step) * step
    return ContourSpec(n=n, beta_max=beta_max, beta_p=beta_p,
                       height=height_in_steps * step)


@dataclass
class Element:
    """Elementary basis functions of one element plus MBF coefficients q (B x M)."""
    kind: str                       # "strip" or "rooftop"
    q: np.ndarray                   # complex (B, M)
    cx: np.ndarray = None           # rooftop centres (B,)
    cy: np.ndarray = None
    direction: np.ndarray = None    # 0 = x, 1 = y
    half_len: np.ndarray = None
    width: np.ndarray = None
    length: float = None            # strip length / width
    strip_width: float = None

    @property
    def n_mbf(self):
        return self.q.shape[1]

    @property
    def n_basis(self):
        return self.q.shape[0]


def strip_element(length=0.45, width=0.02):
    """One cosine strip dipole, a single MBF (M = 1)."""
    return Element(kind="strip", q=np.ones((1, 1), dtype=np.complex128),
                   length=length, strip_width=width)


def patch_rooftops(n_side=10, pitch=0.05, n_mbf=4, seed=2):
    """Rooftop mesh of a 0.5 x 0.5 lambda0 patch: n_side^2 x-directed and n_side^2
    y-directed rooftops with centres on a square grid (-0.225 .. 0.225 for the
    defaults), half-length = width = pitch, and complex-normal MBF coefficients
    CN(0, 1) drawn with the given seed."""
    ax = (np.arange(n_side) - (n_side - 1) / 2.0) * pitch
    gx, gy = np.meshgrid(ax, ax, indexing="xy")
    cx = np.concatenate([gx.ravel(), gx.ravel()])
    cy = np.concatenate([gy.ravel(), gy.ravel()])
    b = cx.size
    direction = np.concatenate([np.zeros(n_side * n_side, dtype=np.int32),
                                np.ones(n_side * n_side, dtype=np.int32)])
    rng = np.random.default_rng(seed)
    q = (rng.standard_normal((b, n_mbf)) + 1j * rng.standard_normal((b, n_mbf))) / math.sqrt(2.0)
    return Element(kind="rooftop", q=q, cx=cx, cy=cy, direction=direction,
                   half_len=np.full(b, pitch), width=np.full(b, pitch))


def poisson_disc(n_points, radius, r_min, seed):
    """Random sequential adsorption in a disc: uniform darts, rejected when closer
    than r_min to an accepted point, until n_points are accepted.  Returns (n, 2)."""
    rng = np.random.default_rng(seed)
    cell = r_min / math.sqrt(2.0)
    n_cells = int(math.ceil(2.0 * radius / cell)) + 1
    grid = -np.ones((n_cells, n_cells), dtype=np.int64)
    pts = np.empty((n_points, 2))
    count = 0
    attempts = 0
    r2 = r_min * r_min
    while count < n_points:
        batch = rng.random((4096, 2))
        for u, v in batch:
            attempts += 1
            if attempts > 200 * n_points:
                raise RuntimeError("poisson_disc: too dense for r_min")
            rr = radius * math.sqrt(u)
            th = TWO_PI * v
            x, y = rr * math.cos(th), rr * math.sin(th)
            i = int((x + radius) / cell)
            j = int((y + radius) / cell)
            ok = True
            for di in range(-2, 3):
                ii = i + di
                if ii < 0 or ii >= n_cells:
                    continue
                for dj in range(-2, 3):
                    jj = j + dj
                    if jj < 0 or jj >= n_cells:
                        continue
                    k = grid[ii, jj]
                    if k >= 0:
                        dx = pts[k, 0] - x
                        dy = pts[k, 1] - y
                        if dx * dx + dy * dy < r2:
                            ok = False
                            break
                if not ok:
                    break
            if ok:
                pts[count] = (x, y)
                grid[i, j] = count
                count += 1
                if count == n_points:
                    break
    return pts


def rotations(n, seed):
    """Element rotations in {0, 1} (0 or 90 degrees), uniform."""
    return np.random.default_rng(seed).integers(0, 2, size=n).astype(np.int32)


def complex_normal(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


@dataclass
class TableWorkload:
    """One tabulation problem: substrate, element, contour, harmonics, rho grid."""
    name: str
    substrate: Substrate
    element: Element
    contour: ContourSpec
    q_max: int
    rho_max: float
    n_rho: int
    precision: str                  # "fp64" or "fp32"
    rotation_classes: int = 1
    extras: dict = field(default_factory=dict)

    @property
    def qs(self):
        return np.arange(-self.q_max, self.q_max + 1)

    @property
    def rho(self):
        return np.linspace(0.0, self.rho_max, self.n_rho)


def strip_fp64(n=1024, n_rho=1024, rho_max=10.0, q_max=4):
    """Strip-dipole pair on eps_r = 2.2, h = 0.05 lambda0; N = 1024; 1024 rho points to
    10 lambda0; harmonics |q| <= 4; complex128."""
    sub = Substrate(eps_r=2.2, h=0.05)
    return TableWorkload("strip-fp64", sub, strip_element(), default_contour(sub, n),
                         q_max, rho_max, n_rho, "fp64")


def patch_m4(n=16384, n_rho=8192, rho_max=50.0, q_max=16, precision="fp32",
             rotation_classes=1):
    """Rooftop patch, M = 4 MBFs from 200 rooftops, eps_r = 4.4, h = 0.03 lambda0;
    N = 16384; rho to 50 lambda0 (8192 points); |q| <= 16; all 16 MBF pairs."""
    sub = Substrate(eps_r=4.4, h=0.03)
    return TableWorkload("patch-m4", sub, patch_rooftops(), default_contour(sub, n),
                         q_max, rho_max, n_rho, precision, rotation_classes)


def irregular_array(n_elements=10000, radius=60.0, r_min=0.5, seed=3):
    """Poisson-disc positions (radius read as the disc radius) and rotations."""
    return poisson_disc(n_elements, radius, r_min, seed), rotations(n_elements, seed)


def sweep_items(n_freq=64, n_sub=8, seed=4, rho_max=50.0, oversample=3.0, f_lo=0.8, f_hi=1.2,
                n_base=4096, n_levels=5, height_in_steps=6.0, taylor_arg_max=3.0):
    """Batched sweep: n_freq frequencies (k0 = 2 pi f, lengths in wavelengths at the band
    centre) x n_sub substrates with eps_r ~ U[2, 10], h ~ U[0.02, 0.1] (seeded).  Each item
    gets its own contour: beta_max = 5 k_d, beta_p ~ 1.3 k_d on a cell boundary, and
    n = n_base * 2^u with u uniform in {0 .. n_levels-1}, raised until the s-period
    2 pi / step covers 2 rho_max `oversample` times (the 1-D form of the paper's sampling
    rule, Eq. 26).  The height is `height_in_steps` node spacings, capped so that
    height * rho_max <= taylor_arg_max: the contour samples enter the transform weighted
    by exp(beta_I s), up to exp(height * rho_max) at the largest distance, so their float32
    rounding grows by that factor (the small-gamma condition of the Taylor expansion,
    Section III-B-3).  On the coarsest contours the cap leaves about 2.9 spacings."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(2.0, 10.0, n_sub)
    hs = rng.uniform(0.02, 0.1, n_sub)
    freqs = np.linspace(f_lo, f_hi, n_freq)
    items = []
    for fi, f in enumerate(freqs):
        for si in range(n_sub):
            k0 = TWO_PI * f
            kd = k0 * math.sqrt(eps[si])
            beta_max = 5.0 * kd
            n = n_base * 2 ** int(rng.integers(0, n_levels))
            while TWO_PI / (beta_max / n) < 2.0 * rho_max * oversample:
                n *= 2
            step = beta_max / n
            items.append({"eps_r": float(eps[si]), "h": float(hs[si]), "k0": k0, "n": int(n),
                          "beta_max": beta_max, "beta_p": round(1.3 * kd / step) * step,
                          "height": min(height_in_steps * step, taylor_arg_max / rho_max),
                          "taylor_order": -1})
    return items
