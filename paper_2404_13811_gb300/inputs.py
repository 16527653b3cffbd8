"""Seeded synthetic inputs for Darcy problems (permeability fields, sources, boundary data).

This module holds no arithmetic of the multiscale method: it only draws the
problem data (K, f, boundary conditions, decomposition sizes) that both the
CUDA path and the CPU oracle consume.  Every field is a plain numpy array in
C order with shape ``n[::-1]`` (x fastest), i.e. ``(ny, nx)`` in 2D and
``(nz, ny, nx)`` in 3D.

The permeability generators stand in for the SPE10 layers the paper uses
(Sec. 4): a log-normal field with exponential covariance (the smooth upper
formation) and a channelised two-facies field (the fluvial lower formation).
No SPE10 value is reproduced.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NEUMANN = 0
DIRICHLET = 1


@dataclass
class Problem:
    """Darcy problem data on a Cartesian grid (Sec. 2, Eqs. (1a)-(1d)).

    n      -- cells per axis (x, y[, z])
    h      -- cell size per axis
    K      -- scalar cell permeability, shape n[::-1]
    f      -- source density (per unit volume), shape n[::-1]
    bc_kind, bc_value -- per side (x-, x+, y-, y+[, z-, z+]): NEUMANN with the
              outward normal velocity z, or DIRICHLET with the pressure g.
    """

    dim: int
    n: tuple
    h: tuple
    K: np.ndarray
    f: np.ndarray
    bc_kind: tuple
    bc_value: tuple

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))


@dataclass
class Partition:
    """Non-overlapping blocks of ``sub`` cells per axis, oversampled by ``overlap`` cells."""

    sub: tuple
    overlap: int


@dataclass
class MethodParams:
    """Interface space (0 = P0, 1 = P1), Robin parameters and smoothing steps."""

    space: int = 1
    alpha_basis: float = 1.0
    alpha_smooth: float = 1.0
    n_smooth: int = 0


@dataclass
class Case:
    problem: Problem
    partition: Partition
    params: MethodParams
    name: str = ""
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# random fields
# ----------------------------------------------------------------------------

def gaussian_field(n, h, sigma2, corr_len, rng):
    """Zero-mean Gaussian field with covariance sigma2*exp(-r/corr_len).

    Drawn by circulant embedding on a periodic grid padded to twice the size
    along each axis; negative eigenvalues of the embedding are clipped to zero.
    Returns (field shaped n[::-1], clipped fraction of the spectrum).
    """
    d = len(n)
    m = [2 * int(k) for k in n]
    axes = []
    for a in range(d):
        k = np.arange(m[a])
        k = np.minimum(k, m[a] - k)
        axes.append(k * h[a])
    # numpy axis order is reversed (x fastest)
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    r2 = sum(g * g for g in grids)
    c = sigma2 * np.exp(-np.sqrt(r2) / corr_len)
    lam = np.fft.fftn(c).real
    neg = lam < 0
    clipped = float(-lam[neg].sum() / np.abs(lam).sum()) if neg.any() else 0.0
    lam = np.where(neg, 0.0, lam)
    size = lam.size
    xi = rng.standard_normal(lam.shape) + 1j * rng.standard_normal(lam.shape)
    y = np.fft.fftn(np.sqrt(lam / size) * xi).real
    sl = tuple(slice(0, int(k)) for k in n[::-1])
    return np.ascontiguousarray(y[sl]), clipped


def channel_mask(n, width_range, area_fraction, rng, max_channels=400):
    """Boolean mask of sinusoidal channels running along x (2D) or along x in
    horizontal layers (3D).  Each channel has centre line
    y = y0 + A sin(2 pi x / wavelength + phase) and a width in cells drawn
    uniformly from ``width_range``; channels are added until the channel area
    reaches ``area_fraction`` of the grid."""
    d = len(n)
    nx, ny = int(n[0]), int(n[1])
    nz = int(n[2]) if d == 3 else 1
    mask = np.zeros((nz, ny, nx), dtype=bool)
    xs = np.arange(nx) + 0.5
    ys = np.arange(ny) + 0.5
    for _ in range(max_channels):
        if mask.mean() >= area_fraction:
            break
        w = rng.uniform(*width_range)
        y0 = rng.uniform(0, ny)
        amp = rng.uniform(0.05, 0.25) * ny
        wl = rng.uniform(0.5, 1.5) * nx
        ph = rng.uniform(0, 2 * math.pi)
        yc = y0 + amp * np.sin(2 * math.pi * xs / wl + ph)
        band = np.abs(ys[:, None] - yc[None, :]) < 0.5 * w  # (ny, nx)
        if d == 3:
            z0 = int(rng.integers(0, nz))
            thick = int(rng.integers(2, 6))
            mask[z0:z0 + thick] |= band[None]
        else:
            mask[0] |= band
    return mask if d == 3 else mask[0]


def lognormal_K(n, h, sigma2, corr_len, rng):
    y, clipped = gaussian_field(n, h, sigma2, corr_len, rng)
    return np.exp(y), clipped


def channelised_K(n, h, contrast, sigma2_bg, corr_len, rng, width_range=(4.0, 8.0),
                  area_fraction=0.25):
    y, clipped = gaussian_field(n, h, sigma2_bg, corr_len, rng)
    mask = channel_mask(n, width_range, area_fraction, rng)
    K = np.exp(y) * np.where(mask, contrast, 1.0)
    return K, clipped


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------

def _bc_left_right(dim):
    kind = [NEUMANN] * (2 * dim)
    val = [0.0] * (2 * dim)
    kind[0] = DIRICHLET
    val[0] = 1.0
    kind[1] = DIRICHLET
    val[1] = 0.0
    return tuple(kind), tuple(val)


def _bc_noflow(dim):
    return tuple([NEUMANN] * (2 * dim)), tuple([0.0] * (2 * dim))


def quarter_five_spot(n, h):
    """+1 / -1 cell-integrated rate at opposite corner cells (as a density)."""
    f = np.zeros(tuple(int(k) for k in n[::-1]))
    vol = float(np.prod(h))
    f.flat[0] = 1.0 / vol
    f.flat[-1] = -1.0 / vol
    return f


def homogeneous_problem(nx, ny=None):
    """The paper's homogeneous test (Sec. 4): K = 1 on the unit square,
    f = 8 pi^2 cos(2 pi x) cos(2 pi y), no-flow boundary, exact pressure
    cos(2 pi x) cos(2 pi y)."""
    ny = nx if ny is None else ny
    h = (1.0 / nx, 1.0 / ny)
    x = (np.arange(nx) + 0.5) * h[0]
    y = (np.arange(ny) + 0.5) * h[1]
    X, Y = np.meshgrid(x, y)
    f = 8 * math.pi ** 2 * np.cos(2 * math.pi * X) * np.cos(2 * math.pi * Y)
    kind, val = _bc_noflow(2)
    return Problem(2, (nx, ny), h, np.ones((ny, nx)), f, kind, val)


def lognormal_problem(n, sigma2=4.0, corr_len=0.1, seed=0, bc="left_right", source=None,
                      length=None):
    n = tuple(int(k) for k in n)
    d = len(n)
    L = length if length is not None else tuple([1.0] * d)
    h = tuple(L[a] / n[a] for a in range(d))
    rng = np.random.default_rng(seed)
    K, _ = lognormal_K(n, h, sigma2, corr_len, rng)
    f = np.zeros(n[::-1])
    if source == "q5":
        f = quarter_five_spot(n, h)
    kind, val = _bc_left_right(d) if bc == "left_right" else _bc_noflow(d)
    return Problem(d, n, h, K, f, kind, val)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def config_small(seed=101):
    """64x64 unit square, 4x4 subdomains of 16x16 oversampled by 2, P0 spaces,
    alpha = 1e-2 for the bases (alpha_smooth = 1), log-normal K (variance 4,
    correlation length 0.1), quarter-five-spot +/-1, no-flow boundary, 4 smoothing steps."""
    prob = lognormal_problem((64, 64), sigma2=4.0, corr_len=0.1, seed=seed, bc="noflow",
                             source="q5")
    return Case(prob, Partition((16, 16), 2), MethodParams(0, 1e-2, 1.0, 4),
                name="2d_64x64_q5_P0_l2")


def config_channel2d(n=512, seed=202, sub=16, overlap=4, n_smooth=8):
    """512x512 unit square, 32x32 subdomains of 16x16 oversampled by 4, P1
    spaces, channelised K (contrast 1e4, background log-normal variance 1),
    p = 1 / 0 on x = 0 / 1, no flow elsewhere, 8 smoothing steps."""
    nn = (n, n)
    h = (1.0 / n, 1.0 / n)
    rng = np.random.default_rng(seed)
    K, _ = channelised_K(nn, h, 1e4, 1.0, 0.1, rng)
    kind, val = _bc_left_right(2)
    prob = Problem(2, nn, h, K, np.zeros((n, n)), kind, val)
    return Case(prob, Partition((sub, sub), overlap), MethodParams(1, 1.0, 1.0, n_smooth),
                name=f"2d_{n}x{n}_channel_P1_l{overlap}")


def config_layered3d(n=(60, 220, 85), sub=(10, 10, 5), overlap=2, seed=303, n_upper=35,
                     n_smooth=4, space=0):
    """3D 60x220x85 cells, subdomains 10x10x5 oversampled by 2: layers z < 35
    log-normal (variance 5), layers z >= 35 channelised (contrast 1e6),
    p = 1 / 0 on the two faces normal to x, no flow elsewhere."""
    n = tuple(int(k) for k in n)
    h = tuple(1.0 / 60 for _ in range(3))
    rng = np.random.default_rng(seed)
    y, _ = gaussian_field(n, h, 5.0, 0.1 * n[0] * h[0], rng)
    K = np.exp(y)
    nz_low = n[2] - n_upper
    if nz_low > 0:
        ylow, _ = gaussian_field((n[0], n[1], nz_low), h, 1.0, 0.1 * n[0] * h[0], rng)
        mask = channel_mask((n[0], n[1], nz_low), (4.0, 8.0), 0.25, rng)
        K[n_upper:] = np.exp(ylow) * np.where(mask, 1e6, 1.0)
    kind, val = _bc_left_right(3)
    prob = Problem(3, n, h, K, np.zeros(n[::-1]), kind, val)
    return Case(prob, Partition(tuple(sub), overlap), MethodParams(space, 1.0, 1.0, n_smooth),
                name=f"3d_{n[0]}x{n[1]}x{n[2]}_layered_P{space}_l{overlap}")


def config_ensemble(count=256, seed=404, nmin=128, nmax=512, sub=16):
    """Ensemble of independent 2D problems: sizes n = 16*round(exp(U[ln nmin, ln nmax])/16),
    each its own log-normal K (variance U[2, 6]), overlap U{2, 3, 4}, P1, 4 smoothing steps."""
    rng = np.random.default_rng(seed)
    cases = []
    for m in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / sub)) * sub
        n = max(n, 2 * sub)
        s2 = float(rng.uniform(2.0, 6.0))
        l = int(rng.integers(2, 5))
        prob = lognormal_problem((n, n), sigma2=s2, corr_len=0.1, seed=seed * 1000 + m)
        cases.append(Case(prob, Partition((sub, sub), l), MethodParams(1, 1.0, 1.0, 4),
                          name=f"ens{m}_{n}"))
    return cases


def sink_cells(n, sub, count, seed, min_dist=2):
    """Cells at least ``min_dist`` cells away from every subdomain boundary."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        c = tuple(int(rng.integers(0, n[a])) for a in range(len(n)))
        ok = all(min_dist <= (c[a] % sub[a]) < sub[a] - min_dist for a in range(len(n)))
        if ok and c not in out:
            out.append(c)
    return out


def config_adjoint(n=256, seed=505, sub=16, overlap=4, n_smooth=6):
    """256x256, 16x16 subdomains oversampled by 4, P1, log-normal K (variance 4),
    8 sink cells of rate -1/8, 6 smoothing steps; the loss target comes from a
    second K drawn from seed + 1."""
    prob = lognormal_problem((n, n), sigma2=4.0, corr_len=0.1, seed=seed)
    sinks = sink_cells((n, n), (sub, sub), 8, seed + 7)
    vol = prob.h[0] * prob.h[1]
    for (ix, iy) in sinks:
        prob.f[iy, ix] = -1.0 / 8.0 / vol
    target = lognormal_problem((n, n), sigma2=4.0, corr_len=0.1, seed=seed + 1)
    target.f[...] = prob.f
    return Case(prob, Partition((sub, sub), overlap), MethodParams(1, 1.0, 1.0, n_smooth),
                name=f"2d_{n}x{n}_adjoint", extra={"sinks": sinks, "target_problem": target})
