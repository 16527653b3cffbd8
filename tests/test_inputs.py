"""The seeded input recipe: the generators draw what the workloads state.

* Gaussian log K: zero mean, variance sigma^2 and the exponential covariance
  sigma^2 exp(-r / l) at one-cell lags, over an ensemble of fields;
* channel masks: channel area reaches the stated fraction (25%) and stops
  within one channel of it;
* the workloads: grid sizes, partitions, subdomain counts, spaces, smoothing
  steps, boundary data, sources (quarter five-spot, sink rates) and ensemble
  size ranges.
"""
import math

import numpy as np
import pytest

from paper_2404_13811_gb300 import inputs as I


def test_gaussian_field_has_the_exponential_covariance():
    n, h, s2, ell = (48, 48), (1.0 / 48, 1.0 / 48), 2.0, 0.1
    rng = np.random.default_rng(11)
    ys = np.stack([I.gaussian_field(n, h, s2, ell, rng)[0] for _ in range(300)])
    assert abs(ys.mean()) < 0.05 * math.sqrt(s2)
    var = ys.var(axis=0).mean()
    assert abs(var - s2) < 0.06 * s2, var
    for ax, lag_h in ((2, h[0]), (1, h[1])):
        a = np.take(ys, range(0, n[0] - 1), axis=ax)
        b = np.take(ys, range(1, n[0]), axis=ax)
        cov = (a * b).mean()
        assert abs(cov - s2 * math.exp(-lag_h / ell)) < 0.06 * s2, (ax, cov)
    # two cells apart along x
    cov2 = (ys[:, :, :-2] * ys[:, :, 2:]).mean()
    assert abs(cov2 - s2 * math.exp(-2 * h[0] / ell)) < 0.06 * s2


@pytest.mark.parametrize("dim", [2, 3])
def test_channel_area_fraction(dim):
    n = (96, 64) if dim == 2 else (48, 40, 12)
    rng = np.random.default_rng(12 + dim)
    m = I.channel_mask(n, (4.0, 8.0), 0.25, rng)
    frac = m.mean()
    assert 0.25 <= frac < 0.45, frac


def test_channel2d_workload():
    case = I.config_channel2d()
    p, part, pm = case.problem, case.partition, case.params
    assert p.dim == 2 and tuple(p.n) == (512, 512) and p.ncells == 262144
    assert tuple(part.sub) == (16, 16) and part.overlap == 4
    assert pm.space == 1 and pm.n_smooth == 8 and pm.alpha_basis == 1.0 and pm.alpha_smooth == 1.0
    assert (512 // 16) ** 2 == 1024
    assert p.K.max() / p.K.min() > 1e4 and np.all(np.isfinite(p.K)) and np.all(p.K > 0)
    assert not np.any(p.f)
    # p = 1 on x = 0, p = 0 on x = 1 (Dirichlet), no flow on the y sides
    assert p.bc_kind[0] == I.DIRICHLET and p.bc_kind[1] == I.DIRICHLET
    assert (p.bc_value[0], p.bc_value[1]) == (1.0, 0.0)
    assert p.bc_kind[2] == I.NEUMANN and p.bc_kind[3] == I.NEUMANN


def test_small_workload_quarter_five_spot():
    case = I.config_small()
    p, part, pm = case.problem, case.partition, case.params
    assert tuple(p.n) == (64, 64) and tuple(part.sub) == (16, 16) and part.overlap == 2
    assert pm.space == 0 and pm.alpha_basis == 1e-2 and pm.alpha_smooth == 1.0 and pm.n_smooth == 4
    vol = p.h[0] * p.h[1]
    nz = np.argwhere(p.f != 0)
    assert len(nz) == 2
    assert p.f[0, 0] * vol == pytest.approx(1.0) and p.f[63, 63] * vol == pytest.approx(-1.0)
    assert all(k == I.NEUMANN for k in p.bc_kind[:4])


def test_adjoint_workload_sinks():
    case = I.config_adjoint()
    p, part = case.problem, case.partition
    assert tuple(p.n) == (256, 256) and tuple(part.sub) == (16, 16) and part.overlap == 4
    sinks = case.extra["sinks"]
    assert len(sinks) == 8 and len(set(sinks)) == 8
    vol = p.h[0] * p.h[1]
    for (ix, iy) in sinks:
        assert 2 <= ix % 16 < 14 and 2 <= iy % 16 < 14
        assert p.f[iy, ix] * vol == pytest.approx(-1.0 / 8.0)
    assert np.count_nonzero(p.f) == 8
    t = case.extra["target_problem"]
    assert np.array_equal(t.f, p.f) and not np.array_equal(t.K, p.K)


def test_layered3d_workload_shape():
    case = I.config_layered3d()
    p, part = case.problem, case.partition
    assert tuple(p.n) == (60, 220, 85) and p.ncells == 1122000
    M = [p.n[a] // part.sub[a] for a in range(3)]
    assert M == [6, 22, 17] and M[0] * M[1] * M[2] == 2244
    # channelised upper layers (contrast 1e6) over the log-normal lower part
    upper, lower = p.K[35:], p.K[:35]
    assert upper.max() / np.median(upper) > 1e4
    assert lower.max() / lower.min() < upper.max() / upper.min()


def test_ensemble_sizes():
    cases = I.config_ensemble()
    assert len(cases) == 256
    sizes = [c.problem.n[0] for c in cases]
    assert all(s % 16 == 0 and 128 <= s <= 512 for s in sizes)
    assert {c.partition.overlap for c in cases} <= {2, 3, 4}
    assert all(c.problem.n[0] == c.problem.n[1] for c in cases)
    total = sum(c.problem.ncells for c in cases)
    assert 1.5e7 < total < 3.5e7, total
