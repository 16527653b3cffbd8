"""Pins of the oracle's discrete adjoint (dL/dlog K of MRCM-OS).

* Complex step: for a real-analytic forward map F, Im F(theta + i t e_j) / t
  equals dF/dtheta_j to O(t^2) with no cancellation, so with t = 1e-30 it is
  exact to rounding.  Run through the forward oracle itself (complex K), it
  checks every component of the hand-written reverse pass.
* Homogeneity in K: the face laws are homogeneous of degree one in K
  (T, 1/beta and the Dirichlet T all scale with K), so under K -> c K
  - with no source and nonzero Dirichlet data, p is unchanged and u scales
    by c:  sum_j dp/dtheta_j = 0, sum_j du/dtheta_j = u;
  - with a source and zero Dirichlet data, p scales by 1/c and u is
    unchanged:  sum_j dp/dtheta_j = -p, sum_j du/dtheta_j = 0,
  for MRCM-O and for every smoothing step (the interface coefficients and the
  Robin data scale consistently).
"""
import dataclasses

import numpy as np
import pytest

from oracle import mrcm_adjoint as AD
from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I


def _problem(n, seed, source=True, g=(1.0, 0.0), sigma2=2.0):
    prob = I.lognormal_problem(n, sigma2=sigma2, corr_len=0.2, seed=seed)
    rng = np.random.default_rng(seed + 5)
    prob.f = rng.standard_normal(prob.f.shape) if source else np.zeros(prob.f.shape)
    bv = list(prob.bc_value)
    bv[0], bv[1] = g
    prob.bc_value = tuple(bv)
    return prob


def _seeds(prob, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(prob.ncells), rng.standard_normal((prob.ncells, 2 * prob.dim))


def _loss(res, wp, wu):
    return np.sum(wp * res.p) + np.sum(wu * res.u)


def _complex_step(prob, j, args, wp, wu, t=1e-30):
    Kc = prob.K.astype(complex)
    Kc.reshape(-1)[j] *= np.exp(1j * t)
    pc = dataclasses.replace(prob, K=Kc)
    return np.imag(_loss(O.mrcm_os(pc, *args), wp, wu)) / t


@pytest.mark.parametrize("space,overlap,n_smooth,alphas", [
    (1, 2, 2, (1.0, 1.0)),
    (0, 0, 1, (0.5, 2.0)),
])
def test_adjoint_matches_complex_step_on_every_parameter(space, overlap, n_smooth, alphas):
    """16x16 cells in 2x2 subdomains of 8x8: every cell's log K, every kind
    of face (interior, Gamma, Robin box sides with and without oversampling,
    Dirichlet and Neumann sides), both smoothing colours of each parity."""
    prob = _problem((16, 16), seed=11 + space)
    wp, wu = _seeds(prob, 3)
    args = ((8, 8), overlap, space, alphas[0], alphas[1], n_smooth)
    _, g = AD.mrcm_os_adjoint(prob, *args, wp, wu)
    cs = np.array([_complex_step(prob, j, args, wp, wu) for j in range(prob.ncells)])
    scale = np.max(np.abs(cs))
    assert scale > 0
    assert np.max(np.abs(g - cs)) <= 1e-9 * scale, np.max(np.abs(g - cs)) / scale


def test_adjoint_matches_complex_step_with_many_subdomains():
    """24x24 cells in 4x4 subdomains of 6x6 oversampled by 2 (interior
    subdomains with four Gamma sides), P1, three smoothing steps; 60 seeded
    parameters."""
    prob = _problem((24, 24), seed=21)
    wp, wu = _seeds(prob, 4)
    args = ((6, 6), 2, 1, 1.0, 1.0, 3)
    _, g = AD.mrcm_os_adjoint(prob, *args, wp, wu)
    js = np.random.default_rng(8).choice(prob.ncells, 60, replace=False)
    cs = np.array([_complex_step(prob, j, args, wp, wu) for j in js])
    scale = np.max(np.abs(cs))
    assert np.max(np.abs(g[js] - cs)) <= 1e-9 * scale


@pytest.mark.parametrize("n_smooth", [0, 2])
@pytest.mark.parametrize("case", ["boundary_driven", "source_driven"])
def test_gradient_sum_follows_homogeneity_in_K(case, n_smooth):
    src = case == "source_driven"
    prob = _problem((32, 32), seed=31, source=src, g=(0.0, 0.0) if src else (1.0, -0.5))
    args = ((8, 8), 2, 1, 1.0, 1.0, n_smooth)
    wp, wu = _seeds(prob, 6)
    res, g = AD.mrcm_os_adjoint(prob, *args, wp, wu)
    total = np.sum(g)
    expect = -np.sum(wp * res.p) if src else np.sum(wu * res.u)
    mag = np.sum(np.abs(wp * res.p)) + np.sum(np.abs(wu * res.u))
    assert abs(total - expect) <= 1e-10 * mag, (total, expect)


def test_adjoint_refuses_pure_neumann():
    prob = I.config_small().problem
    with pytest.raises(NotImplementedError):
        AD.mrcm_os_adjoint(prob, (16, 16), 2, 0, 1.0, 1.0, 0,
                           np.zeros(prob.ncells), np.zeros((prob.ncells, 4)))


def _complex_step_variant(prob, j, args, wp, wu, t=1e-30):
    Kc = prob.K.astype(complex)
    Kc.reshape(-1)[j] *= np.exp(1j * t)
    pc = dataclasses.replace(prob, K=Kc)
    return np.imag(_loss(O.mrcm_os(pc, *args, particular="hat"), wp, wu)) / t


@pytest.mark.parametrize("space,overlap,n_smooth,alphas", [
    (1, 2, 2, (1.0, 1.0)),
    (0, 2, 1, (0.5, 2.0)),
])
def test_adjoint_of_hat_particular_variant_matches_complex_step(space, overlap, n_smooth, alphas):
    """The particular problem on hat-Omega_i (particular="hat"): its reverse
    pass (a source solve on the basis box, its face pressure in the pressure
    rows) against the complex step of the forward variant on every parameter."""
    prob = _problem((16, 16), seed=11 + space)
    wp, wu = _seeds(prob, 3)
    args = ((8, 8), overlap, space, alphas[0], alphas[1], n_smooth)
    _, g = AD.mrcm_os_adjoint(prob, *args, wp, wu, particular="hat")
    cs = np.array([_complex_step_variant(prob, j, args, wp, wu) for j in range(prob.ncells)])
    scale = np.max(np.abs(cs))
    assert np.max(np.abs(g - cs)) <= 1e-9 * scale, np.max(np.abs(g - cs)) / scale
