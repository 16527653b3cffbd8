"""Pins of the oracle's 3D MRCM-OS path and of its interface solve.

The 3D decomposition (multi-index, 8-colour parity and its order), the 3D P1
functions {1, s, t} on the two tangential axes of a face, the interface rows
over 3D faces and the 3D smoothing sweeps are each checked against something
other than the oracle itself: the global fine solution (Prop. 2, smoothing
fixed point, exact linear pressures), and an independent dense mixed RT0
solver (``tests/_mixed_rt0.py``) for one whole smoothing step.  The last test
pins the equilibrated-LU interface solve against a refinement carried in
extended precision.
"""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I
from tests import _mixed_rt0 as MX


def _rand3d(n, seed, bc="left_right", sigma2=1.5):
    prob = I.lognormal_problem(n, sigma2=sigma2, corr_len=0.3, seed=seed, bc=bc)
    rng = np.random.default_rng(seed + 7)
    prob.f = rng.standard_normal(prob.f.shape)
    if bc == "noflow":
        prob.f -= prob.f.mean()
    return prob


def _const_problem(n, h, K0, kinds, values):
    return I.Problem(3, tuple(n), tuple(h), np.full(tuple(n)[::-1], K0), np.zeros(tuple(n)[::-1]),
                     tuple(kinds), tuple(values))


# ---------------------------------------------------------------------------
# Prop. 2 in 3D: l = 0 with the full fine-face trace spaces is the fine solution
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", ["left_right", "noflow"])
def test_prop2_3d_fine_trace_spaces_reproduce_fine_solution(bc):
    """Prop. 2 (Sec. 2.1) on an 8x8x4 grid split into 2x2x2 subdomains of
    4x4x2 cells: with l = 0 and Lambda^i_H = M_H = V_H = every fine-face
    indicator on the 3D skeleton, MRCM-O equals the global fine solution,
    with Dirichlet data and with pure-Neumann data (zero-mean pressure).
    Exercises the 3D multi-index, the interface rows over faces normal to
    each axis and the n^i.n sign on every axis."""
    prob = _rand3d((8, 8, 4), 31, bc=bc)
    pf, uf = O.fine_solve(prob)
    r = O.mrcm_os(prob, (4, 4, 2), 0, space="fine", alpha_basis=0.6)
    p = O.zero_mean(r.p) if bc == "noflow" else r.p
    pref = O.zero_mean(pf) if bc == "noflow" else pf
    assert r.counts["interface_rows"] == r.counts["interface_cols"]
    assert np.max(np.abs(p - pref)) < 1e-10 * np.max(np.abs(pref))
    assert np.max(np.abs(r.u - uf)) < 1e-10 * np.max(np.abs(uf))


# ---------------------------------------------------------------------------
# smoothing fixed point in 3D
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alpha_s", [0.3, 5.0])
def test_smoothing_fixed_point_3d(alpha_s):
    """Sec. 3 in 3D: the global fine solution is invariant under smoothing
    steps (its Robin data -beta u.n + pi on every d hat-Omega_i \\ d Omega,
    8 colours) for overlap 1, with two alpha_smooth values."""
    prob = _rand3d((8, 12, 8), 37)
    pf, uf = O.fine_solve(prob)
    p, u = O.smooth_from(prob, (4, 4, 4), 1, pf, uf, 2, alpha_smooth=alpha_s)
    assert np.max(np.abs(p - pf)) < 1e-11 * np.max(np.abs(pf))
    assert np.max(np.abs(u - uf)) < 1e-10 * np.max(np.abs(uf))


# ---------------------------------------------------------------------------
# 3D P1 = {1, s, t}: exact for linear pressures with constant K
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["z_dirichlet", "oblique_neumann"])
def test_mrcm_l0_p1_exact_for_linear_pressure_3d(case):
    """With l = 0, constant K and the P1 spaces {1, s, t} of Sec. 2.1 the
    Robin trace of a linear pressure is affine in both tangential
    coordinates of every face, so MRCM reproduces the fine solution (itself
    exact at cell centres).  'z_dirichlet': p = 1 on z = 0, p = 0 on z = L,
    no flow elsewhere -- on the x- and y-faces the trace varies along z, the
    second tangential axis, so a P1 space missing that coordinate fails.
    'oblique_neumann': pure Neumann data u.n = -K g.n with g = (0.3, -0.7,
    1.1), so p = g.x (zero mean) varies along every axis on every face.
    Anisotropic cells and subdomains (4x2x3 of 4x4x2 cells)."""
    n, h, K0 = (16, 8, 6), (0.07, 0.11, 0.05), 2.5
    if case == "z_dirichlet":
        kinds = (O.NEUMANN,) * 4 + (O.DIRICHLET, O.DIRICHLET)
        vals = (0.0,) * 4 + (1.0, 0.0)
        L = n[2] * h[2]
        g = np.array([0.0, 0.0, -1.0 / L])
    else:
        g = np.array([0.3, -0.7, 1.1])
        kinds = (O.NEUMANN,) * 6
        # outward u.n = -K g.n on each side
        vals = (K0 * g[0], -K0 * g[0], K0 * g[1], -K0 * g[1], K0 * g[2], -K0 * g[2])
    prob = _const_problem(n, h, K0, kinds, vals)
    pf, uf = O.fine_solve(prob)
    xc = (O.box_cells([0, 0, 0], n) + 0.5) * np.array(h)
    if case == "z_dirichlet":
        pex = 1.0 + xc @ g                  # 1 - z / L
        pref = pf
    else:
        pex = xc @ g
        pex = pex - pex.mean()
        pref = O.zero_mean(pf)
    assert np.max(np.abs(pref - pex)) < 1e-12
    r = O.mrcm_os(prob, (4, 4, 2), 0, space=1, alpha_basis=0.8)
    ep, eu = O.rel_errors(prob, r.p, r.u, pref, uf)
    assert ep < 1e-11 and eu < 1e-11, (ep, eu)
    # the same problem with P0 spaces is not exact: the pin is sensitive to
    # the P1 coordinates, not satisfied by any interface space
    r0 = O.mrcm_os(prob, (4, 4, 2), 0, space=0, alpha_basis=0.8)
    assert O.rel_errors(prob, r0.p, r0.u, pref, uf)[1] > 1e-4


def test_side_coordinates_3d_tangential_axes():
    """The two P1 coordinates of a 3D face are the affine centre coordinates
    along the tangential axes in ascending order, each over its own extent."""
    lo, hi = (2, 3, 1), (6, 5, 4)
    cells = O.box_cells(lo, hi)
    for a in range(3):
        sel = cells[cells[:, a] == lo[a]]
        tc = O.side_coordinates(sel, a, lo, hi)
        tang = [b for b in range(3) if b != a]
        assert len(tc) == 2
        for q, b in enumerate(tang):
            expect = 2.0 * (sel[:, b] + 0.5 - lo[b]) / (hi[b] - lo[b]) - 1.0
            assert np.allclose(tc[q], expect, rtol=0, atol=1e-15)
            assert tc[q].min() > -1 and tc[q].max() < 1


def test_decompose_3d_colours_and_sides():
    """3D multi-index (x fastest), Gamma_i sides and the 8 parity colours
    c = sum_a (i_a mod 2) 2^a: neighbours across any face differ in colour."""
    prob = _rand3d((12, 8, 8), 3)
    subs, M = O.decompose(prob, (4, 4, 4), 1)
    assert M == (3, 2, 2) and len(subs) == 12
    seen = set()
    for sd in subs:
        i = sd.multi
        assert sd.index == i[0] + 3 * (i[1] + 2 * i[2])
        assert sd.colour == (i[0] % 2) + 2 * (i[1] % 2) + 4 * (i[2] % 2)
        seen.add(sd.colour)
        for a in range(3):
            assert (2 * a in sd.sides) == (i[a] > 0)
            assert (2 * a + 1 in sd.sides) == (i[a] < M[a] - 1)
    assert seen == set(range(8))
    for s1 in subs:
        for s2 in subs:
            if sum(abs(s1.multi[a] - s2.multi[a]) for a in range(3)) == 1:
                assert s1.colour != s2.colour


# ---------------------------------------------------------------------------
# one 3D smoothing step recomputed with the independent mixed solver
# ---------------------------------------------------------------------------

def _mixed_local(prob, lo, hi, alpha, Hw, robin, sources):
    d = prob.dim
    sl = tuple(slice(lo[a], hi[a]) for a in range(d))[::-1]
    Kb = prob.K[sl]
    fb = prob.f[sl] if sources else np.zeros_like(prob.f[sl])
    shape = tuple(hi[a] - lo[a] for a in range(d))
    Kf = prob.K.reshape(-1)
    sides = []
    for sid in range(2 * d):
        a, s = sid // 2, sid % 2
        out = lo[a] - 1 if s == 0 else hi[a]
        if out < 0 or out >= prob.n[a]:
            v = prob.bc_value[sid] if sources else 0.0
            sides.append(("dirichlet" if prob.bc_kind[sid] == O.DIRICHLET else "neumann", v))
        else:
            cells = MX.side_cells(shape, sid) + np.array(lo)
            nb = cells.copy()
            nb[:, a] = out
            Kin = Kf[O.flat_index(cells, prob.n)]
            Kout = Kf[O.flat_index(nb, prob.n)]
            beta = alpha * Hw[a] * (Kin + Kout) / (2 * Kin * Kout)
            sides.append(("robin", beta, robin.get(sid, np.zeros(len(cells)))))
    return MX.solve_box(prob.h, Kb, fb, sides)


def test_bruteforce_smoothing_step_3d():
    """One 3D smoothing step (Sec. 3, Eqs. (sm_1)-(sm_2)) recomputed with the
    independent mixed solver: colours 0..7 of the parity colouring in
    increasing order; per subdomain Robin data -beta u.n + pi from the current
    state on d hat-Omega_i \\ d Omega (outward normal of hat-Omega_i, beta
    with alpha_smooth), a mixed solve on hat-Omega_i with the physical
    sources, and an overwrite of Omega_i.  3x2x2 subdomains, so colours hold
    one or two subdomains and the order of the colours decides the result."""
    prob = _rand3d((12, 8, 8), 41)
    sub, l, alpha_s = (4, 4, 4), 1, 1.0
    Hw = tuple(sub[a] * prob.h[a] for a in range(3))
    r = O.mrcm_os(prob, sub, l, space=0, alpha_basis=0.5, n_smooth=0)
    p, u = r.p.copy(), r.u.copy()
    subs, M = O.decompose(prob, sub, l)
    Kf = prob.K.reshape(-1)
    for colour in range(8):
        for sd in [s for s in subs if (s.multi[0] % 2) + 2 * (s.multi[1] % 2) + 4 * (s.multi[2] % 2) == colour]:
            shp = tuple(sd.hi_hat[a] - sd.lo_hat[a] for a in range(3))
            robin = {}
            for sid in range(6):
                a, s = sid // 2, sid % 2
                out = sd.lo_hat[a] - 1 if s == 0 else sd.hi_hat[a]
                if out < 0 or out >= prob.n[a]:
                    continue
                cells = MX.side_cells(shp, sid) + np.array(sd.lo_hat)
                g = O.flat_index(cells, prob.n)
                nb = cells.copy()
                nb[:, a] = out
                Kout = Kf[O.flat_index(nb, prob.n)]
                beta = alpha_s * Hw[a] * (Kf[g] + Kout) / (2 * Kf[g] * Kout)
                un = u[g, sid]
                robin[sid] = -beta * un + (p[g] - un * prob.h[a] / (2 * Kf[g]))
            ph, uh = _mixed_local(prob, sd.lo_hat, sd.hi_hat, alpha_s, Hw, robin, True)
            cells = O.box_cells(sd.lo, sd.hi)
            loc = sum((cells[:, a] - sd.lo_hat[a]) * int(np.prod(shp[:a])) for a in range(3))
            g = O.flat_index(cells, prob.n)
            p[g] = ph[loc]
            u[g] = uh[loc]
    p1, u1 = O.smooth_from(prob, sub, l, r.p, r.u, 1, alpha_smooth=alpha_s)
    assert np.max(np.abs(p1 - p)) < 1e-11 * np.max(np.abs(p))
    assert np.max(np.abs(u1 - u)) < 1e-10 * np.max(np.abs(u))


# ---------------------------------------------------------------------------
# the interface solve against a refinement in extended precision
# ---------------------------------------------------------------------------

def test_solve_square_matches_extended_precision_refinement():
    """The interface system of a high-contrast channel problem (128x128,
    contrast 1e4, 8x8 subdomains, overlap 4, P1; raw condition number near
    1e10 because flux and pressure rows differ in scale) solved by the
    oracle's equilibrated LU with FP64 refinement agrees with the solution
    refined with residuals and iterates carried in extended precision
    (numpy longdouble) to 1e-12 relative, entry by entry in max norm.  A
    plain unscaled LU solve of the same system is shown to be measurably
    further away, so the pin separates the two."""
    case = I.config_channel2d(n=128, n_smooth=0)
    r = O.mrcm_os(case.problem, case.partition.sub, case.partition.overlap, 1, 1.0, 1.0, 0)
    G, rhs, X = r.G, r.rhs, r.X
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended precision type on this platform")
    import scipy.linalg as sla
    Gl = G.astype(np.longdouble)
    bl = rhs.astype(np.longdouble)
    rr = 1.0 / np.abs(G).max(axis=1)
    Ge = G * rr[:, None]
    cc = 1.0 / np.abs(Ge).max(axis=0)
    lu = sla.lu_factor(Ge * cc[None, :])
    Xl = (cc * sla.lu_solve(lu, rr * rhs)).astype(np.longdouble)
    for _ in range(6):
        res = bl - Gl @ Xl
        Xl = Xl + (cc * sla.lu_solve(lu, rr * res.astype(np.float64))).astype(np.longdouble)
    Xl = Xl.astype(np.float64)
    scale = np.max(np.abs(Xl))
    err = np.max(np.abs(X - Xl)) / scale
    assert err < 1e-12, err
    Xplain = np.linalg.solve(G, rhs)
    assert np.max(np.abs(Xplain - Xl)) / scale > 3 * err
