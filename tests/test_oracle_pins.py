"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test would fail under a plausible slip in the oracle (a dropped face
term, a wrong sign of the normal or of n^i.n, a transposed index, a wrong
harmonic mean, the Robin data of the smoothing built with the wrong normal).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I
from tests import _mixed_rt0 as MX

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(n, seed, bc="left_right", sigma2=2.0, h=None):
    prob = I.lognormal_problem(n, sigma2=sigma2, corr_len=0.2, seed=seed, bc=bc)
    if h is not None:
        prob.h = tuple(h)
    rng = np.random.default_rng(seed + 99)
    prob.f = rng.standard_normal(prob.f.shape)
    return prob


# ---------------------------------------------------------------------------
# 1. cell-centred reduction vs an independent mixed RT0 saddle-point solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_ccfd_matches_mixed_rt0_with_all_face_kinds(dim):
    """Sec. 2.2: RT0 + trapezoid/midpoint quadrature equals the cell-centred
    system.  Box with Robin faces (beta from alpha H / K_H), a Dirichlet
    side, a Neumann side with nonzero flux, random K and f, anisotropic h."""
    n = (12, 10) if dim == 2 else (6, 5, 4)
    h = (0.11, 0.07) if dim == 2 else (0.1, 0.13, 0.05)
    prob = _rand_problem(n, 5, h=h)
    kind = list(prob.bc_kind)
    val = list(prob.bc_value)
    kind[2] = O.NEUMANN
    val[2] = 0.37          # inflow/outflow through y-
    kind[0] = O.DIRICHLET
    val[0] = 1.3
    prob.bc_kind, prob.bc_value = tuple(kind), tuple(val)
    # interior box touching x- (Dirichlet) and y- (Neumann); other sides Robin
    lo = tuple([0] * dim)
    hi = tuple(k - 3 for k in n)
    Hw = tuple(4 * h[a] for a in range(dim))
    alpha = 0.7
    sysm = O.assemble_box(prob, lo, hi, alpha, Hw)
    rng = np.random.default_rng(1)
    robin = {}
    sides = []
    shape = sysm.shape
    Kb = prob.K[tuple(slice(lo[a], hi[a]) for a in range(dim))[::-1]]
    fb = prob.f[tuple(slice(lo[a], hi[a]) for a in range(dim))[::-1]]
    for sid in range(2 * dim):
        a, s = sid // 2, sid % 2
        sd = sysm.sides[sid]
        if sd.kind == "robin":
            lam = rng.standard_normal(len(sd.local))
            robin[sid] = lam
            # beta recomputed here from its definition: alpha H / harmonic(K_in, K_out)
            cells = MX.side_cells(shape, sid) + np.array(lo)
            nb = cells.copy()
            nb[:, a] += 1 if s == 1 else -1
            Kin = prob.K.reshape(-1)[O.flat_index(cells, prob.n)]
            Kout = prob.K.reshape(-1)[O.flat_index(nb, prob.n)]
            beta = alpha * Hw[a] * (Kin + Kout) / (2 * Kin * Kout)
            sides.append(("robin", beta, lam))
        elif sd.kind == "dirichlet":
            sides.append(("dirichlet", val[sid]))
        else:
            sides.append(("neumann", val[sid]))
    b = O.box_rhs(prob, sysm, robin, True)
    p = np.linalg.solve(sysm.A.toarray(), b)
    u = O.box_velocities(prob, sysm, p, robin, True)
    p_ref, u_ref = MX.solve_box(prob.h, Kb, fb, sides)
    assert np.max(np.abs(p - p_ref)) <= 1e-12 * np.max(np.abs(p_ref))
    assert np.max(np.abs(u - u_ref)) <= 1e-12 * np.max(np.abs(u_ref))


# ---------------------------------------------------------------------------
# 2. closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_fine_solution_exact_for_linear_pressure(dim):
    """Constant K, p = 1 on x = 0, p = 0 on x = L, no flow elsewhere:
    p(x) = 1 - x / L exactly at cell centres and u = K / L on every x-face."""
    n = (10, 6) if dim == 2 else (8, 4, 3)
    h = (0.1, 0.2) if dim == 2 else (0.125, 0.3, 0.2)
    K0 = 3.7
    prob = I.Problem(dim, n, h, np.full(n[::-1], K0), np.zeros(n[::-1]),
                     *I._bc_left_right(dim))
    p, u = O.fine_solve(prob)
    L = n[0] * h[0]
    x = (O.box_cells([0] * dim, n)[:, 0] + 0.5) * h[0]
    assert np.max(np.abs(p - (1 - x / L))) < 1e-13
    assert np.max(np.abs(u[:, 1] - K0 / L)) < 1e-12
    assert np.max(np.abs(u[:, 0] + K0 / L)) < 1e-12
    assert np.max(np.abs(u[:, 2:])) < 1e-12


def test_fine_solution_second_order_on_homogeneous_problem():
    """Sec. 4 homogeneous problem: K = 1, f = 8 pi^2 cos cos, no flow; the
    exact pressure is cos(2 pi x) cos(2 pi y).  The cell-centred RT0
    solution converges at O(h^2) at cell centres."""
    errs = []
    for n in (16, 32, 64):
        prob = I.homogeneous_problem(n)
        p, _ = O.fine_solve(prob)
        c = (O.box_cells([0, 0], (n, n)) + 0.5) / n
        pex = np.cos(2 * math.pi * c[:, 0]) * np.cos(2 * math.pi * c[:, 1])
        errs.append(np.sqrt(np.mean((p - pex) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_mrcm_l0_p1_exact_for_linear_pressure():
    """With l = 0 and P1 spaces the Robin trace of a linear pressure field
    with constant K is P1 on every edge, so MRCM reproduces it exactly."""
    n = (24, 16)
    prob = I.Problem(2, n, (1 / 24, 1 / 16), np.full(n[::-1], 2.0), np.zeros(n[::-1]),
                     *I._bc_left_right(2))
    pf, uf = O.fine_solve(prob)
    r = O.mrcm_os(prob, (8, 8), 0, space=1, alpha_basis=1.0)
    ep, eu = O.rel_errors(prob, r.p, r.u, pf, uf)
    assert ep < 1e-12 and eu < 1e-12


# ---------------------------------------------------------------------------
# 3. structural identities
# ---------------------------------------------------------------------------

def test_prop1_dimension_count_and_cost_table():
    """Prop. 1 (dim M_H = dim V_H, sum_i dim Lambda^i = dim M_H + dim V_H)
    and Table cost_table: NLC per interior subdomain, local problem size and
    interface size, for 20x20 local grids."""
    tab = json.load(open(os.path.join(GOLDEN, "cost_table.json")))
    M = 4
    prob = _rand_problem((20 * M, 20 * M), 11)
    for row in tab["rows"]:
        r = O.mrcm_os(prob, (20, 20), row["l"], space=row["space"], alpha_basis=1.0,
                      n_smooth=row["kS"])
        subs = r.subs
        interior = [sd for sd in subs if len(sd.sides) == 4]
        for sd in interior:
            assert r.counts["local_solves"][sd.index] == row["NLC"], row
            lp = [sd.hi_hat[a] - sd.lo_hat[a] for a in range(2)]
            assert lp == row["LP"], row
        npsi = 1 if row["space"] == 0 else 2
        dim_MH = npsi * r.counts["edges"]
        assert r.counts["interface_rows"] == 2 * dim_MH          # M rows + V rows
        assert r.counts["interface_cols"] == 2 * dim_MH          # sum_i N_i
        expect = {"4M(M-1)": 4 * M * (M - 1), "2M(M-1)": 2 * M * (M - 1)}[row["IP"]]
        assert dim_MH == expect, row


@pytest.mark.parametrize("overlap", [1, 2, 3])
def test_remark_mbf_equals_restriction(overlap):
    """Remark after Eq. (uhatphat): the Omega_i problem with Robin data phi_k
    on Gamma_i is solved by the restriction of the hat-Omega_i solution."""
    prob = _rand_problem((24, 24), 3)
    r = O.mrcm_os(prob, (8, 8), overlap, space=1, alpha_basis=0.3)
    Hw = (8 * prob.h[0], 8 * prob.h[1])
    for sd in r.subs[:5]:
        sys_i = O.assemble_box(prob, sd.lo, sd.hi, 0.3, Hw)
        for k in range(len(sd.data["Psi"])):
            lam = {sid: sd.data["PHI"][k][sid] for sid in sd.sides}
            b = O.box_rhs(prob, sys_i, lam, sources=False)
            p = np.linalg.solve(sys_i.A.toarray(), b)
            u = O.box_velocities(prob, sys_i, p, lam, sources=False)
            assert np.max(np.abs(p - sd.data["Psi"][k])) < 1e-11 * np.max(np.abs(p))
            assert np.max(np.abs(u - sd.data["U"][k])) < 1e-10 * np.max(np.abs(u))


@pytest.mark.parametrize("bc", ["left_right", "noflow"])
def test_prop2_fine_trace_spaces_reproduce_fine_solution(bc):
    """Prop. 2: with l = 0 and M_H = V_H = Lambda^i_H = all fine-face
    functions on the skeleton, MRCM-O equals the global fine solution."""
    prob = _rand_problem((16, 12), 7, bc=bc)
    if bc == "noflow":
        prob.f -= prob.f.mean()
    pf, uf = O.fine_solve(prob)
    r = O.mrcm_os(prob, (4, 4), 0, space="fine", alpha_basis=0.5)
    p = O.zero_mean(r.p) if bc == "noflow" else r.p
    pref = O.zero_mean(pf) if bc == "noflow" else pf
    assert np.max(np.abs(p - pref)) < 1e-11 * np.max(np.abs(pref))
    assert np.max(np.abs(r.u - uf)) < 1e-10 * np.max(np.abs(uf))


@pytest.mark.parametrize("overlap,alpha", [(1, 1.0), (2, 0.05), (3, 20.0)])
def test_smoothing_fixed_point(overlap, alpha):
    """Sec. 3: the global fine solution is invariant under a smoothing step
    (its Robin data on d hat-Omega_i reproduce it on every hat-Omega_i)."""
    prob = _rand_problem((24, 16), 13)
    pf, uf = O.fine_solve(prob)
    p, u = O.smooth_from(prob, (8, 8), overlap, pf, uf, 2, alpha_smooth=alpha)
    assert np.max(np.abs(p - pf)) < 1e-11 * np.max(np.abs(pf))
    assert np.max(np.abs(u - uf)) < 1e-10 * np.max(np.abs(uf))


def test_error_falls_with_overlap_and_smoothing_steps():
    """Secs. 4.2-4.3 on the paper's homogeneous problem (K = 1, cos cos
    source, no flow; 8x8 subdomains, P1, alpha = 1): the MRCM-O flux error
    against the fine solution falls as the overlap grows, and the flux error
    falls with every smoothing step (to well over an order of magnitude
    after four steps)."""
    prob = I.homogeneous_problem(64)
    pf, uf = O.fine_solve(prob)
    pf = O.zero_mean(pf)
    e_l = []
    for l in (1, 2, 3):
        r = O.mrcm_os(prob, (8, 8), l, space=1, alpha_basis=1.0)
        e_l.append(O.rel_errors(prob, r.p, r.u, pf, uf)[1])
    assert e_l[2] < e_l[1] < e_l[0], e_l
    r = O.mrcm_os(prob, (8, 8), 2, space=1, alpha_basis=1.0, n_smooth=6, keep_stages=True)
    errs = [O.rel_errors(prob, *r.stages[k], pf, uf)[1]
            for k in ["mrcm_o"] + [f"smooth{i}" for i in range(1, 7)]]
    assert all(errs[i + 1] < errs[i] for i in range(6)), errs
    assert errs[4] < 0.05 * errs[0], errs


def test_informed_space_misses_inhomogeneous_dirichlet_data():
    """Eq. (oversampling_problem) gives the informed-space problems
    homogeneous physical data, so for l > 0 a subdomain whose oversampled box
    reaches a Dirichlet side with g != 0 cannot represent the exact Robin
    trace: MRCM-O loses the l = 0 exactness for a linear pressure, the error
    sits in the subdomains next to that side, and smoothing removes it."""
    n = (64, 64)
    prob = I.Problem(2, n, (1 / 64, 1 / 64), np.ones(n), np.zeros(n), *I._bc_left_right(2))
    pf, uf = O.fine_solve(prob)
    r0 = O.mrcm_os(prob, (16, 16), 0, space=1, alpha_basis=1.0)
    assert O.rel_errors(prob, r0.p, r0.u, pf, uf)[1] < 1e-6
    r = O.mrcm_os(prob, (16, 16), 2, space=1, alpha_basis=1.0, n_smooth=4, keep_stages=True)
    err = np.abs(r.stages["mrcm_o"][1] - uf).max(axis=1).reshape(64, 64)
    blk = err.reshape(4, 16, 4, 16).max(axis=(1, 3))
    assert blk[:, 0].min() > 10 * blk[:, 2:].max()
    e0 = O.rel_errors(prob, *r.stages["mrcm_o"], pf, uf)[1]
    e4 = O.rel_errors(prob, r.p, r.u, pf, uf)[1]
    assert e4 < 1e-2 * e0


def test_mass_conservation_every_stage():
    """Eq. (12d) holds cell by cell with each cell's own face velocities
    after MRCM-O and after every smoothing step."""
    prob = _rand_problem((32, 32), 17)
    r = O.mrcm_os(prob, (8, 8), 2, space=1, alpha_basis=1.0, n_smooth=2, keep_stages=True)
    for key, (p, u) in r.stages.items():
        scale = max(np.max(np.abs(prob.f)) * np.prod(prob.h), np.max(np.abs(u)) * prob.h[0])
        assert np.max(np.abs(O.mass_residual(prob, u))) < 1e-12 * scale, key


def test_smoothing_is_additive_in_steps():
    prob = _rand_problem((24, 24), 19)
    r = O.mrcm_os(prob, (8, 8), 2, space=0, alpha_basis=1.0, n_smooth=0)
    p3, u3 = O.smooth_from(prob, (8, 8), 2, r.p, r.u, 3)
    p1, u1 = O.smooth_from(prob, (8, 8), 2, r.p, r.u, 1)
    p12, u12 = O.smooth_from(prob, (8, 8), 2, p1, u1, 2)
    assert np.array_equal(p3, p12) and np.array_equal(u3, u12)


# ---------------------------------------------------------------------------
# 4. brute force: the monolithic MRCM-O system (11d)-(14d) on a tiny case
# ---------------------------------------------------------------------------

def _mixed_local(prob, lo, hi, alpha, Hw, robin, sources):
    """Local solve through the independent mixed solver; robin: sid -> lam."""
    d = prob.dim
    sl = tuple(slice(lo[a], hi[a]) for a in range(d))[::-1]
    Kb = prob.K[sl]
    fb = prob.f[sl] if sources else np.zeros_like(prob.f[sl])
    shape = tuple(hi[a] - lo[a] for a in range(d))
    sides = []
    Kf = prob.K.reshape(-1)
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
    return MX.solve_box(prob.h, Kb, fb, sides), sides


@pytest.mark.parametrize("space,bc", [(0, "left_right"), (1, "left_right"), (1, "noflow")])
def test_bruteforce_monolithic_mrcm_o(space, bc):
    """Eqs. (11d)-(14d) assembled as one linear system -- local mixed
    unknowns of every Omega_i, Robin data lambda^i = sum_j X_j phi_j from
    informed functions computed by the independent mixed solver on
    hat-Omega_i, flux and pressure continuity rows -- on 2x2 subdomains of
    4x4 cells, solved densely, against the oracle's superposition."""
    prob = _rand_problem((8, 8), 23, bc=bc)
    if bc == "noflow":
        prob.f -= prob.f.mean()
    sub, l, alpha = (4, 4), 1, 0.8
    Hw = (4 * prob.h[0], 4 * prob.h[1])
    vol = prob.h[0] * prob.h[1]
    subs, M = O.decompose(prob, sub, l)
    # informed functions phi_k on Gamma_i from hat-Omega_i mixed solves
    phis = []
    for sd in subs:
        shp = tuple(sd.hi_hat[a] - sd.lo_hat[a] for a in range(2))
        lst = []
        for sid in sd.sides:
            a = sid // 2
            cells = MX.side_cells(shp, sid) + np.array(sd.lo_hat)
            tcoord = 2 * (cells[:, 1 - a] + 0.5 - sd.lo_hat[1 - a]) / (sd.hi_hat[1 - a] - sd.lo_hat[1 - a]) - 1
            fun = [np.ones(len(cells))] + ([tcoord] if space == 1 else [])
            for g in fun:
                (p, u), _ = _mixed_local(prob, sd.lo_hat, sd.hi_hat, alpha, Hw, {sid: g}, False)
                phi = {}
                for sj in sd.sides:
                    aj = sj // 2
                    gc = O.gamma_faces(sd, sj)
                    loc = (gc[:, 0] - sd.lo_hat[0]) + shp[0] * (gc[:, 1] - sd.lo_hat[1])
                    nb = gc.copy()
                    nb[:, aj] += 1 if sj % 2 else -1
                    Kin = prob.K.reshape(-1)[O.flat_index(gc, prob.n)]
                    Kout = prob.K.reshape(-1)[O.flat_index(nb, prob.n)]
                    beta = alpha * Hw[aj] * (Kin + Kout) / (2 * Kin * Kout)
                    uo = u[loc, sj]
                    pi = p[loc] - uo * prob.h[aj] / (2 * Kin)
                    phi[sj] = -beta * uo + pi
                lst.append(phi)
        phis.append(lst)
    # monolithic system: unknowns = for each i the mixed local solution as a
    # linear function of its X (superposition of mixed solves is avoided: the
    # local problem is linear in lambda, so it is sampled column by column)
    cols = []
    for i, sd in enumerate(subs):
        for k in range(len(phis[i])):
            cols.append((i, k))
    nX = len(cols)
    base = []
    resp = []
    for i, sd in enumerate(subs):
        (p0, u0), _ = _mixed_local(prob, sd.lo, sd.hi, alpha, Hw, {}, True)
        base.append((p0, u0))
        rr = []
        for k in range(len(phis[i])):
            (pk, uk), _ = _mixed_local(prob, sd.lo, sd.hi, alpha, Hw, phis[i][k], False)
            rr.append((pk, uk))
        resp.append(rr)
    # rows: continuity of flux (13d) and of beta u.n + lambda (14d) per edge and test function
    G = []
    rhs = []
    for a in range(2):
        for sd in subs:
            if sd.multi[a] == M[a] - 1:
                continue
            mj = list(sd.multi)
            mj[a] += 1
            j = mj[0] + M[0] * mj[1]
            cells = O.gamma_faces(sd, 2 * a + 1)
            tcoord = 2 * (cells[:, 1 - a] + 0.5 - sd.lo[1 - a]) / sub[1 - a] - 1
            tests = [np.ones(len(cells))] + ([tcoord] if space == 1 else [])
            area = vol / prob.h[a]
            nb = cells.copy()
            nb[:, a] += 1
            Kin = prob.K.reshape(-1)[O.flat_index(cells, prob.n)]
            Kout = prob.K.reshape(-1)[O.flat_index(nb, prob.n)]
            beta = alpha * Hw[a] * (Kin + Kout) / (2 * Kin * Kout)
            for kind in ("M", "V"):
                for tst in tests:
                    row = np.zeros(nX)
                    rv = 0.0
                    for (ii, sid, sgn) in ((sd.index, 2 * a + 1, 1.0), (j, 2 * a, -1.0)):
                        sdi = subs[ii]
                        gc = O.gamma_faces(sdi, sid)
                        loc = (gc[:, 0] - sdi.lo[0]) + sub[0] * (gc[:, 1] - sdi.lo[1])
                        for c, (ci, k) in enumerate(cols):
                            if ci != ii:
                                continue
                            uk = resp[ii][k][1][loc, sid]
                            lam = phis[ii][k][sid]
                            if kind == "M":
                                row[c] += area * np.dot(tst, uk)
                            else:
                                row[c] += sgn * area * np.dot(tst, beta * uk + lam)
                        u0 = base[ii][1][loc, sid]
                        if kind == "M":
                            rv -= area * np.dot(tst, u0)
                        else:
                            rv -= sgn * area * np.dot(tst, beta * u0)
                    G.append(row)
                    rhs.append(rv)
    G = np.array(G)
    rhs = np.array(rhs)
    X = np.linalg.lstsq(G, rhs, rcond=None)[0]
    p = np.zeros(prob.ncells)
    u = np.zeros((prob.ncells, 4))
    c0 = 0
    for i, sd in enumerate(subs):
        pi_, ui = base[i][0].copy(), base[i][1].copy()
        for k in range(len(phis[i])):
            pi_ += X[c0 + k] * resp[i][k][0]
            ui += X[c0 + k] * resp[i][k][1]
        c0 += len(phis[i])
        g = O.flat_index(O.box_cells(sd.lo, sd.hi), prob.n)
        p[g] = pi_
        u[g] = ui
    r = O.mrcm_os(prob, sub, l, space=space, alpha_basis=alpha)
    if bc == "noflow":
        p = O.zero_mean(p)
    assert np.max(np.abs(r.p - p)) < 1e-10 * np.max(np.abs(p))
    assert np.max(np.abs(r.u - u)) < 1e-10 * np.max(np.abs(u))


def test_bruteforce_smoothing_step():
    """One smoothing step (Sec. 3) recomputed with the independent mixed
    solver: per colour in increasing order, Robin data -beta u.n + pi from
    the current state on d hat-Omega_i (outward normal of hat-Omega_i),
    solve on hat-Omega_i with the physical sources, restrict to Omega_i."""
    prob = _rand_problem((12, 12), 29)
    sub, l, alpha_s = (6, 6), 2, 1.0
    Hw = (6 * prob.h[0], 6 * prob.h[1])
    r = O.mrcm_os(prob, sub, l, space=0, alpha_basis=0.5, n_smooth=0)
    p, u = r.p.copy(), r.u.copy()
    subs, M = O.decompose(prob, sub, l)
    Kf = prob.K.reshape(-1)
    for colour in range(4):
        for sd in [s for s in subs if s.colour == colour]:
            shp = tuple(sd.hi_hat[a] - sd.lo_hat[a] for a in range(2))
            robin = {}
            for sid in range(4):
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
            (ph, uh), _ = _mixed_local(prob, sd.lo_hat, sd.hi_hat, alpha_s, Hw, robin, True)
            cells = O.box_cells(sd.lo, sd.hi)
            loc = (cells[:, 0] - sd.lo_hat[0]) + shp[0] * (cells[:, 1] - sd.lo_hat[1])
            g = O.flat_index(cells, prob.n)
            p[g] = ph[loc]
            u[g] = uh[loc]
    p1, u1 = O.smooth_from(prob, sub, l, r.p, r.u, 1, alpha_smooth=alpha_s)
    assert np.max(np.abs(p1 - p)) < 1e-11 * np.max(np.abs(p))
    assert np.max(np.abs(u1 - u)) < 1e-10 * np.max(np.abs(u))


def test_decompose_rejects_bad_overlap():
    prob = _rand_problem((16, 16), 1)
    with pytest.raises(ValueError):
        O.decompose(prob, (8, 8), 4)
    with pytest.raises(ValueError):
        O.decompose(prob, (5, 8), 1)
