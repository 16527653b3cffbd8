"""Discrete adjoint of the MRCM-OS oracle with respect to log K.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this module; the library never does, and
nothing here is shared with the CUDA path.

The forward map is the oracle's ``mrcm_os`` (Algorithm 1 followed by the
smoothing steps of Sec. 3) with theta = log K per cell as the parameters.
For seeds gp = dL/dp and gu = dL/du of any scalar loss L of the returned
(p, u), ``mrcm_os_adjoint`` returns dL/dtheta by running the forward steps
backwards:

* smoothing steps and colours in reverse order (each colour's solve re-run
  from the state recorded before that colour, Eqs. (sm_1)-(sm_2));
* the superposition of Eqs. (addu), (addp), (uhatphat);
* the interface system of Eqs. (int_ujump)-(int_pjump), through its
  transpose;
* the N_i basis problems on every hat-Omega_i (Eq. (oversampling_problem))
  and the particular problem on every Omega_i (Eqs. (111dbar)-(122dbar)),
  each through one adjoint solve with the same (symmetric) operator;
* the face laws of the cell-centred RT0 system (Sec. 2.2), whose
  transmissibilities, Robin parameters beta = alpha H / K_H and face
  pressures are the only places where K enters.

For one box solve A(K) p = b(K, lambda), u = V(K, p, lambda) with seeds
(gp, gu) the adjoint is mu = A^{-1} (gp + dV/dp^T gu) and, per face
coefficient c, dL/dc = -mu^T (dA/dc) p + mu^T (db/dc) + gu . dV/dc.

Pure-Neumann problems are not differentiated here (their interface solve is
a minimum-norm least-squares solution): use Dirichlet data on some side.

particular="hat" differentiates the oracle's variant in which the
particular problem is posed on hat-Omega_i with the basis operator: it then
runs backwards like a basis problem (sources instead of Robin data, its face
pressure pi-bar = p - u.n h / (2K) in the pressure rows).
"""
from __future__ import annotations

import numpy as np

from oracle import mrcm_oracle as O


# ----------------------------------------------------------------------------
# derivatives of the face laws (Sec. 2.2, Eq. (genRobin))
# ----------------------------------------------------------------------------

def _dT_inner(area, h, KL, KR):
    """d/dK_L and d/dK_R of T = a 2 K_L K_R / (h (K_L + K_R))."""
    s2 = (KL + KR) ** 2
    return area * 2.0 * KR ** 2 / (h * s2), area * 2.0 * KL ** 2 / (h * s2)


def _dbeta(alpha, H, Kin, Kout):
    """d/dK_in and d/dK_out of beta = alpha H (K_in + K_out) / (2 K_in K_out)."""
    return -alpha * H / (2.0 * Kin ** 2), -alpha * H / (2.0 * Kout ** 2)


def _dT_robin(area, h, alpha, H, Kin, Kout):
    """d/dK_in and d/dK_out of T = a / (h / (2 K_in) + beta)."""
    beta = O.robin_beta(alpha, H, Kin, Kout)
    D = h / (2.0 * Kin) + beta
    dbi, dbo = _dbeta(alpha, H, Kin, Kout)
    dDi = -h / (2.0 * Kin ** 2) + dbi
    return -area * dDi / D ** 2, -area * dbo / D ** 2


def _outside_cells(bs, n):
    """Global flat indices of the cells across a box side."""
    nb = bs.cells.copy()
    nb[:, bs.axis] += 1 if bs.s == 1 else -1
    return O.flat_index(nb, n)


# ----------------------------------------------------------------------------
# one box solve backwards
# ----------------------------------------------------------------------------

def box_adjoint(prob, sysm, fac, p, lam, sources, gp, gu, alpha, Hw, gK):
    """Adjoint of  A p = b(lambda),  u = velocities(p, lambda)  on one box.

    p        -- the forward solution on the box
    lam      -- Robin data per side id (None: zero)
    gp, gu   -- seeds dL/dp (nloc,) and dL/du (nloc, 2d) on the box
    gK       -- global dL/dK, accumulated in place
    Returns dL/dlambda per Robin side id."""
    d = prob.dim
    vol = float(np.prod(prob.h))
    gidx = O.flat_index(sysm.cells, prob.n)
    Kf = prob.K.reshape(-1)
    # right-hand side of the adjoint system: gp + (du/dp)^T gu
    rt = gp.astype(float).copy()
    for a in range(d):
        area = vol / prob.h[a]
        L, R, T = sysm.inner[a]
        dlt = gu[L, 2 * a + 1] - gu[R, 2 * a]
        np.add.at(rt, L, T * dlt / area)
        np.add.at(rt, R, -T * dlt / area)
    for sid, bs in enumerate(sysm.sides):
        if bs.kind in ("robin", "dirichlet"):
            area = vol / prob.h[bs.axis]
            np.add.at(rt, bs.local, bs.T * gu[bs.local, sid] / area)
    mu = fac.solve(rt)
    # face coefficients
    for a in range(d):
        area = vol / prob.h[a]
        L, R, T = sysm.inner[a]
        dp = p[L] - p[R]
        gT = -(mu[L] - mu[R]) * dp + (gu[L, 2 * a + 1] - gu[R, 2 * a]) * dp / area
        dL_, dR_ = _dT_inner(area, prob.h[a], Kf[gidx[L]], Kf[gidx[R]])
        np.add.at(gK, gidx[L], gT * dL_)
        np.add.at(gK, gidx[R], gT * dR_)
    glam = {}
    for sid, bs in enumerate(sysm.sides):
        a = bs.axis
        area = vol / prob.h[a]
        loc = bs.local
        gin = gidx[loc]
        if bs.kind == "robin":
            lv = lam.get(sid) if lam else None
            lv = np.zeros(len(loc)) if lv is None else lv
            gT = (p[loc] - lv) * (gu[loc, sid] / area - mu[loc])
            gout = _outside_cells(bs, prob.n)
            di, do = _dT_robin(area, prob.h[a], alpha, Hw[a], Kf[gin], Kf[gout])
            np.add.at(gK, gin, gT * di)
            np.add.at(gK, gout, gT * do)
            glam[sid] = bs.T * (mu[loc] - gu[loc, sid] / area)
        elif bs.kind == "dirichlet":
            g = bs.value if sources else 0.0
            gT = (p[loc] - g) * (gu[loc, sid] / area - mu[loc])
            np.add.at(gK, gin, gT * 2.0 * area / prob.h[a])
    return glam


# ----------------------------------------------------------------------------
# the whole method backwards
# ----------------------------------------------------------------------------

def _add_beta(prob, sd, sid, alpha, Hw, gbeta, gK):
    """Accumulates dL/dbeta on the faces of side ``sid`` of Gamma_i into gK."""
    a, s = sid // 2, sid % 2
    cells = O.gamma_faces(sd, sid)
    nb = cells.copy()
    nb[:, a] += 1 if s == 1 else -1
    gi, go = O.flat_index(cells, prob.n), O.flat_index(nb, prob.n)
    Kf = prob.K.reshape(-1)
    di, do = _dbeta(alpha, Hw[a], Kf[gi], Kf[go])
    np.add.at(gK, gi, gbeta * di)
    np.add.at(gK, go, gbeta * do)


def mrcm_os_adjoint(prob, sub, overlap, space, alpha_basis, alpha_smooth, n_smooth, gp, gu,
                    particular="omega"):
    """Returns (Result of the forward run, dL/dlog K (ncells,)) for the seeds
    gp (ncells,) and gu (ncells, 2d) of a scalar loss of the returned (p, u)."""
    if O.is_pure_neumann(prob):
        raise NotImplementedError("the adjoint needs Dirichlet data on some side")
    d = prob.dim
    h = prob.h
    vol = float(np.prod(h))
    Hw = tuple(sub[a] * h[a] for a in range(d))
    Kf = prob.K.reshape(-1)
    hat = particular == "hat"
    res = O.mrcm_os(prob, sub, overlap, space, alpha_basis, alpha_smooth, 0, particular=particular)
    subs, col0, X, G = res.subs, res.col0, res.X, res.G
    _, M = O.decompose(prob, sub, overlap)

    # forward smoothing again, recording the state before every colour
    p, u = res.p.copy(), res.u.copy()
    sm = O.Smoother(prob, subs, sub, alpha_basis, alpha_smooth) if n_smooth > 0 else None
    tape = []
    for step in range(n_smooth):
        for c in range(sm.ncolours):
            tape.append((c, p.copy(), u.copy()))
            todo = [sd for sd in subs if sd.colour == c]
            out = [sm.solve_one(sd, p, u) for sd in todo]
            for sd, (pi_, ui) in zip(todo, out):
                g = O.flat_index(O.box_cells(sd.lo, sd.hi), prob.n)
                p[g] = pi_
                u[g] = ui
    res.p, res.u = p, u

    gK = np.zeros(prob.ncells)
    gp = np.asarray(gp, dtype=float).copy()
    gu = np.asarray(gu, dtype=float).copy()

    # ---- smoothing, backwards (Eqs. (sm_1)-(sm_2)) ----
    for c, p_s, u_s in reversed(tape):
        todo = [sd for sd in subs if sd.colour == c]
        seeds = []
        for sd in todo:
            g = O.flat_index(O.box_cells(sd.lo, sd.hi), prob.n)
            seeds.append((gp[g].copy(), gu[g].copy()))
            gp[g] = 0.0
            gu[g] = 0.0
        for sd, (sgp, sgu) in zip(todo, seeds):
            sys_s = sd.data["sys_s"]
            lam = sm.robin_data(sd, p_s, u_s)
            ph = sd.data["fac_s"].solve(O.box_rhs(prob, sys_s, lam, True))
            nloc = len(sys_s.Kc)
            rmap = O.restriction_map(sd)
            lgp = np.zeros(nloc)
            lgu = np.zeros((nloc, 2 * d))
            lgp[rmap] = sgp
            lgu[rmap] = sgu
            glam = box_adjoint(prob, sys_s, sd.data["fac_s"], ph, lam, True, lgp, lgu,
                               alpha_smooth, Hw, gK)
            # lambda = -beta u.n + p - u.n h / (2K) of the cell inside
            for sid, gl in glam.items():
                bs = sys_s.sides[sid]
                g = O.flat_index(bs.cells, prob.n)
                hh = h[bs.axis]
                un = u_s[g, sid]
                np.add.at(gu, (g, np.full(len(g), sid)), gl * (-bs.beta - hh / (2.0 * Kf[g])))
                np.add.at(gp, g, gl)
                np.add.at(gK, g, gl * un * hh / (2.0 * Kf[g] ** 2))
                di, do = _dbeta(alpha_smooth, Hw[bs.axis], Kf[g], Kf[_outside_cells(bs, prob.n)])
                np.add.at(gK, g, -gl * un * di)
                np.add.at(gK, _outside_cells(bs, prob.n), -gl * un * do)

    # ---- superposition, backwards (Eqs. (addu), (addp)) ----
    nX = int(col0[-1])
    gX = np.zeros(nX)
    seeds_b, seeds_p = {}, {}
    for sd in subs:
        D = sd.data
        g = O.flat_index(O.box_cells(sd.lo, sd.hi), prob.n)
        sgp, sgu = gp[g], gu[g]
        for k in range(len(D["Psi"])):
            gX[col0[sd.index] + k] = np.dot(sgp, D["Psi"][k]) + np.sum(sgu * D["U"][k])
        seeds_p[sd.index] = (sgp.copy(), sgu.copy())
        seeds_b[sd.index] = (sgp.copy(), sgu.copy())

    # ---- interface system, backwards: X = G^{-1} rhs ----
    grhs = O.solve_square(G.T.copy(), gX) if nX else np.zeros(0)
    gG = -np.outer(grhs, X)
    # per subdomain: dL/dF_k, dL/dPHI_k per side; dL/dFbar, dL/dUbar per side
    for sd in subs:
        nk = len(sd.data["Psi"])
        sd.data["gF"] = [{s_: np.zeros(len(sd.data["F"][k][s_])) for s_ in sd.sides} for k in range(nk)]
        sd.data["gPHI"] = [{s_: np.zeros(len(sd.data["F"][k][s_])) for s_ in sd.sides} for k in range(nk)]
        sd.data["gFbar"] = {s_: np.zeros(len(sd.data["Fbar"][s_])) for s_ in sd.sides}
        sd.data["gUbar"] = {s_: np.zeros(len(sd.data["Fbar"][s_])) for s_ in sd.sides}
        sd.data["gPIbar"] = {s_: np.zeros(len(sd.data["Fbar"][s_])) for s_ in sd.sides}
    row = 0
    for a in range(d):
        for sd in subs:
            if sd.multi[a] == M[a] - 1:
                continue
            mj = list(sd.multi)
            mj[a] += 1
            j = sum(mj[b] * int(np.prod(M[:b])) for b in range(d))
            sj = subs[j]
            sid_i, sid_j = 2 * a + 1, 2 * a
            cells = O.gamma_faces(sd, sid_i)
            psi = O.side_basis(space, cells, a, sd.lo, sd.hi)
            area = vol / h[a]
            beta = O.gamma_beta(prob, sd, sid_i, alpha_basis, Hw)
            gbeta = np.zeros(len(beta))
            for kind in ("M", "V"):
                for m in range(psi.shape[1]):
                    for (sdx, sid, sign) in ((sd, sid_i, 1.0), (sj, sid_j, -1.0)):
                        D = sdx.data
                        for k in range(len(D["Psi"])):
                            gg = gG[row, col0[sdx.index] + k]
                            if kind == "M":
                                D["gF"][k][sid] += gg * psi[:, m]
                            else:
                                uk = D["F"][k][sid] / area
                                D["gF"][k][sid] += gg * sign * psi[:, m] * beta
                                D["gPHI"][k][sid] += gg * sign * area * psi[:, m]
                                gbeta += gg * sign * area * psi[:, m] * uk
                        if kind == "M":
                            D["gFbar"][sid] += -grhs[row] * psi[:, m]
                        elif hat:
                            D["gPIbar"][sid] += -grhs[row] * sign * area * psi[:, m]
                        else:
                            D["gUbar"][sid] += -grhs[row] * sign * area * psi[:, m] * beta
                            gbeta += -grhs[row] * sign * area * psi[:, m] * D["Ubar"][sid]
                    row += 1
            _add_beta(prob, sd, sid_i, alpha_basis, Hw, gbeta, gK)
    assert row == G.shape[0]

    # ---- basis problems on hat-Omega_i, backwards (Eq. (informed_space)) ----
    for sd in subs:
        D = sd.data
        sys_hat, fac = D["sys_hat"], D["fac_hat"]
        nloc = len(sys_hat.Kc)
        rmap = O.restriction_map(sd)
        loc_shape = [sd.hi_hat[b] - sd.lo_hat[b] for b in range(d)]
        st = O.strides(loc_shape)
        sgp, sgu = seeds_b[sd.index]
        xs = X[col0[sd.index]:col0[sd.index + 1]]
        k = 0
        for sid in sd.sides:
            bs = sys_hat.sides[sid]
            basis = O.side_basis(space, bs.cells, bs.axis, sd.lo_hat, sd.hi_hat)
            for m in range(basis.shape[1]):
                lam = {sid: basis[:, m]}
                pk = fac.solve(O.box_rhs(prob, sys_hat, lam, sources=False))
                uk = O.box_velocities(prob, sys_hat, pk, lam, sources=False)
                lgp = np.zeros(nloc)
                lgu = np.zeros((nloc, 2 * d))
                lgp[rmap] = xs[k] * sgp
                lgu[rmap] = xs[k] * sgu
                # traces F = a u.n, PHI = -beta u.n + pi, pi = p - u.n h / (2K)
                for s_ in sd.sides:
                    a_ = s_ // 2
                    area = vol / h[a_]
                    cl = O.gamma_faces(sd, s_)
                    loc = sum((cl[:, b] - sd.lo_hat[b]) * st[b] for b in range(d))
                    gi = O.flat_index(cl, prob.n)
                    uo = uk[loc, s_]
                    bet = O.gamma_beta(prob, sd, s_, alpha_basis, Hw)
                    gF, gPHI = D["gF"][k][s_], D["gPHI"][k][s_]
                    np.add.at(lgu, (loc, np.full(len(loc), s_)),
                              area * gF + gPHI * (-bet - h[a_] / (2.0 * Kf[gi])))
                    np.add.at(lgp, loc, gPHI)
                    np.add.at(gK, gi, gPHI * uo * h[a_] / (2.0 * Kf[gi] ** 2))
                    _add_beta(prob, sd, s_, alpha_basis, Hw, -gPHI * uo, gK)
                box_adjoint(prob, sys_hat, fac, pk, lam, False, lgp, lgu, alpha_basis, Hw, gK)
                k += 1

    # ---- particular problems on hat-Omega_i (the variant), backwards ----
    for sd in (subs if hat else ()):
        D = sd.data
        sys_hat, fac = D["sys_hat"], D["fac_hat"]
        nloc = len(sys_hat.Kc)
        rmap = O.restriction_map(sd)
        loc_shape = [sd.hi_hat[b] - sd.lo_hat[b] for b in range(d)]
        st = O.strides(loc_shape)
        sgp, sgu = seeds_p[sd.index]
        ph = fac.solve(O.box_rhs(prob, sys_hat, None, sources=True))
        uh = O.box_velocities(prob, sys_hat, ph, None, sources=True)
        lgp = np.zeros(nloc)
        lgu = np.zeros((nloc, 2 * d))
        lgp[rmap] = sgp
        lgu[rmap] = sgu
        # traces F-bar = a u.n, pi-bar = p - u.n h / (2K)
        for s_ in sd.sides:
            a_ = s_ // 2
            area = vol / h[a_]
            cl = O.gamma_faces(sd, s_)
            loc = sum((cl[:, b] - sd.lo_hat[b]) * st[b] for b in range(d))
            gi = O.flat_index(cl, prob.n)
            uo = uh[loc, s_]
            gPI = D["gPIbar"][s_]
            np.add.at(lgu, (loc, np.full(len(loc), s_)), area * D["gFbar"][s_] - gPI * h[a_] / (2.0 * Kf[gi]))
            np.add.at(lgp, loc, gPI)
            np.add.at(gK, gi, gPI * uo * h[a_] / (2.0 * Kf[gi] ** 2))
        box_adjoint(prob, sys_hat, fac, ph, None, True, lgp, lgu, alpha_basis, Hw, gK)

    # ---- particular problems on Omega_i, backwards (Eqs. (111dbar)-(122dbar)) ----
    for sd in (() if hat else subs):
        D = sd.data
        sys_i = O.assemble_box(prob, sd.lo, sd.hi, alpha_basis, Hw)
        fac_i = O.BandCholesky(sys_i.A)
        pbar = D["pbar"]
        sgp, sgu = seeds_p[sd.index]
        lgp = sgp.copy()
        lgu = sgu.copy()
        for s_ in sd.sides:
            area = vol / h[s_ // 2]
            loc = sys_i.sides[s_].local
            np.add.at(lgu, (loc, np.full(len(loc), s_)), area * D["gFbar"][s_] + D["gUbar"][s_])
        box_adjoint(prob, sys_i, fac_i, pbar, None, True, lgp, lgu, alpha_basis, Hw, gK)

    return res, gK * Kf
