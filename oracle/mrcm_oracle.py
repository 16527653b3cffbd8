"""Plain FP64 CPU oracle of the Multiscale Robin Coupled Method with Oversampling
and Smoothing (MRCM-OS, arXiv 2404.13811).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this module; the library never does, and
nothing here is shared with the CUDA path.

What it computes, in the paper's order:

* the lowest-order Raviart-Thomas discretisation with midpoint/trapezoid
  quadrature, i.e. the cell-centred pressure system (Sec. 2.2), on any box of
  cells with Dirichlet / Neumann data on the physical boundary (Eqs. (1c),(1d))
  and Robin data -beta u.n + p = lambda elsewhere (Eq. (genRobin), beta =
  alpha H / K_H with K_H the harmonic mean of the two cells at the face);
* the global fine solution of Eqs. (eqglo1)-(eqglo2);
* Algorithm 1: factor each oversampled operator once (Step 1), solve the N
  informed-space problems (Eq. (oversampling_problem), Step 2), form the
  informed functions phi (Eq. (informed_space)), assemble the interface rows of
  Eqs. (int_ujump)-(int_pjump) (Step 3), solve the particular problems
  (Eqs. (111dbar)-(122dbar), Step 4), solve the interface system and
  superpose u = ubar + sum X Phi (Eqs. (addu), (uhatphat), Step 5), factor the
  smoothing operator when alpha_smooth differs (Step 6), and run the coloured
  smoothing sweeps of Sec. 3 (Eqs. (sm_1)-(sm_2), Step 7).

Readings of the paper that the text leaves open (normals, K_H, H, P1
coordinates, colour order, the gauge of pure-Neumann problems, error norms) are
stated where they are used.

Conventions: a cell is addressed by its multi-index (ix, iy[, iz]); flat
arrays are x-fastest.  A side of a box is (axis a, s) with s = 0 the low side
and s = 1 the high side; side id = 2a + s.  Velocities are stored per cell and
per side as the OUTWARD normal velocity of that cell (array shape (ncells, 2d)),
so fluxes across the skeleton are double-valued by construction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

NEUMANN = 0
DIRICHLET = 1


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def strides(n):
    s = [1]
    for a in range(len(n) - 1):
        s.append(s[-1] * int(n[a]))
    return s


def box_cells(lo, hi):
    """Global multi-indices (ncells, d) of the cells of box [lo, hi), x fastest."""
    d = len(lo)
    ranges = [np.arange(lo[a], hi[a]) for a in range(d)]
    mesh = np.meshgrid(*ranges[::-1], indexing="ij")
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def flat_index(idx, n):
    st = strides(n)
    return sum(idx[:, a] * st[a] for a in range(len(n)))


def side_coordinates(cells, a, lo, hi):
    """Affine coordinates in [-1, 1] of the face centres of a side normal to
    axis a along each tangential axis (ascending), relative to the extent
    [lo, hi) of that side.  Used for the P1 functions {1, t} / {1, s, t}
    (reading: discontinuous per coarse edge/face, Sec. 2.1)."""
    d = cells.shape[1]
    out = []
    for b in range(d):
        if b == a:
            continue
        out.append(2.0 * (cells[:, b] + 0.5 - lo[b]) / (hi[b] - lo[b]) - 1.0)
    return out


def side_basis(space, cells, a, lo, hi):
    """Matrix (nfaces, npsi) of the piecewise polynomial functions on one side.

    space 0: P0 (constant); 1: P1 ({1, t} in 2D, {1, s, t} in 3D);
    'fine': one indicator per fine face (the full trace space F_h of Prop. 2)."""
    nf = cells.shape[0]
    if space == "fine":
        return np.eye(nf)
    cols = [np.ones(nf)]
    if space == 1:
        cols += side_coordinates(cells, a, lo, hi)
    return np.stack(cols, axis=1)


# ----------------------------------------------------------------------------
# local cell-centred system on a box (Sec. 2.2; Eqs. (11d)-(12d), (genRobin))
# ----------------------------------------------------------------------------

@dataclass
class BoxSide:
    axis: int
    s: int
    kind: str            # 'robin', 'dirichlet' or 'neumann'
    local: np.ndarray    # local cell indices adjacent to the side
    cells: np.ndarray    # their global multi-indices
    T: np.ndarray        # transmissibility of the boundary face (0 for Neumann)
    beta: np.ndarray     # Robin parameter (robin sides only)
    value: float = 0.0   # Dirichlet g or Neumann z (physical sides)


@dataclass
class BoxSystem:
    lo: tuple
    hi: tuple
    shape: tuple
    cells: np.ndarray    # (nloc, d)
    A: sp.csr_matrix
    inner: list          # per axis: (L local idx, R local idx, T)
    sides: list          # BoxSide per side id (2a + s)
    Kc: np.ndarray


def harmonic(k1, k2):
    return 2.0 * k1 * k2 / (k1 + k2)


def robin_beta(alpha, H, K_in, K_out):
    """beta = alpha H / K_H with K_H the harmonic average of the permeabilities
    of the two cells sharing the face (Sec. 2.1, after Eq. (genRobin)).
    H is the width of the non-overlapping subdomain normal to the face."""
    return alpha * H / harmonic(K_in, K_out)


def assemble_box(prob, lo, hi, alpha, Hw):
    """Cell-centred operator of the RT0 mixed problem on box [lo, hi).

    RT0 with the trapezoid rule for (K^-1 u, v) and the midpoint rule for the
    rest gives one equation per cell: the sum of outward face fluxes equals
    the integrated source (Eq. (12d)), where
      interior face:  flux = T (p_L - p_R),  T = a 2 K_L K_R / (h (K_L + K_R));
      Robin face:     flux = T (p - lambda), T = a / (h / (2 K) + beta);
      Dirichlet face: flux = T (p - g),      T = 2 a K / h;
      Neumann face:   flux = a z (data).
    The Robin form follows from Eq. (11d) with (beta u.n, v.n) on the face;
    a = face area, h = cell size normal to the face.
    ``Hw`` is the subdomain width per axis entering beta."""
    d = prob.dim
    n = prob.n
    h = prob.h
    shape = tuple(int(hi[a] - lo[a]) for a in range(d))
    nloc = int(np.prod(shape))
    st = strides(shape)
    cells = box_cells(lo, hi)
    Kflat = prob.K.reshape(-1)
    Kc = Kflat[flat_index(cells, n)]
    vol = float(np.prod(h))
    rows, cols, vals = [], [], []
    diag = np.zeros(nloc, dtype=Kc.dtype)
    inner = []
    sides = [None] * (2 * d)
    loc_idx = np.arange(nloc)
    for a in range(d):
        area = vol / h[a]
        ia = cells[:, a] - lo[a]
        L = loc_idx[ia < shape[a] - 1]
        R = L + st[a]
        T = area * 2.0 * Kc[L] * Kc[R] / (h[a] * (Kc[L] + Kc[R]))
        inner.append((L, R, T))
        np.add.at(diag, L, T)
        np.add.at(diag, R, T)
        rows += [L, R]
        cols += [R, L]
        vals += [-T, -T]
        for s in (0, 1):
            sel = loc_idx[ia == (0 if s == 0 else shape[a] - 1)]
            scells = cells[sel]
            outside = lo[a] - 1 if s == 0 else hi[a]
            Kin = Kc[sel]
            if outside < 0 or outside >= n[a]:
                kind = prob.bc_kind[2 * a + s]
                value = float(prob.bc_value[2 * a + s])
                if kind == DIRICHLET:
                    Tb = 2.0 * area * Kin / h[a]
                    np.add.at(diag, sel, Tb)
                    sides[2 * a + s] = BoxSide(a, s, "dirichlet", sel, scells, Tb,
                                               np.zeros(len(sel)), value)
                else:
                    sides[2 * a + s] = BoxSide(a, s, "neumann", sel, scells,
                                               np.zeros(len(sel)), np.zeros(len(sel)), value)
            else:
                nb = scells.copy()
                nb[:, a] = outside
                Kout = Kflat[flat_index(nb, n)]
                beta = robin_beta(alpha, Hw[a], Kin, Kout)
                Tb = area / (h[a] / (2.0 * Kin) + beta)
                np.add.at(diag, sel, Tb)
                sides[2 * a + s] = BoxSide(a, s, "robin", sel, scells, Tb, beta)
    rows.append(loc_idx)
    cols.append(loc_idx)
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nloc, nloc))
    return BoxSystem(tuple(lo), tuple(hi), shape, cells, A, inner, sides, Kc)


def box_rhs(prob, sysm, robin, sources):
    """Right-hand side of the box system.

    robin   -- dict side id -> Robin data lambda on that side's faces (missing = 0)
    sources -- include f, g and z (True) or set them to zero (False, the
               homogeneous problems of Eq. (oversampling_problem))."""
    vol = float(np.prod(prob.h))
    b = np.zeros(len(sysm.Kc), dtype=sysm.Kc.dtype)
    if sources:
        b += prob.f.reshape(-1)[flat_index(sysm.cells, prob.n)] * vol
    for sid, sd in enumerate(sysm.sides):
        if sd.kind == "robin":
            lam = robin.get(sid) if robin else None
            if lam is not None:
                np.add.at(b, sd.local, sd.T * lam)
        elif sources and sd.kind == "dirichlet":
            np.add.at(b, sd.local, sd.T * sd.value)
        elif sources and sd.kind == "neumann":
            area = vol / prob.h[sd.axis]
            np.add.at(b, sd.local, -area * sd.value)
    return b


def box_velocities(prob, sysm, p, robin, sources):
    """Outward normal velocity of every cell of the box through each of its 2d
    faces, from the pressure p of the box solution (same face laws as
    ``assemble_box``)."""
    d = prob.dim
    vol = float(np.prod(prob.h))
    u = np.zeros((len(p), 2 * d), dtype=np.result_type(p, sysm.Kc))
    for a in range(d):
        area = vol / prob.h[a]
        L, R, T = sysm.inner[a]
        flux = T * (p[L] - p[R])
        u[L, 2 * a + 1] = flux / area
        u[R, 2 * a] = -flux / area
    for sid, sd in enumerate(sysm.sides):
        area = vol / prob.h[sd.axis]
        if sd.kind == "robin":
            lam = robin.get(sid) if robin else None
            lam = 0.0 if lam is None else lam
            u[sd.local, sid] = sd.T * (p[sd.local] - lam) / area
        elif sd.kind == "dirichlet":
            g = sd.value if sources else 0.0
            u[sd.local, sid] = sd.T * (p[sd.local] - g) / area
        else:
            u[sd.local, sid] = sd.value if sources else 0.0
    return u


class BandCholesky:
    """Cholesky factor of an SPD box operator kept for reuse across right-hand
    sides (Algorithm 1, Steps 1 and 6; LDL^T and LL^T are the same
    factorisation for SPD matrices).  Banded storage in the natural x-fastest
    order; LAPACK pbtrf/pbtrs through scipy."""

    def __init__(self, A):
        A = sp.csr_matrix(A)
        n = A.shape[0]
        self.n = n
        self.lu = None
        if np.iscomplexobj(A.data):
            # complex-step derivatives (K + i h): the operator is complex
            # symmetric, not Hermitian, so a conjugating Cholesky would be
            # wrong; an unconjugated sparse LU solves the same system
            self.lu = spla.splu(A.tocsc())
            return
        coo = A.tocoo()
        low = coo.row >= coo.col
        bw = int((coo.row - coo.col)[low].max()) if n > 1 else 0
        ab = np.zeros((bw + 1, n))
        r, c, v = coo.row[low], coo.col[low], coo.data[low]
        ab[r - c, c] = v
        self.cb = sla.cholesky_banded(ab, lower=True)
        self.n = n

    def solve(self, b):
        if self.lu is not None:
            return self.lu.solve(np.asarray(b, dtype=complex))
        return sla.cho_solve_banded((self.cb, True), b)


# ----------------------------------------------------------------------------
# global fine solution (Eqs. (eqglo1)-(eqglo2))
# ----------------------------------------------------------------------------

def is_pure_neumann(prob):
    return all(k == NEUMANN for k in prob.bc_kind)


def zero_mean(p):
    """Gauge of pure-Neumann problems: pressure reported with zero mean
    (uniform cells, so the volume-weighted mean is the plain mean)."""
    return p - p.mean()


def fine_solve(prob):
    """Global fine-grid solution on all of Omega.  Returns (p, u) with p shaped
    (ncells,) and u the per-cell outward velocities (ncells, 2d)."""
    lo = tuple([0] * prob.dim)
    hi = tuple(prob.n)
    sysm = assemble_box(prob, lo, hi, 1.0, tuple([1.0] * prob.dim))
    b = box_rhs(prob, sysm, None, True)
    if is_pure_neumann(prob):
        n = sysm.A.shape[0]
        one = sp.csr_matrix(np.ones((1, n)))
        Ab = sp.bmat([[sysm.A, one.T], [one, None]], format="csc")
        x = spla.spsolve(Ab, np.concatenate([b, [0.0]]))
        p = x[:n]
    else:
        p = spla.spsolve(sysm.A.tocsc(), b)
    u = box_velocities(prob, sysm, p, None, True)
    return p, u


# ----------------------------------------------------------------------------
# decomposition
# ----------------------------------------------------------------------------

@dataclass
class Subdomain:
    index: int
    multi: tuple
    lo: tuple          # Omega_i
    hi: tuple
    lo_hat: tuple      # oversampled hat-Omega_i = Omega_i grown by l cells, clipped to Omega
    hi_hat: tuple
    sides: list        # side ids of Gamma_i = d Omega_i \ d Omega (increasing)
    colour: int
    data: dict = field(default_factory=dict)


def decompose(prob, sub, overlap):
    d = prob.dim
    M = []
    for a in range(d):
        if prob.n[a] % sub[a]:
            raise ValueError("subdomain size must divide the grid")
        M.append(prob.n[a] // sub[a])
    if overlap > 0 and any(2 * overlap >= sub[a] for a in range(d)):
        raise ValueError("colouring needs 2 * overlap < subdomain size")
    subs = []
    for idx in range(int(np.prod(M))):
        multi = []
        r = idx
        for a in range(d):
            multi.append(r % M[a])
            r //= M[a]
        lo = tuple(multi[a] * sub[a] for a in range(d))
        hi = tuple(lo[a] + sub[a] for a in range(d))
        lo_hat = tuple(max(0, lo[a] - overlap) for a in range(d))
        hi_hat = tuple(min(prob.n[a], hi[a] + overlap) for a in range(d))
        sides = []
        for a in range(d):
            if multi[a] > 0:
                sides.append(2 * a)
            if multi[a] < M[a] - 1:
                sides.append(2 * a + 1)
        # colour by index parity (Sec. 3, Fig. colored); c = sum_a (i_a mod 2) 2^a
        colour = sum((multi[a] % 2) << a for a in range(d))
        subs.append(Subdomain(idx, tuple(multi), lo, hi, lo_hat, hi_hat, sides, colour))
    return subs, tuple(M)


def restriction_map(sd):
    """Local indices (in hat-Omega_i) of the cells of Omega_i, x fastest."""
    shape = [sd.hi_hat[a] - sd.lo_hat[a] for a in range(len(sd.lo))]
    st = strides(shape)
    cells = box_cells(sd.lo, sd.hi)
    return sum((cells[:, a] - sd.lo_hat[a]) * st[a] for a in range(len(sd.lo)))


def gamma_faces(sd, sid):
    """Cells of Omega_i adjacent to side ``sid`` of Gamma_i, x fastest."""
    a, s = sid // 2, sid % 2
    lo = list(sd.lo)
    hi = list(sd.hi)
    if s == 0:
        hi[a] = lo[a] + 1
    else:
        lo[a] = hi[a] - 1
    return box_cells(lo, hi)


# ----------------------------------------------------------------------------
# MRCM-O and smoothing (Secs. 2-3, Algorithm 1)
# ----------------------------------------------------------------------------

@dataclass
class Result:
    p: np.ndarray              # (ncells,)
    u: np.ndarray              # (ncells, 2d) outward velocities, owning subdomain's solution
    stages: dict = field(default_factory=dict)
    counts: dict = field(default_factory=dict)
    X: np.ndarray = None
    G: np.ndarray = None
    rhs: np.ndarray = None


def _face_pressure(p_in, u_out, h_a, K_in):
    """RT0 face pressure seen from the cell inside: pi = p - u h / (2 K)."""
    return p_in - u_out * h_a / (2.0 * K_in)


def _gamma_traces(prob, sd, p_hat, u_hat, sys_hat):
    """Traces on Gamma_i of a solution on hat-Omega_i: per side, outward flux
    F = a u and face pressure pi (Eq. (informed_space))."""
    vol = float(np.prod(prob.h))
    rmap = restriction_map(sd)
    out = {}
    loc_shape = [sd.hi_hat[a] - sd.lo_hat[a] for a in range(prob.dim)]
    st = strides(loc_shape)
    for sid in sd.sides:
        a = sid // 2
        area = vol / prob.h[a]
        cells = gamma_faces(sd, sid)
        loc = sum((cells[:, b] - sd.lo_hat[b]) * st[b] for b in range(prob.dim))
        uo = u_hat[loc, sid]
        Kin = sys_hat.Kc[loc]
        pi = _face_pressure(p_hat[loc], uo, prob.h[a], Kin)
        out[sid] = (uo * area, pi, uo)
    del rmap
    return out


def gamma_beta(prob, sd, sid, alpha, Hw):
    """beta on the faces of side ``sid`` of Gamma_i (K_H across the face)."""
    a, s = sid // 2, sid % 2
    cells = gamma_faces(sd, sid)
    nb = cells.copy()
    nb[:, a] += (1 if s == 1 else -1)
    Kf = prob.K.reshape(-1)
    return robin_beta(alpha, Hw[a], Kf[flat_index(cells, prob.n)], Kf[flat_index(nb, prob.n)])


def mrcm_os(prob, sub, overlap, space=1, alpha_basis=1.0, alpha_smooth=1.0, n_smooth=0,
            keep_stages=False, particular="omega"):
    """MRCM-O followed by ``n_smooth`` smoothing steps (MRCM-OS).

    space: 0 (P0), 1 (P1) or 'fine' (Prop. 2).
    particular: 'omega' solves the particular problem on Omega_i (Step 4,
    Eqs. (111dbar)-(122dbar), the paper's method); 'hat' is a variant that is
    not in the paper: the particular problem is posed on hat-Omega_i with the
    basis operator (the same sources f, g, z and zero Robin data on
    the sides of hat-Omega_i inside Omega) and restricted to Omega_i like the basis
    functions, so no Omega_i operator is factored.  It shifts the affine local
    space u = ubar + span{Phi_j} and so changes the result; for l = 0 the two
    coincide.
    Returns a Result with the assembled per-cell pressure and per-cell
    outward velocities."""
    if particular not in ("omega", "hat"):
        raise ValueError("particular must be 'omega' or 'hat'")
    d = prob.dim
    h = prob.h
    vol = float(np.prod(h))
    subs, M = decompose(prob, sub, overlap)
    Hw = tuple(sub[a] * h[a] for a in range(d))
    counts = {"local_solves": np.zeros(len(subs), dtype=int),
              "factorisations": np.zeros(len(subs), dtype=int)}

    # Steps 1-2: factor each hat-Omega_i operator and solve the N informed-space
    # problems (Eq. (oversampling_problem): f = 0, homogeneous physical data,
    # Robin data lambda^k on d hat-Omega_i \ d Omega).
    for sd in subs:
        sys_hat = assemble_box(prob, sd.lo_hat, sd.hi_hat, alpha_basis, Hw)
        fac = BandCholesky(sys_hat.A)
        counts["factorisations"][sd.index] += 1
        sd.data["sys_hat"] = sys_hat
        sd.data["fac_hat"] = fac
        rmap = restriction_map(sd)
        Psi, U, F, PI, PHI = [], [], [], [], []
        for sid in sd.sides:
            bs = sys_hat.sides[sid]
            assert bs.kind == "robin"
            basis = side_basis(space, bs.cells, bs.axis, sd.lo_hat, sd.hi_hat)
            for m in range(basis.shape[1]):
                lam = {sid: basis[:, m]}
                b = box_rhs(prob, sys_hat, lam, sources=False)
                pk = fac.solve(b)
                counts["local_solves"][sd.index] += 1
                uk = box_velocities(prob, sys_hat, pk, lam, sources=False)
                tr = _gamma_traces(prob, sd, pk, uk, sys_hat)
                Psi.append(pk[rmap])          # Psi_k restricted to Omega_i (Remark, Sec. 2.2)
                U.append(uk[rmap])            # Phi_k restricted to Omega_i
                F.append({s_: tr[s_][0] for s_ in sd.sides})
                PI.append({s_: tr[s_][1] for s_ in sd.sides})
                # informed function phi = -beta u.n + pi on Gamma_i (Eq. (informed_space))
                PHI.append({s_: -gamma_beta(prob, sd, s_, alpha_basis, Hw) * tr[s_][2]
                            + tr[s_][1] for s_ in sd.sides})
        sd.data.update(Psi=Psi, U=U, F=F, PI=PI, PHI=PHI)

    # Step 4: particular solutions on Omega_i (Eqs. (111dbar)-(122dbar)): sources
    # f, g, z and zero Robin data on Gamma_i with beta from alpha_basis.
    for sd in subs:
        if particular == "hat":
            # the variant: the same sources and zero Robin data on
            # d hat-Omega_i \ d Omega, solved with the kept basis factor; the
            # restriction and the Gamma_i traces are taken as for the basis
            # functions, and the face pressure pi-bar is the trace itself
            # (the Robin data of the restriction on Gamma_i is not zero)
            sys_hat = sd.data["sys_hat"]
            b = box_rhs(prob, sys_hat, None, sources=True)
            ph = sd.data["fac_hat"].solve(b)
            counts["local_solves"][sd.index] += 1
            uh = box_velocities(prob, sys_hat, ph, None, sources=True)
            rmap = restriction_map(sd)
            tr = _gamma_traces(prob, sd, ph, uh, sys_hat)
            sd.data.update(pbar=ph[rmap], ubar=uh[rmap],
                           Fbar={s_: tr[s_][0] for s_ in sd.sides},
                           Ubar={s_: tr[s_][2] for s_ in sd.sides},
                           PIbar={s_: tr[s_][1] for s_ in sd.sides})
            continue
        sys_i = assemble_box(prob, sd.lo, sd.hi, alpha_basis, Hw)
        fac_i = BandCholesky(sys_i.A)
        counts["factorisations"][sd.index] += 1
        b = box_rhs(prob, sys_i, None, sources=True)
        pbar = fac_i.solve(b)
        counts["local_solves"][sd.index] += 1
        ubar = box_velocities(prob, sys_i, pbar, None, sources=True)
        Fbar, Ubar = {}, {}
        for sid in sd.sides:
            a = sid // 2
            area = vol / h[a]
            loc = sys_i.sides[sid].local
            Ubar[sid] = ubar[loc, sid]
            Fbar[sid] = ubar[loc, sid] * area
        sd.data.update(pbar=pbar, ubar=ubar, Fbar=Fbar, Ubar=Ubar)

    # Step 3 + 4: rows of Eqs. (int_ujump)-(int_pjump) tested with every (M, V)
    # in M_H x V_H.  The unique normal on an interface points out of the
    # subdomain with the smaller index (Sec. 2.1), i.e. along +axis, so
    # n^i . n = +1 for the lower and -1 for the upper subdomain.
    col0 = np.zeros(len(subs) + 1, dtype=int)
    for sd in subs:
        col0[sd.index + 1] = col0[sd.index] + len(sd.data["Psi"])
    nX = int(col0[-1])
    rows, rhs = [], []
    n_edges = 0
    for a in range(d):
        for sd in subs:
            if sd.multi[a] == M[a] - 1:
                continue
            mj = list(sd.multi)
            mj[a] += 1
            j = sum(mj[b] * int(np.prod(M[:b])) for b in range(d))
            sj = subs[j]
            n_edges += 1
            sid_i, sid_j = 2 * a + 1, 2 * a
            cells = gamma_faces(sd, sid_i)
            psi = side_basis(space, cells, a, sd.lo, sd.hi)
            area = vol / h[a]
            beta = gamma_beta(prob, sd, sid_i, alpha_basis, Hw)
            for kind in ("M", "V"):
                for m in range(psi.shape[1]):
                    row = np.zeros(nX, dtype=prob.K.dtype)
                    r = 0.0
                    for (sdx, sid, sign) in ((sd, sid_i, 1.0), (sj, sid_j, -1.0)):
                        D = sdx.data
                        for k in range(len(D["Psi"])):
                            if kind == "M":
                                val = np.dot(psi[:, m], D["F"][k][sid])
                            else:
                                uk = D["F"][k][sid] / area
                                val = sign * area * np.dot(psi[:, m], beta * uk + D["PHI"][k][sid])
                            row[col0[sdx.index] + k] += val
                        if kind == "M":
                            r -= np.dot(psi[:, m], D["Fbar"][sid])
                        elif "PIbar" in D:
                            r -= sign * area * np.dot(psi[:, m], D["PIbar"][sid])
                        else:
                            # zero Robin data on Gamma_i: pi-bar = beta u-bar.n
                            r -= sign * area * np.dot(psi[:, m], beta * D["Ubar"][sid])
                    rows.append(row)
                    rhs.append(r)
    G = np.array(rows) if rows else np.zeros((0, 0))
    rhs = np.array(rhs)
    counts["interface_rows"] = G.shape[0]
    counts["interface_cols"] = nX
    counts["edges"] = n_edges
    if G.shape[0] != nX:
        raise ValueError("interface system is not square (Prop. 1)")

    # Step 5: interface solve (dense, FP64).  Pure-Neumann problems have the
    # one-dimensional null space "same constant in every subdomain"; the
    # minimum-norm least-squares solution is taken and the pressure is then
    # reported with zero mean.
    if nX == 0:
        X = np.zeros(0)
    elif is_pure_neumann(prob):
        X = np.linalg.lstsq(G, rhs, rcond=None)[0]
    else:
        X = solve_square(G, rhs)

    # Superposition u = ubar + sum_j X_j Phi_j, p = pbar + sum_j X_j Psi_j
    # (Eqs. (addu), (addp), (uhatphat)).
    ncell = prob.ncells
    p = np.zeros(ncell, dtype=prob.K.dtype)
    u = np.zeros((ncell, 2 * d), dtype=prob.K.dtype)
    for sd in subs:
        D = sd.data
        xi = X[col0[sd.index]:col0[sd.index + 1]]
        pi_ = D["pbar"].copy()
        ui = D["ubar"].copy()
        for k in range(len(xi)):
            pi_ += xi[k] * D["Psi"][k]
            ui += xi[k] * D["U"][k]
        g = flat_index(box_cells(sd.lo, sd.hi), prob.n)
        p[g] = pi_
        u[g] = ui
    if is_pure_neumann(prob):
        p = zero_mean(p)
    res = Result(p=p, u=u, counts=counts, X=X, G=G, rhs=rhs)
    res.subs = subs
    res.col0 = col0
    if keep_stages:
        res.stages["mrcm_o"] = (p.copy(), u.copy())

    # Steps 6-7: smoothing.
    if n_smooth > 0:
        smoother = Smoother(prob, subs, sub, alpha_basis, alpha_smooth, counts)
        for step in range(n_smooth):
            smoother.step(p, u)
            if is_pure_neumann(prob):
                p[:] = zero_mean(p)
            if keep_stages:
                res.stages[f"smooth{step + 1}"] = (p.copy(), u.copy())
    return res


def solve_square(G, rhs, refine=3):
    """Solution of the square interface system (Prop. 1).  Its flux rows and
    pressure rows differ in scale by many orders of magnitude (raw condition
    numbers near 1e10), so the rows and columns are scaled by their largest
    entries before the LU factorisation and the FP64 residual of the original
    system drives a few steps of refinement."""
    r = 1.0 / np.abs(G).max(axis=1)
    Ge = G * r[:, None]
    c = 1.0 / np.abs(Ge).max(axis=0)
    lu = sla.lu_factor(Ge * c[None, :])
    X = c * sla.lu_solve(lu, r * rhs)
    for _ in range(refine):
        X = X + c * sla.lu_solve(lu, r * (rhs - G @ X))
    return X


class Smoother:
    """Smoothing steps of Sec. 3 (Eqs. (sm_1)-(sm_2); Algorithm 1 Steps 6-7).

    Colours by subdomain-index parity, visited in increasing order
    c = sum_a (i_a mod 2) 2^a (the paper fixes no order; the order matters for
    this multiplicative sweep).  For every subdomain of the colour: Robin data
    lambda = -beta u.n + pi on d hat-Omega_i \\ d Omega from the current global
    solution, with n the outward normal of hat-Omega_i and beta built with
    alpha_smooth; a solve on hat-Omega_i with the physical sources; and an
    overwrite of (u, p) on Omega_i by the restriction."""

    def __init__(self, prob, subs, sub, alpha_basis, alpha_smooth, counts=None):
        self.prob = prob
        self.subs = subs
        d = prob.dim
        self.Hw = tuple(sub[a] * prob.h[a] for a in range(d))
        self.counts = counts
        for sd in subs:
            if alpha_smooth == alpha_basis and "fac_hat" in sd.data:
                sd.data["sys_s"] = sd.data["sys_hat"]
                sd.data["fac_s"] = sd.data["fac_hat"]
            else:
                # Step 6: a second factorisation only when alpha differs.
                sys_s = assemble_box(prob, sd.lo_hat, sd.hi_hat, alpha_smooth, self.Hw)
                sd.data["sys_s"] = sys_s
                sd.data["fac_s"] = BandCholesky(sys_s.A)
                if counts is not None:
                    counts["factorisations"][sd.index] += 1
        self.ncolours = 2 ** d

    def robin_data(self, sd, p, u):
        prob = self.prob
        sys_s = sd.data["sys_s"]
        Kf = prob.K.reshape(-1)
        lam = {}
        for sid, bs in enumerate(sys_s.sides):
            if bs.kind != "robin":
                continue
            g = flat_index(bs.cells, prob.n)
            uo = u[g, sid]                     # outward from hat-Omega_i
            pi = _face_pressure(p[g], uo, prob.h[bs.axis], Kf[g])
            lam[sid] = -bs.beta * uo + pi
        return lam

    def solve_one(self, sd, p, u):
        prob = self.prob
        sys_s = sd.data["sys_s"]
        lam = self.robin_data(sd, p, u)
        b = box_rhs(prob, sys_s, lam, sources=True)
        ph = sd.data["fac_s"].solve(b)
        if self.counts is not None:
            self.counts["local_solves"][sd.index] += 1
        uh = box_velocities(prob, sys_s, ph, lam, sources=True)
        rmap = restriction_map(sd)
        return ph[rmap], uh[rmap]

    def step(self, p, u):
        prob = self.prob
        for c in range(self.ncolours):
            todo = [sd for sd in self.subs if sd.colour == c]
            # subdomains of one colour share no boundary points: their solves
            # read only cells of other colours, so they are independent.
            results = [self.solve_one(sd, p, u) for sd in todo]
            for sd, (pi_, ui) in zip(todo, results):
                g = flat_index(box_cells(sd.lo, sd.hi), prob.n)
                p[g] = pi_
                u[g] = ui


def smooth_from(prob, sub, overlap, p, u, n_steps, alpha_smooth=1.0):
    """Apply ``n_steps`` smoothing steps to an arbitrary global state (p, u)."""
    subs, _ = decompose(prob, sub, overlap)
    sm = Smoother(prob, subs, sub, None, alpha_smooth)
    p = p.copy()
    u = u.copy()
    for _ in range(n_steps):
        sm.step(p, u)
        if is_pure_neumann(prob):
            p[:] = zero_mean(p)
    return p, u


# ----------------------------------------------------------------------------
# norms and residuals
# ----------------------------------------------------------------------------

def rel_errors(prob, p, u, p_ref, u_ref):
    """Relative L2 errors (reading of Sec. 4): pressure sum_c |c| (p - p_ref)^2,
    flux sum_c |c| 1/2 sum_faces (u - u_ref)^2 (the trapezoid RT0 mass norm
    with each cell's own face values), each normalised by the reference norm."""
    ep = math.sqrt(np.sum((p - p_ref) ** 2) / max(np.sum(p_ref ** 2), 1e-300))
    eu = math.sqrt(np.sum((u - u_ref) ** 2) / max(np.sum(u_ref ** 2), 1e-300))
    return ep, eu


def mass_residual(prob, u):
    """Per-cell residual sum_faces a u_out - f |c| (Eq. (12d))."""
    vol = float(np.prod(prob.h))
    r = -prob.f.reshape(-1) * vol
    for a in range(prob.dim):
        area = vol / prob.h[a]
        r = r + area * (u[:, 2 * a] + u[:, 2 * a + 1])
    return r
