"""Independent dense mixed RT0 solver on a box of cells, for pinning the oracle.

Assembles the saddle-point system of Eqs. (11d)-(12d) directly -- one normal
velocity unknown per face (oriented along +axis), one pressure per cell --
with the trapezoid rule for (K^-1 u, v) and exact integration of the
divergence terms, and solves it densely.  It never forms a transmissibility,
so it checks the oracle's cell-centred reduction (Sec. 2.2) rather than
restating it.

Face data per box side (side id 2a + s):
  ('robin', beta[faces], lam[faces])   -beta u.n + p = lam        (Eq. (genRobin))
  ('dirichlet', g)                      p = g                     (Eq. (1c))
  ('neumann', z)                        u.n = z                   (Eq. (1d))
"""
from __future__ import annotations

import numpy as np


def solve_box(h, K, f, sides):
    """K, f: arrays shaped (ny, nx) or (nz, ny, nx) (x fastest).
    sides: list of 2d entries as above, each face list in x-fastest order of
    the tangential axes.  Returns (p [ncells], u_out [ncells, 2d], face_vel)."""
    d = K.ndim
    shape = K.shape[::-1]             # (nx, ny[, nz])
    ncell = int(np.prod(shape))
    vol = float(np.prod(h))
    Kf = K.reshape(-1)
    ff = f.reshape(-1)
    st = [1]
    for a in range(d - 1):
        st.append(st[-1] * shape[a])

    def cid(idx):
        return sum(idx[a] * st[a] for a in range(d))

    # enumerate faces: for axis a, positions 0..shape[a] along a, all tangential cells
    faces = []
    for a in range(d):
        tang = [range(shape[b]) if b != a else range(shape[a] + 1) for b in range(d)]
        grids = np.meshgrid(*[np.array(list(t)) for t in tang[::-1]], indexing="ij")
        pos = np.stack([g.ravel() for g in grids[::-1]], axis=1)
        for q in pos:
            faces.append((a, tuple(int(v) for v in q)))
    nface = len(faces)
    nun = nface + ncell
    A = np.zeros((nun, nun))
    b = np.zeros(nun)
    # per side: counters to map a boundary face to its index in the side list
    side_count = [0] * (2 * d)
    for fi, (a, q) in enumerate(faces):
        area = vol / h[a]
        k = q[a]
        lo_cell = list(q)
        lo_cell[a] = k - 1
        hi_cell = list(q)
        if k == 0:
            side = 2 * a
            s_data = sides[side]
            j = side_count[side]
            side_count[side] += 1
            c = cid(hi_cell)              # the cell is above the face; outward normal is -axis
            if s_data[0] == "neumann":
                A[fi, fi] = 1.0
                b[fi] = -s_data[1]
                continue
            # (K^-1 u, v) on the cell half, -(p, div v) = + a p_c, Robin / Dirichlet terms
            A[fi, fi] += h[a] * area / (2.0 * Kf[c])
            A[fi, nface + c] += area
            if s_data[0] == "robin":
                A[fi, fi] += s_data[1][j] * area
                b[fi] += area * s_data[2][j]
            else:
                b[fi] += area * s_data[1]
        elif k == shape[a]:
            side = 2 * a + 1
            s_data = sides[side]
            j = side_count[side]
            side_count[side] += 1
            c = cid(lo_cell)
            if s_data[0] == "neumann":
                A[fi, fi] = 1.0
                b[fi] = s_data[1]
                continue
            A[fi, fi] += h[a] * area / (2.0 * Kf[c])
            A[fi, nface + c] -= area
            if s_data[0] == "robin":
                A[fi, fi] += s_data[1][j] * area
                b[fi] -= area * s_data[2][j]
            else:
                b[fi] -= area * s_data[1]
        else:
            cL = cid(lo_cell)
            cR = cid(hi_cell)
            A[fi, fi] += h[a] * area / 2.0 * (1.0 / Kf[cL] + 1.0 / Kf[cR])
            A[fi, nface + cL] -= area
            A[fi, nface + cR] += area
    # cell equations: integral of div u over the cell = f |c|
    for fi, (a, q) in enumerate(faces):
        area = vol / h[a]
        k = q[a]
        if k > 0:
            lo_cell = list(q)
            lo_cell[a] = k - 1
            A[nface + cid(lo_cell), fi] += area
        if k < shape[a]:
            A[nface + cid(list(q)), fi] -= area
    b[nface:] = ff * vol
    x = np.linalg.solve(A, b)
    vel = x[:nface]
    p = x[nface:]
    u = np.zeros((ncell, 2 * d))
    for fi, (a, q) in enumerate(faces):
        k = q[a]
        if k > 0:
            lo_cell = list(q)
            lo_cell[a] = k - 1
            u[cid(lo_cell), 2 * a + 1] = vel[fi]
        if k < shape[a]:
            u[cid(list(q)), 2 * a] = -vel[fi]
    return p, u


def side_cells(shape, sid):
    """Local multi-indices of the cells adjacent to side sid, x fastest."""
    d = len(shape)
    a, s = sid // 2, sid % 2
    rng = [np.arange(shape[b]) if b != a else np.array([0 if s == 0 else shape[a] - 1])
           for b in range(d)]
    grids = np.meshgrid(*rng[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)
