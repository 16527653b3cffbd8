"""Differentiation form on the GPU: mrcm_adjoint (dL/dlog K through basis,
interface and smoothing) against the oracle's discrete adjoint, against
central finite differences of the GPU forward, and through the
torch.autograd.Function front end.

Tolerances.  Oracle gradient: max |g - g_oracle| <= 1e-8 max |g_oracle| for
both forms (the forward paths agree with the oracle to ~1e-11 and the reverse
pass is the same sequence of solves).  Finite differences (h = 1e-6, FP64
forward refined to rounding level): error within 1e-6 of the gradient's
scale, per coordinate |FD_j - g_j| <= 1e-6 max_i |g_i| and per direction
|FD_v - g.v| <= 1e-6 |g| |v|.
"""
import numpy as np
import pytest

from oracle import mrcm_adjoint as AD
from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem(n, seed, sigma2=3.0):
    prob = I.lognormal_problem(n, sigma2=sigma2, corr_len=0.15, seed=seed)
    rng = np.random.default_rng(seed + 1)
    prob.f = rng.standard_normal(prob.f.shape)
    return prob


def _seeds(ncells, dim, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(ncells), rng.standard_normal((ncells, 2 * dim))


CASES = [
    # n, sub, overlap, space, alpha_basis, alpha_smooth, n_smooth
    ((64, 48), (16, 16), 2, 1, 1.0, 1.0, 2),
    ((48, 48), (16, 16), 0, 0, 0.5, 2.0, 1),
    ((64, 64), (16, 16), 4, 1, 1.0, 1.0, 3),
    ((64, 32), (16, 16), 3, 1, 2.0, 0.5, 0),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_gradient_matches_oracle_gradient(case, precision):
    from paper_2404_13811_gb300.solver import MRCM
    n, sub, ov, space, ab, as_, ns = CASES[case]
    prob = _problem(n, seed=60 + case)
    wp, wu = _seeds(prob.ncells, 2, 7 + case)
    _, g_ref = AD.mrcm_os_adjoint(prob, sub, ov, space, ab, as_, ns, wp, wu)
    s = MRCM(prob, I.Partition(sub, ov), space=space, alpha_basis=ab, alpha_smooth=as_, precision=precision)
    s.run(ns)
    g = s.adjoint(wp, wu)
    err = np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))
    assert err <= 1e-8, err
    s.close()


def test_ensemble_gradient_matches_oracle_per_member():
    from paper_2404_13811_gb300.solver import MRCM
    specs = [((64, 48), (16, 16), 2), ((48, 80), (16, 16), 3)]
    probs = [_problem(n, seed=80 + m) for m, (n, _, _) in enumerate(specs)]
    parts = [I.Partition(sub, ov) for (_, sub, ov) in specs]
    seeds = [_seeds(p.ncells, 2, 90 + m) for m, p in enumerate(probs)]
    s = MRCM(probs, parts, space=1, precision="fp64")
    s.run(2)
    g = s.adjoint(np.concatenate([a for a, _ in seeds]), np.concatenate([b for _, b in seeds]))
    off = 0
    for prob, part, (wp, wu) in zip(probs, parts, seeds):
        _, g_ref = AD.mrcm_os_adjoint(prob, part.sub, part.overlap, 1, 1.0, 1.0, 2, wp, wu)
        gm = g[off:off + prob.ncells]
        assert np.max(np.abs(gm - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))
        off += prob.ncells
    s.close()


def test_backward_entry_point_matches_adjoint():
    """mrcm_backward (seeds in velocity, pressure order, host arrays) is the
    same reverse pass as mrcm_adjoint.  The face-coefficient adjoints of
    overlapping boxes are summed with FP64 atomics, so two calls agree to
    rounding (1e-10 of the gradient's scale), not bit for bit."""
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300.solver import MRCM
    prob = _problem((64, 48), seed=71)
    wp, wu = _seeds(prob.ncells, 2, 72)
    s = MRCM(prob, I.Partition((16, 16), 2), space=1, precision="mixed")
    s.run(2)
    g1 = s.adjoint(wp, wu)
    g2 = np.empty(prob.ncells)
    L.mrcm_backward(s.h, np.ascontiguousarray(wu), np.ascontiguousarray(wp), g2)
    assert np.max(np.abs(g1 - g2)) <= 1e-10 * np.max(np.abs(g1))
    g3 = np.empty(prob.ncells)
    L.mrcm_backward(s.h, None, np.ascontiguousarray(wp), g3)
    g4 = s.adjoint(wp, None)
    assert np.max(np.abs(g3 - g4)) <= 1e-10 * np.max(np.abs(g4))
    s.close()


def test_adjoint_leaves_the_solution_unchanged_and_refuses_pure_neumann():
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300.solver import MRCM
    prob = _problem((64, 64), seed=5)
    s = MRCM(prob, I.Partition((16, 16), 2), precision="mixed")
    s.run(2)
    p0, u0 = s.fluxes()
    s.adjoint(np.ones(prob.ncells), None)
    p1, u1 = s.fluxes()
    assert np.array_equal(p0, p1) and np.array_equal(u0, u1)
    s.close()
    case = I.config_small()
    s = MRCM(case.problem, case.partition, space=0)
    s.run(1)
    with pytest.raises(L.MrcmError) as ei:
        s.adjoint(np.ones(case.problem.ncells), None)
    assert ei.value.code == -7
    s.close()


# ---------------------------------------------------------------------------
# the 256 x 256 sink-flux workload: autograd front end and finite differences
# ---------------------------------------------------------------------------

def _sink_rows(case):
    n = case.problem.n
    return np.array([ix + n[0] * iy for (ix, iy) in case.extra["sinks"]])


def _target(case):
    t = case.extra["target_problem"]
    pm = case.params
    ref = O.mrcm_os(t, case.partition.sub, case.partition.overlap, pm.space, pm.alpha_basis,
                    pm.alpha_smooth, pm.n_smooth)
    return ref.u


def test_sink_flux_loss_gradient_autograd_vs_finite_differences_and_oracle():
    import torch
    from paper_2404_13811_gb300.solver import MRCM, mrcm_solve
    case = I.config_adjoint()
    prob, pm = case.problem, case.params
    rows = torch.as_tensor(_sink_rows(case), device="cuda")
    ut_all = _target(case)
    ut = torch.as_tensor(ut_all[_sink_rows(case)], device="cuda")
    s = MRCM(prob, case.partition, space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth,
             precision="fp64", ir_tol=1e-15, max_ir=8)
    theta0 = torch.as_tensor(np.log(prob.K).reshape(-1), device="cuda")

    def loss_of(theta):
        p, u = mrcm_solve(s, theta, pm.n_smooth)
        return ((u[rows] - ut) ** 2).sum()

    theta = theta0.clone().requires_grad_(True)
    L0 = loss_of(theta)
    L0.backward()
    g = theta.grad.detach().cpu().numpy()
    gmax = np.max(np.abs(g))
    assert gmax > 0

    # oracle gradient of the same loss: seeds 2 (u - ut) on the sink faces
    ref = O.mrcm_os(prob, case.partition.sub, case.partition.overlap, pm.space, pm.alpha_basis,
                    pm.alpha_smooth, pm.n_smooth)
    gu = np.zeros_like(ref.u)
    sr = _sink_rows(case)
    gu[sr] = 2.0 * (ref.u[sr] - ut_all[sr])
    _, g_ref = AD.mrcm_os_adjoint(prob, case.partition.sub, case.partition.overlap, pm.space, pm.alpha_basis,
                                  pm.alpha_smooth, pm.n_smooth, np.zeros(prob.ncells), gu)
    assert np.max(np.abs(g - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))

    # central differences, h = 1e-6
    h = 1e-6
    rng = np.random.default_rng(2024)
    strong = np.flatnonzero(np.abs(g) >= 1e-2 * gmax)
    coords = np.concatenate([rng.choice(strong, min(32, len(strong)), replace=False),
                             rng.choice(prob.ncells, 64 - min(32, len(strong)), replace=False)])

    def L_at(th):
        with torch.no_grad():
            return float(loss_of(th))

    worst = 0.0
    for j in coords:
        e = torch.zeros_like(theta0)
        e[int(j)] = h
        fd = (L_at(theta0 + e) - L_at(theta0 - e)) / (2 * h)
        worst = max(worst, abs(fd - g[j]) / gmax)
    assert worst <= 1e-6, worst
    gn = np.linalg.norm(g)
    worst = 0.0
    for _ in range(16):
        v = rng.standard_normal(prob.ncells)
        vt = torch.as_tensor(v * h, device="cuda")
        fd = (L_at(theta0 + vt) - L_at(theta0 - vt)) / (2 * h)
        worst = max(worst, abs(fd - g @ v) / (gn * np.linalg.norm(v)))
    assert worst <= 1e-6, worst

    # a second forward on the same handle makes the first graph's backward stale
    theta2 = theta0.clone().requires_grad_(True)
    La = loss_of(theta2)
    loss_of(theta0)
    with pytest.raises(RuntimeError):
        La.backward()
    s.close()
