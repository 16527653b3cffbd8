"""3D subdomains on the GPU: plane-block factorisation, basis / particular
solves, interface, smoothing -- element-by-element parity with the oracle on
problems the oracle finishes in seconds, and properties that hold at any size
on the 60 x 220 x 85 layered workload (per-cell mass conservation, FP64 vs
mixed agreement)."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}


def _problem3(n, seed, bc="left_right", source=True, sigma2=2.0):
    prob = I.lognormal_problem(n, sigma2=sigma2, corr_len=0.2, seed=seed, bc=bc)
    if source:
        rng = np.random.default_rng(seed + 3)
        prob.f = rng.standard_normal(prob.f.shape)
    return prob


CASES = [
    # n, sub, overlap, space, alpha_basis, alpha_smooth, n_smooth, bc
    ((20, 16, 12), (10, 8, 6), 2, 0, 1.0, 1.0, 2, "left_right"),
    ((24, 12, 16), (8, 6, 8), 1, 1, 1.0, 1.0, 1, "left_right"),
    ((16, 16, 8), (8, 8, 4), 1, 0, 1.0, 1.0, 2, "noflow"),
    ((16, 12, 12), (8, 6, 6), 0, 1, 0.5, 1.0, 1, "left_right"),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_3d_matches_oracle(case, precision):
    from paper_2404_13811_gb300.solver import MRCM
    n, sub, ov, space, ab, as_, ns, bc = CASES[case]
    prob = _problem3(n, seed=70 + case, bc=bc)
    if bc == "noflow":
        prob.f -= prob.f.mean()
    ref = O.mrcm_os(prob, sub, ov, space, ab, as_, ns)
    s = MRCM(prob, I.Partition(sub, ov), space=space, alpha_basis=ab, alpha_smooth=as_, precision=precision)
    s.run(ns)
    p, u = s.fluxes()
    ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
    assert ep <= TOL[precision] and eu <= TOL[precision], (ep, eu)
    s.close()


def test_3d_layered_midsize_matches_oracle():
    """The layered character of the 60x220x85 workload (log-normal lower
    layers, channels of contrast 1e6 above) at 30x40x20, subdomains 10x10x5,
    overlap 2, P0, 4 smoothing steps, mixed form."""
    from paper_2404_13811_gb300.solver import MRCM
    case = I.config_layered3d(n=(30, 40, 20), n_upper=8)
    prob, pm = case.problem, case.params
    ref = O.mrcm_os(prob, case.partition.sub, case.partition.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth,
                    pm.n_smooth)
    for precision in ("fp64", "mixed"):
        s = MRCM(prob, case.partition, space=pm.space, precision=precision)
        s.run(pm.n_smooth)
        p, u = s.fluxes()
        ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
        assert ep <= TOL[precision] and eu <= TOL[precision], (precision, ep, eu)
        s.close()


def test_3d_full_size_layered_matches_oracle():
    """60x220x85 (1.12M cells, 2244 subdomains, 10x10x5 oversampled by 2,
    P0, 4 smoothing steps; the oracle takes about a minute): element-by-
    element parity of both forms, and per-cell mass conservation."""
    from paper_2404_13811_gb300.solver import MRCM
    case = I.config_layered3d()
    prob, pm = case.problem, case.params
    ref = O.mrcm_os(prob, case.partition.sub, case.partition.overlap, pm.space, pm.alpha_basis, pm.alpha_smooth,
                    pm.n_smooth)
    for precision in ("mixed", "fp64"):
        s = MRCM(prob, case.partition, space=pm.space, precision=precision)
        s.run(pm.n_smooth)
        p, u = s.fluxes()
        st = s.stats()
        s.close()
        assert st["subdomains"] == 2244
        ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
        assert ep <= TOL[precision] and eu <= TOL[precision], (precision, ep, eu)
        res = O.mass_residual(prob, u)
        flux_scale = np.max(np.abs(u)) * prob.h[1] * prob.h[2]
        assert np.max(np.abs(res)) <= 1e-9 * flux_scale
