"""The particular problem on hat-Omega_i (a variant of Step 4 that is not in
the paper, particular="hat") through the C ABI against the oracle's variant,
element by element; same bars as the method itself: relative L2 of fluxes
and pressures <= 1e-10 in the FP64 form and <= 1e-8 in the mixed form, plus a
max-abs bound of 10x the same tolerance relative to the field's max."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}


def _solver(case, precision, particular="hat"):
    from paper_2404_13811_gb300.solver import MRCM
    pm = case.params
    return MRCM(case.problem, case.partition, space=pm.space, alpha_basis=pm.alpha_basis,
                alpha_smooth=pm.alpha_smooth, precision=precision, particular=particular)


def _compare(prob, p, u, p_ref, u_ref, tol, what):
    ep, eu = O.rel_errors(prob, p, u, p_ref, u_ref)
    assert ep <= tol and eu <= tol, f"{what}: rel L2 p {ep:.2e} u {eu:.2e} > {tol:.0e}"
    assert np.max(np.abs(u - u_ref)) <= 10 * tol * np.max(np.abs(u_ref)), what
    assert np.max(np.abs(p - p_ref)) <= 10 * tol * max(np.max(np.abs(p_ref)), 1e-300), what


def _run_compare(case, precision, stages=(0,)):
    pm = case.params
    ref = O.mrcm_os(case.problem, case.partition.sub, case.partition.overlap, pm.space,
                    pm.alpha_basis, pm.alpha_smooth, max(stages), keep_stages=True, particular="hat")
    s = _solver(case, precision)
    s.build_basis()
    s.solve_interface()
    done = 0
    for k in sorted(stages):
        if k > done:
            s.smooth(k - done)
            done = k
        p, u = s.fluxes()
        rp, ru = ref.stages["mrcm_o" if k == 0 else f"smooth{k}"]
        _compare(case.problem, p, u, rp, ru, TOL[precision], f"{case.name} {precision} stage {k}")
    s.close()
    return ref


def _case(n, sub, overlap, space, alpha_b=1.0, alpha_s=1.0, ns=2, seed=1, h=None):
    prob = I.lognormal_problem(n, sigma2=2.0, corr_len=0.15, seed=seed, bc="left_right")
    prob.f = np.random.default_rng(seed + 11).standard_normal(prob.f.shape)
    if h is not None:
        prob.h = tuple(h)
    return I.Case(prob, I.Partition(sub, overlap), I.MethodParams(space, alpha_b, alpha_s, ns),
                  name=f"{n}_{sub}_l{overlap}_P{space}_hat")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("space", [0, 1])
def test_hat_particular_channel_128(precision, space):
    """128x128 channelised field, 8x8 subdomains of 16 cells, overlap 4:
    MRCM-O and two smoothing steps."""
    case = I.config_channel2d(n=128, sub=16, overlap=4, n_smooth=2)
    case.params.space = space
    _run_compare(case, precision, stages=(0, 2))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hat_particular_ragged_with_sources(precision):
    """Non-square grid and subdomains (6 x 4 blocks of 16 x 12), anisotropic
    h, random sources, boxes truncated at every side of the domain."""
    case = _case((96, 48), (16, 12), 3, 1, h=(1 / 96, 0.6 / 48), ns=3)
    _run_compare(case, precision, stages=(0, 3))


def test_hat_particular_separate_smoothing_factor():
    """alpha_basis != alpha_smooth: the particular problem uses the basis
    factor (alpha_basis), the smoothing its own."""
    case = _case((64, 64), (16, 16), 2, 1, alpha_b=0.05, alpha_s=1.0, ns=2, seed=3)
    _run_compare(case, "fp64", stages=(0, 2))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hat_particular_pure_neumann(precision):
    """64x64 quarter five-spot with no-flow boundary (the gauge), P0, alpha_basis 1e-2."""
    case = I.config_small()
    _run_compare(case, precision, stages=(0, 4))


def test_hat_particular_equals_step4_for_l0():
    """l = 0: hat-Omega_i = Omega_i and the variant is Step 4 itself."""
    case = _case((64, 64), (16, 16), 0, 1, ns=0, seed=5)
    a = _solver(case, "fp64", particular="omega")
    a.run(0)
    pa, ua = a.fluxes()
    a.close()
    b = _solver(case, "fp64", particular="hat")
    b.run(0)
    pb, ub = b.fluxes()
    b.close()
    assert np.max(np.abs(pa - pb)) <= 1e-12 * np.max(np.abs(pa))
    assert np.max(np.abs(ua - ub)) <= 1e-12 * np.max(np.abs(ua))


def test_hat_particular_full_size_channel_512_captured_step():
    """The 512x512 channel workload (32x32 subdomains, P1, overlap 4, 8
    smoothing steps) with the variant, the step captured as one CUDA graph
    (first and second call), mixed form, against the oracle on every cell."""
    case = I.config_channel2d()
    pm = case.params
    ref = O.mrcm_os(case.problem, case.partition.sub, case.partition.overlap, pm.space,
                    pm.alpha_basis, pm.alpha_smooth, pm.n_smooth, particular="hat")
    s = _solver(case, "mixed")
    for call in range(2):
        s.run(pm.n_smooth, graph=True)
        p, u = s.fluxes()
        _compare(case.problem, p, u, ref.p, ref.u, TOL["mixed"], f"hat 512 graph call {call}")
    st = s.stats()
    s.close()
    assert st["subdomains"] == 1024


CASES3 = [
    # n, sub, overlap, space, alpha_basis, alpha_smooth, n_smooth, bc
    ((20, 16, 12), (10, 8, 6), 2, 0, 1.0, 1.0, 2, "left_right"),
    ((24, 12, 16), (8, 6, 8), 1, 1, 1.0, 1.0, 1, "left_right"),
    ((16, 16, 8), (8, 8, 4), 1, 0, 1.0, 1.0, 2, "noflow"),
    ((16, 12, 12), (8, 6, 6), 1, 1, 0.5, 1.0, 1, "left_right"),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", range(len(CASES3)))
def test_hat_particular_3d(case, precision):
    """3D boxes (plane-block factor): the particular problem is the basis
    job's last right-hand side in its group of four; random sources, P0 and
    P1, pure Neumann, Step 6."""
    from paper_2404_13811_gb300.solver import MRCM
    n, sub, ov, space, ab, as_, ns, bc = CASES3[case]
    prob = I.lognormal_problem(n, sigma2=2.0, corr_len=0.2, seed=170 + case, bc=bc)
    prob.f = np.random.default_rng(173 + case).standard_normal(prob.f.shape)
    if bc == "noflow":
        prob.f -= prob.f.mean()
    ref = O.mrcm_os(prob, sub, ov, space, ab, as_, ns, particular="hat")
    s = MRCM(prob, I.Partition(sub, ov), space=space, alpha_basis=ab, alpha_smooth=as_, precision=precision,
             particular="hat")
    s.run(ns)
    p, u = s.fluxes()
    s.close()
    _compare(prob, p, u, ref.p, ref.u, TOL[precision], f"3D case {case} {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [0, 1])
def test_hat_particular_gradient_matches_oracle_gradient(case, precision):
    """mrcm_adjoint with the particular problem on hat-Omega_i against the
    oracle's adjoint of the variant (itself pinned by complex step): max
    |g - g_oracle| <= 1e-8 max |g_oracle|, as for the method."""
    from oracle import mrcm_adjoint as AD
    from paper_2404_13811_gb300.solver import MRCM
    n, sub, ov, space, ab, as_, ns = [((64, 48), (16, 16), 2, 1, 1.0, 1.0, 2),
                                      ((64, 32), (16, 16), 3, 0, 2.0, 0.5, 1)][case]
    prob = I.lognormal_problem(n, sigma2=3.0, corr_len=0.15, seed=260 + case)
    prob.f = np.random.default_rng(261 + case).standard_normal(prob.f.shape)
    rng = np.random.default_rng(270 + case)
    wp, wu = rng.standard_normal(prob.ncells), rng.standard_normal((prob.ncells, 4))
    _, g_ref = AD.mrcm_os_adjoint(prob, sub, ov, space, ab, as_, ns, wp, wu, particular="hat")
    s = MRCM(prob, I.Partition(sub, ov), space=space, alpha_basis=ab, alpha_smooth=as_, precision=precision,
             particular="hat")
    s.run(ns)
    g = s.adjoint(wp, wu)
    s.close()
    err = np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))
    assert err <= 1e-8, err
