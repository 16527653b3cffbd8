"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Bar (stated per result): relative L2 of fluxes and pressures <= 1e-10 in the
FP64 form and <= 1e-8 in the mixed form (FP32 factor + FP64 refinement),
plus a max-abs bound of 10x the same tolerance relative to the field's max.
"""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}


def _solver(case, precision, **kw):
    from paper_2404_13811_gb300.solver import MRCM
    pm = case.params
    return MRCM(case.problem, case.partition, space=pm.space, alpha_basis=pm.alpha_basis,
                alpha_smooth=pm.alpha_smooth, precision=precision, **kw)


def _compare(prob, p, u, p_ref, u_ref, tol, what):
    ep, eu = O.rel_errors(prob, p, u, p_ref, u_ref)
    assert ep <= tol and eu <= tol, f"{what}: rel L2 p {ep:.2e} u {eu:.2e} > {tol:.0e}"
    assert np.max(np.abs(u - u_ref)) <= 10 * tol * np.max(np.abs(u_ref)), what
    assert np.max(np.abs(p - p_ref)) <= 10 * tol * max(np.max(np.abs(p_ref)), 1e-300), what
    return ep, eu


def _run_compare(case, precision, stages=(0,)):
    pm = case.params
    ref = O.mrcm_os(case.problem, case.partition.sub, case.partition.overlap, pm.space,
                    pm.alpha_basis, pm.alpha_smooth, max(stages), keep_stages=True)
    s = _solver(case, precision)
    s.build_basis()
    s.solve_interface()
    done = 0
    out = {}
    for k in sorted(stages):
        if k > done:
            s.smooth(k - done)
            done = k
        p, u = s.fluxes()
        key = "mrcm_o" if k == 0 else f"smooth{k}"
        rp, ru = ref.stages[key]
        out[key] = _compare(case.problem, p, u, rp, ru, TOL[precision], f"{case.name} {precision} {key}")
    st = s.stats()
    s.close()
    return out, st


def _case(n, sub, overlap, space, alpha_b=1.0, alpha_s=1.0, ns=2, seed=1, bc="left_right",
          source=None, h=None, sigma2=2.0):
    prob = I.lognormal_problem(n, sigma2=sigma2, corr_len=0.15, seed=seed, bc=bc, source=source)
    if h is not None:
        prob.h = tuple(h)
    return I.Case(prob, I.Partition(sub, overlap), I.MethodParams(space, alpha_b, alpha_s, ns),
                  name=f"{n}_{sub}_l{overlap}_P{space}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_pure_neumann_p0(precision):
    """64x64, 4x4 subdomains oversampled by 2, P0, alpha_basis = 1e-2,
    quarter-five-spot, no-flow boundary (gauge + zero-mean pressure), 4 steps."""
    case = I.config_small()
    out, st = _run_compare(case, precision, stages=(0, 1, 4))
    assert st["interface_unknowns"] == 48


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("space", [0, 1])
def test_dirichlet_channel_128(precision, space):
    case = I.config_channel2d(n=128, sub=16, overlap=4, n_smooth=2)
    case.params.space = space
    _run_compare(case, precision, stages=(0, 2))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ragged_grid_anisotropic(precision):
    """Non-square grid and subdomains (6 x 4 blocks of 16 x 12), anisotropic h,
    boxes truncated at every side of the domain."""
    case = _case((96, 48), (16, 12), 3, 1, h=(1 / 96, 0.6 / 48), ns=3)
    _run_compare(case, precision, stages=(0, 3))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step6_separate_smoothing_factor(precision):
    """alpha_basis != alpha_smooth: the smoothing operator is factored separately."""
    case = _case((64, 64), (16, 16), 2, 1, alpha_b=0.05, alpha_s=1.0, ns=2, seed=3)
    _run_compare(case, precision, stages=(0, 2))


def test_original_mrcm_l0():
    """l = 0 (the original MRCM): Robin faces of the basis boxes are Gamma_i."""
    case = _case((64, 64), (16, 16), 0, 1, ns=0, seed=5)
    _run_compare(case, "fp64", stages=(0,))


def test_two_subdomains_minimum():
    case = _case((32, 16), (16, 16), 3, 1, ns=2, seed=7)
    _run_compare(case, "fp64", stages=(0, 2))


def test_smoothing_is_additive_bitwise():
    """smooth(2); smooth(1) gives the same bits as smooth(3)."""
    case = _case((64, 64), (16, 16), 2, 1, seed=9)
    a = _solver(case, "mixed")
    a.run(0)
    a.smooth(2)
    a.smooth(1)
    pa, ua = a.fluxes()
    b = _solver(case, "mixed")
    b.run(3)
    pb, ub = b.fluxes()
    assert np.array_equal(pa, pb) and np.array_equal(ua, ub)


def test_call_order_enforced():
    from paper_2404_13811_gb300 import _lib as L
    case = _case((32, 32), (16, 16), 2, 1)
    s = _solver(case, "fp64")
    with pytest.raises(L.MrcmError) as e:
        s.solve_interface()
    assert e.value.code == -2
    with pytest.raises(L.MrcmError):
        s.smooth(1)
    s.build_basis()
    s.solve_interface()
    s.smooth(1)
    p1, u1 = s.fluxes()
    s.build_basis()          # restarts the pipeline
    with pytest.raises(L.MrcmError):
        s.smooth(1)
    s.solve_interface()
    s.smooth(1)
    p2, u2 = s.fluxes()
    assert np.array_equal(p1, p2) and np.array_equal(u1, u2)


_CHANNEL512 = {}


def _channel512():
    """The 512x512 workload and its oracle result, computed once per session."""
    if not _CHANNEL512:
        case = I.config_channel2d()
        pm = case.params
        ref = O.mrcm_os(case.problem, case.partition.sub, case.partition.overlap, pm.space,
                        pm.alpha_basis, pm.alpha_smooth, pm.n_smooth, keep_stages=True)
        _CHANNEL512["v"] = (case, ref)
    return _CHANNEL512["v"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_channel_512(precision):
    """The 512x512 channelised workload (32x32 subdomains, P1, overlap 4,
    8 smoothing steps) through the eager calls, compared with the oracle on
    every cell."""
    case, ref = _channel512()
    s = _solver(case, precision)
    s.build_basis()
    s.solve_interface()
    s.smooth(case.params.n_smooth)
    p, u = s.fluxes()
    s.close()
    rp, ru = ref.stages[f"smooth{case.params.n_smooth}"]
    _compare(case.problem, p, u, rp, ru, TOL[precision], f"{case.name} {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_channel_512_captured_step(precision):
    """The same workload as the benchmark times it: mrcm_run with the step
    captured as one CUDA graph -- the first call (eager run, capture, one
    replay) and a second call (replay only), each compared with the oracle
    on every cell."""
    case, ref = _channel512()
    rp, ru = ref.stages[f"smooth{case.params.n_smooth}"]
    s = _solver(case, precision)
    for call in range(2):
        s.run(case.params.n_smooth, graph=True)
        p, u = s.fluxes()
        _compare(case.problem, p, u, rp, ru, TOL[precision], f"{case.name} {precision} graph call {call}")
    s.close()
