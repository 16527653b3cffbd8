"""Failure detection without a GPU fault: each failure is made on the host
(an unreachable tolerance, out-of-range inputs) or by a bounded wait that is
made to run out; each test checks the error code the host reads back and that
the context stays usable afterwards."""
import numpy as np
import pytest

from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _solver(case, **kw):
    from paper_2404_13811_gb300.solver import MRCM
    pm = case.params
    args = dict(space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth, precision="mixed")
    args.update(kw)
    return MRCM(case.problem, case.partition, **args)


def _still_usable():
    s = _solver(I.config_channel2d(n=64, n_smooth=1))
    s.run(1)
    p, _ = s.fluxes()
    s.close()
    assert np.all(np.isfinite(p))


def test_unreachable_local_tolerance_reports_no_convergence():
    """One refinement step cannot reach a relative residual of 1e-30: the
    local solves flag it and the host returns MRCM_ERR_NO_CONVERGENCE."""
    from paper_2404_13811_gb300 import _lib as L
    s = _solver(I.config_channel2d(n=64, n_smooth=1), ir_tol=1e-30, max_ir=1)
    with pytest.raises(L.MrcmError) as ei:
        s.build_basis()
    assert ei.value.code == -5, ei.value
    s.close()
    _still_usable()


@pytest.mark.parametrize("bad,is_log", [(-1.0, 0), (float("nan"), 0), (float("inf"), 1)])
def test_device_permeability_out_of_range_is_rejected(bad, is_log):
    """mrcm_set_permeability with device values checks them on the device:
    a value <= 0, NaN (K) or an infinite log K returns MRCM_ERR_BAD_INPUT."""
    import torch
    from paper_2404_13811_gb300 import _lib as L
    case = I.config_channel2d(n=64, n_smooth=1)
    s = _solver(case)
    s.run(1)
    v = torch.as_tensor(np.log(case.problem.K) if is_log else case.problem.K, dtype=torch.float64).cuda().reshape(-1)
    v[123] = bad
    with pytest.raises(L.MrcmError) as ei:
        L.mrcm_set_permeability(s.h, v, is_log)
    assert ei.value.code == -1, ei.value
    s.close()
    _still_usable()


def test_device_nan_permeability_gives_non_positive_pivot():
    """Permeability given as device memory is not read back at creation; a NaN
    there reaches the local factorisation, whose pivot test (piv > 0 fails for
    NaN) reports MRCM_ERR_NOT_SPD from mrcm_build_basis."""
    from paper_2404_13811_gb300 import _lib as L
    case = I.config_channel2d(n=64, n_smooth=1)
    case.problem.K = case.problem.K.copy()
    case.problem.K.flat[777] = float("nan")
    s = _solver(case, precision="fp64", device_inputs=True)
    with pytest.raises(L.MrcmError) as ei:
        s.build_basis()
    assert ei.value.code == -4, ei.value
    s.close()
    _still_usable()


def test_late_staged_copy_reports_timeout(monkeypatch):
    """The smoothing kernel waits for its staged factor with a cycle limit.
    With MRCM_TEST_FIRST_WAIT_CYCLES set at creation, the first wait is one
    of that many cycles for a barrier nothing arrives at, so it runs out; the
    kernel waits again at the full limit for the copy in flight, skips the
    solve and flags it, and mrcm_smooth returns MRCM_ERR_TIMEOUT.  A handle
    created afterwards without the variable works."""
    from paper_2404_13811_gb300 import _lib as L
    monkeypatch.setenv("MRCM_TEST_FIRST_WAIT_CYCLES", "20000")
    s = _solver(I.config_channel2d(n=64, n_smooth=1))
    monkeypatch.delenv("MRCM_TEST_FIRST_WAIT_CYCLES")
    s.build_basis()
    s.solve_interface()
    with pytest.raises(L.MrcmError) as ei:
        s.smooth(1)
    assert ei.value.code == -9, ei.value
    s.close()
    _still_usable()
