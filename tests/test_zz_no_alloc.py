"""mrcm_fluxes_static: the output entry point for callers that cannot allocate
device memory when they read results (their device memory is held by another
framework's allocator, or they run in a loop that must not allocate).  It must
give the values of mrcm_fluxes, call after call, while allocating nothing and
using its fixed static gauge scratch.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(case):
    from paper_2404_13811_gb300.solver import MRCM
    pm = case.params
    s = MRCM(case.problem, case.partition, space=pm.space, alpha_basis=pm.alpha_basis,
             alpha_smooth=pm.alpha_smooth, precision="fp64")
    s.run(2)
    return s


@pytest.mark.parametrize("which", ["pure_neumann", "dirichlet"])
def test_fluxes_static_matches_fluxes_on_two_calls(which):
    import torch
    from paper_2404_13811_gb300 import _lib as L
    case = I.config_small() if which == "pure_neumann" else I.config_channel2d(n=128, n_smooth=2)
    s = _run(case)
    p_ref, u_ref = s.fluxes(device=True)          # the existing entry point, device buffers
    torch.cuda.synchronize()
    p_ref, u_ref = p_ref.cpu().numpy(), u_ref.cpu().numpy()
    nc = case.problem.ncells
    for call in range(2):
        p = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
        u = torch.full((nc, 4), float("nan"), dtype=torch.float64, device="cuda")
        L.mrcm_fluxes_static(s.h, 0, u, p)
        torch.cuda.synchronize()
        p, u = p.cpu().numpy(), u.cpu().numpy()
        assert np.max(np.abs(p - p_ref)) <= 1e-10 * np.max(np.abs(p_ref)), (which, call)
        assert np.array_equal(u, u_ref), (which, call)
    s.close()
