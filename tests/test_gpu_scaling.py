"""Scale invariance of the discrete Darcy problem (Eqs. (1a)-(1d)): with
Dirichlet data and no source, K -> c K leaves the pressure unchanged and
scales every velocity by c.  At c far outside the FP32 range this exercises
the FP64 reciprocals of the face laws and pivots (an FP32 seed would be 0 or
infinite there) and the Jacobi scale of the mixed form."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,scales,tol", [("fp64", (1e-300, 1e-45, 1e45, 1e300), 1e-10),
                                                   ("mixed", (1e-30, 1e30), 1e-8)])
def test_permeability_scale_invariance(precision, scales, tol):
    from paper_2404_13811_gb300.solver import MRCM
    case = I.config_channel2d(n=64, n_smooth=2)
    pm = case.params

    def run(K):
        prob = I.Problem(2, case.problem.n, case.problem.h, K, case.problem.f, case.problem.bc_kind,
                         case.problem.bc_value)
        s = MRCM(prob, case.partition, space=pm.space, alpha_basis=pm.alpha_basis, alpha_smooth=pm.alpha_smooth,
                 precision=precision)
        s.run(2)
        p, u = s.fluxes()
        s.close()
        return prob, p, u

    prob, p0, u0 = run(case.problem.K)
    for c in scales:
        _, p, u = run(case.problem.K * c)
        ep, eu = O.rel_errors(prob, p, u / c, p0, u0)
        assert np.all(np.isfinite(p)) and ep <= tol and eu <= tol, (c, ep, eu)
