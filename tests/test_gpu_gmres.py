"""The interface GMRES fallback against the oracle, element by element.

At alpha_basis = 1e5 with overlap the interface system of Eqs.
(int_ujump)-(int_pjump) is too ill-conditioned for stationary refinement
with the FP32 reduction factor; the solve continues with FP64 GMRES
preconditioned by that factor (Algorithm 1, Step 5).  The oracle solves the
same system directly (equilibrated LU with FP64 refinement).  Both stop at
small relative residuals, so their interface coefficients can differ by up
to about cond(equilibrated G) x (the two residuals); the bar is ten times
that bound, computed from the oracle's system and printed with the errors."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("overlap", [2, 4])
def test_interface_gmres_fallback_matches_oracle(overlap):
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300.solver import MRCM
    prob = I.lognormal_problem((128, 128), sigma2=4.0, corr_len=0.1, seed=606)
    prob.f = np.random.default_rng(607).standard_normal(prob.f.shape)
    s = MRCM(prob, I.Partition((16, 16), overlap), space=1, alpha_basis=1e5, alpha_smooth=1.0, precision="fp64")
    s.build_basis()
    s.solve_interface()
    st = L.mrcm_stats(s.h)
    assert st["interface_gmres"], st          # the fallback ran
    p, u = s.fluxes()
    s.close()
    ref = O.mrcm_os(prob, (16, 16), overlap, 1, 1e5, 1.0, 0)
    G, b = ref.G, ref.rhs
    Rr = 1.0 / np.abs(G).max(axis=1)
    Ge = G * Rr[:, None]
    Ge = Ge * (1.0 / np.abs(Ge).max(axis=0))[None, :]
    kappa = np.linalg.cond(Ge)
    res_o = np.abs(G @ ref.X - b).max() / np.abs(b).max()
    bar = 10.0 * kappa * (st["interface_residual"] + res_o)
    ep, eu = O.rel_errors(prob, p, u.reshape(ref.u.shape), ref.p, ref.u)
    print(f"\noverlap {overlap}: cond(equilibrated G) {kappa:.2e}, residuals GPU {st['interface_residual']:.2e} "
          f"oracle {res_o:.2e}; bar {bar:.2e}; rel L2 p {ep:.2e} u {eu:.2e}")
    assert ep <= bar and eu <= bar
