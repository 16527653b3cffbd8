"""The studies of the paper's Sec. 4 on the GPU path, widened: the alpha
sweep 1e-8 .. 1e8 of Fig. hete-OL4-norm, piecewise constant (OC) against
linear (OL) interface spaces and the original MRCM (l = 0) of
Fig. het-OC-norm, and the homogeneous cos-cos problem (Sec. 4.1) of
Figs. analytical-O, homo-number and analytical-OS.  Errors are relative L2
norms of fluxes against the fine-scale solution (the paper's measure);
every table is printed (pytest -s).  The paper's figures carry no numbers
in the text, so the asserts are its stated directions, on the synthetic
stand-in for its heterogeneous field:
* MRCM-OS with oversampling 4h and 4 smoothing steps beats MRCM (l = 0) on
  the flux by a factor 5 at alpha >= 1 and by two orders of magnitude at
  alpha >= 1e2 (the paper's "two orders"; below alpha = 1 oversampling does
  not pay on this field: MRCM-O with oversampling wants a large alpha);
* MRCM (l = 0) does best near alpha = 1 (the paper: optimal outcomes when
  alpha approximates 1);
* OC with oversampling 2h and 2 smoothing steps beats MRCM with linear spaces
  on the flux at alpha = 1 and 1e2, with half its basis functions;
* homogeneous problem: oversampling 4h alone beats l = 0 (the paper: about
  half the error); with oversampling 2h the error falls with every smoothing
  step, by an order of magnitude after 2 steps and two after 4 (the paper:
  one order in pressure, two in flux).  The paper's diminishing gain beyond
  2-4 steps is not seen here: the error falls by about 3x per step up to 8.
The interface factor is FP32 with FP64 refinement: beyond alpha = 1e4 (P0)
or 1e5 (P1) it is too poor a preconditioner, and those solves must fail
loudly (MRCM_ERR_NO_CONVERGENCE or MRCM_ERR_SINGULAR), not return a result.
Sampled configurations are compared with the oracle's MRCM-OS as well."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ALPHAS = (1e-8, 1e-6, 1e-4, 1e-2, 1.0, 1e2, 1e4, 1e5, 1e6, 1e8)
CONVERGE_UP_TO = {"mrcm": 1e5, "ol": 1e5, "oc": 1e4}


def _run(prob, space, l, alpha, steps):
    """Flux errors against the fine solution after each count in steps, or
    None when the interface solve fails (the error code is checked)."""
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300.solver import MRCM
    s = MRCM(prob, I.Partition((16, 16), l), space=space, alpha_basis=alpha, alpha_smooth=1.0, precision="fp64")
    try:
        s.build_basis()
        s.solve_interface()
    except L.MrcmError as exc:
        s.close()
        assert exc.code in (-5, -6), exc   # NO_CONVERGENCE / SINGULAR
        return None, None
    out, done = [], 0
    for k in steps:
        s.smooth(k - done)
        done = k
        out.append(s.fluxes())
    s.close()
    return out, done


def _err(prob, pu, ref):
    p, u = pu
    return O.rel_errors(prob, p, u.reshape(ref[1].shape), ref[0], ref[1])[1]


def test_alpha_sweep_oc_ol_and_mrcm_heterogeneous():
    prob = I.lognormal_problem((128, 128), sigma2=4.0, corr_len=0.1, seed=616)
    prob.f = np.random.default_rng(617).standard_normal(prob.f.shape)
    fine = O.fine_solve(prob)
    rows = {}
    for alpha in ALPHAS:
        mrcm, _ = _run(prob, 1, 0, alpha, (0,))
        ol4, _ = _run(prob, 1, 4, alpha, (0, 4))
        oc2, _ = _run(prob, 0, 2, alpha, (0, 2))
        rows[alpha] = (None if mrcm is None else _err(prob, mrcm[0], fine),
                       None if ol4 is None else [_err(prob, x, fine) for x in ol4],
                       None if oc2 is None else [_err(prob, x, fine) for x in oc2])
        if alpha in (1e-8, 1.0, 1e5) and ol4 is not None:
            # the GPU's MRCM-OS is the method's: the oracle on the same configuration
            ref = O.mrcm_os(prob, (16, 16), 4, 1, alpha, 1.0, 4)
            e_or = O.rel_errors(prob, ol4[1][0], ol4[1][1].reshape(ref.u.shape), ref.p, ref.u)
            assert max(e_or) <= 1e-8, (alpha, e_or)
    fmt = lambda v: "  fails  " if v is None else f"{v:.2e}"
    print("\nflux rel L2 vs the fine solution (128x128 log-normal, 8x8 subdomains)")
    print("  alpha      MRCM(P1,l0)  OL-4      OL-4,4S   OC-2      OC-2,2S")
    for alpha, (m, o4, c2) in rows.items():
        o4s = (fmt(None), fmt(None)) if o4 is None else (fmt(o4[0]), fmt(o4[1]))
        c2s = (fmt(None), fmt(None)) if c2 is None else (fmt(c2[0]), fmt(c2[1]))
        print(f"  {alpha:7.0e}    {fmt(m)}   {o4s[0]}  {o4s[1]}  {c2s[0]}  {c2s[1]}")
    for alpha, (m, o4, c2) in rows.items():
        assert m is not None or alpha > CONVERGE_UP_TO["mrcm"], alpha
        assert o4 is not None or alpha > CONVERGE_UP_TO["ol"], alpha
        assert c2 is not None or alpha > CONVERGE_UP_TO["oc"], alpha
        if m is not None and o4 is not None and alpha >= 1.0:
            assert o4[1] < m / (100.0 if alpha >= 1e2 else 5.0), (alpha, m, o4)
    mrcm = {a: r[0] for a, r in rows.items() if r[0] is not None}
    assert min(mrcm, key=mrcm.get) in (1.0, 1e2), mrcm
    for alpha in (1.0, 1e2):
        m, _, c2 = rows[alpha]
        assert c2[1] < m, (alpha, m, c2)


def test_homogeneous_oversampling_and_smoothing_steps():
    prob = I.homogeneous_problem(128)
    fine = O.fine_solve(prob)
    m, _ = _run(prob, 1, 0, 1.0, (0,))
    o4, _ = _run(prob, 1, 4, 1.0, (0,))
    o2, _ = _run(prob, 1, 2, 1.0, (0, 1, 2, 4, 8))
    em = _err(prob, m[0], fine)
    e4 = _err(prob, o4[0], fine)
    e2 = [_err(prob, x, fine) for x in o2]
    print(f"\nhomogeneous cos-cos, 128x128, 8x8 subdomains, alpha 1: MRCM {em:.2e}, OL-4 {e4:.2e}, "
          f"OL-2 with N_s = 0, 1, 2, 4, 8: " + "  ".join(f"{x:.2e}" for x in e2))
    assert e4 < 0.75 * em
    assert all(e2[i + 1] < e2[i] for i in range(len(e2) - 1)), e2
    assert e2[2] < em / 10 and e2[3] < em / 100, (em, e2)
