"""Batching form: uneven subdomains and whole ensembles in one submission
(mrcm_create_batch: one launch per kernel over all subdomains of all members),
and the whole step replayed as one captured CUDA graph (mrcm_run)."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}


def _members():
    out = []
    specs = [((64, 64), (16, 16), 2, 2.0, "left_right", None),
             ((96, 48), (16, 16), 3, 4.0, "left_right", None),
             ((128, 128), (16, 16), 4, 3.0, "left_right", None),
             ((48, 80), (16, 16), 2, 1.0, "noflow", "q5")]
    for m, (n, sub, l, s2, bc, src) in enumerate(specs):
        prob = I.lognormal_problem(n, sigma2=s2, corr_len=0.15, seed=40 + m, bc=bc, source=src)
        out.append((prob, I.Partition(sub, l)))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_ensemble_matches_oracle_per_member(precision):
    from paper_2404_13811_gb300.solver import MRCM
    mem = _members()
    s = MRCM([p for p, _ in mem], [q for _, q in mem], space=1, precision=precision)
    s.run(2)
    st = s.stats()
    assert st["subdomains"] == sum((p.n[0] // q.sub[0]) * (p.n[1] // q.sub[1]) for p, q in mem)
    for m, (prob, part) in enumerate(mem):
        ref = O.mrcm_os(prob, part.sub, part.overlap, 1, 1.0, 1.0, 2)
        p, u = s.fluxes(m)
        ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
        assert ep <= TOL[precision] and eu <= TOL[precision], (m, ep, eu)
    s.close()


def test_captured_step_replays_the_eager_step():
    """Replays of the captured step are bitwise identical (the step has no
    order-dependent accumulation), and the captured step runs the eager
    step's refinement count.  Against the eager step the bar is 1e-9
    relative, the refinement tolerances (1e-12 relative residuals, interface
    and local) carried through the local solves and the smoothing steps."""
    from paper_2404_13811_gb300.solver import MRCM
    mem = _members()
    a = MRCM([p for p, _ in mem], [q for _, q in mem], space=1, precision="mixed")
    a.run(3)
    ref = [a.fluxes(m) for m in range(len(mem))]
    a.close()
    b = MRCM([p for p, _ in mem], [q for _, q in mem], space=1, precision="mixed")
    first = None
    for rep in range(3):
        b.run(3, graph=True)
        got = [b.fluxes(m) for m in range(len(mem))]
        if first is None:
            first = got
        for m in range(len(mem)):
            p, u = got[m]
            assert np.array_equal(p, first[m][0]) and np.array_equal(u, first[m][1]), (rep, m)
            assert np.max(np.abs(p - ref[m][0])) <= 1e-9 * np.max(np.abs(ref[m][0])), (rep, m)
            assert np.max(np.abs(u - ref[m][1])) <= 1e-9 * np.max(np.abs(ref[m][1])), (rep, m)
    from paper_2404_13811_gb300 import _lib as L
    b.profile(True)
    b.run(3, graph=True)
    tm = b.timings()
    assert tm["graph"][1] == 1 and tm["local_basis"][1] == 0   # one graph launch, no eager launches
    b.close()
