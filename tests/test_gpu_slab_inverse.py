"""Every slab inverse of the interface reduction (block cyclic reduction over
layers of subdomains, Algorithm 1 Step 5) against the CPU oracle: the choice
is forced through the tuning cache, and each variant must give the mixed form
within its bar (relative L2 of fluxes and pressures <= 1e-8) with the slab
sizes of each template of the register-resident Gauss-Jordan inverse (padded
slabs of 128, 256, 512 and 768 unknowns) and of the blocked and LU inverses."""
import json

import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

VARIANTS = ("gauss-jordan-registers", "gauss-jordan", "lu")


def _solve(case):
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300.solver import MRCM
    pm = case.params
    s = MRCM(case.problem, case.partition, space=pm.space, alpha_basis=pm.alpha_basis,
             alpha_smooth=pm.alpha_smooth, precision="mixed")
    s.run(pm.n_smooth)
    st = L.mrcm_stats(s.h)
    p, u = s.fluxes()
    s.close()
    return st, p, u


CASES = {
    # (grid, space): the largest slab is a layer of n_x / 16 subdomains
    "128x128_P1": ((128, 128), 1),     # slabs of at most 60 unknowns -> 128 template
    "384x128_P1": ((384, 128), 1),     # at most 188 -> 256 template
    "1024x64_P0": ((1024, 64), 0),     # at most 254 -> 256 template
    "1024x64_P1": ((1024, 64), 1),     # at most 508 -> 512 template (8-CTA clusters)
    "1536x64_P1": ((1536, 64), 1),     # at most 764 -> 768 template (16-CTA clusters)
}


@pytest.mark.parametrize("name", list(CASES))
def test_each_slab_inverse_matches_the_oracle(name, tmp_path, monkeypatch):
    n, space = CASES[name]
    prob = I.lognormal_problem(n, sigma2=2.0, corr_len=0.15, seed=7)
    case = I.Case(prob, I.Partition((16, 16), 4), I.MethodParams(space, 1.0, 1.0, 1), name=name)
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("MRCM_TUNE_CACHE", str(cache))
    ref = O.mrcm_os(prob, (16, 16), 4, space, 1.0, 1.0, 1)
    st, _, _ = _solve(case)
    assert st["slab_inverse_source"] == "measured", st
    assert st["tune_ms"]["gauss-jordan-registers"] > 0 and st["tune_ms"]["lu"] > 0, st
    (key, entry), = json.loads(cache.read_text()).items()
    npad = int(key.split("npad")[1].split()[0])
    tried = []
    for v in VARIANTS:
        if v == "gauss-jordan" and npad > 256:
            continue   # the blocked Gauss-Jordan inverse takes slabs of at most 256 unknowns
        cache.write_text(json.dumps({key: {"slab_inverse": v}}) + "\n")
        st, p, u = _solve(case)
        assert st["slab_inverse_source"] == "cache" and st["slab_inverse"] == v, (v, st)
        assert not st["interface_gmres"], (v, st)
        ep, eu = O.rel_errors(prob, p, u, ref.p, ref.u)
        assert ep <= 1e-8 and eu <= 1e-8, f"{name} {v}: rel L2 p {ep:.2e} u {eu:.2e}"
        assert np.max(np.abs(u - ref.u)) <= 1e-7 * np.max(np.abs(ref.u)), (name, v)
        tried.append((v, st["interface_ir_steps"]))
    assert len(tried) >= 2, tried
