"""The bounds-check build (libmrcm_check.so, -DMRCM_CHECK=1): every kernel
check compiled in -- shared-memory layouts against the launch's dynamic shared
memory, the bulk copy of the smoothing pack, the slab inverses' pivot records
and inverse writes, the state and slab-block write indices -- on workloads that
reach every checked kernel (2D basis, interface with each slab-inverse variant,
smoothing and assembly; 3D basis and smoothing), run in a child process with
MRCM_CHECK=1.  No check may fire, and the results agree with the production
library's to 1e-12 relative (the checks only guard accesses; both runs take
the slab-inverse choice from one tuning cache)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2404_13811_gb300 import inputs as I
from paper_2404_13811_gb300.solver import MRCM
out = {}
c2 = I.config_channel2d(n=128, n_smooth=2)
for prec in ("mixed", "fp64"):
    s = MRCM(c2.problem, c2.partition, space=1, precision=prec)
    s.run(2)
    p, u = s.fluxes()
    out["2d_" + prec] = [float(np.sum(p)), float(np.sum(np.abs(u)))]
    s.close()
c3 = I.config_layered3d(n=(20, 20, 10), n_upper=4)
s = MRCM(c3.problem, c3.partition, space=0, precision="mixed")
s.run(1)
p, u = s.fluxes()
out["3d_mixed"] = [float(np.sum(p)), float(np.sum(np.abs(u)))]
s.close()
print(json.dumps(out))
"""


def _child(check, cache):
    env = dict(os.environ)
    env["MRCM_CHECK"] = "1" if check else "0"
    env["MRCM_TUNE_CACHE"] = str(cache)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_check_build_runs_clean_and_matches(tmp_path):
    from paper_2404_13811_gb300 import build as B
    B.build(check=True)
    cache = tmp_path / "tune.json"
    checked = _child(True, cache)
    plain = _child(False, cache)
    assert checked.keys() == plain.keys()
    for k in plain:
        assert np.allclose(checked[k], plain[k], rtol=1e-12, atol=0), (k, checked[k], plain[k])
