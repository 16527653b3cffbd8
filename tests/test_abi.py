"""The C ABI library builds, loads and exports every entry point include/mrcm.h declares;
argument validation runs on the host, so bad inputs are rejected without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(mrcm_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_13811_gb300 import build
    build.build()
    from paper_2404_13811_gb300 import _lib as L
    return L.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "mrcm_create" in names and "mrcm_smooth" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2404_13811_gb300 import _lib as L
    assert sorted(L.EXPORTS) == _declared()


def test_bad_inputs_rejected_on_host(lib):
    from paper_2404_13811_gb300 import _lib as L
    K = np.ones(16 * 16)
    f = np.zeros(16 * 16)
    prm = L.make_params(1, 1.0, 1.0, L.MRCM_FP64)
    cases = [
        ((4, (16, 16), (1, 1), (0,) * 6, (0.0,) * 6, (8, 8), 1), "dim"),
        ((2, (16, 16), (1, 1), (0,) * 6, (0.0,) * 6, (5, 8), 1), "divide"),
        ((2, (16, 16), (1, 1), (0,) * 6, (0.0,) * 6, (8, 8), 4), "overlap"),
        ((2, (16, 16), (1, -1), (0,) * 6, (0.0,) * 6, (8, 8), 1), "positive"),
        ((2, (16, 16), (1, 1), (7, 0, 0, 0, 0, 0), (0.0,) * 6, (8, 8), 1), "kind"),
    ]
    for args, word in cases:
        dim = args[0]
        g = L.mrcm_grid()
        g.dim = dim
        for a in range(2):
            g.n[a] = args[1][a]
            g.h[a] = args[2][a]
        b = L.mrcm_bc()
        for s in range(6):
            b.kind[s] = args[3][s]
        p = L.mrcm_partition()
        p.sub[0], p.sub[1] = args[5]
        p.overlap = args[6]
        with pytest.raises(L.MrcmError) as e:
            L.mrcm_create(g, K.ctypes.data, f.ctypes.data, b, p, prm, 0, 0)
        assert e.value.code == -1, (word, e.value)
    # negative permeability
    g, b, p = L.make_structs(2, (16, 16), (1, 1), (0,) * 4, (0.0,) * 4, (8, 8), 1)
    Kbad = K.copy()
    Kbad[5] = -1.0
    with pytest.raises(L.MrcmError) as e:
        L.mrcm_create(g, Kbad.ctypes.data, f.ctypes.data, b, p, prm, 0, 0)
    assert e.value.code == -1


def test_particular_option_checked_on_host(lib):
    """mrcm_params.particular: 0 (Step 4 on Omega_i) or 1 (the hat-Omega_i
    variant); other values are rejected before any device work."""
    from paper_2404_13811_gb300 import _lib as L
    K = np.ones(16 * 16)
    f = np.zeros(16 * 16)
    g, b, p = L.make_structs(2, (16, 16), (1, 1), (0,) * 4, (0.0,) * 4, (8, 8), 1)
    with pytest.raises(L.MrcmError) as e:
        L.mrcm_create(g, K.ctypes.data, f.ctypes.data, b, p, L.make_params(1, 1.0, 1.0, L.MRCM_FP64, particular=2), 0, 0)
    assert e.value.code == -1
