"""The oracle still reproduces its stored regression fixtures (tests/golden)."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("name", ["oracle_2d_p2_K4", "oracle_3d_p2_K3_curved"])
def test_golden(oracle_mod, name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    elems, Km, Mm = mg.compute(name)
    stored = np.loadtxt(os.path.join(HERE, "golden", name + ".txt"))
    N = Km.shape[1]
    stored = stored.reshape(len(elems), 2, N, N)
    np.testing.assert_array_equal(stored[:, 0], Km)
    np.testing.assert_array_equal(stored[:, 1], Mm)
