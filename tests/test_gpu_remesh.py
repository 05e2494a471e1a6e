"""Recursive re-meshing (Sec. 4.1) on the GPU against the oracle, through the C-ABI.

Box bounds and centres are exact in FP64, so the output point sets are equal
bit for bit (the GPU writes the boxes level by level, the oracle depth first:
the sets are compared after sorting).
"""
import numpy as np
import pytest

import oracle as O
from paper_2411_03040_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgt():
    from paper_2411_03040_gb300 import build, mgt as binding
    build.build()
    binding.load()
    return binding


def _sorted(a):
    return a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("case,r_max,lmax,n_side", [
    ("sphere", 0.4, 12, 6), ("shell", 0.2, 8, 4), ("constant", 0.4, 12, 3), ("step", 0.5, 6, 2), ("depth0", 0.1, 0, 3)])
def test_remesh_matches_oracle(mgt, case, r_max, lmax, n_side):
    if case == "sphere":
        m = synth.config_model(1, n_points=3000)
        pos, rho = m.pos, m.n_coll
    elif case == "shell":
        m = synth.shell_model(20000, 2, 1, 3, seed=4, name="shell-20k")
        pos, rho = m.pos, m.n_coll
    else:
        rng = np.random.default_rng(9)
        pos = rng.uniform(-1, 1, size=(5000, 3))
        rho = np.full(5000, 3.0) if case != "step" else np.where(pos[:, 0] < 0.05, 1.0, 10.0)
        if case == "depth0":
            rho = rng.uniform(1, 2, 5000)
    out, flags = mgt.mgt_remesh(pos, rho, r_max, lmax, n_side)
    ref, rflags, leaves = O.remesh(pos, rho, r_max, lmax, n_side)
    assert out.shape == ref.shape and flags.sum() == rflags.sum()
    assert np.array_equal(_sorted(out[flags == 0]), _sorted(ref[rflags == 0]))
    assert np.array_equal(out[flags == 1], ref[rflags == 1])


def test_remesh_rejects_bad_input(mgt):
    pos = np.zeros((4, 3))
    with pytest.raises(mgt.MgtError):
        mgt.mgt_remesh(pos, np.array([1.0, 2.0, -1.0, 1.0]), 0.4, 5, 3)
    with pytest.raises(mgt.MgtError):
        mgt.mgt_remesh(pos, np.ones(4), 0.4, 5, 1)
