"""mgt_ng_extrapolate_noalloc against the model's own Ng step (mgt_ng_accelerate).

The no-allocation entry point serves callers that cannot allocate device
memory: an application whose allocator owns the whole GPU, or an iteration
loop that must stay free of cudaMalloc/cudaFree because they can synchronise
the device.  It keeps its working memory in one static device array shared by
every call, so this test makes two calls in a row with different iterate
counts and checks each against the prediction mgt_ng_accelerate applied to the
model's populations and against the CPU oracle's Ng prediction from the same
iterates, within the FP64 tolerance of the parity tests.  A further call must
leave the device's free memory unchanged: it allocates nothing.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2411_03040_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def _ng_cycle(mgt, h, n_spec, n_steps):
    """n_steps regular iterations with classical Ng; returns the fractional
    iterates the model's history held (oldest first) and the populations after
    its prediction was applied."""
    hist = [mgt.mgt_get_populations(h) / n_spec[:, None]]
    for i in range(n_steps):
        mgt.mgt_formal_solve(h, mgt.MGT_FP64, want=False)
        mgt.mgt_stat_equilibrium(h, want=False)
        hist.append(mgt.mgt_get_populations(h) / n_spec[:, None])
        accepted, _ = mgt.mgt_ng_accelerate(h, mgt.MGT_NG_CLASSICAL, n_steps=n_steps)
        assert accepted == (i == n_steps - 1)
    return np.stack(hist), mgt.mgt_get_populations(h)


def test_noalloc_ng_matches_model_ng_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2411_03040_gb300 import build, mgt
    build.build()
    mgt.load()
    m = synth.sphere_model(400, n_levels=5, nside=1, n_quad=11, seed=11, name="noalloc")
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    # two Ng cycles of the model from LTE, far from convergence where the
    # predictions are well conditioned: 4 iterations (5 iterates), then 3
    # (4 iterates)
    hist1, pred1 = _ng_cycle(mgt, h, m.n_spec, 4)
    mgt.mgt_set_populations(h)
    hist2, pred2 = _ng_cycle(mgt, h, m.n_spec, 3)
    mgt.mgt_sync(h)

    X1 = torch.from_numpy(hist1.reshape(hist1.shape[0], -1)).cuda()
    X2 = torch.from_numpy(hist2.reshape(hist2.shape[0], -1)).cuda()
    out1 = torch.full((X1.shape[1],), float("nan"), dtype=torch.float64, device="cuda")
    out2 = torch.full((X2.shape[1],), float("nan"), dtype=torch.float64, device="cuda")
    c1, neg1 = mgt.mgt_ng_extrapolate_noalloc(X1, out1)
    c2, neg2 = mgt.mgt_ng_extrapolate_noalloc(X2, out2)
    torch.cuda.synchronize()

    import oracle as O
    for c, neg, out, pred, nres, hist in ((c1, neg1, out1, pred1, 4, hist1), (c2, neg2, out2, pred2, 3, hist2)):
        assert c.shape == (nres,)
        assert abs(c.sum() - 1.0) < 1e-12
        assert neg == 0
        frac = out.cpu().numpy()
        got = frac.reshape(pred.shape) * m.n_spec[:, None]
        assert np.all(np.isfinite(got))
        assert _rel(got, pred) < TOL64
        ref = O.ng_predict(hist.reshape(hist.shape[0], -1))
        np.testing.assert_allclose(c, O.ng_coefficients(hist.reshape(hist.shape[0], -1)), rtol=1e-8)
        assert _rel(frac, ref) < TOL64

    # a further call allocates no device memory (the free memory the driver
    # reports does not move), and still gives the same prediction
    out3 = torch.full_like(out1, float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    mgt.mgt_ng_extrapolate_noalloc(X1, out3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out3, out1)


def test_noalloc_ng_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2411_03040_gb300 import build, mgt
    build.build()
    mgt.load()
    n = 18      # one more than MGT_NG_NOALLOC_MAX_ITERATES
    X = torch.zeros((n, 64), dtype=torch.float64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_ng_extrapolate_noalloc(X, out)
    assert e.value.status == mgt.MGT_ERR_ARG
    assert "n_iterates" in str(e.value)
    # the C entry point itself refuses a prediction that overlaps the iterates
    import ctypes
    Y = torch.zeros((3, 64), dtype=torch.float64, device="cuda")
    st = mgt.load().mgt_ng_extrapolate_noalloc(3, ctypes.c_void_p(Y.data_ptr()), 64,
                                               ctypes.c_void_p(Y[1].data_ptr()), None, None, None)
    assert st == mgt.MGT_ERR_ARG
    assert "overlaps" in mgt.mgt_last_error()
