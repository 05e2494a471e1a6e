"""Batches of uneven models (mgt_batch_*) and the schedule autotuner, through the C-ABI.

A batched launch runs the same per-item code as the model's own staged
launch, so the batch's J-bar, Lambda* and populations are compared with the
single-model calls bit for bit (schedule 2, the model's lines per thread);
one small model of the batch is also compared with the oracle within the
FP32-mixed tolerance of the parity tests (1e-4 relative).
"""
import numpy as np
import pytest

import oracle as O
from paper_2411_03040_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def mgt():
    from paper_2411_03040_gb300 import build, mgt as binding
    build.build()
    binding.load()
    return binding


# (points, levels, HEALPix nside, bins, lines per thread): uneven sizes, every
# level count of the batched workload, both ray counts, both schedules of lines
SPECS = [(900, 41, 2, 31, 8), (400, 5, 1, 31, 4), (1500, 11, 1, 13, 8), (600, 21, 2, 31, 4),
         (250, 11, 2, 7, 4), (1200, 5, 2, 31, 8)]


def _models():
    return [synth.sphere_model(n, L, ns, q, seed=300 + i, name=f"b{i}") for i, (n, L, ns, q, _) in enumerate(SPECS)]


@pytest.fixture(scope="module")
def batch_models():
    return _models()


def _handle(mgt, m, lpt):
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, lines_per_thread=lpt, schedule=2)
    mgt.mgt_trace_rays(h)
    return h


def test_batch_formal_solve_and_se_match_single_model_calls(mgt, batch_models):
    hs = [_handle(mgt, m, s[4]) for m, s in zip(batch_models, SPECS)]
    singles = []
    for h in hs:
        J, L = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
        mgt.mgt_stat_equilibrium(h, want=False)
        singles.append((J, L, mgt.mgt_get_populations(h)))
        mgt.mgt_set_populations(h)                        # back to LTE
    b = mgt.mgt_batch_create(hs)
    lay = mgt.mgt_batch_get_layout(b)
    assert lay["n_models"] == len(hs)
    assert lay["graph_kernels"] == 0
    assert lay["fs_threads"] == 160                       # 31 bins x 5 groups of 8 lines, in warps
    # one launch per (CTA width, per-thread coefficients, lines per thread):
    # width 160 at 8 and at 4 lines per thread; width 32 with the shared
    # pre-pass at 8 and 4 (10 lines), with per-thread coefficients at 4 and 8
    # (the 4-line models)
    assert lay["fs_launches"] == 6
    # launch order: most work per item first
    assert sorted(lay["order"].tolist()) == list(range(len(hs)))
    mgt.mgt_batch_formal_solve(b)
    for h, (J, L, _) in zip(hs, singles):
        Jb, Lb = mgt.mgt_get_jbar(h)
        np.testing.assert_array_equal(Jb, J)
        np.testing.assert_array_equal(Lb, L)
    mgt.mgt_batch_stat_equilibrium(b)
    for h, (_, _, P) in zip(hs, singles):
        np.testing.assert_array_equal(mgt.mgt_get_populations(h), P)
    mgt.mgt_sync(hs[0])


def test_batch_jbar_matches_oracle(mgt, batch_models):
    # the 400-point 5-level model of the batch against the oracle
    hs = [_handle(mgt, m, s[4]) for m, s in zip(batch_models, SPECS)]
    b = mgt.mgt_batch_create(hs)
    mgt.mgt_batch_formal_solve(b)
    m = batch_models[1]
    Jb, Lb = mgt.mgt_get_jbar(hs[1])
    rays = O.trace(m)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    J, L = O.formal_solve(m, rays, chi, S)
    assert np.max(np.abs(Jb.T - J) / np.abs(J)) < TOL32
    assert np.max(np.abs(Lb.T - L) / np.abs(L)) < TOL32


@pytest.mark.parametrize("ng_mode", [0, 1], ids=["plain", "classical"])
def test_batch_iterate_graph_matches_ali_per_model(mgt, batch_models, ng_mode):
    n_iter = 6
    ref = []
    for m, s in zip(batch_models, SPECS):
        h = _handle(mgt, m, s[4])
        st = mgt.mgt_ali_solve(h, n_iter=n_iter, precision=mgt.MGT_FP32_MIXED, ng_mode=ng_mode, n_steps=3)
        ref.append((mgt.mgt_get_populations(h), st))
    hs = [_handle(mgt, m, s[4]) for m, s in zip(batch_models, SPECS)]
    b = mgt.mgt_batch_create(hs)
    n0 = mgt.mgt_launch_count()
    stats = mgt.mgt_batch_iterate(b, n_iter=n_iter, ng_mode=ng_mode, n_steps=3, want_stats=True)
    lay = mgt.mgt_batch_get_layout(b)
    # range-flag reset and line data; per CTA width the two-row formal solution
    # and its one-row fallback; SE
    assert lay["graph_kernels"] == 3 + 2 * lay["fs_launches"]
    assert mgt.mgt_launch_count() - n0 >= 3 * n_iter
    for h, (P, st), bs in zip(hs, ref, stats):
        np.testing.assert_array_equal(mgt.mgt_get_populations(h), P)
        assert bs["iterations"] == n_iter
        assert bs["ng_accepted"] == st["ng_accepted"]
        assert bs["last_maxrel"] == st["last_maxrel"]
    # a second call replays the same graph
    mgt.mgt_batch_iterate(b, n_iter=1)
    assert mgt.mgt_batch_get_layout(b)["graph_kernels"] == 3 + 2 * lay["fs_launches"]


def test_large_model_runs_its_single_model_launch_inside_the_batch(mgt):
    # a 40k-point 4-line model is more than 8 waves of its persistent class
    # (one-warp CTAs, 16 per SM): the batch launches it through the
    # single-model kernel, also inside the captured iteration; the small model
    # stays in a persistent launch.  Both give the single-model values.
    models = [synth.sphere_model(40_000, 5, 1, 31, seed=401, name="big"),
              synth.sphere_model(600, 21, 1, 31, seed=402, name="small")]
    ref = []
    for m in models:
        h = _handle(mgt, m, 4)
        mgt.mgt_set_solve_opts(h, lines_per_thread=4, schedule=0)
        J, L = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
        st = mgt.mgt_ali_solve(h, n_iter=3, precision=mgt.MGT_FP32_MIXED, ng_mode=0)
        ref.append((J, L, mgt.mgt_get_populations(h)))
    hs = []
    for m in models:
        h = _handle(mgt, m, 4)
        mgt.mgt_set_solve_opts(h, lines_per_thread=4, schedule=0)
        hs.append(h)
    b = mgt.mgt_batch_create(hs)
    lay = mgt.mgt_batch_get_layout(b)
    assert lay["fs_solo"] == 1 and lay["fs_launches"] == 2
    assert lay["order"].tolist() == [1, 0]              # the model launched on its own last
    mgt.mgt_batch_formal_solve(b)
    for h, (J, L, _) in zip(hs, ref):
        Jb, Lb = mgt.mgt_get_jbar(h)
        np.testing.assert_array_equal(Jb, J)
        np.testing.assert_array_equal(Lb, L)
    for h in hs:
        mgt.mgt_set_populations(h)                        # back to LTE
    mgt.mgt_batch_iterate(b, n_iter=3)
    assert mgt.mgt_batch_get_layout(b)["graph_kernels"] == 3 + 2 * 2
    for h, (_, _, P) in zip(hs, ref):
        np.testing.assert_array_equal(mgt.mgt_get_populations(h), P)


def test_extreme_bin_counts_in_one_batch(mgt):
    # 1, 2 and 64 bins in one batch: at 64 bins 40 lines take 2 (8 lines per
    # thread) or 3 (4 per thread) line blocks per origin, each a batch item of
    # a 256-thread class; J-bar, Lambda* and SE populations bit-identical to
    # the models' own calls, and the 64-bin 40-line model within the FP32
    # tolerance of the oracle
    specs = [(300, 41, 1, 64, 8), (300, 41, 1, 64, 4), (300, 5, 1, 1, 4), (300, 11, 1, 2, 8), (300, 5, 1, 64, 4)]
    models = [synth.sphere_model(n, L, ns, q, seed=500 + i, name=f"x{i}") for i, (n, L, ns, q, _) in enumerate(specs)]
    hs = [_handle(mgt, m, s[4]) for m, s in zip(models, specs)]
    singles = []
    for h in hs:
        J, L = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
        mgt.mgt_stat_equilibrium(h, want=False)
        singles.append((J, L, mgt.mgt_get_populations(h)))
        mgt.mgt_set_populations(h)                        # back to LTE
    b = mgt.mgt_batch_create(hs)
    mgt.mgt_batch_formal_solve(b)
    for h, (J, L, _) in zip(hs, singles):
        Jb, Lb = mgt.mgt_get_jbar(h)
        np.testing.assert_array_equal(Jb, J)
        np.testing.assert_array_equal(Lb, L)
    mgt.mgt_batch_stat_equilibrium(b)
    for h, (_, _, P) in zip(hs, singles):
        np.testing.assert_array_equal(mgt.mgt_get_populations(h), P)
    m = models[0]
    rays = O.trace(m)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    J, L = O.formal_solve(m, rays, chi, S)
    assert np.max(np.abs(singles[0][0].T - J) / np.abs(J)) < TOL32
    assert np.max(np.abs(singles[0][1].T - L) / np.abs(L)) < TOL32


def test_batch_follows_model_changes(mgt, batch_models):
    hs = [_handle(mgt, m, s[4]) for m, s in zip(batch_models[:3], SPECS[:3])]
    b = mgt.mgt_batch_create(hs)
    mgt.mgt_batch_iterate(b, n_iter=1)
    # change one model's lines per thread and another's populations between calls
    mgt.mgt_set_solve_opts(hs[0], lines_per_thread=4, schedule=2)
    rng = np.random.default_rng(4)
    P = mgt.mgt_get_populations(hs[2]) * rng.uniform(0.5, 1.5, size=(batch_models[2].n_points, 11))
    mgt.mgt_set_populations(hs[2], P)
    mgt.mgt_batch_formal_solve(b)
    got = [mgt.mgt_get_jbar(h) for h in hs]
    for h, (Jb, Lb) in zip(hs, got):
        Js, Ls = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
        np.testing.assert_array_equal(Jb, Js)
        np.testing.assert_array_equal(Lb, Ls)


def test_batch_rejects_bad_inputs(mgt, batch_models):
    m = batch_models[1]
    h = _handle(mgt, m, 4)
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_batch_create([h, h])
    assert e.value.status == mgt.MGT_ERR_ARG
    u = mgt.mgt_model_create(m)                            # not traced
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_batch_create([h, u])
    assert e.value.status == mgt.MGT_ERR_STATE
    pb = mgt.mgt_model_create(batch_models[0])
    mgt.mgt_set_solve_opts(pb, pairs_per_batch=2)
    mgt.mgt_trace_rays(pb)
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_batch_create([h, pb])
    assert e.value.status == mgt.MGT_ERR_ARG
    b = mgt.mgt_batch_create([h])
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_batch_stat_equilibrium(mgt.mgt_batch_create([_handle(mgt, batch_models[4], 4)]))
    assert e.value.status == mgt.MGT_ERR_STATE
    del b


def test_staged_schedule_on_small_blocks_matches_oracle(mgt):
    # 5 lines x 9 bins: one warp per origin in the staged kernel (as the
    # batched launch runs small models); schedule 4 (per-thread coefficients)
    # with the 5 lines in one group of 8
    m = synth.sphere_model(700, n_levels=6, nside=1, n_quad=9, seed=77, name="ragged")
    rays = O.trace(m)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    J, L = O.formal_solve(m, rays, chi, S)
    for sched in (2, 3, 4):
        for lpt in (4, 8):
            if sched == 4 and lpt == 4:
                continue                                  # 5 lines: two groups of 4
            h = mgt.mgt_model_create(m)
            mgt.mgt_set_solve_opts(h, lines_per_thread=lpt, schedule=sched)
            mgt.mgt_trace_rays(h)
            Jg, Lg = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
            assert np.max(np.abs(Jg.T - J) / np.abs(J)) < TOL32
            assert np.max(np.abs(Lg.T - L) / np.abs(L)) < TOL32
            if sched == 4:
                # FP64 runs 4 lines per thread: the 5 lines need two groups
                with pytest.raises(mgt.MgtError):
                    mgt.mgt_formal_solve(h, mgt.MGT_FP64)
                continue
            Jg, Lg = mgt.mgt_formal_solve(h, mgt.MGT_FP64)
            assert np.max(np.abs(Jg.T - J) / np.abs(J)) < 1e-10


def test_autotune_picks_a_timed_candidate(mgt, batch_models):
    m = batch_models[0]
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    r = mgt.mgt_autotune(h, mgt.MGT_FP32_MIXED, reps=2)
    assert len(r["tried"]) == 6
    assert {(s, l) for s, l, _ in r["tried"]} == {(s, l) for s in (1, 2, 3) for l in (4, 8)}
    best = min(r["tried"], key=lambda t: t[2])
    assert (r["schedule"], r["lines_per_thread"]) == best[:2]
    assert all(t[2] > 0 for t in r["tried"])
    # the chosen options stay set: a formal solution now equals one with them set by hand
    Ja, La = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
    h2 = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h2, schedule=r["schedule"], lines_per_thread=r["lines_per_thread"])
    mgt.mgt_trace_rays(h2)
    Jb, Lb = mgt.mgt_formal_solve(h2, mgt.MGT_FP32_MIXED)
    np.testing.assert_array_equal(Ja, Jb)
    r64 = mgt.mgt_autotune(h, mgt.MGT_FP64, staged_only=True, reps=1)
    assert [(s, l) for s, l, _ in r64["tried"]] == [(0, 4)]
