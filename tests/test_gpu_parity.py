"""CUDA path vs the CPU oracle, element by element, through the C-ABI.

Tolerances (relative, max over elements): ray point lists bit-exact; J-bar
and Lambda* 1e-10 on the FP64 path and 1e-4 on the FP32-mixed path;
statistical-equilibrium populations fed by either path's own J-bar 1e-8
(FP64); converged ALI populations 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2411_03040_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def mgt():
    from paper_2411_03040_gb300 import build, mgt as binding
    build.build()
    binding.load()
    return binding


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape
    return float(np.max(np.abs(a - b) / np.abs(b)))


def oracle_fields(model, rays, origins=None):
    pops = O.lte_populations(model.temp, model.n_spec, model.lines.energy_J, model.lines.g)
    chi, S, _ = O.line_chi_S(pops, model.lines)
    return O.formal_solve(model, rays, chi, S, origins=origins)


def gpu_fields(mgt, h, precision):
    J, L = mgt.mgt_formal_solve(h, precision)
    return J.T, L.T            # -> [N][M], the oracle's layout


# ------------------------------------------------------------------- tracing
def _models_for_trace():
    out = [synth.config_model(1), synth.lattice_model(n_side=7),
           synth.shell_model(4000, 3, 2, 5, seed=7, name="shell-4k"),
           synth.shell_model(3000, 3, 2, 5, grf_sigma=5e3, seed=8, name="grf-3k")]
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "trace_tiny.json")))
    for case in g["cases"]:
        pos = np.asarray(case["pos"], np.float64)
        off = np.zeros(len(case["nbrs"]) + 1, np.int64)
        for i, v in enumerate(case["nbrs"]):
            off[i + 1] = off[i] + len(v)
        nb = np.concatenate([np.asarray(v, np.int32) for v in case["nbrs"]])
        n = len(pos)
        out.append(synth.Model(case["name"], pos, np.zeros_like(pos), np.full(n, 50.0), np.zeros(n),
                               np.ones(n), np.ones(n), off, nb, np.asarray(case["boundary"], np.int32),
                               np.asarray(case["dirs"], np.float64), 3,
                               synth.linear_rotor(2, np.random.default_rng(0))))
    return out


@pytest.mark.parametrize("model", _models_for_trace(), ids=lambda m: m.name)
def test_trace_bit_exact(mgt, model):
    h = mgt.mgt_model_create(model)
    st = mgt.mgt_trace_rays(h)
    off, idx = mgt.mgt_get_rays(h)
    ref = O.trace(model)
    np.testing.assert_array_equal(off, ref.off)
    np.testing.assert_array_equal(idx, ref.idx)
    assert st["n_stalls"] == ref.stalls
    assert st["total_steps"] == ref.off[-1]


# --------------------------------------------------------- formal solution
@pytest.fixture(scope="module")
def sphere(mgt):
    m = synth.config_model(1)
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    rays = O.trace(m)
    J, L = oracle_fields(m, rays)
    return m, h, rays, J, L


def test_sphere_fp64_all_points(mgt, sphere):
    m, h, rays, J, L = sphere
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP64)
    assert rel_err(Jg, J) < TOL64
    assert rel_err(Lg, L) < TOL64


def test_sphere_fp32_all_points(mgt, sphere):
    m, h, rays, J, L = sphere
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert rel_err(Jg, J) < TOL32
    assert rel_err(Lg, L) < TOL32


def test_fp32_is_deterministic(mgt, sphere):
    m, h, *_ = sphere
    a = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    b = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_device_outputs_match_host_outputs(mgt, sphere):
    torch = pytest.importorskip("torch")
    m, h, *_ = sphere
    Jh, Lh = mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
    Jd = torch.empty(Jh.shape, dtype=torch.float64, device="cuda")
    Ld = torch.empty(Lh.shape, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED, Jd, Ld, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(Jd.cpu().numpy(), Jh)
    np.testing.assert_array_equal(Ld.cpu().numpy(), Lh)


@pytest.mark.parametrize("lpt", [4, 8])
def test_ragged_line_count_both_schedules(mgt, lpt):
    # 6 levels -> 5 lines: one full group of 4 plus a ragged one, or one
    # group of 8 with three padding lines
    m = synth.sphere_model(700, n_levels=6, nside=1, n_quad=9, seed=77, name="ragged")
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, lines_per_thread=lpt)
    mgt.mgt_trace_rays(h)
    rays = O.trace(m)
    J, L = oracle_fields(m, rays)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert rel_err(Jg, J) < TOL32 and rel_err(Lg, L) < TOL32
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP64)
    assert rel_err(Jg, J) < TOL64 and rel_err(Lg, L) < TOL64


@pytest.mark.parametrize("schedule", [0, 1], ids=["staged", "gather"])
@pytest.mark.parametrize("grf", [0.0, 5e3], ids=["shell", "shell-grf"])
def test_shell_41_levels_sampled(mgt, grf, schedule):
    # the 41-level rotor with 50 (or 40) bins on a small shell outflow, through
    # the bulk-copy staged kernel and the gather kernel; with the random
    # velocity field most segments take the erf branch
    q = 50 if grf == 0.0 else 40
    m = synth.shell_model(5000, 41, 2, q, grf_sigma=grf, seed=9 if grf == 0 else 10,
                          name="shell-5k")
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, schedule=schedule)
    mgt.mgt_trace_rays(h)
    rays = O.trace(m)
    rng = np.random.default_rng(1)
    orig = np.sort(np.concatenate([rng.choice(m.n_points, 30, replace=False), m.boundary[:4]]))
    J, L = oracle_fields(m, rays, orig)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP64)
    assert rel_err(Jg[orig], J) < TOL64
    assert rel_err(Lg[orig], L) < TOL64
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert rel_err(Jg[orig], J) < TOL32
    assert rel_err(Lg[orig], L) < TOL32


@pytest.mark.parametrize("lpt", [4, 8])
def test_items_outside_the_two_row_range_are_redone_exactly(mgt, lpt):
    # points in the inner half of the sphere get a species density 1e12 times
    # higher: their segments reach optical depths of ~1e12, far outside the
    # range of the two-row elimination (whose state would overflow FP32 there);
    # those items are redone with the one-row form, the others keep the
    # two-row form, and every point must still match the oracle
    m = synth.config_model(1, n_points=800)
    r = np.linalg.norm(m.pos, axis=1)
    m.n_spec = np.where(r < 0.5 * r.max(), m.n_spec * 1e12, m.n_spec)
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, lines_per_thread=lpt)
    mgt.mgt_trace_rays(h)
    rays = O.trace(m)
    J, L = oracle_fields(m, rays)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert np.all(np.isfinite(Jg)) and np.all(np.isfinite(Lg))
    assert rel_err(Jg, J) < TOL32 and rel_err(Lg, L) < TOL32
    J64, L64 = gpu_fields(mgt, h, mgt.MGT_FP64)
    assert rel_err(J64, J) < TOL64 and rel_err(L64, L) < TOL64


@pytest.mark.parametrize("lpt", [4, 8])
@pytest.mark.parametrize("thick", [False, True], ids=["two-row", "one-row"])
def test_per_thread_coefficients_bit_identical_to_shared_prepass(mgt, lpt, thick):
    # schedule 4 (each thread computes its own bin's segment coefficients)
    # against schedule 2 (the CTA computes them once per bin in shared memory):
    # one function computes every coefficient, so J-bar and Lambda* agree bit
    # for bit in both precisions, with the two-row elimination and with the
    # one-row fallback (inner points optically thick, as in the test above)
    m = synth.config_model(1, n_points=800)
    if thick:
        r = np.linalg.norm(m.pos, axis=1)
        m.n_spec = np.where(r < 0.5 * r.max(), m.n_spec * 1e12, m.n_spec)
    out = {}
    for sched in (2, 4):
        h = mgt.mgt_model_create(m)
        mgt.mgt_set_solve_opts(h, lines_per_thread=lpt, schedule=sched)
        mgt.mgt_trace_rays(h)
        out[sched] = [mgt.mgt_formal_solve(h, p) for p in (mgt.MGT_FP32_MIXED, mgt.MGT_FP64)]
    for (J2, L2), (J4, L4) in zip(out[2], out[4]):
        assert np.all(np.isfinite(J2)) and np.all(np.isfinite(L2))
        np.testing.assert_array_equal(J4, J2)
        np.testing.assert_array_equal(L4, L2)


def test_per_thread_coefficients_need_one_line_group(mgt):
    # 10 lines do not fit one group of 4 or 8 lines per thread
    m = synth.sphere_model(300, n_levels=11, nside=1, n_quad=7, seed=5, name="ten-lines")
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, lines_per_thread=8, schedule=4)
    mgt.mgt_trace_rays(h)
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED)
    assert e.value.status == mgt.MGT_ERR_ARG and "one group" in str(e.value)


@pytest.mark.parametrize("q,levels,lpt", [(1, 5, 4), (2, 11, 8), (64, 41, 8), (64, 41, 4), (64, 5, 4)],
                         ids=["1bin-4lines", "2bins-10lines", "64bins-40lines-lpt8", "64bins-40lines-lpt4",
                              "64bins-4lines"])
def test_extreme_bin_counts_and_line_blocks(mgt, q, levels, lpt):
    # the smallest and largest bin counts the model accepts: with 1 bin every
    # pre-pass pair spans two steps, with 2 bins every pair is one step; 64
    # bins leave room for 4 line groups per CTA, so 40 lines take 2 (8 per
    # thread) or 3 (4 per thread) line blocks per origin, the last one partly
    # empty.  Every schedule that applies (gather, staged, and per-thread
    # coefficients where the lines fit one group), both precisions, all points.
    m = synth.sphere_model(500, n_levels=levels, nside=1, n_quad=q, seed=31, name=f"bins{q}")
    rays = O.trace(m)
    J, L = oracle_fields(m, rays)
    schedules = [1, 2] + ([4] if m.lines.n_lines <= lpt else [])
    for sched in schedules:
        h = mgt.mgt_model_create(m)
        mgt.mgt_set_solve_opts(h, lines_per_thread=lpt, schedule=sched)
        mgt.mgt_trace_rays(h)
        Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
        assert rel_err(Jg, J) < TOL32 and rel_err(Lg, L) < TOL32, sched
        Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP64)
        assert rel_err(Jg, J) < TOL64 and rel_err(Lg, L) < TOL64, sched
        h.close()


def test_single_point_model_is_background(mgt):
    # no neighbours: every half-ray is empty, u = I_bg, Lambda* = 0
    lines = synth.linear_rotor(3, np.random.default_rng(0))
    m = synth.Model("single", np.zeros((1, 3)), np.zeros((1, 3)), np.array([40.0]), np.array([1e6]),
                    np.array([1e9]), np.array([1e3]), np.zeros(2, np.int64), np.zeros(0, np.int32),
                    np.array([0], np.int32), synth.healpix_directions(1), 7, lines)
    h = mgt.mgt_model_create(m)
    st = mgt.mgt_trace_rays(h)
    assert st["total_steps"] == 0
    x, w = O.gauss_hermite(7)
    for prec in (mgt.MGT_FP64, mgt.MGT_FP32_MIXED):
        Jg, Lg = gpu_fields(mgt, h, prec)
        for k in range(lines.n_lines):
            dnu = O.line_width(lines.freq_Hz[k], 40.0, 1e6, lines.mol_mass_kg)
            exact = np.sum(w * O.planck(lines.freq_Hz[k] + x * dnu, m.T_bg))
            assert abs(Jg[0, k] / exact - 1) < (TOL64 if prec == mgt.MGT_FP64 else TOL32)
        assert np.all(Lg == 0.0)


# ----------------------------------------------------- statistical equilibrium
def test_stat_equilibrium_parity(mgt, sphere):
    m, h, rays, J, L = sphere
    mgt.mgt_set_populations(h, None)
    mgt.mgt_formal_solve(h, mgt.MGT_FP64, want=False)
    pg = mgt.mgt_stat_equilibrium(h)
    p0 = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    po = O.stat_equilibrium(p0, J, L, m.temp, m.n_coll, m.n_spec, m.lines)
    assert rel_err(pg, po) < 1e-8
    np.testing.assert_allclose(pg.sum(1), m.n_spec, rtol=1e-13)


@pytest.mark.parametrize("lpt", [4, 8])
def test_two_level_model(mgt, lpt):
    # the smallest molecule: two levels, one line (one group of lines padded
    # to 4 or 8): J-bar and Lambda* in both precisions and the SE populations
    # from the FP64 J-bar against the oracle
    m = synth.sphere_model(600, n_levels=2, nside=1, n_quad=15, seed=41, name="two-level")
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, lines_per_thread=lpt)
    mgt.mgt_trace_rays(h)
    rays = O.trace(m)
    J, L = oracle_fields(m, rays)
    assert J.shape == (m.n_points, 1)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert rel_err(Jg, J) < TOL32 and rel_err(Lg, L) < TOL32
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP64)
    assert rel_err(Jg, J) < TOL64 and rel_err(Lg, L) < TOL64
    pg = mgt.mgt_stat_equilibrium(h)
    p0 = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    po = O.stat_equilibrium(p0, J, L, m.temp, m.n_coll, m.n_spec, m.lines)
    assert rel_err(pg, po) < 1e-8
    np.testing.assert_allclose(pg.sum(1), m.n_spec, rtol=1e-13)


def test_stat_equilibrium_tiny_populations_41_levels(mgt):
    # cold gas: upper levels ~1e-60 of the ground level keep full relative accuracy
    m = synth.shell_model(1500, 41, 1, 7, seed=12, name="cold")
    m.temp = np.full(m.n_points, 25.0)
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    mgt.mgt_formal_solve(h, mgt.MGT_FP64, want=False)
    pg = mgt.mgt_stat_equilibrium(h)
    rays = O.trace(m)
    J, L = oracle_fields(m, rays)
    p0 = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    po = O.stat_equilibrium(p0, J, L, m.temp, m.n_coll, m.n_spec, m.lines)
    assert (po / m.n_spec[:, None]).min() < 1e-50
    assert rel_err(pg, po) < 1e-8


# ------------------------------------------------------------------- ALI + Ng
def nonlte_sphere():
    # 400-point sphere with the collider density lowered 1e4 times: non-LTE,
    # plain ALI converges linearly (about x0.7 per iteration), so Ng matters
    m = synth.config_model(1, n_points=400)
    m.n_coll = m.n_coll * 1e-4
    m.name = "sphere-400-nonlte"
    return m


@pytest.fixture(scope="module")
def ali_ref():
    m = nonlte_sphere()
    rays = O.trace(m)
    ref, ch = O.ali_solve(m, rays, n_iter=90)
    assert ch[-1] < 1e-13
    return m, rays, ref


@pytest.mark.parametrize("mode,prec", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)],
                         ids=["plain64", "classical64", "adaptive64", "classical32", "adaptive32"])
def test_ali_converges_to_oracle_fixed_point(mgt, ali_ref, mode, prec):
    m, rays, ref = ali_ref
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    n_iter = 60 if mode == 0 else 20
    st = mgt.mgt_ali_solve(h, n_iter=n_iter, precision=prec, ng_mode=mode, n_steps=4, n_max=8)
    assert st["iterations"] == n_iter
    if mode != 0:
        assert st["ng_accepted"] >= 1
    pg = mgt.mgt_get_populations(h)
    assert rel_err(pg, ref) < 1e-5


@pytest.mark.parametrize("mode", ["classical", "adaptive"])
def test_ng_step_by_step_matches_oracle_controller(mgt, ali_ref, mode):
    # the same ALI sequence on both sides: the accept pattern, the maximum
    # relative change and the populations after every step agree
    m, rays, _ = ali_ref
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    ng = O.NgClassical(4) if mode == "classical" else O.NgAdaptive(6)
    ng.reset((pops / m.n_spec[:, None]).ravel())
    gmode = mgt.MGT_NG_CLASSICAL if mode == "classical" else mgt.MGT_NG_ADAPTIVE
    accepted = 0
    for it in range(12):
        chi, S, _ = O.line_chi_S(pops, m.lines)
        J, L = O.formal_solve(m, rays, chi, S)
        new = O.stat_equilibrium(pops, J, L, m.temp, m.n_coll, m.n_spec, m.lines)
        mr = O.maxrel(new, pops)
        x, acc = ng.push((new / m.n_spec[:, None]).ravel())
        if acc:
            new = x.reshape(pops.shape) * m.n_spec[:, None]
        pops = new
        accepted += acc
        mgt.mgt_formal_solve(h, mgt.MGT_FP64, want=False)
        mgt.mgt_stat_equilibrium(h, want=False)
        acc_g, mr_g = mgt.mgt_ng_accelerate(h, gmode, n_steps=4, n_max=6)
        assert acc_g == acc, it
        assert abs(mr_g / mr - 1) < 1e-6
        assert rel_err(mgt.mgt_get_populations(h), pops) < 1e-8
    assert accepted >= 1


@pytest.mark.parametrize("scale,faster", [(1e-4, True), (1e-2, False)], ids=["low-density", "mid-density"])
def test_ng_reaches_the_plain_fixed_point_in_fewer_iterations(mgt, scale, faster):
    # Sec. 4.2's Ng experiment on the synthetic stand-in: the sphere with the
    # collider density lowered 1e4 times (strongly non-LTE, slow plain ALI)
    # and 1e2 times (plain ALI converges in a few iterations).  Plain ALI,
    # classical and adaptive Ng (FP64) iterate until the regular iterate
    # changes by less than 1e-9; all three land on the same populations; Ng
    # needs fewer iterations where plain ALI is slow and never more.
    m = synth.config_model(1, n_points=400)
    m.n_coll = m.n_coll * scale
    result = {}
    for mode in (mgt.MGT_NG_NONE, mgt.MGT_NG_CLASSICAL, mgt.MGT_NG_ADAPTIVE):
        h = mgt.mgt_model_create(m)
        mgt.mgt_trace_rays(h)
        it = 0
        while True:
            it += 1
            st = mgt.mgt_ali_solve(h, n_iter=1, precision=mgt.MGT_FP64, ng_mode=mode, n_steps=4, n_max=8)
            if st["last_maxrel"] < 1e-9 or it >= 400:
                break
        assert it < 400, (mode, it)
        result[mode] = (it, mgt.mgt_get_populations(h))
    it_plain, p_plain = result[mgt.MGT_NG_NONE]
    for mode in (mgt.MGT_NG_CLASSICAL, mgt.MGT_NG_ADAPTIVE):
        it_ng, p_ng = result[mode]
        assert rel_err(p_ng, p_plain) < 1e-7, mode
        assert it_ng < it_plain if faster else it_ng <= it_plain, (mode, it_ng, it_plain)


def test_ali_resumes_from_saved_populations(mgt):
    # checkpoint and resume: three plain ALI iterations, the populations saved
    # to the host, restored into a fresh model of the same inputs, three more
    # iterations; the result is bit-identical to six uninterrupted iterations
    m = nonlte_sphere()
    for prec in (mgt.MGT_FP64, mgt.MGT_FP32_MIXED):
        h = mgt.mgt_model_create(m)
        mgt.mgt_trace_rays(h)
        mgt.mgt_ali_solve(h, n_iter=6, precision=prec)
        straight = mgt.mgt_get_populations(h)
        a = mgt.mgt_model_create(m)
        mgt.mgt_trace_rays(a)
        mgt.mgt_ali_solve(a, n_iter=3, precision=prec)
        saved = mgt.mgt_get_populations(a)
        a.close()
        b = mgt.mgt_model_create(m)
        mgt.mgt_trace_rays(b)
        mgt.mgt_set_populations(b, saved)
        mgt.mgt_ali_solve(b, n_iter=3, precision=prec)
        np.testing.assert_array_equal(mgt.mgt_get_populations(b), straight)


# ------------------------------------------------ full size, sampled outputs
@pytest.mark.slow
def test_full_size_shell_100k_sampled(mgt):
    # the benchmark workload in its launch configuration; the oracle computes
    # sampled origins one by one
    m = synth.config_model(2)
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    rays = O.trace(m)
    off, idx = mgt.mgt_get_rays(h)
    np.testing.assert_array_equal(off, rays.off)
    np.testing.assert_array_equal(idx, rays.idx)
    rng = np.random.default_rng(2)
    orig = np.sort(rng.choice(m.n_points, 24, replace=False))
    J, L = oracle_fields(m, rays, orig)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert rel_err(Jg[orig], J) < TOL32
    assert rel_err(Lg[orig], L) < TOL32
    assert np.all(np.isfinite(Jg)) and np.all(Lg >= 0) and np.all(Lg < 1)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP64)
    assert rel_err(Jg[orig], J) < TOL64
    assert rel_err(Lg[orig], L) < TOL64
    # statistical equilibrium at every point, fed by the FP64 J-bar; the
    # oracle's at the sampled points, fed by its own
    pg = mgt.mgt_stat_equilibrium(h)
    p0 = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    po = O.stat_equilibrium(p0[orig], J, L, m.temp[orig], m.n_coll[orig], m.n_spec[orig], m.lines)
    assert rel_err(pg[orig], po) < 1e-8
    np.testing.assert_allclose(pg.sum(1), m.n_spec, rtol=1e-12)
    h.close()


@pytest.mark.slow
def test_full_size_shells_grf_1m_sampled(mgt):
    # the 1M-point workload (192 rays, 40 lines x 40 bins, random velocity
    # field) in the launch configuration the benchmark times for it: pair
    # batches of 8, each traced inside the formal solution.  FP32-mixed only:
    # an FP64 solution of this size takes minutes.
    m = synth.config_model(3)
    h = mgt.mgt_model_create(m)
    mgt.mgt_set_solve_opts(h, pairs_per_batch=8)
    st = mgt.mgt_trace_rays(h)
    assert st["n_stalls"] == 0
    rng = np.random.default_rng(3)
    orig = np.sort(rng.choice(m.n_points, 12, replace=False))
    rays = O.trace(m, origins=orig)
    assert rays.stalls == 0
    assert int(np.diff(rays.off).max()) <= st["max_half_ray"]
    J, L = oracle_fields(m, rays, orig)
    Jg, Lg = gpu_fields(mgt, h, mgt.MGT_FP32_MIXED)
    assert rel_err(Jg[orig], J) < TOL32
    assert rel_err(Lg[orig], L) < TOL32
    assert np.all(np.isfinite(Jg)) and np.all(Lg >= 0) and np.all(Lg < 1)
    # populations at every point: finite and conserving the species density
    pg = mgt.mgt_stat_equilibrium(h)
    assert np.all(np.isfinite(pg))
    np.testing.assert_allclose(pg.sum(1), m.n_spec, rtol=1e-12)
    h.close()


# ------------------------------------------- subdivision reference (Sec. 4.3 study)
@pytest.mark.parametrize("prec,tol", [(1, TOL32), (0, TOL64)], ids=["fp32", "fp64"])
def test_subdivision_reference_mode(mgt, prec, tol):
    m = synth.shell_model(2500, 5, 1, 7, grf_sigma=5e3, seed=21, name="grf-2500")
    h = mgt.mgt_model_create(m)
    mgt.mgt_trace_rays(h)
    mgt.mgt_set_solve_opts(h, subdivisions=16)
    J, L = gpu_fields(mgt, h, prec)
    rays = O.trace(m)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    Jr, Lr = O.formal_solve(m, rays, chi, S, subdiv=16)
    assert rel_err(J, Jr) < tol
    assert rel_err(L, Lr) < tol


# ------------------------------------------------------------- pair batches
@pytest.mark.parametrize("prec,tol", [(1, TOL32), (0, TOL64)], ids=["fp32", "fp64"])
def test_pair_batches_match_oracle_and_full_trace(mgt, prec, tol):
    m = synth.shell_model(2500, 5, 2, 7, grf_sigma=5e3, seed=23, name="grf-2500-48")   # 48 rays, 24 pairs
    h = mgt.mgt_model_create(m)
    full = mgt.mgt_trace_rays(h)
    Jf, Lf = gpu_fields(mgt, h, prec)
    mgt.mgt_set_solve_opts(h, pairs_per_batch=5)                 # batches of 5, 5, 5, 5, 4 pairs
    st = mgt.mgt_trace_rays(h)
    for k in ("total_steps", "n_stalls", "max_half_ray", "n_fp64_steps"):
        assert st[k] == full[k], k
    J, L = gpu_fields(mgt, h, prec)
    with pytest.raises(mgt.MgtError):
        mgt.mgt_get_rays(h)
    Jr, Lr = oracle_fields(m, O.trace(m))
    assert rel_err(J, Jr) < tol and rel_err(L, Lr) < tol
    assert rel_err(J, Jf) < 1e-5 if prec == 1 else rel_err(J, Jf) < 1e-12
    # back to all pairs at once
    mgt.mgt_set_solve_opts(h)
    J2, _ = gpu_fields(mgt, h, prec)
    assert np.array_equal(J2, Jf)
