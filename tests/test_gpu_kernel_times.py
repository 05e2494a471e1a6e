"""Per-kernel event timing of the library (mgt_kernel_timing / mgt_kernel_times),
which the benchmark uses for its step breakdown, roofline and DRAM rates."""
import numpy as np
import pytest

from paper_2411_03040_gb300 import synth

pytestmark = pytest.mark.gpu


def test_kernel_times_cover_one_ali_step():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2411_03040_gb300 import build, mgt
    build.build()
    mgt.load()
    m = synth.sphere_model(1500, n_levels=5, nside=1, n_quad=11, seed=21, name="ktimes")
    h = mgt.mgt_model_create(m)
    # 4 lines fit one line group: the automatic staged choice is the kernel
    # with per-thread coefficients (k_fs_fused)
    mgt.mgt_kernel_timing(True)
    mgt.mgt_trace_rays(h)
    mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED, want=False)
    mgt.mgt_formal_solve(h, mgt.MGT_FP64, want=False)
    mgt.mgt_stat_equilibrium(h, want=False)
    for _ in range(3):
        mgt.mgt_ng_accelerate(h, mgt.MGT_NG_ADAPTIVE, n_max=8)
    mgt.mgt_sync(h)
    kt = mgt.mgt_kernel_times()
    mgt.mgt_kernel_timing(False)
    for name in ("k_walk<fused>", "k_walk_compact", "k_line_data", "k_fs_fused<f32>", "k_fs_fused<f64>", "k_se",
                 "k_ng_push"):
        assert name in kt, (name, sorted(kt))
        assert kt[name]["launches"] >= 1 and kt[name]["total_ms"] > 0.0, (name, kt[name])
    assert kt["k_fs_fused<f32>"]["launches"] == 1 and kt["k_fs_fused<f64>"]["launches"] == 1
    assert "k_fs_staged<f32>" not in kt
    # the line-data launch states its bytes: populations and w in, both rows out
    N, L, M = m.n_points, m.lines.n_levels, m.lines.n_lines
    Mpad = -(-M // 8) * 8
    want = N * (8.0 * L + 8.0 + 4.0 * (2 * Mpad + 4) + 8.0 * (2 * Mpad + 2))
    assert kt["k_line_data"]["bytes"] in (pytest.approx(want), pytest.approx(N * (8.0 * L + 8.0 + 4.0 * (2 * Mpad + 4))))
    # nothing more is recorded while timing is off, and switching it on clears
    mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED, want=False)
    mgt.mgt_sync(h)
    assert mgt.mgt_kernel_times()["k_fs_fused<f32>"]["launches"] == 1
    # schedule 2 runs the kernel with the shared pre-pass
    mgt.mgt_set_solve_opts(h, schedule=2)
    mgt.mgt_kernel_timing(True)
    mgt.mgt_formal_solve(h, mgt.MGT_FP32_MIXED, want=False)
    mgt.mgt_sync(h)
    kt = mgt.mgt_kernel_times()
    assert kt["k_fs_staged<f32>"]["launches"] == 1 and "k_fs_fused<f32>" not in kt
    mgt.mgt_kernel_timing(False)
    mgt.mgt_kernel_timing(True)
    assert mgt.mgt_kernel_times() == {}
    mgt.mgt_kernel_timing(False)
    h.close()
