"""The C-ABI library builds, loads and exports what include/*.h declares.

CPU only: no compute call reaches the GPU.  Invalid inputs are rejected by
argument validation, which runs before any CUDA call.
"""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "magritte_gpu.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2411_03040_gb300 import build, mgt
    build.build()
    return mgt.load()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mgt_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2411_03040_gb300", "libmgt.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(mgt_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    # the binding declares every entry point
    from paper_2411_03040_gb300 import mgt
    assert set(names) <= set(mgt.SIGNATURES)


def test_struct_layout_matches_header(tmp_path):
    from paper_2411_03040_gb300 import mgt
    structs = {
        "mgt_model_desc": mgt.mgt_model_desc,
        "mgt_solve_opts": mgt.mgt_solve_opts,
        "mgt_trace_stats": mgt.mgt_trace_stats,
        "mgt_ng_opts": mgt.mgt_ng_opts,
        "mgt_ali_opts": mgt.mgt_ali_opts,
        "mgt_ali_stats": mgt.mgt_ali_stats,
        "mgt_autotune_result": mgt.mgt_autotune_result,
        "mgt_batch_layout": mgt.mgt_batch_layout,
        "mgt_kernel_time": mgt.mgt_kernel_time,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def _with(a, i, v):
    a = np.array(a, copy=True)
    a[i] = v
    return a


def _swap_line_levels(lines, k):
    up, lo = lines.up[k], lines.lo[k]
    lines.up = _with(lines.up, k, lo)
    lines.lo = _with(lines.lo, k, up)


def _small_model():
    from paper_2411_03040_gb300 import synth
    return synth.config_model(1, n_points=60)


@pytest.mark.parametrize("breaker,fragment", [
    (lambda m: setattr(m, "temp", np.where(np.arange(m.n_points) == 3, -1.0, m.temp)), "temperature"),
    (lambda m: setattr(m, "pos", np.where(np.arange(3 * m.n_points).reshape(-1, 3) == 7, np.nan, m.pos)), "finite"),
    (lambda m: setattr(m, "dirs", m.dirs[:-1]), "even"),
    (lambda m: setattr(m, "dirs", m.dirs * 1.01), "unit"),
    (lambda m: setattr(m, "nbrs", np.where(np.arange(m.nbrs.shape[0]) == 5, m.n_points, m.nbrs)), "neighbour"),
    (lambda m: setattr(m, "n_quad", 65), "n_quad"),
    (lambda m: setattr(m, "boundary", np.append(m.boundary, -2)), "boundary"),
    (lambda m: setattr(m.lines, "A", -m.lines.A), "line A"),
    (lambda m: setattr(m, "n_spec", np.zeros_like(m.n_spec)), "n_spec"),
    (lambda m: setattr(m, "vturb2", -np.ones_like(m.vturb2)), "vturb2"),
    (lambda m: setattr(m, "nbr_offsets", _with(m.nbr_offsets, 5, m.nbr_offsets[4] - 1)), "decrease"),
    (lambda m: setattr(m.lines, "up", _with(m.lines.up, 0, m.lines.n_levels)), "line level"),
    (lambda m: _swap_line_levels(m.lines, 0), "above lower"),
    (lambda m: (setattr(m.lines, "up", _with(m.lines.up, 1, m.lines.up[0])),
                setattr(m.lines, "lo", _with(m.lines.lo, 1, m.lines.lo[0]))), "duplicate radiative"),
    (lambda m: setattr(m.lines, "freq_Hz", _with(m.lines.freq_Hz, 1, m.lines.freq_Hz[0] * (1 + 1e-7))),
     "overlapping"),
    (lambda m: setattr(m.lines, "cup", _with(m.lines.cup, 0, m.lines.n_levels)), "collision level"),
    (lambda m: setattr(m.lines, "K_ul", _with(m.lines.K_ul, 0, -1e-17)), "K_ul"),
    (lambda m: setattr(m.lines, "g", _with(m.lines.g, 0, 0.0)), "weights"),
    (lambda m: setattr(m.lines, "mol_mass_kg", 0.0), "mol_mass"),
])
def test_invalid_inputs_rejected_before_any_device_work(lib, breaker, fragment):
    from paper_2411_03040_gb300 import mgt
    m = _small_model()
    breaker(m)
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_model_create(m)
    assert e.value.status == mgt.MGT_ERR_ARG
    assert fragment in str(e.value)


def test_unpaired_direction_rejected(lib):
    from paper_2411_03040_gb300 import mgt
    m = _small_model()
    d = m.dirs.copy()
    d[0] = d[0] + np.array([0.0, 1e-6, 0.0])
    d[0] /= np.linalg.norm(d[0])
    m.dirs = d
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_model_create(m)
    assert e.value.status == mgt.MGT_ERR_ARG and "antipode" in str(e.value)


def test_null_arguments(lib):
    assert lib.mgt_model_create(None, None, None) == 1
    assert lib.mgt_trace_rays(None, None, None) == 1
    assert lib.mgt_formal_solve(None, 0, None, None, 0, None) == 1
    assert lib.mgt_model_destroy(None) == 0
    assert b"NULL" in lib.mgt_last_error()
    # batches and the autotuner reject their arguments before any device call
    out = ctypes.c_void_p()
    assert lib.mgt_batch_create(ctypes.byref(out), None, 0, None) == 1
    assert out.value is None
    assert lib.mgt_batch_create(None, None, 1, None) == 1
    assert lib.mgt_batch_formal_solve(None, None) == 1
    assert lib.mgt_batch_stat_equilibrium(None, None) == 1
    assert lib.mgt_batch_iterate(None, 1, None, None, None) == 1
    assert lib.mgt_batch_get_layout(None, None, None) == 1
    assert lib.mgt_batch_destroy(None) == 0
    assert lib.mgt_autotune(None, 1, 0, 3, None, None) == 1
    assert lib.mgt_get_jbar(None, None, None, 0, None) == 1


def test_binding_fails_loudly_without_library(tmp_path):
    code = ("import paper_2411_03040_gb300.mgt as g\n"
            f"g.LIB_PATH = {str(tmp_path / 'nope.so')!r}\n"
            "try:\n    g.load()\nexcept RuntimeError as e:\n    print('RAISED', 'no CPU fallback' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT).stdout
    assert "RAISED True" in out


def test_batch_workload_specs_are_seeded_and_in_range():
    # the batch workload's sizes: log-uniform points in [5k, 200k], levels from
    # {5, 11, 21, 41}, HEALPix nside 1 or 2, the same on every call
    from paper_2411_03040_gb300 import synth
    a = synth.batch_specs(256)
    assert a == synth.batch_specs(256)
    n = np.array([x[0] for x in a])
    assert n.min() >= 5_000 and n.max() <= 200_000
    assert {x[1] for x in a} == {5, 11, 21, 41}
    assert {x[2] for x in a} == {1, 2}
    # log-uniform: about half the models below the geometric mean of the range
    assert 0.35 < np.mean(n < np.sqrt(5_000 * 200_000)) < 0.65
    assert len({x[4] for x in a}) == 256            # one seed per model


@pytest.mark.parametrize("kw,fragment", [
    (dict(rho=np.array([1.0, 2.0, -1.0, 1.0])), "rho"),
    (dict(pos=np.where(np.arange(12).reshape(4, 3) == 5, np.inf, 0.0)), "positions"),
    (dict(r_max=-0.1), "r_max"),
    (dict(max_level=31), "max_level"),
    (dict(n_side=1), "n_side"),
    (dict(pos=np.zeros((0, 3)), rho=np.zeros(0)), "n_points"),
])
def test_remesh_rejects_bad_input_before_any_device_work(lib, kw, fragment):
    from paper_2411_03040_gb300 import mgt
    args = dict(pos=np.zeros((4, 3)), rho=np.ones(4), r_max=0.4, max_level=5, n_side=3)
    args.update(kw)
    with pytest.raises(mgt.MgtError) as e:
        mgt.mgt_remesh(args["pos"], args["rho"], args["r_max"], args["max_level"], args["n_side"])
    assert e.value.status == mgt.MGT_ERR_ARG
    assert fragment in str(e.value)


def test_noalloc_ng_rejects_sizes_and_null_pointers_before_any_device_work(lib):
    import ctypes as C
    buf = (C.c_double * 4)()
    neg = C.c_int64()
    # n_iterates outside 2..17, an empty vector, null device pointers
    for n, ln, it, pr in [(1, 4, buf, buf), (18, 4, buf, buf), (3, 0, buf, buf), (3, 4, None, buf), (3, 4, buf, None)]:
        st = lib.mgt_ng_extrapolate_noalloc(n, it, ln, pr, buf, C.byref(neg), None)
        assert st == 1, (n, ln)
        assert b"mgt_ng_extrapolate_noalloc" in lib.mgt_last_error()


def test_noalloc_wrapper_rejects_bad_tensors_before_the_library():
    # the C entry point sees only pointers and a length: the binding checks
    # dtype, shape, layout and device first (these CPU tensors never reach it)
    torch = pytest.importorskip("torch")
    from paper_2411_03040_gb300 import mgt
    X = torch.zeros((3, 8), dtype=torch.float64)
    out = torch.zeros(8, dtype=torch.float64)
    cases = [
        (X.float(), out, "float64"),
        (X, out.float(), "float64"),
        (X.reshape(-1), out, "2-D"),
        (X, torch.zeros(7, dtype=torch.float64), "entries per iterate"),
        (torch.zeros((8, 3), dtype=torch.float64).t(), out, "contiguous"),
        (X, out, "CUDA device"),
    ]
    for it, pr, msg in cases:
        with pytest.raises(ValueError, match=msg):
            mgt.mgt_ng_extrapolate_noalloc(it, pr)


def test_binding_checks_caller_buffers_before_the_library():
    # the C entry points see only pointers: every wrapper that passes a
    # caller's array or tensor checks its dtype, size, layout, writability and
    # memory kind first (these CPU-side cases never reach the library)
    from paper_2411_03040_gb300 import mgt
    ok = np.zeros((4, 5), np.float64)
    assert mgt._buffer("f", "x", ok, 20, np.float64, writable=True) == 0
    ro = np.zeros((4, 5), np.float64)
    ro.flags.writeable = False
    cases = [
        (np.zeros((4, 5), np.float32), 20, {}, "float64 array"),
        (np.zeros((4, 4), np.float64), 20, {}, "16 elements, expected 20"),
        (np.zeros((5, 4), np.float64).T, 20, {}, "C-contiguous"),
        (ro, 20, {"writable": True}, "read-only"),
        ([0.0] * 20, 20, {}, "numpy array or a torch CUDA tensor"),
        (ok, 20, {"device": True}, "torch CUDA tensor"),
    ]
    for a, n, kw, msg in cases:
        with pytest.raises(ValueError, match=msg):
            mgt._buffer("f", "x", a, n, np.float64, **kw)
    torch = pytest.importorskip("torch")
    for t, msg in [(torch.zeros(20, dtype=torch.float32), "float64 tensor"),
                   (torch.zeros((5, 4), dtype=torch.float64).t(), "contiguous"),
                   (torch.zeros(20, dtype=torch.float64), "current CUDA device")]:
        with pytest.raises(ValueError, match=msg):
            mgt._buffer("f", "x", t, 20, np.float64)
