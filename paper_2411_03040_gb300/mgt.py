"""Thin ctypes binding of libmgt.so (the C-ABI in include/magritte_gpu.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions carry the C names.  Arrays are numpy (host) or anything with
``data_ptr()`` (a torch CUDA tensor, used with ``on_device=1``); ``stream`` is
a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None (the legacy
default stream).

Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgt.so")

MGT_OK, MGT_ERR_ARG, MGT_ERR_CUDA, MGT_ERR_OOM, MGT_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
MGT_ERR_SINGULAR, MGT_ERR_TIMEOUT, MGT_ERR_BOUNDS, MGT_ERR_STATE = 5, 6, 7, 8
MGT_FP64, MGT_FP32_MIXED = 0, 1
MGT_NG_NONE, MGT_NG_CLASSICAL, MGT_NG_ADAPTIVE = 0, 1, 2

_P = ctypes.c_void_p
_i64, _i32, _f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double


class mgt_model_desc(ctypes.Structure):
    _fields_ = [
        ("n_points", _i64), ("pos", _P), ("vel", _P), ("temp", _P), ("vturb2", _P), ("n_coll", _P),
        ("n_spec", _P), ("nbr_offsets", _P), ("nbrs", _P), ("n_boundary", _i32), ("boundary", _P),
        ("n_rays", _i32), ("dirs", _P), ("n_quad", _i32), ("mol_mass_kg", _f64), ("T_bg", _f64),
        ("n_levels", _i32), ("energy_J", _P), ("g", _P), ("n_lines", _i32), ("up", _P), ("lo", _P),
        ("A", _P), ("freq_Hz", _P), ("n_coll_trans", _i32), ("cup", _P), ("clo", _P), ("K_ul", _P),
    ]


class mgt_solve_opts(ctypes.Structure):
    _fields_ = [("switch_threshold", _f64), ("width_mode", _i32), ("lines_per_thread", _i32),
                ("schedule", _i32), ("subdivisions", _i32), ("pairs_per_batch", _i32)]


class mgt_trace_stats(ctypes.Structure):
    _fields_ = [("total_steps", _i64), ("n_stalls", _i64), ("max_half_ray", _i32), ("mean_half_ray", _f64),
                ("n_fp64_steps", _i64)]


class mgt_ng_opts(ctypes.Structure):
    _fields_ = [("mode", _i32), ("n_steps", _i32), ("n_max", _i32)]


class mgt_ali_opts(ctypes.Structure):
    _fields_ = [("n_iter", _i32), ("precision", _i32), ("ng", mgt_ng_opts)]


class mgt_ali_stats(ctypes.Structure):
    _fields_ = [("iterations", _i32), ("ng_accepted", _i32), ("last_maxrel", _f64)]


class mgt_autotune_result(ctypes.Structure):
    _fields_ = [("schedule", _i32), ("lines_per_thread", _i32), ("n_tried", _i32),
                ("schedules", _i32 * 8), ("lines", _i32 * 8), ("ms", ctypes.c_float * 8)]


class mgt_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", _i64), ("total_ms", _f64), ("bytes", _f64)]


class mgt_batch_layout(ctypes.Structure):
    _fields_ = [("n_models", _i32), ("fs_items", _i64), ("fs_grid", _i32), ("fs_threads", _i32),
                ("fs_smem_bytes", _i64), ("se_blocks", _i64), ("graph_kernels", _i32), ("fs_launches", _i32),
                ("fs_solo", _i32)]


# name -> argtypes (every function returns an int status, except mgt_last_error)
SIGNATURES = {
    "mgt_model_create": [ctypes.POINTER(_P), ctypes.POINTER(mgt_model_desc), _P],
    "mgt_model_destroy": [_P],
    "mgt_set_solve_opts": [_P, ctypes.POINTER(mgt_solve_opts)],
    "mgt_trace_rays": [_P, ctypes.POINTER(mgt_trace_stats), _P],
    "mgt_get_rays": [_P, _P, _P, _P],
    "mgt_set_populations": [_P, _P, _P],
    "mgt_get_populations": [_P, _P, ctypes.c_int, _P],
    "mgt_formal_solve": [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P],
    "mgt_stat_equilibrium": [_P, _P, _P],
    "mgt_get_jbar": [_P, _P, _P, ctypes.c_int, _P],
    "mgt_ng_accelerate": [_P, ctypes.POINTER(mgt_ng_opts), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(_f64), _P],
    "mgt_ali_solve": [_P, ctypes.POINTER(mgt_ali_opts), ctypes.POINTER(mgt_ali_stats), _P],
    "mgt_image": [_P, _P, _i32, _i32, _i32, _f64, _f64, _P, ctypes.c_int, _P],
    "mgt_image_adjoint": [_P, _P, _i32, _i32, _i32, _f64, _f64, _P, _P, _P, _P, ctypes.c_int, _P],
    "mgt_image_rays": [_P, _P, _i32, _i32, _P, _P, _P, _P],
    "mgt_set_point_fields": [_P, _P, _P, _P, ctypes.c_int, _P],
    "mgt_remesh": [_i64, _P, _P, _f64, _i32, _i32, _P, _P, _i64, ctypes.POINTER(_i64), _P],
    "mgt_ng_extrapolate_noalloc": [_i32, _P, _i64, _P, _P, ctypes.POINTER(_i64), _P],
    "mgt_autotune": [_P, ctypes.c_int, _i32, _i32, ctypes.POINTER(mgt_autotune_result), _P],
    "mgt_batch_create": [ctypes.POINTER(_P), ctypes.POINTER(_P), _i32, _P],
    "mgt_batch_destroy": [_P],
    "mgt_batch_formal_solve": [_P, _P],
    "mgt_batch_stat_equilibrium": [_P, _P],
    "mgt_batch_iterate": [_P, _i32, ctypes.POINTER(mgt_ng_opts), _P, _P],
    "mgt_batch_get_layout": [_P, ctypes.POINTER(mgt_batch_layout), _P],
    "mgt_sync": [_P, _P],
    "mgt_model_sizes": [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                        ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
    "mgt_launch_count": [ctypes.POINTER(_i64)],
    "mgt_kernel_timing": [_i32],
    "mgt_kernel_times": [_i32, ctypes.POINTER(mgt_kernel_time), ctypes.POINTER(_i32)],
    "mgt_last_error": [],
}

_lib = None


class MgtError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load libmgt.so (built by paper_2411_03040_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2411_03040_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "mgt_last_error" else ctypes.c_int
    _lib = lib
    return lib


def _check(status, where):
    if status != MGT_OK:
        raise MgtError(status, where, load().mgt_last_error().decode())


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _buffer(fn, name, a, n, dtype, device=None, writable=False):
    """Check a caller's buffer before its pointer goes to the library, which
    sees only the pointer: ``n`` elements of ``dtype``, C-contiguous, either a
    numpy array (host) or a torch tensor on the current CUDA device.
    ``device`` True or False asks for one of the two kinds.  Returns 1 for a
    device buffer, 0 for a host one; ValueError otherwise."""
    dt = np.dtype(dtype)
    if hasattr(a, "data_ptr"):
        kind = 1
        if str(a.dtype) != "torch." + dt.name:
            raise ValueError(f"{fn}: {name} must be a {dt.name} tensor, not {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{fn}: {name} must be contiguous")
        if not a.is_cuda:
            raise ValueError(f"{fn}: {name} must be a numpy array or a tensor on the current CUDA device")
        import torch
        if a.device.index != torch.cuda.current_device():
            raise ValueError(f"{fn}: {name} must be on the current CUDA device")
        size = int(a.numel())
    elif isinstance(a, np.ndarray):
        kind = 0
        if a.dtype != dt:
            raise ValueError(f"{fn}: {name} must be a {dt.name} array, not {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{fn}: {name} must be C-contiguous")
        if writable and not a.flags.writeable:
            raise ValueError(f"{fn}: {name} is read-only")
        size = int(a.size)
    else:
        raise ValueError(f"{fn}: {name} must be a numpy array or a torch CUDA tensor")
    if size != n:
        raise ValueError(f"{fn}: {name} has {size} elements, expected {n}")
    if device is not None and kind != int(bool(device)):
        raise ValueError(f"{fn}: {name} must be " + ("a torch CUDA tensor" if device else "a host numpy array"))
    return kind


class Model:
    """Owns one mgt_model handle and keeps its host inputs alive while in use."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        try:
            if self.handle:
                load().mgt_model_destroy(self.handle)
        except Exception:
            pass
        self.handle = None

    def close(self):
        if self.handle:
            _check(load().mgt_model_destroy(self.handle), "mgt_model_destroy")
            self.handle = None


def mgt_model_create(model, stream=None) -> Model:
    """``model`` has the fields of paper_2411_03040_gb300.synth.Model."""
    lib = load()
    ln = model.lines
    arr = lambda a, t: np.ascontiguousarray(a, dtype=t)
    keep = dict(
        pos=arr(model.pos, np.float64), vel=arr(model.vel, np.float64), temp=arr(model.temp, np.float64),
        vturb2=arr(model.vturb2, np.float64), n_coll=arr(model.n_coll, np.float64),
        n_spec=arr(model.n_spec, np.float64), off=arr(model.nbr_offsets, np.int64),
        nbrs=arr(model.nbrs, np.int32), bnd=arr(model.boundary, np.int32), dirs=arr(model.dirs, np.float64),
        E=arr(ln.energy_J, np.float64), g=arr(ln.g, np.float64), up=arr(ln.up, np.int32),
        lo=arr(ln.lo, np.int32), A=arr(ln.A, np.float64), nu=arr(ln.freq_Hz, np.float64),
        cup=arr(ln.cup, np.int32), clo=arr(ln.clo, np.int32), K=arr(ln.K_ul, np.float64))
    k = keep
    d = mgt_model_desc(
        n_points=model.n_points, pos=_ptr(k["pos"]), vel=_ptr(k["vel"]), temp=_ptr(k["temp"]),
        vturb2=_ptr(k["vturb2"]), n_coll=_ptr(k["n_coll"]), n_spec=_ptr(k["n_spec"]),
        nbr_offsets=_ptr(k["off"]), nbrs=_ptr(k["nbrs"]), n_boundary=k["bnd"].shape[0], boundary=_ptr(k["bnd"]),
        n_rays=k["dirs"].shape[0], dirs=_ptr(k["dirs"]), n_quad=int(model.n_quad),
        mol_mass_kg=float(ln.mol_mass_kg), T_bg=float(model.T_bg), n_levels=int(ln.n_levels),
        energy_J=_ptr(k["E"]), g=_ptr(k["g"]), n_lines=int(ln.n_lines), up=_ptr(k["up"]), lo=_ptr(k["lo"]),
        A=_ptr(k["A"]), freq_Hz=_ptr(k["nu"]), n_coll_trans=int(k["cup"].shape[0]), cup=_ptr(k["cup"]),
        clo=_ptr(k["clo"]), K_ul=_ptr(k["K"]))
    h = ctypes.c_void_p()
    _check(lib.mgt_model_create(ctypes.byref(h), ctypes.byref(d), _stream(stream)), "mgt_model_create")
    return Model(h, keep)


def mgt_model_sizes(m: Model):
    n, r, l, mm, q = _i64(), _i32(), _i32(), _i32(), _i32()
    _check(load().mgt_model_sizes(m.handle, ctypes.byref(n), ctypes.byref(r), ctypes.byref(l), ctypes.byref(mm),
                                  ctypes.byref(q)), "mgt_model_sizes")
    return dict(n_points=n.value, n_rays=r.value, n_levels=l.value, n_lines=mm.value, n_quad=q.value)


def mgt_set_solve_opts(m: Model, switch_threshold=0.35, width_mode=0, lines_per_thread=0, schedule=0,
                       subdivisions=0, pairs_per_batch=0):
    o = mgt_solve_opts(switch_threshold, width_mode, lines_per_thread, schedule, subdivisions, pairs_per_batch)
    _check(load().mgt_set_solve_opts(m.handle, ctypes.byref(o)), "mgt_set_solve_opts")


def mgt_trace_rays(m: Model, stream=None) -> dict:
    st = mgt_trace_stats()
    _check(load().mgt_trace_rays(m.handle, ctypes.byref(st), _stream(stream)), "mgt_trace_rays")
    return dict(total_steps=st.total_steps, n_stalls=st.n_stalls, max_half_ray=st.max_half_ray,
                mean_half_ray=st.mean_half_ray, n_fp64_steps=st.n_fp64_steps)


def mgt_get_rays(m: Model, stream=None):
    s = mgt_model_sizes(m)
    off = np.zeros(s["n_rays"] * s["n_points"] + 1, np.int64)
    _check(load().mgt_get_rays(m.handle, _ptr(off), None, _stream(stream)), "mgt_get_rays")
    idx = np.zeros(int(off[-1]), np.int32)
    _check(load().mgt_get_rays(m.handle, None, _ptr(idx) if idx.size else None, _stream(stream)), "mgt_get_rays")
    return off, idx


def mgt_set_populations(m: Model, pops=None, stream=None):
    p = None
    if pops is not None:
        s = mgt_model_sizes(m)
        p = np.ascontiguousarray(pops, np.float64)
        _buffer("mgt_set_populations", "pops", p, s["n_points"] * s["n_levels"], np.float64, device=False)
    _check(load().mgt_set_populations(m.handle, _ptr(p), _stream(stream)), "mgt_set_populations")


def mgt_get_populations(m: Model, out=None, stream=None):
    s = mgt_model_sizes(m)
    if out is None:
        out = np.zeros((s["n_points"], s["n_levels"]), np.float64)
    on_dev = _buffer("mgt_get_populations", "out", out, s["n_points"] * s["n_levels"], np.float64, writable=True)
    _check(load().mgt_get_populations(m.handle, _ptr(out), on_dev, _stream(stream)), "mgt_get_populations")
    return out


def _jbar_buffers(fn, Jbar, Lstar, sizes):
    """Both outputs [M][N] f64, of one memory kind; returns that kind."""
    n = sizes["n_lines"] * sizes["n_points"]
    on_dev = _buffer(fn, "Jbar", Jbar, n, np.float64, writable=True)
    _buffer(fn, "Lstar", Lstar, n, np.float64, device=bool(on_dev), writable=True)
    return on_dev


def mgt_formal_solve(m: Model, precision=MGT_FP32_MIXED, Jbar=None, Lstar=None, want=True, stream=None):
    """Returns (Jbar, Lstar) [M][N].  With ``want`` False nothing is copied out.
    Given torch CUDA tensors the results are written on the device."""
    if not want:
        _check(load().mgt_formal_solve(m.handle, precision, None, None, 0, _stream(stream)), "mgt_formal_solve")
        return None, None
    s = mgt_model_sizes(m)
    if Jbar is None:
        Jbar = np.zeros((s["n_lines"], s["n_points"]), np.float64)
    if Lstar is None:
        Lstar = np.zeros((s["n_lines"], s["n_points"]), np.float64)
    on_dev = _jbar_buffers("mgt_formal_solve", Jbar, Lstar, s)
    _check(load().mgt_formal_solve(m.handle, precision, _ptr(Jbar), _ptr(Lstar), on_dev, _stream(stream)),
           "mgt_formal_solve")
    return Jbar, Lstar


def mgt_get_jbar(m: Model, Jbar=None, Lstar=None, stream=None):
    """The model's last J-bar and Lambda*, [M][N] (host, or the given torch CUDA tensors)."""
    s = mgt_model_sizes(m)
    if Jbar is None:
        Jbar = np.zeros((s["n_lines"], s["n_points"]), np.float64)
    if Lstar is None:
        Lstar = np.zeros((s["n_lines"], s["n_points"]), np.float64)
    on_dev = _jbar_buffers("mgt_get_jbar", Jbar, Lstar, s)
    _check(load().mgt_get_jbar(m.handle, _ptr(Jbar), _ptr(Lstar), on_dev, _stream(stream)), "mgt_get_jbar")
    return Jbar, Lstar


def mgt_stat_equilibrium(m: Model, want=True, stream=None, out=None):
    """New populations [N][L]; into ``out`` (host array, e.g. pinned) if given."""
    if want and out is None:
        s = mgt_model_sizes(m)
        out = np.zeros((s["n_points"], s["n_levels"]), np.float64)
    if not want:
        out = None
    else:
        s = mgt_model_sizes(m)
        _buffer("mgt_stat_equilibrium", "out", out, s["n_points"] * s["n_levels"], np.float64, device=False,
                writable=True)
    _check(load().mgt_stat_equilibrium(m.handle, _ptr(out), _stream(stream)), "mgt_stat_equilibrium")
    return out


def mgt_ng_accelerate(m: Model, mode=MGT_NG_NONE, n_steps=4, n_max=8, stream=None):
    o = mgt_ng_opts(mode, n_steps, n_max)
    acc = ctypes.c_int(0)
    mr = _f64(0.0)
    _check(load().mgt_ng_accelerate(m.handle, ctypes.byref(o), ctypes.byref(acc), ctypes.byref(mr),
                                    _stream(stream)), "mgt_ng_accelerate")
    return bool(acc.value), mr.value


def mgt_ali_solve(m: Model, n_iter=20, precision=MGT_FP32_MIXED, ng_mode=MGT_NG_NONE, n_steps=4, n_max=8,
                  stream=None):
    o = mgt_ali_opts(n_iter, precision, mgt_ng_opts(ng_mode, n_steps, n_max))
    st = mgt_ali_stats()
    _check(load().mgt_ali_solve(m.handle, ctypes.byref(o), ctypes.byref(st), _stream(stream)), "mgt_ali_solve")
    return dict(iterations=st.iterations, ng_accepted=st.ng_accepted, last_maxrel=st.last_maxrel)


def _dir(direction):
    return np.ascontiguousarray(direction, np.float64)


def mgt_image(m: Model, direction, npx, npy, nfreq, fmin, fmax, out=None, stream=None):
    """Image [nfreq][npy][npx] f32; ``out`` may be a torch CUDA tensor."""
    d = _dir(direction)
    if out is None:
        out = np.zeros((nfreq, npy, npx), np.float32)
    on_dev = _buffer("mgt_image", "out", out, int(nfreq) * int(npy) * int(npx), np.float32, writable=True)
    _check(load().mgt_image(m.handle, _ptr(d), npx, npy, nfreq, float(fmin), float(fmax), _ptr(out), on_dev,
                            _stream(stream)), "mgt_image")
    return out


def mgt_image_adjoint(m: Model, direction, npx, npy, nfreq, fmin, fmax, grad_out, g_logT=None, g_logn=None,
                      g_vel=None, stream=None):
    """(g_logT [N], g_logn [N], g_vel [N][3]) for dL/dI = grad_out.  With a
    torch CUDA ``grad_out`` the outputs must be torch CUDA tensors too."""
    d = _dir(direction)
    fn = "mgt_image_adjoint"
    on_dev = 1 if hasattr(grad_out, "data_ptr") else 0
    n = mgt_model_sizes(m)["n_points"]
    if not on_dev:
        grad_out = np.ascontiguousarray(grad_out, np.float32)
        g_logT = np.zeros(n) if g_logT is None else g_logT
        g_logn = np.zeros(n) if g_logn is None else g_logn
        g_vel = np.zeros((n, 3)) if g_vel is None else g_vel
    _buffer(fn, "grad_out", grad_out, int(nfreq) * int(npy) * int(npx), np.float32, device=bool(on_dev))
    for name, g, k in (("g_logT", g_logT, 1), ("g_logn", g_logn, 1), ("g_vel", g_vel, 3)):
        if g is not None:
            _buffer(fn, name, g, k * n, np.float64, device=bool(on_dev), writable=True)
    _check(load().mgt_image_adjoint(m.handle, _ptr(d), npx, npy, nfreq, float(fmin), float(fmax), _ptr(grad_out),
                                    _ptr(g_logT), _ptr(g_logn), _ptr(g_vel), on_dev, _stream(stream)),
           "mgt_image_adjoint")
    return g_logT, g_logn, g_vel


def mgt_image_rays(m: Model, direction, npx, npy, stream=None):
    """(anchor, ray_off, pts) of the pixel rays, host arrays."""
    d = _dir(direction)
    npix = npx * npy
    anchor = np.zeros(npix, np.int32)
    off = np.zeros(npix + 1, np.int64)
    _check(load().mgt_image_rays(m.handle, _ptr(d), npx, npy, _ptr(anchor), _ptr(off), None, _stream(stream)),
           "mgt_image_rays")
    pts = np.zeros(max(int(off[-1]), 1), np.int32)
    _check(load().mgt_image_rays(m.handle, _ptr(d), npx, npy, None, None, _ptr(pts), _stream(stream)),
           "mgt_image_rays")
    return anchor, off, pts[:int(off[-1])]


def mgt_set_point_fields(m: Model, temp=None, n_spec=None, vel=None, stream=None):
    """Replace T [N], n_spec [N] and/or v [N][3] (numpy or torch CUDA tensors)."""
    arrs = [temp, n_spec, vel]
    on_dev = 1 if any(hasattr(a, "data_ptr") for a in arrs if a is not None) else 0
    if not on_dev:
        arrs = [None if a is None else np.ascontiguousarray(a, np.float64) for a in arrs]
    n = mgt_model_sizes(m)["n_points"]
    for name, a, k in zip(("temp", "n_spec", "vel"), arrs, (1, 1, 3)):
        if a is not None:
            _buffer("mgt_set_point_fields", name, a, k * n, np.float64, device=bool(on_dev))
    _check(load().mgt_set_point_fields(m.handle, *[_ptr(a) for a in arrs], on_dev, _stream(stream)),
           "mgt_set_point_fields")


def mgt_remesh(pos, rho, r_max, max_level, n_side, stream=None):
    """Re-meshed point cloud: (points [K][3], boundary flags [K])."""
    pos = np.ascontiguousarray(pos, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    n = pos.shape[0]
    k = _i64(0)
    _check(load().mgt_remesh(n, _ptr(pos), _ptr(rho), float(r_max), int(max_level), int(n_side), None, None, 0,
                             ctypes.byref(k), _stream(stream)), "mgt_remesh")
    out = np.zeros((k.value, 3), np.float64)
    flags = np.zeros(k.value, np.uint8)
    _check(load().mgt_remesh(n, _ptr(pos), _ptr(rho), float(r_max), int(max_level), int(n_side), _ptr(out),
                             _ptr(flags), k.value, ctypes.byref(k), _stream(stream)), "mgt_remesh")
    return out, flags


def _check_noalloc_tensors(iterates, prediction):
    """The C side sees only pointers and sizes, so the tensors' dtype, shape,
    layout, device and disjointness are checked here, before the library is
    touched; ValueError otherwise."""
    for name, t in (("iterates", iterates), ("prediction", prediction)):
        if str(getattr(t, "dtype", None)) != "torch.float64":
            raise ValueError(f"mgt_ng_extrapolate_noalloc: {name} must be a float64 torch tensor")
    if iterates.dim() != 2:
        raise ValueError("mgt_ng_extrapolate_noalloc: iterates must be 2-D [n_iterates][len]")
    if int(iterates.shape[1]) != int(prediction.numel()):
        raise ValueError(f"mgt_ng_extrapolate_noalloc: iterates have {int(iterates.shape[1])} entries per iterate, "
                         f"prediction has {int(prediction.numel())}")
    for name, t in (("iterates", iterates), ("prediction", prediction)):
        if not t.is_contiguous():
            raise ValueError(f"mgt_ng_extrapolate_noalloc: {name} must be contiguous")
    import torch
    for name, t in (("iterates", iterates), ("prediction", prediction)):
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"mgt_ng_extrapolate_noalloc: {name} must be on the current CUDA device")
    p0, i0 = prediction.data_ptr(), iterates.data_ptr()
    if p0 < i0 + iterates.numel() * 8 and i0 < p0 + prediction.numel() * 8:
        raise ValueError("mgt_ng_extrapolate_noalloc: prediction overlaps the iterates")


def mgt_ng_extrapolate_noalloc(iterates, prediction, stream=None):
    """Ng prediction from ``iterates`` (device tensor [n][len] f64, oldest
    first) into ``prediction`` (device tensor [len] f64) without any device
    allocation; returns (coefficients, number of negative entries)."""
    _check_noalloc_tensors(iterates, prediction)
    n = int(iterates.shape[0])
    ln = int(prediction.numel())
    coef = np.zeros(max(n - 1, 1), np.float64)
    neg = _i64(0)
    _check(load().mgt_ng_extrapolate_noalloc(n, _ptr(iterates), ln, _ptr(prediction), _ptr(coef),
                                             ctypes.byref(neg), _stream(stream)), "mgt_ng_extrapolate_noalloc")
    return coef[:n - 1], neg.value


def mgt_autotune(m: Model, precision=MGT_FP32_MIXED, staged_only=False, reps=3, stream=None) -> dict:
    """Time the candidate schedules, set the fastest in the model's options."""
    r = mgt_autotune_result()
    _check(load().mgt_autotune(m.handle, precision, int(bool(staged_only)), reps, ctypes.byref(r), _stream(stream)),
           "mgt_autotune")
    n = r.n_tried
    return dict(schedule=r.schedule, lines_per_thread=r.lines_per_thread,
                tried=[(r.schedules[i], r.lines[i], r.ms[i]) for i in range(n)])


class Batch:
    """Owns one mgt_batch handle and keeps its models alive while in use."""

    def __init__(self, handle, models):
        self.handle = handle
        self.models = list(models)

    def __del__(self):
        try:
            if self.handle:
                load().mgt_batch_destroy(self.handle)
        except Exception:
            pass
        self.handle = None

    def close(self):
        if self.handle:
            _check(load().mgt_batch_destroy(self.handle), "mgt_batch_destroy")
            self.handle = None


def mgt_batch_create(models, stream=None) -> Batch:
    lib = load()
    arr = (_P * len(models))(*[m.handle for m in models])
    h = _P()
    _check(lib.mgt_batch_create(ctypes.byref(h), arr, len(models), _stream(stream)), "mgt_batch_create")
    return Batch(h, models)


def mgt_batch_formal_solve(b: Batch, stream=None):
    _check(load().mgt_batch_formal_solve(b.handle, _stream(stream)), "mgt_batch_formal_solve")


def mgt_batch_stat_equilibrium(b: Batch, stream=None):
    _check(load().mgt_batch_stat_equilibrium(b.handle, _stream(stream)), "mgt_batch_stat_equilibrium")


def mgt_batch_iterate(b: Batch, n_iter=1, ng_mode=MGT_NG_NONE, n_steps=4, n_max=8, want_stats=False, stream=None):
    """n_iter ALI iterations of every model; per-model stats (caller's order) if asked."""
    o = mgt_ng_opts(ng_mode, n_steps, n_max)
    st = (mgt_ali_stats * len(b.models))() if want_stats else None
    _check(load().mgt_batch_iterate(b.handle, n_iter, ctypes.byref(o), st, _stream(stream)), "mgt_batch_iterate")
    if not want_stats:
        return None
    return [dict(iterations=x.iterations, ng_accepted=x.ng_accepted, last_maxrel=x.last_maxrel) for x in st]


def mgt_batch_get_layout(b: Batch) -> dict:
    lay = mgt_batch_layout()
    order = np.zeros(len(b.models), dtype=np.int32)
    _check(load().mgt_batch_get_layout(b.handle, ctypes.byref(lay), _ptr(order)), "mgt_batch_get_layout")
    d = {k: getattr(lay, k) for k, _ in mgt_batch_layout._fields_}
    d["order"] = order
    return d


def mgt_sync(m: Model, stream=None):
    _check(load().mgt_sync(m.handle, _stream(stream)), "mgt_sync")


def mgt_launch_count() -> int:
    c = _i64(0)
    _check(load().mgt_launch_count(ctypes.byref(c)), "mgt_launch_count")
    return c.value


def mgt_kernel_timing(enable: bool):
    """Start (clearing the totals) or stop per-kernel event timing."""
    _check(load().mgt_kernel_timing(int(bool(enable))), "mgt_kernel_timing")


def mgt_kernel_times() -> dict:
    """{kernel name: {"launches", "total_ms", "bytes"}} of the timed launches so far."""
    n = _i32(0)
    _check(load().mgt_kernel_times(0, None, ctypes.byref(n)), "mgt_kernel_times")
    arr = (mgt_kernel_time * max(n.value, 1))()
    _check(load().mgt_kernel_times(n.value, arr, ctypes.byref(n)), "mgt_kernel_times")
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
                                   "bytes": float(arr[i].bytes)} for i in range(n.value)}


def mgt_last_error() -> str:
    return load().mgt_last_error().decode()
