"""Plain FP64 reference of the Magritte line-transfer hot path (arXiv 2411.03040).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA library never calls it, and it imports nothing from the CUDA
path; the two share only the seeded input generator.

What is here, each step in the paper's notation:
  * Planck function, Gauss-Hermite frequency quadrature (Sec. 3.2 ``nquads``).
  * Line widths (Sec. 4.3, eq. line width), Einstein coefficients, line
    opacity chi^{ij} and source function S^{ij} from level populations.
  * LTE (Boltzmann) populations (Listing 3, compute_LTE_level_populations).
  * Ray tracing, segment optical depths (Sec. 4.3: trapezoidal rule and the
    semi-analytic erf form with the 0.35 switch) and the second-order formal
    solution with J-bar / Lambda* (in ``oracle_c.c``).
  * Statistical equilibrium with an approximate-Lambda preconditioning, solved
    per point by state reduction (componentwise accurate for tiny populations).
  * Ng-acceleration for a general number of iterates (Sec. 4.2, eq. for c and
    Appendix A), classical and adaptive variants.
  * The accelerated-Lambda-iteration driver (Listing 3,
    compute_level_populations_sparse).
  * The synthetic image (Listing 3, compute_image_new) and its gradient with
    respect to per-point log T, log n_spec and velocity by a plain reverse
    sweep (in ``oracle_c.c``).

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, limits, invariants, brute force or an independent library route.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

H = 6.62607015e-34
C = 299792458.0
KB = 1.380649e-23
SQRT_PI = math.sqrt(math.pi)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_c.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle_c.c into liboracle.so (gcc, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lib_lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.oracle_trace_lengths.argtypes = [i64, P, P, P, P, i32, P, i64, P, P, P]
            lib.oracle_trace_fill.argtypes = [i64, P, P, P, P, i32, P, i64, P, P, P]
            lib.oracle_planck.argtypes = [f64, f64]
            lib.oracle_planck.restype = f64
            lib.oracle_segment_dtau.argtypes = [f64] * 9
            lib.oracle_segment_dtau.restype = f64
            lib.oracle_feautrier_at.argtypes = [i64, P, P, f64, f64, i64, P, P]
            lib.oracle_formal_solve.argtypes = [i64, P, P, P, P, f64, i32, P, i32, P, P, P,
                                                i32, P, P, P, i32, P, P, f64, f64, f64, ctypes.c_int,
                                                ctypes.c_int, i64, P, P, P]
            lib.oracle_segment_dtau_subdiv.argtypes = [f64] * 7 + [ctypes.c_int]
            lib.oracle_segment_dtau_subdiv.restype = f64
            lib.oracle_image_weights.argtypes = [f64, P, P, P]
            lib.oracle_image_frame.argtypes = [i64, P, P, i32, i32, P, P, P]
            lib.oracle_image_rays.argtypes = [i64, P, P, P, P, P, i64, P, P, P, P, P, P]
            lib.oracle_image_solve.argtypes = [i64, P, P, P, P, f64, P, i32, P, P, P, f64, f64, i64, P, P,
                                               i32, P, P]
            lib.oracle_image_adjoint.argtypes = [i64, P, P, P, P, f64, P, i32, P, P, P, f64, f64, i64, P, P,
                                                 i32, P, P, P, P, P]
            lib.oracle_image_branches.argtypes = [i64, P, P, P, P, f64, P, i32, P, f64, i64, P, P, i32, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Radiation and quadrature
# --------------------------------------------------------------------------
def planck(nu, T):
    """B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1), SI."""
    nu = np.asarray(nu, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    with np.errstate(over="ignore", divide="ignore"):
        x = H * nu / (KB * np.where(T > 0, T, 1.0))
        out = 2.0 * H * nu ** 3 / C ** 2 / np.expm1(x)
    return np.where(T > 0, out, 0.0)


def gauss_hermite(Q: int):
    """Nodes x_q and weights normalised to sum 1 (w_q / sqrt(pi)) for the
    Gaussian line profile, so that sum_q w_q f(x_q) ~ int phi(nu) f dnu."""
    x, w = np.polynomial.hermite.hermgauss(Q)
    return x.astype(np.float64), (w / SQRT_PI).astype(np.float64)


def line_width(nu_ij, T, vturb2, mol_mass):
    """Sec. 4.3, eq. line width: dnu = nu_ij/c sqrt(2 k T / m + v_turb^2)."""
    return nu_ij / C * np.sqrt(2.0 * KB * T / mol_mass + vturb2)


def einstein_B(A, nu, g_u, g_l):
    """B_ul = A_ul c^2 / (2 h nu^3) (per unit J_nu), B_lu = (g_u/g_l) B_ul."""
    Bul = A * C ** 2 / (2.0 * H * nu ** 3)
    return Bul, Bul * g_u / g_l


# --------------------------------------------------------------------------
# Populations -> line opacity and source function
# --------------------------------------------------------------------------
def lte_populations(T, n_spec, energy, g):
    """Boltzmann populations over the model's levels (partition function
    truncated to those levels), [N][L]."""
    T = np.asarray(T, np.float64)[:, None]
    x = -(energy[None, :] - energy[0]) / (KB * T)
    w = g[None, :] * np.exp(x)
    return n_spec[:, None] * w / w.sum(axis=1, keepdims=True)


def line_chi_S(pops, lines):
    """chi^{ij} = (h nu/4 pi)(n_l B_lu - n_u B_ul) and S^{ij} = eta/chi with
    eta = (h nu/4 pi) n_u A_ul, both [M][N] in SI (chi in m^-1 Hz).

    Inverted or empty lines: the net (n_l B_lu - n_u B_ul) is floored at
    1e-30 (n_l B_lu + n_u B_ul); the number of floored entries is returned.
    """
    up, lo = lines.up, lines.lo
    nu = lines.freq_Hz
    Bul, Blu = einstein_B(lines.A, nu, lines.g[up], lines.g[lo])
    nu_ = pops[:, up].T      # [M][N]
    nl_ = pops[:, lo].T
    pref = (H * nu / (4.0 * math.pi))[:, None]
    a = nl_ * Blu[:, None]
    b = nu_ * Bul[:, None]
    net = a - b
    floor = 1e-30 * (a + b)
    clamped = net < floor
    net = np.where(clamped, floor, net)
    chi = pref * net
    eta = pref * nu_ * lines.A[:, None]
    with np.errstate(invalid="ignore", divide="ignore"):
        S = np.where(chi > 0, eta / np.where(chi > 0, chi, 1.0), 0.0)
    return chi, S, int(clamped.sum())


# --------------------------------------------------------------------------
# Directions and ray tracing
# --------------------------------------------------------------------------
def direction_pairs(dirs, tol=1e-12):
    """Antipodal pairs (r, rb), r < rb, with n_rb = -n_r; raises if unpaired."""
    R = dirs.shape[0]
    used = np.zeros(R, bool)
    pairs = []
    for r in range(R):
        if used[r]:
            continue
        d = np.linalg.norm(dirs + dirs[r][None, :], axis=1)
        d[r] = np.inf
        d[used] = np.inf
        rb = int(np.argmin(d))
        if d[rb] > tol:
            raise ValueError(f"direction {r} has no antipode")
        used[r] = used[rb] = True
        pairs.append((r, rb))
    return np.asarray(pairs, dtype=np.int32)


@dataclass
class Rays:
    off: np.ndarray     # [R*N+1] int64 exclusive prefix of half-ray lengths
    idx: np.ndarray     # [total] int32 point indices, origin excluded, outward order
    stalls: int
    N: int
    R: int
    stall: np.ndarray = None   # [R*N] uint8, 1 where the walk stalled

    def half(self, r, o):
        t = r * self.N + o
        return self.idx[self.off[t]:self.off[t + 1]]


def trace(model, origins=None) -> Rays:
    """Trace every half-ray of every origin (rule in oracle_c.c); with
    ``origins`` only those origins' half-rays (the others stay empty)."""
    lib = _load()
    N, R = model.n_points, model.dirs.shape[0]
    pos = np.ascontiguousarray(model.pos, np.float64)
    off = np.ascontiguousarray(model.nbr_offsets, np.int64)
    nb = np.ascontiguousarray(model.nbrs, np.int32)
    bnd = np.zeros(N, np.uint8)
    bnd[model.boundary] = 1
    dirs = np.ascontiguousarray(model.dirs, np.float64)
    lens = np.zeros(R * N, np.int64)
    stall = np.zeros(R * N, np.uint8)
    org = None if origins is None else np.ascontiguousarray(origins, np.int64)
    n_org = 0 if org is None else org.shape[0]
    lib.oracle_trace_lengths(N, _p(pos), _p(off), _p(nb), _p(bnd), R, _p(dirs), n_org,
                             None if org is None else _p(org), _p(lens), _p(stall))
    ray_off = np.zeros(R * N + 1, np.int64)
    np.cumsum(lens, out=ray_off[1:])
    idx = np.zeros(int(ray_off[-1]), np.int32)
    lib.oracle_trace_fill(N, _p(pos), _p(off), _p(nb), _p(bnd), R, _p(dirs), n_org,
                          None if org is None else _p(org), _p(ray_off), _p(idx))
    return Rays(ray_off, idx, int(stall.sum()), N, R, stall)


# --------------------------------------------------------------------------
# Segment optical depth and the two-point system (thin wrappers for tests)
# --------------------------------------------------------------------------
def segment_dtau(dx, chi0, chi1, dnu0, dnu1, dnubar, off0, off1, thr=0.35):
    return _load().oracle_segment_dtau(dx, chi0, chi1, dnu0, dnu1, dnubar, off0, off1, thr)


def segment_dtau_subdiv(dx, chi0, chi1, dnu0, dnu1, off0, off1, n):
    return _load().oracle_segment_dtau_subdiv(dx, chi0, chi1, dnu0, dnu1, off0, off1, n)


def feautrier_at(dtau, S, I_left, I_right, io):
    dtau = np.ascontiguousarray(dtau, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    u = ctypes.c_double()
    L = ctypes.c_double()
    _load().oracle_feautrier_at(S.shape[0], _p(dtau), _p(S), I_left, I_right, io,
                                ctypes.byref(u), ctypes.byref(L))
    return u.value, L.value


def formal_solve(model, rays: Rays, chi, S, origins=None, tau_min=1e-150, thr=0.35,
                 width_mode=0, subdiv=0):
    """J-bar and Lambda* ([n][M], SI) at ``origins`` (default: all points).
    ``subdiv`` > 0 replaces every segment's optical depth by the subdivided
    trapezoidal rule with that many pieces."""
    lib = _load()
    N = model.n_points
    pairs = direction_pairs(model.dirs)
    x, w = gauss_hermite(model.n_quad)
    origins = np.arange(N, dtype=np.int64) if origins is None else np.asarray(origins, np.int64)
    M = model.lines.n_lines
    J = np.zeros((origins.shape[0], M))
    L = np.zeros((origins.shape[0], M))
    arr = lambda a, t=np.float64: np.ascontiguousarray(a, t)
    pos, vel, T, vt2 = arr(model.pos), arr(model.vel), arr(model.temp), arr(model.vturb2)
    dirs, pr = arr(model.dirs), arr(pairs, np.int32)
    nu, chi_, S_ = arr(model.lines.freq_Hz), arr(chi), arr(S)
    lib.oracle_formal_solve(N, _p(pos), _p(vel), _p(T), _p(vt2), float(model.lines.mol_mass_kg),
                            model.dirs.shape[0], _p(dirs), pairs.shape[0], _p(pr),
                            _p(rays.off), _p(rays.idx), M, _p(nu), _p(chi_), _p(S_),
                            x.shape[0], _p(x), _p(w), float(model.T_bg), tau_min, thr, width_mode, int(subdiv),
                            origins.shape[0], _p(origins), _p(J), _p(L))
    return J, L


# --------------------------------------------------------------------------
# Statistical equilibrium
# --------------------------------------------------------------------------
def rate_matrix(pops_old, Jbar, Lstar, T, n_coll, n_spec, lines):
    """Per-point transition-rate matrices R[p, i, j] (rate i -> j, s^-1).

    Radiative, preconditioned with the diagonal approximate Lambda operator
    (Rybicki & Hummer 1991): with J_eff = Jbar - Lstar S_old,
      u -> l : A_ul (1 - Lstar) + B_ul J_eff,   l -> u : B_lu J_eff,
    each floored at 0 (both are non-negative in exact arithmetic, since the
    formal solution gives Jbar >= Lstar S_o and 0 < Lstar < 1).
    Collisional: C_ul = n_coll K_ul, C_lu = C_ul (g_u/g_l) exp(-(E_u-E_l)/kT).
    Jbar, Lstar are [N][M].
    """
    N, L = pops_old.shape
    _, S_old, _ = line_chi_S(pops_old, lines)
    S_old = S_old.T                       # [N][M]
    Bul, Blu = einstein_B(lines.A, lines.freq_Hz, lines.g[lines.up], lines.g[lines.lo])
    Jeff = Jbar - Lstar * S_old
    R = np.zeros((N, L, L))
    for k in range(lines.n_lines):
        u, l = lines.up[k], lines.lo[k]
        R[:, u, l] += np.maximum(lines.A[k] * (1.0 - Lstar[:, k]) + Bul[k] * Jeff[:, k], 0.0)
        R[:, l, u] += np.maximum(Blu[k] * Jeff[:, k], 0.0)
    for k in range(lines.cup.shape[0]):
        u, l = lines.cup[k], lines.clo[k]
        Cul = n_coll * lines.K_ul[k]
        Clu = Cul * lines.g[u] / lines.g[l] * np.exp(-(lines.energy_J[u] - lines.energy_J[l]) / (KB * T))
        R[:, u, l] += Cul
        R[:, l, u] += Clu
    return R


def stat_equilibrium(pops_old, Jbar, Lstar, T, n_coll, n_spec, lines):
    """New populations [N][L] from the steady state of the rate equations,
    sum_j n_j R_ji = n_i sum_j R_ij, normalised to sum_i n_i = n_spec.

    Solved by state reduction (Grassmann, Taksar & Heyman 1985): levels are
    eliminated from the top, the rates among the remaining levels gaining the
    paths through the eliminated one, R_ij += R_in R_nj / S_n with
    S_n = sum_{j<n} R_nj; then n_0 = 1, n_k = sum_{i<k} n_i R_ik / S_k, and a
    final normalisation.  Only sums and products of non-negative numbers
    occur, so even populations of order 1e-60 keep full relative accuracy
    (a dense LU on the same equations does not).
    """
    R = rate_matrix(pops_old, Jbar, Lstar, T, n_coll, n_spec, lines)
    N, L = pops_old.shape
    idx = np.arange(L)
    R[:, idx, idx] = 0.0
    S = np.zeros((N, L))
    for n in range(L - 1, 0, -1):
        s = R[:, n, :n].sum(axis=1)
        s = np.where(s > 0.0, s, 1e-300)
        S[:, n] = s
        R[:, :n, :n] += R[:, :n, n][:, :, None] * (R[:, n, :n] / s[:, None])[:, None, :]
    x = np.zeros((N, L))
    x[:, 0] = 1.0
    for n in range(1, L):
        x[:, n] = np.sum(x[:, :n] * R[:, :n, n], axis=1) / S[:, n]
    return x / x.sum(axis=1, keepdims=True) * n_spec[:, None]


def stat_equilibrium_dense(pops_old, Jbar, Lstar, T, n_coll, n_spec, lines):
    """The same equations with the last balance row replaced by the
    conservation row, solved by dense LU with partial pivoting
    (numpy.linalg.solve).  Accurate only when no population is tiny; kept as
    an independent route for the tests."""
    R = rate_matrix(pops_old, Jbar, Lstar, T, n_coll, n_spec, lines)
    N, L = pops_old.shape
    idx = np.arange(L)
    R[:, idx, idx] = 0.0
    Mt = np.transpose(R, (0, 2, 1)).copy()            # Mt[p, i, j] = R[p, j, i]
    Mt[:, idx, idx] = -R.sum(axis=2)
    Mt[:, L - 1, :] = 1.0
    rhs = np.zeros((N, L))
    rhs[:, L - 1] = n_spec
    return np.linalg.solve(Mt, rhs[:, :, None])[:, :, 0]


# --------------------------------------------------------------------------
# Ng-acceleration (Sec. 4.2 and Appendix A)
# --------------------------------------------------------------------------
def maxrel(a, b):
    """Maximum relative change max |a - b| / |b| over entries with b != 0."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    m = b != 0
    if not m.any():
        return 0.0
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def ng_coefficients(iterates):
    """c = (R R^T)^-1 1 / (1^T (R R^T)^-1 1) from the residuals of the given
    iterates (oldest first): r_k = x_{k+1} - x_k, k = 1..N-1.

    Near convergence the Gram matrix R R^T is close to singular (an exact
    combination of the residuals is a null vector), and the normalised
    coefficients stay well defined in that limit; so the Gram matrix (scaled
    by its trace) is solved by LU with partial pivoting and only a solve that
    is not finite (an exactly singular matrix) is rejected, returning None.
    """
    X = np.asarray(iterates, dtype=np.float64)
    Rm = X[1:] - X[:-1]
    G = Rm @ Rm.T
    n = G.shape[0]
    tr = np.trace(G)
    if not np.isfinite(tr) or tr <= 0.0:
        return None
    try:
        y = np.linalg.solve(G / tr, np.ones(n))
    except np.linalg.LinAlgError:
        return None
    s = y.sum()
    if not np.all(np.isfinite(y)) or s == 0.0 or not np.isfinite(s):
        return None
    c = y / s
    if not np.all(np.isfinite(c)):
        return None
    return c


def ng_predict(iterates):
    """Ng prediction sum_k c_k x_{k+1}: the coefficients applied to the images
    of the inputs (the newest N-1 iterates)."""
    c = ng_coefficients(iterates)
    if c is None:
        return None
    X = np.asarray(iterates, dtype=np.float64)
    return c @ X[1:]


class NgClassical:
    """Fixed N_steps: after N_steps regular iterations since the last reset,
    the prediction from all iterates replaces the newest one."""

    def __init__(self, n_steps=4):
        self.n_steps = n_steps
        self.hist = []

    def reset(self, x):
        self.hist = [np.array(x, dtype=np.float64)]

    def push(self, x):
        self.hist.append(np.array(x, dtype=np.float64))
        if len(self.hist) < self.n_steps + 1:
            return x, False
        pred = ng_predict(self.hist)
        ok = pred is not None and np.all(pred >= 0)
        out = pred if ok else x
        self.reset(out)
        return out, ok


class NgAdaptive:
    """Adaptive Ng (Sec. 4.2): after each regular iteration with m >= 3
    iterates since the last prediction was used, compute the running
    prediction P_m from all of them; use it when max-rel-change(P_m, P_{m-1})
    < max-rel-change(x_m, x_{m-1}) (P_2 := x_2), or unconditionally once m
    reaches N_max.  A prediction chosen for use but holding a negative
    population is not used and the history restarts from x_m; an exactly
    singular Gram matrix restarts it too."""

    def __init__(self, n_max=8):
        self.n_max = n_max
        self.hist = []
        self.prev_pred = None

    def reset(self, x):
        self.hist = [np.array(x, dtype=np.float64)]
        self.prev_pred = None

    def push(self, x):
        self.hist.append(np.array(x, dtype=np.float64))
        m = len(self.hist)
        if m == 2:
            self.prev_pred = self.hist[1]
            return x, False
        if m < 3:
            return x, False
        pred = ng_predict(self.hist)
        if pred is None:
            self.reset(x)
            return x, False
        use = maxrel(pred, self.prev_pred) < maxrel(self.hist[-1], self.hist[-2]) or m >= self.n_max
        if use:
            if not np.all(pred >= 0):
                self.reset(x)
                return x, False
            self.reset(pred)
            return pred, True
        self.prev_pred = pred
        return x, False


# --------------------------------------------------------------------------
# Accelerated Lambda iteration
# --------------------------------------------------------------------------
def ali_solve(model, rays=None, n_iter=20, ng=None, pops0=None, tau_min=1e-150, thr=0.35,
              callback=None):
    """LTE start (or pops0), then n_iter regular iterations of
    {chi,S from pops -> formal solution (Jbar, Lstar) -> statistical equilibrium
    -> optional Ng step}.  Ng works on fractional populations n_i / n_spec.
    Returns (pops [N][L], history of per-iteration max relative change)."""
    lines = model.lines
    if rays is None:
        rays = trace(model)
    pops = lte_populations(model.temp, model.n_spec, lines.energy_J, lines.g) if pops0 is None \
        else np.array(pops0, dtype=np.float64)
    frac = lambda p: (p / model.n_spec[:, None]).ravel()
    unfrac = lambda x: x.reshape(pops.shape) * model.n_spec[:, None]
    if ng is not None:
        ng.reset(frac(pops))
    changes = []
    for it in range(n_iter):
        chi, S, _ = line_chi_S(pops, lines)
        J, L = formal_solve(model, rays, chi, S, tau_min=tau_min, thr=thr)
        new = stat_equilibrium(pops, J, L, model.temp, model.n_coll, model.n_spec, lines)
        changes.append(maxrel(new, pops))
        if ng is not None:
            x, acc = ng.push(frac(new))
            if acc:
                new = unfrac(x)
        pops = new
        if callback is not None:
            callback(it, pops)
    return pops, changes


# --------------------------------------------------------------------------
# Synthetic image (Listing 3, compute_image_new), readings in oracle_c.c
# --------------------------------------------------------------------------
def image_weights(t):
    """(e^-t, w0, w1) of the piecewise-linear source update over depth t."""
    E, w0, w1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().oracle_image_weights(t, ctypes.byref(E), ctypes.byref(w0), ctypes.byref(w1))
    return E.value, w0.value, w1.value


def image_frequencies(nfreq, fmin, fmax):
    """Channel frequencies: nfreq points from fmin to fmax inclusive
    (compute_spectral_discretisation(fmin, fmax, N)); one channel is fmin."""
    if nfreq == 1:
        return np.array([float(fmin)])
    return fmin + np.arange(nfreq, dtype=np.float64) * ((fmax - fmin) / (nfreq - 1))


@dataclass
class ImageRays:
    ref: np.ndarray      # [npix][3] pixel reference points (image plane through the model)
    anchor: np.ndarray   # [npix] point closest to each pixel line
    off: np.ndarray      # [npix+1] offsets of the full rays in pts
    pts: np.ndarray      # full rays, far end first
    e1: np.ndarray
    e2: np.ndarray


def image_rays(model, direction, npx, npy) -> ImageRays:
    lib = _load()
    N = model.n_points
    n = np.ascontiguousarray(direction, np.float64)
    pos = np.ascontiguousarray(model.pos, np.float64)
    e1, e2 = np.zeros(3), np.zeros(3)
    npix = npx * npy
    ref = np.zeros((npix, 3))
    lib.oracle_image_frame(N, _p(pos), _p(n), npx, npy, _p(e1), _p(e2), _p(ref))
    off = np.ascontiguousarray(model.nbr_offsets, np.int64)
    nb = np.ascontiguousarray(model.nbrs, np.int32)
    bnd = np.zeros(N, np.uint8)
    bnd[model.boundary] = 1
    anchor = np.zeros(npix, np.int32)
    nfar = np.zeros(npix, np.int64)
    nnear = np.zeros(npix, np.int64)
    lib.oracle_image_rays(N, _p(pos), _p(off), _p(nb), _p(bnd), _p(n), npix, _p(ref), _p(anchor), _p(nfar),
                          _p(nnear), None, None)
    ray_off = np.zeros(npix + 1, np.int64)
    np.cumsum(nfar + nnear + 1, out=ray_off[1:])
    pts = np.zeros(int(ray_off[-1]), np.int32)
    lib.oracle_image_rays(N, _p(pos), _p(off), _p(nb), _p(bnd), _p(n), npix, _p(ref), _p(anchor), _p(nfar),
                          _p(nnear), _p(ray_off), _p(pts))
    return ImageRays(ref, anchor, ray_off, pts, e1, e2)


def image(model, pops, direction, npx, npy, nfreq, fmin, fmax, thr=0.35, rays=None):
    """Intensity toward the observer [nfreq][npy][npx] (W m^-2 Hz^-1 sr^-1)
    from the level populations ``pops`` [N][L]; each channel uses the line
    nearest to it.  Returns (image, rays)."""
    lib = _load()
    if rays is None:
        rays = image_rays(model, direction, npx, npy)
    chi, S, _ = line_chi_S(pops, model.lines)
    nu_f = image_frequencies(nfreq, fmin, fmax)
    arr = lambda a, t=np.float64: np.ascontiguousarray(a, t)
    npix = npx * npy
    out = np.zeros((nfreq, npix))
    lib.oracle_image_solve(model.n_points, _p(arr(model.pos)), _p(arr(model.vel)), _p(arr(model.temp)),
                           _p(arr(model.vturb2)), float(model.lines.mol_mass_kg), _p(arr(direction)),
                           model.lines.n_lines, _p(arr(model.lines.freq_Hz)), _p(arr(chi)), _p(arr(S)),
                           float(model.T_bg), thr, npix, _p(rays.off), _p(rays.pts), nfreq, _p(nu_f), _p(out))
    return out.reshape(nfreq, npy, npx), rays


# --------------------------------------------------------------------------
# Recursive re-meshing (Sec. 4.1)
# --------------------------------------------------------------------------
def box_variation(rho):
    """Sec. 4.1, eq. subdivision criterion: 2 (rho_max - rho_min) / (rho_max + rho_min)."""
    rmax, rmin = float(np.max(rho)), float(np.min(rho))
    return 2.0 * ((rmax - rmin) / (rmax + rmin))


def remesh(pos, rho, r_max, max_level, n_side):
    """Recursive re-meshing of a point cloud with tracer rho (Sec. 4.1).

    Start from the bounding box of all points.  A box whose variation exceeds
    r_max, below level max_level, is divided into 8 equal boxes (a point goes
    to the upper half of an axis when its coordinate is >= the midpoint); each
    non-empty part is cropped to the bounding box of its points and treated
    the same way.  Every other box becomes one point at its centre.  Then an
    evenly spaced set of boundary points is added on the surface of the
    outermost box: the n_side^3 lattice over it, surface nodes only.

    Returns (points [K][3], boundary flags [K], leaves) with leaves a list of
    (lo, hi, level, member indices), in depth-first order, children in octant
    order (bit d set for the upper half of axis d).
    """
    pos = np.asarray(pos, np.float64)
    rho = np.asarray(rho, np.float64)
    leaves = []
    stack = [(np.arange(pos.shape[0]), 0)]
    root_lo, root_hi = pos.min(axis=0), pos.max(axis=0)
    while stack:
        idx, level = stack.pop()
        p = pos[idx]
        lo, hi = p.min(axis=0), p.max(axis=0)
        if level < max_level and box_variation(rho[idx]) > r_max:
            mid = (lo + hi) * 0.5
            octant = ((p[:, 0] >= mid[0]).astype(int) | ((p[:, 1] >= mid[1]).astype(int) << 1)
                      | ((p[:, 2] >= mid[2]).astype(int) << 2))
            for o in range(7, -1, -1):          # pushed in reverse: popped in octant order
                sel = idx[octant == o]
                if sel.size:
                    stack.append((sel, level + 1))
        else:
            leaves.append((lo, hi, level, idx))
    inner = np.array([(lo + hi) * 0.5 for lo, hi, _, _ in leaves]).reshape(-1, 3)
    g = np.arange(n_side)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    on = (I == 0) | (I == n_side - 1) | (J == 0) | (J == n_side - 1) | (K == 0) | (K == n_side - 1)
    lat = np.stack([I[on], J[on], K[on]], axis=1).astype(np.float64)
    bnd = root_lo + lat / (n_side - 1) * (root_hi - root_lo)
    pts = np.concatenate([inner, bnd], axis=0)
    flags = np.concatenate([np.zeros(inner.shape[0], np.uint8), np.ones(bnd.shape[0], np.uint8)])
    return pts, flags, leaves


def image_adjoint(model, pops, direction, npx, npy, nfreq, fmin, fmax, gimg, thr=0.35, rays=None):
    """Gradient of L = sum(gimg * image) with respect to every point's log T,
    log n_spec and velocity, from a plain FP64 reverse sweep of the image solve
    (each segment's branch held; populations held as fractions of n_spec).
    Returns (g_logT [N], g_logn [N], g_v [N][3]); g_v is along the line of sight,
    the only velocity component the image depends on."""
    lib = _load()
    if rays is None:
        rays = image_rays(model, direction, npx, npy)
    chi, S, _ = line_chi_S(pops, model.lines)
    nu_f = image_frequencies(nfreq, fmin, fmax)
    arr = lambda a, t=np.float64: np.ascontiguousarray(a, t)
    N = model.n_points
    g = arr(np.asarray(gimg, np.float64).reshape(nfreq, npx * npy))
    gT, gn, gl = np.zeros(N), np.zeros(N), np.zeros(N)
    d = arr(direction)
    lib.oracle_image_adjoint(N, _p(arr(model.pos)), _p(arr(model.vel)), _p(arr(model.temp)), _p(arr(model.vturb2)),
                             float(model.lines.mol_mass_kg), _p(d), model.lines.n_lines, _p(arr(model.lines.freq_Hz)),
                             _p(arr(chi)), _p(arr(S)), float(model.T_bg), thr, npx * npy, _p(rays.off), _p(rays.pts),
                             nfreq, _p(nu_f), _p(g), _p(gT), _p(gn), _p(gl))
    return gT, gn, gl[:, None] * d[None, :]


def image_branches(model, direction, nfreq, fmin, fmax, rays, thr=0.35):
    """Branch of every segment of every (channel, pixel ray) of the image solve,
    [nfreq][segments], 1 = trapezoid, 0 = semi-analytic."""
    lib = _load()
    nu_f = image_frequencies(nfreq, fmin, fmax)
    arr = lambda a, t=np.float64: np.ascontiguousarray(a, t)
    npix = rays.off.shape[0] - 1
    n_seg = int(rays.off[-1]) - npix
    out = np.zeros((nfreq, n_seg), np.uint8)
    lib.oracle_image_branches(model.n_points, _p(arr(model.pos)), _p(arr(model.vel)), _p(arr(model.temp)),
                              _p(arr(model.vturb2)), float(model.lines.mol_mass_kg), _p(arr(direction)),
                              model.lines.n_lines, _p(arr(model.lines.freq_Hz)), thr, npix, _p(rays.off),
                              _p(rays.pts), nfreq, _p(nu_f), _p(out))
    return out
