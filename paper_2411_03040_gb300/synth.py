"""Seeded synthetic models shaped like the workloads of Magritte (arXiv 2411.03040).

This module only *generates inputs*: point clouds, neighbour graphs, boundary
lists, ray directions, a synthetic linear-rotor line list and the physical
fields (velocity, temperature, densities, turbulence).  It holds none of the
line-transfer arithmetic (no opacities, no optical depths, no formal solution,
no level populations): both the CUDA library and the CPU oracle receive its
arrays as plain inputs.

The model fields follow the constructor calls of the paper's Listing 2
(Sec. 3.2): positions, velocities, neighbours (flat list + counts), boundary
points, temperature, turbulence, species abundances, uniform rays, line data
and a quadrature order.

Units are SI throughout.  One model "length unit" is 1e13 cm = 1e11 m.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants used only to build line data (CODATA 2018, exact where defined).
_H = 6.62607015e-34        # J s
_C = 299792458.0           # m/s
_AMU = 1.66053906660e-27   # kg
_DEBYE_CGS = 1e-18         # esu cm
_H_CGS = 6.62607015e-27    # erg s
_C_CGS = 2.99792458e10     # cm/s

LENGTH_UNIT_M = 1e11       # 1e13 cm
SEED_BASE = 2411030400


# --------------------------------------------------------------------------
# Directions: HEALPix pixel centres (Gorski et al. 2005, ring scheme)
# --------------------------------------------------------------------------
def healpix_directions(nside: int) -> np.ndarray:
    """Unit vectors of the 12*nside^2 HEALPix pixel centres (ring scheme).

    Ring i = 1 .. 4*nside-1 from the north pole.  Polar-cap rings (i < nside)
    hold 4i pixels at z = 1 - i^2/(3 nside^2), phi = pi/(2i) (j - 1/2); belt
    rings (nside <= i <= 3 nside) hold 4 nside pixels at
    z = 4/3 - 2i/(3 nside), phi = pi/(2 nside) (j - s/2) with
    s = (i - nside + 1) mod 2; southern rings mirror the northern ones.
    The set is antipodally symmetric, so directions come in exact pairs.
    """
    if nside < 1:
        raise ValueError("nside must be >= 1")
    out = []
    for i in range(1, 4 * nside):
        if i < nside:
            z = 1.0 - i * i / (3.0 * nside * nside)
            phis = [math.pi / (2 * i) * (j - 0.5) for j in range(1, 4 * i + 1)]
        elif i <= 3 * nside:
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            s = (i - nside + 1) % 2
            phis = [math.pi / (2 * nside) * (j - s / 2.0) for j in range(1, 4 * nside + 1)]
        else:
            ip = 4 * nside - i
            z = -(1.0 - ip * ip / (3.0 * nside * nside))
            phis = [math.pi / (2 * ip) * (j - 0.5) for j in range(1, 4 * ip + 1)]
        st = math.sqrt(max(0.0, (1.0 - z) * (1.0 + z)))
        for ph in phis:
            out.append((st * math.cos(ph), st * math.sin(ph), z))
    d = np.asarray(out, dtype=np.float64)
    assert d.shape[0] == 12 * nside * nside
    return d


# --------------------------------------------------------------------------
# Line data: synthetic linear rotor (LAMDA-like)
# --------------------------------------------------------------------------
@dataclass
class LineData:
    n_levels: int
    energy_J: np.ndarray      # [L]
    g: np.ndarray             # [L]
    up: np.ndarray            # [M] int32 upper level of each radiative line
    lo: np.ndarray            # [M] int32
    A: np.ndarray             # [M] s^-1
    freq_Hz: np.ndarray       # [M]
    cup: np.ndarray           # [K] int32 collisional upper level
    clo: np.ndarray           # [K] int32
    K_ul: np.ndarray          # [K] m^3/s downward rate coefficient
    mol_mass_kg: float = 28.0 * _AMU

    @property
    def n_lines(self) -> int:
        return int(self.up.shape[0])


def linear_rotor(n_levels: int, rng: np.random.Generator, B_Hz: float = 57.6e9,
                 mu_debye: float = 0.11, mass_amu: float = 28.0,
                 k_range_cm3: tuple[float, float] = (1e-11, 1e-10)) -> LineData:
    """Rigid linear rotor: E_J = h B J(J+1), g_J = 2J+1, lines J -> J-1 at 2BJ.

    Spontaneous rates from the dipole formula (cgs)
    A = 64 pi^4 nu^3 mu^2 / (3 h c^3) * J/(2J+1).  Collision rate
    coefficients are drawn log-uniformly in ``k_range_cm3`` for every level
    pair u > l and converted to m^3/s.
    """
    J = np.arange(n_levels, dtype=np.float64)
    E = _H * B_Hz * J * (J + 1.0)
    g = 2.0 * J + 1.0
    up = np.arange(1, n_levels, dtype=np.int32)
    lo = up - 1
    nu = 2.0 * B_Hz * up.astype(np.float64)
    mu = mu_debye * _DEBYE_CGS
    Ju = up.astype(np.float64)
    A = 64.0 * math.pi ** 4 * nu ** 3 * mu * mu / (3.0 * _H_CGS * _C_CGS ** 3) * Ju / (2.0 * Ju + 1.0)
    cu, cl = [], []
    for u in range(1, n_levels):
        for l in range(u):
            cu.append(u)
            cl.append(l)
    cup = np.asarray(cu, dtype=np.int32)
    clo = np.asarray(cl, dtype=np.int32)
    lo_k, hi_k = np.log(k_range_cm3[0]), np.log(k_range_cm3[1])
    K = np.exp(rng.uniform(lo_k, hi_k, size=cup.shape[0])) * 1e-6
    return LineData(n_levels, E, g, up, lo, A, nu, cup, clo, K, mass_amu * _AMU)


# --------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------
def delaunay_graph(pos: np.ndarray):
    """Neighbour graph (CSR) of the Delaunay tetrahedralisation + hull vertices."""
    from scipy.spatial import Delaunay
    tri = Delaunay(pos)
    indptr, indices = tri.vertex_neighbor_vertices
    hull = np.unique(tri.convex_hull.ravel()).astype(np.int32)
    off = np.asarray(indptr, dtype=np.int64)
    nb = np.asarray(indices, dtype=np.int32)
    # sort each neighbour list (deterministic, independent of qhull's order)
    row = np.repeat(np.arange(pos.shape[0], dtype=np.int64), np.diff(off))
    nb = nb[np.lexsort((nb, row))]
    return off, nb, hull


def grf_velocity(pos_units: np.ndarray, sigma_ms: float, ell_units: float,
                 rng: np.random.Generator, n_modes: int = 512) -> np.ndarray:
    """Gaussian random velocity field from random Fourier features.

    v_i(x) = sigma sqrt(2/M) sum_k a_ik cos(w_k . x + p_k) with w_k ~ N(0, I/ell^2),
    a ~ N(0, 1), p ~ U(0, 2 pi): each component has variance sigma^2 and a
    Gaussian correlation exp(-|dx|^2 / (2 ell^2)) (Rahimi & Recht 2007).
    """
    w = rng.normal(size=(n_modes, 3)) / ell_units
    a = rng.normal(size=(3, n_modes))
    p = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    out = np.empty_like(pos_units)
    chunk = 65536
    for s in range(0, pos_units.shape[0], chunk):
        ph = np.cos(pos_units[s:s + chunk] @ w.T + p)     # [n, M]
        out[s:s + chunk] = ph @ a.T
    return out * sigma_ms * math.sqrt(2.0 / n_modes)


@dataclass
class Model:
    """All inputs of one synthetic model, in SI units."""
    name: str
    pos: np.ndarray           # [N,3] m
    vel: np.ndarray           # [N,3] m/s
    temp: np.ndarray          # [N] K
    vturb2: np.ndarray        # [N] m^2/s^2
    n_coll: np.ndarray        # [N] m^-3 (H2)
    n_spec: np.ndarray        # [N] m^-3 (line species)
    nbr_offsets: np.ndarray   # [N+1] int64
    nbrs: np.ndarray          # [nnz] int32
    boundary: np.ndarray      # [B] int32
    dirs: np.ndarray          # [R,3]
    n_quad: int
    lines: LineData
    T_bg: float = 2.725
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return int(self.pos.shape[0])


def _outflow_fields(r_units: np.ndarray, rhat: np.ndarray, v_inf=15e3, r_floor=0.2,
                    T0=2000.0, nH0_cm3=1e10, abundance=3e-4, vturb=1e3):
    re = np.maximum(r_units, r_floor)
    v = v_inf * (1.0 - 0.2 / re)
    vel = rhat * v[:, None]
    T = T0 * re ** -0.7
    nH2 = nH0_cm3 * re ** -2 * 1e6
    return vel, T, np.full_like(T, vturb * vturb), nH2, abundance * nH2


def sphere_model(n_points=2000, n_levels=5, nside=1, n_quad=31, seed=None,
                 name="sphere") -> Model:
    """Uniform-random points in a unit sphere with a radial outflow.

    v(r) = 15 km/s (1 - 0.2/r), T = 2000 K r^-0.7, n_H2 = 1e10 cm^-3 r^-2,
    abundance 3e-4, turbulence 1 km/s; the laws are evaluated at max(r, 0.2).
    Delaunay neighbours; the convex-hull vertices are the boundary.
    """
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    # uniform in the unit ball: direction * U^(1/3)
    d = rng.normal(size=(n_points, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = rng.uniform(0.0, 1.0, size=n_points) ** (1.0 / 3.0)
    pu = d * r[:, None]
    off, nb, hull = delaunay_graph(pu)
    rr = np.linalg.norm(pu, axis=1)
    rhat = pu / np.maximum(rr, 1e-300)[:, None]
    vel, T, vt2, nH2, ns = _outflow_fields(rr, rhat)
    lines = linear_rotor(n_levels, rng)
    return Model(name, pu * LENGTH_UNIT_M, vel, T, vt2, nH2, ns, off, nb, hull,
                 healpix_directions(nside), n_quad, lines)


def shell_model(n_points=100_000, n_levels=41, nside=2, n_quad=50, r_in=1.0, r_out=100.0,
                grf_sigma=0.0, grf_ell=0.05, seed=None, name="shells") -> Model:
    """AGB-wind-like outflow on log-spaced radial shells with random angles.

    Equal point counts per shell in ln r; the innermost and outermost shells
    (and every convex-hull vertex) are boundary points.  Optionally adds a
    Gaussian random velocity field of rms ``grf_sigma`` per component.
    """
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    ln_lo, ln_hi = math.log(r_in), math.log(r_out)
    # shell thickness comparable to the mean point spacing (in ln r)
    spacing = (4.0 * math.pi * (ln_hi - ln_lo) / n_points) ** (1.0 / 3.0)
    n_shells = max(3, int(round((ln_hi - ln_lo) / spacing)))
    shell = np.arange(n_points) % n_shells
    edges = np.linspace(ln_lo, ln_hi, n_shells + 1)
    lnr = edges[shell] + rng.uniform(0.0, 1.0, size=n_points) * (edges[1] - edges[0])
    r = np.exp(lnr)
    d = rng.normal(size=(n_points, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pu = d * r[:, None]
    off, nb, hull = delaunay_graph(pu)
    bnd = np.union1d(hull, np.nonzero((shell == 0) | (shell == n_shells - 1))[0]).astype(np.int32)
    vel, T, vt2, nH2, ns = _outflow_fields(r, d)
    if grf_sigma > 0.0:
        vel = vel + grf_velocity(pu, grf_sigma, grf_ell, rng)
    lines = linear_rotor(n_levels, rng)
    return Model(name, pu * LENGTH_UNIT_M, vel, T, vt2, nH2, ns, off, nb, bnd,
                 healpix_directions(nside), n_quad, lines,
                 meta={"n_shells": n_shells})


def lattice_model(n_side=9, spacing_m=1e11, n_levels=2, n_quad=11, temp=100.0,
                  n_spec=1.0, n_coll=1e12, dirs=None, seed=0, name="lattice") -> Model:
    """Static uniform cubic lattice with a 6-neighbour graph; faces are boundary.

    A test geometry: with axis-aligned directions a ray walks straight along a
    lattice line to the face, so path lengths are known in closed form.
    """
    rng = np.random.default_rng(seed)
    ax = np.arange(n_side, dtype=np.float64) - (n_side - 1) / 2.0
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    pu = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    N = pu.shape[0]
    idx = np.arange(N).reshape(n_side, n_side, n_side)
    nbl = [[] for _ in range(N)]
    for axis in range(3):
        for sgn in (-1, 1):
            sh = np.roll(idx, -sgn, axis=axis)
            valid = np.ones_like(idx, dtype=bool)
            sl = [slice(None)] * 3
            sl[axis] = slice(n_side - 1, None) if sgn == 1 else slice(0, 1)
            valid[tuple(sl)] = False
            for a, b in zip(idx[valid].ravel(), sh[valid].ravel()):
                nbl[a].append(b)
    off = np.zeros(N + 1, dtype=np.int64)
    for i in range(N):
        off[i + 1] = off[i] + len(nbl[i])
    nb = np.concatenate([np.sort(np.asarray(v, dtype=np.int32)) for v in nbl]).astype(np.int32)
    face = np.nonzero(np.any(np.abs(pu) == (n_side - 1) / 2.0, axis=1))[0].astype(np.int32)
    if dirs is None:
        dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                        dtype=np.float64)
    lines = linear_rotor(n_levels, rng)
    return Model(name, pu * spacing_m, np.zeros_like(pu), np.full(N, temp), np.zeros(N),
                 np.full(N, n_coll), np.full(N, n_spec), off, nb, face, np.asarray(dirs, np.float64),
                 n_quad, lines)


# --------------------------------------------------------------------------
# Batches of uneven models
# --------------------------------------------------------------------------
def batch_specs(n_models=256, n_min=5_000, n_max=200_000, levels=(5, 11, 21, 41), nsides=(1, 2), n_quad=31,
                seed=None):
    """Seeded sizes of a batch of independent sphere models: point counts
    log-uniform in [n_min, n_max], level counts drawn from ``levels``, HEALPix
    nside from ``nsides`` (12 or 48 rays).  Returns (points, levels, nside,
    bins, seed) tuples; ``batch_model`` builds one."""
    rng = np.random.default_rng(SEED_BASE + 40 if seed is None else seed)
    n = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_models)).astype(np.int64)
    lv = rng.choice(np.asarray(levels), size=n_models)
    ns = rng.choice(np.asarray(nsides), size=n_models)
    base = int(rng.integers(1 << 30))
    return [(int(n[i]), int(lv[i]), int(ns[i]), int(n_quad), base + i) for i in range(n_models)]


def batch_model(spec) -> Model:
    n, L, nside, q, seed = spec
    return sphere_model(n, L, nside, q, seed=seed, name=f"sphere-{n}-L{L}-R{12 * nside * nside}")


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------
def config_model(index: int, n_points: int | None = None) -> Model:
    """Workload ``index`` (1-based):

    1: 2,000-point sphere, 5-level rotor, 12 rays, 31 bins per line.
    2: 100k-point shell outflow, 41 levels, 48 rays, 50 bins per line.
    3: 1M-point shell outflow + random velocity field (5 km/s, 0.05), 41 levels,
       192 rays, 40 bins per line.
    ``n_points`` overrides the size (same laws) for small test variants.
    """
    seed = SEED_BASE + index
    if index == 1:
        return sphere_model(n_points or 2000, 5, 1, 31, seed=seed, name="sphere-2k")
    if index == 2:
        n = n_points or 100_000
        return shell_model(n, 41, 2, 50, seed=seed, name=f"shells-{n}")
    if index == 3:
        n = n_points or 1_000_000
        return shell_model(n, 41, 4, 40, grf_sigma=5e3, grf_ell=0.05, seed=seed,
                           name=f"shells-grf-{n}")
    raise ValueError(f"unknown workload {index}")
