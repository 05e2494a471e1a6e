"""Pins of the oracle's synthetic image (Listing 3, compute_image_new) on the CPU.

Each pin is independent of the oracle's own expressions: closed forms for a
uniform static column, a numerical quadrature of the piecewise-linear source
update, a brute-force anchor search, the Doppler shift of a uniformly moving
model, and the geometry of the image frame.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2411_03040_gb300 import synth


def _lattice(n_side=7, temp=80.0, n_spec=1e-2, v=(0.0, 0.0, 0.0)):
    m = synth.lattice_model(n_side=n_side, n_levels=3, temp=temp, n_spec=n_spec, n_coll=1e12)
    m.vel = np.tile(np.asarray(v, np.float64), (m.n_points, 1))
    return m


def test_frame_is_orthonormal_and_pixels_lie_in_the_plane():
    m = synth.config_model(1, n_points=300)
    n = np.array([0.2, 0.9, -0.4])
    n /= np.linalg.norm(n)
    r = O.image_rays(m, n, 5, 4)
    for v in (r.e1, r.e2):
        assert abs(np.linalg.norm(v) - 1.0) < 1e-15
    assert abs(r.e1 @ n) < 1e-15 and abs(r.e2 @ n) < 1e-15 and abs(r.e1 @ r.e2) < 1e-15
    assert np.allclose(np.cross(n, r.e1), r.e2, atol=1e-15)
    assert np.max(np.abs(r.ref @ n)) < 1e-3 * np.max(np.abs(m.pos))
    # pixel spacing: uniform and square grid
    g = r.ref.reshape(4, 5, 3)
    d1 = np.diff(g @ r.e1, axis=1)
    d2 = np.diff(g @ r.e2, axis=0)
    assert np.allclose(d1, d1[0, 0], rtol=1e-9) and np.allclose(d2, d2[0, 0], rtol=1e-9)


def test_anchor_is_the_closest_point_and_rays_are_monotone():
    m = synth.config_model(1, n_points=400)
    n = np.array([0.6, 0.0, 0.8])
    r = O.image_rays(m, n, 6, 6)
    for q in range(36):
        p = r.ref[q]
        d = np.linalg.norm(np.cross(m.pos - p, n), axis=1)      # an independent distance formula
        assert d[r.anchor[q]] <= d.min() * (1 + 1e-9)
        ray = r.pts[r.off[q]:r.off[q + 1]]
        assert r.anchor[q] in ray
        Z = (m.pos[ray] - p) @ n
        assert np.all(np.diff(Z) > 0)


def test_weights_match_quadrature_of_a_linear_source():
    for t in (1e-6, 1e-3 * 0.7, 2e-3, 0.3, 1.0, 7.5):
        E, w0, w1 = O.image_weights(t)
        assert abs(E - math.exp(-t)) < 1e-15
        # I(t) for I(0) = 0 and S linear from S0 = 1 to S1 = 0 (and 0 -> 1)
        f0 = integrate.quad(lambda s: (1 - s / t) * math.exp(-(t - s)), 0, t, epsabs=0, epsrel=1e-13)[0]
        f1 = integrate.quad(lambda s: (s / t) * math.exp(-(t - s)), 0, t, epsabs=0, epsrel=1e-13)[0]
        assert abs(w0 - f0) <= 1e-9 * f0 + 1e-18
        assert abs(w1 - f1) <= 1e-9 * f1 + 1e-18


def test_uniform_static_column_closed_form():
    # axis-aligned line of sight through a uniform static lattice: each ray is a
    # lattice column of 7 points, length 6 spacings; constant S, so
    # I = S + (I_bg - S) exp(-tau) with tau = alpha 6 h exactly
    m = _lattice()
    n = np.array([0.0, 0.0, 1.0])
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    nu0 = m.lines.freq_Hz[0]
    w = math.sqrt(2 * O.KB * 80.0 / m.lines.mol_mass_kg) / O.C
    nf = 7
    img, rays = O.image(m, pops, n, 7, 7, nf, nu0 * (1 - 2 * w), nu0 * (1 + 2 * w))
    # columns on the lattice's side faces start on boundary points and stop at
    # once; the 5 x 5 interior columns run face to face
    full = np.diff(rays.off) == 7
    assert full.sum() == 25
    full = full.reshape(7, 7)
    h = 1e11
    for f, nu in enumerate(O.image_frequencies(nf, nu0 * (1 - 2 * w), nu0 * (1 + 2 * w))):
        dnu = nu0 * w
        alpha = chi[0, 0] * math.exp(-((nu - nu0) / dnu) ** 2) / (dnu * math.sqrt(math.pi))
        tau = alpha * 6 * h
        Ib = O.planck(nu, m.T_bg)
        ref = S[0, 0] + (Ib - S[0, 0]) * math.exp(-tau)
        assert np.max(np.abs(img[f][full] - ref) / ref) < 1e-12


def test_optically_thin_limit_is_background():
    m = _lattice(n_spec=1e-30)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    nu0 = m.lines.freq_Hz[0]
    img, _ = O.image(m, pops, np.array([0.0, 1.0, 0.0]), 5, 5, 3, nu0 * (1 - 1e-6), nu0 * (1 + 1e-6))
    for f, nu in enumerate(O.image_frequencies(3, nu0 * (1 - 1e-6), nu0 * (1 + 1e-6))):
        assert np.max(np.abs(img[f] / O.planck(nu, m.T_bg) - 1)) < 1e-12


@pytest.mark.parametrize("v", [3e3, -7e3])
def test_uniform_velocity_shifts_the_spectrum(v):
    # a model moving as a whole with speed v toward the observer sees channel
    # nu where the static model sees nu (1 - v/c)
    n = np.array([0.0, 0.0, 1.0])
    ms = synth.config_model(1, n_points=300)
    ms.vel = np.zeros_like(ms.vel)
    mv = synth.config_model(1, n_points=300)
    mv.vel = np.tile(v * n, (mv.n_points, 1))
    pops = O.lte_populations(ms.temp, ms.n_spec, ms.lines.energy_J, ms.lines.g)
    nu0 = ms.lines.freq_Hz[0]
    lo, hi = nu0 * (1 - 3e-5), nu0 * (1 + 3e-5)
    iv, _ = O.image(mv, pops, n, 6, 6, 11, lo, hi)
    b = 1 - v / O.C
    isv, _ = O.image(ms, pops, n, 6, 6, 11, lo * b, hi * b)
    # the optical depths and sources are the same; the backgrounds differ
    # (Planck at nu and at nu (1 - v/c)), so compare with the background off
    ms.T_bg = mv.T_bg = 0.0
    iv0, _ = O.image(mv, pops, n, 6, 6, 11, lo, hi)
    is0, _ = O.image(ms, pops, n, 6, 6, 11, lo * b, hi * b)
    assert np.max(np.abs(iv0 - is0) / np.max(np.abs(is0))) < 1e-9


# ------------------------------------------------------------- image gradient
def test_image_gradient_uniform_column_closed_form():
    # uniform static lattice, line of sight along a lattice axis: every full
    # column gives I = S + (I_bg - S) exp(-tau), tau proportional to n_spec and
    # to phi(nu - nu0; dnu) = exp(-u^2) / (dnu sqrt(pi)), u = (nu - nu0)/dnu,
    # dnu proportional to sqrt(2kT/m) (no turbulence here).  Changing every
    # point of a column together:
    #   d I / d log n  = (S - I_bg) e^-tau tau
    #   d I / d log T  = (S - I_bg) e^-tau tau (2 u^2 - 1) / 2
    #   d I / d (n.v)  = (S - I_bg) e^-tau tau (-2 u / dnu) (-nu / c)
    # so the oracle's per-point gradients summed over a column must give these.
    m = _lattice()
    n = np.array([0.0, 0.0, 1.0])
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    nu0 = m.lines.freq_Hz[0]
    w = math.sqrt(2 * O.KB * 80.0 / m.lines.mol_mass_kg) / O.C
    nf = 7
    lo, hi = nu0 * (1 - 2 * w), nu0 * (1 + 2 * w)
    rays = O.image_rays(m, n, 7, 7)
    full = np.nonzero(np.diff(rays.off) == 7)[0]
    assert full.size == 25
    h = 1e11
    dnu = nu0 * w
    for f, nu in enumerate(O.image_frequencies(nf, lo, hi)):
        gimg = np.zeros((nf, 7, 7))
        gimg[f] = 1.0
        gT, gn, gv = O.image_adjoint(m, pops, n, 7, 7, nf, lo, hi, gimg, rays=rays)
        u = (nu - nu0) / dnu
        tau = chi[0, 0] * math.exp(-u * u) / (dnu * math.sqrt(math.pi)) * 6 * h
        base = (S[0, 0] - O.planck(nu, m.T_bg)) * math.exp(-tau) * tau
        for q in full:
            col = rays.pts[rays.off[q]:rays.off[q + 1]]
            for got, want in ((gn[col].sum(), base), (gT[col].sum(), base * (2 * u * u - 1) / 2),
                              ((gv[col] @ n).sum(), base * (-2 * u / dnu) * (-nu / O.C))):
                assert abs(got - want) <= 1e-10 * abs(base) + 1e-10 * abs(want), (f, q, got, want)


def test_image_gradient_matches_finite_differences_of_the_oracle_image():
    # per point and field, against central differences of the oracle's own FP64
    # image; a (point, field) whose perturbation moves any segment across the
    # trapezoid / erf switch (a jump of the image) is left out and counted
    m = synth.config_model(1, n_points=500)
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    npx = npy = 8
    nf = 9
    nu0 = m.lines.freq_Hz[0]
    lo, hi = nu0 * (1 - 4e-5), nu0 * (1 + 4e-5)
    rng = np.random.default_rng(31)
    gimg = rng.uniform(0.0, 1.0, size=(nf, npy, npx))
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    rays = O.image_rays(m, d, npx, npy)
    gT, gn, gv = O.image_adjoint(m, pops, d, npx, npy, nf, lo, hi, gimg, rays=rays)
    base_br = O.image_branches(m, d, nf, lo, hi, rays)
    pick = rng.choice(np.unique(rays.pts), size=24, replace=False)
    skipped = 0
    # the velocity step is 0.1 m/s: a shift of ~40 Hz in offsets formed as differences of
    # frequencies of ~1e11 Hz (rounding ~1e-5 Hz), far below a line width (~5e5 Hz)
    for key, g, step in (("T", gT, 1e-6), ("n", gn, 1e-6), ("v", gv @ d, 0.1)):
        fd, got = [], []
        for c in pick:
            vals, same = [], True
            for sgn in (1, -1):
                mm = synth.Model(m.name, m.pos, m.vel.copy(), m.temp.copy(), m.vturb2, m.n_coll, m.n_spec.copy(),
                                 m.nbr_offsets, m.nbrs, m.boundary, m.dirs, m.n_quad, m.lines, m.T_bg)
                pp = pops.copy()
                if key == "T":
                    mm.temp[c] *= math.exp(sgn * step)
                elif key == "n":
                    mm.n_spec[c] *= math.exp(sgn * step)
                    pp[c] *= math.exp(sgn * step)
                else:
                    mm.vel[c] = mm.vel[c] + sgn * step * d
                same = same and np.array_equal(O.image_branches(mm, d, nf, lo, hi, rays), base_br)
                img, _ = O.image(mm, pp, d, npx, npy, nf, lo, hi, rays=rays)
                vals.append(float(np.sum(gimg * img)))
            if not same:
                skipped += 1
                continue
            fd.append((vals[0] - vals[1]) / (2 * step))
            got.append(g[c])
        fd, got = np.asarray(fd), np.asarray(got)
        scale = np.max(np.abs(fd))
        assert scale > 0
        err = np.abs(got - fd)
        assert np.all(err <= 1e-6 * scale + 1e-5 * np.abs(fd)), (key, np.max(err / scale))
    assert skipped <= 3
