"""Pins of the CPU oracle against what the mathematics and the paper fix.

Every check here uses something other than the oracle's own formula: closed
forms, limits, invariants, brute force on tiny inputs or an independent
library route.  No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2411_03040_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- radiation
def test_planck_stefan_boltzmann_and_limits():
    # int B_nu dnu = sigma T^4 / pi, sigma = 2 pi^5 k^4 / (15 h^3 c^2)
    T = 300.0
    sigma = 2 * math.pi ** 5 * O.KB ** 4 / (15 * O.H ** 3 * O.C ** 2)
    tot, _ = integrate.quad(lambda nu: float(O.planck(nu, T)), 1e8, 2e15, limit=400, points=[1e13, 3e13])
    assert abs(tot / (sigma * T ** 4 / math.pi) - 1) < 1e-8
    # Rayleigh-Jeans: h nu << k T -> 2 nu^2 k T / c^2
    nu = 1e6
    assert abs(O.planck(nu, 1000.0) / (2 * nu ** 2 * O.KB * 1000.0 / O.C ** 2) - 1) < 1e-6
    # Wien: h nu >> kT -> 2 h nu^3/c^2 exp(-h nu/kT)
    nu = 1e15
    w = 2 * O.H * nu ** 3 / O.C ** 2 * math.exp(-O.H * nu / (O.KB * 100.0))
    assert abs(O.planck(nu, 100.0) / w - 1) < 1e-12
    # the C copy used inside the formal solve agrees
    lib = O._load()
    for nu, T in [(1.15e11, 2.725), (4.6e12, 2.725), (3e11, 80.0)]:
        assert abs(lib.oracle_planck(nu, T) / O.planck(nu, T) - 1) < 1e-14


def test_gauss_hermite_golden_and_moments():
    g = json.load(open(os.path.join(GOLDEN, "gauss_hermite_q3.json")))
    x, w = O.gauss_hermite(3)
    np.testing.assert_allclose(x, g["x"], atol=1e-15)
    np.testing.assert_allclose(w, g["w_normalised"], rtol=1e-14)
    for Q in (7, 31, 40, 50):
        x, w = O.gauss_hermite(Q)
        # E[x^(2k)] for the density exp(-x^2)/sqrt(pi) is Gamma(k+1/2)/sqrt(pi)
        for k in range(0, min(Q, 12)):
            exact = special.gamma(k + 0.5) / math.sqrt(math.pi)
            assert abs(np.sum(w * x ** (2 * k)) / exact - 1) < 1e-10
        assert abs(np.sum(w * x ** 3)) < 1e-12


# ------------------------------------------------------------- line physics
def test_line_data_lte_closed_forms():
    rng = np.random.default_rng(3)
    lines = synth.linear_rotor(6, rng)
    # dipole formula self-check: mu = 0.11 D, J = 1 -> A ~ 7.2e-8 s^-1
    assert abs(lines.A[0] / 7.18e-8 - 1) < 0.01
    T = np.array([20.0, 100.0, 1500.0])
    n = np.array([1.0, 2.0, 3.0])
    pops = O.lte_populations(T, n, lines.energy_J, lines.g)
    np.testing.assert_allclose(pops.sum(1), n, rtol=1e-14)
    # Boltzmann ratios
    for k in range(lines.n_lines):
        u, l = lines.up[k], lines.lo[k]
        np.testing.assert_allclose(pops[:, u] / pops[:, l],
                                   lines.g[u] / lines.g[l] * np.exp(-O.H * lines.freq_Hz[k] / (O.KB * T)),
                                   rtol=1e-12)
    chi, S, ncl = O.line_chi_S(pops, lines)
    assert ncl == 0
    # LTE source function is the Planck function; chi = (h nu/4pi) n_l B_lu (1 - exp(-h nu/kT))
    for k in range(lines.n_lines):
        np.testing.assert_allclose(S[k], O.planck(lines.freq_Hz[k], T), rtol=1e-11)
        _, Blu = O.einstein_B(lines.A[k], lines.freq_Hz[k], lines.g[lines.up[k]], lines.g[lines.lo[k]])
        expect = O.H * lines.freq_Hz[k] / (4 * math.pi) * pops[:, lines.lo[k]] * Blu * \
            -np.expm1(-O.H * lines.freq_Hz[k] / (O.KB * T))
        np.testing.assert_allclose(chi[k], expect, rtol=1e-10)
        # Kirchhoff: in LTE the opacity is the spontaneous emissivity
        # (h nu / 4 pi) n_u A_ul over the Planck function, with no B coefficient
        emis = O.H * lines.freq_Hz[k] / (4 * math.pi) * pops[:, lines.up[k]] * lines.A[k]
        np.testing.assert_allclose(chi[k], emis / O.planck(lines.freq_Hz[k], T), rtol=1e-10)


# ------------------------------------------------------ segment optical depth
def _phi(off, dnu):
    return math.exp(-(off / dnu) ** 2) / (dnu * math.sqrt(math.pi))


def test_profile_normalisation_through_static_segment():
    # static segment (no shift) -> trapezoid of chi phi(offset): integrating over
    # the offset must give dx * chi (the profile has unit area).
    dnu = 3.7e5
    f = lambda off: O.segment_dtau(2.0, 1.5, 1.5, dnu, dnu, dnu, off, off)
    tot, _ = integrate.quad(f, -12 * dnu, 12 * dnu, limit=200)
    assert abs(tot / 3.0 - 1) < 1e-10


@pytest.mark.parametrize("T,vturb", [(40.0, 0.0), (2000.0, 0.0), (300.0, 1.0e3)])
def test_line_width_is_the_maxwellian_velocity_spread(T, vturb):
    # a thermal line of sight velocity has variance kT/m (one component of a
    # Maxwell-Boltzmann distribution), so the profile's variance in frequency
    # is (nu/c)^2 kT/m; the turbulent term enters as v_turb^2 next to 2kT/m
    # (Sec. 4.3, eq. line width), i.e. adds (nu/c)^2 v_turb^2 / 2.  The profile
    # is read back through a static segment of unit length and opacity.
    nu, mass = 230.5e9, 28 * 1.66053906660e-27
    dnu = O.line_width(nu, T, vturb ** 2, mass)
    f = lambda off: off * off * O.segment_dtau(1.0, 1.0, 1.0, dnu, dnu, dnu, off, off)
    var, _ = integrate.quad(f, -12 * dnu, 12 * dnu, limit=200)
    expect = (nu / 299792458.0) ** 2 * (1.380649e-23 * T / mass + vturb ** 2 / 2)
    assert abs(var / expect - 1) < 1e-9


@pytest.mark.parametrize("off0,shift", [(0.0, 0.5), (-1.3, 2.0), (0.4, -3.0), (2.5, 1.2),
                                        (-6.0, -0.8), (3.0, 0.35), (5.0, 8.0)])
def test_semi_analytic_exact_for_constant_opacity(off0, shift):
    # constant chi and width, linear Doppler shift along the segment: the
    # semi-analytic branch is the exact integral of the Gaussian (Sec. 4.3).
    dnu = 2.0e5
    o0, o1 = off0 * dnu, (off0 + shift) * dnu
    got = O.segment_dtau(1.7, 0.9, 0.9, dnu, dnu, dnu, o0, o1)
    exact, _ = integrate.quad(lambda lam: 1.7 * 0.9 * _phi(o0 + lam * (o1 - o0), dnu), 0, 1,
                              epsabs=0, epsrel=1e-13, limit=200)
    # Gauss-Legendre, 64 nodes, as a second independent quadrature
    xg, wg = np.polynomial.legendre.leggauss(64)
    lam = 0.5 * (xg + 1)
    gl = 0.5 * np.sum(wg * np.array([1.7 * 0.9 * _phi(o0 + l * (o1 - o0), dnu) for l in lam]))
    assert abs(got / exact - 1) < 1e-12
    assert abs(got / gl - 1) < 1e-10


def test_trapezoid_branch_and_switch():
    dnu = 1e5
    # below threshold: the trapezoid of the endpoint values
    got = O.segment_dtau(2.0, 1.0, 3.0, dnu, 1.2 * dnu, 1.1 * dnu, 0.1 * dnu, 0.3 * dnu)
    expect = 2.0 * 0.5 * (1.0 * _phi(0.1 * dnu, dnu) + 3.0 * _phi(0.3 * dnu, 1.2 * dnu))
    assert abs(got / expect - 1) < 1e-14
    # exactly at the threshold the semi-analytic branch is taken
    a = O.segment_dtau(1.0, 1.0, 1.0, dnu, dnu, dnu, 0.0, 0.35 * dnu)
    semi = 1.0 * 1.0 * (math.erf(0.35) - 0.0) / (2 * 0.35 * dnu)
    assert abs(a / semi - 1) < 1e-14
    # both branches tend to dx chi phi as the shift vanishes
    for s in (1e-3, 1e-5):
        tr = O.segment_dtau(1.0, 1.0, 1.0, dnu, dnu, dnu, 0.2 * dnu, (0.2 + s) * dnu, thr=10.0)
        sa = O.segment_dtau(1.0, 1.0, 1.0, dnu, dnu, dnu, 0.2 * dnu, (0.2 + s) * dnu, thr=0.0)
        assert abs(tr / sa - 1) < 2 * s
    # orientation does not matter
    x1 = O.segment_dtau(1.0, 2.0, 0.5, dnu, dnu, dnu, -0.4 * dnu, 1.9 * dnu)
    x2 = O.segment_dtau(1.0, 0.5, 2.0, dnu, dnu, dnu, 1.9 * dnu, -0.4 * dnu)
    assert abs(x1 / x2 - 1) < 1e-14


def test_semi_analytic_vs_fine_subdivision():
    # varying opacity: compare with 1000x subdivision of the full integrand
    # (linear chi^{ij}, linear width); the semi-analytic form keeps the
    # error small where the plain trapezoid is far off.
    dnu0, dnu1 = 1.0e5, 1.3e5
    chi0, chi1 = 1.0, 1.6
    o0, o1 = -2.0e5, 2.5e5
    dnub = 0.5 * (dnu0 + dnu1)
    lam = np.linspace(0, 1, 100001)
    ch = chi0 + lam * (chi1 - chi0)
    dn = dnu0 + lam * (dnu1 - dnu0)
    of = o0 + lam * (o1 - o0)
    fine = integrate.simpson(ch * np.exp(-(of / dn) ** 2) / (dn * math.sqrt(math.pi)), x=lam)
    semi = O.segment_dtau(1.0, chi0, chi1, dnu0, dnu1, dnub, o0, o1)
    trap = O.segment_dtau(1.0, chi0, chi1, dnu0, dnu1, dnub, o0, o1, thr=1e9)
    assert abs(semi / fine - 1) < 0.1
    assert abs(trap / fine - 1) > 0.5


def test_subdivision_reference_converges_to_the_integral():
    # the subdivided trapezoid of the study mode: n = 1 is the plain trapezoid,
    # and it converges at second order to the integral of the linearly
    # interpolated integrand (Simpson on 100k points as the reference)
    dnu0, dnu1, chi0, chi1, o0, o1 = 1.0e5, 1.3e5, 1.0, 1.6, -2.0e5, 2.5e5
    lam = np.linspace(0, 1, 100001)
    ch = chi0 + lam * (chi1 - chi0)
    dn = dnu0 + lam * (dnu1 - dnu0)
    of = o0 + lam * (o1 - o0)
    fine = integrate.simpson(ch * np.exp(-(of / dn) ** 2) / (dn * math.sqrt(math.pi)), x=lam)
    t1 = O.segment_dtau_subdiv(1.0, chi0, chi1, dnu0, dnu1, o0, o1, 1)
    trap = O.segment_dtau(1.0, chi0, chi1, dnu0, dnu1, 0.5 * (dnu0 + dnu1), o0, o1, thr=1e9)
    assert abs(t1 / trap - 1) < 1e-14
    errs = [abs(O.segment_dtau_subdiv(1.0, chi0, chi1, dnu0, dnu1, o0, o1, n) / fine - 1) for n in (16, 32, 64)]
    assert errs[0] < 1e-2
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


# ----------------------------------------------------- the two-point system
def _dense_system(dtau, S, Il, Ir):
    D = len(S)
    T = np.zeros((D, D))
    rhs = np.array(S, dtype=np.float64)
    t = dtau[0]
    T[0, 0], T[0, 1] = 1 + 2 / t + 2 / t ** 2, -2 / t ** 2
    rhs[0] += 2 * Il / t
    t = dtau[-1]
    T[-1, -1], T[-1, -2] = 1 + 2 / t + 2 / t ** 2, -2 / t ** 2
    rhs[-1] += 2 * Ir / t
    for d in range(1, D - 1):
        a, b = dtau[d - 1], dtau[d]
        A, Cc = 2 / (a * (a + b)), 2 / (b * (a + b))
        T[d, d - 1], T[d, d], T[d, d + 1] = -A, 1 + A + Cc, -Cc
    return T, rhs


def test_feautrier_matches_dense_lu():
    rng = np.random.default_rng(11)
    for D in range(2, 9):
        for _ in range(5):
            dtau = np.exp(rng.uniform(np.log(0.05), np.log(20.0), D - 1))
            S = rng.uniform(0.1, 3.0, D)
            Il, Ir = rng.uniform(0, 2, 2)
            T, rhs = _dense_system(dtau, S, Il, Ir)
            sol = np.linalg.solve(T, rhs)
            Tinv = np.linalg.inv(T)
            for io in range(D):
                u, L = O.feautrier_at(dtau, S, Il, Ir, io)
                assert abs(u / sol[io] - 1) < 1e-12
                assert abs(L / Tinv[io, io] - 1) < 1e-12
                assert 0 < L < 1


def _exact_solve(dtau, S, Il, Ir, io):
    """u_io and (T^-1)_{io,io} of the assembled system in exact rational
    arithmetic (the float inputs converted exactly; Gauss-Jordan elimination)."""
    from fractions import Fraction as Fr
    D = len(S)
    dt = [Fr(float(x)) for x in dtau]
    T = [[Fr(0)] * D for _ in range(D)]
    rhs = [Fr(float(x)) for x in S]
    t = dt[0]
    T[0][0], T[0][1] = 1 + 2 / t + 2 / t ** 2, -2 / t ** 2
    rhs[0] += 2 * Fr(float(Il)) / t
    t = dt[-1]
    T[D - 1][D - 1], T[D - 1][D - 2] = 1 + 2 / t + 2 / t ** 2, -2 / t ** 2
    rhs[D - 1] += 2 * Fr(float(Ir)) / t
    for d in range(1, D - 1):
        a, b = dt[d - 1], dt[d]
        A, Cc = 2 / (a * (a + b)), 2 / (b * (a + b))
        T[d][d - 1], T[d][d], T[d][d + 1] = -A, 1 + A + Cc, -Cc
    e = [Fr(int(k == io)) for k in range(D)]
    M = [T[k][:] + [rhs[k], e[k]] for k in range(D)]
    for c in range(D):
        p = next(r for r in range(c, D) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(D):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return float(M[io][D] / M[io][io]), float(M[io][D + 1] / M[io][io])


def test_feautrier_exact_rational_at_extreme_depths():
    # optically thin segments (down to the 1e-150 floor), thick ones and mixed
    # rays: the oracle's solve against exact rational arithmetic
    rng = np.random.default_rng(13)
    cases = []
    for D in range(2, 7):
        for lo, hi in [(-150, -140), (-12, -6), (-3, 3), (2, 6), (-150, 6)]:
            cases.append((D, np.exp(rng.uniform(lo, hi, D - 1) * np.log(10.0))))
    for D, dtau in cases:
        S = rng.uniform(0.1, 3.0, D)
        Il, Ir = rng.uniform(0.0, 2.0, 2)
        for io in range(D):
            u_ex, L_ex = _exact_solve(dtau, S, Il, Ir, io)
            u, L = O.feautrier_at(dtau, S, Il, Ir, io)
            assert abs(u / u_ex - 1) < 1e-13, (D, dtau, io, u, u_ex)
            assert L_ex == 0.0 or abs(L / L_ex - 1) < 1e-13, (D, dtau, io, L, L_ex)


def _rh_two_sweep(dtau, S, Il, Ir, io):
    """Cross-check: Rybicki-Hummer elimination from both ends toward io,
    F_d = (1 + A_d F_{d-1}/(1 + F_{d-1})) / C_d with its source sweep, and the
    mirrored sweep from the far end, combined at io (a formulation the oracle
    does not use)."""
    D = len(S)
    F = z = G = w = 0.0
    for d in range(io):
        if d == 0:
            t = dtau[0]
            F = (1 + 2 / t) * t * t / 2
            z = (S[0] + 2 * Il / t) / (1 + 2 / t + 2 / t ** 2)
        else:
            a, b = dtau[d - 1], dtau[d]
            A, Cc = 2 / (a * (a + b)), 2 / (b * (a + b))
            Fn = (1 + A * F / (1 + F)) / Cc
            z = (S[d] + A * z) / (Cc * (1 + Fn))
            F = Fn
    for d in range(D - 1, io, -1):
        if d == D - 1:
            t = dtau[D - 2]
            G = (1 + 2 / t) * t * t / 2
            w = (S[D - 1] + 2 * Ir / t) / (1 + 2 / t + 2 / t ** 2)
        else:
            a, b = dtau[d - 1], dtau[d]
            A, Cc = 2 / (a * (a + b)), 2 / (b * (a + b))
            Gn = (1 + Cc * G / (1 + G)) / A
            w = (S[d] + Cc * w) / (A * (1 + Gn))
            G = Gn
    if io == 0:
        t = dtau[0]
        Cc = 2 / (t * t)
        den, num = 1 + 2 / t + Cc * G / (1 + G), S[0] + 2 * Il / t + Cc * w
    elif io == D - 1:
        t = dtau[D - 2]
        A = 2 / (t * t)
        den, num = 1 + 2 / t + A * F / (1 + F), S[D - 1] + 2 * Ir / t + A * z
    else:
        a, b = dtau[io - 1], dtau[io]
        A, Cc = 2 / (a * (a + b)), 2 / (b * (a + b))
        den, num = 1 + A * F / (1 + F) + Cc * G / (1 + G), S[io] + A * z + Cc * w
    return num / den, 1 / den


def test_feautrier_matches_two_sided_elimination_on_long_rays():
    rng = np.random.default_rng(14)
    for D in (17, 60, 301):
        for lo, hi in [(-30, -8), (-4, 1), (-1, 4), (-30, 4)]:
            dtau = np.exp(rng.uniform(lo, hi, D - 1) * np.log(10.0))
            S = rng.uniform(0.1, 3.0, D)
            Il, Ir = rng.uniform(0.0, 2.0, 2)
            for io in (0, D // 3, D - 1):
                u, L = O.feautrier_at(dtau, S, Il, Ir, io)
                u2, L2 = _rh_two_sweep(dtau, S, Il, Ir, io)
                assert abs(u / u2 - 1) < 1e-12 and abs(L / L2 - 1) < 1e-11, (D, lo, io, u, u2, L, L2)


def test_feautrier_uniform_slab_second_order():
    # uniform static medium: u(o) -> S + (I - S)(e^-tau+ + e^-tau-)/2
    S, I = 2.0, 0.5
    for tp, tm in [(1.0, 3.0), (0.3, 0.3), (5.0, 0.2)]:
        exact = S + (I - S) * (math.exp(-tp) + math.exp(-tm)) / 2
        errs = []
        for n in (16, 32, 64, 128):
            h = 1.0 / n
            dtau = np.concatenate([np.full(n, tm * h), np.full(n, tp * h)])
            u, _ = O.feautrier_at(dtau, np.full(2 * n + 1, S), I, I, n)
            errs.append(abs(u - exact))
        ratios = [errs[i] / errs[i + 1] for i in range(3)]
        assert all(3.5 < r < 4.5 for r in ratios), (errs, ratios)
        assert errs[-1] < 1e-4


def test_feautrier_limits():
    # optically thin: u -> I_bg, L* -> 0; thick: u -> S, L* -> 1
    dt = np.full(20, 1e-9)
    u, L = O.feautrier_at(dt, np.full(21, 7.0), 1.0, 1.0, 10)
    assert abs(u - 1.0) < 1e-7 and L < 1e-8
    dt = np.full(20, 50.0)
    u, L = O.feautrier_at(dt, np.full(21, 7.0), 1.0, 1.0, 10)
    assert abs(u / 7.0 - 1) < 1e-10 and abs(L - 1) < 1e-3
    # one-sided ray (origin at an end) and the degenerate single point
    u, L = O.feautrier_at(np.array([1e-12]), np.array([3.0, 3.0]), 0.25, 0.25, 0)
    assert abs(u - 0.25) < 1e-9
    u, L = O.feautrier_at(np.zeros(0), np.array([3.0]), 0.25, 0.25, 0)
    assert u == 0.25 and L == 0.0


# -------------------------------------------------------------- ray tracing
def _tiny_model(case):
    pos = np.asarray(case["pos"], np.float64)
    nb = case["nbrs"]
    off = np.zeros(len(nb) + 1, np.int64)
    for i, v in enumerate(nb):
        off[i + 1] = off[i] + len(v)
    flat = np.concatenate([np.asarray(v, np.int32) for v in nb])
    m = synth.Model("tiny", pos, np.zeros_like(pos), np.ones(len(pos)), np.zeros(len(pos)),
                    np.ones(len(pos)), np.ones(len(pos)), off, flat, np.asarray(case["boundary"], np.int32),
                    np.asarray(case["dirs"], np.float64), 3, synth.linear_rotor(2, np.random.default_rng(0)))
    return m


def test_trace_hand_derived_golden():
    g = json.load(open(os.path.join(GOLDEN, "trace_tiny.json")))
    for case in g["cases"]:
        m = _tiny_model(case)
        rays = O.trace(m)
        o = case["origin"]
        for r, exp in enumerate(case["expected_rays"]):
            assert list(rays.half(r, o)) == exp, (case["name"], r)
        N, R = m.n_points, m.dirs.shape[0]
        st = rays.stall
        assert [bool(st[r * N + o]) for r in range(R)] == case["expected_stall"]


def test_trace_lattice_closed_form():
    n = 7
    m = synth.lattice_model(n_side=n)
    rays = O.trace(m)
    assert rays.stalls == 0
    idx = np.arange(n ** 3).reshape(n, n, n)
    rng = np.random.default_rng(0)
    face = np.zeros(n ** 3, bool)
    face[m.boundary] = True

    def until_face(line):
        out = []
        for c in line:
            out.append(c)
            if face[c]:
                break
        return np.asarray(out, dtype=np.int64)

    for o in rng.choice(n ** 3, 80, replace=False):
        i, j, k = np.unravel_index(o, (n, n, n))
        np.testing.assert_array_equal(rays.half(0, o), until_face(idx[i + 1:, j, k]))
        np.testing.assert_array_equal(rays.half(1, o), until_face(idx[:i, j, k][::-1]))
        np.testing.assert_array_equal(rays.half(4, o), until_face(idx[i, j, k + 1:]))
        if 0 < j < n - 1 and 0 < k < n - 1:
            assert len(rays.half(0, o)) == n - 1 - i


def test_trace_invariants_delaunay_sphere():
    m = synth.config_model(1, n_points=600)
    rays = O.trace(m)
    assert rays.stalls == 0          # interior Delaunay vertices see every half-space
    bset = set(m.boundary.tolist())
    nbr = [set(m.nbrs[m.nbr_offsets[i]:m.nbr_offsets[i + 1]].tolist()) for i in range(m.n_points)]
    for r in range(m.dirs.shape[0]):
        n = m.dirs[r]
        for o in range(m.n_points):
            h = rays.half(r, o)
            if len(h) == 0:
                assert o in bset
                continue
            Z = (m.pos[h] - m.pos[o]) @ n
            assert np.all(np.diff(Z) > 0) and Z[0] > 0
            prev = o
            for c in h:
                assert c in nbr[prev]
                prev = c
            assert h[-1] in bset
            assert not any(c in bset for c in h[:-1])


# ---------------------------------------------------- statistical equilibrium
def test_se_lte_limit_detailed_balance():
    rng = np.random.default_rng(5)
    lines = synth.linear_rotor(41, rng)
    N = 50
    T = 10 ** rng.uniform(1.0, 3.3, N)          # 10 K .. 2000 K: populations down to 1e-190
    nspec = rng.uniform(1, 10, N)
    ncoll = 10 ** rng.uniform(6, 14, N)
    pops0 = O.lte_populations(rng.uniform(10, 3000, N), nspec, lines.energy_J, lines.g)
    J = np.stack([O.planck(lines.freq_Hz[k], T) for k in range(lines.n_lines)], axis=1)
    new = O.stat_equilibrium(pops0, J, np.zeros_like(J), T, ncoll, nspec, lines)
    x = lines.g[None, :] * np.exp(-lines.energy_J[None, :] / (O.KB * T[:, None]))
    boltz = nspec[:, None] * x / x.sum(1, keepdims=True)
    assert (boltz / nspec[:, None]).min() < 1e-100
    np.testing.assert_allclose(new, boltz, rtol=1e-11)    # componentwise, tiny levels included


def test_se_matches_dense_lu_where_populations_are_not_tiny_and_balances_every_level():
    rng = np.random.default_rng(15)
    lines = synth.linear_rotor(8, rng)
    N = 60
    T = rng.uniform(300, 2000, N)
    nspec = rng.uniform(1, 10, N)
    ncoll = 10 ** rng.uniform(6, 12, N)
    M = lines.n_lines
    J = np.stack([O.planck(lines.freq_Hz[k], 2.725) + O.planck(lines.freq_Hz[k], T) * rng.uniform(0, 0.5, N)
                  for k in range(M)], axis=1)
    Lst = rng.uniform(0.0, 0.5, (N, M))
    p0 = O.lte_populations(T, nspec, lines.energy_J, lines.g)
    a = O.stat_equilibrium(p0, J, Lst, T, ncoll, nspec, lines)
    b = O.stat_equilibrium_dense(p0, J, Lst, T, ncoll, nspec, lines)
    assert (b / nspec[:, None]).min() > 1e-6
    np.testing.assert_allclose(a, b, rtol=1e-9)
    # every level balances to rounding (relative to its own outflow), low T included
    T2 = np.full(N, 25.0)
    c = O.stat_equilibrium(O.lte_populations(T2, nspec, lines.energy_J, lines.g), J, Lst, T2,
                           ncoll, nspec, lines)
    R = O.rate_matrix(O.lte_populations(T2, nspec, lines.energy_J, lines.g), J, Lst, T2, ncoll,
                      nspec, lines)
    inflow = np.einsum("pj,pji->pi", c, R)
    outflow = c * R.sum(axis=2)
    assert np.all(c > 0)
    assert np.max(np.abs(inflow - outflow) / outflow) < 1e-12


def _tree_theorem_stationary(R):
    """Steady state of the rate matrix R[i, j] (i -> j) by the Markov chain tree
    theorem: the population of level i is proportional to the sum, over all
    spanning trees directed toward i, of the product of their rates.  Trees
    are enumerated by brute force (each other level picks a successor; keep
    the choices whose paths all reach i).  Only products and sums of positive
    numbers: exact to rounding however small the populations are."""
    import itertools
    L = R.shape[0]
    w = np.zeros(L)
    for root in range(L):
        others = [j for j in range(L) if j != root]
        total = 0.0
        for succ in itertools.product(range(L), repeat=len(others)):
            f = dict(zip(others, succ))
            if any(f[j] == j for j in others):
                continue
            ok = True
            for j in others:
                seen, k = set(), j
                while k != root:
                    if k in seen:
                        ok = False
                        break
                    seen.add(k)
                    k = f[k]
                if not ok:
                    break
            if ok:
                total += float(np.prod([R[j, f[j]] for j in others]))
        w[root] = total
    return w / w.sum()


def test_se_matches_markov_chain_tree_theorem_down_to_tiny_populations():
    # cold gas and a weak field: the top level sits ~1e-41 below the ground
    rng = np.random.default_rng(16)
    lines = synth.linear_rotor(5, rng)
    N = 4
    T = np.array([0.6, 1.5, 8.0, 60.0])
    nspec = rng.uniform(1, 10, N)
    ncoll = 10 ** rng.uniform(3, 9, N)
    M = lines.n_lines
    J = np.stack([O.planck(lines.freq_Hz[k], 0.5) * rng.uniform(0.5, 2.0, N) for k in range(M)], axis=1)
    Lst = rng.uniform(0.0, 0.6, (N, M))
    p0 = O.lte_populations(T, nspec, lines.energy_J, lines.g)
    new = O.stat_equilibrium(p0, J, Lst, T, ncoll, nspec, lines)
    R = O.rate_matrix(p0, J, Lst, T, ncoll, nspec, lines)
    for p in range(N):
        Rp = R[p].copy()
        np.fill_diagonal(Rp, 0.0)
        ref = _tree_theorem_stationary(Rp) * nspec[p]
        np.testing.assert_allclose(new[p], ref, rtol=1e-12)
    assert (new / nspec[:, None]).min() < 1e-40


def test_se_two_level_closed_form_and_high_density():
    rng = np.random.default_rng(6)
    lines = synth.linear_rotor(2, rng)
    A, nu = lines.A[0], lines.freq_Hz[0]
    Bul, Blu = O.einstein_B(A, nu, lines.g[1], lines.g[0])
    N = 20
    T = rng.uniform(10, 500, N)
    ncoll = 10 ** rng.uniform(4, 12, N)
    J = rng.uniform(0, 3, N) * O.planck(nu, 30.0)
    nspec = np.full(N, 2.0)
    new = O.stat_equilibrium(O.lte_populations(T, nspec, lines.energy_J, lines.g), J[:, None],
                             np.zeros((N, 1)), T, ncoll, nspec, lines)
    Cul = ncoll * lines.K_ul[0]
    Clu = Cul * lines.g[1] / lines.g[0] * np.exp(-O.H * nu / (O.KB * T))
    ratio = (Blu * J + Clu) / (A + Bul * J + Cul)
    np.testing.assert_allclose(new[:, 1] / new[:, 0], ratio, rtol=1e-11)
    np.testing.assert_allclose(new.sum(1), nspec, rtol=1e-14)
    # collision-dominated -> Boltzmann whatever the radiation field
    lines5 = synth.linear_rotor(5, rng)
    T = np.full(4, 150.0)
    J = np.zeros((4, 4))
    new = O.stat_equilibrium(O.lte_populations(T, np.ones(4), lines5.energy_J, lines5.g), J, J, T,
                             np.full(4, 1e25), np.ones(4), lines5)
    np.testing.assert_allclose(new, O.lte_populations(T, np.ones(4), lines5.energy_J, lines5.g), rtol=1e-6)


def test_se_lambda_star_terms_vanish_at_fixed_point():
    # The approximate-Lambda terms add -L* [n_u (A + B_ul S) - n_l B_lu S] to
    # each line's net rate, which is zero when S is the source function of the
    # populations themselves.  So: solve without L* -> p1; then with any L* and
    # S_old = S(p1) the solution must be p1 again.  A wrong sign or a missing
    # L* term in either rate breaks this.
    rng = np.random.default_rng(8)
    lines = synth.linear_rotor(5, rng)
    N = 40
    T = rng.uniform(30, 300, N)
    nspec = rng.uniform(0.5, 2.0, N)
    ncoll = 10 ** rng.uniform(11, 13, N)
    M = lines.n_lines
    # sub-thermal radiation (no level inversions, so no opacity floor is hit)
    J = np.stack([O.planck(lines.freq_Hz[k], T) * rng.uniform(0.1, 1.0, N) for k in range(M)], axis=1)
    p0 = O.lte_populations(T, nspec, lines.energy_J, lines.g)
    p1 = O.stat_equilibrium(p0, J, np.zeros((N, M)), T, ncoll, nspec, lines)
    assert O.line_chi_S(p1, lines)[2] == 0
    # a formal solution always has Jbar >= Lstar S (J_eff >= 0): draw L* that way
    S1 = O.line_chi_S(p1, lines)[1].T
    Lst = rng.uniform(0.0, 0.95, (N, M)) * np.minimum(1.0, J / S1)
    p2 = O.stat_equilibrium(p1, J, Lst, T, ncoll, nspec, lines)
    np.testing.assert_allclose(p2, p1, rtol=1e-9)
    # and with S_old from other populations the answer does move
    p3 = O.stat_equilibrium(p0, J, Lst, T, ncoll, nspec, lines)
    assert O.maxrel(p3, p1) > 1e-3


# ----------------------------------------------------------------------- Ng
def test_ng_coefficients_constrained_least_squares():
    rng = np.random.default_rng(9)
    for n in (3, 5, 8):
        X = rng.normal(size=(n, 40))
        c = O.ng_coefficients(X)
        assert abs(c.sum() - 1) < 1e-13
        # independent route: minimise |sum c_k r_k|^2 on the affine set sum c = 1
        Rm = X[1:] - X[:-1]
        k = n - 1
        Z = np.zeros((k, k - 1))
        for i in range(k - 1):
            Z[i, i], Z[i + 1, i] = 1.0, -1.0
        c0 = np.zeros(k)
        c0[0] = 1.0
        y, *_ = np.linalg.lstsq(Rm.T @ Z, -(Rm.T @ c0), rcond=None)
        np.testing.assert_allclose(c, c0 + Z @ y, atol=1e-10)


def test_ng_exact_on_linear_map():
    # x -> M x + b with the initial error in a k-dim invariant subspace: an Ng
    # step with k+1 residuals lands on the fixed point.
    rng = np.random.default_rng(10)
    n, k = 30, 3
    Qm, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.concatenate([[0.9, 0.7, -0.5], rng.uniform(-0.5, 0.5, n - 3)])
    Mm = Qm @ np.diag(lam) @ Qm.T
    b = rng.normal(size=n)
    xstar = np.linalg.solve(np.eye(n) - Mm, b)
    x = xstar + Qm[:, :k] @ rng.normal(size=k)
    it = [x]
    for _ in range(k + 1):
        it.append(Mm @ it[-1] + b)
    pred = O.ng_predict(it)
    assert np.max(np.abs(pred - xstar)) < 1e-10 * np.max(np.abs(xstar))
    # the newest plain iterate is still far off
    assert np.max(np.abs(it[-1] - xstar)) > 1e-3


def test_ng_controllers_reach_fixed_point_faster():
    rng = np.random.default_rng(12)
    n = 50
    Qm, _ = np.linalg.qr(rng.normal(size=(n, n)))
    Mm = Qm @ np.diag(rng.uniform(0.0, 0.95, n)) @ Qm.T
    xstar = rng.uniform(0.5, 1.0, n)          # positive, like populations
    b = (np.eye(n) - Mm) @ xstar

    def run(ctrl, iters=40):
        x = np.ones(n)
        if ctrl:
            ctrl.reset(x)
        for _ in range(iters):
            x = Mm @ x + b
            if ctrl:
                x, _ = ctrl.push(x)
        return np.max(np.abs(x - xstar) / np.abs(xstar))

    plain, cl, ad = run(None), run(O.NgClassical(4)), run(O.NgAdaptive(8))
    assert cl < plain and ad < plain
    assert ad < 1e-6


# Hand-worked controller sequences (Sec. 4.2).  The iterates are small dyadic
# vectors, so every coefficient and prediction below is a short fraction,
# derived by hand from the closed form of the two-residual solve:
#   G = [[r1.r1, r1.r2], [r1.r2, r2.r2]],  c proportional to
#   (G22 - G12, G11 - G12), normalised to sum 1,
# and for orthogonal residuals c_k proportional to 1/|r_k|^2.
def _x(*v):
    return np.array(v, dtype=np.float64)


def test_ng_adaptive_first_running_prediction_is_the_newest_iterate():
    # x1 = (1, 1), x2 = (1/2, 1), x3 = (1/2, 3/4): orthogonal residuals
    # r1 = (-1/2, 0), r2 = (0, -1/4); c = (1/16, 1/4) / (5/16) = (1/5, 4/5);
    # P3 = x2/5 + 4 x3/5 = (1/2, 4/5).  With P2 = x2 (the prediction of two
    # iterates is the newer one): maxrel(P3, x2) = 1/5 < maxrel(x3, x2) = 1/4,
    # so P3 is used.  (Reading P2 as x1 would give maxrel(P3, x1) = 1/2 > 1/4.)
    ng = O.NgAdaptive(n_max=8)
    ng.reset(_x(1, 1))
    out, acc = ng.push(_x(0.5, 1))
    assert not acc and np.array_equal(out, _x(0.5, 1))
    out, acc = ng.push(_x(0.5, 0.75))
    assert acc
    np.testing.assert_allclose(out, _x(0.5, 0.8), rtol=1e-14)


def test_ng_adaptive_compares_with_the_previous_running_prediction():
    # x1 = (1, 1, 1), x2 = (3/2, 3/2, 19/16), x3 = (15/8, 15/8, 11/8),
    # x4 = (9/4, 37/16, 21/16).
    # m = 3: r1 = (1/2, 1/2, 3/16), r2 = (3/8, 3/8, 3/16), G = [[137, 105],
    #   [105, 81]] / 256, c = (-24, 32) / 8 = (-3, 4), P3 = -3 x2 + 4 x3
    #   = (3, 3, 31/16); maxrel(P3, x2) = 1 >= maxrel(x3, x2) = 1/4: not used,
    #   P3 becomes the running prediction.
    # m = 4: c = (-35, 38, 8) / 11, P4 = (147/44, 149/44, 339/176);
    #   maxrel(P4, P3) = 17/132 < maxrel(x4, x3) = 7/30: used.  (Comparing with
    #   a running prediction left at P2 = x2 would give 83/66 > 7/30.)
    ng = O.NgAdaptive(n_max=8)
    ng.reset(_x(1, 1, 1))
    for x in (_x(1.5, 1.5, 19 / 16), _x(15 / 8, 15 / 8, 11 / 8)):
        out, acc = ng.push(x)
        assert not acc and np.array_equal(out, x)
    out, acc = ng.push(_x(9 / 4, 37 / 16, 21 / 16))
    assert acc
    np.testing.assert_allclose(out, _x(147 / 44, 149 / 44, 339 / 176), rtol=1e-13)


def test_ng_adaptive_forced_at_exactly_n_max_iterates():
    # N_max = 4.  x1 = (1, 1, 1), x2 = (3/4, 1/2, 1/2), x3 = (5/8, 3/8, 1/4),
    # x4 = (3/8, 3/8, 3/8).
    # m = 3: r1 = (-1/4, -1/2, -1/2), r2 = (-1/8, -1/8, -1/4), G = [[18, 7],
    #   [7, 3]] / 32, c = (-4, 11) / 7, P3 = (31/56, 17/56, 3/28);
    #   maxrel(P3, x2) = 11/14 >= 1/2: not used.
    # m = 4: c = (-4, 11, 2) / 9, P4 = (37/72, 23/72, 1/6);
    #   maxrel(P4, P3) = 5/9 >= maxrel(x4, x3) = 1/2, but m = N_max: used anyway.
    ng = O.NgAdaptive(n_max=4)
    ng.reset(_x(1, 1, 1))
    for x in (_x(0.75, 0.5, 0.5), _x(5 / 8, 3 / 8, 0.25)):
        out, acc = ng.push(x)
        assert not acc
    out, acc = ng.push(_x(3 / 8, 3 / 8, 3 / 8))
    assert acc
    np.testing.assert_allclose(out, _x(37 / 72, 23 / 72, 1 / 6), rtol=1e-13)
    # with N_max = 5 the same sequence is not accelerated at m = 4
    ng = O.NgAdaptive(n_max=5)
    ng.reset(_x(1, 1, 1))
    accs = [ng.push(x)[1] for x in (_x(0.75, 0.5, 0.5), _x(5 / 8, 3 / 8, 0.25), _x(3 / 8, 3 / 8, 3 / 8))]
    assert accs == [False, False, False]


def test_ng_adaptive_negative_prediction_restarts_from_the_regular_iterate():
    # N_max = 3.  x1 = (1, 1), x2 = (1/2, 1), x3 = (1/8, 17/16):
    # r1 = (-1/2, 0), r2 = (-3/8, 1/16), G = [[64, 48], [48, 37]] / 256,
    # c = (-11, 16) / 5, P3 = (-7/10, 6/5): forced at m = N_max but negative, so
    # x3 is kept and the history restarts from it.  Then x4 = (1/8, 21/16),
    # x5 = (3/16, 21/16): residuals (0, 1/4), (1/16, 0) from x3, c = (1, 16) / 17,
    # P = (25/136, 21/16), used at m = 3 of the new history.
    ng = O.NgAdaptive(n_max=3)
    ng.reset(_x(1, 1))
    assert not ng.push(_x(0.5, 1))[1]
    out, acc = ng.push(_x(1 / 8, 17 / 16))
    assert not acc and np.array_equal(out, _x(1 / 8, 17 / 16))
    assert not ng.push(_x(1 / 8, 21 / 16))[1]
    out, acc = ng.push(_x(3 / 16, 21 / 16))
    assert acc
    np.testing.assert_allclose(out, _x(25 / 136, 21 / 16), rtol=1e-14)


def test_ng_classical_restarts_from_its_prediction():
    # N_steps = 2.  y0 = (1, 1, 1), y1 = (1/2, 1, 1), y2 = (1/2, 3/4, 1):
    # orthogonal residuals of sizes 1/2, 1/4, c = (1/5, 4/5), Q1 = (1/2, 4/5, 1)
    # replaces y2 and is the first iterate of the next history.  y3 = (1/2, 4/5,
    # 1/2), y4 = (3/4, 4/5, 1/2): residuals from Q1 of sizes 1/2, 1/4 again,
    # Q2 = y3/5 + 4 y4/5 = (7/10, 4/5, 1/2).
    ng = O.NgClassical(n_steps=2)
    ng.reset(_x(1, 1, 1))
    assert not ng.push(_x(0.5, 1, 1))[1]
    out, acc = ng.push(_x(0.5, 0.75, 1))
    assert acc
    np.testing.assert_allclose(out, _x(0.5, 0.8, 1), rtol=1e-14)
    assert not ng.push(_x(0.5, 0.8, 0.5))[1]
    out, acc = ng.push(_x(0.75, 0.8, 0.5))
    assert acc
    np.testing.assert_allclose(out, _x(0.7, 0.8, 0.5), rtol=1e-14)


# -------------------------------------------------- whole-model closed forms
def _uniform_model(chi_scale, n_side=9, temp=40.0):
    m = synth.lattice_model(n_side=n_side, n_levels=2, n_quad=11, temp=temp, n_coll=1e30)
    m.n_spec[:] = chi_scale
    return m


def test_formal_solve_thin_limit_is_background():
    m = _uniform_model(1e-12)
    rays = O.trace(m)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    J, L = O.formal_solve(m, rays, chi, S, origins=np.arange(0, m.n_points, 37))
    x, w = O.gauss_hermite(m.n_quad)
    dnu = O.line_width(m.lines.freq_Hz[0], m.temp[0], 0.0, m.lines.mol_mass_kg)
    Ibg = np.sum(w * O.planck(m.lines.freq_Hz[0] + x * dnu, m.T_bg))
    np.testing.assert_allclose(J[:, 0], Ibg, rtol=1e-8)
    assert np.all(L < 1e-6)


def test_formal_solve_thick_lte_is_source_function():
    m = _uniform_model(1e16, temp=40.0)
    rays = O.trace(m)
    pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
    chi, S, _ = O.line_chi_S(pops, m.lines)
    centre = (m.n_points - 1) // 2
    J, L = O.formal_solve(m, rays, chi, S, origins=[centre])
    # deep inside: J-bar -> S = B_nu(T) and L* -> 1 (bins weighted over the profile)
    assert abs(J[0, 0] / O.planck(m.lines.freq_Hz[0], 40.0) - 1) < 1e-6
    assert L[0, 0] > 0.95


def test_formal_solve_uniform_static_lattice_closed_form():
    # axis-aligned rays in a static uniform cube: each pair's u_o converges to
    # S + (I - S)(e^-tau+ + e^-tau-)/2 with tau = chi phi(nu) * path length.
    # Compare per bin by building the closed form J-bar over the 6 directions.
    errs = []
    for n_side in (9, 17, 33):
        spacing = 8e11 / (n_side - 1)
        m = synth.lattice_model(n_side=n_side, spacing_m=spacing, n_levels=2, n_quad=5,
                                temp=40.0, n_coll=1e30)
        m.n_spec[:] = 5e7       # line-centre optical depth of order one across the cube
        rays = O.trace(m)
        pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
        chi, S, _ = O.line_chi_S(pops, m.lines)
        o = int(np.ravel_multi_index(((n_side - 1) // 4, (n_side - 1) // 2, (n_side - 1) // 2),
                                     (n_side,) * 3))
        J, _ = O.formal_solve(m, rays, chi, S, origins=[o])
        x, w = O.gauss_hermite(m.n_quad)
        nu0 = m.lines.freq_Hz[0]
        dnu = O.line_width(nu0, 40.0, 0.0, m.lines.mol_mass_kg)
        Sv = S[0, 0]
        exact = 0.0
        ii = (n_side - 1) // 4
        for q in range(m.n_quad):
            kap = chi[0, 0] * math.exp(-x[q] ** 2) / (dnu * math.sqrt(math.pi))
            I = O.planck(nu0 + x[q] * dnu, m.T_bg)
            # x-axis pair: distances ii and (n_side-1-ii); y and z pairs: half each
            lx = [ii * spacing, (n_side - 1 - ii) * spacing]
            ly = [(n_side - 1) / 2 * spacing] * 2
            for (a, b) in (lx, ly, ly):
                u = Sv + (I - Sv) * (math.exp(-kap * a) + math.exp(-kap * b)) / 2
                exact += (1.0 / 3.0) * w[q] * u
        errs.append(abs(J[0, 0] / exact - 1))
        assert abs(J[0, 0] / O.planck(nu0, m.T_bg) - 1) > 0.05   # far from the thin limit
    assert errs[0] < 1e-2
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


@pytest.mark.parametrize("widths", [2.4, 20.0], ids=["trapezoid", "semi-analytic"])
def test_formal_solve_linear_velocity_lattice_closed_form(widths):
    # the static lattice above with v_x = g x: along the x axis the comoving
    # offset of bin q grows linearly with the distance s from the origin, in
    # both directions, nu_q g s / c (Sec. 4.3, the Doppler-shifted profile),
    # so tau(l) = chi [erf(x_q + k l / dnu) - erf(x_q)] / (2 k), k = nu_q g / c,
    # and u_o tends to S + (I - S)(e^-tau+ + e^-tau-)/2 at second order.  The
    # origin is off centre, so its own velocity is not zero.  A shift of 2.4
    # line widths across the cube keeps every segment below the 0.35 switch
    # (trapezoid); 20 widths keep every segment above it (semi-analytic).
    errs = []
    for n_side in (9, 17, 33):
        size = 8e11
        spacing = size / (n_side - 1)
        m = synth.lattice_model(n_side=n_side, spacing_m=spacing, n_levels=2, n_quad=5,
                                temp=40.0, n_coll=1e30)
        m.n_spec[:] = 5e7
        nu0 = m.lines.freq_Hz[0]
        dnu = O.line_width(nu0, 40.0, 0.0, m.lines.mol_mass_kg)
        g = widths * (dnu / nu0) * O.C / size
        m.vel = np.zeros_like(m.pos)
        m.vel[:, 0] = g * m.pos[:, 0]
        ii = (n_side - 1) // 4
        o = int(np.ravel_multi_index((ii, (n_side - 1) // 2, (n_side - 1) // 2), (n_side,) * 3))
        rays = O.trace(m, origins=[o])
        pops = O.lte_populations(m.temp, m.n_spec, m.lines.energy_J, m.lines.g)
        chi, S, _ = O.line_chi_S(pops, m.lines)
        J, _ = O.formal_solve(m, rays, chi, S, origins=[o])
        x, w = O.gauss_hermite(m.n_quad)
        Sv, ch = S[0, 0], chi[0, 0]
        lx = [ii * spacing, (n_side - 1 - ii) * spacing]
        ly = (n_side - 1) / 2 * spacing
        moving = static = 0.0
        for q in range(m.n_quad):
            nuq = nu0 + x[q] * dnu
            I = O.planck(nuq, m.T_bg)
            k = nuq * g / O.C
            tau = [ch / (2 * k) * (special.erf(x[q] + k * l / dnu) - special.erf(x[q])) for l in lx]
            kap = ch * math.exp(-x[q] ** 2) / (dnu * math.sqrt(math.pi))
            uy = Sv + (I - Sv) * math.exp(-kap * ly)
            ux = Sv + (I - Sv) * (math.exp(-tau[0]) + math.exp(-tau[1])) / 2
            ux0 = Sv + (I - Sv) * (math.exp(-kap * lx[0]) + math.exp(-kap * lx[1])) / 2
            moving += w[q] * (ux + 2 * uy) / 3
            static += w[q] * (ux0 + 2 * uy) / 3
        errs.append(abs(J[0, 0] / moving - 1))
    assert errs[0] < 1e-3
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs
    # the velocity field matters far more than the remaining error
    assert abs(moving / static - 1) > 1000 * errs[2]


# ------------------------------------------------------------- ALI end to end
@pytest.mark.slow
def test_ali_plain_and_ng_same_fixed_point():
    # non-LTE (collider density lowered 1e4 times): plain ALI converges
    # linearly; classical and adaptive Ng reach the same fixed point sooner
    m = synth.config_model(1, n_points=400)
    m.n_coll = m.n_coll * 1e-4
    rays = O.trace(m)
    ref, ch = O.ali_solve(m, rays, n_iter=90)
    assert ch[-1] < 1e-13
    plain, _ = O.ali_solve(m, rays, n_iter=16)
    cl, _ = O.ali_solve(m, rays, n_iter=16, ng=O.NgClassical(4))
    ad, _ = O.ali_solve(m, rays, n_iter=16, ng=O.NgAdaptive(8))
    assert O.maxrel(cl, ref) < 1e-5
    assert O.maxrel(ad, ref) < 1e-5
    assert O.maxrel(ad, ref) < 0.1 * O.maxrel(plain, ref)
    assert O.maxrel(cl, ref) < 0.1 * O.maxrel(plain, ref)
    assert np.all(ref > 0)
    np.testing.assert_allclose(ref.sum(1), m.n_spec, rtol=1e-12)
