/*
 * Plain FP64 reference for the ray-based line formal solution of Magritte
 * (arXiv 2411.03040).  TEST INFRASTRUCTURE ONLY: nothing in the product path
 * links, loads or calls this file; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark do.
 *
 * Deliberately slow and literal: every (origin, ray pair, frequency bin, line)
 * rebuilds its full ray, evaluates the opacity at every point in the paper's
 * own frequency variables, assembles the second-order (Feautrier) system of
 * the whole ray and solves it by the Thomas algorithm (forward elimination and
 * back substitution), twice: once for u, once for the diagonal of the inverse.
 * OpenMP runs over origin points only.
 * Built with -ffp-contract=off so that no multiply-add is fused: the ray-walk
 * predicates must round exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C     299792458.0
#define OR_KB    1.380649e-23
#define OR_H     6.62607015e-34
#define OR_SQRTPI 1.7724538509055160273

/* ------------------------------------------------------------------------ */
/* Ray walk through the neighbour graph.                                     */
/*                                                                           */
/* The paper defers the tracer to its earlier Magritte papers (Sec. 2, 3.4). */
/* Rule used here: from the current point c (initially the origin o), the    */
/* candidates are the neighbours m of c whose projection                     */
/*   Z_m = (x_m - x_o) . n                                                   */
/* exceeds Z_c; among them take the one with the smallest squared distance   */
/* to the ray line, |(x_m - x_o) - Z_m n|^2, ties to the smaller index.  The */
/* walk ends on a boundary point (kept as the last ray point) or when no     */
/* candidate exists (a stall, except for a boundary origin with no           */
/* candidate, whose half-ray is simply empty).                               */
/* ------------------------------------------------------------------------ */
static int64_t walk(int64_t o, const double *n, const double *pos, const int64_t *off,
                    const int32_t *nb, const uint8_t *bnd, int64_t N,
                    int32_t *out, int *stalled)
{
    int64_t c = o, len = 0;
    double Zc = 0.0;
    const double xo = pos[3 * o], yo = pos[3 * o + 1], zo = pos[3 * o + 2];
    *stalled = 0;
    for (;;) {
        int64_t best = -1;
        double bestd = 0.0, bestZ = 0.0;
        for (int64_t k = off[c]; k < off[c + 1]; ++k) {
            int64_t m = nb[k];
            double dx = pos[3 * m] - xo;
            double dy = pos[3 * m + 1] - yo;
            double dz = pos[3 * m + 2] - zo;
            double Z = dx * n[0] + dy * n[1] + dz * n[2];
            if (!(Z > Zc)) continue;
            double px = dx - Z * n[0];
            double py = dy - Z * n[1];
            double pz = dz - Z * n[2];
            double d2 = px * px + py * py + pz * pz;
            if (best < 0 || d2 < bestd || (d2 == bestd && m < best)) {
                best = m;
                bestd = d2;
                bestZ = Z;
            }
        }
        if (best < 0) {
            if (!(c == o && bnd[o])) *stalled = 1;
            return len;
        }
        if (out) out[len] = (int32_t)best;
        ++len;
        c = best;
        Zc = bestZ;
        if (bnd[best] || len > N) return len;
    }
}

/* Half-ray lengths for every direction r and origin o in orig[0..n_orig)
 * (all points when orig is NULL): len[r*N + o]; other entries are untouched. */
void oracle_trace_lengths(int64_t N, const double *pos, const int64_t *off, const int32_t *nb,
                          const uint8_t *bnd, int32_t R, const double *dirs,
                          int64_t n_orig, const int64_t *orig, int64_t *len, uint8_t *stall)
{
    int64_t n = orig ? n_orig : N;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < (int64_t)R * n; ++t) {
        int64_t r = t / n, o = orig ? orig[t % n] : t % n;
        int st;
        len[r * N + o] = walk(o, dirs + 3 * r, pos, off, nb, bnd, N, NULL, &st);
        stall[r * N + o] = (uint8_t)st;
    }
}

/* Fill the point lists; ray_off has R*N+1 entries (exclusive prefix of lengths). */
void oracle_trace_fill(int64_t N, const double *pos, const int64_t *off, const int32_t *nb,
                       const uint8_t *bnd, int32_t R, const double *dirs,
                       int64_t n_orig, const int64_t *orig, const int64_t *ray_off, int32_t *idx)
{
    int64_t n = orig ? n_orig : N;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < (int64_t)R * n; ++t) {
        int64_t r = t / n, o = orig ? orig[t % n] : t % n;
        int st;
        walk(o, dirs + 3 * r, pos, off, nb, bnd, N, idx + ray_off[r * N + o], &st);
    }
}

/* ------------------------------------------------------------------------ */
/* Planck function B_nu(T) in W m^-2 Hz^-1 sr^-1.                            */
/* ------------------------------------------------------------------------ */
double oracle_planck(double nu, double T)
{
    if (T <= 0.0) return 0.0;
    return 2.0 * OR_H * nu * nu * nu / (OR_C * OR_C) / expm1(OR_H * nu / (OR_KB * T));
}

/* Gaussian line profile (Sec. 4.3, eq. gaussian) at offset (nu - nu_ij). */
static double profile(double offset, double dnu)
{
    double t = offset / dnu;
    return exp(-t * t) / (dnu * OR_SQRTPI);
}

/* ------------------------------------------------------------------------ */
/* Optical depth of one segment between points 0 and 1 (Sec. 4.3).           */
/*   dx      : Euclidean length of the segment                                */
/*   chi0/1  : chi^{ij} at the endpoints (frequency-integrated line opacity)  */
/*   dnu0/1  : line widths at the endpoints (eq. line width)                  */
/*   dnubar  : width from the segment-averaged temperature and turbulence     */
/*   off0/1  : comoving-frame offset from line centre, nu_cmf - nu_ij, of the */
/*             frequency bin at each endpoint                                 */
/*   thr     : switch threshold on |Doppler shift| / dnubar (0.35 in Magritte)*/
/* Below the threshold: trapezoidal rule (eq. trapezoidal rule) of the full   */
/* integrand chi^{ij} phi(nu) evaluated at the endpoints.  At or above it: the */
/* semi-analytic form (eq. semi-analytic): the average of chi^{ij} times the   */
/* exact integral of the Gaussian, (erf(t1) - erf(t0)) / (2 Delta nu), with    */
/* t = offset / dnubar; same-sign tails use erfc to avoid cancellation.       */
/* ------------------------------------------------------------------------ */
double oracle_segment_dtau(double dx, double chi0, double chi1, double dnu0, double dnu1,
                           double dnubar, double off0, double off1, double thr)
{
    double shift = off1 - off0;
    if (fabs(shift) < thr * dnubar) {
        return dx * 0.5 * (chi0 * profile(off0, dnu0) + chi1 * profile(off1, dnu1));
    }
    double t0 = off0 / dnubar, t1 = off1 / dnubar, E;
    if (t0 > 0.0 && t1 > 0.0)
        E = erfc(t0) - erfc(t1);
    else if (t0 < 0.0 && t1 < 0.0)
        E = erfc(-t1) - erfc(-t0);
    else
        E = erf(t1) - erf(t0);
    return dx * 0.5 * (chi0 + chi1) * E / (2.0 * shift);
}

/* Reference optical depth by subdivision (the accuracy study of Sec. 4.3):   */
/* the segment is cut into n equal pieces and the trapezoidal rule applied to */
/* each, with chi^{ij}, the line width and the comoving offset interpolated  */
/* linearly along the segment.  n = 1 is the plain trapezoidal rule.          */
double oracle_segment_dtau_subdiv(double dx, double chi0, double chi1, double dnu0, double dnu1, double off0,
                                  double off1, int n)
{
    double sum = 0.0;
    for (int k = 0; k <= n; ++k) {
        double x = (double)k / n;
        double ch = chi0 + x * (chi1 - chi0);
        double dn = dnu0 + x * (dnu1 - dnu0);
        double of = off0 + x * (off1 - off0);
        double wk = (k == 0 || k == n) ? 0.5 : 1.0;
        sum += wk * ch * profile(of, dn);
    }
    return dx / n * sum;
}

/* ------------------------------------------------------------------------ */
/* Second-order (Feautrier) two-point system on one ray, solved at point io. */
/*                                                                           */
/* Points d = 0..D-1, dtau[d] = optical depth of segment (d, d+1).  The      */
/* tridiagonal system  -A_d u_{d-1} + B_d u_d - C_d u_{d+1} = r_d  is first  */
/* assembled row by row:                                                     */
/*   interior rows (a = dtau[d-1], b = dtau[d]):                             */
/*     A_d = 2/(a(a+b)),  C_d = 2/(b(a+b)),  B_d = 1 + A_d + C_d,  r_d = S_d;*/
/*   end rows (second-order boundary condition of Auer 1967, t the optical   */
/*   depth of the end segment):                                              */
/*     row 0:   B_0 = 1 + 2/t + 2/t^2,  C_0 = 2/t^2,  r_0 = S_0 + (2/t) I_left*/
/*     row D-1: A = 2/t^2,  B = 1 + 2/t + 2/t^2,  r = S_{D-1} + (2/t) I_right.*/
/* It is then solved by the Thomas algorithm over the whole ray: forward     */
/* elimination from row 0 to row D-1 (pivots m_d, reduced right-hand sides   */
/* r'_d), and back substitution from row D-1 down to row io, u_io = x_io.    */
/* Lambda*_oo, the io-th diagonal entry of the inverse matrix, is x_io of a  */
/* second Thomas solve with right-hand side e_io.                            */
/*                                                                           */
/* Pivots.  The textbook pivot m_d = B_d - A_d C_{d-1} / m_{d-1} subtracts   */
/* numbers of size 1/dtau^2 whose difference is of order 1 + 2/dtau: for    */
/* optically thin segments (dtau^2 below the rounding unit, common in the    */
/* line wings) it loses every digit of the row's excess.  Each row's excess  */
/* B_d - A_d - C_d is known exactly (1 inside, 1 + 2/t at the ends), so the  */
/* same pivot is evaluated as                                                */
/*   m_d = x_d + C_d,  x_d = (B_d - A_d - C_d) + A_d x_{d-1} / m_{d-1},      */
/* with x_d the excess of the reduced row (x_0 = 1 + 2/t): algebraically the  */
/* textbook value, formed from positive terms only.  The forward and back    */
/* substitutions add positive terms too (all A, C, S, I >= 0).               */
/* D == 1: no system; u = background, L = 0.                                 */
/* ------------------------------------------------------------------------ */
static void thomas_at(int64_t D, const double *dtau, const double *S, double I_left, double I_right, int64_t io,
                      double *w, double *u_out, double *L_out)
{
    double *A = w, *C = w + D, *X = w + 2 * D, *R = w + 3 * D, *m = w + 4 * D, *rp = w + 5 * D;
    /* assemble: sub-diagonal A, super-diagonal C, row excess X = B - A - C, right-hand side R */
    for (int64_t d = 0; d < D; ++d) {
        if (d == 0) {
            double t = dtau[0];
            A[d] = 0.0;
            C[d] = 2.0 / (t * t);
            X[d] = 1.0 + 2.0 / t;
            R[d] = S[0] + 2.0 * I_left / t;
        } else if (d == D - 1) {
            double t = dtau[D - 2];
            A[d] = 2.0 / (t * t);
            C[d] = 0.0;
            X[d] = 1.0 + 2.0 / t;
            R[d] = S[D - 1] + 2.0 * I_right / t;
        } else {
            double a = dtau[d - 1], b = dtau[d];
            A[d] = 2.0 / (a * (a + b));
            C[d] = 2.0 / (b * (a + b));
            X[d] = 1.0;
            R[d] = S[d];
        }
    }
    /* forward elimination: m[d] pivot, X[d] reduced excess, rp[d] reduced rhs */
    for (int64_t d = 0; d < D; ++d) {
        if (d > 0) X[d] = X[d] + A[d] * (X[d - 1] / m[d - 1]);
        m[d] = X[d] + C[d];
        rp[d] = d > 0 ? (R[d] + A[d] * rp[d - 1]) / m[d] : R[d] / m[d];
    }
    /* back substitution x_d = r'_d + (C_d / m_d) x_{d+1}, from D-1 to io */
    double x = rp[D - 1];
    for (int64_t d = D - 2; d >= io; --d) x = rp[d] + C[d] / m[d] * x;
    *u_out = x;
    /* second solve, right-hand side e_io: r'_d = 0 below io */
    double q = 0.0;
    for (int64_t d = io; d < D; ++d) {
        q = d == io ? 1.0 / m[d] : A[d] * q / m[d];
        rp[d] = q;
    }
    x = rp[D - 1];
    for (int64_t d = D - 2; d >= io; --d) x = rp[d] + C[d] / m[d] * x;
    *L_out = x;
}

void oracle_feautrier_at(int64_t D, const double *dtau, const double *S,
                         double I_left, double I_right, int64_t io,
                         double *u_out, double *L_out)
{
    if (D <= 1) {
        *u_out = 0.5 * (I_left + I_right);
        *L_out = 0.0;
        return;
    }
    double *w = malloc(sizeof(double) * 6 * (size_t)D);
    thomas_at(D, dtau, S, I_left, I_right, io, w, u_out, L_out);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* J-bar and Lambda* at a list of origin points.                             */
/*                                                                           */
/* For origin o, ray pair (r, rb) (n_rb = -n_r), GH bin q and line ij:        */
/*  - the full ray runs from the far end of the rb half-ray through o to the  */
/*    far end of the r half-ray (points from the trace);                      */
/*  - the bin frequency is nu_q = nu_ij + x_q dnu_ij(o), centred on the line  */
/*    in o's comoving frame;                                                  */
/*  - a point c on half-ray h sees the photons travelling toward o at the     */
/*    comoving frequency nu_q (1 + n_h . (v_c - v_o)/c), so its offset from   */
/*    line centre is x_q dnu_ij(o) + nu_q n_h . (v_c - v_o)/c;                */
/*  - segment optical depths follow oracle_segment_dtau (or, with subdiv > 0, */
/*    oracle_segment_dtau_subdiv), floored at tau_min;                        */
/*  - both ends see the background I_bg = B_nu(T_bg) at nu_q;                 */
/*  - Jbar  += (2/R) w_q u_o,  Lstar += (2/R) w_q L*_oo  (w_q normalised GH). */
/* width_mode 0: dnubar from the averaged T and vturb^2; 1: mean of widths.   */
/* chi and S are [M][N] (SI); outputs are [n_orig][M].                        */
/* ------------------------------------------------------------------------ */
void oracle_formal_solve(int64_t N, const double *pos, const double *vel, const double *temp,
                         const double *vturb2, double mol_mass,
                         int32_t R, const double *dirs, int32_t P, const int32_t *pairs,
                         const int64_t *ray_off, const int32_t *ray_idx,
                         int32_t M, const double *nu, const double *chi, const double *S,
                         int32_t Q, const double *xq, const double *wq, double T_bg,
                         double tau_min, double thr, int width_mode, int subdiv,
                         int64_t n_orig, const int64_t *orig, double *Jbar, double *Lstar)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t io_ = 0; io_ < n_orig; ++io_) {
        int64_t o = orig[io_];
        /* longest full ray over the pairs */
        int64_t Dmax = 1;
        for (int32_t p = 0; p < P; ++p) {
            int64_t r = pairs[2 * p], rb = pairs[2 * p + 1];
            int64_t D = 1 + (ray_off[r * N + o + 1] - ray_off[r * N + o])
                          + (ray_off[rb * N + o + 1] - ray_off[rb * N + o]);
            if (D > Dmax) Dmax = D;
        }
        int64_t *pt = malloc(sizeof(int64_t) * Dmax);
        double *beta = malloc(sizeof(double) * Dmax);
        double *dx = malloc(sizeof(double) * Dmax);
        double *dnu = malloc(sizeof(double) * Dmax);
        double *off = malloc(sizeof(double) * Dmax);
        double *dtau = malloc(sizeof(double) * Dmax);
        double *Sd = malloc(sizeof(double) * Dmax);
        double *work = malloc(sizeof(double) * 6 * Dmax);
        for (int32_t m = 0; m < M; ++m) {
            Jbar[io_ * M + m] = 0.0;
            Lstar[io_ * M + m] = 0.0;
        }
        for (int32_t p = 0; p < P; ++p) {
            int64_t r = pairs[2 * p], rb = pairs[2 * p + 1];
            const double *nr = dirs + 3 * r, *nrb = dirs + 3 * rb;
            int64_t b0 = ray_off[rb * N + o], nrbl = ray_off[rb * N + o + 1] - b0;
            int64_t f0 = ray_off[r * N + o], nrl = ray_off[r * N + o + 1] - f0;
            int64_t D = 1 + nrbl + nrl, d_o = nrbl;
            /* assemble the full ray: far end of rb ... o ... far end of r */
            for (int64_t k = 0; k < nrbl; ++k) {
                int64_t c = ray_idx[b0 + (nrbl - 1 - k)];
                pt[k] = c;
                beta[k] = (nrb[0] * (vel[3 * c] - vel[3 * o]) + nrb[1] * (vel[3 * c + 1] - vel[3 * o + 1])
                           + nrb[2] * (vel[3 * c + 2] - vel[3 * o + 2])) / OR_C;
            }
            pt[d_o] = o;
            beta[d_o] = 0.0;
            for (int64_t k = 0; k < nrl; ++k) {
                int64_t c = ray_idx[f0 + k];
                pt[d_o + 1 + k] = c;
                beta[d_o + 1 + k] = (nr[0] * (vel[3 * c] - vel[3 * o]) + nr[1] * (vel[3 * c + 1] - vel[3 * o + 1])
                                     + nr[2] * (vel[3 * c + 2] - vel[3 * o + 2])) / OR_C;
            }
            for (int64_t d = 0; d + 1 < D; ++d) {
                int64_t a = pt[d], b = pt[d + 1];
                double ex = pos[3 * b] - pos[3 * a], ey = pos[3 * b + 1] - pos[3 * a + 1],
                       ez = pos[3 * b + 2] - pos[3 * a + 2];
                dx[d] = sqrt(ex * ex + ey * ey + ez * ez);
            }
            for (int32_t m = 0; m < M; ++m) {
                double nij = nu[m];
                for (int64_t d = 0; d < D; ++d) {
                    int64_t c = pt[d];
                    dnu[d] = nij / OR_C * sqrt(2.0 * OR_KB * temp[c] / mol_mass + vturb2[c]);
                    Sd[d] = S[(int64_t)m * N + c];
                }
                for (int32_t q = 0; q < Q; ++q) {
                    double nuq = nij + xq[q] * dnu[d_o];
                    double Ibg = oracle_planck(nuq, T_bg);
                    for (int64_t d = 0; d < D; ++d)
                        off[d] = xq[q] * dnu[d_o] + nuq * beta[d];
                    for (int64_t d = 0; d + 1 < D; ++d) {
                        int64_t a = pt[d], b = pt[d + 1];
                        double dnb;
                        if (width_mode == 0) {
                            double Tb = 0.5 * (temp[a] + temp[b]);
                            double vb = 0.5 * (vturb2[a] + vturb2[b]);
                            dnb = nij / OR_C * sqrt(2.0 * OR_KB * Tb / mol_mass + vb);
                        } else {
                            dnb = 0.5 * (dnu[d] + dnu[d + 1]);
                        }
                        double t = subdiv > 0
                            ? oracle_segment_dtau_subdiv(dx[d], chi[(int64_t)m * N + a], chi[(int64_t)m * N + b],
                                                         dnu[d], dnu[d + 1], off[d], off[d + 1], subdiv)
                            : oracle_segment_dtau(dx[d], chi[(int64_t)m * N + a], chi[(int64_t)m * N + b],
                                                  dnu[d], dnu[d + 1], dnb, off[d], off[d + 1], thr);
                        dtau[d] = t > tau_min ? t : tau_min;
                    }
                    double u, L;
                    if (D <= 1) {
                        u = Ibg;
                        L = 0.0;
                    } else {
                        thomas_at(D, dtau, Sd, Ibg, Ibg, d_o, work, &u, &L);
                    }
                    Jbar[io_ * M + m] += (2.0 / R) * wq[q] * u;
                    Lstar[io_ * M + m] += (2.0 / R) * wq[q] * L;
                }
            }
        }
        free(pt); free(beta); free(dx); free(dnu); free(off); free(dtau); free(Sd); free(work);
    }
}

/* ------------------------------------------------------------------------ */
/* Synthetic image (Listing 3, compute_image_new: an image along a ray      */
/* direction with N_pix_x x N_pix_y pixels).  The paper gives no algorithm; */
/* readings used here:                                                       */
/*  - n is the unit direction toward the observer; the image plane basis is  */
/*    e1 = unit(a x n) with a the coordinate axis least aligned with n       */
/*    (lowest index on ties), e2 = n x e1;                                   */
/*  - the pixel grid is square and covers the projections of all points:     */
/*    centre (c1, c2) = mid-range of the projections, half-width H = half    */
/*    the larger range; pixel (i, j) has reference point                     */
/*    p = (c1 - H + (i + 1/2) 2H/npx) e1 + (c2 - H + (j + 1/2) 2H/npy) e2;   */
/*  - the pixel's anchor is the point closest to the pixel line (p, n)       */
/*    (squared perpendicular distance, ties to the smaller index);           */
/*  - the pixel ray is the walk (rule of walk() above, distances to the      */
/*    pixel line, Z measured from p) from the anchor along -n, reversed,     */
/*    then the anchor, then the walk along +n.                               */
/* Everything in FP64, expressions in the order written, no FMA.             */
/* ------------------------------------------------------------------------ */
void oracle_image_frame(int64_t N, const double *pos, const double *n, int32_t npx, int32_t npy,
                        double *e1, double *e2, double *ref /* [npy*npx][3] */)
{
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (fabs(n[k]) < fabs(n[ax])) ax = k;
    double a[3] = {0.0, 0.0, 0.0};
    a[ax] = 1.0;
    double c[3] = {a[1] * n[2] - a[2] * n[1], a[2] * n[0] - a[0] * n[2], a[0] * n[1] - a[1] * n[0]};
    double cl = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    for (int k = 0; k < 3; ++k) e1[k] = c[k] / cl;
    e2[0] = n[1] * e1[2] - n[2] * e1[1];
    e2[1] = n[2] * e1[0] - n[0] * e1[2];
    e2[2] = n[0] * e1[1] - n[1] * e1[0];
    double lo1 = 1e300, hi1 = -1e300, lo2 = 1e300, hi2 = -1e300;
    for (int64_t i = 0; i < N; ++i) {
        double s1 = pos[3 * i] * e1[0] + pos[3 * i + 1] * e1[1] + pos[3 * i + 2] * e1[2];
        double s2 = pos[3 * i] * e2[0] + pos[3 * i + 1] * e2[1] + pos[3 * i + 2] * e2[2];
        if (s1 < lo1) lo1 = s1;
        if (s1 > hi1) hi1 = s1;
        if (s2 < lo2) lo2 = s2;
        if (s2 > hi2) hi2 = s2;
    }
    double c1 = 0.5 * (lo1 + hi1), c2 = 0.5 * (lo2 + hi2);
    double H = 0.5 * ((hi1 - lo1) > (hi2 - lo2) ? (hi1 - lo1) : (hi2 - lo2));
    for (int32_t j = 0; j < npy; ++j)
        for (int32_t i = 0; i < npx; ++i) {
            double t1 = c1 - H + (i + 0.5) * (2.0 * H / npx);
            double t2 = c2 - H + (j + 0.5) * (2.0 * H / npy);
            double *p = ref + 3 * ((int64_t)j * npx + i);
            for (int k = 0; k < 3; ++k) p[k] = t1 * e1[k] + t2 * e2[k];
        }
}

/* Walk of an image half-ray: reference point p, direction d (unit), start
 * point a with projection Za = (x_a - p).d; same rule as walk(). */
static int64_t walk_ref(int64_t a, const double *p, const double *d, double Za, const double *pos,
                        const int64_t *off, const int32_t *nb, const uint8_t *bnd, int64_t N, int32_t *out)
{
    int64_t c = a, len = 0;
    double Zc = Za;
    for (;;) {
        int64_t best = -1;
        double bestd = 0.0, bestZ = 0.0;
        for (int64_t k = off[c]; k < off[c + 1]; ++k) {
            int64_t m = nb[k];
            double dx = pos[3 * m] - p[0];
            double dy = pos[3 * m + 1] - p[1];
            double dz = pos[3 * m + 2] - p[2];
            double Z = dx * d[0] + dy * d[1] + dz * d[2];
            if (!(Z > Zc)) continue;
            double px = dx - Z * d[0];
            double py = dy - Z * d[1];
            double pz = dz - Z * d[2];
            double d2 = px * px + py * py + pz * pz;
            if (best < 0 || d2 < bestd || (d2 == bestd && m < best)) {
                best = m;
                bestd = d2;
                bestZ = Z;
            }
        }
        if (best < 0) return len;
        if (out) out[len] = (int32_t)best;
        ++len;
        c = best;
        Zc = bestZ;
        if (bnd[best] || len > N) return len;
    }
}

/* Anchor (closest point to the pixel line) and the two half-ray lengths of
 * each pixel; with `pts` the full rays are written at ray_off. */
void oracle_image_rays(int64_t N, const double *pos, const int64_t *off, const int32_t *nb, const uint8_t *bnd,
                       const double *n, int64_t npix, const double *ref, int32_t *anchor, int64_t *nfar,
                       int64_t *nnear, const int64_t *ray_off, int32_t *pts)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
        const double *p = ref + 3 * q;
        int64_t best = -1;
        double bestd = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double dx = pos[3 * i] - p[0];
            double dy = pos[3 * i + 1] - p[1];
            double dz = pos[3 * i + 2] - p[2];
            double Z = dx * n[0] + dy * n[1] + dz * n[2];
            double px = dx - Z * n[0];
            double py = dy - Z * n[1];
            double pz = dz - Z * n[2];
            double d2 = px * px + py * py + pz * pz;
            if (best < 0 || d2 < bestd) {
                best = i;
                bestd = d2;
            }
        }
        anchor[q] = (int32_t)best;
        double m[3] = {-n[0], -n[1], -n[2]};
        const double *xa = pos + 3 * best;
        double Zf = (xa[0] - p[0]) * m[0] + (xa[1] - p[1]) * m[1] + (xa[2] - p[2]) * m[2];
        double Zn = (xa[0] - p[0]) * n[0] + (xa[1] - p[1]) * n[1] + (xa[2] - p[2]) * n[2];
        if (!pts) {
            nfar[q] = walk_ref(best, p, m, Zf, pos, off, nb, bnd, N, NULL);
            nnear[q] = walk_ref(best, p, n, Zn, pos, off, nb, bnd, N, NULL);
        } else {
            int32_t *r = pts + ray_off[q];
            int64_t nf = walk_ref(best, p, m, Zf, pos, off, nb, bnd, N, r);
            for (int64_t k = 0; k < nf / 2; ++k) {          /* far half outward -> inward */
                int32_t t = r[k];
                r[k] = r[nf - 1 - k];
                r[nf - 1 - k] = t;
            }
            r[nf] = (int32_t)best;
            walk_ref(best, p, n, Zn, pos, off, nb, bnd, N, r + nf + 1);
        }
    }
}

/* First-order (short-characteristics) formal solution toward the observer
 * along one image ray for one channel.  Points P_0 (far) .. P_D (near);
 * with piecewise-linear S in optical depth the exact update over a segment
 * of depth t is I <- e^-t I + w0(t) S_far + w1(t) S_near,
 *   w0 = (1 - e^-t)/t - e^-t,  w1 = 1 - (1 - e^-t)/t,
 * evaluated by their Taylor series for t < 1e-3.  The segment depth follows
 * oracle_segment_dtau at the comoving offsets nu_f (1 - n.v/c) - nu_line. */
void oracle_image_weights(double t, double *E, double *w0, double *w1)
{
    *E = exp(-t);
    if (t < 1e-3) {
        /* (1 - e^-t)/t = 1 - t/2 + t^2/6 - t^3/24 + t^4/120 */
        double g = 1.0 - t / 2.0 + t * t / 6.0 - t * t * t / 24.0 + t * t * t * t / 120.0;
        *w0 = g - *E;
        *w1 = 1.0 - g;
    } else {
        double g = (1.0 - *E) / t;
        *w0 = g - *E;
        *w1 = 1.0 - g;
    }
}

void oracle_image_solve(int64_t N, const double *pos, const double *vel, const double *temp, const double *vturb2,
                        double mol_mass, const double *n, int32_t M, const double *nu_line, const double *chi,
                        const double *S, double T_bg, double thr, int64_t npix, const int64_t *ray_off,
                        const int32_t *pts, int32_t nfreq, const double *nu_f, double *image /* [nfreq][npix] */)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < npix; ++q) {
        const int32_t *r = pts + ray_off[q];
        int64_t D = ray_off[q + 1] - ray_off[q] - 1;   /* segments */
        for (int32_t f = 0; f < nfreq; ++f) {
            double nu = nu_f[f];
            int32_t l = 0;                              /* nearest line */
            for (int32_t k = 1; k < M; ++k)
                if (fabs(nu - nu_line[k]) < fabs(nu - nu_line[l])) l = k;
            double nl = nu_line[l];
            double I = oracle_planck(nu, T_bg);
            for (int64_t d = 0; d < D; ++d) {
                int64_t a = r[d], b = r[d + 1];
                double ex = pos[3 * b] - pos[3 * a], ey = pos[3 * b + 1] - pos[3 * a + 1],
                       ez = pos[3 * b + 2] - pos[3 * a + 2];
                double dx = sqrt(ex * ex + ey * ey + ez * ez);
                double va = (n[0] * vel[3 * a] + n[1] * vel[3 * a + 1] + n[2] * vel[3 * a + 2]) / OR_C;
                double vb = (n[0] * vel[3 * b] + n[1] * vel[3 * b + 1] + n[2] * vel[3 * b + 2]) / OR_C;
                double offa = nu * (1.0 - va) - nl, offb = nu * (1.0 - vb) - nl;
                double dna = nl / OR_C * sqrt(2.0 * OR_KB * temp[a] / mol_mass + vturb2[a]);
                double dnb = nl / OR_C * sqrt(2.0 * OR_KB * temp[b] / mol_mass + vturb2[b]);
                double Tb = 0.5 * (temp[a] + temp[b]), vb2 = 0.5 * (vturb2[a] + vturb2[b]);
                double dnbar = nl / OR_C * sqrt(2.0 * OR_KB * Tb / mol_mass + vb2);
                double t = oracle_segment_dtau(dx, chi[(int64_t)l * N + a], chi[(int64_t)l * N + b], dna, dnb, dnbar,
                                               offa, offb, thr);
                double E, w0, w1;
                oracle_image_weights(t, &E, &w0, &w1);
                I = E * I + w0 * S[(int64_t)l * N + a] + w1 * S[(int64_t)l * N + b];
            }
            image[(int64_t)f * npix + q] = I;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Gradient of the image (reverse sweep of oracle_image_solve).              */
/*                                                                           */
/* For a loss L = sum over channels and pixels of gimg * image, returns       */
/* dL/d log T_p, dL/d log n_spec,p and dL/d (n . v_p) for every point p.      */
/* Readings (the paper does not differentiate the image): populations are    */
/* held as fractions of n_spec, so chi^{ij} scales with n_spec and S does not */
/* change; T enters only through the Doppler widths (of the end points and    */
/* of the segment's averaged width); each segment keeps the branch           */
/* (trapezoid or semi-analytic) that the forward solve takes.                */
/* Plain reverse mode, FP64: every (pixel, channel) reruns its forward solve, */
/* keeping the intensity at every point, then walks back from the near end,  */
/* lambda = dL/dI, lambda_d = e^-t lambda_{d+1}, and adds                     */
/* lambda_{d+1} dI_{d+1}/dt dt/d(field) to the segment's two end points.      */
/* ------------------------------------------------------------------------ */

/* Partial derivatives of oracle_segment_dtau with its branch held:
 * g[0..6] = dt / d(chi0, chi1, dnu0, dnu1, dnubar, off0, off1). */
static void segment_dtau_grad(double dx, double chi0, double chi1, double dnu0, double dnu1, double dnubar,
                              double off0, double off1, double thr, double *g)
{
    double shift = off1 - off0;
    for (int k = 0; k < 7; ++k) g[k] = 0.0;
    if (fabs(shift) < thr * dnubar) {
        /* t = dx/2 (chi0 phi(off0, dnu0) + chi1 phi(off1, dnu1)),
         * phi(o, d) = exp(-(o/d)^2) / (d sqrt(pi)):
         * dphi/do = phi (-2 o / d^2),  dphi/dd = phi (2 o^2 / d^3 - 1/d) */
        double p0 = profile(off0, dnu0), p1 = profile(off1, dnu1);
        g[0] = 0.5 * dx * p0;
        g[1] = 0.5 * dx * p1;
        g[2] = 0.5 * dx * chi0 * p0 * (2.0 * off0 * off0 / (dnu0 * dnu0 * dnu0) - 1.0 / dnu0);
        g[3] = 0.5 * dx * chi1 * p1 * (2.0 * off1 * off1 / (dnu1 * dnu1 * dnu1) - 1.0 / dnu1);
        g[5] = 0.5 * dx * chi0 * p0 * (-2.0 * off0 / (dnu0 * dnu0));
        g[6] = 0.5 * dx * chi1 * p1 * (-2.0 * off1 / (dnu1 * dnu1));
        return;
    }
    /* t = dx/2 (chi0 + chi1) E / (2 shift),  E = erf(u1) - erf(u0),  u = off / dnubar;
     * dE/du = +-(2/sqrt(pi)) exp(-u^2) */
    double u0 = off0 / dnubar, u1 = off1 / dnubar, E;
    if (u0 > 0.0 && u1 > 0.0)
        E = erfc(u0) - erfc(u1);
    else if (u0 < 0.0 && u1 < 0.0)
        E = erfc(-u1) - erfc(-u0);
    else
        E = erf(u1) - erf(u0);
    double c = 0.5 * dx * (chi0 + chi1);
    double dE_du0 = -2.0 / OR_SQRTPI * exp(-u0 * u0), dE_du1 = 2.0 / OR_SQRTPI * exp(-u1 * u1);
    g[0] = g[1] = 0.5 * dx * E / (2.0 * shift);
    g[4] = c / (2.0 * shift) * (dE_du0 * (-u0 / dnubar) + dE_du1 * (-u1 / dnubar));
    g[5] = c / (2.0 * shift) * dE_du0 / dnubar + c * E / (2.0 * shift * shift);
    g[6] = c / (2.0 * shift) * dE_du1 / dnubar - c * E / (2.0 * shift * shift);
}

/* d/dt of the update I' = e^-t I + w0 S0 + w1 S1 (oracle_image_weights):
 * with g(t) = (1 - e^-t)/t, w0 = g - e^-t, w1 = 1 - g,
 * dI'/dt = -e^-t I + (g' + e^-t) S0 - g' S1,  g' = (t e^-t - 1 + e^-t)/t^2,
 * by its Taylor series -1/2 + t/3 - t^2/8 + t^3/30 for t < 1e-3. */
static double image_update_dt(double t, double I, double S0, double S1)
{
    double E = exp(-t), gp;
    if (t < 1e-3)
        gp = -0.5 + t / 3.0 - t * t / 8.0 + t * t * t / 30.0;
    else
        gp = (t * E - 1.0 + E) / (t * t);
    return -E * I + (gp + E) * S0 - gp * S1;
}

void oracle_image_adjoint(int64_t N, const double *pos, const double *vel, const double *temp, const double *vturb2,
                          double mol_mass, const double *n, int32_t M, const double *nu_line, const double *chi,
                          const double *S, double T_bg, double thr, int64_t npix, const int64_t *ray_off,
                          const int32_t *pts, int32_t nfreq, const double *nu_f, const double *gimg,
                          double *g_logT, double *g_logn, double *g_vlos)
{
    for (int64_t p = 0; p < N; ++p) g_logT[p] = g_logn[p] = g_vlos[p] = 0.0;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < npix; ++q) {
        const int32_t *r = pts + ray_off[q];
        int64_t D = ray_off[q + 1] - ray_off[q] - 1;   /* segments */
        double *Iv = malloc(sizeof(double) * (size_t)(D + 1));
        for (int32_t f = 0; f < nfreq; ++f) {
            double lam = gimg[(int64_t)f * npix + q];
            if (lam == 0.0) continue;
            double nu = nu_f[f];
            int32_t l = 0;
            for (int32_t k = 1; k < M; ++k)
                if (fabs(nu - nu_line[k]) < fabs(nu - nu_line[l])) l = k;
            double nl = nu_line[l];
            /* forward, keeping I at every point */
            Iv[0] = oracle_planck(nu, T_bg);
            for (int64_t d = 0; d < D; ++d) {
                int64_t a = r[d], b = r[d + 1];
                double ex = pos[3 * b] - pos[3 * a], ey = pos[3 * b + 1] - pos[3 * a + 1],
                       ez = pos[3 * b + 2] - pos[3 * a + 2];
                double dx = sqrt(ex * ex + ey * ey + ez * ez);
                double va = (n[0] * vel[3 * a] + n[1] * vel[3 * a + 1] + n[2] * vel[3 * a + 2]) / OR_C;
                double vb = (n[0] * vel[3 * b] + n[1] * vel[3 * b + 1] + n[2] * vel[3 * b + 2]) / OR_C;
                double dna = nl / OR_C * sqrt(2.0 * OR_KB * temp[a] / mol_mass + vturb2[a]);
                double dnb = nl / OR_C * sqrt(2.0 * OR_KB * temp[b] / mol_mass + vturb2[b]);
                double Tb = 0.5 * (temp[a] + temp[b]), vb2 = 0.5 * (vturb2[a] + vturb2[b]);
                double dnbar = nl / OR_C * sqrt(2.0 * OR_KB * Tb / mol_mass + vb2);
                double t = oracle_segment_dtau(dx, chi[(int64_t)l * N + a], chi[(int64_t)l * N + b], dna, dnb, dnbar,
                                               nu * (1.0 - va) - nl, nu * (1.0 - vb) - nl, thr);
                double E, w0, w1;
                oracle_image_weights(t, &E, &w0, &w1);
                Iv[d + 1] = E * Iv[d] + w0 * S[(int64_t)l * N + a] + w1 * S[(int64_t)l * N + b];
            }
            /* reverse */
            for (int64_t d = D - 1; d >= 0; --d) {
                int64_t a = r[d], b = r[d + 1];
                double ex = pos[3 * b] - pos[3 * a], ey = pos[3 * b + 1] - pos[3 * a + 1],
                       ez = pos[3 * b + 2] - pos[3 * a + 2];
                double dx = sqrt(ex * ex + ey * ey + ez * ez);
                double va = (n[0] * vel[3 * a] + n[1] * vel[3 * a + 1] + n[2] * vel[3 * a + 2]) / OR_C;
                double vb = (n[0] * vel[3 * b] + n[1] * vel[3 * b + 1] + n[2] * vel[3 * b + 2]) / OR_C;
                double Aa = 2.0 * OR_KB * temp[a] / mol_mass + vturb2[a];
                double Ab = 2.0 * OR_KB * temp[b] / mol_mass + vturb2[b];
                double Abar = 2.0 * OR_KB * (0.5 * (temp[a] + temp[b])) / mol_mass + 0.5 * (vturb2[a] + vturb2[b]);
                double dna = nl / OR_C * sqrt(Aa), dnb = nl / OR_C * sqrt(Ab), dnbar = nl / OR_C * sqrt(Abar);
                double ca = chi[(int64_t)l * N + a], cb = chi[(int64_t)l * N + b];
                double oa = nu * (1.0 - va) - nl, ob = nu * (1.0 - vb) - nl;
                double t = oracle_segment_dtau(dx, ca, cb, dna, dnb, dnbar, oa, ob, thr);
                double tb = lam * image_update_dt(t, Iv[d], S[(int64_t)l * N + a], S[(int64_t)l * N + b]);
                double g[7];
                segment_dtau_grad(dx, ca, cb, dna, dnb, dnbar, oa, ob, thr, g);
                /* chain to the point fields */
                double kTa = OR_KB * temp[a] / mol_mass, kTb = OR_KB * temp[b] / mol_mass;
                double dlogTa = g[2] * dna * kTa / Aa + g[4] * dnbar * kTa / (2.0 * Abar);
                double dlogTb = g[3] * dnb * kTb / Ab + g[4] * dnbar * kTb / (2.0 * Abar);
                #pragma omp atomic
                g_logT[a] += tb * dlogTa;
                #pragma omp atomic
                g_logT[b] += tb * dlogTb;
                #pragma omp atomic
                g_logn[a] += tb * g[0] * ca;
                #pragma omp atomic
                g_logn[b] += tb * g[1] * cb;
                #pragma omp atomic
                g_vlos[a] += tb * g[5] * (-nu / OR_C);
                #pragma omp atomic
                g_vlos[b] += tb * g[6] * (-nu / OR_C);
                lam *= exp(-t);
            }
        }
        free(Iv);
    }
}

/* Branch of every segment of every (channel, pixel ray) in the forward solve:
 * out[f * n_seg + s] = 1 for the trapezoid, 0 for the semi-analytic form, with
 * s the segment's index over all rays (ray q's segments start at
 * ray_off[q] - q). */
void oracle_image_branches(int64_t N, const double *pos, const double *vel, const double *temp, const double *vturb2,
                           double mol_mass, const double *n, int32_t M, const double *nu_line, double thr,
                           int64_t npix, const int64_t *ray_off, const int32_t *pts, int32_t nfreq,
                           const double *nu_f, uint8_t *out)
{
    int64_t n_seg = ray_off[npix] - npix;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
        const int32_t *r = pts + ray_off[q];
        int64_t D = ray_off[q + 1] - ray_off[q] - 1, s0 = ray_off[q] - q;
        for (int32_t f = 0; f < nfreq; ++f) {
            double nu = nu_f[f];
            int32_t l = 0;
            for (int32_t k = 1; k < M; ++k)
                if (fabs(nu - nu_line[k]) < fabs(nu - nu_line[l])) l = k;
            double nl = nu_line[l];
            for (int64_t d = 0; d < D; ++d) {
                int64_t a = r[d], b = r[d + 1];
                double va = (n[0] * vel[3 * a] + n[1] * vel[3 * a + 1] + n[2] * vel[3 * a + 2]) / OR_C;
                double vb = (n[0] * vel[3 * b] + n[1] * vel[3 * b + 1] + n[2] * vel[3 * b + 2]) / OR_C;
                double Tb = 0.5 * (temp[a] + temp[b]), vb2 = 0.5 * (vturb2[a] + vturb2[b]);
                double dnbar = nl / OR_C * sqrt(2.0 * OR_KB * Tb / mol_mass + vb2);
                double shift = (nu * (1.0 - vb) - nl) - (nu * (1.0 - va) - nl);
                out[(int64_t)f * n_seg + s0 + d] = fabs(shift) < thr * dnbar ? 1 : 0;
            }
        }
    }
}
