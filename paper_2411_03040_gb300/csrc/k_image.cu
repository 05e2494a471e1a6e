// Synthetic image of the model along a line of sight (Listing 3,
// compute_image_new) and its adjoint with respect to the per-point
// temperature, species density and velocity.
//
// Each pixel ray (k_geom.cu: anchor point and two walks) runs from its far end
// P_0 to its near end P_D.  For channel frequency nu_f (observer frame) and
// the line nearest to it, a point c sees the comoving offset
//   z_c = (nu_f / nu_l)(1 - n.v_c/c) - 1      (in units of nu_l),
// the Gaussian opacity chi~_c exp(-(z_c/w_c)^2) and the source function S_c.
// Segment optical depths follow the formal solution's rule (Sec. 4.3:
// trapezoid below the switch, semi-analytic erf form at or above it), and the
// intensity toward the observer is integrated with a source linear in optical
// depth over each segment (exact for such a source):
//   I_{d+1} = e^-t I_d + w0(t) S_d + w1(t) S_{d+1},
//   w0 = (1 - e^-t)/t - e^-t,  w1 = 1 - (1 - e^-t)/t,
// from I_0 = B_nu_f(T_bg).  All in FP32 in the line's scaled units (S / U_line).
//
// Adjoint: for a loss with dL/dI given per pixel and channel, the reverse
// sweep carries lambda_d = dL/dI_d (lambda_d = e^-t lambda_{d+1}) and adds
// lambda_{d+1} dI_{d+1}/dt_d dt_d/dtheta to the gradients of the segment's two
// end points, theta = (log T, log n_spec, n.v/c).  Populations are held as
// fractions of n_spec, so chi~ scales with n_spec and S does not change; T
// enters through the Doppler width.  The forward intensities are kept at 64
// checkpoints per ray and recomputed one segment block at a time in reverse.
#include <cmath>
#include <vector>

#include "mgt_common.cuh"
#include "mgt_erfc.cuh"

namespace mgt {

namespace {

constexpr int kCk = 64;            // intensity checkpoints per ray (adjoint)
constexpr int kBlk = 64;           // segments per checkpoint block, so rays up to kCk * kBlk segments
constexpr float kImgBand = 2e-4f;  // |du| this close (relative) to the switch is re-decided in FP64
constexpr float kSqrtPiF = 1.77245385090551602730f;
constexpr int kImgStage = 128;     // pixel-ray points staged in shared memory at a time
static_assert(kBlk + 1 <= kImgStage, "one adjoint checkpoint block must fit one stage");

struct Chan;

struct ImgArgs {
    int64_t N, npix;
    int32_t M, Mpad, RS, nfreq, width_mode;
    const float *line;        // [N][RS] rows: chi~' of every line, S' of every line, w, 1/w
    const float *pos_hl, *vel_hl;
    const double *vel, *w64, *temp;
    const double *line_tab;   // [8][Mpad]: nu, A, Bul, Blu, nbgmax, h nu/k T_bg, U_line, unused
    const int64_t *off;
    const int32_t *pts;
    double fmin, fstep;       // nu_f = fmin + f fstep
    double n64[3];
    float n0, n1, n2;
    float inv_Lunit;
    double thr;
    float theta_k;            // k_B / (m c^2): theta = theta_k T = d w / d log T * w
    const Chan *chan;         // [nfreq] per-channel constants (k_image_chan)
    float *out;               // [nfreq][npix] intensity (SI)
    const float *gout;        // [nfreq][npix] dL/dI (SI)
    double *g_logT, *g_logn, *g_beta;
};

struct Chan {
    int l;
    float rf, rf1, I0, U;
    double rf64;
};

__device__ Chan channel(const ImgArgs &a, int f)
{
    Chan c;
    const double nu = a.fmin + f * a.fstep;
    int l = 0;
    for (int k = 1; k < a.M; ++k)
        if (fabs(nu - a.line_tab[k]) < fabs(nu - a.line_tab[l])) l = k;
    c.l = l;
    const double r = nu / a.line_tab[l];
    c.rf64 = r;
    c.rf = (float)r;
    c.rf1 = (float)(r - 1.0);
    const double hk = a.line_tab[5 * a.Mpad + l], nbg = a.line_tab[4 * a.Mpad + l];
    c.I0 = hk > 0.0 ? (float)(r * r * r / expm1(hk * r) / nbg) : 0.0f;
    c.U = (float)a.line_tab[6 * a.Mpad + l];
    return c;
}

struct Pt {
    int64_t c;
    float chi, S, w, winv, beta, theta;
};

__device__ __forceinline__ float seg_length(const ImgArgs &a, int64_t ca, int64_t cb)
{
    const float *pa = a.pos_hl + 6 * ca, *pb = a.pos_hl + 6 * cb;
    const float ex = (pb[0] - pa[0]) + (pb[3] - pa[3]);
    const float ey = (pb[1] - pa[1]) + (pb[4] - pa[4]);
    const float ez = (pb[2] - pa[2]) + (pb[5] - pa[5]);
    return sqrtf(fmaf(ez, ez, fmaf(ey, ey, ex * ex))) * a.inv_Lunit;
}

// The trapezoid / erf decision in FP64 for a segment whose FP32 Doppler
// shift ratio lies within rounding of the threshold.
__device__ __noinline__ bool img_trapezoid_fp64(const ImgArgs &a, double rf, int64_t ca, int64_t cb)
{
    const double *va = a.vel + 3 * ca, *vb = a.vel + 3 * cb;
    const double ba = (a.n64[0] * va[0] + a.n64[1] * va[1] + a.n64[2] * va[2]) / kC;
    const double bb = (a.n64[0] * vb[0] + a.n64[1] * vb[1] + a.n64[2] * vb[2]) / kC;
    const double wa = a.w64[ca], wb = a.w64[cb];
    const double wbar = a.width_mode == 0 ? sqrt(0.5 * (wa * wa + wb * wb)) : 0.5 * (wa + wb);
    return fabs(rf * (ba - bb) / wbar) < a.thr;
}

// Optical depth of segment (A -> B) for channel ch; with `want` also its
// partial derivatives d[0..2] = d/d(log T_A, log n_A, beta_A) and
// d[3..5] = the same for B.
template <bool want>
__device__ __forceinline__ float seg_dtau(const ImgArgs &a, const Chan &ch, const Pt &A, const Pt &B, float dx,
                                          float iwbar, float (&d)[6])
{
    const float za = fmaf(-ch.rf, A.beta, ch.rf1), zb = fmaf(-ch.rf, B.beta, ch.rf1);
    const float du = (zb - za) * iwbar;
    const float thr = (float)a.thr;
    bool trap = fabsf(du) < thr;
    if (fabsf(fabsf(du) - thr) < kImgBand * thr) trap = img_trapezoid_fp64(a, ch.rf64, A.c, B.c);
    if (trap) {
        const float ua = za * A.winv, ub = zb * B.winv;
        const float ga = __expf(-ua * ua), gb = __expf(-ub * ub);
        if constexpr (want) {
            d[0] = 0.5f * dx * A.chi * ga * (A.theta * A.winv * A.winv) * (2.0f * ua * ua - 1.0f);
            d[1] = 0.5f * dx * A.chi * ga;
            d[2] = dx * A.chi * ga * ua * ch.rf * A.winv;
            d[3] = 0.5f * dx * B.chi * gb * (B.theta * B.winv * B.winv) * (2.0f * ub * ub - 1.0f);
            d[4] = 0.5f * dx * B.chi * gb;
            d[5] = dx * B.chi * gb * ub * ch.rf * B.winv;
        }
        return 0.5f * dx * (A.chi * ga + B.chi * gb);
    }
    const float a_ = za * iwbar, b_ = zb * iwbar;
    float lo = a_, hi = b_;
    if (lo + hi < 0.0f) {   // reflect: same difference, no cancellation
        lo = -b_;
        hi = -a_;
    }
    const float2 ef = erfc_fit2(lo, hi);          // both fits on packed FP32
    const float E = ef.x - ef.y;
    const float Delta = zb - za;
    // the MUFU reciprocal (relative error about 2^-23): |Delta| >= switch x
    // mean width in the erf branch, so no IEEE division is needed
    const float iD = rcp_mufu(Delta);
    const float Kc = dx * (0.25f * kSqrtPiF);
    const float K = Kc * (A.chi * A.w + B.chi * B.w);
    if constexpr (want) {
        const float ea = (2.0f / kSqrtPiF) * __expf(-a_ * a_), eb = (2.0f / kSqrtPiF) * __expf(-b_ * b_);
        const float dza = K * (E * iD - ea * iwbar) * iD;
        const float dzb = K * (eb * iwbar - E * iD) * iD;
        const float dwb = K * iD * (ea * a_ - eb * b_) * iwbar;
        const float wta = a.width_mode == 0 ? 0.5f * A.theta * iwbar : 0.5f * A.theta * A.winv;
        const float wtb = a.width_mode == 0 ? 0.5f * B.theta * iwbar : 0.5f * B.theta * B.winv;
        d[0] = dwb * wta;
        d[1] = Kc * A.chi * A.w * E * iD;
        d[2] = -ch.rf * dza;
        d[3] = dwb * wtb;
        d[4] = Kc * B.chi * B.w * E * iD;
        d[5] = -ch.rf * dzb;
    }
    return K * E * iD;
}

// e^-t, w0, w1 and g' = d/dt (1 - e^-t)/t, by series for small t.
__device__ __forceinline__ void weights(float t, float &E, float &w0, float &w1, float &gp)
{
    E = __expf(-t);
    if (t < 0.05f) {
        w1 = t * (0.5f - t * (1.0f / 6.0f - t * (1.0f / 24.0f - t * (1.0f / 120.0f))));
        w0 = t * (0.5f - t * (1.0f / 3.0f - t * (1.0f / 8.0f - t * (1.0f / 30.0f - t * (1.0f / 144.0f)))));
        gp = -0.5f + t * (1.0f / 3.0f - t * (1.0f / 8.0f - t * (1.0f / 30.0f - t * (1.0f / 144.0f))));
    } else {
        const float rt = rcp_mufu(t);           // t >= 0.05 here
        const float g = (1.0f - E) * rt;
        w0 = g - E;
        w1 = 1.0f - g;
        gp = (E - g) * rt;
    }
}

// Stage ray points c0 .. c0+n-1 of pixel ray `base` (n <= kImgStage): the
// velocity projection, width, 1/width and length of the segment ending at the
// point, that segment's inverse mean width, and, with `theta`, the width's
// temperature factor.  Every thread of the block calls it.
__device__ __forceinline__ void stage_points(const ImgArgs &a, int64_t base, int64_t c0, int n, bool theta,
                                             float4 *geo, float *siw, float *sth, int32_t *pid)
{
    __syncthreads();                 // the previous stage is consumed
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t d = c0 + i;
        const int32_t c = a.pts[base + d];
        const float *row = a.line + (int64_t)c * a.RS;
        const float *v = a.vel_hl + 6 * (int64_t)c;
        const float beta = fmaf(a.n2, v[2] + v[5], fmaf(a.n1, v[1] + v[4], a.n0 * (v[0] + v[3])));
        const float wb = row[2 * a.Mpad];
        float dx = 0.0f, iw = 0.0f;
        if (d > 0) {
            const int32_t cp = a.pts[base + d - 1];
            dx = seg_length(a, cp, c);
            const float wa = a.line[(int64_t)cp * a.RS + 2 * a.Mpad];
            iw = 1.0f / (a.width_mode == 0 ? sqrtf(0.5f * (wa * wa + wb * wb)) : 0.5f * (wa + wb));
        }
        geo[i] = make_float4(beta, wb, row[2 * a.Mpad + 1], dx);
        siw[i] = iw;
        pid[i] = c;
        if (theta) sth[i] = a.theta_k * (float)a.temp[c];
    }
    __syncthreads();
}

// Staged point i with line l's scaled opacity and source function.
__device__ __forceinline__ Pt staged_pt(const ImgArgs &a, const float4 *geo, const float *sth, const int32_t *pid,
                                        int i, int l, bool theta)
{
    const float4 g = geo[i];
    Pt p;
    p.c = pid[i];
    const float *row = a.line + p.c * a.RS;
    p.chi = row[l];
    p.S = row[a.Mpad + l];
    p.w = g.y;
    p.winv = g.z;
    p.beta = g.x;
    p.theta = theta ? sth[i] : 0.0f;
    return p;
}

// The channel constants depend only on the channel: computed once per call.
__global__ void k_image_chan(ImgArgs a, Chan *__restrict__ out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < a.nfreq) out[f] = channel(a, f);
}

// One block per pixel, threads over channels.  The ray's point geometry (the
// velocity projection, the widths and the segment lengths) is the same for
// every channel: the block stages it in shared memory, kImgStage points at a
// time, and each thread reads only its line's opacity and source function per
// point.
__global__ void __launch_bounds__(256) k_image_fwd(ImgArgs a)
{
    __shared__ float4 geo[kImgStage];
    __shared__ float siw[kImgStage];
    __shared__ int32_t pid[kImgStage];
    const int64_t q = blockIdx.x;
    const int64_t base = a.off[q];
    const int64_t np = a.off[q + 1] - base;  // points on the ray (segments + 1)
    float dd[6];
    for (int f0 = 0; f0 < a.nfreq; f0 += blockDim.x) {   // the same trip count for the whole block
        const int f = f0 + threadIdx.x;
        const bool active = f < a.nfreq;
        const Chan ch = a.chan[active ? f : 0];
        float I = ch.I0;
        Pt A{};
        for (int64_t c0 = 0; c0 < np; c0 += kImgStage) {
            const int n = (int)min((int64_t)kImgStage, np - c0);
            stage_points(a, base, c0, n, false, geo, siw, nullptr, pid);
            if (!active) continue;
            for (int i = 0; i < n; ++i) {
                const Pt B = staged_pt(a, geo, nullptr, pid, i, ch.l, false);
                if (c0 + i > 0) {
                    const float t = seg_dtau<false>(a, ch, A, B, geo[i].w, siw[i], dd);
                    float E, w0, w1, gp;
                    weights(t, E, w0, w1, gp);
                    I = fmaf(E, I, fmaf(w0, A.S, w1 * B.S));
                }
                A = B;
            }
        }
        if (active) a.out[(int64_t)f * a.npix + q] = I * ch.U;
    }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of the warp's contributions to point c (every lane calls).
__device__ __forceinline__ void flush_point(const ImgArgs &a, int64_t c, float gT, float gn, float gb)
{
    gT = warp_sum_f(gT);
    gn = warp_sum_f(gn);
    gb = warp_sum_f(gb);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.g_logT + c, (double)gT);
        atomicAdd(a.g_logn + c, (double)gn);
        atomicAdd(a.g_beta + c, (double)gb);
    }
}

// Adjoint: one block per pixel, threads over channels (the whole block runs
// the same number of channel rounds, so every warp intrinsic and barrier is
// uniform; threads past the last channel run channel 0 with zero weight).  The
// ray's points are staged in shared memory: 128 at a time for the forward pass
// that keeps the checkpoints, then one checkpoint block (at most kBlk + 1
// points) at a time for its recomputation and reverse sweep.
__global__ void __launch_bounds__(128) k_image_adj(ImgArgs a)
{
    __shared__ float4 geo[kImgStage];
    __shared__ float siw[kImgStage];
    __shared__ float sth[kImgStage];
    __shared__ int32_t pid[kImgStage];
    const int64_t q = blockIdx.x;
    const int64_t base = a.off[q];
    const int64_t D = a.off[q + 1] - base - 1;
    // segments per checkpoint block: as many as a block holds (kBlk), so that a
    // short ray is one block (one staging of its points); at most kCk blocks
    // because the host admits rays of up to kCk * kBlk segments
    const int64_t s = D > 0 ? min(D, (int64_t)kBlk) : 1;
    const int64_t nblk = D > 0 ? (D + s - 1) / s : 0;
    float dd[6];
    float ck[kCk], loc[kBlk];
    for (int f0 = 0; f0 < a.nfreq; f0 += blockDim.x) {
        const int f = f0 + threadIdx.x;
        const bool active = f < a.nfreq;
        const Chan ch = a.chan[active ? f : 0];
        // forward, keeping checkpoints
        float I = ch.I0;
        {
            Pt A{};
            int64_t next_ck = 0;                           // segment d of the next checkpoint (every s-th)
            int ick = 0;
            for (int64_t c0 = 0; c0 <= D; c0 += kImgStage) {
                const int n = (int)min((int64_t)kImgStage, D + 1 - c0);
                stage_points(a, base, c0, n, false, geo, siw, sth, pid);
                for (int i = 0; i < n; ++i) {
                    const Pt B = staged_pt(a, geo, sth, pid, i, ch.l, false);
                    const int64_t d = c0 + i - 1;              // the segment ending at this point
                    if (d >= 0) {
                        if (d == next_ck) {
                            ck[ick++] = I;
                            next_ck += s;
                        }
                        const float t = seg_dtau<false>(a, ch, A, B, geo[i].w, siw[i], dd);
                        float E, w0, w1, gp;
                        weights(t, E, w0, w1, gp);
                        I = fmaf(E, I, fmaf(w0, A.S, w1 * B.S));
                    }
                    A = B;
                }
            }
        }
        float lam = active ? a.gout[(int64_t)f * a.npix + q] * ch.U : 0.0f;
        float pT = 0.0f, pn = 0.0f, pb = 0.0f;      // pending gradient of point P_{d+1}
        for (int64_t blk = nblk - 1; blk >= 0; --blk) {
            const int64_t d0 = blk * s, d1 = min(D, d0 + s);
            stage_points(a, base, d0, (int)(d1 - d0 + 1), true, geo, siw, sth, pid);
            float Ir = ck[blk];
            Pt A = staged_pt(a, geo, sth, pid, 0, ch.l, false);
            for (int64_t d = d0; d < d1; ++d) {
                const int i = (int)(d - d0) + 1;
                loc[i - 1] = Ir;
                const Pt B = staged_pt(a, geo, sth, pid, i, ch.l, false);
                const float t = seg_dtau<false>(a, ch, A, B, geo[i].w, siw[i], dd);
                float E, w0, w1, gp;
                weights(t, E, w0, w1, gp);
                Ir = fmaf(E, Ir, fmaf(w0, A.S, w1 * B.S));
                A = B;
            }
            for (int64_t d = d1 - 1; d >= d0; --d) {
                const int i = (int)(d - d0);
                const Pt Pa = staged_pt(a, geo, sth, pid, i, ch.l, true);
                const Pt Pb = staged_pt(a, geo, sth, pid, i + 1, ch.l, true);
                const float t = seg_dtau<true>(a, ch, Pa, Pb, geo[i + 1].w, siw[i + 1], dd);
                float E, w0, w1, gp;
                weights(t, E, w0, w1, gp);
                const float dIdt = -E * loc[i] + (gp + E) * Pa.S - gp * Pb.S;
                const float G = active ? lam * dIdt : 0.0f;
                flush_point(a, Pb.c, pT + G * dd[3], pn + G * dd[4], pb + G * dd[5]);
                pT = G * dd[0];
                pn = G * dd[1];
                pb = G * dd[2];
                lam *= E;
            }
        }
        flush_point(a, a.pts[base], pT, pn, pb);
    }
}

__global__ void k_beta_to_vel(int64_t N, const double *__restrict__ g_beta, double n0, double n1, double n2,
                              double *__restrict__ g_vel)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const double g = g_beta[c] / kC;
    g_vel[3 * c] = g * n0;
    g_vel[3 * c + 1] = g * n1;
    g_vel[3 * c + 2] = g * n2;
}

__global__ void k_rescale_pops(int64_t N, int L, const double *__restrict__ ns_old, const double *__restrict__ ns_new,
                               double *__restrict__ pops, double *__restrict__ pops_prev)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * L) return;
    const int64_t p = e / L;
    const double f = ns_new[p] / ns_old[p];
    pops[e] *= f;
    pops_prev[e] *= f;
}

__global__ void k_vel_hl(int64_t N, const double *__restrict__ vel, float *__restrict__ vel_hl)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 3; ++c) {
        const double vb = vel[3 * i + c] / kC;
        const float vh = (float)vb;
        vel_hl[6 * i + c] = vh;
        vel_hl[6 * i + 3 + c] = (float)(vb - (double)vh);
    }
}

mgt_status check_image_args(const double *dir, int32_t npx, int32_t npy, int32_t nfreq, double fmin, double fmax)
{
    if (!dir) return set_error(MGT_ERR_ARG, "image direction is NULL");
    if (!std::isfinite(dir[0]) || !std::isfinite(dir[1]) || !std::isfinite(dir[2]))
        return set_error(MGT_ERR_ARG, "image direction must be finite");
    const double nn = dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2];
    if (std::fabs(nn - 1.0) > 1e-12) return set_error(MGT_ERR_ARG, "image direction must be a unit vector");
    if (npx < 1 || npy < 1 || (int64_t)npx * npy > ((int64_t)1 << 26))
        return set_error(MGT_ERR_ARG, "pixel counts must be >= 1 with npx * npy <= 2^26");
    if (nfreq < 1 || nfreq > 65536) return set_error(MGT_ERR_ARG, "nfreq must be 1..65536");
    if (!std::isfinite(fmin) || !std::isfinite(fmax) || !(fmin > 0.0) || fmax < fmin)
        return set_error(MGT_ERR_ARG, "need 0 < fmin <= fmax");
    return MGT_OK;
}

ImgArgs image_args(mgt_model *m, const double *dir, int32_t nfreq, double fmin, double fmax)
{
    ImgArgs a{};
    a.N = m->N;
    a.npix = (int64_t)m->img.npx * m->img.npy;
    a.M = m->M;
    a.Mpad = m->Mpad;
    a.RS = row_stride32(m->Mpad);
    a.nfreq = nfreq;
    a.width_mode = m->opts.width_mode;
    a.line = m->d_line32;
    a.pos_hl = m->d_pos_hl;
    a.vel_hl = m->d_vel_hl;
    a.vel = m->d_vel;
    a.w64 = m->d_w64;
    a.temp = m->d_temp;
    a.line_tab = m->d_line_tab;
    a.off = m->img.d_off;
    a.pts = m->img.d_pts;
    a.fmin = fmin;
    a.fstep = nfreq > 1 ? (fmax - fmin) / (nfreq - 1) : 0.0;
    for (int k = 0; k < 3; ++k) a.n64[k] = dir[k];
    a.n0 = (float)dir[0];
    a.n1 = (float)dir[1];
    a.n2 = (float)dir[2];
    a.inv_Lunit = (float)(1.0 / (m->pos_scale * m->L_unit));
    a.thr = m->opts.switch_threshold;
    a.theta_k = (float)(kKB / (m->mol_mass * kC * kC));
    return a;
}

// The per-channel constants of one call, stream-ordered; the caller frees a.chan.
mgt_status image_channels(ImgArgs &a, cudaStream_t s)
{
    Chan *c = nullptr;
    MGT_CUDA(cudaMallocAsync(&c, sizeof(Chan) * a.nfreq, s));
    k_image_chan<<<ceil_div(a.nfreq, 128), 128, 0, s>>>(a, c);
    MGT_LAUNCH_CHECK("k_image_chan");
    a.chan = c;
    return MGT_OK;
}

mgt_status image_prepare(mgt_model *m, const double *dir, int32_t npx, int32_t npy, cudaStream_t s)
{
    MGT_TRY_STATUS(trace_image(m, dir, npx, npy, s));
    if (m->line_dirty) MGT_TRY_STATUS(launch_line_data(m, s));
    return MGT_OK;
}

}  // namespace

}  // namespace mgt

using namespace mgt;

extern "C" {

mgt_status mgt_image_rays(mgt_model *m, const double dir[3], int32_t npx, int32_t npy, int32_t *anchor,
                          int64_t *ray_off, int32_t *pts, void *stream)
{
    MGT_RANGE("mgt_image_rays");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    MGT_TRY_STATUS(check_image_args(dir, npx, npy, 1, 1.0, 1.0));
    cudaStream_t s = (cudaStream_t)stream;
    MGT_TRY_STATUS(trace_image(m, dir, npx, npy, s));
    const int64_t npix = (int64_t)npx * npy;
    if (anchor) MGT_CUDA(cudaMemcpyAsync(anchor, m->img.d_anchor, sizeof(int32_t) * npix, cudaMemcpyDeviceToHost, s));
    if (ray_off) MGT_CUDA(cudaMemcpyAsync(ray_off, m->img.d_off, sizeof(int64_t) * (npix + 1), cudaMemcpyDeviceToHost, s));
    if (pts && m->img.total > 0)
        MGT_CUDA(cudaMemcpyAsync(pts, m->img.d_pts, sizeof(int32_t) * m->img.total, cudaMemcpyDeviceToHost, s));
    return check_device_error(m, s);
}

mgt_status mgt_image(mgt_model *m, const double dir[3], int32_t npx, int32_t npy, int32_t nfreq, double fmin,
                     double fmax, float *out, int on_device, void *stream)
{
    MGT_RANGE("mgt_image");
    if (!m || !out) return set_error(MGT_ERR_ARG, "model or output is NULL");
    MGT_TRY_STATUS(check_image_args(dir, npx, npy, nfreq, fmin, fmax));
    cudaStream_t s = (cudaStream_t)stream;
    MGT_TRY_STATUS(image_prepare(m, dir, npx, npy, s));
    ImgArgs a = image_args(m, dir, nfreq, fmin, fmax);
    const int64_t n = a.npix * nfreq;
    float *dev = out;
    if (!on_device) MGT_CUDA(cudaMallocAsync(&dev, sizeof(float) * n, s));
    a.out = dev;
    MGT_TRY_STATUS(image_channels(a, s));
    const int bd = nfreq >= 256 ? 256 : (nfreq + 31) / 32 * 32;
    k_image_fwd<<<(unsigned)a.npix, bd, 0, s>>>(a);
    MGT_LAUNCH_CHECK("k_image_fwd");
    MGT_CUDA(cudaFreeAsync((void *)a.chan, s));
    if (!on_device) {
        MGT_CUDA(cudaMemcpyAsync(out, dev, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
        MGT_CUDA(cudaFreeAsync(dev, s));
        return check_device_error(m, s);
    }
    return MGT_OK;
}

mgt_status mgt_image_adjoint(mgt_model *m, const double dir[3], int32_t npx, int32_t npy, int32_t nfreq, double fmin,
                             double fmax, const float *grad_out, double *g_logT, double *g_logn, double *g_vel,
                             int on_device, void *stream)
{
    MGT_RANGE("mgt_image_adjoint");
    if (!m || !grad_out) return set_error(MGT_ERR_ARG, "model or grad_out is NULL");
    MGT_TRY_STATUS(check_image_args(dir, npx, npy, nfreq, fmin, fmax));
    cudaStream_t s = (cudaStream_t)stream;
    MGT_TRY_STATUS(image_prepare(m, dir, npx, npy, s));
    if ((int64_t)m->img.max_len - 1 > (int64_t)kCk * kBlk)
        return set_error(MGT_ERR_ARG, "a pixel ray is longer than the adjoint's checkpoint capacity (4096 segments)");
    ImgArgs a = image_args(m, dir, nfreq, fmin, fmax);
    const int64_t n = a.npix * nfreq, N = m->N;
    double *acc = nullptr, *gv = nullptr;
    float *gdev = nullptr;
    MGT_CUDA(cudaMallocAsync(&acc, sizeof(double) * 3 * N, s));
    MGT_CUDA(cudaMallocAsync(&gv, sizeof(double) * 3 * N, s));
    MGT_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * N, s));
    if (!on_device) {
        MGT_CUDA(cudaMallocAsync(&gdev, sizeof(float) * n, s));
        MGT_CUDA(cudaMemcpyAsync(gdev, grad_out, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    }
    a.gout = on_device ? grad_out : gdev;
    a.g_logT = acc;
    a.g_logn = acc + N;
    a.g_beta = acc + 2 * N;
    MGT_TRY_STATUS(image_channels(a, s));
    const int bd = nfreq >= 128 ? 128 : (nfreq + 31) / 32 * 32;
    k_image_adj<<<(unsigned)a.npix, bd, 0, s>>>(a);
    MGT_LAUNCH_CHECK("k_image_adj");
    MGT_CUDA(cudaFreeAsync((void *)a.chan, s));
    k_beta_to_vel<<<ceil_div(N, 256), 256, 0, s>>>(N, a.g_beta, dir[0], dir[1], dir[2], gv);
    MGT_LAUNCH_CHECK("k_beta_to_vel");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (g_logT) MGT_CUDA(cudaMemcpyAsync(g_logT, a.g_logT, sizeof(double) * N, kind, s));
    if (g_logn) MGT_CUDA(cudaMemcpyAsync(g_logn, a.g_logn, sizeof(double) * N, kind, s));
    if (g_vel) MGT_CUDA(cudaMemcpyAsync(g_vel, gv, sizeof(double) * 3 * N, kind, s));
    MGT_CUDA(cudaFreeAsync(acc, s));
    MGT_CUDA(cudaFreeAsync(gv, s));
    if (gdev) MGT_CUDA(cudaFreeAsync(gdev, s));
    if (!on_device) return check_device_error(m, s);
    return MGT_OK;
}

mgt_status mgt_set_point_fields(mgt_model *m, const double *temp, const double *n_spec, const double *vel,
                                int on_device, void *stream)
{
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = m->N;
    if (!on_device) {
        for (int64_t i = 0; i < N; ++i) {
            if (temp && (!(temp[i] > 0.0) || !std::isfinite(temp[i])))
                return set_error(MGT_ERR_ARG, "temperature must be finite and > 0");
            if (n_spec && (!(n_spec[i] > 0.0) || !std::isfinite(n_spec[i])))
                return set_error(MGT_ERR_ARG, "n_spec must be finite and > 0");
        }
        if (vel)
            for (int64_t i = 0; i < 3 * N; ++i)
                if (!std::isfinite(vel[i])) return set_error(MGT_ERR_ARG, "velocities must be finite");
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n_spec) {
        double *ns = nullptr;
        MGT_CUDA(cudaMallocAsync(&ns, sizeof(double) * N, s));
        MGT_CUDA(cudaMemcpyAsync(ns, n_spec, sizeof(double) * N, kind, s));
        k_rescale_pops<<<ceil_div(N * m->L, 256), 256, 0, s>>>(N, m->L, m->d_nspec, ns, m->d_pops, m->d_pops_prev);
        MGT_LAUNCH_CHECK("k_rescale_pops");
        MGT_CUDA(cudaMemcpyAsync(m->d_nspec, ns, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        MGT_CUDA(cudaFreeAsync(ns, s));
    }
    if (temp) {
        MGT_CUDA(cudaMemcpyAsync(m->d_temp, temp, sizeof(double) * N, kind, s));
        MGT_TRY_STATUS(launch_widths(m, s));
    }
    if (vel) {
        MGT_CUDA(cudaMemcpyAsync(m->d_vel, vel, sizeof(double) * 3 * N, kind, s));
        k_vel_hl<<<ceil_div(N, 256), 256, 0, s>>>(N, m->d_vel, m->d_vel_hl);
        MGT_LAUNCH_CHECK("k_vel_hl");
    }
    m->line_dirty = true;
    m->have_J = false;
    if (temp || vel) m->traced = false;   // the ray step records hold widths and velocity projections
    if (!on_device) return check_device_error(m, s);
    return MGT_OK;
}

}  // extern "C"
