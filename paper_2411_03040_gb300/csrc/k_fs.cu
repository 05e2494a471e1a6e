// Formal solution of the line transfer equation along every ray pair, frequency
// bin and line, reduced into J-bar and Lambda* (the hot loop).
//
// Mapping: each thread owns one Gauss-Hermite bin q and LPT consecutive lines
// of one origin and loops over all ray pairs.  All threads of an origin walk
// the same ray, so trip counts never diverge; the per-step, line-independent
// work (comoving frequency, Gaussian, the trapezoid/erf switch, erf) is done
// once per (q, step) and shared by the thread's LPT lines.
//
// Three kernels:
//  * k_fs_staged: one CTA per origin.  Each half-ray is cut into chunks of CH
//    steps; warp 0 moves the next chunk's step records and point rows (line
//    data + width) into shared memory with bulk asynchronous copies
//    (cp.async.bulk, completion on an mbarrier) while the CTA eliminates the
//    current chunk from shared memory.
//  * k_fs_gather: several origins per CTA (small bin x line counts); every
//    thread gathers its rows straight from global memory.
//  * k_fs_batch: the staged body for the items (model, origin, line block) of
//    many models in one persistent launch.
//
// Second-order (Feautrier) system along a ray with points d = 0..D-1 and
// segment optical depths, rows -A u_{d-1} + (1 + A + C) u_d - C u_{d+1} = S_d,
// A = 2/(a(a+b)), C = 2/(b(a+b)), with the second-order boundary rows carrying
// I_bg at both ends.  It is eliminated from each far end toward the origin in
// a reparametrised Rybicki-Hummer form: with a, b the optical depths of the
// segments behind and ahead of row d (a = 0 at the end row),
//     h = (a + b)/2,  H = h + P,  q = 1/(1 + b H),  P <- H q,  Y <- (S h + Y) q,
// starting from P = 1, Y = I_bg.  q is the Thomas coefficient u_d = q u_{d+1}
// + b Y, every term is a sum of positive numbers, and no 1/dtau appears, so
// dtau -> 0 is exact and FP32 keeps its relative accuracy.  At the origin,
// with h = (a_L + a_R)/2 from the two adjacent segments,
//     u = (S h + Y_L + Y_R) / (h + P_L + P_R),  Lambda*_oo = h / (h + P_L + P_R).
// The kernels carry half depths (alpha = a/2, beta = b/2) and Pi = 2P, which
// removes the halving from every row: h = alpha + beta, G = 2h + Pi (= 2H),
// q = 1/(1 + beta G), Pi <- G q, Y <- (S h + Y) q -- eight FP32 operations
// and one reciprocal per line and step, from Pi = 2, alpha = 0 at the far end.
//
// Staged kernel, per chunk of a half-ray: first the CTA's threads (in a CTA of
// 128 threads or more all but warp 0, which issues the copies) compute
// line-independent segment coefficients for a share of the chunk's (bin,
// step) pairs (Gaussian at both ends, trapezoid/erf switch, erf difference)
// into shared memory, then each thread eliminates its lines reading one
// coefficient pair per step, two steps per trip.  The line groups of a bin
// do not repeat the coefficient work.
#include <algorithm>
#include <cstring>

#include "mgt_common.cuh"
#include "mgt_erfc.cuh"

namespace mgt {

namespace {

template <typename T> struct Prec;

template <> struct Prec<float> {
    using V2 = float2;
    static __device__ __forceinline__ float rcp(float x)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    // exp(-u^2) = 2^(-u^2 log2 e) with the MUFU exponential, explicitly rounded
    // (gauss2 below is the same arithmetic on a pair)
    static __device__ __forceinline__ float gauss(float u)
    {
        return mgt::ex2_mufu(__fmul_rn(__fmul_rn(u, u), -mgt::kLog2E));
    }
    static __device__ __forceinline__ float erfc_(float x) { return mgt::erfc_fit(x); }
    // erfc(a) - erfc(b), the two fits on packed FP32
    static __device__ __forceinline__ float erfc_diff(float a, float b)
    {
        const float2 r = mgt::erfc_fit2(a, b);
        return __fsub_rn(r.x, r.y);
    }
    // explicitly rounded operations (never contracted differently by context)
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float bg(float f, float hk) { return f * f * f / expm1f(hk * f); }
};

template <> struct Prec<double> {
    using V2 = double2;
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double gauss(double u) { return exp(-__dmul_rn(u, u)); }
    static __device__ __forceinline__ double erfc_(double x) { return erfc(x); }
    static __device__ __forceinline__ double erfc_diff(double a, double b) { return __dsub_rn(erfc(a), erfc(b)); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double bg(double f, double hk) { return f * f * f / expm1(hk * f); }
};

// A bin's comoving offset z = Aq + Bq beta at a point (beta its velocity
// projection), and the point's Gaussian exp(-(z/w)^2) from its 1/w, with
// explicit roundings, so that every schedule computes them identically.
template <typename T> __device__ __forceinline__ T bin_z(T Aq, T Bq, T beta) { return Prec<T>::fma(Bq, beta, Aq); }
template <typename T> __device__ __forceinline__ T point_gauss(T z, T rw) { return Prec<T>::gauss(Prec<T>::mul(z, rw)); }

struct FSArgs {
    int64_t N;
    int R, P, Q, M, Mpad, RS, Gtot, Gb, OPB;
    const int2 *pairs;
    const int64_t *ray_off;
    const Step32 *s32;
    const Step64 *s64;
    const void *line;          // float* or double*, [N][RS] rows (see row_stride32/64)
    const int32_t *order;      // origin visiting order (space-filling curve), [N]
    const double *xq, *wq;
    const double *line_tab;    // [8][Mpad]
    const double *vel, *dirs, *w64;
    double thr;
    int width_mode;
    int subdiv;                // > 0: every segment by the trapezoidal rule over this many pieces
    const int32_t *dir_map;    // pair directions -> model directions (NULL: the same)
    int accumulate;            // add to J / Lstar (later pair batches) instead of writing them
    int lpt;                   // lines per thread of the staged schedule (batched launches)
    int nblk;                  // line blocks per origin (ceil(Gtot / Gb))
    int fused;                 // staged schedule with each thread's coefficients in registers (Gtot == 1)
    double *J, *Lst;           // [N][M]
    int *err;
    const int *range_bad;      // nonzero: a point's range figure exceeds 1 (set by the line data)
    int64_t n_rec;             // step records held (the ray offsets index below this)
};

// Geometry of one traced step in the solver's precision.
template <typename T> struct StepG {
    T dx, beta, dbw;
};

template <typename T> __device__ __forceinline__ StepG<T> step_from(const void *p);

template <> __device__ __forceinline__ StepG<float> step_from<float>(const void *p)
{
    const int4 v = *reinterpret_cast<const int4 *>(p);
    return {__int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w)};
}

template <> __device__ __forceinline__ StepG<double> step_from<double>(const void *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 v0 = q[0], v1 = q[1];
    return {v0.x, v0.y, v1.x};
}

template <typename T> __device__ __forceinline__ StepG<T> step_global(const FSArgs &a, int64_t s);

template <> __device__ __forceinline__ StepG<float> step_global<float>(const FSArgs &a, int64_t s)
{
    const int4 v = __ldg(a.s32 + s);
    return {__int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w)};
}

template <> __device__ __forceinline__ StepG<double> step_global<double>(const FSArgs &a, int64_t s)
{
    const double2 *q = reinterpret_cast<const double2 *>(a.s64 + s);
    const double2 v0 = __ldg(q), v1 = __ldg(q + 1);
    return {v0.x, v0.y, v1.x};
}

// LPT consecutive scalars of a row (global or shared memory), 16-byte aligned.
template <int LPT> __device__ __forceinline__ void load_vec(const float *p, float (&v)[LPT])
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < LPT / 4; ++i) {
        const float4 x = q[i];
        v[4 * i] = x.x;
        v[4 * i + 1] = x.y;
        v[4 * i + 2] = x.z;
        v[4 * i + 3] = x.w;
    }
}

template <int LPT> __device__ __forceinline__ void load_vec(const double *p, double (&v)[LPT])
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < LPT / 2; ++i) {
        const double2 x = q[i];
        v[2 * i] = x.x;
        v[2 * i + 1] = x.y;
    }
}

// The trapezoid / erf decision re-taken in FP64 for a segment whose FP32
// Doppler-shift ratio lies within rounding of the threshold, so that both
// precisions (and the FP64 reference) branch alike.  The FP32 ratio comes from
// velocity projections formed from hi + lo floats of v/c: its error is about
// 2e-7 |v_far - v_near|_1 / (c wbar) + 4e-7 |du|, below 7e-5 (2e-4 of the
// threshold 0.35) for velocity jumps up to ~300 line widths between
// neighbouring points.
constexpr float kSwitchBand = 2e-4f;
__device__ __noinline__ bool trapezoid_fp64(const FSArgs &a, int r, int64_t c_far, int64_t c_near, double xq64,
                                            double wo64)
{
    if (c_far < 0 || c_far >= a.N || c_near < 0 || c_near >= a.N) {   // index check: record, use point 0
        if (atomicCAS(a.err, 0, (int)kDevBounds) == 0) {
            a.err[1] = 22;
            a.err[2] = (int)c_far;
            a.err[3] = (int)c_near;
        }
        c_far = c_far < 0 || c_far >= a.N ? 0 : c_far;
        c_near = c_near < 0 || c_near >= a.N ? 0 : c_near;
    }
    const double *n = a.dirs + 3 * (a.dir_map ? a.dir_map[r] : r);
    const double *vf = a.vel + 3 * c_far, *vn = a.vel + 3 * c_near;
    const double dbeta = (n[0] * (vf[0] - vn[0]) + n[1] * (vf[1] - vn[1]) + n[2] * (vf[2] - vn[2])) / kC;
    const double wf = a.w64[c_far], wn = a.w64[c_near];
    const double wbar = a.width_mode == 0 ? sqrt(0.5 * (wf * wf + wn * wn)) : 0.5 * (wf + wn);
    const double du = (1.0 + xq64 * wo64) * dbeta / wbar;
    return fabs(du) < a.thr;
}

// Line-independent coefficients of one segment: dtau_line = cf chi_far + cn chi_near.
//   du    : reduced Doppler shift near minus far, in units of the averaged width
//   trap  : trapezoid branch (|du| below the threshold)
// Semi-analytic branch: with ubar the reduced frequencies at the averaged
// width, E = erf(ubar_near) - erf(ubar_far).  Reflecting (a, b) -> (-b, -a)
// when a + b < 0 leaves E unchanged, after which E = erfc(a) - erfc(b) has no
// cancellation: either both arguments are >= 0 (tails as differences of small
// erfc values) or they straddle zero and E >= erf(|du|/2) (|du| >= threshold).
// Both coefficients are returned halved: half the segment's optical depth is
// cf chi~_far + cn chi~_near.
template <typename T>
__device__ __forceinline__ void segment_coefs(bool trap, T dx, T du, T z_f, T g_f, T w_f, T g_n, T w_n, int width_mode,
                                              T &cf, T &cn)
{
    using P = Prec<T>;
    if (trap) {
        const T q = P::mul(T(0.25), dx);
        cf = P::mul(q, g_f);
        cn = P::mul(q, g_n);
    } else {
        const T iwbar = width_mode == 0 ? P::rsqrt_(P::mul(T(0.5), P::fma(w_f, w_f, P::mul(w_n, w_n))))
                                        : P::rcp(P::mul(T(0.5), P::add(w_f, w_n)));
        T a = P::mul(z_f, iwbar), b = P::add(a, du);
        if (P::add(a, b) < T(0)) {
            const T t = a;
            a = -b;
            b = -t;
        }
        const T E = P::erfc_diff(a, b);
        const T kk = P::mul(P::mul(P::mul(P::mul(dx, T(0.125 * kSqrtPi)), E), iwbar), P::rcp(du));
        cf = P::mul(kk, w_f);
        cn = P::mul(kk, w_n);
    }
}

// Reference coefficients of the accuracy study (Sec. 4.3): the segment cut
// into n equal pieces, the trapezoidal rule on each, with the line opacity
// chi^{ij} = chi~ w (nu sqrt(pi)), the width and the comoving offset
// interpolated linearly; halved, like segment_coefs.
template <typename T>
__device__ __forceinline__ void subdiv_coefs(int n, T dx, T z_f, T w_f, T z_n, T w_n, T &cf, T &cn)
{
    using P = Prec<T>;
    T sf = T(0), sn = T(0);
    const T inv_n = T(1) / T(n);
    for (int k = 0; k <= n; ++k) {
        const T x = P::mul(T(k), inv_n);
        const T z = P::fma(x, P::sub(z_n, z_f), z_f), w = P::fma(x, P::sub(w_n, w_f), w_f);
        const T u = z / w;
        const T g = P::mul(P::gauss(u) / w, (k == 0 || k == n) ? T(0.5) : T(1));
        sf = P::fma(P::sub(T(1), x), g, sf);
        sn = P::fma(x, g, sn);
    }
    const T c = P::mul(P::mul(P::mul(T(0.5), dx), inv_n), w_f);
    cf = P::mul(c, sf);
    cn = P::mul(P::mul(P::mul(P::mul(T(0.5), dx), inv_n), w_n), sn);
}

// One elimination row for the thread's LPT lines, in the halved variables:
// cf, cn halved coefficients; aa[l] = alpha (half depth of the previous
// segment); P[l] = Pi = 2P.
template <typename T, int LPT>
__device__ __forceinline__ void eliminate_row_scalar(T cf, T cn, const T (&chi_f)[LPT], const T (&S_f)[LPT],
                                                     const T (&chi_n)[LPT], T (&P)[LPT], T (&Y)[LPT], T (&aa)[LPT])
{
    using Op = Prec<T>;
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        const T b = Op::fma(cf, chi_f[l], Op::mul(cn, chi_n[l]));   // beta, half the segment depth
        const T h = Op::add(aa[l], b);
        const T G = Op::fma(T(2), h, P[l]);
        const T q = Op::rcp(Op::fma(b, G, T(1)));
        P[l] = Op::mul(G, q);
        Y[l] = Op::mul(Op::fma(S_f[l], h, Y[l]), q);
        aa[l] = b;
    }
}

// The same row in FP32 on line pairs with Blackwell's packed FP32 operations
// (two lanes of arithmetic per issue slot): eight packed operations and two
// reciprocals per pair of lines, so 5 issue slots per line and step instead of 9.
template <int LPT>
__device__ __forceinline__ void eliminate_row_packed(float cf, float cn, const float (&chi_f)[LPT],
                                                     const float (&S_f)[LPT], const float (&chi_n)[LPT],
                                                     float (&P)[LPT], float (&Y)[LPT], float (&aa)[LPT])
{
    static_assert(LPT % 2 == 0, "line pairs");
    const float2 cf2 = make_float2(cf, cf), cn2 = make_float2(cn, cn);
    const float2 two = make_float2(2.0f, 2.0f), one = make_float2(1.0f, 1.0f);
#pragma unroll
    for (int l = 0; l < LPT; l += 2) {
        const float2 cx = make_float2(chi_f[l], chi_f[l + 1]), nx = make_float2(chi_n[l], chi_n[l + 1]);
        const float2 b = __ffma2_rn(cf2, cx, __fmul2_rn(cn2, nx));
        const float2 h = __fadd2_rn(make_float2(aa[l], aa[l + 1]), b);
        const float2 G = __ffma2_rn(two, h, make_float2(P[l], P[l + 1]));
        const float2 den = __ffma2_rn(b, G, one);
        const float2 q = make_float2(Prec<float>::rcp(den.x), Prec<float>::rcp(den.y));
        const float2 Pn = __fmul2_rn(G, q);
        const float2 Yn = __fmul2_rn(__ffma2_rn(make_float2(S_f[l], S_f[l + 1]), h, make_float2(Y[l], Y[l + 1])), q);
        P[l] = Pn.x;
        P[l + 1] = Pn.y;
        Y[l] = Yn.x;
        Y[l + 1] = Yn.y;
        aa[l] = b.x;
        aa[l + 1] = b.y;
    }
}

// Two rows per reciprocal (FP32, line pairs packed).  The row map
//     (Pi, Y) -> (G q, (S h + Y) q),  G = 2h + Pi,  q = 1/(1 + beta G)
// is linear-fractional, so in homogeneous coordinates Pi = p/d, Y = y/d it is
// the linear map
//     p' = p + 2 h d,  y' = y + S h d,  d' = d + beta p'
// with no division.  Two rows are taken from d = 1 and the state is brought
// back to Pi, Y with one reciprocal of the final d: 15 packed operations and
// two reciprocals per line pair and two steps, against 16 and four for two
// eliminate_row calls, and a dependent chain without the reciprocal's
// latency in every row.  d grows by 1 + beta G per row; the caller takes this
// path only while that growth and the source terms provably stay inside the
// FP32 range (the range guard below), so the two forms differ by rounding alone.
template <int LPT>
__device__ __forceinline__ void homog_row1_packed(float cf, float cn, const float (&chi_f)[LPT],
                                                  const float (&S_f)[LPT], const float (&chi_n)[LPT],
                                                  float (&P)[LPT], float (&Y)[LPT], float (&aa)[LPT],
                                                  float (&D)[LPT])
{
    static_assert(LPT % 2 == 0, "line pairs");
    const float2 cf2 = make_float2(cf, cf), cn2 = make_float2(cn, cn);
    const float2 two = make_float2(2.0f, 2.0f), one = make_float2(1.0f, 1.0f);
#pragma unroll
    for (int l = 0; l < LPT; l += 2) {
        const float2 cx = make_float2(chi_f[l], chi_f[l + 1]), nx = make_float2(chi_n[l], chi_n[l + 1]);
        const float2 b = __ffma2_rn(cf2, cx, __fmul2_rn(cn2, nx));
        const float2 h = __fadd2_rn(make_float2(aa[l], aa[l + 1]), b);
        const float2 p = __ffma2_rn(two, h, make_float2(P[l], P[l + 1]));
        const float2 y = __ffma2_rn(make_float2(S_f[l], S_f[l + 1]), h, make_float2(Y[l], Y[l + 1]));
        const float2 d = __ffma2_rn(b, p, one);
        P[l] = p.x;
        P[l + 1] = p.y;
        Y[l] = y.x;
        Y[l + 1] = y.y;
        D[l] = d.x;
        D[l + 1] = d.y;
        aa[l] = b.x;
        aa[l + 1] = b.y;
    }
}

template <int LPT>
__device__ __forceinline__ void homog_row2_packed(float cf, float cn, const float (&chi_f)[LPT],
                                                  const float (&S_f)[LPT], const float (&chi_n)[LPT],
                                                  float (&P)[LPT], float (&Y)[LPT], float (&aa)[LPT],
                                                  const float (&D)[LPT])
{
    const float2 cf2 = make_float2(cf, cf), cn2 = make_float2(cn, cn);
    const float2 two = make_float2(2.0f, 2.0f);
#pragma unroll
    for (int l = 0; l < LPT; l += 2) {
        const float2 cx = make_float2(chi_f[l], chi_f[l + 1]), nx = make_float2(chi_n[l], chi_n[l + 1]);
        const float2 b = __ffma2_rn(cf2, cx, __fmul2_rn(cn2, nx));
        const float2 h = __fadd2_rn(make_float2(aa[l], aa[l + 1]), b);
        const float2 d1 = make_float2(D[l], D[l + 1]);
        const float2 hd = __fmul2_rn(h, d1);
        const float2 p = __ffma2_rn(two, hd, make_float2(P[l], P[l + 1]));
        const float2 y = __ffma2_rn(make_float2(S_f[l], S_f[l + 1]), hd, make_float2(Y[l], Y[l + 1]));
        const float2 d = __ffma2_rn(b, p, d1);
        const float2 r = make_float2(Prec<float>::rcp(d.x), Prec<float>::rcp(d.y));
        const float2 Pn = __fmul2_rn(p, r), Yn = __fmul2_rn(y, r);
        P[l] = Pn.x;
        P[l + 1] = Pn.y;
        Y[l] = Yn.x;
        Y[l + 1] = Yn.y;
        aa[l] = b.x;
        aa[l + 1] = b.y;
    }
}

// Back to Pi = p/d, Y = y/d and d = 1 after the first of two rows (both lines
// of each pair); followed by homog_row2_packed this is eliminate_row twice,
// operation for operation.
template <int LPT>
__device__ __forceinline__ void renormalize_packed(float (&P)[LPT], float (&Y)[LPT], float (&D)[LPT])
{
#pragma unroll
    for (int l = 0; l < LPT; l += 2) {
        const float2 r = make_float2(Prec<float>::rcp(D[l]), Prec<float>::rcp(D[l + 1]));
        const float2 Pn = __fmul2_rn(make_float2(P[l], P[l + 1]), r), Yn = __fmul2_rn(make_float2(Y[l], Y[l + 1]), r);
        P[l] = Pn.x;
        P[l + 1] = Pn.y;
        Y[l] = Yn.x;
        Y[l + 1] = Yn.y;
        D[l] = 1.0f;
        D[l + 1] = 1.0f;
    }
}

// Range of the two-row form.  A row's half depth is at most
// 0.5 dx (chi~max_far + chi~max_near), with chi~max the largest chi~' of a
// point over the lines: the trapezoid has cf <= dx/4, the semi-analytic form
// |erf difference| <= (2/sqrt(pi)) |du|, so cf <= dx w_far/(4 wbar) <= dx/2
// for either averaged width.  A point's row stores
//   G = max(chi~max dxmax / kFastB, S'max / kFastS)
// with dxmax its longest graph edge (every walk step is a graph edge), and the
// line data set the model's range flag when any point has G > 1, a
// non-finite figure or a Doppler width of 1 % of c or more (below that the
// background stays under kFastY whatever the line and T_bg).  With the flag
// clear, every row between two points has a half depth <= kFastB and sources
// <= kFastS, and on a half-ray shorter than kFastSteps with the switch rule's
// optical depths (not the subdivided reference's): alpha, beta <= 2^8
// (h <= 2^9), Pi <= 2^16 at every row (Pi' <= 1/beta after a row, and it
// grows by less than 2^-13 per row while beta < 2^-15, so rising past 2^16
// takes more than 2^27 rows), Y < 2^117 (Y grows by at most S' h <= 2^89 per
// row), and within a two-row step d < 2^26 after the first row, then
// p < 2^37, y < 2^117, d < 2^46: all finite and normal in FP32.  A model with
// the flag set is eliminated one row at a time (k_fs_exact).
constexpr float kFastB = kTwoRowDepth;           // 2^8
constexpr float kFastY = 1.2676506002282294e30f;  // 2^100
constexpr float kFastS = kTwoRowSource;           // 2^80
static_assert(kFastB == 256.0f && kFastS == 1.2089258196146292e24f && kFastY == 1.2676506002282294e30f,
              "range of the two-row elimination");
constexpr int kFastSteps = 1 << 27;

template <typename T, int LPT>
__device__ __forceinline__ void eliminate_row(T cf, T cn, const T (&chi_f)[LPT], const T (&S_f)[LPT],
                                              const T (&chi_n)[LPT], T (&P)[LPT], T (&Y)[LPT], T (&aa)[LPT])
{
    if constexpr (sizeof(T) == 4)
        eliminate_row_packed<LPT>(cf, cn, chi_f, S_f, chi_n, P, Y, aa);
    else
        eliminate_row_scalar<T, LPT>(cf, cn, chi_f, S_f, chi_n, P, Y, aa);
}

// Combine both halves at the origin and accumulate w_q u (compensated) and
// w_q Lambda*_oo (plain: at most a few hundred positive terms of similar size,
// relative error ~1e-6) in shared memory, one column per thread:
// acc[0] sum of J, acc[1] its compensation, acc[2] sum of Lambda*.  Inputs in
// the halved variables of eliminate_row.
template <typename T, int LPT>
__device__ __forceinline__ void combine_accumulate(T wqn, const T (&So)[LPT], const T (&PL)[LPT], const T (&YL)[LPT],
                                                   const T (&aL)[LPT], const T (&PR)[LPT], const T (&YR)[LPT],
                                                   const T (&aR)[LPT], T *acc, int bd, int tid)
{
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        const T h = aL[l] + aR[l];
        const T inv = Prec<T>::rcp(h + T(0.5) * (PL[l] + PR[l]));
        const T u = (So[l] * h + YL[l] + YR[l]) * inv;
        const T Ls = h * inv;
        T *sJ = acc + (0 * LPT + l) * bd + tid, *cJ = acc + (1 * LPT + l) * bd + tid;
        T *sL = acc + (2 * LPT + l) * bd + tid;
        const T y = wqn * u - *cJ, tt = *sJ + y;
        *cJ = (tt - *sJ) - y;
        *sJ = tt;
        *sL += wqn * Ls;
    }
}

// Slot of accumulator / first-half value c (0..2) of the thread's line l in
// the staged item's shared arrays: FP32 keeps line pairs adjacent ([3][LPT/2]
// [bd][2]) for float2 accesses, FP64 the plain [3][LPT][bd] layout.
template <typename T, int LPT> __device__ __forceinline__ int pair_slot(int c, int l, int bd, int tid)
{
    if constexpr (sizeof(T) == 4)
        return ((c * (LPT / 2) + l / 2) * bd + tid) * 2 + (l & 1);
    else
        return (c * LPT + l) * bd + tid;
}

// combine_accumulate on line pairs in packed FP32 with explicit roundings,
// the accumulators in the pair_slot layout (float2 per line pair).
template <int LPT>
__device__ __forceinline__ void combine_accumulate_packed(float wqn, const float (&So)[LPT], const float (&PL)[LPT],
                                                          const float (&YL)[LPT], const float (&aL)[LPT],
                                                          const float (&PR)[LPT], const float (&YR)[LPT],
                                                          const float (&aR)[LPT], float *acc, int bd, int tid)
{
    float2 *a2 = reinterpret_cast<float2 *>(acc);
    const float2 w2 = make_float2(wqn, wqn);
#pragma unroll
    for (int l = 0; l < LPT; l += 2) {
        const float2 h = __fadd2_rn(make_float2(aL[l], aL[l + 1]), make_float2(aR[l], aR[l + 1]));
        const float2 den = __ffma2_rn(make_float2(0.5f, 0.5f),
                                      __fadd2_rn(make_float2(PL[l], PL[l + 1]), make_float2(PR[l], PR[l + 1])), h);
        const float2 inv = make_float2(Prec<float>::rcp(den.x), Prec<float>::rcp(den.y));
        const float2 num = __fadd2_rn(__ffma2_rn(make_float2(So[l], So[l + 1]), h, make_float2(YL[l], YL[l + 1])),
                                      make_float2(YR[l], YR[l + 1]));
        const float2 u = __fmul2_rn(num, inv), Ls = __fmul2_rn(h, inv);
        float2 *sJ = a2 + (0 * (LPT / 2) + l / 2) * bd + tid, *cJ = a2 + (1 * (LPT / 2) + l / 2) * bd + tid;
        float2 *sL = a2 + (2 * (LPT / 2) + l / 2) * bd + tid;
        const float2 s0 = *sJ, c0 = *cJ;
        const float2 y = __ffma2_rn(w2, u, make_float2(-c0.x, -c0.y));
        const float2 tt = __fadd2_rn(s0, y);
        *cJ = __fadd2_rn(__fadd2_rn(tt, make_float2(-s0.x, -s0.y)), make_float2(-y.x, -y.y));
        *sJ = tt;
        *sL = __ffma2_rn(w2, Ls, *sL);
    }
}

// B_nu_q(T_bg) / U_line for the thread's bin and lines (depends on the origin
// through nu_q = nu (1 + x_q w_o)).
template <typename T, int LPT>
__device__ __forceinline__ void background(const FSArgs &a, int line0, double xq64, double wo64, T (&Ibg)[LPT])
{
    const T f = T(1) + T(xq64) * T(wo64);
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        const int k = line0 + l;
        const double hk = a.line_tab[5 * a.Mpad + k], nbg = a.line_tab[4 * a.Mpad + k];
        Ibg[l] = (k < a.M && hk > 0.0) ? Prec<T>::bg(f, T(hk)) / T(nbg) : T(0);
    }
}

// Final reduction over bins: red[2][OPB][Mb][Q] -> J, Lstar of the block's lines.
__device__ __forceinline__ void reduce_out(const FSArgs &a, const double *red, int Mb, int mline0, int64_t o_base,
                                           bool ordered)
{
    const double wdir = 2.0 / a.R;
    for (int e = threadIdx.x; e < a.OPB * Mb; e += blockDim.x) {
        const int lo2 = e / Mb, lb = e - lo2 * Mb;
        const int line = mline0 + lb;
        const int64_t oi = o_base + lo2;
        if (oi >= a.N || line >= a.M) continue;
        const int64_t o2 = ordered ? (int64_t)a.order[oi] : oi;
        if (o2 < 0 || o2 >= a.N) continue;      // a bad visiting-order entry (recorded by the item)
        double sJ = 0.0, sL = 0.0;
        for (int qq = 0; qq < a.Q; ++qq) {
            sJ += red[((0 * a.OPB + lo2) * Mb + lb) * a.Q + qq];
            sL += red[((1 * a.OPB + lo2) * Mb + lb) * a.Q + qq];
        }
        const double vJ = sJ * wdir * a.line_tab[6 * a.Mpad + line], vL = sL * wdir;
        if (a.accumulate) {
            a.J[o2 * a.M + line] += vJ;
            a.Lst[o2 * a.M + line] += vL;
        } else {
            a.J[o2 * a.M + line] = vJ;
            a.Lst[o2 * a.M + line] = vL;
        }
    }
}

// ---------------------------------------------------------------------------
// Gather kernel: OPB origins per CTA, rows read from global memory.
// ---------------------------------------------------------------------------
template <typename T, int LPT>
__device__ __forceinline__ void sweep_gather(const FSArgs &a, int64_t o, int r, int line0, T Aq, T Bq, const T *Ibg,
                                             double xq64, double wo64, T (&P)[LPT], T (&Y)[LPT], T (&aa)[LPT])
{
    const T *line = reinterpret_cast<const T *>(a.line);
    const int64_t t = (int64_t)r * a.N + o;
    const int64_t s0 = a.ray_off[t];
    const int n = (int)(a.ray_off[t + 1] - s0);
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        P[l] = T(2);
        Y[l] = Ibg[l];
        aa[l] = T(0);
    }
    if (n == 0) return;
    const T thr = (T)a.thr;
    // a point index from the ray records out of range: record it, use point 0
    auto checked = [&](int64_t c) -> int64_t {
        if (c >= 0 && c < a.N) return c;
        if (atomicCAS(a.err, 0, (int)kDevBounds) == 0) {
            a.err[1] = 21;
            a.err[2] = (int)o;
            a.err[3] = (int)c;
        }
        return 0;
    };
    int64_t c_f = checked(a.s32[s0 + n - 1].x);
    StepG<T> sf = step_global<T>(a, s0 + n - 1);
    T chi_f[LPT], S_f[LPT];
    load_vec<LPT>(line + c_f * a.RS + line0, chi_f);
    load_vec<LPT>(line + c_f * a.RS + a.Mpad + line0, S_f);
    T w_f = line[c_f * a.RS + 2 * a.Mpad];
    T z_f = bin_z<T>(Aq, Bq, sf.beta);
    T g_f = point_gauss<T>(z_f, line[c_f * a.RS + 2 * a.Mpad + 1]);
    for (int k = n; k >= 1; --k) {
        int64_t c_n = o;
        StepG<T> sn{T(0), T(0), T(0)};
        if (k > 1) {
            c_n = checked(a.s32[s0 + k - 2].x);
            sn = step_global<T>(a, s0 + k - 2);
        }
        const T *row = line + c_n * a.RS;
        T chi_n[LPT], S_n[LPT];
        load_vec<LPT>(row + line0, chi_n);
        load_vec<LPT>(row + a.Mpad + line0, S_n);
        const T w_n = row[2 * a.Mpad];
        const T z_n = bin_z<T>(Aq, Bq, sn.beta);
        const T g_n = point_gauss<T>(z_n, row[2 * a.Mpad + 1]);
        const T du = -Prec<T>::mul(Bq, sf.dbw);
        bool trap = fabs(du) < thr;
        if (sizeof(T) == 4 && fabs(fabs(du) - thr) < T(kSwitchBand) * thr) trap = trapezoid_fp64(a, r, c_f, c_n, xq64, wo64);
        T cf, cn;
        if (a.subdiv > 0)
            subdiv_coefs<T>(a.subdiv, sf.dx, z_f, w_f, z_n, w_n, cf, cn);
        else
            segment_coefs<T>(trap, sf.dx, du, z_f, g_f, w_f, g_n, w_n, a.width_mode, cf, cn);
        eliminate_row<T, LPT>(cf, cn, chi_f, S_f, chi_n, P, Y, aa);
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            chi_f[l] = chi_n[l];
            S_f[l] = S_n[l];
        }
        z_f = z_n;
        g_f = g_n;
        w_f = w_n;
        sf = sn;
        c_f = c_n;
    }
}

template <typename T, int LPT> __global__ void __launch_bounds__(256) k_fs_gather(FSArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const int QG = a.Q * a.Gb;
    const int Mb = a.Gb * LPT;
    T *acc = reinterpret_cast<T *>(smem_raw);                       // [3][LPT][bd]
    double *red = reinterpret_cast<double *>(acc + 4 * LPT * bd);   // [2][OPB][Mb][Q] (acc rounded up to 4 rows)

    const int lo_ = tid / QG, rem = tid - lo_ * QG, gl = rem / a.Q, q = rem - gl * a.Q;
    const int gg = blockIdx.y * a.Gb + gl;
    const int line0 = gg * LPT;
    const int64_t o = (int64_t)blockIdx.x * a.OPB + lo_;
    const bool active = lo_ < a.OPB && o < a.N && gg < a.Gtot;

    if (active) {
        const double xq64 = a.xq[q], wo64 = a.w64[o];
        T Ibg[LPT];
        background<T, LPT>(a, line0, xq64, wo64, Ibg);
#pragma unroll
        for (int l = 0; l < LPT; ++l)
            for (int c = 0; c < 3; ++c) acc[(c * LPT + l) * bd + tid] = T(0);
        const T Aq = T(xq64) * T(wo64), Bq = T(1) + Aq;
        const T wqn = T(a.wq[q]);
        const T *line = reinterpret_cast<const T *>(a.line);
        T So[LPT];
        load_vec<LPT>(line + o * a.RS + a.Mpad + line0, So);
        for (int p = 0; p < a.P; ++p) {
            const int2 pr = a.pairs[p];
            T PL[LPT], YL[LPT], aL[LPT], PR[LPT], YR[LPT], aR[LPT];
            sweep_gather<T, LPT>(a, o, pr.y, line0, Aq, Bq, Ibg, xq64, wo64, PL, YL, aL);
            sweep_gather<T, LPT>(a, o, pr.x, line0, Aq, Bq, Ibg, xq64, wo64, PR, YR, aR);
            combine_accumulate<T, LPT>(wqn, So, PL, YL, aL, PR, YR, aR, acc, bd, tid);
        }
        const int lb = gl * LPT;
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            if (line0 + l < a.M) {
                red[((0 * a.OPB + lo_) * Mb + lb + l) * a.Q + q] =
                    (double)acc[(0 * LPT + l) * bd + tid] - (double)acc[(1 * LPT + l) * bd + tid];
                red[((1 * a.OPB + lo_) * Mb + lb + l) * a.Q + q] =
                    (double)acc[(2 * LPT + l) * bd + tid];
            }
        }
    }
    __syncthreads();
    reduce_out(a, red, Mb, blockIdx.y * Mb, (int64_t)blockIdx.x * a.OPB, false);
}

// ---------------------------------------------------------------------------
// Staged kernel: one origin per CTA, ray chunks moved to shared memory by
// bulk asynchronous copies one chunk ahead of the elimination.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.b32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity; gives up after ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer_ns() - t0 > 2000000000ull) return false;
    }
}

struct Chunk {
    int p, h;          // pair, half (0: the pair's second direction, 1: its first)
    int64_t s0;        // first step record of the half-ray
    int n;             // half-ray length
    int k_lo, k_hi;    // steps covered by the chunk
};

// The origin's half-rays as {first step record, length}, ext[2 p + h], read
// from the ray offsets once per item into shared memory.
__device__ __forceinline__ void fill_extents(const FSArgs &a, int64_t o, longlong2 *ext, int tid, int bd)
{
    for (int t = tid; t < 2 * a.P; t += bd) {
        const int2 pr = a.pairs[t >> 1];
        const int r = (t & 1) == 0 ? pr.y : pr.x;
        const int64_t i = (int64_t)r * a.N + o;
        const int64_t s0 = a.ray_off[i], len = a.ray_off[i + 1] - s0;
        if (s0 < 0 || len < 0 || len > a.N || s0 + len > a.n_rec) {   // index check: record, empty half-ray
            if (atomicCAS(a.err, 0, (int)kDevBounds) == 0) {
                a.err[1] = 23;
                a.err[2] = (int)o;
                a.err[3] = (int)t;
            }
            ext[t] = make_longlong2(0, 0);
        } else {
            ext[t] = make_longlong2(s0, len);
        }
    }
}

__device__ __forceinline__ void half_extent(const longlong2 *ext, int p, int h, int64_t &s0, int &n)
{
    const longlong2 e = ext[2 * p + h];
    s0 = e.x;
    n = (int)e.y;
}

// First chunk at or after half (p, h); false if none.
__device__ __forceinline__ bool first_chunk_from(const longlong2 *ext, int P, int p, int h, int CH, Chunk &c)
{
    for (; p < P; ++p, h = 0) {
        for (; h < 2; ++h) {
            int64_t s0;
            int n;
            half_extent(ext, p, h, s0, n);
            if (n > 0) {
                c = {p, h, s0, n, max(1, n - CH + 1), n};
                return true;
            }
        }
    }
    return false;
}

__device__ __forceinline__ bool next_chunk(const longlong2 *ext, int P, const Chunk &cur, int CH, Chunk &nx)
{
    if (cur.k_lo > 1) {
        nx = cur;
        nx.k_hi = cur.k_lo - 1;
        nx.k_lo = max(1, nx.k_hi - CH + 1);
        return true;
    }
    return cur.h == 0 ? first_chunk_from(ext, P, cur.p, 1, CH, nx) : first_chunk_from(ext, P, cur.p + 1, 0, CH, nx);
}

// Issue the copies of chunk c into one buffer (warp 0).  Point slot j holds
// c_{k_lo-1+j} (c_0 = o); step slot j holds the record of step k_lo-1+j
// (slot 0 unused when k_lo = 1).
template <typename T>
__device__ __forceinline__ void issue_chunk(const FSArgs &a, int64_t o, const Chunk &c, unsigned char *steps_buf,
                                            unsigned char *rows_buf, uint64_t *bar, int rowB, int lane)
{
    constexpr int SB = sizeof(T) == 4 ? 16 : 32;
    const int npts = c.k_hi - c.k_lo + 2;
    const int kf = max(1, c.k_lo - 1);
    const int nsteps = c.k_hi - kf + 1;
    const uint32_t bytes = (uint32_t)(npts * rowB + nsteps * SB);
    const unsigned char *lines = reinterpret_cast<const unsigned char *>(a.line);
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane < npts) {
        const int k = c.k_lo - 1 + lane;
        int64_t pt = k == 0 ? o : (int64_t)__ldg(&a.s32[c.s0 + k - 1].x);
        if (pt < 0 || pt >= a.N) {   // a point index from the ray records out of range: record, copy row 0
            if (atomicCAS(a.err, 0, (int)kDevBounds) == 0) {
                a.err[1] = 20;
                a.err[2] = (int)o;
                a.err[3] = (int)pt;
            }
            pt = 0;
        }
        bulk_g2s(rows_buf + lane * rowB, lines + pt * (int64_t)rowB, (uint32_t)rowB, bar);
    }
    if (lane == 0) {
        const void *src = sizeof(T) == 4 ? (const void *)(a.s32 + c.s0 + kf - 1) : (const void *)(a.s64 + c.s0 + kf - 1);
        bulk_g2s(steps_buf + (kf - (c.k_lo - 1)) * SB, src, (uint32_t)(nsteps * SB), bar);
    }
}

// Shared-memory carve-out of the staged kernel (bytes from the dynamic base),
// computed identically on the host (launch size) and the device.
struct StagedLayout {
    int stage, coef, ibg, sab, acc, half0, ext, total;
};

// Staging buffers [2] and coefficient buffers [2] are contiguous; the final
// FP64 reduction area aliases them once the last chunk is done.
template <typename T, int LPT, int CH>
__host__ __device__ inline StagedLayout staged_layout(int Q, int Mb, int RS, int bd, int P, bool fused)
{
    constexpr int SB = sizeof(T) == 4 ? 16 : 32;
    constexpr int NPT = CH + 1;
    auto up = [](int x) { return (x + 15) & ~15; };
    StagedLayout L;
    const int rowB = RS * (int)sizeof(T);
    const int stage_bytes = 2 * NPT * (SB + rowB);
    const int coef_bytes = fused ? 0 : 2 * (CH + 1) * Q * 2 * (int)sizeof(T);
    const int red_bytes = 2 * Mb * Q * (int)sizeof(double);
    L.stage = 128;
    L.coef = L.stage + up(stage_bytes);
    const int pipe_end = L.coef + up(coef_bytes);
    L.ibg = pipe_end > L.stage + up(red_bytes) ? pipe_end : L.stage + up(red_bytes);
    L.sab = L.ibg + up(Mb * Q * (int)sizeof(T));
    L.acc = L.sab + up(2 * Q * (int)sizeof(T));
    L.half0 = L.acc + up(3 * LPT * bd * (int)sizeof(T));
    L.ext = L.half0 + up(3 * LPT * bd * (int)sizeof(T));
    L.total = L.ext + 2 * P * 16;
    return L;
}

// Halved {cf, cn} of step k (far point in staged slot jf = k - k_lo + 1, near
// point in slot jf - 1) for the bin with offsets Aq, Bq: z_f = Aq + Bq beta_far;
// gpair() gives the Gaussians {g_f, g_n} of the two points, which only the
// trapezoid uses.  One function for every schedule, so that all of them
// compute bit-identical coefficients.
template <typename T, typename GP>
__device__ __forceinline__ typename Prec<T>::V2 segment_item(const FSArgs &a, int64_t o, int r, int k, int q,
                                                             const unsigned char *Sb, const T *Rb, int jf, T Aq, T Bq,
                                                             const StepG<T> &sf, T z_f, GP gpair)
{
    using V2 = typename Prec<T>::V2;
    constexpr int SB = sizeof(T) == 4 ? 16 : 32;
    const T thr = (T)a.thr;
    const int jn = jf - 1;
    const T *rowf = Rb + jf * a.RS, *rown = Rb + jn * a.RS;
    const T w_f = rowf[2 * a.Mpad], w_n = rown[2 * a.Mpad];
    const T du = -Prec<T>::mul(Bq, sf.dbw);
    bool trap = fabs(du) < thr;
    if (sizeof(T) == 4 && fabs(fabs(du) - thr) < T(kSwitchBand) * thr) {
        const int64_t c_f = reinterpret_cast<const int4 *>(Sb + jf * SB)->x;
        const int64_t c_n = k > 1 ? (int64_t)reinterpret_cast<const int4 *>(Sb + jn * SB)->x : o;
        trap = trapezoid_fp64(a, r, c_f, c_n, a.xq[q], a.w64[o]);
    }
    T cf, cn;
    if (a.subdiv > 0) {
        const T z_n = bin_z<T>(Aq, Bq, k > 1 ? step_from<T>(Sb + jn * SB).beta : T(0));
        subdiv_coefs<T>(a.subdiv, sf.dx, z_f, w_f, z_n, w_n, cf, cn);
    } else if (trap) {
        const V2 g = gpair();
        segment_coefs<T>(true, sf.dx, du, z_f, g.x, w_f, g.y, w_n, a.width_mode, cf, cn);
    } else {
        segment_coefs<T>(false, sf.dx, du, z_f, T(0), w_f, T(0), w_n, a.width_mode, cf, cn);
    }
    return V2{cf, cn};
}

// Two items of the FP32 pre-pass at once on packed FP32 (one lane per item),
// lane for lane the arithmetic of segment_item / segment_coefs, so the
// coefficients are bit-identical.  An item's inputs:
struct PairIn {
    float dx, z_f, z_n, du, w_f, w_n, rw_f, rw_n;
    bool trap, band;
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 f2s(float x) { return make_float2(x, x); }

// Both items on the same branch (neither near the switch): their halved
// {cf, cn} in c0, c1.
__device__ __forceinline__ void segment_pair(const PairIn &i0, const PairIn &i1, int width_mode, float2 &c0,
                                             float2 &c1)
{
    const float2 dx = f2(i0.dx, i1.dx), wf = f2(i0.w_f, i1.w_f), wn = f2(i0.w_n, i1.w_n);
    float2 cf, cn;
    if (i0.trap) {
        // Gaussians of the far and near points (point_gauss on each lane)
        const float2 uf = __fmul2_rn(f2(i0.z_f, i1.z_f), f2(i0.rw_f, i1.rw_f));
        const float2 un = __fmul2_rn(f2(i0.z_n, i1.z_n), f2(i0.rw_n, i1.rw_n));
        const float2 yf = __fmul2_rn(__fmul2_rn(uf, uf), f2s(-kLog2E));
        const float2 yn = __fmul2_rn(__fmul2_rn(un, un), f2s(-kLog2E));
        const float2 gf = f2(ex2_mufu(yf.x), ex2_mufu(yf.y)), gn = f2(ex2_mufu(yn.x), ex2_mufu(yn.y));
        const float2 q = __fmul2_rn(f2s(0.25f), dx);
        cf = __fmul2_rn(q, gf);
        cn = __fmul2_rn(q, gn);
    } else {
        float2 iw;
        if (width_mode == 0) {
            const float2 h = __fmul2_rn(f2s(0.5f), __ffma2_rn(wf, wf, __fmul2_rn(wn, wn)));
            iw = f2(rsqrtf(h.x), rsqrtf(h.y));
        } else {
            const float2 h = __fmul2_rn(f2s(0.5f), __fadd2_rn(wf, wn));
            iw = f2(Prec<float>::rcp(h.x), Prec<float>::rcp(h.y));
        }
        const float2 du = f2(i0.du, i1.du);
        float2 a = __fmul2_rn(f2(i0.z_f, i1.z_f), iw);
        float2 b = __fadd2_rn(a, du);
        const float2 sab = __fadd2_rn(a, b);
        if (sab.x < 0.0f) {
            const float t = a.x;
            a.x = -b.x;
            b.x = -t;
        }
        if (sab.y < 0.0f) {
            const float t = a.y;
            a.y = -b.y;
            b.y = -t;
        }
        const float2 ea = erfc_fit2(a.x, a.y), eb = erfc_fit2(b.x, b.y);
        const float2 E = __fadd2_rn(ea, f2(-eb.x, -eb.y));
        const float2 rdu = f2(Prec<float>::rcp(du.x), Prec<float>::rcp(du.y));
        const float2 kk =
            __fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(dx, f2s(float(0.125 * kSqrtPi))), E), iw), rdu);
        cf = __fmul2_rn(kk, wf);
        cn = __fmul2_rn(kk, wn);
    }
    c0 = f2(cf.x, cn.x);
    c1 = f2(cf.y, cn.y);
}

// Line-independent coefficients of every (bin, step) of one chunk, shared by
// the CTA's line groups: coef[q * cs + (k - k_lo)] = halved {cf, cn} of step k
// for bin q.  Each bin's steps are contiguous, so the elimination steps its
// pointer by a constant; the row stride cs = CH + 1 is odd, so the threads of
// consecutive bins read different banks.
// Two ways to share the items among the CTA's threads:
//  * strided (CARRY false): item kk * Q + q to thread (kk * Q + q) mod bd;
//  * runs (CARRY true): thread t takes bin t mod Q and a run of consecutive
//    steps; the near point of a step is the far point of the step before, so
//    its Gaussian is carried instead of recomputed.  This pays where the
//    pre-pass dominates (few lines per origin, 4 lines per thread), while with
//    many lines the extra live registers cost more than the saved exponentials.
template <typename T, bool CARRY>
__device__ __forceinline__ void chunk_coefs(const FSArgs &a, int64_t o, int r, int k_lo, int k_hi,
                                            const unsigned char *Sb, const T *Rb, const T *sA, const T *sB,
                                            typename Prec<T>::V2 *coef, int cs, int tid, int bd)
{
    using V2 = typename Prec<T>::V2;
    constexpr int SB = sizeof(T) == 4 ? 16 : 32;
    const int nst = k_hi - k_lo + 1;
    // one segment's coefficients into the chunk's buffer
    auto one = [&](int kk, int q, T Aq, T Bq, const StepG<T> &sf, T z_f, auto gpair) {
        coef[q * cs + kk] = segment_item<T>(a, o, r, k_lo + kk, q, Sb, Rb, kk + 1, Aq, Bq, sf, z_f, gpair);
    };
    if constexpr (CARRY) {
        const int nseg = bd / a.Q;                     // Q <= bd: bins x line groups fit the CTA
        const int seg = tid / a.Q, q = tid - seg * a.Q;
        const int sps = (nst + nseg - 1) / nseg;
        const int kk0 = seg * sps, kk1 = min(nst, kk0 + sps);
        if (seg >= nseg || kk0 >= kk1) return;
        const T Aq = sA[q], Bq = sB[q];
        T g_n = point_gauss<T>(bin_z<T>(Aq, Bq, k_lo + kk0 > 1 ? step_from<T>(Sb + kk0 * SB).beta : T(0)),
                               Rb[kk0 * a.RS + 2 * a.Mpad + 1]);
#pragma unroll 1
        for (int kk = kk0; kk < kk1; ++kk) {
            const StepG<T> sf = step_from<T>(Sb + (kk + 1) * SB);
            const T z_f = bin_z<T>(Aq, Bq, sf.beta);
            const T g_f = point_gauss<T>(z_f, Rb[(kk + 1) * a.RS + 2 * a.Mpad + 1]);
            one(kk, q, Aq, Bq, sf, z_f, [&] { return V2{g_f, g_n}; });
            g_n = g_f;
        }
    } else {
        // warp 0 issues the bulk copies after the barrier: in a wide CTA it
        // takes no items, and the last threads take the extra items of an
        // uneven split
        // item it = kk Q + q; the stride advances (kk, q) by (dk, dq)
        // without a division per item
        const int items = a.Q * nst;
        const int pw = bd >= 128 ? 32 : 0;
        const int stride = bd - pw;
        const int dk = stride / a.Q, dq = stride - dk * a.Q;
        const int it0 = tid >= pw ? bd - 1 - tid : items;
        int kk = it0 / a.Q, q = it0 - kk * a.Q;
        if constexpr (sizeof(T) == 4) {
            if (a.subdiv == 0) {
                // two adjacent items per trip (bins q and q + 1 of one step,
                // or the last bin of a step and the first of the next), on
                // packed FP32 when both take the same branch away from the
                // switch
                auto item_in = [&](int kk_, int q_, PairIn &in, StepG<T> &sf, T &Aq, T &Bq, T &beta_n) {
                    const int k = k_lo + kk_, jf = kk_ + 1;
                    sf = step_from<T>(Sb + jf * SB);
                    beta_n = k > 1 ? step_from<T>(Sb + kk_ * SB).beta : T(0);
                    Aq = sA[q_];
                    Bq = sB[q_];
                    in.dx = sf.dx;
                    in.z_f = bin_z<T>(Aq, Bq, sf.beta);
                    in.z_n = bin_z<T>(Aq, Bq, beta_n);
                    in.w_f = Rb[jf * a.RS + 2 * a.Mpad];
                    in.w_n = Rb[kk_ * a.RS + 2 * a.Mpad];
                    in.rw_f = Rb[jf * a.RS + 2 * a.Mpad + 1];
                    in.rw_n = Rb[kk_ * a.RS + 2 * a.Mpad + 1];
                    in.du = -Prec<T>::mul(Bq, sf.dbw);
                    in.trap = fabs(in.du) < (T)a.thr;
                    in.band = fabs(fabs(in.du) - (T)a.thr) < T(kSwitchBand) * (T)a.thr;
                };
                auto single = [&](int kk_, int q_, const StepG<T> &sf, T Aq, T Bq, const PairIn &in) {
                    one(kk_, q_, Aq, Bq, sf, in.z_f, [&] {
                        return V2{point_gauss<T>(in.z_f, in.rw_f), point_gauss<T>(in.z_n, in.rw_n)};
                    });
                };
                const int npairs = (items + 1) >> 1;
                const int pstride2 = 2 * stride;
                const int dk2 = pstride2 / a.Q, dq2 = pstride2 - dk2 * a.Q;
                const int p0 = tid >= pw ? bd - 1 - tid : npairs;
                int kk0 = (2 * p0) / a.Q, q0 = 2 * p0 - kk0 * a.Q;
#pragma unroll 1
                for (int pi = p0; pi < npairs; pi += stride) {
                    int kk1 = kk0, q1 = q0 + 1;
                    if (q1 >= a.Q) {
                        q1 = 0;
                        ++kk1;
                    }
                    PairIn in0, in1;
                    StepG<T> sf0, sf1;
                    T A0, B0, bn0, A1, B1, bn1;
                    item_in(kk0, q0, in0, sf0, A0, B0, bn0);
                    if (2 * pi + 1 < items) {
                        item_in(kk1, q1, in1, sf1, A1, B1, bn1);
                        if (!in0.band && !in1.band && in0.trap == in1.trap) {
                            float2 c0, c1;
                            segment_pair(in0, in1, a.width_mode, c0, c1);
                            coef[q0 * cs + kk0] = c0;
                            coef[q1 * cs + kk1] = c1;
                        } else {
                            single(kk0, q0, sf0, A0, B0, in0);
                            single(kk1, q1, sf1, A1, B1, in1);
                        }
                    } else {
                        single(kk0, q0, sf0, A0, B0, in0);
                    }
                    kk0 += dk2;
                    q0 += dq2;
                    if (q0 >= a.Q) {
                        q0 -= a.Q;
                        ++kk0;
                    }
                }
                return;
            }
        }
#pragma unroll 1
        for (int it = it0; it < items; it += stride) {
            const int k = k_lo + kk;
            const StepG<T> sf = step_from<T>(Sb + (kk + 1) * SB);
            const T beta_n = k > 1 ? step_from<T>(Sb + kk * SB).beta : T(0);
            const T Aq = sA[q], Bq = sB[q];
            const T z_f = bin_z<T>(Aq, Bq, sf.beta);
            one(kk, q, Aq, Bq, sf, z_f, [&] {
                return V2{point_gauss<T>(z_f, Rb[(kk + 1) * a.RS + 2 * a.Mpad + 1]),
                          point_gauss<T>(bin_z<T>(Aq, Bq, beta_n), Rb[kk * a.RS + 2 * a.Mpad + 1])};
            });
            kk += dk;
            q += dq;
            if (q >= a.Q) {
                q -= a.Q;
                ++kk;
            }
        }
    }
}

// The origin of visiting-order entry oi; an entry outside the model is
// recorded in the error word (site 24) and replaced by point 0.
__device__ __noinline__ int64_t checked_origin(const FSArgs &a, int64_t oi, int tid)
{
    const int64_t o = a.order[oi];
    if (o >= 0 && o < a.N) return o;
    if (tid == 0 && atomicCAS(a.err, 0, (int)kDevBounds) == 0) {
        a.err[1] = 24;
        a.err[2] = (int)oi;
        a.err[3] = (int)o;
    }
    return 0;
}

// One (origin, line block) item of the staged schedule, run by the whole CTA:
// origin order index oi, line block blk.  The mbarriers at the base of shared
// memory are initialised once per CTA; `ci` counts the chunks the CTA has
// consumed so far, so their phases carry over from one item to the next.
// Returns false if a wait gave up: the error word is set and no copy of this
// CTA is left in flight.
template <typename T, int LPT, int CH, bool FAST, bool FUSED>
__device__ __forceinline__ bool fs_staged_item(const FSArgs &a, int64_t oi, int blk, unsigned char *smem, int &ci)
{
    using V2 = typename Prec<T>::V2;
    constexpr int SB = sizeof(T) == 4 ? 16 : 32;
    constexpr int NPT = CH + 1;
    static_assert(NPT <= 32, "one point row per producer lane");
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rowB = a.RS * (int)sizeof(T);
    const int Mb = a.Gb * LPT;
    const StagedLayout lay = staged_layout<T, LPT, CH>(a.Q, Mb, a.RS, bd, a.P, FUSED);

    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);                   // [2]
    int *abort_flag = reinterpret_cast<int *>(smem + 16);
    unsigned char *steps_s = smem + lay.stage;                            // steps [2][NPT][SB]
    unsigned char *rows_s = steps_s + 2 * NPT * SB;                       // rows [2][NPT][rowB]
    V2 *coef = reinterpret_cast<V2 *>(smem + lay.coef);                   // [2][Q][CH + 1]
    T *ibg = reinterpret_cast<T *>(smem + lay.ibg);                       // [Mb][Q]
    T *sA = reinterpret_cast<T *>(smem + lay.sab), *sB = sA + a.Q;        // [Q] each
    T *acc = reinterpret_cast<T *>(smem + lay.acc);                       // [3][LPT][bd]
    T *half0 = reinterpret_cast<T *>(smem + lay.half0);                   // [3][LPT][bd] first half's P, Y, a
    longlong2 *ext = reinterpret_cast<longlong2 *>(smem + lay.ext);       // [2 P] half-ray extents
    double *red = reinterpret_cast<double *>(smem + lay.stage);           // reuses staging + coefficients at the end

    const int64_t o = checked_origin(a, oi, tid);
    const int gl = tid / a.Q, q = tid - gl * a.Q;
    const int gg = blk * a.Gb + gl;
    const int line0 = gg * LPT;
    const bool active = tid < a.Q * a.Gb && gg < a.Gtot;

    const double wo64 = a.w64[o];
    fill_extents(a, o, ext, tid, bd);
    if (tid < a.Q) {
        const T Aq = T(a.xq[tid]) * T(wo64);
        sA[tid] = Aq;
        sB[tid] = T(1) + Aq;
    }
    if (active) {
        T Ibg[LPT];
        background<T, LPT>(a, line0, a.xq[q], wo64, Ibg);
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            ibg[(gl * LPT + l) * a.Q + q] = Ibg[l];
            for (int c = 0; c < 3; ++c) acc[pair_slot<T, LPT>(c, l, bd, tid)] = T(0);
        }
    }
    __syncthreads();

    Chunk cur;
    const bool any = first_chunk_from(ext, a.P, 0, 0, CH, cur);
    if (any && warp == 0) issue_chunk<T>(a, o, cur, steps_s + (ci & 1) * NPT * SB, rows_s + (ci & 1) * NPT * rowB,
                                         &bar[ci & 1], rowB, lane);

    const T wqn = active ? T(a.wq[q]) : T(0);
    bool ok = true;
    T P[LPT], Y[LPT], aa[LPT];
    // FUSED (one line group: the thread is the only reader of its bin's
    // coefficients): the bin's offsets, and the Gaussian of the far point of
    // the next step, carried down the half-ray
    T Aq = T(0), Bq = T(0), gcar = T(0);
    if constexpr (FUSED) {
        if (active) {
            Aq = sA[q];
            Bq = sB[q];
        }
    }
    for (int p = 0; p < a.P; ++p) {
        const int2 pr = a.pairs[p];
        for (int h = 0; h < 2; ++h) {
            const int r = h == 0 ? pr.y : pr.x;
            int64_t s0;
            int n;
            half_extent(ext, p, h, s0, n);
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                P[l] = T(2);
                Y[l] = active ? ibg[(gl * LPT + l) * a.Q + q] : T(0);
                aa[l] = T(0);
            }
            for (int k_hi = n; k_hi >= 1; k_hi -= CH) {
                const int k_lo = max(1, k_hi - CH + 1);
                ok = mbar_wait_bounded(&bar[ci & 1], (ci >> 1) & 1);
                const unsigned char *Sb = steps_s + (ci & 1) * NPT * SB;
                const T *Rb = reinterpret_cast<const T *>(rows_s + (ci & 1) * NPT * rowB);
                V2 *cf_buf = coef + (ci & 1) * (CH + 1) * a.Q;
                if constexpr (!FUSED) {
                    if (ok) chunk_coefs<T, LPT == 4>(a, o, r, k_lo, k_hi, Sb, Rb, sA, sB, cf_buf, CH + 1, tid, bd);
                }
                // one barrier per chunk: this chunk's coefficients are complete, and
                // everyone is done with the previous chunk (its staging buffer is
                // refilled next, its coefficient buffer on the following chunk);
                // stop together if any wait gave up
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) *abort_flag = 1;
                    goto done;
                }

                if (warp == 0) {
                    Chunk nx;
                    const Chunk c{p, h, s0, n, k_lo, k_hi};
                    if (next_chunk(ext, a.P, c, CH, nx))
                        issue_chunk<T>(a, o, nx, steps_s + ((ci + 1) & 1) * NPT * SB,
                                       rows_s + ((ci + 1) & 1) * NPT * rowB, &bar[(ci + 1) & 1], rowB, lane);
                }
                if (FUSED && active) {
                    // the same rows with each step's coefficients computed here
                    // (segment_item, as the pre-pass does) instead of read
                    const T *row = Rb + (k_hi - k_lo + 1) * a.RS + line0;
                    auto coef_of = [&](int k) -> V2 {
                        const int jf = k - k_lo + 1;
                        const StepG<T> sf = step_from<T>(Sb + jf * SB);
                        const T z_f = bin_z<T>(Aq, Bq, sf.beta);
                        const T z_n = bin_z<T>(Aq, Bq, k > 1 ? step_from<T>(Sb + (jf - 1) * SB).beta : T(0));
                        const T g_f = gcar;
                        gcar = point_gauss<T>(z_n, Rb[(jf - 1) * a.RS + 2 * a.Mpad + 1]);
                        const T g_n = gcar;
                        return segment_item<T>(a, o, r, k, q, Sb, Rb, jf, Aq, Bq, sf, z_f,
                                               [&] { return V2{g_f, g_n}; });
                    };
                    if (k_hi == n) {                   // the half-ray's far end
                        const int jf = n - k_lo + 1;
                        gcar = point_gauss<T>(bin_z<T>(Aq, Bq, step_from<T>(Sb + jf * SB).beta),
                                              Rb[jf * a.RS + 2 * a.Mpad + 1]);
                    }
                    T chiA[LPT], chiB[LPT], S_f[LPT];
                    load_vec<LPT>(row, chiA);
                    int k = k_hi;
                    if constexpr (FAST) {
                        T D[LPT];
#pragma unroll 1
                        for (; k - 1 >= k_lo; k -= 2) {
                            V2 cc = coef_of(k);
                            load_vec<LPT>(row + a.Mpad, S_f);
                            load_vec<LPT>(row - a.RS, chiB);
                            homog_row1_packed<LPT>(cc.x, cc.y, chiA, S_f, chiB, P, Y, aa, D);
                            cc = coef_of(k - 1);
                            load_vec<LPT>(row - a.RS + a.Mpad, S_f);
                            load_vec<LPT>(row - 2 * a.RS, chiA);
                            homog_row2_packed<LPT>(cc.x, cc.y, chiB, S_f, chiA, P, Y, aa, D);
                            row -= 2 * a.RS;
                        }
                    } else {
#pragma unroll 1
                        for (; k - 1 >= k_lo; k -= 2) {
                            V2 cc = coef_of(k);
                            load_vec<LPT>(row + a.Mpad, S_f);
                            load_vec<LPT>(row - a.RS, chiB);
                            eliminate_row<T, LPT>(cc.x, cc.y, chiA, S_f, chiB, P, Y, aa);
                            cc = coef_of(k - 1);
                            load_vec<LPT>(row - a.RS + a.Mpad, S_f);
                            load_vec<LPT>(row - 2 * a.RS, chiA);
                            eliminate_row<T, LPT>(cc.x, cc.y, chiB, S_f, chiA, P, Y, aa);
                            row -= 2 * a.RS;
                        }
                    }
                    if (k == k_lo) {
                        const V2 cc = coef_of(k);
                        load_vec<LPT>(row + a.Mpad, S_f);
                        load_vec<LPT>(row - a.RS, chiB);
                        eliminate_row<T, LPT>(cc.x, cc.y, chiA, S_f, chiB, P, Y, aa);
                    }
                } else if (!FUSED && active) {
                    // step k reads rows jf = k - k_lo + 1 and jn = jf - 1; the
                    // near row's chi is the next step's far chi, so two steps
                    // per trip swap the two chi arrays instead of reloading
                    const T *row = Rb + (k_hi - k_lo + 1) * a.RS + line0;
                    const V2 *cfp = cf_buf + q * (CH + 1) + (k_hi - k_lo);
                    T chiA[LPT], chiB[LPT], S_f[LPT];
                    load_vec<LPT>(row, chiA);
                    int k = k_hi;
                    if constexpr (FAST) {
                        // two rows per reciprocal (the launch checked the range)
                        T D[LPT];
#pragma unroll 1
                        for (; k - 1 >= k_lo; k -= 2) {
                            V2 cc = *cfp;
                            load_vec<LPT>(row + a.Mpad, S_f);
                            load_vec<LPT>(row - a.RS, chiB);
                            homog_row1_packed<LPT>(cc.x, cc.y, chiA, S_f, chiB, P, Y, aa, D);
                            cc = *(cfp - 1);
                            load_vec<LPT>(row - a.RS + a.Mpad, S_f);
                            load_vec<LPT>(row - 2 * a.RS, chiA);
                            homog_row2_packed<LPT>(cc.x, cc.y, chiB, S_f, chiA, P, Y, aa, D);
                            row -= 2 * a.RS;
                            cfp -= 2;
                        }
                    } else {
#pragma unroll 1
                        for (; k - 1 >= k_lo; k -= 2) {
                            V2 cc = *cfp;
                            load_vec<LPT>(row + a.Mpad, S_f);
                            load_vec<LPT>(row - a.RS, chiB);
                            eliminate_row<T, LPT>(cc.x, cc.y, chiA, S_f, chiB, P, Y, aa);
                            cc = *(cfp - 1);
                            load_vec<LPT>(row - a.RS + a.Mpad, S_f);
                            load_vec<LPT>(row - 2 * a.RS, chiA);
                            eliminate_row<T, LPT>(cc.x, cc.y, chiB, S_f, chiA, P, Y, aa);
                            row -= 2 * a.RS;
                            cfp -= 2;
                        }
                    }
                    if (k == k_lo) {
                        const V2 cc = *cfp;
                        load_vec<LPT>(row + a.Mpad, S_f);
                        load_vec<LPT>(row - a.RS, chiB);
                        eliminate_row<T, LPT>(cc.x, cc.y, chiA, S_f, chiB, P, Y, aa);
                    }
                }
                ++ci;
            }
            if (h == 0) {
                if (active) {
#pragma unroll
                    for (int l = 0; l < LPT; ++l) {
                        half0[pair_slot<T, LPT>(0, l, bd, tid)] = P[l];
                        half0[pair_slot<T, LPT>(1, l, bd, tid)] = Y[l];
                        half0[pair_slot<T, LPT>(2, l, bd, tid)] = aa[l];
                    }
                }
            } else if (active) {
                T So[LPT], PL[LPT], YL[LPT], aL[LPT];
                load_vec<LPT>(reinterpret_cast<const T *>(a.line) + o * a.RS + a.Mpad + line0, So);
#pragma unroll
                for (int l = 0; l < LPT; ++l) {
                    PL[l] = half0[pair_slot<T, LPT>(0, l, bd, tid)];
                    YL[l] = half0[pair_slot<T, LPT>(1, l, bd, tid)];
                    aL[l] = half0[pair_slot<T, LPT>(2, l, bd, tid)];
                }
                if constexpr (sizeof(T) == 4)
                    combine_accumulate_packed<LPT>(wqn, So, PL, YL, aL, P, Y, aa, acc, bd, tid);
                else
                    combine_accumulate<T, LPT>(wqn, So, PL, YL, aL, P, Y, aa, acc, bd, tid);
            }
        }
    }
done:
    __syncthreads();
    if (*abort_flag) {
        // give in-flight copies a bounded chance to land before the CTA exits
        if (tid == 0) {
            if (atomicCAS(a.err, 0, (int)kDevTimeout) == 0) {
                a.err[1] = 3;
                a.err[2] = (int)oi;
                a.err[3] = ci;
            }
            mbar_wait_bounded(&bar[ci & 1], (ci >> 1) & 1);
            mbar_wait_bounded(&bar[(ci + 1) & 1], ((ci + 1) >> 1) & 1);
        }
        return false;
    }
    if (active) {
        const int lb = gl * LPT;
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            if (line0 + l < a.M) {
                red[(0 * Mb + lb + l) * a.Q + q] =
                    (double)acc[pair_slot<T, LPT>(0, l, bd, tid)] - (double)acc[pair_slot<T, LPT>(1, l, bd, tid)];
                red[(1 * Mb + lb + l) * a.Q + q] = (double)acc[pair_slot<T, LPT>(2, l, bd, tid)];
            }
        }
    }
    __syncthreads();
    reduce_out(a, red, Mb, blk * Mb, oi, true);
    // the next item's bulk copies land where this item's reduction was written
    // through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    return true;
}

__device__ __forceinline__ void staged_init(unsigned char *smem)
{
    if (threadIdx.x == 0) {
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *reinterpret_cast<int *>(smem + 16) = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// One CTA per (origin, line block): blockIdx.x is the origin's place in the
// visiting order, blockIdx.y the line block.  FAST: the two-row elimination,
// which only runs when no point of the model is outside its range (the line
// data set *range_bad otherwise; every CTA then returns at once and
// k_fs_exact does the work).
template <typename T, int LPT, int CH, int MINB, bool FAST, bool FUSED>
__global__ void __launch_bounds__(256, MINB) k_fs_staged(FSArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if constexpr (FAST) {
        if (*a.range_bad) return;
    }
    staged_init(smem);
    int ci = 0;
    fs_staged_item<T, LPT, CH, FAST, FUSED>(a, (int64_t)blockIdx.x, (int)blockIdx.y, smem, ci);
}

// The one-row elimination of every item of a model whose range figures
// exclude the two-row form (*range_bad set), in a persistent grid; launched
// after the two-row kernel, it returns at once for every other model.
template <typename T, int LPT, int CH, bool FUSED> __global__ void __launch_bounds__(256, 2) k_fs_exact(FSArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (!*a.range_bad) return;
    staged_init(smem);
    int ci = 0;
    const int64_t items = a.N * a.nblk;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t oi = it / a.nblk;
        if (!fs_staged_item<T, LPT, CH, false, FUSED>(a, oi, (int)(it - oi * a.nblk), smem, ci)) return;
    }
}

// Many models in one persistent launch.  Items (model, origin, line block)
// are numbered model after model (models in the order of the table, origins
// in each model's visiting order, the line blocks of an origin together);
// each CTA takes the next item from a global counter until none is left.
// item_end[i] is one past the last item of model i.
struct FSBatchArgs {
    const FSArgs *args;        // [n_models]
    const int64_t *item_end;   // [n_models]
    int n_models;
    int64_t n_items;
    unsigned long long *next;  // item counter, zero at launch
};

// A model's items take the two-row elimination: no point outside its range,
// half-rays shorter than kFastSteps, and the switch rule's optical depths.
__device__ __forceinline__ bool two_row_ok(const FSArgs &a)
{
    return !*a.range_bad && a.subdiv == 0 && a.N < kFastSteps;
}

template <typename T, int CH, bool FUSED, int LPT> __global__ void __launch_bounds__(256, 2) k_fs_batch(FSBatchArgs b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ FSArgs sa;
    __shared__ int64_t s_item, s_first;
    __shared__ int s_model;
    staged_init(smem);
    int ci = 0, cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t it = (int64_t)atomicAdd(b.next, 1ull);
            int model = -1;
            if (it < b.n_items) {
                int lo = 0, hi = b.n_models - 1;       // first model whose end is past the item
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (b.item_end[mid] > it) hi = mid; else lo = mid + 1;
                }
                model = lo;
                s_first = lo > 0 ? b.item_end[lo - 1] : 0;
                if (lo != cur) sa = b.args[lo];
            }
            s_item = it;
            s_model = model;
        }
        __syncthreads();
        const int model = s_model;
        if (model < 0) return;
        cur = model;
        if (!two_row_ok(sa)) continue;            // the model's items are k_fs_batch_exact's
        const int64_t local = s_item - s_first;
        const int64_t oi = local / sa.nblk;
        const int blk = (int)(local - oi * sa.nblk);
        const bool ok = fs_staged_item<T, LPT, CH, true, FUSED>(sa, oi, blk, smem, ci);
        if (!ok) return;
    }
}

// The items of the batch's models whose range figures exclude the two-row
// form, with the one-row elimination: every CTA walks the models and takes
// every gridDim.x-th item of each such model (returns at once when there is
// none).
template <typename T, int CH, bool FUSED, int LPT>
__global__ void __launch_bounds__(256, 2) k_fs_batch_exact(FSBatchArgs b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ FSArgs sa;
    staged_init(smem);
    int ci = 0;
    for (int mdl = 0; mdl < b.n_models; ++mdl) {
        if (two_row_ok(b.args[mdl])) continue;    // the same for every thread
        __syncthreads();                          // the previous model's items are done with sa
        if (threadIdx.x == 0) sa = b.args[mdl];
        __syncthreads();
        const int64_t first = mdl > 0 ? b.item_end[mdl - 1] : 0, n = b.item_end[mdl] - first;
        for (int64_t it = blockIdx.x; it < n; it += gridDim.x) {
            const int64_t oi = it / sa.nblk;
            const int blk = (int)(it - oi * sa.nblk);
            const bool ok = fs_staged_item<T, LPT, CH, false, FUSED>(sa, oi, blk, smem, ci);
            if (!ok) return;
        }
    }
}

constexpr int kChunk = 30;

template <typename T, int LPT> FSArgs fill_fs_args(const mgt_model *m, bool accumulate)
{
    FSArgs a{};
    const bool all = m->rays_p0 == 0 && m->rays_np == m->P;
    a.N = m->N;
    a.R = m->R;
    a.P = m->rays_np;
    a.Q = m->Q;
    a.M = m->M;
    a.Mpad = m->Mpad;
    a.RS = sizeof(T) == 4 ? row_stride32(m->Mpad) : row_stride64(m->Mpad);
    a.Gtot = (m->M + LPT - 1) / LPT;              // groups covering the real lines
    int gb = a.Gtot;
    while (gb > 1 && a.Q * gb > 256) --gb;
    a.Gb = gb;
    a.OPB = (a.Q * a.Gb >= 256) ? 1 : 256 / (a.Q * a.Gb);
    a.pairs = all ? m->d_pairs : m->d_batch_pairs;
    a.dir_map = all ? nullptr : m->d_dir_map;
    a.accumulate = accumulate ? 1 : 0;
    a.ray_off = m->d_ray_off;
    a.s32 = m->d_steps32;
    a.s64 = m->d_steps64;
    a.line = sizeof(T) == 4 ? (const void *)m->d_line32 : (const void *)m->d_line64;
    a.order = m->d_order;
    a.xq = m->d_xq;
    a.wq = m->d_wq;
    a.line_tab = m->d_line_tab;
    a.vel = m->d_vel;
    a.dirs = m->d_dirs;
    a.w64 = m->d_w64;
    a.thr = m->opts.switch_threshold;
    a.width_mode = m->opts.width_mode;
    a.subdiv = m->opts.subdivisions;
    a.J = m->d_J;
    a.Lst = m->d_Lst;
    a.err = m->d_err;
    a.range_bad = m->d_range_bad;
    a.n_rec = m->total_steps;
    a.lpt = LPT;
    a.nblk = ceil_div(a.Gtot, a.Gb);
    return a;
}

// The staged launch: the two-row kernel and, for the two-row form, the
// one-row fallback.  run = false only raises the kernels' shared-memory limits.
template <typename T, int LPT, int MINB, bool FAST, bool FUSED>
mgt_status launch_staged(const FSArgs &a, dim3 grid, int bd, size_t smem, double fs_bytes, cudaStream_t s, bool run)
{
    auto kfast = k_fs_staged<T, LPT, kChunk, MINB, FAST, FUSED>;
    MGT_TRY_STATUS(raise_smem_limit((const void *)kfast, smem));
    auto kern = k_fs_exact<T, LPT, kChunk, FUSED>;
    if constexpr (FAST) MGT_TRY_STATUS(raise_smem_limit((const void *)kern, smem));
    if (!run) return MGT_OK;
    {
        MGT_KTIMER_BYTES(FUSED ? (sizeof(T) == 4 ? "k_fs_fused<f32>" : "k_fs_fused<f64>")
                               : (sizeof(T) == 4 ? "k_fs_staged<f32>" : "k_fs_staged<f64>"),
                         s, fs_bytes);
        kfast<<<grid, bd, smem, s>>>(a);
    }
    MGT_LAUNCH_CHECK("k_fs_staged");
    if constexpr (FAST) {
        // the same items with the one-row elimination if the model is outside
        // the two-row range (a persistent grid; it returns at once otherwise)
        int dev = 0, sms = 0, per_sm = 0;
        MGT_CUDA(cudaGetDevice(&dev));
        MGT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MGT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bd, smem));
        const int64_t items = (int64_t)grid.x * grid.y;
        const int g = (int)std::min<int64_t>(items, (int64_t)sms * std::max(per_sm, 1));
        {
            MGT_KTIMER("k_fs_exact", s);
            kern<<<g, bd, smem, s>>>(a);
        }
        MGT_LAUNCH_CHECK("k_fs_exact");
    }
    return MGT_OK;
}

template <typename T, int LPT>
mgt_status launch_typed(mgt_model *m, cudaStream_t s, int schedule, bool accumulate, bool run = true)
{
    FSArgs a = fill_fs_args<T, LPT>(m, accumulate);
    // least traffic of a launch: every step record of the held rays once, every
    // point's row once, J-bar and Lambda* written
    const double fs_bytes = (double)m->total_steps * (sizeof(T) == 4 ? 16.0 : 32.0) +
                            (double)m->N * (double)a.RS * sizeof(T) + 16.0 * (double)m->N * m->M;
    const int Mb = a.Gb * LPT;
    // one origin per CTA: the staged kernel (schedule 2: register-capped for
    // two blocks per SM; 3: one block per SM; 4: each thread computes its own
    // bin's coefficients, for models whose lines fit one line group).  The
    // automatic choice is 4 where it applies, else 2.  The staged kernel beats
    // the gather kernel also when one origin fills a single warp (1.5x at 4
    // lines x 31 bins, 3x at 10 lines)
    if (schedule == 4 && a.Gtot != 1)
        return set_error(MGT_ERR_ARG, "formal solve: schedule 4 needs the lines in one group (lines <= lines per thread)");
    const bool staged = schedule != 1;
    if (staged) {
        a.OPB = 1;
        a.fused = (schedule == 4 || (schedule == 0 && a.Gtot == 1)) ? 1 : 0;
        const int threads = a.Q * a.Gb;
        const int bd = ((threads + 31) / 32) * 32;
        if (bd > 256) return set_error(MGT_ERR_ARG, "formal solve: more than 256 bins per origin");
        const size_t smem = (size_t)staged_layout<T, LPT, kChunk>(a.Q, Mb, a.RS, bd, a.P, a.fused != 0).total;
        dim3 grid((unsigned)m->N, (unsigned)ceil_div(a.Gtot, a.Gb));
        // the two-row elimination in FP32 (the subdivided reference keeps the
        // one-row form; the range argument needs half-rays below kFastSteps)
        if constexpr (sizeof(T) == 4) {
            if (a.subdiv == 0 && m->N < kFastSteps) {
                if (a.fused) return launch_staged<T, LPT, 2, true, true>(a, grid, bd, smem, fs_bytes, s, run);
                return schedule == 3 ? launch_staged<T, LPT, 1, true, false>(a, grid, bd, smem, fs_bytes, s, run)
                                     : launch_staged<T, LPT, 2, true, false>(a, grid, bd, smem, fs_bytes, s, run);
            }
        }
        if (a.fused) return launch_staged<T, LPT, 2, false, true>(a, grid, bd, smem, fs_bytes, s, run);
        return schedule == 3 ? launch_staged<T, LPT, 1, false, false>(a, grid, bd, smem, fs_bytes, s, run)
                             : launch_staged<T, LPT, 2, false, false>(a, grid, bd, smem, fs_bytes, s, run);
    }
    const int threads = a.OPB * a.Q * a.Gb;
    const int bd = ((threads + 31) / 32) * 32;
    if (bd > 256) return set_error(MGT_ERR_ARG, "formal solve: too many bins x line groups per block");
    const size_t smem = sizeof(T) * 4 * LPT * bd + sizeof(double) * 2 * a.OPB * Mb * a.Q;
    MGT_TRY_STATUS(raise_smem_limit((const void *)k_fs_gather<T, LPT>, smem));
    dim3 grid((unsigned)ceil_div(m->N, a.OPB), (unsigned)ceil_div(a.Gtot, a.Gb));
    {
        MGT_KTIMER_BYTES(sizeof(T) == 4 ? "k_fs_gather<f32>" : "k_fs_gather<f64>", s, fs_bytes);
        k_fs_gather<T, LPT><<<grid, bd, smem, s>>>(a);
    }
    MGT_LAUNCH_CHECK("k_fs_gather");
    return MGT_OK;
}

}  // namespace

int fs_lines_per_thread(const mgt_model *m, mgt_precision p)
{
    if (p == MGT_FP64) return 4;
    if (m->opts.lines_per_thread == 4 || m->opts.lines_per_thread == 8) return m->opts.lines_per_thread;
    return m->M <= 4 ? 4 : 8;
}

mgt_status launch_formal_solve(mgt_model *m, mgt_precision p, cudaStream_t s, bool accumulate)
{
    const int lpt = fs_lines_per_thread(m, p);
    if (m->Mpad % lpt != 0) return set_error(MGT_ERR_STATE, "line padding does not match the schedule");
    // 0: automatic, 1: gather kernel, 2: staged (two blocks per SM), 3: staged (one block per SM),
    // 4: staged with per-thread coefficients (lines in one group)
    const int sch = m->opts.schedule;
    if (p == MGT_FP64) return launch_typed<double, 4>(m, s, sch, accumulate);
    return lpt == 4 ? launch_typed<float, 4>(m, s, sch, accumulate) : launch_typed<float, 8>(m, s, sch, accumulate);
}


// ---------------------------------------------------------------------------
// Batched launch (k_fs_batch): FP32-mixed, staged schedule, all rays resident.
// ---------------------------------------------------------------------------
size_t fs_args_bytes() { return sizeof(FSArgs); }

mgt_status fs_batch_args(const mgt_model *m, void *args, int *threads, int64_t *items, int *fused, int *lines)
{
    const int lpt = fs_lines_per_thread(m, MGT_FP32_MIXED);
    if (m->Mpad % lpt != 0) return set_error(MGT_ERR_STATE, "line padding does not match the schedule");
    FSArgs a = lpt == 4 ? fill_fs_args<float, 4>(m, false) : fill_fs_args<float, 8>(m, false);
    a.OPB = 1;
    a.fused = a.Gtot == 1 ? 1 : 0;     // as the automatic single-model choice
    const int bd = ((a.Q * a.Gb + 31) / 32) * 32;
    if (bd > 256) return set_error(MGT_ERR_ARG, "batched formal solve: more than 256 bins per origin");
    *threads = bd;
    *items = a.N * a.nblk;
    *fused = a.fused;
    *lines = a.lpt;
    std::memcpy(args, &a, sizeof a);
    return MGT_OK;
}

// One-warp CTAs (models with few lines) take chunks of 14 steps: half the
// staging and coefficient buffers, so twice as many CTAs fit on an SM, and a
// barrier of one warp costs little.  Fused items hold no coefficient buffers,
// and their one-warp CTAs are limited by registers, not shared memory: they
// keep the long chunks.  The arithmetic does not depend on the chunk length.
constexpr int kChunkNarrow = 14;

bool narrow_chunks(int bd, int fused) { return bd == 32 && !fused; }

size_t fs_batch_smem(const void *args, int bd)
{
    FSArgs a;
    std::memcpy(&a, args, sizeof a);
    const int Mb = a.Gb * a.lpt;
    const bool f = a.fused != 0;
    if (narrow_chunks(bd, a.fused))
        return a.lpt == 4 ? (size_t)staged_layout<float, 4, kChunkNarrow>(a.Q, Mb, a.RS, bd, a.P, f).total
                          : (size_t)staged_layout<float, 8, kChunkNarrow>(a.Q, Mb, a.RS, bd, a.P, f).total;
    return a.lpt == 4 ? (size_t)staged_layout<float, 4, kChunk>(a.Q, Mb, a.RS, bd, a.P, f).total
                      : (size_t)staged_layout<float, 8, kChunk>(a.Q, Mb, a.RS, bd, a.P, f).total;
}

namespace {

// The persistent kernels of one class of a batch (one instance per chunk
// length, fused flag and lines per thread, so that each holds one item body
// and keeps the registers of the single-model kernel): one-warp CTAs of
// unfused models take the narrow chunk length.
struct BatchKernels {
    void (*fast)(FSBatchArgs);
    void (*exact)(FSBatchArgs);
};

template <int CH, bool FUSED, int LPT> BatchKernels batch_instance()
{
    return BatchKernels{k_fs_batch<float, CH, FUSED, LPT>, k_fs_batch_exact<float, CH, FUSED, LPT>};
}

BatchKernels batch_kernels(int bd, int fused, int lpt)
{
    if (narrow_chunks(bd, fused))
        return lpt == 8 ? batch_instance<kChunkNarrow, false, 8>() : batch_instance<kChunkNarrow, false, 4>();
    if (fused) return lpt == 8 ? batch_instance<kChunk, true, 8>() : batch_instance<kChunk, true, 4>();
    return lpt == 8 ? batch_instance<kChunk, false, 8>() : batch_instance<kChunk, false, 4>();
}

}  // namespace

mgt_status fs_batch_grid(int bd, int fused, int lpt, size_t smem, size_t max_smem, int *grid)
{
    const BatchKernels k = batch_kernels(bd, fused, lpt);
    MGT_TRY_STATUS(raise_smem_limit((const void *)k.fast, max_smem));
    MGT_TRY_STATUS(raise_smem_limit((const void *)k.exact, max_smem));
    int dev = 0, sms = 0, per_sm = 0;
    MGT_CUDA(cudaGetDevice(&dev));
    MGT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MGT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fast, bd, smem));
    if (per_sm < 1) return set_error(MGT_ERR_ARG, "batched formal solve: a CTA does not fit on an SM");
    *grid = sms * per_sm;
    return MGT_OK;
}

int64_t fs_batch_wave(const void *args, int bd, size_t smem)
{
    FSArgs a;
    std::memcpy(&a, args, sizeof a);
    const BatchKernels k = batch_kernels(bd, a.fused, a.lpt);
    if (raise_smem_limit((const void *)k.fast, smem) != MGT_OK) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fast, bd, smem) != cudaSuccess)
        return 0;
    return (int64_t)sms * per_sm;
}

mgt_status fs_batch_solo(mgt_model *m, cudaStream_t s, bool run)
{
    const int lpt = fs_lines_per_thread(m, MGT_FP32_MIXED);
    if (m->Mpad % lpt != 0) return set_error(MGT_ERR_STATE, "line padding does not match the schedule");
    // the automatic staged schedule, as the persistent launches run it
    return lpt == 4 ? launch_typed<float, 4>(m, s, 0, false, run) : launch_typed<float, 8>(m, s, 0, false, run);
}

mgt_status fs_batch_launch(const void *d_args, const int64_t *d_item_end, int n_models, int64_t n_items,
                           unsigned long long *d_next, int bd, int fused, int lpt, size_t smem, int grid,
                           cudaStream_t s)
{
    FSBatchArgs b{static_cast<const FSArgs *>(d_args), d_item_end, n_models, n_items, d_next};
    MGT_CUDA(cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), s));
    const int64_t g = std::min<int64_t>(grid, n_items);
    {
        MGT_KTIMER("k_fs_batch", s);
        batch_kernels(bd, fused, lpt).fast<<<(unsigned)g, bd, smem, s>>>(b);
    }
    MGT_LAUNCH_CHECK("k_fs_batch");
    // the items of models outside the two-row range (returns at once without)
    {
        MGT_KTIMER("k_fs_batch_exact", s);
        batch_kernels(bd, fused, lpt).exact<<<(unsigned)g, bd, smem, s>>>(b);
    }
    MGT_LAUNCH_CHECK("k_fs_batch_exact");
    return MGT_OK;
}

}  // namespace mgt
