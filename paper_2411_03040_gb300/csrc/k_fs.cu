// Formal solution of the line transfer equation along every ray pair, frequency
// bin and line, reduced into J-bar and Lambda* (the hot loop).
//
// Mapping: one CTA per origin point (or OPB origins when Q * groups is small);
// each thread owns one Gauss-Hermite bin q and LPT consecutive lines and loops
// over all ray pairs.  Every thread of an origin walks the same ray, so trip
// counts never diverge; the per-step, line-independent work (comoving
// frequency, Gaussian, the trapezoid/erf switch, erf) is done once per (q,
// step) and shared by the thread's LPT lines.
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
#include "mgt_common.cuh"

namespace mgt {

namespace {

template <typename T> struct Prec;

template <> struct Prec<float> {
    using LD = float2;
    static __device__ __forceinline__ float rcp(float x)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float gauss(float u) { return __expf(-u * u); }
    static __device__ __forceinline__ float erf_(float x) { return erff(x); }
    static __device__ __forceinline__ float erfc_(float x) { return erfcf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float bg(float f, float hk) { return f * f * f / expm1f(hk * f); }
};

template <> struct Prec<double> {
    using LD = double2;
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double gauss(double u) { return exp(-u * u); }
    static __device__ __forceinline__ double erf_(double x) { return erf(x); }
    static __device__ __forceinline__ double erfc_(double x) { return erfc(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double bg(double f, double hk) { return f * f * f / expm1(hk * f); }
};

struct FSArgs {
    int64_t N;
    int R, P, Q, M, Mpad, Gtot, Gb, OPB;
    const int2 *pairs;
    const int64_t *ray_off;
    const Step32 *s32;
    const Step64 *s64;
    const float2 *w32;
    const double *w64;
    const void *line;          // float2* or double2*, [N][Mpad] {chi~', S'}
    const double *xq, *wq;
    const double *line_tab;    // [8][Mpad]
    const double *vel, *dirs;
    double thr;
    int width_mode;
    double *J, *Lst;           // [N][M]
};

template <typename T> struct StepG {
    int64_t idx;
    T dx, beta, dbw;
};

template <typename T> __device__ __forceinline__ StepG<T> get_step(const FSArgs &a, int64_t s);

template <> __device__ __forceinline__ StepG<float> get_step<float>(const FSArgs &a, int64_t s)
{
    int4 v = __ldg(a.s32 + s);
    return {(int64_t)v.x, __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w)};
}

template <> __device__ __forceinline__ StepG<double> get_step<double>(const FSArgs &a, int64_t s)
{
    int idx = __ldg(&a.s32[s].x);
    const double2 *p = reinterpret_cast<const double2 *>(a.s64 + s);
    double2 v0 = __ldg(p), v1 = __ldg(p + 1);
    return {(int64_t)idx, v0.x, v0.y, v1.x};
}

template <typename T> struct WG {
    T w, iw;
};

template <typename T> __device__ __forceinline__ WG<T> get_w(const FSArgs &a, int64_t c);

template <> __device__ __forceinline__ WG<float> get_w<float>(const FSArgs &a, int64_t c)
{
    float2 v = __ldg(a.w32 + c);
    return {v.x, v.y};
}

template <> __device__ __forceinline__ WG<double> get_w<double>(const FSArgs &a, int64_t c)
{
    double w = __ldg(a.w64 + c);
    return {w, 1.0 / w};
}

template <int LPT> __device__ __forceinline__ void load_line(const float2 *p, float (&chi)[LPT], float (&S)[LPT])
{
    const float4 *v = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < LPT / 2; ++i) {
        float4 x = __ldg(v + i);
        chi[2 * i] = x.x;
        S[2 * i] = x.y;
        chi[2 * i + 1] = x.z;
        S[2 * i + 1] = x.w;
    }
}

template <int LPT> __device__ __forceinline__ void load_line(const double2 *p, double (&chi)[LPT], double (&S)[LPT])
{
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        double2 x = __ldg(p + i);
        chi[i] = x.x;
        S[i] = x.y;
    }
}

// The trapezoid / erf decision re-taken in FP64 for a segment whose FP32
// Doppler-shift ratio lies within rounding of the threshold, so that both
// precisions (and the FP64 reference) branch alike.
__device__ __noinline__ bool trapezoid_fp64(const FSArgs &a, int r, int64_t o, int64_t c_far, int64_t c_near,
                                            double xq64, double wo64)
{
    const double *n = a.dirs + 3 * r;
    const double *vf = a.vel + 3 * c_far, *vn = a.vel + 3 * c_near;
    double dbeta = (n[0] * (vf[0] - vn[0]) + n[1] * (vf[1] - vn[1]) + n[2] * (vf[2] - vn[2])) / kC;
    double wf = a.w64[c_far], wn = a.w64[c_near];
    double wbar = a.width_mode == 0 ? sqrt(0.5 * (wf * wf + wn * wn)) : 0.5 * (wf + wn);
    double du = (1.0 + xq64 * wo64) * dbeta / wbar;
    (void)o;
    return fabs(du) < a.thr;
}

// Eliminate one half-ray from its far end inward to the origin.
template <typename T, int LPT>
__device__ __forceinline__ void sweep(const FSArgs &a, int64_t o, int r, int line0, T Aq, T Bq, const T *Ibg,
                                      double xq64, double wo64, T (&P)[LPT], T (&Y)[LPT], T (&aa)[LPT])
{
    using LD = typename Prec<T>::LD;
    const LD *line = reinterpret_cast<const LD *>(a.line);
    const int64_t t = (int64_t)r * a.N + o;
    const int64_t s0 = a.ray_off[t];
    const int n = (int)(a.ray_off[t + 1] - s0);
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        P[l] = T(1);
        Y[l] = Ibg[l];
        aa[l] = T(0);
    }
    if (n == 0) return;
    const T thr = (T)a.thr;
    StepG<T> sf = get_step<T>(a, s0 + n - 1);
    T chi_f[LPT], S_f[LPT];
    load_line<LPT>(line + sf.idx * a.Mpad + line0, chi_f, S_f);
    WG<T> wf = get_w<T>(a, sf.idx);
    T z_f = Aq + Bq * sf.beta;
    T g_f = Prec<T>::gauss(z_f * wf.iw);
    for (int k = n; k >= 1; --k) {
        StepG<T> sn;
        if (k > 1) {
            sn = get_step<T>(a, s0 + k - 2);
        } else {
            sn.idx = o;
            sn.dx = T(0);
            sn.beta = T(0);
            sn.dbw = T(0);
        }
        T chi_n[LPT], S_n[LPT];
        load_line<LPT>(line + sn.idx * a.Mpad + line0, chi_n, S_n);
        WG<T> wn = get_w<T>(a, sn.idx);
        const T z_n = Aq + Bq * sn.beta;
        const T g_n = Prec<T>::gauss(z_n * wn.iw);
        // reduced Doppler shift across the segment, near minus far, in units
        // of the segment-averaged width
        const T du = -Bq * sf.dbw;
        bool trap = fabs(du) < thr;
        if (sizeof(T) == 4 && fabs(fabs(du) - thr) < T(2e-5) * thr)
            trap = trapezoid_fp64(a, r, o, sf.idx, sn.idx, xq64, wo64);
        T cf, cn;
        if (trap) {
            cf = T(0.5) * sf.dx * g_f;
            cn = T(0.5) * sf.dx * g_n;
        } else {
            const T iwbar = a.width_mode == 0 ? Prec<T>::rsqrt_(T(0.5) * (wf.w * wf.w + wn.w * wn.w))
                                              : T(2) / (wf.w + wn.w);
            const T ubf = z_f * iwbar, ubn = ubf + du;
            T E;
            if (ubf > T(0) && ubn > T(0))
                E = Prec<T>::erfc_(ubf) - Prec<T>::erfc_(ubn);
            else if (ubf < T(0) && ubn < T(0))
                E = Prec<T>::erfc_(-ubn) - Prec<T>::erfc_(-ubf);
            else
                E = Prec<T>::erf_(ubn) - Prec<T>::erf_(ubf);
            const T kk = sf.dx * T(kSqrtPi) * E * iwbar / (T(4) * du);
            cf = kk * wf.w;
            cn = kk * wn.w;
        }
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const T b = cf * chi_f[l] + cn * chi_n[l];
            const T h = T(0.5) * (aa[l] + b);
            const T H = h + P[l];
            const T q = Prec<T>::rcp(T(1) + b * H);
            P[l] = H * q;
            Y[l] = (S_f[l] * h + Y[l]) * q;
            aa[l] = b;
            chi_f[l] = chi_n[l];
            S_f[l] = S_n[l];
        }
        z_f = z_n;
        g_f = g_n;
        wf = wn;
        sf = sn;
    }
}

template <typename T, int LPT> __global__ void __launch_bounds__(256) k_fs(FSArgs a)
{
    using LD = typename Prec<T>::LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const int QG = a.Q * a.Gb;
    const int Mb = a.Gb * LPT;                       // lines covered by this block
    T *acc = reinterpret_cast<T *>(smem_raw);        // [4][LPT][bd]: J, J-comp, L, L-comp
    double *red = reinterpret_cast<double *>(acc + 4 * LPT * bd);   // [2][OPB][Mb][Q]

    const int lo_ = tid / QG, rem = tid - lo_ * QG, gl = rem / a.Q, q = rem - gl * a.Q;
    const int gg = blockIdx.y * a.Gb + gl;
    const int line0 = gg * LPT;
    const int64_t o = (int64_t)blockIdx.x * a.OPB + lo_;
    const bool active = lo_ < a.OPB && o < a.N && gg < a.Gtot;
    const int mline0 = blockIdx.y * Mb;              // first line of this block

    // background B_nu_q(T_bg) / U_line for this thread's bin and lines; it
    // depends on the origin through nu_q = nu (1 + x_q w_o)
    T Ibg[LPT];
    const double xq64 = active ? a.xq[q] : 0.0;
    const double wo64 = active ? a.w64[o] : 0.0;
    if (active) {
        const T f = T(1) + T(xq64) * T(wo64);
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int k = line0 + l;
            const double hk = a.line_tab[5 * a.Mpad + k], nbg = a.line_tab[4 * a.Mpad + k];
            Ibg[l] = (k < a.M && hk > 0.0) ? Prec<T>::bg(f, T(hk)) / T(nbg) : T(0);
        }
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            acc[(0 * LPT + l) * bd + tid] = T(0);
            acc[(1 * LPT + l) * bd + tid] = T(0);
            acc[(2 * LPT + l) * bd + tid] = T(0);
            acc[(3 * LPT + l) * bd + tid] = T(0);
        }
        const T x = T(xq64), wo = T(wo64);
        const T Aq = x * wo, Bq = T(1) + Aq;
        const T wqn = T(a.wq[q]);
        const LD *line = reinterpret_cast<const LD *>(a.line);
        T So[LPT], dummy[LPT];
        load_line<LPT>(line + o * a.Mpad + line0, dummy, So);
        for (int p = 0; p < a.P; ++p) {
            const int2 pr = a.pairs[p];
            T PL[LPT], YL[LPT], aL[LPT], PR[LPT], YR[LPT], aR[LPT];
            sweep<T, LPT>(a, o, pr.y, line0, Aq, Bq, Ibg, xq64, wo64, PL, YL, aL);
            sweep<T, LPT>(a, o, pr.x, line0, Aq, Bq, Ibg, xq64, wo64, PR, YR, aR);
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                const T h = T(0.5) * (aL[l] + aR[l]);
                const T inv = Prec<T>::rcp(h + PL[l] + PR[l]);
                const T u = (So[l] * h + YL[l] + YR[l]) * inv;
                const T Ls = h * inv;
                // compensated (Kahan) accumulation of w_q u and w_q Lambda*
                T *sJ = acc + (0 * LPT + l) * bd + tid, *cJ = acc + (1 * LPT + l) * bd + tid;
                T *sL = acc + (2 * LPT + l) * bd + tid, *cL = acc + (3 * LPT + l) * bd + tid;
                T y = wqn * u - *cJ, tt = *sJ + y;
                *cJ = (tt - *sJ) - y;
                *sJ = tt;
                y = wqn * Ls - *cL;
                tt = *sL + y;
                *cL = (tt - *sL) - y;
                *sL = tt;
            }
        }
        const int lb = gl * LPT;                     // line offset within the block
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            if (line0 + l < a.M) {
                red[((0 * a.OPB + lo_) * Mb + lb + l) * a.Q + q] =
                    (double)acc[(0 * LPT + l) * bd + tid] - (double)acc[(1 * LPT + l) * bd + tid];
                red[((1 * a.OPB + lo_) * Mb + lb + l) * a.Q + q] =
                    (double)acc[(2 * LPT + l) * bd + tid] - (double)acc[(3 * LPT + l) * bd + tid];
            }
        }
    }
    __syncthreads();
    const double wdir = 2.0 / a.R;
    for (int e = tid; e < a.OPB * Mb; e += bd) {
        const int lo2 = e / Mb, lb = e - lo2 * Mb;
        const int line = mline0 + lb;
        const int64_t o2 = (int64_t)blockIdx.x * a.OPB + lo2;
        if (o2 >= a.N || line >= a.M) continue;
        double sJ = 0.0, sL = 0.0;
        for (int qq = 0; qq < a.Q; ++qq) {
            sJ += red[((0 * a.OPB + lo2) * Mb + lb) * a.Q + qq];
            sL += red[((1 * a.OPB + lo2) * Mb + lb) * a.Q + qq];
        }
        a.J[o2 * a.M + line] = sJ * wdir * a.line_tab[6 * a.Mpad + line];
        a.Lst[o2 * a.M + line] = sL * wdir;
    }
}

template <typename T, int LPT> mgt_status launch_typed(mgt_model *m, cudaStream_t s)
{
    FSArgs a{};
    a.N = m->N;
    a.R = m->R;
    a.P = m->P;
    a.Q = m->Q;
    a.M = m->M;
    a.Mpad = m->Mpad;
    a.Gtot = (m->M + LPT - 1) / LPT;              // groups covering the real lines
    int gb = a.Gtot;
    while (gb > 1 && a.Q * gb > 256) --gb;
    a.Gb = gb;
    a.OPB = (a.Q * a.Gb >= 256) ? 1 : 256 / (a.Q * a.Gb);
    a.pairs = m->d_pairs;
    a.ray_off = m->d_ray_off;
    a.s32 = m->d_steps32;
    a.s64 = m->d_steps64;
    a.w32 = m->d_w32;
    a.w64 = m->d_w64;
    a.line = sizeof(T) == 4 ? (const void *)m->d_line32 : (const void *)m->d_line64;
    a.xq = m->d_xq;
    a.wq = m->d_wq;
    a.line_tab = m->d_line_tab;
    a.vel = m->d_vel;
    a.dirs = m->d_dirs;
    a.thr = m->opts.switch_threshold;
    a.width_mode = m->opts.width_mode;
    a.J = m->d_J;
    a.Lst = m->d_Lst;
    int threads = a.OPB * a.Q * a.Gb;
    int bd = ((threads + 31) / 32) * 32;
    if (bd > 1024) return set_error(MGT_ERR_ARG, "formal solve: too many bins x line groups per block");
    const int Mb = a.Gb * LPT;
    size_t smem = sizeof(T) * 4 * LPT * bd + sizeof(double) * 2 * a.OPB * Mb * a.Q;
    MGT_CUDA(cudaFuncSetAttribute(k_fs<T, LPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)ceil_div(m->N, a.OPB), (unsigned)ceil_div(a.Gtot, a.Gb));
    k_fs<T, LPT><<<grid, bd, smem, s>>>(a);
    MGT_LAUNCH_CHECK("k_fs");
    return MGT_OK;
}

}  // namespace

int fs_lines_per_thread(const mgt_model *m, mgt_precision p)
{
    if (p == MGT_FP64) return 4;
    if (m->opts.lines_per_thread == 4 || m->opts.lines_per_thread == 8) return m->opts.lines_per_thread;
    return m->M <= 4 ? 4 : 8;
}

mgt_status launch_formal_solve(mgt_model *m, mgt_precision p, cudaStream_t s)
{
    const int lpt = fs_lines_per_thread(m, p);
    if (m->Mpad % lpt != 0) return set_error(MGT_ERR_STATE, "line padding does not match the schedule");
    if (p == MGT_FP64) return launch_typed<double, 4>(m, s);
    return lpt == 4 ? launch_typed<float, 4>(m, s) : launch_typed<float, 8>(m, s);
}

}  // namespace mgt
