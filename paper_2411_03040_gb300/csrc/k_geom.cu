// Per-point kernels: line widths, LTE populations, line opacity / source
// function, and the ray walk through the neighbour graph.
#include <cub/cub.cuh>

#include "mgt_common.cuh"

namespace mgt {

// ---------------------------------------------------------------------------
// Relative line width w = dnu/nu = sqrt(2 k T / m + vturb^2) / c (Sec. 4.3,
// eq. line width); one value per point serves every line of the species.
// ---------------------------------------------------------------------------
__global__ void k_widths(int64_t N, const double *__restrict__ T, const double *__restrict__ vt2,
                         double two_k_over_m, double inv_c, double *__restrict__ w64,
                         float2 *__restrict__ w32)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= N) return;
    double w = sqrt(two_k_over_m * T[p] + vt2[p]) * inv_c;
    w64[p] = w;
    w32[p] = make_float2((float)w, (float)(1.0 / w));
}

mgt_status launch_widths(mgt_model *m, cudaStream_t s)
{
    k_widths<<<ceil_div(m->N, 256), 256, 0, s>>>(m->N, m->d_temp, m->d_vturb2, 2.0 * kKB / m->mol_mass,
                                                 1.0 / kC, m->d_w64, m->d_w32);
    MGT_LAUNCH_CHECK("k_widths");
    return MGT_OK;
}

// ---------------------------------------------------------------------------
// LTE: n_i = n_spec g_i exp(-(E_i - E_0)/kT) / sum_j g_j exp(-(E_j - E_0)/kT).
// ---------------------------------------------------------------------------
__global__ void k_lte(int64_t N, int L, const double *__restrict__ T, const double *__restrict__ nspec,
                      const double *__restrict__ level_tab, double *__restrict__ pops)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= N) return;
    const double *E = level_tab, *g = level_tab + L;
    double beta = 1.0 / (kKB * T[p]);
    double Z = 0.0;
    for (int i = 0; i < L; ++i) Z += g[i] * exp(-(E[i] - E[0]) * beta);
    double f = nspec[p] / Z;
    for (int i = 0; i < L; ++i) pops[p * L + i] = f * g[i] * exp(-(E[i] - E[0]) * beta);
}

mgt_status launch_lte(mgt_model *m, cudaStream_t s)
{
    k_lte<<<ceil_div(m->N, 128), 128, 0, s>>>(m->N, m->L, m->d_temp, m->d_nspec, m->d_level_tab, m->d_pops);
    MGT_LAUNCH_CHECK("k_lte");
    m->line_dirty = true;
    return MGT_OK;
}

// ---------------------------------------------------------------------------
// Line data per (point, line) from the populations.
//   net = n_l B_lu - n_u B_ul, floored at 1e-30 (n_l B_lu + n_u B_ul) (counted),
//   chi^{ij} = (h nu / 4 pi) net,  S^{ij} = n_u A_ul / net.
// Stored scaled for the solver:
//   chi~' = chi^{ij} / (nu w sqrt(pi)) * L_unit  -- opacity per length unit at
//           line centre, so that chi(nu) = chi~ exp(-u^2);
//   S'    = S^{ij} / U_line, U_line = (2 h nu^3/c^2) max(n_bg(nu), 1e-30)
//         = n_u B_ul / (net * nbgmax).
// Row layout (see row_stride32): chi~' of every line, then S' of every line,
// then w and 1/w of the point.  One thread per (point, line slot).
// ---------------------------------------------------------------------------
__global__ void k_line_data(int64_t N, int L, int M, int Mpad, const double *__restrict__ pops,
                            const double *__restrict__ w64, const double *__restrict__ line_tab,
                            const int32_t *__restrict__ line_ul, double Lunit,
                            float *__restrict__ out32, double *__restrict__ out64,
                            unsigned long long *__restrict__ n_floor)
{
    const int RS = row_stride32(Mpad), RS64 = row_stride64(Mpad);
    const int slots = Mpad + 2;                      // Mpad lines + {w, 1/w} + {0, 0}
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= N * slots) return;
    int64_t p = t / slots;
    int k = (int)(t - p * slots);
    double a0 = 0.0, a1 = 0.0;
    if (k < M) {
        int u = line_ul[k], l = line_ul[Mpad + k];
        double Bul = line_tab[2 * Mpad + k], Blu = line_tab[3 * Mpad + k];
        double nbgmax = line_tab[4 * Mpad + k];
        double nu_ = pops[p * L + u], nl_ = pops[p * L + l];
        double a = nl_ * Blu, b = nu_ * Bul;
        double net = a - b, floor_ = 1e-30 * (a + b);
        if (net < floor_) {
            net = floor_;
            atomicAdd(n_floor, 1ULL);
        }
        if (net > 0.0) {
            a0 = kH * net * Lunit / (4.0 * kPi * kSqrtPi * w64[p]);
            a1 = b / (net * nbgmax);
        }
    } else if (k == Mpad) {
        a0 = w64[p];
        a1 = 1.0 / a0;
    }
    float *r32 = out32 + p * RS;
    if (k < Mpad) {
        r32[k] = (float)a0;
        r32[Mpad + k] = (float)a1;
        if (out64) {
            out64[p * RS64 + k] = a0;
            out64[p * RS64 + Mpad + k] = a1;
        }
    } else if (k == Mpad) {
        r32[2 * Mpad] = (float)a0;
        r32[2 * Mpad + 1] = (float)a1;
        if (out64) {
            out64[p * RS64 + 2 * Mpad] = a0;
            out64[p * RS64 + 2 * Mpad + 1] = a1;
        }
    } else {
        r32[2 * Mpad + 2] = 0.0f;
        r32[2 * Mpad + 3] = 0.0f;
    }
}

mgt_status launch_line_data(mgt_model *m, cudaStream_t s)
{
    int64_t n = m->N * (m->Mpad + 2);
    k_line_data<<<ceil_div(n, 256), 256, 0, s>>>(m->N, m->L, m->M, m->Mpad, m->d_pops, m->d_w64, m->d_line_tab,
                                                m->d_line_ul, m->L_unit, m->d_line32, m->d_line64,
                                                m->d_count + 0);
    MGT_LAUNCH_CHECK("k_line_data");
    m->line_dirty = false;
    return MGT_OK;
}

// ---------------------------------------------------------------------------
// Ray walk (bit-exact FP64 predicates; no multiply-add fusion).
//
// From the current point c (start c = o) the candidates are the neighbours m
// of c with Z_m = (x_m - x_o).n > Z_c; the winner minimises the squared
// distance to the ray line |(x_m - x_o) - Z_m n|^2, ties to the smaller index.
// The walk ends on a boundary point (kept) or stalls without a candidate (a
// boundary origin without candidates just has an empty half-ray).
// ---------------------------------------------------------------------------
struct WalkArgs {
    int64_t N;
    int32_t R;
    const double *pos;
    const int32_t *off;
    const int32_t *nb;
    const double *nb_pos;     // [nnz][3] position of each neighbour entry (contiguous per point)
    const float *nb_hl;       // [nnz][6] the same positions split into float hi + lo parts
    const uint8_t *bnd;
    const double *dirs;
    const int32_t *order;     // walks of one direction are visited in this point order
    float pos_slack;          // bound on |x - (hi + lo)| over all coordinates
    unsigned long long *n_exact;   // steps decided by the FP64 predicates
};

__device__ __forceinline__ double dot3_exact(double ax, double ay, double az, double bx, double by, double bz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
}

// Next point of the walk from c in FP64, the defining arithmetic, or -1.
// Writes the winner's Z and its neighbour-entry index.
__device__ __noinline__ int64_t walk_next_exact(const WalkArgs &a, int64_t c, double xo, double yo, double zo, double n0,
                                                double n1, double n2, double Zc, double *Znext)
{
    int64_t best = -1;
    double bestd = 0.0, bestZ = 0.0;
    const int32_t k1 = a.off[c + 1];
    for (int32_t k = a.off[c]; k < k1; ++k) {
        int64_t mm = a.nb[k];
        double dx = __dsub_rn(a.nb_pos[3 * (int64_t)k], xo);
        double dy = __dsub_rn(a.nb_pos[3 * (int64_t)k + 1], yo);
        double dz = __dsub_rn(a.nb_pos[3 * (int64_t)k + 2], zo);
        double Z = dot3_exact(dx, dy, dz, n0, n1, n2);
        if (!(Z > Zc)) continue;
        double px = __dsub_rn(dx, __dmul_rn(Z, n0));
        double py = __dsub_rn(dy, __dmul_rn(Z, n1));
        double pz = __dsub_rn(dz, __dmul_rn(Z, n2));
        double d2 = dot3_exact(px, py, pz, px, py, pz);
        if (best < 0 || d2 < bestd || (d2 == bestd && mm < best)) {
            best = mm;
            bestd = d2;
            bestZ = Z;
        }
    }
    *Znext = bestZ;
    return best;
}

// Per-walk constants of the filtered step.
struct WalkFrame {
    double xo, yo, zo, n0, n1, n2;     // FP64 origin and direction
    float ohx, ohy, ohz, olx, oly, olz; // origin split into hi + lo floats
    float f0, f1, f2;                  // direction in FP32
};

// Next point of the walk, decided with FP32 arithmetic when error bounds
// prove that the FP64 predicates give the same answer, else by
// walk_next_exact.  Bounds (generous multiples of the rounding analysis):
//   offsets   |d32 - d64| <= ed = 2e-6 (|d32|_max + slack)
//   projection |Z32 - Z64| <= eZ = 2e-6 |d32|_1 + 2 ed, plus 1e-7 |Z_c| for Z_c
//   perpendicular components  ep = ed + eZ + 2e-7 (|p32|_max + |Z32|)
//   squared distance |d2_32 - d2_64| <= 4 |p32| ep + 4 ep^2 + 1e-6 d2_32.
// A neighbour is a candidate only if Z32 - eZ clears Z_c; not one only if
// Z32 + eZ stays below it; otherwise the step is undecided.  The FP32 winner
// is accepted only if its upper d2 bound is below every other candidate's
// lower bound (so ties always go to FP64).
__device__ __forceinline__ int64_t walk_next(const WalkArgs &a, const WalkFrame &f, int64_t c, double Zc, double *Znext)
{
    const float Zcf = (float)Zc;
    const float eZc = 1e-7f * fabsf(Zcf) + 1e-30f;
    int32_t kbest = -1;
    float d2best = 0.0f, Ubest = 0.0f, Lbest = 0.0f, minLother = 3.0e38f;
    bool undecided = false;
    const int32_t k0 = a.off[c], k1 = a.off[c + 1];
    for (int32_t k = k0; k < k1; ++k) {
        const float *hl = a.nb_hl + 6 * (int64_t)k;
        const float dx = (hl[0] - f.ohx) + (hl[3] - f.olx);
        const float dy = (hl[1] - f.ohy) + (hl[4] - f.oly);
        const float dz = (hl[2] - f.ohz) + (hl[5] - f.olz);
        const float adx = fabsf(dx), ady = fabsf(dy), adz = fabsf(dz);
        const float ed = 2e-6f * (fmaxf(adx, fmaxf(ady, adz)) + a.pos_slack);
        const float Z = fmaf(dz, f.f2, fmaf(dy, f.f1, dx * f.f0));
        const float eZ = 2e-6f * (adx + ady + adz) + 2.0f * ed + eZc;
        if (Z - eZ > Zcf) {
            const float px = fmaf(-Z, f.f0, dx), py = fmaf(-Z, f.f1, dy), pz = fmaf(-Z, f.f2, dz);
            const float d2 = fmaf(pz, pz, fmaf(py, py, px * px));
            const float ep = ed + eZ + 2e-7f * (fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))) + fabsf(Z));
            const float e2 = 4.0f * sqrtf(d2) * ep + 4.0f * ep * ep + 1e-6f * d2;
            const float U = d2 + e2, Lo = d2 - e2;
            if (kbest < 0 || d2 < d2best) {
                if (kbest >= 0) minLother = fminf(minLother, Lbest);
                kbest = k;
                d2best = d2;
                Ubest = U;
                Lbest = Lo;
            } else {
                minLother = fminf(minLother, Lo);
            }
        } else if (!(Z + eZ < Zcf)) {
            undecided = true;
            break;
        }
    }
    if (undecided || (kbest >= 0 && !(Ubest < minLother))) {
        atomicAdd(a.n_exact, 1ULL);
        return walk_next_exact(a, c, f.xo, f.yo, f.zo, f.n0, f.n1, f.n2, Zc, Znext);
    }
    if (kbest < 0) {
        *Znext = 0.0;
        return -1;
    }
    const double *q = a.nb_pos + 3 * (int64_t)kbest;
    *Znext = dot3_exact(__dsub_rn(q[0], f.xo), __dsub_rn(q[1], f.yo), __dsub_rn(q[2], f.zo), f.n0, f.n1, f.n2);
    return a.nb[kbest];
}

__device__ __forceinline__ WalkFrame make_frame(const WalkArgs &a, int64_t o, int r)
{
    WalkFrame f;
    f.n0 = a.dirs[3 * r];
    f.n1 = a.dirs[3 * r + 1];
    f.n2 = a.dirs[3 * r + 2];
    f.xo = a.pos[3 * o];
    f.yo = a.pos[3 * o + 1];
    f.zo = a.pos[3 * o + 2];
    f.ohx = (float)f.xo;
    f.ohy = (float)f.yo;
    f.ohz = (float)f.zo;
    f.olx = (float)(f.xo - (double)f.ohx);
    f.oly = (float)(f.yo - (double)f.ohy);
    f.olz = (float)(f.zo - (double)f.ohz);
    f.f0 = (float)f.n0;
    f.f1 = (float)f.n1;
    f.f2 = (float)f.n2;
    return f;
}

// Pass 1: half-ray length and stall flag of every (direction, origin).
__global__ void k_trace_count(WalkArgs a, int64_t *__restrict__ len, unsigned long long *__restrict__ n_stall)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)a.R * a.N) return;
    int r = (int)(t / a.N);
    int64_t o = a.order[t - (int64_t)r * a.N];
    const WalkFrame f = make_frame(a, o, r);
    int64_t c = o, n = 0;
    double Zc = 0.0;
    for (;;) {
        double Zn;
        int64_t nx = walk_next(a, f, c, Zc, &Zn);
        if (nx < 0) {
            if (!(c == o && a.bnd[o])) atomicAdd(n_stall, 1ULL);
            break;
        }
        ++n;
        c = nx;
        Zc = Zn;
        if (a.bnd[nx] || n >= a.N) break;   // Z strictly increases: at most N-1 steps
    }
    len[(int64_t)r * a.N + o] = n;
}

// Pass 2: the same walk, writing the point list and its single-precision
// geometry (see Step32).  `off` is the exclusive prefix of the lengths.
__global__ void k_trace_fill(WalkArgs a, const int64_t *__restrict__ off, const double *__restrict__ vel,
                             const double *__restrict__ w64, double inv_Lunit, int width_mode,
                             Step32 *__restrict__ steps, int *__restrict__ err)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)a.R * a.N) return;
    int r = (int)(t / a.N);
    int64_t o = a.order[t - (int64_t)r * a.N];
    const int64_t w = (int64_t)r * a.N + o;
    const WalkFrame f = make_frame(a, o, r);
    const double vox = vel[3 * o], voy = vel[3 * o + 1], voz = vel[3 * o + 2];
    const int64_t base = off[w], cap = off[w + 1] - base;
    int64_t c = o, n = 0;
    double Zc = 0.0;
    double px = f.xo, py = f.yo, pz = f.zo;      // previous point (c_{k-1})
    double pvx = vox, pvy = voy, pvz = voz, pw = w64[o];
    for (;;) {
        double Zn;
        int64_t nx = walk_next(a, f, c, Zc, &Zn);
        if (nx < 0) break;
        if (n >= cap) {                          // cannot happen for a deterministic walk
            atomicCAS(err, 0, (int)kDevBounds);
            return;
        }
        double qx = a.pos[3 * nx], qy = a.pos[3 * nx + 1], qz = a.pos[3 * nx + 2];
        double vx = vel[3 * nx], vy = vel[3 * nx + 1], vz = vel[3 * nx + 2], wq = w64[nx];
        double ex = qx - px, ey = qy - py, ez = qz - pz;
        double dx = sqrt(ex * ex + ey * ey + ez * ez) * inv_Lunit;
        double beta = (f.n0 * (vx - vox) + f.n1 * (vy - voy) + f.n2 * (vz - voz)) / kC;
        double dbeta = (f.n0 * (vx - pvx) + f.n1 * (vy - pvy) + f.n2 * (vz - pvz)) / kC;
        double wbar = width_mode == 0 ? sqrt(0.5 * (wq * wq + pw * pw)) : 0.5 * (wq + pw);
        steps[base + n] = make_int4((int)nx, __float_as_int((float)dx), __float_as_int((float)beta),
                                    __float_as_int((float)(dbeta / wbar)));
        ++n;
        c = nx;
        Zc = Zn;
        px = qx; py = qy; pz = qz;
        pvx = vx; pvy = vy; pvz = vz; pw = wq;
        if (a.bnd[nx] || n >= a.N) break;
    }
    if (n != cap) atomicCAS(err, 0, (int)kDevBounds);
}

// Double-precision step geometry for the FP64 formal solution, from the
// traced point lists (one thread per half-ray).
__global__ void k_steps64(int64_t N, int32_t R, const int64_t *__restrict__ off, const Step32 *__restrict__ s32,
                          const double *__restrict__ pos, const double *__restrict__ vel,
                          const double *__restrict__ w64, const double *__restrict__ dirs, double inv_Lunit,
                          int width_mode, Step64 *__restrict__ s64)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * N) return;
    int r = (int)(t / N);
    int64_t o = t - (int64_t)r * N;
    double n0 = dirs[3 * r], n1 = dirs[3 * r + 1], n2 = dirs[3 * r + 2];
    const double vox = vel[3 * o], voy = vel[3 * o + 1], voz = vel[3 * o + 2];
    double px = pos[3 * o], py = pos[3 * o + 1], pz = pos[3 * o + 2];
    double pvx = vox, pvy = voy, pvz = voz, pw = w64[o];
    for (int64_t s = off[t]; s < off[t + 1]; ++s) {
        int64_t c = s32[s].x;
        double qx = pos[3 * c], qy = pos[3 * c + 1], qz = pos[3 * c + 2];
        double vx = vel[3 * c], vy = vel[3 * c + 1], vz = vel[3 * c + 2], wq = w64[c];
        double ex = qx - px, ey = qy - py, ez = qz - pz;
        Step64 st;
        st.dx = sqrt(ex * ex + ey * ey + ez * ez) * inv_Lunit;
        st.beta = (n0 * (vx - vox) + n1 * (vy - voy) + n2 * (vz - voz)) / kC;
        double dbeta = (n0 * (vx - pvx) + n1 * (vy - pvy) + n2 * (vz - pvz)) / kC;
        double wbar = width_mode == 0 ? sqrt(0.5 * (wq * wq + pw * pw)) : 0.5 * (wq + pw);
        st.dbw = dbeta / wbar;
        st.pad = 0.0;
        s64[s] = st;
        px = qx; py = qy; pz = qz;
        pvx = vx; pvy = vy; pvz = vz; pw = wq;
    }
}

mgt_status trace_all(mgt_model *m, cudaStream_t s)
{
    const int64_t W = (int64_t)m->R * m->N;
    WalkArgs a{m->N, m->R, m->d_pos, m->d_nbr_off, m->d_nbrs, m->d_nbr_pos, m->d_nbr_hl, m->d_bnd, m->d_dirs,
               m->d_order, m->pos_slack, m->d_count + 2};
    if (!m->d_ray_off) MGT_CUDA(cudaMalloc(&m->d_ray_off, sizeof(int64_t) * (W + 1)));
    int64_t *d_len = nullptr;
    MGT_CUDA(cudaMallocAsync(&d_len, sizeof(int64_t) * (W + 1), s));
    MGT_CUDA(cudaMemsetAsync(m->d_count + 1, 0, 2 * sizeof(unsigned long long), s));
    k_trace_count<<<ceil_div(W, 128), 128, 0, s>>>(a, d_len, m->d_count + 1);
    MGT_LAUNCH_CHECK("k_trace_count");
    MGT_CUDA(cudaMemsetAsync(d_len + W, 0, sizeof(int64_t), s));
    size_t tmp_bytes = 0;
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_len, m->d_ray_off, W + 1, s));
    void *tmp = nullptr;
    MGT_CUDA(cudaMallocAsync(&tmp, tmp_bytes, s));
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, d_len, m->d_ray_off, W + 1, s));
    // longest half-ray
    int64_t *d_max = nullptr;
    MGT_CUDA(cudaMallocAsync(&d_max, sizeof(int64_t), s));
    size_t tmp2 = 0;
    MGT_CUDA(cub::DeviceReduce::Max(nullptr, tmp2, d_len, d_max, W, s));
    void *tmpb = nullptr;
    MGT_CUDA(cudaMallocAsync(&tmpb, tmp2, s));
    MGT_CUDA(cub::DeviceReduce::Max(tmpb, tmp2, d_len, d_max, W, s));
    int64_t total = 0, mx = 0;
    unsigned long long stalls = 0, exact_steps = 0;
    MGT_CUDA(cudaMemcpyAsync(&total, m->d_ray_off + W, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&mx, d_max, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&stalls, m->d_count + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&exact_steps, m->d_count + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    MGT_CUDA(cudaFreeAsync(tmp, s));
    MGT_CUDA(cudaFreeAsync(tmpb, s));
    MGT_CUDA(cudaFreeAsync(d_max, s));
    MGT_CUDA(cudaFreeAsync(d_len, s));
    if (m->d_steps32 && total > m->total_steps) {
        MGT_CUDA(cudaFree(m->d_steps32));
        m->d_steps32 = nullptr;
    }
    if (m->d_steps64) {
        MGT_CUDA(cudaFree(m->d_steps64));
        m->d_steps64 = nullptr;
        m->steps64_width_mode = -1;
    }
    if (!m->d_steps32 && total > 0) {
        cudaError_t e = cudaMalloc(&m->d_steps32, sizeof(Step32) * total);
        if (e != cudaSuccess) return set_error(MGT_ERR_OOM, "cannot allocate the ray buffer");
    }
    m->total_steps = total;
    m->max_half = (int32_t)mx;
    m->n_stalls = (int64_t)stalls;
    m->n_exact_steps = (int64_t)exact_steps;   // pass 1 only
    if (total > 0) {
        k_trace_fill<<<ceil_div(W, 128), 128, 0, s>>>(a, m->d_ray_off, m->d_vel, m->d_w64, 1.0 / m->L_unit,
                                                      m->opts.width_mode, m->d_steps32, m->d_err);
        MGT_LAUNCH_CHECK("k_trace_fill");
    }
    m->steps_width_mode = m->opts.width_mode;
    m->traced = true;
    return MGT_OK;
}

mgt_status build_steps64(mgt_model *m, cudaStream_t s)
{
    if (m->total_steps == 0) return MGT_OK;
    if (!m->d_steps64) {
        cudaError_t e = cudaMalloc(&m->d_steps64, sizeof(Step64) * m->total_steps);
        if (e != cudaSuccess) return set_error(MGT_ERR_OOM, "cannot allocate the FP64 ray geometry");
    }
    const int64_t W = (int64_t)m->R * m->N;
    k_steps64<<<ceil_div(W, 128), 128, 0, s>>>(m->N, m->R, m->d_ray_off, m->d_steps32, m->d_pos, m->d_vel,
                                               m->d_w64, m->d_dirs, 1.0 / m->L_unit, m->opts.width_mode,
                                               m->d_steps64);
    MGT_LAUNCH_CHECK("k_steps64");
    m->steps64_width_mode = m->opts.width_mode;
    return MGT_OK;
}

}  // namespace mgt
