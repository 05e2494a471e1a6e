// Per-point kernels: line widths, LTE populations, line opacity / source
// function, and the ray walk through the neighbour graph.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

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
// Walk tables built on the device at model set-up (from the uploaded
// positions, velocities, neighbour lists and boundary mask):
//  * positions times pos_scale and v/c, each split into float hi + lo;
//  * the FP64 position of every neighbour entry;
//  * the packed neighbour rows (see WalkEntry in mgt_common.cuh);
//  * the Morton (Z-curve) visiting order of the points: 21 bits per axis of
//    the point's place in the bounding box, sorted with ties to the lower
//    index.
// The arithmetic is the host definition's (IEEE operations, no contraction),
// so the tables do not depend on where they are built.
// ---------------------------------------------------------------------------
__global__ void k_split_hl(int64_t N, const double *__restrict__ pos, const double *__restrict__ vel, double scale,
                           double inv_c, float *__restrict__ pos_hl, float *__restrict__ vel_hl)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    const int64_t i = t / 3;
    const int c = (int)(t - 3 * i);
    const double xs = __dmul_rn(pos[t], scale);
    const float hi = __double2float_rn(xs);
    pos_hl[6 * i + c] = hi;
    pos_hl[6 * i + 3 + c] = __double2float_rn(__dsub_rn(xs, (double)hi));
    const double vb = __dmul_rn(vel[t], inv_c);
    const float vh = __double2float_rn(vb);
    vel_hl[6 * i + c] = vh;
    vel_hl[6 * i + 3 + c] = __double2float_rn(__dsub_rn(vb, (double)vh));
}

__global__ void k_nbr_pos(int64_t nnz, const int32_t *__restrict__ nb, const double *__restrict__ pos,
                          double *__restrict__ nb_pos)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * nnz) return;
    const int64_t k = t / 3;
    nb_pos[t] = pos[3 * (int64_t)nb[k] + (t - 3 * k)];
}

__device__ __forceinline__ void put_entry(float4 *ent, int64_t e, const float *phl, int64_t mpt, uint32_t word,
                                          int32_t noff)
{
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (mpt >= 0)
        for (int c = 0; c < 6; ++c) v[c] = phl[6 * mpt + c];
    ent[2 * e] = make_float4(v[0], v[1], v[2], v[3]);
    ent[2 * e + 1] = make_float4(v[4], v[5], __uint_as_float(word), __int_as_float(noff));
}

// One thread per point (rows of ~15 entries), then the 16 pad entries.
__global__ void k_pack_rows(int64_t N, int64_t ne, const int32_t *__restrict__ off, const int32_t *__restrict__ nb,
                            const uint8_t *__restrict__ bnd, const float *__restrict__ phl,
                            const int32_t *__restrict__ eoff, float4 *__restrict__ ent)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N + 16) return;
    if (i >= N) {
        put_entry(ent, ne + (i - N), phl, -1, kEntEmpty | kEntLast, 0);
        return;
    }
    const int32_t k0 = off[i], k1 = off[i + 1];
    const int64_t e0 = eoff[i];
    if (k1 == k0) {
        put_entry(ent, e0, phl, -1, kEntEmpty | kEntLast, 0);
        return;
    }
    for (int32_t k = k0; k < k1; ++k) {
        const int32_t mpt = nb[k];
        uint32_t word = (uint32_t)mpt;
        if (k == k1 - 1) word |= kEntLast;
        if (bnd[mpt]) word |= kEntBnd;
        put_entry(ent, e0 + (k - k0), phl, mpt, word, eoff[mpt]);
    }
}

__device__ __forceinline__ uint64_t morton_spread(uint64_t v)
{
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

__global__ void k_morton_keys(int64_t N, const double *__restrict__ pos, double lo0, double lo1, double lo2,
                              double sp0, double sp1, double sp2, uint64_t *__restrict__ key,
                              int32_t *__restrict__ idx)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double lo[3] = {lo0, lo1, lo2}, sp[3] = {sp0, sp1, sp2};
    uint64_t k = 0;
    for (int d = 0; d < 3; ++d) {
        const double x = __dmul_rn(__ddiv_rn(__dsub_rn(pos[3 * i + d], lo[d]), sp[d]), 2097151.0);
        const uint64_t q = (uint64_t)fmin(2097151.0, fmax(0.0, x));
        k |= morton_spread(q) << d;
    }
    key[i] = k;
    idx[i] = (int32_t)i;
}

// Longest graph edge at each point, over the edges of its own neighbour list
// and those that name it (so that every step of a walk, from a point to one of
// its neighbours, is no longer than dxmax at either end): FP64 distance in
// length units, rounded up to FP32 with a margin over the walk's own FP32 step
// lengths.  Non-negative floats order like their bit patterns.
__global__ void k_edge_max(int64_t N, const int32_t *__restrict__ off, const int32_t *__restrict__ nbrs,
                           const double *__restrict__ pos, double inv_Lunit, float *__restrict__ dxmax)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= N) return;
    int *dm = reinterpret_cast<int *>(dxmax);
    float best = 0.0f;
    for (int32_t k = off[p]; k < off[p + 1]; ++k) {
        const int64_t q = nbrs[k];
        const double dx = pos[3 * q] - pos[3 * p], dy = pos[3 * q + 1] - pos[3 * p + 1],
                     dz = pos[3 * q + 2] - pos[3 * p + 2];
        const float d = __double2float_ru(sqrt(dx * dx + dy * dy + dz * dz) * inv_Lunit * (1.0 + 1e-5));
        best = fmaxf(best, d);
        atomicMax(dm + q, __float_as_int(d));
    }
    atomicMax(dm + p, __float_as_int(best));
}

mgt_status build_walk_tables(mgt_model *m, const double lo[3], const double hi[3], cudaStream_t s)
{
    const int64_t N = m->N;
    MGT_CUDA(cudaMemsetAsync(m->d_dxmax, 0, sizeof(float) * N, s));
    k_edge_max<<<ceil_div(N, 256), 256, 0, s>>>(N, m->d_nbr_off, m->d_nbrs, m->d_pos, 1.0 / m->L_unit, m->d_dxmax);
    MGT_LAUNCH_CHECK("k_edge_max");
    k_split_hl<<<ceil_div(3 * N, 256), 256, 0, s>>>(N, m->d_pos, m->d_vel, m->pos_scale, 1.0 / kC, m->d_pos_hl,
                                                    m->d_vel_hl);
    MGT_LAUNCH_CHECK("k_split_hl");
    if (m->nnz > 0) {
        k_nbr_pos<<<ceil_div(3 * m->nnz, 256), 256, 0, s>>>(m->nnz, m->d_nbrs, m->d_pos, m->d_nbr_pos);
        MGT_LAUNCH_CHECK("k_nbr_pos");
    }
    k_pack_rows<<<ceil_div(N + 16, 128), 128, 0, s>>>(N, m->n_ent - 16, m->d_nbr_off, m->d_nbrs, m->d_bnd,
                                                      m->d_pos_hl, m->d_ent_off, m->d_ent);
    MGT_LAUNCH_CHECK("k_pack_rows");
    // Morton order: keys, then a stable radix sort of (key, index)
    uint64_t *keys = nullptr;
    int32_t *idx = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    mgt_status st = MGT_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        if (st == MGT_OK) st = cuda_status(e, what);
    };
    cudaError_t e = cudaMallocAsync(&keys, sizeof(uint64_t) * 2 * N, s);
    if (e != cudaSuccess) fail(e, "cudaMallocAsync");
    if (st == MGT_OK && (e = cudaMallocAsync(&idx, sizeof(int32_t) * N, s)) != cudaSuccess) fail(e, "cudaMallocAsync");
    double sp[3];
    for (int d = 0; d < 3; ++d) sp[d] = hi[d] > lo[d] ? hi[d] - lo[d] : 1.0;
    if (st == MGT_OK) {
        k_morton_keys<<<ceil_div(N, 256), 256, 0, s>>>(N, m->d_pos, lo[0], lo[1], lo[2], sp[0], sp[1], sp[2], keys,
                                                      idx);
        e = cudaGetLastError();
        if (e != cudaSuccess) fail(e, "k_morton_keys");
        else note_launch();
    }
    if (st == MGT_OK &&
        (e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys + N, idx, m->d_order, (int)N, 0, 64,
                                             s)) != cudaSuccess)
        fail(e, "cub::DeviceRadixSort::SortPairs");
    if (st == MGT_OK && (e = cudaMallocAsync(&tmp, tmp_bytes, s)) != cudaSuccess) fail(e, "cudaMallocAsync");
    if (st == MGT_OK &&
        (e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys + N, idx, m->d_order, (int)N, 0, 64, s)) !=
            cudaSuccess)
        fail(e, "cub::DeviceRadixSort::SortPairs");
    if (tmp) cudaFreeAsync(tmp, s);
    if (idx) cudaFreeAsync(idx, s);
    if (keys) cudaFreeAsync(keys, s);
    return st;
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
//   S'    = S^{ij} / U_line, U_line = (2 h nu^3/c^2) max(n_bg(nu), 1e-15)
//         = n_u B_ul / (net * nbgmax).
// Row layout (see row_stride32): chi~' of every line, then S' of every line,
// then w and 1/w of the point, then (FP32 rows only) the range figure
// G = max(chi~max dxmax / 2^8, S'max / 2^80) of the formal solution's two-row
// elimination (chi~max, S'max the largest over the point's lines, dxmax its
// longest graph edge) and a zero.
// One warp per point; lane j takes line slots j, j + 32, ...
// ---------------------------------------------------------------------------
struct LDArgs {
    int64_t N;
    int L, M, Mpad;
    const double *pops, *w64, *line_tab;
    const int32_t *line_ul;
    const float *dxmax;
    double Lunit;
    float *out32;
    double *out64;
    unsigned long long *n_floor;
    int *range_bad;           // set when a point's range figure exceeds 1 (zeroed before the launch)
};

__device__ __forceinline__ void line_data_point(const LDArgs &d, int64_t p, int lane)
{
    if (p >= d.N) return;                            // whole warp: p is warp-uniform
    const int Mpad = d.Mpad, RS = row_stride32(Mpad), RS64 = row_stride64(Mpad);
    const double *__restrict__ line_tab = d.line_tab;
    const int32_t *__restrict__ line_ul = d.line_ul;
    float *__restrict__ r32 = d.out32 + p * RS;
    double *__restrict__ r64 = d.out64 ? d.out64 + p * RS64 : nullptr;
    float chi_max = 0.0f, S_max = 0.0f;
    // h L_unit / (4 pi sqrt(pi) w): one FP64 division per point (lane 0), not per line
    double cw = 0.0;
    if (lane == 0) cw = kH * d.Lunit / (4.0 * kPi * kSqrtPi * d.w64[p]);
    cw = __shfl_sync(0xffffffffu, cw, 0);
    for (int k = lane; k < Mpad; k += 32) {
        double a0 = 0.0, a1 = 0.0;
        if (k < d.M) {
            const int u = line_ul[k], l = line_ul[Mpad + k];
            const double Bul = line_tab[2 * Mpad + k], Blu = line_tab[3 * Mpad + k];
            const double nbgmax = line_tab[4 * Mpad + k];
            const double nu_ = d.pops[p * d.L + u], nl_ = d.pops[p * d.L + l];
            const double a = nl_ * Blu, b = nu_ * Bul;
            double net = a - b;
            const double floor_ = 1e-30 * (a + b);
            if (net < floor_) {
                net = floor_;
                atomicAdd(d.n_floor, 1ULL);
            }
            if (net > 0.0) {
                a0 = net * cw;
                a1 = b / (net * nbgmax);
            }
        }
        const float f0 = (float)a0, f1 = (float)a1;
        r32[k] = f0;
        r32[Mpad + k] = f1;
        // !(x <= m) also carries a NaN into the bound, which then disables the
        // fast elimination for every step through this point
        chi_max = !(f0 <= chi_max) ? f0 : chi_max;
        S_max = !(f1 <= S_max) ? f1 : S_max;
        if (r64) {
            r64[k] = a0;
            r64[Mpad + k] = a1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float c = __shfl_xor_sync(0xffffffffu, chi_max, o), t = __shfl_xor_sync(0xffffffffu, S_max, o);
        chi_max = !(c <= chi_max) ? c : chi_max;
        S_max = !(t <= S_max) ? t : S_max;
    }
    if (lane == 0) {
        const double w = d.w64[p];
        r32[2 * Mpad] = (float)w;
        r32[2 * Mpad + 1] = (float)(1.0 / w);
        // range figure of the formal solution's two-row elimination: at most 1
        // when every step through the point has half depths <= kTwoRowDepth and
        // sources <= kTwoRowSource; NaN and infinity give a figure above 1
        // (a width above 1% of c, where no real line is, would also let the
        // background of the far bins outgrow the range: it sets the flag too)
        const float G = fmaxf(chi_max * d.dxmax[p] / kTwoRowDepth, S_max / kTwoRowSource);
        const bool inside = chi_max == chi_max && S_max == S_max && G <= 1.0f && w < 0.01;
        r32[2 * Mpad + 2] = inside ? G : 2.0f;
        r32[2 * Mpad + 3] = 0.0f;
        if (!inside) atomicOr(d.range_bad, 1);
        if (r64) {
            r64[2 * Mpad] = w;
            r64[2 * Mpad + 1] = 1.0 / w;
        }
    }
}

constexpr int kLDThreads = 256, kLDPointsPerBlock = kLDThreads / 32;

__global__ void __launch_bounds__(kLDThreads) k_line_data(LDArgs d)
{
    line_data_point(d, (int64_t)blockIdx.x * kLDPointsPerBlock + (threadIdx.x >> 5), threadIdx.x & 31);
}

// Many models in one launch: blk_end[i] is one past the last CTA of model i.
__global__ void __launch_bounds__(kLDThreads) k_line_data_batch(const LDArgs *__restrict__ args,
                                                                const int64_t *__restrict__ blk_end, int n_models)
{
    __shared__ LDArgs sd;
    __shared__ int64_t s_first;
    if (threadIdx.x == 0) {
        const int64_t b = blockIdx.x;
        int lo = 0, hi = n_models - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (blk_end[mid] > b) hi = mid; else lo = mid + 1;
        }
        sd = args[lo];
        s_first = lo > 0 ? blk_end[lo - 1] : 0;
    }
    __syncthreads();
    line_data_point(sd, ((int64_t)blockIdx.x - s_first) * kLDPointsPerBlock + (threadIdx.x >> 5), threadIdx.x & 31);
}

static LDArgs fill_ld_args(const mgt_model *m)
{
    return LDArgs{m->N, m->L, m->M, m->Mpad, m->d_pops, m->d_w64, m->d_line_tab, m->d_line_ul, m->d_dxmax,
                  m->L_unit, m->d_line32, m->d_line64, m->d_count + 0, m->d_range_bad};
}

mgt_status launch_line_data(mgt_model *m, cudaStream_t s)
{
    MGT_CUDA(cudaMemsetAsync(m->d_range_bad, 0, sizeof(int), s));
    {
        // populations and w in; the FP32 row (and the FP64 row if kept) out
        const double ld_bytes = (double)m->N * (8.0 * m->L + 8.0 + 4.0 * row_stride32(m->Mpad) +
                                                 (m->d_line64 ? 8.0 * row_stride64(m->Mpad) : 0.0));
        MGT_KTIMER_BYTES("k_line_data", s, ld_bytes);
        k_line_data<<<ceil_div(m->N, (int64_t)kLDPointsPerBlock), kLDThreads, 0, s>>>(fill_ld_args(m));
    }
    MGT_LAUNCH_CHECK("k_line_data");
    m->line_dirty = false;
    return MGT_OK;
}

size_t ld_args_bytes() { return sizeof(LDArgs); }

mgt_status ld_batch_args(const mgt_model *m, void *args, int64_t *blocks)
{
    const LDArgs a = fill_ld_args(m);
    std::memcpy(args, &a, sizeof a);
    *blocks = ceil_div(m->N, (int64_t)kLDPointsPerBlock);
    return MGT_OK;
}

// Zero every model's range flag before the batched line data set them.
__global__ void k_reset_range(const LDArgs *__restrict__ args, int n_models)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_models) *args[i].range_bad = 0;
}

mgt_status ld_batch_launch(const void *d_args, const int64_t *d_blk_end, int n_models, int64_t n_blocks,
                           cudaStream_t s)
{
    k_reset_range<<<ceil_div(n_models, 256), 256, 0, s>>>(static_cast<const LDArgs *>(d_args), n_models);
    MGT_LAUNCH_CHECK("k_reset_range");
    k_line_data_batch<<<(unsigned)n_blocks, kLDThreads, 0, s>>>(static_cast<const LDArgs *>(d_args), d_blk_end, n_models);
    MGT_LAUNCH_CHECK("k_line_data_batch");
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
    double pos_scale;         // power of two near 1 / (largest coordinate): exact scaling
    const uint8_t *bnd;
    const double *dirs;
    const float4 *ent;        // packed neighbour entries, two float4 each (WalkEntry layout)
    const int32_t *ent_off;   // [N] first packed entry of each point's row
    const float *pos_hl;      // [N][6] positions times pos_scale, split into float hi + lo
    const float4 *dirs32;     // [R] directions in FP32
    const int32_t *order;     // walks of one direction are visited in this point order
    float pos_slack;          // bound on |x - (hi + lo)| over all coordinates
    unsigned long long *n_exact;   // steps decided by the FP64 predicates
    int32_t max_row_chunks;   // bound on the 16-entry chunks of one row scan (packed entries / 16 + 2)
    int64_t n_ent;            // packed entries (index bound)
    const int32_t *dir_map;   // walk direction r -> model direction (NULL: the same); R counts walk directions
};

__device__ __forceinline__ uint64_t walk_clock_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First device error wins; err[1..3] say where (site) and which walk / step.
__device__ __forceinline__ void walk_give_up(int *err, int site, int64_t wg, int64_t n)
{
    if (atomicCAS(err, 0, (int)kDevTimeout) == 0) {
        err[1] = site;
        err[2] = (int)wg;
        err[3] = (int)n;
    }
}

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

// Per-walk constants, all FP32 (GB300's FP64 pipe is far too narrow for
// per-walk or per-step FP64 work; the FP64 values are loaded only on the rare
// steps the FP32 filter cannot settle).
struct WalkFrame {
    float ohx, ohy, ohz, olx, oly, olz; // origin (scaled) split into hi + lo floats
    float f0, f1, f2;                  // direction in FP32
};

__device__ __forceinline__ WalkFrame make_frame(const WalkArgs &a, int64_t o, int r)
{
    WalkFrame f;
    const float *p = a.pos_hl + 6 * o;
    f.ohx = p[0];
    f.ohy = p[1];
    f.ohz = p[2];
    f.olx = p[3];
    f.oly = p[4];
    f.olz = p[5];
    const float4 n = a.dirs32[r];
    f.f0 = n.x;
    f.f1 = n.y;
    f.f2 = n.z;
    return f;
}


// Step records of `cnt` consecutive steps, one per lane of a 16-lane group
// (the whole warp calls; cnt = 0 in a group with nothing to write): lane j < cnt writes the record of the step
// ending at its point my_pt, the step starting at the previous lane's point
// (prev_last for lane 0).  All in FP32: dx from the hi + lo scaled positions,
// beta = n.(v_c - v_o)/c and dbeta = n.(v_c - v_prev)/c from hi + lo values
// of v/c (relative error about 1e-7 of |v_c - v_o|/c), the averaged width of
// the segment.
__device__ __forceinline__ void write_step_records(const WalkArgs &a, int64_t o, int r, int64_t prev_last,
                                                   int32_t my_pt, int cnt, const float *__restrict__ vel_hl,
                                                   const float2 *__restrict__ w32, float inv_Lunit, int width_mode,
                                                   Step32 *__restrict__ out, int sl)
{
    int64_t prev = __shfl_up_sync(0xffffffffu, my_pt, 1, 16);
    if (sl == 0) prev = prev_last;
    if (sl >= cnt) return;
    const int64_t c = my_pt;
    const float *pc = a.pos_hl + 6 * c, *pp = a.pos_hl + 6 * prev;
    const float *vc = vel_hl + 6 * c, *vp = vel_hl + 6 * prev, *vo = vel_hl + 6 * o;
    const float4 n = a.dirs32[r];
    float e[3], db[3], dp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        e[d] = (pc[d] - pp[d]) + (pc[3 + d] - pp[3 + d]);
        db[d] = (vc[d] - vo[d]) + (vc[3 + d] - vo[3 + d]);
        dp[d] = (vc[d] - vp[d]) + (vc[3 + d] - vp[3 + d]);
    }
    const float dxs = sqrtf(fmaf(e[2], e[2], fmaf(e[1], e[1], e[0] * e[0]))) * inv_Lunit;
    const float beta = fmaf(n.z, db[2], fmaf(n.y, db[1], n.x * db[0]));
    const float dbeta = fmaf(n.z, dp[2], fmaf(n.y, dp[1], n.x * dp[0]));
    const float wc = w32[c].x, wp = w32[prev].x;
    const float wbar = width_mode == 0 ? sqrtf(0.5f * (wc * wc + wp * wp)) : 0.5f * (wc + wp);
    out[sl] = make_int4((int)c, __float_as_int(dxs), __float_as_int(beta), __float_as_int(dbeta / wbar));
}

// Minimum over the calling lane's 16-lane group of a non-negative float: two
// whole-warp integer min-reductions (non-negative floats order like their bit
// patterns), each lane keeping its own group's.  One reduction instruction per
// group instead of four dependent shuffle-and-min steps.
__device__ __forceinline__ float group16_min_nonneg(float v, int grp)
{
    const unsigned k = __float_as_uint(v);
    const unsigned k0 = __reduce_min_sync(0xffffffffu, grp == 0 ? k : 0xffffffffu);
    const unsigned k1 = __reduce_min_sync(0xffffffffu, grp == 1 ? k : 0xffffffffu);
    return __uint_as_float(grp ? k1 : k0);
}

// ---------------------------------------------------------------------------
// Two walks per warp, one per 16-lane group.  Each step reads the current
// point's row of packed neighbour entries (WalkEntry: the neighbour's scaled
// position as float hi + lo, its index with its boundary flag and a
// last-of-row flag, and the offset of its own row), 16 entries per load, so
// the next step's row offset, the winner's index and its boundary flag arrive
// with the candidates: one dependent L2 round trip per step.
//
// The lanes evaluate the candidates with FP32 arithmetic and error bounds that
// cover both the FP32 and the FP64 rounding (generous multiples of the
// rounding analysis):
//   offsets    |d32 - d64| <= ed = 2e-6 (|d32|_max + slack)
//   projection |Z32 - Z64| <= eZ = 2e-6 |d32|_1 + 2 ed
//   perpendicular components  ep = ed + eZ + 2e-7 (|p32|_max + |Z32|)
//   squared distance |d2_32 - d2_64| <= 4 |p32| ep + 4 ep^2 + 1e-6 d2_32.
// The current point's projection Z_c is carried as the winner's FP32 value
// with its bound eZ_c.  A neighbour is a candidate when Z32 - eZ clears
// Z_c + eZ_c, not one when Z32 + eZ stays at or below Z_c - eZ_c; anything in
// between leaves the step undecided.  The FP32 winner (smallest d2, lowest
// lane) is accepted only if its upper d2 bound is below every other
// candidate's lower bound, so near-ties never decide.  Undecided steps run
// walk_next_exact, the FP64 predicates themselves (exact Z_c recomputed by
// the same expression), on lane 0 of the group.  The point lists are
// therefore those of the FP64 rule.
//
// Two modes share the walk:
//  * kWalkFused: every walk of the grid.  Writes the half-ray length, counts
//    stalls, and writes the step records (see Step32), 16 at a time, into a
//    fixed-stride scratch area (K records per walk); records of steps >= K are
//    not kept (such walks are redone by the list mode).
//  * kWalkList: the walks named in `list` only, records written to their final
//    place (ray offsets known).
//  * kWalkImgCount / kWalkImgFill: the two half-rays of every image pixel
//    (walk 2q + h: h = 0 along -n, h = 1 along +n, n toward the observer),
//    from the pixel's anchor point, distances to the pixel line, Z measured
//    from the pixel's reference point; the count mode writes the lengths, the
//    fill mode the point indices of the full ray (far half reversed, anchor,
//    near half).
// ---------------------------------------------------------------------------
constexpr int kWalkFused = 0, kWalkList = 1, kWalkImgCount = 2, kWalkImgFill = 3;

struct ImgWalkArgs {
    const double *ref;        // [npix][3] pixel reference points
    const int32_t *anchor;    // [npix] start point of both half-rays
    const int64_t *off;       // [npix+1] full-ray offsets (fill mode)
    int32_t *pts;             // full rays (fill mode)
    int64_t npix;
    double n[3];              // unit direction toward the observer
};

// Blocks of 128 threads, eight per SM (registers capped at 64): the walk is
// bound by dependent latency (L2 row loads, shuffle chains), and 32 resident
// warps per SM beat the spill-free 93-register build at 16 (workload 2 trace:
// 91 -> 73 ms; 128-thread blocks instead of 256 a further 3 %).  Every launch
// uses kWalkThreads.
constexpr int kWalkThreads = 128;
template <int MODE>
__global__ void __launch_bounds__(kWalkThreads, 8) k_walk(WalkArgs a, int64_t *__restrict__ lens, const int64_t *__restrict__ ray_off,
                                              const int64_t *__restrict__ list, int64_t n_list, int32_t K,
                                              unsigned long long *__restrict__ n_stall,
                                              const float *__restrict__ vel_hl, const float2 *__restrict__ w32,
                                              float inv_Lunit, int width_mode, Step32 *__restrict__ steps,
                                              int *__restrict__ err, ImgWalkArgs im)
{
    constexpr bool IMG = MODE == kWalkImgCount || MODE == kWalkImgFill;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, sl = lane & 15, grp = lane >> 4;
    const unsigned gmask = 0xffffu << (16 * grp);
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4;   // walk slot
    const int64_t W = MODE == kWalkFused ? (int64_t)a.R * a.N : IMG ? 2 * im.npix : n_list;
    if ((wg & ~(int64_t)1) >= W) return;                       // both walks of the warp absent
    bool live = wg < W;
    int r = 0;
    int64_t o = 0;
    if (live) {
        if (MODE == kWalkFused) {
            r = (int)(wg / a.N);
            o = a.order[wg - (int64_t)r * a.N];
        } else if (IMG) {
            r = (int)(wg & 1);
            o = im.anchor[wg >> 1];
        } else {
            const int64_t t = list[wg];
            r = (int)(t / a.N);
            o = t - (int64_t)r * a.N;
        }
    }
    if (o < 0 || o >= a.N || r < 0 || r >= (IMG ? 2 : a.R)) {   // index check: record and skip
        walk_give_up(err, 13, wg, o);
        o = 0;
        r = 0;
        live = false;
    }
    const int64_t wi = (int64_t)r * a.N + o;
    const int rg = (!IMG && a.dir_map) ? a.dir_map[r] : r;   // the model's direction index
    // the walk's frame: origin o and direction r, or for image walks the pixel's
    // reference point and -n / +n (FP64 values are loaded again where needed)
    WalkFrame f;
    double img_Z0 = 0.0;                        // image walks: Z of the anchor
    if (IMG) {
        const double sg = r == 0 ? -1.0 : 1.0;
        const double *pr = im.ref + 3 * (wg >> 1);
        const double sx = pr[0] * a.pos_scale, sy = pr[1] * a.pos_scale, sz = pr[2] * a.pos_scale;
        f.ohx = (float)sx;
        f.ohy = (float)sy;
        f.ohz = (float)sz;
        f.olx = (float)(sx - (double)f.ohx);
        f.oly = (float)(sy - (double)f.ohy);
        f.olz = (float)(sz - (double)f.ohz);
        f.f0 = (float)(sg * im.n[0]);
        f.f1 = (float)(sg * im.n[1]);
        f.f2 = (float)(sg * im.n[2]);
        const double *q = a.pos + 3 * o;
        img_Z0 = dot3_exact(__dsub_rn(q[0], pr[0]), __dsub_rn(q[1], pr[1]), __dsub_rn(q[2], pr[2]), sg * im.n[0],
                            sg * im.n[1], sg * im.n[2]);
    } else {
        f = make_frame(a, o, rg);
    }
    // records go to out[0 .. cap): the walk's scratch slot, or its final place
    int64_t cap = K;
    Step32 *out = steps + wi * (int64_t)K;
    if (MODE == kWalkList && live) {
        out = steps + ray_off[wi];
        cap = ray_off[wi + 1] - ray_off[wi];
    }
    if (IMG) cap = a.N;
    int64_t img_nfar = 0, img_base = 0;         // fill: far-half length and the pixel's ray offset
    if (MODE == kWalkImgFill && live) {
        img_nfar = lens[wg & ~(int64_t)1];
        img_base = im.off[wg >> 1];
        cap = lens[wg];
    }
    // step records are built 16 at a time: lane j of the group keeps the point
    // of step (chunk start + j); prev_last is the point before the chunk
    int32_t my_pt = 0;
    int64_t prev_last = o;
    int64_t c = o, n = 0;
    int32_t c_off = live ? a.ent_off[o] : 0;   // the current point's row of packed entries
    float Zc = 0.0f, eZc = 0.0f;                // Z of o is exactly 0 (image walks: the anchor's Z)
    if (IMG) {
        Zc = (float)(img_Z0 * a.pos_scale);     // the filter works in scaled units (exact factor)
        eZc = 1e-7f * fabsf(Zc) + 1e-30f;
    }
    bool done = !live;
    // every loop below is bounded: the walk by the point count and a 2 s
    // clock, a row scan by the number of packed entries; running out records
    // the site and returns
    const uint64_t t_start = walk_clock_ns();
    bool gave_up = false;
    uint32_t iter = 0;                          // the same in every lane (the loop test is a warp vote)
    while (!__all_sync(full, done)) {
        if ((++iter & 15u) == 0u && __any_sync(full, walk_clock_ns() - t_start > 2000000000ull)) {
            if (sl == 0 && !done) walk_give_up(err, 1, wg, n);
            gave_up = true;
            break;
        }
        // each lane keeps the best of its own entries over the row's chunks
        // (smallest d2, the earlier chunk on ties) and the least lower bound
        // of its other candidates; the group decides once per step
        float bd2 = 3.0e38f, bU = 0.0f, bLo = 3.0e38f, bZ = 0.0f, beZ = 0.0f, lo2 = 3.0e38f;
        uint32_t bword = 0u;
        int32_t boff = 0;
        bool und_lane = false, row_open = !done;
        int32_t chunks = 0;
        for (int32_t kb = c_off; __any_sync(full, row_open); kb += 16) {
            if (++chunks > a.max_row_chunks) {
                if (sl == 0 && row_open) walk_give_up(err, 2, wg, n);
                gave_up = true;
                break;
            }
            bool last = false;
            uint32_t word = 0u;
            int32_t eoff = 0;
            float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0;
            if (row_open && (kb + sl < 0 || kb + sl >= a.n_ent)) {   // index check: record and skip
                walk_give_up(err, 10, wg, kb + sl);
                row_open = false;
            }
            if (row_open) {
                const float4 *ep = reinterpret_cast<const float4 *>(a.ent + 2 * (int64_t)(kb + sl));
                e0 = ep[0];
                e1 = ep[1];
                word = __float_as_uint(e1.z);
                eoff = __float_as_int(e1.w);
                last = (word & kEntLast) != 0u;
            }
            // entries up to the group's first last-of-row flag belong to the row
            const unsigned lastbits = (__ballot_sync(full, last) & gmask) >> (16 * grp);
            const bool inrow = row_open && (lastbits & ((1u << sl) - 1u)) == 0u;
            if (inrow && (word & kEntIdx) != kEntEmpty) {
                const float dx = (e0.x - f.ohx) + (e0.w - f.olx);
                const float dy = (e0.y - f.ohy) + (e1.x - f.oly);
                const float dz = (e0.z - f.ohz) + (e1.y - f.olz);
                const float adx = fabsf(dx), ady = fabsf(dy), adz = fabsf(dz);
                const float ed = 2e-6f * (fmaxf(adx, fmaxf(ady, adz)) + a.pos_slack);
                const float Z = fmaf(dz, f.f2, fmaf(dy, f.f1, dx * f.f0));
                const float eZ = 2e-6f * (adx + ady + adz) + 2.0f * ed;
                if (Z - eZ > Zc + eZc) {
                    const float px = fmaf(-Z, f.f0, dx), py = fmaf(-Z, f.f1, dy), pz = fmaf(-Z, f.f2, dz);
                    const float d2 = fmaf(pz, pz, fmaf(py, py, px * px));
                    const float ep = ed + eZ + 2e-7f * (fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))) + fabsf(Z));
                    // |p32| from the approximate square root, raised by 2^-10
                    // (far above its error) so that the bound stays an upper one
                    float rp;
                    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rp) : "f"(d2));
                    const float e2 = 4.0f * (rp * 1.0009765625f) * ep + 4.0f * ep * ep + 1e-6f * d2;
                    const float U = d2 + e2, Lo = d2 - e2;
                    if (d2 < bd2) {
                        lo2 = fminf(lo2, bLo);
                        bd2 = d2;
                        bU = U;
                        bLo = Lo;
                        bZ = Z;
                        beZ = eZ;
                        bword = word;
                        boff = eoff;
                    } else {
                        lo2 = fminf(lo2, Lo);
                    }
                } else if (!(Z + eZ <= Zc - eZc)) {
                    und_lane = true;
                }
            }
            row_open = row_open && lastbits == 0u;
        }
        if (gave_up) break;
        // The decision runs in both groups in lockstep (a finished group only
        // predicates itself off), so every warp intrinsic below names the
        // whole warp.  The FP32 winner is the group's smallest d2 (lowest lane
        // on ties); it is accepted only if every other candidate's lower bound
        // lies above its upper bound (a negative lower bound always fails,
        // since upper bounds are >= 0), so a tie never decides.
        const bool undecided = (__ballot_sync(full, und_lane) & gmask) != 0u;
        const float m = group16_min_nonneg(bd2, grp);
        const bool have = m < 3.0e38f;
        const unsigned wins = (__ballot_sync(full, have && bd2 == m) & gmask) >> (16 * grp);
        const int wl = wins ? __ffs(wins) - 1 : sl;
        const int src = 16 * grp + wl;
        bU = __shfl_sync(full, bU, src);
        bZ = __shfl_sync(full, bZ, src);
        beZ = __shfl_sync(full, beZ, src);
        bword = __shfl_sync(full, bword, src);
        boff = __shfl_sync(full, boff, src);
        const float lo_other = sl == wl ? lo2 : fminf(bLo, lo2);
        const bool close = (__ballot_sync(full, have && lo_other <= bU) & gmask) != 0u;
        const bool exact = !done && (undecided || close);
        int64_t v = -1;
        double Zn = 0.0;
        if (exact && sl == 0) {
            // FP64 predicates, evaluated by lane 0 of the group
            if (!IMG) atomicAdd(a.n_exact, 1ULL);
            double xo, yo, zo, n0, n1, n2;
            if (IMG) {
                const double *pr = im.ref + 3 * (wg >> 1);
                const double sg = r == 0 ? -1.0 : 1.0;
                xo = pr[0];
                yo = pr[1];
                zo = pr[2];
                n0 = sg * im.n[0];
                n1 = sg * im.n[1];
                n2 = sg * im.n[2];
            } else {
                xo = a.pos[3 * o];
                yo = a.pos[3 * o + 1];
                zo = a.pos[3 * o + 2];
                n0 = a.dirs[3 * rg];
                n1 = a.dirs[3 * rg + 1];
                n2 = a.dirs[3 * rg + 2];
            }
            double Zc64 = 0.0;
            if (c != o || IMG) {
                const double *q = a.pos + 3 * c;
                Zc64 = dot3_exact(__dsub_rn(q[0], xo), __dsub_rn(q[1], yo), __dsub_rn(q[2], zo), n0, n1, n2);
            }
            v = walk_next_exact(a, c, xo, yo, zo, n0, n1, n2, Zc64, &Zn);
        }
        if (__any_sync(full, exact)) {          // (rare) the FP64 result of lane 0 to its group
            v = __shfl_sync(full, v, 16 * grp);
            Zn = __shfl_sync(full, Zn, 16 * grp);
        }
        int64_t nx = -1;
        bool nx_bnd = false;
        if (!done) {
            if (exact) {
                nx = v;
                if (nx >= a.N) {
                    walk_give_up(err, 11, wg, nx);
                    nx = -1;
                }
                Zc = (float)(Zn * a.pos_scale);      // the filter works in scaled units (exact factor)
                eZc = 1e-7f * fabsf(Zc) + 1e-30f;
                nx_bnd = nx >= 0 && a.bnd[nx] != 0;
                if (nx >= 0) c_off = a.ent_off[nx];
            } else if (have) {
                nx = (int64_t)(bword & kEntIdx);
                if (nx >= a.N || boff < 0 || boff >= a.n_ent) {
                    walk_give_up(err, 12, wg, nx);
                    nx = -1;
                }
                nx_bnd = (bword & kEntBnd) != 0u;
                c_off = boff;
                Zc = bZ;
                eZc = beZ;
            }
        }
        bool flush_full = false, flush_last = false;   // a full chunk of 16 records / the walk's tail
        if (!done) {
            if (nx < 0) {
                if (MODE == kWalkFused && sl == 0 && !(c == o && a.bnd[o])) atomicAdd(n_stall, 1ULL);
                done = true;
                flush_last = (n & 15) != 0;
            } else if ((MODE == kWalkList || MODE == kWalkImgFill) && n >= cap) {   // cannot happen: deterministic walk
                if (sl == 0) atomicCAS(err, 0, (int)kDevBounds);
                done = true;
            } else {
                if (sl == (int)(n & 15)) my_pt = (int32_t)nx;
                flush_full = (n & 15) == 15;
                ++n;
                c = nx;
                if (nx_bnd || n >= a.N) {
                    done = true;
                    flush_last = (n & 15) != 0;
                }
            }
        }
        if (IMG) {
            // image fill: the group's buffered point indices to their place in
            // the pixel's full ray (far half reversed, then anchor, then near half)
            if (MODE == kWalkImgFill && __any_sync(full, flush_full || flush_last)) {
                const int cnt = flush_full ? 16 : (int)(n & 15);
                const int64_t first = flush_full ? n - 16 : (n & ~(int64_t)15);
                if ((flush_full || flush_last) && sl < cnt) {
                    const int64_t k = first + sl;
                    const int64_t at = r == 0 ? img_base + img_nfar - 1 - k : img_base + img_nfar + 1 + k;
                    im.pts[at] = my_pt;
                }
            }
        } else if (__any_sync(full, flush_full || flush_last)) {
            // records of the group's buffered steps (n already counts the newest);
            // chunks start at multiples of 16 and cap is one (fused mode) or
            // exactly the walk's length (list mode), so a chunk is kept whole or
            // not at all
            const int cnt = flush_full ? 16 : (int)(n & 15);
            const int64_t first = flush_full ? n - 16 : (n & ~(int64_t)15);
            const bool keep = (flush_full || flush_last) && first < cap;
            write_step_records(a, o, rg, prev_last, my_pt, keep ? cnt : 0, vel_hl, w32, inv_Lunit, width_mode,
                               out + first, sl);
            if (flush_full) prev_last = nx;
        }
    }
    if (live && sl == 0) {
        if (MODE == kWalkFused)
            lens[wi] = gave_up ? 0 : n;
        else if (MODE == kWalkImgCount)
            lens[wg] = gave_up ? 0 : n;
        else if (n != cap && !gave_up)
            atomicCAS(err, 0, (int)kDevBounds);
    }
}

// Walks whose records did not fit their scratch slot (length > K).
__global__ void k_walk_overflow(int64_t W, const int64_t *__restrict__ lens, int32_t K, int64_t *__restrict__ list,
                                unsigned long long *__restrict__ count)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= W || lens[t] <= K) return;
    list[atomicAdd(count, 1ULL)] = t;
}

// Move each walk's records (at most K) from its scratch slot to its final
// place: one warp per walk, 16-byte records.
__global__ void k_walk_compact(int64_t W, const int64_t *__restrict__ ray_off, int32_t K,
                               const Step32 *__restrict__ scratch, Step32 *__restrict__ steps)
{
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= W) return;
    const int64_t b = ray_off[t], n = ray_off[t + 1] - b;
    const int64_t m = n < K ? n : K;
    for (int64_t j = lane; j < m; j += 32) steps[b + j] = scratch[t * (int64_t)K + j];
}

// Double-precision step geometry for the FP64 formal solution, from the
// traced point lists (one thread per half-ray).
__global__ void k_steps64(int64_t N, int32_t R, const int64_t *__restrict__ off, const Step32 *__restrict__ s32,
                          const double *__restrict__ pos, const double *__restrict__ vel,
                          const double *__restrict__ w64, const double *__restrict__ dirs,
                          const int32_t *__restrict__ dir_map, double inv_Lunit, int width_mode,
                          Step64 *__restrict__ s64)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * N) return;
    int r = (int)(t / N);
    int64_t o = t - (int64_t)r * N;
    const int rg = dir_map ? dir_map[r] : r;
    double n0 = dirs[3 * rg], n1 = dirs[3 * rg + 1], n2 = dirs[3 * rg + 2];
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

mgt_status trace_all(mgt_model *m, cudaStream_t s) { return trace_range(m, s, 0, m->P); }

// Trace the rays of pairs [p0, p0 + np).  All pairs: walk direction = model
// direction, ray offsets direction-major over all R directions.  A batch:
// walk directions 2i and 2i+1 are the two directions of pair p0 + i (see
// d_dir_map, d_batch_pairs), ray offsets over the batch's 2 np directions.
mgt_status trace_range(mgt_model *m, cudaStream_t s, int32_t p0, int32_t np)
{
    const bool all = p0 == 0 && np == m->P;
    const int32_t Rw = all ? m->R : 2 * np;
    if (!all) {
        std::vector<int32_t> map(2 * np);
        std::vector<int2> bp(np);
        for (int32_t i = 0; i < np; ++i) {
            map[2 * i] = m->pairs[2 * (p0 + i)];
            map[2 * i + 1] = m->pairs[2 * (p0 + i) + 1];
            bp[i] = make_int2(2 * i, 2 * i + 1);
        }
        MGT_CUDA(cudaMemcpyAsync(m->d_dir_map, map.data(), sizeof(int32_t) * map.size(), cudaMemcpyHostToDevice, s));
        MGT_CUDA(cudaMemcpyAsync(m->d_batch_pairs, bp.data(), sizeof(int2) * bp.size(), cudaMemcpyHostToDevice, s));
        MGT_CUDA(cudaStreamSynchronize(s));
    }
    const int64_t W = (int64_t)Rw * m->N;
    WalkArgs a{m->N,        Rw,            m->d_pos,  m->d_nbr_off, m->d_nbrs,   m->d_nbr_pos,
               m->pos_scale, m->d_bnd,     m->d_dirs, m->d_ent,     m->d_ent_off, m->d_pos_hl,
               m->d_dirs32,  m->d_order,   m->pos_slack, m->d_count + 2,
               (int32_t)((m->n_ent + 15) / 16 + 2), m->n_ent, all ? nullptr : m->d_dir_map};
    if (!m->d_ray_off) MGT_CUDA(cudaMalloc(&m->d_ray_off, sizeof(int64_t) * ((int64_t)m->R * m->N + 1)));
    // Scratch slot per walk: K records, a multiple of 16; the longest half-ray
    // of this model's previous trace when there was one, else 4 N^(1/3) + 16
    // (a few times the mean half-ray of a cloud of N points), kept within a
    // third of the free device memory (counting what the scratch pool holds
    // unused).  Longer walks are redone.
    int64_t K = m->max_half > 0 ? (m->max_half + 15) / 16 * 16
                                : ((int64_t)(4.0 * std::cbrt((double)m->N)) + 16 + 15) / 16 * 16;
    cudaMemPool_t pool = nullptr;
    MGT_TRY_STATUS(scratch_pool(&pool));
    {
        size_t freeb = 0, totalb = 0;
        MGT_CUDA(cudaMemGetInfo(&freeb, &totalb));
        uint64_t reserved = 0, used = 0;
        MGT_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
        MGT_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
        freeb += reserved > used ? (size_t)(reserved - used) : 0;
        while (K > 16 && (size_t)(W * K) * sizeof(Step32) > freeb / 3) K -= 16;
    }
    int64_t *d_len = nullptr, *d_list = nullptr, *d_max = nullptr;
    Step32 *d_scratch = nullptr;
    unsigned long long *d_nover = nullptr;
    void *tmp = nullptr, *tmpb = nullptr;
    auto release = [&]() {
        if (tmp) cudaFreeAsync(tmp, s);
        if (tmpb) cudaFreeAsync(tmpb, s);
        if (d_max) cudaFreeAsync(d_max, s);
        if (d_len) cudaFreeAsync(d_len, s);
        if (d_list) cudaFreeAsync(d_list, s);
        if (d_nover) cudaFreeAsync(d_nover, s);
        if (d_scratch) cudaFreeAsync(d_scratch, s);
    };
    struct Guard {
        decltype(release) &f;
        ~Guard() { f(); }
    } guard{release};
    MGT_CUDA(cudaMallocFromPoolAsync(&d_len, sizeof(int64_t) * (W + 1), pool, s));
    MGT_CUDA(cudaMallocFromPoolAsync(&d_list, sizeof(int64_t) * W, pool, s));
    MGT_CUDA(cudaMallocFromPoolAsync(&d_nover, sizeof(unsigned long long), pool, s));
    if (cudaMallocFromPoolAsync(&d_scratch, sizeof(Step32) * W * K, pool, s) != cudaSuccess) {
        cudaGetLastError();
        d_scratch = nullptr;
        return set_error(MGT_ERR_OOM, "cannot allocate the walk scratch");
    }
    MGT_CUDA(cudaMemsetAsync(m->d_count + 1, 0, 2 * sizeof(unsigned long long), s));
    MGT_CUDA(cudaMemsetAsync(d_nover, 0, sizeof(unsigned long long), s));
    const float inv_Lunit = (float)(1.0 / (m->pos_scale * m->L_unit));
    {
        MGT_KTIMER("k_walk<fused>", s);
        k_walk<kWalkFused><<<ceil_div(W * 16, kWalkThreads), kWalkThreads, 0, s>>>(a, d_len, nullptr, nullptr, 0, (int32_t)K,
                                                                 m->d_count + 1, m->d_vel_hl, m->d_w32, inv_Lunit,
                                                                 m->opts.width_mode, d_scratch, m->d_err, ImgWalkArgs{});
    }
    MGT_LAUNCH_CHECK("k_walk<fused>");
    MGT_CUDA(cudaMemsetAsync(d_len + W, 0, sizeof(int64_t), s));
    size_t tmp_bytes = 0;
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_len, m->d_ray_off, W + 1, s));
    MGT_CUDA(cudaMallocFromPoolAsync(&tmp, tmp_bytes, pool, s));
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, d_len, m->d_ray_off, W + 1, s));
    // longest half-ray
    MGT_CUDA(cudaMallocFromPoolAsync(&d_max, sizeof(int64_t), pool, s));
    size_t tmp2 = 0;
    MGT_CUDA(cub::DeviceReduce::Max(nullptr, tmp2, d_len, d_max, W, s));
    MGT_CUDA(cudaMallocFromPoolAsync(&tmpb, tmp2, pool, s));
    MGT_CUDA(cub::DeviceReduce::Max(tmpb, tmp2, d_len, d_max, W, s));
    k_walk_overflow<<<ceil_div(W, 256), 256, 0, s>>>(W, d_len, (int32_t)K, d_list, d_nover);
    MGT_LAUNCH_CHECK("k_walk_overflow");
    int64_t total = 0, mx = 0;
    unsigned long long stalls = 0, exact_steps = 0, n_over = 0;
    MGT_CUDA(cudaMemcpyAsync(&total, m->d_ray_off + W, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&mx, d_max, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&stalls, m->d_count + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&exact_steps, m->d_count + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaMemcpyAsync(&n_over, d_nover, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    MGT_TRY_STATUS(check_device_error(m, s));     // a walk that gave up leaves the lengths unusable
    // the ray buffer comes from the same pool: a model created after another
    // one was destroyed reuses its mapping.  A formal solution on another
    // stream may still read the old buffer, hence the device-wide wait.
    if (m->d_steps32 && total > m->steps32_cap) {
        MGT_CUDA(cudaDeviceSynchronize());
        MGT_CUDA(cudaFreeAsync(m->d_steps32, s));
        m->d_steps32 = nullptr;
    }
    m->steps64_width_mode = -1;                // the FP64 geometry describes the previous rays
    if (!m->d_steps32 && total > 0) {
        cudaError_t e = cudaMallocFromPoolAsync(&m->d_steps32, sizeof(Step32) * total, pool, s);
        if (e != cudaSuccess) return set_error(MGT_ERR_OOM, "cannot allocate the ray buffer");
        m->steps32_cap = total;
    }
    m->total_steps = total;
    m->max_half = (int32_t)mx;
    m->n_stalls = (int64_t)stalls;
    m->n_exact_steps = (int64_t)exact_steps;   // the walks of the fused pass
    if (total > 0) {
        {
            // each record read once from its slot and written once, plus the offsets
            MGT_KTIMER_BYTES("k_walk_compact", s, 32.0 * (double)total + 8.0 * (double)W);
            k_walk_compact<<<ceil_div(W * 32, 256), 256, 0, s>>>(W, m->d_ray_off, (int32_t)K, d_scratch, m->d_steps32);
        }
        MGT_LAUNCH_CHECK("k_walk_compact");
        if (n_over > 0) {
            {
                MGT_KTIMER("k_walk<list>", s);
                k_walk<kWalkList><<<ceil_div((int64_t)n_over * 16, kWalkThreads), kWalkThreads, 0, s>>>(
                    a, nullptr, m->d_ray_off, d_list, (int64_t)n_over, 0, nullptr, m->d_vel_hl, m->d_w32, inv_Lunit,
                    m->opts.width_mode, m->d_steps32, m->d_err, ImgWalkArgs{});
            }
            MGT_LAUNCH_CHECK("k_walk<list>");
        }
    }
    m->steps_width_mode = m->opts.width_mode;
    m->rays_p0 = p0;
    m->rays_np = np;
    m->traced = true;
    return MGT_OK;
}

mgt_status build_steps64(mgt_model *m, cudaStream_t s)
{
    if (m->total_steps == 0) return MGT_OK;
    if (m->d_steps64 && m->steps64_cap < m->total_steps) {
        MGT_CUDA(cudaFree(m->d_steps64));
        m->d_steps64 = nullptr;
    }
    if (!m->d_steps64) {
        m->steps64_cap = m->total_steps;
        cudaError_t e = cudaMalloc(&m->d_steps64, sizeof(Step64) * m->total_steps);
        if (e != cudaSuccess) return set_error(MGT_ERR_OOM, "cannot allocate the FP64 ray geometry");
    }
    const bool all = m->rays_p0 == 0 && m->rays_np == m->P;
    const int32_t Rw = all ? m->R : 2 * m->rays_np;
    const int64_t W = (int64_t)Rw * m->N;
    k_steps64<<<ceil_div(W, 128), 128, 0, s>>>(m->N, Rw, m->d_ray_off, m->d_steps32, m->d_pos, m->d_vel,
                                               m->d_w64, m->d_dirs, all ? nullptr : m->d_dir_map, 1.0 / m->L_unit,
                                               m->opts.width_mode, m->d_steps64);
    MGT_LAUNCH_CHECK("k_steps64");
    m->steps64_width_mode = m->opts.width_mode;
    return MGT_OK;
}

}  // namespace mgt

namespace mgt {

// ---------------------------------------------------------------------------
// Synthetic image geometry (Listing 3, compute_image_new).  The paper gives
// no algorithm; the image plane, the pixel reference points, the anchor of a
// pixel (the point closest to the pixel line) and the two walks from it follow
// the definition written out in the model-independent form below, in FP64
// with every expression in the order written (host code is compiled without
// multiply-add contraction).
// ---------------------------------------------------------------------------
void image_frame(const double *pos, int64_t N, const double n[3], int32_t npx, int32_t npy, double e1[3],
                 double e2[3], std::vector<double> &ref)
{
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (std::fabs(n[k]) < std::fabs(n[ax])) ax = k;
    double av[3] = {0.0, 0.0, 0.0};
    av[ax] = 1.0;
    const double c[3] = {av[1] * n[2] - av[2] * n[1], av[2] * n[0] - av[0] * n[2], av[0] * n[1] - av[1] * n[0]};
    const double cl = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    for (int k = 0; k < 3; ++k) e1[k] = c[k] / cl;
    e2[0] = n[1] * e1[2] - n[2] * e1[1];
    e2[1] = n[2] * e1[0] - n[0] * e1[2];
    e2[2] = n[0] * e1[1] - n[1] * e1[0];
    double lo1 = 1e300, hi1 = -1e300, lo2 = 1e300, hi2 = -1e300;
    for (int64_t i = 0; i < N; ++i) {
        const double s1 = pos[3 * i] * e1[0] + pos[3 * i + 1] * e1[1] + pos[3 * i + 2] * e1[2];
        const double s2 = pos[3 * i] * e2[0] + pos[3 * i + 1] * e2[1] + pos[3 * i + 2] * e2[2];
        if (s1 < lo1) lo1 = s1;
        if (s1 > hi1) hi1 = s1;
        if (s2 < lo2) lo2 = s2;
        if (s2 > hi2) hi2 = s2;
    }
    const double c1 = 0.5 * (lo1 + hi1), c2 = 0.5 * (lo2 + hi2);
    const double H = 0.5 * ((hi1 - lo1) > (hi2 - lo2) ? (hi1 - lo1) : (hi2 - lo2));
    ref.assign(3 * (size_t)npx * npy, 0.0);
    for (int32_t j = 0; j < npy; ++j)
        for (int32_t i = 0; i < npx; ++i) {
            const double t1 = c1 - H + (i + 0.5) * (2.0 * H / npx);
            const double t2 = c2 - H + (j + 0.5) * (2.0 * H / npy);
            double *p = ref.data() + 3 * ((size_t)j * npx + i);
            for (int k = 0; k < 3; ++k) p[k] = t1 * e1[k] + t2 * e2[k];
        }
}

// Anchor of each pixel: the point whose squared distance to the pixel line
// |(x - p) - ((x - p).n) n|^2 is smallest, ties to the smaller index.  One
// warp per pixel; FP32 distances from hi + lo positions with the error bounds
// of the walk, an FP64 scan (the defining expressions) when the bounds do not
// separate the winner from every other point.
__global__ void __launch_bounds__(256) k_img_anchor(WalkArgs a, const double *__restrict__ ref, int64_t npix,
                                                    double n0, double n1, double n2, int32_t *__restrict__ anchor)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= npix) return;                                     // whole warp
    const double *pr = ref + 3 * q;
    const double sx = pr[0] * a.pos_scale, sy = pr[1] * a.pos_scale, sz = pr[2] * a.pos_scale;
    const float ohx = (float)sx, ohy = (float)sy, ohz = (float)sz;
    const float olx = (float)(sx - (double)ohx), oly = (float)(sy - (double)ohy), olz = (float)(sz - (double)ohz);
    const float f0 = (float)n0, f1 = (float)n1, f2 = (float)n2;
    float bd2 = 3.0e38f, bU = 3.0e38f, bL = 3.0e38f, minLo = 3.0e38f;
    int64_t bi = -1;
    for (int64_t i = lane; i < a.N; i += 32) {
        const float *h = a.pos_hl + 6 * i;
        const float dx = (h[0] - ohx) + (h[3] - olx), dy = (h[1] - ohy) + (h[4] - oly), dz = (h[2] - ohz) + (h[5] - olz);
        const float adx = fabsf(dx), ady = fabsf(dy), adz = fabsf(dz);
        const float ed = 2e-6f * (fmaxf(adx, fmaxf(ady, adz)) + a.pos_slack);
        const float Z = fmaf(dz, f2, fmaf(dy, f1, dx * f0));
        const float eZ = 2e-6f * (adx + ady + adz) + 2.0f * ed;
        const float px = fmaf(-Z, f0, dx), py = fmaf(-Z, f1, dy), pz = fmaf(-Z, f2, dz);
        const float d2 = fmaf(pz, pz, fmaf(py, py, px * px));
        const float ep = ed + eZ + 2e-7f * (fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))) + fabsf(Z));
        const float e2 = 4.0f * sqrtf(d2) * ep + 4.0f * ep * ep + 1e-6f * d2;
        if (d2 < bd2) {                       // strictly smaller: the lane's earlier index wins ties
            minLo = fminf(minLo, bL);
            bd2 = d2;
            bU = d2 + e2;
            bL = d2 - e2;
            bi = i;
        } else {
            minLo = fminf(minLo, d2 - e2);
        }
    }
    // warp winner: smallest d2, then smallest index
    float wd2 = bd2;
    int64_t wi = bi < 0 ? INT64_MAX : bi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float od = __shfl_xor_sync(full, wd2, o);
        const int64_t oi = __shfl_xor_sync(full, wi, o);
        if (od < wd2 || (od == wd2 && oi < wi)) {
            wd2 = od;
            wi = oi;
        }
    }
    const bool mine = bi == wi;
    float oth = fminf(minLo, mine ? 3.0e38f : bL);
    float wU = mine ? bU : 3.0e38f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        oth = fminf(oth, __shfl_xor_sync(full, oth, o));
        wU = fminf(wU, __shfl_xor_sync(full, wU, o));
    }
    int64_t best = wi;
    if (!(wU < oth)) {
        // FP64, the defining expressions
        double ed2 = 0.0;
        int64_t ei = -1;
        for (int64_t i = lane; i < a.N; i += 32) {
            const double *x = a.pos + 3 * i;
            const double dx = __dsub_rn(x[0], pr[0]), dy = __dsub_rn(x[1], pr[1]), dz = __dsub_rn(x[2], pr[2]);
            const double Z = dot3_exact(dx, dy, dz, n0, n1, n2);
            const double px = __dsub_rn(dx, __dmul_rn(Z, n0)), py = __dsub_rn(dy, __dmul_rn(Z, n1)),
                         pz = __dsub_rn(dz, __dmul_rn(Z, n2));
            const double d2 = dot3_exact(px, py, pz, px, py, pz);
            if (ei < 0 || d2 < ed2) {
                ed2 = d2;
                ei = i;
            }
        }
        if (ei < 0) ei = INT64_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double od = __shfl_xor_sync(full, ed2, o);
            const int64_t oi = __shfl_xor_sync(full, ei, o);
            if (oi != INT64_MAX && (ei == INT64_MAX || od < ed2 || (od == ed2 && oi < ei))) {
                ed2 = od;
                ei = oi;
            }
        }
        best = ei;
    }
    if (lane == 0) anchor[q] = (int32_t)best;
}

// Full-ray sizes: nfar + anchor + nnear per pixel.
__global__ void k_img_sizes(int64_t npix, const int64_t *__restrict__ lens, int64_t *__restrict__ sizes)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < npix) sizes[q] = lens[2 * q] + lens[2 * q + 1] + 1;
}

__global__ void k_img_place_anchor(int64_t npix, const int64_t *__restrict__ lens, const int64_t *__restrict__ off,
                                   const int32_t *__restrict__ anchor, int32_t *__restrict__ pts)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < npix) pts[off[q] + lens[2 * q]] = anchor[q];
}

void image_free(mgt_model *m)
{
    ImageGeom &g = m->img;
    if (g.d_ref) cudaFree(g.d_ref);
    if (g.d_anchor) cudaFree(g.d_anchor);
    if (g.d_off) cudaFree(g.d_off);
    if (g.d_pts) cudaFree(g.d_pts);
    g = ImageGeom{};
}

mgt_status trace_image(mgt_model *m, const double n[3], int32_t npx, int32_t npy, cudaStream_t s)
{
    ImageGeom &g = m->img;
    if (g.valid && g.npx == npx && g.npy == npy && g.n[0] == n[0] && g.n[1] == n[1] && g.n[2] == n[2])
        return MGT_OK;
    image_free(m);
    const int64_t npix = (int64_t)npx * npy;
    std::vector<double> pos(3 * (size_t)m->N), ref;
    MGT_CUDA(cudaMemcpyAsync(pos.data(), m->d_pos, sizeof(double) * 3 * m->N, cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    double e1[3], e2[3];
    image_frame(pos.data(), m->N, n, npx, npy, e1, e2, ref);
    MGT_CUDA(cudaMalloc(&g.d_ref, sizeof(double) * ref.size()));
    MGT_CUDA(cudaMalloc(&g.d_anchor, sizeof(int32_t) * npix));
    MGT_CUDA(cudaMalloc(&g.d_off, sizeof(int64_t) * (npix + 1)));
    MGT_CUDA(cudaMemcpyAsync(g.d_ref, ref.data(), sizeof(double) * ref.size(), cudaMemcpyHostToDevice, s));
    WalkArgs a{m->N,        m->R,          m->d_pos,  m->d_nbr_off, m->d_nbrs,   m->d_nbr_pos,
               m->pos_scale, m->d_bnd,     m->d_dirs, m->d_ent,     m->d_ent_off, m->d_pos_hl,
               m->d_dirs32,  m->d_order,   m->pos_slack, m->d_count + 3,
               (int32_t)((m->n_ent + 15) / 16 + 2), m->n_ent, nullptr};
    k_img_anchor<<<ceil_div(npix * 32, 256), 256, 0, s>>>(a, g.d_ref, npix, n[0], n[1], n[2], g.d_anchor);
    MGT_LAUNCH_CHECK("k_img_anchor");
    int64_t *d_lens = nullptr, *d_sizes = nullptr;
    void *tmp = nullptr;
    MGT_CUDA(cudaMallocAsync(&d_lens, sizeof(int64_t) * 2 * npix, s));
    MGT_CUDA(cudaMallocAsync(&d_sizes, sizeof(int64_t) * (npix + 1), s));
    ImgWalkArgs im{g.d_ref, g.d_anchor, g.d_off, nullptr, npix, {n[0], n[1], n[2]}};
    k_walk<kWalkImgCount><<<ceil_div(2 * npix * 16, kWalkThreads), kWalkThreads, 0, s>>>(a, d_lens, nullptr, nullptr, 0, 0, nullptr,
                                                                       nullptr, nullptr, 0.0f, 0, nullptr, m->d_err,
                                                                       im);
    MGT_LAUNCH_CHECK("k_walk<image count>");
    k_img_sizes<<<ceil_div(npix, 256), 256, 0, s>>>(npix, d_lens, d_sizes);
    MGT_LAUNCH_CHECK("k_img_sizes");
    MGT_CUDA(cudaMemsetAsync(d_sizes + npix, 0, sizeof(int64_t), s));
    size_t tb = 0;
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, d_sizes, g.d_off, npix + 1, s));
    MGT_CUDA(cudaMallocAsync(&tmp, tb, s));
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tb, d_sizes, g.d_off, npix + 1, s));
    int64_t total = 0;
    MGT_CUDA(cudaMemcpyAsync(&total, g.d_off + npix, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    std::vector<int64_t> sizes(npix);
    MGT_CUDA(cudaMemcpyAsync(sizes.data(), d_sizes, sizeof(int64_t) * npix, cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    const mgt_status st = check_device_error(m, s);
    if (st != MGT_OK) {
        cudaFreeAsync(d_lens, s);
        cudaFreeAsync(d_sizes, s);
        cudaFreeAsync(tmp, s);
        return st;
    }
    MGT_CUDA(cudaMalloc(&g.d_pts, sizeof(int32_t) * (total > 0 ? total : 1)));
    im.pts = g.d_pts;
    k_walk<kWalkImgFill><<<ceil_div(2 * npix * 16, kWalkThreads), kWalkThreads, 0, s>>>(a, d_lens, nullptr, nullptr, 0, 0, nullptr,
                                                                      nullptr, nullptr, 0.0f, 0, nullptr, m->d_err, im);
    MGT_LAUNCH_CHECK("k_walk<image fill>");
    k_img_place_anchor<<<ceil_div(npix, 256), 256, 0, s>>>(npix, d_lens, g.d_off, g.d_anchor, g.d_pts);
    MGT_LAUNCH_CHECK("k_img_place_anchor");
    MGT_CUDA(cudaFreeAsync(d_lens, s));
    MGT_CUDA(cudaFreeAsync(d_sizes, s));
    MGT_CUDA(cudaFreeAsync(tmp, s));
    MGT_TRY_STATUS(check_device_error(m, s));
    int64_t mx = 0;
    for (int64_t v : sizes) mx = std::max(mx, v);
    g.total = total;
    g.max_len = (int32_t)mx;
    g.n[0] = n[0];
    g.n[1] = n[1];
    g.n[2] = n[2];
    g.npx = npx;
    g.npy = npy;
    g.valid = true;
    return MGT_OK;
}

}  // namespace mgt
