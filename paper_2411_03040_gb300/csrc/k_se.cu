// Statistical equilibrium: one warp per point, FP64, state reduction.
//
// Rates i -> j per point (s^-1):
//   radiative, preconditioned by the diagonal approximate Lambda operator
//   (Rybicki & Hummer 1991), J_eff = Jbar - Lambda* S_old:
//       u -> l : max(A_ul (1 - Lambda*) + B_ul J_eff, 0)
//       l -> u : max(B_lu J_eff, 0)
//   collisional: C_ul = n_coll K_ul, C_lu = C_ul (g_u/g_l) exp(-(E_u - E_l)/kT).
// The steady state sum_j n_j R_ji = n_i sum_j R_ij, normalised to n_spec, is
// found by state reduction (Grassmann, Taksar & Heyman 1985): eliminate the
// highest level first, folding the paths through it into the remaining rates,
// R_ij += R_in R_nj / S_n with S_n = sum_{j<n} R_nj; then n_0 = 1,
// n_k = sum_{i<k} n_i R_ik / S_k and normalise.  Only non-negative numbers are
// added, so populations many decades below the ground level keep full
// relative accuracy.  All warp reductions run in a fixed lane order, so the
// result is bitwise reproducible.
#include <algorithm>
#include <cstring>

#include "mgt_common.cuh"

namespace mgt {

namespace {

struct SEArgs {
    int64_t N;
    int L, M, Mpad, K;
    const double *pops_old;   // [N][L]
    const double *J, *Lst;    // [N][M]
    const double *T, *ncoll, *nspec;
    const double *line_tab;   // [8][Mpad]: nu, A, Bul, Blu, ...
    const int32_t *line_ul;   // [2][Mpad]
    const double *level_tab;  // [2][L]: E, g
    const double *Kul;        // [K]
    const int32_t *coll_ul;   // [2][K]
    const int16_t *entry;     // [3][L*L]
    double *pops_out;         // [N][L] (may be pops_old: each warp reads its row before writing it)
    double *pops_prev;        // [N][L] copy of pops_old, or NULL
    int wpb;                  // warps (points) per block
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the warp when only lanes below n hold nonzero values: the xor
// butterfly stops at the smallest power of two >= n, and every lane below n
// ends with the total (fewer FP64 additions on GB300's narrow FP64 pipe).
__device__ __forceinline__ double warp_sum_first(double v, int n)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        if (o < n) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kMaxWarpsPerBlock = 4;

// Point p, solved by one warp in its shared-memory slice sm (LL + 3L + 2 Mpad doubles).
__device__ __forceinline__ void se_point(const SEArgs &a, int64_t p, double *sm, int lane)
{
    const int L = a.L, LL = L * L;
    double *R = sm;                       // R[i*L + j]: rate i -> j
    double *Sn = R + LL;                  // [L] reciprocals of the pivots
    double *xx = Sn + L;                  // [L] unnormalised populations
    double *bz = xx + L;                  // [L] Boltzmann factors g_i exp(-(E_i - E_0)/kT)
    double *rdown = bz + L;               // [Mpad] radiative u -> l rate per line
    double *rup = rdown + a.Mpad;         // [Mpad] radiative l -> u rate per line

    const double *po = a.pops_old + p * L;
    if (a.pops_prev)
        for (int i = lane; i < L; i += 32) a.pops_prev[p * L + i] = po[i];
    const double Tp = a.T[p], nc = a.ncoll[p];
    // per-line preconditioned radiative rates
    for (int k = lane; k < a.M; k += 32) {
        const int u = a.line_ul[k], l = a.line_ul[a.Mpad + k];
        const double A = a.line_tab[a.Mpad + k], Bul = a.line_tab[2 * a.Mpad + k], Blu = a.line_tab[3 * a.Mpad + k];
        const double x_l = po[l] * Blu, x_u = po[u] * Bul;
        double net = x_l - x_u;
        const double fl = 1e-30 * (x_l + x_u);
        if (net < fl) net = fl;
        const double S_old = net > 0.0 ? po[u] * A / net : 0.0;
        const double Js = a.J[p * a.M + k], Ls = a.Lst[p * a.M + k];
        const double Jeff = Js - Ls * S_old;
        rdown[k] = fmax(A * (1.0 - Ls) + Bul * Jeff, 0.0);
        rup[k] = fmax(Blu * Jeff, 0.0);
    }
    const double *E = a.level_tab, *g = a.level_tab + L;
    const double ikT = 1.0 / (kKB * Tp);
    // one exponential per level instead of one per collisional pair: the
    // upward rate C_lu = C_ul (g_u/g_l) exp(-(E_u - E_l)/kT) = C_ul bz_u / bz_l,
    // formed with 1/bz_l from one division per level (kept in xx until the
    // populations need it; FP64 division is a long sequence on this GPU's
    // narrow FP64 pipe, and there are L^2/2 upward pairs)
    for (int i = lane; i < L; i += 32) {
        const double b = g[i] * exp(-(E[i] - E[0]) * ikT);
        bz[i] = b;
        xx[i] = b > 1e-290 ? 1.0 / b : 0.0;
    }
    __syncwarp();
    for (int e = lane; e < LL; e += 32) {
        const int i = e / L, j = e - i * L;
        double v = 0.0;
        if (i != j) {
            const int kd = a.entry[e], ku = a.entry[LL + e], kc = a.entry[2 * LL + e];
            if (kd >= 0) v += rdown[kd];
            if (ku >= 0) v += rup[ku];
            if (kc >= 0) {
                const int cu = a.coll_ul[kc], cl = a.coll_ul[a.K + kc];
                const double Cul = nc * a.Kul[kc];
                if (i == cu)
                    v += Cul;
                else if (bz[cl] > 1e-290 && bz[cu] > 1e-290)
                    v += Cul * bz[cu] * xx[cl];
                else   // a factor near the bottom of the FP64 range: the pair's own exponential
                    v += Cul * g[cu] / g[cl] * exp(-(E[cu] - E[cl]) * ikT);
            }
        }
        R[e] = v;
    }
    __syncwarp();
    // state reduction, highest level first
    for (int n = L - 1; n >= 1; --n) {
        double part = 0.0;
        for (int j = lane; j < n; j += 32) part += R[n * L + j];
        double s = warp_sum_first(part, n);
        s = s > 0.0 ? s : 1e-300;
        // one lane divides (the division is a long FP64 sequence), all read it
        double rs = 0.0;
        if (lane == 0) {
            rs = 1.0 / s;
            Sn[n] = rs;
        }
        rs = __shfl_sync(0xffffffffu, rs, 0);
        for (int j = lane; j < n; j += 32) R[n * L + j] *= rs;
        __syncwarp();
        const int nn = n * n;
        for (int e = lane; e < nn; e += 32) {
            const int i = e / n, j = e - i * n;
            R[i * L + j] += R[i * L + n] * R[n * L + j];
        }
        __syncwarp();
    }
    // back substitution n_k = sum_{i<k} n_i R_ik / S_k, column by column: lane
    // j keeps the running sums of levels j and j + 32, and once n_{k-1} is
    // known every lane adds its term to the levels above it (one FP64
    // multiply-add per lane and level instead of a warp sum per level)
    double acc0 = 0.0, acc1 = 0.0;
    if (lane == 0) xx[0] = 1.0;
    double xprev = 1.0;                   // n_0
    for (int k = 1; k < L; ++k) {
        const int i = k - 1;              // n_i is known: add n_i R_ij to every level j > i
        if (lane > i && lane < L) acc0 += xprev * R[i * L + lane];
        if (lane + 32 > i && lane + 32 < L) acc1 += xprev * R[i * L + lane + 32];
        // n_k = acc[k] / S_k from the lane that holds level k
        const double a = k < 32 ? acc0 : acc1;
        double nk = 0.0;
        if ((k & 31) == lane) {
            nk = a * Sn[k];
            xx[k] = nk;
        }
        xprev = __shfl_sync(0xffffffffu, nk, k & 31);
    }
    __syncwarp();
    double part = 0.0;
    for (int i = lane; i < L; i += 32) part += xx[i];
    const double tot = warp_sum(part);
    const double f = a.nspec[p] / tot;
    for (int i = lane; i < L; i += 32) a.pops_out[p * L + i] = xx[i] * f;
}

__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock) k_se(SEArgs a)
{
    extern __shared__ __align__(16) double sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per_warp = a.L * a.L + 3 * a.L + 2 * a.Mpad;
    const int64_t p = (int64_t)blockIdx.x * a.wpb + warp;
    if (p >= a.N) return;                 // whole warp leaves together
    se_point(a, p, sm + warp * per_warp, lane);
}

// Many models in one launch, kMaxWarpsPerBlock points of one model per CTA:
// blk_end[i] is one past the last CTA of model i.
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock) k_se_batch(const SEArgs *__restrict__ args,
                                                                     const int64_t *__restrict__ blk_end, int n_models)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ SEArgs sa;
    __shared__ int64_t s_first;
    if (threadIdx.x == 0) {
        const int64_t b = blockIdx.x;
        int lo = 0, hi = n_models - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (blk_end[mid] > b) hi = mid; else lo = mid + 1;
        }
        sa = args[lo];
        s_first = lo > 0 ? blk_end[lo - 1] : 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per_warp = sa.L * sa.L + 3 * sa.L + 2 * sa.Mpad;
    const int64_t p = ((int64_t)blockIdx.x - s_first) * kMaxWarpsPerBlock + warp;
    if (p >= sa.N) return;
    se_point(sa, p, sm + warp * per_warp, lane);
}

SEArgs fill_se_args(const mgt_model *m)
{
    SEArgs a{};
    a.N = m->N;
    a.L = m->L;
    a.M = m->M;
    a.Mpad = m->Mpad;
    a.K = m->K;
    a.pops_old = m->d_pops_prev;
    a.J = m->d_J;
    a.Lst = m->d_Lst;
    a.T = m->d_temp;
    a.ncoll = m->d_ncoll;
    a.nspec = m->d_nspec;
    a.line_tab = m->d_line_tab;
    a.line_ul = m->d_line_ul;
    a.level_tab = m->d_level_tab;
    a.Kul = m->d_coll_tab;
    a.coll_ul = m->d_coll_ul;
    a.entry = m->d_entry;
    a.pops_out = m->d_pops;
    return a;
}

size_t se_warp_bytes(const mgt_model *m) { return sizeof(double) * ((size_t)m->L * m->L + 3 * m->L + 2 * m->Mpad); }

}  // namespace

mgt_status launch_stat_eq(mgt_model *m, cudaStream_t s)
{
    SEArgs a = fill_se_args(m);
    const size_t per_warp = sizeof(double) * ((size_t)m->L * m->L + 3 * m->L + 2 * m->Mpad);
    const size_t max_smem = 227 * 1024;
    int wpb = (int)std::min<size_t>(kMaxWarpsPerBlock, max_smem / per_warp);
    if (wpb < 1) return set_error(MGT_ERR_ARG, "statistical equilibrium: too many levels/lines for shared memory");
    a.wpb = wpb;
    const size_t smem = per_warp * wpb;
    MGT_TRY_STATUS(raise_smem_limit((const void *)k_se, smem));
    {
        MGT_KTIMER("k_se", s);
        k_se<<<ceil_div(m->N, wpb), 32 * wpb, smem, s>>>(a);
    }
    MGT_LAUNCH_CHECK("k_se");
    return MGT_OK;
}

// Batched statistical equilibrium: the model's arguments with the previous
// populations read from and written back to d_pops (the copy for Ng made by
// the same warp into d_pops_prev).
size_t se_args_bytes() { return sizeof(SEArgs); }

mgt_status se_batch_args(const mgt_model *m, void *args, int64_t *blocks, size_t *smem)
{
    SEArgs a = fill_se_args(m);
    a.pops_old = m->d_pops;
    a.pops_prev = m->d_pops_prev;
    a.wpb = kMaxWarpsPerBlock;
    *smem = se_warp_bytes(m) * kMaxWarpsPerBlock;
    if (*smem > 227 * 1024) return set_error(MGT_ERR_ARG, "batched statistical equilibrium: too many levels");
    *blocks = (m->N + kMaxWarpsPerBlock - 1) / kMaxWarpsPerBlock;
    std::memcpy(args, &a, sizeof a);
    return MGT_OK;
}

mgt_status se_batch_prepare(size_t smem)
{
    MGT_TRY_STATUS(raise_smem_limit((const void *)k_se_batch, smem));
    return MGT_OK;
}

mgt_status se_batch_launch(const void *d_args, const int64_t *d_blk_end, int n_models, int64_t n_blocks, size_t smem,
                           cudaStream_t s)
{
    k_se_batch<<<(unsigned)n_blocks, 32 * kMaxWarpsPerBlock, smem, s>>>(static_cast<const SEArgs *>(d_args), d_blk_end,
                                                                       n_models);
    MGT_LAUNCH_CHECK("k_se_batch");
    return MGT_OK;
}

}  // namespace mgt
