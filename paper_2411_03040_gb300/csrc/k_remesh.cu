// Recursive re-meshing of a point cloud (Sec. 4.1): divide a box into 8 equal
// parts while the variation 2 (rho_max - rho_min)/(rho_max + rho_min) of the
// tracer inside it exceeds r_max and the recursion level is below l, crop
// each non-empty part to the bounding box of its points, and represent every
// final box by its centre; then add evenly spaced boundary points on the
// surface of the outermost box.
//
// GPU form: the recursion runs level by level.  The points of every open box
// form one contiguous segment of a permutation; per level one block per box
// reduces the box's bounds and tracer range (FP64 minima and maxima, exact in
// any order), the boxes that divide count their points per octant and scatter
// them into the children's segments, and the children (non-empty octants, in
// parent order then octant order) are the next level's boxes.  Final boxes
// are written level by level in box order.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mgt_common.cuh"

namespace mgt {

namespace {

constexpr int kRmThreads = 256;

struct BoxStats {
    double lo[3], hi[3], rmin, rmax;
};

__device__ __forceinline__ double warp_min_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One block per box: bounds and tracer range over the box's segment.
__global__ void __launch_bounds__(kRmThreads) k_rm_stats(const double *__restrict__ pos, const double *__restrict__ rho,
                                                         const int32_t *__restrict__ perm,
                                                         const int64_t *__restrict__ seg_start,
                                                         const int64_t *__restrict__ seg_len, BoxStats *__restrict__ st)
{
    __shared__ double red[8][kRmThreads / 32];
    const int64_t b = blockIdx.x;
    const int64_t s0 = seg_start[b], n = seg_len[b];
    double v[8] = {1e308, 1e308, 1e308, -1e308, -1e308, -1e308, 1e308, -1e308};   // lo xyz, hi xyz, rmin, rmax
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = perm[s0 + i];
        for (int d = 0; d < 3; ++d) {
            const double x = pos[3 * p + d];
            v[d] = fmin(v[d], x);
            v[3 + d] = fmax(v[3 + d], x);
        }
        const double r = rho[p];
        v[6] = fmin(v[6], r);
        v[7] = fmax(v[7], r);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool is_min = k < 3 || k == 6;
        const double w = is_min ? warp_min_d(v[k]) : warp_max_d(v[k]);
        if (lane == 0) red[k][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        const bool is_min = k < 3 || k == 6;
        double w = red[k][0];
        for (int j = 1; j < (int)(blockDim.x / 32); ++j) w = is_min ? fmin(w, red[k][j]) : fmax(w, red[k][j]);
        double *o = &st[b].lo[0];
        o[k] = w;   // lo[3], hi[3], rmin, rmax are contiguous
    }
}

// Division decision and the box's octant counts (0 for boxes that stay).
__global__ void __launch_bounds__(kRmThreads) k_rm_count(const double *__restrict__ pos, const int32_t *__restrict__ perm,
                                                         const int64_t *__restrict__ seg_start,
                                                         const int64_t *__restrict__ seg_len,
                                                         const BoxStats *__restrict__ st, double r_max, int level,
                                                         int max_level, uint8_t *__restrict__ divide,
                                                         int64_t *__restrict__ counts)
{
    __shared__ unsigned long long c[8];
    const int64_t b = blockIdx.x;
    const BoxStats s = st[b];
    const double var = 2.0 * ((s.rmax - s.rmin) / (s.rmax + s.rmin));
    const bool dv = level < max_level && var > r_max;
    if (threadIdx.x < 8) c[threadIdx.x] = 0;
    __syncthreads();
    if (dv) {
        double mid[3];
        for (int d = 0; d < 3; ++d) mid[d] = (s.lo[d] + s.hi[d]) * 0.5;
        const int64_t s0 = seg_start[b], n = seg_len[b];
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const int64_t p = perm[s0 + i];
            int o = 0;
            for (int d = 0; d < 3; ++d) o |= (pos[3 * p + d] >= mid[d] ? 1 : 0) << d;
            atomicAdd(&c[o], 1ULL);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) divide[b] = dv ? 1 : 0;
    if (threadIdx.x < 8) counts[8 * b + threadIdx.x] = (int64_t)c[threadIdx.x];
}

// Scatter a dividing box's points into its children's segments (at the same
// place in the permutation: children are consecutive inside the parent).
__global__ void __launch_bounds__(kRmThreads) k_rm_scatter(const double *__restrict__ pos, const int32_t *__restrict__ perm,
                                                           int32_t *__restrict__ perm_out,
                                                           const int64_t *__restrict__ seg_start,
                                                           const int64_t *__restrict__ seg_len,
                                                           const BoxStats *__restrict__ st,
                                                           const uint8_t *__restrict__ divide,
                                                           const int64_t *__restrict__ counts)
{
    __shared__ unsigned long long cur[8];
    const int64_t b = blockIdx.x;
    const int64_t s0 = seg_start[b], n = seg_len[b];
    if (!divide[b]) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm_out[s0 + i] = perm[s0 + i];
        return;
    }
    if (threadIdx.x == 0) {
        unsigned long long a = 0;
        for (int o = 0; o < 8; ++o) {
            cur[o] = a;
            a += (unsigned long long)counts[8 * b + o];
        }
    }
    __syncthreads();
    const BoxStats s = st[b];
    double mid[3];
    for (int d = 0; d < 3; ++d) mid[d] = (s.lo[d] + s.hi[d]) * 0.5;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = perm[s0 + i];
        int o = 0;
        for (int d = 0; d < 3; ++d) o |= (pos[3 * p + d] >= mid[d] ? 1 : 0) << d;
        const unsigned long long at = atomicAdd(&cur[o], 1ULL);
        perm_out[s0 + (int64_t)at] = (int32_t)p;
    }
}

// Final boxes of this level -> centres; children of dividing boxes -> the
// next level's segments.  leaf_at / child_at are exclusive scans of the flags.
__global__ void k_rm_emit(int64_t nb, const int64_t *__restrict__ seg_start, const BoxStats *__restrict__ st,
                          const uint8_t *__restrict__ divide, const int64_t *__restrict__ counts,
                          const int64_t *__restrict__ leaf_at, int64_t leaf_base, double *__restrict__ out,
                          const int64_t *__restrict__ child_at, int64_t *__restrict__ nstart, int64_t *__restrict__ nlen)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const BoxStats s = st[b];
    if (!divide[b]) {
        double *o = out + 3 * (leaf_base + leaf_at[b]);
        for (int d = 0; d < 3; ++d) o[d] = (s.lo[d] + s.hi[d]) * 0.5;
        return;
    }
    int64_t a = seg_start[b], k = child_at[b];
    for (int o = 0; o < 8; ++o) {
        const int64_t c = counts[8 * b + o];
        if (c > 0) {
            nstart[k] = a;
            nlen[k] = c;
            ++k;
        }
        a += c;
    }
}

__global__ void k_rm_flags(int64_t nb, const uint8_t *__restrict__ divide, const int64_t *__restrict__ counts,
                           int64_t *__restrict__ leaf_flag, int64_t *__restrict__ child_n)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    leaf_flag[b] = divide[b] ? 0 : 1;
    int64_t c = 0;
    if (divide[b])
        for (int o = 0; o < 8; ++o) c += counts[8 * b + o] > 0 ? 1 : 0;
    child_n[b] = c;
}

__global__ void k_rm_iota(int64_t n, int32_t *__restrict__ perm)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int32_t)i;
}

}  // namespace

}  // namespace mgt

using namespace mgt;

extern "C" mgt_status mgt_remesh(int64_t n_points, const double *pos, const double *rho, double r_max,
                                 int32_t max_level, int32_t n_side, double *out_pos, uint8_t *out_boundary,
                                 int64_t capacity, int64_t *n_out, void *stream)
{
    MGT_RANGE("mgt_remesh");
    if (n_points < 1 || n_points >= ((int64_t)1 << 31)) return set_error(MGT_ERR_ARG, "n_points must be 1..2^31-1");
    if (!pos || !rho || !n_out) return set_error(MGT_ERR_ARG, "pos, rho and n_out are required");
    if (!(r_max >= 0.0) || !std::isfinite(r_max)) return set_error(MGT_ERR_ARG, "r_max must be finite and >= 0");
    if (max_level < 0 || max_level > 30) return set_error(MGT_ERR_ARG, "max_level must be 0..30");
    if (n_side < 2 || n_side > 1024) return set_error(MGT_ERR_ARG, "n_side must be 2..1024");
    for (int64_t i = 0; i < n_points; ++i) {
        if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return set_error(MGT_ERR_ARG, "rho must be finite and > 0");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(pos[3 * i + d])) return set_error(MGT_ERR_ARG, "positions must be finite");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = n_points;
    double *d_pos = nullptr, *d_rho = nullptr, *d_out = nullptr;
    int32_t *perm = nullptr, *perm2 = nullptr;
    int64_t *start = nullptr, *len = nullptr, *nstart = nullptr, *nlen = nullptr, *counts = nullptr;
    int64_t *leaf_flag = nullptr, *leaf_at = nullptr, *child_n = nullptr, *child_at = nullptr;
    BoxStats *st = nullptr;
    uint8_t *divide = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    std::vector<void *> owned;
    auto dev = [&](auto **p, size_t n) -> cudaError_t {
        cudaError_t e = cudaMallocAsync((void **)p, sizeof(**p) * (n ? n : 1), s);
        if (e == cudaSuccess) owned.push_back((void *)*p);
        return e;
    };
    struct Release {
        std::vector<void *> &v;
        cudaStream_t s;
        ~Release()
        {
            for (void *p : v) cudaFreeAsync(p, s);
        }
    } release{owned, s};
    MGT_CUDA(dev(&d_pos, 3 * N));
    MGT_CUDA(dev(&d_rho, N));
    MGT_CUDA(dev(&d_out, 3 * N));
    MGT_CUDA(dev(&perm, N));
    MGT_CUDA(dev(&perm2, N));
    for (int64_t **p : {&start, &len, &nstart, &nlen, &leaf_flag, &leaf_at, &child_n, &child_at}) MGT_CUDA(dev(p, N + 1));
    MGT_CUDA(dev(&counts, 8 * N));
    MGT_CUDA(dev(&st, N));
    MGT_CUDA(dev(&divide, N));
    MGT_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, leaf_flag, leaf_at, N + 1, s));
    MGT_CUDA(dev((unsigned char **)&tmp, tmp_bytes));
    MGT_CUDA(cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    MGT_CUDA(cudaMemcpyAsync(d_rho, rho, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    k_rm_iota<<<ceil_div(N, 256), 256, 0, s>>>(N, perm);
    MGT_LAUNCH_CHECK("k_rm_iota");
    const int64_t zero = 0;
    MGT_CUDA(cudaMemcpyAsync(start, &zero, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MGT_CUDA(cudaMemcpyAsync(len, &N, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    int64_t nb = 1, n_leaves = 0;
    BoxStats root{};
    for (int level = 0; nb > 0; ++level) {
        k_rm_stats<<<(unsigned)nb, kRmThreads, 0, s>>>(d_pos, d_rho, perm, start, len, st);
        MGT_LAUNCH_CHECK("k_rm_stats");
        if (level == 0) MGT_CUDA(cudaMemcpyAsync(&root, st, sizeof(BoxStats), cudaMemcpyDeviceToHost, s));
        k_rm_count<<<(unsigned)nb, kRmThreads, 0, s>>>(d_pos, perm, start, len, st, r_max, level, max_level, divide,
                                                        counts);
        MGT_LAUNCH_CHECK("k_rm_count");
        k_rm_scatter<<<(unsigned)nb, kRmThreads, 0, s>>>(d_pos, perm, perm2, start, len, st, divide, counts);
        MGT_LAUNCH_CHECK("k_rm_scatter");
        std::swap(perm, perm2);
        k_rm_flags<<<ceil_div(nb, 256), 256, 0, s>>>(nb, divide, counts, leaf_flag, child_n);
        MGT_LAUNCH_CHECK("k_rm_flags");
        MGT_CUDA(cudaMemsetAsync(leaf_flag + nb, 0, sizeof(int64_t), s));
        MGT_CUDA(cudaMemsetAsync(child_n + nb, 0, sizeof(int64_t), s));
        MGT_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, leaf_flag, leaf_at, nb + 1, s));
        MGT_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, child_n, child_at, nb + 1, s));
        k_rm_emit<<<ceil_div(nb, 256), 256, 0, s>>>(nb, start, st, divide, counts, leaf_at, n_leaves, d_out, child_at,
                                                    nstart, nlen);
        MGT_LAUNCH_CHECK("k_rm_emit");
        int64_t nl = 0, nc = 0;
        MGT_CUDA(cudaMemcpyAsync(&nl, leaf_at + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        MGT_CUDA(cudaMemcpyAsync(&nc, child_at + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        MGT_CUDA(cudaStreamSynchronize(s));
        n_leaves += nl;
        nb = nc;
        std::swap(start, nstart);
        std::swap(len, nlen);
    }
    // evenly spaced boundary points: the surface nodes of the n_side^3 lattice
    // over the outermost box
    std::vector<double> bnd;
    for (int i = 0; i < n_side; ++i)
        for (int j = 0; j < n_side; ++j)
            for (int k = 0; k < n_side; ++k) {
                if (!(i == 0 || i == n_side - 1 || j == 0 || j == n_side - 1 || k == 0 || k == n_side - 1)) continue;
                const int ijk[3] = {i, j, k};
                for (int d = 0; d < 3; ++d)
                    bnd.push_back(root.lo[d] + (double)ijk[d] / (n_side - 1) * (root.hi[d] - root.lo[d]));
            }
    const int64_t nbnd = (int64_t)bnd.size() / 3;
    *n_out = n_leaves + nbnd;
    if (!out_pos) return MGT_OK;
    if (capacity < *n_out) return set_error(MGT_ERR_ARG, "capacity is below the number of output points (see n_out)");
    MGT_CUDA(cudaMemcpyAsync(out_pos, d_out, sizeof(double) * 3 * n_leaves, cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    std::copy(bnd.begin(), bnd.end(), out_pos + 3 * n_leaves);
    if (out_boundary) {
        std::fill(out_boundary, out_boundary + n_leaves, (uint8_t)0);
        std::fill(out_boundary + n_leaves, out_boundary + *n_out, (uint8_t)1);
    }
    return MGT_OK;
}
