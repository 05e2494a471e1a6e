// Ng extrapolation of caller-held iterates with no device allocation
// (mgt_ng_extrapolate_noalloc).
//
// The arithmetic is that of mgt_ng_accelerate's prediction: residuals
// r_k = x_{k+1} - x_k, Gram matrix G = R R^T built one row at a time (block
// partials in a fixed order, then one block), c = G^-1 1 / (1^T G^-1 1) from
// an LU solve of G / tr G on the host, prediction sum_k c_k x_{k+1}.
//
// Working memory lives in one file-scope static device array instead of
// cudaMalloc'd buffers.  In host code the array's name is only a host-side
// stand-in, so each device's address of it is looked up once with
// cudaGetSymbolAddress (with that device current; the first call on the device
// does this) and passed to the kernels.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "mgt_common.cuh"

namespace mgt {

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1216;             // 8 x 152 SMs, as the model's Ng kernels
constexpr int kNaMaxRes = kMaxNgHist;          // residuals per call
static_assert(MGT_NG_NOALLOC_MAX_ITERATES == kNaMaxRes + 1, "header limit and scratch size disagree");

// Scratch layout, in doubles:
//   [0, kNaMaxBlocks * kNaMaxRes)     block partials of one Gram row
//   [kGramOff, kGramOff + kNaMaxRes^2) the reduced Gram matrix (row-major)
//   kCountOff                          count of negative prediction entries (u64 bits)
constexpr int kGramOff = kNaMaxBlocks * kNaMaxRes;
constexpr int kCountOff = kGramOff + kNaMaxRes * kNaMaxRes;
constexpr int kScratchDoubles = kCountOff + 32;   // padded to a 256-byte multiple
static_assert(kScratchDoubles * sizeof(double) == MGT_NG_NOALLOC_SCRATCH_BYTES, "scratch size");

static __device__ __align__(256) double g_ng_noalloc_scratch[kScratchDoubles];

// Row i of the Gram matrix: partials[b][k] = sum over the block's elements of
// r_i r_k for k <= i (the same per-thread and per-block order as the model's
// push kernel, so equal grids give equal sums).
__global__ void __launch_bounds__(kNaThreads) k_ng_na_gram_row(int64_t len, const double *__restrict__ X, int i,
                                                               double *__restrict__ partials)
{
    double acc[kNaMaxRes];
#pragma unroll
    for (int k = 0; k < kNaMaxRes; ++k) acc[k] = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const double r = X[(int64_t)(i + 1) * len + e] - X[(int64_t)i * len + e];
#pragma unroll
        for (int k = 0; k < kNaMaxRes; ++k)
            if (k < i) acc[k] += r * (X[(int64_t)(k + 1) * len + e] - X[(int64_t)k * len + e]);
#pragma unroll
        for (int k = 0; k < kNaMaxRes; ++k)
            if (k == i) acc[k] += r * r;
    }
    __shared__ double red[kNaThreads];
    for (int k = 0; k <= i; ++k) {
        double v = 0.0;
#pragma unroll
        for (int kk = 0; kk < kNaMaxRes; ++kk)
            if (kk == k) v = acc[kk];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int s = kNaThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kNaMaxRes + k] = red[0];
        __syncthreads();
    }
}

// G[i][k] = G[k][i] = sum_b partials[b][k] in block order, k <= i.
__global__ void k_ng_na_gram_finish(int nblocks, int i, const double *__restrict__ partials, double *__restrict__ G)
{
    const int k = threadIdx.x;
    if (k > i) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * kNaMaxRes + k];
    G[i * kNaMaxRes + k] = s;
    G[k * kNaMaxRes + i] = s;
}

struct NaCoef {
    double c[kNaMaxRes];
};

// out[e] = sum_k c_k x_{k+1}[e]; negative entries are counted.
__global__ void __launch_bounds__(kNaThreads) k_ng_na_predict(int64_t len, const double *__restrict__ X, int nc,
                                                              NaCoef cf, double *__restrict__ out,
                                                              unsigned long long *__restrict__ n_neg)
{
    unsigned long long neg = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0;
        for (int k = 0; k < nc; ++k) x += cf.c[k] * X[(int64_t)(k + 1) * len + e];
        out[e] = x;
        neg += x < 0.0;
    }
    if (neg) atomicAdd(n_neg, neg);
}

// Per-device address of the scratch array.  The lookup runs with the device
// current and is cached only once it has succeeded: a failed lookup (a
// transient error) is retried by the next call on that device.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double *g_na_ptr[kNaMaxDevices];

mgt_status scratch_address(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_ng_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_ng_noalloc_scratch)");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return MGT_OK;
}

}  // namespace

}  // namespace mgt

using namespace mgt;

extern "C" mgt_status mgt_ng_extrapolate_noalloc(int32_t n_iterates, const double *iterates, int64_t len,
                                                 double *prediction, double *coef, int64_t *n_negative, void *stream)
{
    if (n_iterates < 2 || n_iterates > MGT_NG_NOALLOC_MAX_ITERATES)
        return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: n_iterates must be 2.." +
                                          std::to_string(MGT_NG_NOALLOC_MAX_ITERATES) + " (the static scratch "
                                          "holds a Gram matrix of at most " + std::to_string(kNaMaxRes) +
                                          " residuals), got " + std::to_string(n_iterates));
    if (len < 1) return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: len must be >= 1");
    if (!iterates || !prediction) return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: null pointer");
    int dev = 0;
    MGT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: device id too large");
    for (const void *p : {(const void *)iterates, (const void *)prediction}) {
        cudaPointerAttributes at{};
        MGT_CUDA(cudaPointerGetAttributes(&at, p));
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: iterates and prediction must be device memory");
        if (at.device != dev)
            return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: buffers are not on the current device");
    }
    {
        // the prediction may not overlap any iterate (it is written while they are read)
        const char *pb = reinterpret_cast<const char *>(prediction), *ib = reinterpret_cast<const char *>(iterates);
        const uint64_t pn = (uint64_t)len * sizeof(double), in = (uint64_t)n_iterates * pn;
        if ((uint64_t)(uintptr_t)pb < (uint64_t)(uintptr_t)ib + in && (uint64_t)(uintptr_t)ib < (uint64_t)(uintptr_t)pb + pn)
            return set_error(MGT_ERR_ARG, "mgt_ng_extrapolate_noalloc: prediction overlaps the iterates");
    }
    double *scratch = nullptr;
    MGT_TRY_STATUS(scratch_address(dev, &scratch));
    double *partials = scratch, *G = scratch + kGramOff;
    unsigned long long *count = reinterpret_cast<unsigned long long *>(scratch + kCountOff);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const int nres = n_iterates - 1;
    int64_t b = (len + kNaThreads - 1) / kNaThreads;
    const int grid = (int)(b < kNaMaxBlocks ? b : kNaMaxBlocks);
    for (int i = 0; i < nres; ++i) {
        k_ng_na_gram_row<<<grid, kNaThreads, 0, s>>>(len, iterates, i, partials);
        MGT_LAUNCH_CHECK("k_ng_na_gram_row");
        k_ng_na_gram_finish<<<1, 32, 0, s>>>(grid, i, partials, G);
        MGT_LAUNCH_CHECK("k_ng_na_gram_finish");
    }
    double Gh[kNaMaxRes * kNaMaxRes];
    MGT_CUDA(cudaMemcpyAsync(Gh, G, sizeof(double) * nres * kNaMaxRes, cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    NaCoef cf{};
    if (!ng_solve_coefficients(Gh, kNaMaxRes, nres, cf.c))
        return set_error(MGT_ERR_SINGULAR, "mgt_ng_extrapolate_noalloc: the residual Gram matrix is singular");
    MGT_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    k_ng_na_predict<<<grid, kNaThreads, 0, s>>>(len, iterates, nres, cf, prediction, count);
    MGT_LAUNCH_CHECK("k_ng_na_predict");
    unsigned long long neg = 0;
    MGT_CUDA(cudaMemcpyAsync(&neg, count, sizeof(neg), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    if (coef)
        for (int k = 0; k < nres; ++k) coef[k] = cf.c[k];
    if (n_negative) *n_negative = (int64_t)neg;
    return MGT_OK;
}
