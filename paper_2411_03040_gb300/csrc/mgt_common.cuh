// Internal declarations of the GB300 line-transfer library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "../../include/magritte_gpu.h"

namespace mgt {

// Physical constants (CODATA 2018, exact SI definitions).
constexpr double kH = 6.62607015e-34;
constexpr double kC = 299792458.0;
constexpr double kKB = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;

// Device error word codes (first error wins).
enum DevErr : int { kDevOk = 0, kDevBounds = 1, kDevTimeout = 2 };

constexpr int kMaxQuad = 64;
constexpr int kMaxLevels = 64;
constexpr int kMaxNgHist = 16;

// One traced step in the single-precision layout, 16 bytes:
//   x: point index c_k
//   y: |x_{c_k} - x_{c_{k-1}}| in model length units (f32 bits)
//   z: beta_k = n.(v_{c_k} - v_o)/c (f32 bits)
//   w: (beta_k - beta_{k-1}) / wbar_k (f32 bits), wbar the segment's averaged
//      relative line width (dimensionless, delta nu / nu)
// c_0 = o, beta_0 = 0.
using Step32 = int4;

// Packed neighbour entry of the ray walk, 32 bytes (two float4):
//   {hx, hy, hz, lx}, {ly, lz, word, off}
// h + l = the neighbour's position times pos_scale (float hi + lo); word holds
// the neighbour's index (bits 0-29), a last-entry-of-this-row flag (bit 30)
// and the neighbour's boundary flag (bit 31); off is the first entry of the
// neighbour's own row.  A point without neighbours has one entry with index
// kEntEmpty; 16 such entries pad the array's end.
constexpr uint32_t kEntLast = 1u << 30;
constexpr uint32_t kEntBnd = 1u << 31;
constexpr uint32_t kEntIdx = kEntLast - 1u;
constexpr uint32_t kEntEmpty = kEntIdx;

// Double-precision geometry of the same step: {dx, beta, dbeta/wbar, unused}.
struct alignas(32) Step64 {
    double dx, beta, dbw, pad;
};

// Pixel rays of the last image geometry (direction and pixel counts).
struct ImageGeom {
    bool valid = false;
    double n[3] = {0, 0, 0};
    int32_t npx = 0, npy = 0;
    int64_t total = 0;                  // points over all pixel rays
    int32_t max_len = 0;                // longest pixel ray (points)
    double *d_ref = nullptr;            // [npix][3] pixel reference points
    int32_t *d_anchor = nullptr;        // [npix]
    int64_t *d_off = nullptr;           // [npix+1]
    int32_t *d_pts = nullptr;           // [total] far end first
};

// What a started Ng step still has to do (see ng_step).
struct NgPending {
    int phase = 0;          // 0 idle, 1 push in flight, 2 prediction in flight, 3 prediction singular
    bool none = false;      // mode NONE: only the maximum change
    int mh = 0, snew = -1;  // history length before the push, slot of the new iterate
    int mcount = 0;         // history length after the push
    double maxrel = 0.0, mr_pred = 0.0;
    bool negative = false;
    int accepted = 0;
};

struct NgState {
    mgt_ng_opts opts{MGT_NG_NONE, 4, 8};
    int n_slots = 0;
    std::vector<int> hist;              // slot ids, oldest first
    std::vector<double> G;              // Gram of residuals, kMaxNgHist^2 (row-major)
    int pred_slot = -1, prev_pred_slot = -1;
    bool have_prev_pred = false;
    double *d_slots = nullptr;          // [n_slots][N*L]
    double *d_partials = nullptr;       // block partials of the reductions
    double *d_red = nullptr;            // reduced values (dots, maxrel, negatives)
    double *h_red = nullptr;            // pinned host copy
    size_t partial_cap = 0;
    NgPending pend;
};

}  // namespace mgt

struct mgt_model {
    int device = 0;
    int64_t N = 0;
    int32_t R = 0, P = 0, Q = 0, L = 0, M = 0, Mpad = 0, K = 0, n_boundary = 0;
    int64_t nnz = 0;
    double mol_mass = 0, T_bg = 0, L_unit = 1.0;
    mgt_solve_opts opts{0.35, 0, 0, 0, 0, 0};

    // host copies of the small tables
    std::vector<double> energy, g, A, freq, Kul;
    std::vector<int32_t> up, lo, cup, clo;
    std::vector<int32_t> pairs;                // [P][2] (r, rb)
    std::vector<double> xq, wq;                // Gauss-Hermite nodes / normalised weights
    std::vector<double> nbg_line, hnu_kTbg, U_line;  // per padded line

    // device: per point
    double *d_pos = nullptr, *d_vel = nullptr, *d_temp = nullptr, *d_vturb2 = nullptr;
    double *d_ncoll = nullptr, *d_nspec = nullptr, *d_w64 = nullptr;
    float2 *d_w32 = nullptr;                   // {w, 1/w}
    float *d_dxmax = nullptr;                  // [N] longest graph edge at each point, in length units (rounded up)
    int32_t *d_nbr_off = nullptr, *d_nbrs = nullptr;
    double *d_nbr_pos = nullptr;               // [nnz][3] position of each neighbour entry
    float4 *d_ent = nullptr;                   // packed neighbour rows for the walk (see WalkEntry)
    int32_t *d_ent_off = nullptr;              // [N] first packed entry of each point's row
    int64_t n_ent = 0;                         // packed entries, including the 16 pad entries
    float *d_pos_hl = nullptr;                 // [N][6] positions times pos_scale, float hi + lo
    float *d_vel_hl = nullptr;                 // [N][6] velocities / c, float hi + lo
    float4 *d_dirs32 = nullptr;                // [R] directions in FP32 {n0, n1, n2, 0}
    double pos_scale = 1.0;                    // power of two near 1 / (largest coordinate)
    float pos_slack = 0.0f;                    // bound on |x pos_scale - (hi + lo)|
    int32_t *d_order = nullptr;                // [N] points in Morton (Z-curve) order
    uint8_t *d_bnd = nullptr;
    double *d_dirs = nullptr;
    int2 *d_pairs = nullptr;
    // device: per line / level tables
    double *d_xq = nullptr, *d_wq = nullptr;
    double *d_line_tab = nullptr;              // [8][Mpad]: nu, A, Bul, Blu, nbgmax, hnu_kTbg, U, unused
    int32_t *d_line_ul = nullptr;              // [2][Mpad]: up, lo (-1 for padding)
    double *d_level_tab = nullptr;             // [2][L]: energy, g
    double *d_coll_tab = nullptr;              // [K]: K_ul
    int32_t *d_coll_ul = nullptr;              // [2][K]
    int16_t *d_entry = nullptr;                // [3][L*L]: radiative-down line, radiative-up line, collision
    // device: state
    double *d_pops = nullptr, *d_pops_prev = nullptr;   // [N][L]
    float *d_line32 = nullptr;                 // [N][row_stride32] chi~', S', w, 1/w, 0, 0
    double *d_line64 = nullptr;                // [N][row_stride64] chi~', S', w, 1/w
    double *d_J = nullptr, *d_Lst = nullptr;   // [N][M]
    int *d_err = nullptr;                      // [4]
    int *d_range_bad = nullptr;                // set by the line data when a point is outside the two-row range
    unsigned long long *d_count = nullptr;     // [4] counters (opacity floors, stalls)
    // rays
    int64_t *d_ray_off = nullptr;              // [R*N+1]
    mgt::Step32 *d_steps32 = nullptr;
    mgt::Step64 *d_steps64 = nullptr;
    int64_t total_steps = 0;                   // steps of the rays currently held
    int64_t steps32_cap = 0, steps64_cap = 0;  // allocated records
    int32_t rays_p0 = 0, rays_np = 0;          // pair range whose rays are held (all pairs: 0, P)
    int32_t *d_dir_map = nullptr;              // [R] walk direction -> model direction of a pair batch
    int2 *d_batch_pairs = nullptr;             // [P] the batch's pairs in walk directions
    mgt_trace_stats stats{};                   // of the last mgt_trace_rays over all pairs
    int32_t max_half = 0;
    int64_t n_stalls = 0;
    int64_t n_exact_steps = 0;
    bool traced = false, have_J = false, line_dirty = true;
    int steps_width_mode = 0, steps64_width_mode = -1;

    mgt::NgState ng;
    mgt::ImageGeom img;
};

namespace mgt {

// The library's stream-ordered pool for large temporaries (the walk scratch),
// one per device, created on first use.  Freed blocks stay reserved in the
// pool for the next trace instead of going back to the driver (mapping tens of
// GB again on every trace costs more than the walk itself); the reserve is
// released when the last model of the process is destroyed (api.cu).
mgt_status scratch_pool(cudaMemPool_t *pool);

// Per-kernel CUDA-event timing for measurement (mgt_kernel_timing): while it
// is on, a KernelTimer records an event before the launch that follows it in
// the same scope and one when the scope ends, on the launch's stream, with the
// launch's algorithmic bytes (what the kernel must read and write at least;
// 0 where the site states none).  Off by default, and skipped on a capturing
// stream.
class KernelTimer {
public:
    KernelTimer(const char *name, cudaStream_t s, double bytes = 0.0);
    ~KernelTimer();
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

private:
    const char *name_;
    cudaStream_t s_;
    double bytes_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};
#define MGT_KTIMER(name, s) ::mgt::KernelTimer mgt_ktimer_(name, s)
#define MGT_KTIMER_BYTES(name, s, bytes) ::mgt::KernelTimer mgt_ktimer_(name, s, bytes)

// error helpers (api.cu)
void note_launch();
mgt_status set_error(mgt_status s, const std::string &msg);
mgt_status cuda_status(cudaError_t e, const char *what);
mgt_status check_device_error(mgt_model *m, cudaStream_t s);

// geometry / line-data kernels (k_geom.cu)
mgt_status launch_widths(mgt_model *m, cudaStream_t s);
mgt_status launch_lte(mgt_model *m, cudaStream_t s);
mgt_status launch_line_data(mgt_model *m, cudaStream_t s);
mgt_status build_walk_tables(mgt_model *m, const double lo[3], const double hi[3], cudaStream_t s);
mgt_status trace_all(mgt_model *m, cudaStream_t s);
mgt_status trace_range(mgt_model *m, cudaStream_t s, int32_t p0, int32_t np);
mgt_status build_steps64(mgt_model *m, cudaStream_t s);

mgt_status trace_image(mgt_model *m, const double n[3], int32_t npx, int32_t npy, cudaStream_t s);
void image_free(mgt_model *m);
void image_frame(const double *pos, int64_t N, const double n[3], int32_t npx, int32_t npy, double e1[3],
                 double e2[3], std::vector<double> &ref);

// rays of every pair held and current for the model's options (api.cu)
mgt_status ensure_rays(mgt_model *m, mgt_precision p, cudaStream_t s);
void note_launches(long long n);

// formal solution (k_fs.cu)
mgt_status launch_formal_solve(mgt_model *m, mgt_precision p, cudaStream_t s, bool accumulate);
int fs_lines_per_thread(const mgt_model *m, mgt_precision p);

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least smem bytes.  It never lowers the limit, so launches of one kernel with
// different sizes (any model, any batch) all stay valid, and it calls the
// runtime only when the limit grows, so a launch prepared once makes no
// attribute call while its stream is being captured.
mgt_status raise_smem_limit(const void *func, size_t smem);

// batched launches over many models (argument tables built per model, read on
// the device by table slot; see batch.cu)
size_t fs_args_bytes();
// (fused: the model's lines fit one group, its items run with per-thread
// coefficients; lines: its lines per thread; models are launched in classes of
// equal width, fused flag and lines per thread)
mgt_status fs_batch_args(const mgt_model *m, void *args, int *threads, int64_t *items, int *fused, int *lines);
size_t fs_batch_smem(const void *args, int threads);
mgt_status fs_batch_grid(int threads, int fused, int lines, size_t smem, size_t max_smem, int *grid);
mgt_status fs_batch_launch(const void *d_args, const int64_t *d_item_end, int n_models, int64_t n_items,
                           unsigned long long *d_next, int threads, int fused, int lines, size_t smem, int grid,
                           cudaStream_t s);
// resident CTAs on the device of the model's persistent instance (0 if unknown)
int64_t fs_batch_wave(const void *args, int threads, size_t smem);
// one model's formal solution in a batch through its single-model launch
// (the automatic staged schedule: the same values as the persistent launch);
// run = false prepares it (kernel attributes) without launching
mgt_status fs_batch_solo(mgt_model *m, cudaStream_t s, bool run);
size_t se_args_bytes();
mgt_status se_batch_args(const mgt_model *m, void *args, int64_t *blocks, size_t *smem);
mgt_status se_batch_prepare(size_t smem);
mgt_status se_batch_launch(const void *d_args, const int64_t *d_blk_end, int n_models, int64_t n_blocks, size_t smem,
                           cudaStream_t s);
size_t ld_args_bytes();
mgt_status ld_batch_args(const mgt_model *m, void *args, int64_t *blocks);
mgt_status ld_batch_launch(const void *d_args, const int64_t *d_blk_end, int n_models, int64_t n_blocks,
                           cudaStream_t s);

// statistical equilibrium (k_se.cu)
mgt_status launch_stat_eq(mgt_model *m, cudaStream_t s);

// Ng (k_ng.cu)
mgt_status ng_reset(mgt_model *m, cudaStream_t s);
mgt_status ng_step(mgt_model *m, const mgt_ng_opts *o, int *accepted, double *maxrel, cudaStream_t s);
mgt_status ng_begin(mgt_model *m, const mgt_ng_opts *o, cudaStream_t s);
mgt_status ng_after_push(mgt_model *m, cudaStream_t s);
mgt_status ng_after_predict(mgt_model *m, cudaStream_t s);
void ng_free(mgt_model *m);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Ng coefficients from a Gram matrix G (n x n, row stride ld, n <= kMaxNgHist):
// (G / tr G) y = 1 by LU with partial pivoting on a copy, c = y / sum(y).
// False when the trace is not positive and finite, a pivot is exactly zero or
// the result is not finite.  Used by the model's Ng step and by the
// no-allocation entry point, so both give the same coefficients.
inline bool ng_solve_coefficients(const double *G, int ld, int n, double *c)
{
    double a[kMaxNgHist][kMaxNgHist], y[kMaxNgHist];
    if (n < 1 || n > kMaxNgHist) return false;
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += G[i * ld + i];
    if (!(tr > 0.0) || !std::isfinite(tr)) return false;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) a[i][j] = G[i * ld + j] / tr;
        y[i] = 1.0;
    }
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(a[i][k]) > std::fabs(a[piv][k])) piv = i;
        if (a[piv][k] == 0.0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(a[k][j], a[piv][j]);
            std::swap(y[k], y[piv]);
        }
        for (int i = k + 1; i < n; ++i) {
            const double f = a[i][k] / a[k][k];
            for (int j = k; j < n; ++j) a[i][j] -= f * a[k][j];
            y[i] -= f * y[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int j = i + 1; j < n; ++j) s -= a[i][j] * y[j];
        y[i] = s / a[i][i];
    }
    double sum = 0.0;
    for (int i = 0; i < n; ++i) sum += y[i];
    if (!std::isfinite(sum) || sum == 0.0) return false;
    for (int i = 0; i < n; ++i) {
        c[i] = y[i] / sum;
        if (!std::isfinite(c[i])) return false;
    }
    return true;
}

// NVTX range over one C-ABI call (visible to profilers that record NVTX, such
// as ncu's --nvtx filters; a few nanoseconds when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define MGT_RANGE(name) ::mgt::NvtxRange mgt_nvtx_range_(name)

// Per-point line-data rows, in scalars of the row's precision:
//   [0, Mpad)        chi~'  per line (zero for padding lines)
//   [Mpad, 2 Mpad)   S'     per line
//   2 Mpad, 2 Mpad+1 the point's w and 1/w; FP32 rows end with the range
//                    figure of the two-row elimination (k_fs.cu) and a zero
// Mpad is a multiple of 8, so a row is a multiple of 16 bytes (one bulk copy)
// and every group of 4 (FP32) or 2 (FP64) lines starts 16-byte aligned.
__host__ __device__ inline int row_stride32(int Mpad) { return 2 * Mpad + 4; }   // floats

// Range of the formal solution's two-row elimination (k_fs.cu): per-row half
// depths up to kTwoRowDepth and sources S' up to kTwoRowSource.  The line data
// store each point's figure G = max(chi~max dxmax / kTwoRowDepth,
// S'max / kTwoRowSource) in its FP32 row (k_geom.cu).
constexpr float kTwoRowDepth = 256.0f;                     // 2^8
constexpr float kTwoRowSource = 1.2089258196146292e24f;    // 2^80
__host__ __device__ inline int row_stride64(int Mpad) { return 2 * Mpad + 2; }   // doubles

}  // namespace mgt

#define MGT_CUDA(call)                                                      \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return ::mgt::cuda_status(e_, #call);        \
    } while (0)

#define MGT_TRY_STATUS(x)                                                   \
    do {                                                                    \
        mgt_status st_ = (x);                                               \
        if (st_ != MGT_OK) return st_;                                      \
    } while (0)

#define MGT_LAUNCH_CHECK(what)                                              \
    do {                                                                    \
        cudaError_t e_ = cudaGetLastError();                                \
        if (e_ != cudaSuccess) return ::mgt::cuda_status(e_, what);         \
        ::mgt::note_launch();                                               \
    } while (0)
