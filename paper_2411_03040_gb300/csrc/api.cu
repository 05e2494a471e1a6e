// C-ABI entry points, input validation, model set-up and the ALI driver.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "mgt_common.cuh"

namespace mgt {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

mgt_status raise_smem_limit(const void *func, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> lim;   // (kernel, device) -> limit set
    int dev = 0;
    MGT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = lim[{func, dev}];
    if (smem <= cur) return MGT_OK;
    MGT_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cur = smem;
    return MGT_OK;
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Per-kernel event timing (measurement only).  Event pairs are recorded while
// timing is on and resolved into per-name totals by mgt_kernel_times.
namespace {
struct KtRecord {
    const char *name;
    cudaEvent_t a, b;
    double bytes;
};
struct KtTotal {
    std::string name;
    long long launches;
    double ms, bytes;
};
std::mutex g_kt_mu;
std::atomic<bool> g_kt_on{false};
std::vector<KtRecord> g_kt_pending;
std::vector<cudaEvent_t> g_kt_spare;
std::vector<KtTotal> g_kt_totals;

cudaEvent_t kt_event()
{
    if (!g_kt_spare.empty()) {
        cudaEvent_t e = g_kt_spare.back();
        g_kt_spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

KernelTimer::KernelTimer(const char *name, cudaStream_t s, double bytes) : name_(name), s_(s), bytes_(bytes)
{
    if (!g_kt_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    a_ = kt_event();
    b_ = kt_event();
    if (!a_ || !b_ || cudaEventRecord(a_, s) != cudaSuccess) {
        if (a_) g_kt_spare.push_back(a_);
        if (b_) g_kt_spare.push_back(b_);
        a_ = b_ = nullptr;
    }
}

KernelTimer::~KernelTimer()
{
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    if (cudaEventRecord(b_, s_) == cudaSuccess) {
        g_kt_pending.push_back({name_, a_, b_, bytes_});
    } else {
        g_kt_spare.push_back(a_);
        g_kt_spare.push_back(b_);
    }
}

// Scratch pools, one per device, and the number of live models per device.
constexpr int kMaxPoolDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[kMaxPoolDevices];
static int g_live_models[kMaxPoolDevices];

mgt_status scratch_pool(cudaMemPool_t *pool)
{
    int dev = 0;
    MGT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxPoolDevices) return set_error(MGT_ERR_ARG, "device id too large for the scratch pool");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        MGT_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t keep = ~0ull;
        cudaError_t e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return cuda_status(e, "cudaMemPoolSetAttribute");
        }
        g_pools[dev] = p;
    }
    *pool = g_pools[dev];
    return MGT_OK;
}

static void model_born(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev >= 0 && dev < kMaxPoolDevices) ++g_live_models[dev];
}

// The last model of a device gone: give the pool's reserve back to the driver.
static void model_gone(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= kMaxPoolDevices) return;
    if (g_live_models[dev] > 0 && --g_live_models[dev] == 0 && g_pools[dev]) cudaMemPoolTrimTo(g_pools[dev], 0);
}

mgt_status set_error(mgt_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

mgt_status cuda_status(cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(e == cudaErrorMemoryAllocation ? MGT_ERR_OOM : MGT_ERR_CUDA, msg);
}

mgt_status check_device_error(mgt_model *m, cudaStream_t s)
{
    int h[4] = {0, 0, 0, 0};
    MGT_CUDA(cudaMemcpyAsync(h, m->d_err, sizeof(h), cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    if (h[0] == kDevOk) return MGT_OK;
    MGT_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int) * 4, s));
    const std::string where = " (site " + std::to_string(h[1]) + ", item " + std::to_string(h[2]) + ", step " +
                              std::to_string(h[3]) + ")";
    if (h[0] == kDevTimeout) return set_error(MGT_ERR_TIMEOUT, "a bounded device loop ran out" + where);
    return set_error(MGT_ERR_BOUNDS, "a device index check failed" + where);
}

// ---------------------------------------------------------------------------
// Gauss-Hermite nodes and weights for the weight exp(-x^2): the nodes are the
// eigenvalues of the Jacobi matrix (zero diagonal, off-diagonal sqrt(k/2)),
// found by bisection on Sturm counts; the weights are the Christoffel numbers
// 1 / sum_k p_k(x)^2 of the orthonormal Hermite polynomials
// (p_0 = pi^-1/4, x p_k = sqrt((k+1)/2) p_{k+1} + sqrt(k/2) p_{k-1}).
// Returned weights are divided by sqrt(pi), so that they sum to one.
// ---------------------------------------------------------------------------
static void gauss_hermite(int Q, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(Q, 0.0);
    w.assign(Q, 0.0);
    auto below = [&](double lam) {
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < Q; ++i) {
            const double b2 = i == 0 ? 0.0 : i / 2.0;
            d = -lam - (i == 0 ? 0.0 : b2 / d);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++cnt;
        }
        return cnt;
    };
    const double bound = std::sqrt(2.0 * Q + 1.0) + 1.0;
    for (int k = 0; k < Q; ++k) {
        double lo = -bound, hi = bound;
        for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (below(mid) > k)
                hi = mid;
            else
                lo = mid;
        }
        x[k] = 0.5 * (lo + hi);
    }
    // exact symmetry of the node set
    for (int k = 0; k < Q / 2; ++k) {
        const double v = 0.5 * (x[Q - 1 - k] - x[k]);
        x[k] = -v;
        x[Q - 1 - k] = v;
    }
    if (Q % 2 == 1) x[Q / 2] = 0.0;
    for (int k = 0; k < Q; ++k) {
        double pm = 0.0, p = std::pow(kPi, -0.25), s = p * p;
        for (int j = 0; j + 1 < Q; ++j) {
            const double pn = (x[k] * p - std::sqrt(j / 2.0) * pm) / std::sqrt((j + 1) / 2.0);
            pm = p;
            p = pn;
            s += p * p;
        }
        w[k] = 1.0 / s / kSqrtPi;
    }
}

// Antipodal direction pairs (r, rb), n_rb = -n_r to 1e-12; false if one is missing.
static bool find_pairs(const double *dirs, int R, std::vector<int32_t> &pairs)
{
    pairs.clear();
    std::vector<char> used(R, 0);
    for (int r = 0; r < R; ++r) {
        if (used[r]) continue;
        int best = -1;
        double bd = 1e300;
        for (int q = 0; q < R; ++q) {
            if (q == r || used[q]) continue;
            const double *a = dirs + 3 * r, *b = dirs + 3 * q;
            const double e = std::sqrt((a[0] + b[0]) * (a[0] + b[0]) + (a[1] + b[1]) * (a[1] + b[1]) +
                                       (a[2] + b[2]) * (a[2] + b[2]));
            if (e < bd) {
                bd = e;
                best = q;
            }
        }
        if (best < 0 || bd > 1e-12) return false;
        used[r] = used[best] = 1;
        pairs.push_back(r);
        pairs.push_back(best);
    }
    return true;
}

static bool finite_all(const double *a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

static mgt_status validate(const mgt_model_desc *d)
{
    if (!d) return set_error(MGT_ERR_ARG, "desc is NULL");
    const int64_t N = d->n_points;
    if (N < 1) return set_error(MGT_ERR_ARG, "n_points must be >= 1");
    if (N >= (int64_t)kEntEmpty) return set_error(MGT_ERR_ARG, "n_points must be below 2^30 - 1");
    if (!d->pos || !d->vel || !d->temp || !d->vturb2 || !d->n_coll || !d->n_spec || !d->nbr_offsets || !d->nbrs ||
        !d->dirs || !d->energy_J || !d->g || !d->up || !d->lo || !d->A || !d->freq_Hz)
        return set_error(MGT_ERR_ARG, "a required input pointer is NULL");
    if (!finite_all(d->pos, 3 * N) || !finite_all(d->vel, 3 * N))
        return set_error(MGT_ERR_ARG, "positions and velocities must be finite");
    for (int64_t i = 0; i < N; ++i) {
        if (!(d->temp[i] > 0.0) || !std::isfinite(d->temp[i])) return set_error(MGT_ERR_ARG, "temperature must be > 0");
        if (!(d->vturb2[i] >= 0.0) || !std::isfinite(d->vturb2[i])) return set_error(MGT_ERR_ARG, "vturb2 must be >= 0");
        if (!(d->n_coll[i] >= 0.0) || !std::isfinite(d->n_coll[i])) return set_error(MGT_ERR_ARG, "n_coll must be >= 0");
        if (!(d->n_spec[i] > 0.0) || !std::isfinite(d->n_spec[i])) return set_error(MGT_ERR_ARG, "n_spec must be > 0");
    }
    if (d->nbr_offsets[0] != 0) return set_error(MGT_ERR_ARG, "nbr_offsets[0] must be 0");
    for (int64_t i = 0; i < N; ++i)
        if (d->nbr_offsets[i + 1] < d->nbr_offsets[i]) return set_error(MGT_ERR_ARG, "nbr_offsets must not decrease");
    const int64_t nnz = d->nbr_offsets[N];
    if (nnz + N + 16 >= ((int64_t)1 << 31)) return set_error(MGT_ERR_ARG, "too many neighbour entries");
    for (int64_t k = 0; k < nnz; ++k)
        if (d->nbrs[k] < 0 || d->nbrs[k] >= N) return set_error(MGT_ERR_ARG, "neighbour index out of range");
    if (d->n_boundary < 0 || (d->n_boundary > 0 && !d->boundary)) return set_error(MGT_ERR_ARG, "bad boundary list");
    for (int32_t k = 0; k < d->n_boundary; ++k)
        if (d->boundary[k] < 0 || d->boundary[k] >= N) return set_error(MGT_ERR_ARG, "boundary index out of range");
    const int R = d->n_rays;
    if (R < 2 || R % 2 != 0 || R > 3072) return set_error(MGT_ERR_ARG, "n_rays must be even, 2..3072");
    if (!finite_all(d->dirs, 3 * (int64_t)R)) return set_error(MGT_ERR_ARG, "directions must be finite");
    for (int r = 0; r < R; ++r) {
        const double *n = d->dirs + 3 * r;
        if (std::fabs(std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]) - 1.0) > 1e-9)
            return set_error(MGT_ERR_ARG, "directions must be unit vectors");
    }
    {
        std::vector<int32_t> pr;
        if (!find_pairs(d->dirs, R, pr)) return set_error(MGT_ERR_ARG, "a direction has no antipode");
    }
    if (d->n_quad < 1 || d->n_quad > kMaxQuad) return set_error(MGT_ERR_ARG, "n_quad must be 1..64");
    if (!(d->mol_mass_kg > 0.0) || !std::isfinite(d->mol_mass_kg)) return set_error(MGT_ERR_ARG, "mol_mass_kg must be > 0");
    if (!(d->T_bg >= 0.0) || !std::isfinite(d->T_bg)) return set_error(MGT_ERR_ARG, "T_bg must be >= 0");
    const int L = d->n_levels, M = d->n_lines, K = d->n_coll_trans;
    if (L < 2 || L > kMaxLevels) return set_error(MGT_ERR_ARG, "n_levels must be 2..64");
    if (M < 1 || M > L * (L - 1) / 2) return set_error(MGT_ERR_ARG, "n_lines out of range");
    if (K < 0 || K > L * (L - 1) / 2 || (K > 0 && (!d->cup || !d->clo || !d->K_ul)))
        return set_error(MGT_ERR_ARG, "bad collisional data");
    if (!finite_all(d->energy_J, L)) return set_error(MGT_ERR_ARG, "energies must be finite");
    for (int i = 0; i < L; ++i)
        if (!(d->g[i] > 0.0) || !std::isfinite(d->g[i])) return set_error(MGT_ERR_ARG, "weights must be > 0");
    std::set<std::pair<int, int>> seen;
    for (int k = 0; k < M; ++k) {
        const int u = d->up[k], l = d->lo[k];
        if (u < 0 || u >= L || l < 0 || l >= L || u == l) return set_error(MGT_ERR_ARG, "line level out of range");
        if (!(d->energy_J[u] > d->energy_J[l])) return set_error(MGT_ERR_ARG, "line upper level must lie above lower");
        if (!(d->A[k] > 0.0) || !std::isfinite(d->A[k]) || !(d->freq_Hz[k] > 0.0) || !std::isfinite(d->freq_Hz[k]))
            return set_error(MGT_ERR_ARG, "line A and frequency must be > 0");
        if (!seen.insert({u, l}).second) return set_error(MGT_ERR_ARG, "duplicate radiative line");
    }
    seen.clear();
    for (int k = 0; k < K; ++k) {
        const int u = d->cup[k], l = d->clo[k];
        if (u < 0 || u >= L || l < 0 || l >= L || u == l) return set_error(MGT_ERR_ARG, "collision level out of range");
        if (!(d->energy_J[u] > d->energy_J[l])) return set_error(MGT_ERR_ARG, "collision upper level must lie above lower");
        if (!(d->K_ul[k] >= 0.0) || !std::isfinite(d->K_ul[k])) return set_error(MGT_ERR_ARG, "K_ul must be >= 0");
        if (!seen.insert({std::min(u, l), std::max(u, l)}).second)
            return set_error(MGT_ERR_ARG, "duplicate collisional transition");
    }
    // each frequency bin sees only its own line: reject lines within 50 Doppler widths
    double wmax = 0.0;
    for (int64_t i = 0; i < N; ++i)
        wmax = std::max(wmax, std::sqrt(2.0 * kKB * d->temp[i] / d->mol_mass_kg + d->vturb2[i]) / kC);
    std::vector<double> f(d->freq_Hz, d->freq_Hz + M);
    std::sort(f.begin(), f.end());
    for (int k = 0; k + 1 < M; ++k)
        if (f[k + 1] - f[k] < 50.0 * wmax * f[k + 1]) return set_error(MGT_ERR_ARG, "overlapping lines are not supported");
    return MGT_OK;
}

static void free_model(mgt_model *m)
{
    void *ptrs[] = {m->d_dir_map, m->d_batch_pairs, m->d_nbr_pos, m->d_ent, m->d_ent_off, m->d_pos_hl, m->d_vel_hl, m->d_dirs32, m->d_order, m->d_pos, m->d_vel, m->d_temp, m->d_vturb2, m->d_ncoll, m->d_nspec, m->d_w64, m->d_w32, m->d_dxmax,
                    m->d_nbr_off, m->d_nbrs, m->d_bnd, m->d_dirs, m->d_pairs, m->d_xq, m->d_wq, m->d_line_tab,
                    m->d_line_ul, m->d_level_tab, m->d_coll_tab, m->d_coll_ul, m->d_entry, m->d_pops,
                    m->d_pops_prev, m->d_line32, m->d_line64, m->d_J, m->d_Lst, m->d_err, m->d_range_bad, m->d_count,
                    m->d_ray_off, m->d_steps64};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->d_steps32) {   // from the library's pool: back to its reserve
        cudaFreeAsync(m->d_steps32, nullptr);
        cudaStreamSynchronize(nullptr);
    }
    ng_free(m);
    image_free(m);
    delete m;
}

template <typename T> static mgt_status dalloc(T **p, size_t n)
{
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
    return MGT_OK;
}

template <typename T> static mgt_status upload(T *dst, const T *src, size_t n, cudaStream_t s)
{
    if (n == 0) return MGT_OK;
    MGT_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, s));
    return MGT_OK;
}

#define MGT_TRY(x)                         \
    do {                                   \
        mgt_status st_ = (x);              \
        if (st_ != MGT_OK) return st_;     \
    } while (0)


static mgt_status build_model(mgt_model *m, const mgt_model_desc *d, cudaStream_t s)
{
    const int64_t N = d->n_points;
    m->N = N;
    m->R = d->n_rays;
    m->P = m->R / 2;
    m->Q = d->n_quad;
    m->L = d->n_levels;
    m->M = d->n_lines;
    m->Mpad = (m->M + 7) / 8 * 8;
    m->K = d->n_coll_trans;
    m->n_boundary = d->n_boundary;
    m->nnz = d->nbr_offsets[N];
    m->mol_mass = d->mol_mass_kg;
    m->T_bg = d->T_bg;
    MGT_CUDA(cudaGetDevice(&m->device));

    if (!find_pairs(d->dirs, m->R, m->pairs)) return set_error(MGT_ERR_ARG, "a direction has no antipode");
    // length unit: the largest coordinate magnitude
    double Lu = 0.0;
    for (int64_t i = 0; i < 3 * N; ++i) Lu = std::max(Lu, std::fabs(d->pos[i]));
    m->L_unit = Lu > 0.0 ? Lu : 1.0;

    m->energy.assign(d->energy_J, d->energy_J + m->L);
    m->g.assign(d->g, d->g + m->L);
    m->up.assign(d->up, d->up + m->M);
    m->lo.assign(d->lo, d->lo + m->M);
    m->A.assign(d->A, d->A + m->M);
    m->freq.assign(d->freq_Hz, d->freq_Hz + m->M);
    if (m->K > 0) {
        m->cup.assign(d->cup, d->cup + m->K);
        m->clo.assign(d->clo, d->clo + m->K);
        m->Kul.assign(d->K_ul, d->K_ul + m->K);
    }
    gauss_hermite(m->Q, m->xq, m->wq);

    const int Mp = m->Mpad, L = m->L, K = m->K;
    std::vector<double> tab(8 * (size_t)Mp, 0.0);
    std::vector<int32_t> ul(2 * (size_t)Mp, 0);
    for (int k = 0; k < m->M; ++k) {
        const double nu = m->freq[k];
        const double Bul = m->A[k] * kC * kC / (2.0 * kH * nu * nu * nu);
        const double Blu = Bul * m->g[m->up[k]] / m->g[m->lo[k]];
        const double hk = m->T_bg > 0.0 ? kH * nu / (kKB * m->T_bg) : 0.0;
        const double nbg = hk > 0.0 ? 1.0 / std::expm1(hk) : 0.0;
        const double nbgmax = std::max(nbg, 1e-15);
        tab[0 * Mp + k] = nu;
        tab[1 * Mp + k] = m->A[k];
        tab[2 * Mp + k] = Bul;
        tab[3 * Mp + k] = Blu;
        tab[4 * Mp + k] = nbgmax;
        tab[5 * Mp + k] = hk;
        tab[6 * Mp + k] = 2.0 * kH * nu * nu * nu / (kC * kC) * nbgmax;
        ul[k] = m->up[k];
        ul[Mp + k] = m->lo[k];
    }
    for (int k = m->M; k < Mp; ++k) tab[4 * Mp + k] = 1.0;
    std::vector<double> lev(2 * (size_t)L);
    for (int i = 0; i < L; ++i) {
        lev[i] = m->energy[i];
        lev[L + i] = m->g[i];
    }
    std::vector<int16_t> entry(3 * (size_t)L * L, (int16_t)-1);
    for (int k = 0; k < m->M; ++k) {
        entry[m->up[k] * L + m->lo[k]] = (int16_t)k;              // down
        entry[(size_t)L * L + m->lo[k] * L + m->up[k]] = (int16_t)k; // up
    }
    std::vector<int32_t> cul(2 * (size_t)std::max(K, 1), 0);
    for (int k = 0; k < K; ++k) {
        entry[2 * (size_t)L * L + m->cup[k] * L + m->clo[k]] = (int16_t)k;
        entry[2 * (size_t)L * L + m->clo[k] * L + m->cup[k]] = (int16_t)k;
        cul[k] = m->cup[k];
        cul[K + k] = m->clo[k];
    }
    std::vector<int32_t> off32(N + 1);
    for (int64_t i = 0; i <= N; ++i) off32[i] = (int32_t)d->nbr_offsets[i];
    std::vector<uint8_t> bnd(N, 0);
    for (int32_t k = 0; k < d->n_boundary; ++k) bnd[d->boundary[k]] = 1;

    MGT_TRY(dalloc(&m->d_pos, 3 * N));
    MGT_TRY(dalloc(&m->d_vel, 3 * N));
    MGT_TRY(dalloc(&m->d_temp, N));
    MGT_TRY(dalloc(&m->d_vturb2, N));
    MGT_TRY(dalloc(&m->d_ncoll, N));
    MGT_TRY(dalloc(&m->d_nspec, N));
    MGT_TRY(dalloc(&m->d_w64, N));
    MGT_TRY(dalloc(&m->d_w32, N));
    MGT_TRY(dalloc(&m->d_dxmax, N));
    MGT_TRY(dalloc(&m->d_nbr_off, N + 1));
    MGT_TRY(dalloc(&m->d_nbrs, m->nnz));
    MGT_TRY(dalloc(&m->d_nbr_pos, 3 * m->nnz));
    MGT_TRY(dalloc(&m->d_pos_hl, 6 * N));
    MGT_TRY(dalloc(&m->d_vel_hl, 6 * N));
    MGT_TRY(dalloc(&m->d_dirs32, (size_t)m->R));
    MGT_TRY(dalloc(&m->d_order, N));
    MGT_TRY(dalloc(&m->d_bnd, N));
    MGT_TRY(dalloc(&m->d_dirs, 3 * (size_t)m->R));
    MGT_TRY(dalloc(&m->d_pairs, m->P));
    MGT_TRY(dalloc(&m->d_dir_map, (size_t)m->R));
    MGT_TRY(dalloc(&m->d_batch_pairs, (size_t)m->P));
    MGT_TRY(dalloc(&m->d_xq, m->Q));
    MGT_TRY(dalloc(&m->d_wq, m->Q));
    MGT_TRY(dalloc(&m->d_line_tab, tab.size()));
    MGT_TRY(dalloc(&m->d_line_ul, ul.size()));
    MGT_TRY(dalloc(&m->d_level_tab, lev.size()));
    MGT_TRY(dalloc(&m->d_coll_tab, std::max(K, 1)));
    MGT_TRY(dalloc(&m->d_coll_ul, cul.size()));
    MGT_TRY(dalloc(&m->d_entry, entry.size()));
    MGT_TRY(dalloc(&m->d_pops, N * L));
    MGT_TRY(dalloc(&m->d_pops_prev, N * L));
    MGT_TRY(dalloc(&m->d_line32, N * row_stride32(Mp)));
    MGT_TRY(dalloc(&m->d_line64, N * row_stride64(Mp)));
    MGT_TRY(dalloc(&m->d_J, N * m->M));
    MGT_TRY(dalloc(&m->d_Lst, N * m->M));
    MGT_TRY(dalloc(&m->d_err, 4));
    MGT_TRY(dalloc(&m->d_range_bad, 1));
    MGT_TRY(dalloc(&m->d_count, 4));

    MGT_TRY(upload(m->d_pos, d->pos, 3 * N, s));
    MGT_TRY(upload(m->d_vel, d->vel, 3 * N, s));
    MGT_TRY(upload(m->d_temp, d->temp, N, s));
    MGT_TRY(upload(m->d_vturb2, d->vturb2, N, s));
    MGT_TRY(upload(m->d_ncoll, d->n_coll, N, s));
    MGT_TRY(upload(m->d_nspec, d->n_spec, N, s));
    MGT_TRY(upload(m->d_nbr_off, off32.data(), N + 1, s));
    MGT_TRY(upload(m->d_nbrs, d->nbrs, m->nnz, s));
    MGT_TRY(upload(m->d_bnd, bnd.data(), N, s));
    {
        // exact power-of-two scaling that brings coordinates to order one, so
        // FP32 squared distances cannot overflow; the bounding box for the
        // visiting order
        double xmax = 0.0, lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) {
                const double x = d->pos[3 * i + c];
                xmax = std::max(xmax, std::fabs(x));
                lo[c] = std::min(lo[c], x);
                hi[c] = std::max(hi[c], x);
            }
        int ex = 0;
        std::frexp(xmax > 0.0 ? xmax : 1.0, &ex);
        m->pos_scale = std::ldexp(1.0, -ex);
        // |xs - (hi + lo)| <= 2^-24 |lo| <= 2^-48 |xs| <= 2^-48; four times that, for both endpoints
        m->pos_slack = (float)std::ldexp(1.0, -46);
        // packed walk rows: every point's neighbours in CSR order, the last one
        // flagged; an empty row holds one kEntEmpty entry; 16 pad entries
        std::vector<int32_t> eoff(N);
        int64_t ne = 0;
        for (int64_t i = 0; i < N; ++i) {
            eoff[i] = (int32_t)ne;
            const int64_t deg = d->nbr_offsets[i + 1] - d->nbr_offsets[i];
            ne += deg > 0 ? deg : 1;
        }
        // the packed entries carry their rows' offsets as 32-bit integers
        if (ne + 16 > (int64_t)0x7fffffff) return set_error(MGT_ERR_ARG, "more than 2^31 - 1 neighbour entries");
        m->n_ent = ne + 16;
        MGT_TRY(dalloc(&m->d_ent, 2 * (size_t)m->n_ent));
        MGT_TRY(dalloc(&m->d_ent_off, (size_t)N));
        MGT_TRY(upload(m->d_ent_off, eoff.data(), (size_t)N, s));
        std::vector<float4> d32(m->R);
        for (int r = 0; r < m->R; ++r)
            d32[r] = make_float4((float)d->dirs[3 * r], (float)d->dirs[3 * r + 1], (float)d->dirs[3 * r + 2], 0.0f);
        MGT_TRY(upload(m->d_dirs32, d32.data(), d32.size(), s));
        // hi + lo splits, neighbour positions, packed rows and the visiting order
        MGT_TRY(build_walk_tables(m, lo, hi, s));
        MGT_CUDA(cudaStreamSynchronize(s));   // the host staging vectors go out of scope
    }

    MGT_TRY(upload(m->d_dirs, d->dirs, 3 * (size_t)m->R, s));
    std::vector<int2> pr(m->P);
    for (int p = 0; p < m->P; ++p) pr[p] = make_int2(m->pairs[2 * p], m->pairs[2 * p + 1]);
    MGT_TRY(upload(m->d_pairs, pr.data(), m->P, s));
    MGT_TRY(upload(m->d_xq, m->xq.data(), m->Q, s));
    MGT_TRY(upload(m->d_wq, m->wq.data(), m->Q, s));
    MGT_TRY(upload(m->d_line_tab, tab.data(), tab.size(), s));
    MGT_TRY(upload(m->d_line_ul, ul.data(), ul.size(), s));
    MGT_TRY(upload(m->d_level_tab, lev.data(), lev.size(), s));
    if (K > 0) MGT_TRY(upload(m->d_coll_tab, m->Kul.data(), K, s));
    MGT_TRY(upload(m->d_coll_ul, cul.data(), cul.size(), s));
    MGT_TRY(upload(m->d_entry, entry.data(), entry.size(), s));
    MGT_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int) * 4, s));
    MGT_CUDA(cudaMemsetAsync(m->d_count, 0, sizeof(unsigned long long) * 4, s));
    MGT_TRY(launch_widths(m, s));
    MGT_TRY(launch_lte(m, s));
    MGT_CUDA(cudaMemcpyAsync(m->d_pops_prev, m->d_pops, sizeof(double) * N * L, cudaMemcpyDeviceToDevice, s));
    MGT_TRY(ng_reset(m, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    return MGT_OK;
}

__global__ void k_transpose_out(int64_t N, int M, const double *__restrict__ in, double *__restrict__ out)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= N * M) return;
    int k = (int)(t / N);
    int64_t o = t - (int64_t)k * N;
    out[t] = in[o * M + k];
}

static bool batched(const mgt_model *m) { return m->opts.pairs_per_batch > 0 && m->opts.pairs_per_batch < m->P; }

mgt_status ensure_rays(mgt_model *m, mgt_precision p, cudaStream_t s)
{
    if (!m->traced) return set_error(MGT_ERR_STATE, "mgt_trace_rays must be called first");
    const bool all = m->rays_p0 == 0 && m->rays_np == m->P;
    if (!all || m->steps_width_mode != m->opts.width_mode) MGT_TRY(trace_all(m, s));
    if (p == MGT_FP64 && (!m->d_steps64 || m->steps64_width_mode != m->opts.width_mode))
        MGT_TRY(build_steps64(m, s));
    return MGT_OK;
}

static mgt_status formal_solve_device(mgt_model *m, mgt_precision p, cudaStream_t s)
{
    if (p != MGT_FP64 && p != MGT_FP32_MIXED) return set_error(MGT_ERR_ARG, "unknown precision");
    if (batched(m)) {
        // rays of at most B pairs at a time: trace, solve, add, next batch
        if (!m->traced) return set_error(MGT_ERR_STATE, "mgt_trace_rays must be called first");
        if (m->line_dirty) MGT_TRY(launch_line_data(m, s));
        const int32_t B = m->opts.pairs_per_batch;
        for (int32_t p0 = 0; p0 < m->P; p0 += B) {
            const int32_t np = std::min(B, m->P - p0);
            if (!(m->rays_p0 == p0 && m->rays_np == np && m->steps_width_mode == m->opts.width_mode))
                MGT_TRY(trace_range(m, s, p0, np));
            if (p == MGT_FP64 && (!m->d_steps64 || m->steps64_width_mode != m->opts.width_mode))
                MGT_TRY(build_steps64(m, s));
            MGT_TRY(launch_formal_solve(m, p, s, p0 > 0));
        }
        m->have_J = true;
        return MGT_OK;
    }
    MGT_TRY(ensure_rays(m, p, s));
    if (m->line_dirty) MGT_TRY(launch_line_data(m, s));
    MGT_TRY(launch_formal_solve(m, p, s, false));
    m->have_J = true;
    return MGT_OK;
}

static mgt_status stat_eq_device(mgt_model *m, cudaStream_t s)
{
    if (!m->have_J) return set_error(MGT_ERR_STATE, "mgt_formal_solve must be called first");
    MGT_CUDA(cudaMemcpyAsync(m->d_pops_prev, m->d_pops, sizeof(double) * m->N * m->L, cudaMemcpyDeviceToDevice, s));
    MGT_TRY(launch_stat_eq(m, s));
    m->line_dirty = true;
    return MGT_OK;
}

}  // namespace mgt

using namespace mgt;

extern "C" {

const char *mgt_last_error(void) { return g_last_error.c_str(); }

mgt_status mgt_model_create(mgt_model **out, const mgt_model_desc *desc, void *stream)
{
    MGT_RANGE("mgt_model_create");
    if (!out) return set_error(MGT_ERR_ARG, "out is NULL");
    *out = nullptr;
    MGT_TRY(validate(desc));
    mgt_model *m = new mgt_model();
    mgt_status st = build_model(m, desc, (cudaStream_t)stream);
    if (st != MGT_OK) {
        std::string keep = g_last_error;
        cudaStreamSynchronize((cudaStream_t)stream);
        free_model(m);
        g_last_error = keep;
        return st;
    }
    model_born(m->device);
    *out = m;
    return MGT_OK;
}

mgt_status mgt_model_destroy(mgt_model *m)
{
    if (!m) return MGT_OK;
    cudaDeviceSynchronize();
    const int dev = m->device;
    free_model(m);
    model_gone(dev);
    return MGT_OK;
}

mgt_status mgt_set_solve_opts(mgt_model *m, const mgt_solve_opts *o)
{
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    mgt_solve_opts d{0.35, 0, 0, 0, 0, 0};
    if (o) {
        if (o->schedule < 0 || o->schedule > 4) return set_error(MGT_ERR_ARG, "schedule must be 0..4");
        if (o->subdivisions < 0 || o->subdivisions > 256) return set_error(MGT_ERR_ARG, "subdivisions must be 0..256");
        if (o->pairs_per_batch < 0) return set_error(MGT_ERR_ARG, "pairs_per_batch must be >= 0");
        if (!(o->switch_threshold >= 0.0) || !std::isfinite(o->switch_threshold))
            return set_error(MGT_ERR_ARG, "switch_threshold must be >= 0");
        if (o->width_mode != 0 && o->width_mode != 1) return set_error(MGT_ERR_ARG, "width_mode must be 0 or 1");
        if (o->lines_per_thread != 0 && o->lines_per_thread != 4 && o->lines_per_thread != 8)
            return set_error(MGT_ERR_ARG, "lines_per_thread must be 0, 4 or 8");
        d = *o;
    }
    m->opts = d;
    return MGT_OK;
}

mgt_status mgt_trace_rays(mgt_model *m, mgt_trace_stats *stats, void *stream)
{
    MGT_RANGE("mgt_trace_rays");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    mgt_trace_stats st{};
    const int32_t B = batched(m) ? m->opts.pairs_per_batch : m->P;
    for (int32_t p0 = 0; p0 < m->P; p0 += B) {
        MGT_TRY(trace_range(m, s, p0, std::min(B, m->P - p0)));
        st.total_steps += m->total_steps;
        st.n_stalls += m->n_stalls;
        st.max_half_ray = std::max(st.max_half_ray, m->max_half);
        st.n_fp64_steps += m->n_exact_steps;
    }
    st.mean_half_ray = (double)st.total_steps / ((double)m->N * m->R);
    m->stats = st;
    if (stats) {
        MGT_TRY(check_device_error(m, s));
        *stats = st;
    }
    return MGT_OK;
}

mgt_status mgt_get_rays(mgt_model *m, int64_t *ray_off, int32_t *idx, void *stream)
{
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    if (!m->traced) return set_error(MGT_ERR_STATE, "mgt_trace_rays must be called first");
    if (batched(m)) return set_error(MGT_ERR_STATE, "rays are held one pair batch at a time (pairs_per_batch)");
    if (!(m->rays_p0 == 0 && m->rays_np == m->P)) MGT_TRY(trace_all(m, (cudaStream_t)stream));
    cudaStream_t s = (cudaStream_t)stream;
    if (ray_off)
        MGT_CUDA(cudaMemcpyAsync(ray_off, m->d_ray_off, sizeof(int64_t) * ((int64_t)m->R * m->N + 1),
                                 cudaMemcpyDeviceToHost, s));
    if (idx && m->total_steps > 0)
        MGT_CUDA(cudaMemcpy2DAsync(idx, sizeof(int32_t), m->d_steps32, sizeof(Step32), sizeof(int32_t),
                                   (size_t)m->total_steps, cudaMemcpyDeviceToHost, s));
    return check_device_error(m, s);
}

mgt_status mgt_set_populations(mgt_model *m, const double *pops, void *stream)
{
    MGT_RANGE("mgt_set_populations");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (pops) {
        const int64_t n = m->N * m->L;
        for (int64_t i = 0; i < n; ++i)
            if (!(pops[i] >= 0.0) || !std::isfinite(pops[i]))
                return set_error(MGT_ERR_ARG, "populations must be finite and >= 0");
        MGT_CUDA(cudaMemcpyAsync(m->d_pops, pops, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    } else {
        MGT_TRY(launch_lte(m, s));
    }
    MGT_CUDA(cudaMemcpyAsync(m->d_pops_prev, m->d_pops, sizeof(double) * m->N * m->L, cudaMemcpyDeviceToDevice, s));
    m->line_dirty = true;
    m->have_J = false;
    MGT_TRY(ng_reset(m, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    return MGT_OK;
}

mgt_status mgt_get_populations(mgt_model *m, double *pops, int on_device, void *stream)
{
    if (!m || !pops) return set_error(MGT_ERR_ARG, "model or output is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    MGT_CUDA(cudaMemcpyAsync(pops, m->d_pops, sizeof(double) * m->N * m->L,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (on_device) return MGT_OK;
    return check_device_error(m, s);
}

static mgt_status copy_out_jbar(mgt_model *m, double *Jbar, double *Lstar, int on_device, cudaStream_t s)
{
    if (!Jbar && !Lstar) return MGT_OK;
    const int64_t n = m->N * m->M;
    double *tmp = nullptr;
    if (!on_device) MGT_CUDA(cudaMallocAsync(&tmp, sizeof(double) * n, s));
    const double *srcs[2] = {m->d_J, m->d_Lst};
    double *dsts[2] = {Jbar, Lstar};
    for (int i = 0; i < 2; ++i) {
        if (!dsts[i]) continue;
        double *target = on_device ? dsts[i] : tmp;
        k_transpose_out<<<ceil_div(n, 256), 256, 0, s>>>(m->N, m->M, srcs[i], target);
        MGT_LAUNCH_CHECK("k_transpose_out");
        if (!on_device) MGT_CUDA(cudaMemcpyAsync(dsts[i], tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    if (!on_device) {
        MGT_CUDA(cudaFreeAsync(tmp, s));
        return check_device_error(m, s);
    }
    return MGT_OK;
}

mgt_status mgt_formal_solve(mgt_model *m, mgt_precision p, double *Jbar, double *Lstar, int on_device, void *stream)
{
    MGT_RANGE("mgt_formal_solve");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    MGT_TRY(formal_solve_device(m, p, s));
    return copy_out_jbar(m, Jbar, Lstar, on_device, s);
}

mgt_status mgt_get_jbar(mgt_model *m, double *Jbar, double *Lstar, int on_device, void *stream)
{
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    if (!m->have_J) return set_error(MGT_ERR_STATE, "no formal solution yet");
    return copy_out_jbar(m, Jbar, Lstar, on_device, (cudaStream_t)stream);
}

mgt_status mgt_stat_equilibrium(mgt_model *m, double *pops_out, void *stream)
{
    MGT_RANGE("mgt_stat_equilibrium");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    MGT_TRY(stat_eq_device(m, s));
    if (pops_out) {
        MGT_CUDA(cudaMemcpyAsync(pops_out, m->d_pops, sizeof(double) * m->N * m->L, cudaMemcpyDeviceToHost, s));
        return check_device_error(m, s);
    }
    return MGT_OK;
}

mgt_status mgt_ng_accelerate(mgt_model *m, const mgt_ng_opts *o, int *accepted, double *maxrel, void *stream)
{
    MGT_RANGE("mgt_ng_accelerate");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    if (o) {
        if (o->mode < MGT_NG_NONE || o->mode > MGT_NG_ADAPTIVE) return set_error(MGT_ERR_ARG, "unknown Ng mode");
        if (o->mode == MGT_NG_CLASSICAL && (o->n_steps < 2 || o->n_steps > kMaxNgHist - 1))
            return set_error(MGT_ERR_ARG, "n_steps must be 2..15");
        if (o->mode == MGT_NG_ADAPTIVE && (o->n_max < 3 || o->n_max > kMaxNgHist))
            return set_error(MGT_ERR_ARG, "n_max must be 3..16");
    }
    return ng_step(m, o, accepted, maxrel, (cudaStream_t)stream);
}

mgt_status mgt_ali_solve(mgt_model *m, const mgt_ali_opts *o, mgt_ali_stats *stats, void *stream)
{
    MGT_RANGE("mgt_ali_solve");
    if (!m || !o) return set_error(MGT_ERR_ARG, "model or options NULL");
    if (o->n_iter < 0) return set_error(MGT_ERR_ARG, "n_iter must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int acc_total = 0;
    double mr = 0.0;
    for (int it = 0; it < o->n_iter; ++it) {
        MGT_TRY(formal_solve_device(m, o->precision, s));
        MGT_TRY(stat_eq_device(m, s));
        int acc = 0;
        MGT_TRY(mgt_ng_accelerate(m, &o->ng, &acc, &mr, stream));
        acc_total += acc;
        if (!std::isfinite(mr)) {
            if (stats) *stats = {it + 1, acc_total, mr};
            return set_error(MGT_ERR_NOT_CONVERGED, "populations became non-finite");
        }
    }
    if (stats) *stats = {o->n_iter, acc_total, mr};
    return check_device_error(m, s);
}

mgt_status mgt_sync(mgt_model *m, void *stream)
{
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    return check_device_error(m, (cudaStream_t)stream);
}

mgt_status mgt_launch_count(int64_t *count)
{
    if (!count) return set_error(MGT_ERR_ARG, "count is NULL");
    *count = g_launches.load(std::memory_order_relaxed);
    return MGT_OK;
}

mgt_status mgt_kernel_timing(int32_t enable)
{
    std::lock_guard<std::mutex> lk(g_kt_mu);
    if (enable) {
        for (const KtRecord &r : g_kt_pending) {
            cudaEventSynchronize(r.b);
            g_kt_spare.push_back(r.a);
            g_kt_spare.push_back(r.b);
        }
        g_kt_pending.clear();
        g_kt_totals.clear();
    }
    g_kt_on.store(enable != 0, std::memory_order_relaxed);
    return MGT_OK;
}

mgt_status mgt_kernel_times(int32_t capacity, mgt_kernel_time *out, int32_t *n_out)
{
    if (capacity < 0 || (capacity > 0 && !out) || !n_out) return set_error(MGT_ERR_ARG, "mgt_kernel_times: bad output");
    std::lock_guard<std::mutex> lk(g_kt_mu);
    cudaError_t err = cudaSuccess;
    for (const KtRecord &r : g_kt_pending) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        auto it = std::find_if(g_kt_totals.begin(), g_kt_totals.end(),
                               [&](const KtTotal &t) { return t.name == r.name; });
        if (it == g_kt_totals.end()) {
            g_kt_totals.push_back({r.name, 0, 0.0, 0.0});
            it = g_kt_totals.end() - 1;
        }
        it->launches += 1;
        it->ms += ms;
        it->bytes += r.bytes;
        g_kt_spare.push_back(r.a);
        g_kt_spare.push_back(r.b);
    }
    g_kt_pending.clear();
    if (err != cudaSuccess) return cuda_status(err, "mgt_kernel_times");
    const int n = (int)g_kt_totals.size();
    for (int i = 0; i < n && i < capacity; ++i) {
        std::memset(out[i].name, 0, sizeof out[i].name);
        std::strncpy(out[i].name, g_kt_totals[i].name.c_str(), sizeof out[i].name - 1);
        out[i].launches = g_kt_totals[i].launches;
        out[i].total_ms = g_kt_totals[i].ms;
        out[i].bytes = g_kt_totals[i].bytes;
    }
    *n_out = n;
    return MGT_OK;
}

mgt_status mgt_model_sizes(const mgt_model *m, int64_t *n_points, int32_t *n_rays, int32_t *n_levels,
                           int32_t *n_lines, int32_t *n_quad)
{
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    if (n_points) *n_points = m->N;
    if (n_rays) *n_rays = m->R;
    if (n_levels) *n_levels = m->L;
    if (n_lines) *n_lines = m->M;
    if (n_quad) *n_quad = m->Q;
    return MGT_OK;
}

}  // extern "C"
