// Ng-acceleration (Sec. 4.2, Appendix A): device streaming kernels and the
// host-side controller (classical and adaptive).
//
// The iterate is the vector of fractional populations x = n_i / n_spec over
// all points and levels.  Residuals r_k = x_{k+1} - x_k of the iterates since
// the last prediction build the Gram matrix G = R R^T; the coefficients are
// c = G^-1 1 / (1^T G^-1 1) and the prediction is sum_k c_k x_{k+1}.
// Reductions are two-stage (fixed-order block partials, then one block), so
// every number is bitwise reproducible.
#include <cmath>
#include <cstring>

#include "mgt_common.cuh"

namespace mgt {

namespace {

constexpr int kNgThreads = 256;
constexpr int kNgMaxBlocks = 1216;   // 8 x 152 SMs

struct Slots {
    const double *h[kMaxNgHist + 1];  // history iterates, oldest first
};

__device__ __forceinline__ void atomic_max_pos(double *addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// Push: x_new = pops / n_spec into `out` (if not null); dots[k] = <r_new, r_k>
// for the m-1 stored residuals and dots[m-1] = <r_new, r_new>, r_new = x_new -
// h[m-1]; maxrel = max |pops - prev| / |prev| over prev != 0.
__global__ void __launch_bounds__(kNgThreads) k_ng_push(int64_t n, int L, const double *__restrict__ pops,
                                                        const double *__restrict__ prev,
                                                        const double *__restrict__ nspec, double *__restrict__ out,
                                                        Slots hs, int m, double *__restrict__ partials,
                                                        double *__restrict__ maxrel)
{
    double acc[kMaxNgHist];
#pragma unroll
    for (int k = 0; k < kMaxNgHist; ++k) acc[k] = 0.0;
    double mr = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double pv = pops[e], pp = prev[e];
        if (pp != 0.0) mr = fmax(mr, fabs(pv - pp) / fabs(pp));
        if (m > 0) {
            const double x = pv / nspec[e / L];
            if (out) out[e] = x;
            const double r = x - hs.h[m - 1][e];
#pragma unroll
            for (int k = 0; k < kMaxNgHist; ++k) {
                if (k < m - 1) acc[k] += r * (hs.h[k + 1][e] - hs.h[k][e]);
            }
#pragma unroll
            for (int k = 0; k < kMaxNgHist; ++k)
                if (k == m - 1) acc[k] += r * r;
        } else if (out) {
            out[e] = pv / nspec[e / L];
        }
    }
    atomic_max_pos(maxrel, mr);
    __shared__ double red[kNgThreads];
    for (int k = 0; k < m; ++k) {
        double v = 0.0;
#pragma unroll
        for (int kk = 0; kk < kMaxNgHist; ++kk)
            if (kk == k) v = acc[kk];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int s = kNgThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxNgHist + k] = red[0];
        __syncthreads();
    }
}

// Sum block partials in block order: out[k] = sum_b partials[b][k].
__global__ void k_ng_finish(int nblocks, int m, const double *__restrict__ partials, double *__restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= m) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * kMaxNgHist + k];
    out[k] = s;
}

struct Coef {
    double c[kMaxNgHist];
};

// Prediction x* = sum_k c_k h[k+1]; counts negative entries; maxrel against
// the previous running prediction when given.
__global__ void __launch_bounds__(kNgThreads) k_ng_predict(int64_t n, Slots hs, int nc, Coef cf,
                                                           double *__restrict__ out, const double *__restrict__ prev,
                                                           double *__restrict__ red)
{
    double mr = 0.0, neg = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0;
        for (int k = 0; k < nc; ++k) x += cf.c[k] * hs.h[k + 1][e];
        out[e] = x;
        if (x < 0.0) neg = 1.0;
        if (prev) {
            const double pp = prev[e];
            if (pp != 0.0) mr = fmax(mr, fabs(x - pp) / fabs(pp));
        }
    }
    atomic_max_pos(red + 0, mr);
    atomic_max_pos(red + 1, neg);
}

__global__ void k_ng_apply(int64_t n, int L, const double *__restrict__ x, const double *__restrict__ nspec,
                           double *__restrict__ pops)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        pops[e] = x[e] * nspec[e / L];
}

int grid_for(int64_t n)
{
    int64_t b = (n + kNgThreads - 1) / kNgThreads;
    return (int)(b < kNgMaxBlocks ? (b < 1 ? 1 : b) : kNgMaxBlocks);
}

int slots_needed(const mgt_ng_opts &o)
{
    if (o.mode == MGT_NG_CLASSICAL) return o.n_steps + 2;
    if (o.mode == MGT_NG_ADAPTIVE) return o.n_max + 3;
    return 0;
}

int free_slot(const NgState &ng)
{
    for (int s = 0; s < ng.n_slots; ++s) {
        bool used = (s == ng.pred_slot) || (ng.have_prev_pred && s == ng.prev_pred_slot);
        for (int h : ng.hist) used = used || (h == s);
        if (!used) return s;
    }
    return -1;
}

}  // namespace

void ng_free(mgt_model *m)
{
    NgState &ng = m->ng;
    if (ng.d_slots) cudaFree(ng.d_slots);
    if (ng.d_partials) cudaFree(ng.d_partials);
    if (ng.d_red) cudaFree(ng.d_red);
    if (ng.h_red) cudaFreeHost(ng.h_red);
    ng.d_slots = ng.d_partials = ng.d_red = ng.h_red = nullptr;
    ng.n_slots = 0;
    ng.hist.clear();
}

mgt_status ng_reset(mgt_model *m, cudaStream_t)
{
    m->ng.hist.clear();
    m->ng.have_prev_pred = false;
    m->ng.G.assign(kMaxNgHist * kMaxNgHist, 0.0);
    return MGT_OK;
}

static mgt_status ng_alloc(mgt_model *m, const mgt_ng_opts &o)
{
    NgState &ng = m->ng;
    const int64_t n = m->N * m->L;
    if (!ng.d_partials) {
        MGT_CUDA(cudaMalloc(&ng.d_partials, sizeof(double) * kNgMaxBlocks * kMaxNgHist));
        MGT_CUDA(cudaMalloc(&ng.d_red, sizeof(double) * (kMaxNgHist + 4)));
        MGT_CUDA(cudaMallocHost(&ng.h_red, sizeof(double) * (kMaxNgHist + 4)));
    }
    const int need = slots_needed(o);
    if (need > ng.n_slots) {
        if (ng.d_slots) MGT_CUDA(cudaFree(ng.d_slots));
        ng.d_slots = nullptr;
        cudaError_t e = cudaMalloc(&ng.d_slots, sizeof(double) * n * need);
        if (e != cudaSuccess) return set_error(MGT_ERR_OOM, "cannot allocate the Ng history");
        ng.n_slots = need;
        ng.hist.clear();
        ng.have_prev_pred = false;
    }
    if (ng.G.empty()) ng.G.assign(kMaxNgHist * kMaxNgHist, 0.0);
    return MGT_OK;
}

// One Ng step after a statistical-equilibrium solve: pops = new regular
// iterate, pops_prev = the populations it was computed from.  It runs in three
// phases so that a batch of models can share each host synchronisation:
//   ng_begin        push the new iterate (Gram row, maximum change), copy the
//                   reductions to the host asynchronously;
//   ng_after_push   (reductions on the host) update the Gram matrix and, when
//                   a prediction is due, launch it and copy its checks back;
//   ng_after_predict (checks on the host) use the prediction or not.
// ng_step runs the three with a stream synchronisation between them.
namespace {

Slots hist_slots(const NgState &ng, double *slot, int64_t n, int count)
{
    Slots h{};
    for (int k = 0; k < count; ++k) h.h[k] = slot + (size_t)ng.hist[k] * n;
    return h;
}

}  // namespace

mgt_status ng_begin(mgt_model *m, const mgt_ng_opts *o, cudaStream_t s)
{
    NgState &ng = m->ng;
    const int64_t n = m->N * m->L;
    ng.pend = NgPending{};
    const mgt_ng_opts opts = o ? *o : mgt_ng_opts{MGT_NG_NONE, 4, 8};
    if (opts.mode != ng.opts.mode || opts.n_steps != ng.opts.n_steps || opts.n_max != ng.opts.n_max) {
        ng.opts = opts;
        ng_reset(m, s);
    }
    mgt_status st = ng_alloc(m, opts);
    if (st != MGT_OK) return st;
    const int grid = grid_for(n);
    double *slot = ng.d_slots;

    if (opts.mode == MGT_NG_NONE) {
        MGT_CUDA(cudaMemsetAsync(ng.d_red + kMaxNgHist, 0, sizeof(double), s));
        Slots hs{};
        {
            MGT_KTIMER_BYTES("k_ng_push", s, 16.0 * n);
            k_ng_push<<<grid, kNgThreads, 0, s>>>(n, m->L, m->d_pops, m->d_pops_prev, m->d_nspec, nullptr, hs, 0,
                                                  ng.d_partials, ng.d_red + kMaxNgHist);
        }
        MGT_LAUNCH_CHECK("k_ng_push");
        MGT_CUDA(cudaMemcpyAsync(ng.h_red, ng.d_red + kMaxNgHist, sizeof(double), cudaMemcpyDeviceToHost, s));
        ng.pend.phase = 1;
        ng.pend.none = true;
        return MGT_OK;
    }

    // first call after a reset: the populations the iterate came from start the history
    if (ng.hist.empty()) {
        const int s0 = free_slot(ng);
        Slots hs{};
        {
            MGT_KTIMER_BYTES("k_ng_push", s, 16.0 * n + 8.0 * m->N);
            k_ng_push<<<grid, kNgThreads, 0, s>>>(n, m->L, m->d_pops_prev, m->d_pops_prev, m->d_nspec,
                                                  slot + (size_t)s0 * n, hs, 0, ng.d_partials,
                                                  ng.d_red + kMaxNgHist + 1);
        }
        MGT_LAUNCH_CHECK("k_ng_push");
        ng.hist.push_back(s0);
        ng.G.assign(kMaxNgHist * kMaxNgHist, 0.0);
        ng.have_prev_pred = false;
    }
    // push the new iterate
    const int mh = (int)ng.hist.size();
    const int snew = free_slot(ng);
    if (snew < 0 || mh > kMaxNgHist) return set_error(MGT_ERR_STATE, "Ng history overflow");
    const Slots hs = hist_slots(ng, slot, n, mh);
    MGT_CUDA(cudaMemsetAsync(ng.d_red + kMaxNgHist, 0, sizeof(double), s));
    {
        // populations, previous populations and every history slot in, the new slot out
        MGT_KTIMER_BYTES("k_ng_push", s, (3.0 + mh) * 8.0 * n + 8.0 * m->N);
        k_ng_push<<<grid, kNgThreads, 0, s>>>(n, m->L, m->d_pops, m->d_pops_prev, m->d_nspec, slot + (size_t)snew * n,
                                              hs, mh, ng.d_partials, ng.d_red + kMaxNgHist);
    }
    MGT_LAUNCH_CHECK("k_ng_push");
    k_ng_finish<<<1, 32, 0, s>>>(grid, mh, ng.d_partials, ng.d_red);
    MGT_LAUNCH_CHECK("k_ng_finish");
    MGT_CUDA(cudaMemcpyAsync(ng.h_red, ng.d_red, sizeof(double) * (kMaxNgHist + 1), cudaMemcpyDeviceToHost, s));
    ng.pend.phase = 1;
    ng.pend.mh = mh;
    ng.pend.snew = snew;
    return MGT_OK;
}

mgt_status ng_after_push(mgt_model *m, cudaStream_t s)
{
    NgState &ng = m->ng;
    NgPending &pd = ng.pend;
    if (pd.phase != 1) return set_error(MGT_ERR_STATE, "Ng: no push in flight");
    pd.phase = 0;
    if (pd.none) {
        pd.maxrel = ng.h_red[0];
        return MGT_OK;
    }
    const int64_t n = m->N * m->L;
    const int grid = grid_for(n);
    double *slot = ng.d_slots;
    pd.maxrel = ng.h_red[kMaxNgHist];
    // new residual index mh-1 (residual between hist[mh-1] and the new iterate)
    const int rn = pd.mh - 1;
    for (int k = 0; k <= rn; ++k) {
        ng.G[rn * kMaxNgHist + k] = ng.h_red[k];
        ng.G[k * kMaxNgHist + rn] = ng.h_red[k];
    }
    ng.hist.push_back(pd.snew);
    const int mcount = (int)ng.hist.size();
    pd.mcount = mcount;
    const double *prev = nullptr;
    if (ng.opts.mode == MGT_NG_CLASSICAL) {
        if (mcount < ng.opts.n_steps + 1) return MGT_OK;
    } else {
        if (mcount == 2) {
            ng.prev_pred_slot = ng.hist[1];   // P_2 := x_2
            ng.have_prev_pred = true;
            return MGT_OK;
        }
        if (mcount < 3) return MGT_OK;
        if (ng.have_prev_pred) prev = slot + (size_t)ng.prev_pred_slot * n;
    }
    // a prediction from the residuals' Gram matrix
    const int nres = mcount - 1;
    Coef cf{};
    if (!ng_solve_coefficients(ng.G.data(), kMaxNgHist, nres, cf.c)) {   // exactly singular: no prediction
        pd.negative = true;
        pd.mr_pred = INFINITY;
        pd.phase = 3;
        return MGT_OK;
    }
    if (ng.pred_slot < 0 || ng.pred_slot == ng.prev_pred_slot) {
        ng.pred_slot = -1;
        ng.pred_slot = free_slot(ng);
    }
    const Slots h2 = hist_slots(ng, slot, n, mcount);
    MGT_CUDA(cudaMemsetAsync(ng.d_red + kMaxNgHist + 1, 0, sizeof(double) * 2, s));
    {
        MGT_KTIMER_BYTES("k_ng_predict", s, (nres + 1.0 + (prev ? 1.0 : 0.0)) * 8.0 * n);
        k_ng_predict<<<grid, kNgThreads, 0, s>>>(n, h2, nres, cf, slot + (size_t)ng.pred_slot * n, prev,
                                                 ng.d_red + kMaxNgHist + 1);
    }
    MGT_LAUNCH_CHECK("k_ng_predict");
    MGT_CUDA(cudaMemcpyAsync(ng.h_red + kMaxNgHist + 1, ng.d_red + kMaxNgHist + 1, sizeof(double) * 2,
                             cudaMemcpyDeviceToHost, s));
    pd.phase = 2;
    return MGT_OK;
}

mgt_status ng_after_predict(mgt_model *m, cudaStream_t s)
{
    NgState &ng = m->ng;
    NgPending &pd = ng.pend;
    if (pd.phase != 2 && pd.phase != 3) return MGT_OK;   // no prediction this step
    if (pd.phase == 2) {
        pd.mr_pred = ng.h_red[kMaxNgHist + 1];
        pd.negative = ng.h_red[kMaxNgHist + 2] != 0.0;
    }
    pd.phase = 0;
    const int64_t n = m->N * m->L;
    const int grid = grid_for(n);
    auto use_prediction = [&]() -> mgt_status {
        {
            MGT_KTIMER_BYTES("k_ng_apply", s, 16.0 * n + 8.0 * m->N);
            k_ng_apply<<<grid, kNgThreads, 0, s>>>(n, m->L, ng.d_slots + (size_t)ng.pred_slot * n, m->d_nspec,
                                                   m->d_pops);
        }
        MGT_LAUNCH_CHECK("k_ng_apply");
        const int keep = ng.pred_slot;
        ng.hist.assign(1, keep);
        ng.pred_slot = -1;
        ng.have_prev_pred = false;
        ng.G.assign(kMaxNgHist * kMaxNgHist, 0.0);
        m->line_dirty = true;
        pd.accepted = 1;
        return MGT_OK;
    };
    auto restart_from_newest = [&]() {
        const int keep = ng.hist.back();
        ng.hist.assign(1, keep);
        ng.have_prev_pred = false;
        ng.G.assign(kMaxNgHist * kMaxNgHist, 0.0);
    };
    if (ng.opts.mode == MGT_NG_CLASSICAL) {
        if (pd.negative) {
            restart_from_newest();
            return MGT_OK;
        }
        return use_prediction();
    }
    // adaptive
    if (std::isinf(pd.mr_pred)) {          // singular Gram matrix
        restart_from_newest();
        return MGT_OK;
    }
    if (pd.mr_pred < pd.maxrel || pd.mcount >= ng.opts.n_max) {
        if (pd.negative) {
            restart_from_newest();
            return MGT_OK;
        }
        return use_prediction();
    }
    // keep the running prediction for the next comparison
    ng.prev_pred_slot = ng.pred_slot;
    ng.have_prev_pred = true;
    ng.pred_slot = -1;
    return MGT_OK;
}

mgt_status ng_step(mgt_model *m, const mgt_ng_opts *o, int *accepted, double *maxrel, cudaStream_t s)
{
    if (accepted) *accepted = 0;
    mgt_status st = ng_begin(m, o, s);
    if (st != MGT_OK) return st;
    MGT_CUDA(cudaStreamSynchronize(s));
    st = ng_after_push(m, s);
    if (st != MGT_OK) return st;
    if (m->ng.pend.phase == 2) MGT_CUDA(cudaStreamSynchronize(s));
    st = ng_after_predict(m, s);
    if (st != MGT_OK) return st;
    if (accepted) *accepted = m->ng.pend.accepted;
    if (maxrel) *maxrel = m->ng.pend.maxrel;
    return check_device_error(m, s);
}

}  // namespace mgt
