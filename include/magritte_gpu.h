/*
 * magritte_gpu.h -- C-ABI of the GB300 (sm_103a) line radiative-transfer hot
 * path of Magritte (arXiv 2411.03040).
 *
 * The calls follow the paper's statement of the problem: a model built from
 * positions, velocities, neighbours, boundary points, temperature, turbulence,
 * species densities, uniform rays, line data and a quadrature order (Sec. 3.2,
 * Listing 2), and the solver steps of Listing 3 (compute the radiation field,
 * compute level populations with Ng-acceleration).
 *
 * Conventions shared by every entry point
 *  - All arrays are plain C pointers.  Host arrays passed to mgt_model_create
 *    are borrowed for the duration of the call and copied; the library owns all
 *    device memory of a model until mgt_model_destroy.
 *  - A model lives on the device that is current when mgt_model_create is
 *    called; every later call on it, mgt_model_destroy included, must be made
 *    with that device current (the library never switches devices).
 *  - Output pointers are caller-owned.  Where an `on_device` flag is taken,
 *    nonzero means the pointer is a device address on the model's device,
 *    zero means host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is stream-ordered.  Calls that return data to host memory
 *    synchronise the stream before returning.
 *  - Every call returns an mgt_status.  MGT_ERR_ARG means the arguments were
 *    rejected before any work or allocation.  Device-side problems (a kernel's
 *    bounded loop running out, an index out of range) are recorded in a device
 *    error word and reported as MGT_ERR_BOUNDS / MGT_ERR_TIMEOUT by the next
 *    synchronising call or by mgt_sync.  mgt_last_error() returns a
 *    thread-local message describing the last non-OK status.
 *  - SI units throughout (m, s, K, kg, J, Hz, W m^-2 Hz^-1 sr^-1).
 */
#ifndef MAGRITTE_GPU_H
#define MAGRITTE_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgt_model mgt_model;

typedef enum {
    MGT_OK = 0,
    MGT_ERR_ARG = 1,           /* invalid argument; nothing was done */
    MGT_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    MGT_ERR_OOM = 3,           /* device allocation failed */
    MGT_ERR_NOT_CONVERGED = 4, /* ALI ended with non-finite populations */
    MGT_ERR_SINGULAR = 5,      /* a linear system could not be solved */
    MGT_ERR_TIMEOUT = 6,       /* a bounded device loop ran out */
    MGT_ERR_BOUNDS = 7,        /* a device index check failed */
    MGT_ERR_STATE = 8          /* call out of order (e.g. solve before trace) */
} mgt_status;

typedef enum {
    MGT_FP64 = 0,        /* every step of the formal solution in FP64 */
    MGT_FP32_MIXED = 1   /* opacity, optical depth and elimination in FP32, FP32
                            compensated accumulation of J-bar / Lambda*; the
                            trapezoid/erf switch is re-decided in FP64 next to
                            the threshold; SE and Ng stay FP64 */
} mgt_precision;

/*
 * Model inputs (Sec. 3.2, Listing 2: geometry.points.{position, velocity,
 * neighbors, n_neighbors}, geometry.boundary.boundary2point,
 * thermodynamics.{temperature.gas, turbulence.vturb2},
 * chemistry.species.abundance, uniform rays, LAMDA-style line data,
 * quadrature order).  All pointers are host pointers.
 */
typedef struct {
    int64_t n_points;            /* N >= 1 */
    const double *pos;           /* [N][3] m */
    const double *vel;           /* [N][3] m/s */
    const double *temp;          /* [N] K, > 0 */
    const double *vturb2;        /* [N] m^2/s^2, >= 0 (microturbulence squared) */
    const double *n_coll;        /* [N] m^-3 collision-partner density, >= 0 */
    const double *n_spec;        /* [N] m^-3 line-species density, > 0 */
    const int64_t *nbr_offsets;  /* [N+1] CSR offsets into nbrs, nbr_offsets[0] = 0 */
    const int32_t *nbrs;         /* [nbr_offsets[N]] neighbour indices in [0, N) */
    int32_t n_boundary;          /* number of boundary points */
    const int32_t *boundary;     /* [n_boundary] boundary point indices */
    int32_t n_rays;              /* R, even; every direction has its antipode */
    const double *dirs;          /* [R][3] unit vectors */
    int32_t n_quad;              /* Q Gauss-Hermite bins per line, 1..64 */
    double mol_mass_kg;          /* molecular mass of the line species, > 0 */
    double T_bg;                 /* background (CMB) temperature in K, >= 0 */
    int32_t n_levels;            /* L, 2..64 */
    const double *energy_J;      /* [L] level energies */
    const double *g;             /* [L] statistical weights */
    int32_t n_lines;             /* M radiative lines, 1..L*(L-1)/2 */
    const int32_t *up;           /* [M] upper level */
    const int32_t *lo;           /* [M] lower level */
    const double *A;             /* [M] Einstein A_ul, s^-1 */
    const double *freq_Hz;       /* [M] line centre frequencies */
    int32_t n_coll_trans;        /* K collisional transitions */
    const int32_t *cup;          /* [K] upper level */
    const int32_t *clo;          /* [K] lower level */
    const double *K_ul;          /* [K] downward rate coefficients, m^3/s */
} mgt_model_desc;

/* Numerical options of the formal solution (Sec. 4.3). */
typedef struct {
    double switch_threshold;  /* trapezoid below |Doppler shift|/dnu_bar, erf form at or
                                 above it; default 0.35 (Sec. 4.3) */
    int32_t width_mode;       /* dnu_bar of a segment: 0 = from the averaged temperature
                                 and turbulence (default), 1 = mean of the endpoint widths */
    int32_t lines_per_thread; /* FP32 kernel schedule: 0 = auto, else 4 or 8 */
    int32_t schedule;         /* formal-solve kernel: 0 = auto (4 where it applies, else 2),
                                 1 = per-thread gathers from global memory, 2 = bulk-copy staging
                                 of ray chunks in shared memory, the segment coefficients of a
                                 chunk computed once per bin in shared memory (registers capped
                                 for two blocks per SM), 3 = as 2 with one block per SM, 4 = as 2
                                 with each thread computing its own bin's coefficients in
                                 registers (only when the lines fit one group: lines <=
                                 lines_per_thread; MGT_ERR_ARG otherwise).  All staged schedules
                                 give bit-identical results */
    int32_t subdivisions;     /* 0 = the switch rule above (default); n = 1..256: every segment's
                                 optical depth by the trapezoidal rule over n equal pieces with
                                 chi^{ij}, the width and the comoving offset interpolated linearly
                                 (the reference of the Sec. 4.3 accuracy study; n = 1 is the plain
                                 trapezoidal rule) */
    int32_t pairs_per_batch;  /* 0 = trace every ray pair once and keep the rays (default);
                                 B > 0 = hold the rays of at most B pairs at a time: the formal
                                 solution traces and solves the pairs batch by batch, summing J-bar
                                 and Lambda* (for models whose rays do not fit in device memory);
                                 mgt_get_rays is then unavailable */
} mgt_solve_opts;

typedef struct {
    int64_t total_steps;      /* sum of half-ray lengths over all points and directions */
    int64_t n_stalls;         /* walks that ended without reaching a boundary point */
    int32_t max_half_ray;     /* longest half-ray (points) */
    double mean_half_ray;     /* total_steps / (N * R) */
    int64_t n_fp64_steps;     /* walk steps that FP32 error bounds could not settle and that
                                 were decided by the FP64 predicates themselves */
} mgt_trace_stats;

typedef enum { MGT_NG_NONE = 0, MGT_NG_CLASSICAL = 1, MGT_NG_ADAPTIVE = 2 } mgt_ng_mode;

typedef struct {
    int32_t mode;       /* mgt_ng_mode */
    int32_t n_steps;    /* classical: regular iterations between predictions (>= 2) */
    int32_t n_max;      /* adaptive: maximum iterates kept (3..16) */
} mgt_ng_opts;

typedef struct {
    int32_t n_iter;             /* regular ALI iterations */
    mgt_precision precision;    /* formal-solution precision */
    mgt_ng_opts ng;
} mgt_ali_opts;

typedef struct {
    int32_t iterations;         /* regular iterations done */
    int32_t ng_accepted;        /* Ng predictions used */
    double last_maxrel;         /* max relative population change of the last iteration */
} mgt_ali_stats;

/*
 * Create a model from host inputs (Sec. 3.2, Listing 2).  Validates every
 * input (finite values, unit directions with antipodes, indices in range,
 * N >= 1, sizes within the limits above); on MGT_ERR_ARG nothing is
 * allocated and *out is left NULL.  Level populations start at LTE
 * (compute_LTE_level_populations, Listing 3).  The Gauss-Hermite nodes
 * (set_quadrature) and the per-point line widths (Sec. 4.3, eq. line width)
 * are computed here.  `stream` orders the uploads.
 */
mgt_status mgt_model_create(mgt_model **out, const mgt_model_desc *desc, void *stream);

/* Free all device and host memory of a model (NULL is a no-op); waits for the
 * device first.  Its ray buffer goes back to the library's memory pool, which
 * returns its reserve to the driver when the last model on the device is
 * destroyed.  Always MGT_OK. */
mgt_status mgt_model_destroy(mgt_model *m);

/* Set the numerical options of mgt_formal_solve; NULL restores the defaults. */
mgt_status mgt_set_solve_opts(mgt_model *m, const mgt_solve_opts *opts);

/*
 * Trace every half-ray: for each point o and direction n, the chain of points
 * o -> c1 -> c2 ... through the neighbour graph (the tracer of the paper's
 * earlier Magritte papers, Sec. 2 / Sec. 4.1 cost ~ points per ray).  Rule:
 * from the current point c, candidates are neighbours m with
 * Z_m = (x_m - x_o).n > Z_c; the candidate with the smallest squared distance
 * to the ray line wins (ties to the smaller index); the walk ends on a
 * boundary point (included) or stalls when no candidate exists.  All
 * predicates are evaluated in FP64 without fused multiply-adds, so the point
 * lists are bit-exact with any implementation of the same expressions.
 * Most steps are settled by FP32 arithmetic with rigorous error bounds that
 * prove the FP64 predicates agree; the others are evaluated in FP64.
 * Stores the ray geometry on the device.  `stats` (host, may be NULL) is
 * filled after a stream synchronisation.  The walk's working memory (one
 * record slot per walk and step, a few GB for 10^5 points and 48 rays) comes
 * from a memory pool of this library, one per device, that keeps it reserved
 * for the next trace of any model; the reserve is returned to the driver when
 * the last model on that device is destroyed.  The model's ray buffer (16 B
 * per step) comes from the same pool and is returned to it by
 * mgt_model_destroy.
 */
mgt_status mgt_trace_rays(mgt_model *m, mgt_trace_stats *stats, void *stream);

/* Copy the traced rays to host memory: ray_off [R*N+1] (exclusive prefix of
 * half-ray lengths, direction-major: entry r*N+o) and idx [total_steps] point
 * indices in outward order.  Either pointer may be NULL.  The stream is
 * synchronised before returning.  MGT_ERR_STATE before mgt_trace_rays, and
 * while pairs_per_batch > 0 (rays are then held one pair batch at a time). */
mgt_status mgt_get_rays(mgt_model *m, int64_t *ray_off, int32_t *idx, void *stream);

/* Set level populations [N][L] (m^-3; host pointer), or LTE when pops is
 * NULL.  Resets the Ng history.  The stream is synchronised before returning,
 * so `pops` may be reused at once.  MGT_ERR_ARG for a non-finite or negative
 * entry, with the model unchanged. */
mgt_status mgt_set_populations(mgt_model *m, const double *pops, void *stream);

/* Copy the current level populations [N][L] to `pops` (host or device). */
mgt_status mgt_get_populations(mgt_model *m, double *pops, int on_device, void *stream);

/*
 * Radiation field from the current populations: per point and line the line
 * opacity and source function, per (point, ray pair, Gauss-Hermite bin, line)
 * the Doppler-shifted Gaussian opacity along the ray, segment optical depths
 * (Sec. 4.3: trapezoidal rule, or the semi-analytic erf form when the Doppler
 * shift across the segment reaches switch_threshold line widths), the
 * second-order two-point (Feautrier) system with background B_nu(T_bg) at both
 * ends, and its solution u and Lambda*_oo at the origin, reduced into
 *   Jbar[m][o]  = sum_pairs (2/R) sum_q w_q u,
 *   Lstar[m][o] = sum_pairs (2/R) sum_q w_q Lambda*_oo.
 * Jbar in W m^-2 Hz^-1 sr^-1, Lstar dimensionless; both [M][N] f64, line-major.
 * Either output may be NULL (the result stays on the device for
 * mgt_stat_equilibrium).  Requires mgt_trace_rays.
 */
mgt_status mgt_formal_solve(mgt_model *m, mgt_precision p, double *Jbar, double *Lstar,
                            int on_device, void *stream);

/*
 * The model's J-bar and Lambda* of its last formal solution (mgt_formal_solve
 * or a batched one), without solving again: [M][N] f64 each, host or device
 * as on_device says, either may be NULL.  MGT_ERR_STATE before any formal
 * solution.  Synchronises the stream for host outputs.
 */
mgt_status mgt_get_jbar(mgt_model *m, double *Jbar, double *Lstar, int on_device, void *stream);

/*
 * Statistical equilibrium (Listing 3, compute_level_populations; the paper's
 * Sec. 5 "solution of the statistical equilibrium equations"): per point the
 * steady state of the rate equations with radiative rates preconditioned by
 * Lambda* (down: A(1 - Lambda*) + B_ul J_eff, up: B_lu J_eff,
 * J_eff = Jbar - Lambda* S_old, floored at zero) and collisional rates in
 * detailed balance, normalised to n_spec; solved in FP64 by state reduction.
 * Uses the Jbar/Lambda* of the last mgt_formal_solve.  The result becomes the
 * current populations (the previous ones are kept for mgt_ng_accelerate) and
 * is copied to pops_out [N][L] (host) when not NULL.
 */
mgt_status mgt_stat_equilibrium(mgt_model *m, double *pops_out, void *stream);

/*
 * Ng-acceleration step after mgt_stat_equilibrium (Sec. 4.2, Appendix A).
 * Pushes the new populations (as fractions n_i/n_spec) into the history and
 * writes the maximum relative change against the previous populations to
 * *maxrel (host, may be NULL).  Classical mode: after n_steps regular
 * iterations the prediction sum_k c_k x_{k+1},
 * c = (R R^T)^-1 1 / (1^T (R R^T)^-1 1), replaces the populations.  Adaptive
 * mode: with m >= 3 iterates since the last prediction, the running prediction
 * is used when its maximum relative change is below that of the regular
 * iterates, or when m reaches n_max.  A prediction with a negative population
 * or a non-finite coefficient solve is not used (the history restarts).
 * *accepted (host, may be NULL) is 1 when a prediction replaced the
 * populations.  Synchronises the stream.
 */
mgt_status mgt_ng_accelerate(mgt_model *m, const mgt_ng_opts *opts, int *accepted, double *maxrel,
                             void *stream);

/*
 * Accelerated Lambda iteration (Listing 3, compute_level_populations with
 * Ng_acc and N_iter_max): from the current populations, opts->n_iter regular
 * iterations of {formal solution, statistical equilibrium, Ng step}.
 * Requires mgt_trace_rays.  Returns MGT_ERR_NOT_CONVERGED if the populations
 * become non-finite.  `stats` (host) may be NULL.
 */
mgt_status mgt_ali_solve(mgt_model *m, const mgt_ali_opts *opts, mgt_ali_stats *stats, void *stream);

/*
 * Synthetic image along a line of sight (Listing 3, compute_image_new(rx, ry,
 * rz, N_pix_x, N_pix_y), with the channels of compute_spectral_discretisation(
 * fmin, fmax, N)).  The paper gives no algorithm; the definition used here:
 *  - dir (host, [3]) is the unit direction toward the observer; the image
 *    plane has basis e1 = unit(a x dir), a the coordinate axis least aligned
 *    with dir (lowest index on ties), e2 = dir x e1; the square pixel grid
 *    covers the projections of all points (centre: mid-range of the
 *    projections, half-width: half the larger range); pixel (i, j) has the
 *    reference point p = (c1 - H + (i + 1/2) 2H/npx) e1 + (c2 - H + (j + 1/2)
 *    2H/npy) e2;
 *  - the pixel ray starts from the pixel's anchor, the point closest to the
 *    line (p, dir) (ties to the smaller index), and walks along -dir and +dir
 *    by the rule of mgt_trace_rays with distances to that line and Z measured
 *    from p; the ray runs from its far end to its near end;
 *  - channel f has observer-frame frequency fmin + f (fmax - fmin)/(nfreq - 1)
 *    (fmin for nfreq = 1) and sees the line nearest to it; a point moving with
 *    v sees the comoving frequency nu_f (1 - dir.v/c);
 *  - segment optical depths follow mgt_formal_solve (Sec. 4.3: trapezoid, or
 *    the semi-analytic erf form at or above switch_threshold); the intensity
 *    toward the observer is integrated with a source function linear in
 *    optical depth over each segment, from B_nu_f(T_bg) at the far end.
 * Uses the current populations.  out: [nfreq][npy][npx] f32 intensities in
 * W m^-2 Hz^-1 sr^-1, host or device per on_device.  Pixel rays are traced on
 * the first call for a (dir, npx, npy) and kept.  The image is computed in
 * FP32.  MGT_ERR_ARG for a non-unit or non-finite dir, npx * npy > 2^26,
 * nfreq outside 1..65536 or not 0 < fmin <= fmax.
 */
mgt_status mgt_image(mgt_model *m, const double dir[3], int32_t npx, int32_t npy, int32_t nfreq, double fmin,
                     double fmax, float *out, int on_device, void *stream);

/*
 * Gradient of a loss of the image with respect to the per-point fields
 * (the hand-written adjoint of mgt_image; the paper has no counterpart, its
 * differentiation is asked for by this library's users).  grad_out [nfreq][npy]
 * [npx] f32 holds dL/dI (host or device per on_device).  Outputs (same memory
 * kind, any may be NULL): g_logT [N] = dL/d log T, g_logn [N] = dL/d log n_spec,
 * g_vel [N][3] = dL/dv in (W m^-2 Hz^-1 sr^-1)^-1 L per m/s.  Level populations
 * are held as fractions of n_spec (so the opacity scales with n_spec and the
 * source function does not); T enters through the Doppler width.  The branch
 * of each segment's optical depth (trapezoid or erf form) is held fixed.
 * Rays longer than 4096 segments give MGT_ERR_ARG.  Arguments as mgt_image.
 */
mgt_status mgt_image_adjoint(mgt_model *m, const double dir[3], int32_t npx, int32_t npy, int32_t nfreq,
                             double fmin, double fmax, const float *grad_out, double *g_logT, double *g_logn,
                             double *g_vel, int on_device, void *stream);

/*
 * The pixel rays of mgt_image for (dir, npx, npy), copied to host memory:
 * anchor [npx*npy], ray_off [npx*npy+1] (offsets into pts), pts [ray_off[npix]]
 * point indices, far end first.  Any pointer may be NULL.
 */
mgt_status mgt_image_rays(mgt_model *m, const double dir[3], int32_t npx, int32_t npy, int32_t *anchor,
                          int64_t *ray_off, int32_t *pts, void *stream);

/*
 * Replace per-point fields (Sec. 3.2, Listing 2 inputs): temp [N] K, n_spec
 * [N] m^-3, vel [N][3] m/s; NULL leaves a field unchanged.  Level populations
 * keep their fractions n_i / n_spec.  Host inputs are validated (finite,
 * T > 0, n_spec > 0); device inputs (on_device nonzero) are not.  Changing T or
 * v makes the traced rays stale: mgt_trace_rays must run again before
 * mgt_formal_solve.  Pixel rays of mgt_image stay valid (positions do not
 * change).
 */
mgt_status mgt_set_point_fields(mgt_model *m, const double *temp, const double *n_spec, const double *vel,
                                int on_device, void *stream);

/*
 * Recursive re-meshing of a point cloud (Sec. 4.1), a pre-processing step
 * before mgt_model_create.  Starting from the bounding box of all points, a
 * box whose tracer variation 2 (rho_max - rho_min)/(rho_max + rho_min)
 * (Sec. 4.1, eq. subdivision criterion) exceeds r_max, below recursion level
 * max_level, is divided into 8 equal boxes (a point goes to the upper half of
 * an axis when its coordinate is >= the midpoint) and each non-empty part is
 * cropped to the bounding box of its points; every other box becomes one
 * point at its centre.  Then evenly spaced boundary points are added on the
 * surface of the outermost box: the surface nodes of the n_side^3 lattice
 * over it (6 n_side^2 - 12 n_side + 8 points).
 *   pos [N][3], rho [N] > 0: host inputs.
 *   out_pos [capacity][3], out_boundary [capacity] (may be NULL): host
 *   outputs, box centres first (level by level), then the boundary points
 *   (flag 1).  *n_out receives the number of output points; with out_pos NULL
 *   only that count is computed, and a capacity below it gives MGT_ERR_ARG.
 * Computed on the GPU in FP64 (box bounds and centres are exact).
 */
mgt_status mgt_remesh(int64_t n_points, const double *pos, const double *rho, double r_max, int32_t max_level,
                      int32_t n_side, double *out_pos, uint8_t *out_boundary, int64_t capacity, int64_t *n_out,
                      void *stream);

/*
 * Ng extrapolation without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory -- an application whose own allocator owns the whole GPU (a pool
 * carved out at start-up that nothing else may grow), or an iteration loop
 * that must not call cudaMalloc/cudaFree because those calls can synchronise
 * the device and stall the caller's other streams.
 *
 * Computes the prediction of mgt_ng_accelerate from iterates the caller holds:
 * with r_k = x_{k+1} - x_k (k = 0..n_iterates-2) and G = R R^T,
 * c = G^-1 1 / (1^T G^-1 1) and prediction = sum_k c_k x_{k+1}.
 *   n_iterates  2..MGT_NG_NOALLOC_MAX_ITERATES; larger counts are rejected
 *               with MGT_ERR_ARG (the scratch holds at most 16 residuals)
 *   iterates    device, [n_iterates][len] f64 row-major, oldest first
 *   len         elements per iterate, >= 1
 *   prediction  device, [len] f64 (caller-owned; a prediction overlapping the
 *               iterates is rejected with MGT_ERR_ARG)
 *   coef        host, [n_iterates-1] coefficients c_k, may be NULL
 *   n_negative  host, number of negative prediction entries, may be NULL
 * Both device buffers must be on the current device.  MGT_ERR_SINGULAR (the
 * Gram matrix cannot be solved) leaves `prediction` untouched.  Synchronises
 * `stream`.
 *
 * Working memory is one static device array of MGT_NG_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits; the call
 * itself allocates nothing on the device.  The first call on a device does a
 * one-time set-up, looking up that device's address of the array
 * (cudaGetSymbolAddress, retried by the next call if it fails), so make that
 * first call before any stream capture.  All calls share the one array, which
 * keeps the last call's contents (each call clears what it accumulates):
 * calls that can overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.
 */
#define MGT_NG_NOALLOC_MAX_ITERATES 17
#define MGT_NG_NOALLOC_SCRATCH_BYTES 157952
mgt_status mgt_ng_extrapolate_noalloc(int32_t n_iterates, const double *iterates, int64_t len,
                                      double *prediction, double *coef, int64_t *n_negative, void *stream);

/*
 * Schedule autotuner.  Times the formal solution of model m in precision p
 * with every candidate (schedule, lines_per_thread) -- schedules 1, 2, 3, and 4
 * where the lines fit one group (only 0, the automatic staged choice that
 * batched launches make, when staged_only != 0) times 4 or 8 lines per thread
 * (FP32-mixed; 4 only in FP64) -- as the median of `reps`
 * (1..100) launches after one warm-up, with CUDA events on `stream`, and sets
 * the fastest in the model's options.  Needs mgt_trace_rays and every ray
 * pair resident (pairs_per_batch = 0); overwrites the model's J-bar and
 * Lambda*.  `res` (host, may be NULL) receives the choice and the timings.
 * Synchronises the stream.
 */
typedef struct {
    int32_t schedule;          /* chosen schedule (also set in the model's options) */
    int32_t lines_per_thread;  /* chosen lines per thread (likewise) */
    int32_t n_tried;           /* candidates timed */
    int32_t schedules[8];      /* candidate i: schedule */
    int32_t lines[8];          /* candidate i: lines per thread */
    float ms[8];               /* candidate i: median time of one formal solution, ms */
} mgt_autotune_result;
mgt_status mgt_autotune(mgt_model *m, mgt_precision p, int32_t staged_only, int32_t reps, mgt_autotune_result *res,
                        void *stream);

/*
 * Batches: the per-iteration work of many models (uneven point, level and ray
 * counts) in single launches.  The paper solves one model at a time; a batch
 * keeps the GPU full with models too small to fill it alone.
 *
 * mgt_batch_create borrows n_models (1..65536) distinct models (host array
 * of handles, copied): they must stay alive and on the current device while
 * the batch is used, be traced (mgt_trace_rays) and hold every ray pair
 * (pairs_per_batch = 0); otherwise MGT_ERR_STATE / MGT_ERR_ARG and *out stays
 * NULL.  Limits: bins x line groups of one origin <= 256 threads, and the
 * statistical-equilibrium workspace of 4 points (8 (L^2 + 3L + 2 Mpad) bytes
 * each) within 227 KB.  Each model's lines_per_thread option (4 or 8, 0 = the
 * automatic choice; e.g. set by mgt_autotune with staged_only) picks its
 * schedule inside the batched formal solution; schedule and precision options
 * do not apply (batched solutions are FP32-mixed with the staged schedule).
 * Options, rays or populations of a model may change between batch calls:
 * every call rebuilds the batch's argument tables and uploads them when they
 * changed.
 *
 * mgt_batch_formal_solve: line data of every model from its current
 * populations, then J-bar and Lambda* of every model (the values of
 * mgt_formal_solve in FP32-mixed with schedule 2 and the model's lines per
 * thread) in one persistent launch per class of models (one CTA width -- bins
 * x line groups of one origin, rounded to warps -- and, within it, models
 * whose lines fit one group, which run schedule 4's per-thread coefficients,
 * apart from the rest): CTAs take (model, origin, line block) items from a
 * counter, models with the most work per item first.
 * mgt_batch_stat_equilibrium: the statistical equilibrium of every point of
 * every model in one launch (the values of mgt_stat_equilibrium).
 * mgt_batch_iterate: n_iter ALI iterations of every model.  The first call
 * captures {line data, formal solution, statistical equilibrium} in a CUDA
 * graph, and each iteration replays it; then, when ng->mode != MGT_NG_NONE or
 * stats is not NULL, each model takes its Ng step as mgt_ng_accelerate would,
 * all models phase by phase (two stream synchronisations per iteration for
 * the whole batch).  ng (host) may be NULL (no Ng);
 * stats (host, [n_models] in the caller's order) may be NULL.  The results
 * equal those of mgt_ali_solve per model with FP32-mixed precision and
 * schedule 2.  Returns
 * MGT_ERR_NOT_CONVERGED when a model's populations became non-finite.
 * All three are stream-ordered; device errors surface as for the models.
 */
typedef struct mgt_batch mgt_batch;
typedef struct {
    int32_t n_models;
    int64_t fs_items;          /* (model, origin, line block) items of the formal solution */
    int32_t fs_grid;           /* CTAs of the persistent formal-solution launches, summed */
    int32_t fs_threads;        /* threads per CTA of the widest launch */
    int64_t fs_smem_bytes;     /* largest dynamic shared memory per CTA */
    int64_t se_blocks;         /* CTAs of the statistical-equilibrium launch */
    int32_t graph_kernels;     /* kernels per replay of the captured iteration (0 before the
                                  first mgt_batch_iterate) */
    int32_t fs_launches;       /* formal-solution launches: one persistent launch per class of
                                  models, plus one per model launched on its own */
    int32_t fs_solo;           /* models launched on their own (at least 8 waves of CTAs of their
                                  persistent class: the single-model kernel, the same values) */
} mgt_batch_layout;
mgt_status mgt_batch_create(mgt_batch **out, mgt_model *const *models, int32_t n_models, void *stream);
mgt_status mgt_batch_destroy(mgt_batch *b);
mgt_status mgt_batch_formal_solve(mgt_batch *b, void *stream);
mgt_status mgt_batch_stat_equilibrium(mgt_batch *b, void *stream);
mgt_status mgt_batch_iterate(mgt_batch *b, int32_t n_iter, const mgt_ng_opts *ng, mgt_ali_stats *stats,
                             void *stream);
/* Launch layout, and (order, host [n_models], may be NULL) the caller's index
 * of each model in launch order. */
mgt_status mgt_batch_get_layout(const mgt_batch *b, mgt_batch_layout *layout, int32_t *order);

/* Wait for the model's work on `stream` and report any device-side error. */
mgt_status mgt_sync(mgt_model *m, void *stream);

/* Model sizes: any pointer may be NULL. */
mgt_status mgt_model_sizes(const mgt_model *m, int64_t *n_points, int32_t *n_rays, int32_t *n_levels,
                           int32_t *n_lines, int32_t *n_quad);

/* Number of kernels this library has launched in the process so far (all
 * models, all threads); library kernels such as CUB scans are not counted. */
mgt_status mgt_launch_count(int64_t *count);

/*
 * Per-kernel timing, for measurement (the paper has no counterpart: it times
 * whole runs).  mgt_kernel_timing(1) clears the totals and starts recording a
 * CUDA event before and after each instrumented kernel launch of this library
 * (line data, ray walk and compaction, formal solution, statistical
 * equilibrium, Ng), on the launch's own stream; launches on a capturing stream
 * are not recorded.  mgt_kernel_timing(0) stops recording.
 * mgt_kernel_times waits for the recorded events, adds their durations to the
 * per-kernel totals and returns up to `capacity` of them in `out` (host,
 * caller-owned) with their number in *n_out (the number of kernels timed so
 * far, which may exceed `capacity`).  Timing adds two event records per launch.
 */
typedef struct {
    char name[48];          /* kernel name, NUL-terminated */
    int64_t launches;       /* launches recorded */
    double total_ms;        /* summed event-to-event durations */
    double bytes;           /* summed algorithmic bytes (least the kernel must read
                               and write) of the launches, 0 where not stated */
} mgt_kernel_time;
mgt_status mgt_kernel_timing(int32_t enable);
mgt_status mgt_kernel_times(int32_t capacity, mgt_kernel_time *out, int32_t *n_out);

/* Thread-local description of the last non-OK status of this thread. */
const char *mgt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MAGRITTE_GPU_H */
