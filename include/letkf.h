/*
 * letkf.h - C ABI of the GB300 local ETKF control law (arXiv:1310.5954).
 *
 * One context = one adaptive-optics system: its geometry, its filter model and
 * its ensemble, all resident on one GPU.  The filter is the local ensemble
 * transform Kalman filter of Sect. 2.3: every frame, each estimation domain
 * runs an independent ensemble-transform analysis against the slopes of its
 * observation region, then every member is propagated by the AR(1) model of
 * Sect. 2.1.
 *
 * Model (Sect. 2.1, Sect. 3):
 *   state     x = [phi_k ; phi_{k-1}] on the valid actuators (Fried geometry),
 *             n = 2 * n_act, rows: all actuators of the first instant, then the
 *             second, valid actuators numbered in row-major grid order;
 *   dynamics  x_{k+1} = A1 x_k + [v_k ; 0],  A1 = [[a I, a2 I], [I, 0]] (AR(2); a2 = 0: AR(1)),
 *             v ~ N(0, Q);
 *   slopes    y_k = C x_k + w_k,  C = [0 D] (obs_block = 1) or [D 0] (obs_block = 0),
 *             D the Fried difference operator, p = 2 * n_subv, all x-slopes then
 *             all y-slopes of the valid subapertures in row-major grid order;
 *             R = sigma^2 I.
 * Update (ETKF with symmetric square root, Sect. 2.2, refs. [8-10], [14]):
 *   G = Y'^T R^-1 Y',  w_bar = [(m-1)I + G]^-1 Y'^T R^-1 (y - y_bar),
 *   T = sqrt(m-1) [(m-1)I + G]^(-1/2),  X_a = x_bar 1^T + X' (w_bar 1^T + T),
 * per domain, on the domain's own actuators (both instants) with the slopes
 * of its observation region.
 *
 * Conventions for every entry point:
 *   - Every function returns a letkf_status and never throws or aborts.
 *   - Device buffers are plain device pointers owned by the caller; the
 *     library reads or writes them in stream order on the context's stream and
 *     never keeps them after the call's work completes.
 *   - Element type of every device buffer ("state type"): double when the
 *     context's precision is LETKF_PREC_FP64, float otherwise.  Matrices are
 *     row-major with no padding: an (r x m) buffer holds element (i, j) at i*m + j.
 *   - Work is asynchronous.  Errors detected on the device (non-finite input,
 *     a bounded wait that ran out, an iteration that hit its limit) are
 *     latched in the context and reported by letkf_sync (and by the next
 *     letkf_sync only: reading clears them).
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef LETKF_H
#define LETKF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct letkf_ctx letkf_ctx;

typedef enum letkf_status {
    LETKF_OK = 0,
    LETKF_EINVAL = -1,      /* invalid argument or unsupported configuration */
    LETKF_ENOMEM = -2,      /* device or host allocation failed */
    LETKF_ECUDA = -3,       /* a CUDA runtime call failed */
    LETKF_ETIMEOUT = -4,    /* a bounded device-side wait gave up */
    LETKF_ENONFINITE = -5,  /* non-finite slopes: that frame was rejected, state unchanged */
    LETKF_ESTATE = -6,      /* call out of order (e.g. analyze twice without a forecast) */
    LETKF_ENOCONV = -7,     /* a domain's eigensolve (plain path: Jacobi sweeps) or inverse square
                               root (fused and global paths: Newton-Schulz steps) hit its iteration
                               limit (result still written) */
    LETKF_ESCRATCH = -8,    /* the problem does not fit letkf_analyze_static's fixed scratch */
    LETKF_EBUSY = -9        /* refused for now (letkf_serve.h): HBM budget or frame queue full */
} letkf_status;

typedef enum letkf_precision {
    LETKF_PREC_FP64 = 0,    /* everything in FP64 (plain path only) */
    LETKF_PREC_FP32 = 1,    /* everything in FP32 */
    LETKF_PREC_MIXED = 2    /* fused path only: BF16 tensor-core products with FP32 accumulation
                               (single-BF16 Gram, split-BF16 Newton-Schulz and transform), mean
                               weights refined in FP32 against the exact slopes, mean updates
                               summed in compensated FP32 (twice the working precision); small
                               domains (simt_q_max) in FP32 on the CUDA cores */
} letkf_precision;

typedef enum letkf_path {
    LETKF_PATH_PLAIN = 0,   /* one kernel per stage, one CTA per domain */
    LETKF_PATH_FUSED = 1,   /* one persistent kernel per frame over all domains */
    LETKF_PATH_GLOBAL = 2   /* global ETKF (Sect. 2.2): one domain, the whole pupil, for large
                               ensembles (2 <= m <= 4096, FP32 only): the Gram, the Newton-Schulz
                               inverse square root, the transform and the process-noise draw as
                               split-BF16 tensor-core products; dom_sub and halo are ignored */
} letkf_path;

/* Differential pistons between domains (Sect. 3.1, discussion of Fig. 3; Sect. 5).  The domains
 * are analysed independently, so the stitched estimate carries one piston error per domain.  After
 * each frame one piston per domain is fitted by least squares to the slope residual y_k - D x_hat of
 * the prediction, on the subapertures whose corners lie in more than one domain, with the free
 * constant of each connected group of domains chosen so that the correction adds no piston; the
 * prediction returned is x_hat plus each actuator's domain piston.  The operator is formed on the
 * host at create time (FP64 Cholesky of the domains' normal matrix, n_dom^2 elements on the
 * device).  A rejected frame (non-finite slopes) is returned uncorrected. */
typedef enum {
    LETKF_PISTON_OFF = 0,       /* no correction */
    LETKF_PISTON_OUTPUT = 1,    /* correct the returned prediction only (post-processing) */
    LETKF_PISTON_IN_LOOP = 2    /* also shift every member of both instants of each domain's
                                   owned actuators, so the next analysis starts corrected */
} letkf_piston;

typedef struct letkf_params {
    int n_sub;                      /* N: subapertures across; (N+1)^2 actuator grid (Fried) */
    const unsigned char* sub_valid; /* host N*N row-major validity mask, or NULL: circular pupil
                                       rule (a subaperture is valid when >= half of its area,
                                       sampled on a 20x20 midpoint grid, lies in the annulus
                                       [obstruction*N/2, N/2] pitches around the grid centre) */
    double obstruction;             /* central obstruction ratio, used when sub_valid is NULL */
    double ar1_a;                   /* AR(1) coefficient a of A1, |a| < 1 */
    int obs_block;                  /* 1: slopes see the second instant (C = [0 D]); 0: the first */
    const double* q_sqrt;           /* host n_act*n_act row-major L with Q = L L^T (lower
                                       triangular or dense), or NULL for white noise q_white */
    double q_white;                 /* process-noise std when q_sqrt is NULL */
    const double* p0_sqrt;          /* host n_act*n_act factor of the stationary covariance of
                                       one phase instant, for the initial ensemble; NULL means
                                       L / sqrt(1 - a^2) */
    double sigma;                   /* slope-noise std: R = sigma^2 I */
    int m;                          /* ensemble size, 2 <= m <= 256 (plain FP64: <= 112,
                                       plain FP32: <= 160) */
    int dom_sub;                    /* estimation-domain side in subapertures (>= 1) */
    int halo;                       /* observation halo in subapertures (>= 0) */
    int precision;                  /* letkf_precision */
    int path;                       /* letkf_path */
    unsigned long long seed;        /* key of the Philox4x32-10 draws (initial ensemble,
                                       process noise) */
    int device;                     /* CUDA device ordinal */
    void* stream;                   /* cudaStream_t borrowed from the caller (NULL: default) */
    double ar2_a;                   /* AR coefficient a2 of the second instant (Sect. 2.1, "AR 1 or
                                       AR 2"): A1 = [[a I, a2 I], [I, 0]]; 0 is the AR(1) model.
                                       The AR(2) must be stationary: |a2| < 1, a + a2 < 1,
                                       a2 - a < 1 (for a2 = 0: |a| < 1) */
    int piston;                     /* letkf_piston: differential-piston removal between domains
                                       (letkf_step and the server only) */
    int simt_q_max;                 /* fused path, m <= 127: a domain whose smaller Gram dimension
                                       min(p_loc, m) is at most this takes an FP32 analysis on the
                                       CUDA cores (Newton-Schulz on that q x q form) instead of
                                       tensor-core products; 0 selects the default (32), a negative
                                       value turns it off, at most 128.  Lowered at create time to
                                       what shared memory holds. */
    int dom_offset;                 /* shift of the block grid, in subapertures along both axes,
                                       0 <= dom_offset < dom_sub: block (I, J) spans subaperture
                                       rows [dom_sub I - dom_offset, dom_sub (I + 1) - dom_offset)
                                       and columns likewise (the second partition of the two
                                       parallel local filters of Sect. 5; letkf_step_pair) */
} letkf_params;

typedef struct letkf_info {
    int n_sub, n_act, n_subv, n, p, m;
    int n_domains;
    int n_loc_max;                  /* largest number of state rows a domain updates */
    int p_loc_max;                  /* largest number of slopes a domain observes */
    int state_bytes;                /* 8 (FP64) or 4 */
    int precision, path;
    unsigned long long frame;       /* frames forecast so far */
    size_t device_bytes;            /* device memory held by the context */
    int n_domains_observing;        /* domains with at least one observed subaperture */
    long long sum_p_loc;            /* total slopes over domains (each counted once per domain) */
    long long sum_n_loc;            /* total state rows over domains (= n) */
    int simt_q;                     /* fused path: domains with min(p_loc, m) <= simt_q take the FP32
                                       SIMT analysis (letkf_params.simt_q_max); 0: none */
    int n_domains_simt;             /* observing domains that take it */
} letkf_info;

/*
 * letkf_create: build the geometry (Sect. 3: Fried actuators on the corners
 * of the valid subapertures), the domain decomposition (Sect. 2.3: dom_sub x
 * dom_sub blocks of subapertures own their actuators; the observation region is
 * the block grown by `halo` subapertures), the device tables, and the initial
 * ensemble (Sect. 2.2): second instant = P0 xi0, first instant = a * second + L xi1,
 * with xi0, xi1 Philox normals (stream 0, frames 0 and 1).  The new context is
 * in the forecast phase at frame 0.  *out is set to NULL on failure.
 */
int letkf_create(const letkf_params* params, letkf_ctx** out);

/*
 * letkf_footprint: device bytes a context created with these parameters holds (geometry
 * tables, the two ensemble buffers, process-noise buffers and the path's scratch; equal to
 * letkf_info.device_bytes after letkf_create), computed on the host without touching a GPU.
 * Creation itself briefly needs up to 2 * n_act^2 * 8 more bytes for the FP64 factors.
 * LETKF_EINVAL for parameters letkf_create would reject on the host.
 */
int letkf_footprint(const letkf_params* params, unsigned long long* bytes);

/*
 * letkf_fused_plan: the fused path's launch plan for these parameters, computed on the host
 * without a device (the same computation letkf_create makes): the dynamic shared memory of the
 * fused kernel, the SIMT threshold in use (simt_q_max lowered until its workspace fits, 0 in the
 * dual form m >= 128) and how many observing domains take the SIMT analysis.  LETKF_EINVAL for
 * invalid parameters, a path other than LETKF_PATH_FUSED, or a system the fused kernel does not
 * hold (more than 128 slopes per domain).  Outputs are host ints owned by the caller.
 */
int letkf_fused_plan(const letkf_params* params, int* smem_bytes, int* simt_q, int* n_domains_simt);

/*
 * letkf_domain_tables: the geometry and domain decomposition letkf_create would build for these
 * parameters (Sect. 2.3; host only, no GPU).  sizes is filled first; every array may be NULL and
 * otherwise holds: own_off[n_dom + 1] / own[own_total] the valid actuators each domain updates
 * (both instants), obs_off[n_dom + 1] / obs_sub[obs_total] its observed valid subapertures,
 * halo_off[n_dom + 1] / halo[halo_total] the valid actuators at the corners of those
 * subapertures (the rows of the observed instant its analysis reads), block[n_dom] its block
 * index I * blocks_per_side + J.  Indices are valid-actuator / valid-subaperture numbers.
 */
typedef struct letkf_domain_sizes {
    int n_sub, n_act, n_subv, n_dom, blocks_per_side;
    int own_total, obs_total, halo_total;
} letkf_domain_sizes;

int letkf_domain_tables(const letkf_params* params, letkf_domain_sizes* sizes, int* own_off, int* own,
                        int* obs_off, int* obs_sub, int* halo_off, int* halo, int* block);

/*
 * letkf_piston_operator: the least-squares operator of the differential-piston removal
 * (letkf_piston) for these parameters, on the host (no GPU): *n_dom is set first; K, if not
 * NULL, receives n_dom * n_dom doubles, row-major, with delta = K g where
 * g_l = sum over boundary rows r of (D P)[r, l] (y - D x_hat)[r] (domain numbering as in
 * letkf_domain_tables).  K = Pi M^+ with M = (D P)^T (D P) and Pi the projection that makes each
 * connected group's correction add no piston.  LETKF_EINVAL for parameters letkf_create rejects.
 */
int letkf_piston_operator(const letkf_params* params, double* K, int* n_dom);

/*
 * letkf_gemm_selftest (tests): C (M x N, row-major) = A (M x K) B (N x K)^T with A, B FP32 row-major
 * device arrays, through the library's tiled tensor-core GEMM (BF16 operands; split = 1 adds the
 * two low-part products, ~2^-16 relative per element; bn = 64, 128 or 256 columns per CTA tile).  With
 * b_mn = 1 (bn = 64 only) B is given as K x N row-major and C = A B, the tiles of B read MN-major.
 * Ordered on `stream` and synchronised.  LETKF_ETIMEOUT if a bounded wait inside gave up.
 */
int letkf_gemm_selftest(const float* A, const float* B, float* C, int M, int N, int K, int split, int bn,
                        int b_mn, void* stream);

/*
 * letkf_global_stats (LETKF_PATH_GLOBAL): Newton-Schulz steps taken by the last analysis (the
 * first, product-free step included; each further step is three products) and the spectral bound
 * s = 1 + ||G||_F / (m-1) the iteration was scaled by.  Synchronises the context's stream;
 * LETKF_ESTATE on other paths.
 */
int letkf_global_stats(letkf_ctx* ctx, int* ns_steps, double* s_bound);

/*
 * letkf_set_capture (tests, LETKF_PATH_FUSED): from the next analysis on, the analysis of domain
 * `domain` (numbering of letkf_domain_tables) also writes what it computed for the transform of
 * Sect. 2.2-2.3 (w_bar = [(m-1)I + G]^-1 Y'^T R^-1 d and T = sqrt(m-1) [(m-1)I + G]^(-1/2)) into
 * cap_dev, a caller-owned device array of cap_floats FP32 elements, at least
 * 8 + m + max(m * m, 2 * p_loc_max * m).  Layout: [0] form (0: m x m form on the tensor cores,
 * 1: observation-space form on the tensor cores, 2: m x m form on the CUDA cores, 3:
 * observation-space form on the CUDA cores), [1] q (m for forms 0 and 2, the domain's slope
 * count p for 1 and 3), [2] the conditioning bound s = 1 + ||G||_F/(m-1), [3] Newton-Schulz
 * steps, [4..7] zero; then w_bar (m); then for forms 0 and 2 T (m x m, row-major), for forms 1
 * and 3 W (q x m) and M = (I + Z)^-1 W (q x m), row-major, with T = I - W^T M.  A domain the
 * frame skips (no observation, rejected frame) writes nothing.  cap_dev == NULL stops the
 * capture.  LETKF_ESTATE on other paths, LETKF_EINVAL for a domain out of range or too small an
 * array.  The array must stay allocated while captured frames run.
 */
int letkf_set_capture(letkf_ctx* ctx, int domain, float* cap_dev, long long cap_floats);

/*
 * letkf_set_domain_mask (fault injection, local paths): active[d] == 0 skips domain d from the
 * next analysis on: its actuators keep their forecast, as a domain without observations does
 * (Sect. 2.3; a lost node of a distributed implementation).  active has n_dom entries in the
 * numbering of letkf_domain_tables; NULL restores every domain.  Synchronises the stream;
 * LETKF_EINVAL on the global path.
 */
int letkf_set_domain_mask(letkf_ctx* ctx, const unsigned char* active);

/* letkf_destroy: release everything; NULL is accepted.  Synchronises the stream. */
int letkf_destroy(letkf_ctx* ctx);

int letkf_get_info(const letkf_ctx* ctx, letkf_info* out);

/* Host copies of the validity masks: sub_valid N*N, act_valid (N+1)*(N+1); either may be NULL. */
int letkf_get_geometry(const letkf_ctx* ctx, unsigned char* sub_valid, unsigned char* act_valid);

/*
 * letkf_analyze: local ETKF analysis (Sect. 2.3) of the current forecast
 * ensemble with slopes y_dev (p elements, state type).  sigma > 0 replaces the
 * noise std from this frame on; sigma <= 0 keeps it.  Requires the forecast
 * phase (else LETKF_ESTATE); leaves the context in the analysis phase.  A frame
 * with a non-finite slope is rejected on the device: the ensemble is left
 * unchanged, the following letkf_forecast is skipped as well, and letkf_sync
 * reports LETKF_ENONFINITE.
 */
int letkf_analyze(letkf_ctx* ctx, const void* y_dev, double sigma);

/*
 * letkf_forecast: AR(1) forecast of every member (Sect. 2.1): first instant
 * <- a * first + v, second instant <- first.  v_dev: n_act x m perturbations
 * (state type), or NULL to draw v = L xi with xi Philox normals (stream 1, frame
 * = the context's frame counter).  Advances the frame counter.  Allowed in both
 * phases (a forecast without analysis is a prediction with no data).
 */
int letkf_forecast(letkf_ctx* ctx, const void* v_dev);

/*
 * letkf_step: one filter frame in the prediction form of Eq. 1: analysis with
 * y_k, then forecast with internally drawn noise; writes x_hat(k+1|k), the
 * ensemble mean of the first instant (n_act elements, state type), to xpred_dev
 * (may be NULL).  Requires the forecast phase.
 */
int letkf_step(letkf_ctx* ctx, const void* y_dev, double sigma, void* xpred_dev);

/*
 * letkf_step_pair: two local ETKFs run together on the same slopes, with two different domain
 * partitions (Sect. 5), and their predictions combined: one letkf_step of each filter, both
 * filters' domains analysed in one launch of the fused kernel, then xpred_dev (n_act elements,
 * FP32, required) = (x_hat_a + x_hat_b) / 2.  Each filter keeps its own ensemble, noise draws and
 * frame counter; neither sees the other's estimate (the combination is the output only).  The
 * partitions differ by letkf_params.dom_offset (e.g. 0 and dom_sub / 2), the noise streams by
 * the seed.  Requirements (else LETKF_EINVAL): two distinct fused-path contexts on the same
 * device and the same stream, the same pupil (n_act and p), differential pistons off; both in
 * the forecast phase (else LETKF_ESTATE).  A frame with a non-finite slope is rejected by both.
 */
int letkf_step_pair(letkf_ctx* a, letkf_ctx* b, const void* y_dev, double sigma, void* xpred_dev);

/* Ensemble as an n x m matrix (state type) and the frame counter (either may be NULL). */
int letkf_get_state(letkf_ctx* ctx, void* x_dev, unsigned long long* frame);

/* Replace the ensemble (n x m, state type) and frame counter; puts the context in the forecast
 * phase.  With letkf_get_state this checkpoints and resumes a filter bit for bit. */
int letkf_set_state(letkf_ctx* ctx, const void* x_dev, unsigned long long frame);

/*
 * letkf_set_graph: run letkf_step of a fused-path context as a CUDA graph launch (enable = 1) or
 * as separate launches (0, the default).  Per frame parity the graph holds the
 * fused kernel and, on a forked branch, the next frame's noise draw (normals kernel and GEMM);
 * each call updates the kernel nodes' arguments (slopes, output, frame counter, ensemble
 * buffers) and launches it on the context's stream.  Results are identical either way.  If the
 * step cannot be captured, the context goes back to separate launches (letkf_get_graph reads
 * the current mode).
 * Plain-path contexts: enable = 1 is LETKF_EINVAL, 0 is accepted.  Synchronises the stream.
 */
int letkf_set_graph(letkf_ctx* ctx, int enable);
int letkf_get_graph(const letkf_ctx* ctx, int* enabled);

/*
 * Launch tuning of the fused path (the paper has no counterpart).  Neither knob changes any
 * result: fused_grid is the number of CTAs of the fused kernel for this context (0: one per SM,
 * capped at the number of domains; at most the SM count), graph is letkf_set_graph's mode.
 * letkf_autotune times `frames` letkf_step calls with the slopes y_dev (p elements) for each
 * candidate (one CTA per SM, or the fewest CTAs taking the same number of rounds of domains;
 * graph off or on), keeps the fastest and reports it and its milliseconds per frame (either
 * pointer may be NULL).  The context's ensemble, frame counter, noise std and latched status
 * are restored afterwards.  Plain-path contexts: tuning is fixed at {0, 0}.
 */
typedef struct letkf_tuning {
    int fused_grid;
    int graph;
} letkf_tuning;

int letkf_get_tuning(const letkf_ctx* ctx, letkf_tuning* out);
int letkf_set_tuning(letkf_ctx* ctx, const letkf_tuning* tuning);
int letkf_autotune(letkf_ctx* ctx, const void* y_dev, int frames, letkf_tuning* best, double* ms_per_frame);

/* Wait for the context's queued work and return the first latched device error, clearing it. */
int letkf_sync(letkf_ctx* ctx);

/*
 * letkf_analyze_static: the analysis of letkf_analyze on a plain-path context, without any
 * allocation, for callers that cannot call the CUDA allocator while they run, e.g. a real-time
 * controller that reserves its device memory before its loop and must not block on or fail in
 * an allocation with a frame deadline pending.  The paper has no counterpart.
 *
 * Reads the context's current forecast ensemble and the slopes y_dev (p elements, state type),
 * and writes the analysis ensemble to xa_dev (n x m, state type, caller-owned).  It leaves the
 * context's ensemble, phase and frame counter untouched; a non-finite slope makes xa_dev a
 * copy of the forecast and latches LETKF_ENONFINITE for letkf_sync.  sigma > 0 is used for
 * this call only.
 *
 * All intermediate storage comes from one fixed 16 MiB array per GPU that exists while the
 * library is loaded (every GPU that loads the library holds it).  A problem needing more
 * returns LETKF_ESCRATCH before any work is queued (the ELT-class 80x80, m = 100 system needs
 * ~43 MiB; the 8x8 and 40x40 systems fit).  Every call shares that array and it keeps the last
 * call's contents: calls whose work may overlap on the device (other streams, other contexts
 * on the same GPU) race and must be serialised by the caller.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and raises the analysis kernels'
 * dynamic shared-memory limit (as letkf_analyze's first call does); make that first call before
 * any stream capture.  Plain-path contexts only (LETKF_EINVAL otherwise); requires the forecast phase
 * (LETKF_ESTATE).
 */
int letkf_analyze_static(letkf_ctx* ctx, const void* y_dev, double sigma, void* xa_dev);

/* Static English description of a status code. */
const char* letkf_status_string(int status);

/*
 * Stage timing (instrumentation; the paper has no counterpart).  Stages:
 * 0 slope check, 1 process-noise draw (normals + GEMM), 2 observed anomalies,
 * 3 Gram, 4 eigensolve and weights, 5 transform, 6 forecast, 7 fused
 * analysis+forecast, 8 differential pistons (each of its two kernels is one record).  letkf_profile(ctx, 1, NULL) starts recording a pair of
 * CUDA events around every stage launched on the context's stream (previous
 * records are dropped); letkf_profile(ctx, 0, out) stops, waits for the recorded
 * work and writes, per stage, the summed event time in milliseconds and the
 * number of launches.  Recording adds two event records per launch.
 */
#define LETKF_N_STAGES 9
typedef struct letkf_stage_times {
    double ms[LETKF_N_STAGES];
    int launches[LETKF_N_STAGES];
} letkf_stage_times;

int letkf_profile(letkf_ctx* ctx, int enable, letkf_stage_times* out);

/* Static name of a stage index (0 .. LETKF_N_STAGES-1), or "unknown". */
const char* letkf_stage_name(int stage);

/*
 * Self-test of the tensor-core product used by the fused path (diagnostic; the paper has no
 * counterpart).  D (128 x n) = A (128 x k) * op(B), FP32 row-major device buffers owned by the
 * caller: b_layout = 0 gives B as n x k and op(B) = B^T; b_layout = 1 gives B as k x n and
 * op(B) = B.  16 <= n <= 256 and 16 <= k <= 128, both multiples of 16.  The operands are
 * rounded to BF16 (terms = 1) or split into BF16 high and low parts whose three cross products
 * are accumulated (terms = 3), with FP32 accumulation in tensor memory.  Runs one CTA on
 * `stream` (cudaStream_t, NULL: default) and synchronises it.  Returns LETKF_EINVAL for other
 * arguments, LETKF_ETIMEOUT if the completion wait ran out.
 */
int letkf_umma_selftest(const float* a_dev, const float* b_dev, float* d_dev, int n, int k, int terms,
                        int b_layout, void* stream);

/*
 * Self-test of the bounded device-side wait (diagnostic; the paper has no counterpart).  Every
 * kernel of the library waits on its mbarriers for a bounded number of SM cycles, then latches
 * LETKF_ETIMEOUT and returns instead of hanging.  This runs that wait in one CTA on a barrier
 * that completes only if arrive = 1, with the given limit (1000 .. 2e9 cycles), on `stream`, and
 * synchronises: LETKF_OK when the barrier completed, LETKF_ETIMEOUT when the limit ran out (the
 * CUDA context stays usable), LETKF_EINVAL for other arguments.
 */
int letkf_wait_selftest(long long limit_cycles, int arrive, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LETKF_H */
