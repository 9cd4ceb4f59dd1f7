/*
 * pat.h - C ABI of the GB300 PDHG reconstruction library for photoacoustic tomography.
 *
 * Method: Boink, Lagerwerf, Steenbergen, van Gils, Manohar, Brune, "A Framework for
 * Directional and Higher-Order Reconstruction in Photoacoustic Tomography".  The library
 * solves  min_u 1/2 ||K u - f||^2 + alpha R(u)  (Sec. 2, eq. (min_prob)) with the
 * preconditioned first-order primal-dual algorithm PDHGM (Sec. 3.3, Algorithms 1 and 2)
 * for R = TV (eq. (min_TV)), TGV^2 (eq. (min_TGV)) or directional TV.
 *
 * Conventions shared by every entry point
 *  - Images are N x N, row-major: u[iy*N + ix]; pixel (ix, iy) has its centre at
 *    (xmin + (ix + 1/2) hx, ymin + (iy + 1/2) hy), hx = (xmax - xmin)/N.
 *  - Data are detector-major: y[d*T + k] is the integral over the circle of radius
 *    r_k = r0 + (k + 1/2) dr around detector d (speed of sound 1, so time = radius).
 *  - Vector fields are stored component-major: p[c*N*N + iy*N + ix].
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; they must not
 *    alias each other unless stated.  Pointers named *_host are host memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *    stream-ordered: it enqueues work and returns; results are valid once the stream
 *    reaches the call, except where a call says it synchronises.
 *  - Return value: PAT_OK (0) or a negative PAT_ERR_* code; pat_error_string() names it
 *    and pat_last_error() gives the message of the last failure on the calling thread.
 *    There is no CPU fallback: without a usable GPU every compute call fails with
 *    PAT_ERR_CUDA.
 */
#ifndef PAT_H
#define PAT_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define PAT_OK                0
#define PAT_ERR_INVALID_ARG  (-1)   /* a size, pointer or parameter is out of range        */
#define PAT_ERR_CUDA         (-2)   /* a CUDA runtime call or kernel launch failed          */
#define PAT_ERR_OOM          (-3)   /* device memory allocation failed                      */
#define PAT_ERR_NONFINITE    (-4)   /* an iterate or the duality gap became NaN / Inf       */
#define PAT_ERR_TIMEOUT      (-5)   /* a bounded device-side wait gave up                   */

/* ---- regularisers, step-size rules, solver status --------------------------------- */
#define PAT_TV   0   /* R(u) = ||grad u||_{1,2}                       Sec. 2.1, eq. (min_TV)  */
#define PAT_TGV  1   /* R(u) = min_v ||grad u - v|| + beta ||E v||    Sec. 2.1, eq. (min_TGV) */
#define PAT_DTV  2   /* R(u) = ||D_xi grad u||_{1,2}, D_xi = I - gamma xi xi^T (not in the
                        paper; the directional TV of Ehrhardt and Betcke)                  */
#define PAT_WAV  3   /* R(u) = ||W u||_1, Sec. 2.2 eq. (min_wav), W a tight frame
                        (W^-1 = W^T), periodic, pat_params.wavelet_levels levels:
                        pat_params.wavelet_kind selects the paper's dual-tree complex
                        transform (PAT_WAVELET_DTCWT; ||.||_1 sums complex moduli) or an
                        orthonormal Daubechies-4 transform (PAT_WAVELET_DWT)             */
#define PAT_WAVELET_DWT    0   /* orthonormal separable DWT, N*N coefficients             */
#define PAT_WAVELET_DTCWT  1   /* dual-tree complex wavelet transform (Kingsbury), 4*N*N
                                  real coefficients: see pat_dtcwt_transform            */

#define PAT_PRECOND_DIAG     0  /* Pock-Chambolle diagonal steps (alpha = 1): sigma_i =
                                   1/sum_j|A_ij|, tau_j = 1/sum_i|A_ij|   Sec. 3.3.2      */
#define PAT_PRECOND_SCALAR2  1  /* the paper's two-block scalar rule sigma_i tau L_i^2 <
                                   1/4 with tau = 1/L1, L by power iteration  Sec. 3.3.2 */

#define PAT_STATUS_CONVERGED 0  /* rel_gap <= tol at a gap evaluation                     */
#define PAT_STATUS_MAXITER   1  /* ran all iterations (tol = 0, or not reached)           */
#define PAT_STATUS_DIVERGED  2  /* the gap became NaN / Inf (then PAT_ERR_NONFINITE)      */

/* ---- geometry (Sec. 3.3.1 discretisation; Sec. 4.2 eq. (K_def)) ------------------ */
typedef struct pat_geometry pat_geometry;   /* opaque, immutable after creation */

typedef struct {
    int    n;                  /* image side N >= 2                                       */
    double xmin, xmax;         /* image extent in x (xmax > xmin)                         */
    double ymin, ymax;         /* image extent in y (ymax > ymin)                         */
    int    n_det;              /* number of point detectors D >= 1                        */
    const double* det_xy_host; /* 2*D doubles (x0, y0, x1, y1, ...), copied at creation  */
    int    n_t;                /* radius (time) samples per detector T >= 1               */
    double r0, dr;             /* r_k = r0 + (k + 1/2) dr, r0 >= 0, dr > 0                */
    int    quad_m;             /* quadrature points per circle M, 1..8192                 */
} pat_geometry_desc;

/* Discrete circular-mean operator K of eq. (K_def): quadrature point m of circle (d, k)
 * is x_d + r_k (cos phi_m, sin phi_m), phi_m = 2 pi (m + 1/2)/M, the image is
 * interpolated bilinearly between pixel centres with zero outside the grid, and each
 * point carries the arc-length weight 2 pi r_k / M.  Creation copies the description,
 * builds the device tables on the current CUDA device and synchronises.  *out receives
 * a geometry owned by the caller and released with pat_destroy_geometry. */
int  pat_create_geometry(const pat_geometry_desc* desc, pat_geometry** out);
void pat_destroy_geometry(pat_geometry* g);              /* NULL is ignored; synchronises */

/* Launch shapes of a geometry's kernels (the engineering of the hot path, not Sec. 3).
 * Every shape computes the same operators; K variants may differ in the FP32 rounding of
 * a row's sum (different partial-sum orders), K^T waves and update tiles give the same
 * bits.  pat_tune_shapes picks them by timing; pat_create_geometry starts with
 * {PAT_FWD_AUTO resolved, 1, PAT_UPD_32X4}. */
#define PAT_FWD_AUTO      -1  /* slab kernel for images up to 320 pixels, else global       */
#define PAT_FWD_SLAB_TWO   0  /* K: image slabs in shared memory, two CTAs per SM           */
#define PAT_FWD_SLAB_ONE   1  /* K: image slabs in shared memory, one CTA per SM            */
#define PAT_FWD_GLOBAL     2  /* K: taps read from global memory                            */
#define PAT_UPD_32X4       0  /* fused update tile of 32 x 4 pixels                         */
#define PAT_UPD_32X8       1  /* 32 x 8                                                     */
#define PAT_UPD_64X4       2  /* 64 x 4                                                     */
typedef struct {
    int forward;        /* PAT_FWD_*; get returns the variant in use (AUTO resolved; a slab
                           variant that does not fit the device falls back to GLOBAL)      */
    int adjoint_waves;  /* K^T work items fill this many waves of resident CTAs, 1..4     */
    int update_tile;    /* PAT_UPD_*                                                        */
} pat_shapes;
/* Rebuilds the geometry's K plan and K^T work list for the shapes.  The call waits for the
 * device to be idle; no other call may use the geometry meanwhile. */
int  pat_geometry_set_shapes(pat_geometry* g, const pat_shapes* s);
int  pat_geometry_get_shapes(const pat_geometry* g, pat_shapes* s);


/* y = K u.  u_dev: N*N floats, y_dev: D*T floats (overwritten). */
int  pat_forward(const pat_geometry* g, const float* u_dev, float* y_dev, void* stream);

/* u = K^T y, the exact transpose of pat_forward's weights (Sec. 3.3.1: the adjoint is
 * the transposed matrix, not a discretised continuous adjoint).  y_dev: D*T floats,
 * u_dev: N*N floats (overwritten). */
int  pat_adjoint(const pat_geometry* g, const float* y_dev, float* u_dev, void* stream);

/* Direction field for directional TV: xi = grad w / sqrt(|grad w|^2 + eta^2) with the
 * forward differences of the TV gradient.  w_dev: N*N, xi_dev: 2*N*N (overwritten). */
int  pat_direction_field(int n, const float* w_dev, double eta, float* xi_dev, void* stream);

/* ---- reconstruction (Sec. 3, Algorithms 1 and 2) ---------------------------------- */
typedef struct {
    int    reg;          /* PAT_TV, PAT_TGV or PAT_DTV                                    */
    double alpha;        /* regularisation weight alpha >= 0                              */
    double beta;         /* TGV second-order weight beta >= 0 (F3 = alpha beta ||.||)     */
    double gamma;        /* dTV: 0 <= gamma <= 1                                          */
    const float* xi_dev; /* dTV: direction field, 2*N*N floats, |xi| <= 1 pointwise       */
    int    iters;        /* maximum number of PDHG iterations >= 0                        */
    double tol;          /* stop at the first gap evaluation with rel_gap <= tol (0: never) */
    int    gap_every;    /* evaluate the gap every gap_every iterations (0: only at the end) */
    int    precond;      /* PAT_PRECOND_DIAG or PAT_PRECOND_SCALAR2                       */
    double theta;        /* extrapolation theta in [0, 1] (PDHGM: 1)                      */
    double box_u, box_v; /* half-widths of the box on which the duality gap is taken     */
    /* optional warm start (NULL = zero); layouts: x = [u (N*N), v (2*N*N, TGV only)],
       y = [q (D*T), r (2*N*N), s (3*N*N, TGV only)]; xbar defaults to x0 */
    const float* x0_dev;
    const float* xbar0_dev;
    const float* y0_dev;
    /* optional export of the final state in the same layouts (NULL = not written) */
    float* x_out_dev;
    float* xbar_out_dev;
    float* y_out_dev;
    /* primal-dual balance s > 0 of the diagonal steps: every primal step tau_j becomes
       s tau_j and every dual step sigma_i becomes sigma_i / s.  This leaves
       ||Sigma^1/2 A T^1/2|| and so the convergence condition of Sec. 3.3.2 unchanged.
       Default 1. */
    double step_ratio;
    /* PAT_ADAPT_NONE keeps s fixed.  PAT_ADAPT_BALANCE re-balances s at every gap
       evaluation that does not stop the run (residual balancing after Goldstein, Li, Yuan,
       Esser and Baraniuk 2015).  The gap splits into
         stationarity = U ||A_u^T y||_1 + V ||A_v^T y||_1 + <x, A^T y>, reduced by larger
         primal steps, and
         the Fenchel-Young part = gap - stationarity, reduced by larger dual steps.
       When the two differ by more than a factor 2, s is multiplied by the square root of
       their ratio (clamped to [1/2, 2], raised to 0.97^k after k adjustments; s stays in
       [1e-3, 1e3]). */
    int    adapt;
    /* PAT_WAV: levels J of the transform, 1..12, with N divisible by 2^J (0: 4) */
    int    wavelet_levels;
    /* The primal iterates x = (u, v) are kept as compensated pairs hi + lo (every update
       is added with an error-free two-sum), and x_out_dev receives the high words.  The
       low word is stored as a bfloat16 (8 significant bits, so the pair holds about 32).
       x_lo_out_dev (layout of x, NULL = not written) receives the low words, and
       x_lo0_dev (layout of x, NULL = zero) starts a run from them, rounded to bfloat16
       (exported words are bfloat16 values already).  Passing x_out,
       xbar_out, y_out and x_lo_out of one run as x0, xbar0, y0 and x_lo0 of the next
       continues it bit for bit (the gap schedule restarts at the resumed iteration).
       PAT_WAV iterates are plain FP32: its low words are zero.  Not Sec. 3: a numerical
       device of this library. */
    const float* x_lo0_dev;
    float* x_lo_out_dev;
    /* PAT_WAV: PAT_WAVELET_DWT (default) or PAT_WAVELET_DTCWT.  With the DT-CWT, r in y
       has 4*N*N entries (the layout of pat_dtcwt_transform's output), and the filters are
       those of pat_dtcwt_transform (NULL: the closed-form defaults). */
    int    wavelet_kind;
    const double* dtcwt_h1_host;   /* level-1 low-pass, dtcwt_l1 taps (host memory)      */
    int    dtcwt_l1;
    const double* dtcwt_hq_host;   /* Q-shift low-pass of tree a, dtcwt_lq taps          */
    int    dtcwt_lq;
} pat_params;

#define PAT_ADAPT_NONE     0
#define PAT_ADAPT_BALANCE  1

typedef struct {
    int    iters_done;   /* iterations run                                                */
    int    status;       /* PAT_STATUS_*                                                  */
    double primal;       /* P(x) = 1/2||Ku - f||^2 + alpha R(u) at the last gap evaluation */
    double dual;         /* box-restricted dual value D_B(y) at the same evaluation       */
    double gap;          /* primal - dual (FP64)                                          */
    double rel_gap;      /* gap / primal                                                  */
    double residual;     /* ||x^{n+1} - x^n|| / ||x^n|| over the primal variables         */
    double ms;           /* device time of the call in milliseconds (CUDA events)         */
    double step_ratio;   /* the primal-dual balance s at the end (adapt may have moved it) */
} pat_info;

/* Fills *p with defaults: TV, alpha 0.05, beta 1, gamma 0.95, 100 iterations, tol 0,
 * gap every 10 iterations, diagonal preconditioning, theta 1, box 2 / 4, no warm start. */
void pat_params_default(pat_params* p);

/* Runs PDHGM: iteration n computes (Alg. 2 order)
 *   q   <- prox_{Sigma_q F1*}(q + Sigma_q K ubar)          F1* prox: (z - s f)/(1 + s)
 *   r   <- proj_{|.|<=alpha}(r + Sigma_r (grad ubar - vbar))       (dTV: D_xi grad ubar)
 *   s   <- proj_{|.|<=alpha beta}(s + Sigma_s E vbar)                         (TGV)
 *   u+  <- u - T_u (K^T q - div r)                 (dTV: div(D_xi r))
 *   v+  <- v - T_v (E^T s - r)                                                (TGV)
 *   ubar <- u+ + theta (u+ - u),  vbar <- v+ + theta (v+ - v)
 * with the box-restricted duality gap and residual of Sec. 3.3.3 evaluated in FP64 on
 * the device.  f_dev: D*T floats; u_dev: N*N floats, receives the final u.  *info
 * (host) is filled after the call synchronises `stream`.  Workspace is allocated from
 * the stream-ordered pool and released before returning.  Returns PAT_ERR_NONFINITE
 * (status DIVERGED) when the gap stops being finite. */
int  pat_reconstruct(const pat_geometry* g, const float* f_dev, const pat_params* p,
                     float* u_dev, pat_info* info, void* stream);

/* Runs `count` independent reconstructions (each with its own geometry, data, params
 * and output) on one stream, interleaving their iterations so that problems of very
 * different sizes share the GPU.  Arrays have `count` entries; infos is host memory. */
int  pat_reconstruct_batched(int count, const pat_geometry* const* g, const float* const* f_dev,
                             const pat_params* p, float* const* u_dev, pat_info* infos,
                             void* stream);

/* Step sizes that pat_reconstruct uses for (g, p) (Sec. 3.3.2), computed with FP64
 * sums: sig_q (D*T), tau_u (N*N), sig_r (N*N, one value per pointwise r group; PAT_WAV
 * with the DT-CWT: 4*N*N, one value per coefficient, shared by the two of a complex pair),
 * sig_s (N*N, TGV; may be NULL otherwise), tau_v (2*N*N, TGV; may be NULL otherwise).
 * Output pointers are device memory and may be NULL to skip. */
int  pat_steps(const pat_geometry* g, const pat_params* p, float* sig_q_dev, float* tau_u_dev,
               float* sig_r_dev, float* sig_s_dev, float* tau_v_dev, void* stream);

/* Probe-based choice of the primal-dual balance s (pat_params.step_ratio).
 * Each of the n_candidates values (1..64, each > 0) runs probe_iters PDHG iterations of
 * (g, f, p) from p's start.  All probes run as one lockstep batch, and the one with the
 * smallest relative gap after the probe wins.  best_host receives its s, and rel_gaps_host
 * (may be NULL) each probe's relative gap.  p's iters, tol, gap_every, adapt and outputs
 * are ignored; nothing is written to the caller's buffers.  The call synchronises
 * `stream`.  Scratch comes from the stream-ordered pool. */
int  pat_tune_step_ratio(const pat_geometry* g, const float* f_dev, const pat_params* p,
                         const double* candidates_host, int n_candidates, int probe_iters,
                         double* best_host, double* rel_gaps_host, void* stream);

/* The same for `count` problems at once: every (problem, candidate) probe runs in one
 * lockstep batch.  best_host receives count values, and rel_gaps_host (may be NULL)
 * count * n_candidates values, problem-major. */
int  pat_tune_step_ratio_batched(int count, const pat_geometry* const* g, const float* const* f_dev,
                                 const pat_params* p, const double* candidates_host, int n_candidates,
                                 int probe_iters, double* best_host, double* rel_gaps_host, void* stream);

/* Launch-shape autotuner for `count` problems (arrays as in pat_reconstruct_batched; the
 * geometries' shapes are changed, so no other call may use them meanwhile).  For each
 * geometry whose key (N, D, T, M, regulariser, GPU name) the JSON file cache_path (NULL:
 * no cache) does not hold yet, the K variants, then the K^T waves (1, 2), then the update
 * tiles are timed on that problem (20 iterations, then each candidate's phase in a CUDA
 * graph of `reps` launches, as pat_time_phases) and the fastest of each is kept; cached
 * keys are applied without timing, and new ones are added to the file.  chosen_host (may
 * be NULL) receives each geometry's shapes.  Synchronises `stream`. */
int  pat_tune_shapes(int count, pat_geometry* const* g, const float* const* f_dev, const pat_params* p, int reps,
                     const char* cache_path, pat_shapes* chosen_host, void* stream);

/* Box-restricted duality gap (Sec. 3.3.3, FP64 accumulation) of a primal point x and a
 * dual-feasible point y in the layouts of pat_params.  out4_host receives
 * {primal, dual, gap, rel_gap}; the call synchronises `stream`. */
int  pat_duality_gap(const pat_geometry* g, const float* f_dev, const pat_params* p,
                     const float* x_dev, const float* y_dev, double* out4_host, void* stream);

/* ---- the wavelet transform of PAT_WAV ------------------------------------------------ */
/* out = W in (inverse = 0) or W^T in = W^-1 in (inverse != 0) for N x N images, with the
 * transform of PAT_WAV (`levels` levels).  in and out are distinct device buffers. */
int  pat_wavelet_transform(int n, int levels, const float* in_dev, float* out_dev, int inverse, void* stream);

/* The dual-tree complex wavelet transform (Sec. 2.2; Kingsbury's dual tree) of N x N
 * images with `levels` levels (N divisible by 2^levels), periodic extension.
 *  - Two orthonormal filter banks, trees a and b.  Level 1: low-pass h1_host (l1 taps) in
 *    both trees, tree b's input index offset by one sample.  Levels >= 2: the Q-shift
 *    low-pass hq_host (lq taps) in tree a and its time reverse in tree b.  High-pass
 *    g[n] = (-1)^n h[L - 1 - n].  One step: a[k] = sum_n h[n] x[(2k + n + o) mod M].
 *    NULL selects the closed-form defaults: Daubechies' 4-tap filter at level 1 and the
 *    orthonormal 4-tap (5 - s15, 5 + s15, 3 + s15, 3 - s15) / (8 sqrt 2) (s15 = sqrt 15),
 *    centre a quarter sample before its midpoint, at levels >= 2.  Filters must be
 *    orthonormal (to 1e-6) with an even length 2..16.
 *  - Four separable transforms T_t, t = 2 p + q (tree p along x, q along y), each in the
 *    Mallat layout.  out (inverse = 0, 4*N*N floats, four planes): (1/2) T u with every
 *    detail position changed to z1 = ((aa - bb) + i (ab + ba)) / sqrt 2 and
 *    z2 = ((aa + bb) + i (ba - ab)) / sqrt 2 stored as (Re z1, Im z1, Re z2, Im z2); at
 *    the LL positions of the last level plane c holds (1/2) T_c.  W^T W = I.
 *  - inverse != 0: out (N*N) = W^T in (in: 4*N*N floats).
 * in and out are distinct device buffers; filters are host arrays. */
int  pat_dtcwt_transform(int n, int levels, const double* h1_host, int l1, const double* hq_host, int lq,
                         const float* in_dev, float* out_dev, int inverse, void* stream);

/* ---- measurement pre-processing (Sec. 4.3) ------------------------------------------ */
/* Data f (D*T, detector-major) for the reconstruction from measured pressures p and the
 * calibration measurements p_cal of an approximate delta pulse at x_p (both D*T, the
 * samples of pat_geometry_desc: t_k = r0 + (k + 1/2) dr, speed of sound 1).  Per detector:
 *   f_t = F^-1{ F{p} conj(F{h}) / (|F{h}|^2 + eps) }          (eq. (deconv))
 * with h the calibration moved to the retarded time t - |x_d - x_p| (eq. (FW_full)),
 * then f = t / |x_d - x_p| f_t                                   (eq. (f_rewrite)).
 * Readings where the paper is silent:
 *  - The transform length is the smallest power of two >= 2T, with zero padding (a linear
 *    convolution), and the first T samples are kept.
 *  - The time convolution is dr * sum.
 *  - The travel-time shift uses the shift theorem (FFT phase ramp).
 *  - eps = eps_rel * max |F{dr h}|^2 per detector.
 * Arithmetic: FP32 transforms, FP64 times and delays.
 * Constraints: T <= 2048, eps_rel > 0, x_p (2 doubles, host) not on a detector. */
int  pat_preprocess(const pat_geometry* g, const float* p_dev, const float* pcal_dev,
                    const double* xp_host, double eps_rel, float* f_dev, void* stream);

/* ---- K^T without device allocation -------------------------------------------------- */
/* u = K^T y like pat_adjoint, but the call allocates no device memory: no cudaMalloc,
 * cudaFree, stream-ordered pool or other allocating routine.  This is for callers that
 * must not allocate at the time of the call.  Examples: real-time loops that must not
 * touch an allocator, and host applications whose device memory is owned by another
 * allocator or fixed at start-up.  The paper has no counterpart; this is a deployment
 * variant of the adjoint.
 *  - Scratch: a device array of 4 MiB + 256 bytes built into the library.  Every GPU that
 *    loads the library holds it until the process exits.  Its contents persist from call
 *    to call, and the call clears what it needs.
 *  - Limits: image side N <= 1024 (larger sizes return PAT_ERR_INVALID_ARG).
 *  - Preparation: the geometry must have been prepared once, while allocation is allowed,
 *    by pat_steps, pat_adjoint or pat_reconstruct (they compute the FP64 K sums that scale
 *    the fixed-point accumulation).  Otherwise PAT_ERR_INVALID_ARG.
 *  - Set-up: the first call on a device looks up the scratch's device address for that
 *    device (current at the call) and keeps it for the life of the process.  Make that
 *    first call before any stream capture.  The kept address does not survive
 *    cudaDeviceReset: do not call this entry point after resetting the device.
 *  - Concurrency: all calls on one device share the scratch.  Calls that overlap on the
 *    GPU (other streams, or other host threads without ordering) race; order them on
 *    one stream.
 *  - Result: identical to pat_adjoint's (same kernels, same fixed-point arithmetic).
 *  y_dev: D*T floats; u_dev: N*N floats (overwritten); both caller-owned device memory. */
int  pat_adjoint_noalloc(const pat_geometry* g, const float* y_dev, float* u_dev, void* stream);

/* ---- diagnostics ------------------------------------------------------------------ */
/* Phases of one PDHG iteration timed by the optional profiler (CUDA events recorded
 * around each launch on the caller's stream; the events add a few microseconds of host
 * work per launch and nothing between kernels on the device). */
#define PAT_PHASE_FORWARD_PROX 0   /* K ubar and the q prox                          */
#define PAT_PHASE_ADJ_CLEAR    1   /* zeroing the K^T q accumulator                  */
#define PAT_PHASE_ADJOINT      2   /* K^T q                                          */
#define PAT_PHASE_UPDATE       3   /* fused primal step, extrapolation, dual step    */
#define PAT_PHASE_GAP          4   /* FP64 duality gap and residual                  */
#define PAT_NPHASES            5
/* Turns per-phase timing of pat_reconstruct on (1) or off (0) for the whole process. */
int  pat_profile_enable(int on);
/* ms_host[PAT_NPHASES]: summed device milliseconds per phase; launches_host[PAT_NPHASES]:
 * number of timed launches per phase (either may be NULL).  reset != 0 clears the sums. */
int  pat_profile_read(double* ms_host, long long* launches_host, int reset);
/* Device time of each phase of the batched iteration, measured without per-launch
 * bracketing: the `count` problems (arrays as in pat_reconstruct_batched) first run
 * p[0].iters iterations as pat_reconstruct_batched would (tol and adapt ignored), then
 * each phase's launch (one launch over all problems; the update counts its per-regulariser
 * launches together, the gap its three kernels) is captured `reps` times (1..100000) in a
 * CUDA graph and replayed once to warm up and once between two CUDA events on the
 * library's loop stream.  us_host[PAT_NPHASES] receives microseconds per launch
 * (PAT_PHASE_ADJ_CLEAR: 0).  Nothing is written to the caller's buffers; the call
 * synchronises `stream`.  Fails if the per-launch profiler is on.  Not Sec. 3: a
 * measurement aid. */
int  pat_time_phases(int count, const pat_geometry* const* g, const float* const* f_dev,
                     const pat_params* p, int reps, double* us_host, void* stream);
/* Number of kernels this library has launched in the process so far. */
long long pat_kernel_launches(void);

const char* pat_error_string(int code);
const char* pat_last_error(void);
/* Geometry sizes: out6 = {N, D, T, M, number of quadrature points evaluated per K
 * application (inside the angular windows), number of quadrature points whose
 * bilinear taps touch the grid (the algorithmic work of one K or K^T)}. */
int  pat_geometry_info(const pat_geometry* g, long long* out6_host);

/* Host only: the work list of the K^T kernel (Sec. 3.3.1's adjoint, evaluated by pixel
 * tiles) that pat_create_geometry builds for `desc`, for a GPU that holds `slots` K^T
 * CTAs at once.  With slots > 0 no CUDA call is made; slots <= 0 sizes it for the
 * current device.  counts3_host = {ray segments, work items, candidate points}.
 * rays_host (4 ints per segment: detector, angle index m, first radius index k,
 * exclusive prefix within its tile; after each tile a sentinel {-1, 0, 0, tile total})
 * and items_host (5 ints per item: tile, first segment, segment count, first and end
 * candidate within the tile) are written when not NULL.  Their capacities are in
 * entries; if one is too small, PAT_ERR_INVALID_ARG is returned after counts3_host is
 * written, so a first call with NULL outputs gives the sizes.  The caller owns all
 * buffers. */
int  pat_adjoint_worklist(const pat_geometry_desc* desc, int slots, int* rays_host, long long rays_cap,
                          int* items_host, long long items_cap, long long* counts3_host);

/* Host only: the work plan of the forward projector K (Sec. 3.3.1, eq. (K_def)) that
 * pat_create_geometry builds for `desc`.  Row group rg = d * ceil(T/8) + k/8 holds 8
 * consecutive radii of one detector.  The image is cut into S horizontal slabs of R rows
 * of upper tap rows (slab s holds the quadrature points whose upper-left tap row j0 lies
 * in [s R - 1, (s + 1) R - 1); R = 0 means one slab read from global memory).  K runs as
 * clusters of S CTAs: rank s stages slab s in shared memory, and a cluster owns a list of
 * row groups, processed in rounds of 256.  A work unit is one row group restricted to one
 * slab: at most two circular angular windows.  `sms` is the SM count to plan for (<= 0:
 * the current device, with its cluster occupancy; with sms > 0 no CUDA call is made).
 * budget_bytes > 0 caps a slab's staged image (for tests); 0 uses the library's budget.
 * info8_host = {S, R, shared-memory row stride in floats, units, CTAs, points inside the
 * units' windows, dynamic shared memory of a CTA in bytes, round offsets}.  When not NULL:
 *   units_host: 4 ints per unit {detector, window 0, window 1, (k / 8) << 16 | the row
 *     group's index in its round}; a window is m_first | count << 16, a circular range of
 *     angles;
 *   ctas_host: 4 ints per CTA, cluster-major and rank-minor {first entry in rgs, row
 *     groups of the cluster, first entry in roff, 0};
 *   roff_host: per CTA, unit offsets of its rounds (rounds + 1 entries);
 *   rgs_host: every cluster's row groups in processing order.
 * Capacities are in entries; too small a capacity returns PAT_ERR_INVALID_ARG after
 * info8_host is written.  The caller owns all buffers. */
int  pat_forward_plan(const pat_geometry_desc* desc, int budget_bytes, int sms, int* units_host,
                      long long units_cap, int* ctas_host, long long ctas_cap, int* roff_host,
                      long long roff_cap, int* rgs_host, long long rgs_cap, long long* info8_host);

#ifdef __cplusplus
}
#endif
#endif /* PAT_H */
