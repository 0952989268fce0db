/*
 * ba.h -- C ABI of the GB300 (sm_103a) Levenberg-Marquardt bundle-adjustment
 * library.
 *
 * The library solves the non-linear least-squares problem of Eq. 1 (Sec.
 * III-A): minimise, over cameras theta_c and points X_j, the sum over the
 * OBSERVED (camera, point) pairs k of rho(|pi(theta_c(k), X_p(k)) - x_k|^2),
 * with the LM iteration of Alg. 1 / Eq. 2 (Sec. III-B).
 *
 * Camera model (the BAL camera of the paper's benchmark data, Sec. V): a
 * camera is 9 numbers (omega[3] angle-axis, t[3], f, k1, k2).  A point X
 * maps to X_cam = R(omega) X + t, p = -X_cam[0:2] / X_cam[2],
 * pi = f (1 + k1 |p|^2 + k2 |p|^4) p.  All parameters update additively.
 *
 * Conventions shared by every entry point:
 *  - Floating-point arrays have the type selected by ba_options.precision:
 *    double for BA_PREC_F64, float for BA_PREC_F32.  Reductions (normal-
 *    equation sums, dot products, costs, the gain ratio) are FP64 in both.
 *  - cams is [C][9], points [P][3], pixels [O][2], row-major, contiguous.
 *    cam_idx / pt_idx are int32 [O].
 *  - Pointers marked "any" may be host (pageable or pinned) or device
 *    memory; they are copied with a stream-ordered copy.  Pointers marked
 *    "dev" must be device memory of the current device.  The caller owns
 *    every pointer it passes; the library never keeps one.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All work is ordered on it; only calls documented as synchronising
 *    block the host.
 *  - Every call returns a ba_status; on failure ba_last_error() returns a
 *    message for the calling thread.  No call aborts, traps or spins
 *    without a bound.
 */
#ifndef BA_GB300_H
#define BA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_problem ba_problem; /* opaque, owned by the library */

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1, /* bad size, pointer, index or option */
  BA_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  BA_ERR_NONFINITE = 3,   /* a non-finite parameter, pixel or cost */
  BA_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
  BA_ERR_NOT_CONVERGED = 5,
  BA_ERR_OOM = 6,         /* device allocation failed */
  BA_ERR_STATE = 7        /* call not valid in the problem's current state */
} ba_status;

enum { BA_PREC_F64 = 0, BA_PREC_F32 = 1 };

/* How the passes after the linearisation get the Jacobian blocks:
 * BA_JAC_STORE writes them once per linearisation (18 numbers per
 * observation, twice) and streams them; BA_JAC_RECOMPUTE rebuilds them in
 * every pass from the parameters (no per-observation storage but sqrt(w)
 * under a robust loss); BA_JAC_AUTO picks RECOMPUTE for BA_PREC_F32 and
 * STORE for BA_PREC_F64.  Both give the same blocks up to rounding. */
enum { BA_JAC_AUTO = 0, BA_JAC_RECOMPUTE = 1, BA_JAC_STORE = 2 };

/* How each LM trial solves the reduced camera system S dc = b (Sec. IV-C:
 * the paper offers PCG and a sparse direct solver, a Cholesky
 * factorisation).  BA_SOLVER_PCG: block-Jacobi PCG with the implicit S x
 * product (pcg_maxiter, pcg_tol).  BA_SOLVER_CHOLESKY: S formed explicitly
 * as a dense 9C x 9C FP64 matrix and factored by a tiled Cholesky on the
 * GPU (the factorisation and both triangular solves in one cooperative
 * launch), for problems with 9C <= BA_DENSE_MAX_DIM (the matrix and its
 * tiles take 81 C^2 x 8 bytes each, plus up to 8 partial copies of S while
 * it is built for small C); a trial whose S is not positive definite in
 * FP64 takes a zero step (rejected, counted in
 * ba_iter_stats.precond_fallbacks). */
enum { BA_SOLVER_PCG = 0, BA_SOLVER_CHOLESKY = 1 };
#define BA_DENSE_MAX_DIM 18432

/* Solver options.  up/down are the trust-region factors of the paper's
 * minimum code example (TrustRegion(up=2.0, down=0.5**4), Sec. IV); its
 * PCG(tol=1e-4, maxiter=250) gives pcg_tol / pcg_maxiter.  diag_min/diag_max
 * are the bounds of diagonal clamping (Sec. IV-B).  The remaining constants
 * are this library's readings of a paper that gives none. */
typedef struct {
  int precision;       /* BA_PREC_F64 or BA_PREC_F32 */
  double huber_delta;  /* > 0: Huber loss on |r| with this delta (pixels) */
  double lambda0;      /* initial damping, 1e-4 */
  double up;           /* lambda /= up after a very good step, 2 */
  double down;         /* lambda /= down after a bad or rejected step, 1/16 */
  double rho_good;     /* gain ratio above which lambda shrinks, 0.75 */
  double rho_bad;      /* gain ratio below which lambda grows, 0.25 */
  double lambda_min;   /* 1e-16 */
  double lambda_max;   /* 1e32 */
  double diag_min;     /* clamp of diag(J^T J) before lambda scaling, 1e-6 */
  double diag_max;     /* 1e32 */
  int pcg_maxiter;     /* PCG iterations per LM trial, 250 */
  double pcg_tol;      /* stop when |r|_2 <= pcg_tol |b|_2, 1e-4 */
  int use_graph;       /* 1: ba_solve replays a captured CUDA graph (not with
                          BA_SOLVER_CHOLESKY: its trials are direct launches) */
  int max_stats;       /* capacity of the per-trial statistics ring, 4096 */
  int jacobian_mode;   /* BA_JAC_AUTO, BA_JAC_RECOMPUTE or BA_JAC_STORE */
  int solver;          /* BA_SOLVER_PCG or BA_SOLVER_CHOLESKY */
} ba_options;

/* Statistics of one LM trial (Alg. 1, one pass of the loop body). */
typedef struct {
  double cost;        /* F(theta) before the trial, F = 1/2 sum rho(|r|^2) */
  double cost_trial;  /* F(theta + Delta) */
  double model;       /* Delta L = -g^T Delta - 1/2 sum_k w_k |J_k Delta|^2 */
  double rho;         /* (cost - cost_trial) / model */
  double lambda;      /* damping used by this trial */
  double pcg_rel_res; /* |r|/|b| of the reduced system at exit */
  int32_t accepted;   /* 1 if theta <- theta + Delta */
  int32_t pcg_iters;  /* PCG iterations run */
  int32_t precond_fallbacks; /* cameras whose block-Jacobi block was not SPD;
                                with BA_SOLVER_CHOLESKY: 1 if S was not */
  int32_t reserved;
} ba_iter_stats;

/* Fill *opt with the defaults listed above (the trust-region factors and
 * PCG settings of the paper's minimum code example, Sec. IV; the rest are
 * this library's readings). */
ba_status ba_options_default(ba_options* opt);

/* Create a problem (C cameras, P points, O observations), run the cached
 * symbolic phase (Sec. IV-B: stable device radix sorts of the observations
 * by camera and by point) and evaluate the initial cost.
 * cams (any, [C][9]), points (any, [P][3]), cam_idx / pt_idx (any, int32
 * [O]), pixels (any, [O][2]) are copied.  Errors: BA_ERR_INVALID_ARG for
 * C, P or O < 1, a NULL pointer, an index out of range or bad options;
 * BA_ERR_NONFINITE for a non-finite parameter, pixel or initial cost;
 * BA_ERR_OOM.  Synchronises the stream.  On error *out is NULL. */
ba_status ba_problem_create(ba_problem** out, int C, int P, int O,
                            const void* cams, const void* points,
                            const int32_t* cam_idx, const int32_t* pt_idx,
                            const void* pixels, const ba_options* opt,
                            void* stream);

/* Free a problem and everything it owns (NULL is accepted).  Resource
 * management: no counterpart in the paper. */
ba_status ba_problem_destroy(ba_problem* h);

/* One LM trial (Alg. 1 loop body): linearise if theta changed (a1, a2),
 * damp and reduce (a3), solve the reduced camera system by block-Jacobi PCG
 * with implicit S x (a4), back-substitute (a5), evaluate the trial and
 * accept or reject it, update lambda (a6).  With use_graph, one replay of
 * the trial graph that ba_solve captures.  No host synchronisation. */
ba_status ba_lm_step(ba_problem* h, void* stream);

/* iters LM trials; with use_graph the trial is captured once as a CUDA graph
 * (App. B) and replayed.  No host synchronisation. */
ba_status ba_solve(ba_problem* h, int iters, void* stream);

/* Copy the current (last accepted) parameters theta of Eq. 1 (Sec. III-A)
 * to cams_out [C][9] and points_out [P][3] (any). Either may be NULL.  Stream-ordered (no host
 * synchronisation): into pinned or device memory the copy completes on the
 * stream; the caller synchronises before reading. */
ba_status ba_get_params(ba_problem* h, void* cams_out, void* points_out,
                        void* stream);

/* Replace the parameters theta of Eq. 1 (any; either may be NULL to keep
 * it); the cost is
 * re-evaluated by the next trial or by the next call that reads it
 * (ba_get_scalars, ba_get_state), and the next trial re-linearises.  lambda
 * is kept.  Stream-ordered: a pinned or device source must stay valid until
 * the stream reaches the copy. */
ba_status ba_set_params(ba_problem* h, const void* cams, const void* points,
                        void* stream);

/* Replace the observed pixels x_k of Eq. 1 (any, [O][2]); the observation
 * structure is
 * kept; the cost is re-evaluated as after ba_set_params and the next trial
 * re-linearises. */
ba_status ba_set_pixels(ba_problem* h, const void* pixels, void* stream);

/* Copy up to cap statistics records, one per pass of Alg. 1's loop (Sec.
 * III-B; the gain ratio is the ratio of actual to predicted reduction of
 * Sec. IV), oldest first among the last cap trials, to host_out; *n_out = number copied.  Synchronises the stream of
 * the problem.  Returns BA_ERR_NONFINITE if a trial since the last call saw
 * a non-finite trial cost (such trials are rejected, theta is unchanged). */
ba_status ba_get_stats(ba_problem* h, ba_iter_stats* host_out, int cap,
                       int* n_out);

/* Current cost F(theta) (Eq. 1) and damping lambda (Eq. 2), copied to the
 * host.  Synchronises. */
ba_status ba_get_scalars(ba_problem* h, double* cost, double* lambda);

/* Set the damping lambda of Eq. 2 for the next trial (lambda > 0, e.g. to
 * restart a solve after new observations).  Synchronises. */
ba_status ba_set_lambda(ba_problem* h, double lambda);

/* Checkpoint (no counterpart in the paper): the number of doubles
 * ba_get_state writes (9C + 3P + 4). */
size_t ba_state_size(const ba_problem* h);
/* Checkpoint (no counterpart in the paper): write theta, cost, lambda and
 * the trial counter to host_state (host,
 * ba_state_size doubles; parameters converted to double).  Synchronises. */
ba_status ba_get_state(ba_problem* h, double* host_state);
/* Resume (no counterpart in the paper): restore a state written by
 * ba_get_state on a problem with the same C, P, O and precision.
 * Synchronises. */
ba_status ba_set_state(ba_problem* h, const double* host_state);

/* Freeze camera parameters: mask (any, uint8 [C][9], nonzero = frozen) or
 * NULL to free them all.  Frozen parameters never move; each LM step solves
 * the system restricted to the free ones (S -> m S m + (I - m), b -> m b).
 * Freezing all nine parameters of one camera and one translation component
 * of another removes the 7-dimensional similarity gauge of BA, which the
 * adjoint needs for a well-defined derivative.  Not in the paper. */
ba_status ba_set_fixed(ba_problem* h, const uint8_t* mask, void* stream);

/* Implicit-function adjoint at the current parameters theta* (meant to be a
 * converged solution, where the gradient vanishes).  With the Gauss-Newton
 * H* = J^T W J + lambda clamp(diag), restricted to the free parameters,
 * v = H*^{-1} dL/dtheta is solved by the same Schur / block-Jacobi PCG as the
 * forward step (maxiter, tol), then
 *   dL/dx_k      = w_k J_k v                      (r_k = pi_k - x_k)
 *   dL/dtheta0   = dL/dtheta - (H* v) on frozen camera parameters, 0 on free
 *                  ones and on points (theta* does not depend on where the
 *                  free parameters start).
 * Not in the paper (its bilevel use of BA, Sec. VI, motivates it).  Inputs
 * dL_dcams [C][9], dL_dpoints [P][3] (dev, precision type, either may be
 * NULL = zero); outputs dL_dpixels_out [O][2] (required),
 * dL_dcams0_out [C][9], dL_dpoints0_out [P][3] (dev, may be NULL); iters /
 * rel_res (host, may be NULL: then no synchronisation).  The next LM trial
 * re-linearises.  For a BA_PREC_F32 problem the adjoint system is solved in
 * FP64 (its rounding amplification, condition x cancellation of the
 * implicit Schur product, is ~1e6): the first call builds an FP64 copy of
 * the problem (same observations, the FP32 parameters and pixels promoted;
 * it allocates and synchronises), later calls refresh its parameters,
 * pixels and frozen mask; inputs and outputs stay FP32. */
ba_status ba_backward(ba_problem* h, double lambda, int maxiter, double tol,
                      const void* dL_dcams, const void* dL_dpoints,
                      void* dL_dpixels_out, void* dL_dcams0_out,
                      void* dL_dpoints0_out, int* iters, double* rel_res,
                      void* stream);

/* Thread-local message of the last failing call ("" if none).  Error
 * reporting: no counterpart in the paper. */
const char* ba_last_error(void);

/* ---- point-partitioned problems (several GPUs) -------------------------
 *
 * One problem split by points: each part holds a subset of the points with
 * ALL of their observations and every camera (cameras replicated, the same
 * values in every part).  The LM iteration of Alg. 1 then needs sums over
 * all parts at six places of a trial: U and gc of the linearisation, the
 * Schur pass's per-camera sums (b and the block-Jacobi blocks), the pass-B
 * sum of every PCG iteration (9C values), and the cost, model and gp . dp
 * scalars of the trial and of a stale cost; everything else (the PCG
 * vectors and dot products, the decision, lambda) is computed identically
 * in every part from those sums.  Not in the paper (it runs on one GPU).
 *
 * fn(n, stream, ctx) must replace the first n doubles of xbuf (the caller's
 * device buffer, which the library fills first) by their sum over all parts,
 * ordered on stream (a cudaStream_t as void*: enqueue, e.g. an NCCL
 * all-reduce, or synchronise), and return 0 (nonzero: the trial fails with
 * BA_ERR_CUDA).  Every part must call the same entry points in the same
 * order.  xbuf must hold cap >= BA_EXCHANGE_CAP(C) doubles. */
typedef int (*ba_exchange_fn)(size_t n, void* stream, void* ctx);
#define BA_EXCHANGE_CAP(C) (64 * (size_t)(C) + 8)

/* Make h one part of a point-partitioned problem (fn, ctx, xbuf, cap as
 * above; fn NULL returns to a problem of its own).  The LM iteration is the
 * one of Alg. 1 (Sec. III-B); the partitioning has no counterpart in the
 * paper.  From then on ba_lm_step
 * and ba_solve run with direct launches (no graph) and call fn at each
 * exchange; the cost is re-evaluated (summed) at the next trial.  The
 * step-level entry points, the learned preconditioner, the direct solver and
 * ba_backward act on this part alone and are not for partitioned use.
 * Synchronises. */
ba_status ba_set_exchange(ba_problem* h, ba_exchange_fn fn, void* ctx, double* xbuf, size_t cap);

/* ---- step-level entry points (same arithmetic as ba_lm_step) ---------- */

/* Copy the cached symbolic phase (Sec. IV-B): perm_cam [O] lists the
 * observations in camera order (ties by observation index), rowptr_cam
 * [C+1]; likewise perm_pt [O], rowptr_pt [P+1].  All dev, int32. */
ba_status ba_get_csr(ba_problem* h, int32_t* perm_cam, int32_t* rowptr_cam,
                     int32_t* perm_pt, int32_t* rowptr_pt, void* stream);

/* a1 + a2 at the current theta: residuals, Jacobian blocks (Sec. III-C), the
 * block normal equations (Alg. 1: A = J^T J and J^T R), then copy
 *   U [C][9][9], V [P][3][3], gc [C][9], gp [P][3]  (dev, double; any may be
 *   NULL), and per observation, in input order, the weighted blocks
 *   sqrt(w) Jc [O][2][9], sqrt(w) Jp [O][2][3] and w [O] (dev, precision
 *   type; any may be NULL). */
ba_status ba_linearize(ba_problem* h, double* U, double* V, double* gc,
                       double* gp, void* Jc, void* Jp, void* w,
                       void* stream);

/* y = S x for the reduced camera system damped with lambda (Eq. 2 with the
 * Schur complement of the point blocks), never forming S.  x, y: dev double
 * [C][9].  Uses the linearisation of the last ba_linearize / LM trial. */
ba_status ba_schur_matvec(ba_problem* h, double lambda, const double* x,
                          double* y, void* stream);

/* One damped solve (Eq. 2) at the current linearisation: block-Jacobi PCG
 * on the reduced system with the given maxiter / tol, then back-
 * substitution.  dc (dev double [C][9]), dp (dev, precision type, [P][3]);
 * iters / rel_res (host, may be NULL) get the PCG count and |r|/|b|.
 * Synchronises. */
ba_status ba_damped_solve(ba_problem* h, double lambda, int maxiter,
                          double tol, double* dc, void* dp, int* iters,
                          double* rel_res, void* stream);

/* ---- stand-alone operations -------------------------------------------- */

/* pixels_out[k] = pi(cams[cam_idx[k]], points[pt_idx[k]]) for k < O: the
 * projection of Eq. 1 with the camera model above.
 * All pointers dev; precision selects float or double.  Indices are not
 * checked (they must be in range). */
ba_status ba_project(int precision, int C, int P, int O, const void* cams,
                     const void* points, const int32_t* cam_idx,
                     const int32_t* pt_idx, void* pixels_out, void* stream);

/* Stable sort of n keys in [0, n_keys) (the symbolic phase, Sec. IV-B):
 * perm_out [n] (dev) lists indices in key order, ties by index; rowptr_out
 * [n_keys + 1] (dev) are the key ranges.  n may be 0.  Keys out of range
 * give BA_ERR_INVALID_ARG.  Allocates its scratch on the device and
 * synchronises the stream. */
ba_status ba_csr_build(const int32_t* keys, int n, int n_keys,
                       int32_t* perm_out, int32_t* rowptr_out, void* stream);

/* Largest n accepted by ba_csr_build_noalloc. */
#define BA_NOALLOC_MAX_KEYS (1 << 20)

/* ba_csr_build without any device allocation, for callers that may not
 * allocate device memory while they run (real-time loops where cudaMalloc /
 * cudaFree could stall the device, processes whose device memory belongs to
 * another allocator, code allowed to allocate only at start-up).  The paper
 * has no counterpart: it is an interface choice of this library.
 * Same arguments, output and errors as ba_csr_build (keys, perm_out,
 * rowptr_out dev; n in [0, BA_NOALLOC_MAX_KEYS], larger n gives
 * BA_ERR_INVALID_ARG); synchronises the stream.  Its scratch is one fixed
 * __device__ array of about 17 MB.  The library's device code is loaded on
 * a device lazily, so the FIRST call on a device (and the first after a
 * cudaDeviceReset) loads it there and reserves the array, which the device
 * then holds until exit: callers that may allocate only at start-up make one
 * warm-up call then (n = 0 is enough), before any stream capture.  Every
 * call looks up the array's device address with the caller's device
 * current; no address is kept across calls.  All calls share the array:
 * calls whose GPU work overlaps race and must be serialised by the caller. */
ba_status ba_csr_build_noalloc(const int32_t* keys, int n, int n_keys,
                               int32_t* perm_out, int32_t* rowptr_out,
                               void* stream);

/* Number of kernel launches the library has issued in this process (for
 * launch accounting in benchmarks; graph replays count every node).
 * Measurement aid: no counterpart in the paper. */
uint64_t ba_kernel_launch_count(void);

/* Entries of ba_get_layout. */
enum {
  BA_LAYOUT_PIECES = 0,  /* camera-major pieces (per-piece partials of the camera passes) */
  BA_LAYOUT_CHUNKS = 1,  /* point chunks (one CTA each in the point-major passes) */
  BA_LAYOUT_FUSED_A = 2, /* 1 if pass A runs fused (point-major, recompute mode) */
  BA_LAYOUT_STORED = 3,  /* 1 if the Jacobian blocks are stored (BA_JAC_STORE) */
  BA_LAYOUT_COUNT = 4
};

/* Layout counts of problem h (see the enum above) into out[0 .. n) (host;
 * entries past BA_LAYOUT_COUNT are 0), for algorithmic-byte accounting in
 * benchmarks.  Measurement aid: no counterpart in the paper. */
ba_status ba_get_layout(const ba_problem* h, int64_t* out, int n);

/* Measured FMA throughput of the CUDA cores in TFLOP/s (2 flops per fused
 * multiply-add), for precision BA_PREC_F64 (double) or BA_PREC_F32
 * (float), into *tflops_out (host): the best of three timed launches of
 * independent FMA chains on every SM, after one warm-up launch.  The
 * denominator of the ALU roofline of kernels bound by arithmetic.
 * Measurement aid: no counterpart in the paper.  Allocates a few bytes and
 * synchronises the stream. */
ba_status ba_measure_fma_peak(int precision, double* tflops_out, void* stream);

/* Kernel classes timed by ba_profile_trials. */
enum {
  BA_K_LIN_CAM = 0,   /* a1+a2 camera-major linearisation pass */
  BA_K_LIN_PT = 1,    /* a1+a2 point-major linearisation pass */
  BA_K_SCHUR_CAM = 2, /* a3 camera-major Schur / block-Jacobi pass */
  BA_K_PASS_A = 3,    /* a4 PCG pass A1 (camera-major, Jp^T Jc p per observation) */
  BA_K_PASS_B = 4,    /* a4 PCG pass B (camera-major, W t) */
  BA_K_COST = 5,      /* a6 trial cost + model reduction pass */
  BA_K_BACKSUB = 6,   /* a5 back-substitution passes */
  BA_K_OTHER = 7,     /* per-camera / per-point / scalar kernels */
  BA_K_PASS_A2 = 8,   /* a4 PCG pass A2 (point-major sum, V*^{-1}) */
  BA_K_PASS_FA = 9,   /* a4 fused point-major pass A (A1 + A2, recompute mode) */
  BA_K_COUNT = 10
};

typedef struct {
  double ms[BA_K_COUNT];        /* summed device time (CUDA events) */
  int64_t launches[BA_K_COUNT]; /* launches that did work */
  double trial_ms;              /* event time of the whole trials */
} ba_kernel_times;

/* Measurement aid (no counterpart in the paper).  Run iters LM trials
 * (Alg. 1; same arithmetic and state changes as ba_solve) with
 * direct launches and a CUDA event pair around every kernel, on the
 * problem's stream, and sum the durations per kernel class into *out (host).
 * PCG launches after convergence (which exit at once) are not counted.
 * Synchronises. */
ba_status ba_profile_trials(ba_problem* h, int iters, ba_kernel_times* out);

/* ------------------------------------------------------------------------
 * Batched form: many independent small problems (sliding windows of
 * uneven size) solved by one persistent launch.  Each problem runs the LM
 * iteration of Alg. 1 with the Schur / block-Jacobi PCG solve as a
 * ba_problem of its own would: same options, same device code, same
 * reduction order.  The compiler forms fused multiply-adds per kernel, so
 * the trials agree with ba_solve's to rounding (not bit for bit).  The
 * paper solves one problem at a time; batching is an interface of this
 * library.
 * ------------------------------------------------------------------------ */

typedef struct ba_batch ba_batch; /* opaque, owned by the library */

/* Cameras per problem accepted by the batched form. */
#define BA_BATCH_MAX_CAMS 28

/* Create a batch of nprob problems, each the problem of Eq. 1 with its own
 * symbolic phase (Sec. IV-B); batching itself has no counterpart in the
 * paper.  cam_counts, pt_counts, obs_counts
 * (host, [nprob]) give problem b's C_b in [1, BA_BATCH_MAX_CAMS], P_b >= 1
 * and O_b >= 1; the totals must fit in int32.  cams [sum C_b][9], points
 * [sum P_b][3], pixels [sum O_b][2] (any) and cam_idx, pt_idx [sum O_b]
 * (dev) are the problems' arrays concatenated in problem order, with
 * cam_idx / pt_idx LOCAL to the problem (camera in [0, C_b), point in
 * [0, P_b)).  Every point must be observed at least once.  opt as for
 * ba_problem_create (pcg_maxiter, pcg_tol, the loss and the damping
 * constants apply to every problem; use_graph is ignored: a solve is
 * always one graph launch).  Out-of-range indices give BA_ERR_INVALID_ARG,
 * non-finite inputs BA_ERR_NONFINITE.  Synchronises. */
ba_status ba_batch_create(ba_batch** out, int nprob, const int32_t* cam_counts,
                          const int32_t* pt_counts, const int32_t* obs_counts,
                          const void* cams, const void* points,
                          const int32_t* cam_idx, const int32_t* pt_idx,
                          const void* pixels, const ba_options* opt,
                          void* stream);
/* Free a batch (NULL is accepted).  Resource management: no counterpart in
 * the paper. */
ba_status ba_batch_destroy(ba_batch* h);

/* Run iters LM trials (Alg. 1, Sec. III-B) of every problem: ONE persistent
 * kernel launch
 * (replayed from a CUDA graph) in which each CTA takes whole problems
 * from a work list.  Stream-ordered. */
ba_status ba_batch_solve(ba_batch* h, int iters, void* stream);

/* Current parameters theta (Eq. 1) of every problem, concatenated in the
 * caller's order
 * (cams_out [sum C_b][9], points_out [sum P_b][3], dev; either may be
 * NULL).  Stream-ordered. */
ba_status ba_batch_get_params(ba_batch* h, void* cams_out, void* points_out,
                              void* stream);

/* Restart every problem (Alg. 1 from its start) from the given parameters
 * (any; NULL: the
 * parameters given at creation): damping lambda0, trial count and
 * statistics cleared, cost re-evaluated on the next solve.
 * Stream-ordered. */
ba_status ba_batch_reset(ba_batch* h, const void* cams, const void* points,
                         void* stream);

/* Per-problem statistics, the records of ba_get_stats (one per pass of
 * Alg. 1's loop): host_out [nprob][cap] (host) receives, for each
 * problem, its last min(trials, cap, max_stats) trials oldest first in row
 * b; n_out [nprob] (host) their counts.  Synchronises.  Returns
 * BA_ERR_NONFINITE (after filling the outputs) if a trial of some problem
 * had a non-finite cost since the last call. */
ba_status ba_batch_get_stats(ba_batch* h, ba_iter_stats* host_out, int cap,
                             int* n_out);

/* Cost F (Eq. 1) at the current parameters and next damping lambda (Eq. 2)
 * of every problem
 * (host [nprob] each; either may be NULL).  Synchronises. */
ba_status ba_batch_get_scalars(ba_batch* h, double* cost, double* lambda);

/* Launch configuration of ba_batch_solve (no counterpart in the paper;
 * results do not depend on it):
 * ctas_per_sm in [1, 64] CTAs per SM in the persistent grid (capped at
 * the number of problems), variant 0 or 1 (register budget for 1 or 2
 * resident CTAs per SM), order 0 (largest problems first) or 1 (the
 * caller's order).  Synchronises. */
ba_status ba_batch_set_launch(ba_batch* h, int ctas_per_sm, int variant, int order);
/* The current launch configuration and the persistent grid size (host
 * outputs, any may be NULL; no counterpart in the paper). */
ba_status ba_batch_get_launch(ba_batch* h, int* ctas_per_sm, int* variant, int* order,
                              int* grid);

/* Segment sizes of the batched solve (no counterpart in the paper; the
 * symbolic phase's cut, Sec. IV-B): each camera's observations in equal
 * pieces of at most piece_max slots (32..2048, default 2048) and each
 * problem's points in chunks of at most chunk_slots observations (32..1024,
 * default 1024) and chunk_pts points (1..512, default 512).  Another cut
 * changes the order of some sums (results move by rounding).  Synchronises. */
ba_status ba_batch_set_segments(ba_batch* h, int piece_max, int chunk_slots, int chunk_pts);

/* The current segment sizes (host outputs, any may be NULL; no counterpart
 * in the paper). */
ba_status ba_batch_get_segments(ba_batch* h, int* piece_max, int* chunk_slots, int* chunk_pts);

/* Autotuner (no counterpart in the paper): time `iters` trials of the
 * batch under every launch
 * configuration (variant x CTAs per SM up to the occupancy limit x
 * order), from the batch's current state each time, and keep the fastest;
 * then, at that launch, every segment size of {256, 512, 1024, 2048} piece
 * slots x {256 / 128, 512 / 256, 1024 / 512} chunk slots / points, keeping
 * the fastest whose final cost of every problem is within 1e-6 (relative)
 * of the current segments' (the gate on the rounding a cut changes); the
 * batch's state is restored afterwards.  With cache_path (host
 * string, may be NULL) the choice is looked up first in, and then appended
 * to, a JSON-lines file keyed by the GPU name, precision, Jacobian mode and
 * a histogram of the problem sizes.  best_ms (host, may be NULL) receives
 * the chosen configuration's time (0 when taken from the cache).
 * Synchronises. */
ba_status ba_batch_autotune(ba_batch* h, int iters, const char* cache_path,
                            double* best_ms);

/* ------------------------------------------------------------------------
 * Learned block-Jacobi correction (not in the paper: its PCG uses a
 * diagonal preconditioner, Sec. IV-C).  A 96-64-64-45 ReLU network maps
 * per-camera quantities of the reduced camera system S to a lower-triangular
 * G (off-diagonal: the outputs; diagonal: exp of the outputs) and the PCG
 * uses M_i = L_i^{-T} G G^T L_i^{-1}, L_i = chol(S_ii), in place of the
 * block-Jacobi inverse S_ii^{-1} (SPD for any output; output 0 gives
 * block-Jacobi).  Features x_i (96, FP32), in the scaled coordinates
 * D = diag(S_ii), S^ = D^{-1/2} S D^{-1/2}: the 36 off-diagonal entries of
 * S^_ii (row-major upper triangle); the 45 entries (row-major upper
 * triangle with diagonal) of R^ = D^{-1/2} (U*_i - S_ii) D^{-1/2} divided by
 * sqrt((1 + R^_aa)(1 + R^_bb)); (ln D_a - mean_a ln D_a) / 10;
 * log10(lambda) / 8; log10(1 + observations of camera i) / 4; 1; three
 * zeros.  Parameters: FP32 [BA_MLP_NPARAM] laid out W1 [64][96], b1 [64],
 * W2 [64][64], b2 [64], W3 [45][64], b3 [45]; the kernels feed the tensor
 * cores BF16 copies of the weights, inputs and activations and accumulate
 * in FP32.  Training loss (per camera, K Rademacher probes z^_k, y^_k =
 * S^ z^_k, A = chol(S^_ii)^{-1}): 1/(9K) sum_k |A^T G G^T A y^_k - z^_k|^2,
 * averaged over the cameras (E_z |M S z - z|^2 in the scaled coordinates).
 * ------------------------------------------------------------------------ */

#define BA_MLP_FIN 96
#define BA_MLP_FOUT 45
#define BA_MLP_NPARAM 13293
#define BA_MLP_KMAX 16

/* Learned correction of the PCG preconditioner (Sec. IV-C uses a fixed
 * diagonal one; this has no counterpart in the paper).  Use the network
 * with parameters params (any, FP32 [BA_MLP_NPARAM], copied) for the
 * preconditioner of every later ba_lm_step / ba_solve /
 * ba_damped_solve of h; NULL returns to block-Jacobi.  Cameras whose S_ii is
 * not positive definite, whose block is not finite or that have a frozen
 * parameter keep the block-Jacobi inverse (counted in precond_fallbacks).
 * ba_backward always uses block-Jacobi. */
ba_status ba_set_preconditioner(ba_problem* h, const float* params, void* stream);

/* Training data for the learned correction (no counterpart in the paper)
 * at the current parameters and damping lambda (> 0):
 * X_out [C][96] features, Ahat_out [C][45] A = chol(S^_ii)^{-1} (packed
 * lower triangle, row-major), and for the K (0..BA_MLP_KMAX) probes zhat
 * [C][K][9] (+-1, FP32) the products Yhat_out [C][K][9] = S^ z^ (one
 * implicit Schur product per probe), and, if D_out is not NULL, the scales
 * D_out [C][9] = diag(S_ii) (FP64).  All dev.  Any +-1 or real probe
 * vectors may be given (e.g. D^{1/2} times slow error components of a
 * truncated PCG).  A camera whose S_ii is not positive definite gets zero
 * features, A = 0, D = 0 and y^ = 0.  The next trial re-linearises.
 * Stream-ordered. */
ba_status ba_learn_collect(ba_problem* h, double lambda, int K, const float* zhat, float* X_out,
                           float* Ahat_out, float* Yhat_out, double* D_out, void* stream);

/* Training probes for the learned correction (no counterpart in the
 * paper): vectors along the slow modes of the block-Jacobi PCG (Sec. IV-C)
 * at the current
 * parameters and damping lambda: x_ref = the PCG solution after maxiter_ref
 * iterations / relative tolerance tol_ref, x_k = the PCG iterate after
 * k = iters[j] iterations (iters host [n], n <= BA_MLP_KMAX), and
 * zhat_out [C][n][9] (dev, FP32) = D^{1/2} (x_ref - x_k) scaled to unit
 * root-mean-square per j (D = diag(S_ii)).  The error of a truncated PCG is
 * dominated by the slow modes of the preconditioned system, which Rademacher
 * probes barely weight.  Synchronises. */
ba_status ba_learn_slow_probes(ba_problem* h, double lambda, int n, const int* iters, int maxiter_ref,
                               double tol_ref, float* zhat_out, void* stream);

/* Network output E_out [n][45] for features X [n][96] (dev, FP32) of the
 * learned correction (no counterpart in the paper).  n >= 0; a NULL
 * pointer with n > 0 gives BA_ERR_INVALID_ARG.  Stream-ordered. */
ba_status ba_mlp_forward(const float* params, int n, const float* X, float* E_out, void* stream);

/* Learned correction (no counterpart in the paper): mean training loss
 * over n samples (X [n][96], Ahat [n][45], Yhat, Zhat
 * [n][K][9], dev, FP32) into *loss_out (host, may be NULL) and its gradient
 * grad_out [BA_MLP_NPARAM] (dev, FP64; summed over fixed tiles of 64 samples
 * in a fixed order).  Synchronises. */
ba_status ba_mlp_loss_grad(const float* params, int n, int K, const float* X, const float* Ahat,
                           const float* Yhat, const float* Zhat, double* grad_out, double* loss_out,
                           void* stream);

/* Training of the learned correction (no counterpart in the paper): Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on params with
 * moments adam_m, adam_v (dev, FP32 [BA_MLP_NPARAM], in/out; zero them for a
 * fresh start), over `epochs` passes of the n samples in minibatches of
 * `batch` consecutive samples (a shorter tail is skipped; shuffle the samples
 * beforehand).  loss_hist (host [epochs], may be NULL) receives each epoch's
 * mean minibatch loss.  Synchronises. */
ba_status ba_mlp_train(float* params, float* adam_m, float* adam_v, int n, int K, const float* X,
                       const float* Ahat, const float* Yhat, const float* Zhat, int epochs, int batch,
                       double lr, double* loss_hist, void* stream);

/* ------------------------------------------------------------------------
 * Pose-graph optimisation (Sec. IV-D, "Generalization to Other
 * Optimization Problems", Eqs. 3-4): poses zeta_i in SE(3), edges e = (i,
 * j) with a measured relative pose T_e and a 6 x 6 information matrix
 * Omega_e; minimise F = 1/2 sum_e r_e^T Omega_e r_e with
 * r_e = Log(zeta_i^{-1} zeta_j T_e^{-1}), by the LM loop of Alg. 1 with
 * the bundle-adjustment loop's options, statistics and decision rule.
 *
 * Conventions (readings: the paper leaves them to its Lie-group library):
 *  - a pose is 7 doubles (tx, ty, tz, qx, qy, qz, qw); quaternions are
 *    normalised on input and returned unit with qw >= 0;
 *  - tangent vectors are (rho, phi), translation first; an LM step updates
 *    zeta_i <- Exp(delta_i) zeta_i (left retraction);
 *  - info is the upper triangle of Omega_e, row by row, 21 doubles;
 *  - fixed (optional, uint8 [N], nonzero = fixed) holds poses in place: the
 *    cost is invariant under a common SE(3) motion of all poses (gauge), so
 *    a problem normally fixes one.
 * Everything is FP64 (ba_options.precision must be BA_PREC_F64, huber_delta
 * 0).  BA_SOLVER_PCG runs block-Jacobi PCG (6 x 6 blocks) on the implicit
 * product (H x)_i = sum_{e at i} B_e (x_i - x_other), B_e = A_e^T Omega_e
 * A_e, in one cooperative launch whose grid barriers wait at most about a
 * second (BA_ERR_TIMEOUT); BA_SOLVER_CHOLESKY factors the 6N x 6N system
 * H + D within its band, in the node order or a reverse Cuthill-McKee order
 * computed at create when that is narrower: half-bandwidth
 * b = 6 max_e |pos(i) - pos(j)| + 5 unknowns.  Only the band is stored
 * (32 x 32 tiles, about 6N (b + 64) doubles; BA_ERR_OOM at create when it
 * does not fit), and the factorisation and both triangular solves run in one
 * cooperative launch in O(N b^2) (up to the dense O(N^3) for a graph with no
 * narrow band).  A pivot that is not positive, or a wait of that launch that
 * runs out (about a second), gives dx = 0 for the trial (a rejection).
 * ------------------------------------------------------------------------ */
typedef struct ba_pgo ba_pgo; /* opaque, owned by the library */

/* Create a pose graph (Sec. IV-D, Eq. 3) of N >= 2 poses and E >= 1 edges:
 * poses (any,
 * [N][7]), ei / ej (any, int32 [E], distinct nodes in [0, N)), meas (any,
 * [E][7], T_e), info (any, [E][21]), fixed (any, uint8 [N], or NULL: none).
 * Evaluates the initial cost.  Errors: BA_ERR_INVALID_ARG (sizes, NULL
 * arrays, an index out of range or an edge from a node to itself, options);
 * BA_ERR_NONFINITE (a non-finite or zero-quaternion input, a non-finite
 * cost); BA_ERR_OOM.  Synchronises the stream; on error *out is NULL. */
ba_status ba_pgo_create(ba_pgo** out, int N, int E, const double* poses,
                        const int32_t* ei, const int32_t* ej,
                        const double* meas, const double* info,
                        const uint8_t* fixed, const ba_options* opt,
                        void* stream);

/* Free a pose graph (NULL is accepted); not in the paper (resource
 * management). */
ba_status ba_pgo_destroy(ba_pgo* h);

/* Run iters LM trials of the pose graph (Alg. 1, Sec. IV-D; a rejected
 * trial counts as one).  Synchronises the stream at the end and reports a device error of any
 * trial (BA_ERR_TIMEOUT for a PCG barrier that ran out). */
ba_status ba_pgo_solve(ba_pgo* h, int iters, void* stream);

/* Current poses Z of Eq. 3 into poses_out (any, [N][7]).  Synchronises. */
ba_status ba_pgo_get_poses(ba_pgo* h, double* poses_out, void* stream);

/* Replace the poses Z of Eq. 3 (any, [N][7]) and re-evaluate the cost;
 * lambda and the statistics are kept.  Synchronises. */
ba_status ba_pgo_set_poses(ba_pgo* h, const double* poses, void* stream);

/* The last min(cap, trials run, max_stats) LM trial records (Alg. 1),
 * oldest first, into host_out; *n_out gets the count.  Synchronises the
 * device. */
ba_status ba_pgo_get_stats(ba_pgo* h, ba_iter_stats* host_out, int cap,
                           int* n_out);

/* Cost F of Eq. 3 at the current poses and the damping of the next trial
 * (Alg. 1).  Synchronises the device. */
ba_status ba_pgo_get_scalars(ba_pgo* h, double* cost, double* lambda);

/* Damping lambda of the next trial (Alg. 1, > 0).  Synchronises the
 * device. */
ba_status ba_pgo_set_lambda(ba_pgo* h, double lambda);

/* Step-level access for parity checks (the residual of Eq. 4 and its
 * Jacobian, Sec. IV-D), at the current poses (each output
 * is any and optional, NULL to skip): r [E][6] residuals, A [E][36]
 * row-major dr_e/d(delta_j) = J_l(r_e)^{-1} Ad(zeta_i^{-1}) (dr_e/d(delta_i)
 * = -A), B [E][36] = A^T Omega A, Hd [N][21] the upper triangles of the
 * diagonal blocks H_ii, g [N][6] = J^T Omega r, *cost = F.  Synchronises. */
ba_status ba_pgo_linearize(ba_pgo* h, double* r, double* A, double* B,
                           double* Hd, double* g, double* cost, void* stream);

/* y = (H + D) x (the damped system of Alg. 1 for Eq. 3) at the current
 * poses with D = lambda clamp(diag H_ii,
 * diag_min, diag_max), over the free poses (x taken as 0 and y set to 0 at
 * fixed ones); x, y any [N][6].  Synchronises. */
ba_status ba_pgo_matvec(ba_pgo* h, double lambda, const double* x, double* y,
                        void* stream);

/* Solve (H + D) dx = -g (one LM step of Alg. 1, Sec. IV-C solvers) at the
 * current poses (fixed poses: dx = 0) with the problem's solver (PCG: maxiter, tol; Cholesky: both ignored); dx any
 * [N][6]; *iters, *rel (optional) the PCG iterations and |r|/|b| at exit.
 * The LM state is not changed.  Synchronises. */
ba_status ba_pgo_damped_solve(ba_pgo* h, double lambda, int maxiter,
                              double tol, double* dx, int* iters, double* rel,
                              void* stream);

/* Synthetic inputs (not in the paper, which reads benchmark files) from
 * given poses (any [N][7]): meas_out (any, [E][7]) =
 * Exp(noise_e) zeta_i^{-1} zeta_j with noise (any, [E][6]) and, if
 * init_out is not NULL, init_out (any, [N][7]) = Exp(drift_n) zeta_n with
 * drift (any, [N][6]).  Synchronises. */
ba_status ba_pgo_synthesize(int N, int E, const double* poses_gt,
                            const int32_t* ei, const int32_t* ej,
                            const double* noise, const double* drift,
                            double* meas_out, double* init_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BA_GB300_H */
