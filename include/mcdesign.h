/*
 * mcdesign -- Monte Carlo engine for the design objective of biomarker
 * clinical trials on NVIDIA GB300 (sm_103a).
 *
 * The objective (Sec. 2.1, Eq. 4 with a point prior; Eq. 2 at mu = 0) is the
 * probability that a trial succeeds,
 *
 *     p = P(X_i > b_i for some i),   X ~ N(mu, Sigma),  d = dim X <= 20,
 *
 * i.e. 1 - Phi_Sigma(b - mu).  The engine estimates p for many designs at
 * once by the Monte Carlo method of Sec. 2.2 (Eq. 6-7) with independent
 * draws per design, returns derivatives of p (Appendix A.3 proves p
 * smooth), and smooths a grid of estimates and takes its argmax (Sec. 2.3).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an mcd_status.  Argument errors are found on the
 *    host and returned at once, before any work is queued.  Errors found by
 *    kernels (a non-positive-definite Sigma, a NaN input) are written to a
 *    device status word of the context and returned by mcd_sync_status().
 *    Nothing aborts the process and no kernel traps.
 *  - Pointers marked DEVICE are device memory of the context's GPU, owned
 *    by the caller, and must stay valid until the queued work has run.
 *    Pointers marked HOST are read during the call only.
 *  - Work is queued on the given stream (NULL: the legacy default stream)
 *    and the call returns without waiting for it, except where noted.
 *  - Host threads: calls on one context may come from several threads (its
 *    autotuning cache is locked), but the context has one error text and one
 *    device status word, so errors of concurrent calls overwrite each other.
 *    To keep them apart, use one context per thread; one plan must not be
 *    launched from two threads at once.
 *  - Determinism: a hit count depends only on (seed, key, draw_begin,
 *    n_draws, d, t = b - mu); it is bit-identical across runs, plans,
 *    batchings, tile sizes and chunkings of the draw range.  Gradient sums
 *    are bit-identical across runs of the same plan.
 *  - Random numbers: normal number m = n*d + i (draw n of the design, axis
 *    i) is taken from Philox4x32-10 (Salmon et al., SC'11) call c = m/4,
 *    output word m%4, counter (c_lo, c_hi, key_lo, key_hi), Philox key
 *    (seed_lo, seed_hi); word x -> u = (2 floor(x/2^9) + 1) 2^-24; words
 *    (0,1) and (2,3) are Box-Muller pairs z = sqrt(-2 ln u0) (cos, sin)(2 pi u1).
 *    Designs with equal keys see identical draws (common random numbers).
 */
#ifndef MCDESIGN_H
#define MCDESIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mcd_status;
#define MCD_OK            0
#define MCD_EINVAL        1  /* bad argument (found on the host)                 */
#define MCD_ENOTSPD       2  /* Sigma of scenario mcd_error_index() is not SPD   */
#define MCD_ECUDA         3  /* a CUDA runtime call failed (text in last_error)  */
#define MCD_ENOMEM        5  /* device or host allocation failed                 */
#define MCD_EUNSUPPORTED  6  /* dimension above MCD_MAX_D, or no sm_103a device  */
#define MCD_ENAN          7  /* NaN in mu or b of design mcd_error_index()       */

#define MCD_MAX_D 20

/* Region whose probability is estimated. */
#define MCD_ANY_EXCEEDS 0    /* some X_i > b_i: success, Eq. 4 (1 - Phi_Sigma)  */
#define MCD_ALL_BELOW   1    /* all X_i <= b_i: the CDF of Eq. 6                 */

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* mcd_stream;

typedef struct mcd_ctx mcd_ctx;
typedef struct mcd_plan mcd_plan;

/* A batch of designs.  Scenario s has dimension scen_d[s] and correlation
 * (or covariance) matrix Sigma_s; design j belongs to scenario
 * design_scen[j] and has mean shift mu_j and thresholds b_j. */
typedef struct {
    int32_t n_scen;               /* S >= 1                                      */
    int32_t n_design;             /* J >= 0                                      */
    const int32_t*  scen_d;       /* HOST [S], each 1..MCD_MAX_D                 */
    const int32_t*  design_scen;  /* HOST [J], each 0..S-1                       */
    const uint64_t* n_draws;      /* HOST [J], draws N_j (0 allowed: p = 0)      */
    const uint64_t* draw_begin;   /* HOST [J] first draw index, or NULL for 0;   */
                                  /*   (draw_begin + n_draws) * d < 2^62          */
    const uint64_t* key;          /* HOST [J] stream key of each design          */
    const double*   Sigma;        /* DEVICE: S row-major d_s x d_s blocks, packed */
                                  /*   in scenario order, symmetric, SPD          */
    const double*   mu;           /* DEVICE: J blocks of d values, design order  */
    const double*   b;            /* DEVICE: same layout as mu; +inf drops a test */
    int32_t region;               /* MCD_ANY_EXCEEDS or MCD_ALL_BELOW            */
} mcd_problem;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` (which must be sm_103).  The
 * context owns a device status word; it allocates nothing else. */
mcd_status mcd_create(mcd_ctx** ctx, int device);
void       mcd_destroy(mcd_ctx* ctx);
/* Text of the last error of this context (never NULL). */
const char* mcd_last_error(const mcd_ctx* ctx);
/* Scenario or design index of the last ENOTSPD / ENAN error, else -1. */
int64_t    mcd_error_index(const mcd_ctx* ctx);
/* Wait for `stream`, then read and clear the device status word. */
mcd_status mcd_sync_status(mcd_ctx* ctx, mcd_stream stream);

/* ---- plans: set up once, launch many times ------------------------------ */

#define MCD_PLAN_GRAD      1  /* also allocate the workspace of mcd_plan_grad  */
#define MCD_PLAN_AUTOTUNE  2  /* time tile shapes on this GPU, keep the fastest */
#define MCD_PLAN_GRAPH     4  /* replay launches from a captured CUDA graph    */
#define MCD_PLAN_FP64      8  /* all-FP64 sampling (normals, L z, sums); one d */
#define MCD_PLAN_TIMING   16  /* record CUDA events around the sampling kernels */
#define MCD_PLAN_SHARED   32  /* shared-draw kernel for common-random-number groups */

/* MCD_PLAN_SHARED: designs with equal (design_scen, key, draw_begin, n_draws)
 * see the same draws (common random numbers).  Groups of at least
 * MCD_SHARED_MIN such designs are evaluated by the shared-draw kernel, which
 * makes each draw once per block and tests it against every design of the
 * group: hit counts are bit-identical to the per-design kernel, the
 * likelihood-ratio sums equal up to FP32 rounding.  The sigmoid sums skip,
 * warp by warp, the draws whose every contribution is zero or below 3e-8
 * (no design of the warp within 25 h / log2(e) of the region's boundary in
 * its smallest margin), which moves the sigmoid gradient's G / N by less
 * than 3e-8.  Smaller groups keep the per-design kernel.  Not with
 * MCD_PLAN_FP64 (MCD_EUNSUPPORTED). */
#define MCD_SHARED_MIN    32

/* Plan a problem.  Reads the HOST arrays (copied), keeps the DEVICE
 * pointers Sigma, mu, b (their contents are read at each launch), uploads
 * the tile schedule and allocates the workspace (blocking).  With
 * MCD_PLAN_AUTOTUNE it runs timing launches on the GPU (blocking).
 * k: number of design parameters of the Jacobian that mcd_plan_grad takes
 * (1..8), or 0 for gradients with respect to mu.
 * With MCD_PLAN_GRAD a design's draws are spread over at most 32 batch
 * slots whose sums are 64-bit fixed point; a design that would put more
 * than 2^32 draws into one slot (about 1.3e11 draws per design) is refused
 * with MCD_EINVAL and its index, since its sums could overflow. */
mcd_status mcd_plan_create(mcd_ctx* ctx, const mcd_problem* prob, int32_t flags,
                           int32_t k, mcd_plan** plan);
/* Free a plan.  It may be called before or after mcd_destroy of its context
 * (the plan keeps its own device index), but not while its work runs. */
void       mcd_plan_destroy(mcd_plan* plan);

/* Estimate p for every design (Sec. 2.2, Eq. 7 with independent draws).
 *   hits[J] (DEVICE, u64, may be NULL): draws in the region, exact;
 *   p[J]    (DEVICE, may be NULL): hits / N;
 *   se[J]   (DEVICE, may be NULL): sqrt(p (1 - p) / N), the standard error
 *           that Eq. 8 bounds by 1 / (2 sqrt N). */
mcd_status mcd_plan_eval(mcd_plan* plan, uint64_t seed, uint64_t* hits, double* p,
                         double* se, mcd_stream stream);

/* Estimate p and its derivatives in the same sampling pass.
 *   dt_dtheta (DEVICE, [J][d][k] row-major per design, or NULL when the plan
 *     has k = 0): Jacobian of t = b - mu with respect to k design parameters.
 *   h_sigmoid: bandwidth (in units of X) of the smoothed indicator
 *     1 - prod_i sigma((b_i - X_i) / h), sigma(u) = 1 / (1 + e^-u); <= 0 skips it.
 *   grad_lr  [J][k] (or packed like mu when k = 0): likelihood-ratio
 *     estimate, grad_mu p = Sigma^-1 E[(1_R - p)(X - mu)], chained as
 *     grad_theta p = -(dt/dtheta)^T grad_mu p (the sign of grad_mu flips
 *     for MCD_ALL_BELOW);
 *   grad_sig [J][k] (or like mu): the same derivative of the smoothed
 *     indicator (pathwise), or untouched when h_sigmoid <= 0;
 *   grad_se  [J][k] (or like mu): batch-means standard error of grad_lr;
 *   hits, p as in mcd_plan_eval.  Any output pointer may be NULL. */
mcd_status mcd_plan_grad(mcd_plan* plan, uint64_t seed, const double* dt_dtheta,
                         double h_sigmoid, uint64_t* hits, double* p, double* grad_lr,
                         double* grad_sig, double* grad_se, mcd_stream stream);

/* Launch configuration chosen by the plan for dimension d: threads per
 * block, draws per tile and resident blocks per SM (for reports). */
mcd_status mcd_plan_config(const mcd_plan* plan, int32_t d, int32_t* threads,
                           int64_t* tile_draws, int32_t* blocks_per_sm);

/* Number of tiles in the plan's schedule. */
int64_t    mcd_plan_tiles(const mcd_plan* plan);

/* For a plan created with MCD_PLAN_TIMING: wait for the last launch and
 * return the time from the start of its first sampling kernel to the end of
 * its last one, in milliseconds (CUDA events on the launch stream). */
mcd_status mcd_plan_kernel_ms(mcd_plan* plan, float* ms);

/* ---- one-shot calls (plan, launch, release) ----------------------------- */

/* Plan, launch and release in one call.  The planning reads the HOST
 * arrays before returning; the workspace is allocated and freed in stream
 * order (cudaMallocAsync / cudaFreeAsync).  Not for use under stream capture;
 * plans are. */
mcd_status mc_design_eval(mcd_ctx* ctx, const mcd_problem* prob, uint64_t seed,
                          uint64_t* hits, double* p, double* se, mcd_stream stream);

/* Estimate p and its derivatives for every design in one call (plan with
 * MCD_PLAN_GRAD and k, launch mcd_plan_grad, release).  Appendix A.3 shows
 * that the objective is a smooth function of the design, and its derivative
 * an integral over the same law as p itself, so it is estimated from the
 * same draws:
 *   likelihood ratio: grad_mu p = Sigma^-1 E[(1_R - p)(X - mu)]
 *     = L^-T E[(1_R - p) z] (X = mu + L z; the control variate p E[z] = 0
 *     lowers the variance), chained as grad_theta p = -(dt/dtheta)^T grad_mu p;
 *   sigmoid (pathwise): the derivative of E[1 - prod_i sigma((b_i - X_i)/h)],
 *     a smoothed indicator with bandwidth h, when h_sigmoid > 0.
 * Arguments and outputs as in mcd_plan_create (k) and mcd_plan_grad; the
 * workspace is allocated and freed in stream order (cudaMallocAsync /
 * cudaFreeAsync), so not for use under stream capture. */
mcd_status mc_design_grad(mcd_ctx* ctx, const mcd_problem* prob, uint64_t seed,
                          int32_t k, const double* dt_dtheta, double h_sigmoid,
                          uint64_t* hits, double* p, double* grad_lr, double* grad_sig,
                          double* grad_se, mcd_stream stream);

/* Estimate p for the designs of one scenario without allocating memory.
 * The paper has no counterpart: this is an entry point for callers that
 * cannot allocate device memory at the point where they evaluate designs --
 * code that hands all device memory to its own pool up front (a stray
 * cudaMalloc there can fail or fragment the pool), loops that must not take
 * the implicit synchronisation of cudaMalloc / cudaFree, processes whose
 * allocator belongs to another runtime.  It needs no context and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   Scratch: the hit counters, stream keys and Cholesky factor live in one
 *   static device array of the library (about 260 KB, held on every GPU that
 *   loads the library until the process exits).  All calls share it and it
 *   keeps the last call's contents (the counters are cleared by each call);
 *   calls whose GPU work overlaps -- on different streams, or from several
 *   host threads -- race on it and must be serialised by the caller.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current.
 *   Limits: n_scen == 1, n_design <= 16384, every n_draws[j] equal,
 *   draw_begin NULL or all 0; otherwise MCD_EINVAL, before any work.
 *   Inputs and outputs as in mc_design_eval (the stream keys are copied from
 *   the HOST array on `stream`).  A non-positive-definite Sigma gives p = se =
 *   NaN and hits = 0 for every design, a NaN in mu_j or b_j the same for
 *   design j; hits are bit-identical to mc_design_eval's otherwise. */
mcd_status mc_design_eval_noalloc(int device, const mcd_problem* prob, uint64_t seed,
                                  uint64_t* hits, double* p, double* se, mcd_stream stream);

/* ---- FWER calibration (Eq. 2) ------------------------------------------- */

/* Calibrate each design's alpha split to the family-wise error rate alpha0
 * on the device.  Eq. 2 constrains the thresholds b_i = Z_{1 - alpha_i} so
 * that, under the null hypothesis (mu = 0), 1 - Phi_Sigma(b) = alpha0; as in
 * the paper's reparametrisation (Sec. 2.1) the split w of the alpha budget
 * is fixed and its scale s solved for: alpha = s w.
 *   prob: scenarios (DEVICE Sigma), and per design its scenario, stream key,
 *     draw count and first draw (HOST); prob->mu and prob->b are not read,
 *     prob->region must be MCD_ANY_EXCEEDS.  Designs whose scenario, key and
 *     draw range agree share their draws (MCD_PLAN_SHARED).
 *   w (DEVICE [sum d], layout of mu): the split, w_i >= 0 and finite, some
 *     w_i > 0; w_i = 0 drops test i (b_i = +inf).  A split that breaks this
 *     is reported by mcd_sync_status as MCD_EINVAL with the design index, and
 *     its outputs are NaN.
 *   alpha0 in (0, 1); rounds in 2..200 evaluation rounds: rounds 0 and 1
 *     evaluate the Bonferroni bracket [alpha0 / sum w, alpha0 / max w], later
 *     rounds false-position (Illinois) steps inside it.
 *   scale (DEVICE [J]): the scale of the last round;  b (DEVICE [sum d]):
 *     its thresholds Z_{1 - scale w} (also the sampler's thresholds during
 *     the call);  fwer (DEVICE [J]): the Monte Carlo FWER at that scale.
 * Every round uses the same draws, so each design's estimated FWER is a
 * nondecreasing step function of s and the bracket keeps the crossing; the
 * scale's error is that of the estimate, about
 * sqrt(alpha0 (1 - alpha0) / N) / (dFWER/ds).  The workspace is allocated
 * and freed in stream order; not for use under stream capture. */
mcd_status mc_fwer_calibrate(mcd_ctx* ctx, const mcd_problem* prob, const double* w, double alpha0,
                             int32_t rounds, uint64_t seed, double* scale, double* b, double* fwer,
                             mcd_stream stream);

/* ---- thin-plate spline smoothing and its maximiser (Sec. 2.3) ---------- */

/* Fit a thin-plate smoothing spline to each of n_surf sets of n_pts
 * scattered estimates in k = 1..3 dimensions (Sec. 2.3 fits a TPS to the
 * N3 estimates P_hat(alpha)):
 *   f(x) = sum_i c_i eta(|x - x_i|) + d_0 + sum_j d_j x_j,
 *   (K + smoothing I) c + P d = y,  P^T c = 0,  P = [1, x],
 * eta(r) = r^3 (k = 1), r^2 log r (k = 2), -r (k = 3); smoothing = 0
 * interpolates.  Solved on the device in FP64: Householder QR of P removes
 * the side condition, a blocked Cholesky factors the projected system.
 *   x (DEVICE [n_surf][n_pts][k]), y (DEVICE [n_surf][n_pts]);
 *   coef (DEVICE [n_surf][n_pts + k + 1]): c_0..c_{n_pts-1}, d_0..d_k;
 *   fitted (DEVICE [n_surf][n_pts], may be NULL): f at the data, y - smoothing c.
 * Needs k + 2 <= n_pts <= 16384 and points that P does not make singular
 * (not all on one line for k = 2, ...).  A system that is not positive
 * definite after the projection (repeated points with smoothing 0) gives NaN
 * outputs for that surface and MCD_ENOTSPD with its index at mcd_sync_status.
 * Workspace n_pts^2 doubles, allocated and freed in stream order; not for use
 * under stream capture.  Several surfaces are fitted at once on up to four
 * worker streams, each with its own workspace (the workspace above per
 * worker, at most about 4 GB in all), and the factorisation also runs
 * kernels on a stream of its own; all of these are joined to `stream` by
 * events, so all of the call's work is done when the work queued on
 * `stream` is. */
mcd_status mc_tps_fit(mcd_ctx* ctx, int32_t n_surf, int32_t n_pts, int32_t k, const double* x,
                      const double* y, double smoothing, double* coef, double* fitted, mcd_stream stream);

/* Generalised cross-validation score of the smoothing spline of one set of
 * estimates for each of n_s smoothing values: with A_s the influence matrix
 * (fitted values = A_s y), V(s) = n_pts |(I - A_s) y|^2 / tr(I - A_s)^2.
 * The smoothing that minimises V is the usual automatic choice for a thin
 * plate spline (Sec. 2.3 does not state how its spline was tuned).
 *   x, y: DEVICE as in mc_tps_fit (one surface);  s_values: HOST [n_s],
 *   each finite and > 0, n_s in 1..256;  score: DEVICE [n_s], NaN where the
 *   system is singular to working precision at that s.
 * Per value one FP64 Cholesky and one triangular inverse (tr(I - A_s) is
 * s |L^{-1}|_F^2); workspace 3 n_pts^2 doubles, in stream order; not for use
 * under stream capture.  Like mc_tps_fit, it also uses a stream of its own,
 * joined to `stream` by events. */
mcd_status mc_tps_gcv(mcd_ctx* ctx, int32_t n_pts, int32_t k, const double* x, const double* y,
                      int32_t n_s, const double* s_values, double* score, mcd_stream stream);

/* Maximise each fitted spline inside the box lo <= x <= hi (DEVICE [k] each,
 * shared by all surfaces), as Sec. 2.3 does with a quasi-Newton method
 * started at the best fitted point: projected BFGS with Armijo backtracking,
 * at most `iters` iterations, started at the data point inside the box with
 * the largest fitted value (lowest index on ties).
 *   x, coef, fitted: as written by mc_tps_fit;
 *   x_best (DEVICE [n_surf][k]), f_best (DEVICE [n_surf]): the maximiser and
 *   f there. */
mcd_status mc_tps_argmax(mcd_ctx* ctx, int32_t n_surf, int32_t n_pts, int32_t k, const double* x,
                         const double* coef, const double* fitted, const double* lo, const double* hi,
                         int32_t iters, double* x_best, double* f_best, mcd_stream stream);

/* ---- smoothing and argmax (Sec. 2.3) ------------------------------------ */

/* Local-polynomial smoothing of n_scen grids of g1 x g2 values (row-major,
 * scenario-major; a grid with g1 == 1 or g2 == 1 is smoothed along its one
 * axis), then the argmax per scenario.
 *   value (DEVICE [S*g1*g2]): the noisy estimates, e.g. p from mcd_plan_eval;
 *   bandwidth: tricube half-width in grid steps, 1 < bandwidth <= 4 (points
 *     closer than this get positive weight);  degree: 0, 1 or 2 (2 fits
 *     {1, x, y, x^2, xy, y^2});  windows are cut at the grid edges and the
 *     least-squares weights are solved in FP64;
 *   smoothed (DEVICE [S*g1*g2], may be NULL): smoothed values, applied in
 *     FP32 from FP64 weights (absolute error below 1e-6 for values in [0,1]);
 *   argmax_idx / argmax_val (DEVICE [S]): lowest row-major index of the
 *     largest smoothed value, and that value;
 *   raw_idx / raw_val (DEVICE [S], may be NULL): the same for the input.
 * Needs g1, g2 >= 1 and, along each smoothed axis, at least degree + 1
 * points within every window.  Limits: g1 * g2 < 2^31, n_scen <= 65535 and,
 * for 2-D grids, g1 <= 65535 * 32; beyond them MCD_EINVAL. */
mcd_status mc_smooth_argmax(mcd_ctx* ctx, int32_t n_scen, int32_t g1, int32_t g2,
                            const double* value, double bandwidth, int32_t degree,
                            double* smoothed, int64_t* argmax_idx, double* argmax_val,
                            int64_t* raw_idx, double* raw_val, mcd_stream stream);

/* mc_smooth_argmax on FP32 grids (the same smoothing of Sec. 2.3, weights,
 * edge rules, limits and errors): value, smoothed, argmax_val and raw_val are
 * FP32 (DEVICE).  The stencil already runs in FP32, so the results equal
 * mc_smooth_argmax's on the same values rounded to FP32; the grid moves half
 * the bytes through HBM.  Estimates p in [0, 1] lose nothing that matters
 * against their Monte Carlo error (FP32 spacing 6e-8 at 1). */
mcd_status mc_smooth_argmax_f32(mcd_ctx* ctx, int32_t n_scen, int32_t g1, int32_t g2,
                                const float* value, double bandwidth, int32_t degree,
                                float* smoothed, int64_t* argmax_idx, float* argmax_val,
                                int64_t* raw_idx, float* raw_val, mcd_stream stream);

/* ---- unit-check entry points -------------------------------------------- */

/* Normals m_begin .. m_begin+count-1 of stream (seed, key) exactly as the
 * sampling kernels make them: FP32 path into z32, FP64 path into z64 and the
 * raw Philox words of calls m_begin/4 .. (m_begin+count-1)/4 into words
 * (4 per call).  Any output (DEVICE) may be NULL. */
mcd_status mcd_debug_normals(mcd_ctx* ctx, uint64_t seed, uint64_t key, uint64_t m_begin,
                             uint64_t count, float* z32, double* z64, uint32_t* words,
                             mcd_stream stream);

/* Host-side fault injection for tests of error handling: the next launch
 * of any plan of this context (mcd_plan_eval, mcd_plan_grad, the one-shot
 * calls) queues no GPU work and returns MCD_ECUDA, with the text of CUDA
 * error `cuda_error` and "injected" in mcd_last_error().  0 clears a pending
 * injection.  Nothing reaches the GPU, so the context stays usable. */
mcd_status mcd_debug_fail_next(mcd_ctx* ctx, int32_t cuda_error);

/* ---- measurement --------------------------------------------------------- */

/* Instruction classes of the sampling kernels, for mcd_pipe_rate. */
#define MCD_PIPE_MUL_WIDE  0   /* mad.wide.u32: 32x32->64 multiply-add (Philox)    */
#define MCD_PIPE_MAD_LO    1   /* mad.lo.u32: 32-bit integer multiply-add          */
#define MCD_PIPE_LOP3      2   /* lop3.b32: three-input logic (Philox xors)        */
#define MCD_PIPE_FFMA      3   /* fma.rn.f32 (L z, Box-Muller, adjoint sums)       */
#define MCD_PIPE_LG2       4   /* lg2.approx.ftz.f32 (Box-Muller radius)           */
#define MCD_PIPE_SQRT      5   /* sqrt.approx.ftz.f32 (Box-Muller radius)          */
#define MCD_PIPE_SIN       6   /* sin.approx.ftz.f32 (Box-Muller angle)            */
#define MCD_PIPE_COS       7   /* cos.approx.ftz.f32 (Box-Muller angle)            */
#define MCD_PIPE_EX2       8   /* ex2.approx.ftz.f32 (sigmoid of the adjoint)      */
#define MCD_PIPE_RCP       9   /* rcp.approx.ftz.f32 (sigmoid of the adjoint)      */
#define MCD_PIPE_MIXED    10   /* half fma.rn.f32, half lop3.b32 (co-issue)        */
#define MCD_PIPE_LDS128   11   /* ld.shared.v4 at a warp-uniform address (L, d > 6) */
#define MCD_PIPE_PHILOX   12   /* Philox rounds 2..10 as sampled, per wide multiply */
#define MCD_PIPE_FFMA2    13   /* fma.rn.f32x2: two FP32 FMAs per instruction (L z) */
#define MCD_PIPE_COUNT    14

/* Throughput of one instruction class on this device, in operations per SM
 * clock: the median over SMs of a microbenchmark in which every thread runs
 * eight dependency chains of that instruction, 8 blocks of 256 threads per
 * SM, timed with the SM's cycle counter (MCD_PIPE_FFMA2: packed instructions,
 * each two FMAs, per SM clock).  With the per-draw operation counts
 * of the estimator (Sec. 2.2) this bounds draw-evaluations per clock per SM
 * from above.
 *   op: MCD_PIPE_*;  iters: chain steps per thread, 1 <= iters <= 2^20 (each
 *     thread issues 8 * iters instructions of the class, 36 * iters wide
 *     multiplies for MCD_PIPE_PHILOX);
 *   rate (HOST [1]): operations per SM clock.
 * Allocates and frees its own device buffers on the stream and synchronises
 * it.  MCD_EINVAL for an unknown op or iters out of range. */
mcd_status mcd_pipe_rate(mcd_ctx* ctx, int32_t op, int32_t iters, double* rate, mcd_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MCDESIGN_H */
