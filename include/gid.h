/*
 * gid.h -- C ABI of the B300 (sm_103a) illumination decomposition solver.
 *
 * The library computes, per video frame, the decomposition of Sec. 3
 * (eq:imageformation)
 *
 *     I(x) = R(x) * sum_{k=0..K} b_k T_k(x),   b_0 = (1, 1, 1),
 *
 * into reflectance R, direct illumination T_0 and K indirect layers T_1..T_K,
 * by the alternating sparse-dense solve of Sec. 6.1: a Gauss-Newton step on the
 * layers (normal equations of eq:optimization solved by M steps of Jacobi-
 * preconditioned conjugate gradient, IRLS reweighting of Sec. 5.3) with the base
 * colours fixed, then the base-colour refinement of eq:basecolorrefinement with
 * the layers fixed.  The energy is eq:giv-energy with the terms of Sec. 5.
 *
 * Conventions shared by every call:
 *   - Every function returns GID_OK (0) or a negative GID_ERR_* code and never
 *     throws; gid_last_error() gives a message for the last failure.
 *   - Image buffers are planar, contiguous, float32 (or uint8 for labels):
 *     channel-major [C][H][W].  Pointers named *_dev are CUDA device pointers,
 *     *_host are host pointers.  The caller owns every buffer it passes; the
 *     library copies what it keeps.  The context owns its internal device
 *     buffers and frees them in gid_destroy().
 *   - Work is enqueued on the CUDA stream given to gid_create() (0 = legacy
 *     default stream) and is asynchronous unless a call says it synchronises.
 *   - There is no CPU fallback: without a usable CUDA device gid_create() fails
 *     with GID_ERR_CUDA.
 */
#ifndef GID_H
#define GID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GID_OK 0
#define GID_ERR_INVALID_ARG (-1) /* bad size, pointer or flag */
#define GID_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define GID_ERR_OOM (-3)         /* device allocation failed */
#define GID_ERR_STATE (-4)       /* call out of order, e.g. gid_run before gid_set_frame */
#define GID_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */
#define GID_ERR_NUMERIC (-6)     /* non-finite energy/state or a singular base-colour system */

#define GID_MAX_K 10     /* base colours (the paper uses an upper bound of K = 10, Sec. 4.1) */
#define GID_MAX_PAIRS 8  /* consistency pair offsets per kind (spatial / temporal) */

/* Term weights and solver readings.  Defaults (gid_default_weights) are the
 * fixed parameter set of Sec. 7 "Parameters": lambda_clustering 200,
 * lambda_rsparsity 20, p 1, lambda_isparsity 3, lambda_smoothness 3,
 * lambda_nonneg 1000, lambda_data 5000, lambda_IR 10, lambda_CR 100,
 * lambda_rconsistency = lambda_monochrome = 10; eps 0.002 (Sec. 5.3.1);
 * soft-Retinex sharpness 50 (Sec. 5.2). */
typedef struct {
  float lambda_data, lambda_clustering, lambda_rsparsity, p, lambda_rconsistency, lambda_monochrome,
      lambda_isparsity, lambda_smoothness, lambda_nonneg, lambda_IR, lambda_CR, eps, retinex_sharpness;
  float consistency_tau;  /* soft chromaticity closeness exp(-|dC|^2/tau^2) of the pairs, default 0.05 */
  int nonneg_strict;      /* 1 (default): non-neg weight is 0 only for T > 0, as printed in Sec. 5.3.1 */
  int irls_half;          /* 1: halve every IRLS weight (majorise-minimise variant); default 0 */
  int rcluster_follows_b; /* 1: R_cluster uses the refined base colours; default 0 (initial colours) */
  int temporal;           /* 1: temporal consistency pairs against the previous solved frame */
  int refine_base_colors; /* 0 off, 1 after every Gauss-Newton step (default), 2 on the first frame only */
  int n_spatial_pairs;    /* <= GID_MAX_PAIRS */
  int n_temporal_pairs;   /* <= GID_MAX_PAIRS */
  int spatial_offsets[2 * GID_MAX_PAIRS];  /* (dy, dx) per pair, |dy|,|dx| <= 3 */
  int temporal_offsets[2 * GID_MAX_PAIRS]; /* (dy, dx) per pair into the previous frame, |dy|,|dx| <= 3 */
} gid_weights;

typedef struct gid_ctx gid_ctx;

/* Fill *w with the defaults above, no pairs and temporal off. */
void gid_default_weights(gid_weights* w);

/* Create a solver for H x W frames with K base colours (1 <= K <= GID_MAX_K,
 * H, W >= 1).  Allocates about (11 K + 67) planes of H x W floats on the
 * current device.  stream: a cudaStream_t or NULL.  On success *out owns the
 * context; on failure *out is NULL and the code says why (GID_ERR_OOM,
 * GID_ERR_CUDA, GID_ERR_INVALID_ARG). */
int gid_create(int H, int W, int K, const gid_weights* w, void* stream, gid_ctx** out);

/* Free every device buffer of the context.  NULL is a no-op. */
void gid_destroy(gid_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing gid_create
 * when ctx is NULL).  Valid until the next call on ctx. */
const char* gid_last_error(const gid_ctx* ctx);

/* Initial base colours b_1..b_K (K x 3 row-major, host): the clustered colours
 * of Sec. 4.1.  They are the anchor of the refinement (eq:basecolorrefinement)
 * and the colours of R_cluster.  Also resets the refined colours to them.
 * Every value must be finite and > 0 (R_cluster uses ln b).  Synchronises. */
int gid_set_base_colors(gid_ctx* ctx, const float* b_host);

/* Current (refined) base colours b_1..b_K into b_host (K x 3).  Synchronises. */
int gid_get_base_colors(gid_ctx* ctx, float* b_host);

/* Ingest a frame: rgb_dev is 3 x H x W float32 (the frame I), labels_dev is
 * H x W uint8 with values 0..K-1, the cluster of each pixel (label k-1 means
 * base colour b_k).  Computes the chromaticity C = I / (I_R + I_G + I_B + 1e-6)
 * (Sec. 4.1), the soft-Retinex weight w_SR of Sec. 5.2 and the consistency pair
 * weights.  If temporal pairs are on and a frame was solved before, that
 * frame's log reflectance and chromaticity become the previous frame.  Labels
 * >= K are reported as GID_ERR_INVALID_ARG by the next synchronising call. */
int gid_set_frame(gid_ctx* ctx, const float* rgb_dev, const uint8_t* labels_dev);

/* Start a new video on this context: forget the previous frame (the next frame
 * gets no temporal pairs), reset the refined base colours to the initial ones
 * and count the next frame as the first (refine_base_colors = 2).  Async. */
int gid_new_sequence(gid_ctx* ctx);

/* Initial state: mode 0 = cold start (r = ln R_cluster, T_0 = mean_c I /
 * mean_c R_cluster, T_k = 0), mode 1 = warm start (keep the previous frame's
 * layers and base colours; needs a solved frame).  Requires gid_set_frame. */
int gid_init(gid_ctx* ctx, int mode);

/* Run n_outer flip-flop iterations (Sec. 6.1): each a Gauss-Newton step of
 * exactly m_inner PCG steps on the layers, then (per refine_base_colors) the
 * base-colour step.  Asynchronous.  n_outer >= 0, m_inner >= 1.  The launch
 * sequence is recorded once per (n_outer, m_inner, refinement, temporal pairs,
 * tile shape) as a CUDA graph and replayed on a context-owned stream, ordered
 * after earlier work on the context stream and before later work on it. */
int gid_run(gid_ctx* ctx, int n_outer, int m_inner);

/* enable = 0: launch gid_run's kernels one by one on the context stream
 * (profiling does this automatically); 1 (default): graph replay. */
int gid_set_graphs(gid_ctx* ctx, int enable);

/* Layers of the current state: R_dev (3 x H x W) = exp(r), T_dev ((K+1) x H x W)
 * = T_0..T_K.  Either pointer may be NULL.  Asynchronous. */
int gid_get_layers(gid_ctx* ctx, float* R_dev, float* T_dev);

/* Layer recombination for the editing applications of Sec. 7.4, from the
 * current layers and refined base colours b:
 *     out(x) = R'(x) * (T_0(x) + sum_k g_k b'_k T_k(x)),
 *     R'_c(x) = R_c(x) * b'_jc / b_jc where mask(x) = j in 1..K and b_jc != 0,
 *               else R_c(x).
 * Recolouring an object: a new colour b'_j and a mask of its pixels (its
 * indirect light on other surfaces follows b'_j); colour keying: a new colour
 * for one indirect layer, no mask; spill suppression: gain g_k = 0 for the
 * spilling layer.  b_new_host K x 3 (finite; NULL = b), gain_host K
 * (NULL = all 1), mask_dev H x W uint8 (NULL = none; values > K count as 0),
 * out_dev 3 x H x W float32, device.  Async unless b_new_host is NULL. */
int gid_recombine(gid_ctx* ctx, const float* b_new_host, const float* gain_host, const uint8_t* mask_dev,
                  float* out_dev);

/* Raw unknowns X ((K+4) x H x W: r_R, r_G, r_B, T_0..T_K, r = ln R) to / from
 * device memory.  gid_set_state also marks the context initialised.  Async. */
int gid_get_state(gid_ctx* ctx, float* X_dev);
int gid_set_state(gid_ctx* ctx, const float* X_dev);

/* One base-colour step (eq:basecolorrefinement) on the current layers, as
 * gid_run does after each Gauss-Newton step: b = b_init + Delta b from the
 * three K x K normal equations (FP64 Cholesky).  A singular block is reported
 * as GID_ERR_NUMERIC by the next synchronising call.  Async. */
int gid_base_color_step(gid_ctx* ctx);

/* Exact energy of the current state (eq:giv-energy; the l1, l_p and max terms
 * exactly, not their IRLS surrogates): per_term[8] in the order data,
 * clustering, r-sparsity, r-consistency, monochrome, i-sparsity, smoothness,
 * non-neg; *total their sum (FP64 reductions).  Either pointer may be NULL.
 * Synchronises; returns GID_ERR_NUMERIC if the state is not finite, and any
 * error a device step recorded since the last synchronising call. */
int gid_energy(gid_ctx* ctx, double* total, double* per_term);

/* gid_energy restricted to the pixels where mask_dev (H x W uint8, device) is
 * nonzero: each pixel contributes its data, clustering, monochrome, i-sparsity
 * and non-neg terms and the r-sparsity, smoothness and consistency terms
 * evaluated at it (so complementary masks add up to gid_energy).  NULL = all
 * pixels.  Synchronises. */
int gid_energy_region(gid_ctx* ctx, const uint8_t* mask_dev, double* total, double* per_term);

/* One whole frame with host buffers: copy rgb_host (3 x H x W) and labels_host
 * (H x W) to the device, gid_set_frame, gid_init(init_mode), gid_run(n_outer,
 * m_inner), copy R (3 x H x W), T ((K+1) x H x W) and the refined base colours
 * (K x 3) back.  Output pointers may be NULL.  Staging buffers are allocated on
 * the first call.  Synchronises. */
int gid_solve_frame_host(gid_ctx* ctx, const float* rgb_host, const uint8_t* labels_host, int init_mode,
                         int n_outer, int m_inner, float* R_host, float* T_host, float* b_host);

/* A sequence of n frames with host buffers, pipelined: frame t + 1's upload and
 * frame t's download run on a context-owned copy stream while frame t is
 * solved (double-buffered device staging, ordered by events).  Per frame:
 * gid_set_frame, gid_init (first_init_mode, 0 or 1, for frame 0; warm start
 * for the others), gid_run(n_outer, m_inner), then R, T and the refined base
 * colours of that frame.  rgb_host n x 3 x H x W, labels_host n x H x W,
 * R_host n x 3 x H x W, T_host n x (K+1) x H x W, b_host n x K x 3 (outputs may
 * be NULL).  Host buffers should be page-locked for the copies to overlap.
 * Results equal n calls of gid_solve_frame_host.  Synchronises. */
int gid_solve_video_host(gid_ctx* ctx, int n, const float* rgb_host, const uint8_t* labels_host,
                         int first_init_mode, int n_outer, int m_inner, float* R_host, float* T_host, float* b_host);

/* Chromaticity clustering of Sec. 4.1, on the GPU: the initial base colours
 * and the cluster labels a solve starts from.  Chromaticity C = I /
 * (I_R + I_G + I_B + 1e-6); a histogram with 10 partitions per axis of C in
 * [0, 1]^3 (outside values in the edge bins); weighted k-means on the occupied
 * bins' mid-points weighted by their populations, at most k_max centres
 * initialised at the k_max most populated bins (ties by bin index), iterated
 * until no bin changes cluster (at most 100 times); while two centres are
 * closer than merge_dist (the paper's 0.2) the smaller cluster joins the
 * larger (population-weighted centre, closest pair first); clusters ordered by
 * decreasing population; every pixel labelled with its closest centre; initial
 * base colours = the mean RGB of each cluster's pixels.
 *   rgb_dev     3 x H x W float32 frame (device)
 *   k_max       1..GID_MAX_K (the paper uses 10)
 *   labels_dev  out, H x W uint8 in 0..k_out-1 (device)
 *   b_host      out, k_out x 3 float32 (room for k_max x 3)
 *   k_out       out, the number of clusters after merging
 * Allocates and frees its own scratch; synchronises the stream.  Errors are
 * written to errbuf (may be NULL). */
int gid_cluster(int H, int W, const float* rgb_dev, int k_max, float merge_dist, void* stream, uint8_t* labels_dev,
                float* b_host, int* k_out, char* errbuf, int errbuf_len);

/* ---- single stages, for kernel-level checks (same kernels as gid_run) ---- */

/* Per-frame precompute outputs: w_SR (H x W), spatial pair weights
 * (n_spatial x H x W) and temporal pair weights (n_temporal x H x W; zeros if
 * the temporal pairs are inactive for this frame).  NULL pointers skip. Async. */
int gid_stage_precompute(gid_ctx* ctx, float* wsr_dev, float* omega_s_dev, float* omega_t_dev);

/* Normal equations at the current state X: g_dev = -J^T F and diag_dev =
 * diag(J^T J), each (K+4) x H x W.  Does not change X.  Async. */
int gid_stage_linearize(gid_ctx* ctx, float* g_dev, float* diag_dev);

/* q_dev = J^T J p_dev at the current state (both (K+4) x H x W).  Async. */
int gid_stage_apply(gid_ctx* ctx, const float* p_dev, float* q_dev);

/* delta_dev = the Gauss-Newton update after exactly m_inner PCG steps at the
 * current state, without applying it.  Async. */
int gid_stage_pcg(gid_ctx* ctx, int m_inner, float* delta_dev);

/* Base-colour normal equations at the current state: A_host (3 x K x K) and
 * g_host (3 x K), one K x K block per channel (eq:basecolorrefinement).
 * Synchronises. */
int gid_stage_dense_normal(gid_ctx* ctx, double* A_host, double* g_host);

/* ---- operator tile shape ---- */

/* How the PCG loop of each Gauss-Newton step (Sec. 6.1) runs.  rows = 2, 4, 8,
 * 16 or 17: one operator kernel and one vector kernel per PCG step, operator
 * tiles of 128 x rows pixels (17 runs one 544-thread block per SM at up to 96
 * registers a thread, 16 one 512-thread block at up to 128).  A new context
 * starts with 17 if the frame's 128 x 17 tiles fit in one wave (at most one
 * per SM), else 4.
 * rows = 0: all PCG steps of a Gauss-Newton step in one cooperative launch
 * (one block per SM streaming every vector, operator and vector phases
 * separated by grid barriers whose waits are bounded; a barrier that gives up
 * is reported as GID_ERR_TIMEOUT by the next synchronising call).
 * rows = GID_PCG_RESIDENT: one cooperative launch as well, in which each block
 * owns one tile of the frame for the whole Gauss-Newton step and keeps that
 * tile's z (with the stencil's halo) and p in shared memory; only q, delta,
 * M^-1 and the operator coefficients stream through L2, and neighbouring
 * tiles exchange the border rows and columns of z through a global buffer
 * after every vector phase.  It needs the whole frame's tiles co-resident (one
 * block per SM), so it exists only for frames up to a few hundred thousand
 * pixels (640 x 480 at K = 6 is 148 tiles of 160 x 13 on 148 SMs); the first
 * selection allocates its exchange buffers (V planes + 12 KB) and synchronises.
 * rows = 2, 4, 8 or 17 | GID_PCG_FUSED: one kernel per PCG step whose
 * operator tile also does the previous step's vector update (for the tile and
 * the stencil's halo, so each block computes its halo's z itself); z and M^-1 q
 * alternate between two buffers by step parity, and the PCG scalars come from
 * one set of block partials per step (<p, q>, <z, q>, <q, M^-1 q>: rho of the
 * next step by the expanded recurrence instead of a second reduction).  Fewer
 * bytes per step than the two-kernel loop (no separate pass over the PCG
 * vectors); the first selection allocates 2 V planes and synchronises.
 * Jacobi preconditioner only for the single-launch and fused loops
 * (GID_PRECOND_BLOCK keeps the two-kernel loop).
 * GID_ERR_INVALID_ARG if the device cannot co-schedule the chosen loop or the
 * frame does not fit; GID_ERR_OOM if a loop's buffers cannot be allocated.
 * Results agree to FP32 rounding order; only speed differs. */
#define GID_PCG_RESIDENT (-1)
#define GID_PCG_FUSED 256
int gid_set_apply_tile(gid_ctx* ctx, int rows);

/* on != 0: the PCG launches (operator, vector and fused steps) carry an L2
 * access-policy window over the operator coefficient planes (NC planes, written
 * once per Gauss-Newton step and read by every PCG step of it) and as many of
 * the PCG vectors q, p and z (in that order) as fit with them: accesses to them
 * are marked persisting, up to the device's persisting-L2 limit, which the
 * first context to turn this on raises to the window's size (capped by the
 * device maximum) for this process; the set-aside is released when the last
 * context turns it off or is destroyed; while it is held, the rest of the L2
 * is all that other work on the device (other contexts, batches) can use.  Only
 * speed changes.  Synchronises and drops the context's cached graphs.
 * GID_ERR_INVALID_ARG if the device has no persisting L2 or the coefficient
 * planes alone do not fit in its maximum
 * set-aside (a partial window thrashes it: 1920 x 1080 K = 8 ran 52 % slower
 * with one).
 * gid_autotune times its chosen loop with and without the window and keeps the
 * faster. */
int gid_set_l2_window(gid_ctx* ctx, int on);

/* 1 if the context's PCG launches carry the L2 window, 0 if not, -1 for NULL. */
int gid_get_l2_window(const gid_ctx* ctx);

/* The context's PCG loop (*rows as passed to gid_set_apply_tile) and the tile
 * geometry the resident loop has, or would have, on this frame: tile_w x
 * tile_h pixels, `blocks` tiles (0, 0, 0 if it does not fit).  Any pointer may
 * be NULL. */
int gid_get_pcg_layout(gid_ctx* ctx, int* rows, int* tile_w, int* tile_h, int* blocks);

/* ---- PCG history ---- */

/* Recording of the PCG history, off by default: when on, each PCG step's rho
 * is copied into a device-side history by one 8-byte device copy after its
 * operator step (the kernels themselves are unchanged, so the default path
 * pays nothing for it).  The persistent PCG kernel (gid_set_apply_tile(0),
 * Jacobi) always records.  Changing it synchronises the context's streams and
 * drops its cached graphs. */
int gid_set_pcg_history(gid_ctx* ctx, int on);

/* rho_m = <r_m, z_m> (residual against preconditioned residual, Sec. 6.1's
 * PCG) of the latest Gauss-Newton step that ran, for m = 0 .. n-1 with
 * n = min(its PCG steps, 64, max_n) written to *n_out (rho_0 at the start;
 * the last step's final rho is not formed); n = 0 if that step did not record.
 * FP64 totals of the same block partials the solver uses for alpha and beta.
 * rho_host: host array of at least max_n doubles.  Synchronises, and reports
 * any error a device step recorded since the last synchronising call. */
int gid_pcg_history(gid_ctx* ctx, double* rho_host, int max_n, int* n_out);

/* ---- fault injection (tests) ---- */

/* Host-side fault injection for failure-detection tests (the paper has no
 * counterpart).  phantom_blocks > 0 adds that many participants that never
 * arrive to every grid barrier of the persistent and resident PCG kernels
 * (gid_set_apply_tile(0) or GID_PCG_RESIDENT), so every block's bounded wait
 * runs out; spin_limit
 * > 0 replaces the barrier's poll limit (default 2^22 polls of about 64 ns),
 * so that the wait gives up after spin_limit polls.  A barrier that gives up
 * records a status bit and its kernel returns without updating the state; the
 * next synchronising call returns GID_ERR_TIMEOUT and clears the bit, and the
 * context stays usable.  gid_debug_inject(ctx, 0, 0) restores the defaults
 * (a new context starts with them).  Negative arguments: GID_ERR_INVALID_ARG.
 * Synchronises. */
int gid_debug_inject(gid_ctx* ctx, int phantom_blocks, long long spin_limit);

/* ---- preconditioner ---- */

/* Sec. 6.1 solves each Gauss-Newton system by preconditioned conjugate
 * gradient without naming the preconditioner.  GID_PRECOND_JACOBI (default):
 * M = diag(J^T J).  GID_PRECOND_BLOCK: M = the per-pixel (K+4) x (K+4) diagonal
 * blocks of J^T J (the unknowns r_R, r_G, r_B, T_0..T_K of one pixel coupled
 * through the data and monochrome terms), factored once per Gauss-Newton step
 * in FP32 per pixel (the reflectance part is diagonal: its Schur complement on
 * the layers is Cholesky-factored; a pixel whose block rounding made
 * indefinite falls back to its diagonal).  The block form stores
 * 6 + (K+1)(K+2)/2 extra planes
 * (allocated on the first switch; GID_ERR_OOM if that fails) and always runs
 * one operator and one vector kernel per PCG step (the persistent loop of
 * gid_set_apply_tile(0) is Jacobi only).  Synchronises the context's streams
 * and drops its cached graphs.  A batch captures its graph on its first run:
 * set the preconditioner of its contexts (gid_batch_ctx) before that. */
#define GID_PRECOND_JACOBI 0
#define GID_PRECOND_BLOCK 1
int gid_set_preconditioner(gid_ctx* ctx, int kind);

/* The context's preconditioner (GID_PRECOND_*), -1 for a NULL ctx. */
int gid_get_preconditioner(const gid_ctx* ctx);

/* Time reps PCG steps with each of the eleven ways above on the current frame
 * and state (CUDA events on the context stream) and keep the fastest.  Writes
 * the chosen rows (0 = persistent, GID_PCG_RESIDENT, rows | GID_PCG_FUSED) to
 * *rows_out and the eleven timings (us per PCG step; shapes 2, 4, 8, 17,
 * persistent, resident, fused 2, 4, 8, 17, shape 16; -1 if unavailable) to
 * us_out[GID_AUTOTUNE_TIMINGS]; either may be NULL.  The single-launch and
 * fused loops are timed as the difference of two Gauss-Newton steps (reps + 2
 * and 2 PCG steps), so that the linearisation does not count.  Where the
 * operator coefficients fit in the persisting L2 set-aside, the chosen loop is
 * then timed that way with and without gid_set_l2_window and the faster kept.  Needs gid_set_frame and a state; leaves the state X
 * unchanged (the PCG vectors are scratch until the next gid_run).  Call it
 * between runs.  Synchronises. */
#define GID_AUTOTUNE_TIMINGS 11
int gid_autotune(gid_ctx* ctx, int reps, int* rows_out, float* us_out);

/* ---- batches of videos (many videos of uneven size, one graph per step) ---- */

typedef struct gid_batch gid_batch;

/* n videos, video i of H[i] x W[i] with K[i] base colours.  w points to one
 * gid_weights for all (per_video = 0) or to n of them (per_video = 1); NULL for
 * the defaults.  Each video gets its own context and CUDA stream; stream is
 * the caller's stream the batch calls are ordered with (NULL: legacy default). */
int gid_batch_create(int n, const int* H, const int* W, const int* K, const gid_weights* w, int per_video,
                     void* stream, gid_batch** out);
void gid_batch_destroy(gid_batch* batch);
const char* gid_batch_last_error(const gid_batch* batch);

/* Video i's context, for gid_set_base_colors / gid_get_layers / gid_energy...
 * (those calls then run on the video's own stream).  NULL if i is out of range. */
gid_ctx* gid_batch_ctx(gid_batch* batch, int i);

/* gid_set_frame / gid_init / gid_new_sequence for every video (arrays of n
 * device pointers, as gid_set_frame). */
int gid_batch_set_frames(gid_batch* batch, const float* const* rgb_dev, const uint8_t* const* labels_dev);
int gid_batch_init(gid_batch* batch, int mode);
int gid_batch_new_sequence(gid_batch* batch);

/* gid_run(n_outer, m_inner) for every video as ONE CUDA graph launch
 * (recorded once per configuration).  Work-list form (the default, when every
 * video uses the Jacobi preconditioner): per Gauss-Newton step each video
 * linearises on its own stream, then each of the M PCG steps (Sec. 6.1) is one
 * operator launch and one vector launch per distinct K covering the tiles and
 * planes of every video with that K (operator tiles of 128 x 4 pixels), then
 * each video takes its base-colour step on its own stream.  Branch form
 * (gid_batch_set_worklist(batch, 0), or any video with the block
 * preconditioner): each video's own multi-kernel launch sequence (tile rows
 * 2, 4, 8 or 17, as gid_set_apply_tile / gid_batch_autotune chose) is a branch
 * of the graph.  Per video the two forms compute the same arithmetic except
 * for the grouping of FP32 partial sums in the PCG reductions (tile shape and
 * vector-block count), so their results agree to rounding, not bit for bit.
 * Asynchronous. */
int gid_batch_run(gid_batch* batch, int n_outer, int m_inner);

/* on = 1: the work-list form of gid_batch_run (default); 2: the work list as
 * one cooperative launch per K group and Gauss-Newton step (all M PCG steps,
 * operator and vector phases separated by bounded grid barriers; the launch
 * fails with GID_ERR_CUDA where the device cannot co-schedule it); 0: the
 * branch form.  Takes effect at the next gid_batch_run (graphs of every form
 * are kept).  GID_ERR_INVALID_ARG for a NULL batch. */
int gid_batch_set_worklist(gid_batch* batch, int on);

/* Choose every video's operator tile shape for the branch form: from the
 * cache file (lines "H W K rows") if it lists the video's shape, else by
 * gid_autotune(reps) on the video's current frame and state (the fastest
 * multi-launch loop: a tile shape of the two-kernel loop or of the fused step;
 * batches do not run the single-launch loops), then
 * append the new shapes to the file (cache_path may be NULL: no cache).  The
 * work-list form always uses 4-row tiles.  Needs frames and states.
 * Synchronises. */
int gid_batch_autotune(gid_batch* batch, const char* cache_path, int reps);

/* ---- learned initial state (BF16 encoder-decoder) ---- */

/* The paper has no network; Sec. 8 names learned priors as future work.  This
 * one predicts the initial state of a frame's solve so that fewer Gauss-Newton
 * steps reach a given energy.  Architecture (widths w1..w4, default 32, 64, 96,
 * 128): input 16 channels (the frame I in 0..2, R_cluster = b_init[label] in
 * 3..5, the cold-start shading estimate mean_c I / mean_c R_cluster in 6, the
 * one-hot label in 7..7+K-1, zeros); encoder levels 1..4, each two 3x3 convolutions with ReLU, a 2x2
 * average pool before levels 2..4; decoder levels 3, 2, 1, each a nearest 2x
 * upsampling of the level below concatenated (first) with the encoder output
 * of the level, then two 3x3 convolutions with ReLU; a 1x1 head to 2K + 1
 * channels: K logits w, T_0, T_1..T_K.  Outputs r = ln sum_k softmax(w)_k b_k
 * (the frame's K x 3 palette b, index-aligned with the solver's base colours)
 * and T = softplus(T_0..T_K) = ln(1 + exp(.)) (non-negative layers).  Loss: mean squared error of r over B x 3 x H x W values plus that of
 * T over B x (K+1) x H x W values.  Weights: FP32 masters, BF16 copies for the
 * tensor-core convolutions (FP32 accumulation), BF16 activations.
 * Weight blob (host float32, gid_net_num_params values): per layer in the
 * order e1a e1b e2a e2b e3a e3b e4a e4b d3a d3b d2a d2b d1a d1b head, the
 * weights as (C_out, C_in, k, k) then the biases (C_out). */
typedef struct gid_net gid_net;

/* Create a network for K base colours (1..9: the input holds 7 + K channels of
 * 16); widths: 4 ints, each a
 * multiple of 32 in [32, 256], or NULL for the defaults.  Weights He-normal
 * from seed (splitmix64 + Box-Muller), biases zero.  stream: cudaStream_t or
 * NULL; every call below runs on it.  Synchronises. */
int gid_net_create(int K, const int* widths, uint64_t seed, void* stream, gid_net** out);
void gid_net_destroy(gid_net* net);
const char* gid_net_last_error(const gid_net* net);
long gid_net_num_params(const gid_net* net);
long long gid_net_launch_count(const gid_net* net);

/* Weights (and gradients of the last gid_net_backward) as a blob, host.
 * Setting weights resets the Adam moments.  Synchronise. */
int gid_net_set_weights(gid_net* net, const float* blob_host);
int gid_net_get_weights(gid_net* net, float* blob_host);
int gid_net_get_grads(gid_net* net, float* blob_host);

/* Inference on B frames of H x W (H, W multiples of 8): rgb_dev B x 3 x H x W
 * float32, labels_dev B x H x W uint8 (>= K read as 0), palette_dev B x K x 3
 * float32 (> 0), all device.  Writes r_dev (B x 3 x H x W) and T_dev
 * (B x (K+1) x H x W); either may be NULL.  The activation buffers grow on
 * demand (a device allocation when a larger batch is first seen).  Async. */
int gid_net_forward(gid_net* net, int B, int H, int W, const float* rgb_dev, const uint8_t* labels_dev,
                    const float* palette_dev, float* r_dev, float* T_dev);

/* Forward pass, loss against the targets r_target_dev (B x 3 x H x W) and
 * T_target_dev (B x (K+1) x H x W), and the gradient of the loss with respect
 * to every weight (kept in the network for gid_net_adam_step / get_grads).
 * loss_host: if not NULL, the loss (FP64 sum of FP64 block partials) -- this
 * synchronises; NULL keeps the call asynchronous. */
int gid_net_backward(gid_net* net, int B, int H, int W, const float* rgb_dev, const uint8_t* labels_dev,
                     const float* palette_dev, const float* r_target_dev, const float* T_target_dev,
                     double* loss_host);

/* Weights of the loss's three parts: the r error, the T_0 error and the
 * T_1..T_K error (each a mean over its values as above); default 1, 1, 1.
 * Finite and >= 0, else GID_ERR_INVALID_ARG. */
int gid_net_set_loss_weights(gid_net* net, float w_r, float w_T0, float w_Tk);

/* One Adam step (Kingma and Ba 2015, bias-corrected) on the FP32 masters with
 * the last gradients; repacks the BF16 copies.  Async. */
int gid_net_adam_step(gid_net* net, float lr, float beta1, float beta2, float eps);

/* Learned initial state for the context's current frame: the network's r and
 * T (palette = the initial base colours) become the state, indirect values
 * T_1..T_K below zero_below (>= 0) written as exactly 0 (the i-sparsity
 * prior's default; the IRLS weights of Sec. 5.3 hold exact zeros, while a
 * strictly positive value has non-negativity weight 0 and can overshoot
 * below zero in the next Gauss-Newton step), T_0 refit per
 * pixel to the data term (eq:data-term; closed form, clipped at 0) with R,
 * T_1..T_K and b fixed, then, when base
 * colours are refined, one base-colour step (eq:basecolorrefinement) on those
 * layers.  Needs gid_set_base_colors and gid_set_frame, the same K, and H, W
 * multiples of 8.  Runs on the context stream.  Async. */
int gid_init_learned(gid_ctx* ctx, gid_net* net, float zero_below);

/* ---- misclustering correction (Sec. 4.2) ---- */

/* Reflectance correction of a misclustered region: for every candidate base
 * colour k = 1..K, a full decomposition of the frame (cold start, n_outer x
 * m_inner, refinement per the weights) with the region's pixels labelled k;
 * the K candidates are solved together as one batch (one graph launch per
 * outer step).  Each candidate's i-sparsity energy (eq:shading-sparsity-term)
 * over the region is measured and the sparsest candidate is the region's
 * corrected reflectance (the paper's criterion).  The region itself comes from
 * the user in the paper (clicks, flood fill, tracking); here it is a mask.
 *   rgb_dev       3 x H x W float32 frame; labels_dev H x W uint8 (0..K-1)
 *   b_init_host   K x 3 initial base colours (finite, > 0)
 *   region_dev    H x W uint8, nonzero on the region
 *   best_out      out, the winning label (colour index - 1)
 *   sparsity_out  out, K doubles (i-sparsity over the region per candidate) or NULL
 *   labels_out_dev out, H x W uint8: the labels with the region set to the winner, or NULL
 * Creates and destroys its own K contexts; synchronises.  Errors are reported
 * by gid_last_error(NULL). */
int gid_correct_region(int H, int W, int K, const gid_weights* w, const float* rgb_dev, const uint8_t* labels_dev,
                       const float* b_init_host, const uint8_t* region_dev, int n_outer, int m_inner, void* stream,
                       int* best_out, double* sparsity_out, uint8_t* labels_out_dev);

/* ---- instrumentation ---- */

/* Kernel kinds for gid_profile_read. */
#define GID_KIND_FRAME 0     /* frame ingest + prior weights */
#define GID_KIND_INIT 1      /* cold start */
#define GID_KIND_LINEARIZE 2 /* fused residual / Jacobian / preconditioner / PCG start */
#define GID_KIND_APPLY 3     /* PCG operator step q = J^T J p */
#define GID_KIND_UPDATE 4    /* PCG vector step */
#define GID_KIND_DENSE 5     /* base-colour normal equations + solve */
#define GID_KIND_ENERGY 6
#define GID_KIND_READOUT 7
#define GID_KIND_PCG 8       /* persistent PCG loop (all steps of a Gauss-Newton step) */
#define GID_NUM_KINDS 9

/* Number of kernels this context has launched since gid_create. */
int gid_launch_count(const gid_ctx* ctx, long long* n);

/* enable != 0: record a CUDA event on the context stream before the first and
 * after every later kernel launch (up to 16384 launches between reads); each
 * kernel is timed from the previous kernel's end event to its own, its launch
 * gap included, so the kernels partition the profiled time.  Profiled runs
 * launch kernel by kernel (no graph replay).  0 stops recording. */
int gid_profile(gid_ctx* ctx, int enable);

/* Synchronise and return, per kind, the summed device time (ms[GID_NUM_KINDS])
 * and launch count (count[GID_NUM_KINDS]) recorded since the previous read. */
int gid_profile_read(gid_ctx* ctx, double* ms, long long* count);

/* ---- base-colour step without device allocation ---- */

/* Bytes of the file-scope device array that gid_dense_refine_noalloc uses as
 * scratch.  Every GPU that loads the library holds this much until exit. */
#define GID_NOALLOC_SCRATCH_BYTES (512 * 1024)

/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory (code living inside another framework's memory pool,
 * real-time loops that must not block on the allocator, processes that are only
 * handed device pointers).  It computes the same base-colour step as gid_run's
 * dense stage -- the three K x K normal equations of eq:basecolorrefinement at
 * the layers X and their FP64 Cholesky solve -- without a context and without
 * any cudaMalloc / cudaFree: its scratch is a static device array of
 * GID_NOALLOC_SCRATCH_BYTES, enough for every K <= GID_MAX_K and every frame up
 * to 2^28 pixels (the reduction uses at most 296 x 3 blocks).
 *   X_dev       (K+4) x H x W float32 unknowns (r_R, r_G, r_B, T_0..T_K), device
 *   rgb_dev     3 x H x W float32 frame, device
 *   b_init_host K x 3 initial base colours (finite, > 0), host
 *   w           weights; lambda_data, lambda_IR and lambda_CR are used
 *   stream      cudaStream_t or NULL
 *   A_dev       out, 3 x K x K doubles (device) or NULL
 *   g_dev       out, 3 x K doubles (device) or NULL
 *   b_dev       out, K x 3 floats, refined colours b_init + Delta b (device) or NULL
 *   errbuf      optional caller buffer of errbuf_len bytes for an error message
 * Returns GID_ERR_INVALID_ARG for a NULL input, K outside 1..GID_MAX_K or a
 * frame beyond 2^28 pixels, GID_ERR_NUMERIC if a channel's K x K block is not
 * positive definite (each colour channel is solved on its own: the channels
 * whose block failed keep b_init in b_dev, the others are refined),
 * GID_ERR_CUDA on a runtime error.  Copies the small results with ordinary
 * asynchronous copies and synchronises the stream before returning, so it
 * cannot be called while the stream is being captured into a CUDA graph.  The
 * first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process: after cudaDeviceReset the call must not be used again in that
 * process.  All calls on a device share the one array and it keeps the last
 * call's contents (the call clears what must start at zero itself): calls that
 * overlap on the GPU, from several streams or threads, race and must be
 * serialised by the caller. */
int gid_dense_refine_noalloc(int H, int W, int K, const float* X_dev, const float* rgb_dev,
                             const float* b_init_host, const gid_weights* w, void* stream, double* A_dev,
                             double* g_dev, float* b_dev, char* errbuf, int errbuf_len);

#ifdef __cplusplus
}
#endif
#endif /* GID_H */
