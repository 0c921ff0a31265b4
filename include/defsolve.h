/*
 * defsolve — per-frame non-rigid surface deformation solve on one GB300 (sm_103a).
 *
 * C ABI of the library libdefsolve.so. The operation is the deformation recovery of
 * Zhou & Jagadeesan, "Real-time Surface Deformation Recovery from Stereo Videos":
 *   - a depth template is deformed by sparse control points, each carrying a rigid warp W_i
 *     (Section 2: dual-quaternion warp; a template point moves with a blend of the control
 *     points near it);
 *   - the warps minimise f_ICP + w_ORB f_ORB + w_ARAP f_ARAP (Eq. 1): point-to-plane ICP with
 *     Tukey weights from projective association (Section 2), feature matches weighted by
 *     1-point RANSAC + reweighting (Section 2.1, Eq. 2-4) and dense all-pairs ARAP
 *     (Section 2.2, Eq. 5-6);
 *   - by damped Gauss-Newton over every control point's rotation and translation, solving the
 *     normal equations with a Cholesky factorisation (Section 2, LM + Cholesky).
 *
 * Conventions shared by every call:
 *   - Images are row-major H x W, pixel (u, v) at index v * W + u, pixel centres at integer
 *     coordinates. Camera frame x right, y down, z forward; units are millimetres.
 *   - Input pointers may be host (pageable or pinned) or device pointers; the library copies
 *     them with cudaMemcpyAsync(cudaMemcpyDefault) on the handle's stream. Pageable host input
 *     is copied before the call returns; pinned host or device input must stay valid and
 *     unchanged until the handle's stream reaches the copy (any ds_get_* call, or a stream
 *     synchronisation, guarantees that).
 *   - Output pointers are caller-allocated host or device memory; every ds_get_* call
 *     synchronises the handle's stream before it returns.
 *   - The handle owns all of its device memory; calls on one handle must not run
 *     concurrently from several host threads. Distinct handles are independent.
 *   - Every call returns a ds_status; nothing aborts the process. A CUDA error is returned as
 *     DS_ERR_CUDA and leaves the handle usable only for ds_destroy.
 */
#ifndef DEFSOLVE_H
#define DEFSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DS_OK = 0,
  DS_ERR_ARG = 1,       /* a null pointer, a size out of range, an index outside the image  */
  DS_ERR_OOM = 2,       /* a device allocation failed                                       */
  DS_ERR_BAD_INPUT = 3, /* non-finite depth or match coordinates                             */
  DS_ERR_NOT_SPD = 4,   /* a Cholesky pivot <= 0 (or NaN); it was replaced by 1 so that the
                           iteration stays finite, and the frame's result is not reliable     */
  DS_ERR_STATE = 5,     /* call order violated (e.g. solve before submit_frame)              */
  DS_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up                                */
  DS_ERR_CUDA = 7       /* any other CUDA runtime error                                      */
} ds_status;

/* Precision of the normal-equation solve. Residuals, Jacobians and J^T W J are FP32 in every
 * mode; the state is kept in FP64. */
typedef enum {
  DS_PREC_FP64 = 0,        /* FP64 Cholesky + FP64 triangular solves + refinement steps whose
                              residual b - A x against the FP32 matrix is accumulated in
                              double-float FP32 arithmetic (FMA-exact products, two-sum
                              accumulation: ~48 significant bits) and subtracted from b in FP64 */
  DS_PREC_FP32 = 1,        /* plain: FP32 Cholesky and solves, no refinement                   */
  DS_PREC_FP32_REFINE = 2  /* FP32 Cholesky and solves + the same refinement steps            */
} ds_precision;

#define DS_MAX_ITERS 64
#define DS_MAX_HYP 64
#define DS_FACTOR_AUTO (-1)   /* ds_params.factor_tc: the factor kernel is tuned per batch */

typedef struct ds_ctx* ds_handle;

typedef struct {
  float fx, fy, cx, cy; /* pinhole intrinsics, shared by the template and every frame */
} ds_intrinsics;

/* Method parameters. ds_default_params() fills the paper's values where it gives them
 * (w_orb = 10 after Eq. 1; w_angle = 20 and w_rot = 100 after Eq. 5; 10 reweighting iterations
 * and 30 references in Section 2.1) and the library's readings elsewhere. */
typedef struct {
  double w_orb;             /* weight of f_ORB in Eq. 1                                          */
  double w_angle;           /* weight of f_angle in Eq. 5                                        */
  double w_rot;             /* weight of f_rotation in Eq. 5                                     */
  double w_arap0;           /* w_ARAP = w_arap0 * (sum ICP weights + w_orb * sum ORB weights) / N */
  double H_mm;              /* threshold H of Eq. 4 (also the 5H ramp of the ORB weights)        */
  double tukey_c_mm;        /* Tukey constant of the ICP term                                    */
  double sigma_blend_scale; /* blend sigma = scale * mean nearest-neighbour node spacing         */
  double sigma_arap_scale;  /* ARAP pair sigma = scale * node bounding-box diagonal              */
  double lambda;            /* damping: A + lambda (diag(A) + eps_damp)                          */
  double eps_damp;
  double keep_frac;         /* a RANSAC reference is kept iff its score >= keep_frac * best      */
  int32_t n_hyp;            /* number of RANSAC references (<= DS_MAX_HYP)                       */
  int32_t n_reweight;       /* reweighting iterations per reference                              */
  int32_t n_nearest;        /* control points blended per template point; must be 4             */
  int32_t precision;        /* ds_precision                                                      */
  int32_t refine_steps;     /* refinement steps in DS_PREC_FP64 / DS_PREC_FP32_REFINE (0..3)     */
  int32_t use_graph;        /* 1: replay the GN loop as a CUDA graph (default), 0: plain launches */
  int32_t factor_tc;        /* FP32 precisions, the factorisation kernel: 0 = FP32 SIMT pipes, 64 x 64
                             * tiles; on the tensor cores (tcgen05 kind::tf32, each product as
                             * three TF32 terms hi*hi + hi*lo + lo*hi, FP32-level accuracy) with
                             * 1 = 64 x 64 tiles, 2 = 128 x 128 blocks, 3 = 128 x 128 blocks with
                             * two rows x two block columns per task (each operand block streamed
                             * once per two products, four accumulators), 4 = 128 x 128 blocks
                             * with the block columns taken in pairs (each row panel streamed once
                             * per two block columns, two accumulators), 5 = 128 x 128 blocks with
                             * each task's K loop (one streaming warp, two tensor-memory
                             * accumulators) overlapping the previous task's epilogue;
                             * DS_FACTOR_AUTO (default) = picked per batch by timing the six on
                             * the batch's sizes at its first solve (ds_batch_tune). Ignored in
                             * DS_PREC_FP64. Handles of one batch must agree.                     */
  int32_t solver;           /* 0 = one Cholesky of the dense 6N x 6N damped system (default);
                             * 1 = block-Jacobi: each control point's 6 unknowns from its own 6 x 6
                             * damped diagonal block (FP64 Cholesky per node), the reading of
                             * Section 2's separate update of every W_i; no factorisation of
                             * the coupled system and no refinement. Handles of one batch agree.  */
  int32_t assoc;            /* ICP association (Section 2, projective "rasterization"):
                             * 0 = nearest pixel, floor(u + 1/2) (default);
                             * 1 = bilinear: target point and normal blended from the usable
                             * pixels among the 4 around the projection (weights (1-a)(1-b),
                             * a(1-b), (1-a)b, ab with a, b the fractional parts, renormalised over
                             * the usable ones), normal renormalised; valid iff the usable weight
                             * is >= 1/2. The Jacobian holds the blended point and normal fixed, as
                             * with the nearest pixel.                                            */
  int32_t jtj;              /* Precision of the ICP term's J^T W J (Section 2, ICP paragraph):
                             * 0 = FP32 on the SIMT pipes (default);
                             * 1 = BF16 Jacobian rows on the tensor cores with FP32 accumulation
                             * (warp-level mma, 16 points per product). The gradient J^T W r stays
                             * FP32 in both, so the Gauss-Newton fixed point is the same; the step
                             * of an iteration differs by the rounding of the Jacobian to BF16.
                             * Handles of one batch must agree.                                   */
  int32_t ransac_o1;        /* o1 of Eq. 2 (the template side of each match) in the RANSAC:
                             * 0 = the template point at the matched pixel (default);
                             * 1 = warm start: that point warped by the handle's current warps
                             * (the state the frame's solve starts from), in FP64, so the rigid
                             * model only has to explain the motion since the previous frame.     */
} ds_params;

/* Per-solve statistics (filled by ds_solve when its `out` is not NULL). */
typedef struct {
  int32_t iters;                  /* iterations run                                          */
  int32_t n_inliers;              /* preselected matches                                     */
  int32_t n_kept;                 /* kept RANSAC references                                  */
  int32_t n_icp_valid_last;       /* valid ICP associations at the last linearisation        */
  double w_arap;                  /* the frame's w_ARAP                                       */
  double cost[DS_MAX_ITERS];      /* Eq. 1 at each linearisation point                        */
  double cost_icp[DS_MAX_ITERS];
  double cost_orb[DS_MAX_ITERS];
  double cost_arap[DS_MAX_ITERS];
} ds_solve_stats;

/* Fills *p with the defaults listed above. */
void ds_default_params(ds_params* p);

/* Creates a handle from a template depth map (Section 2: the template is generated from the
 * first frame). depth_hw: H x W FP32 depths in mm, <= 0 = no surface (NaN / inf are rejected).
 * W, H in [8, 4096]. p may be NULL (defaults). cuda_stream: the cudaStream_t to run on, or
 * NULL for a stream owned by the handle. On success *out receives the handle.
 * Errors: DS_ERR_ARG, DS_ERR_BAD_INPUT (NaN/inf depth), DS_ERR_OOM, DS_ERR_CUDA. */
int ds_create_template(const float* depth_hw, int32_t W, int32_t H, ds_intrinsics K,
                       const ds_params* p, void* cuda_stream, ds_handle* out);

/* Places N control points at template pixels pixel_index[0..N) (Section 2: sparse control
 * points on the template); g_i is the template point at that pixel. Builds the blend tables
 * (4 nearest control points by 3D distance, Gaussian weights) and resets every warp to the
 * identity. N in [5, 2048]; every index must be a distinct valid template pixel.
 * Errors: DS_ERR_ARG, DS_ERR_OOM, DS_ERR_CUDA. */
int ds_set_control_points(ds_handle h, const int32_t* pixel_index, int32_t N);

/* Submits one live frame: depth_hw (H x W FP32, same size as the template; <= 0 = no data),
 * M feature matches (match_tmpl_idx[k] = template pixel of match k, match_xyz[3k..3k+2] = its
 * live 3D point), and hyp_list[0..n_hyp) = the reference match ids of the 1-point RANSAC
 * (Section 2.1). Runs the frame preparation (live points and normals) and the RANSAC
 * preselection on the handle's stream. M in [0, 65536]; with M == 0 hyp_list may be NULL.
 * Host-memory indices are checked before the call returns. Device-memory indices are checked
 * on the device without a host synchronisation: an out-of-range template pixel (or one without
 * a template point) is replaced by the first valid template pixel and an out-of-range reference
 * id by 0 before any kernel reads them, and the next synchronising call (ds_solve with
 * stats, any ds_get_*) returns DS_ERR_ARG. Non-finite depth or match coordinates are reported
 * the same way as DS_ERR_BAD_INPUT.
 * A handle keeps two frame slots: a frame goes to the slot the last solve did not read, so it
 * may be submitted while that solve (e.g. a batch on another stream) still runs; it waits only
 * for the solve that last read its slot (and, with ransac_o1 = 1, for the last solve, whose
 * state it warps). A solve uses the latest submitted frame.
 * Errors: DS_ERR_ARG, DS_ERR_BAD_INPUT, DS_ERR_STATE (no control points), DS_ERR_CUDA. */
int ds_submit_frame(ds_handle h, const float* depth_hw, const int32_t* match_tmpl_idx,
                    const float* match_xyz, int32_t M, const int32_t* hyp_list);

/* Runs `iters` damped Gauss-Newton iterations (1..DS_MAX_ITERS) of Eq. 1 on the submitted
 * frame, starting from the current warps (warm start). Asynchronous unless `out` is not NULL,
 * in which case the stream is synchronised and *out filled.
 * Errors: DS_ERR_ARG (also a bad device-side index of the frame), DS_ERR_STATE (no frame),
 * DS_ERR_BAD_INPUT (non-finite frame data), DS_ERR_NOT_SPD, DS_ERR_TIMEOUT, DS_ERR_CUDA; the
 * errors found on the device are returned by the synchronising calls. */
int ds_solve(ds_handle h, int32_t iters, ds_solve_stats* out);

/* Batched solves of uneven problems. A batch groups n handles (same precision and refinement
 * steps, control points set) and runs the Gauss-Newton iterations of all of them together:
 * every kernel launch of an iteration covers the work lists of all problems (ICP tiles, ORB
 * matches, ARAP rows, factorisation tile tasks, solve tiles), and the iterations are captured
 * once as a CUDA graph per iteration count. Handles keep their own stream for submit_frame and
 * ds_get_*; the batch orders its work after the handles' pending work and their earlier solves;
 * a handle's later calls that read or change its solve state (ds_get_*, ds_set_deformation,
 * ds_linearize, ds_set_control_points, ds_destroy) wait for its last solve, and its later
 * submissions only for the solve that read the frame slot they reuse. A handle may belong to
 * several batches, once in each. A batch's work tables are built from its handles' control
 * points: once a handle gets new control points (ds_set_control_points) or is destroyed, every
 * batch listing it refuses to solve (DS_ERR_STATE) and is only good for ds_batch_destroy;
 * batches and handles may be destroyed in either order. cuda_stream: stream of the batch or NULL
 * (owned). Errors: DS_ERR_ARG (empty, mixed precision, a handle without control points, a handle
 * listed twice), DS_ERR_OOM. */
typedef struct ds_batch_s* ds_batch;
int ds_batch_create(const ds_handle* hs, int32_t n, void* cuda_stream, ds_batch* out);
/* Runs `iters` iterations (1..DS_MAX_ITERS) on every handle of the batch; each handle must have
 * a submitted frame (else DS_ERR_STATE, also for a stale batch). Asynchronous; results are read
 * per handle (ds_get_*), and
 * ds_batch_status synchronises the batch and reports DS_ERR_TIMEOUT / DS_ERR_NOT_SPD. */
int ds_batch_solve(ds_batch b, int32_t iters);
/* As ds_batch_solve, on the handles p with active[p] != 0 only (active: n host bytes in the
 * batch's handle order; at least one set; each active handle must have a submitted frame). The
 * launches still cover the whole batch (the same captured graph is replayed for every mask);
 * the left-out handles' work items return at once and nothing of theirs is read or written, so
 * a long-lived batch serves any subset of its handles without new allocations or captures.
 * Two batches listing the same handles may have solves in flight together only when their
 * active sets are disjoint (a continuous-batching server keeps two such batches). A batch of
 * DS_FACTOR_AUTO handles tunes on its first solve's active set. Errors as ds_batch_solve, and
 * DS_ERR_ARG for a NULL or all-zero mask. */
int ds_batch_solve_masked(ds_batch b, const uint8_t* active, int32_t iters);
int ds_batch_status(ds_batch b);
int ds_batch_destroy(ds_batch b);
/* Phase tracing of a batch, as ds_set_tracing / ds_get_phase_times for a handle (summed over
 * the last ds_batch_solve's iterations; the phases cover all problems of the batch). */
int ds_batch_set_tracing(ds_batch b, int32_t on);
int ds_batch_phase_times(ds_batch b, double* ms4);
/* Graph replay of a batch: 1 (default when every handle's use_graph is set) captures the
 * Gauss-Newton loop into a CUDA graph on the first ds_batch_solve and replays it; 0 launches the
 * kernels directly (no capture cost, for batch compositions used once). DS_ERR_ARG on NULL. */
int ds_batch_set_graph(ds_batch b, int32_t on);

/* Factor-kernel tuner. Times the FP32 factorisation kernels on synthetic SPD systems of the
 * batch's problem sizes, written into the handles' factor buffers (no allocation; a later solve
 * assembles its own systems over them), `reps` launches each (1..100), and makes the fastest the
 * batch's kernel for its later solves, whatever factor_tc its handles carry. Kernel index =
 * the factor_tc value that selects it (0..5). *choice (may be NULL) receives the index (-1 for FP64 or
 * block-Jacobi batches, which have one kernel only), ms6 (may be NULL) the six kernels' best
 * times in ms. The choice is also cached for the process by batch shape (largest system, summed
 * n^3), where batches of DS_FACTOR_AUTO handles look it up at their first solve; without an entry
 * they tune themselves then (2 launches per kernel). Synchronises the batch stream; make the
 * first solve of an auto batch outside any stream capture. Errors: DS_ERR_ARG, DS_ERR_STATE
 * (stale batch), DS_ERR_TIMEOUT, DS_ERR_CUDA. */
int ds_batch_tune(ds_batch b, int32_t reps, int32_t* choice, double* ms6);
/* The batch's factor kernel index now and the tuner's last times (ms6[k] = -1: not timed). */
int ds_batch_factor_kernel(ds_batch b, int32_t* choice, double* ms6);

/* Convenience: a temporary batch over n handles, solved and synchronised. */
int ds_solve_batch(ds_handle* hs, int32_t n, int32_t iters);

/* Copies the current warps out: q_N4 (w, x, y, z per node), t_N3, and the control-point
 * positions p_i = W_i(g_i) = g_i + t_i (Eq. 6 notation) into pos_N3. Any pointer may be NULL. */
int ds_get_deformation(ds_handle h, float* q_N4, float* t_N3, float* pos_N3);

/* FP64 copy of the warps (q_N4, t_N3); either may be NULL. */
int ds_get_deformation64(ds_handle h, double* q_N4, double* t_N3);

/* Overwrites the warps (resume / warm start from a saved state). q rows are normalised. */
int ds_set_deformation(ds_handle h, const float* q_N4, const float* t_N3);

/* RANSAC results of the last submitted frame: bits[ceil(M/32)] preselection mask (bit k of
 * word k/32), w_M[M] match weights (max over kept references), kept_bits (bit h = reference h
 * kept), score_nh[n_hyp] (sum of weights of each reference). Any pointer may be NULL. */
int ds_get_inlier_mask(ds_handle h, uint32_t* bits);
int ds_get_ransac(ds_handle h, float* w_M, uint32_t* kept_bits, double* score_nh);

/* Eq. 1 cost at the last linearisation point of the last solve. */
int ds_get_cost(ds_handle h, double* F);

/* Inspection of intermediate results, for tests and tracing. */
/* Blend table in template pixel order for the P valid template pixels (ascending pixel index):
 * pix_P, node ids nid_P4 (nearest first) and weights alpha_P4. Any pointer may be NULL.
 * *P_out receives P. */
int ds_get_blend_table(ds_handle h, int32_t* P_out, int32_t* pix_P, int32_t* nid_P4,
                       float* alpha_P4);
/* Live points (x, y, z, valid) and normals (nx, ny, nz, 0) of the last frame, H*W*4 floats. */
int ds_get_frame_points(ds_handle h, float* pts4, float* nrm4);
/* Linearises Eq. 1 at the current warps without stepping: the undamped normal equations
 * A_nn (full symmetric, n = 6N, row-major), b_n = -J^T W r, and cost3 = {ICP, ORB, ARAP}.
 * If w_arap_in > 0 it is used as w_ARAP; otherwise the per-frame rule sets it from this state.
 * *w_arap_out (may be NULL) receives the w_ARAP used. */
int ds_linearize(ds_handle h, double w_arap_in, double* A_nn, double* b_n, double* cost3,
                 double* w_arap_out);

/* Tracing. When on (set before the next ds_solve), the solve records CUDA events on the handle's
 * stream around each phase of every iteration (inside the captured graph). ds_get_phase_times
 * synchronises and returns the summed milliseconds of the last solve per phase:
 * ms4[0] linearisation (ICP, ORB, dense ARAP and assembly), ms4[1] Cholesky factorisation,
 * ms4[2] triangular solves and refinement, ms4[3] state update.
 * ds_get_counters returns the number of kernels the handle has launched so far (graph kernel
 * nodes count once per replay); with h == NULL, the number the whole library has launched. */
int ds_set_tracing(ds_handle h, int32_t on);
int ds_get_phase_times(ds_handle h, double* ms4);
int ds_get_counters(ds_handle h, int64_t* kernels_launched);

/* Device bytes the handle holds now: every buffer it has allocated and not yet released (the
 * template, the control-point tables and normal-equation buffers sized at
 * ds_set_control_points, the two frame slots' match and RANSAC buffers sized by the largest M
 * submitted so far). Batches and captured graphs are not included. For admission control by
 * device memory (the serving loop of the paper's real-time setting runs many streams on one
 * GPU). No synchronisation. Errors: DS_ERR_ARG (NULL). */
int ds_get_device_bytes(ds_handle h, int64_t* bytes);

/* The task order of the 128 x 128 block Cholesky factorisation (Section 2: the damped normal
 * equations are solved by a Cholesky factorisation) of an nb x nb block matrix, as the factor
 * kernels claim it within one problem: paired = 0 for the single-block kernels (factor_tc 2 and
 * 5), 1 for the column-pair kernel (factor_tc 4), 2 for the two-row two-column kernel
 * (factor_tc 3). Task k is written to out[3 k .. 3 k + 2] = (type, I, J): type 0 = DIAG(J)
 * (factor block (J, J)), 1 = OFF(I, J) (block (I, J), I > J), 2 = the two blocks (I, J) and
 * (I, J + 1), 3 = the four blocks (I, J), (I, J + 1), (I + 1, J), (I + 1, J + 1). out (host
 * memory, caller-owned) holds cap tasks; the count is written to *ntasks (also when it exceeds
 * cap, then nothing past cap is written). Host only, no GPU. Errors: DS_ERR_ARG (nb < 1, paired
 * not 0..2, ntasks NULL, out NULL with cap > 0). */
int ds_factor_tasks(int32_t nb, int32_t paired, int32_t* out, int32_t cap, int32_t* ntasks);

/* 1-point RANSAC preselection without any allocation, for callers that cannot allocate device
 * memory (for example a host process that runs inside a pre-sized memory pool, or a real-time
 * loop where an allocation can block on a device-wide synchronisation). The paper has no
 * counterpart: it is the same preselection that ds_submit_frame runs, written into
 * caller-provided device buffers.
 * All pointers are device memory owned by the caller: depth0 (H x W template depth), the M match
 * pixels and live points, the n_hyp reference ids; outputs mask_bits[ceil(M/32)], w_M[M],
 * kept_bits[2], score_nh[n_hyp]. Limits: 1 <= M <= DS_NOALLOC_MAX_MATCHES, n_hyp <= DS_MAX_HYP.
 * The working memory is one fixed array compiled into the library (about 1.1 MB, held on every
 * device that loads the library until the process exits). The first call on a device looks up
 * that array's device address and sets the kernel's shared-memory limit there (a failure of
 * either is returned as DS_ERR_CUDA and retried by the next call); make that first call before
 * any stream capture. All calls share
 * the array: calls that overlap on the GPU (other streams, other threads) race and must not be
 * issued. The call runs on cuda_stream (NULL: the legacy default stream) and synchronises it
 * before returning. Errors: DS_ERR_ARG (sizes beyond the limits, a null or host pointer, an
 * out-of-range match pixel or reference id — reported after the run, whose outputs then refer
 * to the index 0 in place of the bad ones), DS_ERR_CUDA. */
#define DS_NOALLOC_MAX_MATCHES 4000
int ds_ransac_noalloc(const float* depth0, int32_t W, int32_t H, ds_intrinsics K,
                      const int32_t* match_tmpl_idx, const float* match_xyz, int32_t M,
                      const int32_t* hyp_list, int32_t n_hyp, int32_t n_reweight, double H_mm,
                      double keep_frac, uint32_t* mask_bits, float* w_M, uint32_t* kept_bits,
                      double* score_nh, void* cuda_stream);

/* Failure-detection self-test of the bounded device-side waits behind every hand-off between
 * CTAs (the factorisation's tile counters and the triangular solves' row flags). One thread
 * waits for a device flag that nothing sets, by acquire polling (kind 0: the waits of the SIMT
 * factorisation and of the solves) or by polling with sleeps (kind 1: the tensor-core
 * factorisation), with a budget of budget_ns (1e3..1e8 ns). With peer_error = 1 the error word
 * is raised before the wait, as when another CTA has already given up, and the wait must end at
 * once. No GPU fault is involved and the context stays usable. Synchronous (a stream of its
 * own). Returns DS_ERR_TIMEOUT when the wait gave up (the designed outcome), DS_OK if it saw
 * the flag, DS_ERR_ARG (kind, budget or peer_error out of range), DS_ERR_OOM, DS_ERR_CUDA.
 * *waited_ms (may be NULL) receives the device time the wait took. */
int ds_selftest_bounded_wait(int32_t kind, int64_t budget_ns, int32_t peer_error,
                             double* waited_ms);

/* Releases everything the handle owns. NULL is accepted. */
int ds_destroy(ds_handle h);

/* Static description of a status code. */
const char* ds_status_str(int status);

/* Library build identification (sm_103a build flags and version). */
const char* ds_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DEFSOLVE_H */
