// C ABI of libdefsolve (declared in include/defsolve.h): handle life cycle, template and
// control-point set-up, frame submission, batched damped Gauss-Newton solves.
//
// Set-up (once per template / control-point set):
//   * the template depth is back-projected in FP64; control points g_i are template points;
//   * the blend table (4 nearest control points, Gaussian weights) is computed on the device;
//   * the host sorts the valid template points by their node quadruple, so that points sharing
//     the same 4 nodes are contiguous ("segments"), enumerates the node pairs that share a point
//     (the block-sparse pattern of the ICP and ORB contributions to A) and lists the tile tasks
//     of the factorisation;
//   * a device descriptor (ProbDesc) gathers every pointer and size the kernels need.
// Per frame: copy-in, device-side index validation, live points and normals, RANSAC, into the
// frame slot (of two per handle) that the last solve did not read.
// Per Gauss-Newton iteration (for every problem of a batch at once): counters reset, ICP, ORB,
// dense ARAP + assembly + damping, persistent Cholesky, persistent solves (+ refinement steps
// with double-float residuals), state update. A single-handle solve is a batch of one. The iterations of a solve are captured
// once as a CUDA graph per batch and iteration count and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "ds_internal.cuh"

using namespace ds;

namespace ds {
thread_local int64_t g_launches = 0;
}

static std::atomic<int64_t> g_total_kernels{0};
void ds::count_kernels(int64_t n) { g_total_kernels += n; }

struct ds_batch_s {
  std::vector<ds_ctx*> hs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool fp64 = false;
  int refine_steps = 0;
  bool block_jacobi = false;   // per-node 6 x 6 solves instead of the dense factorisation
  bool no_graph = false;       // ds_batch_set_graph(b, 0): direct launches
  BatchTabs tabs{};
  const ProbDesc** d_descs = nullptr;
  int2* d_tab = nullptr;   // all work tables, back to back
  int* d_words = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_iters = -1;
  int64_t g_kernels = 0;
  bool tracing = false;
  cudaEvent_t ev[DS_MAX_ITERS][5] = {};
  bool ev_made = false;
  int cur_it = 0;
  int last_iters = 0;
  cudaEvent_t ev_done = nullptr;
  std::vector<cudaEvent_t> ev_in;
  std::vector<const ProbDesc*> h_descs;  // the descriptor table as last uploaded
  // pinned staging of the table's uploads (two, alternating), so that an upload does not make
  // the host wait for the batch stream; each is reused only after its last copy has run
  const ProbDesc** h_tab_pin[2] = {nullptr, nullptr};
  cudaEvent_t ev_tab[2] = {nullptr, nullptr};
  bool tab_pending[2] = {false, false};
  int tab_i = 0;
  // side stream of the linearisation: the ORB pass runs beside the ICP pass (both only add
  // into the block table and the gradient)
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
  bool error = false;
  // a handle's control points changed, or it was destroyed (its entry in hs is then NULL): the
  // work tables and descriptor pointers are the old ones, so the batch no longer runs
  bool stale = false;
  // factor kernel chosen by timing (DS_FACTOR_AUTO handles): tuned once, before the first solve
  bool auto_factor = false;
  bool tuned = false;
  double tune_ms[6] = {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0};
};

struct ds_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int W = 0, H = 0;
  ds_intrinsics K{};
  ds_params prm{};
  // template
  std::vector<float> h_depth0;
  std::vector<double> h_X64;
  std::vector<int> h_pidx;  // valid template pixels, ascending
  float* d_depth0 = nullptr;
  double* d_X64 = nullptr;
  int* d_pidx = nullptr;
  // control points and state
  int N = 0, n = 0;
  std::vector<int> h_nodepix;
  double* d_g64 = nullptr;
  double* d_gc = nullptr;
  double sigma_b = 0, sigma_A = 0;
  double* d_q64 = nullptr;
  double* d_t64 = nullptr;
  NodeGPU* d_node = nullptr;
  PairNode* d_pn = nullptr;
  // sorted template
  int P = 0, S = 0, nbp = 0;
  float4* d_tp = nullptr;
  float4* d_tw = nullptr;
  int* d_rank = nullptr;
  int4* d_seg = nullptr;
  int* d_segbp = nullptr;
  int* d_segstart = nullptr;
  int* d_rowptr = nullptr;
  int* d_rowcol = nullptr;
  int* d_rowbp = nullptr;
  std::vector<int4> h_nid_pix;
  std::vector<float4> h_alpha_pix;
  // frame. Two slots of everything a solve reads from a submitted frame (live points and
  // normals, matches, RANSAC results, the descriptor): a frame is prepared in one slot while a
  // solve may still read the other, so submissions overlap the previous frame's solve.
  float* d_depth = nullptr;
  float4* d_tpts = nullptr;   // 2 slots of W H
  float4* d_tnrm = nullptr;
  int M = 0, M_cap = 0;       // M of the latest frame; slot capacity
  int Ms[2] = {0, 0};         // M per slot
  int fs = 0;                 // slot of the latest submitted frame
  int solved_fs = 0;          // slot the last solve read
  cudaEvent_t ev_slot_free[2] = {nullptr, nullptr};  // after the last solve that read a slot
  bool slot_pending[2] = {false, false};
  int* d_midx = nullptr;      // 2 slots of M_cap
  float* d_mxyz = nullptr;    // 2 slots of 3 M_cap
  int* d_hyp = nullptr;
  bool have_frame = false;
  // ransac
  double* d_rs_scratch = nullptr;
  uint32_t* d_rs_hbits = nullptr;
  float* d_rs_hw = nullptr;
  double* d_rs_score = nullptr;   // 2 slots of DS_MAX_HYP
  uint32_t* d_rs_mask = nullptr;  // 2 slots of ceil(M_cap / 32)
  float* d_rs_what = nullptr;     // 2 slots of M_cap
  double* d_rs_o1 = nullptr;      // warm-start o1 points (M x 3 FP64)
  float* d_rs_o1df = nullptr;     // o1 points as double-float coordinates (M x 6 floats)
  uint32_t* d_rs_kept = nullptr;  // 2 slots of 2
  int* d_rs_counts = nullptr;     // 2 slots of 4
  // linear system
  float* d_A32 = nullptr;     // FP32 system (factor in DS_PREC_FP32, reference otherwise)
  double* d_A64 = nullptr;    // FP64 factor (DS_PREC_FP64)
  float* d_Af32 = nullptr;    // FP32 factor copy (DS_PREC_FP32_REFINE)
  void* d_Dinv = nullptr;
  float* d_blk = nullptr;
  float* d_adiag = nullptr;   // per node ARAP-only diagonal block + gradient (deferred assembly)
  float* d_gdata = nullptr;
  double* d_b = nullptr;
  double* d_x = nullptr;
  double* d_r = nullptr;
  float2* d_xf = nullptr;
  void* d_v2 = nullptr;
  void* d_v3 = nullptr;
  int* d_lcnt = nullptr;      // factorisation task counters
  int* d_lflags = nullptr;    // solve row flags
  void* d_Lp = nullptr;       // packed transposed factor tiles
  int4* d_tasks = nullptr;
  int ntasks = 0;
  int4* d_tasks_b = nullptr;  // 128-block factorisation tasks
  int ntasks_b = 0;
  int4* d_tasks_p = nullptr;  // the same with the block columns in pairs
  int ntasks_p = 0;
  int4* d_tasks_q = nullptr;  // the same with two rows x two block columns per task
  int ntasks_q = 0;
  int nt = 0;
  bool prec_fp64 = false;
  double* d_acc = nullptr;
  double* d_hist = nullptr;   // DS_MAX_ITERS x 6
  int* d_flag = nullptr;
  // descriptor: hdesc holds the fields common to both slots; d_desc[s] is slot s's
  ProbDesc hdesc{};
  ProbDesc* d_desc = nullptr;
  // pinned staging of the two slots' descriptor uploads (a copy from pageable memory would make
  // the host wait for the handle's stream); a slot's staging is reused once its last copy has run
  ProbDesc* h_desc_pin = nullptr;
  cudaEvent_t ev_desc[2] = {nullptr, nullptr};
  bool desc_pending[2] = {false, false};
  // the batch of one used by ds_solve
  ds_batch_s* self = nullptr;
  std::vector<ds_batch_s*> batches;   // every batch that lists this handle (self included)
  bool tracing = false;
  int64_t kernels = 0;
  int last_iters = 0;
  bool error = false;
  // device bytes this handle holds (every buffer it allocated and has not freed), by pointer
  std::unordered_map<const void*, size_t> alloc_bytes;
  size_t device_bytes = 0;
};

namespace {

#define DS_TRY(expr)                                          \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) {                                  \
      if (_e == cudaErrorMemoryAllocation) return DS_ERR_OOM; \
      return DS_ERR_CUDA;                                     \
    }                                                         \
  } while (0)

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DS_ERR_OOM : DS_ERR_CUDA;
  }
  return DS_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Allocation and release of a handle's buffers, counted in the handle's device bytes.
template <typename T>
int halloc(ds_ctx* h, T** p, size_t count) {
  const int rc = dalloc(p, count);
  if (rc == DS_OK) {
    const size_t b = sizeof(T) * (count ? count : 1);
    h->alloc_bytes[(const void*)*p] = b;
    h->device_bytes += b;
  }
  return rc;
}
template <typename T>
void hfree(ds_ctx* h, T*& p) {
  if (p) {
    auto it = h->alloc_bytes.find((const void*)p);
    if (it != h->alloc_bytes.end()) {
      h->device_bytes -= it->second;
      h->alloc_bytes.erase(it);
    }
  }
  dfree(p);
}

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return DS_OK;
  DS_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return DS_OK;
}

size_t npx_of(const ds_ctx* h) { return (size_t)h->W * h->H; }
float4* slot_tpts(ds_ctx* h, int s) { return h->d_tpts + s * npx_of(h); }
float4* slot_tnrm(ds_ctx* h, int s) { return h->d_tnrm + s * npx_of(h); }
int* slot_midx(ds_ctx* h, int s) { return h->d_midx ? h->d_midx + (size_t)s * h->M_cap : nullptr; }
float* slot_mxyz(ds_ctx* h, int s) {
  return h->d_mxyz ? h->d_mxyz + (size_t)s * 3 * h->M_cap : nullptr;
}
uint32_t* slot_mask(ds_ctx* h, int s) {
  return h->d_rs_mask ? h->d_rs_mask + (size_t)s * ((h->M_cap + 31) / 32) : nullptr;
}
float* slot_what(ds_ctx* h, int s) {
  return h->d_rs_what ? h->d_rs_what + (size_t)s * h->M_cap : nullptr;
}
double* slot_score(ds_ctx* h, int s) { return h->d_rs_score + s * DS_MAX_HYP; }
uint32_t* slot_kept(ds_ctx* h, int s) { return h->d_rs_kept + 2 * s; }
int* slot_counts(ds_ctx* h, int s) { return h->d_rs_counts + 4 * s; }

// Slot s's descriptor: the common fields with the slot's frame buffers, uploaded on the handle's
// stream from the slot's pinned staging.
void push_desc(ds_ctx* h, int s) {
  if (h->desc_pending[s]) cudaEventSynchronize(h->ev_desc[s]);
  ProbDesc& D = h->h_desc_pin[s];
  D = h->hdesc;
  D.M = h->Ms[s];
  D.tpts = slot_tpts(h, s);
  D.tnrm = slot_tnrm(h, s);
  D.midx = slot_midx(h, s);
  D.mxyz = slot_mxyz(h, s);
  D.mask = slot_mask(h, s);
  D.what = slot_what(h, s);
  cudaMemcpyAsync(h->d_desc + s, &D, sizeof(ProbDesc), cudaMemcpyHostToDevice, h->stream);
  cudaEventRecord(h->ev_desc[s], h->stream);
  h->desc_pending[s] = true;
}

// Orders the handle's stream after its last solve (a batch on another stream).
void wait_solved(ds_ctx* h) {
  if (h->slot_pending[h->solved_fs])
    cudaStreamWaitEvent(h->stream, h->ev_slot_free[h->solved_fs], 0);
}

void destroy_batch(ds_batch_s* b);

// The factor kernels the tuner chooses from, by kernel index: SIMT 64 x 64 tiles, tensor cores
// with 64 x 64 tiles, tensor cores with 128 x 128 blocks (64 KB K-loop stages); 3 the 128-block
// kernel with the block columns taken in pairs and the rows below each pair also in pairs (two
// rows x two columns per task: each operand block streamed once per two products); 4 with the
// block columns in pairs only; 5 the 128-block kernel whose K loops (one streaming warp, two
// tensor-memory accumulators) overlap the epilogues of the previous tasks (eight warps).
constexpr int kFactorKernels = 6;
void set_factor_kernel(BatchTabs& T, int k) {
  static const int ftc[kFactorKernels] = {0, 1, 2, 2, 2, 2}, g[kFactorKernels] = {2, 2, 2, 2, 2, 1},
                   pairs[kFactorKernels] = {0, 0, 0, 0, 1, 0},
                   quad[kFactorKernels] = {0, 0, 0, 1, 0, 0},
                   pipe[kFactorKernels] = {0, 0, 0, 0, 0, 1};
  T.factor_tc = ftc[k];
  T.tcb_g = g[k];
  T.tcb_pairs = pairs[k];
  T.tcb_quad = quad[k];
  T.tcb_pipe = pipe[k];
}
int factor_kernel_of(const BatchTabs& T) {
  if (T.factor_tc < 2) return T.factor_tc;
  if (T.tcb_pipe) return 5;
  return T.tcb_pairs ? 4 : (T.tcb_quad ? 3 : 2);
}

// The handle's batches stop running: its control points change or (leaving) it goes away, and
// then no batch keeps a pointer to it.
void invalidate_batches(ds_ctx* h, bool leaving) {
  for (ds_batch_s* b : h->batches) {
    b->stale = true;
    if (leaving) std::replace(b->hs.begin(), b->hs.end(), h, (ds_ctx*)nullptr);
  }
  if (leaving) h->batches.clear();
}

void free_cp(ds_ctx* h) {
  if (h->self) {
    destroy_batch(h->self);
    h->self = nullptr;
  }
  invalidate_batches(h, false);
  hfree(h, h->d_g64); hfree(h, h->d_gc); hfree(h, h->d_q64); hfree(h, h->d_t64); hfree(h, h->d_node);
  hfree(h, h->d_pn); hfree(h, h->d_tp); hfree(h, h->d_tw); hfree(h, h->d_rank); hfree(h, h->d_seg);
  hfree(h, h->d_segbp); hfree(h, h->d_segstart); hfree(h, h->d_rowptr); hfree(h, h->d_rowcol); hfree(h, h->d_rowbp);
  hfree(h, h->d_A32); hfree(h, h->d_A64); hfree(h, h->d_Af32); hfree(h, h->d_Dinv); hfree(h, h->d_blk); hfree(h, h->d_adiag);
  hfree(h, h->d_gdata); hfree(h, h->d_b); hfree(h, h->d_x); hfree(h, h->d_r); hfree(h, h->d_xf);
  hfree(h, h->d_v2); hfree(h, h->d_v3); hfree(h, h->d_lcnt); hfree(h, h->d_lflags); hfree(h, h->d_tasks);
  hfree(h, h->d_tasks_b);
  hfree(h, h->d_tasks_p);
  hfree(h, h->d_tasks_q);
  hfree(h, h->d_Lp);
  hfree(h, h->d_desc);
  h->N = h->n = 0;
  h->have_frame = false;
}

int check_sticky(ds_ctx* h) {
  if (h->error) return DS_ERR_CUDA;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->error = true;
    return DS_ERR_CUDA;
  }
  return DS_OK;
}

int batch_words_status(ds_batch_s* b) {
  int te = 0;
  if (cudaMemcpy(&te, b->d_words + 5, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DS_ERR_CUDA;
  return te ? DS_ERR_TIMEOUT : DS_OK;
}

int sync_status(ds_ctx* h) {
  wait_solved(h);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->error = true;
    return DS_ERR_CUDA;
  }
  if (h->have_frame) {
    int flag = 0;
    if (cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      h->error = true;
      return DS_ERR_CUDA;
    }
    if (flag & 2) return DS_ERR_ARG;
    if (flag & 1) return DS_ERR_BAD_INPUT;
  }
  if (h->self) {
    int rc = batch_words_status(h->self);
    if (rc) return rc;
  }
  if (h->N > 0) {
    double st = 0;
    if (cudaMemcpy(&st, h->d_acc + ACC_STATUS, sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      h->error = true;
      return DS_ERR_CUDA;
    }
    if (st != 0.0) return DS_ERR_NOT_SPD;
  }
  return DS_OK;
}

// Device-side check of the frame's indices: an out-of-range template pixel (or one without a
// template point) or reference id is replaced by 0 and flagged (bit 2) before any kernel uses it.
__global__ void k_validate(int* __restrict__ midx, int M, const float* __restrict__ depth0,
                           int npx, int* __restrict__ hyp, int n_hyp, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) {
    int j = midx[i];
    if (j < 0 || j >= npx || !(depth0[j] > 0.f)) {
      midx[i] = -1;
      atomicOr(flag, 2);
    }
  }
  if (i < n_hyp) {
    int k = hyp[i];
    if (k < 0 || k >= M) {
      hyp[i] = 0;
      atomicOr(flag, 2);
    }
  }
}

// Replaces flagged match indices by the first valid template pixel (a harmless placeholder).
__global__ void k_sanitize(int* __restrict__ midx, int M, int first_valid) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M && midx[i] < 0) midx[i] = first_valid;
}

// Tile tasks of one problem's left-looking factorisation, column by column: DIAG(j), then
// OFF(j+1, j), ..., OFF(nt-1, j). Every task depends only on tasks earlier in this order.
// Encoding: {0, type, i, j} with type 0 = DIAG, 1 = OFF.
void make_chol_tasks(int nt, std::vector<int4>& out) {
  for (int j = 0; j < nt; ++j) {
    out.push_back(make_int4(0, 0, j, j));
    for (int i = j + 1; i < nt; ++i) out.push_back(make_int4(0, 1, i, j));
  }
}

// Block tasks of the 128 x 128 block factorisation (same encoding), column by column with a
// lookahead of one: DIAG(j + 1) follows OFF(j + 1, j), its last dependency, ahead of the rest
// of column j, so that the diagonal block the next column's products need is started early.
// Every task still depends only on tasks earlier in this order.
void make_chol_tasks_b(int nb, std::vector<int4>& out) {
  if (nb < 1) return;
  out.push_back(make_int4(0, 0, 0, 0));
  for (int j = 0; j < nb; ++j) {
    if (j + 1 < nb) {
      out.push_back(make_int4(0, 1, j + 1, j));
      out.push_back(make_int4(0, 0, j + 1, j + 1));
    }
    for (int i = j + 2; i < nb; ++i) out.push_back(make_int4(0, 1, i, j));
  }
}

// Block tasks with the block columns and the rows below each column pair taken in pairs: the
// pair's panel as below, then {0, 3, I, J0} for the rows I, I + 1 (blocks (I, J0), (I, J1),
// (I + 1, J0), (I + 1, J1) as one task), a lone last row as {0, 2, I, J0}; the next pair's panel
// follows the first of these (the two rows it depends on). Topological.
void make_chol_tasks_q(int nb, std::vector<int4>& out) {
  auto panel = [&](int j0) {
    out.push_back(make_int4(0, 0, j0, j0));
    if (j0 + 1 < nb) {
      out.push_back(make_int4(0, 1, j0 + 1, j0));
      out.push_back(make_int4(0, 0, j0 + 1, j0 + 1));
    }
  };
  auto rows = [&](int i, int j0) {
    out.push_back(make_int4(0, i + 1 < nb ? 3 : 2, i, j0));
  };
  if (nb < 1) return;
  panel(0);
  for (int j0 = 0; j0 + 1 < nb; j0 += 2) {
    int i = j0 + 2;
    if (i < nb) {
      rows(i, j0);
      i += 2;
    }
    if (j0 + 2 < nb) panel(j0 + 2);
    for (; i < nb; i += 2) rows(i, j0);
  }
}

// Block tasks with the block columns taken in pairs (J0 = 2 p, J1 = J0 + 1): the pair's panel
// DIAG(J0), OFF(J1, J0), DIAG(J1), then {0, 2, I, J0} for I = J1 + 1 .. nb - 1, the two blocks
// (I, J0) and (I, J1) as one task; a lone last column is DIAG alone. The next pair's panel
// follows the first two of these (the rows it depends on), ahead of the others. Topological,
// like the single order.
void make_chol_tasks_p(int nb, std::vector<int4>& out) {
  auto panel = [&](int j0) {
    out.push_back(make_int4(0, 0, j0, j0));
    if (j0 + 1 < nb) {
      out.push_back(make_int4(0, 1, j0 + 1, j0));
      out.push_back(make_int4(0, 0, j0 + 1, j0 + 1));
    }
  };
  if (nb < 1) return;
  panel(0);
  for (int j0 = 0; j0 + 1 < nb; j0 += 2) {
    int i = j0 + 2;
    for (; i < nb && i < j0 + 4; ++i) out.push_back(make_int4(0, 2, i, j0));
    if (j0 + 2 < nb) panel(j0 + 2);
    for (; i < nb; ++i) out.push_back(make_int4(0, 2, i, j0));
  }
}

// Claim order of the factorisation tickets of a batch: problems interleaved round-robin, each
// problem's tasks in their own (topological) order, so every task waits only on earlier tickets.
void make_chol_tickets(const std::vector<int>& ntasks, std::vector<int2>& out) {
  int mx = 0;
  for (int v : ntasks) mx = std::max(mx, v);
  for (int k = 0; k < mx; ++k)
    for (int p = 0; p < (int)ntasks.size(); ++p)
      if (k < ntasks[p]) out.push_back(make_int2(p, k));
}

// Events recorded while the stream is captured become event-record nodes of the graph only with
// cudaEventRecordExternal (a plain record is a capture-internal dependency marker).
void trace(ds_batch_s* b, int it, int k) {
  if (b->tracing) cudaEventRecordWithFlags(b->ev[it][k], b->stream, cudaEventRecordExternal);
}

// ----------------------------------------------------------------------------- batches

void destroy_batch(ds_batch_s* b) {
  if (!b) return;
  for (ds_ctx* h : b->hs)
    if (h) h->batches.erase(std::remove(h->batches.begin(), h->batches.end(), b), h->batches.end());
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->ev_made)
    for (int i = 0; i < DS_MAX_ITERS; ++i)
      for (int k = 0; k < 5; ++k) cudaEventDestroy(b->ev[i][k]);
  if (b->side) cudaStreamSynchronize(b->side);
  if (b->side2) cudaStreamSynchronize(b->side2);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->ev_join2) cudaEventDestroy(b->ev_join2);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->side2) cudaStreamDestroy(b->side2);
  for (auto e : b->ev_in) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (b->ev_tab[i]) cudaEventDestroy(b->ev_tab[i]);
    if (b->h_tab_pin[i]) cudaFreeHost(b->h_tab_pin[i]);
  }
  dfree(b->d_descs);
  dfree(b->d_tab);
  dfree(b->d_words);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int make_batch(ds_ctx* const* hs, int n, cudaStream_t stream, bool own, ds_batch_s** out) {
  *out = nullptr;
  if (n < 1) return DS_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->N == 0 || hs[i]->error) return DS_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return DS_ERR_ARG;   // one problem per handle
  }
  const bool fp64 = hs[0]->prec_fp64;
  const int prec = hs[0]->prm.precision;
  const int steps = prec == DS_PREC_FP32 ? 0 : hs[0]->prm.refine_steps;
  const int ftc = fp64 ? 0 : hs[0]->prm.factor_tc;   // DS_FACTOR_AUTO: tuned per batch
  const int solver = hs[0]->prm.solver;
  for (int i = 1; i < n; ++i) {
    const int ps = hs[i]->prm.precision == DS_PREC_FP32 ? 0 : hs[i]->prm.refine_steps;
    const int ft = hs[i]->prec_fp64 ? 0 : hs[i]->prm.factor_tc;
    if (hs[i]->prec_fp64 != fp64 || (hs[i]->prm.precision == DS_PREC_FP32) != (prec == DS_PREC_FP32) ||
        ps != steps || ft != ftc || hs[i]->prm.solver != solver ||
        hs[i]->prm.jtj != hs[0]->prm.jtj)
      return DS_ERR_ARG;
  }
  ds_batch_s* b = new ds_batch_s();
  b->hs.assign(hs, hs + n);
  b->fp64 = fp64;
  b->refine_steps = steps;
  b->block_jacobi = solver == 1;
  b->stream = stream;
  b->own_stream = own;
  std::vector<int2> icp, rows, nodes, res, chol, chol_b, chol_p, chol_q;
  std::vector<int> ntasks(n), ntasks_b(n), ntasks_p(n), ntasks_q(n);
  int max_tasks = 0, max_nt = 0;
  std::vector<const ProbDesc*> descs(n);
  for (int p = 0; p < n; ++p) {
    ds_ctx* h = hs[p];
    descs[p] = h->d_desc + h->fs;
    for (int t = 0; t * kSegPerCta * kSegPerWarp < h->S; ++t) icp.push_back(make_int2(p, t));
    for (int i = 0; i < h->N; ++i) rows.push_back(make_int2(p, i));
    for (int c = 0; c * 128 < h->N; ++c) nodes.push_back(make_int2(p, c));
    for (int c = 0; c * 8 < h->n; ++c) res.push_back(make_int2(p, c));
    ntasks[p] = h->ntasks;
    ntasks_b[p] = h->ntasks_b;
    ntasks_p[p] = h->ntasks_p;
    ntasks_q[p] = h->ntasks_q;
    max_tasks = std::max(max_tasks, h->ntasks);
    max_nt = std::max(max_nt, h->nt);
  }
  make_chol_tickets(ntasks, chol);
  make_chol_tickets(ntasks_b, chol_b);
  make_chol_tickets(ntasks_p, chol_p);
  make_chol_tickets(ntasks_q, chol_q);
  const size_t ntab = icp.size() + rows.size() + nodes.size() + res.size() + chol.size() +
                      chol_b.size() + chol_p.size() + chol_q.size();
  int rc;
  if ((rc = dalloc(&b->d_descs, n)) || (rc = dalloc(&b->d_tab, ntab)) ||
      (rc = dalloc(&b->d_words, 8))) {
    destroy_batch(b);
    return rc;
  }
  std::vector<int2> all;
  all.reserve(ntab);
  for (auto* v : {&icp, &rows, &nodes, &res, &chol, &chol_b, &chol_p, &chol_q})
    all.insert(all.end(), v->begin(), v->end());
  cudaMemcpy(b->d_descs, descs.data(), sizeof(void*) * n, cudaMemcpyHostToDevice);
  b->h_descs = descs;
  cudaMemcpy(b->d_tab, all.data(), sizeof(int2) * ntab, cudaMemcpyHostToDevice);
  cudaMemset(b->d_words, 0, sizeof(int) * 8);
  BatchTabs& T = b->tabs;
  T.d = b->d_descs;
  T.P = n;
  size_t off = 0;
  T.icp = b->d_tab + off; T.n_icp = (int)icp.size(); off += icp.size();
  T.rows = b->d_tab + off; T.n_rows = (int)rows.size(); off += rows.size();
  T.nodes = b->d_tab + off; T.n_nodes = (int)nodes.size(); off += nodes.size();
  T.res = b->d_tab + off; T.n_res = (int)res.size(); off += res.size();
  T.chol = b->d_tab + off; T.n_chol = (int)chol.size(); off += chol.size();
  T.chol_b = b->d_tab + off; T.n_chol_b = (int)chol_b.size(); off += chol_b.size();
  T.chol_p = b->d_tab + off; T.n_chol_p = (int)chol_p.size(); off += chol_p.size();
  T.chol_q = b->d_tab + off; T.n_chol_q = (int)chol_q.size(); off += chol_q.size();
  T.orb_ctas = 16;
  b->auto_factor = ftc == DS_FACTOR_AUTO;
  set_factor_kernel(T, b->auto_factor ? 0 : ftc);
  T.jtj = hs[0]->prm.jtj;
  T.max_tasks = max_tasks;
  T.max_nt = max_nt;
  T.words = b->d_words;
  for (int i = 0; i < 2; ++i)
    if (cudaMallocHost((void**)&b->h_tab_pin[i], sizeof(void*) * n) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_tab[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      destroy_batch(b);
      return DS_ERR_OOM;
    }
  if (cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->side2, cudaStreamNonBlocking) != cudaSuccess) {
    destroy_batch(b);
    return DS_ERR_CUDA;
  }
  b->ev_in.resize(n, nullptr);
  for (int p = 0; p < n; ++p)
    if (cudaEventCreateWithFlags(&b->ev_in[p], cudaEventDisableTiming) != cudaSuccess) {
      destroy_batch(b);
      return DS_ERR_CUDA;
    }
  for (ds_ctx* h : b->hs) h->batches.push_back(b);
  *out = b;
  return DS_OK;
}

template <typename T>
void enqueue_factor_solve(ds_batch_s* b) {
  cudaStream_t s = b->stream;
  const BatchTabs& B = b->tabs;
  launch_chol_dag<T>(B, s);
  trace(b, b->cur_it, 2);
  launch_trsv_dag<T>(B, 1, false, true, s);
  for (int k = 0; k < b->refine_steps; ++k) {
    launch_residual64(B, s);
    launch_trsv_dag<T>(B, 2 + k, true, false, s);
  }
}

// ICP on the batch stream, ORB beside it on the side stream (fork / join through events, which
// stream capture turns into graph edges).
void linearize_data_terms(ds_batch_s* b, cudaStream_t s) {
  const BatchTabs& B = b->tabs;
  cudaEventRecord(b->ev_fork, s);
  cudaStreamWaitEvent(b->side, b->ev_fork, 0);
  launch_orb(B, b->side);
  cudaEventRecord(b->ev_join, b->side);
  launch_icp(B, s);
  cudaStreamWaitEvent(s, b->ev_join, 0);
}

void enqueue_solve(ds_batch_s* b, int iters) {
  cudaStream_t s = b->stream;
  const BatchTabs& B = b->tabs;
  launch_iter_end(B, -1, false, s);  // node tables of the current state, accumulators cleared
  for (int it = 0; it < iters; ++it) {
    b->cur_it = it;
    trace(b, it, 0);
    launch_iter_begin(B, s);
    linearize_data_terms(b, s);
    if (b->block_jacobi) {
      // diagonal blocks and gradient only, then one FP64 6 x 6 Cholesky solve per control point
      if (b->fp64)
        launch_arap_assemble<double>(B, it == 0, false, s, true);
      else
        launch_arap_assemble<float>(B, it == 0, false, s, true);
      trace(b, it, 1);
      if (b->fp64)
        launch_block_jacobi<double>(B, s);
      else
        launch_block_jacobi<float>(B, s);
      trace(b, it, 2);
      trace(b, it, 4);
      launch_iter_end(B, it, true, s);
      continue;
    }
    if (it > 0) {
      // w_ARAP is fixed after the frame's first linearisation, so the pair assembly runs beside
      // the data terms (second side stream); the data blocks, damping and b follow the join
      cudaStreamWaitEvent(b->side2, b->ev_fork, 0);
      if (b->fp64)
        launch_arap_deferred<double>(B, b->side2);
      else
        launch_arap_deferred<float>(B, b->side2);
      cudaEventRecord(b->ev_join2, b->side2);
      cudaStreamWaitEvent(s, b->ev_join2, 0);
      if (b->fp64)
        launch_arap_finalize<double>(B, s);
      else
        launch_arap_finalize<float>(B, s);
    } else if (b->fp64) {
      launch_arap_assemble<double>(B, true, false, s);
    } else {
      launch_arap_assemble<float>(B, true, false, s);
    }
    trace(b, it, 1);
    if (b->fp64)
      enqueue_factor_solve<double>(b);
    else
      enqueue_factor_solve<float>(b);
    trace(b, it, 4);
    launch_iter_end(B, it, true, s);
  }
  trace(b, iters - 1, 3);
}

// The batch's descriptor table for the next solve: each handle's latest frame slot, or a null
// entry for a handle left out of the solve (active[p] == 0; active == NULL: every handle), which
// every kernel of the solve skips.
void update_desc_table(ds_batch_s* b, const uint8_t* active = nullptr) {
  bool changed = false;
  for (size_t p = 0; p < b->hs.size(); ++p) {
    const ProbDesc* d =
        (active && !active[p]) ? nullptr : b->hs[p]->d_desc + b->hs[p]->fs;
    if (b->h_descs[p] != d) {
      b->h_descs[p] = d;
      changed = true;
    }
  }
  if (!changed) return;
  const int i = b->tab_i ^= 1;
  if (b->tab_pending[i]) cudaEventSynchronize(b->ev_tab[i]);
  std::copy(b->h_descs.begin(), b->h_descs.end(), b->h_tab_pin[i]);
  cudaMemcpyAsync(b->d_descs, b->h_tab_pin[i], sizeof(void*) * b->hs.size(),
                  cudaMemcpyHostToDevice, b->stream);
  cudaEventRecord(b->ev_tab[i], b->stream);
  b->tab_pending[i] = true;
}

// Orders the batch stream after each (active) handle's last solve (possibly in another batch) and
// its pending work (submit_frame on its own stream).
void order_after_handles(ds_batch_s* b, const uint8_t* active = nullptr) {
  cudaStream_t s = b->stream;
  for (size_t p = 0; p < b->hs.size(); ++p) {
    if (active && !active[p]) continue;
    ds_ctx* h = b->hs[p];
    if (h->slot_pending[h->solved_fs]) cudaStreamWaitEvent(s, h->ev_slot_free[h->solved_fs], 0);
    if (h->stream != s) {
      cudaEventRecord(b->ev_in[p], h->stream);
      cudaStreamWaitEvent(s, b->ev_in[p], 0);
    }
  }
}

// Tuned factor-kernel choices by coarse batch shape (ceil log2 of the largest system, rounded
// log2 of the summed n^3), shared by every batch of the process.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tune_cache;


std::pair<int, int> tune_key(const ds_batch_s* b) {
  int mx = 1;
  double f = 0.0;
  for (const ds_ctx* h : b->hs) {
    mx = std::max(mx, h->n);
    f += (double)h->n * h->n * h->n;
  }
  return {(int)ceil(log2((double)mx)), (int)lround(log2(f))};
}

// Times the candidate FP32 factor kernels (SIMT 64 x 64 tiles, tensor cores with 64 x 64 tiles
// and with 128 x 128 blocks) on synthetic SPD systems of the batch's sizes, written into the
// factor buffers (the next solve assembles its own systems over them), and keeps the fastest.
// Each candidate's time is the minimum over `reps` launches (CUDA events on the batch stream).
int tune_factor(ds_batch_s* b, int reps, const uint8_t* active = nullptr) {
  cudaStream_t s = b->stream;
  BatchTabs& T = b->tabs;
  order_after_handles(b, active);
  update_desc_table(b, active);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DS_ERR_CUDA;
  }
  int best = 0;
  double best_ms = INFINITY;
  int rc = DS_OK;
  for (int c = 0; c < kFactorKernels && rc == DS_OK; ++c) {
    set_factor_kernel(T, c);
    float mn = INFINITY;
    for (int r = 0; r < reps; ++r) {
      launch_fill_spd(T, s);
      launch_iter_begin(T, s);
      cudaEventRecord(e0, s);
      launch_chol_dag<float>(T, s);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = DS_ERR_CUDA;
        break;
      }
      mn = std::min(mn, ms);
    }
    g_total_kernels += 3 * reps;
    b->tune_ms[c] = mn;
    if (mn < best_ms) {
      best_ms = mn;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == DS_OK) rc = batch_words_status(b);
  // the synthetic systems are SPD; clear the pivot words anyway so that no tuning run reports
  for (size_t p = 0; p < b->hs.size(); ++p)
    if (!active || active[p]) cudaMemsetAsync(b->hs[p]->d_acc + ACC_STATUS, 0, sizeof(double), s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    rc = DS_ERR_CUDA;
  set_factor_kernel(T, best);
  b->tuned = rc == DS_OK;
  if (b->gexec) {   // a captured loop holds the previous kernel choice
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->g_iters = -1;
  }
  if (rc != DS_OK) b->error = true;
  return rc;
}

int run_batch(ds_batch_s* b, int iters, bool use_graph, const uint8_t* active = nullptr) {
  cudaStream_t s = b->stream;
  if (b->auto_factor && !b->tuned) {
    const auto key = tune_key(b);
    int choice = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) choice = it->second;
    }
    if (choice >= 0) {
      set_factor_kernel(b->tabs, choice);
      b->tuned = true;
    } else {
      const int rc = tune_factor(b, 2, active);
      if (rc) return rc;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune_cache[key] = factor_kernel_of(b->tabs);
    }
  }
  order_after_handles(b, active);
  // the descriptor table points at each (active) handle's latest frame slot
  update_desc_table(b, active);
  const int64_t before = g_launches;
  int64_t launched = 0;
  if (use_graph) {
    if (!b->gexec || b->g_iters != iters) {
      if (b->gexec) cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
      cudaGraph_t g;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        b->error = true;
        return DS_ERR_CUDA;
      }
      enqueue_solve(b, iters);
      if (cudaStreamEndCapture(s, &g) != cudaSuccess) {
        cudaGetLastError();
        b->error = true;
        return DS_ERR_CUDA;
      }
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
      b->g_kernels = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
          ++b->g_kernels;
      }
      cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->gexec = nullptr;
        b->error = true;
        return DS_ERR_CUDA;
      }
      b->g_iters = iters;
    }
    if (cudaGraphLaunch(b->gexec, s) != cudaSuccess) {
      b->error = true;
      return DS_ERR_CUDA;
    }
    launched = b->g_kernels;
  } else {
    enqueue_solve(b, iters);
    launched = g_launches - before;
  }
  g_total_kernels += launched;
  b->last_iters = iters;
  // the slots this solve read are free again after it; the handles' later calls that touch
  // solve state wait for it (wait_solved), their next submissions only for their slot
  cudaEventRecord(b->ev_done, s);
  for (size_t p = 0; p < b->hs.size(); ++p) {
    if (active && !active[p]) continue;
    ds_ctx* h = b->hs[p];
    cudaEventRecord(h->ev_slot_free[h->fs], s);
    h->slot_pending[h->fs] = true;
    h->solved_fs = h->fs;
    h->last_iters = iters;
    h->kernels += launched;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    b->error = true;
    return DS_ERR_CUDA;
  }
  return DS_OK;
}

bool valid_params(const ds_params& p) {
  return p.n_nearest == 4 && p.n_hyp >= 1 && p.n_hyp <= DS_MAX_HYP && p.n_reweight >= 1 &&
         p.n_reweight <= 1000 && p.H_mm > 0 && p.tukey_c_mm > 0 && p.lambda >= 0 &&
         p.eps_damp >= 0 && p.keep_frac >= 0 && p.keep_frac <= 1 && p.sigma_blend_scale > 0 &&
         p.sigma_arap_scale > 0 && p.precision >= 0 && p.precision <= 2 && p.refine_steps >= 0 &&
         p.refine_steps <= 3 && p.w_orb >= 0 && p.w_angle >= 0 && p.w_rot >= 0 &&
         p.w_arap0 >= 0 && (p.factor_tc >= DS_FACTOR_AUTO && p.factor_tc <= 5) &&
         (p.solver == 0 || p.solver == 1) && (p.assoc == 0 || p.assoc == 1) &&
         (p.ransac_o1 == 0 || p.ransac_o1 == 1) && (p.jtj == 0 || p.jtj == 1);
}

bool is_host_ptr(const void* p);

}  // namespace

extern "C" {

void ds_default_params(ds_params* p) {
  if (!p) return;
  p->w_orb = 10.0;
  p->w_angle = 20.0;
  p->w_rot = 100.0;
  p->w_arap0 = 1.0;
  p->H_mm = 2.0;
  p->tukey_c_mm = 10.0;
  p->sigma_blend_scale = 1.0;
  p->sigma_arap_scale = 0.25;
  p->lambda = 1e-4;
  p->eps_damp = 1e-9;
  p->keep_frac = 0.5;
  p->n_hyp = 30;
  p->n_reweight = 10;
  p->n_nearest = 4;
  p->precision = DS_PREC_FP64;
  p->refine_steps = 2;
  p->use_graph = 1;
  p->factor_tc = DS_FACTOR_AUTO;
  p->solver = 0;
  p->assoc = 0;
  p->ransac_o1 = 0;
  p->jtj = 0;
}

const char* ds_status_str(int status) {
  switch (status) {
    case DS_OK: return "ok";
    case DS_ERR_ARG: return "invalid argument";
    case DS_ERR_OOM: return "device out of memory";
    case DS_ERR_BAD_INPUT: return "non-finite input";
    case DS_ERR_NOT_SPD: return "normal equations not positive definite";
    case DS_ERR_STATE: return "call out of order";
    case DS_ERR_TIMEOUT: return "bounded device wait gave up";
    case DS_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

const char* ds_version(void) { return "defsolve 0.1 (sm_103a)"; }

int ds_create_template(const float* depth_hw, int32_t W, int32_t H, ds_intrinsics K,
                       const ds_params* p, void* cuda_stream, ds_handle* out) {
  if (!out || !depth_hw || W < 8 || H < 8 || W > 4096 || H > 4096) return DS_ERR_ARG;
  if (!(K.fx > 0) || !(K.fy > 0) || !isfinite(K.cx) || !isfinite(K.cy)) return DS_ERR_ARG;
  *out = nullptr;
  ds_params prm;
  ds_default_params(&prm);
  if (p) prm = *p;
  if (!valid_params(prm)) return DS_ERR_ARG;
  ds_ctx* h = new ds_ctx();
  h->W = W;
  h->H = H;
  h->K = K;
  h->prm = prm;
  cudaGetDevice(&h->dev);
  int rc = DS_OK;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return DS_ERR_CUDA;
    }
    h->own_stream = true;
  }
  size_t npx = (size_t)W * H;
  h->h_depth0.resize(npx);
  if (cudaMemcpy(h->h_depth0.data(), depth_hw, sizeof(float) * npx, cudaMemcpyDefault) !=
      cudaSuccess) {
    ds_destroy(h);
    return DS_ERR_ARG;
  }
  for (size_t i = 0; i < npx; ++i)
    if (!isfinite(h->h_depth0[i])) {
      ds_destroy(h);
      return DS_ERR_BAD_INPUT;
    }
  for (size_t i = 0; i < npx; ++i)
    if (h->h_depth0[i] > 0.f) h->h_pidx.push_back((int)i);
  if ((rc = halloc(h, &h->d_depth0, npx)) || (rc = halloc(h, &h->d_X64, 3 * npx)) ||
      (rc = halloc(h, &h->d_pidx, h->h_pidx.size())) || (rc = halloc(h, &h->d_depth, npx)) ||
      (rc = halloc(h, &h->d_tpts, 2 * npx)) || (rc = halloc(h, &h->d_tnrm, 2 * npx)) ||
      (rc = halloc(h, &h->d_acc, ACC_COUNT)) || (rc = halloc(h, &h->d_hist, 6 * DS_MAX_ITERS)) ||
      (rc = halloc(h, &h->d_flag, 4)) || (rc = halloc(h, &h->d_hyp, DS_MAX_HYP)) ||
      (rc = halloc(h, &h->d_rs_score, 2 * DS_MAX_HYP)) || (rc = halloc(h, &h->d_rs_kept, 4)) ||
      (rc = halloc(h, &h->d_rs_counts, 8))) {
    ds_destroy(h);
    return rc;
  }
  for (int k = 0; k < 2; ++k)
    if (cudaEventCreateWithFlags(&h->ev_slot_free[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_desc[k], cudaEventDisableTiming) != cudaSuccess) {
      ds_destroy(h);
      return DS_ERR_CUDA;
    }
  if (cudaMallocHost((void**)&h->h_desc_pin, 2 * sizeof(ProbDesc)) != cudaSuccess) {
    cudaGetLastError();
    h->h_desc_pin = nullptr;
    ds_destroy(h);
    return DS_ERR_OOM;
  }
  cudaMemcpy(h->d_depth0, h->h_depth0.data(), sizeof(float) * npx, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_pidx, h->h_pidx.data(), sizeof(int) * h->h_pidx.size(), cudaMemcpyHostToDevice);
  cudaMemset(h->d_acc, 0, sizeof(double) * ACC_COUNT);
  launch_backproject64(h->d_depth0, W, H, K, h->d_X64, h->stream);
  h->h_X64.resize(3 * npx);
  cudaMemcpyAsync(h->h_X64.data(), h->d_X64, sizeof(double) * 3 * npx, cudaMemcpyDeviceToHost,
                  h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    ds_destroy(h);
    return DS_ERR_CUDA;
  }
  *out = h;
  return DS_OK;
}

int ds_set_control_points(ds_handle h, const int32_t* pixel_index, int32_t N) {
  if (!h || !pixel_index || N < 5 || N > 2048) return DS_ERR_ARG;
  if (h->error) return DS_ERR_CUDA;
  std::vector<int> pix(N);
  if (cudaMemcpy(pix.data(), pixel_index, sizeof(int) * N, cudaMemcpyDefault) != cudaSuccess)
    return DS_ERR_ARG;
  const int npx = h->W * h->H;
  {
    std::vector<int> srt(pix);
    std::sort(srt.begin(), srt.end());
    for (int i = 0; i < N; ++i) {
      if (srt[i] < 0 || srt[i] >= npx || !(h->h_depth0[srt[i]] > 0.f)) return DS_ERR_ARG;
      if (i > 0 && srt[i] == srt[i - 1]) return DS_ERR_ARG;
    }
  }
  wait_solved(h);
  cudaStreamSynchronize(h->stream);
  free_cp(h);
  h->N = N;
  h->n = 6 * N;
  h->h_nodepix = pix;
  // node positions, spacing, bounding box, centroid (FP64, host)
  std::vector<double> g(3 * N);
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) g[3 * i + a] = h->h_X64[3 * (size_t)pix[i] + a];
  double msum = 0.0;
  for (int i = 0; i < N; ++i) {
    double best = INFINITY;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double dx = g[3 * i] - g[3 * j], dy = g[3 * i + 1] - g[3 * j + 1],
             dz = g[3 * i + 2] - g[3 * j + 2];
      best = std::min(best, dx * dx + dy * dy + dz * dz);
    }
    msum += sqrt(best);
  }
  h->sigma_b = h->prm.sigma_blend_scale * (msum / N);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double gc[3] = {0, 0, 0};
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], g[3 * i + a]);
      hi[a] = std::max(hi[a], g[3 * i + a]);
      gc[a] += g[3 * i + a] / N;
    }
  h->sigma_A = h->prm.sigma_arap_scale *
               sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                    (hi[2] - lo[2]) * (hi[2] - lo[2]));
  int rc;
  const int P = (int)h->h_pidx.size();
  h->P = P;
  int4* d_nid = nullptr;
  float4* d_alpha = nullptr;
  if ((rc = halloc(h, &h->d_g64, 3 * N)) || (rc = halloc(h, &h->d_gc, 3)) ||
      (rc = dalloc(&d_nid, P)) || (rc = dalloc(&d_alpha, P))) {
    dfree(d_nid);
    dfree(d_alpha);
    free_cp(h);
    return rc;
  }
  cudaMemcpy(h->d_g64, g.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_gc, gc, sizeof(double) * 3, cudaMemcpyHostToDevice);
  launch_knn(h->d_X64, h->d_pidx, P, h->d_g64, N, h->sigma_b, d_nid, d_alpha, h->stream);
  h->h_nid_pix.resize(P);
  h->h_alpha_pix.resize(P);
  cudaMemcpyAsync(h->h_nid_pix.data(), d_nid, sizeof(int4) * P, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(h->h_alpha_pix.data(), d_alpha, sizeof(float4) * P, cudaMemcpyDeviceToHost,
                  h->stream);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  dfree(d_nid);
  dfree(d_alpha);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    free_cp(h);
    h->error = true;
    return DS_ERR_CUDA;
  }
  // sort points by their sorted node quadruple (then pixel)
  std::vector<uint64_t> key(P);
  std::vector<int> order(P);
  for (int j = 0; j < P; ++j) {
    int4 q = h->h_nid_pix[j];
    int s[4] = {q.x, q.y, q.z, q.w};
    std::sort(s, s + 4);
    key[j] = ((uint64_t)s[0] << 48) | ((uint64_t)s[1] << 32) | ((uint64_t)s[2] << 16) | (uint64_t)s[3];
    order[j] = j;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
  std::vector<float4> tp(P), tw(P);
  std::vector<int> rank(npx, -1);
  std::vector<int4> segn;
  std::vector<int> segbp, segstart;
  std::unordered_map<uint64_t, int> bpmap;
  std::vector<std::pair<int, int>> bplist;
  auto bp_of = [&](int a, int b) {
    uint64_t k = ((uint64_t)a << 32) | (uint64_t)b;
    auto it = bpmap.find(k);
    if (it != bpmap.end()) return it->second;
    int id = (int)bplist.size();
    bpmap.emplace(k, id);
    bplist.emplace_back(a, b);
    return id;
  };
  for (int r = 0; r < P; ++r) {
    int j = order[r];
    if (r == 0 || key[j] != key[order[r - 1]]) {
      int4 q = h->h_nid_pix[j];
      int s[4] = {q.x, q.y, q.z, q.w};
      std::sort(s, s + 4);
      segn.push_back(make_int4(s[0], s[1], s[2], s[3]));
      segstart.push_back(r);
      for (int k = 0; k < 10; ++k) {
        int i = kSlotPairI(k), jj = kSlotPairJ(k);
        segbp.push_back(bp_of(s[i], s[jj]));
      }
    }
    int seg = (int)segn.size() - 1;
    int4 sq = segn.back();
    int sn[4] = {sq.x, sq.y, sq.z, sq.w};
    int4 q = h->h_nid_pix[j];
    int on[4] = {q.x, q.y, q.z, q.w};
    float4 al = h->h_alpha_pix[j];
    float oa[4] = {al.x, al.y, al.z, al.w};
    float sa[4] = {0, 0, 0, 0};
    int near_slot = 0;
    for (int k = 0; k < 4; ++k)
      for (int t = 0; t < 4; ++t)
        if (sn[t] == on[k]) {
          sa[t] = oa[k];
          if (k == 0) near_slot = t;
        }
    int pixel = h->h_pidx[j];
    int bits = (seg << 2) | near_slot;
    float fbits;
    memcpy(&fbits, &bits, 4);
    tp[r] = make_float4((float)h->h_X64[3 * (size_t)pixel], (float)h->h_X64[3 * (size_t)pixel + 1],
                        (float)h->h_X64[3 * (size_t)pixel + 2], fbits);
    tw[r] = make_float4(sa[0], sa[1], sa[2], sa[3]);
    rank[pixel] = r;
  }
  h->S = (int)segn.size();
  segstart.push_back(P);
  h->nbp = (int)bplist.size();
  // CSR of the data blocks by node row, both triangles: pair (a, b), a >= b, is listed in row a
  // (column b, block id) and, when a > b, in row b (column a, block id | kBlkTransposed)
  std::vector<int> rowptr(N + 1, 0);
  for (auto& pr : bplist) {
    rowptr[pr.first + 1]++;
    if (pr.first != pr.second) rowptr[pr.second + 1]++;
  }
  for (int i = 0; i < N; ++i) rowptr[i + 1] += rowptr[i];
  const int nent = rowptr[N];
  std::vector<int> rowcol(std::max(nent, 1)), rowbp(std::max(nent, 1));
  {
    std::vector<int> fill(rowptr.begin(), rowptr.end() - 1);
    for (int id = 0; id < h->nbp; ++id) {
      const int a = bplist[id].first, bb = bplist[id].second;
      rowcol[fill[a]] = bb;
      rowbp[fill[a]] = id;
      fill[a]++;
      if (a != bb) {
        rowcol[fill[bb]] = a;
        rowbp[fill[bb]] = id | kBlkTransposed;
        fill[bb]++;
      }
    }
  }
  const int n = h->n;
  const int prec = h->prm.precision;
  const size_t nn = (size_t)n * n;
  const int TB = prec == DS_PREC_FP64 ? chol_tile<double>() : chol_tile<float>();
  const int nt = (n + TB - 1) / TB;
  h->nt = nt;
  const size_t tsz = prec == DS_PREC_FP64 ? sizeof(double) : sizeof(float);
  if ((rc = halloc(h, &h->d_q64, 4 * N)) || (rc = halloc(h, &h->d_t64, 3 * N)) ||
      (rc = halloc(h, &h->d_node, N)) || (rc = halloc(h, &h->d_pn, N)) || (rc = halloc(h, &h->d_tp, P)) ||
      (rc = halloc(h, &h->d_tw, P)) || (rc = halloc(h, &h->d_rank, npx)) ||
      (rc = halloc(h, &h->d_seg, h->S)) || (rc = halloc(h, &h->d_segbp, 10 * h->S)) ||
      (rc = halloc(h, &h->d_segstart, h->S + 1)) ||
      (rc = halloc(h, &h->d_rowptr, N + 1)) || (rc = halloc(h, &h->d_rowcol, rowcol.size())) ||
      (rc = halloc(h, &h->d_rowbp, rowbp.size())) || (rc = halloc(h, &h->d_A32, nn)) ||
      (rc = halloc(h, &h->d_blk, 36 * (size_t)h->nbp)) || (rc = halloc(h, &h->d_gdata, n)) ||
      (rc = halloc(h, &h->d_adiag, 48 * (size_t)N)) ||
      (rc = halloc(h, &h->d_b, n)) || (rc = halloc(h, &h->d_x, n)) || (rc = halloc(h, &h->d_r, n)) ||
      (rc = halloc(h, &h->d_xf, n)) ||
      (rc = halloc(h, (char**)&h->d_v2, tsz * n)) ||
      (rc = halloc(h, (char**)&h->d_v3, tsz * n)) ||
      (rc = halloc(h, (char**)&h->d_Dinv, tsz * (size_t)nt * TB * TB)) ||
      (rc = halloc(h, &h->d_lcnt, (size_t)nt + 2 * (size_t)nt * nt)) ||
      (rc = halloc(h, &h->d_lflags, 2 * (size_t)nt)) ||
      (rc = halloc(h, (char**)&h->d_Lp, tsz * (prec == DS_PREC_FP64 ? chol_packed_elems<double>(nt)
                                                                 : chol_packed_elems<float>(nt))))) {
    free_cp(h);
    return rc;
  }
  if (prec == DS_PREC_FP64 && (rc = halloc(h, &h->d_A64, nn))) {
    free_cp(h);
    return rc;
  }
  if (prec == DS_PREC_FP32_REFINE && (rc = halloc(h, &h->d_Af32, nn))) {
    free_cp(h);
    return rc;
  }
  {
    std::vector<int4> tasks;
    make_chol_tasks(nt, tasks);
    h->ntasks = (int)tasks.size();
    if ((rc = halloc(h, &h->d_tasks, tasks.size()))) {
      free_cp(h);
      return rc;
    }
    cudaMemcpy(h->d_tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice);
    std::vector<int4> tasks_b;
    make_chol_tasks_b((n + 127) / 128, tasks_b);
    h->ntasks_b = (int)tasks_b.size();
    if ((rc = halloc(h, &h->d_tasks_b, tasks_b.size()))) {
      free_cp(h);
      return rc;
    }
    cudaMemcpy(h->d_tasks_b, tasks_b.data(), sizeof(int4) * tasks_b.size(),
               cudaMemcpyHostToDevice);
    std::vector<int4> tasks_p;
    make_chol_tasks_p((n + 127) / 128, tasks_p);
    h->ntasks_p = (int)tasks_p.size();
    if ((rc = halloc(h, &h->d_tasks_p, tasks_p.size()))) {
      free_cp(h);
      return rc;
    }
    cudaMemcpy(h->d_tasks_p, tasks_p.data(), sizeof(int4) * tasks_p.size(),
               cudaMemcpyHostToDevice);
    std::vector<int4> tasks_q;
    make_chol_tasks_q((n + 127) / 128, tasks_q);
    h->ntasks_q = (int)tasks_q.size();
    if ((rc = halloc(h, &h->d_tasks_q, tasks_q.size()))) {
      free_cp(h);
      return rc;
    }
    cudaMemcpy(h->d_tasks_q, tasks_q.data(), sizeof(int4) * tasks_q.size(),
               cudaMemcpyHostToDevice);
  }
  h->prec_fp64 = prec == DS_PREC_FP64;
  {
    ProbDesc& D = h->hdesc;
    memset(&D, 0, sizeof(D));
    D.W = h->W;
    D.H = h->H;
    D.P = P;
    D.N = N;
    D.n = n;
    D.M = 0;
    D.nbp = h->nbp;
    D.fx = h->K.fx;
    D.fy = h->K.fy;
    D.cx = h->K.cx;
    D.cy = h->K.cy;
    D.tukey_c = (float)h->prm.tukey_c_mm;
    D.H_mm = (float)h->prm.H_mm;
    D.w_orb = (float)h->prm.w_orb;
    D.w_angle = (float)h->prm.w_angle;
    D.w_rot = (float)h->prm.w_rot;
    D.inv2sig2 = (float)(1.0 / (2.0 * h->sigma_A * h->sigma_A));
    D.w_arap0 = h->prm.w_arap0;
    D.lam = h->prm.lambda;
    D.eps = h->prm.eps_damp;
    D.write_ref = (prec != DS_PREC_FP32 && h->prm.refine_steps > 0) ? 1 : 0;
    D.assoc = h->prm.assoc;
    D.jtj = h->prm.jtj;
    D.tp = h->d_tp;
    D.tw = h->d_tw;
    D.seg = h->d_seg;
    D.segbp = h->d_segbp;
    D.segstart = h->d_segstart;
    D.S = h->S;
    D.rank = h->d_rank;
    D.tpts = h->d_tpts;
    D.tnrm = h->d_tnrm;
    D.rowptr = h->d_rowptr;
    D.rowcol = h->d_rowcol;
    D.rowbp = h->d_rowbp;
    D.g64 = h->d_g64;
    D.gc = h->d_gc;
    D.node = h->d_node;
    D.pn = h->d_pn;
    D.blk = h->d_blk;
    D.adiag = h->d_adiag;
    D.gdata = h->d_gdata;
    D.acc = h->d_acc;
    D.hist = h->d_hist;
    D.q64 = h->d_q64;
    D.t64 = h->d_t64;
    D.Aref = h->d_A32;
    D.b = h->d_b;
    D.x = h->d_x;
    D.r = h->d_r;
    D.xf = h->d_xf;
    LinProblem& lp = D.lp;
    lp.A = prec == DS_PREC_FP64 ? (void*)h->d_A64
                                : (prec == DS_PREC_FP32_REFINE ? (void*)h->d_Af32 : (void*)h->d_A32);
    lp.Dinv = h->d_Dinv;
    lp.Lp = h->d_Lp;
    lp.n = n;
    lp.nt = nt;
    lp.cnt = h->d_lcnt;
    lp.flags = h->d_lflags;
    lp.tasks = h->d_tasks;
    lp.ntasks = h->ntasks;
    lp.tasks_b = h->d_tasks_b;
    lp.ntasks_b = h->ntasks_b;
    lp.tasks_p = h->d_tasks_p;
    lp.tasks_q = h->d_tasks_q;
    lp.nb = (n + 127) / 128;
    lp.status = h->d_acc + ACC_STATUS;
    lp.y = h->d_v3;
    lp.x = h->d_v2;
    if ((rc = halloc(h, &h->d_desc, 2))) {
      free_cp(h);
      return rc;
    }
    push_desc(h, 0);
    push_desc(h, 1);
  }
  std::vector<double> q0(4 * N, 0.0), t0(3 * N, 0.0);
  for (int i = 0; i < N; ++i) q0[4 * i] = 1.0;
  cudaMemcpy(h->d_q64, q0.data(), sizeof(double) * 4 * N, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_t64, t0.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_tp, tp.data(), sizeof(float4) * P, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_tw, tw.data(), sizeof(float4) * P, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_rank, rank.data(), sizeof(int) * npx, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_seg, segn.data(), sizeof(int4) * h->S, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_segbp, segbp.data(), sizeof(int) * 10 * h->S, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_segstart, segstart.data(), sizeof(int) * (h->S + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_rowptr, rowptr.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_rowcol, rowcol.data(), sizeof(int) * rowcol.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_rowbp, rowbp.data(), sizeof(int) * rowbp.size(), cudaMemcpyHostToDevice);
  cudaMemset(h->d_A32, 0, sizeof(float) * nn);
  if (h->d_A64) cudaMemset(h->d_A64, 0, sizeof(double) * nn);
  if (h->d_Af32) cudaMemset(h->d_Af32, 0, sizeof(float) * nn);
  cudaMemset(h->d_acc, 0, sizeof(double) * ACC_COUNT);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    h->error = true;
    return DS_ERR_CUDA;
  }
  return DS_OK;
}

}  // extern "C"

namespace {
bool is_host_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}
}  // namespace

extern "C" {

int ds_submit_frame(ds_handle h, const float* depth_hw, const int32_t* match_tmpl_idx,
                    const float* match_xyz, int32_t M, const int32_t* hyp_list) {
  if (!h || !depth_hw || M < 0 || M > 65536) return DS_ERR_ARG;
  if (M > 0 && (!match_tmpl_idx || !match_xyz || !hyp_list)) return DS_ERR_ARG;
  if (M > 0 && h->prm.n_hyp > M) return DS_ERR_ARG;
  if (h->N == 0) return DS_ERR_STATE;
  if (h->error) return DS_ERR_CUDA;
  cudaStream_t s = h->stream;
  const int npx = h->W * h->H;
  const int n_hyp = h->prm.n_hyp;
  int rc;
  if (M > 0 && is_host_ptr(match_tmpl_idx)) {
    for (int k = 0; k < M; ++k) {
      int j = match_tmpl_idx[k];
      if (j < 0 || j >= npx || !(h->h_depth0[j] > 0.f)) return DS_ERR_ARG;
    }
  }
  if (M > 0 && is_host_ptr(hyp_list)) {
    for (int k = 0; k < n_hyp; ++k)
      if (hyp_list[k] < 0 || hyp_list[k] >= M) return DS_ERR_ARG;
  }
  // the new frame goes to the other slot, once the last solve that read that slot is done
  const int ns = h->fs ^ 1;
  if (h->slot_pending[ns]) cudaStreamWaitEvent(s, h->ev_slot_free[ns], 0);
  if (M > h->M_cap) {
    // new slot buffers: every solve and submission still running must be done first
    wait_solved(h);
    cudaStreamSynchronize(s);
    hfree(h, h->d_midx); hfree(h, h->d_mxyz); hfree(h, h->d_rs_scratch); hfree(h, h->d_rs_hbits);
    hfree(h, h->d_rs_hw); hfree(h, h->d_rs_mask); hfree(h, h->d_rs_what); hfree(h, h->d_rs_o1);
    hfree(h, h->d_rs_o1df);
    int cap = std::max(M, 64);
    int words = (cap + 31) / 32;
    if ((rc = halloc(h, &h->d_midx, 2 * (size_t)cap)) || (rc = halloc(h, &h->d_mxyz, 6 * (size_t)cap)) ||
        (rc = halloc(h, &h->d_rs_scratch, (size_t)7 * cap * DS_MAX_HYP)) ||
        (rc = halloc(h, &h->d_rs_hbits, (size_t)words * DS_MAX_HYP)) ||
        (rc = halloc(h, &h->d_rs_hw, (size_t)cap * DS_MAX_HYP)) ||
        (rc = halloc(h, &h->d_rs_mask, 2 * (size_t)words)) ||
        (rc = halloc(h, &h->d_rs_what, 2 * (size_t)cap)) ||
        (rc = halloc(h, &h->d_rs_o1, 3 * (size_t)cap)) ||
        (rc = halloc(h, &h->d_rs_o1df, 6 * (size_t)cap))) {
      // no slot may keep pointers into the freed buffers: both hold no frame now
      h->M_cap = 0;
      h->Ms[0] = h->Ms[1] = 0;
      push_desc(h, 0);
      push_desc(h, 1);
      h->have_frame = false;
      return rc;
    }
    h->M_cap = cap;
    // the other slot's matches are gone: it keeps its live points, with no matches
    h->Ms[h->fs] = 0;
    push_desc(h, h->fs);
  }
  if (h->prm.ransac_o1 == 1) wait_solved(h);   // o1 from the state the last solve left
  int* midx = slot_midx(h, ns);
  float* mxyz = slot_mxyz(h, ns);
  const int64_t launches0 = g_launches;
  if ((rc = copy_in(h->d_depth, depth_hw, sizeof(float) * npx, s))) return rc;
  if ((rc = copy_in(midx, match_tmpl_idx, sizeof(int) * M, s))) return rc;
  if ((rc = copy_in(mxyz, match_xyz, sizeof(float) * 3 * (size_t)M, s))) return rc;
  if (M > 0 && (rc = copy_in(h->d_hyp, hyp_list, sizeof(int) * n_hyp, s))) return rc;
  cudaMemsetAsync(h->d_flag, 0, sizeof(int), s);
  if (M > 0) {
    int nt = std::max(M, n_hyp);
    k_validate<<<(nt + 255) / 256, 256, 0, s>>>(midx, M, h->d_depth0, npx, h->d_hyp, n_hyp,
                                                h->d_flag);
    k_sanitize<<<(M + 255) / 256, 256, 0, s>>>(midx, M, h->h_pidx.empty() ? 0 : h->h_pidx[0]);
    g_launches += 2;
  }
  launch_check_finite(h->d_depth, npx, h->d_flag, s);
  launch_check_finite(mxyz, 3 * M, h->d_flag, s);
  launch_frame_prep(h->d_depth, h->W, h->H, h->K, slot_tpts(h, ns), slot_tnrm(h, ns), s);
  if (M > 0) {
    const bool warm = h->prm.ransac_o1 == 1;
    if (warm)
      launch_warm_o1(midx, M, h->d_rank, h->d_tp, h->d_seg, h->d_X64, h->d_g64, h->d_q64,
                     h->d_t64, h->sigma_b, h->d_rs_o1, s);
    launch_ransac(h->d_depth0, h->W, h->K, midx, mxyz, M, h->d_hyp, n_hyp,
                  h->prm.n_reweight, h->prm.H_mm, h->prm.keep_frac,
                  warm ? h->d_rs_o1 : nullptr, h->d_rs_o1df, h->d_rs_scratch,
                  h->d_rs_hbits, h->d_rs_hw, slot_score(h, ns), slot_mask(h, ns),
                  slot_what(h, ns), slot_kept(h, ns), slot_counts(h, ns), s);
  }
  h->Ms[ns] = M;
  push_desc(h, ns);
  h->fs = ns;
  h->M = M;
  h->kernels += g_launches - launches0;
  if ((rc = check_sticky(h))) return rc;
  h->have_frame = true;
  return DS_OK;
}

static int finish_solve(ds_handle h, int iters, ds_solve_stats* out) {
  int rc = sync_status(h);
  if (rc) return rc;
  if (out) {
    memset(out, 0, sizeof(*out));
    std::vector<double> hist(6 * DS_MAX_ITERS);
    cudaMemcpy(hist.data(), h->d_hist, sizeof(double) * 6 * iters, cudaMemcpyDeviceToHost);
    int counts[4] = {0, 0, 0, 0};
    if (h->Ms[h->solved_fs] > 0)
      cudaMemcpy(counts, slot_counts(h, h->solved_fs), sizeof(int) * 4, cudaMemcpyDeviceToHost);
    out->iters = iters;
    out->n_inliers = counts[0];
    out->n_kept = counts[1];
    for (int i = 0; i < iters; ++i) {
      out->cost[i] = hist[6 * i];
      out->cost_icp[i] = hist[6 * i + 1];
      out->cost_orb[i] = hist[6 * i + 2];
      out->cost_arap[i] = hist[6 * i + 3];
    }
    out->n_icp_valid_last = (int)hist[6 * (iters - 1) + 4];
    out->w_arap = hist[6 * (iters - 1) + 5];
  }
  return check_sticky(h);
}

static int ensure_self(ds_handle h) {
  if (h->self) return DS_OK;
  ds_ctx* one[1] = {h};
  int rc = make_batch(one, 1, h->stream, false, &h->self);
  if (rc) return rc;
  h->self->tracing = h->tracing;
  if (h->tracing) {
    for (int i = 0; i < DS_MAX_ITERS; ++i)
      for (int k = 0; k < 5; ++k) cudaEventCreate(&h->self->ev[i][k]);
    h->self->ev_made = true;
  }
  return DS_OK;
}

int ds_solve(ds_handle h, int32_t iters, ds_solve_stats* out) {
  if (!h || iters < 1 || iters > DS_MAX_ITERS) return DS_ERR_ARG;
  if (h->N == 0 || !h->have_frame) return DS_ERR_STATE;
  if (h->error) return DS_ERR_CUDA;
  int rc = ensure_self(h);
  if (rc) return rc;
  rc = run_batch(h->self, iters, h->prm.use_graph != 0);
  if (rc) {
    h->error = true;
    return rc;
  }
  if (out) return finish_solve(h, iters, out);
  return DS_OK;
}

int ds_batch_create(const ds_handle* hs, int32_t n, void* cuda_stream, ds_batch* out) {
  if (!hs || !out || n < 1) return DS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return DS_ERR_CUDA;
    own = true;
  }
  std::vector<ds_ctx*> v(hs, hs + n);
  int rc = make_batch(v.data(), n, s, own, out);
  if (rc && own) cudaStreamDestroy(s);
  return rc;
}

int ds_batch_solve(ds_batch b, int32_t iters) {
  if (!b || iters < 1 || iters > DS_MAX_ITERS) return DS_ERR_ARG;
  if (b->error) return DS_ERR_CUDA;
  if (b->stale) return DS_ERR_STATE;
  for (ds_ctx* h : b->hs)
    if (!h->have_frame || h->N == 0) return DS_ERR_STATE;
  bool graph = !b->no_graph;
  for (ds_ctx* h : b->hs) graph = graph && h->prm.use_graph;
  return run_batch(b, iters, graph);
}

int ds_batch_solve_masked(ds_batch b, const uint8_t* active, int32_t iters) {
  if (!b || !active || iters < 1 || iters > DS_MAX_ITERS) return DS_ERR_ARG;
  if (b->error) return DS_ERR_CUDA;
  if (b->stale) return DS_ERR_STATE;
  int n_on = 0;
  for (size_t p = 0; p < b->hs.size(); ++p) {
    if (!active[p]) continue;
    ++n_on;
    if (!b->hs[p]->have_frame || b->hs[p]->N == 0) return DS_ERR_STATE;
  }
  if (n_on == 0) return DS_ERR_ARG;
  bool graph = !b->no_graph;
  for (ds_ctx* h : b->hs) graph = graph && h->prm.use_graph;
  return run_batch(b, iters, graph, active);
}

int ds_batch_tune(ds_batch b, int32_t reps, int32_t* choice, double* ms6) {
  if (!b || reps < 1 || reps > 100) return DS_ERR_ARG;
  if (b->error) return DS_ERR_CUDA;
  if (b->stale) return DS_ERR_STATE;
  if (b->fp64 || b->block_jacobi) {
    if (choice) *choice = -1;   // one kernel only: nothing to choose
    if (ms6)
      for (int c = 0; c < kFactorKernels; ++c) ms6[c] = -1.0;
    return DS_OK;
  }
  const int rc = tune_factor(b, reps);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[tune_key(b)] = factor_kernel_of(b->tabs);
  }
  if (choice) *choice = factor_kernel_of(b->tabs);
  if (ms6)
    for (int c = 0; c < kFactorKernels; ++c) ms6[c] = b->tune_ms[c];
  return DS_OK;
}

int ds_batch_factor_kernel(ds_batch b, int32_t* choice, double* ms6) {
  if (!b || !choice) return DS_ERR_ARG;
  *choice = (b->fp64 || b->block_jacobi) ? -1 : factor_kernel_of(b->tabs);
  if (ms6)
    for (int c = 0; c < kFactorKernels; ++c) ms6[c] = b->tune_ms[c];
  return DS_OK;
}

int ds_batch_set_graph(ds_batch b, int32_t on) {
  if (!b) return DS_ERR_ARG;
  b->no_graph = on == 0;
  return DS_OK;
}

int ds_batch_status(ds_batch b) {
  if (!b) return DS_ERR_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DS_ERR_CUDA;
  int rc = batch_words_status(b);
  if (rc) return rc;
  if (b->stale) return DS_OK;   // nothing ran since the change; the handles report their own
  for (ds_ctx* h : b->hs) {
    double st = 0;
    cudaMemcpy(&st, h->d_acc + ACC_STATUS, sizeof(double), cudaMemcpyDeviceToHost);
    if (st != 0.0) return DS_ERR_NOT_SPD;
  }
  return DS_OK;
}

int ds_batch_destroy(ds_batch b) {
  destroy_batch(b);
  return DS_OK;
}

int ds_solve_batch(ds_handle* hs, int32_t n, int32_t iters) {
  if (!hs || n < 1) return DS_ERR_ARG;
  ds_batch b = nullptr;
  int rc = ds_batch_create(hs, n, nullptr, &b);
  if (rc) return rc;
  rc = ds_batch_solve(b, iters);
  if (!rc) rc = ds_batch_status(b);
  ds_batch_destroy(b);
  return rc;
}

int ds_get_deformation(ds_handle h, float* q_N4, float* t_N3, float* pos_N3) {
  if (!h) return DS_ERR_ARG;
  if (h->N == 0) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  int N = h->N;
  std::vector<double> q(4 * N), t(3 * N);
  cudaMemcpy(q.data(), h->d_q64, sizeof(double) * 4 * N, cudaMemcpyDeviceToHost);
  cudaMemcpy(t.data(), h->d_t64, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost);
  std::vector<float> qf(4 * N), tf(3 * N), pf(3 * N);
  for (int i = 0; i < 4 * N; ++i) qf[i] = (float)q[i];
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) {
      tf[3 * i + a] = (float)t[3 * i + a];
      pf[3 * i + a] = (float)(h->h_X64[3 * (size_t)h->h_nodepix[i] + a] + t[3 * i + a]);
    }
  if (q_N4 && cudaMemcpy(q_N4, qf.data(), sizeof(float) * 4 * N, cudaMemcpyDefault)) return DS_ERR_ARG;
  if (t_N3 && cudaMemcpy(t_N3, tf.data(), sizeof(float) * 3 * N, cudaMemcpyDefault)) return DS_ERR_ARG;
  if (pos_N3 && cudaMemcpy(pos_N3, pf.data(), sizeof(float) * 3 * N, cudaMemcpyDefault))
    return DS_ERR_ARG;
  return rc;
}

int ds_get_deformation64(ds_handle h, double* q_N4, double* t_N3) {
  if (!h) return DS_ERR_ARG;
  if (h->N == 0) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  if (q_N4 && cudaMemcpy(q_N4, h->d_q64, sizeof(double) * 4 * h->N, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (t_N3 && cudaMemcpy(t_N3, h->d_t64, sizeof(double) * 3 * h->N, cudaMemcpyDefault))
    return DS_ERR_ARG;
  return rc;
}

int ds_set_deformation(ds_handle h, const float* q_N4, const float* t_N3) {
  if (!h || !q_N4 || !t_N3) return DS_ERR_ARG;
  if (h->N == 0) return DS_ERR_STATE;
  if (h->error) return DS_ERR_CUDA;
  int N = h->N;
  std::vector<float> qf(4 * N), tf(3 * N);
  if (cudaMemcpy(qf.data(), q_N4, sizeof(float) * 4 * N, cudaMemcpyDefault) ||
      cudaMemcpy(tf.data(), t_N3, sizeof(float) * 3 * N, cudaMemcpyDefault))
    return DS_ERR_ARG;
  std::vector<double> q(4 * N), t(3 * N);
  for (int i = 0; i < N; ++i) {
    double a = qf[4 * i], b = qf[4 * i + 1], c = qf[4 * i + 2], d = qf[4 * i + 3];
    double nn = sqrt(a * a + b * b + c * c + d * d);
    if (!(nn > 0) || !isfinite(nn)) return DS_ERR_BAD_INPUT;
    if (a < 0) nn = -nn;
    q[4 * i] = a / nn;
    q[4 * i + 1] = b / nn;
    q[4 * i + 2] = c / nn;
    q[4 * i + 3] = d / nn;
    for (int k = 0; k < 3; ++k) {
      if (!isfinite(tf[3 * i + k])) return DS_ERR_BAD_INPUT;
      t[3 * i + k] = tf[3 * i + k];
    }
  }
  wait_solved(h);
  cudaStreamSynchronize(h->stream);
  cudaMemcpy(h->d_q64, q.data(), sizeof(double) * 4 * N, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_t64, t.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice);
  return check_sticky(h);
}

int ds_get_inlier_mask(ds_handle h, uint32_t* bits) {
  if (!h || !bits) return DS_ERR_ARG;
  if (!h->have_frame) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  if (h->M > 0 && cudaMemcpy(bits, slot_mask(h, h->fs), sizeof(uint32_t) * ((h->M + 31) / 32),
                             cudaMemcpyDefault))
    return DS_ERR_ARG;
  return DS_OK;
}

int ds_get_ransac(ds_handle h, float* w_M, uint32_t* kept_bits, double* score_nh) {
  if (!h) return DS_ERR_ARG;
  if (!h->have_frame) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  if (h->M == 0) return DS_OK;
  if (w_M && cudaMemcpy(w_M, slot_what(h, h->fs), sizeof(float) * h->M, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (kept_bits &&
      cudaMemcpy(kept_bits, slot_kept(h, h->fs), sizeof(uint32_t) * 2, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (score_nh &&
      cudaMemcpy(score_nh, slot_score(h, h->fs), sizeof(double) * h->prm.n_hyp, cudaMemcpyDefault))
    return DS_ERR_ARG;
  return DS_OK;
}

int ds_get_cost(ds_handle h, double* F) {
  if (!h || !F) return DS_ERR_ARG;
  if (h->last_iters == 0) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  double v = 0;
  cudaMemcpy(&v, h->d_hist + 6 * (h->last_iters - 1), sizeof(double), cudaMemcpyDeviceToHost);
  *F = v;
  return rc;
}

int ds_get_blend_table(ds_handle h, int32_t* P_out, int32_t* pix_P, int32_t* nid_P4,
                       float* alpha_P4) {
  if (!h) return DS_ERR_ARG;
  if (h->N == 0) return DS_ERR_STATE;
  int P = h->P;
  if (P_out) *P_out = P;
  if (pix_P && cudaMemcpy(pix_P, h->h_pidx.data(), sizeof(int) * P, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (nid_P4 && cudaMemcpy(nid_P4, h->h_nid_pix.data(), sizeof(int4) * P, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (alpha_P4 &&
      cudaMemcpy(alpha_P4, h->h_alpha_pix.data(), sizeof(float4) * P, cudaMemcpyDefault))
    return DS_ERR_ARG;
  return DS_OK;
}

int ds_get_frame_points(ds_handle h, float* pts4, float* nrm4) {
  if (!h) return DS_ERR_ARG;
  if (!h->have_frame) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  size_t npx = (size_t)h->W * h->H;
  if (pts4 && cudaMemcpy(pts4, slot_tpts(h, h->fs), sizeof(float4) * npx, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (nrm4 && cudaMemcpy(nrm4, slot_tnrm(h, h->fs), sizeof(float4) * npx, cudaMemcpyDefault))
    return DS_ERR_ARG;
  return DS_OK;
}

int ds_linearize(ds_handle h, double w_arap_in, double* A_nn, double* b_n, double* cost3,
                 double* w_arap_out) {
  if (!h) return DS_ERR_ARG;
  if (h->N == 0 || !h->have_frame) return DS_ERR_STATE;
  if (h->error) return DS_ERR_CUDA;
  int rc = ensure_self(h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  wait_solved(h);
  update_desc_table(h->self);
  const BatchTabs& B = h->self->tabs;
  launch_iter_end(B, -1, false, s);
  const bool first = !(w_arap_in > 0);
  if (!first)
    cudaMemcpyAsync(h->d_acc + ACC_W_ARAP, &w_arap_in, sizeof(double), cudaMemcpyHostToDevice, s);
  launch_iter_begin(B, s);
  linearize_data_terms(h->self, s);
  launch_arap_assemble<float>(B, first, true, s);
  rc = sync_status(h);
  if (rc) return rc;
  double acc[ACC_COUNT];
  cudaMemcpy(acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost);
  if (cost3) {
    cost3[0] = acc[ACC_COST_ICP];
    cost3[1] = acc[ACC_COST_ORB];
    cost3[2] = acc[ACC_COST_ARAP];
  }
  if (w_arap_out) *w_arap_out = acc[ACC_W_ARAP];
  if (b_n && cudaMemcpy(b_n, h->d_b, sizeof(double) * h->n, cudaMemcpyDefault)) return DS_ERR_ARG;
  if (A_nn) {
    double* tmp = nullptr;
    if ((rc = dalloc(&tmp, (size_t)h->n * h->n))) return rc;
    launch_sym_unpack(h->d_A32, h->n, tmp, s);
    cudaError_t e = cudaMemcpyAsync(A_nn, tmp, sizeof(double) * (size_t)h->n * h->n,
                                    cudaMemcpyDefault, s);
    cudaStreamSynchronize(s);
    dfree(tmp);
    if (e != cudaSuccess) return DS_ERR_ARG;
  }
  return check_sticky(h);
}

int ds_set_tracing(ds_handle h, int32_t on) {
  if (!h) return DS_ERR_ARG;
  if (h->error) return DS_ERR_CUDA;
  const bool want = on != 0;
  if (want != h->tracing && h->self) {
    destroy_batch(h->self);  // the graph is re-captured with (or without) the events
    h->self = nullptr;
  }
  h->tracing = want;
  return DS_OK;
}

static int batch_phase_times(ds_batch_s* b, double* ms4) {
  for (int k = 0; k < 4; ++k) ms4[k] = 0.0;
  const int it_n = b->last_iters;
  for (int it = 0; it < it_n; ++it) {
    float a = 0, bb = 0, c = 0, d = 0;
    cudaError_t e = cudaEventElapsedTime(&a, b->ev[it][0], b->ev[it][1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&bb, b->ev[it][1], b->ev[it][2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&c, b->ev[it][2], b->ev[it][4]);
    if (e == cudaSuccess)
      e = cudaEventElapsedTime(&d, b->ev[it][4],
                               it + 1 < it_n ? b->ev[it + 1][0] : b->ev[it_n - 1][3]);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not a sticky error: the events were not recorded by this solve
      return DS_ERR_STATE;
    }
    ms4[0] += a;
    ms4[1] += bb;
    ms4[2] += c;
    ms4[3] += d;
  }
  return DS_OK;
}

int ds_get_phase_times(ds_handle h, double* ms4) {
  if (!h || !ms4) return DS_ERR_ARG;
  if (!h->tracing || !h->self || h->self->last_iters == 0) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  return batch_phase_times(h->self, ms4);
}

int ds_batch_set_tracing(ds_batch b, int32_t on) {
  if (!b) return DS_ERR_ARG;
  const bool want = on != 0;
  if (want && !b->ev_made) {
    for (int i = 0; i < DS_MAX_ITERS; ++i)
      for (int k = 0; k < 5; ++k)
        if (cudaEventCreate(&b->ev[i][k]) != cudaSuccess) return DS_ERR_CUDA;
    b->ev_made = true;
  }
  if (want != b->tracing && b->gexec) {
    cudaStreamSynchronize(b->stream);
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->g_iters = -1;
  }
  b->tracing = want;
  return DS_OK;
}

int ds_batch_phase_times(ds_batch b, double* ms4) {
  if (!b || !ms4) return DS_ERR_ARG;
  if (!b->tracing || b->last_iters == 0) return DS_ERR_STATE;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DS_ERR_CUDA;
  return batch_phase_times(b, ms4);
}

int ds_get_device_bytes(ds_handle h, int64_t* bytes) {
  if (!h || !bytes) return DS_ERR_ARG;
  *bytes = (int64_t)h->device_bytes;
  return DS_OK;
}

int ds_factor_tasks(int32_t nb, int32_t paired, int32_t* out, int32_t cap, int32_t* ntasks) {
  if (nb < 1 || paired < 0 || paired > 2 || !ntasks || (cap > 0 && !out)) return DS_ERR_ARG;
  std::vector<int4> t;
  if (paired == 2)
    make_chol_tasks_q(nb, t);
  else if (paired == 1)
    make_chol_tasks_p(nb, t);
  else
    make_chol_tasks_b(nb, t);
  *ntasks = (int32_t)t.size();
  for (int k = 0; k < (int)t.size() && k < cap; ++k) {
    out[3 * k] = t[k].y;
    out[3 * k + 1] = t[k].z;
    out[3 * k + 2] = t[k].w;
  }
  return DS_OK;
}

int ds_get_counters(ds_handle h, int64_t* kernels_launched) {
  if (!kernels_launched) return DS_ERR_ARG;
  *kernels_launched = h ? h->kernels : g_total_kernels.load();
  return DS_OK;
}

int ds_destroy(ds_handle h) {
  if (!h) return DS_OK;
  if (h->stream) {
    wait_solved(h);
    cudaStreamSynchronize(h->stream);
  }
  invalidate_batches(h, true);
  free_cp(h);
  hfree(h, h->d_depth0); hfree(h, h->d_X64); hfree(h, h->d_pidx); hfree(h, h->d_depth); hfree(h, h->d_tpts);
  hfree(h, h->d_tnrm); hfree(h, h->d_midx); hfree(h, h->d_mxyz); hfree(h, h->d_hyp);
  hfree(h, h->d_rs_scratch); hfree(h, h->d_rs_hbits); hfree(h, h->d_rs_hw); hfree(h, h->d_rs_score);
  hfree(h, h->d_rs_mask); hfree(h, h->d_rs_what); hfree(h, h->d_rs_kept); hfree(h, h->d_rs_counts);
  hfree(h, h->d_rs_o1); hfree(h, h->d_rs_o1df);
  hfree(h, h->d_acc); hfree(h, h->d_hist); hfree(h, h->d_flag);
  for (int k = 0; k < 2; ++k) {
    if (h->ev_slot_free[k]) cudaEventDestroy(h->ev_slot_free[k]);
    if (h->ev_desc[k]) cudaEventDestroy(h->ev_desc[k]);
  }
  if (h->h_desc_pin) cudaFreeHost(h->h_desc_pin);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return DS_OK;
}

}  // extern "C"
