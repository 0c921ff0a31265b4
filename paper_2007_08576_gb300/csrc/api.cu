// C ABI of libdefsolve (declared in include/defsolve.h): handle life cycle, template and
// control-point set-up, frame submission and the damped Gauss-Newton loop.
//
// Set-up (once per template / control-point set):
//   * the template depth is back-projected in FP64; control points g_i are template points;
//   * the blend table (4 nearest control points, Gaussian weights) is computed on the device;
//   * the host sorts the valid template points by their node quadruple, so that points sharing
//     the same 4 nodes are contiguous ("segments"), and enumerates the node pairs that share a
//     point (the block-sparse pattern of the ICP and ORB contributions to A).
// Per frame: copy-in, live points and normals, RANSAC preselection.
// Per Gauss-Newton iteration: ICP + ORB accumulation, dense ARAP + assembly + damping,
// Cholesky, triangular solves (+ FP64 refinement), state update. The whole loop of a solve is
// captured once as a CUDA graph per iteration count and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "ds_internal.cuh"

using namespace ds;

namespace ds {
thread_local int64_t g_launches = 0;
}

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
  int* d_rowptr = nullptr;
  int* d_rowcol = nullptr;
  int* d_rowbp = nullptr;
  std::vector<int4> h_nid_pix;
  std::vector<float4> h_alpha_pix;
  // frame
  float* d_depth = nullptr;
  float4* d_tpts = nullptr;
  float4* d_tnrm = nullptr;
  int M = 0, M_cap = 0;
  int* d_midx = nullptr;
  float* d_mxyz = nullptr;
  int* d_hyp = nullptr;
  bool have_frame = false;
  // ransac
  double* d_rs_scratch = nullptr;
  uint32_t* d_rs_hbits = nullptr;
  float* d_rs_hw = nullptr;
  double* d_rs_score = nullptr;
  uint32_t* d_rs_mask = nullptr;
  float* d_rs_what = nullptr;
  uint32_t* d_rs_kept = nullptr;
  int* d_rs_counts = nullptr;
  // linear system
  float* d_A32 = nullptr;     // FP32 system (factor in DS_PREC_FP32, reference otherwise)
  double* d_A64 = nullptr;    // FP64 factor (DS_PREC_FP64)
  float* d_Af32 = nullptr;    // FP32 factor copy (DS_PREC_FP32_REFINE)
  void* d_Dinv = nullptr;
  float* d_blk = nullptr;
  float* d_gdata = nullptr;
  double* d_b = nullptr;
  double* d_x = nullptr;
  double* d_r = nullptr;
  void* d_v1 = nullptr;
  void* d_v2 = nullptr;
  void* d_v3 = nullptr;
  // persistent factorisation / solve
  LinProblem* d_lp = nullptr;
  int* d_lcnt = nullptr;      // factorisation task counters
  int* d_lflags = nullptr;    // solve row flags
  int4* d_tasks = nullptr;
  int ntasks = 0;
  int2* d_tickets = nullptr;
  int ntickets = 0;
  int* d_lhead = nullptr;     // [0] factorisation ticket head, [1] solve ticket head
  int* d_lerr = nullptr;      // bounded-wait timeout word
  int nt = 0;
  double* d_acc = nullptr;
  double* d_hist = nullptr;   // DS_MAX_ITERS x 6
  int* d_flag = nullptr;
  // graph
  cudaGraphExec_t gexec = nullptr;
  int g_iters = -1;
  int64_t g_kernels = 0;       // kernel nodes in the instantiated graph
  int64_t kernels = 0;         // kernels launched so far
  // tracing
  bool tracing = false;
  int cur_it = 0;
  cudaEvent_t ev[DS_MAX_ITERS][5] = {};
  bool ev_made = false;
  int last_iters = 0;
  bool error = false;
};

namespace {

#define DS_TRY(expr)                                 \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) {                         \
      if (_e == cudaErrorMemoryAllocation) return DS_ERR_OOM; \
      return DS_ERR_CUDA;                            \
    }                                                \
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

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return DS_OK;
  DS_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return DS_OK;
}

void free_cp(ds_ctx* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  h->g_iters = -1;
  dfree(h->d_g64); dfree(h->d_gc); dfree(h->d_q64); dfree(h->d_t64); dfree(h->d_node);
  dfree(h->d_pn); dfree(h->d_tp); dfree(h->d_tw); dfree(h->d_rank); dfree(h->d_seg);
  dfree(h->d_segbp); dfree(h->d_rowptr); dfree(h->d_rowcol); dfree(h->d_rowbp);
  dfree(h->d_A32); dfree(h->d_A64); dfree(h->d_Af32); dfree(h->d_Dinv); dfree(h->d_blk);
  dfree(h->d_gdata); dfree(h->d_b); dfree(h->d_x); dfree(h->d_r); dfree(h->d_v1);
  dfree(h->d_v2); dfree(h->d_v3); dfree(h->d_lp); dfree(h->d_lcnt); dfree(h->d_lflags);
  dfree(h->d_tasks); dfree(h->d_tickets); dfree(h->d_lhead); dfree(h->d_lerr);
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

int sync_status(ds_ctx* h) {
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
  if (h->d_lerr) {
    int te = 0;
    if (cudaMemcpy(&te, h->d_lerr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      h->error = true;
      return DS_ERR_CUDA;
    }
    if (te) return DS_ERR_TIMEOUT;
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

__global__ void k_record_clear(double* acc, double* hist, int it) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double* hrow = hist + 6 * it;
    hrow[0] = acc[ACC_COST_ICP] + acc[ACC_COST_ORB] + acc[ACC_COST_ARAP];
    hrow[1] = acc[ACC_COST_ICP];
    hrow[2] = acc[ACC_COST_ORB];
    hrow[3] = acc[ACC_COST_ARAP];
    hrow[4] = acc[ACC_NVALID];
    hrow[5] = acc[ACC_W_ARAP];
    for (int i = 0; i < ACC_W_ARAP; ++i) acc[i] = 0.0;
  }
}

__global__ void k_clear_acc(double* acc, int keep_w) {
  if (threadIdx.x < ACC_COUNT) {
    if (!(keep_w && threadIdx.x == ACC_W_ARAP)) acc[threadIdx.x] = 0.0;
  }
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

// Events recorded while the stream is captured become event-record nodes of the graph only with
// cudaEventRecordExternal (a plain record is a capture-internal dependency marker).
// Tile tasks of one problem's factorisation in a topological order with one step of look-ahead:
// CRIT(k) (last update of (k,k), POTRF(k), TRSM(k+1,k)), TRSM(i>k+1, k), the rest of step k-1's
// trailing update, then step k's update of column k+1 (which the next critical task needs).
// Encoding: {problem, type | k << 4, i, j}.
void make_chol_tasks(int p, int nt, std::vector<int4>& out) {
  auto C = [&](int k) { out.push_back(make_int4(p, 0 | (k << 4), k, k)); };
  auto T = [&](int i, int k) { out.push_back(make_int4(p, 1 | (k << 4), i, k)); };
  auto G = [&](int i, int j, int k) { out.push_back(make_int4(p, 2 | (k << 4), i, j)); };
  for (int k = 0; k < nt; ++k) {
    C(k);
    for (int i = k + 2; i < nt; ++i) T(i, k);
    if (k >= 1)
      for (int j = k + 1; j < nt; ++j)
        for (int i = j; i < nt; ++i) G(i, j, k - 1);
    if (k + 1 < nt)
      for (int i = k + 2; i < nt; ++i) G(i, k + 1, k);
  }
}

void trace_ev(ds_ctx* h, cudaEvent_t e) {
  if (h->tracing) cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
}
void trace(ds_ctx* h, int it, int k) { trace_ev(h, h->ev[it][k]); }

// One linearisation (ICP + ORB + ARAP + assembly) into the buffers of the handle's precision.
void enqueue_linearize(ds_ctx* h, bool first, double lam, bool factor_buffers) {
  cudaStream_t s = h->stream;
  const ds_params& p = h->prm;
  cudaMemsetAsync(h->d_blk, 0, sizeof(float) * 36 * (size_t)h->nbp, s);
  cudaMemsetAsync(h->d_gdata, 0, sizeof(float) * h->n, s);
  launch_icp(h->d_tp, h->d_tw, h->d_seg, h->d_segbp, h->P, h->d_node, h->d_tpts, h->d_tnrm, h->W,
             h->H, h->K, (float)p.tukey_c_mm, h->d_blk, h->d_gdata, h->d_acc, s);
  launch_orb(h->d_midx, h->d_mxyz, h->M, h->d_rank, h->d_tp, h->d_tw, h->d_seg, h->d_segbp,
             h->d_node, h->d_rs_mask, h->d_rs_what, (float)p.H_mm, (float)p.w_orb, h->d_blk,
             h->d_gdata, h->d_acc, s);
  float inv2sig2 = (float)(1.0 / (2.0 * h->sigma_A * h->sigma_A));
  if (factor_buffers && p.precision == DS_PREC_FP64) {
    launch_arap_assemble<double>(h->d_pn, h->N, inv2sig2, h->d_rowptr, h->d_rowcol, h->d_rowbp,
                                 h->d_blk, h->d_gdata, h->d_acc, first, p.w_arap0,
                                 (float)p.w_orb, (float)p.w_angle, (float)p.w_rot, lam,
                                 p.eps_damp, h->d_A64,
                                 p.refine_steps > 0 ? h->d_A32 : nullptr, h->d_b, s);
  } else if (factor_buffers && p.precision == DS_PREC_FP32_REFINE) {
    launch_arap_assemble<float>(h->d_pn, h->N, inv2sig2, h->d_rowptr, h->d_rowcol, h->d_rowbp,
                                h->d_blk, h->d_gdata, h->d_acc, first, p.w_arap0, (float)p.w_orb,
                                (float)p.w_angle, (float)p.w_rot, lam, p.eps_damp, h->d_Af32,
                                h->d_A32, h->d_b, s);
  } else {
    launch_arap_assemble<float>(h->d_pn, h->N, inv2sig2, h->d_rowptr, h->d_rowcol, h->d_rowbp,
                                h->d_blk, h->d_gdata, h->d_acc, first, p.w_arap0, (float)p.w_orb,
                                (float)p.w_angle, (float)p.w_rot, lam, p.eps_damp, h->d_A32,
                                nullptr, h->d_b, s);
  }
}

template <typename T>
void enqueue_trsv(ds_ctx* h) {
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->d_lflags, 0, sizeof(int) * 2 * h->nt, s);
  cudaMemsetAsync(h->d_lhead + 1, 0, sizeof(int), s);
  launch_trsv_dag<T>(h->d_lp, h->d_tickets, h->ntickets, h->d_lhead + 1, h->d_lerr, s);
}

template <typename T>
void enqueue_factor_solve(ds_ctx* h, int steps) {
  cudaStream_t s = h->stream;
  int n = h->n;
  T* v1 = (T*)h->d_v1;
  T* v2 = (T*)h->d_v2;
  const size_t ncnt = (size_t)h->nt + 2 * (size_t)h->nt * h->nt;
  cudaMemsetAsync(h->d_lcnt, 0, sizeof(int) * ncnt, s);
  cudaMemsetAsync(h->d_lhead, 0, sizeof(int), s);
  launch_chol_dag<T>(h->d_lp, h->d_tasks, h->ntasks, h->d_lhead, h->d_lerr, s);
  trace(h, h->cur_it, 2);
  launch_cast_from64<T>(h->d_b, v1, n, s);
  enqueue_trsv<T>(h);
  launch_axpy_to64<T>(v2, h->d_x, n, true, s);
  for (int k = 0; k < steps; ++k) {
    launch_residual64(h->d_A32, n, h->d_b, h->d_x, h->d_r, s);
    launch_cast_from64<T>(h->d_r, v1, n, s);
    enqueue_trsv<T>(h);
    launch_axpy_to64<T>(v2, h->d_x, n, false, s);
  }
}

void enqueue_solve(ds_ctx* h, int iters) {
  cudaStream_t s = h->stream;
  const ds_params& p = h->prm;
  launch_node_update(nullptr, h->N, h->d_q64, h->d_t64, h->d_g64, h->d_gc, h->d_node, h->d_pn,
                     s);
  k_clear_acc<<<1, 32, 0, s>>>(h->d_acc, 0);
  for (int it = 0; it < iters; ++it) {
    h->cur_it = it;
    trace(h, it, 0);
    enqueue_linearize(h, it == 0, p.lambda, true);
    trace(h, it, 1);
    if (p.precision == DS_PREC_FP64)
      enqueue_factor_solve<double>(h, p.refine_steps);
    else if (p.precision == DS_PREC_FP32_REFINE)
      enqueue_factor_solve<float>(h, p.refine_steps);
    else
      enqueue_factor_solve<float>(h, 0);
    trace(h, it, 4);
    k_record_clear<<<1, 32, 0, s>>>(h->d_acc, h->d_hist, it);
    launch_node_update(h->d_x, h->N, h->d_q64, h->d_t64, h->d_g64, h->d_gc, h->d_node, h->d_pn,
                       s);
  }
  trace(h, iters - 1, 3);
}

bool valid_params(const ds_params& p) {
  return p.n_nearest == 4 && p.n_hyp >= 1 && p.n_hyp <= DS_MAX_HYP && p.n_reweight >= 1 &&
         p.n_reweight <= 1000 && p.H_mm > 0 && p.tukey_c_mm > 0 && p.lambda >= 0 &&
         p.eps_damp >= 0 && p.keep_frac >= 0 && p.keep_frac <= 1 && p.sigma_blend_scale > 0 &&
         p.sigma_arap_scale > 0 && p.precision >= 0 && p.precision <= 2 && p.refine_steps >= 0 &&
         p.refine_steps <= 4 && p.w_orb >= 0 && p.w_angle >= 0 && p.w_rot >= 0 &&
         p.w_arap0 >= 0;
}

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
  if ((rc = dalloc(&h->d_depth0, npx)) || (rc = dalloc(&h->d_X64, 3 * npx)) ||
      (rc = dalloc(&h->d_pidx, h->h_pidx.size())) || (rc = dalloc(&h->d_depth, npx)) ||
      (rc = dalloc(&h->d_tpts, npx)) || (rc = dalloc(&h->d_tnrm, npx)) ||
      (rc = dalloc(&h->d_acc, ACC_COUNT)) || (rc = dalloc(&h->d_hist, 6 * DS_MAX_ITERS)) ||
      (rc = dalloc(&h->d_flag, 4)) || (rc = dalloc(&h->d_hyp, DS_MAX_HYP)) ||
      (rc = dalloc(&h->d_rs_score, DS_MAX_HYP)) || (rc = dalloc(&h->d_rs_kept, 2)) ||
      (rc = dalloc(&h->d_rs_counts, 4))) {
    ds_destroy(h);
    return rc;
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
  if ((rc = dalloc(&h->d_g64, 3 * N)) || (rc = dalloc(&h->d_gc, 3)) ||
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
  std::vector<int> segbp;
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
  h->nbp = (int)bplist.size();
  // CSR of the block pairs by row
  std::vector<int> rowptr(N + 1, 0), rowcol(h->nbp), rowbp(h->nbp);
  for (auto& pr : bplist) rowptr[pr.first + 1]++;
  for (int i = 0; i < N; ++i) rowptr[i + 1] += rowptr[i];
  {
    std::vector<int> fill(rowptr.begin(), rowptr.end() - 1);
    for (int id = 0; id < h->nbp; ++id) {
      int a = bplist[id].first;
      rowcol[fill[a]] = bplist[id].second;
      rowbp[fill[a]] = id;
      fill[a]++;
    }
  }
  const int n = h->n;
  const int prec = h->prm.precision;
  const size_t nn = (size_t)n * n;
  const int TB = prec == DS_PREC_FP64 ? chol_tile<double>() : chol_tile<float>();
  const int nt = (n + TB - 1) / TB;
  h->nt = nt;
  const size_t tsz = prec == DS_PREC_FP64 ? sizeof(double) : sizeof(float);
  if ((rc = dalloc(&h->d_q64, 4 * N)) || (rc = dalloc(&h->d_t64, 3 * N)) ||
      (rc = dalloc(&h->d_node, N)) || (rc = dalloc(&h->d_pn, N)) || (rc = dalloc(&h->d_tp, P)) ||
      (rc = dalloc(&h->d_tw, P)) || (rc = dalloc(&h->d_rank, npx)) ||
      (rc = dalloc(&h->d_seg, h->S)) || (rc = dalloc(&h->d_segbp, 10 * h->S)) ||
      (rc = dalloc(&h->d_rowptr, N + 1)) || (rc = dalloc(&h->d_rowcol, h->nbp)) ||
      (rc = dalloc(&h->d_rowbp, h->nbp)) || (rc = dalloc(&h->d_A32, nn)) ||
      (rc = dalloc(&h->d_blk, 36 * (size_t)h->nbp)) || (rc = dalloc(&h->d_gdata, n)) ||
      (rc = dalloc(&h->d_b, n)) || (rc = dalloc(&h->d_x, n)) || (rc = dalloc(&h->d_r, n)) ||
      (rc = dalloc((char**)&h->d_v1, tsz * n)) || (rc = dalloc((char**)&h->d_v2, tsz * n)) ||
      (rc = dalloc((char**)&h->d_v3, tsz * n)) ||
      (rc = dalloc((char**)&h->d_Dinv, tsz * (size_t)nt * TB * TB)) ||
      (rc = dalloc(&h->d_lp, 1)) || (rc = dalloc(&h->d_lcnt, (size_t)nt + 2 * (size_t)nt * nt)) ||
      (rc = dalloc(&h->d_lflags, 2 * (size_t)nt)) || (rc = dalloc(&h->d_lhead, 2)) ||
      (rc = dalloc(&h->d_lerr, 1))) {
    free_cp(h);
    return rc;
  }
  if (prec == DS_PREC_FP64 && (rc = dalloc(&h->d_A64, nn))) {
    free_cp(h);
    return rc;
  }
  if (prec == DS_PREC_FP32_REFINE && (rc = dalloc(&h->d_Af32, nn))) {
    free_cp(h);
    return rc;
  }
  {
    std::vector<int4> tasks;
    make_chol_tasks(0, nt, tasks);
    std::vector<int2> tickets;
    for (int t = 0; t < 2 * nt; ++t) tickets.push_back(make_int2(0, t));
    h->ntasks = (int)tasks.size();
    h->ntickets = (int)tickets.size();
    if ((rc = dalloc(&h->d_tasks, tasks.size())) || (rc = dalloc(&h->d_tickets, tickets.size()))) {
      free_cp(h);
      return rc;
    }
    cudaMemcpy(h->d_tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(h->d_tickets, tickets.data(), sizeof(int2) * tickets.size(), cudaMemcpyHostToDevice);
    LinProblem lp;
    lp.A = prec == DS_PREC_FP64 ? (void*)h->d_A64
                                : (prec == DS_PREC_FP32_REFINE ? (void*)h->d_Af32 : (void*)h->d_A32);
    lp.Dinv = h->d_Dinv;
    lp.n = n;
    lp.nt = nt;
    lp.cnt = h->d_lcnt;
    lp.flags = h->d_lflags;
    lp.status = h->d_acc + ACC_STATUS;
    lp.rhs = h->d_v1;
    lp.y = h->d_v3;
    lp.x = h->d_v2;
    cudaMemcpy(h->d_lp, &lp, sizeof(lp), cudaMemcpyHostToDevice);
    cudaMemset(h->d_lerr, 0, sizeof(int));
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
  cudaMemcpy(h->d_rowptr, rowptr.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_rowcol, rowcol.data(), sizeof(int) * h->nbp, cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_rowbp, rowbp.data(), sizeof(int) * h->nbp, cudaMemcpyHostToDevice);
  cudaMemset(h->d_A32, 0, sizeof(float) * nn);
  if (h->d_A64) cudaMemset(h->d_A64, 0, sizeof(double) * nn);
  if (h->d_Af32) cudaMemset(h->d_Af32, 0, sizeof(float) * nn);
  cudaMemset(h->d_acc, 0, sizeof(double) * ACC_COUNT);
  launch_node_update(nullptr, N, h->d_q64, h->d_t64, h->d_g64, h->d_gc, h->d_node, h->d_pn,
                     h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    h->error = true;
    return DS_ERR_CUDA;
  }
  return DS_OK;
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

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
  if (M > h->M_cap) {
    cudaStreamSynchronize(s);
    dfree(h->d_midx); dfree(h->d_mxyz); dfree(h->d_rs_scratch); dfree(h->d_rs_hbits);
    dfree(h->d_rs_hw); dfree(h->d_rs_mask); dfree(h->d_rs_what);
    int cap = std::max(M, 64);
    int words = (cap + 31) / 32;
    if ((rc = dalloc(&h->d_midx, cap)) || (rc = dalloc(&h->d_mxyz, 3 * (size_t)cap)) ||
        (rc = dalloc(&h->d_rs_scratch, (size_t)7 * cap * DS_MAX_HYP)) ||
        (rc = dalloc(&h->d_rs_hbits, (size_t)words * DS_MAX_HYP)) ||
        (rc = dalloc(&h->d_rs_hw, (size_t)cap * DS_MAX_HYP)) ||
        (rc = dalloc(&h->d_rs_mask, words)) || (rc = dalloc(&h->d_rs_what, cap))) {
      h->M_cap = 0;
      return rc;
    }
    h->M_cap = cap;
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
      h->g_iters = -1;
    }
  }
  // a new M changes the captured graph's launch shapes
  if (M != h->M && h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_iters = -1;
  }
  h->M = M;
  const int64_t launches0 = g_launches;
  if ((rc = copy_in(h->d_depth, depth_hw, sizeof(float) * npx, s))) return rc;
  if ((rc = copy_in(h->d_midx, match_tmpl_idx, sizeof(int) * M, s))) return rc;
  if ((rc = copy_in(h->d_mxyz, match_xyz, sizeof(float) * 3 * (size_t)M, s))) return rc;
  if (M > 0 && (rc = copy_in(h->d_hyp, hyp_list, sizeof(int) * n_hyp, s))) return rc;
  cudaMemsetAsync(h->d_flag, 0, sizeof(int), s);
  if (M > 0) {
    int nt = std::max(M, n_hyp);
    k_validate<<<(nt + 255) / 256, 256, 0, s>>>(h->d_midx, M, h->d_depth0, npx, h->d_hyp, n_hyp,
                                                h->d_flag);
    k_sanitize<<<(M + 255) / 256, 256, 0, s>>>(h->d_midx, M, h->h_pidx.empty() ? 0 : h->h_pidx[0]);
    g_launches += 2;
  }
  launch_check_finite(h->d_depth, npx, h->d_flag, s);
  launch_check_finite(h->d_mxyz, 3 * M, h->d_flag, s);
  launch_frame_prep(h->d_depth, h->W, h->H, h->K, h->d_tpts, h->d_tnrm, s);
  if (M > 0) {
    launch_ransac(h->d_depth0, h->W, h->K, h->d_midx, h->d_mxyz, M, h->d_hyp, n_hyp,
                  h->prm.n_reweight, h->prm.H_mm, h->prm.keep_frac, h->d_rs_scratch,
                  h->d_rs_hbits, h->d_rs_hw, h->d_rs_score, h->d_rs_mask, h->d_rs_what,
                  h->d_rs_kept, h->d_rs_counts, s);
  }
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
    if (h->M > 0) cudaMemcpy(counts, h->d_rs_counts, sizeof(int) * 4, cudaMemcpyDeviceToHost);
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

int ds_solve(ds_handle h, int32_t iters, ds_solve_stats* out) {
  if (!h || iters < 1 || iters > DS_MAX_ITERS) return DS_ERR_ARG;
  if (h->N == 0 || !h->have_frame) return DS_ERR_STATE;
  if (h->error) return DS_ERR_CUDA;
  cudaStream_t s = h->stream;
  if (h->prm.use_graph) {
    if (!h->gexec || h->g_iters != iters) {
      if (h->gexec) cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
      cudaGraph_t g;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->error = true;
        return DS_ERR_CUDA;
      }
      enqueue_solve(h, iters);
      if (cudaStreamEndCapture(s, &g) != cudaSuccess) {
        cudaGetLastError();
        h->error = true;
        return DS_ERR_CUDA;
      }
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
      h->g_kernels = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
          ++h->g_kernels;
      }
      cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        h->gexec = nullptr;
        h->error = true;
        return DS_ERR_CUDA;
      }
      h->g_iters = iters;
    }
    if (cudaGraphLaunch(h->gexec, s) != cudaSuccess) {
      h->error = true;
      return DS_ERR_CUDA;
    }
    h->kernels += h->g_kernels;
  } else {
    int64_t before = g_launches;
    enqueue_solve(h, iters);
    h->kernels += g_launches - before;
  }
  h->last_iters = iters;
  int rc = check_sticky(h);
  if (rc) return rc;
  if (out) return finish_solve(h, iters, out);
  return DS_OK;
}

int ds_solve_batch(ds_handle* hs, int32_t n, int32_t iters) {
  if (!hs || n < 0) return DS_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    int rc = ds_solve(hs[i], iters, nullptr);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    int rc = sync_status(hs[i]);
    if (rc) return rc;
  }
  return DS_OK;
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
  if (h->M > 0 && cudaMemcpy(bits, h->d_rs_mask, sizeof(uint32_t) * ((h->M + 31) / 32),
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
  if (w_M && cudaMemcpy(w_M, h->d_rs_what, sizeof(float) * h->M, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (kept_bits && cudaMemcpy(kept_bits, h->d_rs_kept, sizeof(uint32_t) * 2, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (score_nh &&
      cudaMemcpy(score_nh, h->d_rs_score, sizeof(double) * h->prm.n_hyp, cudaMemcpyDefault))
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
  if (pts4 && cudaMemcpy(pts4, h->d_tpts, sizeof(float4) * npx, cudaMemcpyDefault))
    return DS_ERR_ARG;
  if (nrm4 && cudaMemcpy(nrm4, h->d_tnrm, sizeof(float4) * npx, cudaMemcpyDefault))
    return DS_ERR_ARG;
  return DS_OK;
}

int ds_linearize(ds_handle h, double w_arap_in, double* A_nn, double* b_n, double* cost3,
                 double* w_arap_out) {
  if (!h) return DS_ERR_ARG;
  if (h->N == 0 || !h->have_frame) return DS_ERR_STATE;
  if (h->error) return DS_ERR_CUDA;
  cudaStream_t s = h->stream;
  launch_node_update(nullptr, h->N, h->d_q64, h->d_t64, h->d_g64, h->d_gc, h->d_node, h->d_pn, s);
  k_clear_acc<<<1, 32, 0, s>>>(h->d_acc, 0);
  bool first = !(w_arap_in > 0);
  if (!first) cudaMemcpyAsync(h->d_acc + ACC_W_ARAP, &w_arap_in, sizeof(double),
                              cudaMemcpyHostToDevice, s);
  enqueue_linearize(h, first, 0.0, false);
  int rc = sync_status(h);
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
  // the captured graph and the next solve start from fresh accumulators
  k_clear_acc<<<1, 32, 0, s>>>(h->d_acc, 0);
  return check_sticky(h);
}

int ds_set_tracing(ds_handle h, int32_t on) {
  if (!h) return DS_ERR_ARG;
  if (h->error) return DS_ERR_CUDA;
  bool want = on != 0;
  if (want && !h->ev_made) {
    for (int i = 0; i < DS_MAX_ITERS; ++i)
      for (int k = 0; k < 5; ++k)
        if (cudaEventCreate(&h->ev[i][k]) != cudaSuccess) return DS_ERR_CUDA;
    h->ev_made = true;
  }
  if (want != h->tracing && h->gexec) {
    cudaStreamSynchronize(h->stream);
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_iters = -1;
  }
  h->tracing = want;
  return DS_OK;
}

int ds_get_phase_times(ds_handle h, double* ms4) {
  if (!h || !ms4) return DS_ERR_ARG;
  if (!h->tracing || h->last_iters == 0) return DS_ERR_STATE;
  int rc = sync_status(h);
  if (rc && rc != DS_ERR_NOT_SPD) return rc;
  for (int k = 0; k < 4; ++k) ms4[k] = 0.0;
  int it_n = h->last_iters;
  for (int it = 0; it < it_n; ++it) {
    float a = 0, b = 0, c = 0, d = 0;
    cudaError_t e = cudaEventElapsedTime(&a, h->ev[it][0], h->ev[it][1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, h->ev[it][1], h->ev[it][2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&c, h->ev[it][2], h->ev[it][4]);
    if (e == cudaSuccess)
      e = cudaEventElapsedTime(&d, h->ev[it][4],
                               it + 1 < it_n ? h->ev[it + 1][0] : h->ev[it_n - 1][3]);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not a sticky error: the events were not recorded by this solve
      return DS_ERR_STATE;
    }
    ms4[0] += a;
    ms4[1] += b;
    ms4[2] += c;
    ms4[3] += d;
  }
  return DS_OK;
}

int ds_get_counters(ds_handle h, int64_t* kernels_launched) {
  if (!h || !kernels_launched) return DS_ERR_ARG;
  *kernels_launched = h->kernels;
  return DS_OK;
}

int ds_destroy(ds_handle h) {
  if (!h) return DS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_cp(h);
  dfree(h->d_depth0); dfree(h->d_X64); dfree(h->d_pidx); dfree(h->d_depth); dfree(h->d_tpts);
  dfree(h->d_tnrm); dfree(h->d_midx); dfree(h->d_mxyz); dfree(h->d_hyp);
  dfree(h->d_rs_scratch); dfree(h->d_rs_hbits); dfree(h->d_rs_hw); dfree(h->d_rs_score);
  dfree(h->d_rs_mask); dfree(h->d_rs_what); dfree(h->d_rs_kept); dfree(h->d_rs_counts);
  dfree(h->d_acc); dfree(h->d_hist); dfree(h->d_flag);
  if (h->ev_made)
    for (int i = 0; i < DS_MAX_ITERS; ++i)
      for (int k = 0; k < 5; ++k) cudaEventDestroy(h->ev[i][k]);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return DS_OK;
}

}  // extern "C"
