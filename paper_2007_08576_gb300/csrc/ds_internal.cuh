// Internal declarations of libdefsolve: device-side data layouts, small math helpers and the
// host launchers of every kernel. Only the library's own translation units include this file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "defsolve.h"

namespace ds {

// ----------------------------------------------------------------------------- layouts

// Per-node data the point terms read every iteration (64 B, one float4 each):
//   q = rotation quaternion (w, x, y, z), d = dual part 1/2 (0, T) (x) q,
//   T = translation of the node's rigid map x -> R x + T (T = g + t - R g),
//   w = R g + T / 2 (enters the Jacobian of the blended warp).
struct NodeGPU {
  float4 q, d, T, w;
};

// Per-node data of the dense ARAP pass (96 B): q, g (centred), p = g + t (centred), rows of R.
struct PairNode {
  float4 q, g, p, R0, R1, R2;
};

// Device-side scalars of one linearisation (FP64 accumulators).
enum {
  ACC_COST_ICP = 0,
  ACC_COST_ORB,
  ACC_COST_ARAP,
  ACC_WSUM_ICP,
  ACC_WSUM_ORB,
  ACC_NVALID,
  ACC_W_ARAP,     // the frame's w_ARAP (kept across the frame's iterations)
  ACC_STATUS,     // nonzero: a Cholesky pivot was <= 0 (1 + pivot row)
  ACC_COUNT = 8
};

// Slot pairs (i >= j) of the 4 blended nodes of a point: the 10 lower blocks of its 24 x 24
// J^T J contribution; the block of slot pair (i, j) sits at (node_i, node_j) of A.
__host__ __device__ constexpr int kSlotPairI(int k) {
  return k < 1 ? 0 : k < 3 ? 1 : k < 6 ? 2 : 3;
}
__host__ __device__ constexpr int kSlotPairJ(int k) {
  return k < 1 ? k : k < 3 ? k - 1 : k < 6 ? k - 3 : k - 6;
}

// One dense SPD system for the persistent factorisation / solve kernels (one per problem of a
// batch). A: n x n lower, factored in place; Dinv: inverses of the nt diagonal tiles (TB x TB);
// cnt: task counters of the factorisation (nt + 2 nt^2 ints); flags: 2 nt ints of the solve;
// status: FP64 word receiving 1 + row of a non-positive pivot; rhs / y / x: vectors of the
// solve (T).
struct LinProblem {
  void* A;
  void* Dinv;
  int n, nt;
  int* cnt;
  int* flags;
  double* status;
  void* rhs;
  void* y;
  void* x;
};

constexpr int kTile = 256;        // points per CTA of the ICP pass
constexpr int kOuts = 10 * 36 + 24;  // per-segment outputs: 10 blocks of 6x6, 24 gradient entries

// Kernels enqueued by this host thread (stream launches, including those recorded into a graph
// under capture); the API layer reads differences of it.
extern thread_local int64_t g_launches;

// ----------------------------------------------------------------------------- launchers
// frame.cu
void launch_backproject64(const float* depth, int W, int H, ds_intrinsics K, double* X64,
                          cudaStream_t s);
void launch_knn(const double* X64, const int* pidx, int P, const double* g64, int N,
                double sigma_b, int4* nid, float4* alpha, cudaStream_t s);
void launch_frame_prep(const float* depth, int W, int H, ds_intrinsics K, float4* pts,
                       float4* nrm, cudaStream_t s);
void launch_check_finite(const float* v, int n, int* flag, cudaStream_t s);

// ransac.cu
int ransac_smem_bytes(int M);
void launch_ransac(const float* depth0, int W, ds_intrinsics K, const int* midx,
                   const float* mxyz, int M, const int* hyp, int n_hyp, int n_reweight, double H,
                   double keep_frac, double* scratch, uint32_t* hbits, float* hw, double* score,
                   uint32_t* mask, float* what, uint32_t* kept, int* counts, cudaStream_t s);

// terms.cu
void launch_node_update(const double* x, int N, double* q64, double* t64, const double* g64,
                        const double* gc, NodeGPU* node, PairNode* pn, cudaStream_t s);
void launch_icp(const float4* tp, const float4* tw, const int4* segnodes, const int* segbp,
                int P, const NodeGPU* node, const float4* tgt_pt, const float4* tgt_nrm,
                int W, int H, ds_intrinsics K, float c, float* blk, float* gdata, double* acc,
                cudaStream_t s);
void launch_orb(const int* midx, const float* mxyz, int M, const int* rank, const float4* tp,
                const float4* tw, const int4* segnodes, const int* segbp, const NodeGPU* node,
                const uint32_t* mask, const float* what, float H, float w_orb, float* blk,
                float* gdata, double* acc, cudaStream_t s);
// dense ARAP + assembly of A (lower blocks, damped) and b; T = float or double (factor type)
template <typename T>
void launch_arap_assemble(const PairNode* pn, int N, float inv2sig2, const int* rowptr,
                          const int* rowcol, const int* rowbp, const float* blk,
                          const float* gdata, double* acc, bool first_iter, double w_arap0,
                          float w_orb, float w_angle, float w_rot, double lam, double eps,
                          T* Afac, float* Aref, double* b, cudaStream_t s);

// chol.cu
template <typename T>
int chol_tile();
template <typename T>
void launch_chol_dag(const LinProblem* probs, const int4* tasks, int ntasks, int* head, int* err,
                     cudaStream_t s);
template <typename T>
void launch_trsv_dag(const LinProblem* probs, const int2* tickets, int ntk, int* head, int* err,
                     cudaStream_t s);
void launch_residual64(const float* Aref, int n, const double* b, const double* x, double* r,
                       cudaStream_t s);
template <typename T>
void launch_cast_from64(const double* in, T* out, int n, cudaStream_t s);
template <typename T>
void launch_axpy_to64(const T* d, double* x, int n, bool assign, cudaStream_t s);
void launch_sym_unpack(const float* A, int n, double* out, cudaStream_t s);

}  // namespace ds
