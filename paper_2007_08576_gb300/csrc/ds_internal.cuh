// Internal declarations of libdefsolve: device-side data layouts, small math helpers and the
// host launchers of every kernel. Only the library's own translation units include this file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "defsolve.h"
#include "per_device.h"

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
// cnt: task counters of the factorisation (nt + 2 nt^2 ints); flags: 2 nt ints of the solves
// (a row is done for solve s when its flag equals s); tasks: the problem's factorisation tasks
// in topological order; status: FP64 word receiving 1 + row of a non-positive pivot; y / x:
// the forward and backward solutions of the solve (T).
struct LinProblem {
  void* A;
  void* Dinv;
  void* Lp;  // packed transposed tiles of L (and of the diagonal inverses), nt (nt + 1) / 2 slots
  int n, nt;
  int* cnt;
  int* flags;
  const int4* tasks;
  int ntasks;
  const int4* tasks_b;  // the tasks of the 128 x 128 block factorisation (tensor cores)
  int ntasks_b;
  const int4* tasks_p;  // the same with the block columns taken in pairs
  const int4* tasks_q;  // the same with the rows below each pair also taken in pairs
  int nb;               // 128-row blocks
  double* status;
  void* y;
  void* x;
};

// Everything the per-iteration kernels need about one problem (one handle). Lives in device
// memory; kernels read sizes that change per frame (M) from it, so captured graphs stay valid.
struct ProbDesc {
  int W, H, P, N, n, M, nbp, S;
  float fx, fy, cx, cy;
  float tukey_c, H_mm, w_orb, w_angle, w_rot, inv2sig2;
  double w_arap0, lam, eps;
  int write_ref;           // the refinement needs the FP32 system (full symmetric) besides the factor
  int assoc;               // ICP association: 0 nearest pixel, 1 bilinear blend of 4 pixels
  int jtj;                 // ICP J^T W J: 0 FP32 SIMT, 1 BF16 on the tensor cores (FP32 accumulate)
  const float4* tp;        // sorted template points (x, y, z, bits(seg << 2 | nearest slot))
  const float4* tw;        // blend weights per sorted point (slot order)
  const int4* seg;         // node quadruple of each segment (ascending ids)
  const int* segbp;        // 10 block-pair ids per segment
  const int* segstart;     // first sorted point of each segment (S + 1 entries)
  const int* rank;         // template pixel -> sorted position, -1 if no point
  const float4* tpts;      // live points (x, y, z, valid)
  const float4* tnrm;      // live normals
  const int* midx;
  const float* mxyz;
  const uint32_t* mask;
  const float* what;
  const int* rowptr;       // CSR of the data blocks by node row (both triangles)
  const int* rowcol;
  const int* rowbp;
  const double* g64;       // node positions (FP64)
  const double* gc;        // node centroid
  NodeGPU* node;
  PairNode* pn;
  float* blk;              // block-sparse data-term blocks (36 floats per pair)
  float* adiag;            // per node: ARAP-only diagonal block (36) and gradient (6), 48 floats
  float* gdata;            // data-term gradient
  double* acc;             // ACC_* scalars
  double* hist;            // DS_MAX_ITERS x 6
  double* q64;
  double* t64;
  float* Aref;             // FP32 system (reference of the refinement, or the factor itself)
  double* b;
  double* x;
  double* r;
  float2* xf;              // x as an unevaluated sum of two floats (hi, lo), for the residual
  LinProblem lp;
};

constexpr int kBlkTransposed = 1 << 30;  // CSR flag: the row uses the block transposed
constexpr int kTile = 256;        // threads per CTA of the ICP pass
constexpr int kSegPerCta = kTile / 32;  // warps (concurrent segments) per CTA of the ICP pass
constexpr int kSegPerWarp = 4;          // segments each ICP warp takes in turn
constexpr int kOuts = 10 * 36 + 24;  // per-segment outputs: 10 blocks of 6x6, 24 gradient entries

// ----------------------------------------------------------------------------- launch set-up

// A launch setting computed once per device (a shared-memory attribute set, an occupancy, the SM
// count): kernel attributes are per device, so the value is cached per device (PerDeviceValue,
// per_device.h) for the device current in the calling thread.
class PerDevice {
 public:
  template <typename F>
  int get(F&& compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    const int v = cache_.get(dev, compute);
    if (v <= 0) cudaGetLastError();
    return v;
  }

 private:
  PerDeviceValue cache_;
};

// Sets a kernel's dynamic shared-memory limit once per device; false if the attribute call fails.
template <typename K>
bool set_smem_once(PerDevice& pd, K kernel, int bytes) {
  return pd.get([&] {
           return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       bytes) == cudaSuccess ? 1 : 0;
         }) > 0;
}

// Resident CTAs per SM of a kernel (clamped to [1, cap]), once per device.
template <typename K>
int ctas_per_sm_once(PerDevice& pd, K kernel, int threads, size_t smem, int cap) {
  const int v = pd.get([&] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess)
      return 0;
    return n < 1 ? 1 : (n > cap ? cap : n);
  });
  return v > 0 ? v : 1;
}

// SMs of the current device (once per device).
inline int num_sms() {
  static PerDevice pd;
  const int v = pd.get([] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    return sms;
  });
  return v > 0 ? v : 1;
}

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
// o1w: NULL (o1 = template points back-projected from depth0) or M x 3 FP64 o1 points;
// o1df: 6 M floats of working space (the o1 points as double-float coordinates)
void launch_ransac(const float* depth0, int W, ds_intrinsics K, const int* midx,
                   const float* mxyz, int M, const int* hyp, int n_hyp, int n_reweight, double H,
                   double keep_frac, const double* o1w, float* o1df, double* scratch,
                   uint32_t* hbits, float* hw, double* score, uint32_t* mask, float* what,
                   uint32_t* kept, int* counts, cudaStream_t s);
// warm-start o1: the matched template points warped by the current FP64 state (blend weights
// recomputed in FP64 from the template point, the 4 nodes of its segment and sigma_b)
void launch_warm_o1(const int* midx, int M, const int* rank, const float4* tp, const int4* seg,
                    const double* X64, const double* g64, const double* q64, const double* t64,
                    double sigma_b, double* o1, cudaStream_t s);

// Work tables of a batch (device arrays of (problem, index) pairs) and its shared words.
struct BatchTabs {
  const ProbDesc* const* d;  // descriptor pointer per problem
  int P;                     // problems
  const int2* icp;           // (problem, group of kSegPerCta x kSegPerWarp segments)
  int n_icp;
  const int2* rows;          // (problem, node) of the dense ARAP pass
  int n_rows;
  const int2* nodes;         // (problem, 128-node chunk)
  int n_nodes;
  const int2* res;           // (problem, 8-row chunk of the refinement residual)
  int n_res;
  int orb_ctas;              // CTAs per problem of the ORB pass (grid-stride over M)
  const int2* chol;          // (problem, task) per factorisation ticket, in claim order
  int n_chol;
  const int2* chol_b;        // the same for the 128 x 128 block tasks
  int n_chol_b;
  int factor_tc;             // FP32 factorisation: 0 SIMT 64-tiles, 1 tensor cores 64-tiles,
                             // 2 tensor cores 128-blocks
  int tcb_g;                 // 128-block kernel: K sub-chunks of 16 per operand and stage (1, 2)
  int tcb_pairs;             // 128-block kernel: block columns taken in pairs
  int tcb_pipe;              // 128-block kernel: K loops overlapping the epilogues (warp roles)
  int tcb_quad;              // 128-block kernel: two rows x two block columns per task
  const int2* chol_q;        // the tickets of those tasks, in claim order
  int n_chol_q;
  const int2* chol_p;        // the tickets of the paired block tasks, in claim order
  int n_chol_p;
  int jtj;                   // ICP J^T W J on the tensor cores (BF16, FP32 accumulation)
  int max_tasks;             // max factorisation tasks over the problems
  int max_nt;                // max tile rows over the problems
  int* words;                // [0] factorisation head, [1..4] solve heads, [5] timeout word
};

// terms.cu (batched over the problems of a BatchTabs)
void launch_iter_begin(const BatchTabs& B, cudaStream_t s);
void launch_icp(const BatchTabs& B, cudaStream_t s);
void launch_orb(const BatchTabs& B, cudaStream_t s);
template <typename T>
void launch_arap_assemble(const BatchTabs& B, bool first, bool lin_only, cudaStream_t s,
                          bool diag_only = false);
template <typename T>
void launch_block_jacobi(const BatchTabs& B, cudaStream_t s);
// ARAP pairs without the data terms (beside the ICP / ORB passes), then the data blocks, the
// diagonal blocks with damping and the right-hand side
template <typename T>
void launch_arap_deferred(const BatchTabs& B, cudaStream_t s);
template <typename T>
void launch_arap_finalize(const BatchTabs& B, cudaStream_t s);
void launch_iter_end(const BatchTabs& B, int it, bool step, cudaStream_t s);

// chol.cu
template <typename T>
int chol_tile();
template <typename T>
size_t chol_packed_elems(int nt);  // elements of the packed L tiles (every FP32 kernel's layout)
template <typename T>
void launch_chol_dag(const BatchTabs& B, cudaStream_t s);
template <typename T>
void launch_trsv_dag(const BatchTabs& B, int solve_id, bool from_r, bool assign, cudaStream_t s);
// refinement residual r = b - A x against the FP32 system (double-float accumulation)
void launch_residual64(const BatchTabs& B, cudaStream_t s);
void launch_sym_unpack(const float* A, int n, double* out, cudaStream_t s);
// synthetic SPD systems of the batch's sizes in the FP32 factor buffers (factor kernel timing)
void launch_fill_spd(const BatchTabs& B, cudaStream_t s);

// Kernels enqueued by this host thread (stream launches, including those recorded into a graph
// under capture); the API layer reads differences of it.
extern thread_local int64_t g_launches;
// Adds kernels launched outside a handle (feature contexts) to the library-wide count that
// ds_get_counters(NULL) reports.
void count_kernels(int64_t n);

}  // namespace ds
