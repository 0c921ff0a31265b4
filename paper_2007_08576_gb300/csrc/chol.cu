// Cholesky factorisation of the damped normal equations (Section 2 solves the step for the
// warps W_i through a Cholesky factorisation), for T = double (FP64 factor, TB = 32) or T = float
// (FP32 factor, TB = 64; on the SIMT pipes, or on the tensor cores in k_chol_tc).
//
// Layout: A is n x n row-major; only the lower triangle is read or written. The matrix is cut
// into TB x TB tiles (the last row/column of tiles is ragged).
//
// One persistent launch per Gauss-Newton iteration runs the tile tasks of a left-looking blocked
// Cholesky for every problem of a batch, one task per output tile, in column order:
//   DIAG(j)     C = A_jj - sum_{k<j} L_jk L_jk^T;  L_jj = chol(C) with its inverse L_jj^-1
//   OFF(i, j)   C = A_ij - sum_{k<j} L_ik L_jk^T;  L_ij = C (L_jj^-1)^T          (i > j)
// The finished tiles are also kept in packed slots (transposed and padded for the SIMT kernel,
// TF32 hi / lo parts in the K-major core-matrix layout for the tensor-core kernel) that the
// later tasks stream into shared memory with bulk copies. CTAs claim tasks from an atomic ticket
// counter through a per-batch claim-order table; a task waits on per-tile counters written by
// earlier tickets. Every ticket a CTA waits on was claimed earlier by a running CTA, so the waits
// always end; they are bounded anyway (globaltimer deadline) and a timeout sets an error word,
// after which all CTAs drain the queue without computing. Tiles written inside the launch are
// read through L2 (ld.global.cg, bulk copies) because L1 is not coherent across SMs.
//
// A pivot <= 0 (or NaN) is recorded in the problem's status word as 1 + its row and replaced by
// 1 so that the rest stays finite; the host reports DS_ERR_NOT_SPD.
#include <math.h>

#include "dev_util.cuh"
#include "ds_internal.cuh"

namespace ds {



template <typename T>
__device__ __forceinline__ T tsqrt(T x);
template <>
__device__ __forceinline__ double tsqrt<double>(double x) {
  return sqrt(x);
}
template <>
__device__ __forceinline__ float tsqrt<float>(float x) {
  return sqrtf(x);
}

template <typename T, int TB>
struct TileCfg {
  static constexpr int RT = TB / 16;               // register block per thread (16 x 16 threads)
  static constexpr int LDT = TB + 16 / sizeof(T);  // transposed shared tile row stride (16 B pad)
};

// Stores (or subtracts from) this thread's RT x RT block of tile (ti, tj); lower_only keeps
// r >= c (diagonal tiles). Interior blocks of an aligned matrix move as one 16-byte vector per row.
template <typename T, int TB, bool SUB>
__device__ __forceinline__ void store_block(T* A, int n, int ti, int tj,
                                            const T (&v)[TileCfg<T, TB>::RT][TileCfg<T, TB>::RT],
                                            bool lower_only) {
  constexpr int RT = TileCfg<T, TB>::RT;
  const int tr = (threadIdx.x / 16) * RT, tc = (threadIdx.x % 16) * RT;
  const int rb = ti * TB + tr, cb = tj * TB + tc;
  const bool vec = !lower_only && rb + RT <= n && cb + RT <= n && ((n * sizeof(T)) % 16 == 0);
  if (vec) {
#pragma unroll
    for (int a = 0; a < RT; ++a) {
      T* p = A + (size_t)(rb + a) * n + cb;
      if constexpr (RT == 4) {
        float4 o = SUB ? __ldcg(reinterpret_cast<const float4*>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
        o.x = SUB ? o.x - v[a][0] : v[a][0];
        o.y = SUB ? o.y - v[a][1] : v[a][1];
        o.z = SUB ? o.z - v[a][2] : v[a][2];
        o.w = SUB ? o.w - v[a][3] : v[a][3];
        __stcg(reinterpret_cast<float4*>(p), o);
      } else {
        double2 o = SUB ? __ldcg(reinterpret_cast<const double2*>(p)) : make_double2(0.0, 0.0);
        o.x = SUB ? o.x - v[a][0] : v[a][0];
        o.y = SUB ? o.y - v[a][1] : v[a][1];
        __stcg(reinterpret_cast<double2*>(p), o);
      }
    }
    return;
  }
#pragma unroll
  for (int a = 0; a < RT; ++a) {
    const int r = rb + a;
    if (r >= n) continue;
#pragma unroll
    for (int b = 0; b < RT; ++b) {
      const int c = cb + b;
      if (c < n && (!lower_only || c <= r)) {
        T* p = A + (size_t)r * n + c;
        __stcg(p, SUB ? ldcg(p) - v[a][b] : v[a][b]);
      }
    }
  }
}

// 1/sqrt(p) to working precision: hardware estimate refined by Newton steps
// y <- y (3 - p y^2) / 2 (one step in FP32, two in FP64 from the FP32 estimate).
template <typename T>
__device__ __forceinline__ T rsqrt_newton(T p);
template <>
__device__ __forceinline__ float rsqrt_newton<float>(float p) {
  float y = rsqrtf(p);
  return y * (1.5f - 0.5f * p * y * y);
}
template <>
__device__ __forceinline__ double rsqrt_newton<double>(double p) {
  double y = (double)rsqrtf((float)p);
  y = y * (1.5 - 0.5 * p * y * y);
  return y * (1.5 - 0.5 * p * y * y);
}


// One doubling level of a lower-triangular inverse held in shared memory (row stride TB + 1,
// zeros above the diagonal): for every pair of H x H diagonal blocks starting at s0 = 2 H g,
// Tm = L21 X11 and X21 = -X22 Tm, with L21 = L[s0 + H.., s0..], X11 / X22 the diagonal blocks.
// Each thread forms K consecutive outputs of a row (K = 1..4) with the shared row operand reused.
// Barrier of the threads that run the tile code: the whole block (BAR 0), or the 256 threads of
// named barrier BAR in a block whose other warps have another role.
template <int BAR>
__device__ __forceinline__ void bsync() {
  if constexpr (BAR == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, 256;" ::"n"(BAR) : "memory");
}

template <typename T, int TB, int H, int BAR = 0>
__device__ __forceinline__ void inverse_level(const T* L, T* X, T* Tm) {
  constexpr int LDS = TB + 1, TOTAL = TB * H / 2;
  constexpr int K = TOTAL >= 1024 ? 4 : (TOTAL >= 512 ? 2 : 1);
  constexpr int NT = TOTAL / K;   // working threads
  const int tid = threadIdx.x;
  if (tid < NT) {
    const int e = tid * K, g = e / (H * H), r = (e % (H * H)) / H, c = e % H, s0 = 2 * H * g;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (T)0;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const T l = L[(s0 + H + r) * LDS + s0 + m];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += l * X[(s0 + m) * LDS + s0 + c + k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) Tm[e + k] = v[k];
  }
  bsync<BAR>();
  if (tid < NT) {
    const int e = tid * K, g = e / (H * H), r = (e % (H * H)) / H, c = e % H, s0 = 2 * H * g;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (T)0;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const T xv = X[(s0 + H + r) * LDS + s0 + H + m];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += xv * Tm[g * H * H + m * H + c + k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) X[(s0 + H + r) * LDS + s0 + c + k] = -v[k];
  }
  bsync<BAR>();
}

// Register-blocked Cholesky of a diagonal tile with its inverse. Thread (ty, tx) = (tid / 16,
// tid % 16) holds a[p][q] = C[ty RT + p][tx RT + q] (lower part used; identity padding past the
// matrix). Columns are taken in blocks of PB = 2 RT; the PB x PB diagonal block kb is held by four
// threads of warp kb, so
//   (1) warp kb gathers the block in shared memory, every lane factors it in registers and lane c
//       solves column c of its inverse D (no block-wide barrier);
//   (2) the two threads holding each RT-row slice of the panel below exchange their halves with a
//       shuffle and form L_rb = A_rb D^T, published transposed for the update;
//   (4) every thread right of the panel subtracts the rank-PB product from its registers.
// Two barriers per block. The inverse's off-diagonal blocks then follow by recursive doubling,
// X21 = -X22 (L21 X11), for h = PB, 2 PB, 4 PB (two barriers per level). Output: L (lower part)
// and X = L^-1 in shared memory with row stride TB + 1; X must be zero on entry. Scratch: Pt
// (PB x (TB + 16 / sizeof(T))), Dsm (PB x PB), Tm (TB x TB / 4).
template <typename T, int TB, int BAR = 0>
__device__ void potrf_regs(T (&a)[TileCfg<T, TB>::RT][TileCfg<T, TB>::RT], T* L, T* X, T* Pt,
                           T* Dsm, T* Tm, int row0, double* status) {
  constexpr int RT = TileCfg<T, TB>::RT, PB = 2 * RT, NBK = TB / PB, LDS = TB + 1;
  constexpr int LDP = TileCfg<T, TB>::LDT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = tid / 16, tx = tid % 16, tr = ty * RT, tc = tx * RT;
  for (int kb = 0; kb < NBK; ++kb) {
    const int c0 = kb * PB;
    if (warp == kb) {
      if ((tx >> 1) == kb) {
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q)
            if (tc + q <= tr + p) L[(tr + p) * LDS + tc + q] = a[p][q];
      }
      __syncwarp();
      T l[PB][PB], dinv[PB];
#pragma unroll
      for (int r = 0; r < PB; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) l[r][c] = L[(c0 + r) * LDS + c0 + c];
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        T piv = l[j][j];
#pragma unroll
        for (int q = 0; q < j; ++q) piv -= l[j][q] * l[j][q];
        if (!(piv > (T)0)) {
          if (status && lane == 0)
            atomicCAS((unsigned long long*)status, 0ull,
                      __double_as_longlong((double)(row0 + c0 + j + 1)));
          piv = (T)1;
        }
        const T inv = rsqrt_newton<T>(piv);
        dinv[j] = inv;
        l[j][j] = piv * inv;
#pragma unroll
        for (int r = j + 1; r < PB; ++r) {
          T v = l[r][j];
#pragma unroll
          for (int q = 0; q < j; ++q) v -= l[r][q] * l[j][q];
          l[r][j] = v * inv;
        }
      }
      // lane c < PB: column c of the inverse, x_c = 1 / l_cc, x_r = -(sum_{c<=q<r} l_rq x_q) / l_rr
      const int c = lane;
      T x[PB];
#pragma unroll
      for (int r = 0; r < PB; ++r) {
        T v = (T)0;
#pragma unroll
        for (int q = 0; q < r; ++q) v -= (q >= c ? l[r][q] : (T)0) * x[q];
        x[r] = r == c ? dinv[r] : (r > c ? v * dinv[r] : (T)0);
      }
      __syncwarp();
      // lane q writes column q of L's block (values picked by select, no divergent branches)
#pragma unroll
      for (int r = 0; r < PB; ++r) {
        T v = l[r][0];
#pragma unroll
        for (int q = 1; q <= r; ++q) v = lane == q ? l[r][q] : v;
        if (lane <= r) L[(c0 + r) * LDS + c0 + lane] = v;
      }
      if (lane < PB) {
#pragma unroll
        for (int r = 0; r < PB; ++r) {
          X[(c0 + r) * LDS + c0 + c] = x[r];
          Dsm[r * PB + c] = x[r];
        }
      }
    }
    bsync<BAR>();
    // (2) panel below the block: threads tx = 2 kb, 2 kb + 1 (adjacent lanes), rows past the block
    if ((tx >> 1) == kb && tr >= c0 + PB) {
      const unsigned pair = 3u << (lane & 30);
      const int half = tx & 1;
      T row[RT][PB];
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) {
          const T other = __shfl_xor_sync(pair, a[p][q], 1);
          row[p][q] = half ? other : a[p][q];
          row[p][RT + q] = half ? a[p][q] : other;
        }
#pragma unroll
      for (int q = 0; q < RT; ++q) {
        const int qg = half * RT + q;
        T d[PB];
#pragma unroll
        for (int m = 0; m < PB; ++m) d[m] = m <= qg ? Dsm[qg * PB + m] : (T)0;
#pragma unroll
        for (int p = 0; p < RT; ++p) {
          T v = (T)0;
#pragma unroll
          for (int m = 0; m < PB; ++m) v += row[p][m] * d[m];
          L[(tr + p) * LDS + c0 + qg] = v;
          Pt[qg * LDP + tr + p] = v;
        }
      }
    }
    bsync<BAR>();
    // (4) rank-PB update of the register blocks right of the panel (lower part)
    if (tc >= c0 + PB && tc <= tr + RT - 1) {
#pragma unroll
      for (int m = 0; m < PB; ++m) {
        T xv[RT], yv[RT];
        if constexpr (RT == 4) {
          const float4 u = *reinterpret_cast<const float4*>(Pt + m * LDP + tr);
          const float4 w = *reinterpret_cast<const float4*>(Pt + m * LDP + tc);
          xv[0] = u.x; xv[1] = u.y; xv[2] = u.z; xv[3] = u.w;
          yv[0] = w.x; yv[1] = w.y; yv[2] = w.z; yv[3] = w.w;
        } else {
          const double2 u = *reinterpret_cast<const double2*>(Pt + m * LDP + tr);
          const double2 w = *reinterpret_cast<const double2*>(Pt + m * LDP + tc);
          xv[0] = u.x; xv[1] = u.y;
          yv[0] = w.x; yv[1] = w.y;
        }
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) a[p][q] -= xv[p] * yv[q];
      }
    }
  }
  // off-diagonal blocks of the inverse by recursive doubling (X zero above the diagonal)
  inverse_level<T, TB, PB, BAR>(L, X, Tm);
  inverse_level<T, TB, 2 * PB, BAR>(L, X, Tm);
  inverse_level<T, TB, 4 * PB, BAR>(L, X, Tm);
  static_assert(8 * PB == TB, "three doubling levels");
}

// ----------------------------------------------------------------------------- factorisation

// 1-D bulk copies global -> shared on the TMA engine, completing on an mbarrier (transaction
// bytes). Used only for the packed L tiles, which are 16-byte aligned and a multiple of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for phase `parity` of a bulk-copy barrier; false (and *err raised) on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err,
                                          unsigned long long budget_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_test(bar, parity)) {
    if (globaltimer() - t0 > budget_ns) {
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Orders this thread's earlier generic-proxy global writes before later async-proxy (bulk copy)
// reads of the same data by any thread that synchronises with it.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// acc[a][b] += sum_m P^T[m][tr + a] Q^T[m][tc + b] (transposed operand tiles, row stride LDT).
template <typename T, int TB>
__device__ __forceinline__ void tile_abt_acc(const T* Pt, const T* Qt,
                                             T (&acc)[TileCfg<T, TB>::RT][TileCfg<T, TB>::RT]) {
  constexpr int RT = TileCfg<T, TB>::RT, LDT = TileCfg<T, TB>::LDT;
  const int tr = (threadIdx.x / 16) * RT, tc = (threadIdx.x % 16) * RT;
#ifndef DS_KSTEP_UNROLL
#define DS_KSTEP_UNROLL 16  // measured: 16 beats 4 and 8 by 8 % and 5 % on a 32-problem batch
#endif
  constexpr int kUnroll = DS_KSTEP_UNROLL;
#pragma unroll kUnroll
  for (int m = 0; m < TB; ++m) {
    T x[RT], y[RT];
    if constexpr (RT == 4) {
      float4 xv = *reinterpret_cast<const float4*>(Pt + m * LDT + tr);
      float4 yv = *reinterpret_cast<const float4*>(Qt + m * LDT + tc);
      x[0] = xv.x; x[1] = xv.y; x[2] = xv.z; x[3] = xv.w;
      y[0] = yv.x; y[1] = yv.y; y[2] = yv.z; y[3] = yv.w;
    } else {
      double2 xv = *reinterpret_cast<const double2*>(Pt + m * LDT + tr);
      double2 yv = *reinterpret_cast<const double2*>(Qt + m * LDT + tc);
      x[0] = xv.x; x[1] = xv.y;
      y[0] = yv.x; y[1] = yv.y;
    }
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < RT; ++b) acc[a][b] += x[a] * y[b];
  }
}

// Packed tile slot of (i, k), k <= i: slot i (i + 1) / 2 + k of TB x LDT elements. Off-diagonal
// slots hold L_ik transposed (slot[m * LDT + r] = L_ik[r][m]); diagonal slots hold
// (L_kk^-1)^T in the same form (slot[m * LDT + c] = (L_kk^-1)[c][m]).
__host__ __device__ __forceinline__ size_t tile_slot(int i, int k) {
  return (size_t)i * (i + 1) / 2 + k;
}

// This thread's RT x RT block of tile (ti, tj) of A (zero outside the matrix).
template <typename T, int TB>
__device__ __forceinline__ void load_block(const T* A, int n, int ti, int tj,
                                           T (&v)[TileCfg<T, TB>::RT][TileCfg<T, TB>::RT]) {
  constexpr int RT = TileCfg<T, TB>::RT;
  const int rb = ti * TB + (threadIdx.x / 16) * RT, cb = tj * TB + (threadIdx.x % 16) * RT;
  const bool vec = rb + RT <= n && cb + RT <= n && ((n * sizeof(T)) % 16 == 0);
#pragma unroll
  for (int a = 0; a < RT; ++a) {
    const T* p = A + (size_t)(rb + a) * n + cb;
    if (vec) {
      if constexpr (RT == 4) {
        const float4 o = __ldcg(reinterpret_cast<const float4*>(p));
        v[a][0] = o.x; v[a][1] = o.y; v[a][2] = o.z; v[a][3] = o.w;
      } else {
        const double2 o = __ldcg(reinterpret_cast<const double2*>(p));
        v[a][0] = o.x; v[a][1] = o.y;
      }
    } else {
#pragma unroll
      for (int b = 0; b < RT; ++b)
        v[a][b] = (rb + a < n && cb + b < n) ? ldcg(p + b) : (T)0;
    }
  }
}

// Counters of a problem: [0, nt) diagonal tile done (L_kk, its inverse), [nt, nt + nt^2) tile
// (i, k) done (i * nt + k). Task types: 0 DIAG(j), 1 OFF(i, j), i > j.
#ifndef DS_CHOL_CTAS_PER_SM
#define DS_CHOL_CTAS_PER_SM 3  // register budget: 3 CTAs of 256 threads per SM
#endif
template <typename T, int TB>
__global__ __launch_bounds__(256, DS_CHOL_CTAS_PER_SM) void k_chol_dag(
    const ProbDesc* const* __restrict__ descs, const int2* __restrict__ tickets, int nticket,
    int* __restrict__ head, int* __restrict__ err, unsigned long long budget_ns) {
  constexpr int RT = TileCfg<T, TB>::RT, LDT = TileCfg<T, TB>::LDT, LDS = TB + 1;
  constexpr int TILE = TB * LDT;
  constexpr unsigned TBYTES = TILE * sizeof(T);
  extern __shared__ __align__(128) unsigned char smraw[];
  T* buf = reinterpret_cast<T*>(smraw);  // 4 tiles: stage 0 (P, Q), stage 1 (P, Q)
  __shared__ unsigned long long bar[2];
  __shared__ int s_t, s_ok, s_iss, s_dok;
  const int tid = threadIdx.x;
  const int tr = (tid / 16) * RT, tc = (tid % 16) * RT;
  if (tid == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};
  for (;;) {
    if (tid == 0) s_t = atomicAdd(head, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= nticket) break;
    // ticket -> (problem, task); each problem's tasks appear in their own order
    const int2 pt = tickets[t];
    if (!descs[pt.x]) {   // not in this solve
      __syncthreads();
      continue;
    }
    const LinProblem& P = descs[pt.x]->lp;
    const int4 tk = P.tasks[pt.y];
#if defined(DS_TASK_TRACE)
    if (tid == 0) ds_trace_mark(t, 0);
#endif
    const bool diag = (tk.y & 15) == 0;
    const int i = tk.z, j = tk.w, nt = P.nt, n = P.n;
    int* pdone = P.cnt;
    int* tdone = P.cnt + nt;
    T* A = (T*)P.A;
    T* Lp = (T*)P.Lp;
    const T* Li = Lp + tile_slot(i, 0) * TILE;   // row panel i (slots (i, 0..i))
    const T* Lj = Lp + tile_slot(j, 0) * TILE;
    // dependencies are read with acquire loads (the producers publish with release stores), so
    // a copy needs only the proxy fence before it
    auto ready = [&](int k) {
      return ld_acquire(&tdone[i * nt + k]) >= 1 && (diag || ld_acquire(&tdone[j * nt + k]) >= 1);
    };
    auto wait_deps = [&](int k) {
      return wait_flag(&tdone[i * nt + k], 1, err, budget_ns) &&
             (diag || wait_flag(&tdone[j * nt + k], 1, err, budget_ns));
    };
    auto issue = [&](int k, int s) {
      fence_proxy_async_global();
      T* dst = buf + 2 * s * TILE;
      mbar_expect(&bar[s], diag ? TBYTES : 2 * TBYTES);
      bulk_load(dst, Li + (size_t)k * TILE, TBYTES, &bar[s]);
      if (!diag) bulk_load(dst + TILE, Lj + (size_t)k * TILE, TBYTES, &bar[s]);
    };

    // ---- C = A_ij - sum_{k < j} L_ik L_jk^T, streamed through two stages of packed tiles
    T acc[RT][RT];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < RT; ++b) acc[a][b] = (T)0;
    const int K = j;
    if (tid == 0) {
      s_ok = *(volatile int*)err == 0;
      if (K > 0 && s_ok) {
        s_ok = wait_deps(0);
        if (s_ok) issue(0, 0);
      }
    }
    __syncthreads();
    bool ok = s_ok;
    for (int k = 0; k < K && ok; ++k) {
      const int s = k & 1;
      if (tid == 0) {
        s_iss = 0;
        if (k + 1 < K && ready(k + 1)) {
          issue(k + 1, s ^ 1);
          s_iss = 1;
        }
      }
      const bool got = mbar_wait(&bar[s], ph[s], err, budget_ns);
      ph[s] ^= 1u;
      if (__syncthreads_or(!got)) {
        // a copy did not complete in time: let any copy in flight land, then leave
        if (tid == 0) s_ok = 0;
        mbar_wait(&bar[s ^ 1], ph[s ^ 1], err, budget_ns);
        return;
      }
      const T* Pt = buf + 2 * s * TILE;
      tile_abt_acc<T, TB>(Pt, diag ? Pt : Pt + TILE, acc);
      if (tid == 0 && k + 1 < K && !s_iss) {
        s_ok = wait_deps(k + 1);
        if (s_ok) issue(k + 1, s ^ 1);
      }
      __syncthreads();
      ok = s_ok;
    }
#if defined(DS_TASK_TRACE)
    if (tid == 0) ds_trace_mark(t, 1);
#endif

    if (ok) {
      T* Ls = buf;                 // the stage buffers are free again
      T* Xs = Ls + TB * LDS;
      if (diag) {
        // ---- DIAG(j): L_jj = chol(C), X = L_jj^-1; identity padding past n
        T* Pt = Xs + TB * LDS;
        T* Dsm = Pt + 2 * RT * LDT;
        T* Tm = Dsm + 4 * RT * RT;
        const int r0 = j * TB;
        T v[RT][RT];
        load_block<T, TB>(A, n, j, j, v);
#pragma unroll
        for (int a = 0; a < RT; ++a)
#pragma unroll
          for (int b = 0; b < RT; ++b) {
            const int r = tr + a, c = tc + b;
            v[a][b] = (r0 + r < n && r0 + c < n) ? v[a][b] - acc[a][b] : (r == c ? (T)1 : (T)0);
          }
        for (int e = tid; e < TB * LDS; e += blockDim.x) Xs[e] = (T)0;
        __syncthreads();
        potrf_regs<T, TB>(v, Ls, Xs, Pt, Dsm, Tm, r0, P.status);
#if defined(DS_TASK_TRACE)
        if (tid == 0) ds_trace_mark(t, 3);
#endif
        // L_jj -> A (lower), X -> Dinv (row-major, for the solves) and X^T -> packed slot
        T* D = (T*)P.Dinv + (size_t)j * TB * TB;
        T* S = Lp + tile_slot(j, j) * TILE;
        for (int e = tid; e < TB * TB; e += blockDim.x) {
          const int r = e / TB, c = e % TB;
          __stcg(D + e, c <= r ? Xs[r * LDS + c] : (T)0);
          __stcg(S + r * LDT + c, c >= r ? Xs[c * LDS + r] : (T)0);
          if (c <= r && r0 + r < n) __stcg(A + (size_t)(r0 + r) * n + r0 + c, Ls[r * LDS + c]);
        }
      } else {
        // ---- OFF(i, j): L_ij = C (L_jj^-1)^T
        T v[RT][RT];
        load_block<T, TB>(A, n, i, j, v);
        T* Ct = buf;                // C^T
        T* Dt = buf + TILE;         // (L_jj^-1)^T, packed
        if (tid == 0) {
          s_dok = wait_flag(&pdone[j], 1, err, budget_ns);
          if (s_dok) {
            fence_proxy_async_global();
            mbar_expect(&bar[0], TBYTES);
            bulk_load(Dt, Lp + tile_slot(j, j) * TILE, TBYTES, &bar[0]);
          }
        }
#pragma unroll
        for (int a = 0; a < RT; ++a)
#pragma unroll
          for (int b = 0; b < RT; ++b) Ct[(tc + b) * LDT + tr + a] = v[a][b] - acc[a][b];
        __syncthreads();
        if (s_dok) {
          const bool got = mbar_wait(&bar[0], ph[0], err, budget_ns);
          ph[0] ^= 1u;
          if (__syncthreads_or(!got)) return;
#pragma unroll
          for (int a = 0; a < RT; ++a)
#pragma unroll
            for (int b = 0; b < RT; ++b) acc[a][b] = (T)0;
          tile_abt_acc<T, TB>(Ct, Dt, acc);
          store_block<T, TB, false>(A, n, i, j, acc, false);
          // L_ij^T -> packed slot, staged in shared memory for coalesced stores
          T* St = buf + 2 * TILE;
#pragma unroll
          for (int a = 0; a < RT; ++a)
#pragma unroll
            for (int b = 0; b < RT; ++b) St[(tc + b) * LDT + tr + a] = acc[a][b];
          __syncthreads();
          T* S = Lp + tile_slot(i, j) * TILE;
          constexpr int VE = 16 / sizeof(T);
          for (int e = tid; e < TILE / VE; e += blockDim.x) {
            if constexpr (VE == 4)
              __stcg(reinterpret_cast<float4*>(S) + e, reinterpret_cast<const float4*>(St)[e]);
            else
              __stcg(reinterpret_cast<double2*>(S) + e, reinterpret_cast<const double2*>(St)[e]);
          }
        }
      }
    }
    // generic shared writes above happen before the next task's bulk copies into the same bytes
    fence_proxy_async_shared();
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async_global();
#if defined(DS_TASK_TRACE)
      ds_trace_mark(t, 2);
#endif
      // published even when skipped after an error, so that no task waits on it
      if (diag)
        st_release(&pdone[j], 1);
      else
        st_release(&tdone[i * nt + j], 1);
    }
  }
}

template <typename T>
int chol_tile() {
  return sizeof(T) == 8 ? 32 : 64;
}
template int chol_tile<float>();
template int chol_tile<double>();

// ----------------------------------------------------------------------------- tensor-core factor

// FP32 factorisation on the 5th-generation tensor cores. The same left-looking tile tasks as
// k_chol_dag, with every 64 x 64 x 64 product done by tcgen05.mma (kind::tf32, M = N = 64,
// accumulator in tensor memory) in three terms, A_hi B_hi + A_hi B_lo + A_lo B_hi, where
// x = x_hi + x_lo with x_hi the round-to-nearest TF32 value of x: products accurate to about
// 2^-21 relative, i.e. at FP32 level for the refinement that follows.
//
// Packed slots: 8192 floats per tile, TF32 hi part then lo part, each in the canonical K-major
// layout without swizzle (core matrices of 8 rows x 16 bytes; element (r, m) at float offset
// ((r / 8) * 16 + m / 4) * 32 + (r % 8) * 4 + m % 4; K-direction core stride 128 B, row-group
// stride 2048 B). Off-diagonal slot (i, k) holds L_ik (rows r, K index m); diagonal slot (j, j)
// holds X = L_jj^-1 (rows c, K index m), the B operand of C X^T.
//
// Thread 0 runs each task's K loop alone: it waits for the producers, streams the two operand
// slots of step k into one of two shared-memory stages with bulk copies, issues the 24 MMAs and
// commits them to the stage's mbarrier, which frees the stage for step k + 2. All 256 threads
// then read the accumulator (warp w: rows 16 (w % 4) + lane for lanes < 16, columns
// 32 (w / 4) .. + 31) for the diagonal Cholesky (SIMT, potrf_regs) or for C = A_ij - acc, whose
// product with X^T is one more 3-term MMA.
#ifndef DS_TC_PROF
#define DS_TC_PROF(slot, t0)
#endif

namespace tc {

constexpr int kSlot = 8192;             // floats per packed slot (hi + lo)
constexpr unsigned kSlotBytes = 32768;
constexpr unsigned kStageBytes = 2 * kSlotBytes;
constexpr unsigned kSmem = 2 * kStageBytes;
// kind::tf32, D = F32 (bit 4), A = B = TF32 (bits 7, 10), K-major A and B, N = 64, M = 64
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((64u >> 4) << 24);

__device__ __forceinline__ int kmaj(int r, int m) {
  return ((r >> 3) * 16 + (m >> 2)) * 32 + (r & 7) * 4 + (m & 3);
}
__device__ __forceinline__ uint64_t sdesc(unsigned saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(2048 >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}
__device__ __forceinline__ void mma(unsigned tmem, uint64_t a, uint64_t b, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
// D (+)= A B^T over K = 64 for two packed slots in shared memory, three TF32 terms
__device__ __forceinline__ void mma_3x(unsigned tmem, const float* a, const float* b,
                                       bool accumulate) {
  const unsigned sa = smem_u32(a), sb = smem_u32(b);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const unsigned ah = t == 2 ? sa + 16384u : sa, bh = t == 1 ? sb + 16384u : sb;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
      mma(tmem, sdesc(ah + 256u * kk), sdesc(bh + 256u * kk),
          (accumulate || t > 0 || kk > 0) ? 1u : 0u);
  }
}
__device__ __forceinline__ void commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// this thread's 32 accumulator values (lanes >= 16 receive values of unused lanes)
__device__ __forceinline__ void tmem_read32(unsigned tmem, float (&v)[32]) {
  const int warp = threadIdx.x >> 5;
  const unsigned ta = tmem + ((unsigned)(32 * (warp & 3)) << 16) + 32u * (warp >> 2);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta + 16u * h));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[16 * h + i] = __uint_as_float(r[i]);
  }
}
// writes 4 consecutive values (row r, columns m .. m + 3, m % 4 == 0) of a tile into a packed
// slot as hi and lo parts
__device__ __forceinline__ void put4(float* slot, int r, int m, float a, float b, float c,
                                     float d) {
  const float ha = tf32_rna(a), hb = tf32_rna(b), hc = tf32_rna(c), hd = tf32_rna(d);
  const int o = kmaj(r, m);
  *reinterpret_cast<float4*>(slot + o) = make_float4(ha, hb, hc, hd);
  *reinterpret_cast<float4*>(slot + 4096 + o) = make_float4(
      tf32_rna(a - ha), tf32_rna(b - hb), tf32_rna(c - hc), tf32_rna(d - hd));
}
__device__ __forceinline__ void put4_global(float* slot, int r, int m, float a, float b, float c,
                                            float d) {
  const float ha = tf32_rna(a), hb = tf32_rna(b), hc = tf32_rna(c), hd = tf32_rna(d);
  const int o = kmaj(r, m);
  __stcg(reinterpret_cast<float4*>(slot + o), make_float4(ha, hb, hc, hd));
  __stcg(reinterpret_cast<float4*>(slot + 4096 + o),
         make_float4(tf32_rna(a - ha), tf32_rna(b - hb), tf32_rna(c - hc), tf32_rna(d - hd)));
}

}  // namespace tc

__global__ __launch_bounds__(256, 1) void k_chol_tc(const ProbDesc* const* __restrict__ descs,
                                                    const int2* __restrict__ tickets,
                                                    int nticket, int* __restrict__ head,
                                                    int* __restrict__ err,
                                                    unsigned long long budget_ns) {
  constexpr int TB = 64, LDS = TB + 1, RT = 4;
  constexpr int LDT = TileCfg<float, TB>::LDT;
  extern __shared__ __align__(1024) unsigned char smtc[];
  float* buf = reinterpret_cast<float*>(smtc);  // stage s: A slot at s * 16384, B slot + 8192
  __shared__ __align__(8) unsigned long long bcopy[2], bmma[2], bfin;
  __shared__ unsigned s_tmem;
  __shared__ int s_t, s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tr = (tid / 16) * RT, tc_ = (tid % 16) * RT;
  // accumulator coordinates of this thread (valid for lane < 16)
  const int arow = 16 * (warp & 3) + lane, acol = 32 * (warp >> 2);
  if (tid == 0) {
    mbar_init(&bcopy[0]);
    mbar_init(&bcopy[1]);
    mbar_init(&bmma[0]);
    mbar_init(&bmma[1]);
    mbar_init(&bfin);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                     smem_u32(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = s_tmem;
  unsigned cph[2] = {0u, 0u};   // thread 0: parity of the next copy wait per stage
  int mc[2] = {0, 0}, mw[2] = {0, 0};  // thread 0: commits issued / waited per stage
  unsigned fph = 0u;            // all threads: parity of the next task-level MMA wait
  for (;;) {
    if (tid == 0) s_t = atomicAdd(head, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= nticket) break;
    const int2 pt = tickets[t];
    if (!descs[pt.x]) {   // not in this solve
      __syncthreads();
      continue;
    }
    const LinProblem& P = descs[pt.x]->lp;
    const int4 tk = P.tasks[pt.y];
#if defined(DS_TASK_TRACE)
    if (tid == 0) ds_trace_mark(t, 0);
#endif
    const bool diag = (tk.y & 15) == 0;
    const int i = tk.z, j = tk.w, nt = P.nt, n = P.n;
    int* pdone = P.cnt;
    int* tdone = P.cnt + nt;
    float* A = (float*)P.A;
    float* Lp = (float*)P.Lp;
    const int K = j;
    // ---- K loop (thread 0): C = A_ij - sum_{k < j} L_ik L_jk^T accumulated in tensor memory
    if (tid == 0) {
      const float* Li = Lp + tile_slot(i, 0) * tc::kSlot;
      const float* Lj = Lp + tile_slot(j, 0) * tc::kSlot;
      auto wait_deps = [&](int k) {
        return wait_ge(&tdone[i * nt + k], 1, err, budget_ns) &&
               (diag || wait_ge(&tdone[j * nt + k], 1, err, budget_ns));
      };
      auto issue = [&](int k, int s) {
        __threadfence();
        fence_proxy_async_global();
        float* st = buf + s * 16384;
        mbar_expect(&bcopy[s], diag ? tc::kSlotBytes : 2 * tc::kSlotBytes);
        bulk_load(st, Li + (size_t)k * tc::kSlot, tc::kSlotBytes, &bcopy[s]);
        if (!diag) bulk_load(st + 8192, Lj + (size_t)k * tc::kSlot, tc::kSlotBytes, &bcopy[s]);
      };
      auto wait_mma = [&](int s) {
        const bool ok = mbar_wait(&bmma[s], (unsigned)(mw[s] & 1), err, budget_ns);
        ++mw[s];
        return ok;
      };
      bool ok = *(volatile int*)err == 0;
      int issued = 0;   // copies issued in this task; each is waited exactly once below
      if (K > 0 && ok) {
        ok = wait_deps(0);
        if (ok) {
          issue(0, 0);
          issued = 1;
        }
      }
      for (int k = 0; k < issued; ++k) {
        const int s = k & 1;
        [[maybe_unused]] long long c0 = clock64();
        const bool got = mbar_wait(&bcopy[s], cph[s], err, budget_ns);
        DS_TC_PROF(0, c0);   // waiting for the operand copies
        cph[s] ^= 1u;
        if (!got) {   // timed out (error word raised): no further copies or products
          ok = false;
          break;
        }
        tc::fence_after();
        const float* st = buf + s * 16384;
        c0 = clock64();
        tc::mma_3x(tmem, st, diag ? st : st + 8192, k > 0);
        tc::commit(&bmma[s]);
        DS_TC_PROF(1, c0);   // issuing the products
        ++mc[s];
        if (ok && k + 1 < K) {
          c0 = clock64();
          if (mw[s ^ 1] < mc[s ^ 1]) ok = wait_mma(s ^ 1);   // step k - 1 released stage s ^ 1
          DS_TC_PROF(2, c0);   // waiting for the previous step's products
          c0 = clock64();
          if (ok) ok = wait_deps(k + 1);
          DS_TC_PROF(3, c0);   // waiting for producers
          if (ok) {
            issue(k + 1, s ^ 1);
            ++issued;
          }
        }
      }
      tc::commit(&bfin);   // arrives when every product issued so far has completed
      for (int s = 0; s < 2; ++s)
        while (mw[s] < mc[s]) wait_mma(s);
      s_ok = ok;
    }
    __syncthreads();
    {
      const bool got = mbar_wait(&bfin, fph, err, budget_ns);
      fph ^= 1u;
      if (__syncthreads_or(!got)) {
        break;
      }
    }
    tc::fence_after();
#if defined(DS_TASK_TRACE)
    if (tid == 0) ds_trace_mark(t, 1);
#endif
    const bool ok = s_ok;
    float acc[32];
    if (ok && K > 0) {
      tc::tmem_read32(tmem, acc);
    } else {
#pragma unroll
      for (int e = 0; e < 32; ++e) acc[e] = 0.f;
    }
    tc::fence_before();
    __syncthreads();   // accumulator read before the stage buffers / tensor memory are reused
    if (ok) {
      float* Ls = buf;
      float* Xs = Ls + TB * LDS;
      if (diag) {
        // ---- DIAG(j): C = A_jj - acc (lower; identity padding), L_jj = chol(C), X = L_jj^-1
        float* Pt = Xs + TB * LDS;
        float* Dsm = Pt + 2 * RT * LDT;
        float* Tm = Dsm + 4 * RT * RT;
        const int r0 = j * TB;
        if (lane < 16) {
          const int r = arow;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int c = acol + e;
            float x;
            if (r0 + r < n && r0 + c < n)
              x = c <= r ? ldcg(A + (size_t)(r0 + r) * n + r0 + c) - acc[e] : 0.f;
            else
              x = (r == c) ? 1.f : 0.f;
            Ls[r * LDS + c] = x;
          }
        }
        for (int e = tid; e < TB * LDS; e += blockDim.x) Xs[e] = 0.f;
        __syncthreads();
        float v[RT][RT];
#pragma unroll
        for (int a = 0; a < RT; ++a)
#pragma unroll
          for (int b = 0; b < RT; ++b) v[a][b] = Ls[(tr + a) * LDS + tc_ + b];
        __syncthreads();
        potrf_regs<float, TB>(v, Ls, Xs, Pt, Dsm, Tm, r0, P.status);
#if defined(DS_TASK_TRACE)
        if (tid == 0) ds_trace_mark(t, 3);
#endif
        float* D = (float*)P.Dinv + (size_t)j * TB * TB;
        float* S = Lp + tile_slot(j, j) * tc::kSlot;
        for (int e = tid; e < TB * TB; e += blockDim.x) {
          const int r = e / TB, c = e % TB;
          __stcg(D + e, c <= r ? Xs[r * LDS + c] : 0.f);
          if (c <= r && r0 + r < n) __stcg(A + (size_t)(r0 + r) * n + r0 + c, Ls[r * LDS + c]);
        }
        // X in the packed K-major hi / lo form (rows c, K index m), 4 columns per thread step
        for (int e = tid; e < TB * TB / 4; e += blockDim.x) {
          const int r = e / (TB / 4), m = 4 * (e % (TB / 4));
          float x4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) x4[q] = m + q <= r ? Xs[r * LDS + m + q] : 0.f;
          tc::put4_global(S, r, m, x4[0], x4[1], x4[2], x4[3]);
        }
      } else {
        // ---- OFF(i, j): C = A_ij - acc, L_ij = C X^T with X = L_jj^-1 from slot (j, j)
        float* Cs = buf;            // C as a packed operand (hi / lo)
        float* Xp = buf + 8192;     // X slot
        if (tid == 0) {
          s_ok = wait_ge(&pdone[j], 1, err, budget_ns);
          if (s_ok) {
            __threadfence();
            fence_proxy_async_global();
            mbar_expect(&bcopy[0], tc::kSlotBytes);
            bulk_load(Xp, Lp + tile_slot(j, j) * tc::kSlot, tc::kSlotBytes, &bcopy[0]);
          }
        }
        if (lane < 16) {
          const int r = arow, rg = i * TB + r;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const int c = acol + 4 * g, cg = j * TB + c;
            float a4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              a4[q] = (rg < n && cg + q < n) ? ldcg(A + (size_t)rg * n + cg + q) - acc[4 * g + q]
                                             : 0.f;
            tc::put4(Cs, r, c, a4[0], a4[1], a4[2], a4[3]);
          }
        }
        fence_proxy_async_shared();
        __syncthreads();
        const bool dok = s_ok;
        if (dok) {
          if (tid == 0) {
            const bool got = mbar_wait(&bcopy[0], cph[0], err, budget_ns);
            cph[0] ^= 1u;
            if (got) {
              tc::fence_after();
              tc::mma_3x(tmem, Cs, Xp, false);
            }
            tc::commit(&bfin);
          }
          const bool got = mbar_wait(&bfin, fph, err, budget_ns);
          fph ^= 1u;
          if (__syncthreads_or(!got)) {
            break;
          }
          tc::fence_after();
          float l[32];
          tc::tmem_read32(tmem, l);
          tc::fence_before();
          if (lane < 16) {
            const int r = arow, rg = i * TB + r;
            float* S = Lp + tile_slot(i, j) * tc::kSlot;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              const int c = acol + 4 * g, cg = j * TB + c;
              if (rg < n) {
                if (cg + 3 < n && (n & 3) == 0) {
                  __stcg(reinterpret_cast<float4*>(A + (size_t)rg * n + cg),
                         make_float4(l[4 * g], l[4 * g + 1], l[4 * g + 2], l[4 * g + 3]));
                } else {
#pragma unroll
                  for (int q = 0; q < 4; ++q)
                    if (cg + q < n) __stcg(A + (size_t)rg * n + cg + q, l[4 * g + q]);
                }
              }
              tc::put4_global(S, r, c, l[4 * g], l[4 * g + 1], l[4 * g + 2], l[4 * g + 3]);
            }
          }
        }
      }
    }
    // generic shared writes above happen before the next task's bulk copies into the same bytes
    fence_proxy_async_shared();
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      fence_proxy_async_global();
#if defined(DS_TASK_TRACE)
      ds_trace_mark(t, 2);
#endif
      if (diag)
        atomicExch(&pdone[j], 1);
      else
        atomicExch(&tdone[i * nt + j], 1);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  }
}

// ----------------------------------------------------------------------------- 128-block tensor-core factor

// FP32 factorisation on the tensor cores with 128 x 128 blocks: the same left-looking scheme as
// k_chol_dag, one task per output block, in block-column order:
//   DIAG(J)     C = A_JJ - sum_{k<J} L_Jk L_Jk^T;  L_JJ = chol(C), X_JJ = L_JJ^-1
//   OFF(I, J)   C = A_IJ - sum_{k<J} L_Ik L_Jk^T;  L_IJ = C X_JJ^T                (I > J)
// Every block product is a tcgen05.mma chain with M = N = 128 (kind::tf32, 3 terms per product:
// a_hi b_hi + a_hi b_lo + a_lo b_hi, x = x_hi + x_lo with x_hi the round-to-nearest TF32 value of
// x, so each product is accurate to about 2^-21 relative: FP32 level for the refinement steps).
// The 128 x 128 accumulator lives in tensor memory (128 lanes x 128 columns).
//
// Packed block slots (one per finished block (I, J), J <= I): 128 rows x 128 K values as eight
// K sub-chunks of 16; sub-chunk q holds the TF32 hi part (2048 floats) then the lo part (2048
// floats), each in the canonical K-major layout without swizzle: core matrices of 8 rows x 4
// floats (128 B), element (r, m) of the sub-chunk at ((r / 8) * 4 + m / 4) * 32 + (r % 8) * 4 +
// m % 4, i.e. 128 B between core matrices along K and 512 B between 8-row groups. Slot (I, J),
// I > J, holds L_IJ (row r, K index = column); slot (J, J) holds X_JJ (row c, K index m), the B
// operand of C X^T.
//
// Thread 0 streams the operand sub-chunks of a product through 192 KB of shared memory in
// stages of G sub-chunks of A and G of B (G = 2: three 64 KB stages; G = 1: six 32 KB stages;
// the tuner times both), issues a stage's 6 G MMAs as soon as its bulk copies land and refills
// the stage of the previous one once that stage's MMAs have completed (tcgen05.commit on the
// stage's mbarrier), so the tensor pipe always has the next stage queued. The diagonal block is
// factored on the SIMT pipes from the accumulator in 64 x 64 halves (potrf_regs), with its
// 128 x 128 inverse by X10 = -X11 (L10 X00). An off-diagonal block's C = A_IJ - acc is split
// into hi / lo parts in shared memory (128 KB, the A operand of C X_JJ^T) while X_JJ streams
// through the remaining 64 KB in four 16 KB stages. The finished blocks are written to A
// (row-major, for the triangular solves) and to the packed slots; the diagonal 64 x 64 inverses
// go to Dinv for the solves.
namespace tcb {

constexpr int BS = 128;                   // block size
constexpr int KS = 16;                    // K per sub-chunk
constexpr int kPart = BS * KS;            // floats of one part (hi or lo) of a sub-chunk
constexpr int kSub = 2 * kPart;           // floats of a sub-chunk (hi + lo)
constexpr int kSlot = (BS / KS) * kSub;   // floats per slot (8 sub-chunks)
constexpr unsigned kSubBytes = kSub * 4u;            // 16 KB
constexpr unsigned kSmem = 192u * 1024u;             // stage area
constexpr unsigned kCBytes = (BS / KS) * kSubBytes;  // 128 KB: the C operand of the OFF product
constexpr int kXStages = 4;                          // 16 KB stages of X after the C operand
// kind::tf32, D = F32, A = B = TF32, both K-major, N = 128, M = 128
constexpr unsigned kIdesc =
    (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
// the same with N = 256 (two 128-row B blocks as one operand, D over 256 TMEM columns)
constexpr unsigned kIdesc256 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__host__ __device__ __forceinline__ size_t slot(int i, int j) { return (size_t)i * (i + 1) / 2 + j; }
// offset of element (r, k) of a block (row r, K index k) in its slot (hi part; lo at + kPart)
__device__ __forceinline__ int soff(int r, int k) {
  return (k >> 4) * kSub + (((r >> 3) * 4 + ((k & 15) >> 2)) * 32 + (r & 7) * 4 + (k & 3));
}
__device__ __forceinline__ uint64_t sdesc(unsigned saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma(unsigned tmem, uint64_t a, uint64_t b, unsigned acc,
                                    unsigned idesc = kIdesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// D (256 columns) (+)= A [B0; B1]^T over one sub-chunk: A at sa (hi, lo parts), the two B
// blocks interleaved at sb as [B0 hi][B1 hi][B0 lo][B1 lo] (one 256-row operand per part)
__device__ __forceinline__ void mma_sub256(unsigned tmem, unsigned sa, unsigned sb,
                                           bool accumulate) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const unsigned ah = t == 2 ? sa + kPart * 4u : sa, bh = t == 1 ? sb + kPart * 8u : sb;
#pragma unroll
    for (int kk = 0; kk < KS / 8; ++kk)
      mma(tmem, sdesc(ah + 256u * kk), sdesc(bh + 256u * kk),
          (accumulate || t > 0 || kk > 0) ? 1u : 0u, kIdesc256);
  }
}
// D (+)= A B^T over the 16 K values of one sub-chunk pair (A at sa, B at sb; hi then lo parts)
__device__ __forceinline__ void mma_sub(unsigned tmem, unsigned sa, unsigned sb, bool accumulate) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const unsigned ah = t == 2 ? sa + kPart * 4u : sa, bh = t == 1 ? sb + kPart * 4u : sb;
#pragma unroll
    for (int kk = 0; kk < KS / 8; ++kk)
      mma(tmem, sdesc(ah + 256u * kk), sdesc(bh + 256u * kk),
          (accumulate || t > 0 || kk > 0) ? 1u : 0u);
  }
}
// 32 consecutive accumulator columns of this thread's lane (row)
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// This thread's 64 accumulator values: row 32 (warp % 4) + lane, columns 64 (warp / 4) + 0..63.
__device__ __forceinline__ void tmem_row64(unsigned tmem, float (&v)[64]) {
  const int warp = threadIdx.x >> 5;
  const unsigned ta = tmem + ((unsigned)(32 * (warp & 3)) << 16) + 64u * (warp >> 2);
  float h[32];
  tmem_ld32(ta, h);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = h[i];
  tmem_ld32(ta + 32u, h);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[32 + i] = h[i];
}
// four consecutive values (row r, K index k..k+3, k % 4 == 0) of a block into a slot layout,
// in global memory (slot) or shared memory (the C operand)
__device__ __forceinline__ void put4(float* slot, int r, int k, float a, float b, float c, float d) {
  const float ha = tc::tf32_rna(a), hb = tc::tf32_rna(b), hc = tc::tf32_rna(c),
              hd = tc::tf32_rna(d);
  const int o = soff(r, k);
  __stcg(reinterpret_cast<float4*>(slot + o), make_float4(ha, hb, hc, hd));
  __stcg(reinterpret_cast<float4*>(slot + kPart + o),
         make_float4(tc::tf32_rna(a - ha), tc::tf32_rna(b - hb), tc::tf32_rna(c - hc),
                     tc::tf32_rna(d - hd)));
}
__device__ __forceinline__ void put4_smem(float* base, int r, int k, float a, float b, float c,
                                          float d) {
  const float ha = tc::tf32_rna(a), hb = tc::tf32_rna(b), hc = tc::tf32_rna(c),
              hd = tc::tf32_rna(d);
  const int o = soff(r, k);
  *reinterpret_cast<float4*>(base + o) = make_float4(ha, hb, hc, hd);
  *reinterpret_cast<float4*>(base + kPart + o) =
      make_float4(tc::tf32_rna(a - ha), tc::tf32_rna(b - hb), tc::tf32_rna(c - hc),
                  tc::tf32_rna(d - hd));
}

// Stage ring of thread 0, kept across tasks so the barrier phases stay in step: NS stages of
// `bytes` each at smem offset `base`; cph = parity of the next copy completion, mc / mw = MMA
// commits issued / waited per stage.
template <int NS>
struct Ring {
  unsigned long long copy[NS], mma[NS];
  unsigned cph[NS];
  int mc[NS], mw[NS];
};

// Thread 0: the copies of chunk c into its stage of the ring (A, B, B2 from global at pa(c),
// pb(c), pb2(c) where not nullptr, in that order), after the stage's previous products are done
// with it and dep(c) holds. False if a wait gave up (nothing of chunk c issued then).
template <int NS, int G, int NOPS, typename PA, typename PB, typename PB2, typename DEP>
__device__ bool issue_chunk(int c, unsigned stg, Ring<NS>& rg, PA& pa, PB& pb, PB2& pb2, DEP& dep,
                            int* err, unsigned long long budget) {
  constexpr unsigned kChunkBytes = G * kSubBytes;
  constexpr unsigned kStage = NOPS * kChunkBytes;
  const int s = c % NS;
  while (rg.mw[s] < rg.mc[s]) {   // the stage's previous MMAs are done with it
    const bool g = mbar_wait(&rg.mma[s], (unsigned)(rg.mw[s] & 1), err, budget);
    ++rg.mw[s];
    if (!g) return false;
  }
  if (!dep(c)) return false;   // dep(c) orders the copies after what it acquired (proxy fence)
  const float* a = pa(c);
  const float* b = pb(c);
  const float* b2 = pb2(c);
  const unsigned nops = (a ? 1u : 0u) + (b ? 1u : 0u) + (b2 ? 1u : 0u);
  unsigned d = stg + s * kStage;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(&rg.copy[s])),
               "r"(nops * kChunkBytes)
               : "memory");
  auto copy = [&](unsigned dst, const float* src) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"(src), "r"(kChunkBytes), "r"(smem_u32(&rg.copy[s]))
        : "memory");
  };
  if (a) {
    copy(d, a);
    d += kChunkBytes;
  }
  if (b) {
    copy(d, b);
    d += kChunkBytes;
  }
  if (b2) copy(d, b2);
  return true;
}

// Thread 0: issues the first min(NS, nck) chunks of a stream ahead of its products (so that the
// copies overlap other work of the CTA); returns how many were issued. After a failed wait the
// copies already issued are waited for (bounded) and -1 is returned.
template <int NS, int G, int NOPS, typename PA, typename PB, typename PB2, typename DEP>
__device__ int prime(unsigned stg, Ring<NS>& rg, int nck, PA pa, PB pb, PB2 pb2, DEP dep,
                     int* err, unsigned long long budget) {
  int issued = 0;
  while (issued < nck && issued < NS) {
    if (!issue_chunk<NS, G, NOPS>(issued, stg, rg, pa, pb, pb2, dep, err, budget)) {
      for (int c = 0; c < issued; ++c) {
        mbar_wait(&rg.copy[c % NS], rg.cph[c % NS], err, budget);
        rg.cph[c % NS] ^= 1u;
      }
      return -1;
    }
    ++issued;
  }
  return issued;
}

// Thread 0: D = sum_{c < nck} A_c B_c^T over chunks c of G sub-chunks each (and, with a second
// B operand, D2 = sum_c A_c B2_c^T into tmem2). A_c: from global at pa(c) (G sub-chunks,
// contiguous) into the stage, or, with pa(c) == nullptr, resident in shared memory at
// sa_res(c); B_c: from global at pb(c), or (pb(c) == nullptr) the stage's A; B2_c: from global
// at pb2(c) when not nullptr. A stage holds up to NOPS chunks, [A][B][B2]. The first `pre`
// chunks were issued by prime(). The first product starts the accumulators afresh unless
// acc_first. dep(c) is waited before the copies of chunk c. Every issued copy is waited exactly
// once and every commit is waited before return, so the phases stay in step; bfin is committed
// after the last MMA. False if a wait gave up (error word raised); the accumulators are then not
// meaningful.
template <int NS, int G, int NOPS, typename PA, typename RA, typename PB, typename PB2,
          typename DEP>
__device__ bool stream(unsigned tmem, unsigned tmem2, unsigned stg, Ring<NS>& rg,
                       unsigned long long* bfin, int nck, int pre, bool acc_first, PA pa,
                       RA sa_res, PB pb, PB2 pb2, DEP dep, int* err, unsigned long long budget) {
  constexpr unsigned kChunkBytes = G * kSubBytes;
  constexpr unsigned kStage = NOPS * kChunkBytes;
  bool ok = true;
  int issued = pre;
  auto issue = [&](int c) {
    return issue_chunk<NS, G, NOPS>(c, stg, rg, pa, pb, pb2, dep, err, budget);
  };
  while (ok && issued < nck && issued < NS) {
    ok = issue(issued);
    if (ok) ++issued;
  }
  for (int c = 0; c < issued; ++c) {
    const int s = c % NS;
    const bool got = mbar_wait(&rg.copy[s], rg.cph[s], err, budget);
    rg.cph[s] ^= 1u;
    if (!got) ok = false;
    if (ok) {
      tc::fence_after();
      const bool a_st = pa(c) != nullptr, b_st = pb(c) != nullptr, b2_st = pb2(c) != nullptr;
      const unsigned d = stg + s * kStage;
      const unsigned sa = a_st ? d : sa_res(c);
      const unsigned sb = b_st ? d + (a_st ? kChunkBytes : 0u) : sa;
      const unsigned sb2 = d + ((a_st ? 1u : 0u) + (b_st ? 1u : 0u)) * kChunkBytes;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const bool acc = acc_first || c > 0 || g > 0;
        mma_sub(tmem, sa + g * kSubBytes, sb + g * kSubBytes, acc);
        if (b2_st) mma_sub(tmem2, sa + g * kSubBytes, sb2 + g * kSubBytes, acc);
      }
      tc::commit(&rg.mma[s]);
      ++rg.mc[s];
      if (c >= 1 && issued < nck) {   // refill the stage chunk c - 1 used
        ok = issue(issued);
        if (ok) ++issued;
      }
    }
  }
  tc::commit(bfin);
  for (int s = 0; s < NS; ++s)
    while (rg.mw[s] < rg.mc[s]) {
      mbar_wait(&rg.mma[s], (unsigned)(rg.mw[s] & 1), err, budget);
      ++rg.mw[s];
    }
  return ok;
}

// A K-loop ring whose copies (one producer thread) and products (one consumer thread) run
// decoupled: full[s] completes when the copies into stage s have landed, empty[s] when the
// products that read it are done. Chunk c of a loop is the ring's (pos + c)-th use overall (pos:
// the chunks through the ring before, counted alike by both threads). pdone / nissued: set only
// when the producer stops short of a loop's end, with the ring position it got to.
template <int NS>
struct WRing {
  unsigned long long full[NS], empty[NS];
  int nissued, pdone;
};

template <int NS>
__device__ __forceinline__ void wring_init(WRing<NS>& r) {
  for (int s = 0; s < NS; ++s) {
    mbar_init(&r.full[s]);
    mbar_init(&r.empty[s]);
  }
  r.nissued = 0;
  r.pdone = 0;
}

// Producer: for c < nck, once the stage's previous products are done and dep(c) holds, the
// copies of chunk c (A, B, B2 from global at pa(c), pb(c), pb2(c) where not nullptr) into its
// stage; with IL (G = 1) B and B2 go in interleaved, [B hi][B2 hi][B lo][B2 lo], as one 256-row
// operand. Stops early (and says so in pdone / nissued) if a wait gives up or the error word is
// raised.
template <int NS, int G, int NOPS, bool IL = false, typename PA, typename PB, typename PB2,
          typename DEP>
__device__ void ws_produce(unsigned stg, WRing<NS>& r, unsigned pos, int nck, PA pa, PB pb,
                           PB2 pb2, DEP dep, int* err, unsigned long long budget) {
  constexpr unsigned kChunkBytes = G * kSubBytes;
  constexpr unsigned kStage = NOPS * kChunkBytes;
  int c = 0;
  if (*(volatile int*)err == 0) {
    for (; c < nck; ++c) {
      const unsigned q = pos + (unsigned)c, s = q % NS, g = q / NS;
      if (g >= 1 && !mbar_wait(&r.empty[s], (g - 1) & 1u, err, budget)) break;
      if (!dep(c)) break;
      const float* a = pa(c);
      const float* b = pb(c);
      const float* b2 = pb2(c);
      const unsigned nops = (a ? 1u : 0u) + (b ? 1u : 0u) + (b2 ? 1u : 0u);
      unsigned d = stg + s * kStage;
      const unsigned bar = smem_u32(&r.full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(nops * kChunkBytes)
                   : "memory");
      auto copy = [&](unsigned dst, const float* src) {
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(dst),
            "l"(src), "r"(kChunkBytes), "r"(bar)
            : "memory");
      };
      if (a) {
        copy(d, a);
        d += kChunkBytes;
      }
      if constexpr (IL) {
        static_assert(G == 1, "interleaved pairs take one sub-chunk per stage");
        constexpr unsigned kHalf = kChunkBytes / 2;
        auto copy_half = [&](unsigned dst, const float* src) {
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
              "[%3];" ::"r"(dst),
              "l"(src), "r"(kHalf), "r"(bar)
              : "memory");
        };
        copy_half(d, b);
        copy_half(d + kHalf, b2);
        copy_half(d + 2 * kHalf, b + kPart);
        copy_half(d + 3 * kHalf, b2 + kPart);
      } else {
        if (b) {
          copy(d, b);
          d += kChunkBytes;
        }
        if (b2) copy(d, b2);
      }
    }
  }
  if (c < nck) {
    *(volatile int*)&r.nissued = (int)pos + c;
    __threadfence_block();
    *(volatile int*)&r.pdone = 1;
  }
}

// Consumer: D (+)= sum_c A_c B_c^T (and D2 with B2 into tmem2) over the chunks as their copies
// land, each stage released to the producer by a commit on empty[s]; bfin is committed after the
// last product. If the producer stopped short, the chunks it did issue are waited for and
// released, and false is returned (the accumulators are then not meaningful).
template <int NS, int G, int NOPS, bool IL = false, typename PA, typename PB, typename PB2>
__device__ bool ws_consume(unsigned tmem, unsigned tmem2, unsigned stg, WRing<NS>& r,
                           unsigned pos, unsigned long long* bfin, int nck, PA pa, PB pb,
                           PB2 pb2, int* err, unsigned long long budget) {
  constexpr unsigned kChunkBytes = G * kSubBytes;
  constexpr unsigned kStage = NOPS * kChunkBytes;
  const volatile int* vdone = &r.pdone;
  const volatile int* vn = &r.nissued;
  bool ok = true;
  int c = 0;
  for (; c < nck; ++c) {
    const unsigned q = pos + (unsigned)c, s = q % NS, g = q / NS;
    bool got = mbar_test(&r.full[s], g & 1u);
    if (!got) {
      const unsigned long long t0 = globaltimer();
      for (;;) {
        if (mbar_test(&r.full[s], g & 1u)) {
          got = true;
          break;
        }
        if (*vdone && (int)pos + c >= *vn) break;   // the producer stopped before chunk c
        if (globaltimer() - t0 > budget) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    if (!got) {
      ok = false;
      break;
    }
    tc::fence_after();
    const bool a_st = pa(c) != nullptr, b_st = pb(c) != nullptr, b2_st = pb2(c) != nullptr;
    const unsigned d = stg + s * kStage;
    const unsigned sa = d;
    const unsigned sb = b_st ? d + (a_st ? kChunkBytes : 0u) : sa;
    const unsigned sb2 = d + ((a_st ? 1u : 0u) + (b_st ? 1u : 0u)) * kChunkBytes;
    if constexpr (IL) {
      mma_sub256(tmem, sa, sb, c > 0);   // tmem2 = tmem + 128 holds the B2 half of D
      (void)sb2;
      (void)tmem2;
    } else {
#pragma unroll
      for (int gg = 0; gg < G; ++gg) {
        const bool acc = c > 0 || gg > 0;
        mma_sub(tmem, sa + gg * kSubBytes, sb + gg * kSubBytes, acc);
        if (b2_st) mma_sub(tmem2, sa + gg * kSubBytes, sb2 + gg * kSubBytes, acc);
      }
    }
    tc::commit(&r.empty[s]);
  }
  if (!ok) {
    // the producer's last word, then its chunks past c: wait for their copies, release stages
    const unsigned long long t0 = globaltimer();
    while (!*vdone && globaltimer() - t0 <= budget) {
    }
    const int n_iss = *vdone ? *vn - (int)pos : c;
    for (int k = c; k < n_iss; ++k) {
      const unsigned q = pos + (unsigned)k, s = q % NS, g = q / NS;
      mbar_wait(&r.full[s], g & 1u, err, budget);
      mbar_arrive(&r.empty[s]);
    }
  }
  tc::commit(bfin);
  return ok;
}

// The same producer / consumer pair for two rows and two block columns: stage
// [A0][A1][B0 hi][B1 hi][B0 lo][B1 lo] (64 KB), products A0 [B0; B1]^T into D0 (256 TMEM
// columns at tmem) and A1 [B0; B1]^T into D1 (at tmem + 256), one N = 256 MMA per term each.
template <int NS, typename PA, typename PA2, typename PB, typename PB2, typename DEP>
__device__ void ws_produce4(unsigned stg, WRing<NS>& r, unsigned pos, int nck, PA pa, PA2 pa2,
                            PB pb, PB2 pb2, DEP dep, int* err, unsigned long long budget) {
  constexpr unsigned kStage = 4 * kSubBytes, kHalf = kSubBytes / 2;
  int c = 0;
  if (*(volatile int*)err == 0) {
    for (; c < nck; ++c) {
      const unsigned q = pos + (unsigned)c, s = q % NS, g = q / NS;
      if (g >= 1 && !mbar_wait(&r.empty[s], (g - 1) & 1u, err, budget)) break;
      if (!dep(c)) break;
      const unsigned d = stg + s * kStage, bar = smem_u32(&r.full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(kStage)
                   : "memory");
      auto copy = [&](unsigned dst, const float* src, unsigned bytes) {
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(dst),
            "l"(src), "r"(bytes), "r"(bar)
            : "memory");
      };
      const float* b = pb(c);
      const float* b2 = pb2(c);
      copy(d, pa(c), kSubBytes);
      copy(d + kSubBytes, pa2(c), kSubBytes);
      copy(d + 2 * kSubBytes, b, kHalf);
      copy(d + 2 * kSubBytes + kHalf, b2, kHalf);
      copy(d + 3 * kSubBytes, b + kPart, kHalf);
      copy(d + 3 * kSubBytes + kHalf, b2 + kPart, kHalf);
    }
  }
  if (c < nck) {
    *(volatile int*)&r.nissued = (int)pos + c;
    __threadfence_block();
    *(volatile int*)&r.pdone = 1;
  }
}

template <int NS>
__device__ bool ws_consume4(unsigned tmem, unsigned stg, WRing<NS>& r, unsigned pos,
                            unsigned long long* bfin, int nck, int* err,
                            unsigned long long budget) {
  constexpr unsigned kStage = 4 * kSubBytes;
  const volatile int* vdone = &r.pdone;
  const volatile int* vn = &r.nissued;
  bool ok = true;
  int c = 0;
  for (; c < nck; ++c) {
    const unsigned q = pos + (unsigned)c, s = q % NS, g = q / NS;
    bool got = mbar_test(&r.full[s], g & 1u);
    if (!got) {
      const unsigned long long t0 = globaltimer();
      for (;;) {
        if (mbar_test(&r.full[s], g & 1u)) {
          got = true;
          break;
        }
        if (*vdone && (int)pos + c >= *vn) break;   // the producer stopped before chunk c
        if (globaltimer() - t0 > budget) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    if (!got) {
      ok = false;
      break;
    }
    tc::fence_after();
    const unsigned d = stg + s * kStage;
    mma_sub256(tmem, d, d + 2 * kSubBytes, c > 0);
    mma_sub256(tmem + 256u, d + kSubBytes, d + 2 * kSubBytes, c > 0);
    tc::commit(&r.empty[s]);
  }
  if (!ok) {
    const unsigned long long t0 = globaltimer();
    while (!*vdone && globaltimer() - t0 <= budget) {
    }
    const int n_iss = *vdone ? *vn - (int)pos : c;
    for (int k = c; k < n_iss; ++k) {
      const unsigned q = pos + (unsigned)k, s = q % NS, g = q / NS;
      mbar_wait(&r.full[s], g & 1u, err, budget);
      mbar_arrive(&r.empty[s]);
    }
  }
  tc::commit(bfin);
  return ok;
}

template <int NS>
__device__ __forceinline__ void ring_init(Ring<NS>& rg) {
  for (int s = 0; s < NS; ++s) {
    mbar_init(&rg.copy[s]);
    mbar_init(&rg.mma[s]);
    rg.cph[s] = 0u;
    rg.mc[s] = rg.mw[s] = 0;
  }
}

}  // namespace tcb

// Every K loop runs on two threads: thread 32 issues the bulk copies of the operand stages,
// thread 0 the MMAs, linked by full / empty mbarriers per stage (WRing).
// G: sub-chunks per operand per stage of the single-block K loop (stages of 2 G x 16 KB, 6 / G of
// them). PAIRS: block columns are taken two at a time (J0 = 2 p, J1 = 2 p + 1): DIAG(J0),
// OFF(J1, J0), DIAG(J1), then OFF2(I; J0, J1) for every row block I below, which accumulates
// the two blocks (I, J0) and (I, J1) over k < J0 with one stream of the A operand L_Ik (stages
// [L_Ik][L_J0k, L_J1k interleaved] of 48 KB, one N = 256 MMA per term into 256 TMEM columns),
// finishes (I, J0), adds the k = J0 term L_IJ0 L_J1J0^T to the second accumulator from the
// just-finished block held in shared memory, and finishes (I, J1): the row panel I is read once
// per two block columns instead of once per column. With quads (the task list of two rows x two
// columns), OFF4(I; J0, J1) does the same for the rows I and I + 1 at once (stages
// [L_Ik][L_I+1,k][L_J0k, L_J1k] of 64 KB, four accumulators over all 512 TMEM columns), so that
// the column panels are also read once per two rows.
template <int G, bool PAIRS>
__global__ __launch_bounds__(256, 1) void k_chol_tcb(const ProbDesc* const* __restrict__ descs,
                                                     const int2* __restrict__ tickets,
                                                     int nticket, int* __restrict__ head,
                                                     int* __restrict__ err,
                                                     unsigned long long budget_ns, int quads) {
  using namespace tcb;
  constexpr int NS = 6 / G;
  constexpr int TB = 64, LDS = TB + 1, RT = 4;
  constexpr int LDC = BS + 1;
  constexpr unsigned kTmemCols = PAIRS ? 512u : 128u;
  extern __shared__ __align__(1024) unsigned char smb[];
  float* sm = reinterpret_cast<float*>(smb);
  __shared__ __align__(8) unsigned long long s_bfin;
  __shared__ unsigned s_tmem;
  __shared__ int s_t, s_ok, s_pre;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tr = (tid / 16) * RT, tcl = (tid % 16) * RT;      // 64 x 64 register blocks
  const int arow = 32 * (warp & 3) + lane, acol = 64 * (warp >> 2);   // accumulator ownership
  // stage rings of thread 0 (barriers and their phase counters, used by thread 0 only)
  __shared__ __align__(8) WRing<NS> wring_k;        // single-block K-loop stages
  __shared__ __align__(8) Ring<kXStages> ring_x;    // stages of the products with a resident A
  __shared__ __align__(8) WRing<4> wring_p;         // paired K-loop stages (48 KB)
  __shared__ __align__(8) WRing<3> wring_q;         // K-loop stages of two rows x two columns
  unsigned long long* bfin = &s_bfin;
  if (tid == 0) {
    wring_init(wring_k);
    ring_init(ring_x);
    wring_init(wring_p);
    wring_init(wring_q);
    mbar_init(bfin);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = s_tmem;
  const unsigned stg = smem_u32(smb);
  unsigned fph = 0u;   // parity of the next bfin completion (all threads)
  float* Cs = sm;      // OFF epilogue: the C (or L) operand, 8 sub-chunks (128 KB)
  float* Tb = sm;      // a 128 x 128 FP32 block, swizzled (first 64 KB, before / after Cs is used)
  // Every thread: wait for thread 0's products (bfin) when it streamed; false if any thread saw
  // a failure (then the CTA leaves its ticket loop).
  auto join = [&](bool streamed) {
    bool bad = !s_ok;
    if (streamed) {
      const bool got = mbar_wait(bfin, fph, err, budget_ns);
      fph ^= 1u;
      bad = bad || !got;
    }
    return !__syncthreads_or(bad);
  };
  // Row-major 128 x 128 FP32 block in shared memory with its float4 groups permuted by row & 7:
  // whole rows (a warp, float2 per lane) and row segments (the row's owner thread, float4) are
  // then both conflict-free.
  auto tpos = [](int r, int c) { return r * BS + ((((c >> 2) ^ (r & 7)) << 2) | (c & 3)); };
  // A block (rows I BS.., columns Jx BS..) into registers with coalesced loads: warp w takes
  // rows 16 w .. 16 w + 15, lane l columns 2 l, 2 l + 1, 64 + 2 l, 65 + 2 l (zero past n; n even)
  auto load_rows = [&](const float* A, int n, int I, int Jx, float (&a)[64]) {
    const int c0 = Jx * BS + 2 * lane;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = I * BS + 16 * warp + q;
      float2 p0 = make_float2(0.f, 0.f), p1 = p0;
      if (r < n) {
        const float* row = A + (size_t)r * n;
        if (c0 < n) p0 = __ldcg(reinterpret_cast<const float2*>(row + c0));
        if (c0 + 64 < n) p1 = __ldcg(reinterpret_cast<const float2*>(row + c0 + 64));
      }
      a[4 * q] = p0.x;
      a[4 * q + 1] = p0.y;
      a[4 * q + 2] = p1.x;
      a[4 * q + 3] = p1.y;
    }
  };
  // the registers of load_rows -> Tb
  auto stage_rows = [&](const float (&a)[64]) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = 16 * warp + q;
      *reinterpret_cast<float2*>(Tb + tpos(r, 2 * lane)) = make_float2(a[4 * q], a[4 * q + 1]);
      *reinterpret_cast<float2*>(Tb + tpos(r, 64 + 2 * lane)) =
          make_float2(a[4 * q + 2], a[4 * q + 3]);
    }
  };
  // C = A_block - v (A_block staged in Tb; zero on rows past n) as the hi / lo A operand in Cs;
  // v is overwritten with C
  auto form_c = [&](int n, int I, float (&v)[64]) {
    const bool in = I * BS + arow < n;
#pragma unroll
    for (int e = 0; e < 64; e += 4) {
      const float4 t = *reinterpret_cast<const float4*>(Tb + tpos(arow, acol + e));
      v[e] = in ? t.x - v[e] : 0.f;
      v[e + 1] = in ? t.y - v[e + 1] : 0.f;
      v[e + 2] = in ? t.z - v[e + 2] : 0.f;
      v[e + 3] = in ? t.w - v[e + 3] : 0.f;
    }
    __syncthreads();   // Tb read before Cs (which covers it) is written
#pragma unroll
    for (int e = 0; e < 64; e += 4)
      tcb::put4_smem(Cs, arow, acol + e, v[e], v[e + 1], v[e + 2], v[e + 3]);
    fence_proxy_async_shared();
  };
  auto no_src = [](int) -> const float* { return nullptr; };
  // after flags were acquired: the copies (async proxy) that follow see the data they guard
  auto acquired = [](bool ok) {
    fence_proxy_async_global();
    return ok;
  };
  auto res_a = [&](int c) { return stg + (unsigned)c * kSubBytes; };
  // thread 0: the first stages of D (+)= [resident A in Cs] B^T, B = 8 sub-chunks at src, issued
  // after flag (overlapping the copies with the CTA's epilogue work); returns the count or -1
  auto prime_product = [&](const float* src, const int* flag) {
    return prime<kXStages, 1, 1>(
        stg + kCBytes, ring_x, BS / KS, no_src,
        [&](int c) -> const float* { return src + (size_t)c * kSub; }, no_src,
        [&](int c) { return c > 0 || acquired(wait_flag(flag, 1, err, budget_ns)); }, err,
        budget_ns);
  };
  // thread 0: D (at tm) (+)= [resident A in Cs] B^T, the first `pre` stages already issued
  auto resident_product = [&](unsigned tm, const float* src, bool acc_first, const int* flag,
                              int pre) {
    return stream<kXStages, 1, 1>(
        tm, 0u, stg + kCBytes, ring_x, bfin, BS / KS, pre, acc_first, no_src, res_a,
        [&](int c) -> const float* { return src + (size_t)c * kSub; }, no_src,
        [&](int c) { return c > 0 || acquired(wait_flag(flag, 1, err, budget_ns)); }, err,
        budget_ns);
  };
  // L block v -> A (row-major, through Tb: coalesced rows) and its slot
  auto write_block = [&](float* A, float* Lp, int n, int I, int Jx, const float (&v)[64]) {
#pragma unroll
    for (int e = 0; e < 64; e += 4)
      *reinterpret_cast<float4*>(Tb + tpos(arow, acol + e)) =
          make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
    float* S = Lp + slot(I, Jx) * kSlot;
#pragma unroll
    for (int e = 0; e < 64; e += 4)
      tcb::put4(S, arow, acol + e, v[e], v[e + 1], v[e + 2], v[e + 3]);
    __syncthreads();
    const int c0 = Jx * BS + 2 * lane;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = 16 * warp + q, rg = I * BS + r;
      if (rg < n) {
        float* row = A + (size_t)rg * n;
        __stcg(reinterpret_cast<float2*>(row + c0),
               *reinterpret_cast<const float2*>(Tb + tpos(r, 2 * lane)));
        __stcg(reinterpret_cast<float2*>(row + c0 + 64),
               *reinterpret_cast<const float2*>(Tb + tpos(r, 64 + 2 * lane)));
      }
    }
  };
  auto publish = [&](int* f) {
    fence_proxy_async_shared();
    fence_proxy_async_global();
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(f, 1);
    }
  };
  // A wait that gives up raises the error word; every CTA then leaves its ticket loop (after its
  // copies and products in flight have completed), and the host reports DS_ERR_TIMEOUT.
  // K loops: thread 32 issues the copies, thread 0 the products; pos_*: chunks through each ring
  unsigned pos_k = 0u, pos_p = 0u, pos_q = 0u;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(head, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= nticket) break;
    const int2 pt = tickets[t];
    if (!descs[pt.x]) {   // not in this solve
      __syncthreads();
      continue;
    }
    const LinProblem& P = descs[pt.x]->lp;
    const int4 tk = PAIRS ? (quads ? P.tasks_q[pt.y] : P.tasks_p[pt.y]) : P.tasks_b[pt.y];
    const int nb = P.nb, n = P.n;
    int* pdone = P.cnt;
    int* tdone = P.cnt + nb;
    float* A = (float*)P.A;
    float* Lp = (float*)P.Lp;
    float a[64];   // the task's block of A, loaded while the K loop runs
    float v[64];   // this thread's accumulator row segment
    if (PAIRS && tk.y >= 2) {
      // ---- OFF2(I; J0, J1): blocks (I, J0), (I, J1); OFF4(I; J0, J1) (type 3): the same for
      // rows I and I + 1, each B block read once for both rows
      const bool quad = tk.y == 3;
      const int I = tk.z, J0 = tk.w, J1 = J0 + 1;
      const int nck = (BS / KS) * J0;
      load_rows(A, n, I, J0, a);
      const bool str = nck > 0;
      if (str && (tid == 0 || tid == 32)) {
        auto src = [&](int row, int c) {
          return Lp + slot(row, c >> 3) * kSlot + (size_t)(c & 7) * kSub;
        };
        auto pa = [&](int c) -> const float* { return src(I, c); };
        auto pa2 = [&](int c) -> const float* { return src(I + 1, c); };
        auto pb = [&](int c) -> const float* { return src(J0, c); };
        auto pb2 = [&](int c) -> const float* { return src(J1, c); };
        auto dep = [&](int c) {
          if (c & 7) return true;
          const int kb = c >> 3;
          return acquired(wait_flag(&tdone[I * nb + kb], 1, err, budget_ns) &&
                          (!quad || wait_flag(&tdone[(I + 1) * nb + kb], 1, err, budget_ns)) &&
                          wait_flag(&tdone[J0 * nb + kb], 1, err, budget_ns) &&
                          wait_flag(&tdone[J1 * nb + kb], 1, err, budget_ns));
        };
        if (quad) {
          if (tid == 32)
            ws_produce4<3>(stg, wring_q, pos_q, nck, pa, pa2, pb, pb2, dep, err, budget_ns);
          else
            s_ok = ws_consume4<3>(tmem, stg, wring_q, pos_q, bfin, nck, err, budget_ns);
        } else {
          if (tid == 32)
            ws_produce<4, 1, 3, true>(stg, wring_p, pos_p, nck, pa, pb, pb2, dep, err, budget_ns);
          else
            s_ok = ws_consume<4, 1, 3, true>(tmem, tmem + 128u, stg, wring_p, pos_p, bfin, nck,
                                             pa, pb, pb2, err, budget_ns);
        }
      }
      if (tid == 0 && !str) s_ok = *(volatile int*)err == 0;
      if (str) (quad ? pos_q : pos_p) += (unsigned)nck;
      __syncthreads();
      if (!join(str)) break;
      // Row Ir of the pair of block columns, its accumulators at tb (J0) and tb + 128 (J1); a
      // holds block (Ir, J0) of A on entry (and block (Ir + 1, J0) on return when next_row).
      auto pair_rows = [&](int Ir, unsigned tb, bool next_row) {
        if (tid == 0) {   // X_J0 J0's first stages while the C operand is formed
          s_pre = prime_product(Lp + slot(J0, J0) * kSlot, &pdone[J0]);
          s_ok = s_pre >= 0;
        }
        // block (Ir, J0): C = A - acc0, L = C X_J0^T
        tc::fence_after();
        if (nck > 0) {
          tcb::tmem_row64(tb, v);
        } else {
#pragma unroll
          for (int e = 0; e < 64; ++e) v[e] = 0.f;
        }
        tc::fence_before();
        stage_rows(a);
        __syncthreads();
        load_rows(A, n, Ir, J1, a);   // block (Ir, J1) of A, used after the next two products
        form_c(n, Ir, v);
        __syncthreads();
        if (tid == 0 && s_ok)
          s_ok = resident_product(tb, Lp + slot(J0, J0) * kSlot, false, &pdone[J0], s_pre);
        __syncthreads();
        if (!join(s_pre >= 0)) return false;
        if (tid == 0) {   // the k = J0 term's B operand while L_IrJ0 is written
          s_pre = prime_product(Lp + slot(J1, J0) * kSlot, &tdone[J1 * nb + J0]);
          s_ok = s_pre >= 0;
        }
        tc::fence_after();
        tcb::tmem_row64(tb, v);
        tc::fence_before();
        write_block(A, Lp, n, Ir, J0, v);
        __syncthreads();   // Tb read before Cs (which covers it) is written
        // the finished L_IrJ0 as the resident A operand of the k = J0 term of block (Ir, J1)
#pragma unroll
        for (int e = 0; e < 64; e += 4)
          tcb::put4_smem(Cs, arow, acol + e, v[e], v[e + 1], v[e + 2], v[e + 3]);
        publish(&tdone[Ir * nb + J0]);
        if (tid == 0 && s_ok)
          s_ok = resident_product(tb + 128u, Lp + slot(J1, J0) * kSlot, nck > 0,
                                  &tdone[J1 * nb + J0], s_pre);
        __syncthreads();
        if (!join(s_pre >= 0)) return false;
        if (tid == 0) {
          s_pre = prime_product(Lp + slot(J1, J1) * kSlot, &pdone[J1]);
          s_ok = s_pre >= 0;
        }
        // block (Ir, J1): C = A - acc1, L = C X_J1^T
        tc::fence_after();
        tcb::tmem_row64(tb + 128u, v);
        tc::fence_before();
        stage_rows(a);
        __syncthreads();
        if (next_row) load_rows(A, n, Ir + 1, J0, a);   // the next row's first block of A
        form_c(n, Ir, v);
        __syncthreads();
        if (tid == 0 && s_ok)
          s_ok = resident_product(tb + 128u, Lp + slot(J1, J1) * kSlot, false, &pdone[J1],
                                  s_pre);
        __syncthreads();
        if (!join(s_pre >= 0)) return false;
        tc::fence_after();
        tcb::tmem_row64(tb + 128u, v);
        tc::fence_before();
        write_block(A, Lp, n, Ir, J1, v);
        publish(&tdone[Ir * nb + J1]);
        return true;
      };
      if (!pair_rows(I, tmem, quad)) break;
      if (quad && !pair_rows(I + 1, tmem + 256u, false)) break;
      continue;
    }
    const bool diag = tk.y == 0;
    const int I = tk.z, J = tk.w;
    constexpr int CPB = (BS / KS) / G;   // chunks per K block
    const int nck = CPB * J;
    load_rows(A, n, I, J, a);
    // ---- K loop: acc = sum_{k<J} L_Ik L_Jk^T
    const bool str = nck > 0;
    if (str && (tid == 0 || tid == 32)) {
      const float* si = Lp + slot(I, 0) * kSlot;
      const float* sj = Lp + slot(J, 0) * kSlot;
      auto src = [&](const float* base, int c) {
        return base + (size_t)(c / CPB) * kSlot + (c % CPB) * G * kSub;
      };
      auto pa = [&](int c) -> const float* { return src(si, c); };
      auto pb = [&](int c) -> const float* { return diag ? nullptr : src(sj, c); };
      if (tid == 32)
        ws_produce<NS, G, 2>(
            stg, wring_k, pos_k, nck, pa, pb, no_src,
            [&](int c) {
              if (c % CPB) return true;
              const int kb = c / CPB;
              return acquired(wait_flag(&tdone[I * nb + kb], 1, err, budget_ns) &&
                              (diag || wait_flag(&tdone[J * nb + kb], 1, err, budget_ns)));
            },
            err, budget_ns);
      else
        s_ok = ws_consume<NS, G, 2>(tmem, 0u, stg, wring_k, pos_k, bfin, nck, pa, pb, no_src, err,
                                    budget_ns);
    }
    if (tid == 0 && !str) s_ok = *(volatile int*)err == 0;
    if (str) pos_k += (unsigned)nck;
    __syncthreads();
    if (!join(str)) break;
    if (!diag && tid == 0) {   // X_JJ's first stages while the C operand is formed
      s_pre = prime_product(Lp + slot(J, J) * kSlot, &pdone[J]);
      s_ok = s_pre >= 0;
    }
    tc::fence_after();
    if (nck > 0) {
      tcb::tmem_row64(tmem, v);
    } else {
#pragma unroll
      for (int e = 0; e < 64; ++e) v[e] = 0.f;
    }
    tc::fence_before();
    __syncthreads();   // accumulator read before the stages / tensor memory are reused
    const int rg = I * BS + arow;   // this thread's matrix row
    if (diag) {
      // ---- DIAG(J): C (lower, identity padding) -> L_JJ, X_JJ on the SIMT pipes
      float* Cs = sm;                       // 128 x 129
      float* L00 = Cs + BS * LDC;           // 64 x 65 each
      float* X00 = L00 + TB * LDS;
      float* L11 = X00 + TB * LDS;
      float* X11 = L11 + TB * LDS;
      float* X10 = X11 + TB * LDS;
      float* Tt = X10 + TB * LDS;
      float* Pt = Tt + TB * LDS;            // potrf_regs scratch
      float* Dsm = Pt + 8 * TileCfg<float, TB>::LDT;
      float* Tm = Dsm + 64;
      const int r0 = J * BS;
      // the block of A (rows by warps) into Cs, then each row's owner keeps the lower part of
      // C = A - acc inside the matrix, the identity on the padding past n and zero above
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float* row = Cs + (16 * warp + q) * LDC;
        row[2 * lane] = a[4 * q];
        row[2 * lane + 1] = a[4 * q + 1];
        row[64 + 2 * lane] = a[4 * q + 2];
        row[65 + 2 * lane] = a[4 * q + 3];
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 64; ++e) {
        const int c = acol + e;
        float x;
        if (rg < n && r0 + c < n)
          x = c <= arow ? Cs[arow * LDC + c] - v[e] : 0.f;
        else
          x = c == arow ? 1.f : 0.f;
        Cs[arow * LDC + c] = x;
      }
      for (int e = tid; e < TB * LDS; e += blockDim.x) {
        X00[e] = 0.f;
        X11[e] = 0.f;
      }
      __syncthreads();
      float a[RT][RT];
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) a[p][q] = Cs[(tr + p) * LDC + tcl + q];
      potrf_regs<float, TB>(a, L00, X00, Pt, Dsm, Tm, r0, P.status);
      // L10 = C10 X00^T
      float w[RT][RT];
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) w[p][q] = 0.f;
      for (int m = 0; m < TB; ++m) {
        float x[RT], y[RT];
#pragma unroll
        for (int p = 0; p < RT; ++p) x[p] = Cs[(TB + tr + p) * LDC + m];
#pragma unroll
        for (int q = 0; q < RT; ++q) y[q] = X00[(tcl + q) * LDS + m];
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) w[p][q] += x[p] * y[q];
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) Cs[(TB + tr + p) * LDC + tcl + q] = w[p][q];
      __syncthreads();
      // C11 - L10 L10^T
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) a[p][q] = Cs[(TB + tr + p) * LDC + TB + tcl + q];
      for (int m = 0; m < TB; ++m) {
        float x[RT], y[RT];
#pragma unroll
        for (int p = 0; p < RT; ++p) x[p] = Cs[(TB + tr + p) * LDC + m];
#pragma unroll
        for (int q = 0; q < RT; ++q) y[q] = Cs[(TB + tcl + q) * LDC + m];
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) a[p][q] -= x[p] * y[q];
      }
      potrf_regs<float, TB>(a, L11, X11, Pt, Dsm, Tm, r0 + TB, P.status);
      // T = L10 X00, X10 = -X11 T
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) w[p][q] = 0.f;
      for (int m = 0; m < TB; ++m) {
        float x[RT], y[RT];
#pragma unroll
        for (int p = 0; p < RT; ++p) x[p] = Cs[(TB + tr + p) * LDC + m];
#pragma unroll
        for (int q = 0; q < RT; ++q) y[q] = X00[m * LDS + tcl + q];
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) w[p][q] += x[p] * y[q];
      }
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) Tt[(tr + p) * LDS + tcl + q] = w[p][q];
      __syncthreads();
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) w[p][q] = 0.f;
      for (int m = 0; m < TB; ++m) {
        float x[RT], y[RT];
#pragma unroll
        for (int p = 0; p < RT; ++p) x[p] = X11[(tr + p) * LDS + m];
#pragma unroll
        for (int q = 0; q < RT; ++q) y[q] = Tt[m * LDS + tcl + q];
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) w[p][q] -= x[p] * y[q];
      }
#pragma unroll
      for (int p = 0; p < RT; ++p)
#pragma unroll
        for (int q = 0; q < RT; ++q) X10[(tr + p) * LDS + tcl + q] = w[p][q];
      __syncthreads();
      // outputs: L_JJ -> A (lower, in range), X00 / X11 -> Dinv, X_JJ -> slot (J, J)
      const int nt64 = P.nt;
      float* D0 = (float*)P.Dinv + (size_t)(2 * J) * TB * TB;
      for (int e = tid; e < TB * TB; e += blockDim.x) {
        const int r = e / TB, c = e % TB;
        __stcg(D0 + e, c <= r ? X00[r * LDS + c] : 0.f);
        if (2 * J + 1 < nt64) __stcg(D0 + TB * TB + e, c <= r ? X11[r * LDS + c] : 0.f);
      }
      for (int e = tid; e < BS * BS; e += blockDim.x) {
        const int r = e / BS, c = e % BS;
        if (c > r || r0 + r >= n) continue;
        const float l = r < TB ? L00[r * LDS + c]
                               : (c < TB ? Cs[r * LDC + c] : L11[(r - TB) * LDS + c - TB]);
        __stcg(A + (size_t)(r0 + r) * n + r0 + c, l);
      }
      float* S = Lp + slot(J, J) * kSlot;
      for (int e = tid; e < BS * BS / 4; e += blockDim.x) {
        const int r = e / (BS / 4), k = 4 * (e % (BS / 4));
        float x4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = k + q;
          float x = 0.f;
          if (c <= r) {
            if (r < TB) x = X00[r * LDS + c];
            else if (c < TB) x = X10[(r - TB) * LDS + c];
            else x = X11[(r - TB) * LDS + c - TB];
          }
          x4[q] = x;
        }
        tcb::put4(S, r, k, x4[0], x4[1], x4[2], x4[3]);
      }
    } else {
      // ---- OFF(I, J): C = A_IJ - acc as hi / lo operand in shared memory, L_IJ = C X_JJ^T
      stage_rows(a);
      __syncthreads();
      form_c(n, I, v);
      __syncthreads();
      if (tid == 0 && s_ok)
        s_ok = resident_product(tmem, Lp + slot(J, J) * kSlot, false, &pdone[J], s_pre);
      __syncthreads();
      if (!join(s_pre >= 0)) break;
      tc::fence_after();
      tcb::tmem_row64(tmem, v);
      tc::fence_before();
      write_block(A, Lp, n, I, J, v);
    }
    publish(diag ? &pdone[J] : &tdone[I * nb + J]);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// ----------------------------------------------------------------------------- pipelined blocks
// The 128 x 128 block factorisation with the K loop of one task overlapping the epilogue of the
// previous one: warp 8 (one thread) claims the tickets and issues each task's K-loop copies, warp
// 9 (one thread) its products into one of two tensor-memory accumulators; warps 0..7 take the
// finished accumulators in the same order
// and run the epilogues (DIAG: SIMT Cholesky and inverse of the block; OFF: C = A - acc and
// L = C X^T on the tensor cores, in two K halves so that the epilogue's shared memory and the
// K loop's stages fit side by side). Same tasks, slots, flags and results as k_chol_tcb.
namespace tcp {
constexpr int kThreads = 320;
constexpr int kNS = 3;                                 // K-loop stages of 32 KB (A, B)
constexpr int TB = 64, LDS = TB + 1;
constexpr int kTile = TB * LDS;                        // floats of a 64 x 65 tile
constexpr int kPt = 8 * TileCfg<float, TB>::LDT;       // potrf scratch (floats)
constexpr int kScratch = kPt + 64 + TB * TB / 4;
constexpr unsigned kEBytes = 104u * 1024u;             // epilogue area
static_assert(6 * kTile * 4 + kScratch * 4 <= (int)kEBytes, "DIAG tiles fit");
static_assert(4 * tcb::kSubBytes + 2 * tcb::kSubBytes <= kEBytes, "OFF half + X stages fit");
constexpr unsigned kRBytes = kNS * 2 * tcb::kSubBytes;  // K-loop stages (96 KB)
constexpr unsigned kSmem = kEBytes + kRBytes;
}  // namespace tcp

// named barrier 1 over the 256 epilogue threads, with an OR of a predicate
__device__ __forceinline__ void ebar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool ebar_or(bool p) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\tbar.red.or.pred q, 1, 256, p;\n\t"
      "selp.b32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)p)
      : "memory");
  return r != 0;
}
__global__ __launch_bounds__(tcp::kThreads, 1) void k_chol_tcp(
    const ProbDesc* const* __restrict__ descs, const int2* __restrict__ tickets, int nticket,
    int* __restrict__ head, int* __restrict__ err, unsigned long long budget_ns) {
  using namespace tcb;
  using tcp::TB;
  using tcp::LDS;
  constexpr int RT = 4;
  extern __shared__ __align__(1024) unsigned char smb[];
  float* sm = reinterpret_cast<float*>(smb);
  __shared__ __align__(8) unsigned long long bar_task[2], bar_full[2], bar_empty[2], bar_efin;
  __shared__ __align__(8) WRing<tcp::kNS> wring;   // K-loop stages (producer / MMA thread)
  __shared__ __align__(8) Ring<2> ring_x;          // epilogue thread 0
  __shared__ int4 s_task[2];                       // (problem, type, I, J); type -1: no more
  __shared__ unsigned s_tmem;
  __shared__ int s_ok, s_pre;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_task[b]);
      mbar_init(&bar_full[b]);
      mbar_init(&bar_empty[b]);
    }
    mbar_init(&bar_efin);
    wring_init(wring);
    ring_init(ring_x);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     smem_u32(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = s_tmem;
  const unsigned ebase = smem_u32(smb), rbase = ebase + tcp::kEBytes;
  auto no_src = [](int) -> const float* { return nullptr; };
  auto acquired = [](bool ok) {
    fence_proxy_async_global();
    return ok;
  };
  if (warp == 8) {
    // ---- producer: claim, publish the task (buffer u & 1), issue its K-loop copies
    if (lane == 0) {
      int u = 0;
      unsigned pos = 0u;
      auto finish = [&](int b) {
        s_task[b] = make_int4(-1, -1, 0, 0);
        mbar_arrive(&bar_task[b]);
      };
      for (;;) {
        const int b = u & 1;
        if (u >= 2 && !mbar_wait(&bar_empty[b], (unsigned)(((u >> 1) - 1) & 1), err, budget_ns)) {
          finish(b);
          break;
        }
        const int t = atomicAdd(head, 1);
        if (t >= nticket || *(volatile int*)err) {
          finish(b);
          break;
        }
        const int2 pt = tickets[t];
        if (!descs[pt.x]) continue;   // not in this solve
        const LinProblem& P = descs[pt.x]->lp;
        const int4 tk = P.tasks_b[pt.y];
        const bool diag = tk.y == 0;
        const int I = tk.z, J = tk.w, nb = P.nb;
        const int* tdone = P.cnt + nb;
        const float* Lp = (const float*)P.Lp;
        s_task[b] = make_int4(pt.x, tk.y, I, J);
        mbar_arrive(&bar_task[b]);   // release: the task to the MMA thread and the epilogue
        const int nck = (BS / KS) * J;
        if (nck > 0) {
          const float* si = Lp + slot(I, 0) * kSlot;
          const float* sj = Lp + slot(J, 0) * kSlot;
          ws_produce<tcp::kNS, 1, 2>(
              rbase, wring, pos, nck,
              [&](int c) -> const float* { return si + (size_t)(c >> 3) * kSlot + (c & 7) * kSub; },
              [&](int c) -> const float* {
                return diag ? nullptr : sj + (size_t)(c >> 3) * kSlot + (c & 7) * kSub;
              },
              no_src,
              [&](int c) {
                if (c & 7) return true;
                const int kb = c >> 3;
                return acquired(wait_flag(&tdone[I * nb + kb], 1, err, budget_ns) &&
                                (diag || wait_flag(&tdone[J * nb + kb], 1, err, budget_ns)));
              },
              err, budget_ns);
          pos += (unsigned)nck;
          if (*(volatile int*)&wring.pdone) {   // stopped short: no more tasks
            finish((u + 1) & 1);
            break;
          }
        }
        ++u;
      }
    }
    __syncwarp();
  } else if (warp == 9) {
    // ---- MMA thread: each published task's K loop into accumulator u & 1
    if (lane == 0) {
      unsigned pos = 0u;
      for (int u = 0;; ++u) {
        const int b = u & 1;
        if (!mbar_wait(&bar_task[b], (unsigned)((u >> 1) & 1), err, budget_ns)) break;
        const int4 tk = s_task[b];
        if (tk.y < 0) break;
        const LinProblem& P = descs[tk.x]->lp;
        const bool diag = tk.y == 0;
        const int I = tk.z, J = tk.w;
        const float* Lp = (const float*)P.Lp;
        const int nck = (BS / KS) * J;
        if (nck == 0) {
          mbar_arrive(&bar_full[b]);
          continue;
        }
        const float* si = Lp + slot(I, 0) * kSlot;
        const float* sj = Lp + slot(J, 0) * kSlot;
        const bool ok = ws_consume<tcp::kNS, 1, 2>(
            tmem + 128u * b, 0u, rbase, wring, pos, &bar_full[b], nck,
            [&](int c) -> const float* { return si + (size_t)(c >> 3) * kSlot + (c & 7) * kSub; },
            [&](int c) -> const float* {
              return diag ? nullptr : sj + (size_t)(c >> 3) * kSlot + (c & 7) * kSub;
            },
            no_src, err, budget_ns);
        pos += (unsigned)nck;
        if (!ok) break;   // the error word is raised; the epilogue sees it
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue (warps 0..7)
    const int tr = (tid / 16) * RT, tcl = (tid % 16) * RT;               // 64 x 64 register blocks
    const int arow = 32 * (warp & 3) + lane, acol = 64 * (warp >> 2);   // accumulator ownership
    float* Tb = sm;       // OFF: the block of A (swizzled rows), later the block of L
    float* Ch = sm;       // OFF: one K half of C as the hi / lo A operand (4 sub-chunks, 64 KB)
    const unsigned xstg = ebase + 4u * kSubBytes;   // OFF: stages of X (2 x 16 KB)
    float* C00 = sm;      // DIAG: 64 x 65 tiles of the block (C01 is not kept), then of L
    float* C10 = C00 + tcp::kTile;
    float* C11 = C10 + tcp::kTile;
    float* X00 = C11 + tcp::kTile;
    float* X11 = X00 + tcp::kTile;
    float* Tt = X11 + tcp::kTile;   // L10 X00, then X10
    float* Pt = Tt + tcp::kTile;
    float* Dsm = Pt + tcp::kPt;
    float* Tm = Dsm + 64;
    auto tpos = [](int r, int c) { return r * BS + ((((c >> 2) ^ (r & 7)) << 2) | (c & 3)); };
    unsigned efph = 0u;   // parity of the next bar_efin completion
    // thread 0: the first stages of a K-half product, B = 4 sub-chunks at src (after flag)
    auto half_prime = [&](const float* src, const int* flag) {
      return prime<2, 1, 1>(
          xstg, ring_x, 4, no_src, [&](int c) -> const float* { return src + (size_t)c * kSub; },
          no_src,
          [&](int c) {
            return c > 0 || flag == nullptr || acquired(wait_flag(flag, 1, err, budget_ns));
          },
          err, budget_ns);
    };
    // thread 0: D (+)= [C half in Ch] B^T, the first `pre` stages already issued
    auto half_product = [&](unsigned tm, const float* src, bool acc_first, int pre) {
      return stream<2, 1, 1>(
          tm, 0u, xstg, ring_x, &bar_efin, 4, pre, acc_first, no_src,
          [&](int c) { return ebase + (unsigned)c * kSubBytes; },
          [&](int c) -> const float* { return src + (size_t)c * kSub; }, no_src,
          [&](int) { return true; }, err, budget_ns);
    };
    // every epilogue thread: wait for thread 0's product (when it streamed); false on a failure
    auto ejoin = [&](bool streamed) {
      bool bad = !s_ok;
      if (streamed) {
        const bool got = mbar_wait(&bar_efin, efph, err, budget_ns);
        efph ^= 1u;
        bad = bad || !got;
      }
      return !ebar_or(bad);
    };
    auto epublish = [&](int* f) {
      fence_proxy_async_shared();
      fence_proxy_async_global();
      ebar();
      if (tid == 0) {
        __threadfence();
        st_release(f, 1);
      }
    };
    float v[64];
    for (int e = 0;; ++e) {
      const int b = e & 1;
      const unsigned ph = (unsigned)((e >> 1) & 1);
      const bool got = mbar_wait(&bar_task[b], ph, err, budget_ns);
      const int4 tk = s_task[b];
      if (ebar_or(!got || tk.y < 0)) break;
      const LinProblem& P = descs[tk.x]->lp;
      const int I = tk.z, J = tk.w, nb = P.nb, n = P.n;
      int* pdone = P.cnt;
      int* tdone = P.cnt + nb;
      float* A = (float*)P.A;
      float* Lp = (float*)P.Lp;
      const unsigned tmb = tmem + 128u * b;
      if (tk.y == 0) {
        // ---- DIAG(J): block (J, J) of A into the tiles (rows by warps, coalesced)
        const int r0 = J * BS, c0 = r0 + 2 * lane;
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
          const int r = 16 * warp + q, rg = r0 + r;
          float2 p0 = make_float2(0.f, 0.f), p1 = p0;
          if (rg < n) {
            const float* row = A + (size_t)rg * n;
            if (c0 < n) p0 = __ldcg(reinterpret_cast<const float2*>(row + c0));
            if (r >= TB && c0 + 64 < n) p1 = __ldcg(reinterpret_cast<const float2*>(row + c0 + 64));
          }
          float* t0 = r < TB ? C00 + r * LDS : C10 + (r - TB) * LDS;
          t0[2 * lane] = p0.x;
          t0[2 * lane + 1] = p0.y;
          if (r >= TB) {
            float* t1 = C11 + (r - TB) * LDS;
            t1[2 * lane] = p1.x;
            t1[2 * lane + 1] = p1.y;
          }
        }
        for (int e2 = tid; e2 < tcp::kTile; e2 += 256) {
          X00[e2] = 0.f;
          X11[e2] = 0.f;
        }
        const bool okf = mbar_wait(&bar_full[b], ph, err, budget_ns);
        if (ebar_or(!okf || *(volatile int*)err != 0)) break;
        tc::fence_after();
        if (J > 0) {
          tcb::tmem_row64(tmb, v);
        } else {
#pragma unroll
          for (int q = 0; q < 64; ++q) v[q] = 0.f;
        }
        tc::fence_before();
        ebar();
        if (tid == 0) mbar_arrive(&bar_empty[b]);   // the accumulator is read
        // C = A - acc: lower part inside the matrix, identity on the padding past n, zero above
        const int rg = r0 + arow;
        if (arow >= TB || acol == 0) {
          float* tl = arow < TB ? C00 + arow * LDS : (acol == 0 ? C10 : C11) + (arow - TB) * LDS;
#pragma unroll
          for (int q = 0; q < 64; ++q) {
            const int c = acol + q;
            float x;
            if (rg < n && r0 + c < n)
              x = c <= arow ? tl[q] - v[q] : 0.f;
            else
              x = c == arow ? 1.f : 0.f;
            tl[q] = x;
          }
        }
        ebar();
        float a[RT][RT], w[RT][RT];
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) a[p][q] = C00[(tr + p) * LDS + tcl + q];
        ebar();   // C00 read before its Cholesky factor overwrites it
        potrf_regs<float, TB, 1>(a, C00, X00, Pt, Dsm, Tm, r0, P.status);
        // L10 = C10 X00^T, in place
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) w[p][q] = 0.f;
        for (int m = 0; m < TB; ++m) {
          float x[RT], y[RT];
#pragma unroll
          for (int p = 0; p < RT; ++p) x[p] = C10[(tr + p) * LDS + m];
#pragma unroll
          for (int q = 0; q < RT; ++q) y[q] = X00[(tcl + q) * LDS + m];
#pragma unroll
          for (int p = 0; p < RT; ++p)
#pragma unroll
            for (int q = 0; q < RT; ++q) w[p][q] += x[p] * y[q];
        }
        ebar();
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) C10[(tr + p) * LDS + tcl + q] = w[p][q];
        ebar();
        // C11 - L10 L10^T, factored in place
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) a[p][q] = C11[(tr + p) * LDS + tcl + q];
        for (int m = 0; m < TB; ++m) {
          float x[RT], y[RT];
#pragma unroll
          for (int p = 0; p < RT; ++p) x[p] = C10[(tr + p) * LDS + m];
#pragma unroll
          for (int q = 0; q < RT; ++q) y[q] = C10[(tcl + q) * LDS + m];
#pragma unroll
          for (int p = 0; p < RT; ++p)
#pragma unroll
            for (int q = 0; q < RT; ++q) a[p][q] -= x[p] * y[q];
        }
        ebar();   // C11 read before its factor overwrites it
        potrf_regs<float, TB, 1>(a, C11, X11, Pt, Dsm, Tm, r0 + TB, P.status);
        // T = L10 X00, then X10 = -X11 T (in place)
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) w[p][q] = 0.f;
        for (int m = 0; m < TB; ++m) {
          float x[RT], y[RT];
#pragma unroll
          for (int p = 0; p < RT; ++p) x[p] = C10[(tr + p) * LDS + m];
#pragma unroll
          for (int q = 0; q < RT; ++q) y[q] = X00[m * LDS + tcl + q];
#pragma unroll
          for (int p = 0; p < RT; ++p)
#pragma unroll
            for (int q = 0; q < RT; ++q) w[p][q] += x[p] * y[q];
        }
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) Tt[(tr + p) * LDS + tcl + q] = w[p][q];
        ebar();
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) w[p][q] = 0.f;
        for (int m = 0; m < TB; ++m) {
          float x[RT], y[RT];
#pragma unroll
          for (int p = 0; p < RT; ++p) x[p] = X11[(tr + p) * LDS + m];
#pragma unroll
          for (int q = 0; q < RT; ++q) y[q] = Tt[m * LDS + tcl + q];
#pragma unroll
          for (int p = 0; p < RT; ++p)
#pragma unroll
            for (int q = 0; q < RT; ++q) w[p][q] -= x[p] * y[q];
        }
        ebar();
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
          for (int q = 0; q < RT; ++q) Tt[(tr + p) * LDS + tcl + q] = w[p][q];
        ebar();
        // outputs: L_JJ -> A (lower, in range), X00 / X11 -> Dinv, X_JJ -> slot (J, J)
        const int nt64 = P.nt;
        float* D0 = (float*)P.Dinv + (size_t)(2 * J) * TB * TB;
        for (int e2 = tid; e2 < TB * TB; e2 += 256) {
          const int r = e2 / TB, c = e2 % TB;
          __stcg(D0 + e2, c <= r ? X00[r * LDS + c] : 0.f);
          if (2 * J + 1 < nt64) __stcg(D0 + TB * TB + e2, c <= r ? X11[r * LDS + c] : 0.f);
        }
        for (int e2 = tid; e2 < BS * BS; e2 += 256) {
          const int r = e2 / BS, c = e2 % BS;
          if (c > r || r0 + r >= n) continue;
          const float l = r < TB ? C00[r * LDS + c]
                                 : (c < TB ? C10[(r - TB) * LDS + c] : C11[(r - TB) * LDS + c - TB]);
          __stcg(A + (size_t)(r0 + r) * n + r0 + c, l);
        }
        float* S = Lp + slot(J, J) * kSlot;
        for (int e2 = tid; e2 < BS * BS / 4; e2 += 256) {
          const int r = e2 / (BS / 4), k = 4 * (e2 % (BS / 4));
          float x4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = k + q;
            float x = 0.f;
            if (c <= r) {
              if (r < TB) x = X00[r * LDS + c];
              else if (c < TB) x = Tt[(r - TB) * LDS + c];
              else x = X11[(r - TB) * LDS + c - TB];
            }
            x4[q] = x;
          }
          tcb::put4(S, r, k, x4[0], x4[1], x4[2], x4[3]);
        }
        epublish(&pdone[J]);
        continue;
      }
      // ---- OFF(I, J): block (I, J) of A into Tb (its columns lie inside the matrix)
      {
        const int c0 = J * BS + 2 * lane;
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
          const int r = 16 * warp + q, rg = I * BS + r;
          float2 p0 = make_float2(0.f, 0.f), p1 = p0;
          if (rg < n) {
            const float* row = A + (size_t)rg * n;
            p0 = __ldcg(reinterpret_cast<const float2*>(row + c0));
            p1 = __ldcg(reinterpret_cast<const float2*>(row + c0 + 64));
          }
          *reinterpret_cast<float2*>(Tb + tpos(r, 2 * lane)) = p0;
          *reinterpret_cast<float2*>(Tb + tpos(r, 64 + 2 * lane)) = p1;
        }
      }
      const bool okf = mbar_wait(&bar_full[b], ph, err, budget_ns);
      if (ebar_or(!okf || *(volatile int*)err != 0)) break;
      tc::fence_after();
      if (J > 0) {
        tcb::tmem_row64(tmb, v);
      } else {
#pragma unroll
        for (int q = 0; q < 64; ++q) v[q] = 0.f;
      }
      tc::fence_before();
      const float* sx = Lp + slot(J, J) * kSlot;
      if (tid == 0) {   // X_JJ's first stages while C is formed
        s_pre = half_prime(sx, &pdone[J]);
        s_ok = s_pre >= 0;
      }
      // C = A - acc on this thread's row segment (zero on rows past n)
      {
        const bool in = I * BS + arow < n;
#pragma unroll
        for (int q = 0; q < 64; q += 4) {
          const float4 t4 = *reinterpret_cast<const float4*>(Tb + tpos(arow, acol + q));
          v[q] = in ? t4.x - v[q] : 0.f;
          v[q + 1] = in ? t4.y - v[q + 1] : 0.f;
          v[q + 2] = in ? t4.z - v[q + 2] : 0.f;
          v[q + 3] = in ? t4.w - v[q + 3] : 0.f;
        }
      }
      ebar();   // Tb read before the C half overwrites it
      if (acol == 0) {
#pragma unroll
        for (int q = 0; q < 64; q += 4)
          tcb::put4_smem(Ch, arow, q, v[q], v[q + 1], v[q + 2], v[q + 3]);
        fence_proxy_async_shared();
      }
      ebar();
      if (tid == 0 && s_ok) s_ok = half_product(tmb, sx, false, s_pre);
      ebar();
      if (!ejoin(s_pre >= 0)) break;
      // second K half: X sub-chunks 4..7 against columns 64..127 of C
      if (tid == 0) {
        s_pre = half_prime(sx + 4 * kSub, nullptr);
        s_ok = s_pre >= 0;
      }
      if (acol == TB) {
#pragma unroll
        for (int q = 0; q < 64; q += 4)
          tcb::put4_smem(Ch, arow, q, v[q], v[q + 1], v[q + 2], v[q + 3]);
        fence_proxy_async_shared();
      }
      ebar();
      if (tid == 0 && s_ok) s_ok = half_product(tmb, sx + 4 * kSub, true, s_pre);
      ebar();
      if (!ejoin(s_pre >= 0)) break;
      tc::fence_after();
      tcb::tmem_row64(tmb, v);
      tc::fence_before();
      ebar();
      if (tid == 0) mbar_arrive(&bar_empty[b]);   // the accumulator is free again
      // L_IJ -> its slot, and through Tb (rows) -> A
#pragma unroll
      for (int q = 0; q < 64; q += 4)
        *reinterpret_cast<float4*>(Tb + tpos(arow, acol + q)) =
            make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      float* S = Lp + slot(I, J) * kSlot;
#pragma unroll
      for (int q = 0; q < 64; q += 4)
        tcb::put4(S, arow, acol + q, v[q], v[q + 1], v[q + 2], v[q + 3]);
      ebar();
      {
        const int c0 = J * BS + 2 * lane;
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
          const int r = 16 * warp + q, rg = I * BS + r;
          if (rg < n) {
            float* row = A + (size_t)rg * n;
            __stcg(reinterpret_cast<float2*>(row + c0),
                   *reinterpret_cast<const float2*>(Tb + tpos(r, 2 * lane)));
            __stcg(reinterpret_cast<float2*>(row + c0 + 64),
                   *reinterpret_cast<const float2*>(Tb + tpos(r, 64 + 2 * lane)));
          }
        }
      }
      epublish(&tdone[I * nb + J]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

template <typename T>
size_t chol_packed_elems(int nt) {
  constexpr int TB = sizeof(T) == 8 ? 32 : 64;
  // FP32: room for the larger of the tensor-core layouts (64-tile and 128-block slots, hi + lo,
  // K-major), which also holds the SIMT kernel's transposed padded tiles; FP64: transposed
  // padded tiles
  const int nb = (nt + 1) / 2;   // 128-row blocks
  return sizeof(T) == 4 ? std::max(tile_slot(nt, 0) * (size_t)tc::kSlot,
                                   tcb::slot(nb, 0) * (size_t)tcb::kSlot)
                        : tile_slot(nt, 0) * (size_t)TB * TileCfg<T, TB>::LDT;
}
template size_t chol_packed_elems<float>(int);
template size_t chol_packed_elems<double>(int);



// Synthetic SPD system of every problem's size, for timing the factorisation kernels (FP32
// precisions): A_ii = n, A_ij = 1 / (2 (1 + |i - j|)^2) below the diagonal (diagonally dominant).
__global__ void k_fill_spd(const ProbDesc* const* __restrict__ descs) {
  if (!descs[blockIdx.y]) return;
  const LinProblem& P = descs[blockIdx.y]->lp;
  const int n = P.n;
  float* A = (float*)P.A;
  const size_t tot = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (j > i) continue;
    const float d = 1.f + (float)(i - j);
    A[e] = i == j ? (float)n : 0.5f / (d * d);
  }
}

void launch_fill_spd(const BatchTabs& B, cudaStream_t s) {
  k_fill_spd<<<dim3(64, B.P), 256, 0, s>>>(B.d);
  ++g_launches;
}

template <typename T>
void launch_chol_dag(const BatchTabs& B, cudaStream_t s) {
  if (sizeof(T) == 4 && B.factor_tc == 2) {
    const int nticket = B.tcb_quad ? B.n_chol_q : B.tcb_pairs ? B.n_chol_p : B.n_chol_b;
    const int2* tickets = B.tcb_quad ? B.chol_q : B.tcb_pairs ? B.chol_p : B.chol_b;
    const int grid = std::min(nticket, num_sms());
    auto go = [&](auto kern, PerDevice& attr) {
      set_smem_once(attr, kern, (int)tcb::kSmem);
      kern<<<grid, 256, tcb::kSmem, s>>>(B.d, tickets, nticket, B.words + 0, B.words + 5,
                                         2000000000ull, B.tcb_quad);
    };
    static PerDevice attr[4];
    if (B.tcb_pipe) {
      set_smem_once(attr[0], k_chol_tcp, (int)tcp::kSmem);
      k_chol_tcp<<<grid, tcp::kThreads, tcp::kSmem, s>>>(B.d, tickets, nticket, B.words + 0,
                                                          B.words + 5, 2000000000ull);
    } else if (B.tcb_pairs || B.tcb_quad)
      go(k_chol_tcb<2, true>, attr[1]);
    else if (B.tcb_g == 1)
      go(k_chol_tcb<1, false>, attr[2]);
    else
      go(k_chol_tcb<2, false>, attr[3]);
    ++g_launches;
    return;
  }
  if (sizeof(T) == 4 && B.factor_tc) {
    static PerDevice attr_tc, occ_tc;
    set_smem_once(attr_tc, k_chol_tc, (int)tc::kSmem);
    const int per_sm = ctas_per_sm_once(occ_tc, k_chol_tc, 256, tc::kSmem, 2);
    const int grid = std::min(B.n_chol, per_sm * num_sms());
    k_chol_tc<<<grid, 256, tc::kSmem, s>>>(B.d, B.chol, B.n_chol, B.words + 0, B.words + 5,
                                            2000000000ull);
    ++g_launches;
    return;
  }
  constexpr int TB = sizeof(T) == 8 ? 32 : 64;
  const size_t sm = 4 * sizeof(T) * TB * TileCfg<T, TB>::LDT;
  static PerDevice attr, occ;
  set_smem_once(attr, k_chol_dag<T, TB>, (int)sm);
  const int per_sm = ctas_per_sm_once(occ, k_chol_dag<T, TB>, 256, sm, 4);
  const int grid = std::min(B.n_chol, per_sm * num_sms());
  k_chol_dag<T, TB><<<grid, 256, sm, s>>>(B.d, B.chol, B.n_chol, B.words + 0, B.words + 5,
                                          2000000000ull);
  ++g_launches;
}

template void launch_chol_dag<float>(const BatchTabs&, cudaStream_t);
template void launch_chol_dag<double>(const BatchTabs&, cudaStream_t);

}  // namespace ds
