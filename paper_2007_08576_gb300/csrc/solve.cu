// Triangular solves and the refinement residual of the damped normal equations (Section 2:
// the Cholesky factors solve the Gauss-Newton step; iterative refinement against the FP32
// system), for T = double (TB = 32) or T = float (TB = 64).
//
// Triangular solves: one launch, one ticket per tile row and direction (forward tickets first,
// then backward in reverse row order): y_i = L_ii^-1 (b_i - sum_{j<i} L_ij y_j), then
// x_i = L_ii^-T (y_i - sum_{j>i} L_ji^T x_j), each term consumed as soon as its producer
// publishes it; L_ii^-1 is the diagonal-tile inverse the factorisation stored.
#include <math.h>

#include "dev_util.cuh"
#include "ds_internal.cuh"

namespace ds {

// ----------------------------------------------------------------------------- solves

// Register-prefetched tile GEMVs of the triangular solves (256 threads).
// Row form (forward): thread (warp w, lane l) holds M[r][c] for r = w + 8 s, c = l + 32 t.
// Column form (backward): thread (r = tid % TB, slice sl = tid / TB) holds M[c][r] for
// c = sl + SL q, SL = 256 / TB. Both hold TB * TB / 256 values per thread.
template <typename T, int TB>
struct SolveTile {
  static constexpr int NV = TB * TB / 256;
  static constexpr int RS = TB / 8;    // rows per warp (row form)
  static constexpr int CS = TB / 32;   // columns per lane (row form)
  static constexpr int SL = 256 / TB;  // slices (column form)
};

template <typename T, int TB>
__device__ __forceinline__ void prefetch_rows(const T* M, size_t ld, int nr, int nc,
                                              T (&v)[SolveTile<T, TB>::NV]) {
  constexpr int RS = SolveTile<T, TB>::RS, CS = SolveTile<T, TB>::CS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < RS; ++s)
#pragma unroll
    for (int t = 0; t < CS; ++t) {
      const int r = warp + 8 * s, c = lane + 32 * t;
      v[s * CS + t] = (r < nr && c < nc) ? ldcg(M + (size_t)r * ld + c) : (T)0;
    }
}

template <typename T, int TB>
__device__ __forceinline__ void prefetch_cols(const T* M, size_t ld, int nr, int nc,
                                              T (&v)[SolveTile<T, TB>::NV]) {
  constexpr int SL = SolveTile<T, TB>::SL, NV = SolveTile<T, TB>::NV;
  const int r = threadIdx.x % TB, sl = threadIdx.x / TB;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int c = sl + SL * q;
    v[q] = (r < nr && c < nc) ? ldcg(M + (size_t)c * ld + r) : (T)0;
  }
}

// acc[r] (-)= sum_c M[r][c] vin[c] from prefetched row-form values.
template <typename T, int TB>
__device__ __forceinline__ void gemv_rows_pf(const T (&v)[SolveTile<T, TB>::NV], const T* vin,
                                             T* acc, bool sub) {
  constexpr int RS = SolveTile<T, TB>::RS, CS = SolveTile<T, TB>::CS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < RS; ++s) {
    T sum = (T)0;
#pragma unroll
    for (int t = 0; t < CS; ++t) sum += v[s * CS + t] * vin[lane + 32 * t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) acc[warp + 8 * s] = sub ? acc[warp + 8 * s] - sum : sum;
  }
}

// acc[r] (-)= sum_c M[c][r] vin[c] from prefetched column-form values (reduction through part).
template <typename T, int TB>
__device__ __forceinline__ void gemv_cols_pf(const T (&v)[SolveTile<T, TB>::NV], const T* vin,
                                             T* acc, bool sub, T (*part)[17]) {
  constexpr int SL = SolveTile<T, TB>::SL, NV = SolveTile<T, TB>::NV;
  const int r = threadIdx.x % TB, sl = threadIdx.x / TB;
  T sum = (T)0;
#pragma unroll
  for (int q = 0; q < NV; ++q) sum += v[q] * vin[sl + SL * q];
  part[r][sl] = sum;
  __syncthreads();
  if (threadIdx.x < TB) {
    T a = (T)0;
#pragma unroll
    for (int q = 0; q < SL; ++q) a += part[threadIdx.x][q];
    acc[threadIdx.x] = sub ? acc[threadIdx.x] - a : a;
  }
}

// Row hand-offs: the producer's threads store the row, meet at a CTA barrier, and thread 0
// publishes the flag with a GPU-scope release store (st_release); the consumer polls it with
// GPU-scope acquire loads (wait_flag): no full fences, no sleep between polls, since the chain of
// rows is the solve's critical path.

// Tickets per problem: [0, nt) forward rows 0..nt-1, [nt, 2nt) backward rows nt-1..0.
// flags: [0, nt) forward row done, [nt, 2nt) backward row done. The tiles of L a ticket needs do
// not depend on other tickets and stream ahead of their use (a few tiles in flight); the inputs
// they multiply are taken a ready prefix at a time (one acquire load per tile, by as many
// threads), so only the producers that are still running cost a hand-off each.
// The forward tickets read the right-hand side from b (first solve) or from the refinement
// residual r (from_r) in FP64; the backward tickets also write the solution into the FP64 x
// (assigned, or added to it for a refinement step) and its two-float split for the residual.
template <typename T, int TB>
__global__ __launch_bounds__(256, 2) void k_trsv_dag(const ProbDesc* const* __restrict__ descs,
                                                  int np, int nticket, int solve_id, int from_r,
                                                  int assign, int* __restrict__ head,
                                                  int* __restrict__ err,
                                                  unsigned long long budget_ns) {
  constexpr int NV = SolveTile<T, TB>::NV;
  constexpr int kPF = sizeof(T) == 8 ? 4 : 2;   // tiles of L in flight per CTA
  constexpr int kSpan = 2048 / TB;           // tiles whose inputs fit the shared buffer
  __shared__ T acc[TB];
  __shared__ T vin[TB];
  __shared__ T part[TB][17];
  __shared__ T ysm[kSpan * TB];
  __shared__ int s_t, s_ok, s_first;
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(head, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= nticket) return;
    if (!descs[t % np]) {   // not in this solve
      __syncthreads();
      continue;
    }
    const ProbDesc& PD = *descs[t % np];
    const LinProblem& P = PD.lp;
    const int2 tk = make_int2(t % np, t / np);
    if (tk.y >= 2 * P.nt) {
      __syncthreads();
      continue;
    }
    const int nt = P.nt, n = P.n;
    const bool fwd = tk.y < nt;
    const int i = fwd ? tk.y : 2 * nt - 1 - tk.y;
    const int r0 = i * TB;
    const int nr = min(TB, n - r0);
    const T* L = (const T*)P.A;
    const T* D = (const T*)P.Dinv + (size_t)i * TB * TB;
    int* flag = P.flags;
    T* y = (T*)P.y;
    T* x = (T*)P.x;
    const double* rhs = from_r ? PD.r : PD.b;
    const T* src = fwd ? y : x;
    T dv[NV];  // the diagonal block's inverse, prefetched
    if (fwd)
      prefetch_rows<T, TB>(D, TB, TB, TB, dv);
    else
      prefetch_cols<T, TB>(D, TB, TB, TB, dv);
    bool ok = true;
    if (threadIdx.x == 0) {
      ok = fwd ? true : wait_flag(&flag[i], solve_id, err, budget_ns);
      s_ok = ok;
    }
    __syncthreads();
    ok = s_ok;
    if (threadIdx.x < TB)
      acc[threadIdx.x] = (threadIdx.x < nr && ok)
                             ? (fwd ? (T)ldcg(rhs + r0 + threadIdx.x) : ldcg(y + r0 + threadIdx.x))
                             : (T)0;
    const int cnt = fwd ? i : nt - 1 - i;
    // The tiles before the diagonal, in order: tile q is row tile jt(q) of this row's L (forward)
    // or column tile of L^T (backward). Flags of the producing rows are prefix-ordered (a row is
    // published only after it consumed its predecessor), so a ready prefix is found with one
    // acquire load per tile, its inputs go to shared memory at once, and its tiles are consumed
    // back to back (PF tiles of L in flight) with row partial sums kept in registers.
    auto jtile = [&](int q) { return fwd ? q : nt - 1 - q; };
    auto fidx = [&](int jt) { return fwd ? jt : nt + jt; };
    auto fetch = [&](int q, T (&v)[NV]) {
      const int jt = jtile(q), c0 = jt * TB, nc = min(TB, n - c0);
      if (fwd)
        prefetch_rows<T, TB>(L + (size_t)r0 * n + c0, n, nr, nc, v);
      else
        prefetch_cols<T, TB>(L + (size_t)c0 * n + r0, n, nr, nc, v);
    };
    T lv[kPF][NV];
#pragma unroll
    for (int p = 0; p < kPF; ++p)
      if (p < cnt) fetch(p, lv[p]);
    T ps[SolveTile<T, TB>::RS];   // forward: rows warp + 8 s; backward: ps[0] for (r, slice)
#pragma unroll
    for (int k = 0; k < SolveTile<T, TB>::RS; ++k) ps[k] = (T)0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cr = threadIdx.x % TB, csl = threadIdx.x / TB;
    int done = 0;
    while (ok && done < cnt) {
      const int span = min(cnt - done, kSpan);
      if (threadIdx.x == 0) s_first = span;
      __syncthreads();
      if ((int)threadIdx.x < span &&
          ld_acquire(&flag[fidx(jtile(done + threadIdx.x))]) < solve_id)
        atomicMin(&s_first, (int)threadIdx.x);
      __syncthreads();
      int m = done + s_first;
      if (m == done) {   // nothing ready yet: wait for the next producer
        if (threadIdx.x == 0)
          s_ok = wait_flag(&flag[fidx(jtile(done))], solve_id, err, budget_ns);
        __syncthreads();
        ok = s_ok;
        if (!ok) break;
        m = done + 1;
      }
      for (int e = threadIdx.x; e < (m - done) * TB; e += blockDim.x) {
        const int c = jtile(done + e / TB) * TB + e % TB;
        ysm[e] = c < n ? ldcg(src + c) : (T)0;
      }
      __syncthreads();
      for (int q = done; q < m; ++q) {
        T cur[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) cur[e] = lv[0][e];
#pragma unroll
        for (int p = 0; p + 1 < kPF; ++p)
#pragma unroll
          for (int e = 0; e < NV; ++e) lv[p][e] = lv[p + 1][e];
        if (q + kPF < cnt) fetch(q + kPF, lv[kPF - 1]);
        const T* yv = ysm + (q - done) * TB;
        if (fwd) {
          constexpr int RS = SolveTile<T, TB>::RS, CS = SolveTile<T, TB>::CS;
#pragma unroll
          for (int s2 = 0; s2 < RS; ++s2)
#pragma unroll
            for (int t = 0; t < CS; ++t) ps[s2] += cur[s2 * CS + t] * yv[lane + 32 * t];
        } else {
          constexpr int SL = SolveTile<T, TB>::SL;
#pragma unroll
          for (int e = 0; e < NV; ++e) ps[0] += cur[e] * yv[csl + SL * e];
        }
      }
      done = m;
      __syncthreads();   // ysm is refilled next round
    }
    if (ok && cnt > 0) {   // acc -= the partial sums
      if (fwd) {
        constexpr int RS = SolveTile<T, TB>::RS;
#pragma unroll
        for (int s2 = 0; s2 < RS; ++s2) {
          T sum = ps[s2];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (lane == 0) acc[warp + 8 * s2] -= sum;
        }
      } else {
        constexpr int SL = SolveTile<T, TB>::SL;
        part[cr][csl] = ps[0];
        __syncthreads();
        if (threadIdx.x < TB) {
          T a = (T)0;
#pragma unroll
          for (int q = 0; q < SL; ++q) a += part[threadIdx.x][q];
          acc[threadIdx.x] -= a;
        }
      }
      __syncthreads();
    }
    if (ok) {
      if (threadIdx.x < TB) vin[threadIdx.x] = acc[threadIdx.x];
      __syncthreads();
      if (fwd)
        gemv_rows_pf<T, TB>(dv, vin, acc, false);
      else
        gemv_cols_pf<T, TB>(dv, vin, acc, false, part);
      __syncthreads();
      if (threadIdx.x < nr) {
        const T v = acc[threadIdx.x];
        __stcg((fwd ? y : x) + r0 + threadIdx.x, v);
        if (!fwd) {
          const int e = r0 + threadIdx.x;
          const double xi = assign ? (double)v : PD.x[e] + (double)v;
          PD.x[e] = xi;
          const float hi = __double2float_rn(xi);
          PD.xf[e] = make_float2(hi, __double2float_rn(xi - (double)hi));
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release(&flag[fwd ? i : nt + i], solve_id);
  }
}


template <typename T>
void launch_trsv_dag(const BatchTabs& B, int solve_id, bool from_r, bool assign, cudaStream_t s) {
  constexpr int TB = sizeof(T) == 8 ? 32 : 64;
  static PerDevice occ;
  const int per_sm = ctas_per_sm_once(occ, k_trsv_dag<T, TB>, 256, 0, 4);
  const int nticket = B.P * 2 * B.max_nt;
  const int grid = std::min(nticket, per_sm * num_sms());
  k_trsv_dag<T, TB><<<grid, 256, 0, s>>>(B.d, B.P, nticket, solve_id, from_r ? 1 : 0,
                                          assign ? 1 : 0, B.words + solve_id, B.words + 5,
                                          2000000000ull);
  ++g_launches;
}

// r = b - A x with A the full symmetric FP32 matrix and x = hi + lo (two floats, written with x):
// each product a x_hi is split exactly with an FMA (a x_hi = p + e), a x_lo is added to the error
// term, and the sum is kept as an unevaluated pair of floats (two-sum), i.e. about 48 significant
// bits, the precision of FP64 accumulation for these sums, at FP32 instruction rates (the FP64
// pipe of this GPU is 1/64 of FP32). One warp per row, (problem, 8-row chunk) per CTA.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_add_term(float a, float2 x, float& sh, float& sl) {
  const float p = __fmul_rn(a, x.x);
  const float t = __fmaf_rn(a, x.y, __fmaf_rn(a, x.x, -p));  // (a x_hi - p) + a x_lo
  float e;
  two_sum(sh, p, sh, e);
  sl = __fadd_rn(sl, __fadd_rn(e, t));
}
__global__ __launch_bounds__(256) void k_residual64(const ProbDesc* const* __restrict__ descs,
                                                    const int2* __restrict__ tab) {
  const int2 w = tab[blockIdx.x];
  if (!descs[w.x]) return;   // not in this solve
  const ProbDesc& D = *descs[w.x];
  const int n = D.n;
  const int row = w.y * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* a = D.Aref + (size_t)row * n;
  const float2* __restrict__ x = D.xf;
  float sh = 0.f, sl = 0.f;
  if ((n & 3) == 0) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    for (int q = lane; q < (n >> 2); q += 32) {
      const float4 v = __ldcs(a4 + q);
      df_add_term(v.x, x[4 * q], sh, sl);
      df_add_term(v.y, x[4 * q + 1], sh, sl);
      df_add_term(v.z, x[4 * q + 2], sh, sl);
      df_add_term(v.w, x[4 * q + 3], sh, sl);
    }
  } else {
    for (int j = lane; j < n; j += 32) df_add_term(a[j], x[j], sh, sl);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
    float e;
    two_sum(sh, oh, sh, e);
    sl = __fadd_rn(sl, __fadd_rn(ol, e));
  }
  if (lane == 0) D.r[row] = D.b[row] - ((double)sh + (double)sl);
}

void launch_residual64(const BatchTabs& B, cudaStream_t s) {
  k_residual64<<<B.n_res, 256, 0, s>>>(B.d, B.res);
  ++g_launches;
}

// Full symmetric FP64 copy of a lower-stored FP32 matrix (inspection only).
__global__ void k_sym_unpack(const float* __restrict__ A, int n, double* __restrict__ out) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  out[e] = (double)(i >= j ? A[(size_t)i * n + j] : A[(size_t)j * n + i]);
}
void launch_sym_unpack(const float* A, int n, double* out, cudaStream_t s) {
  size_t tot = (size_t)n * n;
  k_sym_unpack<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A, n, out);
  ++g_launches;
}

template void launch_trsv_dag<float>(const BatchTabs&, int, bool, bool, cudaStream_t);
template void launch_trsv_dag<double>(const BatchTabs&, int, bool, bool, cudaStream_t);

}  // namespace ds
