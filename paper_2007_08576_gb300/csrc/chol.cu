// Cholesky factorisation and triangular solves of the damped normal equations (Section 2:
// "we perform Cholesky decomposition to update W_i"), for T = double (FP64 factor) or
// T = float (FP32 factor), plus the FP64 residual of the refinement steps.
//
// Layout: A is n x n row-major; only the lower triangle (row >= col) is read or written. The
// factorisation is right-looking and blocked with NB = 32 columns per panel:
//   panel kernel  : every CTA factors the NB x NB diagonal block in shared memory and inverts
//                   it; CTA 0 stores L_kk and L_kk^-1 (Dinv), the others solve
//                   L_ik = A_ik L_kk^-T for their RB rows of the panel as a product with L_kk^-T;
//   update kernel : A_ij -= L_ik L_jk^T on 64 x 64 tiles of the trailing lower triangle.
// A pivot <= 0 (or NaN) is recorded in acc[ACC_STATUS] as 1 + its row and replaced by 1 so that
// the remaining launches stay finite; the host reports DS_ERR_NOT_SPD.
// Triangular solves use the stored inverses of the diagonal blocks: forward y_k = Dinv_k r_k,
// then r_i -= L_ik y_k below; backward x_k = Dinv_k^T r_k, then r_j -= L_kj^T x_k to the left.
#include <math.h>

#include "ds_internal.cuh"

namespace ds {

constexpr int NB = 32;    // panel width
constexpr int RB = 64;    // panel rows per CTA in the panel kernel
constexpr int TS = 64;    // trailing-update tile

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

// Factor the nb x nb lower block in shared memory (L[i][j], stride NB+1) and write its inverse
// into Li (same layout). 256 threads.
template <typename T>
__device__ void factor_invert_diag(T (*L)[NB + 1], T (*Li)[NB + 1], int nb, int k0,
                                   double* acc) {
  const int tid = threadIdx.x;
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      T d = L[j][j];
      if (!(d > (T)0)) {
        if (acc) atomicCAS((unsigned long long*)&acc[ACC_STATUS], 0ull,
                           __double_as_longlong((double)(k0 + j + 1)));
        d = (T)1;
      }
      L[j][j] = tsqrt(d);
    }
    __syncthreads();
    T piv = L[j][j];
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) L[i][j] /= piv;
    __syncthreads();
    // trailing update of the block: rows i > j, cols j < c <= i
    int m = nb - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) L[i][c] -= L[i][j] * L[c][j];
    }
    __syncthreads();
  }
  // inverse of the lower-triangular L: column c by forward substitution, one row at a time
  for (int i = 0; i < nb; ++i) {
    for (int c = tid; c <= i; c += blockDim.x) {
      T v;
      if (c == i) {
        v = (T)1 / L[i][i];
      } else {
        T s = (T)0;
        for (int k = c; k < i; ++k) s += L[i][k] * Li[k][c];
        v = -s / L[i][i];
      }
      Li[i][c] = v;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ __launch_bounds__(256) void k_chol_panel(T* __restrict__ A, int n, int k0,
                                                    T* __restrict__ Dinv, double* acc) {
  __shared__ T L[NB][NB + 1];
  __shared__ T Li[NB][NB + 1];
  const int nb = min(NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int i = e / NB, j = e % NB;
    L[i][j] = (i < nb && j <= i) ? A[(size_t)(k0 + i) * n + k0 + j] : (T)0;
    Li[i][j] = (T)0;
  }
  __syncthreads();
  factor_invert_diag<T>(L, Li, nb, k0, blockIdx.x == 0 ? acc : nullptr);
  if (blockIdx.x == 0) {
    T* D = Dinv + (size_t)(k0 / NB) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      if (i < nb && j <= i) A[(size_t)(k0 + i) * n + k0 + j] = L[i][j];
      D[e] = (i < nb && j <= i) ? Li[i][j] : (T)0;
    }
    return;
  }
  // rows of this CTA: X = B L^-T, X[r][j] = sum_{m <= j} B[r][m] Li[j][m]
  __shared__ T Bs[RB][NB + 1];
  const int r0 = k0 + nb + (blockIdx.x - 1) * RB;
  const int rows = min(RB, n - r0);
  for (int e = threadIdx.x; e < RB * NB; e += blockDim.x) {
    int r = e / NB, j = e % NB;
    Bs[r][j] = (r < rows && j < nb) ? A[(size_t)(r0 + r) * n + k0 + j] : (T)0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
    int r = e / nb, j = e % nb;
    T s = (T)0;
    for (int m = 0; m <= j; ++m) s += Bs[r][m] * Li[j][m];
    A[(size_t)(r0 + r) * n + k0 + j] = s;
  }
}

// A[i][j] -= sum_m L[i][k0+m] L[j][k0+m], m < nb, for the lower tiles of the trailing matrix.
template <typename T>
__global__ __launch_bounds__(256) void k_chol_update(T* __restrict__ A, int n, int k0, int nb,
                                                     int nt) {
  // blockIdx.x -> lower tile (I, J), I >= J, of the nt x nt trailing tile grid
  int t = blockIdx.x;
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  int J = t - I * (I + 1) / 2;
  const int s0 = k0 + nb;
  const int i0 = s0 + I * TS, j0 = s0 + J * TS;
  __shared__ T Ls[TS][NB + 1];
  __shared__ T Ms[TS][NB + 1];
  for (int e = threadIdx.x; e < TS * NB; e += blockDim.x) {
    int r = e / NB, m = e % NB;
    Ls[r][m] = (i0 + r < n && m < nb) ? A[(size_t)(i0 + r) * n + k0 + m] : (T)0;
    Ms[r][m] = (j0 + r < n && m < nb) ? A[(size_t)(j0 + r) * n + k0 + m] : (T)0;
  }
  __syncthreads();
  // 256 threads, 4 x 4 outputs each
  const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
  T c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) c[a][bb] = (T)0;
  for (int m = 0; m < NB; ++m) {
    T x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = Ls[tr + a][m];
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) y[bb] = Ms[tc + bb][m];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) c[a][bb] += x[a] * y[bb];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int i = i0 + tr + a;
    if (i >= n) continue;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      int j = j0 + tc + bb;
      if (j < n && j <= i) A[(size_t)i * n + j] -= c[a][bb];
    }
  }
}

template <typename T>
void launch_cholesky(T* A, int n, T* Dinv, double* acc, cudaStream_t s) {
  for (int k0 = 0; k0 < n; k0 += NB) {
    int nb = min(NB, n - k0);
    int below = n - k0 - nb;
    int grid = 1 + (below + RB - 1) / RB;
    k_chol_panel<T><<<grid, 256, 0, s>>>(A, n, k0, Dinv, acc);
    ++g_launches;
    if (below > 0) {
      int nt = (below + TS - 1) / TS;
      k_chol_update<T><<<nt * (nt + 1) / 2, 256, 0, s>>>(A, n, k0, nb, nt);
      ++g_launches;
    }
  }
}

// ----------------------------------------------------------------------------- solves

// forward step k: y_k = Dinv_k r_k (every CTA computes it; CTA 0 stores it), then rows below
// the block: r_i -= L[i, k-block] y_k. One warp per row.
template <typename T>
__global__ __launch_bounds__(256) void k_trsv_fwd(const T* __restrict__ L,
                                                  const T* __restrict__ Dinv, int n, int kb,
                                                  T* __restrict__ r, T* __restrict__ y) {
  __shared__ T ys[NB];
  const int k0 = kb * NB, nb = min(NB, n - k0);
  const T* D = Dinv + (size_t)kb * NB * NB;
  if (threadIdx.x < nb) {
    T s = (T)0;
    for (int m = 0; m <= (int)threadIdx.x; ++m) s += D[threadIdx.x * NB + m] * r[k0 + m];
    ys[threadIdx.x] = s;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nb) y[k0 + threadIdx.x] = ys[threadIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = k0 + nb + blockIdx.x * 8 + warp;
  if (row < n) {
    T s = lane < nb ? L[(size_t)row * n + k0 + lane] * ys[lane] : (T)0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) r[row] -= s;
  }
}

// backward step k: x_k = Dinv_k^T r_k, then r_j -= sum_{i in block k} L[i][j] x_i for j < k0.
template <typename T>
__global__ __launch_bounds__(256) void k_trsv_bwd(const T* __restrict__ L,
                                                  const T* __restrict__ Dinv, int n, int kb,
                                                  T* __restrict__ r, T* __restrict__ x) {
  __shared__ T xs[NB];
  const int k0 = kb * NB, nb = min(NB, n - k0);
  const T* D = Dinv + (size_t)kb * NB * NB;
  if (threadIdx.x < nb) {
    T s = (T)0;
    for (int m = threadIdx.x; m < nb; ++m) s += D[m * NB + threadIdx.x] * r[k0 + m];
    xs[threadIdx.x] = s;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nb) x[k0 + threadIdx.x] = xs[threadIdx.x];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k0) {
    T s = (T)0;
    for (int i = 0; i < nb; ++i) s += L[(size_t)(k0 + i) * n + j] * xs[i];
    r[j] -= s;
  }
}

template <typename T>
void launch_trsv(const T* L, const T* Dinv, int n, const T* rhs, T* x, T* tmp, cudaStream_t s) {
  // tmp holds the running right-hand side; x receives y then the solution
  cudaMemcpyAsync(tmp, rhs, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
  int nblk = (n + NB - 1) / NB;
  for (int kb = 0; kb < nblk; ++kb) {
    int below = n - (kb * NB + min(NB, n - kb * NB));
    int grid = max(1, (below + 7) / 8);
    k_trsv_fwd<T><<<grid, 256, 0, s>>>(L, Dinv, n, kb, tmp, x);
    ++g_launches;
  }
  cudaMemcpyAsync(tmp, x, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
  for (int kb = nblk - 1; kb >= 0; --kb) {
    int left = kb * NB;
    int grid = max(1, (left + 255) / 256);
    k_trsv_bwd<T><<<grid, 256, 0, s>>>(L, Dinv, n, kb, tmp, x);
    ++g_launches;
  }
}

// r = b - A x with A the full symmetric FP32 matrix, accumulated in FP64. One warp per row.
__global__ __launch_bounds__(256) void k_residual64(const float* __restrict__ A, int n,
                                                    const double* __restrict__ b,
                                                    const double* __restrict__ x,
                                                    double* __restrict__ r) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* a = A + (size_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += (double)a[j] * x[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[row] = b[row] - s;
}

void launch_residual64(const float* Aref, int n, const double* b, const double* x, double* r,
                       cudaStream_t s) {
  k_residual64<<<(n + 7) / 8, 256, 0, s>>>(Aref, n, b, x, r);
  ++g_launches;
}

template <typename T>
__global__ void k_cast_from64(const double* __restrict__ in, T* __restrict__ out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)in[i];
}
template <typename T>
void launch_cast_from64(const double* in, T* out, int n, cudaStream_t s) {
  k_cast_from64<T><<<(n + 255) / 256, 256, 0, s>>>(in, out, n);
  ++g_launches;
}

template <typename T>
__global__ void k_axpy_to64(const T* __restrict__ d, double* __restrict__ x, int n, int assign) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = assign ? (double)d[i] : x[i] + (double)d[i];
}
template <typename T>
void launch_axpy_to64(const T* d, double* x, int n, bool assign, cudaStream_t s) {
  k_axpy_to64<T><<<(n + 255) / 256, 256, 0, s>>>(d, x, n, assign ? 1 : 0);
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

template void launch_cholesky<float>(float*, int, float*, double*, cudaStream_t);
template void launch_cholesky<double>(double*, int, double*, double*, cudaStream_t);
template void launch_trsv<float>(const float*, const float*, int, const float*, float*, float*,
                                 cudaStream_t);
template void launch_trsv<double>(const double*, const double*, int, const double*, double*,
                                  double*, cudaStream_t);
template void launch_cast_from64<float>(const double*, float*, int, cudaStream_t);
template void launch_cast_from64<double>(const double*, double*, int, cudaStream_t);
template void launch_axpy_to64<float>(const float*, double*, int, bool, cudaStream_t);
template void launch_axpy_to64<double>(const double*, double*, int, bool, cudaStream_t);

}  // namespace ds
