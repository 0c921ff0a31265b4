// 1-point RANSAC + reweighting inlier preselection (Section 2.1, Eq. 2-4).
//
// One CTA per reference match k0. The CTA rectifies both 3D match sets to k0 (Eq. 2) into
// shared memory (FP64, 56 B per match: S1, S2, w), then alternates n_reweight times
//   R <- rotation maximising sum_k w_k S2(k)^T R S1(k)        (Eq. 3, weighted)
//   d_k = |S2(k) - R S1(k)|,  w_k = min(H / d_k, 1)            (Eq. 4)
// The rotation is Horn's unit quaternion: the eigenvector of the largest eigenvalue of the 4x4
// symmetric matrix built from M = sum_k w_k S1(k) S2(k)^T. The largest eigenvalue is found by
// Newton's method on the characteristic polynomial from a Gershgorin upper bound (monotone for
// a polynomial with real roots), the eigenvector as the dominant column of the adjugate of
// N - lambda I. A fit is degenerate (R = I) if sum w < 1e-12 or the two largest eigenvalues are
// within 2e-12 |M|_F of each other.
// After the last update the CTA writes its score sum_{k != k0} w_k, a bitset of d_k <= H
// (warp ballots) and its weights; a second kernel keeps references whose score is at least
// keep_frac times the best and combines them (mask = OR, weight = max).
// Everything that decides a mask bit is FP64.
#include <math.h>

#include <mutex>

#include "ds_internal.cuh"

namespace ds {

static constexpr int kRansacThreads = 256;

__device__ __forceinline__ double det3(double a, double b, double c, double d, double e, double f,
                                       double g, double h, double i) {
  return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}

// Rotation matrix (row-major) from M[a][b] = sum w S1_a S2_b. Returns false if degenerate.
__device__ bool horn_rotation(const double* M, double wsum, double* R) {
  double Sxx = M[0], Sxy = M[1], Sxz = M[2];
  double Syx = M[3], Syy = M[4], Syz = M[5];
  double Szx = M[6], Szy = M[7], Szz = M[8];
  double fro = 0.0;
  for (int i = 0; i < 9; ++i) fro += M[i] * M[i];
  fro = sqrt(fro);
  if (!(wsum >= 1e-12) || !(fro > 0.0)) return false;
  double N[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                    {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                    {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                    {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
  // det(lambda I - N) = lambda^4 + e2 lambda^2 - e3 lambda + e4 (N is traceless)
  double e2 = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) e2 += N[i][i] * N[j][j] - N[i][j] * N[i][j];
  double e3 = 0.0;
  for (int skip = 0; skip < 4; ++skip) {
    int r[3], c = 0;
    for (int i = 0; i < 4; ++i)
      if (i != skip) r[c++] = i;
    e3 += det3(N[r[0]][r[0]], N[r[0]][r[1]], N[r[0]][r[2]], N[r[1]][r[0]], N[r[1]][r[1]],
               N[r[1]][r[2]], N[r[2]][r[0]], N[r[2]][r[1]], N[r[2]][r[2]]);
  }
  double e4 = 0.0;
  for (int j = 0; j < 4; ++j) {
    int c[3], k = 0;
    for (int i = 0; i < 4; ++i)
      if (i != j) c[k++] = i;
    double m = det3(N[1][c[0]], N[1][c[1]], N[1][c[2]], N[2][c[0]], N[2][c[1]], N[2][c[2]],
                    N[3][c[0]], N[3][c[1]], N[3][c[2]]);
    e4 += ((j & 1) ? -1.0 : 1.0) * N[0][j] * m;
  }
  // Newton from a Gershgorin bound
  double lam = -INFINITY;
  for (int i = 0; i < 4; ++i) {
    double r = N[i][i];
    for (int j = 0; j < 4; ++j)
      if (j != i) r += fabs(N[i][j]);
    lam = fmax(lam, r);
  }
  for (int it = 0; it < 100; ++it) {
    double l2 = lam * lam;
    double p = (l2 + e2) * l2 - e3 * lam + e4;
    double dp = 4.0 * l2 * lam + 2.0 * e2 * lam - e3;
    if (!(dp > 0.0)) break;
    double step = p / dp;
    double nl = lam - step;
    if (!(nl < lam)) break;
    lam = nl;
    if (step <= 1e-16 * fabs(lam)) break;
  }
  // deflate: p(x) / (x - lam) = x^3 + c2 x^2 + c1 x + c0, largest root by Newton from lam
  double c2 = lam, c1 = e2 + lam * lam, c0 = -e3 + lam * c1;
  double mu = lam;
  for (int it = 0; it < 100; ++it) {
    double p = ((mu + c2) * mu + c1) * mu + c0;
    double dp = (3.0 * mu + 2.0 * c2) * mu + c1;
    if (!(dp > 0.0)) break;
    double step = p / dp;
    double nm = mu - step;
    if (!(nm < mu)) break;
    mu = nm;
    if (step <= 1e-16 * fabs(mu) + 1e-300) break;
  }
  if (!(lam - mu > 2e-12 * fro)) return false;
  // adjugate of A = N - lam I: choose the largest diagonal cofactor, take its column
  double A[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) A[i][j] = N[i][j] - (i == j ? lam : 0.0);
  double best = -1.0;
  int jb = 0;
  for (int j = 0; j < 4; ++j) {
    int r[3], k = 0;
    for (int i = 0; i < 4; ++i)
      if (i != j) r[k++] = i;
    double m = fabs(det3(A[r[0]][r[0]], A[r[0]][r[1]], A[r[0]][r[2]], A[r[1]][r[0]],
                         A[r[1]][r[1]], A[r[1]][r[2]], A[r[2]][r[0]], A[r[2]][r[1]],
                         A[r[2]][r[2]]));
    if (m > best) {
      best = m;
      jb = j;
    }
  }
  double q[4];
  {
    int cols[3], k = 0;
    for (int i = 0; i < 4; ++i)
      if (i != jb) cols[k++] = i;
    for (int i = 0; i < 4; ++i) {
      int rows[3], kk = 0;
      for (int t = 0; t < 4; ++t)
        if (t != i) rows[kk++] = t;
      // cofactor C_{i, jb}: delete row i, column jb (A symmetric, so this is column jb of adj)
      double m = det3(A[rows[0]][cols[0]], A[rows[0]][cols[1]], A[rows[0]][cols[2]],
                      A[rows[1]][cols[0]], A[rows[1]][cols[1]], A[rows[1]][cols[2]],
                      A[rows[2]][cols[0]], A[rows[2]][cols[1]], A[rows[2]][cols[2]]);
      q[i] = (((i + jb) & 1) ? -1.0 : 1.0) * m;
    }
  }
  double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0.0)) return false;
  double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
  return true;
}

// FP64 template point at pixel j, ((u - cx) z) / fx with single roundings.
__device__ __forceinline__ void tmpl_point64(const float* depth0, int W, double fx, double fy,
                                             double cx, double cy, int j, double* o) {
  int u = j % W, v = j / W;
  double z = (double)depth0[j];
  o[0] = __ddiv_rn(__dmul_rn(__dsub_rn((double)u, cx), z), fx);
  o[1] = __ddiv_rn(__dmul_rn(__dsub_rn((double)v, cy), z), fy);
  o[2] = z;
}

template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* red /* NV * 32 */) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * 32 + warp] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += red[i * 32 + w];  // fixed order
    v[i] = x;
  }
  __syncthreads();
}

__global__ __launch_bounds__(kRansacThreads) void k_ransac_hyp(
    const float* __restrict__ depth0, int W, double fx, double fy, double cx, double cy,
    const int* __restrict__ midx, const float* __restrict__ mxyz, int M,
    const int* __restrict__ hyp, int n_reweight, double H, const double* __restrict__ o1w,
    int use_smem,
    double* __restrict__ scratch, uint32_t* __restrict__ hbits, float* __restrict__ hw,
    double* __restrict__ score) {
  extern __shared__ double sm[];
  __shared__ double red[10 * 32];
  __shared__ double sR[9];
  const int h = blockIdx.x;
  const int k0 = hyp[h];
  double* S = use_smem ? sm : scratch + (size_t)h * 7 * M;
  double* S1x = S;
  double* S1y = S + M;
  double* S1z = S + 2 * M;
  double* S2x = S + 3 * M;
  double* S2y = S + 4 * M;
  double* S2z = S + 5 * M;
  double* w = S + 6 * M;
  double r1[3], r2[3];
  // o1 of match k: the template point at its pixel, or the given (warm-start) point
  auto o1_of = [&](int k, double* o) {
    if (o1w) {
      o[0] = o1w[3 * k];
      o[1] = o1w[3 * k + 1];
      o[2] = o1w[3 * k + 2];
    } else {
      tmpl_point64(depth0, W, fx, fy, cx, cy, midx[k], o);
    }
  };
  o1_of(k0, r1);
  r2[0] = (double)mxyz[3 * k0 + 0];
  r2[1] = (double)mxyz[3 * k0 + 1];
  r2[2] = (double)mxyz[3 * k0 + 2];
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    double o1[3];
    o1_of(k, o1);
    S1x[k] = o1[0] - r1[0];
    S1y[k] = o1[1] - r1[1];
    S1z[k] = o1[2] - r1[2];
    S2x[k] = (double)mxyz[3 * k + 0] - r2[0];
    S2y[k] = (double)mxyz[3 * k + 1] - r2[1];
    S2z[k] = (double)mxyz[3 * k + 2] - r2[2];
    w[k] = 1.0;
  }
  __syncthreads();
  const int words = (M + 31) / 32;
  const double H2 = H * H;
  for (int it = 0; it < n_reweight; ++it) {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      double wk = w[k];
      double a0 = wk * S1x[k], a1 = wk * S1y[k], a2 = wk * S1z[k];
      double b0 = S2x[k], b1 = S2y[k], b2 = S2z[k];
      acc[0] += a0 * b0;
      acc[1] += a0 * b1;
      acc[2] += a0 * b2;
      acc[3] += a1 * b0;
      acc[4] += a1 * b1;
      acc[5] += a1 * b2;
      acc[6] += a2 * b0;
      acc[7] += a2 * b1;
      acc[8] += a2 * b2;
      acc[9] += wk;
    }
    block_sum<10>(acc, red);
    if (threadIdx.x == 0) {
      double R[9];
      if (!horn_rotation(acc, acc[9], R)) {
        for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
      }
      for (int i = 0; i < 9; ++i) sR[i] = R[i];
    }
    __syncthreads();
    double R0 = sR[0], R1 = sR[1], R2 = sR[2], R3 = sR[3], R4 = sR[4], R5 = sR[5], R6 = sR[6],
           R7 = sR[7], R8 = sR[8];
    const bool last = it == n_reweight - 1;
    double sc = 0.0;
    // warp-uniform trip count so that every lane reaches the ballot
    for (int base = (threadIdx.x & ~31); base < M; base += blockDim.x) {
      int k = base + (threadIdx.x & 31);
      bool inl = false;
      if (k < M) {
        double x = S1x[k], y = S1y[k], z = S1z[k];
        double e0 = S2x[k] - (R0 * x + R1 * y + R2 * z);
        double e1 = S2y[k] - (R3 * x + R4 * y + R5 * z);
        double e2 = S2z[k] - (R6 * x + R7 * y + R8 * z);
        // d <= H  <=>  d^2 <= H^2, and w = H / d = H rsqrt(d^2) when d > H: no FP64 sqrt or
        // division (each costs tens of instructions on the FP64 pipe)
        const double d2 = e0 * e0 + e1 * e1 + e2 * e2;
        const bool within = d2 <= H2;
        double wk = 1.0;
        if (!within) {
          double y0 = (double)rsqrtf((float)d2);
          y0 = y0 * (1.5 - 0.5 * d2 * y0 * y0);
          y0 = y0 * (1.5 - 0.5 * d2 * y0 * y0);
          wk = fmin(H * y0, 1.0);
        }
        w[k] = wk;
        if (last) {
          inl = within;
          hw[(size_t)h * M + k] = (float)wk;
          if (k != k0) sc += wk;
        }
      }
      if (last) {
        uint32_t bits = __ballot_sync(0xffffffffu, inl);
        if ((threadIdx.x & 31) == 0) hbits[(size_t)h * words + base / 32] = bits;
      }
    }
    if (last) {
      double v[1] = {sc};
      block_sum<1>(v, red);
      if (threadIdx.x == 0) score[h] = v[0];
    }
    __syncthreads();
  }
}

// Keep references with score >= keep_frac * best; mask = OR of kept bitsets, weight = max of
// kept weights. Every CTA derives the kept set from the scores itself and handles a slice of the
// matches; CTA 0 also writes the kept bitset and the counts.
__global__ void k_ransac_combine(const uint32_t* __restrict__ hbits, const float* __restrict__ hw,
                                 const double* __restrict__ score, int n_hyp, int M,
                                 double keep_frac, uint32_t* __restrict__ mask,
                                 float* __restrict__ what, uint32_t* __restrict__ kept,
                                 int* __restrict__ counts) {
  __shared__ uint32_t skept[2];
  __shared__ int sin;
  if (threadIdx.x == 0) {
    double best = -INFINITY;
    for (int h = 0; h < n_hyp; ++h) best = fmax(best, score[h]);
    uint32_t k0 = 0, k1 = 0;
    int nk = 0;
    for (int h = 0; h < n_hyp; ++h)
      if (score[h] >= keep_frac * best) {
        if (h < 32)
          k0 |= 1u << h;
        else
          k1 |= 1u << (h - 32);
        ++nk;
      }
    skept[0] = k0;
    skept[1] = k1;
    if (blockIdx.x == 0) {
      kept[0] = k0;
      kept[1] = k1;
      counts[1] = nk;
    }
    sin = 0;
  }
  __syncthreads();
  const int words = (M + 31) / 32;
  // this CTA: matches [blockIdx.x * 256, +256) = words [blockIdx.x * 8, +8)
  int local = 0;
  const int wd = blockIdx.x * 8 + (threadIdx.x >> 5);
  if ((threadIdx.x & 31) == 0 && wd < words) {
    uint32_t m = 0;
    for (int h = 0; h < n_hyp; ++h)
      if ((skept[h >> 5] >> (h & 31)) & 1u) m |= hbits[(size_t)h * words + wd];
    if (wd == words - 1 && (M & 31)) m &= (1u << (M & 31)) - 1u;
    mask[wd] = m;
    local = __popc(m);
  }
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (k < M) {
    float b = 0.f;
    for (int h = 0; h < n_hyp; ++h)
      if ((skept[h >> 5] >> (h & 31)) & 1u) b = fmaxf(b, hw[(size_t)h * M + k]);
    what[k] = b;
  }
  if (local) atomicAdd(&sin, local);
  __syncthreads();
  if (threadIdx.x == 0 && sin) atomicAdd(&counts[0], sin);
}

int ransac_smem_bytes(int M) { return 7 * (int)sizeof(double) * M; }

void launch_ransac(const float* depth0, int W, ds_intrinsics K, const int* midx,
                   const float* mxyz, int M, const int* hyp, int n_hyp, int n_reweight, double H,
                   double keep_frac, const double* o1w, double* scratch, uint32_t* hbits,
                   float* hw, double* score, uint32_t* mask, float* what, uint32_t* kept,
                   int* counts, cudaStream_t s) {
  if (M <= 0 || n_hyp <= 0) return;
  int sm = ransac_smem_bytes(M);
  int use_smem = sm <= 220 * 1024;
  if (use_smem) {
    static bool attr_done = false;
    if (!attr_done) {
      cudaFuncSetAttribute(k_ransac_hyp, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
      attr_done = true;
    }
  } else {
    sm = 0;
  }
  k_ransac_hyp<<<n_hyp, kRansacThreads, sm, s>>>(depth0, W, K.fx, K.fy, K.cx, K.cy, midx, mxyz,
                                                 M, hyp, n_reweight, H, o1w, use_smem, scratch,
                                                 hbits, hw, score);
  ++g_launches;
  cudaMemsetAsync(counts, 0, sizeof(int), s);  // counts[0] is accumulated by every CTA
  k_ransac_combine<<<(M + 255) / 256, 256, 0, s>>>(hbits, hw, score, n_hyp, M, keep_frac, mask,
                                                     what, kept, counts);
  ++g_launches;
}

// ----------------------------------------------------------------------------- warm-start o1

// o1 of match k = its template point p warped by the current state (the reading of Section 2.1
// where the rigid preselection starts from the previous frame's deformation instead of the
// template), in FP64 throughout so that the RANSAC decisions stay those of an FP64 pipeline:
// the point's 4 nodes (its segment), blend weights exp(-|p - g|^2 / (2 sigma_b^2)) normalised
// to 1, node dual quaternions (q, 1/2 (0, T) (x) q) with T = g + t - R g, each sign-aligned to
// the nearest node's quaternion, blended and applied: x' = (b_r p b_r* + 2 b_d b_r*) / |b_r|^2.
// One thread per match.
__global__ void k_warm_o1(const int* __restrict__ midx, int M, const int* __restrict__ rank,
                          const float4* __restrict__ tp, const int4* __restrict__ seg,
                          const double* __restrict__ X64, const double* __restrict__ g64,
                          const double* __restrict__ q64, const double* __restrict__ t64,
                          double inv2s2, double* __restrict__ o1) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const int j = midx[k];
  const int sp = rank[j];
  const int bits = __float_as_int(tp[sp].w);
  const int4 nn = seg[bits >> 2];
  const int near = bits & 3;
  const int ids[4] = {nn.x, nn.y, nn.z, nn.w};
  const double px = X64[3 * j], py = X64[3 * j + 1], pz = X64[3 * j + 2];
  const int in = ids[near];
  const double nw = q64[4 * in], nx = q64[4 * in + 1], ny = q64[4 * in + 2], nz = q64[4 * in + 3];
  double a[4], asum = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = ids[s];
    const double dx = px - g64[3 * i], dy = py - g64[3 * i + 1], dz = pz - g64[3 * i + 2];
    a[s] = exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
    asum += a[s];
  }
  double bw = 0, bx = 0, by = 0, bz = 0, cw = 0, cx = 0, cy = 0, cz = 0;  // b_r, b_d
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = ids[s];
    const double qw = q64[4 * i], qx = q64[4 * i + 1], qy = q64[4 * i + 2], qz = q64[4 * i + 3];
    const double gx = g64[3 * i], gy = g64[3 * i + 1], gz = g64[3 * i + 2];
    // R g
    const double Rgx = (1 - 2 * (qy * qy + qz * qz)) * gx + 2 * (qx * qy - qw * qz) * gy +
                       2 * (qx * qz + qw * qy) * gz;
    const double Rgy = 2 * (qx * qy + qw * qz) * gx + (1 - 2 * (qx * qx + qz * qz)) * gy +
                       2 * (qy * qz - qw * qx) * gz;
    const double Rgz = 2 * (qx * qz - qw * qy) * gx + 2 * (qy * qz + qw * qx) * gy +
                       (1 - 2 * (qx * qx + qy * qy)) * gz;
    const double Tx = gx + t64[3 * i] - Rgx, Ty = gy + t64[3 * i + 1] - Rgy,
                 Tz = gz + t64[3 * i + 2] - Rgz;
    // d = 1/2 (0, T) (x) q
    const double dw = 0.5 * (-Tx * qx - Ty * qy - Tz * qz);
    const double dx = 0.5 * (Tx * qw + Ty * qz - Tz * qy);
    const double dy = 0.5 * (-Tx * qz + Ty * qw + Tz * qx);
    const double dz = 0.5 * (Tx * qy - Ty * qx + Tz * qw);
    const double sg = (qw * nw + qx * nx + qy * ny + qz * nz) >= 0.0 ? 1.0 : -1.0;
    const double w = sg * (a[s] / asum);
    bw += w * qw; bx += w * qx; by += w * qy; bz += w * qz;
    cw += w * dw; cx += w * dx; cy += w * dy; cz += w * dz;
  }
  // y = vec(b_r (x) (0, p) (x) b_r*) + 2 vec(b_d (x) b_r*)
  const double bvp = bx * px + by * py + bz * pz;
  const double bvv = bx * bx + by * by + bz * bz;
  const double s2 = bw * bw + bvv;
  const double k0 = bw * bw - bvv;
  double yx = k0 * px + 2 * bvp * bx + 2 * bw * (by * pz - bz * py);
  double yy = k0 * py + 2 * bvp * by + 2 * bw * (bz * px - bx * pz);
  double yz = k0 * pz + 2 * bvp * bz + 2 * bw * (bx * py - by * px);
  // vec(b_d (x) b_r*) = bw c_v - cw b_v - c_v x b_v
  yx += 2 * (bw * cx - cw * bx - (cy * bz - cz * by));
  yy += 2 * (bw * cy - cw * by - (cz * bx - cx * bz));
  yz += 2 * (bw * cz - cw * bz - (cx * by - cy * bx));
  o1[3 * k] = yx / s2;
  o1[3 * k + 1] = yy / s2;
  o1[3 * k + 2] = yz / s2;
}

void launch_warm_o1(const int* midx, int M, const int* rank, const float4* tp, const int4* seg,
                    const double* X64, const double* g64, const double* q64, const double* t64,
                    double sigma_b, double* o1, cudaStream_t s) {
  if (M <= 0) return;
  k_warm_o1<<<(M + 127) / 128, 128, 0, s>>>(midx, M, rank, tp, seg, X64, g64, q64, t64,
                                             1.0 / (2.0 * sigma_b * sigma_b), o1);
  ++g_launches;
}

// ----------------------------------------------------------------------------- no-allocation entry

// Scratch of ds_ransac_noalloc: a file-scope device array, so the entry point never allocates.
// Limits: M <= DS_NOALLOC_MAX_MATCHES matches (the shared-memory path of the kernel, no global
// staging), n_hyp <= DS_MAX_HYP references. Layout (256-byte aligned sections): per-reference
// bitsets, per-reference weights, validated copies of the match and reference indices, the
// match count word and the invalid-index flag.
namespace {
constexpr int kNaWords = (DS_NOALLOC_MAX_MATCHES + 31) / 32;
constexpr size_t kNaAlign(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaBits = 0;
constexpr size_t kNaW = kNaBits + kNaAlign(sizeof(uint32_t) * DS_MAX_HYP * kNaWords);
constexpr size_t kNaMidx = kNaW + kNaAlign(sizeof(float) * DS_MAX_HYP * DS_NOALLOC_MAX_MATCHES);
constexpr size_t kNaHyp = kNaMidx + kNaAlign(sizeof(int) * DS_NOALLOC_MAX_MATCHES);
constexpr size_t kNaCnt = kNaHyp + kNaAlign(sizeof(int) * DS_MAX_HYP);
constexpr size_t kNaTotal = kNaCnt + 256;
}  // namespace

static __device__ __align__(256) unsigned char g_ransac_scratch[kNaTotal];

// Copies the caller's indices into the scratch, replacing any out-of-range template pixel or
// reference id by 0 (so no kernel reads out of bounds) and raising the flag.
__global__ void k_na_indices(const int* __restrict__ midx_in, int M, const int* __restrict__ hyp_in,
                             int n_hyp, int npx, const float* __restrict__ depth0,
                             int* __restrict__ midx, int* __restrict__ hyp, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) {
    int j = midx_in[i];
    if (j < 0 || j >= npx || !(depth0[j] > 0.f)) {
      j = 0;
      atomicOr(flag, 1);
    }
    midx[i] = j;
  }
  if (i < n_hyp) {
    int k = hyp_in[i];
    if (k < 0 || k >= M) {
      k = 0;
      atomicOr(flag, 1);
    }
    hyp[i] = k;
  }
}

}  // namespace ds

namespace {
bool device_memory(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" int ds_ransac_noalloc(const float* depth0, int32_t W, int32_t H, ds_intrinsics K,
                                 const int32_t* match_tmpl_idx, const float* match_xyz, int32_t M,
                                 const int32_t* hyp_list, int32_t n_hyp, int32_t n_reweight,
                                 double H_mm, double keep_frac, uint32_t* mask_bits, float* w_M,
                                 uint32_t* kept_bits, double* score_nh, void* cuda_stream) {
  using namespace ds;
  if (W < 8 || H < 8 || W > 4096 || H > 4096 || M < 1 || M > DS_NOALLOC_MAX_MATCHES ||
      n_hyp < 1 || n_hyp > DS_MAX_HYP || n_hyp > M || n_reweight < 1 || n_reweight > 1000 ||
      !(H_mm > 0) || !(keep_frac >= 0 && keep_frac <= 1) || !(K.fx > 0) || !(K.fy > 0))
    return DS_ERR_ARG;
  const void* ptrs[] = {depth0, match_tmpl_idx, match_xyz, hyp_list, mask_bits, w_M, kept_bits,
                        score_nh};
  for (const void* p : ptrs)
    if (!p || !device_memory(p)) return DS_ERR_ARG;
  // the scratch's device address, looked up once per device with that device current
  static std::mutex mu;
  static void* base_of[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DS_ERR_CUDA;
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!base_of[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_ransac_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DS_ERR_CUDA;
      }
      base_of[dev] = p;
      cudaFuncSetAttribute(k_ransac_hyp, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    }
    base = (unsigned char*)base_of[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  uint32_t* hbits = (uint32_t*)(base + kNaBits);
  float* hw = (float*)(base + kNaW);
  int* midx = (int*)(base + kNaMidx);
  int* hyp = (int*)(base + kNaHyp);
  int* counts = (int*)(base + kNaCnt);
  int* flag = counts + 2;
  // the array keeps the previous call's contents: clear the words that accumulate
  cudaMemsetAsync(counts, 0, 4 * sizeof(int), s);
  const int npx = W * H;
  const int nt = M > n_hyp ? M : n_hyp;
  k_na_indices<<<(nt + 255) / 256, 256, 0, s>>>(match_tmpl_idx, M, hyp_list, n_hyp, npx, depth0,
                                                 midx, hyp, flag);
  const int sm = ransac_smem_bytes(M);  // <= 220 KB for M <= DS_NOALLOC_MAX_MATCHES
  k_ransac_hyp<<<n_hyp, kRansacThreads, sm, s>>>(depth0, W, K.fx, K.fy, K.cx, K.cy, midx,
                                                 match_xyz, M, hyp, n_reweight, H_mm, nullptr, 1,
                                                 nullptr, hbits, hw, score_nh);
  k_ransac_combine<<<(M + 255) / 256, 256, 0, s>>>(hbits, hw, score_nh, n_hyp, M, keep_frac,
                                                     mask_bits, w_M, kept_bits, counts);
  if (cudaGetLastError() != cudaSuccess) return DS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DS_ERR_CUDA;
  int bad = 0;
  if (cudaMemcpy(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DS_ERR_CUDA;
  return bad ? DS_ERR_ARG : DS_OK;
}

