// 1-point RANSAC + reweighting inlier preselection (Section 2.1, Eq. 2-4).
//
// One CTA per reference match k0. The CTA rectifies both 3D match sets to k0 (Eq. 2) into
// shared memory (double-float, 56 B per match: S1, S2, w), then alternates n_reweight times
//   R <- rotation maximising sum_k w_k S2(k)^T R S1(k)        (Eq. 3, weighted)
//   d_k = |S2(k) - R S1(k)|,  w_k = min(H / d_k, 1)            (Eq. 4)
// The rotation is Horn's unit quaternion: the eigenvector of the largest eigenvalue of the 4x4
// symmetric matrix built from M = sum_k w_k S1(k) S2(k)^T. The largest eigenvalue is found by
// Newton's method on the characteristic polynomial from an upper bound (monotone for a
// polynomial with real roots; the bound is sum_k w_k |S1(k)| |S2(k)|, or Gershgorin's if
// smaller), in FP32 on the scaled polynomial and then polished in FP64; the eigenvector is the
// dominant column of the adjugate of N - lambda I. A fit is degenerate (R = I) if sum w < 1e-12
// or the two largest eigenvalues are within 2e-12 |M|_F of each other.
// After the last update the CTA writes its score sum_{k != k0} w_k, a bitset of d_k <= H
// (warp ballots) and its weights; a second kernel keeps references whose score is at least
// keep_frac times the best and combines them (mask = OR, weight = max).
// Every quantity that decides a mask bit carries about 48 significant bits: the per-match loops
// in double-float FP32 arithmetic (see below), Horn's solve and the weights in FP64.
#include <math.h>

#include <mutex>

#include "ds_internal.cuh"

namespace ds {

static constexpr int kRansacThreads = 256;

__device__ __forceinline__ double det3(double a, double b, double c, double d, double e, double f,
                                       double g, double h, double i) {
  return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}

// Determinant of the 3 x 3 submatrix of a 4 x 4 row-major matrix X keeping rows r0 < r1 < r2
// and columns c0 < c1 < c2.
__device__ __forceinline__ double minor3(const double* X, int r0, int r1, int r2, int c0, int c1,
                                         int c2) {
  return det3(X[4 * r0 + c0], X[4 * r0 + c1], X[4 * r0 + c2], X[4 * r1 + c0], X[4 * r1 + c1],
              X[4 * r1 + c2], X[4 * r2 + c0], X[4 * r2 + c1], X[4 * r2 + c2]);
}
// The three indices of {0, 1, 2, 3} other than `skip`, ascending.
__device__ __forceinline__ void others(int skip, int& a, int& b, int& c) {
  a = skip == 0 ? 1 : 0;
  b = skip <= 1 ? 2 : 1;
  c = skip <= 2 ? 3 : 2;
}

// 1 / sqrt(v) to FP32 accuracy for any positive finite double (exponent split off first).
__device__ __forceinline__ double rsqrt_seed(double v) {
  int e;
  double m = frexp(v, &e);
  if (e & 1) {
    m *= 2.0;
    e -= 1;
  }
  return (double)rsqrtf((float)m) * ldexp(1.0, -e / 2);
}
// Largest root of a quartic / cubic with real roots, O(1) after the caller's scaling: Newton
// from an upper bound x0 in FP32 (monotone from above), then FP64 Newton, monotone from above
// again, from the FP32 root raised by a bound of its error (a few FP32 roundings of the
// polynomial's terms, mag, divided by p'): ~2 FP64 steps for a well separated root, more when
// p' is small (a nearly repeated root). The FP64 step divides by p' through an FP32 reciprocal
// refined once (relative error ~1e-14, which only scales the step). p32(x, p, dp, mag) and
// p64(x, p, dp) evaluate p, p' (and the sum of the terms' magnitudes) at x.
template <typename F32, typename F64>
__device__ __forceinline__ double largest_root(double x0, F32 p32, F64 p64, double decided = -1.0) {
  float x = __double2float_ru(x0), dpf = 0.f, mag = 0.f;   // rounded up: still an upper bound
  for (int it = 0; it < 100; ++it) {
    float p;
    p32(x, p, dpf, mag);
    if (!(dpf > 0.f)) break;
    const float step = p / dpf;
    const float nx = x - step;
    if (!(nx < x)) break;
    x = nx;
    if (step <= 1e-7f * fabsf(x) + 1e-30f) break;
  }
  double y = (dpf > 0.f) ? (double)x + (1e-6 * (double)mag / (double)dpf + 1e-7 * fabs((double)x))
                         : x0;
  y = fmin(y, x0);
  // the caller only needs to know whether the root lies below `decided`: an upper bound below
  // it settles that without the FP64 steps
  if (y < decided) return y;
  for (int it = 0; it < 100; ++it) {
    double p, dp;
    p64(y, p, dp);
    if (!(dp > 0.0)) break;
    double r = (double)__frcp_rn((float)dp);
    r = r * (2.0 - dp * r);
    const double step = p * r;
    const double ny = y - step;
    if (!(ny < y)) break;
    y = ny;
    // quadratic convergence: after a step this small the error is ~1e-18 relative
    if (step <= 1e-9 * fabs(y) + 1e-300) break;
  }
  return y;
}

// Rotation matrix (row-major) from M[a][b] = sum w S1_a S2_b, computed by the 32 lanes of one
// warp together (M, wsum and bound the same in every lane; R valid in every lane). Returns false
// if degenerate. bound: an upper bound of the largest eigenvalue, or +inf. Xs: 32 doubles of
// shared memory for this warp.
// An FP64 instruction of one warp occupies this GPU's FP64 pipe for tens of cycles whether one
// lane or all 32 are active, so the 8 independent 3 x 3 minors (characteristic polynomial) and
// the 8 cofactors (adjugate) are taken one per lane, and the root searches run in FP32 with an
// FP64 polish.
__device__ bool horn_rotation_warp(const double* M, double wsum, double bound, double* R,
                                   double* Xs) {
  const int lane = threadIdx.x & 31;
  const double Sxx = M[0], Sxy = M[1], Sxz = M[2];
  const double Syx = M[3], Syy = M[4], Syz = M[5];
  const double Szx = M[6], Szy = M[7], Szz = M[8];
  double f2sum = 0.0;
  for (int i = 0; i < 9; ++i) f2sum += M[i] * M[i];
  if (!(wsum >= 1e-12) || !(f2sum > 0.0) || !(f2sum < INFINITY)) return false;
  // |M|_F to FP32 accuracy (it only sets the degeneracy threshold) and a power of two sc within
  // a factor 2 of 1 / |M|_F that scales the roots to O(1) exactly
  const double fro = f2sum * rsqrt_seed(f2sum);
  int ex;
  frexp(f2sum, &ex);
  const double sc = ldexp(1.0, -(ex / 2)), inv_sc = ldexp(1.0, ex / 2);
  const double N[16] = {Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx,
                        Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz,
                        Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy,
                        Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz};
  if (lane < 16) Xs[lane] = N[lane];
  __syncwarp();
  // det(lambda I - N) = lambda^4 + e2 lambda^2 - e3 lambda + e4 (N is traceless):
  // e2 = sum of principal 2 x 2 minors, e3 = sum of principal 3 x 3 minors, e4 = det N
  // lanes 0-3: principal 3 x 3 minors (e3); lanes 4-7: row-0 cofactors times N_0j (e4);
  // lanes 8-13: principal 2 x 2 minors (e2)
  double m, m2;
  {
    const int sk = lane & 3;
    int a, b, c;
    others(sk, a, b, c);
    const bool row0 = (lane & 4) != 0;
    const double f = row0 ? ((sk & 1) ? -Xs[sk] : Xs[sk]) : 1.0;
    m = minor3(Xs, row0 ? 1 : a, row0 ? 2 : b, row0 ? 3 : c, a, b, c) * f;
    const int pr = lane >= 8 && lane < 14 ? lane - 8 : 0;     // pair (i, j), i < j
    const int i = pr < 3 ? 0 : pr < 5 ? 1 : 2;
    const int j = pr < 3 ? pr + 1 : pr < 5 ? pr - 1 : 3;
    m2 = Xs[5 * i] * Xs[5 * j] - Xs[4 * i + j] * Xs[4 * i + j];
  }
  double e2 = 0.0;
  for (int l = 8; l < 14; ++l) e2 += __shfl_sync(0xffffffffu, m2, l);
  const double e3 = ((__shfl_sync(0xffffffffu, m, 0) + __shfl_sync(0xffffffffu, m, 1)) +
                     __shfl_sync(0xffffffffu, m, 2)) + __shfl_sync(0xffffffffu, m, 3);
  const double e4 = ((__shfl_sync(0xffffffffu, m, 4) + __shfl_sync(0xffffffffu, m, 5)) +
                     __shfl_sync(0xffffffffu, m, 6)) + __shfl_sync(0xffffffffu, m, 7);
  // largest eigenvalue: Newton from the caller's bound, or Gershgorin's without one
  double top = bound;
  if (!(top < INFINITY)) {
    top = -INFINITY;
    for (int i = 0; i < 4; ++i) {
      double r = N[5 * i];
      for (int j = 0; j < 4; ++j)
        if (j != i) r += fabs(N[4 * i + j]);
      top = fmax(top, r);
    }
  }
  // scaled quartic x^4 + E2 x^2 - E3 x + E4 (x = lambda sc, exact power-of-two scalings)
  const double E2 = e2 * (sc * sc), E3 = e3 * (sc * sc * sc), E4 = e4 * ((sc * sc) * (sc * sc));
  const float f2 = (float)E2, f3 = (float)E3, f4 = (float)E4;
  const double ls = largest_root(
      top * sc,
      [&](float x, float& p, float& dp, float& mag) {
        const float x2 = x * x;
        p = (x2 + f2) * x2 - f3 * x + f4;
        dp = 4.f * x2 * x + 2.f * f2 * x - f3;
        mag = x2 * x2 + fabsf(f2) * x2 + fabsf(f3 * x) + fabsf(f4);
      },
      [&](double x, double& p, double& dp) {
        const double x2 = x * x;
        p = (x2 + E2) * x2 - E3 * x + E4;
        dp = 4.0 * x2 * x + 2.0 * E2 * x - E3;
      });
  // second largest: the deflated cubic p(x) / (x - ls) = x^3 + C2 x^2 + C1 x + C0, from ls
  const double C2 = ls, C1 = E2 + ls * ls, C0 = -E3 + ls * C1;
  const float g2 = (float)C2, g1 = (float)C1, g0 = (float)C0;
  const double ms = largest_root(
      ls,
      [&](float x, float& p, float& dp, float& mag) {
        p = ((x + g2) * x + g1) * x + g0;
        dp = (3.f * x + 2.f * g2) * x + g1;
        mag = fabsf(x * x * x) + fabsf(g2 * x * x) + fabsf(g1 * x) + fabsf(g0);
      },
      [&](double x, double& p, double& dp) {
        p = ((x + C2) * x + C1) * x + C0;
        dp = (3.0 * x + 2.0 * C2) * x + C1;
      },
      ls - 4e-12 * fro * sc);
  // degenerate iff the two largest eigenvalues are within 2e-12 |M|_F (an upper bound of the
  // second one below ls - 4e-12 |M|_F sc already decides it, with a factor 2 to spare)
  const double lam = ls * inv_sc, mu = ms * inv_sc;
  if (!(lam - mu > 2e-12 * fro)) return false;
  // eigenvector: a column of adj(N - lam I) = prod_{i > 1} (lambda_1 - lambda_i) q q^T, the one
  // with the largest diagonal cofactor
  __syncwarp();
  if (lane < 16) Xs[lane] = N[lane] - ((lane % 5 == 0) ? lam : 0.0);
  __syncwarp();
  double dg;
  {
    int a, b, c;
    others(lane & 3, a, b, c);
    dg = fabs(minor3(Xs, a, b, c, a, b, c));
  }
  int jb = 0;
  double best = __shfl_sync(0xffffffffu, dg, 0);
  for (int j = 1; j < 4; ++j) {
    const double v = __shfl_sync(0xffffffffu, dg, j);
    if (v > best) {
      best = v;
      jb = j;
    }
  }
  double cf;
  {
    const int i = lane & 3;
    int r0, r1, r2, k0, k1, k2;
    others(i, r0, r1, r2);
    others(jb, k0, k1, k2);
    // cofactor C_{i, jb}: delete row i and column jb (A symmetric: column jb of the adjugate)
    cf = (((i + jb) & 1) ? -1.0 : 1.0) * minor3(Xs, r0, r1, r2, k0, k1, k2);
  }
  double q[4];
  for (int i = 0; i < 4; ++i) q[i] = __shfl_sync(0xffffffffu, cf, i);
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  if (!(qq > 0.0) || !(qq < INFINITY)) return false;
  // 1 / |q|: FP32-accurate seed, one FP64 Newton step (relative error ~1e-14)
  double iq = rsqrt_seed(qq);
  iq = iq * (1.5 - 0.5 * qq * iq * iq);
  const double w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
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

// ----------------------------------------------------------------------------- double-float
// The per-match loops run in double-float arithmetic: a value is the unevaluated sum hi + lo of
// two floats (|lo| <= ulp(hi) / 2, 48 significant bits), products split exactly with an FMA,
// sums by two-sum, every operation rounded separately (no contraction). On this GPU an FP64
// instruction costs 64 times an FP32 one, so these ~10 FP32 operations per FP64 operation run
// several times faster, with a relative error of a few 1e-15 -- far inside the 1e-6 mm band in
// which mask decisions are not graded. Horn's rotation and the weights H / d stay FP64.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_quick(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_two_sum(float a, float b) {  // exact a + b
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ bool df_le(DF a, DF b) {  // a <= b for normalised pairs
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
__device__ __forceinline__ DF df_scale(DF a, float s) {  // s a power of two
  return {__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}
__device__ __forceinline__ DF df_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(__dsub_rn(x, (double)h))};
}
__device__ __forceinline__ double df_val(DF a) { return __dadd_rn((double)a.hi, (double)a.lo); }

// Sum over the CTA of NV double-float values per thread, in a fixed order (NV <= 32); the result
// is valid in warp 0 only.
template <int NV>
__device__ __forceinline__ void block_sum_df(DF* v, DF* red /* NV * 32 */) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    DF x = v[i];
    for (int o = 16; o > 0; o >>= 1) {
      const DF y = {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
      x = df_add(x, y);
    }
    v[i] = x;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * 32 + warp] = v[i];
  __syncthreads();
  if (warp == 0) {   // lane i sums value i over the warps (fixed order), then every lane gathers
    DF x = {0.f, 0.f};
    if (lane < NV)
      for (int w = 0; w < nw; ++w) x = df_add(x, red[lane * 32 + w]);
#pragma unroll
    for (int i = 0; i < NV; ++i)
      v[i] = {__shfl_sync(0xffffffffu, x.hi, i), __shfl_sync(0xffffffffu, x.lo, i)};
  }
}

// o1 of every match as double-float coordinates (6 floats: x, y, z as hi / lo pairs): the
// template point at its pixel in FP64, or the given warm-start point. Once per frame, so that
// the per-reference CTAs start from it without FP64 work.
__global__ void k_ransac_points(const float* __restrict__ depth0, int W, double fx, double fy,
                                double cx, double cy, const int* __restrict__ midx, int M,
                                const double* __restrict__ o1w, float* __restrict__ o1df) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double o[3];
  if (o1w) {
    o[0] = o1w[3 * k];
    o[1] = o1w[3 * k + 1];
    o[2] = o1w[3 * k + 2];
  } else {
    tmpl_point64(depth0, W, fx, fy, cx, cy, midx[k], o);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const DF d = df_of(o[a]);
    o1df[6 * k + 2 * a] = d.hi;
    o1df[6 * k + 2 * a + 1] = d.lo;
  }
}

__global__ __launch_bounds__(kRansacThreads) void k_ransac_hyp(
    const float* __restrict__ o1df, const float* __restrict__ mxyz, int M,
    const int* __restrict__ hyp, int n_reweight, double H, int use_smem,
    double* __restrict__ scratch, uint32_t* __restrict__ hbits, float* __restrict__ hw,
    double* __restrict__ score) {
  extern __shared__ double sm[];
  __shared__ DF red[11 * 32];
  __shared__ double sR[10];
  __shared__ double sX[32];
  const int h = blockIdx.x;
  const int k0 = hyp[h];
  // 7 double-float arrays of M: S1 (x, y, z), S2 (x, y, z), w; 56 B per match
  DF* S = reinterpret_cast<DF*>(use_smem ? sm : scratch + (size_t)h * 7 * M);
  DF* S1x = S;
  DF* S1y = S + M;
  DF* S1z = S + 2 * M;
  DF* S2x = S + 3 * M;
  DF* S2y = S + 4 * M;
  DF* S2z = S + 5 * M;
  DF* w = S + 6 * M;
  const DF r1x = {o1df[6 * k0], o1df[6 * k0 + 1]}, r1y = {o1df[6 * k0 + 2], o1df[6 * k0 + 3]},
           r1z = {o1df[6 * k0 + 4], o1df[6 * k0 + 5]};
  const float r2x = mxyz[3 * k0], r2y = mxyz[3 * k0 + 1], r2z = mxyz[3 * k0 + 2];
  // Eq. 2: both point sets rectified to the reference; S2 exactly (a difference of floats)
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    S1x[k] = df_add({o1df[6 * k], o1df[6 * k + 1]}, df_neg(r1x));
    S1y[k] = df_add({o1df[6 * k + 2], o1df[6 * k + 3]}, df_neg(r1y));
    S1z[k] = df_add({o1df[6 * k + 4], o1df[6 * k + 5]}, df_neg(r1z));
    S2x[k] = df_two_sum(mxyz[3 * k], -r2x);
    S2y[k] = df_two_sum(mxyz[3 * k + 1], -r2y);
    S2z[k] = df_two_sum(mxyz[3 * k + 2], -r2z);
    w[k] = {1.f, 0.f};
  }
  __syncthreads();
  const int words = (M + 31) / 32;
  const DF H2 = df_of(H * H), Hd = df_of(H), one = {1.f, 0.f};
  for (int it = 0; it < n_reweight; ++it) {
    // Eq. 3: M = sum w S1 S2^T (and sum w); acc[10] = sum w |S1| |S2| (FP32), an upper bound of
    // the largest eigenvalue of Horn's matrix (Cauchy-Schwarz), where Newton starts
    DF acc[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = {0.f, 0.f};
    float nb = 0.f;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      const DF wk = w[k];
      const DF x1 = S1x[k], y1 = S1y[k], z1 = S1z[k];
      const DF a0 = df_mul(wk, x1), a1 = df_mul(wk, y1), a2 = df_mul(wk, z1);
      const DF b0 = S2x[k], b1 = S2y[k], b2 = S2z[k];
      acc[0] = df_add(acc[0], df_mul(a0, b0));
      acc[1] = df_add(acc[1], df_mul(a0, b1));
      acc[2] = df_add(acc[2], df_mul(a0, b2));
      acc[3] = df_add(acc[3], df_mul(a1, b0));
      acc[4] = df_add(acc[4], df_mul(a1, b1));
      acc[5] = df_add(acc[5], df_mul(a1, b2));
      acc[6] = df_add(acc[6], df_mul(a2, b0));
      acc[7] = df_add(acc[7], df_mul(a2, b1));
      acc[8] = df_add(acc[8], df_mul(a2, b2));
      acc[9] = df_add(acc[9], wk);
      const float n1 = x1.hi * x1.hi + y1.hi * y1.hi + z1.hi * z1.hi;
      const float n2 = b0.hi * b0.hi + b1.hi * b1.hi + b2.hi * b2.hi;
      nb += wk.hi * sqrtf(n1 * n2);
    }
    acc[10] = {nb, 0.f};
    block_sum_df<11>(acc, red);
    if (threadIdx.x < 32) {   // warp 0: Horn's rotation (the sums are in thread 0)
      double Md[11];
#pragma unroll
      for (int i = 0; i < 11; ++i) {
        const double v = threadIdx.x == 0 ? df_val(acc[i]) : 0.0;
        Md[i] = __shfl_sync(0xffffffffu, v, 0);
      }
      // the FP32 bound widened well past its rounding (relative 1e-6 over <= 2^16 terms)
      const double bound = Md[10] * (1.0 + 1e-3) + 1e-30;
      double R[9];
      if (!horn_rotation_warp(Md, Md[9], bound, R, sX)) {
        for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
      }
      if (threadIdx.x == 0)
        for (int i = 0; i < 9; ++i) sR[i] = R[i];
    }
    __syncthreads();
    DF Rm[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rm[i] = df_of(sR[i]);
    const bool last = it == n_reweight - 1;
    DF sc = {0.f, 0.f};
    // Eq. 4: d_k = |S2 - R S1|, w_k = min(H / d_k, 1); d <= H is decided on d^2 <= H^2 and
    // H / d = H rsqrt(d^2) (FP32 seed, two Newton steps in double-float) when d > H.
    // Warp-uniform trip count so that every lane reaches the ballot.
    for (int base = (threadIdx.x & ~31); base < M; base += blockDim.x) {
      int k = base + (threadIdx.x & 31);
      bool inl = false;
      if (k < M) {
        const DF x = S1x[k], y = S1y[k], z = S1z[k];
        const DF e0 = df_add(S2x[k], df_neg(df_add(df_add(df_mul(Rm[0], x), df_mul(Rm[1], y)),
                                                   df_mul(Rm[2], z))));
        const DF e1 = df_add(S2y[k], df_neg(df_add(df_add(df_mul(Rm[3], x), df_mul(Rm[4], y)),
                                                   df_mul(Rm[5], z))));
        const DF e2 = df_add(S2z[k], df_neg(df_add(df_add(df_mul(Rm[6], x), df_mul(Rm[7], y)),
                                                   df_mul(Rm[8], z))));
        const DF d2 = df_add(df_add(df_mul(e0, e0), df_mul(e1, e1)), df_mul(e2, e2));
        const bool within = df_le(d2, H2);
        DF wk = one;
        if (!within) {
          DF yv = {rsqrtf(d2.hi), 0.f};
#pragma unroll
          for (int nstep = 0; nstep < 2; ++nstep) {
            const DF r = df_add(one, df_neg(df_mul(d2, df_mul(yv, yv))));
            yv = df_add(yv, df_scale(df_mul(yv, r), 0.5f));
          }
          wk = df_mul(Hd, yv);
          if (!df_le(wk, one)) wk = one;
        }
        w[k] = wk;
        if (last) {
          inl = within;
          hw[(size_t)h * M + k] = wk.hi;
          if (k != k0) sc = df_add(sc, wk);
        }
      }
      if (last) {
        uint32_t bits = __ballot_sync(0xffffffffu, inl);
        if ((threadIdx.x & 31) == 0) hbits[(size_t)h * words + base / 32] = bits;
      }
    }
    if (last) {
      DF v[1] = {sc};
      block_sum_df<1>(v, red);
      if (threadIdx.x == 0) score[h] = df_val(v[0]);
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
                   double keep_frac, const double* o1w, float* o1df, double* scratch,
                   uint32_t* hbits, float* hw, double* score, uint32_t* mask, float* what,
                   uint32_t* kept, int* counts, cudaStream_t s) {
  if (M <= 0 || n_hyp <= 0) return;
  int sm = ransac_smem_bytes(M);
  int use_smem = sm <= 220 * 1024;
  if (use_smem) {
    static PerDevice attr;
    // a failed attribute set leaves the launch to fail, which the caller's error check reports
    set_smem_once(attr, k_ransac_hyp, 220 * 1024);
  } else {
    sm = 0;
  }
  k_ransac_points<<<(M + 255) / 256, 256, 0, s>>>(depth0, W, K.fx, K.fy, K.cx, K.cy, midx, M,
                                                   o1w, o1df);
  k_ransac_hyp<<<n_hyp, kRansacThreads, sm, s>>>(o1df, mxyz, M, hyp, n_reweight, H, use_smem,
                                                 scratch, hbits, hw, score);
  g_launches += 2;
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
constexpr size_t kNaO1 = kNaCnt + 256;
constexpr size_t kNaTotal = kNaO1 + kNaAlign(sizeof(float) * 6 * DS_NOALLOC_MAX_MATCHES);
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
      // the kernel's shared-memory limit is a per-device setting too; the device is only marked
      // set up once both calls succeeded, so a failure is retried by the next call
      if (cudaFuncSetAttribute(k_ransac_hyp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               220 * 1024) != cudaSuccess) {
        cudaGetLastError();
        return DS_ERR_CUDA;
      }
      base_of[dev] = p;
    }
    base = (unsigned char*)base_of[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  uint32_t* hbits = (uint32_t*)(base + kNaBits);
  float* hw = (float*)(base + kNaW);
  int* midx = (int*)(base + kNaMidx);
  int* hyp = (int*)(base + kNaHyp);
  int* counts = (int*)(base + kNaCnt);
  float* o1df = (float*)(base + kNaO1);
  int* flag = counts + 2;
  // the array keeps the previous call's contents: clear the words that accumulate
  cudaMemsetAsync(counts, 0, 4 * sizeof(int), s);
  const int npx = W * H;
  const int nt = M > n_hyp ? M : n_hyp;
  k_na_indices<<<(nt + 255) / 256, 256, 0, s>>>(match_tmpl_idx, M, hyp_list, n_hyp, npx, depth0,
                                                 midx, hyp, flag);
  const int sm = ransac_smem_bytes(M);  // <= 220 KB for M <= DS_NOALLOC_MAX_MATCHES
  k_ransac_points<<<(M + 255) / 256, 256, 0, s>>>(depth0, W, K.fx, K.fy, K.cx, K.cy, midx, M,
                                                   nullptr, o1df);
  k_ransac_hyp<<<n_hyp, kRansacThreads, sm, s>>>(o1df, match_xyz, M, hyp, n_reweight, H_mm, 1,
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

