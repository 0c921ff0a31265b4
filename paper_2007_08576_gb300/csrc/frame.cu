// Frame preparation and template set-up kernels.
//
// * Back-projection X = ((u - cx) z / fx, (v - cy) z / fy, z) of a depth map. The template is
//   back-projected in FP64 with explicit round-to-nearest operations (no contraction), so that
//   the nearest-control-point decisions of the blend table are taken on exactly the values
//   a plain FP64 evaluation of the same formula produces.
// * Blend table: the 4 nearest control points of every template point by 3D distance at
//   time 0 (Section 2: a template point moves with a blend of the control points near it),
//   ties to the lower node id, Gaussian weights normalised to one.
// * Live frame: FP32 points and central-difference normals (Section 2: only the distance
//   along the normal direction is used by ICP), oriented toward the camera.
#include <math.h>

#include "ds_internal.cuh"

namespace ds {

__global__ void k_backproject64(const float* __restrict__ depth, int W, int H, double fx,
                                double fy, double cx, double cy, double* __restrict__ X64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  int u = i % W, v = i / W;
  double z = (double)depth[i];
  // ((u - cx) * z) / fx, evaluated left to right with single roundings
  X64[3 * i + 0] = __ddiv_rn(__dmul_rn(__dsub_rn((double)u, cx), z), fx);
  X64[3 * i + 1] = __ddiv_rn(__dmul_rn(__dsub_rn((double)v, cy), z), fy);
  X64[3 * i + 2] = z;
}

void launch_backproject64(const float* depth, int W, int H, ds_intrinsics K, double* X64,
                          cudaStream_t s) {
  int n = W * H;
  k_backproject64<<<(n + 255) / 256, 256, 0, s>>>(depth, W, H, K.fx, K.fy, K.cx, K.cy, X64);
  ++g_launches;
}

// One thread per valid template point; node positions staged in shared memory.
__global__ void k_knn(const double* __restrict__ X64, const int* __restrict__ pidx, int P,
                      const double* __restrict__ g64, int N, double inv2s2,
                      int4* __restrict__ nid, float4* __restrict__ alpha) {
  extern __shared__ double sg[];
  for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) sg[i] = g64[i];
  __syncthreads();
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const double* x = X64 + 3 * (size_t)pidx[j];
  double px = x[0], py = x[1], pz = x[2];
  double bd[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  int bi[4] = {-1, -1, -1, -1};
  for (int i = 0; i < N; ++i) {
    double dx = __dsub_rn(px, sg[3 * i + 0]);
    double dy = __dsub_rn(py, sg[3 * i + 1]);
    double dz = __dsub_rn(pz, sg[3 * i + 2]);
    // (dx*dx + dy*dy) + dz*dz with single roundings, as the plain formula reads
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < bd[3]) {
      int p = 3;
      while (p > 0 && d2 < bd[p - 1]) {
        bd[p] = bd[p - 1];
        bi[p] = bi[p - 1];
        --p;
      }
      bd[p] = d2;
      bi[p] = i;
    }
  }
  double a[4], s = 0.0;
  for (int k = 0; k < 4; ++k) {
    a[k] = exp(-bd[k] * inv2s2);
    s += a[k];
  }
  if (!(s > 0.0)) {
    for (int k = 0; k < 4; ++k) a[k] = 0.25;
    s = 1.0;
  }
  nid[j] = make_int4(bi[0], bi[1], bi[2], bi[3]);
  alpha[j] = make_float4((float)(a[0] / s), (float)(a[1] / s), (float)(a[2] / s),
                         (float)(a[3] / s));
}

void launch_knn(const double* X64, const int* pidx, int P, const double* g64, int N,
                double sigma_b, int4* nid, float4* alpha, cudaStream_t s) {
  if (P == 0) return;
  double inv2s2 = 1.0 / (2.0 * sigma_b * sigma_b);
  size_t sm = sizeof(double) * 3 * N;
  k_knn<<<(P + 127) / 128, 128, sm, s>>>(X64, pidx, P, g64, N, inv2s2, nid, alpha);
  ++g_launches;
}

__device__ __forceinline__ float3 bp32(const float* depth, int W, int u, int v, float fx,
                                       float fy, float cx, float cy, bool* ok) {
  float z = depth[v * W + u];
  *ok = isfinite(z) && z > 0.f;
  return make_float3((u - cx) * z / fx, (v - cy) * z / fy, z);
}

__global__ void k_frame_prep(const float* __restrict__ depth, int W, int H, float fx, float fy,
                             float cx, float cy, float4* __restrict__ pts,
                             float4* __restrict__ nrm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  int u = i % W, v = i / W;
  bool ok;
  float3 X = bp32(depth, W, u, v, fx, fy, cx, cy, &ok);
  float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
  bool good = false;
  if (ok && u > 0 && v > 0 && u < W - 1 && v < H - 1) {
    bool o1, o2, o3, o4;
    float3 xr = bp32(depth, W, u + 1, v, fx, fy, cx, cy, &o1);
    float3 xl = bp32(depth, W, u - 1, v, fx, fy, cx, cy, &o2);
    float3 xd = bp32(depth, W, u, v + 1, fx, fy, cx, cy, &o3);
    float3 xu = bp32(depth, W, u, v - 1, fx, fy, cx, cy, &o4);
    if (o1 && o2 && o3 && o4) {
      float3 du = make_float3(xr.x - xl.x, xr.y - xl.y, xr.z - xl.z);
      float3 dv = make_float3(xd.x - xu.x, xd.y - xu.y, xd.z - xu.z);
      float cxp = du.y * dv.z - du.z * dv.y;
      float cyp = du.z * dv.x - du.x * dv.z;
      float czp = du.x * dv.y - du.y * dv.x;
      float cn = sqrtf(cxp * cxp + cyp * cyp + czp * czp);
      if (cn > 0.f) {
        float sgn = czp > 0.f ? -1.f : 1.f;
        n = make_float4(sgn * cxp / cn, sgn * cyp / cn, sgn * czp / cn, 0.f);
        good = true;
      }
    }
  }
  pts[i] = make_float4(X.x, X.y, X.z, good ? 1.f : 0.f);
  nrm[i] = n;
}

void launch_frame_prep(const float* depth, int W, int H, ds_intrinsics K, float4* pts,
                       float4* nrm, cudaStream_t s) {
  int n = W * H;
  k_frame_prep<<<(n + 255) / 256, 256, 0, s>>>(depth, W, H, K.fx, K.fy, K.cx, K.cy, pts, nrm);
  ++g_launches;
}

__global__ void k_check_finite(const float* __restrict__ v, int n, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = i < n && !isfinite(v[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_check_finite(const float* v, int n, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  k_check_finite<<<(n + 255) / 256, 256, 0, s>>>(v, n, flag);
  ++g_launches;
}

}  // namespace ds
