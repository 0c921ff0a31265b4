// Uniform ORB features (Section 2.1, first paragraph): FAST-9 corners with per-pixel neighbour
// suppression, steered binary descriptors and mutual-nearest Hamming matching of the template's
// features to a live frame's. The definitions are those of include/defsolve_orb.h.
//
// Per image (one ds_orb_detect):
//   k_fast_box   one thread per pixel: FAST-9 response (16 circle reads, bright / dark masks,
//                9-run test on the doubled 16-bit mask) and the 5 x 5 box sum of the pixel;
//   k_keep_count 256 pixels per CTA in row-major order: keypoint test (response > 0, no
//                neighbour larger, inside the border, positive depth), CTA count;
//   k_block_offsets  one CTA: exclusive prefix sums of the CTA counts and the totals;
//   k_compact    the same test again, each CTA's keypoints at its offset, in-CTA order by
//                ballots: keypoints land in ascending pixel order with no sort;
//   k_describe   one warp per keypoint: intensity-centroid moments over the radius-15 disc,
//                the orientation bin in FP64, 256 tests as 8 ballots of 32 lanes.
// Matching (ds_orb_match): k_nearest twice (template -> live, live -> template), one warp per
// query, reference descriptors staged through shared memory, nearest as the minimum of
// (distance << 32 | index); k_match_out keeps mutual pairs within max_dist in template order
// (one CTA, ballot compaction) and back-projects the live keypoints.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "defsolve_orb.h"
#include "dev_util.cuh"
#include "ds_internal.cuh"

namespace ds {
namespace {

constexpr int kNbins = 32;
constexpr int kTests = 256;
constexpr int kDiscR = 15;

// the radius-3 digital circle in angular order (cyclic contiguity is what the test uses)
__constant__ int8_t c_circ[16][2] = {{-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}, {0, -3}, {1, -3},
                                     {2, -2},  {3, -1},  {3, 0},   {3, 1},   {2, 2},  {1, 3},
                                     {0, 3},   {-1, 3},  {-2, 2},  {-3, 1}};

__global__ void k_fast_box(const uint8_t* __restrict__ img, int W, int H, int t,
                           int* __restrict__ score, int* __restrict__ box) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= W || v >= H) return;
  const int i = v * W + u;
  int s = 0;
  if (u >= 3 && v >= 3 && u < W - 3 && v < H - 3) {
    const int p = img[i];
    unsigned mb = 0, md = 0;
    int sb = 0, sd = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int c = img[(v + c_circ[k][1]) * W + u + c_circ[k][0]];
      if (c > p + t) {
        mb |= 1u << k;
        sb += c - p - t;
      } else if (c < p - t) {
        md |= 1u << k;
        sd += p - c - t;
      }
    }
    // a cyclic run of 9 set bits: AND of 9 shifts of the doubled mask
    unsigned rb = mb | (mb << 16), rd = md | (md << 16);
    unsigned xb = rb, xd = rd;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
      xb &= rb >> k;
      xd &= rd >> k;
    }
    if ((xb | xd) & 0xFFFFu) s = max(sb, sd);
  }
  score[i] = s;
  int b = 0;
  if (u >= 2 && v >= 2 && u < W - 2 && v < H - 2) {
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
      for (int dx = -2; dx <= 2; ++dx) b += img[(v + dy) * W + u + dx];
  }
  box[i] = b;
}

__device__ __forceinline__ bool is_keypoint(const int* __restrict__ score,
                                            const float* __restrict__ depth, int W, int H,
                                            int border, int i) {
  if (i >= W * H) return false;
  const int u = i % W, v = i / W;
  if (u < border || v < border || u >= W - border || v >= H - border) return false;
  const int s = score[i];
  if (s <= 0) return false;
  if (depth && !(depth[i] > 0.f)) return false;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
      if ((dx || dy) && score[i + dy * W + dx] > s) return false;
  return true;
}

__global__ __launch_bounds__(256) void k_keep_count(const int* __restrict__ score,
                                                    const float* __restrict__ depth, int W, int H,
                                                    int border, int* __restrict__ cnt) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int c = __syncthreads_count(is_keypoint(score, depth, W, H, border, i));
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// Exclusive prefix sums of the CTA counts (one CTA of 1024 threads, 1024 counts per round) and
// the keypoint totals.
__global__ __launch_bounds__(1024) void k_block_offsets(const int* __restrict__ cnt, int nblk,
                                                        int max_kp, int* __restrict__ off,
                                                        int* __restrict__ nkp) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblk; b0 += 1024) {
    const int b = b0 + tid;
    const int v = b < nblk ? cnt[b] : 0;
    int x = v;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {   // inclusive scan of the warp totals
      int w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    if (b < nblk) off[b] = s_base + (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
    __syncthreads();
    if (tid == 0) s_base += s_warp[31];
    __syncthreads();
  }
  if (tid == 0) {
    nkp[0] = min(s_base, max_kp);
    nkp[1] = s_base;
  }
}

// Keypoints of each CTA's 256 pixels at its offset, in pixel order (ballots within the CTA).
__global__ __launch_bounds__(256) void k_compact(const int* __restrict__ score,
                                                 const float* __restrict__ depth, int W, int H,
                                                 int border, const int* __restrict__ off,
                                                 int max_kp, int* __restrict__ kp_pix,
                                                 int* __restrict__ kp_score) {
  __shared__ int s_warp[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = blockIdx.x * 256 + tid;
  const bool kp = is_keypoint(score, depth, W, H, border, i);
  const unsigned bal = __ballot_sync(0xffffffffu, kp);
  if (lane == 0) s_warp[warp] = __popc(bal);
  __syncthreads();
  int woff = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w)
    if (w < warp) woff += s_warp[w];
  const int idx = off[blockIdx.x] + woff + __popc(bal & ((1u << lane) - 1u));
  if (kp && idx < max_kp) {
    kp_pix[idx] = i;
    kp_score[idx] = score[i];
  }
}

// Rotated test offsets of every orientation bin, (dx_a, dy_a, dx_b, dy_b) as bytes.
__global__ void k_pattern_table(const double* __restrict__ pat, char4* __restrict__ tab) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNbins * kTests) return;
  const int k = e / kTests, i = e % kTests;
  const double phi = 2.0 * M_PI * (double)k / (double)kNbins;
  const double c = cos(phi), s = sin(phi);
  const double ax = pat[4 * i], ay = pat[4 * i + 1], bx = pat[4 * i + 2], by = pat[4 * i + 3];
  // separately rounded products (no fused multiply-add), as a plain FP64 evaluation
  const double axr = __dsub_rn(__dmul_rn(ax, c), __dmul_rn(ay, s));
  const double ayr = __dadd_rn(__dmul_rn(ax, s), __dmul_rn(ay, c));
  const double bxr = __dsub_rn(__dmul_rn(bx, c), __dmul_rn(by, s));
  const double byr = __dadd_rn(__dmul_rn(bx, s), __dmul_rn(by, c));
  tab[e] = make_char4((signed char)rint(axr), (signed char)rint(ayr), (signed char)rint(bxr),
                      (signed char)rint(byr));
}

__global__ __launch_bounds__(256) void k_describe(const uint8_t* __restrict__ img,
                                                  const int* __restrict__ box, int W,
                                                  const int* __restrict__ kp_pix,
                                                  const int* __restrict__ nkp,
                                                  const char4* __restrict__ tab,
                                                  int* __restrict__ kp_bin,
                                                  uint32_t* __restrict__ desc) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= nkp[0]) return;
  const int p = kp_pix[k];
  const int u = p % W, v = p / W;
  int m10 = 0, m01 = 0;
  constexpr int D = 2 * kDiscR + 1;
  for (int e = lane; e < D * D; e += 32) {
    const int dx = e % D - kDiscR, dy = e / D - kDiscR;
    if (dx * dx + dy * dy <= kDiscR * kDiscR) {
      const int val = img[(v + dy) * W + u + dx];
      m10 += dx * val;
      m01 += dy * val;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m10 += __shfl_xor_sync(0xffffffffu, m10, o);
    m01 += __shfl_xor_sync(0xffffffffu, m01, o);
  }
  const double theta = atan2((double)m01, (double)m10);
  int b = (int)rint(theta / (2.0 * M_PI / (double)kNbins));
  b = ((b % kNbins) + kNbins) % kNbins;
  const char4* tb = tab + b * kTests;
  uint32_t word = 0;
#pragma unroll
  for (int w = 0; w < kTests / 32; ++w) {
    const char4 o = tb[32 * w + lane];
    const int sa = box[(v + o.y) * W + u + o.x];
    const int sb = box[(v + o.w) * W + u + o.z];
    const unsigned bits = __ballot_sync(0xffffffffu, sa < sb);
    if (lane == w) word = bits;
  }
  if (lane < 8) desc[(size_t)k * 8 + lane] = word;
  if (lane == 0) kp_bin[k] = b;
}

// Nearest reference descriptor of every query: best[q] = (distance << 32) | index, ties to the
// lower index; ~0 when there is no reference. 8 queries per CTA (one warp each), references
// staged 256 at a time.
__global__ __launch_bounds__(256) void k_nearest(const uint32_t* __restrict__ Dq,
                                                 const int* __restrict__ nq_p,
                                                 const uint32_t* __restrict__ Dr,
                                                 const int* __restrict__ nr_p,
                                                 unsigned long long* __restrict__ best) {
  __shared__ uint4 sR[256][2];
  const int nq = *nq_p, nr = *nr_p;
  const int q0 = blockIdx.x * 8;
  if (q0 >= nq) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = q0 + warp;
  const bool active = q < nq;
  uint32_t qd[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) qd[w] = active ? Dq[(size_t)q * 8 + w] : 0u;
  unsigned long long key = ~0ull;
  for (int r0 = 0; r0 < nr; r0 += 256) {
    __syncthreads();
    const int r = r0 + threadIdx.x;
    if (r < nr) {
      const uint4* src = reinterpret_cast<const uint4*>(Dr + (size_t)r * 8);
      sR[threadIdx.x][0] = src[0];
      sR[threadIdx.x][1] = src[1];
    }
    __syncthreads();
    if (active) {
      const int m = min(256, nr - r0);
      for (int j = lane; j < m; j += 32) {
        const uint4 a = sR[j][0], c = sR[j][1];
        const int d = __popc(qd[0] ^ a.x) + __popc(qd[1] ^ a.y) + __popc(qd[2] ^ a.z) +
                      __popc(qd[3] ^ a.w) + __popc(qd[4] ^ c.x) + __popc(qd[5] ^ c.y) +
                      __popc(qd[6] ^ c.z) + __popc(qd[7] ^ c.w);
        const unsigned long long kk = ((unsigned long long)d << 32) | (unsigned)(r0 + j);
        key = kk < key ? kk : key;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
    key = other < key ? other : key;
  }
  if (active && lane == 0) best[q] = key;
}

// Mutual nearest pairs within max_dist, in ascending template index; one CTA of 1024 threads.
__global__ __launch_bounds__(1024) void k_match_out(
    const unsigned long long* __restrict__ best_t, const unsigned long long* __restrict__ best_l,
    const int* __restrict__ nt_p, const int* __restrict__ nl_p, int max_dist,
    const int* __restrict__ tmpl_pix, const int* __restrict__ live_pix,
    const float* __restrict__ live_depth, int W, float fx, float fy, float cx, float cy,
    int* __restrict__ m_t, int* __restrict__ m_l, int* __restrict__ m_dist,
    int* __restrict__ m_pix, float* __restrict__ m_xyz, int* __restrict__ nm) {
  __shared__ int s_warp[32];
  const int nt = *nt_p, nl = *nl_p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = 0;
  for (int t0 = 0; t0 < nt; t0 += 1024) {
    const int t = t0 + threadIdx.x;
    bool ok = false;
    int l = 0, d = 0;
    if (t < nt && nl > 0) {
      const unsigned long long k = best_t[t];
      l = (int)(k & 0xffffffffull);
      d = (int)(k >> 32);
      ok = d <= max_dist && (int)(best_l[l] & 0xffffffffull) == t;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int woff = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) woff += s_warp[w];
      tot += s_warp[w];
    }
    if (ok) {
      const int idx = base + woff + __popc(bal & ((1u << lane) - 1u));
      const int lp = live_pix[l];
      const float z = live_depth[lp];
      m_t[idx] = t;
      m_l[idx] = l;
      m_dist[idx] = d;
      m_pix[idx] = tmpl_pix[t];
      m_xyz[3 * idx] = ((float)(lp % W) - cx) * z / fx;
      m_xyz[3 * idx + 1] = ((float)(lp / W) - cy) * z / fy;
      m_xyz[3 * idx + 2] = z;
    }
    base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *nm = base;
}

template <typename T>
int orb_alloc(T** p, size_t count) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DS_ERR_OOM : DS_ERR_CUDA;
  }
  return DS_OK;
}
template <typename T>
void orb_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

}  // namespace
}  // namespace ds

struct ds_orb_s {
  int W = 0, H = 0;
  ds_intrinsics K{};
  ds_orb_params prm{};
  int max_kp = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev = nullptr;
  double h_pat[4 * ds::kTests];
  bool detected = false, have_depth = false;
  uint8_t* d_img = nullptr;
  float* d_depth = nullptr;
  int* d_score = nullptr;
  int* d_box = nullptr;
  int* d_cnt = nullptr;
  int* d_off = nullptr;        // exclusive prefix sums of d_cnt
  int nblk = 0;
  char4* d_tab = nullptr;
  int* d_kp_pix = nullptr;
  int* d_kp_score = nullptr;
  int* d_kp_bin = nullptr;
  uint32_t* d_desc = nullptr;
  int* d_nkp = nullptr;        // [0] kept, [1] found, [2] matches
  unsigned long long* d_best_l = nullptr;   // per live keypoint (this object as the live side)
  unsigned long long* d_best_t = nullptr;   // per template keypoint
  int best_t_cap = 0;
  int* d_m = nullptr;          // matches: t, l, dist, pixel (4 arrays of max_kp)
  float* d_m_xyz = nullptr;
};

namespace {

int orb_check(ds_orb o) {
  if (cudaGetLastError() != cudaSuccess) return DS_ERR_CUDA;
  return DS_OK;
}

void orb_release(ds_orb o) {
  using ds::orb_free;
  orb_free(o->d_img); orb_free(o->d_depth); orb_free(o->d_score); orb_free(o->d_box);
  orb_free(o->d_cnt); orb_free(o->d_off); orb_free(o->d_tab); orb_free(o->d_kp_pix); orb_free(o->d_kp_score);
  orb_free(o->d_kp_bin); orb_free(o->d_desc); orb_free(o->d_nkp); orb_free(o->d_best_l);
  orb_free(o->d_best_t); orb_free(o->d_m); orb_free(o->d_m_xyz);
  if (o->ev) cudaEventDestroy(o->ev);
  if (o->own_stream && o->stream) cudaStreamDestroy(o->stream);
}

}  // namespace

extern "C" {

void ds_orb_default_params(ds_orb_params* p) {
  if (!p) return;
  p->fast_t = 20;
  p->border = 16;
  p->max_dist = 64;
  p->max_kp = 0;
}

int ds_orb_create(int32_t W, int32_t H, ds_intrinsics K, const ds_orb_params* p,
                  const double* pattern, void* cuda_stream, ds_orb* out) {
  using ds::orb_alloc;
  if (!out || !pattern) return DS_ERR_ARG;
  *out = nullptr;
  ds_orb_params prm;
  ds_orb_default_params(&prm);
  if (p) prm = *p;
  if (W < 40 || H < 40 || W > 4096 || H > 4096) return DS_ERR_ARG;
  if (prm.fast_t < 0 || prm.fast_t > 255 || prm.border < 16 || 2 * prm.border >= W ||
      2 * prm.border >= H || prm.max_dist < 0 || prm.max_dist > 256 || prm.max_kp < 0 ||
      prm.max_kp > W * H)
    return DS_ERR_ARG;
  if (!(K.fx > 0.f) || !(K.fy > 0.f)) return DS_ERR_ARG;
  ds_orb o = new ds_orb_s;
  o->W = W;
  o->H = H;
  o->K = K;
  o->prm = prm;
  o->max_kp = prm.max_kp > 0 ? prm.max_kp : std::max(1, W * H / 8);
  if (cudaMemcpy(o->h_pat, pattern, sizeof(o->h_pat), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    delete o;
    return DS_ERR_ARG;
  }
  for (int i = 0; i < 4 * ds::kTests; ++i)
    if (!(fabs(o->h_pat[i]) <= 13.0)) {
      delete o;
      return DS_ERR_ARG;
    }
  for (int i = 0; i < ds::kTests; ++i)
    for (int j = 0; j < 2; ++j) {
      const double x = o->h_pat[4 * i + 2 * j], y = o->h_pat[4 * i + 2 * j + 1];
      if (x * x + y * y > 169.0) {
        delete o;
        return DS_ERR_ARG;
      }
    }
  if (cuda_stream) {
    o->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&o->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete o;
      return DS_ERR_CUDA;
    }
    o->own_stream = true;
  }
  const size_t npx = (size_t)W * H;
  o->nblk = (int)((npx + 255) / 256);
  const int K8 = o->max_kp;
  int rc;
  double* d_pat = nullptr;
  if ((rc = orb_alloc(&o->d_img, npx)) || (rc = orb_alloc(&o->d_depth, npx)) ||
      (rc = orb_alloc(&o->d_score, npx)) || (rc = orb_alloc(&o->d_box, npx)) ||
      (rc = orb_alloc(&o->d_cnt, (size_t)o->nblk)) || (rc = orb_alloc(&o->d_off, (size_t)o->nblk)) ||
      (rc = orb_alloc(&o->d_tab, (size_t)ds::kNbins * ds::kTests)) ||
      (rc = orb_alloc(&o->d_kp_pix, (size_t)K8)) || (rc = orb_alloc(&o->d_kp_score, (size_t)K8)) ||
      (rc = orb_alloc(&o->d_kp_bin, (size_t)K8)) || (rc = orb_alloc(&o->d_desc, (size_t)K8 * 8)) ||
      (rc = orb_alloc(&o->d_nkp, 4)) || (rc = orb_alloc(&o->d_best_l, (size_t)K8)) ||
      (rc = orb_alloc(&o->d_m, (size_t)K8 * 4)) || (rc = orb_alloc(&o->d_m_xyz, (size_t)K8 * 3)) ||
      (rc = orb_alloc(&d_pat, 4 * (size_t)ds::kTests))) {
    ds::orb_free(d_pat);
    orb_release(o);
    delete o;
    return rc;
  }
  if (cudaEventCreateWithFlags(&o->ev, cudaEventDisableTiming) != cudaSuccess) {
    ds::orb_free(d_pat);
    orb_release(o);
    delete o;
    return DS_ERR_CUDA;
  }
  cudaMemsetAsync(o->d_nkp, 0, 4 * sizeof(int), o->stream);
  cudaMemcpyAsync(d_pat, o->h_pat, sizeof(o->h_pat), cudaMemcpyHostToDevice, o->stream);
  ds::k_pattern_table<<<(ds::kNbins * ds::kTests + 255) / 256, 256, 0, o->stream>>>(d_pat, o->d_tab);
  ++ds::g_launches;
  ds::count_kernels(1);
  const cudaError_t e = cudaStreamSynchronize(o->stream);
  ds::orb_free(d_pat);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    orb_release(o);
    delete o;
    return DS_ERR_CUDA;
  }
  *out = o;
  return DS_OK;
}

int ds_orb_detect(ds_orb o, const uint8_t* image_hw, const float* depth_hw) {
  if (!o || !image_hw) return DS_ERR_ARG;
  const int W = o->W, H = o->H;
  const size_t npx = (size_t)W * H;
  cudaStream_t s = o->stream;
  if (cudaMemcpyAsync(o->d_img, image_hw, npx, cudaMemcpyDefault, s) != cudaSuccess) {
    cudaGetLastError();
    return DS_ERR_ARG;
  }
  if (depth_hw &&
      cudaMemcpyAsync(o->d_depth, depth_hw, npx * sizeof(float), cudaMemcpyDefault, s) != cudaSuccess) {
    cudaGetLastError();
    return DS_ERR_ARG;
  }
  const dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  ds::k_fast_box<<<grd, blk, 0, s>>>(o->d_img, W, H, o->prm.fast_t, o->d_score, o->d_box);
  const float* dep = depth_hw ? o->d_depth : nullptr;
  ds::k_keep_count<<<o->nblk, 256, 0, s>>>(o->d_score, dep, W, H, o->prm.border, o->d_cnt);
  ds::k_block_offsets<<<1, 1024, 0, s>>>(o->d_cnt, o->nblk, o->max_kp, o->d_off, o->d_nkp);
  ds::k_compact<<<o->nblk, 256, 0, s>>>(o->d_score, dep, W, H, o->prm.border, o->d_off,
                                        o->max_kp, o->d_kp_pix, o->d_kp_score);
  ds::k_describe<<<(o->max_kp + 7) / 8, 256, 0, s>>>(o->d_img, o->d_box, W, o->d_kp_pix, o->d_nkp,
                                                     o->d_tab, o->d_kp_bin, o->d_desc);
  ds::g_launches += 5;
  ds::count_kernels(5);
  o->detected = true;
  o->have_depth = depth_hw != nullptr;
  cudaEventRecord(o->ev, s);
  return orb_check(o);
}

int ds_orb_num_keypoints(ds_orb o, int32_t* n_kept, int32_t* n_total) {
  if (!o) return DS_ERR_ARG;
  int h[2] = {0, 0};
  if (cudaMemcpyAsync(h, o->d_nkp, 2 * sizeof(int), cudaMemcpyDeviceToHost, o->stream) != cudaSuccess ||
      cudaStreamSynchronize(o->stream) != cudaSuccess)
    return DS_ERR_CUDA;
  if (n_kept) *n_kept = h[0];
  if (n_total) *n_total = h[1];
  return DS_OK;
}

int ds_orb_get_keypoints(ds_orb o, int32_t* pix, int32_t* score, int32_t* bin, uint32_t* desc_8) {
  int n = 0;
  int rc = ds_orb_num_keypoints(o, &n, nullptr);
  if (rc) return rc;
  if (n == 0) return DS_OK;
  const size_t b = sizeof(int) * (size_t)n;
  if ((pix && cudaMemcpy(pix, o->d_kp_pix, b, cudaMemcpyDefault) != cudaSuccess) ||
      (score && cudaMemcpy(score, o->d_kp_score, b, cudaMemcpyDefault) != cudaSuccess) ||
      (bin && cudaMemcpy(bin, o->d_kp_bin, b, cudaMemcpyDefault) != cudaSuccess) ||
      (desc_8 && cudaMemcpy(desc_8, o->d_desc, 8 * b, cudaMemcpyDefault) != cudaSuccess))
    return DS_ERR_CUDA;
  return DS_OK;
}

int ds_orb_match(ds_orb tmpl, ds_orb live) {
  if (!tmpl || !live) return DS_ERR_ARG;
  if (tmpl->W != live->W || tmpl->H != live->H) return DS_ERR_ARG;
  if (memcmp(tmpl->h_pat, live->h_pat, sizeof(live->h_pat)) != 0) return DS_ERR_ARG;
  if (!tmpl->detected || !live->detected || !live->have_depth) return DS_ERR_STATE;
  cudaStream_t s = live->stream;
  if (tmpl != live) cudaStreamWaitEvent(s, tmpl->ev, 0);
  if (live->best_t_cap < tmpl->max_kp) {
    cudaStreamSynchronize(s);
    ds::orb_free(live->d_best_t);
    int rc = ds::orb_alloc(&live->d_best_t, (size_t)tmpl->max_kp);
    if (rc) {
      live->best_t_cap = 0;
      return rc;
    }
    live->best_t_cap = tmpl->max_kp;
  }
  ds::k_nearest<<<(tmpl->max_kp + 7) / 8, 256, 0, s>>>(tmpl->d_desc, tmpl->d_nkp, live->d_desc,
                                                       live->d_nkp, live->d_best_t);
  ds::k_nearest<<<(live->max_kp + 7) / 8, 256, 0, s>>>(live->d_desc, live->d_nkp, tmpl->d_desc,
                                                       tmpl->d_nkp, live->d_best_l);
  const int K8 = live->max_kp;
  ds::k_match_out<<<1, 1024, 0, s>>>(live->d_best_t, live->d_best_l, tmpl->d_nkp, live->d_nkp,
                                     live->prm.max_dist, tmpl->d_kp_pix, live->d_kp_pix,
                                     live->d_depth, live->W, live->K.fx, live->K.fy, live->K.cx,
                                     live->K.cy, live->d_m, live->d_m + K8, live->d_m + 2 * K8,
                                     live->d_m + 3 * K8, live->d_m_xyz, live->d_nkp + 2);
  ds::g_launches += 3;
  ds::count_kernels(3);
  cudaEventRecord(live->ev, s);
  // later work on the template's stream (a new detection) waits until the match has read it
  if (tmpl != live) cudaStreamWaitEvent(tmpl->stream, live->ev, 0);
  return orb_check(live);
}

int ds_orb_num_matches(ds_orb live, int32_t* M) {
  if (!live || !M) return DS_ERR_ARG;
  int h = 0;
  if (cudaMemcpyAsync(&h, live->d_nkp + 2, sizeof(int), cudaMemcpyDeviceToHost, live->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(live->stream) != cudaSuccess)
    return DS_ERR_CUDA;
  *M = h;
  return DS_OK;
}

int ds_orb_get_matches(ds_orb live, int32_t* tmpl_kp, int32_t* live_kp, int32_t* dist,
                       int32_t* tmpl_pixel, float* xyz_3) {
  int M = 0;
  int rc = ds_orb_num_matches(live, &M);
  if (rc) return rc;
  if (M == 0) return DS_OK;
  const int K8 = live->max_kp;
  const size_t b = sizeof(int) * (size_t)M;
  if ((tmpl_kp && cudaMemcpy(tmpl_kp, live->d_m, b, cudaMemcpyDefault) != cudaSuccess) ||
      (live_kp && cudaMemcpy(live_kp, live->d_m + K8, b, cudaMemcpyDefault) != cudaSuccess) ||
      (dist && cudaMemcpy(dist, live->d_m + 2 * K8, b, cudaMemcpyDefault) != cudaSuccess) ||
      (tmpl_pixel && cudaMemcpy(tmpl_pixel, live->d_m + 3 * K8, b, cudaMemcpyDefault) != cudaSuccess) ||
      (xyz_3 && cudaMemcpy(xyz_3, live->d_m_xyz, 3 * sizeof(float) * (size_t)M, cudaMemcpyDefault) !=
                    cudaSuccess))
    return DS_ERR_CUDA;
  return DS_OK;
}

int ds_orb_match_device(ds_orb live, const int32_t** tmpl_pixel, const float** xyz_3) {
  if (!live) return DS_ERR_ARG;
  if (tmpl_pixel) *tmpl_pixel = live->d_m + 3 * live->max_kp;
  if (xyz_3) *xyz_3 = live->d_m_xyz;
  return DS_OK;
}

int ds_orb_destroy(ds_orb o) {
  if (!o) return DS_OK;
  if (o->stream) cudaStreamSynchronize(o->stream);
  orb_release(o);
  delete o;
  return DS_OK;
}

}  // extern "C"
