// The three terms of Eq. 1 and the assembly of the damped normal equations.
//
// Unknowns: 6 per control point, (dtheta, dt), node-major. A step moves node i by
// q_i <- exp(dtheta_i / 2) (x) q_i, t_i <- t_i + dt_i; the node's rigid map is
// W_i(x) = R_i (x - g_i) + g_i + t_i, i.e. the dual quaternion (q_i, 1/2 (0, T_i) (x) q_i) with
// T_i = g_i + t_i - R_i g_i (Section 2, dual-quaternion warps).
//
// Point terms (ICP, ORB) warp a template point p by dual-quaternion blending of its 4 nodes:
// b = sum_k alpha_k s_k dq_k (s_k aligns each quaternion with the nearest node's),
// x' = y(b) / |b_r|^2 with y = vec(b_r (x) (0,p) (x) b_r*) + 2 vec(b_d (x) b_r*).
// For a direction n, h = d(n . x')/db is evaluated in closed form, and the Jacobian of n . x'
// with respect to node k's (dtheta, dt) is alpha_k s_k times
//   dtheta: 1/2 f_v - 1/4 e_w T_k + 1/2 e_v x (R_k g_k + T_k / 2),   dt: 1/2 e_v
// with f = h_r (x) q_k*, e = h_d (x) q_k*.
//
// ICP (Section 2): r = n_q . (x' - q) at the pixel the warped point projects to (nearest
// pixel centre, or the bilinear blend of the usable pixels among the 4 around the projection,
// weights renormalised, valid iff their weight is >= 1/2, normal renormalised), Tukey IRLS
// weight (1 - (r/c)^2)^2; only the normal-direction distance counts.
// ORB (Section 2.1): r = x'(j_k) - o2_k, weight w_ORB * omega_k, omega_k = RANSAC weight of a
// preselected match, else clamp(1 - |r| / (5H), 0, 1).
// ARAP (Section 2.2, Eq. 5-6): all ordered pairs of control points, closed-form J^T W J blocks.
//
// Accumulation: the ICP and ORB passes add their 6x6 blocks into a block-sparse table (one
// entry per node pair that shares a template point) and their gradients into a vector; the
// ARAP pass builds each control point's 6 rows of A once (every pair block, the data blocks,
// the damping lambda (diag + eps)) and b = -(J^T W r), writing the full rows into the refinement
// matrix and the part left of the diagonal block, then the damped diagonal block, into the
// matrix the factorisation overwrites.
#include <math.h>

#include "ds_internal.cuh"

namespace ds {

struct Q {
  float w, x, y, z;
};
struct V {
  float x, y, z;
};

__device__ __forceinline__ Q q4(float4 a) { return {a.x, a.y, a.z, a.w}; }
__device__ __forceinline__ V v3(float4 a) { return {a.x, a.y, a.z}; }
__device__ __forceinline__ Q qmul(Q a, Q b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
          a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
          a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ Q qconj(Q a) { return {a.w, -a.x, -a.y, -a.z}; }
__device__ __forceinline__ float qdot(Q a, Q b) {
  return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z;
}
__device__ __forceinline__ float dot(V a, V b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V cross(V a, V b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V add(V a, V b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V sub(V a, V b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V mul(V a, float s) { return {a.x * s, a.y * s, a.z * s}; }

// ----------------------------------------------------------------------------- node update

// FP64 state step and the FP32 node tables of the next linearisation, one thread per node.
// step: apply x (the Gauss-Newton step); it >= 0: the first CTA of each problem records the
// linearisation's costs into hist[it]; the accumulators are cleared for the next linearisation
// (it < 0, the start of a solve, also clears w_ARAP and the status word).
__device__ void node_update(const ProbDesc& D, int i, bool step) {
  const double* x = D.x;
  double* q64 = D.q64;
  double* t64 = D.t64;
  const double* g64 = D.g64;
  const double* gc = D.gc;
  double qw = q64[4 * i], qx = q64[4 * i + 1], qy = q64[4 * i + 2], qz = q64[4 * i + 3];
  double tx = t64[3 * i], ty = t64[3 * i + 1], tz = t64[3 * i + 2];
  if (step) {
    double a = x[6 * i], b = x[6 * i + 1], c = x[6 * i + 2];
    double th = sqrt(a * a + b * b + c * c);
    double ew, sf;
    if (th > 0.0) {
      ew = cos(0.5 * th);
      sf = sin(0.5 * th) / th;
    } else {
      ew = 1.0;
      sf = 0.5;
    }
    double ex = sf * a, ey = sf * b, ez = sf * c;
    // (ew, e) (x) q
    double nw = ew * qw - ex * qx - ey * qy - ez * qz;
    double nx = ew * qx + ex * qw + ey * qz - ez * qy;
    double ny = ew * qy - ex * qz + ey * qw + ez * qx;
    double nz = ew * qz + ex * qy - ey * qx + ez * qw;
    double nn = 1.0 / sqrt(nw * nw + nx * nx + ny * ny + nz * nz);
    if (nw < 0) nn = -nn;
    qw = nw * nn;
    qx = nx * nn;
    qy = ny * nn;
    qz = nz * nn;
    tx += x[6 * i + 3];
    ty += x[6 * i + 4];
    tz += x[6 * i + 5];
    q64[4 * i] = qw;
    q64[4 * i + 1] = qx;
    q64[4 * i + 2] = qy;
    q64[4 * i + 3] = qz;
    t64[3 * i] = tx;
    t64[3 * i + 1] = ty;
    t64[3 * i + 2] = tz;
  }
  double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                 2 * (qx * qy + qw * qz),     1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                 2 * (qx * qz - qw * qy),     2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
  double gx = g64[3 * i], gy = g64[3 * i + 1], gz = g64[3 * i + 2];
  double Rgx = R[0] * gx + R[1] * gy + R[2] * gz;
  double Rgy = R[3] * gx + R[4] * gy + R[5] * gz;
  double Rgz = R[6] * gx + R[7] * gy + R[8] * gz;
  double Tx = gx + tx - Rgx, Ty = gy + ty - Rgy, Tz = gz + tz - Rgz;
  // d = 1/2 (0, T) (x) q
  double dw = 0.5 * (-Tx * qx - Ty * qy - Tz * qz);
  double dx = 0.5 * (Tx * qw + Ty * qz - Tz * qy);
  double dy = 0.5 * (-Tx * qz + Ty * qw + Tz * qx);
  double dz = 0.5 * (Tx * qy - Ty * qx + Tz * qw);
  NodeGPU nd;
  nd.q = make_float4((float)qw, (float)qx, (float)qy, (float)qz);
  nd.d = make_float4((float)dw, (float)dx, (float)dy, (float)dz);
  nd.T = make_float4((float)Tx, (float)Ty, (float)Tz, 0.f);
  nd.w = make_float4((float)(Rgx + 0.5 * Tx), (float)(Rgy + 0.5 * Ty), (float)(Rgz + 0.5 * Tz),
                     0.f);
  D.node[i] = nd;
  PairNode p;
  double cxg = gx - gc[0], cyg = gy - gc[1], czg = gz - gc[2];
  p.q = nd.q;
  p.g = make_float4((float)cxg, (float)cyg, (float)czg, 0.f);
  p.p = make_float4((float)(cxg + tx), (float)(cyg + ty), (float)(czg + tz), 0.f);
  p.R0 = make_float4((float)R[0], (float)R[1], (float)R[2], 0.f);
  p.R1 = make_float4((float)R[3], (float)R[4], (float)R[5], 0.f);
  p.R2 = make_float4((float)R[6], (float)R[7], (float)R[8], 0.f);
  D.pn[i] = p;
}

__global__ void k_iter_end(const ProbDesc* const* __restrict__ descs, const int2* __restrict__ tab,
                           int it, int step) {
  const int2 w = tab[blockIdx.x];
  if (!descs[w.x]) return;   // not in this solve
  const ProbDesc& D = *descs[w.x];
  if (w.y == 0 && threadIdx.x == 0) {
    double* acc = D.acc;
    if (it >= 0) {
      double* hrow = D.hist + 6 * it;
      hrow[0] = acc[ACC_COST_ICP] + acc[ACC_COST_ORB] + acc[ACC_COST_ARAP];
      hrow[1] = acc[ACC_COST_ICP];
      hrow[2] = acc[ACC_COST_ORB];
      hrow[3] = acc[ACC_COST_ARAP];
      hrow[4] = acc[ACC_NVALID];
      hrow[5] = acc[ACC_W_ARAP];
    }
    const int upto = it < 0 ? ACC_COUNT : ACC_W_ARAP;
    for (int k = 0; k < upto; ++k) acc[k] = 0.0;
  }
  const int i = w.y * 128 + threadIdx.x;
  if (i < D.N) node_update(D, i, step != 0);
}

void launch_iter_end(const BatchTabs& B, int it, bool step, cudaStream_t s) {
  k_iter_end<<<B.n_nodes, 128, 0, s>>>(B.d, B.nodes, it, step ? 1 : 0);
  ++g_launches;
}

// Zeroes the data-term blocks / gradient and the factorisation / solve counters of every
// problem, and the batch's ticket heads (not its timeout word).
__global__ void k_iter_begin(const ProbDesc* const* __restrict__ descs, int* __restrict__ words) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 5) words[threadIdx.x] = 0;
  if (!descs[blockIdx.x]) return;   // not in this solve
  const ProbDesc& D = *descs[blockIdx.x];
  const int nth = blockDim.x * gridDim.y;
  const int t0 = blockIdx.y * blockDim.x + threadIdx.x;
  float* blk = D.blk;
  const int nb = 36 * D.nbp;
  for (int e = t0; e < nb; e += nth) blk[e] = 0.f;
  for (int e = t0; e < D.n; e += nth) D.gdata[e] = 0.f;
  const int nt = D.lp.nt;
  const int nc = nt + 2 * nt * nt;
  for (int e = t0; e < nc; e += nth) D.lp.cnt[e] = 0;
  for (int e = t0; e < 2 * nt; e += nth) D.lp.flags[e] = 0;
}

void launch_iter_begin(const BatchTabs& B, cudaStream_t s) {
  k_iter_begin<<<dim3(B.P, 8), 256, 0, s>>>(B.d, B.words);
  ++g_launches;
}

// ----------------------------------------------------------------------------- blending

struct Blend {
  Q br, bd;      // blended dual quaternion (unnormalised)
  float inv_s;   // 1 / |b_r|^2
  V x;           // warped point
  float sgn[4];  // sign alignment per slot
};

// Blends the 4 node transforms in nd[] (registers or shared memory) at template point p.
__device__ __forceinline__ void blend_nodes(const NodeGPU* nd, const float* alpha, int near, V p,
                                            Blend& B) {
  // the nearest node's rotation, picked by selects (a runtime index into a register array would
  // place it in local memory)
  const float4 qn4 = near == 0 ? nd[0].q : near == 1 ? nd[1].q : near == 2 ? nd[2].q : nd[3].q;
  Q qn = q4(qn4);
  Q br = {0, 0, 0, 0}, bd = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Q qk = q4(nd[k].q), dk = q4(nd[k].d);
    float s = qdot(qk, qn) >= 0.f ? 1.f : -1.f;
    B.sgn[k] = s;
    float a = alpha[k] * s;
    br.w += a * qk.w;
    br.x += a * qk.x;
    br.y += a * qk.y;
    br.z += a * qk.z;
    bd.w += a * dk.w;
    bd.x += a * dk.x;
    bd.y += a * dk.y;
    bd.z += a * dk.z;
  }
  V bv = {br.x, br.y, br.z}, dv = {bd.x, bd.y, bd.z};
  float bw = br.w, dw = bd.w;
  float s = bw * bw + dot(bv, bv);
  // rotation part (bw^2 - |bv|^2) p + 2 (bv.p) bv + 2 bw (bv x p)
  V y = add(add(mul(p, bw * bw - dot(bv, bv)), mul(bv, 2.f * dot(bv, p))),
            mul(cross(bv, p), 2.f * bw));
  // translation part 2 (bw dv - dw bv + bv x dv)
  y = add(y, mul(sub(sub(mul(dv, bw), mul(bv, dw)), mul(cross(dv, bv), 1.f)), 2.f));
  B.br = br;
  B.bd = bd;
  B.inv_s = 1.f / s;
  B.x = mul(y, B.inv_s);
}

__device__ __forceinline__ void blend_point(const NodeGPU* __restrict__ node, const int* nid,
                                            const float* alpha, int near, V p, Blend& B,
                                            NodeGPU* nd) {
#pragma unroll
  for (int k = 0; k < 4; ++k) nd[k] = node[nid[k]];
  blend_nodes(nd, alpha, near, p, B);
}

// h = d(n . x') / db for a direction n (8 entries: b_r then b_d).
__device__ __forceinline__ void dir_grad(V n, V p, const Blend& B, float* h) {
  V bv = {B.br.x, B.br.y, B.br.z}, dv = {B.bd.x, B.bd.y, B.bd.z};
  float bw = B.br.w, dw = B.bd.w;
  float np = dot(n, p), nbv = dot(n, bv), bvp = dot(bv, p), nx = dot(n, B.x);
  float g0 = 2.f * bw * np + 2.f * dot(n, cross(bv, p)) + 2.f * dot(n, dv);
  V gv = add(add(mul(bv, -2.f * np), mul(add(mul(p, nbv), mul(n, bvp)), 2.f)),
             add(mul(cross(p, n), 2.f * bw), add(mul(n, -2.f * dw), mul(cross(dv, n), 2.f))));
  float gdw = -2.f * nbv;
  V gdv = add(mul(n, 2.f * bw), mul(cross(n, bv), 2.f));
  float is = B.inv_s, t = 2.f * nx;
  h[0] = (g0 - t * bw) * is;
  h[1] = (gv.x - t * bv.x) * is;
  h[2] = (gv.y - t * bv.y) * is;
  h[3] = (gv.z - t * bv.z) * is;
  h[4] = gdw * is;
  h[5] = gdv.x * is;
  h[6] = gdv.y * is;
  h[7] = gdv.z * is;
}

// Jacobian (6) of n . x' w.r.t. one node's (dtheta, dt), scaled by `scale`.
__device__ __forceinline__ void slot_jac(const float* h, const NodeGPU& nd, float scale,
                                         float* J) {
  Q qc = qconj(q4(nd.q));
  Q f = qmul({h[0], h[1], h[2], h[3]}, qc);
  Q e = qmul({h[4], h[5], h[6], h[7]}, qc);
  V ev = {e.x, e.y, e.z};
  V ew = cross(ev, v3(nd.w));
  V T = v3(nd.T);
  J[0] = scale * (0.5f * f.x - 0.25f * e.w * T.x + 0.5f * ew.x);
  J[1] = scale * (0.5f * f.y - 0.25f * e.w * T.y + 0.5f * ew.y);
  J[2] = scale * (0.5f * f.z - 0.25f * e.w * T.z + 0.5f * ew.z);
  J[3] = scale * 0.5f * ev.x;
  J[4] = scale * 0.5f * ev.y;
  J[5] = scale * 0.5f * ev.z;
}

// ----------------------------------------------------------------------------- ICP

// One warp per segment (a run of sorted template points sharing the same 4 nodes); a CTA's
// warp w takes segments base + w + 8 k, k < kSegPerWarp. The segment's 4 node transforms are
// staged in the warp's shared memory. The lanes take 32 of the segment's points at a time: each
// forms its point's association, Tukey weight and sqrt-weighted Jacobian row (24 entries, plus
// the weighted residual) and stages it in the warp's shared block, column-major (column e of
// point t at [e][t], so that four consecutive points of a column are one 16-byte load); then
// every lane accumulates 12 fixed entries of the segment's 384 outputs over those points, four
// points per step (points past the segment's end were staged as zeros). While a batch is
// worked on, the next batch's template points are prefetched into L2, and the target point and
// normal of a pixel are loaded together. Lanes 0..29 own two rows of one 6 x 6 slot-pair block
// (block l / 3, rows 2 (l % 3) and 2 (l % 3) + 1), lanes 30 and 31 own twelve gradient entries
// each. At the end of the segment each lane adds its 12 entries with
// one atomic each; cost, weight and count go out with one atomic triple per warp. Warps never
// wait for one another.
// BF16 x BF16 -> FP32 warp-level tensor-core product D += A B (m16n8k16, A row-major 16 x 16,
// B column-major 16 x 8, fragments as the PTX ISA lays them out for lane (g = lane / 4,
// t = lane % 4)).
__device__ __forceinline__ void mma_bf16_16x8x16(float (&d)[4], const unsigned (&a)[4],
                                                 const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// two floats rounded to BF16 (nearest even) and packed, the first in the low half
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  unsigned r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

template <bool kTcJtj>
__global__ __launch_bounds__(kTile, 2) void k_icp(const ProbDesc* const* __restrict__ descs,
                                                  const int2* __restrict__ tab) {
  const int2 wk = tab[blockIdx.x];
  if (!descs[wk.x]) return;   // not in this solve
  const ProbDesc& D = *descs[wk.x];
  const float4* __restrict__ tp = D.tp;
  const float4* __restrict__ tw = D.tw;
  const int4* __restrict__ segnodes = D.seg;
  const int* __restrict__ segbp = D.segbp;
  const int* __restrict__ segstart = D.segstart;
  const NodeGPU* __restrict__ node = D.node;
  const float4* __restrict__ tgt_pt = D.tpts;
  const float4* __restrict__ tgt_nrm = D.tnrm;
  const int W = D.W, H = D.H;
  const float fx = D.fx, fy = D.fy, cx = D.cx, cy = D.cy, c = D.tukey_c;
  const bool bilinear = D.assoc == 1;
  float* __restrict__ blk = D.blk;
  float* __restrict__ gdata = D.gdata;
  double* __restrict__ acc = D.acc;
  // point stride of a staged column: a multiple of 4 floats for the FP32 path's 4-point loads;
  // a multiple of 2 for the tensor-core path's point pairs, whose segment sums below must also
  // fit in the 48 KB of static shared memory
  constexpr int kJS = kTcJtj ? 34 : 36;
  __shared__ __align__(16) float sJ[kSegPerCta][25][kJS];
  __shared__ NodeGPU sNode[kSegPerCta][4];
  // tensor-core path: each warp's running 24 x 24 segment sum (entries owned by fixed lanes)
  __shared__ float sAcc[kTcJtj ? kSegPerCta : 1][kTcJtj ? 24 * 24 : 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool grad = lane >= 30;
  const int q = grad ? 0 : lane / 3;
  const int ra = 6 * kSlotPairI(q) + 2 * (lane % 3);   // this lane's two Jacobian rows
  const int cb = 6 * kSlotPairJ(q);                    // and the partner slot's columns
  const int g0 = (lane - 30) * 12;                     // gradient entries of lanes 30, 31
  float(*cols)[kJS] = sJ[warp];
  NodeGPU* nd = sNode[warp];
  float cost = 0.f, wsum = 0.f, nval = 0.f;
  const int mg = lane >> 2, mt4 = lane & 3;   // mma fragment coordinates (tensor-core path)
  float* sacc = sAcc[kTcJtj ? warp : 0];
  if (kTcJtj) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = 16 * i + mg + (e >= 2 ? 8 : 0), col = 8 * j + 2 * mt4 + (e & 1);
          if (row < 24) sacc[row * 24 + col] = 0.f;
        }
  }
  for (int k = 0; k < kSegPerWarp; ++k) {
    const int sg = wk.y * kSegPerCta * kSegPerWarp + k * kSegPerCta + warp;
    if (sg >= D.S) break;
    const int lo = segstart[sg], hi = segstart[sg + 1];
    const int4 nn = segnodes[sg];
    __syncwarp();
    if (lane < 16) {
      const int sl = lane >> 2, f = lane & 3;
      const int id = sl == 0 ? nn.x : sl == 1 ? nn.y : sl == 2 ? nn.z : nn.w;
      reinterpret_cast<float4*>(&nd[sl])[f] = reinterpret_cast<const float4*>(&node[id])[f];
    }
    __syncwarp();
    float a[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) a[e] = 0.f;
    for (int c0 = lo; c0 < hi; c0 += 32) {
      const int pidx = c0 + lane;
      if (pidx + 32 < hi) {   // the next batch's template point and weights, into L2
        asm volatile("prefetch.global.L2 [%0];" ::"l"(tp + pidx + 32));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(tw + pidx + 32));
      }
      float rt = 0.f;
      bool staged = false;   // the point's Jacobian row is in the staging block
      if (pidx < hi) {
        const float4 pa = tp[pidx];
        const int near = __float_as_int(pa.w) & 3;
        const float4 al = tw[pidx];
        const float alp[4] = {al.x, al.y, al.z, al.w};
        const V p = {pa.x, pa.y, pa.z};
        Blend B;
        blend_nodes(nd, alp, near, p, B);
        const V x = B.x;
        bool assoc_ok = false;
        V tqv = {0.f, 0.f, 0.f}, n = {0.f, 0.f, 0.f};
        if (x.z > 0.f) {
          const float u = fx * x.x / x.z + cx;
          const float v = fy * x.y / x.z + cy;
          if (!bilinear) {
            const float pu = floorf(u + 0.5f), pv = floorf(v + 0.5f);
            if (pu >= 0.f && pu < (float)W && pv >= 0.f && pv < (float)H) {
              const int pix = (int)pv * W + (int)pu;
              const float4 tq = tgt_pt[pix];
              const float4 n4 = tgt_nrm[pix];
              if (tq.w > 0.f) {
                tqv = {tq.x, tq.y, tq.z};
                n = {n4.x, n4.y, n4.z};
                assoc_ok = true;
              }
            }
          } else {
            // the 4 pixels around (u, v), bilinear weights from the fractional parts; corners
            // outside the image or not usable are dropped and the rest renormalised, valid iff
            // the usable weight is >= 1/2
            const float u0 = floorf(u), v0 = floorf(v);
            const float a = u - u0, b = v - v0;
            const float wc[4] = {(1.f - a) * (1.f - b), a * (1.f - b), (1.f - a) * b, a * b};
            float ws = 0.f;
            V qs = {0.f, 0.f, 0.f}, ns = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
              const float cu = u0 + (float)(c4 & 1), cv = v0 + (float)(c4 >> 1);
              if (cu >= 0.f && cu <= (float)(W - 1) && cv >= 0.f && cv <= (float)(H - 1)) {
                const int pc = (int)cv * W + (int)cu;
                const float4 Xc = tgt_pt[pc];
                const float4 Nc = tgt_nrm[pc];
                if (Xc.w > 0.f) {
                  ws += wc[c4];
                  qs = add(qs, mul({Xc.x, Xc.y, Xc.z}, wc[c4]));
                  ns = add(ns, mul({Nc.x, Nc.y, Nc.z}, wc[c4]));
                }
              }
            }
            const float l2 = dot(ns, ns);
            if (ws >= 0.5f && l2 > 0.f) {
              tqv = mul(qs, 1.f / ws);
              n = mul(ns, rsqrtf(l2));
              assoc_ok = true;
            }
          }
        }
        if (assoc_ok) {
          const float r = dot(n, sub(x, tqv));
          nval += 1.f;
          const float cc6 = c * c * (1.f / 6.f);
          if (fabsf(r) < c) {
            const float uu = r / c;
            const float sig = 1.f - uu * uu;
            wsum += sig * sig;
            cost += cc6 * (1.f - sig * sig * sig);
            float h[8];
            dir_grad(n, p, B, h);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              float J6[6];
              slot_jac(h, nd[s], alp[s] * B.sgn[s] * sig, J6);
#pragma unroll
              for (int i = 0; i < 6; ++i) cols[6 * s + i][lane] = J6[i];
            }
            rt = sig * r;
            staged = true;
          } else {
            cost += cc6;
          }
        }
      }
      if (!staged) {
#pragma unroll
        for (int i = 0; i < 24; ++i) cols[i][lane] = 0.f;
      }
      cols[24][lane] = rt;
      __syncwarp();
      const int np = min(32, hi - c0);
      if (kTcJtj) {
        // this 32-point batch's 24 x 24 J^T W J in FP32 mma accumulators, 2 row tiles (rows
        // 0..15, 16..31; rows >= 24 are zero) x 3 column tiles (columns 0..23), then added to the
        // lane's own entries of the segment sum in shared memory (fixed fragment ownership, so no
        // lane touches another's entries); rows of the points past the segment's end are zero,
        // so whole 16-point steps are summed
        float cm[2][3][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) cm[i][j][e] = 0.f;
        for (int k0 = 0; k0 < np; k0 += 16) {
          // entries (point k0 + 2 t4 + {0, 1}) and (point k0 + 2 t4 + {8, 9}) of a column
          const int t0 = k0 + 2 * mt4;
          auto pair = [&](int m, int t) {
            const float2 v = *reinterpret_cast<const float2*>(&cols[m][t]);
            return pack_bf16(v.x, v.y);
          };
          unsigned af[2][4];
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            // A = J^T (row m = Jacobian column m, column k = point k0 + k)
            const int m0 = 16 * i + mg, m1 = m0 + 8;
            const bool v1 = m1 < 24;
            af[i][0] = pair(m0, t0);
            af[i][1] = v1 ? pair(m1, t0) : 0u;
            af[i][2] = pair(m0, t0 + 8);
            af[i][3] = v1 ? pair(m1, t0 + 8) : 0u;
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            // B = J (row k = point, column n = Jacobian column 8 j + n)
            const int nn = 8 * j + mg;
            const unsigned bf[2] = {pair(nn, t0), pair(nn, t0 + 8)};
#pragma unroll
            for (int i = 0; i < 2; ++i) mma_bf16_16x8x16(cm[i][j], af[i], bf);
          }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int row = 16 * i + mg + (e >= 2 ? 8 : 0), col = 8 * j + 2 * mt4 + (e & 1);
              if (row < 24) sacc[row * 24 + col] += cm[i][j][e];
            }
        // the gradient J^T W r stays FP32: lane l < 24 sums entry l
        if (lane < 24) {
          for (int t = 0; t < np; ++t) a[0] += cols[lane][t] * cols[24][t];
        }
      } else if (!grad) {
        // four points per step, in point order (the points past np add exact zeros)
        for (int t = 0; t < np; t += 4) {
          const float4 x0 = *reinterpret_cast<const float4*>(&cols[ra][t]);
          const float4 x1 = *reinterpret_cast<const float4*>(&cols[ra + 1][t]);
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) {
            const float4 y = *reinterpret_cast<const float4*>(&cols[cb + cc][t]);
            a[cc] += x0.x * y.x;
            a[6 + cc] += x1.x * y.x;
            a[cc] += x0.y * y.y;
            a[6 + cc] += x1.y * y.y;
            a[cc] += x0.z * y.z;
            a[6 + cc] += x1.z * y.z;
            a[cc] += x0.w * y.w;
            a[6 + cc] += x1.w * y.w;
          }
        }
      } else {
        for (int t = 0; t < np; t += 4) {
          const float4 rr = *reinterpret_cast<const float4*>(&cols[24][t]);
#pragma unroll
          for (int e = 0; e < 12; ++e) {
            const float4 x = *reinterpret_cast<const float4*>(&cols[g0 + e][t]);
            a[e] += x.x * rr.x;
            a[e] += x.y * rr.y;
            a[e] += x.z * rr.z;
            a[e] += x.w * rr.w;
          }
        }
      }
      __syncwarp();
    }
    if (kTcJtj) {
      // the lane's entries of the segment sum: accumulator element (row, col) of tile (i, j) is
      // row 16 i + g (+ 8 for e >= 2), column 8 j + 2 t (+ 1 for odd e); it belongs to slot-pair
      // block (row / 6, col / 6) when that is a lower pair. Zeroed again for the next segment.
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int row = 16 * i + mg + (e >= 2 ? 8 : 0), col = 8 * j + 2 * mt4 + (e & 1);
            const int si = row / 6, sj = col / 6;
            if (row >= 24) continue;
            const float v = sacc[row * 24 + col];
            sacc[row * 24 + col] = 0.f;
            if (si >= sj && v != 0.f)
              atomicAdd(blk + (size_t)segbp[sg * 10 + si * (si + 1) / 2 + sj] * 36 +
                            (row % 6) * 6 + col % 6,
                        v);
          }
      if (lane < 24 && a[0] != 0.f) {
        const int sl = lane / 6;
        const int ndi = sl == 0 ? nn.x : sl == 1 ? nn.y : sl == 2 ? nn.z : nn.w;
        atomicAdd(&gdata[6 * ndi + lane % 6], a[0]);
      }
    } else if (!grad) {
      float* dst = blk + (size_t)segbp[sg * 10 + q] * 36 + 12 * (lane % 3);
#pragma unroll
      for (int e = 0; e < 12; ++e)
        if (a[e] != 0.f) atomicAdd(dst + e, a[e]);
    } else {
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const int kk = g0 + e, sl = kk / 6;
        const int ndi = sl == 0 ? nn.x : sl == 1 ? nn.y : sl == 2 ? nn.z : nn.w;
        if (a[e] != 0.f) atomicAdd(&gdata[6 * ndi + kk % 6], a[e]);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cost += __shfl_xor_sync(0xffffffffu, cost, o);
    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    nval += __shfl_xor_sync(0xffffffffu, nval, o);
  }
  if (lane == 0 && nval != 0.f) {
    atomicAdd(&acc[ACC_COST_ICP], (double)cost);
    atomicAdd(&acc[ACC_WSUM_ICP], (double)wsum);
    atomicAdd(&acc[ACC_NVALID], (double)nval);
  }
}

void launch_icp(const BatchTabs& B, cudaStream_t s) {
  if (B.n_icp <= 0) return;
  if (B.jtj)
    k_icp<true><<<B.n_icp, kTile, 0, s>>>(B.d, B.icp);
  else
    k_icp<false><<<B.n_icp, kTile, 0, s>>>(B.d, B.icp);
  ++g_launches;
}

// ----------------------------------------------------------------------------- ORB

__global__ __launch_bounds__(128) void k_orb(const ProbDesc* const* __restrict__ descs,
                                             int ctas_per_problem) {
  if (!descs[blockIdx.x / ctas_per_problem]) return;   // not in this solve
  const ProbDesc& D = *descs[blockIdx.x / ctas_per_problem];
  const int* __restrict__ midx = D.midx;
  const float* __restrict__ mxyz = D.mxyz;
  const int M = D.M;
  const int* __restrict__ rank = D.rank;
  const float4* __restrict__ tp = D.tp;
  const float4* __restrict__ tw = D.tw;
  const int4* __restrict__ segnodes = D.seg;
  const int* __restrict__ segbp = D.segbp;
  const NodeGPU* __restrict__ node = D.node;
  const uint32_t* __restrict__ mask = D.mask;
  const float* __restrict__ what = D.what;
  const float H = D.H_mm, w_orb = D.w_orb;
  float* __restrict__ blk = D.blk;
  float* __restrict__ gdata = D.gdata;
  double* __restrict__ acc = D.acc;
  const int stride = ctas_per_problem * blockDim.x;
  const int first = (blockIdx.x % ctas_per_problem) * blockDim.x + threadIdx.x;
  const int rounds = (M + stride - 1) / stride;
  for (int rd = 0; rd < rounds; ++rd) {
  const int k = first + rd * stride;
  float cost = 0.f, wsum = 0.f;
  if (k < M) {
    int sp = rank[midx[k]];
    if (sp >= 0) {
      float4 a = tp[sp];
      int bits = __float_as_int(a.w);
      int seg = bits >> 2, near = bits & 3;
      int4 nn = segnodes[seg];
      float4 al = tw[sp];
      int nid[4] = {nn.x, nn.y, nn.z, nn.w};
      float alp[4] = {al.x, al.y, al.z, al.w};
      V p = {a.x, a.y, a.z};
      Blend B;
      NodeGPU nd[4];
      blend_point(node, nid, alp, near, p, B, nd);
      V r = sub(B.x, {mxyz[3 * k], mxyz[3 * k + 1], mxyz[3 * k + 2]});
      float d = sqrtf(dot(r, r));
      bool pre = (mask[k >> 5] >> (k & 31)) & 1u;
      float om = pre ? what[k] : fminf(fmaxf(1.f - d / (5.f * H), 0.f), 1.f);
      cost = 0.5f * w_orb * om * dot(r, r);
      wsum = om;
      float sig = sqrtf(w_orb * om);
      if (sig > 0.f) {
        float J[3][24];
        const V ax[3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
        for (int row = 0; row < 3; ++row) {
          float h[8];
          dir_grad(ax[row], p, B, h);
#pragma unroll
          for (int s = 0; s < 4; ++s) slot_jac(h, nd[s], alp[s] * B.sgn[s] * sig, &J[row][6 * s]);
        }
        float rr[3] = {sig * r.x, sig * r.y, sig * r.z};
        // fully unrolled so that J stays in registers
#pragma unroll
        for (int kk = 0; kk < 10; ++kk) {
          float* dst = blk + (size_t)segbp[seg * 10 + kk] * 36;
          const int ib = 6 * kSlotPairI(kk), jb = 6 * kSlotPairJ(kk);
#pragma unroll
          for (int e = 0; e < 36; ++e) {
            const int ai = ib + e / 6, bj = jb + e % 6;
            const float v = J[0][ai] * J[0][bj] + J[1][ai] * J[1][bj] + J[2][ai] * J[2][bj];
            if (v != 0.f) atomicAdd(dst + e, v);
          }
        }
#pragma unroll
        for (int a2 = 0; a2 < 24; ++a2) {
          const float v = J[0][a2] * rr[0] + J[1][a2] * rr[1] + J[2][a2] * rr[2];
          const int ndid = a2 < 6 ? nn.x : a2 < 12 ? nn.y : a2 < 18 ? nn.z : nn.w;
          if (v != 0.f) atomicAdd(&gdata[6 * ndid + a2 % 6], v);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cost += __shfl_xor_sync(0xffffffffu, cost, o);
    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  }
  if ((threadIdx.x & 31) == 0 && (cost != 0.f || wsum != 0.f)) {
    atomicAdd(&acc[ACC_COST_ORB], (double)cost);
    atomicAdd(&acc[ACC_WSUM_ORB], (double)wsum);
  }
  }
}

void launch_orb(const BatchTabs& B, cudaStream_t s) {
  k_orb<<<B.P * B.orb_ctas, 128, 0, s>>>(B.d, B.orb_ctas);
  ++g_launches;
}

// ----------------------------------------------------------------------------- ARAP + assembly

template <typename T>
__device__ __forceinline__ void store_out(T* p, float v) {
  *p = (T)v;
}

constexpr int kArapMaxN = 2048;   // control points per problem (the API's limit)
constexpr int kArapChunk = 256;   // partner nodes per panel chunk (= threads per CTA)

// Copies len floats of a shared-memory row to global memory: 16-byte stores (FP32, row start
// 16-byte aligned) with a scalar tail; FP64 destinations are converted element by element.
template <typename T>
__device__ __forceinline__ void row_out(T* dst, const float* src, int len, bool aligned) {
  if constexpr (sizeof(T) == 4) {
    if (aligned) {
      const int n4 = len >> 2;
      for (int k = threadIdx.x; k < n4; k += blockDim.x)
        reinterpret_cast<float4*>(dst)[k] = reinterpret_cast<const float4*>(src)[k];
      for (int k = 4 * n4 + threadIdx.x; k < len; k += blockDim.x) dst[k] = src[k];
      return;
    }
  }
  for (int k = threadIdx.x; k < len; k += blockDim.x) store_out(dst + k, src[k]);
}

// The terms of one ordered pair (i1 = the CTA's row node with state q1, g1, p1, R1 rows; i2 = o)
// shared by the diagonal block, the gradient and the off-diagonal block A(i1, i2); adds the
// pair's diagonal-block, gradient and cost contributions to the caller's accumulators.
struct ArapPair {
  Q r;           // q_i2 (x) q_i1*
  V v, u2;       // unit(p_i2 - p_i1), unit(R_i2 (g_i1 - g_i2))
  float s, Wr, ca;
  float C[9];    // W_a [u]x P / l
  float Tm[6];   // W_l v v^T + W_a P / l^2 (symmetric, xx xy xz yy yz zz)
};
__device__ __forceinline__ ArapPair arap_pair(const PairNode& o, Q q1, V g1, V p1, V R1a, V R1b,
                                              V R1c, float wA, float inv2sig2, float w_angle,
                                              float w_rot, float (&Dtt)[6], float (&Dtx)[9],
                                              float (&Dxx)[6], float (&G)[6], float& cost) {
  ArapPair pr;
  const Q q2 = q4(o.q);
  const V g2 = v3(o.g), p2 = v3(o.p);
  V dg = sub(g2, g1);
  float L0 = sqrtf(dot(dg, dg));
  V e = sub(p2, p1);
  float l = sqrtf(dot(e, e));
  float il = 1.f / l;
  V v = mul(e, il);
  V a = {dot(R1a, dg), dot(R1b, dg), dot(R1c, dg)};
  V u = mul(a, rsqrtf(dot(a, a)));
  V mdg = {-dg.x, -dg.y, -dg.z};
  V a2 = {dot(v3(o.R0), mdg), dot(v3(o.R1), mdg), dot(v3(o.R2), mdg)};
  V u2 = mul(a2, rsqrtf(dot(a2, a2)));
  Q r = qmul(q2, qconj(q1));
  float qq = qdot(q1, q2);
  float s = qq >= 0.f ? 1.f : -1.f;
  float w = wA * __expf(-dot(dg, dg) * inv2sig2);
  float Wl = w, Wa = w * w_angle, Wr = w * w_rot;
  float rl = l - L0;
  V ang = sub(u, v);
  Q rot = {q1.w - s * q2.w, q1.x - s * q2.x, q1.y - s * q2.y, q1.z - s * q2.z};
  cost += 0.5f * (Wl * rl * rl + Wa * dot(ang, ang) + Wr * qdot(rot, rot));
  // C = W_a [u]x P / l with P = I - v v^T:  [u]x - (u x v) v^T
  V uxv = cross(u, v);
  float ca = Wa * il;
  const float C[9] = {ca * (0.f - uxv.x * v.x), ca * (-u.z - uxv.x * v.y), ca * (u.y - uxv.x * v.z),
                      ca * (u.z - uxv.y * v.x), ca * (0.f - uxv.y * v.y), ca * (-u.x - uxv.y * v.z),
                      ca * (-u.y - uxv.z * v.x), ca * (u.x - uxv.z * v.y), ca * (0.f - uxv.z * v.z)};
  // Tm = W_l v v^T + W_a (I - v v^T) / l^2
  float tb = Wa * il * il;
  float tv = Wl - tb;
  const float Tm[6] = {tb + tv * v.x * v.x, tv * v.x * v.y, tv * v.x * v.z,
                       tb + tv * v.y * v.y, tv * v.y * v.z, tb + tv * v.z * v.z};
  // diag
  float hr = 0.5f * Wr;
  Dtt[0] += Wa * (1.f - u.x * u.x) + hr;
  Dtt[1] += -Wa * u.x * u.y;
  Dtt[2] += -Wa * u.x * u.z;
  Dtt[3] += Wa * (1.f - u.y * u.y) + hr;
  Dtt[4] += -Wa * u.y * u.z;
  Dtt[5] += Wa * (1.f - u.z * u.z) + hr;
#pragma unroll
  for (int i = 0; i < 9; ++i) Dtx[i] += C[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) Dxx[i] += 2.f * Tm[i];
  // gradient
  V rv = {r.x, r.y, r.z};
  G[0] += -Wa * uxv.x - s * Wr * rv.x;
  G[1] += -Wa * uxv.y - s * Wr * rv.y;
  G[2] += -Wa * uxv.z - s * Wr * rv.z;
  V Pu = sub(u, mul(v, dot(v, u)));
  V Pu2 = sub(u2, mul(v, dot(v, u2)));
  V gt = add(mul(v, -2.f * Wl * rl), mul(sub(Pu, Pu2), Wa * il));
  G[3] += gt.x;
  G[4] += gt.y;
  G[5] += gt.z;
  pr.r = r;
  pr.v = v;
  pr.u2 = u2;
  pr.s = s;
  pr.Wr = Wr;
  pr.ca = ca;
#pragma unroll
  for (int i = 0; i < 9; ++i) pr.C[i] = C[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) pr.Tm[i] = Tm[i];
  return pr;
}

// One CTA per block row i1. For every partner i2 != i1 the CTA evaluates both ordered pairs
// (i1, i2) and (i2, i1) in closed form; with u = unit(R_a (g_b - g_a)), v = unit(p_b - p_a),
// l = |p_b - p_a|, P = I - v v^T, r = q_b (x) q_a*, s = sign(q_a . q_b) and per-pair weights
// W_l = w, W_a = w w_angle, W_r = w w_rot (w = w_ARAP exp(-|g_a - g_b|^2 / 2 sigma^2)):
//   diag(i1)   += [[W_a (I - u u^T) + W_r/2 I, C], [C^T, 2 Tm]],  C = W_a [u]x P / l,
//                 Tm = W_l v v^T + W_a P / l^2
//   A(i1, i2)   = [[-s W_r / 2 (r_w I - [r_v]x), -C], [-C'^T, -2 Tm]]   (C' of the reverse pair)
//   grad(i1)   += [-W_a u x v - s W_r r_v, -2 W_l (l - l0) v + W_a (P u - P u') / l]
// (u' = unit(R_i2 (g_i1 - g_i2))). Only the lower blocks (i2 <= i1) are written.
template <typename T>
__global__ __launch_bounds__(256) void k_arap_assemble(const ProbDesc* const* __restrict__ descs,
                                                       const int2* __restrict__ tab,
                                                       int first_iter, int lin_only,
                                                       int diag_only, int deferred) {
  const int2 wk = tab[blockIdx.x];
  if (!descs[wk.x]) return;   // not in this solve
  const ProbDesc& D = *descs[wk.x];
  const PairNode* __restrict__ pn = D.pn;
  const int N = D.N;
  const float inv2sig2 = D.inv2sig2;
  const int* __restrict__ rowptr = D.rowptr;
  const int* __restrict__ rowcol = D.rowcol;
  const int* __restrict__ rowbp = D.rowbp;
  const float* __restrict__ blk = D.blk;
  const float* __restrict__ gdata = D.gdata;
  double* __restrict__ acc = D.acc;
  const double w_arap0 = D.w_arap0, eps = D.eps;
  const double lam = lin_only ? 0.0 : D.lam;
  const float w_orb = D.w_orb, w_angle = D.w_angle, w_rot = D.w_rot;
  T* __restrict__ Afac = lin_only ? (T*)D.Aref : (T*)D.lp.A;
  float* __restrict__ Aref = (!lin_only && D.write_ref) ? D.Aref : nullptr;
  double* __restrict__ b = D.b;
  float* __restrict__ D_adiag = D.adiag;
  extern __shared__ __align__(16) int smap[];          // node -> data block code of this row
  float* panel = reinterpret_cast<float*>(smap + kArapMaxN);  // 6 rows x kArapChunk nodes
  __shared__ float sRed[28][8];
  const int i1 = wk.y;
  const int n = 6 * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) smap[i] = -1;
  __syncthreads();
  for (int e = rowptr[i1] + threadIdx.x; e < rowptr[i1 + 1]; e += blockDim.x)
    smap[rowcol[e]] = rowbp[e];
  double wa64;
  if (first_iter)
    wa64 = w_arap0 * (acc[ACC_WSUM_ICP] + (double)w_orb * acc[ACC_WSUM_ORB]) / N;
  else
    wa64 = acc[ACC_W_ARAP];
  __syncthreads();
  if (first_iter && i1 == 0 && threadIdx.x == 0) acc[ACC_W_ARAP] = wa64;
  const float wA = (float)wa64;
  const PairNode me = pn[i1];
  const Q q1 = q4(me.q);
  const V g1 = v3(me.g), p1 = v3(me.p);
  const V R1a = v3(me.R0), R1b = v3(me.R1), R1c = v3(me.R2);
  // diag accumulators: theta-theta (sym 6: xx xy xz yy yz zz), theta-t (9), t-t (sym 6)
  float Dtt[6] = {0, 0, 0, 0, 0, 0}, Dtx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  float Dxx[6] = {0, 0, 0, 0, 0, 0}, G[6] = {0, 0, 0, 0, 0, 0}, cost = 0.f;
  // The CTA builds its 6 matrix rows chunk by chunk (kArapChunk partner nodes, one per thread)
  // in shared memory and streams them out with coalesced 16-byte stores: the full rows into the
  // refinement matrix, the part left of the diagonal block into the factor. A(i1, i2) for
  // i2 > i1 is the transpose of A(i2, i1); the pair formula below, taken with i1 as the row,
  // gives it directly.
  constexpr int PW = 6 * kArapChunk;  // panel row width (floats)
  for (int ch = 0; ch * kArapChunk < N; ++ch) {
    const int i2 = ch * kArapChunk + threadIdx.x;
    const int ncol = 6 * min(kArapChunk, N - ch * kArapChunk);
    float* pc = panel + 6 * threadIdx.x;
    if (diag_only) {
      // block-Jacobi solves need only the diagonal block and the gradient of this row
      if (i2 < N && i2 != i1)
        arap_pair(pn[i2], q1, g1, p1, R1a, R1b, R1c, wA, inv2sig2, w_angle, w_rot, Dtt, Dtx, Dxx,
                  G, cost);
      continue;
    }
    if (i2 < N && i2 == i1) {
#pragma unroll
      for (int rr = 0; rr < 6; ++rr)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) pc[rr * PW + cc] = 0.f;  // written after the reduction
    } else if (i2 < N) {
      const ArapPair pr = arap_pair(pn[i2], q1, g1, p1, R1a, R1b, R1c, wA, inv2sig2, w_angle,
                                    w_rot, Dtt, Dtx, Dxx, G, cost);
      const Q r = pr.r;
      const V u2 = pr.u2, v = pr.v;
      const float s = pr.s, Wr = pr.Wr, ca = pr.ca;
      const float* C = pr.C;
      const float* Tm = pr.Tm;
      // off-diagonal block A(i1, i2) (rows: i1's theta,t; cols: i2's theta,t)
      float O[36];
      float hs = -0.5f * s * Wr;
      // theta-theta: hs (r_w I - [r_v]x)
      O[0 * 6 + 0] = hs * r.w;
      O[0 * 6 + 1] = hs * r.z;
      O[0 * 6 + 2] = -hs * r.y;
      O[1 * 6 + 0] = -hs * r.z;
      O[1 * 6 + 1] = hs * r.w;
      O[1 * 6 + 2] = hs * r.x;
      O[2 * 6 + 0] = hs * r.y;
      O[2 * 6 + 1] = -hs * r.x;
      O[2 * 6 + 2] = hs * r.w;
      // theta-t: -C
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) O[rr * 6 + 3 + cc] = -C[rr * 3 + cc];
      // t-theta: -C'^T, C' = W_a/l ([u2]x - (u2 x v) v^T)
      V u2xv = cross(u2, v);
      float Cp[9] = {ca * (0.f - u2xv.x * v.x), ca * (-u2.z - u2xv.x * v.y),
                     ca * (u2.y - u2xv.x * v.z), ca * (u2.z - u2xv.y * v.x),
                     ca * (0.f - u2xv.y * v.y), ca * (-u2.x - u2xv.y * v.z),
                     ca * (-u2.y - u2xv.z * v.x), ca * (u2.x - u2xv.z * v.y),
                     ca * (0.f - u2xv.z * v.z)};
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) O[(3 + rr) * 6 + cc] = -Cp[cc * 3 + rr];
      // t-t: -2 Tm
      O[3 * 6 + 3] = -2.f * Tm[0];
      O[3 * 6 + 4] = -2.f * Tm[1];
      O[3 * 6 + 5] = -2.f * Tm[2];
      O[4 * 6 + 3] = -2.f * Tm[1];
      O[4 * 6 + 4] = -2.f * Tm[3];
      O[4 * 6 + 5] = -2.f * Tm[4];
      O[5 * 6 + 3] = -2.f * Tm[2];
      O[5 * 6 + 4] = -2.f * Tm[4];
      O[5 * 6 + 5] = -2.f * Tm[5];
      const int code = deferred ? -1 : smap[i2];   // deferred: data blocks added later
      if (code >= 0) {
        const float* db = blk + (size_t)(code & ~kBlkTransposed) * 36;
        if (code & kBlkTransposed) {
#pragma unroll
          for (int rr = 0; rr < 6; ++rr)
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) O[rr * 6 + cc] += db[cc * 6 + rr];
        } else {
#pragma unroll
          for (int i = 0; i < 36; ++i) O[i] += db[i];
        }
      }
#pragma unroll
      for (int rr = 0; rr < 6; ++rr)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) pc[rr * PW + cc] = O[rr * 6 + cc];
    }
    __syncthreads();
    const int c0 = ch * PW;
    const int nlo = max(0, min(ncol, 6 * i1 - c0));  // factor columns left of the diagonal block
#pragma unroll 1
    for (int rr = 0; rr < 6; ++rr) {
      const float* src = panel + rr * PW;
      const size_t rowoff = (size_t)(6 * i1 + rr) * n + c0;
      if (Aref) row_out<float>(Aref + rowoff, src, ncol, (n & 3) == 0);
      row_out<T>(Afac + rowoff, src, nlo, (n & 3) == 0);
    }
    __syncthreads();
  }
  // block reduction of the 28 per-thread sums
  float vals[28];
#pragma unroll
  for (int i = 0; i < 6; ++i) vals[i] = Dtt[i];
#pragma unroll
  for (int i = 0; i < 9; ++i) vals[6 + i] = Dtx[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) vals[15 + i] = Dxx[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) vals[21 + i] = G[i];
  vals[27] = cost;
#pragma unroll
  for (int i = 0; i < 28; ++i) {
    float x = vals[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    vals[i] = x;
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < 28; ++i) sRed[i][warp] = vals[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    float t[28];
    for (int i = 0; i < 28; ++i) {
      float x = 0.f;
      for (int w = 0; w < nw; ++w) x += sRed[i][w];
      t[i] = x;
    }
    float D[36];
    // theta-theta
    D[0] = t[0]; D[1] = t[1]; D[2] = t[2];
    D[6] = t[1]; D[7] = t[3]; D[8] = t[4];
    D[12] = t[2]; D[13] = t[4]; D[14] = t[5];
    // theta-t and t-theta
    for (int rr = 0; rr < 3; ++rr)
      for (int cc = 0; cc < 3; ++cc) {
        D[rr * 6 + 3 + cc] = t[6 + rr * 3 + cc];
        D[(3 + cc) * 6 + rr] = t[6 + rr * 3 + cc];
      }
    // t-t
    D[21] = t[15]; D[22] = t[16]; D[23] = t[17];
    D[27] = t[16]; D[28] = t[18]; D[29] = t[19];
    D[33] = t[17]; D[34] = t[19]; D[35] = t[20];
    if (deferred) {   // ARAP-only diagonal block and gradient, for k_arap_finalize
      float* ad = D_adiag + 48 * (size_t)i1;
      for (int i = 0; i < 36; ++i) ad[i] = D[i];
      for (int j = 0; j < 6; ++j) ad[36 + j] = t[21 + j];
      atomicAdd(&acc[ACC_COST_ARAP], (double)t[27]);
      return;
    }
    int bp = smap[i1];
    if (bp >= 0) {
      const float* db = blk + (size_t)bp * 36;
      for (int i = 0; i < 36; ++i) D[i] += db[i];
    }
    for (int j = 0; j < 6; ++j) D[j * 7] += (float)(lam * ((double)D[j * 7] + eps));
    for (int rr = 0; rr < 6; ++rr)
      for (int cc = 0; cc < 6; ++cc) {
        store_out(Afac + (size_t)(6 * i1 + rr) * n + 6 * i1 + cc, D[rr * 6 + cc]);
        if (Aref) Aref[(size_t)(6 * i1 + rr) * n + 6 * i1 + cc] = D[rr * 6 + cc];
      }
    for (int j = 0; j < 6; ++j) b[6 * i1 + j] = -((double)t[21 + j] + (double)gdata[6 * i1 + j]);
    atomicAdd(&acc[ACC_COST_ARAP], (double)t[27]);
  }
}

template <typename T>
void launch_arap_assemble(const BatchTabs& B, bool first, bool lin_only, cudaStream_t s,
                          bool diag_only) {
  // dynamic shared memory: the node -> data block map of the row and the 6-row panel
  const int sm = sizeof(int) * kArapMaxN + sizeof(float) * 6 * 6 * kArapChunk;
  static PerDevice attr;
  set_smem_once(attr, k_arap_assemble<T>, sm);
  k_arap_assemble<T><<<B.n_rows, kArapChunk, sm, s>>>(B.d, B.rows, first ? 1 : 0,
                                                       lin_only ? 1 : 0, diag_only ? 1 : 0, 0);
  ++g_launches;
}

template void launch_arap_assemble<float>(const BatchTabs&, bool, bool, cudaStream_t, bool);
template void launch_arap_assemble<double>(const BatchTabs&, bool, bool, cudaStream_t, bool);

template <typename T>
void launch_arap_deferred(const BatchTabs& B, cudaStream_t s) {
  const int sm = sizeof(int) * kArapMaxN + sizeof(float) * 6 * 6 * kArapChunk;
  static PerDevice attr;
  set_smem_once(attr, k_arap_assemble<T>, sm);
  k_arap_assemble<T><<<B.n_rows, kArapChunk, sm, s>>>(B.d, B.rows, 0, 0, 0, 1);
  ++g_launches;
}

// After the deferred ARAP pass and the data terms: adds every data block of node row i (both
// triangles of the refinement matrix, the lower one of the factor copy), forms the diagonal
// block = ARAP + data, damps it and writes b_i = -(ARAP + data gradient). One CTA of 64 threads
// per node row; the row's block entries are spread over the threads (36 values each).
template <typename T>
__global__ __launch_bounds__(64) void k_arap_finalize(const ProbDesc* const* __restrict__ descs,
                                                      const int2* __restrict__ tab) {
  const int2 w = tab[blockIdx.x];
  if (!descs[w.x]) return;   // not in this solve
  const ProbDesc& D = *descs[w.x];
  const int i = w.y, n = D.n;
  T* Afac = (T*)D.lp.A;
  float* Aref = D.write_ref ? D.Aref : nullptr;
  const float* ad = D.adiag + 48 * (size_t)i;
  __shared__ float Db[36];
  if (threadIdx.x < 36) Db[threadIdx.x] = ad[threadIdx.x];
  __syncthreads();
  const int e0 = D.rowptr[i], ne = D.rowptr[i + 1] - e0;
  for (int q = threadIdx.x; q < 36 * ne; q += blockDim.x) {
    const int e = e0 + q / 36, k = q % 36, r = k / 6, cc = k % 6;
    const int c = D.rowcol[e], code = D.rowbp[e];
    const float* db = D.blk + (size_t)(code & ~kBlkTransposed) * 36;
    const float v = (code & kBlkTransposed) ? db[cc * 6 + r] : db[k];
    if (c == i) {
      Db[k] += v;   // the diagonal pair appears once in its row: one thread per entry
      continue;
    }
    const size_t off = (size_t)(6 * i + r) * n + 6 * c + cc;
    if (Aref) Aref[off] += v;
    if (c < i) Afac[off] += (T)v;
  }
  __syncthreads();
  if (threadIdx.x < 36) {
    const int r = threadIdx.x / 6, cc = threadIdx.x % 6;
    float v = Db[threadIdx.x];
    if (r == cc) v += (float)(D.lam * ((double)v + D.eps));
    const size_t off = (size_t)(6 * i + r) * n + 6 * i + cc;
    Afac[off] = (T)v;
    if (Aref) Aref[off] = v;
  }
  if (threadIdx.x < 6)
    D.b[6 * i + threadIdx.x] = -((double)ad[36 + threadIdx.x] + (double)D.gdata[6 * i + threadIdx.x]);
}

template <typename T>
void launch_arap_finalize(const BatchTabs& B, cudaStream_t s) {
  k_arap_finalize<T><<<B.n_rows, 64, 0, s>>>(B.d, B.rows);
  ++g_launches;
}
template void launch_arap_deferred<float>(const BatchTabs&, cudaStream_t);
template void launch_arap_deferred<double>(const BatchTabs&, cudaStream_t);
template void launch_arap_finalize<float>(const BatchTabs&, cudaStream_t);
template void launch_arap_finalize<double>(const BatchTabs&, cudaStream_t);

// Block-Jacobi step: x_i = A_ii^-1 b_i for every control point i, A_ii the damped 6 x 6 diagonal
// block written by the assembly; FP64 Cholesky of each block, one thread per node.
template <typename T>
__global__ void k_block_jacobi(const ProbDesc* const* __restrict__ descs,
                               const int2* __restrict__ tab) {
  const int2 w = tab[blockIdx.x];
  if (!descs[w.x]) return;   // not in this solve
  const ProbDesc& D = *descs[w.x];
  const int i = w.y * 128 + threadIdx.x;
  if (i >= D.N) return;
  const int n = D.n;
  const T* A = (const T*)D.lp.A;
  double L[6][6], y[6];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) L[r][c] = c <= r ? (double)A[(size_t)(6 * i + r) * n + 6 * i + c] : 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double p = L[j][j];
#pragma unroll
    for (int q = 0; q < j; ++q) p -= L[j][q] * L[j][q];
    if (!(p > 0.0)) {
      atomicCAS((unsigned long long*)(D.acc + ACC_STATUS), 0ull,
                __double_as_longlong((double)(6 * i + j + 1)));
      p = 1.0;
    }
    const double d = sqrt(p);
    L[j][j] = d;
#pragma unroll
    for (int r = j + 1; r < 6; ++r) {
      double v = L[r][j];
#pragma unroll
      for (int q = 0; q < j; ++q) v -= L[r][q] * L[j][q];
      L[r][j] = v / d;
    }
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double v = D.b[6 * i + r];
#pragma unroll
    for (int q = 0; q < r; ++q) v -= L[r][q] * y[q];
    y[r] = v / L[r][r];
  }
#pragma unroll
  for (int r = 5; r >= 0; --r) {
    double v = y[r];
#pragma unroll
    for (int q = r + 1; q < 6; ++q) v -= L[q][r] * y[q];
    y[r] = v / L[r][r];
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) D.x[6 * i + r] = y[r];
}

template <typename T>
void launch_block_jacobi(const BatchTabs& B, cudaStream_t s) {
  k_block_jacobi<T><<<B.n_nodes, 128, 0, s>>>(B.d, B.nodes);
  ++g_launches;
}
template void launch_block_jacobi<float>(const BatchTabs&, cudaStream_t);
template void launch_block_jacobi<double>(const BatchTabs&, cudaStream_t);

}  // namespace ds
