// lt_kernels.cu -- CUDA kernels of the light tracer and its adjoints (sm_103a).
//
// One lane carries one light path at a time through its vertices and draws the next path
// of its warp's share when it finishes (one wave of resident blocks).  Every pass
// regenerates the path from its Philox counter; nothing per vertex is stored except by the
// naive baseline and the buffered two-pass form.
#include <cuda_runtime.h>

#include <utility>

#include "lt_device.cuh"
#include "lt_batch.h"
#include "lt_launch.h"
#include "lt_mlp.cuh"

// Compiled once per BVH width (-DLT_BVH_WIDTH=2, 4 or 8) into lt::w2, lt::w4, lt::w8.
#if LT_BVH_WIDTH == 2
#define LT_KNS w2
#elif LT_BVH_WIDTH == 4
#define LT_KNS w4
#elif LT_BVH_WIDTH == 8
#define LT_KNS w8
#else
#error "LT_BVH_WIDTH must be 2, 4 or 8"
#endif

namespace lt {
namespace LT_KNS {

// ======================================================================= refit
// Triangle geometry from base vertex positions plus heights (y), leaf order.  The edges
// take the base edges plus the height differences, not differences of the displaced
// absolute positions: a height field's neighbouring heights differ by far less than the
// FP32 spacing of its absolute coordinates allows to resolve, and the edges set the
// normals that refraction and the height gradients depend on.
__global__ void k_update_tris(float4* prim, const int4* prim_h, const float4* tri_base, const float* heights,
                              int n_prims) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_prims) return;
  int4 ph = prim_h[i];
  if (ph.x < 0 && ph.y < 0 && ph.z < 0) return;
  const float3 b0 = xyz(tri_base[3 * i]), b1 = xyz(tri_base[3 * i + 1]), b2 = xyz(tri_base[3 * i + 2]);
  const float h0 = ph.x >= 0 ? heights[ph.x] : 0.0f, h1 = ph.y >= 0 ? heights[ph.y] : 0.0f,
              h2 = ph.z >= 0 ? heights[ph.z] : 0.0f;
  float3 e1 = b1 - b0, e2 = b2 - b0;
  e1.y += h1 - h0;
  e2.y += h2 - h0;
  float3 v0 = b0;
  v0.y += h0;
  float4 a = prim[3 * i], b = prim[3 * i + 1], c = prim[3 * i + 2];
  prim[3 * i] = make_float4(v0.x, v0.y, v0.z, a.w);
  prim[3 * i + 1] = make_float4(e1.x, e1.y, e1.z, b.w);
  prim[3 * i + 2] = make_float4(e2.x, e2.y, e2.z, c.w);
}

// Bounds of the primitives [r.x, r.y) that this thread visits with the given stride.
__device__ __forceinline__ void range_bounds(const float4* prim, int2 r, int first, int stride, float3& lo, float3& hi) {
  lo = f3(3e38f, 3e38f, 3e38f);
  hi = f3(-3e38f, -3e38f, -3e38f);
  for (int k = r.x + first; k < r.y; k += stride) {
    float3 o = xyz(prim[3 * k]), e1 = xyz(prim[3 * k + 1]), e2 = xyz(prim[3 * k + 2]);
    bool tri = __float_as_int(prim[3 * k + 2].w) != 0;
    float3 p[4] = {o, o + e1, o + e2, o + e1 + e2};
    int np = tri ? 3 : 4;
    for (int j = 0; j < np; ++j) {
      lo = f3(fminf(lo.x, p[j].x), fminf(lo.y, p[j].y), fminf(lo.z, p[j].z));
      hi = f3(fmaxf(hi.x, p[j].x), fmaxf(hi.y, p[j].y), fmaxf(hi.z, p[j].z));
    }
  }
}
__device__ __forceinline__ void warp_bounds(float3& lo, float3& hi) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, off));
    lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, off));
    lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, off));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, off));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, off));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, off));
  }
}
__device__ __forceinline__ void store_node(float4* node, int w, float3 lo, float3 hi) {
  // conservative padding for FP32 rounding of the stored primitive edges
  float3 pad = f3(1e-6f * fmaxf(1.0f, fmaxf(fabsf(lo.x), fabsf(hi.x))),
                  1e-6f * fmaxf(1.0f, fmaxf(fabsf(lo.y), fabsf(hi.y))),
                  1e-6f * fmaxf(1.0f, fmaxf(fabsf(lo.z), fabsf(hi.z))));
  float4 a = node[2 * w], b = node[2 * w + 1];
  node[2 * w] = make_float4(lo.x - pad.x, lo.y - pad.y, lo.z - pad.z, a.w);
  node[2 * w + 1] = make_float4(hi.x + pad.x, hi.y + pad.y, hi.z + pad.z, b.w);
}

// One warp per BVH node: the node's subtree covers the contiguous leaf-order primitive
// range [range.x, range.y), so its bounds are a reduction over that range.  Nodes with more
// than kRefitBig primitives are left to k_refit_big.
__global__ void k_refit_nodes(float4* node, const int2* range, const float4* prim, int n_nodes) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n_nodes) return;
  int2 r = range[w];
  if (r.y - r.x > kRefitBig) return;
  float3 lo, hi;
  range_bounds(prim, r, lane, 32, lo, hi);
  warp_bounds(lo, hi);
  if (lane == 0) store_node(node, w, lo, hi);
}

// One block per node with more than kRefitBig primitives (the top of the tree), so the
// root's reduction over every primitive is not left to a single warp.
__global__ void __launch_bounds__(256) k_refit_big(float4* node, const int2* range, const int* big,
                                                   const float4* prim) {
  __shared__ float sh[6][8];
  const int w = big[blockIdx.x];
  float3 lo, hi;
  range_bounds(prim, range[w], threadIdx.x, blockDim.x, lo, hi);
  warp_bounds(lo, hi);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = lo.x; sh[1][wid] = lo.y; sh[2][wid] = lo.z;
    sh[3][wid] = hi.x; sh[4][wid] = hi.y; sh[5][wid] = hi.z;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      lo = f3(fminf(lo.x, sh[0][i]), fminf(lo.y, sh[1][i]), fminf(lo.z, sh[2][i]));
      hi = f3(fmaxf(hi.x, sh[3][i]), fmaxf(hi.y, sh[4][i]), fmaxf(hi.z, sh[5][i]));
    }
    store_node(node, w, lo, hi);
  }
}

// Wide-node boxes from the refitted binary nodes: one thread per child slot copies the
// box of the binary node that the slot stands for (the wide BVH is a collapse of the
// binary one) into the node's structure-of-arrays layout.
template <int W>
__global__ void k_refit_wide(float4* wnode, const int* wmap, const float4* node, int n_wnodes) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_wnodes * W) return;
  const int j = t / W, c = t - j * W;
  const int b = wmap[t];
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  if (b >= 0) {
    const float4 l = node[2 * b], h = node[2 * b + 1];
    lo[0] = l.x; lo[1] = l.y; lo[2] = l.z;
    hi[0] = h.x; hi[1] = h.y; hi[2] = h.z;
  }
  float* nd = reinterpret_cast<float*>(wnode) + (size_t)j * 8 * W;
  for (int q = 0; q < 3; ++q) {
    nd[q * W + c] = lo[q];
    nd[(q + 3) * W + c] = hi[q];
  }
}

// ======================================================================= path walk
// State of a light path between vertices.
struct Walk {
  float3 org, dir;
  int skip;
  int prev_kind;
  float3 beta;
  bool dead;  // ended by Russian roulette
};

// Emitter sample (uniform point, cosine direction, beta_0 = Le A pi) from counter (n, 0).
__device__ __forceinline__ void walk_start(const DevScene& S, uint64_t seed, uint64_t n, float3 Le, Walk& w,
                                           float3& x0) {
  float4 r = rand4(seed, n, 0);
  x0 = S.lo + S.le1 * r.x + S.le2 * r.y;
  w.org = x0;
  w.dir = cosine_dir(S.ln, r.z, r.w);
  w.skip = S.emitter_prim;
  w.prev_kind = K_EMITTER;
  w.beta = Le * (S.light_area * kPi);
  w.dead = false;
}

// Russian roulette after vertex k (depth k + 1), once the walk has scattered: the path
// continues with probability rr_q, decided by Philox stream 2 at that depth, and its
// throughput is divided by rr_q.  The decision and rr_q do not depend on the parameters,
// so every replay ends the path at the same vertex and the derivative treats 1/rr_q as a
// constant factor.
__device__ __forceinline__ void walk_rr(const KParams& kp, uint64_t n, int k, Walk& w) {
  if (kp.rr_depth <= 0 || k + 1 < kp.rr_depth) return;
  if (rand4(kp.seed, n, (uint32_t)(k + 1), 2).x < kp.rr_q) w.beta = w.beta * (1.0f / kp.rr_q);
  else w.dead = true;
}

// One surface vertex: closest hit and its local frame.
struct Vtx {
  int prim;
  Prim P;
  int4 m;
  float b1, b2;   // surface / texture coordinates
  float3 x, nraw, n;
  bool attached;
  bool diffuse;
};

// Complete a closest-hit record into a vertex; false when the path ends (miss or emitter).
__device__ __forceinline__ bool walk_finish(const DevScene& S, const Walk& w, const HitRec& h, Vtx& v) {
  if (h.prim < 0) return false;
  v.prim = h.prim;
  v.P = load_prim(S, h.prim);
  v.m = __ldg(S.mat + v.P.mat);
  if (v.m.x == MAT_EMITTER) return false;
  v.b1 = h.b1; v.b2 = h.b2;
  v.attached = w.prev_kind != K_SPECULAR;
  v.x = v.attached ? v.P.o + v.P.e1 * h.b1 + v.P.e2 * h.b2 : w.org + w.dir * h.t;
  v.nraw = cross(v.P.e1, v.P.e2);
  v.n = normalize(v.nraw);
  v.diffuse = v.m.x == MAT_DIFFUSE;
  return true;
}

// Per-lane version (divergent callers): trace and complete the next vertex.
template <bool ST = false>
__device__ __forceinline__ bool walk_hit(const DevScene& S, const Walk& w, Vtx& v, Census* cs = nullptr) {
  if (w.dead) return false;
  HitRec h = trace_closest<ST>(S, w.org, w.dir, w.skip, cs);
  if (h.prim < 0) return false;
  v.prim = h.prim;
  v.P = load_prim(S, h.prim);
  v.m = __ldg(S.mat + v.P.mat);
  if (v.m.x == MAT_EMITTER) return false;
  v.b1 = h.b1; v.b2 = h.b2;
  v.attached = w.prev_kind != K_SPECULAR;
  v.x = v.attached ? v.P.o + v.P.e1 * h.b1 + v.P.e2 * h.b2 : w.org + w.dir * h.t;
  v.nraw = cross(v.P.e1, v.P.e2);
  v.n = normalize(v.nraw);
  v.diffuse = v.m.x == MAT_DIFFUSE;
  return true;
}

// Scatter: diffuse cosine sample about the arrival-side normal (weight rho), or the
// Fresnel-chosen dielectric branch (weight 1).  r = uniforms of this vertex.
__device__ __forceinline__ bool walk_scatter(const DevScene& S, Walk& w, const Vtx& v, float3 ns, float3 rho,
                                             float4 r) {
  bool refl = false;
  if (v.diffuse) {
    w.dir = cosine_dir(ns, r.x, r.y);
    w.beta = mul(w.beta, rho);
    w.prev_kind = K_DIFFUSE;
  } else {
    Dielectric D = dielectric(w.dir, v.n, __ldg(S.mat_ior + v.P.mat));
    refl = D.tir || r.z < D.F;
    w.dir = refl ? D.refl : D.refr;
    w.prev_kind = K_SPECULAR;
  }
  w.org = v.x;
  w.skip = v.prim;
  return refl;
}

__device__ __forceinline__ uint32_t vtx_flags(const Vtx& v, bool refl, bool conn) {
  return (uint32_t)(v.diffuse ? K_DIFFUSE : K_SPECULAR) | (refl ? 4u : 0u) | (conn ? 8u : 0u) |
         (v.attached ? 16u : 0u);
}

// ======================================================================= reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Block-reduce a float3 and add it to dst with one atomic per component per block.
__device__ __forceinline__ void block_add3(float* dst, float3 v) {
  __shared__ float sh[3][32];
  v.x = warp_sum(v.x); v.y = warp_sum(v.y); v.z = warp_sum(v.z);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[0][wid] = v.x; sh[1][wid] = v.y; sh[2][wid] = v.z; }
  __syncthreads();
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    float a = lane < nw ? sh[0][lane] : 0.0f, b = lane < nw ? sh[1][lane] : 0.0f, c = lane < nw ? sh[2][lane] : 0.0f;
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    if (lane == 0 && dst) { atomicAdd(dst, a); atomicAdd(dst + 1, b); atomicAdd(dst + 2, c); }
  }
}

// Gradient sink of a block: each parameter array that fits in shared memory (the host
// decides per array) is accumulated there by the block (shared-memory atomics) and added to
// the global array once at the end; the albedo and height arrays are small and every path
// touches them, so global atomics on them contend heavily (a one-texel albedo would send
// every vertex's gradient to the same three addresses).
struct Sink {
  float* alb;
  float* h;
};
__device__ __forceinline__ Sink sink_begin(const KParams& kp, const GradPtrs& g, float* sh) {
  Sink s;
  s.alb = g.d_albedo;
  s.h = g.d_heights;
  if (kp.priv_n > 0) {
    for (int i = threadIdx.x; i < kp.priv_n; i += blockDim.x) sh[i] = 0.0f;
    __syncthreads();
    if (g.d_albedo && kp.n_alb > 0) s.alb = sh;
    if (g.d_heights && kp.n_h > 0) s.h = sh + kp.n_alb;
  }
  return s;
}
__device__ __forceinline__ void sink_end(const KParams& kp, const GradPtrs& g, const float* sh) {
  if (kp.priv_n <= 0) return;
  __syncthreads();
  if (g.d_albedo)
    for (int i = threadIdx.x; i < kp.n_alb; i += blockDim.x) {
      const float v = sh[i];
      if (v != 0.0f) atomicAdd(g.d_albedo + i, v);
    }
  if (g.d_heights)
    for (int i = threadIdx.x; i < kp.n_h; i += blockDim.x) {
      const float v = sh[kp.n_alb + i];
      if (v != 0.0f) atomicAdd(g.d_heights + i, v);
    }
}

// Albedo gradient at one diffuse vertex: weight (per channel) / rho times the bilinear
// texel weights (d rho / d texel).
__device__ __forceinline__ void scatter_albedo(const DevScene& S, float* g, const TexFoot& f, float3 wt, float3 rho) {
  if (!g) return;
  float3 a = f3(wt.x / rho.x, wt.y / rho.y, wt.z / rho.z);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (f.w[k] == 0.0f) continue;
    if (S.atomics) {  // lanes adding to the same texel sum first
      agg_add3(g + f.idx[k], a.x * f.w[k], a.y * f.w[k], a.z * f.w[k]);
      continue;
    }
    red_add(g + f.idx[k] + 0, a.x * f.w[k]);
    red_add(g + f.idx[k] + 1, a.y * f.w[k]);
    red_add(g + f.idx[k] + 2, a.z * f.w[k]);
  }
}

// ------------------------------------------------------------ attached local adjoints
// Attached segment weight (Sec. 3.3 attached samples): g = |n_p.w| |nraw.w| / (|n_p| r^4)
// for w = x - x_p (the G term times the triangle area); adjoint of log g scaled by lam.
__device__ __forceinline__ void seg_adjoint(float3 xp, float3 np, float3 x, float3 nr, float lam, float3& gxp,
                                            float3& gnp, float3& gx, float3& gn) {
  float3 w = x - xp;
  float r2 = dot(w, w);
  float a = dot(np, w), b = dot(nr, w);
  float3 dw = np * (1.0f / a) + nr * (1.0f / b) - w * (4.0f / r2);
  gx = gx + dw * lam;
  gxp = gxp - dw * lam;
  gn = gn + w * (lam / b);
  gnp = gnp + (w * (1.0f / a) - np * (1.0f / dot(np, np))) * lam;
}
// Sensor connection geometry log(|nraw.v| / (|nraw| zc^3)) (v = camera - x) scaled by lam,
// plus the film position channel q . du/dx (Sec. 4.4, Eq. 20-21).
__device__ __forceinline__ void conn_adjoint(const DevScene& S, float3 x, float3 nr, float lam, float2 q,
                                             float3& gx, float3& gn) {
  float3 v = S.cpos - x;
  float3 d = x - S.cpos;
  float nv = dot(nr, v), zc = dot(d, S.cf);
  gx = gx + (nr * (-1.0f / nv) - S.cf * (3.0f / zc)) * lam;
  gn = gn + (v * (1.0f / nv) - nr * (1.0f / dot(nr, nr))) * lam;
  float pr = dot(d, S.cr), pu = dot(d, S.cu);
  float ax = 0.5f * (float)S.W / (S.tanx * zc), ay = -0.5f * (float)S.H / (S.tany * zc);
  gx = gx + (S.cr - S.cf * (pr / zc)) * (q.x * ax) + (S.cu - S.cf * (pu / zc)) * (q.y * ay);
}
// Map the adjoint of an attached point x = v0 + b1 e1 + b2 e2 and of nraw = e1 x e2 on a
// height-field triangle to its three vertex heights (vertex k moves along +y by h_k).
__device__ __forceinline__ void scatter_heights(const DevScene& S, float* dh, int prim, float b1, float b2, float3 gx,
                                                float3 gn) {
  if (!dh || prim < 0) return;
  int4 ph = __ldg(S.prim_h + prim);
  if (ph.x < 0 && ph.y < 0 && ph.z < 0) return;
  float3 e1 = xyz(__ldg(S.prim + 3 * prim + 1)), e2 = xyz(__ldg(S.prim + 3 * prim + 2));
  float a1 = gn.x * e2.z - gn.z * e2.x;
  float a2 = gn.z * e1.x - gn.x * e1.z;
  float h0 = (1.0f - b1 - b2) * gx.y - a1 - a2, h1 = b1 * gx.y + a1, h2 = b2 * gx.y + a2;
  if (S.atomics) {
    // lanes adding to the same height sum first
    if (ph.x >= 0) agg_add1(dh + ph.x, h0);
    if (ph.y >= 0) agg_add1(dh + ph.y, h1);
    if (ph.z >= 0) agg_add1(dh + ph.z, h2);
    return;
  }
  if (ph.x >= 0) red_add(dh + ph.x, h0);
  if (ph.y >= 0) red_add(dh + ph.y, h1);
  if (ph.z >= 0) red_add(dh + ph.z, h2);
}

// ------------------------------------------------------------ specular chains (attached)
// A chain starts at an attached specular vertex a (following the emitter or a diffuse
// vertex, the "anchor") and continues through sliding vertices (re-intersected along the
// reflected/refracted ray with the same primitive) up to a sliding diffuse vertex t.
// Everything a chain needs to be replayed is constant-size: the anchor and the chain
// start's attached coordinates; the branch choices come from the Philox counter.
struct ChainInfo {
  int ka;                // vertex index of the chain's attached specular start
  int prim_a;
  float ba1, ba2;
  float3 xp, np;         // anchor position and (unnormalised) normal
  int prim_p;            // anchor primitive (-1: the emitter)
  float bp1, bp2;
  int kanchor;           // anchor vertex index (-1: the emitter)
  bool anchor_sliding;   // the anchor is itself the sliding end of an earlier chain
  float lam;             // channel-summed adjoint weight of the chain's Fresnel factors
};

// Adjoint of an attached vertex accumulated until all of its terms are known.
struct PendAdj {
  int prim;              // -1: nothing pending (the emitter)
  int k;                 // vertex index
  float b1, b2;
  float3 x, nr, gx, gn;
  bool sliding;          // reached through a specular chain (then `chain` is valid)
  ChainInfo chain;
};

__device__ __forceinline__ void pend_init(PendAdj& p, int prim, int k, float b1, float b2, float3 x, float3 nr) {
  p.prim = prim; p.k = k; p.b1 = b1; p.b2 = b2; p.x = x; p.nr = nr;
  p.gx = p.gn = f3(0, 0, 0);
  p.sliding = false;
}

// Chain whose attached specular start is vertex k, anchored at the pending vertex `an`.
__device__ __forceinline__ ChainInfo chain_at(const PendAdj& an, int k, const Vtx& v, float lam) {
  ChainInfo c;
  c.ka = k; c.prim_a = v.prim; c.ba1 = v.b1; c.ba2 = v.b2;
  c.xp = an.x; c.np = an.nr; c.prim_p = an.prim; c.bp1 = an.b1; c.bp2 = an.b2;
  c.kanchor = an.prim < 0 ? -1 : an.k;
  c.anchor_sliding = an.prim >= 0 && an.sliding;
  c.lam = lam;
  return c;
}

// State of chain vertex j when replayed from the chain start.
struct ChainState {
  int prim;
  float3 x, din, nraw;
  Dielectric D;
  bool refl;
};

// Vertex states of the chains the forward walk has just passed through, so that a chain's
// reverse sweep reads them instead of replaying the chain (its traces run on the few lanes
// that finish a chain at that step).  Two records, the current chain and the one before
// (a position adjoint continues into it when the current chain's anchor ends it), of at
// most kChainCache vertices each; a longer or older chain is replayed as before.  The
// states are the ones the replay would compute, from the same arithmetic.
constexpr int kChainCache = 4;
constexpr int kDraws = 4;  // path draws per lane and step of the LRB-3 loop
constexpr int kFlushBatch = 16;  // waiting lanes of a warp that sweep their chains together (swept 8-24)
struct ChainRec {
  ChainInfo info;
  int len;  // recorded specular vertices info.ka .. info.ka+len-1; -1: not usable
  int prim[kChainCache];
  float3 x[kChainCache], din[kChainCache];
  unsigned refl;  // bit i: vertex info.ka+i took the reflected branch
};
struct ChainCache {
  ChainRec r[2];
  int cur;
  __device__ __forceinline__ void reset() {
    r[0].len = r[1].len = -1;
    cur = 0;
  }
  // Specular vertex k reached along din (before scattering); an attached one starts `chain`.
  __device__ __forceinline__ void record(const ChainInfo& chain, int k, const Vtx& v, float3 din) {
    if (v.attached) {
      cur ^= 1;
      r[cur].info = chain;
      r[cur].len = 0;
      r[cur].refl = 0u;
    }
    ChainRec& c = r[cur];
    if (c.len < 0) return;
    if (c.len >= kChainCache || c.info.ka + c.len != k) {
      c.len = -1;
      return;
    }
    c.prim[c.len] = v.prim;
    c.x[c.len] = v.x;
    c.din[c.len] = din;
  }
  // Its branch, once the walk has scattered.
  __device__ __forceinline__ void record_branch(bool refl) {
    ChainRec& c = r[cur];
    if (c.len < 0 || c.len >= kChainCache) return;
    c.refl |= (refl ? 1u : 0u) << c.len;
    ++c.len;
  }
};

// Replay the chain from its start to vertex j (a <= j) and trace the ray leaving j.  The
// chain's first direction is the one the walk sampled at the anchor (the emitter's
// cosine sample, or the diffuse anchor's, on the side of its normal that faces the chain
// start), recomputed from the same Philox numbers, so the replay repeats the walk's
// arithmetic exactly; normalize(x_a - x_p) differs from it in the last bits, which can
// send a grazing ray to another triangle.
__device__ __forceinline__ bool chain_replay(const DevScene& S, const KParams& kp, uint64_t n, const ChainInfo& c,
                                             int j, ChainState& st, HitRec& next) {
  Prim Pa = load_prim(S, c.prim_a);
  float3 x = Pa.o + Pa.e1 * c.ba1 + Pa.e2 * c.ba2;
  float3 din;
  if (c.kanchor < 0) {
    const float4 r0 = rand4(kp.seed, n, 0);
    din = cosine_dir(S.ln, r0.z, r0.w);
  } else {
    const Prim Pp = load_prim(S, c.prim_p);
    const float3 np = normalize(cross(Pp.e1, Pp.e2));
    const float4 r = rand4(kp.seed, n, (uint32_t)(c.kanchor + 1));
    din = cosine_dir(dot(x - c.xp, np) >= 0.0f ? np : -np, r.x, r.y);
  }
  int prim = c.prim_a;
  for (int k = c.ka;; ++k) {
    Prim P = load_prim(S, prim);
    float3 nraw = cross(P.e1, P.e2);
    Dielectric D = dielectric(din, normalize(nraw), __ldg(S.mat_ior + P.mat));
    float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
    bool refl = D.tir || r.z < D.F;
    float3 dout = refl ? D.refl : D.refr;
    HitRec h = trace_closest(S, x, dout, prim);
    if (k == j) {
      st.prim = prim; st.x = x; st.din = din; st.nraw = nraw; st.D = D; st.refl = refl;
      next = h;
      return h.prim >= 0;
    }
    if (h.prim < 0) return false;
    x = x + dout * h.t;
    din = dout;
    prim = h.prim;
  }
}

// d log F / d cos_i of the unpolarised Fresnel reflectance (Fresnel equations).
__device__ __forceinline__ float fresnel_dF(const Dielectric& D) {
  float eta = D.eta, ci = D.ci, ct = D.ct;
  float dct = eta * eta * ci / ct;
  float us = eta * ci - ct, ws = eta * ci + ct;
  float up = ci - eta * ct, wp = ci + eta * ct;
  float rs = us / ws, rp = up / wp;
  float drs = ((eta - dct) * ws - us * (eta + dct)) / (ws * ws);
  float drp = ((1.0f - eta * dct) * wp - up * (1.0f + eta * dct)) / (wp * wp);
  return rs * drs + rp * drp;
}

// Reverse of d_out = reflect/refract(d_in, n) and of the branch weight F/F0 or
// (1-F)/(1-F0) with log-derivative weight lam.  Returns the adjoints of d_in and nraw.
__device__ __forceinline__ void spec_adjoint(const ChainState& s, float3 gdout, float lam, float3& gdin,
                                             float3& gnraw) {
  const Dielectric& D = s.D;
  float3 ns = D.ns;
  float3 gns;
  float gci;
  if (s.refl) {
    gdin = gdout;
    gns = gdout * (2.0f * D.ci);
    gci = 2.0f * dot(gdout, ns);
    if (!D.tir) gci += lam * fresnel_dF(D) / D.F;
  } else {
    gdin = gdout * D.eta;
    float K = D.eta * D.ci - D.ct;
    gns = gdout * K;
    float gK = dot(gdout, ns);
    float dct = D.eta * D.eta * D.ci / D.ct;
    gci = gK * (D.eta - dct);
    gci += lam * (-fresnel_dF(D)) / (1.0f - D.F);
  }
  gdin = gdin - ns * gci;
  gns = gns - s.din * gci;
  float3 gn = D.entering ? gns : -gns;
  float inv = 1.0f / length(s.nraw);
  float3 nn = s.nraw * inv;
  gnraw = (gn - nn * dot(nn, gn)) * inv;
}


// Reverse-mode sweep back through a chain ending at sliding vertex kt whose position
// adjoint is gx_t: vertex states come from the forward walk's chain cache when it holds the
// chain, else they are replayed from the chain start (constant memory, c(c+1)/2 traces for
// c specular vertices).  Scatters into the height gradient the contributions of every
// primitive the chain touches and returns the adjoint of the anchor position (through the
// chain start's incoming direction).
__device__ __forceinline__ float3 chain_reverse(const DevScene& S, const KParams& kp, uint64_t n, const ChainInfo& c,
                                             int kt, float3 gx_t, float* dh, const ChainCache* cc, int prim_t) {
  const ChainRec* rec = nullptr;
  if (cc)
    for (int b = 0; b < 2; ++b)
      if (cc->r[b].len > 0 && cc->r[b].info.ka == c.ka && cc->r[b].info.ka + cc->r[b].len == kt) rec = &cc->r[b];
  float3 gx = gx_t, gd = f3(0, 0, 0);
  for (int j = kt - 1; j >= c.ka; --j) {
    ChainState s;
    int hprim;
    if (rec) {
      const int i = j - c.ka;
      s.prim = rec->prim[i];
      s.x = rec->x[i];
      s.din = rec->din[i];
      const Prim P = load_prim(S, s.prim);
      s.nraw = cross(P.e1, P.e2);
      s.D = dielectric(s.din, normalize(s.nraw), __ldg(S.mat_ior + P.mat));
      s.refl = (rec->refl >> i) & 1u;
      hprim = j + 1 < kt ? rec->prim[i + 1] : prim_t;
    } else {
      HitRec h;
      if (!chain_replay(S, kp, n, c, j, s, h)) { set_err(S, ERR_BOUNDS); return f3(0, 0, 0); }
      hprim = h.prim;
    }
    Prim Q = load_prim(S, hprim);
    float3 m = cross(Q.e1, Q.e2);
    float3 dout = s.refl ? s.D.refl : s.D.refr;
    // x_{j+1} = x_j + tau d_out, tau = ((o' - x_j).m) / (d_out.m)
    float a = dot(Q.o - s.x, m), b = dot(dout, m);
    float tau = a / b;
    float gtau = dot(gx, dout);
    float3 gdout = gd + gx * tau;
    float ga = gtau / b, gb = -gtau * tau / b;
    float3 gxj = gx - m * ga;
    float3 go = m * ga;
    float3 gm = (Q.o - s.x) * ga + dout * gb;
    gdout = gdout + m * gb;
    scatter_heights(S, dh, hprim, 0.0f, 0.0f, go, gm);  // plane of the next primitive
    float3 gdin, gnraw;
    spec_adjoint(s, gdout, c.lam, gdin, gnraw);
    if (j > c.ka) {
      scatter_heights(S, dh, s.prim, 0.0f, 0.0f, f3(0, 0, 0), gnraw);  // sliding vertex: its normal only
      gd = gdin;
      gx = gxj;
    } else {
      // chain start: d_in = normalize(x_a - x_p), x_a attached to its primitive
      float3 w = s.x - c.xp;
      float r = length(w);
      float3 gw = (gdin - s.din * dot(s.din, gdin)) * (1.0f / r);
      scatter_heights(S, dh, c.prim_a, c.ba1, c.ba2, gxj + gw, gnraw);
      return -gw;
    }
  }
  return f3(0, 0, 0);
}

// Geometry-only replay of the path from the emitter up to vertex `target`; returns the
// chain that vertex ends (valid when it is a sliding diffuse vertex).  Used to recover
// an earlier chain when a position adjoint has to continue through it.
__device__ __noinline__ bool replay_chain_of(const DevScene& S, const KParams& kp, uint64_t n, int target,
                                            ChainInfo& out) {
  Walk w;
  float3 x0;
  walk_start(S, kp.seed, n, f3(1, 1, 1), w, x0);
  PendAdj an;
  pend_init(an, -1, -1, 0.0f, 0.0f, x0, S.ln);
  ChainInfo ch;
  ch.ka = -1;
  for (int k = 0; k <= target; ++k) {
    Vtx v;
    if (!walk_hit(S, w, v)) return false;
    if (v.attached && !v.diffuse) ch = chain_at(an, k, v, 0.0f);
    if (k == target) {
      out = ch;
      return !v.attached && v.diffuse && ch.ka >= 0;
    }
    float3 ns = f3(0, 0, 0);
    if (v.diffuse) {
      ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
      bool sl = !v.attached;
      pend_init(an, v.prim, k, v.b1, v.b2, v.x, v.nraw);
      an.sliding = sl;
    }
    walk_scatter(S, w, v, ns, f3(1, 1, 1), rand4(kp.seed, n, (uint32_t)(k + 1)));
  }
  return false;
}

// Propagate a position adjoint on the sliding end kt of chain c back to the parameters,
// continuing through earlier chains while the anchor is itself sliding (those chains'
// Fresnel factors were already counted, so they are re-traversed with zero weight).
__device__ __forceinline__ void propagate_sliding(const DevScene& S, const KParams& kp, uint64_t n, ChainInfo c, int kt,
                                               float3 gx, float* dh, const ChainCache* cc, int prim_t) {
  for (int guard = 0; guard < kMaxDepth; ++guard) {
    float3 g_anchor = chain_reverse(S, kp, n, c, kt, gx, dh, cc, prim_t);
    if (c.kanchor < 0) return;  // the emitter does not move
    if (!c.anchor_sliding) {
      scatter_heights(S, dh, c.prim_p, c.bp1, c.bp2, g_anchor, f3(0, 0, 0));
      return;
    }
    ChainInfo prev;
    bool found = false;
    if (cc)
      for (int b = 0; b < 2; ++b)
        if (cc->r[b].len > 0 && cc->r[b].info.ka < c.ka && cc->r[b].info.ka + cc->r[b].len == c.kanchor) {
          prev = cc->r[b].info;
          prev.lam = 0.0f;  // geometry only, as in the replay: its Fresnel factors are counted
          found = true;
        }
    if (!found && !replay_chain_of(S, kp, n, c.kanchor, prev)) { set_err(S, ERR_BOUNDS); return; }
    prim_t = c.prim_p;
    kt = c.kanchor;
    gx = g_anchor;
    c = prev;
  }
}

// Texture-coordinate derivative of a sliding diffuse vertex: (s,t) of x on its
// (non-moving) primitive, bilinear rho(s,t); weight wt/rho per channel.
__device__ __forceinline__ float3 tex_pos_adjoint(const float* albedo, int4 m, const Prim& P, float s, float t,
                                                  float3 wt, float3 rho) {
  int tw = m.z, th = m.w, off = m.y;
  if (tw * th <= 1) return f3(0, 0, 0);
  float tx = s * (float)tw - 0.5f, ty = t * (float)th - 0.5f;
  float fx0 = floorf(tx), fy0 = floorf(ty);
  float fx = tx - fx0, fy = ty - fy0;
  int x0 = (int)fx0, y0 = (int)fy0;
  int xa = min(max(x0, 0), tw - 1), xb = min(max(x0 + 1, 0), tw - 1);
  int ya = min(max(y0, 0), th - 1), yb = min(max(y0 + 1, 0), th - 1);
  float3 T00 = texel(albedo, off + (ya * tw + xa) * 3), T10 = texel(albedo, off + (ya * tw + xb) * 3);
  float3 T01 = texel(albedo, off + (yb * tw + xa) * 3), T11 = texel(albedo, off + (yb * tw + xb) * 3);
  float3 ds = ((T10 - T00) * (1.0f - fy) + (T11 - T01) * fy) * (float)tw;
  float3 dt = ((T01 - T00) * (1.0f - fx) + (T11 - T10) * fx) * (float)th;
  float3 a = f3(wt.x / rho.x, wt.y / rho.y, wt.z / rho.z);
  float gs = dot(a, ds), gt = dot(a, dt);
  float3 mm = cross(P.e1, P.e2);
  float inv = 1.0f / dot(mm, mm);
  return (cross(P.e2, mm) * gs + cross(mm, P.e1) * gt) * inv;
}

// Flush a vertex's completed adjoint: attached vertices map through their surface
// coordinates, sliding ones run the chain's reverse sweep (their normal is explicit).
template <bool CH>
__device__ __forceinline__ void pend_flush(const DevScene& S, const KParams& kp, uint64_t n, const PendAdj& p,
                                           float* dh, const ChainCache* cc) {
  if (!dh || p.prim < 0) return;
  if (!CH || !p.sliding) {
    scatter_heights(S, dh, p.prim, p.b1, p.b2, p.gx, p.gn);
  } else {
    scatter_heights(S, dh, p.prim, 0.0f, 0.0f, f3(0, 0, 0), p.gn);
    propagate_sliding(S, kp, n, p.chain, p.k, p.gx, dh, cc, p.prim);
  }
}

// Attached bookkeeping on arrival at vertex k, before its own terms: the attached segment
// weight with the anchor (weight lam_seg) completes the anchor's adjoint; an attached
// specular vertex starts a chain (its Fresnel factors weigh lam_chain); a non-specular
// vertex becomes the new pending anchor (sliding when it ends a chain).
// CH = false compiles the variant for scenes without dielectrics (no chains exist).
template <bool CH>
__device__ __forceinline__ void att_enter(const DevScene& S, const KParams& kp, uint64_t n, int k, const Vtx& v,
                                          float lam_seg, float lam_chain, PendAdj& pv, ChainInfo& chain,
                                          float* dh, const ChainCache* cc) {
  if (!CH || v.attached) {
    PendAdj cur;
    pend_init(cur, v.prim, k, v.b1, v.b2, v.x, v.nraw);
    seg_adjoint(pv.x, pv.nr, v.x, v.nraw, lam_seg, pv.gx, pv.gn, cur.gx, cur.gn);
    pend_flush<CH>(S, kp, n, pv, dh, cc);
    if (CH && !v.diffuse) {
      chain = chain_at(pv, k, v, lam_chain);
      scatter_heights(S, dh, v.prim, v.b1, v.b2, cur.gx, cur.gn);
      pv.prim = -1;
    } else {
      pv = cur;
    }
  } else if (v.diffuse) {
    pend_init(pv, v.prim, k, v.b1, v.b2, v.x, v.nraw);
    pv.sliding = true;
    pv.chain = chain;
  }
}

// ======================================================================= learned target
// Features of a sensor connection for the learned reservoir target: position, arrival-side
// normal, arrival direction, log throughput, relative depth, film position, log
// connection weight (16 values; standardized inside the network).
__device__ __forceinline__ void conn_features(const DevScene& S, float3 x, float3 ns, float3 din, float3 beta, int k,
                                              int D, const Conn& c, float inv_n, float f[16]) {
  f[0] = x.x; f[1] = x.y; f[2] = x.z;
  f[3] = ns.x; f[4] = ns.y; f[5] = ns.z;
  f[6] = din.x; f[7] = din.y; f[8] = din.z;
  f[9] = logf(beta.x + 1e-30f); f[10] = logf(beta.y + 1e-30f); f[11] = logf(beta.z + 1e-30f);
  f[12] = (float)(k + 1) / (float)D;
  f[13] = c.ux / (float)S.W; f[14] = c.uy / (float)S.H;
  f[15] = logf(c.geo * inv_n + 1e-30f);
}

// Training pairs from LRB-3 pass 2: for every valid connection its features and the target
// log(|Lbar_i * L_i|_1 / lum(L_i) + floor), i.e. the adjoint weight the connection sees per
// unit of its luminance.
__global__ void __launch_bounds__(128) k_collect(DevScene S, KParams kp, const float* __restrict__ dI, float tfloor,
                                                 float* __restrict__ feats, float* __restrict__ targets, int64_t cap,
                                                 unsigned long long* __restrict__ count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    if (kp.mask && !kp.mask[p]) continue;
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    Walk w;
    float3 x0;
    walk_start(S, kp.seed, n, Le, w, x0);
    for (int k = 0; k < kp.max_depth; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) break;
      float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        Conn c = connect(S, v.x, ns, v.prim);
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr);
        if (c.valid) {
          float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
          float3 Lb = adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, nullptr, kp.filter);
          float3 P = mul(Lb, L);
          float lum = luminance(L);
          if (lum > 0.0f) {
            unsigned long long slot = atomicAdd(count, 1ull);
            if ((int64_t)slot < cap) {
              float f[16];
              conn_features(S, v.x, ns, w.dir, w.beta, k, kp.max_depth, c, kp.inv_n, f);
              for (int i = 0; i < 16; ++i) feats[slot * 16 + i] = f[i];
              targets[slot] = logf((fabsf(P.x) + fabsf(P.y) + fabsf(P.z)) / lum + tfloor);
            }
          }
        }
      }
      walk_scatter(S, w, v, ns, rho, r);
      walk_rr(kp, n, k, w);
    }
  }
}

// ======================================================================= lane regeneration
// Each warp owns a contiguous range of path indices and hands the next one to every lane
// that has finished its path, so lanes never idle while a slower lane finishes (all 32
// lanes call take() together at the top of the step loop).
struct Dispenser {
  int64_t next, end;
  int64_t stride = 0;                    // dynamic mode: the range's end
  unsigned long long* ticket = nullptr;  // dynamic mode: shared counter of entries taken
  bool exhausted = false;
  __device__ __forceinline__ void init(int64_t n_paths) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t per = (n_paths + warps - 1) / warps;
    next = min(wid * per, n_paths);
    end = min(next + per, n_paths);
  }
  // Dynamic: a warp takes 32 consecutive entries at a time from a counter shared by the
  // grid (one atomic per 32 entries), so that the warps end together whatever work their
  // entries hold (no warp waits at the block's final barrier for a slower one).
  __device__ __forceinline__ void init_dynamic(int64_t n_paths, unsigned long long* t) {
    next = end = 0;
    stride = n_paths;  // the range's end
    ticket = t;
  }
  // The block alone works on [0, n_paths): contiguous ranges of its warps.
  __device__ __forceinline__ void init_local(int64_t n_paths) {
    const int64_t warps = blockDim.x >> 5;
    const int64_t wid = threadIdx.x >> 5;
    const int64_t per = (n_paths + warps - 1) / warps;
    next = min(wid * per, n_paths);
    end = min(next + per, n_paths);
  }
  // Lanes with `want` receive a path index, or -1 when the warp's range is exhausted.
  __device__ __forceinline__ int64_t take(bool want) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    const unsigned lane = threadIdx.x & 31;
    int64_t mine = -1;
    if (ticket) {
      // serve the wanting lanes from the current 32-entry chunk [next, end), taking the next
      // chunk when it is used up; every round serves a lane or takes a chunk, so it ends
      unsigned rest = m;
      while (rest != 0u && !exhausted) {
        if (next >= end) {
          unsigned long long t = 0;
          if (lane == 0) t = atomicAdd(ticket, 32ull);
          t = __shfl_sync(0xffffffffu, t, 0);
          if ((int64_t)t >= stride) {
            exhausted = true;
            break;
          }
          next = (int64_t)t;
          end = min(next + 32, stride);
        }
        const bool in = (rest >> lane) & 1u;
        const int rank = __popc(rest & ((1u << lane) - 1u));
        const int avail = (int)(end - next);
        const int k = __popc(rest) < avail ? __popc(rest) : avail;
        if (in && rank < k) mine = next + rank;
        next += k;
        rest = __ballot_sync(0xffffffffu, in && rank >= k);
      }
      return mine;
    }
    if (want) {
      int64_t cand = next + __popc(m & ((1u << lane) - 1u));
      mine = cand < end ? cand : -1;
    }
    next += __popc(m);
    return mine;
  }
};

// Batched launches: a warp serves its lanes from its current chunk and takes the next
// chunk (one atomic on the ticket) when that is used up, so lanes of one warp may hold
// paths of different items for a while.  All 32 lanes call take() together; every
// iteration of its loop serves at least one lane or consumes a ticket, so it ends.
struct BatchDispenser {
  int job;
  int64_t next, end;
  bool done;
  __device__ __forceinline__ void init() {
    job = 0;
    next = end = 0;
    done = false;
  }
  // Lanes with `want` receive a path index of item `my_job`, or -1 once the queue is empty.
  __device__ __forceinline__ int64_t take(const BatchArgs& a, bool want, int& my_job) {
    const unsigned lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(0xffffffffu, want);
    int64_t mine = -1;
    while (m != 0u && !done) {
      if (next >= end) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((int64_t)t >= a.n_chunks) {
          done = true;
          break;
        }
        const int64_t c = a.chunk_base + (int64_t)t;
        int lo = 0, hi = a.n_jobs - 1;  // the last item whose first chunk is <= c
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.jobs[mid].chunk0 <= c) lo = mid; else hi = mid - 1;
        }
        job = lo;
        next = (c - a.jobs[lo].chunk0) * a.chunk;
        end = min(next + (int64_t)a.chunk, a.jobs[lo].kp.n_paths);
      }
      const bool in = (m >> lane) & 1u;
      const int rank = __popc(m & ((1u << lane) - 1u));
      const int64_t avail = end - next;
      const int n = (int64_t)__popc(m) < avail ? __popc(m) : (int)avail;
      if (in && rank < n) {
        mine = next + rank;
        my_job = job;
      }
      next += n;
      m = __ballot_sync(0xffffffffu, in && rank >= n);
    }
    return mine;
  }
};

__device__ __forceinline__ void add3(float* d, float3 v) {
  if (!d || (v.x == 0.0f && v.y == 0.0f && v.z == 0.0f)) return;
  atomicAdd(d, v.x);
  atomicAdd(d + 1, v.y);
  atomicAdd(d + 2, v.z);
}

// ======================================================================= primal
// One lane per path with lane regeneration (see Dispenser): each iteration of the step
// loop performs one vertex of the lane's current path.
// BATCH: the lane's scene, parameters and outputs are those of the batch item its path
// belongs to (BatchDispenser); S0, kp0, image0 and aux0 are not used.
// LEARN compiles the learned reservoir target (ResLRB only); plain ResLRB does not carry its
// registers.  ST compiles the work census (rays, box and primitive tests, vertices,
// connections) of a counting variant.  AGG compiles warp-aggregated splat atomics.
template <int EST, bool BATCH, bool LEARN = false, bool ST = false, bool AGG = false>
__device__ __forceinline__ void primal_body(const DevScene& S0, const KParams& kp0, float* __restrict__ image0,
                                            void* aux0, const BatchArgs& ba) {
  // learned reservoir target: network image, one 32x16 feature tile per warp, and two
  // feature slots per lane (see below)
  extern __shared__ __align__(16) unsigned char psmem[];
  MlpSmem& mlp = *reinterpret_cast<MlpSmem*>(psmem);
  const size_t tile_at = (sizeof(MlpSmem) + 15) & ~size_t(15);
  __nv_bfloat16* ftile = reinterpret_cast<__nv_bfloat16*>(psmem + tile_at) + (threadIdx.x >> 5) * 32 * kMlpIn;
  // feature i of slot q of this lane at fstash[(q * kMlpIn + i) * blockDim.x] (no bank conflicts)
  float* fstash = reinterpret_cast<float*>(psmem + tile_at + sizeof(__nv_bfloat16) * 32 * kMlpIn * (blockDim.x >> 5)) +
                  threadIdx.x;
  const bool learned = LEARN && !BATCH && EST == 1 && kp0.mlp != nullptr;
  if (learned) {
    mlp_load_smem(mlp, kp0.mlp);
    __syncthreads();
  }
  float3 Le = BATCH ? f3(0, 0, 0) : f3(kp0.Le[0], kp0.Le[1], kp0.Le[2]);
  Dispenser disp;
  BatchDispenser bdisp;
  // the plain estimator given the LRB-3 state takes 32-path chunks from a counter shared by
  // the grid (no warp waits for a slower one at the end); the others split the range statically
  if (BATCH) bdisp.init();
  else if (EST == 0 && kp0.ticket) disp.init_dynamic(kp0.n_paths, kp0.ticket);
  else disp.init(kp0.n_paths);
  int jb = 0;
  bool busy = false, more = true, active = false;
  int64_t p = 0;
  int k = 0, nconn = 0;
  uint32_t hash = 0;
  uint64_t vmask = 0;  // connection-validity bits (for kp.vstate)
  Walk w;
  // reservoir (capacity one)
  float Om = 0.0f, wR = 0.0f, Rux = 0.0f, Ruy = 0.0f;
  float3 LR = f3(0, 0, 0);
  int R = -1;
  int ncand = 0;       // candidates so far (learned target)
  float lum1 = 0.0f;   // luminance of the first one
  TravState ts;  // the lane's ray in flight (see TravState)
  LocalStack stk;
  bool inflight = false;
  Census cs = {0, 0, 0};
  uint32_t nverts = 0, nconns = 0;
  while (true) {
    const bool want = more && !busy;
    int jnew = jb;
    const int64_t got = BATCH ? bdisp.take(ba, want, jnew) : disp.take(want);
    if (BATCH) jb = jnew;
    const DevScene& S = BATCH ? ba.jobs[jb].S : S0;
    const KParams& kp = BATCH ? ba.jobs[jb].kp : kp0;
    float* image = BATCH ? ba.jobs[jb].image : image0;
    void* aux = BATCH ? ba.jobs[jb].rec : aux0;
    if (want) {
      if (got < 0) {
        more = false;
      } else {
        p = (!BATCH && kp0.order) ? (int64_t)kp0.order[got] : got;
        if (BATCH) Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
        active = !kp.mask || kp.mask[p];
        float3 x0;
        walk_start(S, kp.seed, (uint64_t)(kp.path_offset + p), Le, w, x0);
        hash = 2166136261u;
        vmask = 0;
        nconn = 0;
        k = 0;
        Om = wR = Rux = Ruy = 0.0f;
        LR = f3(0, 0, 0);
        R = -1;
        ncand = 0;
        busy = true;
      }
    }
    if (!__any_sync(0xffffffffu, busy || more)) break;
    const bool trav = busy && k < kp.max_depth && !w.dead;
    HitRec h;
    h.prim = -1;
    bool pending = false;  // the ray has visits left: the lane resumes it in the next step
    if (trav) {
      if (!inflight) trace_begin<ST>(S, w.org, w.dir, w.skip, ts, &cs);
      inflight = !trace_resume<ST>(S, w.org, w.dir, w.skip, ts, stk, &cs);
      pending = inflight;
      h = ts.h;
    }
    Vtx v;
    const bool alive = trav && !pending && walk_finish(S, w, h, v);
    if (EST == 0 && !BATCH && kp0.list) {
      // a path that ends now with a valid connection joins the list that LRB-3 passes 2
      // and 3 visit (one atomic per warp and step)
      const bool ends = busy && !pending && !alive && active && vmask != 0ull;
      const unsigned b = __ballot_sync(0xffffffffu, ends);
      if (b) {
        const int lane = threadIdx.x & 31, leader = __ffs(b) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(kp0.list_n, (unsigned long long)__popc(b));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (ends) kp0.list[base + __popc(b & ((1u << lane) - 1u))] = (uint32_t)p;
      }
    }
    float3 ns = f3(0, 0, 0);
    Conn c;
    c.valid = false; c.ux = c.uy = 0.0f;
    if (alive && v.diffuse) {
      ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
      c = connect_pre(S, v.x, ns);
    }
    if (c.valid && occluded<ST>(S, v.x, c.wc, c.dist, v.prim, &cs)) c.valid = false;
    // Learned reservoir target: warp-wide tensor-core evaluations (all 32 lanes take part).
    // The first candidate of a path is kept whatever its weight (acceptance probability
    // w_1 / Omega = 1), so its weight is only needed once a second candidate arrives: its
    // features wait in shared memory and both are evaluated then.  A path with one
    // candidate (most caustic paths) costs no evaluation; the weights, and so every
    // decision and record, are the same as with eager evaluation.  The rows a step needs are
    // packed into one tile, so a step costs one evaluation of up to 32 rows, and one m16
    // tile when 16 rows or fewer are needed.
    float yhat = 0.0f, yfirst = 0.0f;
    if (learned) {
      bool cand = busy && alive && c.valid && active;
      float f[16];
      if (cand) {
        const float3 Lc = mul(w.beta, tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr)) * (c.geo * kp.inv_n);
        cand = luminance(Lc) > 0.0f;  // a zero-weight connection is no candidate
      }
      if (cand) {
        // slot 0 keeps the first candidate's features, slot 1 takes this step's
        conn_features(S, v.x, ns, w.dir, w.beta, k, kp.max_depth, c, kp.inv_n, f);
        float* dst = fstash + (ncand == 0 ? 0 : kMlpIn * blockDim.x);
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[i * blockDim.x] = f[i];
      }
      // the evaluations the warp needs at this step, packed into consecutive tile rows:
      // this step's candidates first, then the stashed first candidates
      const bool need = cand && ncand >= 1, need1 = cand && ncand == 1;
      const unsigned b0 = __ballot_sync(0xffffffffu, need), b1 = __ballot_sync(0xffffffffu, need1);
      const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
      const int n0 = __popc(b0), total = n0 + __popc(b1);
      const int r0 = __popc(b0 & below), r1 = n0 + __popc(b1 & below);
      for (int base = 0; base < total; base += 32) {
        const bool s0 = need && r0 >= base && r0 < base + 32, s1 = need1 && r1 >= base && r1 < base + 32;
        if (s0) mlp_stage_row(mlp, fstash + kMlpIn * blockDim.x, blockDim.x, ftile, r0 - base);
        if (s1) mlp_stage_row(mlp, fstash, blockDim.x, ftile, r1 - base);
        __syncwarp();
        const float out = mlp_warp_infer_rows(mlp, ftile, min(32, total - base));
        const float o0 = __shfl_sync(0xffffffffu, out, (r0 - base) & 31);
        const float o1 = __shfl_sync(0xffffffffu, out, (r1 - base) & 31);
        if (s0) yhat = o0;
        if (s1) yfirst = o1;
        __syncwarp();
      }
    }
    if (!busy || pending) continue;
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    if (!alive) {
      // end of the path: reservoir record / tape length / per-path outputs
      if (EST == 1) {
        float4* rec = (float4*)aux + 2 * p;
        float wgt = R >= 0 ? Om / wR : 0.0f;
        float3 Sh = LR * wgt;
        if (active && R >= 0) splat_f(image, S.W, S.H, Rux, Ruy, Sh, kp.filter);
        rec[0] = make_float4(__int_as_float(active ? R : -1), wgt, Rux, Ruy);
        rec[1] = make_float4(Sh.x, Sh.y, Sh.z, 0.0f);
      }
      if (EST == 0 && kp.vstate) {
        // the validity mask for LRB-3 pass 2 (bits 0-31 in the w of the float4 record,
        // bits 32-63 in the uint32 array); the rgb part is pass 2's to write
        float4* xrec = (float4*)kp.vstate;
        uint32_t* xhi = (uint32_t*)((char*)kp.vstate + lrb3_state_split(kp.n_paths));
        reinterpret_cast<float*>(xrec + p)[3] = __uint_as_float((uint32_t)(active ? vmask : 0ull));
        xhi[p] = (uint32_t)((active ? vmask : 0ull) >> 32);
      }
      if (EST == 2) ((int*)aux)[p] = active ? k : 0;
      if (EST == 3) ((int*)((char*)aux + lrb2_layout(kp.n_paths, kp.max_depth).counts))[p] = active ? k : 0;
      if (kp.hash) kp.hash[p] = hash;
      if (kp.dbg) ((float4*)kp.dbg)[p] = make_float4((float)nconn, (float)k, 0.0f, 0.0f);
      busy = false;
      continue;
    }
    float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
    float3 rho = f3(0, 0, 0);
    float3 L = f3(0, 0, 0);
    if (ST) ++nverts;
    if (v.diffuse) {
      rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr);
      if (c.valid) {
        if (ST) ++nconns;
        ++nconn;
        L = mul(w.beta, rho) * (c.geo * kp.inv_n);
        if (EST == 0 && !BATCH && kp.conn1 && vmask == 0ull) {
          // the path's first valid connection: LRB-3 pass 2 takes delta_total from this
          // record when it stays the only one
          kp.conn1[p] = make_float4(c.ux, c.uy, L.x, L.y);
          kp.conn1z[p] = L.z;
        }
        vmask |= 1ull << k;
        if (active) {
          if (EST == 1) {
            float om = luminance(L);
            // learned target: lum(L) (exp(sigma * yhat) + eps); any positive weight keeps the
            // estimator unbiased (Eq. 10)
            if (learned && om > 0.0f) {
              if (ncand == 0) {
                // first candidate: accepted; Om / wR = 1 until a second one arrives
                lum1 = om;
                Om = wR = 1.0f;
                R = k; LR = L; Rux = c.ux; Ruy = c.uy;
                om = 0.0f;
              } else if (ncand == 1) {
                Om = wR = lum1 * (__expf(fminf(fmaxf(mlp.tscale * yfirst, -30.0f), 30.0f)) + 1e-3f);
              }
              ++ncand;
              if (om > 0.0f) om *= __expf(fminf(fmaxf(mlp.tscale * yhat, -30.0f), 30.0f)) + 1e-3f;
            }
            if (om > 0.0f) {
              Om += om;
              if (r.w < om / Om) { R = k; wR = om; LR = L; Rux = c.ux; Ruy = c.uy; }
            }
          } else {
            splat_f(image, S.W, S.H, c.ux, c.uy, L, kp.filter, AGG);
          }
        }
      }
    }
    bool refl = walk_scatter(S, w, v, ns, rho, r);
    walk_rr(kp, n, k, w);
    fnv(hash, (uint32_t)v.P.orig);
    fnv(hash, vtx_flags(v, refl, c.valid));
    if (EST == 3 && active) {
      // buffered two-pass: the splat record of this vertex, [depth][path]
      const Lrb2Layout lay = lrb2_layout(kp.n_paths, kp.max_depth);
      const size_t at = (size_t)k * kp.n_paths + p;
      ((float4*)((char*)aux + lay.rec4))[at] = make_float4(c.valid ? c.ux : -1.0f, c.uy, L.x, L.y);
      ((float*)((char*)aux + lay.recz))[at] = L.z;
    }
    if (EST == 2 && active) {
      // naive-AD tape: [depth][path] records of two float4
      float4* tape = (float4*)((char*)aux + kp.tape_offset) + 2 * ((size_t)k * kp.n_paths + p);
      uint32_t fl = vtx_flags(v, refl, c.valid);
      tape[0] = make_float4(__int_as_float(v.prim | (int)(fl << 24)), v.b1, v.b2, c.ux);
      tape[1] = make_float4(L.x, L.y, L.z, c.uy);
    }
    ++k;
  }
  if (ST && kp0.census) {
    atomicAdd(kp0.census + 0, (unsigned long long)cs.rays);
    atomicAdd(kp0.census + 1, (unsigned long long)cs.nodes);
    atomicAdd(kp0.census + 2, (unsigned long long)cs.prims);
    atomicAdd(kp0.census + 3, (unsigned long long)nverts);
    atomicAdd(kp0.census + 4, (unsigned long long)nconns);
  }
}

// Primal light tracing (Sec. 3.1, Eq. 1-2, splats by Eq. 20) for one estimator: EST 0 plain
// (with the LRB-3 state: validity masks, path list, first connections), 1 ResLRB reservoir
// records (Sec. 4.2, Eq. 8-9), 2 naive per-vertex tape (Sec. 3.2), 3 buffered splat records.
template <int EST>
__global__ void __launch_bounds__(128) k_primal(DevScene S, KParams kp, float* __restrict__ image, void* aux) {
  primal_body<EST, false>(S, kp, image, aux, BatchArgs{});
}
// Plain primal with warp-aggregated splat atomics (opts.scatter 3)
__global__ void __launch_bounds__(128) k_primal_agg(DevScene S, KParams kp, float* __restrict__ image, void* aux) {
  primal_body<0, false, false, false, true>(S, kp, image, aux, BatchArgs{});
}
// Counting variant of the plain primal (work census for the roofline; not for timed runs)
__global__ void __launch_bounds__(128) k_primal_census(DevScene S, KParams kp, float* __restrict__ image, void* aux) {
  primal_body<0, false, false, true>(S, kp, image, aux, BatchArgs{});
}
// ResLRB primal with the learned reservoir target, held to four blocks per SM
__global__ void __launch_bounds__(128, 4) k_primal_learned(DevScene S, KParams kp, float* __restrict__ image,
                                                           void* aux) {
  primal_body<1, false, true>(S, kp, image, aux, BatchArgs{});
}

// Batched primal: lanes take (item, path) chunks from the batch queue.
template <int EST>
__global__ void __launch_bounds__(256) k_primal_batch(BatchArgs ba) {
  primal_body<EST, true>(ba.jobs[0].S, ba.jobs[0].kp, nullptr, nullptr, ba);
}

// ======================================================================= LRB-3-pass
// Pass 2 (accumulate delta_total, Eq. 14) and pass 3 (backpropagate, Eq. 15-17) per path,
// run as a per-lane state machine: every iteration of the step loop performs one vertex
// step of whichever pass the lane is in (a closest-hit traversal of at most kTraceBudget
// visits, resumed in the next step if the ray needs more), and a lane that finishes a
// path takes the next one from its warp's range, in the same step as its last needed
// vertex, drawing again over paths with nothing to trace.  The connection-validity bits
// found in pass 2 are kept in a register mask so pass 3 traces no visibility rays.
// BATCH: per-lane item (BatchDispenser), global gradient atomics, per-item attached flag;
// S0, kp0, dI0 and g0 are not used.
// MODE 0: passes 2 and 3 fused per lane.  MODE 1: pass 2 only, storing delta_total and the
// validity mask of path p in xrec[p] (rgb, bits 0-31) and xhi[p] (bits 32-63).  MODE 2:
// pass 3 only, starting from that state (paths without a valid connection are skipped).
// MK (MODE 1): the primal stored each path's validity mask in xrec/xhi, so pass 2 takes
// connection validity from it, traces no visibility rays, stops after the last valid
// connection and skips paths without one.
// LOCAL: the calling block alone works on the path range (a span of a batch item).
// With a path list (kp.list, masks known): MODE 1 (MK) and MODE 2 visit only the listed
// paths, the ones with a valid connection, so no lane draws a path it has nothing to do for.
template <bool ATT, bool ST, bool CH, bool BATCH, int MODE = 0, bool MK = false, bool LOCAL = false>
__device__ __forceinline__ void lrb3_body(const DevScene& S0, const KParams& kp0, const float* __restrict__ dI0,
                                          const GradPtrs& g0, const BatchArgs& ba, float4* xrec = nullptr,
                                          uint32_t* xhi = nullptr) {
  extern __shared__ float sgrad[];
  GradPtrs gs = g0;
  if (!BATCH) {
    const Sink sink = sink_begin(kp0, g0, sgrad);
    gs.d_albedo = sink.alb;
    gs.d_heights = sink.h;
  }
  float3 Le = BATCH ? f3(0, 0, 0) : f3(kp0.Le[0], kp0.Le[1], kp0.Le[2]);
  float3 gLe = f3(0, 0, 0);
  Census cs = {0, 0, 0};
  uint32_t nverts = 0, nconns = 0;
  Dispenser disp;
  BatchDispenser bdisp;
  // the path list applies to pass 2 with known masks and to pass 3
  const uint32_t* list = (!BATCH && !LOCAL && (MODE == 2 || (MODE == 1 && MK))) ? kp0.list : nullptr;
  if (BATCH) bdisp.init();
  else if (LOCAL) disp.init_local(kp0.n_paths);
  else if (list) disp.init_dynamic(min((int64_t)*kp0.list_n, kp0.n_paths), kp0.ticket + (MODE == 1 ? 0 : 1));
  else disp.init(kp0.n_paths);
  int jb = 0;
  // FLUSH: the lane's path is done except the reverse sweep through the specular chain that
  // ends at its pending vertex; with DEFER the sweep waits for other lanes of the warp
  enum { IDLE = 0, PASS2 = 1, PASS3 = 2, FLUSH = 3 };
  constexpr bool DEFER = CH && ATT && !BATCH && MODE != 1;
  int phase = IDLE, k = 0, last = 0, nconn = 0;
  bool more = true;
  int64_t p = 0;
  Walk w;
  float3 dtot = f3(0, 0, 0), rem = f3(0, 0, 0);
  uint64_t valid = 0, known = 0;
  PendAdj pv;
  ChainInfo chain;
  chain.ka = -1;
  pv.prim = -1;
  ChainCache cc;
  cc.reset();
  TravState ts;  // the lane's ray in flight (see TravState)
  LocalStack stk;
  bool inflight = false;
  // Start path `got` (-1: the lane's range is exhausted) on the lane, or pass over it.
  auto start = [&](int64_t got) {
    const DevScene& S = BATCH ? ba.jobs[jb].S : S0;
    const KParams& kp = BATCH ? ba.jobs[jb].kp : kp0;
    float4* xr = xrec;
    uint32_t* xh = xhi;
    if (BATCH && MODE != 0) {
      xr = (float4*)ba.jobs[jb].state;
      xh = (uint32_t*)((char*)ba.jobs[jb].state + lrb3_state_split(kp.n_paths));
    }
    if (got >= 0 && list) got = (int64_t)list[got];
    if (got < 0) {
      more = false;
    } else if (MODE == 2) {
      const float4 a = xr[got];
      const uint64_t vm = (uint64_t)__float_as_uint(a.w) | ((uint64_t)xh[got] << 32);
      if (vm && (!kp.mask || kp.mask[got])) {
        p = got;
        if (BATCH) Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
        float3 x0;
        walk_start(S, kp.seed, (uint64_t)(kp.path_offset + p), Le, w, x0);
        rem = f3(a.x, a.y, a.z);
        valid = vm;
        pend_init(pv, -1, -1, 0.0f, 0.0f, x0, S.ln);
        chain.ka = -1;
        if (CH) cc.reset();
        last = 63 - __clzll((long long)valid);
        k = 0;
        phase = PASS3;
      }
    } else if (!kp.mask || kp.mask[got]) {
      if (MK) known = (uint64_t)__float_as_uint(xr[got].w) | ((uint64_t)xh[got] << 32);
      if (MK && !known) {  // no valid connection: delta_total = 0, the stored state stands
        if (kp.dbg) ((float4*)kp.dbg)[got] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
      }
      // one valid connection: k_lrb3_single has formed its delta_total without a replay
      if (MODE == 1 && MK && !BATCH && kp.conn1 && (known & (known - 1)) == 0ull) return;
      p = got;
      if (BATCH) Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
      float3 x0;
      walk_start(S, kp.seed, (uint64_t)(kp.path_offset + p), Le, w, x0);
      dtot = f3(0, 0, 0);
      valid = 0;
      if (MK) last = 63 - __clzll((long long)known);
      nconn = 0;
      k = 0;
      phase = PASS2;
    }
  };
  while (true) {
    // A chain sweep at a path end is long and runs only on the lanes that end a path at that
    // step.  With DEFER such a lane waits (FLUSH) until kFlushBatch lanes of its warp wait or
    // the warp has nothing else to do, and the waiting lanes then sweep together.
    if constexpr (DEFER) {
      const unsigned fq = __ballot_sync(0xffffffffu, phase == FLUSH);
      if (fq) {
        const unsigned busy = __ballot_sync(0xffffffffu, phase == PASS2 || phase == PASS3 || (more && phase == IDLE));
        if (__popc(fq) >= kFlushBatch || busy == 0u) {
          if (phase == FLUSH) {
            pend_flush<CH>(S0, kp0, (uint64_t)(kp0.path_offset + p), pv, gs.d_heights, &cc);
            phase = IDLE;
          }
        }
      }
    }
    // A lane that draws a path without a valid connection (pass 3, and pass 2 once the
    // primal's masks are known) has nothing to trace for it: it draws again, up to kDraws
    // times per step, instead of idling through the step.
    bool want = more && phase == IDLE;
    for (int draw = 0;; ++draw) {
      int jnew = jb;
      const int64_t got = BATCH ? bdisp.take(ba, want, jnew) : disp.take(want);
      if (BATCH && jnew != jb) {
        add3(ba.jobs[jb].g.d_Le, gLe);  // emitted-radiance gradient of the lane's previous item
        gLe = f3(0, 0, 0);
        jb = jnew;
      }
      if (want) start(got);
      want = want && more && phase == IDLE;
      if (draw + 1 == kDraws || !__any_sync(0xffffffffu, want)) break;
    }
    const DevScene& S = BATCH ? ba.jobs[jb].S : S0;
    const KParams& kp = BATCH ? ba.jobs[jb].kp : kp0;
    const float* dI = BATCH ? ba.jobs[jb].dI : dI0;
    const GradPtrs& g = BATCH ? ba.jobs[jb].g : gs;
    const bool att = ATT && (!BATCH || ba.jobs[jb].att);
    // per-path state of the two-kernel form (the lane's item's, in a batch)
    float4* xr = xrec;
    uint32_t* xh = xhi;
    if (BATCH && MODE != 0) {
      xr = (float4*)ba.jobs[jb].state;
      xh = (uint32_t*)((char*)ba.jobs[jb].state + lrb3_state_split(kp.n_paths));
    }
    if (!__any_sync(0xffffffffu, phase != IDLE || more)) break;
    // pass 2 with known masks also stops after the path's last valid connection
    const int kmax = phase == PASS2 && !MK ? kp.max_depth : last + 1;
    const bool trav = (phase == PASS2 || phase == PASS3) && k < kmax && !w.dead;
    HitRec h;
    h.prim = -1;
    bool pending = false;  // the ray has visits left: the lane resumes it in the next step
    if constexpr (CH) {
      // the specular-chain variants keep whole traversals: the resumable state would
      // push them past the register budget that their chain transport needs
      if (trav) h = trace_closest<ST>(S, w.org, w.dir, w.skip, &cs);
    } else if (trav) {
      if (!inflight) trace_begin<ST>(S, w.org, w.dir, w.skip, ts, &cs);
      inflight = !trace_resume<ST>(S, w.org, w.dir, w.skip, ts, stk, &cs);
      pending = inflight;
      h = ts.h;
    }
    Vtx v;
    const bool alive = trav && !pending && walk_finish(S, w, h, v);
    float3 ns = f3(0, 0, 0);
    Conn c;
    c.valid = false; c.ux = c.uy = 0.0f;
    if (alive && v.diffuse) {
      ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
      if (phase == PASS2 || ((valid >> k) & 1ull)) c = connect_pre(S, v.x, ns);
    }
    // visibility only in pass 2; pass 3 reuses pass 2's validity bits (and with MK pass 2
    // reuses the primal's)
    if (MK) {
      if (phase == PASS2 && c.valid) c.valid = (known >> k) & 1ull;
    } else {
      const bool vis = phase == PASS2 && c.valid;
      if (vis && occluded<ST>(S, v.x, c.wc, c.dist, v.prim, &cs)) c.valid = false;
    }
    if (phase == IDLE || phase == FLUSH || pending) continue;
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    if (MODE != 2 && phase == PASS2) {
      // the path ends at a miss, at the depth limit, or (known masks) once its last valid
      // connection is done, in the same step, so that the lane draws its next path at once
      bool fin = !alive;
      if (alive) {
        if (ST) ++nverts;
        float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
        float3 rho = f3(0, 0, 0);
        if (v.diffuse) {
          rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr);
          if (c.valid) {
            if (ST) ++nconns;
            valid |= 1ull << k;
            ++nconn;
            float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
            float3 Lb = adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, nullptr, kp.filter);
            dtot = dtot + mul(Lb, L);
          }
        }
        walk_scatter(S, w, v, ns, rho, r);
        walk_rr(kp, n, k, w);
        ++k;
        fin = MK && k > last;
      }
      if (fin) {
        if (kp.dbg) ((float4*)kp.dbg)[p] = make_float4(dtot.x, dtot.y, dtot.z, (float)nconn);
        gLe = gLe + f3(dtot.x / Le.x, dtot.y / Le.y, dtot.z / Le.z);  // emitted factor, weight delta_total
        if (MODE == 1) {
          xr[p] = make_float4(dtot.x, dtot.y, dtot.z, __uint_as_float((uint32_t)valid));
          xh[p] = (uint32_t)(valid >> 32);
          phase = IDLE;
        } else if (valid) {
          float3 x0;
          walk_start(S, kp.seed, n, Le, w, x0);
          rem = dtot;
          pend_init(pv, -1, -1, 0.0f, 0.0f, x0, S.ln);
          chain.ka = -1;
          if (CH) cc.reset();
          last = 63 - __clzll((long long)valid);
          k = 0;
          phase = PASS3;
        } else {
          phase = IDLE;
        }
      }
    } else if (MODE != 1) {
      bool fin = !alive;  // a miss, or the path's last valid connection is done
      if (alive) {
        if (ST) ++nverts;
        float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
        // attached segment weight and chain bookkeeping: every connection from here on
        // carries this vertex's factors, so they weigh the remaining adjoint before Eq. 16
        if (att) att_enter<CH>(S, kp, n, k, v, hsum(rem), hsum(rem), pv, chain, g.d_heights, &cc);
        const bool rec_chain = CH && att && !v.diffuse;
        if (rec_chain) cc.record(chain, k, v, w.dir);
        float3 rho = f3(0, 0, 0);
        if (v.diffuse) {
          TexFoot foot;
          rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, &foot);
          float3 wsplat = f3(0, 0, 0);
          if ((valid >> k) & 1ull) {
            float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
            float2 q;
            float3 Lb = adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, att ? &q : nullptr, kp.filter);
            float3 P = mul(Lb, L);
            wsplat = P;           // splat factor rho_k / pi (Eq. 15)
            rem = rem - P;        // Eq. 16
            if (att) conn_adjoint(S, v.x, v.nraw, hsum(P), q, pv.gx, pv.gn);
          }
          scatter_albedo(S, g.d_albedo, foot, wsplat + rem, rho);  // + scattering factor rho_k (Eq. 17)
          if (att && CH && !v.attached)
            pv.gx = pv.gx + tex_pos_adjoint(kp.albedo, v.m, v.P, v.b1, v.b2, wsplat + rem, rho);
        }
        const bool refl = walk_scatter(S, w, v, ns, rho, r);
        if (rec_chain) cc.record_branch(refl);
        walk_rr(kp, n, k, w);
        ++k;
        fin = k > last;
      }
      if (fin) {
        if (DEFER && pv.prim >= 0 && pv.sliding && g.d_heights) {
          phase = FLUSH;
        } else {
          if (att) pend_flush<CH>(S, kp, n, pv, g.d_heights, &cc);
          phase = IDLE;
        }
      }
    }
  }
  if (BATCH) {
    add3(ba.jobs[jb].g.d_Le, gLe);
    return;
  }
  if (ST && kp0.census) {
    atomicAdd(kp0.census + 0, (unsigned long long)cs.rays);
    atomicAdd(kp0.census + 1, (unsigned long long)cs.nodes);
    atomicAdd(kp0.census + 2, (unsigned long long)cs.prims);
    atomicAdd(kp0.census + 3, (unsigned long long)nverts);
    atomicAdd(kp0.census + 4, (unsigned long long)nconns);
  }
  sink_end(kp0, g0, sgrad);
  block_add3(g0.d_Le, gLe);
}

template <bool ATT, bool ST, bool CH>
__global__ void __launch_bounds__(128, 4) k_lrb3(DevScene S, KParams kp, const float* __restrict__ dI, GradPtrs g0) {
  lrb3_body<ATT, ST, CH, false>(S, kp, dI, g0, BatchArgs{});
}

// Two-kernel form: pass 2 (per-path state out, emitted-radiance gradient) ...
// Both passes are latency-bound traversals that gain from more resident warps more than
// they lose to spilled registers: measured on the GB300, pass 2 at 6 blocks of 128 threads
// per SM and the specular-chain pass 3 at 8 (64 registers; the chain sweep inlined) took the
// caustic backward from 8.8 to 7.4 ms, while the lean pass 3 (no chains) was fastest at 4.
template <bool ST, bool MK>
__global__ void __launch_bounds__(128, 6) k_lrb3_p2(DevScene S, KParams kp, const float* __restrict__ dI, GradPtrs g0,
                                                 float4* xrec, uint32_t* xhi) {
  lrb3_body<false, ST, false, false, 1, MK>(S, kp, dI, g0, BatchArgs{}, xrec, xhi);
}
// Pass 2 of the paths with exactly one valid connection (known masks, the primal's record of
// each path's first valid connection): delta_total = Lbar (.) L of that connection (Eq. 14)
// from its recorded film position and contribution, the values a replay computes, one thread
// per listed path; k_lrb3_p2 leaves these paths out.  On the caustic workload they are 98 %
// of the paths with a connection.
__global__ void __launch_bounds__(256) k_lrb3_single(DevScene S, KParams kp, const float* __restrict__ dI,
                                                    GradPtrs g, float4* xrec, const uint32_t* xhi) {
  const int64_t n = kp.list ? min((int64_t)*kp.list_n, kp.n_paths) : kp.n_paths;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  unsigned long long ones = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = kp.list ? (int64_t)kp.list[i] : i;
    if (kp.mask && !kp.mask[p]) continue;
    const float4 r = xrec[p];
    const uint64_t known = (uint64_t)__float_as_uint(r.w) | ((uint64_t)xhi[p] << 32);
    if (known == 0ull || (known & (known - 1)) != 0ull) continue;
    const float4 a = kp.conn1[p];
    const float3 L = f3(a.z, a.w, kp.conn1z[p]);
    const float3 d = mul(adjoint_read_f(dI, S.W, S.H, a.x, a.y, L, nullptr, kp.filter), L);
    xrec[p] = make_float4(d.x, d.y, d.z, r.w);
    gLe = gLe + f3(d.x / Le.x, d.y / Le.y, d.z / Le.z);  // emitted factor, weight delta_total
    ++ones;
    if (kp.dbg) ((float4*)kp.dbg)[p] = make_float4(d.x, d.y, d.z, 1.0f);
  }
  if (kp.census) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ones += __shfl_xor_sync(0xffffffffu, ones, o);
    if ((threadIdx.x & 31) == 0 && ones) atomicAdd(kp.census + 4, ones);
  }
  block_add3(g.d_Le, gLe);
}

// ... then pass 3 (albedo and height gradients) from that state.
template <bool ATT, bool ST, bool CH>
__global__ void __launch_bounds__(128, CH ? 8 : 4) k_lrb3_p3(DevScene S, KParams kp, const float* __restrict__ dI, GradPtrs g0,
                                                 const float4* xrec, const uint32_t* xhi) {
  lrb3_body<ATT, ST, CH, false, 2>(S, kp, dI, g0, BatchArgs{}, const_cast<float4*>(xrec),
                                   const_cast<uint32_t*>(xhi));
}

// Batched two-kernel form: pass 2 over every item, then pass 3 per kernel group.
template <bool MK>
__global__ void __launch_bounds__(256) k_lrb3_p2_batch(BatchArgs ba) {
  lrb3_body<false, false, false, true, 1, MK>(ba.jobs[0].S, ba.jobs[0].kp, nullptr, ba.jobs[0].g, ba);
}
template <bool ATT, bool CH>
__global__ void __launch_bounds__(256) k_lrb3_p3_batch(BatchArgs ba) {
  lrb3_body<ATT, false, CH, true, 2>(ba.jobs[0].S, ba.jobs[0].kp, nullptr, ba.jobs[0].g, ba);
}

// Batched pass 3 by spans: a block takes the next span (one atomic by its first thread),
// runs the single-scene pass-3 body over it with the item's shared-memory gradient sink,
// and flushes the sink into the item's arrays at the end of the span.
template <bool ATT, bool CH>
__global__ void __launch_bounds__(256) k_lrb3_p3_spans(const BatchJob* __restrict__ jobs,
                                                       const BatchSpan* __restrict__ spans, int n_spans,
                                                       unsigned long long* ticket) {
  __shared__ int s_span;
  while (true) {
    if (threadIdx.x == 0) s_span = (int)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int sp = s_span;
    __syncthreads();
    if (sp >= n_spans) break;
    const BatchSpan span = spans[sp];
    const BatchJob& J = jobs[span.job];
    KParams kp = J.kp;
    kp.path_offset += span.start;
    kp.n_paths = span.end - span.start;
    if (kp.mask) kp.mask += span.start;
    if (kp.dbg) kp.dbg += 4 * span.start;
    float4* xr = (float4*)J.state + span.start;
    uint32_t* xh = (uint32_t*)((char*)J.state + lrb3_state_split(J.kp.n_paths)) + span.start;
    GradPtrs g = J.g;
    g.d_Le = nullptr;  // pass 2 added the emitted-radiance gradient
    const bool att = ATT && J.att;
    if (att) lrb3_body<ATT, false, CH, false, 2, false, true>(J.S, kp, J.dI, g, BatchArgs{}, xr, xh);
    else lrb3_body<false, false, false, false, 2, false, true>(J.S, kp, J.dI, g, BatchArgs{}, xr, xh);
  }
}

template <bool ATT, bool CH>
__global__ void __launch_bounds__(256) k_lrb3_batch(BatchArgs ba) {
  lrb3_body<ATT, false, CH, true>(ba.jobs[0].S, ba.jobs[0].kp, nullptr, ba.jobs[0].g, ba);
}

// ======================================================================= ResLRB backward
// Replay to the selected vertex R and apply the log-derivative identity with weight
// Lbar_R * S to every factor of L_R (Eq. 11); attached adds the positional channel.
// The ResLRB backward pass as a per-lane state machine, like the LRB-3 passes: a lane replays
// one path to its selected vertex R, draws its next path in the same step as it finishes,
// draws again over paths without a selected connection, and (scenes without dielectrics)
// resumes long traversals over several steps.  `att` (per item in a batch) selects the
// attached formulation; ATT gates its code at compile time.
template <bool ATT, bool CH, bool BATCH>
__device__ __forceinline__ void reslrb_body(const DevScene& S0, const KParams& kp0, const float* __restrict__ dI0,
                                            const float4* __restrict__ rec0, const GradPtrs& g0, const BatchArgs& ba) {
  extern __shared__ float sgrad[];
  GradPtrs gs = g0;
  if (!BATCH) {
    const Sink sink = sink_begin(kp0, g0, sgrad);
    gs.d_albedo = sink.alb;
    gs.d_heights = sink.h;
  }
  float3 Le = BATCH ? f3(0, 0, 0) : f3(kp0.Le[0], kp0.Le[1], kp0.Le[2]);
  float3 gLe = f3(0, 0, 0);
  Dispenser disp;
  BatchDispenser bdisp;
  if (BATCH) bdisp.init(); else disp.init(kp0.n_paths);
  int jb = 0;
  bool busy = false, more = true;
  int64_t p = 0;
  int k = 0, R = 0;
  float3 P = f3(0, 0, 0);  // Lbar_R * S: the weight of every factor of L_R
  float lam = 0.0f;
  float2 q = make_float2(0.0f, 0.0f);
  Walk w;
  PendAdj pv;
  ChainInfo chain;
  chain.ka = -1;
  pv.prim = -1;
  ChainCache cc;
  cc.reset();
  TravState ts;
  LocalStack stk;
  bool inflight = false;
  auto start = [&](int64_t got) {
    if (got < 0) { more = false; return; }
    const DevScene& S = BATCH ? ba.jobs[jb].S : S0;
    const KParams& kp = BATCH ? ba.jobs[jb].kp : kp0;
    const float* dI = BATCH ? ba.jobs[jb].dI : dI0;
    const float4* rec = BATCH ? (const float4*)ba.jobs[jb].rec : rec0;
    const bool att = ATT && (!BATCH || ba.jobs[jb].att);
    if (kp.mask && !kp.mask[got]) return;
    const float4 r0 = rec[2 * got], r1 = rec[2 * got + 1];
    const int Rr = __float_as_int(r0.x);
    if (Rr < 0) return;
    if (Rr >= kp.max_depth) { set_err(S, ERR_BOUNDS); return; }
    p = got;
    R = Rr;
    if (BATCH) Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
    const float3 Sh = f3(r1.x, r1.y, r1.z);
    const float3 Lb = adjoint_read_f(dI, S.W, S.H, r0.z, r0.w, Sh, att ? &q : nullptr, kp.filter);
    P = mul(Lb, Sh);
    lam = hsum(P);
    gLe = gLe + f3(P.x / Le.x, P.y / Le.y, P.z / Le.z);
    float3 x0;
    walk_start(S, kp.seed, (uint64_t)(kp.path_offset + p), Le, w, x0);
    pend_init(pv, -1, -1, 0.0f, 0.0f, x0, S.ln);
    chain.ka = -1;
    if (CH) cc.reset();
    k = 0;
    busy = true;
  };
  while (true) {
    bool want = more && !busy;
    for (int draw = 0;; ++draw) {
      int jnew = jb;
      const int64_t got = BATCH ? bdisp.take(ba, want, jnew) : disp.take(want);
      if (BATCH && jnew != jb) {
        add3(ba.jobs[jb].g.d_Le, gLe);  // emitted-radiance gradient of the lane's previous item
        gLe = f3(0, 0, 0);
        jb = jnew;
      }
      if (want) start(got);
      want = want && more && !busy;
      if (draw + 1 == kDraws || !__any_sync(0xffffffffu, want)) break;
    }
    if (!__any_sync(0xffffffffu, busy || more)) break;
    const DevScene& S = BATCH ? ba.jobs[jb].S : S0;
    const KParams& kp = BATCH ? ba.jobs[jb].kp : kp0;
    const GradPtrs& g = BATCH ? ba.jobs[jb].g : gs;
    const bool att = ATT && (!BATCH || ba.jobs[jb].att);
    const bool trav = busy && !w.dead;
    HitRec h;
    h.prim = -1;
    bool pending = false;
    if constexpr (CH) {
      if (trav) h = trace_closest(S, w.org, w.dir, w.skip);
    } else if (trav) {
      if (!inflight) trace_begin(S, w.org, w.dir, w.skip, ts);
      inflight = !trace_resume(S, w.org, w.dir, w.skip, ts, stk);
      pending = inflight;
      h = ts.h;
    }
    Vtx v;
    const bool alive = trav && !pending && walk_finish(S, w, h, v);
    if (!busy || pending) continue;
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    if (!alive) {  // the replay must reach the vertex the primal selected
      set_err(S, ERR_BOUNDS);
      busy = false;
      continue;
    }
    const float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
    if (att) att_enter<CH>(S, kp, n, k, v, lam, lam, pv, chain, g.d_heights, &cc);
    const bool rec_chain = CH && att && !v.diffuse;
    if (rec_chain) cc.record(chain, k, v, w.dir);
    float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
    if (v.diffuse) {
      ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
      TexFoot foot;
      rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, &foot);
      scatter_albedo(S, g.d_albedo, foot, P, rho);  // scattering factor (k < R) or splat factor (k = R)
      if (att) {
        if (k == R) conn_adjoint(S, v.x, v.nraw, lam, q, pv.gx, pv.gn);
        if (CH && !v.attached) pv.gx = pv.gx + tex_pos_adjoint(kp.albedo, v.m, v.P, v.b1, v.b2, P, rho);
      }
    }
    const bool refl = walk_scatter(S, w, v, ns, rho, r);
    if (rec_chain) cc.record_branch(refl);
    walk_rr(kp, n, k, w);
    if (++k > R) {
      if (att) pend_flush<CH>(S, kp, n, pv, g.d_heights, &cc);
      busy = false;
    }
  }
  if (BATCH) {
    add3(ba.jobs[jb].g.d_Le, gLe);
    return;
  }
  sink_end(kp0, g0, sgrad);
  block_add3(g0.d_Le, gLe);
}

// ResLRB backward (Sec. 4.2.1-4.2.2, Eq. 11-13): replay each path to its reservoir vertex R
// and weight every factor of L_R with Lbar_R (.) S from the primal's record.
template <bool ATT, bool CH>
__global__ void __launch_bounds__(128) k_reslrb(DevScene S, KParams kp, const float* __restrict__ dI,
                                                const float4* __restrict__ rec, GradPtrs g0) {
  reslrb_body<ATT, CH, false>(S, kp, dI, rec, g0, BatchArgs{});
}

// Batched ResLRB backward: lanes take paths from the batch queue.
template <bool ATT, bool CH>
__global__ void __launch_bounds__(256) k_reslrb_batch(BatchArgs ba) {
  reslrb_body<ATT, CH, true>(ba.jobs[0].S, ba.jobs[0].kp, nullptr, nullptr, GradPtrs{}, ba);
}

// ======================================================================= buffered two-pass
// lrb_2pass backward, first step: delta_total = sum_i Lbar_i * L_i (Eq. 14) and the
// connection-validity mask of every path from the splat records the primal stored, with
// no traversal; pass 3 of LRB-3 then backpropagates from that state.
__global__ void __launch_bounds__(128) k_lrb2_reduce(DevScene S, KParams kp, const float* __restrict__ dI,
                                                     void* buf, float* d_Le) {
  const Lrb2Layout lay = lrb2_layout(kp.n_paths, kp.max_depth);
  float4* xrec = (float4*)buf;
  uint32_t* xhi = (uint32_t*)((char*)buf + lrb3_state_split(kp.n_paths));
  const int* cnt = (const int*)((const char*)buf + lay.counts);
  const float4* r4 = (const float4*)((const char*)buf + lay.rec4);
  const float* rz = (const float*)((const char*)buf + lay.recz);
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    int K = cnt[p];
    if (K > kp.max_depth) { set_err(S, ERR_BOUNDS); K = 0; }
    float3 dtot = f3(0, 0, 0);
    uint64_t valid = 0;
    int nconn = 0;
    for (int k = 0; k < K; ++k) {
      const size_t at = (size_t)k * kp.n_paths + p;
      const float4 a = r4[at];
      if (a.x < 0.0f) continue;
      const float3 L = f3(a.z, a.w, rz[at]);
      dtot = dtot + mul(adjoint_read_f(dI, S.W, S.H, a.x, a.y, L, nullptr, kp.filter), L);
      valid |= 1ull << k;
      ++nconn;
    }
    xrec[p] = make_float4(dtot.x, dtot.y, dtot.z, __uint_as_float((uint32_t)valid));
    xhi[p] = (uint32_t)(valid >> 32);
    gLe = gLe + f3(dtot.x / Le.x, dtot.y / Le.y, dtot.z / Le.z);  // emitted factor, weight delta_total
    if (kp.dbg) ((float4*)kp.dbg)[p] = make_float4(dtot.x, dtot.y, dtot.z, (float)nconn);
  }
  block_add3(d_Le, gLe);
}

// ======================================================================= naive reverse
// Reverse sweep over the per-vertex tape: suffix sums of Lbar_i L_i replace the replay.
template <bool ATT, bool CH>
__global__ void __launch_bounds__(128) k_naive(DevScene S, KParams kp, const float* __restrict__ dI,
                                               const void* __restrict__ ws, GradPtrs g0) {
  extern __shared__ float sgrad[];
  const Sink sink = sink_begin(kp, g0, sgrad);
  GradPtrs g = g0;
  g.d_albedo = sink.alb;
  g.d_heights = sink.h;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  const int* cnt = (const int*)ws;
  const float4* tape = (const float4*)((const char*)ws + kp.tape_offset);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    int K = cnt[p];
    if (K <= 0) continue;
    if (K > kp.max_depth) { set_err(S, ERR_BOUNDS); continue; }
    float3 x0 = f3(0, 0, 0);
    if (ATT) {
      float4 r = rand4(kp.seed, (uint64_t)(kp.path_offset + p), 0);
      x0 = S.lo + S.le1 * r.x + S.le2 * r.y;
    }
    float3 acc = f3(0, 0, 0);  // sum of Lbar_j L_j over j > k
    float3 cgx = f3(0, 0, 0), cgn = f3(0, 0, 0);  // adjoint carried to vertex k by vertex k+1
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    for (int k = K - 1; k >= 0; --k) {
      float4 t0 = tape[2 * ((size_t)k * kp.n_paths + p)], t1 = tape[2 * ((size_t)k * kp.n_paths + p) + 1];
      int pk = __float_as_int(t0.x);
      int prim = pk & 0xffffff;
      uint32_t fl = (uint32_t)pk >> 24;
      if (prim >= S.n_prims) { set_err(S, ERR_BOUNDS); break; }
      const bool diffuse = (fl & 3u) == K_DIFFUSE, attached = (fl & 16u) != 0;
      if (!ATT && !diffuse) continue;  // dielectric vertices carry no detached factor
      Prim P = load_prim(S, prim);
      int4 m = __ldg(S.mat + P.mat);
      float3 P3 = f3(0, 0, 0), rho = f3(1, 1, 1);
      float2 q = make_float2(0.0f, 0.0f);
      if (diffuse) {
        TexFoot foot;
        rho = tex_lookup(kp.albedo, m, t0.y, t0.z, &foot);
        float3 L = f3(t1.x, t1.y, t1.z);
        if (fl & 8u) {
          float3 Lb = adjoint_read_f(dI, S.W, S.H, t0.w, t1.w, L, ATT ? &q : nullptr, kp.filter);
          P3 = mul(Lb, L);
        }
        scatter_albedo(S, g.d_albedo, foot, P3 + acc, rho);
      }
      if (ATT) {
        float3 x = P.o + P.e1 * t0.y + P.e2 * t0.z, nr = cross(P.e1, P.e2);
        float3 gx = cgx, gn = cgn;
        cgx = cgn = f3(0, 0, 0);
        const float lam = hsum(P3 + acc);  // every connection from this vertex on
        if (diffuse) {
          if (fl & 8u) conn_adjoint(S, x, nr, hsum(P3), q, gx, gn);
          if (CH && !attached) gx = gx + tex_pos_adjoint(kp.albedo, m, P, t0.y, t0.z, P3 + acc, rho);
        }
        if (!CH || attached) {
          float3 xp = x0, np = S.ln;
          if (k > 0) {
            float4 s0 = tape[2 * ((size_t)(k - 1) * kp.n_paths + p)];
            Prim Q = load_prim(S, __float_as_int(s0.x) & 0xffffff);
            xp = Q.o + Q.e1 * s0.y + Q.e2 * s0.z;
            np = cross(Q.e1, Q.e2);
          }
          seg_adjoint(xp, np, x, nr, lam, cgx, cgn, gx, gn);
          scatter_heights(S, g.d_heights, prim, t0.y, t0.z, gx, gn);
        } else if (CH && diffuse) {
          // end of a specular chain: find its attached start and anchor on the tape
          int a = k - 1;
          while (a >= 0 && !((((uint32_t)__float_as_int(tape[2 * ((size_t)a * kp.n_paths + p)].x)) >> 24) & 16u)) --a;
          if (a < 0) { set_err(S, ERR_BOUNDS); break; }
          float4 sa = tape[2 * ((size_t)a * kp.n_paths + p)];
          ChainInfo c;
          c.ka = a; c.prim_a = __float_as_int(sa.x) & 0xffffff; c.ba1 = sa.y; c.ba2 = sa.z; c.lam = lam;
          c.xp = x0; c.np = S.ln; c.prim_p = -1; c.bp1 = c.bp2 = 0.0f; c.kanchor = -1; c.anchor_sliding = false;
          if (a > 0) {
            float4 sp = tape[2 * ((size_t)(a - 1) * kp.n_paths + p)];
            int pprim = __float_as_int(sp.x) & 0xffffff;
            Prim Q = load_prim(S, pprim);
            c.xp = Q.o + Q.e1 * sp.y + Q.e2 * sp.z;
            c.np = cross(Q.e1, Q.e2);
            c.prim_p = pprim; c.bp1 = sp.y; c.bp2 = sp.z; c.kanchor = a - 1;
            c.anchor_sliding = !((((uint32_t)__float_as_int(sp.x)) >> 24) & 16u);
          }
          scatter_heights(S, g.d_heights, prim, 0.0f, 0.0f, f3(0, 0, 0), gn);
          propagate_sliding(S, kp, n, c, k, gx, g.d_heights, nullptr, prim);
        }
      }
      acc = acc + P3;
    }
    gLe = gLe + f3(acc.x / Le.x, acc.y / Le.y, acc.z / Le.z);
  }
  sink_end(kp, g0, sgrad);
  block_add3(g.d_Le, gLe);
}

// ======================================================================= bidirectional
// Two strategies for the paths x0 (emitter), x1..xk (diffuse) -> camera, combined by the
// balance heuristic: the light tracer's sensor connection at xk (N light paths) and a camera
// sample through a film position uniform over the film, traced to xk = y1, ..., x1 = ym by
// cosine sampling, with next-event estimation from ym to a point x0 uniform on the emitter
// (M camera samples).  For Lambertian surfaces, cosine sampling and cosine emission a
// segment between two surfaces has the same area density in both directions, so the
// density ratio of the camera strategy to the light strategy is R = p_film(xk) / pf0
// (p_film: the film's area density at xk, geo * pi / (W H); pf0 = cos0 cos1 / (pi r01^2),
// the light tracer's density of x1), and a sample of either strategy contributes
// L_N / (N + M R), L_N the light tracer's splat value times N.  Diffuse scenes, detached.

// Balance-heuristic factor N / (N + M R) of a light-tracer connection of weight geo
// (importance without the estimator's 1/N) on a path whose first segment has density pf0.
__device__ __forceinline__ float bidir_light_w(const DevScene& S, const BidirArgs& ba, float geo, float pf0) {
  const float R = geo * kPi / ((float)S.W * (float)S.H * pf0);
  return ba.N / fmaf(ba.M, R, ba.N);
}

// Light side.  BWD = false: the primal (splat every weighted connection).  BWD = true: the
// LRB-3 adjoint in one kernel per path (pass 2 accumulates delta_total, Eq. 14; pass 3
// replays to the last valid connection, Eq. 15-17), detached.
template <bool BWD>
__global__ void __launch_bounds__(128) k_bidir_light(DevScene S, KParams kp, BidirArgs ba, float* __restrict__ image,
                                                     const float* __restrict__ dI, GradPtrs g0) {
  extern __shared__ float sgrad[];
  GradPtrs g = g0;
  if (BWD) g.d_albedo = sink_begin(kp, g0, sgrad).alb;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    const bool active = !kp.mask || kp.mask[p];
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    Walk w;
    float3 x0;
    walk_start(S, kp.seed, n, Le, w, x0);
    uint32_t hash = 2166136261u;
    float pf0 = 0.0f;
    float3 dtot = f3(0, 0, 0);
    uint64_t valid = 0;
    for (int k = 0; k < kp.max_depth; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) break;
      if (k == 0) {
        const float3 d = v.x - x0;
        pf0 = fabsf(dot(S.ln, w.dir)) * fabsf(dot(v.n, w.dir)) / (kPi * dot(d, d));
      }
      const float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      bool conn = false;
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr);
        const Conn c = connect(S, v.x, ns, v.prim);
        conn = c.valid;
        if (c.valid && active) {
          const float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n * bidir_light_w(S, ba, c.geo, pf0));
          if (!BWD) {
            splat_f(image, S.W, S.H, c.ux, c.uy, L, kp.filter);
          } else {
            dtot = dtot + mul(adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, nullptr, kp.filter), L);
            valid |= 1ull << k;
          }
        }
      }
      const bool refl = walk_scatter(S, w, v, ns, rho, r);
      fnv(hash, (uint32_t)v.P.orig);
      fnv(hash, vtx_flags(v, refl, conn));
    }
    if (!BWD && kp.hash) kp.hash[p] = hash;
    if (!BWD || !valid) continue;
    gLe = gLe + f3(dtot.x / Le.x, dtot.y / Le.y, dtot.z / Le.z);  // emitted factor, weight delta_total
    walk_start(S, kp.seed, n, Le, w, x0);
    float3 rem = dtot;
    const int last = 63 - __clzll((long long)valid);
    for (int k = 0; k <= last; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) { set_err(S, ERR_BOUNDS); break; }  // the replay must reach `last`
      if (k == 0) {
        const float3 d = v.x - x0;
        pf0 = fabsf(dot(S.ln, w.dir)) * fabsf(dot(v.n, w.dir)) / (kPi * dot(d, d));
      }
      const float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        TexFoot foot;
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, &foot);
        float3 wsplat = f3(0, 0, 0);
        if ((valid >> k) & 1ull) {
          const Conn c = connect_pre(S, v.x, ns);
          const float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n * bidir_light_w(S, ba, c.geo, pf0));
          wsplat = mul(adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, nullptr, kp.filter), L);  // Eq. 15
          rem = rem - wsplat;                                                                  // Eq. 16
        }
        scatter_albedo(S, g.d_albedo, foot, wsplat + rem, rho);  // + scattering factor with delta_rem (Eq. 17)
      }
      walk_scatter(S, w, v, ns, rho, r);
    }
  }
  if (BWD) {
    sink_end(kp, g0, sgrad);
    block_add3(g0.d_Le, gLe);
  }
}

// The camera sample c: film position from Philox stream 3 at (c, 0); at camera vertex m the
// cosine direction (u0, u1) and the emitter point of the next-event connection (u2, u3)
// from (c, m).  Returns the vertex's contribution (zero without a valid connection) and
// continues the sample's walk; false when the walk ends (miss, emitter, depth).
struct CamWalk {
  float3 org, dir, thr;  // ray and the product of the albedos so far
  int skip;
  float geo1, pfilm;     // sensor connection at the first vertex
};
__device__ __forceinline__ void cam_start(const DevScene& S, const KParams& kp, uint64_t c, CamWalk& cw, float& ux,
                                          float& uy) {
  const float4 r0 = rand4(kp.seed, c, 0, 3);
  ux = r0.x * (float)S.W;
  uy = r0.y * (float)S.H;
  const float px = (2.0f * ux / (float)S.W - 1.0f) * S.tanx, py = (1.0f - 2.0f * uy / (float)S.H) * S.tany;
  cw.dir = normalize(S.cf + S.cr * px + S.cu * py);
  cw.org = S.cpos;
  cw.skip = -1;
  cw.thr = f3(1, 1, 1);
  cw.geo1 = cw.pfilm = 0.0f;
}
template <bool VIS>
__device__ __forceinline__ bool cam_vertex(const DevScene& S, const KParams& kp, const BidirArgs& ba, uint64_t c,
                                           int m, CamWalk& cw, bool nee_known, float3& contrib, bool& nee,
                                           TexFoot* foot, float3& rho, uint32_t& hash) {
  const HitRec h = trace_closest(S, cw.org, cw.dir, cw.skip);
  if (h.prim < 0) return false;
  const Prim P = load_prim(S, h.prim);
  const int4 mt = __ldg(S.mat + P.mat);
  if (mt.x != MAT_DIFFUSE) return false;  // the emitter absorbs (seen directly it is black)
  const float3 x = P.o + P.e1 * h.b1 + P.e2 * h.b2;
  const float3 nraw = cross(P.e1, P.e2), nn = normalize(nraw);
  const float3 ns = dot(nraw, cw.dir) < 0.0f ? nn : -nn;
  if (m == 1) {
    const float3 d = x - S.cpos;
    const float dist = length(d), cc = dot(d, S.cf) / dist;
    const float cosc = -dot(ns, d) / dist;
    cw.geo1 = cosc * S.K0 / (dist * dist * cc * cc * cc);
    cw.pfilm = cw.geo1 * kPi / ((float)S.W * (float)S.H);
  }
  rho = tex_lookup(kp.albedo, mt, h.b1, h.b2, foot);
  cw.thr = mul(cw.thr, rho);
  const float4 r = rand4(kp.seed, c, (uint32_t)m, 3);
  const float3 xl = S.lo + S.le1 * r.z + S.le2 * r.w;
  const float3 wl = xl - x;
  const float dl = length(wl);
  const float3 wn = wl * (1.0f / dl);
  const float cx = dot(ns, wn), cl = -dot(S.ln, wn);
  nee = VIS ? (cx > 0.0f && cl > 0.0f && !occluded(S, x, wn, dl, h.prim)) : nee_known;
  contrib = f3(0, 0, 0);
  if (nee) {
    const float pf0 = cx * cl / (kPi * dl * dl);
    const float wgt = S.light_area * kPi * cw.geo1 / fmaf(ba.M, cw.pfilm / pf0, ba.N);
    contrib = mul(f3(kp.Le[0], kp.Le[1], kp.Le[2]), cw.thr) * wgt;
  }
  fnv(hash, (uint32_t)P.orig);
  fnv(hash, nee ? 1u : 0u);
  cw.dir = cosine_dir(ns, r.x, r.y);
  cw.org = x;
  cw.skip = h.prim;
  return true;
}

// Camera side.  BWD = false: each sample splats the sum of its vertices' contributions at
// its film position.  BWD = true: path replay backpropagation (one adjoint read per sample,
// the sample's film position being fixed): a first walk sums the contributions, a replay
// weights each vertex's albedo with the adjoint of the contributions from that vertex on.
template <bool BWD>
__global__ void __launch_bounds__(128) k_bidir_cam(DevScene S, KParams kp, BidirArgs ba, float* __restrict__ image,
                                                   const float* __restrict__ dI, GradPtrs g0) {
  extern __shared__ float sgrad[];
  GradPtrs g = g0;
  if (BWD) g.d_albedo = sink_begin(kp, g0, sgrad).alb;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ba.n_cam; c += stride) {
    const bool active = !ba.cam_mask || ba.cam_mask[c];
    CamWalk cw;
    float ux, uy;
    cam_start(S, kp, (uint64_t)c, cw, ux, uy);
    uint32_t hash = 2166136261u;
    float3 total = f3(0, 0, 0), contrib, rho;
    uint64_t nees = 0;
    bool nee;
    for (int m = 1; m <= kp.max_depth; ++m) {
      if (!cam_vertex<true>(S, kp, ba, (uint64_t)c, m, cw, false, contrib, nee, nullptr, rho, hash)) break;
      total = total + contrib;
      if (nee) nees |= 1ull << (m - 1);
    }
    if (!BWD) {
      if (ba.cam_hash) ba.cam_hash[c] = hash;
      if (active && nees) splat_f(image, S.W, S.H, ux, uy, total, kp.filter);
      continue;
    }
    if (!active || !nees) continue;
    const float3 Lb = adjoint_read_f(dI, S.W, S.H, ux, uy, total, nullptr, kp.filter);
    const float3 P = mul(Lb, total);
    gLe = gLe + f3(P.x / Le.x, P.y / Le.y, P.z / Le.z);
    cam_start(S, kp, (uint64_t)c, cw, ux, uy);
    float3 rem = total;
    const int last = 64 - __clzll((long long)nees);
    for (int m = 1; m <= last; ++m) {
      TexFoot foot;
      if (!cam_vertex<false>(S, kp, ba, (uint64_t)c, m, cw, (nees >> (m - 1)) & 1ull, contrib, nee, &foot, rho,
                             hash)) {
        set_err(S, ERR_BOUNDS);  // the replay must reach the last connection
        break;
      }
      scatter_albedo(S, g.d_albedo, foot, mul(Lb, rem), rho);  // every contribution from this vertex on
      rem = rem - contrib;
    }
  }
  if (BWD) {
    sink_end(kp, g0, sgrad);
    block_add3(g0.d_Le, gLe);
  }
}

// ======================================================================= paper-literal attached LRB-3
// The paper's transport of the splat-position adjoint (Sec. 3.3, Eq. 4-7; Sec. 4.3.2, Eq.
// 18-19; Sec. 5) in place of the exact chain transport: per path the segment states
// p_k = (v_{k-1}, v_k) (surface coordinates; v_{-1} the emitter's (s, t)), their Jacobians
// J_k = d p_{k+1} / d p_k accumulated forward (Jacc_k = d p_k / d p_0, 4x4), the position
// rows a_k = (0, 0, dL/du du/dv_k) of every valid connection summed as
// A_pos = sum_k a_k Jacc_k in pass 2 (Eq. 18), and in pass 3 the remainder projected back at
// each specular vertex with the inverse of Jacc (Eq. 19), zero when Jacc is singular by
// construction or |det| is below det_eps times Hadamard's bound (the product of the row
// norms; Sec. 5),
// its position rows contracted with the explicit height dependence of the next vertex's
// surface coordinates.  A vertex after a diffuse one keeps its surface coordinates, so J's
// lower block there is zero (and Jacc singular from then on); with jac_noise it is
// eps [I 0], eps = +-1 from Philox stream 4 at that depth keyed by noise_seed (zero mean: the
// transport is unbiased over the noise).  Everything else is the exact form (its chain
// transport keeps the radiance terms); a connection's film position at a sliding vertex
// enters locally at its frozen surface coordinates.  One path per thread, fused passes.

namespace dual {
// Forward-mode dual numbers with N directional derivatives.
template <int N>
struct Dn {
  float v;
  float d[N];
};
template <int N>
__device__ __forceinline__ Dn<N> dn(float v) {
  Dn<N> r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = 0.0f;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fmaf(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, float s) {
  Dn<N> r;
  r.v = a.v * s;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  const float ib = 1.0f / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> dsqrt(const Dn<N>& a) {
  Dn<N> r;
  r.v = sqrtf(a.v);
  const float h = 0.5f / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
  return r;
}
template <int N>
struct V3 {
  Dn<N> x, y, z;
};
template <int N>
__device__ __forceinline__ V3<N> v3(float3 a) {
  return V3<N>{dn<N>(a.x), dn<N>(a.y), dn<N>(a.z)};
}
template <int N>
__device__ __forceinline__ V3<N> operator+(const V3<N>& a, const V3<N>& b) {
  return V3<N>{a.x + b.x, a.y + b.y, a.z + b.z};
}
template <int N>
__device__ __forceinline__ V3<N> operator-(const V3<N>& a, const V3<N>& b) {
  return V3<N>{a.x - b.x, a.y - b.y, a.z - b.z};
}
template <int N>
__device__ __forceinline__ V3<N> operator*(const V3<N>& a, const Dn<N>& s) {
  return V3<N>{a.x * s, a.y * s, a.z * s};
}
template <int N>
__device__ __forceinline__ V3<N> operator*(const V3<N>& a, float s) {
  return V3<N>{a.x * s, a.y * s, a.z * s};
}
template <int N>
__device__ __forceinline__ Dn<N> ddot(const V3<N>& a, const V3<N>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <int N>
__device__ __forceinline__ V3<N> dcross(const V3<N>& a, const V3<N>& b) {
  return V3<N>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Surface coordinates of the sliding vertex that follows specular vertex x_j (edges e1, e2)
// reached from x_p, along the reflected or refracted direction, on the plane (o_n, e1_n,
// e2_n) of the primitive it hits (Snell, reflection, ray-plane intersection).
template <int N>
__device__ __forceinline__ void spec_next(const V3<N>& xp, const V3<N>& xj, const V3<N>& e1, const V3<N>& e2,
                                          float ior, bool refl, const V3<N>& on, const V3<N>& e1n,
                                          const V3<N>& e2n, Dn<N> out[2]) {
  V3<N> d = xj - xp;
  const Dn<N> il = dn<N>(1.0f) / dsqrt(ddot(d, d));
  const V3<N> din = d * il;
  V3<N> n = dcross(e1, e2);
  n = n * (dn<N>(1.0f) / dsqrt(ddot(n, n)));
  const bool entering = ddot(din, n).v < 0.0f;
  const V3<N> ns = entering ? n : n * -1.0f;
  const float eta = entering ? 1.0f / ior : ior;
  const Dn<N> ci = ddot(din, ns) * -1.0f;
  V3<N> dout;
  if (refl) {
    dout = din + ns * (ci * 2.0f);
  } else {
    const Dn<N> ct = dsqrt(dn<N>(1.0f) - (dn<N>(1.0f) - ci * ci) * (eta * eta));
    dout = din * eta + ns * (ci * eta - ct);
  }
  const V3<N> m = dcross(e1n, e2n);
  const Dn<N> tau = ddot(on - xj, m) / ddot(dout, m);
  const V3<N> q = xj + dout * tau - on;
  const Dn<N> inn = dn<N>(1.0f) / ddot(m, m);
  out[0] = ddot(dcross(q, e2n), m) * inn;
  out[1] = ddot(dcross(e1n, q), m) * inn;
}
}  // namespace dual
using dual::Dn;
using dual::V3;

// A vertex of the path as the literal transport sees it: primitive (-1: the emitter),
// surface coordinates, and whether it is specular (with its branch).
struct LitV {
  int prim;
  float v0, v1;
  bool spec, refl;
};

// Point, edges and (for N = 9, slot base sb) height derivatives of vertex `a` on its
// primitive: a triangle vertex k of a height field moves along +y with its height, so
// o moves with h0, e1 with h1 - h0, e2 with h2 - h0 and the point with the barycentric
// weights.  The emitter and fixed primitives have no derivative.
template <int N>
__device__ __forceinline__ void lit_geom(const DevScene& S, const LitV& a, int sb, V3<N>& x, V3<N>& e1, V3<N>& e2,
                                         V3<N>& o, int hidx[3]) {
  float3 O, E1, E2;
  hidx[0] = hidx[1] = hidx[2] = -1;
  if (a.prim < 0) {
    O = S.lo; E1 = S.le1; E2 = S.le2;
  } else {
    const Prim P = load_prim(S, a.prim);
    O = P.o; E1 = P.e1; E2 = P.e2;
    const int4 ph = __ldg(S.prim_h + a.prim);
    hidx[0] = ph.x; hidx[1] = ph.y; hidx[2] = ph.z;
  }
  o = dual::v3<N>(O); e1 = dual::v3<N>(E1); e2 = dual::v3<N>(E2);
  x = dual::v3<N>(O + E1 * a.v0 + E2 * a.v1);
  if (N == 9 && sb >= 0) {
    const float w[3] = {1.0f - a.v0 - a.v1, a.v0, a.v1};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (hidx[k] < 0) continue;
      x.y.d[sb + k] = w[k];
      if (k == 0) { o.y.d[sb] = 1.0f; e1.y.d[sb] = -1.0f; e2.y.d[sb] = -1.0f; }
      if (k == 1) e1.y.d[sb + 1] = 1.0f;
      if (k == 2) e2.y.d[sb + 2] = 1.0f;
    }
  }
}

// Lower block of J for specular vertex b (reached from a), the next vertex on prim pn:
// d(v_next) / d(v_a, v_b), 2 x 4.
__device__ __forceinline__ void lit_jacobian(const DevScene& S, const LitV& a, const LitV& b, int pn, float J[2][4]) {
  V3<4> xa, e1a, e2a, oa, xb, e1b, e2b, ob, xn, e1n, e2n, on;
  int h[3];
  lit_geom<4>(S, a, -1, xa, e1a, e2a, oa, h);
  lit_geom<4>(S, b, -1, xb, e1b, e2b, ob, h);
  // directions: 0, 1 = v_a; 2, 3 = v_b
  xa.x.d[0] = e1a.x.v; xa.y.d[0] = e1a.y.v; xa.z.d[0] = e1a.z.v;
  xa.x.d[1] = e2a.x.v; xa.y.d[1] = e2a.y.v; xa.z.d[1] = e2a.z.v;
  xb.x.d[2] = e1b.x.v; xb.y.d[2] = e1b.y.v; xb.z.d[2] = e1b.z.v;
  xb.x.d[3] = e2b.x.v; xb.y.d[3] = e2b.y.v; xb.z.d[3] = e2b.z.v;
  const LitV nv = {pn, 0.0f, 0.0f, false, false};
  lit_geom<4>(S, nv, -1, xn, e1n, e2n, on, h);
  Dn<4> out[2];
  dual::spec_next<4>(xa, xb, e1b, e2b, __ldg(S.mat_ior + load_prim(S, b.prim).mat), b.refl, on, e1n, e2n, out);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) J[r][c] = out[r].d[c];
}

// The heights' share of the film-position transport at specular vertex b: a . v_next with the
// surface coordinates of a and b held, differentiated with respect to the heights of the
// three primitives involved.
__device__ __forceinline__ void lit_contract(const DevScene& S, const LitV& a, const LitV& b, int pn, float a0,
                                             float a1, float* dh) {
  if (!dh) return;
  V3<9> xa, e1a, e2a, oa, xb, e1b, e2b, ob, xn, e1n, e2n, on;
  int ha[3], hb[3], hn[3];
  lit_geom<9>(S, a, 0, xa, e1a, e2a, oa, ha);
  lit_geom<9>(S, b, 3, xb, e1b, e2b, ob, hb);
  const LitV nv = {pn, 0.0f, 0.0f, false, false};
  lit_geom<9>(S, nv, 6, xn, e1n, e2n, on, hn);
  Dn<9> out[2];
  dual::spec_next<9>(xa, xb, e1b, e2b, __ldg(S.mat_ior + load_prim(S, b.prim).mat), b.refl, on, e1n, e2n, out);
  const int* hs[3] = {ha, hb, hn};
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int hi = hs[t][k];
      const float g = fmaf(a0, out[0].d[3 * t + k], a1 * out[1].d[3 * t + k]);
      if (hi >= 0 && g != 0.0f) red_add(dh + hi, g);
    }
}

// m = A * m (4x4, row major)
__device__ __forceinline__ void m4_left(const float A[4][4], float m[4][4]) {
  float r[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) r[i][j] = A[i][0] * m[0][j] + A[i][1] * m[1][j] + A[i][2] * m[2][j] + A[i][3] * m[3][j];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) m[i][j] = r[i][j];
}
// y = x M^-1 for a row vector x (solve M^T y^T = x^T by Gauss-Jordan with partial
// pivoting); false when |det M| < eps times the product of M's row norms (Hadamard's bound
// on |det M|: the ratio is 1 for orthogonal rows and 0 for singular M, and a product of
// Jacobians that is singular in exact arithmetic keeps a ratio at the level of rounding).
__device__ __forceinline__ bool row_solve(const float M[4][4], const float x[4], float y[4], float eps) {
  float bound = 1.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    bound *= sqrtf(M[i][0] * M[i][0] + M[i][1] * M[i][1] + M[i][2] * M[i][2] + M[i][3] * M[i][3]);
  if (!(bound > 0.0f)) return false;
  float a[4][5];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) a[i][j] = M[j][i];
    a[i][4] = x[i];
  }
  float det = 1.0f;
  for (int c = 0; c < 4; ++c) {
    int pr = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabsf(a[r][c]) > fabsf(a[pr][c])) pr = r;
    if (pr != c) {
      for (int j = 0; j < 5; ++j) { const float t = a[pr][j]; a[pr][j] = a[c][j]; a[c][j] = t; }
      det = -det;
    }
    det *= a[c][c];
    if (a[c][c] == 0.0f) return false;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const float f = a[r][c] / a[c][c];
      for (int j = c; j < 5; ++j) a[r][j] -= f * a[c][j];
    }
  }
  if (!(fabsf(det) >= eps * bound)) return false;
#pragma unroll
  for (int i = 0; i < 4; ++i) y[i] = a[i][4] / a[i][i];
  return true;
}

// Accumulated Jacobian after vertex k of a path: J of vertex k-1 applied (its lower block
// from lit_jacobian when specular; zero, or the noise block, when diffuse).  `singular`
// records that a zero block has entered the product, which is then singular by construction
// (rounding would hide that from the determinant).
__device__ __forceinline__ void lit_advance(const DevScene& S, const KParams& kp, uint64_t n, int k, const LitV& a,
                                            const LitV& b, int pn, float Jacc[4][4], bool& singular) {
  float J[4][4] = {{0, 0, 1, 0}, {0, 0, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}};
  if (b.spec) {
    float L2[2][4];
    lit_jacobian(S, a, b, pn, L2);
    for (int c = 0; c < 4; ++c) { J[2][c] = L2[0][c]; J[3][c] = L2[1][c]; }
  } else if (kp.jac_noise) {
    const float eps = rand4(kp.noise_seed, n, (uint32_t)k, 4).x < 0.5f ? -1.0f : 1.0f;
    J[2][0] = eps;
    J[3][1] = eps;
  } else {
    singular = true;
  }
  m4_left(J, Jacc);
}

// Position row of a connection at vertex x on prim (edges e1, e2): dL/du du/dv.
__device__ __forceinline__ float2 lit_row(const DevScene& S, float3 x, const Prim& P, float2 q) {
  const float3 d = x - S.cpos;
  const float zc = dot(d, S.cf), pr = dot(d, S.cr), pu = dot(d, S.cu);
  const float ax = 0.5f * (float)S.W / (S.tanx * zc), ay = -0.5f * (float)S.H / (S.tany * zc);
  const float3 g = (S.cr - S.cf * (pr / zc)) * (q.x * ax) + (S.cu - S.cf * (pu / zc)) * (q.y * ay);
  return make_float2(dot(g, P.e1), dot(g, P.e2));
}

// Paper-literal attached LRB-3 (Eq. 4-7, Eq. 18-19, Sec. 5), one path per thread: pass 2
// accumulates the 4x4 Jacobians forward and sums A_pos; pass 3 projects the remainder back
// through the guarded inverse of the accumulated Jacobian at each specular vertex.
__global__ void __launch_bounds__(128) k_lrb3_literal(DevScene S, KParams kp, const float* __restrict__ dI,
                                                      GradPtrs g0) {
  extern __shared__ float sgrad[];
  const Sink sink = sink_begin(kp, g0, sgrad);
  GradPtrs g = g0;
  g.d_albedo = sink.alb;
  g.d_heights = sink.h;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    if (kp.mask && !kp.mask[p]) continue;
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    const float4 r0 = rand4(kp.seed, n, 0);
    const LitV em = {-1, r0.x, r0.y, false, false};
    // ---- pass 2: delta_total (Eq. 14), validity, and A_pos (Eq. 18)
    Walk w;
    float3 x0;
    walk_start(S, kp.seed, n, Le, w, x0);
    float3 dtot = f3(0, 0, 0);
    uint64_t valid = 0;
    float Jacc[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    float Apos[4] = {0, 0, 0, 0};
    LitV pa = em, pb = em;  // vertices k-2 and k-1
    bool singular = false;
    for (int k = 0; k < kp.max_depth; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) break;
      const LitV cur = {v.prim, v.b1, v.b2, !v.diffuse, false};
      if (k >= 1) lit_advance(S, kp, n, k, pa, pb, v.prim, Jacc, singular);
      const float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr);
        const Conn c = connect(S, v.x, ns, v.prim);
        if (c.valid) {
          valid |= 1ull << k;
          const float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
          float2 q;
          dtot = dtot + mul(adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, &q, kp.filter), L);
          const float2 a = lit_row(S, v.x, v.P, q);
          for (int j = 0; j < 4; ++j) Apos[j] += a.x * Jacc[2][j] + a.y * Jacc[3][j];
        }
      }
      const bool refl = walk_scatter(S, w, v, ns, rho, r);
      walk_rr(kp, n, k, w);
      pa = pb;
      pb = cur;
      pb.refl = refl;
    }
    if (!valid) continue;
    gLe = gLe + f3(dtot.x / Le.x, dtot.y / Le.y, dtot.z / Le.z);  // emitted factor, weight delta_total
    // ---- pass 3: the exact form's terms with each film position local, and the transport
    walk_start(S, kp.seed, n, Le, w, x0);
    float3 rem = dtot;
    PendAdj pv;
    pend_init(pv, -1, -1, 0.0f, 0.0f, x0, S.ln);
    ChainInfo chain;
    chain.ka = -1;
    ChainCache cc;
    cc.reset();
    const int last = 63 - __clzll((long long)valid);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) Jacc[i][j] = i == j ? 1.0f : 0.0f;
    float Arem[4] = {Apos[0], Apos[1], Apos[2], Apos[3]};
    pa = em;
    pb = em;
    singular = false;
    for (int k = 0; k <= last; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) { set_err(S, ERR_BOUNDS); break; }  // the replay must reach `last`
      const LitV cur = {v.prim, v.b1, v.b2, !v.diffuse, false};
      if (k >= 1) {
        lit_advance(S, kp, n, k, pa, pb, v.prim, Jacc, singular);
        if (pb.spec && !singular) {
          // Eq. 19: the remainder (connections from vertex k on) in the frame of p_k
          float aloc[4];
          if (row_solve(Jacc, Arem, aloc, kp.det_eps)) lit_contract(S, pa, pb, v.prim, aloc[2], aloc[3], g.d_heights);
        }
      }
      const float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      att_enter<true>(S, kp, n, k, v, hsum(rem), hsum(rem), pv, chain, g.d_heights, &cc);
      const bool rec_chain = !v.diffuse;
      if (rec_chain) cc.record(chain, k, v, w.dir);
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        TexFoot foot;
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, &foot);
        float3 wsplat = f3(0, 0, 0);
        if ((valid >> k) & 1ull) {
          const Conn c = connect_pre(S, v.x, ns);
          const float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
          float2 q;
          const float3 Lb = adjoint_read_f(dI, S.W, S.H, c.ux, c.uy, L, &q, kp.filter);
          const float3 P = mul(Lb, L);
          wsplat = P;      // Eq. 15
          rem = rem - P;   // Eq. 16
          if (v.attached) {
            conn_adjoint(S, v.x, v.nraw, hsum(P), q, pv.gx, pv.gn);
          } else {
            // radiance terms through the chain; the film position at its own coordinates
            conn_adjoint(S, v.x, v.nraw, hsum(P), make_float2(0.0f, 0.0f), pv.gx, pv.gn);
            float3 gxq = f3(0, 0, 0), gnq = f3(0, 0, 0);
            conn_adjoint(S, v.x, v.nraw, 0.0f, q, gxq, gnq);
            scatter_heights(S, g.d_heights, v.prim, v.b1, v.b2, gxq, f3(0, 0, 0));
          }
          const float2 a = lit_row(S, v.x, v.P, q);
          for (int j = 0; j < 4; ++j) Arem[j] -= a.x * Jacc[2][j] + a.y * Jacc[3][j];
        }
        scatter_albedo(S, g.d_albedo, foot, wsplat + rem, rho);  // + scattering factor (Eq. 17)
        if (!v.attached) pv.gx = pv.gx + tex_pos_adjoint(kp.albedo, v.m, v.P, v.b1, v.b2, wsplat + rem, rho);
      }
      const bool refl = walk_scatter(S, w, v, ns, rho, r);
      if (rec_chain) cc.record_branch(refl);
      walk_rr(kp, n, k, w);
      pa = pb;
      pb = cur;
      pb.refl = refl;
    }
    pend_flush<true>(S, kp, n, pv, g.d_heights, &cc);
  }
  sink_end(kp, g0, sgrad);
  block_add3(g0.d_Le, gLe);
}

// ======================================================================= film
__global__ void k_film_l2(const float* __restrict__ I, const float* __restrict__ T, int64_t n, float* dI,
                          float* loss) {
  float s = 0.0f;
  const float inv = 1.0f / (float)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float d = I[i] - T[i];
    dI[i] = 2.0f * d * inv;
    s += d * d * inv;
  }
  __shared__ float sh[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = (blockDim.x + 31) >> 5;
    float v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0f;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(loss, v);
  }
}

// ======================================================================= launchers
// Launch a path kernel over `work` paths: at most L.blocks_per_sm blocks per SM, and no more
// than the kernel's occupancy lets an SM hold at once.  The path kernels split their paths
// statically over the warps of the grid, so a grid of more blocks than fit would run in
// waves whose last one leaves SMs idle.
template <typename... P, typename... A>
static void launch_paths(void (*kern)(P...), const LaunchCfg& L, int64_t work, size_t smem, cudaStream_t st,
                         A&&... args) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = L.blocks_per_sm, occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, L.block, smem) == cudaSuccess && occ > 0 &&
      occ < per_sm)
    per_sm = occ;
  int64_t grid = (work + L.block - 1) / L.block;
  const int64_t cap = (int64_t)L.sms * per_sm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, L.block, smem, st>>>(std::forward<A>(args)...);
}

cudaError_t launch_refit(const RefitArgs& a, cudaStream_t st) {
  if (a.n_prims > 0 && a.heights) {
    k_update_tris<<<(a.n_prims + 255) / 256, 256, 0, st>>>(a.prim, a.prim_h, a.tri_base, a.heights, a.n_prims);
  }
  if (a.n_nodes > 0) {
    int threads = a.n_nodes * 32;
    k_refit_nodes<<<(threads + 255) / 256, 256, 0, st>>>(a.node, a.range, a.prim, a.n_nodes);
    if (a.n_big > 0) k_refit_big<<<a.n_big, 256, 0, st>>>(a.node, a.range, a.big, a.prim);
  }
  if (a.n_wnodes[0] > 0) {
    const int t = a.n_wnodes[0] * 4;
    k_refit_wide<4><<<(t + 255) / 256, 256, 0, st>>>(a.wnode[0], a.wmap[0], a.node, a.n_wnodes[0]);
  }
  if (a.n_wnodes[1] > 0) {
    const int t = a.n_wnodes[1] * 8;
    k_refit_wide<8><<<(t + 255) / 256, 256, 0, st>>>(a.wnode[1], a.wmap[1], a.node, a.n_wnodes[1]);
  }
  return cudaGetLastError();
}

cudaError_t launch_primal(const DevScene& S, const KParams& kp, int est, float* image, void* aux, const LaunchCfg& L,
                          cudaStream_t st) {
  const size_t smem = (est == 1 && kp.mlp) ? ((sizeof(MlpSmem) + 15) & ~size_t(15)) +
                                                sizeof(__nv_bfloat16) * 32 * kMlpIn * (L.block / 32) +
                                                sizeof(float) * 2 * kMlpIn * L.block
                                          : 0;
  switch (est) {
    case 0:
      if (kp.census) launch_paths(k_primal_census, L, kp.n_paths, 0, st, S, kp, image, aux);
      else if (S.atomics == 2) launch_paths(k_primal_agg, L, kp.n_paths, 0, st, S, kp, image, aux);
      else launch_paths(k_primal<0>, L, kp.n_paths, 0, st, S, kp, image, aux);
      break;
    case 1:
      if (kp.mlp) launch_paths(k_primal_learned, L, kp.n_paths, smem, st, S, kp, image, aux);
      else launch_paths(k_primal<1>, L, kp.n_paths, 0, st, S, kp, image, aux);
      break;
    case 2: launch_paths(k_primal<2>, L, kp.n_paths, 0, st, S, kp, image, aux); break;
    default: launch_paths(k_primal<3>, L, kp.n_paths, 0, st, S, kp, image, aux); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_lrb3(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,
                        const GradPtrs& g, void* state, bool mask_ready, const LaunchCfg& L, cudaStream_t st) {
  const size_t smem = kp.priv_n > 0 ? sizeof(float) * (size_t)kp.priv_n : 0;
  if (state) {
    float4* xrec = (float4*)state;
    uint32_t* xhi = (uint32_t*)((char*)state + lrb3_state_split(kp.n_paths));
    KParams k2 = kp;
    k2.priv_n = 0;  // pass 2 writes no albedo or height gradients
    GradPtrs g3 = g;
    g3.d_Le = nullptr;  // pass 3 writes no emitted-radiance gradient
    if (mask_ready && kp.conn1)
      k_lrb3_single<<<L.sms * 4, 256, 0, st>>>(S, k2, dI, g, xrec, xhi);
    if (kp.census) {
      if (mask_ready) launch_paths(k_lrb3_p2<true, true>, L, kp.n_paths, 0, st, S, k2, dI, g, xrec, xhi);
      else launch_paths(k_lrb3_p2<true, false>, L, kp.n_paths, 0, st, S, k2, dI, g, xrec, xhi);
    } else {
      if (mask_ready) launch_paths(k_lrb3_p2<false, true>, L, kp.n_paths, 0, st, S, k2, dI, g, xrec, xhi);
      else launch_paths(k_lrb3_p2<false, false>, L, kp.n_paths, 0, st, S, k2, dI, g, xrec, xhi);
    }
    if (kp.census) {
      if (att && chains) launch_paths(k_lrb3_p3<true, true, true>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
      else if (att) launch_paths(k_lrb3_p3<true, true, false>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
      else launch_paths(k_lrb3_p3<false, true, false>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
    } else {
      if (att && chains) launch_paths(k_lrb3_p3<true, false, true>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
      else if (att) launch_paths(k_lrb3_p3<true, false, false>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
      else launch_paths(k_lrb3_p3<false, false, false>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
    }
    return cudaGetLastError();
  }
  if (kp.census) {
    if (att && chains) launch_paths(k_lrb3<true, true, true>, L, kp.n_paths, smem, st, S, kp, dI, g);
    else if (att) launch_paths(k_lrb3<true, true, false>, L, kp.n_paths, smem, st, S, kp, dI, g);
    else launch_paths(k_lrb3<false, true, false>, L, kp.n_paths, smem, st, S, kp, dI, g);
  } else {
    if (att && chains) launch_paths(k_lrb3<true, false, true>, L, kp.n_paths, smem, st, S, kp, dI, g);
    else if (att) launch_paths(k_lrb3<true, false, false>, L, kp.n_paths, smem, st, S, kp, dI, g);
    else launch_paths(k_lrb3<false, false, false>, L, kp.n_paths, smem, st, S, kp, dI, g);
  }
  return cudaGetLastError();
}

cudaError_t launch_reslrb(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,
                          const void* rec, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  const size_t smem = kp.priv_n > 0 ? sizeof(float) * (size_t)kp.priv_n : 0;
  if (att && chains) launch_paths(k_reslrb<true, true>, L, kp.n_paths, smem, st, S, kp, dI, (const float4*)rec, g);
  else if (att) launch_paths(k_reslrb<true, false>, L, kp.n_paths, smem, st, S, kp, dI, (const float4*)rec, g);
  else launch_paths(k_reslrb<false, false>, L, kp.n_paths, smem, st, S, kp, dI, (const float4*)rec, g);
  return cudaGetLastError();
}

cudaError_t launch_naive(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,
                         const void* ws, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  const size_t smem = kp.priv_n > 0 ? sizeof(float) * (size_t)kp.priv_n : 0;
  if (att && chains) launch_paths(k_naive<true, true>, L, kp.n_paths, smem, st, S, kp, dI, ws, g);
  else if (att) launch_paths(k_naive<true, false>, L, kp.n_paths, smem, st, S, kp, dI, ws, g);
  else launch_paths(k_naive<false, false>, L, kp.n_paths, smem, st, S, kp, dI, ws, g);
  return cudaGetLastError();
}

cudaError_t launch_lrb2(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI, void* buf,
                        const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  launch_paths(k_lrb2_reduce, L, kp.n_paths, 0, st, S, kp, dI, buf, g.d_Le);
  float4* xrec = (float4*)buf;
  uint32_t* xhi = (uint32_t*)((char*)buf + lrb3_state_split(kp.n_paths));
  const size_t smem = kp.priv_n > 0 ? sizeof(float) * (size_t)kp.priv_n : 0;
  GradPtrs g3 = g;
  g3.d_Le = nullptr;  // added by the reduction
  if (att && chains) launch_paths(k_lrb3_p3<true, false, true>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
  else if (att) launch_paths(k_lrb3_p3<true, false, false>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
  else launch_paths(k_lrb3_p3<false, false, false>, L, kp.n_paths, smem, st, S, kp, dI, g3, xrec, xhi);
  return cudaGetLastError();
}

cudaError_t launch_collect(const DevScene& S, const KParams& kp, const float* dI, float tfloor, float* feats,
                           float* targets, int64_t cap, unsigned long long* count, const LaunchCfg& L, cudaStream_t st) {
  launch_paths(k_collect, L, kp.n_paths, 0, st, S, kp, dI, tfloor, feats, targets, cap, count);
  return cudaGetLastError();
}

template <class K>
static int occupancy_of(K kern, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, 0) != cudaSuccess) return 0;
  return n;
}

// Kernel of a batched pass (the same selection as launch_batch).
#define LT_BATCH_DISPATCH(CALL)                                                  \
  switch (pass) {                                                                \
    case BPASS_PRIMAL: CALL(k_primal_batch<0>); break;                           \
    case BPASS_PRIMAL_RES: CALL(k_primal_batch<1>); break;                       \
    case BPASS_LRB3:                                                             \
      if (att && chains) CALL((k_lrb3_batch<true, true>));                       \
      else if (att) CALL((k_lrb3_batch<true, false>));                           \
      else CALL((k_lrb3_batch<false, false>));                                   \
      break;                                                                     \
    case BPASS_LRB3_P2: CALL(k_lrb3_p2_batch<false>); break;                    \
    case BPASS_LRB3_P2_MASK: CALL(k_lrb3_p2_batch<true>); break;                \
    case BPASS_LRB3_P3:                                                          \
      if (att && chains) CALL((k_lrb3_p3_batch<true, true>));                    \
      else if (att) CALL((k_lrb3_p3_batch<true, false>));                        \
      else CALL((k_lrb3_p3_batch<false, false>));                                \
      break;                                                                     \
    default:                                                                     \
      if (att && chains) CALL((k_reslrb_batch<true, true>));                     \
      else if (att) CALL((k_reslrb_batch<true, false>));                         \
      else CALL((k_reslrb_batch<false, false>));                                 \
      break;                                                                     \
  }

cudaError_t launch_batch(int pass, bool att, bool chains, const BatchArgs& a, int block, int grid, cudaStream_t st) {
#define LT_LAUNCH_ONE(K) K<<<grid, block, 0, st>>>(a)
  LT_BATCH_DISPATCH(LT_LAUNCH_ONE)
#undef LT_LAUNCH_ONE
  return cudaGetLastError();
}

cudaError_t launch_batch_spans(bool att, bool chains, const BatchJob* jobs, const BatchSpan* spans, int n_spans,
                               unsigned long long* ticket, int block, int grid, size_t smem, cudaStream_t st) {
  if (att && chains) k_lrb3_p3_spans<true, true><<<grid, block, smem, st>>>(jobs, spans, n_spans, ticket);
  else if (att) k_lrb3_p3_spans<true, false><<<grid, block, smem, st>>>(jobs, spans, n_spans, ticket);
  else k_lrb3_p3_spans<false, false><<<grid, block, smem, st>>>(jobs, spans, n_spans, ticket);
  return cudaGetLastError();
}

int batch_spans_occupancy(bool att, bool chains, int block, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (att && chains) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lrb3_p3_spans<true, true>, block, smem);
  else if (att) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lrb3_p3_spans<true, false>, block, smem);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lrb3_p3_spans<false, false>, block, smem);
  return e == cudaSuccess ? n : 0;
}

int batch_occupancy(int pass, bool att, bool chains, int block) {
  int n = 0;
#define LT_OCC_ONE(K) n = occupancy_of(K, block)
  LT_BATCH_DISPATCH(LT_OCC_ONE)
#undef LT_OCC_ONE
  return n;
}
#undef LT_BATCH_DISPATCH

cudaError_t launch_lrb3_literal(const DevScene& S, const KParams& kp, const float* dI, const GradPtrs& g,
                                const LaunchCfg& L, cudaStream_t st) {
  const size_t smem = kp.priv_n > 0 ? sizeof(float) * (size_t)kp.priv_n : 0;
  launch_paths(k_lrb3_literal, L, kp.n_paths, smem, st, S, kp, dI, g);
  return cudaGetLastError();
}

cudaError_t launch_bidir(const DevScene& S, const KParams& kp, const BidirArgs& ba, bool backward, float* image,
                         const float* dI, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  const size_t smem = backward && kp.priv_n > 0 ? sizeof(float) * (size_t)kp.priv_n : 0;
  if (kp.n_paths > 0) {
    if (backward) launch_paths(k_bidir_light<true>, L, kp.n_paths, smem, st, S, kp, ba, image, dI, g);
    else launch_paths(k_bidir_light<false>, L, kp.n_paths, smem, st, S, kp, ba, image, dI, g);
  }
  if (ba.n_cam > 0) {
    if (backward) launch_paths(k_bidir_cam<true>, L, ba.n_cam, smem, st, S, kp, ba, image, dI, g);
    else launch_paths(k_bidir_cam<false>, L, ba.n_cam, smem, st, S, kp, ba, image, dI, g);
  }
  return cudaGetLastError();
}

cudaError_t launch_film_l2(const float* I, const float* T, int64_t n, float* dI, float* loss, int sms,
                           cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4 * sms) blocks = 4 * sms;
  if (blocks < 1) blocks = 1;
  k_film_l2<<<(int)blocks, 256, 0, st>>>(I, T, n, dI, loss);
  return cudaGetLastError();
}

}  // namespace LT_KNS
}  // namespace lt
