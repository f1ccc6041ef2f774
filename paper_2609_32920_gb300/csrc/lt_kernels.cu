// lt_kernels.cu -- CUDA kernels of the light tracer and its adjoints (sm_103a).
//
// One thread carries one light path through all of its vertices (grid-stride over the
// path range, persistent grid sized to the SM count).  Every pass regenerates the path
// from its Philox counter; nothing per vertex is stored except by the naive baseline.
#include <cuda_runtime.h>

#include "lt_device.cuh"
#include "lt_launch.h"

namespace lt {

// ======================================================================= refit
// Triangle geometry from base vertex positions plus heights (y), leaf order.
__global__ void k_update_tris(float4* prim, const int4* prim_h, const float4* tri_base, const float* heights,
                              int n_prims) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_prims) return;
  int4 ph = prim_h[i];
  if (ph.x < 0 && ph.y < 0 && ph.z < 0) return;
  float3 v0 = xyz(tri_base[3 * i]), v1 = xyz(tri_base[3 * i + 1]), v2 = xyz(tri_base[3 * i + 2]);
  if (ph.x >= 0) v0.y += heights[ph.x];
  if (ph.y >= 0) v1.y += heights[ph.y];
  if (ph.z >= 0) v2.y += heights[ph.z];
  float4 a = prim[3 * i], b = prim[3 * i + 1], c = prim[3 * i + 2];
  float3 e1 = v1 - v0, e2 = v2 - v0;
  prim[3 * i] = make_float4(v0.x, v0.y, v0.z, a.w);
  prim[3 * i + 1] = make_float4(e1.x, e1.y, e1.z, b.w);
  prim[3 * i + 2] = make_float4(e2.x, e2.y, e2.z, c.w);
}

// One warp per BVH node: the node's subtree covers the contiguous leaf-order primitive
// range [range.x, range.y), so its bounds are a reduction over that range.
__global__ void k_refit_nodes(float4* node, const int2* range, const float4* prim, int n_nodes) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n_nodes) return;
  int2 r = range[w];
  float3 lo = f3(3e38f, 3e38f, 3e38f), hi = f3(-3e38f, -3e38f, -3e38f);
  for (int k = r.x + lane; k < r.y; k += 32) {
    float3 o = xyz(prim[3 * k]), e1 = xyz(prim[3 * k + 1]), e2 = xyz(prim[3 * k + 2]);
    bool tri = __float_as_int(prim[3 * k + 2].w) != 0;
    float3 p[4] = {o, o + e1, o + e2, o + e1 + e2};
    int np = tri ? 3 : 4;
    for (int j = 0; j < np; ++j) {
      lo = f3(fminf(lo.x, p[j].x), fminf(lo.y, p[j].y), fminf(lo.z, p[j].z));
      hi = f3(fmaxf(hi.x, p[j].x), fmaxf(hi.y, p[j].y), fmaxf(hi.z, p[j].z));
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, off));
    lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, off));
    lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, off));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, off));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, off));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, off));
  }
  if (lane == 0) {
    // conservative padding for FP32 rounding of the stored primitive edges
    float3 pad = f3(1e-6f * fmaxf(1.0f, fmaxf(fabsf(lo.x), fabsf(hi.x))),
                    1e-6f * fmaxf(1.0f, fmaxf(fabsf(lo.y), fabsf(hi.y))),
                    1e-6f * fmaxf(1.0f, fmaxf(fabsf(lo.z), fabsf(hi.z))));
    float4 a = node[2 * w], b = node[2 * w + 1];
    node[2 * w] = make_float4(lo.x - pad.x, lo.y - pad.y, lo.z - pad.z, a.w);
    node[2 * w + 1] = make_float4(hi.x + pad.x, hi.y + pad.y, hi.z + pad.z, b.w);
  }
}

// ======================================================================= path walk
// State of a light path between vertices.
struct Walk {
  float3 org, dir;
  int skip;
  int prev_kind;
  float3 beta;
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

// Returns false when the path ends (miss or emitter hit).
__device__ __forceinline__ bool walk_hit(const DevScene& S, const Walk& w, Vtx& v) {
  HitRec h = trace_closest(S, w.org, w.dir, w.skip);
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

// Albedo gradient at one diffuse vertex: weight (per channel) / rho times the bilinear
// texel weights (d rho / d texel).
__device__ __forceinline__ void scatter_albedo(float* g, const TexFoot& f, float3 wt, float3 rho) {
  if (!g) return;
  float3 a = f3(wt.x / rho.x, wt.y / rho.y, wt.z / rho.z);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (f.w[k] == 0.0f) continue;
    atomicAdd(g + f.idx[k] + 0, a.x * f.w[k]);
    atomicAdd(g + f.idx[k] + 1, a.y * f.w[k]);
    atomicAdd(g + f.idx[k] + 2, a.z * f.w[k]);
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
  if (ph.x >= 0) atomicAdd(dh + ph.x, h0);
  if (ph.y >= 0) atomicAdd(dh + ph.y, h1);
  if (ph.z >= 0) atomicAdd(dh + ph.z, h2);
}

// Adjoint of an attached vertex accumulated until all of its terms are known.
struct PendAdj {
  int prim;
  float b1, b2;
  float3 x, nr, gx, gn;
};

// ======================================================================= primal
template <int EST>
__global__ void __launch_bounds__(128) k_primal(DevScene S, KParams kp, float* __restrict__ image, void* aux) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    const bool active = !kp.mask || kp.mask[p];
    Walk w;
    float3 x0;
    walk_start(S, kp.seed, n, Le, w, x0);
    uint32_t hash = 2166136261u;
    int nconn = 0, depth = 0;
    // reservoir (capacity one)
    float Om = 0.0f, wR = 0.0f, Rux = 0.0f, Ruy = 0.0f;
    float3 LR = f3(0, 0, 0);
    int R = -1;
    for (int k = 0; k < kp.max_depth; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) break;
      depth = k + 1;
      float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      Conn c;
      c.valid = false; c.ux = c.uy = 0.0f;
      float3 L = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        c = connect(S, v.x, ns, v.prim);
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, nullptr);
        if (c.valid) {
          ++nconn;
          L = mul(w.beta, rho) * (c.geo * kp.inv_n);
          if (active) {
            if (EST == 1) {
              float om = luminance(L);
              if (om > 0.0f) {
                Om += om;
                if (r.w < om / Om) { R = k; wR = om; LR = L; Rux = c.ux; Ruy = c.uy; }
              }
            } else {
              splat(image, S.W, S.H, c.ux, c.uy, L);
            }
          }
        }
      }
      bool refl = walk_scatter(S, w, v, ns, rho, r);
      fnv(hash, (uint32_t)v.P.orig);
      fnv(hash, vtx_flags(v, refl, c.valid));
      if (EST == 2 && active) {
        // naive-AD tape: [depth][path] records of two float4
        float4* tape = (float4*)((char*)aux + kp.tape_offset) + 2 * ((size_t)k * kp.n_paths + p);
        uint32_t fl = vtx_flags(v, refl, c.valid);
        tape[0] = make_float4(__int_as_float(v.prim | (int)(fl << 24)), v.b1, v.b2, c.ux);
        tape[1] = make_float4(L.x, L.y, L.z, c.uy);
      }
    }
    if (EST == 1) {
      float4* rec = (float4*)aux + 2 * p;
      float wgt = R >= 0 ? Om / wR : 0.0f;
      float3 Sh = LR * wgt;
      if (active && R >= 0) splat(image, S.W, S.H, Rux, Ruy, Sh);
      rec[0] = make_float4(__int_as_float(active ? R : -1), wgt, Rux, Ruy);
      rec[1] = make_float4(Sh.x, Sh.y, Sh.z, 0.0f);
    }
    if (EST == 2) ((int*)aux)[p] = active ? depth : 0;
    if (kp.hash) kp.hash[p] = hash;
    if (kp.dbg) ((float4*)kp.dbg)[p] = make_float4((float)nconn, (float)depth, 0.0f, 0.0f);
  }
}

// ======================================================================= LRB-3-pass
// Pass 2 (accumulate delta_total, Eq. 14) and pass 3 (backpropagate, Eq. 15-17) fused per
// path: both replay the path from its counter; the connection-validity bits found in
// pass 2 are kept in a register mask so pass 3 does not re-test visibility.
template <bool ATT>
__global__ void __launch_bounds__(128) k_lrb3(DevScene S, KParams kp, const float* __restrict__ dI, GradPtrs g) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    if (kp.mask && !kp.mask[p]) continue;
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    // ---------------- pass 2
    Walk w;
    float3 x0;
    walk_start(S, kp.seed, n, Le, w, x0);
    float3 dtot = f3(0, 0, 0);
    uint64_t valid = 0;
    int nconn = 0;
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
          valid |= 1ull << k;
          ++nconn;
          float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
          float3 Lb = adjoint_read(dI, S.W, S.H, c.ux, c.uy, L, nullptr);
          dtot = dtot + mul(Lb, L);
        }
      }
      walk_scatter(S, w, v, ns, rho, r);
    }
    if (kp.dbg) ((float4*)kp.dbg)[p] = make_float4(dtot.x, dtot.y, dtot.z, (float)nconn);
    // ---------------- pass 3
    gLe = gLe + f3(dtot.x / Le.x, dtot.y / Le.y, dtot.z / Le.z);
    if (valid == 0) continue;
    float3 rem = dtot;
    walk_start(S, kp.seed, n, Le, w, x0);
    PendAdj pv;
    pv.prim = -1; pv.x = x0; pv.nr = S.ln; pv.gx = pv.gn = f3(0, 0, 0); pv.b1 = pv.b2 = 0.0f;
    const int last = 63 - __clzll((long long)valid);
    for (int k = 0; k <= last; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) break;
      float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        TexFoot foot;
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, &foot);
        PendAdj cur;
        cur.prim = v.prim; cur.b1 = v.b1; cur.b2 = v.b2; cur.x = v.x; cur.nr = v.nraw;
        cur.gx = cur.gn = f3(0, 0, 0);
        if (ATT) {
          // attached segment weight: every connection from here on carries it
          seg_adjoint(pv.x, pv.nr, v.x, v.nraw, hsum(rem), pv.gx, pv.gn, cur.gx, cur.gn);
          scatter_heights(S, g.d_heights, pv.prim, pv.b1, pv.b2, pv.gx, pv.gn);
        }
        float3 wsplat = f3(0, 0, 0);
        if ((valid >> k) & 1ull) {
          Conn c = connect(S, v.x, ns, v.prim, false);
          float3 L = mul(w.beta, rho) * (c.geo * kp.inv_n);
          float2 q;
          float3 Lb = adjoint_read(dI, S.W, S.H, c.ux, c.uy, L, ATT ? &q : nullptr);
          float3 P = mul(Lb, L);
          wsplat = P;           // splat factor rho_k / pi (Eq. 15)
          rem = rem - P;        // Eq. 16
          if (ATT) conn_adjoint(S, v.x, v.nraw, hsum(P), q, cur.gx, cur.gn);
        }
        scatter_albedo(g.d_albedo, foot, wsplat + rem, rho);  // + scattering factor rho_k (Eq. 17)
        pv = cur;
      }
      walk_scatter(S, w, v, ns, rho, r);
    }
    if (ATT) scatter_heights(S, g.d_heights, pv.prim, pv.b1, pv.b2, pv.gx, pv.gn);
  }
  block_add3(g.d_Le, gLe);
}

// ======================================================================= ResLRB backward
// Replay to the selected vertex R and apply the log-derivative identity with weight
// Lbar_R * S to every factor of L_R (Eq. 11); attached adds the positional channel.
template <bool ATT>
__global__ void __launch_bounds__(128) k_reslrb(DevScene S, KParams kp, const float* __restrict__ dI,
                                                const float4* __restrict__ rec, GradPtrs g) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float3 Le = f3(kp.Le[0], kp.Le[1], kp.Le[2]);
  float3 gLe = f3(0, 0, 0);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < kp.n_paths; p += stride) {
    if (kp.mask && !kp.mask[p]) continue;
    float4 r0 = rec[2 * p], r1 = rec[2 * p + 1];
    int R = __float_as_int(r0.x);
    if (R < 0) continue;
    if (R >= kp.max_depth) { set_err(S, ERR_BOUNDS); continue; }
    const uint64_t n = (uint64_t)(kp.path_offset + p);
    float3 Sh = f3(r1.x, r1.y, r1.z);
    float2 q;
    float3 Lb = adjoint_read(dI, S.W, S.H, r0.z, r0.w, Sh, ATT ? &q : nullptr);
    float3 P = mul(Lb, Sh);
    float lam = hsum(P);
    gLe = gLe + f3(P.x / Le.x, P.y / Le.y, P.z / Le.z);
    Walk w;
    float3 x0;
    walk_start(S, kp.seed, n, Le, w, x0);
    PendAdj pv;
    pv.prim = -1; pv.x = x0; pv.nr = S.ln; pv.gx = pv.gn = f3(0, 0, 0); pv.b1 = pv.b2 = 0.0f;
    for (int k = 0; k <= R; ++k) {
      Vtx v;
      if (!walk_hit(S, w, v)) { set_err(S, ERR_BOUNDS); break; }
      float4 r = rand4(kp.seed, n, (uint32_t)(k + 1));
      float3 ns = f3(0, 0, 0), rho = f3(0, 0, 0);
      if (v.diffuse) {
        ns = dot(v.nraw, w.dir) < 0.0f ? v.n : -v.n;
        TexFoot foot;
        rho = tex_lookup(kp.albedo, v.m, v.b1, v.b2, &foot);
        scatter_albedo(g.d_albedo, foot, P, rho);
        PendAdj cur;
        cur.prim = v.prim; cur.b1 = v.b1; cur.b2 = v.b2; cur.x = v.x; cur.nr = v.nraw;
        cur.gx = cur.gn = f3(0, 0, 0);
        if (ATT) {
          seg_adjoint(pv.x, pv.nr, v.x, v.nraw, lam, pv.gx, pv.gn, cur.gx, cur.gn);
          scatter_heights(S, g.d_heights, pv.prim, pv.b1, pv.b2, pv.gx, pv.gn);
          if (k == R) conn_adjoint(S, v.x, v.nraw, lam, q, cur.gx, cur.gn);
        }
        pv = cur;
      }
      walk_scatter(S, w, v, ns, rho, r);
    }
    if (ATT) scatter_heights(S, g.d_heights, pv.prim, pv.b1, pv.b2, pv.gx, pv.gn);
  }
  block_add3(g.d_Le, gLe);
}

// ======================================================================= naive reverse
// Reverse sweep over the per-vertex tape: suffix sums of Lbar_i L_i replace the replay.
template <bool ATT>
__global__ void __launch_bounds__(128) k_naive(DevScene S, KParams kp, const float* __restrict__ dI,
                                               const void* __restrict__ ws, GradPtrs g) {
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
    for (int k = K - 1; k >= 0; --k) {
      float4 t0 = tape[2 * ((size_t)k * kp.n_paths + p)], t1 = tape[2 * ((size_t)k * kp.n_paths + p) + 1];
      int pk = __float_as_int(t0.x);
      int prim = pk & 0xffffff;
      uint32_t fl = (uint32_t)pk >> 24;
      if (prim >= S.n_prims) { set_err(S, ERR_BOUNDS); break; }
      if ((fl & 3u) != K_DIFFUSE) continue;  // dielectric vertices carry no detached factor
      Prim P = load_prim(S, prim);
      int4 m = __ldg(S.mat + P.mat);
      TexFoot foot;
      float3 rho = tex_lookup(kp.albedo, m, t0.y, t0.z, &foot);
      float3 P3 = f3(0, 0, 0);
      float2 q = make_float2(0.0f, 0.0f);
      float3 L = f3(t1.x, t1.y, t1.z);
      if (fl & 8u) {
        float3 Lb = adjoint_read(dI, S.W, S.H, t0.w, t1.w, L, ATT ? &q : nullptr);
        P3 = mul(Lb, L);
      }
      scatter_albedo(g.d_albedo, foot, P3 + acc, rho);
      if (ATT) {
        PendAdj cur;
        cur.prim = prim; cur.b1 = t0.y; cur.b2 = t0.z;
        cur.x = P.o + P.e1 * t0.y + P.e2 * t0.z;
        cur.nr = cross(P.e1, P.e2);
        cur.gx = cur.gn = f3(0, 0, 0);
        if (fl & 8u) conn_adjoint(S, cur.x, cur.nr, hsum(P3), q, cur.gx, cur.gn);
        // own segment weight with the predecessor (previous tape record or the emitter)
        float3 xp = x0, np = S.ln;
        int pprim = -1;
        float pb1 = 0.0f, pb2 = 0.0f;
        if (k > 0) {
          float4 s0 = tape[2 * ((size_t)(k - 1) * kp.n_paths + p)];
          pprim = __float_as_int(s0.x) & 0xffffff;
          Prim Q = load_prim(S, pprim);
          pb1 = s0.y; pb2 = s0.z;
          xp = Q.o + Q.e1 * pb1 + Q.e2 * pb2;
          np = cross(Q.e1, Q.e2);
        }
        float3 gxp = f3(0, 0, 0), gnp = f3(0, 0, 0);
        seg_adjoint(xp, np, cur.x, cur.nr, hsum(P3 + acc), gxp, gnp, cur.gx, cur.gn);
        scatter_heights(S, g.d_heights, pprim, pb1, pb2, gxp, gnp);
        scatter_heights(S, g.d_heights, cur.prim, cur.b1, cur.b2, cur.gx, cur.gn);
      }
      acc = acc + P3;
    }
    gLe = gLe + f3(acc.x / Le.x, acc.y / Le.y, acc.z / Le.z);
  }
  block_add3(g.d_Le, gLe);
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
static int grid_for(const LaunchCfg& L, int64_t work) {
  int64_t want = (work + L.block - 1) / L.block;
  int64_t cap = (int64_t)L.sms * L.blocks_per_sm;
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

cudaError_t launch_refit(const RefitArgs& a, cudaStream_t st) {
  if (a.n_prims > 0 && a.heights) {
    k_update_tris<<<(a.n_prims + 255) / 256, 256, 0, st>>>(a.prim, a.prim_h, a.tri_base, a.heights, a.n_prims);
  }
  int threads = a.n_nodes * 32;
  k_refit_nodes<<<(threads + 255) / 256, 256, 0, st>>>(a.node, a.range, a.prim, a.n_nodes);
  return cudaGetLastError();
}

cudaError_t launch_primal(const DevScene& S, const KParams& kp, int est, float* image, void* aux, const LaunchCfg& L,
                          cudaStream_t st) {
  int grid = grid_for(L, kp.n_paths);
  switch (est) {
    case 0: k_primal<0><<<grid, L.block, 0, st>>>(S, kp, image, aux); break;
    case 1: k_primal<1><<<grid, L.block, 0, st>>>(S, kp, image, aux); break;
    default: k_primal<2><<<grid, L.block, 0, st>>>(S, kp, image, aux); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_lrb3(const DevScene& S, const KParams& kp, bool att, const float* dI, const GradPtrs& g,
                        const LaunchCfg& L, cudaStream_t st) {
  int grid = grid_for(L, kp.n_paths);
  if (att) k_lrb3<true><<<grid, L.block, 0, st>>>(S, kp, dI, g);
  else k_lrb3<false><<<grid, L.block, 0, st>>>(S, kp, dI, g);
  return cudaGetLastError();
}

cudaError_t launch_reslrb(const DevScene& S, const KParams& kp, bool att, const float* dI, const void* rec,
                          const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  int grid = grid_for(L, kp.n_paths);
  if (att) k_reslrb<true><<<grid, L.block, 0, st>>>(S, kp, dI, (const float4*)rec, g);
  else k_reslrb<false><<<grid, L.block, 0, st>>>(S, kp, dI, (const float4*)rec, g);
  return cudaGetLastError();
}

cudaError_t launch_naive(const DevScene& S, const KParams& kp, bool att, const float* dI, const void* ws,
                         const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  int grid = grid_for(L, kp.n_paths);
  if (att) k_naive<true><<<grid, L.block, 0, st>>>(S, kp, dI, ws, g);
  else k_naive<false><<<grid, L.block, 0, st>>>(S, kp, dI, ws, g);
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

}  // namespace lt
