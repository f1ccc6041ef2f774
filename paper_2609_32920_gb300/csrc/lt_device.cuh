// lt_device.cuh -- device-side scene layout and per-vertex building blocks of the light
// tracer (sm_103a).  Everything a light path needs for one vertex: Philox random numbers,
// emitter sampling, closest-hit and any-hit traversal of a threaded (stackless) BVH,
// sensor connection with its importance, tent-filter splat/read, dielectric scattering.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lt {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTMin = 1e-5f;  // ray t lower bound (metres), also the shadow-ray end margin
constexpr int kMaxDepth = 64;

enum { MAT_DIFFUSE = 0, MAT_DIELECTRIC = 1, MAT_EMITTER = 2 };
enum { K_EMITTER = 0, K_DIFFUSE = 1, K_SPECULAR = 2 };

enum ErrBits : int { ERR_BOUNDS = 1, ERR_TIMEOUT = 2, ERR_NAN = 4 };

// Scene as seen by kernels (passed by value).  Primitives are stored in BVH leaf order:
//   prim[3i+0] = (o.xyz,  material id as int bits)
//   prim[3i+1] = (e1.xyz, original primitive id as int bits)
//   prim[3i+2] = (e2.xyz, 1 if triangle else 0 as int bits)
//   prim_h[i]  = height-parameter indices of the three triangle vertices (or -1)
//   node[2j+0] = (lo.xyz, skip index)  node[2j+1] = (hi.xyz, leaf first*256 + count)
// Threaded BVH in depth-first preorder over primitives [n_direct, n_prims): the first child
// of an inner node j is j+1, and `skip` is the next node after j's subtree; leaves have
// count > 0.  The few large analytic quads [0, n_direct) are tested directly by every ray.
struct DevScene {
  const float4* prim;
  const int4* prim_h;
  const float4* node;
  int n_nodes, n_prims;
  int n_direct;           // primitives [0, n_direct) are tested directly by every ray (large quads)
  const int4* mat;        // (type, tex_off, tex_w, tex_h)
  const float* mat_ior;
  int emitter_prim;       // index in leaf order
  float3 lo, le1, le2, ln;  // emitter quad and unit normal
  float light_area;
  float3 cpos, cf, cr, cu;  // camera position and frame (forward, right, up)
  float tanx, tany;
  float K0;               // W * H / (A_img * pi); per call divided by N
  int W, H;
  int* err;               // device error word
  // Wide BVH over the same primitives (width 4 or 8, chosen per call; width 2 = the
  // threaded binary BVH above).  Node j holds, for its `width` children c, the box
  // component q (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z) at float q*width + c and the child
  // code at float 6*width + c (stride 8*width floats): code >= 0 is a wide node index,
  // code = 0x80000000 | first << 4 | count is a leaf over leaf-order primitives
  // [first, first + count), code = -1 an empty slot (its box is empty).
  const float4* wnode;
  int n_wnodes;
  int width;
  // Global atomics of one call: 0 plain; 1 warp-aggregated for gradient arrays in global
  // memory; 2 warp-aggregated for those and for the plain primal's splats (see agg_add).
  int atomics;
};

// ------------------------------------------------------------------ small vector ops
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
// Dot and cross products as explicit fused multiply-adds: the kernels are compiled without
// implicit contraction (every pass must round a path's arithmetic identically), and an
// explicit fmaf is the same operation in every kernel.
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return f3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float length(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float3 normalize(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
__device__ __forceinline__ float hsum(float3 a) { return a.x + a.y + a.z; }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
__device__ __forceinline__ uint4 philox(uint32_t k0, uint32_t k1, uint4 c) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}
// Four uniforms in [0,1) with 24-bit mantissas for (path n, vertex depth d, stream s).
__device__ __forceinline__ float4 rand4(uint64_t seed, uint64_t n, uint32_t d, uint32_t s = 0) {
  uint4 o = philox((uint32_t)seed, (uint32_t)(seed >> 32), make_uint4((uint32_t)n, (uint32_t)(n >> 32), d, s));
  const float k = 1.0f / 16777216.0f;
  return make_float4((float)(o.x >> 8) * k, (float)(o.y >> 8) * k, (float)(o.z >> 8) * k, (float)(o.w >> 8) * k);
}

// Orthonormal basis from a unit normal (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
  float sign = copysignf(1.0f, n.z);
  float a = -1.0f / (sign + n.z);
  float bb = n.x * n.y * a;
  t = f3(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
  b = f3(bb, sign + n.y * n.y * a, -n.y);
}
// Cosine-weighted direction about n from two uniforms.
__device__ __forceinline__ float3 cosine_dir(float3 n, float u0, float u1) {
  float3 t, b;
  onb(n, t, b);
  float r = sqrtf(u0), s, c;
  sincospif(2.0f * u1, &s, &c);
  return t * (r * c) + b * (r * s) + n * sqrtf(fmaxf(0.0f, 1.0f - u0));
}

// FNV-1a over the four bytes of x.
__device__ __forceinline__ void fnv(uint32_t& h, uint32_t x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) { h ^= (x >> (8 * i)) & 0xffu; h *= 16777619u; }
}

// Add v at p, which points to shared or to global memory: a reduction without return value
// in the pointer's own space.  Given a pointer that may be either, the compiler would issue a
// generic atomic that returns the old value.
__device__ __forceinline__ void red_add(float* p, float v) {
  if (__isShared(p)) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
  } else {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
  }
}

// Atomic adds of N values at consecutive addresses p..p+N-1 with warp aggregation: the lanes
// executing the call together that add at the same address first sum their values (a tree
// over the peers in lane order: at step d the peer of rank r, r a multiple of 2d, adds the
// partial sum of rank r + d), then the first of them issues the atomics.  When no two lanes
// share an address (the common case for incoherent paths) each lane adds its own values.
template <int N>
__device__ __forceinline__ void agg_add(float* p, const float (&v)[N]) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, (unsigned long long)p);
  const unsigned lane = threadIdx.x & 31;
  float s[N];
#pragma unroll
  for (int k = 0; k < N; ++k) s[k] = v[k];
  if (!__all_sync(act, peers == (1u << lane))) {
    const int rank = __popc(peers & ((1u << lane) - 1u));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned src = __fns(peers, lane, d + 1);  // the peer d ranks above, if any
      const int from = src < 32u ? (int)src : (int)lane;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float o = __shfl_sync(act, s[k], from);
        if (src < 32u && (rank & (2 * d - 1)) == 0) s[k] += o;
      }
    }
    if (rank != 0) return;
  }
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (s[k] != 0.0f) red_add(p + k, s[k]);
}

// Out-of-line forms for the gradient scatter (opts.scatter 3 only), so that the path
// kernels' hot loops do not carry the aggregation code.
static __device__ __noinline__ void agg_add1(float* p, float v) {
  const float a[1] = {v};
  agg_add<1>(p, a);
}
static __device__ __noinline__ void agg_add3(float* p, float x, float y, float z) {
  const float a[3] = {x, y, z};
  agg_add<3>(p, a);
}

// ------------------------------------------------------------------ primitives
struct Prim {
  float3 o, e1, e2;
  int mat, orig, is_tri;
};
__device__ __forceinline__ Prim load_prim(const DevScene& S, int i) {
  float4 a = __ldg(S.prim + 3 * i), b = __ldg(S.prim + 3 * i + 1), c = __ldg(S.prim + 3 * i + 2);
  Prim p;
  p.o = xyz(a); p.e1 = xyz(b); p.e2 = xyz(c);
  p.mat = __float_as_int(a.w); p.orig = __float_as_int(b.w); p.is_tri = __float_as_int(c.w);
  return p;
}

// Moller-Trumbore (1997) for triangles (s,t >= 0, s+t <= 1) and parallelograms (s,t in [0,1]).
__device__ __forceinline__ bool hit_prim(float3 o, float3 e1, float3 e2, bool tri, float3 org, float3 dir,
                                         float& t, float& u, float& v) {
  float3 pv = cross(dir, e2);
  float det = dot(e1, pv);
  if (det == 0.0f) return false;
  float inv = 1.0f / det;
  float3 tv = org - o;
  u = dot(tv, pv) * inv;
  float3 qv = cross(tv, e1);
  v = dot(dir, qv) * inv;
  t = dot(e2, qv) * inv;
  if (tri) return u >= 0.0f && v >= 0.0f && u + v <= 1.0f;
  return u >= 0.0f && u <= 1.0f && v >= 0.0f && v <= 1.0f;
}

__device__ __forceinline__ bool hit_box(float4 lo, float4 hi, float3 org, float3 inv, float tmax) {
  float tx0 = (lo.x - org.x) * inv.x, tx1 = (hi.x - org.x) * inv.x;
  float ty0 = (lo.y - org.y) * inv.y, ty1 = (hi.y - org.y) * inv.y;
  float tz0 = (lo.z - org.z) * inv.z, tz1 = (hi.z - org.z) * inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  return tn <= tf;
}

__device__ __forceinline__ float3 safe_inv(float3 d) {
  const float big = 1e30f;
  return f3(d.x != 0.0f ? 1.0f / d.x : copysignf(big, d.x), d.y != 0.0f ? 1.0f / d.y : copysignf(big, d.y),
            d.z != 0.0f ? 1.0f / d.z : copysignf(big, d.z));
}

struct HitRec {
  int prim;  // leaf-order index, -1 = miss
  float t, b1, b2;
};

// Work census of one thread (only in the counting kernel variants): rays, box tests and
// primitive tests.
struct Census {
  uint32_t rays, nodes, prims;
};

// Closest hit: smallest t > kTMin, ties to the smaller original primitive id; `skip`
// (leaf-order index) is the primitive the ray leaves.  Stackless threaded traversal in
// "while-while" form (Aila & Laine, "Understanding the efficiency of ray traversal on
// GPUs", HPG 2009): each lane walks inner nodes until it has a leaf pending (or is done),
// then the warp tests all pending leaves together, so leaf work is not serialised lane by
// lane.
template <bool ST = false>
__device__ __forceinline__ HitRec trace_closest2(const DevScene& S, float3 org, float3 dir, int skip,
                                                 Census* cs = nullptr) {
  if (ST) cs->rays++;
  HitRec h;
  h.prim = -1; h.t = 3.0e38f; h.b1 = 0; h.b2 = 0;
  int best_orig = 0x7fffffff;
  for (int k = 0; k < S.n_direct; ++k) {
    if (k == skip) continue;
    if (ST) cs->prims++;
    const Prim p = load_prim(S, k);
    float t, u, v;
    if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin &&
        (t < h.t || (t == h.t && p.orig < best_orig))) {
      h.prim = k; h.t = t; h.b1 = u; h.b2 = v; best_orig = p.orig;
    }
  }
  const float3 inv = safe_inv(dir);
  int i = 0;
  while (true) {
    int first = 0, cnt = 0;
    while (i < S.n_nodes) {
      const float4 lo = __ldg(S.node + 2 * i), hi = __ldg(S.node + 2 * i + 1);
      const int skipi = __float_as_int(lo.w);
      if (ST) cs->nodes++;
      if (hit_box(lo, hi, org, inv, h.t)) {
        const int leaf = __float_as_int(hi.w);
        if (leaf & 255) {
          first = leaf >> 8;
          cnt = leaf & 255;
          i = skipi;
          break;
        }
        i = i + 1;
      } else {
        i = skipi;
      }
    }
    if (!cnt) break;
    for (int k = first; k < first + cnt; ++k) {
      if (k == skip) continue;
      if (ST) cs->prims++;
      const Prim p = load_prim(S, k);
      float t, u, v;
      if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin &&
          (t < h.t || (t == h.t && p.orig < best_orig))) {
        h.prim = k; h.t = t; h.b1 = u; h.b2 = v; best_orig = p.orig;
      }
    }
  }
  return h;
}

// Any hit in (kTMin, dist - kTMin) (sensor-connection visibility), same traversal form.
template <bool ST = false>
__device__ __forceinline__ bool occluded2(const DevScene& S, float3 org, float3 dir, float dist, int skip,
                                          Census* cs = nullptr) {
  if (ST) cs->rays++;
  const float tmax = dist - kTMin;
  for (int k = 0; k < S.n_direct; ++k) {
    if (k == skip) continue;
    if (ST) cs->prims++;
    const Prim p = load_prim(S, k);
    float t, u, v;
    if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin && t < tmax) return true;
  }
  const float3 inv = safe_inv(dir);
  int i = 0;
  while (true) {
    int first = 0, cnt = 0;
    while (i < S.n_nodes) {
      const float4 lo = __ldg(S.node + 2 * i), hi = __ldg(S.node + 2 * i + 1);
      const int skipi = __float_as_int(lo.w);
      if (ST) cs->nodes++;
      if (hit_box(lo, hi, org, inv, tmax)) {
        const int leaf = __float_as_int(hi.w);
        if (leaf & 255) {
          first = leaf >> 8;
          cnt = leaf & 255;
          i = skipi;
          break;
        }
        i = i + 1;
      } else {
        i = skipi;
      }
    }
    if (!cnt) return false;
    for (int k = first; k < first + cnt; ++k) {
      if (k == skip) continue;
      if (ST) cs->prims++;
      const Prim p = load_prim(S, k);
      float t, u, v;
      if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin && t < tmax) return true;
    }
  }
}

// ------------------------------------------------------------------ wide BVH traversal
constexpr int kWideStack = 64;
constexpr int kCodeDone = -1;

// Rows of a wide node's plane arrays (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z) that a ray enters
// and leaves each slab by: with inv.x >= 0 it enters the x slab at lo.x and leaves at hi.x,
// else the reverse.  fmaf(plane, inv, -oi) is monotone in the plane coordinate, so the entry
// and exit distances read from these rows equal the per-axis min and max exactly (for every
// box with lo <= hi), and the slab test needs no min/max per axis.
struct Oct {
  int r[6];  // rows of the near x, y, z planes, then of the far ones
};
__device__ __forceinline__ Oct ray_oct(float3 inv) {
  Oct o;
  o.r[0] = inv.x < 0.0f ? 3 : 0; o.r[1] = inv.y < 0.0f ? 4 : 1; o.r[2] = inv.z < 0.0f ? 5 : 2;
  o.r[3] = 3 - o.r[0]; o.r[4] = 5 - o.r[1]; o.r[5] = 7 - o.r[2];
  return o;
}
// Slab test of the `W` children of wide node `j` against a ray (origin times inverse
// direction precomputed, near and far rows from ray_oct): tn[c] = entry distance, +inf when
// the child is missed, empty or entered only beyond tmax.
template <int W>
__device__ __forceinline__ void wide_boxes(const DevScene& S, int j, float3 inv, float3 oi, float tmax, float tn[W],
                                           int code[W], const Oct& o) {
  const float* nd = reinterpret_cast<const float*>(S.wnode) + (size_t)j * 8 * W;
  float v[6][W];
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int c4 = 0; c4 < W / 4; ++c4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(nd + o.r[q] * W) + c4);
      v[q][4 * c4] = a.x; v[q][4 * c4 + 1] = a.y; v[q][4 * c4 + 2] = a.z; v[q][4 * c4 + 3] = a.w;
    }
#pragma unroll
  for (int c4 = 0; c4 < W / 4; ++c4) {
    const int4 cc = __ldg(reinterpret_cast<const int4*>(nd + 6 * W) + c4);
    code[4 * c4] = cc.x; code[4 * c4 + 1] = cc.y; code[4 * c4 + 2] = cc.z; code[4 * c4 + 3] = cc.w;
  }
#pragma unroll
  for (int c = 0; c < W; ++c) {
    // entry (near) and exit (far) distance of each slab
    const float txn = fmaf(v[0][c], inv.x, -oi.x), txf = fmaf(v[3][c], inv.x, -oi.x);
    const float tyn = fmaf(v[1][c], inv.y, -oi.y), tyf = fmaf(v[4][c], inv.y, -oi.y);
    const float tzn = fmaf(v[2][c], inv.z, -oi.z), tzf = fmaf(v[5][c], inv.z, -oi.z);
    const float a = fmaxf(fmaxf(txn, tyn), fmaxf(tzn, 0.0f));
    const float b = fminf(fminf(txf, tyf), fminf(tzf, tmax));
    // an empty slot (code -1) is rejected by its code, whatever box it stores
    tn[c] = (a <= b && code[c] != -1) ? a : __int_as_float(0x7f800000);
  }
}

// Sort (key, code) pairs ascending by key: the optimal 5-comparator network for 4
// children, insertion order otherwise.
__device__ __forceinline__ void cas(float* k, int* c, int a, int b) {
  const bool sw = k[b] < k[a];
  const float ka = sw ? k[b] : k[a], kb = sw ? k[a] : k[b];
  const int ca = sw ? c[b] : c[a], cb = sw ? c[a] : c[b];
  k[a] = ka; k[b] = kb; c[a] = ca; c[b] = cb;
}
template <int W>
__device__ __forceinline__ void sort_children(float k[W], int c[W]) {
  if constexpr (W == 4) {
    cas(k, c, 0, 1); cas(k, c, 2, 3); cas(k, c, 0, 2); cas(k, c, 1, 3); cas(k, c, 1, 2);
  } else {
#pragma unroll
    for (int i = 1; i < W; ++i)
#pragma unroll
      for (int j = i; j > 0; --j) cas(k, c, j - 1, j);
  }
}

// Closest hit through the wide BVH, same result rules as trace_closest2.  Stack-based
// ordered traversal: the children of a node that the ray enters are pushed far to near
// with their entry distance, so the nearest is visited next and entries beyond the
// current hit are dropped when popped.  Leaves are tested in a separate loop (while-while
// form) so that a warp tests its lanes' pending leaves together.  A stack overflow (a
// tree deeper than the stack allows) drops the entry and sets ERR_BOUNDS.
//
// The traversal is resumable: its state (hit so far, next entry, stack depth; the stack in
// a caller-owned LocalStack) survives between calls, and a call stops after `budget` node
// and leaf visits.  A path kernel gives each lane a fixed budget per step of its main loop,
// so a warp's step no longer waits for the lane with the longest ray: that lane resumes in
// the next step while the others shade and start their next rays (the few rays that graze
// a height field visit several times more nodes than the average ray).  Split or not, the
// visits and their order are the same, and so is the hit.

// Traversal stack of (entry code, entry distance) pairs, one 8-byte word per entry, in the
// thread's local memory.
struct LocalStack {
  static constexpr int kCap = kWideStack;
  int2 e[kWideStack];
  __device__ __forceinline__ void put(int i, int code, float t) { e[i] = make_int2(code, __float_as_int(t)); }
  __device__ __forceinline__ int2 get(int i) const { return e[i]; }
};

struct TravState {
  HitRec h;
  int best_orig;  // original id of the current hit (ties go to the smaller)
  int next;       // entry to visit next: an inner node (>= 0), a leaf (< -1) or kCodeDone
  int sp;         // entries on the stack
};

template <bool ST = false>
__device__ __forceinline__ void trav_begin(const DevScene& S, float3 org, float3 dir, int skip, TravState& T,
                                           Census* cs = nullptr) {
  if (ST) cs->rays++;
  T.h.prim = -1; T.h.t = 3.0e38f; T.h.b1 = 0; T.h.b2 = 0;
  T.best_orig = 0x7fffffff;
  for (int k = 0; k < S.n_direct; ++k) {
    if (k == skip) continue;
    if (ST) cs->prims++;
    const Prim p = load_prim(S, k);
    float t, u, v;
    if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin &&
        (t < T.h.t || (t == T.h.t && p.orig < T.best_orig))) {
      T.h.prim = k; T.h.t = t; T.h.b1 = u; T.h.b2 = v; T.best_orig = p.orig;
    }
  }
  T.next = S.n_wnodes == 0 ? kCodeDone : 0;  // the root
  T.sp = 0;
}

// Continue a traversal for at most `budget` visits (a leaf found within the budget is tested
// in the same call); true when it has finished and T.h holds the closest hit.
template <int W, bool ST = false, class STK>
__device__ __forceinline__ bool trav_resume(const DevScene& S, float3 org, float3 dir, int skip, TravState& T,
                                            STK& stk, int budget, Census* cs = nullptr) {
  int next = T.next, sp = T.sp;
  if (next == kCodeDone) return true;
  const float3 inv = safe_inv(dir);
  const float3 oi = f3(org.x * inv.x, org.y * inv.y, org.z * inv.z);
  const Oct oct = ray_oct(inv);
  while (next != kCodeDone && budget > 0) {
    while (next >= 0 && budget > 0) {
      --budget;
      float tn[W];
      int code[W];
      if (ST) cs->nodes += W;
      wide_boxes<W>(S, next, inv, oi, T.h.t, tn, code, oct);
      sort_children<W>(tn, code);
#pragma unroll
      for (int c = W - 1; c >= 0; --c) {
        if (tn[c] <= T.h.t) {
          if (sp < STK::kCap) { stk.put(sp, code[c], tn[c]); ++sp; }
          else atomicOr(S.err, ERR_BOUNDS);
        }
      }
      next = kCodeDone;
      while (sp > 0) {
        --sp;
        const int2 e = stk.get(sp);
        if (__int_as_float(e.y) <= T.h.t) { next = e.x; break; }
      }
    }
    if (next >= 0 || next == kCodeDone) break;  // out of budget at an inner node, or finished
    --budget;
    const int first = (next & 0x7fffffff) >> 4, cnt = next & 15;
    for (int k = first; k < first + cnt; ++k) {
      if (k == skip) continue;
      if (ST) cs->prims++;
      const Prim p = load_prim(S, k);
      float t, u, v;
      if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin &&
          (t < T.h.t || (t == T.h.t && p.orig < T.best_orig))) {
        T.h.prim = k; T.h.t = t; T.h.b1 = u; T.h.b2 = v; T.best_orig = p.orig;
      }
    }
    next = kCodeDone;
    while (sp > 0) {
      --sp;
      const int2 e = stk.get(sp);
      if (__int_as_float(e.y) <= T.h.t) { next = e.x; break; }
    }
  }
  T.next = next;
  T.sp = sp;
  return next == kCodeDone;
}

// The same traversal in one call, with its state in registers and a local stack.
template <int W, bool ST = false>
__device__ __forceinline__ HitRec trace_closest_w(const DevScene& S, float3 org, float3 dir, int skip,
                                                  Census* cs = nullptr) {
  if (ST) cs->rays++;
  HitRec h;
  h.prim = -1; h.t = 3.0e38f; h.b1 = 0; h.b2 = 0;
  int best_orig = 0x7fffffff;
  for (int k = 0; k < S.n_direct; ++k) {
    if (k == skip) continue;
    if (ST) cs->prims++;
    const Prim p = load_prim(S, k);
    float t, u, v;
    if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin &&
        (t < h.t || (t == h.t && p.orig < best_orig))) {
      h.prim = k; h.t = t; h.b1 = u; h.b2 = v; best_orig = p.orig;
    }
  }
  if (S.n_wnodes == 0) return h;
  const float3 inv = safe_inv(dir);
  const float3 oi = f3(org.x * inv.x, org.y * inv.y, org.z * inv.z);
  const Oct oct = ray_oct(inv);
  int st_code[kWideStack];
  float st_t[kWideStack];
  int sp = 0;
  bool overflow = false;
  int next = 0;  // the root
  while (next != kCodeDone) {
    while (next >= 0) {
      float tn[W];
      int code[W];
      if (ST) cs->nodes += W;
      wide_boxes<W>(S, next, inv, oi, h.t, tn, code, oct);
      sort_children<W>(tn, code);
#pragma unroll
      for (int c = W - 1; c >= 0; --c) {
        if (tn[c] <= h.t) {
          if (sp < kWideStack) { st_code[sp] = code[c]; st_t[sp] = tn[c]; ++sp; }
          else overflow = true;
        }
      }
      next = kCodeDone;
      while (sp > 0) {
        --sp;
        if (st_t[sp] <= h.t) { next = st_code[sp]; break; }
      }
    }
    if (next == kCodeDone) break;
    const int first = (next & 0x7fffffff) >> 4, cnt = next & 15;
    for (int k = first; k < first + cnt; ++k) {
      if (k == skip) continue;
      if (ST) cs->prims++;
      const Prim p = load_prim(S, k);
      float t, u, v;
      if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin &&
          (t < h.t || (t == h.t && p.orig < best_orig))) {
        h.prim = k; h.t = t; h.b1 = u; h.b2 = v; best_orig = p.orig;
      }
    }
    next = kCodeDone;
    while (sp > 0) {
      --sp;
      if (st_t[sp] <= h.t) { next = st_code[sp]; break; }
    }
  }
  if (overflow) atomicOr(S.err, ERR_BOUNDS);
  return h;
}

// Any hit in (kTMin, dist - kTMin) through the wide BVH (children in stored order).
template <int W, bool ST = false>
__device__ __forceinline__ bool occluded_w(const DevScene& S, float3 org, float3 dir, float dist, int skip,
                                           Census* cs = nullptr) {
  if (ST) cs->rays++;
  const float tmax = dist - kTMin;
  for (int k = 0; k < S.n_direct; ++k) {
    if (k == skip) continue;
    if (ST) cs->prims++;
    const Prim p = load_prim(S, k);
    float t, u, v;
    if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin && t < tmax) return true;
  }
  if (S.n_wnodes == 0) return false;
  const float3 inv = safe_inv(dir);
  const float3 oi = f3(org.x * inv.x, org.y * inv.y, org.z * inv.z);
  const Oct oct = ray_oct(inv);
  int st_code[kWideStack];
  int sp = 0;
  bool overflow = false;
  int next = 0;
  bool hit = false;
  while (next != kCodeDone && !hit) {
    while (next >= 0) {
      float tn[W];
      int code[W];
      if (ST) cs->nodes += W;
      wide_boxes<W>(S, next, inv, oi, tmax, tn, code, oct);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (tn[c] <= tmax) {
          if (sp < kWideStack) st_code[sp++] = code[c];
          else overflow = true;
        }
      }
      next = sp > 0 ? st_code[--sp] : kCodeDone;
    }
    if (next == kCodeDone) break;
    const int first = (next & 0x7fffffff) >> 4, cnt = next & 15;
    for (int k = first; k < first + cnt; ++k) {
      if (k == skip) continue;
      if (ST) cs->prims++;
      const Prim p = load_prim(S, k);
      float t, u, v;
      if (hit_prim(p.o, p.e1, p.e2, p.is_tri, org, dir, t, u, v) && t > kTMin && t < tmax) { hit = true; break; }
    }
    next = sp > 0 ? st_code[--sp] : kCodeDone;
  }
  if (overflow) atomicOr(S.err, ERR_BOUNDS);
  return hit;
}

// Traversal entry points.  The BVH width is fixed per translation unit (LT_BVH_WIDTH):
// the kernels are compiled once per width, so each variant carries only its own
// traversal's registers; the host picks the variant that matches the call's width.
#ifndef LT_BVH_WIDTH
#define LT_BVH_WIDTH 4
#endif
template <bool ST = false>
__device__ __forceinline__ HitRec trace_closest(const DevScene& S, float3 org, float3 dir, int skip,
                                                Census* cs = nullptr) {
#if LT_BVH_WIDTH == 2
  return trace_closest2<ST>(S, org, dir, skip, cs);
#else
  return trace_closest_w<LT_BVH_WIDTH, ST>(S, org, dir, skip, cs);
#endif
}
// Resumable closest hit (see TravState): the binary BVH finishes in the first call.
#ifndef LT_TRACE_BUDGET
#define LT_TRACE_BUDGET 5
#endif
constexpr int kTraceBudget = LT_TRACE_BUDGET;  // node and leaf visits per lane per step
template <bool ST = false>
__device__ __forceinline__ void trace_begin(const DevScene& S, float3 org, float3 dir, int skip, TravState& T,
                                            Census* cs = nullptr) {
#if LT_BVH_WIDTH == 2
  T.h = trace_closest2<ST>(S, org, dir, skip, cs);
  T.next = kCodeDone;
#else
  trav_begin<ST>(S, org, dir, skip, T, cs);
#endif
}
template <bool ST = false, class STK>
__device__ __forceinline__ bool trace_resume(const DevScene& S, float3 org, float3 dir, int skip, TravState& T,
                                             STK& stk, Census* cs = nullptr) {
#if LT_BVH_WIDTH == 2
  return true;
#else
  return trav_resume<LT_BVH_WIDTH, ST>(S, org, dir, skip, T, stk, kTraceBudget, cs);
#endif
}
template <bool ST = false>
__device__ __forceinline__ bool occluded(const DevScene& S, float3 org, float3 dir, float dist, int skip,
                                         Census* cs = nullptr) {
#if LT_BVH_WIDTH == 2
  return occluded2<ST>(S, org, dir, dist, skip, cs);
#else
  return occluded_w<LT_BVH_WIDTH, ST>(S, org, dir, dist, skip, cs);
#endif
}

// ------------------------------------------------------------------ camera / film
// Film coordinates in pixels (row 0 at the top); false when behind the camera.
__device__ __forceinline__ bool project(const DevScene& S, float3 x, float& ux, float& uy, float& zc) {
  float3 d = x - S.cpos;
  zc = dot(d, S.cf);
  if (zc <= 0.0f) return false;
  float px = dot(d, S.cr) / zc, py = dot(d, S.cu) / zc;
  ux = 0.5f * (float)S.W * (1.0f + px / S.tanx);
  uy = 0.5f * (float)S.H * (1.0f - py / S.tany);
  return true;
}

// Sensor connection at a diffuse vertex x with arrival-side unit normal ns (Sec. 3.1,
// Eq. 1): valid when the camera lies in the arrival hemisphere, in front of the camera,
// on the film and unoccluded.  geo = |n . w_c| * W*H / (A_img * pi * r^2 * cos^3 theta_c)
// (the importance of a pinhole with image plane at distance 1, with the Lambertian 1/pi).
struct Conn {
  bool valid;
  float ux, uy, geo;
  float3 wc;   // unit direction to the camera
  float dist;  // distance to the camera
};

// The connection tests that need no ray: camera in the arrival hemisphere, in front of
// the camera and on the film.  Fills geo, u, wc and dist; valid = candidate.
__device__ __forceinline__ Conn connect_pre(const DevScene& S, float3 x, float3 ns) {
  Conn c;
  c.valid = false; c.ux = c.uy = c.geo = 0.0f;
  float3 cv = S.cpos - x;
  c.dist = length(cv);
  c.wc = cv * (1.0f / c.dist);
  float cosc = dot(ns, c.wc);
  if (!(cosc > 0.0f)) return c;
  float zc;
  if (!project(S, x, c.ux, c.uy, zc)) return c;
  if (!(c.ux >= 0.0f && c.ux < (float)S.W && c.uy >= 0.0f && c.uy < (float)S.H)) return c;
  float cc = zc / c.dist;
  c.geo = cosc * S.K0 / (c.dist * c.dist * cc * cc * cc);
  c.valid = true;
  return c;
}
template <bool ST = false>
__device__ __forceinline__ Conn connect(const DevScene& S, float3 x, float3 ns, int prim, bool test_vis = true,
                                        Census* cs = nullptr) {
  Conn c;
  c.valid = false; c.ux = c.uy = c.geo = 0.0f;
  float3 cv = S.cpos - x;
  float dist = length(cv);
  float3 wc = cv * (1.0f / dist);
  float cosc = dot(ns, wc);
  if (!(cosc > 0.0f)) return c;
  float zc;
  if (!project(S, x, c.ux, c.uy, zc)) return c;
  if (!(c.ux >= 0.0f && c.ux < (float)S.W && c.uy >= 0.0f && c.uy < (float)S.H)) return c;
  if (test_vis && occluded<ST>(S, x, wc, dist, prim, cs)) return c;
  float cc = zc / dist;
  c.geo = cosc * S.K0 / (dist * dist * cc * cc * cc);
  c.valid = true;
  return c;
}

// Tent (bilinear) reconstruction filter of radius 1 pixel over pixel centres: the two
// taps per axis around u and their weights; taps off the film are dropped.
struct Taps {
  int x0, y0;
  float fx, fy;
};
__device__ __forceinline__ Taps taps(float ux, float uy) {
  float gx = ux - 0.5f, gy = uy - 0.5f;
  float x0 = floorf(gx), y0 = floorf(gy);
  Taps t;
  t.x0 = (int)x0; t.y0 = (int)y0; t.fx = gx - x0; t.fy = gy - y0;
  return t;
}

__device__ __forceinline__ void splat(float* img, int W, int H, float ux, float uy, float3 L, bool agg = false) {
  Taps t = taps(ux, uy);
  const float wx[2] = {1.0f - t.fx, t.fx}, wy[2] = {1.0f - t.fy, t.fy};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    int Y = t.y0 + j;
    if (Y < 0 || Y >= H) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int X = t.x0 + i;
      if (X < 0 || X >= W) continue;
      float w = wx[i] * wy[j];
      float* p = img + 3 * ((size_t)Y * W + X);
      if (agg) {
        const float v[3] = {w * L.x, w * L.y, w * L.z};
        agg_add<3>(p, v);
      } else {
        atomicAdd(p + 0, w * L.x);
        atomicAdd(p + 1, w * L.y);
        atomicAdd(p + 2, w * L.z);
      }
    }
  }
}

// Filter-weighted adjoint read Lbar = sum_p F(u,p) dI[p] (Eq. 21 with the same filter as
// the splat) and, when wanted, the position adjoint q = d(Lbar . L)/du (Eq. 20-21).
__device__ __forceinline__ float3 adjoint_read(const float* dI, int W, int H, float ux, float uy, float3 L,
                                               float2* q) {
  Taps t = taps(ux, uy);
  const float wx[2] = {1.0f - t.fx, t.fx}, wy[2] = {1.0f - t.fy, t.fy};
  const float sx[2] = {-1.0f, 1.0f};
  float3 Lb = f3(0, 0, 0);
  float qx = 0.0f, qy = 0.0f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    int Y = t.y0 + j;
    if (Y < 0 || Y >= H) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int X = t.x0 + i;
      if (X < 0 || X >= W) continue;
      const float* p = dI + 3 * ((size_t)Y * W + X);
      float3 v = f3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
      Lb = Lb + v * (wx[i] * wy[j]);
      float lv = dot(v, L);
      qx += sx[i] * wy[j] * lv;
      qy += sx[j] * wx[i] * lv;
    }
  }
  if (q) *q = make_float2(qx, qy);
  return Lb;
}

// Wider filter (filter 1): separable truncated Gaussian of standard deviation 0.5 pixel
// over pixel centres, shifted down by its value at the radius 1.5 pixel so that it falls
// continuously to zero, normalised to unit integral per axis:
// g(d) = (exp(-2 d^2) - exp(-4.5)) / C, C = sqrt(pi/2) erf(1.5 sqrt(2)) - 3 exp(-4.5).
// Up to three taps per axis; taps off the film are dropped.
constexpr float kGaussInvC = 0.82196051292f;  // 1 / C
constexpr float kGaussCut = 0.01110899654f;   // exp(-4.5)
struct Axis3 {
  int x[3];
  float w[3], dw[3];  // weights and their derivatives along u
  int n;
};
__device__ __forceinline__ Axis3 gauss_axis(float u, int extent) {
  Axis3 a;
  a.n = 0;
  const int b = (int)floorf(u - 0.5f);
#pragma unroll
  for (int i = -1; i <= 2; ++i) {
    const int X = b + i;
    const float d = u - ((float)X + 0.5f);
    if (fabsf(d) < 1.5f && X >= 0 && X < extent && a.n < 3) {
      const float e = expf(-2.0f * d * d);
      a.x[a.n] = X;
      a.w[a.n] = (e - kGaussCut) * kGaussInvC;
      a.dw[a.n] = -4.0f * d * e * kGaussInvC;
      ++a.n;
    }
  }
  return a;
}

// Splat and adjoint read with the chosen filter (0 tent, 1 Gaussian).
__device__ __forceinline__ void splat_f(float* img, int W, int H, float ux, float uy, float3 L, int filter,
                                        bool agg = false) {
  if (filter == 0) {
    splat(img, W, H, ux, uy, L, agg);
    return;
  }
  const Axis3 ax = gauss_axis(ux, W), ay = gauss_axis(uy, H);
  for (int j = 0; j < ay.n; ++j)
    for (int i = 0; i < ax.n; ++i) {
      const float w = ax.w[i] * ay.w[j];
      float* p = img + 3 * ((size_t)ay.x[j] * W + ax.x[i]);
      atomicAdd(p + 0, w * L.x);
      atomicAdd(p + 1, w * L.y);
      atomicAdd(p + 2, w * L.z);
    }
}
__device__ __forceinline__ float3 adjoint_read_f(const float* dI, int W, int H, float ux, float uy, float3 L,
                                                 float2* q, int filter) {
  if (filter == 0) return adjoint_read(dI, W, H, ux, uy, L, q);
  const Axis3 ax = gauss_axis(ux, W), ay = gauss_axis(uy, H);
  float3 Lb = f3(0, 0, 0);
  float qx = 0.0f, qy = 0.0f;
  for (int j = 0; j < ay.n; ++j)
    for (int i = 0; i < ax.n; ++i) {
      const float* p = dI + 3 * ((size_t)ay.x[j] * W + ax.x[i]);
      const float3 v = f3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
      Lb = Lb + v * (ax.w[i] * ay.w[j]);
      const float lv = dot(v, L);
      qx += ax.dw[i] * ay.w[j] * lv;
      qy += ax.w[i] * ay.dw[j] * lv;
    }
  if (q) *q = make_float2(qx, qy);
  return Lb;
}

// ------------------------------------------------------------------ materials
__device__ __forceinline__ float3 texel(const float* albedo, int idx) {
  return f3(__ldg(albedo + idx), __ldg(albedo + idx + 1), __ldg(albedo + idx + 2));
}
// Bilinear lookup at texture coordinates (s,t): texel centres (i+0.5)/w, clamp to edge.
// Returns the four texel offsets and weights too (for the albedo gradient scatter).
struct TexFoot {
  int idx[4];
  float w[4];
};
__device__ __forceinline__ float3 tex_lookup(const float* albedo, int4 m, float s, float t, TexFoot* foot) {
  int tw = m.z, th = m.w, off = m.y;
  float tx = s * (float)tw - 0.5f, ty = t * (float)th - 0.5f;
  float fx0 = floorf(tx), fy0 = floorf(ty);
  float fx = tx - fx0, fy = ty - fy0;
  int x0 = (int)fx0, y0 = (int)fy0;
  int xa = min(max(x0, 0), tw - 1), xb = min(max(x0 + 1, 0), tw - 1);
  int ya = min(max(y0, 0), th - 1), yb = min(max(y0 + 1, 0), th - 1);
  int i00 = off + (ya * tw + xa) * 3, i10 = off + (ya * tw + xb) * 3;
  int i01 = off + (yb * tw + xa) * 3, i11 = off + (yb * tw + xb) * 3;
  float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy), w01 = (1.0f - fx) * fy, w11 = fx * fy;
  if (foot) {
    foot->idx[0] = i00; foot->idx[1] = i10; foot->idx[2] = i01; foot->idx[3] = i11;
    foot->w[0] = w00; foot->w[1] = w10; foot->w[2] = w01; foot->w[3] = w11;
  }
  return texel(albedo, i00) * w00 + texel(albedo, i10) * w10 + texel(albedo, i01) * w01 + texel(albedo, i11) * w11;
}

// Smooth dielectric: Fresnel reflectance F for unpolarised light, reflected and
// refracted directions; `entering` when arriving against the geometric normal n.
struct Dielectric {
  float F, ci, ct, eta;
  bool tir, entering;
  float3 ns, refl, refr;
};
__device__ __forceinline__ Dielectric dielectric(float3 din, float3 n, float ior) {
  Dielectric D;
  D.entering = dot(din, n) < 0.0f;
  D.ns = D.entering ? n : -n;
  D.eta = D.entering ? 1.0f / ior : ior;
  D.ci = -dot(din, D.ns);
  D.refl = din + D.ns * (2.0f * D.ci);
  float s2t = D.eta * D.eta * (1.0f - D.ci * D.ci);
  D.tir = s2t >= 1.0f;
  if (D.tir) { D.F = 1.0f; D.ct = 0.0f; D.refr = D.refl; return D; }
  D.ct = sqrtf(1.0f - s2t);
  float rs = (D.eta * D.ci - D.ct) / (D.eta * D.ci + D.ct);
  float rp = (D.ci - D.eta * D.ct) / (D.ci + D.eta * D.ct);
  D.F = 0.5f * (rs * rs + rp * rp);
  D.refr = din * D.eta + D.ns * (D.eta * D.ci - D.ct);
  return D;
}

__device__ __forceinline__ float luminance(float3 L) { return 0.2126f * L.x + 0.7152f * L.y + 0.0722f * L.z; }

__device__ __forceinline__ void set_err(const DevScene& S, int bit) { atomicOr(S.err, bit); }

}  // namespace lt
