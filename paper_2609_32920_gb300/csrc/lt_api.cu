// lt_api.cu -- host side of liblt: argument validation, scene construction (binned-SAH
// BVH build, flattened to a threaded depth-first layout), device buffers and the
// extern "C" entry points declared in include/lt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lt.h"
#include "lt_batch.h"
#include "lt_device.cuh"
#include "lt_launch.h"

using namespace lt;

namespace {

thread_local std::string g_last_error;

lt_status fail(lt_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define LT_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(LT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct HV {
  float x, y, z;
};
HV hv(float x, float y, float z) { return HV{x, y, z}; }
HV operator+(HV a, HV b) { return hv(a.x + b.x, a.y + b.y, a.z + b.z); }
HV operator-(HV a, HV b) { return hv(a.x - b.x, a.y - b.y, a.z - b.z); }
HV operator*(HV a, float s) { return hv(a.x * s, a.y * s, a.z * s); }
float hdot(HV a, HV b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
HV hcross(HV a, HV b) { return hv(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
HV hnorm(HV a) { return a * (1.0f / std::sqrt(hdot(a, a))); }

// ------------------------------------------------------------------ BVH build (host)
struct Box {
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  void grow(const Box& b) {
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
  }
  void grow(const float* p) {
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); }
  }
  float area() const {
    if (hi[0] < lo[0]) return 0.0f;
    float d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
    return 2.0f * (d0 * d1 + d1 * d2 + d2 * d0);
  }
};

struct BNode {
  Box box;
  int left = -1, right = -1;
  int begin = 0, end = 0;  // primitive index range in the build order
};

struct Builder {
  const std::vector<Box>& pb;
  std::vector<float> cen;  // [n][3]
  std::vector<int> idx;
  std::vector<BNode> nodes;
  static constexpr int kBins = 16, kMaxLeaf = 8;

  explicit Builder(const std::vector<Box>& boxes) : pb(boxes) {
    int n = (int)boxes.size();
    cen.resize(3 * n);
    idx.resize(n);
    for (int i = 0; i < n; ++i) {
      idx[i] = i;
      for (int k = 0; k < 3; ++k) cen[3 * i + k] = 0.5f * (boxes[i].lo[k] + boxes[i].hi[k]);
    }
  }

  int build(int begin, int end, int depth) {
    int me = (int)nodes.size();
    nodes.emplace_back();
    Box b, cb;
    for (int i = begin; i < end; ++i) { b.grow(pb[idx[i]]); cb.grow(&cen[3 * idx[i]]); }
    nodes[me].box = b;
    nodes[me].begin = begin;
    nodes[me].end = end;
    int n = end - begin;
    if (n <= 2 || depth > 60) return me;
    // binned SAH over the axis of largest centroid extent, then the other axes
    float best = 3e38f;
    int best_axis = -1, best_bin = -1;
    for (int axis = 0; axis < 3; ++axis) {
      float lo = cb.lo[axis], ext = cb.hi[axis] - cb.lo[axis];
      if (!(ext > 0)) continue;
      Box bins[kBins];
      int cnt[kBins] = {0};
      for (int i = begin; i < end; ++i) {
        int bi = std::min(kBins - 1, (int)((cen[3 * idx[i] + axis] - lo) / ext * kBins));
        bins[bi].grow(pb[idx[i]]);
        ++cnt[bi];
      }
      float rightA[kBins];
      int rightN[kBins];
      Box acc;
      int an = 0;
      for (int k = kBins - 1; k > 0; --k) {
        acc.grow(bins[k]);
        an += cnt[k];
        rightA[k] = acc.area();
        rightN[k] = an;
      }
      Box lacc;
      int ln = 0;
      for (int k = 1; k < kBins; ++k) {
        lacc.grow(bins[k - 1]);
        ln += cnt[k - 1];
        if (ln == 0 || rightN[k] == 0) continue;
        float cost = lacc.area() * ln + rightA[k] * rightN[k];
        if (cost < best) { best = cost; best_axis = axis; best_bin = k; }
      }
    }
    float leaf_cost = b.area() * n;
    const float trav = 1.0f;
    bool split = best_axis >= 0 && (best + trav * b.area() < leaf_cost || n > kMaxLeaf);
    if (!split && n <= kMaxLeaf) return me;
    int mid;
    if (best_axis >= 0) {
      float lo = cb.lo[best_axis], ext = cb.hi[best_axis] - cb.lo[best_axis];
      int* p = std::partition(idx.data() + begin, idx.data() + end, [&](int i) {
        return std::min(kBins - 1, (int)((cen[3 * i + best_axis] - lo) / ext * kBins)) < best_bin;
      });
      mid = (int)(p - idx.data());
      if (mid == begin || mid == end) mid = begin + n / 2;
    } else {
      mid = begin + n / 2;  // coincident centroids: split by count
    }
    int l = build(begin, mid, depth + 1);
    int r = build(mid, end, depth + 1);
    nodes[me].left = l;
    nodes[me].right = r;
    return me;
  }
};

}  // namespace

struct lt_scene {
  DevScene dev{};
  int device = 0;
  int n_albedo = 0, n_heights = 0, n_tris_h = 0;
  bool has_dielectric = false;
  int sms = 1;
  int smem_optin = 48 * 1024;  // opt-in dynamic shared memory per block
  // device buffers
  float4* d_prim = nullptr;
  int4* d_prim_h = nullptr;
  float4* d_tri_base = nullptr;
  float4* d_node = nullptr;
  int2* d_range = nullptr;
  int* d_big = nullptr;  // binary nodes refitted by a whole block
  int n_big = 0;
  int4* d_mat = nullptr;
  float* d_ior = nullptr;
  int* d_err = nullptr;
  int n_nodes = 0, n_prims = 0;
  // wide BVHs of width 4 and 8 (collapses of the binary tree)
  float4* d_wnode[2] = {};
  int* d_wmap[2] = {};
  int n_wnodes[2] = {};
};

namespace {

void free_scene(lt_scene* s) {
  if (!s) return;
  cudaFree(s->d_prim); cudaFree(s->d_prim_h); cudaFree(s->d_tri_base); cudaFree(s->d_node);
  cudaFree(s->d_range); cudaFree(s->d_big); cudaFree(s->d_mat); cudaFree(s->d_ior); cudaFree(s->d_err);
  for (int k = 0; k < 2; ++k) { cudaFree(s->d_wnode[k]); cudaFree(s->d_wmap[k]); }
  delete s;
}

RefitArgs refit_args(const lt_scene* s, const float* heights) {
  RefitArgs ra{s->d_prim, s->d_prim_h, s->d_tri_base, heights, s->n_prims, s->d_node, s->d_range, s->n_nodes,
               s->d_big, s->n_big,
               {s->d_wnode[0], s->d_wnode[1]}, {s->d_wmap[0], s->d_wmap[1]}, {s->n_wnodes[0], s->n_wnodes[1]}};
  return ra;
}

// The scene as one call's kernels see it: BVH width from opts (0 = 4), plain atomics.
DevScene dev_for(const lt_scene* s, int width) {
  if (width == 0) width = 4;
  DevScene S = s->dev;
  S.width = 2;
  S.wnode = nullptr;
  S.n_wnodes = 0;
  if (width == 4 || width == 8) {
    const int k = width == 4 ? 0 : 1;
    S.width = width;
    S.wnode = s->d_wnode[k];
    S.n_wnodes = s->n_wnodes[k];
  }
  S.atomics = 0;
  return S;
}
// ... and with the call's atomics (opts->scatter).
DevScene dev_for(const lt_scene* s, const lt_render_opts* o) {
  DevScene S = dev_for(s, o->bvh_width);
  S.atomics = o->scatter == 3 ? 2 : 0;
  return S;
}

// Collapse the binary tree into nodes of up to W children: starting from a node's two
// children, the internal child of largest surface area is replaced by its own two
// children until there are W or only leaves remain.  Returns, per wide node, the child
// codes (see DevScene::wnode) and the binary node (flat index) whose box each slot takes.
void collapse_wide(const Builder& B, int W, int nd, const std::vector<int>& flat_of, std::vector<int>& codes,
                   std::vector<int>& wmap) {
  codes.clear();
  wmap.clear();
  if (B.nodes.empty()) return;
  std::vector<int> wq = {0};
  for (size_t wi = 0; wi < wq.size(); ++wi) {
    const int b = wq[wi];
    std::vector<int> ch;
    if (B.nodes[b].left < 0) {
      ch.push_back(b);
    } else {
      ch.push_back(B.nodes[b].left);
      ch.push_back(B.nodes[b].right);
    }
    while ((int)ch.size() < W) {
      int best = -1;
      float ba = -1.0f;
      for (int k = 0; k < (int)ch.size(); ++k) {
        const BNode& n = B.nodes[ch[k]];
        if (n.left >= 0 && n.box.area() > ba) { ba = n.box.area(); best = k; }
      }
      if (best < 0) break;
      const int x = ch[best];
      ch.erase(ch.begin() + best);
      ch.push_back(B.nodes[x].left);
      ch.push_back(B.nodes[x].right);
    }
    for (int c = 0; c < W; ++c) {
      if (c < (int)ch.size()) {
        const BNode& n = B.nodes[ch[c]];
        wmap.push_back(flat_of[ch[c]]);
        if (n.left >= 0) {
          codes.push_back((int)wq.size());
          wq.push_back(ch[c]);
        } else {
          const unsigned leaf = 0x80000000u | ((unsigned)(nd + n.begin) << 4) | (unsigned)(n.end - n.begin);
          codes.push_back((int)leaf);
        }
      } else {
        wmap.push_back(-1);
        codes.push_back(-1);
      }
    }
  }
}

lt_status validate_desc(const lt_scene_desc* d) {
  if (!d) return fail(LT_ERR_INVALID_ARG, "desc is NULL");
  if (d->n_quads < 1 || !d->quads) return fail(LT_ERR_INVALID_ARG, "need at least one quad (the emitter)");
  if (d->n_tris < 0 || d->n_verts < 0) return fail(LT_ERR_INVALID_ARG, "negative counts");
  if (d->n_tris > 0 && (!d->tris || !d->verts || !d->vert_h)) return fail(LT_ERR_INVALID_ARG, "triangle arrays missing");
  if ((int64_t)d->n_quads + d->n_tris >= (1 << 23)) return fail(LT_ERR_INVALID_ARG, "too many primitives");
  if (!d->prim_mat || d->n_mats < 1 || !d->mat_type || !d->mat_ior || !d->mat_tex_off || !d->mat_tex_w ||
      !d->mat_tex_h)
    return fail(LT_ERR_INVALID_ARG, "material arrays missing");
  if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384)
    return fail(LT_ERR_INVALID_ARG, "film size out of range");
  if (!(d->fov_y_deg > 0 && d->fov_y_deg < 179)) return fail(LT_ERR_INVALID_ARG, "fov_y_deg out of range");
  if (d->emitter_quad < 0 || d->emitter_quad >= d->n_quads) return fail(LT_ERR_INVALID_ARG, "emitter_quad out of range");
  for (int i = 0; i < d->n_mats; ++i) {
    int t = d->mat_type[i];
    if (t < 0 || t > 2) return fail(LT_ERR_INVALID_ARG, "unknown material type");
    if (t == LT_MAT_DIFFUSE) {
      int64_t end = (int64_t)d->mat_tex_off[i] + 3ll * d->mat_tex_w[i] * d->mat_tex_h[i];
      if (d->mat_tex_w[i] < 1 || d->mat_tex_h[i] < 1 || d->mat_tex_off[i] < 0 || end > d->n_albedo)
        return fail(LT_ERR_INVALID_ARG, "diffuse texture outside the albedo array");
    }
    if (t == LT_MAT_DIELECTRIC && !(d->mat_ior[i] > 0)) return fail(LT_ERR_INVALID_ARG, "ior must be positive");
  }
  for (int i = 0; i < d->n_quads + d->n_tris; ++i)
    if (d->prim_mat[i] < 0 || d->prim_mat[i] >= d->n_mats) return fail(LT_ERR_INVALID_ARG, "prim_mat out of range");
  if (d->mat_type[d->prim_mat[d->emitter_quad]] != LT_MAT_EMITTER)
    return fail(LT_ERR_INVALID_ARG, "emitter_quad must have an emitter material");
  for (int i = 0; i < 3 * d->n_tris; ++i)
    if (d->tris[i] < 0 || d->tris[i] >= d->n_verts) return fail(LT_ERR_INVALID_ARG, "triangle vertex index out of range");
  for (int i = 0; i < d->n_verts; ++i)
    if (d->vert_h[i] < -1 || d->vert_h[i] >= d->n_heights) return fail(LT_ERR_INVALID_ARG, "vert_h out of range");
  return LT_OK;
}

LaunchCfg cfg_for(const lt_scene* s, const lt_render_opts* o) {
  LaunchCfg L;
  L.block = (o && o->block_size > 0) ? o->block_size : 128;
  L.blocks_per_sm = (o && o->blocks_per_sm > 0) ? o->blocks_per_sm : 8;
  L.sms = s->sms;
  return L;
}

lt_status check_opts(const lt_scene* s, const lt_params* p, const lt_render_opts* o) {
  if (!s) return fail(LT_ERR_INVALID_ARG, "scene is NULL");
  if (!p || !p->Le || (s->n_albedo > 0 && !p->albedo)) return fail(LT_ERR_INVALID_ARG, "params missing");
  if (!o) return fail(LT_ERR_INVALID_ARG, "opts is NULL");
  if (o->max_depth < 1 || o->max_depth > kMaxDepth) return fail(LT_ERR_INVALID_ARG, "max_depth must be in 1..64");
  if (o->n_paths < 0 || o->path_offset < 0 || o->n_norm < 0) return fail(LT_ERR_INVALID_ARG, "negative path counts");
  // every byte count derived from n_paths (records, states, tapes up to 64 vertices of
  // 32 B) stays far inside size_t, and path indices inside the 64-bit Philox counter
  if (o->n_paths > LT_MAX_PATHS || o->path_offset > LT_MAX_PATHS)
    return fail(LT_ERR_INVALID_ARG, "n_paths and path_offset must be at most 2^40");
  if (o->block_size != 0 && (o->block_size < 32 || o->block_size > 1024 || o->block_size % 32))
    return fail(LT_ERR_INVALID_ARG, "block_size must be a multiple of 32 in 32..1024 (or 0)");
  if (o->block_size > 128) return fail(LT_ERR_INVALID_ARG, "kernels are compiled for at most 128 threads per block");
  if (o->target != LT_TARGET_LUMINANCE && o->target != LT_TARGET_MLP) return fail(LT_ERR_INVALID_ARG, "unknown reservoir target");
  if (o->target == LT_TARGET_MLP && !o->mlp) return fail(LT_ERR_INVALID_ARG, "LT_TARGET_MLP needs opts->mlp");
  if (o->bvh_width != 0 && o->bvh_width != 2 && o->bvh_width != 4 && o->bvh_width != 8)
    return fail(LT_ERR_INVALID_ARG, "bvh_width must be 0, 2, 4 or 8");
  if (o->rr_depth < 0 || (o->rr_depth > 0 && !(o->rr_prob > 0.0f && o->rr_prob <= 1.0f)))
    return fail(LT_ERR_INVALID_ARG, "rr_depth must be >= 0 and rr_prob in (0, 1]");
  if (o->filter != 0 && o->filter != 1) return fail(LT_ERR_INVALID_ARG, "filter must be 0 (tent) or 1 (Gaussian)");
  if (o->scatter < 0 || o->scatter > 3) return fail(LT_ERR_INVALID_ARG, "scatter must be 0, 1, 2 or 3");
  if (o->literal != 0 && o->literal != 1) return fail(LT_ERR_INVALID_ARG, "literal must be 0 or 1");
  if (o->det_eps < 0.0f) return fail(LT_ERR_INVALID_ARG, "det_eps must be >= 0");
  return LT_OK;
}

KParams kparams(const lt_params* p, const lt_render_opts* o) {
  KParams k;
  k.seed = o->seed;
  k.path_offset = o->path_offset;
  k.n_paths = o->n_paths;
  k.max_depth = o->max_depth;
  k.inv_n = 1.0f / (float)(o->n_norm > 0 ? o->n_norm : (o->n_paths > 0 ? o->n_paths : 1));
  k.Le = p->Le;
  k.albedo = p->albedo;
  k.mask = o->path_mask;
  k.hash = o->path_hash;
  k.dbg = o->path_dbg;
  k.tape_offset = ((size_t)o->n_paths * sizeof(int) + 255) & ~(size_t)255;
  k.census = (unsigned long long*)o->census;
  k.n_alb = k.n_h = k.priv_n = 0;
  k.mlp = o->target == LT_TARGET_MLP ? (const float*)o->mlp : nullptr;
  k.vstate = nullptr;
  k.rr_depth = o->rr_depth;
  k.rr_q = o->rr_prob;
  k.filter = o->filter;
  k.list = nullptr;
  k.list_n = nullptr;
  k.ticket = nullptr;
  k.conn1 = nullptr;
  k.conn1z = nullptr;
  k.order = nullptr;
  k.jac_noise = o->jac_noise;
  k.noise_seed = o->noise_seed;
  k.det_eps = o->det_eps > 0.0f ? o->det_eps : 1e-6f;
  return k;
}

// Gradients accumulate per block in shared memory for each parameter array that fits in
// the budget (opts->scatter 0: the default 48 KB shared-memory limit less room for static
// shared memory, 46 KB; 1: the device's opt-in limit less 4 KB; 2, 3: none): the albedo
// array first (usually small and hit by every diffuse vertex), then the heights if room
// remains; an array that does not fit goes to global memory.
void set_privatization(const lt_scene* s, const lt_grads* g, KParams& kp, int scatter = 0) {
  const int budget = scatter >= 2 ? 0
                     : scatter == 1 ? (s->smem_optin - 4096) / (int)sizeof(float)
                                    : (46 * 1024) / (int)sizeof(float);
  kp.n_alb = (g && g->d_albedo && s->n_albedo > 0 && s->n_albedo <= budget) ? s->n_albedo : 0;
  kp.n_h = (g && g->d_heights && s->n_heights > 0 && s->n_heights <= budget - kp.n_alb) ? s->n_heights : 0;
  kp.priv_n = kp.n_alb + kp.n_h;
}

lt_status prep_grads(const lt_scene* s, const lt_grads* g, cudaStream_t st, GradPtrs& gp) {
  if (!g) return fail(LT_ERR_INVALID_ARG, "grads is NULL");
  gp.d_albedo = g->d_albedo;
  gp.d_Le = g->d_Le;
  gp.d_heights = g->d_heights;
  if (!g->accumulate) {
    if (g->d_albedo && s->n_albedo) LT_CUDA(cudaMemsetAsync(g->d_albedo, 0, sizeof(float) * s->n_albedo, st));
    if (g->d_Le) LT_CUDA(cudaMemsetAsync(g->d_Le, 0, sizeof(float) * 3, st));
    if (g->d_heights && s->n_heights) LT_CUDA(cudaMemsetAsync(g->d_heights, 0, sizeof(float) * s->n_heights, st));
  }
  return LT_OK;
}

}  // namespace

// Fixed tape for lt_naive_gradient_static: file-scope device memory, so that call never
// allocates.  Host code must not use this name as an address; it looks the device
// address up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_naive_static_tape[LT_NAIVE_STATIC_BYTES];

namespace {
std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
void* g_static_tape[kMaxDevices] = {};

// Device address of the fixed tape on the current device (looked up on first use).
lt_status static_tape(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(LT_ERR_UNSUPPORTED, "device index beyond the static tape table");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_tape[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_naive_static_tape);
    if (e != cudaSuccess || !p)
      return fail(LT_ERR_CUDA, std::string("lt_naive_gradient_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_tape[dev] = p;
  }
  *out = g_static_tape[dev];
  return LT_OK;
}
}  // namespace

extern "C" {

const char* lt_last_error(void) { return g_last_error.c_str(); }

lt_status lt_naive_gradient_static(lt_scene* s, const lt_params* p, const lt_render_opts* o, const float* dI,
                                   float* image, const lt_grads* g, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI || !image) return fail(LT_ERR_INVALID_ARG, "lt_naive_gradient_static: d_image or image is NULL");
  // bound the path count first (32 B per vertex) so that the size below cannot wrap
  const size_t need = o->n_paths > (int64_t)(LT_NAIVE_STATIC_BYTES / (32u * (unsigned)o->max_depth))
                          ? (size_t)-1
                          : lt_naive_workspace_bytes(o);
  if (need > (size_t)LT_NAIVE_STATIC_BYTES)
    return fail(LT_ERR_INVALID_ARG, "lt_naive_gradient_static: the tape needs " + std::to_string(need) +
                                        " bytes, more than the fixed scratch of " +
                                        std::to_string((size_t)LT_NAIVE_STATIC_BYTES) + " bytes (fewer paths or depth)");
  int dev = -1;
  LT_CUDA(cudaGetDevice(&dev));
  if (dev != s->device) return fail(LT_ERR_INVALID_ARG, "lt_naive_gradient_static: the scene's device is not current");
  void* tape = nullptr;
  v = static_tape(dev, &tape);
  if (v != LT_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  LT_CUDA(cudaMemsetAsync(image, 0, sizeof(float) * 3 * (size_t)s->dev.W * s->dev.H, st));
  GradPtrs gp;
  v = prep_grads(s, g, st, gp);
  if (v != LT_OK) return v;
  if (o->n_paths == 0) return LT_OK;
  const LaunchCfg L = cfg_for(s, o);
  cudaError_t e = launch_primal(dev_for(s, o), kparams(p, o), LT_EST_NAIVE, image, tape, L, st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_naive_gradient_static: ") + cudaGetErrorString(e));
  KParams kb = kparams(p, o);
  set_privatization(s, g, kb, o->scatter);
  e = launch_naive(dev_for(s, o), kb, o->attached != 0, s->has_dielectric, dI, tape, gp, L, st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_naive_gradient_static: ") + cudaGetErrorString(e));
  return LT_OK;
}

const char* lt_version(void) { return "liblt 0.1 (sm_103a)"; }

lt_status lt_scene_create(const lt_scene_desc* d, void* stream, lt_scene** out) {
  if (!out) return fail(LT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  lt_status v = validate_desc(d);
  if (v != LT_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  const int nq = d->n_quads, nt = d->n_tris, np = nq + nt;
  // host geometry at zero heights
  std::vector<HV> O(np), E1(np), E2(np);
  std::vector<Box> boxes(np);
  for (int i = 0; i < np; ++i) {
    HV o, e1, e2;
    if (i < nq) {
      const float* q = d->quads + 9 * i;
      o = hv(q[0], q[1], q[2]); e1 = hv(q[3], q[4], q[5]); e2 = hv(q[6], q[7], q[8]);
    } else {
      const int* t = d->tris + 3 * (i - nq);
      HV v0 = hv(d->verts[3 * t[0]], d->verts[3 * t[0] + 1], d->verts[3 * t[0] + 2]);
      HV v1 = hv(d->verts[3 * t[1]], d->verts[3 * t[1] + 1], d->verts[3 * t[1] + 2]);
      HV v2 = hv(d->verts[3 * t[2]], d->verts[3 * t[2] + 1], d->verts[3 * t[2] + 2]);
      o = v0; e1 = v1 - v0; e2 = v2 - v0;
    }
    O[i] = o; E1[i] = e1; E2[i] = e2;
    float pts[4][3] = {{o.x, o.y, o.z}, {o.x + e1.x, o.y + e1.y, o.z + e1.z}, {o.x + e2.x, o.y + e2.y, o.z + e2.z},
                       {o.x + e1.x + e2.x, o.y + e1.y + e2.y, o.z + e1.z + e2.z}};
    for (int k = 0; k < (i < nq ? 4 : 3); ++k) boxes[i].grow(pts[k]);
  }
  // Up to kDirect analytic quads (walls, emitters: few and large) are tested directly by
  // every ray; the BVH covers the remaining primitives.
  const int kDirect = 32;
  const int nd = nq <= kDirect ? nq : 0;
  std::vector<Box> bvh_boxes(boxes.begin() + nd, boxes.end());
  Builder B(bvh_boxes);
  if (np > nd) B.build(0, np - nd, 0);
  // flatten in depth-first preorder; leaves take consecutive slots of the leaf order
  std::vector<float4> node;
  std::vector<int2> range;
  std::vector<int> order;  // leaf order -> original primitive
  std::vector<int> pre;  // preorder of builder nodes
  if (!B.nodes.empty()) {
    std::vector<int> stk = {0};
    while (!stk.empty()) {
      int b = stk.back();
      stk.pop_back();
      pre.push_back(b);
      if (B.nodes[b].left >= 0) { stk.push_back(B.nodes[b].right); stk.push_back(B.nodes[b].left); }
    }
  }
  int nn = (int)pre.size();
  std::vector<int> flat_of(B.nodes.size());
  for (int i = 0; i < nn; ++i) flat_of[pre[i]] = i;
  // subtree sizes for skip indices
  std::vector<int> size(B.nodes.size(), 1);
  for (int i = nn - 1; i >= 0; --i) {
    const BNode& bn = B.nodes[pre[i]];
    if (bn.left >= 0) size[pre[i]] = 1 + size[bn.left] + size[bn.right];
  }
  node.resize(2 * nn);
  range.resize(nn);
  for (int i = 0; i < nn; ++i) {
    const BNode& bn = B.nodes[pre[i]];
    int skip = i + size[pre[i]];
    int leafinfo = 0;
    if (bn.left < 0) {
      int first = nd + (int)order.size();
      for (int k = bn.begin; k < bn.end; ++k) order.push_back(nd + B.idx[k]);
      leafinfo = (first << 8) | (bn.end - bn.begin);
    }
    node[2 * i] = make_float4(bn.box.lo[0], bn.box.lo[1], bn.box.lo[2], 0.0f);
    node[2 * i + 1] = make_float4(bn.box.hi[0], bn.box.hi[1], bn.box.hi[2], 0.0f);
    std::memcpy(&node[2 * i].w, &skip, 4);
    std::memcpy(&node[2 * i + 1].w, &leafinfo, 4);
  }
  // prim ranges: the builder kept each subtree contiguous in B.idx and leaves were
  // emitted in preorder, so build-order positions equal leaf-order positions
  for (int i = 0; i < nn; ++i) range[i] = make_int2(nd + B.nodes[pre[i]].begin, nd + B.nodes[pre[i]].end);
  for (int i = 0; i < np - nd; ++i)
    if (order[i] != nd + B.idx[i]) return fail(LT_ERR_INVALID_ARG, "internal: BVH leaf order mismatch");
  {
    std::vector<int> full(np);
    for (int i = 0; i < nd; ++i) full[i] = i;
    for (int i = nd; i < np; ++i) full[i] = order[i - nd];
    order.swap(full);
  }
  // leaf-order primitive arrays
  std::vector<float4> prim(3 * np), tri_base(3 * np, make_float4(0, 0, 0, 0));
  std::vector<int4> prim_h(np, make_int4(-1, -1, -1, -1));
  bool has_diel = false;
  int emitter_leaf = -1;
  for (int j = 0; j < np; ++j) {
    int i = order[j];
    int mat = d->prim_mat[i];
    int is_tri = i >= nq ? 1 : 0;
    float fm, fo, ft;
    std::memcpy(&fm, &mat, 4); std::memcpy(&fo, &i, 4); std::memcpy(&ft, &is_tri, 4);
    prim[3 * j] = make_float4(O[i].x, O[i].y, O[i].z, fm);
    prim[3 * j + 1] = make_float4(E1[i].x, E1[i].y, E1[i].z, fo);
    prim[3 * j + 2] = make_float4(E2[i].x, E2[i].y, E2[i].z, ft);
    if (is_tri) {
      const int* t = d->tris + 3 * (i - nq);
      for (int k = 0; k < 3; ++k)
        tri_base[3 * j + k] = make_float4(d->verts[3 * t[k]], d->verts[3 * t[k] + 1], d->verts[3 * t[k] + 2], 0.0f);
      prim_h[j] = make_int4(d->vert_h[t[0]], d->vert_h[t[1]], d->vert_h[t[2]], i);
    }
    if (d->mat_type[mat] == LT_MAT_DIELECTRIC) has_diel = true;
    if (i == d->emitter_quad) emitter_leaf = j;
  }
  std::vector<int4> mats(d->n_mats);
  std::vector<float> iors(d->n_mats);
  for (int m = 0; m < d->n_mats; ++m) {
    mats[m] = make_int4(d->mat_type[m], d->mat_tex_off[m], d->mat_tex_w[m], d->mat_tex_h[m]);
    iors[m] = d->mat_ior[m];
  }
  lt_scene* s = new lt_scene();
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  if (cudaDeviceGetAttribute(&s->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device) != cudaSuccess ||
      s->smem_optin < 48 * 1024)
    s->smem_optin = 48 * 1024;
  s->n_albedo = d->n_albedo;
  s->n_heights = d->n_heights;
  s->has_dielectric = has_diel;
  s->n_nodes = nn;
  s->n_prims = np;
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  cudaError_t e = cudaSuccess;
  if (!e) e = up((void**)&s->d_prim, prim.data(), prim.size() * sizeof(float4));
  if (!e) e = up((void**)&s->d_prim_h, prim_h.data(), prim_h.size() * sizeof(int4));
  if (!e) e = up((void**)&s->d_tri_base, tri_base.data(), tri_base.size() * sizeof(float4));
  if (!e) e = up((void**)&s->d_node, node.data(), node.size() * sizeof(float4));
  if (!e) e = up((void**)&s->d_range, range.data(), range.size() * sizeof(int2));
  std::vector<int> big;
  for (int i = 0; i < nn; ++i)
    if (range[i].y - range[i].x > kRefitBig) big.push_back(i);
  s->n_big = (int)big.size();
  if (!e && !big.empty()) e = up((void**)&s->d_big, big.data(), big.size() * sizeof(int));
  if (!e) e = up((void**)&s->d_mat, mats.data(), mats.size() * sizeof(int4));
  if (!e) e = up((void**)&s->d_ior, iors.data(), iors.size() * sizeof(float));
  for (int k = 0; k < 2 && !e; ++k) {
    const int W = k == 0 ? 4 : 8;
    std::vector<int> codes, wmap;
    collapse_wide(B, W, nd, flat_of, codes, wmap);
    const int nw = (int)codes.size() / W;
    s->n_wnodes[k] = nw;
    std::vector<float> wn((size_t)nw * 8 * W, 0.0f);  // boxes are written by the refit
    for (int j = 0; j < nw; ++j)
      for (int c = 0; c < W; ++c) std::memcpy(&wn[(size_t)j * 8 * W + 6 * W + c], &codes[j * W + c], 4);
    if (nw > 0) {
      e = up((void**)&s->d_wnode[k], wn.data(), wn.size() * sizeof(float));
      if (!e) e = up((void**)&s->d_wmap[k], wmap.data(), wmap.size() * sizeof(int));
    }
  }
  if (!e) e = cudaMalloc((void**)&s->d_err, sizeof(int) * 4);
  if (!e) e = cudaMemsetAsync(s->d_err, 0, sizeof(int) * 4, st);
  if (e) {
    free_scene(s);
    return fail(e == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA,
                std::string("lt_scene_create: ") + cudaGetErrorString(e));
  }
  DevScene& S = s->dev;
  S.width = 2;
  S.prim = s->d_prim; S.prim_h = s->d_prim_h; S.node = s->d_node; S.n_nodes = nn; S.n_prims = np;
  S.n_direct = nd;
  S.mat = s->d_mat; S.mat_ior = s->d_ior; S.emitter_prim = emitter_leaf; S.err = s->d_err;
  const float* q = d->quads + 9 * d->emitter_quad;
  HV lo = hv(q[0], q[1], q[2]), le1 = hv(q[3], q[4], q[5]), le2 = hv(q[6], q[7], q[8]);
  HV lnr = hcross(le1, le2);
  HV ln = hnorm(lnr);
  S.lo = make_float3(lo.x, lo.y, lo.z); S.le1 = make_float3(le1.x, le1.y, le1.z);
  S.le2 = make_float3(le2.x, le2.y, le2.z); S.ln = make_float3(ln.x, ln.y, ln.z);
  S.light_area = std::sqrt(hdot(lnr, lnr));
  HV cp = hv(d->cam_pos[0], d->cam_pos[1], d->cam_pos[2]);
  HV look = hv(d->cam_look[0], d->cam_look[1], d->cam_look[2]);
  HV upv = hv(d->cam_up[0], d->cam_up[1], d->cam_up[2]);
  HV cf = hnorm(look - cp), cr = hnorm(hcross(cf, upv)), cu = hcross(cr, cf);
  S.cpos = make_float3(cp.x, cp.y, cp.z); S.cf = make_float3(cf.x, cf.y, cf.z);
  S.cr = make_float3(cr.x, cr.y, cr.z); S.cu = make_float3(cu.x, cu.y, cu.z);
  double tany = std::tan(0.5 * d->fov_y_deg * 3.14159265358979323846 / 180.0);
  double tanx = tany * d->width / d->height;
  S.tanx = (float)tanx; S.tany = (float)tany;
  S.K0 = (float)((double)d->width * d->height / (4.0 * tanx * tany * 3.14159265358979323846));
  S.W = d->width; S.H = d->height;
  // initial bounds
  RefitArgs ra = refit_args(s, nullptr);
  e = launch_refit(ra, st);
  if (e) { free_scene(s); return fail(LT_ERR_CUDA, std::string("refit: ") + cudaGetErrorString(e)); }
  *out = s;
  return LT_OK;
}

lt_status lt_scene_refit(lt_scene* s, const float* heights, void* stream) {
  if (!s) return fail(LT_ERR_INVALID_ARG, "scene is NULL");
  if (s->n_heights > 0 && !heights) return fail(LT_ERR_INVALID_ARG, "heights is NULL");
  cudaError_t e = launch_refit(refit_args(s, heights), (cudaStream_t)stream);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_scene_refit: ") + cudaGetErrorString(e));
  return LT_OK;
}

void lt_scene_destroy(lt_scene* s) { free_scene(s); }

size_t lt_record_size(const lt_render_opts*) { return 32; }

size_t lt_lrb2_buffer_bytes(const lt_render_opts* o) {
  if (!o || o->n_paths < 0 || o->n_paths > LT_MAX_PATHS || o->max_depth < 1 || o->max_depth > kMaxDepth) return 0;
  return lrb2_layout(o->n_paths, o->max_depth).total;
}

size_t lt_lrb3_state_bytes(const lt_render_opts* o) {
  if (!o || o->n_paths < 0 || o->n_paths > LT_MAX_PATHS) return 0;
  return lrb3_state_bytes(o->n_paths);
}

size_t lt_naive_workspace_bytes(const lt_render_opts* o) {
  if (!o || o->n_paths < 0 || o->n_paths > LT_MAX_PATHS || o->max_depth < 1 || o->max_depth > kMaxDepth) return 0;
  size_t head = ((size_t)o->n_paths * sizeof(int) + 255) & ~(size_t)255;
  return head + (size_t)o->n_paths * (size_t)o->max_depth * 32;
}

namespace {
// Order of the plain primal's paths: a counting sort by the cell of the path's first direction
// (64 x 64 cells of the two uniforms of the emitter's cosine sample, Eq. 2), so that the lanes
// of a warp, and the warps running at the same time, trace first rays that leave in similar
// directions, and so do their next few rays (measured on the caustic: cells of the emitter
// point as well, 16 x 16 x 4 x 4 or 32 x 32 x 2 x 2, were slightly slower).  Every
// path's result depends only on its index, so the order changes no result, only the
// coherence of the traversals (and, through the path list, of LRB-3 passes 2 and 3).
__device__ __forceinline__ int sort_key(uint64_t seed, uint64_t n) {
  const float4 r = rand4(seed, n, 0);
  const int a = min((int)(r.z * 64.0f), 63), b = min((int)(r.w * 64.0f), 63);
  return a * 64 + b;
}
__device__ __forceinline__ int64_t sort_range(int64_t n, int blk) {
  return (n + kSortBlocks - 1) / kSortBlocks * blk;
}
// counts[bin][block] of the block's contiguous range of paths
__global__ void __launch_bounds__(1024) k_sort_count(uint64_t seed, uint64_t off, int64_t n, unsigned* counts) {
  __shared__ unsigned h[kSortBins];
  for (int i = threadIdx.x; i < kSortBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t lo = min(sort_range(n, blockIdx.x), n), hi = min(sort_range(n, blockIdx.x + 1), n);
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) atomicAdd(&h[sort_key(seed, off + p)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kSortBins; i += blockDim.x) counts[(size_t)i * kSortBlocks + blockIdx.x] = h[i];
}
// exclusive scan of counts in bin-major order: one thread per bin scans its blocks, then one
// block scans the bins' totals into the bin starts
__global__ void __launch_bounds__(256) k_sort_rows(unsigned* counts, unsigned* totals) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= kSortBins) return;
  unsigned* row = counts + (size_t)bin * kSortBlocks;
  unsigned acc = 0;
  for (int b = 0; b < kSortBlocks; ++b) {
    const unsigned v = row[b];
    row[b] = acc;
    acc += v;
  }
  totals[bin] = acc;
}
__global__ void __launch_bounds__(1024) k_sort_bins(unsigned* totals) {
  __shared__ unsigned wsum[32];
  constexpr int per = kSortBins / 1024;
  unsigned loc = 0;
  for (int j = 0; j < per; ++j) loc += totals[threadIdx.x * per + j];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const unsigned w = wsum[lane];
    unsigned wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    wsum[lane] = wi - w;
  }
  __syncthreads();
  unsigned run = wsum[wid] + inc - loc;
  for (int j = 0; j < per; ++j) {
    const unsigned c = totals[threadIdx.x * per + j];
    totals[threadIdx.x * per + j] = run;
    run += c;
  }
}
// each block places its range's paths at bin start + its blocks-before offset + rank
__global__ void __launch_bounds__(1024) k_sort_place(uint64_t seed, uint64_t off, int64_t n, const unsigned* counts,
                                                     const unsigned* starts, uint32_t* order) {
  __shared__ unsigned at[kSortBins];
  for (int i = threadIdx.x; i < kSortBins; i += blockDim.x)
    at[i] = starts[i] + counts[(size_t)i * kSortBlocks + blockIdx.x];
  __syncthreads();
  const int64_t lo = min(sort_range(n, blockIdx.x), n), hi = min(sort_range(n, blockIdx.x + 1), n);
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x)
    order[atomicAdd(&at[sort_key(seed, off + p)], 1u)] = (uint32_t)p;
}
}  // namespace

lt_status lt_primal(lt_scene* s, const lt_params* p, const lt_render_opts* o, int est, float* image, void* aux,
                    size_t aux_bytes, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!image) return fail(LT_ERR_INVALID_ARG, "image is NULL");
  if (est < LT_EST_PLAIN || est > LT_EST_BUFFERED) return fail(LT_ERR_INVALID_ARG, "unknown estimator");
  if (est == LT_EST_RESLRB && (!aux || aux_bytes < (size_t)o->n_paths * lt_record_size(o)))
    return fail(LT_ERR_INVALID_ARG, "ResLRB records buffer missing or too small");
  if (est == LT_EST_NAIVE && (!aux || aux_bytes < lt_naive_workspace_bytes(o)))
    return fail(LT_ERR_OOM, "naive-AD workspace missing or smaller than lt_naive_workspace_bytes()");
  if (est == LT_EST_BUFFERED && (!aux || aux_bytes < lt_lrb2_buffer_bytes(o)))
    return fail(LT_ERR_OOM, "buffered two-pass buffer missing or smaller than lt_lrb2_buffer_bytes()");
  if (est == LT_EST_PLAIN && o->lrb3_state && o->lrb3_state_bytes < lt_lrb3_state_bytes(o))
    return fail(LT_ERR_INVALID_ARG, "lrb3_state smaller than lt_lrb3_state_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  LT_CUDA(cudaMemsetAsync(image, 0, sizeof(float) * 3 * (size_t)s->dev.W * s->dev.H, st));
  if (o->n_paths == 0) return LT_OK;
  KParams kp = kparams(p, o);
  if (est == LT_EST_PLAIN && o->lrb3_state) {
    kp.vstate = o->lrb3_state;
    kp.conn1 = (float4*)((char*)o->lrb3_state + lrb3_state_conn4(o->n_paths));
    kp.conn1z = (float*)((char*)o->lrb3_state + lrb3_state_connz(o->n_paths));
    if (o->n_paths <= kListMaxPaths) {
      // the list of the paths with a valid connection, for LRB-3 passes 2 and 3
      char* base = (char*)o->lrb3_state;
      kp.list = (uint32_t*)(base + lrb3_state_list(o->n_paths));
      kp.list_n = (unsigned long long*)(base + lrb3_state_count(o->n_paths));
      kp.ticket = kp.list_n + 1;  // the primal's chunk counter (the backward zeroes it again)
      LT_CUDA(cudaMemsetAsync(kp.list_n, 0, 2 * sizeof(unsigned long long), st));
      // the order of the paths (see sort_key)
      uint32_t* order = (uint32_t*)(base + lrb3_state_order(o->n_paths));
      unsigned* counts = (unsigned*)(base + lrb3_state_sort(o->n_paths));
      unsigned* starts = counts + (size_t)kSortBins * kSortBlocks;
      const uint64_t off = (uint64_t)o->path_offset;
      k_sort_count<<<kSortBlocks, 1024, 0, st>>>(o->seed, off, o->n_paths, counts);
      k_sort_rows<<<kSortBins / 256, 256, 0, st>>>(counts, starts);
      k_sort_bins<<<1, 1024, 0, st>>>(starts);
      k_sort_place<<<kSortBlocks, 1024, 0, st>>>(o->seed, off, o->n_paths, counts, starts, order);
      LT_CUDA(cudaGetLastError());
      kp.order = order;
    }
  }
  cudaError_t e = launch_primal(dev_for(s, o), kp, est, image, aux, cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_primal: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_backward_lrb3(lt_scene* s, const lt_params* p, const lt_render_opts* o, const float* dI,
                           const lt_grads* g, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI) return fail(LT_ERR_INVALID_ARG, "d_image is NULL");
  if (o->lrb3_state && o->lrb3_state_bytes < lt_lrb3_state_bytes(o))
    return fail(LT_ERR_INVALID_ARG, "lrb3_state smaller than lt_lrb3_state_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  GradPtrs gp;
  v = prep_grads(s, g, st, gp);
  if (v != LT_OK) return v;
  if (o->n_paths == 0) return LT_OK;
  KParams kp = kparams(p, o);
  set_privatization(s, g, kp, o->scatter);
  if (o->literal) {
    if (!o->attached) return fail(LT_ERR_INVALID_ARG, "the literal transport is for attached gradients");
    cudaError_t e = launch_lrb3_literal(dev_for(s, o), kp, dI, gp, cfg_for(s, o), st);
    if (e) return fail(LT_ERR_CUDA, std::string("lt_backward_lrb3: ") + cudaGetErrorString(e));
    return LT_OK;
  }
  if (o->lrb3_state && o->lrb3_mask_ready) {
    // the primal recorded each path's first valid connection: pass 2 takes delta_total of a
    // path with one valid connection from it
    kp.conn1 = (float4*)((char*)o->lrb3_state + lrb3_state_conn4(o->n_paths));
    kp.conn1z = (float*)((char*)o->lrb3_state + lrb3_state_connz(o->n_paths));
  }
  if (o->lrb3_state && o->lrb3_mask_ready && o->n_paths <= kListMaxPaths) {
    // the primal listed the paths with a valid connection: passes 2 and 3 visit only those
    char* base = (char*)o->lrb3_state;
    kp.list = (uint32_t*)(base + lrb3_state_list(o->n_paths));
    kp.list_n = (unsigned long long*)(base + lrb3_state_count(o->n_paths));
    kp.ticket = kp.list_n + 1;
    LT_CUDA(cudaMemsetAsync(kp.ticket, 0, 2 * sizeof(unsigned long long), st));
  }
  cudaError_t e = launch_lrb3(dev_for(s, o), kp, o->attached != 0, s->has_dielectric, dI, gp,
                              o->lrb3_state, o->lrb3_state && o->lrb3_mask_ready, cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_backward_lrb3: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_backward_reslrb(lt_scene* s, const lt_params* p, const lt_render_opts* o, const float* dI,
                             const void* rec, const lt_grads* g, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI || !rec) return fail(LT_ERR_INVALID_ARG, "d_image or records is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  GradPtrs gp;
  v = prep_grads(s, g, st, gp);
  if (v != LT_OK) return v;
  if (o->n_paths == 0) return LT_OK;
  KParams kp = kparams(p, o);
  set_privatization(s, g, kp, o->scatter);
  cudaError_t e = launch_reslrb(dev_for(s, o), kp, o->attached != 0, s->has_dielectric, dI, rec, gp, cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_backward_reslrb: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_backward_lrb2(lt_scene* s, const lt_params* p, const lt_render_opts* o, const float* dI, void* buf,
                           size_t buf_bytes, const lt_grads* g, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI) return fail(LT_ERR_INVALID_ARG, "d_image is NULL");
  if (!buf || buf_bytes < lt_lrb2_buffer_bytes(o))
    return fail(LT_ERR_OOM, "buffered two-pass buffer missing or smaller than lt_lrb2_buffer_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  GradPtrs gp;
  v = prep_grads(s, g, st, gp);
  if (v != LT_OK) return v;
  if (o->n_paths == 0) return LT_OK;
  KParams kp = kparams(p, o);
  set_privatization(s, g, kp, o->scatter);
  cudaError_t e = launch_lrb2(dev_for(s, o), kp, o->attached != 0, s->has_dielectric, dI, buf, gp,
                              cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_backward_lrb2: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_backward_naive(lt_scene* s, const lt_params* p, const lt_render_opts* o, const float* dI,
                            const void* ws, size_t ws_bytes, const lt_grads* g, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI) return fail(LT_ERR_INVALID_ARG, "d_image is NULL");
  if (!ws || ws_bytes < lt_naive_workspace_bytes(o))
    return fail(LT_ERR_OOM, "naive-AD workspace missing or smaller than lt_naive_workspace_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  GradPtrs gp;
  v = prep_grads(s, g, st, gp);
  if (v != LT_OK) return v;
  if (o->n_paths == 0) return LT_OK;
  KParams kp = kparams(p, o);
  set_privatization(s, g, kp, o->scatter);
  cudaError_t e = launch_naive(dev_for(s, o), kp, o->attached != 0, s->has_dielectric, dI, ws, gp, cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_backward_naive: ") + cudaGetErrorString(e));
  return LT_OK;
}

namespace {
lt_status check_bidir(const lt_scene* s, const lt_render_opts* o, const lt_bidir_opts* b, BidirArgs& ba) {
  if (!b) return fail(LT_ERR_INVALID_ARG, "bidir opts is NULL");
  if (b->n_cam < 0 || b->n_cam > LT_MAX_PATHS) return fail(LT_ERR_INVALID_ARG, "n_cam must be in 0..2^40");
  if (o->attached) return fail(LT_ERR_UNSUPPORTED, "the bidirectional estimator is detached only");
  if (s->has_dielectric) return fail(LT_ERR_UNSUPPORTED, "the bidirectional estimator needs a scene without dielectrics");
  if (o->rr_depth > 0) return fail(LT_ERR_UNSUPPORTED, "the bidirectional estimator has no Russian roulette");
  ba.N = (float)(o->n_norm > 0 ? o->n_norm : o->n_paths);
  ba.M = (float)b->n_cam;
  ba.n_cam = b->n_cam;
  ba.cam_mask = b->cam_mask;
  ba.cam_hash = b->cam_hash;
  return LT_OK;
}
}  // namespace

lt_status lt_bidir_primal(lt_scene* s, const lt_params* p, const lt_render_opts* o, const lt_bidir_opts* b,
                          float* image, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!image) return fail(LT_ERR_INVALID_ARG, "image is NULL");
  BidirArgs ba;
  v = check_bidir(s, o, b, ba);
  if (v != LT_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  LT_CUDA(cudaMemsetAsync(image, 0, sizeof(float) * 3 * (size_t)s->dev.W * s->dev.H, st));
  if (o->n_paths == 0 && b->n_cam == 0) return LT_OK;
  cudaError_t e = launch_bidir(dev_for(s, o), kparams(p, o), ba, false, image, nullptr, GradPtrs{},
                               cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_bidir_primal: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_bidir_backward(lt_scene* s, const lt_params* p, const lt_render_opts* o, const lt_bidir_opts* b,
                            const float* dI, const lt_grads* g, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI) return fail(LT_ERR_INVALID_ARG, "d_image is NULL");
  BidirArgs ba;
  v = check_bidir(s, o, b, ba);
  if (v != LT_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GradPtrs gp;
  v = prep_grads(s, g, st, gp);
  if (v != LT_OK) return v;
  if (o->n_paths == 0 && b->n_cam == 0) return LT_OK;
  KParams kp = kparams(p, o);
  set_privatization(s, g, kp, o->scatter);
  kp.n_h = 0;  // detached: no height gradients
  kp.priv_n = kp.n_alb;
  cudaError_t e = launch_bidir(dev_for(s, o), kp, ba, true, nullptr, dI, gp, cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_bidir_backward: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_film_l2(const float* I, const float* T, int64_t n, float* dI, float* loss, void* stream) {
  if (!I || !T || !dI || !loss || n <= 0) return fail(LT_ERR_INVALID_ARG, "lt_film_l2: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  LT_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
  cudaError_t e = launch_film_l2(I, T, n, dI, loss, sms, st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_film_l2: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_mlp_collect(lt_scene* s, const lt_params* p, const lt_render_opts* o, const float* dI, float tfloor,
                         float* feats, float* targets, int64_t cap, int64_t* count, void* stream) {
  lt_status v = check_opts(s, p, o);
  if (v != LT_OK) return v;
  if (!dI || !count || (cap > 0 && (!feats || !targets)) || cap < 0)
    return fail(LT_ERR_INVALID_ARG, "lt_mlp_collect: bad buffers");
  if (!(tfloor >= 0)) return fail(LT_ERR_INVALID_ARG, "lt_mlp_collect: target_floor must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  LT_CUDA(cudaMemsetAsync(count, 0, sizeof(int64_t), st));
  if (o->n_paths == 0) return LT_OK;
  cudaError_t e = launch_collect(dev_for(s, o), kparams(p, o), dI, tfloor, feats, targets, cap, (unsigned long long*)count,
                                 cfg_for(s, o), st);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_mlp_collect: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_mlp_init_stats(float* mlp, const float* feats, const float* targets, int64_t n, void* stream) {
  if (!mlp || !feats || !targets || n <= 1) return fail(LT_ERR_INVALID_ARG, "lt_mlp_init_stats: bad arguments");
  cudaError_t e = launch_mlp_moments(feats, targets, n, mlp, (cudaStream_t)stream);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_mlp_init_stats: ") + cudaGetErrorString(e));
  return LT_OK;
}

static int device_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

lt_status lt_mlp_grad(const float* mlp, const float* feats, const float* targets, int64_t n, int64_t batch,
                      float* grad, float* loss, void* stream) {
  if (!mlp || !grad || n < 0 || batch <= 0 || n > batch || (n > 0 && (!feats || !targets)))
    return fail(LT_ERR_INVALID_ARG, "lt_mlp_grad: bad arguments");
  if (n == 0) return LT_OK;
  cudaError_t e = launch_mlp_grad(mlp, feats, targets, n, 1.0f / (float)batch, grad, loss, device_sms(),
                                  (cudaStream_t)stream);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_mlp_grad: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_mlp_adam(float* mlp, float* m, float* v, const float* grad, int step, float lr, void* stream) {
  if (!mlp || !m || !v || !grad || step < 1 || !(lr > 0)) return fail(LT_ERR_INVALID_ARG, "lt_mlp_adam: bad arguments");
  cudaError_t e = launch_mlp_adam(mlp, m, v, grad, step, lr, (cudaStream_t)stream);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_mlp_adam: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_mlp_forward(const float* mlp, const float* feats, int64_t n, float* out, void* stream) {
  if (!mlp || n < 0 || (n > 0 && (!feats || !out))) return fail(LT_ERR_INVALID_ARG, "lt_mlp_forward: bad arguments");
  if (n == 0) return LT_OK;
  cudaError_t e = launch_mlp_forward(mlp, feats, n, out, device_sms(), (cudaStream_t)stream);
  if (e) return fail(LT_ERR_CUDA, std::string("lt_mlp_forward: ") + cudaGetErrorString(e));
  return LT_OK;
}

lt_status lt_sync_status(lt_scene* s, void* stream) {
  if (!s) return fail(LT_ERR_INVALID_ARG, "scene is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  LT_CUDA(cudaStreamSynchronize(st));
  int h = 0;
  LT_CUDA(cudaMemcpy(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  LT_CUDA(cudaMemset(s->d_err, 0, sizeof(int)));
  if (h & ERR_TIMEOUT) return fail(LT_ERR_TIMEOUT, "a bounded device wait timed out");
  if (h) return fail(LT_ERR_DEVICE_CHECK, "device-side check failed (bits " + std::to_string(h) + ")");
  return LT_OK;
}

// ------------------------------------------------------------------ batched passes
}  // extern "C"

// Kernel groups of a batch: the specular-chain variant of the attached backward kernels
// needs about twice the registers of the lean variant (half the resident warps), so only
// items that can form chains (attached, scene with dielectrics) run it.  The item table
// holds the lean group first, then the chain group; the backward passes launch one
// persistent kernel per non-empty group, as two parallel branches of the pass's graph.
struct lt_batch {
  int device = 0, sms = 1;
  std::vector<lt_batch_item> items;  // table order (lean group, then chain group)
  int n_lean = 0;                    // items [0, n_lean) form the lean group
  bool att_lean = false, all_rec = true;
  // every item carries an LRB-3 state: the LRB-3 pass runs pass 2 (all items) and pass 3
  // (per group) as separate launches; mask_ready: pass 2 reuses the primal pass's masks
  bool all_state = true, mask_ready = true;
  // one item table per chunk size (32 * paths_per_thread, paths_per_thread = 1, 2, 4, 8)
  // and BVH width (2, 4, 8): only the first-chunk indices and the scenes' BVH selection
  // differ, and a configuration change must not rewrite a table that a running pass may
  // still read
  BatchJob* d_jobs[12] = {};
  int64_t n_chunks[4] = {};   // whole batch
  int64_t split[4] = {};      // first chunk of the chain group
  unsigned long long* d_ticket = nullptr;  // [4 passes][3 launches]
  // pass-3 spans of the lean and the specular-chain group, and the gradient-sink size
  BatchSpan* d_spans[2] = {};
  int n_spans[2] = {};
  size_t span_smem = 0;
  cudaStream_t cap = nullptr, cap2 = nullptr;  // capture streams (main, second branch)
  cudaEvent_t fork = nullptr, join = nullptr;
  lt_batch_config cfg{128, 4, 0, 4};
  cudaGraphExec_t exec[4] = {};
};

namespace {

int ppt_slot(int ppt) { return ppt == 1 ? 0 : ppt == 2 ? 1 : ppt == 4 ? 2 : ppt == 8 ? 3 : -1; }
int width_slot(int w) { return w == 2 ? 0 : w == 4 ? 1 : w == 8 ? 2 : -1; }
int table_of(const lt_batch_config& c) { return 3 * ppt_slot(c.paths_per_thread) + width_slot(c.bvh_width); }

void drop_graphs(lt_batch* b) {
  for (auto& e : b->exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
}

void free_batch(lt_batch* b) {
  if (!b) return;
  drop_graphs(b);
  for (auto* j : b->d_jobs) cudaFree(j);
  for (auto* sp : b->d_spans) cudaFree(sp);
  cudaFree(b->d_ticket);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

lt_status check_batch_cfg(const lt_batch_config* c) {
  if (!c) return fail(LT_ERR_INVALID_ARG, "config is NULL");
  if (c->block_size != 64 && c->block_size != 128 && c->block_size != 256)
    return fail(LT_ERR_INVALID_ARG, "block_size must be 64, 128 or 256");
  if (ppt_slot(c->paths_per_thread) < 0) return fail(LT_ERR_INVALID_ARG, "paths_per_thread must be 1, 2, 4 or 8");
  if (c->blocks_per_sm < 0 || c->blocks_per_sm > 32) return fail(LT_ERR_INVALID_ARG, "blocks_per_sm must be in 0..32");
  if (width_slot(c->bvh_width) < 0) return fail(LT_ERR_INVALID_ARG, "bvh_width must be 2, 4 or 8");
  return LT_OK;
}

int kernel_pass(int pass) {
  return pass == LT_PASS_PRIMAL ? BPASS_PRIMAL
         : pass == LT_PASS_PRIMAL_RESLRB ? BPASS_PRIMAL_RES
         : pass == LT_PASS_LRB3 ? BPASS_LRB3 : BPASS_RESLRB;
}

// One persistent launch over the items [j0, j1) of the table: kernel `kpass` (BatchPass,
// or kSpanPass: pass 3 over the group's spans), queue ticket `slot` of its pass.
constexpr int kSpanPass = 100;
struct GroupLaunch {
  int j0 = 0, j1 = 0;
  int64_t c0 = 0, c1 = 0;  // chunk range
  bool att = false, chains = false;
  int kpass = 0, slot = 0;
  int per_sm = 0;
};

std::vector<GroupLaunch> plan_pass(const lt_batch* b, int pass) {
  const int slot = ppt_slot(b->cfg.paths_per_thread);
  const int n = (int)b->items.size();
  std::vector<GroupLaunch> out;
  const bool primal = pass == LT_PASS_PRIMAL || pass == LT_PASS_PRIMAL_RESLRB;
  const int kp = kernel_pass(pass);
  if (primal) {
    out.push_back(GroupLaunch{0, n, 0, b->n_chunks[slot], false, false, kp, 0, 0});
  } else if (pass == LT_PASS_LRB3 && b->all_state) {
    const int p2 = b->mask_ready ? BPASS_LRB3_P2_MASK : BPASS_LRB3_P2;
    out.push_back(GroupLaunch{0, n, 0, b->n_chunks[slot], false, false, p2, 2, 0});
    out.push_back(GroupLaunch{0, b->n_lean, 0, b->n_spans[0], b->att_lean, false, kSpanPass, 0, 0});
    out.push_back(GroupLaunch{b->n_lean, n, 0, b->n_spans[1], true, true, kSpanPass, 1, 0});
  } else {
    out.push_back(GroupLaunch{0, b->n_lean, 0, b->split[slot], b->att_lean, false, kp, 0, 0});
    out.push_back(GroupLaunch{b->n_lean, n, b->split[slot], b->n_chunks[slot], true, true, kp, 1, 0});
  }
  std::vector<GroupLaunch> keep;
  for (GroupLaunch& g : out) {
    if (g.c1 <= g.c0) continue;
    g.per_sm = b->cfg.blocks_per_sm > 0 ? b->cfg.blocks_per_sm
               : g.kpass == kSpanPass
                   ? batch_spans_occupancy(b->cfg.bvh_width, g.att, g.chains, b->cfg.block_size, b->span_smem)
                   : batch_occupancy(b->cfg.bvh_width, g.kpass, g.att, g.chains, b->cfg.block_size);
    keep.push_back(g);
  }
  return keep;
}

lt_status launch_group(lt_batch* b, int pass, const GroupLaunch& g, cudaStream_t st) {
  unsigned long long* ticket = b->d_ticket + 3 * pass + g.slot;
  LT_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), st));
  const int block = b->cfg.block_size;
  if (g.kpass == kSpanPass) {
    // a resident grid, but no more blocks than spans
    const int64_t grid = std::min<int64_t>((int64_t)b->sms * g.per_sm, g.c1);
    cudaError_t e = launch_batch_spans(b->cfg.bvh_width, g.att, g.chains, b->d_jobs[table_of(b->cfg)],
                                       b->d_spans[g.slot], (int)g.c1, ticket, block,
                                       (int)std::max<int64_t>(grid, 1), b->span_smem, st);
    if (e) return fail(LT_ERR_CUDA, std::string("batched pass 3: ") + cudaGetErrorString(e));
    return LT_OK;
  }
  // a resident grid, but no more warps than chunks
  const int64_t nch = g.c1 - g.c0;
  const int64_t warps_per_block = block / 32;
  int64_t grid = std::min<int64_t>((int64_t)b->sms * g.per_sm, (nch + warps_per_block - 1) / warps_per_block);
  BatchArgs a{b->d_jobs[table_of(b->cfg)] + g.j0, g.j1 - g.j0, 32 * b->cfg.paths_per_thread, g.c0, nch, ticket};
  cudaError_t e = launch_batch(b->cfg.bvh_width, g.kpass, g.att, g.chains, a, block, (int)std::max<int64_t>(grid, 1),
                               st);
  if (e) return fail(LT_ERR_CUDA, std::string("batched pass: ") + cudaGetErrorString(e));
  return LT_OK;
}

// Enqueue one pass on `st`: clears and refits of every item, a pass-2 launch if the plan
// has one, then the group launches (a second group runs on a forked branch `st2`, joined
// back into `st`).
lt_status enqueue_pass(lt_batch* b, int pass, const std::vector<GroupLaunch>& full_plan, cudaStream_t st,
                       cudaStream_t st2) {
  const bool primal = pass == LT_PASS_PRIMAL || pass == LT_PASS_PRIMAL_RESLRB;
  for (const lt_batch_item& it : b->items) {
    const lt_scene* s = it.scene;
    if (primal) {
      if (it.heights && s->n_heights > 0) {
        cudaError_t e = launch_refit(refit_args(s, it.heights), st);
        if (e) return fail(LT_ERR_CUDA, std::string("batch refit: ") + cudaGetErrorString(e));
      }
      LT_CUDA(cudaMemsetAsync(it.image, 0, sizeof(float) * 3 * (size_t)s->dev.W * s->dev.H, st));
    } else {
      GradPtrs gp;
      lt_status v = prep_grads(s, &it.grads, st, gp);
      if (v != LT_OK) return v;
    }
  }
  std::vector<GroupLaunch> plan;
  for (const GroupLaunch& g : full_plan) {
    if (g.kpass == BPASS_LRB3_P2 || g.kpass == BPASS_LRB3_P2_MASK) {
      lt_status v = launch_group(b, pass, g, st);  // pass 2 of every item before any pass 3
      if (v != LT_OK) return v;
    } else {
      plan.push_back(g);
    }
  }
  if (plan.size() == 2) {
    LT_CUDA(cudaEventRecord(b->fork, st));
    LT_CUDA(cudaStreamWaitEvent(st2, b->fork, 0));
    lt_status v = launch_group(b, pass, plan[1], st2);
    if (v != LT_OK) return v;
    LT_CUDA(cudaEventRecord(b->join, st2));
  }
  if (!plan.empty()) {
    lt_status v = launch_group(b, pass, plan[0], st);
    if (v != LT_OK) return v;
  }
  if (plan.size() == 2) LT_CUDA(cudaStreamWaitEvent(st, b->join, 0));
  return LT_OK;
}

// Capture the pass on the batch's own streams and instantiate it.
lt_status capture_pass(lt_batch* b, int pass) {
  const std::vector<GroupLaunch> plan = plan_pass(b, pass);
  for (const GroupLaunch& g : plan)
    if (g.per_sm < 1) return fail(LT_ERR_CUDA, "batched kernel cannot be resident at this block size");
  LT_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  lt_status v = enqueue_pass(b, pass, plan, b->cap, b->cap2);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (v != LT_OK) {
    if (g) cudaGraphDestroy(g);
    return v;
  }
  if (e != cudaSuccess) return fail(LT_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec[pass], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec[pass] = nullptr;
    return fail(LT_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  }
  return LT_OK;
}

lt_status check_pass(const lt_batch* b, int pass) {
  if (!b) return fail(LT_ERR_INVALID_ARG, "batch is NULL");
  if (pass < LT_PASS_PRIMAL || pass > LT_PASS_RESLRB) return fail(LT_ERR_INVALID_ARG, "unknown pass");
  if ((pass == LT_PASS_PRIMAL_RESLRB || pass == LT_PASS_RESLRB) && !b->all_rec)
    return fail(LT_ERR_INVALID_ARG, "a ResLRB pass needs records for every item");
  return LT_OK;
}

}  // namespace

extern "C" {

lt_status lt_batch_create(const lt_batch_item* items, int n, void* stream, lt_batch** out) {
  if (!out) return fail(LT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!items || n < 1) return fail(LT_ERR_INVALID_ARG, "need at least one item");
  int dev = 0;
  LT_CUDA(cudaGetDevice(&dev));
  std::unique_ptr<lt_batch, void (*)(lt_batch*)> b(new lt_batch, free_batch);
  b->device = dev;
  std::vector<lt_batch_item> lean, chain;
  for (int i = 0; i < n; ++i) {
    lt_batch_item it = items[i];
    const std::string at = "item " + std::to_string(i) + ": ";
    if (!it.scene) return fail(LT_ERR_INVALID_ARG, at + "scene is NULL");
    if (it.scene->device != dev) return fail(LT_ERR_INVALID_ARG, at + "scene is on another device");
    // launch shape and the learned target are batch-wide; the census is single-scene only
    it.opts.block_size = 0;
    it.opts.blocks_per_sm = 0;
    it.opts.target = LT_TARGET_LUMINANCE;
    it.opts.mlp = nullptr;
    it.opts.census = nullptr;
    it.opts.bvh_width = 0;
    if (it.opts.lrb3_state && it.opts.lrb3_state_bytes < lt_lrb3_state_bytes(&it.opts))
      return fail(LT_ERR_INVALID_ARG, at + "lrb3_state smaller than lt_lrb3_state_bytes()");
    lt_status v = check_opts(it.scene, &it.params, &it.opts);
    if (v != LT_OK) return fail(v, at + g_last_error);
    if (!it.image || !it.d_image) return fail(LT_ERR_INVALID_ARG, at + "image or d_image is NULL");
    if (it.heights && it.scene->n_heights > 0)
      for (int j = 0; j < i; ++j)
        if (items[j].scene == it.scene && items[j].heights)
          return fail(LT_ERR_INVALID_ARG, at + "two items with heights share a scene");
    b->sms = it.scene->sms;
    b->all_rec &= it.records != nullptr || it.opts.n_paths == 0;
    b->all_state &= it.opts.lrb3_state != nullptr || it.opts.n_paths == 0;
    b->mask_ready &= it.opts.lrb3_mask_ready != 0 || it.opts.n_paths == 0;
    if (it.opts.attached != 0 && it.scene->has_dielectric) {
      chain.push_back(it);
    } else {
      b->att_lean |= it.opts.attached != 0;
      lean.push_back(it);
    }
  }
  b->n_lean = (int)lean.size();
  b->items = lean;
  b->items.insert(b->items.end(), chain.begin(), chain.end());
  std::vector<BatchJob> jobs(n);
  for (int i = 0; i < n; ++i) {
    const lt_batch_item& it = b->items[i];
    BatchJob& J = jobs[i];
    J.S = it.scene->dev;
    J.kp = kparams(&it.params, &it.opts);
    J.dI = it.d_image;
    J.g = GradPtrs{it.grads.d_albedo, it.grads.d_Le, it.grads.d_heights};
    J.image = it.image;
    J.rec = it.records;
    J.state = it.opts.lrb3_state;
    J.kp.vstate = it.opts.lrb3_state;  // the batched plain primal stores validity masks there
    set_privatization(it.scene, &it.grads, J.kp);  // used by pass 3 over spans only
    b->span_smem = std::max(b->span_smem, sizeof(float) * (size_t)J.kp.priv_n);
    J.att = it.opts.attached != 0;
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int slot = 0; slot < 4; ++slot) {
    const int64_t chunk = 32ll << slot;
    int64_t c = 0;
    for (int i = 0; i < n; ++i) {
      if (i == b->n_lean) b->split[slot] = c;
      jobs[i].chunk0 = c;
      c += (jobs[i].kp.n_paths + chunk - 1) / chunk;
    }
    if (b->n_lean == n) b->split[slot] = c;
    b->n_chunks[slot] = c;
    for (int ws = 0; ws < 3; ++ws) {
      const int w = 2 << ws;
      for (int i = 0; i < n; ++i) jobs[i].S = dev_for(b->items[i].scene, w);
      BatchJob*& dst = b->d_jobs[3 * slot + ws];
      LT_CUDA(cudaMalloc(&dst, sizeof(BatchJob) * n));
      LT_CUDA(cudaMemcpyAsync(dst, jobs.data(), sizeof(BatchJob) * n, cudaMemcpyHostToDevice, st));
      // the upload must finish before the host table changes for the next width
      LT_CUDA(cudaStreamSynchronize(st));
    }
  }
  LT_CUDA(cudaMalloc(&b->d_ticket, 12 * sizeof(unsigned long long)));
  // pass-3 spans: each group's items cut into spans of at most kSpan paths
  const int64_t kSpan = 16384;
  for (int grp = 0; grp < 2; ++grp) {
    std::vector<BatchSpan> spans;
    const int j0 = grp == 0 ? 0 : b->n_lean, j1 = grp == 0 ? b->n_lean : n;
    for (int j = j0; j < j1; ++j)
      for (int64_t a = 0; a < jobs[j].kp.n_paths; a += kSpan)
        spans.push_back(BatchSpan{j, a, std::min<int64_t>(a + kSpan, jobs[j].kp.n_paths)});
    b->n_spans[grp] = (int)spans.size();
    if (!spans.empty()) {
      LT_CUDA(cudaMalloc(&b->d_spans[grp], sizeof(BatchSpan) * spans.size()));
      LT_CUDA(cudaMemcpyAsync(b->d_spans[grp], spans.data(), sizeof(BatchSpan) * spans.size(),
                              cudaMemcpyHostToDevice, st));
      LT_CUDA(cudaStreamSynchronize(st));
    }
  }
  LT_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  LT_CUDA(cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking));
  LT_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  LT_CUDA(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
  LT_CUDA(cudaStreamSynchronize(st));  // the host copy of the table goes out of scope
  *out = b.release();
  return LT_OK;
}

lt_status lt_batch_run(lt_batch* b, int pass, void* stream) {
  lt_status v = check_pass(b, pass);
  if (v != LT_OK) return v;
  if (!b->exec[pass]) {
    v = capture_pass(b, pass);
    if (v != LT_OK) return v;
  }
  LT_CUDA(cudaGraphLaunch(b->exec[pass], (cudaStream_t)stream));
  return LT_OK;
}

lt_status lt_batch_set_config(lt_batch* b, const lt_batch_config* cfg) {
  if (!b) return fail(LT_ERR_INVALID_ARG, "batch is NULL");
  lt_status v = check_batch_cfg(cfg);
  if (v != LT_OK) return v;
  b->cfg = *cfg;
  drop_graphs(b);
  return LT_OK;
}

lt_status lt_batch_get_config(const lt_batch* b, lt_batch_config* cfg) {
  if (!b || !cfg) return fail(LT_ERR_INVALID_ARG, "batch or cfg is NULL");
  *cfg = b->cfg;
  return LT_OK;
}

// Time one configuration: capture (first run, also the warm-up) then the best of `reps`
// graph replays.
static lt_status time_config(lt_batch* b, int pass, const lt_batch_config& c, int reps, cudaStream_t st, cudaEvent_t e0,
                             cudaEvent_t e1, float* ms_out) {
  lt_status v = lt_batch_set_config(b, &c);
  if (v != LT_OK) return v;
  v = lt_batch_run(b, pass, st);
  if (v != LT_OK) return v;
  float t_min = 3e38f;
  for (int r = 0; r < reps; ++r) {
    cudaError_t e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec[pass], st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return fail(LT_ERR_CUDA, std::string("lt_batch_tune: ") + cudaGetErrorString(e));
    t_min = std::min(t_min, ms);
  }
  *ms_out = t_min;
  return LT_OK;
}

lt_status lt_batch_tune(lt_batch* b, int pass, int reps, void* stream, lt_batch_config* best, float* best_ms) {
  lt_status v = check_pass(b, pass);
  if (v != LT_OK) return v;
  if (reps < 1) return fail(LT_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  LT_CUDA(cudaEventCreate(&e0));
  LT_CUDA(cudaEventCreate(&e1));
  const lt_batch_config keep = b->cfg;
  lt_batch_config win{128, 4, 0, 4};
  float win_ms = 3e38f;
  lt_status res = LT_OK;
  // stage 1: BVH width at the default launch shape; stage 2: launch shape at that width
  for (int w : {2, 4, 8}) {
    if (res != LT_OK) break;
    const lt_batch_config c{128, 4, 0, w};
    float ms = 0.0f;
    res = time_config(b, pass, c, reps, st, e0, e1, &ms);
    if (res == LT_OK && ms < win_ms) { win_ms = ms; win = c; }
  }
  const int width = win.bvh_width;
  for (int block : {64, 128, 256}) {
    for (int ppt : {1, 2, 4, 8}) {
      if (res != LT_OK || (block == 128 && ppt == 4)) continue;
      const lt_batch_config c{block, ppt, 0, width};
      float ms = 0.0f;
      res = time_config(b, pass, c, reps, st, e0, e1, &ms);
      if (res == LT_OK && ms < win_ms) { win_ms = ms; win = c; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (res != LT_OK) {
    lt_batch_set_config(b, &keep);
    return res;
  }
  lt_batch_set_config(b, &win);
  v = lt_batch_run(b, pass, stream);  // outputs: one complete run of the chosen shape
  if (v != LT_OK) return v;
  LT_CUDA(cudaStreamSynchronize(st));
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return LT_OK;
}

void lt_batch_destroy(lt_batch* b) { free_batch(b); }

}  // extern "C"
