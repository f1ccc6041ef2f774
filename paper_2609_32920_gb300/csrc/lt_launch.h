// lt_launch.h -- internal interface between the C-ABI host code and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lt {

struct DevScene;

// Per-call kernel parameters (by value).
struct KParams {
  uint64_t seed;
  int64_t path_offset;
  int64_t n_paths;
  int max_depth;
  float inv_n;               // 1 / N of the estimator
  const float* Le;           // DEVICE [3]
  const float* albedo;       // DEVICE [n_albedo]
  const uint8_t* mask;       // DEVICE [n_paths] or null
  uint32_t* hash;            // DEVICE [n_paths] or null
  float* dbg;                // DEVICE [n_paths][4] or null
  size_t tape_offset;        // naive tape: bytes before the first record
  unsigned long long* census;  // DEVICE [5] or null: rays, box tests, primitive tests, vertices, connections
  int n_alb, n_h;              // albedo / height gradients accumulated in shared memory per block
                               // (array lengths, or 0: that array goes to global memory directly)
  int priv_n;                  // n_alb + n_h: floats of dynamic shared memory per block
  const float* mlp;            // learned reservoir target parameters (DEVICE) or null (luminance)
  const uint32_t* order;       // plain primal: the order in which it takes the paths (or null)
  void* vstate;                // plain primal: LRB-3 per-path state that receives each path's
                               // connection-validity mask (or null)
  int rr_depth;                // Russian roulette after vertices of depth >= rr_depth (0: off)
  float rr_q;                  // survival probability of the roulette
  int filter;                  // reconstruction filter: 0 tent, 1 truncated Gaussian
  uint32_t* list;              // paths with a valid connection (plain primal: appends;
                               // LRB-3 passes 2 and 3 with known masks: visit only these) or null
  unsigned long long* list_n;  // length of `list`
  unsigned long long* ticket;  // zeroed counters of entries taken: [0] pass 2, [1] pass 3 (plain
                               // primal with the LRB-3 state: [0] its 32-path chunks)
  float4* conn1;               // per path: film position and contribution (u_x, u_y, L.r, L.g) of
  float* conn1z;               // its first valid connection, and L.b (plain primal: writes; LRB-3
                               // pass 2 with known masks: reads for paths with one connection)
  int jac_noise;               // paper-literal transport: Jacobian noise at diffuse vertices
  uint64_t noise_seed;         // its Philox key
  float det_eps;               // its determinant guard
};

struct GradPtrs {
  float* d_albedo;
  float* d_Le;
  float* d_heights;
};

struct LaunchCfg {
  int block;
  int blocks_per_sm;
  int sms;
};

struct RefitArgs {
  float4* prim;
  const int4* prim_h;
  const float4* tri_base;
  const float* heights;
  int n_prims;
  float4* node;
  const int2* range;
  int n_nodes;
  const int* big;  // nodes whose primitive range exceeds kRefitBig: a whole block reduces each
  int n_big;
  // wide BVHs (width 4 and 8): child slot -> binary node whose box it takes (-1: empty)
  float4* wnode[2];
  const int* wmap[2];
  int n_wnodes[2];
};

// Binary BVH nodes with more primitives than this are refitted by a block each, the rest
// by a warp each.
constexpr int kRefitBig = 1024;

struct BatchArgs;

// Bidirectional estimator (light-tracer connections + camera samples with next-event
// estimation, balance heuristic): counts N (light paths of the estimator) and M (camera
// samples), the camera samples' optional mask and decision hashes.
struct BidirArgs {
  float N, M;
  int64_t n_cam;
  const uint8_t* cam_mask;
  uint32_t* cam_hash;
};

// Kernel launchers.  lt_kernels.cu is compiled once per BVH width into namespaces w2, w4
// and w8; the functions of the same names in lt itself pick the variant by the scene's
// width (DevScene::width).
#define LT_KERNEL_LAUNCHERS                                                                                        \
  cudaError_t launch_refit(const RefitArgs& a, cudaStream_t st);                                                  \
  cudaError_t launch_primal(const DevScene& S, const KParams& kp, int est, float* image, void* aux,               \
                            const LaunchCfg& L, cudaStream_t st);                                                 \
  cudaError_t launch_lrb3(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,           \
                          const GradPtrs& g, void* state, bool mask_ready, const LaunchCfg& L, cudaStream_t st);  \
  cudaError_t launch_reslrb(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,         \
                            const void* rec, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st);             \
  cudaError_t launch_naive(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,           \
                           const void* ws, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st);               \
  cudaError_t launch_lrb2(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,           \
                          void* buf, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st);                     \
  cudaError_t launch_collect(const DevScene& S, const KParams& kp, const float* dI, float tfloor, float* feats,   \
                             float* targets, int64_t cap, unsigned long long* count, const LaunchCfg& L,          \
                             cudaStream_t st);                                                                    \
  cudaError_t launch_film_l2(const float* I, const float* T, int64_t n, float* dI, float* loss, int sms,          \
                             cudaStream_t st);                                                                    \
  cudaError_t launch_bidir(const DevScene& S, const KParams& kp, const BidirArgs& ba, bool backward, float* image, \
                           const float* dI, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st);             \
  cudaError_t launch_lrb3_literal(const DevScene& S, const KParams& kp, const float* dI, const GradPtrs& g,       \
                                  const LaunchCfg& L, cudaStream_t st);

namespace w2 { LT_KERNEL_LAUNCHERS }
namespace w4 { LT_KERNEL_LAUNCHERS }
namespace w8 { LT_KERNEL_LAUNCHERS }
LT_KERNEL_LAUNCHERS

// `state` of launch_lrb3 (or null: fused kernel): per-path state of the two-kernel form,
// layout float4[n_paths] then, at byte lrb3_state_split(n_paths), uint32[n_paths] (together
// lrb3_state_core bytes); then the list of the paths that have a valid connection (uint32
// indices relative to the call, at lrb3_state_list) and its length (uint64, at
// lrb3_state_count), written by a plain primal so that passes 2 and 3 visit only those;
// then each path's first valid connection, float4 (u_x, u_y, L.r, L.g) at lrb3_state_conn4
// and float L.b at lrb3_state_connz, written by the plain primal; then the order in which the
// plain primal takes the paths (uint32[n_paths] at lrb3_state_order) and the counting sort's
// work area that builds it (kSortBins x kSortBlocks counts, then kSortBins bin starts).
constexpr int kSortBins = 4096;   // 64 x 64 cells of the first direction
constexpr int kSortBlocks = 256;  // blocks of the sort, each over a contiguous range of paths
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
__host__ __device__ inline size_t lrb3_state_split(int64_t n) { return align256((size_t)n * 16); }
__host__ __device__ inline size_t lrb3_state_core(int64_t n) { return lrb3_state_split(n) + align256((size_t)n * 4); }
__host__ __device__ inline size_t lrb3_state_list(int64_t n) { return lrb3_state_core(n); }
__host__ __device__ inline size_t lrb3_state_count(int64_t n) { return lrb3_state_list(n) + align256((size_t)n * 4); }
__host__ __device__ inline size_t lrb3_state_conn4(int64_t n) { return lrb3_state_count(n) + 256; }
__host__ __device__ inline size_t lrb3_state_connz(int64_t n) { return lrb3_state_conn4(n) + align256((size_t)n * 16); }
__host__ __device__ inline size_t lrb3_state_order(int64_t n) { return lrb3_state_connz(n) + align256((size_t)n * 4); }
__host__ __device__ inline size_t lrb3_state_sort(int64_t n) { return lrb3_state_order(n) + align256((size_t)n * 4); }
__host__ __device__ inline size_t lrb3_state_bytes(int64_t n) {
  return lrb3_state_sort(n) + align256(sizeof(unsigned) * (size_t)kSortBins * (kSortBlocks + 1));
}
// After the list's length (uint64) at lrb3_state_count: the two passes' counters of list
// entries taken (uint64 each).
// The path list is used for calls of at most this many paths (uint32 indices).
constexpr int64_t kListMaxPaths = 0xffffffffll;

// Buffer of the buffered two-pass estimator (lrb_2pass): the LRB-3 per-path state, then
// per path its traced vertex count (int), then per vertex [depth][path] the splat record
// (u_x, u_y, L.r, L.g) (float4; u_x < 0 = no valid connection) and L.b (float).
struct Lrb2Layout {
  size_t counts, rec4, recz, total;
};
__host__ __device__ inline Lrb2Layout lrb2_layout(int64_t n, int d) {
  Lrb2Layout L;
  L.counts = lrb3_state_core(n);
  L.rec4 = L.counts + align256((size_t)n * 4);
  L.recz = L.rec4 + align256((size_t)n * (size_t)d * 16);
  L.total = L.recz + align256((size_t)n * (size_t)d * 4);
  return L;
}
size_t mlp_grad_smem_bytes();
cudaError_t launch_mlp_grad(const float* P, const float* X, const float* T, int64_t n, float inv_batch, float* g,
                            float* loss, int sms, cudaStream_t st);
cudaError_t launch_mlp_adam(float* P, float* M, float* V, const float* g, int step, float lr, cudaStream_t st);
cudaError_t launch_mlp_moments(const float* X, const float* T, int64_t n, float* P, cudaStream_t st);
cudaError_t launch_mlp_forward(const float* P, const float* X, int64_t n, float* out, int sms, cudaStream_t st);

}  // namespace lt
