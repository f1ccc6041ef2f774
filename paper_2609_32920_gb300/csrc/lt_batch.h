// lt_batch.h -- internal interface of the batched passes: one persistent launch runs the
// paths of many scenes, each with its own parameters, path budget, depth and outputs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lt_device.cuh"
#include "lt_launch.h"

namespace lt {

// One item of a batch as the kernels see it (device memory, read per lane).
struct BatchJob {
  DevScene S;
  KParams kp;        // priv_n = 0 (gradients go to global memory), census = null
  const float* dI;   // adjoint image
  GradPtrs g;
  float* image;      // primal image
  void* rec;         // ResLRB records (32 B per path) or null
  void* state;       // LRB-3 per-path state (two-kernel form) or null; kp.vstate = state
  int att;           // attached formulation
  int64_t chunk0;    // index of this item's first chunk in the batch's chunk sequence
};

// Work queue: the items' path ranges are cut into chunks of `chunk` paths (an item's last
// chunk may be shorter); a warp takes the next chunk with one atomic on `ticket`, which
// the pass resets to zero before the launch.
// A launch serves the items jobs[0, n_jobs): ticket t (0 <= t < n_chunks) is chunk
// chunk_base + t of the batch.
struct BatchArgs {
  const BatchJob* jobs;
  int n_jobs;
  int chunk;
  int64_t chunk_base;
  int64_t n_chunks;
  unsigned long long* ticket;
};

// A span of one item's paths [start, end), handed to one block at a time (LRB-3 pass 3 of a
// batch: the block accumulates the item's parameter gradients in shared memory as the
// single-scene kernels do, and adds them to the item's arrays when the span is done).
struct BatchSpan {
  int job;
  int64_t start, end;
};

// Kernel of a batched launch: the fused LRB-3 kernel, or its two-kernel form (pass 2,
// with or without the primal's validity masks, then pass 3).
enum BatchPass {
  BPASS_PRIMAL = 0,
  BPASS_PRIMAL_RES = 1,
  BPASS_LRB3 = 2,
  BPASS_RESLRB = 3,
  BPASS_LRB3_P2 = 4,
  BPASS_LRB3_P2_MASK = 5,
  BPASS_LRB3_P3 = 6
};

// `chains`: some attached item's scene has dielectrics (compiles the specular-chain variant).
// Per BVH width (namespaces w2, w4, w8, see lt_launch.h) and, in lt, by `width`.
#define LT_BATCH_LAUNCHERS                                                                                  \
  cudaError_t launch_batch(int pass, bool att, bool chains, const BatchArgs& a, int block, int grid,       \
                           cudaStream_t st);                                                               \
  /* resident blocks per SM of the pass's kernel at `block` threads (0 on error) */                        \
  int batch_occupancy(int pass, bool att, bool chains, int block);                                         \
  /* LRB-3 pass 3 over spans (see BatchSpan), `smem` bytes of gradient sink per block */                   \
  cudaError_t launch_batch_spans(bool att, bool chains, const BatchJob* jobs, const BatchSpan* spans,      \
                                 int n_spans, unsigned long long* ticket, int block, int grid, size_t smem, \
                                 cudaStream_t st);                                                         \
  int batch_spans_occupancy(bool att, bool chains, int block, size_t smem);
namespace w2 { LT_BATCH_LAUNCHERS }
namespace w4 { LT_BATCH_LAUNCHERS }
namespace w8 { LT_BATCH_LAUNCHERS }
cudaError_t launch_batch(int width, int pass, bool att, bool chains, const BatchArgs& a, int block, int grid,
                         cudaStream_t st);
int batch_occupancy(int width, int pass, bool att, bool chains, int block);
cudaError_t launch_batch_spans(int width, bool att, bool chains, const BatchJob* jobs, const BatchSpan* spans,
                               int n_spans, unsigned long long* ticket, int block, int grid, size_t smem,
                               cudaStream_t st);
int batch_spans_occupancy(int width, bool att, bool chains, int block, size_t smem);

}  // namespace lt
