// lt_dispatch.cu -- the kernel launchers in lt pick the variant compiled for the call's
// BVH width (lt_kernels.cu is built once per width into lt::w2, lt::w4 and lt::w8).
#include <cuda_runtime.h>

#include "lt_batch.h"
#include "lt_device.cuh"
#include "lt_launch.h"

namespace lt {

#define LT_BY_WIDTH(w, call) ((w) == 4 ? w4::call : (w) == 8 ? w8::call : w2::call)

cudaError_t launch_refit(const RefitArgs& a, cudaStream_t st) { return w4::launch_refit(a, st); }

cudaError_t launch_primal(const DevScene& S, const KParams& kp, int est, float* image, void* aux, const LaunchCfg& L,
                          cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_primal(S, kp, est, image, aux, L, st));
}

cudaError_t launch_lrb3(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,
                        const GradPtrs& g, void* state, bool mask_ready, const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_lrb3(S, kp, att, chains, dI, g, state, mask_ready, L, st));
}

cudaError_t launch_reslrb(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,
                          const void* rec, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_reslrb(S, kp, att, chains, dI, rec, g, L, st));
}

cudaError_t launch_naive(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI,
                         const void* ws, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_naive(S, kp, att, chains, dI, ws, g, L, st));
}

cudaError_t launch_lrb2(const DevScene& S, const KParams& kp, bool att, bool chains, const float* dI, void* buf,
                        const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_lrb2(S, kp, att, chains, dI, buf, g, L, st));
}

cudaError_t launch_collect(const DevScene& S, const KParams& kp, const float* dI, float tfloor, float* feats,
                           float* targets, int64_t cap, unsigned long long* count, const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_collect(S, kp, dI, tfloor, feats, targets, cap, count, L, st));
}

cudaError_t launch_film_l2(const float* I, const float* T, int64_t n, float* dI, float* loss, int sms,
                           cudaStream_t st) {
  return w4::launch_film_l2(I, T, n, dI, loss, sms, st);
}

cudaError_t launch_lrb3_literal(const DevScene& S, const KParams& kp, const float* dI, const GradPtrs& g,
                                const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_lrb3_literal(S, kp, dI, g, L, st));
}

cudaError_t launch_bidir(const DevScene& S, const KParams& kp, const BidirArgs& ba, bool backward, float* image,
                         const float* dI, const GradPtrs& g, const LaunchCfg& L, cudaStream_t st) {
  return LT_BY_WIDTH(S.width, launch_bidir(S, kp, ba, backward, image, dI, g, L, st));
}

cudaError_t launch_batch(int width, int pass, bool att, bool chains, const BatchArgs& a, int block, int grid,
                         cudaStream_t st) {
  return LT_BY_WIDTH(width, launch_batch(pass, att, chains, a, block, grid, st));
}

int batch_occupancy(int width, int pass, bool att, bool chains, int block) {
  return LT_BY_WIDTH(width, batch_occupancy(pass, att, chains, block));
}

cudaError_t launch_batch_spans(int width, bool att, bool chains, const BatchJob* jobs, const BatchSpan* spans,
                               int n_spans, unsigned long long* ticket, int block, int grid, size_t smem,
                               cudaStream_t st) {
  return LT_BY_WIDTH(width, launch_batch_spans(att, chains, jobs, spans, n_spans, ticket, block, grid, smem, st));
}

int batch_spans_occupancy(int width, bool att, bool chains, int block, size_t smem) {
  return LT_BY_WIDTH(width, batch_spans_occupancy(att, chains, block, smem));
}

}  // namespace lt
