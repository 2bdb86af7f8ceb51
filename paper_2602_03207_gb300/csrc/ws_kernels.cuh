// Launchers of the render-path kernels (host side, called by ws_api.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ws_common.cuh"

namespace ws {

cudaError_t launch_preprocess(int64_t n, const float* means, const float* log_scales,
                              const float* quats, const float* logits, const float* sh,
                              const Frame& f, float* splats, float* depth, uint16_t* rect,
                              uint32_t* tiles_touched, cudaStream_t stream);

// ---- compaction (scan of tiles_touched + key emission)
size_t cull_scratch_bytes(int64_t n);
cudaError_t launch_cull(int64_t n, const uint32_t* tiles_touched, const uint16_t* rect,
                        const float* depth, const Frame& f, uint32_t* offsets, uint64_t* keys,
                        uint32_t* vals, int64_t key_capacity, uint32_t* num_keys,
                        uint32_t* status, void* scratch, cudaStream_t stream);

// ws_cull fused with the first partition pass of the segmented tile sort:
// the keys come out stably partitioned by the low `digit_bits` bits of the
// tile id (one view; digit_bits 4..8, cull_partition_supported).
bool cull_partition_supported(int digit_bits);
size_t cull_partition_scratch_bytes(int64_t n);
cudaError_t launch_cull_partition(int64_t n, const uint32_t* tiles_touched, const uint16_t* rect, const float* depth,
                                  const Frame& f, int digit_bits, uint32_t* offsets, uint64_t* keys, uint32_t* vals,
                                  int64_t key_capacity, uint32_t* num_keys, uint32_t* status, void* scratch,
                                  void* part_scratch, cudaStream_t stream);

cudaError_t launch_cull_batch(int64_t n, const ViewGrid& grid, const uint32_t* tiles_touched,
                              const uint16_t* rect, const float* depth, uint32_t* offsets, uint64_t* keys,
                              uint32_t* vals, int64_t key_capacity, uint32_t* num_keys, uint32_t* status,
                              void* scratch, cudaStream_t stream);

// ---- radix sort
size_t sort_scratch_bytes(int64_t key_capacity, int digit_bits);
bool sort_digit_supported(int digit_bits);
cudaError_t launch_sort(const uint32_t* num_keys, int64_t key_capacity, int begin_bit,
                        int end_bit, int digit_bits, uint64_t* keys, uint32_t* vals,
                        uint64_t* keys_alt, uint32_t* vals_alt, void* scratch, int* in_alt,
                        cudaStream_t stream);

// single-sweep (decoupled look-back) variant
bool sort_segmented_supported(int64_t key_capacity, int begin_bit, int end_bit);
size_t sort_segmented_scratch_bytes(int64_t key_capacity);
// ranges (optional, ntiles entries of [start, end)): each segment's bounds
// in the sorted output, for the segments below ntiles.
// first_pass_done: the keys are already stably partitioned by the first
// digit, sort_segmented_first_digit bits wide (launch_cull_partition).
int sort_segmented_first_digit(int end_bit, int digit_bits);
cudaError_t launch_sort_segmented(const uint32_t* num_keys, int64_t key_capacity, int begin_bit, int end_bit,
                                  int digit_bits, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                  uint32_t* vals_alt, void* scratch, int* in_alt, cudaStream_t stream,
                                  uint32_t* ranges = nullptr, uint32_t ntiles = 0, bool first_pass_done = false);
bool sort_lookback_supported(int digit_bits, int begin_bit, int end_bit);
size_t sort_lookback_scratch_bytes(int64_t key_capacity);
cudaError_t launch_sort_lookback(const uint32_t* num_keys, int64_t key_capacity, int begin_bit, int end_bit,
                                 int digit_bits, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                 uint32_t* vals_alt, void* scratch, uint32_t* flags, int drop_tile, int* in_alt,
                                 cudaStream_t stream);

// allocation-free variant: histogram scratch in a static device array
int64_t sort_noalloc_max_keys();
size_t sort_noalloc_scratch_bytes();
cudaError_t launch_sort_noalloc(const uint32_t* num_keys, int64_t key_capacity, int begin_bit,
                                int end_bit, int digit_bits, uint64_t* keys, uint32_t* vals,
                                uint64_t* keys_alt, uint32_t* vals_alt, int* in_alt,
                                cudaStream_t stream);

// ---- rasterisation
// Skipped (ranges taken as given) when flags has WS_CFG_RANGES_GIVEN.
cudaError_t launch_tile_ranges(const uint64_t* keys, const uint32_t* num_keys, uint32_t* ranges, uint32_t ntiles,
                               uint32_t flags, cudaStream_t stream);
cudaError_t launch_rasterize(const uint32_t* num_keys, int64_t key_capacity_hint,
                             const uint64_t* keys, const uint32_t* vals, const float* splats,
                             const Frame& f, uint32_t* ranges, float* image, float* t_final,
                             uint32_t* n_contrib, cudaStream_t stream);

// ---- packed-record variant
cudaError_t launch_preprocess_packed(int64_t n, const float* means, const float* log_scales, const float* quats,
                                     const float* logits, const float* sh, const Frame& f, float* mean2d,
                                     uint32_t* axes, uint32_t* rgba, float* depth, uint16_t* rect,
                                     uint32_t* tiles_touched, cudaStream_t stream);
cudaError_t launch_rasterize_packed(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                                    const float* mean2d, const uint32_t* axes, const uint32_t* rgba, const Frame& f,
                                    uint32_t* ranges, float* image, float* t_final, uint32_t* n_contrib,
                                    cudaStream_t stream);

// ---- the paper's quad design (global depth sort + back-to-front quads)
struct QuadLayout {
    size_t sort, cull, dkeys, dkeys_alt, dvals, dvals_alt, offsets, quad, one, rect, zdepth, num_vis, ranges, total;
};
QuadLayout quad_layout(int64_t n, int64_t key_capacity, int64_t ntiles);
cudaError_t launch_render_quads(int64_t n, const float* splats, const float* depth, const uint32_t* tiles_touched,
                                const Frame& f, int64_t key_capacity, uint64_t* keys, uint32_t* vals,
                                uint64_t* keys_alt, uint32_t* vals_alt, uint32_t* num_keys, float* image,
                                float* t_final, void* workspace, cudaStream_t stream);

// ---- backward
size_t backward_scratch_bytes(int64_t key_capacity);
cudaError_t launch_backward(int64_t n, const float* means, const float* log_scales, const float* quats,
                            const float* sh, const Frame& f, const float* splats, const uint16_t* rect,
                            const uint32_t* offsets, const uint32_t* tiles_touched,
                            const uint32_t* vals, const uint32_t* ranges, const float* t_final,
                            const uint32_t* n_contrib, const float* d_image, float* d_means,
                            float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                            int64_t key_capacity, void* scratch, cudaStream_t stream);

// ---- batched views (view-major per-(view, Gaussian) arrays)
cudaError_t launch_preprocess_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                                    const float* logits, const float* sh, const FrameTable& ft, float* splats,
                                    float* depth, uint16_t* rect, uint32_t* tiles_touched, cudaStream_t stream);
cudaError_t launch_rasterize_batch(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals, int64_t n,
                                   const float* splats, const FrameTable& ft, uint32_t* ranges, float* image, float* t_final,
                                   uint32_t* n_contrib, cudaStream_t stream);
cudaError_t launch_backward_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                                  const float* sh, const FrameTable& ft, const float* splats, const uint16_t* rect,
                                  const uint32_t* offsets, const uint32_t* tiles_touched, const uint32_t* vals,
                                  const uint32_t* ranges, const float* t_final, const uint32_t* n_contrib,
                                  const float* d_image, float* d_means, float* d_log_scales, float* d_quats,
                                  float* d_logits, float* d_sh, int64_t key_capacity, void* scratch,
                                  cudaStream_t stream);
cudaError_t launch_residual(int64_t count, const float* image, const float* target, float* d_image,
                            cudaStream_t stream);

// ---- fused training step (blend forward + L2 residual + backward records,
// then the per-Gaussian adjoint)
cudaError_t launch_train(int64_t n, const float* means, const float* log_scales, const float* quats, const float* sh,
                         const Frame& f, const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                         const float* splats, const uint16_t* rect, const uint32_t* offsets,
                         const uint32_t* tiles_touched, const float* target, uint32_t* ranges, float* image,
                         float* t_final, uint32_t* n_contrib, float* d_means, float* d_log_scales, float* d_quats,
                         float* d_logits, float* d_sh, int64_t key_capacity, void* scratch, cudaStream_t stream);
cudaError_t launch_train_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                               const float* sh, const FrameTable& ft, const uint32_t* num_keys, const uint64_t* keys,
                               const uint32_t* vals, const float* splats, const uint16_t* rect,
                               const uint32_t* offsets, const uint32_t* tiles_touched, const float* target,
                               uint32_t* ranges, float* image, float* t_final, uint32_t* n_contrib, float* d_means,
                               float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                               int64_t key_capacity, bool persistent, void* scratch, cudaStream_t stream);

}  // namespace ws
