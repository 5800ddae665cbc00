// Launchers of the kernels in each translation unit (host functions in namespace dass). The
// extern "C" entry points and the stage drivers validate arguments, build camera tables and call
// these; every launcher enqueues on the given stream and returns a dass_status.
#pragma once

#include "common.cuh"

namespace dass {

// rows (optional, with the device count n_rows and a host bound rows_cap): project only those
// Gaussians; every other record keeps its contents.
int preprocess_launch(long long n, int deg, const float* means, const float* log_scales, const float* quats,
                      const float* opacity_logit, const float* sh, const uint8_t* keep, const CamTable& ct,
                      dass_splat* splats, cudaStream_t st, const int* rows = nullptr,
                      const long long* n_rows = nullptr, long long rows_cap = 0,
                      unsigned long long* vis = nullptr);
int preprocess_scenes_launch(const dass_scene* scenes, int deg, const CamTable& ct, dass_splat* splats,
                             cudaStream_t st, long long n_max = 0);
int preprocess_bwd_launch(long long n, int deg, const float* means, const float* log_scales, const float* quats,
                          const float* opacity_logit, const float* sh, const uint8_t* keep, const CamTable& ct,
                          const dass_splat* splats, const dass_splat_grad* gsp, const int* rows, long long n_rows,
                          unsigned flags, int accumulate, float* d_means, float* d_log_scales, float* d_quats,
                          float* d_opacity_logit, float* d_sh, float* d_keep, cudaStream_t st);
int densify_stats_launch(long long n, const CamTable& ct, const dass_splat* splats, const dass_splat_grad* gsp,
                         float* accum, int* count, cudaStream_t st);
// The same statistics from the per-Gaussian visibility masks preprocess_launch writes (vis).
int densify_stats_vis_launch(long long n, const CamTable& ct, const unsigned long long* vis,
                             const dass_splat_grad* gsp, float* accum, int* count, cudaStream_t st);
size_t bin_sort_workspace_bytes(long long n_rec, long long cap);
int bin_sort_launch(const dass_splat* splats, long long n_rec, const CamTable& ct, uint32_t* pair_rec, long long cap,
                    uint32_t* tile_ranges, long long* counters, void* ws, size_t ws_bytes, cudaStream_t st);
// Incremental binning: the static part (the pairs of every row not flagged as moving, binned and sorted
// once, with each pair's depth key and each tile's first position) and the moving rows' records.
struct StaticBins {
    uint32_t* rec;              // [cap] record of each static pair, in (tile, depth, record) order
    uint32_t* depth;            // [cap] its depth key
    uint32_t* start;            // [tiles_total + 1] first position of each tile
    long long* counters;        // [3] as bin_sort_launch's
    uint32_t* moving;           // [n_cams * n_rows] records of the moving rows, camera-major, ascending
    long long* n_moving;        // [1] their count
    int* rows;                  // [n_rows] moving rows, ascending
    long long* n_rows_moving;   // [1]
};
size_t bin_sort_split_workspace_bytes(long long n_rows, long long n_rec, long long cap);
int bin_sort_split_launch(const dass_splat* splats, long long n_rows, const CamTable& ct, const uint8_t* moving_rows,
                          long long cap, const StaticBins& sb, void* ws, size_t ws_bytes, cudaStream_t st);
size_t bin_sort_merge_workspace_bytes(long long moving_cap, long long cap, int tiles_total);
int bin_sort_merge_launch(const dass_splat* splats, const CamTable& ct, const StaticBins& sb, long long moving_cap,
                          long long cap, uint32_t* pair_rec, uint32_t* tile_ranges, long long* counters, void* ws,
                          size_t ws_bytes, cudaStream_t st);
// order (optional, device, ct.tiles_total entries): a permutation of the tiles, the order in which the
// launch's blocks take them (tile_order_launch: longest lists first); null: tile order.
int render_fwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, float* image, float* T_final, int* n_last, cudaStream_t st,
                      unsigned long long* work = nullptr, const uint8_t* full_grad = nullptr,
                      long long rec_stride = 1, const uint32_t* order = nullptr);
int render_prepare(int tile, int batch);
// mean_grads false (with a full_grad mask): the Gaussians outside the mask get no gradient at all
// (their dL/dmean2D is left as it was), the pixels' state still passes them exactly.
int render_bwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, const float* T_final, const int* n_last, const float* dL_dimage,
                      const uint8_t* full_grad, long long rec_stride, dass_splat_grad* gsplat, cudaStream_t st,
                      bool mean_grads = true, const uint32_t* order = nullptr);
// Tiles by descending list length (bucketed), into order[tiles]: the block order of the compositing
// launches, so that the longest lists start first and no long list is left for the end of a launch.
int tile_order_launch(const uint32_t* ranges, int tiles, uint32_t* order, cudaStream_t st);
size_t loss_workspace_bytes(const CamTable& ct);
int loss_launch(const float* image, const float* target, const CamTable& ct, float lambda, float inv_cams, float* dL,
                double* loss, void* ws, size_t ws_bytes, cudaStream_t st, const float* target_stats = nullptr);
int target_stats_launch(const float* target, const CamTable& ct, float* stats, cudaStream_t st);
int shift_launch(long long n_dyn, const int* idx, const float* off, const float* means, const float* quats, float* om,
                 float* oq, cudaStream_t st);
int shift_bwd_launch(long long n_dyn, const int* idx, const float* off, const float* quats, const float* dm,
                     const float* dq, float* doff, float* dqin, cudaStream_t st);
int adam_launch(long long n_sel, int width, const int* rows, float* p, const float* g, float* m, float* v,
                int* step_dev, const float* lr, float b1, float b2, float eps, int inc, cudaStream_t st);
size_t inherit_workspace_bytes(long long n);
int inherit_launch(long long n, int deg, const float* means, const float* ls, const float* quats, const float* logit,
                   const float* sh, const uint8_t* is_var, const float* m, int erase, float* om, float* ols, float* oq,
                   float* ologit, float* osh, uint8_t* ovar, int* remap, long long* n_out, void* ws, size_t ws_bytes,
                   cudaStream_t st);
int inherit_keep_launch(long long n, const uint8_t* is_var, const float* m, uint8_t* keep, cudaStream_t st);
int render_features_launch(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct,
                           const float* feats, int F, long long stride, float* out, cudaStream_t st);
int object_ids_launch(const float* x, long long n, int F, const float* W, const float* b, int K, int* ids,
                      cudaStream_t st);
int dynamic_objects_launch(const int* ids, const uint8_t* dyn_area, long long n, int K, unsigned int min_pixels,
                           uint8_t* obj_mask, unsigned int* hist, cudaStream_t st);
int dynamic_gaussians_launch(const float* feats, long long n, int F, const float* W, const float* b, int K,
                             const uint8_t* obj_mask, uint8_t* dyn_mask, cudaStream_t st);
size_t mask_rows_workspace_bytes(long long n);
int mask_rows_launch(const uint8_t* mask, long long n, int* rows, long long* count, void* ws, size_t ws_bytes,
                     cudaStream_t st);
int field_fwd_launch(const dass_field* f, long long n_rows, const int* rows, const float* means, float* out,
                     cudaStream_t st);
int field_bwd_launch(const dass_field* f, long long n_rows, const int* rows, const float* means, const float* dof,
                     float* dt, float* dw1, float* db1, float* dw2, float* db2, cudaStream_t st);
int prune_logits_launch(long long n, const float* logit, float min_opacity, float* m, cudaStream_t st);
int inherit_mask_grad_launch(long long n_rows, const int* rows, const float* m, const float* d_keep, float lambda,
                             float* grad, double* loss, cudaStream_t st);
size_t error_pass_workspace_bytes(const CamTable& ct);
int error_pass_launch(const float* img, const float* tgt, const CamTable& ct, double quantile, long long n,
                      const float* means, const uint8_t* is_var, float* error_map, float* gamma, uint8_t* s_err,
                      void* ws, size_t ws_bytes, cudaStream_t st);
size_t select_workspace_bytes(long long n);
int select_launch(long long n, const float* accum, const int* count, const uint8_t* s_err, const uint8_t* is_var,
                  float tau_pos, float tau_err, int k_max, int* selected, int* n_selected, void* ws, size_t ws_bytes,
                  cudaStream_t st);
int spawn_launch(long long n, int deg, float* means, float* ls, float* quats, float* logit, float* sh, uint8_t* is_var,
                 const int* selected, const int* n_sel, int k_max, const float* z, long long* n_total,
                 cudaStream_t st);

size_t scan_partials_bytes(long long len);
bool batch_ok(int batch);   // list entries a compositing warp examines per round: 32, 64, 128 or 256
void set_error_message(const char* msg);

}  // namespace dass
