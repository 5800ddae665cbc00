// extern "C" entry points of libdass: argument checks, camera tables and dispatch to the kernel
// launchers. The stage drivers and the whole-timestep driver are in timestep.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <mutex>
#include <set>
#include <utility>

#include "common.cuh"
#include "launch.cuh"

namespace dass {

static thread_local char g_err[512] = {0};
static thread_local long long g_launches = 0;

void count_launch(long long k) { g_launches += k; }
long long launches_so_far() { return g_launches; }
void set_launches(long long v) { g_launches = v; }

void set_error_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

void set_last_error(const char* what, cudaError_t e) {
    snprintf(g_err, sizeof(g_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

int allow_dynamic_smem(const void* kernel, int bytes) {
    if (bytes <= 48 * 1024) return DASS_OK;
    int dev = 0;
    DASS_CHECK_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return DASS_OK;
    DASS_CHECK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.insert({kernel, dev});
    return DASS_OK;
}

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(what, e);
        return DASS_ERR_CUDA;
    }
    return DASS_OK;
}

bool make_cam_table(const dass_camera* cams, int n_cams, int tile, long long rec_stride, CamTable* out,
                    const int64_t* rec_offsets) {
    if (!cams || n_cams < 1 || n_cams > DASS_MAX_CAMERAS) return false;
    if (tile != 8 && tile != 16 && tile != 32) return false;
    if (rec_offsets) {
        if (rec_offsets[0] != 0) return false;
        for (int i = 0; i < n_cams; ++i)
            if (rec_offsets[i + 1] < rec_offsets[i]) return false;
        if (rec_offsets[n_cams] >= (1ll << 32)) return false;
    }
    std::memset(out, 0, sizeof(CamTable));
    out->n = n_cams;
    out->tile = tile;
    out->rec_stride = rec_offsets ? 0 : rec_stride;
    long long tiles = 0, pix = 0;
    for (int i = 0; i < n_cams; ++i) {
        const dass_camera& c = cams[i];
        if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f)) return false;
        if ((long long)(c.width + 16) * (c.height + 16) >= (1ll << 31)) return false;   // 32-bit pixel offsets
        CamInfo& ci = out->c[i];
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) ci.R[3 * r + k] = c.viewmat[4 * r + k];
            ci.t[r] = c.viewmat[4 * r + 3];
        }
        ci.fx = c.fx; ci.fy = c.fy; ci.cx = c.cx; ci.cy = c.cy;
        ci.W = c.width; ci.H = c.height;
        for (int k = 0; k < 3; ++k)
            ci.campos[k] = -(ci.R[k] * ci.t[0] + ci.R[3 + k] * ci.t[1] + ci.R[6 + k] * ci.t[2]);
        // Alg. 1 full projection T (row vectors): [P,1] T = (p_x, p_y, p_z, p_hom) with p_hom = z
        // and x_norm chosen so that 0.5((x_norm + 1) W - 1) = fx X/Z + cx. Built in double.
        double W = c.width, H = c.height, zn = 0.01, zf = 100.0;
        double K[4][4] = {{2.0 * c.fx / W, 0.0, (2.0 * c.cx + 1.0) / W - 1.0, 0.0},
                          {0.0, 2.0 * c.fy / H, (2.0 * c.cy + 1.0) / H - 1.0, 0.0},
                          {0.0, 0.0, (zf + zn) / (zf - zn), -2.0 * zf * zn / (zf - zn)},
                          {0.0, 0.0, 1.0, 0.0}};
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 4; ++k) {
                double s = 0.0;
                for (int j = 0; j < 4; ++j) s += K[r][j] * (double)c.viewmat[4 * j + k];
                ci.proj[4 * k + r] = (float)s;   // transpose: row-vector convention
            }
        ci.tiles_x = (c.width + tile - 1) / tile;
        ci.tiles_y = (c.height + tile - 1) / tile;
        ci.tile_base = (int)tiles;
        ci.pix_base = pix;
        ci.rec_base = rec_offsets ? (long long)rec_offsets[i] : (long long)i * rec_stride;
        tiles += (long long)ci.tiles_x * ci.tiles_y;
        pix += (long long)c.width * c.height;
    }
    if (tiles >= (1ll << 31)) return false;
    out->tiles_total = (int)tiles;
    out->pixels_total = pix;
    return true;
}

}  // namespace dass

using namespace dass;

static float3 bg3(const float* bg) { return bg ? make_float3(bg[0], bg[1], bg[2]) : make_float3(0.f, 0.f, 0.f); }

DASS_API int dass_version(void) { return DASS_VERSION; }

DASS_API const char* dass_status_string(int s) {
    switch (s) {
        case DASS_OK: return "ok";
        case DASS_ERR_INVALID_ARG: return "invalid argument";
        case DASS_ERR_CUDA: return "CUDA error";
        case DASS_ERR_OOM: return "workspace too small";
        case DASS_ERR_CAPACITY: return "capacity exceeded";
        case DASS_ERR_TIMEOUT: return "bounded wait timed out";
        case DASS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

DASS_API const char* dass_last_error(void) { return dass::g_err; }

DASS_API int64_t dass_kernel_launches(void) { return (int64_t)dass::launches_so_far(); }

DASS_API int dass_tile_layout(const dass_camera* cams, int n_cams, int tile, int32_t* tiles_total,
                              int64_t* pixels_total) {
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, 0, &ct)) return DASS_ERR_INVALID_ARG;
    if (tiles_total) *tiles_total = ct.tiles_total;
    if (pixels_total) *pixels_total = ct.pixels_total;
    return DASS_OK;
}

DASS_API int dass_preprocess(int64_t n, int sh_degree, const float* means, const float* log_scales, const float* quats,
                             const float* opacity_logit, const float* sh, const uint8_t* keep, const dass_camera* cams,
                             int n_cams, int tile, dass_splat* splats, void* stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3) return DASS_ERR_INVALID_ARG;
    if (n > 0 && (!means || !log_scales || !quats || !opacity_logit || !sh || !splats)) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, n, &ct)) return DASS_ERR_INVALID_ARG;
    if (n == 0) return DASS_OK;
    return preprocess_launch(n, sh_degree, means, log_scales, quats, opacity_logit, sh, keep, ct, splats,
                             as_stream(stream));
}

DASS_API int dass_preprocess_scenes(const dass_scene* scenes, const dass_camera* cams, int n_cams, int tile,
                                   int64_t rec_stride, dass_splat* splats, void* stream) {
    if (!scenes || rec_stride < 0 || n_cams < 1 || n_cams > DASS_MAX_CAMERAS) return DASS_ERR_INVALID_ARG;
    int deg = scenes[0].sh_degree;
    if (deg < 0 || deg > 3) return DASS_ERR_INVALID_ARG;
    for (int c = 0; c < n_cams; ++c) {
        const dass_scene& sc = scenes[c];
        if (sc.sh_degree != deg || sc.n < 0 || sc.n > rec_stride) return DASS_ERR_INVALID_ARG;
        if (sc.n > 0 && (!sc.means || !sc.log_scales || !sc.quats || !sc.opacity_logit || !sc.sh))
            return DASS_ERR_INVALID_ARG;
    }
    if ((long long)n_cams * rec_stride >= (1ll << 32)) return DASS_ERR_INVALID_ARG;
    if (rec_stride > 0 && !splats) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, rec_stride, &ct)) return DASS_ERR_INVALID_ARG;
    return preprocess_scenes_launch(scenes, deg, ct, splats, as_stream(stream));
}

DASS_API int dass_preprocess_scenes_packed(const dass_scene* scenes, const dass_camera* cams, int n_cams, int tile,
                                          const int64_t* rec_offsets, dass_splat* splats, void* stream) {
    if (!scenes || !rec_offsets || n_cams < 1 || n_cams > DASS_MAX_CAMERAS) return DASS_ERR_INVALID_ARG;
    int deg = scenes[0].sh_degree;
    if (deg < 0 || deg > 3) return DASS_ERR_INVALID_ARG;
    long long n_max = 0;
    for (int c = 0; c < n_cams; ++c) {
        const dass_scene& sc = scenes[c];
        if (sc.sh_degree != deg || sc.n < 0 || rec_offsets[c + 1] - rec_offsets[c] != sc.n) return DASS_ERR_INVALID_ARG;
        if (sc.n > 0 && (!sc.means || !sc.log_scales || !sc.quats || !sc.opacity_logit || !sc.sh))
            return DASS_ERR_INVALID_ARG;
        n_max = sc.n > n_max ? sc.n : n_max;
    }
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, 0, &ct, rec_offsets)) return DASS_ERR_INVALID_ARG;
    if (rec_offsets[n_cams] > 0 && !splats) return DASS_ERR_INVALID_ARG;
    return preprocess_scenes_launch(scenes, deg, ct, splats, as_stream(stream), n_max);
}

DASS_API int dass_bin_sort_workspace(int64_t n_records, int64_t pair_capacity, int32_t tiles_total, size_t* bytes) {
    if (n_records < 0 || pair_capacity < 0 || tiles_total < 0 || !bytes) return DASS_ERR_INVALID_ARG;
    if (n_records >= (1ll << 32) || pair_capacity >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    *bytes = bin_sort_workspace_bytes(n_records, pair_capacity);
    return DASS_OK;
}

DASS_API int dass_bin_sort(const dass_splat* splats, int64_t rec_stride, const dass_camera* cams, int n_cams, int tile,
                           uint32_t* pair_rec, int64_t pair_capacity, uint32_t* tile_ranges, int64_t* counters,
                           void* workspace, size_t workspace_bytes, void* stream) {
    if (rec_stride < 0 || pair_capacity < 0 || !tile_ranges || !counters) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, rec_stride, &ct)) return DASS_ERR_INVALID_ARG;
    long long n_rec = (long long)n_cams * rec_stride;
    // sorted-pair positions are held as int32 by the compositing kernels: capacity < 2^31
    if (n_rec >= (1ll << 32) || pair_capacity >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    if (n_rec > 0 && (!splats || !pair_rec || !workspace)) return DASS_ERR_INVALID_ARG;
    if (workspace_bytes < bin_sort_workspace_bytes(n_rec, pair_capacity)) return DASS_ERR_OOM;
    return bin_sort_launch(splats, n_rec, ct, pair_rec, pair_capacity, tile_ranges, (long long*)counters, workspace,
                           workspace_bytes, as_stream(stream));
}

DASS_API int dass_bin_sort_packed(const dass_splat* splats, const int64_t* rec_offsets, const dass_camera* cams,
                                 int n_cams, int tile, uint32_t* pair_rec, int64_t pair_capacity,
                                 uint32_t* tile_ranges, int64_t* counters, void* workspace, size_t workspace_bytes,
                                 void* stream) {
    if (!rec_offsets || pair_capacity < 0 || !tile_ranges || !counters) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, 0, &ct, rec_offsets)) return DASS_ERR_INVALID_ARG;
    long long n_rec = rec_offsets[n_cams];
    if (pair_capacity >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    if (n_rec > 0 && (!splats || !pair_rec || !workspace)) return DASS_ERR_INVALID_ARG;
    if (workspace_bytes < bin_sort_workspace_bytes(n_rec, pair_capacity)) return DASS_ERR_OOM;
    return bin_sort_launch(splats, n_rec, ct, pair_rec, pair_capacity, tile_ranges, (long long*)counters, workspace,
                           workspace_bytes, as_stream(stream));
}

DASS_API int dass_bin_sort_split_workspace(int64_t n_rows, int n_cams, int64_t pair_capacity, size_t* bytes) {
    if (n_rows <= 0 || n_cams <= 0 || pair_capacity < 1 || pair_capacity >= (1ll << 31) || !bytes)
        return DASS_ERR_INVALID_ARG;
    if ((long long)n_cams * n_rows >= (1ll << 32)) return DASS_ERR_INVALID_ARG;
    *bytes = bin_sort_split_workspace_bytes(n_rows, (long long)n_cams * n_rows, pair_capacity);
    return DASS_OK;
}

DASS_API int dass_bin_sort_split(const dass_splat* splats, int64_t n_rows, const dass_camera* cams, int n_cams,
                                 int tile, const uint8_t* moving, int64_t pair_capacity, uint32_t* static_rec,
                                 uint32_t* static_depth, uint32_t* tile_start, int64_t* static_counters,
                                 uint32_t* moving_rec, int64_t* n_moving_rec, int32_t* moving_rows,
                                 int64_t* n_moving_rows, void* workspace, size_t workspace_bytes, void* stream) {
    if (n_rows <= 0 || pair_capacity < 1 || pair_capacity >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    if (!splats || !moving || !static_rec || !static_depth || !tile_start || !static_counters || !moving_rec ||
        !n_moving_rec || !moving_rows || !n_moving_rows || !workspace)
        return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, n_rows, &ct)) return DASS_ERR_INVALID_ARG;
    if ((long long)n_cams * n_rows >= (1ll << 32)) return DASS_ERR_INVALID_ARG;
    if (workspace_bytes < bin_sort_split_workspace_bytes(n_rows, (long long)n_cams * n_rows, pair_capacity))
        return DASS_ERR_OOM;
    const StaticBins sb{static_rec, static_depth, tile_start, (long long*)static_counters, moving_rec,
                        (long long*)n_moving_rec, moving_rows, (long long*)n_moving_rows};
    return bin_sort_split_launch(splats, n_rows, ct, moving, pair_capacity, sb, workspace, workspace_bytes,
                                 as_stream(stream));
}

DASS_API int dass_bin_sort_merge_workspace(int64_t moving_capacity, int64_t pair_capacity, int32_t tiles_total,
                                           size_t* bytes) {
    if (moving_capacity < 0 || moving_capacity >= (1ll << 32) || pair_capacity < 1 ||
        pair_capacity >= (1ll << 31) || tiles_total < 0 || !bytes)
        return DASS_ERR_INVALID_ARG;
    *bytes = bin_sort_merge_workspace_bytes(moving_capacity, pair_capacity, tiles_total);
    return DASS_OK;
}

DASS_API int dass_bin_sort_merge(const dass_splat* splats, int64_t n_rows, const dass_camera* cams, int n_cams,
                                 int tile, const uint32_t* moving_rec, const int64_t* n_moving_rec,
                                 int64_t moving_capacity, const uint32_t* static_rec, const uint32_t* static_depth,
                                 const uint32_t* tile_start, const int64_t* static_counters, uint32_t* pair_rec,
                                 int64_t pair_capacity, uint32_t* tile_ranges, int64_t* counters, void* workspace,
                                 size_t workspace_bytes, void* stream) {
    if (n_rows <= 0 || pair_capacity < 1 || pair_capacity >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    if (moving_capacity < 0 || moving_capacity >= (1ll << 32)) return DASS_ERR_INVALID_ARG;
    if (!splats || !moving_rec || !n_moving_rec || !static_rec || !static_depth || !tile_start || !static_counters ||
        !pair_rec || !tile_ranges || !counters || !workspace)
        return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, n_rows, &ct)) return DASS_ERR_INVALID_ARG;
    if (workspace_bytes < bin_sort_merge_workspace_bytes(moving_capacity, pair_capacity, ct.tiles_total))
        return DASS_ERR_OOM;
    const StaticBins sb{const_cast<uint32_t*>(static_rec), const_cast<uint32_t*>(static_depth),
                        const_cast<uint32_t*>(tile_start), (long long*)static_counters,
                        const_cast<uint32_t*>(moving_rec), (long long*)n_moving_rec, nullptr, nullptr};
    return bin_sort_merge_launch(splats, ct, sb, moving_capacity, pair_capacity, pair_rec, tile_ranges,
                                 (long long*)counters, workspace, workspace_bytes, as_stream(stream));
}

bool dass::batch_ok(int b) { return b == 32 || b == 64 || b == 128 || b == 256; }

DASS_API int dass_render_fwd(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* tile_ranges,
                             const dass_camera* cams, int n_cams, int tile, int batch, const float* bg, float* image,
                             float* T_final, int32_t* n_last, const uint32_t* tile_order, void* stream) {
    if (!batch_ok(batch) || !tile_ranges || !image || !T_final || !n_last) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, 0, &ct)) return DASS_ERR_INVALID_ARG;
    return render_fwd_launch(splats, pair_rec, tile_ranges, ct, batch, bg3(bg), image, T_final, n_last,
                             as_stream(stream), nullptr, nullptr, 1, tile_order);
}

DASS_API int dass_tile_order(const uint32_t* tile_ranges, int tiles_total, uint32_t* tile_order, void* stream) {
    if (tiles_total > 0 && (!tile_ranges || !tile_order)) return DASS_ERR_INVALID_ARG;
    return tile_order_launch(tile_ranges, tiles_total, tile_order, as_stream(stream));
}

DASS_API int dass_render_work(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* tile_ranges,
                              const dass_camera* cams, int n_cams, int tile, int batch, const uint8_t* full_grad,
                              int64_t rec_stride, float* image, float* T_final, int32_t* n_last, uint64_t* work,
                              void* stream) {
    if (!batch_ok(batch) || !tile_ranges || !image || !T_final || !n_last || !work) return DASS_ERR_INVALID_ARG;
    if (full_grad && rec_stride <= 0) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, 0, &ct)) return DASS_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    DASS_CHECK_CUDA(cudaMemsetAsync(work, 0, sizeof(uint64_t) * 5, st));
    return render_fwd_launch(splats, pair_rec, tile_ranges, ct, batch, make_float3(0.f, 0.f, 0.f), image, T_final,
                             n_last, st, reinterpret_cast<unsigned long long*>(work), full_grad,
                             rec_stride > 0 ? rec_stride : 1);
}

DASS_API int dass_render_bwd(const dass_splat* splats, int64_t n_records, const uint32_t* pair_rec,
                             const uint32_t* tile_ranges, const dass_camera* cams, int n_cams, int tile, int batch,
                             const float* bg, const float* T_final, const int32_t* n_last, const float* dL_dimage,
                             const uint8_t* full_grad, int64_t rec_stride, dass_splat_grad* splat_grads,
                             const uint32_t* tile_order, void* stream) {
    if (!batch_ok(batch) || n_records < 0 || !tile_ranges || !T_final || !n_last || !dL_dimage)
        return DASS_ERR_INVALID_ARG;
    if (full_grad && rec_stride <= 0) return DASS_ERR_INVALID_ARG;
    if (n_records > 0 && !splat_grads) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, 0, &ct)) return DASS_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    if (n_records > 0) DASS_CHECK_CUDA(cudaMemsetAsync(splat_grads, 0, sizeof(dass_splat_grad) * n_records, st));
    return render_bwd_launch(splats, pair_rec, tile_ranges, ct, batch, bg3(bg), T_final, n_last, dL_dimage,
                             full_grad, rec_stride > 0 ? rec_stride : 1, splat_grads, st, true, tile_order);
}

DASS_API int dass_preprocess_bwd(int64_t n, int sh_degree, const float* means, const float* log_scales,
                                 const float* quats, const float* opacity_logit, const float* sh, const uint8_t* keep,
                                 const dass_camera* cams, int n_cams, const dass_splat* splats,
                                 const dass_splat_grad* splat_grads, const int32_t* rows, int64_t n_rows,
                                 uint32_t grad_flags, int accumulate, float* d_means, float* d_log_scales,
                                 float* d_quats, float* d_opacity_logit, float* d_sh, void* stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || (grad_flags & ~DASS_GRAD_ALL)) return DASS_ERR_INVALID_ARG;
    long long nr = rows ? n_rows : n;
    if (nr < 0) return DASS_ERR_INVALID_ARG;
    if (nr > 0 && (!means || !log_scales || !quats || !opacity_logit || !sh || !splats || !splat_grads))
        return DASS_ERR_INVALID_ARG;
    if ((grad_flags & DASS_GRAD_MEANS) && !d_means) return DASS_ERR_INVALID_ARG;
    if ((grad_flags & DASS_GRAD_SCALES) && !d_log_scales) return DASS_ERR_INVALID_ARG;
    if ((grad_flags & DASS_GRAD_QUATS) && !d_quats) return DASS_ERR_INVALID_ARG;
    if ((grad_flags & DASS_GRAD_OPACITY) && !d_opacity_logit) return DASS_ERR_INVALID_ARG;
    if ((grad_flags & DASS_GRAD_SH) && !d_sh) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 8, n, &ct)) return DASS_ERR_INVALID_ARG;
    return preprocess_bwd_launch(n, sh_degree, means, log_scales, quats, opacity_logit, sh, keep, ct, splats,
                                 splat_grads, rows, nr, grad_flags, accumulate, d_means, d_log_scales, d_quats,
                                 d_opacity_logit, d_sh, nullptr, as_stream(stream));
}

DASS_API int dass_keep_grad(int64_t n, int sh_degree, const float* means, const float* log_scales, const float* quats,
                            const float* opacity_logit, const float* sh, const uint8_t* keep,
                            const dass_camera* cams, int n_cams, const dass_splat* splats,
                            const dass_splat_grad* splat_grads, const int32_t* rows, int64_t n_rows, float* d_keep,
                            void* stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3) return DASS_ERR_INVALID_ARG;
    long long nr = rows ? n_rows : n;
    if (nr < 0) return DASS_ERR_INVALID_ARG;
    if (nr > 0 && (!means || !log_scales || !quats || !opacity_logit || !sh || !splats || !splat_grads || !d_keep))
        return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 8, n, &ct)) return DASS_ERR_INVALID_ARG;
    return preprocess_bwd_launch(n, sh_degree, means, log_scales, quats, opacity_logit, sh, keep, ct, splats,
                                 splat_grads, rows, nr, 0u, 0, nullptr, nullptr, nullptr, nullptr, nullptr, d_keep,
                                 as_stream(stream));
}

DASS_API int dass_densify_stats(int64_t n, const dass_splat* splats, const dass_splat_grad* splat_grads,
                                const dass_camera* cams, int n_cams, float* accum, int32_t* count, void* stream) {
    if (n < 0 || (n > 0 && (!splats || !splat_grads || !accum || !count))) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 8, n, &ct)) return DASS_ERR_INVALID_ARG;
    return densify_stats_launch(n, ct, splats, splat_grads, accum, count, as_stream(stream));
}

DASS_API int dass_shift(int64_t n_dyn, const int32_t* dyn_idx, const float* offsets, const float* means,
                        const float* quats, float* out_means, float* out_quats, void* stream) {
    if (n_dyn < 0) return DASS_ERR_INVALID_ARG;
    if (n_dyn > 0 && (!dyn_idx || !offsets || !means || !quats || !out_means || !out_quats))
        return DASS_ERR_INVALID_ARG;
    return shift_launch(n_dyn, dyn_idx, offsets, means, quats, out_means, out_quats, as_stream(stream));
}

DASS_API int dass_shift_bwd(int64_t n_dyn, const int32_t* dyn_idx, const float* offsets, const float* quats,
                            const float* d_out_means, const float* d_out_quats, float* d_offsets, float* d_quats,
                            void* stream) {
    if (n_dyn < 0) return DASS_ERR_INVALID_ARG;
    if (n_dyn > 0 && (!dyn_idx || !offsets || !quats || !d_out_means || !d_out_quats || !d_offsets))
        return DASS_ERR_INVALID_ARG;
    return shift_bwd_launch(n_dyn, dyn_idx, offsets, quats, d_out_means, d_out_quats, d_offsets, d_quats,
                            as_stream(stream));
}

DASS_API int dass_adam(int64_t n_rows, int row_width, const int32_t* rows, int64_t n_sel, float* param,
                       const float* grad, float* adam_m, float* adam_v, int32_t* step_dev, const float* lr, float beta1,
                       float beta2, float eps, int increment_step, void* stream) {
    if (n_rows < 0 || row_width < 1 || row_width > 16 || !lr || !step_dev) return DASS_ERR_INVALID_ARG;
    long long ns = rows ? n_sel : n_rows;
    if (ns < 0) return DASS_ERR_INVALID_ARG;
    if (ns > 0 && (!param || !grad || !adam_m || !adam_v)) return DASS_ERR_INVALID_ARG;
    return adam_launch(ns, row_width, rows, param, grad, adam_m, adam_v, step_dev, lr, beta1, beta2, eps,
                       increment_step, as_stream(stream));
}

DASS_API int dass_loss_workspace(const dass_camera* cams, int n_cams, size_t* bytes) {
    static thread_local CamTable ct;
    if (!bytes || !make_cam_table(cams, n_cams, 16, 0, &ct)) return DASS_ERR_INVALID_ARG;
    *bytes = loss_workspace_bytes(ct);
    return DASS_OK;
}

DASS_API int dass_loss(const float* image, const float* target, const dass_camera* cams, int n_cams, float lambda,
                       float* dL_dimage, double* loss, void* workspace, size_t workspace_bytes, void* stream) {
    if (!image || !target || !dL_dimage || !loss || !(lambda >= 0.f && lambda <= 1.f)) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 16, 0, &ct)) return DASS_ERR_INVALID_ARG;
    if (lambda > 0.f && workspace_bytes < loss_workspace_bytes(ct)) return DASS_ERR_OOM;
    if (lambda > 0.f && reinterpret_cast<uintptr_t>(workspace) % 8) return DASS_ERR_INVALID_ARG;   // float2 maps
    return loss_launch(image, target, ct, lambda, 1.f / (float)n_cams, dL_dimage, loss, workspace, workspace_bytes,
                       as_stream(stream));
}

DASS_API int dass_loss_target_stats(const float* target, const dass_camera* cams, int n_cams, float* stats,
                                   void* stream) {
    if (!target || !stats || reinterpret_cast<uintptr_t>(stats) % 8) return DASS_ERR_INVALID_ARG;   // float2 pairs
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 16, 0, &ct)) return DASS_ERR_INVALID_ARG;
    return target_stats_launch(target, ct, stats, as_stream(stream));
}

DASS_API int dass_loss_cached(const float* image, const float* target, const float* target_stats,
                              const dass_camera* cams, int n_cams, float lambda, float* dL_dimage, double* loss,
                              void* workspace, size_t workspace_bytes, void* stream) {
    if (!image || !target || !target_stats || !dL_dimage || !loss || !(lambda >= 0.f && lambda <= 1.f))
        return DASS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(target_stats) % 8) return DASS_ERR_INVALID_ARG;   // float2 pairs
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 16, 0, &ct)) return DASS_ERR_INVALID_ARG;
    if (lambda > 0.f && workspace_bytes < loss_workspace_bytes(ct)) return DASS_ERR_OOM;
    if (lambda > 0.f && reinterpret_cast<uintptr_t>(workspace) % 8) return DASS_ERR_INVALID_ARG;   // float2 maps
    return loss_launch(image, target, ct, lambda, 1.f / (float)n_cams, dL_dimage, loss, workspace, workspace_bytes,
                       as_stream(stream), target_stats);
}

DASS_API int dass_inherit_workspace(int64_t n, size_t* bytes) {
    if (n < 0 || !bytes) return DASS_ERR_INVALID_ARG;
    *bytes = inherit_workspace_bytes(n);
    return DASS_OK;
}

DASS_API int dass_render_features(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* tile_ranges,
                                  const dass_camera* cams, int n_cams, int tile, const float* features,
                                  int n_features, int64_t rec_stride, float* out, void* stream) {
    if (rec_stride <= 0 || !features || !out || !pair_rec || !tile_ranges || !splats) return DASS_ERR_INVALID_ARG;
    if (rec_stride >= (1ll << 31) || reinterpret_cast<uintptr_t>(features) % 16) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, tile, rec_stride, &ct)) return DASS_ERR_INVALID_ARG;
    return render_features_launch(splats, pair_rec, tile_ranges, ct, features, n_features, rec_stride, out,
                                  as_stream(stream));
}

DASS_API int dass_object_ids(const float* x, int64_t n, int n_features, const float* W, const float* b,
                             int n_classes, int32_t* ids, void* stream) {
    if (n < 0 || n_classes < 1 || (n > 0 && (!x || !W || !b || !ids))) return DASS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(W)) % 16) return DASS_ERR_INVALID_ARG;  // float4 rows
    return object_ids_launch(x, n, n_features, W, b, n_classes, ids, as_stream(stream));
}

DASS_API int dass_dynamic_objects(const int32_t* ids, const uint8_t* dyn_area, int64_t n, int n_classes,
                                  uint32_t min_pixels, uint8_t* obj_mask, uint32_t* hist, void* stream) {
    if (n < 0 || n_classes < 1 || !obj_mask || !hist || (n > 0 && (!ids || !dyn_area))) return DASS_ERR_INVALID_ARG;
    return dynamic_objects_launch(ids, dyn_area, n, n_classes, min_pixels, obj_mask, hist, as_stream(stream));
}

DASS_API int dass_dynamic_gaussians(const float* features, int64_t n, int n_features, const float* W,
                                    const float* b, int n_classes, const uint8_t* obj_mask, uint8_t* dyn_mask,
                                    void* stream) {
    if (n < 0 || n_classes < 1 || (n > 0 && (!features || !W || !b || !obj_mask || !dyn_mask)))
        return DASS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(features) | reinterpret_cast<uintptr_t>(W)) % 16)
        return DASS_ERR_INVALID_ARG;   // rows are read as float4
    return dynamic_gaussians_launch(features, n, n_features, W, b, n_classes, obj_mask, dyn_mask, as_stream(stream));
}

DASS_API int dass_mask_rows_workspace(int64_t n, size_t* bytes) {
    if (n < 0 || !bytes) return DASS_ERR_INVALID_ARG;
    *bytes = mask_rows_workspace_bytes(n);
    return DASS_OK;
}

DASS_API int dass_mask_rows(const uint8_t* mask, int64_t n, int32_t* rows, int64_t* count, void* workspace,
                            size_t workspace_bytes, void* stream) {
    if (n < 0 || !count || (n > 0 && (!mask || !rows || !workspace))) return DASS_ERR_INVALID_ARG;
    return mask_rows_launch(mask, n, rows, reinterpret_cast<long long*>(count), workspace, workspace_bytes,
                            as_stream(stream));
}

DASS_API int dass_field_fwd(const dass_field* field, int64_t n_rows, const int32_t* rows, const float* means,
                            float* offsets, void* stream) {
    if (n_rows < 0 || (n_rows > 0 && (!means || !offsets))) return DASS_ERR_INVALID_ARG;
    return field_fwd_launch(field, n_rows, rows, means, offsets, as_stream(stream));
}

DASS_API int dass_field_bwd(const dass_field* field, int64_t n_rows, const int32_t* rows, const float* means,
                            const float* d_offsets, float* d_table, float* d_w1, float* d_b1, float* d_w2,
                            float* d_b2, void* stream) {
    if (n_rows < 0 || (n_rows > 0 && (!means || !d_offsets || !d_table || !d_w1 || !d_b1 || !d_w2 || !d_b2)))
        return DASS_ERR_INVALID_ARG;
    return field_bwd_launch(field, n_rows, rows, means, d_offsets, d_table, d_w1, d_b1, d_w2, d_b2,
                            as_stream(stream));
}

DASS_API int dass_prune_logits(int64_t n, const float* opacity_logit, float min_opacity, float* m, void* stream) {
    if (n < 0 || (n > 0 && (!opacity_logit || !m)) || !(min_opacity > 0.f && min_opacity < 1.f))
        return DASS_ERR_INVALID_ARG;
    return prune_logits_launch(n, opacity_logit, min_opacity, m, as_stream(stream));
}

DASS_API int dass_inherit_keep(int64_t n, const uint8_t* is_var, const float* m, uint8_t* keep, void* stream) {
    if (n < 0 || (n > 0 && (!is_var || !m || !keep))) return DASS_ERR_INVALID_ARG;
    return inherit_keep_launch(n, is_var, m, keep, as_stream(stream));
}

DASS_API int dass_inherit_mask_grad(int64_t n_rows, const int32_t* rows, const float* m, const float* d_keep,
                                    float lambda_inher, float* grad, double* loss, void* stream) {
    if (n_rows < 0 || (n_rows > 0 && (!m || !d_keep || !grad))) return DASS_ERR_INVALID_ARG;
    return inherit_mask_grad_launch(n_rows, rows, m, d_keep, lambda_inher, grad, loss, as_stream(stream));
}

DASS_API int dass_inherit(int64_t n, int sh_degree, const float* means, const float* log_scales, const float* quats,
                          const float* opacity_logit, const float* sh, const uint8_t* is_var, const float* m,
                          int erase, float* out_means, float* out_log_scales, float* out_quats,
                          float* out_opacity_logit, float* out_sh, uint8_t* is_var_out, int32_t* remap,
                          int64_t* n_out, void* workspace, size_t workspace_bytes, void* stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !n_out) return DASS_ERR_INVALID_ARG;
    if (n > 0 && (!means || !log_scales || !quats || !opacity_logit || !sh || !is_var || !out_means ||
                  !out_log_scales || !out_quats || !out_opacity_logit || !out_sh || !is_var_out || !remap))
        return DASS_ERR_INVALID_ARG;
    return inherit_launch(n, sh_degree, means, log_scales, quats, opacity_logit, sh, is_var, m, erase, out_means,
                          out_log_scales, out_quats, out_opacity_logit, out_sh, is_var_out, remap, (long long*)n_out,
                          workspace, workspace_bytes, as_stream(stream));
}

DASS_API int dass_error_pass_workspace(const dass_camera* cams, int n_cams, size_t* bytes) {
    static thread_local CamTable ct;
    if (!bytes || !make_cam_table(cams, n_cams, 16, 0, &ct)) return DASS_ERR_INVALID_ARG;
    *bytes = error_pass_workspace_bytes(ct);
    return DASS_OK;
}

DASS_API int dass_error_pass(const float* image, const float* target, const dass_camera* cams, int n_cams,
                             float quantile, int64_t n, const float* means, const uint8_t* is_var, float* error_map,
                             float* gamma, uint8_t* s_err, void* workspace, size_t workspace_bytes, void* stream) {
    if (!image || !target || n < 0 || !(quantile >= 0.f && quantile <= 1.f)) return DASS_ERR_INVALID_ARG;
    if (n > 0 && (!means || !s_err)) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(cams, n_cams, 16, 0, &ct)) return DASS_ERR_INVALID_ARG;
    return error_pass_launch(image, target, ct, (double)quantile, n, means, is_var, error_map, gamma, s_err, workspace,
                             workspace_bytes, as_stream(stream));
}

DASS_API int dass_densify_select_workspace(int64_t n, size_t* bytes) {
    if (n < 0 || !bytes) return DASS_ERR_INVALID_ARG;
    *bytes = select_workspace_bytes(n);
    return DASS_OK;
}

DASS_API int dass_densify_select(int64_t n, const float* accum, const int32_t* count, const uint8_t* s_err,
                                 const uint8_t* is_var, float tau_pos, float tau_err, int32_t k_max, int32_t* selected,
                                 int32_t* n_selected, void* workspace, size_t workspace_bytes, void* stream) {
    if (n < 0 || k_max < 0 || !n_selected || !(tau_pos >= 0.f) || !(tau_err >= 0.f)) return DASS_ERR_INVALID_ARG;
    if (n > 0 && (!accum || !count || (k_max > 0 && !selected))) return DASS_ERR_INVALID_ARG;
    if (n >= (1ll << 31)) return DASS_ERR_INVALID_ARG;
    return select_launch(n, accum, count, s_err, is_var, tau_pos, tau_err, k_max, selected, n_selected, workspace,
                         workspace_bytes, as_stream(stream));
}

DASS_API int dass_spawn(int64_t n, int sh_degree, float* means, float* log_scales, float* quats, float* opacity_logit,
                        float* sh, uint8_t* is_var, const int32_t* selected, const int32_t* n_selected, int32_t k_max,
                        const float* z, int64_t* n_total, void* stream) {
    if (n < 0 || k_max < 0 || sh_degree < 0 || sh_degree > 3 || !n_selected || !n_total) return DASS_ERR_INVALID_ARG;
    if (!means || !log_scales || !quats || !opacity_logit || !sh || !is_var || (k_max > 0 && (!selected || !z)))
        return DASS_ERR_INVALID_ARG;
    return spawn_launch(n, sh_degree, means, log_scales, quats, opacity_logit, sh, is_var, selected, n_selected, k_max,
                        z, (long long*)n_total, as_stream(stream));
}

