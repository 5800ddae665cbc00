/*
 * dass.h -- C ABI of libdass, the GB300 (sm_103a) hot path of
 * "Dynamics-Aware Gaussian Splatting Streaming" (DASS, arXiv 2411.14847).
 *
 * Problem statement (Sec. 3.1): at timestep t the method starts from the Gaussians
 * G_{t-1} and derives G_t from the C synchronised views of timestep t, in three stages:
 * selective inheritance (Sec. 3.2), dynamics-aware shift (Sec. 3.3) and error-guided
 * densification (Sec. 3.4). Every stage optimises Gaussians through the differentiable
 * 3D Gaussian-splatting renderer of App. A.1 (projection, depth-ordered alpha blending).
 *
 * Conventions shared by every entry point
 *  - Return value: DASS_OK (0) or a negative dass_status. Argument errors are detected on
 *    the host before anything is launched; DASS_ERR_CUDA reports a failed launch or CUDA
 *    call (see dass_last_error()).
 *  - Memory: every array argument is a DEVICE pointer owned by the caller, except where a
 *    parameter says "host". The library never allocates device memory (dass_bin_sort_static
 *    uses one file-scope device array instead). Scratch memory is a caller-provided
 *    `workspace` whose size the matching *_workspace() query returns.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). Calls only
 *    enqueue work; none synchronises the host except the stage drivers (dass_step,
 *    dass_inherit_step, dass_densify_step) and dass_timestep, as documented there.
 *    Results are valid once the stream reaches them.
 *  - Layout: float32, structure of arrays, N-major, contiguous. Gaussians:
 *      means[N][3], log_scales[N][3], quats[N][4] (w,x,y,z; need not be unit),
 *      opacity_logit[N], sh[N][K][3] with K = (sh_degree+1)^2 real-SH coefficients
 *      (index k = l*l + l + m, basis without Condon-Shortley phase), sh_degree <= 3.
 *  - Cameras (host arrays of dass_camera): viewmat is the row-major world->camera 4x4
 *    (OpenCV axes: x right, y down, z forward); pixel centres sit at integer coordinates.
 *    At most DASS_MAX_CAMERAS cameras per call.
 *  - Projected records: one dass_splat per (camera, Gaussian), record index
 *    c * rec_stride + g (rec_stride = N for one scene seen by all cameras).
 *  - Images are planar per camera, cameras concatenated: camera c occupies
 *    3*H_c*W_c floats starting at 3 * sum_{c'<c} H_c' W_c', channel-major then row-major.
 *  - Tiles: B x B pixel tiles (B in {8,16,32}); camera c owns the global tile ids
 *    [tile_base_c, tile_base_c + ceil(W/B)*ceil(H/B)), row-major, cameras in order.
 */
#ifndef DASS_H
#define DASS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DASS_MAX_CAMERAS 64
#define DASS_VERSION 1

typedef enum dass_status {
    DASS_OK = 0,
    DASS_ERR_INVALID_ARG = -1,  /* bad size, NULL pointer, unsupported tile/batch/degree */
    DASS_ERR_CUDA = -2,         /* a CUDA launch or call failed; dass_last_error() has text */
    DASS_ERR_OOM = -3,          /* workspace smaller than the matching *_workspace() size */
    DASS_ERR_CAPACITY = -4,     /* pair or Gaussian capacity exceeded; grow and retry */
    DASS_ERR_TIMEOUT = -5,      /* a bounded wait gave up */
    DASS_ERR_UNSUPPORTED = -6
} dass_status;

/* Camera of App. A.1's projection: world->camera viewmat, pinhole intrinsics. 88 bytes.
 * width, height > 0 with (width + 16) * (height + 16) < 2^31 (pixel offsets within a plane
 * are 32-bit); every entry taking cameras returns DASS_ERR_INVALID_ARG otherwise. */
typedef struct dass_camera {
    float viewmat[16];
    float fx, fy, cx, cy;
    int32_t width, height;
} dass_camera;

/* Screen-space record of one Gaussian in one camera (App. A.1), written by dass_preprocess.
 * radius == 0 marks a Gaussian that contributes to no pixel of that camera (behind the
 * near plane z <= 0.2, opacity <= 1/255, or footprint outside every tile). 48 bytes. */
typedef struct dass_splat {
    float mean2d[2];   /* pixel coordinates (u, v) */
    float conic[3];    /* inverse 2D covariance (a, b, c): power = -(a dx^2 + 2 b dx dy + c dy^2)/2 */
    float opacity;     /* sigmoid(logit), times the inheritance mask (Eq. 1) */
    float rgb[3];      /* view-dependent colour max(SH(d) + 0.5, 0) */
    float depth;       /* camera-space z */
    int32_t radius;    /* opacity-aware pixel radius of the alpha >= 1/255 footprint */
    int32_t tiles;     /* tiles covered by [u-r,u+r] x [v-r,v+r] at the tile size of the call */
} dass_splat;

/* Gradient of the loss w.r.t. the fields of one dass_splat (accumulated by dass_render_bwd). */
typedef struct dass_splat_grad {
    float mean2d[2];
    float conic[3];
    float opacity;
    float rgb[3];
    float pad[3];
} dass_splat_grad;

/* grad_flags of dass_preprocess_bwd: which parameter gradients to produce. */
#define DASS_GRAD_MEANS   1u
#define DASS_GRAD_SCALES  2u
#define DASS_GRAD_QUATS   4u
#define DASS_GRAD_OPACITY 8u
#define DASS_GRAD_SH      16u
#define DASS_GRAD_ALL     31u

/* ------------------------------------------------------------------ utilities */

int dass_version(void);
const char* dass_status_string(int status);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char* dass_last_error(void);

/* Number of libdass kernels this host thread has enqueued so far (a CUDA-graph replay counts
 * every kernel it runs). Used to report the kernel launches inside a timed region. */
int64_t dass_kernel_launches(void);

/* Host helper: total tiles and pixels of a camera set at tile size B. */
int dass_tile_layout(const dass_camera* cams, int n_cams, int tile, int32_t* tiles_total,
                     int64_t* pixels_total);

/* ------------------------------------------------------------------ rasteriser (App. A.1) */

/* Projection of every Gaussian into every camera (App. A.1: Sigma = R S S^T R^T,
 * Sigma_2D = J W Sigma W^T J^T, plus 0.3 I low-pass; SH colour), one record per
 * (camera, Gaussian) at splats[c * n + g]. `keep` (optional, N bytes, NULL = all 1) is the
 * quantised inheritance mask of Eq. 1, multiplying the activated opacity and scale.
 * `tile` only fills dass_splat.tiles. One launch for all cameras. */
int dass_preprocess(int64_t n, int sh_degree, const float* means, const float* log_scales,
                    const float* quats, const float* opacity_logit, const float* sh,
                    const uint8_t* keep, const dass_camera* cams /* host */, int n_cams,
                    int tile, dass_splat* splats, void* stream);

/* Gaussian set of one scene (device pointers, layout as above). */
typedef struct dass_scene {
    int64_t n;
    int32_t sh_degree;
    int32_t pad;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logit;
    const float* sh;
} dass_scene;

/* Serving form of dass_preprocess (novel-view rendering of resident scenes, no paper section:
 * the render of App. A.1 applied to requests of several scenes in one launch). Camera c shows
 * scenes[c] (host array [n_cams]; all scenes of one call share sh_degree); its records are
 * splats[c * rec_stride + g] for g < scenes[c].n, and the records g in [scenes[c].n, rec_stride)
 * are written as culled (radius 0), so dass_bin_sort / dass_render_fwd with the same rec_stride
 * render every request of the batch in one launch each. rec_stride >= max n. */
int dass_preprocess_scenes(const dass_scene* scenes /* host */, const dass_camera* cams /* host */,
                           int n_cams, int tile, int64_t rec_stride, dass_splat* splats, void* stream);

/* Packed serving form (same render, no padding): camera c's records are the segment
 * splats[rec_offsets[c] + g], g < scenes[c].n, with rec_offsets (host, n_cams + 1 values)
 * rec_offsets[0] = 0 and rec_offsets[c + 1] = rec_offsets[c] + scenes[c].n, total < 2^32.
 * A batch of requests of small and large scenes then projects and sorts sum_c n_c records instead
 * of n_cams * max_c n_c. Pair with dass_bin_sort_packed (same offsets) and dass_render_fwd.
 * DASS_ERR_INVALID_ARG if the offsets do not match the scene sizes. */
int dass_preprocess_scenes_packed(const dass_scene* scenes /* host */, const dass_camera* cams /* host */,
                                  int n_cams, int tile, const int64_t* rec_offsets /* host */,
                                  dass_splat* splats, void* stream);

/* Bytes of scratch that dass_bin_sort needs for n_records = n_cams * rec_stride records,
 * `pair_capacity` (tile, Gaussian) pairs and `tiles_total` tiles. n_records < 2^32 and
 * pair_capacity < 2^31 (sorted-pair positions are 32-bit signed in the compositing kernels),
 * else DASS_ERR_INVALID_ARG. */
int dass_bin_sort_workspace(int64_t n_records, int64_t pair_capacity, int32_t tiles_total,
                            size_t* bytes);

/* Tile binning and device radix sort (tile-based rasterisation, Sec. 1 / Sec. 4.2).
 * Each visible record (radius > 0) emits one (tile, record) pair per tile that its footprint
 * ellipse {d : d^T conic d <= 2 ln(255 o) + 0.01} reaches (at a pixel centre of the tile; every
 * pixel with alpha >= 1/255 lies inside that ellipse, so no contribution is lost); pairs are ordered by
 * the 64-bit key (global tile id << 32 | depth bits), stable in record order: an LSD radix
 * sort whose 32 depth-bit passes run on the records before duplication and whose tile-bit
 * passes run on the pairs. Outputs: pair_rec[M] (record id per sorted pair),
 * tile_ranges[2*tiles_total] ([start, end) per tile, 0,0 when empty) and
 * counters[0] = M, counters[1] = 1 if M > pair_capacity (pairs beyond the capacity are
 * dropped: the render is then incomplete and the caller must grow and rerun; a pair count of
 * 2^31 or more cannot be stored by any capacity the call accepts).
 * Returns DASS_ERR_INVALID_ARG if pair_capacity >= 2^31 and DASS_ERR_OOM if workspace_bytes <
 * dass_bin_sort_workspace(). */
int dass_bin_sort(const dass_splat* splats, int64_t rec_stride, const dass_camera* cams /* host */,
                  int n_cams, int tile, uint32_t* pair_rec, int64_t pair_capacity,
                  uint32_t* tile_ranges, int64_t* counters, void* workspace,
                  size_t workspace_bytes, void* stream);

/* dass_bin_sort over packed per-camera record segments (camera c owns records
 * [rec_offsets[c], rec_offsets[c + 1]), rec_offsets a host array of n_cams + 1 non-decreasing values
 * with rec_offsets[0] = 0 and total < 2^32), e.g. the output of dass_preprocess_scenes_packed. Same
 * outputs, order and errors as dass_bin_sort; the workspace is dass_bin_sort_workspace(
 * rec_offsets[n_cams], pair_capacity, tiles_total). */
int dass_bin_sort_packed(const dass_splat* splats, const int64_t* rec_offsets /* host */,
                         const dass_camera* cams /* host */, int n_cams, int tile, uint32_t* pair_rec,
                         int64_t pair_capacity, uint32_t* tile_ranges, int64_t* counters, void* workspace,
                         size_t workspace_bytes, void* stream);

/* Incremental binning for the stage iterations (Sec. 3.2-3.4). A stage trains only a subset of the
 * Gaussians -- the dynamic rows in the shift stage (Sec. 3.3), the var rows in the inheritance and
 * densification stages (Sec. 3.2, 3.4) -- so the records of every other row are the same at every
 * iteration of the stage. dass_bin_sort_split bins and sorts those static records once;
 * dass_bin_sort_merge then bins and sorts only the moving rows' records and merges them into the
 * static per-tile lists. Its pair_rec, tile_ranges and counters equal those of dass_bin_sort over
 * all records, pair for pair (both follow the key (tile, depth bits, record id)).
 *
 * Records are camera-major, n_rows per camera (record c * n_rows + row, as dass_preprocess writes
 * them with rec_stride = n_rows). moving[n_rows] (device, nonzero = moving row). Outputs of
 * the split (device, caller-owned, kept for the merges):
 *   static_rec[pair_capacity], static_depth[pair_capacity]: record and depth key (float bits) of each
 *     static pair in sorted order;
 *   tile_start[tiles_total + 1]: first static position of each tile;
 *   static_counters[3]: as dass_bin_sort's counters, for the static pairs;
 *   moving_rec[n_cams * n_rows]: records of the moving rows, camera by camera, ascending;
 *   n_moving_rec[1] (int64): their count;
 *   moving_rows[n_rows] (int32) and n_moving_rows[1] (int64): the moving rows, ascending.
 * Workspace: dass_bin_sort_split_workspace. DASS_ERR_INVALID_ARG for n_rows <= 0 or
 * n_cams * n_rows >= 2^32 or pair_capacity >= 2^31. */
int dass_bin_sort_split_workspace(int64_t n_rows, int n_cams, int64_t pair_capacity, size_t* bytes);
int dass_bin_sort_split(const dass_splat* splats, int64_t n_rows, const dass_camera* cams /* host */, int n_cams,
                        int tile, const uint8_t* moving, int64_t pair_capacity, uint32_t* static_rec,
                        uint32_t* static_depth, uint32_t* tile_start, int64_t* static_counters,
                        uint32_t* moving_rec, int64_t* n_moving_rec, int32_t* moving_rows,
                        int64_t* n_moving_rows, void* workspace, size_t workspace_bytes, void* stream);

/* The merge: splats hold the current records of every row (the static rows' unchanged since the
 * split); moving_capacity >= *n_moving_rec (host bound: n_cams times the number of moving rows;
 * larger counts are cut to it). Outputs as dass_bin_sort: pair_rec[pair_capacity], tile_ranges[2 *
 * tiles_total], counters[3] (counters[1] = 1 when the static and moving pairs together exceed
 * pair_capacity; positions beyond it are dropped and the ranges clamped). Workspace:
 * dass_bin_sort_merge_workspace. The call enqueues work only (graph-capturable). */
int dass_bin_sort_merge_workspace(int64_t moving_capacity, int64_t pair_capacity, int32_t tiles_total,
                                  size_t* bytes);
int dass_bin_sort_merge(const dass_splat* splats, int64_t n_rows, const dass_camera* cams /* host */, int n_cams,
                        int tile, const uint32_t* moving_rec, const int64_t* n_moving_rec,
                        int64_t moving_capacity, const uint32_t* static_rec, const uint32_t* static_depth,
                        const uint32_t* tile_start, const int64_t* static_counters, uint32_t* pair_rec,
                        int64_t pair_capacity, uint32_t* tile_ranges, int64_t* counters, void* workspace,
                        size_t workspace_bytes, void* stream);

/* Size of the static device scratch array used by dass_bin_sort_static (64 MiB). */
#define DASS_BIN_SORT_STATIC_BYTES (64ull << 20)

/* Same result as dass_bin_sort, for callers that cannot allocate device memory: the paper has no
 * counterpart to this entry point. Some hosts own every device allocation through their own
 * pool and do not allow a library to call cudaMalloc (real-time render plugins, engines with a
 * fixed memory budget), and for some callers an allocation would block or synchronise the
 * device at a moment they cannot afford. This variant takes the same inputs and outputs as
 * dass_bin_sort but no workspace: its scratch is a file-scope device array of
 * DASS_BIN_SORT_STATIC_BYTES bytes that every GPU loading the library holds until the process
 * exits. The call itself allocates nothing.
 *  - Limit: dass_bin_sort_workspace(n_cams * rec_stride, pair_capacity, ...) must not exceed
 *    DASS_BIN_SORT_STATIC_BYTES (e.g. 500k records with 4M pairs fit); larger requests return
 *    DASS_ERR_OOM with an explanation in dass_last_error() and launch nothing.
 *  - Set-up: the first call on a device looks up the device address of the array (once per
 *    device, with that device current); make that first call before any stream capture. The
 *    address is kept for the life of the process: do not use this entry point across a
 *    cudaDeviceReset or another teardown of the device's primary context.
 *  - Sharing: every call uses the same array, which keeps the previous call's contents; the
 *    sort writes every scratch word before reading it, so nothing needs clearing. Calls whose
 *    work overlaps on the GPU (other streams, other threads) race on the array: serialise them. */
int dass_bin_sort_static(const dass_splat* splats, int64_t rec_stride, const dass_camera* cams /* host */,
                         int n_cams, int tile, uint32_t* pair_rec, int64_t pair_capacity,
                         uint32_t* tile_ranges, int64_t* counters, void* stream);

/* Forward compositing of every tile of every camera in one launch (App. A.1 blending):
 * per pixel, front to back over its tile's list, alpha = min(0.99, o exp(power)); alpha
 * < 1/255 is skipped; before adding a Gaussian, T (1 - alpha) < 1e-4 stops the pixel and
 * the Gaussian is not added. Writes image (planar), T_final[pixels] and n_last[pixels]
 * (sorted-pair position of the last added Gaussian, -1 if none). bg: host float[3] or NULL
 * (black). batch in {32, 64, 128, 256}: list entries each compositing warp (one 8 x 16 pixel block,
 * 8 x 8 at 8-pixel tiles) examines and stages in shared memory per round; the result does not
 * depend on it. tile_order: the order in which the launch's blocks take the tiles (a permutation
 * of 0 .. tiles_total - 1, as dass_tile_order writes it), or NULL for tile order; the result does
 * not depend on it (entries outside that range are skipped, and a tile left out of the order is
 * not composited). */
int dass_render_fwd(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* tile_ranges,
                    const dass_camera* cams /* host */, int n_cams, int tile, int batch,
                    const float* bg /* host, 3 */, float* image, float* T_final, int32_t* n_last,
                    const uint32_t* tile_order /* device or NULL */, void* stream);

/* Schedule of the compositing launches (no counterpart in the paper, whose rasteriser renders one
 * view per launch): writes tile_order (device uint32[tiles_total]), a permutation of the tiles
 * sorted by descending list length (tile_ranges[2 t + 1] - tile_ranges[2 t], bucketed by 8 steps
 * per power of two; empty lists last). Passed as tile_order to dass_render_fwd / dass_render_bwd,
 * it makes the launch's blocks take the longest lists first, so that the launch does not end on a
 * few long tiles; the results are the same with or without it (the order within a bucket is not
 * deterministic and does not need to be). One 1024-thread block; tiles_total <= 0 is a no-op. */
int dass_tile_order(const uint32_t* tile_ranges, int tiles_total, uint32_t* tile_order, void* stream);

/* Measurement variant of dass_render_fwd (same outputs, black background) that also counts
 * the work of the compositing: work[0] = (pixel, Gaussian) pairs whose alpha the forward
 * evaluates (after the per-warp footprint culling, up to each pixel's own stop), work[1] = pairs
 * added to a pixel (the algorithmic work), work[2] = sum over pixels of the length of the tile
 * list prefix up to the pixel's last added Gaussian, work[3] = pixels, work[4] = added pairs whose
 * Gaussian g = record % rec_stride has full_grad[g] != 0 (all of them if full_grad is NULL).
 * work: device uint64[5], zeroed by the call. Not used on the timed path. */
int dass_render_work(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* tile_ranges,
                     const dass_camera* cams /* host */, int n_cams, int tile, int batch,
                     const uint8_t* full_grad, int64_t rec_stride, float* image, float* T_final,
                     int32_t* n_last, uint64_t* work, void* stream);

/* Reverse-order backward of dass_render_fwd. Recomputes alpha from the saved T_final and
 * n_last (T_j = T_{j+1} / (1 - alpha_j)); per Gaussian the 9 gradients of each 8 x 16 pixel block
 * are reduced across the block's warp with shuffles and added to splat_grads[record] with global
 * vector atomics. splat_grads (n_records entries) is zeroed by this call first.
 * full_grad (optional, device uint8 per Gaussian g = record % rec_stride; NULL = all): Gaussians
 * with full_grad[g] == 0 only receive splat_grads.mean2d (what the densification statistics
 * read), their other fields stay 0 -- e.g. the static Gaussians of the shift stage (Sec. 3.3),
 * whose parameters are not optimised; transmittance and colours are propagated identically.
 * batch and tile_order as in dass_render_fwd. */
int dass_render_bwd(const dass_splat* splats, int64_t n_records, const uint32_t* pair_rec,
                    const uint32_t* tile_ranges, const dass_camera* cams /* host */, int n_cams,
                    int tile, int batch, const float* bg /* host, 3 */, const float* T_final,
                    const int32_t* n_last, const float* dL_dimage, const uint8_t* full_grad,
                    int64_t rec_stride, dass_splat_grad* splat_grads,
                    const uint32_t* tile_order /* device or NULL */, void* stream);

/* Chain rule from splat gradients to parameter gradients (App. A.1 projection, SH colour,
 * sigmoid/exp activations, Eq. 1 mask), summed over cameras. rows (optional, n_rows
 * Gaussian indices) restricts the work to those Gaussians and makes the outputs compact
 * ([n_rows][...]); rows == NULL means all n Gaussians. Only the outputs selected by
 * grad_flags are written (others may be NULL). accumulate != 0 adds to the outputs. */
int dass_preprocess_bwd(int64_t n, int sh_degree, const float* means, const float* log_scales,
                        const float* quats, const float* opacity_logit, const float* sh,
                        const uint8_t* keep, const dass_camera* cams /* host */, int n_cams,
                        const dass_splat* splats, const dass_splat_grad* splat_grads,
                        const int32_t* rows, int64_t n_rows, uint32_t grad_flags, int accumulate,
                        float* d_means, float* d_log_scales, float* d_quats,
                        float* d_opacity_logit, float* d_sh, void* stream);

/* dL/dkeep of the inheritance mask (Sec. 3.2, Eq. 1: the mask multiplies the activated opacity
 * and scale, so dL/dkeep = o dL/do_r + sum_j s_j dL/ds_r,j with o = sigmoid(logit), s_j =
 * exp(log_scale_j)), summed over cameras, at the mask `keep` the splats were rendered with.
 * Same inputs and row selection as dass_preprocess_bwd; d_keep is [n_rows] (rows given) or [n].
 * A row rendered with keep = 0 has no footprint and gets 0. */
int dass_keep_grad(int64_t n, int sh_degree, const float* means, const float* log_scales,
                   const float* quats, const float* opacity_logit, const float* sh,
                   const uint8_t* keep, const dass_camera* cams /* host */, int n_cams,
                   const dass_splat* splats, const dass_splat_grad* splat_grads,
                   const int32_t* rows, int64_t n_rows, float* d_keep, void* stream);

/* ------------------------------------------------------------------ deformation fields (Sec. 3.3) */

/* Hash-encoding deformation field (Sec. 3.3, App. B.2: multiresolution hash encoding of I-NGP
 * followed by a small MLP). For a Gaussian at position p:
 *   x = clamp((p - bbox_min) / (bbox_max - bbox_min), 0, 1)^3;
 *   level l < levels: N_l = res[l] cells per axis, vertices 0..N_l; the 8 vertices of x's cell
 *   are looked up in table[l][T][features] (T = 2^log2_table) at index
 *   i + j (N_l + 1) + k (N_l + 1)^2 when (N_l + 1)^3 <= T, else the spatial hash
 *   (i * 1 ^ j * 2654435761 ^ k * 805459861) mod T (uint32 arithmetic), and trilinearly
 *   interpolated: enc = concat_l interp_l  (levels * features values);
 *   h = relu(w1 enc + b1) (hidden units), out = w2 h + b2 (7 values);
 *   offsets = (out[0..2], 1 + out[3], out[4], out[5], out[6]) = (dmu, sigma) for dass_shift.
 * All arrays are FP32 device memory: table [levels][T][features], w1 [hidden][levels*features],
 * b1 [hidden], w2 [7][hidden], b2 [7]. Limits: levels <= 16, features in {2, 4},
 * levels * features <= 64, hidden == 64. */
typedef struct dass_field {
    int32_t levels;
    int32_t features;
    int32_t log2_table;
    int32_t hidden;
    int32_t res[16];          /* N_l per level */
    float bbox_min[3];
    float bbox_max[3];
    const float* table;
    const float* w1;
    const float* b1;
    const float* w2;
    const float* b2;
} dass_field;

/* offsets[r][7] of rows r < n_rows (row g = rows[r], or r if rows == NULL) at positions
 * means[g] (n x 3). */
int dass_field_fwd(const dass_field* field, int64_t n_rows, const int32_t* rows, const float* means,
                   float* offsets, void* stream);

/* Gradients of the field's parameters from d_offsets[n_rows][7] (e.g. dass_shift_bwd's
 * d_offsets): ADDED to d_table, d_w1, d_b1, d_w2, d_b2 (same shapes as the parameters; the
 * caller zeroes them). The forward is recomputed; table gradients are scattered with atomics. */
int dass_field_bwd(const dass_field* field, int64_t n_rows, const int32_t* rows, const float* means,
                   const float* d_offsets, float* d_table, float* d_w1, float* d_b1, float* d_w2,
                   float* d_b2, void* stream);

/* ------------------------------------------------------------------ dynamics mask (Sec. 3.3) */

/* Identity-feature rendering (Sec. 3.3: Gaussian Grouping object features, rendered like colour
 * to query object IDs in any view): the lists, alpha, skip and stop rules of dass_render_fwd
 * (no background) compositing per-Gaussian feature vectors features[g][n_features], g = record
 * % rec_stride (< 2^31). n_features in {4, 8, 16, 32}; features 16-byte aligned (its rows are read
 * as float4). out: pixel-major [pixels_total][n_features]. */
int dass_render_features(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* tile_ranges,
                         const dass_camera* cams /* host */, int n_cams, int tile, const float* features,
                         int n_features, int64_t rec_stride, float* out, void* stream);

/* Object IDs of feature rows (the linear classifier of Gaussian Grouping):
 * ids[i] = argmax_k (W x_i + b)_k over n_classes (ties to the lower k), W [n_classes][n_features].
 * x and W must be 16-byte aligned (DASS_ERR_INVALID_ARG otherwise); n_features in {4, 8, 16, 32}. */
int dass_object_ids(const float* x, int64_t n, int n_features, const float* W, const float* b, int n_classes,
                    int32_t* ids, void* stream);

/* Dynamic objects (Sec. 3.3: the IDs rendered inside the dynamic image areas): obj_mask[k] = 1 iff
 * at least min_pixels pixels i with dyn_area[i] != 0 have ids[i] == k. hist: device scratch
 * [n_classes] uint32. The dynamic areas (optical flow above a threshold) are an input. */
int dass_dynamic_objects(const int32_t* ids, const uint8_t* dyn_area, int64_t n, int n_classes,
                         uint32_t min_pixels, uint8_t* obj_mask, uint32_t* hist, void* stream);

/* Per-Gaussian dynamics mask (Sec. 3.3): dyn_mask[g] = obj_mask[argmax_k (W f_g + b)_k] for the
 * Gaussians' own identity features f_g (features and W 16-byte aligned, as in dass_object_ids). */
int dass_dynamic_gaussians(const float* features, int64_t n, int n_features, const float* W, const float* b,
                           int n_classes, const uint8_t* obj_mask, uint8_t* dyn_mask, void* stream);

/* Stable compaction of a byte mask: rows[0..*count) = the indices i with mask[i] != 0, ascending
 * (count: device int64), e.g. the dyn_idx of the shift stage from dass_dynamic_gaussians. */
int dass_mask_rows_workspace(int64_t n, size_t* bytes);
int dass_mask_rows(const uint8_t* mask, int64_t n, int32_t* rows, int64_t* count, void* workspace,
                   size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------ DASS stages */

/* Low-opacity pruning of the densification stage (Sec. 3.4: var Gaussians of very low opacity
 * are eliminated) expressed as keep logits for dass_inherit: m[g] = opacity_logit[g] -
 * logit(min_opacity), positive iff sigmoid(opacity_logit[g]) > min_opacity. Passing m to
 * dass_inherit (erase = 0) keeps every base row and the var rows above the threshold, in order.
 * min_opacity in (0, 1). */
int dass_prune_logits(int64_t n, const float* opacity_logit, float min_opacity, float* m, void* stream);

/* Rendering mask of the selective-inheritance stage (Sec. 3.2, Eq. 1): keep[g] =
 * Quant(sigmoid(m[g])) = [m[g] > 0] for var rows (is_var[g] != 0), 1 for base rows. */
int dass_inherit_keep(int64_t n, const uint8_t* is_var, const float* m, uint8_t* keep, void* stream);

/* Straight-through gradient of the inheritance logits (App. B.2 STE applied to the loss of
 * Eq. 2): for r < n_rows, g = rows[r] (rows == NULL: g = r),
 * grad[g] = (d_keep[r] + lambda_inher) * sigmoid(m[g]) (1 - sigmoid(m[g])), where d_keep[r] is
 * dL/dkeep from dass_keep_grad. loss (optional, device double) accumulates the mask loss
 * lambda_inher * sum_r sigmoid(m[rows[r]]). grad rows outside `rows` are not written. */
int dass_inherit_mask_grad(int64_t n_rows, const int32_t* rows, const float* m, const float* d_keep,
                           float lambda_inher, float* grad, double* loss, void* stream);

/* Dynamics-aware shift (Sec. 3.3), dynamic rows only: for d < n_dyn with n = dyn_idx[d],
 * out_means[n] = means[n] + dmu_d and out_quats[n] = norm(quats[n]) x norm(sigma_d)
 * (Hamilton product). offsets[n_dyn][7] = (dmu[3], sigma[4]). Static rows of out_* are not
 * touched (the caller keeps them equal to the inputs). n_dyn == 0 is a no-op. */
int dass_shift(int64_t n_dyn, const int32_t* dyn_idx, const float* offsets, const float* means,
               const float* quats, float* out_means, float* out_quats, void* stream);

/* Backward of dass_shift: from compact d_out_means[n_dyn][3], d_out_quats[n_dyn][4] (the
 * gradients of the shifted rows, e.g. from dass_preprocess_bwd with rows = dyn_idx) to
 * d_offsets[n_dyn][7]. Only dynamic Gaussians receive gradients (Sec. 3.3). d_quats (optional,
 * compact [n_dyn][4], NULL = not computed) receives the gradient w.r.t. the input quaternion
 * quats[dyn_idx[d]] through norm(q) x norm(sigma); the input means' gradient equals d_out_means
 * (the shift adds dmu). */
int dass_shift_bwd(int64_t n_dyn, const int32_t* dyn_idx, const float* offsets, const float* quats,
                   const float* d_out_means, const float* d_out_quats, float* d_offsets,
                   float* d_quats, void* stream);

/* Masked Adam step (optimiser not named by the paper; the 3DGS family uses Adam):
 * for each selected row r (rows == NULL: all n_rows rows) and k < row_width:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr_k m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps),
 * with t = *step_dev + 1 read on the device (so one captured launch serves every step) and
 * lr_k = lr[k] (host array of row_width learning rates). Unselected rows are untouched.
 * If increment_step != 0 the call also does *step_dev += 1 after the update. */
int dass_adam(int64_t n_rows, int row_width, const int32_t* rows, int64_t n_sel, float* param,
              const float* grad, float* adam_m, float* adam_v, int32_t* step_dev,
              const float* lr /* host, row_width */, float beta1, float beta2, float eps,
              int increment_step, void* stream);

/* Bytes of scratch for dass_loss over a camera set (3 SSIM partial maps per pixel/channel); the
 * workspace must be 8-byte aligned. */
int dass_loss_workspace(const dass_camera* cams, int n_cams, size_t* bytes);

/* Fidelity loss of Eq. 3: L = mean_c[(1-lambda) L1_c + lambda (1 - SSIM_c)], SSIM with an
 * 11x11 Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2). Writes
 * dL_dimage (planar, like image) and adds L to *loss (device double; the caller zeroes it).
 * lambda == 0 skips SSIM. */
int dass_loss(const float* image, const float* target, const dass_camera* cams /* host */,
              int n_cams, float lambda, float* dL_dimage, double* loss, void* workspace,
              size_t workspace_bytes, void* stream);

/* Window statistics of a target for the SSIM term of Eq. 3, computed once per fixed target set:
 * for every pixel-channel i (planar like the image, P = sum of W*H over cams, 3P of them)
 * stats[2i] = (w * y)_i (the window mean) and stats[2i + 1] = (w * y^2)_i (its second moment),
 * w the 11x11 window of dass_loss with zero padding. stats: device, 6P floats, 8-byte aligned,
 * caller-owned. */
int dass_loss_target_stats(const float* target, const dass_camera* cams /* host */, int n_cams,
                           float* stats, void* stream);

/* dass_loss with the target's window statistics taken from dass_loss_target_stats (same cams,
 * same target) instead of filtered again: same loss and gradient up to FP32 rounding order.
 * The workspace is dass_loss_workspace's. */
int dass_loss_cached(const float* image, const float* target, const float* target_stats,
                     const dass_camera* cams /* host */, int n_cams, float lambda,
                     float* dL_dimage, double* loss, void* workspace, size_t workspace_bytes,
                     void* stream);

/* Per-iteration statistics of error-guided densification (Sec. 3.4): for every Gaussian g
 * and camera c with a visible record (radius > 0 and the square of half-side radius around
 * mean2d overlapping the image), accum[g] += |(dL/du W/2, dL/dv H/2)| (the view-space
 * positional gradient in NDC units) and count[g] += 1. */
int dass_densify_stats(int64_t n, const dass_splat* splats, const dass_splat_grad* splat_grads,
                       const dass_camera* cams /* host */, int n_cams, float* accum,
                       int32_t* count, void* stream);

/* Selective inheritance copy (Sec. 3.2, Eq. 1, App. B.2): output = every base row
 * (is_var == 0) in order, then every var row with Quant(sigmoid(m)) = 1, i.e. m > 0, in order;
 * erase != 0 (every 20th timestep) drops all var rows. Writes the compacted parameters,
 * is_var_out, remap[n] (old -> new row, -1 if dropped) and *n_out (device). The output
 * arrays must not alias the inputs. */
int dass_inherit_workspace(int64_t n, size_t* bytes);
int dass_inherit(int64_t n, int sh_degree, const float* means, const float* log_scales,
                 const float* quats, const float* opacity_logit, const float* sh,
                 const uint8_t* is_var, const float* m, int erase, float* out_means,
                 float* out_log_scales, float* out_quats, float* out_opacity_logit, float* out_sh,
                 uint8_t* is_var_out, int32_t* remap, int64_t* n_out, void* workspace,
                 size_t workspace_bytes, void* stream);

/* Error pass of Sec. 3.4: per camera E^c = mean_RGB |image - target| (float32, order
 * ((|dr|+|dg|)+|db|)/3), gamma^c = the element floor(q (P-1)) of the ascending sort of E^c
 * (radix select), D^c = [E^c > gamma^c]; each base Gaussian (is_var == 0 or is_var == NULL)
 * is projected with Alg. 1 (x_n = floor(0.5((x_norm+1)W - 1) + 0.5), y likewise with H) and
 * s_err[g] = 1 if D^c(y_n, x_n) = 1 for some camera (p_hom <= 0 or outside: no hit).
 * error_map (optional, [pixels]) receives E; gamma (device, [n_cams]) the thresholds. */
int dass_error_pass_workspace(const dass_camera* cams, int n_cams, size_t* bytes);
int dass_error_pass(const float* image, const float* target, const dass_camera* cams /* host */,
                    int n_cams, float quantile, int64_t n, const float* means, const uint8_t* is_var,
                    float* error_map, float* gamma, uint8_t* s_err, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Eq. 4 selection: g_n = accum/count (float32 division; 0 if count = 0);
 * S = {base n : g_n > tau_pos} U (S_err n {base n : g_n > tau_err}); of S the at most k_max
 * members with the largest g_n (ties: smaller index) are written to selected[] in ascending
 * index order and their number to *n_selected (device). */
int dass_densify_select_workspace(int64_t n, size_t* bytes);
int dass_densify_select(int64_t n, const float* accum, const int32_t* count, const uint8_t* s_err,
                        const uint8_t* is_var, float tau_pos, float tau_err, int32_t k_max,
                        int32_t* selected, int32_t* n_selected, void* workspace,
                        size_t workspace_bytes, void* stream);

/* Spawn densification (Sec. 3.4; the mechanism is not described, reading): for i <
 * *n_selected with source s = selected[i], row n + i of every parameter array becomes a new
 * var Gaussian: mean = mu_s + R_s diag(s_s) z_s, log-scale = log(s_s / 1.6), rotation,
 * opacity logit and SH copied; is_var[n + i] = 1. z[n][3] holds the caller's N(0,1) draws
 * indexed by source. Arrays must have room for n + k_max rows. *n_total (device) = n + count. */
int dass_spawn(int64_t n, int sh_degree, float* means, float* log_scales, float* quats,
               float* opacity_logit, float* sh, uint8_t* is_var, const int32_t* selected,
               const int32_t* n_selected, int32_t k_max, const float* z, int64_t* n_total,
               void* stream);

/* ------------------------------------------------------------------ per-timestep driver */

/* All buffers of one shift-stage optimisation (Sec. 3.3 with the fidelity loss of Eq. 3).
 * Every pointer is a device pointer owned by the caller unless noted. */
typedef struct dass_step_desc {
    /* scene: n Gaussians (read-only during the stage) */
    int64_t n;
    int32_t sh_degree;
    int32_t n_cams;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logit;
    const float* sh;
    const dass_camera* cams;          /* host [n_cams] */
    const float* targets;             /* ground-truth images, planar like image */
    /* dynamic group and its learned offsets */
    int64_t n_dyn;
    const int32_t* dyn_idx;           /* [n_dyn] */
    const uint8_t* dyn_mask;          /* [n] 1 for dynamic Gaussians (optional: NULL = full splat
                                         gradients for every Gaussian in the backward) */
    float* offsets;                   /* [n_dyn][7] (dmu, sigma), updated in place */
    float* offset_grad;               /* [n_dyn][7] */
    float* adam_m;                    /* [n_dyn][7] */
    float* adam_v;                    /* [n_dyn][7] */
    int32_t* adam_step;               /* device int, incremented once per iteration */
    float lr_mu, lr_sigma, beta1, beta2, eps, lambda_dssim;
    /* rendering buffers */
    int32_t tile, batch;
    float* render_means;              /* [n][3]: means with the dynamic rows shifted */
    float* render_quats;              /* [n][4] */
    float* d_means_dyn;               /* [n_dyn][3] scratch */
    float* d_quats_dyn;               /* [n_dyn][4] scratch */
    dass_splat* splats;               /* [n_cams * n] */
    dass_splat_grad* splat_grads;     /* [n_cams * n] */
    uint32_t* pair_rec;               /* [pair_capacity] */
    int64_t pair_capacity;
    uint32_t* tile_ranges;            /* [2 * tiles_total] */
    int64_t* counters;                /* [4] */
    float* image;                     /* [pixels * 3] */
    float* T_final;                   /* [pixels] */
    int32_t* n_last;                  /* [pixels] */
    float* dL_dimage;                 /* [pixels * 3] */
    double* loss;                     /* [1], loss of the last iteration */
    float* stat_accum;                /* [n] or NULL: densification statistics */
    int32_t* stat_count;              /* [n] or NULL */
    void* workspace;                  /* >= dass_step_workspace() bytes */
    size_t workspace_bytes;
} dass_step_desc;

#define DASS_STEP_BATCHED 0   /* all cameras per launch, CUDA-graph replay of one iteration */
#define DASS_STEP_PLAIN 1     /* one launch per camera per kernel, no graph */

int dass_step_workspace(const dass_step_desc* d, size_t* bytes);

/* Runs n_iters optimisation iterations of the shift stage: shift -> preprocess -> bin/sort
 * -> forward -> loss -> backward -> preprocess backward (dynamic rows) -> shift backward ->
 * [statistics] -> masked Adam on the offsets. mode DASS_STEP_BATCHED captures one iteration
 * into a CUDA graph on `stream` (which must not be the legacy default stream) and replays it
 * n_iters times; DASS_STEP_PLAIN launches per camera without a graph. With lambda_dssim > 0 the
 * call first computes the targets' SSIM window statistics into the workspace once
 * (dass_loss_target_stats) and every iteration's loss reads them (dass_loss_cached).
 * In DASS_STEP_BATCHED mode with n_dyn <= n / 2 the binning is incremental: only the dynamic rows
 * move during the stage, so the other rows' pairs are binned and sorted once when the call starts
 * (dass_bin_sort_split) and every iteration bins the dynamic rows' records and merges them in
 * (dass_bin_sort_merge), with the same pair lists as a full dass_bin_sort; the workspace then also
 * holds the static lists (2 * pair_capacity words and more: dass_step_workspace sizes it).
 * The inheritance and densification stage drivers and dass_timestep do the same with their var
 * rows as the moving set. render_means/quats
 * must hold a copy of means/quats before the first call. The call ends with one stream
 * synchronisation and a read of the pair-overflow flag: it returns DASS_ERR_CAPACITY if any
 * iteration overflowed pair_capacity (results of the stage are then unreliable). */
int dass_step(const dass_step_desc* d, int n_iters, int mode, void* stream);

/* All buffers of one selective-inheritance stage (Sec. 3.2, Eq. 1-2, App. B.2): learns one logit m
 * per var Gaussian of G_{t-1} against the views of timestep t, every other parameter fixed. One
 * iteration: keep = Quant(sigmoid(m)) on var rows (1 on base rows) -> projection with opacity and
 * scale multiplied by keep (Eq. 1) -> bin/sort -> forward -> fidelity loss of Eq. 3 -> backward
 * (full splat gradients for var rows only) -> dL/dkeep -> straight-through gradient of the loss of
 * Eq. 2 (fidelity + lambda_inher sum sigmoid(m) over var rows) -> Adam on m (var rows).
 * Device pointers owned by the caller unless noted. */
typedef struct dass_inherit_step_desc {
    int64_t n;
    int32_t sh_degree;
    int32_t n_cams;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logit;
    const float* sh;
    const uint8_t* is_var;            /* [n] 1 on var rows */
    const dass_camera* cams;          /* host [n_cams] */
    const float* targets;             /* images of timestep t, planar like image */
    int64_t n_var;
    const int32_t* var_rows;          /* [n_var] the var rows, ascending */
    float* m;                         /* [n] logits, updated in place on the var rows */
    uint8_t* keep;                    /* [n] scratch (the rendering mask) */
    float* m_grad;                    /* [n] scratch */
    float* adam_m;                    /* [n] */
    float* adam_v;                    /* [n] */
    int32_t* adam_step;               /* device int, incremented once per iteration */
    float* d_keep;                    /* [n_var] dL/dkeep of the last iteration */
    float lr, beta1, beta2, eps, lambda_dssim, lambda_inher;
    int32_t tile, batch;
    dass_splat* splats;               /* [n_cams * n] */
    dass_splat_grad* splat_grads;     /* [n_cams * n] */
    uint32_t* pair_rec;               /* [pair_capacity] */
    int64_t pair_capacity;            /* < 2^31 */
    uint32_t* tile_ranges;            /* [2 * tiles_total] */
    int64_t* counters;                /* [4] */
    float* image;                     /* [pixels * 3] */
    float* T_final;                   /* [pixels] */
    int32_t* n_last;                  /* [pixels] */
    float* dL_dimage;                 /* [pixels * 3] */
    double* loss;                     /* [1] loss of Eq. 2 at the last iteration */
    void* workspace;                  /* >= dass_inherit_step_workspace() bytes */
    size_t workspace_bytes;
} dass_inherit_step_desc;

int dass_inherit_step_workspace(const dass_inherit_step_desc* d, size_t* bytes);

/* Runs n_iters iterations of the selective-inheritance stage, one iteration captured as a CUDA graph
 * on `stream` (not the legacy default stream) and replayed; the targets' SSIM window statistics are
 * computed once into the workspace first. Ends with one stream synchronisation; returns
 * DASS_ERR_CAPACITY if any iteration overflowed pair_capacity (the learned m is then unreliable;
 * counters[0] holds the last iteration's pair count). n_var == 0 renders and leaves m unchanged. */
int dass_inherit_step(const dass_inherit_step_desc* d, int n_iters, void* stream);

/* All buffers of the densification-stage training (Sec. 3.4: the new and inherited var Gaussians
 * are optimised with the fidelity loss of Eq. 3, base Gaussians fixed). The var rows must be the
 * contiguous tail [n_base, n) of the arrays (the layout dass_inherit and dass_spawn produce). One
 * iteration: projection -> bin/sort -> forward -> loss -> backward (full splat gradients for var rows
 * only) -> parameter gradients of the var rows -> Adam on each parameter slice of the tail with the
 * learning rates below (the SH degree-0 band and the higher bands separately). */
typedef struct dass_densify_step_desc {
    int64_t n;
    int32_t sh_degree;
    int32_t n_cams;
    float* means;                     /* rows [n_base, n) of every parameter are updated in place */
    float* log_scales;
    float* quats;
    float* opacity_logit;
    float* sh;
    int64_t n_base;
    const uint8_t* is_var;            /* [n] 1 exactly on [n_base, n) */
    const dass_camera* cams;          /* host [n_cams] */
    const float* targets;
    /* gradients and Adam moments of the var rows, each (11 + 3K)(n - n_base) floats, parameter-major:
     * means [n_var][3], log_scales [n_var][3], quats [n_var][4], opacity_logit [n_var], sh [n_var][K][3] */
    float* grad;
    float* adam_m;
    float* adam_v;
    int32_t* adam_step;
    float lr_means, lr_log_scales, lr_quats, lr_opacity, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps, lambda_dssim;
    int32_t tile, batch;
    dass_splat* splats;
    dass_splat_grad* splat_grads;
    uint32_t* pair_rec;
    int64_t pair_capacity;
    uint32_t* tile_ranges;
    int64_t* counters;
    float* image;
    float* T_final;
    int32_t* n_last;
    float* dL_dimage;
    double* loss;                     /* [1] loss of the last iteration */
    void* workspace;                  /* >= dass_densify_step_workspace() bytes */
    size_t workspace_bytes;
} dass_densify_step_desc;

int dass_densify_step_workspace(const dass_densify_step_desc* d, size_t* bytes);

/* Runs n_iters densification-stage iterations (graph capture and replay, one synchronisation at the
 * end, DASS_ERR_CAPACITY on a pair overflow, as dass_inherit_step). */
int dass_densify_step(const dass_densify_step_desc* d, int n_iters, void* stream);

/* One whole timestep of the streaming reconstruction (Sec. 3.1: from G_{t-1} and the C views of
 * timestep t derive G_t):
 *   1. selective inheritance (Sec. 3.2): unless t is a multiple of erase_every (every var row is then
 *      erased, App. B.2) or n_inherit == 0 or G_{t-1} has no var rows, n_inherit iterations of the
 *      inheritance stage learn m (initialised to inherit_m0); the copy keeps every base row and the
 *      var rows with m > 0 (all var rows when the stage did not run);
 *   2. dynamics-aware shift (Sec. 3.3): n_shift iterations of the shift stage of dass_step (offsets
 *      of the dynamic rows dyn_idx start at offsets_init), then the learned offsets are applied to the
 *      dynamic rows;
 *   3. error-guided densification (Sec. 3.4, Eq. 4, Alg. 1): error pass on the last shift render
 *      (quantile), Eq. 4 selection (tau_pos, tau_err, at most k_max) and spawn (z);
 *   4. densification stage (Sec. 3.4): if n_densify > 0 and var rows exist, n_densify iterations over
 *      the var rows, then var rows of opacity <= prune_opacity are pruned.
 * Every stage captures one iteration as a CUDA graph and replays it. G_{t-1} is read from the scene
 * arrays and G_t written back into them (rows [0, *n)); base rows come first and keep their
 * indices, so dyn_idx indexes base rows. */
typedef struct dass_timestep_desc {
    /* scene arrays: G_{t-1} on entry, G_t on return; room for n_max rows (>= *n + k_max) */
    int64_t n_max;
    int32_t sh_degree;
    int32_t n_cams;
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logit;
    float* sh;
    uint8_t* is_var;                  /* [n_max] */
    int64_t* n;                       /* HOST: rows of G_{t-1} on entry, of G_t on return */
    const dass_camera* cams;          /* host [n_cams] */
    float* targets;                   /* device images of timestep t, planar like the render */
    const float* targets_host;        /* optional host images: copied into targets at the start */
    int32_t t;                        /* timestep index */
    int32_t erase_every;              /* 20 in the paper; 0 = never erase */
    int64_t n_dyn;
    const int32_t* dyn_idx;           /* [n_dyn] dynamic base rows */
    const float* offsets_init;        /* [n_dyn][7] initial (dmu, sigma) */
    float* offsets;                   /* [n_dyn][7] the learned offsets on return */
    const float* z;                   /* [n_max][3] N(0,1) draws of the spawn, indexed by source row */
    int32_t n_inherit, n_shift, n_densify, k_max;    /* s1, s2, s3 and the spawn limit */
    int32_t tile, batch;
    float lambda_dssim, lambda_inher, inherit_m0, quantile, tau_pos, tau_err, prune_opacity;
    float lr_inherit, lr_mu, lr_sigma;
    float lr_means, lr_log_scales, lr_quats, lr_opacity, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps;
    int64_t pair_capacity;            /* pair buffer of every stage's render, < 2^31 */
    void* workspace;                  /* >= dass_timestep_workspace() bytes */
    size_t workspace_bytes;
    /* optional HOST copies of G_t (rows [0, *n), capacity n_max) written before the call returns */
    float* host_means;
    float* host_log_scales;
    float* host_quats;
    float* host_opacity_logit;
    float* host_sh;
    uint8_t* host_is_var;
    /* optional upload of the NEXT timestep's images, overlapped with this timestep's stages (a
     * streaming caller's input pipeline). With both set, next_targets_host (host, pinned for an
     * asynchronous copy) is copied into next_targets (device, 3 * pixels floats like targets, not
     * overlapping targets) on a stream of the call's own, ordered after the work already queued on
     * `stream`. The call returns only once that copy has completed, on success and on error. The
     * caller passes next_targets as the next call's targets, with targets_host NULL. Both NULL:
     * no prefetch; only one of them set, or next_targets overlapping targets: DASS_ERR_INVALID_ARG. */
    const float* next_targets_host;
    float* next_targets;
} dass_timestep_desc;

/* What one timestep did (host struct filled by dass_timestep). */
typedef struct dass_timestep_stats {
    int64_t n_in;                     /* rows of G_{t-1} */
    int64_t n_var_in;                 /* its var rows */
    int64_t n_inherited;              /* rows after the inheritance copy */
    int64_t n_spawned;                /* rows added by the spawn */
    int64_t n_var_trained;            /* var rows of the densification stage */
    int64_t n_out;                    /* rows of G_t */
    int64_t pairs_max;                /* largest pair count of any iteration (size pair_capacity from it) */
    int32_t erased;                   /* 1 if this timestep erased every var row */
    int32_t inherit_ran;              /* 1 if the inheritance stage ran */
    double loss_inherit;              /* last iteration of each stage (0 if it did not run) */
    double loss_shift;
    double loss_densify;
} dass_timestep_stats;

int dass_timestep_workspace(const dass_timestep_desc* d, size_t* bytes);

/* Runs the timestep on `stream` (not the legacy default stream). Host synchronisations: after the
 * inheritance stage, the copy, the shift stage, the spawn and the densification stage (row counts
 * and overflow flags are read back). The scene arrays and *n are written only at the end: on any
 * error, including DASS_ERR_CAPACITY (a pair overflow in some stage; stats->pairs_max says how many
 * pairs were needed), G_{t-1} is left as it was and the call can be repeated with a larger
 * pair_capacity and workspace. DASS_ERR_INVALID_ARG if *n + k_max > n_max. */
int dass_timestep(const dass_timestep_desc* d, dass_timestep_stats* stats /* host */, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DASS_H */
