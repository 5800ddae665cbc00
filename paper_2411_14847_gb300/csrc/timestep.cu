// Stage drivers of the per-timestep optimisation and the whole-timestep driver (Sec. 3.1-3.4):
//   dass_step          dynamics-aware shift stage (Sec. 3.3): learned offsets of the dynamic rows;
//   dass_inherit_step  selective-inheritance stage (Sec. 3.2, Eq. 1-2): learned mask logits of the
//                      var rows;
//   dass_densify_step  densification-stage training (Sec. 3.4): every parameter of the var rows;
//   dass_timestep      G_{t-1} -> G_t: inheritance stage, copy, shift stage, error pass, Eq. 4
//                      selection, spawn, densification stage, pruning.
// Every stage captures one iteration (all cameras per launch) as a CUDA graph and replays it, so an
// iteration costs a fixed set of kernel launches and no host round trip; the drivers synchronise
// the host only between stages, to read row counts and pair-overflow flags.
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace dass {
namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Sequential carving of a caller workspace; a null base only measures.
struct Arena {
    char* base;
    size_t used = 0;
    template <class T>
    T* take(long long count) {
        const size_t bytes = al256((size_t)(count > 0 ? count : 1) * sizeof(T));
        T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
        used += bytes;
        return p;
    }
};

// Pair-overflow tracking over the iterations of a stage: track[0] = 1 once any iteration overflowed
// the pair buffer, track[1] = the largest pair count seen.
__global__ void track_pairs_kernel(const long long* __restrict__ counters, long long* __restrict__ track) {
    if (counters[1]) track[0] = 1;
    if (counters[0] > track[1]) track[1] = counters[0];
}

__global__ void fill_f32_kernel(float* __restrict__ p, long long n, float v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// mask[rows[i]] = 1 for the rows inside [0, n) (the others are ignored).
__global__ void mark_rows_kernel(const int* __restrict__ rows, long long n_rows, long long n,
                                 uint8_t* __restrict__ mask) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    const int r = rows[i];
    if (r >= 0 && r < n) mask[r] = 1;
}

__global__ void iota_kernel(int* __restrict__ rows, long long n, long long first) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rows[i] = (int)(first + i);
}

// Rows of the SH coefficients of nv Gaussians viewed as [nv * K][3]: the degree-0 band (row r K) and
// the higher bands (rows r K + j, j = 1..K-1), which take different learning rates.
__global__ void band_rows_kernel(long long nv, int K, int* __restrict__ dc, int* __restrict__ rest) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv * K) return;
    const long long r = i / K;
    const int j = (int)(i - r * K);
    if (j == 0) dc[r] = (int)i;
    else rest[r * (K - 1) + j - 1] = (int)i;
}

// Gaussian set a stage renders (device pointers).
struct Scene {
    long long n;
    int deg;
    const float* means;
    const float* ls;
    const float* quats;
    const float* logit;
    const float* sh;
};

// Buffers of the render part of a stage iteration.
struct RenderBufs {
    dass_splat* splats;
    dass_splat_grad* grads;
    uint32_t* pair_rec;
    long long cap;
    uint32_t* ranges;
    long long* counters;
    float* image;
    float* T;
    int* n_last;
    float* dL;
    double* loss;
    long long* track;        // [2] overflow flag, largest pair count
    void* bin_ws;
    size_t bin_ws_bytes;
    void* loss_ws;
    size_t loss_ws_bytes;
    const float* ystats;     // the targets' SSIM window statistics (lambda > 0), else null
    // incremental binning of a stage whose moving rows are few (inc_on): the static lists are built
    // once by inc_begin and every iteration merges the moving rows' pairs into them
    bool inc_on;
    long long inc_rows;      // most moving rows the scratch holds (0: no incremental scratch)
    long long moving_cap;    // records of the current stage's moving rows (host bound)
    StaticBins sb;
    uint8_t* moving;         // [n] moving-row mask built for the shift stage
    void* merge_ws;
    size_t merge_ws_bytes;
    unsigned long long* vis; // [n] cameras whose record the densification statistics count (or null)
    uint32_t* order;         // [tiles_total] the compositing launches' tile order, longest list first
};

// Scratch of the render part (sort and loss workspaces, cached target statistics, tracking) and,
// when inc_rows > 0, of the incremental binning for stages that move at most inc_rows of the n rows.
void carve_render_scratch(Arena& a, const CamTable& ct, long long n_rec, long long cap, float lam, RenderBufs& b,
                          long long n = 0, long long inc_rows = 0) {
    b.bin_ws_bytes = bin_sort_workspace_bytes(n_rec, cap);
    if (inc_rows > 0) {
        const size_t sp = bin_sort_split_workspace_bytes(n, n_rec, cap);
        b.bin_ws_bytes = sp > b.bin_ws_bytes ? sp : b.bin_ws_bytes;
    }
    b.bin_ws = a.take<char>((long long)b.bin_ws_bytes);
    b.loss_ws_bytes = loss_workspace_bytes(ct);
    b.loss_ws = a.take<char>((long long)b.loss_ws_bytes);
    float* ys = a.take<float>(lam > 0.f ? 6 * ct.pixels_total : 1);
    b.ystats = lam > 0.f ? ys : nullptr;
    b.track = a.take<long long>(2);
    b.order = a.take<uint32_t>(ct.tiles_total);
    b.inc_on = false;
    b.inc_rows = inc_rows;
    b.moving_cap = 0;
    b.sb = StaticBins{};
    b.moving = nullptr;
    b.merge_ws = nullptr;
    b.merge_ws_bytes = 0;
    b.vis = (n > 0 && ct.n <= 64) ? a.take<unsigned long long>(n) : nullptr;
    if (inc_rows > 0) {
        b.sb.rec = a.take<uint32_t>(cap);
        b.sb.depth = a.take<uint32_t>(cap);
        b.sb.start = a.take<uint32_t>((long long)ct.tiles_total + 1);
        b.sb.counters = a.take<long long>(4);
        b.sb.moving = a.take<uint32_t>(n_rec);
        b.sb.n_moving = a.take<long long>(1);
        b.sb.rows = a.take<int>(n);
        b.sb.n_rows_moving = a.take<long long>(1);
        b.moving = a.take<uint8_t>(n);
        b.merge_ws_bytes = bin_sort_merge_workspace_bytes((long long)ct.n * inc_rows, cap, ct.tiles_total);
        b.merge_ws = a.take<char>((long long)b.merge_ws_bytes);
    }
}

// Rows a stage may move and still bin incrementally: beyond half of the rows the full binning costs
// less than the static lists plus the merge.
long long inc_rows_bound(long long n) { return n / 2; }

// Start of the incremental binning of a stage: when the stage moves at most b.inc_rows rows (host
// bound n_moving, then the count the mask flags) and its records are camera-major with stride g.n,
// project every row once and build the static lists of the rows not flagged in moving; else the
// stage bins fully at every iteration. Ends with one stream synchronisation.
int inc_begin(const Scene& g, const CamTable& ct, const uint8_t* moving, long long n_moving, RenderBufs& b,
              cudaStream_t st) {
    b.inc_on = false;
    if (b.inc_rows <= 0 || n_moving > b.inc_rows || ct.rec_stride != g.n || !moving) return DASS_OK;
    int rc = preprocess_launch(g.n, g.deg, g.means, g.ls, g.quats, g.logit, g.sh, nullptr, ct, b.splats, st, nullptr,
                               nullptr, 0, b.vis);
    if (rc) return rc;
    rc = bin_sort_split_launch(b.splats, g.n, ct, moving, b.cap, b.sb, b.bin_ws, b.bin_ws_bytes, st);
    if (rc) return rc;
    track_pairs_kernel<<<1, 1, 0, st>>>(b.sb.counters, b.track);   // a static overflow fails the stage
    count_launch();
    if ((rc = check_launch("inc_begin"))) return rc;
    // the iterations are sized by the moving rows the mask actually flags (one read per stage)
    long long m = 0;
    DASS_CHECK_CUDA(cudaMemcpyAsync(&m, b.sb.n_rows_moving, sizeof(long long), cudaMemcpyDeviceToHost, st));
    DASS_CHECK_CUDA(cudaStreamSynchronize(st));
    if (m > b.inc_rows) return DASS_OK;      // more than the scratch holds: full binning
    b.moving_cap = (long long)ct.n * (m > 0 ? m : 1);
    b.inc_on = true;
    return DASS_OK;
}

// preprocess -> bin/sort -> forward -> fidelity loss (Eq. 3) -> backward: the part every stage
// iteration shares. keep: Eq. 1 mask or null; full_grad: Gaussians whose complete splat gradient is
// wanted (null: all).
int render_iteration(const Scene& g, const uint8_t* keep, const CamTable& ct, const float* targets, float lam,
                     const uint8_t* full_grad, int batch, RenderBufs& b, cudaStream_t st, bool mean_grads = true) {
    const long long n_rec = (long long)ct.n * g.n;
    const float3 bg = make_float3(0.f, 0.f, 0.f);
    // incremental binning: the static rows' records are those inc_begin wrote; only the moving rows
    // are projected again
    int rc = b.inc_on ? preprocess_launch(g.n, g.deg, g.means, g.ls, g.quats, g.logit, g.sh, keep, ct, b.splats, st,
                                          b.sb.rows, b.sb.n_rows_moving, b.moving_cap / ct.n, b.vis)
                      : preprocess_launch(g.n, g.deg, g.means, g.ls, g.quats, g.logit, g.sh, keep, ct, b.splats, st,
                                          nullptr, nullptr, 0, b.vis);
    if (rc) return rc;
    if (b.inc_on)
        rc = bin_sort_merge_launch(b.splats, ct, b.sb, b.moving_cap, b.cap, b.pair_rec, b.ranges, b.counters,
                                   b.merge_ws, b.merge_ws_bytes, st);
    else
        rc = bin_sort_launch(b.splats, n_rec, ct, b.pair_rec, b.cap, b.ranges, b.counters, b.bin_ws, b.bin_ws_bytes,
                             st);
    if (rc) return rc;
    track_pairs_kernel<<<1, 1, 0, st>>>(b.counters, b.track);
    count_launch();
    if ((rc = tile_order_launch(b.ranges, ct.tiles_total, b.order, st))) return rc;
    rc = render_fwd_launch(b.splats, b.pair_rec, b.ranges, ct, batch, bg, b.image, b.T, b.n_last, st, nullptr,
                           nullptr, 1, b.order);
    if (rc) return rc;
    DASS_CHECK_CUDA(cudaMemsetAsync(b.loss, 0, sizeof(double), st));
    rc = loss_launch(b.image, targets, ct, lam, 1.f / (float)ct.n, b.dL, b.loss, b.loss_ws, b.loss_ws_bytes, st,
                     b.ystats);
    if (rc) return rc;
    DASS_CHECK_CUDA(cudaMemsetAsync(b.grads, 0, sizeof(dass_splat_grad) * (size_t)n_rec, st));
    return render_bwd_launch(b.splats, b.pair_rec, b.ranges, ct, batch, bg, b.T, b.n_last, b.dL, full_grad, g.n,
                             b.grads, st, mean_grads, b.order);
}

// Start of a stage: tracking cleared, the targets' window statistics computed once (the targets are
// fixed for the whole stage), kernel attributes set outside capture.
int stage_begin(const CamTable& ct, const float* targets, int batch, RenderBufs& b, cudaStream_t st) {
    DASS_CHECK_CUDA(cudaMemsetAsync(b.track, 0, 2 * sizeof(long long), st));
    if (b.ystats)
        if (int rc = target_stats_launch(targets, ct, const_cast<float*>(b.ystats), st)) return rc;
    return render_prepare(ct.tile, batch);
}

// Capture one iteration as a CUDA graph on st and replay it n_iters times (no host synchronisation;
// the executable graph is released once its launches complete).
template <class F>
int replay(cudaStream_t st, int n_iters, F&& iteration) {
    if (n_iters <= 0) return DASS_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    DASS_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const long long l0 = launches_so_far();
    const int rc = iteration();
    const long long per_iter = launches_so_far() - l0;
    set_launches(l0 + per_iter * (long long)n_iters);   // every replay runs the captured kernels
    cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess) { set_last_error("cudaStreamEndCapture", ec); return DASS_ERR_CUDA; }
    ec = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) { set_last_error("cudaGraphInstantiate", ec); return DASS_ERR_CUDA; }
    for (int i = 0; i < n_iters; ++i) {
        ec = cudaGraphLaunch(exec, st);
        if (ec != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            set_last_error("cudaGraphLaunch", ec);
            return DASS_ERR_CUDA;
        }
    }
    cudaGraphExecDestroy(exec);
    return DASS_OK;
}

// End of a stage: wait for it and read the tracking; DASS_ERR_CAPACITY if any iteration overflowed.
int stage_end(const RenderBufs& b, cudaStream_t st, int64_t* pairs_max = nullptr) {
    long long tr[2] = {0, 0};
    DASS_CHECK_CUDA(cudaMemcpyAsync(tr, b.track, sizeof(tr), cudaMemcpyDeviceToHost, st));
    DASS_CHECK_CUDA(cudaStreamSynchronize(st));
    if (pairs_max && tr[1] > *pairs_max) *pairs_max = tr[1];
    return tr[0] ? DASS_ERR_CAPACITY : DASS_OK;
}

// ----------------------------------------------------------------- shift stage (Sec. 3.3)

struct ShiftState {
    long long n_dyn;
    const int* dyn_idx;
    const uint8_t* dyn_mask;     // [n] 1 on dynamic rows (null: full splat gradients for all)
    float* offsets;              // [n_dyn][7] (dmu, sigma)
    float* offset_grad;
    float* am;
    float* av;
    int* step;
    float lr[7];
    float b1, b2, eps;
    float* render_means;         // [n][3]: means with the dynamic rows shifted
    float* render_quats;         // [n][4]
    float* d_means_dyn;          // [n_dyn][3]
    float* d_quats_dyn;          // [n_dyn][4]
    float* stat_accum;           // [n] densification statistics or null
    int* stat_count;
};

// One batched shift-stage iteration: shift -> render (static rows: dL/dmean2D only) -> preprocess
// backward of the dynamic rows -> [statistics] -> shift backward -> masked Adam on the offsets.
int shift_iteration(const Scene& g, const CamTable& ct, const float* targets, float lam, int batch,
                    const ShiftState& s, RenderBufs& b, cudaStream_t st) {
    int rc = shift_launch(s.n_dyn, s.dyn_idx, s.offsets, g.means, g.quats, s.render_means, s.render_quats, st);
    if (rc) return rc;
    const Scene gr{g.n, g.deg, s.render_means, g.ls, s.render_quats, g.logit, g.sh};
    rc = render_iteration(gr, nullptr, ct, targets, lam, s.dyn_mask, batch, b, st);
    if (rc) return rc;
    rc = preprocess_bwd_launch(g.n, g.deg, s.render_means, g.ls, s.render_quats, g.logit, g.sh, nullptr, ct, b.splats,
                               b.grads, s.dyn_idx, s.n_dyn, DASS_GRAD_MEANS | DASS_GRAD_QUATS, 0, s.d_means_dyn,
                               nullptr, s.d_quats_dyn, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    if (s.stat_accum && s.stat_count) {
        rc = b.vis ? densify_stats_vis_launch(g.n, ct, b.vis, b.grads, s.stat_accum, s.stat_count, st)
                   : densify_stats_launch(g.n, ct, b.splats, b.grads, s.stat_accum, s.stat_count, st);
        if (rc) return rc;
    }
    rc = shift_bwd_launch(s.n_dyn, s.dyn_idx, s.offsets, g.quats, s.d_means_dyn, s.d_quats_dyn, s.offset_grad,
                          nullptr, st);
    if (rc) return rc;
    return adam_launch(s.n_dyn, 7, nullptr, s.offsets, s.offset_grad, s.am, s.av, s.step, s.lr, s.b1, s.b2, s.eps, 1,
                       st);
}

// The same iteration with one launch per camera and kernel (the plain form the batched one is
// measured against).
int shift_iteration_plain(const Scene& g, const CamTable& all, const std::vector<CamTable>& per,
                          const float* targets, float lam, int batch, const ShiftState& s, RenderBufs& b,
                          cudaStream_t st) {
    int rc = shift_launch(s.n_dyn, s.dyn_idx, s.offsets, g.means, g.quats, s.render_means, s.render_quats, st);
    if (rc) return rc;
    DASS_CHECK_CUDA(cudaMemsetAsync(b.loss, 0, sizeof(double), st));
    const float3 bg = make_float3(0.f, 0.f, 0.f);
    const float inv_cams = 1.f / (float)all.n;
    for (int c = 0; c < all.n; ++c) {
        const CamTable& ct = per[c];
        const long long pb = all.c[c].pix_base;
        dass_splat* sp = b.splats + (long long)c * g.n;
        dass_splat_grad* gs = b.grads + (long long)c * g.n;
        rc = preprocess_launch(g.n, g.deg, s.render_means, g.ls, s.render_quats, g.logit, g.sh, nullptr, ct, sp, st);
        if (rc) return rc;
        rc = bin_sort_launch(sp, g.n, ct, b.pair_rec, b.cap, b.ranges, b.counters, b.bin_ws, b.bin_ws_bytes, st);
        if (rc) return rc;
        track_pairs_kernel<<<1, 1, 0, st>>>(b.counters, b.track);
        count_launch();
        rc = render_fwd_launch(sp, b.pair_rec, b.ranges, ct, batch, bg, b.image + 3 * pb, b.T + pb, b.n_last + pb, st);
        if (rc) return rc;
        rc = loss_launch(b.image + 3 * pb, targets + 3 * pb, ct, lam, inv_cams, b.dL + 3 * pb, b.loss, b.loss_ws,
                         b.loss_ws_bytes, st, b.ystats ? b.ystats + 2 * 3 * pb : nullptr);
        if (rc) return rc;
        DASS_CHECK_CUDA(cudaMemsetAsync(gs, 0, sizeof(dass_splat_grad) * (size_t)g.n, st));
        rc = render_bwd_launch(sp, b.pair_rec, b.ranges, ct, batch, bg, b.T + pb, b.n_last + pb, b.dL + 3 * pb,
                               s.dyn_mask, g.n, gs, st);
        if (rc) return rc;
        rc = preprocess_bwd_launch(g.n, g.deg, s.render_means, g.ls, s.render_quats, g.logit, g.sh, nullptr, ct, sp,
                                   gs, s.dyn_idx, s.n_dyn, DASS_GRAD_MEANS | DASS_GRAD_QUATS, c > 0, s.d_means_dyn,
                                   nullptr, s.d_quats_dyn, nullptr, nullptr, nullptr, st);
        if (rc) return rc;
        if (s.stat_accum && s.stat_count) {
            rc = densify_stats_launch(g.n, ct, sp, gs, s.stat_accum, s.stat_count, st);
            if (rc) return rc;
        }
    }
    rc = shift_bwd_launch(s.n_dyn, s.dyn_idx, s.offsets, g.quats, s.d_means_dyn, s.d_quats_dyn, s.offset_grad,
                          nullptr, st);
    if (rc) return rc;
    return adam_launch(s.n_dyn, 7, nullptr, s.offsets, s.offset_grad, s.am, s.av, s.step, s.lr, s.b1, s.b2, s.eps, 1,
                       st);
}

// ----------------------------------------------------------------- inheritance stage (Sec. 3.2)

struct InheritState {
    const uint8_t* is_var;
    long long n_var;
    const int* var_rows;
    float* m;
    uint8_t* keep;
    float* m_grad;
    float* am;
    float* av;
    int* step;
    float* d_keep;
    float lr, b1, b2, eps, lam_inher;
};

// keep = Quant(sigmoid(m)) -> render with Eq. 1 (var rows get full splat gradients) -> dL/dkeep ->
// STE gradient of Eq. 2 (mask loss added to the loss) -> Adam on m over the var rows.
int inherit_iteration(const Scene& g, const CamTable& ct, const float* targets, float lam, int batch,
                      const InheritState& s, RenderBufs& b, cudaStream_t st) {
    int rc = inherit_keep_launch(g.n, s.is_var, s.m, s.keep, st);
    if (rc) return rc;
    // only the var rows' gradients are used: the base rows need no dL/dmean2D here
    rc = render_iteration(g, s.keep, ct, targets, lam, s.is_var, batch, b, st, false);
    if (rc || s.n_var == 0) return rc;
    rc = preprocess_bwd_launch(g.n, g.deg, g.means, g.ls, g.quats, g.logit, g.sh, s.keep, ct, b.splats, b.grads,
                               s.var_rows, s.n_var, 0u, 0, nullptr, nullptr, nullptr, nullptr, nullptr, s.d_keep, st);
    if (rc) return rc;
    rc = inherit_mask_grad_launch(s.n_var, s.var_rows, s.m, s.d_keep, s.lam_inher, s.m_grad, b.loss, st);
    if (rc) return rc;
    return adam_launch(s.n_var, 1, s.var_rows, s.m, s.m_grad, s.am, s.av, s.step, &s.lr, s.b1, s.b2, s.eps, 1, st);
}

// ----------------------------------------------------------------- densification stage (Sec. 3.4)

struct DensifyState {
    float* means;                // mutable views of the scene (the var tail is trained)
    float* ls;
    float* quats;
    float* logit;
    float* sh;
    long long n_base, n_var;
    const int* var_rows;         // n_base .. n-1
    const uint8_t* is_var;
    float* grad;                 // (11 + 3K) n_var floats each, parameter-major
    float* am;
    float* av;
    int* step;
    const int* dc_rows;          // [n_var] SH rows of the degree-0 band ([n_var * K][3] view)
    const int* rest_rows;        // [n_var (K - 1)] SH rows of the higher bands
    float lr[6];                 // means, log-scales, rotations, opacity logits, SH DC, higher SH bands
    float b1, b2, eps;
};

// render (var rows: full splat gradients) -> parameter gradients of the var rows -> Adam on each
// parameter slice of the tail; the SH degree-0 band and the higher bands take their own rates.
int densify_iteration(const Scene& g, const CamTable& ct, const float* targets, float lam, int batch,
                      const DensifyState& s, RenderBufs& b, cudaStream_t st) {
    // only the var tail is trained and no statistics are gathered: the base rows need no gradient
    int rc = render_iteration(g, nullptr, ct, targets, lam, s.is_var, batch, b, st, false);
    if (rc || s.n_var == 0) return rc;
    const long long nv = s.n_var, nb = s.n_base;
    const int K = (g.deg + 1) * (g.deg + 1);
    const long long off[6] = {0, 3 * nv, 6 * nv, 10 * nv, 11 * nv, 0};
    float* G = s.grad;
    rc = preprocess_bwd_launch(g.n, g.deg, g.means, g.ls, g.quats, g.logit, g.sh, nullptr, ct, b.splats, b.grads,
                               s.var_rows, nv, DASS_GRAD_ALL, 0, G + off[0], G + off[1], G + off[2], G + off[3],
                               G + off[4], nullptr, st);
    if (rc) return rc;
    float* params[4] = {s.means + 3 * nb, s.ls + 3 * nb, s.quats + 4 * nb, s.logit + nb};
    const int widths[4] = {3, 3, 4, 1};
    for (int k = 0; k < 4; ++k) {
        float lr[4] = {s.lr[k], s.lr[k], s.lr[k], s.lr[k]};
        rc = adam_launch(nv, widths[k], nullptr, params[k], G + off[k], s.am + off[k], s.av + off[k], s.step, lr,
                         s.b1, s.b2, s.eps, 0, st);
        if (rc) return rc;
    }
    float* shv = s.sh + 3 * (long long)K * nb;              // [nv * K][3]
    const float dc[3] = {s.lr[4], s.lr[4], s.lr[4]}, hi[3] = {s.lr[5], s.lr[5], s.lr[5]};
    rc = adam_launch(nv, 3, s.dc_rows, shv, G + off[4], s.am + off[4], s.av + off[4], s.step, dc, s.b1, s.b2, s.eps,
                     K == 1, st);
    if (rc || K == 1) return rc;
    return adam_launch(nv * (K - 1), 3, s.rest_rows, shv, G + off[4], s.am + off[4], s.av + off[4], s.step, hi, s.b1,
                       s.b2, s.eps, 1, st);
}

// Band row lists of the densification stage's SH Adam steps.
int densify_prepare(long long nv, int K, int* dc_rows, int* rest_rows, cudaStream_t st) {
    if (nv <= 0) return DASS_OK;
    band_rows_kernel<<<div_up(nv * K, 256), 256, 0, st>>>(nv, K, dc_rows, rest_rows);
    count_launch();
    return check_launch("band_rows_kernel");
}

bool scene_ok(long long n, int deg, const void* a, const void* b, const void* c, const void* d, const void* e) {
    return n > 0 && n < (1ll << 31) && deg >= 0 && deg <= 3 && a && b && c && d && e;
}

bool render_ok(int n_cams, long long n, int batch, long long cap, const void* splats, const void* grads,
               const void* pair_rec, const void* ranges, const void* counters, const void* image, const void* T,
               const void* n_last, const void* dL, const void* loss, const void* targets) {
    if ((long long)n_cams * n >= (1ll << 32) || !batch_ok(batch) || cap < 1 || cap >= (1ll << 31)) return false;
    return splats && grads && pair_rec && ranges && counters && image && T && n_last && dL && loss && targets;
}

}  // namespace
}  // namespace dass

using namespace dass;

// ----------------------------------------------------------------- dass_step

namespace {

bool step_desc_ok(const dass_step_desc* d) {
    if (!d || d->n_dyn < 0 || d->n_dyn >= (1ll << 31)) return false;
    if (!scene_ok(d->n, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh)) return false;
    if (!render_ok(d->n_cams, d->n, d->batch, d->pair_capacity, d->splats, d->splat_grads, d->pair_rec,
                   d->tile_ranges, d->counters, d->image, d->T_final, d->n_last, d->dL_dimage, d->loss, d->targets))
        return false;
    if (d->n_dyn > 0 && (!d->dyn_idx || !d->offsets || !d->offset_grad || !d->adam_m || !d->adam_v ||
                         !d->d_means_dyn || !d->d_quats_dyn))
        return false;
    return d->adam_step && d->render_means && d->render_quats && d->workspace;
}

size_t step_scratch(const dass_step_desc* d, const CamTable& ct, int mode, char* base, RenderBufs* b) {
    Arena a{base};
    RenderBufs tmp{};
    RenderBufs& r = b ? *b : tmp;
    const bool inc = mode == DASS_STEP_BATCHED && d->n_dyn <= inc_rows_bound(d->n);
    carve_render_scratch(a, ct, mode == DASS_STEP_PLAIN ? d->n : (long long)d->n_cams * d->n, d->pair_capacity,
                         d->lambda_dssim, r, d->n, inc ? (d->n_dyn > 0 ? d->n_dyn : 1) : 0);
    return a.used;
}

}  // namespace

DASS_API int dass_step_workspace(const dass_step_desc* d, size_t* bytes) {
    if (!d || !bytes) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n, &ct)) return DASS_ERR_INVALID_ARG;
    *bytes = step_scratch(d, ct, DASS_STEP_BATCHED, nullptr, nullptr);
    return DASS_OK;
}

DASS_API int dass_step(const dass_step_desc* d, int n_iters, int mode, void* stream) {
    if (!step_desc_ok(d) || n_iters < 0 || (mode != DASS_STEP_BATCHED && mode != DASS_STEP_PLAIN))
        return DASS_ERR_INVALID_ARG;
    if (d->lambda_dssim < 0.f || d->lambda_dssim > 1.f) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n, &ct)) return DASS_ERR_INVALID_ARG;
    if (d->workspace_bytes < step_scratch(d, ct, mode, nullptr, nullptr)) return DASS_ERR_OOM;
    cudaStream_t st = as_stream(stream);
    if (mode == DASS_STEP_BATCHED && st == nullptr) return DASS_ERR_INVALID_ARG;   // not capturable
    RenderBufs b{d->splats, d->splat_grads, d->pair_rec, d->pair_capacity, d->tile_ranges, (long long*)d->counters,
                 d->image, d->T_final, d->n_last, d->dL_dimage, d->loss};
    step_scratch(d, ct, mode, reinterpret_cast<char*>(d->workspace), &b);
    DASS_CHECK_CUDA(cudaMemsetAsync(d->counters, 0, sizeof(int64_t) * 4, st));
    if (int rc = stage_begin(ct, d->targets, d->batch, b, st)) return rc;
    if (n_iters == 0) return DASS_OK;
    const Scene g{d->n, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh};
    ShiftState s{d->n_dyn, d->dyn_idx, d->dyn_mask, d->offsets, d->offset_grad, d->adam_m, d->adam_v, d->adam_step,
                 {d->lr_mu, d->lr_mu, d->lr_mu, d->lr_sigma, d->lr_sigma, d->lr_sigma, d->lr_sigma},
                 d->beta1, d->beta2, d->eps, d->render_means, d->render_quats, d->d_means_dyn, d->d_quats_dyn,
                 d->stat_accum, d->stat_count};
    if (mode == DASS_STEP_BATCHED) {
        if (b.inc_rows > 0) {     // the dynamic rows move; the others keep their records all stage
            DASS_CHECK_CUDA(cudaMemsetAsync(b.moving, 0, (size_t)d->n, st));
            if (d->n_dyn > 0) {
                mark_rows_kernel<<<div_up(d->n_dyn, 256), 256, 0, st>>>(d->dyn_idx, d->n_dyn, d->n, b.moving);
                count_launch();
            }
            const Scene gr{d->n, d->sh_degree, d->render_means, d->log_scales, d->render_quats, d->opacity_logit,
                           d->sh};
            if (int rc = inc_begin(gr, ct, b.moving, d->n_dyn, b, st)) return rc;
        }
        if (int rc = replay(st, n_iters, [&] { return shift_iteration(g, ct, d->targets, d->lambda_dssim, d->batch, s,
                                                                       b, st); }))
            return rc;
    } else {
        std::vector<CamTable> per(d->n_cams);
        for (int c = 0; c < d->n_cams; ++c)
            if (!make_cam_table(d->cams + c, 1, d->tile, d->n, &per[c])) return DASS_ERR_INVALID_ARG;
        for (int i = 0; i < n_iters; ++i)
            if (int rc = shift_iteration_plain(g, ct, per, d->targets, d->lambda_dssim, d->batch, s, b, st)) return rc;
    }
    return stage_end(b, st);
}

// ----------------------------------------------------------------- dass_inherit_step

namespace {

bool inherit_desc_ok(const dass_inherit_step_desc* d) {
    if (!d || !scene_ok(d->n, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh)) return false;
    if (!render_ok(d->n_cams, d->n, d->batch, d->pair_capacity, d->splats, d->splat_grads, d->pair_rec,
                   d->tile_ranges, d->counters, d->image, d->T_final, d->n_last, d->dL_dimage, d->loss, d->targets))
        return false;
    if (d->n_var < 0 || d->n_var > d->n || (d->n_var > 0 && (!d->var_rows || !d->d_keep))) return false;
    if (!(d->lambda_dssim >= 0.f && d->lambda_dssim <= 1.f)) return false;
    return d->is_var && d->m && d->keep && d->m_grad && d->adam_m && d->adam_v && d->adam_step && d->workspace;
}

size_t inherit_scratch(const dass_inherit_step_desc* d, const CamTable& ct, char* base, RenderBufs* b) {
    Arena a{base};
    RenderBufs tmp{};
    const long long inc = d->n_var <= inc_rows_bound(d->n) ? (d->n_var > 0 ? d->n_var : 1) : 0;
    carve_render_scratch(a, ct, (long long)d->n_cams * d->n, d->pair_capacity, d->lambda_dssim, b ? *b : tmp, d->n,
                         inc);
    return a.used;
}

}  // namespace

DASS_API int dass_inherit_step_workspace(const dass_inherit_step_desc* d, size_t* bytes) {
    if (!d || !bytes) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n, &ct)) return DASS_ERR_INVALID_ARG;
    *bytes = inherit_scratch(d, ct, nullptr, nullptr);
    return DASS_OK;
}

DASS_API int dass_inherit_step(const dass_inherit_step_desc* d, int n_iters, void* stream) {
    if (!inherit_desc_ok(d) || n_iters < 0) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n, &ct)) return DASS_ERR_INVALID_ARG;
    if (d->workspace_bytes < inherit_scratch(d, ct, nullptr, nullptr)) return DASS_ERR_OOM;
    cudaStream_t st = as_stream(stream);
    if (st == nullptr) return DASS_ERR_INVALID_ARG;
    RenderBufs b{d->splats, d->splat_grads, d->pair_rec, d->pair_capacity, d->tile_ranges, (long long*)d->counters,
                 d->image, d->T_final, d->n_last, d->dL_dimage, d->loss};
    inherit_scratch(d, ct, reinterpret_cast<char*>(d->workspace), &b);
    if (int rc = stage_begin(ct, d->targets, d->batch, b, st)) return rc;
    const Scene g{d->n, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh};
    const InheritState s{d->is_var, d->n_var, d->var_rows, d->m, d->keep, d->m_grad, d->adam_m, d->adam_v,
                         d->adam_step, d->d_keep, d->lr, d->beta1, d->beta2, d->eps, d->lambda_inher};
    // the var rows' masks change; the base rows (keep = 1) keep their records all stage
    if (int rc = inc_begin(g, ct, d->is_var, d->n_var, b, st)) return rc;
    if (int rc = replay(st, n_iters, [&] { return inherit_iteration(g, ct, d->targets, d->lambda_dssim, d->batch, s, b,
                                                                     st); }))
        return rc;
    return stage_end(b, st);
}

// ----------------------------------------------------------------- dass_densify_step

namespace {

bool densify_desc_ok(const dass_densify_step_desc* d) {
    if (!d || !scene_ok(d->n, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh)) return false;
    if (!render_ok(d->n_cams, d->n, d->batch, d->pair_capacity, d->splats, d->splat_grads, d->pair_rec,
                   d->tile_ranges, d->counters, d->image, d->T_final, d->n_last, d->dL_dimage, d->loss, d->targets))
        return false;
    if (d->n_base < 0 || d->n_base > d->n) return false;
    const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
    if ((d->n - d->n_base) * K >= (1ll << 31)) return false;
    if (!(d->lambda_dssim >= 0.f && d->lambda_dssim <= 1.f)) return false;
    return d->is_var && d->grad && d->adam_m && d->adam_v && d->adam_step && d->workspace;
}

struct DensifyScratch {
    int* var_rows;
    int* dc_rows;
    int* rest_rows;
};

size_t densify_scratch(const dass_densify_step_desc* d, const CamTable& ct, char* base, RenderBufs* b,
                       DensifyScratch* ds) {
    Arena a{base};
    RenderBufs tmp{};
    const long long nv = d->n - d->n_base;
    const long long inc = nv <= inc_rows_bound(d->n) ? (nv > 0 ? nv : 1) : 0;
    carve_render_scratch(a, ct, (long long)d->n_cams * d->n, d->pair_capacity, d->lambda_dssim, b ? *b : tmp, d->n,
                         inc);
    const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
    int* vr = a.take<int>(nv);
    int* dc = a.take<int>(nv);
    int* rest = a.take<int>(nv * (K - 1));
    if (ds) *ds = DensifyScratch{vr, dc, rest};
    return a.used;
}

}  // namespace

DASS_API int dass_densify_step_workspace(const dass_densify_step_desc* d, size_t* bytes) {
    if (!d || !bytes) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n, &ct)) return DASS_ERR_INVALID_ARG;
    *bytes = densify_scratch(d, ct, nullptr, nullptr, nullptr);
    return DASS_OK;
}

DASS_API int dass_densify_step(const dass_densify_step_desc* d, int n_iters, void* stream) {
    if (!densify_desc_ok(d) || n_iters < 0) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n, &ct)) return DASS_ERR_INVALID_ARG;
    if (d->workspace_bytes < densify_scratch(d, ct, nullptr, nullptr, nullptr)) return DASS_ERR_OOM;
    cudaStream_t st = as_stream(stream);
    if (st == nullptr) return DASS_ERR_INVALID_ARG;
    RenderBufs b{d->splats, d->splat_grads, d->pair_rec, d->pair_capacity, d->tile_ranges, (long long*)d->counters,
                 d->image, d->T_final, d->n_last, d->dL_dimage, d->loss};
    DensifyScratch ds;
    densify_scratch(d, ct, reinterpret_cast<char*>(d->workspace), &b, &ds);
    if (int rc = stage_begin(ct, d->targets, d->batch, b, st)) return rc;
    const long long nv = d->n - d->n_base;
    const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
    if (nv > 0) {
        iota_kernel<<<div_up(nv, 256), 256, 0, st>>>(ds.var_rows, nv, d->n_base);
        count_launch();
        if (int rc = check_launch("iota_kernel")) return rc;
        if (int rc = densify_prepare(nv, K, ds.dc_rows, ds.rest_rows, st)) return rc;
    }
    const Scene g{d->n, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh};
    const DensifyState s{d->means, d->log_scales, d->quats, d->opacity_logit, d->sh, d->n_base, nv, ds.var_rows,
                         d->is_var, d->grad, d->adam_m, d->adam_v, d->adam_step, ds.dc_rows, ds.rest_rows,
                         {d->lr_means, d->lr_log_scales, d->lr_quats, d->lr_opacity, d->lr_sh_dc, d->lr_sh_rest},
                         d->beta1, d->beta2, d->eps};
    // the var tail is trained; the base rows keep their records all stage
    if (int rc = inc_begin(g, ct, d->is_var, nv, b, st)) return rc;
    if (int rc = replay(st, n_iters, [&] { return densify_iteration(g, ct, d->targets, d->lambda_dssim, d->batch, s, b,
                                                                     st); }))
        return rc;
    return stage_end(b, st);
}

// ----------------------------------------------------------------- dass_timestep

namespace {

// Every buffer of one timestep, carved from the caller's workspace.
struct TsBufs {
    // second scene buffer: the inheritance copy writes it, the stages train it, pruning copies back
    float* means; float* ls; float* quats; float* logit; float* sh; uint8_t* is_var;
    RenderBufs r;
    // shift stage
    float* render_means; float* render_quats;
    float* stat_accum; int* stat_count; uint8_t* dyn_mask;
    float* off_grad; float* off_m; float* off_v; float* d_means_dyn; float* d_quats_dyn;
    // inheritance stage
    float* m; uint8_t* keep; float* m_grad; float* m_am; float* m_av; float* d_keep; int* var_rows;
    // densification stage
    float* dgrad; float* dm; float* dv; int* dc_rows; int* rest_rows; float* prune_m;
    // error pass, selection, spawn, copies
    uint8_t* s_err; float* gamma; int* sel; int* n_sel; int* remap;
    long long* scal;        // [4]: copy count, spawn total, compaction count, spare
    int* steps;             // [4]: Adam step counters of the three stages
    double* losses;         // [3]
    void* misc_ws; size_t misc_ws_bytes;   // error pass / selection / copy / compaction scratch (one at a time)
};

size_t carve_timestep(const dass_timestep_desc* d, const CamTable& ct, char* base, TsBufs* out) {
    Arena a{base};
    TsBufs t{};
    const long long N = d->n_max;
    const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
    const long long n_rec = (long long)d->n_cams * N;
    const long long nd = d->n_dyn > 0 ? d->n_dyn : 1;
    t.means = a.take<float>(3 * N); t.ls = a.take<float>(3 * N); t.quats = a.take<float>(4 * N);
    t.logit = a.take<float>(N); t.sh = a.take<float>(3 * K * N); t.is_var = a.take<uint8_t>(N);
    t.r.splats = a.take<dass_splat>(n_rec);
    t.r.grads = a.take<dass_splat_grad>(n_rec);
    t.r.cap = d->pair_capacity;
    t.r.pair_rec = a.take<uint32_t>(d->pair_capacity);
    t.r.ranges = a.take<uint32_t>(2 * (long long)ct.tiles_total);
    t.r.counters = a.take<long long>(4);
    t.r.image = a.take<float>(3 * ct.pixels_total);
    t.r.T = a.take<float>(ct.pixels_total);
    t.r.n_last = a.take<int>(ct.pixels_total);
    t.r.dL = a.take<float>(3 * ct.pixels_total);
    t.r.loss = a.take<double>(1);
    carve_render_scratch(a, ct, n_rec, d->pair_capacity, d->lambda_dssim, t.r, N, inc_rows_bound(N));
    t.render_means = a.take<float>(3 * N); t.render_quats = a.take<float>(4 * N);
    t.stat_accum = a.take<float>(N); t.stat_count = a.take<int>(N); t.dyn_mask = a.take<uint8_t>(N);
    t.off_grad = a.take<float>(7 * nd); t.off_m = a.take<float>(7 * nd); t.off_v = a.take<float>(7 * nd);
    t.d_means_dyn = a.take<float>(3 * nd); t.d_quats_dyn = a.take<float>(4 * nd);
    t.m = a.take<float>(N); t.keep = a.take<uint8_t>(N); t.m_grad = a.take<float>(N);
    t.m_am = a.take<float>(N); t.m_av = a.take<float>(N); t.d_keep = a.take<float>(N); t.var_rows = a.take<int>(N);
    t.dgrad = a.take<float>((11 + 3 * K) * N); t.dm = a.take<float>((11 + 3 * K) * N);
    t.dv = a.take<float>((11 + 3 * K) * N);
    t.dc_rows = a.take<int>(N); t.rest_rows = a.take<int>(N * (K - 1)); t.prune_m = a.take<float>(N);
    t.s_err = a.take<uint8_t>(N); t.gamma = a.take<float>(d->n_cams);
    t.sel = a.take<int>(d->k_max > 0 ? d->k_max : 1); t.n_sel = a.take<int>(1); t.remap = a.take<int>(N);
    t.scal = a.take<long long>(4); t.steps = a.take<int>(4); t.losses = a.take<double>(3);
    size_t misc = error_pass_workspace_bytes(ct);
    const size_t cand[3] = {select_workspace_bytes(N), inherit_workspace_bytes(N), mask_rows_workspace_bytes(N)};
    for (size_t c : cand) misc = c > misc ? c : misc;
    t.misc_ws_bytes = misc;
    t.misc_ws = a.take<char>((long long)misc);
    if (out) *out = t;
    return a.used;
}

bool timestep_desc_ok(const dass_timestep_desc* d) {
    if (!d || !d->n || d->n_max <= 0 || d->n_max >= (1ll << 31)) return false;
    if (!scene_ok(d->n_max, d->sh_degree, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh)) return false;
    if (!d->is_var || !d->targets || !d->workspace || !d->offsets || !d->z) return false;
    if ((long long)d->n_cams * d->n_max >= (1ll << 32) || !batch_ok(d->batch)) return false;
    if (d->pair_capacity < 1 || d->pair_capacity >= (1ll << 31)) return false;
    if (d->n_dyn < 0 || (d->n_dyn > 0 && (!d->dyn_idx || !d->offsets_init))) return false;
    if (d->k_max < 0 || d->n_inherit < 0 || d->n_shift < 0 || d->n_densify < 0 || d->erase_every < 0) return false;
    if (!(d->lambda_dssim >= 0.f && d->lambda_dssim <= 1.f) || !(d->quantile >= 0.f && d->quantile <= 1.f))
        return false;
    if (!(d->prune_opacity > 0.f && d->prune_opacity < 1.f) || !(d->tau_pos >= 0.f) || !(d->tau_err >= 0.f))
        return false;
    if (!d->next_targets_host != !d->next_targets) return false;
    const long long n = *d->n;
    return n > 0 && n + d->k_max <= d->n_max;
}

// Upload of the next timestep's images on a stream of its own, overlapped with the stages running on
// the timestep's stream; finish() (also run by the destructor, so every return path waits) blocks
// until the copy has landed.
class Prefetch {
  public:
    int start(float* dst, const float* src, size_t bytes, cudaStream_t after) {
        DASS_CHECK_CUDA(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
        DASS_CHECK_CUDA(cudaEventCreateWithFlags(&ev_, cudaEventDisableTiming));
        DASS_CHECK_CUDA(cudaEventRecord(ev_, after));      // after the last readers of dst queued so far
        DASS_CHECK_CUDA(cudaStreamWaitEvent(cs_, ev_, 0));
        DASS_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs_));
        return DASS_OK;
    }
    int finish() {
        cudaError_t e = cudaSuccess;
        if (cs_) {
            e = cudaStreamSynchronize(cs_);
            cudaStreamDestroy(cs_);
            cs_ = nullptr;
        }
        if (ev_) {
            cudaEventDestroy(ev_);
            ev_ = nullptr;
        }
        if (e != cudaSuccess) {
            set_last_error("cudaStreamSynchronize(prefetch)", e);
            return DASS_ERR_CUDA;
        }
        return DASS_OK;
    }
    ~Prefetch() { finish(); }

  private:
    cudaStream_t cs_ = nullptr;
    cudaEvent_t ev_ = nullptr;
};

int read_scalar(const long long* dev, long long* host, cudaStream_t st) {
    DASS_CHECK_CUDA(cudaMemcpyAsync(host, dev, sizeof(long long), cudaMemcpyDeviceToHost, st));
    DASS_CHECK_CUDA(cudaStreamSynchronize(st));
    return DASS_OK;
}

int fill(float* p, long long n, float v, cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    fill_f32_kernel<<<div_up(n, 256), 256, 0, st>>>(p, n, v);
    count_launch();
    return check_launch("fill_f32_kernel");
}

// Copy rows [0, n) of a scene from src arrays to dst arrays (same layout), on st.
int copy_scene(long long n, int K, const float* sm, const float* sl, const float* sq, const float* so, const float* ss,
               const uint8_t* sv, float* dm, float* dl, float* dq, float* dop, float* ds, uint8_t* dv,
               cudaMemcpyKind kind, cudaStream_t st) {
    DASS_CHECK_CUDA(cudaMemcpyAsync(dm, sm, sizeof(float) * 3 * n, kind, st));
    DASS_CHECK_CUDA(cudaMemcpyAsync(dl, sl, sizeof(float) * 3 * n, kind, st));
    DASS_CHECK_CUDA(cudaMemcpyAsync(dq, sq, sizeof(float) * 4 * n, kind, st));
    DASS_CHECK_CUDA(cudaMemcpyAsync(dop, so, sizeof(float) * n, kind, st));
    DASS_CHECK_CUDA(cudaMemcpyAsync(ds, ss, sizeof(float) * 3 * K * n, kind, st));
    DASS_CHECK_CUDA(cudaMemcpyAsync(dv, sv, n, kind, st));
    return DASS_OK;
}

int timestep_run(const dass_timestep_desc* d, const CamTable& ct, TsBufs& w, dass_timestep_stats& out,
                 cudaStream_t st) {
    const int deg = d->sh_degree, K = (deg + 1) * (deg + 1);
    const long long n0 = *d->n;
    const float lam = d->lambda_dssim;
    const bool erase = d->erase_every > 0 && d->t % d->erase_every == 0;
    out.n_in = n0;
    out.erased = erase ? 1 : 0;
    DASS_CHECK_CUDA(cudaMemsetAsync(w.steps, 0, 4 * sizeof(int), st));
    DASS_CHECK_CUDA(cudaMemsetAsync(w.losses, 0, 3 * sizeof(double), st));
    DASS_CHECK_CUDA(cudaMemsetAsync(w.r.counters, 0, 4 * sizeof(long long), st));
    if (d->targets_host)
        DASS_CHECK_CUDA(cudaMemcpyAsync(d->targets, d->targets_host, sizeof(float) * 3 * (size_t)ct.pixels_total,
                                        cudaMemcpyHostToDevice, st));
    if (int rc = stage_begin(ct, d->targets, d->batch, w.r, st)) return rc;   // statistics of this timestep's targets
    RenderBufs& r = w.r;
    int rc;

    // 1. selective inheritance (Sec. 3.2): the var rows of G_{t-1}, then s1 iterations learning m
    rc = mask_rows_launch(d->is_var, n0, w.var_rows, w.scal + 2, w.misc_ws, w.misc_ws_bytes, st);
    if (rc) return rc;
    long long n_var = 0;
    if ((rc = read_scalar(w.scal + 2, &n_var, st))) return rc;
    out.n_var_in = n_var;
    const float* keep_m = nullptr;
    if (!erase && d->n_inherit > 0 && n_var > 0) {
        if ((rc = fill(w.m, n0, d->inherit_m0, st))) return rc;
        DASS_CHECK_CUDA(cudaMemsetAsync(w.m_am, 0, sizeof(float) * n0, st));
        DASS_CHECK_CUDA(cudaMemsetAsync(w.m_av, 0, sizeof(float) * n0, st));
        const Scene g{n0, deg, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh};
        const InheritState s{d->is_var, n_var, w.var_rows, w.m, w.keep, w.m_grad, w.m_am, w.m_av, w.steps + 0,
                             w.d_keep, d->lr_inherit, d->beta1, d->beta2, d->eps, d->lambda_inher};
        if ((rc = inc_begin(g, ct, d->is_var, n_var, r, st))) return rc;
        rc = replay(st, d->n_inherit, [&] { return inherit_iteration(g, ct, d->targets, lam, d->batch, s, r, st); });
        if (rc) return rc;
        DASS_CHECK_CUDA(cudaMemcpyAsync(w.losses + 0, r.loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
        if ((rc = stage_end(r, st, &out.pairs_max))) return rc;
        keep_m = w.m;
        out.inherit_ran = 1;
    }
    // the copy: every base row, then the kept var rows (all of them if the stage did not run)
    rc = inherit_launch(n0, deg, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh, d->is_var, keep_m,
                        erase ? 1 : 0, w.means, w.ls, w.quats, w.logit, w.sh, w.is_var, w.remap, w.scal + 0,
                        w.misc_ws, w.misc_ws_bytes, st);
    if (rc) return rc;
    long long n1 = 0;
    if ((rc = read_scalar(w.scal + 0, &n1, st))) return rc;
    out.n_inherited = n1;

    // 2. dynamics-aware shift (Sec. 3.3) on the copy; the dynamic rows are base rows (same indices)
    DASS_CHECK_CUDA(cudaMemsetAsync(w.stat_accum, 0, sizeof(float) * n1, st));
    DASS_CHECK_CUDA(cudaMemsetAsync(w.stat_count, 0, sizeof(int) * n1, st));
    DASS_CHECK_CUDA(cudaMemsetAsync(w.dyn_mask, 0, n1, st));
    if (d->n_dyn > 0) {
        mark_rows_kernel<<<div_up(d->n_dyn, 256), 256, 0, st>>>(d->dyn_idx, d->n_dyn, n1, w.dyn_mask);
        count_launch();
        if ((rc = check_launch("mark_rows_kernel"))) return rc;
        DASS_CHECK_CUDA(cudaMemcpyAsync(d->offsets, d->offsets_init, sizeof(float) * 7 * d->n_dyn,
                                        cudaMemcpyDeviceToDevice, st));
        DASS_CHECK_CUDA(cudaMemsetAsync(w.off_m, 0, sizeof(float) * 7 * d->n_dyn, st));
        DASS_CHECK_CUDA(cudaMemsetAsync(w.off_v, 0, sizeof(float) * 7 * d->n_dyn, st));
    }
    DASS_CHECK_CUDA(cudaMemcpyAsync(w.render_means, w.means, sizeof(float) * 3 * n1, cudaMemcpyDeviceToDevice, st));
    DASS_CHECK_CUDA(cudaMemcpyAsync(w.render_quats, w.quats, sizeof(float) * 4 * n1, cudaMemcpyDeviceToDevice, st));
    static thread_local CamTable ct1;
    ct1 = ct;
    for (int c = 0; c < ct1.n; ++c) ct1.c[c].rec_base = (long long)c * n1;
    ct1.rec_stride = n1;
    const Scene g1{n1, deg, w.means, w.ls, w.quats, w.logit, w.sh};
    ShiftState ss{d->n_dyn, d->dyn_idx, w.dyn_mask, d->offsets, w.off_grad, w.off_m, w.off_v, w.steps + 1,
                  {d->lr_mu, d->lr_mu, d->lr_mu, d->lr_sigma, d->lr_sigma, d->lr_sigma, d->lr_sigma},
                  d->beta1, d->beta2, d->eps, w.render_means, w.render_quats, w.d_means_dyn, w.d_quats_dyn,
                  w.stat_accum, w.stat_count};
    if (d->n_shift > 0) {
        DASS_CHECK_CUDA(cudaMemsetAsync(r.track, 0, 2 * sizeof(long long), st));
        const Scene g1r{n1, deg, w.render_means, w.ls, w.render_quats, w.logit, w.sh};
        if ((rc = inc_begin(g1r, ct1, w.dyn_mask, d->n_dyn, r, st))) return rc;
        rc = replay(st, d->n_shift, [&] { return shift_iteration(g1, ct1, d->targets, lam, d->batch, ss, r, st); });
        if (rc) return rc;
        DASS_CHECK_CUDA(cudaMemcpyAsync(w.losses + 1, r.loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
        if ((rc = stage_end(r, st, &out.pairs_max))) return rc;
        // the learned offsets move the dynamic rows (render_* hold the unshifted static rows)
        rc = shift_launch(d->n_dyn, d->dyn_idx, d->offsets, w.means, w.quats, w.render_means, w.render_quats, st);
        if (rc) return rc;
        DASS_CHECK_CUDA(cudaMemcpyAsync(w.means, w.render_means, sizeof(float) * 3 * n1, cudaMemcpyDeviceToDevice, st));
        DASS_CHECK_CUDA(cudaMemcpyAsync(w.quats, w.render_quats, sizeof(float) * 4 * n1, cudaMemcpyDeviceToDevice, st));

        // 3. error-guided densification (Sec. 3.4): error pass on the last shift render, Eq. 4, spawn
        rc = error_pass_launch(r.image, d->targets, ct1, (double)d->quantile, n1, w.means, w.is_var, nullptr, w.gamma,
                               w.s_err, w.misc_ws, w.misc_ws_bytes, st);
        if (rc) return rc;
        rc = select_launch(n1, w.stat_accum, w.stat_count, w.s_err, w.is_var, d->tau_pos, d->tau_err, d->k_max, w.sel,
                           w.n_sel, w.misc_ws, w.misc_ws_bytes, st);
        if (rc) return rc;
    } else {
        DASS_CHECK_CUDA(cudaMemsetAsync(w.n_sel, 0, sizeof(int), st));
    }
    rc = spawn_launch(n1, deg, w.means, w.ls, w.quats, w.logit, w.sh, w.is_var, w.sel, w.n_sel, d->k_max, d->z,
                      w.scal + 1, st);
    if (rc) return rc;
    long long n2 = 0;
    if ((rc = read_scalar(w.scal + 1, &n2, st))) return rc;
    out.n_spawned = n2 - n1;

    // 4. densification stage (Sec. 3.4) over the var tail, then low-opacity pruning into the scene
    rc = mask_rows_launch(w.is_var, n2, w.var_rows, w.scal + 2, w.misc_ws, w.misc_ws_bytes, st);
    if (rc) return rc;
    long long nv2 = 0;
    if ((rc = read_scalar(w.scal + 2, &nv2, st))) return rc;
    const long long nb2 = n2 - nv2;          // var rows are the tail [nb2, n2) by construction
    long long n3 = n2;
    if (d->n_densify > 0 && nv2 > 0) {
        out.n_var_trained = nv2;
        const size_t wbytes = sizeof(float) * (size_t)(11 + 3 * K) * nv2;
        DASS_CHECK_CUDA(cudaMemsetAsync(w.dm, 0, wbytes, st));
        DASS_CHECK_CUDA(cudaMemsetAsync(w.dv, 0, wbytes, st));
        if ((rc = densify_prepare(nv2, K, w.dc_rows, w.rest_rows, st))) return rc;
        static thread_local CamTable ct2;
        ct2 = ct;
        for (int c = 0; c < ct2.n; ++c) ct2.c[c].rec_base = (long long)c * n2;
        ct2.rec_stride = n2;
        const Scene g2{n2, deg, w.means, w.ls, w.quats, w.logit, w.sh};
        const DensifyState s{w.means, w.ls, w.quats, w.logit, w.sh, nb2, nv2, w.var_rows, w.is_var, w.dgrad, w.dm,
                             w.dv, w.steps + 2, w.dc_rows, w.rest_rows,
                             {d->lr_means, d->lr_log_scales, d->lr_quats, d->lr_opacity, d->lr_sh_dc, d->lr_sh_rest},
                             d->beta1, d->beta2, d->eps};
        DASS_CHECK_CUDA(cudaMemsetAsync(r.track, 0, 2 * sizeof(long long), st));
        if ((rc = inc_begin(g2, ct2, w.is_var, nv2, r, st))) return rc;
        rc = replay(st, d->n_densify, [&] { return densify_iteration(g2, ct2, d->targets, lam, d->batch, s, r, st); });
        if (rc) return rc;
        DASS_CHECK_CUDA(cudaMemcpyAsync(w.losses + 2, r.loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
        if ((rc = stage_end(r, st, &out.pairs_max))) return rc;
        if ((rc = prune_logits_launch(n2, w.logit, d->prune_opacity, w.prune_m, st))) return rc;
        rc = inherit_launch(n2, deg, w.means, w.ls, w.quats, w.logit, w.sh, w.is_var, w.prune_m, 0, d->means,
                            d->log_scales, d->quats, d->opacity_logit, d->sh, d->is_var, w.remap, w.scal + 0,
                            w.misc_ws, w.misc_ws_bytes, st);
        if (rc) return rc;
        if ((rc = read_scalar(w.scal + 0, &n3, st))) return rc;
    } else {
        rc = copy_scene(n2, K, w.means, w.ls, w.quats, w.logit, w.sh, w.is_var, d->means, d->log_scales, d->quats,
                        d->opacity_logit, d->sh, d->is_var, cudaMemcpyDeviceToDevice, st);
        if (rc) return rc;
    }
    *d->n = n3;
    out.n_out = n3;
    double losses[3];
    DASS_CHECK_CUDA(cudaMemcpyAsync(losses, w.losses, sizeof(losses), cudaMemcpyDeviceToHost, st));
    if (d->host_means && d->host_log_scales && d->host_quats && d->host_opacity_logit && d->host_sh && d->host_is_var)
        if ((rc = copy_scene(n3, K, d->means, d->log_scales, d->quats, d->opacity_logit, d->sh, d->is_var,
                             d->host_means, d->host_log_scales, d->host_quats, d->host_opacity_logit, d->host_sh,
                             d->host_is_var, cudaMemcpyDeviceToHost, st)))
            return rc;
    DASS_CHECK_CUDA(cudaStreamSynchronize(st));
    out.loss_inherit = losses[0];
    out.loss_shift = losses[1];
    out.loss_densify = losses[2];
    return DASS_OK;
}

}  // namespace

DASS_API int dass_timestep_workspace(const dass_timestep_desc* d, size_t* bytes) {
    if (!d || !bytes || d->n_max <= 0 || d->sh_degree < 0 || d->sh_degree > 3 || d->pair_capacity < 1 ||
        d->pair_capacity >= (1ll << 31) || d->k_max < 0 || d->n_dyn < 0)
        return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n_max, &ct)) return DASS_ERR_INVALID_ARG;
    *bytes = carve_timestep(d, ct, nullptr, nullptr);
    return DASS_OK;
}

DASS_API int dass_timestep(const dass_timestep_desc* d, dass_timestep_stats* stats, void* stream) {
    if (!timestep_desc_ok(d) || !stats) return DASS_ERR_INVALID_ARG;
    static thread_local CamTable ct;
    if (!make_cam_table(d->cams, d->n_cams, d->tile, d->n_max, &ct)) return DASS_ERR_INVALID_ARG;
    const size_t image_bytes = sizeof(float) * 3 * (size_t)ct.pixels_total;
    if (d->next_targets) {   // the prefetched images may not land in this timestep's images
        const char* a = reinterpret_cast<const char*>(d->targets);
        const char* b = reinterpret_cast<const char*>(d->next_targets);
        if (a < b + image_bytes && b < a + image_bytes) return DASS_ERR_INVALID_ARG;
    }
    if (d->workspace_bytes < carve_timestep(d, ct, nullptr, nullptr)) return DASS_ERR_OOM;
    cudaStream_t st = as_stream(stream);
    if (st == nullptr) return DASS_ERR_INVALID_ARG;
    TsBufs w;
    carve_timestep(d, ct, reinterpret_cast<char*>(d->workspace), &w);
    std::memset(stats, 0, sizeof(*stats));
    // the first stage renders G_{t-1}: camera c's records start at c * n
    static thread_local CamTable ct0;
    ct0 = ct;
    for (int c = 0; c < ct0.n; ++c) ct0.c[c].rec_base = (long long)c * *d->n;
    ct0.rec_stride = *d->n;
    Prefetch next;
    if (d->next_targets) {
        if (int rc = next.start(d->next_targets, d->next_targets_host, image_bytes, st)) return rc;
    }
    int rc = timestep_run(d, ct0, w, *stats, st);
    if (rc) cudaStreamSynchronize(st);   // nothing of the failed timestep stays in flight
    const int rc_next = next.finish();
    return rc ? rc : rc_next;
}
