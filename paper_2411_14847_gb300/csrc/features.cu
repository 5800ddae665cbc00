// Identity-feature rendering and the per-Gaussian dynamics query of the shift stage (Sec. 3.3):
// every Gaussian carries an object-identity feature vector (Gaussian Grouping); the vectors are
// alpha-composited exactly like colours, a linear classifier turns rendered features into
// per-pixel object IDs, the IDs seen inside the dynamic image areas are collected, and the
// Gaussians whose own feature classifies into one of them form the dynamic group.
//
// The compositor walks the sorted tile lists of dass_bin_sort with the forward's alpha, skip and
// stop rules (scalar form, one pixel per thread, each tile split into 16 x 16 CTAs), staging each
// batch's splat parameters and feature rows through shared memory; each warp (two pixel rows)
// walks only the staged splats whose footprint reaches its rows.
#include "common.cuh"

namespace dass {

namespace {

constexpr int kFeatCT = 16;                // CTA side (pixels)
constexpr int kFeatBatch = 128;            // staged Gaussians per round
constexpr int kFeatThreads = kFeatCT * kFeatCT;
static_assert(kFeatBatch <= 256, "warp lists hold 8-bit indices");

template <int F>
__global__ void __launch_bounds__(kFeatThreads) render_features_kernel(
    const dass_splat* __restrict__ splats, const uint32_t* __restrict__ pair_rec, const uint32_t* __restrict__ ranges,
    CamTable ct, const float* __restrict__ feats, long long rec_stride, float* __restrict__ out) {
    constexpr int NW = kFeatThreads / 32;
    __shared__ float4 sA[kFeatBatch];      // u, v, a', b2'
    __shared__ float2 sB[kFeatBatch];      // c', o
    __shared__ float4 sK[kFeatBatch];      // footprint (a, b, c, k2)
    __shared__ __align__(16) float sF[kFeatBatch][F + 4];   // rows 16-byte aligned
    __shared__ unsigned char sList[NW][kFeatBatch];
    const int TILE = ct.tile;
    const int S = TILE > kFeatCT ? TILE / kFeatCT : 1;   // CTAs per tile side
    const int CT = TILE > kFeatCT ? kFeatCT : TILE;
    const int tile_id = blockIdx.x / (S * S);
    const int sub = blockIdx.x % (S * S);
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = tid % kFeatCT, ly = tid / kFeatCT;
    const int x0 = (local % cam.tiles_x) * TILE + (sub % S) * CT, y0 = (local / cam.tiles_x) * TILE + (sub / S) * CT;
    const int px = x0 + lx, py = y0 + ly;
    const bool inside = lx < CT && ly < CT && px < cam.W && py < cam.H;
    // this warp's pixels: columns x0 .. x0 + CT - 1 of rows y0 + 2 warp, y0 + 2 warp + 1
    const float wbx = (float)x0, wby = (float)(y0 + 2 * warp), wwm1 = (float)(CT - 1);
    const uint32_t start = ranges[2 * tile_id], end = ranges[2 * tile_id + 1];
    const uint32_t stride32 = (uint32_t)rec_stride;    // records fit 32 bits (n_cams n < 2^32)
    float acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.f;
    float T = 1.f;
    bool done = !inside;
    const float fx = (float)px, fy = (float)py;
    for (uint32_t base = start; base < end; base += kFeatBatch) {
        if (__syncthreads_count(done) == kFeatThreads) break;
        const int cnt = min((uint32_t)kFeatBatch, end - base);
        // one staged entry per thread: its splat parameters and its feature row (float4 loads)
        for (int e = tid; e < cnt; e += kFeatThreads) {
            const uint32_t rec = pair_rec[base + e];
            const float4* sp = reinterpret_cast<const float4*>(splats + rec);
            const float4 s0 = __ldg(sp), s1 = __ldg(sp + 1);
            sA[e] = make_float4(s0.x, s0.y, __fmul_rn(s0.z, kNegHalfLog2e), __fmul_rn(2.f * s0.w, kNegHalfLog2e));
            sB[e] = make_float2(__fmul_rn(s1.x, kNegHalfLog2e), s1.y);
            sK[e] = make_float4(s0.z, s0.w, s1.x, footprint_k2(s0.z, s0.w, s1.x, s1.y));
            const float4* fr = reinterpret_cast<const float4*>(feats + (size_t)(rec % stride32) * F);
#pragma unroll
            for (int k = 0; k < F / 4; ++k) *reinterpret_cast<float4*>(&sF[e][4 * k]) = __ldg(fr + k);
        }
        __syncthreads();
        // the warp's list: staged splats whose footprint reaches its two pixel rows (ascending)
        int nl = 0;
        if (__any_sync(0xffffffffu, !done)) {
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                const int j = j0 + lane;
                const bool hit = j < cnt && footprint_reaches_rect(-sA[j].x, -sA[j].y, sK[j], wbx, wby, wwm1, 1.f);
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) sList[warp][nl + __popc(m & ((1u << lane) - 1u))] = (unsigned char)j;
                nl += __popc(m);
            }
            __syncwarp();
        }
        for (int t = 0; t < nl && !done; ++t) {
            const int j = sList[warp][t];
            const float4 A = sA[j];
            const float2 B = sB[j];
            const float dx = __fsub_rn(fx, A.x), dy = __fsub_rn(fy, A.y);
            const float alpha = splat_alpha(B.y, splat_gauss(A.z, A.w, B.x, dx, dy));
            if (alpha < kAlphaMin) continue;
            const float test = __fmaf_rn(-alpha, T, T);     // T - alpha T, as the colour forward
            if (test < kTStop) {
                done = true;
                break;
            }
            const float w = __fmul_rn(alpha, T);
#pragma unroll
            for (int f = 0; f < F; ++f) acc[f] = __fmaf_rn(sF[j][f], w, acc[f]);
            T = test;
        }
    }
    if (inside) {
        float* dst = out + (cam.pix_base + (long long)py * cam.W + px) * F;
#pragma unroll
        for (int f = 0; f < F; ++f) dst[f] = acc[f];
    }
}

// Argmax over K classes of W x + b for R rows of x (F features each, rows r of x at x + r F);
// ties take the lower class. x and W are 16-byte aligned (F is a multiple of 4): the rows and
// the weight rows are read as float4, each weight load serving the R rows.
template <int F, int R>
__device__ __forceinline__ void classify(const float* __restrict__ x, int rows, const float* W, const float* b, int K,
                                         int (&best)[R]) {
    float v[R][F];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int f = 0; f < F; f += 4) {
            const float4 q = r < rows ? __ldg(reinterpret_cast<const float4*>(x + r * F + f))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            v[r][f] = q.x;
            v[r][f + 1] = q.y;
            v[r][f + 2] = q.z;
            v[r][f + 3] = q.w;
        }
    float best_v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        best[r] = 0;
        best_v[r] = -3.4e38f;
    }
    for (int k = 0; k < K; ++k) {
        float s[R];
#pragma unroll
        for (int r = 0; r < R; ++r) s[r] = b[k];
#pragma unroll
        for (int f = 0; f < F; f += 4) {
            const float4 w = *reinterpret_cast<const float4*>(W + k * F + f);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                s[r] = fmaf(w.x, v[r][f], s[r]);
                s[r] = fmaf(w.y, v[r][f + 1], s[r]);
                s[r] = fmaf(w.z, v[r][f + 2], s[r]);
                s[r] = fmaf(w.w, v[r][f + 3], s[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (s[r] > best_v[r]) {
                best_v[r] = s[r];
                best[r] = k;
            }
    }
}

// Rows classified per thread: 2 (a weight load serves both) unless the feature rows are long.
template <int F>
constexpr int cls_rows() { return F <= 16 ? 2 : 1; }

// Classifier weights staged in shared memory when they fit (kClassifierSmem floats, 32 KB: below
// the default dynamic shared-memory limit), else read through the cache.
constexpr int kClassifierSmem = 8192;

template <int F>
__device__ __forceinline__ const float* stage_classifier(const float* __restrict__ W, const float* __restrict__ b,
                                                         int K, float* sm, const float*& bs) {
    if (K * (F + 1) > kClassifierSmem) {
        bs = b;
        return W;
    }
    for (int i = threadIdx.x; i < K * F; i += blockDim.x) sm[i] = W[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) sm[K * F + i] = b[i];
    __syncthreads();
    bs = sm + K * F;
    return sm;
}

template <int F>
__global__ void object_ids_kernel(const float* __restrict__ x, long long n, const float* __restrict__ W,
                                  const float* __restrict__ b, int K, int* __restrict__ ids) {
    constexpr int R = cls_rows<F>();
    extern __shared__ __align__(16) float s_cls[];
    const float* bs;
    const float* Ws = stage_classifier<F>(W, b, K, s_cls, bs);
    const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * R;
    if (i0 >= n) return;
    const int rows = n - i0 < R ? (int)(n - i0) : R;
    int best[R];
    classify<F, R>(x + i0 * F, rows, Ws, bs, K, best);
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (r < rows) ids[i0 + r] = best[r];
}

// Class histogram of the dynamic-area pixels: grid-stride, per-block counts in shared memory
// (K <= kHistSmem), one global add per class and block.
constexpr int kHistSmem = 4096;

__global__ void dynamic_id_hist_kernel(const int* __restrict__ ids, const uint8_t* __restrict__ dyn_area, long long n,
                                       int K, unsigned int* __restrict__ hist) {
    __shared__ unsigned int sh[kHistSmem];
    const bool local = K <= kHistSmem;
    if (local) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) sh[k] = 0u;
        __syncthreads();
    }
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
        if (!dyn_area[i]) continue;
        if (local)
            atomicAdd(sh + ids[i], 1u);
        else
            atomicAdd(hist + ids[i], 1u);
    }
    if (local) {
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x)
            if (sh[k]) atomicAdd(hist + k, sh[k]);
    }
}

__global__ void dynamic_id_mask_kernel(const unsigned int* __restrict__ hist, int K, unsigned int min_pixels,
                                       uint8_t* __restrict__ obj_mask) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) obj_mask[k] = hist[k] >= min_pixels ? 1 : 0;
}

template <int F>
__global__ void dynamic_gaussians_kernel(const float* __restrict__ feats, long long n, const float* __restrict__ W,
                                         const float* __restrict__ b, int K, const uint8_t* __restrict__ obj_mask,
                                         uint8_t* __restrict__ dyn_mask) {
    constexpr int R = cls_rows<F>();
    extern __shared__ __align__(16) float s_cls[];
    const float* bs;
    const float* Ws = stage_classifier<F>(W, b, K, s_cls, bs);
    const long long g0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * R;
    if (g0 >= n) return;
    const int rows = n - g0 < R ? (int)(n - g0) : R;
    int best[R];
    classify<F, R>(feats + g0 * F, rows, Ws, bs, K, best);
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (r < rows) dyn_mask[g0 + r] = obj_mask[best[r]];
}

__global__ void mask_flags_kernel(const uint8_t* __restrict__ mask, long long n, uint32_t* __restrict__ flags) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = mask[i] ? 1u : 0u;
}

__global__ void mask_scatter_kernel(const uint8_t* __restrict__ mask, const uint32_t* __restrict__ pos, long long n,
                                    const long long* __restrict__ total, int* __restrict__ rows,
                                    long long* __restrict__ count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *count = *total;
    if (i < n && mask[i]) rows[pos[i]] = (int)i;
}

__global__ void set_len_kernel(long long* dst, long long v) { *dst = v; }

template <int F>
int features_launch(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct,
                    const float* feats, long long stride, float* out, cudaStream_t st) {
    const int S = ct.tile > kFeatCT ? ct.tile / kFeatCT : 1;
    render_features_kernel<F><<<ct.tiles_total * S * S, kFeatThreads, 0, st>>>(sp, pr, rg, ct, feats, stride, out);
    count_launch();
    return check_launch("render_features_kernel");
}

template <int F>
int ids_launch(const float* x, long long n, const float* W, const float* b, int K, int* ids, cudaStream_t st) {
    const size_t sm = K * (F + 1) <= kClassifierSmem ? sizeof(float) * (size_t)K * (F + 1) : 0;
    object_ids_kernel<F><<<div_up(div_up(n, cls_rows<F>()), 256), 256, sm, st>>>(x, n, W, b, K, ids);
    count_launch();
    return check_launch("object_ids_kernel");
}

template <int F>
int dyn_gauss_launch(const float* feats, long long n, const float* W, const float* b, int K, const uint8_t* om,
                     uint8_t* dm, cudaStream_t st) {
    const size_t sm = K * (F + 1) <= kClassifierSmem ? sizeof(float) * (size_t)K * (F + 1) : 0;
    dynamic_gaussians_kernel<F><<<div_up(div_up(n, cls_rows<F>()), 256), 256, sm, st>>>(feats, n, W, b, K, om, dm);
    count_launch();
    return check_launch("dynamic_gaussians_kernel");
}

#define DASS_FEAT_DISPATCH(FN, F, ...)           \
    switch (F) {                                 \
        case 4: return FN<4>(__VA_ARGS__);       \
        case 8: return FN<8>(__VA_ARGS__);       \
        case 16: return FN<16>(__VA_ARGS__);     \
        case 32: return FN<32>(__VA_ARGS__);     \
        default: return DASS_ERR_UNSUPPORTED;    \
    }

}  // namespace

int scan_u32_public(const uint32_t* in, uint32_t* out, const long long* len_dev, long long len_cap,
                    unsigned long long* partial, long long* total, cudaStream_t st);
size_t scan_partials_bytes(long long len);

int render_features_launch(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct,
                           const float* feats, int F, long long stride, float* out, cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    DASS_FEAT_DISPATCH(features_launch, F, sp, pr, rg, ct, feats, stride, out, st)
}

int object_ids_launch(const float* x, long long n, int F, const float* W, const float* b, int K, int* ids,
                      cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    DASS_FEAT_DISPATCH(ids_launch, F, x, n, W, b, K, ids, st)
}

int dynamic_objects_launch(const int* ids, const uint8_t* dyn_area, long long n, int K, unsigned int min_pixels,
                           uint8_t* obj_mask, unsigned int* hist, cudaStream_t st) {
    DASS_CHECK_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * (size_t)K, st));
    if (n > 0) {
        const long long nb = div_up(n, 256);
        dynamic_id_hist_kernel<<<nb < 152 * 8 ? (int)nb : 152 * 8, 256, 0, st>>>(ids, dyn_area, n, K, hist);
        count_launch();
        if (int rc = check_launch("dynamic_id_hist_kernel")) return rc;
    }
    dynamic_id_mask_kernel<<<div_up(K, 256), 256, 0, st>>>(hist, K, min_pixels, obj_mask);
    count_launch();
    return check_launch("dynamic_id_mask_kernel");
}

int dynamic_gaussians_launch(const float* feats, long long n, int F, const float* W, const float* b, int K,
                             const uint8_t* obj_mask, uint8_t* dyn_mask, cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    DASS_FEAT_DISPATCH(dyn_gauss_launch, F, feats, n, W, b, K, obj_mask, dyn_mask, st)
}

size_t mask_rows_workspace_bytes(long long n) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(sizeof(long long) * 2) + 2 * al(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)) + al(scan_partials_bytes(n));
}

int mask_rows_launch(const uint8_t* mask, long long n, int* rows, long long* count, void* ws, size_t ws_bytes,
                     cudaStream_t st) {
    if (ws_bytes < mask_rows_workspace_bytes(n)) return DASS_ERR_OOM;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char* p = reinterpret_cast<char*>(ws);
    long long* sc = reinterpret_cast<long long*>(p);
    p += al(sizeof(long long) * 2);
    uint32_t* flags = reinterpret_cast<uint32_t*>(p);
    p += al(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t* pos = reinterpret_cast<uint32_t*>(p);
    p += al(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    unsigned long long* part = reinterpret_cast<unsigned long long*>(p);
    if (n <= 0) {
        DASS_CHECK_CUDA(cudaMemsetAsync(count, 0, sizeof(long long), st));
        return DASS_OK;
    }
    set_len_kernel<<<1, 1, 0, st>>>(sc + 0, n);
    count_launch();
    mask_flags_kernel<<<div_up(n, 256), 256, 0, st>>>(mask, n, flags);
    count_launch();
    if (int rc = scan_u32_public(flags, pos, sc + 0, n, part, sc + 1, st)) return rc;
    mask_scatter_kernel<<<div_up(n, 256), 256, 0, st>>>(mask, pos, n, sc + 1, rows, count);
    count_launch();
    return check_launch("mask_rows");
}

}  // namespace dass
