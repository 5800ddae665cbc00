// Forward and backward alpha compositing (App. A.1) over every tile of every camera in one
// launch. One CTA per B x B tile; each warp owns an 8 x 4 block of pixels, one pixel per lane.
// The tile's depth-sorted Gaussians are staged through shared memory in batches; after each
// batch is staged, every warp compacts (ballot + prefix popcount, order preserved) the entries
// whose alpha >= 1/255 footprint ellipse reaches its own 8 x 4 block, and composites only
// those. The backward walks the lists in reverse from the last contributor, recomputing alpha
// and T_j = T_{j+1}/(1-alpha_j) from the saved T_final, and reduces per-Gaussian gradients
// warp-wide (shuffles), then block-wide (shared-memory atomics), then into global memory
// (vector atomics).
#include "common.cuh"

namespace dass {

namespace {

struct Staged {
    float4 A;    // u, v, a * kNegHalfLog2e, c * kNegHalfLog2e
    float4 B;    // 2 b * kNegHalfLog2e, o, r, g
    float4 F;    // a, b, c, k2 (footprint ellipse d^T conic d <= k2)
    float blue;
};

// Stage one splat into its shared-memory form (identical in forward and backward).
__device__ __forceinline__ void stage_splat(const dass_splat* __restrict__ splats, uint32_t rec, float4& A, float4& Bv,
                                            float4& F, float& blue) {
    const float4* sp = reinterpret_cast<const float4*>(splats + rec);
    float4 s0 = __ldg(sp);
    float4 s1 = __ldg(sp + 1);
    float s2 = __ldg(reinterpret_cast<const float*>(sp + 2));
    A = make_float4(s0.x, s0.y, __fmul_rn(s0.z, kNegHalfLog2e), __fmul_rn(s1.x, kNegHalfLog2e));
    Bv = make_float4(__fmul_rn(2.f * s0.w, kNegHalfLog2e), s1.y, s1.z, s1.w);
    Footprint f;
    float k2 = footprint_of(s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, f) ? f.k2 : -1.f;
    F = make_float4(s0.z, s0.w, s1.x, k2);
    blue = s2;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Does the footprint of staged entry (A.xy = centre, F = conic + k2) reach the warp's 8x4 block
// whose first pixel centre is (bx, by)? Ellipse-rectangle test: the quadratic form is evaluated
// at a point of each edge facing the centre (the clamped 1-D minimiser, computed with a fast
// division); any point of the rectangle gives an upper bound of its minimum, so a Gaussian is
// culled only if every pixel of the block is outside its footprint (up to k2's slack).
__device__ __forceinline__ bool reaches_block(const float4 A, const float4 F, float bx, float by) {
    if (F.w < 0.f) return false;
    const float x0 = bx - A.x, x1 = bx + 7.f - A.x, y0 = by - A.y, y1 = by + 3.f - A.y;
    const bool in_x = x0 <= 0.f && x1 >= 0.f, in_y = y0 <= 0.f && y1 >= 0.f;
    if (in_x && in_y) return true;
    float qmin = 3.4e38f;
    if (!in_x) {
        const float X = x0 > 0.f ? x0 : x1;
        const float dy = fminf(fmaxf(__fdividef(-F.y * X, F.z), y0), y1);
        qmin = fminf(qmin, F.x * X * X + 2.f * F.y * X * dy + F.z * dy * dy);
    }
    if (!in_y) {
        const float Y = y0 > 0.f ? y0 : y1;
        const float dx = fminf(fmaxf(__fdividef(-F.y * Y, F.x), x0), x1);
        qmin = fminf(qmin, F.x * dx * dx + 2.f * F.y * dx * Y + F.z * Y * Y);
    }
    return qmin <= F.w;
}

// Compact the indices [0, cnt) of the staged batch whose footprint reaches this warp's block
// into list[] (ascending), optionally only indices <= jmax. Returns the count (warp-uniform).
__device__ __forceinline__ int warp_compact(const float4* __restrict__ sA, const float4* __restrict__ sF, int cnt,
                                            int jmax, float bx, float by, unsigned short* list, int lane) {
    int n = 0;
    int lim = min(cnt, jmax + 1);
    for (int j0 = 0; j0 < lim; j0 += 32) {
        int j = j0 + lane;
        bool hit = j < lim && reaches_block(sA[j], sF[j], bx, by);
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[n + __popc(m & lanemask_lt())] = (unsigned short)j;
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

template <int TILE>
struct Layout {
    static constexpr int NT = TILE * TILE;
    static constexpr int NW = NT / 32;
    static constexpr int WX = TILE / 8;   // warp blocks per tile row
};

// Pixel of (tile, thread): warp w covers the 8x4 block (w % WX, w / WX) of the tile.
template <int TILE>
__device__ __forceinline__ void pixel_of(const CamInfo& cam, int local, int tid, int& px, int& py, float& bx,
                                         float& by) {
    const int warp = tid >> 5, lane = tid & 31;
    const int tx0 = (local % cam.tiles_x) * TILE, ty0 = (local / cam.tiles_x) * TILE;
    const int wx = (warp % Layout<TILE>::WX) * 8, wy = (warp / Layout<TILE>::WX) * 4;
    px = tx0 + wx + (lane & 7);
    py = ty0 + wy + (lane >> 3);
    bx = (float)(tx0 + wx);
    by = (float)(ty0 + wy);
}

// COUNT = true is a separate instantiation used only to measure the algorithmic work of a
// render (pairs each pixel evaluates before its own stop, pairs it adds, and pairs the
// backward evaluates); the timed kernels are the COUNT = false instantiations.
template <int TILE, int BATCH, bool COUNT>
__global__ void __launch_bounds__(TILE* TILE) render_fwd_kernel(const dass_splat* __restrict__ splats,
                                                               const uint32_t* __restrict__ pair_rec,
                                                               const uint32_t* __restrict__ ranges, CamTable ct,
                                                               float3 bg, float* __restrict__ image,
                                                               float* __restrict__ T_final, int* __restrict__ n_last,
                                                               unsigned long long* __restrict__ work) {
    constexpr int NT = Layout<TILE>::NT;
    constexpr int NW = Layout<TILE>::NW;
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ float4 sF[BATCH];
    __shared__ float sC[BATCH];
    __shared__ unsigned short sList[NW][BATCH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile_id = blockIdx.x;
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    int px, py;
    float bx, by;
    pixel_of<TILE>(cam, tile_id - cam.tile_base, tid, px, py, bx, by);
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t start = ranges[2 * tile_id], end = ranges[2 * tile_id + 1];
    const float fx = (float)px, fy = (float)py;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int last = -1;
    bool done = !inside;
    unsigned long long n_eval = 0, n_add = 0;
    for (uint32_t base = start; base < end; base += BATCH) {
        if (__syncthreads_count(done) == NT) break;
        const int cnt = min((uint32_t)BATCH, end - base);
        for (int i = tid; i < cnt; i += NT) stage_splat(splats, pair_rec[base + i], sA[i], sB[i], sF[i], sC[i]);
        __syncthreads();
        if (__all_sync(0xffffffffu, done)) continue;
        const int nl = warp_compact(sA, sF, cnt, BATCH, bx, by, sList[warp], lane);
        if (!done) {
            for (int t = 0; t < nl; ++t) {
                const int j = sList[warp][t];
                const float4 A = sA[j];
                const float4 Bv = sB[j];
                const float dx = __fsub_rn(fx, A.x), dy = __fsub_rn(fy, A.y);
                const float G = splat_gauss(A.z, Bv.x, A.w, dx, dy);
                const float alpha = splat_alpha(Bv.y, G);
                if (COUNT) ++n_eval;
                if (alpha < kAlphaMin) continue;
                const float test = __fmul_rn(T, __fsub_rn(1.f, alpha));
                if (test < kTStop) { done = true; break; }
                if (COUNT) ++n_add;
                const float w = __fmul_rn(alpha, T);
                C0 = __fmaf_rn(Bv.z, w, C0);
                C1 = __fmaf_rn(Bv.w, w, C1);
                C2 = __fmaf_rn(sC[j], w, C2);
                T = test;
                last = (int)(base + j);
            }
        }
    }
    if (inside) {
        const long long plane = (long long)cam.W * cam.H;
        const long long pix = (long long)py * cam.W + px;
        float* img = image + 3 * cam.pix_base;
        img[pix] = __fmaf_rn(T, bg.x, C0);
        img[plane + pix] = __fmaf_rn(T, bg.y, C1);
        img[2 * plane + pix] = __fmaf_rn(T, bg.z, C2);
        T_final[cam.pix_base + pix] = T;
        n_last[cam.pix_base + pix] = last;
    }
    if (COUNT) {
        unsigned long long n_bwd = last >= 0 ? (unsigned long long)(last - (int)start + 1) : 0ull;
        atomicAdd(work + 0, n_eval);
        atomicAdd(work + 1, n_add);
        atomicAdd(work + 2, n_bwd);
        if (inside) atomicAdd(work + 3, 1ull);
    }
}

// Sum 8 values across the warp with a transposed butterfly (4+2+1+1+1 shuffles). Lane l with
// (l & 3) == 0 ends with the full sum of value index ((l>>4)&1)*4 + ((l>>3)&1)*2 + ((l>>2)&1).
__device__ __forceinline__ float warp_reduce8(float v[8], int lane) {
    const bool h4 = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float send = h4 ? v[i] : v[i + 4];
        float keep = h4 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    const bool h3 = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float send = h3 ? v[i] : v[i + 2];
        float keep = h3 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const bool h2 = lane & 4;
    float send = h2 ? v[0] : v[1];
    float keep = h2 ? v[1] : v[0];
    float r = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE* TILE) render_bwd_kernel(
    const dass_splat* __restrict__ splats, const uint32_t* __restrict__ pair_rec, const uint32_t* __restrict__ ranges,
    CamTable ct, float3 bg, const float* __restrict__ T_final, const int* __restrict__ n_last,
    const float* __restrict__ dL_dimage, dass_splat_grad* __restrict__ gsplat) {
    constexpr int NT = Layout<TILE>::NT;
    constexpr int NW = Layout<TILE>::NW;
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ float4 sF[BATCH];
    __shared__ float sC[BATCH];
    __shared__ uint32_t sRec[BATCH];
    __shared__ float sG[BATCH][12];
    __shared__ unsigned short sList[NW][BATCH];
    __shared__ int s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile_id = blockIdx.x;
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    int px, py;
    float bx, by;
    pixel_of<TILE>(cam, tile_id - cam.tile_base, tid, px, py, bx, by);
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t start = ranges[2 * tile_id];
    const float fx = (float)px, fy = (float)py;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    int last = -1;
    if (inside) {
        const long long plane = (long long)cam.W * cam.H;
        const long long pix = (long long)py * cam.W + px;
        const float* gi = dL_dimage + 3 * cam.pix_base;
        g0 = gi[pix];
        g1 = gi[plane + pix];
        g2 = gi[2 * plane + pix];
        T = T_final[cam.pix_base + pix];
        last = n_last[cam.pix_base + pix];
    }
    if (tid == 0) s_maxlast = -1;
    __syncthreads();
    const int wlast = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0 && wlast >= 0) atomicMax(&s_maxlast, wlast);
    __syncthreads();
    const long long endpos = (long long)s_maxlast + 1;
    float R0 = bg.x, R1 = bg.y, R2 = bg.z;   // colour behind the current Gaussian (incl. background)
    for (long long hi = endpos; hi > (long long)start; hi -= BATCH) {
        const long long lo = hi - BATCH > (long long)start ? hi - BATCH : (long long)start;
        const int cnt = (int)(hi - lo);
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            uint32_t rec = pair_rec[lo + i];
            sRec[i] = rec;
            stage_splat(splats, rec, sA[i], sB[i], sF[i], sC[i]);
#pragma unroll
            for (int k = 0; k < 12; ++k) sG[i][k] = 0.f;
        }
        __syncthreads();
        const int jmax = (int)((long long)wlast - lo);   // entries beyond every lane's last are skipped
        const int nl = jmax >= 0 ? warp_compact(sA, sF, cnt, jmax, bx, by, sList[warp], lane) : 0;
        for (int t = nl - 1; t >= 0; --t) {
            const int j = sList[warp][t];
            const long long pos = lo + j;
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float eb = 0.f;
            bool contrib = false;
            if (pos <= (long long)last) {
                const float4 A = sA[j];
                const float4 Bv = sB[j];
                const float dx = __fsub_rn(fx, A.x), dy = __fsub_rn(fy, A.y);
                const float G = splat_gauss(A.z, Bv.x, A.w, dx, dy);
                const float alpha = splat_alpha(Bv.y, G);
                if (alpha >= kAlphaMin) {
                    contrib = true;
                    const float om = 1.f - alpha;
                    const float Tj = T / om;
                    const float w = alpha * Tj;
                    const float c2 = sC[j];
                    v[6] = w * g0;
                    v[7] = w * g1;
                    eb = w * g2;
                    const float dLda = Tj * ((Bv.z - R0) * g0 + (Bv.w - R1) * g1 + (c2 - R2) * g2);
                    R0 = Bv.z * alpha + om * R0;
                    R1 = Bv.w * alpha + om * R1;
                    R2 = c2 * alpha + om * R2;
                    T = Tj;
                    const float oG = Bv.y * G;
                    if (oG < kAlphaMax) {
                        const float4 F = sF[j];   // (a, b, c) of the conic
                        const float dpow = dLda * alpha;
                        v[5] = dLda * G;
                        v[0] = dpow * (F.x * dx + F.y * dy);
                        v[1] = dpow * (F.z * dy + F.y * dx);
                        v[2] = -0.5f * dx * dx * dpow;
                        v[3] = -dx * dy * dpow;
                        v[4] = -0.5f * dy * dy * dpow;
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, contrib)) {
                float r = warp_reduce8(v, lane);
                float e = warp_sum(eb);
                if ((lane & 3) == 0) {
                    int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                    atomicAdd(&sG[j][idx], r);
                }
                if (lane == 1) atomicAdd(&sG[j][8], e);
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            float4 a = make_float4(sG[i][0], sG[i][1], sG[i][2], sG[i][3]);
            float4 b = make_float4(sG[i][4], sG[i][5], sG[i][6], sG[i][7]);
            float c = sG[i][8];
            bool nz = (a.x != 0.f) | (a.y != 0.f) | (a.z != 0.f) | (a.w != 0.f) | (b.x != 0.f) | (b.y != 0.f) |
                      (b.z != 0.f) | (b.w != 0.f) | (c != 0.f);
            if (nz) {
                float4* dst = reinterpret_cast<float4*>(gsplat + sRec[i]);
                atomicAdd(dst, a);
                atomicAdd(dst + 1, b);
                atomicAdd(reinterpret_cast<float*>(dst + 2), c);
            }
        }
    }
}

template <int TILE, int BATCH>
int launch_fwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               float* img, float* tf, int* nl, unsigned long long* work, cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    if (work)
        render_fwd_kernel<TILE, BATCH, true><<<ct.tiles_total, TILE * TILE, 0, st>>>(sp, pr, rg, ct, bg, img, tf, nl,
                                                                                    work);
    else
        render_fwd_kernel<TILE, BATCH, false><<<ct.tiles_total, TILE * TILE, 0, st>>>(sp, pr, rg, ct, bg, img, tf, nl,
                                                                                     nullptr);
    count_launch();
    return check_launch("render_fwd_kernel");
}

template <int TILE, int BATCH>
int launch_bwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               const float* tf, const int* nl, const float* dimg, dass_splat_grad* gs, cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    render_bwd_kernel<TILE, BATCH><<<ct.tiles_total, TILE * TILE, 0, st>>>(sp, pr, rg, ct, bg, tf, nl, dimg, gs);
    count_launch();
    return check_launch("render_bwd_kernel");
}

}  // namespace

#define DASS_DISPATCH(FN, ...)                                                        \
    switch (ct.tile * 1000 + batch) {                                                 \
        case 8064: return FN<8, 64>(__VA_ARGS__);                                     \
        case 8128: return FN<8, 128>(__VA_ARGS__);                                    \
        case 8256: return FN<8, 256>(__VA_ARGS__);                                    \
        case 16064: return FN<16, 64>(__VA_ARGS__);                                   \
        case 16128: return FN<16, 128>(__VA_ARGS__);                                  \
        case 16256: return FN<16, 256>(__VA_ARGS__);                                  \
        case 32064: return FN<32, 64>(__VA_ARGS__);                                   \
        case 32128: return FN<32, 128>(__VA_ARGS__);                                  \
        case 32256: return FN<32, 256>(__VA_ARGS__);                                  \
        default: return DASS_ERR_INVALID_ARG;                                         \
    }

int render_fwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, float* image, float* T_final, int* n_last, cudaStream_t st,
                      unsigned long long* work) {
    DASS_DISPATCH(launch_fwd, splats, pair_rec, ranges, ct, bg, image, T_final, n_last, work, st)
}

int render_bwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, const float* T_final, const int* n_last, const float* dL_dimage,
                      dass_splat_grad* gsplat, cudaStream_t st) {
    DASS_DISPATCH(launch_bwd, splats, pair_rec, ranges, ct, bg, T_final, n_last, dL_dimage, gsplat, st)
}

}  // namespace dass
