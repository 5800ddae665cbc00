// Forward and backward alpha compositing (App. A.1) over every tile of every camera in one
// launch. One CTA per B x B tile; each warp owns an 8 x 8 block of pixels, two pixels per lane.
// The tile's depth-sorted Gaussians are staged through shared memory in batches; after each
// batch is staged, every warp compacts (ballot + prefix popcount, order preserved) the entries
// whose alpha >= 1/255 footprint ellipse reaches its own block of pixels, and composites only
// those. The backward walks the lists in reverse from the last contributor, recomputing alpha
// and T_j = T_{j+1}/(1-alpha_j) from the saved T_final, and reduces per-Gaussian gradients
// warp-wide (shuffles), then block-wide (shared-memory atomics), then into global memory
// (vector atomics).
#include "common.cuh"

namespace dass {

namespace {

// Stage one splat into its shared-memory form (identical in forward and backward):
//   A = (u, v, a * kNegHalfLog2e, c * kNegHalfLog2e), B = (2 b * kNegHalfLog2e, o, r, g),
//   F = (a, b, c, k2) with the footprint ellipse d^T conic d <= k2 (k2 < 0: no footprint).
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
template <int BH>
__device__ __forceinline__ bool reaches_block(const float4 A, const float4 F, float bx, float by) {
    if (F.w < 0.f) return false;
    const float x0 = bx - A.x, x1 = bx + 7.f - A.x, y0 = by - A.y, y1 = by + (float)(BH - 1) - A.y;
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

// Compact the indices [0, cnt) of the staged batch whose footprint reaches this warp's 8 x BH
// block into list[] (ascending), only indices <= jmax. Returns the count (warp-uniform).
template <int BH>
__device__ __forceinline__ int warp_compact(const float4* __restrict__ sA, const float4* __restrict__ sF, int cnt,
                                            int jmax, float bx, float by, unsigned short* list, int lane) {
    int n = 0;
    int lim = min(cnt, jmax + 1);
    for (int j0 = 0; j0 < lim; j0 += 32) {
        int j = j0 + lane;
        bool hit = j < lim && reaches_block<BH>(sA[j], sF[j], bx, by);
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[n + __popc(m & lanemask_lt())] = (unsigned short)j;
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

// Forward state of one pixel.
struct PixFwd {
    float fy, T, C0, C1, C2;
    int last;
    bool done;
    unsigned long long n_eval, n_add, n_full;
};

template <bool COUNT>
__device__ __forceinline__ void pix_fwd_step(PixFwd& p, int pos, float dx, const float4 A, const float4 Bv,
                                             const float* __restrict__ sC, int j, bool full = false) {
    if (p.done) return;
    const float dy = __fsub_rn(p.fy, A.y);
    const float G = splat_gauss(A.z, Bv.x, A.w, dx, dy);
    const float alpha = splat_alpha(Bv.y, G);
    if (COUNT) ++p.n_eval;
    if (alpha < kAlphaMin) return;
    const float test = __fmul_rn(p.T, __fsub_rn(1.f, alpha));
    if (test < kTStop) { p.done = true; return; }
    if (COUNT) { ++p.n_add; p.n_full += full ? 1ull : 0ull; }
    const float w = __fmul_rn(alpha, p.T);
    p.C0 = __fmaf_rn(Bv.z, w, p.C0);
    p.C1 = __fmaf_rn(Bv.w, w, p.C1);
    p.C2 = __fmaf_rn(sC[j], w, p.C2);
    p.T = test;
    p.last = pos;
}

__device__ __forceinline__ void pix_fwd_store(const PixFwd& p, const CamInfo& cam, int px, int py, float3 bg,
                                              float* __restrict__ image, float* __restrict__ T_final,
                                              int* __restrict__ n_last) {
    if (!(px < cam.W && py < cam.H)) return;
    const long long plane = (long long)cam.W * cam.H;
    const long long pix = (long long)py * cam.W + px;
    float* img = image + 3 * cam.pix_base;
    img[pix] = __fmaf_rn(p.T, bg.x, p.C0);
    img[plane + pix] = __fmaf_rn(p.T, bg.y, p.C1);
    img[2 * plane + pix] = __fmaf_rn(p.T, bg.z, p.C2);
    T_final[cam.pix_base + pix] = p.T;
    n_last[cam.pix_base + pix] = p.last;
}

// One CTA per tile with TILE*TILE/2 threads: warp w owns the 8 x 8 block (w % (TILE/8), w / (TILE/8))
// and each lane the two pixels (x, y) and (x, y + 4) of it.
// COUNT = true is a separate instantiation used only to measure the work of a render (pairs
// evaluated, pairs added, list prefixes); the timed kernels are the COUNT = false instantiations.
template <int TILE, int BATCH, bool COUNT, int CT = TILE>
__global__ void __launch_bounds__(CT* CT / 2) render_fwd_kernel(const dass_splat* __restrict__ splats,
                                                                   const uint32_t* __restrict__ pair_rec,
                                                                   const uint32_t* __restrict__ ranges, CamTable ct,
                                                                   float3 bg, float* __restrict__ image,
                                                                   float* __restrict__ T_final,
                                                                   int* __restrict__ n_last,
                                                                   unsigned long long* __restrict__ work,
                                                                   const uint8_t* __restrict__ full_grad,
                                                                   long long rec_stride) {
    constexpr int NT = CT * CT / 2;
    constexpr int NW = NT / 32;
    constexpr int WX = CT / 8;
    constexpr int S = TILE / CT;      // CTAs per tile side
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ float4 sF[BATCH];
    __shared__ float sC[BATCH];
    __shared__ unsigned short sList[NW][BATCH];
    __shared__ uint8_t sFullC[COUNT ? BATCH : 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile_id = blockIdx.x / (S * S);
    const int sub = blockIdx.x % (S * S);
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int tx0 = (local % cam.tiles_x) * TILE + (sub % S) * CT, ty0 = (local / cam.tiles_x) * TILE + (sub / S) * CT;
    const int bxi = tx0 + (warp % WX) * 8, byi = ty0 + (warp / WX) * 8;
    const int px = bxi + (lane & 7);
    const int py = byi + (lane >> 3);
    const float bx = (float)bxi, by = (float)byi;
    const uint32_t start = ranges[2 * tile_id], end = ranges[2 * tile_id + 1];
    const float fx = (float)px;
    PixFwd p0{(float)py, 1.f, 0.f, 0.f, 0.f, -1, !(px < cam.W && py < cam.H), 0ull, 0ull, 0ull};
    PixFwd p1{(float)(py + 4), 1.f, 0.f, 0.f, 0.f, -1, !(px < cam.W && py + 4 < cam.H), 0ull, 0ull, 0ull};
    for (uint32_t base = start; base < end; base += BATCH) {
        if (__syncthreads_count(p0.done && p1.done) == NT) break;
        const int cnt = min((uint32_t)BATCH, end - base);
        for (int i = tid; i < cnt; i += NT) {
            const uint32_t rec = pair_rec[base + i];
            stage_splat(splats, rec, sA[i], sB[i], sF[i], sC[i]);
            if (COUNT) sFullC[i] = full_grad ? full_grad[rec % (unsigned long long)rec_stride] : (uint8_t)1;
        }
        __syncthreads();
        if (__all_sync(0xffffffffu, p0.done && p1.done)) continue;
        const int nl = warp_compact<8>(sA, sF, cnt, BATCH, bx, by, sList[warp], lane);
        for (int t = 0; t < nl; ++t) {
            if (p0.done && p1.done) break;
            const int j = sList[warp][t];
            const float4 A = sA[j];
            const float4 Bv = sB[j];
            const float dx = __fsub_rn(fx, A.x);
            const bool full = COUNT ? sFullC[COUNT ? j : 0] != 0 : false;
            pix_fwd_step<COUNT>(p0, (int)(base + j), dx, A, Bv, sC, j, full);
            pix_fwd_step<COUNT>(p1, (int)(base + j), dx, A, Bv, sC, j, full);
        }
    }
    pix_fwd_store(p0, cam, px, py, bg, image, T_final, n_last);
    pix_fwd_store(p1, cam, px, py + 4, bg, image, T_final, n_last);
    if (COUNT) {
        unsigned long long n_bwd = (p0.last >= 0 ? (unsigned long long)(p0.last - (int)start + 1) : 0ull) +
                                   (p1.last >= 0 ? (unsigned long long)(p1.last - (int)start + 1) : 0ull);
        atomicAdd(work + 0, p0.n_eval + p1.n_eval);
        atomicAdd(work + 1, p0.n_add + p1.n_add);
        atomicAdd(work + 2, n_bwd);
        atomicAdd(work + 3, (unsigned long long)((px < cam.W && py < cam.H) + (px < cam.W && py + 4 < cam.H)));
        atomicAdd(work + 4, p0.n_full + p1.n_full);
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

// Backward state of one pixel: transmittance behind the current Gaussian, upstream gradient,
// colour behind the current Gaussian (background included) and last added list position.
struct PixBwd {
    float fy, T, g0, g1, g2, R0, R1, R2;
    int last;
};

__device__ __forceinline__ void pix_bwd_load(PixBwd& p, const CamInfo& cam, int px, int py, float3 bg,
                                             const float* __restrict__ T_final, const int* __restrict__ n_last,
                                             const float* __restrict__ dL_dimage) {
    p.fy = (float)py;
    p.T = 1.f; p.g0 = p.g1 = p.g2 = 0.f; p.last = -1;
    p.R0 = bg.x; p.R1 = bg.y; p.R2 = bg.z;
    if (px < cam.W && py < cam.H) {
        const long long plane = (long long)cam.W * cam.H;
        const long long pix = (long long)py * cam.W + px;
        const float* gi = dL_dimage + 3 * cam.pix_base;
        p.g0 = gi[pix];
        p.g1 = gi[plane + pix];
        p.g2 = gi[2 * plane + pix];
        p.T = T_final[cam.pix_base + pix];
        p.last = n_last[cam.pix_base + pix];
    }
}

// Gradient contribution of staged Gaussian (A, Bv, F, blue) at one pixel, added into v[0..7], eb.
__device__ __forceinline__ bool pix_bwd_step(PixBwd& p, long long pos, float dx, const float4 A, const float4 Bv,
                                             const float4 F, float blue, float* v, float& eb) {
    if (pos > (long long)p.last) return false;
    const float dy = __fsub_rn(p.fy, A.y);
    const float G = splat_gauss(A.z, Bv.x, A.w, dx, dy);
    const float alpha = splat_alpha(Bv.y, G);
    if (alpha < kAlphaMin) return false;
    const float om = 1.f - alpha;
    const float Tj = __fdividef(p.T, om);
    const float w = alpha * Tj;
    v[6] += w * p.g0;
    v[7] += w * p.g1;
    eb += w * p.g2;
    const float dLda = Tj * ((Bv.z - p.R0) * p.g0 + (Bv.w - p.R1) * p.g1 + (blue - p.R2) * p.g2);
    p.R0 = Bv.z * alpha + om * p.R0;
    p.R1 = Bv.w * alpha + om * p.R1;
    p.R2 = blue * alpha + om * p.R2;
    p.T = Tj;
    if (Bv.y * G < kAlphaMax) {
        const float dpow = dLda * alpha;
        v[5] += dLda * G;
        v[0] += dpow * (F.x * dx + F.y * dy);
        v[1] += dpow * (F.z * dy + F.y * dx);
        v[2] += -0.5f * dx * dx * dpow;
        v[3] += -dx * dy * dpow;
        v[4] += -0.5f * dy * dy * dpow;
    }
    return true;
}

// The same pixel step when only dL/d(mean2D) of the Gaussian is wanted (its other splat gradients
// are not needed by the caller): transmittance and behind-colour are updated exactly as above,
// and only the two mean2D components are accumulated (su, sv).
__device__ __forceinline__ bool pix_bwd_step_mean(PixBwd& p, long long pos, float dx, const float4 A,
                                                  const float4 Bv, const float4 F, float blue, float& su, float& sv) {
    if (pos > (long long)p.last) return false;
    const float dy = __fsub_rn(p.fy, A.y);
    const float G = splat_gauss(A.z, Bv.x, A.w, dx, dy);
    const float alpha = splat_alpha(Bv.y, G);
    if (alpha < kAlphaMin) return false;
    const float om = 1.f - alpha;
    const float Tj = __fdividef(p.T, om);
    const float dLda = Tj * ((Bv.z - p.R0) * p.g0 + (Bv.w - p.R1) * p.g1 + (blue - p.R2) * p.g2);
    p.R0 = Bv.z * alpha + om * p.R0;
    p.R1 = Bv.w * alpha + om * p.R1;
    p.R2 = blue * alpha + om * p.R2;
    p.T = Tj;
    if (Bv.y * G < kAlphaMax) {
        const float dpow = dLda * alpha;
        su += dpow * (F.x * dx + F.y * dy);
        sv += dpow * (F.z * dy + F.y * dx);
    }
    return true;
}

// Sum two values across the warp: lane 0 ends with the sum of a, lane 16 with the sum of b.
__device__ __forceinline__ float warp_reduce2(float a, float b, int lane) {
    const bool h = lane & 16;
    float r = (h ? b : a) + __shfl_xor_sync(0xffffffffu, h ? a : b, 16);
    r += __shfl_xor_sync(0xffffffffu, r, 8);
    r += __shfl_xor_sync(0xffffffffu, r, 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

// One CTA per tile with TILE*TILE/PPL threads: warp w owns the 8 x 4*PPL block
// (w % (TILE/8), w / (TILE/8)) and each lane the PPL pixels (x, y + 4k), k < PPL, of it, so the
// per-Gaussian warp reduction is shared by 32*PPL pixels. full_grad (optional, per Gaussian of
// the record stride) selects Gaussians whose complete splat gradient is wanted; the others only
// receive dL/d(mean2D).
template <int TILE, int BATCH, int PPL, int CT = TILE>
__global__ void __launch_bounds__(CT* CT / PPL) render_bwd_kernel(
    const dass_splat* __restrict__ splats, const uint32_t* __restrict__ pair_rec, const uint32_t* __restrict__ ranges,
    CamTable ct, float3 bg, const float* __restrict__ T_final, const int* __restrict__ n_last,
    const float* __restrict__ dL_dimage, const uint8_t* __restrict__ full_grad, long long rec_stride,
    dass_splat_grad* __restrict__ gsplat) {
    constexpr int NT = CT * CT / PPL;
    constexpr int NW = NT / 32;
    constexpr int WX = CT / 8;
    constexpr int BH = 4 * PPL;
    constexpr int S = TILE / CT;      // CTAs per tile side
    static_assert(BH <= CT, "warp block taller than the CTA tile");
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ float4 sF[BATCH];
    __shared__ float sC[BATCH];
    __shared__ uint32_t sRec[BATCH];
    __shared__ float sG[BATCH][12];
    __shared__ unsigned short sList[NW][BATCH];
    __shared__ uint8_t sFull[BATCH];
    __shared__ int s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile_id = blockIdx.x / (S * S);
    const int sub = blockIdx.x % (S * S);
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int tx0 = (local % cam.tiles_x) * TILE + (sub % S) * CT, ty0 = (local / cam.tiles_x) * TILE + (sub / S) * CT;
    const int bxi = tx0 + (warp % WX) * 8, byi = ty0 + (warp / WX) * BH;
    const int px = bxi + (lane & 7);
    const int py = byi + (lane >> 3);
    const float bx = (float)bxi, by = (float)byi;
    const uint32_t start = ranges[2 * tile_id];
    const float fx = (float)px;
    PixBwd pp[PPL];
    int mylast = -1;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        pix_bwd_load(pp[k], cam, px, py + 4 * k, bg, T_final, n_last, dL_dimage);
        mylast = max(mylast, pp[k].last);
    }
    if (tid == 0) s_maxlast = -1;
    __syncthreads();
    const int wlast = __reduce_max_sync(0xffffffffu, mylast);
    if (lane == 0 && wlast >= 0) atomicMax(&s_maxlast, wlast);
    __syncthreads();
    const long long endpos = (long long)s_maxlast + 1;
    for (long long hi = endpos; hi > (long long)start; hi -= BATCH) {
        const long long lo = hi - BATCH > (long long)start ? hi - BATCH : (long long)start;
        const int cnt = (int)(hi - lo);
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            uint32_t rec = pair_rec[lo + i];
            sRec[i] = rec;
            sFull[i] = full_grad ? full_grad[rec % (unsigned long long)rec_stride] : (uint8_t)1;
            stage_splat(splats, rec, sA[i], sB[i], sF[i], sC[i]);
#pragma unroll
            for (int k = 0; k < 12; ++k) sG[i][k] = 0.f;
        }
        __syncthreads();
        const int jmax = (int)((long long)wlast - lo);   // entries beyond every lane's last are skipped
        const int nl = jmax >= 0 ? warp_compact<BH>(sA, sF, cnt, jmax, bx, by, sList[warp], lane) : 0;
        for (int t = nl - 1; t >= 0; --t) {
            const int j = sList[warp][t];
            const long long pos = lo + j;
            const float4 A = sA[j];
            const float4 Bv = sB[j];
            const float4 F = sF[j];
            const float blue = sC[j];
            const float dx = __fsub_rn(fx, A.x);
            bool contrib = false;
            if (sFull[j]) {          // warp-uniform: the same Gaussian for every lane
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float eb = 0.f;
#pragma unroll
                for (int k = 0; k < PPL; ++k) contrib |= pix_bwd_step(pp[k], pos, dx, A, Bv, F, blue, v, eb);
                if (__ballot_sync(0xffffffffu, contrib)) {
                    float r = warp_reduce8(v, lane);
                    float e = warp_sum(eb);
                    if ((lane & 3) == 0) {
                        int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                        atomicAdd(&sG[j][idx], r);
                    }
                    if (lane == 1) atomicAdd(&sG[j][8], e);
                }
            } else {
                float su = 0.f, sv = 0.f;
#pragma unroll
                for (int k = 0; k < PPL; ++k) contrib |= pix_bwd_step_mean(pp[k], pos, dx, A, Bv, F, blue, su, sv);
                if (__ballot_sync(0xffffffffu, contrib)) {
                    float r = warp_reduce2(su, sv, lane);
                    if ((lane & 15) == 0) atomicAdd(&sG[j][lane >> 4], r);
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            float4 a = make_float4(sG[i][0], sG[i][1], sG[i][2], sG[i][3]);
            float4 b = make_float4(sG[i][4], sG[i][5], sG[i][6], sG[i][7]);
            float c = sG[i][8];
            float4* dst = reinterpret_cast<float4*>(gsplat + sRec[i]);
            if ((a.x != 0.f) | (a.y != 0.f) | (a.z != 0.f) | (a.w != 0.f)) atomicAdd(dst, a);
            if ((b.x != 0.f) | (b.y != 0.f) | (b.z != 0.f) | (b.w != 0.f)) atomicAdd(dst + 1, b);
            if (c != 0.f) atomicAdd(reinterpret_cast<float*>(dst + 2), c);
        }
    }
}

// CTA side of the compositing kernels for a binning tile: a tile's list can be composited by
// (TILE/CT)^2 independent CTAs, each covering a CT x CT part of the tile. Measured on the 300k x
// 20-view workload: 32-pixel bins are composited fastest by 16 x 16 forward CTAs (fewer warps
// wait at each staged batch) and by whole-tile backward CTAs.
template <int TILE>
constexpr int fwd_cta() { return TILE == 32 ? 16 : TILE; }
template <int TILE>
constexpr int bwd_cta() { return TILE; }

template <int TILE, int BATCH>
int launch_fwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               float* img, float* tf, int* nl, unsigned long long* work, const uint8_t* full, long long stride,
               cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    constexpr int CT = fwd_cta<TILE>();
    constexpr int NB = (TILE / CT) * (TILE / CT);
    if (work)
        render_fwd_kernel<TILE, BATCH, true, CT><<<ct.tiles_total * NB, CT * CT / 2, 0, st>>>(sp, pr, rg, ct, bg, img,
                                                                                             tf, nl, work, full, stride);
    else
        render_fwd_kernel<TILE, BATCH, false, CT><<<ct.tiles_total * NB, CT * CT / 2, 0, st>>>(
            sp, pr, rg, ct, bg, img, tf, nl, nullptr, nullptr, 1);
    count_launch();
    return check_launch("render_fwd_kernel");
}

// Pixels per lane of the backward (measured on the 300k x 20-view workload): 2 for 8- and
// 16-pixel tiles (8 x 8 warp blocks), 4 for 32-pixel tiles (8 x 16).
template <int TILE>
constexpr int bwd_ppl() { return TILE == 32 ? 4 : 2; }

template <int TILE, int BATCH>
int launch_bwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               const float* tf, const int* nl, const float* dimg, const uint8_t* full, long long stride,
               dass_splat_grad* gs, cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    constexpr int PPL = bwd_ppl<TILE>();
    constexpr int CT = bwd_cta<TILE>();
    constexpr int NB = (TILE / CT) * (TILE / CT);
    render_bwd_kernel<TILE, BATCH, PPL, CT><<<ct.tiles_total * NB, CT * CT / PPL, 0, st>>>(sp, pr, rg, ct, bg, tf, nl,
                                                                                          dimg, full, stride, gs);
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
                      unsigned long long* work, const uint8_t* full_grad, long long rec_stride) {
    DASS_DISPATCH(launch_fwd, splats, pair_rec, ranges, ct, bg, image, T_final, n_last, work, full_grad, rec_stride,
                  st)
}

int render_bwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, const float* T_final, const int* n_last, const float* dL_dimage,
                      const uint8_t* full_grad, long long rec_stride, dass_splat_grad* gsplat, cudaStream_t st) {
    DASS_DISPATCH(launch_bwd, splats, pair_rec, ranges, ct, bg, T_final, n_last, dL_dimage, full_grad, rec_stride,
                  gsplat, st)
}

}  // namespace dass
