// Forward and backward alpha compositing (App. A.1) over every tile of every camera in one
// launch. A CTA covers a CT x CT part of a binning tile; each warp owns an 8 x 4*PPL block of
// pixels and each lane PPL pixels of one column (rows y + 4k), handled as pixel pairs with the
// packed FP32x2 arithmetic of sm_100+ (two-lane add/mul/fma that round like their scalar forms,
// so the packed alpha is bit-identical to a scalar evaluation). The tile's depth-sorted
// Gaussians are staged through shared memory in batches; after each batch is staged, every
// warp compacts (ballot + prefix popcount, order preserved) the entries whose alpha >= 1/255
// footprint ellipse reaches its own block of pixels, and composites only those. The backward
// walks the lists in reverse from the last contributor, recomputing alpha and
// T_j = T_{j+1}/(1-alpha_j) from the saved T_final, and reduces per-Gaussian gradients
// warp-wide (shuffles), then block-wide (shared-memory atomics), then into global memory
// (vector atomics).
#include "common.cuh"

namespace dass {

namespace {

// Staged form of a splat: NG float4 groups in structure-of-arrays shared memory. Every scalar
// of the per-pixel math is stored twice, so one shared load yields the operand pair of the
// packed arithmetic without register moves:
//   P0 = (-u, -u, -v, -v)     P1 = (a', a', b2', b2')     P2 = (c', c', o, o)
//   P3 = (r, r, g, g)         P4 = (blue, blue, 0, 0)
// with a' = a kNegHalfLog2e, b2' = 2 b kNegHalfLog2e, c' = c kNegHalfLog2e (see splat_gauss);
// F = (a, b, c, k2) is the footprint ellipse d^T conic d <= k2 (k2 < 0: no footprint).
// NEG (forward only): o, r, g and blue are staged negated, so that the forward works with -alpha
// and forms T - alpha T with one packed FMA (the negations are exact: alpha is unchanged).
template <int NG, int BATCH, bool NEG = false>
__device__ __forceinline__ void stage_splat(const dass_splat* __restrict__ splats, uint32_t rec, int i,
                                            float4 (&sP)[NG][BATCH], float4 (&sF)[BATCH]) {
    const float4* sp = reinterpret_cast<const float4*>(splats + rec);
    const float4 s0 = __ldg(sp);        // u, v, a, b
    const float4 s1 = __ldg(sp + 1);    // c, o, r, g
    const float bl = __ldg(reinterpret_cast<const float*>(sp + 2));
    const float ap = __fmul_rn(s0.z, kNegHalfLog2e), b2p = __fmul_rn(2.f * s0.w, kNegHalfLog2e),
                cp = __fmul_rn(s1.x, kNegHalfLog2e);
    const float sg = NEG ? -1.f : 1.f;
    sP[0][i] = make_float4(-s0.x, -s0.x, -s0.y, -s0.y);
    sP[1][i] = make_float4(ap, ap, b2p, b2p);
    sP[2][i] = make_float4(cp, cp, sg * s1.y, sg * s1.y);
    sP[3][i] = make_float4(sg * s1.z, sg * s1.z, sg * s1.w, sg * s1.w);
    sP[4][i] = make_float4(sg * bl, sg * bl, 0.f, 0.f);
    sF[i] = make_float4(s0.z, s0.w, s1.x, footprint_k2(s0.z, s0.w, s1.x, s1.y));
}

__device__ __forceinline__ float2 lo2(const float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 v) { return make_float2(v.z, v.w); }

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Compact the indices [0, cnt) of the staged batch whose footprint reaches this warp's 8 x BH
// block into list[] (ascending), only indices <= jmax. Returns the count (warp-uniform).
template <int BH, int BATCH>
__device__ __forceinline__ int warp_compact(const float4* __restrict__ sP0, const float4* __restrict__ sF, int cnt,
                                            int jmax, float bx, float by, unsigned short* list, int lane) {
    int n = 0;
    int lim = min(cnt, jmax + 1);
    for (int j0 = 0; j0 < lim; j0 += 32) {
        int j = j0 + lane;
        bool hit = false;
        if (j < lim) {
            const float4 c = sP0[j];
            hit = footprint_reaches_rect(c.x, c.z, sF[j], bx, by, 7.f, (float)(BH - 1));
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[n + __popc(m & lanemask_lt())] = (unsigned short)j;
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

// Forward state of a lane's pixel pair (rows y and y + 4 of one column).
struct PixFwd2 {
    float2 fy, T, C0, C1, C2;
    int last0, last1;
    bool done0, done1;
    unsigned long long n_eval, n_add, n_full;
};

// Front-to-back step of staged entry P0..P4 (list position pos) for both pixels: skip alpha <
// 1/255, stop before T (1 - alpha) < 1e-4, else blend. The entry is staged negated (o, r, g,
// blue), so the step carries na = -alpha and forms T - alpha T = fma(na, T, T) in one rounding. A
// pixel that skips or is done gets alpha = 0 in the packed blend, which leaves its colour and
// transmittance exactly unchanged.
template <bool COUNT>
__device__ __forceinline__ void pix_fwd_step2(PixFwd2& p, int pos, float2 A, float2 B, const float4 P0,
                                              const float4 P2, const float4 P3, float2 nblue, bool full) {
    const float2 dy = __fadd2_rn(p.fy, hi2(P0));
    const float2 G = splat_gauss2(lo2(P2), dy, A, B);
    const float2 noG = __fmul2_rn(hi2(P2), G);                 // -o G
    float2 na = make_float2(fmaxf(-kAlphaMax, noG.x), fmaxf(-kAlphaMax, noG.y));
    const float2 test = __ffma2_rn(na, p.T, p.T);
    bool ok0 = !p.done0 && !(na.x > -kAlphaMin);
    bool ok1 = !p.done1 && !(na.y > -kAlphaMin);
    if (COUNT) p.n_eval += (unsigned long long)(!p.done0) + (unsigned long long)(!p.done1);
    const bool stop0 = ok0 && test.x < kTStop, stop1 = ok1 && test.y < kTStop;
    p.done0 = p.done0 || stop0;
    p.done1 = p.done1 || stop1;
    ok0 = ok0 && !stop0;
    ok1 = ok1 && !stop1;
    if (COUNT) {
        const unsigned long long k = (unsigned long long)ok0 + (unsigned long long)ok1;
        p.n_add += k;
        p.n_full += full ? k : 0ull;
    }
    na.x = ok0 ? na.x : 0.f;
    na.y = ok1 ? na.y : 0.f;
    const float2 nw = __fmul2_rn(na, p.T);                     // -alpha T
    p.C0 = __ffma2_rn(lo2(P3), nw, p.C0);                      // (-r)(-alpha T)
    p.C1 = __ffma2_rn(hi2(P3), nw, p.C1);
    p.C2 = __ffma2_rn(nblue, nw, p.C2);
    p.T = __ffma2_rn(na, p.T, p.T);     // = test where the pixel blends, T where alpha = 0
    p.last0 = ok0 ? pos : p.last0;
    p.last1 = ok1 ? pos : p.last1;
}

__device__ __forceinline__ void pix_fwd_store(float T, float C0, float C1, float C2, int last, const CamInfo& cam,
                                              int px, int py, float3 bg, float* __restrict__ image,
                                              float* __restrict__ T_final, int* __restrict__ n_last) {
    if (!(px < cam.W && py < cam.H)) return;
    const long long plane = (long long)cam.W * cam.H;
    const long long pix = (long long)py * cam.W + px;
    float* img = image + 3 * cam.pix_base;
    img[pix] = __fmaf_rn(T, bg.x, C0);
    img[plane + pix] = __fmaf_rn(T, bg.y, C1);
    img[2 * plane + pix] = __fmaf_rn(T, bg.z, C2);
    T_final[cam.pix_base + pix] = T;
    n_last[cam.pix_base + pix] = last;
}

// One CTA per CT x CT part of a tile with CT*CT/PPL threads: warp w owns the 8 x 4*PPL block
// (w % (CT/8), w / (CT/8)) and each lane the PPL pixels (x, y + 4k), k < PPL, of it, as PPL/2
// packed pixel pairs. COUNT = true is a separate instantiation used only to measure the work of a
// render (pairs evaluated, pairs added, list prefixes); the timed kernels are the COUNT = false
// instantiations.
template <int TILE, int BATCH, bool COUNT, int CT = TILE, int PPL = 2>
__global__ void __launch_bounds__(CT* CT / PPL) render_fwd_kernel(const dass_splat* __restrict__ splats,
                                                                     const uint32_t* __restrict__ pair_rec,
                                                                     const uint32_t* __restrict__ ranges,
                                                                     CamTable ct, float3 bg,
                                                                     float* __restrict__ image,
                                                                     float* __restrict__ T_final,
                                                                     int* __restrict__ n_last,
                                                                     unsigned long long* __restrict__ work,
                                                                     const uint8_t* __restrict__ full_grad,
                                                                     long long rec_stride) {
    constexpr int NT = CT * CT / PPL;
    constexpr int NW = NT / 32;
    constexpr int WX = CT / 8;
    constexpr int BH = 4 * PPL;
    constexpr int NP = PPL / 2;       // pixel pairs per lane
    constexpr int S = TILE / CT;      // CTAs per tile side
    static_assert(BH <= CT && PPL % 2 == 0, "warp block taller than the CTA tile, or odd pixels per lane");
    __shared__ float4 sP[5][BATCH];
    __shared__ float4 sF[BATCH];
    __shared__ unsigned short sList[NW][BATCH];
    __shared__ uint8_t sFullC[COUNT ? BATCH : 1];
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
    const uint32_t start = ranges[2 * tile_id], end = ranges[2 * tile_id + 1];
    const float2 fx2 = make_float2((float)px, (float)px);
    PixFwd2 pp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int y0 = py + 8 * k;
        pp[k].fy = make_float2((float)y0, (float)(y0 + 4));
        pp[k].T = make_float2(1.f, 1.f);
        pp[k].C0 = pp[k].C1 = pp[k].C2 = make_float2(0.f, 0.f);
        pp[k].last0 = pp[k].last1 = -1;
        pp[k].done0 = !(px < cam.W && y0 < cam.H);
        pp[k].done1 = !(px < cam.W && y0 + 4 < cam.H);
        pp[k].n_eval = pp[k].n_add = pp[k].n_full = 0ull;
    }
    auto all_done = [&]() {
        bool d = true;
#pragma unroll
        for (int k = 0; k < NP; ++k) d = d && pp[k].done0 && pp[k].done1;
        return d;
    };
    for (uint32_t base = start; base < end; base += BATCH) {
        if (__syncthreads_count(all_done()) == NT) break;
        const int cnt = min((uint32_t)BATCH, end - base);
        for (int i = tid; i < cnt; i += NT) {
            const uint32_t rec = pair_rec[base + i];
            stage_splat<5, BATCH, true>(splats, rec, i, sP, sF);
            if (COUNT) sFullC[i] = full_grad ? full_grad[rec % (unsigned long long)rec_stride] : (uint8_t)1;
        }
        __syncthreads();
        if (__all_sync(0xffffffffu, all_done())) continue;
        const int nl = warp_compact<BH, BATCH>(sP[0], sF, cnt, BATCH, bx, by, sList[warp], lane);
#pragma unroll 8
        for (int t = 0; t < nl; ++t) {
            // warp-uniform early exit, tested every 4 entries (pixels that are done blend alpha = 0)
            if ((t & 3) == 0 && __all_sync(0xffffffffu, all_done())) break;
            const int j = sList[warp][t];
            const float4 P0 = sP[0][j], P1 = sP[1][j], P2 = sP[2][j], P3 = sP[3][j];
            const float2 nblue = lo2(sP[4][j]);
            const float2 dx = __fadd2_rn(fx2, lo2(P0));
            float2 A, B;
            splat_column2(lo2(P1), hi2(P1), dx, A, B);
            const bool full = COUNT ? sFullC[COUNT ? j : 0] != 0 : false;
#pragma unroll
            for (int k = 0; k < NP; ++k) pix_fwd_step2<COUNT>(pp[k], (int)(base + j), A, B, P0, P2, P3, nblue, full);
        }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const PixFwd2& p = pp[k];
        const int y0 = py + 8 * k;
        pix_fwd_store(p.T.x, p.C0.x, p.C1.x, p.C2.x, p.last0, cam, px, y0, bg, image, T_final, n_last);
        pix_fwd_store(p.T.y, p.C0.y, p.C1.y, p.C2.y, p.last1, cam, px, y0 + 4, bg, image, T_final, n_last);
        if (COUNT) {
            unsigned long long n_bwd = (p.last0 >= 0 ? (unsigned long long)(p.last0 - (int)start + 1) : 0ull) +
                                       (p.last1 >= 0 ? (unsigned long long)(p.last1 - (int)start + 1) : 0ull);
            atomicAdd(work + 0, p.n_eval);
            atomicAdd(work + 1, p.n_add);
            atomicAdd(work + 2, n_bwd);
            atomicAdd(work + 3,
                      (unsigned long long)((px < cam.W && y0 < cam.H) + (px < cam.W && y0 + 4 < cam.H)));
            atomicAdd(work + 4, p.n_full);
        }
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

// Sum four values across the warp with a transposed butterfly (2+1+1+1+1 shuffles). Lane l with
// (l & 7) == 0 ends with the full sum of value index ((l >> 4) & 1) * 2 + ((l >> 3) & 1).
__device__ __forceinline__ float warp_reduce4(float v0, float v1, float v2, float v3, int lane) {
    const bool h4 = lane & 16;
    const float a = (h4 ? v2 : v0) + __shfl_xor_sync(0xffffffffu, h4 ? v0 : v2, 16);
    const float b = (h4 ? v3 : v1) + __shfl_xor_sync(0xffffffffu, h4 ? v1 : v3, 16);
    const bool h3 = lane & 8;
    float r = (h3 ? b : a) + __shfl_xor_sync(0xffffffffu, h3 ? a : b, 8);
    r += __shfl_xor_sync(0xffffffffu, r, 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
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

// Backward state of a lane's pixel pair: transmittance behind the current Gaussian, upstream
// gradient g = dL/dC, S = g . R with R the colour behind the current Gaussian (background
// included), last added list position. dL/dalpha_j only needs R through g . R, and R's recurrence
// R_j = alpha_j c_j + (1 - alpha_j) R_{j+1} carries over to S_j = alpha_j (g . c_j) + (1 - alpha_j) S_{j+1},
// so one scalar replaces the three channels.
struct PixBwd2 {
    float2 fy, T, S;
    int last0, last1;
};

__device__ __forceinline__ void pix_bwd_load1(const CamInfo& cam, int px, int py, const float* __restrict__ T_final,
                                              const int* __restrict__ n_last, const float* __restrict__ dL_dimage,
                                              float& T, float& g0, float& g1, float& g2, int& last) {
    T = 1.f; g0 = g1 = g2 = 0.f; last = -1;
    if (px < cam.W && py < cam.H) {
        const long long plane = (long long)cam.W * cam.H;
        const long long pix = (long long)py * cam.W + px;
        const float* gi = dL_dimage + 3 * cam.pix_base;
        g0 = gi[pix];
        g1 = gi[plane + pix];
        g2 = gi[2 * plane + pix];
        T = T_final[cam.pix_base + pix];
        last = n_last[cam.pix_base + pix];
    }
}

// Loads the pair's state; its upstream gradient goes to shared memory, gp[0], gp[NT], gp[2 NT]
// (per-thread slots, read back at every step instead of being held in registers).
template <int NT>
__device__ __forceinline__ void pix_bwd_load2(PixBwd2& p, float2* gp, const CamInfo& cam, int px, int py, float3 bg,
                                              const float* __restrict__ T_final, const int* __restrict__ n_last,
                                              const float* __restrict__ dL_dimage) {
    float2 g0, g1, g2;
    p.fy = make_float2((float)py, (float)(py + 4));
    pix_bwd_load1(cam, px, py, T_final, n_last, dL_dimage, p.T.x, g0.x, g1.x, g2.x, p.last0);
    pix_bwd_load1(cam, px, py + 4, T_final, n_last, dL_dimage, p.T.y, g0.y, g1.y, g2.y, p.last1);
    p.S = __ffma2_rn(g2, make_float2(bg.z, bg.z),
                     __ffma2_rn(g1, make_float2(bg.y, bg.y), __fmul2_rn(g0, make_float2(bg.x, bg.x))));
    gp[0] = g0;
    gp[NT] = g1;
    gp[2 * NT] = g2;
}

// Reverse step of staged entry P0..P4 (list position pos) for both pixels of the pair; adds the
// entry's gradient contributions: vm[0..1] (packed, both pixels) the sums of dx and dy times
// dL/d(power) -- dL/d(u, v) = (a X + b Y, b X + c Y) of those sums X, Y, applied once per
// staged Gaussian when the CTA's block sums are flushed, since the conic is the Gaussian's. If
// FULL, the lane's shared dx is factored out: vm[0] holds sum dL/d(power) (X = dx vm[0], and the
// dx^2 moment dx X), vm[1] the dy moment Y (the dx dy moment is dx Y), vf[2] the dy^2 moment --
// the three second moments give dL/d(a, b, c) after scaling by -1/2, -1, -1/2 -- and vf[3]
// dL/do, vf[4..6] dL/d(r, g, blue). A pixel whose list ends before pos, or where alpha <
// 1/255, takes alpha = 0, which leaves its T and R exactly unchanged and adds nothing. The step is
// branch-free (no early exit when neither pixel takes part: under SIMT the warp runs the body
// whenever any lane needs it, and the divergent exits cost more than the masked work; measured
// 5.95 -> 5.31 ms on the 300k x 20-view backward). Returns whether either pixel took part.
template <bool FULL, int NT>
__device__ __forceinline__ bool pix_bwd_step2(PixBwd2& p, const float2* gp, int pos, float2 dx, float2 A, float2 B,
                                              const float4 P0, const float4 P2, const float4 P3, const float4 P4,
                                              float2* vm, float2* vf) {
    bool val0 = pos <= p.last0, val1 = pos <= p.last1;
    const float2 dy = __fadd2_rn(p.fy, hi2(P0));
    const float2 G = splat_gauss2(lo2(P2), dy, A, B);
    const float2 oG = __fmul2_rn(hi2(P2), G);
    const float2 alpha = make_float2(fminf(kAlphaMax, oG.x), fminf(kAlphaMax, oG.y));
    val0 = val0 && !(alpha.x < kAlphaMin);
    val1 = val1 && !(alpha.y < kAlphaMin);
    const float2 am = make_float2(val0 ? alpha.x : 0.f, val1 ? alpha.y : 0.f);
    const float2 om = one_minus2(am);
    // a pixel that takes no part has om = 1 exactly, and rcp.approx(1) = 1 exactly (checked on
    // sm_103), so its T passes through unchanged without a select
    const float2 Tj = __fmul2_rn(p.T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
    const float2 g0 = gp[0], g1 = gp[NT], g2 = gp[2 * NT];
    const float2 gc = __ffma2_rn(lo2(P4), g2, __ffma2_rn(hi2(P3), g1, __fmul2_rn(lo2(P3), g0)));
    const float2 d = sub2(gc, p.S);
    const float2 dLda = __fmul2_rn(Tj, d);
    p.S = __ffma2_rn(am, d, p.S);       // alpha gc + (1 - alpha) S = S + alpha (gc - S)
    p.T = Tj;
    // the clamp alpha = 0.99 has zero derivative
    const bool cm0 = val0 && oG.x < kAlphaMax, cm1 = val1 && oG.y < kAlphaMax;
    const float2 dpow = __fmul2_rn(dLda, make_float2(cm0 ? alpha.x : 0.f, cm1 ? alpha.y : 0.f));
    if (FULL) {
        // a lane's pixels share dx: vm[0] collects sum dpow (times dx, and dx^2, once per entry)
        // and vm[1], vf[2] the sums of dpow dy and dpow dy^2; sum dpow dx dy = dx sum dpow dy
        vm[0] = __fadd2_rn(vm[0], dpow);
        const float2 t = __fmul2_rn(dpow, dy);
        vm[1] = __fadd2_rn(vm[1], t);
        vf[2] = __ffma2_rn(t, dy, vf[2]);
        vf[3] = __ffma2_rn(dLda, make_float2(cm0 ? G.x : 0.f, cm1 ? G.y : 0.f), vf[3]);
        const float2 w = __fmul2_rn(am, Tj);
        vf[4] = __ffma2_rn(w, g0, vf[4]);
        vf[5] = __ffma2_rn(w, g1, vf[5]);
        vf[6] = __ffma2_rn(w, g2, vf[6]);
    } else {
        vm[0] = __ffma2_rn(dpow, dx, vm[0]);
        vm[1] = __ffma2_rn(dpow, dy, vm[1]);
    }
    return val0 || val1;
}

// Dynamic shared-memory layout of the backward CTA (byte offsets; every part 16-byte aligned).
template <int BATCH, int NT, int NP>
struct BwdSmem {
    static constexpr int kP = 0;                                  // float4 [5][BATCH] staged splats
    static constexpr int kF = kP + 5 * BATCH * 16;                // float4 [BATCH] footprints
    static constexpr int kGp = kF + BATCH * 16;                   // float2 [NP][3][NT] dL/dC of the lanes' pixels
    static constexpr int kG = kGp + NP * 3 * NT * 8;              // float [BATCH][9] block-reduced gradients
    static constexpr int kRec = kG + ((BATCH * 9 * 4 + 15) / 16) * 16;   // uint32 [BATCH] record indices
    static constexpr int kList = kRec + BATCH * 4;                // ushort [NT/32][BATCH] per-warp lists
    static constexpr int kFull = kList + ((NT / 32) * BATCH * 2 + 15) / 16 * 16;   // uint8 [BATCH]
    static constexpr int kBytes = kFull + ((BATCH + 15) / 16) * 16;
};

// One CTA per CT x CT part of a tile with CT*CT/PPL threads: warp w owns the 8 x 4*PPL block
// (w % (CT/8), w / (CT/8)) and each lane the PPL pixels (x, y + 4k), k < PPL, of it, so the
// per-Gaussian warp reduction is shared by 32*PPL pixels. full_grad (optional, per Gaussian of
// the record stride) selects Gaussians whose complete splat gradient is wanted; the others only
// receive dL/d(mean2D). With 4 pixels per lane the kernel is held to 64 registers (no spills) so
// that four 256-thread CTAs share an SM (the upstream gradients live in shared memory for that
// reason): warps waiting at a CTA's batch barrier leave issue slots to the other CTAs. Measured
// on the 300k x 20-view backward: 3 CTAs per SM (80 registers) 5.31 ms, 4 CTAs 5.06 ms.
template <int TILE, int BATCH, int PPL, int CT = TILE>
__global__ void __launch_bounds__(CT* CT / PPL, PPL == 4 ? 4 : 1) render_bwd_kernel(
    const dass_splat* __restrict__ splats, const uint32_t* __restrict__ pair_rec, const uint32_t* __restrict__ ranges,
    CamTable ct, float3 bg, const float* __restrict__ T_final, const int* __restrict__ n_last,
    const float* __restrict__ dL_dimage, const uint8_t* __restrict__ full_grad, long long rec_stride,
    dass_splat_grad* __restrict__ gsplat) {
    constexpr int NT = CT * CT / PPL;
    constexpr int NW = NT / 32;
    constexpr int WX = CT / 8;
    constexpr int BH = 4 * PPL;
    constexpr int NP = PPL / 2;       // pixel pairs per lane
    constexpr int S = TILE / CT;      // CTAs per tile side
    static_assert(BH <= CT && PPL % 2 == 0, "warp block taller than the CTA tile, or odd pixels per lane");
    using L = BwdSmem<BATCH, NT, NP>;
    extern __shared__ __align__(16) unsigned char smem[];
    auto& sP = *reinterpret_cast<float4(*)[5][BATCH]>(smem + L::kP);
    auto& sF = *reinterpret_cast<float4(*)[BATCH]>(smem + L::kF);
    float2* sGp = reinterpret_cast<float2*>(smem + L::kGp);        // [NP][3][NT] upstream gradients
    auto& sG = *reinterpret_cast<float(*)[BATCH][9]>(smem + L::kG);
    uint32_t* sRec = reinterpret_cast<uint32_t*>(smem + L::kRec);
    auto& sList = *reinterpret_cast<unsigned short(*)[NW][BATCH]>(smem + L::kList);
    uint8_t* sFull = smem + L::kFull;
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
    const float2 fx2 = make_float2((float)px, (float)px);
    const uint32_t stride = (uint32_t)rec_stride;
    // the reduced dx^2, dx dy, dy^2 sums become dL/d(a, b, c) after this lane-constant scale
    const int gidx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    const float gscale = gidx == 3 ? -1.f : (gidx == 2 || gidx == 4) ? -0.5f : 1.f;
    PixBwd2 pp[NP];
    int mylast = -1;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        pix_bwd_load2<NT>(pp[k], sGp + 3 * NT * k + tid, cam, px, py + 8 * k, bg, T_final, n_last, dL_dimage);
        mylast = max(mylast, max(pp[k].last0, pp[k].last1));
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
            const uint32_t rec = pair_rec[lo + i];
            sRec[i] = rec;
            sFull[i] = full_grad ? full_grad[rec % stride] : (uint8_t)1;
            stage_splat<5, BATCH>(splats, rec, i, sP, sF);
#pragma unroll
            for (int k = 0; k < 9; ++k) sG[i][k] = 0.f;
        }
        __syncthreads();
        const int jmax = (int)((long long)wlast - lo);   // entries beyond every lane's last are skipped
        const int nl = jmax >= 0 ? warp_compact<BH, BATCH>(sP[0], sF, cnt, jmax, bx, by, sList[warp], lane) : 0;
        // reverse pair steps of the mean-only entry j (dL/dmean2D moments into vm); returns whether a
        // pixel of this lane took part
        auto mean_steps = [&](int j, float2* vm) {
            const int pos = (int)(lo + j);
            const float4 P0 = sP[0][j], P1 = sP[1][j], P2 = sP[2][j], P3 = sP[3][j], P4 = sP[4][j];
            const float2 dx = __fadd2_rn(fx2, lo2(P0));
            float2 A, B;
            splat_column2(lo2(P1), hi2(P1), dx, A, B);
            bool c = false;
#pragma unroll
            for (int k = 0; k < NP; ++k)
                c |= pix_bwd_step2<false, NT>(pp[k], sGp + 3 * NT * k + tid, pos, dx, A, B, P0, P2, P3, P4, vm,
                                              nullptr);
            return c;
        };
        for (int t = nl - 1; t >= 0; --t) {
            const int j = sList[warp][t];
            bool contrib = false;
            float2 vm[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (sFull[j]) {          // warp-uniform: the same Gaussian for every lane
                const int pos = (int)(lo + j);
                const float4 P0 = sP[0][j], P1 = sP[1][j], P2 = sP[2][j], P3 = sP[3][j], P4 = sP[4][j];
                const float2 dx = __fadd2_rn(fx2, lo2(P0));
                float2 A, B;
                splat_column2(lo2(P1), hi2(P1), dx, A, B);
                float2 vf[7];      // vf[0], vf[1] unused: formed from vm below
#pragma unroll
                for (int i = 0; i < 7; ++i) vf[i] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    contrib |= pix_bwd_step2<true, NT>(pp[k], sGp + 3 * NT * k + tid, pos, dx, A, B, P0, P2, P3, P4,
                                                       vm, vf);
                if (__ballot_sync(0xffffffffu, contrib)) {
                    const float X = dx.x * (vm[0].x + vm[0].y), Y = vm[1].x + vm[1].y;
                    float r[8] = {X, Y, dx.x * X, dx.x * Y, vf[2].x + vf[2].y, vf[3].x + vf[3].y,
                                  vf[4].x + vf[4].y, vf[5].x + vf[5].y};
                    float s = warp_reduce8(r, lane);
                    const float e = warp_sum(vf[6].x + vf[6].y);
                    // lanes 0 and 4 hold the moments X and Y (the conic is applied at the flush)
                    if ((lane & 3) == 0) atomicAdd(&sG[j][gidx], s * gscale);
                    if (lane == 1) atomicAdd(&sG[j][8], e);
                }
            } else {
                // mean-only entries are taken two at a time when the next one is mean-only too
                // (warp-uniform), so that one 4-value reduction serves both
                const int j2 = t >= 1 ? sList[warp][t - 1] : 0;
                const bool two = t >= 1 && !sFull[j2];
                contrib = mean_steps(j, vm);
                float2 vm2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                if (two) {
                    contrib |= mean_steps(j2, vm2);
                    --t;
                }
                if (__ballot_sync(0xffffffffu, contrib)) {
                    if (two) {
                        const float r = warp_reduce4(vm[0].x + vm[0].y, vm[1].x + vm[1].y, vm2[0].x + vm2[0].y,
                                                     vm2[1].x + vm2[1].y, lane);
                        // lanes 0, 8 hold X, Y of j; lanes 16, 24 those of j2 (conic at the flush)
                        if ((lane & 7) == 0) atomicAdd(&sG[(lane & 16) ? j2 : j][(lane >> 3) & 1], r);
                    } else {
                        const float r = warp_reduce2(vm[0].x + vm[0].y, vm[1].x + vm[1].y, lane);
                        // lane 0 holds X, lane 16 holds Y (the conic is applied at the flush)
                        if ((lane & 15) == 0) atomicAdd(&sG[j][lane >> 4], r);
                    }
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            // block sums X = sum dpow dx, Y = sum dpow dy -> dL/du = a X + b Y, dL/dv = b X + c Y
            const float4 F = sF[i];
            const float X = sG[i][0], Y = sG[i][1];
            float4 a = make_float4(F.x * X + F.y * Y, F.y * X + F.z * Y, sG[i][2], sG[i][3]);
            float4 b = make_float4(sG[i][4], sG[i][5], sG[i][6], sG[i][7]);
            float c = sG[i][8];
            float4* dst = reinterpret_cast<float4*>(gsplat + sRec[i]);
            if ((a.x != 0.f) | (a.y != 0.f) | (a.z != 0.f) | (a.w != 0.f)) atomicAdd(dst, a);
            if ((b.x != 0.f) | (b.y != 0.f) | (b.z != 0.f) | (b.w != 0.f)) atomicAdd(dst + 1, b);
            if (c != 0.f) atomicAdd(reinterpret_cast<float*>(dst + 2), c);
        }
    }
}

// CTA side and pixels per lane of the compositing kernels for a binning tile: a tile's list can
// be composited by (TILE/CT)^2 independent CTAs, each covering a CT x CT part of the tile, and a
// lane owns PPL pixels of a column. Measured on the 300k x 20-view workload: 32-pixel bins are
// composited fastest by whole-tile CTAs with 4 pixels per lane (8 x 16 warp blocks) in both
// passes; 16 x 16 forward CTAs were best with 2 pixels per lane (2.76 vs 2.69 ms).
template <int TILE>
constexpr int fwd_cta() { return TILE; }
template <int TILE>
constexpr int fwd_ppl() { return TILE == 32 ? 4 : 2; }
template <int TILE>
constexpr int bwd_cta() { return TILE; }

template <int TILE, int BATCH>
int launch_fwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               float* img, float* tf, int* nl, unsigned long long* work, const uint8_t* full, long long stride,
               cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    constexpr int CT = fwd_cta<TILE>();
    constexpr int PPL = fwd_ppl<TILE>();
    constexpr int NB = (TILE / CT) * (TILE / CT);
    if (work)
        render_fwd_kernel<TILE, BATCH, true, CT, PPL><<<ct.tiles_total * NB, CT * CT / PPL, 0, st>>>(
            sp, pr, rg, ct, bg, img, tf, nl, work, full, stride);
    else
        render_fwd_kernel<TILE, BATCH, false, CT, PPL><<<ct.tiles_total * NB, CT * CT / PPL, 0, st>>>(
            sp, pr, rg, ct, bg, img, tf, nl, nullptr, nullptr, 1);
    count_launch();
    return check_launch("render_fwd_kernel");
}

// Pixels per lane of the backward (measured on the 300k x 20-view workload): 2 for 8- and
// 16-pixel tiles (8 x 8 warp blocks), 4 for 32-pixel tiles (8 x 16).
template <int TILE>
constexpr int bwd_ppl() { return TILE == 32 ? 4 : 2; }

template <int TILE, int BATCH>
int prepare_bwd() {
    constexpr int PPL = bwd_ppl<TILE>();
    constexpr int CT = bwd_cta<TILE>();
    constexpr int bytes = BwdSmem<BATCH, CT * CT / PPL, PPL / 2>::kBytes;
    return allow_dynamic_smem(reinterpret_cast<const void*>(render_bwd_kernel<TILE, BATCH, PPL, CT>), bytes);
}

template <int TILE, int BATCH>
int launch_bwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               const float* tf, const int* nl, const float* dimg, const uint8_t* full, long long stride,
               dass_splat_grad* gs, cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    constexpr int PPL = bwd_ppl<TILE>();
    constexpr int CT = bwd_cta<TILE>();
    constexpr int NB = (TILE / CT) * (TILE / CT);
    constexpr int NT = CT * CT / PPL;
    constexpr int bytes = BwdSmem<BATCH, NT, PPL / 2>::kBytes;
    if (int rc = prepare_bwd<TILE, BATCH>()) return rc;
    render_bwd_kernel<TILE, BATCH, PPL, CT><<<ct.tiles_total * NB, NT, bytes, st>>>(sp, pr, rg, ct, bg, tf, nl, dimg,
                                                                                   full, stride, gs);
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

// Kernel attributes that must be set outside stream capture (dynamic shared memory above 48 KB).
int render_prepare(int tile, int batch) {
    struct { int tile; } ct{tile};
    DASS_DISPATCH(prepare_bwd)
}

}  // namespace dass
