// Forward and backward alpha compositing (App. A.1) over every tile of every camera in one
// launch. Each CTA is one warp that owns an 8 x 4*PPL block of pixels of a binning tile; each lane
// owns PPL pixels of one column (rows y + 4k), handled as pixel pairs with the packed FP32x2
// arithmetic of sm_100+ (two-lane add/mul/fma that round like their scalar forms, so the packed
// alpha is bit-identical to a scalar evaluation). The warp walks its tile's depth-sorted list in
// rounds: the lanes test the round's entries against the block (the alpha >= 1/255 footprint
// ellipse against the rectangle of the block's pixel centres), compact the hits in list order
// (ballot + prefix popcount) into the warp's shared memory and composite only those. Warps of the
// same tile never wait for each other. The backward walks the lists in reverse from the block's last
// contributor, recomputing alpha and T_j = T_{j+1}/(1-alpha_j) from the saved T_final, reduces each
// Gaussian's gradient across the warp with shuffles and adds it to global memory with vector atomics.
// A round in which no staged entry can reach the 0.99 alpha clamp (the usual case: it needs an
// opacity near 0.99) runs a loop instantiation without the clamp's selects, and a backward round
// whose entries all lie at or before every pixel's last contributor one without the position test;
// both give the same bits as the general loop.
#include <type_traits>

#include "launch.cuh"

namespace dass {

namespace {

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

// Whether the alpha clamp at 0.99 can take effect for some pixel of the block [bx, bx + wm1] x
// [by, by + hm1] (pixel centres). Exactly, alpha = o G with G = exp(-q/2) <= 1 for a positive definite
// conic, so only o >= 0.99 could clamp. In FP32 the exponent q' = -(log2 e / 2) q is evaluated with
// four roundings, each off by at most 2^-24 of a value bounded by 0.722 M, where M = a DX^2 +
// 2|b| DX DY + c DY^2 and DX, DY are the block's largest offsets from the mean; so q' <= 1.72e-7 M,
// and with ex2.approx's relative error (below 2^-22) G <= (1 + 1.3e-7 M)(1 + 2.4e-7) for M <= 1e6.
// Then o (1 + 5e-7 M) < 0.985 keeps o G below 0.99 at every pixel of the block. Returns true (the
// clamp may act) otherwise, and for a conic that is not positive definite or not finite.
__device__ __forceinline__ bool clamp_possible(float nu, float nv, float a, float b, float c, float o, float bx,
                                               float by, float wm1, float hm1) {
    const float DX = fmaxf(fabsf(bx + nu), fabsf((bx + wm1) + nu));
    const float DY = fmaxf(fabsf(by + nv), fabsf((by + hm1) + nv));
    const float M = a * DX * DX + 2.f * fabsf(b) * DX * DY + c * DY * DY;
    return !(a > 0.f) || !(M <= 1e6f) || !(o * (1.f + 5e-7f * M) < 0.985f);
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
// CLAMP = false: no entry of the round can reach the clamp (clamp_possible), so -o G is used as is.
template <bool CLAMP, bool COUNT>
__device__ __forceinline__ void pix_fwd_step2(PixFwd2& p, int pos, float2 A, float2 B, const float4 P0,
                                              const float4 P2, const float4 P3, float2 nblue, bool full) {
    const float2 dy = __fadd2_rn(p.fy, hi2(P0));
    const float2 G = splat_gauss2(lo2(P2), dy, A, B);
    const float2 noG = __fmul2_rn(hi2(P2), G);                 // -o G
    float2 na = CLAMP ? make_float2(fmaxf(-kAlphaMax, noG.x), fmaxf(-kAlphaMax, noG.y)) : noG;
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

// Forward compositing, one warp per CTA owning one 8 x 4*PPL block of a tile (blockIdx.x = slot * WPT
// + block, the tile of a slot given by order, else the slot itself). The warp walks the tile's list
// in rounds of BATCH entries: lane i reads entries i, i + 32, ... of the round, tests whether each
// footprint reaches the block and stages the entries that do at their compacted slots (list order)
// in the warp's shared memory; the warp then composites the round's compacted entries. Warps never
// wait for each other, a warp whose pixels are all done exits at once, and the hardware gives its
// slot to the next block.
template <int TILE, int BATCH, bool COUNT, int PPL = 4>
__global__ void __launch_bounds__(32, 32) render_fwd_warp_kernel(const dass_splat* __restrict__ splats,
                                                            const uint32_t* __restrict__ pair_rec,
                                                            const uint32_t* __restrict__ ranges, CamTable ct,
                                                            float3 bg, float* __restrict__ image,
                                                            float* __restrict__ T_final, int* __restrict__ n_last,
                                                            unsigned long long* __restrict__ work,
                                                            const uint8_t* __restrict__ full_grad,
                                                            long long rec_stride,
                                                            const uint32_t* __restrict__ order) {
    constexpr int BH = 4 * PPL;
    constexpr int WX = TILE / 8, WY = TILE / BH, WPT = WX * WY;
    constexpr int NP = PPL / 2;
    static_assert(TILE % BH == 0 && BATCH % 32 == 0, "block taller than the tile, or a partial round");
    __shared__ float4 sP[5][BATCH];
    __shared__ int sPos[BATCH];
    __shared__ uint8_t sFullC[COUNT ? BATCH : 1];
    const int lane = threadIdx.x;
    // the WPT blocks of the tile order[blockIdx.x / WPT] (longest lists first), or of tile blockIdx.x / WPT
    const int tile_id = order ? (int)order[blockIdx.x / WPT] : (int)(blockIdx.x / WPT);
    if ((unsigned)tile_id >= (unsigned)ct.tiles_total) return;     // not a tile: an order that is no permutation
    const int wb = blockIdx.x % WPT;
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int bxi = (local % cam.tiles_x) * TILE + (wb % WX) * 8, byi = (local / cam.tiles_x) * TILE + (wb / WX) * BH;
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
        if (__all_sync(0xffffffffu, all_done())) break;
        int nl = 0;
        bool clamp = false;
#pragma unroll
        for (int r = 0; r < BATCH / 32; ++r) {
            const uint32_t j = base + 32 * r + lane;
            bool hit = false, cl = false;
            float4 s0, s1, F;
            float bl = 0.f;
            uint32_t rec = 0;
            if (j < end) {
                rec = pair_rec[j];
                const float4* sp = reinterpret_cast<const float4*>(splats + rec);
                s0 = __ldg(sp);        // u, v, a, b
                s1 = __ldg(sp + 1);    // c, o, r, g
                bl = __ldg(reinterpret_cast<const float*>(sp + 2));
                F = make_float4(s0.z, s0.w, s1.x, footprint_k2(s0.z, s0.w, s1.x, s1.y));
                hit = footprint_reaches_rect(-s0.x, -s0.y, F, bx, by, 7.f, (float)(BH - 1));
                cl = hit && clamp_possible(-s0.x, -s0.y, s0.z, s0.w, s1.x, s1.y, bx, by, 7.f, (float)(BH - 1));
            }
            clamp = clamp || __any_sync(0xffffffffu, cl);
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int i = nl + __popc(m & lanemask_lt());
                const float ap = __fmul_rn(s0.z, kNegHalfLog2e), b2p = __fmul_rn(2.f * s0.w, kNegHalfLog2e),
                            cp = __fmul_rn(s1.x, kNegHalfLog2e);
                sP[0][i] = make_float4(-s0.x, -s0.x, -s0.y, -s0.y);
                sP[1][i] = make_float4(ap, ap, b2p, b2p);
                sP[2][i] = make_float4(cp, cp, -s1.y, -s1.y);
                sP[3][i] = make_float4(-s1.z, -s1.z, -s1.w, -s1.w);
                sP[4][i] = make_float4(-bl, -bl, 0.f, 0.f);
                sPos[i] = (int)j;
                if (COUNT) sFullC[i] = full_grad ? full_grad[rec % (unsigned long long)rec_stride] : (uint8_t)1;
            }
            nl += __popc(m);
        }
        __syncwarp();
        // the round's entries, with the clamp only where some entry of the round may reach it
        auto composite = [&](auto clamp_tag) {
            constexpr bool CL = decltype(clamp_tag)::value;
#pragma unroll 8
            for (int t = 0; t < nl; ++t) {
                if ((t & 3) == 3 && __all_sync(0xffffffffu, all_done())) break;
                const float4 P0 = sP[0][t], P1 = sP[1][t], P2 = sP[2][t], P3 = sP[3][t];
                const float2 nblue = lo2(sP[4][t]);
                const float2 dx = __fadd2_rn(fx2, lo2(P0));
                float2 A, B;
                splat_column2(lo2(P1), hi2(P1), dx, A, B);
                const bool full = COUNT ? sFullC[COUNT ? t : 0] != 0 : false;
                const int pos = sPos[t];
#pragma unroll
                for (int k = 0; k < NP; ++k) pix_fwd_step2<CL, COUNT>(pp[k], pos, A, B, P0, P2, P3, nblue, full);
            }
        };
        if (clamp) composite(std::true_type{});
        else composite(std::false_type{});
        __syncwarp();
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
    float2 g0, g1, g2;
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

// Loads the pair's state, its upstream gradient included (held in registers for the whole walk).
__device__ __forceinline__ void pix_bwd_load2(PixBwd2& p, const CamInfo& cam, int px, int py, float3 bg,
                                              const float* __restrict__ T_final, const int* __restrict__ n_last,
                                              const float* __restrict__ dL_dimage) {
    float2 g0, g1, g2;
    p.fy = make_float2((float)py, (float)(py + 4));
    pix_bwd_load1(cam, px, py, T_final, n_last, dL_dimage, p.T.x, g0.x, g1.x, g2.x, p.last0);
    pix_bwd_load1(cam, px, py + 4, T_final, n_last, dL_dimage, p.T.y, g0.y, g1.y, g2.y, p.last1);
    p.S = __ffma2_rn(g2, make_float2(bg.z, bg.z),
                     __ffma2_rn(g1, make_float2(bg.y, bg.y), __fmul2_rn(g0, make_float2(bg.x, bg.x))));
    p.g0 = g0;
    p.g1 = g1;
    p.g2 = g2;
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
// CLAMP = false: no entry of the round can reach the clamp (clamp_possible), so alpha = o G and the
// clamp's derivative mask equals the blend mask. VALID: pos is at or before both pixels' last
// contributor (the caller checked it for the whole round), so the position test is dropped.
template <bool FULL, bool CLAMP, bool VALID>
__device__ __forceinline__ bool pix_bwd_step2(PixBwd2& p, int pos, float2 dx, float2 A, float2 B, const float4 P0,
                                              const float4 P2, const float4 P3, const float4 P4, float2* vm,
                                              float2* vf) {
    bool val0 = VALID || pos <= p.last0, val1 = VALID || pos <= p.last1;
    const float2 dy = __fadd2_rn(p.fy, hi2(P0));
    const float2 G = splat_gauss2(lo2(P2), dy, A, B);
    const float2 oG = __fmul2_rn(hi2(P2), G);
    const float2 alpha = CLAMP ? make_float2(fminf(kAlphaMax, oG.x), fminf(kAlphaMax, oG.y)) : oG;
    val0 = val0 && !(alpha.x < kAlphaMin);
    val1 = val1 && !(alpha.y < kAlphaMin);
    const float2 am = make_float2(val0 ? alpha.x : 0.f, val1 ? alpha.y : 0.f);
    const float2 om = one_minus2(am);
    // a pixel that takes no part has om = 1 exactly, and rcp.approx(1) = 1 exactly (checked on
    // sm_103), so its T passes through unchanged without a select
    const float2 Tj = __fmul2_rn(p.T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
    const float2 g0 = p.g0, g1 = p.g1, g2 = p.g2;
    const float2 gc = __ffma2_rn(lo2(P4), g2, __ffma2_rn(hi2(P3), g1, __fmul2_rn(lo2(P3), g0)));
    const float2 d = sub2(gc, p.S);
    const float2 dLda = __fmul2_rn(Tj, d);
    p.S = __ffma2_rn(am, d, p.S);       // alpha gc + (1 - alpha) S = S + alpha (gc - S)
    p.T = Tj;
    // the clamp alpha = 0.99 has zero derivative
    const bool cm0 = CLAMP ? val0 && oG.x < kAlphaMax : val0, cm1 = CLAMP ? val1 && oG.y < kAlphaMax : val1;
    const float2 dpow = CLAMP ? __fmul2_rn(dLda, make_float2(cm0 ? alpha.x : 0.f, cm1 ? alpha.y : 0.f))
                              : __fmul2_rn(dLda, am);
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

// Reverse step of staged entry P0..P4 that only carries the pixels' state past it (T and S, the
// same operations as pix_bwd_step2), for a Gaussian whose gradient nobody needs.
template <bool CLAMP, bool VALID>
__device__ __forceinline__ void pix_bwd_recur2(PixBwd2& p, int pos, float2 dx, float2 A, float2 B, const float4 P0,
                                               const float4 P2, const float4 P3, const float4 P4) {
    bool val0 = VALID || pos <= p.last0, val1 = VALID || pos <= p.last1;
    const float2 dy = __fadd2_rn(p.fy, hi2(P0));
    const float2 G = splat_gauss2(lo2(P2), dy, A, B);
    const float2 oG = __fmul2_rn(hi2(P2), G);
    const float2 alpha = CLAMP ? make_float2(fminf(kAlphaMax, oG.x), fminf(kAlphaMax, oG.y)) : oG;
    val0 = val0 && !(alpha.x < kAlphaMin);
    val1 = val1 && !(alpha.y < kAlphaMin);
    const float2 am = make_float2(val0 ? alpha.x : 0.f, val1 ? alpha.y : 0.f);
    const float2 om = one_minus2(am);
    const float2 Tj = __fmul2_rn(p.T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
    const float2 g0 = p.g0, g1 = p.g1, g2 = p.g2;
    const float2 gc = __ffma2_rn(lo2(P4), g2, __ffma2_rn(hi2(P3), g1, __fmul2_rn(lo2(P3), g0)));
    const float2 d = sub2(gc, p.S);
    p.S = __ffma2_rn(am, d, p.S);
    p.T = Tj;
}

// Backward compositing, one warp per CTA owning one 8 x 4*PPL block of a tile. The warp walks the
// tile's list in reverse from its pixels' last contributor, in rounds of BATCH entries: the lanes
// read the round's entries (ascending), test each footprint against the block and stage the entries
// that reach it (compacted, in list order) in the warp's shared memory; the warp then runs the
// reverse pair steps over the round's entries from the last one down, reduces each Gaussian's
// gradient across the warp with shuffles and adds it to splat_grads[record] with vector atomics (one
// float2 for a mean-only Gaussian: dL/du = a X + b Y, dL/dv = b X + c Y of the block sums X, Y). The
// upstream gradients of the lanes' pixels stay in registers instead of being re-read from shared
// memory at every step (those loads made up most of the kernel's shared-memory traffic); at 64
// registers (a few spills in the full-gradient path) 32 warps stay resident per SM, which measured
// faster than 72 registers at 28 warps. Rounds of 128 or 256 entries need more registers (at 64 they
// spill heavily: 3.3 -> 6.0 ms), so those instantiations keep 72 registers and 28 warps.
// MEANS: every entry not flagged in full_grad still gets dL/dmean2D (the shift stage's
// densification statistics need it); else those entries only carry the recurrence past them.
template <int TILE, int BATCH, int PPL = 4, bool MEANS = true>
__global__ void __launch_bounds__(32, BATCH <= 64 ? 32 : 28) render_bwd_warp_kernel(
    const dass_splat* __restrict__ splats, const uint32_t* __restrict__ pair_rec, const uint32_t* __restrict__ ranges,
    CamTable ct, float3 bg, const float* __restrict__ T_final, const int* __restrict__ n_last,
    const float* __restrict__ dL_dimage, const uint8_t* __restrict__ full_grad, long long rec_stride,
    dass_splat_grad* __restrict__ gsplat, const uint32_t* __restrict__ order) {
    constexpr int BH = 4 * PPL;
    constexpr int WX = TILE / 8, WY = TILE / BH, WPT = WX * WY;
    constexpr int NP = PPL / 2;
    static_assert(TILE % BH == 0 && BATCH % 32 == 0, "block taller than the tile, or a partial round");
    __shared__ float4 sP[5][BATCH];
    __shared__ float4 sF[BATCH];
    __shared__ uint32_t sRec[BATCH];
    __shared__ int sPos[BATCH];
    __shared__ uint8_t sFull[BATCH];
    const int lane = threadIdx.x;
    // the WPT blocks of the tile order[blockIdx.x / WPT] (longest lists first), or of tile blockIdx.x / WPT
    const int tile_id = order ? (int)order[blockIdx.x / WPT] : (int)(blockIdx.x / WPT);
    if ((unsigned)tile_id >= (unsigned)ct.tiles_total) return;     // not a tile: an order that is no permutation
    const int wb = blockIdx.x % WPT;
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int bxi = (local % cam.tiles_x) * TILE + (wb % WX) * 8, byi = (local / cam.tiles_x) * TILE + (wb / WX) * BH;
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
        pix_bwd_load2(pp[k], cam, px, py + 8 * k, bg, T_final, n_last, dL_dimage);
        mylast = max(mylast, max(pp[k].last0, pp[k].last1));
    }
    const int wlast = __reduce_max_sync(0xffffffffu, mylast);
    int myfirst = 0x7fffffff;
#pragma unroll
    for (int k = 0; k < NP; ++k) myfirst = min(myfirst, min(pp[k].last0, pp[k].last1));
    // smallest last contributor of the block (-1 where a pixel has none or lies outside the image, so
    // such a block never takes the rounds without the position test)
    const int wmin = __reduce_min_sync(0xffffffffu, myfirst);
    __syncwarp();
    for (long long hi = (long long)wlast + 1; hi > (long long)start; hi -= BATCH) {
        const long long lo = hi - BATCH > (long long)start ? hi - BATCH : (long long)start;
        int nl = 0;
        bool clamp = false;
#pragma unroll
        for (int r = 0; r < BATCH / 32; ++r) {
            const long long pos = lo + 32 * r + lane;
            bool hit = false, cl = false;
            float4 s0, s1, F;
            float bl = 0.f;
            uint32_t rec = 0;
            if (pos < hi) {
                rec = pair_rec[pos];
                const float4* sp = reinterpret_cast<const float4*>(splats + rec);
                s0 = __ldg(sp);        // u, v, a, b
                s1 = __ldg(sp + 1);    // c, o, r, g
                bl = __ldg(reinterpret_cast<const float*>(sp + 2));
                F = make_float4(s0.z, s0.w, s1.x, footprint_k2(s0.z, s0.w, s1.x, s1.y));
                hit = footprint_reaches_rect(-s0.x, -s0.y, F, bx, by, 7.f, (float)(BH - 1));
                cl = hit && clamp_possible(-s0.x, -s0.y, s0.z, s0.w, s1.x, s1.y, bx, by, 7.f, (float)(BH - 1));
            }
            clamp = clamp || __any_sync(0xffffffffu, cl);
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int i = nl + __popc(m & lanemask_lt());
                const float ap = __fmul_rn(s0.z, kNegHalfLog2e), b2p = __fmul_rn(2.f * s0.w, kNegHalfLog2e),
                            cp = __fmul_rn(s1.x, kNegHalfLog2e);
                sP[0][i] = make_float4(-s0.x, -s0.x, -s0.y, -s0.y);
                sP[1][i] = make_float4(ap, ap, b2p, b2p);
                sP[2][i] = make_float4(cp, cp, s1.y, s1.y);
                sP[3][i] = make_float4(s1.z, s1.z, s1.w, s1.w);
                sP[4][i] = make_float4(bl, bl, 0.f, 0.f);
                sF[i] = make_float4(s0.z, s0.w, s1.x, 0.f);
                sRec[i] = rec;
                sPos[i] = (int)pos;
                sFull[i] = full_grad ? full_grad[rec % stride] : (uint8_t)1;
            }
            nl += __popc(m);
        }
        __syncwarp();
        // the round's entries, with the clamp only where some entry of the round may reach it
        auto reverse_round = [&](auto clamp_tag, auto valid_tag) {
            constexpr bool CL = decltype(clamp_tag)::value;
            constexpr bool VA = decltype(valid_tag)::value;
            // reverse pair steps of the mean-only entry j (dL/dmean2D moments into vm). A mean-only
            // entry's sums are reduced and added whether or not a pixel took part (adding zeros is exact,
            // and testing for it cost more than the rare all-zero reductions it saved)
            auto mean_steps = [&](int j, float2* vm) {
                const int p = sPos[j];
                const float4 P0 = sP[0][j], P1 = sP[1][j], P2 = sP[2][j], P3 = sP[3][j], P4 = sP[4][j];
                const float2 dx = __fadd2_rn(fx2, lo2(P0));
                float2 A, B;
                splat_column2(lo2(P1), hi2(P1), dx, A, B);
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    pix_bwd_step2<false, CL, VA>(pp[k], p, dx, A, B, P0, P2, P3, P4, vm, nullptr);
            };
            for (int t = nl - 1; t >= 0; --t) {
                bool contrib = false;
                float2 vm[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                if (sFull[t]) {          // warp-uniform: the same Gaussian for every lane
                    const int p = sPos[t];
                    const float4 P0 = sP[0][t], P1 = sP[1][t], P2 = sP[2][t], P3 = sP[3][t], P4 = sP[4][t];
                    const float2 dx = __fadd2_rn(fx2, lo2(P0));
                    float2 A, B;
                    splat_column2(lo2(P1), hi2(P1), dx, A, B);
                    float2 vf[7];      // vf[0], vf[1] unused: formed from vm below
#pragma unroll
                    for (int i = 0; i < 7; ++i) vf[i] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < NP; ++k)
                        contrib |= pix_bwd_step2<true, CL, VA>(pp[k], p, dx, A, B, P0, P2, P3, P4, vm, vf);
                    if (__ballot_sync(0xffffffffu, contrib)) {
                        const float X = dx.x * (vm[0].x + vm[0].y), Y = vm[1].x + vm[1].y;
                        float r[8] = {X, Y, dx.x * X, dx.x * Y, vf[2].x + vf[2].y, vf[3].x + vf[3].y,
                                      vf[4].x + vf[4].y, vf[5].x + vf[5].y};
                        const float sm = warp_reduce8(r, lane) * gscale;
                        const float e = warp_sum(vf[6].x + vf[6].y);
                        // lane 4 g (g < 8) holds reduced value g: X, Y, dL/da, dL/db, dL/dc, dL/do, dL/dr, dL/dg
                        const float Xs = __shfl_sync(0xffffffffu, sm, 0), Ys = __shfl_sync(0xffffffffu, sm, 4);
                        const float v2 = __shfl_sync(0xffffffffu, sm, 8), v3 = __shfl_sync(0xffffffffu, sm, 12);
                        const float v4 = __shfl_sync(0xffffffffu, sm, 16), v5 = __shfl_sync(0xffffffffu, sm, 20);
                        const float v6 = __shfl_sync(0xffffffffu, sm, 24), v7 = __shfl_sync(0xffffffffu, sm, 28);
                        if (lane == 0) {
                            const float4 F = sF[t];
                            float4* dst = reinterpret_cast<float4*>(gsplat + sRec[t]);
                            atomicAdd(dst, make_float4(F.x * Xs + F.y * Ys, F.y * Xs + F.z * Ys, v2, v3));
                            atomicAdd(dst + 1, make_float4(v4, v5, v6, v7));
                            atomicAdd(reinterpret_cast<float*>(dst + 2), e);
                        }
                    }
                } else if constexpr (!MEANS) {
                    const int p = sPos[t];
                    const float4 P0 = sP[0][t], P1 = sP[1][t], P2 = sP[2][t], P3 = sP[3][t], P4 = sP[4][t];
                    const float2 dx = __fadd2_rn(fx2, lo2(P0));
                    float2 A, B;
                    splat_column2(lo2(P1), hi2(P1), dx, A, B);
#pragma unroll
                    for (int k = 0; k < NP; ++k)
                        pix_bwd_recur2<CL, VA>(pp[k], p, dx, A, B, P0, P2, P3, P4);
                } else {
                    // mean-only entries are taken four at a time when the next three are mean-only too
                    // (warp-uniform), so that one 8-value reduction serves all four
                    if (t >= 3 && !sFull[t - 1] && !sFull[t - 2] && !sFull[t - 3]) {
                        float r8[8];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float2 v[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                            mean_steps(t - e, v);
                            r8[2 * e] = v[0].x + v[0].y;
                            r8[2 * e + 1] = v[1].x + v[1].y;
                        }
                        // lane 8 e holds X of entry t - e, lane 8 e + 4 its Y
                        const float r = warp_reduce8(r8, lane);
                        const float Yp = __shfl_down_sync(0xffffffffu, r, 4);
                        if ((lane & 7) == 0) {
                            const int e = t - (lane >> 3);
                            const float4 F = sF[e];
                            atomicAdd(reinterpret_cast<float2*>(gsplat + sRec[e]),
                                      make_float2(F.x * r + F.y * Yp, F.y * r + F.z * Yp));
                        }
                        t -= 3;
                        continue;
                    }
                    // else two at a time when the next one is mean-only too
                    const bool two = t >= 1 && !sFull[t - 1];
                    mean_steps(t, vm);
                    float2 vm2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    if (two) mean_steps(t - 1, vm2);
                    if (two) {
                        const float r = warp_reduce4(vm[0].x + vm[0].y, vm[1].x + vm[1].y, vm2[0].x + vm2[0].y,
                                                     vm2[1].x + vm2[1].y, lane);
                        // lanes 0, 8 hold X, Y of entry t; lanes 16, 24 those of entry t - 1
                        const float Yp = __shfl_down_sync(0xffffffffu, r, 8);
                        if ((lane & 15) == 0) {
                            const int e = (lane & 16) ? t - 1 : t;
                            const float4 F = sF[e];
                            atomicAdd(reinterpret_cast<float2*>(gsplat + sRec[e]),
                                      make_float2(F.x * r + F.y * Yp, F.y * r + F.z * Yp));
                        }
                    } else {
                        const float r = warp_reduce2(vm[0].x + vm[0].y, vm[1].x + vm[1].y, lane);
                        // lane 0 holds X, lane 16 holds Y
                        const float Yp = __shfl_sync(0xffffffffu, r, 16);
                        if (lane == 0) {
                            const float4 F = sF[t];
                            atomicAdd(reinterpret_cast<float2*>(gsplat + sRec[t]),
                                      make_float2(F.x * r + F.y * Yp, F.y * r + F.z * Yp));
                        }
                    }
                    if (two) --t;
                }
            }
        };
        // every pixel of the block has its last contributor at or after the round's last entry
        const bool all_valid = hi - 1 <= (long long)wmin;
        if (clamp) {
            if (all_valid) reverse_round(std::true_type{}, std::true_type{});
            else reverse_round(std::true_type{}, std::false_type{});
        } else {
            if (all_valid) reverse_round(std::false_type{}, std::true_type{});
            else reverse_round(std::false_type{}, std::false_type{});
        }
        __syncwarp();
    }
}

template <int TILE, int BATCH>
int launch_fwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               float* img, float* tf, int* nl, unsigned long long* work, const uint8_t* full, long long stride,
               const uint32_t* order, cudaStream_t st) {
    if (ct.tiles_total <= 0) return DASS_OK;
    constexpr int PPL = TILE == 8 ? 2 : 4;
    constexpr int WPT = (TILE / 8) * (TILE / (4 * PPL));
    const long long grid = (long long)ct.tiles_total * WPT;
    if (work)
        render_fwd_warp_kernel<TILE, BATCH, true, PPL><<<(unsigned)grid, 32, 0, st>>>(sp, pr, rg, ct, bg, img, tf, nl, work,
                                                                              full, stride, order);
    else
        render_fwd_warp_kernel<TILE, BATCH, false, PPL><<<(unsigned)grid, 32, 0, st>>>(sp, pr, rg, ct, bg, img, tf, nl,
                                                                               nullptr, nullptr, 1, order);
    count_launch();
    return check_launch("render_fwd_warp_kernel");
}

template <int TILE, int BATCH>
int launch_bwd(const dass_splat* sp, const uint32_t* pr, const uint32_t* rg, const CamTable& ct, float3 bg,
               const float* tf, const int* nl, const float* dimg, const uint8_t* full, long long stride,
               dass_splat_grad* gs, cudaStream_t st, bool means, const uint32_t* order) {
    if (ct.tiles_total <= 0) return DASS_OK;
    constexpr int PPL = TILE == 8 ? 2 : 4;
    constexpr int WPT = (TILE / 8) * (TILE / (4 * PPL));
    const long long grid = (long long)ct.tiles_total * WPT;
    if (means || !full)
        render_bwd_warp_kernel<TILE, BATCH, PPL, true><<<(unsigned)grid, 32, 0, st>>>(sp, pr, rg, ct, bg, tf, nl, dimg,
                                                                                  full, stride, gs, order);
    else
        render_bwd_warp_kernel<TILE, BATCH, PPL, false><<<(unsigned)grid, 32, 0, st>>>(sp, pr, rg, ct, bg, tf, nl, dimg,
                                                                                   full, stride, gs, order);
    count_launch();
    return check_launch("render_bwd_warp_kernel");
}

}  // namespace

#define DASS_DISPATCH(FN, ...)                                                        \
    switch (ct.tile * 1000 + batch) {                                                 \
        case 8032: return FN<8, 32>(__VA_ARGS__);                                     \
        case 8064: return FN<8, 64>(__VA_ARGS__);                                     \
        case 8128: return FN<8, 128>(__VA_ARGS__);                                    \
        case 8256: return FN<8, 256>(__VA_ARGS__);                                    \
        case 16032: return FN<16, 32>(__VA_ARGS__);                                   \
        case 16064: return FN<16, 64>(__VA_ARGS__);                                   \
        case 16128: return FN<16, 128>(__VA_ARGS__);                                  \
        case 16256: return FN<16, 256>(__VA_ARGS__);                                  \
        case 32032: return FN<32, 32>(__VA_ARGS__);                                   \
        case 32064: return FN<32, 64>(__VA_ARGS__);                                   \
        case 32128: return FN<32, 128>(__VA_ARGS__);                                  \
        case 32256: return FN<32, 256>(__VA_ARGS__);                                  \
        default: return DASS_ERR_INVALID_ARG;                                         \
    }

int render_fwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, float* image, float* T_final, int* n_last, cudaStream_t st,
                      unsigned long long* work, const uint8_t* full_grad, long long rec_stride,
                      const uint32_t* order) {
    DASS_DISPATCH(launch_fwd, splats, pair_rec, ranges, ct, bg, image, T_final, n_last, work, full_grad, rec_stride,
                  order, st)
}

int render_bwd_launch(const dass_splat* splats, const uint32_t* pair_rec, const uint32_t* ranges, const CamTable& ct,
                      int batch, float3 bg, const float* T_final, const int* n_last, const float* dL_dimage,
                      const uint8_t* full_grad, long long rec_stride, dass_splat_grad* gsplat, cudaStream_t st,
                      bool mean_grads, const uint32_t* order) {
    DASS_DISPATCH(launch_bwd, splats, pair_rec, ranges, ct, bg, T_final, n_last, dL_dimage, full_grad, rec_stride,
                  gsplat, st, mean_grads, order)
}

namespace {

// Order of the compositing launches' tiles, longest list first: a counting sort of the tiles by
// list length in 8 buckets per octave (e = floor(log2 len), the 3 bits below the leading one),
// descending, empty lists last. One CTA; the order within a bucket follows the shared-memory atomics
// and only affects the schedule, never a result (every block's pixels and gradient sums are its own).
__global__ void __launch_bounds__(1024) tile_order_kernel(const uint32_t* __restrict__ ranges, int tiles,
                                                          uint32_t* __restrict__ order) {
    __shared__ int count[256];
    __shared__ int base[256];
    auto bucket = [&](int t) {
        const uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len == 0) return 255;
        const int e = 31 - __clz((int)len);
        const int m = e >= 3 ? (int)(len >> (e - 3)) & 7 : (int)(len << (3 - e)) & 7;
        return 254 - min(e * 8 + m, 254);
    };
    for (int i = threadIdx.x; i < 256; i += blockDim.x) count[i] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) atomicAdd(&count[bucket(t)], 1);
    __syncthreads();
    if (threadIdx.x < 32) {          // exclusive scan of the 256 counts, 8 per lane
        const int l = threadIdx.x;
        int v[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = s;
            s += count[8 * l + k];
        }
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (l >= o) incl += u;
        }
        const int excl = incl - s;
#pragma unroll
        for (int k = 0; k < 8; ++k) base[8 * l + k] = excl + v[k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) order[atomicAdd(&base[bucket(t)], 1)] = (uint32_t)t;
}

}  // namespace

int tile_order_launch(const uint32_t* ranges, int tiles, uint32_t* order, cudaStream_t st) {
    if (tiles <= 0) return DASS_OK;
    tile_order_kernel<<<1, 1024, 0, st>>>(ranges, tiles, order);
    count_launch();
    return check_launch("tile_order_kernel");
}

// Checks a (tile, batch) shape before a stage is captured. The compositing kernels use static shared
// memory only (at most 48 KB), so no kernel attribute has to be set outside capture.
int render_prepare(int tile, int batch) {
    return ((tile == 8 || tile == 16 || tile == 32) && batch_ok(batch)) ? DASS_OK : DASS_ERR_INVALID_ARG;
}

}  // namespace dass
