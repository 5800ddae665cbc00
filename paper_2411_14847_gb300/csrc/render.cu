// Forward and backward alpha compositing (App. A.1) over every tile of every camera in one
// launch. One CTA per B x B tile, one thread per pixel; the tile's depth-sorted Gaussians are
// staged through shared memory in batches. The backward walks each tile's list in reverse
// from the last contributor, recomputing alpha and the transmittance T_j = T_{j+1}/(1-alpha_j)
// from the saved T_final, and reduces per-Gaussian gradients warp-wide (shuffles), then
// block-wide (shared-memory atomics), then into global memory (vector atomics).
#include "common.cuh"

namespace dass {

namespace {

// Stage one splat into its shared-memory form (identical in forward and backward).
__device__ __forceinline__ void stage_splat(const dass_splat* __restrict__ splats, uint32_t rec, float4& A,
                                            float4& Bv, float& blue, float4& raw) {
    const float4* sp = reinterpret_cast<const float4*>(splats + rec);
    float4 s0 = __ldg(sp);
    float4 s1 = __ldg(sp + 1);
    float s2 = __ldg(reinterpret_cast<const float*>(sp + 2));
    A = make_float4(s0.x, s0.y, __fmul_rn(s0.z, kNegHalfLog2e), __fmul_rn(s1.x, kNegHalfLog2e));
    Bv = make_float4(__fmul_rn(2.f * s0.w, kNegHalfLog2e), s1.y, s1.z, s1.w);
    blue = s2;
    raw = make_float4(s0.z, s0.w, s1.x, 0.f);
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
    constexpr int NT = TILE * TILE;
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ float sC[BATCH];
    const int tid = threadIdx.x;
    const int tile_id = blockIdx.x;
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int px = (local % cam.tiles_x) * TILE + (tid % TILE);
    const int py = (local / cam.tiles_x) * TILE + (tid / TILE);
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
        for (int i = tid; i < cnt; i += NT) {
            float4 raw;
            stage_splat(splats, pair_rec[base + i], sA[i], sB[i], sC[i], raw);
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
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
    constexpr int NT = TILE * TILE;
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ float4 sRaw[BATCH];
    __shared__ float sC[BATCH];
    __shared__ uint32_t sRec[BATCH];
    __shared__ float sG[BATCH][12];
    __shared__ int s_maxlast;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tile_id = blockIdx.x;
    const CamInfo& cam = ct.c[cam_of_tile(ct, tile_id)];
    const int local = tile_id - cam.tile_base;
    const int px = (local % cam.tiles_x) * TILE + (tid % TILE);
    const int py = (local / cam.tiles_x) * TILE + (tid / TILE);
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
    if (last >= 0) atomicMax(&s_maxlast, last);
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
            stage_splat(splats, rec, sA[i], sB[i], sC[i], sRaw[i]);
#pragma unroll
            for (int k = 0; k < 12; ++k) sG[i][k] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
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
                        const float4 raw = sRaw[j];   // (a, b, c) of the conic
                        const float dpow = dLda * alpha;
                        v[5] = dLda * G;
                        v[0] = dpow * (raw.x * dx + raw.y * dy);
                        v[1] = dpow * (raw.z * dy + raw.y * dx);
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
