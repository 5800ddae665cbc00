// Fidelity loss of Eq. 3, L = mean_c[(1-lambda) L1_c + lambda (1 - SSIM_c)], and dL/dimage.
// SSIM uses an 11x11 Gaussian window (sigma 1.5) applied separably with zero padding. Two
// stencil kernels over 32x32 output tiles staged with a 5-pixel halo in shared memory:
//   pass 1: local means/variances, SSIM map and its partials w.r.t. (mu_x, sigma_x^2, sigma_xy),
//           combined into three maps g1 = dS/dmu_x - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy,
//           g2 = dS/dsigma_x^2, g3 = dS/dsigma_xy, plus the loss partial sums;
//   pass 2: dSSIM/dx = (w * g1) + 2 x (w * g2) + y (w * g3) (the window is symmetric, so the
//           adjoint of the zero-padded filter is the same filter), combined with the L1 term.
#include <cmath>
#include <type_traits>

#include "common.cuh"

namespace dass {

namespace {


constexpr int kR = 5;            // window radius

constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Window {
    float w[11];
};

struct LossArgs {
    const float* x;       // image
    const float* y;       // target
    float* dx;            // dL/dimage
    float* g;             // gradient maps: (g1, g2) pairs [3 * pixels_total][2], then g3 [3 * pixels_total]
    double* loss;
    const float2* ystats; // optional cached target statistics, (w * y, w * y^2) per pixel-channel
    float lambda;
    float inv_cams;
    long long map_stride;  // 3 * pixels_total
};

__device__ __forceinline__ void plane_of(const CamTable& ct, int z, const CamInfo*& cam, long long& off) {
    int ci = z / 3, ch = z % 3;
    cam = &ct.c[ci];
    off = 3 * cam->pix_base + (long long)ch * cam->W * cam->H;
}

__device__ __forceinline__ void block_add(double* dst, float v) {
    __shared__ float red[8];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        atomicAdd(dst, (double)s);
    }
}

// Register-blocked separable filtering with packed FP32x2 arithmetic. A block computes a 32 x 32
// output tile from a 42 x 42 staged input (5-pixel halo). The quantities travel in pairs through
// both passes -- (x, y) and (x^2, y^2) in the forward, (g1, g2) in the backward -- plus one
// scalar quantity (xy, resp. g3), so one packed FMA applies a tap to two quantities.
// Horizontal pass: a job is (row, 4 consecutive output columns); the thread loads the 14 inputs
// it needs once and produces 4 outputs per quantity. Jobs are numbered row-fastest so that the
// 16 lanes of a shared-memory wavefront read 16 different rows (odd padded row length: no bank
// conflicts). Vertical pass: each thread owns (column, 4 consecutive output rows) and slides the
// window over 14 staged values per quantity.
constexpr int kO = 32;            // output tile side
constexpr int kI = kO + 2 * kR;   // staged side (42)
constexpr int kIP = kI + 1;       // padded row length of the staged input (odd)
constexpr int kHP = kO + 1;       // padded row length of the horizontal results (odd)

struct Window2 {
    float2 w[11];                 // (w_t, w_t): the window as packed operands
};

// Staged input: a packed pair per pixel, plus a scalar plane in the backward.
struct TileF {
    float2 p[kI][kIP];
};
struct TileB {
    float2 p[kI][kIP];
    float s[kI][kIP];
};
// Horizontal results: the pair, the squared pair (forward only) and the scalar quantity.
struct HorF {
    float2 p[kI][kHP];
    float2 q[kI][kHP];
    float s[kI][kHP];
};
struct HorB {
    float2 p[kI][kHP];
    float s[kI][kHP];
};

// Quantities filtered by the passes, from the staged pair (and scalar):
//   kPairScalar: the staged pair and the staged scalar as they are;
//   kSquares:    staged (x, y) -> the pairs (x, y), (x^2, y^2) and the scalar x*y;
//   kCached:     staged (x, y) -> the pair (x, x^2) and the scalar x*y (the target's window
//                statistics come from a cache).
enum Mode { kPairScalar = 0, kSquares = 1, kCached = 2 };

template <int MODE, class Tile, class Hor>
__device__ __forceinline__ void hpass2(const Tile& src, Hor& dst, const Window2& win) {
    for (int job = threadIdx.x; job < kI * (kO / 4); job += 256) {
        const int r = job % kI, c0 = (job / kI) * 4;
        float2 a[4], b[4];
        float c[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            a[o] = make_float2(0.f, 0.f);
            b[o] = make_float2(0.f, 0.f);
            c[o] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const float2 xy = src.p[r][c0 + k];
            float2 in = xy, sq = make_float2(0.f, 0.f);
            float sc = 0.f;
            if constexpr (MODE == kSquares) {
                sq = __fmul2_rn(xy, xy);
                sc = xy.x * xy.y;
            } else if constexpr (MODE == kCached) {
                in = make_float2(xy.x, xy.x * xy.x);
                sc = xy.x * xy.y;
            } else {
                sc = src.s[r][c0 + k];
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int t = k - o;
                if (t >= 0 && t < 11) {
                    a[o] = __ffma2_rn(win.w[t], in, a[o]);
                    if constexpr (MODE == kSquares) b[o] = __ffma2_rn(win.w[t], sq, b[o]);
                    c[o] = fmaf(win.w[t].x, sc, c[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            dst.p[r][c0 + o] = a[o];
            if constexpr (MODE == kSquares) dst.q[r][c0 + o] = b[o];
            dst.s[r][c0 + o] = c[o];
        }
    }
}

// Vertical pass for the thread's column and 4 output rows r0 + o.
template <bool SQUARES, class Hor>
__device__ __forceinline__ void vpass2(const Hor& h, const Window2& win, int col, int r0, float2 a[4], float2 b[4],
                                       float c[4]) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        a[o] = make_float2(0.f, 0.f);
        b[o] = make_float2(0.f, 0.f);
        c[o] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        const float2 ia = h.p[r0 + k][col];
        float2 ib = make_float2(0.f, 0.f);
        if constexpr (SQUARES) ib = h.q[r0 + k][col];
        const float ic = h.s[r0 + k][col];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int t = k - o;
            if (t >= 0 && t < 11) {
                a[o] = __ffma2_rn(win.w[t], ia, a[o]);
                if (SQUARES) b[o] = __ffma2_rn(win.w[t], ib, b[o]);
                c[o] = fmaf(win.w[t].x, ic, c[o]);
            }
        }
    }
}

// Stage the 42 x 42 window of the pair (p0, p1) -- for TileB the pair is stored interleaved at p0
// (p1 unused) -- and the scalar plane ps (TileB) of the plane at element offset off, with zeros
// outside the image. Each thread issues all of its global loads
// before its first shared store, so the block waits for one memory latency, not one per element.
// A thread's elements are threadIdx.x + 256 e; their (row, column) advance by (6, 4) per step
// (256 = 6 * 42 + 4), and the plane offsets are 32-bit (a plane has fewer than 2^31 pixels).
template <class Tile>
__device__ __forceinline__ void stage2(Tile& dst, const float* p0, const float* p1, const float* ps, long long off,
                                       int W, int H, int ox, int oy) {
    constexpr int kPer = (kI * kI + 255) / 256;
    constexpr bool kScalar = std::is_same_v<Tile, TileB>;   // backward: p0 holds interleaved pairs
    static_assert(256 / kI == 6 && 256 % kI == 4, "element stepping assumes a 42-wide window");
    const float* __restrict__ b0 = kScalar ? nullptr : p0 + off;
    const float* __restrict__ b1 = kScalar ? nullptr : p1 + off;
    const float2* __restrict__ b01 = kScalar ? reinterpret_cast<const float2*>(p0) + off : nullptr;
    const float* __restrict__ bs = kScalar ? ps + off : nullptr;
    float2 v[kPer];
    float sv[kPer];
    int so[kPer];
    int r = threadIdx.x / kI, c = threadIdx.x % kI;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int gx = ox + c - kR, gy = oy + r - kR;
        const bool in = r < kI && (unsigned)gx < (unsigned)W && (unsigned)gy < (unsigned)H;
        const int q = gy * W + gx;
        if constexpr (kScalar)
            v[e] = in ? __ldg(b01 + q) : make_float2(0.f, 0.f);
        else
            v[e] = in ? make_float2(__ldg(b0 + q), __ldg(b1 + q)) : make_float2(0.f, 0.f);
        if constexpr (kScalar) sv[e] = in ? __ldg(bs + q) : 0.f;
        so[e] = r < kI ? r * kIP + c : -1;
        c += 4;
        r += 6;
        if (c >= kI) {
            c -= kI;
            ++r;
        }
    }
    float2* dp = &dst.p[0][0];
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        if (so[e] >= 0) {
            dp[so[e]] = v[e];
            if constexpr (kScalar) (&dst.s[0][0])[so[e]] = sv[e];
        }
    }
}

// Forward SSIM of one 32 x 32 output tile. CACHED: the target's window mean and second moment
// come from a_.ystats (dass_loss_target_stats) and only x, x^2 and x*y are filtered here.
template <bool CACHED>
__global__ void __launch_bounds__(256, 5) ssim_fwd_kernel(CamTable ct, Window2 win, LossArgs a) {
    using Hor = std::conditional_t<CACHED, HorB, HorF>;
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kO, oy = blockIdx.y * kO;
    if (ox >= W || oy >= H) return;
    __shared__ TileF sin;
    __shared__ Hor sh;
    const int col = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
    float ym[4], y2[4];
    if constexpr (CACHED) {      // requested before the stencil work
        const float2* __restrict__ ms = a.ystats + off;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int gx = ox + col, gy = oy + r0 + o;
            const bool in = gx < W && gy < H;
            const int q = gy * W + gx;
            const float2 v = in ? __ldg(ms + q) : make_float2(0.f, 0.f);
            ym[o] = v.x;
            y2[o] = v.y;
        }
    }
    stage2(sin, a.x, a.y, nullptr, off, W, H, ox, oy);
    __syncthreads();
    float2 m[4], e[4];
    float exy[4];
    if constexpr (CACHED) {
        hpass2<kCached>(sin, sh, win);
        __syncthreads();
        float2 unused[4];
        vpass2<false>(sh, win, col, r0, m, unused, exy);   // m = (mean x, mean x^2)
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            e[o] = make_float2(m[o].y, y2[o]);
            m[o] = make_float2(m[o].x, ym[o]);
        }
    } else {
        hpass2<kSquares>(sin, sh, win);
        __syncthreads();
        vpass2<true>(sh, win, col, r0, m, e, exy);
    }
    const float inv_n = a.inv_cams / (3.f * (float)W * (float)H);
    float2* __restrict__ g12 = reinterpret_cast<float2*>(a.g) + off;
    float* __restrict__ g3 = a.g + 2 * a.map_stride + off;
    float contrib = 0.f;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int gx = ox + col, gy = oy + r0 + o;
        if (gx >= W || gy >= H) continue;
        const float mx = m[o].x, my = m[o].y;
        const float vx = e[o].x - mx * mx, vy = e[o].y - my * my, cxy = exy[o] - mx * my;
        const float A1 = 2.f * mx * my + kC1, B1 = mx * mx + my * my + kC1;
        const float A2 = 2.f * cxy + kC2, B2 = vx + vy + kC2;
        const float inv = __fdividef(1.f, B1 * B2);  // 1/B1 = B2 inv, 1/B2 = B1 inv (B1 B2 >= C1 C2 > 0)
        const float S = A1 * A2 * inv;
        const float dmu = 2.f * inv * (my * A2 - mx * S * B2);
        const float dvx = -S * B1 * inv;
        const float dcxy = 2.f * A1 * inv;
        const int q = gy * W + gx;
        g12[q] = make_float2(dmu - 2.f * mx * dvx - my * dcxy, dvx);
        g3[q] = dcxy;
        const float2 c = sin.p[r0 + o + kR][col + kR];
        contrib += inv_n * ((1.f - a.lambda) * fabsf(c.x - c.y) - a.lambda * S);
    }
    // the constant lambda * 1 of the D-SSIM term, once per camera of this call
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
        atomicAdd(a.loss, (double)a.lambda * (double)ct.n * (double)a.inv_cams);
    block_add(a.loss, contrib);
}

__global__ void __launch_bounds__(256, 4) ssim_bwd_kernel(CamTable ct, Window2 win, LossArgs a) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kO, oy = blockIdx.y * kO;
    if (ox >= W || oy >= H) return;
    __shared__ TileB sin;
    __shared__ HorB sh;
    const int col = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
    // the image and target values of the epilogue are requested before the stencil work
    float xv[4], yv[4];
    const float* __restrict__ xb = a.x + off;
    const float* __restrict__ yb = a.y + off;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int gx = ox + col, gy = oy + r0 + o;
        const bool in = gx < W && gy < H;
        const int q = gy * W + gx;
        xv[o] = in ? __ldg(xb + q) : 0.f;
        yv[o] = in ? __ldg(yb + q) : 0.f;
    }
    stage2(sin, a.g, nullptr, a.g + 2 * a.map_stride, off, W, H, ox, oy);
    __syncthreads();
    hpass2<kPairScalar>(sin, sh, win);
    __syncthreads();
    float2 c12[4], unused[4];
    float c3[4];
    vpass2<false>(sh, win, col, r0, c12, unused, c3);
    const float inv_n = a.inv_cams / (3.f * (float)W * (float)H);
    float* __restrict__ dxb = a.dx + off;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int gx = ox + col, gy = oy + r0 + o;
        if (gx >= W || gy >= H) continue;
        const float dS = c12[o].x + 2.f * xv[o] * c12[o].y + yv[o] * c3[o];
        const float d = xv[o] - yv[o];
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dxb[gy * W + gx] = inv_n * ((1.f - a.lambda) * sgn - a.lambda * dS);
    }
}

// Window statistics of the target (cached across the iterations of a stage): ystats[i] =
// (w * y, w * y^2) at pixel-channel i, planar like the image.
__global__ void __launch_bounds__(256, 4) ssim_target_stats_kernel(CamTable ct, Window2 win, const float* y,
                                                                   float2* ystats) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kO, oy = blockIdx.y * kO;
    if (ox >= W || oy >= H) return;
    __shared__ TileF sin;
    __shared__ HorB sh;
    stage2(sin, y, y, nullptr, off, W, H, ox, oy);
    __syncthreads();
    hpass2<kCached>(sin, sh, win);      // staged (y, y): pair (y, y^2)
    __syncthreads();
    const int col = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
    float2 m[4], unused[4];
    float c[4];
    vpass2<false>(sh, win, col, r0, m, unused, c);
    float2* __restrict__ so = ystats + off;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int gx = ox + col, gy = oy + r0 + o;
        if (gx >= W || gy >= H) continue;
        const int q = gy * W + gx;
        so[q] = m[o];
    }
}

__global__ void __launch_bounds__(256) l1_kernel(CamTable ct, LossArgs a) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.y, cam, off);
    long long plane = (long long)cam->W * cam->H;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float contrib = 0.f;
    if (i < plane) {
        float d = a.x[off + i] - a.y[off + i];
        float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        float inv_n = a.inv_cams / (3.f * (float)plane);
        a.dx[off + i] = inv_n * (1.f - a.lambda) * sgn;
        contrib = inv_n * (1.f - a.lambda) * fabsf(d);
    }
    block_add(a.loss, contrib);
}

Window make_window() {
    Window w;
    double s = 0.0, t[11];
    for (int k = 0; k < 11; ++k) {
        double x = k - 5.0;
        t[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        s += t[k];
    }
    for (int k = 0; k < 11; ++k) w.w[k] = (float)(t[k] / s);
    return w;
}

}  // namespace

size_t loss_workspace_bytes(const CamTable& ct) { return sizeof(float) * 9 * (size_t)ct.pixels_total; }

int loss_launch(const float* image, const float* target, const CamTable& ct, float lambda, float inv_cams, float* dL,
                double* loss, void* ws, size_t ws_bytes, cudaStream_t st, const float* target_stats) {
    LossArgs a;
    a.ystats = reinterpret_cast<const float2*>(target_stats);
    a.x = image;
    a.y = target;
    a.dx = dL;
    a.g = reinterpret_cast<float*>(ws);
    a.loss = loss;
    a.lambda = lambda;
    a.inv_cams = inv_cams;
    a.map_stride = 3 * ct.pixels_total;
    int maxW = 0, maxH = 0;
    long long maxP = 0;
    for (int i = 0; i < ct.n; ++i) {
        maxW = ct.c[i].W > maxW ? ct.c[i].W : maxW;
        maxH = ct.c[i].H > maxH ? ct.c[i].H : maxH;
        long long p = (long long)ct.c[i].W * ct.c[i].H;
        maxP = p > maxP ? p : maxP;
    }
    if (lambda == 0.f) {
        dim3 grid(div_up(maxP, 256), 3 * ct.n);
        l1_kernel<<<grid, 256, 0, st>>>(ct, a); count_launch();
        return check_launch("l1_kernel");
    }
    if (ws_bytes < loss_workspace_bytes(ct)) return DASS_ERR_OOM;
    Window w = make_window();
    Window2 w2;
    for (int t = 0; t < 11; ++t) w2.w[t] = make_float2(w.w[t], w.w[t]);
    dim3 grid(div_up(maxW, kO), div_up(maxH, kO), 3 * ct.n);
    if (target_stats)
        ssim_fwd_kernel<true><<<grid, 256, 0, st>>>(ct, w2, a);
    else
        ssim_fwd_kernel<false><<<grid, 256, 0, st>>>(ct, w2, a);
    count_launch();
    int rc = check_launch("ssim_fwd_kernel");
    if (rc) return rc;
    ssim_bwd_kernel<<<grid, 256, 0, st>>>(ct, w2, a); count_launch();
    return check_launch("ssim_bwd_kernel");
}

int target_stats_launch(const float* target, const CamTable& ct, float* stats, cudaStream_t st) {
    int maxW = 0, maxH = 0;
    for (int i = 0; i < ct.n; ++i) {
        maxW = ct.c[i].W > maxW ? ct.c[i].W : maxW;
        maxH = ct.c[i].H > maxH ? ct.c[i].H : maxH;
    }
    Window w = make_window();
    Window2 w2;
    for (int t = 0; t < 11; ++t) w2.w[t] = make_float2(w.w[t], w.w[t]);
    dim3 grid(div_up(maxW, kO), div_up(maxH, kO), 3 * ct.n);
    ssim_target_stats_kernel<<<grid, 256, 0, st>>>(ct, w2, target, reinterpret_cast<float2*>(stats));
    count_launch();
    return check_launch("ssim_target_stats_kernel");
}

}  // namespace dass
