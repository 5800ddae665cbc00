// Fidelity loss of Eq. 3, L = mean_c[(1-lambda) L1_c + lambda (1 - SSIM_c)], and dL/dimage.
// SSIM uses an 11x11 Gaussian window (sigma 1.5) applied separably with zero padding. Two
// stencil kernels over 32x32 output tiles staged with a 5-pixel halo in shared memory:
//   pass 1: local means/variances, SSIM map and its partials w.r.t. (mu_x, sigma_x^2, sigma_xy),
//           combined into three maps g1 = dS/dmu_x - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy,
//           g2 = dS/dsigma_x^2, g3 = dS/dsigma_xy, plus the loss partial sums;
//   pass 2: dSSIM/dx = (w * g1) + 2 x (w * g2) + y (w * g3) (the window is symmetric, so the
//           adjoint of the zero-padded filter is the same filter), combined with the L1 term.
#include <cmath>

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
    float* g;             // 3 maps, each 3 * pixels_total
    double* loss;
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

// Register-blocked separable filtering. A block computes a 32 x 32 output tile from a
// 42 x 42 staged input (5-pixel halo). Horizontal pass: a job is (row, 4 consecutive output
// columns); the thread loads the 14 inputs it needs once and produces 4 outputs per quantity.
// Vertical pass: each thread owns (column, 4 consecutive output rows) and slides the window
// over 14 staged values per quantity. Shared-memory loads per output drop from ~90 to ~26.
constexpr int kO = 32;            // output tile side
constexpr int kI = kO + 2 * kR;   // staged side (42)
constexpr int kIP = kI + 1;       // padded row length of the staged input
constexpr int kHP = kO + 1;       // padded row length of the horizontal results

template <int Q>
__device__ __forceinline__ void hpass(const float (*src)[kI][kIP], float (*dst)[kI][kHP], const Window& win,
                                      bool squares) {
    // jobs: 42 rows x 8 groups of 4 columns
    for (int job = threadIdx.x; job < kI * (kO / 4); job += 256) {
        const int r = job >> 3, c0 = (job & 7) * 4;
        float acc[Q][4];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[q][o] = 0.f;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            float in[Q];
            if (squares) {   // Q == 5: x, y, x^2, y^2, xy from the two staged inputs
                const float xv = src[0][r][c0 + k], yv = src[1][r][c0 + k];
                in[0] = xv; in[1] = yv;
                if (Q == 5) { in[2 % Q] = xv * xv; in[3 % Q] = yv * yv; in[4 % Q] = xv * yv; }
            } else {
#pragma unroll
                for (int q = 0; q < Q; ++q) in[q] = src[q][r][c0 + k];
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int t = k - o;
                if (t >= 0 && t < 11) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) acc[q][o] += win.w[t] * in[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) dst[q][r][c0 + o] = acc[q][o];
    }
}

// Vertical pass for the thread's column and 4 output rows: out[q][o] for rows r0 + o.
template <int Q>
__device__ __forceinline__ void vpass(const float (*h)[kI][kHP], const Window& win, int col, int r0,
                                      float out[Q][4]) {
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int o = 0; o < 4; ++o) out[q][o] = 0.f;
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        float in[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) in[q] = h[q][r0 + k][col];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int t = k - o;
            if (t >= 0 && t < 11) {
#pragma unroll
                for (int q = 0; q < Q; ++q) out[q][o] += win.w[t] * in[q];
            }
        }
    }
}

__device__ __forceinline__ void stage_planes(const float* const* planes, int n, float (*dst)[kI][kIP], long long off,
                                             int W, int H, int ox, int oy) {
    for (int i = threadIdx.x; i < kI * kI; i += 256) {
        const int r = i / kI, c = i % kI;
        const int gx = ox + c - kR, gy = oy + r - kR;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const long long idx = off + (long long)gy * W + gx;
        for (int q = 0; q < n; ++q) dst[q][r][c] = in ? planes[q][idx] : 0.f;
    }
}

__global__ void __launch_bounds__(256) ssim_fwd_kernel(CamTable ct, Window win, LossArgs a) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kO, oy = blockIdx.y * kO;
    if (ox >= W || oy >= H) return;
    __shared__ float sin[2][kI][kIP];
    __shared__ float sh[5][kI][kHP];
    const float* planes[2] = {a.x, a.y};
    stage_planes(planes, 2, sin, off, W, H, ox, oy);
    __syncthreads();
    hpass<5>(sin, sh, win, true);
    __syncthreads();
    const int col = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
    float m[5][4];
    vpass<5>(sh, win, col, r0, m);
    const float inv_n = a.inv_cams / (3.f * (float)W * (float)H);
    float contrib = 0.f;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int gx = ox + col, gy = oy + r0 + o;
        if (gx >= W || gy >= H) continue;
        const float mx = m[0][o], my = m[1][o];
        const float vx = m[2][o] - mx * mx, vy = m[3][o] - my * my, cxy = m[4][o] - mx * my;
        const float A1 = 2.f * mx * my + kC1, B1 = mx * mx + my * my + kC1;
        const float A2 = 2.f * cxy + kC2, B2 = vx + vy + kC2;
        const float den = B1 * B2;
        const float S = (A1 * A2) / den;
        const float dmu = 2.f * my * A2 / den - 2.f * mx * S / B1;
        const float dvx = -S / B2;
        const float dcxy = 2.f * A1 / den;
        const long long idx = off + (long long)gy * W + gx;
        a.g[idx] = dmu - 2.f * mx * dvx - my * dcxy;
        a.g[a.map_stride + idx] = dvx;
        a.g[2 * a.map_stride + idx] = dcxy;
        const float xc = sin[0][r0 + o + kR][col + kR], yc = sin[1][r0 + o + kR][col + kR];
        contrib += inv_n * ((1.f - a.lambda) * fabsf(xc - yc) - a.lambda * S);
    }
    // the constant lambda * 1 of the D-SSIM term, once per camera of this call
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
        atomicAdd(a.loss, (double)a.lambda * (double)ct.n * (double)a.inv_cams);
    block_add(a.loss, contrib);
}

__global__ void __launch_bounds__(256) ssim_bwd_kernel(CamTable ct, Window win, LossArgs a) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kO, oy = blockIdx.y * kO;
    if (ox >= W || oy >= H) return;
    __shared__ float sin[3][kI][kIP];
    __shared__ float sh[3][kI][kHP];
    const float* planes[3] = {a.g, a.g + a.map_stride, a.g + 2 * a.map_stride};
    stage_planes(planes, 3, sin, off, W, H, ox, oy);
    __syncthreads();
    hpass<3>(sin, sh, win, false);
    __syncthreads();
    const int col = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
    float c[3][4];
    vpass<3>(sh, win, col, r0, c);
    const float inv_n = a.inv_cams / (3.f * (float)W * (float)H);
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int gx = ox + col, gy = oy + r0 + o;
        if (gx >= W || gy >= H) continue;
        const long long idx = off + (long long)gy * W + gx;
        const float xv = a.x[idx], yv = a.y[idx];
        const float dS = c[0][o] + 2.f * xv * c[1][o] + yv * c[2][o];
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        a.dx[idx] = inv_n * ((1.f - a.lambda) * sgn - a.lambda * dS);
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
                double* loss, void* ws, size_t ws_bytes, cudaStream_t st) {
    LossArgs a;
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
    dim3 grid(div_up(maxW, kO), div_up(maxH, kO), 3 * ct.n);
    ssim_fwd_kernel<<<grid, 256, 0, st>>>(ct, w, a); count_launch();
    int rc = check_launch("ssim_fwd_kernel");
    if (rc) return rc;
    ssim_bwd_kernel<<<grid, 256, 0, st>>>(ct, w, a); count_launch();
    return check_launch("ssim_bwd_kernel");
}

}  // namespace dass
