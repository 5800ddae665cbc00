// Fidelity loss of Eq. 3, L = mean_c[(1-lambda) L1_c + lambda (1 - SSIM_c)], and dL/dimage.
// SSIM uses an 11x11 Gaussian window (sigma 1.5) applied separably with zero padding. Two
// stencil kernels over 16x16 output tiles staged with a 5-pixel halo in shared memory:
//   pass 1: local means/variances, SSIM map and its partials w.r.t. (mu_x, sigma_x^2, sigma_xy),
//           combined into three maps g1 = dS/dmu_x - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy,
//           g2 = dS/dsigma_x^2, g3 = dS/dsigma_xy, plus the loss partial sums;
//   pass 2: dSSIM/dx = (w * g1) + 2 x (w * g2) + y (w * g3) (the window is symmetric, so the
//           adjoint of the zero-padded filter is the same filter), combined with the L1 term.
#include <cmath>

#include "common.cuh"

namespace dass {

namespace {

constexpr int kT = 16;           // output tile
constexpr int kR = 5;            // window radius
constexpr int kS = kT + 2 * kR;  // staged tile side (26)
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

__global__ void __launch_bounds__(256) ssim_fwd_kernel(CamTable ct, Window win, LossArgs a) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kT, oy = blockIdx.y * kT;
    if (ox >= W || oy >= H) return;
    __shared__ float sx[kS][kS + 1];
    __shared__ float sy[kS][kS + 1];
    __shared__ float hq[5][kS][kT + 1];
    const int tid = threadIdx.x;
    for (int i = tid; i < kS * kS; i += 256) {
        int r = i / kS, c = i % kS;
        int gx = ox + c - kR, gy = oy + r - kR;
        bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        long long idx = off + (long long)gy * W + gx;
        sx[r][c] = in ? a.x[idx] : 0.f;
        sy[r][c] = in ? a.y[idx] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kS * kT; i += 256) {
        int r = i / kT, c = i % kT;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            float xv = sx[r][c + k], yv = sy[r][c + k], w = win.w[k];
            m0 += w * xv;
            m1 += w * yv;
            m2 += w * xv * xv;
            m3 += w * yv * yv;
            m4 += w * xv * yv;
        }
        hq[0][r][c] = m0; hq[1][r][c] = m1; hq[2][r][c] = m2; hq[3][r][c] = m3; hq[4][r][c] = m4;
    }
    __syncthreads();
    const int tx = tid % kT, ty = tid / kT;
    const int gx = ox + tx, gy = oy + ty;
    float contrib = 0.f;
    if (gx < W && gy < H) {
        float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            float w = win.w[k];
            mx += w * hq[0][ty + k][tx];
            my += w * hq[1][ty + k][tx];
            xx += w * hq[2][ty + k][tx];
            yy += w * hq[3][ty + k][tx];
            xy += w * hq[4][ty + k][tx];
        }
        float vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
        float A1 = 2.f * mx * my + kC1, B1 = mx * mx + my * my + kC1;
        float A2 = 2.f * cxy + kC2, B2 = vx + vy + kC2;
        float den = B1 * B2;
        float S = (A1 * A2) / den;
        float dmu = 2.f * my * A2 / den - 2.f * mx * S / B1;
        float dvx = -S / B2;
        float dcxy = 2.f * A1 / den;
        long long idx = off + (long long)gy * W + gx;
        a.g[idx] = dmu - 2.f * mx * dvx - my * dcxy;
        a.g[a.map_stride + idx] = dvx;
        a.g[2 * a.map_stride + idx] = dcxy;
        float xc = sx[ty + kR][tx + kR], yc = sy[ty + kR][tx + kR];
        float inv_n = a.inv_cams / (3.f * (float)W * (float)H);
        contrib = inv_n * ((1.f - a.lambda) * fabsf(xc - yc) - a.lambda * S);
    }
    // the constant lambda * 1 of the D-SSIM term, once per camera of this call
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0)
        atomicAdd(a.loss, (double)a.lambda * (double)ct.n * (double)a.inv_cams);
    block_add(a.loss, contrib);
}

__global__ void __launch_bounds__(256) ssim_bwd_kernel(CamTable ct, Window win, LossArgs a) {
    const CamInfo* cam;
    long long off;
    plane_of(ct, blockIdx.z, cam, off);
    const int W = cam->W, H = cam->H;
    const int ox = blockIdx.x * kT, oy = blockIdx.y * kT;
    if (ox >= W || oy >= H) return;
    __shared__ float sg[3][kS][kS + 1];
    __shared__ float hq[3][kS][kT + 1];
    const int tid = threadIdx.x;
    for (int i = tid; i < kS * kS; i += 256) {
        int r = i / kS, c = i % kS;
        int gx = ox + c - kR, gy = oy + r - kR;
        bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        long long idx = off + (long long)gy * W + gx;
        sg[0][r][c] = in ? a.g[idx] : 0.f;
        sg[1][r][c] = in ? a.g[a.map_stride + idx] : 0.f;
        sg[2][r][c] = in ? a.g[2 * a.map_stride + idx] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kS * kT; i += 256) {
        int r = i / kT, c = i % kT;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            float w = win.w[k];
            m0 += w * sg[0][r][c + k];
            m1 += w * sg[1][r][c + k];
            m2 += w * sg[2][r][c + k];
        }
        hq[0][r][c] = m0; hq[1][r][c] = m1; hq[2][r][c] = m2;
    }
    __syncthreads();
    const int tx = tid % kT, ty = tid / kT;
    const int gx = ox + tx, gy = oy + ty;
    if (gx < W && gy < H) {
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            float w = win.w[k];
            c0 += w * hq[0][ty + k][tx];
            c1 += w * hq[1][ty + k][tx];
            c2 += w * hq[2][ty + k][tx];
        }
        long long idx = off + (long long)gy * W + gx;
        float xv = a.x[idx], yv = a.y[idx];
        float dS = c0 + 2.f * xv * c1 + yv * c2;
        float d = xv - yv;
        float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        float inv_n = a.inv_cams / (3.f * (float)W * (float)H);
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
    dim3 grid(div_up(maxW, kT), div_up(maxH, kT), 3 * ct.n);
    ssim_fwd_kernel<<<grid, 256, 0, st>>>(ct, w, a); count_launch();
    int rc = check_launch("ssim_fwd_kernel");
    if (rc) return rc;
    ssim_bwd_kernel<<<grid, 256, 0, st>>>(ct, w, a); count_launch();
    return check_launch("ssim_bwd_kernel");
}

}  // namespace dass
