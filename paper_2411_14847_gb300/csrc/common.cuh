// Shared device/host helpers of libdass (sm_103a). Hot-path math lives here so that the
// forward and backward kernels evaluate alpha with bit-identical operation sequences.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dass.h"

#define DASS_API extern "C" __attribute__((visibility("default")))

namespace dass {

// ----------------------------------------------------------------- error plumbing

void set_last_error(const char* what, cudaError_t e);
int check_launch(const char* what);   // returns DASS_OK or DASS_ERR_CUDA
// Number of kernels this thread has enqueued (graph replays count every captured kernel).
void count_launch(long long k = 1);
long long launches_so_far();
void set_launches(long long v);
// Opt a kernel in to `bytes` of dynamic shared memory on the current device (once per kernel and
// device; a no-op up to the default 48 KB). Not to be first called under stream capture.
int allow_dynamic_smem(const void* kernel, int bytes);

#define DASS_CHECK_CUDA(call)                                              \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) { dass::set_last_error(#call, e_); return DASS_ERR_CUDA; } \
    } while (0)

#define DASS_RETURN_IF(cond, code) do { if (cond) return (code); } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------------------- constants (App. A.1 readings)

constexpr float kNear = 0.2f;            // near-plane cull on camera z
constexpr float kLowPass = 0.3f;         // EWA low-pass added to the 2D covariance diagonal
constexpr float kAlphaMax = 0.99f;       // alpha clamp
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip threshold
constexpr float kTStop = 1e-4f;          // transmittance stop threshold
constexpr float kRadiusSlack = 0.01f;    // added to 2 ln(255 o) for the footprint radius
// power = -q/2 with q = d^T conic d; alpha = o * 2^(q * kNegHalfLog2e)
constexpr float kNegHalfLog2e = -0.72134752044448170f;

// ----------------------------------------------------------------- camera table (kernel params)

struct CamInfo {
    float R[9];        // world->camera rotation, row-major
    float t[3];
    float fx, fy, cx, cy;
    float campos[3];   // camera centre in world space
    float proj[16];    // Alg. 1 full projection T (row-vector convention), float32
    int W, H;
    int tiles_x, tiles_y;
    int tile_base;     // first global tile id of this camera
    int pad0;
    long long pix_base;  // first pixel (not float) index of this camera
    long long rec_base;  // first record index
};

struct CamTable {
    int n;
    int tile;
    int tiles_total;
    int pad;
    long long pixels_total;
    long long rec_stride;   // records per camera; 0 = packed segments (camera c owns [rec_base_c, rec_base_c+1))
    CamInfo c[DASS_MAX_CAMERAS];
};

// Fill a CamTable on the host. Returns false on bad arguments. With rec_offsets (host, n_cams + 1
// non-decreasing values starting at 0) camera c's records are [rec_offsets[c], rec_offsets[c + 1])
// and rec_stride is stored as 0 (packed segments); otherwise camera c's records start at c * rec_stride.
bool make_cam_table(const dass_camera* cams, int n_cams, int tile, long long rec_stride, CamTable* out,
                    const int64_t* rec_offsets = nullptr);

__device__ __forceinline__ int cam_of_tile(const CamTable& ct, int tile_id) {
    int lo = 0, hi = ct.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ct.c[mid].tile_base <= tile_id) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Camera of a record: a division for a uniform record stride, else the last camera whose segment
// starts at or before the record (empty segments share their start with the next camera's).
__device__ __forceinline__ int cam_of_record(const CamTable& ct, long long rec) {
    if (ct.rec_stride > 0) return (int)(rec / ct.rec_stride);
    int lo = 0, hi = ct.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ct.c[mid].rec_base <= rec) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ----------------------------------------------------------------- alpha (shared fwd/bwd)

// Splat as staged in shared memory for the compositing kernels.
//   A = (u, v, a', c') with a' = a * kNegHalfLog2e, c' = c * kNegHalfLog2e
//   B = (b2', o, r, g) with b2' = 2 b * kNegHalfLog2e;  blue separately.
// q' = a' dx^2 + b2' dx dy + c' dy^2 = -(d^T conic d)/2 * log2(e); G = 2^q'.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Explicit round-to-nearest intrinsics fix the operation sequence (no contraction choices
// by the compiler), so the same pixel/splat pair yields the same alpha in every kernel.
// q' is evaluated as dy (c' dy + B) + A with the column terms B = b2' dx and A = (a' dx) dx,
// which every pixel of a column shares (the compositing kernels compute them once per entry).
__device__ __forceinline__ float splat_gauss(float ap, float b2p, float cp, float dx, float dy) {
    const float B = __fmul_rn(b2p, dx);
    const float A = __fmul_rn(__fmul_rn(ap, dx), dx);
    return ex2_approx(__fmaf_rn(dy, __fmaf_rn(cp, dy, B), A));
}

__device__ __forceinline__ float splat_alpha(float o, float G) {
    return fminf(kAlphaMax, __fmul_rn(o, G));
}

// Packed FP32x2 forms (sm_100+ two-lane add/mul/fma, round-to-nearest on each lane): the same
// operation sequence as splat_gauss for two pixels at once, bit-identical lane by lane.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b, one rounding
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 one_minus2(float2 a) { return sub2(make_float2(1.f, 1.f), a); }

// Column terms (A, B) of splat_gauss for a packed column pair dx.
__device__ __forceinline__ void splat_column2(float2 ap, float2 b2p, float2 dx, float2& A, float2& B) {
    B = __fmul2_rn(b2p, dx);
    A = __fmul2_rn(__fmul2_rn(ap, dx), dx);
}
__device__ __forceinline__ float2 splat_gauss2(float2 cp, float2 dy, float2 A, float2 B) {
    const float2 q = __ffma2_rn(dy, __ffma2_rn(cp, dy, B), A);
    return make_float2(ex2_approx(q.x), ex2_approx(q.y));
}

// Does the footprint F = (a, b, c, k2) of a splat centred at (u, v) = -(nu, nv) reach the
// rectangle of pixel centres [bx, bx + wm1] x [by, by + hm1]? Ellipse-rectangle test: the quadratic
// form is evaluated at a point of each edge facing the centre (the clamped 1-D minimiser, computed
// with a fast division); any point of the rectangle gives an upper bound of its minimum, so a
// splat is culled only if every pixel of the rectangle is outside its footprint (up to k2's
// slack). Used to cull staged splats per warp block in the compositing kernels.
__device__ __forceinline__ bool footprint_reaches_rect(float nu, float nv, const float4 F, float bx, float by,
                                                       float wm1, float hm1) {
    if (F.w < 0.f) return false;
    const float x0 = bx + nu, x1 = (bx + wm1) + nu, y0 = by + nv, y1 = (by + hm1) + nv;
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

// ----------------------------------------------------------------- real SH (degree <= 3)

// Real spherical harmonics without the Condon-Shortley phase, k = l*l + l + m. Constants are
// K_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0) multiplied by the
// constant factor of d^|m| P_l / dz^|m|, written out per basis function:
//   Y00 = 1/(2 sqrt(pi));  Y1m = sqrt(3/(4 pi)) (y, z, x);
//   Y2,-2 = sqrt(15/(4 pi)) xy;  Y2,-1 = sqrt(15/(4 pi)) yz;  Y20 = sqrt(5/(16 pi)) (3z^2 - 1);
//   Y21 = sqrt(15/(4 pi)) xz;  Y22 = sqrt(15/(16 pi)) (x^2 - y^2);
//   Y3,-3 = sqrt(35/(32 pi)) y(3x^2 - y^2);  Y3,-2 = sqrt(105/(4 pi)) xyz;
//   Y3,-1 = sqrt(21/(32 pi)) y(5z^2 - 1);  Y30 = sqrt(7/(16 pi)) z(5z^2 - 3);
//   Y31 = sqrt(21/(32 pi)) x(5z^2 - 1);  Y32 = sqrt(105/(16 pi)) z(x^2 - y^2);
//   Y33 = sqrt(35/(32 pi)) x(x^2 - 3y^2).
constexpr float kY00 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.09254843059207907f;   // sqrt(15/(4 pi))
constexpr float kY20 = 0.31539156525252005f;   // sqrt(5/(16 pi))
constexpr float kY22 = 0.54627421529603953f;   // sqrt(15/(16 pi))
constexpr float kY33 = 0.59004358992664352f;   // sqrt(35/(32 pi))
constexpr float kY32n = 2.89061144264055405f;  // sqrt(105/(4 pi))
constexpr float kY31 = 0.45704579946446573f;   // sqrt(21/(32 pi))
constexpr float kY30 = 0.37317633259011540f;   // sqrt(7/(16 pi))
constexpr float kY32 = 1.44530572132027738f;   // sqrt(105/(16 pi))

// Basis values Y[0..K) for unit direction (x, y, z).
__device__ __forceinline__ void sh_eval_basis(int deg, float x, float y, float z, float* Y) {
    Y[0] = kY00;
    if (deg < 1) return;
    Y[1] = kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = kY1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;
    Y[5] = kY2a * y * z;
    Y[6] = kY20 * (3.f * zz - 1.f);
    Y[7] = kY2a * x * z;
    Y[8] = kY22 * (xx - yy);
    if (deg < 3) return;
    Y[9] = kY33 * y * (3.f * xx - yy);
    Y[10] = kY32n * x * y * z;
    Y[11] = kY31 * y * (5.f * zz - 1.f);
    Y[12] = kY30 * z * (5.f * zz - 3.f);
    Y[13] = kY31 * x * (5.f * zz - 1.f);
    Y[14] = kY32 * z * (xx - yy);
    Y[15] = kY33 * x * (xx - 3.f * yy);
}

// Gradient of sum_k w_k Y_k(x,y,z) w.r.t. (x, y, z), treating (x, y, z) as free variables.
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, const float* w,
                                              float& gx, float& gy, float& gz) {
    gx = gy = gz = 0.f;
    if (deg < 1) return;
    gy += kY1 * w[1];
    gz += kY1 * w[2];
    gx += kY1 * w[3];
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    gx += kY2a * y * w[4];  gy += kY2a * x * w[4];
    gy += kY2a * z * w[5];  gz += kY2a * y * w[5];
    gz += kY20 * 6.f * z * w[6];
    gx += kY2a * z * w[7];  gz += kY2a * x * w[7];
    gx += kY22 * 2.f * x * w[8];  gy -= kY22 * 2.f * y * w[8];
    if (deg < 3) return;
    // Y9 = c y (3x^2 - y^2)
    gx += kY33 * 6.f * x * y * w[9];
    gy += kY33 * (3.f * xx - 3.f * yy) * w[9];
    // Y10 = c xyz
    gx += kY32n * y * z * w[10]; gy += kY32n * x * z * w[10]; gz += kY32n * x * y * w[10];
    // Y11 = c y (5z^2 - 1)
    gy += kY31 * (5.f * zz - 1.f) * w[11]; gz += kY31 * 10.f * y * z * w[11];
    // Y12 = c z (5z^2 - 3) = c (5z^3 - 3z)
    gz += kY30 * (15.f * zz - 3.f) * w[12];
    // Y13 = c x (5z^2 - 1)
    gx += kY31 * (5.f * zz - 1.f) * w[13]; gz += kY31 * 10.f * x * z * w[13];
    // Y14 = c z (x^2 - y^2)
    gx += kY32 * 2.f * x * z * w[14]; gy -= kY32 * 2.f * y * z * w[14]; gz += kY32 * (xx - yy) * w[14];
    // Y15 = c x (x^2 - 3y^2) = c (x^3 - 3 x y^2)
    gx += kY33 * (3.f * xx - 3.f * yy) * w[15]; gy -= kY33 * 6.f * x * y * w[15];
}

// ----------------------------------------------------------------- quaternions

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// ----------------------------------------------------------------- tile rectangle (FP32)

// 1 / tile for the bin sizes 8, 16, 32 (the tables accept no others): a power of two, so x * (1 /
// tile) is the same correctly rounded number as x / tile, without a division.
__device__ __forceinline__ float inv_tile(int tile) { return tile == 8 ? 0.125f : tile == 16 ? 0.0625f : 0.03125f; }

// [x0, x1] x [y0, y1] tiles of the square [u-r, u+r] x [v-r, v+r]; empty if x0 > x1 or y0 > y1.
__device__ __forceinline__ void tile_rect(float u, float v, int r, int tiles_x, int tiles_y, int tile,
                                          int& x0, int& x1, int& y0, int& y1) {
    float rf = (float)r;
    x0 = max(0, (int)floorf(__fmul_rn(__fsub_rn(u, rf), inv_tile(tile))));
    x1 = min(tiles_x - 1, (int)floorf(__fmul_rn(__fadd_rn(u, rf), inv_tile(tile))));
    y0 = max(0, (int)floorf(__fmul_rn(__fsub_rn(v, rf), inv_tile(tile))));
    y1 = min(tiles_y - 1, (int)floorf(__fmul_rn(__fadd_rn(v, rf), inv_tile(tile))));
}

__device__ __forceinline__ int tile_count(float u, float v, int r, int tiles_x, int tiles_y, int tile) {
    if (r <= 0) return 0;
    int x0, x1, y0, y1;
    tile_rect(u, v, r, tiles_x, tiles_y, tile, x0, x1, y0, y1);
    if (x0 > x1 || y0 > y1) return 0;
    return (x1 - x0 + 1) * (y1 - y0 + 1);
}

// ----------------------------------------------------------------- ellipse footprint (FP32)

// The alpha >= 1/255 footprint of a splat is the ellipse d^T conic d <= k2 with
// k2 = 2 ln(255 o) + kRadiusSlack around (u, v). Its axis-aligned bounding box has half-extents
// sqrt(k2 Sigma_xx), sqrt(k2 Sigma_yy) with Sigma = conic^-1 (Sigma_xx = c/det, Sigma_yy = a/det).
struct Footprint {
    float u, v, a, b, c, k2, ex, ey;
};

// k2 of the footprint, or -1 if the splat has none (opacity <= 1/255 or a degenerate conic).
__device__ __forceinline__ float footprint_k2(float a, float b, float c, float o) {
    if (!(255.f * o > 1.f)) return -1.f;
    float det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
    if (!(det > 0.f)) return -1.f;
    return __fadd_rn(__fmul_rn(2.f, logf(__fmul_rn(255.f, o))), kRadiusSlack);
}

__device__ __forceinline__ bool footprint_of(float u, float v, float a, float b, float c, float o, Footprint& f) {
    if (!(255.f * o > 1.f)) return false;
    float det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
    if (!(det > 0.f)) return false;
    f.u = u; f.v = v; f.a = a; f.b = b; f.c = c;
    f.k2 = footprint_k2(a, b, c, o);
    f.ex = __fsqrt_rn(__fdiv_rn(__fmul_rn(f.k2, c), det));
    f.ey = __fsqrt_rn(__fdiv_rn(__fmul_rn(f.k2, a), det));
    return true;
}

// Candidate tiles from the bounding box, clamped to the camera's tile grid.
__device__ __forceinline__ void footprint_tiles(const Footprint& f, int tiles_x, int tiles_y, int tile, int& x0, int& x1,
                                                int& y0, int& y1) {
    x0 = max(0, (int)floorf(__fmul_rn(__fsub_rn(f.u, f.ex), inv_tile(tile))));
    x1 = min(tiles_x - 1, (int)floorf(__fmul_rn(__fadd_rn(f.u, f.ex), inv_tile(tile))));
    y0 = max(0, (int)floorf(__fmul_rn(__fsub_rn(f.v, f.ey), inv_tile(tile))));
    y1 = min(tiles_y - 1, (int)floorf(__fmul_rn(__fadd_rn(f.v, f.ey), inv_tile(tile))));
}

// Tiles of row ty that the footprint reaches. The slice of the ellipse over the band of pixel
// rows dy in [ya, yb] (offsets from v) projects onto an x-interval [L, R]: its right end is the
// ellipse's rightmost point (+ex, -b ex / c) when that lies in the band, otherwise the right end
// of the ellipse's chord on the band edge nearest to it (the right boundary is concave in dy);
// the left end likewise. A tile of the row is reached iff its pixel-centre columns meet [L, R].
// Returns false if the band misses the ellipse.
__device__ __forceinline__ bool footprint_row(const Footprint& f, int ty, int tile, int tiles_x, int& tx0, int& tx1) {
    const float B = (float)tile;
    const float ya = __fsub_rn((float)(ty * tile), f.v);
    const float yb = __fsub_rn((float)(ty * tile + tile - 1), f.v);
    const float det = __fsub_rn(__fmul_rn(f.a, f.c), __fmul_rn(f.b, f.b));
    const float ak2 = __fmul_rn(f.a, f.k2);
    const float dyr = __fdiv_rn(-__fmul_rn(f.b, f.ex), f.c);   // dy of the rightmost point
    float R, L;
    if (dyr >= ya && dyr <= yb) {
        R = f.ex;
    } else {
        const float yy = dyr < ya ? ya : yb;
        const float disc = __fsub_rn(ak2, __fmul_rn(det, __fmul_rn(yy, yy)));
        if (disc < 0.f) return false;
        R = __fdiv_rn(__fadd_rn(-__fmul_rn(f.b, yy), __fsqrt_rn(disc)), f.a);
    }
    const float dyl = -dyr;                                     // dy of the leftmost point
    if (dyl >= ya && dyl <= yb) {
        L = -f.ex;
    } else {
        const float yy = dyl < ya ? ya : yb;
        const float disc = __fsub_rn(ak2, __fmul_rn(det, __fmul_rn(yy, yy)));
        if (disc < 0.f) return false;
        L = __fdiv_rn(__fsub_rn(-__fmul_rn(f.b, yy), __fsqrt_rn(disc)), f.a);
    }
    tx0 = max(0, (int)ceilf(__fmul_rn(__fsub_rn(__fadd_rn(f.u, L), B - 1.f), inv_tile(tile))));
    tx1 = min(tiles_x - 1, (int)floorf(__fmul_rn(__fadd_rn(f.u, R), inv_tile(tile))));
    return tx0 <= tx1;
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace dass
