// Projection of Gaussians into all cameras (App. A.1) and its backward; densification
// statistics (Sec. 3.4). Gaussian-major: one thread loads a Gaussian's parameters once and
// loops over the cameras, so parameters are read once per iteration for every view.
#include "common.cuh"

namespace dass {

namespace {

struct Params {
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logit;
    const float* sh;
    const uint8_t* keep;
};

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + __expf(-x)); }

// Load the K*3 SH coefficients of Gaussian g (vectorised when rows are 16-byte multiples).
template <int K>
__device__ __forceinline__ void load_sh(const float* sh, long long g, float* c) {
    const float* row = sh + g * (3 * K);
    if constexpr ((3 * K) % 4 == 0) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int i = 0; i < (3 * K) / 4; ++i) {
            float4 v = __ldg(r4 + i);
            c[4 * i] = v.x; c[4 * i + 1] = v.y; c[4 * i + 2] = v.z; c[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 3 * K; ++i) c[i] = __ldg(row + i);
    }
}

// Everything of the forward projection of one Gaussian in one camera that the backward
// needs again.
struct Proj {
    float X, Y, Z;        // camera space
    float T[6];           // J W, 2x3 row-major
    float a, b, c;        // Sigma_2D (with low-pass)
    float det;
    float u, v;
};

__device__ __forceinline__ void project_one(const CamInfo& cam, const float* p, const float* Sig, Proj& P) {
    const float* R = cam.R;
    P.X = R[0] * p[0] + R[1] * p[1] + R[2] * p[2] + cam.t[0];
    P.Y = R[3] * p[0] + R[4] * p[1] + R[5] * p[2] + cam.t[1];
    P.Z = R[6] * p[0] + R[7] * p[1] + R[8] * p[2] + cam.t[2];
    float iz = 1.f / P.Z;
    float iz2 = iz * iz;
    float j00 = cam.fx * iz, j02 = -cam.fx * P.X * iz2;
    float j11 = cam.fy * iz, j12 = -cam.fy * P.Y * iz2;
    // T = J W
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P.T[k] = j00 * R[k] + j02 * R[6 + k];
        P.T[3 + k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    // Sigma symmetric: Sig = (s00, s01, s02, s11, s12, s22)
    float m[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float* t = P.T + 3 * r;
        m[r][0] = t[0] * Sig[0] + t[1] * Sig[1] + t[2] * Sig[2];
        m[r][1] = t[0] * Sig[1] + t[1] * Sig[3] + t[2] * Sig[4];
        m[r][2] = t[0] * Sig[2] + t[1] * Sig[4] + t[2] * Sig[5];
    }
    P.a = m[0][0] * P.T[0] + m[0][1] * P.T[1] + m[0][2] * P.T[2] + kLowPass;
    P.b = m[0][0] * P.T[3] + m[0][1] * P.T[4] + m[0][2] * P.T[5];
    P.c = m[1][0] * P.T[3] + m[1][1] * P.T[4] + m[1][2] * P.T[5] + kLowPass;
    P.det = P.a * P.c - P.b * P.b;
    P.u = cam.fx * P.X * iz + cam.cx;
    P.v = cam.fy * P.Y * iz + cam.cy;
}

// Opacity-aware radius: ceil(sqrt(lambda_max) * sqrt(2 ln(255 o) + slack)); 0 if 255 o <= 1.
__device__ __forceinline__ int footprint_radius(float a, float b, float c, float o) {
    if (!(255.f * o > 1.f)) return 0;
    float mid = 0.5f * (a + c);
    float disc = fmaxf(mid * mid - (a * c - b * b), 0.f);
    float lam = mid + sqrtf(disc);
    float k2 = 2.f * logf(255.f * o) + kRadiusSlack;
    return (int)ceilf(sqrtf(lam) * sqrtf(k2));
}

// Activated attributes of Gaussian g: mean, opacity, 3D covariance (6 unique entries), SH.
template <int K>
__device__ __forceinline__ void gaussian_setup(const Params& prm, long long g, float* p, float& o, float* Sig,
                                               float* coef) {
    float ls[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) { p[i] = __ldg(prm.means + 3 * g + i); ls[i] = __ldg(prm.log_scales + 3 * g + i); }
    float4 q4 = __ldg(reinterpret_cast<const float4*>(prm.quats) + g);
    float kp = prm.keep ? (float)prm.keep[g] : 1.f;
    o = sigmoidf_(__ldg(prm.opacity_logit + g)) * kp;
    float s[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = __expf(ls[i]) * kp;
    float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    float R[9];
    quat_to_rot(q4.x * qn, q4.y * qn, q4.z * qn, q4.w * qn, R);
    // M = R diag(s); Sigma = M M^T
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * s[c];
    Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    load_sh<K>(prm.sh, g, coef);
}

// Project one Gaussian into one camera and write its record (culled records: radius 0).
template <int K>
// Writes the record and returns whether the densification statistics count it: radius > 0 and the
// square of that radius around (u, v) reaching [0, W - 1] x [0, H - 1] (the rule the statistics
// kernel applies to a stored record).
__device__ __forceinline__ bool write_record(const CamInfo& cam, int tile, int deg, const float* p, float o,
                                             const float* Sig, const float* coef, dass_splat* __restrict__ rec) {
    Proj P;
    project_one(cam, p, Sig, P);
    int radius = 0;
    int tiles = 0;
    float conic_a = 0.f, conic_b = 0.f, conic_c = 0.f;
    float rgb[3] = {0.f, 0.f, 0.f};
    if (P.Z > kNear && P.det > 0.f) {
        float idet = 1.f / P.det;
        conic_a = P.c * idet;
        conic_b = -P.b * idet;
        conic_c = P.a * idet;
        radius = footprint_radius(P.a, P.b, P.c, o);
        tiles = tile_count(P.u, P.v, radius, cam.tiles_x, cam.tiles_y, tile);
        if (tiles == 0) radius = 0;
    }
    if (radius > 0) {
        float dx = p[0] - cam.campos[0], dy = p[1] - cam.campos[1], dz = p[2] - cam.campos[2];
        float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Yb[16];
        sh_eval_basis(deg, dx, dy, dz, Yb);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += coef[3 * k + ch] * Yb[k];
            rgb[ch] = fmaxf(acc, 0.f);
        }
    }
    float4* dst = reinterpret_cast<float4*>(rec);
    if (radius > 0) {
        dst[0] = make_float4(P.u, P.v, conic_a, conic_b);
        dst[1] = make_float4(conic_c, o, rgb[0], rgb[1]);
        dst[2] = make_float4(rgb[2], P.Z, __int_as_float(radius), __int_as_float(tiles));
    } else {
        dst[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        dst[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        dst[2] = make_float4(0.f, P.Z, __int_as_float(0), __int_as_float(0));
    }
    const float rf = (float)radius;
    return radius > 0 && !(P.u + rf < 0.f || P.u - rf > (float)(cam.W - 1) || P.v + rf < 0.f ||
                           P.v - rf > (float)(cam.H - 1));
}

// Thread i projects Gaussian i, or Gaussian rows[i] for i < *n_rows when a row list is given (the
// other records keep their contents). vis (optional): bit c of vis[g] = camera c's record counts in
// the densification statistics.
template <int K>
__global__ void __launch_bounds__(128) preprocess_kernel(long long n, int deg, Params prm, CamTable ct,
                                                         dass_splat* __restrict__ out, const int* __restrict__ rows,
                                                         const long long* __restrict__ n_rows,
                                                         unsigned long long* __restrict__ vis) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long g = i;
    if (rows) {
        if (i >= *n_rows) return;
        g = rows[i];
    }
    if (g < 0 || g >= n) return;
    float p[3], o, Sig[6], coef[3 * K];
    gaussian_setup<K>(prm, g, p, o, Sig, coef);
    unsigned long long m = 0ull;
    for (int ci = 0; ci < ct.n; ++ci)
        if (write_record<K>(ct.c[ci], ct.tile, deg, p, o, Sig, coef, out + ct.c[ci].rec_base + g))
            m |= 1ull << ci;
    if (vis) vis[g] = m;
}

// Serving form: camera c shows its own scene; thread (g, c) writes record rec_base_c + g. With a
// uniform record stride the records g in [n_c, rec_stride) are written as culled (radius 0); with
// packed segments (rec_stride 0) camera c has exactly n_c records.
struct SceneTable {
    Params prm[DASS_MAX_CAMERAS];
    long long n[DASS_MAX_CAMERAS];
};

template <int K>
__global__ void __launch_bounds__(128) preprocess_scenes_kernel(int deg, SceneTable st, CamTable ct,
                                                                dass_splat* __restrict__ out) {
    const int ci = blockIdx.y;
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (ct.rec_stride > 0 ? ct.rec_stride : st.n[ci])) return;
    const CamInfo& cam = ct.c[ci];
    dass_splat* rec = out + cam.rec_base + g;
    if (g >= st.n[ci]) {
        float4* dst = reinterpret_cast<float4*>(rec);
        dst[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        dst[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        dst[2] = make_float4(0.f, 0.f, __int_as_float(0), __int_as_float(0));
        return;
    }
    float p[3], o, Sig[6], coef[3 * K];
    gaussian_setup<K>(st.prm[ci], g, p, o, Sig, coef);
    write_record<K>(cam, ct.tile, deg, p, o, Sig, coef, rec);
}

// Internal gradient flag (beyond the public DASS_GRAD_* set): dL/dkeep of the inheritance mask.
constexpr unsigned kGradKeep = 1u << 8;

struct Grads {
    float* d_means;
    float* d_log_scales;
    float* d_quats;
    float* d_opacity_logit;
    float* d_sh;
    float* d_keep;
};

// Gradient of the projection for the rows [rows] (or all rows): one thread per row, cameras in
// order, each camera's record radius and splat gradient requested one camera ahead.
template <int K>
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(long long n, int deg, Params prm, CamTable ct,
                                                             const dass_splat* __restrict__ splats,
                                                             const dass_splat_grad* __restrict__ gsp,
                                                             const int* __restrict__ rows, long long n_rows,
                                                             unsigned flags, int accumulate, Grads out) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    long long g = rows ? (long long)rows[r] : r;
    float p[3], ls[3], q[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) { p[i] = __ldg(prm.means + 3 * g + i); ls[i] = __ldg(prm.log_scales + 3 * g + i); }
    float4 q4 = __ldg(reinterpret_cast<const float4*>(prm.quats) + g);
    q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
    float kp = prm.keep ? (float)prm.keep[g] : 1.f;
    float o_raw = sigmoidf_(__ldg(prm.opacity_logit + g));
    float s[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = __expf(ls[i]) * kp;
    float qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float qh[4] = {q[0] / qnorm, q[1] / qnorm, q[2] / qnorm, q[3] / qnorm};
    float R[9];
    quat_to_rot(qh[0], qh[1], qh[2], qh[3], R);
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[3 * a + b] = R[3 * a + b] * s[b];
    float Sig[6];
    Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    const bool want_sh = (flags & DASS_GRAD_SH) && out.d_sh;
    const bool want_geo = (flags & (DASS_GRAD_MEANS | DASS_GRAD_SCALES | DASS_GRAD_QUATS | kGradKeep)) != 0;
    float coef[3 * K];
    load_sh<K>(prm.sh, g, coef);
    float dcoef[3 * K];
#pragma unroll
    for (int i = 0; i < 3 * K; ++i) dcoef[i] = 0.f;
    float dp[3] = {0.f, 0.f, 0.f};
    float dSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // gradient w.r.t. symmetric entries (off-diag counted once)
    float d_o = 0.f;

    // the next camera's radius and splat gradient are requested before this camera's work
    int nx_radius = 0;
    float4 nx0 = make_float4(0.f, 0.f, 0.f, 0.f), nx1 = nx0, nx2 = nx0;
    if (ct.n > 0) {
        const long long rec = ct.c[0].rec_base + g;
        nx_radius = __float_as_int(__ldg(reinterpret_cast<const float*>(splats + rec) + 10));
        const float4* gp = reinterpret_cast<const float4*>(gsp + rec);
        nx0 = __ldg(gp); nx1 = __ldg(gp + 1); nx2 = __ldg(gp + 2);
    }
    for (int ci = 0; ci < ct.n; ++ci) {
        const CamInfo& cam = ct.c[ci];
        const int radius = nx_radius;
        const float4 g0 = nx0, g1 = nx1, g2 = nx2;
        if (ci + 1 < ct.n) {
            const long long rn = ct.c[ci + 1].rec_base + g;
            nx_radius = __float_as_int(__ldg(reinterpret_cast<const float*>(splats + rn) + 10));
            const float4* gp = reinterpret_cast<const float4*>(gsp + rn);
            nx0 = __ldg(gp); nx1 = __ldg(gp + 1); nx2 = __ldg(gp + 2);
        }
        if (radius <= 0) continue;
        float du = g0.x, dv = g0.y, dA = g0.z, dB = g0.w, dC = g1.x;
        float dop = g1.y;
        float drgb[3] = {g1.z, g1.w, g2.x};
        d_o += dop;
        // ---- colour: rgb = max(sum_k coef_k Y_k(d) + 0.5, 0), d = normalize(p - campos)
        float vx = p[0] - cam.campos[0], vy = p[1] - cam.campos[1], vz = p[2] - cam.campos[2];
        float vlen = sqrtf(vx * vx + vy * vy + vz * vz);
        float dx = vx / vlen, dy = vy / vlen, dz = vz / vlen;
        float Yb[16];
        sh_eval_basis(deg, dx, dy, dz, Yb);
        float wdir[16];
#pragma unroll
        for (int k = 0; k < K; ++k) wdir[k] = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += coef[3 * k + ch] * Yb[k];
            float gch = acc < 0.f ? 0.f : drgb[ch];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dcoef[3 * k + ch] += gch * Yb[k];
                wdir[k] += gch * coef[3 * k + ch];
            }
        }
        if (K > 1 && (flags & DASS_GRAD_MEANS)) {
            float gx, gy, gz;
            sh_basis_grad(deg, dx, dy, dz, wdir, gx, gy, gz);
            float dot = gx * dx + gy * dy + gz * dz;
            dp[0] += (gx - dot * dx) / vlen;
            dp[1] += (gy - dot * dy) / vlen;
            dp[2] += (gz - dot * dz) / vlen;
        }
        if (!want_geo) continue;
        // ---- geometry
        Proj P;
        project_one(cam, p, Sig, P);
        float a = P.a, b = P.b, c = P.c, det = P.det;
        float id2 = 1.f / (det * det);
        // conic (A, B, C) = (c, -b, a) / det
        float da = (-c * c * dA + b * c * dB - b * b * dC) * id2;
        float db = (2.f * b * c * dA - (a * c + b * b) * dB + 2.f * a * b * dC) * id2;
        float dc = (-b * b * dA + a * b * dB - a * a * dC) * id2;
        // Sigma_2D = T Sigma T^T + 0.3 I; G2 = [[da, db/2], [db/2, dc]]
        float G00 = da, G01 = 0.5f * db, G11 = dc;
        const float* T = P.T;
        // dSigma = T^T G2 T (symmetric); accumulate entries with off-diagonals counted once:
        // dL/dSig_ij (i != j) = 2 (T^T G2 T)_ij
        float GT[2][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            GT[0][k] = G00 * T[k] + G01 * T[3 + k];
            GT[1][k] = G01 * T[k] + G11 * T[3 + k];
        }
        float S[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) S[i][j] = T[i] * GT[0][j] + T[3 + i] * GT[1][j];
        dSig[0] += S[0][0];
        dSig[1] += 2.f * S[0][1];
        dSig[2] += 2.f * S[0][2];
        dSig[3] += S[1][1];
        dSig[4] += 2.f * S[1][2];
        dSig[5] += S[2][2];
        // dL/dT = 2 G2 T Sigma
        float SigF[9] = {Sig[0], Sig[1], Sig[2], Sig[1], Sig[3], Sig[4], Sig[2], Sig[4], Sig[5]};
        float TS[2][3];
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                TS[r2][k] = T[3 * r2] * SigF[k] + T[3 * r2 + 1] * SigF[3 + k] + T[3 * r2 + 2] * SigF[6 + k];
        float dT[2][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dT[0][k] = 2.f * (G00 * TS[0][k] + G01 * TS[1][k]);
            dT[1][k] = 2.f * (G01 * TS[0][k] + G11 * TS[1][k]);
        }
        // T = J W  ->  dJ = dT W^T (only the J entries that vary matter)
        const float* W = cam.R;
        float dJ00 = dT[0][0] * W[0] + dT[0][1] * W[1] + dT[0][2] * W[2];
        float dJ02 = dT[0][0] * W[6] + dT[0][1] * W[7] + dT[0][2] * W[8];
        float dJ11 = dT[1][0] * W[3] + dT[1][1] * W[4] + dT[1][2] * W[5];
        float dJ12 = dT[1][0] * W[6] + dT[1][1] * W[7] + dT[1][2] * W[8];
        float iz = 1.f / P.Z, iz2 = iz * iz, iz3 = iz2 * iz;
        float dX = -cam.fx * iz2 * dJ02;
        float dY = -cam.fy * iz2 * dJ12;
        float dZ = -cam.fx * iz2 * dJ00 + 2.f * cam.fx * P.X * iz3 * dJ02 - cam.fy * iz2 * dJ11 +
                   2.f * cam.fy * P.Y * iz3 * dJ12;
        // mean2D
        dX += du * cam.fx * iz;
        dY += dv * cam.fy * iz;
        dZ += -du * cam.fx * P.X * iz2 - dv * cam.fy * P.Y * iz2;
        // X_c = W p + t
        dp[0] += W[0] * dX + W[3] * dY + W[6] * dZ;
        dp[1] += W[1] * dX + W[4] * dY + W[7] * dZ;
        dp[2] += W[2] * dX + W[5] * dY + W[8] * dZ;
    }
    long long orow = r;
    if (flags & DASS_GRAD_OPACITY && out.d_opacity_logit) {
        float v = d_o * kp * o_raw * (1.f - o_raw);
        out.d_opacity_logit[orow] = accumulate ? out.d_opacity_logit[orow] + v : v;
    }
    if (want_sh) {
        float* d = out.d_sh + orow * (3 * K);
#pragma unroll
        for (int i = 0; i < 3 * K; ++i) d[i] = accumulate ? d[i] + dcoef[i] : dcoef[i];
    }
    if (flags & DASS_GRAD_MEANS && out.d_means) {
        float* d = out.d_means + 3 * orow;
#pragma unroll
        for (int i = 0; i < 3; ++i) d[i] = accumulate ? d[i] + dp[i] : dp[i];
    }
    // dL/dkeep of the inheritance mask (Eq. 1: o_r = keep o, s_r = keep s) at the current keep
    float d_keep = d_o * o_raw;
    if (flags & (DASS_GRAD_SCALES | DASS_GRAD_QUATS | kGradKeep)) {
        // Sigma = M M^T: dM = 2 dSigmaFull M with dSigmaFull the symmetric matrix whose
        // off-diagonals are half the accumulated (once-counted) values.
        float D[9] = {dSig[0], 0.5f * dSig[1], 0.5f * dSig[2], 0.5f * dSig[1], dSig[3], 0.5f * dSig[4],
                      0.5f * dSig[2], 0.5f * dSig[4], dSig[5]};
        float dM[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                dM[3 * i + j] = 2.f * (D[3 * i] * M[j] + D[3 * i + 1] * M[3 + j] + D[3 * i + 2] * M[6 + j]);
        if (flags & DASS_GRAD_SCALES && out.d_log_scales) {
            float* d = out.d_log_scales + 3 * orow;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float ds = dM[j] * R[j] + dM[3 + j] * R[3 + j] + dM[6 + j] * R[6 + j];
                float v = ds * s[j];   // s already includes the keep mask: d s_r / d log s = s_r
                d[j] = accumulate ? d[j] + v : v;
            }
        }
        if (flags & kGradKeep) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
                d_keep += (dM[j] * R[j] + dM[3 + j] * R[3 + j] + dM[6 + j] * R[6 + j]) * __expf(ls[j]);
        }
        if (flags & DASS_GRAD_QUATS && out.d_quats) {
            float G[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) G[3 * i + j] = dM[3 * i + j] * s[j];
            float w = qh[0], x = qh[1], y = qh[2], z = qh[3];
            float dw = 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
            float dx = 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] -
                              2.f * x * G[8]);
            float dy = 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] -
                              2.f * y * G[8]);
            float dz = 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] +
                              x * G[6] + y * G[7]);
            // q_hat = q / |q|
            float dot = dw * w + dx * x + dy * y + dz * z;
            float v[4] = {(dw - dot * w) / qnorm, (dx - dot * x) / qnorm, (dy - dot * y) / qnorm,
                          (dz - dot * z) / qnorm};
            float* d = out.d_quats + 4 * orow;
#pragma unroll
            for (int i = 0; i < 4; ++i) d[i] = accumulate ? d[i] + v[i] : v[i];
        }
    }
    if ((flags & kGradKeep) && out.d_keep) out.d_keep[orow] = accumulate ? out.d_keep[orow] + d_keep : d_keep;
}

__global__ void densify_stats_kernel(long long n, CamTable ct, const dass_splat* __restrict__ splats,
                                     const dass_splat_grad* __restrict__ gsp, float* accum, int* count) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float sum = 0.f;
    int cnt = 0;
    for (int ci = 0; ci < ct.n; ++ci) {
        const CamInfo& cam = ct.c[ci];
        long long rec = cam.rec_base + g;
        const float4* sp = reinterpret_cast<const float4*>(splats + rec);
        float4 s0 = __ldg(sp);
        float4 s2 = __ldg(sp + 2);
        int r = __float_as_int(s2.z);
        if (r <= 0) continue;
        float rf = (float)r;
        if (s0.x + rf < 0.f || s0.x - rf > (float)(cam.W - 1) || s0.y + rf < 0.f || s0.y - rf > (float)(cam.H - 1))
            continue;
        float2 gm = __ldg(reinterpret_cast<const float2*>(gsp + rec));
        float gu = gm.x * (0.5f * cam.W), gv = gm.y * (0.5f * cam.H);
        sum += sqrtf(gu * gu + gv * gv);
        cnt += 1;
    }
    if (cnt) {
        accum[g] += sum;
        count[g] += cnt;
    }
}

// Densification statistics from the visibility masks the preprocess wrote: only the counted
// cameras' gradients are read (8 of the 48 bytes of each), eight cameras' loads issued at a time.
// The sum runs over the cameras in order, as in densify_stats_kernel, so the results are equal.
__global__ void densify_stats_vis_kernel(long long n, CamTable ct, const unsigned long long* __restrict__ vis,
                                         const dass_splat_grad* __restrict__ gsp, float* accum, int* count) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const unsigned long long m = vis[g];
    if (!m) return;
    float sum = 0.f;
    int cnt = 0;
    for (int c0 = 0; c0 < ct.n; c0 += 8) {
        float2 gm[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int ci = c0 + k;
            gm[k] = (ci < ct.n && ((m >> ci) & 1ull))
                        ? __ldg(reinterpret_cast<const float2*>(gsp + ct.c[ci].rec_base + g))
                        : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int ci = c0 + k;
            if (ci < ct.n && ((m >> ci) & 1ull)) {
                const CamInfo& cam = ct.c[ci];
                const float gu = gm[k].x * (0.5f * cam.W), gv = gm[k].y * (0.5f * cam.H);
                sum += sqrtf(gu * gu + gv * gv);
                cnt += 1;
            }
        }
    }
    accum[g] += sum;
    count[g] += cnt;
}

template <int K>
int launch_pre(long long n, int deg, const Params& prm, const CamTable& ct, dass_splat* out, cudaStream_t st,
               const int* rows, const long long* n_rows, long long rows_cap, unsigned long long* vis) {
    int threads = 128;
    preprocess_kernel<K><<<div_up(rows ? rows_cap : n, threads), threads, 0, st>>>(n, deg, prm, ct, out, rows,
                                                                                    n_rows, vis);
    count_launch();
    return check_launch("preprocess_kernel");
}

template <int K>
int launch_pre_scenes(int deg, const SceneTable& stb, const CamTable& ct, long long rows, dass_splat* out,
                      cudaStream_t st) {
    dim3 grid(div_up(rows, 128), ct.n);
    preprocess_scenes_kernel<K><<<grid, 128, 0, st>>>(deg, stb, ct, out); count_launch();
    return check_launch("preprocess_scenes_kernel");
}

template <int K>
int launch_pre_bwd(long long n, int deg, const Params& prm, const CamTable& ct, const dass_splat* sp,
                   const dass_splat_grad* gsp, const int* rows, long long n_rows, unsigned flags, int acc,
                   const Grads& gr, cudaStream_t st) {
    constexpr int threads = 128;
    preprocess_bwd_kernel<K><<<div_up(n_rows, threads), threads, 0, st>>>(n, deg, prm, ct, sp, gsp, rows,
                                                                                  n_rows, flags, acc, gr);
    count_launch();
    return check_launch("preprocess_bwd_kernel");
}

}  // namespace

int preprocess_launch(long long n, int deg, const float* means, const float* log_scales, const float* quats,
                      const float* opacity_logit, const float* sh, const uint8_t* keep, const CamTable& ct,
                      dass_splat* splats, cudaStream_t st, const int* rows, const long long* n_rows,
                      long long rows_cap, unsigned long long* vis) {
    Params prm{means, log_scales, quats, opacity_logit, sh, keep};
    if (rows && (!n_rows || rows_cap <= 0)) return DASS_ERR_INVALID_ARG;
    if (vis && ct.n > 64) return DASS_ERR_INVALID_ARG;
    switch (deg) {
        case 0: return launch_pre<1>(n, deg, prm, ct, splats, st, rows, n_rows, rows_cap, vis);
        case 1: return launch_pre<4>(n, deg, prm, ct, splats, st, rows, n_rows, rows_cap, vis);
        case 2: return launch_pre<9>(n, deg, prm, ct, splats, st, rows, n_rows, rows_cap, vis);
        case 3: return launch_pre<16>(n, deg, prm, ct, splats, st, rows, n_rows, rows_cap, vis);
    }
    return DASS_ERR_INVALID_ARG;
}

int preprocess_scenes_launch(const dass_scene* scenes, int deg, const CamTable& ct, dass_splat* splats,
                             cudaStream_t st, long long n_max) {
    static thread_local SceneTable stb;
    for (int c = 0; c < ct.n; ++c) {
        stb.prm[c] = Params{scenes[c].means, scenes[c].log_scales, scenes[c].quats, scenes[c].opacity_logit,
                            scenes[c].sh, nullptr};
        stb.n[c] = scenes[c].n;
    }
    const long long rows = ct.rec_stride > 0 ? ct.rec_stride : n_max;   // threads per camera
    if (rows <= 0) return DASS_OK;
    switch (deg) {
        case 0: return launch_pre_scenes<1>(deg, stb, ct, rows, splats, st);
        case 1: return launch_pre_scenes<4>(deg, stb, ct, rows, splats, st);
        case 2: return launch_pre_scenes<9>(deg, stb, ct, rows, splats, st);
        case 3: return launch_pre_scenes<16>(deg, stb, ct, rows, splats, st);
    }
    return DASS_ERR_INVALID_ARG;
}

int preprocess_bwd_launch(long long n, int deg, const float* means, const float* log_scales, const float* quats,
                          const float* opacity_logit, const float* sh, const uint8_t* keep, const CamTable& ct,
                          const dass_splat* splats, const dass_splat_grad* gsp, const int* rows, long long n_rows,
                          unsigned flags, int accumulate, float* d_means, float* d_log_scales, float* d_quats,
                          float* d_opacity_logit, float* d_sh, float* d_keep, cudaStream_t st) {
    Params prm{means, log_scales, quats, opacity_logit, sh, keep};
    Grads gr{d_means, d_log_scales, d_quats, d_opacity_logit, d_sh, d_keep};
    if (d_keep) flags |= kGradKeep;
    if (n_rows <= 0) return DASS_OK;
    switch (deg) {
        case 0: return launch_pre_bwd<1>(n, deg, prm, ct, splats, gsp, rows, n_rows, flags, accumulate, gr, st);
        case 1: return launch_pre_bwd<4>(n, deg, prm, ct, splats, gsp, rows, n_rows, flags, accumulate, gr, st);
        case 2: return launch_pre_bwd<9>(n, deg, prm, ct, splats, gsp, rows, n_rows, flags, accumulate, gr, st);
        case 3: return launch_pre_bwd<16>(n, deg, prm, ct, splats, gsp, rows, n_rows, flags, accumulate, gr, st);
    }
    return DASS_ERR_INVALID_ARG;
}

int densify_stats_vis_launch(long long n, const CamTable& ct, const unsigned long long* vis,
                             const dass_splat_grad* gsp, float* accum, int* count, cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    densify_stats_vis_kernel<<<div_up(n, 256), 256, 0, st>>>(n, ct, vis, gsp, accum, count); count_launch();
    return check_launch("densify_stats_vis_kernel");
}

int densify_stats_launch(long long n, const CamTable& ct, const dass_splat* splats, const dass_splat_grad* gsp,
                         float* accum, int* count, cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    densify_stats_kernel<<<div_up(n, 256), 256, 0, st>>>(n, ct, splats, gsp, accum, count); count_launch();
    return check_launch("densify_stats_kernel");
}

}  // namespace dass
