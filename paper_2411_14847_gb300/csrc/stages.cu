// Per-Gaussian work of the DASS stages: dynamics-aware shift and its backward (Sec. 3.3),
// masked Adam, selective-inheritance copy (Sec. 3.2), and the error pass, Eq. 4 selection and
// spawn of error-guided densification (Sec. 3.4). All HBM-bound elementwise/gather kernels.
#include <cmath>

#include "common.cuh"

namespace dass {

int scan_u32_public(const uint32_t* in, uint32_t* out, const long long* len_dev, long long len_cap,
                    unsigned long long* partial, long long* total, cudaStream_t st);
size_t scan_partials_bytes(long long len);

namespace {

// ----------------------------------------------------------------- shift (Sec. 3.3)

__device__ __forceinline__ void qmul(const float* a, const float* b, float* o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

__global__ void shift_fwd_kernel(long long n_dyn, const int* __restrict__ idx, const float* __restrict__ off,
                                 const float* __restrict__ means, const float* __restrict__ quats,
                                 float* __restrict__ out_means, float* __restrict__ out_quats) {
    long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_dyn) return;
    long long n = idx[d];
    const float* o = off + 7 * d;
#pragma unroll
    for (int k = 0; k < 3; ++k) out_means[3 * n + k] = means[3 * n + k] + o[k];
    float4 q4 = reinterpret_cast<const float4*>(quats)[n];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    float qn = 1.f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float s[4] = {o[3], o[4], o[5], o[6]};
    float sn = 1.f / sqrtf(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) { q[k] *= qn; s[k] *= sn; }
    float r[4];
    qmul(q, s, r);
    reinterpret_cast<float4*>(out_quats)[n] = make_float4(r[0], r[1], r[2], r[3]);
}

__global__ void shift_bwd_kernel(long long n_dyn, const int* __restrict__ idx, const float* __restrict__ off,
                                 const float* __restrict__ quats, const float* __restrict__ dm,
                                 const float* __restrict__ dq, float* __restrict__ doff, float* __restrict__ dqin) {
    long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_dyn) return;
    long long n = idx[d];
    const float* o = off + 7 * d;
    float* g = doff + 7 * d;
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = dm[3 * d + k];
    float4 q4 = reinterpret_cast<const float4*>(quats)[n];
    float qn = 1.f / sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    float gq[4] = {dq[4 * d], dq[4 * d + 1], dq[4 * d + 2], dq[4 * d + 3]};
    // q' = L(q_hat) sigma_hat; dL/dsigma_hat = L(q_hat)^T dL/dq'
    float gs[4];
    gs[0] = w * gq[0] + x * gq[1] + y * gq[2] + z * gq[3];
    gs[1] = -x * gq[0] + w * gq[1] + z * gq[2] - y * gq[3];
    gs[2] = -y * gq[0] - z * gq[1] + w * gq[2] + x * gq[3];
    gs[3] = -z * gq[0] + y * gq[1] - x * gq[2] + w * gq[3];
    float s[4] = {o[3], o[4], o[5], o[6]};
    float len = sqrtf(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
    float sh[4] = {s[0] / len, s[1] / len, s[2] / len, s[3] / len};
    float dot = gs[0] * sh[0] + gs[1] * sh[1] + gs[2] * sh[2] + gs[3] * sh[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) g[3 + k] = (gs[k] - dot * sh[k]) / len;
    if (dqin) {
        // q' = q_hat x sigma_hat = R(sigma_hat) q_hat: dL/dq_hat = R(sigma_hat)^T dL/dq', then through
        // q_hat = q / |q|
        float gh[4];
        gh[0] = sh[0] * gq[0] + sh[1] * gq[1] + sh[2] * gq[2] + sh[3] * gq[3];
        gh[1] = -sh[1] * gq[0] + sh[0] * gq[1] - sh[3] * gq[2] + sh[2] * gq[3];
        gh[2] = -sh[2] * gq[0] + sh[3] * gq[1] + sh[0] * gq[2] - sh[1] * gq[3];
        gh[3] = -sh[3] * gq[0] - sh[2] * gq[1] + sh[1] * gq[2] + sh[0] * gq[3];
        float d2 = gh[0] * w + gh[1] * x + gh[2] * y + gh[3] * z;
        float qh[4] = {w, x, y, z};
#pragma unroll
        for (int k = 0; k < 4; ++k) dqin[4 * d + k] = (gh[k] - d2 * qh[k]) * qn;
    }
}

// ----------------------------------------------------------------- masked Adam

struct LR {
    float v[16];
};

__global__ void adam_kernel(long long n_sel, int width, const int* __restrict__ rows, float* __restrict__ p,
                            const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            const int* __restrict__ step_dev, LR lr, float b1, float b2, float eps) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_sel * width) return;
    long long r = e / width;
    int k = (int)(e - r * width);
    long long row = rows ? (long long)rows[r] : r;
    long long i = row * width + k;
    float t = (float)(*step_dev + 1);
    float bc1 = 1.f - powf(b1, t);
    float bc2 = 1.f - powf(b2, t);
    float gi = g[i];
    float mm = b1 * m[i] + (1.f - b1) * gi;
    float vv = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mm;
    v[i] = vv;
    p[i] = p[i] - lr.v[k] * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

__global__ void step_inc_kernel(int* step) { *step += 1; }

// ----------------------------------------------------------------- inheritance (Sec. 3.2)

__global__ void inherit_flags_kernel(long long n, const uint8_t* __restrict__ is_var, const float* __restrict__ m,
                                     int erase, uint32_t* __restrict__ fb, uint32_t* __restrict__ fv) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool var = is_var[i] != 0;
    fb[i] = var ? 0u : 1u;
    fv[i] = (var && !erase && (m == nullptr || m[i] > 0.f)) ? 1u : 0u;
}

// Rendering mask of the inheritance stage: keep = Quant(sigmoid(m)) = [m > 0] on var rows, 1 on
// base rows (Eq. 1).
__global__ void inherit_keep_kernel(long long n, const uint8_t* __restrict__ is_var, const float* __restrict__ m,
                                    uint8_t* __restrict__ keep) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keep[i] = (is_var[i] == 0 || m[i] > 0.f) ? 1 : 0;
}

// Straight-through gradient of the inheritance logits (App. B.2 STE on Eq. 2): the rendering
// uses m_op = Quant(sigmoid(m)) whose surrogate derivative is sigmoid'(m), and the mask loss
// lambda sum sigmoid(m) adds lambda sigmoid'(m); grad[rows[r]] = (d_keep[r] + lambda) s (1 - s).
// loss (optional) accumulates lambda * sum sigmoid(m) over the rows.
__global__ void inherit_mask_grad_kernel(long long n_rows, const int* __restrict__ rows, const float* __restrict__ m,
                                         const float* __restrict__ d_keep, float lambda, float* __restrict__ grad,
                                         double* loss) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float reg = 0.f;
    if (r < n_rows) {
        const long long g = rows ? (long long)rows[r] : r;
        const float sg = 1.f / (1.f + __expf(-m[g]));
        grad[g] = (d_keep[r] + lambda) * sg * (1.f - sg);
        reg = lambda * sg;
    }
    if (loss) {
        for (int o = 16; o > 0; o >>= 1) reg += __shfl_xor_sync(0xffffffffu, reg, o);
        if ((threadIdx.x & 31) == 0 && reg != 0.f) atomicAdd(loss, (double)reg);
    }
}

__global__ void inherit_scatter_kernel(long long n, int K3, const uint32_t* __restrict__ fb,
                                       const uint32_t* __restrict__ fv, const uint32_t* __restrict__ sb,
                                       const uint32_t* __restrict__ sv, const long long* __restrict__ totals,
                                       const float* means, const float* log_scales, const float* quats,
                                       const float* logit, const float* sh, float* o_means, float* o_log_scales,
                                       float* o_quats, float* o_logit, float* o_sh, uint8_t* o_var, int* remap,
                                       long long* n_out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nb = totals[0];
    if (i == 0) *n_out = nb + totals[1];
    if (i >= n) return;
    long long pos = -1;
    if (fb[i]) pos = sb[i];
    else if (fv[i]) pos = nb + sv[i];
    remap[i] = (int)pos;
    if (pos < 0) return;
    for (int k = 0; k < 3; ++k) { o_means[3 * pos + k] = means[3 * i + k]; o_log_scales[3 * pos + k] = log_scales[3 * i + k]; }
    reinterpret_cast<float4*>(o_quats)[pos] = reinterpret_cast<const float4*>(quats)[i];
    o_logit[pos] = logit[i];
    for (int k = 0; k < K3; ++k) o_sh[pos * K3 + k] = sh[i * K3 + k];
    o_var[pos] = fb[i] ? 0 : 1;
}

// ----------------------------------------------------------------- radix select (MSB first)

// Segments: keys[base[s] .. base[s] + len[s]); each round narrows the value of ascending rank
// rank[s] by 8 bits. State in device memory: prefix[s], rank[s] (rank within the values that
// share the prefix) and neq[s] (count of elements equal to the result after the last round).
struct Segs {
    long long base[DASS_MAX_CAMERAS];
    long long len[DASS_MAX_CAMERAS];
    long long rank[DASS_MAX_CAMERAS];
};

__global__ void set_ranks_kernel(Segs sg, int n, long long* rank) {
    int i = threadIdx.x;
    if (i < n) rank[i] = sg.rank[i];
}

__global__ void set_i64_kernel(long long* dst, long long v) { *dst = v; }

__global__ void select_hist_kernel(const uint32_t* __restrict__ keys, Segs sg,
                                   const uint32_t* __restrict__ prefix, uint32_t* __restrict__ hist, int shift) {
    int s = blockIdx.y;
    long long base = sg.base[s], len = sg.len[s];
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    uint32_t pre = prefix[s];
    int hs = shift + 8;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        uint32_t k = keys[base + i];
        bool match = hs >= 32 ? true : ((k >> hs) == (pre >> hs));
        if (match) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[s * 256 + i], h[i]);
}

// One block per segment: locate the digit holding the wanted rank.
__global__ void select_decide_kernel(uint32_t* __restrict__ hist, uint32_t* __restrict__ prefix,
                                     long long* __restrict__ rank, long long* __restrict__ neq, int shift) {
    int s = blockIdx.x;
    __shared__ uint32_t h[256];
    h[threadIdx.x] = hist[s * 256 + threadIdx.x];
    hist[s * 256 + threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long r = rank[s];
        long long cum = 0;
        int b = 0;
        for (; b < 256; ++b) {
            if (r < cum + (long long)h[b]) break;
            cum += h[b];
        }
        if (b == 256) b = 255;   // rank beyond the data (cannot happen for valid ranks)
        prefix[s] |= (uint32_t)b << shift;
        rank[s] = r - cum;
        neq[s] = h[b];
    }
}

// ----------------------------------------------------------------- error pass (Sec. 3.4)

__global__ void error_map_kernel(const float* __restrict__ img, const float* __restrict__ tgt, CamTable ct,
                                 float* __restrict__ E, uint32_t* __restrict__ keys) {
    int c = blockIdx.y;
    const CamInfo& cam = ct.c[c];
    long long plane = (long long)cam.W * cam.H;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const float* a = img + 3 * cam.pix_base;
    const float* b = tgt + 3 * cam.pix_base;
    float e0 = fabsf(__fsub_rn(a[i], b[i]));
    float e1 = fabsf(__fsub_rn(a[plane + i], b[plane + i]));
    float e2 = fabsf(__fsub_rn(a[2 * plane + i], b[2 * plane + i]));
    float e = __fdiv_rn(__fadd_rn(__fadd_rn(e0, e1), e2), 3.f);
    E[cam.pix_base + i] = e;
    keys[cam.pix_base + i] = __float_as_uint(e);
}

__global__ void s_err_kernel(long long n, const float* __restrict__ means, const uint8_t* __restrict__ is_var,
                             CamTable ct, const float* __restrict__ E, const uint32_t* __restrict__ gamma_bits,
                             uint8_t* __restrict__ s_err) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    uint8_t hit = 0;
    if (!(is_var && is_var[g])) {
        float P0 = means[3 * g], P1 = means[3 * g + 1], P2 = means[3 * g + 2];
        for (int c = 0; c < ct.n && !hit; ++c) {
            const CamInfo& cam = ct.c[c];
            const float* T = cam.proj;
            // [P, 1] T in float32, fixed order ((P0 T0k + P1 T1k) + P2 T2k) + T3k
            float px = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P0, T[0]), __fmul_rn(P1, T[4])), __fmul_rn(P2, T[8])), T[12]);
            float py = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P0, T[1]), __fmul_rn(P1, T[5])), __fmul_rn(P2, T[9])), T[13]);
            float pw = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P0, T[3]), __fmul_rn(P1, T[7])), __fmul_rn(P2, T[11])), T[15]);
            if (!(pw > 0.f)) continue;
            float xn = __fdiv_rn(px, pw), yn = __fdiv_rn(py, pw);
            float xc = __fmul_rn(0.5f, __fsub_rn(__fmul_rn(__fadd_rn(xn, 1.f), (float)cam.W), 1.f));
            float yc = __fmul_rn(0.5f, __fsub_rn(__fmul_rn(__fadd_rn(yn, 1.f), (float)cam.H), 1.f));
            float xi = floorf(__fadd_rn(xc, 0.5f)), yi = floorf(__fadd_rn(yc, 0.5f));
            if (!(xi >= 0.f && xi < (float)cam.W && yi >= 0.f && yi < (float)cam.H)) continue;
            float e = E[cam.pix_base + (long long)yi * cam.W + (long long)xi];
            if (__float_as_uint(e) > gamma_bits[c]) hit = 1;
        }
    }
    s_err[g] = hit;
}

// ----------------------------------------------------------------- Eq. 4 selection

__global__ void select_keys_kernel(long long n, const float* __restrict__ accum, const int* __restrict__ count,
                                   const uint8_t* __restrict__ s_err, const uint8_t* __restrict__ is_var,
                                   float tau_pos, float tau_err, uint32_t* __restrict__ keys,
                                   unsigned long long* __restrict__ n_cand) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool cand = false;
    if (i < n) {
        int c = count[i];
        float gm = c > 0 ? __fdiv_rn(accum[i], (float)c) : 0.f;
        bool base = !(is_var && is_var[i]);
        cand = base && (gm > tau_pos || (s_err && s_err[i] && gm > tau_err));
        keys[i] = cand ? __float_as_uint(gm) : 0u;
    }
    unsigned b = __ballot_sync(0xffffffffu, cand);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_cand, (unsigned long long)__popc(b));
}

__global__ void select_prepare_kernel(long long n, const unsigned long long* n_cand, int k_max, long long* rank) {
    // ascending rank of the k_max-th largest key
    long long nc = (long long)*n_cand;
    rank[0] = nc > k_max ? n - k_max : 0;
}

__global__ void select_eq_flags_kernel(long long n, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ prefix,
                                       uint32_t* __restrict__ eq) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) eq[i] = keys[i] == prefix[0] ? 1u : 0u;
}

__global__ void select_flags_kernel(long long n, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ prefix,
                                    const uint32_t* __restrict__ eq_rank, const long long* __restrict__ rank_rem,
                                    const long long* __restrict__ neq, const unsigned long long* __restrict__ n_cand,
                                    int k_max, uint32_t* __restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = keys[i];
    bool sel;
    if ((long long)*n_cand <= k_max) {
        sel = k > 0u;
    } else {
        uint32_t thr = prefix[0];
        long long need = neq[0] - rank_rem[0];
        sel = k > thr || (k == thr && (long long)eq_rank[i] < need);
    }
    flag[i] = sel ? 1u : 0u;
}

__global__ void compact_kernel(long long n, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                               const long long* __restrict__ total, int k_max, int* __restrict__ out,
                               int* __restrict__ n_out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *n_out = (int)(*total < k_max ? *total : k_max);
    if (i < n && flag[i] && pos[i] < (uint32_t)k_max) out[pos[i]] = (int)i;
}

// ----------------------------------------------------------------- spawn (Sec. 3.4)

__global__ void spawn_kernel(long long n, int K3, float* means, float* log_scales, float* quats, float* logit, float* sh,
                             uint8_t* is_var, const int* __restrict__ selected, const int* __restrict__ n_sel,
                             int k_max, const float* __restrict__ z, long long* n_total, float log_div) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = *n_sel;
    if (i == 0) *n_total = n + cnt;
    if (i >= cnt || i >= k_max) return;
    long long s = selected[i];
    long long row = n + i;
    float4 q4 = reinterpret_cast<const float4*>(quats)[s];
    float qn = 1.f / sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    float R[9];
    quat_to_rot(q4.x * qn, q4.y * qn, q4.z * qn, q4.w * qn, R);
    float sc[3], zz[3];
    for (int k = 0; k < 3; ++k) { sc[k] = expf(log_scales[3 * s + k]); zz[k] = z[3 * s + k]; }
    for (int r = 0; r < 3; ++r) {
        float d = R[3 * r] * sc[0] * zz[0] + R[3 * r + 1] * sc[1] * zz[1] + R[3 * r + 2] * sc[2] * zz[2];
        means[3 * row + r] = means[3 * s + r] + d;
        log_scales[3 * row + r] = log_scales[3 * s + r] - log_div;
    }
    reinterpret_cast<float4*>(quats)[row] = q4;
    logit[row] = logit[s];
    for (int k = 0; k < K3; ++k) sh[row * K3 + k] = sh[s * K3 + k];
    is_var[row] = 1;
}

struct Carve {
    char* p;
    size_t used = 0;
    template <class T>
    T* take(long long count) {
        size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
        T* r = reinterpret_cast<T*>(p ? p + used : nullptr);
        used += bytes;
        return r;
    }
};

}  // namespace

// ----------------------------------------------------------------- launchers

int shift_launch(long long n_dyn, const int* idx, const float* off, const float* means, const float* quats,
                 float* om, float* oq, cudaStream_t st) {
    if (n_dyn <= 0) return DASS_OK;
    shift_fwd_kernel<<<div_up(n_dyn, 256), 256, 0, st>>>(n_dyn, idx, off, means, quats, om, oq); count_launch();
    return check_launch("shift_fwd_kernel");
}

int shift_bwd_launch(long long n_dyn, const int* idx, const float* off, const float* quats, const float* dm,
                     const float* dq, float* doff, float* dqin, cudaStream_t st) {
    if (n_dyn <= 0) return DASS_OK;
    shift_bwd_kernel<<<div_up(n_dyn, 256), 256, 0, st>>>(n_dyn, idx, off, quats, dm, dq, doff, dqin); count_launch();
    return check_launch("shift_bwd_kernel");
}

int adam_launch(long long n_sel, int width, const int* rows, float* p, const float* g, float* m, float* v,
                int* step_dev, const float* lr, float b1, float b2, float eps, int inc, cudaStream_t st) {
    if (width < 1 || width > 16) return DASS_ERR_INVALID_ARG;
    LR l;
    for (int k = 0; k < 16; ++k) l.v[k] = k < width ? lr[k] : 0.f;
    long long tot = n_sel * width;
    if (tot > 0) {
        adam_kernel<<<div_up(tot, 256), 256, 0, st>>>(n_sel, width, rows, p, g, m, v, step_dev, l, b1, b2, eps); count_launch();
        int rc = check_launch("adam_kernel");
        if (rc) return rc;
    }
    if (inc) {
        step_inc_kernel<<<1, 1, 0, st>>>(step_dev); count_launch();
        return check_launch("step_inc_kernel");
    }
    return DASS_OK;
}

size_t inherit_workspace_bytes(long long n) {
    Carve c{nullptr};
    c.take<uint32_t>(n); c.take<uint32_t>(n); c.take<uint32_t>(n); c.take<uint32_t>(n);
    c.take<long long>(4);
    c.take<unsigned long long>((long long)(scan_partials_bytes(n) / 8 + 1));
    return c.used;
}

// Keep logits of the low-opacity pruning (Sec. 3.4): m[g] = opacity_logit[g] - logit(min_opacity),
// positive iff sigmoid(opacity_logit[g]) > min_opacity, for the inheritance copy to keep or drop
// var rows by.
__global__ void prune_logits_kernel(long long n, const float* __restrict__ logit, float thr, float* __restrict__ m) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) m[i] = logit[i] - thr;
}

int prune_logits_launch(long long n, const float* logit, float min_opacity, float* m, cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    const float thr = logf(min_opacity / (1.f - min_opacity));
    prune_logits_kernel<<<div_up(n, 256), 256, 0, st>>>(n, logit, thr, m); count_launch();
    return check_launch("prune_logits_kernel");
}

int inherit_keep_launch(long long n, const uint8_t* is_var, const float* m, uint8_t* keep, cudaStream_t st) {
    if (n <= 0) return DASS_OK;
    inherit_keep_kernel<<<div_up(n, 256), 256, 0, st>>>(n, is_var, m, keep); count_launch();
    return check_launch("inherit_keep_kernel");
}

int inherit_mask_grad_launch(long long n_rows, const int* rows, const float* m, const float* d_keep, float lambda,
                             float* grad, double* loss, cudaStream_t st) {
    if (n_rows <= 0) return DASS_OK;
    inherit_mask_grad_kernel<<<div_up(n_rows, 256), 256, 0, st>>>(n_rows, rows, m, d_keep, lambda, grad, loss);
    count_launch();
    return check_launch("inherit_mask_grad_kernel");
}

int inherit_launch(long long n, int deg, const float* means, const float* ls, const float* quats, const float* logit,
                   const float* sh, const uint8_t* is_var, const float* m, int erase, float* om, float* ols, float* oq,
                   float* ologit, float* osh, uint8_t* ovar, int* remap, long long* n_out, void* ws, size_t ws_bytes,
                   cudaStream_t st) {
    if (ws_bytes < inherit_workspace_bytes(n)) return DASS_ERR_OOM;
    Carve c{reinterpret_cast<char*>(ws)};
    uint32_t* fb = c.take<uint32_t>(n);
    uint32_t* fv = c.take<uint32_t>(n);
    uint32_t* sb = c.take<uint32_t>(n);
    uint32_t* sv = c.take<uint32_t>(n);
    long long* sc = c.take<long long>(4);
    unsigned long long* part = c.take<unsigned long long>((long long)(scan_partials_bytes(n) / 8 + 1));
    if (n == 0) {
        DASS_CHECK_CUDA(cudaMemsetAsync(n_out, 0, sizeof(long long), st));
        return DASS_OK;
    }
    set_i64_kernel<<<1, 1, 0, st>>>(sc + 2, n); count_launch();
    inherit_flags_kernel<<<div_up(n, 256), 256, 0, st>>>(n, is_var, m, erase, fb, fv); count_launch();
    int rc = check_launch("inherit_flags");
    if (rc) return rc;
    rc = scan_u32_public(fb, sb, sc + 2, n, part, sc + 0, st);
    if (rc) return rc;
    rc = scan_u32_public(fv, sv, sc + 2, n, part, sc + 1, st);
    if (rc) return rc;
    int K3 = 3 * (deg + 1) * (deg + 1);
    inherit_scatter_kernel<<<div_up(n, 256), 256, 0, st>>>(n, K3, fb, fv, sb, sv, sc, means, ls, quats, logit, sh, om,
                                                           ols, oq, ologit, osh, ovar, remap, n_out); count_launch();
    return check_launch("inherit_scatter");
}

size_t error_pass_workspace_bytes(const CamTable& ct) {
    Carve c{nullptr};
    c.take<float>(ct.pixels_total);
    c.take<uint32_t>(ct.pixels_total);
    c.take<uint32_t>(256 * DASS_MAX_CAMERAS);
    c.take<uint32_t>(DASS_MAX_CAMERAS);
    c.take<long long>(DASS_MAX_CAMERAS);
    c.take<long long>(DASS_MAX_CAMERAS);
    return c.used;
}

int error_pass_launch(const float* img, const float* tgt, const CamTable& ct, double quantile, long long n,
                      const float* means, const uint8_t* is_var, float* error_map, float* gamma, uint8_t* s_err,
                      void* ws, size_t ws_bytes, cudaStream_t st) {
    if (ws_bytes < error_pass_workspace_bytes(ct)) return DASS_ERR_OOM;
    Carve c{reinterpret_cast<char*>(ws)};
    float* E = c.take<float>(ct.pixels_total);
    uint32_t* keys = c.take<uint32_t>(ct.pixels_total);
    uint32_t* hist = c.take<uint32_t>(256 * DASS_MAX_CAMERAS);
    uint32_t* prefix = c.take<uint32_t>(DASS_MAX_CAMERAS);
    long long* rank = c.take<long long>(DASS_MAX_CAMERAS);
    long long* neq = c.take<long long>(DASS_MAX_CAMERAS);
    if (error_map) E = error_map;
    Segs sg;
    long long maxP = 0;
    for (int i = 0; i < ct.n; ++i) {
        long long P = (long long)ct.c[i].W * ct.c[i].H;
        sg.base[i] = ct.c[i].pix_base;
        sg.len[i] = P;
        sg.rank[i] = (long long)std::floor(quantile * (double)(P - 1));
        maxP = P > maxP ? P : maxP;
    }
    DASS_CHECK_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 256 * ct.n, st));
    DASS_CHECK_CUDA(cudaMemsetAsync(prefix, 0, sizeof(uint32_t) * ct.n, st));
    set_ranks_kernel<<<1, DASS_MAX_CAMERAS, 0, st>>>(sg, ct.n, rank); count_launch();
    dim3 g1(div_up(maxP, 256), ct.n);
    error_map_kernel<<<g1, 256, 0, st>>>(img, tgt, ct, E, keys); count_launch();
    int rc = check_launch("error_map");
    if (rc) return rc;
    dim3 g2(64, ct.n);
    for (int shift = 24; shift >= 0; shift -= 8) {
        select_hist_kernel<<<g2, 256, 0, st>>>(keys, sg, prefix, hist, shift); count_launch();
        select_decide_kernel<<<ct.n, 256, 0, st>>>(hist, prefix, rank, neq, shift); count_launch();
        rc = check_launch("error_select");
        if (rc) return rc;
    }
    if (gamma) {
        DASS_CHECK_CUDA(cudaMemcpyAsync(gamma, prefix, sizeof(uint32_t) * ct.n, cudaMemcpyDeviceToDevice, st));
    }
    if (n > 0) {
        s_err_kernel<<<div_up(n, 256), 256, 0, st>>>(n, means, is_var, ct, E, prefix, s_err); count_launch();
        return check_launch("s_err");
    }
    return DASS_OK;
}

size_t select_workspace_bytes(long long n) {
    Carve c{nullptr};
    c.take<uint32_t>(n); c.take<uint32_t>(n); c.take<uint32_t>(n); c.take<uint32_t>(n);
    c.take<uint32_t>(256); c.take<uint32_t>(4); c.take<long long>(8); c.take<unsigned long long>(2);
    c.take<unsigned long long>((long long)(scan_partials_bytes(n) / 8 + 1));
    return c.used;
}

int select_launch(long long n, const float* accum, const int* count, const uint8_t* s_err, const uint8_t* is_var,
                  float tau_pos, float tau_err, int k_max, int* selected, int* n_selected, void* ws, size_t ws_bytes,
                  cudaStream_t st) {
    if (ws_bytes < select_workspace_bytes(n)) return DASS_ERR_OOM;
    Carve c{reinterpret_cast<char*>(ws)};
    uint32_t* keys = c.take<uint32_t>(n);
    uint32_t* eq = c.take<uint32_t>(n);
    uint32_t* eqr = c.take<uint32_t>(n);
    uint32_t* flag = c.take<uint32_t>(n);
    uint32_t* hist = c.take<uint32_t>(256);
    uint32_t* prefix = c.take<uint32_t>(4);
    long long* sc = c.take<long long>(8);   // 0 rank, 1 neq, 2 len, 3 eq total, 4 sel total
    unsigned long long* n_cand = c.take<unsigned long long>(2);
    unsigned long long* part = c.take<unsigned long long>((long long)(scan_partials_bytes(n) / 8 + 1));
    if (n == 0 || k_max <= 0) {
        DASS_CHECK_CUDA(cudaMemsetAsync(n_selected, 0, sizeof(int), st));
        return DASS_OK;
    }
    set_i64_kernel<<<1, 1, 0, st>>>(sc + 2, n); count_launch();
    DASS_CHECK_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 256, st));
    DASS_CHECK_CUDA(cudaMemsetAsync(prefix, 0, sizeof(uint32_t) * 4, st));
    DASS_CHECK_CUDA(cudaMemsetAsync(n_cand, 0, sizeof(unsigned long long) * 2, st));
    int nb = div_up(n, 256);
    select_keys_kernel<<<nb, 256, 0, st>>>(n, accum, count, s_err, is_var, tau_pos, tau_err, keys, n_cand); count_launch();
    select_prepare_kernel<<<1, 1, 0, st>>>(n, n_cand, k_max, sc + 0); count_launch();
    int rc = check_launch("select_keys");
    if (rc) return rc;
    Segs one;
    one.base[0] = 0;
    one.len[0] = n;
    one.rank[0] = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        select_hist_kernel<<<dim3(div_up(n, 256) < 256 ? div_up(n, 256) : 256, 1), 256, 0, st>>>(keys, one, prefix,
                                                                                                 hist, shift); count_launch();
        select_decide_kernel<<<1, 256, 0, st>>>(hist, prefix, sc + 0, sc + 1, shift); count_launch();
        rc = check_launch("select_radix");
        if (rc) return rc;
    }
    select_eq_flags_kernel<<<nb, 256, 0, st>>>(n, keys, prefix, eq); count_launch();
    rc = scan_u32_public(eq, eqr, sc + 2, n, part, sc + 3, st);
    if (rc) return rc;
    select_flags_kernel<<<nb, 256, 0, st>>>(n, keys, prefix, eqr, sc + 0, sc + 1, n_cand, k_max, flag); count_launch();
    rc = scan_u32_public(flag, eq, sc + 2, n, part, sc + 4, st);
    if (rc) return rc;
    compact_kernel<<<nb, 256, 0, st>>>(n, flag, eq, sc + 4, k_max, selected, n_selected); count_launch();
    return check_launch("select_compact");
}

int spawn_launch(long long n, int deg, float* means, float* ls, float* quats, float* logit, float* sh, uint8_t* is_var,
                 const int* selected, const int* n_sel, int k_max, const float* z, long long* n_total,
                 cudaStream_t st) {
    int K3 = 3 * (deg + 1) * (deg + 1);
    float log_div = logf(1.6f);
    spawn_kernel<<<div_up(k_max > 0 ? k_max : 1, 256), 256, 0, st>>>(n, K3, means, ls, quats, logit, sh, is_var,
                                                                     selected, n_sel, k_max, z, n_total, log_div); count_launch();
    return check_launch("spawn_kernel");
}

}  // namespace dass
