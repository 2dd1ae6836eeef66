// K1 (Gaussian transformation, Sec. 2.1 step 1) and K8 (its backward).
//
// One thread per Gaussian walks all B views of the call, so a Gaussian's 240
// bytes of parameters are read from HBM once per batch rather than once per
// view; the per-view outputs are written structure-of-arrays ([B][N] float4
// planes) so every store is coalesced.  FP32 throughout, IEEE division and
// square root (no fast-math), precise expf for the activations.
#include "gs_internal.cuh"

namespace gs {
namespace {

// Real SH basis, degree <= 3, Condon-Shortley phase, k = l*l + l + m.
// Constants are the closed forms rounded to float:
//   c0 = 1/(2 sqrt(pi)), c1 = sqrt(3/(4 pi)), a2 = sqrt(15/pi)/2,
//   b2 = sqrt(5/pi)/4, c2 = sqrt(15/pi)/4, e3 = sqrt(35/(2 pi))/4,
//   f3 = sqrt(105/pi)/2, g3 = sqrt(21/(2 pi))/4, h3 = sqrt(7/pi)/4,
//   k3 = sqrt(105/pi)/4.
constexpr float SH_C0 = 2.820947918e-01f;
constexpr float SH_C1 = 4.886025119e-01f;
constexpr float SH_A2 = 1.092548431e+00f;
constexpr float SH_B2 = 3.153915653e-01f;
constexpr float SH_C2 = 5.462742153e-01f;
constexpr float SH_E3 = 5.900435899e-01f;
constexpr float SH_F3 = 2.890611443e+00f;
constexpr float SH_G3 = 4.570457995e-01f;
constexpr float SH_H3 = 3.731763326e-01f;
constexpr float SH_K3 = 1.445305721e+00f;

__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[16])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = SH_C0;
    Y[1] = -SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = -SH_C1 * x;
    Y[4] = SH_A2 * x * y;
    Y[5] = -SH_A2 * y * z;
    Y[6] = SH_B2 * (3.f * zz - 1.f);
    Y[7] = -SH_A2 * x * z;
    Y[8] = SH_C2 * (xx - yy);
    Y[9] = -SH_E3 * y * (3.f * xx - yy);
    Y[10] = SH_F3 * x * y * z;
    Y[11] = -SH_G3 * y * (5.f * zz - 1.f);
    Y[12] = SH_H3 * z * (5.f * zz - 3.f);
    Y[13] = -SH_G3 * x * (5.f * zz - 1.f);
    Y[14] = SH_K3 * z * (xx - yy);
    Y[15] = -SH_E3 * x * (xx - 3.f * yy);
}

// Gradient of sum_k w_k Y_k(x, y, z) with respect to (x, y, z), treating the
// basis as polynomials (the caller projects onto the sphere's tangent plane).
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, const float w[16], int nk, float &gx,
                                            float &gy, float &gz)
{
    gx = 0.f; gy = 0.f; gz = 0.f;
    if (nk > 1) {
        gy += -SH_C1 * w[1];
        gz += SH_C1 * w[2];
        gx += -SH_C1 * w[3];
    }
    if (nk > 4) {
        gx += SH_A2 * y * w[4];           gy += SH_A2 * x * w[4];
        gy += -SH_A2 * z * w[5];          gz += -SH_A2 * y * w[5];
        gz += 6.f * SH_B2 * z * w[6];
        gx += -SH_A2 * z * w[7];          gz += -SH_A2 * x * w[7];
        gx += 2.f * SH_C2 * x * w[8];     gy += -2.f * SH_C2 * y * w[8];
    }
    if (nk > 9) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += -6.f * SH_E3 * x * y * w[9];  gy += -3.f * SH_E3 * (xx - yy) * w[9];
        gx += SH_F3 * y * z * w[10];        gy += SH_F3 * x * z * w[10];  gz += SH_F3 * x * y * w[10];
        gy += -SH_G3 * (5.f * zz - 1.f) * w[11];  gz += -10.f * SH_G3 * y * z * w[11];
        gz += SH_H3 * (15.f * zz - 3.f) * w[12];
        gx += -SH_G3 * (5.f * zz - 1.f) * w[13];  gz += -10.f * SH_G3 * x * z * w[13];
        gx += 2.f * SH_K3 * x * z * w[14];  gy += -2.f * SH_K3 * y * z * w[14];  gz += SH_K3 * (xx - yy) * w[14];
        gx += -3.f * SH_E3 * (xx - yy) * w[15];  gy += 6.f * SH_E3 * x * y * w[15];
    }
}

__device__ __forceinline__ bool finite4(const float4 &a)
{
    return isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w);
}

// Rotation of a unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

struct Geom {        // view-independent Gaussian state
    float x, y, z, o;
    float s[3];
    float qn[4], qnorm;
    float Rq[9];
    float S[6];      // 3D covariance: 00 01 02 11 12 22
    bool ok;
};

__device__ __forceinline__ Geom load_geom(const SceneView &s, int64_t g)
{
    Geom G;
    const float4 mo = s.mo[g], ls = s.ls[g], q = s.q[g];
    G.ok = finite4(mo) && finite4(ls) && finite4(q);
    G.x = mo.x; G.y = mo.y; G.z = mo.z;
    G.o = 1.f / (1.f + expf(-mo.w));
    G.s[0] = expf(ls.x); G.s[1] = expf(ls.y); G.s[2] = expf(ls.z);
    const float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    G.ok = G.ok && n2 > 0.f;
    G.qnorm = sqrtf(n2);
    const float inv = 1.f / G.qnorm;
    G.qn[0] = q.x * inv; G.qn[1] = q.y * inv; G.qn[2] = q.z * inv; G.qn[3] = q.w * inv;
    quat_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.Rq);
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = G.Rq[3 * i + j] * G.s[j];
    G.S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    return G;
}

// Error-free sum of two floats: s = RN(a + b) and a + b = s + e exactly
// (Knuth's TwoSum; explicitly rounded operations, so nothing is contracted).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Depth of a point in view space, as the fragment order defines it: the sum
// t2 + R6 x + R7 y + R8 z evaluated left to right in double precision (each
// product of two floats is exact in double, each of the three additions is
// rounded to double) and then rounded to float; *above: whether that double
// sum exceeds `near`.  Double-precision arithmetic runs at a small fraction
// of the float rate on this GPU, so the sum is first evaluated in float
// arithmetic without losing the rounding decision:
//  - each product splits into an exact pair h + l (h = RN(R x), l by fma);
//  - t2 + h1 + h2 + h3 by error-free TwoSums, their errors and the l's added
//    in float: s + e is within 20 * 2^-48 M < 2^-43 M of the exact sum
//    (M = |t2| + |h1| + |h2| + |h3|);
//  - the double chain is within 3.01 * 2^-53 M < 2^-51 M of the exact sum;
//  - f = RN(s + e) with s + e = f + r exactly; if |r| + B, B = 2^-41 M (twice
//    the 2^-42 M of the two bounds together), is below half the gap from f to
//    its nearer float neighbour, the double sum lies strictly inside f's
//    rounding interval, so its float rounding is f; and f > near (f < near)
//    implies the double sum is above (below) near, near being a float.
// Otherwise (f within B of a rounding boundary, f == near, a tiny, huge or
// non-finite value: rare) the double chain itself is evaluated, out of line
// so that it holds no registers on the common path.
__device__ __noinline__ double depth_chain(float t, float r6, float r7, float r8, float x, float y, float z)
{
    double zd = (double)t;
    zd = __dadd_rn(zd, __dmul_rn((double)r6, (double)x));
    zd = __dadd_rn(zd, __dmul_rn((double)r7, (double)y));
    return __dadd_rn(zd, __dmul_rn((double)r8, (double)z));
}

__device__ __forceinline__ float view_depth(const ViewCam &c, float x, float y, float z, bool *above)
{
    const float t = c.t[2];
    const float h1 = __fmul_rn(c.R[6], x), l1 = __fmaf_rn(c.R[6], x, -h1);
    const float h2 = __fmul_rn(c.R[7], y), l2 = __fmaf_rn(c.R[7], y, -h2);
    const float h3 = __fmul_rn(c.R[8], z), l3 = __fmaf_rn(c.R[8], z, -h3);
    float s, e1, e2, e3;
    two_sum(t, h1, s, e1);
    two_sum(s, h2, s, e2);
    two_sum(s, h3, s, e3);
    const float e = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, l1)), __fadd_rn(l2, l3));
    float f, r;
    two_sum(s, e, f, r);
    const float M = __fadd_rn(__fadd_rn(fabsf(t), fabsf(h1)), __fadd_rn(fabsf(h2), fabsf(h3)));
    const float B = __fmul_rn(M, 0x1p-41f);
    const uint32_t bits = __float_as_uint(fabsf(f)), ex = bits >> 23;
    bool fast = isfinite(M) && ex >= 25u && ex <= 253u && f != c.near_z;
    if (fast) {
        const float ulp = __uint_as_float((ex - 23u) << 23);      // 2^(exponent - 23) of a normal f
        const float half_gap = (bits & 0x7fffffu) ? 0.5f * ulp : 0.25f * ulp;
        fast = __fadd_rn(fabsf(r), B) < half_gap;
    }
    if (fast) {
        *above = f > c.near_z;
        return f;
    }
    const double zd = depth_chain(t, c.R[6], c.R[7], c.R[8], x, y, z);
    *above = zd > (double)c.near_z;
    return __double2float_rn(zd);
}

// Register use is capped for 6 resident blocks (a few spills): more warps hide
// the latency of the scattered per-view stores better (measured: C3 5.0 ->
// 4.3 ms).
__global__ void __launch_bounds__(128, 6) k_preprocess_fwd(SceneView s, ViewBatch vb, ProjView p, uint32_t *ntiles,
                                                        uint2 *rect, DevStatus *status, int strict, uint4 *rm,
                                                        float cull_alpha)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= s.N) return;
    const Geom G = load_geom(s, g);
    if (!G.ok) {
        atomicAdd(&status->counters[3], 1ull);
        if (strict) atomicCAS(&status->code, 0, (int)GS_ERR_NONFINITE);
    }
    const int nk = (s.deg + 1) * (s.deg + 1);
    float4 shv[12];
    bool sh_loaded = false;
    const float inv_tile = 1.f / (float)vb.tile;
    for (int v = 0; v < vb.B; ++v) {
        const ViewCam &c = vb.v[v];
        const int64_t idx = (int64_t)v * s.N + g;
        const float px = c.R[0] * G.x + c.R[1] * G.y + c.R[2] * G.z + c.t[0];
        const float py = c.R[3] * G.x + c.R[4] * G.y + c.R[5] * G.z + c.t[1];
        // the depth that orders the fragments: the double-precision sum
        // rounded to float, as the oracle defines it (view_depth)
        bool above_near;
        const float pz = view_depth(c, G.x, G.y, G.z, &above_near);
        uint32_t area = 0;
        int r_int = 0;
        uint2 rc = pack_rect(1u, 0u, 0u, 0u);     // empty
        if (G.ok && above_near) {
            const float iz = 1.f / pz;
            const float u = c.fx * px * iz + c.cx;
            const float vv = c.fy * py * iz + c.cy;
            const float tx = fminf(c.limx, fmaxf(-c.limx, px * iz));
            const float ty = fminf(c.limy, fmaxf(-c.limy, py * iz));
            const float J00 = c.fx * iz, J02 = -c.fx * tx * iz;
            const float J11 = c.fy * iz, J12 = -c.fy * ty * iz;
            float T0[3], T1[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T0[j] = J00 * c.R[j] + J02 * c.R[6 + j];
                T1[j] = J11 * c.R[3 + j] + J12 * c.R[6 + j];
            }
            // TS = T Sigma (rows), Sigma' = TS T^T
            const float *S = G.S;
            const float a0 = T0[0] * S[0] + T0[1] * S[1] + T0[2] * S[2];
            const float a1 = T0[0] * S[1] + T0[1] * S[3] + T0[2] * S[4];
            const float a2 = T0[0] * S[2] + T0[1] * S[4] + T0[2] * S[5];
            const float b0 = T1[0] * S[0] + T1[1] * S[1] + T1[2] * S[2];
            const float b1 = T1[0] * S[1] + T1[1] * S[3] + T1[2] * S[4];
            const float b2 = T1[0] * S[2] + T1[1] * S[4] + T1[2] * S[5];
            const float A = a0 * T0[0] + a1 * T0[1] + a2 * T0[2] + 0.3f;
            const float Bc = a0 * T1[0] + a1 * T1[1] + a2 * T1[2];
            const float Cc = b0 * T1[0] + b1 * T1[1] + b2 * T1[2] + 0.3f;
            const float det = A * Cc - Bc * Bc;
            if (det > 0.f) {
                const float idet = 1.f / det;
                const float m = 0.5f * (A + Cc);
                const float lam = m + sqrtf(fmaxf(0.f, m * m - det));
                const float rf = fminf(ceilf(3.f * sqrtf(lam)), 16777216.f);
                // tile rectangle: IEEE single ops only (subtract, times exact 1/tile, floor)
                float x0 = floorf(__fmul_rn(__fsub_rn(u, rf), inv_tile));
                float x1 = floorf(__fmul_rn(__fadd_rn(u, rf), inv_tile));
                float y0 = floorf(__fmul_rn(__fsub_rn(vv, rf), inv_tile));
                float y1 = floorf(__fmul_rn(__fadd_rn(vv, rf), inv_tile));
                x0 = fmaxf(x0, 0.f);
                y0 = fmaxf(y0, 0.f);
                x1 = fminf(x1, (float)(c.TX - 1));
                y1 = fminf(y1, (float)(c.TY - 1));
                if (x0 <= x1 && y0 <= y1) {
                    area = (uint32_t)((int)(x1 - x0) + 1) * (uint32_t)((int)(y1 - y0) + 1);
                    rc = pack_rect((uint32_t)x0, (uint32_t)x1, (uint32_t)y0, (uint32_t)y1);
                    r_int = (int)rf;
                    if (!sh_loaded) {
#pragma unroll
                        for (int k = 0; k < 12; ++k) shv[k] = s.sh[(int64_t)k * s.N + g];
                        sh_loaded = true;
                    }
                    float dx = G.x - c.C[0], dy = G.y - c.C[1], dz = G.z - c.C[2];
                    const float il = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
                    dx *= il; dy *= il; dz *= il;
                    float Y[16];
                    sh_eval(dx, dy, dz, Y);
                    const float *shf = reinterpret_cast<const float *>(shv);
                    float rgb[3];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (k < nk) acc += shf[3 * k + ch] * Y[k];
                        rgb[ch] = fmaxf(acc + 0.5f, 0.f);
                    }
                    const float4 co = make_float4(Cc * idet, -Bc * idet, A * idet, G.o);
                    p.xy[idx] = make_float2(u, vv);
                    p.conic_o[idx] = co;
                    p.rgb_d[idx] = make_float4(rgb[0], rgb[1], rgb[2], pz);
                    if (rm) {                      // cull the rectangle's tiles against the alpha ellipse
                        uint64_t keep = ~0ull;
                        if (area <= TILE_CULL_MAX_AREA) {
                            keep = row_interval_mask(co, ellipse_terms(co, cull_alpha), u, vv, (uint32_t)x0,
                                                     (uint32_t)x1, (uint32_t)y0, (uint32_t)y1, (float)vb.tile);
                            area = (uint32_t)__popcll(keep);
                        }
                        rm[idx] = make_uint4(rc.x, rc.y, (uint32_t)keep, (uint32_t)(keep >> 32));
                    }
                }
            }
        }
        p.radius[idx] = r_int;
        ntiles[idx] = area;
        if (rect) rect[idx] = rc;
    }
}

// The blending backward's moments -> gradients of gs_proj, in place.
__global__ void __launch_bounds__(256) k_moments_to_grads(ProjView p, int64_t n, GradView gv)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 gxo, gco;
    moments_to_grads(p.conic_o[i], gv.d_xy_o[i], gv.d_conic[i], gxo, gco);
    gv.d_xy_o[i] = gxo;
    gv.d_conic[i] = gco;
}

// K8: chain rule from dL/d(u, v, conic, opacity, rgb) per view to the 59
// parameters; views summed in a fixed order (deterministic), times 1/B.
// Capped for 4 resident blocks (128 registers, 8 bytes of spill), which the
// two passes over the views make room for: one pass holding the 48 SH
// coefficients, the other their 48 gradient sums (in one pass both, 168
// registers at 3 blocks: C2 2.24 -> 1.98 ms, C3 2.08 -> 1.90 ms).  Caps of
// 5 and 6 blocks spill 224 and 360 bytes.
__global__ void __launch_bounds__(128, 4) k_preprocess_bwd(SceneView s, ViewBatch vb, ProjView p, GradView gv,
                                                        bool grads_ready, SceneMut out, uint8_t *vis,
                                                        float *dacc, uint32_t *dcnt, const DevStatus *status,
                                                        float scale)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= s.N) return;
    const int nk = (s.deg + 1) * (s.deg + 1);
    bool any = false;
    for (int v = 0; v < vb.B; ++v) any |= p.radius[(int64_t)v * s.N + g] > 0;
    const float invB = scale;                    // 1/B: the batch mean (Sec. 4); 1: the sum over views
    if (vis) {                                   // visible-only Adam: unseen rows stay unwritten
        vis[g] = any ? 1 : 0;
        if (!any) return;
    }
    if (!any) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        out.mo[g] = z4; out.ls[g] = z4; out.q[g] = z4;
        for (int k = 0; k < 12; ++k) out.sh[(int64_t)k * s.N + g] = z4;
        return;
    }
    const Geom G = load_geom(s, g);
    float4 shv[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) shv[k] = s.sh[(int64_t)k * s.N + g];
    const float *shf = reinterpret_cast<const float *>(shv);
    // two passes over the views: the first takes every gradient but the SH
    // coefficients' (it needs the coefficients, for the clamp test and the
    // direction term), recording per view and channel whether the colour was
    // clamped; the second sums the coefficients' gradients Y (x) dL/drgb.  The
    // coefficients and their 48 gradient sums are then never live together.
    uint32_t clampm[3] = {0u, 0u, 0u};                 // bit v: channel clamped at 0 in view v
    float dX[3] = {0.f, 0.f, 0.f};
    float dlogit = 0.f;
    float dS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // dL/dSigma (symmetric), summed over views
    float dnorm = 0.f;
    uint32_t dviews = 0u;

    for (int v = 0; v < vb.B; ++v) {
        const int64_t idx = (int64_t)v * s.N + g;
        if (p.radius[idx] <= 0) continue;
        const ViewCam &c = vb.v[v];
        const float4 co = p.conic_o[idx];
        float4 gxo = gv.d_xy_o[idx], gco = gv.d_conic[idx];
        const float4 grg = gv.d_rgb[idx];
        if (!grads_ready) moments_to_grads(co, float4(gxo), float4(gco), gxo, gco);
        if (dacc) {                              // densification statistics of this view
            dnorm += sqrtf(gxo.x * gxo.x + gxo.y * gxo.y);
            ++dviews;
        }
        dlogit += gxo.z * G.o * (1.f - G.o);
        // ---- colour -> SH and viewing direction
        float ddx = G.x - c.C[0], ddy = G.y - c.C[1], ddz = G.z - c.C[2];
        const float dist = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
        const float il = 1.f / dist;
        ddx *= il; ddy *= il; ddz *= il;
        float Y[16];
        sh_eval(ddx, ddy, ddz, Y);
        float drgb[3] = {grg.x, grg.y, grg.z};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < nk) acc += shf[3 * k + ch] * Y[k];
            if (acc + 0.5f < 0.f) {
                drgb[ch] = 0.f;
                clampm[ch] |= 1u << v;
            }
        }
        float w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            w[k] = 0.f;
            if (k < nk) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) w[k] += shf[3 * k + ch] * drgb[ch];
            }
        }
        float gx, gy, gz;
        sh_grad_dot(ddx, ddy, ddz, w, nk, gx, gy, gz);
        const float dd = ddx * gx + ddy * gy + ddz * gz;
        dX[0] += (gx - ddx * dd) * il;
        dX[1] += (gy - ddy * dd) * il;
        dX[2] += (gz - ddz * dd) * il;
        // ---- recompute the projection pieces
        const float px = c.R[0] * G.x + c.R[1] * G.y + c.R[2] * G.z + c.t[0];
        const float py = c.R[3] * G.x + c.R[4] * G.y + c.R[5] * G.z + c.t[1];
        const float pz = c.R[6] * G.x + c.R[7] * G.y + c.R[8] * G.z + c.t[2];
        const float iz = 1.f / pz, iz2 = iz * iz;
        const float rx = px * iz, ry = py * iz;
        const bool clx = rx > c.limx || rx < -c.limx;
        const bool cly = ry > c.limy || ry < -c.limy;
        const float tx = fminf(c.limx, fmaxf(-c.limx, rx));
        const float ty = fminf(c.limy, fmaxf(-c.limy, ry));
        const float J00 = c.fx * iz, J02 = -c.fx * tx * iz;
        const float J11 = c.fy * iz, J12 = -c.fy * ty * iz;
        float T0[3], T1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T0[j] = J00 * c.R[j] + J02 * c.R[6 + j];
            T1[j] = J11 * c.R[3 + j] + J12 * c.R[6 + j];
        }
        // ---- conic -> 2D covariance: dS2 = -Q Gq Q, Gq = [[da, db/2], [db/2, dc]]
        const float qa = co.x, qb = co.y, qc = co.z;
        const float ga = gco.x, gb = 0.5f * gco.y, gc = gco.z;
        const float m00 = qa * ga + qb * gb, m01 = qa * gb + qb * gc;
        const float m10 = qb * ga + qc * gb, m11 = qb * gb + qc * gc;
        const float d00 = -(m00 * qa + m01 * qb);
        const float d01 = -(m00 * qb + m01 * qc);
        const float d11 = -(m10 * qb + m11 * qc);
        // ---- dSigma += T^T dS2 T
        {
            float U0[3], U1[3];   // dS2 T (2x3)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                U0[j] = d00 * T0[j] + d01 * T1[j];
                U1[j] = d01 * T0[j] + d11 * T1[j];
            }
            dS[0] += T0[0] * U0[0] + T1[0] * U1[0];
            dS[1] += T0[0] * U0[1] + T1[0] * U1[1];
            dS[2] += T0[0] * U0[2] + T1[0] * U1[2];
            dS[3] += T0[1] * U0[1] + T1[1] * U1[1];
            dS[4] += T0[1] * U0[2] + T1[1] * U1[2];
            dS[5] += T0[2] * U0[2] + T1[2] * U1[2];
            // dT = 2 dS2 T Sigma  (2x3), with Sigma symmetric
            const float *S = G.S;
            float dT0[3], dT1[3];
            dT0[0] = 2.f * (U0[0] * S[0] + U0[1] * S[1] + U0[2] * S[2]);
            dT0[1] = 2.f * (U0[0] * S[1] + U0[1] * S[3] + U0[2] * S[4]);
            dT0[2] = 2.f * (U0[0] * S[2] + U0[1] * S[4] + U0[2] * S[5]);
            dT1[0] = 2.f * (U1[0] * S[0] + U1[1] * S[1] + U1[2] * S[2]);
            dT1[1] = 2.f * (U1[0] * S[1] + U1[1] * S[3] + U1[2] * S[4]);
            dT1[2] = 2.f * (U1[0] * S[2] + U1[1] * S[4] + U1[2] * S[5]);
            // dJ = dT R^T: only J00, J02, J11, J12 depend on the mean
            const float dJ00 = dT0[0] * c.R[0] + dT0[1] * c.R[1] + dT0[2] * c.R[2];
            const float dJ02 = dT0[0] * c.R[6] + dT0[1] * c.R[7] + dT0[2] * c.R[8];
            const float dJ11 = dT1[0] * c.R[3] + dT1[1] * c.R[4] + dT1[2] * c.R[5];
            const float dJ12 = dT1[0] * c.R[6] + dT1[1] * c.R[7] + dT1[2] * c.R[8];
            float dpx = 0.f, dpy = 0.f, dpz = 0.f;
            // J00 = fx/z, J02 = -fx xt/z^2 with xt = tx z; J11, J12 likewise
            dpz += -dJ00 * c.fx * iz2 + dJ02 * 2.f * c.fx * tx * iz2
                   - dJ11 * c.fy * iz2 + dJ12 * 2.f * c.fy * ty * iz2;
            const float dxt = -dJ02 * c.fx * iz2, dyt = -dJ12 * c.fy * iz2;
            if (clx) dpz += dxt * tx; else dpx += dxt;
            if (cly) dpz += dyt * ty; else dpy += dyt;
            // u = fx x/z + cx, v = fy y/z + cy
            dpx += gxo.x * c.fx * iz;
            dpy += gxo.y * c.fy * iz;
            dpz += -(gxo.x * c.fx * rx + gxo.y * c.fy * ry) * iz;
            // p = R x + t
            dX[0] += c.R[0] * dpx + c.R[3] * dpy + c.R[6] * dpz;
            dX[1] += c.R[1] * dpx + c.R[4] * dpy + c.R[7] * dpz;
            dX[2] += c.R[2] * dpx + c.R[5] * dpy + c.R[8] * dpz;
        }
    }
    // ---- second pass: the SH coefficients, dsh = sum over views of Y (x) dL/drgb
    float dsh[48];
#pragma unroll
    for (int j = 0; j < 48; ++j) dsh[j] = 0.f;
    for (int v = 0; v < vb.B; ++v) {
        const int64_t idx = (int64_t)v * s.N + g;
        if (p.radius[idx] <= 0) continue;
        const ViewCam &c = vb.v[v];
        const float4 grg = gv.d_rgb[idx];
        float ddx = G.x - c.C[0], ddy = G.y - c.C[1], ddz = G.z - c.C[2];
        const float il = 1.f / sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
        ddx *= il; ddy *= il; ddz *= il;
        float Y[16];
        sh_eval(ddx, ddy, ddz, Y);
        const float drgb[3] = {(clampm[0] >> v) & 1u ? 0.f : grg.x, (clampm[1] >> v) & 1u ? 0.f : grg.y,
                               (clampm[2] >> v) & 1u ? 0.f : grg.z};
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < nk) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) dsh[3 * k + ch] += Y[k] * drgb[ch];
            }
    }
    // ---- Sigma = M M^T, M = Rq diag(s): dM = 2 dSigma M
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = G.Rq[3 * i + j] * G.s[j];
    const float Sf[9] = {dS[0], dS[1], dS[2], dS[1], dS[3], dS[4], dS[2], dS[4], dS[5]};
    float dRq[9], dls[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float ds = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float dMij = 2.f * (Sf[3 * i] * M[j] + Sf[3 * i + 1] * M[3 + j] + Sf[3 * i + 2] * M[6 + j]);
            ds += dMij * G.Rq[3 * i + j];
            dRq[3 * i + j] = dMij * G.s[j];
        }
        dls[j] = ds * G.s[j];
    }
    const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
    const float *d = dRq;
    float dq[4];
    dq[0] = 2.f * (-z * d[1] + y * d[2] + z * d[3] - x * d[5] - y * d[6] + x * d[7]);
    dq[1] = 2.f * (y * d[1] + z * d[2] + y * d[3] - 2.f * x * d[4] - w * d[5] + z * d[6] + w * d[7] - 2.f * x * d[8]);
    dq[2] = 2.f * (-2.f * y * d[0] + x * d[1] + w * d[2] + x * d[3] + z * d[5] - w * d[6] + z * d[7] - 2.f * y * d[8]);
    dq[3] = 2.f * (-2.f * z * d[0] - w * d[1] + x * d[2] + w * d[3] - 2.f * z * d[4] + y * d[5] + x * d[6] + y * d[7]);
    const float pr = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    const float iq = 1.f / G.qnorm;
    // a step whose binning overflowed or whose sort gave up is run again or
    // dropped: its statistics are not added
    if (dacc && status->code != GS_ERR_CAPACITY && status->code != GS_ERR_TIMEOUT) {
        dacc[g] += dnorm;
        dcnt[g] += dviews;
    }
    out.mo[g] = make_float4(dX[0] * invB, dX[1] * invB, dX[2] * invB, dlogit * invB);
    out.ls[g] = make_float4(dls[0] * invB, dls[1] * invB, dls[2] * invB, 0.f);
    out.q[g] = make_float4((dq[0] - w * pr) * iq * invB, (dq[1] - x * pr) * iq * invB,
                           (dq[2] - y * pr) * iq * invB, (dq[3] - z * pr) * iq * invB);
#pragma unroll
    for (int k = 0; k < 12; ++k)
        out.sh[(int64_t)k * s.N + g] =
            make_float4(dsh[4 * k] * invB, dsh[4 * k + 1] * invB, dsh[4 * k + 2] * invB, dsh[4 * k + 3] * invB);
}

}  // namespace

void launch_preprocess_fwd(const SceneView &s, const ViewBatch &vb, const ProjView &p, uint32_t *ntiles,
                           uint2 *rect, DevStatus *status, int strict, cudaStream_t st, uint4 *rm, float cull_alpha)
{
    if (s.N == 0) return;
    const int threads = 128;
    const int64_t blocks = (s.N + threads - 1) / threads;
    k_preprocess_fwd<<<(unsigned)blocks, threads, 0, st>>>(s, vb, p, ntiles, rect, status, strict,
                                                           rect ? rm : nullptr, cull_alpha);
    count_launches(1);
}

void launch_preprocess_bwd(const SceneView &s, const ViewBatch &vb, const ProjView &p, const GradView &g,
                           bool grads_ready, const SceneMut &out, uint8_t *vis, cudaStream_t st, float *dacc,
                           uint32_t *dcnt, const DevStatus *status, float scale)
{
    if (s.N == 0) return;
    const int threads = 128;
    const int64_t blocks = (s.N + threads - 1) / threads;
    if (scale < 0.f) scale = 1.f / (float)vb.B;
    k_preprocess_bwd<<<(unsigned)blocks, threads, 0, st>>>(s, vb, p, g, grads_ready, out, vis, dacc, dcnt, status,
                                                           scale);
    count_launches(1);
}

void launch_moments_to_grads(const ProjView &p, int64_t n, const GradView &g, cudaStream_t st)
{
    if (n <= 0) return;
    k_moments_to_grads<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, g);
    count_launches(1);
}

}  // namespace gs
