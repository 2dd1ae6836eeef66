// K6 (front-to-back compositing, Sec. 2.1 step 2) and K7 (its backward).
//
// One CTA per screen tile (tile x tile pixels, one pixel per thread).  The
// tile's depth-sorted fragment list is walked in batches of BATCH Gaussians
// staged into shared memory (coalesced 8/16-byte gathers of the screen-space
// state), so every Gaussian is read from global memory once per tile.
// Forward: a warp stops iterating once all of its pixels have saturated, and
// the CTA stops fetching batches once __syncthreads_count says every pixel
// has (early termination on transmittance).
// Backward: walks the same list back to front from the tile's largest
// n_contrib, recovers the transmittance before each contributor by division
// from T_final (no per-fragment state is stored), reduces the nine gradient
// components across the warp with shuffles, and issues three float4 atomics
// per (warp, Gaussian) instead of 9 scalar atomics per (pixel, Gaussian).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr float LOG2E = 1.4426950408889634f;

struct SmemG {        // one staged Gaussian (forward)
    float2 xy;
    float4 q;         // (-a/2, -b, -c/2) * log2(e), opacity
    float4 rgb;
};

// Exponent (base 2) of the Gaussian at offset (dx, dy); written with explicit
// round-to-nearest operations so the forward and the backward evaluate it to
// the same bits whatever the compiler fuses around it.
__device__ __forceinline__ float power2(const float4 &q, float dx, float dy)
{
    const float dxdx = __fmul_rn(dx, dx), dydy = __fmul_rn(dy, dy), dxdy = __fmul_rn(dx, dy);
    return __fmaf_rn(q.x, dxdx, __fmaf_rn(q.z, dydy, __fmul_rn(q.y, dxdy)));
}

__device__ __forceinline__ float4 stage_q(const float4 &co)
{
    return make_float4(-0.5f * LOG2E * co.x, -LOG2E * co.y, -0.5f * LOG2E * co.z, co.w);
}

__device__ __forceinline__ int find_view(const ViewBatch &vb, uint32_t tile_id)
{
    int v = 0;
    while (v + 1 < vb.B && vb.v[v + 1].tile_base <= tile_id) ++v;
    return v;
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE *TILE) k_blend_fwd(ViewBatch vb, ProjView p, const uint32_t *vals,
                                                          const uint2 *ranges, BlendParams bp, DevStatus *status)
{
    constexpr int NT = TILE * TILE;
    __shared__ SmemG sg[BATCH];
    __shared__ uint32_t s_red[NT / 32];
    const uint32_t tile_id = blockIdx.x;
    const int v = find_view(vb, tile_id);
    const ViewCam &c = vb.v[v];
    const uint32_t local = tile_id - c.tile_base;
    const int ty = (int)(local / (uint32_t)c.TX), tx = (int)(local % (uint32_t)c.TX);
    const int px = tx * TILE + (int)(threadIdx.x % TILE);
    const int py = ty * TILE + (int)(threadIdx.x / TILE);
    const bool inside = px < c.W && py < c.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 rg = ranges[tile_id];
    const int64_t vbase = (int64_t)v * p.N;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t nc = 0, ne = 0;
    bool done = !inside;
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += BATCH) {
        if (__syncthreads_count(done) == NT) break;
        for (int t = threadIdx.x; t < BATCH; t += NT) {
            const uint32_t j = b0 + t;
            if (j < rg.y) {
                const int64_t idx = vbase + vals[j];
                SmemG s;
                s.xy = p.xy[idx];
                s.q = stage_q(p.conic_o[idx]);
                s.rgb = p.rgb_d[idx];
                sg[t] = s;
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BATCH, rg.y - b0);
        if (!done) {
            int k = 0;
            for (; k < cnt; ++k) {
                const SmemG &s = sg[k];
                const float dx = __fsub_rn(fx, s.xy.x), dy = __fsub_rn(fy, s.xy.y);
                const float pw = power2(s.q, dx, dy);
                if (pw > 0.f) continue;
                const float alpha = fminf(bp.alpha_max, s.q.w * exp2f(pw));
                if (alpha < bp.alpha_min) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < bp.T_min) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                C0 += s.rgb.x * w;
                C1 += s.rgb.y * w;
                C2 += s.rgb.z * w;
                T = Tn;
                nc = b0 - rg.x + k + 1;
            }
            ne = b0 - rg.x + min(k + 1, cnt);
        }
    }
    if (inside) {
        const int64_t pix = (int64_t)py * c.W + px;
        const int64_t hw = (int64_t)c.W * c.H;
        c.img[pix] = C0 + T * bp.bg[0];
        c.img[hw + pix] = C1 + T * bp.bg[1];
        c.img[2 * hw + pix] = C2 + T * bp.bg[2];
        c.T_final[pix] = T;
        c.n_contrib[pix] = nc;
    }
    // (pixel, fragment) evaluations for the roofline counters
    uint32_t s = inside ? ne : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < NT / 32; ++w) tot += s_red[w];
        if (tot) atomicAdd(&status->counters[1], tot);
    }
}

struct SmemGB {       // one staged Gaussian (backward)
    float2 xy;
    float4 q;         // as forward
    float4 conic;     // (a, b, c, -)
    float4 rgb;
    uint32_t g;
};

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE *TILE) k_blend_bwd(ViewBatch vb, ProjView p, const uint32_t *vals,
                                                          const uint2 *ranges, BlendParams bp, GradView gv,
                                                          DevStatus *status)
{
    constexpr int NT = TILE * TILE;
    __shared__ SmemGB sg[BATCH];
    __shared__ uint32_t s_red[NT / 32];
    const uint32_t tile_id = blockIdx.x;
    const int v = find_view(vb, tile_id);
    const ViewCam &c = vb.v[v];
    const uint32_t local = tile_id - c.tile_base;
    const int ty = (int)(local / (uint32_t)c.TX), tx = (int)(local % (uint32_t)c.TX);
    const int px = tx * TILE + (int)(threadIdx.x % TILE);
    const int py = ty * TILE + (int)(threadIdx.x / TILE);
    const bool inside = px < c.W && py < c.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 rg = ranges[tile_id];
    const int64_t vbase = (int64_t)v * p.N;
    const int lane = threadIdx.x & 31;

    float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
    uint32_t nc = 0;
    if (inside) {
        const int64_t pix = (int64_t)py * c.W + px;
        const int64_t hw = (int64_t)c.W * c.H;
        T = c.T_final[pix];
        nc = c.n_contrib[pix];
        dC0 = c.d_img[pix];
        dC1 = c.d_img[hw + pix];
        dC2 = c.d_img[2 * hw + pix];
    }
    // largest n_contrib in the tile bounds the backward walk
    uint32_t m = nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    uint32_t maxnc = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) maxnc = max(maxnc, s_red[w]);
    maxnc = min(maxnc, rg.y - rg.x);   // never walk past the tile's list, whatever n_contrib holds
    __syncthreads();

    float B0 = bp.bg[0], B1 = bp.bg[1], B2 = bp.bg[2];   // colour behind (normalised)
    uint32_t evals = 0;
    for (int64_t end = (int64_t)rg.x + maxnc; end > (int64_t)rg.x; end -= BATCH) {
        const int64_t start = max((int64_t)rg.x, end - BATCH);
        const int cnt = (int)(end - start);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += NT) {
            const uint32_t j = (uint32_t)(end - 1 - t);
            const uint32_t g = vals[j];
            const int64_t idx = vbase + g;
            const float4 co = p.conic_o[idx];
            SmemGB s;
            s.xy = p.xy[idx];
            s.q = stage_q(co);
            s.conic = co;
            s.rgb = p.rgb_d[idx];
            s.g = g;
            sg[t] = s;
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const uint32_t rel = (uint32_t)(end - 1 - k - rg.x);
            const SmemGB &s = sg[k];
            bool act = rel < nc;
            float gu = 0.f, gvv = 0.f, go = 0.f, ga = 0.f, gb = 0.f, gc = 0.f, gr = 0.f, gg = 0.f, gbl = 0.f;
            if (act) {
                const float dx = __fsub_rn(fx, s.xy.x), dy = __fsub_rn(fy, s.xy.y);
                const float pw = power2(s.q, dx, dy);
                const float G = exp2f(pw);
                const float oG = s.q.w * G;
                const float alpha = fminf(bp.alpha_max, oG);
                act = !(pw > 0.f) && !(alpha < bp.alpha_min);
                if (act) {
                    ++evals;
                    const float Tj = __fdividef(T, 1.f - alpha);
                    const float w = alpha * Tj;
                    gr = w * dC0;
                    gg = w * dC1;
                    gbl = w * dC2;
                    const float dalpha = Tj * ((s.rgb.x - B0) * dC0 + (s.rgb.y - B1) * dC1 + (s.rgb.z - B2) * dC2);
                    B0 = alpha * s.rgb.x + (1.f - alpha) * B0;
                    B1 = alpha * s.rgb.y + (1.f - alpha) * B1;
                    B2 = alpha * s.rgb.z + (1.f - alpha) * B2;
                    T = Tj;
                    if (oG < bp.alpha_max) {
                        const float dpow = alpha * dalpha;
                        go = G * dalpha;
                        gu = (s.conic.x * dx + s.conic.y * dy) * dpow;
                        gvv = (s.conic.y * dx + s.conic.z * dy) * dpow;
                        ga = -0.5f * dx * dx * dpow;
                        gb = -dx * dy * dpow;
                        gc = -0.5f * dy * dy * dpow;
                    }
                }
            }
            if (__any_sync(0xffffffffu, act)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    gu += __shfl_xor_sync(0xffffffffu, gu, o);
                    gvv += __shfl_xor_sync(0xffffffffu, gvv, o);
                    go += __shfl_xor_sync(0xffffffffu, go, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    gb += __shfl_xor_sync(0xffffffffu, gb, o);
                    gc += __shfl_xor_sync(0xffffffffu, gc, o);
                    gr += __shfl_xor_sync(0xffffffffu, gr, o);
                    gg += __shfl_xor_sync(0xffffffffu, gg, o);
                    gbl += __shfl_xor_sync(0xffffffffu, gbl, o);
                }
                if (lane == 0) {
                    const int64_t idx = vbase + s.g;
                    atomicAdd(&gv.d_xy_o[idx], make_float4(gu, gvv, go, 0.f));
                    atomicAdd(&gv.d_conic[idx], make_float4(ga, gb, gc, 0.f));
                    atomicAdd(&gv.d_rgb[idx], make_float4(gr, gg, gbl, 0.f));
                }
            }
        }
    }
    uint32_t s = evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < NT / 32; ++w) tot += s_red[w];
        if (tot) atomicAdd(&status->counters[2], tot);
    }
}

template <int TILE>
void fwd_tile(int batch, const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
              const BlendParams &bp, DevStatus *status, cudaStream_t st)
{
    const unsigned grid = vb.total_tiles;
    if (batch <= 128)
        k_blend_fwd<TILE, 128><<<grid, TILE * TILE, 0, st>>>(vb, p, vals, ranges, bp, status);
    else if (batch <= 256)
        k_blend_fwd<TILE, 256><<<grid, TILE * TILE, 0, st>>>(vb, p, vals, ranges, bp, status);
    else
        k_blend_fwd<TILE, 512><<<grid, TILE * TILE, 0, st>>>(vb, p, vals, ranges, bp, status);
}

template <int TILE>
void bwd_tile(int batch, const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
              const BlendParams &bp, const GradView &g, DevStatus *status, cudaStream_t st)
{
    const unsigned grid = vb.total_tiles;
    if (batch <= 128)
        k_blend_bwd<TILE, 128><<<grid, TILE * TILE, 0, st>>>(vb, p, vals, ranges, bp, g, status);
    else if (batch <= 256)
        k_blend_bwd<TILE, 256><<<grid, TILE * TILE, 0, st>>>(vb, p, vals, ranges, bp, g, status);
    else
        k_blend_bwd<TILE, 512><<<grid, TILE * TILE, 0, st>>>(vb, p, vals, ranges, bp, g, status);
}

}  // namespace

void launch_blend_fwd(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                      const BlendParams &bp, int batch, DevStatus *status, cudaStream_t st)
{
    if (vb.total_tiles == 0) return;
    switch (vb.tile) {
    case 8: fwd_tile<8>(batch, vb, p, vals, ranges, bp, status, st); break;
    case 32: fwd_tile<32>(batch, vb, p, vals, ranges, bp, status, st); break;
    default: fwd_tile<16>(batch, vb, p, vals, ranges, bp, status, st); break;
    }
    count_launches(1);
}

void launch_blend_bwd(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                      const BlendParams &bp, int batch, const GradView &g, DevStatus *status, cudaStream_t st)
{
    if (vb.total_tiles == 0) return;
    switch (vb.tile) {
    case 8: bwd_tile<8>(batch, vb, p, vals, ranges, bp, g, status, st); break;
    case 32: bwd_tile<32>(batch, vb, p, vals, ranges, bp, g, status, st); break;
    default: bwd_tile<16>(batch, vb, p, vals, ranges, bp, g, status, st); break;
    }
    count_launches(1);
}

}  // namespace gs
