// K6 (front-to-back compositing, Sec. 2.1 step 2) and K7 (its backward).
//
// One CTA per screen tile of TILE x TILE pixels; a thread blends PPT pixels
// of one column (rows 4 apart), so warp w owns an 8 x 4 PPT block of the
// tile.  Warps work independently (no block-wide
// barrier inside the walk): a warp reads the tile's depth-sorted list in
// rounds of 32 entries (lane i gathers entry i with coalesced 8/16-byte loads;
// the warps of a tile hit the same L1 lines; the next round's gathers are
// issued before the current round is used), keeps only the Gaussians whose
// alpha >= alpha_min ellipse meets the warp's block (ballot + prefix
// compaction into the warp's buffer of CH entries in shared memory, order
// preserved), and walks the buffer when another round could overflow it.  So
// a warp spends nothing on list entries that cannot reach its pixels, and
// finishes as soon as its own pixels do (no block-wide barrier at all).  The staged record holds
// the midpoint of the exponent interval [cut, 0] outside which alpha <
// alpha_min (or the pixel is off the quadratic form), so most (pixel,
// Gaussian) pairs are rejected before the exponential.
// With more than one pixel per thread, a lane's k-th pixels form row k of
// the warp's block: for each staged entry both passes evaluate every pixel's
// exponent, vote per row whether any lane passes, and run the blending
// arithmetic only for those rows, without per-pixel branches (a pixel that
// does not blend takes alpha 0 or weight 0).
// Forward: a pixel stops once it would saturate; the warp stops refilling
// when all its pixels have (early termination on transmittance).
// Backward: each warp walks back to front from its own largest n_contrib,
// recovers the transmittance before each contributor by division from
// T_final (no per-fragment state is stored), accumulates per Gaussian the
// moments of dpow = alpha dL/dalpha (M, Mx, My, Mxx, Mxy, Myy; the mean,
// conic and opacity gradients are linear in them; a lane's pixels share one
// column, so it sums only M, My, Myy and scales by dx once per entry) and the
// colour gradient, and adds these nine values to the Gaussian as three float4 atomics: from
// each contributing lane directly when few lanes contribute, after a
// reduce-scatter over the warp (17 shuffles) or a fold of the upper half-warp
// when many do (add_sums, flush_one).  The moments become gradients once per
// (view, Gaussian) afterwards (moments_to_grads).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr float LOG2E = 1.4426950408889634f;

// Base-2 exponent of the Gaussian at offset (dx, dy), evaluated as
// dy (C dy + B dx) + A dx^2 with explicitly rounded operations, so the
// forward and the backward get the same bits whatever the compiler fuses
// around it; q = (A, B, C, o) = (-a/2, -b, -c/2) log2(e), opacity.  The dx
// terms are shared by the pixels of one column.
struct DxTerms {
    float adx2, bdx;          // A dx^2 and B dx
};

__device__ __forceinline__ DxTerms dx_terms(const float4 &q, float dx)
{
    return DxTerms{__fmul_rn(q.x, __fmul_rn(dx, dx)), __fmul_rn(q.y, dx)};
}

__device__ __forceinline__ float power2(const float4 &q, const DxTerms &t, float dy)
{
    return __fmaf_rn(dy, __fmaf_rn(q.z, dy, t.bdx), t.adx2);
}

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float4 stage_q(const float4 &co)
{
    return make_float4(-0.5f * LOG2E * co.x, -LOG2E * co.y, -0.5f * LOG2E * co.z, co.w);
}

// The exponents worth an exponential lie in [cut, 0] (below cut, o * 2^pw <
// alpha_min; above 0, the pixel is off the Gaussian's quadratic form).  The
// staged record keeps the interval's midpoint m = cut / 2 (exact), so that one
// subtraction and one comparison, |pw - m| <= -m, test both ends.  Forward and
// backward use the same test, so their decisions agree exactly.
__device__ __forceinline__ float exponent_mid(float o, float alpha_min);
__device__ __forceinline__ bool in_cut(float pw, float mid)
{
    return fabsf(__fsub_rn(pw, mid)) <= -mid;
}

__device__ __forceinline__ float exponent_cut(float o, float alpha_min)
{
    return o > alpha_min ? __log2f(__fdividef(alpha_min, o)) : 1.f;
}

__device__ __forceinline__ float exponent_mid(float o, float alpha_min)
{
    return 0.5f * exponent_cut(o, alpha_min);
}

// The tile's [start, end) in the fragment list.  A reversed range (the
// ranges of a sort that failed, which is reported already) or one that ends
// past the list (only a caller's corrupt ranges) is treated as empty, so no
// read leaves the list; the second also records GS_ERR_INVALID_ARG.
__device__ __forceinline__ uint2 checked_range(const uint2 *ranges, uint32_t tile_id, const BlendParams &bp,
                                               DevStatus *status)
{
    const uint2 rg = ranges[tile_id];
    if (rg.x <= rg.y && rg.y <= bp.list_cap) return rg;
    if (rg.y > bp.list_cap && threadIdx.x == 0) atomicCAS(&status->code, 0, (int)GS_ERR_INVALID_ARG);
    return make_uint2(0u, 0u);
}

__device__ __forceinline__ int find_view(const ViewBatch &vb, uint32_t tile_id)
{
    int v = 0;
    while (v + 1 < vb.B && vb.v[v + 1].tile_base <= tile_id) ++v;
    return v;
}

// Warp-wide sums of one entry's nine values v[0..8] (the moments and colour
// sums of GradView), added to entry idx.  v[0..7] go through a reduce-scatter
// (at each level a lane keeps half of its values and ships the other half:
// 4 + 2 + 1 + 1 + 1 = 9 shuffles, after which value k is in lanes
// 4k .. 4k+3), v[8] through a butterfly (5); lanes 0..2 gather three values
// each (3 shuffles) and add one float4 each.
__device__ __forceinline__ void flush_one(const GradView &gv, int64_t idx, const float v[9], int lane)
{
    float w[4], x[2];
    const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float send = b4 ? v[j] : v[j + 4];
        const float keep = b4 ? v[j + 4] : v[j];
        w[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float send = b3 ? w[j] : w[j + 2];
        const float keep = b3 ? w[j + 2] : w[j];
        x[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    float t = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const int src = 12 * (lane < 3 ? lane : 0);
    const float g0 = __shfl_sync(0xffffffffu, y, src);
    const float g1 = __shfl_sync(0xffffffffu, y, src + 4);
    const float g2 = __shfl_sync(0xffffffffu, y, (src + 8) & 31);
    if (lane < 3) {
        float4 *dst = lane == 0 ? &gv.d_xy_o[idx] : lane == 1 ? &gv.d_conic[idx] : &gv.d_rgb[idx];
        atomicAdd(dst, make_float4(g0, g1, lane == 2 ? t : g2, 0.f));
    }
}

// One lane's own sums of an entry (moments in vv[0..5], colour sums in
// vv[6], vv[7], b), added to entry idx as three float4 atomics.
__device__ __forceinline__ void add_sums(const GradView &gv, int64_t idx, const float vv[8], float b)
{
    atomicAdd(&gv.d_xy_o[idx], make_float4(vv[0], vv[1], vv[2], 0.f));
    atomicAdd(&gv.d_conic[idx], make_float4(vv[3], vv[4], vv[5], 0.f));
    atomicAdd(&gv.d_rgb[idx], make_float4(vv[6], vv[7], b, 0.f));
}

// How an entry's sums leave the warp, by the number of contributing lanes
// (measured on GB300 over the launch shapes the autotuner picks).  Float4
// atomics from many lanes to one address are cheap next to the 17-shuffle
// reduce-scatter until about 20 lanes contribute; with 4 pixels per thread,
// folding the upper half-warp (9 shuffles) and adding from at most 16 lanes
// beats both.
constexpr int DIRECT_UP_TO = 20;   // 1 or 2 pixels per thread: lanes adding directly, else reduce-scatter
constexpr int FOLD_ABOVE = 16;     // 4 pixels per thread: fold when more lanes contribute

// Tile-local geometry of this thread's PPT pixels (one column, rows 4 apart)
// and its warp's 8 x 4 PPT block.
template <int PPT>
struct PixelSite {
    int px, py[PPT];
    bool inside[PPT];
    float fx, fy[PPT];        // pixel centres
    float bx0, bx1, by0, by1; // pixel-centre extent of the warp's block
};

template <int TILE, int PPT>
__device__ __forceinline__ PixelSite<PPT> pixel_site(const ViewCam &c, uint32_t local, int warp, int lane)
{
    PixelSite<PPT> s;
    const int ty = (int)(local / (uint32_t)c.TX), tx = (int)(local % (uint32_t)c.TX);
    const int wx = (warp % (TILE / 8)) * 8, wy = (warp / (TILE / 8)) * (4 * PPT);
    s.px = tx * TILE + wx + (lane & 7);
    s.fx = (float)s.px + 0.5f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        s.py[k] = ty * TILE + wy + (lane >> 3) + 4 * k;
        s.inside[k] = s.px < c.W && s.py[k] < c.H;
        s.fy[k] = (float)s.py[k] + 0.5f;
    }
    s.bx0 = (float)(tx * TILE + wx) + 0.5f;
    s.bx1 = s.bx0 + 7.f;
    s.by0 = (float)(ty * TILE + wy) + 0.5f;
    s.by1 = s.by0 + (float)(4 * PPT - 1);
    return s;
}

// Compile-time pixel index (k) for the per-pixel bodies of the blending kernels.
template <int K>
struct PixelK {
    static constexpr int value = K;
};

// One list entry as gathered by a lane during a refill.
struct Entry {
    bool ok;
    uint32_t g;
    float2 xy;
    float4 co;
};

__device__ __forceinline__ Entry fetch_entry(const ProjView &p, const uint32_t *vals, int64_t vbase, int64_t j,
                                             bool valid)
{
    Entry e;
    e.g = valid ? vals[j] : 0u;
    e.ok = valid && (int64_t)e.g < p.N;           // an index >= N only after a failed (timed-out) sort
    e.xy = make_float2(0.f, 0.f);
    e.co = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e.ok) {
        const int64_t idx = vbase + e.g;
        e.xy = p.xy[idx];
        e.co = p.conic_o[idx];
    }
    return e;
}

// Bytes of dynamic shared memory per CTA: three float4 per staged entry.
template <int TILE, int CH, int PPT>
constexpr size_t smem_bytes()
{
    return (size_t)(TILE * TILE / (32 * PPT)) * CH * 3 * sizeof(float4);
}

// Measured cost of one warp's part of a tile (for the Algorithm 1 schedule):
// elapsed SM cycles / 1024, plus 1 so that an empty tile still counts.
__device__ __forceinline__ void add_cost(uint32_t *cost, uint32_t tile_id, long long t0, int lane)
{
    if (cost && lane == 0) atomicAdd(&cost[tile_id], (uint32_t)((clock64() - t0) >> 10) + 1u);
}

// The forward of one tile (tile_id, global over the batch's views) by this
// CTA; each warp works alone, so a CTA can go on to another tile warp by warp.
template <int TILE, int CH, int PPT, bool COUNT>
__device__ __forceinline__ void blend_fwd_tile(uint32_t tile_id, const ViewBatch &vb, const ProjView &p,
                                               const uint32_t *vals, const uint2 *ranges, const BlendParams &bp,
                                               DevStatus *status, uint32_t *cost)
{
    constexpr int NW = TILE * TILE / (32 * PPT);
    extern __shared__ float4 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *s_xyc = smem + warp * CH;              // u, v, exponent_mid, list position + 1 (bits)
    float4 *s_q = smem + (NW + warp) * CH;         // A, B, C, opacity
    float4 *s_rgb = smem + (2 * NW + warp) * CH;
    const long long t0 = cost ? clock64() : 0ll;

    const int v = find_view(vb, tile_id);
    const ViewCam &c = vb.v[v];
    const PixelSite<PPT> ps = pixel_site<TILE, PPT>(c, tile_id - c.tile_base, warp, lane);
    const uint2 rg = checked_range(ranges, tile_id, bp, status);
    const int64_t vbase = (int64_t)v * p.N;
    const uint32_t lt = (1u << lane) - 1u;

    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t nc[PPT], ne[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        nc[k] = ne[k] = 0u;
        done[k] = !ps.inside[k];
    }
    // Rounds of 32 entries, software-pipelined: the gathers of the next round
    // are in flight while the current one is tested and staged.  Hits pile up
    // in the warp's buffer, which is walked when another round could overflow
    // it, or at the end of the list.
    int n = 0;
    Entry nxt = fetch_entry(p, vals, vbase, (int64_t)rg.x + lane, rg.x + lane < rg.y);
    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        const Entry e = nxt;
        const uint32_t j = base + lane;
        if (base + 32 < rg.y) nxt = fetch_entry(p, vals, vbase, (int64_t)j + 32, j + 32 < rg.y);
        const bool hit = e.ok && ellipse_box_hits(e.co, e.xy.x, e.xy.y, bp.alpha_min, ps.bx0, ps.bx1, ps.by0, ps.by1);
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int slot = n + __popc(bal & lt);
            const float4 q = stage_q(e.co);
            s_xyc[slot] = make_float4(e.xy.x, e.xy.y, exponent_mid(q.w, bp.alpha_min), __uint_as_float(j - rg.x + 1u));
            s_q[slot] = q;
            s_rgb[slot] = p.rgb_d[vbase + e.g];
        }
        n += __popc(bal);
        const bool last = base + 32 >= rg.y;
        if (n > CH - 32 || last) {
            __syncwarp();
            bool all_done = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) all_done = all_done && done[k];
            // (more than one pixel per thread: the walk votes across the warp, so every lane enters it)
            if (PPT > 1 ? !__all_sync(0xffffffffu, all_done) : !all_done) {
                for (int i = 0; i < n; ++i) {
                    const float4 xyc = s_xyc[i];
                    const float4 q = s_q[i];
                    const DxTerms dt = dx_terms(q, __fsub_rn(ps.fx, xyc.x));
                    const uint32_t pos1 = __float_as_uint(xyc.w);
                    if constexpr (PPT == 1) {
                        // one pixel: without branches (a miss blends with weight 0)
                        if (done[0]) break;
                        const float pw = power2(q, dt, __fsub_rn(ps.fy[0], xyc.y));
                        const float a0 = fminf(bp.alpha_max, q.w * ex2(pw));
                        bool hit = in_cut(pw, xyc.z) && a0 >= bp.alpha_min;
                        const float Tn = T[0] * (1.f - a0);
                        if (hit && Tn < bp.T_min) {
                            done[0] = true;
                            if constexpr (COUNT) ne[0] = pos1;
                            hit = false;
                        }
                        const float4 rgb = s_rgb[i];
                        const float w = hit ? a0 * T[0] : 0.f;
                        C0[0] += rgb.x * w;
                        C1[0] += rgb.y * w;
                        C2[0] += rgb.z * w;
                        T[0] = hit ? Tn : T[0];
                        nc[0] = hit ? pos1 : nc[0];
                    } else {
                        // two or four pixels: the exponents first, then the
                        // blending only for the pixel rows where some lane
                        // passes (warp-uniform branches, no per-pixel ones);
                        // the lanes leave together once every pixel is done
                        float pw[PPT];
                        bool pass[PPT];
                        uint32_t rows = 0u;
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            pw[k] = power2(q, dt, __fsub_rn(ps.fy[k], xyc.y));
                            pass[k] = !done[k] && in_cut(pw[k], xyc.z);
                            rows |= __any_sync(0xffffffffu, pass[k]) ? 1u << k : 0u;
                        }
                        if (rows == 0u) {
                            bool fin = true;
#pragma unroll
                            for (int k = 0; k < PPT; ++k) fin = fin && done[k];
                            if (__all_sync(0xffffffffu, fin)) break;
                            continue;
                        }
                        const float4 rgb = s_rgb[i];
                        auto pixel = [&](auto kc) {
                            constexpr int k = decltype(kc)::value;
                            const float a0 = fminf(bp.alpha_max, q.w * ex2(pw[k]));
                            bool hit = pass[k] && a0 >= bp.alpha_min;
                            const float Tn = T[k] * (1.f - a0);
                            const bool term = hit && Tn < bp.T_min;     // would saturate: stop before it
                            done[k] = done[k] || term;
                            if constexpr (COUNT) ne[k] = term ? pos1 : ne[k];
                            hit = hit && !term;
                            const float w = hit ? a0 * T[k] : 0.f;
                            C0[k] += rgb.x * w;
                            C1[k] += rgb.y * w;
                            C2[k] += rgb.z * w;
                            T[k] = hit ? Tn : T[k];
                            nc[k] = hit ? pos1 : nc[k];
                        };
                        if constexpr (PPT == 2) {
                            if (rows == 3u) {                       // both rows: the two pixels interleave
                                pixel(PixelK<0>{});
                                pixel(PixelK<1>{});
                            } else if (rows == 1u) {
                                pixel(PixelK<0>{});
                            } else {
                                pixel(PixelK<1>{});
                            }
                        } else {
                            if (rows & 1u) pixel(PixelK<0>{});
                            if (rows & 2u) pixel(PixelK<1>{});
                            if (rows & 4u) pixel(PixelK<2>{});
                            if (rows & 8u) pixel(PixelK<3>{});
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (COUNT && !done[k]) ne[k] = min(base + 32, rg.y) - rg.x;
            }
            n = 0;
            __syncwarp();
            bool fin = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) fin = fin && done[k];
            if (__all_sync(0xffffffffu, fin)) break;
        }
    }
    const int64_t hw = (int64_t)c.W * c.H;
    uint32_t evals = 0, contrib = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!ps.inside[k]) continue;
        const int64_t pix = (int64_t)ps.py[k] * c.W + ps.px;
        c.img[pix] = C0[k] + T[k] * bp.bg[0];
        c.img[hw + pix] = C1[k] + T[k] * bp.bg[1];
        c.img[2 * hw + pix] = C2[k] + T[k] * bp.bg[2];
        c.T_final[pix] = T[k];
        c.n_contrib[pix] = nc[k];
        evals += ne[k];
        contrib += nc[k];
    }
    // (pixel, list position) evaluations until termination, and positions
    // below n_contrib (the backward's share), for the roofline counters when
    // asked; each warp adds its own (no block barrier: warps finish apart)
    if constexpr (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            evals += __shfl_xor_sync(0xffffffffu, evals, o);
            contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        }
        if (lane == 0 && evals) atomicAdd(&status->counters[1], (unsigned long long)evals);
        if (lane == 0 && contrib) atomicAdd(&status->counters[5], (unsigned long long)contrib);
    }
    add_cost(cost, tile_id, t0, lane);
}

// One CTA per tile, in launch order `order` (null: index order).
template <int TILE, int CH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE *TILE / PPT) k_blend_fwd(ViewBatch vb, ProjView p, const uint32_t *vals,
                                                                const uint2 *ranges, BlendParams bp,
                                                                DevStatus *status, const uint32_t *order,
                                                                uint32_t *cost)
{
    const uint32_t tile_id = order ? order[blockIdx.x] : blockIdx.x;   // launch order (launch_tile_order)
    blend_fwd_tile<TILE, CH, PPT, COUNT>(tile_id, vb, p, vals, ranges, bp, status, cost);
}

// Algorithm 1 schedule: CTA k blends the tiles [div[k], div[k + 1]) one after
// another (the last range ends at the last tile), ranges of about equal
// measured cost.
template <int TILE, int CH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE *TILE / PPT) k_blend_fwd_ranges(ViewBatch vb, ProjView p,
                                                                       const uint32_t *vals, const uint2 *ranges,
                                                                       BlendParams bp, DevStatus *status,
                                                                       const uint32_t *div, uint32_t *cost)
{
    const uint32_t lo = div[blockIdx.x];
    const uint32_t hi = blockIdx.x + 1 < gridDim.x ? min(div[blockIdx.x + 1], vb.total_tiles) : vb.total_tiles;
    for (uint32_t t = lo; t < hi; ++t) blend_fwd_tile<TILE, CH, PPT, COUNT>(t, vb, p, vals, ranges, bp, status, cost);
}

// Next position of a persistent CTA's work queue: thread 0 takes it from
// the global counter, every thread reads it, and no thread leaves the read
// before thread 0 may overwrite the slot for the next tile.
__device__ __forceinline__ uint32_t pool_next(uint32_t *queue)
{
    __shared__ uint32_t s_next;
    if (threadIdx.x == 0) s_next = atomicAdd(queue, 1u);
    __syncthreads();
    const uint32_t t = s_next;
    __syncthreads();
    return t;
}

// Persistent pool: a CTA per resident slot pulls the next tile of `order`
// (the previous step's measured costs, heaviest first; null: index order)
// from the queue counter until every tile is taken.
template <int TILE, int CH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE *TILE / PPT) k_blend_fwd_pool(ViewBatch vb, ProjView p,
                                                                     const uint32_t *vals, const uint2 *ranges,
                                                                     BlendParams bp, DevStatus *status,
                                                                     const uint32_t *order, uint32_t *queue,
                                                                     uint32_t *cost)
{
    for (uint32_t t = pool_next(queue); t < vb.total_tiles; t = pool_next(queue))
        blend_fwd_tile<TILE, CH, PPT, COUNT>(order ? order[t] : t, vb, p, vals, ranges, bp, status, cost);
}

// With 2 pixels per thread the backward is held to 64 registers (8 CTAs of
// 128 threads per SM; 4 bytes of spill): 1% faster on GB300 than at 68
// registers and 7 CTAs.  Other shapes keep the compiler's choice.
template <int TILE, int CH, int PPT, bool COUNT>
__device__ __forceinline__ void blend_bwd_tile(uint32_t tile_id, const ViewBatch &vb, const ProjView &p,
                                               const uint32_t *vals, const uint2 *ranges, const BlendParams &bp,
                                               const GradView &gv, DevStatus *status, uint32_t *cost)
{
    constexpr int NW = TILE * TILE / (32 * PPT);
    extern __shared__ float4 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *s_xyc = smem + warp * CH;                // u, v, exponent_mid, list position (bits)
    float4 *s_q = smem + (NW + warp) * CH;
    float4 *s_rgb = smem + (2 * NW + warp) * CH;    // r, g, b, Gaussian index (bits)
    const long long t0 = cost ? clock64() : 0ll;

    const int v = find_view(vb, tile_id);
    const ViewCam &c = vb.v[v];
    const PixelSite<PPT> ps = pixel_site<TILE, PPT>(c, tile_id - c.tile_base, warp, lane);
    const uint2 rg = checked_range(ranges, tile_id, bp, status);
    const int64_t vbase = (int64_t)v * p.N;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t hw = (int64_t)c.W * c.H;

    // Per pixel: T, dL/dC, and S = B . dL/dC, where B is the colour behind
    // the current entry (normalised by the transmittance in front of it).
    // dL/dalpha_i = T_i (c_i - B_i) . dL/dC = T_i (c_i . dL/dC - S_i), and
    // B_{i-1} = alpha_i c_i + (1 - alpha_i) B_i, so S obeys the same
    // recursion: one scalar instead of the three channels of B.
    float T[PPT], dC0[PPT], dC1[PPT], dC2[PPT], S[PPT];
    uint32_t nc[PPT], wnc = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.f;
        dC0[k] = dC1[k] = dC2[k] = 0.f;
        nc[k] = 0u;
        if (ps.inside[k]) {
            const int64_t pix = (int64_t)ps.py[k] * c.W + ps.px;
            T[k] = c.T_final[pix];
            nc[k] = c.n_contrib[pix];
            dC0[k] = c.d_img[pix];
            dC1[k] = c.d_img[hw + pix];
            dC2[k] = c.d_img[2 * hw + pix];
        }
        S[k] = bp.bg[0] * dC0[k] + bp.bg[1] * dC1[k] + bp.bg[2] * dC2[k];
        wnc = max(wnc, nc[k]);
    }
    // this warp walks back to front from its own largest n_contrib, never past the list
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wnc = max(wnc, __shfl_xor_sync(0xffffffffu, wnc, o));
    wnc = min(wnc, rg.y - rg.x);

    uint32_t evals = 0, walked = 0;
    // Rounds of 32 entries from the walk's top down, software-pipelined like
    // the forward; hits are staged in descending list order and walked when
    // another round could overflow the warp's buffer, or at the bottom.
    const int64_t top = (int64_t)rg.x + wnc;
    int n = 0;
    Entry nxt = fetch_entry(p, vals, vbase, top - 1 - lane, top - 1 - lane >= (int64_t)rg.x);
    for (int64_t hi = top; hi > (int64_t)rg.x; hi -= 32) {
        const Entry e = nxt;
        const int64_t j = hi - 1 - lane;
        if (hi - 32 > (int64_t)rg.x) nxt = fetch_entry(p, vals, vbase, j - 32, j - 32 >= (int64_t)rg.x);
        const bool hit = e.ok && ellipse_box_hits(e.co, e.xy.x, e.xy.y, bp.alpha_min, ps.bx0, ps.bx1, ps.by0, ps.by1);
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int slot = n + __popc(bal & lt);
            const float4 q = stage_q(e.co);
            const float4 rgbd = p.rgb_d[vbase + e.g];
            s_xyc[slot] = make_float4(e.xy.x, e.xy.y, exponent_mid(q.w, bp.alpha_min),
                                      __uint_as_float((uint32_t)(j - rg.x)));
            s_q[slot] = q;
            s_rgb[slot] = make_float4(rgbd.x, rgbd.y, rgbd.z, __uint_as_float(e.g));
        }
        n += __popc(bal);
        if (n <= CH - 32 && hi - 32 > (int64_t)rg.x) continue;
        __syncwarp();
        for (int i = 0; i < n; ++i) {
            const float4 xyc = s_xyc[i];
            const uint32_t rel = __float_as_uint(xyc.w);
            const float4 q = s_q[i];
            const float dx = __fsub_rn(ps.fx, xyc.x);
            const DxTerms dt = dx_terms(q, dx);
            // The exponent of every pixel first; the rest only for the pixel
            // rows (k) where some lane passes the cut (warp-uniform branches:
            // an entry that reaches only one of a lane's pixels costs one
            // pixel's arithmetic), there without branches: a pixel that does
            // not blend takes alpha = 0, which leaves T, S and every sum
            // unchanged.
            // This lane's sums over its pixels: M = sum dpow, My = sum dpow dy,
            // Myy = sum dpow dy^2 (the lane's pixels share one column, so the
            // dx moments follow from these: Mx = dx M, Mxx = dx^2 M, Mxy =
            // dx My) and the colour sums r, g, b.
            float dy[PPT], pw[PPT];
            bool pass[PPT];
            uint32_t rows = 0u;                           // bit k: some lane passes at pixel k
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const bool walk = rel < nc[k];
                if constexpr (COUNT) walked += walk;
                dy[k] = __fsub_rn(ps.fy[k], xyc.y);
                pw[k] = power2(q, dt, dy[k]);
                pass[k] = walk && in_cut(pw[k], xyc.z);
                rows |= __any_sync(0xffffffffu, pass[k]) ? 1u << k : 0u;
            }
            if (rows == 0u) continue;
            const float4 rgb = s_rgb[i];
            float M = 0.f, My = 0.f, Myy = 0.f, cr = 0.f, cg = 0.f, cb = 0.f;
            bool any = false;
            auto pixel = [&](auto kc) {
                constexpr int k = decltype(kc)::value;
                const float oG = q.w * ex2(pw[k]);
                const float alpha = fminf(bp.alpha_max, oG);
                const bool bl = pass[k] && alpha >= bp.alpha_min;
                const float a = bl ? alpha : 0.f;
                const float Tj = __fdividef(T[k], 1.f - a);
                const float w = a * Tj;
                cr = fmaf(w, dC0[k], cr);
                cg = fmaf(w, dC1[k], cg);
                cb = fmaf(w, dC2[k], cb);
                const float e = fmaf(rgb.x, dC0[k], fmaf(rgb.y, dC1[k], fmaf(rgb.z, dC2[k], -S[k])));
                S[k] = fmaf(a, e, S[k]);
                T[k] = bl ? Tj : T[k];
                const float dpow = oG < bp.alpha_max ? w * e : 0.f;   // alpha dL/dalpha (alpha unclamped; w = 0 unless blended)
                const float dpy = dpow * dy[k];
                M += dpow;
                My += dpy;
                Myy = fmaf(dpy, dy[k], Myy);
                any = any || bl;
                if constexpr (COUNT) evals += bl;
            };
            if constexpr (PPT == 1) {
                pixel(PixelK<0>{});
            } else if constexpr (PPT == 2) {
                if (rows == 3u) {                             // both: the two pixels interleave
                    pixel(PixelK<0>{});
                    pixel(PixelK<1>{});
                } else if (rows == 1u) {
                    pixel(PixelK<0>{});
                } else {
                    pixel(PixelK<1>{});
                }
            } else {
                if (rows & 1u) pixel(PixelK<0>{});
                if (rows & 2u) pixel(PixelK<1>{});
                if (rows & 4u) pixel(PixelK<2>{});
                if (rows & 8u) pixel(PixelK<3>{});
            }
            const uint32_t ballot = __ballot_sync(0xffffffffu, any);
            if (ballot == 0u) continue;
            const int64_t idx = vbase + __float_as_uint(s_rgb[i].w);
            const int contributing = __popc(ballot);
            if constexpr (PPT == 4) {
                // fold the upper half-warp onto the lower one when it pays
                // (lanes l and l + 16 share a column, so the compact sums
                // add), then every contributing lane adds its own sums
                if (contributing > FOLD_ABOVE) {
                    M += __shfl_down_sync(0xffffffffu, M, 16);
                    My += __shfl_down_sync(0xffffffffu, My, 16);
                    Myy += __shfl_down_sync(0xffffffffu, Myy, 16);
                    cr += __shfl_down_sync(0xffffffffu, cr, 16);
                    cg += __shfl_down_sync(0xffffffffu, cg, 16);
                    cb += __shfl_down_sync(0xffffffffu, cb, 16);
                    any = lane < 16 && ((ballot >> lane) & 0x10001u) != 0u;
                }
                if (any) {
                    const float Mx = dx * M;
                    const float vv[8] = {M, Mx, My, dx * Mx, dx * My, Myy, cr, cg};
                    add_sums(gv, idx, vv, cb);
                }
            } else {
                const float Mx = dx * M;
                const float vv[9] = {M, Mx, My, dx * Mx, dx * My, Myy, cr, cg, cb};
                if (contributing <= DIRECT_UP_TO) {
                    if (any) add_sums(gv, idx, vv, cb);
                    continue;
                }
                flush_one(gv, idx, vv, lane);
            }
        }
        n = 0;
        __syncwarp();
    }
    // blended (pixel, Gaussian) pairs and walked (pixel, position) pairs
    if constexpr (COUNT) {
        unsigned long long e = evals, wk = walked;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            wk += __shfl_xor_sync(0xffffffffu, wk, o);
        }
        if (lane == 0) {
            if (e) atomicAdd(&status->counters[2], e);
            if (wk) atomicAdd(&status->counters[4], wk);
        }
    }
    add_cost(cost, tile_id, t0, lane);
}

template <int TILE, int CH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE *TILE / PPT, (PPT == 2 ? 8 : 1)) k_blend_bwd(ViewBatch vb, ProjView p, const uint32_t *vals,
                                                                const uint2 *ranges, BlendParams bp, GradView gv,
                                                                DevStatus *status, const uint32_t *order,
                                                                uint32_t *cost)
{
    const uint32_t tile_id = order ? order[blockIdx.x] : blockIdx.x;   // launch order (launch_tile_order)
    blend_bwd_tile<TILE, CH, PPT, COUNT>(tile_id, vb, p, vals, ranges, bp, gv, status, cost);
}

template <int TILE, int CH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE *TILE / PPT, (PPT == 2 ? 8 : 1))
    k_blend_bwd_ranges(ViewBatch vb, ProjView p, const uint32_t *vals, const uint2 *ranges, BlendParams bp,
                       GradView gv, DevStatus *status, const uint32_t *div, uint32_t *cost)
{
    const uint32_t lo = div[blockIdx.x];
    const uint32_t hi = blockIdx.x + 1 < gridDim.x ? min(div[blockIdx.x + 1], vb.total_tiles) : vb.total_tiles;
    for (uint32_t t = lo; t < hi; ++t)
        blend_bwd_tile<TILE, CH, PPT, COUNT>(t, vb, p, vals, ranges, bp, gv, status, cost);
}

template <int TILE, int CH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TILE *TILE / PPT, (PPT == 2 ? 8 : 1))
    k_blend_bwd_pool(ViewBatch vb, ProjView p, const uint32_t *vals, const uint2 *ranges, BlendParams bp,
                     GradView gv, DevStatus *status, const uint32_t *order, uint32_t *queue, uint32_t *cost)
{
    for (uint32_t t = pool_next(queue); t < vb.total_tiles; t = pool_next(queue))
        blend_bwd_tile<TILE, CH, PPT, COUNT>(order ? order[t] : t, vb, p, vals, ranges, bp, gv, status, cost);
}

// Launch order of the tiles, heaviest list first.  With few waves of CTAs
// per launch the kernel ends when its slowest tiles do, and in index order the
// long lists of a dense region can start last.  A counting sort on
// floor(log2(list length)) puts the longest lists first; within a length
// class the order is that of the atomic scatter (results do not depend on the
// launch order: tiles are independent).  buckets: 64 words, [0, 32) counts
// of each class, [32, 64) their write cursors.
// With `cost` (the measured cost of each tile) the classes are
// floor(log2(cost)) instead.
__device__ __forceinline__ uint32_t length_class(const uint2 *ranges, const uint32_t *cost, uint32_t t)
{
    uint32_t len;
    if (cost) {
        len = cost[t];
    } else {
        const uint2 r = ranges[t];
        len = r.y > r.x ? r.y - r.x : 0u;
    }
    return len ? (uint32_t)__clz(len) : 31u;   // 31 - floor(log2 len): the longest lists in class 0
}

__global__ void __launch_bounds__(256) k_order_count(const uint2 *ranges, const uint32_t *cost, uint32_t n,
                                                     uint32_t *buckets)
{
    __shared__ uint32_t h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        atomicAdd(&h[length_class(ranges, cost, t)], 1u);
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&buckets[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_order_offsets(uint32_t *buckets)
{
    const int lane = threadIdx.x;               // one warp: exclusive prefix of the 32 counts
    const uint32_t c = buckets[lane];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    buckets[32 + lane] = incl - c;
}

__global__ void __launch_bounds__(256) k_order_scatter(const uint2 *ranges, const uint32_t *cost, uint32_t n,
                                                       uint32_t *buckets, uint32_t *order)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint32_t pos = atomicAdd(&buckets[32 + length_class(ranges, cost, t)], 1u);
        if (pos < n) order[pos] = t;           // the counts add up to n: always true
    }
}

// Kernels needing more than 48 KB of dynamic shared memory opt in once.
template <class K>
bool smem_opt_in(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

// Schedule of a blending launch: one CTA per tile in `order` (null: index
// order); with div, Algorithm 1's ranges for `ctas` persistent CTAs; with
// queue, `ctas` persistent CTAs pulling tiles of `order` from the queue
// counter (zero at launch).  cost (optional) receives each tile's measured
// cost.
struct Sched {
    const uint32_t *order;
    const uint32_t *div;
    uint32_t ctas;
    uint32_t *cost;
    uint32_t *queue;
};

template <int TILE, int CH, int PPT, bool COUNT>
void fwd_launch_counting(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                const BlendParams &bp, DevStatus *status, const Sched &sc, cudaStream_t st)
{
    constexpr size_t sm = smem_bytes<TILE, CH, PPT>();
    static const bool ok = smem_opt_in(k_blend_fwd<TILE, CH, PPT, COUNT>, sm) &&
                           smem_opt_in(k_blend_fwd_ranges<TILE, CH, PPT, COUNT>, sm) &&
                           smem_opt_in(k_blend_fwd_pool<TILE, CH, PPT, COUNT>, sm);
    (void)ok;
    if (sc.queue)
        k_blend_fwd_pool<TILE, CH, PPT, COUNT><<<sc.ctas, TILE * TILE / PPT, sm, st>>>(vb, p, vals, ranges, bp, status,
                                                                              sc.order, sc.queue, sc.cost);
    else if (sc.div)
        k_blend_fwd_ranges<TILE, CH, PPT, COUNT><<<sc.ctas, TILE * TILE / PPT, sm, st>>>(vb, p, vals, ranges, bp, status,
                                                                                sc.div, sc.cost);
    else
        k_blend_fwd<TILE, CH, PPT, COUNT><<<vb.total_tiles, TILE * TILE / PPT, sm, st>>>(vb, p, vals, ranges, bp, status,
                                                                                 sc.order, sc.cost);
}

// The forward's counts (evaluations until termination, list positions below
// n_contrib) are taken only when asked (bp.count_work), like the backward's.
template <int TILE, int CH, int PPT>
void fwd_launch(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                const BlendParams &bp, DevStatus *status, const Sched &sc, cudaStream_t st)
{
    if (bp.count_work)
        fwd_launch_counting<TILE, CH, PPT, true>(vb, p, vals, ranges, bp, status, sc, st);
    else
        fwd_launch_counting<TILE, CH, PPT, false>(vb, p, vals, ranges, bp, status, sc, st);
}

template <int TILE, int CH, int PPT, bool COUNT>
void bwd_launch_counting(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                         const BlendParams &bp, const GradView &g, DevStatus *status, const Sched &sc, cudaStream_t st)
{
    constexpr size_t sm = smem_bytes<TILE, CH, PPT>();
    static const bool ok = smem_opt_in(k_blend_bwd<TILE, CH, PPT, COUNT>, sm) &&
                           smem_opt_in(k_blend_bwd_ranges<TILE, CH, PPT, COUNT>, sm) &&
                           smem_opt_in(k_blend_bwd_pool<TILE, CH, PPT, COUNT>, sm);
    (void)ok;
    if (sc.queue)
        k_blend_bwd_pool<TILE, CH, PPT, COUNT><<<sc.ctas, TILE * TILE / PPT, sm, st>>>(
            vb, p, vals, ranges, bp, g, status, sc.order, sc.queue, sc.cost);
    else if (sc.div)
        k_blend_bwd_ranges<TILE, CH, PPT, COUNT><<<sc.ctas, TILE * TILE / PPT, sm, st>>>(
            vb, p, vals, ranges, bp, g, status, sc.div, sc.cost);
    else
        k_blend_bwd<TILE, CH, PPT, COUNT><<<vb.total_tiles, TILE * TILE / PPT, sm, st>>>(
            vb, p, vals, ranges, bp, g, status, sc.order, sc.cost);
}

// The walked and blended pairs are counted only when asked (bp.count_work):
// the two counts cost about 3% of the backward's issued instructions.
template <int TILE, int CH, int PPT>
void bwd_launch(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                const BlendParams &bp, const GradView &g, DevStatus *status, const Sched &sc, cudaStream_t st)
{
    if (bp.count_work)
        bwd_launch_counting<TILE, CH, PPT, true>(vb, p, vals, ranges, bp, g, status, sc, st);
    else
        bwd_launch_counting<TILE, CH, PPT, false>(vb, p, vals, ranges, bp, g, status, sc, st);
}

template <class K>
cudaError_t occupancy(int *per_sm, K kernel, int threads, size_t sm)
{
    smem_opt_in(kernel, sm);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, sm);
}

// Resident CTAs of the range kernel (POOL: of the pool kernel) on the whole
// device.
template <int TILE, int CH, int PPT, bool BWD, bool POOL = false>
uint32_t resident_ctas()
{
    static uint32_t n = 0;
    if (!n) {
        constexpr size_t sm = smem_bytes<TILE, CH, PPT>();
        constexpr int threads = TILE * TILE / PPT;
        int per_sm = 0;
        cudaError_t e;
        if (BWD)
            e = POOL ? occupancy(&per_sm, k_blend_bwd_pool<TILE, CH, PPT, false>, threads, sm)
                     : occupancy(&per_sm, k_blend_bwd_ranges<TILE, CH, PPT, false>, threads, sm);
        else
            e = POOL ? occupancy(&per_sm, k_blend_fwd_pool<TILE, CH, PPT, false>, threads, sm)
                     : occupancy(&per_sm, k_blend_fwd_ranges<TILE, CH, PPT, false>, threads, sm);
        if (e != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        n = (uint32_t)per_sm * (uint32_t)sm_count();
    }
    return n;
}

// Algorithm 1 (division points), with the tiles as the pixel blocks and the
// persistent CTAs as the GPUs: CT = cumsum(cost) (inclusive), ET = CT[T - 1]
// / P, thresholds k ET for k = 0 .. P - 1, div[k] = searchsorted(CT, k ET)
// (the first tile whose cumulative cost reaches the threshold) = the first
// tile of range k; range k is [div[k], div[k + 1]) and the last ends at T.
// The comparison CT[i] >= k CT[T - 1] / P is evaluated exactly as
// P CT[i] >= k CT[T - 1] in 64-bit integers.  excl: the exclusive prefix
// sums (CT = excl + cost).
__global__ void k_division_points(const uint32_t *excl, const uint32_t *cost, uint32_t T, uint32_t P,
                                  const unsigned long long *total, uint32_t *div)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const unsigned long long thr = *total * (unsigned long long)k;
    uint32_t lo = 0, hi = T;                       // first i with P CT[i] >= k total
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const unsigned long long ct = (unsigned long long)excl[mid] + cost[mid];
        if (ct * P >= thr) hi = mid; else lo = mid + 1;
    }
    div[k] = lo;
}

// cost[t] = min(cost[t], cap): with cap = (2^32 - 1) / T the 32-bit prefix
// sums cannot wrap, so the division points stay monotone and the ranges
// cover every tile exactly once.
__global__ void k_clamp_cost(uint32_t *cost, uint32_t T, uint32_t cap)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        cost[t] = min(cost[t], cap);
}

// cost[t] = the tile's list length + 1 (the cost model before any step has
// been measured).
__global__ void k_list_cost(const uint2 *ranges, uint32_t T, uint32_t *cost)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const uint2 r = ranges[t];
        cost[t] = (r.y > r.x ? r.y - r.x : 0u) + 1u;
    }
}

}  // namespace

// Built (tile, entries per warp refill, pixels per thread) combinations.
// One pixel per thread (warp = 8 x 4 pixels): tile 8 or 16 with 32, 64 or
// 128 entries; tile 32 with 32 or 64 (its 32 warps' slices must fit in shared
// memory).  Two (warp = 8 x 8): any tile with 32, 64 or 128.  Four (8 x 16):
// tile 16 or 32 with 32, 64 or 128.
bool blend_config_ok(int tile, int chunk, int ppt)
{
    if (chunk != 32 && chunk != 64 && chunk != 128) return false;
    if (ppt == 1) return tile == 8 || tile == 16 || (tile == 32 && chunk <= 64);
    if (ppt == 2) return true;
    if (ppt == 4) return tile == 16 || tile == 32;
    return false;
}

#define GS_BLEND_CASES(X)                                                                                      \
    X(8, 32, 1) X(8, 64, 1) X(8, 128, 1) X(16, 32, 1) X(16, 64, 1) X(16, 128, 1) X(32, 32, 1) X(32, 64, 1)   \
    X(8, 32, 2) X(8, 64, 2) X(8, 128, 2) X(16, 32, 2) X(16, 64, 2) X(16, 128, 2) X(32, 32, 2) X(32, 64, 2) X(32, 128, 2) X(16, 32, 4) X(16, 64, 4)   \
    X(16, 128, 4) X(32, 32, 4) X(32, 64, 4) X(32, 128, 4)

void launch_blend_fwd(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                      const BlendParams &bp, int chunk, int ppt, DevStatus *status, const uint32_t *order,
                      cudaStream_t st, const uint32_t *div, uint32_t *cost, uint32_t *queue)
{
    if (vb.total_tiles == 0) return;
    Sched sc{order, queue ? nullptr : div, 0u, cost, queue};
    switch (vb.tile * 10000 + chunk * 10 + ppt) {
#define GS_FWD_CASE(T, C, P) \
    case T * 10000 + C * 10 + P: \
        sc.ctas = queue ? resident_ctas<T, C, P, false, true>() : div ? resident_ctas<T, C, P, false>() : 0u; \
        fwd_launch<T, C, P>(vb, p, vals, ranges, bp, status, sc, st); break;
        GS_BLEND_CASES(GS_FWD_CASE)
#undef GS_FWD_CASE
    default: sc.div = nullptr; sc.queue = nullptr; fwd_launch<16, 64, 1>(vb, p, vals, ranges, bp, status, sc, st); break;
    }
    count_launches(1);
}

void launch_blend_bwd(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                      const BlendParams &bp, int chunk, int ppt, const GradView &g, DevStatus *status,
                      const uint32_t *order, cudaStream_t st, const uint32_t *div, uint32_t *cost, uint32_t *queue)
{
    if (vb.total_tiles == 0) return;
    Sched sc{order, queue ? nullptr : div, 0u, cost, queue};
    switch (vb.tile * 10000 + chunk * 10 + ppt) {
#define GS_BWD_CASE(T, C, P) \
    case T * 10000 + C * 10 + P: \
        sc.ctas = queue ? resident_ctas<T, C, P, true, true>() : div ? resident_ctas<T, C, P, true>() : 0u; \
        bwd_launch<T, C, P>(vb, p, vals, ranges, bp, g, status, sc, st); break;
        GS_BLEND_CASES(GS_BWD_CASE)
#undef GS_BWD_CASE
    default: sc.div = nullptr; sc.queue = nullptr; bwd_launch<16, 64, 1>(vb, p, vals, ranges, bp, g, status, sc, st); break;
    }
    count_launches(1);
}

uint32_t blend_resident_ctas(int tile, int chunk, int ppt, bool bwd)
{
    switch (tile * 10000 + chunk * 10 + ppt) {
#define GS_RES_CASE(T, C, P) \
    case T * 10000 + C * 10 + P: return bwd ? resident_ctas<T, C, P, true>() : resident_ctas<T, C, P, false>();
        GS_BLEND_CASES(GS_RES_CASE)
#undef GS_RES_CASE
    default: return 0u;
    }
}

void launch_division_points(uint32_t *cost, uint32_t T, uint32_t P, uint32_t *excl, void *scan_tmp,
                            unsigned long long *total, uint32_t *div, cudaStream_t st)
{
    if (T == 0 || P == 0) return;
    const unsigned blocks = (T + 255) / 256 < 4096u ? (T + 255) / 256 : 4096u;
    k_clamp_cost<<<blocks, 256, 0, st>>>(cost, T, 0xffffffffu / T);
    count_launches(1);
    launch_exclusive_scan(cost, excl, T, total, scan_tmp, st);
    k_division_points<<<(P + 255) / 256, 256, 0, st>>>(excl, cost, T, P, total, div);
    count_launches(1);
}

void launch_list_cost(const uint2 *ranges, uint32_t T, uint32_t *cost, cudaStream_t st)
{
    if (T == 0) return;
    const unsigned blocks = (T + 255) / 256 < 4096u ? (T + 255) / 256 : 4096u;
    k_list_cost<<<blocks, 256, 0, st>>>(ranges, T, cost);
    count_launches(1);
}

int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    }
    return sms;
}

bool tile_order_pays(uint32_t total_tiles)
{
    // measured on GB300: 1M Gaussians at 1080p (8,160 tiles, 54 per SM) gains
    // 13 % per training step, 16 views at 1080p (130,560 tiles, 859 per SM)
    // 1.1 % with the per-row-vote blending kernels (the long lists of a dense
    // region no longer start last), and 256 tiles lose to the ordering's own
    // launches; above 2,000 tiles per SM nothing was measured
    const uint32_t sms = (uint32_t)sm_count();
    return total_tiles >= 4u * sms && total_tiles <= 2000u * sms;
}

void launch_tile_order(const uint2 *ranges, uint32_t n, uint32_t *order, uint32_t *buckets, cudaStream_t st,
                       const uint32_t *cost)
{
    if (n == 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 2u * (uint32_t)sm_count() ? (n + 255) / 256
                                                                                   : 2u * (uint32_t)sm_count());
    cudaMemsetAsync(buckets, 0, 32 * sizeof(uint32_t), st);
    k_order_count<<<blocks, 256, 0, st>>>(ranges, cost, n, buckets);
    k_order_offsets<<<1, 32, 0, st>>>(buckets);
    k_order_scatter<<<blocks, 256, 0, st>>>(ranges, cost, n, buckets, order);
    count_launches(3);
}

}  // namespace gs
