// Internal declarations shared by the libgs translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int MAXV = GS_MAX_VIEWS;

// Per-view state passed by value in kernel parameters (no device copy of the
// camera array is needed, and CUDA-graph capture records it with the launch).
struct ViewCam {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_z;
    float limx, limy;      // 1.3 * tan(fov/2): off-axis clamp of x/z and y/z
    float C[3];            // camera centre in world space
    int32_t W, H, TX, TY;  // image and tile-grid size
    uint32_t tile_base;    // first global tile id of this view
    uint32_t pix_base;     // unused for per-view pointers; kept for packed layouts
    float *img;            // [3][H][W]
    float *T_final;        // [H][W]
    uint32_t *n_contrib;   // [H][W]
    const float *d_img;    // [3][H][W]
};

struct ViewBatch {
    int32_t B;
    int32_t tile;
    int32_t log2_tile;
    uint32_t total_tiles;
    ViewCam v[MAXV];
};

struct BlendParams {
    float alpha_min, alpha_max, T_min;
    float bg[3];
    uint32_t list_cap;   // entries in the fragment list: a tile range beyond it is refused
    int32_t count_work;  // nonzero: the blending kernels count their work (counters[1], [2], [4], [5])
};

struct SceneView {     // read-only parameter planes
    const float4 *mo, *ls, *q, *sh;
    int64_t N;
    int32_t deg;
};

struct SceneMut {
    float4 *mo, *ls, *q, *sh;
    int64_t N;
};

struct ProjView {
    float2 *xy;
    float4 *conic_o;
    float4 *rgb_d;
    int32_t *radius;
    int64_t N;
};

// Gradients per (view, Gaussian) entry: three separate float4 arrays (the
// three atomics of an entry then go to different L2 slices).  The blending
// backward accumulates, over the pixels where the Gaussian blends with alpha
// below alpha_max, the moments of dpow = alpha dL/dalpha at offset
// (dx, dy) = pixel - centre:
//   d_xy_o = (M, Mx, My) = sum (dpow, dpow dx, dpow dy),
//   d_conic = (Mxx, Mxy, Myy) = sum (dpow dx^2, dpow dx dy, dpow dy^2),
// and d_rgb = sum T alpha dL/dC (the colour gradient itself);
// moments_to_grads turns the first two into gradients.
struct GradView {
    float4 *d_xy_o, *d_conic, *d_rgb;
};

// From the moments to dL/d(u, v, opacity) and dL/d(a, b, c) of one entry with
// conic_o = (a, b, c, o).  With power = -(a dx^2 + 2 b dx dy + c dy^2) / 2,
// dx = px - u and alpha = o exp(power): d alpha / d power = alpha, so
// dL/du = sum dpow (a dx + b dy), dL/dv = sum dpow (b dx + c dy),
// dL/dopacity = sum dL/dalpha G = M / o, dL/da = -Mxx / 2, dL/db = -Mxy,
// dL/dc = -Myy / 2.
__host__ __device__ __forceinline__ void moments_to_grads(const float4 &co, const float4 &m_xy,
                                                          const float4 &m_cn, float4 &g_xy_o, float4 &g_conic)
{
    g_xy_o = make_float4(co.x * m_xy.y + co.y * m_xy.z, co.y * m_xy.y + co.z * m_xy.z,
                         co.w > 0.f ? m_xy.x / co.w : 0.f, 0.f);
    g_conic = make_float4(-0.5f * m_cn.x, -m_cn.y, -0.5f * m_cn.z, 0.f);
}

// Device status word layout (one per context).
struct DevStatus {
    int32_t code;          // first gs_status error, 0 = OK
    int32_t pad;
    unsigned long long needed;  // fragments requested by the last binning
    // F, forward (pixel, fragment) evaluations, backward blended pairs,
    // Gaussians culled as non-finite, backward walked (pixel, position) pairs,
    // forward sum of n_contrib over the pixels
    unsigned long long counters[6];
};

// Process-wide count of kernel launches (incremented by every launcher).
void count_launches(int n);

// Launchers (all asynchronous on `st`).
// ntiles[i]: tiles covered by pair i; rect[i] (optional): its packed tile
// rectangle (pack_rect, the same arithmetic as the binning's).
// rm (optional, with rect): also cull each pair's rectangle against the
// alpha >= cull_alpha ellipse (row_interval_mask, rectangles of at most
// TILE_CULL_MAX_AREA tiles): rm[i] = (rectangle words, kept-tile bits low,
// high) for every pair with tiles, and ntiles[i] = the kept count.
void launch_preprocess_fwd(const SceneView &s, const ViewBatch &vb, const ProjView &p, uint32_t *ntiles,
                           uint2 *rect, DevStatus *status, int strict, cudaStream_t st, uint4 *rm = nullptr,
                           float cull_alpha = 0.f);
// g holds the blending backward's moments (GradView) unless grads_ready.
// vis (optional): vis[g] = 1 if some view has the Gaussian's radius > 0,
// else 0; with vis the rows of unseen Gaussians are not written.
// dacc / dcnt (optional, densification statistics): for each view in which
// the Gaussian is visible, |dL_v/d(u, v)| is added to dacc[g] and 1 to dcnt[g],
// unless status holds GS_ERR_CAPACITY or GS_ERR_TIMEOUT (status is read only
// with dacc).
// scale (negative: 1/B, the batch mean) multiplies the sum over the views.
void launch_preprocess_bwd(const SceneView &s, const ViewBatch &vb, const ProjView &p, const GradView &g,
                           bool grads_ready, const SceneMut &out, uint8_t *vis, cudaStream_t st,
                           float *dacc = nullptr, uint32_t *dcnt = nullptr, const DevStatus *status = nullptr,
                           float scale = -1.f);
// In place: the moments of n entries -> gradients (moments_to_grads).
void launch_moments_to_grads(const ProjView &p, int64_t n, const GradView &g, cudaStream_t st);

// Exclusive scan of n uint32 values (n < 2^31); total (uint64) to *total.
// n_dev (optional): a device count that caps n (items past it are neither
// read nor written); nonzero: scan (value != 0) instead of the value.
size_t scan_temp_bytes(int64_t n);
void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *total, void *temp,
                           cudaStream_t st, const uint32_t *n_dev = nullptr, bool nonzero = false);

// Can alpha = o exp(-f/2), f(d) = a dx^2 + 2 b dx dy + c dy^2 (d = pixel -
// (u, v)), reach alpha_min anywhere in the pixel-centre box [x0, x1] x
// [y0, y1]?  f is convex with its minimum 0 at the centre, so for a centre
// outside the box the minimum lies on an edge that faces it (x = clamp(u) or
// y = clamp(v)); along such an edge f is a parabola, minimised at the clamp
// of its vertex and evaluated as c (dy - dy*)^2 + (det / c) dx^2 (non-negative
// terms, no cancellation; det by Kahan's form).  The acceptance bound
// L = 2 ln(o / alpha_min) is widened by 0.1 %, 1e-6 x a bound on the conic's
// condition number and 1e-4 -- beyond the rounding of the per-pixel exponent and of the
// approximate reciprocals here -- so the test never drops a Gaussian the
// per-pixel test would blend.  A non-positive-definite conic is kept.  Every
// operation is explicitly rounded.
// The per-Gaussian part of the test: (threshold, 1/a, 1/c, det);
// threshold -1: alpha never reaches alpha_min; +inf: not positive definite.
__device__ __forceinline__ float4 ellipse_terms(const float4 &co, float alpha_min)
{
    if (!(co.w > alpha_min)) return make_float4(-1.f, 0.f, 0.f, 0.f);
    const float a = co.x, b = co.y, c = co.z;
    const float bb = __fmul_rn(b, b);
    const float det = __fadd_rn(__fmaf_rn(a, c, -bb), __fmaf_rn(-b, b, bb));
    if (!(det > 0.f && a > 0.f && c > 0.f)) return make_float4(INFINITY, 0.f, 0.f, 0.f);
    const float L = __fmul_rn(2.f, __logf(__fdividef(co.w, alpha_min)));
    // (a + c)^2 / det = 4 tr^2 / (tr^2 - r^2) >= (tr + r) / (tr - r), the
    // condition number (eigenvalues tr +- r): a bound without the square root
    const float apc = __fadd_rn(a, c);
    const float kappa = __fdividef(__fmul_rn(apc, apc), det);
    return make_float4(__fmaf_rn(L, __fmaf_rn(1e-6f, kappa, 1.001f), 1e-4f), __fdividef(1.f, a),
                       __fdividef(1.f, c), det);
}

// The per-box part, with t = ellipse_terms(co) and (a, b, c) = co.xyz.
__device__ __forceinline__ bool ellipse_terms_box_hits(const float4 &t, float a, float b, float c, float u, float v,
                                                       float x0, float x1, float y0, float y1)
{
    if (!(t.x >= 0.f)) return false;                       // never reaches alpha_min
    if (t.x == INFINITY) return true;                      // not positive definite: keep
    const float ex = fminf(fmaxf(u, x0), x1), ey = fminf(fmaxf(v, y0), y1);
    if (ex == u && ey == v) return true;                   // centre inside the box
    float fmin = INFINITY;
    if (ex != u) {                                         // edge x = ex
        const float dx = __fsub_rn(ex, u);
        const float dys = __fmul_rn(__fmul_rn(-b, dx), t.z);
        const float s = __fsub_rn(fminf(fmaxf(dys, __fsub_rn(y0, v)), __fsub_rn(y1, v)), dys);
        fmin = __fmaf_rn(__fmul_rn(c, s), s, __fmul_rn(__fmul_rn(t.w, t.z), __fmul_rn(dx, dx)));
    }
    if (ey != v) {                                         // edge y = ey
        const float dy = __fsub_rn(ey, v);
        const float dxs = __fmul_rn(__fmul_rn(-b, dy), t.y);
        const float s = __fsub_rn(fminf(fmaxf(dxs, __fsub_rn(x0, u)), __fsub_rn(x1, u)), dxs);
        fmin = fminf(fmin, __fmaf_rn(__fmul_rn(a, s), s, __fmul_rn(__fmul_rn(t.w, t.y), __fmul_rn(dy, dy))));
    }
    return fmin <= t.x;
}

__device__ __forceinline__ bool ellipse_box_hits(const float4 &co, float u, float v, float alpha_min, float x0,
                                                 float x1, float y0, float y1)
{
    return ellipse_terms_box_hits(ellipse_terms(co, alpha_min), co.x, co.y, co.z, u, v, x0, x1, y0, y1);
}

// Footprint rectangles of at most this many tiles are culled tile by tile
// against the alpha ellipse in a training step (one bit per tile of the
// rectangle); larger ones keep every tile.
constexpr uint32_t TILE_CULL_MAX_AREA = 64;

// sqrt(x) for x >= 0 from the approximate reciprocal square root (0 at 0).
__device__ __forceinline__ float sqrt_approx(float x)
{
    return x > 0.f ? x * rsqrtf(x) : 0.f;
}

// Tiles of a footprint rectangle culled against the alpha >= cull_alpha
// ellipse (the transformation kernel does it per pair in a training step or
// a render).  With f(d) = a dx^2 + 2 b dx dy + c dy^2 the ellipse is f <= L
// (L = the widened threshold of ellipse_terms).  Per tile row, the
// pixel-centre rows of the row give a band dy in [dy0, dy1]; the ellipse
// meets the band where |dy| <= Y = sqrt(a L / det), and there its x-range is
// the interval between
//   xl(dy) = (-b dy - sqrt(a L - det dy^2)) / a  and
//   xr(dy) = (-b dy + sqrt(a L - det dy^2)) / a.
// xr is concave in dy with its maximum at dy_r = -b sqrt(L / (c det)) (the
// ellipse's rightmost point) and xl convex with its minimum at -dy_r, so the
// band's x-range is [xl(clamp(-dy_r)), xr(clamp(dy_r))], each clamped into the
// band.  A tile of the row is kept when its pixel-centre columns meet that
// range.  This is the box test of ellipse_box_hits done once per tile row
// instead of once per tile; the band limits, the range and Y are widened by
// 1e-3 relative plus 1e-2 pixel, above the rounding of the approximate square
// roots and reciprocals (the threshold L already carries ellipse_terms'
// margin), so a tile is never dropped where the per-pixel test could blend.
// Returns the kept-tile bits (row-major in the rectangle [x0, x1] x [y0, y1]
// of tiles of edge T; at most TILE_CULL_MAX_AREA tiles).
__device__ __forceinline__ uint64_t row_interval_mask(const float4 &co, const float4 &te, float u, float v,
                                                      uint32_t x0, uint32_t x1, uint32_t y0, uint32_t y1, float T)
{
    if (!(te.x >= 0.f)) return 0ull;                     // alpha never reaches the cut
    const uint32_t w = x1 - x0 + 1u;
    const uint32_t ra = w * (y1 - y0 + 1u);
    const uint64_t all = ra >= 64u ? ~0ull : ((1ull << ra) - 1ull);
    if (te.x == INFINITY) return all;                     // not positive definite: keep every tile
    const float a = co.x, b = co.y, L = te.x, det = te.w;
    constexpr float REL = 1e-3f, ABS = 1e-2f;
    const float aL = a * L;
    const float Y = sqrt_approx(__fdividef(aL, det)) * (1.f + REL) + ABS;   // |dy| reach of the ellipse
    const float dyr = -b * sqrt_approx(L * te.z / det);                       // dy of the rightmost point (te.z = 1/c)
    const float ia = te.y;                                                     // 1/a
    const float iT = 1.f / T;                                                  // exact: T is a power of two
    uint64_t mask = 0ull;
    for (uint32_t ty = y0; ty <= y1; ++ty) {
        const float py0 = (float)ty * T + 0.5f - v;               // the row's pixel-centre dy range
        const float lo = fmaxf(py0 - ABS, -Y), hi = fminf(py0 + (T - 1.f) + ABS, Y);
        if (!(lo <= hi)) continue;
        const float dr = fminf(fmaxf(dyr, lo), hi), dl = fminf(fmaxf(-dyr, lo), hi);
        const float sr = sqrt_approx(aL - det * dr * dr), sl = sqrt_approx(aL - det * dl * dl);
        float xr = (sr - b * dr) * ia, xl = -(sl + b * dl) * ia;
        const float m = (xr - xl) * REL + ABS;
        xr = u + xr + m;
        xl = u + xl - m;
        // tiles whose pixel-centre columns [tx T + 0.5, tx T + T - 0.5] meet [xl, xr]
        const float fl = ceilf((xl - (T - 0.5f)) * iT), fh = floorf((xr - 0.5f) * iT);
        const int tl = (int)fmaxf(fl, (float)x0), th = (int)fminf(fh, (float)x1);
        if (tl > th) continue;
        const uint32_t s = (ty - y0) * w + ((uint32_t)tl - x0), len = (uint32_t)(th - tl) + 1u;
        mask |= (~0ull >> (64u - len)) << s;
    }
    return mask & all;
}

// A footprint's tile rectangle packed as {x0 | x1 << 16, y0 | y1 << 16}
// (tile coordinates fit 16 bits); (1, 0) is the empty rectangle.
__host__ __device__ __forceinline__ uint2 pack_rect(uint32_t x0, uint32_t x1, uint32_t y0, uint32_t y1)
{
    return make_uint2(x0 | (x1 << 16), y0 | (y1 << 16));
}

// Binning in depth order: (1) per (view, Gaussian) pair its tile rectangle;
// the visible pairs (those covering a tile) compacted in index order and
// sorted stably by depth (four passes of 8-bit digits over an order-preserving
// integer image of the float32 depth); (2) tile counts
// gathered in that order and scanned; (3) fragments emitted pair by pair in
// that order, key = global tile id, value = Gaussian index; (4) a stable sort
// on the tile id.  Within a tile the fragments then follow (depth, Gaussian
// index).
//
// launch_depth_order: rect[i] and area[i] (tile count) for every pair, from
// gs_proj unless rect_ready (the transformation kernel wrote them); returns
// the buffer whose first *n_vis entries are the visible pair indices in depth
// order (keys, keys_alt, order_alt and pos are scratch of n entries each;
// *total also receives the visible count).
uint32_t *launch_depth_order(const ViewBatch &vb, const ProjView &p, bool rect_ready, uint2 *rect, uint32_t *area,
                             uint32_t *keys, uint32_t *order, uint32_t *keys_alt, uint32_t *order_alt,
                             uint32_t *pos, uint32_t *n_vis, unsigned long long *total, void *scan_tmp,
                             void *sort_tmp, DevStatus *status, cudaStream_t st);
// For pair order[j], j < *n_vis: rx / ry its rectangle words and counts its
// tile count; with rm (culled) also keep[j] = its kept-tile bits, else counts
// come from area[].
void launch_gather_counts(const uint32_t *order, const uint2 *rect, const uint32_t *area, const uint4 *rm, int64_t n,
                          const uint32_t *n_vis, uint32_t *counts, uint32_t *rx, uint32_t *ry, uint2 *keep,
                          cudaStream_t st);
// keep / cull_alpha: as given to launch_gather_counts.
void launch_emit_keys(const ViewBatch &vb, int64_t N, const uint32_t *n_vis, const uint32_t *order,
                      const uint32_t *rx, const uint32_t *ry, const uint2 *keep, const uint32_t *offsets,
                      uint32_t *keys, uint32_t *vals, uint64_t capacity, const unsigned long long *total,
                      DevStatus *status, uint32_t *count_out, float cull_alpha, cudaStream_t st);

// Sort scratch for the pair sort of `pairs` keys and the fragment sort of
// `fragments` keys (one buffer serves both, one after the other).
size_t sort_temp_bytes(uint64_t pairs, uint64_t fragments);
// Stable LSD radix sort of 32-bit tile ids (one-sweep passes).  The result
// lands in keys/vals when the number of passes is even, else in the alt
// buffers.  A look-back wait that exceeds its spin limit sets GS_ERR_TIMEOUT
// in *status.
int fragment_sort_passes(int tile_bits);
void launch_sort_fragments(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                           uint64_t capacity, const uint32_t *count, int tile_bits, void *temp, DevStatus *status,
                           cudaStream_t st);

// Storage order: perm = the Gaussians sorted stably by the Morton code of
// their positions (10 bits per axis over the finite positions' bounding box);
// temp holds spatial_order_temp_bytes(N).  launch_permute: dst[i] = src[perm[i]]
// for all 15 planes.
size_t spatial_order_temp_bytes(int64_t N);
void launch_spatial_order(const float4 *mo, int64_t N, uint32_t *perm, void *temp, DevStatus *status,
                          cudaStream_t st);
void launch_permute(const SceneView &src, const uint32_t *perm, const SceneMut &dst, cudaStream_t st);

// Densification (densify.cu).  Thresholds in the float32 domain the kernels
// compare in: grad_thr (pixels), log_scale_thr = log(scale threshold),
// logit_min = logit(min opacity), log_div = log(split divisor).
struct DensifyArgs {
    float grad_thr, log_scale_thr, logit_min, log_div;
};
// counts[g] = 0 (prune), 1 (keep) or 2 (clone or split).
void launch_densify_count(const SceneView &p, const float *acc, const uint32_t *cnt, const DensifyArgs &d,
                          uint32_t *counts, cudaStream_t st);
// Writes every output row at offsets[g] (the exclusive scan of counts),
// nothing when *total exceeds the outputs' N (their capacity).
void launch_densify_emit(const SceneView &p, const SceneView &m, const SceneView &v, const float *acc,
                         const uint32_t *cnt, const float *normals, const DensifyArgs &d, const uint32_t *offsets,
                         const unsigned long long *total, const SceneMut &po, const SceneMut &mo,
                         const SceneMut &vo, cudaStream_t st);
void launch_reset_opacity(const SceneMut &p, const SceneMut &m, const SceneMut &v, float logit_max, cudaStream_t st);

// Test hook (gs_debug_set_lookback): look-back spin limit (0 = default) and
// whether tile 0 of every sort pass withholds its look-back words.
void set_lookback_debug(uint32_t spin_limit, int withhold_first);

void launch_tile_ranges(const uint32_t *keys, const uint32_t *count, uint64_t capacity, uint2 *ranges,
                        uint32_t total_tiles, cudaStream_t st);
// keys[i] = tiles[i] << 32 | depth bits of fragment i (the public key format).
void launch_compose_keys(const ViewBatch &vb, int64_t N, const uint32_t *tiles, const uint32_t *vals,
                         const uint32_t *count, uint64_t capacity, const float4 *rgb_d, uint64_t *keys,
                         cudaStream_t st);

// chunk: list entries a warp gathers and filters per shared-memory refill;
// ppt: pixels per thread (blend_config_ok says which combinations are built).
bool blend_config_ok(int tile, int chunk, int ppt);
// div (optional): Algorithm 1's range starts for blend_resident_ctas(...)
// persistent CTAs (launch_division_points), used instead of one CTA per
// tile; queue (optional, wins over div): a zeroed counter from which
// persistent CTAs, one per resident slot, pull the tiles of `order` (null:
// index order); cost (optional): each tile's measured cost is added there.
void launch_blend_fwd(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                      const BlendParams &bp, int chunk, int ppt, DevStatus *status, const uint32_t *order,
                      cudaStream_t st, const uint32_t *div = nullptr, uint32_t *cost = nullptr,
                      uint32_t *queue = nullptr);
void launch_blend_bwd(const ViewBatch &vb, const ProjView &p, const uint32_t *vals, const uint2 *ranges,
                      const BlendParams &bp, int chunk, int ppt, const GradView &g, DevStatus *status,
                      const uint32_t *order, cudaStream_t st, const uint32_t *div = nullptr,
                      uint32_t *cost = nullptr, uint32_t *queue = nullptr);
uint32_t blend_resident_ctas(int tile, int chunk, int ppt, bool bwd);
int sm_count();
// Algorithm 1 over T tile costs for P ranges: div[k] = the first tile of
// range k (costs are first clamped to (2^32 - 1) / T in place; excl: T words
// of scratch; scan_tmp: scan_temp_bytes(T); total: one word).
void launch_division_points(uint32_t *cost, uint32_t T, uint32_t P, uint32_t *excl, void *scan_tmp,
                            unsigned long long *total, uint32_t *div, cudaStream_t st);
// cost[t] = list length of tile t + 1.
void launch_list_cost(const uint2 *ranges, uint32_t T, uint32_t *cost, cudaStream_t st);
// Tile launch order for the blending kernels (order: launch slot -> tile;
// null = index order): heaviest list first, worth it only for a few waves of
// CTAs (tile_order_pays).  With cost, heaviest measured cost first instead.
// buckets: 64 words of scratch.
bool tile_order_pays(uint32_t total_tiles);
void launch_tile_order(const uint2 *ranges, uint32_t n, uint32_t *order, uint32_t *buckets, cudaStream_t st,
                       const uint32_t *cost = nullptr);

// status: a staging wait that runs out records GS_ERR_TIMEOUT there.
void launch_loss(const float *img, const float *target, int B, int W, int H, float lambda, float *loss_out,
                 float *d_img, float *maps, double *acc, DevStatus *status, cudaStream_t st);

struct AdamArgs {
    float lr[15][4];   // per plane, per lane (already times sqrt(B) when asked)
    float b1, b2, eps;
    float bc1, bc2;    // 1 - b1^t, 1 - b2^t (host step)
    long long *dstep;  // non-null: [0] step counter on the device, ticked before the update;
                       // [1] holds the float bias corrections the tick computes
    const uint8_t *vis; // non-null: only Gaussians with vis[i] != 0 are updated (visible-only Adam)
};
void launch_adam(const SceneMut &p, const SceneView &g, const SceneMut &m, const SceneMut &v, const AdamArgs &a,
                 const DevStatus *status, cudaStream_t st);

}  // namespace gs
