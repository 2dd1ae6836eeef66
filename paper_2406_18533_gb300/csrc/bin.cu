// K2 (depth order of the (view, Gaussian) pairs and the offsets scan), K3
// (fragment emission), K4 (LSD radix sort, 8- or 9-bit digits) and K5
// (per-tile ranges): the "intersection test" and "increasing depth"
// ordering of Sec. 2.1 step 2, built on 16x16 pixel blocks (Fig. 2).
//
// Sizes that depend on the data (the fragment count F) stay on the device:
// every kernel after the scan reads F from device memory and grids are sized
// from the caller's capacity, so the whole binning needs no host round trip
// and can be captured in a CUDA graph.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;   // 2048 values per block

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t &excl, uint32_t *smem_warp)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) smem_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? smem_warp[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < (int)(blockDim.x >> 5)) smem_warp[lane] = si - s;
        if (lane == 31) smem_warp[32] = si;
    }
    __syncthreads();
    excl = smem_warp[w] + inc - x;
    const uint32_t total = smem_warp[32];
    __syncthreads();
    return total;
}

// Scan input value: the value itself, or 1 for a nonzero value (NZ).
template <bool NZ>
__device__ __forceinline__ uint32_t scan_in(uint32_t x)
{
    return NZ ? (x != 0u) : x;
}

// n_dev, when set, caps the count on the device (items past it read as 0 and
// get no output).
__device__ __forceinline__ int64_t scan_count(int64_t n, const uint32_t *n_dev)
{
    return n_dev && (int64_t)*n_dev < n ? (int64_t)*n_dev : n;
}

template <bool NZ>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t *in, int64_t n, const uint32_t *n_dev,
                                                              uint32_t *block_sums)
{
    __shared__ uint32_t sw[33];
    n = scan_count(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += scan_in<NZ>(in[base + k]);
    uint32_t excl;
    const uint32_t tot = block_excl_scan(s, excl, sw);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// One block of 1024 threads scans the block sums (uint64 running total).
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t *block_sums, int64_t nb, unsigned long long *total)
{
    __shared__ unsigned long long sw[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t lo = (int64_t)threadIdx.x * per;
    unsigned long long s = 0;
    for (int64_t i = lo; i < lo + per && i < nb; ++i) s += block_sums[i];
    unsigned long long inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sw[w] = inc;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = sw[lane];
        unsigned long long vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        sw[lane] = vi - v;
        if (lane == 31) sw[32] = vi;
    }
    __syncthreads();
    unsigned long long run = sw[w] + inc - s;
    for (int64_t i = lo; i < lo + per && i < nb; ++i) {
        const uint32_t x = block_sums[i];
        block_sums[i] = (uint32_t)run;   // wraps above 2^32: callers check *total first
        run += x;
    }
    if (threadIdx.x == 0 && total) *total = sw[32];
}

template <bool NZ>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t *in, uint32_t *out, int64_t n,
                                                            const uint32_t *n_dev, const uint32_t *block_offs)
{
    __shared__ uint32_t sw[33];
    n = scan_count(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? scan_in<NZ>(in[base + k]) : 0u;
        s += v[k];
    }
    uint32_t excl;
    block_excl_scan(s, excl, sw);
    uint32_t run = block_offs[blockIdx.x] + excl;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// Tile rectangle covered by a (view, Gaussian) footprint (centre uv, radius
// r in pixels), with the same IEEE single operations as the transformation
// kernel, packed as {x0 | x1 << 16, y0 | y1 << 16}; empty (x0 > x1) when the
// Gaussian is culled or its footprint misses the image.  Tile coordinates fit
// 16 bits (at most 65536 / 8 tiles per axis).
__device__ __forceinline__ uint2 tile_rect(const ViewCam &c, float2 uv, int r, int tile)
{
    const uint2 empty = make_uint2(1u, 0u);
    if (r <= 0) return empty;
    const float rf = (float)r;
    const float inv_tile = 1.f / (float)tile;
    const float x0 = fmaxf(floorf(__fmul_rn(__fsub_rn(uv.x, rf), inv_tile)), 0.f);
    const float x1 = fminf(floorf(__fmul_rn(__fadd_rn(uv.x, rf), inv_tile)), (float)(c.TX - 1));
    const float y0 = fmaxf(floorf(__fmul_rn(__fsub_rn(uv.y, rf), inv_tile)), 0.f);
    const float y1 = fminf(floorf(__fmul_rn(__fadd_rn(uv.y, rf), inv_tile)), (float)(c.TY - 1));
    if (!(x0 <= x1 && y0 <= y1)) return empty;
    return pack_rect((uint32_t)x0, (uint32_t)x1, (uint32_t)y0, (uint32_t)y1);
}

__device__ __forceinline__ uint32_t rect_area(uint2 r)
{
    const uint32_t x0 = r.x & 0xffffu, x1 = r.x >> 16, y0 = r.y & 0xffffu, y1 = r.y >> 16;
    return (x0 <= x1 && y0 <= y1) ? (x1 - x0 + 1u) * (y1 - y0 + 1u) : 0u;
}

// Float depth -> unsigned integer of the same order (-0 taken as +0).
__device__ __forceinline__ uint32_t depth_order_bits(float d)
{
    const uint32_t b = __float_as_uint(d + 0.f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Per (view, Gaussian) pair i: its tile rectangle and tile count (nonzero =
// visible: the input of the scan that compacts the visible pairs).  The
// transformation kernel writes the same two arrays in a training step.
__global__ void __launch_bounds__(256) k_pair_rect(ViewBatch vb, ProjView p, uint2 *rect, uint32_t *area)
{
    const int64_t n = (int64_t)vb.B * p.N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 rc = tile_rect(vb.v[(int)(i / p.N)], p.xy[i], p.radius[i], vb.tile);
        rect[i] = rc;
        area[i] = rect_area(rc);
    }
}

// The visible pairs, compacted in index order (so the stable sort keeps equal
// depths in ascending index): key = depth_order_bits(depth), value = pair
// index.  Thread 0 writes the visible count.
__global__ void __launch_bounds__(256) k_pair_compact(int64_t n, const float4 *rgb_d, const uint32_t *area,
                                                      const uint32_t *pos, const unsigned long long *total,
                                                      uint32_t *keys, uint32_t *vals, uint32_t *n_vis)
{
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i0 == 0) *n_vis = (uint32_t)*total;
    for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!area[i]) continue;
        const uint32_t j = pos[i];
        keys[j] = depth_order_bits(reinterpret_cast<const float *>(rgb_d)[4 * i + 3]);
        vals[j] = (uint32_t)i;
    }
}

// The visible pairs' tile rectangles and tile counts in depth order (the
// counts are the input of the offsets scan), so that the emission reads
// everything in order; with culling (rm non-null) one 16-byte random read per
// pair brings the rectangle and the kept-tile bits.
__global__ void __launch_bounds__(256) k_gather_counts(const uint32_t *order, const uint2 *rect,
                                                       const uint32_t *area, const uint4 *rm, int64_t n,
                                                       const uint32_t *n_vis, uint32_t *counts, uint32_t *rx,
                                                       uint32_t *ry, uint2 *keep)
{
    // GU pairs per thread per round, all their loads issued before any is
    // used: the random record reads are latency-bound, so more in flight
    constexpr int GU = 4;
    const int64_t nv = (int64_t)*n_vis < n ? (int64_t)*n_vis : n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j0 < nv; j0 += GU * stride) {
        uint32_t o[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int64_t j = j0 + u * stride;
            o[u] = j < nv ? order[j] : 0xffffffffu;
        }
        if (rm) {
            uint4 r[GU];
#pragma unroll
            for (int u = 0; u < GU; ++u)       // o >= n only past nv or after a failed (timed-out) sort
                r[u] = o[u] < n ? rm[o[u]] : make_uint4(1u, 0u, 0u, 0u);
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int64_t j = j0 + u * stride;
                if (j >= nv) break;
                const uint32_t ra = rect_area(make_uint2(r[u].x, r[u].y));
                const uint64_t m = ((uint64_t)r[u].w << 32) | r[u].z;
                counts[j] = ra <= TILE_CULL_MAX_AREA ? (uint32_t)__popcll(m) : ra;
                rx[j] = r[u].x;
                ry[j] = r[u].y;
                keep[j] = make_uint2(r[u].z, r[u].w);
            }
        } else {
            uint2 rc[GU];
            uint32_t ar[GU];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const bool ok = o[u] < n;
                rc[u] = ok ? rect[o[u]] : make_uint2(1u, 0u);
                ar[u] = ok ? area[o[u]] : 0u;
            }
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int64_t j = j0 + u * stride;
                if (j >= nv) break;
                counts[j] = ar[u];
                rx[j] = rc[u].x;
                ry[j] = rc[u].y;
            }
        }
    }
}

// ---------------------------------------------------------------- K3 emit

// Position of the k-th (from 0) set bit of m; m has more than k set bits.
__device__ __forceinline__ uint32_t select_bit32(uint32_t m, uint32_t k)
{
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t c = (uint32_t)__popc(m & ((1u << w) - 1u));   // set bits in the low w
        const bool up = k >= c;
        k = up ? k - c : k;
        m = up ? m >> w : m;
        pos += up ? (uint32_t)w : 0u;
    }
    return pos;
}

// The same for the 64-bit mask (hi:lo).
__device__ __forceinline__ uint32_t select_bit64(uint32_t lo, uint32_t hi, uint32_t k)
{
    const uint32_t c = (uint32_t)__popc(lo);
    return k < c ? select_bit32(lo, k) : 32u + select_bit32(hi, k - c);
}

// Emits the fragments of pair order[j] at offsets[j]: key = global tile id,
// value = Gaussian index.  Visiting the pairs in depth order puts every
// tile's fragments in (depth, index) order, so a stable sort on the tile id
// alone finishes the job.  The work is split by output slots, not by pairs:
// warp w writes fragments [w S, (w + 1) S) (S = EMIT_SLOTS).  It finds the
// pair holding its first slot by a 32-way search of the offsets, then keeps
// a window of 32 consecutive pairs (lane l holds pair p + l) and writes 32
// slots per round, slot f by lane f mod 32 (coalesced stores), each lane
// finding its slot's pair in the window by binary search over the lanes'
// offsets; the window moves on when a round runs past it.  Since every pair
// in the depth order has at least one fragment, a window that starts at the
// pair holding a round's first slot covers the round; a slot past the window
// (only after a failed pair sort) is looked up in the offsets directly.  A
// pair that covers many tiles (a large Gaussian near a camera) is thus
// shared by many warps instead of holding up one.  Thread 0 publishes F
// (status, count_out); nothing is written past capacity.
constexpr uint32_t EMIT_SLOTS = 512;

// One pair of the depth order, as a lane of the emission window sees it.
struct EmitPair {
    uint32_t start, count, corner, wdt, tx_row, g, mlo, mhi;
};

__device__ __forceinline__ EmitPair emit_pair(const ViewBatch &vb, int64_t N, int64_t nb, int64_t n, int64_t p,
                                              const uint32_t *order, const uint32_t *rx, const uint32_t *ry,
                                              const uint2 *keep, const uint32_t *offsets, uint32_t F,
                                              float cull_alpha)
{
    EmitPair e{F, 0u, 0u, 1u, 0u, 0u, 0xffffffffu, 0xffffffffu};
    if (p < 0 || p >= n) return e;
    e.start = offsets[p];
    const int64_t i = (int64_t)order[p];
    const uint2 rc = make_uint2(rx[p], ry[p]);
    uint32_t area = rect_area(rc);
    if (area && i < nb) {                        // i >= B * N only after a failed (timed-out) pair sort
        const int v = (int)(i / N);
        e.g = (uint32_t)(i - (int64_t)v * N);
        const uint32_t x0 = rc.x & 0xffffu;
        e.wdt = (rc.x >> 16) - x0 + 1u;
        e.tx_row = (uint32_t)vb.v[v].TX;
        e.corner = vb.v[v].tile_base + (rc.y & 0xffffu) * e.tx_row + x0;   // tile (x0, y0)
        if (cull_alpha > 0.f && area <= TILE_CULL_MAX_AREA) {
            const uint2 k = keep[p];
            e.mlo = k.x;
            e.mhi = k.y;
        }
    } else {
        area = 0u;
    }
    // a whole rectangle (mask all ones) or the set bits of a culled one's mask
    e.count = (e.mlo & e.mhi) == 0xffffffffu ? area : (uint32_t)(__popc(e.mlo) + __popc(e.mhi));
    return e;
}

// The tile of the local-th kept tile of a pair.
__device__ __forceinline__ uint32_t emit_tile(const EmitPair &e, uint32_t local)
{
    const uint32_t slot = (e.mlo & e.mhi) == 0xffffffffu ? local : select_bit64(e.mlo, e.mhi, local);
    const uint32_t dy = slot / e.wdt, dx = slot - dy * e.wdt;
    return e.corner + dy * e.tx_row + dx;
}

__global__ void __launch_bounds__(256) k_emit_keys(ViewBatch vb, int64_t N, const uint32_t *n_vis,
                                                   const uint32_t *order, const uint32_t *rx, const uint32_t *ry,
                                                   const uint2 *keep, const uint32_t *offsets, uint32_t *keys,
                                                   uint32_t *vals, uint64_t capacity,
                                                   const unsigned long long *total, DevStatus *status,
                                                   uint32_t *count_out, float cull_alpha)
{
    const int64_t nb = (int64_t)vb.B * N;
    const int64_t n = (int64_t)*n_vis < nb ? (int64_t)*n_vis : nb;   // pairs in depth order
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long F = *total;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status->needed = F;
        status->counters[0] = F;
        status->counters[1] = 0ull;
        status->counters[2] = 0ull;
        status->counters[4] = 0ull;
        status->counters[5] = 0ull;
        if (F > capacity) {
            atomicCAS(&status->code, 0, (int)GS_ERR_CAPACITY);
            *count_out = 0u;
        } else {
            *count_out = (uint32_t)F;
        }
    }
    const uint64_t f_begin = warp * EMIT_SLOTS;
    if (F > capacity || f_begin >= F || n <= 0) return;   // uniform over the warp
    const uint32_t f_end = (uint32_t)(f_begin + EMIT_SLOTS < F ? f_begin + EMIT_SLOTS : F);
    const uint32_t fb = (uint32_t)f_begin, F32 = (uint32_t)F;
    // the pair holding slot fb: the last p < n with offsets[p] <= fb (offsets[0] = 0)
    int64_t lo = 0, hi = n;
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t q = lo + lane * step;
        const uint32_t b = __ballot_sync(0xffffffffu, q < hi && offsets[q] <= fb);
        lo += (int64_t)(31 - __clz(b)) * step;   // lane 0 (q = lo) always qualifies
        hi = lo + step < hi ? lo + step : hi;
    }
    {
        const uint32_t b = __ballot_sync(0xffffffffu, lo + lane < hi && offsets[lo + lane] <= fb);
        lo += 31 - __clz(b);
    }
    int64_t pw = lo;
    EmitPair e = emit_pair(vb, N, nb, n, pw + lane, order, rx, ry, keep, offsets, F32, cull_alpha);
    for (uint32_t fr = fb; fr < f_end; fr += 32) {
        const uint32_t last = fr + 31 < f_end ? fr + 31 : f_end - 1;
        const uint32_t wend = __shfl_sync(0xffffffffu, e.start + e.count, 31);
        if (last >= wend) {                      // move the window to the pair holding fr
            const uint32_t b = __ballot_sync(0xffffffffu, e.start <= fr);
            pw += 31 - __clz(b);
            e = emit_pair(vb, N, nb, n, pw + lane, order, rx, ry, keep, offsets, F32, cull_alpha);
        }
        const uint32_t f = fr + lane;
        int L = 0;                               // last lane of the window with start <= f
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t s = __shfl_sync(0xffffffffu, e.start, L + step);
            if (s <= f) L += step;
        }
        EmitPair h;
        h.start = __shfl_sync(0xffffffffu, e.start, L);
        h.count = __shfl_sync(0xffffffffu, e.count, L);
        h.corner = __shfl_sync(0xffffffffu, e.corner, L);
        h.wdt = __shfl_sync(0xffffffffu, e.wdt, L);
        h.tx_row = __shfl_sync(0xffffffffu, e.tx_row, L);
        h.g = __shfl_sync(0xffffffffu, e.g, L);
        h.mlo = __shfl_sync(0xffffffffu, e.mlo, L);
        h.mhi = __shfl_sync(0xffffffffu, e.mhi, L);
        if (f >= f_end) continue;
        if (f - h.start >= h.count) {
            // past the window (pairs without fragments, only after a failed pair
            // sort): the last pair with offsets <= f, found directly
            int64_t a = pw, c = n;
            while (c - a > 1) {
                const int64_t m = (a + c) >> 1;
                if (offsets[m] <= f) a = m; else c = m;
            }
            h = emit_pair(vb, N, nb, n, a, order, rx, ry, keep, offsets, F32, cull_alpha);
            if (f - h.start >= h.count) continue;
        }
        keys[f] = emit_tile(h, f - h.start);
        vals[f] = h.g;
    }
}

// ---------------------------------------------------------------- K4 radix sort (one-sweep)
//
// LSD radix sort of 32-bit keys with 32-bit values on RB-bit digits (RB = 8
// or 9), stable.  An upfront kernel histograms every digit position in one
// read of the keys; each pass is then a single kernel: a CTA takes the next
// tile of RS_TILE keys (tile order = launch order, from an atomic counter),
// ranks its keys stably, publishes its per-digit counts, finds the keys of
// all earlier tiles per digit by decoupled look-back, stages its keys in
// shared memory in output order and writes them out so that consecutive
// threads store consecutive addresses of a digit's run.  The look-back spin
// is bounded: a wait that runs out sets GS_ERR_TIMEOUT and the pass finishes
// with wrong positions instead of hanging.  Every store is checked against
// the key count, so even a pass whose input came out of a failed pass (keys
// duplicated or missing, so the up-front digit histogram no longer matches)
// stays inside the buffers.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_WARP_KEYS = 32 * RS_ITEMS;         // 512 consecutive keys per warp
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;      // 4096 keys per tile
constexpr int RS_MAX_PASSES = 4;
constexpr int RS_MAX_NB = 512;
constexpr uint32_t LB_AGG = 1u << 30;               // look-back flag: tile count available
constexpr uint32_t LB_PRE = 2u << 30;               // look-back flag: inclusive prefix available
constexpr uint32_t LB_VAL = (1u << 30) - 1u;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;        // default polls of one look-back wait
constexpr int LB_BATCH = 8;                         // look-back words read per round

// Test hooks (gs_debug_set_lookback): the spin limit, and whether tile 0 of
// every pass withholds its look-back words (a flag nothing sets), so that a
// test can make the bounded wait run out.
uint32_t g_lb_spin_limit = LB_SPIN_LIMIT;
int g_lb_withhold = 0;

// Digit histograms of every pass.  A thread takes 16 consecutive keys (four
// 16-byte loads: the key buffers are 16-byte aligned) and adds runs of equal
// digits at once, which keeps the shared-memory atomics of skewed digit
// positions (float exponents, the high bits of tile ids) few.
template <int RB>
__global__ void __launch_bounds__(RS_THREADS) k_digit_hist(const uint32_t *keys, const uint32_t *count, int passes,
                                                           uint32_t *ghist)
{
    constexpr int NB = 1 << RB;
    __shared__ uint32_t h[RS_MAX_PASSES * NB];
    for (int i = threadIdx.x; i < RS_MAX_PASSES * NB; i += RS_THREADS) h[i] = 0u;
    __syncthreads();
    const uint32_t n = *count;
    const uint64_t chunks = ((uint64_t)n + 15) / 16;
    for (uint64_t c = blockIdx.x * (uint64_t)RS_THREADS + threadIdx.x; c < chunks;
         c += (uint64_t)gridDim.x * RS_THREADS) {
        const uint64_t b = c * 16;
        const int m = (int)((uint64_t)n - b < 16 ? (uint64_t)n - b : 16);
        uint32_t k[16];
        if (m == 16) {
            const uint4 *q = reinterpret_cast<const uint4 *>(keys + b);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint4 x = q[u];
                k[4 * u] = x.x;
                k[4 * u + 1] = x.y;
                k[4 * u + 2] = x.z;
                k[4 * u + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 16; ++u) k[u] = u < m ? keys[b + u] : 0u;
        }
        for (int p = 0; p < passes; ++p) {
            const int sh = RB * p;
            uint32_t cur = (k[0] >> sh) & (uint32_t)(NB - 1), run = 1;
#pragma unroll
            for (int u = 1; u < 16; ++u) {
                if (u < m) {
                    const uint32_t d = (k[u] >> sh) & (uint32_t)(NB - 1);
                    if (d == cur) {
                        ++run;
                    } else {
                        atomicAdd(&h[p * NB + cur], run);
                        cur = d;
                        run = 1;
                    }
                }
            }
            atomicAdd(&h[p * NB + cur], run);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * NB; i += RS_THREADS) {
        const uint32_t c = h[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

// Exclusive scan of each pass's digit counts (one CTA per pass).
template <int RB>
__global__ void __launch_bounds__(RS_THREADS) k_digit_offsets(uint32_t *ghist)
{
    constexpr int NB = 1 << RB, DPT = NB / RS_THREADS;
    __shared__ uint32_t sw[33];
    uint32_t *h = ghist + NB * blockIdx.x;
    uint32_t x[DPT], s = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        x[k] = h[threadIdx.x * DPT + k];
        s += x[k];
    }
    uint32_t excl;
    block_excl_scan(s, excl, sw);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        h[threadIdx.x * DPT + k] = excl;
        excl += x[k];
    }
}

// Ranking: warp w owns the RS_WARP_KEYS consecutive keys t0 + w*RS_WARP_KEYS
// + [0, RS_WARP_KEYS), item i of lane l being key t0 + w*RS_WARP_KEYS + 32 i
// + l.  Items are ranked in order against per-warp running digit counts
// (the lanes sharing a digit found with one ballot per digit bit), so ranks
// are stable within the warp; per-digit
// prefixes over the warps and over the digits then give every key its
// position in the tile's output order.
template <int RB>
__global__ void __launch_bounds__(RS_THREADS, 4) k_onesweep(const uint32_t *kin, const uint32_t *vin,
                                                            uint32_t *kout, uint32_t *vout, const uint32_t *count,
                                                            int shift, const uint32_t *doff, uint32_t *look,
                                                            uint32_t *tile_ctr, DevStatus *status,
                                                            uint32_t spin_limit, int withhold_first)
{
    constexpr int NB = 1 << RB, DPT = NB / RS_THREADS;
    constexpr int UNION_WORDS = RS_WARPS * NB > 2 * RS_TILE ? RS_WARPS * NB : 2 * RS_TILE;
    __shared__ __align__(16) uint32_t sm[UNION_WORDS];
    __shared__ uint32_t gofs[NB];
    __shared__ uint32_t sw[33];
    __shared__ uint32_t s_tile;
    uint32_t *wcnt = sm;                              // ranking: [RS_WARPS][NB] running counts
    uint32_t *skey = sm, *sval = sm + RS_TILE;        // afterwards: the tile in output order
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t n = *count;
    if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int j = t; j < RS_WARPS * NB; j += RS_THREADS) wcnt[j] = 0u;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t t0 = (uint64_t)tile * RS_TILE;
    if (t0 >= n) return;
    const uint32_t lt = lanemask_lt();
    const uint64_t wb = t0 + (uint64_t)w * RS_WARP_KEYS;
    uint32_t key[RS_ITEMS], pos[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t idx = wb + 32 * i + lane;
        key[i] = idx < n ? kin[idx] : 0u;
    }
    uint32_t *mycnt = wcnt + w * NB;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const bool valid = wb + 32 * i + lane < n;
        const uint32_t d = valid ? ((key[i] >> shift) & (uint32_t)(NB - 1)) : (uint32_t)NB;
        // the valid lanes holding the same digit: one ballot per digit bit
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
        const uint32_t base = valid ? mycnt[d] : 0u;
        pos[i] = base + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0u) mycnt[d] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t owns digits t*DPT .. t*DPT + DPT - 1: warp prefixes in place, tile counts
    uint32_t cnt[DPT];
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        const int d = t * DPT + k;
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < RS_WARPS; ++j) {
            const uint32_t c = wcnt[j * NB + d];
            wcnt[j * NB + d] = run;
            run += c;
        }
        cnt[k] = run;
        if (!(withhold_first && tile == 0)) atomicExch(look + (size_t)tile * NB + d, (tile == 0 ? LB_PRE : LB_AGG) | run);
    }
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) tsum += cnt[k];
    uint32_t start;
    block_excl_scan(tsum, start, sw);                // tile-local start of digit t*DPT
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        const int d = t * DPT + k;
        uint32_t excl = 0;
        if (tile > 0) {
            // walk back over earlier tiles, LB_BATCH words in flight at a time
            int64_t pt = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (true) {
                uint32_t v[LB_BATCH];
#pragma unroll
                for (int b = 0; b < LB_BATCH; ++b)
                    v[b] = pt - b >= 0 ? *(const volatile uint32_t *)(look + (size_t)(pt - b) * NB + d) : LB_PRE;
                bool stop = false, blocked = false;
#pragma unroll
                for (int b = 0; b < LB_BATCH; ++b) {
                    if (!stop && !blocked) {
                        if ((v[b] & (LB_AGG | LB_PRE)) == 0u) {
                            blocked = true;              // not published yet: read again from here
                        } else {
                            excl += v[b] & LB_VAL;
                            --pt;
                            stop = (v[b] & LB_PRE) != 0u;
                        }
                    }
                }
                if (stop) break;
                if (blocked) {                       // wait on that word alone, then read a batch again
                    const volatile uint32_t *q = look + (size_t)pt * NB + d;
                    bool timed_out = false;
                    while ((*q & (LB_AGG | LB_PRE)) == 0u) {
                        if (++spins > spin_limit) {      // give up: report instead of hanging
                            atomicCAS(&status->code, 0, (int)GS_ERR_TIMEOUT);
                            timed_out = true;
                            break;
                        }
                    }
                    if (timed_out) break;
                }
            }
            atomicExch(look + (size_t)tile * NB + d, LB_PRE | (excl + cnt[k]));
        }
#pragma unroll
        for (int j = 0; j < RS_WARPS; ++j) wcnt[j * NB + d] += start;
        gofs[d] = doff[d] + excl - start;             // output index = gofs[d] + tile position
        start += cnt[k];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i)
        if (wb + 32 * i + lane < n) pos[i] += mycnt[(key[i] >> shift) & (uint32_t)(NB - 1)];
    __syncthreads();                                  // the counts are dead: stage the tile over them
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t idx = wb + 32 * i + lane;
        if (idx < n) {
            skey[pos[i]] = key[i];
            sval[pos[i]] = vin[idx];                  // values are read only now, to save registers
        }
    }
    __syncthreads();
    const uint32_t tile_n = (uint32_t)((uint64_t)n - t0 < (uint64_t)RS_TILE ? (uint64_t)n - t0 : (uint64_t)RS_TILE);
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t idx = (uint32_t)(k * RS_THREADS + t);
        if (idx < tile_n) {
            const uint32_t kk = skey[idx];
            const uint32_t dst = gofs[(kk >> shift) & (uint32_t)(NB - 1)] + idx;
            if (dst < n) {                            // always, unless an earlier pass failed
                kout[dst] = kk;
                vout[dst] = sval[idx];
            }
        }
    }
}

// ---------------------------------------------------------------- K5 ranges

__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t *keys, const uint32_t *count, uint2 *ranges,
                                                     uint32_t total_tiles)
{
    // four keys per thread (one 16-byte load: the key buffers are 16-byte aligned)
    const uint32_t n = *count;
    const uint64_t quads = ((uint64_t)n + 3) / 4;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < quads; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i0 = 4 * q;
        uint32_t k[6];                            // keys i0-1 .. i0+4
        k[0] = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
        if (i0 + 4 <= n) {
            const uint4 x = *reinterpret_cast<const uint4 *>(keys + i0);
            k[1] = x.x; k[2] = x.y; k[3] = x.z; k[4] = x.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) k[1 + u] = i0 + u < n ? keys[i0 + u] : 0xffffffffu;
        }
        k[5] = i0 + 4 < n ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = i0 + u;
            const uint32_t tile = k[1 + u];
            if (i >= n || tile >= total_tiles) continue;
            if (i == 0 || k[u] != tile) ranges[tile].x = (uint32_t)i;
            if (i + 1 == n || k[2 + u] != tile) ranges[tile].y = (uint32_t)(i + 1);
        }
    }
}

// The 64-bit fragment keys of the binning's public output: tile id << 32 |
// float bits of the fragment's depth in its view.
__global__ void __launch_bounds__(256) k_compose_keys(ViewBatch vb, int64_t N, const uint32_t *tiles,
                                                      const uint32_t *vals, const uint32_t *count,
                                                      const float4 *rgb_d, uint64_t *keys)
{
    const uint32_t n = *count;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t tile = tiles[i], g = vals[i];
        int v = 0;
        while (v + 1 < vb.B && vb.v[v + 1].tile_base <= tile) ++v;
        // g >= N only after a failed (timed-out) sort, which the status reports
        const float depth =
            (int64_t)g < N ? reinterpret_cast<const float *>(rgb_d)[4 * ((int64_t)v * N + g) + 3] : 0.f;
        keys[i] = ((uint64_t)tile << 32) | __float_as_uint(depth);
    }
}

// ---------------------------------------------------------------- storage order (Morton code)

// Order-preserving unsigned image of a float (for atomicMin / atomicMax).
__device__ __forceinline__ uint32_t float_order_bits(float f)
{
    const uint32_t b = __float_as_uint(f + 0.f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float float_from_order_bits(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Bounding box of the finite positions: bb[0..2] = min x, y, z, bb[3..5] = max
// (order bits; bb starts at {~0 x3, 0 x3}).
// bb[0..5] = empty box, bb[6] = the key count for the sort.
__global__ void k_bbox_init(uint32_t *bb, uint32_t n)
{
    if (threadIdx.x < 6) bb[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
    if (threadIdx.x == 6) bb[6] = n;
}

__global__ void __launch_bounds__(256) k_bbox(const float4 *mo, int64_t N, uint32_t *bb)
{
    __shared__ uint32_t s[6];
    if (threadIdx.x < 6) s[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
    __syncthreads();
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 m = mo[i];
        if (!(isfinite(m.x) && isfinite(m.y) && isfinite(m.z))) continue;
        const uint32_t k[3] = {float_order_bits(m.x), float_order_bits(m.y), float_order_bits(m.z)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], k[a]);
            hi[a] = max(hi[a], k[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        atomicMin(&s[a], lo[a]);
        atomicMax(&s[3 + a], hi[a]);
    }
    __syncthreads();
    if (threadIdx.x < 3) atomicMin(&bb[threadIdx.x], s[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&bb[threadIdx.x], s[threadIdx.x]);
}

// 10-bit cell of coordinate x in [lo, hi]: floor((x - lo) * (1024 / (hi - lo)))
// with each float operation explicitly rounded, clamped to 1023 (a flat axis
// or a non-finite x gives 0).
__device__ __forceinline__ uint32_t morton_cell(float x, float lo, float hi)
{
    if (!(hi > lo) || !isfinite(x)) return 0u;
    const float scale = __fdiv_rn(1024.f, __fsub_rn(hi, lo));
    const float q = floorf(__fmul_rn(__fsub_rn(x, lo), scale));
    return q >= 1023.f ? 1023u : (q <= 0.f ? 0u : (uint32_t)q);
}

// Bits of v spread to every third position (bit b -> bit 3b).
__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(256) k_morton(const float4 *mo, int64_t N, const uint32_t *bb, uint32_t *keys,
                                                uint32_t *vals)
{
    const float lx = float_from_order_bits(bb[0]), ly = float_from_order_bits(bb[1]), lz = float_from_order_bits(bb[2]);
    const float hx = float_from_order_bits(bb[3]), hy = float_from_order_bits(bb[4]), hz = float_from_order_bits(bb[5]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 m = mo[i];
        const bool ok = isfinite(m.x) && isfinite(m.y) && isfinite(m.z);
        const uint32_t cx = ok ? morton_cell(m.x, lx, hx) : 0u, cy = ok ? morton_cell(m.y, ly, hy) : 0u,
                       cz = ok ? morton_cell(m.z, lz, hz) : 0u;
        keys[i] = spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
        vals[i] = (uint32_t)i;
    }
}

// dst plane k, entry i = src plane k, entry perm[i] (15 float4 planes).
__global__ void __launch_bounds__(256) k_permute(SceneView src, const uint32_t *perm, SceneMut dst)
{
    const int pl = blockIdx.y;
    const float4 *sp = pl == 0 ? src.mo : pl == 1 ? src.ls : pl == 2 ? src.q : src.sh + (int64_t)(pl - 3) * src.N;
    float4 *dp = pl == 0 ? dst.mo : pl == 1 ? dst.ls : pl == 2 ? dst.q : dst.sh + (int64_t)(pl - 3) * dst.N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < src.N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = perm[i];
        dp[i] = (int64_t)j < src.N ? sp[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

}  // namespace

void set_lookback_debug(uint32_t spin_limit, int withhold_first)
{
    g_lb_spin_limit = spin_limit ? spin_limit : LB_SPIN_LIMIT;
    g_lb_withhold = withhold_first ? 1 : 0;
}

// Blocks of 256 threads for a grid-stride loop over `items`: enough to fill
// every SM several times, no more (small blocks are bound by block launches).
static unsigned stride_blocks(uint64_t items)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0, m = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        sms = m;
    }
    const uint64_t need = (items + 255) / 256, cap = (uint64_t)sms * 16;
    return (unsigned)(need < 1 ? 1 : need < cap ? need : cap);
}

size_t scan_temp_bytes(int64_t n)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(nb + 1) * sizeof(uint32_t) + 64;
}

void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *total, void *temp,
                           cudaStream_t st, const uint32_t *n_dev, bool nonzero)
{
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(unsigned long long), st);
        return;
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t *bs = reinterpret_cast<uint32_t *>(temp);
    if (nonzero)
        k_scan_reduce<true><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, n_dev, bs);
    else
        k_scan_reduce<false><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, n_dev, bs);
    k_scan_blocks<<<1, 1024, 0, st>>>(bs, nb, total);
    if (nonzero)
        k_scan_down<true><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, n_dev, bs);
    else
        k_scan_down<false><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, n_dev, bs);
    count_launches(3);
}

template <int RB>
static void radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint64_t capacity,
                       const uint32_t *count, int passes, void *temp, DevStatus *status, cudaStream_t st);

uint32_t *launch_depth_order(const ViewBatch &vb, const ProjView &p, bool rect_ready, uint2 *rect, uint32_t *area,
                             uint32_t *keys, uint32_t *order, uint32_t *keys_alt, uint32_t *order_alt,
                             uint32_t *pos, uint32_t *n_vis, unsigned long long *total, void *scan_tmp,
                             void *sort_tmp, DevStatus *status, cudaStream_t st)
{
    const int64_t n = (int64_t)vb.B * p.N;
    if (!rect_ready && n > 0) {
        k_pair_rect<<<stride_blocks((uint64_t)n), 256, 0, st>>>(vb, p, rect, area);
        count_launches(1);
    }
    launch_exclusive_scan(area, pos, n, total, scan_tmp, st, nullptr, true);
    k_pair_compact<<<stride_blocks(n > 0 ? (uint64_t)n : 1), 256, 0, st>>>(n, p.rgb_d, area, pos, total, keys, order,
                                                                          n_vis);
    count_launches(1);
    radix_sort<8>(keys, order, keys_alt, order_alt, (uint64_t)n, n_vis, 4, sort_tmp, status, st);
    return order;                                 // four passes: back in the first buffers
}


void launch_gather_counts(const uint32_t *order, const uint2 *rect, const uint32_t *area, const uint4 *rm, int64_t n,
                          const uint32_t *n_vis, uint32_t *counts, uint32_t *rx, uint32_t *ry, uint2 *keep,
                          cudaStream_t st)
{
    if (n <= 0) return;
    k_gather_counts<<<stride_blocks((uint64_t)n), 256, 0, st>>>(order, rect, area, rm, n, n_vis, counts, rx, ry,
                                                               keep);
    count_launches(1);
}

void launch_emit_keys(const ViewBatch &vb, int64_t N, const uint32_t *n_vis, const uint32_t *order,
                      const uint32_t *rx, const uint32_t *ry, const uint2 *keep, const uint32_t *offsets,
                      uint32_t *keys, uint32_t *vals, uint64_t capacity, const unsigned long long *total,
                      DevStatus *status, uint32_t *count_out, float cull_alpha, cudaStream_t st)
{
    // one warp per EMIT_SLOTS output slots of the capacity (warps past F return at once)
    const uint64_t warps = (capacity + EMIT_SLOTS - 1) / EMIT_SLOTS;
    const uint64_t blocks = warps > 0 ? (warps + 7) / 8 : 1;
    k_emit_keys<<<(unsigned)blocks, 256, 0, st>>>(vb, N, n_vis, order, rx, ry, keep, offsets, keys, vals, capacity,
                                                 total, status, count_out, cull_alpha);
    count_launches(1);
}

size_t sort_temp_bytes(uint64_t pairs, uint64_t fragments)
{
    // digit offsets (passes x NB), tile counters, look-back words (tiles x NB):
    // 256 digits for the pair sort, at most 512 for the fragment sort
    const uint64_t tp = (pairs + RS_TILE - 1) / RS_TILE, tf = (fragments + RS_TILE - 1) / RS_TILE;
    const uint64_t look = tp * 256 > tf * 512 ? tp * 256 : tf * 512;
    return (size_t)RS_MAX_PASSES * RS_MAX_NB * 4 + 256 + (size_t)(look ? look : 1) * 4 + 256;
}

template <int RB>
static void radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint64_t capacity,
                       const uint32_t *count, int passes, void *temp, DevStatus *status, cudaStream_t st)
{
    constexpr int NB = 1 << RB;
    if (capacity == 0 || passes <= 0) return;
    const uint64_t tiles = (capacity + RS_TILE - 1) / RS_TILE;
    char *tp = reinterpret_cast<char *>(temp);
    uint32_t *ghist = reinterpret_cast<uint32_t *>(tp);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(tp + (size_t)RS_MAX_PASSES * RS_MAX_NB * 4);
    uint32_t *look = reinterpret_cast<uint32_t *>(tp + (size_t)RS_MAX_PASSES * RS_MAX_NB * 4 + 256);
    cudaMemsetAsync(tp, 0, (size_t)RS_MAX_PASSES * RS_MAX_NB * 4 + 256, st);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t hb = (capacity + RS_THREADS * 16 - 1) / (RS_THREADS * 16);
    if (hb > (uint64_t)sms * 8) hb = (uint64_t)sms * 8;
    k_digit_hist<RB><<<(unsigned)(hb ? hb : 1), RS_THREADS, 0, st>>>(keys, count, passes, ghist);
    k_digit_offsets<RB><<<passes, RS_THREADS, 0, st>>>(ghist);
    count_launches(2);
    uint32_t *ki = keys, *ko = keys_alt, *vi = vals, *vo = vals_alt;
    for (int ps = 0; ps < passes; ++ps) {
        cudaMemsetAsync(look, 0, (size_t)tiles * NB * 4, st);
        k_onesweep<RB><<<(unsigned)tiles, RS_THREADS, 0, st>>>(ki, vi, ko, vo, count, RB * ps, ghist + NB * ps, look,
                                                              ctr + ps, status, g_lb_spin_limit, g_lb_withhold);
        count_launches(1);
        uint32_t *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
}

// Digit width and pass count for tile ids of `tile_bits` bits: 9-bit digits
// where they save a pass (e.g. 17 bits: two passes instead of three).
static void fragment_plan(int tile_bits, int &rb, int &passes)
{
    const int p8 = (tile_bits + 7) / 8, p9 = (tile_bits + 8) / 9;
    rb = p9 < p8 ? 9 : 8;
    passes = p9 < p8 ? p9 : p8;
}

int fragment_sort_passes(int tile_bits)
{
    int rb, passes;
    fragment_plan(tile_bits, rb, passes);
    return passes;
}

void launch_sort_fragments(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                           uint64_t capacity, const uint32_t *count, int tile_bits, void *temp, DevStatus *status,
                           cudaStream_t st)
{
    int rb, passes;
    fragment_plan(tile_bits, rb, passes);
    if (rb == 9)
        radix_sort<9>(keys, vals, keys_alt, vals_alt, capacity, count, passes, temp, status, st);
    else
        radix_sort<8>(keys, vals, keys_alt, vals_alt, capacity, count, passes, temp, status, st);
}

void launch_tile_ranges(const uint32_t *keys, const uint32_t *count, uint64_t capacity, uint2 *ranges,
                        uint32_t total_tiles, cudaStream_t st)
{
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st);
    if (capacity == 0) return;
    k_tile_ranges<<<stride_blocks((capacity + 3) / 4), 256, 0, st>>>(keys, count, ranges, total_tiles);
    count_launches(1);
}

void launch_compose_keys(const ViewBatch &vb, int64_t N, const uint32_t *tiles, const uint32_t *vals,
                         const uint32_t *count, uint64_t capacity, const float4 *rgb_d, uint64_t *keys,
                         cudaStream_t st)
{
    if (capacity == 0) return;
    k_compose_keys<<<stride_blocks(capacity), 256, 0, st>>>(vb, N, tiles, vals, count, rgb_d, keys);
    count_launches(1);
}

// Three arrays of n words, each starting on a 256-byte boundary, then 256
// bytes of counters and the sort's scratch.
static uint64_t spatial_stride(uint64_t n) { return (n + 63) / 64 * 64; }

size_t spatial_order_temp_bytes(int64_t N)
{
    const uint64_t n = (uint64_t)(N > 0 ? N : 1);
    return 3 * 4 * spatial_stride(n) + 256 + sort_temp_bytes(n, 0);
}

void launch_spatial_order(const float4 *mo, int64_t N, uint32_t *perm, void *temp, DevStatus *status,
                          cudaStream_t st)
{
    if (N <= 0) return;
    const uint64_t n = (uint64_t)N;
    char *t = reinterpret_cast<char *>(temp);
    const uint64_t sn = spatial_stride(n);
    uint32_t *keys = reinterpret_cast<uint32_t *>(t);
    uint32_t *keys_alt = keys + sn, *vals_alt = keys + 2 * sn;
    uint32_t *bb = reinterpret_cast<uint32_t *>(t + 12 * sn);
    void *sort_tmp = t + 12 * sn + 256;
    k_bbox_init<<<1, 32, 0, st>>>(bb, (uint32_t)n);
    k_bbox<<<stride_blocks(n), 256, 0, st>>>(mo, N, bb);
    k_morton<<<stride_blocks(n), 256, 0, st>>>(mo, N, bb, keys, perm);
    count_launches(3);
    // 30-bit codes: four stable passes of 8-bit digits, so the result is back in keys / perm
    radix_sort<8>(keys, perm, keys_alt, vals_alt, n, bb + 6, 4, sort_tmp, status, st);
}

void launch_permute(const SceneView &src, const uint32_t *perm, const SceneMut &dst, cudaStream_t st)
{
    if (src.N <= 0) return;
    const unsigned bx = stride_blocks((uint64_t)src.N);
    k_permute<<<dim3(bx, 15), 256, 0, st>>>(src, perm, dst);
    count_launches(1);
}


}  // namespace gs
