// K2 (exclusive scan), K3 (key emission), K4 (LSD radix sort, 8-bit digits)
// and K5 (per-tile ranges): the "intersection test" and "increasing depth"
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

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t *in, int64_t n, uint32_t *block_sums)
{
    __shared__ uint32_t sw[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
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

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t *in, uint32_t *out, int64_t n,
                                                            const uint32_t *block_offs)
{
    __shared__ uint32_t sw[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
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

// Tiles covered by each (view, Gaussian) footprint rectangle, recomputed from
// gs_proj with the same IEEE single operations as the transformation kernel.
__global__ void __launch_bounds__(256) k_count_tiles(ViewBatch vb, ProjView p, uint32_t *ntiles)
{
    const int64_t n = (int64_t)vb.B * p.N;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = p.radius[i];
    uint32_t area = 0;
    if (r > 0) {
        const ViewCam &c = vb.v[(int)(i / p.N)];
        const float2 uv = p.xy[i];
        const float rf = (float)r;
        const float inv_tile = 1.f / (float)vb.tile;
        const float x0 = fmaxf(floorf(__fmul_rn(__fsub_rn(uv.x, rf), inv_tile)), 0.f);
        const float x1 = fminf(floorf(__fmul_rn(__fadd_rn(uv.x, rf), inv_tile)), (float)(c.TX - 1));
        const float y0 = fmaxf(floorf(__fmul_rn(__fsub_rn(uv.y, rf), inv_tile)), 0.f);
        const float y1 = fminf(floorf(__fmul_rn(__fadd_rn(uv.y, rf), inv_tile)), (float)(c.TY - 1));
        if (x0 <= x1 && y0 <= y1) area = (uint32_t)((int)(x1 - x0) + 1) * (uint32_t)((int)(y1 - y0) + 1);
    }
    ntiles[i] = area;
}

// ---------------------------------------------------------------- K3 emit

__global__ void __launch_bounds__(256) k_emit_keys(ViewBatch vb, ProjView p, const uint32_t *ntiles,
                                                   const uint32_t *offsets, uint64_t *keys, uint32_t *vals,
                                                   uint64_t capacity, const unsigned long long *total,
                                                   DevStatus *status, uint32_t *count_out)
{
    const int64_t n = (int64_t)vb.B * p.N;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const unsigned long long F = *total;
    if (i == 0) {
        status->needed = F;
        status->counters[0] = F;
        status->counters[1] = 0ull;
        status->counters[2] = 0ull;
        status->counters[4] = 0ull;
        if (F > capacity) {
            atomicCAS(&status->code, 0, (int)GS_ERR_CAPACITY);
            *count_out = 0u;
        } else {
            *count_out = (uint32_t)F;
        }
    }
    if (F > capacity || i >= n) return;
    const uint32_t cnt = ntiles[i];
    if (cnt == 0) return;
    const int v = (int)(i / p.N);
    const uint32_t g = (uint32_t)(i - (int64_t)v * p.N);
    const ViewCam &c = vb.v[v];
    const float2 uv = p.xy[i];
    const float rf = (float)p.radius[i];
    const float inv_tile = 1.f / (float)vb.tile;
    int x0 = (int)fmaxf(floorf(__fmul_rn(__fsub_rn(uv.x, rf), inv_tile)), 0.f);
    int x1 = (int)fminf(floorf(__fmul_rn(__fadd_rn(uv.x, rf), inv_tile)), (float)(c.TX - 1));
    int y0 = (int)fmaxf(floorf(__fmul_rn(__fsub_rn(uv.y, rf), inv_tile)), 0.f);
    int y1 = (int)fminf(floorf(__fmul_rn(__fadd_rn(uv.y, rf), inv_tile)), (float)(c.TY - 1));
    const uint32_t dbits = __float_as_uint(p.rgb_d[i].w);
    uint64_t o = offsets[i];
    for (int ty = y0; ty <= y1; ++ty)
        for (int tx = x0; tx <= x1; ++tx) {
            const uint64_t tid = (uint64_t)c.tile_base + (uint64_t)ty * c.TX + tx;
            keys[o] = (tid << 32) | dbits;
            vals[o] = g;
            ++o;
        }
}

// ---------------------------------------------------------------- K4 radix sort (one-sweep)
//
// LSD radix sort on 8-bit digits of the 64-bit keys (only the digits that can
// be nonzero: 4 depth bytes + the tile-id bytes), stable, so equal keys keep
// the emission order (ascending Gaussian index).  An upfront kernel
// histograms every digit position in one read of the keys; each pass is then
// a single kernel: a CTA takes the next tile of RS_TILE keys (tile order =
// launch order, from an atomic counter), ranks its keys stably in shared
// memory, publishes its per-digit counts, and finds the keys of all earlier
// tiles with the same digit by a decoupled look-back over their published
// counts, so each pass reads and writes the keys once.

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_WARP_KEYS = 32 * RS_ITEMS;         // 512 consecutive keys per warp
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;      // 4096 keys per tile
constexpr int RS_MAX_PASSES = 8;
constexpr uint32_t LB_AGG = 1u << 30;               // look-back flag: tile count available
constexpr uint32_t LB_PRE = 2u << 30;               // look-back flag: inclusive prefix available
constexpr uint32_t LB_VAL = (1u << 30) - 1u;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;

__global__ void __launch_bounds__(RS_THREADS) k_digit_hist(const uint64_t *keys, const uint32_t *count, int passes,
                                                           uint32_t *ghist)
{
    __shared__ uint32_t h[RS_MAX_PASSES][256];
    for (int i = threadIdx.x; i < RS_MAX_PASSES * 256; i += RS_THREADS) h[i / 256][i % 256] = 0u;
    __syncthreads();
    const uint32_t n = *count;
    for (uint64_t i = blockIdx.x * (uint64_t)RS_THREADS + threadIdx.x; i < n; i += (uint64_t)gridDim.x * RS_THREADS) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += RS_THREADS) {
        const uint32_t c = h[i / 256][i % 256];
        if (c) atomicAdd(&ghist[i], c);
    }
}

// Exclusive scan of each pass's 256 digit counts (one CTA per pass).
__global__ void __launch_bounds__(256) k_digit_offsets(uint32_t *ghist)
{
    __shared__ uint32_t sw[33];
    uint32_t *h = ghist + 256 * blockIdx.x;
    const uint32_t x = h[threadIdx.x];
    uint32_t excl;
    block_excl_scan(x, excl, sw);
    h[threadIdx.x] = excl;
}

// Ranking: warp w owns the 512 consecutive keys t0 + w*512 + [0, 512), item i
// of lane l being key t0 + w*512 + 32 i + l.  Items are ranked in order with
// __match_any_sync against per-warp running digit counts, so ranks are stable
// within the warp; one block-wide prefix over the warps' counts then orders
// the warps.  Two block barriers per 4096-key tile.
__global__ void __launch_bounds__(RS_THREADS) k_onesweep(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                                         uint32_t *vout, const uint32_t *count, int shift,
                                                         const uint32_t *doff, uint32_t *look, uint32_t *tile_ctr,
                                                         DevStatus *status)
{
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t s_tile;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t n = *count;
    if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
#pragma unroll
    for (int j = 0; j < 8; ++j) wcnt[w][lane + 32 * j] = 0u;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t t0 = (uint64_t)tile * RS_TILE;
    if (t0 >= n) return;
    const uint32_t lt = lanemask_lt();
    const uint64_t wb = t0 + (uint64_t)w * RS_WARP_KEYS;
    uint64_t key[RS_ITEMS];
    uint32_t val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t idx = wb + 32 * i + lane;
        const bool valid = idx < n;
        key[i] = valid ? kin[idx] : 0ull;
        val[i] = valid ? vin[idx] : 0u;
    }
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const bool valid = wb + 32 * i + lane < n;
        const uint32_t d = valid ? ((uint32_t)(key[i] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t base = valid ? wcnt[w][d] : 0u;
        rank[i] = base + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0u) wcnt[w][d] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // digit t: exclusive prefix over the warps, tile count, look-back over earlier tiles
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < RS_WARPS; ++j) {
        const uint32_t c = wcnt[j][t];
        wcnt[j][t] = mine;
        mine += c;
    }
    uint32_t *lk = look + (size_t)tile * 256 + t;
    if (tile == 0) {
        atomicExch(lk, LB_PRE | mine);
        gbase[t] = doff[t];
    } else {
        atomicExch(lk, LB_AGG | mine);
        uint32_t excl = 0;
        bool timed_out = false;
        for (int64_t pt = (int64_t)tile - 1; pt >= 0; --pt) {
            const volatile uint32_t *q = look + (size_t)pt * 256 + t;
            uint32_t v = *q, spins = 0;
            while ((v & (LB_AGG | LB_PRE)) == 0u) {
                if (++spins > LB_SPIN_LIMIT) {       // give up: report instead of hanging
                    atomicCAS(&status->code, 0, (int)GS_ERR_TIMEOUT);
                    timed_out = true;
                    break;
                }
                v = *q;
            }
            excl += v & LB_VAL;
            if ((v & LB_PRE) || timed_out) break;
        }
        atomicExch(lk, LB_PRE | (excl + mine));
        gbase[t] = doff[t] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t idx = wb + 32 * i + lane;
        if (idx < n) {
            const uint32_t d = (uint32_t)(key[i] >> shift) & 255u;
            const uint32_t dst = gbase[d] + wcnt[w][d] + rank[i];
            kout[dst] = key[i];
            vout[dst] = val[i];
        }
    }
}

// ---------------------------------------------------------------- K5 ranges

__global__ void __launch_bounds__(256) k_tile_ranges(const uint64_t *keys, const uint32_t *count, uint2 *ranges,
                                                     uint32_t total_tiles)
{
    const uint32_t n = *count;
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t tile = (uint32_t)(keys[i] >> 32);
    if (tile >= total_tiles) return;
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[tile].x = (uint32_t)i;
    if (i + 1 == n || (uint32_t)(keys[i + 1] >> 32) != tile) ranges[tile].y = (uint32_t)(i + 1);
}

}  // namespace

size_t scan_temp_bytes(int64_t n)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(nb + 1) * sizeof(uint32_t) + 64;
}

void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *total, void *temp,
                           cudaStream_t st)
{
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(unsigned long long), st);
        return;
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t *bs = reinterpret_cast<uint32_t *>(temp);
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, bs);
    k_scan_blocks<<<1, 1024, 0, st>>>(bs, nb, total);
    k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, bs);
    count_launches(3);
}

void launch_count_tiles(const ViewBatch &vb, const ProjView &p, uint32_t *ntiles, cudaStream_t st)
{
    const int64_t n = (int64_t)vb.B * p.N;
    if (n <= 0) return;
    k_count_tiles<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(vb, p, ntiles);
    count_launches(1);
}

void launch_emit_keys(const ViewBatch &vb, const ProjView &p, const uint32_t *ntiles, const uint32_t *offsets,
                       uint64_t *keys, uint32_t *vals, uint64_t capacity, const unsigned long long *total,
                       DevStatus *status, uint32_t *count_out, cudaStream_t st)
{
    const int64_t n = (int64_t)vb.B * p.N;
    const int64_t blocks = n > 0 ? (n + 255) / 256 : 1;
    k_emit_keys<<<(unsigned)blocks, 256, 0, st>>>(vb, p, ntiles, offsets, keys, vals, capacity, total, status,
                                                 count_out);
    count_launches(1);
}

size_t sort_temp_bytes(uint64_t capacity)
{
    const uint64_t tiles = capacity > 0 ? (capacity + RS_TILE - 1) / RS_TILE : 1;
    // digit offsets (passes x 256), tile counters, look-back words (tiles x 256)
    return (size_t)RS_MAX_PASSES * 256 * 4 + 256 + (size_t)tiles * 256 * 4 + 256;
}

void launch_radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t capacity,
                       const uint32_t *count, int high_bits, void *temp, DevStatus *status, cudaStream_t st)
{
    if (capacity == 0) return;
    const int passes = 4 + (high_bits + 7) / 8;
    const uint64_t tiles = (capacity + RS_TILE - 1) / RS_TILE;
    char *tp = reinterpret_cast<char *>(temp);
    uint32_t *ghist = reinterpret_cast<uint32_t *>(tp);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(tp + (size_t)RS_MAX_PASSES * 256 * 4);
    uint32_t *look = reinterpret_cast<uint32_t *>(tp + (size_t)RS_MAX_PASSES * 256 * 4 + 256);
    cudaMemsetAsync(tp, 0, (size_t)RS_MAX_PASSES * 256 * 4 + 256, st);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t hb = (capacity + RS_THREADS * 16 - 1) / (RS_THREADS * 16);
    if (hb > (uint64_t)sms * 8) hb = (uint64_t)sms * 8;
    k_digit_hist<<<(unsigned)(hb ? hb : 1), RS_THREADS, 0, st>>>(keys, count, passes, ghist);
    k_digit_offsets<<<passes, 256, 0, st>>>(ghist);
    count_launches(2);
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int ps = 0; ps < passes; ++ps) {
        cudaMemsetAsync(look, 0, (size_t)tiles * 256 * 4, st);
        k_onesweep<<<(unsigned)tiles, RS_THREADS, 0, st>>>(ki, vi, ko, vo, count, 8 * ps, ghist + 256 * ps, look,
                                                           ctr + ps, status);
        count_launches(1);
        uint64_t *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
}

void launch_tile_ranges(const uint64_t *keys, const uint32_t *count, uint64_t capacity, uint2 *ranges,
                        uint32_t total_tiles, cudaStream_t st)
{
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st);
    if (capacity == 0) return;
    const uint64_t blocks = (capacity + 255) / 256;
    k_tile_ranges<<<(unsigned)blocks, 256, 0, st>>>(keys, count, ranges, total_tiles);
    count_launches(1);
}

}  // namespace gs
