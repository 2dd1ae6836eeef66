// C ABI of libgs (declared in include/gs.h): argument checks, the context and
// its scratch memory, and the sequencing of the kernels of one training
// iteration (Sec. 2.1 steps 1-3 + backward, Sec. 4 Adam).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>
#include <vector>

#include "gs_internal.cuh"

using namespace gs;

namespace gs {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
// Allocation-failure injection (gs_debug_fail_alloc): -1 off; n >= 0: that
// many more device allocations succeed, the next one fails with GS_ERR_OOM.
static std::atomic<long long> g_fail_alloc_after{-1};
}  // namespace gs

namespace {

struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
    bool in_ws = false;    // carved from the caller's workspace (not freed by the library)
};

}  // namespace

struct gs_ctx {
    gs_hparams hp;
    DevStatus *status = nullptr;       // device
    long long *dstep = nullptr;        // device step counter (step == 0 calls)
    DevStatus *h_status = nullptr;     // pinned host mirror
    char err[512];
    // binning scratch
    DBuf ntiles, offsets, scan_tmp, total, keys_alt, vals_alt, sort_tmp;
    DBuf pk, pv, pk_alt, pv_alt;   // (view, Gaussian) pairs sorted by depth
    DBuf rect;                     // their tile rectangles
    DBuf kmask;                    // their kept tiles (bits of the rectangle), in depth order
    DBuf rmask;                    // rectangle and kept tiles per pair, in index order
    // iteration scratch (gs_train_step / gs_render)
    DBuf xy, conic_o, rgb_d, radius, g_proj, keys, vals, ranges, count;
    DBuf img, dimg, T_final, n_contrib, maps, acc;
    DBuf tile_order;               // blending launch order (tiles) + 64 words of counters
    DBuf vis;                      // visible-only Adam: one byte per Gaussian
    DBuf order_tmp;                // gs_spatial_order: Morton keys, sort buffers
    DBuf dens_cnt, dens_off;       // gs_densify: output counts and their offsets
    DBuf tile_cost, tile_excl;     // Algorithm 1 schedule: measured cost per tile, its prefix sums
    DBuf div_f, div_b, div_tot;    // division points of the forward / backward ranges, a total
    DBuf pool_q;                   // persistent pool schedule: queue counters (forward, backward)
    uint32_t cost_tiles = 0;       // tiles the cost buffer describes (0: nothing measured yet)
    float *dacc = nullptr;         // densification statistics (caller-owned), see gs_set_densify_stats
    uint32_t *dcnt = nullptr;
    int64_t dN = 0;
    uint64_t frag_cap = 0;
    bool count_work = false;       // gs_count_work: the backward counts walked and blended pairs
    // caller workspace (gs_set_workspace): scratch is carved from [ws, ws +
    // ws_bytes) in order, ws_used so far; a dry run only adds up what would be
    // carved (gs_workspace_size)
    char *ws = nullptr;
    size_t ws_bytes = 0, ws_used = 0;
    bool dry = false;
    // tracing: events around the stages of gs_train_step
    int trace_max = 0, trace_step = 0;
    bool trace_on = false;
    std::vector<cudaEvent_t> trace_ev;
};

namespace {

gs_status fail(gs_ctx *c, gs_status s, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return s;
}

gs_status cuda_check(gs_ctx *c, const char *where)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    return GS_OK;
}

// True when the allocation-failure injection says this allocation fails.
bool injected_alloc_failure()
{
    long long n = g_fail_alloc_after.load();
    while (n >= 0) {
        if (n == 0) {
            g_fail_alloc_after.store(-1);   // one failure, then off again
            return true;
        }
        if (g_fail_alloc_after.compare_exchange_weak(n, n - 1)) return false;
    }
    return false;
}

// cudaMalloc through the injection point; out-of-memory and injected failures
// give GS_ERR_OOM, other CUDA errors GS_ERR_CUDA.
gs_status device_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_alloc_failure()) return GS_ERR_OOM;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) return GS_OK;
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

void release(DBuf &b)
{
    if (b.p && !b.in_ws) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    b.in_ws = false;
}

// Grows b to hold `bytes` (plus an eighth, rounded to 256 bytes): from
// cudaMalloc, or carved from the caller's workspace (a grown buffer's old
// region is not reused), or, in a dry run, only counted.
gs_status ensure(gs_ctx *c, DBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return GS_OK;
    release(b);
    const size_t nb = ((bytes + bytes / 8) + 255) & ~(size_t)255;
    if (c->dry) {
        c->ws_used += nb;
        b.cap = nb;
        return GS_OK;
    }
    if (c->ws) {
        if (nb > c->ws_bytes - c->ws_used)
            return fail(c, GS_ERR_OOM, "workspace of %zu bytes too small: %zu more needed", c->ws_bytes,
                        nb - (c->ws_bytes - c->ws_used));
        b.p = c->ws + c->ws_used;
        b.in_ws = true;
        c->ws_used += nb;
        b.cap = nb;
        return GS_OK;
    }
    const gs_status r = device_alloc(&b.p, nb);
    if (r != GS_OK) return fail(c, r, "device allocation of %zu bytes failed", nb);
    b.cap = nb;
    return GS_OK;
}

template <class T> T *ptr(DBuf &b) { return reinterpret_cast<T *>(b.p); }

bool finite_f(float x) { return std::isfinite(x); }

int ilog2_exact(int t) { return t == 8 ? 3 : t == 16 ? 4 : t == 32 ? 5 : -1; }

int bits_for(uint32_t n)   // bits needed to hold values 0 .. n-1
{
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < (uint64_t)n) ++b;
    return b;
}

// Validates host cameras and builds the kernel-parameter view batch.
gs_status make_views(gs_ctx *c, const gs_camera *cams, int32_t B, ViewBatch &vb, bool uniform)
{
    if (!cams) return fail(c, GS_ERR_INVALID_ARG, "cams is NULL");
    if (B < 1 || B > GS_MAX_VIEWS) return fail(c, GS_ERR_INVALID_ARG, "B=%d outside 1..%d", B, GS_MAX_VIEWS);
    memset(&vb, 0, sizeof vb);
    vb.B = B;
    vb.tile = c->hp.tile;
    vb.log2_tile = ilog2_exact(c->hp.tile);
    uint64_t base = 0;
    for (int v = 0; v < B; ++v) {
        const gs_camera &k = cams[v];
        if (k.W < 1 || k.H < 1 || k.W > 65536 || k.H > 65536)
            return fail(c, GS_ERR_INVALID_ARG, "view %d: bad size %dx%d", v, k.W, k.H);
        if (!(k.near_z > 0.f) || !(k.fx > 0.f) || !(k.fy > 0.f))
            return fail(c, GS_ERR_INVALID_ARG, "view %d: near_z, fx, fy must be > 0", v);
        bool ok = finite_f(k.fx) && finite_f(k.fy) && finite_f(k.cx) && finite_f(k.cy) && finite_f(k.near_z);
        for (int i = 0; i < 9; ++i) ok = ok && finite_f(k.R[i]);
        for (int i = 0; i < 3; ++i) ok = ok && finite_f(k.t[i]);
        if (!ok) return fail(c, GS_ERR_INVALID_ARG, "view %d: non-finite camera", v);
        if (uniform && (k.W != cams[0].W || k.H != cams[0].H))
            return fail(c, GS_ERR_INVALID_ARG, "view %d: all views of this call must share W and H", v);
        ViewCam &o = vb.v[v];
        memcpy(o.R, k.R, sizeof o.R);
        memcpy(o.t, k.t, sizeof o.t);
        o.fx = k.fx; o.fy = k.fy; o.cx = k.cx; o.cy = k.cy;
        o.near_z = k.near_z;
        o.limx = 1.3f * (0.5f * (float)k.W / k.fx);
        o.limy = 1.3f * (0.5f * (float)k.H / k.fy);
        for (int i = 0; i < 3; ++i)
            o.C[i] = -(k.R[0 * 3 + i] * k.t[0] + k.R[1 * 3 + i] * k.t[1] + k.R[2 * 3 + i] * k.t[2]);
        o.W = k.W; o.H = k.H;
        o.TX = (k.W + c->hp.tile - 1) / c->hp.tile;
        o.TY = (k.H + c->hp.tile - 1) / c->hp.tile;
        o.tile_base = (uint32_t)base;
        base += (uint64_t)o.TX * o.TY;
    }
    if (base >= ((uint64_t)1 << 31)) return fail(c, GS_ERR_INVALID_ARG, "too many tiles in one call");
    vb.total_tiles = (uint32_t)base;
    return GS_OK;
}

void set_images(ViewBatch &vb, float *img, float *T_final, uint32_t *n_contrib, const float *d_img)
{
    for (int v = 0; v < vb.B; ++v) {
        const int64_t hw = (int64_t)vb.v[v].W * vb.v[v].H;
        vb.v[v].img = img ? img + 3 * hw * v : nullptr;
        vb.v[v].T_final = T_final ? T_final + hw * v : nullptr;
        vb.v[v].n_contrib = n_contrib ? n_contrib + hw * v : nullptr;
        vb.v[v].d_img = d_img ? d_img + 3 * hw * v : nullptr;
    }
}

bool scene_ok(const gs_scene *s)
{
    if (!s || s->N < 0 || s->sh_degree < 0 || s->sh_degree > 3) return false;
    if (s->N == 0) return true;
    if (!s->mo || !s->ls || !s->q || !s->sh) return false;
    const uintptr_t a = (uintptr_t)s->mo | (uintptr_t)s->ls | (uintptr_t)s->q | (uintptr_t)s->sh;
    return (a & 15) == 0;
}

SceneView view_of(const gs_scene *s)
{
    return SceneView{reinterpret_cast<const float4 *>(s->mo), reinterpret_cast<const float4 *>(s->ls),
                     reinterpret_cast<const float4 *>(s->q), reinterpret_cast<const float4 *>(s->sh), s->N,
                     s->sh_degree};
}

SceneMut mut_of(gs_scene *s)
{
    return SceneMut{reinterpret_cast<float4 *>(s->mo), reinterpret_cast<float4 *>(s->ls),
                    reinterpret_cast<float4 *>(s->q), reinterpret_cast<float4 *>(s->sh), s->N};
}

ProjView proj_of(const gs_proj *p)
{
    return ProjView{reinterpret_cast<float2 *>(p->xy), reinterpret_cast<float4 *>(p->conic_o),
                    reinterpret_cast<float4 *>(p->rgb_d), p->radius, p->N};
}

BlendParams blend_of(const gs_ctx *c, uint64_t list_cap)
{
    const gs_hparams &hp = c->hp;
    return BlendParams{hp.alpha_min, hp.alpha_max, hp.T_min, {hp.bg[0], hp.bg[1], hp.bg[2]},
                       (uint32_t)(list_cap < 0xffffffffull ? list_cap : 0xffffffffull), c->count_work ? 1 : 0};
}

cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

constexpr int NSTAGE = GS_TRACE_STAGES;

// Records the boundary event `k` (0 .. NSTAGE) of the current traced step.
void mark(gs_ctx *c, cudaStream_t st, int k)
{
    if (c->trace_on) cudaEventRecord(c->trace_ev[(size_t)c->trace_step * (NSTAGE + 1) + k], st);
}

void trace_free(gs_ctx *c)
{
    for (cudaEvent_t e : c->trace_ev) cudaEventDestroy(e);
    c->trace_ev.clear();
    c->trace_max = 0;
    c->trace_step = 0;
    c->trace_on = false;
}

// Bins the fragments of `p` into (vals, ranges, count) in depth order; the
// fragments' tile ids stay in c->keys.  rect_ready: c->rect and c->ntiles
// already hold the pairs' tile rectangles and counts (the transformation
// kernel wrote them).  With keys64 non-null it also writes the public 64-bit
// keys (tile id << 32 | depth bits).
gs_status run_binning(gs_ctx *c, const ViewBatch &vb, const ProjView &p, bool rect_ready, uint64_t *keys64,
                      uint32_t *vals, uint2 *ranges, uint32_t *count, uint64_t capacity, cudaStream_t st)
{
    const int64_t n = (int64_t)vb.B * p.N;
    if ((uint64_t)n > GS_MAX_FRAGMENTS) return fail(c, GS_ERR_INVALID_ARG, "B*N above 2^30-1 (view, Gaussian) pairs");
    const size_t n1 = (size_t)(n > 0 ? n : 1);
    const uint64_t cap1 = capacity ? capacity : 1;
    gs_status r;
    if ((r = ensure(c, c->offsets, 4 * n1)) || (r = ensure(c, c->scan_tmp, scan_temp_bytes(n))) ||
        (r = ensure(c, c->ntiles, 4 * n1)) ||
        (r = ensure(c, c->total, 64)) || (r = ensure(c, c->pk, 4 * n1)) || (r = ensure(c, c->pv, 4 * n1)) ||
        (r = ensure(c, c->pk_alt, 4 * n1)) || (r = ensure(c, c->pv_alt, 4 * n1)) || (r = ensure(c, c->rect, 8 * n1)) ||
        (r = ensure(c, c->kmask, 8 * n1)) || (r = ensure(c, c->rmask, 16 * n1)) ||
        (r = ensure(c, c->keys, 4 * (size_t)cap1)) || (r = ensure(c, c->keys_alt, 4 * (size_t)cap1)) ||
        (r = ensure(c, c->vals_alt, 4 * (size_t)cap1)) || (r = ensure(c, c->sort_tmp, sort_temp_bytes((uint64_t)n, capacity))))
        return r;
    const int high = bits_for(vb.total_tiles);
    const bool even = fragment_sort_passes(high) % 2 == 0;
    auto *total = ptr<unsigned long long>(c->total);
    uint32_t *n_vis = reinterpret_cast<uint32_t *>(ptr<char>(c->total) + 8);
    uint32_t *pk = ptr<uint32_t>(c->pk), *pv = ptr<uint32_t>(c->pv), *pk_alt = ptr<uint32_t>(c->pk_alt);
    uint2 *rect = ptr<uint2>(c->rect);
    uint32_t *tk = ptr<uint32_t>(c->keys), *tk_alt = ptr<uint32_t>(c->keys_alt), *v_alt = ptr<uint32_t>(c->vals_alt);
    // a training step or a render culled footprint tiles against the alpha
    // ellipse in the transformation kernel (rect_ready); gs_bin keeps whole rectangles
    const float cull_alpha = rect_ready ? c->hp.alpha_min : 0.f;
    uint4 *rm = cull_alpha > 0.f ? ptr<uint4>(c->rmask) : nullptr;
    uint2 *keep = ptr<uint2>(c->kmask);
    // (1) the visible (view, Gaussian) pairs in depth order
    uint32_t *order = launch_depth_order(vb, p, rect_ready, rect, ptr<uint32_t>(c->ntiles), pk, pv, pk_alt,
                                         ptr<uint32_t>(c->pv_alt), ptr<uint32_t>(c->offsets), n_vis, total,
                                         c->scan_tmp.p, c->sort_tmp.p, c->status, st);
    // (2) their rectangles and tile counts in that order (in the sort's dead
    // buffers), counts scanned into fragment offsets
    uint32_t *counts = order == pv ? pk : pv;
    uint32_t *rx = order == pv ? ptr<uint32_t>(c->pv_alt) : pk, *ry = pk_alt;
    launch_gather_counts(order, rect, ptr<uint32_t>(c->ntiles), rm, n, n_vis, counts, rx, ry, keep, st);
    launch_exclusive_scan(counts, ptr<uint32_t>(c->offsets), n, total, c->scan_tmp.p, st, n_vis);
    mark(c, st, 2);
    // (3) fragments pair by pair in depth order, into the buffers the tile sort ends in
    launch_emit_keys(vb, p.N, n_vis, order, rx, ry, keep, ptr<uint32_t>(c->offsets), even ? tk : tk_alt,
                     even ? vals : v_alt, capacity, total, c->status, count, cull_alpha, st);
    mark(c, st, 3);
    // (4) stable sort on the tile id
    launch_sort_fragments(even ? tk : tk_alt, even ? vals : v_alt, even ? tk_alt : tk, even ? v_alt : vals, capacity,
                          count, high, c->sort_tmp.p, c->status, st);
    mark(c, st, 4);
    launch_tile_ranges(tk, count, capacity, ranges, vb.total_tiles, st);
    if (keys64) launch_compose_keys(vb, p.N, tk, vals, count, capacity, p.rgb_d, keys64, st);
    mark(c, st, 5);
    return cuda_check(c, "binning");
}

// Iteration scratch for B views of N Gaussians with a fragment capacity.
gs_status ensure_iter(gs_ctx *c, int64_t N, const ViewBatch &vb, uint64_t cap)
{
    const size_t n = (size_t)vb.B * (size_t)(N > 0 ? N : 1);
    size_t pix = 0;
    for (int v = 0; v < vb.B; ++v) pix += (size_t)vb.v[v].W * vb.v[v].H;
    gs_status r;
    if ((r = ensure(c, c->xy, 8 * n)) || (r = ensure(c, c->conic_o, 16 * n)) || (r = ensure(c, c->rgb_d, 16 * n)) ||
        (r = ensure(c, c->radius, 4 * n)) || (r = ensure(c, c->ntiles, 4 * n)) || (r = ensure(c, c->offsets, 4 * n)) ||
        (r = ensure(c, c->pk, 4 * n)) || (r = ensure(c, c->pv, 4 * n)) || (r = ensure(c, c->pk_alt, 4 * n)) ||
        (r = ensure(c, c->pv_alt, 4 * n)) || (r = ensure(c, c->rect, 8 * n)) || (r = ensure(c, c->kmask, 8 * n)) ||
        (r = ensure(c, c->rmask, 16 * n)) ||
        (r = ensure(c, c->scan_tmp, scan_temp_bytes((int64_t)n))) || (r = ensure(c, c->total, 64)) ||
        (r = ensure(c, c->keys_alt, 4 * (size_t)(cap ? cap : 1))) || (r = ensure(c, c->vals_alt, 4 * (size_t)(cap ? cap : 1))) ||
        (r = ensure(c, c->sort_tmp, sort_temp_bytes((uint64_t)n, cap))))
        return r;
    if ((r = ensure(c, c->keys, 4 * (size_t)(cap ? cap : 1))) || (r = ensure(c, c->vals, 4 * (size_t)(cap ? cap : 1))) ||
        (r = ensure(c, c->ranges, 8 * (size_t)vb.total_tiles)) || (r = ensure(c, c->count, 64)) ||
        (r = ensure(c, c->tile_order, 4 * ((size_t)vb.total_tiles + 64))))
        return r;
    if ((r = ensure(c, c->T_final, 4 * pix)) || (r = ensure(c, c->n_contrib, 4 * pix))) return r;
    if (c->hp.schedule == 1 || c->hp.schedule == 2) {
        const size_t T = (size_t)vb.total_tiles + 1;
        const size_t P = (size_t)blend_resident_ctas(c->hp.tile, c->hp.smem_batch, c->hp.px_per_thread, true) +
                         blend_resident_ctas(c->hp.tile, c->hp.smem_batch, c->hp.px_per_thread, false) + 1;
        const void *had = c->tile_cost.p;
        if ((r = ensure(c, c->tile_cost, 4 * T)) != GS_OK) return r;
        if (c->tile_cost.p != had) c->cost_tiles = 0;   // a new buffer holds no measurements
        if ((r = ensure(c, c->tile_excl, 4 * T)) ||
            (r = ensure(c, c->div_f, 4 * P)) || (r = ensure(c, c->div_b, 4 * P)) || (r = ensure(c, c->div_tot, 64)) ||
            (r = ensure(c, c->pool_q, 64)) ||
            (r = ensure(c, c->scan_tmp, scan_temp_bytes((int64_t)T))))
            return r;
    }
    return GS_OK;
}

// Launch order of the blending kernels' tiles (launch_tile_order), or null
// when index order is as fast; the context's buffer must hold the batch's
// tiles (ensure_iter).
const uint32_t *tile_order_for(gs_ctx *c, const ViewBatch &vb, const uint2 *ranges, cudaStream_t st)
{
    if (!tile_order_pays(vb.total_tiles) || c->tile_order.cap < 4 * ((size_t)vb.total_tiles + 64)) return nullptr;
    uint32_t *order = ptr<uint32_t>(c->tile_order);
    launch_tile_order(ranges, vb.total_tiles, order, order + vb.total_tiles, st);
    return order;
}

gs_status ensure_train(gs_ctx *c, int64_t N, const ViewBatch &vb)
{
    const size_t n = (size_t)vb.B * (size_t)(N > 0 ? N : 1);
    const size_t pix = (size_t)vb.B * vb.v[0].W * vb.v[0].H;
    gs_status r;
    if ((r = ensure(c, c->g_proj, 48 * n)) != GS_OK) return r;
    if (c->hp.sparse_adam && (r = ensure(c, c->vis, (size_t)(N > 0 ? N : 1))) != GS_OK) return r;
    if ((r = ensure(c, c->img, 12 * pix)) || (r = ensure(c, c->dimg, 12 * pix)) || (r = ensure(c, c->maps, 36 * pix)) ||
        (r = ensure(c, c->acc, 16 * (size_t)vb.B + 64)))
        return r;
    return GS_OK;
}

// Reads the fragment total of the scan just issued on `st` (synchronises).
gs_status read_total(gs_ctx *c, cudaStream_t st, uint64_t *F)
{
    unsigned long long h = 0;
    if (cudaMemcpyAsync(&c->h_status->needed, c->total.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_check(c, "read_total");
    h = c->h_status->needed;
    *F = h;
    return GS_OK;
}

AdamArgs adam_args(const gs_hparams &hp, int64_t step, int32_t B, long long *dstep)
{
    AdamArgs a;
    a.dstep = step == 0 ? dstep : nullptr;
    a.vis = nullptr;
    if (step == 0) step = 1;   // placeholders; the kernel computes the corrections
    const double b1 = hp.scale_beta_pow_b ? pow((double)hp.beta1, B) : hp.beta1;
    const double b2 = hp.scale_beta_pow_b ? pow((double)hp.beta2, B) : hp.beta2;
    const double lf = hp.scale_lr_sqrt_b ? sqrt((double)B) : 1.0;
    a.b1 = (float)b1;
    a.b2 = (float)b2;
    a.eps = hp.eps;
    a.bc1 = (float)(1.0 - pow(b1, (double)step));
    a.bc2 = (float)(1.0 - pow(b2, (double)step));
    const float lm = (float)(hp.lr[0] * lf), lsc = (float)(hp.lr[1] * lf), lq = (float)(hp.lr[2] * lf);
    const float lo = (float)(hp.lr[3] * lf), ldc = (float)(hp.lr[4] * lf), lrest = (float)(hp.lr[5] * lf);
    const float planes[3][4] = {{lm, lm, lm, lo}, {lsc, lsc, lsc, 0.f}, {lq, lq, lq, lq}};
    for (int p = 0; p < 3; ++p)
        for (int l = 0; l < 4; ++l) a.lr[p][l] = planes[p][l];
    for (int p = 3; p < 15; ++p)
        for (int l = 0; l < 4; ++l) {
            const int j = 4 * (p - 3) + l;   // flat SH index; 0..2 are the DC coefficients
            a.lr[p][l] = j < 3 ? ldc : lrest;
        }
    return a;
}

gs_status check_hparams(gs_ctx *c, const gs_hparams *hp)
{
    if (ilog2_exact(hp->tile) < 0) return fail(c, GS_ERR_INVALID_ARG, "tile must be 8, 16 or 32");
    if (hp->px_per_thread != 1 && hp->px_per_thread != 2 && hp->px_per_thread != 4)
        return fail(c, GS_ERR_INVALID_ARG, "px_per_thread must be 1, 2 or 4");
    if (hp->sparse_adam != 0 && hp->sparse_adam != 1) return fail(c, GS_ERR_INVALID_ARG, "sparse_adam must be 0 or 1");
    if (hp->schedule < 0 || hp->schedule > 2) return fail(c, GS_ERR_INVALID_ARG, "schedule must be 0, 1 or 2");
    if (!blend_config_ok(hp->tile, hp->smem_batch, hp->px_per_thread))
        return fail(c, GS_ERR_INVALID_ARG,
                    "unsupported (tile, smem_batch, px_per_thread): smem_batch 32, 64 or 128 (32 or 64 with tile 32 "
                    "and one pixel per thread); four pixels per thread need tile 16 or 32");
    if (!(hp->alpha_max > 0.f && hp->alpha_max < 1.f) || !(hp->alpha_min >= 0.f) || !(hp->T_min >= 0.f))
        return fail(c, GS_ERR_INVALID_ARG, "blend thresholds out of range");
    return GS_OK;
}

}  // namespace

extern "C" {

int32_t gs_abi_version(void) { return GS_ABI_VERSION; }

uint64_t gs_kernel_launches(void) { return gs::g_launches.load(); }

gs_status gs_trace_enable(gs_ctx *c, int32_t max_steps)
{
    if (!c || max_steps < 0) return GS_ERR_INVALID_ARG;
    trace_free(c);
    if (max_steps == 0) return GS_OK;
    c->trace_ev.resize((size_t)max_steps * (NSTAGE + 1));
    for (auto &e : c->trace_ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            trace_free(c);
            return cuda_check(c, "gs_trace_enable");
        }
    c->trace_max = max_steps;
    c->trace_step = 0;
    return GS_OK;
}

gs_status gs_trace_read(gs_ctx *c, float *ms, int32_t *steps)
{
    if (!c || !ms || !steps) return GS_ERR_INVALID_ARG;
    *steps = 0;
    for (int s = 0; s < c->trace_step; ++s) {
        cudaEvent_t *e = &c->trace_ev[(size_t)s * (NSTAGE + 1)];
        if (cudaEventSynchronize(e[NSTAGE]) != cudaSuccess) return cuda_check(c, "gs_trace_read");
        for (int k = 0; k < NSTAGE; ++k) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, e[k], e[k + 1]) != cudaSuccess) return cuda_check(c, "gs_trace_read");
            ms[(size_t)s * NSTAGE + k] = t;
        }
    }
    *steps = c->trace_step;
    c->trace_step = 0;
    return GS_OK;
}

gs_status gs_default_hparams(gs_hparams *hp)
{
    if (!hp) return GS_ERR_INVALID_ARG;
    memset(hp, 0, sizeof *hp);
    hp->tile = 16;
    hp->smem_batch = 64;
    hp->px_per_thread = 1;
    hp->strict_nonfinite = 0;
    hp->alpha_min = 1.0f / 255.0f;
    hp->alpha_max = 0.99f;
    hp->T_min = 1e-4f;
    const float lr[6] = {1.6e-4f, 5e-3f, 1e-3f, 5e-2f, 2.5e-3f, 2.5e-4f};
    memcpy(hp->lr, lr, sizeof lr);
    hp->beta1 = 0.9f;
    hp->beta2 = 0.999f;
    hp->eps = 1e-15f;
    hp->scale_lr_sqrt_b = 1;
    hp->scale_beta_pow_b = 1;
    hp->lambda_dssim = 0.2f;
    return GS_OK;
}

gs_status gs_create(gs_ctx **out, const gs_hparams *hp)
{
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_ctx *c = new (std::nothrow) gs_ctx();
    if (!c) return GS_ERR_OOM;
    c->err[0] = 0;
    if (hp) c->hp = *hp; else gs_default_hparams(&c->hp);
    gs_status r = check_hparams(c, &c->hp);
    if (r != GS_OK) { delete c; return r; }
    void *st = nullptr, *ds = nullptr;
    if ((r = device_alloc(&st, sizeof(DevStatus))) == GS_OK) c->status = static_cast<DevStatus *>(st);
    if (r == GS_OK && (r = device_alloc(&ds, 2 * sizeof(long long))) == GS_OK) c->dstep = static_cast<long long *>(ds);
    if (r == GS_OK && cudaMallocHost(&c->h_status, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        c->h_status = nullptr;
        r = GS_ERR_CUDA;
    }
    if (r != GS_OK) {
        if (c->status) cudaFree(c->status);
        if (c->dstep) cudaFree(c->dstep);
        delete c;
        return r;
    }
    cudaMemset(c->status, 0, sizeof(DevStatus));
    cudaMemset(c->dstep, 0, 2 * sizeof(long long));
    memset(c->h_status, 0, sizeof(DevStatus));
    if (cudaDeviceSynchronize() != cudaSuccess) { cudaGetLastError(); }
    *out = c;
    return GS_OK;
}

gs_status gs_debug_set_lookback(uint32_t spin_limit, int32_t withhold_first_tile)
{
    set_lookback_debug(spin_limit, withhold_first_tile);
    return GS_OK;
}

gs_status gs_debug_fail_alloc(int64_t after)
{
    if (after < -1) return GS_ERR_INVALID_ARG;
    g_fail_alloc_after.store(after);
    return GS_OK;
}

// Every scratch buffer of the context.
void release_all(gs_ctx *c)
{
    DBuf *bufs[] = {&c->ntiles, &c->offsets, &c->scan_tmp, &c->total, &c->keys_alt, &c->vals_alt, &c->sort_tmp,
                    &c->pk, &c->pv, &c->pk_alt, &c->pv_alt, &c->rect, &c->kmask, &c->rmask,
                    &c->xy, &c->conic_o, &c->rgb_d, &c->radius, &c->g_proj, &c->keys,
                    &c->vals, &c->ranges, &c->count, &c->img, &c->dimg, &c->T_final, &c->n_contrib, &c->maps,
                    &c->acc, &c->tile_order, &c->vis, &c->order_tmp, &c->dens_cnt, &c->dens_off,
                    &c->tile_cost, &c->tile_excl, &c->div_f, &c->div_b, &c->div_tot, &c->pool_q};
    for (DBuf *b : bufs) release(*b);
    c->cost_tiles = 0;
}

gs_status gs_set_workspace(gs_ctx *c, void *ws, size_t bytes, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (ws && (reinterpret_cast<uintptr_t>(ws) & 255u))
        return fail(c, GS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return cuda_check(c, "gs_set_workspace");
    release_all(c);
    c->ws = static_cast<char *>(ws);
    c->ws_bytes = ws ? bytes : 0;
    c->ws_used = 0;
    return GS_OK;
}

gs_status gs_get_step(gs_ctx *c, int64_t *step, void *stream)
{
    if (!c || !step) return GS_ERR_INVALID_ARG;
    long long h = 0;
    cudaStream_t st = S(stream);
    if (cudaMemcpyAsync(&h, c->dstep, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_check(c, "gs_get_step");
    *step = (int64_t)h;
    return GS_OK;
}

gs_status gs_set_step(gs_ctx *c, int64_t step, void *stream)
{
    if (!c || step < 0) return GS_ERR_INVALID_ARG;
    const long long h = (long long)step;
    cudaStream_t st = S(stream);
    // the bias corrections next to the counter are recomputed from it by the next step's tick
    if (cudaMemcpyAsync(c->dstep, &h, sizeof h, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_check(c, "gs_set_step");
    return GS_OK;
}

gs_status gs_destroy(gs_ctx *c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    release_all(c);
    trace_free(c);
    if (c->status) cudaFree(c->status);
    if (c->dstep) cudaFree(c->dstep);
    if (c->h_status) cudaFreeHost(c->h_status);
    delete c;
    return GS_OK;
}

gs_status gs_set_hparams(gs_ctx *c, const gs_hparams *hp)
{
    if (!c || !hp) return GS_ERR_INVALID_ARG;
    gs_status r = check_hparams(c, hp);
    if (r != GS_OK) return r;
    c->hp = *hp;
    return GS_OK;
}

const char *gs_last_error(const gs_ctx *c) { return c ? c->err : "null context"; }

gs_status gs_get_status(gs_ctx *c, void *stream, int32_t *status, uint64_t *needed)
{
    if (!c || !status) return GS_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    if (cudaMemcpyAsync(c->h_status, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_check(c, "gs_get_status");
    *status = c->h_status->code;
    if (needed) *needed = c->h_status->needed;
    if (c->h_status->code != 0) {
        cudaMemsetAsync(c->status, 0, sizeof(int32_t), st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "gs_get_status clear");
    }
    return GS_OK;
}

gs_status gs_get_counters(gs_ctx *c, void *stream, uint64_t out[6])
{
    if (!c || !out) return GS_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    if (cudaMemcpyAsync(c->h_status, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_check(c, "gs_get_counters");
    out[0] = c->h_status->counters[0];
    out[1] = c->h_status->counters[1];
    out[2] = c->h_status->counters[2];
    out[3] = c->h_status->counters[4];
    out[4] = c->h_status->counters[3];
    out[5] = c->h_status->counters[5];
    return GS_OK;
}

gs_status gs_count_work(gs_ctx *c, int32_t on)
{
    if (!c) return GS_ERR_INVALID_ARG;
    c->count_work = on != 0;
    return GS_OK;
}

gs_status gs_reserve(gs_ctx *c, int64_t N, const gs_camera *cams, int32_t B, uint64_t frag_capacity)
{
    if (!c || N < 0) return GS_ERR_INVALID_ARG;
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, false);
    if (r != GS_OK) return r;
    if (frag_capacity > GS_MAX_FRAGMENTS) return fail(c, GS_ERR_INVALID_ARG, "fragment capacity above 2^30-1");
    if (frag_capacity > c->frag_cap) c->frag_cap = frag_capacity;
    if ((r = ensure_iter(c, N, vb, c->frag_cap)) != GS_OK) return r;
    bool uniform = true;
    for (int v = 1; v < B; ++v) uniform = uniform && cams[v].W == cams[0].W && cams[v].H == cams[0].H;
    if (uniform && (r = ensure_train(c, N, vb)) != GS_OK) return r;
    return GS_OK;
}

gs_status gs_workspace_size(const gs_hparams *hp, int64_t N, const gs_camera *cams, int32_t B,
                            uint64_t frag_capacity, size_t *bytes)
{
    if (!bytes || !cams || B < 1 || B > GS_MAX_VIEWS || N < 0) return GS_ERR_INVALID_ARG;
    // a dry run of gs_reserve on a context that only counts: exactly what a
    // fresh workspace gives up to gs_reserve with these sizes
    gs_ctx d;
    d.err[0] = 0;
    if (hp) d.hp = *hp; else gs_default_hparams(&d.hp);
    if (check_hparams(&d, &d.hp) != GS_OK) return GS_ERR_INVALID_ARG;
    d.dry = true;
    const gs_status r = gs_reserve(&d, N, cams, B, frag_capacity);
    if (r != GS_OK) return r;
    *bytes = d.ws_used;
    return GS_OK;
}

gs_status gs_preprocess(gs_ctx *c, const gs_scene *scene, const gs_camera *cams, int32_t B, gs_proj *out,
                        void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(scene)) return fail(c, GS_ERR_INVALID_ARG, "bad scene (null/unaligned planes or sh_degree)");
    if (!out || out->N != scene->N || out->B != B) return fail(c, GS_ERR_INVALID_ARG, "gs_proj N/B mismatch");
    if (scene->N > 0 && (!out->xy || !out->conic_o || !out->rgb_d || !out->radius))
        return fail(c, GS_ERR_INVALID_ARG, "gs_proj has null arrays");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, false);
    if (r != GS_OK) return r;
    const int64_t n = (int64_t)B * scene->N;
    if ((r = ensure(c, c->ntiles, 4 * (size_t)(n > 0 ? n : 1))) != GS_OK) return r;
    launch_preprocess_fwd(view_of(scene), vb, proj_of(out), ptr<uint32_t>(c->ntiles), nullptr, c->status,
                          c->hp.strict_nonfinite, S(stream));
    return cuda_check(c, "gs_preprocess");
}

gs_status gs_bin(gs_ctx *c, const gs_proj *proj, const gs_camera *cams, int32_t B, gs_bins *out,
                 uint64_t *needed_host, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!proj || proj->B != B || proj->N < 0) return fail(c, GS_ERR_INVALID_ARG, "bad gs_proj");
    if (!out || !out->ranges || !out->count || (out->capacity > 0 && (!out->keys || !out->vals)))
        return fail(c, GS_ERR_INVALID_ARG, "bad gs_bins");
    if (out->capacity > GS_MAX_FRAGMENTS) return fail(c, GS_ERR_INVALID_ARG, "capacity above 2^30-1");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, false);
    if (r != GS_OK) return r;
    cudaStream_t st = S(stream);
    r = run_binning(c, vb, proj_of(proj), false, out->keys, out->vals, reinterpret_cast<uint2 *>(out->ranges),
                    out->count, out->capacity, st);
    if (r != GS_OK) return r;
    if (needed_host) {
        uint64_t F = 0;
        if ((r = read_total(c, st, &F)) != GS_OK) return r;
        *needed_host = F;
        if (F > out->capacity) return fail(c, GS_ERR_CAPACITY, "need %llu fragments, capacity %llu",
                                           (unsigned long long)F, (unsigned long long)out->capacity);
    }
    return GS_OK;
}

gs_status gs_render_fwd(gs_ctx *c, const gs_proj *proj, const gs_bins *bins, const gs_camera *cams, int32_t B,
                        float *img, float *T_final, uint32_t *n_contrib, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!proj || proj->B != B || !bins || !img || !T_final || !n_contrib)
        return fail(c, GS_ERR_INVALID_ARG, "null argument");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, true);
    if (r != GS_OK) return r;
    set_images(vb, img, T_final, n_contrib, nullptr);
    const uint2 *ranges = reinterpret_cast<const uint2 *>(bins->ranges);
    if (tile_order_pays(vb.total_tiles) && (r = ensure(c, c->tile_order, 4 * ((size_t)vb.total_tiles + 64))) != GS_OK)
        return r;
    launch_blend_fwd(vb, proj_of(proj), bins->vals, ranges, blend_of(c, bins->capacity), c->hp.smem_batch, c->hp.px_per_thread,
                     c->status, tile_order_for(c, vb, ranges, S(stream)), S(stream));
    return cuda_check(c, "gs_render_fwd");
}

gs_status gs_render_bwd(gs_ctx *c, const gs_proj *proj, const gs_bins *bins, const gs_camera *cams, int32_t B,
                        const float *T_final, const uint32_t *n_contrib, const float *d_img, gs_proj_grad *out,
                        void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!proj || proj->B != B || !bins || !T_final || !n_contrib || !d_img || !out)
        return fail(c, GS_ERR_INVALID_ARG, "null argument");
    if (proj->N > 0 && (!out->d_xy_o || !out->d_conic || !out->d_rgb))
        return fail(c, GS_ERR_INVALID_ARG, "null gradient arrays");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, true);
    if (r != GS_OK) return r;
    set_images(vb, nullptr, const_cast<float *>(T_final), const_cast<uint32_t *>(n_contrib), d_img);
    cudaStream_t st = S(stream);
    const size_t bytes = 16 * (size_t)B * (size_t)proj->N;
    if (bytes) {
        cudaMemsetAsync(out->d_xy_o, 0, bytes, st);
        cudaMemsetAsync(out->d_conic, 0, bytes, st);
        cudaMemsetAsync(out->d_rgb, 0, bytes, st);
    }
    GradView gv{reinterpret_cast<float4 *>(out->d_xy_o), reinterpret_cast<float4 *>(out->d_conic),
                reinterpret_cast<float4 *>(out->d_rgb)};
    const uint2 *ranges = reinterpret_cast<const uint2 *>(bins->ranges);
    if (tile_order_pays(vb.total_tiles) && (r = ensure(c, c->tile_order, 4 * ((size_t)vb.total_tiles + 64))) != GS_OK)
        return r;
    launch_blend_bwd(vb, proj_of(proj), bins->vals, ranges, blend_of(c, bins->capacity), c->hp.smem_batch, c->hp.px_per_thread, gv,
                     c->status, tile_order_for(c, vb, ranges, st), st);
    launch_moments_to_grads(proj_of(proj), (int64_t)B * proj->N, gv, st);
    return cuda_check(c, "gs_render_bwd");
}

gs_status gs_preprocess_bwd(gs_ctx *c, const gs_scene *scene, const gs_camera *cams, int32_t B, const gs_proj *proj,
                            const gs_proj_grad *dproj, gs_scene *grad, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (B < 1) return fail(c, GS_ERR_INVALID_ARG, "B < 1");
    return gs_preprocess_bwd_scaled(c, scene, cams, B, proj, dproj, grad, 1.f / (float)B, stream);
}

gs_status gs_preprocess_bwd_scaled(gs_ctx *c, const gs_scene *scene, const gs_camera *cams, int32_t B,
                                   const gs_proj *proj, const gs_proj_grad *dproj, gs_scene *grad, float scale,
                                   void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!(scale >= 0.f) || scale == INFINITY) return fail(c, GS_ERR_INVALID_ARG, "scale must be finite and >= 0");
    if (!scene_ok(scene) || !scene_ok(grad) || grad->N != scene->N)
        return fail(c, GS_ERR_INVALID_ARG, "bad scene or gradient planes");
    if (!proj || proj->B != B || proj->N != scene->N || !dproj) return fail(c, GS_ERR_INVALID_ARG, "bad gs_proj");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, false);
    if (r != GS_OK) return r;
    GradView gv{reinterpret_cast<float4 *>(dproj->d_xy_o), reinterpret_cast<float4 *>(dproj->d_conic),
                reinterpret_cast<float4 *>(dproj->d_rgb)};
    launch_preprocess_bwd(view_of(scene), vb, proj_of(proj), gv, true, mut_of(grad), nullptr, S(stream), nullptr,
                          nullptr, nullptr, scale);
    return cuda_check(c, "gs_preprocess_bwd");
}

gs_status gs_loss(gs_ctx *c, const float *img, const float *target, int32_t B, int32_t W, int32_t H,
                  float *loss_out, float *d_img, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!img || !target || !loss_out || !d_img || B < 1 || B > GS_MAX_VIEWS || W < 1 || H < 1)
        return fail(c, GS_ERR_INVALID_ARG, "bad loss arguments");
    const size_t pix = (size_t)B * W * H;
    gs_status r;
    if ((r = ensure(c, c->maps, 36 * pix)) || (r = ensure(c, c->acc, 16 * (size_t)B + 64))) return r;
    launch_loss(img, target, B, W, H, c->hp.lambda_dssim, loss_out, d_img, ptr<float>(c->maps), ptr<double>(c->acc),
                c->status, S(stream));
    return cuda_check(c, "gs_loss");
}

gs_status gs_adam_step(gs_ctx *c, gs_scene *p, const gs_scene *g, gs_scene *m, gs_scene *v, int64_t step, int32_t B,
                       void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(p) || !scene_ok(g) || !scene_ok(m) || !scene_ok(v) || g->N != p->N || m->N != p->N ||
        v->N != p->N)
        return fail(c, GS_ERR_INVALID_ARG, "bad parameter / moment planes");
    if (step < 0 || B < 1) return fail(c, GS_ERR_INVALID_ARG, "step must be >= 0 and B >= 1");
    launch_adam(mut_of(p), view_of(g), mut_of(m), mut_of(v), adam_args(c->hp, step, B, c->dstep), c->status, S(stream));
    return cuda_check(c, "gs_adam_step");
}

gs_status gs_adam_step_sparse(gs_ctx *c, gs_scene *p, const gs_scene *g, gs_scene *m, gs_scene *v,
                              const uint8_t *visible, int64_t step, int32_t B, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(p) || !scene_ok(g) || !scene_ok(m) || !scene_ok(v) || g->N != p->N || m->N != p->N ||
        v->N != p->N)
        return fail(c, GS_ERR_INVALID_ARG, "bad parameter / moment planes");
    if (step < 0 || B < 1) return fail(c, GS_ERR_INVALID_ARG, "step must be >= 0 and B >= 1");
    if (!visible && p->N > 0) return fail(c, GS_ERR_INVALID_ARG, "visible is NULL");
    AdamArgs a = adam_args(c->hp, step, B, c->dstep);
    a.vis = visible;
    launch_adam(mut_of(p), view_of(g), mut_of(m), mut_of(v), a, c->status, S(stream));
    return cuda_check(c, "gs_adam_step_sparse");
}

gs_status gs_set_densify_stats(gs_ctx *c, float *grad_acc, uint32_t *grad_cnt, int64_t N)
{
    if (!c || N < 0 || (!grad_acc) != (!grad_cnt)) return GS_ERR_INVALID_ARG;
    c->dacc = grad_acc;
    c->dcnt = grad_cnt;
    c->dN = grad_acc ? N : 0;
    return GS_OK;
}

gs_status gs_densify(gs_ctx *c, const gs_scene *p, const gs_scene *m, const gs_scene *v, const float *grad_acc,
                     const uint32_t *grad_cnt, const float *normals, const gs_densify_params *dp, gs_scene *p_out,
                     gs_scene *m_out, gs_scene *v_out, int64_t capacity, int64_t *n_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(p) || !scene_ok(m) || !scene_ok(v) || m->N != p->N || v->N != p->N)
        return fail(c, GS_ERR_INVALID_ARG, "bad parameter / moment planes");
    if (!scene_ok(p_out) || !scene_ok(m_out) || !scene_ok(v_out) || capacity < 0 || p_out->N != capacity ||
        m_out->N != capacity || v_out->N != capacity)
        return fail(c, GS_ERR_INVALID_ARG, "output planes must hold capacity Gaussians (their N = capacity)");
    if (!dp || !n_out || (p->N > 0 && (!grad_acc || !grad_cnt || !normals)))
        return fail(c, GS_ERR_INVALID_ARG, "null statistics, normals, params or n_out");
    if (!(dp->scale_threshold > 0.f) || !(dp->min_opacity > 0.f && dp->min_opacity < 1.f) ||
        !(dp->split_div > 0.f) || !(dp->grad_threshold >= 0.f))
        return fail(c, GS_ERR_INVALID_ARG, "densify params out of range");
    if (p->N >= ((int64_t)1 << 31) || capacity >= ((int64_t)1 << 32))
        return fail(c, GS_ERR_INVALID_ARG, "N must be below 2^31 and capacity below 2^32");
    const int64_t N = p->N;
    gs_status r;
    if ((r = ensure(c, c->dens_cnt, 4 * (size_t)(N > 0 ? N : 1))) || (r = ensure(c, c->dens_off, 4 * (size_t)(N > 0 ? N : 1))) ||
        (r = ensure(c, c->scan_tmp, scan_temp_bytes(N))) || (r = ensure(c, c->total, 64)))
        return r;
    cudaStream_t st = S(stream);
    DensifyArgs d;
    d.grad_thr = dp->grad_threshold;
    // thresholds rounded once from double, so a float32 reimplementation can match them bit for bit
    d.log_scale_thr = (float)log((double)dp->scale_threshold);
    d.logit_min = (float)log((double)dp->min_opacity / (1.0 - (double)dp->min_opacity));
    d.log_div = (float)log((double)dp->split_div);
    launch_densify_count(view_of(p), grad_acc, grad_cnt, d, ptr<uint32_t>(c->dens_cnt), st);
    launch_exclusive_scan(ptr<uint32_t>(c->dens_cnt), ptr<uint32_t>(c->dens_off), N,
                          ptr<unsigned long long>(c->total), c->scan_tmp.p, st);
    launch_densify_emit(view_of(p), view_of(m), view_of(v), grad_acc, grad_cnt, normals, d,
                        ptr<uint32_t>(c->dens_off), ptr<unsigned long long>(c->total), mut_of(p_out),
                        mut_of(m_out), mut_of(v_out), st);
    if ((r = cuda_check(c, "gs_densify")) != GS_OK) return r;
    uint64_t total = 0;
    if ((r = read_total(c, st, &total)) != GS_OK) return r;
    *n_out = (int64_t)total;
    if ((int64_t)total > capacity) return fail(c, GS_ERR_CAPACITY, "densify needs %llu Gaussians, capacity %lld",
                                               (unsigned long long)total, (long long)capacity);
    return GS_OK;
}

gs_status gs_reset_opacity(gs_ctx *c, gs_scene *p, gs_scene *m, gs_scene *v, float max_opacity, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(p) || !scene_ok(m) || !scene_ok(v) || m->N != p->N || v->N != p->N)
        return fail(c, GS_ERR_INVALID_ARG, "bad parameter / moment planes");
    if (!(max_opacity > 0.f && max_opacity < 1.f)) return fail(c, GS_ERR_INVALID_ARG, "max_opacity outside (0, 1)");
    const float logit_max = (float)log((double)max_opacity / (1.0 - (double)max_opacity));
    launch_reset_opacity(mut_of(p), mut_of(m), mut_of(v), logit_max, S(stream));
    return cuda_check(c, "gs_reset_opacity");
}

gs_status gs_division_points(gs_ctx *c, const uint32_t *cost, int64_t T, int32_t P, uint32_t *div, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!cost || !div || T < 1 || T >= ((int64_t)1 << 31) || P < 1 || P > (1 << 20))
        return fail(c, GS_ERR_INVALID_ARG, "bad cost / div / T / P");
    gs_status r;
    if ((r = ensure(c, c->tile_cost, 4 * (size_t)T)) || (r = ensure(c, c->tile_excl, 4 * (size_t)T)) ||
        (r = ensure(c, c->scan_tmp, scan_temp_bytes(T))) || (r = ensure(c, c->div_tot, 64)))
        return r;
    c->cost_tiles = 0;                              // the schedule's measured costs are overwritten
    cudaStream_t st = S(stream);
    cudaMemcpyAsync(c->tile_cost.p, cost, 4 * (size_t)T, cudaMemcpyDeviceToDevice, st);
    launch_division_points(ptr<uint32_t>(c->tile_cost), (uint32_t)T, (uint32_t)P, ptr<uint32_t>(c->tile_excl),
                           c->scan_tmp.p, ptr<unsigned long long>(c->div_tot), div, st);
    return cuda_check(c, "gs_division_points");
}

gs_status gs_spatial_order(gs_ctx *c, const gs_scene *scene, uint32_t *perm, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(scene) || (scene->N > 0 && !perm)) return fail(c, GS_ERR_INVALID_ARG, "bad scene / perm");
    if (scene->N >= ((int64_t)1 << 31)) return fail(c, GS_ERR_INVALID_ARG, "N must be below 2^31");
    gs_status r;
    if ((r = ensure(c, c->order_tmp, spatial_order_temp_bytes(scene->N))) != GS_OK) return r;
    launch_spatial_order(reinterpret_cast<const float4 *>(scene->mo), scene->N, perm, c->order_tmp.p, c->status,
                         S(stream));
    return cuda_check(c, "gs_spatial_order");
}

gs_status gs_permute(gs_ctx *c, const gs_scene *src, const uint32_t *perm, gs_scene *dst, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(src) || !scene_ok(dst) || dst->N != src->N || (src->N > 0 && !perm))
        return fail(c, GS_ERR_INVALID_ARG, "bad planes / perm");
    if (src->mo == dst->mo || src->ls == dst->ls || src->q == dst->q || src->sh == dst->sh)
        return fail(c, GS_ERR_INVALID_ARG, "gs_permute works out of place");
    launch_permute(view_of(src), perm, mut_of(dst), S(stream));
    return cuda_check(c, "gs_permute");
}

gs_status gs_train_step(gs_ctx *c, gs_scene *p, gs_scene *g, gs_scene *m, gs_scene *v, int64_t step,
                        const gs_camera *cams, int32_t B, const float *targets, float *loss_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(p) || !scene_ok(g) || !scene_ok(m) || !scene_ok(v) || g->N != p->N || m->N != p->N ||
        v->N != p->N)
        return fail(c, GS_ERR_INVALID_ARG, "bad parameter / moment planes");
    if (!targets || !loss_out || step < 0) return fail(c, GS_ERR_INVALID_ARG, "bad targets / loss_out / step");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, true);
    if (r != GS_OK) return r;
    cudaStream_t st = S(stream);
    const int64_t N = p->N;
    const int64_t n = (int64_t)B * N;
    if ((r = ensure_iter(c, N, vb, c->frag_cap)) != GS_OK) return r;
    if ((r = ensure_train(c, N, vb)) != GS_OK) return r;
    gs_proj pr{ptr<float>(c->xy), ptr<float>(c->conic_o), ptr<float>(c->rgb_d), ptr<int32_t>(c->radius), N, B, 0};
    const ProjView pv = proj_of(&pr);
    const SceneView sv = view_of(p);
    c->trace_on = c->trace_max > 0 && c->trace_step < c->trace_max;
    mark(c, st, 0);
    launch_preprocess_fwd(sv, vb, pv, ptr<uint32_t>(c->ntiles), ptr<uint2>(c->rect), c->status,
                          c->hp.strict_nonfinite, st, ptr<uint4>(c->rmask), c->hp.alpha_min);
    mark(c, st, 1);
    if (c->frag_cap == 0) {
        // first call on this context: size the fragment buffers from an exact count
        if ((r = ensure(c, c->scan_tmp, scan_temp_bytes(n))) || (r = ensure(c, c->total, 64))) return r;
        launch_exclusive_scan(ptr<uint32_t>(c->ntiles), ptr<uint32_t>(c->offsets), n,
                              ptr<unsigned long long>(c->total), c->scan_tmp.p, st);
        uint64_t F = 0;
        if ((r = read_total(c, st, &F)) != GS_OK) return r;
        uint64_t cap = 2 * F + 4096;   // the culled count; growth during training stays inside
        if (cap > GS_MAX_FRAGMENTS) cap = GS_MAX_FRAGMENTS;
        c->frag_cap = cap;
        if ((r = ensure_iter(c, N, vb, c->frag_cap)) != GS_OK) return r;
    }
    r = run_binning(c, vb, pv, true, nullptr, ptr<uint32_t>(c->vals),
                    ptr<uint2>(c->ranges), ptr<uint32_t>(c->count), c->frag_cap, st);
    if (r != GS_OK) return r;
    set_images(vb, ptr<float>(c->img), ptr<float>(c->T_final), ptr<uint32_t>(c->n_contrib), ptr<float>(c->dimg));
    const BlendParams bp = blend_of(c, c->frag_cap);
    const uint32_t *order = nullptr, *div_f = nullptr, *div_b = nullptr;
    uint32_t *cost = nullptr, *queue = nullptr;
    if (c->hp.schedule == 1 && vb.total_tiles > 0) {
        // Algorithm 1 over the previous step's measured tile costs (list lengths before the first)
        const uint32_t T = vb.total_tiles;
        cost = ptr<uint32_t>(c->tile_cost);
        if (c->cost_tiles != T) {
            launch_list_cost(ptr<uint2>(c->ranges), T, cost, st);
            c->cost_tiles = T;
        }
        const uint32_t Pf = blend_resident_ctas(c->hp.tile, c->hp.smem_batch, c->hp.px_per_thread, false);
        const uint32_t Pb = blend_resident_ctas(c->hp.tile, c->hp.smem_batch, c->hp.px_per_thread, true);
        launch_division_points(cost, T, Pf, ptr<uint32_t>(c->tile_excl), c->scan_tmp.p,
                               ptr<unsigned long long>(c->div_tot), ptr<uint32_t>(c->div_f), st);
        launch_division_points(cost, T, Pb, ptr<uint32_t>(c->tile_excl), c->scan_tmp.p,
                               ptr<unsigned long long>(c->div_tot), ptr<uint32_t>(c->div_b), st);
        cudaMemsetAsync(cost, 0, 4 * (size_t)T, st);    // this step measures afresh
        div_f = ptr<uint32_t>(c->div_f);
        div_b = ptr<uint32_t>(c->div_b);
    } else if (c->hp.schedule == 2 && vb.total_tiles > 0) {
        // persistent pool over the previous step's measured costs, heaviest first
        const uint32_t T = vb.total_tiles;
        cost = ptr<uint32_t>(c->tile_cost);
        if (c->cost_tiles != T) {
            launch_list_cost(ptr<uint2>(c->ranges), T, cost, st);
            c->cost_tiles = T;
        }
        order = ptr<uint32_t>(c->tile_order);
        launch_tile_order(ptr<uint2>(c->ranges), T, ptr<uint32_t>(c->tile_order), ptr<uint32_t>(c->tile_order) + T,
                          st, cost);
        cudaMemsetAsync(cost, 0, 4 * (size_t)T, st);
        queue = ptr<uint32_t>(c->pool_q);               // two counters (forward, backward), zero at launch
        cudaMemsetAsync(queue, 0, 8, st);
    } else {
        order = tile_order_for(c, vb, ptr<uint2>(c->ranges), st);   // shared by both passes
    }
    launch_blend_fwd(vb, pv, ptr<uint32_t>(c->vals), ptr<uint2>(c->ranges), bp, c->hp.smem_batch, c->hp.px_per_thread,
                     c->status, order, st, div_f, cost, queue);
    mark(c, st, 6);
    launch_loss(ptr<float>(c->img), targets, B, vb.v[0].W, vb.v[0].H, c->hp.lambda_dssim, loss_out,
                ptr<float>(c->dimg), ptr<float>(c->maps), ptr<double>(c->acc), c->status, st);
    mark(c, st, 7);
    // three gradient planes of n float4 each, in one buffer: (u, v, opacity), conic, rgb
    if (n) cudaMemsetAsync(c->g_proj.p, 0, 48 * (size_t)n, st);
    mark(c, st, 8);
    float4 *gp = ptr<float4>(c->g_proj);
    const GradView gv{gp, gp + n, gp + 2 * n};
    launch_blend_bwd(vb, pv, ptr<uint32_t>(c->vals), ptr<uint2>(c->ranges), bp, c->hp.smem_batch, c->hp.px_per_thread,
                     gv, c->status, order, st, div_b, cost, queue ? queue + 1 : nullptr);
    mark(c, st, 9);
    uint8_t *vis = c->hp.sparse_adam ? ptr<uint8_t>(c->vis) : nullptr;
    const bool stats = c->dacc && c->dN == N;
    launch_preprocess_bwd(sv, vb, pv, gv, false, mut_of(g), vis, st, stats ? c->dacc : nullptr,
                          stats ? c->dcnt : nullptr, c->status);
    mark(c, st, 10);
    AdamArgs aa = adam_args(c->hp, step, B, c->dstep);
    aa.vis = vis;
    launch_adam(mut_of(p), view_of(g), mut_of(m), mut_of(v), aa, c->status, st);
    mark(c, st, 11);
    if (c->trace_on) ++c->trace_step;
    c->trace_on = false;
    return cuda_check(c, "gs_train_step");
}

gs_status gs_render(gs_ctx *c, const gs_scene *scene, const gs_camera *cams, int32_t B, float *const *imgs,
                    void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_ok(scene) || !imgs) return fail(c, GS_ERR_INVALID_ARG, "bad scene or image array");
    ViewBatch vb;
    gs_status r = make_views(c, cams, B, vb, false);
    if (r != GS_OK) return r;
    for (int v = 0; v < B; ++v)
        if (!imgs[v]) return fail(c, GS_ERR_INVALID_ARG, "imgs[%d] is NULL", v);
    cudaStream_t st = S(stream);
    const int64_t N = scene->N;
    const int64_t n = (int64_t)B * N;
    if ((r = ensure_iter(c, N, vb, c->frag_cap)) != GS_OK) return r;
    gs_proj pr{ptr<float>(c->xy), ptr<float>(c->conic_o), ptr<float>(c->rgb_d), ptr<int32_t>(c->radius), N, B, 0};
    const ProjView pv = proj_of(&pr);
    launch_preprocess_fwd(view_of(scene), vb, pv, ptr<uint32_t>(c->ntiles), ptr<uint2>(c->rect), c->status,
                          c->hp.strict_nonfinite, st, ptr<uint4>(c->rmask), c->hp.alpha_min);
    if (c->frag_cap == 0) {
        if ((r = ensure(c, c->scan_tmp, scan_temp_bytes(n))) || (r = ensure(c, c->total, 64))) return r;
        launch_exclusive_scan(ptr<uint32_t>(c->ntiles), ptr<uint32_t>(c->offsets), n,
                              ptr<unsigned long long>(c->total), c->scan_tmp.p, st);
        uint64_t F = 0;
        if ((r = read_total(c, st, &F)) != GS_OK) return r;
        uint64_t cap = 2 * F + 4096;   // the culled count; growth during training stays inside
        if (cap > GS_MAX_FRAGMENTS) cap = GS_MAX_FRAGMENTS;
        c->frag_cap = cap;
        if ((r = ensure_iter(c, N, vb, c->frag_cap)) != GS_OK) return r;
    }
    r = run_binning(c, vb, pv, true, nullptr, ptr<uint32_t>(c->vals),
                    ptr<uint2>(c->ranges), ptr<uint32_t>(c->count), c->frag_cap, st);
    if (r != GS_OK) return r;
    size_t off = 0;
    for (int v = 0; v < B; ++v) {
        const size_t hw = (size_t)vb.v[v].W * vb.v[v].H;
        vb.v[v].img = imgs[v];
        vb.v[v].T_final = ptr<float>(c->T_final) + off;
        vb.v[v].n_contrib = ptr<uint32_t>(c->n_contrib) + off;
        off += hw;
    }
    const uint32_t *order = tile_order_for(c, vb, ptr<uint2>(c->ranges), st);
    launch_blend_fwd(vb, pv, ptr<uint32_t>(c->vals), ptr<uint2>(c->ranges), blend_of(c, c->frag_cap), c->hp.smem_batch,
                     c->hp.px_per_thread, c->status, order, st);
    return cuda_check(c, "gs_render");
}

}  // extern "C"
