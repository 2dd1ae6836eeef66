// gs_bin_noalloc: the binning of gs_bin with every byte of its scratch in one
// file-scope device array, for callers that must not allocate device memory.
//
// The array is part of the library's device image: every GPU on which the
// library's kernels are loaded holds it (NOALLOC_SCRATCH_BYTES) until the
// process exits.  Host code must not pass the array's name to a kernel (on
// the host it is only a stand-in symbol); the device address comes from
// cudaGetSymbolAddress, taken once per device below.
#include <cstring>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

// Limits of the allocation-free binning (also stated in include/gs.h).
constexpr int64_t NA_MAX_PAIRS = (int64_t)1 << 18;    // B * N (view, Gaussian) pairs
constexpr uint64_t NA_MAX_FRAGS = (uint64_t)1 << 20;  // fragment capacity of the output

// Byte layout of the scratch array (each region 256-byte aligned).
constexpr size_t OFF_OFFSETS = 0;                                      // uint32[pairs] fragment offsets
constexpr size_t OFF_RECT = OFF_OFFSETS + 4 * (size_t)NA_MAX_PAIRS;    // uint2[pairs] tile rectangles
constexpr size_t OFF_AREA = OFF_RECT + 8 * (size_t)NA_MAX_PAIRS;       // uint32[pairs] tile counts
constexpr size_t OFF_SCAN = OFF_AREA + 4 * (size_t)NA_MAX_PAIRS;       // scan temp, 4 KiB
constexpr size_t OFF_TOTAL = OFF_SCAN + 4096;                          // uint64 total, uint32 pair count
constexpr size_t OFF_STATUS = OFF_TOTAL + 256;                         // DevStatus
constexpr size_t OFF_TK = OFF_STATUS + 256;                            // uint32[frags] tile ids
constexpr size_t OFF_TK_ALT = OFF_TK + 4 * (size_t)NA_MAX_FRAGS;       // uint32[frags]
constexpr size_t OFF_VALS = OFF_TK_ALT + 4 * (size_t)NA_MAX_FRAGS;     // uint32[frags]
constexpr size_t OFF_PK = OFF_VALS + 4 * (size_t)NA_MAX_FRAGS;         // uint32[pairs] depth keys
constexpr size_t OFF_PV = OFF_PK + 4 * (size_t)NA_MAX_PAIRS;           // uint32[pairs] pair indices
constexpr size_t OFF_PK_ALT = OFF_PV + 4 * (size_t)NA_MAX_PAIRS;       // uint32[pairs]
constexpr size_t OFF_PV_ALT = OFF_PK_ALT + 4 * (size_t)NA_MAX_PAIRS;   // uint32[pairs]
constexpr size_t OFF_SORT = OFF_PV_ALT + 4 * (size_t)NA_MAX_PAIRS;     // sort temp, 640 KiB
constexpr size_t NOALLOC_SCRATCH_BYTES = OFF_SORT + 640 * 1024;        // 20.63 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
unsigned char *g_scratch_ptr[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, with that device
// current.  Outside stream capture it is looked up on every call (a cheap
// query that allocates nothing), so an address made stale by a
// cudaDeviceReset is never used; during capture the address of the last call
// outside capture on this device is used (module loading may not happen
// inside a capture).
gs_status scratch_on_current_device(cudaStream_t st, unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

int bits_for(uint32_t n)
{
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < (uint64_t)n) ++b;
    return b;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_bin_noalloc(const gs_proj *proj, const gs_camera *cams, int32_t B, int32_t tile,
                                    gs_bins *out, uint64_t *needed_host, void *stream)
{
    if (!proj || !cams || !out || B < 1 || B > GS_MAX_VIEWS || proj->B != B || proj->N < 0)
        return GS_ERR_INVALID_ARG;
    if (tile != 8 && tile != 16 && tile != 32) return GS_ERR_INVALID_ARG;
    if (!out->ranges || !out->count || (out->capacity > 0 && (!out->keys || !out->vals))) return GS_ERR_INVALID_ARG;
    const int64_t n = (int64_t)B * proj->N;
    if (n > NA_MAX_PAIRS || out->capacity > NA_MAX_FRAGS) return GS_ERR_INVALID_ARG;   // beyond the fixed scratch
    if (n > 0 && (!proj->xy || !proj->radius || !proj->rgb_d)) return GS_ERR_INVALID_ARG;
    if (scan_temp_bytes(n) > OFF_TOTAL - OFF_SCAN || sort_temp_bytes((uint64_t)n, out->capacity) > NOALLOC_SCRATCH_BYTES - OFF_SORT)
        return GS_ERR_INVALID_ARG;
    // view batch (host-side validation of the cameras as in gs_bin)
    ViewBatch vb;
    memset(&vb, 0, sizeof vb);
    vb.B = B;
    vb.tile = tile;
    uint64_t base = 0;
    for (int v = 0; v < B; ++v) {
        const gs_camera &k = cams[v];
        if (k.W < 1 || k.H < 1 || k.W > 65536 || k.H > 65536) return GS_ERR_INVALID_ARG;
        ViewCam &o = vb.v[v];
        o.W = k.W;
        o.H = k.H;
        o.TX = (k.W + tile - 1) / tile;
        o.TY = (k.H + tile - 1) / tile;
        o.tile_base = (uint32_t)base;
        base += (uint64_t)o.TX * o.TY;
    }
    if (base >= ((uint64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    vb.total_tiles = (uint32_t)base;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *s = nullptr;
    gs_status r = scratch_on_current_device(st, &s);
    if (r != GS_OK) return r;
    auto *offsets = reinterpret_cast<uint32_t *>(s + OFF_OFFSETS);
    auto *rect = reinterpret_cast<uint2 *>(s + OFF_RECT);
    auto *area = reinterpret_cast<uint32_t *>(s + OFF_AREA);
    auto *total = reinterpret_cast<unsigned long long *>(s + OFF_TOTAL);
    auto *n_vis = reinterpret_cast<uint32_t *>(s + OFF_TOTAL + 8);
    auto *status = reinterpret_cast<DevStatus *>(s + OFF_STATUS);
    auto *tk = reinterpret_cast<uint32_t *>(s + OFF_TK);
    auto *tk_alt = reinterpret_cast<uint32_t *>(s + OFF_TK_ALT);
    auto *vals_alt = reinterpret_cast<uint32_t *>(s + OFF_VALS);
    auto *pk = reinterpret_cast<uint32_t *>(s + OFF_PK);
    auto *pv_order = reinterpret_cast<uint32_t *>(s + OFF_PV);
    auto *pk_alt = reinterpret_cast<uint32_t *>(s + OFF_PK_ALT);
    auto *pv_alt = reinterpret_cast<uint32_t *>(s + OFF_PV_ALT);
    void *sort_tmp = s + OFF_SORT;
    // The array keeps the previous call's contents: the status word must start at zero.
    cudaMemsetAsync(status, 0, sizeof(DevStatus), st);

    const ProjView pv{reinterpret_cast<float2 *>(proj->xy), reinterpret_cast<float4 *>(proj->conic_o),
                      reinterpret_cast<float4 *>(proj->rgb_d), proj->radius, proj->N};
    const int high = bits_for(vb.total_tiles);
    const bool even = fragment_sort_passes(high) % 2 == 0;
    uint32_t *order = launch_depth_order(vb, pv, false, rect, area, pk, pv_order, pk_alt, pv_alt, offsets, n_vis,
                                         total, s + OFF_SCAN, sort_tmp, status, st);
    // the sort's dead buffers take the counts and rectangles in depth order
    uint32_t *counts = order == pv_order ? pk : pv_order;
    uint32_t *rx = order == pv_order ? pv_alt : pk, *ry = pk_alt;
    launch_gather_counts(order, rect, area, nullptr, n, n_vis, counts, rx, ry, nullptr, st);
    launch_exclusive_scan(counts, offsets, n, total, s + OFF_SCAN, st, n_vis);
    launch_emit_keys(vb, pv.N, n_vis, order, rx, ry, nullptr, offsets, even ? tk : tk_alt,
                     even ? out->vals : vals_alt, out->capacity, total, status, out->count, 0.f, st);
    launch_sort_fragments(even ? tk : tk_alt, even ? out->vals : vals_alt, even ? tk_alt : tk,
                          even ? vals_alt : out->vals, out->capacity, out->count, high, sort_tmp, status, st);
    launch_tile_ranges(tk, out->count, out->capacity, reinterpret_cast<uint2 *>(out->ranges), vb.total_tiles, st);
    launch_compose_keys(vb, pv.N, tk, out->vals, out->count, out->capacity, pv.rgb_d, out->keys, st);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    if (needed_host) {
        unsigned long long F = 0;
        if (cudaMemcpyAsync(&F, total, sizeof F, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        *needed_host = F;
        if (F > out->capacity) return GS_ERR_CAPACITY;
    }
    return GS_OK;
}
