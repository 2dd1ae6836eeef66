// K10: loss = (1 - l) mean|I - I*| + l (1 - mean SSIM(I, I*)) and dL/dI
// (Sec. 2.1 step 3: "L1 and SSIM loss ... computed per-pixel for both forward
// and backward").  SSIM uses an 11x11 Gaussian window (sigma 1.5), zero
// padding, C1 = 0.01^2, C2 = 0.03^2.
//
// Two passes, each a separable convolution sliding down strips of 128 x 64
// pixels (see k_ssim_fwd):
//   pass A: the five local moments -> SSIM map value and its partials with
//           respect to (mu_x, sigma_xx, sigma_xy), stored as three maps
//           m1 = dS/dmu - 2 mu_x dS/dsxx - mu_y dS/dsxy, m2 = dS/dsxx,
//           m3 = dS/dsxy; L1 and SSIM sums accumulate per view;
//   pass B: dS/dx = (w * m1) + 2 x (w * m2) + y (w * m3) (the window is
//           symmetric, so the adjoint of the zero-padded correlation is the
//           same correlation), plus the L1 term.
//
// Staging: when the image width is a multiple of 4 floats (the row pitch of a
// TMA tensor is a multiple of 16 bytes), each chunk of 11 input rows comes in
// as 2D tiles of a 3D tensor map (x, y, plane) with one
// cp.async.bulk.tensor per plane issued by one thread and tracked by an
// mbarrier; the tile starts at column x0 - 8 (16-byte aligned) and rows
// outside the image arrive as zeros (the padding).  Other widths use 4-byte
// cp.async copies per element.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int LC = 128;             // output columns per CTA, one per thread
constexpr int LROWS = 64;           // output rows per CTA
constexpr int HALO = 5;
constexpr int WIN = 11;
constexpr int LW = LC + 2 * HALO;   // staged row width (element copies)
constexpr int LWT = LC + 16;        // staged row pitch; a TMA tile spans x0 - 8 .. x0 + LC + 7
constexpr int TMA_OFF = 8 - HALO;   // column of x0 - 5 in a TMA tile
constexpr int WINP = WIN + 1;       // rows per staged buffer: 12 x LWT floats = 6912 bytes keeps every
                                    // buffer 128-byte aligned for the TMA (the last row is unused)
static_assert((WINP * LWT * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 24;   // polls of one mbarrier wait before giving up
constexpr float SSIM_C1 = 0.0001f;
constexpr float SSIM_C2 = 0.0009f;

struct Win { float w[11]; };

// Asynchronous 4-byte global -> shared copies (cp.async, sm_80+); an invalid
// source copies nothing and zero-fills the destination.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0u;
}

// Bounded wait for phase `parity` of bar: past the limit the error is recorded
// and the wait goes on, bounded again, for the copies still in flight (the
// buffer must not be released while the copy engine writes it).  Returns
// false if the copies never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, DevStatus *status)
{
    for (uint32_t i = 0; i < TMA_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (status) atomicCAS(&status->code, 0, (int)GS_ERR_TIMEOUT);
    for (uint32_t i = 0; i < TMA_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// A 3D tile (x, y, plane) of `map` into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier shared-memory reads before later copies of the
// asynchronous proxy into the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Input rows r0 .. r0+10 of plane `src` (zero outside the image), columns
// x0 - 5 .. x0 + LC + 4, into buf, asynchronously (one commit group).
__device__ __forceinline__ void load_chunk(float (*buf)[LWT], const float *src, int r0, int x0, int W, int H)
{
    for (int i = threadIdx.x; i < WIN * LW; i += LC) {
        const int row = i / LW, col = i - row * LW;
        const int r = r0 + row, gx = x0 - HALO + col;
        const bool ok = r >= 0 && r < H && gx >= 0 && gx < W;
        cp_async4(&buf[row][col], ok ? src + (int64_t)r * W + gx : src, ok);
    }
}

// Both passes slide down a strip of LC columns x LROWS rows.  Input rows come
// in chunks of 11, loaded asynchronously into a double buffer while the
// previous chunk is used (two barriers per chunk).  Each thread convolves a
// row horizontally at its column, keeps the last 11 horizontal results in a
// register ring (the row loop is unrolled by 11, so ring slots are static),
// and once 11 rows are in, convolves vertically for the output row 5 rows up.
// Every input value is read once per strip (plus the 10-row and 10-column
// halo).
template <bool TMA>
__global__ void __launch_bounds__(LC) k_ssim_fwd(const float *img, const float *tgt, int W, int H, Win win,
                                                 float *maps, double *acc, const __grid_constant__ CUtensorMap mx,
                                                 const __grid_constant__ CUtensorMap my, DevStatus *status)
{
    __shared__ __align__(128) float sx[2][WINP][LWT];
    __shared__ __align__(128) float sy[2][WINP][LWT];
    __shared__ float red[2][LC / 32];
    __shared__ __align__(8) uint64_t bar[2];
    const int plane = blockIdx.z, view = plane / 3;
    const int64_t hw = (int64_t)W * H, tot = (int64_t)gridDim.z * hw;
    const float *X = img + plane * hw, *Y = tgt + plane * hw;
    const int x0 = blockIdx.x * LC, y0 = blockIdx.y * LROWS;
    const int t = threadIdx.x, gx = x0 + t;
    const int nrows = min(LROWS, H - y0);
    const int nin = nrows + 2 * HALO;
    constexpr int off = TMA ? TMA_OFF : 0;
    constexpr uint32_t chunk_bytes = 2u * WIN * LWT * 4u;
    float ring[WIN][5];
    float l1 = 0.f, ss = 0.f;
    uint32_t phase = 0u;                                // bit b: parity of buffer b's next completion
    if constexpr (TMA) {
        if (t == 0) {
            mbar_init(&bar[0]);
            mbar_init(&bar[1]);
            mbar_expect_tx(&bar[0], chunk_bytes);
            tma_load_3d(&sx[0][0][0], &mx, x0 - 8, y0 - HALO, plane, &bar[0]);
            tma_load_3d(&sy[0][0][0], &my, x0 - 8, y0 - HALO, plane, &bar[0]);
        }
        __syncthreads();
    } else {
        load_chunk(sx[0], X, y0 - HALO, x0, W, H);
        load_chunk(sy[0], Y, y0 - HALO, x0, W, H);
        cp_async_commit();
    }
    for (int rb = 0, cb = 0; rb < nin; rb += WIN, cb ^= 1) {
        if constexpr (TMA) {
            if (t == 0 && rb + WIN < nin) {             // the other buffer was released by the last barrier
                fence_proxy_async();
                mbar_expect_tx(&bar[cb ^ 1], chunk_bytes);
                tma_load_3d(&sx[cb ^ 1][0][0], &mx, x0 - 8, y0 - HALO + rb + WIN, plane, &bar[cb ^ 1]);
                tma_load_3d(&sy[cb ^ 1][0][0], &my, x0 - 8, y0 - HALO + rb + WIN, plane, &bar[cb ^ 1]);
            }
            mbar_wait(&bar[cb], (phase >> cb) & 1u, status);
            phase ^= 1u << cb;
        } else {
            if (rb + WIN < nin) {
                load_chunk(sx[cb ^ 1], X, y0 - HALO + rb + WIN, x0, W, H);
                load_chunk(sy[cb ^ 1], Y, y0 - HALO + rb + WIN, x0, W, H);
            }
            cp_async_commit();
            cp_async_wait<1>();                         // this chunk has landed
            __syncthreads();
        }
#pragma unroll
        for (int s = 0; s < WIN; ++s) {
            const int q = rb + s;                       // input row within the strip
            if (q >= nin) break;                        // the same for every thread
            const float *bx = sx[cb][s] + off, *by = sy[cb][s] + off;
            float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k < WIN; ++k) {
                const float xv = bx[t + k], yv = by[t + k], w = win.w[k];
                a += w * xv;
                b += w * yv;
                aa += w * xv * xv;
                bb += w * yv * yv;
                ab += w * xv * yv;
            }
            ring[s][0] = a; ring[s][1] = b; ring[s][2] = aa; ring[s][3] = bb; ring[s][4] = ab;
            if (q < 2 * HALO) continue;
            // rows q-10 .. q are in the ring, oldest at slot (s + 1) % 11
            float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
            for (int k = 0; k < WIN; ++k) {
                const int sl = (s + 1 + k) % WIN;
                const float w = win.w[k];
                mx += w * ring[sl][0];
                my += w * ring[sl][1];
                exx += w * ring[sl][2];
                eyy += w * ring[sl][3];
                exy += w * ring[sl][4];
            }
            const int gy = y0 + q - 2 * HALO;
            if (gx < W) {
                const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                const float n1 = 2.f * mx * my + SSIM_C1, n2 = 2.f * sxy + SSIM_C2;
                const float d1 = mx * mx + my * my + SSIM_C1, d2 = sxx + syy + SSIM_C2;
                const float id = 1.f / (d1 * d2);
                const float S = n1 * n2 * id;
                const float A = 2.f * my * n2 * id - S * 2.f * mx / d1;
                const float Bm = -S / d2;
                const float Cm = 2.f * n1 * id;
                const int64_t pix = (int64_t)gy * W + gx;
                maps[plane * hw + pix] = A - 2.f * mx * Bm - my * Cm;
                maps[tot + plane * hw + pix] = Bm;
                maps[2 * tot + plane * hw + pix] = Cm;
                l1 += fabsf(X[pix] - Y[pix]);     // (the previous chunk's buffer is being refilled)
                ss += S;
            }
        }
        __syncthreads();                                // the next chunk's load may overwrite cb ^ 1
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if ((t & 31) == 0) { red[0][t >> 5] = l1; red[1][t >> 5] = ss; }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < LC / 32; ++w) { a += red[0][w]; b += red[1][w]; }
        atomicAdd(&acc[2 * view], a);
        atomicAdd(&acc[2 * view + 1], b);
    }
}

// mm: a 3D tensor map over the three maps as 3 x (3 B) planes.
template <bool TMA>
__global__ void __launch_bounds__(LC) k_ssim_bwd(const float *img, const float *tgt, int W, int H, Win win,
                                                 const float *maps, float lambda, float *dimg,
                                                 const __grid_constant__ CUtensorMap mm, DevStatus *status)
{
    __shared__ __align__(128) float sm[2][3][WINP][LWT];
    __shared__ __align__(8) uint64_t bar[2];
    const int plane = blockIdx.z;
    const int64_t hw = (int64_t)W * H, tot = (int64_t)gridDim.z * hw;
    const float *M[3] = {maps + plane * hw, maps + tot + plane * hw, maps + 2 * tot + plane * hw};
    const int x0 = blockIdx.x * LC, y0 = blockIdx.y * LROWS;
    const int t = threadIdx.x, gx = x0 + t;
    const int nrows = min(LROWS, H - y0);
    const int nin = nrows + 2 * HALO;
    const float n = 3.f * (float)hw;
    constexpr int off = TMA ? TMA_OFF : 0;
    constexpr uint32_t chunk_bytes = 3u * WIN * LWT * 4u;
    const int P = (int)gridDim.z;
    float ring[WIN][3];
    uint32_t phase = 0u;
    if constexpr (TMA) {
        if (t == 0) {
            mbar_init(&bar[0]);
            mbar_init(&bar[1]);
            mbar_expect_tx(&bar[0], chunk_bytes);
#pragma unroll
            for (int m = 0; m < 3; ++m) tma_load_3d(&sm[0][m][0][0], &mm, x0 - 8, y0 - HALO, m * P + plane, &bar[0]);
        }
        __syncthreads();
    } else {
#pragma unroll
        for (int m = 0; m < 3; ++m) load_chunk(sm[0][m], M[m], y0 - HALO, x0, W, H);
        cp_async_commit();
    }
    for (int rb = 0, cb = 0; rb < nin; rb += WIN, cb ^= 1) {
        if constexpr (TMA) {
            if (t == 0 && rb + WIN < nin) {
                fence_proxy_async();
                mbar_expect_tx(&bar[cb ^ 1], chunk_bytes);
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    tma_load_3d(&sm[cb ^ 1][m][0][0], &mm, x0 - 8, y0 - HALO + rb + WIN, m * P + plane, &bar[cb ^ 1]);
            }
            mbar_wait(&bar[cb], (phase >> cb) & 1u, status);
            phase ^= 1u << cb;
        } else {
            if (rb + WIN < nin) {
#pragma unroll
                for (int m = 0; m < 3; ++m) load_chunk(sm[cb ^ 1][m], M[m], y0 - HALO + rb + WIN, x0, W, H);
            }
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
        }
#pragma unroll
        for (int s = 0; s < WIN; ++s) {
            const int q = rb + s;
            if (q >= nin) break;
            float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
            for (int k = 0; k < WIN; ++k) {
                const float w = win.w[k];
                h0 += w * sm[cb][0][s][t + k + off];
                h1 += w * sm[cb][1][s][t + k + off];
                h2 += w * sm[cb][2][s][t + k + off];
            }
            ring[s][0] = h0; ring[s][1] = h1; ring[s][2] = h2;
            if (q < 2 * HALO) continue;
            float a = 0.f, bb = 0.f, c = 0.f;
#pragma unroll
            for (int k = 0; k < WIN; ++k) {
                const int sl = (s + 1 + k) % WIN;
                const float w = win.w[k];
                a += w * ring[sl][0];
                bb += w * ring[sl][1];
                c += w * ring[sl][2];
            }
            const int gy = y0 + q - 2 * HALO;
            if (gx < W) {
                const int64_t o = plane * hw + (int64_t)gy * W + gx;
                const float x = img[o], y = tgt[o];
                const float dS = a + 2.f * x * bb + y * c;
                const float sgn = x > y ? 1.f : (x < y ? -1.f : 0.f);
                dimg[o] = ((1.f - lambda) * sgn - lambda * dS) / n;
            }
        }
        __syncthreads();
    }
}

__global__ void k_loss_finish(const double *acc, int B, double n, float lambda, float *loss_out)
{
    const int v = threadIdx.x;
    if (v < B) loss_out[v] = (float)((1.0 - lambda) * acc[2 * v] / n + lambda * (1.0 - acc[2 * v + 1] / n));
}

Win make_window()
{
    Win w;
    double g[11], s = 0.0;
    for (int k = 0; k < 11; ++k) {
        const double x = k - 5.0;
        g[k] = exp(-x * x / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k < 11; ++k) w.w[k] = (float)(g[k] / s);
    return w;
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link against
// libcuda); null when unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// A 3D float32 tensor map (W, H, planes) with boxes of LWT x WIN x 1; zero
// fill outside the tensor.  False when the layout cannot be mapped (the row
// pitch must be a multiple of 16 bytes) or encoding fails.
bool encode_planes(CUtensorMap *map, const float *base, int W, int H, int64_t planes)
{
    auto enc = tensor_map_encoder();
    if (!enc || (W & 3) != 0 || W < 4 || planes < 1 || ((uintptr_t)base & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 4, (cuuint64_t)W * H * 4};
    const cuuint32_t box[3] = {(cuuint32_t)LWT, (cuuint32_t)WIN, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

void launch_loss(const float *img, const float *target, int B, int W, int H, float lambda, float *loss_out,
                 float *d_img, float *maps, double *acc, DevStatus *status, cudaStream_t st)
{
    static const Win win = make_window();
    cudaMemsetAsync(acc, 0, sizeof(double) * 2 * B, st);
    const dim3 grid((W + LC - 1) / LC, (H + LROWS - 1) / LROWS, 3 * B);
    CUtensorMap mx, my, mm;
    const bool tma = encode_planes(&mx, img, W, H, 3 * (int64_t)B) && encode_planes(&my, target, W, H, 3 * (int64_t)B) &&
                     encode_planes(&mm, maps, W, H, 9 * (int64_t)B);
    if (tma) {
        k_ssim_fwd<true><<<grid, LC, 0, st>>>(img, target, W, H, win, maps, acc, mx, my, status);
        k_ssim_bwd<true><<<grid, LC, 0, st>>>(img, target, W, H, win, maps, lambda, d_img, mm, status);
    } else {
        memset(&mx, 0, sizeof mx);
        k_ssim_fwd<false><<<grid, LC, 0, st>>>(img, target, W, H, win, maps, acc, mx, mx, status);
        k_ssim_bwd<false><<<grid, LC, 0, st>>>(img, target, W, H, win, maps, lambda, d_img, mx, status);
    }
    k_loss_finish<<<1, 32, 0, st>>>(acc, B, 3.0 * (double)W * H, lambda, loss_out);
    count_launches(3);
}

}  // namespace gs
