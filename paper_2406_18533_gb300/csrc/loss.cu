// K10: loss = (1 - l) mean|I - I*| + l (1 - mean SSIM(I, I*)) and dL/dI
// (Sec. 2.1 step 3: "L1 and SSIM loss ... computed per-pixel for both forward
// and backward").  SSIM uses an 11x11 Gaussian window (sigma 1.5), zero
// padding, C1 = 0.01^2, C2 = 0.03^2.
//
// Two passes over 16x16 pixel tiles with a 5-pixel halo staged in shared
// memory, separable convolution in each:
//   pass A: the five local moments -> SSIM map value and its partials with
//           respect to (mu_x, sigma_xx, sigma_xy), stored as three maps
//           m1 = dS/dmu - 2 mu_x dS/dsxx - mu_y dS/dsxy, m2 = dS/dsxx,
//           m3 = dS/dsxy; L1 and SSIM sums accumulate per view;
//   pass B: dS/dx = (w * m1) + 2 x (w * m2) + y (w * m3) (the window is
//           symmetric, so the adjoint of the zero-padded correlation is the
//           same correlation), plus the L1 term.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int LT = 16;              // output tile edge
constexpr int HALO = 5;
constexpr int LR = LT + 2 * HALO;   // 26: staged region edge
constexpr float SSIM_C1 = 0.0001f;
constexpr float SSIM_C2 = 0.0009f;

struct Win { float w[11]; };

__global__ void __launch_bounds__(LT *LT) k_ssim_fwd(const float *img, const float *tgt, int W, int H, Win win,
                                                    float *maps, double *acc)
{
    __shared__ float sx[LR][LR], sy[LR][LR];
    __shared__ float h[5][LR][LT];
    const int plane = blockIdx.z;              // view * 3 + channel
    const int view = plane / 3;
    const int64_t hw = (int64_t)W * H;
    const float *X = img + plane * hw;
    const float *Y = tgt + plane * hw;
    const int ox = blockIdx.x * LT - HALO, oy = blockIdx.y * LT - HALO;
    const int t = threadIdx.x;
    for (int i = t; i < LR * LR; i += LT * LT) {
        const int r = i / LR, cc = i % LR;
        const int gx = ox + cc, gy = oy + r;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        sx[r][cc] = in ? X[(int64_t)gy * W + gx] : 0.f;
        sy[r][cc] = in ? Y[(int64_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    // horizontal pass over all LR rows, LT output columns
    for (int i = t; i < LR * LT; i += LT * LT) {
        const int r = i / LT, cc = i % LT;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float xv = sx[r][cc + k], yv = sy[r][cc + k], w = win.w[k];
            a += w * xv;
            b += w * yv;
            aa += w * xv * xv;
            bb += w * yv * yv;
            ab += w * xv * yv;
        }
        h[0][r][cc] = a; h[1][r][cc] = b; h[2][r][cc] = aa; h[3][r][cc] = bb; h[4][r][cc] = ab;
    }
    __syncthreads();
    const int lx = t % LT, ly = t / LT;
    const int gx = blockIdx.x * LT + lx, gy = blockIdx.y * LT + ly;
    float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
    for (int k = 0; k < 11; ++k) {
        const float w = win.w[k];
        mx += w * h[0][ly + k][lx];
        my += w * h[1][ly + k][lx];
        exx += w * h[2][ly + k][lx];
        eyy += w * h[3][ly + k][lx];
        exy += w * h[4][ly + k][lx];
    }
    float l1 = 0.f, ss = 0.f;
    if (gx < W && gy < H) {
        const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
        const float n1 = 2.f * mx * my + SSIM_C1, n2 = 2.f * sxy + SSIM_C2;
        const float d1 = mx * mx + my * my + SSIM_C1, d2 = sxx + syy + SSIM_C2;
        const float id = 1.f / (d1 * d2);
        const float S = n1 * n2 * id;
        const float A = 2.f * my * n2 * id - S * 2.f * mx / d1;
        const float Bm = -S / d2;
        const float Cm = 2.f * n1 * id;
        const int64_t pix = (int64_t)gy * W + gx;
        const int64_t tot = (int64_t)gridDim.z * hw;
        maps[plane * hw + pix] = A - 2.f * mx * Bm - my * Cm;
        maps[tot + plane * hw + pix] = Bm;
        maps[2 * tot + plane * hw + pix] = Cm;
        l1 = fabsf(sx[ly + HALO][lx + HALO] - sy[ly + HALO][lx + HALO]);
        ss = S;
    }
    // block reduction of the two sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    __shared__ float red[2][LT * LT / 32];
    if ((t & 31) == 0) { red[0][t >> 5] = l1; red[1][t >> 5] = ss; }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < LT * LT / 32; ++w) { a += red[0][w]; b += red[1][w]; }
        atomicAdd(&acc[2 * view], a);
        atomicAdd(&acc[2 * view + 1], b);
    }
}

__global__ void __launch_bounds__(LT *LT) k_ssim_bwd(const float *img, const float *tgt, int W, int H, Win win,
                                                    const float *maps, float lambda, float *dimg)
{
    __shared__ float sm[3][LR][LR];
    __shared__ float h[3][LR][LT];
    const int plane = blockIdx.z;
    const int64_t hw = (int64_t)W * H;
    const int64_t tot = (int64_t)gridDim.z * hw;
    const int ox = blockIdx.x * LT - HALO, oy = blockIdx.y * LT - HALO;
    const int t = threadIdx.x;
    for (int i = t; i < LR * LR; i += LT * LT) {
        const int r = i / LR, cc = i % LR;
        const int gx = ox + cc, gy = oy + r;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const int64_t o = plane * hw + (int64_t)gy * W + gx;
        sm[0][r][cc] = in ? maps[o] : 0.f;
        sm[1][r][cc] = in ? maps[tot + o] : 0.f;
        sm[2][r][cc] = in ? maps[2 * tot + o] : 0.f;
    }
    __syncthreads();
    for (int i = t; i < LR * LT; i += LT * LT) {
        const int r = i / LT, cc = i % LT;
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.w[k];
            a += w * sm[0][r][cc + k];
            b += w * sm[1][r][cc + k];
            c += w * sm[2][r][cc + k];
        }
        h[0][r][cc] = a; h[1][r][cc] = b; h[2][r][cc] = c;
    }
    __syncthreads();
    const int lx = t % LT, ly = t / LT;
    const int gx = blockIdx.x * LT + lx, gy = blockIdx.y * LT + ly;
    if (gx >= W || gy >= H) return;
    float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < 11; ++k) {
        const float w = win.w[k];
        a += w * h[0][ly + k][lx];
        b += w * h[1][ly + k][lx];
        c += w * h[2][ly + k][lx];
    }
    const int64_t o = plane * hw + (int64_t)gy * W + gx;
    const float x = img[o], y = tgt[o];
    const float n = 3.f * (float)hw;
    const float dS = a + 2.f * x * b + y * c;
    const float sgn = x > y ? 1.f : (x < y ? -1.f : 0.f);
    dimg[o] = ((1.f - lambda) * sgn - lambda * dS) / n;
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

}  // namespace

void launch_loss(const float *img, const float *target, int B, int W, int H, float lambda, float *loss_out,
                 float *d_img, float *maps, double *acc, cudaStream_t st)
{
    static const Win win = make_window();
    cudaMemsetAsync(acc, 0, sizeof(double) * 2 * B, st);
    const dim3 grid((W + LT - 1) / LT, (H + LT - 1) / LT, 3 * B);
    k_ssim_fwd<<<grid, LT * LT, 0, st>>>(img, target, W, H, win, maps, acc);
    k_ssim_bwd<<<grid, LT * LT, 0, st>>>(img, target, W, H, win, maps, lambda, d_img);
    k_loss_finish<<<1, 32, 0, st>>>(acc, B, 3.0 * (double)W * H, lambda, loss_out);
    count_launches(3);
}

}  // namespace gs
