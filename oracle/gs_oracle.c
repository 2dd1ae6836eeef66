/*
 * FP64 CPU oracle for the 3D Gaussian Splatting training hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (arXiv 2406.18533, Sec. 2.1, "Background on 3D Gaussian
 * Training"): step 1 "Gaussian transformation" (projected centre, depth,
 * footprint radius and view-dependent SH colour of every Gaussian), step 2
 * "Rendering" (each pixel composites the Gaussians that intersect it, in
 * increasing depth, until a transmittance threshold is reached) and the
 * backward pass of both ("standard approaches to backpropagation").  The paper
 * defers the formulas to the original 3DGS method; the readings used here are
 * listed in the design notes and repeated at each function.
 *
 * Style: plain double-precision loops, one Gaussian or one pixel at a time, in
 * the order the definition states.  OpenMP only splits independent pixels or
 * Gaussians across threads.  Build with -ffp-contract=off so the float32
 * binning routine rounds exactly like IEEE single precision.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form isotropic Gaussian,
 * sum(alpha*T) + T_final = 1, brute-force per-pixel compositing on tiny
 * scenes, central finite differences of every gradient, SH orthonormality by
 * quadrature, quaternion orthogonality.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Camera: cam[16] = R (row-major world->camera), t, fx, fy, cx, cy.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double R[9], t[3], fx, fy, cx, cy, near_z;
    int W, H;
} ocam;

static ocam mk_cam(const double *c, int W, int H, double near_z)
{
    ocam k;
    for (int i = 0; i < 9; ++i) k.R[i] = c[i];
    for (int i = 0; i < 3; ++i) k.t[i] = c[9 + i];
    k.fx = c[12]; k.fy = c[13]; k.cx = c[14]; k.cy = c[15];
    k.W = W; k.H = H; k.near_z = near_z;
    return k;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 with the Condon-Shortley phase.    */
/* Index k = l*l + l + m.  Constants come from their closed forms.           */
/* ------------------------------------------------------------------------ */
static void sh_basis(const double d[3], double Y[16], double dY[16][3])
{
    const double pi = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    const double c0 = 0.5 / sqrt(pi);
    const double c1 = sqrt(3.0 / (4.0 * pi));
    const double a2 = 0.5 * sqrt(15.0 / pi);    /* xy, yz, xz terms      */
    const double b2 = 0.25 * sqrt(5.0 / pi);    /* 3z^2 - 1              */
    const double c2 = 0.25 * sqrt(15.0 / pi);   /* x^2 - y^2             */
    const double e3 = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double f3 = 0.5 * sqrt(105.0 / pi);
    const double g3 = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double h3 = 0.25 * sqrt(7.0 / pi);
    const double k3 = 0.25 * sqrt(105.0 / pi);

    Y[0] = c0;
    Y[1] = -c1 * y;  Y[2] = c1 * z;  Y[3] = -c1 * x;
    Y[4] = a2 * x * y;
    Y[5] = -a2 * y * z;
    Y[6] = b2 * (3.0 * z * z - 1.0);
    Y[7] = -a2 * x * z;
    Y[8] = c2 * (x * x - y * y);
    Y[9] = -e3 * y * (3.0 * x * x - y * y);
    Y[10] = f3 * x * y * z;
    Y[11] = -g3 * y * (5.0 * z * z - 1.0);
    Y[12] = h3 * z * (5.0 * z * z - 3.0);
    Y[13] = -g3 * x * (5.0 * z * z - 1.0);
    Y[14] = k3 * z * (x * x - y * y);
    Y[15] = -e3 * x * (x * x - 3.0 * y * y);

    if (!dY) return;
    memset(dY, 0, sizeof(double) * 48);
    dY[1][1] = -c1;
    dY[2][2] = c1;
    dY[3][0] = -c1;
    dY[4][0] = a2 * y;            dY[4][1] = a2 * x;
    dY[5][1] = -a2 * z;           dY[5][2] = -a2 * y;
    dY[6][2] = 6.0 * b2 * z;
    dY[7][0] = -a2 * z;           dY[7][2] = -a2 * x;
    dY[8][0] = 2.0 * c2 * x;      dY[8][1] = -2.0 * c2 * y;
    dY[9][0] = -6.0 * e3 * x * y; dY[9][1] = -e3 * (3.0 * x * x - 3.0 * y * y);
    dY[10][0] = f3 * y * z;       dY[10][1] = f3 * x * z;  dY[10][2] = f3 * x * y;
    dY[11][1] = -g3 * (5.0 * z * z - 1.0);  dY[11][2] = -10.0 * g3 * y * z;
    dY[12][2] = h3 * (15.0 * z * z - 3.0);
    dY[13][0] = -g3 * (5.0 * z * z - 1.0);  dY[13][2] = -10.0 * g3 * x * z;
    dY[14][0] = 2.0 * k3 * x * z; dY[14][1] = -2.0 * k3 * y * z; dY[14][2] = k3 * (x * x - y * y);
    dY[15][0] = -e3 * (3.0 * x * x - 3.0 * y * y); dY[15][1] = 6.0 * e3 * x * y;
}

/* Exported for the orthonormality pin. */
void or_sh_eval(int64_t n, const double *dirs, double *Y)
{
    for (int64_t i = 0; i < n; ++i) sh_basis(dirs + 3 * i, Y + 16 * i, NULL);
}

/* ------------------------------------------------------------------------ */
/* Quaternion (w, x, y, z), normalised, to a rotation matrix (row-major).     */
/* ------------------------------------------------------------------------ */
static void quat_to_rot(const double q[4], double R[9])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Exported for the orthogonality pin: q[n*4] (any norm) -> R[n*9]. */
void or_quat_rot(int64_t n, const double *q, double *R)
{
    for (int64_t i = 0; i < n; ++i) {
        double qq[4], nq = 0;
        for (int j = 0; j < 4; ++j) nq += q[4 * i + j] * q[4 * i + j];
        nq = sqrt(nq);
        for (int j = 0; j < 4; ++j) qq[j] = q[4 * i + j] / nq;
        quat_to_rot(qq, R + 9 * i);
    }
}

/* ------------------------------------------------------------------------ */
/* Per-Gaussian forward ("Gaussian transformation", Sec. 2.1 step 1).        */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* parameters, promoted to double */
    double x[3], logit, logs[3], q[4], sh[16][3];
    /* activations */
    double o, s[3], qn[4], qnorm, Rq[9], M[9], Sig[9];
    /* camera space */
    double pc[3];
    int culled;           /* 1: z <= near, or singular 2D covariance */
    int clamp_x, clamp_y; /* off-axis clamp of x/z, y/z active */
    double Lx, Ly;        /* clamp bounds (signed) when active */
    double xt, yt;        /* clamped x, y used in the Jacobian */
    double J[6], T[6];    /* 2x3, row-major */
    double S2[3];         /* 2D covariance after dilation: (A, B, C) */
    double det, conic[3], lam, ext3;
    int radius, rect[4], visible;
    double u, v, depth;
    double dir[3], dist, Y[16], dY[16][3], rgb_raw[3], rgb[3];
} gfwd;

static void load_params(const float *mo, const float *ls, const float *q, const float *sh,
                        int64_t N, int64_t g, gfwd *f)
{
    for (int i = 0; i < 3; ++i) f->x[i] = mo[4 * g + i];
    f->logit = mo[4 * g + 3];
    for (int i = 0; i < 3; ++i) f->logs[i] = ls[4 * g + i];
    for (int i = 0; i < 4; ++i) f->q[i] = q[4 * g + i];
    for (int k = 0; k < 16; ++k)
        for (int ch = 0; ch < 3; ++ch) {
            int j = 3 * k + ch;
            f->sh[k][ch] = sh[((int64_t)(j >> 2) * N + g) * 4 + (j & 3)];
        }
}

/* Tile rectangle (inclusive) of a footprint, in double precision. */
static int rect_f64(double u, double v, int r, int W, int H, int tile, int rect[4])
{
    const int TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
    double x0 = floor((u - r) / tile), x1 = floor((u + r) / tile);
    double y0 = floor((v - r) / tile), y1 = floor((v + r) / tile);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > TX - 1) x1 = TX - 1;
    if (y1 > TY - 1) y1 = TY - 1;
    if (!(x0 <= x1 && y0 <= y1)) { rect[0] = rect[1] = rect[2] = rect[3] = 0; return 0; }
    rect[0] = (int)x0; rect[1] = (int)x1; rect[2] = (int)y0; rect[3] = (int)y1;
    return 1;
}

static void g_forward(const ocam *cam, int deg, int tile, gfwd *f)
{
    /* activations: sigmoid opacity, exp scale, normalised quaternion */
    f->o = 1.0 / (1.0 + exp(-f->logit));
    for (int i = 0; i < 3; ++i) f->s[i] = exp(f->logs[i]);
    double nq = 0;
    for (int i = 0; i < 4; ++i) nq += f->q[i] * f->q[i];
    f->qnorm = sqrt(nq);
    for (int i = 0; i < 4; ++i) f->qn[i] = f->q[i] / f->qnorm;
    quat_to_rot(f->qn, f->Rq);
    /* M = Rq * diag(s); Sigma = M M^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f->M[3 * i + j] = f->Rq[3 * i + j] * f->s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->M[3 * i + k] * f->M[3 * j + k];
            f->Sig[3 * i + j] = acc;
        }
    /* camera space */
    for (int i = 0; i < 3; ++i) {
        double acc = cam->t[i];
        for (int k = 0; k < 3; ++k) acc += cam->R[3 * i + k] * f->x[k];
        f->pc[i] = acc;
    }
    f->visible = 0; f->radius = 0; f->culled = 0;
    memset(f->rect, 0, sizeof f->rect);
    const double z = f->pc[2];
    /* colour needs only the camera centre; compute it even when culled */
    {
        double C[3];
        for (int i = 0; i < 3; ++i) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc -= cam->R[3 * k + i] * cam->t[k];
            C[i] = acc;
        }
        double dd = 0;
        for (int i = 0; i < 3; ++i) { f->dir[i] = f->x[i] - C[i]; dd += f->dir[i] * f->dir[i]; }
        f->dist = sqrt(dd);
        for (int i = 0; i < 3; ++i) f->dir[i] /= f->dist;
        sh_basis(f->dir, f->Y, f->dY);
        const int nk = (deg + 1) * (deg + 1);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0;
            for (int k = 0; k < nk; ++k) acc += f->sh[k][ch] * f->Y[k];
            f->rgb_raw[ch] = acc + 0.5;
            f->rgb[ch] = f->rgb_raw[ch] < 0 ? 0 : f->rgb_raw[ch];
        }
    }
    if (!(z > cam->near_z)) { f->culled = 1; return; }
    /* pinhole projection, pixel centres at (i + 0.5, j + 0.5) */
    f->u = cam->fx * f->pc[0] / z + cam->cx;
    f->v = cam->fy * f->pc[1] / z + cam->cy;
    f->depth = z;
    /* EWA Jacobian with the off-axis clamp of x/z and y/z at 1.3 tan(fov/2) */
    const double limx = 1.3 * (0.5 * cam->W / cam->fx);
    const double limy = 1.3 * (0.5 * cam->H / cam->fy);
    double tx = f->pc[0] / z, ty = f->pc[1] / z;
    f->clamp_x = 0; f->clamp_y = 0; f->Lx = 0; f->Ly = 0;
    if (tx > limx) { f->clamp_x = 1; f->Lx = limx; tx = limx; }
    else if (tx < -limx) { f->clamp_x = 1; f->Lx = -limx; tx = -limx; }
    if (ty > limy) { f->clamp_y = 1; f->Ly = limy; ty = limy; }
    else if (ty < -limy) { f->clamp_y = 1; f->Ly = -limy; ty = -limy; }
    f->xt = tx * z; f->yt = ty * z;
    f->J[0] = cam->fx / z; f->J[1] = 0; f->J[2] = -cam->fx * f->xt / (z * z);
    f->J[3] = 0; f->J[4] = cam->fy / z; f->J[5] = -cam->fy * f->yt / (z * z);
    /* T = J * Rcam (2x3) */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->J[3 * i + k] * cam->R[3 * k + j];
            f->T[3 * i + j] = acc;
        }
    /* Sigma' = T Sigma T^T + 0.3 I */
    double S2f[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += f->T[3 * i + a] * f->Sig[3 * a + b] * f->T[3 * j + b];
            S2f[2 * i + j] = acc;
        }
    f->S2[0] = S2f[0] + 0.3;
    f->S2[1] = 0.5 * (S2f[1] + S2f[2]);
    f->S2[2] = S2f[3] + 0.3;
    f->det = f->S2[0] * f->S2[2] - f->S2[1] * f->S2[1];
    if (!(f->det > 0)) { f->culled = 1; return; }
    f->conic[0] = f->S2[2] / f->det;
    f->conic[1] = -f->S2[1] / f->det;
    f->conic[2] = f->S2[0] / f->det;
    /* footprint radius: 3 sigma of the major axis, rounded up to whole pixels */
    const double m = 0.5 * (f->S2[0] + f->S2[2]);
    double disc = m * m - f->det;
    if (disc < 0) disc = 0;
    f->lam = m + sqrt(disc);
    f->ext3 = 3.0 * sqrt(f->lam);
    f->radius = (int)ceil(f->ext3);
    f->visible = rect_f64(f->u, f->v, f->radius, cam->W, cam->H, tile, f->rect);
    if (!f->visible) f->radius = 0;
}

/*
 * or_preprocess: Sec. 2.1 step 1 for one view, all N Gaussians.
 * Outputs (double unless noted), one row per Gaussian:
 *   xy[2N]=(u,v), conic_o[4N]=(a,b,c,o), rgb[3N] (clamped), rgb_raw[3N],
 *   depth[N], ext3[N]=3*sqrt(lambda_max), radius[N] (int, 0 = not visible),
 *   rect[4N] (int; x0,x1,y0,y1 inclusive).
 */
void or_preprocess(int64_t N, const float *mo, const float *ls, const float *q, const float *sh,
                   int deg, const double *cam16, int W, int H, double near_z, int tile,
                   double *xy, double *conic_o, double *rgb, double *rgb_raw, double *depth,
                   double *ext3, int32_t *radius, int32_t *rect)
{
    const ocam cam = mk_cam(cam16, W, H, near_z);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < N; ++g) {
        gfwd f;
        load_params(mo, ls, q, sh, N, g, &f);
        g_forward(&cam, deg, tile, &f);
        xy[2 * g] = f.culled ? 0 : f.u;
        xy[2 * g + 1] = f.culled ? 0 : f.v;
        for (int i = 0; i < 3; ++i) conic_o[4 * g + i] = f.culled ? 0 : f.conic[i];
        conic_o[4 * g + 3] = f.o;
        for (int i = 0; i < 3; ++i) { rgb[3 * g + i] = f.rgb[i]; rgb_raw[3 * g + i] = f.rgb_raw[i]; }
        depth[g] = f.culled ? 0 : f.depth;
        ext3[g] = f.culled ? 0 : f.ext3;
        radius[g] = f.visible ? f.radius : 0;
        for (int i = 0; i < 4; ++i) rect[4 * g + i] = f.rect[i];
    }
}

/*
 * or_rect_f32: tile rectangle of a footprint computed with IEEE single
 * precision operations only (subtract, multiply by the exact power-of-two
 * 1/tile, floor), for the bit-exact stage check of binning.  radius <= 0 means
 * not visible.  Returns per Gaussian rect[4] and vis (0/1).
 */
/* or_rect_f64: the double-precision tile rectangle of the transformation
 * (rect_f64) for given centres and integer radii, exported for its pin. */
void or_rect_f64(int64_t n, const double *u, const double *v, const int32_t *radius,
                 int W, int H, int tile, int32_t *rect, int32_t *vis)
{
    for (int64_t g = 0; g < n; ++g) {
        int r4[4];
        vis[g] = radius[g] > 0 ? rect_f64(u[g], v[g], radius[g], W, H, tile, r4) : 0;
        if (!vis[g]) r4[0] = r4[1] = r4[2] = r4[3] = 0;
        for (int i = 0; i < 4; ++i) rect[4 * g + i] = r4[i];
    }
}

/*
 * or_fp32_bounds: a model of how far a float32 evaluation of the
 * transformation (the same float32 parameters and camera; IEEE single
 * operations in any order, fused multiply-adds allowed) can land from the
 * exact values of or_preprocess.  It is the standard forward error analysis
 * (each operation rounds with relative error at most u = 2^-24, a sum of n
 * terms errs by at most about n u times the sum of the terms' magnitudes),
 * componentwise, widened by a factor of 2.  Per Gaussian of one view:
 *   err[6g..6g+5] = (du, dv, dA, dB, dC, rinv):
 *     du, dv      bound the error of the projected centre (pixels);
 *     dA, dB, dC  bound the error of the 2D covariance entries (pixels^2)
 *                 formed as T Sigma T^T + 0.3 I with T = J R and Sigma =
 *                 M M^T, M = Rq diag(s): the rotation of the normalised
 *                 quaternion errs absolutely (a few u per entry), so M errs
 *                 by <= 9u s_k per entry of column k, Sigma by that times
 *                 |M|, and T Sigma T^T carries those and T's own rounding
 *                 through |T|;
 *     rinv        the relative error added by inverting the 2D covariance;
 *   de[g]     bounds the error of 3 sqrt(lambda_max) (pixels), including the
 *             cancellation in m^2 - det for nearly isotropic footprints;
 *   rect_in   the tiles every such evaluation covers (empty: x0 > x1);
 *   rect_out  the tiles some such evaluation may cover, vis_out = nonempty.
 * The float32 pipeline's tile rectangle then lies between rect_in and
 * rect_out.  Culling at the near plane is taken as decided alike on both
 * sides (no Gaussian of these workloads lies near z = near).
 */
void or_fp32_bounds(int64_t N, const float *mo, const float *ls, const float *q, const float *sh,
                    int deg, const double *cam16, int W, int H, double near_z, int tile,
                    double *err, double *de, int32_t *rect_in, int32_t *rect_out, int32_t *vis_out)
{
    const ocam cam = mk_cam(cam16, W, H, near_z);
    const double u = ldexp(1.0, -24), safety = 2.0;
    const int TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < N; ++g) {
        gfwd f;
        load_params(mo, ls, q, sh, N, g, &f);
        g_forward(&cam, deg, tile, &f);
        double *e = err + 6 * g;
        for (int i = 0; i < 6; ++i) e[i] = 0;
        de[g] = 0;
        int32_t *ri = rect_in + 4 * g, *ro = rect_out + 4 * g;
        ri[0] = 1; ri[1] = 0; ri[2] = 1; ri[3] = 0;
        ro[0] = 1; ro[1] = 0; ro[2] = 1; ro[3] = 0;
        vis_out[g] = 0;
        if (f.culled) continue;
        const double z = f.pc[2];
        /* camera-space x, y: three products and three sums each */
        double sx = fabs(cam.t[0]), sy = fabs(cam.t[1]);
        for (int k = 0; k < 3; ++k) {
            sx += fabs(cam.R[k] * f.x[k]);
            sy += fabs(cam.R[3 + k] * f.x[k]);
        }
        const double epx = 8 * u * sx, epy = 8 * u * sy;
        /* u = fx x (1/z) + cx: z rounded once, a division, two products, a sum */
        const double du = fabs(cam.fx / z) * epx + 6 * u * fabs(cam.fx * f.pc[0] / z) + u * fabs(f.u);
        const double dv = fabs(cam.fy / z) * epy + 6 * u * fabs(cam.fy * f.pc[1] / z) + u * fabs(f.v);
        /* Sigma = M M^T with |dM_ak| <= 9u s_k (the rotation errs
         * absolutely); Sigma' = T Sigma T^T + 0.3 I with T = J R, carried
         * through |T| (sums of the terms' magnitudes), plus T's own rounding */
        double dS[9], aS[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0, am = 0;
                for (int k = 0; k < 3; ++k) {
                    acc += 9 * u * f.s[k] * (fabs(f.M[3 * a + k]) + fabs(f.M[3 * b + k]));
                    am += fabs(f.M[3 * a + k]) * fabs(f.M[3 * b + k]);
                }
                dS[3 * a + b] = acc + 4 * u * am;
                aS[3 * a + b] = am;            /* >= |Sigma_ab| */
            }
        double Ta[6];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += fabs(f.J[3 * i + k] * cam.R[3 * k + j]);
                Ta[3 * i + j] = acc;
            }
        double dSig2[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        acc += Ta[3 * i + a] * (dS[3 * a + b] + 20 * u * aS[3 * a + b]) * Ta[3 * j + b];
                dSig2[2 * i + j] = safety * (acc + 2 * u * fabs(f.S2[i + j]));
            }
        const double A = f.S2[0], B = f.S2[1], C = f.S2[2];
        const double rinv = safety * (4 * u + 2 * u * (A * C + B * B) / f.det);
        e[0] = safety * du;
        e[1] = safety * dv;
        e[2] = dSig2[0];
        e[3] = dSig2[1];
        e[4] = dSig2[3];
        e[5] = rinv;
        /* lambda_max = m + sqrt(m^2 - det) */
        const double dA = dSig2[0], dC = dSig2[3], dB = dSig2[1];
        const double m = 0.5 * (A + C);
        const double dm = 0.5 * (dA + dC) + u * m;
        const double ddet = dA * C + A * dC + 2 * fabs(B) * dB + 2 * u * (A * C + B * B);
        double disc = m * m - f.det;
        if (disc < 0) disc = 0;
        const double ddisc = 2 * m * dm + ddet + 2 * u * (m * m + f.det);
        const double dsq = ddisc / sqrt(disc > ddisc ? disc : ddisc) + u * sqrt(disc);
        const double dlam = dm + dsq + u * f.lam;
        const double dext = safety * (1.5 * dlam / sqrt(f.lam) + 4 * u * f.ext3);
        de[g] = dext;
        /* radius and tile edges of any such evaluation */
        double rlo = ceil(f.ext3 - dext), rhi = ceil(f.ext3 + dext);
        if (rlo < 0) rlo = 0;
        const double cu[2] = {f.u, f.v}, dd[2] = {safety * du, safety * dv};
        const int lim[2] = {TX - 1, TY - 1};
        int lo_min[2], lo_max[2], hi_min[2], hi_max[2];
        for (int a = 0; a < 2; ++a) {
            const double r1 = u * (fabs(cu[a]) + rhi);   /* rounding of u -+ r */
            lo_min[a] = (int)floor((cu[a] - dd[a] - rhi - r1) / tile);
            lo_max[a] = (int)floor((cu[a] + dd[a] - rlo + r1) / tile);
            hi_min[a] = (int)floor((cu[a] - dd[a] + rlo - r1) / tile);
            hi_max[a] = (int)floor((cu[a] + dd[a] + rhi + r1) / tile);
            if (lo_min[a] < 0) lo_min[a] = 0;
            if (lo_max[a] < 0) lo_max[a] = 0;
            if (hi_min[a] > lim[a]) hi_min[a] = lim[a];
            if (hi_max[a] > lim[a]) hi_max[a] = lim[a];
        }
        if (lo_min[0] <= hi_max[0] && lo_min[1] <= hi_max[1]) {
            ro[0] = lo_min[0]; ro[1] = hi_max[0]; ro[2] = lo_min[1]; ro[3] = hi_max[1];
            vis_out[g] = 1;
        }
        if (rlo > 0 && lo_max[0] <= hi_min[0] && lo_max[1] <= hi_min[1]) {
            ri[0] = lo_max[0]; ri[1] = hi_min[0]; ri[2] = lo_max[1]; ri[3] = hi_min[1];
        }
    }
}

void or_rect_f32(int64_t n, const float *u, const float *v, const int32_t *radius,
                 int W, int H, int tile, int32_t *rect, int32_t *vis)
{
    const int TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
    const float inv = 1.0f / (float)tile;
    for (int64_t g = 0; g < n; ++g) {
        vis[g] = 0;
        rect[4 * g] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = 0;
        if (radius[g] <= 0) continue;
        const float r = (float)radius[g];
        float fx0 = floorf((u[g] - r) * inv), fx1 = floorf((u[g] + r) * inv);
        float fy0 = floorf((v[g] - r) * inv), fy1 = floorf((v[g] + r) * inv);
        if (fx0 < 0.0f) fx0 = 0.0f;
        if (fy0 < 0.0f) fy0 = 0.0f;
        if (fx1 > (float)(TX - 1)) fx1 = (float)(TX - 1);
        if (fy1 > (float)(TY - 1)) fy1 = (float)(TY - 1);
        if (!(fx0 <= fx1 && fy0 <= fy1)) continue;
        vis[g] = 1;
        rect[4 * g] = (int)fx0; rect[4 * g + 1] = (int)fx1;
        rect[4 * g + 2] = (int)fy0; rect[4 * g + 3] = (int)fy1;
    }
}

/*
 * or_bin: the per-tile Gaussian lists of one view.  Gaussian g belongs to
 * every tile in its rectangle (vis[g] != 0).  Each tile's list is ordered by
 * depth rounded to float32, ascending, ties by Gaussian index ascending.
 * Output: CSR offsets toff[TX*TY+1] and indices gidx[F] (F = toff[TX*TY],
 * the caller sizes gidx from or_bin_count).
 */
int64_t or_bin_count(int64_t n, const int32_t *rect, const int32_t *vis)
{
    int64_t F = 0;
    for (int64_t g = 0; g < n; ++g)
        if (vis[g]) F += (int64_t)(rect[4 * g + 1] - rect[4 * g] + 1) * (rect[4 * g + 3] - rect[4 * g + 2] + 1);
    return F;
}

static const float *g_sort_depth;
static int cmp_depth_index(const void *pa, const void *pb)
{
    const int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    const float da = g_sort_depth[a], db = g_sort_depth[b];
    if (da < db) return -1;
    if (da > db) return 1;
    return (a > b) - (a < b);
}

void or_bin(int64_t n, const int32_t *rect, const int32_t *vis, const float *depth_f32,
            int W, int H, int tile, int64_t *toff, int32_t *gidx)
{
    const int TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
    const int64_t nt = (int64_t)TX * TY;
    int64_t *cnt = (int64_t *)calloc((size_t)nt, sizeof(int64_t));
    for (int64_t g = 0; g < n; ++g) {
        if (!vis[g]) continue;
        for (int ty = rect[4 * g + 2]; ty <= rect[4 * g + 3]; ++ty)
            for (int tx = rect[4 * g]; tx <= rect[4 * g + 1]; ++tx) cnt[(int64_t)ty * TX + tx]++;
    }
    toff[0] = 0;
    for (int64_t t = 0; t < nt; ++t) toff[t + 1] = toff[t] + cnt[t];
    for (int64_t t = 0; t < nt; ++t) cnt[t] = toff[t];
    for (int64_t g = 0; g < n; ++g) {
        if (!vis[g]) continue;
        for (int ty = rect[4 * g + 2]; ty <= rect[4 * g + 3]; ++ty)
            for (int tx = rect[4 * g]; tx <= rect[4 * g + 1]; ++tx) gidx[cnt[(int64_t)ty * TX + tx]++] = (int32_t)g;
    }
    free(cnt);
    /* qsort with a file-scope key array: keep it single threaded */
    g_sort_depth = depth_f32;
    for (int64_t t = 0; t < nt; ++t)
        qsort(gidx + toff[t], (size_t)(toff[t + 1] - toff[t]), sizeof(int32_t), cmp_depth_index);
}

/* ------------------------------------------------------------------------ */
/* Rendering (Sec. 2.1 step 2): front-to-back compositing per pixel.         */
/* ------------------------------------------------------------------------ */
typedef struct { double alpha_min, alpha_max, T_min, bg[3]; } oblend;

static double rel_margin(double x, double thr) { return fabs(x - thr) / thr; }

/*
 * or_render_fwd: for every pixel p (centre (i+0.5, j+0.5)) of a W x H view,
 * walk the list of p's tile in order.  For each Gaussian: power =
 * -1/2 (a dx^2 + c dy^2) - b dx dy (skip if > 0); alpha = min(alpha_max,
 * o exp(power)); skip if alpha < alpha_min; T' = T (1 - alpha); stop before
 * blending it if T' < T_min; otherwise C += rgb alpha T, T = T', and
 * n_contrib = list position + 1.  Output C + T bg (img, CHW), T_final,
 * n_contrib, and per pixel the smallest relative distance of any threshold
 * decision to its threshold (margin), plus the per-pixel number of list
 * entries examined (n_eval).
 */
void or_render_fwd(int W, int H, int tile, const int64_t *toff, const int32_t *gidx,
                   const double *xy, const double *conic_o, const double *rgb, const double *params5,
                   double *img, double *T_final, int32_t *n_contrib, double *margin, int32_t *n_eval)
{
    const oblend bp = {params5[0], params5[1], params5[2], {params5[3], params5[4], params5[5]}};
    const int TX = (W + tile - 1) / tile;
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const int64_t t = (int64_t)(py / tile) * TX + px / tile;
            double T = 1.0, C[3] = {0, 0, 0}, marg = INFINITY;
            int32_t nc = 0, ne = 0;
            for (int64_t k = toff[t]; k < toff[t + 1]; ++k) {
                const int32_t g = gidx[k];
                ne = (int32_t)(k - toff[t] + 1);
                const double dx = px + 0.5 - xy[2 * g], dy = py + 0.5 - xy[2 * g + 1];
                const double a = conic_o[4 * g], b = conic_o[4 * g + 1], c = conic_o[4 * g + 2];
                const double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                if (power > 0) continue;
                const double oa = conic_o[4 * g + 3] * exp(power);
                double m1 = rel_margin(oa, bp.alpha_max);
                const double alpha = oa < bp.alpha_max ? oa : bp.alpha_max;
                double m2 = rel_margin(alpha, bp.alpha_min);
                if (m1 < marg) marg = m1;
                if (m2 < marg) marg = m2;
                if (alpha < bp.alpha_min) continue;
                const double Tn = T * (1.0 - alpha);
                double m3 = rel_margin(Tn, bp.T_min);
                if (m3 < marg) marg = m3;
                if (Tn < bp.T_min) break;
                for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
                T = Tn;
                nc = (int32_t)(k - toff[t] + 1);
            }
            const int64_t p = (int64_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) img[ch * HW + p] = C[ch] + T * bp.bg[ch];
            T_final[p] = T;
            n_contrib[p] = nc;
            if (margin) margin[p] = marg;
            if (n_eval) n_eval[p] = ne;
        }
}

/*
 * The set of results a float32 evaluation of the compositing may give.
 *
 * The definition above decides, per pixel and list entry, three things with
 * a threshold: whether the Gaussian is in the pixel's tile list (tile
 * membership of its rectangle), whether it passes (power <= 0 and alpha >=
 * alpha_min), and whether blending it would take T below T_min (stop).  A
 * float32 evaluation with inputs within the bounds of or_fp32_bounds may
 * decide any of them the other way when the exact quantity lies within that
 * evaluation's error of the threshold; everywhere else both decide alike and
 * differ only by rounding.  or_render_fwd_set walks each pixel's list as
 * or_render_fwd does (the primary result, identical to it), and wherever a
 * decision is ambiguous it also follows the other outcome to the end of the
 * list: every leaf of that tree is an admissible result.
 *
 * Relative error bound of alpha at an entry (from the power's error dp):
 *   dp = m0 + 8u (|a| dx^2/2 + |b dx dy| + |c| dy^2/2)     (evaluation)
 *        + |g_x| du + |g_y| dv                              (centre)
 *        + (g_x^2 dA + 2 |g_x g_y| dB + g_y^2 dC) / 2       (2D covariance)
 *        + |power| rinv                                     (inversion)
 * with g = (a dx + b dy, b dx + c dy) the gradient of power in the centre
 * (err == NULL: exact screen-space inputs, only the first line).  The alpha
 * cut (and the clamp) can go the other way only where ln(o) + power lies
 * within dp of ln(alpha_min) (of ln(alpha_max)); a blended alpha errs by at
 * most m_alpha = expm1(dp) relative, and the transmittance carries, after
 * each blend, the relative error bound sum alpha/(1 - alpha) m_alpha +
 * 2u/(1 - alpha).
 *
 * Membership: with rect != NULL the lists are built from the rectangles
 * every evaluation may cover (or_fp32_bounds' rect_out); an entry belongs to
 * the primary list when its tile lies in rect[g] (the exact rectangle) and
 * is certain when it lies in rect_in[g].
 */
typedef struct {
    double C[3], T, eT;
    int32_t nc, pos;
} or_state;

typedef struct {
    int W, H, tile, TX;
    const int64_t *toff;
    const int32_t *gidx;
    const double *xy, *conic_o, *rgb, *err;
    const int32_t *rect, *rect_in;
    oblend bp;
    double m0;
} or_setin;

typedef struct {
    double *alt;        /* NULL: count only; else 5 doubles per leaf */
    int n, cap, overflow, clamp_amb;
} or_setout;

enum { OUT_SKIP = 1, OUT_BLEND = 2, OUT_STOP = 4 };

static int in_rect(const int32_t *r, int tx, int ty) { return r[0] <= tx && tx <= r[1] && r[2] <= ty && ty <= r[3]; }

static void set_leaf(const or_setin *s, const or_state *st, or_setout *o)
{
    if (o->n >= o->cap) { o->overflow = 1; return; }
    if (o->alt) {
        double *a = o->alt + 5 * (int64_t)o->n;
        for (int ch = 0; ch < 3; ++ch) a[ch] = st->C[ch] + st->T * s->bp.bg[ch];
        a[3] = st->T;
        a[4] = st->nc;
    }
    o->n++;
}

/* Walks pixel (px, py) of tile t from list index k in state st; alternative
 * outcomes are walked recursively and recorded as leaves; the walk's own end
 * state is returned in *end (the primary result at the top level). */
static void set_walk(const or_setin *s, int px, int py, int64_t t, int64_t k, or_state st, int primary,
                     or_setout *o, or_state *end)
{
    const double u = ldexp(1.0, -24);
    const int tx = px / s->tile, ty = py / s->tile;
    for (; k < s->toff[t + 1]; ++k) {
        const int32_t g = s->gidx[k];
        int prim = 1, amb_memb = 0;
        if (s->rect) {
            prim = in_rect(s->rect + 4 * g, tx, ty);
            amb_memb = !in_rect(s->rect_in + 4 * g, tx, ty);
        }
        const double dx = px + 0.5 - s->xy[2 * g], dy = py + 0.5 - s->xy[2 * g + 1];
        const double a = s->conic_o[4 * g], b = s->conic_o[4 * g + 1], c = s->conic_o[4 * g + 2];
        const double o_ = s->conic_o[4 * g + 3];
        const double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        double dp = s->m0 + 8 * u * (0.5 * fabs(a) * dx * dx + fabs(b * dx * dy) + 0.5 * fabs(c) * dy * dy);
        if (s->err) {
            const double *e = s->err + 6 * g;
            const double gx = fabs(a * dx + b * dy), gy = fabs(b * dx + c * dy);
            dp += gx * e[0] + gy * e[1] + 0.5 * (gx * gx * e[2] + 2 * gx * gy * e[3] + gy * gy * e[4])
                + fabs(power) * e[5];
        }
        const double ma = expm1(dp);
        const double oa = o_ * exp(power);
        const double alpha = oa < s->bp.alpha_max ? oa : s->bp.alpha_max;
        /* pass: power <= 0 and alpha >= alpha_min.  A float32 evaluation has
         * o exp(power') with |power' - power| <= dp, so the alpha cut can go
         * the other way only when ln(o) + power lies within dp of
         * ln(alpha_min) (the clamp at alpha_max is far above the cut) */
        const double lcut = log(s->bp.alpha_min / o_);
        const int pass_p = power <= 0 && alpha >= s->bp.alpha_min;
        const int pass_amb = (fabs(power) <= dp && power + dp >= lcut)
                          || (fabs(power - lcut) <= dp && power <= dp);
        const double Tn = st.T * (1.0 - alpha);
        const double eTn = st.eT + alpha / (1.0 - alpha) * ma + 2 * u / (1.0 - alpha);
        const int stop_p = Tn < s->bp.T_min;
        const int stop_amb = fabs(Tn - s->bp.T_min) <= s->bp.T_min * (eTn + 4 * u);
        /* outcome of the exact decisions, and the set of possible ones */
        const int out_p = !(prim && pass_p) ? OUT_SKIP : stop_p ? OUT_STOP : OUT_BLEND;
        int outs = 0;
        for (int inc = 0; inc < 2; ++inc) {
            if (inc != prim && !amb_memb) continue;
            if (!inc) { outs |= OUT_SKIP; continue; }
            for (int ps = 0; ps < 2; ++ps) {
                if (ps != pass_p && !pass_amb) continue;
                if (!ps) { outs |= OUT_SKIP; continue; }
                outs |= stop_p ? OUT_STOP : OUT_BLEND;
                if (stop_amb) outs |= stop_p ? OUT_BLEND : OUT_STOP;
            }
        }
        if (primary && out_p == OUT_BLEND && fabs(power - log(s->bp.alpha_max / o_)) <= dp) o->clamp_amb = 1;
        for (int alt = OUT_SKIP; alt <= OUT_STOP; alt <<= 1) {
            if (alt == out_p || !(outs & alt)) continue;
            if (o->n >= o->cap) { o->overflow = 1; continue; }
            or_state sa = st;
            if (alt == OUT_STOP) { set_leaf(s, &sa, o); continue; }
            if (alt == OUT_SKIP) {
                sa.pos += prim;
            } else {
                sa.pos += 1;
                for (int ch = 0; ch < 3; ++ch) sa.C[ch] += s->rgb[3 * g + ch] * alpha * sa.T;
                sa.T = Tn;
                sa.eT = eTn;
                sa.nc = sa.pos;
            }
            or_state e2;
            set_walk(s, px, py, t, k + 1, sa, 0, o, &e2);
            set_leaf(s, &e2, o);
        }
        if (out_p == OUT_STOP) break;
        if (out_p == OUT_SKIP) { st.pos += prim; continue; }
        st.pos += 1;
        for (int ch = 0; ch < 3; ++ch) st.C[ch] += s->rgb[3 * g + ch] * alpha * st.T;
        st.T = Tn;
        st.eT = eTn;
        st.nc = st.pos;
    }
    *end = st;
}

/*
 * or_render_fwd_set: img, T_final and n_contrib as or_render_fwd (the exact
 * decisions), plus the other admissible results of every pixel.
 * flags[p]: 1 = other results exist, 2 = alpha within its bound of the
 * alpha_max clamp at a blended entry (the value is continuous there, the
 * gradient is not), 4 = more than `cap` leaves (the set is incomplete).
 * With alt == NULL only n_alt[p] (the count of other results) is written;
 * with alt != NULL (5 doubles per result: r, g, b, T, n_contrib, pixel by
 * pixel at alt_off[p]) the results are written.  err == NULL: exact
 * screen-space inputs; rect == NULL: exact membership (lists as given).
 */
void or_render_fwd_set(int W, int H, int tile, const int64_t *toff, const int32_t *gidx,
                       const double *xy, const double *conic_o, const double *rgb, const double *params5,
                       const double *err, const int32_t *rect, const int32_t *rect_in, double m0, int cap,
                       double *img, double *T_final, int32_t *n_contrib, int32_t *flags, int32_t *n_alt,
                       const int64_t *alt_off, double *alt)
{
    or_setin s;
    s.W = W; s.H = H; s.tile = tile; s.TX = (W + tile - 1) / tile;
    s.toff = toff; s.gidx = gidx; s.xy = xy; s.conic_o = conic_o; s.rgb = rgb; s.err = err;
    s.rect = rect; s.rect_in = rect_in; s.m0 = m0;
    s.bp.alpha_min = params5[0]; s.bp.alpha_max = params5[1]; s.bp.T_min = params5[2];
    for (int ch = 0; ch < 3; ++ch) s.bp.bg[ch] = params5[3 + ch];
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const int64_t p = (int64_t)py * W + px;
            const int64_t t = (int64_t)(py / tile) * s.TX + px / tile;
            or_setout o;
            o.alt = alt ? alt + 5 * alt_off[p] : NULL;
            o.n = 0; o.cap = cap; o.overflow = 0; o.clamp_amb = 0;
            if (alt) o.cap = (int)(alt_off[p + 1] - alt_off[p]);
            or_state st = {{0, 0, 0}, 1.0, 0.0, 0, 0};
            or_state end;
            set_walk(&s, px, py, t, toff[t], st, 1, &o, &end);
            if (!alt) {
                for (int ch = 0; ch < 3; ++ch) img[ch * HW + p] = end.C[ch] + end.T * s.bp.bg[ch];
                T_final[p] = end.T;
                n_contrib[p] = end.nc;
                flags[p] = (o.n > 0 ? 1 : 0) | (o.clamp_amb ? 2 : 0) | (o.overflow ? 4 : 0);
                n_alt[p] = o.n;
            }
        }
}

/*
 * or_render_bwd: vector-Jacobian product of <dL/dimg, img> with respect to
 * the per-Gaussian screen-space features of one view.  Per pixel the forward
 * walk is repeated, the contributors (alpha, T before blending, exp value,
 * offsets) are kept, and they are visited back to front with the colour
 * behind B (B = bg behind the last contributor; B <- alpha rgb + (1-alpha) B):
 *   dC/drgb_j = alpha_j T_j,   dC/dalpha_j = T_j (rgb_j - B_j),
 *   dalpha/do = G, dalpha/dpower = alpha (both 0 when alpha is clamped),
 *   dpower/d(a,b,c) = (-dx^2/2, -dx dy, -dy^2/2),
 *   dpower/d(u,v) = (a dx + b dy, b dx + c dy).
 * Accumulates into g2d[9*n] = (du, dv, da, db, dc, do, dr, dg, db) (+=).
 */
void or_render_bwd(int W, int H, int tile, const int64_t *toff, const int32_t *gidx,
                   const double *xy, const double *conic_o, const double *rgb, const double *params5,
                   const double *dimg, double *g2d)
{
    const oblend bp = {params5[0], params5[1], params5[2], {params5[3], params5[4], params5[5]}};
    const int TX = (W + tile - 1) / tile;
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel
    {
        int cap = 256;
        int32_t *cg = (int32_t *)malloc(sizeof(int32_t) * cap);
        double *ca = (double *)malloc(sizeof(double) * cap * 6);
#pragma omp for schedule(dynamic, 4)
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < W; ++px) {
                const int64_t t = (int64_t)(py / tile) * TX + px / tile;
                const int64_t p = (int64_t)py * W + px;
                double T = 1.0;
                int n = 0;
                for (int64_t k = toff[t]; k < toff[t + 1]; ++k) {
                    const int32_t g = gidx[k];
                    const double dx = px + 0.5 - xy[2 * g], dy = py + 0.5 - xy[2 * g + 1];
                    const double a = conic_o[4 * g], b = conic_o[4 * g + 1], c = conic_o[4 * g + 2];
                    const double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                    if (power > 0) continue;
                    const double G = exp(power);
                    const double oa = conic_o[4 * g + 3] * G;
                    const int clamped = !(oa < bp.alpha_max);
                    const double alpha = clamped ? bp.alpha_max : oa;
                    if (alpha < bp.alpha_min) continue;
                    const double Tn = T * (1.0 - alpha);
                    if (Tn < bp.T_min) break;
                    if (n == cap) {
                        cap *= 2;
                        cg = (int32_t *)realloc(cg, sizeof(int32_t) * cap);
                        ca = (double *)realloc(ca, sizeof(double) * cap * 6);
                    }
                    cg[n] = g;
                    ca[6 * n] = alpha; ca[6 * n + 1] = T; ca[6 * n + 2] = G;
                    ca[6 * n + 3] = dx; ca[6 * n + 4] = dy; ca[6 * n + 5] = clamped;
                    ++n;
                    T = Tn;
                }
                const double dC[3] = {dimg[p], dimg[HW + p], dimg[2 * HW + p]};
                double Bb[3] = {bp.bg[0], bp.bg[1], bp.bg[2]};
                for (int j = n - 1; j >= 0; --j) {
                    const int32_t g = cg[j];
                    const double alpha = ca[6 * j], Tj = ca[6 * j + 1], G = ca[6 * j + 2];
                    const double dx = ca[6 * j + 3], dy = ca[6 * j + 4];
                    const int clamped = ca[6 * j + 5] != 0;
                    const double a = conic_o[4 * g], b = conic_o[4 * g + 1], c = conic_o[4 * g + 2];
                    double dalpha = 0;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double col = rgb[3 * g + ch];
#pragma omp atomic
                        g2d[9 * (int64_t)g + 6 + ch] += alpha * Tj * dC[ch];
                        dalpha += Tj * (col - Bb[ch]) * dC[ch];
                        Bb[ch] = alpha * col + (1.0 - alpha) * Bb[ch];
                    }
                    if (clamped) continue;
                    const double dpow = alpha * dalpha;
                    const double gu = (a * dx + b * dy) * dpow, gv = (b * dx + c * dy) * dpow;
                    const double ga = -0.5 * dx * dx * dpow, gb = -dx * dy * dpow, gc = -0.5 * dy * dy * dpow;
                    const double go = G * dalpha;
#pragma omp atomic
                    g2d[9 * (int64_t)g + 0] += gu;
#pragma omp atomic
                    g2d[9 * (int64_t)g + 1] += gv;
#pragma omp atomic
                    g2d[9 * (int64_t)g + 2] += ga;
#pragma omp atomic
                    g2d[9 * (int64_t)g + 3] += gb;
#pragma omp atomic
                    g2d[9 * (int64_t)g + 4] += gc;
#pragma omp atomic
                    g2d[9 * (int64_t)g + 5] += go;
                }
            }
        free(cg);
        free(ca);
    }
}

/* ------------------------------------------------------------------------ */
/* Backward of the Gaussian transformation (chain rule to the 59 parameters) */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double *A, const double *B, double *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = acc;
        }
}

/*
 * or_preprocess_bwd: for one view, given per-Gaussian gradients g2d[9n] with
 * respect to (u, v, a, b, c, o, r, g, b) (the clamped colour), accumulate
 * dL/dparams into grad[60n] laid out as (x, y, z, logit, logs0..2, pad,
 * qw, qx, qy, qz, sh flat 0..47).  Gaussians the forward culls (z <= near or
 * singular 2D covariance) or that touch no tile get no gradient.
 * Chain: colour (clamp at 0 gives 0) -> SH coefficients and the viewing
 * direction -> mean; conic -> 2D covariance (dQ^-1 = -Q^-1 dQ Q^-1) -> 3D
 * covariance and Jacobian -> camera-space mean (the off-axis clamp passes no
 * x/z gradient, and its bound scales with z) -> mean; 3D covariance ->
 * M = Rq S -> scale (through exp) and normalised quaternion -> quaternion
 * (through the normalisation); opacity through the sigmoid.
 */
void or_preprocess_bwd(int64_t N, const float *mo, const float *ls, const float *q, const float *sh,
                       int deg, const double *cam16, int W, int H, double near_z, int tile,
                       const double *g2d, double *grad)
{
    const ocam cam = mk_cam(cam16, W, H, near_z);
    const int nk = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < N; ++g) {
        gfwd f;
        load_params(mo, ls, q, sh, N, g, &f);
        g_forward(&cam, deg, tile, &f);
        if (!f.visible) continue;
        const double *G2 = g2d + 9 * g;
        double *out = grad + 60 * g;
        double dx[3] = {0, 0, 0};
        /* opacity */
        out[3] += G2[5] * f.o * (1.0 - f.o);
        /* colour -> SH coefficients and direction */
        double drgb[3];
        for (int ch = 0; ch < 3; ++ch) drgb[ch] = f.rgb_raw[ch] < 0 ? 0 : G2[6 + ch];
        double ddir[3] = {0, 0, 0};
        for (int k = 0; k < nk; ++k) {
            double w = 0;
            for (int ch = 0; ch < 3; ++ch) {
                out[12 + 3 * k + ch] += f.Y[k] * drgb[ch];
                w += f.sh[k][ch] * drgb[ch];
            }
            for (int i = 0; i < 3; ++i) ddir[i] += w * f.dY[k][i];
        }
        {
            double dd = 0;
            for (int i = 0; i < 3; ++i) dd += f.dir[i] * ddir[i];
            for (int i = 0; i < 3; ++i) dx[i] += (ddir[i] - f.dir[i] * dd) / f.dist;
        }
        /* conic -> 2D covariance.  Q = [[a,b],[b,c]]; dL/dQ (full) = [[da, db/2],[db/2, dc]] */
        const double Q[4] = {f.conic[0], f.conic[1], f.conic[1], f.conic[2]};
        const double Gq[4] = {G2[2], 0.5 * G2[3], 0.5 * G2[3], G2[4]};
        double QG[4], dS2[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) QG[2 * i + j] = Q[2 * i] * Gq[j] + Q[2 * i + 1] * Gq[2 + j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) dS2[2 * i + j] = -(QG[2 * i] * Q[j] + QG[2 * i + 1] * Q[2 + j]);
        /* Sigma' = T Sigma T^T + 0.3 I  ->  dSigma = T^T dS2 T,  dT = 2 dS2 T Sigma */
        double dSig[9], dT[6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) acc += f.T[3 * i + a] * dS2[2 * i + j] * f.T[3 * j + b];
                dSig[3 * a + b] = acc;
            }
        for (int i = 0; i < 2; ++i)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int j = 0; j < 2; ++j)
                    for (int a = 0; a < 3; ++a) acc += dS2[2 * i + j] * f.T[3 * j + a] * f.Sig[3 * a + b];
                dT[3 * i + b] = 2.0 * acc;
            }
        /* T = J Rcam  ->  dJ = dT Rcam^T */
        double dJ[6];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += dT[3 * i + j] * cam.R[3 * k + j];
                dJ[3 * i + k] = acc;
            }
        const double z = f.pc[2], z2 = z * z, z3 = z2 * z;
        double dpc[3] = {0, 0, 0};
        /* J00 = fx/z, J02 = -fx xt/z^2, J11 = fy/z, J12 = -fy yt/z^2 */
        dpc[2] += dJ[0] * (-cam.fx / z2) + dJ[2] * (2.0 * cam.fx * f.xt / z3)
                + dJ[4] * (-cam.fy / z2) + dJ[5] * (2.0 * cam.fy * f.yt / z3);
        const double dxt = dJ[2] * (-cam.fx / z2), dyt = dJ[5] * (-cam.fy / z2);
        if (f.clamp_x) dpc[2] += dxt * f.Lx; else dpc[0] += dxt;
        if (f.clamp_y) dpc[2] += dyt * f.Ly; else dpc[1] += dyt;
        /* u = fx x/z + cx, v = fy y/z + cy */
        dpc[0] += G2[0] * cam.fx / z;
        dpc[2] += G2[0] * (-cam.fx * f.pc[0] / z2);
        dpc[1] += G2[1] * cam.fy / z;
        dpc[2] += G2[1] * (-cam.fy * f.pc[1] / z2);
        /* pc = R x + t */
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) dx[k] += cam.R[3 * i + k] * dpc[i];
        for (int i = 0; i < 3; ++i) out[i] += dx[i];
        /* Sigma = M M^T -> dM = (dSig + dSig^T) M */
        double dSs[9], dM[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dSs[3 * i + j] = dSig[3 * i + j] + dSig[3 * j + i];
        mat3_mul(dSs, f.M, dM);
        /* M = Rq diag(s) */
        double dRq[9];
        for (int j = 0; j < 3; ++j) {
            double ds = 0;
            for (int i = 0; i < 3; ++i) {
                ds += dM[3 * i + j] * f.Rq[3 * i + j];
                dRq[3 * i + j] = dM[3 * i + j] * f.s[j];
            }
            out[4 + j] += ds * f.s[j];
        }
        /* Rq(qn) */
        const double w = f.qn[0], x = f.qn[1], y = f.qn[2], zq = f.qn[3];
        const double *d = dRq;
        double dqn[4];
        dqn[0] = 2 * (-zq * d[1] + y * d[2] + zq * d[3] - x * d[5] - y * d[6] + x * d[7]);
        dqn[1] = 2 * (y * d[1] + zq * d[2] + y * d[3] - 2 * x * d[4] - w * d[5] + zq * d[6] + w * d[7] - 2 * x * d[8]);
        dqn[2] = 2 * (-2 * y * d[0] + x * d[1] + w * d[2] + x * d[3] + zq * d[5] - w * d[6] + zq * d[7] - 2 * y * d[8]);
        dqn[3] = 2 * (-2 * zq * d[0] - w * d[1] + x * d[2] + w * d[3] - 2 * zq * d[4] + y * d[5] + x * d[6] + y * d[7]);
        double pr = 0;
        for (int i = 0; i < 4; ++i) pr += f.qn[i] * dqn[i];
        for (int i = 0; i < 4; ++i) out[8 + i] += (dqn[i] - f.qn[i] * pr) / f.qnorm;
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
