// Densification (App. A.1): clone or split the Gaussians whose projected
// position keeps moving (the mean length of their per-view position gradient
// over the steps since the last densification reaches a threshold), by whether
// their largest scale exceeds a threshold; prune those of low opacity; reset
// opacity now and then.
//
// One pass decides each Gaussian's action and output count (0, 1 or 2); an
// exclusive scan turns the counts into output positions (stream compaction
// that keeps the input order); a second pass writes every output row of the
// parameters and both Adam moments.  All decisions are float32 comparisons
// with explicitly rounded operands, so they are reproducible exactly.
#include "gs_internal.cuh"

namespace gs {
namespace {

enum : uint32_t { D_PRUNE = 0u, D_KEEP = 1u, D_CLONE = 2u, D_SPLIT = 3u };

__device__ __forceinline__ uint32_t densify_action(const float4 &mo, const float4 &ls, float acc, uint32_t cnt,
                                                   const DensifyArgs &d)
{
    if (!(mo.w >= d.logit_min)) return D_PRUNE;              // opacity below the minimum
    const bool grow = cnt > 0u && acc >= __fmul_rn(d.grad_thr, (float)cnt);
    if (!grow) return D_KEEP;
    const float smax = fmaxf(ls.x, fmaxf(ls.y, ls.z));
    return smax <= d.log_scale_thr ? D_CLONE : D_SPLIT;
}

__device__ __forceinline__ uint32_t action_count(uint32_t a)
{
    return a == D_PRUNE ? 0u : a == D_KEEP ? 1u : 2u;
}

__global__ void __launch_bounds__(256) k_densify_count(SceneView p, const float *acc, const uint32_t *cnt,
                                                       DensifyArgs d, uint32_t *counts)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.N; g += (int64_t)gridDim.x * blockDim.x)
        counts[g] = action_count(densify_action(p.mo[g], p.ls[g], acc[g], cnt[g], d));
}

// Plane k of a scene (0: mo, 1: ls, 2: q, 3..14: sh).
__device__ __forceinline__ const float4 *plane_of(const SceneView &s, int k)
{
    return k == 0 ? s.mo : k == 1 ? s.ls : k == 2 ? s.q : s.sh + (int64_t)(k - 3) * s.N;
}
__device__ __forceinline__ float4 *plane_of(const SceneMut &s, int k)
{
    return k == 0 ? s.mo : k == 1 ? s.ls : k == 2 ? s.q : s.sh + (int64_t)(k - 3) * s.N;
}

__global__ void __launch_bounds__(256) k_densify_emit(SceneView p, SceneView m, SceneView v, const float *acc,
                                                      const uint32_t *cnt, const float *normals, DensifyArgs d,
                                                      const uint32_t *offsets, const unsigned long long *total,
                                                      SceneMut po, SceneMut mo_, SceneMut vo)
{
    if (*total > (unsigned long long)po.N) return;          // over capacity: nothing is written
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.N; g += (int64_t)gridDim.x * blockDim.x) {
        const float4 pm = p.mo[g], pl = p.ls[g];
        const uint32_t a = densify_action(pm, pl, acc[g], cnt[g], d);
        if (a == D_PRUNE) continue;
        const int64_t o = offsets[g];
        if (a == D_KEEP || a == D_CLONE) {
#pragma unroll 1
            for (int k = 0; k < 15; ++k) {
                const float4 x = plane_of(p, k)[g];
                plane_of(po, k)[o] = x;
                plane_of(mo_, k)[o] = plane_of(m, k)[g];
                plane_of(vo, k)[o] = plane_of(v, k)[g];
                if (a == D_CLONE) {                          // the copy starts with zero moments
                    plane_of(po, k)[o + 1] = x;
                    plane_of(mo_, k)[o + 1] = z4;
                    plane_of(vo, k)[o + 1] = z4;
                }
            }
            continue;
        }
        // split: two children at mean + Rq diag(s) xi_k, scale / split_div
        const float4 q = p.q[g];
        const float inv = 1.f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        const float w = q.x * inv, x = q.y * inv, y = q.z * inv, zq = q.w * inv;
        const float R[9] = {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq), 2.f * (x * zq + w * y),
                            2.f * (x * y + w * zq), 1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x),
                            2.f * (x * zq - w * y), 2.f * (y * zq + w * x), 1.f - 2.f * (x * x + y * y)};
        const float s[3] = {expf(pl.x), expf(pl.y), expf(pl.z)};
        const float4 cls = make_float4(pl.x - d.log_div, pl.y - d.log_div, pl.z - d.log_div, 0.f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float *xi = normals + 6 * g + 3 * c;
            const float l0 = s[0] * xi[0], l1 = s[1] * xi[1], l2 = s[2] * xi[2];
            const float4 cm = make_float4(pm.x + R[0] * l0 + R[1] * l1 + R[2] * l2,
                                          pm.y + R[3] * l0 + R[4] * l1 + R[5] * l2,
                                          pm.z + R[6] * l0 + R[7] * l1 + R[8] * l2, pm.w);
            po.mo[o + c] = cm;
            po.ls[o + c] = cls;
            po.q[o + c] = q;
            for (int k = 3; k < 15; ++k) plane_of(po, k)[o + c] = plane_of(p, k)[g];
            for (int k = 0; k < 15; ++k) {
                plane_of(mo_, k)[o + c] = z4;
                plane_of(vo, k)[o + c] = z4;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_reset_opacity(SceneMut p, SceneMut m, SceneMut v, float logit_max)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.N; g += (int64_t)gridDim.x * blockDim.x) {
        float4 a = p.mo[g];
        a.w = fminf(a.w, logit_max);
        p.mo[g] = a;
        m.mo[g].w = 0.f;
        v.mo[g].w = 0.f;
    }
}

unsigned grid_for(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535 * 16 ? 65535 * 16 : b));
}

}  // namespace

void launch_densify_count(const SceneView &p, const float *acc, const uint32_t *cnt, const DensifyArgs &d,
                          uint32_t *counts, cudaStream_t st)
{
    if (p.N <= 0) return;
    k_densify_count<<<grid_for(p.N), 256, 0, st>>>(p, acc, cnt, d, counts);
    count_launches(1);
}

void launch_densify_emit(const SceneView &p, const SceneView &m, const SceneView &v, const float *acc,
                         const uint32_t *cnt, const float *normals, const DensifyArgs &d, const uint32_t *offsets,
                         const unsigned long long *total, const SceneMut &po, const SceneMut &mo,
                         const SceneMut &vo, cudaStream_t st)
{
    if (p.N <= 0) return;
    k_densify_emit<<<grid_for(p.N), 256, 0, st>>>(p, m, v, acc, cnt, normals, d, offsets, total, po, mo, vo);
    count_launches(1);
}

void launch_reset_opacity(const SceneMut &p, const SceneMut &m, const SceneMut &v, float logit_max, cudaStream_t st)
{
    if (p.N <= 0) return;
    k_reset_opacity<<<grid_for(p.N), 256, 0, st>>>(p, m, v, logit_max);
    count_launches(1);
}

}  // namespace gs
