// K9: Adam over every Gaussian parameter (Sec. 4), with the batch-size
// scaling of Eq. 1 (lr' = lr sqrt(B)) and Eq. 2 (beta' = beta^B) folded into
// the arguments by the host.  A pure streaming kernel: per float4 it reads
// p, g, m, v and writes p, m, v (112 bytes), coalesced and vectorised;
// gridDim.y selects one of the 15 float4 planes (mo, ls, q, sh[0..11]).
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ float4 *plane_ptr(const SceneMut &s, int pl)
{
    return pl == 0 ? s.mo : pl == 1 ? s.ls : pl == 2 ? s.q : s.sh + (int64_t)(pl - 3) * s.N;
}

__device__ __forceinline__ const float4 *plane_ptr(const SceneView &s, int pl)
{
    return pl == 0 ? s.mo : pl == 1 ? s.ls : pl == 2 ? s.q : s.sh + (int64_t)(pl - 3) * s.N;
}

// One Adam update; ibc1, ibc2 = 1 / (1 - b^t).  The divisions are
// reciprocal-multiplies (within an ulp or two of the quotients).
__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                      float ibc1, float ibc2, float eps)
{
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    const float mh = m * ibc1, vh = v * ibc2;
    p -= lr * mh * __frcp_rn(sqrtf(vh) + eps);
}

__device__ __forceinline__ void adam4(float4 &p, const float4 &g, float4 &m, float4 &v, const float4 &lr, float b1,
                                      float b2, float ibc1, float ibc2, float eps)
{
    adam1(p.x, g.x, m.x, v.x, lr.x, b1, b2, ibc1, ibc2, eps);
    adam1(p.y, g.y, m.y, v.y, lr.y, b1, b2, ibc1, ibc2, eps);
    adam1(p.z, g.z, m.z, v.z, lr.z, b1, b2, ibc1, ibc2, eps);
    adam1(p.w, g.w, m.w, v.w, lr.w, b1, b2, ibc1, ibc2, eps);
}

// A step whose binning overflowed the fragment buffer or whose sort gave up
// (a look-back wait ran out) has an incomplete or wrong gradient: the update
// and the step counter are skipped, so the parameters stay as they were.
__device__ __forceinline__ bool step_failed(const DevStatus *status)
{
    const int c = status->code;
    return c == GS_ERR_CAPACITY || c == GS_ERR_TIMEOUT;
}

// Advances the device-side step counter (graph-replayable training loops) and
// stores the bias corrections 1 - b1^t, 1 - b2^t next to it for the update.
__global__ void k_step_tick(long long *dstep, float b1, float b2, const DevStatus *status)
{
    if (step_failed(status)) return;
    const long long t = dstep[0] + 1;
    dstep[0] = t;
    float *bc = reinterpret_cast<float *>(dstep + 1);
    bc[0] = (float)(1.0 - pow((double)b1, (double)t));
    bc[1] = (float)(1.0 - pow((double)b2, (double)t));
}

// Grid-stride over one plane per gridDim.y, two float4 per thread per round
// (eight 16-byte loads in flight).  The plane's learning rates are picked with
// static selects (a runtime index into the parameter struct would copy it to
// local memory).
__global__ void __launch_bounds__(256) k_adam(SceneMut P, SceneView G, SceneMut M, SceneMut V, AdamArgs a,
                                              const DevStatus *status)
{
    if (step_failed(status)) return;             // the step's gradient is incomplete: skip the update
    float bc1 = a.bc1, bc2 = a.bc2;
    if (a.dstep) {
        const float *bc = reinterpret_cast<const float *>(a.dstep + 1);
        bc1 = bc[0];
        bc2 = bc[1];
    }
    const float ibc1 = 1.f / bc1, ibc2 = 1.f / bc2;
    const int pl = blockIdx.y;
    float4 lr = make_float4(a.lr[0][0], a.lr[0][1], a.lr[0][2], a.lr[0][3]);
#pragma unroll
    for (int k = 1; k < 15; ++k)
        if (pl == k) lr = make_float4(a.lr[k][0], a.lr[k][1], a.lr[k][2], a.lr[k][3]);
    float4 *pp = plane_ptr(P, pl);
    const float4 *gp = plane_ptr(G, pl);
    float4 *mp = plane_ptr(M, pl);
    float4 *vp = plane_ptr(V, pl);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.N; i += 2 * stride) {
        const int64_t i2 = i + stride;
        // visible-only Adam: an unseen Gaussian's p, m, v are neither read nor written
        const bool one = !a.vis || a.vis[i];
        const bool two = i2 < P.N && (!a.vis || a.vis[i2]);
        float4 p, m, v, g, p2, m2, v2, g2;
        if (one) {
            p = pp[i];
            m = mp[i];
            v = vp[i];
            g = gp[i];
        }
        if (two) {
            p2 = pp[i2];
            m2 = mp[i2];
            v2 = vp[i2];
            g2 = gp[i2];
        }
        if (one) {
            adam4(p, g, m, v, lr, a.b1, a.b2, ibc1, ibc2, a.eps);
            pp[i] = p;
            mp[i] = m;
            vp[i] = v;
        }
        if (two) {
            adam4(p2, g2, m2, v2, lr, a.b1, a.b2, ibc1, ibc2, a.eps);
            pp[i2] = p2;
            mp[i2] = m2;
            vp[i2] = v2;
        }
    }
}

}  // namespace

void launch_adam(const SceneMut &p, const SceneView &g, const SceneMut &m, const SceneMut &v, const AdamArgs &a,
                 const DevStatus *status, cudaStream_t st)
{
    if (a.dstep) {
        k_step_tick<<<1, 1, 0, st>>>(a.dstep, a.b1, a.b2, status);
        count_launches(1);
    }
    if (p.N == 0) return;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t bx = ((int64_t)sms * 8 + 14) / 15;
    const int64_t need = (p.N + 255) / 256;
    if (bx > need) bx = need;
    if (bx < 1) bx = 1;
    k_adam<<<dim3((unsigned)bx, 15), 256, 0, st>>>(p, g, m, v, a, status);
    count_launches(1);
}

}  // namespace gs
