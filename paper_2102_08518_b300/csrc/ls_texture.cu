// Linear texture fetch evaluation of tensor-product splines (Sec. 4.4.1).
//
// The paper folds pairs of terms into hardware linear interpolation: for two
// neighbouring sites s, s+1 along an axis with non-negative weights w_a, w_b,
//     w_a c_s + w_b c_{s+1} = (w_a + w_b) * lerp(c_s, c_{s+1}, w_b / (w_a + w_b)),
// and a trilinear texture fetch does this on all three axes at once.  A
// tensor-product spline with at most four sites per axis then needs at most
// 2 x 2 x 2 fetches (the tricubic: 8 instead of 64 gathers).  The texture
// unit's interpolation fractions are fixed point with 8 bits, so the result is
// off by up to 6/256 of the largest coefficient (typically ~1e-3); it is
// reported beside the FP32 gather kernels, not used for them.
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "ls_internal.h"

namespace {

struct TexSpline {
    int nsite[3];                  // sites per axis (1..4)
    int s0[3];                     // first site offset per axis (sites are s0, s0+1, ...)
    float coef[3][4][4];           // coef[axis][site][power] of the 1D weight in u = y - center
    float center[3];
    int degree[3];
    int roe;                       // 0: k = floor(x) (region [0,1)^3), 1: k = rint(x) (Voronoi cube)
};

__global__ void linear_fetch_kernel(cudaTextureObject_t tex, const float *pts, long long n, float *out, TexSpline sp)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x[3] = {__ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2)};
        if (!(fabsf(x[0]) < 4194304.0f && fabsf(x[1]) < 4194304.0f && fabsf(x[2]) < 4194304.0f)) {
            const bool isn = (x[0] != x[0]) || (x[1] != x[1]) || (x[2] != x[2]);
            out[i] = isn ? __int_as_float(0x7fffffff) : 0.0f;
            continue;
        }
        float pos[3][2], gw[3][2];
        int nf[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float k = sp.roe ? rintf(x[a]) : floorf(x[a]);
            const float u = x[a] - k - sp.center[a];
            float w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float acc = 0.0f;
                for (int d = sp.degree[a]; d >= 0; --d) acc = fmaf(acc, u, sp.coef[a][j][d]);
                w[j] = j < sp.nsite[a] ? acc : 0.0f;
            }
            // pairs (0,1) and (2,3); a lone last site is fetched at its own position
            int f = 0;
            for (int j = 0; j < sp.nsite[a]; j += 2) {
                const float wa = w[j], wb = (j + 1 < sp.nsite[a]) ? w[j + 1] : 0.0f;
                const float g = wa + wb;
                const float t = g != 0.0f ? wb / g : 0.0f;
                gw[a][f] = g;
                pos[a][f] = k + (float)(sp.s0[a] + j) + t + 0.5f;   // texel centres sit at index + 1/2
                ++f;
            }
            nf[a] = f;
        }
        float acc = 0.0f;
        for (int f2 = 0; f2 < nf[2]; ++f2)
            for (int f1 = 0; f1 < nf[1]; ++f1)
                for (int f0 = 0; f0 < nf[0]; ++f0)
                    acc = fmaf(gw[0][f0] * gw[1][f1] * gw[2][f2], tex3D<float>(tex, pos[0][f0], pos[1][f1], pos[2][f2]),
                               acc);
        out[i] = acc;
    }
}

ls_status tex_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return ls_fail(LS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" ls_status ls_volume_texture_sync(ls_volume v, ls_stream stream)
{
    if (!v) return ls_fail(LS_ERR_INVALID_ARG, "volume is NULL");
    const ls::Table &t = v->spline->table;
    if (t.sep.empty() || t.dim != 3 || t.cosets.size() != 1 || v->spline->dtype != LS_F32 ||
        v->layout >= LS_LAYOUT_BRICKED)
        return ls_fail(LS_ERR_UNSUPPORTED,
                       "linear fetch needs a 3D tensor-product spline with FP32 coefficients in one array");
    for (const auto &ax : t.sep)
        if (ax.sites.size() > 4 || ax.degree > 3)
            return ls_fail(LS_ERR_UNSUPPORTED, "linear fetch needs at most 4 sites and degree 3 per axis");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (!v->tex_array) {
        cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
        e = cudaMalloc3DArray(&v->tex_array, &ch, make_cudaExtent(v->ext[0], v->ext[1], v->ext[2]));
        if (e != cudaSuccess) {
            v->tex_array = nullptr;
            cudaGetLastError();
            return ls_fail(LS_ERR_OOM, "cudaMalloc3DArray for the texture copy");
        }
        cudaResourceDesc rd;
        memset(&rd, 0, sizeof rd);
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = v->tex_array;
        cudaTextureDesc td;
        memset(&td, 0, sizeof td);
        for (int i = 0; i < 3; ++i) td.addressMode[i] = cudaAddressModeBorder;   // zero beyond the arrays
        td.filterMode = cudaFilterModeLinear;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&v->tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            cudaFreeArray(v->tex_array);
            v->tex_array = nullptr;
            v->tex = 0;
            return tex_fail(e, "cudaCreateTextureObject");
        }
    }
    cudaMemcpy3DParms p;
    memset(&p, 0, sizeof p);
    p.srcPtr = make_cudaPitchedPtr(v->coef, (size_t)v->ext[0] * sizeof(float), (size_t)v->ext[0], (size_t)v->ext[1]);
    p.dstArray = v->tex_array;
    p.extent = make_cudaExtent(v->ext[0], v->ext[1], v->ext[2]);
    p.kind = cudaMemcpyDeviceToDevice;
    e = cudaMemcpy3DAsync(&p, st);
    if (e != cudaSuccess) return tex_fail(e, "cudaMemcpy3DAsync into the texture array");
    v->tex_ready = true;
    return LS_OK;
}

extern "C" ls_status ls_eval_linear_fetch(ls_volume v, const float *pts, int64_t n, float *out, ls_stream stream)
{
    if (!v || (n > 0 && (!pts || !out))) return ls_fail(LS_ERR_INVALID_ARG, "volume, pts or out is NULL");
    if (n < 0) return ls_fail(LS_ERR_INVALID_ARG, "n < 0");
    if (!v->tex_ready) return ls_fail(LS_ERR_INVALID_ARG, "call ls_volume_texture_sync first");
    if (n == 0) return LS_OK;
    const ls::Table &t = v->spline->table;
    TexSpline sp;
    memset(&sp, 0, sizeof sp);
    sp.roe = t.roe == LS_ROE_VORONOI ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        const ls::Axis &ax = t.sep[a];
        sp.nsite[a] = (int)ax.sites.size();
        sp.s0[a] = ax.sites[0];
        for (size_t j = 1; j < ax.sites.size(); ++j)
            if (ax.sites[j] != ax.sites[0] + (int)j)
                return ls_fail(LS_ERR_UNSUPPORTED, "linear fetch needs consecutive sites per axis");
        sp.degree[a] = ax.degree;
        sp.center[a] = (float)ax.center;
        for (size_t j = 0; j < ax.sites.size(); ++j)
            for (int d = 0; d <= ax.degree; ++d) sp.coef[a][j][d] = (float)ax.coef[j * (ax.degree + 1) + d];
    }
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)v->spline->num_sms * 8;
    if (blocks > cap) blocks = cap;
    linear_fetch_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(v->tex, pts, n, out, sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tex_fail(e, "linear fetch kernel");
    return LS_OK;
}
