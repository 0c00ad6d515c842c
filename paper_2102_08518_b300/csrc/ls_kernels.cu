// Spline-independent kernels: storage conversion and FP64 reductions.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <map>
#include <mutex>

#include "ls_kernels.h"

namespace lsk {
namespace {

enum { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2, DT_F64 = 3 };

__device__ __forceinline__ double load_any(const void *p, int dt, long long i)
{
    switch (dt) {
    case DT_F32: return (double)((const float *)p)[i];
    case DT_BF16: return (double)__bfloat162float(((const __nv_bfloat16 *)p)[i]);
    case DT_F16: return (double)__half2float(((const __half *)p)[i]);
    default: return ((const double *)p)[i];
    }
}

// Element index of (coset j, grid index q) in a coefficient layout (ls_layout):
// 0 coset-major, 1 interleaved, 2 bricked (2 x 2 x 2 grid indices per brick,
// 2 x 2 in 2D (e2 == 1), cosets interleaved inside, x fastest), 3 four bricked
// copies whose brick grids are shifted by (sx, sy) in {0,1}^2 grid indices
// (copy sx + 2 sy over extents e0 + 2, e1 + 2, e2; copy 0 is read here), 4 the
// same with eight copies shifted on all three axes (copy sx + 2 sy + 4 sz over
// extents e0 + 2, e1 + 2, e2 + 2).
__device__ __forceinline__ long long brick_index(int ncos, int e0, int e1, int e2, int j, int q0, int q1, int q2)
{
    const int bv = e2 == 1 ? 4 : 8;
    const long long bk = (q0 >> 1) + (long long)(e0 >> 1) * ((q1 >> 1) + (long long)(e1 >> 1) * (q2 >> 1));
    const int wi = (q0 & 1) + 2 * (q1 & 1) + 4 * (q2 & 1);
    return (bk * bv + wi) * ncos + j;
}

__device__ __forceinline__ long long lay_index(const LayoutGeom &g, int j, int q0, int q1, int q2)
{
    const long long lin = q0 + (long long)g.e0 * (q1 + (long long)g.e1 * q2);
    if (g.layout == 0) return (long long)j * g.per + lin;
    if (g.layout == 1) return lin * g.ncos + j;
    if (g.layout == 3) return brick_index(g.ncos, g.e0 + 2, g.e1 + 2, g.e2, j, q0, q1, q2);
    if (g.layout == 4) return brick_index(g.ncos, g.e0 + 2, g.e1 + 2, g.e2 + 2, j, q0, q1, q2);
    return brick_index(g.ncos, g.e0, g.e1, g.e2, j, q0, q1, q2);
}

__device__ __forceinline__ void brick_decode(long long i, int ncos, int e0, int e1, int e2, int &j, int &q0, int &q1,
                                             int &q2)
{
    const int bv = e2 == 1 ? 4 : 8;
    j = (int)(i % ncos);
    const long long w = i / ncos;
    const int wi = (int)(w % bv);
    long long bk = w / bv;
    q0 = (int)(bk % (e0 >> 1)) * 2 + (wi & 1);
    bk /= (e0 >> 1);
    q1 = (int)(bk % (e1 >> 1)) * 2 + ((wi >> 1) & 1);
    bk /= (e1 >> 1);
    q2 = (int)bk * 2 + (wi >> 2);
}

// (coset, grid index) of element i; false for the padding of layout 3
__device__ __forceinline__ bool lay_decode(const LayoutGeom &g, long long i, int &j, int &q0, int &q1, int &q2)
{
    if (g.layout == 3 || g.layout == 4) {
        const int pz = g.layout == 4 ? 2 : 0;
        const long long copy_elems = (long long)g.ncos * (g.e0 + 2) * (g.e1 + 2) * (g.e2 + pz);
        const int c = (int)(i / copy_elems);
        brick_decode(i % copy_elems, g.ncos, g.e0 + 2, g.e1 + 2, g.e2 + pz, j, q0, q1, q2);
        q0 -= c & 1;
        q1 -= (c >> 1) & 1;
        q2 -= c >> 2;
        return q0 >= 0 && q0 < g.e0 && q1 >= 0 && q1 < g.e1 && q2 >= 0 && q2 < g.e2;
    }
    if (g.layout == 2) {
        brick_decode(i, g.ncos, g.e0, g.e1, g.e2, j, q0, q1, q2);
        return true;
    }
    long long r;
    if (g.layout == 0) {
        j = (int)(i / g.per);
        r = i % g.per;
    } else {
        j = (int)(i % g.ncos);
        r = i / g.ncos;
    }
    q0 = (int)(r % g.e0);
    r /= g.e0;
    q1 = (int)(r % g.e1);
    q2 = (int)(r / g.e1);
    return true;
}

// Source index of destination element i when the layout changes from s to d
// (-1: padding of the destination, which gets 0).
__device__ __forceinline__ long long relayout_src(long long i, const LayoutGeom &s, const LayoutGeom &d)
{
    if (s.layout == d.layout) return i;
    int j, q0, q1, q2;
    if (!lay_decode(d, i, j, q0, q1, q2)) return -1;
    return lay_index(s, j, q0, q1, q2);
}

__global__ void convert_kernel(const void *src, int sdt, void *dst, int ddt, long long n, LayoutGeom sg,
                               LayoutGeom dg)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long si = relayout_src(i, sg, dg);
        const double v = si < 0 ? 0.0 : load_any(src, sdt, si);
        switch (ddt) {
        case DT_F32: ((float *)dst)[i] = (float)v; break;
        case DT_BF16: ((__nv_bfloat16 *)dst)[i] = __float2bfloat16_rn((float)v); break;
        case DT_F16: ((__half *)dst)[i] = __float2half_rn((float)v); break;
        default: ((double *)dst)[i] = v; break;
        }
    }
}

template <typename T>
__global__ void relayout_kernel(const T *src, T *dst, long long n, LayoutGeom sg, LayoutGeom dg)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    {
        const long long si = relayout_src(i, sg, dg);
        dst[i] = si < 0 ? (T)0 : src[si];
    }
}

constexpr int kDotBlocks = 296;   // 2 per SM on 148 SMs
constexpr int kDotThreads = 512;

// Per-block FP64 partial sums in a fixed order; the last block to finish (ticket
// counter, no waiting) adds the partials in block order and resets the counter.
// ABS = 1 sums |a[i]| (b unused).
template <int ABS>
__global__ void __launch_bounds__(kDotThreads) dot_kernel(const float *a, const float *b, long long n,
                                                           double *partials, unsigned *ticket, double *result)
{
    __shared__ double red[kDotThreads];
    __shared__ bool last;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s = ABS ? s + fabs((double)a[i]) : fma((double)a[i], (double)b[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = red[0];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) tot += ((volatile double *)partials)[k];
        *result = tot;
        *ticket = 0u;
    }
}

std::mutex g_mu;
std::map<int, void *> g_ws;

__global__ void cg_cr_kernel(float *c, const float *p, long long nc, float *r, const float *q, long long nr,
                             const double *sc, double lambda)
{
    const double den = sc[1] + lambda * sc[2];
    const double alpha = den > 0.0 ? sc[0] / den : 0.0;
    const float af = (float)alpha;
    const long long n = nc > nr ? nc : nr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (i < nc) c[i] = fmaf(af, p[i], c[i]);
        if (i < nr) r[i] = fmaf(-af, q[i], r[i]);
    }
}

__global__ void cg_p_kernel(float *p, const float *s, long long nc, double *sc)
{
    const double beta = sc[0] > 0.0 ? sc[3] / sc[0] : 0.0;
    const float bf = (float)beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x)
        p[i] = fmaf(bf, p[i], s[i]);
}

__global__ void cg_shift_gamma(double *sc) { sc[0] = sc[3]; }

// Scale of the fixed-point adjoint: 2^s with s = 61 - ceil(log2(bound)), bound =
// sum|g| * wmax >= any accumulated |value|, so every int64 sum stays below 2^62.
__global__ void fixed_scale_kernel(const double *gsum, double wmax, float *scale, double *inv)
{
    const double b = *gsum * wmax;
    int s = 0;
    if (b > 0.0 && b < 1e300) {
        int e = 0;
        frexp(b, &e);                  // b < 2^e
        s = 61 - e;
        s = s < -126 ? -126 : (s > 126 ? 126 : s);
    }
    *scale = ldexpf(1.0f, s);
    *inv = ldexp(1.0, -s);
}

__global__ void fixed_finish_kernel(const unsigned long long *acc, const double *inv, float *dcoef, long long n)
{
    const double iv = *inv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dcoef[i] += (float)((double)(long long)acc[i] * iv);
}

__global__ void axpby_kernel(float a, const float *x, float b, float *y, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], b * y[i]);
}

__global__ void sub_from_kernel(const float *y, float *r, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = y[i] - r[i];
}

unsigned grid_of(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 148 * 16) b = 148 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t cg_step_cr(float *c, const float *p, long long nc, float *r, const float *q, long long nr,
                       const double *sc, double lambda, cudaStream_t st)
{
    cg_cr_kernel<<<grid_of(nc > nr ? nc : nr), 256, 0, st>>>(c, p, nc, r, q, nr, sc, lambda);
    return cudaGetLastError();
}

cudaError_t cg_step_p(float *p, const float *s, long long nc, double *sc, cudaStream_t st)
{
    cg_p_kernel<<<grid_of(nc), 256, 0, st>>>(p, s, nc, sc);
    cg_shift_gamma<<<1, 1, 0, st>>>(sc);
    return cudaGetLastError();
}

cudaError_t axpby(float a, const float *x, float b, float *y, long long n, cudaStream_t st)
{
    axpby_kernel<<<grid_of(n), 256, 0, st>>>(a, x, b, y, n);
    return cudaGetLastError();
}

cudaError_t sub_from(const float *y, float *r, long long n, cudaStream_t st)
{
    sub_from_kernel<<<grid_of(n), 256, 0, st>>>(y, r, n);
    return cudaGetLastError();
}

namespace {
}  // namespace

cudaError_t convert(const void *src, int sdt, void *dst, int ddt, long long n, cudaStream_t st)
{
    LayoutGeom g{0, 1, n, (int)n, 1, 1};
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    convert_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, sdt, dst, ddt, n, g, g);
    return cudaGetLastError();
}

cudaError_t convert_relayout(const void *src, int sdt, const LayoutGeom &sg, void *dst, int ddt, const LayoutGeom &dg,
                             cudaStream_t st)
{
    const long long n = layout_elems(dg);
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    convert_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, sdt, dst, ddt, n, sg, dg);
    return cudaGetLastError();
}

cudaError_t relayout(const void *src, const LayoutGeom &sg, void *dst, const LayoutGeom &dg, int elem_bytes,
                     cudaStream_t st)
{
    const long long n = layout_elems(dg);
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (elem_bytes == 2)
        relayout_kernel<<<(unsigned)blocks, 256, 0, st>>>((const uint16_t *)src, (uint16_t *)dst, n, sg, dg);
    else if (elem_bytes == 4)
        relayout_kernel<<<(unsigned)blocks, 256, 0, st>>>((const uint32_t *)src, (uint32_t *)dst, n, sg, dg);
    else
        relayout_kernel<<<(unsigned)blocks, 256, 0, st>>>((const uint64_t *)src, (uint64_t *)dst, n, sg, dg);
    return cudaGetLastError();
}

long long layout_elems(const LayoutGeom &g)
{
    if (g.layout == 3) return 4LL * g.ncos * (g.e0 + 2) * (g.e1 + 2) * g.e2;
    if (g.layout == 4) return 8LL * g.ncos * (g.e0 + 2) * (g.e1 + 2) * (g.e2 + 2);
    return (long long)g.ncos * g.per;
}

size_t dot_ws_bytes() { return kDotBlocks * sizeof(double) + 256; }

size_t fixed_ws_bytes() { return dot_ws_bytes() + 256; }

cudaError_t fixed_prepare(const float *g, long long n, double wmax, void *ws, float **scale, double **inv,
                          cudaStream_t st)
{
    double *partials = (double *)ws;
    unsigned *ticket = (unsigned *)((char *)ws + kDotBlocks * sizeof(double));
    double *gsum = (double *)((char *)ws + dot_ws_bytes());
    *scale = (float *)(gsum + 1);
    *inv = gsum + 2;
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    dot_kernel<1><<<kDotBlocks, kDotThreads, 0, st>>>(g, g, n, partials, ticket, gsum);
    fixed_scale_kernel<<<1, 1, 0, st>>>(gsum, wmax, *scale, *inv);
    return cudaGetLastError();
}

cudaError_t fixed_finish(const unsigned long long *acc, const double *inv, float *dcoef, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    fixed_finish_kernel<<<grid_of(n), 256, 0, st>>>(acc, inv, dcoef, n);
    return cudaGetLastError();
}

cudaError_t dot_f64_ws(const float *a, const float *b, long long n, double *result, void *ws, cudaStream_t st)
{
    double *partials = (double *)ws;
    unsigned *ticket = (unsigned *)((char *)ws + kDotBlocks * sizeof(double));
    dot_kernel<0><<<kDotBlocks, kDotThreads, 0, st>>>(a, b, n, partials, ticket, result);
    return cudaGetLastError();
}

cudaError_t dot_f64(const float *a, const float *b, long long n, double *result, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find(dev);
        if (it == g_ws.end()) {
            e = cudaMalloc(&ws, dot_ws_bytes());
            if (e != cudaSuccess) return e;
            e = cudaMemset(ws, 0, dot_ws_bytes());
            if (e != cudaSuccess) return e;
            g_ws[dev] = ws;
        } else {
            ws = it->second;
        }
    }
    return dot_f64_ws(a, b, n, result, ws, st);
}

}  // namespace lsk
