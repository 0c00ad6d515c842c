// Spline-independent device kernels (compiled ahead of time by nvcc for sm_103a).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lsk {

// dst[i] = (dst_dtype) src[i]; dtypes as ls_dtype (F32, BF16, F16, F64), round to nearest even.
cudaError_t convert(const void *src, int src_dt, void *dst, int dst_dt, long long n, cudaStream_t st);
// Geometry of a coefficient layout: ls_layout, cosets, elements per coset, extents.
struct LayoutGeom {
    int layout;
    int ncos;
    long long per;
    int e0, e1, e2;
};
// Elements a layout holds (ncos * per; the shifted bricked copies of layout 3
// hold 4 ncos (e0 + 2)(e1 + 2) e2, those of layout 4 8 ncos (e0 + 2)(e1 + 2)
// (e2 + 2), their padding zero).
long long layout_elems(const LayoutGeom &g);
// Conversion of all layout_elems(dg) elements from layout sg to layout dg (same
// cosets and extents), dtypes as in convert.
cudaError_t convert_relayout(const void *src, int src_dt, const LayoutGeom &sg, void *dst, int dst_dt,
                             const LayoutGeom &dg, cudaStream_t st);
// Layout change only, elements of elem_bytes (2, 4 or 8).
cudaError_t relayout(const void *src, const LayoutGeom &sg, void *dst, const LayoutGeom &dg, int elem_bytes,
                     cudaStream_t st);

// *result = sum a[i] b[i] in FP64 (fixed reduction order: bitwise reproducible).
// ws: >= dot_ws_bytes() bytes of device scratch.
size_t dot_ws_bytes();
cudaError_t dot_f64_ws(const float *a, const float *b, long long n, double *result, void *ws, cudaStream_t st);
// Fixed-point adjoint helpers.  fixed_prepare: sum |g| in FP64 (fixed order) and
// the power-of-two scale 2^s (*scale, FP32) and 2^-s (*inv, FP64) with
// sum|g| * wmax * 2^s < 2^61; both pointers point into ws (fixed_ws_bytes()).
// fixed_finish: dcoef[i] += (double)(int64)acc[i] * 2^-s.
size_t fixed_ws_bytes();
cudaError_t fixed_prepare(const float *g, long long n, double wmax, void *ws, float **scale, double **inv,
                          cudaStream_t st);
cudaError_t fixed_finish(const unsigned long long *acc, const double *inv, float *dcoef, long long n, cudaStream_t st);
// Same with a lazily allocated per-device scratch.
cudaError_t dot_f64(const float *a, const float *b, long long n, double *result, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on the low nbits of the keys,
// in place (keys/vals hold the result).  scratch: sort_scratch_bytes(n).
size_t sort_scratch_bytes(long long n);
cudaError_t radix_sort_pairs(uint32_t *keys, int32_t *vals, long long n, int nbits, void *scratch, cudaStream_t st);
// keys[i] = 30-bit Morton code of floor((pts[i] - origin) * (1 / cell)) (clamped to 0..1023), vals[i] = i.
cudaError_t morton_keys(const float *pts, long long n, const float *origin, float cell, uint32_t *keys,
                        int32_t *vals, cudaStream_t st);
cudaError_t iota(int32_t *v, long long n, cudaStream_t st);
cudaError_t permute_rows(const float *src, const int32_t *perm, long long n, int width, int inverse, float *dst,
                         cudaStream_t st);
// start[b] = first index with sorted key >= b, for b in [0, nbins + 1] (keys <= nbins).
cudaError_t bin_starts(const uint32_t *key, long long n, uint32_t nbins, uint32_t *start, cudaStream_t st);
cudaError_t gather_probe(const float *table, long long table_elems, int loads, float *out, long long nthreads,
                         int blocks, cudaStream_t st);

// CGLS vector steps (FP32 vectors, FP64 scalars resident on the device).
//   sc[0] = gamma = ||s||^2, sc[1] = ||q||^2, sc[2] = ||p||^2, sc[3] = gamma_new
// cg_step_cr:  alpha = gamma / (||q||^2 + lambda ||p||^2); c += alpha p; r -= alpha q
cudaError_t cg_step_cr(float *c, const float *p, long long nc, float *r, const float *q, long long nr,
                       const double *sc, double lambda, cudaStream_t st);
// cg_step_p: p = s + (gamma_new / gamma) p, then gamma = gamma_new
cudaError_t cg_step_p(float *p, const float *s, long long nc, double *sc, cudaStream_t st);
// y = a*x + b*y (host scalars)
cudaError_t axpby(float a, const float *x, float b, float *y, long long n, cudaStream_t st);
// r = y - r (in place on r)
cudaError_t sub_from(const float *y, float *r, long long n, cudaStream_t st);

}  // namespace lsk
