// Spline-independent device kernels (compiled ahead of time by nvcc for sm_103a).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lsk {

// dst[i] = (dst_dtype) src[i]; dtypes as ls_dtype (F32, BF16, F16, F64), round to nearest even.
cudaError_t convert(const void *src, int src_dt, void *dst, int dst_dt, long long n, cudaStream_t st);

// *result = sum a[i] b[i] in FP64 (fixed reduction order: bitwise reproducible).
// ws: >= dot_ws_bytes() bytes of device scratch.
size_t dot_ws_bytes();
cudaError_t dot_f64_ws(const float *a, const float *b, long long n, double *result, void *ws, cudaStream_t st);
// Same with a lazily allocated per-device scratch.
cudaError_t dot_f64(const float *a, const float *b, long long n, double *result, cudaStream_t st);

}  // namespace lsk
