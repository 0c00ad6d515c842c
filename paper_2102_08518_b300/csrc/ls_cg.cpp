// Least-squares fit of spline coefficients to scattered samples by CGLS:
//     min_c ||A c - y||^2 + lambda ||c||^2,   A[i, n] = phi(x_i - n)
// A v is ls_eval with coefficients v, A^T w is ls_adjoint_coef; the inner
// products are FP64 reductions on the device and every CG scalar stays in
// device memory (the host reads ||s|| once per iteration for the stopping rule).
#include <cmath>
#include <string>
#include <vector>

#include "ls_internal.h"
#include "ls_kernels.h"

namespace {

struct Ws {
    void *base = nullptr;
    ~Ws()
    {
        if (base) ls::dev_free(base);
    }
};

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" ls_status ls_cg_fit(ls_volume v, const float *pts, const float *y, int64_t n, double lambda,
                               int32_t max_iter, double rel_tol, int32_t adjoint_mode, double *resid_hist,
                               int32_t *iters, ls_stream stream)
{
    if (!v || (n > 0 && (!pts || !y))) return ls_fail(LS_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0 || max_iter < 0 || !(lambda >= 0.0) || !(rel_tol >= 0.0))
        return ls_fail(LS_ERR_INVALID_ARG, "n > 0, max_iter >= 0, lambda >= 0 and rel_tol >= 0 required");
    if (v->spline->dtype != LS_F32) return ls_fail(LS_ERR_UNSUPPORTED, "the fit needs FP32 coefficient storage");
    if (adjoint_mode != LS_ADJ_ATOMIC && adjoint_mode != LS_ADJ_DETERMINISTIC && adjoint_mode != LS_ADJ_ATOMIC_WARP &&
        adjoint_mode != LS_ADJ_DETERMINISTIC_FIXED && adjoint_mode != LS_ADJ_ATOMIC_TILED &&
        adjoint_mode != LS_ADJ_DETERMINISTIC_FIXED_TILED)
        return ls_fail(LS_ERR_INVALID_ARG, "unknown adjoint mode");
    const bool deterministic = adjoint_mode == LS_ADJ_DETERMINISTIC || adjoint_mode == LS_ADJ_DETERMINISTIC_FIXED ||
                               adjoint_mode == LS_ADJ_DETERMINISTIC_FIXED_TILED;
    cudaStream_t st = (cudaStream_t)stream;
    const long long nc = v->total_elems, nr = n;
    const size_t adj_bytes = deterministic ? ls_adjoint_scratch_bytes(v, n) : 0;
    const size_t bytes = al(nc * 4) * 2 + al(nr * 4) * 2 + al(8 * sizeof(double)) + al(lsk::dot_ws_bytes()) + adj_bytes;
    Ws ws;
    if (ls::dev_malloc(&ws.base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return ls_fail(LS_ERR_OOM, "workspace of the CG fit");
    }
    char *q0 = (char *)ws.base;
    float *p = (float *)q0;
    q0 += al(nc * 4);
    float *s = (float *)q0;
    q0 += al(nc * 4);
    float *r = (float *)q0;
    q0 += al(nr * 4);
    float *q = (float *)q0;
    q0 += al(nr * 4);
    double *sc = (double *)q0;          // [gamma, qq, pp, gamma_new, aty2]
    q0 += al(8 * sizeof(double));
    void *dws = q0;
    q0 += al(lsk::dot_ws_bytes());
    void *adj_ws = deterministic ? (void *)q0 : nullptr;
    float *c = (float *)v->coef;
    // the CG scalars and the dot kernel's completion ticket must start at zero
    {
        cudaError_t z = cudaMemsetAsync(sc, 0, al(8 * sizeof(double)) + al(lsk::dot_ws_bytes()), st);
        if (z != cudaSuccess) return ls_fail(LS_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(z));
    }

    ls_volume_s pv = *v;                // same grid, coefficients = p
    pv.coef = p;
    pv.stage = nullptr;
    pv.stage_bytes = 0;
    pv.hs[0] = pv.hs[1] = nullptr;
    pv.hev[0] = pv.hev[1] = pv.hev[2] = nullptr;
    pv.owned = false;

    auto cuda_err = [&](cudaError_t e, const char *what) {
        return ls_fail(LS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    auto adjoint_into = [&](const float *w, float *dst) -> ls_status {
        cudaError_t e = cudaMemsetAsync(dst, 0, nc * 4, st);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemsetAsync");
        return ls_adjoint_coef(v, pts, w, n, dst, adjoint_mode, adj_ws, stream);
    };
    ls_status res;
    cudaError_t e;
    // r = y - A c ; s = A^T r - lambda c ; ||A^T y||^2 for the stopping rule
    if ((res = ls_eval(v, pts, n, r, stream)) != LS_OK) return res;
    if ((e = lsk::sub_from(y, r, nr, st)) != cudaSuccess) return cuda_err(e, "sub_from");
    if ((res = adjoint_into(y, p)) != LS_OK) return res;
    if ((e = lsk::dot_f64_ws(p, p, nc, sc + 4, dws, st)) != cudaSuccess) return cuda_err(e, "dot");
    if ((res = adjoint_into(r, s)) != LS_OK) return res;
    if (lambda > 0.0 && (e = lsk::axpby((float)-lambda, c, 1.0f, s, nc, st)) != cudaSuccess) return cuda_err(e, "axpby");
    if ((e = cudaMemcpyAsync(p, s, nc * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return cuda_err(e, "copy");
    if ((e = lsk::dot_f64_ws(s, s, nc, sc + 0, dws, st)) != cudaSuccess) return cuda_err(e, "dot");
    double host[5];
    if ((e = cudaMemcpyAsync(host, sc, 5 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_err(e, "read CG scalars");
    const double target = rel_tol * std::sqrt(host[4]);
    double gamma = host[0];
    if (resid_hist) resid_hist[0] = std::sqrt(gamma);
    int it = 0;
    while (it < max_iter && std::sqrt(gamma) > target && gamma > 0.0) {
        // q = A p ; alpha = gamma / (||q||^2 + lambda ||p||^2) ; c += alpha p ; r -= alpha q
        if ((res = ls_eval(&pv, pts, n, q, stream)) != LS_OK) return res;
        if ((e = lsk::dot_f64_ws(q, q, nr, sc + 1, dws, st)) != cudaSuccess) return cuda_err(e, "dot");
        if ((e = lsk::dot_f64_ws(p, p, nc, sc + 2, dws, st)) != cudaSuccess) return cuda_err(e, "dot");
        if ((e = lsk::cg_step_cr(c, p, nc, r, q, nr, sc, lambda, st)) != cudaSuccess) return cuda_err(e, "cg step");
        // s = A^T r - lambda c ; gamma_new = ||s||^2 ; p = s + (gamma_new / gamma) p
        if ((res = adjoint_into(r, s)) != LS_OK) return res;
        if (lambda > 0.0 && (e = lsk::axpby((float)-lambda, c, 1.0f, s, nc, st)) != cudaSuccess)
            return cuda_err(e, "axpby");
        if ((e = lsk::dot_f64_ws(s, s, nc, sc + 3, dws, st)) != cudaSuccess) return cuda_err(e, "dot");
        if ((e = lsk::cg_step_p(p, s, nc, sc, st)) != cudaSuccess) return cuda_err(e, "cg step");
        if ((e = cudaMemcpyAsync(host, sc, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_err(e, "read CG scalars");
        gamma = host[0];
        ++it;
        if (resid_hist) resid_hist[it] = std::sqrt(gamma);
    }
    if (iters) *iters = it;
    return LS_OK;
}
