// C ABI of the lattice spline library: descriptor validation, kernel
// generation/loading, coefficient volumes and launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>  // CUtensorMap and its enums; the encoder is fetched from the driver at run time

#include "ls_internal.h"
#include "ls_kernels.h"

namespace {
thread_local std::string g_err;

struct EvalArgsH {
    const float *pts;
    float *out;
    float *grad;
    const void *coef;
    long long n;
    int e0, e1, e2, cstride, cunit;
    unsigned *status;
    float *hess;
    const void *tmap;
};
struct AdjArgsH {
    const float *pts;
    const float *gout;
    float *dcoef;
    long long n;
    int e0, e1, e2, cstride, cunit;
    unsigned long long *iacc;
    const float *iscale;
};
struct BinArgsH {
    const float *pts;
    const float *gout;
    uint32_t *key;
    int32_t *idx;
    void *rec;
    long long n;
    int e0, e1, e2, halo;
    uint32_t nbins;
};
struct GatherArgsH {
    const void *srec;
    const uint32_t *start;
    float *dcoef;
    int e0, e1, e2, cstride, cunit, halo;
};

const char *dtype_tag(ls_dtype d)
{
    switch (d) {
    case LS_F32: return "f32";
    case LS_BF16: return "bf16";
    case LS_F16: return "f16";
    default: return "x";
    }
}

size_t dtype_size(ls_dtype d)
{
    switch (d) {
    case LS_F32: return 4;
    case LS_BF16: return 2;
    case LS_F16: return 2;
    case LS_F64: return 8;
    }
    return 0;
}

ls_status cuda_fail(cudaError_t e, const char *what)
{
    return ls_fail(LS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool valid_name(const char *n)
{
    if (!n) return true;
    size_t len = std::strlen(n);
    if (len == 0 || len > 40) return false;
    for (size_t i = 0; i < len; ++i) {
        char c = n[i];
        if (!((c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_'))
            return false;
    }
    return true;
}

// Copy and validate a descriptor.
ls_status copy_desc(const ls_spline_desc *d, ls::Table &t)
{
    if (!d) return ls_fail(LS_ERR_INVALID_ARG, "descriptor is NULL");
    if (!valid_name(d->name)) return ls_fail(LS_ERR_INVALID_ARG, "name must match [A-Za-z0-9_]{1,40}");
    t.name = d->name ? d->name : "";
    if (d->dim != 2 && d->dim != 3) return ls_fail(LS_ERR_UNSUPPORTED, "dim must be 2 or 3");
    t.dim = d->dim;
    if (d->roe != LS_ROE_PARALLELEPIPED && d->roe != LS_ROE_VORONOI)
        return ls_fail(LS_ERR_INVALID_ARG, "roe must be LS_ROE_PARALLELEPIPED or LS_ROE_VORONOI");
    if (d->fold != LS_FOLD_NONE && d->fold != LS_FOLD_SIGNED_PERM)
        return ls_fail(LS_ERR_INVALID_ARG, "fold must be LS_FOLD_NONE or LS_FOLD_SIGNED_PERM");
    t.roe = d->roe;
    t.fold = d->fold;
    if (d->scale != 1 && d->scale != 2) return ls_fail(LS_ERR_UNSUPPORTED, "scale must be 1 or 2");
    t.scale = d->scale;
    std::memcpy(t.L, d->generator, sizeof t.L);
    if (d->n_cosets < 1 || d->n_cosets > 8 || !d->coset_offsets)
        return ls_fail(LS_ERR_INVALID_ARG, "n_cosets must be 1..8 with coset_offsets");
    if (d->scale == 1 && d->n_cosets != 1) return ls_fail(LS_ERR_BAD_TABLE, "scale 1 has exactly one coset");
    for (int j = 0; j < d->n_cosets; ++j) {
        ls::I3 l{0, 0, 0};
        for (int i = 0; i < d->dim; ++i) {
            int v = d->coset_offsets[j * d->dim + i];
            if (v < 0 || v >= d->scale) return ls_fail(LS_ERR_BAD_TABLE, "coset offset outside [0, scale)");
            l[i] = v;
        }
        for (auto &o : t.cosets)
            if (o == l) return ls_fail(LS_ERR_BAD_TABLE, "duplicate coset offset");
        t.cosets.push_back(l);
    }
    if (d->roe == LS_ROE_PARALLELEPIPED) {
        if (d->scale != 1) return ls_fail(LS_ERR_UNSUPPORTED, "parallelepiped ROE needs the Cartesian grid (scale 1)");
        for (int c = 0; c < d->dim; ++c)
            for (int r = 0; r < d->dim; ++r)
                if (d->generator[3 * c + r] != (r == c ? 1.0 : 0.0))
                    return ls_fail(LS_ERR_UNSUPPORTED, "parallelepiped ROE needs L = I");
    }
    if (d->n_ref < 1 || d->n_ref > 15) return ls_fail(LS_ERR_UNSUPPORTED, "n_ref must be 1..15");
    if (d->n_planes < 0 || d->n_planes > 4) return ls_fail(LS_ERR_UNSUPPORTED, "n_planes must be 0..4");
    if (d->bsp_mod < 1 || d->bsp_mod > 16) return ls_fail(LS_ERR_UNSUPPORTED, "bsp_mod must be 1..16");
    if (d->n_planes > 0 && !d->planes) return ls_fail(LS_ERR_INVALID_ARG, "planes is NULL");
    if (!d->sigma) return ls_fail(LS_ERR_INVALID_ARG, "sigma is NULL");
    for (int p = 0; p < d->n_planes; ++p) {
        std::array<double, 4> pl{0, 0, 0, 0};
        for (int i = 0; i < d->dim; ++i) pl[i] = d->planes[p * (d->dim + 1) + i];
        pl[3] = d->planes[p * (d->dim + 1) + d->dim];
        t.planes.push_back(pl);
    }
    t.bsp_mod = d->bsp_mod;
    bool any_used = false;
    for (int q = 0; q < d->bsp_mod; ++q) {
        int v = d->sigma[q];
        if (v < -1 || v >= d->n_ref) return ls_fail(LS_ERR_BAD_TABLE, "sigma entry outside [-1, n_ref)");
        any_used = any_used || v >= 0;
        t.sigma.push_back(v);
    }
    if (!any_used) return ls_fail(LS_ERR_BAD_TABLE, "sigma maps nothing to a reference sub-region");
    if (d->n_ref > 1 && d->n_planes == 0) return ls_fail(LS_ERR_BAD_TABLE, "several reference sub-regions need BSP planes");
    if (!d->ref) return ls_fail(LS_ERR_INVALID_ARG, "ref is NULL");
    for (int k = 0; k < d->n_ref; ++k) {
        const ls_ref_region &r = d->ref[k];
        if (r.n_sites < 1 || r.n_sites > 128 || !r.sites)
            return ls_fail(LS_ERR_UNSUPPORTED, "a reference sub-region needs 1..128 sites");
        if (r.n_monos < 1 || r.n_monos > 256 || !r.mono_exp || !r.coef)
            return ls_fail(LS_ERR_UNSUPPORTED, "a reference sub-region needs 1..256 monomials");
        ls::RefRegion rr;
        for (int j = 0; j < r.n_sites; ++j) {
            ls::I3 s{0, 0, 0};
            for (int i = 0; i < d->dim; ++i) {
                s[i] = r.sites[j * d->dim + i];
                if (std::abs(s[i]) > 16) return ls_fail(LS_ERR_UNSUPPORTED, "site offset beyond 16");
            }
            for (auto &o : rr.sites)
                if (o == s) return ls_fail(LS_ERR_BAD_TABLE, "duplicate site in a reference sub-region");
            rr.sites.push_back(s);
        }
        for (int a = 0; a < r.n_monos; ++a) {
            ls::I3 m{0, 0, 0};
            int deg = 0;
            for (int i = 0; i < d->dim; ++i) {
                m[i] = r.mono_exp[a * d->dim + i];
                if (m[i] < 0 || m[i] > 12) return ls_fail(LS_ERR_BAD_TABLE, "monomial exponent outside 0..12");
                deg += m[i];
            }
            for (auto &o : rr.mono)
                if (o == m) return ls_fail(LS_ERR_BAD_TABLE, "duplicate monomial");
            rr.mono.push_back(m);
            rr.degree = std::max(rr.degree, deg);
        }
        rr.coef.assign(r.coef, r.coef + (size_t)r.n_sites * r.n_monos);
        for (double v : rr.coef)
            if (!std::isfinite(v)) return ls_fail(LS_ERR_BAD_TABLE, "non-finite polynomial coefficient");
        for (int i = 0; i < 3; ++i) rr.center[i] = i < d->dim ? r.center[i] : 0.0;
        t.ref.push_back(rr);
    }
    if (d->separable) {
        if (d->fold != LS_FOLD_NONE || d->n_ref != 1 || d->scale != 1)
            return ls_fail(LS_ERR_UNSUPPORTED, "separable form needs fold none, one region, the Cartesian grid");
        for (int c = 0; c < d->dim; ++c)
            for (int r = 0; r < d->dim; ++r)
                if (d->generator[3 * c + r] != (c == r ? 1.0 : 0.0))
                    return ls_fail(LS_ERR_UNSUPPORTED, "separable form needs L = I");
        for (int i = 0; i < d->dim; ++i) {
            const ls_axis_factor &a = d->separable[i];
            if (a.n_sites < 1 || a.n_sites > 8 || !a.sites || !a.coef || a.degree < 0 || a.degree > 8)
                return ls_fail(LS_ERR_UNSUPPORTED, "axis factor needs 1..8 sites, degree 0..8");
            ls::Axis ax;
            ax.sites.assign(a.sites, a.sites + a.n_sites);
            ax.degree = a.degree;
            ax.coef.assign(a.coef, a.coef + (size_t)a.n_sites * (a.degree + 1));
            ax.center = a.center;
            t.sep.push_back(ax);
        }
    }
    return LS_OK;
}

int grid_for(long long n, int block, int sms, int per_sm)
{
    long long need = (n + block - 1) / block;
    long long cap = (long long)sms * std::max(per_sm, 1);
    if (need < 1) need = 1;
    return (int)std::min(need, cap);
}

ls_status launch(cudaKernel_t k, int grid, int block, void *args, cudaStream_t stream, size_t smem = 0)
{
    void *argv[] = {args};
    cudaError_t e = cudaLaunchKernel((const void *)k, dim3(grid), dim3(block), argv, smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernel");
    return LS_OK;
}

ls_status get_kernel(ls_spline_s *s, const char *what, cudaKernel_t &k, int &per_sm)
{
    std::string nm = std::string("ls_") + what;
    if (!s->table.name.empty()) nm += "__" + s->table.name;
    cudaError_t e = cudaLibraryGetKernel(&k, s->mod.lib, nm.c_str());
    if (e != cudaSuccess) return cuda_fail(e, ("cudaLibraryGetKernel " + nm).c_str());
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)k, s->var.block, 0);
    if (e != cudaSuccess || nb <= 0) {
        cudaGetLastError();
        nb = 4;
    }
    per_sm = nb;
    return LS_OK;
}

ls_variant default_variant(const ls_variant *v)
{
    ls_variant r{256, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (v) {
        if (v->block > 0) r.block = v->block;
        if (v->pts_per_thread > 0) r.pts_per_thread = v->pts_per_thread > 64 ? 64 : v->pts_per_thread;
        r.branchy = v->branchy;
        r.min_blocks = v->min_blocks > 0 ? v->min_blocks : 0;
        r.group = v->group > 0 ? v->group : 0;
        r.depth = v->depth > 0 ? v->depth : 0;
        r.blocks_per_sm = v->blocks_per_sm > 0 ? v->blocks_per_sm : 0;
        r.brick = v->brick >= 2 && v->brick <= 3 ? v->brick : v->brick ? 1 : 0;
        r.pipeline = v->pipeline ? 1 : 0;
        r.producers = v->producers > 0 ? v->producers : 0;
        r.stage = v->stage > 0 ? v->stage : 0;
        r.tensor = v->tensor > 0 ? v->tensor : 0;
        r.tensor_kind = v->tensor_kind == 1 ? 1 : 0;
        r.plain_transform = v->plain_transform ? 1 : 0;
        r.wait_limit = v->wait_limit > 0 ? v->wait_limit : 0;
        r.wait_probe = v->wait_probe;
        r.prefetch = v->prefetch ? 1 : 0;
        r.l2_keep = v->l2_keep ? 1 : 0;
        r.fma2 = v->fma2 ? 1 : 0;
    }
    return r;
}

}  // namespace

namespace ls {
namespace {
std::mutex g_alloc_mu;
long long g_fail_after = -1;       // allocations left before the injected failure (-1: off)
long long g_live_allocs = 0;       // device allocations the library holds

bool injected_failure()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_fail_after < 0) return false;
    if (g_fail_after == 0) {
        g_fail_after = -1;
        return true;
    }
    --g_fail_after;
    return false;
}

void count_alloc(long long d)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_live_allocs += d;
}
}  // namespace

cudaError_t dev_malloc_raw(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) count_alloc(1);
    else *p = nullptr;
    return e;
}

cudaError_t dev_malloc_async_raw(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) count_alloc(1);
    else *p = nullptr;
    return e;
}

cudaError_t dev_free(void *p)
{
    if (!p) return cudaSuccess;
    count_alloc(-1);
    return cudaFree(p);
}

cudaError_t dev_free_async(void *p, cudaStream_t st)
{
    if (!p) return cudaSuccess;
    count_alloc(-1);
    return cudaFreeAsync(p, st);
}
}  // namespace ls

ls_status ls_fail(ls_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

extern "C" {

const char *ls_status_str(ls_status s)
{
    switch (s) {
    case LS_OK: return "ok";
    case LS_ERR_INVALID_ARG: return "invalid argument";
    case LS_ERR_BAD_TABLE: return "inconsistent sub-region table";
    case LS_ERR_UNSUPPORTED: return "unsupported";
    case LS_ERR_OOM: return "out of memory";
    case LS_ERR_CUDA: return "CUDA error";
    case LS_ERR_COMPILE: return "kernel compilation failed";
    case LS_ERR_TIMEOUT: return "device wait timed out";
    case LS_ERR_DEVICE: return "device-side fault reported";
    }
    return "unknown status";
}

const char *ls_last_error(void) { return g_err.c_str(); }

int32_t ls_abi_version(void) { return 8; }

void ls_debug_fail_alloc(int32_t after)
{
    std::lock_guard<std::mutex> lk(ls::g_alloc_mu);
    ls::g_fail_after = after < 0 ? -1 : after;
}

int64_t ls_debug_live_allocs(void)
{
    std::lock_guard<std::mutex> lk(ls::g_alloc_mu);
    return ls::g_live_allocs;
}

ls_status ls_spline_precompile(const ls_spline_desc *desc, ls_dtype dt, const ls_variant *variant)
{
    ls::Table t;
    ls_status st = copy_desc(desc, t);
    if (st != LS_OK) return st;
    if (dt != LS_F32 && dt != LS_BF16 && dt != LS_F16) return ls_fail(LS_ERR_UNSUPPORTED, "coef dtype");
    ls_variant var = default_variant(variant);
    // tensor-core kernel: slots of 128 points (the 128 lanes of tensor memory)
    if (var.tensor && t.sep.empty()) var.block = 128 * ls::tensor_slots(t, var, dt);
    ls::Generated g = ls::generate(t, dt, var);
    std::vector<char> cubin;
    std::string err;
    st = ls::get_cubin(g.source, "ls_" + (t.name.empty() ? std::string("spline") : t.name) + "_" + dtype_tag(dt),
                       cubin, err);
    if (st != LS_OK) return ls_fail(st, err);
    return LS_OK;
}

ls_status ls_spline_generate_source(const ls_spline_desc *desc, ls_dtype dt, const ls_variant *variant, char *buf,
                                    size_t cap, size_t *len)
{
    if (!len) return ls_fail(LS_ERR_INVALID_ARG, "len is NULL");
    ls::Table t;
    ls_status st = copy_desc(desc, t);
    if (st != LS_OK) return st;
    if (dt != LS_F32 && dt != LS_BF16 && dt != LS_F16) return ls_fail(LS_ERR_UNSUPPORTED, "coef dtype");
    ls_variant var = default_variant(variant);
    if (var.tensor && t.sep.empty()) var.block = 128 * ls::tensor_slots(t, var, dt);
    const ls::Generated g = ls::generate(t, dt, var);
    *len = g.source.size();
    if (buf && cap > 0) {
        const size_t m = g.source.size() < cap - 1 ? g.source.size() : cap - 1;
        std::memcpy(buf, g.source.data(), m);
        buf[m] = '\0';
    }
    return LS_OK;
}

ls_status ls_spline_create(const ls_spline_desc *desc, ls_dtype dt, const ls_variant *variant, ls_spline *out)
{
    if (!out) return ls_fail(LS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dt != LS_F32 && dt != LS_BF16 && dt != LS_F16)
        return ls_fail(LS_ERR_UNSUPPORTED, "coefficient storage must be LS_F32, LS_BF16 or LS_F16");
    auto *s = new (std::nothrow) ls_spline_s;
    if (!s) return ls_fail(LS_ERR_OOM, "host allocation");
    ls_status st = copy_desc(desc, s->table);
    if (st != LS_OK) {
        delete s;
        return st;
    }
    s->dtype = dt;
    s->var = default_variant(variant);
    if (s->var.block % 32 || s->var.block > 1024) {
        delete s;
        return ls_fail(LS_ERR_INVALID_ARG, "block must be a multiple of 32, <= 1024");
    }
    if (s->var.producers > 0 && (s->var.producers > 8 || s->var.producers >= s->var.block / 32)) {
        delete s;
        return ls_fail(LS_ERR_INVALID_ARG, "producers must be 1..8 and leave at least one consumer warp");
    }
    if (s->var.tensor) {
        const char *why = nullptr;
        if (!s->table.sep.empty()) why = "tensor: tensor-product tables use the separable path";
        else if (s->var.stage || s->var.pipeline || s->var.producers > 0 || s->var.pts_per_thread > 1)
            why = "tensor excludes stage, pipeline, producers and pts_per_thread";
        if (why) {
            delete s;
            return ls_fail(LS_ERR_INVALID_ARG, why);
        }
    }
    if (s->var.brick >= 2 && s->table.dim != 3) {
        delete s;
        return ls_fail(LS_ERR_UNSUPPORTED, "brick = 2 or 3 (shifted bricked copies) needs a 3D table");
    }
    if (s->var.wait_probe != 0 && (s->var.wait_probe != 1 || s->var.producers <= 0)) {
        delete s;
        return ls_fail(LS_ERR_INVALID_ARG, "wait_probe 1 needs the warp-specialized kernel (producers > 0)");
    }
    if (variant && variant->tensor_kind != 0 && (variant->tensor_kind != 1 || !s->var.tensor || dt != LS_F32)) {
        delete s;
        return ls_fail(LS_ERR_INVALID_ARG, "tensor_kind 1 needs tensor and FP32 coefficients (0 or 1)");
    }
    if (s->var.tensor) s->var.block = 128 * ls::tensor_slots(s->table, s->var, dt);
    if (s->var.stage > 0) {
        const int C = (int)s->table.cosets.size();
        const int edge = s->var.stage > 1 ? s->var.stage : (s->table.scale == 2 ? 12 : 16);
        const char *why = nullptr;
        if (s->table.dim != 3) why = "the staged kernel is 3D only";
        else if (dt != LS_F32) why = "the staged kernel reads FP32 coefficients";
        else if (s->var.brick || s->var.pipeline || s->var.producers > 0)
            why = "stage excludes brick, pipeline and producers";
        else if (edge % 4 || edge < 4 || edge * C > 256 || edge * edge * edge * C * 4 > 160 * 1024)
            why = "stage: the tile edge must be a multiple of 4, edge * cosets <= 256, tile <= 160 KiB";
        if (why) {
            delete s;
            return ls_fail(LS_ERR_INVALID_ARG, why);
        }
    }
    s->gen = ls::generate(s->table, dt, s->var);
    cudaError_t ce = cudaGetDevice(&s->device);
    if (ce != cudaSuccess) {
        delete s;
        return cuda_fail(ce, "cudaGetDevice");
    }
    ce = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (ce != cudaSuccess) {
        delete s;
        return cuda_fail(ce, "cudaDeviceGetAttribute");
    }
    std::string err;
    std::string tag = "ls_" + (s->table.name.empty() ? std::string("spline") : s->table.name) + "_" + dtype_tag(dt);
    st = ls::compile_and_load(s->gen.source, tag, s->mod, err);
    if (st != LS_OK) {
        delete s;
        return ls_fail(st, err);
    }
    if (ls::dev_malloc((void **)&s->status, 256) != cudaSuccess || cudaMemset(s->status, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        if (s->status) ls::dev_free(s->status);
        cudaLibraryUnload(s->mod.lib);
        delete s;
        return ls_fail(LS_ERR_OOM, "status word");
    }
    if ((st = get_kernel(s, "eval", s->mod.eval, s->mod.blocks_per_sm_eval)) != LS_OK ||
        (st = get_kernel(s, "eval_grad", s->mod.eval_grad, s->mod.blocks_per_sm_grad)) != LS_OK ||
        (st = get_kernel(s, "eval_hess", s->mod.eval_hess, s->mod.blocks_per_sm_hess)) != LS_OK ||
        (st = get_kernel(s, "adjoint_atomic", s->mod.adj_atomic, s->mod.blocks_per_sm_adj)) != LS_OK ||
        (st = get_kernel(s, "adjoint_warpagg", s->mod.adj_warpagg, s->mod.blocks_per_sm_warpagg)) != LS_OK ||
        (st = get_kernel(s, "adjoint_fixed", s->mod.adj_fixed, s->mod.blocks_per_sm_fixed)) != LS_OK ||
        (st = get_kernel(s, "adjoint_tile", s->mod.adj_tile, s->mod.blocks_per_sm_tile)) != LS_OK ||
        (st = get_kernel(s, "adjoint_tile_fixed", s->mod.adj_tile_fixed, s->mod.blocks_per_sm_tile_fixed)) != LS_OK ||
        (st = get_kernel(s, "adjoint_bin", s->mod.roe_key, s->mod.blocks_per_sm_gather)) != LS_OK ||
        (st = get_kernel(s, "adjoint_gather", s->mod.adj_gather, s->mod.blocks_per_sm_gather)) != LS_OK) {
        ls::dev_free(s->status);
        cudaLibraryUnload(s->mod.lib);
        delete s;
        return st;
    }
    if (s->gen.info.eval_smem > 0) {
        // warp-specialized value kernel: dynamic shared memory for its slots
        const int smem = s->gen.info.eval_smem;
        int nb = 0;
        cudaError_t e2 = cudaFuncSetAttribute((const void *)s->mod.eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem);
        if (e2 == cudaSuccess)
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)s->mod.eval, s->var.block, smem);
        if (e2 != cudaSuccess || nb < 1) {
            cudaGetLastError();
            ls::dev_free(s->status);
            cudaLibraryUnload(s->mod.lib);
            delete s;
            return ls_fail(LS_ERR_UNSUPPORTED, "the warp-specialized kernel does not fit on an SM (shared memory)");
        }
        s->mod.blocks_per_sm_eval = nb;
    }
    {
        // tiled adjoint kernels: their shared-memory tile and the resulting occupancy
        const struct { cudaKernel_t k; int smem; int *per; } tk[2] = {
            {s->mod.adj_tile, s->gen.info.adj_tile_smem, &s->mod.blocks_per_sm_tile},
            {s->mod.adj_tile_fixed, s->gen.info.adj_tile_fixed_smem, &s->mod.blocks_per_sm_tile_fixed}};
        for (const auto &x : tk) {
            int nb = 0;
            cudaError_t e2 = cudaFuncSetAttribute((const void *)x.k, cudaFuncAttributeMaxDynamicSharedMemorySize, x.smem);
            if (e2 == cudaSuccess)
                e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)x.k, s->var.block, x.smem);
            if (e2 != cudaSuccess || nb < 1) {
                cudaGetLastError();
                nb = 0;               // the tiled modes then take the per-point kernels
            }
            *x.per = nb;
        }
    }
    if (s->gen.info.tmem_cols > 0)
        // tensor-core value (+ gradient) kernels: one block per SM (a block that
        // allocates tensor memory runs alone on its SM); its slots share the 512 columns
        s->mod.blocks_per_sm_eval = s->mod.blocks_per_sm_grad = 1;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)s->mod.eval) == cudaSuccess) s->mod.regs_eval = fa.numRegs;
    else cudaGetLastError();
    *out = s;
    return LS_OK;
}

ls_status ls_spline_destroy(ls_spline s)
{
    if (!s) return LS_OK;
    if (s->mod.lib) cudaLibraryUnload(s->mod.lib);
    if (s->status) ls::dev_free(s->status);
    delete s;
    return LS_OK;
}

ls_status ls_spline_status(ls_spline s, ls_stream stream)
{
    if (!s) return ls_fail(LS_ERR_INVALID_ARG, "spline is NULL");
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, s->status, sizeof v, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess && v) e = cudaMemsetAsync(s->status, 0, sizeof v, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
    if (v) return ls_fail(LS_ERR_TIMEOUT, "a bounded wait in an evaluation kernel gave up");
    return LS_OK;
}

const char *ls_spline_source(ls_spline s) { return s ? s->gen.source.c_str() : ""; }

ls_status ls_spline_info(ls_spline s, int32_t *n_sites, int32_t *fma_value, int32_t *fma_grad, int32_t *regs)
{
    if (!s) return ls_fail(LS_ERR_INVALID_ARG, "spline is NULL");
    if (n_sites) *n_sites = s->gen.info.n_sites;
    if (fma_value) *fma_value = s->gen.info.fma_value;
    if (fma_grad) *fma_grad = s->gen.info.fma_grad;
    if (regs) *regs = s->mod.regs_eval;
    return LS_OK;
}

// ---------------------------------------------------------------------------
// volumes
// ---------------------------------------------------------------------------

static ls_status init_volume(ls_spline s, const int64_t *ext, int32_t layout, ls_volume_s *v)
{
    if (!s || !ext) return ls_fail(LS_ERR_INVALID_ARG, "spline or ext is NULL");
    if (layout < LS_LAYOUT_COSET_MAJOR || layout > LS_LAYOUT_BRICKED_SHIFTED_XYZ)
        return ls_fail(LS_ERR_INVALID_ARG, "unknown layout");
    const int want_brick = layout == LS_LAYOUT_BRICKED ? 1 : layout == LS_LAYOUT_BRICKED_SHIFTED ? 2
                         : layout == LS_LAYOUT_BRICKED_SHIFTED_XYZ ? 3 : 0;
    if (want_brick != s->var.brick)
        return ls_fail(LS_ERR_INVALID_ARG, "the volume's layout and the spline's variant.brick differ (bricked: 1, "
                                           "shifted copies: 2, eight shifted copies: 3, linear layouts: 0)");
    if (want_brick >= 2 && s->table.dim != 3)
        return ls_fail(LS_ERR_UNSUPPORTED, "the shifted bricked copies are 3D only");
    v->spline = s;
    v->layout = layout;
    int64_t prod = 1;
    for (int i = 0; i < 3; ++i) {
        v->ext[i] = i < s->table.dim ? ext[i] : 1;
        if (v->ext[i] < 1 || v->ext[i] > (1 << 20)) return ls_fail(LS_ERR_INVALID_ARG, "extent outside 1..2^20");
        prod *= v->ext[i];
    }
    v->coset_elems = prod;
    v->total_elems = prod * (int64_t)s->table.cosets.size();
    if (want_brick >= 1 &&
        (v->ext[0] % 2 != 0 || (s->table.dim >= 2 && v->ext[1] % 2 != 0) || (s->table.dim == 3 && v->ext[2] % 2 != 0)))
        return ls_fail(LS_ERR_INVALID_ARG, "bricked layout: ext[0], ext[1] and ext[2] must be even");
    if (layout == LS_LAYOUT_BRICKED_SHIFTED)      // four copies over the padded extents
        v->total_elems = 4 * (int64_t)s->table.cosets.size() * (v->ext[0] + 2) * (v->ext[1] + 2) * v->ext[2];
    if (layout == LS_LAYOUT_BRICKED_SHIFTED_XYZ)  // eight copies
        v->total_elems = 8 * (int64_t)s->table.cosets.size() * (v->ext[0] + 2) * (v->ext[1] + 2) * (v->ext[2] + 2);
    if (v->total_elems >= (int64_t)1 << 31)
        return ls_fail(LS_ERR_UNSUPPORTED, "volume exceeds 2^31 coefficients (32-bit addressing)");
    return LS_OK;
}

// TMA tensor map of the coefficient array for the staged value kernel: the
// interleaved layout as a 3D FP32 tensor (E0 * C, E1, E2), the coset-major one
// as 4D (E0, E1, E2, C); box = the kernel's tile (edge per axis, all cosets);
// out-of-bounds elements read as zero.  Volumes the map cannot describe (rows
// not a multiple of 16 bytes, an unaligned base) keep tmap = NULL, and the
// staged kernel then reads global memory in every block.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static ls_status volume_tensor_map(ls_volume_s *v)
{
    ls_spline_s *s = v->spline;
    const int edge = s->gen.info.stage_edge;
    if (edge <= 0 || s->dtype != LS_F32 || s->table.dim != 3 || v->layout == LS_LAYOUT_BRICKED) return LS_OK;
    const int64_t C = (int64_t)s->table.cosets.size();
    const int64_t E0 = v->ext[0], E1 = v->ext[1], E2 = v->ext[2];
    const bool inter = v->layout == LS_LAYOUT_INTERLEAVED || C == 1;
    const int64_t row = inter ? E0 * C : E0;
    if ((reinterpret_cast<uintptr_t>(v->coef) & 15) || (row * 4) % 16) return LS_OK;
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return ls_fail(LS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        }
        encode = (EncodeTiledFn)fn;
    }
    alignas(64) CUtensorMap m;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    if (inter) {
        rank = 3;
        dims[0] = (cuuint64_t)(E0 * C); dims[1] = (cuuint64_t)E1; dims[2] = (cuuint64_t)E2;
        strides[0] = (cuuint64_t)(E0 * C * 4); strides[1] = (cuuint64_t)(E0 * C * E1 * 4);
        box[0] = (cuuint32_t)(edge * C); box[1] = box[2] = (cuuint32_t)edge;
    } else {
        rank = 4;
        dims[0] = (cuuint64_t)E0; dims[1] = (cuuint64_t)E1; dims[2] = (cuuint64_t)E2; dims[3] = (cuuint64_t)C;
        strides[0] = (cuuint64_t)(E0 * 4); strides[1] = (cuuint64_t)(E0 * E1 * 4);
        strides[2] = (cuuint64_t)(E0 * E1 * E2 * 4);
        box[0] = box[1] = box[2] = (cuuint32_t)edge; box[3] = (cuuint32_t)C;
    }
    if ((box[0] * 4) % 16) return LS_OK;
    CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, v->coef, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return ls_fail(LS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    cudaError_t e = ls::dev_malloc(&v->tmap, sizeof(CUtensorMap));
    if (e != cudaSuccess) {
        v->tmap = nullptr;
        return cuda_fail(e, "cudaMalloc (tensor map)");
    }
    e = cudaMemcpy(v->tmap, &m, sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (tensor map)");
    v->tmap_edge = edge;
    return LS_OK;
}

ls_status ls_volume_create(ls_spline s, const int64_t *ext, int32_t layout, ls_volume *out)
{
    if (!out) return ls_fail(LS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    auto *v = new (std::nothrow) ls_volume_s;
    if (!v) return ls_fail(LS_ERR_OOM, "host allocation");
    ls_status st = init_volume(s, ext, layout, v);
    if (st != LS_OK) {
        delete v;
        return st;
    }
    size_t bytes = (size_t)v->total_elems * dtype_size(s->dtype);
    cudaError_t e = ls::dev_malloc(&v->coef, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete v;
        return ls_fail(LS_ERR_OOM, "cudaMalloc of the coefficient volume failed");
    }
    e = cudaMemset(v->coef, 0, bytes);
    if (e != cudaSuccess) {
        ls::dev_free(v->coef);
        delete v;
        return cuda_fail(e, "cudaMemset");
    }
    v->owned = true;
    st = volume_tensor_map(v);
    if (st != LS_OK) {
        ls_volume_destroy(v);
        return st;
    }
    *out = v;
    return LS_OK;
}

ls_status ls_volume_wrap(ls_spline s, const int64_t *ext, int32_t layout, void *device_coef, ls_volume *out)
{
    if (!out || !device_coef) return ls_fail(LS_ERR_INVALID_ARG, "out or device_coef is NULL");
    *out = nullptr;
    auto *v = new (std::nothrow) ls_volume_s;
    if (!v) return ls_fail(LS_ERR_OOM, "host allocation");
    ls_status st = init_volume(s, ext, layout, v);
    if (st != LS_OK) {
        delete v;
        return st;
    }
    v->coef = device_coef;
    v->owned = false;
    st = volume_tensor_map(v);
    if (st != LS_OK) {
        ls_volume_destroy(v);
        return st;
    }
    *out = v;
    return LS_OK;
}

void *ls_volume_device_ptr(ls_volume v) { return v ? v->coef : nullptr; }

int32_t ls_volume_layout(ls_volume v) { return v ? v->layout : -1; }

ls_status ls_relayout(const void *src, int32_t src_layout, void *dst, int32_t dst_layout, int32_t n_cosets,
                      const int64_t *ext, int32_t elem_bytes, ls_stream stream)
{
    if (!ext || n_cosets < 1 || n_cosets > 8) return ls_fail(LS_ERR_INVALID_ARG, "ext NULL or n_cosets outside 1..8");
    if (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8) return ls_fail(LS_ERR_INVALID_ARG, "elem_bytes");
    int64_t per = 1;
    for (int i = 0; i < 3; ++i) {
        if (ext[i] < 1 || ext[i] > (1 << 20)) return ls_fail(LS_ERR_INVALID_ARG, "extent outside 1..2^20");
        per *= ext[i];
    }
    if (per * n_cosets >= ((int64_t)1 << 31)) return ls_fail(LS_ERR_UNSUPPORTED, "2^31 or more elements");
    for (int32_t l : {src_layout, dst_layout}) {
        if (l < LS_LAYOUT_COSET_MAJOR || l > LS_LAYOUT_BRICKED_SHIFTED_XYZ)
            return ls_fail(LS_ERR_INVALID_ARG, "unknown layout");
        if (l >= LS_LAYOUT_BRICKED && (ext[0] % 2 != 0 || ext[1] % 2 != 0 || (ext[2] != 1 && ext[2] % 2 != 0)))
            return ls_fail(LS_ERR_INVALID_ARG, "bricked layout: extents are not whole bricks");
        if (l >= LS_LAYOUT_BRICKED_SHIFTED && ext[2] == 1)
            return ls_fail(LS_ERR_UNSUPPORTED, "the shifted bricked copies are 3D only");
        if (l >= LS_LAYOUT_BRICKED_SHIFTED &&
            8 * n_cosets * (ext[0] + 2) * (ext[1] + 2) * (ext[2] + 2) >= ((int64_t)1 << 31))
            return ls_fail(LS_ERR_UNSUPPORTED, "2^31 or more elements");
    }
    if (!src || !dst || src == dst) return ls_fail(LS_ERR_INVALID_ARG, "src, dst NULL or the same buffer");
    const lsk::LayoutGeom sg{src_layout, n_cosets, (long long)per, (int)ext[0], (int)ext[1], (int)ext[2]};
    lsk::LayoutGeom dg = sg;
    dg.layout = dst_layout;
    cudaError_t e = lsk::relayout(src, sg, dst, dg, elem_bytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "relayout kernel");
    return LS_OK;
}

ls_status ls_volume_upload(ls_volume v, const void *src, int32_t src_is_device, ls_dtype src_dt, ls_stream stream)
{
    if (!v || !src) return ls_fail(LS_ERR_INVALID_ARG, "volume or src is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const ls_dtype dst_dt = v->spline->dtype;
    const size_t n = (size_t)v->total_elems;
    if (dtype_size(src_dt) == 0) return ls_fail(LS_ERR_INVALID_ARG, "src dtype");
    const int ncos = (int)v->spline->table.cosets.size();
    const lsk::LayoutGeom dg{v->layout, ncos, (long long)v->coset_elems, (int)v->ext[0], (int)v->ext[1],
                             (int)v->ext[2]};
    lsk::LayoutGeom sg = dg;
    sg.layout = LS_LAYOUT_COSET_MAJOR;
    const bool same_order = v->layout == LS_LAYOUT_COSET_MAJOR || (v->layout == LS_LAYOUT_INTERLEAVED && ncos == 1);
    if (src_dt == dst_dt && same_order) {
        cudaError_t e = cudaMemcpyAsync(v->coef, src, n * dtype_size(dst_dt),
                                        src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        return LS_OK;
    }
    const void *dsrc = src;
    void *tmp = nullptr;
    if (!src_is_device) {
        cudaError_t e = ls::dev_malloc_async(&tmp, n * dtype_size(src_dt), st);
        if (e != cudaSuccess) return ls_fail(LS_ERR_OOM, "staging allocation for upload");
        e = cudaMemcpyAsync(tmp, src, n * dtype_size(src_dt), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            ls::dev_free_async(tmp, st);
            return cuda_fail(e, "cudaMemcpyAsync");
        }
        dsrc = tmp;
    }
    cudaError_t e = lsk::convert_relayout(dsrc, (int)src_dt, sg, v->coef, (int)dst_dt, dg, st);
    if (tmp) ls::dev_free_async(tmp, st);
    if (e != cudaSuccess) return cuda_fail(e, "convert kernel");
    return LS_OK;
}

ls_status ls_volume_destroy(ls_volume v)
{
    if (!v) return LS_OK;
    for (int i = 0; i < 2; ++i)
        if (v->hs[i]) {
            cudaStreamSynchronize(v->hs[i]);
            cudaStreamDestroy(v->hs[i]);
        }
    for (int i = 0; i < 3; ++i)
        if (v->hev[i]) cudaEventDestroy(v->hev[i]);
    if (v->owned && v->coef) ls::dev_free(v->coef);
    if (v->stage) ls::dev_free(v->stage);
    if (v->tex) cudaDestroyTextureObject(v->tex);
    if (v->tex_array) cudaFreeArray(v->tex_array);
    if (v->tmap) ls::dev_free(v->tmap);
    delete v;
    return LS_OK;
}

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------

static size_t al256b(size_t b) { return (b + 255) & ~(size_t)255; }

static void fill_eval_args(ls_volume v, const float *pts, int64_t n, float *out, float *grad, EvalArgsH &a)
{
    a.pts = pts;
    a.out = out;
    a.grad = grad;
    a.coef = v->coef;
    a.n = n;
    a.e0 = (int)v->ext[0];
    a.e1 = (int)v->ext[1];
    a.e2 = (int)v->ext[2];
    a.cstride = vol_cstride(v);
    a.cunit = vol_cunit(v);
    a.status = v->spline->status;
    a.hess = nullptr;
    a.tmap = v->tmap;
}

ls_status ls_eval(ls_volume v, const float *pts, int64_t n, float *out, ls_stream stream)
{
    if (!v || (n > 0 && (!pts || !out))) return ls_fail(LS_ERR_INVALID_ARG, "volume, pts or out is NULL");
    if (n < 0) return ls_fail(LS_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return LS_OK;
    ls_spline_s *s = v->spline;
    EvalArgsH a;
    fill_eval_args(v, pts, n, out, nullptr, a);
    const int T = (s->var.pts_per_thread > 1 && s->table.sep.empty()) ? s->var.pts_per_thread : 1;
    const int per_sm = s->var.blocks_per_sm > 0 ? std::min(s->var.blocks_per_sm, s->mod.blocks_per_sm_eval)
                                                : s->mod.blocks_per_sm_eval;
    return launch(s->mod.eval, grid_for((n + T - 1) / T, s->var.block, s->num_sms, per_sm), s->var.block, &a,
                  (cudaStream_t)stream, (size_t)s->gen.info.eval_smem);
}

ls_status ls_eval_grad(ls_volume v, const float *pts, int64_t n, float *val, float *grad, ls_stream stream)
{
    if (!v || (n > 0 && (!pts || !grad))) return ls_fail(LS_ERR_INVALID_ARG, "volume, pts or grad is NULL");
    if (n < 0) return ls_fail(LS_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return LS_OK;
    ls_spline_s *s = v->spline;
    EvalArgsH a;
    fill_eval_args(v, pts, n, val, grad, a);
    const int per_sm = s->var.blocks_per_sm > 0 ? std::min(s->var.blocks_per_sm, s->mod.blocks_per_sm_grad)
                                                : s->mod.blocks_per_sm_grad;
    return launch(s->mod.eval_grad, grid_for(n, s->var.block, s->num_sms, per_sm), s->var.block, &a,
                  (cudaStream_t)stream);
}

ls_status ls_eval_hess(ls_volume v, const float *pts, int64_t n, float *val, float *grad, float *hess,
                       ls_stream stream)
{
    if (!v || (n > 0 && (!pts || !hess))) return ls_fail(LS_ERR_INVALID_ARG, "volume, pts or hess is NULL");
    if (n < 0) return ls_fail(LS_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return LS_OK;
    ls_spline_s *s = v->spline;
    EvalArgsH a;
    fill_eval_args(v, pts, n, val, grad, a);
    a.hess = hess;
    return launch(s->mod.eval_hess, grid_for(n, s->var.block, s->num_sms, s->mod.blocks_per_sm_hess), s->var.block,
                  &a, (cudaStream_t)stream);
}

ls_status ls_eval_host_multi(int32_t n_vol, const ls_volume *vols, const float *host_pts, int64_t n,
                             float *const *host_out, ls_stream stream)
{
    if (n_vol < 1 || !vols || !vols[0] || !host_out || (n > 0 && !host_pts)) return ls_fail(LS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return ls_fail(LS_ERR_INVALID_ARG, "n < 0");
    const int D = vols[0]->spline->table.dim;
    for (int k = 0; k < n_vol; ++k) {
        if (!vols[k] || (n > 0 && !host_out[k])) return ls_fail(LS_ERR_INVALID_ARG, "NULL volume or output");
        if (vols[k]->spline->table.dim != D) return ls_fail(LS_ERR_INVALID_ARG, "volumes of different dimension");
    }
    if (n == 0) return LS_OK;
    ls_volume_s *v = vols[0];
    cudaStream_t user = (cudaStream_t)stream;
    // chunking: two stages, each holding one chunk of points and n_vol outputs
    const int64_t chunk = std::min<int64_t>(n, (int64_t)1 << 20);
    const size_t pbytes = al256b((size_t)chunk * D * 4), obytes = al256b((size_t)chunk * 4);
    const size_t stage_one = pbytes + obytes * n_vol;
    const size_t need = 2 * stage_one;
    cudaError_t e;
    if (!v->hs[0]) {
        for (int i = 0; i < 2; ++i)
            if ((e = cudaStreamCreateWithFlags(&v->hs[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate");
        for (int i = 0; i < 3; ++i)
            if ((e = cudaEventCreateWithFlags(&v->hev[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreate");
    }
    if (v->stage_bytes < need) {
        if (v->stage) {
            cudaStreamSynchronize(v->hs[0]);
            cudaStreamSynchronize(v->hs[1]);
            ls::dev_free(v->stage);
            v->stage = nullptr;
            v->stage_bytes = 0;
        }
        if (ls::dev_malloc(&v->stage, need) != cudaSuccess) {
            cudaGetLastError();
            return ls_fail(LS_ERR_OOM, "staging buffers for ls_eval_host");
        }
        v->stage_bytes = need;
    }
    // order after the caller's queued work
    if ((e = cudaEventRecord(v->hev[2], user)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int i = 0; i < 2; ++i)
        if ((e = cudaStreamWaitEvent(v->hs[i], v->hev[2], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    // an error inside the chunk loop first drains both internal streams, so no
    // copy into the caller's host buffers is still queued when the call returns
    auto drain = [&]() {
        cudaStreamSynchronize(v->hs[0]);
        cudaStreamSynchronize(v->hs[1]);
    };
    int64_t c = 0;
    for (int64_t p0 = 0; p0 < n; p0 += chunk, ++c) {
        const int si = (int)(c & 1);
        cudaStream_t s = v->hs[si];
        const int64_t m = std::min<int64_t>(chunk, n - p0);
        float *dp = (float *)((char *)v->stage + si * stage_one);
        if ((e = cudaMemcpyAsync(dp, host_pts + p0 * D, (size_t)m * D * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
            drain();
            return cuda_fail(e, "cudaMemcpyAsync H2D");
        }
        for (int k = 0; k < n_vol; ++k) {
            float *dout = (float *)((char *)dp + pbytes + k * obytes);
            ls_status st = ls_eval(vols[k], dp, m, dout, (ls_stream)s);
            if (st != LS_OK) {
                drain();
                return st;
            }
            if ((e = cudaMemcpyAsync(host_out[k] + p0, dout, (size_t)m * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
                drain();
                return cuda_fail(e, "cudaMemcpyAsync D2H");
            }
        }
    }
    for (int i = 0; i < 2; ++i)
        if ((e = cudaStreamSynchronize(v->hs[i])) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return LS_OK;
}

ls_status ls_eval_host(ls_volume v, const float *host_pts, int64_t n, float *host_out, ls_stream stream)
{
    return ls_eval_host_multi(1, &v, host_pts, n, &host_out, stream);
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------

namespace {
// Bins of the deterministic adjoint: every lattice site of the haloed grid.
uint64_t adjoint_nbins(ls_volume v)
{
    const int H = v->spline->gen.info.halo;
    uint64_t cs = 1;
    for (int i = 0; i < v->spline->table.dim; ++i) cs *= (uint64_t)(v->ext[i] + 2 * H);
    return cs * v->spline->table.cosets.size();
}
}  // namespace

size_t ls_adjoint_scratch_bytes(ls_volume v, int64_t n)
{
    if (!v || n < 0) return 0;
    const size_t N = (size_t)n;
    const size_t binned = al256b(N * 4) * 2 + al256b(N * 16) * 2 + al256b((adjoint_nbins(v) + 2) * 4) +
                          lsk::sort_scratch_bytes(n > 0 ? n : 1) + 256;
    const size_t fixed = al256b((size_t)v->total_elems * 8) + lsk::fixed_ws_bytes() + 256;
    return binned > fixed ? binned : fixed;
}

// resident blocks per SM for a launch: the occupancy figure, capped by
// variant.blocks_per_sm when set
static int per_sm_of(const ls_spline_s *s, int occupancy)
{
    return s->var.blocks_per_sm > 0 ? std::max(1, std::min(s->var.blocks_per_sm, occupancy)) : occupancy;
}

ls_status ls_adjoint_coef(ls_volume v, const float *pts, const float *gout, int64_t n, float *dcoef,
                          int32_t mode, void *scratch, ls_stream stream)
{
    if (mode != LS_ADJ_ATOMIC && mode != LS_ADJ_DETERMINISTIC && mode != LS_ADJ_ATOMIC_WARP &&
        mode != LS_ADJ_DETERMINISTIC_FIXED && mode != LS_ADJ_ATOMIC_TILED && mode != LS_ADJ_DETERMINISTIC_FIXED_TILED)
        return ls_fail(LS_ERR_INVALID_ARG, "unknown adjoint mode");
    if (!v || (n > 0 && (!pts || !gout || !dcoef))) return ls_fail(LS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return ls_fail(LS_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return LS_OK;
    if (v->layout >= LS_LAYOUT_BRICKED_SHIFTED)
        return ls_fail(LS_ERR_UNSUPPORTED, "the shifted bricked copies are read-only (evaluation kernels)");
    ls_spline_s *s = v->spline;
    cudaStream_t st = (cudaStream_t)stream;
    // the tiled kernels address the linear layouts; elsewhere (and if their
    // tile does not fit an SM) the per-point kernels do the same sums
    const bool tiled_ok = v->layout != LS_LAYOUT_BRICKED;
    if (mode == LS_ADJ_ATOMIC_TILED && (!tiled_ok || s->mod.blocks_per_sm_tile < 1)) mode = LS_ADJ_ATOMIC;
    if (mode == LS_ADJ_DETERMINISTIC_FIXED_TILED && (!tiled_ok || s->mod.blocks_per_sm_tile_fixed < 1))
        mode = LS_ADJ_DETERMINISTIC_FIXED;
    if (mode == LS_ADJ_DETERMINISTIC_FIXED || mode == LS_ADJ_DETERMINISTIC_FIXED_TILED) {
        const size_t need = ls_adjoint_scratch_bytes(v, n);
        void *ws = scratch;
        if (!ws && ls::dev_malloc_async(&ws, need, st) != cudaSuccess) {
            cudaGetLastError();
            return ls_fail(LS_ERR_OOM, "scratch for the fixed-point adjoint");
        }
        unsigned long long *acc = (unsigned long long *)ws;
        void *fws = (char *)ws + al256b((size_t)v->total_elems * 8);
        float *scale = nullptr;
        double *inv = nullptr;
        ls_status res = LS_OK;
        cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)v->total_elems * 8, st);
        if (e == cudaSuccess) e = lsk::fixed_prepare(gout, n, s->gen.info.wmax, fws, &scale, &inv, st);
        if (e != cudaSuccess) res = cuda_fail(e, "fixed-point adjoint setup");
        if (res == LS_OK) {
            AdjArgsH a{pts, gout, dcoef, (long long)n, (int)v->ext[0], (int)v->ext[1], (int)v->ext[2],
                       vol_cstride(v), vol_cunit(v), acc, scale};
            if (mode == LS_ADJ_DETERMINISTIC_FIXED_TILED)
                res = launch(s->mod.adj_tile_fixed, grid_for(n, s->var.block, s->num_sms, per_sm_of(s, s->mod.blocks_per_sm_tile_fixed)),
                             s->var.block, &a, st, (size_t)s->gen.info.adj_tile_fixed_smem);
            else
                res = launch(s->mod.adj_fixed, grid_for(n, s->var.block, s->num_sms, per_sm_of(s, s->mod.blocks_per_sm_fixed)),
                             s->var.block, &a, st);
        }
        if (res == LS_OK && (e = lsk::fixed_finish(acc, inv, dcoef, v->total_elems, st)) != cudaSuccess)
            res = cuda_fail(e, "fixed-point adjoint finish");
        if (!scratch) ls::dev_free_async(ws, st);
        return res;
    }
    if (mode != LS_ADJ_DETERMINISTIC) {
        AdjArgsH a{pts, gout, dcoef, (long long)n, (int)v->ext[0], (int)v->ext[1], (int)v->ext[2],
                   vol_cstride(v), vol_cunit(v), nullptr, nullptr};
        if (mode == LS_ADJ_ATOMIC_WARP)
            return launch(s->mod.adj_warpagg, grid_for(n, s->var.block, s->num_sms, per_sm_of(s, s->mod.blocks_per_sm_warpagg)),
                          s->var.block, &a, st);
        if (mode == LS_ADJ_ATOMIC_TILED)
            return launch(s->mod.adj_tile, grid_for(n, s->var.block, s->num_sms, per_sm_of(s, s->mod.blocks_per_sm_tile)),
                          s->var.block, &a, st, (size_t)s->gen.info.adj_tile_smem);
        return launch(s->mod.adj_atomic, grid_for(n, s->var.block, s->num_sms, per_sm_of(s, s->mod.blocks_per_sm_adj)),
                      s->var.block, &a, st);
    }
    if (n > ((int64_t)1 << 31) - 1) return ls_fail(LS_ERR_UNSUPPORTED, "more than 2^31-1 points");
    const uint64_t nbins = adjoint_nbins(v);
    if (nbins >= ((uint64_t)1 << 31)) return ls_fail(LS_ERR_UNSUPPORTED, "binning grid exceeds 2^31 sites");
    int nbits = 1;
    while (((uint64_t)1 << nbits) <= nbins) ++nbits;
    const size_t N = (size_t)n;
    const size_t need = ls_adjoint_scratch_bytes(v, n);
    void *ws = scratch;
    if (!ws && ls::dev_malloc_async(&ws, need, st) != cudaSuccess) {
        cudaGetLastError();
        return ls_fail(LS_ERR_OOM, "scratch for the deterministic adjoint");
    }
    char *p = (char *)ws;
    uint32_t *key = (uint32_t *)p;
    p += al256b(N * 4);
    int32_t *idx = (int32_t *)p;
    p += al256b(N * 4);
    float *rec = (float *)p;
    p += al256b(N * 16);
    float *srec = (float *)p;
    p += al256b(N * 16);
    uint32_t *start = (uint32_t *)p;
    p += al256b((nbins + 2) * 4);
    void *sort_ws = p;
    const int H = s->gen.info.halo;
    ls_status res = LS_OK;
    BinArgsH ba{pts, gout, key, idx, rec, (long long)n, (int)v->ext[0], (int)v->ext[1], (int)v->ext[2], H,
                (uint32_t)nbins};
    res = launch(s->mod.roe_key, grid_for(n, s->var.block, s->num_sms, 8), s->var.block, &ba, st);
    cudaError_t e = cudaSuccess;
    if (res == LS_OK) e = lsk::radix_sort_pairs(key, idx, n, nbits, sort_ws, st);
    if (res == LS_OK && e == cudaSuccess) e = lsk::permute_rows(rec, idx, n, 4, 0, srec, st);
    if (res == LS_OK && e == cudaSuccess) e = lsk::bin_starts(key, n, (uint32_t)nbins, start, st);
    if (res == LS_OK && e != cudaSuccess) res = cuda_fail(e, "deterministic adjoint kernels");
    if (res == LS_OK) {
        GatherArgsH ga{srec, start, dcoef, (int)v->ext[0], (int)v->ext[1], (int)v->ext[2], vol_cstride(v), vol_cunit(v),
                       H};
        res = launch(s->mod.adj_gather, grid_for(v->total_elems, s->var.block, s->num_sms, 8), s->var.block, &ga, st);
    }
    if (!scratch) ls::dev_free_async(ws, st);
    return res;
}

// ---------------------------------------------------------------------------
// FP64 device dot product
// ---------------------------------------------------------------------------

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t ls_morton_scratch_bytes(int64_t n)
{
    if (n <= 0) return 256;
    return al256((size_t)n * 4) + lsk::sort_scratch_bytes(n);
}

ls_status ls_morton_sort(const float *pts, int64_t n, const float *origin, float cell, int32_t *perm,
                         uint32_t *keys_out, void *scratch, ls_stream stream)
{
    if (n < 0 || (n > 0 && (!pts || !perm)) || !origin) return ls_fail(LS_ERR_INVALID_ARG, "NULL argument");
    if (!(cell > 0.0f) || !std::isfinite(cell)) return ls_fail(LS_ERR_INVALID_ARG, "cell must be positive");
    if (n == 0) return LS_OK;
    if (n > ((int64_t)1 << 31) - 1) return ls_fail(LS_ERR_UNSUPPORTED, "more than 2^31-1 points");
    cudaStream_t st = (cudaStream_t)stream;
    void *ws = scratch;
    const size_t need = ls_morton_scratch_bytes(n);
    if (!ws) {
        if (ls::dev_malloc_async(&ws, need, st) != cudaSuccess) {
            cudaGetLastError();
            return ls_fail(LS_ERR_OOM, "scratch for ls_morton_sort");
        }
    }
    uint32_t *keys = keys_out ? keys_out : (uint32_t *)ws;
    void *sort_ws = (char *)ws + al256((size_t)n * 4);
    cudaError_t e = lsk::morton_keys(pts, n, origin, cell, keys, perm, st);
    if (e == cudaSuccess) e = lsk::radix_sort_pairs(keys, perm, n, 30, sort_ws, st);
    if (!scratch) ls::dev_free_async(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "morton sort kernels");
    return LS_OK;
}

ls_status ls_permute_rows(const float *src, const int32_t *perm, int64_t n, int32_t width, int32_t inverse,
                          float *dst, ls_stream stream)
{
    if (n < 0 || width < 1 || (n > 0 && (!src || !perm || !dst))) return ls_fail(LS_ERR_INVALID_ARG, "bad argument");
    if (src == dst) return ls_fail(LS_ERR_INVALID_ARG, "src and dst must differ");
    cudaError_t e = lsk::permute_rows(src, perm, n, width, inverse, dst, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "permute kernel");
    return LS_OK;
}

ls_status ls_probe_gather(const float *table, int64_t table_elems, int32_t loads, float *out, int64_t nthreads,
                          int32_t blocks, ls_stream stream)
{
    if (!table || !out || table_elems < 1 || loads < 1 || nthreads < 1) return ls_fail(LS_ERR_INVALID_ARG, "bad argument");
    cudaError_t e = lsk::gather_probe(table, table_elems, loads, out, nthreads, blocks > 0 ? blocks : 148 * 8,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gather probe");
    return LS_OK;
}

ls_status ls_dot_f64(const float *a, const float *b, int64_t n, double *result, ls_stream stream)
{
    if (n < 0 || (n > 0 && (!a || !b)) || !result) return ls_fail(LS_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = lsk::dot_f64(a, b, (long long)n, result, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "dot kernel");
    return LS_OK;
}

}  // extern "C"
