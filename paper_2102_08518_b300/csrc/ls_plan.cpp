// Batched persistent evaluation: many volumes (mixed splines and storage
// types), each with its own points, in one launch of a generated kernel that
// takes (volume, tile) work items from a device list.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ls_internal.h"

struct ls_plan_s {
    ls::Module mod;
    cudaKernel_t kernel = nullptr;
    void *dev = nullptr;                 // vols | items | counters
    int n_items = 0;
    int grid = 0;
    int block = 256;
    int tile = 0;
    void *vols_d = nullptr, *items_d = nullptr;
    unsigned *counter_d = nullptr;       // [ticket, exit ticket, status]
};

namespace {

struct BatchVol {
    const float *pts;
    float *out;
    const void *coef;
    long long n;
    int e0, e1, e2, cstride, kind, cunit;
};
struct BatchItem {
    int vol;
    int pad;
    long long p0, p1;
};
struct BatchArgs {
    const void *vols;
    const void *items;
    int nitems;
    int pad;
    unsigned *counter;
    unsigned *status;
};

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

std::mutex g_tune_mu;
std::map<std::string, int> g_tuned;     // (kernel tag, sizes) -> tile

ls_status cuda_err(cudaError_t e, const char *what)
{
    return ls_fail(LS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::vector<BatchItem> make_items(const std::vector<BatchVol> &vols, const std::vector<double> &cost, int tile)
{
    std::vector<std::pair<double, BatchItem>> v;
    for (size_t k = 0; k < vols.size(); ++k)
        for (long long p0 = 0; p0 < vols[k].n; p0 += tile) {
            BatchItem it{(int)k, 0, p0, std::min<long long>(p0 + tile, vols[k].n)};
            v.push_back({cost[k] * (double)(it.p1 - it.p0), it});
        }
    // most expensive items first: dynamic pulling then balances the tail
    std::stable_sort(v.begin(), v.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<BatchItem> out;
    out.reserve(v.size());
    for (auto &x : v) out.push_back(x.second);
    return out;
}

ls_status upload_items(ls_plan_s *p, const std::vector<BatchItem> &items)
{
    if (p->items_d) ls::dev_free(p->items_d);
    p->items_d = nullptr;
    if (ls::dev_malloc(&p->items_d, std::max<size_t>(1, items.size()) * sizeof(BatchItem)) != cudaSuccess) {
        cudaGetLastError();
        return ls_fail(LS_ERR_OOM, "plan work list");
    }
    cudaError_t e = cudaMemcpy(p->items_d, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(e, "upload work list");
    p->n_items = (int)items.size();
    return LS_OK;
}

ls_status launch_plan(ls_plan_s *p, cudaStream_t st)
{
    BatchArgs a{p->vols_d, p->items_d, p->n_items, 0, p->counter_d, p->counter_d + 2};
    void *argv[] = {&a};
    cudaError_t e = cudaLaunchKernel((const void *)p->kernel, dim3(p->grid), dim3(p->block), argv, 0, st);
    if (e != cudaSuccess) return cuda_err(e, "cudaLaunchKernel (plan)");
    return LS_OK;
}

}  // namespace

extern "C" {

ls_status ls_plan_create(int32_t n_vol, const ls_volume *vols, const float *const *pts, const int64_t *n,
                         float *const *out, int32_t tile, ls_plan *plan)
{
    if (!plan || n_vol < 1 || !vols || !pts || !n || !out) return ls_fail(LS_ERR_INVALID_ARG, "bad argument");
    *plan = nullptr;
    if (tile < 0) return ls_fail(LS_ERR_INVALID_ARG, "tile < 0");
    // distinct splines -> kernel kinds
    std::vector<ls_spline_s *> kinds;
    std::vector<BatchVol> bv(n_vol);
    std::vector<double> cost(n_vol);
    for (int k = 0; k < n_vol; ++k) {
        ls_volume_s *v = vols[k];
        if (!v || n[k] < 0 || (n[k] > 0 && (!pts[k] || !out[k]))) return ls_fail(LS_ERR_INVALID_ARG, "bad volume entry");
        auto it = std::find(kinds.begin(), kinds.end(), v->spline);
        int kind = (int)(it - kinds.begin());
        if (it == kinds.end()) kinds.push_back(v->spline);
        bv[k] = BatchVol{pts[k], out[k], v->coef, (long long)n[k], (int)v->ext[0], (int)v->ext[1], (int)v->ext[2],
                         vol_cstride(v), kind, vol_cunit(v)};
        cost[k] = 20.0 + (double)v->spline->gen.info.fma_value;
    }
    if (kinds.size() > 16) return ls_fail(LS_ERR_UNSUPPORTED, "more than 16 distinct splines in one plan");
    std::vector<const ls::Table *> tabs;
    std::vector<ls_dtype> dts;
    std::vector<int> bricks;
    std::string tag = "ls_batch";
    for (auto *s : kinds) {
        tabs.push_back(&s->table);
        dts.push_back(s->dtype);
        bricks.push_back(s->var.brick);
        tag += "_" + (s->table.name.empty() ? std::string("s") : s->table.name);
    }
    if (tag.size() > 120) tag = tag.substr(0, 120);
    ls_variant var{256, 1, 0, 0, 0, 0, 0};
    ls::Generated g = ls::generate_batch(tabs, dts, bricks, var);
    auto *p = new (std::nothrow) ls_plan_s;
    if (!p) return ls_fail(LS_ERR_OOM, "host allocation");
    std::string err;
    ls_status st = ls::compile_and_load(g.source, tag, p->mod, err);
    if (st != LS_OK) {
        delete p;
        return ls_fail(st, err);
    }
    cudaError_t e = cudaLibraryGetKernel(&p->kernel, p->mod.lib, "ls_batch_eval");
    if (e != cudaSuccess) {
        cudaLibraryUnload(p->mod.lib);
        delete p;
        return cuda_err(e, "cudaLibraryGetKernel ls_batch_eval");
    }
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)p->kernel, var.block, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 2;
    }
    p->block = var.block;
    p->grid = sms * per_sm;
    // device arrays: volume table and counters
    if (ls::dev_malloc(&p->dev, al(n_vol * sizeof(BatchVol)) + 256) != cudaSuccess) {
        cudaGetLastError();
        cudaLibraryUnload(p->mod.lib);
        delete p;
        return ls_fail(LS_ERR_OOM, "plan volume table");
    }
    p->vols_d = p->dev;
    p->counter_d = (unsigned *)((char *)p->dev + al(n_vol * sizeof(BatchVol)));
    e = cudaMemcpy(p->vols_d, bv.data(), n_vol * sizeof(BatchVol), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->counter_d, 0, 256);
    if (e != cudaSuccess) {
        ls_plan_destroy(p);
        return cuda_err(e, "plan setup");
    }
    // tile: given, cached, or timed
    std::string key = tag + "|" + std::to_string(g.source.size());
    for (int k = 0; k < n_vol; ++k) key += "|" + std::to_string(kinds.size()) + ":" + std::to_string(bv[k].kind) + "/" + std::to_string(bv[k].n);
    int chosen = tile;
    if (chosen == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) chosen = it->second;
    }
    if (chosen == 0) {
        const int cands[] = {512, 1024, 2048, 4096, 8192, 16384};
        float best = 1e30f;
        cudaStream_t ts;
        cudaEvent_t e0, e1;
        cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int c : cands) {
            if ((st = upload_items(p, make_items(bv, cost, c))) != LS_OK) break;
            launch_plan(p, ts);                            // warm-up
            cudaEventRecord(e0, ts);
            for (int r = 0; r < 3; ++r) launch_plan(p, ts);
            cudaEventRecord(e1, ts);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                chosen = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(ts);
        if (st != LS_OK) {
            ls_plan_destroy(p);
            return st;
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = chosen;
    }
    p->tile = chosen;
    if ((st = upload_items(p, make_items(bv, cost, chosen))) != LS_OK) {
        ls_plan_destroy(p);
        return st;
    }
    *plan = p;
    return LS_OK;
}

ls_status ls_plan_info(ls_plan p, int32_t *tile, int32_t *block, int32_t *n_items, int32_t *grid)
{
    if (!p) return ls_fail(LS_ERR_INVALID_ARG, "plan is NULL");
    if (tile) *tile = p->tile;
    if (block) *block = p->block;
    if (n_items) *n_items = p->n_items;
    if (grid) *grid = p->grid;
    return LS_OK;
}

ls_status ls_plan_launch(ls_plan p, ls_stream stream)
{
    if (!p) return ls_fail(LS_ERR_INVALID_ARG, "plan is NULL");
    return launch_plan(p, (cudaStream_t)stream);
}

ls_status ls_plan_status(ls_plan p, ls_stream stream)
{
    if (!p) return ls_fail(LS_ERR_INVALID_ARG, "plan is NULL");
    unsigned s = 0;
    cudaError_t e = cudaMemcpyAsync(&s, p->counter_d + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(e, "read plan status");
    if (s) return ls_fail(LS_ERR_DEVICE, "a work item named an unknown spline kind");
    return LS_OK;
}

ls_status ls_plan_destroy(ls_plan p)
{
    if (!p) return LS_OK;
    if (p->items_d) ls::dev_free(p->items_d);
    if (p->dev) ls::dev_free(p->dev);
    if (p->mod.lib) cudaLibraryUnload(p->mod.lib);
    delete p;
    return LS_OK;
}

}  // extern "C"
