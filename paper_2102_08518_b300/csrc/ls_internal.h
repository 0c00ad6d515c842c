// Internal structures of the lattice spline library (not part of the ABI).
#pragma once

#include <array>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lattice_spline.h"

namespace ls {

using I3 = std::array<int, 3>;

// One reference sub-region, copied out of the descriptor.
struct RefRegion {
    std::vector<I3> sites;            // lattice offsets s_j (unused axes 0)
    std::vector<I3> mono;             // monomial exponents (unused axes 0)
    std::vector<double> coef;         // sites.size() * mono.size()
    double center[3] = {0, 0, 0};
    int degree = 0;
};

struct Axis {
    std::vector<int> sites;
    int degree = 0;
    std::vector<double> coef;         // sites.size() * (degree + 1)
    double center = 0;
};

struct Table {
    std::string name;
    int dim = 3, roe = 0, fold = 0, scale = 1;
    double L[9] = {0};
    std::vector<I3> cosets;
    std::vector<std::array<double, 4>> planes;   // p (dim) then d at [3]
    int bsp_mod = 1;
    std::vector<int> sigma;
    std::vector<RefRegion> ref;
    std::vector<Axis> sep;                       // empty unless separable
};

// Counts the generator reports.
struct GenInfo {
    int n_sites = 0;        // union stencil
    int reach = 0;          // max |component| of any site offset (bounds fast path)
    int fma_value = 0;
    int fma_grad = 0;
    int fma_hess = 0;
    int n_reverse = 0;      // offsets between a coefficient and the ROE sites that can reach it
    int halo = 0;           // halo of the binning grid (storage units)
    double wmax = 1.0;      // bound on |w_j(u)| over the region of evaluation
    int eval_smem = 0;      // dynamic shared memory of the value kernel (warp-specialized, staged)
    int stage_edge = 0;     // staged value kernel: tile edge in grid indices (0: not staged)
    int tmem_cols = 0;      // tensor-core value kernel: tensor memory columns per block (0: FMA path)
    int adj_tile_smem = 0;  // tiled adjoint kernels: dynamic shared memory (FP32 / fixed-point tile)
    int adj_tile_fixed_smem = 0;
};

struct Generated {
    std::string source;
    GenInfo info;
};

// Code generation (ls_codegen.cpp).
Generated generate(const Table &t, ls_dtype coef_dtype, const ls_variant &var);
// 128-point slots per block of the tensor-core value kernel (its block is 128 x that).
int tensor_slots(const Table &t, const ls_variant &var, ls_dtype coef_dtype);
// One persistent kernel ls_batch_eval over the point functions of several splines.
Generated generate_batch(const std::vector<const Table *> &tables, const std::vector<ls_dtype> &dts,
                         const std::vector<int> &bricks, const ls_variant &var);

// Kernel handles of one compiled module.
struct Module {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t eval = nullptr, eval_grad = nullptr, adj_atomic = nullptr, adj_warpagg = nullptr;
    cudaKernel_t adj_fixed = nullptr, eval_hess = nullptr, adj_tile = nullptr, adj_tile_fixed = nullptr;
    cudaKernel_t roe_key = nullptr, adj_gather = nullptr, batch_eval = nullptr;
    int regs_eval = 0;
    int blocks_per_sm_eval = 0, blocks_per_sm_grad = 0, blocks_per_sm_adj = 0, blocks_per_sm_warpagg = 0;
    int blocks_per_sm_fixed = 0, blocks_per_sm_hess = 0, blocks_per_sm_tile = 0, blocks_per_sm_tile_fixed = 0;
    int blocks_per_sm_gather = 0;
};

// NVRTC compile + disk cache + load (ls_jit.cpp).
ls_status compile_and_load(const std::string &source, const std::string &tag, Module &m,
                           std::string &err);
ls_status get_cubin(const std::string &source, const std::string &tag, std::vector<char> &cubin,
                    std::string &err);

}  // namespace ls

// Opaque ABI objects.
struct ls_spline_s {
    ls::Table table;
    ls_dtype dtype = LS_F32;
    ls_variant var{};
    ls::Generated gen;
    ls::Module mod;
    int device = 0;
    int num_sms = 0;
    unsigned *status = nullptr;       // device word: bounded waits that gave up (warp-specialized kernel)
};

struct ls_volume_s {
    ls_spline_s *spline = nullptr;
    int64_t ext[3] = {1, 1, 1};
    int64_t coset_elems = 0;          // prod(ext)
    int64_t total_elems = 0;          // n_cosets * prod(ext)
    int layout = LS_LAYOUT_COSET_MAJOR;
    void *coef = nullptr;
    bool owned = false;
    // staging for ls_eval_host(_multi): buffers and two streams, made on first use
    void *stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t hs[2] = {nullptr, nullptr};
    cudaEvent_t hev[3] = {nullptr, nullptr, nullptr};
    // texture copy for ls_eval_linear_fetch, made by ls_volume_texture_sync
    cudaArray_t tex_array = nullptr;
    cudaTextureObject_t tex = 0;
    bool tex_ready = false;
    // TMA tensor map (device copy, 128 bytes) for the staged value kernel, made
    // on first use for tile edge tmap_edge
    void *tmap = nullptr;
    int tmap_edge = 0;
};

// Address of coefficient (coset j, per-coset linear index q) is
// j * vol_cstride(v) + q * vol_cunit(v) in the linear layouts; the bricked
// layout's kernels take C = vol_cunit(v) and compute the brick address.
// The shifted bricked copies take the elements per copy in place of the coset stride.
inline int vol_cstride(const ls_volume_s *v)
{
    if (v->layout == LS_LAYOUT_BRICKED_SHIFTED) return (int)(v->total_elems / 4);
    if (v->layout == LS_LAYOUT_BRICKED_SHIFTED_XYZ) return (int)(v->total_elems / 8);
    return v->layout == LS_LAYOUT_COSET_MAJOR ? (int)v->coset_elems : 1;
}
inline int vol_cunit(const ls_volume_s *v)
{
    return v->layout == LS_LAYOUT_COSET_MAJOR ? 1 : (int)v->spline->table.cosets.size();
}

// Device allocations of the library (ls_api.cpp).  One place for the
// host-side allocation-failure injection of the tests (ls_debug_fail_alloc)
// and the count of live allocations (ls_debug_live_allocs).
namespace ls {
cudaError_t dev_malloc_raw(void **p, size_t bytes);
cudaError_t dev_malloc_async_raw(void **p, size_t bytes, cudaStream_t st);
cudaError_t dev_free(void *p);
cudaError_t dev_free_async(void *p, cudaStream_t st);
template <class T> cudaError_t dev_malloc(T **p, size_t bytes) { return dev_malloc_raw((void **)p, bytes); }
template <class T> cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st)
{
    return dev_malloc_async_raw((void **)p, bytes, st);
}
}  // namespace ls

// Thread-local error message helpers (ls_api.cpp).
ls_status ls_fail(ls_status s, const std::string &msg);
