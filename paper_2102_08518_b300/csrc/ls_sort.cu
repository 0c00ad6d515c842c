// Stable LSD radix sort of (uint32 key, int32 value) pairs, Morton keys of
// points, row permutation, and a random-gather probe for the gather roofline.
//
// One radix pass (digits of RB bits, 8 or 10):
//   1. hist:    each block counts the digits of its tile -> hist[digit * nblk + blk]
//   2. scan:    exclusive prefix sum over hist (digit-major, so the offsets of
//               digit d in block b follow all smaller digits and all earlier
//               blocks of digit d: a stable global order)
//   3. scatter: each warp ranks its keys in input order with __match_any_sync
//               (peers with the same digit); the lowest peer adds the group's
//               size to the warp's digit counter with one shared-memory atomic
//               and broadcasts the old value (atomics of one warp on one address
//               keep program order, so ranks stay stable); warps are combined by
//               a per-digit prefix over warps, keys go to offset + rank.
#include <cstdint>

#include "ls_kernels.h"

namespace lsk {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                       // keys per thread
constexpr int kTile = kThreads * kItems;         // 4096 keys per block

template <int RB>
__global__ void __launch_bounds__(kThreads) hist_kernel(const uint32_t *keys, long long n, int shift,
                                                         uint32_t *hist, int nblk)
{
    constexpr int kBins = 1 << RB;
    __shared__ uint32_t h[kBins];
    for (int b = threadIdx.x; b < kBins; b += kThreads) h[b] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kTile;
    for (int it = 0; it < kItems; ++it) {
        long long i = base + (long long)it * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += kThreads) hist[(size_t)b * nblk + blockIdx.x] = h[b];
}

// exclusive scan of n uint32 in three steps with chunk sums in `part`
constexpr int kScanChunk = 2048;

__global__ void __launch_bounds__(1024) scan_reduce(const uint32_t *in, long long n, uint32_t *part)
{
    __shared__ uint32_t red[1024];
    const long long base = (long long)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int k = threadIdx.x; k < kScanChunk; k += 1024) {
        long long i = base + k;
        if (i < n) s += in[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// exclusive scan of the chunk sums by one block (nparts <= 1024 * 8)
__global__ void __launch_bounds__(1024) scan_parts(uint32_t *part, int nparts)
{
    __shared__ uint32_t s[1024];
    constexpr int per = 8;
    uint32_t v[per];
    uint32_t tot = 0;
    for (int k = 0; k < per; ++k) {
        int i = threadIdx.x * per + k;
        v[k] = i < nparts ? part[i] : 0u;
        tot += v[k];
    }
    s[threadIdx.x] = tot;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - tot;
    for (int k = 0; k < per; ++k) {
        int i = threadIdx.x * per + k;
        if (i < nparts) part[i] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(1024) scan_down(const uint32_t *in, long long n, const uint32_t *part, uint32_t *out)
{
    __shared__ uint32_t s[1024];
    constexpr int per = kScanChunk / 1024;
    const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * per;
    uint32_t v[per];
    uint32_t tot = 0;
    for (int k = 0; k < per; ++k) {
        long long i = base + k;
        v[k] = i < n ? in[i] : 0u;
        tot += v[k];
    }
    s[threadIdx.x] = tot;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = part[blockIdx.x] + s[threadIdx.x] - tot;
    for (int k = 0; k < per; ++k) {
        long long i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

// Ranks every key of the tile (stable), stages the tile in shared memory in
// digit order, then writes each digit's run to its global offset: consecutive
// threads write consecutive addresses.
template <int RB>
__global__ void __launch_bounds__(kThreads) scatter_kernel(const uint32_t *keys, const int32_t *vals, long long n,
                                                            int shift, const uint32_t *offs, int nblk,
                                                            uint32_t *keys_out, int32_t *vals_out)
{
    constexpr int kBins = 1 << RB;
    constexpr int kPer = kBins / kThreads;         // digits per thread in the digit scans
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *whist = sm;                          // [kWarps][kBins]
    uint32_t *bstart = whist + kWarps * kBins;     // [kBins]
    uint32_t *goff = bstart + kBins;               // [kBins]
    uint32_t *tsum = goff + kBins;                 // [kThreads] scan scratch
    uint32_t *skey = tsum + kThreads;              // [kTile]
    int32_t *sval = (int32_t *)(skey + kTile);     // [kTile]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = lane; b < kBins; b += 32) whist[warp * kBins + b] = 0;
    __syncwarp();
    // warp w owns the contiguous keys [base + w*32*kItems, ... + 32*kItems), rounds of 32
    const long long tile0 = (long long)blockIdx.x * kTile;
    const long long base = tile0 + (long long)warp * 32 * kItems;
    uint32_t key[kItems];
    int32_t val[kItems];
    uint32_t rank[kItems];
    const unsigned lt = (1u << lane) - 1u;
    for (int it = 0; it < kItems; ++it) {
        long long i = base + (long long)it * 32 + lane;
        const bool valid = i < n;
        key[it] = valid ? keys[i] : 0xFFFFFFFFu;
        val[it] = valid ? vals[i] : 0;
        const uint32_t d = (key[it] >> shift) & (kBins - 1);
        const unsigned active = __ballot_sync(0xFFFFFFFFu, valid);
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, valid ? d : 0xFFFFFFFFu) & active;
        const int leader = peers ? __ffs(peers) - 1 : 0;
        uint32_t before = 0u;
        if (valid && lane == leader) before = atomicAdd(&whist[warp * kBins + d], (uint32_t)__popc(peers));
        before = __shfl_sync(0xFFFFFFFFu, before, leader);
        rank[it] = valid ? before + __popc(peers & lt) : 0u;
    }
    __syncthreads();
    // per digit: warp prefix inside the block, block total
    uint32_t tot[kPer];
    for (int q = 0; q < kPer; ++q) {
        const int b = threadIdx.x * kPer + q;
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = whist[w * kBins + b];
            whist[w * kBins + b] = run;
            run += c;
        }
        tot[q] = run;
        goff[b] = offs[(size_t)b * nblk + blockIdx.x];
    }
    // exclusive scan of the block totals over digits: per-thread sums, then
    // Hillis-Steele over threads
    uint32_t mine = 0;
    for (int q = 0; q < kPer; ++q) mine += tot[q];
    tsum[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < kThreads; off <<= 1) {
        const uint32_t v = threadIdx.x >= off ? tsum[threadIdx.x - off] : 0u;
        __syncthreads();
        tsum[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = tsum[threadIdx.x] - mine;
    for (int q = 0; q < kPer; ++q) {
        bstart[threadIdx.x * kPer + q] = run;
        run += tot[q];
    }
    __syncthreads();
    for (int it = 0; it < kItems; ++it) {
        long long i = base + (long long)it * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[it] >> shift) & (kBins - 1);
            const uint32_t lp = bstart[d] + whist[warp * kBins + d] + rank[it];
            skey[lp] = key[it];
            sval[lp] = val[it];
        }
    }
    __syncthreads();
    const long long cnt = (n - tile0) < kTile ? (n - tile0) : kTile;
    for (int lp = threadIdx.x; lp < cnt; lp += kThreads) {
        const uint32_t k = skey[lp];
        const uint32_t d = (k >> shift) & (kBins - 1);
        const uint32_t dst = goff[d] + (uint32_t)lp - bstart[d];
        keys_out[dst] = k;
        vals_out[dst] = sval[lp];
    }
}

template <int RB>
constexpr size_t scatter_smem()
{
    return ((size_t)kWarps * (1 << RB) + 2 * (1 << RB) + kThreads + 2 * (size_t)kTile) * 4;
}

__global__ void iota_kernel(int32_t *v, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    // bit b of v -> bit 3b
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t cell10(float x, float o, float inv_cell)
{
    float c = floorf((x - o) * inv_cell);
    c = fminf(fmaxf(c, 0.0f), 1023.0f);
    return (c == c) ? (uint32_t)c : 0u;
}

__global__ void morton_kernel(const float *pts, long long n, float o0, float o1, float o2, float inv_cell,
                              uint32_t *keys, int32_t *vals)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t c0 = cell10(pts[3 * i], o0, inv_cell);
        const uint32_t c1 = cell10(pts[3 * i + 1], o1, inv_cell);
        const uint32_t c2 = cell10(pts[3 * i + 2], o2, inv_cell);
        keys[i] = spread10(c0) | (spread10(c1) << 1) | (spread10(c2) << 2);
        vals[i] = (int32_t)i;
    }
}

__global__ void permute_kernel(const float *src, const int32_t *perm, long long n, int width, int inverse, float *dst)
{
    const long long total = n * width;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / width;
        const int c = (int)(t - i * width);
        const long long p = perm[i];
        if (inverse) dst[p * width + c] = src[t];
        else dst[t] = src[p * width + c];
    }
}

// Random 4-byte gathers from an L2-resident table: each thread issues `loads`
// independent loads at hashed indices (no index traffic) and writes one sum.
__global__ void __launch_bounds__(256) gather_probe_kernel(const float *table, uint32_t mask, int loads, float *out,
                                                           long long nthreads)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nthreads;
         t += (long long)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)t * 2654435761u + 0x9E3779B9u;
        float s = 0.0f;
#pragma unroll 8
        for (int k = 0; k < loads; ++k) {
            h ^= h >> 15;
            h *= 0x2C1B3C6Du;
            h ^= h >> 12;
            s += __ldg(table + (h & mask));
        }
        out[t] = s;
    }
}

// start[b] = first position i of the sorted keys with key[i] >= b, b in [0, nbins + 1].
__global__ void bin_starts_kernel(const uint32_t *key, long long n, uint32_t nbins, uint32_t *start)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t lo = (i == 0) ? 0u : key[i - 1] + 1u;
        const uint32_t hi = (i == n) ? nbins + 1u : key[i];
        for (uint32_t b = lo; b <= hi && b <= nbins + 1u; ++b) start[b] = (uint32_t)i;
    }
}

int nblocks_for(long long n) { return (int)((n + kTile - 1) / kTile); }

}  // namespace

constexpr int kMaxBins = 1024;

size_t sort_scratch_bytes(long long n)
{
    const long long nblk = nblocks_for(n);
    const long long nh = nblk * kMaxBins;
    const long long nparts = (nh + kScanChunk - 1) / kScanChunk;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(n * 4) * 2 + al(nh * 4) * 2 + al(nparts * 4) + 256;
}

cudaError_t radix_sort_pairs(uint32_t *keys, int32_t *vals, long long n, int nbits, void *scratch, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    const int nblk = nblocks_for(n);
    // 10-bit digits when that saves a pass (e.g. 30-bit Morton keys: 3 passes, not 4)
    const int rb = ((nbits + 9) / 10 < (nbits + 7) / 8) ? 10 : 8;
    const long long nh = (long long)nblk * (1 << rb);
    const long long nparts = (nh + kScanChunk - 1) / kScanChunk;
    if (nparts > 8192) return cudaErrorInvalidValue;
    cudaError_t ea = rb == 10 ? cudaFuncSetAttribute(scatter_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)scatter_smem<10>())
                              : cudaFuncSetAttribute(scatter_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)scatter_smem<8>());
    if (ea != cudaSuccess) return ea;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *p = (char *)scratch;
    uint32_t *k2 = (uint32_t *)p;
    p += al(n * 4);
    int32_t *v2 = (int32_t *)p;
    p += al(n * 4);
    uint32_t *hist = (uint32_t *)p;
    p += al(nh * 4);
    uint32_t *offs = (uint32_t *)p;
    p += al(nh * 4);
    uint32_t *part = (uint32_t *)p;
    uint32_t *ks = keys, *kd = k2;
    int32_t *vs = vals, *vd = v2;
    int passes = (nbits + rb - 1) / rb;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = rb * ps;
        if (rb == 10) hist_kernel<10><<<nblk, kThreads, 0, st>>>(ks, n, shift, hist, nblk);
        else hist_kernel<8><<<nblk, kThreads, 0, st>>>(ks, n, shift, hist, nblk);
        scan_reduce<<<(unsigned)nparts, 1024, 0, st>>>(hist, nh, part);
        scan_parts<<<1, 1024, 0, st>>>(part, (int)nparts);
        scan_down<<<(unsigned)nparts, 1024, 0, st>>>(hist, nh, part, offs);
        if (rb == 10)
            scatter_kernel<10><<<nblk, kThreads, scatter_smem<10>(), st>>>(ks, vs, n, shift, offs, nblk, kd, vd);
        else
            scatter_kernel<8><<<nblk, kThreads, scatter_smem<8>(), st>>>(ks, vs, n, shift, offs, nblk, kd, vd);
        uint32_t *tk = ks; ks = kd; kd = tk;
        int32_t *tv = vs; vs = vd; vd = tv;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ks != keys) {
        e = cudaMemcpyAsync(keys, ks, n * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(vals, vs, n * 4, cudaMemcpyDeviceToDevice, st);
    }
    return e;
}

cudaError_t morton_keys(const float *pts, long long n, const float *origin, float cell, uint32_t *keys, int32_t *vals,
                        cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    morton_kernel<<<(unsigned)blocks, 256, 0, st>>>(pts, n, origin[0], origin[1], origin[2], 1.0f / cell, keys, vals);
    return cudaGetLastError();
}

cudaError_t iota(int32_t *v, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    iota_kernel<<<(unsigned)blocks, 256, 0, st>>>(v, n);
    return cudaGetLastError();
}

cudaError_t permute_rows(const float *src, const int32_t *perm, long long n, int width, int inverse, float *dst,
                         cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n * width + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    permute_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, perm, n, width, inverse, dst);
    return cudaGetLastError();
}

cudaError_t bin_starts(const uint32_t *key, long long n, uint32_t nbins, uint32_t *start, cudaStream_t st)
{
    long long blocks = (n + 1 + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    bin_starts_kernel<<<(unsigned)blocks, 256, 0, st>>>(key, n, nbins, start);
    return cudaGetLastError();
}

cudaError_t gather_probe(const float *table, long long table_elems, int loads, float *out, long long nthreads,
                         int blocks, cudaStream_t st)
{
    uint32_t mask = 1;
    while ((long long)mask * 2 <= table_elems) mask *= 2;
    mask -= 1;
    gather_probe_kernel<<<blocks, 256, 0, st>>>(table, mask, loads, out, nthreads);
    return cudaGetLastError();
}

}  // namespace lsk
