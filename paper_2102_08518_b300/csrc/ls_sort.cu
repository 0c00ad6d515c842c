// Stable LSD radix sort of (uint32 key, int32 value) pairs, Morton keys of
// points, row permutation, and a random-gather probe for the gather roofline.
//
// One radix pass (digits of RB = 8 bits) over G blocks, each owning a
// contiguous chunk of the input (G = a few blocks per SM, so the per-block
// digit table stays small):
//   1. hist:    each block counts the digits of its chunk -> hist[digit * G + blk]
//   2. scan:    exclusive prefix sum over hist (digit-major, so the offsets of
//               digit d in block b follow all smaller digits and all earlier
//               blocks of digit d: a stable global order)
//   3. scatter: each block walks its chunk in tiles, in order, keeping a running
//               output offset per digit.  Inside a tile each warp ranks its keys
//               in input order with __match_any_sync (peers with the same
//               digit); the lowest peer adds the group's size to the warp's
//               digit counter with one shared-memory atomic (atomics of one
//               warp on one address keep program order, so ranks stay stable;
//               all rounds' atomics are issued before their results are
//               used); warps are combined by a per-digit prefix over warps, the
//               tile is staged in shared memory in digit order and each digit's
//               run is written to its global offset.
#include <atomic>
#include <cstdint>

#include "ls_kernels.h"

namespace lsk {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                       // keys per thread and tile
constexpr int kTile = kThreads * kItems;         // 4096 keys per tile
constexpr int kMaxChunks = 148 * 8;              // most blocks (chunks of the input) in a pass

template <int RB>
__global__ void __launch_bounds__(kThreads) hist_kernel(const uint32_t *keys, long long n, int shift,
                                                         long long chunk, uint32_t *hist, int nblk)
{
    constexpr int kBins = 1 << RB;
    __shared__ uint32_t h[kBins];
    for (int b = threadIdx.x; b < kBins; b += kThreads) h[b] = 0;
    __syncthreads();
    const long long c0 = (long long)blockIdx.x * chunk;
    const long long c1 = (c0 + chunk < n) ? c0 + chunk : n;
    long long done = c0;
    if (((uintptr_t)(keys + c0) & 15) == 0) {
        // 16-byte loads, four in flight per thread
        const long long nv = (c1 - c0) >> 2;
        const uint4 *k4 = (const uint4 *)(keys + c0);
        for (long long v = threadIdx.x; v < nv; v += 4LL * kThreads) {
            uint4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long w = v + (long long)u * kThreads;
                q[u] = w < nv ? __ldg(k4 + w) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (v + (long long)u * kThreads >= nv) continue;
                atomicAdd(&h[(q[u].x >> shift) & (kBins - 1)], 1u);
                atomicAdd(&h[(q[u].y >> shift) & (kBins - 1)], 1u);
                atomicAdd(&h[(q[u].z >> shift) & (kBins - 1)], 1u);
                atomicAdd(&h[(q[u].w >> shift) & (kBins - 1)], 1u);
            }
        }
        done = c0 + (nv << 2);
    }
    for (long long i = done + threadIdx.x; i < c1; i += kThreads)
        atomicAdd(&h[(__ldg(keys + i) >> shift) & (kBins - 1)], 1u);
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

// Ranks the keys of each tile of the block's chunk (stable), stages the tile
// in shared memory in digit order, then writes each digit's run at the block's
// running offset of that digit: consecutive threads write consecutive
// addresses.
template <int RB>
__global__ void __launch_bounds__(kThreads, 2) scatter_kernel(const uint32_t *keys, const int32_t *vals, long long n,
                                                            int shift, long long chunk, const uint32_t *offs,
                                                            int nblk, uint32_t *keys_out, int32_t *vals_out)
{
    constexpr int kBins = 1 << RB;
    constexpr int kPer = kBins / kThreads;         // digits per thread in the digit scans
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *whist = sm;                          // [kWarps][kBins]
    uint32_t *bstart = whist + kWarps * kBins;     // [kBins] tile offsets of the digits
    uint32_t *run = bstart + kBins;                // [kBins] running global offsets of the digits
    uint32_t *tsum = run + kBins;                  // [kThreads] scan scratch
    uint32_t *skey = tsum + kThreads;              // [kTile]
    int32_t *sval = (int32_t *)(skey + kTile);     // [kTile]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int whole = 0;
    for (int q = 0; q < kPer; ++q) {
        const int b = threadIdx.x * kPer + q;
        run[b] = offs[(size_t)b * nblk + blockIdx.x];
        // the digit's count over all blocks (offsets are digit-major)
        const uint32_t end = b + 1 < kBins ? offs[(size_t)(b + 1) * nblk] : (uint32_t)n;
        whole |= (long long)(end - offs[(size_t)b * nblk]) == n;
    }
    const long long c0 = (long long)blockIdx.x * chunk;
    const long long c1 = (c0 + chunk < n) ? c0 + chunk : n;
    // every key has the same digit in this pass (keys narrower than the sort's
    // bits, e.g. Morton keys of a 256-cell box have a zero top digit): the
    // stable order is the input order, so the chunk is copied through
    if (__syncthreads_or(whole)) {
        // 16-byte copies, four in flight per thread, when all four arrays
        // allow them at this chunk; scalar copies for the rest
        long long done = c0;
        const uintptr_t al = (uintptr_t)(keys + c0) | (uintptr_t)(vals + c0) | (uintptr_t)(keys_out + c0) |
                             (uintptr_t)(vals_out + c0);
        if ((al & 15) == 0) {
            const long long nv = (c1 - c0) >> 2;
            const uint4 *ks = (const uint4 *)(keys + c0), *vs = (const uint4 *)(vals + c0);
            uint4 *kd = (uint4 *)(keys_out + c0), *vd = (uint4 *)(vals_out + c0);
            for (long long v = threadIdx.x; v < nv; v += 4LL * kThreads) {
                uint4 a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long w = v + (long long)u * kThreads;
                    if (w < nv) {
                        a[u] = __ldg(ks + w);
                        b[u] = __ldg(vs + w);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long w = v + (long long)u * kThreads;
                    if (w < nv) {
                        kd[w] = a[u];
                        vd[w] = b[u];
                    }
                }
            }
            done = c0 + (nv << 2);
        }
        for (long long i = done + threadIdx.x; i < c1; i += kThreads) {
            keys_out[i] = __ldg(keys + i);
            vals_out[i] = __ldg(vals + i);
        }
        return;
    }
    uint32_t nkey[kItems];
    int32_t nval[kItems];
    {
        const long long b0 = c0 + (long long)warp * 32 * kItems;
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const long long i = b0 + (long long)it * 32 + lane;
            const bool valid = i < c1;
            nkey[it] = valid ? __ldg(keys + i) : 0xFFFFFFFFu;
            nval[it] = valid ? __ldg(vals + i) : 0;
        }
    }
    for (long long tile0 = c0; tile0 < c1; tile0 += kTile) {
        for (int b = lane; b < kBins; b += 32) whist[warp * kBins + b] = 0;
        __syncwarp();
        // warp w owns the contiguous keys [tile0 + w*32*kItems, ... + 32*kItems), rounds of 32
        const long long base = tile0 + (long long)warp * 32 * kItems;
        uint32_t key[kItems], rank[kItems], before[kItems], peers[kItems];
        int32_t val[kItems];
        int leader[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            key[it] = nkey[it];
            val[it] = nval[it];
        }
        // the next tile's keys and values are in flight while this one is ranked
        {
            const long long nb = base + kTile;
#pragma unroll
            for (int it = 0; it < kItems; ++it) {
                const long long i = nb + (long long)it * 32 + lane;
                const bool valid = i < c1;
                nkey[it] = valid ? __ldg(keys + i) : 0xFFFFFFFFu;
                nval[it] = valid ? __ldg(vals + i) : 0;
            }
        }
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const long long i = base + (long long)it * 32 + lane;
            const bool valid = i < c1;
            const uint32_t d = (key[it] >> shift) & (kBins - 1);
            const unsigned active = __ballot_sync(0xFFFFFFFFu, valid);
            peers[it] = __match_any_sync(0xFFFFFFFFu, valid ? d : 0xFFFFFFFFu) & active;
            leader[it] = peers[it] ? __ffs(peers[it]) - 1 : 0;
            before[it] = 0u;
            if (valid && lane == leader[it]) before[it] = atomicAdd(&whist[warp * kBins + d], (uint32_t)__popc(peers[it]));
        }
#pragma unroll
        for (int it = 0; it < kItems; ++it)
            rank[it] = __shfl_sync(0xFFFFFFFFu, before[it], leader[it]) + __popc(peers[it] & lt);
        __syncthreads();
        // per digit: warp prefix inside the tile, tile total
        uint32_t tot[kPer];
        for (int q = 0; q < kPer; ++q) {
            const int b = threadIdx.x * kPer + q;
            uint32_t acc = 0;
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = whist[w * kBins + b];
                whist[w * kBins + b] = acc;
                acc += c;
            }
            tot[q] = acc;
        }
        // exclusive scan of the tile totals over digits: per-thread sums, a
        // shuffle scan inside each warp, then the warps' totals
        uint32_t mine = 0;
        for (int q = 0; q < kPer; ++q) mine += tot[q];
        uint32_t inc = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, inc, off);
            if (lane >= off) inc += v;
        }
        if (lane == 31) tsum[warp] = inc;
        __syncthreads();
        uint32_t wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += tsum[w];
        uint32_t acc = wbase + inc - mine;
        for (int q = 0; q < kPer; ++q) {
            bstart[threadIdx.x * kPer + q] = acc;
            acc += tot[q];
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const long long i = base + (long long)it * 32 + lane;
            if (i < c1) {
                const uint32_t d = (key[it] >> shift) & (kBins - 1);
                const uint32_t lp = bstart[d] + whist[warp * kBins + d] + rank[it];
                skey[lp] = key[it];
                sval[lp] = val[it];
            }
        }
        __syncthreads();
        const int cnt = (int)((c1 - tile0) < kTile ? (c1 - tile0) : kTile);
        for (int lp = threadIdx.x; lp < cnt; lp += kThreads) {
            const uint32_t k = skey[lp];
            const uint32_t d = (k >> shift) & (kBins - 1);
            const uint32_t dst = run[d] + (uint32_t)lp - bstart[d];
            keys_out[dst] = k;
            vals_out[dst] = sval[lp];
        }
        __syncthreads();
        for (int q = 0; q < kPer; ++q) run[threadIdx.x * kPer + q] += tot[q];
        // the next tile's first barrier orders these updates before their use
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

// Rows of W floats (W = 1..4), one row per thread and one thread per row: the
// random side (the permuted row) is fetched as the row's W consecutive floats
// by one thread (on B300, 2^26 rows of 3 floats in a random permutation:
// 1.50 ms against 1.70 for one element per thread; a device copy of the same
// bytes takes 0.25 ms, the rest is the DRAM's random access).
template <int W>
__global__ void permute_rows_kernel(const float *__restrict__ src, const int32_t *__restrict__ perm, long long n,
                                    int inverse, float *__restrict__ dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long p = perm[i];
    const long long s = inverse ? i : p, d = inverse ? p : i;
    float v[W];
#pragma unroll
    for (int c = 0; c < W; ++c) v[c] = src[s * W + c];
#pragma unroll
    for (int c = 0; c < W; ++c) dst[d * W + c] = v[c];
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

// blocks (chunks) of one pass and the keys per chunk, a whole number of tiles:
// at least two tiles per chunk (a small digit table) and at most cap chunks
void chunking(long long n, int cap, int &nblk, long long &chunk)
{
    const long long tiles = (n + kTile - 1) / kTile;
    const long long want = tiles / 2 > 1 ? tiles / 2 : 1;
    nblk = (int)(want < cap ? want : cap);
    chunk = (tiles + nblk - 1) / nblk * kTile;
    nblk = (int)((n + chunk - 1) / chunk);
    if (nblk < 1) nblk = 1;
}

}  // namespace

constexpr int kMaxBins = 256;             // 8-bit digits

size_t sort_scratch_bytes(long long n)
{
    int nblk;
    long long chunk;
    chunking(n, kMaxChunks, nblk, chunk);
    const long long nh = (long long)nblk * kMaxBins;
    const long long nparts = (nh + kScanChunk - 1) / kScanChunk;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(n * 4) * 2 + al(nh * 4) * 2 + al(nparts * 4) + 256;
}

cudaError_t radix_sort_pairs(uint32_t *keys, int32_t *vals, long long n, int nbits, void *scratch, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    // 8-bit digits: on B300 four 8-bit passes over 30-bit keys beat three 10-bit
    // ones (3.24 vs 4.14 ms for 2^26 pairs): a 2048-key tile spreads over 256
    // instead of 1024 digits, so the output runs are 4x longer and the per-warp
    // digit counters 4x smaller
    const int rb = 8;
    // one wave: as many chunks as blocks of the scatter kernel fit on the GPU
    // (cached per device; any thread may fill an entry, all write the same value)
    static std::atomic<int> waves[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        dev = 0;
    }
    int wave = waves[dev].load(std::memory_order_relaxed);
    if (wave == 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaFuncSetAttribute(scatter_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem<8>()) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, scatter_kernel<8>, kThreads, scatter_smem<8>()) != cudaSuccess ||
            per < 1) {
            cudaGetLastError();
            sms = 148;
            per = 2;
        }
        wave = sms * per < kMaxChunks ? sms * per : kMaxChunks;
        waves[dev].store(wave, std::memory_order_relaxed);
    }
    int nblk;
    long long chunk;
    chunking(n, wave, nblk, chunk);
    const long long nh = (long long)nblk * (1 << rb);
    const long long nparts = (nh + kScanChunk - 1) / kScanChunk;
    if (nparts > 8192) return cudaErrorInvalidValue;
    cudaError_t ea = cudaFuncSetAttribute(scatter_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
        hist_kernel<8><<<nblk, kThreads, 0, st>>>(ks, n, shift, chunk, hist, nblk);
        scan_reduce<<<(unsigned)nparts, 1024, 0, st>>>(hist, nh, part);
        scan_parts<<<1, 1024, 0, st>>>(part, (int)nparts);
        scan_down<<<(unsigned)nparts, 1024, 0, st>>>(hist, nh, part, offs);
        scatter_kernel<8><<<nblk, kThreads, scatter_smem<8>(), st>>>(ks, vs, n, shift, chunk, offs, nblk, kd, vd);
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
    if (width >= 1 && width <= 4 && n <= (1LL << 31) * 256 - 256) {
        const unsigned blocks = (unsigned)((n + 255) / 256);
        switch (width) {
        case 1: permute_rows_kernel<1><<<blocks, 256, 0, st>>>(src, perm, n, inverse, dst); break;
        case 2: permute_rows_kernel<2><<<blocks, 256, 0, st>>>(src, perm, n, inverse, dst); break;
        case 3: permute_rows_kernel<3><<<blocks, 256, 0, st>>>(src, perm, n, inverse, dst); break;
        default: permute_rows_kernel<4><<<blocks, 256, 0, st>>>(src, perm, n, inverse, dst); break;
        }
        return cudaGetLastError();
    }
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
