// Top-k selection over large score arrays by radix select.
//
// The k best of `count` floats (score desc, index asc; entries whose keep
// byte is 0 skipped, NaN never selected) are found without sorting the
// array: order-preserving 32-bit keys are histogrammed in three passes
// (12 + 12 + 8 bits), each pass narrowing to the bin that holds the k-th key,
// which gives the k-th key exactly.  Every key above it is then selected
// (appended in any order), and the entries equal to it are taken in index
// order until k entries are selected (per-block counts, an exclusive scan
// and an order-preserving block compaction), so the selected set is exactly
// the k best by (score desc, index asc).  Optionally the selection is sorted
// by the same order (k <= 4096).  Everything runs on the device, queued on
// one stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "epi_host.h"
#include "epi_internal.cuh"

namespace epi {
namespace topk {

constexpr int kHistBins = 4096;
constexpr int kTieBlocks = 1024;
constexpr int kThreads = 256;

struct State {
    uint32_t prefix;       // key bits fixed so far
    int32_t all;           // fewer kept entries than k: select them all
    uint64_t need;         // entries still to select at or below the prefix
    uint64_t gt;           // entries above the final key
    uint64_t eq;           // entries equal to the final key
};

// order-preserving unsigned key of a float; NaN maps to 0 and is never selected
__device__ __forceinline__ uint32_t fkey(float v)
{
    if (v != v) return 0u;
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ bool live(const uint8_t *keep, uint64_t i, uint32_t k)
{
    return k != 0u && (keep == nullptr || keep[i] != 0);
}

// pass p: histogram of the key bits below the prefix of the previous passes
__global__ void __launch_bounds__(kThreads) hist_kernel(const float *__restrict__ v, const uint8_t *__restrict__ keep,
                                                        uint64_t count, const State *__restrict__ st, int pass,
                                                        unsigned long long *__restrict__ hist)
{
    __shared__ uint32_t h[kHistBins];
    const int shift = pass == 0 ? 20 : (pass == 1 ? 8 : 0);
    const int bins = pass == 2 ? 256 : kHistBins;
    const int pshift = pass == 0 ? 32 : (pass == 1 ? 20 : 8);
    const uint32_t prefix = st->prefix;
    for (int i = threadIdx.x; i < bins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k = fkey(v[i]);
        if (!live(keep, i, k)) continue;
        if (pshift < 32 && (k >> pshift) != prefix) continue;
        atomicAdd(&h[(k >> shift) & (uint32_t)(bins - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// the bin holding the need-th key from the top: one block of 1024 threads,
// each owning 4 consecutive bins (from the top), a block-wide suffix sum
__global__ void __launch_bounds__(1024) scan_kernel(unsigned long long *__restrict__ hist, State *__restrict__ st,
                                                    int pass)
{
    __shared__ unsigned long long part[1024];
    __shared__ unsigned long long hb[kHistBins];
    const int bins = pass == 2 ? 256 : kHistBins;
    const int per = bins / 1024 > 0 ? bins / 1024 : 1;
    const int t = threadIdx.x;
    for (int i = t; i < bins; i += blockDim.x) hb[i] = hist[i];
    __syncthreads();
    // thread t owns bins top-down: [bins - per (t + 1), bins - per t)
    unsigned long long own = 0;
    const int hi = bins - per * t, lo = hi - per;
    if (lo >= 0)
        for (int b = lo; b < hi; b++) own += hb[b];
    part[t] = own;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned long long add = t >= off ? part[t - off] : 0ull;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    // part[t] = keys in bins at or above lo (owned by threads 0..t)
    const unsigned long long need = st->need;
    const unsigned long long before = t > 0 ? part[t - 1] : 0ull;
    if (pass == 0 && t == 0 && part[1023] < need) {
        st->all = 1;
    }
    __syncthreads();
    if (st->all) {
        if (t == 0) {
            for (int b = 0; b < bins; b++) hist[b] = 0;
        }
        return;
    }
    if (lo >= 0 && before < need && part[t] >= need) {
        unsigned long long acc = before;
        int b = hi - 1;
        for (; b > lo; b--) {
            if (acc + hb[b] >= need) break;
            acc += hb[b];
        }
        const int width = pass == 2 ? 8 : 12;
        st->prefix = (st->prefix << width) | (uint32_t)b;
        st->gt += acc;
        st->need = need - acc;
        st->eq = hb[b];
    }
    __syncthreads();
    for (int i = t; i < bins; i += blockDim.x) hist[i] = 0;   // ready for the next pass
}

// every key above the final one (any order); every kept key when `all`
__global__ void __launch_bounds__(kThreads) select_gt_kernel(const float *__restrict__ v,
                                                             const uint8_t *__restrict__ keep, uint64_t count,
                                                             const State *__restrict__ st, uint64_t *__restrict__ out,
                                                             unsigned long long *__restrict__ n_out)
{
    const uint32_t thr = st->prefix;
    const bool all = st->all != 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k = fkey(v[i]);
        if (!live(keep, i, k)) continue;
        if (all || k > thr) out[atomicAdd(n_out, 1ull)] = i;
    }
}

__device__ __forceinline__ void block_range(uint64_t count, uint64_t &b, uint64_t &e)
{
    const uint64_t per = (count + gridDim.x - 1) / gridDim.x;
    b = (uint64_t)blockIdx.x * per;
    e = b + per < count ? b + per : count;
    if (b > count) b = count;
}

// per-block counts of the keys equal to the final one
__global__ void __launch_bounds__(kThreads) tie_count_kernel(const float *__restrict__ v,
                                                             const uint8_t *__restrict__ keep, uint64_t count,
                                                             const State *__restrict__ st, uint32_t *__restrict__ cnt)
{
    __shared__ uint32_t c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    if (!st->all) {
        const uint32_t thr = st->prefix;
        uint64_t b, e;
        block_range(count, b, e);
        uint32_t mine = 0;
        for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            const uint32_t k = fkey(v[i]);
            if (live(keep, i, k) && k == thr) mine++;
        }
        atomicAdd(&c, mine);
    }
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// exclusive scan of the per-block tie counts (one block)
__global__ void __launch_bounds__(kTieBlocks) tie_scan_kernel(const uint32_t *__restrict__ cnt, int nb,
                                                              unsigned long long *__restrict__ off)
{
    __shared__ unsigned long long s[kTieBlocks];
    const int t = threadIdx.x;
    s[t] = t < nb ? cnt[t] : 0;
    __syncthreads();
    for (int o = 1; o < kTieBlocks; o <<= 1) {
        const unsigned long long add = t >= o ? s[t - o] : 0ull;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    if (t < nb) off[t] = s[t] - cnt[t];
}

// the ties in index order, as many as still needed, after the gt entries
__global__ void __launch_bounds__(kThreads) tie_write_kernel(const float *__restrict__ v,
                                                             const uint8_t *__restrict__ keep, uint64_t count,
                                                             const State *__restrict__ st,
                                                             const unsigned long long *__restrict__ off,
                                                             uint64_t *__restrict__ out)
{
    if (st->all) return;
    const uint32_t thr = st->prefix;
    const uint64_t need = st->need, base_out = st->gt;
    uint64_t rank = off[blockIdx.x];
    if (rank >= need) return;
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ uint64_t chunk_base;
    uint64_t b, e;
    block_range(count, b, e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t i0 = b; i0 < e; i0 += blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        bool tie = false;
        if (i < e) {
            const uint32_t k = fkey(v[i]);
            tie = live(keep, i, k) && k == thr;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, tie);
        if (lane == 0) wsum[warp] = __popc(m);
        if (threadIdx.x == 0) chunk_base = rank;
        __syncthreads();
        uint64_t before = chunk_base;
        for (int w = 0; w < warp; w++) before += wsum[w];
        before += __popc(m & ((1u << lane) - 1u));
        if (tie && before < need) out[base_out + before] = i;
        uint32_t total = 0;
        for (int w = 0; w < kThreads / 32; w++) total += wsum[w];
        __syncthreads();
        rank += total;
        if (rank >= need) break;
    }
}

__global__ void finish_kernel(const State *__restrict__ st, uint64_t k, const unsigned long long *__restrict__ n_gt,
                              int32_t *__restrict__ n_out)
{
    const uint64_t n = st->all ? (uint64_t)*n_gt : k;
    *n_out = (int32_t)n;
}

// scores of the selected entries, for the final sort
__global__ void gather_kernel(const float *__restrict__ v, const uint64_t *__restrict__ idx,
                              const int32_t *__restrict__ n, float *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < *n; i += gridDim.x * blockDim.x) out[i] = v[idx[i]];
}

struct Layout {
    size_t st, hist, cnt, off, ngt, sel_s, sel_i, total;
};

Layout layout(int64_t k)
{
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = (o + 255) & ~(size_t)255;
        const size_t at = o;
        o += bytes;
        return at;
    };
    L.st = take(sizeof(State));
    L.hist = take(sizeof(unsigned long long) * kHistBins);
    L.cnt = take(sizeof(uint32_t) * kTieBlocks);
    L.off = take(sizeof(unsigned long long) * kTieBlocks);
    L.ngt = take(sizeof(unsigned long long));
    L.sel_s = take(sizeof(float) * (size_t)k);
    L.sel_i = take(sizeof(uint64_t) * (size_t)k);
    L.total = o + 256;
    return L;
}

}  // namespace topk

size_t topk_scratch_bytes(int64_t k) { return topk::layout(k).total; }

cudaError_t launch_topk(const float *scores, const uint8_t *keep, int64_t count, int64_t k, void *scratch, bool sorted,
                        float *out_s, uint64_t *out_i, int32_t *out_n, int num_sms, cudaStream_t st)
{
    using namespace topk;
    const Layout L = layout(k);
    char *base = static_cast<char *>(scratch);
    State *S = reinterpret_cast<State *>(base + L.st);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(base + L.hist);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(base + L.cnt);
    unsigned long long *off = reinterpret_cast<unsigned long long *>(base + L.off);
    unsigned long long *ngt = reinterpret_cast<unsigned long long *>(base + L.ngt);
    float *sel_s = reinterpret_cast<float *>(base + L.sel_s);
    uint64_t *sel_i = sorted ? reinterpret_cast<uint64_t *>(base + L.sel_i) : out_i;
    State init{};
    init.need = (uint64_t)k;
    cudaError_t e = cudaMemcpyAsync(S, &init, sizeof(State), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kHistBins, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ngt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const uint64_t c = count > 0 ? (uint64_t)count : 0;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((c + kThreads - 1) / kThreads, (uint64_t)num_sms * 8));
    for (int pass = 0; pass < 3; pass++) {
        hist_kernel<<<grid, kThreads, 0, st>>>(scores, keep, c, S, pass, hist);
        scan_kernel<<<1, 1024, 0, st>>>(hist, S, pass);
    }
    select_gt_kernel<<<grid, kThreads, 0, st>>>(scores, keep, c, S, sel_i, ngt);
    tie_count_kernel<<<kTieBlocks, kThreads, 0, st>>>(scores, keep, c, S, cnt);
    tie_scan_kernel<<<1, kTieBlocks, 0, st>>>(cnt, kTieBlocks, off);
    tie_write_kernel<<<kTieBlocks, kThreads, 0, st>>>(scores, keep, c, S, off, sel_i);
    finish_kernel<<<1, 1, 0, st>>>(S, (uint64_t)k, ngt, out_n);
    e = cudaGetLastError();
    if (e != cudaSuccess || !sorted) return e;
    // sort the selection: one list of at most k <= 4096 (score, index) pairs
    gather_kernel<<<(int)((k + 255) / 256), 256, 0, st>>>(scores, sel_i, out_n, sel_s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_merge(sel_s, sel_i, out_n, 1, (int)k, (int)k, out_s, out_i, out_n, st, -INFINITY);
}

}  // namespace epi
