// Fused tensor-core inference of the proposer network (tcgen05, sm_103a).
//
// y = W3 . relu(W2 . relu(W1 . x' + b1) + b2) + b3 for 128 rows per step,
// x' = (x - shift) * scale, with BF16 operands and FP32 accumulation in
// tensor memory, and the hidden activations rounded to BF16 between layers
// (the same storage points as the training kernels).  One persistent CTA per
// SM keeps both weight matrices in shared memory for the whole launch:
//   W2   [256 out][256 in]  BF16, K-major, 4 K blocks of 64     128 KiB
//   H1   [128 rows][256]    BF16, 4 K blocks                     64 KiB
//   W1   [256 out][32 in]   BF16, inputs zero-padded to 32       16 KiB
//   X'   2 x [128 rows][32] BF16 (double-buffered input tiles)   16 KiB
// W2 and H1 in the 128-byte swizzle (8-row atoms of 1024 bytes), W1 and X'
// in the 64-byte swizzle (8-row atoms of 512 bytes).  Tensor memory: layer 1
// in columns [0, 256), layer 2 in [256, 512).  Warp roles, pipelined across
// the CTA's 128-row tiles:
//   group A (warps 0-7): load the next tile's input rows straight into
//      registers (thread: one row, 16 inputs), normalise, round to BF16 and
//      write X' while layer 2 of the current tile runs; after layer 1, read
//      lane quadrant w % 4, column half w / 4, add b1, ReLU, round to BF16
//      and write H1;
//   warp 16, one lane: layer 1 (M128 N256 K32: 2 MMAs of K16) once X' is
//      staged (queued behind the previous layer 2), layer 2 (M128 N256 K256:
//      16 MMAs) once H1 is written and the previous tile's layer-2 columns
//      are read;
//   group B (warps 8-15): after layer 2, add b2, ReLU, round to BF16, dot
//      with W3; the two column halves of a row meet in shared memory and b3
//      is added.
// Group B's output of tile t overlaps group A's layer-1 epilogue of tile
// t + 1, and the staging of tile t + 1 overlaps layer 2 of tile t.  Every
// mbarrier wait is bounded (about 2 s); a wait that gives up sets the status
// word, every role leaves its loop, the MMAs are drained and tensor memory is
// freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "epi_host.h"
#include "epi_internal.cuh"
#include "epi_tcgen05.cuh"

namespace epi {
namespace mlptc {

constexpr int kRows = 128;
constexpr int kHidden = 256;
constexpr int kKin = 32;                       // padded inputs
constexpr int kGroupWarps = 8;                 // per epilogue group
constexpr int kGroupThreads = 32 * kGroupWarps;
constexpr int kWarpMma = 2 * kGroupWarps;      // warp 16
constexpr int kThreads = 32 * (2 * kGroupWarps + 1);
constexpr uint32_t kW2Bytes = 4 * kHidden * 128;
constexpr uint32_t kW1Bytes = kHidden * 64;
constexpr uint32_t kH1Bytes = 4 * kRows * 128;
constexpr uint32_t kXBytes = kRows * 64;        // one input tile
constexpr uint32_t kKBlockH = kRows * 128;     // one K block of H1
constexpr uint32_t kKBlockW = kHidden * 128;   // one K block of W2
constexpr unsigned long long kTimeoutNs = 2000000000ull;

// kind::f16 with BF16 A and B, FP32 D, K-major operands, M = 128, N = 256
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHidden >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

// byte offset of 16-byte chunk c (0..7) of row r inside a K block in the
// 128-byte swizzle
__device__ __forceinline__ uint32_t sw(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// the same in the 64-byte swizzle (rows of 64 bytes, chunk c in 0..3; the
// chunk index is XORed with bits 7-8 of the row's byte offset)
__device__ __forceinline__ uint32_t sw64(int r, int c) { return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4)); }

// K-major operand in the 64-byte swizzle: 8-row atoms of 512 bytes stacked
// along M/N (stride 512), descriptor version 1, layout SWIZZLE_64B
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16(v)); }

// bounded wait; every thread calls it, the caller syncs and tests the flag
__device__ __forceinline__ void wait_phase(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return;
    const uint64_t t0 = now_ns();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return;
        if (now_ns() - t0 > kTimeoutNs) {
            *abort_flag = 1;
            return;
        }
    }
}


__device__ __forceinline__ void named_bar(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Every thread of a named-barrier group waits, then the group meets in a
// barrier that ORs the threads' abort flags, so that all of its threads leave
// their loop at the same point when any wait gave up (a group barrier never
// waits for threads that left).
__device__ __forceinline__ bool group_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int group)
{
    wait_phase(bar, parity, abort_flag);
    const int mine = *abort_flag ? 1 : 0;
    int any;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(any)
        : "r"(mine), "r"(group), "r"(kGroupThreads)
        : "memory");
    return !any;
}

// the single MMA thread
__device__ __forceinline__ bool wait_ok(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    wait_phase(bar, parity, abort_flag);
    return !*abort_flag;
}

__global__ void __launch_bounds__(kThreads, 1)
    mlp_forward_kernel(const float *__restrict__ X, int64_t rows, const uint32_t *__restrict__ idx,
                       const int32_t *__restrict__ rows_dev, int n_in, const float *__restrict__ norm,
                       const __nv_bfloat16 *__restrict__ W1, const float *__restrict__ b1,
                       const __nv_bfloat16 *__restrict__ W2, const float *__restrict__ b2,
                       const __nv_bfloat16 *__restrict__ W3, const float *__restrict__ b3, float *__restrict__ y,
                       int32_t *__restrict__ status)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    unsigned char *w2s = smem;
    unsigned char *h1s = w2s + kW2Bytes;
    unsigned char *w1s = h1s + kH1Bytes;
    unsigned char *xs = w1s + kW1Bytes;        // two input tiles
    __shared__ float part[2][kRows];           // row partials of the last layer
    __shared__ float nrm[2][kKin];             // input shift and scale (0 past n_in)
    __shared__ __align__(8) uint64_t x_full, m1_done, h1_full, m2_done, e2_free, drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // with rows_dev, the row count is read on the device (at most `rows`);
    // with idx, row j of the launch is input row idx[j] and its prediction
    // goes to y[idx[j]]
    if (rows_dev) {
        const int64_t rd = *rows_dev;
        rows = rd < rows ? (rd > 0 ? rd : 0) : rows;
    }
    const int64_t n_tiles = (rows + kRows - 1) / kRows;
    const int64_t my_tiles = (int64_t)blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        mbar_init(&x_full, kGroupWarps);
        mbar_init(&m1_done, 1);
        mbar_init(&h1_full, kGroupWarps);
        mbar_init(&m2_done, 1);
        mbar_init(&e2_free, kGroupWarps);
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kWarpMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // weights into the swizzled layouts (all threads)
    for (int idx = tid; idx < kHidden * 32; idx += kThreads) {
        const int n = idx >> 5, c32 = idx & 31;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(W2 + (size_t)n * kHidden) + c32);
        *reinterpret_cast<uint4 *>(w2s + (c32 >> 3) * kKBlockW + sw(n, c32 & 7)) = v;
    }
    const unsigned short *w1u = reinterpret_cast<const unsigned short *>(W1);
    for (int idx = tid; idx < kHidden * 4; idx += kThreads) {
        const int n = idx >> 2, c = idx & 3;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int e0 = 8 * c + 2 * q, e1 = e0 + 1;
            const uint32_t lo = e0 < n_in ? w1u[(size_t)n * n_in + e0] : 0u;
            const uint32_t hi = e1 < n_in ? w1u[(size_t)n * n_in + e1] : 0u;
            w[q] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4 *>(w1s + sw64(n, c)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    for (int e = tid; e < kKin; e += kThreads) {
        nrm[0][e] = e < n_in ? norm[e] : 0.0f;
        nrm[1][e] = e < n_in ? norm[n_in + e] : 0.0f;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    if (warp < kGroupWarps) {
        // ------------------------------------- group A: stage X', layer-1 epilogue
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16);
        // staging: thread tid takes row tid / 2, inputs [16 (tid % 2), +16)
        const int sr = tid >> 1, sh = tid & 1;
        auto stage = [&](int64_t tile, int buf) {
            const int64_t row = tile * kRows + sr;
            const bool valid = row < rows;
            const float *src = X + (idx && valid ? (int64_t)idx[row] : row) * n_in;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int e = 16 * sh + j;
                v[j] = (valid && e < n_in) ? __ldg(src + e) : 0.0f;
            }
#pragma unroll
            for (int cc = 0; cc < 2; cc++) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int j = 8 * cc + 2 * q, e = 16 * sh + j;
                    w[q] = pack_bf16((v[j] - nrm[0][e]) * nrm[1][e], (v[j + 1] - nrm[0][e + 1]) * nrm[1][e + 1]);
                }
                *reinterpret_cast<uint4 *>(xs + buf * kXBytes + sw64(sr, 2 * sh + cc)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&x_full);
        };
        if (my_tiles > 0) stage(blockIdx.x, 0);
        for (int64_t i = 0; i < my_tiles; i++) {
            const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
            // layer 1 done, and H1 free once the previous layer 2 is done
            if (!group_wait(&m1_done, (uint32_t)(i & 1), &abort_flag, 1)) break;
            if (i > 0 && !group_wait(&m2_done, (uint32_t)((i - 1) & 1), &abort_flag, 1)) break;
            tc_fence_after();
#pragma unroll 1
            for (int q = 0; q < 4; q++) {
                const int col0 = 128 * half + 32 * q;
                uint32_t v[32];
                TMEM_LD32(lane_addr + (uint32_t)col0, v);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float4 ba = __ldg(reinterpret_cast<const float4 *>(b1 + col0 + 8 * c));
                    const float4 bb = __ldg(reinterpret_cast<const float4 *>(b1 + col0 + 8 * c + 4));
                    const float bias[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
                    uint32_t w[4];
#pragma unroll
                    for (int p = 0; p < 4; p++) {
                        const int ii = 8 * c + 2 * p;
                        const float a = fmaxf(__uint_as_float(v[ii]) + bias[2 * p], 0.0f);
                        const float b = fmaxf(__uint_as_float(v[ii + 1]) + bias[2 * p + 1], 0.0f);
                        w[p] = pack_bf16(a, b);
                    }
                    const int col = col0 + 8 * c;
                    *reinterpret_cast<uint4 *>(h1s + (col >> 6) * kKBlockH + sw(r, (col & 63) >> 3)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            fence_proxy_async();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&h1_full);
            // the next tile's inputs while layer 2 runs (its layer 1 then
            // follows in the tensor pipe; layer-1 columns were read above)
            if (i + 1 < my_tiles) stage(tile + gridDim.x, (int)((i + 1) & 1));
        }
    } else if (warp < 2 * kGroupWarps) {
        // ------------------------------------- group B: layer-2 epilogue and output
        const int gw = warp - kGroupWarps;
        const int quad = gw & 3, half = gw >> 2;
        const int r = quad * 32 + lane;
        const int gt = tid - kGroupThreads;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16);
        for (int64_t i = 0; i < my_tiles; i++) {
            const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
            if (!group_wait(&m2_done, (uint32_t)(i & 1), &abort_flag, 2)) break;
            tc_fence_after();
            float acc = 0.0f;
#pragma unroll 1
            for (int q = 0; q < 4; q++) {
                const int col0 = 128 * half + 32 * q;
                uint32_t v[32];
                TMEM_LD32(lane_addr + (uint32_t)(kHidden + col0), v);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float4 ba = __ldg(reinterpret_cast<const float4 *>(b2 + col0 + 8 * c));
                    const float4 bb = __ldg(reinterpret_cast<const float4 *>(b2 + col0 + 8 * c + 4));
                    const float bias[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
                    const uint4 w3 = __ldg(reinterpret_cast<const uint4 *>(W3 + col0 + 8 * c));
                    const __nv_bfloat162 *wp = reinterpret_cast<const __nv_bfloat162 *>(&w3);
#pragma unroll
                    for (int p = 0; p < 4; p++) {
                        const float2 wf = __bfloat1622float2(wp[p]);
                        const int ii = 8 * c + 2 * p;
                        const float h0 = bf16_round(fmaxf(__uint_as_float(v[ii]) + bias[2 * p], 0.0f));
                        const float h1 = bf16_round(fmaxf(__uint_as_float(v[ii + 1]) + bias[2 * p + 1], 0.0f));
                        acc = fmaf(h0, wf.x, acc);
                        acc = fmaf(h1, wf.y, acc);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&e2_free);
            part[half][r] = acc;
            named_bar(2, kGroupThreads);
            if (gt < kRows) {
                const int64_t row = tile * kRows + gt;
                if (row < rows) y[idx ? (int64_t)idx[row] : row] = part[0][gt] + part[1][gt] + __ldg(b3);
            }
            named_bar(2, kGroupThreads);
        }
    } else if (warp == kWarpMma) {
        // ------------------------------------- MMA issuer (one elected lane)
        if (lane == 0) {
            const uint64_t bd1 = sdesc64(smem_u32(w1s));
            const uint32_t h0 = smem_u32(h1s), w0 = smem_u32(w2s), x0 = smem_u32(xs);
            bool issued = false;
            for (int64_t i = 0; i < my_tiles; i++) {
                const uint32_t par = (uint32_t)(i & 1);
                if (!wait_ok(&x_full, par, &abort_flag)) break;
                tc_fence_after();
                const uint64_t ad1 = sdesc64(x0 + (uint32_t)(i & 1) * kXBytes);
#pragma unroll
                for (int kk = 0; kk < kKin / 16; kk++) mma_bf16(tmem_base, ad1 + 2 * kk, bd1 + 2 * kk, kk ? 1u : 0u);
                mma_commit(&m1_done);
                issued = true;
                if (!wait_ok(&h1_full, par, &abort_flag)) break;
                if (i > 0 && !wait_ok(&e2_free, (uint32_t)((i - 1) & 1), &abort_flag)) break;
                tc_fence_after();
#pragma unroll
                for (int kb = 0; kb < 4; kb++) {
                    const uint64_t ad = sdesc(h0 + kb * kKBlockH), bd = sdesc(w0 + kb * kKBlockW);
#pragma unroll
                    for (int kk = 0; kk < 4; kk++)
                        mma_bf16(tmem_base + kHidden, ad + 2 * kk, bd + 2 * kk, (kb | kk) ? 1u : 0u);
                }
                mma_commit(&m2_done);
            }
            if (issued) {
                // every MMA finished before tensor memory is freed
                mma_commit(&drain_bar);
                const uint64_t t0 = now_ns();
                while (!mbar_try(&drain_bar, 0) && now_ns() - t0 < kTimeoutNs) {}
            }
            if (abort_flag) atomicOr(status, ST_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kWarpMma) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
}

}  // namespace mlptc

size_t mlp_tc_smem_bytes()
{
    return 1024 + mlptc::kW2Bytes + mlptc::kH1Bytes + mlptc::kW1Bytes + 2 * mlptc::kXBytes;
}

bool mlp_tc_applies(int n_in, int hidden) { return hidden == mlptc::kHidden && n_in >= 1 && n_in <= mlptc::kKin; }

cudaError_t launch_mlp_forward_tc(const float *X, int64_t rows, const uint32_t *idx, const int32_t *rows_dev, int n_in,
                                  const float *norm, const void *W1, const float *b1, const void *W2, const float *b2,
                                  const void *W3, const float *b3, float *y, int32_t *status, int num_sms,
                                  cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    const size_t smem = mlp_tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(mlptc::mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (rows + mlptc::kRows - 1) / mlptc::kRows;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    mlptc::mlp_forward_kernel<<<grid, mlptc::kThreads, smem, st>>>(
        X, rows, idx, rows_dev, n_in, norm, static_cast<const __nv_bfloat16 *>(W1), b1, static_cast<const __nv_bfloat16 *>(W2), b2,
        static_cast<const __nv_bfloat16 *>(W3), b3, y, status);
    return cudaGetLastError();
}

}  // namespace epi
