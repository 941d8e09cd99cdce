// Tensor-core GEMM for the proposer network's training step (tcgen05,
// sm_103a).  The paper has no learned part; this is the contraction of the
// network's layer-2 products, which dominate a training step:
//     forward   Z2 = H1 . W2^T            (rows x 256 x 256)
//     backward  dH1 = dZ2 . W2            (rows x 256 x 256)
//               gW2 = dZ2^T . H1          (256 x 256 x rows)
// All three are written as C[M x N] = sum_k A[m][k] B[n][k] with both
// operands BF16 and K-major (row-major with K contiguous; the callers keep
// transposed copies where a product needs one), FP32 accumulation in tensor
// memory, and C in FP32.
//
// One CTA computes one 128 x NT tile of C over one slice of K: 128 threads
// load 64-wide K chunks of A (128 rows) and B (NT rows) with 16-byte loads
// into shared memory in the 128-byte swizzle (two stages), one thread issues
// the MMAs (M128 x NT x K16, four per chunk) and commits each stage to an
// mbarrier, so the loads of chunk c + 1 overlap the MMAs of chunk c.  Rows,
// columns and K past the matrix edges enter as zeros.  With several K slices
// (split K, for the products whose K is the batch), every slice writes its
// own partial tile and a second kernel adds the slices in a fixed order, so
// results do not depend on scheduling.  Waits are bounded (2 s) and report
// ST_TIMEOUT.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "epi_host.h"
#include "epi_internal.cuh"
#include "epi_tcgen05.cuh"

namespace epi {
namespace gemmtc {

constexpr int kThreads = 128;
constexpr int kM = 128;
constexpr int kKC = 64;                              // K elements per chunk (128 bytes)
constexpr unsigned long long kTimeoutNs = 2000000000ull;

struct Args {
    const __nv_bfloat16 *A;   // [M][lda]
    const __nv_bfloat16 *B;   // [N][ldb]
    float *C;                 // [M][ldc] (one slice) or partials [slices][M][ldc]
    int M, N, K;
    int64_t lda, ldb, ldc;
    int nt;                   // N tile: 32, 64, 128 or 256
    int slices, chunks_per_slice;
    int32_t *status;
};

// kind::f16, BF16 x BF16 -> F32, K-major A and B, M = 128, N = nt
__device__ __forceinline__ uint32_t idesc(int nt)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

// 16-byte chunk c (0..7) of row r in the 128-byte swizzle
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ bool bounded_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (!mbar_try(bar, parity))
        if (now_ns() - t0 > kTimeoutNs) return false;
    return true;
}

// rows [r0, r0 + rows) of X (row stride ld) over K elements [k0, k0 + 64)
// into a swizzled stage; zeros outside [0, R) x [0, K)
__device__ __forceinline__ void load_chunk(unsigned char *dst, const __nv_bfloat16 *X, int64_t ld, int r0, int rows,
                                           int R, int k0, int K)
{
    for (int i = threadIdx.x; i < rows * 8; i += kThreads) {
        const int r = i >> 3, c = i & 7;
        const int row = r0 + r, k = k0 + 8 * c;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < R) {
            const __nv_bfloat16 *src = X + (int64_t)row * ld + k;
            if (k + 8 <= K) {
                v = __ldg(reinterpret_cast<const uint4 *>(src));
            } else if (k < K) {
                uint16_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int e = 0; e < K - k; e++) h[e] = reinterpret_cast<const uint16_t *>(src)[e];
                v = make_uint4(h[0] | (uint32_t)h[1] << 16, h[2] | (uint32_t)h[3] << 16, h[4] | (uint32_t)h[5] << 16,
                               h[6] | (uint32_t)h[7] << 16);
            }
        }
        *reinterpret_cast<uint4 *>(dst + swz(r, c)) = v;
    }
}

__global__ void __launch_bounds__(kThreads) gemm_kernel(const Args P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int stage_bytes = (kM + P.nt) * 128;
    __shared__ __align__(8) uint64_t freed[2], done;
    __shared__ uint32_t tmem_sh;
    __shared__ int bad;
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * kM, n0 = blockIdx.y * P.nt, slice = blockIdx.z;
    const int nk = (P.K + kKC - 1) / kKC;
    const int c_begin = slice * P.chunks_per_slice;
    const int c_end = min(nk, c_begin + P.chunks_per_slice);
    if (tid == 0) {
        mbar_init(&freed[0], 1);
        mbar_init(&freed[1], 1);
        mbar_init(&done, 1);
        bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(P.nt)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    const uint32_t id = idesc(P.nt);
    for (int c = c_begin; c < c_end; c++) {
        const int i = c - c_begin, s = i & 1;
        unsigned char *sa = smem + s * stage_bytes;
        unsigned char *sb = sa + kM * 128;
        // the MMAs that read this stage two chunks ago must have finished
        if (i >= 2 && !bounded_wait(&freed[s], ((i - 2) >> 1) & 1)) bad = 1;
        __syncthreads();
        if (bad) break;
        load_chunk(sa, P.A, P.lda, m0, kM, P.M, c * kKC, P.K);
        load_chunk(sb, P.B, P.ldb, n0, P.nt, P.N, c * kKC, P.K);
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint64_t ad = sdesc(smem_u32(sa)), bd = sdesc(smem_u32(sb));
#pragma unroll
            for (int kk = 0; kk < kKC / 16; kk++)
                mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, id, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&freed[s]);
        }
    }
    // every MMA of the CTA has finished before the accumulator is read
    if (tid == 0) {
        mma_commit(&done);
        if (!bounded_wait(&done, 0)) bad = 1;
    }
    __syncthreads();
    tc_fence_after();
    const bool empty = c_end <= c_begin;
    // thread t reads tile row t (TMEM lane t) in 32-column pieces
    const int row = m0 + tid;
    float *crow = P.C + (size_t)slice * P.M * P.ldc + (int64_t)row * P.ldc;
    for (int cb = 0; cb < P.nt; cb += 32) {
        uint32_t v[32];
        const uint32_t ta = tmem + ((uint32_t)((tid >> 5) * 32) << 16) + (uint32_t)cb;
        TMEM_LD32(ta, v);
        tmem_wait_ld();
        if (row < P.M && !bad) {
#pragma unroll
            for (int q = 0; q < 32; q++) {
                const int col = n0 + cb + q;
                if (col < P.N) crow[col] = empty ? 0.0f : __uint_as_float(v[q]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.nt) : "memory");
    }
    if (tid == 0 && bad) atomicOr(P.status, ST_TIMEOUT);
}

// C[m][n] (+)= sum over the slices of the partial tiles, in slice order
__global__ void sum_slices_kernel(const float *__restrict__ part, int slices, int M, int N, int64_t ldp,
                                  float *__restrict__ C, int64_t ldc, int accumulate)
{
    const int64_t total = (int64_t)M * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / N), n = (int)(i - (int64_t)m * N);
        float s = 0.0f;
        for (int q = 0; q < slices; q++) s += part[((int64_t)q * M + m) * ldp + n];
        float *o = C + (int64_t)m * ldc + n;
        *o = accumulate ? *o + s : s;
    }
}

}  // namespace gemmtc

size_t gemm_tc_smem_bytes(int nt) { return 2 * (size_t)(gemmtc::kM + nt) * 128 + 1024; }

// Partial-tile scratch (floats) a split-K product of M x N needs.
size_t gemm_tc_partial_floats(int M, int N, int K, int num_sms)
{
    int slices = 1;
    const int nk = (K + gemmtc::kKC - 1) / gemmtc::kKC;
    const int nt = N >= 256 ? 256 : (N > 64 ? 128 : (N > 32 ? 64 : 32));
    const int tiles = ((M + gemmtc::kM - 1) / gemmtc::kM) * ((N + nt - 1) / nt);
    if (tiles < num_sms && nk >= 4) slices = std::min(nk / 2, (2 * num_sms + tiles - 1) / tiles);
    return slices > 1 ? (size_t)slices * M * N : 0;
}

// C (FP32 [M][ldc]) = A . B^T with A [M][K], B [N][K] BF16 K-major (row
// strides lda, ldb: multiples of 8 elements, rows 16-byte aligned).  K is
// split over CTAs when the output has fewer tiles than SMs and `partial`
// holds gemm_tc_partial_floats(M, N, K) floats; otherwise one slice.
cudaError_t launch_gemm_tc(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc, int M, int N,
                           int K, float *partial, int32_t *status, int num_sms, cudaStream_t st)
{
    gemmtc::Args P;
    P.A = static_cast<const __nv_bfloat16 *>(A);
    P.B = static_cast<const __nv_bfloat16 *>(B);
    P.M = M; P.N = N; P.K = K;
    P.lda = lda; P.ldb = ldb;
    P.nt = N >= 256 ? 256 : (N > 64 ? 128 : (N > 32 ? 64 : 32));
    const int mtiles = (M + gemmtc::kM - 1) / gemmtc::kM;
    const int nk = (K + gemmtc::kKC - 1) / gemmtc::kKC;
    const size_t need = gemm_tc_partial_floats(M, N, K, num_sms);
    P.slices = (need && partial) ? (int)(need / ((size_t)M * N)) : 1;
    // without a split, narrower N tiles give more CTAs when M alone does not
    // fill the GPU
    if (P.slices == 1 && P.nt == 256 && mtiles < num_sms) P.nt = 128;
    P.chunks_per_slice = (nk + P.slices - 1) / P.slices;
    P.status = status;
    const bool split = P.slices > 1;
    P.C = split ? partial : C;
    P.ldc = split ? N : ldc;
    const size_t smem = gemm_tc_smem_bytes(P.nt);
    cudaError_t e = cudaFuncSetAttribute(gemmtc::gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(mtiles, (N + P.nt - 1) / P.nt, P.slices);
    gemmtc::gemm_kernel<<<grid, gemmtc::kThreads, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess || !split) return e;
    const int64_t total = (int64_t)M * N;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
    gemmtc::sum_slices_kernel<<<blocks, 256, 0, st>>>(partial, P.slices, M, N, N, C, ldc, 0);
    return cudaGetLastError();
}

}  // namespace epi
