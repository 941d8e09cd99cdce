// Rate of the tensor pipe for the counting path's MMA shapes.
//
// The paper has no counterpart: this is a measurement aid.  The roofline of
// the tensor-core counting kernel is the rate at which one SM retires the
// MMA that kernel issues: tcgen05.mma.kind::f8f6f4 M128 N128 K32 with E4M3
// operands (shape 0, the separate-class variant) or M128 N256 K32 with E5M2
// operands (shape 1, the combined-class variant), FP32 accumulation, both
// operands in shared memory in the 128-byte swizzle.  One CTA per SM issues
// that MMA back to back from one thread, accumulating 32 K steps into one of
// two tensor-memory accumulators in turn (the counting kernel's pattern),
// with no other work on the SM; the operands are zero tiles (the rate does
// not depend on the values).  Every CTA records the SM
// cycles of its issue loop up to the completion of its last MMA; the host
// times the launch with events.  The final wait is bounded (2 s) and reports
// ST_TIMEOUT instead of hanging.
#include <cuda_runtime.h>

#include "epi_host.h"
#include "epi_internal.cuh"
#include "epi_tcgen05.cuh"

namespace epi {
namespace peak {

constexpr int kThreads = 128;
constexpr int kTile = 128 * 128;          // one 128 x 128-byte operand stage (A; B of shape 0)
constexpr unsigned long long kTimeoutNs = 2000000000ull;
// kind::f8f6f4 -> F32, K-major A and B, M = 128; format 0 = E4M3, 1 = E5M2
__host__ __device__ constexpr uint32_t idesc_of(uint32_t fmt, uint32_t n)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate, uint32_t idesc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// n: MMA columns (128 or 256); B stage of n rows after the A stage
__global__ void __launch_bounds__(kThreads, 1) mma_rate_kernel(int64_t stages, unsigned long long *cycles,
                                                               int32_t *status, uint32_t n, uint32_t fmt)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_base_sh;
    const int tid = threadIdx.x;
    const int bytes = kTile + (int)n * 128;
    for (int i = tid; i < bytes / 16; i += kThreads) reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    fence_proxy_async();
    if (tid == 0) {
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    if (tid == 0) {
        const uint64_t ad = sdesc(smem_u32(smem)), bd = sdesc(smem_u32(smem + kTile));
        const uint32_t idesc = idesc_of(fmt, n);
        const long long t0 = clock64();
        for (int64_t s = 0; s < stages; s++) {
            const uint32_t acc = tmem + (uint32_t)(((s >> 5) & 1) * 256);
            mma_f8(acc, ad, bd, (s & 31) ? 1u : 0u, idesc);
#pragma unroll
            for (int kk = 1; kk < 4; kk++) mma_f8(acc, ad + 2 * kk, bd + 2 * kk, 1u, idesc);
        }
        mma_commit(&done);
        const uint64_t w0 = now_ns();
        bool ok = true;
        while (!mbar_try(&done, 0)) {
            if (now_ns() - w0 > kTimeoutNs) { ok = false; break; }
        }
        cycles[blockIdx.x] = (unsigned long long)(clock64() - t0);
        if (!ok) atomicOr(status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

}  // namespace peak

size_t mma_rate_smem_bytes(int shape) { return (size_t)peak::kTile + (shape ? 256u : 128u) * 128u + 1024; }

cudaError_t launch_mma_rate(int shape, int64_t stages, unsigned long long *cycles, int32_t *status, int grid,
                            cudaStream_t st)
{
    const size_t smem = mma_rate_smem_bytes(shape);
    cudaError_t e = cudaFuncSetAttribute(peak::mma_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    peak::mma_rate_kernel<<<grid, peak::kThreads, smem, st>>>(stages, cycles, status, shape ? 256u : 128u,
                                                              shape ? 1u : 0u);
    return cudaGetLastError();
}

}  // namespace epi
