// tcgen05_rate_probe.cu -- how many SM clocks one tcgen05.mma (cta_group::1)
// costs as a function of its shape (M, N) and of where its A operand lives
// (shared memory or tensor memory), for the choice of tile shapes in the
// split-precision kernels. Standalone program, not part of the library:
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O2 -o tcgen05_rate_probe tcgen05_rate_probe.cu
//   ./tcgen05_rate_probe
//
// One CTA per SM (160 KB of dynamic shared memory keeps a second one off the
// SM); thread 0 issues R MMAs back to back, all operands fixed at compile time
// (a descriptor or address computed in the issuing loop adds its own cost),
// rotating over ND accumulators so that consecutive MMAs are independent when
// ND > 1. The time is clock64 from the first issue to the completion of the
// last (tcgen05.commit onto an mbarrier, waited on with a bounded loop); the
// operand values (all 1.0) and the results are not looked at.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, no swizzle: lbo = byte stride between the two 16-byte core
// matrices along K, sbo = byte stride between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFF) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

// kind::f16 / kind::tf32 instruction descriptor: FP32 accumulator, A and B of
// type ab (1 = BF16, 2 = TF32), K-major operands, N and M.
__host__ __device__ constexpr uint32_t instr_desc(int ab, int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(ab) << 7) | (static_cast<uint32_t>(ab) << 10) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

constexpr int kSmemBytes = 160 * 1024;
constexpr int kOperandBytes = 40960;  // A at 0 (<= 4 KB), B at 8192 (<= 8 KB)
constexpr uint32_t kAColumn = 256;     // A operand in tensor memory (TS form)

// TF32: K = 8 per MMA (32 bytes a row, as BF16's K = 16), FLOPs per MMA 2*M*N*8.
template <bool TF32, bool TS, int M, int N, int ND>
__global__ void __launch_bounds__(128) mma_rate(int reps, long long *clk, int *timed_out) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint32_t *holder = reinterpret_cast<uint32_t *>(smem + kOperandBytes);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kOperandBytes + 64);
  const int warp = threadIdx.x >> 5;
  const uint32_t one = TF32 ? 0x3F800000u : 0x3F803F80u;
  for (int i = threadIdx.x; i < kOperandBytes / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(smem)[i] = one;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(holder)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;
  if (TS) {  // A operand: 128 lanes x 8 columns from kAColumn
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                     tmem + (static_cast<uint32_t>(warp * 32) << 16) + kAColumn),
                 "r"(one));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint64_t adesc = smem_desc(smem_u32(smem), 8 * (M / 8) * 16, 128);
    const uint64_t bdesc = smem_desc(smem_u32(smem + 8192), static_cast<uint32_t>(N * 16), 128);
    constexpr uint32_t idesc = instr_desc(TF32 ? 2 : 1, M, N);
    const long long t0 = clock64();
    for (int r = 0; r < reps; r += ND) {
#pragma unroll
      for (int d = 0; d < ND; d++) {
        const uint32_t dcol = tmem + static_cast<uint32_t>(d * N);
        if (TS) {
          if (TF32)
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;" ::"r"(dcol),
                         "r"(tmem + kAColumn), "l"(bdesc), "r"(idesc));
          else
            asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 1;" ::"r"(dcol),
                         "r"(tmem + kAColumn), "l"(bdesc), "r"(idesc));
        } else {
          if (TF32)
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(dcol), "l"(adesc),
                         "l"(bdesc), "r"(idesc));
          else
            asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;" ::"r"(dcol), "l"(adesc),
                         "l"(bdesc), "r"(idesc));
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; it++)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(bar))
          : "memory");
    const long long t1 = clock64();
    if (!done) *timed_out = 1;
    if (blockIdx.x == 0) *clk = t1 - t0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

template <bool TF32, bool TS, int M, int N, int ND>
bool run(int nsm, long long *clk, int *timed_out) {
  static_assert(ND * N <= 256, "accumulators must stay below the A operand's columns");
  static_assert(M == 128 || !TS, "the A-in-tensor-memory form is timed at M = 128 only");
  constexpr int reps = 4096;
  cudaFuncSetAttribute(mma_rate<TF32, TS, M, N, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  for (int rep = 0; rep < 2; rep++) {  // the first launch is the warm-up
    mma_rate<TF32, TS, M, N, ND><<<nsm, 128, kSmemBytes>>>(reps, clk, timed_out);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      printf("CUDA error %s\n", cudaGetErrorString(e));
      return false;
    }
  }
  long long c = 0;
  int flag = 0;
  cudaMemcpy(&c, clk, sizeof c, cudaMemcpyDeviceToHost);
  cudaMemcpy(&flag, timed_out, sizeof flag, cudaMemcpyDeviceToHost);
  const double per = static_cast<double>(c) / reps;
  const double flop = 2.0 * M * N * (TF32 ? 8 : 16);
  printf("| %s | %s | %d | %d | %d | %.1f | %.0f |%s\n", TF32 ? "TF32" : "BF16", TS ? "TMEM" : "smem", M, N, ND, per,
         flop / per, flag ? " TIMED OUT" : "");
  return flag == 0;
}

}  // namespace

int main() {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  long long *clk = nullptr;
  int *timed_out = nullptr;
  if (cudaMalloc(&clk, sizeof(long long)) != cudaSuccess || cudaMalloc(&timed_out, sizeof(int)) != cudaSuccess) return 1;
  cudaMemset(timed_out, 0, sizeof(int));
  printf("| kind | A operand | M | N | accumulators | clocks per MMA | FLOP per SM clock |\n|---|---|---|---|---|---|---|\n");
  bool ok = true;
  ok = ok && run<false, true, 128, 16, 1>(nsm, clk, timed_out) && run<false, true, 128, 16, 4>(nsm, clk, timed_out);
  ok = ok && run<false, true, 128, 32, 4>(nsm, clk, timed_out) && run<false, true, 128, 48, 4>(nsm, clk, timed_out);
  ok = ok && run<false, true, 128, 64, 4>(nsm, clk, timed_out) && run<false, true, 128, 96, 2>(nsm, clk, timed_out);
  ok = ok && run<false, true, 128, 128, 2>(nsm, clk, timed_out) && run<false, true, 128, 256, 1>(nsm, clk, timed_out);
  ok = ok && run<false, false, 128, 16, 4>(nsm, clk, timed_out) && run<false, false, 128, 48, 4>(nsm, clk, timed_out);
  ok = ok && run<false, false, 128, 96, 2>(nsm, clk, timed_out) && run<false, false, 128, 256, 1>(nsm, clk, timed_out);
  ok = ok && run<false, false, 64, 16, 4>(nsm, clk, timed_out) && run<false, false, 64, 48, 4>(nsm, clk, timed_out);
  ok = ok && run<false, false, 64, 128, 2>(nsm, clk, timed_out) && run<false, false, 64, 256, 1>(nsm, clk, timed_out);
  ok = ok && run<true, true, 128, 16, 4>(nsm, clk, timed_out) && run<true, true, 128, 32, 4>(nsm, clk, timed_out);
  ok = ok && run<true, true, 128, 64, 4>(nsm, clk, timed_out) && run<true, true, 128, 256, 1>(nsm, clk, timed_out);
  ok = ok && run<true, false, 128, 32, 4>(nsm, clk, timed_out) && run<true, false, 64, 32, 4>(nsm, clk, timed_out);
  cudaFree(clk);
  cudaFree(timed_out);
  return ok ? 0 : 1;
}
