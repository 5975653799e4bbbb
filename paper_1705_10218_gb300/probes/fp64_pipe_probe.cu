// fp64_pipe_probe.cu -- the FP64 rates this GPU reaches, measured, for the
// choice of the FP64 block-product units: FMA (DFMA) fed from registers, DFMA
// with both operands from shared memory (as the packed numeric kernel reads
// them), and the FP64 tensor-core MMA (mma.sync m8n8k4, DMMA). Standalone
// program, not part of the library:
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_pipe_probe fp64_pipe_probe.cu -lnvidia-ml
//   ./fp64_pipe_probe
//
// Each kernel runs independent accumulation chains long enough (a few tens of
// milliseconds) for the launch to be negligible; the rate is FLOPs (2 per FMA,
// 2*8*8*4 per m8n8k4 MMA) over the CUDA-event time, and its fraction of the
// peak derived from the SM count and the SM clock read while it ran.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
#include <nvml.h>

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);     \
      return 1;                                                                    \
    }                                                                              \
  } while (0)

constexpr int kNT = 12;  // independent accumulators per thread

// register-only chains: acc = acc * x + y
__global__ void __launch_bounds__(256) dfma_reg(double *out, int steps, double x, double y) {
  double acc[kNT];
#pragma unroll
  for (int t = 0; t < kNT; t++) acc[t] = threadIdx.x + t;
  for (int u = 0; u < steps; u++) {
#pragma unroll
    for (int t = 0; t < kNT; t++) acc[t] = fma(acc[t], x, y);
  }
  double s = 0;
#pragma unroll
  for (int t = 0; t < kNT; t++) s += acc[t];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// both operands of every FMA loaded from shared memory, base pointers stepping
// through a 2 x 1024-double table (the access pattern of the packed kernel)
__global__ void __launch_bounds__(256) dfma_smem(double *out, int steps) {
  __shared__ double sm[4096];
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) sm[i] = 1.0 + i * 1e-9;
  __syncthreads();
  double acc[kNT];
  uint32_t ia[kNT], ib[kNT];
#pragma unroll
  for (int t = 0; t < kNT; t++) {
    acc[t] = 0.0;
    ia[t] = (threadIdx.x + 32 * t) & 1023;
    ib[t] = (threadIdx.x * 7 + t) & 1023;
  }
  for (int rep = 0; rep < steps / 1024; rep++) {
    const double *A = sm, *B = sm + 2048;
#pragma unroll 1
    for (int u = 0; u < 1024; u++) {
#pragma unroll
      for (int t = 0; t < kNT; t++) acc[t] = fma(A[ia[t]], B[ib[t]], acc[t]);
      A += 1;
      B += 1;
    }
  }
  double s = 0;
#pragma unroll
  for (int t = 0; t < kNT; t++) s += acc[t];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 tensor-core MMA, m8n8k4: 4 independent accumulator pairs per warp
__global__ void __launch_bounds__(256) dmma(double *out, int steps) {
  double a = 1.0 + threadIdx.x * 1e-9, b = 1.0 - threadIdx.x * 1e-9;
  double d[4][2];
#pragma unroll
  for (int j = 0; j < 4; j++) d[j][0] = d[j][1] = j;
  for (int u = 0; u < steps; u++) {
#pragma unroll
    for (int j = 0; j < 4; j++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(d[j][0]), "+d"(d[j][1])
                   : "d"(a), "d"(b));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = d[0][0] + d[1][1] + d[2][0] + d[3][1];
}

int main() {
  int dev = 0, nsm = 0;
  CK(cudaSetDevice(dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  nvmlDevice_t nd;
  const bool nvml = nvmlInit() == NVML_SUCCESS && nvmlDeviceGetHandleByIndex(dev, &nd) == NVML_SUCCESS;
  double *out;
  CK(cudaMalloc(&out, (size_t)nsm * 4 * 256 * sizeof(double)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  printf("SMs %d\n", nsm);
  for (int blocks_per_sm : {1, 2, 4}) {  // 8, 16, 32 warps per SM
    const int grid = nsm * blocks_per_sm;
    for (int kind = 0; kind < 3; kind++) {
      const int steps = kind == 2 ? 1 << 14 : 1 << 16;
      for (int rep = 0; rep < 2; rep++) {  // the first run warms up
        CK(cudaEventRecord(e0));
        if (kind == 0) dfma_reg<<<grid, 256>>>(out, steps, 0.999999, 1e-7);
        else if (kind == 1) dfma_smem<<<grid, 256>>>(out, steps);
        else dmma<<<grid, 256>>>(out, steps);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
      }
      unsigned int mhz = 0;
      if (nvml) nvmlDeviceGetClockInfo(nd, NVML_CLOCK_SM, &mhz);
      // time the measured run again, with the clock read right after it
      CK(cudaEventRecord(e0));
      if (kind == 0) dfma_reg<<<grid, 256>>>(out, steps, 0.999999, 1e-7);
      else if (kind == 1) dfma_smem<<<grid, 256>>>(out, steps);
      else dmma<<<grid, 256>>>(out, steps);
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (nvml) nvmlDeviceGetClockInfo(nd, NVML_CLOCK_SM, &mhz);
      const double threads = (double)grid * 256;
      const double flop = kind == 2 ? threads / 32 * steps * 4 * 2.0 * 8 * 8 * 4
                                    : threads * steps * kNT * 2.0;
      const double gfs = flop / (ms * 1e-3) / 1e9;
      const double peak = nsm * 4.0 * (mhz ? mhz : 2070) / 1e3;  // 2 FP64 FMA per SM per clock
      const char *name = kind == 0 ? "DFMA registers" : kind == 1 ? "DFMA shared-memory operands" : "DMMA m8n8k4";
      printf("%-28s warps/SM %2d: %8.1f GFLOP/s  %.3f of %7.1f (SM clock %u MHz)  %.2f ms\n", name,
             blocks_per_sm * 8, gfs, gfs / peak, peak, mhz, ms);
    }
  }
  return 0;
}
