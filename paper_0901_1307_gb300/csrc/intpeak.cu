// Integer throughput micro-benchmark: the denominator of the scan's roofline.
//
// The scan is bound by 32-bit integer issue (lop3, funnel shifts and additions). Three kernels
// run independent dependency chains on every SM long enough to reach steady state:
//   alu   - lop3 chains only (the integer ALU pipe),
//   fma   - mad.lo chains with a run-time multiplier of 1 (the FMA pipe),
//   mixed - one lop3 chain op and one mad.lo chain op in turn (both pipes, issue-bound).
// Each reports operations per second; block 0 also reads %clock64 and %globaltimer around its
// loop, which gives the SM clock during the run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cv.h"
#include "runtime.h"

using namespace cvk;

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

template <int KIND>  // 0 alu, 1 fma, 2 mixed
__global__ void __launch_bounds__(256) peak_kernel(uint32_t* out, int iters, uint32_t one, uint64_t* clk) {
  uint32_t x[kChains], w[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) {
    x[j] = threadIdx.x * 0x9E3779B9u + j;
    w[j] = blockIdx.x * 0x85EBCA6Bu + j;
  }
  const uint32_t y = threadIdx.x ^ 0x5bd1e995u, z = blockIdx.x ^ 0x27d4eb2fu;
  uint64_t c0 = clock64(), g0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < kUnroll; r++) {
#pragma unroll
      for (int j = 0; j < kChains; j++) {
        if (KIND == 0) {
          x[j] = lop3_xor3(x[j], y, z);
        } else if (KIND == 1) {
          w[j] = imad(w[j], one, y);
        } else {
          if (j & 1) w[j] = imad(w[j], one, y); else x[j] = lop3_xor3(x[j], y, z);
        }
      }
    }
  }
  uint64_t c1 = clock64(), g1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) acc ^= x[j] ^ w[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = c1 - c0;
    clk[1] = g1 - g0;
  }
}

}  // namespace

extern "C" int cv_int_peak(cv_int_peak_info* info) {
  if (!info) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  const int threads = 256, blocks = ctx->sms * 8;
  const int iters = 4000;
  uint32_t* out = nullptr;
  uint64_t* clk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto body = [&]() -> int {
    CV_CUDA(cudaMalloc(&out, (size_t)threads * blocks * 4));
    CV_CUDA(cudaMalloc(&clk, 16));
    CV_CUDA(cudaEventCreate(&e0));
    CV_CUDA(cudaEventCreate(&e1));
    const void* fns[3] = {(const void*)peak_kernel<0>, (const void*)peak_kernel<1>, (const void*)peak_kernel<2>};
    double rate[3];
    double mhz_sum = 0;
    for (int k = 0; k < 3; k++) {
      uint32_t one = 1;
      int it = iters;
      void* args[] = {&out, &it, &one, &clk};
      CV_CUDA(cudaLaunchKernel(fns[k], dim3(blocks), dim3(threads), args, 0, nullptr));  // warm-up
      CV_CUDA(cudaEventRecord(e0, nullptr));
      CV_CUDA(cudaLaunchKernel(fns[k], dim3(blocks), dim3(threads), args, 0, nullptr));
      CV_CUDA(cudaEventRecord(e1, nullptr));
      CV_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      CV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double ops = (double)blocks * threads * iters * kUnroll * kChains;
      rate[k] = ops / (ms * 1e-3);
      uint64_t h[2];
      CV_CUDA(cudaMemcpy(h, clk, 16, cudaMemcpyDeviceToHost));
      mhz_sum += h[1] ? (double)h[0] * 1e3 / (double)h[1] : 0.0;
    }
    info->alu_ops_per_s = rate[0];
    info->fma_ops_per_s = rate[1];
    info->mixed_ops_per_s = rate[2];
    info->sm_clock_mhz = mhz_sum / 3.0;
    info->sms = ctx->sms;
    return CV_OK;
  };
  const int rc = body();
  if (out) cudaFree(out);
  if (clk) cudaFree(clk);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
