// Device side of the seeded input generator (definition in synth_def.h). Input generation
// only: it writes synthetic image and master sectors straight into device memory so that
// large workloads need no host copy. Every byte equals what synth_host.c produces.
#include <cuda_runtime.h>
#include <stdint.h>

#include "synth_def.h"

namespace {

__global__ void k_image(sy_plan p, uint64_t first, uint64_t n, uint64_t* out) {
  uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint64_t buf[64];
  sy_image_sector(&p, first + j, buf);
  uint64_t* dst = out + j * 64;
#pragma unroll 8
  for (int w = 0; w < 64; w++) dst[w] = buf[w];
}

// All sectors of all master files, concatenated in file order. file_base[f] = first sector
// of file f in the concatenation (n_files + 1 entries, the last = total).
__global__ void k_masters(uint64_t mu, const uint64_t* file_base, uint32_t n_files, uint64_t total, uint64_t* out) {
  uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= total) return;
  uint32_t lo = 0, hi = n_files;  // largest f with file_base[f] <= j
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) / 2;
    if (file_base[mid] <= j) lo = mid; else hi = mid;
  }
  uint64_t buf[64];
  sy_master_sector(mu, lo, (uint32_t)(j - file_base[lo]), buf);
  uint64_t* dst = out + j * 64;
#pragma unroll 8
  for (int w = 0; w < 64; w++) dst[w] = buf[w];
}

}  // namespace

extern "C" int synth_image_cuda(uint64_t sigma, uint64_t mu, const int32_t* plant_file, const uint32_t* plant_fcluster,
                                const uint8_t* plant_over, uint64_t n_clusters, const uint32_t* file_nsect,
                                const uint8_t* vocab, uint64_t first, uint64_t n, void* out, void* stream) {
  if (n == 0) return 0;
  if (((uintptr_t)out & 7u) != 0) return (int)cudaErrorInvalidValue;
  sy_plan p;
  p.sigma = sigma;
  p.mu = mu;
  p.plant_file = plant_file;
  p.plant_fcluster = plant_fcluster;
  p.plant_over = plant_over;
  p.file_nsect = file_nsect;
  p.vocab = vocab;
  p.n_clusters = n_clusters;
  const int T = 128;
  uint64_t blocks = (n + T - 1) / T;
  k_image<<<(unsigned)blocks, T, 0, (cudaStream_t)stream>>>(p, first, n, (uint64_t*)out);
  return (int)cudaGetLastError();
}

extern "C" int synth_masters_cuda(uint64_t mu, const uint64_t* file_base, uint32_t n_files, uint64_t total, void* out,
                                  void* stream) {
  if (total == 0 || n_files == 0) return 0;
  if (((uintptr_t)out & 7u) != 0) return (int)cudaErrorInvalidValue;
  const int T = 128;
  uint64_t blocks = (total + T - 1) / T;
  k_masters<<<(unsigned)blocks, T, 0, (cudaStream_t)stream>>>(mu, file_base, n_files, total, (uint64_t*)out);
  return (int)cudaGetLastError();
}
