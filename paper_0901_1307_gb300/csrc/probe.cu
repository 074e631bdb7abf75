// cv_probe_profile: what each lookup of a scan costs in table reads, counted exactly.
//
// The paper measures how the lookup slows as the table fills (Section 4, Figures 10-12, and
// its remark that probing costs more at high occupancy). The scan kernel does not count its
// reads, since a counter there would cost every scan; this entry point replays the same
// lookups outside it. It computes the key words of every sector with the scan's own digest
// pass, then a counting kernel runs the scan's own lookup functions for each sector with a
// counter attached: the Bloom test (when the table has a filter), then either the
// linear-probing walk from the home slot of Eq. 3 (hash layout) or the bisection over the
// sorted keys and the comparison of the records that share the key word (sorted layout).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "cv.h"
#include "cv_internal.h"
#include "cv_launch.h"
#include "handles.h"
#include "runtime.h"
#include "scan_kernel.cuh"

namespace cvk {
namespace {

constexpr uint64_t kProfileChunk = 1ull << 22;  // sectors per digest pass (64 MiB of key words)

// Adds up the reads of the scan's own probe loops (table_probe, sorted_probe).
struct ProbeCount {
  uint64_t* slots;
  uint64_t* keys;
  __device__ __forceinline__ void slot() const { ++*slots; }
  __device__ __forceinline__ void key() const { ++*keys; }
};

// acc: [0] sectors past the Bloom filter, [1] slot records read, [2] sorted keys read,
// [3] sectors whose key is in the table.
__global__ void probe_profile_kernel(const uint4* dig, uint64_t n, uint64_t sector0, TableView tab,
                                     unsigned long long* acc) {
  uint64_t passed = 0, slots = 0, keys = 0, found = 0;
  const ProbeCount cnt{&slots, &keys};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 d = dig[i];
    const uint32_t tau = (uint32_t)((sector0 + i + tab.tau_add) & tab.tau_mask);
    if (tab.use_bloom && !bloom_test(tab, d.y, d.z, d.w, tau)) continue;
    passed++;
    uint32_t post_off = 0;
    const uint32_t c = tab.layout == kLayoutSorted ? sorted_probe(tab, d.x, d.y, d.z, d.w, tau, post_off, cnt)
                                                   : table_probe(tab, d.x, d.y, d.z, d.w, tau, post_off, cnt);
    if (c) found++;
  }
  uint64_t v[4] = {passed, slots, keys, found};
#pragma unroll
  for (int k = 0; k < 4; k++) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], s);
  }
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 4; k++)
      if (v[k]) atomicAdd(acc + k, (unsigned long long)v[k]);
}

}  // namespace
}  // namespace cvk

using namespace cvk;

extern "C" {

int cv_probe_profile(const cv_master* m, const void* image, uint64_t n_bytes, uint64_t base_offset,
                     cv_probe_stats* st, void* stream_) {
  if (!m || !st || st->struct_size < sizeof(cv_probe_stats)) return CV_EINVAL;
  TableView tab;
  int mdev;
  if (master_view(m, &tab, &mdev) != CV_OK || tab.unit != kUnitSector) return CV_EINVAL;
  const uint64_t n = n_bytes / kSector;
  if (n && (!image || ((uintptr_t)image & 15u))) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  if (mdev != ctx->dev) return CV_EINVAL;
  if (n) {
    BufKind kind;
    CV_TRY(classify(ctx, image, &kind));
    if (kind != kDevice) return CV_EINVAL;
  }
  tab.tau_add = (uint32_t)((8u - base_offset % 8u) % 8u);
  cudaStream_t stream = (cudaStream_t)stream_;
  memset((uint8_t*)st + sizeof(uint32_t), 0, sizeof(cv_probe_stats) - sizeof(uint32_t));
  st->layout = tab.layout == kLayoutSorted ? CV_LAYOUT_SORTED : CV_LAYOUT_HASH;
  st->sectors = n;
  if (n == 0) return CV_OK;
  int cfg_i;
  const ScanCfg& cfg = digest_config_for(ctx->cfg_index, (int)tab.sig, &cfg_i);
  Temps tmp(ctx, stream);
  uint4* dig;
  unsigned long long* acc;
  uint32_t* status;
  CV_TRY(tmp.alloc(&dig, (n < kProfileChunk ? n : kProfileChunk) * sizeof(uint4)));
  CV_TRY(tmp.alloc(&acc, 4 * sizeof(unsigned long long) + 16));
  status = (uint32_t*)(acc + 4);
  CV_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long) + 16, stream));
  for (uint64_t s0 = 0; s0 < n; s0 += kProfileChunk) {
    const uint64_t c = n - s0 < kProfileChunk ? n - s0 : kProfileChunk;
    Job job;
    CV_TRY(job.add(ctx, cfg, (const uint8_t*)image + s0 * kSector, c, 0, 0, false));
    CV_TRY(digest_job(ctx, cfg_i, (int)tab.sig, job, dig, nullptr, status, stream, tmp));
    const int threads = 256;
    const uint64_t want = (c + threads - 1) / threads;
    const int blocks = (int)(want < (uint64_t)ctx->sms * 8 ? want : (uint64_t)ctx->sms * 8);
    probe_profile_kernel<<<blocks, threads, 0, stream>>>(dig, c, s0, tab, acc);
    CV_CUDA(cudaGetLastError());
  }
  unsigned long long h[4];
  uint32_t stat = 0;
  CV_CUDA(cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, stream));
  CV_CUDA(cudaMemcpyAsync(&stat, status, 4, cudaMemcpyDeviceToHost, stream));
  CV_CUDA(cudaStreamSynchronize(stream));
  if (stat & kStTimeout) return CV_ETIMEOUT;
  if (stat) return CV_ECORRUPT;
  st->bloom_passed = h[0];
  st->slot_reads = h[1];
  st->key_reads = h[2];
  st->found = h[3];
  return CV_OK;
}

}  // extern "C"
