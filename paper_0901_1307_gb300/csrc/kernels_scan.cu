// Instantiations of the scan kernel (hash + probe + first compaction pass) and of the second
// compaction pass, one per tuned configuration.
#include "compact.cuh"
#include "cv_launch.h"
#include "scan_kernel.cuh"

namespace cvk {

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing completes. The
// wait gives up after timeout_ns, sets kStTimeout and the kernel returns normally.
__global__ void wait_timeout_selftest_kernel(uint32_t* status, uint64_t timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool ok = mbar_wait(smem_addr(&bar), 0, &abort_flag, status, timeout_ns);
    if (ok) atomicOr(status, kStProbeBound);  // must not happen: nothing arrives
  }
}


#define CV_KS(T, SPT, NS, B, MODE, P, MB, SIG) (const void*)scan_kernel<T, SPT, NS, B, MODE, P, MB, SIG, kLayoutHash>
#define CV_KSS(T, SPT, NS, B, P, MB, SIG) (const void*)scan_kernel<T, SPT, NS, B, kModeScan, P, MB, SIG, kLayoutSorted>

// A configuration with MD5 kernels for the hash layout only.
#define CV_SCAN_CFG(T, SPT, NS, B, P, MB)                                                                  \
  ScanCfg {                                                                                                \
    "t" #T "_x" #SPT "_s" #NS "_b" #B "_p" #P, T, SPT, T / SPT + 32, NS, B,                                 \
        {CV_KS(T, SPT, NS, B, kModeScan, P, MB, kSigMd5), nullptr, nullptr, nullptr,                       \
         nullptr, nullptr, nullptr, nullptr},                                                              \
        {CV_KS(T, SPT, NS, B, kModeDigest, P, MB, kSigMd5), nullptr, nullptr, nullptr},                    \
        (const void*)expand_kernel<T>, ScanSmem<T, NS, B>::kAlloc                                          \
  }

// A configuration with kernels for every signature and both table layouts.
#define CV_SCAN_CFG_ALL(T, SPT, NS, B, P, MB)                                                              \
  ScanCfg {                                                                                                \
    "t" #T "_x" #SPT "_s" #NS "_b" #B "_p" #P, T, SPT, T / SPT + 32, NS, B,                                 \
        {CV_KS(T, SPT, NS, B, kModeScan, P, MB, kSigMd5), CV_KS(T, SPT, NS, B, kModeScan, P, MB, kSigMd5NoPad), \
         CV_KS(T, SPT, NS, B, kModeScan, P, MB, kSigDjb2), CV_KS(T, SPT, NS, B, kModeScan, P, MB, kSigCrc64),   \
         CV_KSS(T, SPT, NS, B, P, MB, kSigMd5), CV_KSS(T, SPT, NS, B, P, MB, kSigMd5NoPad),                     \
         CV_KSS(T, SPT, NS, B, P, MB, kSigDjb2), CV_KSS(T, SPT, NS, B, P, MB, kSigCrc64)},                      \
        {CV_KS(T, SPT, NS, B, kModeDigest, P, MB, kSigMd5),                                                \
         CV_KS(T, SPT, NS, B, kModeDigest, P, MB, kSigMd5NoPad),                                           \
         CV_KS(T, SPT, NS, B, kModeDigest, P, MB, kSigDjb2),                                               \
         CV_KS(T, SPT, NS, B, kModeDigest, P, MB, kSigCrc64)},                                             \
        (const void*)expand_kernel<T>, ScanSmem<T, NS, B>::kAlloc                                          \
  }

// The first entry is the default configuration (the fastest measured on GB300 for the 32 GiB
// image workload) and the only one built for every signature and the sorted layout; the others
// stay selectable and are what the batch autotuner tries.
static const ScanCfg kConfigs[] = {
    CV_SCAN_CFG_ALL(256, 1, 2, 64, 3, 0),
    CV_SCAN_CFG(480, 1, 2, 64, 3, 3),
    CV_SCAN_CFG(256, 1, 2, 64, 0, 0),
    CV_SCAN_CFG(256, 1, 2, 64, 2, 0),
    CV_SCAN_CFG(256, 2, 2, 64, 3, 0),
    CV_SCAN_CFG(256, 2, 2, 128, 3, 0),
    CV_SCAN_CFG(256, 1, 3, 64, 3, 0),
    CV_SCAN_CFG(128, 1, 2, 128, 2, 0),
    CV_SCAN_CFG(128, 1, 4, 64, 0, 0),
};

const ScanCfg* scan_configs(int* n) {
  *n = (int)(sizeof(kConfigs) / sizeof(kConfigs[0]));
  return kConfigs;
}

const ScanCfg& scan_config_for(int cfg_i, int kind, int* used) {
  int n;
  const ScanCfg* c = scan_configs(&n);
  if (cfg_i < 0 || cfg_i >= n || kind < 0 || kind >= kTableKinds || !c[cfg_i].scan_fn[kind]) cfg_i = 0;
  if (used) *used = cfg_i;
  return c[cfg_i];
}

int launch_expand(const ScanCfg& cfg, const uint4* hit_rec, const uint32_t* tile_nhit, const uint64_t* tile_off,
                  uint64_t n_out_tiles, const Segment* segs, uint32_t n_segs, const TableView& tab, MatchOut* out,
                  uint64_t out_cap, uint32_t* status, int sms, void* stream) {
  const uint2* post = tab.postings;
  const uint8_t* confirm = sig_is_weak((int)tab.sig) ? tab.confirm : nullptr;
  uint64_t g = (n_out_tiles * 32 + 255) / 256;
  if (g > (uint64_t)sms * 16) g = (uint64_t)sms * 16;
  if (g == 0) g = 1;
  void* args[] = {&hit_rec, &tile_nhit, &tile_off, &n_out_tiles, &segs, &n_segs, &post, &out, &out_cap, &status,
                  &confirm};
  return (int)cudaLaunchKernel(cfg.expand_fn, dim3((unsigned)g), dim3(256), args, 0, (cudaStream_t)stream);
}

int launch_wait_selftest(uint32_t* status, uint64_t timeout_ns, void* stream) {
  wait_timeout_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(status, timeout_ns);
  return (int)cudaGetLastError();
}

uint64_t tile_offsets_scratch_words(uint64_t n_tiles) { return (n_tiles + kOffChunk - 1) / kOffChunk + 1; }

int launch_sum_u32(const uint32_t* v, uint64_t n, uint64_t* out, int sms, void* stream) {
  if (!n) return 0;
  const unsigned g = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 4);
  sum_u32_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(v, n, reinterpret_cast<unsigned long long*>(out));
  return (int)cudaGetLastError();
}

int launch_tile_offsets(const uint64_t* tile_ntrip, uint64_t n_tiles, uint64_t* tile_off, const Segment* segs,
                        uint32_t n_segs, uint32_t scale, uint64_t* seg_off, uint64_t* total, uint64_t* scratch,
                        void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  const uint64_t chunks = (n_tiles + kOffChunk - 1) / kOffChunk;
  if (chunks) chunk_sums_kernel<<<(unsigned)chunks, kOffThreads, 0, stream>>>(tile_ntrip, n_tiles, scratch);
  scan_sums_kernel<<<1, kOffThreads, 0, stream>>>(scratch, chunks, total);
  if (chunks) chunk_scan_kernel<<<(unsigned)chunks, kOffThreads, 0, stream>>>(tile_ntrip, n_tiles, scratch, tile_off);
  if (n_segs) segment_offsets_kernel<<<(n_segs + 255) / 256, 256, 0, stream>>>(tile_off, n_tiles, segs, n_segs, scale,
                                                                               total, seg_off);
  return (int)cudaGetLastError();
}

}  // namespace cvk
