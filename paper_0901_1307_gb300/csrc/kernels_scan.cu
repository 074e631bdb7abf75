// Instantiations of the scan kernel (hash + probe + first compaction pass) and of the second
// compaction pass, one per tuned configuration.
#include "compact.cuh"
#include "cv_launch.h"
#include "scan_kernel.cuh"

namespace cvk {

#define CV_SCAN_CFG(T, NS, B)                                                                              \
  ScanCfg {                                                                                                \
    "t" #T "_s" #NS "_b" #B, T, NS, B, (const void*)scan_kernel<T, NS, B, kModeScan>,                       \
        (const void*)scan_kernel<T, NS, B, kModeDigest>, (const void*)expand_kernel<T>,                    \
        ScanSmem<T, NS, B>::kAlloc                                                                         \
  }

static const ScanCfg kConfigs[] = {
    CV_SCAN_CFG(128, 4, 64),
    CV_SCAN_CFG(128, 2, 128),
    CV_SCAN_CFG(256, 3, 64),
    CV_SCAN_CFG(64, 6, 64),
    CV_SCAN_CFG(128, 3, 128),
};

const ScanCfg* scan_configs(int* n) {
  *n = (int)(sizeof(kConfigs) / sizeof(kConfigs[0]));
  return kConfigs;
}

uint64_t tile_offsets_scratch_words(uint64_t n_tiles) { return (n_tiles + kOffChunk - 1) / kOffChunk + 1; }

int launch_tile_offsets(const uint64_t* tile_ntrip, uint64_t n_tiles, uint64_t* tile_off, const Segment* segs,
                        uint32_t n_segs, uint64_t* seg_off, uint64_t* total, uint64_t* scratch, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  const uint64_t chunks = (n_tiles + kOffChunk - 1) / kOffChunk;
  if (chunks) chunk_sums_kernel<<<(unsigned)chunks, kOffThreads, 0, stream>>>(tile_ntrip, n_tiles, scratch);
  scan_sums_kernel<<<1, kOffThreads, 0, stream>>>(scratch, chunks, total);
  if (chunks) chunk_scan_kernel<<<(unsigned)chunks, kOffThreads, 0, stream>>>(tile_ntrip, n_tiles, scratch, tile_off);
  if (n_segs) segment_offsets_kernel<<<(n_segs + 255) / 256, 256, 0, stream>>>(tile_off, n_tiles, segs, n_segs, total,
                                                                               seg_off);
  return (int)cudaGetLastError();
}

}  // namespace cvk
