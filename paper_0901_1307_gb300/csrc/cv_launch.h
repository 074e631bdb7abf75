// Kernel configurations of the scan, exported by kernels_scan.cu to the host runtime.
#pragma once
#include <stdint.h>

namespace cvk {

struct ScanCfg {
  const char* name;
  int T;      // sectors per tile = hashing threads per block (block = T + 32)
  int NS;     // shared-memory ring stages
  int BOXB;   // bytes of each sector row per stage (64 or 128)
  const void* scan_fn;    // scan_kernel<T, NS, BOXB, kModeScan>
  const void* digest_fn;  // scan_kernel<T, NS, BOXB, kModeDigest>
  const void* expand_fn;  // expand_kernel<T>
  uint32_t smem;          // dynamic shared memory bytes
};

const ScanCfg* scan_configs(int* n);
const void* tile_offsets_fn();

}  // namespace cvk
