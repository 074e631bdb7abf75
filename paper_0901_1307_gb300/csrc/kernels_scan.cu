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

const void* tile_offsets_fn() { return (const void*)tile_offsets_kernel; }

}  // namespace cvk
