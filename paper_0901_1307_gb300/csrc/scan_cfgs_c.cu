// Scan kernel configurations, part c: deeper rings (three and four stages) and 128-sector tiles.
#include "scan_cfg_inst.cuh"

namespace cvk {

const ScanCfg* scan_cfgs_c(int* n) {
  static const ScanCfg c[] = {
    CV_SCAN_CFG(256, 1, 3, 64, 3, 0),
    CV_SCAN_CFG(128, 1, 2, 128, 2, 0),
    CV_SCAN_CFG(128, 1, 4, 64, 0, 0),
  };
  *n = (int)(sizeof(c) / sizeof(c[0]));
  return c;
}

}  // namespace cvk
