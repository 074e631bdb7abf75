// Scan kernel configurations, part b: every other MD5 operation on the FMA pipe, and two sectors per thread (64- and 128-byte
// stages).
#include "scan_cfg_inst.cuh"

namespace cvk {

const ScanCfg* scan_cfgs_b(int* n) {
  static const ScanCfg c[] = {
    CV_SCAN_CFG(256, 1, 2, 64, 2, 0),
    CV_SCAN_CFG(256, 2, 2, 64, 3, 0),
    CV_SCAN_CFG(256, 2, 2, 128, 3, 0),
  };
  *n = (int)(sizeof(c) / sizeof(c[0]));
  return c;
}

}  // namespace cvk
