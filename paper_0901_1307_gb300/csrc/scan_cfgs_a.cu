// Scan kernel configurations, part a: the default configuration first (256-sector tiles, one
// sector per thread, two 64-byte ring stages, two of three MD5 operations adding on the FMA pipe,
// register allocation bounded for five resident blocks per SM: 0.6% faster than unbounded), then
// 480-sector tiles and the all-ALU pipe split.
#include "scan_cfg_inst.cuh"

namespace cvk {

const ScanCfg* scan_cfgs_a(int* n) {
  static const ScanCfg c[] = {
    CV_SCAN_CFG_DIGEST(256, 1, 2, 64, 3, 5),
    CV_SCAN_CFG(480, 1, 2, 64, 3, 3),
    CV_SCAN_CFG(256, 1, 2, 64, 0, 0),
  };
  *n = (int)(sizeof(c) / sizeof(c[0]));
  return c;
}

}  // namespace cvk
