// Scan kernel configurations, part a: the default configuration first (256-sector tiles, one
// sector per thread, two 64-byte ring stages, two of three MD5 operations adding on the FMA pipe,
// register allocation bounded for four resident blocks per SM: with the stage loop unrolled in
// fours, 48 registers and 32 hashing warps per SM measured 0.75% faster than 40 registers and 40
// warps, 1.5% for MD5 without padding; hash tables whose lookups walk long probe runs, at 75-90%
// occupancy without a filter, lose 9-17%, and the automatic layout takes the sorted one there),
// then 480-sector tiles and the all-ALU pipe split.
#include "scan_cfg_inst.cuh"

namespace cvk {

const ScanCfg* scan_cfgs_a(int* n) {
  static const ScanCfg c[] = {
    CV_SCAN_CFG_DIGEST(256, 1, 2, 64, 3, 4),
    CV_SCAN_CFG(480, 1, 2, 64, 3, 3),
    CV_SCAN_CFG(256, 1, 2, 64, 0, 0),
  };
  *n = (int)(sizeof(c) / sizeof(c[0]));
  return c;
}

}  // namespace cvk
