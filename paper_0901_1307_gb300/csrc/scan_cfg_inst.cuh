// Instantiation of one scan configuration: its scan kernels for all eight table kinds (four
// signatures x hash and sorted layouts), optionally its digest-mode kernels, and the matching
// second compaction pass. Included by the scan_cfgs_*.cu units only.
#pragma once
#include "compact.cuh"
#include "cv_launch.h"
#include "scan_kernel.cuh"

#define CV_KS(T, SPT, NS, B, MODE, P, MB, SIG) \
  (const void*)::cvk::scan_kernel<T, SPT, NS, B, MODE, P, MB, SIG, ::cvk::kLayoutHash>
#define CV_KSS(T, SPT, NS, B, P, MB, SIG) \
  (const void*)::cvk::scan_kernel<T, SPT, NS, B, ::cvk::kModeScan, P, MB, SIG, ::cvk::kLayoutSorted>

#define CV_SCAN_KINDS(T, SPT, NS, B, P, MB)                                                                   \
  {CV_KS(T, SPT, NS, B, ::cvk::kModeScan, P, MB, ::cvk::kSigMd5),                                           \
   CV_KS(T, SPT, NS, B, ::cvk::kModeScan, P, MB, ::cvk::kSigMd5NoPad),                                      \
   CV_KS(T, SPT, NS, B, ::cvk::kModeScan, P, MB, ::cvk::kSigDjb2),                                          \
   CV_KS(T, SPT, NS, B, ::cvk::kModeScan, P, MB, ::cvk::kSigCrc64),                                         \
   CV_KSS(T, SPT, NS, B, P, MB, ::cvk::kSigMd5), CV_KSS(T, SPT, NS, B, P, MB, ::cvk::kSigMd5NoPad),          \
   CV_KSS(T, SPT, NS, B, P, MB, ::cvk::kSigDjb2), CV_KSS(T, SPT, NS, B, P, MB, ::cvk::kSigCrc64)}

// A configuration with scan kernels for every table kind and no digest-mode kernels.
#define CV_SCAN_CFG(T, SPT, NS, B, P, MB)                                                      \
  ::cvk::ScanCfg {                                                                             \
    "t" #T "_x" #SPT "_s" #NS "_b" #B "_p" #P, T, SPT, T / SPT + 32, NS, B,                   \
        CV_SCAN_KINDS(T, SPT, NS, B, P, MB), {nullptr, nullptr, nullptr, nullptr},           \
        (const void*)::cvk::expand_kernel<T>, ::cvk::ScanSmem<T, NS, B>::kAlloc              \
  }

// The same with digest-mode kernels for every signature (table builds, cv_sector_signatures).
#define CV_SCAN_CFG_DIGEST(T, SPT, NS, B, P, MB)                                               \
  ::cvk::ScanCfg {                                                                             \
    "t" #T "_x" #SPT "_s" #NS "_b" #B "_p" #P, T, SPT, T / SPT + 32, NS, B,                   \
        CV_SCAN_KINDS(T, SPT, NS, B, P, MB),                                                   \
        {CV_KS(T, SPT, NS, B, ::cvk::kModeDigest, P, MB, ::cvk::kSigMd5),                      \
         CV_KS(T, SPT, NS, B, ::cvk::kModeDigest, P, MB, ::cvk::kSigMd5NoPad),                 \
         CV_KS(T, SPT, NS, B, ::cvk::kModeDigest, P, MB, ::cvk::kSigDjb2),                     \
         CV_KS(T, SPT, NS, B, ::cvk::kModeDigest, P, MB, ::cvk::kSigCrc64)},                   \
        (const void*)::cvk::expand_kernel<T>, ::cvk::ScanSmem<T, NS, B>::kAlloc              \
  }
