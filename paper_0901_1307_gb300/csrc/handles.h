// Handle objects of the C ABI, shared by the translation units that implement it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "cv.h"
#include "cv_internal.h"
#include "runtime.h"

namespace cvk {
constexpr uint32_t kMagicMaster = 0xC7A57E01u;
constexpr uint32_t kMagicResult = 0xC7A57E02u;

// Digests (and exclusion flags) of the job's sectors, written by the scan kernel in digest mode.
int digest_job(DevCtx* ctx, int cfg_i, int sig, Job& job, uint4* digests, uint8_t* trivial, uint32_t* status,
               cudaStream_t stream, Temps& tmp);
}  // namespace cvk

struct cv_master {
  uint32_t magic;
  int dev;
  cvk::TableView tab;
  void* slots;
  void* postings;
  void* bloom;
  void* confirm;  // kept master units in posting order (64-bit signatures)
  void* keys0;    // sorted layout: h0 of every record
  void* frag_l1;  // fragment tables: the shared-memory filter
  cv_master_info info;
  // Matches of the last sector scan against this table (read and written atomically): the
  // next scan launches its expand pass with room for a quarter more, without waiting for the
  // exact count first.
  uint64_t last_matches;
};

struct cv_result {
  uint32_t magic;
  int dev;
  bool on_device;
  uint32_t n_images;
  std::vector<uint64_t> off;  // n_images + 1
  cvk::MatchOut* host;
  cvk::MatchOut* dev_out;     // from the library's pool, released on free_stream
  cudaStream_t free_stream;
  cv_scan_stats st;
  int launches;               // kernel launches of the scan
};
