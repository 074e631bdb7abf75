// Kernel configurations of the scan, exported by kernels_scan.cu to the host runtime.
#pragma once
#include <stdint.h>

#include "cv_internal.h"

namespace cvk {

struct ScanCfg {
  const char* name;
  int T;        // sectors per tile; T / 32 output tiles per tile
  int SPT;      // sectors per hashing thread
  int threads;  // block size: T / SPT hashing threads + one producer warp
  int NS;       // shared-memory ring stages
  int BOXB;   // bytes of each sector row per stage (64 or 128)
  const void* scan_fn[8];    // scan_kernel per table kind (table_kind); null: not built for it
  const void* digest_fn[4];  // digest mode, per signature (kSig*)
  const void* expand_fn;     // expand_kernel<T>
  uint32_t smem;             // dynamic shared memory bytes
};

const ScanCfg* scan_configs(int* n);
// The configurations of each instantiation unit, in table order (scan_cfgs_{a,b,c}.cu).
const ScanCfg* scan_cfgs_a(int* n);
const ScanCfg* scan_cfgs_b(int* n);
const ScanCfg* scan_cfgs_c(int* n);

// Scan kernels are selected by signature and table layout: kind = sig + 4 * layout.
constexpr int kTableKinds = 8;
inline int table_kind(const TableView& t) { return (int)t.sig + 4 * (int)t.layout; }

// Configuration cfg_i if it has a scan kernel for table kind `kind` (table_kind), else the
// default one (index 0, which has every kind); *used receives the index in use.
const ScanCfg& scan_config_for(int cfg_i, int kind, int* used);
// The default scan configuration for a table kind (the fastest measured for its signature).
int preferred_config(int kind);
// Configuration cfg_i if it has a digest-mode kernel for signature sig, else the default one.
const ScanCfg& digest_config_for(int cfg_i, int sig, int* used);

// The expand pass over n_out_tiles output tiles (see expand_kernel). Returns a CUDA error code.
int launch_expand(const ScanCfg& cfg, const uint4* hit_rec, const uint32_t* tile_nhit, const uint64_t* tile_off,
                  uint64_t n_out_tiles, const Segment* segs, uint32_t n_segs, const TableView& tab, MatchOut* out,
                  uint64_t out_cap, uint32_t* status, int sms, void* stream);


// Scratch (u64 words) the offset pass needs for n tiles.
uint64_t tile_offsets_scratch_words(uint64_t n_tiles);

// tile_off[i] = sum of tile_ntrip[0..i) over the n_tiles output tiles; *total = sum of all;
// seg_off[s] = offset of segment s's first output tile (segment tile_base * scale). scratch:
// tile_offsets_scratch_words(n_tiles) u64 words. status: the scan's status word (kStTimeout if
// a wait of the pass gives up). With tile_nhit, the sum of the n_tiles hit counts is added to
// *nhit_sum (device memory, zeroed by the caller). Returns a CUDA error code.
int launch_tile_offsets(const uint64_t* tile_ntrip, uint64_t n_tiles, uint64_t* tile_off, const Segment* segs,
                        uint32_t n_segs, uint32_t scale, uint64_t* seg_off, uint64_t* total, uint64_t* scratch,
                        void* stream, uint32_t* status, const uint32_t* tile_nhit = nullptr,
                        uint64_t* nhit_sum = nullptr);

// ---------------------------------------------------------------- fragment scans (Section 5)
uint64_t frag_windows(uint64_t n_bytes);       // 64-byte windows at 4-byte offsets in n_bytes
uint64_t frag_tiles(int sig, uint64_t n_bytes);  // tiles of sig's fragment kernels over those windows
bool frag_sig_supported(int sig);         // MD5, MD5 without padding, djb2-64

// Key words and exclusion flags of n master fragments at arena (64 bytes each, 16-byte aligned).
int frag_digests(int sig, const uint8_t* arena, uint64_t n, uint4* dig, uint8_t* trivial, int sms, void* stream);
// The filters of a fragment table (zeroed by the caller): the one-word Bloom filter (words, null
// for none; mask = words - 1) and the shared-memory filter l1 (kFragL1Bytes).
int frag_bloom(const uint4* slots, uint32_t n_slots, uint32_t* words, uint32_t mask, uint32_t* l1, int sms,
               void* stream);
// Triples per tile of one device image (16-byte aligned) into tile_ntrip[tile_base ..);
// djb2 candidates dropped by the byte comparison are added to *rejected (when non-null).
int frag_count(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base, uint64_t* tile_ntrip,
               uint32_t* status, unsigned long long* rejected, int sms, void* stream);
// The 16-byte key of every 64-byte window at a 4-byte offset of a device image, through the
// fragment kernels' own signature code (MD5, MD5 without padding, rolled djb2-64).
int frag_window_sigs(int sig, const uint8_t* image, uint64_t n_bytes, uint4* out, int sms, void* stream);
// The triples of the image's tiles that have any, at out[tile_off[tile]..]. list: scratch of
// frag_tiles(n_bytes) + 1 u32 words. *launches counts the kernels launched.
int frag_emit(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base,
              const uint64_t* tile_ntrip, const uint64_t* tile_off, uint32_t* list, MatchOut* out, uint64_t out_cap,
              uint32_t* status, int sms, void* stream, int* launches);

// One block whose single waiting thread waits on an mbarrier nothing completes (bounded by
// timeout_ns): the status word gets the timeout bit. Returns a CUDA error code.
// The offset scan's look-back wait running out (words: lookback_selftest_words() u64).
int launch_lookback_selftest(uint64_t* words, uint32_t* status, uint64_t timeout_ns, void* stream);
constexpr uint64_t lookback_selftest_words() { return 4 * 4096 + 4; }

int launch_wait_selftest(uint32_t* status, uint64_t timeout_ns, void* stream);

}  // namespace cvk
