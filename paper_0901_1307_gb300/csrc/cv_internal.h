// Internal types shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cvk {

constexpr uint32_t kSector = 512;

// Device status word bits (set with atomicOr; read by the host after each launch).
constexpr uint32_t kStTimeout = 1u;     // an mbarrier wait ran out of time
constexpr uint32_t kStProbeBound = 2u;  // a lookup ran past the table's recorded probe bound
constexpr uint32_t kStTableFull = 4u;   // an insert found no free slot
constexpr uint32_t kStOverflow = 8u;    // an output buffer was too small
constexpr uint32_t kStBadTable = 16u;   // a loaded table's slot points outside its postings

// A contiguous run of whole sectors in device memory, scanned as one tensor map. An image
// larger than kMaxSegmentSectors is split into several segments.
constexpr uint64_t kMaxSegmentSectors = 1ull << 30;

struct Segment {
  uint64_t n_sectors;    // whole sectors in the segment
  uint64_t tile_base;    // global index of the segment's first tile
  uint64_t sector_base;  // index within its image of the segment's first sector
  uint64_t row_base;     // row of the segment's first sector in its tensor map
  uint32_t image;        // index of the image the segment belongs to
  uint32_t map;          // index of its tensor map within the job
  const uint8_t* bytes;  // device address of the segment's first sector (byte confirmation)
};

// Signature kinds (the values of CV_SIG_*).
enum : int { kSigMd5 = 0, kSigMd5NoPad = 1, kSigDjb2 = 2, kSigCrc64 = 3 };

__host__ __device__ constexpr bool sig_is_weak(int sig) { return sig == kSigDjb2 || sig == kSigCrc64; }

// Device view of a master table.
//   slots: 2 x uint4 per slot: {d0, d1, d2, d3} and {post_off, post_cnt, tau, 0}; post_cnt == 0
//          marks an empty slot. The home slot of digest d at position tau is
//          tau_home(d0, tau) & slot_mask, d0 & slot_mask when tau = 0 (Eq. 3).
//   postings: (file_id, file_sector) per kept master sector, grouped by slot, ascending.
//   bloom: 8 u32 words (32 bytes) per block; block tau_block(d3, tau) & bloom_mask; in word j the bit
//          (d1 >> 5j) & 31 for j < 6, (d2 >> 5(j-6)) & 31 for j = 6, 7.
//   confirm: for 64-bit signatures, the master sector bytes of posting q at confirm + 512 q.
//   sorted layout: slots holds n_keys records (no empty ones) in ascending order of
//          h0 = tau_home(d0, tau), and keys0[q] is record q's h0: a lookup is a binary search of
//          keys0 (the alternative to linear probing for high occupancy, Section 4), then a
//          comparison of the records whose h0 is equal.
enum : uint32_t { kLayoutHash = 0, kLayoutSorted = 1 };
// What a table's keys are: 512-byte sectors, or 64-byte fragments (a fragment table's Bloom
// filter is one u32 word per block, 3 bits per key: word d3 & bloom_mask, bits from d2).
enum : uint32_t { kUnitSector = 0, kUnitFragment = 1 };

struct TableView {
  const uint4* slots;
  const uint2* postings;
  const uint4* bloom;
  const uint8_t* confirm;
  const uint32_t* keys0;  // sorted layout only
  const uint32_t* frag_l1;  // fragment tables: the shared-memory filter (kFragL1Bytes)
  uint32_t slot_mask;
  uint32_t bloom_mask;
  uint32_t max_probe;  // hash: no stored digest sits further than max_probe - 1 slots from home
  uint32_t use_bloom;
  uint32_t sig;        // kSig* of the table
  uint32_t tau_mask;   // 7 for position-keyed tables (S_tau), 0 for one table over all positions
  uint32_t tau_add;    // (8 - base_offset mod 8) mod 8: disk sector g sits at position (g + tau_add) & 7
  uint32_t layout;     // kLayout*
  uint32_t n_keys;     // sorted layout: records in slots and keys0
  uint32_t unit;       // kUnitSector or kUnitFragment
};

// Position-keyed tables (Section 3.1: one table S_tau per sector position tau of an 8-sector
// cluster) are stored as one open-addressing table whose key is (signature, tau): tau moves the
// home slot and the Bloom block and is stored in the slot's third value word. tau = 0 leaves both
// unchanged, so a table over all positions is the same layout with every tau 0.
__host__ __device__ inline uint32_t tau_home(uint32_t d0, uint32_t tau) { return d0 ^ (tau * 0x9E3779B9u); }
__host__ __device__ inline uint32_t tau_block(uint32_t d3, uint32_t tau) { return d3 ^ (tau * 0x85EBCA6Bu); }

// The four table words of a 64-bit signature h: h itself (low word first, so the home slot is
// given by the signature's least significant bits, Eq. 3) and a SplitMix64-style finalizer of h
// that spreads it over the Bloom bits. Equal words <=> equal h.
__host__ __device__ inline void sig64_words(uint64_t h, uint32_t w[4]) {
  uint64_t z = h + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  w[0] = (uint32_t)h;
  w[1] = (uint32_t)(h >> 32);
  w[2] = (uint32_t)z;
  w[3] = (uint32_t)(z >> 32);
}

// Fragment workloads (Section 5): 64-byte windows at every 4-byte offset of an image against
// the whole 64-byte fragments of the master files.
constexpr uint32_t kFrag = 64;
constexpr uint32_t kFragStride = 4;
// The shared-memory filter of a fragment table: 2^20 bits (128 KiB), bit = top 20 bits of d1.
constexpr uint32_t kFragL1Log2Bits = 20;
constexpr uint32_t kFragL1Bytes = (1u << kFragL1Log2Bits) / 8;

// The four table words of a fragment's 64-bit signature h: h itself (low word first: the home
// slot is given by the signature's least significant bits, Eq. 3) and h times an odd constant,
// whose high bits (mixing every bit of h) choose the Bloom word and bits. Equal words <=> equal h.
__host__ __device__ inline void frag64_words(uint64_t h, uint32_t w[4]) {
  const uint64_t f = h * 0x9E3779B97F4A7C15ull;
  w[0] = (uint32_t)h;
  w[1] = (uint32_t)(h >> 32);
  w[2] = (uint32_t)f;
  w[3] = (uint32_t)(f >> 32);
}

// Byte-for-byte comparison of two device sectors (16-byte aligned).
__device__ inline bool sectors_equal(const uint8_t* a, const uint8_t* b) {
  const uint4* x = reinterpret_cast<const uint4*>(a);
  const uint4* y = reinterpret_cast<const uint4*>(b);
  uint32_t diff = 0;
#pragma unroll 4
  for (int k = 0; k < 32; k++) {
    const uint4 u = __ldg(x + k), v = __ldg(y + k);
    diff |= (u.x ^ v.x) | (u.y ^ v.y) | (u.z ^ v.z) | (u.w ^ v.w);
  }
  return diff == 0;
}

// Tensor maps one launch of the scan kernel can carry.
constexpr int kMapsPerLaunch = 64;

// Parameters of one scan-kernel launch, passed by value as a __grid_constant__ kernel
// parameter: the TMA unit reads the tensor maps straight from the parameter space, so no
// descriptor ever lives in (reused) global memory. Many segments may share one map (images
// placed side by side in one device allocation).
struct ScanParams {
  CUtensorMap maps[kMapsPerLaunch];  // the job's maps [map_base, map_base + kMapsPerLaunch)
  const Segment* segs;               // device: this launch's segments, sorted by tile_base
  uint32_t n_segs;
  uint32_t map_base;
  uint32_t one;         // always 1 (an opaque multiplier for the MD5 additions)
  uint32_t pad;
  uint64_t tile_begin;  // global index of the first tile of this launch
  uint64_t n_tiles;     // tiles of this launch
  TableView tab;
  // scan outputs, indexed by global output tile (32 sectors)
  uint4* hit_rec;        // 32 records per output tile {lane, post_off, post_cnt, triples emitted}
  uint32_t* tile_nhit;   // hit sectors per output tile
  uint64_t* tile_ntrip;  // triples per output tile
  uint32_t* status;
  // digest outputs (digest mode): indexed by segment sector_base + row
  uint4* digests;
  uint8_t* trivial;
  // 64-bit signatures: candidates (disk sector, posting) whose signatures are equal and whose
  // bytes differ are added here; null: not counted
  unsigned long long* rejected;
};

// One output triple (the layout of cv_match).
struct MatchOut {
  uint64_t disk_sector;
  uint32_t file_id;
  uint32_t file_sector;
};

// Index of the segment holding global tile `tile` (segments sorted by tile_base).
__device__ __forceinline__ uint32_t find_segment(const Segment* segs, uint32_t n, uint64_t tile) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (segs[mid].tile_base <= tile) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace cvk
