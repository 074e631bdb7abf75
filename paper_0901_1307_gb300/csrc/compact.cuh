// Second pass of the match compaction: the per-tile triple counts of the scan are turned into
// output offsets by one exclusive scan, then every hit record of every tile is expanded into
// its (disk_sector, file_id, file_sector) triples. Tiles are in sector order, the records of a
// tile are in sector order (ballot ranks), and each digest's postings are sorted by
// (file_id, file_sector), so the output is sorted without a sort; the only waits between thread
// blocks are the offset scan's bounded look-back. (The paper's Section 3.2 writes matches to a
// host-visible buffer in no stated order; the sorted triple list is this library's output
// format.)
#pragma once
#include <stdint.h>

#include "cv_internal.h"

namespace cvk {

// Exclusive scan of the per-tile triple counts in one pass: each block scans a chunk and adds
// its predecessors' published sums (decoupled look-back, every wait bounded). A second small pass
// reads off each segment's first offset. (The kernels are in kernels_scan.cu; this header holds
// the expand pass, instantiated with each configuration.)
constexpr int kOffThreads = 1024;
constexpr int kOffItems = 4;
constexpr uint64_t kOffChunk = (uint64_t)kOffThreads * kOffItems;

// A warp takes 32 consecutive output tiles (32 sectors each) at a time. A hit record is {lane,
// post_off, post_cnt, n_emit}: the sector emits n_emit triples, all of its postings, or with a
// 64-bit signature (confirm != null) those whose master sector equals the disk sector byte for
// byte. The records of the group's tiles with hits are numbered in tile order and taken 32 at a
// time, one per lane, so that the dependent loads of different tiles (offset, record, posting)
// are in flight together: most tiles have no hit, and a tile's few hits would otherwise each
// wait in turn. A record's place in the output is its tile's offset plus the triples of the
// records before it in the tile (a segmented warp scan, carried across passes). out_cap bounds
// the writes (kStOverflow when exceeded). When the scan before it on the stream failed (a wait
// timed out or a lookup ran past the probe bound: its hit records are not to be trusted), the
// pass writes nothing.
template <int T>
__global__ void expand_kernel(const uint4* hit_rec, const uint32_t* tile_nhit, const uint64_t* tile_off,
                              uint64_t n_out_tiles, const Segment* segs, uint32_t n_segs, const uint2* postings,
                              MatchOut* out, uint64_t out_cap, uint32_t* status, const uint8_t* confirm) {
  if (*(volatile const uint32_t*)status & (kStTimeout | kStProbeBound | kStBadTable)) return;
  constexpr uint32_t kW = T / 32;
  constexpr uint32_t kFull = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t u0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; u0 < n_out_tiles;
       u0 += warps * 32) {
    // lane b describes tile u0 + b: its records, the first of them in the group's numbering,
    // its output offset, the image sector of its row 0 and (for confirmation) that row's bytes
    const uint64_t my_u = u0 + lane;
    const uint32_t my_n = my_u < n_out_tiles ? tile_nhit[my_u] : 0u;
    uint32_t incl = my_n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(kFull, incl, d);
      if (lane >= (uint32_t)d) incl += v;
    }
    const uint32_t n_rec = __shfl_sync(kFull, incl, 31);
    if (n_rec == 0u) continue;
    const uint32_t my_first = incl - my_n;
    uint64_t my_off = 0, my_sector = 0;
    const uint8_t* my_bytes = nullptr;
    if (my_n) {
      my_off = tile_off[my_u];
      const uint64_t ctile = my_u / kW;
      const Segment& sg = segs[find_segment(segs, n_segs, ctile)];
      const uint64_t row_first = (ctile - sg.tile_base) * T + (my_u % kW) * 32;  // within the segment
      my_sector = sg.sector_base + row_first;
      if (confirm) my_bytes = sg.bytes + row_first * kSector;
    }
    uint32_t carry = 0, carry_b = 32;  // triples of tile carry_b's records in earlier passes
    for (uint32_t q0 = 0; q0 < n_rec; q0 += 32) {
      const uint32_t q = q0 + lane;
      const bool act = q < n_rec;
      // the record's tile: the last lane b whose first record is at or before q
      uint32_t b = 0;
#pragma unroll
      for (uint32_t step = 16; step > 0; step >>= 1)
        if (__shfl_sync(kFull, my_first, b + step) <= q) b += step;
      const uint32_t i = q - __shfl_sync(kFull, my_first, b);
      const uint64_t off_b = __shfl_sync(kFull, my_off, b);
      const uint64_t sector_b = __shfl_sync(kFull, my_sector, b);
      const uint8_t* bytes_b =
          reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, reinterpret_cast<uintptr_t>(my_bytes), b));
      uint4 rec = make_uint4(0, 0, 0, 0);
      if (act) rec = hit_rec[(u0 + b) * 32 + i];
      // triples of the records before this one in its tile: a scan over the lanes of the same tile
      uint32_t sum = rec.w;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, sum, d);
        const uint32_t vb = __shfl_up_sync(kFull, b, d);
        if (lane >= (uint32_t)d && vb == b) sum += v;
      }
      const uint32_t before = sum - rec.w + (b == carry_b ? carry : 0u);
      const uint32_t last_b = __shfl_sync(kFull, b, 31);
      const uint32_t last_sum = __shfl_sync(kFull, sum, 31);
      carry = last_sum + (last_b == carry_b ? carry : 0u);
      carry_b = last_b;
      if (!act) continue;
      uint64_t o = off_b + before;
      const uint8_t* mine = confirm ? bytes_b + (uint64_t)rec.x * kSector : nullptr;
      for (uint32_t k = 0; k < rec.z; k++) {
        if (confirm && !sectors_equal(mine, confirm + (uint64_t)(rec.y + k) * kSector)) continue;
        if (o < out_cap) {
          const uint2 pf = postings[rec.y + k];
          out[o] = MatchOut{sector_b + rec.x, pf.x, pf.y};
        } else {
          atomicOr(status, kStOverflow);
        }
        o++;
      }
    }
  }
}

}  // namespace cvk
