// Second pass of the match compaction: the per-tile triple counts of the scan are turned into
// output offsets by one exclusive scan, then every hit record of every tile is expanded into
// its (disk_sector, file_id, file_sector) triples. Tiles are in sector order, the records of a
// tile are in sector order (ballot ranks), and each digest's postings are sorted by
// (file_id, file_sector), so the output is sorted without a sort and without any wait between
// thread blocks. (The paper's Section 3.2 writes matches to a host-visible buffer in no stated
// order; the sorted triple list is this library's output format.)
#pragma once
#include <stdint.h>

#include "cv_internal.h"

namespace cvk {

// Exclusive scan of the per-tile triple counts in three coalesced passes: chunk sums, a scan
// of the chunk sums (one block), and the scan within each chunk plus its chunk offset. A fourth
// small pass reads off each segment's first offset. No block waits on another. (The kernels are
// in kernels_scan.cu; this header holds the expand pass, instantiated with each configuration.)
constexpr int kOffThreads = 1024;
constexpr int kOffItems = 4;
constexpr uint64_t kOffChunk = (uint64_t)kOffThreads * kOffItems;

// One warp per output tile (32 consecutive sectors) with hits. A hit record is {lane, post_off,
// post_cnt, n_emit}: the sector emits n_emit triples, all of its postings, or with a 64-bit
// signature (confirm != null) those whose master sector equals the disk sector byte for byte.
// out_cap bounds the writes (kStOverflow when exceeded). When the scan before it on the stream
// failed (a wait timed out or a lookup ran past the probe bound: its hit records are not to be
// trusted), the pass writes nothing.
template <int T>
__global__ void expand_kernel(const uint4* hit_rec, const uint32_t* tile_nhit, const uint64_t* tile_off,
                              uint64_t n_out_tiles, const Segment* segs, uint32_t n_segs, const uint2* postings,
                              MatchOut* out, uint64_t out_cap, uint32_t* status, const uint8_t* confirm) {
  if (*(volatile const uint32_t*)status & (kStTimeout | kStProbeBound | kStBadTable)) return;
  constexpr uint32_t kW = T / 32;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  // A warp reads the hit counts of 32 output tiles at once and expands only those with hits:
  // most tiles have none, and one dependent count load per tile made the pass latency-bound.
  for (uint64_t u0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; u0 < n_out_tiles;
       u0 += warps * 32) {
    const uint32_t mine_n = u0 + lane < n_out_tiles ? tile_nhit[u0 + lane] : 0u;
    uint32_t busy = __ballot_sync(0xFFFFFFFFu, mine_n != 0u);
    while (busy) {
      const int b = __ffs(busy) - 1;
      busy &= busy - 1;
      const uint64_t u = u0 + (uint64_t)b;
      const uint32_t n = __shfl_sync(0xFFFFFFFFu, mine_n, b);
      const uint64_t ctile = u / kW;
      const uint32_t sg = find_segment(segs, n_segs, ctile);
      const uint64_t row_first = (ctile - segs[sg].tile_base) * T + (u % kW) * 32;  // within the segment
      const uint64_t first_sector = segs[sg].sector_base + row_first;
      uint4 rec = make_uint4(0, 0, 0, 0);
      if ((uint32_t)lane < n) rec = hit_rec[u * 32 + lane];
      uint32_t incl = rec.w;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
      }
      uint64_t o = tile_off[u] + (incl - rec.w);
      const uint8_t* mine = confirm ? segs[sg].bytes + (row_first + rec.x) * kSector : nullptr;
      for (uint32_t k = 0; k < rec.z; k++) {
        if (confirm && !sectors_equal(mine, confirm + (uint64_t)(rec.y + k) * kSector)) continue;
        if (o < out_cap) {
          const uint2 pf = postings[rec.y + k];
          out[o] = MatchOut{first_sector + rec.x, pf.x, pf.y};
        } else {
          atomicOr(status, kStOverflow);
        }
        o++;
      }
    }
  }
}

}  // namespace cvk
