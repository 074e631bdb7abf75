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

constexpr int kScanThreads = 1024;

// Exclusive scan of tile_ntrip[0..n) into tile_off, the grand total into *total, and the
// offset of every segment's first tile into seg_off[0..n_segs) (one block of 1024 threads).
__global__ void __launch_bounds__(kScanThreads) tile_offsets_kernel(const uint64_t* tile_ntrip, uint64_t n,
                                                                    uint64_t* tile_off, const Segment* segs,
                                                                    uint32_t n_segs, uint64_t* seg_off,
                                                                    uint64_t* total) {
  __shared__ uint64_t warp_sum[kScanThreads / 32];
  __shared__ uint64_t carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t per = (n + kScanThreads - 1) / kScanThreads;
  const uint64_t lo = per * tid < n ? per * tid : n;
  const uint64_t hi = lo + per < n ? lo + per : n;
  uint64_t sum = 0;
  for (uint64_t i = lo; i < hi; i++) sum += tile_ntrip[i];
  // block-wide exclusive scan of the per-thread sums
  uint64_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = warp_sum[lane];
    uint64_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t v = __shfl_up_sync(0xFFFFFFFFu, wi, d);
      if (lane >= d) wi += v;
    }
    warp_sum[lane] = wi - w;
    if (lane == 31) carry = wi;
  }
  __syncthreads();
  uint64_t run = warp_sum[warp] + incl - sum;
  for (uint64_t i = lo; i < hi; i++) {
    tile_off[i] = run;
    run += tile_ntrip[i];
  }
  __syncthreads();
  if (tid == 0) *total = carry;
  for (uint32_t s = tid; s < n_segs; s += kScanThreads) seg_off[s] = segs[s].tile_base < n ? tile_off[segs[s].tile_base] : carry;
}

// One warp per tile with hits. out_cap bounds the writes (kStOverflow when exceeded).
template <int T>
__global__ void expand_kernel(const uint4* hit_rec, const uint32_t* tile_nhit, const uint64_t* tile_off,
                              uint64_t n_tiles, const Segment* segs, uint32_t n_segs, const uint2* postings,
                              MatchOut* out, uint64_t out_cap, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < n_tiles;
       tile += warps) {
    const uint32_t n = tile_nhit[tile];
    if (n == 0) continue;
    const uint32_t sg = find_segment(segs, n_segs, tile);
    const uint64_t first_sector = segs[sg].sector_base + (tile - segs[sg].tile_base) * T;
    uint64_t pos = tile_off[tile];
    for (uint32_t h0 = 0; h0 < n; h0 += 32) {
      const uint32_t h = h0 + lane;
      uint4 rec = make_uint4(0, 0, 0, 0);
      if (h < n) rec = hit_rec[tile * T + h];
      uint32_t incl = rec.z;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
      }
      const uint64_t my = pos + (incl - rec.z);
      for (uint32_t k = 0; k < rec.z; k++) {
        const uint64_t o = my + k;
        if (o < out_cap) {
          const uint2 pf = postings[rec.y + k];
          out[o] = MatchOut{first_sector + rec.x, pf.x, pf.y};
        } else {
          atomicOr(status, kStOverflow);
        }
      }
      pos += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
  }
}

}  // namespace cvk
