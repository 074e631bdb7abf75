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
// small pass reads off each segment's first offset. No block waits on another.
constexpr int kOffThreads = 1024;
constexpr int kOffItems = 4;
constexpr uint64_t kOffChunk = (uint64_t)kOffThreads * kOffItems;

// Block-wide inclusive scan of one u64 per thread (1024 threads).
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t x, uint64_t* warp_buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t v = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += v;
  }
  if (lane == 31) warp_buf[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = warp_buf[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t v = __shfl_up_sync(0xFFFFFFFFu, w, d);
      if (lane >= d) w += v;
    }
    warp_buf[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  return x + (warp ? warp_buf[warp - 1] : 0ull);
}

__global__ void __launch_bounds__(kOffThreads) chunk_sums_kernel(const uint64_t* v, uint64_t n, uint64_t* sums) {
  __shared__ uint64_t wb[32];
  const uint64_t base = (uint64_t)blockIdx.x * kOffChunk;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kOffItems; k++) {
    const uint64_t i = base + (uint64_t)k * kOffThreads + threadIdx.x;
    if (i < n) s += v[i];
  }
  const uint64_t incl = block_inclusive_scan(s, wb);
  if (threadIdx.x == kOffThreads - 1) sums[blockIdx.x] = incl;
}

// In place: sums[0..m) -> exclusive offsets; *total = the sum of all.
__global__ void __launch_bounds__(kOffThreads) scan_sums_kernel(uint64_t* sums, uint64_t m, uint64_t* total) {
  __shared__ uint64_t wb[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t base = 0; base < m; base += kOffThreads) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t x = i < m ? sums[i] : 0ull;
    const uint64_t incl = block_inclusive_scan(x, wb);
    const uint64_t c = carry;
    if (i < m) sums[i] = c + incl - x;
    __syncthreads();
    if (threadIdx.x == kOffThreads - 1) carry = c + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kOffThreads) chunk_scan_kernel(const uint64_t* v, uint64_t n, const uint64_t* offs,
                                                                 uint64_t* out) {
  __shared__ uint64_t wb[32];
  const uint64_t first = (uint64_t)blockIdx.x * kOffChunk + (uint64_t)threadIdx.x * kOffItems;
  uint64_t x[kOffItems];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kOffItems; k++) {
    x[k] = (first + k < n) ? v[first + k] : 0ull;
    s += x[k];
  }
  uint64_t run = block_inclusive_scan(s, wb) - s + offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kOffItems; k++) {
    if (first + k < n) out[first + k] = run;
    run += x[k];
  }
}

// seg_off[s] = offset of the first output tile of segment s (output tiles per scan tile: scale).
__global__ void segment_offsets_kernel(const uint64_t* tile_off, uint64_t n, const Segment* segs, uint32_t n_segs,
                                       uint32_t scale, const uint64_t* total, uint64_t* seg_off) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_segs; s += gridDim.x * blockDim.x) {
    const uint64_t u = segs[s].tile_base * scale;
    seg_off[s] = u < n ? tile_off[u] : *total;
  }
}

// The sum of n u32 values added to *out: the disk sectors with at least one match, from the
// per-tile hit counts.
__global__ void sum_u32_kernel(const uint32_t* v, uint64_t n, unsigned long long* out) {
  unsigned long long s = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    s += v[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

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
