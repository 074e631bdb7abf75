// Device kernels that build the master signature table (paper Section 3.1: every master
// sector's signature is inserted at the slot given by its low bits, collisions resolved by
// linear probing, Eq. 3).
//
// Steps (one launch each):
//   insert   one thread per master sector: claim the first free slot from the digest's home
//            slot on (atomicCAS of an owner word), or join the slot that already holds an
//            equal digest; record the slot, count its members, track the longest probe run.
//   sort     stable LSD radix sort of (slot, master index) pairs by slot, so every slot's
//            members end up contiguous and in master order, i.e. by (file_id, file_sector).
//   fill     the sorted pairs become the postings; the first pair of each run writes its
//            slot {digest, post_off, post_cnt}.
//   bloom    every occupied slot sets its 8 bits in the blocked Bloom filter.
//   sorted   (sorted layout only) the occupied slots, compacted in slot order, are sorted by
//            h0 and become the searched array.
// Position-keyed tables (one S_tau per cluster position, Section 3.1) key every slot by
// (digest, tau) with tau = file_sector mod 8; the steps are the same.
// Which slot a digest lands in depends on thread timing; the lookup result does not.
#pragma once
#include <stdint.h>

#include "cv_internal.h"

namespace cvk {

// Position of every master sector in its file's clusters: tau[m] = file_sector mod 8, the
// file found by binary search of file_base (n_files + 1 entries: first master index of every
// file, then the total).
__global__ void tau_kernel(const uint64_t* file_base, uint32_t n_files, uint64_t n, uint8_t* tau) {
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_files;  // largest f with file_base[f] <= m
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (file_base[mid] <= m) lo = mid; else hi = mid;
    }
    tau[m] = (uint8_t)((m - file_base[lo]) & 7u);
  }
}

// tau: per master sector position (position-keyed tables), or null for one table over all
// positions (every tau 0). The key is (digest, tau).
__global__ void insert_kernel(const uint4* dig, const uint8_t* trivial, const uint8_t* tau, uint64_t n,
                              uint32_t* owner, uint32_t* cnt, uint32_t* slot_of, uint32_t mask, uint32_t* max_disp,
                              uint32_t* n_kept, uint32_t* status) {
  const uint32_t none = mask + 1u;
  uint32_t kept = 0, longest = 0;  // this thread's, added to the shared counters once per warp
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (uint64_t)gridDim.x * blockDim.x) {
    if (trivial[m]) {
      slot_of[m] = none;
      continue;
    }
    const uint4 d = dig[m];
    const uint32_t t = tau ? tau[m] : 0u;
    uint32_t idx = tau_home(d.x, t) & mask;
    uint32_t c = 0;
    bool placed = false;
    for (; c <= mask; c++) {
      const uint32_t prev = atomicCAS(owner + idx, 0u, (uint32_t)m + 1u);
      if (prev == 0u) {
        placed = true;
        break;
      }
      const uint4 e = dig[prev - 1u];
      const uint32_t te = tau ? tau[prev - 1u] : 0u;
      if (e.x == d.x && e.y == d.y && e.z == d.z && e.w == d.w && te == t) {
        placed = true;
        break;
      }
      idx = (idx + 1u) & mask;
    }
    if (!placed) {
      atomicOr(status, kStTableFull);
      slot_of[m] = none;
      continue;
    }
    slot_of[m] = idx;
    atomicAdd(cnt + idx, 1u);
    longest = c > longest ? c : longest;
    kept++;
  }
  // one update per warp: a per-key atomic on one address serialises the whole build
  kept = __reduce_add_sync(0xFFFFFFFFu, kept);
  longest = __reduce_max_sync(0xFFFFFFFFu, longest);
  if ((threadIdx.x & 31) == 0 && kept) {
    atomicAdd(n_kept, kept);
    atomicMax(max_disp, longest);
  }
}

__global__ void iota_kernel(uint32_t* v, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ stable radix sort pass
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsChunk = kRsThreads * kRsRounds;

// Digit histogram of each 4096-key chunk: hist[digit * n_blocks + block].
__global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const uint32_t* keys, uint64_t n, int shift,
                                                             uint32_t* hist, uint32_t n_blocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kRsChunk;
  for (int r = 0; r < kRsRounds; r++) {
    const uint64_t i = base + (uint64_t)r * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(h + ((keys[i] >> shift) & 255u), 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * n_blocks + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of n u32 values whose total fits in 32 bits, over the whole GPU in
// three launches: the sum of every 4096-value chunk; an exclusive scan of those sums (one
// block); each chunk's own scan, offset by its sum's prefix. Loads and stores are coalesced;
// the per-thread runs are read from a padded shared tile without bank conflicts.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr uint32_t kScanChunk = kScanThreads * kScanItems;

// Exclusive scan of x over the B threads of a block; *total gets the sum (every thread).
template <int B>
__device__ __forceinline__ uint32_t block_exclusive_u32(uint32_t x, uint32_t* total) {
  __shared__ uint32_t ws[B / 32 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < B / 32 ? ws[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < B / 32) ws[lane] = wi - w;
    if (lane == B / 32 - 1) ws[B / 32] = wi;
  }
  __syncthreads();
  const uint32_t r = ws[warp] + incl - x;
  *total = ws[B / 32];
  __syncthreads();  // ws may be reused by the next call
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_chunk_sums_u32_kernel(const uint32_t* v, uint64_t n,
                                                                           uint32_t* sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    const uint64_t i = base + (uint64_t)r * kScanThreads + threadIdx.x;
    if (i < n) s += v[i];
  }
  uint32_t total;
  block_exclusive_u32<kScanThreads>(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_sums_u32_kernel(uint32_t* sums, uint32_t nb) {
  uint32_t carry = 0;
  for (uint32_t t0 = 0; t0 < nb; t0 += 1024) {
    const uint32_t i = t0 + threadIdx.x;
    const uint32_t x = i < nb ? sums[i] : 0u;
    uint32_t total;
    const uint32_t e = block_exclusive_u32<1024>(x, &total);
    if (i < nb) sums[i] = carry + e;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_chunks_u32_kernel(uint32_t* v, uint64_t n, const uint32_t* sums) {
  __shared__ uint32_t tile[kScanChunk + kScanChunk / 32];  // element e at e + e / 32
  const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    const uint32_t e = r * kScanThreads + tid;
    const uint64_t i = base + e;
    tile[e + e / 32] = i < n ? v[i] : 0u;
  }
  __syncthreads();
  uint32_t loc[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    const uint32_t e = tid * kScanItems + j;
    loc[j] = tile[e + e / 32];
    s += loc[j];
  }
  uint32_t total;
  uint32_t run = block_exclusive_u32<kScanThreads>(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    const uint32_t e = tid * kScanItems + j;
    tile[e + e / 32] = run;
    run += loc[j];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    const uint32_t e = r * kScanThreads + tid;
    const uint64_t i = base + e;
    if (i < n) v[i] = tile[e + e / 32];
  }
}

// Scatter of one pass: the keys of a chunk go, in their original order within each digit, to
// the chunk's offset for that digit (hist, after the scan).
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(const uint32_t* kin, const uint32_t* vin,
                                                                uint32_t* kout, uint32_t* vout, uint64_t n, int shift,
                                                                const uint32_t* hist, uint32_t n_blocks) {
  constexpr int kWarps = kRsThreads / 32;
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kWarps][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lane_lt = (1u << lane) - 1u;
  run[tid] = hist[(uint64_t)tid * n_blocks + blockIdx.x];
  const uint64_t base = (uint64_t)blockIdx.x * kRsChunk;
  for (int r = 0; r < kRsRounds; r++) {
#pragma unroll
    for (int w = 0; w < kWarps; w++) wcnt[w][tid] = 0;
    __syncthreads();
    const uint64_t i = base + (uint64_t)r * kRsThreads + tid;
    const bool valid = i < n;
    const uint32_t key = valid ? kin[i] : 0u;
    const uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, digit);
    const uint32_t rank = __popc(peers & lane_lt);
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = run[digit] + rank;
      for (int w = 0; w < warp; w++) pos += wcnt[w][digit];
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) tot += wcnt[w][tid];
    run[tid] += tot;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ fill
// Sorted (slot, master index) pairs -> postings and slot records. file_base has n_files + 1
// entries: the first master index of every file, then the total.
__global__ void fill_kernel(const uint32_t* keys, const uint32_t* vals, uint64_t n, uint32_t n_slots,
                            const uint32_t* owner, const uint32_t* cnt, const uint4* dig, const uint8_t* tau,
                            const uint64_t* file_base, uint32_t n_files, uint4* slots, uint2* postings,
                            uint32_t* n_unique) {
  uint32_t uniq = 0;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t key = keys[q];
    if (key >= n_slots) continue;
    const uint32_t m = vals[q];
    uint32_t lo = 0, hi = n_files;  // largest f with file_base[f] <= m
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (file_base[mid] <= m) lo = mid; else hi = mid;
    }
    postings[q] = make_uint2(lo, (uint32_t)(m - file_base[lo]));
    if (q == 0 || keys[q - 1] != key) {
      const uint32_t o = owner[key] - 1u;
      slots[2ull * key] = dig[o];
      slots[2ull * key + 1] = make_uint4((uint32_t)q, cnt[key], tau ? (uint32_t)tau[o] : 0u, 0u);
      uniq++;
    }
  }
  uniq = __reduce_add_sync(0xFFFFFFFFu, uniq);
  if ((threadIdx.x & 31) == 0 && uniq) atomicAdd(n_unique, uniq);
}

// Kept master units (sectors or fragments of wpu 16-byte words) in posting order: posting q
// (sorted pair q, key < n_slots) is master unit vals[q]; its words go to out + wpu q. One thread
// per 16-byte word.
__global__ void gather_units_kernel(const uint4* arena, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                                    uint32_t n_slots, uint32_t wpu, uint4* out) {
  const uint64_t words = n * wpu;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t q = i / wpu;
    if (keys[q] >= n_slots) continue;
    out[i] = arena[(uint64_t)vals[q] * wpu + i % wpu];
  }
}

// ------------------------------------------------------------------- sorted layout
// Sort key of the occupied-slot compaction: 0 for an occupied slot, 1 for an empty one; a stable
// sort by it puts the occupied slots first, in slot order.
__global__ void occupied_keys_kernel(const uint4* slots, uint32_t n_slots, uint32_t* keys, uint32_t* vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
    keys[i] = slots[2ull * i + 1].y != 0u ? 0u : 1u;
    vals[i] = i;
  }
}

// h0 = tau_home(d0, tau) of the slots vals[0..n).
__global__ void h0_keys_kernel(const uint4* slots, const uint32_t* vals, uint32_t n, uint32_t* keys) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const uint32_t i = vals[q];
    keys[q] = tau_home(slots[2ull * i].x, slots[2ull * i + 1].z);
  }
}

// Slot records in the order of vals (ascending h0): out[q] = slots[vals[q]].
__global__ void gather_slots_kernel(const uint4* slots, const uint32_t* vals, uint32_t n, uint4* out) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const uint32_t i = vals[q];
    out[2ull * q] = slots[2ull * i];
    out[2ull * q + 1] = slots[2ull * i + 1];
  }
}

// ------------------------------------------------------------------- loaded tables
// Every occupied record of a loaded table must name postings inside [0, n_postings).
__global__ void validate_slots_kernel(const uint4* slots, uint64_t n, uint64_t n_postings, uint32_t* status) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 val = slots[2 * i + 1];
    if (val.y != 0u && (uint64_t)val.x + val.y > n_postings) atomicOr(status, kStBadTable);
  }
}

// ----------------------------------------------------------------------------- Bloom
__global__ void bloom_kernel(const uint4* slots, uint32_t n_slots, uint32_t* bloom, uint32_t bloom_mask) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
    const uint4 val = slots[2ull * i + 1];
    if (val.y == 0u) continue;
    const uint4 d = slots[2ull * i];
    uint32_t* blk = bloom + 8ull * (tau_block(d.w, val.z) & bloom_mask);
    atomicOr(blk + 0, 1u << (d.y & 31));
    atomicOr(blk + 1, 1u << ((d.y >> 5) & 31));
    atomicOr(blk + 2, 1u << ((d.y >> 10) & 31));
    atomicOr(blk + 3, 1u << ((d.y >> 15) & 31));
    atomicOr(blk + 4, 1u << ((d.y >> 20) & 31));
    atomicOr(blk + 5, 1u << ((d.y >> 25) & 31));
    atomicOr(blk + 6, 1u << (d.z & 31));
    atomicOr(blk + 7, 1u << ((d.z >> 5) & 31));
  }
}

}  // namespace cvk
