// The fused sector scan: TMA staging -> per-sector MD5 -> Bloom test -> linear probe ->
// warp-ballot compaction of the hits of each tile.
//
// Paper Section 3.2 stages 16x16-word blocks of 16 sectors through shared memory with a
// rotation skew so that a cohort of 16 threads loads coalesced and then hashes one sector per
// thread without bank conflicts (Figures 8 and 9). The same idea on sm_103a: a tile of T
// sectors is brought into shared memory by the Tensor Memory Accelerator as a 2-D box
// (T rows of 512 bytes, BOXB bytes of each row per stage) with the hardware's 16-byte-chunk
// XOR swizzle, which plays the role of Figure 9's skew; thread t then hashes sector t of the
// tile (one sector per thread, Section 3.2), reading its words with conflict-free 16-byte
// shared loads. A dedicated producer warp keeps NS stages in flight through an mbarrier ring,
// so the hashing warps never issue a global load. Tiles are spread over a persistent grid.
//
// Every mbarrier wait is bounded in time: on expiry the kernel sets kStTimeout in the status
// word, stops waiting (its results are then discarded by the host), lets the producer wait
// for its own copies in flight, and returns.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "cv_internal.h"
#include "md5_sector.cuh"

namespace cvk {

constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s per wait

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t* abort_flag,
                                          uint32_t* status, uint64_t timeout_ns = kWaitTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer_ns() - t0 > timeout_ns) {
      *abort_flag = 1u;
      atomicOr(status, kStTimeout);
      return false;
    }
  }
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, uint32_t bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}

// Blocked Bloom test: all eight bits of the digest's block set.
__device__ __forceinline__ bool bloom_test(const TableView& tab, uint32_t d1, uint32_t d2, uint32_t d3,
                                           uint32_t tau) {
  const uint4* blk = tab.bloom + 2ull * (tau_block(d3, tau) & tab.bloom_mask);
  uint4 lo = __ldg(blk);
  uint4 hi = __ldg(blk + 1);
  uint32_t m = (lo.x >> (d1 & 31)) & (lo.y >> ((d1 >> 5) & 31)) & (lo.z >> ((d1 >> 10) & 31)) &
               (lo.w >> ((d1 >> 15) & 31)) & (hi.x >> ((d1 >> 20) & 31)) & (hi.y >> ((d1 >> 25) & 31)) &
               (hi.z >> (d2 & 31)) & (hi.w >> ((d2 >> 5) & 31));
  return (m & 1u) != 0;
}

// What a lookup reads from the table: a slot record (32 bytes) or a sorted key word (4 bytes).
// The scan passes this no-op counter; cv_probe_profile passes one that adds them up, so its
// counts are those of the very loops below.
struct ProbeNoCount {
  __device__ __forceinline__ void slot() const {}
  __device__ __forceinline__ void key() const {}
};

// Linear probing from the home slot (Eq. 3) until the key (digest, tau) or an empty slot is
// found, never beyond the table's probe bound. Returns post_cnt (0: not present) and post_off.
template <class Count = ProbeNoCount>
__device__ __forceinline__ uint32_t table_probe(const TableView& tab, uint32_t d0, uint32_t d1, uint32_t d2,
                                                uint32_t d3, uint32_t tau, uint32_t& post_off, Count cnt = Count()) {
  uint32_t idx = tau_home(d0, tau) & tab.slot_mask;
  for (uint32_t c = 0; c < tab.max_probe; c++) {
    cnt.slot();
    const uint4* s = tab.slots + 2ull * idx;
    uint4 key = __ldg(s);
    uint4 val = __ldg(s + 1);
    if (val.y == 0u) return 0u;
    if (key.x == d0 && key.y == d1 && key.z == d2 && key.w == d3 && val.z == tau) {
      post_off = val.x;
      return val.y;
    }
    idx = (idx + 1u) & tab.slot_mask;
  }
  return 0u;
}

// Sorted layout: branch-free lower bound of h0 = tau_home(d0, tau) in keys0 (ceil(log2 n_keys)
// dependent loads; the first levels are shared by every thread and stay in L1), then the
// records with that h0 are compared in full. Returns post_cnt (0: not present) and post_off.
template <class Count = ProbeNoCount>
__device__ __forceinline__ uint32_t sorted_probe(const TableView& tab, uint32_t d0, uint32_t d1, uint32_t d2,
                                                 uint32_t d3, uint32_t tau, uint32_t& post_off, Count cnt = Count()) {
  const uint32_t h0 = tau_home(d0, tau);
  const uint32_t* k = tab.keys0;
  uint32_t n = tab.n_keys;
  if (n == 0u) return 0u;
  uint32_t base = 0;
  while (n > 1u) {
    const uint32_t half = n >> 1;
    cnt.key();
    base = __ldg(k + base + half) < h0 ? base + half : base;
    n -= half;
  }
  cnt.key();
  for (uint32_t i = base + (__ldg(k + base) < h0 ? 1u : 0u); i < tab.n_keys && (cnt.key(), __ldg(k + i) == h0);
       i++) {
    cnt.slot();
    const uint4* s = tab.slots + 2ull * i;
    const uint4 key = __ldg(s);
    const uint4 val = __ldg(s + 1);
    if (key.x == d0 && key.y == d1 && key.z == d2 && key.w == d3 && val.z == tau) {
      post_off = val.x;
      return val.y;
    }
  }
  return 0u;
}

// Base-33 Horner value of a little-endian word, byte 0 first (Eq. 1 over four bytes):
// b0 33^3 + b1 33^2 + b2 33 + b3, as two 2-way (16-bit weight x 8-bit byte) dot products.
__device__ __forceinline__ uint32_t horner33(uint32_t w) {
  constexpr uint32_t kW01 = (1089u << 16) | 35937u;  // 33^2 (byte 1), 33^3 (byte 0)
  constexpr uint32_t kW23 = (1u << 16) | 33u;         // 1 (byte 3), 33 (byte 2)
  return __dp2a_lo(kW01, w, __dp2a_hi(kW23, w, 0u));
}

// djb2 over one 64-byte block (Eq. 1): four bytes at a time, h = h * 33^4 + the word's bytes
// in Horner form (byte 0 is the word's low byte; at most 255 * 37060 < 2^32).
__device__ __forceinline__ uint64_t djb2_block(uint64_t h, const uint32_t (&X)[16]) {
#pragma unroll
  for (int q = 0; q < 16; q++) h = h * 1185921ull + horner33(X[q]);  // 33^4
  return h;
}

// CRC64 with the generator G = x^64 + x^4 + x^3 + x + 1 (Section 2.1), most significant bit
// first, over one 64-byte block, 32 message bits per step and no table.
//
// With R the remainder of M(x) x^64 mod G, appending a 32-bit word w gives
//   R' = (M x^32 + w) x^64 mod G = r_lo x^32 + (r_hi + w) x^64 mod G,
// and x^64 = x^4 + x^3 + x + 1 (mod G). For v = r_hi + w, of degree < 32, v (x^4 + x^3 + x + 1)
// has degree < 36, so it is already reduced: R' = (r_lo << 32) ^ v(x^4 + x^3 + x + 1), which is
// u ^ (u << 3) with u = v ^ (v << 1), a 33-bit value. Its low word is u_lo ^ (u_lo << 3); its
// high word is (u_lo >> 29) ^ 9 u_32, where u_32 = v >> 31 is the bit shifted out of v << 1.
// The word's first byte in memory holds the highest coefficients, hence the byte swap.
// State: crc = {high word, low word}.
__device__ __forceinline__ void crc64_block(uint32_t& rh, uint32_t& rl, const uint32_t (&X)[16]) {
#pragma unroll
  for (int q = 0; q < 16; q++) {
    const uint32_t v = rh ^ __byte_perm(X[q], 0u, 0x0123u);
    const uint32_t u = v ^ (v << 1);
    rh = rl ^ (u >> 29) ^ ((v >> 31) * 9u);
    rl = u ^ (u << 3);
  }
}

enum : int { kModeScan = 0, kModeDigest = 1 };

template <int T, int NS, int BOXB>
struct ScanSmem {
  static constexpr uint32_t kStageBytes = T * BOXB;
  // stages first (1024-byte aligned), then the barriers and the abort flag
  static constexpr uint32_t kBarOff = NS * kStageBytes;
  static constexpr uint32_t kMiscOff = kBarOff + 2 * NS * 8;
  static constexpr uint32_t kBytes = kMiscOff + 16;
  static constexpr uint32_t kAlloc = kBytes + 1024;  // room to align the base
};

// T: sectors per tile; SPT: sectors per hashing thread (1 or 2; the block has C = T / SPT
// hashing threads plus one producer warp); NS: ring stages; BOXB: bytes of each sector row per
// stage (64 or 128); PIPE: which MD5 additions use the FMA pipe (see md5_fma_adds); MINB: the
// blocks per SM the register allocation must allow (0: no constraint).
// Thread t hashes rows t, t + C, ... of the tile. Matches are compacted per warp and row group:
// rows [32v, 32v + 32) of tile k form output tile k * (T / 32) + v.
template <int T, int SPT, int NS, int BOXB, int MODE, int PIPE, int MINB, int SIG, int LAYOUT>
__global__ void __launch_bounds__(T / SPT + 32, MINB) scan_kernel(const __grid_constant__ ScanParams p) {
  constexpr int C = T / SPT;
  // A tile larger than the 256-row TMA box limit is loaded as several boxes per stage.
  constexpr int kBoxes = (T + 255) / 256;
  constexpr int kBoxRows = T / kBoxes;
  static_assert(T % 32 == 0 && T <= 1024 && C % 32 == 0 && T % kBoxes == 0 && kBoxRows % 8 == 0, "tile rows");
  static_assert(SPT == 1 || SPT == 2, "sectors per thread");
  static_assert(BOXB == 64 || BOXB == 128, "box width");
  static_assert(NS <= 512 / BOXB, "at most a tile of stages in flight (the segment hand-off)");
  using L = ScanSmem<T, NS, BOXB>;
  constexpr int kChunks = 512 / BOXB;         // stages per sector
  constexpr int kBlocksPerChunk = BOXB / 64;  // MD5 blocks per stage
  constexpr uint32_t kW = T / 32;             // output tiles per tile
  constexpr int kCW = C / 32;                 // hashing warps

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* const gbase = smem_raw + (base - raw);
  const uint32_t bar_full = base + L::kBarOff;  // NS x 8 bytes
  const uint32_t bar_empty = bar_full + NS * 8;
  volatile uint32_t* const s_abort = reinterpret_cast<uint32_t*>(gbase + L::kMiscOff);
  // The segment of the block's k-th tile, found by the producer (a binary search over the
  // launch's segments) and read by the hashing warps after the tile's first stage, so that they
  // do not each repeat the search: two entries, by the parity of k.
  volatile uint32_t* const s_seg = reinterpret_cast<uint32_t*>(gbase + L::kMiscOff + 8);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < NS; s++) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, C);
    }
    *s_abort = 0u;
    s_seg[0] = s_seg[1] = 0u;  // in range even if a wait gives up before the producer writes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kCW) {
    // ------------------------------------------------------------------ producer warp
    if (lane != 0) return;
    const uint64_t policy = l2_evict_first_policy();
    uint32_t j = 0;
    bool ok = true;
    for (uint64_t lt = blockIdx.x; lt < p.n_tiles && ok; lt += gridDim.x) {
      const uint64_t tile = p.tile_begin + lt;
      const uint32_t sg = find_segment(p.segs, p.n_segs, tile);
      const Segment& seg = p.segs[sg];
      const CUtensorMap* map = &p.maps[seg.map - p.map_base];
      const int32_t row0 = (int32_t)(seg.row_base + (tile - seg.tile_base) * T);
      for (int c = 0; c < kChunks; c++, j++) {
        const uint32_t s = j % NS;
        if (j >= (uint32_t)NS && !mbar_wait(bar_empty + 8 * s, ((j / NS) - 1) & 1, s_abort, p.status)) {
          ok = false;
          break;
        }
        // published by the arrive below (release), seen after the matching wait (acquire); the
        // entry is rewritten for the tile after next, whose first copy waits for every hashing
        // thread to release a stage of the next tile, long after it read this one
        if (c == 0) s_seg[(j / kChunks) & 1] = sg;
        mbar_arrive_expect_tx(bar_full + 8 * s, L::kStageBytes);
#pragma unroll
        for (int k = 0; k < kBoxes; k++)
          tma_load_2d(base + s * L::kStageBytes + k * kBoxRows * BOXB, map, c * (BOXB / 4), row0 + k * kBoxRows,
                      bar_full + 8 * s, policy);
      }
    }
    // Wait (bounded) for the copies still in flight so none lands after the block exits.
    const uint32_t issued = j;
    const uint32_t first = issued > (uint32_t)NS ? issued - NS : 0u;
    for (uint32_t q = first; q < issued; q++) {
      const uint32_t s = q % NS;
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(bar_full + 8 * s, (q / NS) & 1)) {
        if (globaltimer_ns() - t0 > kWaitTimeoutNs) {
          atomicOr(p.status, kStTimeout);
          break;
        }
      }
    }
    return;
  }

  // -------------------------------------------------------------------- hashing warps
  // Row r of each stage; its 16-byte chunk q sits at chunk q ^ swz(r) (hardware swizzle).
  uint32_t row_off[SPT], swz[SPT];
#pragma unroll
  for (int k = 0; k < SPT; k++) {
    const uint32_t r = (uint32_t)(tid + k * C);
    row_off[k] = r * BOXB;
    swz[k] = (BOXB == 128) ? (r & 7u) : ((r >> 1) & 3u);
  }
  const uint32_t lane_lt = (1u << lane) - 1u;
  uint32_t j = 0;
  for (uint64_t lt = blockIdx.x; lt < p.n_tiles; lt += gridDim.x) {
    const uint64_t tile = p.tile_begin + lt;
    // No-pad MD5 has no padding compression between the last stage and the lookup to hide the
    // segment's loads behind, and measured faster finding its segment itself at the tile start.
    uint32_t sgi = 0;
    if constexpr (SIG == kSigMd5NoPad) sgi = find_segment(p.segs, p.n_segs, tile);
    uint32_t st[SPT][4];
    uint64_t h[SPT];  // djb2 / CRC64 accumulators
    uint32_t diff[SPT], ref[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) {
      md5_init(st[k]);
      h[k] = SIG == kSigDjb2 ? 5381ull : 0ull;
      diff[k] = 0;
      ref[k] = 0;
    }
    // Stages unrolled in groups; with a whole number of ring turns per tile (j = tiles * kChunks
    // + c) the stage index follows from c and is a constant within a group. A group holds at most
    // four MD5 compressions (two without padding): more code than that ran slower. djb2 and CRC64
    // blocks are small and go in pairs.
    constexpr int kCompressions = SPT * kBlocksPerChunk;  // MD5 compressions per stage
    constexpr int kGroupMax = SIG == kSigMd5 ? 4 : 2;     // per unrolled group
    constexpr int kUnroll = sig_is_weak(SIG) ? 2 : (kGroupMax >= kCompressions ? kGroupMax / kCompressions : 1);
#pragma unroll(kUnroll)
    for (int c = 0; c < kChunks; c++, j++) {
      const uint32_t s = (kChunks % NS == 0) ? (uint32_t)c % NS : j % NS;
      mbar_wait(bar_full + 8 * s, (j / NS) & 1, s_abort, p.status);
      if constexpr (SIG != kSigMd5NoPad) {
        if (c == 0) sgi = s_seg[(j / kChunks) & 1];
      }
      const uint32_t stage = base + s * L::kStageBytes;
#pragma unroll
      for (int b = 0; b < kBlocksPerChunk; b++) {
        uint32_t X[SPT][16];
#pragma unroll
        for (int k = 0; k < SPT; k++) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const uint32_t chunk = (uint32_t)(4 * b + q) ^ swz[k];
            const uint4 v = lds128(stage + row_off[k] + chunk * 16u);
            X[k][4 * q + 0] = v.x;
            X[k][4 * q + 1] = v.y;
            X[k][4 * q + 2] = v.z;
            X[k][4 * q + 3] = v.w;
          }
        }
        if (b == kBlocksPerChunk - 1) {
          // The stage is handed back to the copy engine: order this thread's shared-memory
          // reads (generic proxy) before the next TMA write into the stage (async proxy).
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(bar_empty + 8 * s);
        }
        if constexpr (MODE == kModeDigest) {
#pragma unroll
          for (int k = 0; k < SPT; k++) {
            if (c == 0 && b == 0) ref[k] = (X[k][0] & 0xFFu) * 0x01010101u;
#pragma unroll
            for (int q = 0; q < 16; q++) diff[k] |= X[k][q] ^ ref[k];
          }
        }
        if constexpr (SIG == kSigDjb2) {
#pragma unroll
          for (int k = 0; k < SPT; k++) h[k] = djb2_block(h[k], X[k]);
        } else if constexpr (SIG == kSigCrc64) {
#pragma unroll
          for (int k = 0; k < SPT; k++) {
            uint32_t rh = (uint32_t)(h[k] >> 32), rl = (uint32_t)h[k];
            crc64_block(rh, rl, X[k]);
            h[k] = ((uint64_t)rh << 32) | rl;
          }
        } else if constexpr (SPT == 2) {
          md5_compress_x2<PIPE>(st[0], X[0], st[1], X[1], p.one);
        } else {
          md5_compress<PIPE>(st[0], X[0], p.one);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < SPT; k++) {
      if constexpr (SIG == kSigMd5) md5_compress_sector_padding(st[k], p.one);
      if constexpr (sig_is_weak(SIG)) sig64_words(h[k], st[k]);
    }

    const Segment& seg = p.segs[sgi];
    const uint64_t row0 = (tile - seg.tile_base) * T;  // within the segment
#pragma unroll
    for (int k = 0; k < SPT; k++) {
      const uint64_t r = row0 + (uint64_t)(tid + k * C);
      const bool valid = r < seg.n_sectors;
      if constexpr (MODE == kModeDigest) {
        if (valid) {
          const uint64_t g = seg.sector_base + r;
          p.digests[g] = make_uint4(st[k][0], st[k][1], st[k][2], st[k][3]);
          if (p.trivial) p.trivial[g] = diff[k] == 0u ? 1 : 0;
        }
      } else {
        uint32_t post_off = 0, post_cnt = 0;
        // the disk sector's position in its cluster (0 for a table over all positions)
        const uint32_t tau = (uint32_t)(seg.sector_base + r + p.tab.tau_add) & p.tab.tau_mask;
        if (valid && (!p.tab.use_bloom || bloom_test(p.tab, st[k][1], st[k][2], st[k][3], tau)))
          post_cnt = LAYOUT == kLayoutSorted
                         ? sorted_probe(p.tab, st[k][0], st[k][1], st[k][2], st[k][3], tau, post_off)
                         : table_probe(p.tab, st[k][0], st[k][1], st[k][2], st[k][3], tau, post_off);
        // triples this sector emits: every posting, or for a 64-bit signature the postings whose
        // master sector equals this sector byte for byte
        uint32_t n_emit = post_cnt;
        if constexpr (sig_is_weak(SIG)) {
          if (post_cnt) {
            const uint8_t* mine = seg.bytes + r * kSector;
            n_emit = 0;
            for (uint32_t q = 0; q < post_cnt; q++)
              n_emit += sectors_equal(mine, p.tab.confirm + (uint64_t)(post_off + q) * kSector) ? 1u : 0u;
            if (p.rejected && n_emit < post_cnt) atomicAdd(p.rejected, (unsigned long long)(post_cnt - n_emit));
          }
        }
        const bool hit = n_emit != 0u;
        const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, hit);
        const uint32_t wtrip = __reduce_add_sync(0xFFFFFFFFu, n_emit);
        const uint64_t u = tile * kW + (uint64_t)(warp + k * kCW);  // this row group's output tile
        if (hit) p.hit_rec[u * 32 + __popc(ballot & lane_lt)] = make_uint4((uint32_t)lane, post_off, post_cnt, n_emit);
        if (lane == 0) {
          p.tile_nhit[u] = __popc(ballot);
          p.tile_ntrip[u] = wtrip;
        }
      }
    }
  }
}

}  // namespace cvk
