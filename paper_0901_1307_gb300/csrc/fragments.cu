// Fragment scan (paper Section 5): every 64-byte window of a disk image that starts at a
// multiple of 4 bytes is looked up among the whole 64-byte fragments of the master files, to
// find small files (logos, small images) embedded in other files at any 32-bit offset.
//
// Work layout. A tile is one warp's work: 32 x WPT consecutive windows. Each warp stages its own
// tiles (the window starts plus the last window's 60-byte tail) into its own two shared-memory
// buffers with 1-D bulk TMA copies issued by its lane 0, completion on the warp's own mbarriers,
// every wait bounded; warps of a block never wait for one another, so a warp that meets a
// candidate (an L2 probe) holds up no one. Lane l takes windows [WPT l, WPT l + WPT) of the tile;
// with WPT odd the 32 lanes read 32 different banks at every step. Tiles are spread over every
// warp of a persistent grid.
//
//   djb2-64 (Eq. 1) is rolled. With P(x) the base-33 Horner value of a 4-byte word x and
//   g = h - 5381 * 33^64, a window W_k of words x_k .. x_{k+15} has g(W_k) = sum_q
//   P(x_{k+q}) 33^{4 (15 - q)}, so g(W_{k+1}) = 33^4 g(W_k) - 33^64 P(x_k) + P(x_{k+16})
//   (mod 2^64): after a lane's first window each one costs one word and a few multiply-adds.
//   A rolled window is cheap enough that its Bloom lookup, not its hash, sets the pace, and an
//   SM keeps only so many L2 misses in flight: so the djb2 kernel first tests a 2^20-bit filter
//   held in shared memory (loaded once per block) and sends only the windows that pass it to
//   the one-word Bloom filter in global memory.
//   MD5 is computed per window (two compressions, or one without the padding block); there the
//   hash dominates and the global Bloom word is tested directly.
//
// Passes (no worst-case hit buffer). The count kernel hashes every window, filters it, resolves
// the candidates (probe; byte confirmation for djb2) and writes each tile's triple count; an
// exclusive scan gives every tile its output offset; the emit kernel redoes only the tiles
// that have triples and writes them in window order. Filters never drop a match, so the emit
// kernel, which skips the shared-memory filter, finds exactly the counted triples.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "cv_launch.h"
#include "scan_kernel.cuh"

// The djb2 count kernel's block size, tile buffers per warp and Bloom pipeline depth: the
// fastest measured on GB300 (4 GiB fragment workload, count kernel, all exact): 512 threads, two
// buffers, depth 12: 1,431 GB/s; depth 8: 1,425; depth 17: 1,298. With more warps per SM the
// kernel exceeds its register share and spills: 1024 threads, one buffer, depth 6 / 8 / 12:
// 1,312 / 971 / 834; 640 threads, two buffers, depth 8: 892; 768, one buffer, depth 8: 883.
#ifndef CV_FRAG_DJB2_THREADS
#define CV_FRAG_DJB2_THREADS 512
#endif
#ifndef CV_FRAG_DJB2_BUFS
#define CV_FRAG_DJB2_BUFS 2
#endif
#ifndef CV_FRAG_DJB2_BLOOM_DEPTH
#define CV_FRAG_DJB2_BLOOM_DEPTH 12
#endif

namespace cvk {

// Tile geometry per signature (a tile is one warp's work).
template <int SIG>
struct FragGeom {
  static constexpr bool kRolled = SIG == kSigDjb2;
  static constexpr int kThreads = kRolled ? CV_FRAG_DJB2_THREADS : 256;  // block size
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kWPT = kRolled ? 17 : 33;        // windows per lane per tile (odd)
  static constexpr int kBufs = kRolled ? CV_FRAG_DJB2_BUFS : 2;  // tile buffers per warp (count kernel)
  static constexpr int kBloomDepth = CV_FRAG_DJB2_BLOOM_DEPTH;  // Bloom words in flight per lane
  static constexpr uint32_t kTileWin = 32 * kWPT;
  static constexpr uint32_t kTileStep = kTileWin * kFragStride;  // bytes between tile starts
  static constexpr uint32_t kTileBytes = kTileStep + 64;         // bytes staged per tile
  static constexpr bool kL1 = kRolled;                           // shared-memory filter
  static constexpr uint32_t kL1Off = kBufs * kWarps * kTileBytes;  // filter after the warps' buffers
  static constexpr uint32_t kSmemCount = kL1Off + (kL1 ? kFragL1Bytes : 0);
  static constexpr uint32_t kSmemEmit = kWarps * kTileBytes;
  static_assert(kWPT % 2 == 1 && kWPT <= 64 && (!kRolled || kWPT <= 32), "odd window count, masks of 64/32 bits");
  static_assert(kTileBytes % 16 == 0 && kTileStep % 16 == 0, "bulk copies of whole 16-byte chunks");
  static_assert(kBufs == 1 || kBufs == 2, "one or two tile buffers per warp");
  static_assert(kSmemCount <= 227 * 1024, "shared memory of one block");
};

__host__ __device__ constexpr uint64_t pow33(int e) {
  uint64_t r = 1;
  for (int i = 0; i < e; i++) r *= 33u;
  return r;
}
constexpr uint64_t kD33x4 = pow33(4);
constexpr uint64_t kD33x64 = pow33(64);
constexpr uint64_t kDjbInit = 5381ull * pow33(64);  // 5381 * 33^64: the initial value's share

struct FragParams {
  TableView tab;
  const uint8_t* image;
  uint64_t n_bytes;
  uint64_t n_windows;
  uint64_t n_tiles;
  uint64_t tile_base;            // index of this image's first tile in tile_ntrip / tile_off
  uint64_t* tile_ntrip;          // count: triples per tile
  const uint64_t* tile_off;      // emit: output offset per tile
  const uint32_t* hit_tiles;     // emit: this image's tiles with triples (local indices)
  const uint32_t* n_hit_tiles;   // emit: their number (device)
  MatchOut* out;
  uint64_t out_cap;
  uint32_t* status;
  uint32_t one;                  // always 1 (the MD5 kernels' opaque multiplier)
  unsigned long long* rejected;  // count: djb2 candidates dropped by the byte comparison (or null)
};

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                          uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint32_t frag_bloom_bits(uint32_t d2) {
  return (1u << (d2 & 31)) | (1u << ((d2 >> 5) & 31)) | (1u << ((d2 >> 10) & 31));
}

__device__ __forceinline__ bool frag_bloom_test(const TableView& tab, uint32_t d2, uint32_t d3) {
  const uint32_t bits = frag_bloom_bits(d2);
  return (__ldg(reinterpret_cast<const uint32_t*>(tab.bloom) + (d3 & tab.bloom_mask)) & bits) == bits;
}

// djb2-64 of consecutive windows w0, w0 + 1, ... (ws: 32-bit words in shared memory), rolled:
// first() computes window w0 from its 16 words, then next(i) moves to window w0 + i (called for
// i = 1, 2, ... in order) with one new word. P holds the Horner values of the current window's
// words, g = h - 5381 * 33^64.
struct Djb2Roll {
  uint32_t P[16];
  uint64_t g;
  __device__ __forceinline__ uint64_t first(const uint32_t* ws, uint32_t w0) {
    g = 0;
#pragma unroll
    for (int q = 0; q < 16; q++) {
      P[q] = horner33(ws[w0 + q]);
      g = g * kD33x4 + P[q];
    }
    return g + kDjbInit;
  }
  __device__ __forceinline__ uint64_t next(const uint32_t* ws, uint32_t w0, int i) {
    const uint32_t pin = horner33(ws[w0 + i + 15]);
    g = g * kD33x4 - (uint64_t)P[(i - 1) & 15] * kD33x64 + pin;
    P[(i - 1) & 15] = pin;
    return g + kDjbInit;
  }
};

// Key words of the window whose first word is ws[w] (shared memory), computed directly.
template <int SIG>
__device__ __forceinline__ void frag_key(const uint32_t* ws, uint32_t w, uint32_t (&d)[4], uint32_t one) {
  uint32_t X[16];
#pragma unroll
  for (int q = 0; q < 16; q++) X[q] = ws[w + q];
  if constexpr (SIG == kSigDjb2) {
    frag64_words(djb2_block(5381ull, X), d);
  } else {
    md5_init(d);
    md5_compress<3>(d, X, one);
    if constexpr (SIG == kSigMd5) md5_compress_block_padding(d, one);
  }
}

// 64 bytes of the window at ws[w] (shared, 4-byte aligned) against a master fragment (global,
// 16-byte aligned).
__device__ __forceinline__ bool frag_equal(const uint32_t* ws, uint32_t w, const uint8_t* m) {
  const uint4* y = reinterpret_cast<const uint4*>(m);
  uint32_t diff = 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const uint4 v = __ldg(y + q);
    diff |= (ws[w + 4 * q] ^ v.x) | (ws[w + 4 * q + 1] ^ v.y) | (ws[w + 4 * q + 2] ^ v.z) | (ws[w + 4 * q + 3] ^ v.w);
  }
  return diff == 0;
}

// Candidate windows of this thread (bit i: window w0 + i passed the filters; every valid window
// when the table has no Bloom filter). n_valid: the thread's windows inside the image. l1: the
// shared-memory filter, or null to skip it (then every window goes to the global Bloom word).
template <int SIG>
__device__ __forceinline__ uint64_t frag_candidates(const FragParams& p, const uint32_t* ws, uint32_t w0,
                                                    uint32_t n_valid, const uint32_t* l1) {
  using G = FragGeom<SIG>;
  uint64_t cand = 0;
  if constexpr (G::kRolled) {
    // Window by window: the rolled hash, its shared-memory filter bit (from h's high word, d1,
    // with no further mixing) and, when that passes, the request of its one-word Bloom filter
    // word (mixed words d2, d3); each Bloom word is tested kBloomDepth windows later, so that
    // many requests are in flight per lane while only kBloomDepth are held in registers. A window
    // that did not pass keeps (word 0, bits 1), which fails the test.
    constexpr int D = G::kBloomDepth < G::kWPT ? G::kBloomDepth : G::kWPT;
    const uint32_t* bloom = reinterpret_cast<const uint32_t*>(p.tab.bloom);
    const bool use_bloom = p.tab.use_bloom != 0u;
    Djb2Roll roll;
    uint32_t wv[D], wbits[D];
#pragma unroll
    for (int i = 0; i < G::kWPT + D; i++) {
      if (use_bloom && i >= D) {  // window i - D's word, before window i takes its ring slot
        const int j = i - D;
        if ((wv[j % D] & wbits[j % D]) == wbits[j % D]) cand |= 1ull << j;
      }
      if (i < G::kWPT) {
        const uint64_t h = i == 0 ? roll.first(ws, w0) : roll.next(ws, w0, i);
        const uint32_t b = (uint32_t)(h >> 32) >> (32 - kFragL1Log2Bits);
        const bool pass = (uint32_t)i < n_valid && (!l1 || ((l1[b >> 5] >> (b & 31)) & 1u));
        if (!use_bloom) {
          if (pass) cand |= 1ull << i;
        } else {
          wv[i % D] = 0u;
          wbits[i % D] = 1u;
          if (pass) {
            uint32_t d[4];
            frag64_words(h, d);
            wbits[i % D] = frag_bloom_bits(d[2]);
            wv[i % D] = __ldg(bloom + (d[3] & p.tab.bloom_mask));
          }
        }
      }
    }
  } else {
#pragma unroll 1
    for (uint32_t i = 0; i < n_valid; i++) {
      uint32_t d[4];
      frag_key<SIG>(ws, w0 + i, d, p.one);
      if (!p.tab.use_bloom || frag_bloom_test(p.tab, d[2], d[3])) cand |= 1ull << i;
    }
  }
  return cand;
}

// Probe one candidate window; returns the triples it yields (postings, confirmed byte for byte
// for djb2) and the posting range.
template <int SIG, int LAYOUT>
__device__ __forceinline__ uint32_t frag_resolve(const FragParams& p, const uint32_t* ws, uint32_t w,
                                                 uint32_t& post_off, uint32_t& post_cnt) {
  uint32_t d[4];
  frag_key<SIG>(ws, w, d, p.one);
  post_off = 0;
  post_cnt = LAYOUT == kLayoutSorted ? sorted_probe(p.tab, d[0], d[1], d[2], d[3], 0u, post_off)
                                     : table_probe(p.tab, d[0], d[1], d[2], d[3], 0u, post_off);
  if (!sig_is_weak(SIG) || post_cnt == 0) return post_cnt;
  uint32_t n = 0;
  for (uint32_t q = 0; q < post_cnt; q++) n += frag_equal(ws, w, p.tab.confirm + (uint64_t)(post_off + q) * 64) ? 1u : 0u;
  return n;
}

// Triples of this thread's candidate windows; *rejected (when given) adds the candidates that
// the byte comparison dropped.
template <int SIG, int LAYOUT>
__device__ __forceinline__ uint64_t frag_thread_count(const FragParams& p, const uint32_t* ws, uint32_t w0,
                                                      uint64_t cand, uint32_t* rejected = nullptr) {
  uint64_t n = 0;
  while (cand) {
    const int i = __ffsll((long long)cand) - 1;
    cand &= cand - 1;
    uint32_t off, cnt;
    const uint32_t k = frag_resolve<SIG, LAYOUT>(p, ws, w0 + (uint32_t)i, off, cnt);
    n += k;
    if (rejected) *rejected += cnt - k;
  }
  return n;
}

__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int d) {
  const uint32_t lo = __shfl_up_sync(0xFFFFFFFFu, (uint32_t)v, d);
  const uint32_t hi = __shfl_up_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), d);
  return ((uint64_t)hi << 32) | lo;
}

// Warp-wide exclusive scan of one u64 per lane; *total receives the sum (every lane).
__device__ __forceinline__ uint64_t warp_exclusive_u64(uint64_t v, uint64_t* total) {
  const int lane = threadIdx.x & 31;
  uint64_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t x = shfl_up_u64(incl, d);
    if (lane >= d) incl += x;
  }
  const uint32_t lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)incl, 31);
  const uint32_t hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(incl >> 32), 31);
  *total = ((uint64_t)hi << 32) | lo;
  return incl - v;
}

// Lane 0: issue tile `tile` into the buffer at smem address dst (completion on bar).
template <int SIG>
__device__ __forceinline__ void frag_issue(const FragParams& p, uint64_t tile, uint32_t dst, uint32_t bar,
                                           uint64_t policy) {
  using G = FragGeom<SIG>;
  const uint64_t start = tile * G::kTileStep;
  const uint64_t left = p.n_bytes - start;
  const uint32_t avail = left < G::kTileBytes ? (uint32_t)left : G::kTileBytes;
  const uint32_t bulk = avail & ~15u;
  mbar_arrive_expect_tx(bar, bulk);
  if (bulk) bulk_load(dst, p.image + start, bulk, bar, policy);
}

// The bytes of the tile past its last whole 16-byte chunk (the bulk copy moves whole chunks
// only), with plain loads by the warp's lanes; only the image's last tile has any. Ends with a
// warp barrier.
template <int SIG>
__device__ __forceinline__ void frag_tail(const FragParams& p, uint64_t tile, uint8_t* buf) {
  using G = FragGeom<SIG>;
  const uint64_t start = tile * G::kTileStep;
  const uint64_t left = p.n_bytes - start;
  const uint32_t avail = left < G::kTileBytes ? (uint32_t)left : G::kTileBytes;
  const uint32_t b = (avail & ~15u) + (threadIdx.x & 31);
  if (b < avail) buf[b] = p.image[start + b];
  __syncwarp();
}

template <int SIG>
__device__ __forceinline__ uint32_t frag_valid(const FragParams& p, uint64_t tile, uint32_t w0) {
  using G = FragGeom<SIG>;
  const uint64_t k0 = tile * G::kTileWin + w0;
  if (k0 >= p.n_windows) return 0u;
  const uint64_t left = p.n_windows - k0;
  return left < (uint64_t)G::kWPT ? (uint32_t)left : (uint32_t)G::kWPT;
}

template <int SIG, int LAYOUT>
__global__ void __launch_bounds__(FragGeom<SIG>::kThreads, 1) frag_count_kernel(const __grid_constant__ FragParams p) {
  using G = FragGeom<SIG>;
  extern __shared__ __align__(128) uint8_t fsm[];
  constexpr int B = G::kBufs;
  __shared__ __align__(8) uint64_t bars[B * G::kWarps + 1];  // B per warp, the shared-memory filter
  __shared__ uint32_t abort_flag[G::kWarps + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t* l1 = G::kL1 ? reinterpret_cast<const uint32_t*>(fsm + G::kL1Off) : nullptr;
  uint8_t* mybuf = fsm + B * warp * G::kTileBytes;
  const uint32_t bar0 = smem_addr(&bars[B * warp]);
  const uint32_t bar_l1 = smem_addr(&bars[B * G::kWarps]);
  if (tid == 0) {
    for (int b = 0; b < B * G::kWarps + 1; b++) mbar_init(smem_addr(&bars[b]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid <= G::kWarps) abort_flag[tid] = 0;
  __syncthreads();
  const uint64_t policy = l2_evict_first_policy();
  const uint64_t n_warps = (uint64_t)gridDim.x * G::kWarps;
  const uint64_t first = (uint64_t)blockIdx.x * G::kWarps + warp;
  // Buffer s of a warp holds the tiles of its iterations i with i mod B == s; the k-th of them
  // completes phase k of the buffer's barrier. Lane 0 issues the first B tiles, then each tile
  // B iterations ahead.
  if (tid == 0 && G::kL1) {
    mbar_arrive_expect_tx(bar_l1, kFragL1Bytes);
    bulk_load(smem_addr(fsm + G::kL1Off), p.tab.frag_l1, kFragL1Bytes, bar_l1, policy);
  }
  if (lane == 0)
    for (int s = 0; s < B; s++) {
      const uint64_t t = first + s * n_warps;
      if (t < p.n_tiles) frag_issue<SIG>(p, t, smem_addr(mybuf + s * G::kTileBytes), bar0 + 8 * s, policy);
    }
  bool ok = true;
  if constexpr (G::kL1) ok = mbar_wait(bar_l1, 0u, &abort_flag[G::kWarps], p.status);
  bool aborted = !__syncthreads_and(ok);  // the only block-wide barrier: the filter is in place
  uint64_t i = 0;
  for (; !aborted; i++) {
    const uint64_t tile = first + i * n_warps;
    if (tile >= p.n_tiles) break;
    const int s = (int)(i % B);
    uint8_t* buf = mybuf + s * G::kTileBytes;
    ok = mbar_wait(bar0 + 8 * s, (uint32_t)(i / B) & 1u, &abort_flag[warp], p.status);
    if (!__all_sync(0xFFFFFFFFu, ok)) {
      aborted = true;
      break;
    }
    if ((tile + 1) * G::kTileStep + 64 > p.n_bytes) frag_tail<SIG>(p, tile, buf);  // warp-uniform
    const uint32_t* ws = reinterpret_cast<const uint32_t*>(buf);
    const uint32_t w0 = (uint32_t)lane * G::kWPT;
    const uint64_t cand = frag_candidates<SIG>(p, ws, w0, frag_valid<SIG>(p, tile, w0), l1);
    uint32_t rej = 0;
    uint64_t n = frag_thread_count<SIG, LAYOUT>(p, ws, w0, cand, &rej);
    if (sig_is_weak(SIG) && rej && p.rejected) atomicAdd(p.rejected, (unsigned long long)rej);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n += __shfl_xor_sync(0xFFFFFFFFu, n, d);
    __syncwarp();  // every lane is done with the buffer
    if (lane == 0) {
      p.tile_ntrip[p.tile_base + tile] = n;
      const uint64_t next = tile + B * n_warps;
      if (next < p.n_tiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        frag_issue<SIG>(p, next, smem_addr(buf), bar0 + 8 * s, policy);
      }
    }
    __syncwarp();
  }
  if (aborted && lane == 0) {
    // The filter (lane 0 of warp 0) and this warp's iterations i .. i + B - 1 may have copies
    // issued and not waited for: let them land, each wait bounded, before shared memory goes away.
    volatile uint32_t never = 0;
    if (G::kL1 && tid == 0) mbar_wait(bar_l1, 0u, &never, p.status);
    for (uint64_t j = i; j < i + B && first + j * n_warps < p.n_tiles; j++)
      if (!mbar_wait(bar0 + 8 * (j % B), (uint32_t)(j / B) & 1u, &never, p.status)) break;
  }
}

// Tiles of one image with triples, as a list of local tile indices (any order).
__global__ void frag_hit_list_kernel(const uint64_t* tile_ntrip, uint64_t n_tiles, uint32_t* list, uint32_t* count) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += (uint64_t)gridDim.x * blockDim.x)
    if (tile_ntrip[t]) list[atomicAdd(count, 1u)] = (uint32_t)t;
}

template <int SIG, int LAYOUT>
__global__ void __launch_bounds__(FragGeom<SIG>::kThreads, 1) frag_emit_kernel(const __grid_constant__ FragParams p) {
  using G = FragGeom<SIG>;
  extern __shared__ __align__(128) uint8_t fsm[];
  __shared__ __align__(8) uint64_t bars[G::kWarps];
  __shared__ uint32_t abort_flag[G::kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t* buf = fsm + warp * G::kTileBytes;
  const uint32_t bar = smem_addr(&bars[warp]);
  if (lane == 0) {
    abort_flag[warp] = 0;
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint64_t policy = l2_evict_first_policy();
  const uint32_t n_list = *(volatile const uint32_t*)p.n_hit_tiles;
  const uint32_t n_warps = gridDim.x * G::kWarps;
  uint32_t phase = 0;
  for (uint32_t j = blockIdx.x * G::kWarps + warp; j < n_list; j += n_warps) {
    const uint64_t tile = p.hit_tiles[j];
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      frag_issue<SIG>(p, tile, smem_addr(buf), bar, policy);
    }
    const bool ok = mbar_wait(bar, phase & 1u, &abort_flag[warp], p.status);
    if (!__all_sync(0xFFFFFFFFu, ok)) {
      if (lane == 0) {  // the copy may still land: wait for it (bounded) before leaving
        volatile uint32_t never = 0;
        mbar_wait(bar, phase & 1u, &never, p.status);
      }
      return;
    }
    phase++;
    if ((tile + 1) * G::kTileStep + 64 > p.n_bytes) frag_tail<SIG>(p, tile, buf);
    const uint32_t* ws = reinterpret_cast<const uint32_t*>(buf);
    const uint32_t w0 = (uint32_t)lane * G::kWPT;
    const uint64_t cand = frag_candidates<SIG>(p, ws, w0, frag_valid<SIG>(p, tile, w0), nullptr);
    const uint64_t n = frag_thread_count<SIG, LAYOUT>(p, ws, w0, cand);
    uint64_t total;
    uint64_t pos = p.tile_off[p.tile_base + tile] + warp_exclusive_u64(n, &total);
    uint64_t c = cand;
    while (c) {
      const int i = __ffsll((long long)c) - 1;
      c &= c - 1;
      const uint32_t w = w0 + (uint32_t)i;
      uint32_t off, cnt;
      if (!frag_resolve<SIG, LAYOUT>(p, ws, w, off, cnt)) continue;
      const uint64_t k = tile * G::kTileWin + w;
      for (uint32_t q = 0; q < cnt; q++) {
        if (sig_is_weak(SIG) && !frag_equal(ws, w, p.tab.confirm + (uint64_t)(off + q) * 64)) continue;
        if (pos < p.out_cap) {
          const uint2 e = __ldg(p.tab.postings + off + q);
          p.out[pos] = MatchOut{k, e.x, e.y};
        } else {
          atomicOr(p.status, kStOverflow);
        }
        pos++;
      }
    }
    __syncwarp();  // the buffer is free again
  }
}

// The signature of every window of an image, 16 bytes per window, through the count kernel's
// own arithmetic: the rolled djb2 of Djb2Roll (the same tile geometry, each lane's first window
// computed directly and the others rolled), or frag_key for MD5. For djb2 the 16 bytes are the
// table key words (h, then the mixing word of frag64_words). One warp per tile, staged with
// plain loads; a test and diagnostic path, not the scan.
template <int SIG>
__global__ void __launch_bounds__(256) frag_window_sig_kernel(const uint8_t* image, uint64_t n_bytes,
                                                              uint64_t n_windows, uint64_t n_tiles, uint4* out,
                                                              uint32_t one) {
  using G = FragGeom<SIG>;
  extern __shared__ __align__(128) uint8_t fsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* ws = reinterpret_cast<uint32_t*>(fsm + warp * G::kTileBytes);
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < n_tiles; tile += warps) {
    const uint64_t start = tile * G::kTileStep;
    for (uint32_t j = lane; j < G::kTileBytes / 4; j += 32) {
      const uint64_t b = start + 4ull * j;
      uint32_t v = 0;
      if (b + 4 <= n_bytes) {
        v = *reinterpret_cast<const uint32_t*>(image + b);
      } else {
        for (uint32_t q = 0; q < 4; q++)
          if (b + q < n_bytes) v |= (uint32_t)image[b + q] << (8 * q);
      }
      ws[j] = v;
    }
    __syncwarp();
    const uint32_t w0 = (uint32_t)lane * G::kWPT;
    const uint64_t k0 = tile * G::kTileWin + w0;
    if constexpr (G::kRolled) {
      Djb2Roll roll;
#pragma unroll
      for (int i = 0; i < G::kWPT; i++) {
        const uint64_t h = i == 0 ? roll.first(ws, w0) : roll.next(ws, w0, i);
        uint32_t d[4];
        frag64_words(h, d);
        if (k0 + i < n_windows) out[k0 + i] = make_uint4(d[0], d[1], d[2], d[3]);
      }
    } else {
      for (int i = 0; i < G::kWPT; i++) {
        if (k0 + i >= n_windows) break;
        uint32_t d[4];
        frag_key<SIG>(ws, w0 + (uint32_t)i, d, one);
        out[k0 + i] = make_uint4(d[0], d[1], d[2], d[3]);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------ master side
// Key words of every master fragment (64 bytes each, 16-byte aligned) and its exclusion flag
// (all 64 bytes equal).
template <int SIG>
__global__ void frag_digest_kernel(const uint8_t* arena, uint64_t n, uint4* dig, uint8_t* trivial, uint32_t one) {
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (uint64_t)gridDim.x * blockDim.x) {
    const uint4* src = reinterpret_cast<const uint4*>(arena + m * 64);
    uint32_t X[16];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint4 v = src[q];
      X[4 * q] = v.x;
      X[4 * q + 1] = v.y;
      X[4 * q + 2] = v.z;
      X[4 * q + 3] = v.w;
    }
    const uint32_t rep = (X[0] & 0xFFu) * 0x01010101u;
    uint32_t diff = 0;
#pragma unroll
    for (int q = 0; q < 16; q++) diff |= X[q] ^ rep;
    uint32_t d[4];
    if constexpr (SIG == kSigDjb2) {
      frag64_words(djb2_block(5381ull, X), d);
    } else {
      md5_init(d);
      md5_compress<3>(d, X, one);
      if constexpr (SIG == kSigMd5) md5_compress_block_padding(d, one);
    }
    dig[m] = make_uint4(d[0], d[1], d[2], d[3]);
    trivial[m] = diff == 0u ? 1 : 0;
  }
}

// The filters of a fragment table from its occupied slots: the one-word Bloom filter (3 bits
// from d2 in word d3 & mask; none when words is null) and the 2^20-bit shared-memory filter
// (bit: the top 20 bits of d1).
__global__ void frag_bloom_kernel(const uint4* slots, uint32_t n_slots, uint32_t* words, uint32_t mask,
                                  uint32_t* l1) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
    if (slots[2ull * i + 1].y == 0u) continue;
    const uint4 d = slots[2ull * i];
    if (words) atomicOr(words + (d.w & mask), frag_bloom_bits(d.z));
    const uint32_t b = d.y >> (32 - kFragL1Log2Bits);
    atomicOr(l1 + (b >> 5), 1u << (b & 31));
  }
}

// ------------------------------------------------------------------------------ host
namespace {

using KernelFn = const void*;

struct Geom {
  KernelFn count, emit;
  int threads;
  uint32_t tile_win, smem_count, smem_emit;
};

template <int SIG>
Geom geom_t(uint32_t layout) {
  using G = FragGeom<SIG>;
  const bool s = layout == kLayoutSorted;
  return Geom{s ? (KernelFn)frag_count_kernel<SIG, kLayoutSorted> : (KernelFn)frag_count_kernel<SIG, kLayoutHash>,
              s ? (KernelFn)frag_emit_kernel<SIG, kLayoutSorted> : (KernelFn)frag_emit_kernel<SIG, kLayoutHash>,
              G::kThreads, G::kTileWin, G::kSmemCount, G::kSmemEmit};
}

bool geom(int sig, uint32_t layout, Geom* g) {
  switch (sig) {
    case kSigMd5: *g = geom_t<kSigMd5>(layout); return true;
    case kSigMd5NoPad: *g = geom_t<kSigMd5NoPad>(layout); return true;
    case kSigDjb2: *g = geom_t<kSigDjb2>(layout); return true;
    default: return false;
  }
}

struct FragDev {
  bool ready = false;
  int count_blocks[3][2] = {};
};
std::mutex g_frag_mu;
FragDev g_frag_dev[64];

// Shared-memory attributes and resident blocks per SM of every fragment kernel, once per device.
int frag_device(FragDev** out) {
  int dev;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_frag_mu);
  FragDev& d = g_frag_dev[dev];
  if (!d.ready) {
    for (int sig = 0; sig < 3; sig++)
      for (uint32_t l = 0; l < 2; l++) {
        Geom g;
        geom(sig, l, &g);
        if ((e = cudaFuncSetAttribute(g.count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_count)) !=
            cudaSuccess)
          return (int)e;
        if ((e = cudaFuncSetAttribute(g.emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_emit)) !=
            cudaSuccess)
          return (int)e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.count_blocks[sig][l], g.count, g.threads,
                                                               g.smem_count)) != cudaSuccess)
          return (int)e;
        if (d.count_blocks[sig][l] < 1) return (int)cudaErrorInvalidConfiguration;
      }
    d.ready = true;
  }
  *out = &d;
  return 0;
}

FragParams make_params(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base,
                       uint32_t* status) {
  FragParams p;
  memset(&p, 0, sizeof p);
  p.tab = tab;
  p.image = image;
  p.n_bytes = n_bytes;
  p.n_windows = frag_windows(n_bytes);
  p.n_tiles = frag_tiles((int)tab.sig, n_bytes);
  p.tile_base = tile_base;
  p.status = status;
  p.one = 1u;
  return p;
}

}  // namespace

uint64_t frag_windows(uint64_t n_bytes) { return n_bytes >= 64 ? (n_bytes - 64) / kFragStride + 1 : 0; }

uint64_t frag_tiles(int sig, uint64_t n_bytes) {
  Geom g;
  if (!geom(sig, kLayoutHash, &g)) return 0;
  return (frag_windows(n_bytes) + g.tile_win - 1) / g.tile_win;
}

bool frag_sig_supported(int sig) { return sig == kSigMd5 || sig == kSigMd5NoPad || sig == kSigDjb2; }

int frag_digests(int sig, const uint8_t* arena, uint64_t n, uint4* dig, uint8_t* trivial, int sms, void* stream) {
  if (!n) return 0;
  const unsigned g = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8);
  cudaStream_t st = (cudaStream_t)stream;
  if (sig == kSigMd5) frag_digest_kernel<kSigMd5><<<g, 256, 0, st>>>(arena, n, dig, trivial, 1u);
  else if (sig == kSigMd5NoPad) frag_digest_kernel<kSigMd5NoPad><<<g, 256, 0, st>>>(arena, n, dig, trivial, 1u);
  else if (sig == kSigDjb2) frag_digest_kernel<kSigDjb2><<<g, 256, 0, st>>>(arena, n, dig, trivial, 1u);
  else return (int)cudaErrorInvalidValue;
  return (int)cudaGetLastError();
}

int frag_bloom(const uint4* slots, uint32_t n_slots, uint32_t* words, uint32_t mask, uint32_t* l1, int sms,
               void* stream) {
  const unsigned g = (unsigned)std::min<uint64_t>((n_slots + 255) / 256, (uint64_t)sms * 8);
  frag_bloom_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(slots, n_slots, words, mask, l1);
  return (int)cudaGetLastError();
}

int frag_window_sigs(int sig, const uint8_t* image, uint64_t n_bytes, uint4* out, int sms, void* stream) {
  const uint64_t n_win = frag_windows(n_bytes);
  if (!n_win) return 0;
  const void* fn;
  uint32_t win, bytes;
  switch (sig) {
    case kSigMd5:
      fn = (const void*)frag_window_sig_kernel<kSigMd5>;
      win = FragGeom<kSigMd5>::kTileWin;
      bytes = FragGeom<kSigMd5>::kTileBytes;
      break;
    case kSigMd5NoPad:
      fn = (const void*)frag_window_sig_kernel<kSigMd5NoPad>;
      win = FragGeom<kSigMd5NoPad>::kTileWin;
      bytes = FragGeom<kSigMd5NoPad>::kTileBytes;
      break;
    case kSigDjb2:
      fn = (const void*)frag_window_sig_kernel<kSigDjb2>;
      win = FragGeom<kSigDjb2>::kTileWin;
      bytes = FragGeom<kSigDjb2>::kTileBytes;
      break;
    default: return (int)cudaErrorInvalidValue;
  }
  const uint64_t tiles = (n_win + win - 1) / win;
  const uint32_t smem = 8 * bytes;  // 8 warps of 256 threads
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const unsigned grid = (unsigned)std::min<uint64_t>((tiles + 7) / 8, (uint64_t)sms * 8);
  uint32_t one = 1u;
  void* args[] = {&image, &n_bytes, (void*)&n_win, (void*)&tiles, &out, &one};
  return (int)cudaLaunchKernel(fn, dim3(grid), dim3(256), args, smem, (cudaStream_t)stream);
}

int frag_count(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base, uint64_t* tile_ntrip,
               uint32_t* status, unsigned long long* rejected, int sms, void* stream) {
  FragParams p = make_params(tab, image, n_bytes, tile_base, status);
  p.rejected = rejected;
  if (!p.n_tiles) return 0;
  FragDev* d;
  int rc = frag_device(&d);
  if (rc) return rc;
  Geom g;
  if (!geom((int)tab.sig, tab.layout, &g)) return (int)cudaErrorInvalidValue;
  if (tab.sig == kSigDjb2 && !tab.frag_l1) return (int)cudaErrorInvalidValue;  // the kernel copies it in
  p.tile_ntrip = tile_ntrip;
  const uint64_t cap = (uint64_t)sms * (uint64_t)d->count_blocks[tab.sig][tab.layout];
  const uint64_t warps_per_block = (uint64_t)g.threads / 32;
  const unsigned grid = (unsigned)std::min<uint64_t>((p.n_tiles + warps_per_block - 1) / warps_per_block, cap);
  void* args[] = {&p};
  return (int)cudaLaunchKernel(g.count, dim3(grid), dim3(g.threads), args, g.smem_count, (cudaStream_t)stream);
}

int frag_emit(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base,
              const uint64_t* tile_ntrip, const uint64_t* tile_off, uint32_t* list, MatchOut* out, uint64_t out_cap,
              uint32_t* status, int sms, void* stream, int* launches) {
  FragParams p = make_params(tab, image, n_bytes, tile_base, status);
  if (!p.n_tiles) return 0;
  FragDev* d;
  int rc = frag_device(&d);
  if (rc) return rc;
  Geom g;
  if (!geom((int)tab.sig, tab.layout, &g)) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* count = list + p.n_tiles;
  cudaError_t e = cudaMemsetAsync(count, 0, 4, st);
  if (e != cudaSuccess) return (int)e;
  const unsigned gl = (unsigned)std::min<uint64_t>((p.n_tiles + 255) / 256, (uint64_t)sms * 4);
  frag_hit_list_kernel<<<gl, 256, 0, st>>>(tile_ntrip + tile_base, p.n_tiles, list, count);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  p.tile_off = tile_off;
  p.hit_tiles = list;
  p.n_hit_tiles = count;
  p.out = out;
  p.out_cap = out_cap;
  const uint64_t warps_per_block = (uint64_t)g.threads / 32;
  const unsigned grid = (unsigned)std::min<uint64_t>((p.n_tiles + warps_per_block - 1) / warps_per_block,
                                                     (uint64_t)sms * 2);
  void* args[] = {&p};
  e = cudaLaunchKernel(g.emit, dim3(grid), dim3(g.threads), args, g.smem_emit, st);
  if (launches) *launches += 2;
  return (int)e;
}

}  // namespace cvk
