// Fragment scan (paper Section 5): every 64-byte window of a disk image that starts at a
// multiple of 4 bytes is looked up among the whole 64-byte fragments of the master files, to
// find small files (logos, small images) embedded in other files at any 32-bit offset.
//
// Work layout. A tile is kFragTileWin = 256 x 33 consecutive windows: 33,792 bytes of window
// starts, 33,856 bytes staged (the last window's tail). One 1-D bulk TMA copy per tile brings
// the bytes into shared memory, double-buffered over a persistent grid with mbarrier completion
// and bounded waits. Thread t takes windows [33 t, 33 t + 33) of the tile; with an odd count the
// 32 threads of a warp read 32 different banks at every step.
//
//   djb2-64 (Eq. 1) is rolled. With P(x) the base-33 Horner value of a 4-byte word x and
//   g = h - 5381 * 33^64, a window W_k of words x_k .. x_{k+15} has g(W_k) = sum_q
//   P(x_{k+q}) 33^{4 (15 - q)}, so g(W_{k+1}) = 33^4 g(W_k) - 33^64 P(x_k) + P(x_{k+16})
//   (mod 2^64): after a thread's first window each one costs one word and a few multiply-adds.
//   MD5 is computed per window (two compressions, or one without the padding block).
//
// Passes (no worst-case hit buffer). The count kernel hashes every window, tests its key in a
// one-word Bloom filter, resolves the candidates (probe; byte confirmation for djb2) and writes
// the tile's triple count. An exclusive scan gives every tile its output offset. The emit kernel
// redoes only the tiles that have triples and writes them in window order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "cv_launch.h"
#include "scan_kernel.cuh"

namespace cvk {

constexpr int kFragThreads = 256;
constexpr int kFragWPT = 33;                                    // windows per thread per tile
constexpr uint32_t kFragTileWin = kFragThreads * kFragWPT;      // 8448
constexpr uint32_t kFragTileStep = kFragTileWin * kFragStride;  // bytes between tile starts
constexpr uint32_t kFragTileBytes = kFragTileStep + 64;         // bytes staged per tile
constexpr uint32_t kFragSmemCount = 2 * kFragTileBytes;         // two stages
constexpr uint32_t kFragSmemEmit = kFragTileBytes;

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
};

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                          uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}

// Base-33 Horner value of a little-endian word: byte 0 first (Eq. 1 over four bytes).
__device__ __forceinline__ uint32_t horner33(uint32_t w) {
  return (((w & 0xFFu) * 33u + ((w >> 8) & 0xFFu)) * 33u + ((w >> 16) & 0xFFu)) * 33u + (w >> 24);
}

__device__ __forceinline__ bool frag_bloom_test(const TableView& tab, uint32_t d2, uint32_t d3) {
  const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(tab.bloom) + (d3 & tab.bloom_mask));
  const uint32_t m = (1u << (d2 & 31)) | (1u << ((d2 >> 5) & 31)) | (1u << ((d2 >> 10) & 31));
  return (w & m) == m;
}

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
    if constexpr (SIG == kSigMd5) md5_compress_block_padding(d);
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

// Candidate windows of this thread (bit i: window w0 + i passed the Bloom test; every valid
// window when the table has no filter). n_valid: the thread's windows inside the image.
template <int SIG>
__device__ __forceinline__ uint64_t frag_candidates(const FragParams& p, const uint32_t* ws, uint32_t w0,
                                                    uint32_t n_valid) {
  uint64_t cand = 0;
  if constexpr (SIG == kSigDjb2) {
    uint32_t P[16];
    uint64_t g = 0;
#pragma unroll
    for (int q = 0; q < 16; q++) {
      P[q] = horner33(ws[w0 + q]);
      g = g * kD33x4 + P[q];
    }
#pragma unroll
    for (int i = 0; i < kFragWPT; i++) {
      if (i > 0) {
        const uint32_t pin = horner33(ws[w0 + i + 15]);
        g = g * kD33x4 - (uint64_t)P[(i - 1) & 15] * kD33x64 + pin;
        P[(i - 1) & 15] = pin;
      }
      uint32_t d[4];
      frag64_words(g + kDjbInit, d);
      if ((uint32_t)i < n_valid && (!p.tab.use_bloom || frag_bloom_test(p.tab, d[2], d[3]))) cand |= 1ull << i;
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

template <int SIG, int LAYOUT>
__device__ __forceinline__ uint64_t frag_thread_count(const FragParams& p, const uint32_t* ws, uint32_t w0,
                                                      uint64_t cand) {
  uint64_t n = 0;
  while (cand) {
    const int i = __ffsll((long long)cand) - 1;
    cand &= cand - 1;
    uint32_t off, cnt;
    n += frag_resolve<SIG, LAYOUT>(p, ws, w0 + (uint32_t)i, off, cnt);
  }
  return n;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src, bool up) {
  uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  lo = up ? __shfl_up_sync(0xFFFFFFFFu, lo, src) : __shfl_sync(0xFFFFFFFFu, lo, src);
  hi = up ? __shfl_up_sync(0xFFFFFFFFu, hi, src) : __shfl_sync(0xFFFFFFFFu, hi, src);
  return ((uint64_t)hi << 32) | lo;
}

// Block-wide exclusive scan of one u64 per thread; *total receives the sum (all threads).
__device__ __forceinline__ uint64_t block_exclusive_u64(uint64_t v, uint64_t* warp_sums, uint64_t* total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t x = shfl_u64(incl, d, true);
    if (lane >= d) incl += x;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    constexpr int kWarps = kFragThreads / 32;
    uint64_t s = lane < kWarps ? warp_sums[lane] : 0, si = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t x = shfl_u64(si, d, true);
      if (lane >= d) si += x;
    }
    if (lane < kWarps) warp_sums[lane] = si - s;
    if (lane == kWarps - 1) warp_sums[kWarps] = si;
  }
  __syncthreads();
  const uint64_t r = warp_sums[warp] + incl - v;
  *total = warp_sums[kFragThreads / 32];
  return r;
}

// Thread 0: issue tile `tile` into the stage at smem address dst (completion on bar).
__device__ __forceinline__ void frag_issue(const FragParams& p, uint64_t tile, uint32_t dst, uint32_t bar,
                                           uint64_t policy) {
  const uint64_t start = tile * kFragTileStep;
  const uint64_t left = p.n_bytes - start;
  const uint32_t avail = left < kFragTileBytes ? (uint32_t)left : kFragTileBytes;
  const uint32_t bulk = avail & ~15u;
  mbar_arrive_expect_tx(bar, bulk);
  if (bulk) bulk_load(dst, p.image + start, bulk, bar, policy);
}

// Thread 0: the bytes of the tile past its last whole 16-byte chunk (the bulk copy moves whole
// chunks only), with plain loads.
__device__ __forceinline__ void frag_tail(const FragParams& p, uint64_t tile, uint8_t* buf) {
  const uint64_t start = tile * kFragTileStep;
  const uint64_t left = p.n_bytes - start;
  const uint32_t avail = left < kFragTileBytes ? (uint32_t)left : kFragTileBytes;
  for (uint32_t b = avail & ~15u; b < avail; b++) buf[b] = p.image[start + b];
}

__device__ __forceinline__ uint32_t frag_valid(const FragParams& p, uint64_t tile, uint32_t w0) {
  const uint64_t k0 = tile * kFragTileWin + w0;
  if (k0 >= p.n_windows) return 0u;
  const uint64_t left = p.n_windows - k0;
  return left < (uint64_t)kFragWPT ? (uint32_t)left : (uint32_t)kFragWPT;
}

template <int SIG, int LAYOUT>
__global__ void __launch_bounds__(kFragThreads) frag_count_kernel(const __grid_constant__ FragParams p) {
  extern __shared__ __align__(128) uint8_t fsm[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ uint32_t abort_flag;
  __shared__ uint64_t warp_sums[kFragThreads / 32 + 1];
  const int tid = threadIdx.x;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(smem_addr(&full[0]), 1);
    mbar_init(smem_addr(&full[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint64_t policy = l2_evict_first_policy();
  const uint64_t grid = gridDim.x;
  // Stage s holds the tiles of iterations i with i & 1 == s; the k-th of them completes phase k
  // of its barrier. Thread 0 issues the first two tiles, then each tile two iterations ahead.
  if (tid == 0)
    for (int s = 0; s < 2; s++) {
      const uint64_t t = blockIdx.x + s * grid;
      if (t < p.n_tiles) frag_issue(p, t, smem_addr(fsm + s * kFragTileBytes), smem_addr(&full[s]), policy);
    }
  uint64_t i = 0;
  bool aborted = false;
  for (;; i++) {
    const uint64_t tile = blockIdx.x + i * grid;
    if (tile >= p.n_tiles) break;
    const int s = (int)(i & 1);
    uint8_t* buf = fsm + s * kFragTileBytes;
    const bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)(i >> 1) & 1u, &abort_flag, p.status);
    if (!__syncthreads_and(ok)) {
      aborted = true;
      break;
    }
    if (tid == 0) frag_tail(p, tile, buf);
    __syncthreads();
    const uint32_t* ws = reinterpret_cast<const uint32_t*>(buf);
    const uint32_t w0 = (uint32_t)tid * kFragWPT;
    const uint64_t cand = frag_candidates<SIG>(p, ws, w0, frag_valid(p, tile, w0));
    const uint64_t n = frag_thread_count<SIG, LAYOUT>(p, ws, w0, cand);
    uint64_t total;
    block_exclusive_u64(n, warp_sums, &total);
    if (tid == 0) p.tile_ntrip[p.tile_base + tile] = total;
    __syncthreads();  // every thread is done with stage s (and with warp_sums)
    const uint64_t next = tile + 2 * grid;
    if (tid == 0 && next < p.n_tiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      frag_issue(p, next, smem_addr(buf), smem_addr(&full[s]), policy);
    }
  }
  if (aborted && tid == 0) {
    // Iterations i and i + 1 had their copies issued (when their tiles exist) and not waited
    // for: let them land, each wait bounded, before the block's shared memory goes away.
    volatile uint32_t never = 0;
    for (uint64_t j = i; j < i + 2 && blockIdx.x + j * grid < p.n_tiles; j++)
      if (!mbar_wait(smem_addr(&full[j & 1]), (uint32_t)(j >> 1) & 1u, &never, p.status)) break;
  }
}

// Tiles of one image with triples, as a list of local tile indices (any order).
__global__ void frag_hit_list_kernel(const uint64_t* tile_ntrip, uint64_t n_tiles, uint32_t* list, uint32_t* count) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += (uint64_t)gridDim.x * blockDim.x)
    if (tile_ntrip[t]) list[atomicAdd(count, 1u)] = (uint32_t)t;
}

template <int SIG, int LAYOUT>
__global__ void __launch_bounds__(kFragThreads) frag_emit_kernel(const __grid_constant__ FragParams p) {
  extern __shared__ __align__(128) uint8_t fsm[];
  __shared__ __align__(8) uint64_t full;
  __shared__ uint32_t abort_flag;
  __shared__ uint64_t warp_sums[kFragThreads / 32 + 1];
  const int tid = threadIdx.x;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(smem_addr(&full), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint64_t policy = l2_evict_first_policy();
  const uint32_t n_list = *(volatile const uint32_t*)p.n_hit_tiles;
  uint32_t phase = 0;
  for (uint32_t j = blockIdx.x; j < n_list; j += gridDim.x) {
    const uint64_t tile = p.hit_tiles[j];
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      frag_issue(p, tile, smem_addr(fsm), smem_addr(&full), policy);
    }
    const bool ok = mbar_wait(smem_addr(&full), phase & 1u, &abort_flag, p.status);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {  // the copy may still land: wait for it (bounded) before leaving
        volatile uint32_t never = 0;
        mbar_wait(smem_addr(&full), phase & 1u, &never, p.status);
      }
      return;
    }
    phase++;
    if (tid == 0) frag_tail(p, tile, fsm);
    __syncthreads();
    const uint32_t* ws = reinterpret_cast<const uint32_t*>(fsm);
    const uint32_t w0 = (uint32_t)tid * kFragWPT;
    const uint64_t cand = frag_candidates<SIG>(p, ws, w0, frag_valid(p, tile, w0));
    const uint64_t n = frag_thread_count<SIG, LAYOUT>(p, ws, w0, cand);
    uint64_t total;
    uint64_t pos = p.tile_off[p.tile_base + tile] + block_exclusive_u64(n, warp_sums, &total);
    uint64_t c = cand;
    while (c) {
      const int i = __ffsll((long long)c) - 1;
      c &= c - 1;
      const uint32_t w = w0 + (uint32_t)i;
      uint32_t off, cnt;
      if (!frag_resolve<SIG, LAYOUT>(p, ws, w, off, cnt)) continue;
      const uint64_t k = tile * kFragTileWin + w;
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
    __syncthreads();  // the stage is free again
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
      if constexpr (SIG == kSigMd5) md5_compress_block_padding(d);
    }
    dig[m] = make_uint4(d[0], d[1], d[2], d[3]);
    trivial[m] = diff == 0u ? 1 : 0;
  }
}

// One-word Bloom filter of a fragment table: every occupied slot sets 3 bits (from d2) of word
// d3 & mask.
__global__ void frag_bloom_kernel(const uint4* slots, uint32_t n_slots, uint32_t* words, uint32_t mask) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
    if (slots[2ull * i + 1].y == 0u) continue;
    const uint4 d = slots[2ull * i];
    atomicOr(words + (d.w & mask), (1u << (d.z & 31)) | (1u << ((d.z >> 5) & 31)) | (1u << ((d.z >> 10) & 31)));
  }
}

// ------------------------------------------------------------------------------ host
namespace {

using KernelFn = const void*;

KernelFn count_fn(int sig, uint32_t layout) {
  const bool s = layout == kLayoutSorted;
  switch (sig) {
    case kSigMd5: return s ? (KernelFn)frag_count_kernel<kSigMd5, kLayoutSorted> : (KernelFn)frag_count_kernel<kSigMd5, kLayoutHash>;
    case kSigMd5NoPad:
      return s ? (KernelFn)frag_count_kernel<kSigMd5NoPad, kLayoutSorted> : (KernelFn)frag_count_kernel<kSigMd5NoPad, kLayoutHash>;
    case kSigDjb2: return s ? (KernelFn)frag_count_kernel<kSigDjb2, kLayoutSorted> : (KernelFn)frag_count_kernel<kSigDjb2, kLayoutHash>;
    default: return nullptr;
  }
}

KernelFn emit_fn(int sig, uint32_t layout) {
  const bool s = layout == kLayoutSorted;
  switch (sig) {
    case kSigMd5: return s ? (KernelFn)frag_emit_kernel<kSigMd5, kLayoutSorted> : (KernelFn)frag_emit_kernel<kSigMd5, kLayoutHash>;
    case kSigMd5NoPad:
      return s ? (KernelFn)frag_emit_kernel<kSigMd5NoPad, kLayoutSorted> : (KernelFn)frag_emit_kernel<kSigMd5NoPad, kLayoutHash>;
    case kSigDjb2: return s ? (KernelFn)frag_emit_kernel<kSigDjb2, kLayoutSorted> : (KernelFn)frag_emit_kernel<kSigDjb2, kLayoutHash>;
    default: return nullptr;
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
        if ((e = cudaFuncSetAttribute(count_fn(sig, l), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kFragSmemCount)) != cudaSuccess)
          return (int)e;
        if ((e = cudaFuncSetAttribute(emit_fn(sig, l), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kFragSmemEmit)) != cudaSuccess)
          return (int)e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.count_blocks[sig][l], count_fn(sig, l), kFragThreads,
                                                               kFragSmemCount)) != cudaSuccess)
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
  p.n_tiles = frag_tiles(n_bytes);
  p.tile_base = tile_base;
  p.status = status;
  p.one = 1u;
  return p;
}

}  // namespace

uint64_t frag_windows(uint64_t n_bytes) { return n_bytes >= 64 ? (n_bytes - 64) / kFragStride + 1 : 0; }

uint64_t frag_tiles(uint64_t n_bytes) { return (frag_windows(n_bytes) + kFragTileWin - 1) / kFragTileWin; }

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

int frag_bloom(const uint4* slots, uint32_t n_slots, uint32_t* words, uint32_t mask, int sms, void* stream) {
  const unsigned g = (unsigned)std::min<uint64_t>((n_slots + 255) / 256, (uint64_t)sms * 8);
  frag_bloom_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(slots, n_slots, words, mask);
  return (int)cudaGetLastError();
}

int frag_count(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base, uint64_t* tile_ntrip,
               uint32_t* status, int sms, void* stream) {
  FragParams p = make_params(tab, image, n_bytes, tile_base, status);
  if (!p.n_tiles) return 0;
  FragDev* d;
  int rc = frag_device(&d);
  if (rc) return rc;
  KernelFn fn = count_fn((int)tab.sig, tab.layout);
  if (!fn) return (int)cudaErrorInvalidValue;
  p.tile_ntrip = tile_ntrip;
  const uint64_t cap = (uint64_t)sms * (uint64_t)d->count_blocks[tab.sig][tab.layout];
  const unsigned grid = (unsigned)std::min<uint64_t>(p.n_tiles, cap);
  void* args[] = {&p};
  return (int)cudaLaunchKernel(fn, dim3(grid), dim3(kFragThreads), args, kFragSmemCount, (cudaStream_t)stream);
}

int frag_emit(const TableView& tab, const uint8_t* image, uint64_t n_bytes, uint64_t tile_base,
              const uint64_t* tile_ntrip, const uint64_t* tile_off, uint32_t* list, MatchOut* out, uint64_t out_cap,
              uint32_t* status, int sms, void* stream, int* launches) {
  FragParams p = make_params(tab, image, n_bytes, tile_base, status);
  if (!p.n_tiles) return 0;
  FragDev* d;
  int rc = frag_device(&d);
  if (rc) return rc;
  KernelFn fn = emit_fn((int)tab.sig, tab.layout);
  if (!fn) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* count = list + p.n_tiles;
  cudaError_t e = cudaMemsetAsync(count, 0, 4, st);
  if (e != cudaSuccess) return (int)e;
  const unsigned g = (unsigned)std::min<uint64_t>((p.n_tiles + 255) / 256, (uint64_t)sms * 4);
  frag_hit_list_kernel<<<g, 256, 0, st>>>(tile_ntrip + tile_base, p.n_tiles, list, count);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  p.tile_off = tile_off;
  p.hit_tiles = list;
  p.n_hit_tiles = count;
  p.out = out;
  p.out_cap = out_cap;
  const unsigned grid = (unsigned)std::min<uint64_t>(p.n_tiles, (uint64_t)sms * 4);
  void* args[] = {&p};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kFragThreads), args, kFragSmemEmit, st);
  if (launches) *launches += 2;
  return (int)e;
}

}  // namespace cvk
