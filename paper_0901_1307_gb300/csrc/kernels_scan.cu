// The scan configurations (assembled from scan_cfgs_*.cu), the offset pass and the launch of the
// second compaction pass.
#include <string.h>

#include <vector>

#include "compact.cuh"
#include "cv_launch.h"
#include "scan_kernel.cuh"

namespace cvk {

// ------------------------------------------------------------ offset pass (first of two)
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

// Exclusive scan of v (n values) into out in one pass, with *total = the sum of all: chunks of
// kOffChunk values, each scanned by one block; the blocks take chunks in ticket order and publish
// each chunk's sum (flag 1), then its inclusive prefix (flag 2), in one 64-bit word per chunk,
// and a block adds up its predecessors' published words back to the first inclusive one
// (decoupled look-back). A block only waits for chunks taken by blocks that started before it,
// and each wait is bounded by timeout_ns (kStTimeout in *status on expiry; the block then
// publishes what it has, so no wait depends on it for longer). state: chunks words, then the
// ticket, all zero before the launch. With nhit, the sum of the n hit counts is added to
// *nhit_sum in the same pass.
constexpr uint64_t kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbValue = (1ull << 62) - 1;

__global__ void __launch_bounds__(kOffThreads) lookback_scan_kernel(const uint64_t* v, uint64_t n, uint64_t* out,
                                                                    uint64_t* total, uint64_t* state, uint64_t chunks,
                                                                    const uint32_t* nhit,
                                                                    unsigned long long* nhit_sum, uint32_t* status,
                                                                    uint64_t timeout_ns) {
  __shared__ uint64_t wb[32];
  __shared__ uint64_t s_chunk, s_prefix;
  if (threadIdx.x == 0) s_chunk = atomicAdd(reinterpret_cast<unsigned long long*>(state + chunks), 1ull);
  __syncthreads();
  const uint64_t chunk = s_chunk;
  const uint64_t first = chunk * kOffChunk + (uint64_t)threadIdx.x * kOffItems;
  uint64_t x[kOffItems];
  uint64_t sum = 0;
  unsigned long long h = 0;
#pragma unroll
  for (int k = 0; k < kOffItems; k++) {
    const bool in = first + k < n;
    x[k] = in ? v[first + k] : 0ull;
    sum += x[k];
    if (nhit && in) h += nhit[first + k];
  }
  if (nhit) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, d);
    if ((threadIdx.x & 31) == 0 && h) atomicAdd(nhit_sum, h);
  }
  const uint64_t incl = block_inclusive_scan(sum, wb);
  if (threadIdx.x == kOffThreads - 1) {
    volatile uint64_t* st = state;
    uint64_t prefix = 0;
    if (chunk == 0) {
      st[0] = kLbIncl | incl;
    } else {
      st[chunk] = kLbAgg | incl;
      uint64_t q = chunk - 1;
      const uint64_t t0 = globaltimer_ns();
      while (true) {
        const uint64_t w = st[q];
        if ((w >> 62) == 2u) {
          prefix += w & kLbValue;
          break;
        }
        if ((w >> 62) == 1u) {  // chunk 0 always ends in an inclusive word, so q stays >= 0
          prefix += w & kLbValue;
          q--;
          continue;
        }
        if (globaltimer_ns() - t0 > timeout_ns) {
          atomicOr(status, kStTimeout);
          break;
        }
      }
      st[chunk] = kLbIncl | (prefix + incl);
    }
    s_prefix = prefix;
    if (chunk == chunks - 1) *total = prefix + incl;
  }
  __syncthreads();
  uint64_t run = s_prefix + incl - sum;
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

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing completes. The
// wait gives up after timeout_ns, sets kStTimeout and the kernel returns normally.
__global__ void wait_timeout_selftest_kernel(uint32_t* status, uint64_t timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool ok = mbar_wait(smem_addr(&bar), 0, &abort_flag, status, timeout_ns);
    if (ok) atomicOr(status, kStProbeBound);  // must not happen: nothing arrives
  }
}


// The configurations in table order. The first is the default (the fastest measured on GB300
// for the 32 GiB image workload) and the only one with digest-mode kernels; every one has scan
// kernels for all eight table kinds (four signatures x two layouts), so the batch autotuner can
// pick any of them for any table. The kernels are instantiated in scan_cfgs_{a,b,c}.cu, which
// compile in parallel.
static const std::vector<ScanCfg>& all_configs() {
  static const std::vector<ScanCfg> v = [] {
    std::vector<ScanCfg> out;
    for (auto part : {scan_cfgs_a, scan_cfgs_b, scan_cfgs_c}) {
      int n = 0;
      const ScanCfg* c = part(&n);
      out.insert(out.end(), c, c + n);
    }
    return out;
  }();
  return v;
}

const ScanCfg* scan_configs(int* n) {
  const std::vector<ScanCfg>& v = all_configs();
  *n = (int)v.size();
  return v.data();
}

const ScanCfg& scan_config_for(int cfg_i, int kind, int* used) {
  int n;
  const ScanCfg* c = scan_configs(&n);
  if (cfg_i < 0 || cfg_i >= n || kind < 0 || kind >= kTableKinds || !c[cfg_i].scan_fn[kind]) cfg_i = 0;
  if (used) *used = cfg_i;
  return c[cfg_i];
}

int preferred_config(int kind) {
  // Measured on GB300 (32 GiB image, 4,194,304-sector table, kernel time per call): MD5 and
  // MD5 without padding are bound by integer issue and fastest with the first configuration;
  // djb2-64 and CRC64 do far less arithmetic and are bound by the staging of the image, which
  // 128-byte stages of 128-sector tiles serve best (djb2-64 6,241 against 5,146 GB/s; CRC64 5,889
  // against 5,151).
  static const int light = [] {
    int n;
    const ScanCfg* c = scan_configs(&n);
    for (int i = 0; i < n; i++)
      if (strcmp(c[i].name, "t128_x1_s2_b128_p2") == 0) return i;
    return 0;
  }();
  const int sig = kind % 4;
  return (sig == kSigDjb2 || sig == kSigCrc64) ? light : 0;
}

const ScanCfg& digest_config_for(int cfg_i, int sig, int* used) {
  int n;
  const ScanCfg* c = scan_configs(&n);
  if (cfg_i < 0 || cfg_i >= n || sig < 0 || sig > kSigCrc64 || !c[cfg_i].digest_fn[sig]) cfg_i = 0;
  if (used) *used = cfg_i;
  return c[cfg_i];
}

int launch_expand(const ScanCfg& cfg, const uint4* hit_rec, const uint32_t* tile_nhit, const uint64_t* tile_off,
                  uint64_t n_out_tiles, const Segment* segs, uint32_t n_segs, const TableView& tab, MatchOut* out,
                  uint64_t out_cap, uint32_t* status, int sms, void* stream) {
  const uint2* post = tab.postings;
  const uint8_t* confirm = sig_is_weak((int)tab.sig) ? tab.confirm : nullptr;
  uint64_t g = (n_out_tiles * 32 + 255) / 256;
  if (g > (uint64_t)sms * 16) g = (uint64_t)sms * 16;
  if (g == 0) g = 1;
  void* args[] = {&hit_rec, &tile_nhit, &tile_off, &n_out_tiles, &segs, &n_segs, &post, &out, &out_cap, &status,
                  &confirm};
  return (int)cudaLaunchKernel(cfg.expand_fn, dim3((unsigned)g), dim3(256), args, 0, (cudaStream_t)stream);
}

int launch_wait_selftest(uint32_t* status, uint64_t timeout_ns, void* stream) {
  wait_timeout_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(status, timeout_ns);
  return (int)cudaGetLastError();
}

// Self-test of the look-back's bounded wait: two chunks and one block, whose ticket is set to 1
// so that it scans chunk 1 and waits for chunk 0, which no block takes. words: 4 * kOffChunk + 4
// u64 (two chunks of values, two of outputs, the total, two look-back words and the ticket),
// zeroed here.
static_assert(lookback_selftest_words() == 2 * kOffChunk + 2 * kOffChunk + 1 + 2 + 1, "self-test buffer");

int launch_lookback_selftest(uint64_t* words, uint32_t* status, uint64_t timeout_ns, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  uint64_t* v = words;
  uint64_t* out = v + 2 * kOffChunk;
  uint64_t* total = out + 2 * kOffChunk;
  uint64_t* state = total + 1;  // state[0], state[1]: the chunks' words; state[2]: the ticket
  cudaError_t e = cudaMemsetAsync(words, 0, lookback_selftest_words() * 8, stream);
  if (e != cudaSuccess) return (int)e;
  const uint64_t one = 1;
  if ((e = cudaMemcpyAsync(state + 2, &one, 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess) return (int)e;
  lookback_scan_kernel<<<1, kOffThreads, 0, stream>>>(v, 2 * kOffChunk, out, total, state, 2, nullptr, nullptr,
                                                      status, timeout_ns);
  return (int)cudaGetLastError();
}

uint64_t tile_offsets_scratch_words(uint64_t n_tiles) { return (n_tiles + kOffChunk - 1) / kOffChunk + 1; }

int launch_tile_offsets(const uint64_t* tile_ntrip, uint64_t n_tiles, uint64_t* tile_off, const Segment* segs,
                        uint32_t n_segs, uint32_t scale, uint64_t* seg_off, uint64_t* total, uint64_t* scratch,
                        void* stream_, uint32_t* status, const uint32_t* tile_nhit, uint64_t* nhit_sum) {
  cudaStream_t stream = (cudaStream_t)stream_;
  const uint64_t chunks = (n_tiles + kOffChunk - 1) / kOffChunk;
  cudaError_t e;
  if (chunks) {
    // the look-back words and the ticket start at zero
    if ((e = cudaMemsetAsync(scratch, 0, (chunks + 1) * 8, stream)) != cudaSuccess) return (int)e;
    lookback_scan_kernel<<<(unsigned)chunks, kOffThreads, 0, stream>>>(
        tile_ntrip, n_tiles, tile_off, total, scratch, chunks, tile_nhit,
        reinterpret_cast<unsigned long long*>(nhit_sum), status, kWaitTimeoutNs);
  } else if ((e = cudaMemsetAsync(total, 0, 8, stream)) != cudaSuccess) {
    return (int)e;
  }
  if (n_segs) segment_offsets_kernel<<<(n_segs + 255) / 256, 256, 0, stream>>>(tile_off, n_tiles, segs, n_segs, scale,
                                                                               total, seg_off);
  return (int)cudaGetLastError();
}

}  // namespace cvk
