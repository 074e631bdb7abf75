// cv_scan_noalloc: a scan of one device-resident image that allocates no memory at all.
//
// Who needs it: callers that must not allocate while they scan. Examples are code running in
// a real-time or interrupt-driven ingest loop (a network tap handing over fixed buffers),
// processes whose device memory is fully reserved up front by another allocator, and hosts
// that forbid allocation after start-up. cudaMalloc can block, fail, or synchronize the
// device, and none of that is acceptable there. cv_scan draws its scratch from a memory pool;
// this entry point instead uses one fixed scratch array that lives in the library's own
// device memory image, so no allocation happens on any call.
//
// Limits and sharing rules:
//   - The scratch array (kNoAllocScratchBytes, a little over 8 MiB) is part of the library and
//     stays resident on every GPU that loads the library, until the process exits.
//   - An image may hold at most CV_NOALLOC_MAX_SECTORS whole sectors (256 MiB); larger
//     requests are refused with CV_EINVAL before any work is queued.
//   - Every call on a device uses the same array, and it keeps the previous call's contents.
//     The status word is cleared at the start of each call; the kernels rewrite everything
//     else they read. Two calls whose work overlaps on the GPU (different streams or host
//     threads without ordering) race on the array and give wrong results: serialize them.
//   - The first call on each device does a one-time set-up with that device current (the
//     array's device address, kernel attributes, occupancy). Every call copies its segment
//     descriptor from host memory and waits for its stream, so no call can be captured into a
//     CUDA graph: a call on a capturing stream is refused with CV_EINVAL before any work.
//   - On an error return the output buffer's contents are undefined; when the scan failed (a
//     device wait timed out or a lookup ran past its bound) nothing is written to it.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "cv.h"
#include "cv_internal.h"
#include "cv_launch.h"
#include "runtime.h"

using namespace cvk;

namespace {

// Scratch layout (offsets in bytes); sized for CV_NOALLOC_MAX_SECTORS with the smallest tile.
constexpr uint64_t kMaxSectors = CV_NOALLOC_MAX_SECTORS;
constexpr uint64_t kMaxTiles = kMaxSectors / 32 + 32;  // output tiles of 32 sectors, plus a ragged tile
constexpr uint64_t kOffSeg = 128;                               // Segment
constexpr uint64_t kOffCounters = 256;                          // seg_off[1], total, status
constexpr uint64_t kOffSums = 512;                              // chunk sums of the offset pass
constexpr uint64_t kOffNhit = kOffSums + 1024;                  // u32 per tile
constexpr uint64_t kOffNtrip = kOffNhit + ((kMaxTiles * 4 + 255) / 256) * 256;   // u64 per tile
constexpr uint64_t kOffToff = kOffNtrip + ((kMaxTiles * 8 + 255) / 256) * 256;   // u64 per tile
constexpr uint64_t kOffHits = kOffToff + ((kMaxTiles * 8 + 255) / 256) * 256;    // uint4 per sector slot
constexpr uint64_t kHitSlots = kMaxTiles * 32;
constexpr uint64_t kNoAllocScratchBytes = kOffHits + kHitSlots * 16;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDev {
  bool ready = false;
  uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
  int blocks_per_sm = 0;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};

constexpr int kMaxDev = 64;
std::mutex g_mu;
NoAllocDev g_dev[kMaxDev];

int fail(cudaError_t e) {
  cudaGetLastError();
  (void)e;
  return CV_ECUDA;
}

// One-time set-up for the current device.
int setup(int dev, NoAllocDev** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDev& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(e);
    int n;
    const ScanCfg& cfg = scan_configs(&n)[0];
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(e);
    for (int kind = 0; kind < kTableKinds; kind++) {
      if (!cfg.scan_fn[kind]) continue;
      e = cudaFuncSetAttribute(cfg.scan_fn[kind], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
      if (e != cudaSuccess) return fail(e);
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.blocks_per_sm, cfg.scan_fn[0], cfg.threads, cfg.smem);
    if (e != cudaSuccess || d.blocks_per_sm < 1) return fail(e);
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return fail(e);
    d.encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    d.scratch = (uint8_t*)p;
    d.ready = true;
  }
  *out = &d;
  return CV_OK;
}

}  // namespace

extern "C" int cv_scan_noalloc(const cv_master* m, const void* image, uint64_t n_bytes, cv_match* out,
                               uint64_t out_capacity, uint64_t* n_out, void* stream_) {
  if (!m || !n_out || (n_bytes >= CV_SECTOR_BYTES && !image)) return CV_EINVAL;
  if (out_capacity && !out) return CV_EINVAL;
  const uint64_t S = n_bytes / CV_SECTOR_BYTES;
  if (S > kMaxSectors) return CV_EINVAL;
  if (((uintptr_t)image & 15u) || ((uintptr_t)out & 15u)) return CV_EINVAL;
  *n_out = 0;
  TableView tab;
  int mdev;
  if (master_view(m, &tab, &mdev) != CV_OK || tab.unit != kUnitSector) return CV_EINVAL;
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();  // cudaSetDevice binds the primary context for the driver-API calls below
    return CV_ENODEV;
  }
  if (dev != mdev) return CV_EINVAL;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream_, &cap) != cudaSuccess) {
    cudaGetLastError();
    return CV_EINVAL;
  }
  if (cap != cudaStreamCaptureStatusNone) return CV_EINVAL;
  if (S == 0) return CV_OK;
  NoAllocDev* d;
  int rc = setup(dev, &d);
  if (rc != CV_OK) return rc;
  cudaStream_t stream = (cudaStream_t)stream_;
  const ScanCfg& cfg = scan_config_for(0, table_kind(tab), nullptr);

  uint8_t* sc = d->scratch;
  Segment* seg_d = (Segment*)(sc + kOffSeg);
  uint64_t* seg_off_d = (uint64_t*)(sc + kOffCounters);
  uint64_t* total_d = seg_off_d + 1;
  uint32_t* status_d = (uint32_t*)(seg_off_d + 2);
  uint32_t* tile_nhit = (uint32_t*)(sc + kOffNhit);
  uint64_t* tile_ntrip = (uint64_t*)(sc + kOffNtrip);
  uint64_t* tile_off = (uint64_t*)(sc + kOffToff);
  uint4* hit_rec = (uint4*)(sc + kOffHits);

  // The tensor map travels in the kernel's parameters; the segment descriptor is also copied
  // to the scratch array for the compaction kernels.
  ScanParams p;
  memset(&p, 0, sizeof p);
  CUtensorMap& map = p.maps[0];
  cuuint64_t dims[2] = {128, (cuuint64_t)S};
  cuuint64_t strides[1] = {CV_SECTOR_BYTES};
  cuuint32_t box[2] = {(cuuint32_t)(cfg.BOXB / 4), (cuuint32_t)(cfg.T / ((cfg.T + 255) / 256))};
  cuuint32_t es[2] = {1, 1};
  CUresult cr = d->encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(image), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          cfg.BOXB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return CV_ECUDA;
  Segment seg;
  seg.n_sectors = S;
  seg.tile_base = 0;
  seg.sector_base = 0;
  seg.row_base = 0;
  seg.image = 0;
  seg.map = 0;
  seg.bytes = (const uint8_t*)image;
  const uint64_t n_tiles = (S + cfg.T - 1) / cfg.T;
  const uint64_t n_out_tiles = n_tiles * (uint64_t)(cfg.T / 32);  // output tiles of 32 sectors
  if (n_out_tiles > kMaxTiles) return CV_EINVAL;                   // tile wider than the layout allows

  cudaError_t e;
  if ((e = cudaMemsetAsync(status_d, 0, 4, stream)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(seg_d, &seg, sizeof seg, cudaMemcpyHostToDevice, stream)) != cudaSuccess) return fail(e);

  p.segs = seg_d;
  p.n_segs = 1;
  p.map_base = 0;
  p.one = 1u;
  p.tile_begin = 0;
  p.n_tiles = n_tiles;
  p.tab = tab;
  p.hit_rec = hit_rec;
  p.tile_nhit = tile_nhit;
  p.tile_ntrip = tile_ntrip;
  p.status = status_d;
  const uint64_t grid = n_tiles < (uint64_t)d->sms * d->blocks_per_sm ? n_tiles : (uint64_t)d->sms * d->blocks_per_sm;
  void* sargs[] = {&p};
  if ((e = cudaLaunchKernel(cfg.scan_fn[table_kind(tab)], dim3((unsigned)grid), dim3(cfg.threads), sargs, cfg.smem,
                            stream)) !=
      cudaSuccess)
    return fail(e);
  uint32_t one = 1;
  uint64_t nt = n_out_tiles;
  const Segment* segc = seg_d;
  static_assert((kMaxTiles + 4095) / 4096 + 1 <= 1024 / 8, "offset scratch");
  if ((e = (cudaError_t)launch_tile_offsets(tile_ntrip, nt, tile_off, segc, one, (uint32_t)(cfg.T / 32), seg_off_d,
                                            total_d, (uint64_t*)(sc + kOffSums), stream, status_d)) != cudaSuccess)
    return fail(e);
  if ((e = (cudaError_t)launch_expand(cfg, hit_rec, tile_nhit, tile_off, nt, segc, one, tab, (MatchOut*)out,
                                      out_capacity, status_d, d->sms, stream)) != cudaSuccess)
    return fail(e);
  uint64_t hc[2] = {0, 0};  // total, status
  if ((e = cudaMemcpyAsync(hc, total_d, 16, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return fail(e);
  const uint32_t st = (uint32_t)hc[1];
  *n_out = hc[0];
  if (st & kStTimeout) return CV_ETIMEOUT;
  if (hc[0] > out_capacity) return CV_ERANGE;
  if (st) return CV_ECORRUPT;
  return CV_OK;
}
