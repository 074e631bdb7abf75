// Host runtime shared by the entry points: per-device context, pool temporaries, tensor maps,
// scan jobs and kernel launches over them.
#include "runtime.h"

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

namespace cvk {

namespace {
thread_local int g_last_cuda = 0;
constexpr int kMaxDevices = 64;
std::mutex g_ctx_mutex;
DevCtx g_ctx[kMaxDevices];

int find_cfg(const char* name) {
  int n;
  const ScanCfg* c = scan_configs(&n);
  for (int i = 0; i < n; i++)
    if (strcmp(c[i].name, name) == 0) return i;
  return -1;
}
}  // namespace

int cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? CV_ENOMEM : CV_ECUDA;
}

void set_last_cuda(int code) { g_last_cuda = code; }
int last_cuda() { return g_last_cuda; }

int get_ctx(DevCtx** out) {
  int dev;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_last_cuda = (int)e;
    cudaGetLastError();
    return CV_ENODEV;
  }
  if (dev < 0 || dev >= kMaxDevices) return CV_ENODEV;
  // Bind the device's primary context to the calling thread: the library also makes driver-API
  // calls (address ranges, tensor maps), which need a current context and do not create one, and
  // a thread that has made no runtime call yet has none.
  if ((e = cudaSetDevice(dev)) != cudaSuccess) {
    g_last_cuda = (int)e;
    cudaGetLastError();
    return CV_ENODEV;
  }
  std::lock_guard<std::mutex> lk(g_ctx_mutex);
  DevCtx& c = g_ctx[dev];
  if (!c.ready) {
    cudaDeviceProp prop;
    CV_CUDA(cudaGetDeviceProperties(&prop, dev));
    if (prop.major < 10) return CV_ENODEV;
    c.dev = dev;
    c.sms = prop.multiProcessorCount;
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    CV_CUDA(cudaMemPoolCreate(&c.pool, &pp));
    uint64_t thr = UINT64_MAX;
    CV_CUDA(cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &thr));
    CV_CUDA(cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking));
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    CV_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return CV_ENODEV;
    c.encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    fn = nullptr;
    CV_CUDA(cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q));
    c.address_range = (q == cudaDriverEntryPointSuccess) ? (PFN_cuMemGetAddressRange_v3020)fn : nullptr;
    int n;
    const ScanCfg* cfgs = scan_configs(&n);
    c.blocks_per_sm.assign(n, std::array<int, kTableKinds>{});
    c.blocks_per_sm_digest.assign(n, 0);
    for (int i = 0; i < n; i++) {
      for (int kind = 0; kind < kTableKinds; kind++) {
        if (!cfgs[i].scan_fn[kind]) continue;
        CV_CUDA(cudaFuncSetAttribute(cfgs[i].scan_fn[kind], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cfgs[i].smem));
        CV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.blocks_per_sm[i][kind], cfgs[i].scan_fn[kind],
                                                              cfgs[i].threads, cfgs[i].smem));
        if (c.blocks_per_sm[i][kind] < 1) return CV_ECUDA;
      }
      for (int sig = 0; sig < 4; sig++) {
        if (!cfgs[i].digest_fn[sig]) continue;
        CV_CUDA(cudaFuncSetAttribute(cfgs[i].digest_fn[sig], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cfgs[i].smem));
      }
      if (cfgs[i].digest_fn[0]) {
        CV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.blocks_per_sm_digest[i], cfgs[i].digest_fn[0],
                                                              cfgs[i].threads, cfgs[i].smem));
        if (c.blocks_per_sm_digest[i] < 1) return CV_ECUDA;
      }
    }
    if (!cfgs[0].digest_fn[0]) return CV_ECUDA;  // the default configuration serves every digest pass

    c.cfg_index = -1;
    const char* env = getenv("CV_SCAN_CONFIG");
    if (env && *env) {
      int k = find_cfg(env);
      if (k < 0) return CV_EINVAL;
      c.cfg_index = k;
    }
    c.ready = true;
  }
  *out = &c;
  return CV_OK;
}

Temps::~Temps() {
  for (void* p : ptrs) cudaFreeAsync(p, stream);
}

int Temps::alloc_bytes(void** out, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, ctx->pool, stream);
  if (e != cudaSuccess) return cuda_fail(e);
  ptrs.push_back(p);
  *out = p;
  return CV_OK;
}

int DevCtx::take_events(cudaEvent_t* ev, int n) {
  for (int i = 0; i < n; i++) ev[i] = nullptr;
  {
    std::lock_guard<std::mutex> lk(ev_mutex);
    for (int i = 0; i < n && !ev_free.empty(); i++) {
      ev[i] = ev_free.back();
      ev_free.pop_back();
    }
  }
  for (int i = 0; i < n; i++)
    if (!ev[i]) CV_CUDA(cudaEventCreate(&ev[i]));
  return CV_OK;
}

void DevCtx::give_events(cudaEvent_t* ev, int n) {
  std::lock_guard<std::mutex> lk(ev_mutex);
  for (int i = 0; i < n; i++) {
    if (ev[i]) ev_free.push_back(ev[i]);
    ev[i] = nullptr;
  }
}

int classify(DevCtx* ctx, const void* p, BufKind* kind) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *kind = kHost;
    return CV_OK;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    if (a.device != ctx->dev) return CV_EINVAL;
    *kind = kDevice;
  } else {
    *kind = kHost;
  }
  return CV_OK;
}

int make_tmap(DevCtx* ctx, const ScanCfg& cfg, const void* base, uint64_t n_rows, CUtensorMap* out) {
  cuuint64_t dims[2] = {128, (cuuint64_t)n_rows};
  cuuint64_t strides[1] = {kSector};
  cuuint32_t box[2] = {(cuuint32_t)(cfg.BOXB / 4), (cuuint32_t)(cfg.T / ((cfg.T + 255) / 256))};
  cuuint32_t es[2] = {1, 1};
  CUtensorMapSwizzle sw = cfg.BOXB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = ctx->encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    g_last_cuda = (int)r;
    return CV_ECUDA;
  }
  return CV_OK;
}

int Job::add(DevCtx* ctx, const ScanCfg& cfg, const void* base, uint64_t n_in, uint64_t sector_base, uint32_t image,
             bool share_alloc) {
  // Find (or make) the map this range is read through.
  uintptr_t row0_addr = (uintptr_t)base;
  uint64_t row_base = 0;
  int map = -1;
  if (base && share_alloc && ctx->address_range) {
    CUdeviceptr ab = 0;
    size_t asz = 0;
    if (ctx->address_range(&ab, &asz, (CUdeviceptr)(uintptr_t)base) == CUDA_SUCCESS && (ab & 15u) == 0 &&
        ((uintptr_t)base - ab) % kSector == 0 && asz / kSector < (1ull << 31)) {
      row0_addr = (uintptr_t)ab;
      row_base = ((uintptr_t)base - ab) / kSector;
      for (size_t k = 0; k < map_base.size(); k++)
        if (map_base[k] == row0_addr) map = (int)k;
      if (map < 0) {
        CUtensorMap m;
        CV_TRY(make_tmap(ctx, cfg, (const void*)ab, asz / kSector, &m));
        maps.push_back(m);
        map_base.push_back(row0_addr);
        map = (int)maps.size() - 1;
      }
    }
  }
  uint64_t done = 0;
  while (done < n_in) {
    const uint64_t n = std::min<uint64_t>(n_in - done, kMaxSegmentSectors);
    Segment s;
    s.n_sectors = n;
    s.tile_base = n_tiles;
    s.sector_base = sector_base + done;
    s.image = image;
    s.bytes = base ? (const uint8_t*)base + done * kSector : nullptr;
    if (map >= 0) {
      s.map = (uint32_t)map;
      s.row_base = row_base + done;
    } else {
      CUtensorMap m;
      memset(&m, 0, sizeof m);
      if (base) CV_TRY(make_tmap(ctx, cfg, (const uint8_t*)base + done * kSector, n, &m));
      maps.push_back(m);
      map_base.push_back(base ? (uintptr_t)base + done * kSector : 0);
      s.map = (uint32_t)(maps.size() - 1);
      s.row_base = 0;
    }
    segs.push_back(s);
    n_tiles += (n + cfg.T - 1) / cfg.T;
    n_sectors += n;
    done += n;
  }
  return CV_OK;
}

int Job::set_map(DevCtx* ctx, const ScanCfg& cfg, size_t s, const void* base) {
  Segment& sg = segs[s];
  CV_TRY(make_tmap(ctx, cfg, base, sg.n_sectors, &maps[sg.map]));
  map_base[sg.map] = (uintptr_t)base;
  sg.bytes = (const uint8_t*)base;
  return CV_OK;
}

int launch_range(DevCtx* ctx, int cfg_i, bool digest, const Job& job, const Segment* segs_d, size_t s0, size_t s1,
                 const ScanParams& base, cudaStream_t stream, int* launches) {
  int n;
  const ScanCfg& cfg = scan_configs(&n)[cfg_i];
  const void* fn = digest ? cfg.digest_fn[base.tab.sig] : cfg.scan_fn[table_kind(base.tab)];
  if (!fn) return CV_EINVAL;  // the caller picks a configuration built for the signature
  const int bps = digest ? ctx->blocks_per_sm_digest[cfg_i] : ctx->blocks_per_sm[cfg_i][table_kind(base.tab)];
  if (bps < 1) return CV_EINVAL;
  size_t a = s0;
  while (a < s1) {
    // extend the launch while its segments' maps fit in one parameter block
    uint32_t lo = job.segs[a].map, hi = lo;
    size_t b = a + 1;
    while (b < s1) {
      const uint32_t m = job.segs[b].map;
      const uint32_t nlo = std::min(lo, m), nhi = std::max(hi, m);
      if (nhi - nlo + 1 > (uint32_t)kMapsPerLaunch) break;
      lo = nlo;
      hi = nhi;
      b++;
    }
    ScanParams p;
    memset(&p, 0, sizeof p);
    p.tab = base.tab;
    p.hit_rec = base.hit_rec;
    p.tile_nhit = base.tile_nhit;
    p.tile_ntrip = base.tile_ntrip;
    p.status = base.status;
    p.digests = base.digests;
    p.trivial = base.trivial;
    p.rejected = base.rejected;
    for (uint32_t k = lo; k <= hi; k++) p.maps[k - lo] = job.maps[k];
    p.map_base = lo;
    p.one = 1u;
    p.segs = segs_d + a;
    p.n_segs = (uint32_t)(b - a);
    p.tile_begin = job.segs[a].tile_base;
    const uint64_t tile_end = (b < job.segs.size()) ? job.segs[b].tile_base : job.n_tiles;
    p.n_tiles = tile_end - p.tile_begin;
    if (p.n_tiles) {
      const uint64_t grid = std::min<uint64_t>(p.n_tiles, (uint64_t)ctx->sms * bps);
      void* args[] = {&p};
      CV_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(cfg.threads), args, cfg.smem, stream));
      if (launches) (*launches)++;
    }
    a = b;
  }
  return CV_OK;
}

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

unsigned grid_for(uint64_t n, int threads, int sms) {
  uint64_t g = (n + threads - 1) / threads;
  uint64_t cap = (uint64_t)sms * 16;
  if (g > cap) g = cap;
  return (unsigned)(g ? g : 1);
}

}  // namespace cvk
