// Host runtime of libcv.so: the C ABI of include/cv.h, apart from the master tables (master.cu),
// batches (batch.cu), the server (server.cu) and the allocation-free scan (noalloc.cu).
//
// cv_scan  images -> segments (tensor maps over device memory, or host chunks copied into a
//          double-buffered device ring on a side stream) -> scan launches -> tile offsets ->
//          exact-size output -> expand -> per-image sorted matches; over a fragment table,
//          count -> offsets -> emit (fragments.cu).
//
// Temporaries come from a library-owned stream-ordered memory pool; results from the pool or
// from host memory. Every CUDA error is returned as a CV_E* code.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "cv.h"
#include "cv_internal.h"
#include "cv_launch.h"
#include "handles.h"
#include "runtime.h"

using namespace cvk;

void cvk_batch_free(void* h);
void cvk_server_free(void* h);

// ======================================================================= C ABI
extern "C" {

const char* cv_strerror(int code) {
  switch (code) {
    case CV_OK: return "ok";
    case CV_EINVAL: return "invalid argument";
    case CV_ENOMEM: return "out of memory";
    case CV_ECUDA: return "CUDA error";
    case CV_ETABLEFULL: return "signature table full";
    case CV_ECORRUPT: return "device consistency check failed";
    case CV_ETIMEOUT: return "device wait timed out";
    case CV_ENODEV: return "no usable CUDA device";
    case CV_ERANGE: return "index or size out of range";
    case CV_EAGAIN: return "not ready yet";
    case CV_EIO: return "file input/output failed";
    default: return "unknown error";
  }
}

int cv_last_cuda_error(void) { return last_cuda(); }

int cv_selftest_wait_timeout(uint32_t timeout_us, void* stream_) {
  if (timeout_us == 0 || timeout_us > 10000000u) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  cudaStream_t stream = (cudaStream_t)stream_;
  Temps tmp(ctx, stream);
  uint32_t* status;  // one word per wait
  uint64_t* words;
  CV_TRY(tmp.alloc(&status, 8));
  CV_TRY(tmp.alloc(&words, lookback_selftest_words() * 8));
  CV_CUDA(cudaMemsetAsync(status, 0, 8, stream));
  CV_CUDA((cudaError_t)launch_wait_selftest(status, (uint64_t)timeout_us * 1000u, stream));
  CV_CUDA((cudaError_t)launch_lookback_selftest(words, status + 1, (uint64_t)timeout_us * 1000u, stream));
  uint32_t st[2] = {0, 0};
  CV_CUDA(cudaMemcpyAsync(st, status, 8, cudaMemcpyDeviceToHost, stream));
  CV_CUDA(cudaStreamSynchronize(stream));
  if ((st[0] | st[1]) & ~kStTimeout) return CV_ECORRUPT;
  return (st[0] & st[1] & kStTimeout) ? CV_ETIMEOUT : CV_ECORRUPT;  // both waits must run out
}

int cv_kernel_config_count(void) {
  int n;
  scan_configs(&n);
  return n;
}

const char* cv_kernel_config_name(int k) {
  int n;
  const ScanCfg* c = scan_configs(&n);
  return (k >= 0 && k < n) ? c[k].name : nullptr;
}

}  // extern "C"

int cvk::digest_job(DevCtx* ctx, int cfg_i, int sig, Job& job, uint4* digests, uint8_t* trivial, uint32_t* status,
                    cudaStream_t stream, Temps& tmp) {
  Segment* segs_d;
  CV_TRY(tmp.alloc(&segs_d, job.segs.size() * sizeof(Segment)));
  CV_CUDA(cudaMemcpyAsync(segs_d, job.segs.data(), job.segs.size() * sizeof(Segment), cudaMemcpyHostToDevice, stream));
  ScanParams p;
  memset(&p, 0, sizeof p);
  p.status = status;
  p.digests = digests;
  p.trivial = trivial;
  p.tab.sig = (uint32_t)sig;
  CV_TRY(launch_range(ctx, cfg_i, true, job, segs_d, 0, job.segs.size(), p, stream));
  return CV_OK;
}

extern "C" {

int cv_sector_signatures(const void* in, uint64_t n_sectors, uint32_t signature, void* out, uint8_t* trivial,
                         void* stream_) {
  if (signature > CV_SIG_CRC64) return CV_EINVAL;
  if (n_sectors == 0) return CV_OK;
  if (!in || !out) return CV_EINVAL;
  if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u)) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  cudaStream_t stream = (cudaStream_t)stream_;
  int cfg_i;
  const ScanCfg& cfg = digest_config_for(ctx->cfg_index, (int)signature, &cfg_i);
  if (!cfg.digest_fn[signature]) return CV_EINVAL;
  Temps tmp(ctx, stream);
  Job job;
  CV_TRY(job.add(ctx, cfg, in, n_sectors, 0, 0, false));
  uint32_t* status;
  CV_TRY(tmp.alloc(&status, 4));
  CV_CUDA(cudaMemsetAsync(status, 0, 4, stream));
  return digest_job(ctx, cfg_i, (int)signature, job, (uint4*)out, trivial, status, stream, tmp);
}

int cv_sector_digests(const void* in, uint64_t n_sectors, void* digests, uint8_t* trivial, void* stream) {
  return cv_sector_signatures(in, n_sectors, CV_SIG_MD5, digests, trivial, stream);
}

int cv_window_signatures(const void* image, uint64_t n_bytes, uint32_t signature, void* out, void* stream) {
  if (signature != CV_SIG_MD5 && signature != CV_SIG_MD5_NOPAD && signature != CV_SIG_DJB2_64) return CV_EINVAL;
  if (n_bytes < 64) return CV_OK;
  if (!image || !out) return CV_EINVAL;
  if (((uintptr_t)image & 15u) || ((uintptr_t)out & 15u)) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  CV_CUDA((cudaError_t)frag_window_sigs((int)signature, (const uint8_t*)image, n_bytes, (uint4*)out, ctx->sms,
                                        stream));
  return CV_OK;
}

}  // extern "C"

namespace cvk {
// A one-image result holding a copy of n host triples (used by the serving loop).
cv_result* make_host_result(int dev, const MatchOut* data, uint64_t n, uint64_t sectors, float total_ms) {
  cv_result* r = new (std::nothrow) cv_result();
  if (!r) return nullptr;
  r->magic = kMagicResult;
  r->dev = dev;
  r->on_device = false;
  r->n_images = 1;
  r->off.assign(2, 0);
  r->off[1] = n;
  r->host = nullptr;
  r->dev_out = nullptr;
  r->free_stream = nullptr;
  memset(&r->st, 0, sizeof r->st);
  r->st.sectors = sectors;
  r->st.matches = n;
  r->st.total_ms = total_ms;
  r->st.kernel_config = -1;
  r->launches = 0;
  if (n) {
    r->host = (MatchOut*)malloc(n * sizeof(MatchOut));
    if (!r->host) {
      delete r;
      return nullptr;
    }
    memcpy(r->host, data, n * sizeof(MatchOut));
  }
  return r;
}

}  // namespace cvk

namespace {

// cv_scan over a fragment table (Section 5): count kernel per image, one offset scan over all
// tiles, emit kernel per image over its tiles with triples. Host images are copied whole.
int frag_scan(DevCtx* ctx, const cv_master* m, const cv_buf* images, uint32_t n_images, uint32_t flags,
              cudaStream_t stream, cv_result** out) {
  NvtxRange nvtx_range("cv.scan.fragments");
  Temps staging(ctx, stream);
  std::vector<const uint8_t*> dptr(n_images, nullptr);
  std::vector<uint64_t> nbytes(n_images, 0), tile_base(n_images + 1, 0);
  uint64_t windows = 0, max_tiles = 0;
  for (uint32_t i = 0; i < n_images; i++) {
    nbytes[i] = images[i].n_bytes;
    const uint64_t t = frag_tiles((int)m->tab.sig, nbytes[i]);
    tile_base[i + 1] = tile_base[i] + t;
    max_tiles = std::max(max_tiles, t);
    windows += frag_windows(nbytes[i]);
    if (!t) continue;
    if (!images[i].data) return CV_EINVAL;
    BufKind kind;
    CV_TRY(classify(ctx, images[i].data, &kind));
    if (kind == kHost) {
      uint8_t* copy;
      CV_TRY(staging.alloc(&copy, nbytes[i]));
      CV_CUDA(cudaMemcpyAsync(copy, images[i].data, nbytes[i], cudaMemcpyHostToDevice, stream));
      dptr[i] = copy;
    } else {
      if ((uintptr_t)images[i].data & 15u) return CV_EINVAL;
      dptr[i] = (const uint8_t*)images[i].data;
    }
  }
  const uint64_t T = tile_base[n_images];
  if (T >= (1ull << 32)) return CV_EINVAL;

  cv_result* r = new (std::nothrow) cv_result();
  if (!r) return CV_ENOMEM;
  r->magic = kMagicResult;
  r->dev = ctx->dev;
  r->on_device = (flags & CV_KEEP_ON_DEVICE) != 0;
  r->n_images = n_images;
  r->off.assign(n_images + 1, 0);
  r->host = nullptr;
  r->dev_out = nullptr;
  r->free_stream = stream;
  memset(&r->st, 0, sizeof r->st);
  r->launches = 0;
  r->st.sectors = windows;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int rc;
  {
    Temps tmp(ctx, stream);
    auto body = [&]() -> int {
      CV_TRY(ctx->take_events(ev, 4));
      CV_CUDA(cudaEventRecord(ev[0], stream));
      uint64_t *tile_ntrip, *tile_off, *seg_off_d, *scratch;
      uint32_t* list;
      Segment* segs_d;
      CV_TRY(tmp.alloc(&tile_ntrip, std::max<uint64_t>(T, 1) * 8));
      CV_TRY(tmp.alloc(&tile_off, std::max<uint64_t>(T, 1) * 8));
      CV_TRY(tmp.alloc(&seg_off_d, (n_images + 3) * 8));  // seg_off[n], total, status, rejected
      CV_TRY(tmp.alloc(&scratch, tile_offsets_scratch_words(T) * 8 + 8));
      CV_TRY(tmp.alloc(&list, (max_tiles + 1) * 4));
      CV_TRY(tmp.alloc(&segs_d, std::max<uint32_t>(n_images, 1) * sizeof(Segment)));
      std::vector<Segment> segs(n_images);
      memset(segs.data(), 0, segs.size() * sizeof(Segment));
      for (uint32_t i = 0; i < n_images; i++) {
        segs[i].tile_base = tile_base[i];
        segs[i].image = i;
      }
      if (n_images)
        CV_CUDA(cudaMemcpyAsync(segs_d, segs.data(), n_images * sizeof(Segment), cudaMemcpyHostToDevice, stream));
      uint32_t* status = (uint32_t*)(seg_off_d + n_images + 1);
      unsigned long long* rejected = (unsigned long long*)(seg_off_d + n_images + 2);
      CV_CUDA(cudaMemsetAsync(status, 0, 16, stream));
      CV_CUDA(cudaEventRecord(ev[1], stream));
      for (uint32_t i = 0; i < n_images; i++) {
        if (tile_base[i + 1] == tile_base[i]) continue;
        CV_CUDA((cudaError_t)frag_count(m->tab, dptr[i], nbytes[i], tile_base[i], tile_ntrip, status, rejected,
                                        ctx->sms, stream));
        r->launches++;
      }
      CV_CUDA(cudaEventRecord(ev[2], stream));
      CV_CUDA((cudaError_t)launch_tile_offsets(tile_ntrip, T, tile_off, segs_d, n_images, 1, seg_off_d,
                                               seg_off_d + n_images, scratch, stream, status));
      r->launches += 2;
      std::vector<uint64_t> seg_off(n_images + 3, 0);
      CV_CUDA(cudaMemcpyAsync(seg_off.data(), seg_off_d, (n_images + 3) * 8, cudaMemcpyDeviceToHost, stream));
      CV_CUDA(cudaStreamSynchronize(stream));
      const uint32_t st = (uint32_t)seg_off[n_images + 1];
      if (st & kStTimeout) return CV_ETIMEOUT;
      if (st) return CV_ECORRUPT;
      const uint64_t total = seg_off[n_images];
      r->st.confirm_rejected = seg_off[n_images + 2];
      if (total) {
        CV_CUDA(cudaMallocFromPoolAsync((void**)&r->dev_out, total * sizeof(MatchOut), ctx->pool, stream));
        for (uint32_t i = 0; i < n_images; i++) {
          if (tile_base[i + 1] == tile_base[i]) continue;
          CV_CUDA((cudaError_t)frag_emit(m->tab, dptr[i], nbytes[i], tile_base[i], tile_ntrip, tile_off, list,
                                         r->dev_out, total, status, ctx->sms, stream, &r->launches));
        }
      }
      for (uint32_t i = 0; i < n_images; i++) r->off[i] = seg_off[i];
      r->off[n_images] = total;
      r->st.matches = total;
      if (total && !r->on_device) {
        r->host = (MatchOut*)malloc(total * sizeof(MatchOut));
        if (!r->host) return CV_ENOMEM;
        CV_CUDA(cudaMemcpyAsync(r->host, r->dev_out, total * sizeof(MatchOut), cudaMemcpyDeviceToHost, stream));
      }
      uint32_t st2 = 0;
      CV_CUDA(cudaMemcpyAsync(&st2, status, 4, cudaMemcpyDeviceToHost, stream));
      CV_CUDA(cudaEventRecord(ev[3], stream));
      CV_CUDA(cudaStreamSynchronize(stream));
      if (st2 & kStTimeout) return CV_ETIMEOUT;
      if (st2) return CV_ECORRUPT;
      float ms = 0.f;
      CV_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
      r->st.kernel_ms = ms;
      CV_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[3]));
      r->st.total_ms = ms;
      r->st.kernel_launches = (uint32_t)r->launches;
      r->st.kernel_config = -1;
      if (total && !r->on_device) {
        CV_CUDA(cudaFreeAsync(r->dev_out, stream));
        r->dev_out = nullptr;
      }
      return CV_OK;
    };
    rc = body();
  }
  if (rc != CV_OK) cudaStreamSynchronize(stream);
  ctx->give_events(ev, 4);
  if (rc != CV_OK) {
    cv_free(r);
    return rc;
  }
  *out = r;
  return CV_OK;
}

}  // namespace

extern "C" {


int cv_scan(const cv_master* m, const cv_buf* images, uint32_t n_images, const cv_scan_opts* opts, cv_result** out) {
  NvtxRange nvtx_range("cv.scan");
  if (!m || m->magic != kMagicMaster || !out || (n_images && !images)) return CV_EINVAL;
  *out = nullptr;
  if (opts && opts->struct_size < offsetof(cv_scan_opts, base_offset)) return CV_EINVAL;
  const uint64_t base_offset = (opts && opts->struct_size >= sizeof(cv_scan_opts)) ? opts->base_offset : 0u;
  const uint32_t flags = opts ? opts->flags : 0u;
  cudaStream_t stream = opts ? (cudaStream_t)opts->stream : nullptr;
  uint64_t chunk = (opts && opts->chunk_bytes) ? opts->chunk_bytes : (256ull << 20);
  chunk = chunk / kSector * kSector;
  if (chunk == 0) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  if (ctx->dev != m->dev) return CV_EINVAL;
  if (m->tab.unit == kUnitFragment) return frag_scan(ctx, m, images, n_images, flags, stream, out);
  int ncfg;
  scan_configs(&ncfg);
  int cfg_i = ctx->default_config(table_kind(m->tab));
  if (opts && opts->kernel_config) {
    if (opts->kernel_config > (uint32_t)ncfg) return CV_EINVAL;
    cfg_i = (int)opts->kernel_config - 1;
  }
  const int sig = (int)m->tab.sig;
  const ScanCfg& cfg = scan_config_for(cfg_i, table_kind(m->tab), &cfg_i);
  TableView tab = m->tab;  // disk sector g sits at cluster position (g - base_offset) mod 8
  tab.tau_add = (uint32_t)((8u - base_offset % 8u) % 8u);
  // With a 64-bit signature every candidate is confirmed against the disk sector's bytes after
  // the scan, so host images are copied whole to the device instead of streamed through a ring.
  Temps staging(ctx, stream);

  // ------------------------------------------------------------ plan the segments
  std::vector<BufKind> kind(n_images);
  Job job;
  std::vector<size_t> first_seg(n_images + 1, 0);
  struct HostChunk {
    size_t seg;
    const uint8_t* src;
    uint64_t bytes;
  };
  std::vector<HostChunk> hchunks;
  for (uint32_t i = 0; i < n_images; i++) {
    first_seg[i] = job.segs.size();
    const uint64_t ns = images[i].n_bytes / kSector;
    if (ns == 0) continue;
    if (!images[i].data) return CV_EINVAL;
    CV_TRY(classify(ctx, images[i].data, &kind[i]));
    if (kind[i] == kHost && sig_is_weak(sig)) {
      uint8_t* copy;
      CV_TRY(staging.alloc(&copy, ns * kSector));
      CV_CUDA(cudaMemcpyAsync(copy, images[i].data, ns * kSector, cudaMemcpyHostToDevice, stream));
      CV_TRY(job.add(ctx, cfg, copy, ns, 0, i, false));
    } else if (kind[i] == kDevice) {
      if ((uintptr_t)images[i].data & 15u) return CV_EINVAL;
      CV_TRY(job.add(ctx, cfg, images[i].data, ns, 0, i, true));
    } else {
      const uint64_t per = chunk / kSector;
      for (uint64_t s0 = 0; s0 < ns; s0 += per) {
        const uint64_t n = std::min(per, ns - s0);
        hchunks.push_back(HostChunk{job.segs.size(), (const uint8_t*)images[i].data + s0 * kSector, n * kSector});
        CV_TRY(job.add(ctx, cfg, nullptr, n, s0, i, false));
      }
    }
  }
  first_seg[n_images] = job.segs.size();

  cv_result* r = new (std::nothrow) cv_result();
  if (!r) return CV_ENOMEM;
  r->magic = kMagicResult;
  r->dev = ctx->dev;
  r->on_device = (flags & CV_KEEP_ON_DEVICE) != 0;
  r->n_images = n_images;
  r->off.assign(n_images + 1, 0);
  r->host = nullptr;
  r->dev_out = nullptr;
  r->free_stream = stream;
  memset(&r->st, 0, sizeof r->st);
  r->launches = 0;
  r->st.sectors = job.n_sectors;

  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ring_copied[2] = {nullptr, nullptr}, ring_free[2] = {nullptr, nullptr};
  int rc;
  {
    Temps tmp(ctx, stream);
    auto body = [&]() -> int {
      CV_TRY(ctx->take_events(ev, 4));
      CV_CUDA(cudaEventRecord(ev[0], stream));
      const size_t nseg = job.segs.size();
      const uint64_t nt = job.n_tiles;
      uint64_t total = 0;
      std::vector<uint64_t> seg_off(nseg + 4, 0);
      uint32_t* status_keep = nullptr;
      bool expanded_early = false;  // the expand pass ran before the count came back, and sufficed
      if (nseg) {
        void* ring[2] = {nullptr, nullptr};
        if (!hchunks.empty()) {
          const uint64_t ring_bytes = std::min<uint64_t>(chunk, [&] {
            uint64_t mx = 0;
            for (auto& h : hchunks) mx = std::max(mx, h.bytes);
            return mx;
          }());
          for (int b = 0; b < 2; b++) {
            CV_TRY(tmp.alloc(&ring[b], ring_bytes));
            CV_CUDA(cudaEventCreateWithFlags(&ring_copied[b], cudaEventDisableTiming));
            CV_CUDA(cudaEventCreateWithFlags(&ring_free[b], cudaEventDisableTiming));
          }
          for (size_t k = 0; k < hchunks.size(); k++) {
            const size_t s = hchunks[k].seg;
            CV_TRY(job.set_map(ctx, cfg, s, ring[k & 1]));
          }
        }
        Segment* segs_d;
        uint4* hit_rec;
        uint32_t *tile_nhit, *status;
        uint64_t *tile_ntrip, *tile_off, *seg_off_d, *off_scratch;
        // compaction works on output tiles of 32 sectors, T / 32 per scan tile
        const uint64_t n_out = nt * (uint64_t)(cfg.T / 32);
        Carve carve;
        carve.add(&segs_d, nseg * sizeof(Segment));
        carve.add(&hit_rec, n_out * 32 * sizeof(uint4));
        carve.add(&tile_nhit, n_out * 4);
        carve.add(&tile_ntrip, n_out * 8);
        carve.add(&tile_off, n_out * 8);
        // seg_off[nseg], total, status, hit sectors, rejected candidates
        carve.add(&seg_off_d, (nseg + 4) * 8);
        carve.add(&off_scratch, tile_offsets_scratch_words(n_out) * 8);
        CV_TRY(carve.commit(tmp));
        status = (uint32_t*)(seg_off_d + nseg + 1);
        status_keep = status;
        CV_CUDA(cudaMemsetAsync(status, 0, 24, stream));
        CV_CUDA(cudaMemcpyAsync(segs_d, job.segs.data(), nseg * sizeof(Segment), cudaMemcpyHostToDevice, stream));
        ScanParams p;
        memset(&p, 0, sizeof p);
        p.tab = tab;
        p.hit_rec = hit_rec;
        p.tile_nhit = tile_nhit;
        p.tile_ntrip = tile_ntrip;
        p.status = status;
        p.rejected = (unsigned long long*)(seg_off_d + nseg + 3);
        CV_CUDA(cudaEventRecord(ev[1], stream));
        NvtxRange launches_range("cv.scan.launches");
        // device segments: one launch per run of consecutive device segments
        size_t hk = 0;
        size_t s = 0;
        while (s < nseg) {
          if (hk < hchunks.size() && hchunks[hk].seg == s) {
            const int b = (int)(hk & 1);
            if (hk >= 2) CV_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ring_free[b], 0));
            else CV_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ev[1], 0));
            CV_CUDA(cudaMemcpyAsync(ring[b], hchunks[hk].src, hchunks[hk].bytes, cudaMemcpyHostToDevice,
                                    ctx->copy_stream));
            CV_CUDA(cudaEventRecord(ring_copied[b], ctx->copy_stream));
            CV_CUDA(cudaStreamWaitEvent(stream, ring_copied[b], 0));
            CV_TRY(launch_range(ctx, cfg_i, false, job, segs_d, s, s + 1, p, stream, &r->launches));
            CV_CUDA(cudaEventRecord(ring_free[b], stream));
            hk++;
            s++;
          } else {
            size_t e = s;
            while (e < nseg && !(hk < hchunks.size() && hchunks[hk].seg == e)) e++;
            CV_TRY(launch_range(ctx, cfg_i, false, job, segs_d, s, e, p, stream, &r->launches));
            s = e;
          }
        }
        CV_CUDA(cudaEventRecord(ev[2], stream));
        launches_range.end();
        NvtxRange offsets_range("cv.scan.offsets_expand");
        uint64_t* total_d = seg_off_d + nseg;
        uint32_t nseg32 = (uint32_t)nseg;
        uint64_t nt_arg = n_out;
        // the offsets, and the sectors with a match summed in the same pass
        CV_CUDA((cudaError_t)launch_tile_offsets(tile_ntrip, n_out, tile_off, segs_d, nseg32, (uint32_t)(cfg.T / 32),
                                                 seg_off_d, total_d, off_scratch, stream, status, tile_nhit,
                                                 seg_off_d + nseg + 2));
        // The expand pass needs an output buffer before the exact count is known on the host.
        // After a scan against the same table it is launched at once, with room for a quarter more
        // than that scan's matches (one wait for the whole call); the exact count then tells
        // whether the room sufficed (the pass writes nothing beyond it and flags the overflow),
        // and only if not is it run again into an exact buffer.
        const uint64_t hint = __atomic_load_n(&const_cast<cv_master*>(m)->last_matches, __ATOMIC_RELAXED);
        uint64_t room = 0;
        if (hint) {
          room = hint + hint / 4 + 1024;
          CV_CUDA(cudaMallocFromPoolAsync((void**)&r->dev_out, room * sizeof(MatchOut), ctx->pool, stream));
          CV_CUDA((cudaError_t)launch_expand(cfg, hit_rec, tile_nhit, tile_off, n_out, segs_d, nseg32, tab,
                                             r->dev_out, room, status, ctx->sms, stream));
          r->launches += 1;
        }
        CV_CUDA(cudaMemcpyAsync(seg_off.data(), seg_off_d, (nseg + 4) * 8, cudaMemcpyDeviceToHost, stream));
        // the call's end unless more work follows (then recorded again after it): in the common
        // case this one wait for the stream is the call's only one
        CV_CUDA(cudaEventRecord(ev[3], stream));
        CV_CUDA(cudaStreamSynchronize(stream));
        const uint32_t st = (uint32_t)seg_off[nseg + 1];
        if (st & kStTimeout) return CV_ETIMEOUT;
        if (st & ~kStOverflow) return CV_ECORRUPT;
        total = seg_off[nseg];
        r->st.hit_sectors = seg_off[nseg + 2];
        r->st.confirm_rejected = seg_off[nseg + 3];
        __atomic_store_n(&const_cast<cv_master*>(m)->last_matches, total, __ATOMIC_RELAXED);
        if (total > room) {
          if (r->dev_out) {
            CV_CUDA(cudaFreeAsync(r->dev_out, stream));
            r->dev_out = nullptr;
          }
          CV_CUDA(cudaMemsetAsync(status, 0, 4, stream));
          CV_CUDA(cudaMallocFromPoolAsync((void**)&r->dev_out, total * sizeof(MatchOut), ctx->pool, stream));
          CV_CUDA((cudaError_t)launch_expand(cfg, hit_rec, tile_nhit, tile_off, n_out, segs_d, nseg32, tab,
                                             r->dev_out, total, status, ctx->sms, stream));
          r->launches += 1;
        } else if (r->dev_out && !total) {
          CV_CUDA(cudaFreeAsync(r->dev_out, stream));
          r->dev_out = nullptr;
        } else {
          expanded_early = true;
        }
        r->launches += 2;  // the offset pass
      }
      // per-image ranges; an image without sectors gets an empty range
      r->off[n_images] = total;
      for (int64_t i = (int64_t)n_images - 1; i >= 0; i--)
        r->off[i] = (first_seg[i] < first_seg[i + 1]) ? seg_off[first_seg[i]] : r->off[i + 1];
      r->st.matches = total;
      bool more = !nseg || (total && !expanded_early);  // device work after the first wait
      if (total && !r->on_device) {
        r->host = (MatchOut*)malloc(total * sizeof(MatchOut));
        if (!r->host) return CV_ENOMEM;
        CV_CUDA(cudaMemcpyAsync(r->host, r->dev_out, total * sizeof(MatchOut), cudaMemcpyDeviceToHost, stream));
        more = true;
      }
      uint32_t st2 = 0;
      if (nseg && total && !expanded_early)
        CV_CUDA(cudaMemcpyAsync(&st2, status_keep, 4, cudaMemcpyDeviceToHost, stream));
      if (more) {
        CV_CUDA(cudaEventRecord(ev[3], stream));
        CV_CUDA(cudaStreamSynchronize(stream));
      }
      if (st2) return CV_ECORRUPT;
      float ms = 0.f;
      if (nseg) {
        CV_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
        r->st.kernel_ms = ms;
      }
      CV_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[3]));
      r->st.total_ms = ms;
      r->st.kernel_launches = (uint32_t)r->launches;
      r->st.kernel_config = cfg_i;
      if (total && !r->on_device) {
        CV_CUDA(cudaFreeAsync(r->dev_out, stream));
        r->dev_out = nullptr;
      }
      return CV_OK;
    };
    rc = body();
  }
  if (rc != CV_OK) {
    cudaStreamSynchronize(stream);
    cudaStreamSynchronize(ctx->copy_stream);
  }
  ctx->give_events(ev, 4);
  for (int b = 0; b < 2; b++) {
    if (ring_copied[b]) cudaEventDestroy(ring_copied[b]);
    if (ring_free[b]) cudaEventDestroy(ring_free[b]);
  }
  if (rc != CV_OK) {
    cv_free(r);
    return rc;
  }
  *out = r;
  return CV_OK;
}

int cv_matches(const cv_result* r, uint32_t image_index, const cv_match** out, uint64_t* n_out) {
  if (!r || r->magic != kMagicResult || !out || !n_out) return CV_EINVAL;
  if (image_index >= r->n_images) return CV_ERANGE;
  const uint64_t a = r->off[image_index], b = r->off[image_index + 1];
  *n_out = b - a;
  const MatchOut* base = r->on_device ? r->dev_out : r->host;
  *out = (b > a && base) ? (const cv_match*)(base + a) : nullptr;
  return CV_OK;
}

int cv_scan_get_stats(const cv_result* r, cv_scan_stats* st) {
  if (!r || r->magic != kMagicResult || !st) return CV_EINVAL;
  *st = r->st;
  return CV_OK;
}

void cv_free(void* handle) {
  if (!handle) return;
  const uint32_t magic = *(const uint32_t*)handle;
  if (magic == 0xC7A57E03u) {
    cvk_batch_free(handle);
    return;
  }
  if (magic == 0xC7A57E04u) {
    cvk_server_free(handle);
    return;
  }
  if (magic == kMagicMaster) {
    cv_master* m = (cv_master*)handle;
    m->magic = 0;
    if (m->slots) cudaFree(m->slots);
    if (m->postings) cudaFree(m->postings);
    if (m->bloom) cudaFree(m->bloom);
    if (m->confirm) cudaFree(m->confirm);
    if (m->keys0) cudaFree(m->keys0);
    if (m->frag_l1) cudaFree(m->frag_l1);
    free(m);
  } else if (magic == kMagicResult) {
    cv_result* r = (cv_result*)handle;
    r->magic = 0;
    // Results are complete when cv_scan returns, so the buffer goes back to the pool in stream
    // order, without waiting.
    if (r->dev_out) cudaFreeAsync(r->dev_out, r->free_stream);
    free(r->host);
    delete r;
  }
}

}  // extern "C"
