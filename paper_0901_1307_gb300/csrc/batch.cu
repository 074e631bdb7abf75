// Batched scans: many device-resident images against one master table, replayed as one CUDA
// graph. The paper scans several drives at once by multiplexing them onto one GPU (Section 3);
// here all images of a batch are one work list: images that sit in one device allocation share
// a tensor map, the persistent scan kernel takes tiles of every image in one launch, and one
// offset pass and one expand pass produce every image's sorted matches. The whole sequence is
// captured once and replayed with a single graph launch per run.
//
// An optional autotuner times, on the batch itself, every kernel configuration (tile rows,
// sectors per thread, staging width, ring stages, pipe split of the MD5 additions) x table layout
// (the master's; for a hash-layout master also a sorted copy, Section 4's binary search) x Bloom
// prefilter (off; on with the master's filter, or with one the batch builds when the master has
// none), and keeps the fastest; results are cached in-process and, when a cache file is named,
// on disk (one line per key). Section 3.2 notes that the best concurrency has to be found again
// on every GPU generation.
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cv.h"
#include "runtime.h"

using namespace cvk;

namespace {
constexpr uint32_t kMagicBatch = 0xC7A57E03u;

struct Buffers {
  Segment* segs_d = nullptr;
  uint4* hit_rec = nullptr;
  uint32_t* tile_nhit = nullptr;
  uint64_t* tile_ntrip = nullptr;
  uint64_t* tile_off = nullptr;
  uint64_t* off_scratch = nullptr;
  uint64_t* counters_d = nullptr;  // seg_off[nseg], total, status
  MatchOut* out_d = nullptr;
  std::vector<void*> owned;

  int alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_fail(e);
    owned.push_back(*p);
    return CV_OK;
  }
  void release() {
    for (void* p : owned) cudaFree(p);
    owned.clear();
  }
};

// Buffers of a job with one scan configuration and `capacity` output triples.
int make_buffers(const Job& job, const ScanCfg& cfg, uint64_t capacity, Buffers* b) {
  const size_t nseg = job.segs.size();
  const uint64_t n_out = job.n_tiles * (uint64_t)(cfg.T / 32);
  CV_TRY(b->alloc((void**)&b->segs_d, nseg * sizeof(Segment)));
  CV_TRY(b->alloc((void**)&b->hit_rec, n_out * 32 * sizeof(uint4)));
  CV_TRY(b->alloc((void**)&b->tile_nhit, n_out * 4));
  CV_TRY(b->alloc((void**)&b->tile_ntrip, n_out * 8));
  CV_TRY(b->alloc((void**)&b->tile_off, n_out * 8));
  CV_TRY(b->alloc((void**)&b->off_scratch, tile_offsets_scratch_words(n_out) * 8));
  CV_TRY(b->alloc((void**)&b->counters_d, (nseg + 2) * 8));
  CV_TRY(b->alloc((void**)&b->out_d, std::max<uint64_t>(capacity, 1) * sizeof(MatchOut)));
  CV_CUDA(cudaMemcpy(b->segs_d, job.segs.data(), nseg * sizeof(Segment), cudaMemcpyHostToDevice));
  return CV_OK;
}

// Queue one complete run (status reset, scan, offsets, expand, counters to host) on stream.
int enqueue_run(DevCtx* ctx, int cfg_i, const TableView& tab, const Job& job, const Buffers& b, uint64_t capacity,
                uint64_t* counters_h, cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1, int* launches) {
  int ncfg;
  const ScanCfg& cfg = scan_configs(&ncfg)[cfg_i];
  const size_t nseg = job.segs.size();
  const uint64_t n_out = job.n_tiles * (uint64_t)(cfg.T / 32);
  uint32_t* status = (uint32_t*)(b.counters_d + nseg + 1);
  CV_CUDA(cudaMemsetAsync(status, 0, 8, stream));
  ScanParams p;
  memset(&p, 0, sizeof p);
  p.tab = tab;
  p.hit_rec = b.hit_rec;
  p.tile_nhit = b.tile_nhit;
  p.tile_ntrip = b.tile_ntrip;
  p.status = status;
  // Under stream capture a plain record only orders the capture; the external flag makes it an
  // event-record node that every replay of the graph executes, so the timing events see each run.
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  CV_CUDA(cudaStreamIsCapturing(stream, &cap_st));
  const unsigned rec_flags = cap_st == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  if (ev0) CV_CUDA(cudaEventRecordWithFlags(ev0, stream, rec_flags));
  CV_TRY(launch_range(ctx, cfg_i, false, job, b.segs_d, 0, nseg, p, stream, launches));
  if (ev1) CV_CUDA(cudaEventRecordWithFlags(ev1, stream, rec_flags));
  uint64_t* total_d = b.counters_d + nseg;
  CV_CUDA((cudaError_t)launch_tile_offsets(b.tile_ntrip, n_out, b.tile_off, b.segs_d, (uint32_t)nseg,
                                           (uint32_t)(cfg.T / 32), b.counters_d, total_d, b.off_scratch, stream,
                                           status));
  if (launches) *launches += 2;
  CV_CUDA((cudaError_t)launch_expand(cfg, b.hit_rec, b.tile_nhit, b.tile_off, n_out, b.segs_d, (uint32_t)nseg, tab,
                                     b.out_d, capacity, status, ctx->sms, stream));
  if (launches) *launches += 1;
  if (counters_h) CV_CUDA(cudaMemcpyAsync(counters_h, b.counters_d, (nseg + 2) * 8, cudaMemcpyDeviceToHost, stream));
  return CV_OK;
}

// ------------------------------------------------------------------------- tune cache
std::mutex g_tune_mutex;
struct TuneChoice {
  int cfg, bloom, layout;
};
std::map<std::string, TuneChoice> g_tune;  // key -> choice

// table_kind: signature, layout and position keying of the table; unique and occupancy (in
// tenths of the slots): they change the probe's cost and so the choice.
std::string tune_key(const char* gpu, int sms, uint64_t sectors, uint32_t images, uint64_t unique, uint32_t occupancy,
                     bool bloom_avail, uint32_t table_kind) {
  auto lg = [](uint64_t x) {
    int b = 0;
    while (x > 1) {
      x >>= 1;
      b++;
    }
    return b;
  };
  // the device name goes in with its blanks replaced: a cache line is blank-separated
  std::string name(gpu);
  for (char& ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%d|s%d|i%d|u%d|o%u|b%d|t%u", name.c_str(), sms, lg(sectors), lg(images), lg(unique),
           occupancy, bloom_avail ? 1 : 0, table_kind);
  return buf;
}

// Cache lines are "key config_name bloom layout"; lines written before the layout was tuned
// ("key config_name bloom") mean the master's own layout (-1).
bool tune_lookup(const std::string& key, const char* path, TuneChoice* c) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) {
    *c = it->second;
    return true;
  }
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[300], name[64];
    int bl, lay = -1;
    const int got = sscanf(line, "%299[^ ] %63s %d %d", k, name, &bl, &lay);
    if (got >= 3 && key == k) {
      int n;
      const ScanCfg* cf = scan_configs(&n);
      for (int i = 0; i < n; i++)
        if (strcmp(cf[i].name, name) == 0) {
          *c = TuneChoice{i, bl, got == 4 ? lay : -1};
          found = true;
        }
    }
  }
  fclose(f);
  if (found) g_tune[key] = *c;
  return found;
}

void tune_store(const std::string& key, const char* path, const TuneChoice& c) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune[key] = c;
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  int n;
  fprintf(f, "%s %s %d %d\n", key.c_str(), scan_configs(&n)[c.cfg].name, c.bloom, c.layout);
  fclose(f);
}

}  // namespace

struct cv_batch {
  uint32_t magic;
  int dev;
  int cfg_i;
  int bloom;
  int layout;  // kLayout* scanned
  TableView tab;
  void* own_slots = nullptr;  // the batch's sorted copy of a hash table (records, key words)
  void* own_keys0 = nullptr;
  void* own_bloom = nullptr;  // the batch's Bloom filter for a master without one
  Job job;
  uint32_t n_images;
  std::vector<size_t> first_seg;  // n_images + 1
  Buffers buf;
  uint64_t capacity;
  uint64_t* counters_h;  // pinned
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaEvent_t ev0, ev1, done;
  int launches;
  bool ran;
  bool tuned;
};

extern "C" {

int cv_batch_create(const cv_master* m, const cv_buf* images, uint32_t n_images, const cv_batch_opts* opts,
                    cv_batch** out) {
  if (!m || !out || (n_images && !images)) return CV_EINVAL;
  *out = nullptr;
  if (opts && opts->struct_size < offsetof(cv_batch_opts, sorted_copy)) return CV_EINVAL;
  const bool want_sorted = opts && opts->struct_size >= sizeof(cv_batch_opts) && opts->sorted_copy;
  TableView tab;
  int mdev;
  if (master_view(m, &tab, &mdev) != CV_OK || tab.unit != kUnitSector) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  if (ctx->dev != mdev) return CV_EINVAL;
  cudaStream_t stream = opts ? (cudaStream_t)opts->stream : nullptr;
  int ncfg;
  const ScanCfg* cfgs = scan_configs(&ncfg);
  for (uint32_t i = 0; i < n_images; i++) {
    if (images[i].n_bytes < kSector) continue;
    if (!images[i].data || ((uintptr_t)images[i].data & 15u)) return CV_EINVAL;
    BufKind k;
    CV_TRY(classify(ctx, images[i].data, &k));
    if (k != kDevice) return CV_EINVAL;
  }
  const bool bloom_avail = tab.use_bloom != 0;
  int cfg_i = ctx->default_config(table_kind(tab));
  int bloom = bloom_avail ? 1 : 0;
  if (opts && opts->kernel_config) {
    if (opts->kernel_config > (uint32_t)ncfg) return CV_EINVAL;
    cfg_i = (int)opts->kernel_config - 1;
  }
  scan_config_for(cfg_i, table_kind(tab), &cfg_i);
  if (opts && opts->bloom > CV_BATCH_BLOOM_ON) return CV_EINVAL;
  if (opts && opts->bloom == CV_BATCH_BLOOM_OFF) bloom = 0;
  if (opts && opts->bloom == CV_BATCH_BLOOM_ON) bloom = 1;

  cv_batch* b = new (std::nothrow) cv_batch();
  if (!b) return CV_ENOMEM;
  b->magic = kMagicBatch;
  b->dev = ctx->dev;
  b->n_images = n_images;
  b->counters_h = nullptr;
  b->graph = nullptr;
  b->exec = nullptr;
  b->ev0 = b->ev1 = b->done = nullptr;
  b->launches = 0;
  b->ran = false;
  b->tuned = false;

  auto build_job = [&](int k, Job* job, std::vector<size_t>* first) -> int {
    first->assign(n_images + 1, 0);
    for (uint32_t i = 0; i < n_images; i++) {
      (*first)[i] = job->segs.size();
      const uint64_t ns = images[i].n_bytes / kSector;
      if (ns) CV_TRY(job->add(ctx, cfgs[k], images[i].data, ns, 0, i, true));
    }
    (*first)[n_images] = job->segs.size();
    return CV_OK;
  };

  auto body = [&]() -> int {
    CV_CUDA(cudaEventCreate(&b->ev0));
    CV_CUDA(cudaEventCreate(&b->ev1));
    CV_CUDA(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
    uint64_t total_sectors = 0;
    for (uint32_t i = 0; i < n_images; i++) total_sectors += images[i].n_bytes / kSector;
    // ---------------------------------------------------------- table variants
    // Variant v of the table: layout (0: the master's own, 1: a sorted copy of a hash master)
    // and Bloom use (the master's filter, or the batch's own when the master has none).
    TableView sorted_tab = tab, bloom_tab = tab;
    bool have_sorted = false, have_bloom = bloom_avail;
    auto need_sorted = [&]() -> int {
      if (have_sorted || tab.layout != kLayoutHash) return CV_OK;
      CV_TRY(table_sorted_copy(tab, stream, &sorted_tab, &b->own_slots, &b->own_keys0));
      have_sorted = true;
      return CV_OK;
    };
    auto need_bloom = [&]() -> int {
      if (have_bloom) return CV_OK;
      CV_TRY(table_bloom(tab, 16, stream, &bloom_tab, &b->own_bloom));
      have_bloom = true;
      return CV_OK;
    };
    auto variant = [&](int sorted, int bl) {
      TableView t = sorted ? sorted_tab : tab;
      if (bl && !bloom_avail) {  // the batch's own filter over the same keys
        t.bloom = bloom_tab.bloom;
        t.bloom_mask = bloom_tab.bloom_mask;
      }
      t.use_bloom = (uint32_t)bl;
      return t;
    };
    // index into the variants: 0 the master's layout, 1 the sorted copy
    int layout_choice = (want_sorted && tab.layout == kLayoutHash) ? 1 : 0;
    // ---------------------------------------------------------------- autotune
    if (opts && opts->autotune && total_sectors) {
      cudaDeviceProp prop;
      CV_CUDA(cudaGetDeviceProperties(&prop, ctx->dev));
      const uint64_t n_slots = tab.layout == kLayoutSorted ? tab.n_keys : (uint64_t)tab.slot_mask + 1;
      const uint32_t tenths = (uint32_t)(10ull * tab.n_keys / std::max<uint64_t>(n_slots, 1));
      const uint32_t tkey = (uint32_t)table_kind(tab) * 2u + (tab.tau_mask ? 1u : 0u);
      const std::string key =
          tune_key(prop.name, ctx->sms, total_sectors, n_images, tab.n_keys, tenths, bloom_avail, tkey);
      TuneChoice tc;
      if (tune_lookup(key, opts->tune_cache, &tc)) {
        cfg_i = tc.cfg;
        bloom = tc.bloom;
        layout_choice = (tc.layout == (int)kLayoutSorted && tab.layout == kLayoutHash) ? 1 : 0;
      } else {
        CV_TRY(need_sorted());
        CV_TRY(need_bloom());
        const int n_layouts = have_sorted ? 2 : 1;
        float best = 1e30f;
        for (int k = 0; k < ncfg; k++) {
          Job job;
          std::vector<size_t> first;
          CV_TRY(build_job(k, &job, &first));
          Buffers tb_;
          int rc = make_buffers(job, cfgs[k], 0, &tb_);
          if (rc != CV_OK) {
            tb_.release();
            return rc;
          }
          for (int lay = 0; lay < n_layouts && rc == CV_OK; lay++) {
            for (int bl = 0; bl <= 1 && rc == CV_OK; bl++) {
              const TableView t = variant(lay, bl);
              if (!cfgs[k].scan_fn[table_kind(t)]) continue;  // not built for this table kind
              float ms_min = 1e30f;
              for (int rep = 0; rep < 3; rep++) {
                rc = enqueue_run(ctx, k, t, job, tb_, 0, nullptr, stream, b->ev0, b->ev1, nullptr);
                if (rc != CV_OK) break;
                if (cudaEventSynchronize(b->ev1) != cudaSuccess) {
                  rc = CV_ECUDA;
                  break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, b->ev0, b->ev1);
                if (rep) ms_min = std::min(ms_min, ms);  // the first run warms up
              }
              if (rc == CV_OK && ms_min < best) {
                best = ms_min;
                cfg_i = k;
                bloom = bl;
                layout_choice = lay;
              }
            }
          }
          cudaStreamSynchronize(stream);
          tb_.release();
          if (rc != CV_OK) return rc;
        }
        tune_store(key, opts->tune_cache,
                   TuneChoice{cfg_i, bloom, (int)(layout_choice ? kLayoutSorted : tab.layout)});
        b->tuned = true;
      }
    }
    // keep only what the choice uses
    if (layout_choice) CV_TRY(need_sorted());
    if (bloom && !bloom_avail) CV_TRY(need_bloom());
    if (!layout_choice && b->own_slots) {
      cudaFree(b->own_slots);
      cudaFree(b->own_keys0);
      b->own_slots = b->own_keys0 = nullptr;
    }
    if (!bloom && b->own_bloom) {
      cudaFree(b->own_bloom);
      b->own_bloom = nullptr;
    }
    const TableView chosen = variant(layout_choice, bloom);
    scan_config_for(cfg_i, table_kind(chosen), &cfg_i);
    b->cfg_i = cfg_i;
    b->bloom = bloom;
    b->tab = chosen;
    b->layout = (int)chosen.layout;
    CV_TRY(build_job(cfg_i, &b->job, &b->first_seg));
    const size_t nseg = b->job.segs.size();
    CV_CUDA(cudaMallocHost((void**)&b->counters_h, (nseg + 2) * 8));
    memset(b->counters_h, 0, (nseg + 2) * 8);
    // ------------------------------------------------------------------ capacity
    uint64_t cap = opts ? opts->match_capacity : 0;
    if (cap == 0 && nseg) {
      Buffers sb;
      int rc = make_buffers(b->job, cfgs[cfg_i], 0, &sb);
      if (rc == CV_OK) rc = enqueue_run(ctx, cfg_i, b->tab, b->job, sb, 0, b->counters_h, stream, nullptr, nullptr,
                                        nullptr);
      if (rc == CV_OK && cudaStreamSynchronize(stream) != cudaSuccess) rc = CV_ECUDA;
      sb.release();
      if (rc != CV_OK) return rc;
      const uint64_t total = b->counters_h[nseg];
      cap = total + total / 4 + 4096;
    }
    b->capacity = cap;
    if (nseg == 0) return CV_OK;
    CV_TRY(make_buffers(b->job, cfgs[cfg_i], cap, &b->buf));
    // --------------------------------------------------------------- the graph
    cudaStream_t cs;
    CV_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = CV_OK;
    if (e == cudaSuccess) {
      b->launches = 0;
      rc = enqueue_run(ctx, cfg_i, b->tab, b->job, b->buf, cap, b->counters_h, cs, b->ev0, b->ev1, &b->launches);
      e = cudaStreamEndCapture(cs, &b->graph);
    }
    cudaStreamDestroy(cs);
    if (rc != CV_OK) return rc;
    CV_CUDA(e);
    CV_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return CV_OK;
  };
  int rc = body();
  if (rc != CV_OK) {
    cudaStreamSynchronize(stream);
    cv_free(b);
    return rc;
  }
  *out = b;
  return CV_OK;
}

int cv_batch_run(cv_batch* b, void* stream) {
  NvtxRange nvtx_range("cv.batch_run");
  if (!b || b->magic != kMagicBatch) return CV_EINVAL;
  if (!b->exec) {
    b->ran = true;
    return CV_OK;  // nothing to scan
  }
  CV_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  CV_CUDA(cudaEventRecord(b->done, (cudaStream_t)stream));
  b->ran = true;
  return CV_OK;
}

int cv_batch_wait(cv_batch* b, uint64_t* n_matches) {
  if (!b || b->magic != kMagicBatch) return CV_EINVAL;
  if (!b->ran) return CV_EINVAL;
  const size_t nseg = b->job.segs.size();
  if (n_matches) *n_matches = 0;
  if (!b->exec) return CV_OK;
  CV_CUDA(cudaEventSynchronize(b->done));
  const uint64_t total = b->counters_h[nseg];
  const uint32_t st = (uint32_t)b->counters_h[nseg + 1];
  if (n_matches) *n_matches = total;
  if (st & kStTimeout) return CV_ETIMEOUT;
  if (total > b->capacity) return CV_ERANGE;
  if (st) return CV_ECORRUPT;
  return CV_OK;
}

int cv_batch_matches(const cv_batch* b, uint32_t image_index, const cv_match** out, uint64_t* n_out) {
  if (!b || b->magic != kMagicBatch || !out || !n_out) return CV_EINVAL;
  if (image_index >= b->n_images) return CV_ERANGE;
  *out = nullptr;
  *n_out = 0;
  const size_t a = b->first_seg[image_index], e = b->first_seg[image_index + 1];
  if (a == e || !b->exec) return CV_OK;
  const size_t nseg = b->job.segs.size();
  const uint64_t lo = b->counters_h[a];
  const uint64_t hi = (e < nseg) ? b->counters_h[e] : b->counters_h[nseg];
  if (hi > b->capacity) return CV_ERANGE;
  *n_out = hi - lo;
  *out = (hi > lo) ? (const cv_match*)(b->buf.out_d + lo) : nullptr;
  return CV_OK;
}

int cv_batch_get_info(const cv_batch* b, cv_batch_info* info) {
  if (!b || b->magic != kMagicBatch || !info) return CV_EINVAL;
  memset(info, 0, sizeof *info);
  int n;
  info->kernel_config = b->cfg_i;
  info->config_name = scan_configs(&n)[b->cfg_i].name;
  info->bloom = (uint32_t)b->bloom;
  info->layout = (uint32_t)b->layout;
  info->tuned = b->tuned ? 1u : 0u;
  info->kernel_launches = (uint32_t)b->launches;
  info->tensor_maps = (uint32_t)b->job.maps.size();
  info->segments = (uint32_t)b->job.segs.size();
  info->sectors = b->job.n_sectors;
  info->match_capacity = b->capacity;
  float ms = 0.f;
  if (b->ran && b->exec && cudaEventQuery(b->done) == cudaSuccess && cudaEventElapsedTime(&ms, b->ev0, b->ev1) ==
                                                                          cudaSuccess)
    info->scan_ms = ms;
  cudaGetLastError();
  return CV_OK;
}

}  // extern "C"

// Called by cv_free for batch handles.
void cvk_batch_free(void* h) {
  cv_batch* b = (cv_batch*)h;
  if (!b || b->magic != kMagicBatch) return;
  b->magic = 0;
  if (b->done) cudaEventSynchronize(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->buf.release();
  for (void* p : {b->own_slots, b->own_keys0, b->own_bloom})
    if (p) cudaFree(p);
  if (b->counters_h) cudaFreeHost(b->counters_h);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->done) cudaEventDestroy(b->done);
  delete b;
}
