// Serving loop: scans of images that arrive over time against one resident master table.
//
// The paper's system (Section 3.1, Figure 7) feeds several drives into one GPU through
// double-buffered host and device buffers, overlapping transfers with hashing; it names
// overlapping disk I/O with GPU I/O and processing as near-term work (Section 5). Here:
//   - Requests are cut into work units (default 64 MiB of whole sectors).
//   - A device arena of hbm_budget_bytes holds units in flight, one slot per unit. Units are
//     copied host-to-device on side streams as slots free up, round robin over the live
//     requests, fewest bytes left first, with at most max_copy_bytes queued on the streams at
//     once, so a small network chunk is not stuck behind the queued copies of a large drive.
//   - Every engine iteration takes, for each live request, its units that have landed on the
//     device (in order) and scans all of them in one launch (continuous batching). The whole
//     arena is one allocation, so one tensor map covers every unit.
//   - The engine never waits for the GPU. Two scan batches are in flight at once, each on its
//     own stream: a batch's scan and offset pass are launched and their counts copied back;
//     once the counts have landed (an event query) its expansion and the copy of its matches
//     are launched; once those have landed the batch is retired. Meanwhile the engine keeps
//     issuing copies and launches the next batch's scan, so one batch's expansion and readback
//     overlap the next one's scan.
//   - Batches retire in the order they were launched, and a unit's sorted matches are appended
//     to its request then; a request is complete when its last unit has been retired. Units of
//     one request are always scanned in order, so its matches stay sorted and equal a solo
//     cv_scan of the image.
// One engine thread per server; cv_submit and cv_poll may be called from any thread.
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cv.h"
#include "runtime.h"

using namespace cvk;

void cvk_server_free(void* h);

namespace {
constexpr uint32_t kMagicServer = 0xC7A57E04u;
using Clock = std::chrono::steady_clock;

struct Unit {
  uint64_t first_sector;  // within the request
  uint64_t n_sectors;
  int slot = -1;          // arena slot (host requests), -1 when not copied yet
  int copy_stream = 0;
  bool on_device = false;  // device-resident request: no copy needed
  bool copied = false;     // copy issued
  bool scanned = false;
};

struct Request {
  uint64_t ticket;
  uint64_t tag;
  const uint8_t* data;
  uint64_t n_sectors;
  bool device;
  std::vector<Unit> units;
  size_t next_copy = 0;  // first unit not yet given a copy
  size_t next_scan = 0;  // first unit not yet scanned
  std::vector<MatchOut> matches;
  Clock::time_point submitted, done_at;
  bool done = false;
  int error = CV_OK;
  cv_result* result = nullptr;
};

// One scan batch in flight: its stream, events and per-batch device and pinned buffers (grown
// on demand), and the units it scans.
struct ScanBatch {
  enum { kFree = 0, kCounting = 1, kExpanding = 2 };
  int state = kFree;
  cudaStream_t stream = nullptr;
  cudaEvent_t counts_ready = nullptr;  // offsets, total and status are on the host
  cudaEvent_t matches_ready = nullptr;  // the matches are on the host
  struct Ref {
    Request* r;
    size_t unit;
  };
  std::vector<Ref> refs;  // segment k scans refs[k]
  size_t nseg = 0;
  uint64_t n_out = 0;
  uint64_t total = 0;
  uint64_t cap_tiles = 0, cap_segs = 0, cap_out = 0;
  Segment* segs_d = nullptr;
  uint4* hit_rec = nullptr;
  uint32_t* tile_nhit = nullptr;
  uint64_t* tile_ntrip = nullptr;
  uint64_t* tile_off = nullptr;
  uint64_t* off_scratch = nullptr;
  uint64_t* counters_d = nullptr;  // seg_off[nseg], total, status
  uint64_t* counters_h = nullptr;
  Segment* segs_h = nullptr;       // pinned staging of the segment list
  MatchOut* out_d = nullptr;
  MatchOut* out_h = nullptr;
  cudaMemPool_t pool = nullptr;           // device buffers: stream-ordered on `stream`
  std::vector<void*> retired_host;        // pinned buffers outgrown, freed with the batch

  int ensure_buffers(uint64_t tiles, uint64_t segs, uint64_t out);
  void release();
};

constexpr int kBatchesInFlight = 2;
// Work units one scan launch takes at most (64 MiB units: 4 GiB of data, about a millisecond of
// scanning), so that each batch's buffers are sized once, when the server is made.
constexpr size_t kMaxUnitsPerBatch = 64;
constexpr uint64_t kInitialMatches = 1ull << 22;  // matches a batch holds before it must grow

}  // namespace

struct cv_server {
  uint32_t magic;
  int dev;
  DevCtx* ctx;
  int cfg_i;
  TableView tab;
  uint64_t unit_bytes;
  uint64_t unit_sectors;
  uint32_t max_live;
  int n_slots;
  uint8_t* arena = nullptr;
  CUtensorMap arena_map;
  std::vector<cudaStream_t> copy_streams;
  std::vector<cudaEvent_t> slot_event;  // copy of the unit in the slot finished
  std::vector<int> free_slots;
  ScanBatch batch[kBatchesInFlight];
  std::deque<int> in_flight;  // batches not yet retired, in launch order

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> live;
  std::map<uint64_t, Request*> by_ticket;
  uint64_t next_ticket = 1;
  bool stopping = false;
  int fatal = CV_OK;
  std::thread engine;

  // statistics
  cv_server_stats st;
  std::vector<double> lat_ms;
  Clock::time_point first_submit, last_done;
  bool any_submit = false;
  double live_sum = 0;
  uint64_t bytes_in_flight = 0;
  uint64_t copy_cap = 0;      // bytes queued on the copy streams at most (at least one unit)
  uint64_t copy_queued = 0;   // bytes issued and not yet seen landed

  void run();
  int iterate(bool* did_work);
  int issue_copies(const std::vector<Request*>& work);
  int launch_scan(ScanBatch& b, const std::vector<Request*>& work, bool* launched);
  int launch_expand_of(ScanBatch& b);
  void retire(ScanBatch& b);
  void finish(Request* r);
};

namespace {

// Buffers for tiles output tiles, segs segments and out matches. They are sized once when the
// server is made (kMaxUnitsPerBatch units, kInitialMatches matches) and grow only if a batch
// needs more: device buffers are then reallocated in stream order on the batch's stream (no
// device-wide synchronization, so copies queued on the copy streams keep flowing), and the
// outgrown pinned host buffers are kept until the server is freed (freeing pinned memory
// synchronizes the device).
int ScanBatch::ensure_buffers(uint64_t tiles, uint64_t segs, uint64_t out) {
  auto dev_alloc = [&](void** p, size_t bytes) -> int {
    CV_CUDA(cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, stream));
    return CV_OK;
  };
  auto dev_free = [&](void* p) {
    if (p) cudaFreeAsync(p, stream);
  };
  if (tiles > cap_tiles || !hit_rec) {
    uint64_t c = std::max<uint64_t>(tiles, cap_tiles * 2);
    for (void* p : {(void*)hit_rec, (void*)tile_nhit, (void*)tile_ntrip, (void*)tile_off, (void*)off_scratch})
      dev_free(p);
    hit_rec = nullptr;
    CV_TRY(dev_alloc((void**)&hit_rec, c * 32 * sizeof(uint4)));
    CV_TRY(dev_alloc((void**)&tile_nhit, c * 4));
    CV_TRY(dev_alloc((void**)&tile_ntrip, c * 8));
    CV_TRY(dev_alloc((void**)&tile_off, c * 8));
    CV_TRY(dev_alloc((void**)&off_scratch, tile_offsets_scratch_words(c) * 8));
    cap_tiles = c;
  }
  if (segs > cap_segs || !segs_d) {
    uint64_t c = std::max<uint64_t>(segs, cap_segs * 2);
    dev_free(segs_d);
    dev_free(counters_d);
    if (counters_h) retired_host.push_back(counters_h);
    if (segs_h) retired_host.push_back(segs_h);
    counters_h = nullptr;
    segs_h = nullptr;
    CV_TRY(dev_alloc((void**)&segs_d, c * sizeof(Segment)));
    CV_TRY(dev_alloc((void**)&counters_d, (c + 2) * 8));
    CV_CUDA(cudaMallocHost((void**)&counters_h, (c + 2) * 8));
    CV_CUDA(cudaMallocHost((void**)&segs_h, c * sizeof(Segment)));
    cap_segs = c;
  }
  if (out > cap_out || !out_d) {
    uint64_t c = std::max<uint64_t>(std::max<uint64_t>(out, 1024), cap_out * 2);
    dev_free(out_d);
    if (out_h) retired_host.push_back(out_h);
    out_h = nullptr;
    CV_TRY(dev_alloc((void**)&out_d, c * sizeof(MatchOut)));
    CV_CUDA(cudaMallocHost((void**)&out_h, c * sizeof(MatchOut)));
    cap_out = c;
  }
  return CV_OK;
}

void ScanBatch::release() {
  if (stream) {
    for (void* p : {(void*)segs_d, (void*)hit_rec, (void*)tile_nhit, (void*)tile_ntrip, (void*)tile_off,
                    (void*)off_scratch, (void*)counters_d, (void*)out_d})
      if (p) cudaFreeAsync(p, stream);
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
  if (counts_ready) cudaEventDestroy(counts_ready);
  if (matches_ready) cudaEventDestroy(matches_ready);
  if (counters_h) cudaFreeHost(counters_h);
  if (segs_h) cudaFreeHost(segs_h);
  if (out_h) cudaFreeHost(out_h);
  for (void* p : retired_host) cudaFreeHost(p);
}

}  // namespace

void cv_server::finish(Request* r) {
  r->done = true;
  r->done_at = Clock::now();
  if (r->error == CV_OK) {
    const double ms = std::chrono::duration<double, std::milli>(r->done_at - r->submitted).count();
    r->result = make_host_result(dev, r->matches.data(), r->matches.size(), r->n_sectors, (float)ms);
    if (!r->result) r->error = CV_ENOMEM;
    std::vector<MatchOut>().swap(r->matches);
    st.completed++;
    st.bytes_scanned += r->n_sectors * kSector;
    lat_ms.push_back(ms);
    last_done = r->done_at;
  } else {
    st.failed++;
  }
}

// Copies: round robin over live requests, one unit per request per pass, while slots and the
// copy cap last; the request with the fewest bytes left to copy goes first, so a small request
// is not queued behind the rest of a large one.
int cv_server::issue_copies(const std::vector<Request*>& work) {
  std::vector<Request*> order;
  for (Request* r : work)
    if (!r->device && r->next_copy < r->units.size()) order.push_back(r);
  const auto left = [](const Request* r) { return r->n_sectors - r->units[r->next_copy].first_sector; };
  std::stable_sort(order.begin(), order.end(), [&](const Request* a, const Request* b) { return left(a) < left(b); });
  bool issued = true;
  while (issued && !free_slots.empty()) {
    issued = false;
    for (Request* r : order) {
      if (free_slots.empty()) break;
      if (r->next_copy >= r->units.size()) continue;
      Unit& u = r->units[r->next_copy];
      if (copy_queued && copy_queued + u.n_sectors * kSector > copy_cap) continue;
      u.slot = free_slots.back();
      free_slots.pop_back();
      u.copy_stream = (int)(r->next_copy % copy_streams.size());
      cudaStream_t cs = copy_streams[u.copy_stream];
      CV_CUDA(cudaMemcpyAsync(arena + (uint64_t)u.slot * unit_bytes, r->data + u.first_sector * kSector,
                              u.n_sectors * kSector, cudaMemcpyHostToDevice, cs));
      CV_CUDA(cudaEventRecord(slot_event[u.slot], cs));
      u.copied = true;
      bytes_in_flight += u.n_sectors * kSector;
      copy_queued += u.n_sectors * kSector;
      st.peak_bytes_in_flight = std::max(st.peak_bytes_in_flight, bytes_in_flight);
      r->next_copy++;
      issued = true;
    }
  }
  return CV_OK;
}

// Gather every unit that is on the device (in order per request) into batch b and launch its
// scan, offset pass and the copy of its counts; *launched is false when no unit was ready.
int cv_server::launch_scan(ScanBatch& b, const std::vector<Request*>& work, bool* launched) {
  *launched = false;
  Job job;
  int n_ops = 0;
  const ScanCfg& cfg = scan_configs(&n_ops)[cfg_i];
  int live_in_batch = 0;
  job.maps.push_back(arena_map);
  job.map_base.push_back((uintptr_t)arena);
  b.refs.clear();
  for (Request* r : work) {
    bool any = false;
    while (r->next_scan < r->units.size() && b.refs.size() < kMaxUnitsPerBatch) {
      Unit& u = r->units[r->next_scan];
      if (!r->device) {
        if (!u.copied) break;
        cudaError_t q = cudaEventQuery(slot_event[u.slot]);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return cuda_fail(q);
        copy_queued -= u.n_sectors * kSector;  // each unit is gathered once
        Segment sg;
        sg.n_sectors = u.n_sectors;
        sg.tile_base = job.n_tiles;
        sg.sector_base = u.first_sector;
        sg.row_base = (uint64_t)u.slot * unit_sectors;
        sg.image = (uint32_t)b.refs.size();
        sg.map = 0;
        sg.bytes = arena + (uint64_t)u.slot * unit_bytes;
        job.segs.push_back(sg);
        job.n_tiles += (u.n_sectors + cfg.T - 1) / cfg.T;
        job.n_sectors += u.n_sectors;
      } else {
        const size_t before = job.segs.size();
        CV_TRY(job.add(ctx, cfg, r->data + u.first_sector * kSector, u.n_sectors, u.first_sector,
                       (uint32_t)b.refs.size(), true));
        if (job.segs.size() != before + 1) return CV_EINVAL;  // units never exceed a segment
      }
      b.refs.push_back(ScanBatch::Ref{r, r->next_scan});
      r->next_scan++;
      any = true;
    }
    live_in_batch += any ? 1 : 0;
  }
  if (b.refs.empty()) return CV_OK;
  *launched = true;
  b.nseg = job.segs.size();
  b.n_out = job.n_tiles * (uint64_t)(cfg.T / 32);
  CV_TRY(b.ensure_buffers(b.n_out, b.nseg, 0));
  memcpy(b.segs_h, job.segs.data(), b.nseg * sizeof(Segment));
  CV_CUDA(cudaMemcpyAsync(b.segs_d, b.segs_h, b.nseg * sizeof(Segment), cudaMemcpyHostToDevice, b.stream));
  uint32_t* status = (uint32_t*)(b.counters_d + b.nseg + 1);
  CV_CUDA(cudaMemsetAsync(status, 0, 8, b.stream));
  ScanParams p;
  memset(&p, 0, sizeof p);
  p.tab = tab;
  p.hit_rec = b.hit_rec;
  p.tile_nhit = b.tile_nhit;
  p.tile_ntrip = b.tile_ntrip;
  p.status = status;
  CV_TRY(launch_range(ctx, cfg_i, false, job, b.segs_d, 0, b.nseg, p, b.stream));
  CV_CUDA((cudaError_t)launch_tile_offsets(b.tile_ntrip, b.n_out, b.tile_off, b.segs_d, (uint32_t)b.nseg,
                                           (uint32_t)(cfg.T / 32), b.counters_d, b.counters_d + b.nseg,
                                           b.off_scratch, b.stream, status));
  CV_CUDA(cudaMemcpyAsync(b.counters_h, b.counters_d, (b.nseg + 2) * 8, cudaMemcpyDeviceToHost, b.stream));
  CV_CUDA(cudaEventRecord(b.counts_ready, b.stream));
  b.state = ScanBatch::kCounting;
  st.iterations++;
  st.units += b.refs.size();
  live_sum += live_in_batch;
  return CV_OK;
}

// The counts of batch b are on the host: check its status and launch its expansion and the copy
// of its matches.
int cv_server::launch_expand_of(ScanBatch& b) {
  b.total = b.counters_h[b.nseg];
  const uint32_t st0 = (uint32_t)b.counters_h[b.nseg + 1];
  if (st0 & kStTimeout) return CV_ETIMEOUT;
  if (st0) return CV_ECORRUPT;
  if (b.total) {
    int n_ops = 0;
    const ScanCfg& cfg = scan_configs(&n_ops)[cfg_i];
    CV_TRY(b.ensure_buffers(0, 0, b.total));
    uint32_t* status = (uint32_t*)(b.counters_d + b.nseg + 1);
    CV_CUDA((cudaError_t)launch_expand(cfg, b.hit_rec, b.tile_nhit, b.tile_off, b.n_out, b.segs_d,
                                       (uint32_t)b.nseg, tab, b.out_d, b.cap_out, status, ctx->sms, b.stream));
    CV_CUDA(cudaMemcpyAsync(b.out_h, b.out_d, b.total * sizeof(MatchOut), cudaMemcpyDeviceToHost, b.stream));
  }
  CV_CUDA(cudaEventRecord(b.matches_ready, b.stream));
  b.state = ScanBatch::kExpanding;
  return CV_OK;
}

// Batch b's matches are on the host: free its arena slots (scan and expand, which rereads units
// for byte confirmation, are done) and append each unit's matches to its request.
void cv_server::retire(ScanBatch& b) {
  std::vector<Request*> completed;
  for (size_t k = 0; k < b.refs.size(); k++) {
    Request* r = b.refs[k].r;
    Unit& u = r->units[b.refs[k].unit];
    if (u.slot >= 0) {
      free_slots.push_back(u.slot);
      bytes_in_flight -= u.n_sectors * kSector;
      u.slot = -1;
    }
    u.scanned = true;
    const uint64_t lo = b.counters_h[k], hi = (k + 1 < b.nseg) ? b.counters_h[k + 1] : b.total;
    r->matches.insert(r->matches.end(), b.out_h + lo, b.out_h + hi);
    if (b.refs[k].unit + 1 == r->units.size()) completed.push_back(r);
  }
  b.refs.clear();
  b.state = ScanBatch::kFree;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (Request* r : completed) {
      finish(r);
      live.erase(std::find(live.begin(), live.end(), r));
    }
  }
  if (!completed.empty()) cv_done.notify_all();
}

// One engine iteration: admit, issue copies, retire the oldest batch when its matches have
// landed, start the expansion of every batch whose counts have landed, and launch a scan of the
// units that have landed into a free batch. Nothing here waits for the GPU.
int cv_server::iterate(bool* did_work) {
  NvtxRange nvtx_range("cv.server.iteration");
  *did_work = false;
  std::vector<Request*> work;
  {
    std::lock_guard<std::mutex> lk(mu);
    while (!pending.empty() && live.size() < max_live) {
      live.push_back(pending.front());
      pending.pop_front();
    }
    work = live;
  }
  if (work.empty() && in_flight.empty()) return CV_OK;
  CV_TRY(issue_copies(work));
  while (!in_flight.empty()) {
    ScanBatch& b = batch[in_flight.front()];
    if (b.state != ScanBatch::kExpanding) break;
    const cudaError_t q = cudaEventQuery(b.matches_ready);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return cuda_fail(q);
    in_flight.pop_front();
    retire(b);
    *did_work = true;
  }
  for (int i : in_flight) {
    ScanBatch& b = batch[i];
    if (b.state != ScanBatch::kCounting) continue;
    const cudaError_t q = cudaEventQuery(b.counts_ready);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return cuda_fail(q);
    CV_TRY(launch_expand_of(b));
    *did_work = true;
  }
  for (int i = 0; i < kBatchesInFlight; i++) {
    ScanBatch& b = batch[i];
    if (b.state != ScanBatch::kFree) continue;
    bool launched = false;
    CV_TRY(launch_scan(b, work, &launched));
    if (launched) {
      in_flight.push_back(i);
      *did_work = true;
    }
    break;  // one new batch per iteration
  }
  return CV_OK;
}

void cv_server::run() {
  cudaSetDevice(dev);
  while (true) {
    bool did = false;
    const int rc = iterate(&did);
    if (rc != CV_OK) {
      // A device-side failure ends the server: every admitted and queued request fails.
      std::lock_guard<std::mutex> lk(mu);
      fatal = rc;
      for (Request* r : live) {
        r->error = rc;
        finish(r);
      }
      live.clear();
      for (Request* r : pending) {
        r->error = rc;
        finish(r);
      }
      pending.clear();
      cv_done.notify_all();
      return;
    }
    std::unique_lock<std::mutex> lk(mu);
    if (stopping && live.empty() && pending.empty() && in_flight.empty()) return;
    if (!did) {
      if (live.empty() && pending.empty() && in_flight.empty()) {
        cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
    }
  }
}

extern "C" {

int cv_server_create(const cv_master* m, const cv_server_opts* opts, cv_server** out) {
  if (!m || !out) return CV_EINVAL;
  *out = nullptr;
  if (opts && opts->struct_size < offsetof(cv_server_opts, max_copy_bytes)) return CV_EINVAL;
  const uint64_t copy_cap_opt = (opts && opts->struct_size >= sizeof(cv_server_opts)) ? opts->max_copy_bytes : 0u;
  TableView tab;
  int mdev;
  if (master_view(m, &tab, &mdev) != CV_OK || tab.unit != kUnitSector) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  if (ctx->dev != mdev) return CV_EINVAL;
  int ncfg;
  const ScanCfg* cfgs = scan_configs(&ncfg);
  int cfg_i = ctx->default_config(table_kind(tab));
  if (opts && opts->kernel_config) {
    if (opts->kernel_config > (uint32_t)ncfg) return CV_EINVAL;
    cfg_i = (int)opts->kernel_config - 1;
  }
  scan_config_for(cfg_i, table_kind(tab), &cfg_i);
  uint64_t unit = (opts && opts->work_unit_bytes) ? opts->work_unit_bytes : (64ull << 20);
  uint64_t budget = (opts && opts->hbm_budget_bytes) ? opts->hbm_budget_bytes : (8ull << 30);
  if (unit % kSector || unit > kMaxSegmentSectors * kSector || budget < unit) return CV_EINVAL;
  const uint64_t slots = budget / unit;
  if (slots > (1u << 20) || (slots * unit) / kSector >= (1ull << 31)) return CV_EINVAL;
  const uint32_t n_copy = (opts && opts->copy_streams) ? opts->copy_streams : 2u;
  if (n_copy > 16) return CV_EINVAL;

  cv_server* s = new (std::nothrow) cv_server();
  if (!s) return CV_ENOMEM;
  s->magic = kMagicServer;
  s->dev = ctx->dev;
  s->ctx = ctx;
  s->cfg_i = cfg_i;
  s->tab = tab;
  s->unit_bytes = unit;
  s->copy_cap = copy_cap_opt ? copy_cap_opt : (2ull << 30);
  s->unit_sectors = unit / kSector;
  s->max_live = (opts && opts->max_live) ? opts->max_live : 64u;
  s->n_slots = (int)slots;
  memset(&s->st, 0, sizeof s->st);
  auto body = [&]() -> int {
    CV_CUDA(cudaMalloc((void**)&s->arena, slots * unit));
    CV_TRY(make_tmap(ctx, cfgs[cfg_i], s->arena, slots * unit / kSector, &s->arena_map));
    const uint64_t batch_units = std::min<uint64_t>(kMaxUnitsPerBatch, slots);
    const uint64_t batch_tiles = batch_units * ((s->unit_sectors + cfgs[cfg_i].T - 1) / cfgs[cfg_i].T) *
                                 (uint64_t)(cfgs[cfg_i].T / 32);
    for (ScanBatch& b : s->batch) {
      CV_CUDA(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
      CV_CUDA(cudaEventCreateWithFlags(&b.counts_ready, cudaEventDisableTiming));
      CV_CUDA(cudaEventCreateWithFlags(&b.matches_ready, cudaEventDisableTiming));
      b.pool = ctx->pool;
      CV_TRY(b.ensure_buffers(batch_tiles, kMaxUnitsPerBatch, kInitialMatches));
    }
    for (uint32_t k = 0; k < n_copy; k++) {
      cudaStream_t cs;
      CV_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      s->copy_streams.push_back(cs);
    }
    for (uint64_t k = 0; k < slots; k++) {
      cudaEvent_t e;
      CV_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      s->slot_event.push_back(e);
      s->free_slots.push_back((int)(slots - 1 - k));
    }
    return CV_OK;
  };
  int rc = body();
  if (rc != CV_OK) {
    cvk_server_free(s);
    return rc;
  }
  s->engine = std::thread([s] { s->run(); });
  *out = s;
  return CV_OK;
}

int cv_submit(cv_server* s, cv_buf image, uint64_t tag, uint64_t* ticket) {
  if (!s || s->magic != kMagicServer || !ticket) return CV_EINVAL;
  const uint64_t ns = image.n_bytes / kSector;
  if (ns && !image.data) return CV_EINVAL;
  BufKind kind = kHost;
  if (ns) CV_TRY(classify(s->ctx, image.data, &kind));
  if (kind == kDevice && ((uintptr_t)image.data & 15u)) return CV_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return CV_ENOMEM;
  r->tag = tag;
  r->data = (const uint8_t*)image.data;
  r->n_sectors = ns;
  r->device = kind == kDevice;
  for (uint64_t a = 0; a < ns; a += s->unit_sectors) {
    Unit u;
    u.first_sector = a;
    u.n_sectors = std::min(s->unit_sectors, ns - a);
    u.on_device = r->device;
    r->units.push_back(u);
  }
  r->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      delete r;
      return CV_EINVAL;
    }
    if (s->fatal != CV_OK) {
      delete r;
      return s->fatal;
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->by_ticket[r->ticket] = r;
    s->st.submitted++;
    if (!s->any_submit) {
      s->any_submit = true;
      s->first_submit = r->submitted;
    }
    if (r->units.empty()) {
      s->finish(r);  // nothing to scan: done at once
    } else {
      s->pending.push_back(r);
    }
  }
  s->cv_work.notify_one();
  if (r->units.empty()) s->cv_done.notify_all();
  return CV_OK;
}

int cv_poll(cv_server* s, uint64_t ticket, int timeout_ms, cv_result** out) {
  if (!s || s->magic != kMagicServer || !out) return CV_EINVAL;
  *out = nullptr;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return CV_EINVAL;
  Request* r = it->second;
  if (!r->done) {
    if (timeout_ms == 0) return CV_EAGAIN;
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) {
      s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
      return CV_EAGAIN;
    }
  }
  const int err = r->error;
  *out = r->result;
  s->by_ticket.erase(it);
  delete r;
  return err;
}

int cv_server_get_stats(cv_server* s, cv_server_stats* st) {
  if (!s || s->magic != kMagicServer || !st) return CV_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  std::vector<double> l = s->lat_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (double)(l.size() - 1) + 0.5))]; };
    st->p50_ms = q(0.50);
    st->p99_ms = q(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    st->mean_ms = sum / (double)l.size();
    st->max_ms = l.back();
    st->wall_s = std::chrono::duration<double>(s->last_done - s->first_submit).count();
  }
  st->mean_live_per_iteration = s->st.iterations ? s->live_sum / (double)s->st.iterations : 0.0;
  return CV_OK;
}

}  // extern "C"

void cvk_server_free(void* h) {
  cv_server* s = (cv_server*)h;
  if (!s || s->magic != kMagicServer) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  if (s->engine.joinable()) s->engine.join();
  s->magic = 0;
  for (auto& kv : s->by_ticket) {
    if (kv.second->result) cv_free(kv.second->result);
    delete kv.second;
  }
  for (ScanBatch& b : s->batch) b.release();
  for (cudaStream_t cs : s->copy_streams) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  for (cudaEvent_t e : s->slot_event) cudaEventDestroy(e);
  if (s->arena) cudaFree(s->arena);
  delete s;
}
