// Host runtime shared by the library's entry points (not part of the ABI): per-device context,
// stream-ordered temporaries, tensor maps, scan jobs (segments over device memory) and the
// launch of the scan kernel over a job.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cv.h"
#include "cv_internal.h"
#include "cv_launch.h"

namespace cvk {

// A named range on the host timeline for tools that record NVTX (build, scan phases, engine
// iterations); without such a tool attached each push and pop is a no-op call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { end(); }
  void end() {  // close the range early (once)
    if (open_) nvtxRangePop();
    open_ = false;
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;

 private:
  bool open_ = true;
};

// Records the failing CUDA code for cv_last_cuda_error and maps it to a CV_E* code.
int cuda_fail(cudaError_t e);
void set_last_cuda(int code);
int last_cuda();

#define CV_CUDA(expr)                                 \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return ::cvk::cuda_fail(e_); \
  } while (0)

#define CV_TRY(expr)            \
  do {                          \
    int r_ = (expr);            \
    if (r_ != CV_OK) return r_; \
  } while (0)

// Library state of one device, made on first use with that device current.
struct DevCtx {
  bool ready = false;
  int dev = -1;
  int sms = 0;
  cudaMemPool_t pool = nullptr;      // stream-ordered temporaries and results
  cudaStream_t copy_stream = nullptr;  // host-to-device copies of streamed images
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  PFN_cuMemGetAddressRange_v3020 address_range = nullptr;
  std::vector<std::array<int, kTableKinds>> blocks_per_sm;  // per scan configuration and table kind
  std::vector<int> blocks_per_sm_digest;  // per scan configuration (0: no digest-mode kernels)
  int cfg_index = -1;  // scan configuration forced by CV_SCAN_CONFIG, or -1: per table kind

  // The scan configuration for a table kind when the caller asks for the default.
  int default_config(int kind) const { return cfg_index >= 0 ? cfg_index : preferred_config(kind); }

  // Timing events of finished calls, kept for later calls: creating and destroying four events
  // per scan cost host time while the device waited for the next call.
  std::mutex ev_mutex;
  std::vector<cudaEvent_t> ev_free;
  int take_events(cudaEvent_t* ev, int n);     // n timing events, reused or new
  void give_events(cudaEvent_t* ev, int n);   // back for reuse (their work on the device done); nulls them
};

int get_ctx(DevCtx** out);

// Stream-ordered temporaries from the device pool, released on the stream when the scope ends.
struct Temps {
  DevCtx* ctx;
  cudaStream_t stream;
  std::vector<void*> ptrs;
  Temps(DevCtx* c, cudaStream_t s) : ctx(c), stream(s) {}
  ~Temps();
  int alloc_bytes(void** out, size_t bytes);
  template <typename P>
  int alloc(P** out, size_t bytes) {
    void* p = nullptr;
    int rc = alloc_bytes(&p, bytes);
    *out = (P*)p;
    return rc;
  }
};

enum BufKind { kHost = 0, kDevice = 1 };
int classify(DevCtx* ctx, const void* p, BufKind* kind);

// Several device arrays carved out of one pool allocation (256-byte aligned each), so that a
// call makes one allocation for its scratch instead of one per array.
struct Carve {
  struct Part {
    void** slot;
    size_t off;
  };
  std::vector<Part> parts;
  size_t total = 0;
  template <typename P>
  void add(P** slot, size_t bytes) {
    parts.push_back(Part{reinterpret_cast<void**>(slot), total});
    total += (bytes + 255) & ~(size_t)255;
  }
  int commit(Temps& tmp) {
    void* base = nullptr;
    const int rc = tmp.alloc_bytes(&base, total);
    if (rc != CV_OK) return rc;
    for (const Part& q : parts) *q.slot = static_cast<char*>(base) + q.off;
    return CV_OK;
  }
};

// A 2-D tensor map viewing n_rows sectors at base as u32[n_rows][128] with the staging box of cfg.
int make_tmap(DevCtx* ctx, const ScanCfg& cfg, const void* base, uint64_t n_rows, CUtensorMap* out);

// A list of segments over device memory (or over not-yet-filled streaming buffers).
struct Job {
  std::vector<Segment> segs;
  std::vector<CUtensorMap> maps;
  std::vector<uintptr_t> map_base;  // device address of row 0 of each map (0: made later)
  uint64_t n_tiles = 0;
  uint64_t n_sectors = 0;

  // Append n whole sectors at base (split at kMaxSegmentSectors). With share_alloc, images that
  // lie in one device allocation at sector-aligned offsets share one tensor map over the whole
  // allocation; otherwise each segment gets its own map. base == nullptr reserves segments
  // whose map is set later (set_map).
  int add(DevCtx* ctx, const ScanCfg& cfg, const void* base, uint64_t n, uint64_t sector_base, uint32_t image,
          bool share_alloc);
  // Point segment s at a fresh map over base (streamed chunks).
  int set_map(DevCtx* ctx, const ScanCfg& cfg, size_t s, const void* base);
};

// Launch the scan (or digest) kernel over segments [s0, s1) of the job; segs_d is the job's
// segment array in device memory. `base` carries the table and output pointers. Returns the
// number of kernel launches through *launches when non-null.
int launch_range(DevCtx* ctx, int cfg_i, bool digest, const Job& job, const Segment* segs_d, size_t s0, size_t s1,
                 const ScanParams& base, cudaStream_t stream, int* launches = nullptr);

uint64_t next_pow2(uint64_t x);
unsigned grid_for(uint64_t n, int threads, int sms);

// Device view of a master table (capi.cu).
int master_view(const cv_master* m, TableView* tab, int* dev);

// Variants of a built sector table (master.cu), for the batch autotuner. table_sorted_copy: the
// sorted layout of a hash-layout table (its own record and key arrays, *slots_out and *keys0_out,
// owned by the caller; postings, Bloom filter and confirmation copy shared). table_bloom: a
// blocked Bloom filter of bits_per_key bits per distinct key over the table's records
// (*bloom_out owned by the caller). Both return after the work has finished.
int table_sorted_copy(const TableView& tab, cudaStream_t stream, TableView* out, void** slots_out, void** keys0_out);
int table_bloom(const TableView& tab, uint32_t bits_per_key, cudaStream_t stream, TableView* out, void** bloom_out);

// A one-image host result holding a copy of n triples (capi.cu).
cv_result* make_host_result(int dev, const MatchOut* data, uint64_t n, uint64_t sectors, float total_ms);

}  // namespace cvk
