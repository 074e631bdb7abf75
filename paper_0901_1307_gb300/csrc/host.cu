// cv_host_alloc / cv_host_free: host memory for images that are copied to the GPU.
//
// The paper's system reads drives into host buffers and copies them to the GPU (Section 3.1,
// Figure 7); how fast those copies run depends on how the host memory is mapped. On a GB300
// the GPU reads host memory through the CPU's own page tables. Measured on its Grace host
// (64 KiB base pages, 512 MiB transparent huge pages), 8 GiB copies with a serving loop and
// its client running between them:
//   - memory in base pages (cudaHostAlloc memory; memory registered with cudaHostRegister,
//     locked with mlock or not) fell from 210 GB/s to 3-20 GB/s within a minute, with a host
//     page fault for most 64 KiB pages on every pass, in every process tried;
//   - memory in huge pages kept 210 GB/s with no faults through four to six served runs in
//     two processes, and requests served from it kept a 0.21 ms median (base pages: up to
//     120 ms); in two other processes the kernel split some of its huge pages back into base
//     pages during the first served run (11 of 64 in one), and the split part degraded as
//     base pages do;
//   - host memory allocated by the CUDA driver itself (cuMemCreate on a host NUMA node)
//     never faulted but copied at 90 GB/s.
// Huge pages are the best of these, and never worse than base pages, so a block is: a private
// anonymous mapping aligned to the huge-page size and a multiple of it, advised for huge
// pages, every page written once by the host (which is when the kernel backs it, with huge
// pages where it can), locked where the process may lock memory, and registered with the
// CUDA driver.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <sys/mman.h>
#include <unistd.h>

#include <map>
#include <mutex>

#include "cv.h"
#include "runtime.h"

using namespace cvk;

namespace {

struct Block {
  void* raw;        // the mapping
  size_t raw_bytes;
  size_t bytes;     // registered, from the aligned start
};

std::mutex g_host_mutex;
std::map<uintptr_t, Block> g_host_blocks;  // aligned start -> block

// The kernel's transparent huge page size (PMD size), else 2 MiB.
size_t huge_page_bytes() {
  size_t v = 0;
  if (FILE* f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long x = 0;
    if (fscanf(f, "%llu", &x) == 1) v = (size_t)x;
    fclose(f);
  }
  return (v >= 4096 && (v & (v - 1)) == 0) ? v : (size_t)2 << 20;
}

}  // namespace

extern "C" {

int cv_host_alloc(uint64_t n_bytes, void** out) {
  if (!out) return CV_EINVAL;
  *out = nullptr;
  if (n_bytes == 0) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  const size_t huge = huge_page_bytes();
  if (n_bytes > (uint64_t)SIZE_MAX - 2 * huge) return CV_ENOMEM;
  const size_t bytes = ((size_t)n_bytes + huge - 1) / huge * huge;
  const size_t raw_bytes = bytes + huge;
  void* raw = mmap(nullptr, raw_bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return CV_ENOMEM;
  uint8_t* p = (uint8_t*)(((uintptr_t)raw + huge - 1) / huge * huge);
#ifdef MADV_HUGEPAGE
  madvise(p, bytes, MADV_HUGEPAGE);  // a request; without huge pages the block still works
#endif
  const long page = sysconf(_SC_PAGESIZE);
  const size_t step = page > 0 ? (size_t)page : 4096u;
  volatile uint8_t* b = p;
  for (size_t off = 0; off < bytes; off += step) b[off] = 0;
  (void)mlock(p, bytes);  // best effort: refused without RLIMIT_MEMLOCK room, harmless then
  const cudaError_t e = cudaHostRegister(p, bytes, cudaHostRegisterDefault);
  if (e != cudaSuccess) {
    munmap(raw, raw_bytes);
    return cuda_fail(e);
  }
  {
    std::lock_guard<std::mutex> lk(g_host_mutex);
    g_host_blocks[(uintptr_t)p] = Block{raw, raw_bytes, bytes};
  }
  *out = p;
  return CV_OK;
}

int cv_host_free(void* p) {
  if (!p) return CV_OK;
  Block blk;
  {
    std::lock_guard<std::mutex> lk(g_host_mutex);
    auto it = g_host_blocks.find((uintptr_t)p);
    if (it == g_host_blocks.end()) return CV_EINVAL;
    blk = it->second;
    g_host_blocks.erase(it);
  }
  const cudaError_t e = cudaHostUnregister(p);
  munmap(blk.raw, blk.raw_bytes);  // also unlocks
  return e == cudaSuccess ? CV_OK : cuda_fail(e);
}

}  // extern "C"
