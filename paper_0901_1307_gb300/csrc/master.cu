// Master tables: cv_master_build (master bytes -> device arena -> per-unit signatures -> table
// insert -> radix sort by slot -> postings + slots -> filters, optionally the sorted layout),
// cv_master_get_info, and cv_master_save / cv_master_load (the table in a file).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "cv.h"
#include "cv_internal.h"
#include "cv_launch.h"
#include "handles.h"
#include "runtime.h"
#include "table_build.cuh"

using namespace cvk;

namespace {

// Stable LSD radix sort of n (key, value) pairs by the low `bits` bits of the key, 8 bits per
// pass, ping-ponging between (k0, v0) and (k1, v1); *kres/*vres receive the pair holding the
// result.
int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint64_t n, int bits, Temps& tmp,
                     cudaStream_t stream, uint32_t** kres, uint32_t** vres) {
  const uint32_t nb = (uint32_t)((n + kRsChunk - 1) / kRsChunk);
  const uint64_t nh = (uint64_t)std::max<uint32_t>(nb, 1) * 256;
  const uint32_t nc = (uint32_t)((nh + kScanChunk - 1) / kScanChunk);
  uint32_t *hist, *sums;
  CV_TRY(tmp.alloc(&hist, nh * 4));
  CV_TRY(tmp.alloc(&sums, (uint64_t)nc * 4));
  for (int shift = 0; shift < bits && n; shift += 8) {
    rs_hist_kernel<<<nb, kRsThreads, 0, stream>>>(k0, n, shift, hist, nb);
    scan_chunk_sums_u32_kernel<<<nc, kScanThreads, 0, stream>>>(hist, (uint64_t)nb * 256, sums);
    scan_sums_u32_kernel<<<1, 1024, 0, stream>>>(sums, nc);
    scan_chunks_u32_kernel<<<nc, kScanThreads, 0, stream>>>(hist, (uint64_t)nb * 256, sums);
    rs_scatter_kernel<<<nb, kRsThreads, 0, stream>>>(k0, v0, k1, v1, n, shift, hist, nb);
    CV_CUDA(cudaGetLastError());
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  *kres = k0;
  *vres = v0;
  return CV_OK;
}

// One copy of the gather stage: bytes from src to dst_base + dst.
struct CopyPiece {
  const uint8_t* src;
  uint64_t dst;
  uint64_t bytes;
};

constexpr uint64_t kPieceBytes = 4ull << 20;   // device runs are cut into pieces of this size
constexpr uint64_t kHostDirect = 4ull << 20;   // host runs this long are copied by the driver
constexpr uint64_t kStageBytes = 64ull << 20;  // pinned staging chunk for shorter host runs

// Each block copies whole pieces (grid-stride over them), 16 bytes at a time when the source,
// the destination and the length allow it, else byte by byte.
__global__ void gather_pieces_kernel(const CopyPiece* pieces, uint32_t n, uint8_t* dst_base) {
  for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
    const CopyPiece c = pieces[r];
    uint8_t* d = dst_base + c.dst;
    if ((((uintptr_t)c.src | (uintptr_t)d | c.bytes) & 15u) == 0) {
      const uint4* s4 = reinterpret_cast<const uint4*>(c.src);
      uint4* d4 = reinterpret_cast<uint4*>(d);
      for (uint64_t i = threadIdx.x; i < c.bytes / 16; i += blockDim.x) d4[i] = s4[i];
    } else {
      for (uint64_t i = threadIdx.x; i < c.bytes; i += blockDim.x) d[i] = c.src[i];
    }
  }
}

int launch_gather(const std::vector<CopyPiece>& pieces, uint8_t* dst_base, int sms, Temps& tmp, cudaStream_t stream) {
  if (pieces.empty()) return CV_OK;
  CopyPiece* d;
  CV_TRY(tmp.alloc(&d, pieces.size() * sizeof(CopyPiece)));
  CV_CUDA(cudaMemcpyAsync(d, pieces.data(), pieces.size() * sizeof(CopyPiece), cudaMemcpyHostToDevice, stream));
  const uint64_t g = std::min<uint64_t>(pieces.size(), (uint64_t)sms * 8);
  gather_pieces_kernel<<<(unsigned)g, 256, 0, stream>>>(d, (uint32_t)pieces.size(), dst_base);
  CV_CUDA(cudaGetLastError());
  return CV_OK;
}

// The whole units of every file into the arena (file f's at arena + file_base[f] * U). One
// copy call per file costs microseconds of host time each, which dominated the build of master
// sets of many small files. So: files contiguous in memory are merged into runs; runs in this
// GPU's memory are copied by one gather launch; host runs of kHostDirect bytes or more by the
// driver, one call each; shorter host runs are packed by the host into a pinned staging chunk,
// copied to the device in one call per chunk and scattered by a gather launch; anything else
// (managed memory, another GPU's) by the driver. Memory is classified once per CUDA allocation
// (cuMemGetAddressRange), not once per file.
//
// *units receives where the build reads the units from: the arena (allocated here), or, when
// every unit already lies in one 16-byte-aligned run of this GPU's memory in file order, that
// memory itself, with no copy and no arena.
int gather_master_units(DevCtx* ctx, const cv_buf* files, uint32_t n_files, const std::vector<uint64_t>& file_base,
                        uint64_t U, Temps& tmp, cudaStream_t stream, const uint8_t** units) {
  std::vector<CopyPiece> runs;
  for (uint32_t f = 0; f < n_files; f++) {
    const uint64_t bytes = (file_base[f + 1] - file_base[f]) * U;
    if (!bytes) continue;
    const uint8_t* src = (const uint8_t*)files[f].data;
    const uint64_t dst = file_base[f] * U;
    if (!runs.empty() && runs.back().src + runs.back().bytes == src && runs.back().dst + runs.back().bytes == dst)
      runs.back().bytes += bytes;
    else
      runs.push_back(CopyPiece{src, dst, bytes});
  }
  const uint64_t total_bytes = file_base[n_files] * U;
  *units = nullptr;
  if (total_bytes == 0) return CV_OK;
  if (runs.size() == 1 && runs[0].dst == 0 && runs[0].bytes == total_bytes && ((uintptr_t)runs[0].src & 15u) == 0) {
    CUdeviceptr ab = 0;
    size_t asz = 0;
    cudaPointerAttributes at;
    const uintptr_t a = (uintptr_t)runs[0].src;
    if (ctx->address_range && ctx->address_range(&ab, &asz, (CUdeviceptr)a) == CUDA_SUCCESS &&
        a + total_bytes <= (uintptr_t)ab + asz) {
      if (cudaPointerGetAttributes(&at, runs[0].src) == cudaSuccess) {
        if (at.type == cudaMemoryTypeDevice && at.device == ctx->dev) {
          *units = runs[0].src;
          return CV_OK;
        }
      } else {
        cudaGetLastError();
      }
    }
  }
  uint8_t* arena;
  CV_TRY(tmp.alloc(&arena, total_bytes));
  *units = arena;
  // Where a run lives: this GPU's memory (gathered by a kernel), host memory the CPU may read
  // (pageable, pinned or registered: staged, or copied by the driver when long), or anything
  // else (managed memory, another GPU's memory: copied by the driver).
  enum RunKind { kThisGpu, kHostMem, kByDriver };
  std::vector<CopyPiece> dev_pieces, host_short;
  uintptr_t lo = 0, hi = 0;  // the last CUDA allocation classified, and its kind
  RunKind lo_kind = kHostMem;
  for (size_t q = 0; q < runs.size(); q++) {
    CopyPiece r = runs[q];
    const uintptr_t a = (uintptr_t)r.src;
    RunKind kind = kHostMem;  // not inside a CUDA allocation: ordinary host memory
    if (a >= lo && a < hi) {
      kind = lo_kind;
    } else {
      CUdeviceptr ab = 0;
      size_t asz = 0;
      if (ctx->address_range && ctx->address_range(&ab, &asz, (CUdeviceptr)a) == CUDA_SUCCESS) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, r.src) != cudaSuccess) {
          cudaGetLastError();
          kind = kByDriver;
        } else if (at.type == cudaMemoryTypeDevice && at.device == ctx->dev) {
          kind = kThisGpu;
        } else {
          kind = at.type == cudaMemoryTypeHost ? kHostMem : kByDriver;
        }
        lo = (uintptr_t)ab;
        hi = lo + asz;
        lo_kind = kind;
      }
    }
    if (a >= lo && a < hi && a + r.bytes > hi) {
      // files merged across the end of an allocation: the rest is classified on its own
      const uint64_t head = hi - a;
      runs.push_back(CopyPiece{r.src + head, r.dst + head, r.bytes - head});
      r.bytes = head;
    }
    if (kind == kThisGpu) {
      for (uint64_t o = 0; o < r.bytes; o += kPieceBytes)
        dev_pieces.push_back(CopyPiece{r.src + o, r.dst + o, std::min(kPieceBytes, r.bytes - o)});
    } else if (kind == kByDriver || r.bytes >= kHostDirect) {
      CV_CUDA(cudaMemcpyAsync(arena + r.dst, r.src, r.bytes, cudaMemcpyDefault, stream));
    } else {
      host_short.push_back(r);
    }
  }
  CV_TRY(launch_gather(dev_pieces, arena, ctx->sms, tmp, stream));
  if (host_short.empty()) return CV_OK;
  // short host runs: pinned chunk -> device staging -> scattered into the arena
  uint64_t total = 0;
  for (const CopyPiece& r : host_short) total += r.bytes;
  const uint64_t chunk = std::min(total, kStageBytes);
  uint8_t* staged;
  CV_TRY(tmp.alloc(&staged, chunk));
  uint8_t* pinned = nullptr;
  CV_CUDA(cudaMallocHost((void**)&pinned, chunk));
  int rc = CV_OK;
  size_t i = 0;
  while (i < host_short.size() && rc == CV_OK) {
    std::vector<CopyPiece> pieces;
    uint64_t used = 0;
    for (; i < host_short.size() && used + host_short[i].bytes <= chunk; i++) {
      memcpy(pinned + used, host_short[i].src, host_short[i].bytes);
      pieces.push_back(CopyPiece{staged + used, host_short[i].dst, host_short[i].bytes});
      used += host_short[i].bytes;
    }
    cudaError_t e = cudaMemcpyAsync(staged, pinned, used, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    rc = launch_gather(pieces, arena, ctx->sms, tmp, stream);
    // the pinned chunk and the device staging are reused: wait before refilling them, and
    // before the pinned chunk is freed
    if (rc == CV_OK && (e = cudaStreamSynchronize(stream)) != cudaSuccess) rc = cuda_fail(e);
  }
  cudaFreeHost(pinned);
  return rc;
}

// The sorted layout of a hash table's occupied slots (Section 4: binary search for high
// occupancy): the nu occupied records, compacted in slot order, then sorted by h0 =
// tau_home(d0, tau) (a stable sort, so the order is deterministic), and their h0 words. The
// caller owns *slots_out (nu records of 32 bytes) and *keys0_out (nu words); *steps receives
// ceil(log2 nu), the bisection steps of a lookup. Returns after the work has finished.
int sorted_from_hash(DevCtx* ctx, const uint4* slots, uint64_t n_slots, uint32_t nu, Temps& tmp, cudaStream_t stream,
                     void** slots_out, void** keys0_out, uint32_t* steps) {
  uint32_t *ck, *cv, *ck2, *cv2, *kr, *vr;
  CV_TRY(tmp.alloc(&ck, n_slots * 4));
  CV_TRY(tmp.alloc(&cv, n_slots * 4));
  CV_TRY(tmp.alloc(&ck2, n_slots * 4));
  CV_TRY(tmp.alloc(&cv2, n_slots * 4));
  const unsigned gs = grid_for(n_slots, 256, ctx->sms);
  occupied_keys_kernel<<<gs, 256, 0, stream>>>(slots, (uint32_t)n_slots, ck, cv);
  CV_CUDA(cudaGetLastError());
  CV_TRY(radix_sort_pairs(ck, cv, ck2, cv2, n_slots, 1, tmp, stream, &kr, &vr));
  uint32_t* kfree = kr == ck ? ck2 : ck;  // the other key buffer is free for the h0 keys
  uint32_t* vfree = vr == cv ? cv2 : cv;
  const unsigned gu = grid_for(std::max<uint32_t>(nu, 1), 256, ctx->sms);
  h0_keys_kernel<<<gu, 256, 0, stream>>>(slots, vr, nu, kfree);
  CV_CUDA(cudaGetLastError());
  uint32_t *hk, *hv;
  CV_TRY(radix_sort_pairs(kfree, vr, kr, vfree, nu, 32, tmp, stream, &hk, &hv));
  void* out = nullptr;
  void* keys0 = nullptr;
  CV_CUDA(cudaMalloc(&out, std::max<uint64_t>(nu, 1) * 32));
  cudaError_t e = cudaMalloc(&keys0, std::max<uint64_t>(nu, 1) * 4);
  if (e != cudaSuccess) {
    cudaFree(out);
    return cuda_fail(e);
  }
  gather_slots_kernel<<<gu, 256, 0, stream>>>(slots, hv, nu, (uint4*)out);
  e = cudaGetLastError();
  if (e == cudaSuccess && nu) e = cudaMemcpyAsync(keys0, hk, (uint64_t)nu * 4, cudaMemcpyDeviceToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaFree(out);
    cudaFree(keys0);
    return cuda_fail(e);
  }
  *slots_out = out;
  *keys0_out = keys0;
  uint32_t st = 0;
  while ((1ull << st) < nu) st++;
  *steps = st;
  return CV_OK;
}

}  // namespace

extern "C" {

int cv_master_build(const cv_buf* files, uint32_t n_files, const cv_master_opts* opts, cv_master** out) {
  NvtxRange nvtx_range("cv.master_build");
  if (!out || (n_files && !files)) return CV_EINVAL;
  *out = nullptr;
  if (opts && opts->struct_size < offsetof(cv_master_opts, position_mode)) return CV_EINVAL;
  const bool has_v2 = opts && opts->struct_size >= offsetof(cv_master_opts, unit);
  const uint32_t position_mode = has_v2 ? opts->position_mode : CV_POSITION_ANY;
  if (position_mode > CV_POSITION_CLUSTER) return CV_EINVAL;
  const bool by_tau = position_mode == CV_POSITION_CLUSTER;
  uint32_t layout = has_v2 ? opts->layout : CV_LAYOUT_HASH;
  if (layout > CV_LAYOUT_AUTO) return CV_EINVAL;
  const uint32_t unit = (opts && opts->struct_size >= sizeof(cv_master_opts)) ? opts->unit : CV_UNIT_SECTOR;
  if (unit > CV_UNIT_FRAGMENT) return CV_EINVAL;
  const bool frag = unit == CV_UNIT_FRAGMENT;
  const uint64_t U = frag ? kFrag : kSector;  // bytes per master unit
  float max_load = (opts && opts->max_load > 0.f) ? opts->max_load : 0.5f;
  if (!(max_load > 0.f && max_load <= 0.9f)) return CV_EINVAL;
  uint32_t bpk = opts ? opts->bloom_bits_per_key : CV_BLOOM_AUTO;
  if (bpk == CV_BLOOM_AUTO) bpk = 16;
  if (bpk > 64) return CV_EINVAL;
  const int sig = opts ? (int)opts->signature : kSigMd5;
  if (sig < 0 || sig > kSigCrc64) return CV_EINVAL;
  if (frag && (!frag_sig_supported(sig) || by_tau)) return CV_EINVAL;
  cudaStream_t stream = opts ? (cudaStream_t)opts->stream : nullptr;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  int cfg_i;
  const ScanCfg& cfg = digest_config_for(ctx->cfg_index, sig, &cfg_i);

  // whole units (sectors or fragments) of every file, concatenated
  std::vector<uint64_t> file_base(n_files + 1, 0);
  for (uint32_t f = 0; f < n_files; f++) {
    if (files[f].n_bytes && !files[f].data) return CV_EINVAL;
    file_base[f + 1] = file_base[f] + files[f].n_bytes / U;
  }
  const uint64_t M = file_base[n_files];
  if (M >= (1ull << 27)) return CV_EINVAL;

  cv_master* m = (cv_master*)calloc(1, sizeof(cv_master));
  if (!m) return CV_ENOMEM;
  m->magic = kMagicMaster;
  m->dev = ctx->dev;
  int rc = CV_OK;
  {
    Temps tmp(ctx, stream);
    auto body = [&]() -> int {
      const uint64_t n_slots = std::max<uint64_t>(next_pow2((uint64_t)((double)M / max_load) + 1), 2);
      if (n_slots > (1ull << 31)) return CV_EINVAL;
      const uint32_t mask = (uint32_t)(n_slots - 1);
      const uint8_t* arena;  // the master units, back to back in file order (device memory)
      uint4* dig;
      uint8_t* trivial;
      uint32_t *owner, *cnt, *slot_of, *keys2, *vals, *vals2, *counters;
      uint64_t* file_base_d;
      CV_TRY(tmp.alloc(&dig, M * sizeof(uint4)));
      CV_TRY(tmp.alloc(&trivial, M));
      CV_TRY(tmp.alloc(&owner, n_slots * 4));
      CV_TRY(tmp.alloc(&cnt, n_slots * 4));
      CV_TRY(tmp.alloc(&slot_of, M * 4));
      CV_TRY(tmp.alloc(&keys2, M * 4));
      CV_TRY(tmp.alloc(&vals, M * 4));
      CV_TRY(tmp.alloc(&vals2, M * 4));
      CV_TRY(tmp.alloc(&counters, 16));  // max_disp, n_kept, n_unique, status
      CV_TRY(tmp.alloc(&file_base_d, (n_files + 1) * 8));
      uint8_t* tau = nullptr;  // per master sector cluster position (position-keyed tables)
      if (by_tau) CV_TRY(tmp.alloc(&tau, std::max<uint64_t>(M, 1)));
      CV_CUDA(cudaMemsetAsync(owner, 0, n_slots * 4, stream));
      CV_CUDA(cudaMemsetAsync(cnt, 0, n_slots * 4, stream));
      CV_CUDA(cudaMemsetAsync(counters, 0, 16, stream));
      CV_CUDA(cudaMemcpyAsync(file_base_d, file_base.data(), (n_files + 1) * 8, cudaMemcpyHostToDevice, stream));
      CV_TRY(gather_master_units(ctx, files, n_files, file_base, U, tmp, stream, &arena));
      // long-lived table memory
      CV_CUDA(cudaMalloc(&m->slots, n_slots * 32));
      CV_CUDA(cudaMalloc(&m->postings, std::max<uint64_t>(M, 1) * 8));
      CV_CUDA(cudaMemsetAsync(m->slots, 0, n_slots * 32, stream));
      // Bloom blocks: 32 bytes for sector tables, one 32-bit word for fragment tables
      const uint64_t block_bytes = frag ? 4 : 32;
      uint64_t n_blocks = 0;
      if (bpk) {
        n_blocks = std::max<uint64_t>(next_pow2((M * bpk + block_bytes * 8 - 1) / (block_bytes * 8)), frag ? 8 : 1);
        CV_CUDA(cudaMalloc(&m->bloom, n_blocks * block_bytes));
        CV_CUDA(cudaMemsetAsync(m->bloom, 0, n_blocks * block_bytes, stream));
      }
      if (frag) {
        // the shared-memory prefilter of a fragment table exists even when the table is empty
        // (all zero then: no window passes it)
        CV_CUDA(cudaMalloc(&m->frag_l1, kFragL1Bytes));
        CV_CUDA(cudaMemsetAsync(m->frag_l1, 0, kFragL1Bytes, stream));
      }
      if (M) {
        if (frag) {
          CV_CUDA((cudaError_t)frag_digests(sig, arena, M, dig, trivial, ctx->sms, stream));
        } else {
          Job job;
          CV_TRY(job.add(ctx, cfg, arena, M, 0, 0, false));
          CV_TRY(digest_job(ctx, cfg_i, sig, job, dig, trivial, counters + 3, stream, tmp));
        }
        const unsigned g = grid_for(M, 256, ctx->sms);
        if (tau) {
          tau_kernel<<<g, 256, 0, stream>>>(file_base_d, n_files, M, tau);
          CV_CUDA(cudaGetLastError());
        }
        insert_kernel<<<g, 256, 0, stream>>>(dig, trivial, tau, M, owner, cnt, slot_of, mask, counters, counters + 1,
                                            counters + 3);
        CV_CUDA(cudaGetLastError());
        iota_kernel<<<g, 256, 0, stream>>>(vals, M);
        CV_CUDA(cudaGetLastError());
        // stable LSD radix sort of (slot_of, m) by slot_of; keys <= n_slots
        int bits = 1;
        while ((1ull << bits) <= n_slots) bits++;
        uint32_t *kin, *vin;
        CV_TRY(radix_sort_pairs(slot_of, vals, keys2, vals2, M, bits, tmp, stream, &kin, &vin));
        fill_kernel<<<g, 256, 0, stream>>>(kin, vin, M, (uint32_t)n_slots, owner, cnt, dig, tau, file_base_d,
                                          n_files, (uint4*)m->slots, (uint2*)m->postings, counters + 2);
        CV_CUDA(cudaGetLastError());
        if (sig_is_weak(sig)) {
          // a copy of the kept master units in posting order, to confirm matches byte for byte
          CV_CUDA(cudaMalloc(&m->confirm, M * U));
          gather_units_kernel<<<grid_for(M * (U / 16), 256, ctx->sms), 256, 0, stream>>>(
              (const uint4*)arena, kin, vin, M, (uint32_t)n_slots, (uint32_t)(U / 16), (uint4*)m->confirm);
          CV_CUDA(cudaGetLastError());
        }
        if (frag) {
          CV_CUDA((cudaError_t)frag_bloom((const uint4*)m->slots, (uint32_t)n_slots, (uint32_t*)m->bloom,
                                          bpk ? (uint32_t)(n_blocks - 1) : 0u, (uint32_t*)m->frag_l1, ctx->sms,
                                          stream));
        } else if (bpk) {
          bloom_kernel<<<grid_for(n_slots, 256, ctx->sms), 256, 0, stream>>>((const uint4*)m->slots,
                                                                             (uint32_t)n_slots, (uint32_t*)m->bloom,
                                                                             (uint32_t)(n_blocks - 1));
          CV_CUDA(cudaGetLastError());
        }
      }
      uint32_t hc[4];
      CV_CUDA(cudaMemcpyAsync(hc, counters, 16, cudaMemcpyDeviceToHost, stream));
      CV_CUDA(cudaStreamSynchronize(stream));
      if (hc[3] & kStTableFull) return CV_ETABLEFULL;
      if (hc[3] & kStTimeout) return CV_ETIMEOUT;
      if (hc[3]) return CV_ECORRUPT;
      if (layout == CV_LAYOUT_AUTO)  // thresholds from the occupancy sweep (Bloom on / off)
        layout = (double)hc[2] > (bpk ? 0.8 : 0.5) * (double)n_slots ? CV_LAYOUT_SORTED : CV_LAYOUT_HASH;
      uint32_t steps = 0;  // binary-search steps of the sorted layout
      if (layout == CV_LAYOUT_SORTED) {
        void* sorted_slots = nullptr;
        CV_TRY(sorted_from_hash(ctx, (const uint4*)m->slots, n_slots, hc[2], tmp, stream, &sorted_slots, &m->keys0,
                                &steps));
        cudaFree(m->slots);
        m->slots = sorted_slots;
      }
      m->tab.slots = (const uint4*)m->slots;
      m->tab.keys0 = (const uint32_t*)m->keys0;
      m->tab.layout = layout;
      m->tab.n_keys = hc[2];
      m->tab.postings = (const uint2*)m->postings;
      m->tab.bloom = (const uint4*)m->bloom;
      m->tab.slot_mask = mask;
      m->tab.bloom_mask = bpk ? (uint32_t)(n_blocks - 1) : 0u;
      m->tab.max_probe = hc[0] + 1;
      m->tab.use_bloom = bpk ? 1u : 0u;
      m->tab.sig = (uint32_t)sig;
      m->tab.confirm = (const uint8_t*)m->confirm;
      m->tab.tau_mask = by_tau ? 7u : 0u;
      m->tab.unit = unit;
      m->tab.frag_l1 = (const uint32_t*)m->frag_l1;
      m->info.unit = unit;
      m->tab.tau_add = 0u;
      m->info.signature = (uint32_t)sig;
      m->info.position_mode = position_mode;
      m->info.n_files = n_files;
      m->info.n_sectors = M;
      m->info.n_kept = hc[1];
      m->info.n_unique = hc[2];
      m->info.n_slots = n_slots;
      m->info.bloom_bytes = n_blocks * block_bytes;
      m->info.max_probe = layout == CV_LAYOUT_SORTED ? steps : hc[0] + 1;
      m->info.layout = layout;
      const uint64_t table_bytes =
          layout == CV_LAYOUT_SORTED ? std::max<uint64_t>(hc[2], 1) * 36 : n_slots * 32;
      if (layout == CV_LAYOUT_SORTED) m->info.n_slots = hc[2];
      m->info.device_bytes = table_bytes + std::max<uint64_t>(M, 1) * 8 + n_blocks * block_bytes +
                             (m->confirm ? M * U : 0) + (m->frag_l1 ? kFragL1Bytes : 0);
      return CV_OK;
    };
    rc = body();
  }
  if (rc == CV_OK) {
    cudaError_t e = cudaStreamSynchronize(stream);  // temporaries returned
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (rc != CV_OK) {
    cv_free(m);
    return rc;
  }
  *out = m;
  return CV_OK;
}

}  // extern "C"

namespace cvk {
int master_view(const cv_master* m, TableView* tab, int* dev) {
  if (!m || m->magic != kMagicMaster) return CV_EINVAL;
  *tab = m->tab;
  *dev = m->dev;
  return CV_OK;
}
}  // namespace cvk

namespace {

// The table file: this header, then the arrays in header order (byte counts in the header).
struct TableFileHeader {
  char magic[8];              // "CVTABLE" + '\0'
  uint32_t version;           // 1
  uint32_t header_bytes;      // sizeof(TableFileHeader)
  cv_master_info info;
  uint32_t slot_mask, bloom_mask, max_probe, use_bloom, sig, tau_mask, layout, n_keys, unit, reserved;
  uint64_t bytes_slots, bytes_postings, bytes_bloom, bytes_confirm, bytes_keys0, bytes_l1;
};
constexpr char kTableMagic[8] = {'C', 'V', 'T', 'A', 'B', 'L', 'E', 0};
constexpr uint32_t kTableVersion = 1;

uint64_t table_unit_bytes(uint32_t unit) { return unit == kUnitFragment ? kFrag : kSector; }

// Device <-> file in bounded pieces through one host buffer.
int copy_to_file(FILE* f, const void* dev, uint64_t n) {
  std::vector<uint8_t> buf(std::min<uint64_t>(n, 64ull << 20));
  for (uint64_t off = 0; off < n; off += buf.size()) {
    const uint64_t k = std::min<uint64_t>(buf.size(), n - off);
    CV_CUDA(cudaMemcpy(buf.data(), (const uint8_t*)dev + off, k, cudaMemcpyDeviceToHost));
    if (fwrite(buf.data(), 1, k, f) != k) return CV_EIO;
  }
  return CV_OK;
}

int copy_from_file(FILE* f, void* dev, uint64_t n) {
  std::vector<uint8_t> buf(std::min<uint64_t>(n, 64ull << 20));
  for (uint64_t off = 0; off < n; off += buf.size()) {
    const uint64_t k = std::min<uint64_t>(buf.size(), n - off);
    if (fread(buf.data(), 1, k, f) != k) return CV_EIO;
    CV_CUDA(cudaMemcpy((uint8_t*)dev + off, buf.data(), k, cudaMemcpyHostToDevice));
  }
  return CV_OK;
}

}  // namespace

extern "C" {

int cv_master_get_info(const cv_master* m, cv_master_info* info) {
  if (!m || !info || m->magic != kMagicMaster) return CV_EINVAL;
  *info = m->info;
  return CV_OK;
}

int cv_master_save(const cv_master* m, const char* path) {
  NvtxRange nvtx_range("cv.master_save");
  if (!m || m->magic != kMagicMaster || !path) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  if (ctx->dev != m->dev) return CV_EINVAL;
  const cv_master_info& in = m->info;
  const uint64_t unit = table_unit_bytes(in.unit);
  TableFileHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kTableMagic, 8);
  h.version = kTableVersion;
  h.header_bytes = sizeof h;
  h.info = in;
  h.slot_mask = m->tab.slot_mask;
  h.bloom_mask = m->tab.bloom_mask;
  h.max_probe = m->tab.max_probe;
  h.use_bloom = m->tab.use_bloom;
  h.sig = m->tab.sig;
  h.tau_mask = m->tab.tau_mask;
  h.layout = m->tab.layout;
  h.n_keys = m->tab.n_keys;
  h.unit = m->tab.unit;
  h.bytes_slots = (m->tab.layout == kLayoutSorted ? (uint64_t)m->tab.n_keys : in.n_slots) * 32;
  h.bytes_postings = in.n_kept * 8;
  h.bytes_bloom = m->bloom ? in.bloom_bytes : 0;
  h.bytes_confirm = m->confirm ? in.n_kept * unit : 0;
  h.bytes_keys0 = m->keys0 ? (uint64_t)m->tab.n_keys * 4 : 0;
  h.bytes_l1 = m->frag_l1 ? kFragL1Bytes : 0;
  CV_CUDA(cudaDeviceSynchronize());
  FILE* f = fopen(path, "wb");
  if (!f) return CV_EIO;
  int rc = fwrite(&h, sizeof h, 1, f) == 1 ? CV_OK : CV_EIO;
  const void* arrays[6] = {m->slots, m->postings, m->bloom, m->confirm, m->keys0, m->frag_l1};
  const uint64_t sizes[6] = {h.bytes_slots, h.bytes_postings, h.bytes_bloom, h.bytes_confirm, h.bytes_keys0,
                             h.bytes_l1};
  for (int k = 0; k < 6 && rc == CV_OK; k++)
    if (sizes[k]) rc = copy_to_file(f, arrays[k], sizes[k]);
  if (fclose(f) != 0 && rc == CV_OK) rc = CV_EIO;
  return rc;
}

int cv_master_load(const char* path, void* stream_, cv_master** out) {
  NvtxRange nvtx_range("cv.master_load");
  if (!path || !out) return CV_EINVAL;
  *out = nullptr;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  cudaStream_t stream = (cudaStream_t)stream_;
  FILE* f = fopen(path, "rb");
  if (!f) return CV_EIO;
  TableFileHeader h;
  if (fread(&h, sizeof h, 1, f) != 1) {
    fclose(f);
    return CV_EIO;
  }
  // the parameters must describe a table this library could have built
  const cv_master_info& in = h.info;
  const uint64_t unit = table_unit_bytes(h.unit);
  const uint64_t n_records = h.layout == kLayoutSorted ? (uint64_t)h.n_keys : in.n_slots;
  const uint64_t bloom_block = h.unit == kUnitFragment ? 4 : 32;
  const bool ok = memcmp(h.magic, kTableMagic, 8) == 0 && h.version == kTableVersion &&
                  h.header_bytes == sizeof h && h.unit <= kUnitFragment && h.layout <= kLayoutSorted &&
                  h.sig <= (uint32_t)kSigCrc64 && in.unit == h.unit && in.layout == h.layout &&
                  in.signature == h.sig && (h.tau_mask == 0u || h.tau_mask == 7u) && in.n_kept <= in.n_sectors &&
                  in.n_sectors < (1ull << 27) && in.n_unique <= in.n_kept && in.n_slots >= 1 &&
                  in.n_slots <= (1ull << 31) &&
                  (h.layout == kLayoutSorted ? h.n_keys == in.n_unique && in.n_slots == in.n_unique
                                             : ((uint64_t)h.slot_mask + 1 == in.n_slots &&
                                                (in.n_slots & (in.n_slots - 1)) == 0 && h.max_probe <= in.n_slots)) &&
                  h.bytes_slots == n_records * 32 && h.bytes_postings == in.n_kept * 8 &&
                  h.bytes_confirm == (sig_is_weak((int)h.sig) ? in.n_kept * unit : 0) &&
                  h.bytes_keys0 == (h.layout == kLayoutSorted ? (uint64_t)h.n_keys * 4 : 0) &&
                  h.bytes_l1 == (h.unit == kUnitFragment ? kFragL1Bytes : 0) &&
                  h.use_bloom == (h.bytes_bloom ? 1u : 0u) && h.bytes_bloom == in.bloom_bytes &&
                  (!h.use_bloom || ((uint64_t)h.bloom_mask + 1) * bloom_block == h.bytes_bloom) &&
                  (h.bloom_mask & ((uint64_t)h.bloom_mask + 1)) == 0;
  if (!ok) {
    fclose(f);
    return CV_ECORRUPT;
  }
  cv_master* m = (cv_master*)calloc(1, sizeof(cv_master));
  if (!m) {
    fclose(f);
    return CV_ENOMEM;
  }
  m->magic = kMagicMaster;
  m->dev = ctx->dev;
  auto body = [&]() -> int {
    void** arrays[6] = {&m->slots, &m->postings, &m->bloom, &m->confirm, &m->keys0, &m->frag_l1};
    const uint64_t sizes[6] = {h.bytes_slots, h.bytes_postings, h.bytes_bloom, h.bytes_confirm, h.bytes_keys0,
                               h.bytes_l1};
    const bool always[6] = {true, true, false, false, false, false};  // the build allocates these even when empty
    for (int k = 0; k < 6; k++) {
      if (!sizes[k] && !always[k]) continue;
      CV_CUDA(cudaMalloc(arrays[k], std::max<uint64_t>(sizes[k], 32)));
      if (sizes[k]) CV_TRY(copy_from_file(f, *arrays[k], sizes[k]));
    }
    uint8_t extra;
    if (fread(&extra, 1, 1, f) != 0) return CV_ECORRUPT;  // trailing bytes: not this table's file
    uint32_t* status;
    CV_CUDA(cudaMallocAsync((void**)&status, 4, stream));
    CV_CUDA(cudaMemsetAsync(status, 0, 4, stream));
    validate_slots_kernel<<<grid_for(std::max<uint64_t>(n_records, 1), 256, ctx->sms), 256, 0, stream>>>(
        (const uint4*)m->slots, n_records, in.n_kept, status);
    CV_CUDA(cudaGetLastError());
    uint32_t st = 0;
    CV_CUDA(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, stream));
    CV_CUDA(cudaFreeAsync(status, stream));
    CV_CUDA(cudaStreamSynchronize(stream));
    if (st) return CV_ECORRUPT;
    m->tab.slots = (const uint4*)m->slots;
    m->tab.postings = (const uint2*)m->postings;
    m->tab.bloom = (const uint4*)m->bloom;
    m->tab.confirm = (const uint8_t*)m->confirm;
    m->tab.keys0 = (const uint32_t*)m->keys0;
    m->tab.frag_l1 = (const uint32_t*)m->frag_l1;
    m->tab.slot_mask = h.slot_mask;
    m->tab.bloom_mask = h.bloom_mask;
    m->tab.max_probe = h.max_probe;
    m->tab.use_bloom = h.use_bloom;
    m->tab.sig = h.sig;
    m->tab.tau_mask = h.tau_mask;
    m->tab.tau_add = 0;
    m->tab.layout = h.layout;
    m->tab.n_keys = h.n_keys;
    m->tab.unit = h.unit;
    m->info = in;
    return CV_OK;
  };
  const int rc = body();
  fclose(f);
  if (rc != CV_OK) {
    cv_free(m);
    return rc;
  }
  *out = m;
  return CV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- variants of a built table
// (the batch autotuner scans with whichever layout and Bloom use it measures fastest)

int cvk::table_sorted_copy(const TableView& tab, cudaStream_t stream, TableView* out, void** slots_out,
                           void** keys0_out) {
  if (tab.layout != kLayoutHash || tab.unit != kUnitSector) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  const uint64_t n_slots = (uint64_t)tab.slot_mask + 1;
  // the occupied slots: n_keys is kept for the hash layout too (distinct keys)
  const uint32_t nu = tab.n_keys;
  uint32_t steps = 0;
  int rc;
  {
    Temps tmp(ctx, stream);
    rc = sorted_from_hash(ctx, tab.slots, n_slots, nu, tmp, stream, slots_out, keys0_out, &steps);
  }
  if (rc != CV_OK) return rc;
  CV_CUDA(cudaStreamSynchronize(stream));  // temporaries returned
  *out = tab;
  out->slots = (const uint4*)*slots_out;
  out->keys0 = (const uint32_t*)*keys0_out;
  out->layout = kLayoutSorted;
  out->n_keys = nu;
  return CV_OK;
}

int cvk::table_bloom(const TableView& tab, uint32_t bits_per_key, cudaStream_t stream, TableView* out,
                     void** bloom_out) {
  if (tab.unit != kUnitSector || bits_per_key == 0 || bits_per_key > 64) return CV_EINVAL;
  DevCtx* ctx;
  CV_TRY(get_ctx(&ctx));
  const uint64_t n_records = tab.layout == kLayoutSorted ? (uint64_t)tab.n_keys : (uint64_t)tab.slot_mask + 1;
  const uint64_t keys = std::max<uint64_t>(tab.n_keys, 1);
  const uint64_t n_blocks = next_pow2((keys * bits_per_key + 255) / 256);
  void* bloom = nullptr;
  CV_CUDA(cudaMalloc(&bloom, n_blocks * 32));
  cudaError_t e = cudaMemsetAsync(bloom, 0, n_blocks * 32, stream);
  if (e == cudaSuccess && n_records) {
    bloom_kernel<<<grid_for(n_records, 256, ctx->sms), 256, 0, stream>>>(tab.slots, (uint32_t)n_records,
                                                                         (uint32_t*)bloom, (uint32_t)(n_blocks - 1));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaFree(bloom);
    return cuda_fail(e);
  }
  *bloom_out = bloom;
  *out = tab;
  out->bloom = (const uint4*)bloom;
  out->bloom_mask = (uint32_t)(n_blocks - 1);
  out->use_bloom = 1u;
  return CV_OK;
}
