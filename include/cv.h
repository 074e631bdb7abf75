/*
 * cv.h -- C ABI of the GB300 sector-signature carving library (libcv.so).
 *
 * The operation (paper Section 1 and Section 3.1): the sectors of known master files are hashed
 * into a signature table on the GPU; every 512-byte sector of a disk image is hashed on the GPU
 * and looked up in that table; every (disk sector, master file, master sector) whose signatures
 * are equal is reported. The signature is MD5 (RFC 1321; paper Section 2.1) over the 512-byte
 * sector with standard padding, 9 compressions per sector. The table is open addressing with
 * linear probing on the digest's low word (paper Eq. 3), optionally fronted by a blocked Bloom
 * filter. Results are sorted by (disk_sector, file_id, file_sector).
 *
 * Rules that both the library and its tests follow:
 *   - Only whole sectors count. A master file's trailing partial sector and an image's trailing
 *     partial sector are ignored.
 *   - A master sector whose 512 bytes are all equal (all zero or one repeated byte) is excluded.
 *   - Every master sector with the matched digest is reported (duplicates within or across
 *     master files all appear).
 *
 * Conventions:
 *   - Every call returns CV_OK (0) or a negative CV_E* code; nothing aborts or throws.
 *   - Buffers (cv_buf.data) may be host memory (pageable or pinned) or device memory of the
 *     current device; the kind is detected per buffer. Device buffers must be 16-byte aligned.
 *     Inputs are borrowed for the duration of the call only.
 *   - Handles (cv_master, cv_result) and the result arrays they own belong to the library until
 *     cv_free. Handles are not thread-safe; distinct handles may be used from distinct threads.
 *   - All device work runs on the stream given in the options (a cudaStream_t; NULL means the
 *     legacy default stream). The calls return after that work has finished.
 *   - Indices are 0-based: file_id indexes the files[] array given to cv_master_build;
 *     file_sector and disk_sector count 512-byte sectors from the start of their buffer.
 */
#ifndef CV_H
#define CV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CV_SECTOR_BYTES 512u

/* Return codes. */
#define CV_OK 0
#define CV_EINVAL -1     /* bad argument: NULL pointer, misaligned device buffer, size limit */
#define CV_ENOMEM -2     /* device or host allocation failed */
#define CV_ECUDA -3      /* a CUDA call failed (see cv_last_cuda_error) */
#define CV_ETABLEFULL -4 /* the signature table could not take every master sector */
#define CV_ECORRUPT -5   /* a device-side consistency check failed (status word set) */
#define CV_ETIMEOUT -6   /* a device-side wait ran out of time; the results were discarded */
#define CV_ENODEV -7     /* no usable CUDA device (the library has no CPU path) */
#define CV_ERANGE -8     /* image_index out of range, or an output buffer too small */
#define CV_EAGAIN -9     /* not ready yet (cv_poll) */
#define CV_EIO -10       /* a file could not be opened, read or written */

/* One match: disk sector i of image k equals sector file_sector of master file file_id. */
typedef struct {
  uint64_t disk_sector;
  uint32_t file_id;
  uint32_t file_sector;
} cv_match; /* 16 bytes */

/* A borrowed byte buffer in host or device memory. */
typedef struct {
  const void* data;
  uint64_t n_bytes;
} cv_buf;

typedef struct cv_master cv_master; /* signature table of a master set, resident on the GPU */
typedef struct cv_result cv_result; /* the results of one scan */

#define CV_BLOOM_AUTO 0xFFFFFFFFu

/* Sector signatures (cv_master_opts.signature). The paper proposes MD5 (Section 2.1) and
 * measures djb2 with a 64-bit accumulator (Eq. 1) and CRC64 (Section 4). 64-bit signatures
 * collide (Section 4.1), so the library confirms every candidate byte for byte against a copy of
 * the master sectors it keeps on the device (Section 3.1); results are identical for all four. */
#define CV_SIG_MD5 0u        /* RFC 1321 with the padding block: 9 compressions per sector */
#define CV_SIG_MD5_NOPAD 1u  /* the MD5 state after the 8 data blocks (Section 2.1) */
#define CV_SIG_DJB2_64 2u    /* h = 5381; h = 33 h + byte, mod 2^64 (Eq. 1) */
#define CV_SIG_CRC64 3u      /* remainder of M(x) x^64 mod x^64+x^4+x^3+x+1, MSB first, no init/final XOR */

/* Table organisation (cv_master_opts.position_mode). Section 3.1 keeps one table S_tau per
 * sector position tau (0..7) of an 8-sector cluster, so a disk sector only matches master
 * sectors at its own position. CV_POSITION_CLUSTER builds that: a triple (i, f, s) is reported
 * only when (i - base_offset) mod 8 == s mod 8, base_offset being cv_scan_opts.base_offset (the
 * first sector of the partition whose clusters are meant; the paper counts from sector 0).
 * CV_POSITION_ANY (the default) matches every position: one table over all sectors. */
#define CV_POSITION_ANY 0u
#define CV_POSITION_CLUSTER 1u

/* Table layout (cv_master_opts.layout); results do not depend on it.
 * CV_LAYOUT_HASH: open addressing with linear probing from the slot given by the signature's
 *   low bits (Section 3.1, Eq. 3); slots = next power of two above n_kept / max_load.
 * CV_LAYOUT_SORTED: the distinct keys in one array sorted by their first word, searched by
 *   binary search (Section 4 proposes it for high occupancy, after Dandass): every slot is
 *   used, and a lookup costs ceil(log2 n_unique) dependent reads whatever the occupancy. */
#define CV_LAYOUT_HASH 0u
#define CV_LAYOUT_SORTED 1u
/* CV_LAYOUT_AUTO: the hash layout, turned into the sorted one when the built table's occupancy
 * (distinct keys / slots) exceeds 0.8 with a Bloom filter or 0.5 without one, where linear
 * probing measured slower than bisection on GB300. cv_master_info.layout reports the choice. */
#define CV_LAYOUT_AUTO 2u

/* What the master files are cut into (cv_master_opts.unit).
 * CV_UNIT_SECTOR: whole 512-byte sectors; disk images are scanned sector by sector.
 * CV_UNIT_FRAGMENT: whole 64-byte fragments (fragment j of a file is its bytes [64j, 64j+64),
 *   fragments whose 64 bytes are all equal excluded); a scan looks up every 64-byte window of
 *   the image that starts at a multiple of 4 bytes (Section 5: small images and logos embedded
 *   in other files at any 32-bit offset). A match (k, f, j) means image bytes [4k, 4k+64) equal
 *   fragment j of file f: cv_match.disk_sector holds the window index k and cv_match.file_sector
 *   the fragment index j. Signatures: MD5, MD5 without padding (one compression per window) and
 *   djb2-64 (rolled from window to window; every candidate confirmed byte for byte); CRC64 and
 *   CV_POSITION_CLUSTER are refused with CV_EINVAL. The Bloom filter is one 32-bit word per
 *   lookup (3 bits per key). Batched, served and allocation-free scans take sector tables only. */
#define CV_UNIT_SECTOR 0u
#define CV_UNIT_FRAGMENT 1u

typedef struct {
  uint32_t struct_size;         /* sizeof(cv_master_opts); 24 bytes (before position_mode) and
                                   32 bytes (before unit) are accepted: the missing fields take
                                   CV_POSITION_ANY, CV_LAYOUT_HASH and CV_UNIT_SECTOR */
  float max_load;               /* table load factor cap in (0, 0.9]; 0 selects 0.5 */
  uint32_t bloom_bits_per_key;  /* 0 = no Bloom prefilter; CV_BLOOM_AUTO = 16 */
  uint32_t signature;           /* CV_SIG_*; 0 = MD5 */
  void* stream;                 /* cudaStream_t */
  uint32_t position_mode;       /* CV_POSITION_* */
  uint32_t layout;              /* CV_LAYOUT_*; read only together with position_mode */
  uint32_t unit;                /* CV_UNIT_*; read when struct_size covers it (else sectors) */
  uint32_t reserved;            /* 0 */
} cv_master_opts;

/* cv_scan_opts.flags */
#define CV_KEEP_ON_DEVICE 1u /* cv_matches returns device pointers (no device-to-host copy) */

typedef struct {
  uint32_t struct_size;       /* sizeof(cv_scan_opts) */
  uint32_t flags;             /* CV_KEEP_ON_DEVICE */
  void* stream;               /* cudaStream_t */
  uint64_t chunk_bytes;       /* host images are streamed in chunks of this size; 0 = 256 MiB */
  uint32_t kernel_config;     /* 0 = the default for the table's signature (MD5 and MD5 without
                                 padding: configuration 0; djb2-64 and CRC64, whose scans are
                                 bound by the staging of the image: 128-byte stages of
                                 128-sector tiles), or the CV_SCAN_CONFIG environment variable's
                                 configuration (by name) when set; k + 1 selects configuration k */
  uint32_t reserved;
  uint64_t base_offset;       /* position-keyed tables: disk sector of the first cluster (only its
                                 value mod 8 matters); ignored for CV_POSITION_ANY tables. The
                                 size without it (32 bytes) is accepted and means 0. */
} cv_scan_opts;

/* Kernel configurations of the scan (tile rows, sectors per thread, ring stages, staging width,
 * pipe split of the MD5 additions); each is built for every signature and table layout. Every
 * configuration gives the same results; they differ in speed. */
int cv_kernel_config_count(void);
const char* cv_kernel_config_name(int k); /* NULL when k is out of range */

/*
 * Build the signature table of n_files master files (paper Section 3.1: the table S is built
 * by hashing every master sector and inserting its signature; collisions by linear probing,
 * Eq. 3). files[f] is file f. Total whole, non-excluded master sectors must be below 2^27.
 * On success *out receives a handle owning the device table. Errors: CV_EINVAL, CV_ENOMEM,
 * CV_ECUDA, CV_ETABLEFULL, CV_ENODEV.
 */
int cv_master_build(const cv_buf* files, uint32_t n_files, const cv_master_opts* opts, cv_master** out);

typedef struct {
  uint32_t n_files;
  uint32_t position_mode;    /* CV_POSITION_* of the table */
  uint64_t n_sectors;        /* whole master sectors */
  uint64_t n_kept;           /* after the exclusion rule */
  uint64_t n_unique;         /* distinct keys among the kept sectors: digests, or (digest, tau)
                                pairs for position-keyed tables */
  uint64_t n_slots;          /* table slots (hash layout: a power of two; sorted: n_unique) */
  uint64_t bloom_bytes;      /* 0 when there is no Bloom prefilter */
  uint32_t max_probe;        /* hash layout: longest linear-probe run of any stored digest,
                                plus one; sorted layout: binary-search steps, ceil(log2 n_unique) */
  uint32_t signature;        /* CV_SIG_* of the table */
  uint64_t device_bytes;     /* device memory the handle holds */
  uint32_t layout;           /* CV_LAYOUT_* of the table */
  uint32_t unit;             /* CV_UNIT_* of the table (n_sectors, n_kept: units of that size) */
} cv_master_info;

int cv_master_get_info(const cv_master* m, cv_master_info* info);

/*
 * Save a built table to a file and load it back, so that a master set is hashed once and
 * reused across runs (the paper has no counterpart: it rebuilds its tables per run). The file
 * holds the table's device arrays and parameters, little-endian, with a magic tag and a format
 * version; it is valid on any GPU this library runs on. cv_master_load checks the sizes against
 * the parameters and every slot's posting range on the device before accepting the table, so a
 * damaged file yields CV_ECORRUPT rather than out-of-range reads. stream: cudaStream_t or NULL.
 * Errors: CV_EINVAL, CV_EIO, CV_ENOMEM, CV_ECUDA, CV_ECORRUPT, CV_ENODEV.
 */
int cv_master_save(const cv_master* m, const char* path);
int cv_master_load(const char* path, void* stream, cv_master** out);

/*
 * Scan n_images disk images against the table (paper Section 3.1-3.2: every sector hashed,
 * its signature looked up, matches reported to the host). Device images are scanned in one
 * launch; host images are streamed through device buffers in chunks, copies overlapping the
 * hashing. On success *out receives a handle owning the sorted results of every image.
 * With a fragment table (CV_UNIT_FRAGMENT) every 64-byte window at a 4-byte offset is looked up
 * instead; host images are then copied whole to the device, and chunk_bytes, kernel_config and
 * base_offset are ignored.
 * Errors: CV_EINVAL, CV_ENOMEM, CV_ECUDA, CV_ETIMEOUT, CV_ECORRUPT, CV_ENODEV.
 */
int cv_scan(const cv_master* m, const cv_buf* images, uint32_t n_images, const cv_scan_opts* opts,
            cv_result** out);

/*
 * The sorted matches of image image_index: *out points at *n_out entries owned by the result
 * handle (host memory, or device memory when the scan used CV_KEEP_ON_DEVICE), valid until
 * cv_free(result). Errors: CV_EINVAL, CV_ERANGE.
 */
int cv_matches(const cv_result* r, uint32_t image_index, const cv_match** out, uint64_t* n_out);

typedef struct {
  uint64_t sectors;        /* whole sectors scanned (fragment tables: windows scanned) */
  uint64_t matches;        /* triples over all images */
  uint64_t hit_sectors;    /* disk sectors with at least one match (0 for fragment tables) */
  float kernel_ms;         /* device time of the hashing/probe launches */
  float total_ms;          /* device time from the first copy to the last result copy */
  uint32_t kernel_launches; /* kernels the call launched (scan, offsets, expand) */
  int32_t kernel_config;   /* the scan configuration used (cv_kernel_config_name), -1 for
                              fragment scans and results of the serving loop */
  uint64_t confirm_rejected; /* 64-bit signatures: candidate (disk sector, master sector or
                                fragment) pairs whose signatures were equal but whose bytes
                                differed, dropped by the byte confirmation (Section 3.1); 0 for
                                MD5 tables and for batched, served and allocation-free scans */
} cv_scan_stats;

int cv_scan_get_stats(const cv_result* r, cv_scan_stats* st);

/*
 * Lookup cost, counted exactly: what the scan of an image reads from the table (the paper's
 * occupancy study, Section 4, Figures 10-12). The scan's own lookups are replayed outside the
 * scan kernel (which keeps no counters): the Bloom test when the table has a filter, then
 * the linear-probing walk from the home slot of Eq. 3 up to the table's probe bound (hash
 * layout), or the bisection over the sorted key words and the comparison of the records that
 * share the sector's key word (sorted layout).
 *   image        device pointer, 16-byte aligned; n_bytes / 512 whole sectors are looked up.
 *   base_offset  as cv_scan_opts.base_offset (position-keyed tables).
 *   st           st->struct_size = sizeof(cv_probe_stats); filled on success.
 * Sector tables only (a fragment table: CV_EINVAL). Runs on stream and returns after the work
 * has finished. Errors: CV_EINVAL, CV_ENOMEM, CV_ECUDA, CV_ETIMEOUT, CV_ENODEV.
 */
typedef struct {
  uint32_t struct_size;    /* sizeof(cv_probe_stats) */
  uint32_t layout;         /* the table's layout: CV_LAYOUT_HASH or CV_LAYOUT_SORTED */
  uint64_t sectors;        /* sectors looked up */
  uint64_t bloom_passed;   /* of them, those the Bloom filter let through (all, without one) */
  uint64_t slot_reads;     /* 32-byte table records read: the probe walks' slots (hash layout),
                              the records compared after the bisection (sorted layout) */
  uint64_t key_reads;      /* sorted layout: 4-byte key words read by the bisections and the
                              scans over equal key words; 0 for the hash layout */
  uint64_t found;          /* sectors whose key (signature, and position in S_tau tables) is in
                              the table; for 64-bit signatures before byte confirmation */
} cv_probe_stats;
int cv_probe_profile(const cv_master* m, const void* image, uint64_t n_bytes, uint64_t base_offset,
                     cv_probe_stats* st, void* stream);

/* Free a cv_master, cv_result, cv_batch or cv_server handle (NULL is ignored). A server first
 * finishes its admitted requests and stops its engine thread. */
void cv_free(void* handle);

/* Text for a return code. */
const char* cv_strerror(int code);

/* The last CUDA error code seen by the calling thread inside the library (0 if none). */
int cv_last_cuda_error(void);

/*
 * MD5 (RFC 1321, standard padding) of n_sectors consecutive 512-byte sectors, for testing and
 * for callers that want signatures only. in: device pointer, 16-byte aligned, n_sectors*512
 * bytes. digests: device pointer, 16 bytes per sector (the RFC's byte order). trivial: device
 * pointer to one byte per sector set to 1 when all 512 bytes are equal, or NULL. Runs on
 * stream and returns without waiting. Errors: CV_EINVAL, CV_ECUDA, CV_ENODEV.
 */
int cv_sector_digests(const void* in, uint64_t n_sectors, void* digests, uint8_t* trivial, void* stream);

/*
 * The sector signature of n_sectors consecutive 512-byte sectors under any CV_SIG_* (paper
 * Section 2.1 for MD5 and MD5 without padding, Eq. 1 for djb2-64, Section 2.1's generator for
 * CRC64), computed by the same kernel code that hashes sectors in a scan and in a table build.
 * It lets a caller (or a test) compare the library's signatures value by value with another
 * implementation: a wrong but deterministic 64-bit signature would leave every match list
 * unchanged, since equal bytes hash equally and byte confirmation drops every false candidate.
 *   in       device pointer, 16-byte aligned, n_sectors * 512 bytes.
 *   out      device pointer, 16-byte aligned, 16 bytes per sector:
 *              CV_SIG_MD5        the digest (RFC 1321 byte order);
 *              CV_SIG_MD5_NOPAD  the state A, B, C, D after the 8 data blocks, same byte order;
 *              CV_SIG_DJB2_64, CV_SIG_CRC64  bytes 0-7 the 64-bit signature (little-endian),
 *                                bytes 8-15 the library's mixing of it (a SplitMix64 finalizer;
 *                                the table's Bloom bits come from it).
 *   trivial  device pointer to one byte per sector set to 1 when all 512 bytes are equal, or NULL.
 * Runs on stream and returns without waiting. Errors: CV_EINVAL, CV_ECUDA, CV_ENODEV.
 */
int cv_sector_signatures(const void* in, uint64_t n_sectors, uint32_t signature, void* out, uint8_t* trivial,
                         void* stream);

/*
 * The signature of every 64-byte window at a 4-byte offset of a device image (paper Section 5),
 * computed by the fragment scan's own code: window k is bytes [4k, 4k + 64), for every k with
 * 4k + 64 <= n_bytes. signature: CV_SIG_MD5 (the 64-byte message with its padding block),
 * CV_SIG_MD5_NOPAD (the state after the one data block) or CV_SIG_DJB2_64 (rolled from window
 * to window as in the scan: bytes 0-7 the value, little-endian, bytes 8-15 the library's mixing
 * of it); CV_SIG_CRC64 is refused with CV_EINVAL, as for fragment tables.
 *   image  device pointer, 16-byte aligned; out: device pointer, 16-byte aligned, 16 bytes per
 *          window. Fewer than 64 bytes: nothing to do.
 * Runs on stream and returns without waiting. Errors: CV_EINVAL, CV_ECUDA, CV_ENODEV.
 */
int cv_window_signatures(const void* image, uint64_t n_bytes, uint32_t signature, void* out, void* stream);

/* Integer throughput of this GPU: independent lop3 chains (ALU pipe), mad.lo chains (FMA pipe)
 * and the two interleaved, in operations per second, with the SM clock seen during the run.
 * The paper has no counterpart; it is the denominator of the scan's roofline. */
typedef struct {
  double alu_ops_per_s;
  double fma_ops_per_s;
  double mixed_ops_per_s;
  double sm_clock_mhz;
  int sms;
  int reserved;
} cv_int_peak_info;
int cv_int_peak(cv_int_peak_info* info);

/* Failure-path self-test: a kernel waits on a barrier that nothing completes, using the same
 * bounded wait as the scan kernel, and the offset scan's look-back waits for a chunk that no
 * block publishes; each wait has a limit of timeout_us microseconds (1..10^7), gives up, sets
 * its device status word and lets its kernel return. Expected result: CV_ETIMEOUT (both waits
 * ran out), with the device still usable afterwards. The paper has no counterpart. */
int cv_selftest_wait_timeout(uint32_t timeout_us, void* stream);

/*
 * Batched scans (a CUDA graph over many device images). The paper scans several drives at once
 * by multiplexing them onto one GPU (Section 3); a batch makes all of its images one work list
 * for one persistent scan launch (images in one device allocation share a tensor map), then
 * one offset pass and one expand pass, captured once as a CUDA graph and replayed per run.
 *
 * Images must be device buffers (16-byte aligned), borrowed for the life of the batch: each run
 * reads their current contents. Matches of the last run stay in device memory owned by the
 * batch. With autotune set, cv_batch_create times on the batch itself every kernel
 * configuration x table layout x Bloom use, and keeps the fastest: the layouts are the master's
 * own and, for a CV_LAYOUT_HASH master, a sorted copy (CV_LAYOUT_SORTED, Section 4's binary
 * search); Bloom use is off, or on with the master's filter, or, for a master without one, with
 * a 16-bit-per-key filter the batch builds. A copy or filter the choice uses is owned by the
 * batch (its device memory is freed with it). The choice is cached per process and, when
 * tune_cache names a file, in that file (one line per workload key). cv_batch_get_info reports
 * the configuration, layout and Bloom use in effect. Section 3.2 notes that the best
 * concurrency has to be found again for every GPU generation.
 */
typedef struct cv_batch cv_batch;

#define CV_BATCH_BLOOM_AUTO 0u /* use the table's Bloom filter when it has one */
#define CV_BATCH_BLOOM_OFF 1u  /* probe the table directly */
#define CV_BATCH_BLOOM_ON 2u   /* the table's filter, or for a table without one a 16-bit-per-key
                                  filter the batch builds and owns */

typedef struct {
  uint32_t struct_size;     /* sizeof(cv_batch_opts) */
  uint32_t autotune;        /* 1: tune kernel configuration, table layout and Bloom use on this batch */
  void* stream;             /* cudaStream_t for set-up and tuning */
  uint64_t match_capacity;  /* output room in matches; 0 = size it from one scan at set-up */
  uint32_t kernel_config;   /* 0 = the signature's default (or tuned); k + 1 = configuration k */
  uint32_t bloom;           /* CV_BATCH_BLOOM_* (ignored when tuning) */
  const char* tune_cache;   /* file for tuned choices, or NULL */
  uint32_t sorted_copy;     /* 1: scan a sorted copy of a CV_LAYOUT_HASH master (the batch builds
                               and owns it; ignored when tuning). The size without this field and
                               the next (40 bytes on LP64) is accepted and means 0. */
  uint32_t reserved;        /* 0 */
} cv_batch_opts;

typedef struct {
  int kernel_config;          /* index of the configuration in use */
  const char* config_name;
  uint32_t bloom;             /* 1 when the Bloom prefilter is used */
  uint32_t tuned;             /* 1 when this batch ran the tuner (0: default or cached) */
  uint32_t kernel_launches;   /* kernel nodes per run */
  uint32_t tensor_maps;
  uint32_t segments;
  uint32_t layout;            /* CV_LAYOUT_HASH or CV_LAYOUT_SORTED: the table layout scanned */
  uint64_t sectors;
  uint64_t match_capacity;
  float scan_ms;              /* device time of the scan launch(es) of the last finished run */
} cv_batch_info;

/* With a position-keyed table (CV_POSITION_CLUSTER) every image's clusters are counted from its
 * sector 0 (base_offset 0).
 * Errors: CV_EINVAL (host or misaligned image, bad options), CV_ENOMEM, CV_ECUDA, CV_ENODEV. */
int cv_batch_create(const cv_master* m, const cv_buf* images, uint32_t n_images, const cv_batch_opts* opts,
                    cv_batch** out);
/* One graph launch on stream; returns without waiting. */
int cv_batch_run(cv_batch* b, void* stream);
/* Wait for the last run. *n_matches = matches over all images. CV_ERANGE when they exceed the
 * batch's capacity (create the batch again with a larger match_capacity). */
int cv_batch_wait(cv_batch* b, uint64_t* n_matches);
/* Device pointer and count of image image_index's sorted matches from the last run. */
int cv_batch_matches(const cv_batch* b, uint32_t image_index, const cv_match** out, uint64_t* n_out);
int cv_batch_get_info(const cv_batch* b, cv_batch_info* info);

/*
 * Serving: a request loop that scans images as they arrive (drives at a checkpoint, chunks of
 * a network stream) against one resident master table. Requests are cut into work units; the
 * units are copied host-to-device on side streams into a device arena whose size is the HBM
 * budget, and every engine iteration scans the units of all live requests that have arrived
 * on the device in one launch (continuous batching). Each request's matches are identical to
 * a solo cv_scan of the same image. One engine thread per server.
 */
typedef struct cv_server cv_server;

typedef struct {
  uint32_t struct_size;      /* sizeof(cv_server_opts) */
  uint32_t max_live;         /* requests admitted at once; 0 = 64 */
  uint64_t hbm_budget_bytes; /* device arena for request data in flight; 0 = 8 GiB */
  uint64_t work_unit_bytes;  /* request data per work unit (multiple of 512); 0 = 64 MiB */
  uint32_t kernel_config;    /* 0 = the signature's default; k + 1 = configuration k */
  uint32_t copy_streams;     /* host-to-device copy streams; 0 = 2 */
  uint64_t max_copy_bytes;   /* request data queued on the copy streams at once, at least one work
                                unit; more is issued as copies land, first to the live request with
                                the fewest bytes left, so a small request is not stuck behind a
                                large one's copies. 0 = 2 GiB, UINT64_MAX = no limit. The size
                                without this field (32 bytes) is accepted and means 0. */
} cv_server_opts;

typedef struct {
  uint64_t submitted;
  uint64_t completed;
  uint64_t failed;
  uint64_t bytes_scanned;
  uint64_t iterations;          /* engine iterations (scan launches over ready units) */
  uint64_t units;               /* work units scanned */
  uint64_t peak_bytes_in_flight;
  double mean_live_per_iteration; /* requests with units in an iteration, averaged */
  double p50_ms, p99_ms, mean_ms, max_ms; /* submit-to-result latency of completed requests */
  double wall_s;                /* first submit to last completion */
} cv_server_stats;

/* Errors: CV_EINVAL, CV_ENOMEM, CV_ECUDA, CV_ENODEV. The master must outlive the server. With a
 * position-keyed table every request's clusters are counted from its sector 0. */
int cv_server_create(const cv_master* m, const cv_server_opts* opts, cv_server** out);
/* Queue one image (host memory, or device memory of the server's device), borrowed until its
 * result is polled. Never blocks on the GPU. *ticket identifies the request. */
int cv_submit(cv_server* s, cv_buf image, uint64_t tag, uint64_t* ticket);
/* Wait up to timeout_ms (0: do not wait, < 0: forever) for a request. On success *out is its
 * result (one image, host matches; free with cv_free) and the ticket is retired. CV_EAGAIN:
 * not done yet. Other codes: the request failed. */
int cv_poll(cv_server* s, uint64_t ticket, int timeout_ms, cv_result** out);
int cv_server_get_stats(cv_server* s, cv_server_stats* st);

/*
 * Scan one device-resident image without allocating any memory. The paper has no counterpart:
 * this is for callers that cannot allocate while they work, such as a real-time ingest loop
 * handing over fixed buffers, or a process whose device memory is fully reserved by another
 * allocator at start-up, where cudaMalloc could block, fail or synchronize the device.
 *
 * Instead of a memory pool it uses one fixed scratch array built into the library (a little
 * over 8 MiB, resident on every GPU that loads the library until the process exits).
 *   image        device pointer, 16-byte aligned; n_bytes / 512 whole sectors are scanned, at
 *                most CV_NOALLOC_MAX_SECTORS (256 MiB of image), else CV_EINVAL.
 *   out          device pointer, 16-byte aligned, room for out_capacity cv_match entries; the
 *                sorted matches are written there.
 *   *n_out       (host) the number of matches. If it exceeds out_capacity, only out_capacity
 *                entries are written and CV_ERANGE is returned: call again with more room.
 * Runs on stream and returns after the work has finished. Every call shares the one scratch
 * array and finds the previous call's contents there; calls whose work could overlap on the
 * GPU must be serialized by the caller. The first call on a device performs a one-time set-up
 * (the array's device address, kernel attributes). No call can be captured into a CUDA graph
 * (each one waits for its stream): on a capturing stream the call returns CV_EINVAL before any
 * work. With a position-keyed table the image's clusters are counted from its sector 0. On any
 * error other than CV_ERANGE the contents of out are undefined.
 * Errors: CV_EINVAL, CV_ERANGE, CV_ECUDA, CV_ETIMEOUT, CV_ECORRUPT, CV_ENODEV.
 */
#define CV_NOALLOC_MAX_SECTORS (1u << 19)
int cv_scan_noalloc(const cv_master* m, const void* image, uint64_t n_bytes, cv_match* out, uint64_t out_capacity,
                    uint64_t* n_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CV_H */
