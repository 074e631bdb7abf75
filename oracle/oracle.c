/*
 * Sector-signature carving oracle: a plain, slow, obviously correct CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its Python
 * binding) links, loads or calls this file. Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg do. It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes (paper, Section 1 and Section 3.1, "alerts the host ... byte-for-byte
 * comparison"): given master files and a disk image, every triple (i, f, s) such that disk
 * sector i is byte-for-byte equal to sector s of master file f, sorted lexicographically.
 *
 *   - A sector is 512 bytes (Section 2). Only whole sectors count: a master file's partial
 *     tail and an image's trailing partial sector are ignored.
 *   - A master sector whose 512 bytes are all equal (all zero, or one byte repeated) is
 *     excluded from the master set. The paper has no such rule; the library applies the
 *     same one, so both sides agree on it.
 *
 * Two matchers:
 *   oracle_match_brute  - the definition itself: memcmp of every disk sector against every
 *                         kept master sector. Tiny inputs only. Parity pinned by construction.
 *   oracle_match_hash   - the method's route (Section 3.1): a signature per master sector,
 *                         the disk sector's signature looked up among them, equal signatures
 *                         reported. The signature is MD5 (Section 2.1, RFC 1321) over the
 *                         512-byte sector with standard padding (9 compressions). The lookup
 *                         is a sorted array + binary search (the paper's Section 4.2 names
 *                         binary search as an alternative to its hash tables); the table
 *                         layout does not change the result.
 *
 * Fragments (Section 5): oracle_frag_match_brute and oracle_frag_match give the same kind of
 * result for every 64-byte window at a 4-byte offset against the 64-byte fragments of the
 * master files (definition at the functions).
 *
 * Other signatures (Section 2): MD5 without the padding block (Section 2.1 notes it adds nothing
 * for fixed-size sectors), djb2 with a 64-bit accumulator (Eq. 1) and CRC64 with the generator
 * x^64 + x^4 + x^3 + x + 1 (Section 2.1). With a 64-bit signature, equal signatures are only
 * candidates: oracle_match_sig confirms each one byte for byte (Section 3.1), so every
 * signature yields the same result as oracle_match_brute.
 *
 * MD5 (oracle_md5) follows the prose of RFC 1321 Section 3: pad with one 1-bit then zeros to
 * 448 mod 512 bits, append the 64-bit little-endian bit length, then for every 512-bit block
 * run four rounds of sixteen operations a = b + ((a + F(b,c,d) + X[k] + T[i]) <<< s), where
 * T[i] is the integer part of 4294967296 * |sin(i)| (i in radians, i = 1..64), computed here
 * at first use in double precision. Parity is pinned by the test suite against two
 * independent MD5 implementations (Python's hashlib, backed by OpenSSL, and the md5sum tool).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SECTOR 512u

typedef struct {
  uint64_t disk_sector;
  uint32_t file_id;
  uint32_t file_sector;
} oracle_triple;

/* ---------------------------------------------------------------- MD5, RFC 1321 Section 3 */

static uint32_t T_sine[65]; /* 1-based, as in the RFC */
static int T_ready = 0;

static void md5_init_table(void) {
  if (T_ready) return;
  for (int i = 1; i <= 64; i++) T_sine[i] = (uint32_t)floor(4294967296.0 * fabs(sin((double)i)));
  T_ready = 1;
}

/* Per-round left-rotation amounts s (RFC 1321 Section 3.4, each round cycles four amounts). */
static const int rot_amount[4][4] = {{7, 12, 17, 22}, {5, 9, 14, 20}, {4, 11, 16, 23}, {6, 10, 15, 21}};

static uint32_t rotl32(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

static uint32_t aux_F(uint32_t x, uint32_t y, uint32_t z) { return (x & y) | (~x & z); }
static uint32_t aux_G(uint32_t x, uint32_t y, uint32_t z) { return (x & z) | (y & ~z); }
static uint32_t aux_H(uint32_t x, uint32_t y, uint32_t z) { return x ^ y ^ z; }
static uint32_t aux_I(uint32_t x, uint32_t y, uint32_t z) { return y ^ (x | ~z); }

/* Process one 64-byte block into the state ABCD (RFC 1321 Section 3.4). */
static void md5_block(uint32_t st[4], const uint8_t blk[64]) {
  uint32_t X[16];
  for (int j = 0; j < 16; j++)
    X[j] = (uint32_t)blk[4 * j] | ((uint32_t)blk[4 * j + 1] << 8) | ((uint32_t)blk[4 * j + 2] << 16) |
           ((uint32_t)blk[4 * j + 3] << 24);
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
  for (int i = 0; i < 64; i++) {
    int round = i / 16, j = i % 16;
    uint32_t f;
    int k;
    switch (round) {
      case 0: f = aux_F(b, c, d); k = j; break;                 /* X[0], X[1], ... X[15]   */
      case 1: f = aux_G(b, c, d); k = (1 + 5 * j) % 16; break;  /* X[1], X[6], X[11], ...  */
      case 2: f = aux_H(b, c, d); k = (5 + 3 * j) % 16; break;  /* X[5], X[8], X[11], ...  */
      default: f = aux_I(b, c, d); k = (7 * j) % 16; break;     /* X[0], X[7], X[14], ...  */
    }
    uint32_t t = b + rotl32(a + f + X[k] + T_sine[i + 1], rot_amount[round][j % 4]);
    /* the operation updates a; the four registers then rotate roles (a,b,c,d) <- (d,a,b,c) */
    a = d;
    d = c;
    c = b;
    b = t;
  }
  st[0] += a;
  st[1] += b;
  st[2] += c;
  st[3] += d;
}

/* MD5 of an arbitrary byte string (RFC 1321 Sections 3.1-3.5). */
void oracle_md5(const uint8_t* msg, uint64_t len, uint8_t out[16]) {
  md5_init_table();
  uint32_t st[4] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u}; /* Section 3.3 */
  uint64_t full = len / 64;
  for (uint64_t b = 0; b < full; b++) md5_block(st, msg + 64 * b);
  /* Sections 3.1 and 3.2: the tail, a single 1 bit, zeros to 56 mod 64 bytes, bit length LE */
  uint8_t tail[128];
  memset(tail, 0, sizeof tail);
  uint64_t rem = len - 64 * full;
  memcpy(tail, msg + 64 * full, (size_t)rem);
  tail[rem] = 0x80;
  uint64_t tail_len = (rem < 56) ? 64 : 128;
  uint64_t bits = len * 8u;
  for (int j = 0; j < 8; j++) tail[tail_len - 8 + j] = (uint8_t)(bits >> (8 * j));
  md5_block(st, tail);
  if (tail_len == 128) md5_block(st, tail + 64);
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) out[4 * j + q] = (uint8_t)(st[j] >> (8 * q)); /* Section 3.5 */
}

/* MD5 of n consecutive 512-byte sectors; out holds 16 bytes per sector. */
void oracle_md5_sectors(const uint8_t* data, uint64_t n_sectors, uint8_t* out) {
  md5_init_table();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n_sectors; i++) oracle_md5(data + (uint64_t)i * SECTOR, SECTOR, out + 16 * i);
}

/* ----------------------------------------------------- other sector signatures (Section 2) */

/* The MD5 state (A, B, C, D) after the 8 data blocks of a 512-byte message, without the
 * padding block (Section 2.1: for fixed 4096-bit sectors the padding block depends on nothing
 * but the length). 16 bytes, same byte order as an MD5 digest. */
void oracle_md5_nopad(const uint8_t* sector, uint8_t out[16]) {
  md5_init_table();
  uint32_t st[4] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u};
  for (int b = 0; b < 8; b++) md5_block(st, sector + 64 * b);
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) out[4 * j + q] = (uint8_t)(st[j] >> (8 * q));
}

/* Finish a 512-byte message's MD5 from the state oracle_md5_nopad returned: one more block
 * holding the RFC padding for a 4096-bit message. */
void oracle_md5_finish_sector(const uint8_t state[16], uint8_t out[16]) {
  md5_init_table();
  uint32_t st[4];
  for (int j = 0; j < 4; j++)
    st[j] = (uint32_t)state[4 * j] | ((uint32_t)state[4 * j + 1] << 8) | ((uint32_t)state[4 * j + 2] << 16) |
            ((uint32_t)state[4 * j + 3] << 24);
  uint8_t pad[64];
  memset(pad, 0, sizeof pad);
  pad[0] = 0x80;
  const uint64_t bits = 512u * 8u;
  for (int j = 0; j < 8; j++) pad[56 + j] = (uint8_t)(bits >> (8 * j));
  md5_block(st, pad);
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) out[4 * j + q] = (uint8_t)(st[j] >> (8 * q));
}

/* djb2 with a 64-bit accumulator (Eq. 1, Section 4): h = 5381, then h = h * 33 + s_i for
 * every byte s_i, modulo 2^64. */
uint64_t oracle_djb2_64(const uint8_t* msg, uint64_t len) {
  uint64_t h = 5381u;
  for (uint64_t i = 0; i < len; i++) h = h * 33u + msg[i];
  return h;
}

/* CRC64 with the generator polynomial x^64 + x^4 + x^3 + x + 1 (Section 2.1): the remainder
 * of M(x) * x^64 divided by the generator in modulo-2 arithmetic, where M(x) takes the
 * message's bits most significant bit of the first byte first. No initial value and no final
 * XOR (the paper defines the CRC as that remainder). Bit-serial long division. */
uint64_t oracle_crc64(const uint8_t* msg, uint64_t len) {
  const uint64_t low = 0x1Bu; /* x^4 + x^3 + x + 1; the x^64 term is the bit shifted out */
  uint64_t rem = 0;
  for (uint64_t i = 0; i < len; i++) {
    for (int b = 7; b >= 0; b--) {
      const uint64_t in = (msg[i] >> b) & 1u;
      const uint64_t top = rem >> 63;
      rem = (rem << 1) | in;
      if (top) rem ^= low;
    }
  }
  /* the x^64 factor: shift 64 zero bits through */
  for (int b = 0; b < 64; b++) {
    const uint64_t top = rem >> 63;
    rem <<= 1;
    if (top) rem ^= low;
  }
  return rem;
}

/* Signature kinds shared with the library's options. */
#define SIG_MD5 0
#define SIG_MD5_NOPAD 1
#define SIG_DJB2_64 2
#define SIG_CRC64 3

/* The 16-byte signature of one 512-byte sector; 64-bit signatures are stored little-endian in
 * the first 8 bytes, the rest zero. */
void oracle_signature(const uint8_t* sector, int sig, uint8_t out[16]) {
  memset(out, 0, 16);
  if (sig == SIG_MD5) {
    oracle_md5(sector, SECTOR, out);
  } else if (sig == SIG_MD5_NOPAD) {
    oracle_md5_nopad(sector, out);
  } else {
    const uint64_t h = sig == SIG_DJB2_64 ? oracle_djb2_64(sector, SECTOR) : oracle_crc64(sector, SECTOR);
    for (int j = 0; j < 8; j++) out[j] = (uint8_t)(h >> (8 * j));
  }
}

/* The signatures of n consecutive 512-byte sectors, 16 bytes each as oracle_signature writes
 * them (independent sectors, optionally in parallel). */
void oracle_signatures(const uint8_t* data, uint64_t n_sectors, int sig, uint8_t* out) {
  md5_init_table();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n_sectors; i++) oracle_signature(data + (uint64_t)i * SECTOR, sig, out + 16 * i);
}

/* The MD5 state (A, B, C, D) after n_blocks 64-byte blocks of msg, with no padding block
 * (RFC 1321 Section 3.4 applied to the blocks as they are); 16 bytes, digest byte order. For
 * a 64-byte fragment this is Section 2.1's signature without padding, one compression. */
void oracle_md5_blocks(const uint8_t* msg, uint64_t n_blocks, uint8_t out[16]) {
  md5_init_table();
  uint32_t st[4] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u};
  for (uint64_t b = 0; b < n_blocks; b++) md5_block(st, msg + 64 * b);
  for (int j = 0; j < 4; j++)
    for (int q = 0; q < 4; q++) out[4 * j + q] = (uint8_t)(st[j] >> (8 * q));
}

/* The signature of every 64-byte window at a 4-byte offset (Section 5): window k is bytes
 * [4k, 4k + 64) for every k with 4k + 64 <= image_bytes. 16 bytes per window: the MD5 digest of
 * the 64 bytes (SIG_MD5), the state after its one block (SIG_MD5_NOPAD), or djb2-64 of the 64
 * bytes little-endian in the first 8 bytes and zeros after (SIG_DJB2_64). */
void oracle_window_signatures(const uint8_t* image, uint64_t image_bytes, int sig, uint8_t* out) {
  md5_init_table();
  const int64_t n_win = image_bytes >= 64 ? (int64_t)((image_bytes - 64) / 4 + 1) : 0;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_win; k++) {
    const uint8_t* w = image + 4 * (uint64_t)k;
    uint8_t* o = out + 16 * (uint64_t)k;
    memset(o, 0, 16);
    if (sig == SIG_MD5) {
      oracle_md5(w, 64, o);
    } else if (sig == SIG_MD5_NOPAD) {
      oracle_md5_blocks(w, 1, o);
    } else {
      const uint64_t h = oracle_djb2_64(w, 64);
      for (int j = 0; j < 8; j++) o[j] = (uint8_t)(h >> (8 * j));
    }
  }
}

/* ------------------------------------------------------------------ the exclusion rule */

/* A master sector is excluded iff all 512 of its bytes are equal. */
int oracle_sector_trivial(const uint8_t* sector) {
  for (uint32_t j = 1; j < SECTOR; j++)
    if (sector[j] != sector[0]) return 0;
  return 1;
}

/* ---------------------------------------------------------------- shared result helpers */

static int triple_cmp(const void* pa, const void* pb) {
  const oracle_triple* a = (const oracle_triple*)pa;
  const oracle_triple* b = (const oracle_triple*)pb;
  if (a->disk_sector != b->disk_sector) return a->disk_sector < b->disk_sector ? -1 : 1;
  if (a->file_id != b->file_id) return a->file_id < b->file_id ? -1 : 1;
  if (a->file_sector != b->file_sector) return a->file_sector < b->file_sector ? -1 : 1;
  return 0;
}

/* ------------------------------------------------------------- brute force (definition) */

/* Every (i, f, s) with disk sector i byte-equal to kept master sector s of file f, sorted.
 * Returns the number of triples; writes at most cap of them into out. */
int64_t oracle_match_brute(const uint8_t* image, uint64_t image_bytes, const uint8_t* const* files,
                           const uint64_t* file_bytes, uint32_t n_files, oracle_triple* out, uint64_t cap) {
  uint64_t n_disk = image_bytes / SECTOR;
  uint64_t n = 0;
  for (uint64_t i = 0; i < n_disk; i++) {
    const uint8_t* d = image + i * SECTOR;
    for (uint32_t f = 0; f < n_files; f++) {
      uint64_t n_fs = file_bytes[f] / SECTOR;
      for (uint64_t s = 0; s < n_fs; s++) {
        const uint8_t* m = files[f] + s * SECTOR;
        if (oracle_sector_trivial(m)) continue;
        if (memcmp(d, m, SECTOR) != 0) continue;
        if (n < cap) {
          out[n].disk_sector = i;
          out[n].file_id = f;
          out[n].file_sector = (uint32_t)s;
        }
        n++;
      }
    }
  }
  if (n <= cap) qsort(out, (size_t)n, sizeof(oracle_triple), triple_cmp);
  return (int64_t)n;
}

/* ------------------------------------------------------ signature lookup (the method) */

typedef struct {
  uint8_t digest[16];
  uint32_t file_id;
  uint32_t file_sector;
} db_entry;

typedef struct {
  db_entry* e;
  uint64_t n;
  int sig;                     /* signature kind */
  const uint8_t* const* files; /* borrowed; used to confirm matches of 64-bit signatures */
} oracle_db;

static int db_cmp(const void* pa, const void* pb) {
  const db_entry* a = (const db_entry*)pa;
  const db_entry* b = (const db_entry*)pb;
  int c = memcmp(a->digest, b->digest, 16);
  if (c) return c;
  if (a->file_id != b->file_id) return a->file_id < b->file_id ? -1 : 1;
  if (a->file_sector != b->file_sector) return a->file_sector < b->file_sector ? -1 : 1;
  return 0;
}

/* The signature database: one (signature, f, s) entry per kept master sector, sorted. The
 * files stay borrowed by the database (64-bit signatures are confirmed against their bytes). */
oracle_db* oracle_db_build_sig(const uint8_t* const* files, const uint64_t* file_bytes, uint32_t n_files, int sig) {
  md5_init_table();
  uint64_t total = 0;
  for (uint32_t f = 0; f < n_files; f++) total += file_bytes[f] / SECTOR;
  oracle_db* db = (oracle_db*)calloc(1, sizeof(oracle_db));
  if (!db) return NULL;
  db->e = (db_entry*)malloc(sizeof(db_entry) * (total ? total : 1));
  if (!db->e) {
    free(db);
    return NULL;
  }
  uint64_t n = 0;
  for (uint32_t f = 0; f < n_files; f++) {
    uint64_t n_fs = file_bytes[f] / SECTOR;
    for (uint64_t s = 0; s < n_fs; s++) {
      const uint8_t* m = files[f] + s * SECTOR;
      if (oracle_sector_trivial(m)) continue;
      db->e[n].file_id = f;
      db->e[n].file_sector = (uint32_t)s;
      n++;
    }
  }
  /* hash in parallel; every entry is independent */
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < (int64_t)n; q++)
    oracle_signature(files[db->e[q].file_id] + (uint64_t)db->e[q].file_sector * SECTOR, sig, db->e[q].digest);
  qsort(db->e, (size_t)n, sizeof(db_entry), db_cmp);
  db->n = n;
  db->sig = sig;
  db->files = files;
  return db;
}

/* The MD5 database. */
oracle_db* oracle_db_build(const uint8_t* const* files, const uint64_t* file_bytes, uint32_t n_files) {
  return oracle_db_build_sig(files, file_bytes, n_files, SIG_MD5);
}

uint64_t oracle_db_size(const oracle_db* db) { return db->n; }

void oracle_db_free(oracle_db* db) {
  if (!db) return;
  free(db->e);
  free(db);
}

/* First entry whose digest is >= key (binary search over the sorted database). */
static uint64_t db_lower_bound(const oracle_db* db, const uint8_t key[16]) {
  uint64_t lo = 0, hi = db->n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (memcmp(db->e[mid].digest, key, 16) < 0)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* Look up n_sectors consecutive disk sectors whose first one has index first_index. Every
 * triple found is written (at most cap) and the total is returned, sorted. */
int64_t oracle_db_lookup(const oracle_db* db, const uint8_t* sectors, uint64_t n_sectors, uint64_t first_index,
                         oracle_triple* out, uint64_t cap) {
  uint64_t* lo = (uint64_t*)malloc(sizeof(uint64_t) * (n_sectors ? n_sectors : 1));
  uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * (n_sectors ? n_sectors : 1));
  if (!lo || !cnt) {
    free(lo);
    free(cnt);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n_sectors; i++) {
    uint8_t dg[16];
    oracle_signature(sectors + (uint64_t)i * SECTOR, db->sig, dg);
    uint64_t a = db_lower_bound(db, dg), b = a;
    while (b < db->n && memcmp(db->e[b].digest, dg, 16) == 0) b++;
    lo[i] = a;
    cnt[i] = b - a;
  }
  /* 64-bit signatures collide: confirm every candidate byte for byte (Section 3.1) */
  const int confirm = db->sig == SIG_DJB2_64 || db->sig == SIG_CRC64;
  uint64_t n = 0;
  for (uint64_t i = 0; i < n_sectors; i++)
    for (uint64_t q = 0; q < cnt[i]; q++) {
      const db_entry* e = &db->e[lo[i] + q];
      if (confirm && memcmp(sectors + i * SECTOR, db->files[e->file_id] + (uint64_t)e->file_sector * SECTOR,
                            SECTOR) != 0)
        continue;
      if (n < cap) {
        out[n].disk_sector = first_index + i;
        out[n].file_id = db->e[lo[i] + q].file_id;
        out[n].file_sector = db->e[lo[i] + q].file_sector;
      }
      n++;
    }
  free(lo);
  free(cnt);
  if (n <= cap) qsort(out, (size_t)n, sizeof(oracle_triple), triple_cmp);
  return (int64_t)n;
}

/* The whole method over one image with a chosen signature: database, lookup of every whole
 * sector (confirmed for 64-bit signatures), sorted result. */
int64_t oracle_match_sig(const uint8_t* image, uint64_t image_bytes, const uint8_t* const* files,
                         const uint64_t* file_bytes, uint32_t n_files, int sig, oracle_triple* out, uint64_t cap) {
  oracle_db* db = oracle_db_build_sig(files, file_bytes, n_files, sig);
  if (!db) return -1;
  int64_t n = oracle_db_lookup(db, image, image_bytes / SECTOR, 0, out, cap);
  oracle_db_free(db);
  return n;
}

/* Position-keyed matching (Section 3.1: tables S_tau, one per sector position tau in an
 * 8-sector cluster): the result restricted to triples whose disk sector sits at the same cluster
 * position as the master sector, disk positions counted from sector base_offset (the start of
 * the partition the clusters belong to): ((i - base_offset) mod 8) == (s mod 8). */
int64_t oracle_match_position(const uint8_t* image, uint64_t image_bytes, const uint8_t* const* files,
                              const uint64_t* file_bytes, uint32_t n_files, uint64_t base_offset, oracle_triple* out,
                              uint64_t cap) {
  oracle_db* db = oracle_db_build(files, file_bytes, n_files);
  if (!db) return -1;
  const uint64_t n_disk = image_bytes / SECTOR;
  uint64_t cap_all = 1024;
  oracle_triple* all = NULL;
  int64_t n_all;
  for (;;) {
    free(all);
    all = (oracle_triple*)malloc(sizeof(oracle_triple) * cap_all);
    if (!all) {
      oracle_db_free(db);
      return -1;
    }
    n_all = oracle_db_lookup(db, image, n_disk, 0, all, cap_all);
    if (n_all < 0 || (uint64_t)n_all <= cap_all) break;
    cap_all = (uint64_t)n_all;
  }
  oracle_db_free(db);
  if (n_all < 0) {
    free(all);
    return -1;
  }
  uint64_t n = 0;
  for (int64_t k = 0; k < n_all; k++) {
    const uint64_t tau_disk = ((all[k].disk_sector % 8u) + 8u - (base_offset % 8u)) % 8u;
    if (tau_disk != all[k].file_sector % 8u) continue;
    if (n < cap) out[n] = all[k];
    n++;
  }
  free(all);
  return (int64_t)n;
}

/* The whole method over one image: database, lookup of every whole sector, sorted result. */
int64_t oracle_match_hash(const uint8_t* image, uint64_t image_bytes, const uint8_t* const* files,
                          const uint64_t* file_bytes, uint32_t n_files, oracle_triple* out, uint64_t cap) {
  oracle_db* db = oracle_db_build(files, file_bytes, n_files);
  if (!db) return -1;
  int64_t n = oracle_db_lookup(db, image, image_bytes / SECTOR, 0, out, cap);
  oracle_db_free(db);
  return n;
}

/* ------------------------------------------------------ 64-byte fragments (Section 5) */

/* Section 5 proposes scanning every 64-byte fragment of a disk that starts on a 32-bit boundary,
 * to find small images and logos embedded in documents. The definition used here:
 *   window k of the image is its bytes [4k, 4k + 64), for every k with 4k + 64 <= image_bytes;
 *   fragment j of master file f is its bytes [64j, 64j + 64); only whole fragments count;
 *   a fragment whose 64 bytes are all equal is excluded (the sector rule at fragment size);
 *   the result is every (k, f, j) with window k byte-equal to kept fragment j of file f, sorted
 *   (k in the triple's disk_sector field, j in its file_sector field). */
#define FRAG 64u
#define FRAG_STRIDE 4u

int oracle_fragment_trivial(const uint8_t* frag) {
  for (uint32_t j = 1; j < FRAG; j++)
    if (frag[j] != frag[0]) return 0;
  return 1;
}

static uint64_t frag_windows(uint64_t image_bytes) {
  return image_bytes >= FRAG ? (image_bytes - FRAG) / FRAG_STRIDE + 1 : 0;
}

/* The definition itself: every window against every kept fragment. Tiny inputs only. */
int64_t oracle_frag_match_brute(const uint8_t* image, uint64_t image_bytes, const uint8_t* const* files,
                                const uint64_t* file_bytes, uint32_t n_files, oracle_triple* out, uint64_t cap) {
  const uint64_t n_win = frag_windows(image_bytes);
  uint64_t n = 0;
  for (uint64_t k = 0; k < n_win; k++) {
    const uint8_t* w = image + k * FRAG_STRIDE;
    for (uint32_t f = 0; f < n_files; f++) {
      const uint64_t n_fr = file_bytes[f] / FRAG;
      for (uint64_t j = 0; j < n_fr; j++) {
        const uint8_t* m = files[f] + j * FRAG;
        if (oracle_fragment_trivial(m) || memcmp(w, m, FRAG) != 0) continue;
        if (n < cap) {
          out[n].disk_sector = k;
          out[n].file_id = f;
          out[n].file_sector = (uint32_t)j;
        }
        n++;
      }
    }
  }
  if (n <= cap) qsort(out, (size_t)n, sizeof(oracle_triple), triple_cmp);
  return (int64_t)n;
}

typedef struct {
  const uint8_t* bytes;
  uint32_t file_id;
  uint32_t frag;
} frag_entry;

static int frag_cmp(const void* pa, const void* pb) {
  const frag_entry* a = (const frag_entry*)pa;
  const frag_entry* b = (const frag_entry*)pb;
  int c = memcmp(a->bytes, b->bytes, FRAG);
  if (c) return c;
  if (a->file_id != b->file_id) return a->file_id < b->file_id ? -1 : 1;
  if (a->frag != b->frag) return a->frag < b->frag ? -1 : 1;
  return 0;
}

/* First entry whose bytes are >= w (binary search in memcmp order). */
static uint64_t frag_lower_bound(const frag_entry* e, uint64_t n, const uint8_t* w) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (memcmp(e[mid].bytes, w, FRAG) < 0)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* The same result through the kept fragments sorted by their bytes (then by file and
 * fragment): each window is binary-searched and the run of equal fragments reported. Windows
 * are processed in blocks (count in parallel, then write in order), so the output is sorted. */
int64_t oracle_frag_match(const uint8_t* image, uint64_t image_bytes, const uint8_t* const* files,
                          const uint64_t* file_bytes, uint32_t n_files, oracle_triple* out, uint64_t cap) {
  uint64_t total = 0;
  for (uint32_t f = 0; f < n_files; f++) total += file_bytes[f] / FRAG;
  frag_entry* e = (frag_entry*)malloc(sizeof(frag_entry) * (total ? total : 1));
  if (!e) return -1;
  uint64_t m = 0;
  for (uint32_t f = 0; f < n_files; f++)
    for (uint64_t j = 0; j < file_bytes[f] / FRAG; j++) {
      const uint8_t* b = files[f] + j * FRAG;
      if (oracle_fragment_trivial(b)) continue;
      e[m].bytes = b;
      e[m].file_id = f;
      e[m].frag = (uint32_t)j;
      m++;
    }
  qsort(e, (size_t)m, sizeof(frag_entry), frag_cmp);
  const uint64_t n_win = frag_windows(image_bytes);
  const uint64_t block = 1u << 20;
  uint64_t* lo = (uint64_t*)malloc(sizeof(uint64_t) * block);
  uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * block);
  if (!lo || !cnt) {
    free(e);
    free(lo);
    free(cnt);
    return -1;
  }
  uint64_t n = 0;
  for (uint64_t k0 = 0; k0 < n_win; k0 += block) {
    const uint64_t nb = n_win - k0 < block ? n_win - k0 : block;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)nb; i++) {
      const uint8_t* w = image + (k0 + (uint64_t)i) * FRAG_STRIDE;
      uint64_t a = frag_lower_bound(e, m, w), b = a;
      while (b < m && memcmp(e[b].bytes, w, FRAG) == 0) b++;
      lo[i] = a;
      cnt[i] = b - a;
    }
    for (uint64_t i = 0; i < nb; i++)
      for (uint64_t q = 0; q < cnt[i]; q++) {
        if (n < cap) {
          out[n].disk_sector = k0 + i;
          out[n].file_id = e[lo[i] + q].file_id;
          out[n].file_sector = e[lo[i] + q].frag;
        }
        n++;
      }
  }
  free(e);
  free(lo);
  free(cnt);
  return (int64_t)n;
}

/* Threads the parallel loops use (1 when built without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
