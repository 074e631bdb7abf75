/*
 * Seeded synthetic disk images and master files: the one definition that the host generator
 * (synth_host.c) and the device generator (synth_cuda.cu) both compile, so that any sector of
 * any workload has the same bytes on either side.
 *
 * This header holds input generation only: no signature, table or matching arithmetic.
 *
 * Randomness is counter-based: every 64-bit word is sy_hash(seed, stream, a, b), built from the
 * SplitMix64 output function (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so a sector can be produced alone, in any order, on any device.
 *
 * Content of image sector i (seed sigma), following the paper's workload of random-data files
 * placed at 4 KiB cluster granularity (Section 2, Section 4):
 *   - if its cluster q = i / 8 carries a planted master cluster (file f, cluster c) and
 *     k = i % 8 is below the cluster's overwrite count: fresh random bytes (a newer file that
 *     overwrote the first sectors of the cluster, Section 2);
 *   - else if s = 8c + k is a sector of file f: master sector (f, s);
 *   - else background, drawn per sector: 70% uniform random bytes, 15% all-zero, 15% ASCII
 *     text made of words from a 2,000-word vocabulary (lowercase a-z, 2-10 letters) joined by
 *     single spaces and cut at 512 bytes.
 * Master sector (mu, f, s): 64 uniform random words.
 */
#ifndef SYNTH_DEF_H
#define SYNTH_DEF_H

#include <stdint.h>

#ifdef __CUDACC__
#define SY_HD __host__ __device__ __forceinline__
#else
#define SY_HD static inline
#endif

#define SY_SECTOR 512
#define SY_VOCAB 2000
#define SY_VOCAB_STRIDE 16 /* byte 0 = length, bytes 1..10 = letters */

enum {
  SY_STREAM_CLASS = 1,
  SY_STREAM_RAND = 2,
  SY_STREAM_TEXTW = 3,
  SY_STREAM_VOCLEN = 4,
  SY_STREAM_VOCCHR = 5,
  SY_STREAM_MASTER = 6,
  SY_STREAM_OVER = 7
};

/* Background class thresholds out of 100: [0,70) random, [70,85) zero, [85,100) text. */
#define SY_PCT_RANDOM 70u
#define SY_PCT_ZERO 15u

SY_HD uint64_t sy_mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

SY_HD uint64_t sy_hash(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
  return sy_mix(sy_mix(sy_mix(seed ^ (stream * 0xD1B54A32D192ED03ull)) ^ a) ^ b);
}

/* Vocabulary word k of seed sigma into 16 bytes: length, then letters. */
SY_HD void sy_vocab_word(uint64_t sigma, uint32_t k, uint8_t* out16) {
  uint32_t len = 2u + (uint32_t)(sy_hash(sigma, SY_STREAM_VOCLEN, k, 0) % 9u);
  out16[0] = (uint8_t)len;
  for (uint32_t j = 0; j < 15; j++)
    out16[1 + j] = j < len ? (uint8_t)('a' + sy_hash(sigma, SY_STREAM_VOCCHR, k, j) % 26u) : (uint8_t)0;
}

/* 64 uniform random words from (seed, stream, index). */
SY_HD void sy_random_sector(uint64_t seed, uint64_t stream, uint64_t index, uint64_t* out64) {
  for (uint32_t w = 0; w < 64; w++) out64[w] = sy_hash(seed, stream, index, w);
}

/* Text sector i of seed sigma from the vocabulary table (SY_VOCAB x 16 bytes). */
SY_HD void sy_text_sector(uint64_t sigma, uint64_t i, const uint8_t* vocab, uint8_t* out512) {
  uint32_t pos = 0;
  for (uint64_t t = 0; pos < SY_SECTOR; t++) {
    if (t > 0) out512[pos++] = ' ';
    const uint8_t* w = vocab + SY_VOCAB_STRIDE * (uint32_t)(sy_hash(sigma, SY_STREAM_TEXTW, i, t) % SY_VOCAB);
    for (uint32_t j = 0; j < w[0] && pos < SY_SECTOR; j++) out512[pos++] = w[1 + j];
  }
}

/* Background class of sector i: 0 random, 1 zero, 2 text. */
SY_HD uint32_t sy_class(uint64_t sigma, uint64_t i) {
  uint32_t r = (uint32_t)((sy_hash(sigma, SY_STREAM_CLASS, i, 0) >> 32) % 100u);
  return r < SY_PCT_RANDOM ? 0u : (r < SY_PCT_RANDOM + SY_PCT_ZERO ? 1u : 2u);
}

/* Master sector (f, s) of master seed mu. */
SY_HD void sy_master_sector(uint64_t mu, uint32_t f, uint32_t s, uint64_t* out64) {
  sy_random_sector(mu, SY_STREAM_MASTER, ((uint64_t)f << 32) | s, out64);
}

/* Plan of one image: the planted master cluster per image cluster (plant_file < 0: none). */
typedef struct {
  uint64_t sigma;               /* image seed */
  uint64_t mu;                  /* master seed */
  const int32_t* plant_file;    /* per image cluster: file id or -1 */
  const uint32_t* plant_fcluster; /* per image cluster: cluster index within that file */
  const uint8_t* plant_over;    /* per image cluster: leading sectors overwritten (0..8) */
  const uint32_t* file_nsect;   /* per master file: whole sectors */
  const uint8_t* vocab;         /* SY_VOCAB x 16 bytes for sigma */
  uint64_t n_clusters;          /* entries in the plant arrays (0: no planting) */
} sy_plan;

/* Image sector i (8-byte aligned destination). */
SY_HD void sy_image_sector(const sy_plan* p, uint64_t i, uint64_t* out64) {
  uint64_t q = i >> 3;
  uint32_t k = (uint32_t)(i & 7u);
  if (q < p->n_clusters && p->plant_file[q] >= 0) {
    if (k < p->plant_over[q]) {
      sy_random_sector(p->sigma, SY_STREAM_OVER, i, out64);
      return;
    }
    uint32_t f = (uint32_t)p->plant_file[q];
    uint32_t s = 8u * p->plant_fcluster[q] + k;
    if (s < p->file_nsect[f]) {
      sy_master_sector(p->mu, f, s, out64);
      return;
    }
  }
  uint32_t cls = sy_class(p->sigma, i);
  if (cls == 0u) {
    sy_random_sector(p->sigma, SY_STREAM_RAND, i, out64);
  } else if (cls == 1u) {
    for (uint32_t w = 0; w < 64; w++) out64[w] = 0;
  } else {
    sy_text_sector(p->sigma, i, p->vocab, (uint8_t*)out64);
  }
}

#endif
