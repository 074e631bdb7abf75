/*
 * Host side of the seeded input generator (see synth_def.h for the definition of every byte).
 * Input generation only: no signature or matching arithmetic. Used by the tests, the CPU
 * oracle's inputs and the benchmark; built with gcc, OpenMP-parallel over sectors.
 */
#include <stdint.h>
#include <string.h>

#include "synth_def.h"

void synth_vocab(uint64_t sigma, uint8_t* out) {
  for (uint32_t k = 0; k < SY_VOCAB; k++) sy_vocab_word(sigma, k, out + SY_VOCAB_STRIDE * k);
}

/* Sectors [first, first + n) of one image into out (n * 512 bytes, 8-byte aligned). */
void synth_image(uint64_t sigma, uint64_t mu, const int32_t* plant_file, const uint32_t* plant_fcluster,
                 const uint8_t* plant_over, uint64_t n_clusters, const uint32_t* file_nsect, const uint8_t* vocab,
                 uint64_t first, uint64_t n, uint8_t* out) {
  sy_plan p;
  p.sigma = sigma;
  p.mu = mu;
  p.plant_file = plant_file;
  p.plant_fcluster = plant_fcluster;
  p.plant_over = plant_over;
  p.file_nsect = file_nsect;
  p.vocab = vocab;
  p.n_clusters = n_clusters;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)n; j++) sy_image_sector(&p, first + (uint64_t)j, (uint64_t*)(out + (uint64_t)j * SY_SECTOR));
}

/* Sectors [s0, s0 + n) of master file f. */
void synth_master(uint64_t mu, uint32_t f, uint32_t s0, uint32_t n, uint8_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)n; j++) sy_master_sector(mu, f, s0 + (uint32_t)j, (uint64_t*)(out + (uint64_t)j * SY_SECTOR));
}

/* Sectors [first, first + n) of a list of random bytes of a given seed and stream: used for
 * ad-hoc test content (fresh random sectors that no master file holds). */
void synth_random(uint64_t seed, uint64_t stream, uint64_t first, uint64_t n, uint8_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)n; j++) sy_random_sector(seed, stream, first + (uint64_t)j, (uint64_t*)(out + (uint64_t)j * SY_SECTOR));
}

uint64_t synth_hash(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) { return sy_hash(seed, stream, a, b); }
