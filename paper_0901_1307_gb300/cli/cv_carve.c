/*
 * cv_carve: scan disk images for the sectors (or 64-byte fragments) of known files, from the
 * command line, through the C ABI of include/cv.h alone.
 *
 *   cv_carve [-f] [-s SIG] [-p BASE] IMAGE... -- MASTER...
 *
 * Every match is printed as one line "image_index disk_sector file_id file_sector" (with -f,
 * "image_index window fragment..." for 64-byte fragments at 4-byte offsets), in the library's
 * sorted order; a summary goes to stderr. Options: -s 0..3 the signature (MD5, MD5 without
 * padding, djb2-64, CRC64), -p BASE position-keyed tables with clusters counted from sector BASE,
 * -f fragments instead of sectors. Files are read whole into host memory; the library copies
 * them to the device. Exit status: 0 on success, 1 on a usage or I/O error, 2 on a library error.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cv.h"

static void* read_file(const char* path, uint64_t* n) {
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  if (fseek(f, 0, SEEK_END) != 0) {
    fclose(f);
    return NULL;
  }
  long len = ftell(f);
  if (len < 0 || fseek(f, 0, SEEK_SET) != 0) {
    fclose(f);
    return NULL;
  }
  void* buf = malloc(len > 0 ? (size_t)len : 1);
  if (buf && len > 0 && fread(buf, 1, (size_t)len, f) != (size_t)len) {
    free(buf);
    buf = NULL;
  }
  fclose(f);
  *n = (uint64_t)len;
  return buf;
}

static int fail(const char* what, int rc) {
  fprintf(stderr, "cv_carve: %s: %s\n", what, cv_strerror(rc));
  return 2;
}

int main(int argc, char** argv) {
  int frag = 0, position = 0;
  unsigned sig = 0;
  uint64_t base = 0;
  int a = 1;
  for (; a < argc && argv[a][0] == '-' && strcmp(argv[a], "--") != 0; a++) {
    if (strcmp(argv[a], "-f") == 0) {
      frag = 1;
    } else if (strcmp(argv[a], "-s") == 0 && a + 1 < argc) {
      sig = (unsigned)strtoul(argv[++a], NULL, 10);
    } else if (strcmp(argv[a], "-p") == 0 && a + 1 < argc) {
      position = 1;
      base = strtoull(argv[++a], NULL, 10);
    } else {
      fprintf(stderr, "usage: cv_carve [-f] [-s SIG] [-p BASE] IMAGE... -- MASTER...\n");
      return 1;
    }
  }
  int sep = a;
  while (sep < argc && strcmp(argv[sep], "--") != 0) sep++;
  const int n_images = sep - a, n_files = sep < argc ? argc - sep - 1 : 0;
  if (n_images < 1 || sep >= argc) {
    fprintf(stderr, "usage: cv_carve [-f] [-s SIG] [-p BASE] IMAGE... -- MASTER...\n");
    return 1;
  }
  cv_buf* files = (cv_buf*)calloc((size_t)(n_files > 0 ? n_files : 1), sizeof(cv_buf));
  cv_buf* images = (cv_buf*)calloc((size_t)n_images, sizeof(cv_buf));
  if (!files || !images) return 1;
  for (int f = 0; f < n_files; f++) {
    files[f].data = read_file(argv[sep + 1 + f], &files[f].n_bytes);
    if (!files[f].data) {
      fprintf(stderr, "cv_carve: cannot read %s\n", argv[sep + 1 + f]);
      return 1;
    }
  }
  for (int i = 0; i < n_images; i++) {
    images[i].data = read_file(argv[a + i], &images[i].n_bytes);
    if (!images[i].data) {
      fprintf(stderr, "cv_carve: cannot read %s\n", argv[a + i]);
      return 1;
    }
  }

  cv_master_opts mo;
  memset(&mo, 0, sizeof mo);
  mo.struct_size = sizeof mo;
  mo.bloom_bits_per_key = CV_BLOOM_AUTO;
  mo.signature = sig;
  mo.position_mode = position ? CV_POSITION_CLUSTER : CV_POSITION_ANY;
  mo.layout = CV_LAYOUT_HASH;
  mo.unit = frag ? CV_UNIT_FRAGMENT : CV_UNIT_SECTOR;
  cv_master* m = NULL;
  int rc = cv_master_build(files, (uint32_t)n_files, &mo, &m);
  if (rc != CV_OK) return fail("cv_master_build", rc);

  cv_scan_opts so;
  memset(&so, 0, sizeof so);
  so.struct_size = sizeof so;
  so.base_offset = base;
  cv_result* r = NULL;
  rc = cv_scan(m, images, (uint32_t)n_images, &so, &r);
  if (rc != CV_OK) {
    cv_free(m);
    return fail("cv_scan", rc);
  }
  uint64_t total = 0;
  for (int i = 0; i < n_images; i++) {
    const cv_match* hits;
    uint64_t n;
    rc = cv_matches(r, (uint32_t)i, &hits, &n);
    if (rc != CV_OK) {
      cv_free(r);
      cv_free(m);
      return fail("cv_matches", rc);
    }
    for (uint64_t k = 0; k < n; k++)
      printf("%d %llu %u %u\n", i, (unsigned long long)hits[k].disk_sector, hits[k].file_id, hits[k].file_sector);
    total += n;
  }
  cv_scan_stats st;
  if (cv_scan_get_stats(r, &st) == CV_OK)
    fprintf(stderr, "cv_carve: %llu %s scanned, %llu matches, %.3f ms\n", (unsigned long long)st.sectors,
            frag ? "windows" : "sectors", (unsigned long long)total, st.total_ms);
  cv_free(r);
  cv_free(m);
  for (int f = 0; f < n_files; f++) free((void*)files[f].data);
  for (int i = 0; i < n_images; i++) free((void*)images[i].data);
  free(files);
  free(images);
  return 0;
}
