/*
 * A plain C99 client of the detector's C ABI (include/ssd.h): it must compile
 * with -std=c99 -Wall -Wextra -Werror and link against libssd.so, so the
 * boundary stays C. It needs no GPU: it exercises the host-only calls and the
 * error paths of the others.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "ssd.h"

static int fail(const char* what, int rc) {
  fprintf(stderr, "%s: %s (%d) %s\n", what, ssd_strerror(rc), rc, ssd_last_cuda_error());
  return 1;
}

int main(void) {
  ssd_params p;
  memset(&p, 0, sizeof(p));
  p.log2_eta = 11; p.q = 14; p.r = 5; p.delta = 6; p.k = 4; p.theta = 1024;   /* Sec. 5 */
  uint32_t thr = 0;
  if (ssd_params_check(&p) != SSD_OK) return fail("params", SSD_EINVAL);
  int rc = ssd_threshold(&p, &thr);
  if (rc != SSD_OK) return fail("threshold", rc);
  printf("version %d threshold %u\n", ssd_version(), thr);

  /* invalid arguments are refused without touching a GPU */
  ssd_params bad = p;
  bad.delta = 1;                                            /* (r-2)*delta + q < 32 */
  if (ssd_params_check(&bad) != SSD_EINVAL) return fail("bad params accepted", SSD_EINVAL);
  if (ssd_create(NULL, NULL, 0, NULL) != SSD_EINVAL) return fail("null create accepted", SSD_EINVAL);
  if (ssd_sketch_set_view(NULL, SSD_SIDE_CNET, 0, 0) != SSD_EINVAL) return fail("null view", SSD_EINVAL);
  if (ssd_buffer_epoch(NULL) != 0 || ssd_launch_count(NULL) != 0) return fail("null counters", SSD_EINVAL);

  /* every entry point refuses null handles and pointers before it touches the GPU */
  uint64_t u64 = 0;
  uint32_t a = 0, b = 0, c = 0;
  uint16_t rec[8];
  const uint32_t* pp = NULL;
  ssd_tuning tn;
  ssd_stats st;
  memset(&tn, 0, sizeof(tn));
  memset(rec, 0, sizeof(rec));
  const int refusals[] = {
      ssd_params_check(NULL),
      ssd_threshold(NULL, &thr),
      ssd_threshold(&p, NULL),
      ssd_sketch_create(NULL, NULL),
      ssd_sketch_slot(NULL, &u64),
      ssd_sketch_set_slot(NULL, 1),
      ssd_sketch_view(NULL, &a, &b, &c),
      ssd_sketch_occupancy(NULL, &u64, NULL),
      ssd_sketch_export(NULL, 0, 1, rec, NULL),
      ssd_sketch_import(NULL, rec, 0, NULL),
      ssd_scan(NULL, NULL, 0, NULL),
      ssd_scan_host(NULL, NULL, 0, NULL),
      ssd_scan_batch(NULL, &pp, &u64, 1, NULL),
      ssd_advance(NULL, 1, NULL),
      ssd_merge(NULL, 1, NULL, NULL),
      ssd_regain(NULL, NULL, NULL, NULL, 0, &u64, NULL),
      ssd_regain_static(NULL, 0, 0, 0, NULL, NULL, NULL, NULL, 0, &u64, NULL),
      ssd_regain_static(&p, 0, 0, 0, NULL, NULL, NULL, NULL, 0, &u64, NULL),
      ssd_regain_static(&p, 2, 0, 0, NULL, NULL, NULL, NULL, 0, &u64, NULL),
      ssd_min_merge(NULL, NULL, NULL, 1, 8, NULL),
      ssd_sketch_data(NULL, NULL),
      ssd_close_slot(NULL, NULL, 1, NULL, NULL, NULL, 0, NULL, NULL),
      ssd_set_trace(NULL, NULL, NULL, NULL),
      ssd_slot(NULL, NULL, &pp, &u64, 1, NULL, NULL, NULL, 0, NULL, NULL),
      ssd_slot_host(NULL, NULL, &pp, &u64, 1, NULL, NULL, NULL, 0, NULL, NULL),
      ssd_reserve(NULL, 1),
      ssd_tuning_get(NULL, &tn),
      ssd_tuning_set(NULL, &tn),
      ssd_autotune(NULL, NULL, &pp, &u64, 1, NULL, 1, &tn, NULL),
      ssd_stats_get(NULL, &st, NULL),
  };
  for (size_t i = 0; i < sizeof(refusals) / sizeof(refusals[0]); ++i)
    if (refusals[i] != SSD_EINVAL) {
      fprintf(stderr, "refusal %u returned %d\n", (unsigned)i, refusals[i]);
      return 1;
    }
  ssd_destroy(NULL);          /* no-ops */
  ssd_sketch_destroy(NULL);
  if (ssd_sketch_bytes(NULL) != 0) return fail("null sketch bytes", SSD_EINVAL);
  for (int code = 0; code >= -6; --code)
    if (strcmp(ssd_strerror(code), "unknown error") == 0) return fail("strerror", code);
  printf("refusals ok (%u calls)\n", (unsigned)(sizeof(refusals) / sizeof(refusals[0])));

  return 0;
}
