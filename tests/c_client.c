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
  printf("refusals ok\n");

  return 0;
}
