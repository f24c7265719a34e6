/*
 * Brute-force pin for regaining sliding super points: enumerate every IPv4
 * value x in [0, 2^32) FORWARD through the reversible hash functions group and
 * decide membership from the estimators directly, with no tuple search, no
 * overlap test and no bit extraction.
 *
 *   verify mode : x is listed iff RHFG[i](x) is hot in every row i and the
 *                 union of its r estimators has R_k >= threshold.
 *   literal mode: x is listed iff for SOME column h of row 0 the tuple
 *                 (h, h^B(1)(x), ..., h^B(r-1)(x)) is all hot with union
 *                 R_k >= threshold, where B(i)(x) is the q-bit window of x
 *                 starting at bit (i-1)*delta + sh0; R_k is the largest such.
 *
 * sh0 = 0 is the shift the library adopts, (i-1)*delta; sh0 = delta is Eq. 2 as
 * printed, i*delta. Under the printed shift no window holds bits 0..delta-1,
 * and a host is regained when its own tuple (verify mode) passes: the windows
 * fix bits delta..31 and RHFG[0](x) = h fixes the rest.
 *
 * Both follow from Eq. 2-3 and the final test of Algorithm 4. Test helper only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint32_t log2_eta, q, r, delta, k, thr;
  const uint32_t* tables;   /* 2048 words */
  const uint8_t* hot;       /* r * 2^q flags */
  const uint32_t* bitmaps;  /* r * 2^q * (eta/32) words: bit j set iff recorder j < k */
  uint32_t sh0;             /* shift of window B(1): 0, or delta for Eq. 2 as printed */
} bf_in;

static uint32_t fwd_hash(const uint32_t* T, uint32_t x) {
  return T[x & 255] ^ T[256 + ((x >> 8) & 255)] ^ T[512 + ((x >> 16) & 255)] ^ T[768 + (x >> 24)];
}

static uint32_t window(const bf_in* in, uint32_t x, uint32_t i) {
  uint32_t s = (i - 1) * in->delta + in->sh0;
  uint32_t v = s < 32 ? x >> s : 0;
  return v & ((1u << in->q) - 1);
}

static uint32_t union_rk(const bf_in* in, const uint32_t* cols) {
  uint32_t W = (1u << in->log2_eta) / 32, C = 1u << in->q, c = 0;
  for (uint32_t w = 0; w < W; ++w) {
    uint32_t a = 0xFFFFFFFFu;
    for (uint32_t i = 0; i < in->r; ++i) a &= in->bitmaps[((uint64_t)i * C + cols[i]) * W + w];
    c += (uint32_t)__builtin_popcount(a);
  }
  return c;
}

/* out: capacity cap entries of (x, rk); returns the number found (may exceed cap). */
uint64_t bf_enumerate(const bf_in* in, int verify, const uint32_t* h0_list, uint32_t n_h0,
                      uint32_t* out_x, uint32_t* out_rk, uint64_t cap) {
  uint64_t found = 0;
  uint32_t C = 1u << in->q, mask = C - 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t hi = 0; hi < 65536; ++hi) {
    uint32_t cols[16];
    for (uint32_t lo = 0; lo < 65536; ++lo) {
      uint32_t x = ((uint32_t)hi << 16) | lo;
      uint32_t best = 0;
      int ok_any = 0;
      if (verify) {
        uint32_t h = fwd_hash(in->tables + 1024, x) & mask;
        int ok = 1;
        for (uint32_t i = 0; i < in->r && ok; ++i) {
          cols[i] = i == 0 ? h : (h ^ window(in, x, i));
          ok = in->hot[(uint64_t)i * C + cols[i]];
        }
        if (ok) {
          uint32_t rk = union_rk(in, cols);
          if (rk >= in->thr) { ok_any = 1; best = rk; }
        }
      } else {
        for (uint32_t a = 0; a < n_h0; ++a) {
          uint32_t h = h0_list[a];
          int ok = 1;
          for (uint32_t i = 0; i < in->r && ok; ++i) {
            cols[i] = i == 0 ? h : (h ^ window(in, x, i));
            ok = in->hot[(uint64_t)i * C + cols[i]];
          }
          if (!ok) continue;
          uint32_t rk = union_rk(in, cols);
          if (rk >= in->thr) { ok_any = 1; if (rk > best) best = rk; }
        }
      }
      if (ok_any) {
        uint64_t at;
#pragma omp atomic capture
        at = found++;
        if (at < cap) { out_x[at] = x; out_rk[at] = best; }
      }
    }
  }
  return found;
}
