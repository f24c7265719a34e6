/*
 * CPU ORACLE for sliding super point detection (arXiv 1803.11036).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no code, header, table or constant generator
 * with the CUDA library; both take the same seeded inputs (packet pairs and
 * hash tables) from the separate input generator.
 *
 * Plain, slow, single-threaded C that follows the paper step by step:
 *   Part 1 - the precise algorithm (Sec. 3.2, Def. 1-4): exact distinct
 *            opposite-point counting per sliding window.
 *   Part 2 - the literal sketch: sliding estimator (Sec. 3.2), reversible hash
 *            functions group RHFG (Eq. 2-3), RSEA update (Algorithm 2),
 *            distance recorder update (Sec. 4.3), merge (Algorithm 5 with
 *            UnionSE, Algorithm 1), hot estimators (Sec. 3.3), and regaining
 *            sliding super points both recursively (Algorithms 3-4) and level
 *            by level (Algorithms 6-7), plus a monotone-pruned level-wise form
 *            for workloads too large for the literal product.
 *
 * Readings of points the paper leaves open (each is named where it is used):
 *   R1 merge takes the elementwise MIN of distance recorders (the union of
 *      "distance to the nearest slot"); the reconstruction check keeps
 *      Algorithm 1's literal MAX. ORC_MAX_MERGE selects the literal max merge.
 *   R2 Eq. 2 shifts by (i-1)*delta for i >= 1, the only shift for which the
 *      stated coverage condition (r-2)*delta+q >= 32 makes every bit of cip
 *      appear in some B(i). ORC_RHFG_LITERAL takes Eq. 2 as printed, a shift of
 *      i*delta: no window holds bits 0..delta-1, so a tuple fixes only bits
 *      delta..31 and the regain tries the 2^delta completions, keeping those
 *      whose RHFG[0] is he_0 (the only data that pins the missing bits).
 *   R3 the overlap test on adding row i compares the high q-delta bits of
 *      B(i-1) with the low q-delta bits of B(i), B(j) = he_0 XOR he_j.
 *   R4 a tuple is finished when it holds r estimators (rows 0..r-1).
 *   R5 the regained host is the 32-bit value whose q-bit windows are
 *      B(1..r-1); a tuple with no such value (a window bit beyond bit 31 set)
 *      yields no host.
 *   R6 ORC_VERIFY_H0 additionally requires RHFG[0](cip) == he_0 (off by
 *      default, as in the paper).
 *   R7 an estimator is hot when R_k >= ceil(R^_k), R^_k = eta*(1-exp(-theta/eta))
 *      evaluated once in double; R_k counts recorders with value < k.
 *   R8 a host regained by several tuples is listed once, with the largest R_k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))
#define ORC_MAX_R 16
#define ORC_VERIFY_H0 1u
#define ORC_MAX_MERGE 2u
#define ORC_RHFG_LITERAL 4u

typedef struct orc_params {
  uint32_t log2_eta, q, r, delta, k, theta, flags;
} orc_params;

/* ------------------------------------------------------------------ checks */

ORC_API int orc_threshold(uint32_t eta, uint32_t theta, uint32_t* thr, double* rhat);

/* Parameter constraints stated in the paper: delta < q and (r-2)*delta + q >= 32
 * (Eq. 2-3), k < 65535 (Sec. 3.2: a distance recorder is an unsigned short).
 * log2_eta and q are bounded so the arrays stay addressable, and the threshold
 * must round robustly (R7). */
ORC_API int orc_check_params(const orc_params* p) {
  if (p->r < 3 || p->r > ORC_MAX_R) return -1;
  if (p->delta == 0 || p->delta >= p->q || p->q > 24) return -1;
  if ((p->r - 2) * p->delta + p->q < 32) return -1;
  if (p->log2_eta < 1 || p->log2_eta > 15) return -1;
  if (p->k < 1 || p->k > 65534) return -1;
  if (p->theta < 1) return -1;
  uint32_t thr;
  if (orc_threshold(1u << p->log2_eta, p->theta, &thr, NULL)) return -1;
  return 0;
}

/* Hot-estimator threshold (Sec. 3.3): R^_k = eta * (1 - e^(-theta/eta)); an
 * estimator is hot when its integer R_k is at least R^_k, i.e. R_k >= ceil(R^_k)
 * (R7). Returns -1 when R^_k lies within 1e-9 of an integer, where the
 * rounding decision would not be robust. */
ORC_API int orc_threshold(uint32_t eta, uint32_t theta, uint32_t* thr, double* rhat) {
  double e = (double)eta;
  double v = e * (1.0 - exp(-(double)theta / e));
  if (rhat) *rhat = v;
  if (fabs(v - nearbyint(v)) < 1e-9) return -1;
  *thr = (uint32_t)ceil(v);
  return 0;
}

/* Eq. 1 (linear counting): estimate from z0 zero bits of eta; for the sliding
 * estimator z0 = eta - R_k. Display only. */
ORC_API double orc_estimate(uint32_t eta, uint32_t rk) {
  double e = (double)eta;
  double z0 = e - (double)rk;
  if (z0 <= 0.0) return INFINITY;
  return -e * log(z0 / e);
}

/* ------------------------------------------------------------------ hashes */

/* Simple tabulation hashing (the paper's H1 and RHFG[0] cite it): four tables
 * of 256 words indexed by the four bytes of x, XORed. */
static uint32_t tabulation(const uint32_t* T, uint32_t x) {
  uint32_t b0 = x % 256u, b1 = (x / 256u) % 256u, b2 = (x / 65536u) % 256u, b3 = x / 16777216u;
  return T[b0] ^ T[256 + b1] ^ T[512 + b2] ^ T[768 + b3];
}

/* H1: oip -> distance recorder index in [0, eta) (Sec. 3.2, Algorithm 2). */
ORC_API uint32_t orc_h1(const orc_params* p, const uint32_t* tables, uint32_t oip) {
  uint32_t eta = 1u << p->log2_eta;
  return tabulation(tables, oip) % eta;
}

/* The shift of window B(i), i >= 1: (i-1)*delta (R2), or i*delta as Eq. 2 prints it. */
static uint32_t window_shift(const orc_params* p, uint32_t i) {
  return (i - 1 + ((p->flags & ORC_RHFG_LITERAL) ? 1u : 0u)) * p->delta;
}

/* RHFG (Eq. 2 with reading R2): RHFG[0](cip) = random hash mod 2^q;
 * RHFG[i](cip) = ((cip >> ((i-1)*delta)) XOR RHFG[0](cip)) mod 2^q. */
ORC_API void orc_rhfg(const orc_params* p, const uint32_t* tables, uint32_t cip, uint32_t* cols) {
  uint32_t C = 1u << p->q;
  uint32_t h0 = tabulation(tables + 1024, cip) % C;
  cols[0] = h0;
  for (uint32_t i = 1; i < p->r; ++i) {
    uint32_t shift = window_shift(p, i);
    uint32_t shifted = shift < 32 ? (cip >> shift) : 0u;
    cols[i] = (shifted ^ h0) % C;
  }
}

/* B(i) window of cip (Eq. 3): q successive bits starting at bit (i-1)*delta. */
static uint32_t window_of(const orc_params* p, uint32_t cip, uint32_t i) {
  uint32_t shift = window_shift(p, i);
  uint32_t shifted = shift < 32 ? (cip >> shift) : 0u;
  return shifted % (1u << p->q);
}

/* Regain a host from a full tuple of columns (R5): B(i) = he_0 XOR he_i
 * (Eq. 3); each bit b of cip is read from the first window B(i) that holds it,
 * then every window of the result must equal B(i). Returns 0 and sets *cip,
 * or -1 when no 32-bit value has these windows. With ORC_RHFG_LITERAL the bits
 * no window holds (0..delta-1) are left 0 for the caller to complete. */
ORC_API int orc_extract(const orc_params* p, const uint32_t* tuple, uint32_t* cip) {
  uint32_t B[ORC_MAX_R];
  for (uint32_t i = 1; i < p->r; ++i) B[i] = tuple[0] ^ tuple[i];
  uint32_t x = 0;
  for (uint32_t b = 0; b < 32; ++b) {
    int found = 0;
    for (uint32_t i = 1; i < p->r && !found; ++i) {
      uint32_t lo = window_shift(p, i);
      if (b >= lo && b < lo + p->q) {
        if ((B[i] >> (b - lo)) & 1u) x |= 1u << b;
        found = 1;
      }
    }
    if (!found && !((p->flags & ORC_RHFG_LITERAL) && b < p->delta)) return -1;
  }
  for (uint32_t i = 1; i < p->r; ++i)
    if (window_of(p, x, i) != B[i]) return -1;
  *cip = x;
  return 0;
}

/* --------------------------------------------------------------- the RSEA */

static uint64_t n_recorders(const orc_params* p) {
  return (uint64_t)p->r * ((uint64_t)1 << p->q) * ((uint64_t)1 << p->log2_eta);
}

static uint16_t* se_ptr(const orc_params* p, uint16_t* sk, uint32_t row, uint32_t col) {
  uint64_t C = (uint64_t)1 << p->q, eta = (uint64_t)1 << p->log2_eta;
  return sk + ((uint64_t)row * C + col) * eta;
}

ORC_API uint64_t orc_sketch_len(const orc_params* p) { return n_recorders(p); }

/* Every distance recorder starts at its largest value, 65535 (Sec. 3.2). */
ORC_API void orc_sketch_init(const orc_params* p, uint16_t* sk) {
  uint64_t n = n_recorders(p);
  for (uint64_t i = 0; i < n; ++i) sk[i] = 65535;
}

/* Algorithm 2 (Update RSEA), once per pair in order: DRidx = H1(oip); for every
 * row i, the estimator RSEA[i, RHFG[i](cip)] has recorder DRidx set to 0.
 * pairs[2m] = cip, pairs[2m+1] = oip. */
ORC_API void orc_scan(const orc_params* p, const uint32_t* tables, uint16_t* sk,
                      const uint32_t* pairs, uint64_t n) {
  uint32_t cols[ORC_MAX_R];
  for (uint64_t m = 0; m < n; ++m) {
    uint32_t cip = pairs[2 * m], oip = pairs[2 * m + 1];
    uint32_t dr = orc_h1(p, tables, oip);
    orc_rhfg(p, tables, cip, cols);
    for (uint32_t i = 0; i < p->r; ++i) {
      uint16_t* se = se_ptr(p, sk, i, cols[i]);
      se[dr] = 0;
    }
  }
}

/* Distance recorder update (Sec. 3.2 and Sec. 4.3): every recorder below 65535
 * grows by one when the window slides one slot. */
ORC_API void orc_advance(const orc_params* p, uint16_t* sk) {
  uint64_t n = n_recorders(p);
  for (uint64_t i = 0; i < n; ++i)
    if (sk[i] < 65535) sk[i] = (uint16_t)(sk[i] + 1);
}

/* Algorithm 5 (merge RSEA): GRSEA[row, col] = UnionSE over the routers'
 * RSEA[row, col], recorder by recorder. R1: elementwise minimum by default,
 * Algorithm 1's literal maximum with ORC_MAX_MERGE. */
ORC_API void orc_merge(const orc_params* p, const uint16_t* const* routers, int n, uint16_t* out) {
  uint64_t len = n_recorders(p);
  int use_max = (p->flags & ORC_MAX_MERGE) != 0;
  for (uint64_t i = 0; i < len; ++i) {
    uint16_t v = use_max ? 0 : 65535;
    for (int j = 0; j < n; ++j) {
      uint16_t x = routers[j][i];
      if (use_max ? (x > v) : (x < v)) v = x;
    }
    out[i] = v;
  }
}

/* R_k of one estimator: recorders whose value is smaller than k (Sec. 3.2). */
static uint32_t rk_of(const orc_params* p, const uint16_t* se) {
  uint32_t eta = 1u << p->log2_eta, c = 0;
  for (uint32_t j = 0; j < eta; ++j)
    if (se[j] < p->k) ++c;
  return c;
}

ORC_API void orc_rk_row(const orc_params* p, const uint16_t* sk, uint32_t row, uint32_t* rk_out) {
  uint32_t C = 1u << p->q;
  for (uint32_t c = 0; c < C; ++c) rk_out[c] = rk_of(p, se_ptr(p, (uint16_t*)sk, row, c));
}

/* HSE(row): columns whose estimator is hot (Sec. 3.3, R7), ascending. */
ORC_API uint32_t orc_hse(const orc_params* p, const uint16_t* sk, uint32_t row, uint32_t* cols_out) {
  uint32_t thr;
  if (orc_threshold(1u << p->log2_eta, p->theta, &thr, NULL)) return 0;
  uint32_t C = 1u << p->q, n = 0;
  for (uint32_t c = 0; c < C; ++c)
    if (rk_of(p, se_ptr(p, (uint16_t*)sk, row, c)) >= thr) cols_out[n++] = c;
  return n;
}

/* --------------------------------------------------------- regain helpers */

typedef struct {
  uint64_t* v;
  uint64_t n, cap;
} u64vec;

static int vpush(u64vec* a, uint64_t x) {
  if (a->n == a->cap) {
    uint64_t nc = a->cap ? a->cap * 2 : 1024;
    uint64_t* nv = (uint64_t*)realloc(a->v, nc * sizeof(uint64_t));
    if (!nv) return -1;
    a->v = nv; a->cap = nc;
  }
  a->v[a->n++] = x;
  return 0;
}

typedef struct {
  const orc_params* p;
  const uint32_t* tables;
  uint16_t* sk;
  uint32_t thr;
  uint32_t* H[ORC_MAX_R];
  uint32_t nH[ORC_MAX_R];
  u64vec out;           /* (cip << 32) | R_k of accepted tuples */
  uint64_t level[ORC_MAX_R];
  int err;
} regain_ctx;

/* The overlap property (Sec. 3.3): the high q-delta bits of B(i-1) equal the
 * low q-delta bits of B(i); B(j) = he_0 XOR he_j (R3). */
static int overlap_ok(const orc_params* p, uint32_t he0, uint32_t he_prev, uint32_t he_new) {
  uint32_t Bprev = he0 ^ he_prev, Bnew = he0 ^ he_new;
  uint32_t w = p->q - p->delta;
  return (Bprev >> p->delta) == (Bnew % (1u << w));
}

/* Algorithm 1 (UnionSE, literal maximum) over the tuple's r estimators,
 * followed by R_k of the union (Algorithm 4). */
static uint32_t union_rk(regain_ctx* g, const uint32_t* tuple, uint32_t len) {
  const orc_params* p = g->p;
  uint32_t eta = 1u << p->log2_eta, count = 0;
  for (uint32_t j = 0; j < eta; ++j) {
    uint16_t maxV = 0;
    for (uint32_t i = 0; i < len; ++i) {
      uint16_t v = se_ptr(p, g->sk, i, tuple[i])[j];
      if (maxV < v) maxV = v;
    }
    if (maxV < p->k) ++count;
  }
  return count;
}

/* Final test of a full tuple (Algorithm 4): R_k of the union against the
 * threshold, then the host is regained from the tuple (R5, R6). */
static void finish_tuple(regain_ctx* g, const uint32_t* tuple) {
  uint32_t rk = union_rk(g, tuple, g->p->r);
  if (rk < g->thr) return;
  uint32_t cip;
  if (orc_extract(g->p, tuple, &cip)) return;
  if (g->p->flags & ORC_RHFG_LITERAL) {
    /* bits 0..delta-1 are in no window: every completion whose RHFG[0] is he_0 */
    for (uint32_t low = 0; low < (1u << g->p->delta); ++low) {
      uint32_t cols[ORC_MAX_R];
      orc_rhfg(g->p, g->tables, cip | low, cols);
      if (cols[0] == tuple[0] && vpush(&g->out, ((uint64_t)(cip | low) << 32) | rk)) g->err = 1;
    }
    return;
  }
  if (g->p->flags & ORC_VERIFY_H0) {
    uint32_t cols[ORC_MAX_R];
    orc_rhfg(g->p, g->tables, cip, cols);
    if (cols[0] != tuple[0]) return;
  }
  if (vpush(&g->out, ((uint64_t)cip << 32) | rk)) g->err = 1;
}

static int regain_setup(regain_ctx* g, const orc_params* p, const uint32_t* tables, const uint16_t* sk) {
  memset(g, 0, sizeof(*g));
  g->p = p; g->tables = tables; g->sk = (uint16_t*)sk;
  if (orc_check_params(p)) return -1;
  if (orc_threshold(1u << p->log2_eta, p->theta, &g->thr, NULL)) return -1;
  for (uint32_t i = 0; i < p->r; ++i) {
    g->H[i] = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)1 << p->q));
    if (!g->H[i]) return -2;
    g->nH[i] = orc_hse(p, sk, i, g->H[i]);
  }
  return 0;
}

static void regain_free(regain_ctx* g) {
  for (uint32_t i = 0; i < ORC_MAX_R; ++i) free(g->H[i]);
  free(g->out.v);
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y);
}

/* The sliding super point list is a set of hosts (R8): sort by cip, keep the
 * largest R_k of each. Writes at most cap entries; returns the list size. */
static int64_t emit_list(regain_ctx* g, uint32_t* ips, uint32_t* rks, uint64_t cap, uint64_t* raw) {
  if (raw) *raw = g->out.n;
  qsort(g->out.v, g->out.n, sizeof(uint64_t), cmp_u64);
  uint64_t n = 0;
  for (uint64_t i = 0; i < g->out.n; ++i) {
    uint32_t cip = (uint32_t)(g->out.v[i] >> 32), rk = (uint32_t)g->out.v[i];
    int last_of_run = (i + 1 == g->out.n) || ((uint32_t)(g->out.v[i + 1] >> 32) != cip);
    if (!last_of_run) continue;
    if (n < cap) { ips[n] = cip; rks[n] = rk; }
    ++n;
  }
  return (int64_t)n;
}

/* ------------------------------------------- Algorithms 3-4 (recursive) */

/* IRSSP (Algorithm 4): grow tuple ct (holding rows 0..i-1) with every hot
 * estimator of row i that passes the overlap test; finish at r elements (R4). */
static void irssp(regain_ctx* g, uint32_t* ct, uint32_t len, uint32_t i) {
  const orc_params* p = g->p;
  if (len < i) return;
  for (uint32_t a = 0; a < g->nH[i]; ++a) {
    uint32_t he_i = g->H[i][a];
    if (!overlap_ok(p, ct[0], ct[i - 1], he_i)) continue;
    ct[i] = he_i;
    g->level[i]++;
    if (i == p->r - 1) finish_tuple(g, ct);
    else irssp(g, ct, len + 1, i + 1);
  }
}

/* Algorithm 3: triples from HSE(0..2) passing the B(1)/B(2) overlap test,
 * each grown by IRSSP from row 3. Returns the list size (or < 0 on error). */
ORC_API int64_t orc_regain_recursive(const orc_params* p, const uint32_t* tables, const uint16_t* sk,
                                     uint32_t* ips, uint32_t* rks, uint64_t cap, uint64_t* level_counts) {
  regain_ctx g;
  int rc = regain_setup(&g, p, tables, sk);
  if (rc) { regain_free(&g); return rc; }
  uint32_t ct[ORC_MAX_R];
  for (uint32_t a = 0; a < g.nH[0]; ++a)
    for (uint32_t b = 0; b < g.nH[1]; ++b)
      for (uint32_t c = 0; c < g.nH[2]; ++c) {
        ct[0] = g.H[0][a]; ct[1] = g.H[1][b]; ct[2] = g.H[2][c];
        if (!overlap_ok(p, ct[0], ct[1], ct[2])) continue;
        g.level[2]++;
        if (p->r == 3) finish_tuple(&g, ct);
        else irssp(&g, ct, 3, 3);
      }
  g.level[1] = (uint64_t)g.nH[0] * g.nH[1];
  if (level_counts) for (uint32_t i = 0; i < p->r; ++i) level_counts[i] = i == 0 ? g.nH[0] : g.level[i];
  int64_t n = g.err ? -2 : emit_list(&g, ips, rks, cap, NULL);
  regain_free(&g);
  return n;
}

/* ------------------------------------- Algorithms 6-7 (level by level) */

typedef struct {
  uint32_t* t;   /* tuples, stride ORC_MAX_R */
  uint64_t n, cap;
} ctb;

static int ctb_push(ctb* b, const uint32_t* tuple, uint32_t len) {
  if (b->n == b->cap) {
    uint64_t nc = b->cap ? b->cap * 2 : 4096;
    uint32_t* nt = (uint32_t*)realloc(b->t, nc * ORC_MAX_R * sizeof(uint32_t));
    if (!nt) return -1;
    b->t = nt; b->cap = nc;
  }
  memcpy(b->t + b->n * ORC_MAX_R, tuple, len * sizeof(uint32_t));
  b->n++;
  return 0;
}

/* Pruned variant: a partial tuple whose union already has R_k below the
 * threshold is dropped. The union is an elementwise maximum, so R_k can only
 * fall as rows are added; every dropped tuple would fail the final test and
 * the list is unchanged. */
static int keep(regain_ctx* g, int prune, const uint32_t* tuple, uint32_t len) {
  return !prune || union_rk(g, tuple, len) >= g->thr;
}

static int64_t levelwise(const orc_params* p, const uint32_t* tables, const uint16_t* sk,
                         uint32_t* ips, uint32_t* rks, uint64_t cap, uint64_t* level_counts,
                         uint64_t* raw_out, int prune) {
  regain_ctx g;
  int rc = regain_setup(&g, p, tables, sk);
  if (rc) { regain_free(&g); return rc; }
  ctb A = {0}, Bf = {0};
  ctb* rctb = &A;
  ctb* sctb = &Bf;
  uint32_t tup[ORC_MAX_R];
  uint64_t pairs = 0;
  /* Algorithm 6: CT_2 triples from HSE(0) x HSE(1) x HSE(2) */
  for (uint32_t a = 0; a < g.nH[0] && !g.err; ++a)
    for (uint32_t b = 0; b < g.nH[1] && !g.err; ++b) {
      tup[0] = g.H[0][a]; tup[1] = g.H[1][b];
      if (!keep(&g, prune, tup, 2)) continue;
      ++pairs;
      for (uint32_t c = 0; c < g.nH[2]; ++c) {
        tup[2] = g.H[2][c];
        if (!overlap_ok(p, tup[0], tup[1], tup[2])) continue;
        if (!keep(&g, prune, tup, 3)) continue;
        if (ctb_push(rctb, tup, 3)) { g.err = 1; break; }
      }
    }
  g.level[1] = pairs;
  g.level[2] = rctb->n;
  /* Algorithm 7: rows 3..r-1, reading RCTB and storing into SCTB, roles swapped per row */
  for (uint32_t i = 3; i < p->r && !g.err; ++i) {
    sctb->n = 0;
    for (uint64_t m = 0; m < rctb->n && !g.err; ++m) {
      memcpy(tup, rctb->t + m * ORC_MAX_R, i * sizeof(uint32_t));
      for (uint32_t c = 0; c < g.nH[i]; ++c) {
        tup[i] = g.H[i][c];
        if (!overlap_ok(p, tup[0], tup[i - 1], tup[i])) continue;
        if (!keep(&g, prune, tup, i + 1)) continue;
        if (ctb_push(sctb, tup, i + 1)) { g.err = 1; break; }
      }
    }
    g.level[i] = sctb->n;
    ctb* t = rctb; rctb = sctb; sctb = t;
  }
  /* final pass over the full tuples */
  for (uint64_t m = 0; m < rctb->n && !g.err; ++m) finish_tuple(&g, rctb->t + m * ORC_MAX_R);
  if (level_counts) for (uint32_t i = 0; i < p->r; ++i) level_counts[i] = i == 0 ? g.nH[0] : g.level[i];
  int64_t n = g.err ? -2 : emit_list(&g, ips, rks, cap, raw_out);
  free(A.t); free(Bf.t);
  regain_free(&g);
  return n;
}

ORC_API int64_t orc_regain_levelwise(const orc_params* p, const uint32_t* tables, const uint16_t* sk,
                                     uint32_t* ips, uint32_t* rks, uint64_t cap, uint64_t* level_counts,
                                     uint64_t* raw_out) {
  return levelwise(p, tables, sk, ips, rks, cap, level_counts, raw_out, 0);
}

ORC_API int64_t orc_regain_pruned(const orc_params* p, const uint32_t* tables, const uint16_t* sk,
                                  uint32_t* ips, uint32_t* rks, uint64_t cap, uint64_t* level_counts,
                                  uint64_t* raw_out) {
  return levelwise(p, tables, sk, ips, rks, cap, level_counts, raw_out, 1);
}

/* ------------------------------------------- sampled estimators (full size) */

/* The same Algorithm 2 and distance recorder update restricted to a chosen set
 * of estimators, for workloads whose full RSEA is too large to hold here. */
typedef struct orc_sampled {
  orc_params p;
  uint32_t n;          /* tracked estimators */
  uint32_t* rowcol;    /* sorted keys row * 2^q + col */
  uint16_t* dr;        /* n * eta recorders */
} orc_sampled;

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return x < y ? -1 : (x > y);
}

ORC_API orc_sampled* orc_sampled_new(const orc_params* p, const uint32_t* rows, const uint32_t* cols, uint32_t n) {
  orc_sampled* s = (orc_sampled*)calloc(1, sizeof(orc_sampled));
  if (!s) return NULL;
  s->p = *p;
  s->rowcol = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  uint32_t m = 0;
  for (uint32_t i = 0; i < n; ++i) s->rowcol[i] = rows[i] * (1u << p->q) + cols[i];
  qsort(s->rowcol, n, sizeof(uint32_t), cmp_u32);
  for (uint32_t i = 0; i < n; ++i)
    if (m == 0 || s->rowcol[m - 1] != s->rowcol[i]) s->rowcol[m++] = s->rowcol[i];
  s->n = m;
  uint64_t eta = (uint64_t)1 << p->log2_eta;
  s->dr = (uint16_t*)malloc(sizeof(uint16_t) * eta * (m ? m : 1));
  if (!s->dr) { free(s->rowcol); free(s); return NULL; }
  for (uint64_t i = 0; i < eta * m; ++i) s->dr[i] = 65535;
  return s;
}

ORC_API void orc_sampled_free(orc_sampled* s) {
  if (!s) return;
  free(s->rowcol); free(s->dr); free(s);
}

static int64_t sampled_find(const orc_sampled* s, uint32_t key) {
  uint32_t lo = 0, hi = s->n;
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (s->rowcol[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < s->n && s->rowcol[lo] == key) ? (int64_t)lo : -1;
}

ORC_API void orc_sampled_scan(orc_sampled* s, const uint32_t* tables, const uint32_t* pairs, uint64_t n) {
  const orc_params* p = &s->p;
  uint32_t cols[ORC_MAX_R];
  uint64_t eta = (uint64_t)1 << p->log2_eta;
  for (uint64_t m = 0; m < n; ++m) {
    uint32_t cip = pairs[2 * m], oip = pairs[2 * m + 1];
    orc_rhfg(p, tables, cip, cols);
    uint32_t dr = orc_h1(p, tables, oip);
    for (uint32_t i = 0; i < p->r; ++i) {
      int64_t at = sampled_find(s, i * (1u << p->q) + cols[i]);
      if (at >= 0) s->dr[(uint64_t)at * eta + dr] = 0;
    }
  }
}

ORC_API void orc_sampled_advance(orc_sampled* s) {
  uint64_t len = (uint64_t)s->n << s->p.log2_eta;
  for (uint64_t i = 0; i < len; ++i)
    if (s->dr[i] < 65535) s->dr[i] = (uint16_t)(s->dr[i] + 1);
}

/* Copy the recorders of one tracked estimator; -1 if (row, col) is not tracked. */
ORC_API int orc_sampled_get(const orc_sampled* s, uint32_t row, uint32_t col, uint16_t* out) {
  int64_t at = sampled_find(s, row * (1u << s->p.q) + col);
  if (at < 0) return -1;
  uint64_t eta = (uint64_t)1 << s->p.log2_eta;
  memcpy(out, s->dr + (uint64_t)at * eta, eta * sizeof(uint16_t));
  return 0;
}

/* --------------------------------------------- Part 1: precise algorithm */

/* Exact opposite numbers under the sliding window (Def. 1-4, Sec. 3.2): the
 * last slot each <cip, oip> pair appeared in; |OP(cip, SW)| counts the pairs of
 * cip seen within the last k slots (slots 0..t while t < k-1). */
typedef struct orc_exact {
  uint64_t* key;    /* (cip << 32) | oip */
  uint32_t* last;   /* slot + 1; 0 = empty */
  uint64_t cap, used;
  uint32_t k, theta;
  int64_t t;        /* current slot, -1 before the first */
} orc_exact;

static uint64_t hash64(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
  return x;
}

ORC_API orc_exact* orc_exact_new(uint32_t k, uint32_t theta) {
  orc_exact* e = (orc_exact*)calloc(1, sizeof(orc_exact));
  if (!e) return NULL;
  e->cap = 1 << 16;
  e->key = (uint64_t*)calloc(e->cap, sizeof(uint64_t));
  e->last = (uint32_t*)calloc(e->cap, sizeof(uint32_t));
  e->k = k; e->theta = theta; e->t = -1;
  return e;
}

ORC_API void orc_exact_free(orc_exact* e) {
  if (!e) return;
  free(e->key); free(e->last); free(e);
}

static void exact_insert(orc_exact* e, uint64_t key, uint32_t lastp1);

static void exact_grow(orc_exact* e) {
  uint64_t oc = e->cap;
  uint64_t* ok = e->key;
  uint32_t* ol = e->last;
  e->cap = oc * 2;
  e->key = (uint64_t*)calloc(e->cap, sizeof(uint64_t));
  e->last = (uint32_t*)calloc(e->cap, sizeof(uint32_t));
  e->used = 0;
  for (uint64_t i = 0; i < oc; ++i)
    if (ol[i]) exact_insert(e, ok[i], ol[i]);
  free(ok); free(ol);
}

static void exact_insert(orc_exact* e, uint64_t key, uint32_t lastp1) {
  if ((e->used + 1) * 2 > e->cap) exact_grow(e);
  uint64_t mask = e->cap - 1, h = hash64(key) & mask;
  while (e->last[h] && e->key[h] != key) h = (h + 1) & mask;
  if (!e->last[h]) { e->used++; e->key[h] = key; }
  e->last[h] = lastp1;
}

/* Starts the next slot and records its pairs. */
ORC_API void orc_exact_add_slot(orc_exact* e, const uint32_t* pairs, uint64_t n) {
  e->t++;
  for (uint64_t m = 0; m < n; ++m)
    exact_insert(e, ((uint64_t)pairs[2 * m] << 32) | pairs[2 * m + 1], (uint32_t)(e->t + 1));
}

/* Drops pairs that left the window, then lists every cip with |OP| >= theta
 * (Def. 2, 4) in ascending order with its opposite number. Returns the count. */
ORC_API int64_t orc_exact_report(orc_exact* e, uint32_t* ips, uint32_t* deg, uint64_t cap) {
  int64_t lo = e->t - (int64_t)e->k + 1;
  if (lo < 0) lo = 0;
  /* rebuild the table with only in-window pairs */
  uint64_t oc = e->cap;
  uint64_t* ok = e->key;
  uint32_t* ol = e->last;
  e->key = (uint64_t*)calloc(oc, sizeof(uint64_t));
  e->last = (uint32_t*)calloc(oc, sizeof(uint32_t));
  e->used = 0;
  for (uint64_t i = 0; i < oc; ++i)
    if (ol[i] && (int64_t)ol[i] - 1 >= lo) exact_insert(e, ok[i], ol[i]);
  free(ok); free(ol);
  /* count pairs per cip by sorting the cips */
  uint64_t n = 0;
  uint32_t* cips = (uint32_t*)malloc(sizeof(uint32_t) * (e->used ? e->used : 1));
  for (uint64_t i = 0; i < e->cap; ++i)
    if (e->last[i]) cips[n++] = (uint32_t)(e->key[i] >> 32);
  qsort(cips, n, sizeof(uint32_t), cmp_u32);
  uint64_t out = 0;
  for (uint64_t i = 0; i < n;) {
    uint64_t j = i;
    while (j < n && cips[j] == cips[i]) ++j;
    if (j - i >= e->theta) {
      if (out < cap) { ips[out] = cips[i]; deg[out] = (uint32_t)(j - i); }
      ++out;
    }
    i = j;
  }
  free(cips);
  return (int64_t)out;
}

/* |OP(cip, SW)| for the current window (after orc_exact_report has pruned). */
ORC_API uint32_t orc_exact_degree(const orc_exact* e, uint32_t cip) {
  int64_t lo = e->t - (int64_t)e->k + 1;
  if (lo < 0) lo = 0;
  uint32_t c = 0;
  for (uint64_t i = 0; i < e->cap; ++i)
    if (e->last[i] && (uint32_t)(e->key[i] >> 32) == cip && (int64_t)e->last[i] - 1 >= lo) ++c;
  return c;
}

/* ------------------------------------------------ RHFG round trip (pins) */

/* Counts the x in xs[0..n) for which regaining the host from its own tuple
 * RHFG(x) (Eq. 2, then R5) does not give back x. */
ORC_API uint64_t orc_roundtrip_failures(const orc_params* p, const uint32_t* tables, const uint32_t* xs,
                                        uint64_t n) {
  uint32_t cols[ORC_MAX_R];
  uint64_t bad = 0;
  for (uint64_t m = 0; m < n; ++m) {
    uint32_t back;
    orc_rhfg(p, tables, xs[m], cols);
    if (orc_extract(p, cols, &back) || back != xs[m]) ++bad;
  }
  return bad;
}
