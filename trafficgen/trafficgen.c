/*
 * Seeded synthetic (cip, oip) IPv4 pair streams and hash-table draws.
 *
 * This module produces INPUTS only. It holds none of the detector's arithmetic
 * (no sliding estimator, no reversible hash, no threshold): both the CUDA
 * library and the CPU oracle consume what it writes, and neither imports the
 * other.
 *
 * The paper measures on a CAIDA core-link trace (Sec. 5), which is not
 * available here; these streams stand in for it with the same shape: IPv4
 * pairs <cip, oip> per time slot (Sec. 3.1, Def. 1-4), heavy-tailed
 * per-source peer counts, duplicate pairs, planted super points whose window
 * degree is controlled, optional hot sources (write-conflict stress) and
 * several edge routers with overlapping source sets (Sec. 4).
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) as both the sequential generator and the
 * 64-bit mixer, and the murmur3 32-bit finaliser (a bijection on uint32) for
 * distinct host addresses. Everything is integer arithmetic except the Zipf
 * and lognormal draws, which use libm in double (compiled with
 * -ffp-contract=off so x86-64 and aarch64 agree).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TG_API __attribute__((visibility("default")))

typedef struct tg_config {
  uint64_t seed;
  uint32_t routers;      /* edge routers (>= 1) */
  uint32_t n_src;        /* background sources */
  double zipf_s;         /* exponent of the truncated discrete Zipf degree law */
  uint32_t deg_cap;      /* degree cap of background sources */
  double rho;            /* probability that a packet repeats an earlier pair of its slot */
  uint32_t n_planted;    /* planted super points */
  uint32_t planted_lo;   /* planted target window degree, uniform in [lo, hi] */
  uint32_t planted_hi;
  uint32_t k;            /* window length used to pace planted peers (D/k per active slot) */
  uint32_t planted_mode; /* 0: active in every slot; 1: periodic on/off activity */
  uint32_t n_hot;        /* hot sources (each takes hot_frac of a router-slot) */
  double hot_frac;
  uint32_t hot_peers;    /* peers per hot source */
  double shared_frac;    /* fraction of sources present at 2..4 routers */
  uint32_t count_mode;   /* 0 fixed, 1 lognormal, 2 uniform [a, b], 3 even split of total a */
  uint64_t count_a;
  uint64_t count_b;
  double ln_mu;
  double ln_sigma;
} tg_config;

typedef struct tg_alias {
  uint32_t n;
  uint64_t total;   /* sum of weights (each bucket holds `total` units) */
  uint32_t* item;   /* source index of bucket i */
  uint64_t* cut;    /* threshold in [0, total] */
  uint32_t* alias;  /* alternative source index of bucket i */
} tg_alias;

typedef struct tg_state {
  tg_config c;
  uint32_t ipkey;
  uint32_t* deg;      /* [n_src] background degree */
  uint32_t* pdeg;     /* [n_planted] planted target degree */
  uint32_t* pper;     /* [n_planted] activity period (mode 1) */
  uint32_t* pon;      /* [n_planted] active slots per period */
  uint32_t* pphase;   /* [n_planted] phase */
  tg_alias* alias;    /* [routers] */
} tg_state;

enum {
  TAG_IP = 1, TAG_DEG = 2, TAG_SHARE = 3, TAG_SLOT = 4, TAG_BGPEER = 5, TAG_PLPEER = 6,
  TAG_PLROUTE = 7, TAG_PLDEG = 8, TAG_PLACT = 9, TAG_HOTPEER = 10, TAG_COUNT = 11
};

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t sm64_next(uint64_t* s) {
  *s += 0x9E3779B97F4A7C15ull;
  return mix64(*s);
}
static inline uint64_t key3(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b) {
  return mix64(mix64(mix64(seed + tag * 0x9E3779B97F4A7C15ull) ^ a) ^ b);
}
static inline uint32_t fmix32(uint32_t h) {
  h ^= h >> 16; h *= 0x85EBCA6Bu;
  h ^= h >> 13; h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}
/* uniform integer in [0, n) by 64x64 -> high 64 multiply */
static inline uint64_t below(uint64_t x, uint64_t n) {
  return (uint64_t)(((unsigned __int128)x * n) >> 64);
}
static inline double unit53(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Hash tables for the two simple-tabulation hashes, drawn from splitmix64(seed):
 * words 0..1023 = table set 1 (T0..T3, 256 each), words 1024..2047 = table set 2. */
TG_API void tg_hash_tables(uint64_t seed, uint32_t* out) {
  uint64_t s = seed;
  for (int i = 0; i < 2048; ++i) out[i] = (uint32_t)sm64_next(&s);
}

static int alias_build(tg_alias* a, const uint32_t* items, const uint64_t* w, uint32_t n) {
  a->n = n;
  a->item = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  a->cut = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
  a->alias = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!a->item || !a->cut || !a->alias) return -1;
  uint64_t total = 0;
  for (uint32_t i = 0; i < n; ++i) total += w[i];
  a->total = total;
  if (n == 0) return 0;
  /* Vose's alias method in exact integers: bucket units scaled by n. */
  uint64_t* sc = (uint64_t*)malloc(sizeof(uint64_t) * n);
  uint32_t* small = (uint32_t*)malloc(sizeof(uint32_t) * n);
  uint32_t* large = (uint32_t*)malloc(sizeof(uint32_t) * n);
  if (!sc || !small || !large) return -1;
  uint32_t ns = 0, nl = 0;
  for (uint32_t i = 0; i < n; ++i) {
    sc[i] = w[i] * (uint64_t)n;
    if (sc[i] < total) small[ns++] = i; else large[nl++] = i;
  }
  while (ns && nl) {
    uint32_t s = small[--ns], l = large[nl - 1];
    a->item[s] = items[s];
    a->cut[s] = sc[s];
    a->alias[s] = items[l];
    sc[l] -= total - sc[s];
    if (sc[l] < total) { --nl; small[ns++] = l; }
  }
  while (nl) { uint32_t l = large[--nl]; a->item[l] = items[l]; a->cut[l] = total; a->alias[l] = items[l]; }
  while (ns) { uint32_t s = small[--ns]; a->item[s] = items[s]; a->cut[s] = total; a->alias[s] = items[s]; }
  free(sc); free(small); free(large);
  return 0;
}

static inline uint32_t alias_draw(const tg_alias* a, uint64_t* rs) {
  uint64_t b = below(sm64_next(rs), a->n);
  uint64_t u = below(sm64_next(rs), a->total);
  return u < a->cut[b] ? a->item[b] : a->alias[b];
}

TG_API void tg_free(tg_state* st) {
  if (!st) return;
  free(st->deg); free(st->pdeg); free(st->pper); free(st->pon); free(st->pphase);
  if (st->alias) {
    for (uint32_t r = 0; r < st->c.routers; ++r) {
      free(st->alias[r].item); free(st->alias[r].cut); free(st->alias[r].alias);
    }
    free(st->alias);
  }
  free(st);
}

TG_API int tg_setup(const tg_config* cfg, tg_state** out) {
  *out = NULL;
  if (!cfg || cfg->routers == 0 || cfg->k == 0) return -1;
  if ((uint64_t)cfg->n_src + cfg->n_planted + cfg->n_hot >= 0xFFFFFFFFull) return -1;
  if (cfg->n_src && cfg->deg_cap == 0) return -1;
  if (cfg->n_hot && cfg->hot_peers == 0) return -1;
  if (cfg->planted_hi < cfg->planted_lo) return -1;
  tg_state* st = (tg_state*)calloc(1, sizeof(tg_state));
  if (!st) return -2;
  st->c = *cfg;
  st->ipkey = (uint32_t)key3(cfg->seed, TAG_IP, 0, 0);
  uint32_t n = cfg->n_src;
  st->deg = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!st->deg) { tg_free(st); return -2; }
  if (n) {
    /* truncated discrete Zipf on [1, cap]: inverse CDF */
    double* cdf = (double*)malloc(sizeof(double) * cfg->deg_cap);
    double z = 0.0;
    for (uint32_t d = 1; d <= cfg->deg_cap; ++d) { z += pow((double)d, -cfg->zipf_s); cdf[d - 1] = z; }
    for (uint32_t d = 0; d < cfg->deg_cap; ++d) cdf[d] /= z;
    for (uint32_t s = 0; s < n; ++s) {
      double u = unit53(key3(cfg->seed, TAG_DEG, s, 0));
      uint32_t lo = 0, hi = cfg->deg_cap - 1;
      while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (u < cdf[mid]) hi = mid; else lo = mid + 1; }
      st->deg[s] = lo + 1;
    }
    free(cdf);
  }
  uint32_t P = cfg->n_planted;
  st->pdeg = (uint32_t*)malloc(sizeof(uint32_t) * (P ? P : 1));
  st->pper = (uint32_t*)malloc(sizeof(uint32_t) * (P ? P : 1));
  st->pon = (uint32_t*)malloc(sizeof(uint32_t) * (P ? P : 1));
  st->pphase = (uint32_t*)malloc(sizeof(uint32_t) * (P ? P : 1));
  if (!st->pdeg || !st->pper || !st->pon || !st->pphase) { tg_free(st); return -2; }
  for (uint32_t p = 0; p < P; ++p) {
    uint64_t span = (uint64_t)cfg->planted_hi - cfg->planted_lo + 1;
    st->pdeg[p] = cfg->planted_lo + (uint32_t)below(key3(cfg->seed, TAG_PLDEG, p, 0), span);
    uint32_t k = cfg->k;
    st->pper[p] = 2 * k + (uint32_t)below(key3(cfg->seed, TAG_PLACT, p, 1), 2 * (uint64_t)k + 1);
    st->pon[p] = (k + 1) / 2 + (uint32_t)below(key3(cfg->seed, TAG_PLACT, p, 2), (uint64_t)k + 1);
    st->pphase[p] = (uint32_t)below(key3(cfg->seed, TAG_PLACT, p, 3), st->pper[p]);
  }
  /* per-router alias tables over the sources present there, weight deg*12/m */
  uint32_t R = cfg->routers;
  st->alias = (tg_alias*)calloc(R, sizeof(tg_alias));
  if (!st->alias) { tg_free(st); return -2; }
  uint32_t* cnt = (uint32_t*)calloc(R, sizeof(uint32_t));
  uint8_t* m = (uint8_t*)malloc(n ? n : 1);
  uint32_t* base = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!cnt || !m || !base) { tg_free(st); return -2; }
  for (uint32_t s = 0; s < n; ++s) {
    uint32_t mm = 1;
    if (R > 1 && unit53(key3(cfg->seed, TAG_SHARE, s, 0)) < cfg->shared_frac)
      mm = 2 + (uint32_t)below(key3(cfg->seed, TAG_SHARE, s, 1), 3);
    if (mm > R) mm = R;
    m[s] = (uint8_t)mm;
    base[s] = (uint32_t)below(key3(cfg->seed, TAG_SHARE, s, 2), R);
    for (uint32_t j = 0; j < mm; ++j) cnt[(base[s] + j) % R]++;
  }
  for (uint32_t r = 0; r < R; ++r) {
    uint32_t* items = (uint32_t*)malloc(sizeof(uint32_t) * (cnt[r] ? cnt[r] : 1));
    uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * (cnt[r] ? cnt[r] : 1));
    uint32_t f = 0;
    for (uint32_t s = 0; s < n; ++s) {
      uint32_t mm = m[s];
      uint32_t off = (r + R - base[s]) % R;
      if (off < mm) { items[f] = s; w[f] = (uint64_t)st->deg[s] * 12u / mm; ++f; }
    }
    int rc = alias_build(&st->alias[r], items, w, f);
    free(items); free(w);
    if (rc) { free(cnt); free(m); free(base); tg_free(st); return -2; }
  }
  free(cnt); free(m); free(base);
  *out = st;
  return 0;
}

TG_API uint32_t tg_src_ip(const tg_state* st, uint32_t s) { return fmix32(s ^ st->ipkey); }
TG_API uint32_t tg_planted_ip(const tg_state* st, uint32_t p) { return fmix32((st->c.n_src + p) ^ st->ipkey); }
TG_API uint32_t tg_hot_ip(const tg_state* st, uint32_t h) {
  return fmix32((st->c.n_src + st->c.n_planted + h) ^ st->ipkey);
}
TG_API uint32_t tg_planted_degree(const tg_state* st, uint32_t p) { return st->pdeg[p]; }
TG_API uint32_t tg_src_degree(const tg_state* st, uint32_t s) { return st->deg[s]; }

TG_API int tg_planted_active(const tg_state* st, uint32_t p, uint32_t t) {
  if (st->c.planted_mode == 0) return 1;
  return ((t + st->pphase[p]) % st->pper[p]) < st->pon[p];
}

/* packets in router-slot (t, router) */
TG_API uint64_t tg_count(const tg_state* st, uint32_t t, uint32_t router) {
  const tg_config* c = &st->c;
  switch (c->count_mode) {
    case 0: return c->count_a;
    case 1: {
      uint64_t a = key3(c->seed, TAG_COUNT, t, router);
      double u1 = (unit53(a) + 0x1p-54), u2 = unit53(mix64(a));
      double zz = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
      double v = exp(c->ln_mu + c->ln_sigma * zz);
      if (v > 4.0e9) v = 4.0e9;
      return (uint64_t)llround(v);
    }
    case 2: {
      uint64_t span = c->count_b - c->count_a + 1;
      return c->count_a + below(key3(c->seed, TAG_COUNT, t, router), span);
    }
    case 3: {
      uint64_t q = c->count_a / c->routers, rem = c->count_a % c->routers;
      return q + (router == 0 ? rem : 0);
    }
  }
  return 0;
}

/* j-th peer of a host: a bijection of j, so one host's peers are all distinct */
static inline uint32_t peer_of(uint64_t seed, uint64_t tag, uint64_t host, uint32_t j) {
  uint32_t k1 = (uint32_t)key3(seed, tag, host, 0), k2 = (uint32_t)key3(seed, tag, host, 1);
  return fmix32(fmix32(j ^ k1) + k2);
}

static inline uint32_t planted_router(const tg_state* st, uint32_t p, uint32_t j) {
  if (st->c.routers == 1) return 0;
  return (uint32_t)below(key3(st->c.seed, TAG_PLROUTE, p, j), st->c.routers);
}

/* Fill router-slot (t, router) with n pairs: out[2i] = cip, out[2i+1] = oip. */
TG_API int tg_fill(const tg_state* st, uint32_t t, uint32_t router, uint32_t* out, uint64_t n) {
  const tg_config* c = &st->c;
  if (router >= c->routers) return -1;
  uint64_t rs = key3(c->seed, TAG_SLOT, t, router);
  uint64_t pos = 0;
  /* planted super points: D/k fresh peers per active slot, cycling a list of D peers,
   * each peer always routed through the same edge router */
  for (uint32_t p = 0; p < c->n_planted && pos < n; ++p) {
    if (!tg_planted_active(st, p, t)) continue;
    uint32_t D = st->pdeg[p];
    uint64_t mq = ((uint64_t)D + c->k - 1) / c->k;
    uint32_t ip = tg_planted_ip(st, p);
    for (uint64_t j = 0; j < mq && pos < n; ++j) {
      uint32_t idx = (uint32_t)(((uint64_t)t * mq + j) % D);
      if (planted_router(st, p, idx) != router) continue;
      out[2 * pos] = ip;
      out[2 * pos + 1] = peer_of(c->seed, TAG_PLPEER, p, idx);
      ++pos;
    }
  }
  /* hot sources */
  for (uint32_t h = 0; h < c->n_hot && pos < n; ++h) {
    uint64_t cnt = (uint64_t)floor(c->hot_frac * (double)n);
    uint32_t ip = tg_hot_ip(st, h);
    for (uint64_t j = 0; j < cnt && pos < n; ++j) {
      uint64_t pe = below(sm64_next(&rs), c->hot_peers);
      out[2 * pos] = ip;
      out[2 * pos + 1] = peer_of(c->seed, TAG_HOTPEER, h, (uint32_t)pe);
      ++pos;
    }
  }
  /* background: repeats of earlier background pairs of this router-slot, else fresh draws */
  uint64_t rho_cut = (uint64_t)(c->rho * 18446744073709551616.0);
  if (c->rho >= 1.0) rho_cut = UINT64_MAX;
  const tg_alias* al = &st->alias[router];
  const uint64_t bg0 = pos;
  for (uint64_t i = pos; i < n; ++i) {
    uint64_t u = sm64_next(&rs);
    if ((i > bg0 && u < rho_cut) || al->n == 0) {
      if (i == bg0) { out[2 * i] = 0; out[2 * i + 1] = 0; continue; }
      uint64_t j = bg0 + below(sm64_next(&rs), i - bg0);
      out[2 * i] = out[2 * j];
      out[2 * i + 1] = out[2 * j + 1];
    } else {
      uint32_t s = alias_draw(al, &rs);
      uint64_t pe = below(sm64_next(&rs), st->deg[s]);
      out[2 * i] = tg_src_ip(st, s);
      out[2 * i + 1] = peer_of(c->seed, TAG_BGPEER, s, (uint32_t)pe);
    }
  }
  /* Fisher-Yates shuffle so planted and hot pairs are spread through the slot */
  for (uint64_t i = n; i > 1; --i) {
    uint64_t j = below(sm64_next(&rs), i);
    uint32_t a0 = out[2 * (i - 1)], a1 = out[2 * (i - 1) + 1];
    out[2 * (i - 1)] = out[2 * j]; out[2 * (i - 1) + 1] = out[2 * j + 1];
    out[2 * j] = a0; out[2 * j + 1] = a1;
  }
  return 0;
}

typedef struct {
  const tg_state* st;
  const uint32_t* slots;
  const uint32_t* routers;
  const uint64_t* counts;
  uint32_t* const* outs;
  uint64_t njobs;
  uint64_t next;
  pthread_mutex_t mu;
  int rc;
} tg_batch;

static void* batch_worker(void* arg) {
  tg_batch* b = (tg_batch*)arg;
  for (;;) {
    pthread_mutex_lock(&b->mu);
    uint64_t j = b->next++;
    pthread_mutex_unlock(&b->mu);
    if (j >= b->njobs) break;
    int rc = tg_fill(b->st, b->slots[j], b->routers[j], b->outs[j], b->counts[j]);
    if (rc) { pthread_mutex_lock(&b->mu); b->rc = rc; pthread_mutex_unlock(&b->mu); }
  }
  return NULL;
}

/* Fill many router-slots in parallel (jobs are independent). */
TG_API int tg_fill_batch(const tg_state* st, const uint32_t* slots, const uint32_t* routers,
                         const uint64_t* counts, uint32_t* const* outs, uint64_t njobs, int nthreads) {
  tg_batch b;
  b.st = st; b.slots = slots; b.routers = routers; b.counts = counts; b.outs = outs;
  b.njobs = njobs; b.next = 0; b.rc = 0;
  pthread_mutex_init(&b.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > njobs) nthreads = (int)(njobs ? njobs : 1);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  int started = 0;
  for (int i = 0; i < nthreads; ++i)
    if (pthread_create(&th[i], NULL, batch_worker, &b) == 0) ++started;
  if (started == 0) batch_worker(&b);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
  pthread_mutex_destroy(&b.mu);
  return b.rc;
}
