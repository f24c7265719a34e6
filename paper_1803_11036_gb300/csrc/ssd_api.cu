// The C ABI of include/ssd.h: parameter checks, contexts, sketches and the
// launch sequences of scan, advance, merge, regain and slot close.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "ssd_internal.cuh"

struct ssd_ctx {
  ssd_params p;
  int device;
  int sms;
  ssd::Dims d;
  ssd::Scratch s;
  uint32_t* tables;
  uint32_t* hot_idx;
  uint32_t* pool_col;
  uint32_t* pool_rk;
  uint32_t* pool_bm;
  uint32_t* ctb[2];
  unsigned long long* stage;
  ssd::DevCounters* counters;
  uint32_t* bucket_off;
  uint32_t* bucket_cnt;
  uint32_t* bucket_ent;
  unsigned long long* n_out;  // list size of ssd_regain
  uint64_t launches;
  // tracing events (caller-owned)
  cudaEvent_t tr_start, tr_pass, tr_end;
  // host-pair staging of ssd_scan_host
  uint32_t* stage_pairs[2];
  uint64_t stage_alpha;
  cudaStream_t copy_stream;
  cudaEvent_t ev_copied[2], ev_scanned[2];
  // fused slot: double-buffered touch bits and the side stream that fills them
  uint32_t* touch[2];
  uint64_t touch_bytes;
  ssd::Tuning tn;             // launch configuration (ssd_tuning_set / ssd_autotune)
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_touched[2], ev_closed[2];
  // pre-hashed pairs of the one-router fused slot (grown to the largest slot)
  uint2* packed;
  uint64_t packed_cap;
  // per-chunk touch lists of the one-router fused slot (grown to the largest slot) and their counters
  uint32_t* tl_ent;
  uint64_t tl_entries;
  uint32_t* tl_fill;
  // host-pair staging of ssd_slot_host (double-buffered, sized to the largest slot)
  uint32_t* hs_buf[2];
  uint64_t hs_bytes;
  uint64_t hs_calls;
  cudaEvent_t ev_hs_free[2], ev_hs_copied;
  uint64_t epoch;   // ssd_buffer_epoch: bumped when a buffer captured work may hold is replaced
  // debug build only: the status word of the kernels' bound checks and the candidate tuple
  // buffers' allocations with their guard words (ctb[i] = ctb_alloc[i] + kGuardWords)
  unsigned int* dbg;
  uint32_t* ctb_alloc[2];
  // staging of ssd_sketch_export / ssd_sketch_import through host memory (grown on first use)
  uint16_t* xfer;
  uint64_t xfer_count;
};

struct ssd_sketch {
  ssd_ctx* ctx;
  int device;
  uint16_t* dr;    // stamp recorders (ssd_internal.cuh), r * 2^q * eta of them
  uint32_t* tm;    // the sketch's clock, slot mod 65535, in device memory right after the recorders
  uint64_t slot;
  uint32_t view;   // ssd::view_pack(side, group bits, group)
};

namespace {

thread_local char g_cuda_err[256] = "";

// Guard words before and after each candidate tuple buffer in the debug build.
constexpr uint64_t kGuardWords = SSD_DEBUG ? 64 : 0;
constexpr uint32_t kGuard = 0xC0DEC0DEu;

int cuda_fail(cudaError_t e, const char* where) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
  return SSD_ECUDA;
}

#define SSD_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Makes ctx's device current for the duration of a call and restores the caller's.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) == cudaSuccess && prev_ != dev) changed_ = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1;
  bool changed_ = false;
};

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int threshold_of(uint32_t eta, uint32_t theta, uint32_t* thr) {
  // Sec. 3.3: an estimator is hot when R_k >= eta * (1 - e^(-theta/eta)).
  const double e = (double)eta;
  const double v = e * (1.0 - std::exp(-(double)theta / e));
  if (std::fabs(v - std::nearbyint(v)) < 1e-9) return SSD_EINVAL;
  *thr = (uint32_t)std::ceil(v);
  return SSD_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool same_ctx(ssd_sketch* const* v, int n, ssd_ctx** ctx) {
  if (!v || n < 1 || n > SSD_MAX_ROUTERS || !v[0]) return false;
  *ctx = v[0]->ctx;
  for (int i = 0; i < n; ++i)
    if (!v[i] || v[i]->ctx != *ctx) return false;
  return true;
}

// Sketches that are combined (merged) must count the same hosts.
bool same_view(ssd_sketch* const* v, int n) {
  for (int i = 1; i < n; ++i)
    if (v[i]->view != v[0]->view) return false;
  return true;
}

int add_job(ssd::ScanBatch& b, int j, const ssd_sketch* sk, const uint32_t* pairs, uint64_t n, uint64_t* prefix) {
  uint16_t* dr = sk->dr;
  b.view[j] = sk->view;
  b.tm[j] = sk->tm;
  if (n && !pairs) return SSD_EINVAL;
  if (reinterpret_cast<uintptr_t>(pairs) & 7u) return SSD_EINVAL;
  const uint32_t* head = nullptr;
  const uint32_t* body = pairs;
  uint64_t rest = n;
  if (n && (reinterpret_cast<uintptr_t>(pairs) & 15u)) {  // starts at 8 mod 16
    head = pairs;
    body = pairs + 2;
    rest = n - 1;
  }
  b.dr[j] = dr;
  b.vec[j] = reinterpret_cast<const uint4*>(body);
  b.edge[2 * j] = head;
  b.edge[2 * j + 1] = (rest & 1u) ? body + 2 * (rest - 1) : nullptr;
  b.prefix[j] = *prefix;
  *prefix += rest / 2;
  return SSD_OK;
}

// Blocks of a scan, touch or pre-hash launch over nvec pair vectors: enough for
// one step of scan_unroll vectors per thread, at most SMs x scan_blocks_per_sm.
uint64_t scan_grid(const ssd_ctx* ctx, uint64_t nvec) {
  const uint64_t per = (uint64_t)ssd::kBlock * ctx->tn.unroll;
  uint64_t grid = (nvec + per - 1) / per;
  const uint64_t cap = (uint64_t)ctx->sms * ctx->tn.scan_bps;
  if (grid > cap) grid = cap;
  return grid < 1 ? 1 : grid;
}

int scan_jobs(ssd_ctx* ctx, ssd::ScanBatch& b, uint64_t total_vec, bool any_edge, cudaStream_t st) {
  if (total_vec == 0 && !any_edge) return SSD_OK;
  cudaError_t e = ssd::launch_scan(ctx->d, ctx->tables, b, (int)scan_grid(ctx, total_vec), ctx->tn, st);
  if (e != cudaSuccess) return cuda_fail(e, "scan kernel");
  ctx->launches += 1;
  return SSD_OK;
}

int stream_pass(ssd_ctx* ctx, ssd_sketch* const* routers, int n, ssd_sketch* global, int mode, cudaStream_t st) {
  ssd::StreamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  for (int i = 0; i < n; ++i) {
    a.routers[i] = routers[i]->dr;
    a.tm[i] = routers[i]->tm;
  }
  a.global = global ? global->dr : nullptr;
  a.global_tm = global ? global->tm : nullptr;
  cudaError_t e = ssd::launch_stream(ctx->d, ctx->s, a, mode, ctx->sms, ctx->tn, st);
  if (e != cudaSuccess) return cuda_fail(e, "stream kernel");
  ctx->launches += 1;
  return SSD_OK;
}

// The clocks of advanced sketches move on by one slot, after every launch that reads them.
int tick(ssd_ctx* ctx, ssd_sketch* const* sketches, int n, cudaStream_t st) {
  ssd::TickArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  for (int i = 0; i < n; ++i) a.tm[i] = sketches[i]->tm;
  cudaError_t e = ssd::launch_tick(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "tick kernel");
  ctx->launches += 1;
  return SSD_OK;
}

// Every recorder at distance 65535 (kNever) and the clock at slot 0.
cudaError_t reset_sketch(ssd_sketch* sk, uint64_t bytes, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(sk->dr, 0xFF, bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sk->tm, 0, sizeof(uint32_t), st);
  return e;
}

// The export/import staging buffer of at least `count` recorders (at most 16 Mi), grown on demand.
int xfer_buffer(ssd_ctx* ctx, uint64_t want) {
  if (want > (1ull << 24)) want = 1ull << 24;
  if (ctx->xfer && ctx->xfer_count >= want) return SSD_OK;
  SSD_CUDA(cudaDeviceSynchronize());
  cudaFree(ctx->xfer);
  ctx->xfer = nullptr;
  ctx->xfer_count = 0;
  if (cudaMalloc(&ctx->xfer, want * 2) != cudaSuccess) {
    cudaGetLastError();
    return SSD_ENOMEM;
  }
  ctx->xfer_count = want;
  return SSD_OK;
}

// Whether p is memory a kernel of ctx's device can address directly (device or managed memory).
bool device_memory(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int trace(ssd_ctx* ctx, cudaEvent_t ev, cudaStream_t st) {
  if (!ev) return SSD_OK;
  cudaError_t e = cudaEventRecord(ev, st);
  return e == cudaSuccess ? SSD_OK : cuda_fail(e, "cudaEventRecord (trace)");
}

int regain_after_pass(ssd_ctx* ctx, uint32_t* ips, uint32_t* rk, uint64_t cap, unsigned long long* n_out,
                      cudaStream_t st, uint32_t view) {
  int launches = 0;
  cudaError_t e = ssd::launch_regain_tail(ctx->d, ctx->s, ips, rk, cap, n_out, ctx->sms, st, &launches, view,
                                          ctx->tn.pair_level == 0);
  ctx->launches += launches;
  if (e != cudaSuccess) return cuda_fail(e, "regain kernels");
  return SSD_OK;
}

void free_ctx(ssd_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_hs_copied) cudaEventDestroy(c->ev_hs_copied);
  for (int i = 0; i < 2; ++i) {
    if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
    if (c->ev_scanned[i]) cudaEventDestroy(c->ev_scanned[i]);
    if (c->ev_touched[i]) cudaEventDestroy(c->ev_touched[i]);
    if (c->ev_closed[i]) cudaEventDestroy(c->ev_closed[i]);
    cudaFree(c->stage_pairs[i]);
    cudaFree(c->touch[i]);
    if (c->ev_hs_free[i]) cudaEventDestroy(c->ev_hs_free[i]);
    cudaFree(c->hs_buf[i]);
  }
  cudaFree(c->packed);
  cudaFree(c->tl_ent);
  cudaFree(c->tl_fill);

  cudaFree(c->tables);
  cudaFree(c->hot_idx);
  cudaFree(c->pool_col);
  cudaFree(c->pool_rk);
  cudaFree(c->pool_bm);
  for (int i = 0; i < 2; ++i) cudaFree(c->ctb_alloc[i]);
  cudaFree(c->dbg);
  cudaFree(c->stage);
  cudaFree(c->counters);
  cudaFree(c->bucket_off);
  cudaFree(c->bucket_cnt);
  cudaFree(c->bucket_ent);
  cudaFree(c->n_out);
  cudaFree(c->xfer);
  delete c;
}

}  // namespace

extern "C" {

int ssd_version(void) { return 103; }

const char* ssd_strerror(int code) {
  switch (code) {
    case SSD_OK: return "ok";
    case SSD_EINVAL: return "invalid argument or parameter set";
    case SSD_ENOMEM: return "device memory allocation failed";
    case SSD_ECAPACITY: return "a capacity was exceeded";
    case SSD_ECUDA: return "CUDA error";
    case SSD_ETIMEOUT: return "device-side wait timed out";
    case SSD_ESTATE: return "sketches disagree on their slot or context";
    default: return "unknown error";
  }
}

const char* ssd_last_cuda_error(void) { return g_cuda_err; }

int ssd_params_check(const ssd_params* p) {
  if (!p) return SSD_EINVAL;
  if (p->log2_eta < 5 || p->log2_eta > 15) return SSD_EINVAL;
  if (p->r < 3 || p->r > SSD_MAX_R) return SSD_EINVAL;
  if (p->delta == 0 || p->delta >= p->q || p->q > 24) return SSD_EINVAL;
  if ((p->r - 2) * p->delta + p->q < 32) return SSD_EINVAL;  // Eq. 2-3: every bit of cip in some B(i)
  if (p->k < 1 || p->k > 65534) return SSD_EINVAL;            // Sec. 3.2: k < 65535
  if (p->theta < 1) return SSD_EINVAL;
  if (p->flags & ~(SSD_VERIFY_H0 | SSD_NO_PRUNE | SSD_SLOT_CHUNKED | SSD_RHFG_LITERAL)) return SSD_EINVAL;
  if (p->ctb_capacity > (1ull << 32) || p->out_capacity > (1ull << 28)) return SSD_EINVAL;
  uint32_t thr;
  return threshold_of(1u << p->log2_eta, p->theta, &thr);
}

int ssd_threshold(const ssd_params* p, uint32_t* thr) {
  if (!p || !thr) return SSD_EINVAL;
  return threshold_of(1u << p->log2_eta, p->theta, thr);
}

int ssd_create(const ssd_params* p, const uint32_t* tables, int device, ssd_ctx** out) {
  if (!out) return SSD_EINVAL;
  *out = nullptr;
  if (!tables || ssd_params_check(p) != SSD_OK) return SSD_EINVAL;
  int ndev = 0;
  SSD_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return SSD_EINVAL;
  DeviceGuard g(device);
  ssd_ctx* c = new (std::nothrow) ssd_ctx;
  if (!c) return SSD_ENOMEM;
  std::memset(c, 0, sizeof(*c));
  c->p = *p;
  c->device = device;
  c->tn = ssd::default_tuning();
  cudaError_t e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "cudaDeviceGetAttribute"); }

  ssd::Dims& d = c->d;
  d.log2_eta = p->log2_eta; d.q = p->q; d.r = p->r; d.delta = p->delta; d.k = p->k; d.flags = p->flags;
  threshold_of(1u << p->log2_eta, p->theta, &d.thr);
  d.eta = 1u << p->log2_eta;
  d.words = d.eta / 32;
  d.col_mask = (1u << p->q) - 1u;
  d.low_bits = p->q - p->delta;
  d.low_mask = (1u << d.low_bits) - 1u;
  d.sh0 = (p->flags & SSD_RHFG_LITERAL) ? p->delta : 0u;
  const uint64_t C = 1ull << p->q;
  d.hse_cap = p->hse_capacity ? p->hse_capacity : (uint32_t)(C < 65536 ? C : 65536);
  if (d.hse_cap > C) d.hse_cap = (uint32_t)C;
  d.ctb_cap = p->ctb_capacity ? p->ctb_capacity : (1ull << 22);
  d.out_cap = pow2_at_least(p->out_capacity ? p->out_capacity : (1ull << 20));

  const uint64_t R = p->r;
  const uint64_t NB = d.low_bits <= ssd::kMaxBucketBits ? (1ull << d.low_bits) : 0;  // 0: no bucket index
  c->touch_bytes = p->touch_chunk_bytes ? p->touch_chunk_bytes : (32ull << 20);
  c->touch_bytes = (c->touch_bytes + 255) & ~255ull;
  struct Alloc { void** ptr; uint64_t bytes; } allocs[] = {
      {(void**)&c->touch[0], c->touch_bytes},
      {(void**)&c->touch[1], c->touch_bytes},
      {(void**)&c->tables, 2048 * 4},
      {(void**)&c->hot_idx, R * C * 4},
      {(void**)&c->pool_col, R * d.hse_cap * 4},
      {(void**)&c->pool_rk, R * d.hse_cap * 4},
      {(void**)&c->pool_bm, R * d.hse_cap * (uint64_t)d.words * 4},
      {(void**)&c->ctb_alloc[0], (d.ctb_cap * R + 2 * kGuardWords) * 4},
      {(void**)&c->ctb_alloc[1], (d.ctb_cap * R + 2 * kGuardWords) * 4},
      {(void**)&c->dbg, SSD_DEBUG ? 4 : 0},
      {(void**)&c->stage, d.out_cap * 8},
      {(void**)&c->counters, sizeof(ssd::DevCounters)},
      {(void**)&c->n_out, 8},
      {(void**)&c->tl_fill, ssd::kMaxChunks * 4},
      {(void**)&c->bucket_off, NB ? R * (NB + 1) * 4 : 0},
      {(void**)&c->bucket_cnt, NB ? R * NB * 4 : 0},
      {(void**)&c->bucket_ent, NB ? R * d.hse_cap * 4 : 0},
  };
  for (auto& a : allocs) {
    if (a.bytes == 0) continue;
    if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      free_ctx(c);
      return SSD_ENOMEM;
    }
  }
  for (int i = 0; i < 2; ++i) c->ctb[i] = c->ctb_alloc[i] + kGuardWords;
  d.touch_bits = c->touch_bytes * 8;
  d.dbg = c->dbg;
  e = cudaMemcpy(c->tables, tables, 2048 * 4, cudaMemcpyHostToDevice);
#if SSD_DEBUG
  if (e == cudaSuccess) {
    e = cudaMemset(c->dbg, 0, 4);
    uint32_t guard[kGuardWords];
    for (auto& g : guard) g = kGuard;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaMemcpy(c->ctb_alloc[i], guard, kGuardWords * 4, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(c->ctb[i] + d.ctb_cap * R, guard, kGuardWords * 4, cudaMemcpyHostToDevice);
    }
  }
#endif
  if (e == cudaSuccess) e = cudaMemset(c->counters, 0, sizeof(ssd::DevCounters));
  // touch bits start (and are left by every fused slot) all zero
  if (e == cudaSuccess) e = cudaMemset(c->touch[0], 0, c->touch_bytes);
  if (e == cudaSuccess) e = cudaMemset(c->touch[1], 0, c->touch_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&c->ev_touched[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_closed[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "ssd_create"); }
  c->s.tables = c->tables;
  c->s.hot_idx = c->hot_idx;
  c->s.pool_col = c->pool_col;
  c->s.pool_rk = c->pool_rk;
  c->s.pool_bm = c->pool_bm;
  c->s.ctb[0] = c->ctb[0];
  c->s.ctb[1] = c->ctb[1];
  c->s.stage = c->stage;
  c->s.counters = c->counters;
  c->s.bucket_off = c->bucket_off;
  c->s.bucket_cnt = c->bucket_cnt;
  c->s.bucket_ent = c->bucket_ent;
  *out = c;
  return SSD_OK;
}

void ssd_destroy(ssd_ctx* ctx) { free_ctx(ctx); }

uint64_t ssd_sketch_bytes(const ssd_ctx* ctx) {
  if (!ctx) return 0;
  return (uint64_t)ctx->p.r << (ctx->p.q + ctx->p.log2_eta + 1);
}

int ssd_sketch_create(ssd_ctx* ctx, ssd_sketch** out) {
  if (!ctx || !out) return SSD_EINVAL;
  *out = nullptr;
  DeviceGuard g(ctx->device);
  ssd_sketch* s = new (std::nothrow) ssd_sketch;
  if (!s) return SSD_ENOMEM;
  s->ctx = ctx;
  s->device = ctx->device;
  s->slot = 0;
  s->view = 0;
  s->dr = nullptr;
  const uint64_t bytes = ssd_sketch_bytes(ctx);
  // the recorders, then the clock (256 bytes keep the allocation's tail aligned)
  if (cudaMalloc(&s->dr, bytes + 256) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return SSD_ENOMEM;
  }
  s->tm = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(s->dr) + bytes);
  // every distance recorder starts at 65535 (Sec. 3.2): kNever; the clock at slot 0
  cudaError_t e = reset_sketch(s, bytes, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    cudaFree(s->dr);
    delete s;
    return cuda_fail(e, "ssd_sketch_create");
  }
  *out = s;
  return SSD_OK;
}

void ssd_sketch_destroy(ssd_sketch* s) {
  if (!s) return;
  DeviceGuard g(s->device);
  cudaFree(s->dr);
  delete s;
}

int ssd_sketch_slot(const ssd_sketch* s, uint64_t* slot) {
  if (!s || !slot) return SSD_EINVAL;
  *slot = s->slot;
  return SSD_OK;
}

int ssd_sketch_set_slot(ssd_sketch* s, uint64_t slot) {
  if (!s) return SSD_EINVAL;
  s->slot = slot;
  return SSD_OK;
}

int ssd_sketch_set_view(ssd_sketch* s, uint32_t side, uint32_t group_bits, uint32_t group) {
  if (!s || side > SSD_SIDE_ONET || group_bits > SSD_MAX_GROUP_BITS) return SSD_EINVAL;
  if (group >> group_bits) return SSD_EINVAL;
  if (s->slot != 0) return SSD_ESTATE;
  s->view = ssd::view_pack(side, group_bits, group);
  return SSD_OK;
}

int ssd_sketch_view(const ssd_sketch* s, uint32_t* side, uint32_t* group_bits, uint32_t* group) {
  if (!s || !side || !group_bits || !group) return SSD_EINVAL;
  *side = s->view & 1u;
  *group_bits = (s->view >> 1) & 31u;
  *group = s->view >> 16;
  return SSD_OK;
}

int ssd_sketch_occupancy(const ssd_sketch* s, uint64_t* rk_sum, void* stream) {
  if (!s || !rk_sum) return SSD_EINVAL;
  ssd_ctx* ctx = s->ctx;
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  // the list staging buffer (at least 2^20 words) holds the r totals: this call is ordered on the
  // context's one stream like a regain
  unsigned long long* acc = ctx->stage;
  SSD_CUDA(cudaMemsetAsync(acc, 0, SSD_MAX_R * sizeof(unsigned long long), st));
  cudaError_t e = ssd::launch_occupancy(ctx->d, s->dr, s->tm, acc, ctx->sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy kernel");
  ctx->launches += 1;
  unsigned long long h[SSD_MAX_R];
  SSD_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  SSD_CUDA(cudaStreamSynchronize(st));
  for (uint32_t i = 0; i < ctx->d.r; ++i) rk_sum[i] = h[i];
  return SSD_OK;
}

int ssd_sketch_data(const ssd_sketch* s, uint16_t** d_recorders) {
  if (!s || !d_recorders) return SSD_EINVAL;
  *d_recorders = s->dr;
  return SSD_OK;
}

int ssd_min_merge(ssd_ctx* ctx, uint16_t* d_out, const uint16_t* const* d_in, int n, uint64_t count,
                  void* stream) {
  if (!ctx || !d_in || n < 1 || n > SSD_MAX_ROUTERS) return SSD_EINVAL;
  if (!count) return SSD_OK;
  if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15u)) return SSD_EINVAL;
  for (int j = 0; j < n; ++j)
    if (!d_in[j] || (reinterpret_cast<uintptr_t>(d_in[j]) & 15u)) return SSD_EINVAL;
  DeviceGuard g(ctx->device);
  cudaError_t e = ssd::launch_min_ranges(d_out, d_in, n, count, ctx->sms, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "min-merge kernel");
  ctx->launches += (count >> 3) ? 1 : 0;
  ctx->launches += (count & 7u) ? 1 : 0;
  return SSD_OK;
}

int ssd_sketch_export(const ssd_sketch* s, uint64_t first, uint64_t count, uint16_t* dst, void* stream) {
  if (!s || (count && !dst)) return SSD_EINVAL;
  ssd_ctx* ctx = s->ctx;
  const uint64_t n = ssd_sketch_bytes(ctx) / 2;
  if (first > n || count > n - first) return SSD_EINVAL;
  if (!count) return SSD_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  // the stamps read back as the distances of Sec. 3.2 at the sketch's clock
  if (device_memory(dst)) {
    cudaError_t e = ssd::launch_flip(s->dr + first, dst, count, s->tm, 0, nullptr, ctx->sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "export kernel");
    ctx->launches += 1;
  } else {
    int rc = xfer_buffer(ctx, count);
    if (rc != SSD_OK) return rc;
    for (uint64_t done = 0; done < count;) {
      const uint64_t m = count - done < ctx->xfer_count ? count - done : ctx->xfer_count;
      cudaError_t e = ssd::launch_flip(s->dr + first + done, ctx->xfer, m, s->tm, 0, nullptr, ctx->sms, st);
      if (e != cudaSuccess) return cuda_fail(e, "export kernel");
      ctx->launches += 1;
      SSD_CUDA(cudaMemcpyAsync(dst + done, ctx->xfer, m * 2, cudaMemcpyDeviceToHost, st));
      SSD_CUDA(cudaStreamSynchronize(st));   // the staging buffer is reused by the next piece
      done += m;
    }
  }
  SSD_CUDA(cudaStreamSynchronize(st));
  return SSD_OK;
}

int ssd_sketch_import(ssd_sketch* s, const uint16_t* src, uint64_t slot, void* stream) {
  if (!s || !src) return SSD_EINVAL;
  ssd_ctx* ctx = s->ctx;
  const uint64_t n = ssd_sketch_bytes(ctx) / 2;
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  // distances to stamps at the clock of `slot`; the clock is stored with the first piece
  const uint32_t tm = (uint32_t)(slot % 65535u);
  if (device_memory(src)) {
    cudaError_t e = ssd::launch_flip(src, s->dr, n, nullptr, tm, s->tm, ctx->sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "import kernel");
    ctx->launches += 1;
  } else {
    int rc = xfer_buffer(ctx, n);
    if (rc != SSD_OK) return rc;
    for (uint64_t done = 0; done < n;) {
      const uint64_t m = n - done < ctx->xfer_count ? n - done : ctx->xfer_count;
      SSD_CUDA(cudaMemcpyAsync(ctx->xfer, src + done, m * 2, cudaMemcpyHostToDevice, st));
      cudaError_t e = ssd::launch_flip(ctx->xfer, s->dr + done, m, nullptr, tm, done ? nullptr : s->tm, ctx->sms, st);
      if (e != cudaSuccess) return cuda_fail(e, "import kernel");
      ctx->launches += 1;
      SSD_CUDA(cudaStreamSynchronize(st));   // the staging buffer is reused by the next piece
      done += m;
    }
  }
  SSD_CUDA(cudaStreamSynchronize(st));
  s->slot = slot;
  return SSD_OK;
}

int ssd_scan(ssd_sketch* s, const uint32_t* d_pairs, uint64_t n_pairs, void* stream) {
  if (!s) return SSD_EINVAL;
  return ssd_scan_batch(&s, &d_pairs, &n_pairs, 1, stream);
}

int ssd_scan_batch(ssd_sketch* const* sketches, const uint32_t* const* d_pairs, const uint64_t* n_pairs, int n,
                   void* stream) {
  ssd_ctx* ctx = nullptr;
  if (!same_ctx(sketches, n, &ctx) || !d_pairs || !n_pairs) return SSD_EINVAL;
  ssd::ScanBatch b;
  std::memset(&b, 0, sizeof(b));
  b.n = n;
  uint64_t prefix = 0;
  bool any_edge = false;
  for (int j = 0; j < n; ++j) {
    int rc = add_job(b, j, sketches[j], d_pairs[j], n_pairs[j], &prefix);
    if (rc != SSD_OK) return rc;
    any_edge = any_edge || b.edge[2 * j] || b.edge[2 * j + 1];
  }
  b.prefix[n] = prefix;
  DeviceGuard g(ctx->device);
  return scan_jobs(ctx, b, prefix, any_edge, as_stream(stream));
}

int ssd_scan_host(ssd_sketch* s, const uint32_t* h_pairs, uint64_t n_pairs, void* stream) {
  if (!s || (n_pairs && !h_pairs)) return SSD_EINVAL;
  if (n_pairs == 0) return SSD_OK;
  ssd_ctx* ctx = s->ctx;
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  if (!ctx->copy_stream) {  // first call: the two alpha-pair device buffers of Sec. 4.1
    const uint64_t alpha = 1ull << 22;
    for (int i = 0; i < 2; ++i) {
      if (cudaMalloc(&ctx->stage_pairs[i], alpha * 8) != cudaSuccess) {
        cudaGetLastError();
        return SSD_ENOMEM;
      }
      SSD_CUDA(cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming));
      SSD_CUDA(cudaEventCreateWithFlags(&ctx->ev_scanned[i], cudaEventDisableTiming));
    }
    SSD_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    ctx->stage_alpha = alpha;
  }
  // the copy stream starts after whatever the caller queued before this call
  SSD_CUDA(cudaEventRecord(ctx->ev_scanned[0], st));
  SSD_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_scanned[0], 0));
  uint64_t done = 0;
  for (int c = 0; done < n_pairs; ++c) {
    const int b = c & 1;
    const uint64_t m = n_pairs - done < ctx->stage_alpha ? n_pairs - done : ctx->stage_alpha;
    if (c >= 2) SSD_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_scanned[b], 0));  // buffer b is free
    SSD_CUDA(cudaMemcpyAsync(ctx->stage_pairs[b], h_pairs + 2 * done, m * 8, cudaMemcpyHostToDevice,
                             ctx->copy_stream));
    SSD_CUDA(cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
    SSD_CUDA(cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
    const uint32_t* dp = ctx->stage_pairs[b];
    int rc = ssd_scan_batch(&s, &dp, &m, 1, stream);
    if (rc != SSD_OK) return rc;
    SSD_CUDA(cudaEventRecord(ctx->ev_scanned[b], st));
    done += m;
  }
  return SSD_OK;
}

int ssd_set_trace(ssd_ctx* ctx, void* ev_start, void* ev_pass, void* ev_end) {
  if (!ctx) return SSD_EINVAL;
  ctx->tr_start = reinterpret_cast<cudaEvent_t>(ev_start);
  ctx->tr_pass = reinterpret_cast<cudaEvent_t>(ev_pass);
  ctx->tr_end = reinterpret_cast<cudaEvent_t>(ev_end);
  return SSD_OK;
}

int ssd_advance(ssd_sketch* const* sketches, int n, void* stream) {
  ssd_ctx* ctx = nullptr;
  if (!same_ctx(sketches, n, &ctx)) return SSD_EINVAL;
  DeviceGuard g(ctx->device);
  int rc = stream_pass(ctx, sketches, n, nullptr, ssd::kAdvance, as_stream(stream));
  if (rc == SSD_OK) rc = tick(ctx, sketches, n, as_stream(stream));
  if (rc != SSD_OK) return rc;
  for (int i = 0; i < n; ++i) sketches[i]->slot += 1;
  return SSD_OK;
}

int ssd_merge(ssd_sketch* const* routers, int n, ssd_sketch* global, void* stream) {
  ssd_ctx* ctx = nullptr;
  if (!same_ctx(routers, n, &ctx) || !global || global->ctx != ctx) return SSD_EINVAL;
  if (!same_view(routers, n)) return SSD_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (routers[i] == global) return SSD_EINVAL;
    if (routers[i]->slot != routers[0]->slot) return SSD_ESTATE;
  }
  DeviceGuard g(ctx->device);
  int rc = stream_pass(ctx, routers, n, global, 0, as_stream(stream));
  if (rc != SSD_OK) return rc;
  global->slot = routers[0]->slot;
  global->view = routers[0]->view;
  return SSD_OK;
}

int ssd_regain(ssd_ctx* ctx, const ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk, uint64_t cap,
               uint64_t* n_out, void* stream) {
  if (!ctx || !global || global->ctx != ctx || !n_out || (cap && (!d_ips || !d_rk))) return SSD_EINVAL;
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  SSD_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(ssd::DevCounters), st));
  int rc = trace(ctx, ctx->tr_start, st);
  if (rc != SSD_OK) return rc;
  ssd_sketch* one = const_cast<ssd_sketch*>(global);
  rc = stream_pass(ctx, &one, 1, nullptr, ssd::kHot, st);
  if (rc == SSD_OK) rc = trace(ctx, ctx->tr_pass, st);
  if (rc == SSD_OK) rc = regain_after_pass(ctx, d_ips, d_rk, cap, ctx->n_out, st, global->view);
  if (rc == SSD_OK) rc = trace(ctx, ctx->tr_end, st);
  if (rc != SSD_OK) return rc;
  ssd::DevCounters h;
  SSD_CUDA(cudaMemcpyAsync(&h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost, st));
  SSD_CUDA(cudaStreamSynchronize(st));
  *n_out = h.n_out;
  if (h.status & (SSD_STATUS_HSE_OVERFLOW | SSD_STATUS_CTB_OVERFLOW | SSD_STATUS_OUT_OVERFLOW |
                  SSD_STATUS_LIST_OVERFLOW))
    return SSD_ECAPACITY;
  return SSD_OK;
}

int ssd_close_slot(ssd_ctx* ctx, ssd_sketch* const* routers, int n, ssd_sketch* global, uint32_t* d_ips,
                   uint32_t* d_rk, uint64_t cap, uint64_t* d_n_out, void* stream) {
  ssd_ctx* c2 = nullptr;
  if (!ctx || !same_ctx(routers, n, &c2) || c2 != ctx) return SSD_EINVAL;
  if (global && global->ctx != ctx) return SSD_EINVAL;
  if (cap && (!d_ips || !d_rk)) return SSD_EINVAL;
  if (!same_view(routers, n)) return SSD_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (routers[i] == global) return SSD_EINVAL;
    if (routers[i]->slot != routers[0]->slot) return SSD_ESTATE;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  SSD_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(ssd::DevCounters), st));
  int rc = trace(ctx, ctx->tr_start, st);
  if (rc != SSD_OK) return rc;
  rc = stream_pass(ctx, routers, n, global, ssd::kAdvance | ssd::kHot, st);
  if (rc == SSD_OK) rc = trace(ctx, ctx->tr_pass, st);
  unsigned long long* nd = d_n_out ? reinterpret_cast<unsigned long long*>(d_n_out) : ctx->n_out;
  if (rc == SSD_OK) rc = regain_after_pass(ctx, d_ips, d_rk, cap, nd, st, routers[0]->view);
  if (rc == SSD_OK) rc = tick(ctx, routers, n, st);
  if (rc == SSD_OK) rc = trace(ctx, ctx->tr_end, st);
  if (rc != SSD_OK) return rc;
  const uint64_t merged = routers[0]->slot;
  for (int i = 0; i < n; ++i) routers[i]->slot += 1;
  if (global) {
    global->slot = merged;
    global->view = routers[0]->view;
  }
  return SSD_OK;
}

// Entries one touch list of a one-router slot can need: a pair adds at most
// one touch per row, so a chunk inside one row gets at most n_pairs, a chunk of
// m whole rows at most m * n_pairs.
static uint64_t list_cap(const ssd::Dims& d, uint64_t count, uint64_t n_pairs) {
  uint64_t rows = count >> d.q;
  if (rows < 1) rows = 1;
  if (rows > d.r) rows = d.r;
  return n_pairs * rows;
}

// Whether the one-router fused slot takes its touches from per-chunk lists: the
// configuration asks for it and a touch's bit index within its chunk fits 32 bits.
static bool uses_lists(const ssd_ctx* ctx, uint64_t count) {
  return ctx->tn.collect == 0 && (count << ctx->d.log2_eta) <= (1ull << 32);
}

// Grows the touch lists to hold (n_chunks - 1) lists of `cap` entries (waits for the device first).
static int reserve_lists(ssd_ctx* ctx, uint64_t n_chunks, uint64_t cap) {
  const uint64_t need = (n_chunks > 1 ? n_chunks - 1 : 0) * cap;
  if (need <= ctx->tl_entries) return SSD_OK;
  SSD_CUDA(cudaDeviceSynchronize());
  cudaFree(ctx->tl_ent);
  ctx->tl_ent = nullptr;
  ctx->epoch += 1;
  const uint64_t want = need + need / 4 + 64;
  if (cudaMalloc(&ctx->tl_ent, want * 4) != cudaSuccess) {
    cudaGetLastError();
    ctx->tl_entries = 0;
    return SSD_ENOMEM;
  }
  ctx->tl_entries = want;
  return SSD_OK;
}

// Estimators per chunk of a fused slot of n routers (a power of two: each chunk's
// touch bits, one per recorder and router, fit the touch buffer) and the chunk count.
static void chunking(const ssd_ctx* ctx, int n, uint64_t* count, uint64_t* n_chunks) {
  const ssd::Dims& d = ctx->d;
  const uint64_t n_se = (uint64_t)d.r << d.q;
  const uint64_t se_bytes = (uint64_t)n * (d.eta >> 3);  // touch bytes of one estimator, all routers
  uint64_t c = 1;
  while (c * 2 * se_bytes <= ctx->touch_bytes && c * 2 <= pow2_at_least(n_se)) c *= 2;
  *count = c;
  *n_chunks = (n_se + c - 1) / c;
}

// The fused slot of one router (eta >= 256) in chunks on one stream. The touches of the
// slot are found once: by default one launch hashes every pair, sets chunk 0's touch bits
// and writes the others into per-chunk touch lists; each chunk's streaming kernel applies
// its bits and, between estimators, sets the next chunk's from its list. Otherwise (the
// `collect` field of the configuration) the pairs are pre-hashed once and every chunk
// launch re-reads them all.
static int slot_chunks1(ssd_ctx* ctx, ssd_sketch* router, const uint32_t* pairs, uint64_t n_pairs,
                        ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk, uint64_t cap, uint64_t* d_n_out,
                        void* stream, uint64_t count, uint64_t n_chunks) {
  const ssd::Dims& d = ctx->d;
  const uint64_t n_se = (uint64_t)d.r << d.q;
  ssd::ScanBatch b;
  std::memset(&b, 0, sizeof(b));
  b.n = 1;
  uint64_t nvec = 0;
  int rc = add_job(b, 0, router, pairs, n_pairs, &nvec);
  if (rc != SSD_OK) return rc;
  b.prefix[1] = nvec;
  const uint64_t tgrid = scan_grid(ctx, nvec);
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  const bool lists = uses_lists(ctx, count);
  const uint64_t lcap = list_cap(d, count, n_pairs);
  // both hashes of every pair once per slot when they pack into one word (a grouped view
  // keeps the raw pairs: a pair outside the group must be skippable)
  const bool prehash = !lists && d.q + d.log2_eta <= 32 && ((router->view >> 1) & 31u) == 0;
  if (lists) {
    rc = reserve_lists(ctx, n_chunks, lcap);   // a larger slot than any before: grow (waits for the device)
    if (rc != SSD_OK) return rc;
  }
  if (prehash && n_pairs > ctx->packed_cap) {  // a larger slot than any before: grow (waits for `stream`)
    SSD_CUDA(cudaStreamSynchronize(st));
    cudaFree(ctx->packed);
    ctx->packed = nullptr;
    ctx->epoch += 1;
    const uint64_t want = n_pairs + n_pairs / 4 + 64;
    if (cudaMalloc(&ctx->packed, want * 8) != cudaSuccess) {
      cudaGetLastError();
      ctx->packed_cap = 0;
      return SSD_ENOMEM;
    }
    ctx->packed_cap = want;
  }
  SSD_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(ssd::DevCounters), st));
  rc = trace(ctx, ctx->tr_start, st);
  if (rc != SSD_OK) return rc;
  const uint64_t cnt0 = n_se < count ? n_se : count;
  ssd::ChunkArgs a;
  std::memset(&a, 0, sizeof(a));
  a.router = router->dr;
  a.tm = router->tm;
  a.global = global ? global->dr : nullptr;
  a.global_tm = global ? global->tm : nullptr;
  a.view = router->view;
  cudaError_t e;
  if (lists) {
    SSD_CUDA(cudaMemsetAsync(ctx->tl_fill, 0, ssd::kMaxChunks * 4, st));
    ssd::ListArgs la;
    la.log2_count = 0;
    while ((1ull << la.log2_count) < count) ++la.log2_count;
    la.n_chunks = (uint32_t)n_chunks;
    la.cap = lcap;
    la.ent = ctx->tl_ent;
    la.fill = ctx->tl_fill;
    la.touch0 = ctx->touch[0];
    la.counters = ctx->counters;
    e = ssd::launch_lists(d, ctx->tables, b, la, (int)tgrid, ctx->tn, st);
  } else if (prehash) {
    if (n_pairs) {
      e = ssd::launch_prehash(d, ctx->tables, b, ctx->packed, (int)tgrid, st);
      if (e != cudaSuccess) return cuda_fail(e, "prehash kernel");
      ctx->launches += 1;
    }
    a.packed = 1;
    a.vec = reinterpret_cast<const uint4*>(ctx->packed);
    a.nvec = n_pairs / 2;
    a.edge[0] = (n_pairs & 1) ? reinterpret_cast<const uint32_t*>(ctx->packed + (n_pairs - 1)) : nullptr;
    a.edge[1] = nullptr;
    e = ssd::launch_touch_packed(d, a.vec, a.nvec, reinterpret_cast<const uint2*>(a.edge[0]), ctx->touch[0], 0,
                                 cnt0, (int)tgrid, ctx->tn, st);
  } else {
    a.vec = b.vec[0];
    a.nvec = nvec;
    a.edge[0] = b.edge[0];
    a.edge[1] = b.edge[1];
    e = ssd::launch_touch(d, ctx->tables, b, ctx->touch[0], 0, cnt0, (int)tgrid, ctx->tn, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "touch kernel");
  ctx->launches += 1;
  for (uint64_t c = 0; c < n_chunks; ++c) {
    a.se0 = c * count;
    a.count = n_se - a.se0 < count ? n_se - a.se0 : count;
    a.touch = reinterpret_cast<uint8_t*>(ctx->touch[c & 1]);
    if (c + 1 < n_chunks) {
      a.next = ctx->touch[(c + 1) & 1];
      a.nx_se0 = (c + 1) * count;
      a.nx_count = n_se - a.nx_se0 < count ? n_se - a.nx_se0 : count;
      if (lists) {
        a.list = ctx->tl_ent + c * lcap;        // list of chunk c + 1
        a.list_fill = ctx->tl_fill + (c + 1);
      }
    } else {
      a.next = nullptr;
      a.nx_se0 = a.nx_count = 0;
      a.list = nullptr;
      a.list_fill = nullptr;
    }
    e = ssd::launch_chunk(d, ctx->s, a, ctx->sms, ctx->tn, st);
    if (e != cudaSuccess) return cuda_fail(e, "chunk kernel");
    ctx->launches += 1;
  }
  rc = trace(ctx, ctx->tr_pass, st);
  unsigned long long* nd = d_n_out ? reinterpret_cast<unsigned long long*>(d_n_out) : ctx->n_out;
  if (rc == SSD_OK) rc = regain_after_pass(ctx, d_ips, d_rk, cap, nd, st, router->view);
  if (rc == SSD_OK) rc = tick(ctx, &router, 1, st);
  if (rc == SSD_OK) rc = trace(ctx, ctx->tr_end, st);
  if (rc != SSD_OK) return rc;
  if (global) {
    global->slot = router->slot;
    global->view = router->view;
  }
  router->slot += 1;
  return SSD_OK;
}

int ssd_slot(ssd_ctx* ctx, ssd_sketch* const* routers, const uint32_t* const* d_pairs, const uint64_t* n_pairs,
             int n, ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk, uint64_t cap, uint64_t* d_n_out,
             void* stream) {
  ssd_ctx* c2 = nullptr;
  if (!ctx || !same_ctx(routers, n, &c2) || c2 != ctx || !d_pairs || !n_pairs) return SSD_EINVAL;
  if (global && global->ctx != ctx) return SSD_EINVAL;
  if (cap && (!d_ips || !d_rk)) return SSD_EINVAL;
  if (!same_view(routers, n)) return SSD_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (routers[i] == global) return SSD_EINVAL;
    if (routers[i]->slot != routers[0]->slot) return SSD_ESTATE;
    for (int j = 0; j < i; ++j)
      if (routers[j] == routers[i]) return SSD_EINVAL;
  }
  const ssd::Dims& d = ctx->d;
  const uint64_t n_se = (uint64_t)d.r << d.q;
  const uint64_t se_bytes = (uint64_t)n * (d.eta >> 3);  // touch bytes of one estimator, all routers
  uint64_t count = 1, n_chunks = 1;
  chunking(ctx, n, &count, &n_chunks);
  if (n == 1 && d.eta >= 256 && !(d.flags & SSD_SLOT_CHUNKED) && count * se_bytes <= ctx->touch_bytes &&
      count >= 8 && n_chunks <= 32)
    return slot_chunks1(ctx, routers[0], d_pairs[0], n_pairs[0], global, d_ips, d_rk, cap, d_n_out, stream, count,
                        n_chunks);
  if (count * se_bytes > ctx->touch_bytes || count < 8 || n_chunks > 16) {
    int rc = ssd_scan_batch(routers, d_pairs, n_pairs, n, stream);
    if (rc != SSD_OK) return rc;
    return ssd_close_slot(ctx, routers, n, global, d_ips, d_rk, cap, d_n_out, stream);
  }
  ssd::ScanBatch b;
  std::memset(&b, 0, sizeof(b));
  b.n = n;
  uint64_t prefix = 0;
  for (int j = 0; j < n; ++j) {
    int rc = add_job(b, j, routers[j], d_pairs[j], n_pairs[j], &prefix);
    if (rc != SSD_OK) return rc;
  }
  b.prefix[n] = prefix;
  const uint64_t tgrid = scan_grid(ctx, prefix);

  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  SSD_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(ssd::DevCounters), st));
  int rc = trace(ctx, ctx->tr_start, st);
  if (rc != SSD_OK) return rc;
  SSD_CUDA(cudaEventRecord(ctx->ev_fork, st));
  SSD_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  ssd::StreamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  for (int i = 0; i < n; ++i) {
    a.routers[i] = routers[i]->dr;
    a.tm[i] = routers[i]->tm;
  }
  a.global = global ? global->dr : nullptr;
  a.global_tm = global ? global->tm : nullptr;
  for (uint64_t c = 0; c < n_chunks; ++c) {
    const int bsel = (int)(c & 1);
    const uint64_t se0 = c * count;
    const uint64_t cnt = n_se - se0 < count ? n_se - se0 : count;
    if (c >= 2) SSD_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_closed[bsel], 0));  // buffer cleared
    cudaError_t e = ssd::launch_touch(d, ctx->tables, b, ctx->touch[bsel], se0, cnt, (int)tgrid, ctx->tn, ctx->side);
    if (e != cudaSuccess) return cuda_fail(e, "touch kernel");
    ctx->launches += 1;
    SSD_CUDA(cudaEventRecord(ctx->ev_touched[bsel], ctx->side));
    SSD_CUDA(cudaStreamWaitEvent(st, ctx->ev_touched[bsel], 0));
    a.se0 = se0;
    a.se_count = cnt;
    a.touch = reinterpret_cast<uint8_t*>(ctx->touch[bsel]);
    e = ssd::launch_stream(d, ctx->s, a, ssd::kAdvance | ssd::kHot, ctx->sms, ctx->tn, st);
    if (e != cudaSuccess) return cuda_fail(e, "stream kernel");
    ctx->launches += 1;
    SSD_CUDA(cudaEventRecord(ctx->ev_closed[bsel], st));
  }
  rc = trace(ctx, ctx->tr_pass, st);
  unsigned long long* nd = d_n_out ? reinterpret_cast<unsigned long long*>(d_n_out) : ctx->n_out;
  if (rc == SSD_OK) rc = regain_after_pass(ctx, d_ips, d_rk, cap, nd, st, routers[0]->view);
  if (rc == SSD_OK) rc = tick(ctx, routers, n, st);
  if (rc == SSD_OK) rc = trace(ctx, ctx->tr_end, st);
  if (rc != SSD_OK) return rc;
  const uint64_t merged = routers[0]->slot;
  for (int i = 0; i < n; ++i) routers[i]->slot += 1;
  if (global) {
    global->slot = merged;
    global->view = routers[0]->view;
  }
  return SSD_OK;
}

int ssd_slot_host(ssd_ctx* ctx, ssd_sketch* const* routers, const uint32_t* const* h_pairs,
                  const uint64_t* n_pairs, int n, ssd_sketch* global, uint32_t* d_ips, uint32_t* d_rk,
                  uint64_t cap, uint64_t* d_n_out, void* stream) {
  ssd_ctx* c2 = nullptr;
  if (!ctx || !same_ctx(routers, n, &c2) || c2 != ctx || !h_pairs || !n_pairs) return SSD_EINVAL;
  uint64_t off[SSD_MAX_ROUTERS + 1];
  off[0] = 0;
  for (int j = 0; j < n; ++j) {
    if (n_pairs[j] && !h_pairs[j]) return SSD_EINVAL;
    off[j + 1] = off[j] + ((n_pairs[j] * 8 + 15) & ~15ull);  // 16-byte aligned start per router
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  if (!ctx->copy_stream) SSD_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  if (!ctx->ev_hs_copied) {
    SSD_CUDA(cudaEventCreateWithFlags(&ctx->ev_hs_copied, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) SSD_CUDA(cudaEventCreateWithFlags(&ctx->ev_hs_free[i], cudaEventDisableTiming));
  }
  if (off[n] > ctx->hs_bytes) {  // grow the staging areas (waits for the work using them)
    SSD_CUDA(cudaStreamSynchronize(ctx->copy_stream));
    SSD_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < 2; ++i) {
      SSD_CUDA(cudaEventSynchronize(ctx->ev_hs_free[i]));
      cudaFree(ctx->hs_buf[i]);
      ctx->hs_buf[i] = nullptr;
    }
    ctx->epoch += 1;
    const uint64_t want = off[n] + off[n] / 4 + 256;
    for (int i = 0; i < 2; ++i) {
      if (cudaMalloc(&ctx->hs_buf[i], want) != cudaSuccess) {
        cudaGetLastError();
        ctx->hs_bytes = 0;
        return SSD_ENOMEM;
      }
    }
    ctx->hs_bytes = want;
  }
  const int b = (int)(ctx->hs_calls & 1);
  SSD_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_hs_free[b], 0));  // the slot two calls back is done
  const uint32_t* dp[SSD_MAX_ROUTERS];
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->hs_buf[b]);
  for (int j = 0; j < n; ++j) {
    dp[j] = reinterpret_cast<const uint32_t*>(base + off[j]);
    if (n_pairs[j])
      SSD_CUDA(cudaMemcpyAsync(base + off[j], h_pairs[j], n_pairs[j] * 8, cudaMemcpyHostToDevice, ctx->copy_stream));
  }
  SSD_CUDA(cudaEventRecord(ctx->ev_hs_copied, ctx->copy_stream));
  SSD_CUDA(cudaStreamWaitEvent(st, ctx->ev_hs_copied, 0));
  int rc = ssd_slot(ctx, routers, dp, n_pairs, n, global, d_ips, d_rk, cap, d_n_out, stream);
  if (rc != SSD_OK) return rc;
  SSD_CUDA(cudaEventRecord(ctx->ev_hs_free[b], st));
  ctx->hs_calls += 1;
  return SSD_OK;
}

int ssd_reserve(ssd_ctx* ctx, uint64_t max_pairs) {
  if (!ctx) return SSD_EINVAL;
  DeviceGuard g(ctx->device);
  SSD_CUDA(cudaDeviceSynchronize());
  uint64_t count = 1, n_chunks = 1;
  chunking(ctx, 1, &count, &n_chunks);
  if (uses_lists(ctx, count)) {   // the touch lists of a one-router slot
    const int rc = reserve_lists(ctx, n_chunks, list_cap(ctx->d, count, max_pairs));
    if (rc != SSD_OK) return rc;
  }
  if (max_pairs > ctx->packed_cap) {
    cudaFree(ctx->packed);
    ctx->packed = nullptr;
    ctx->epoch += 1;
    if (cudaMalloc(&ctx->packed, max_pairs * 8) != cudaSuccess) {
      cudaGetLastError();
      ctx->packed_cap = 0;
      return SSD_ENOMEM;
    }
    ctx->packed_cap = max_pairs;
  }
  // ssd_slot_host starts each router's pairs on a 16-byte boundary: up to 15 bytes per router more
  const uint64_t bytes = ((max_pairs * 8 + 15) & ~15ull) + 16ull * SSD_MAX_ROUTERS + 256;
  if (bytes > ctx->hs_bytes) {
    ctx->epoch += 1;
    for (int i = 0; i < 2; ++i) {
      cudaFree(ctx->hs_buf[i]);
      ctx->hs_buf[i] = nullptr;
      if (cudaMalloc(&ctx->hs_buf[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->hs_bytes = 0;
        return SSD_ENOMEM;
      }
    }
    ctx->hs_bytes = bytes;
  }
  return SSD_OK;
}

int ssd_stats_get(ssd_ctx* ctx, ssd_stats* out, void* stream) {
  if (!ctx || !out) return SSD_EINVAL;
  DeviceGuard g(ctx->device);
  ssd::DevCounters h;
  SSD_CUDA(cudaMemcpyAsync(&h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost, as_stream(stream)));
  SSD_CUDA(cudaStreamSynchronize(as_stream(stream)));
  std::memset(out, 0, sizeof(*out));
  out->status = h.status;
  out->threshold = ctx->d.thr;
  for (uint32_t i = 0; i < SSD_MAX_R; ++i) {
    out->hot[i] = i < ctx->d.r ? h.hot[i] : 0;
    out->level[i] = i < ctx->d.r ? h.level[i] : 0;
  }
  out->level[0] = out->hot[0];
  out->raw = h.raw;
  out->n_out = h.n_out;
#if SSD_DEBUG
  {   // the kernels' bound checks and the candidate buffers' guard words
    unsigned int dbg = 0;
    SSD_CUDA(cudaMemcpy(&dbg, ctx->dbg, 4, cudaMemcpyDeviceToHost));
    out->status |= dbg;
    uint32_t g[kGuardWords ? kGuardWords : 1];
    const uint64_t words = ctx->d.ctb_cap * ctx->d.r;
    for (int i = 0; i < 2; ++i) {
      for (const uint32_t* at : {ctx->ctb_alloc[i], ctx->ctb[i] + words}) {
        SSD_CUDA(cudaMemcpy(g, at, kGuardWords * 4, cudaMemcpyDeviceToHost));
        for (uint64_t w = 0; w < kGuardWords; ++w)
          if (g[w] != kGuard) out->status |= SSD_STATUS_INTERNAL;
      }
    }
  }
#endif
  return SSD_OK;
}

int ssd_build_flags(void) { return SSD_DEBUG ? SSD_BUILD_DEBUG : 0; }

uint64_t ssd_launch_count(const ssd_ctx* ctx) { return ctx ? ctx->launches : 0; }

uint64_t ssd_buffer_epoch(const ssd_ctx* ctx) { return ctx ? ctx->epoch : 0; }

int ssd_tuning_get(const ssd_ctx* ctx, ssd_tuning* out) {
  if (!ctx || !out) return SSD_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->touch_chunk_bytes = ctx->touch_bytes;
  out->stream_blocks_per_sm = ctx->tn.stream_bps;
  out->scan_blocks_per_sm = ctx->tn.scan_bps;
  out->scan_unroll = ctx->tn.unroll;
  out->merge_group = ctx->tn.group;
  out->combine_touches = ctx->tn.combine;
  out->collect_touches = ctx->tn.collect;
  out->pair_level = ctx->tn.pair_level;
  return SSD_OK;
}

int ssd_tuning_set(ssd_ctx* ctx, const ssd_tuning* t) {
  if (!ctx || !t || t->collect_touches > 1 || t->pair_level > 1 || t->reserved) return SSD_EINVAL;
  if (t->touch_chunk_bytes < (64ull << 10) || t->touch_chunk_bytes > (1ull << 30)) return SSD_EINVAL;
  if (t->stream_blocks_per_sm > 8 || t->scan_blocks_per_sm < 1 || t->scan_blocks_per_sm > 32) return SSD_EINVAL;
  const uint32_t u = t->scan_unroll, g = t->merge_group;
  if (u != 1 && u != 2 && u != 4 && u != 8) return SSD_EINVAL;
  if (g != 2 && g != 4 && g != 8) return SSD_EINVAL;
  if (t->combine_touches > 2) return SSD_EINVAL;
  const uint64_t bytes = (t->touch_chunk_bytes + 255) & ~255ull;
  if (bytes != ctx->touch_bytes) {  // new touch buffers, zeroed, before the old ones go
    DeviceGuard dg(ctx->device);
    SSD_CUDA(cudaDeviceSynchronize());
    uint32_t* nb[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) {
      if (cudaMalloc(&nb[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(nb[0]);
        return SSD_ENOMEM;
      }
    }
    cudaError_t e = cudaMemset(nb[0], 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(nb[1], 0, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaFree(nb[0]);
      cudaFree(nb[1]);
      return cuda_fail(e, "ssd_tuning_set");
    }
    for (int i = 0; i < 2; ++i) {
      cudaFree(ctx->touch[i]);
      ctx->touch[i] = nb[i];
    }
    ctx->touch_bytes = bytes;
    ctx->d.touch_bits = bytes * 8;
    ctx->epoch += 1;
  }
  ctx->tn.stream_bps = t->stream_blocks_per_sm;
  ctx->tn.scan_bps = t->scan_blocks_per_sm;
  ctx->tn.unroll = u;
  ctx->tn.group = g;
  ctx->tn.combine = t->combine_touches;
  ctx->tn.collect = t->collect_touches;
  ctx->tn.pair_level = t->pair_level;
  return SSD_OK;
}

int ssd_autotune(ssd_ctx* ctx, ssd_sketch* const* routers, const uint32_t* const* d_pairs,
                 const uint64_t* n_pairs, int n, ssd_sketch* global, int reps, ssd_tuning* out, void* stream) {
  ssd_ctx* c2 = nullptr;
  if (!ctx || !same_ctx(routers, n, &c2) || c2 != ctx || !d_pairs || !n_pairs) return SSD_EINVAL;
  if (reps < 1 || reps > 16) return SSD_EINVAL;
  if (global && global->ctx != ctx) return SSD_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (routers[i] == global) return SSD_EINVAL;
    if (routers[i]->slot != 0) return SSD_ESTATE;
  }
  if (global && global->slot != 0) return SSD_ESTATE;
  DeviceGuard dg(ctx->device);
  cudaStream_t st = as_stream(stream);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  for (int i = 0; i < 2; ++i) SSD_CUDA(cudaEventCreate(&ev[i]));
  ssd_tuning start;
  ssd_tuning_get(ctx, &start);

  // median time of `reps` slots under t, after one untimed slot (which also
  // makes any first-call allocation of ssd_slot)
  auto measure = [&](const ssd_tuning& t, float* ms) -> int {
    int rc = ssd_tuning_set(ctx, &t);
    if (rc != SSD_OK) return rc;
    float v[16];
    for (int i = -1; i < reps; ++i) {
      if (i >= 0 && cudaEventRecord(ev[0], st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune");
      rc = ssd_slot(ctx, routers, d_pairs, n_pairs, n, global, nullptr, nullptr, 0, nullptr, stream);
      if (rc != SSD_OK) return rc;
      if (i < 0) continue;
      cudaError_t e = cudaEventRecord(ev[1], st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&v[i], ev[0], ev[1]);
      if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    }
    for (int i = 1; i < reps; ++i)  // insertion sort of at most 16 values
      for (int j = i; j > 0 && v[j] < v[j - 1]; --j) {
        const float x = v[j]; v[j] = v[j - 1]; v[j - 1] = x;
      }
    *ms = v[reps / 2];
    return SSD_OK;
  };

  // coordinate descent: one field at a time over its candidates, two sweeps; a
  // new value must beat the current one (measured again beside it) by 1 %
  ssd_tuning best = start;
  int rc = SSD_OK;
  for (int sweep = 0; sweep < 2 && rc == SSD_OK; ++sweep) {
    for (int field = 0; field < 8 && rc == SSD_OK; ++field) {
      uint64_t cand[8];
      int nc = 0;
      switch (field) {
        case 0: for (uint64_t m : {8ull, 16ull, 32ull, 64ull}) cand[nc++] = m << 20; break;
        case 1: for (uint64_t b : {0ull, 1ull, 2ull, 3ull}) cand[nc++] = b; break;
        case 2: for (uint64_t b : {2ull, 4ull, 8ull, 16ull, 32ull}) cand[nc++] = b; break;
        case 3: for (uint64_t u : {1ull, 2ull, 4ull, 8ull}) cand[nc++] = u; break;
        case 4: if (n > 1) for (uint64_t g : {2ull, 4ull, 8ull}) cand[nc++] = g; break;
        case 5: for (uint64_t c : {0ull, 1ull, 2ull}) cand[nc++] = c; break;
        case 6: if (n == 1) for (uint64_t c : {0ull, 1ull}) cand[nc++] = c; break;
        default: for (uint64_t c : {0ull, 1ull}) cand[nc++] = c; break;
      }
      auto with = [&](uint64_t v) {
        ssd_tuning t = best;
        switch (field) {
          case 0: t.touch_chunk_bytes = v; break;
          case 1: t.stream_blocks_per_sm = (uint32_t)v; break;
          case 2: t.scan_blocks_per_sm = (uint32_t)v; break;
          case 3: t.scan_unroll = (uint32_t)v; break;
          case 4: t.merge_group = (uint32_t)v; break;
          case 5: t.combine_touches = (uint32_t)v; break;
          case 6: t.collect_touches = (uint32_t)v; break;
          default: t.pair_level = (uint32_t)v; break;
        }
        return t;
      };
      if (nc == 0) continue;
      float cur = 0.f;
      rc = measure(best, &cur);
      ssd_tuning pick = best;
      float pick_ms = cur;
      for (int i = 0; i < nc && rc == SSD_OK; ++i) {
        const ssd_tuning t = with(cand[i]);
        if (std::memcmp(&t, &best, sizeof(t)) == 0) continue;
        float ms = 0.f;
        rc = measure(t, &ms);
        if (rc == SSD_ENOMEM && field == 0) {  // touch buffers of that size do not fit: skip it
          rc = SSD_OK;
          continue;
        }
        if (rc == SSD_OK && ms < pick_ms && ms < 0.99f * cur) {
          pick = t;
          pick_ms = ms;
        }
      }
      best = pick;
    }
  }
  // the chosen configuration (the starting one when something failed), and the
  // sketches back in their initial state
  int rc2 = ssd_tuning_set(ctx, rc == SSD_OK ? &best : &start);
  if (rc == SSD_OK) rc = rc2;
  cudaError_t e = cudaSuccess;
  const uint64_t bytes = ssd_sketch_bytes(ctx);
  for (int i = 0; i < n + 1 && e == cudaSuccess; ++i) {
    ssd_sketch* sk = i < n ? routers[i] : global;
    if (!sk) continue;
    e = reset_sketch(sk, bytes, st);
    sk->slot = 0;
  }
  // the tuning slots ran with no list capacity: clear the status they left
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->counters, 0, sizeof(ssd::DevCounters), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (int i = 0; i < 2; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess && rc == SSD_OK) rc = cuda_fail(e, "autotune reset");
  if (rc == SSD_OK && out) ssd_tuning_get(ctx, out);
  return rc;
}

}  // extern "C"
