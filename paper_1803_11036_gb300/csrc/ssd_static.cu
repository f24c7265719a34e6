// Regaining sliding super points with no allocation at all: the scratch the
// regain kernels need (hot-estimator pools, candidate tuple buffers, the list
// staging area and the counters) is carved out of one file-scope device array
// of fixed size instead of memory a context allocates.
//
// For callers that cannot allocate device memory: a process whose device memory
// is already claimed by another framework's caching allocator, or a datapath
// that must not pay cudaMalloc's implicit device synchronisation. They pass the
// parameter set, the hash tables and the recorders already in device memory,
// and the output buffers; nothing else is needed.
#include "ssd_internal.cuh"

namespace {

// The whole scratch budget. Every GPU that loads this library holds the array
// until the process exits.
constexpr uint64_t kStaticBytes = 32ull << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch on the caller's current device. In host code the array's
// name is only a host-side stand-in; the address comes from cudaGetSymbolAddress with that device
// current. It is looked up on every call, not cached: after cudaDeviceReset (or any new primary
// context) the module is loaded again and an address kept from before would be stale.
int static_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return SSD_ECUDA;
  }
  *out = p;
  return SSD_OK;
}

uint64_t up256(uint64_t x) { return (x + 255) & ~255ull; }

// Carve the array for one parameter set; SSD_ECAPACITY when the set needs more
// than the array holds.
struct Plan {
  uint64_t counters, n_out, hot_idx, pool_col, pool_rk, pool_bm, ctb0, ctb1, stage, end;
};

int plan_for(ssd::Dims& d, Plan& pl) {
  const uint64_t r = d.r, C = 1ull << d.q;
  d.out_cap = 1ull << 15;
  uint64_t at = 0;
  pl.counters = at; at = up256(at + sizeof(ssd::DevCounters));
  pl.n_out = at;    at = up256(at + 8);
  pl.hot_idx = at;  at = up256(at + r * C * 4);
  pl.stage = at;    at = up256(at + d.out_cap * 8);
  if (at > kStaticBytes / 2) return SSD_ECAPACITY;  // 2^q columns too many for the array
  uint64_t hse = C < 4096 ? C : 4096;
  const uint64_t per_hot = r * (8 + (uint64_t)d.words * 4);
  if (hse * per_hot > kStaticBytes / 4) hse = (kStaticBytes / 4) / per_hot;
  if (hse < 64) return SSD_ECAPACITY;             // estimators too wide for the array
  d.hse_cap = (uint32_t)hse;
  pl.pool_col = at; at = up256(at + r * hse * 4);
  pl.pool_rk = at;  at = up256(at + r * hse * 4);
  pl.pool_bm = at;  at = up256(at + r * hse * (uint64_t)d.words * 4);
  uint64_t ctb = (kStaticBytes - at - 512) / (2 * r * 4);
  if (ctb > (1ull << 20)) ctb = 1ull << 20;
  if (ctb < 1024) return SSD_ECAPACITY;
  d.ctb_cap = ctb;
  pl.ctb0 = at; at = up256(at + ctb * r * 4);
  pl.ctb1 = at; at = up256(at + ctb * r * 4);
  pl.end = at;
  return at <= kStaticBytes ? SSD_OK : SSD_ECAPACITY;
}

}  // namespace

extern "C" int ssd_regain_static(const ssd_params* p, uint32_t side, uint32_t group_bits, uint32_t group,
                                 const uint32_t* d_tables, const uint16_t* d_recorders, uint32_t* d_ips,
                                 uint32_t* d_rk, uint64_t cap, uint64_t* n_out, void* stream) {
  if (!p || !d_tables || !d_recorders || !n_out || (cap && (!d_ips || !d_rk))) return SSD_EINVAL;
  // the view of the sketch the recorders come from, checked as ssd_sketch_set_view checks it
  if (side > SSD_SIDE_ONET || group_bits > SSD_MAX_GROUP_BITS || (group >> group_bits)) return SSD_EINVAL;
  const uint32_t view = ssd::view_pack(side, group_bits, group);
  if (reinterpret_cast<uintptr_t>(d_recorders) & 15u) return SSD_EINVAL;
  if (ssd_params_check(p) != SSD_OK) return SSD_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SSD_ECUDA;
  ssd::Dims d{};
  d.log2_eta = p->log2_eta; d.q = p->q; d.r = p->r; d.delta = p->delta; d.k = p->k; d.flags = p->flags;
  if (ssd_threshold(p, &d.thr) != SSD_OK) return SSD_EINVAL;
  d.eta = 1u << p->log2_eta;
  d.words = d.eta / 32;
  d.col_mask = (1u << p->q) - 1u;
  d.low_bits = p->q - p->delta;
  d.low_mask = (1u << d.low_bits) - 1u;
  d.sh0 = (p->flags & SSD_RHFG_LITERAL) ? p->delta : 0u;
  Plan pl;
  int rc = plan_for(d, pl);
  if (rc != SSD_OK) return rc;
  void* base = nullptr;
  rc = static_address(&base);
  if (rc != SSD_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  ssd::Scratch s;
  s.tables = d_tables;
  s.hot_idx = reinterpret_cast<uint32_t*>(b + pl.hot_idx);
  s.pool_col = reinterpret_cast<uint32_t*>(b + pl.pool_col);
  s.pool_rk = reinterpret_cast<uint32_t*>(b + pl.pool_rk);
  s.pool_bm = reinterpret_cast<uint32_t*>(b + pl.pool_bm);
  s.ctb[0] = reinterpret_cast<uint32_t*>(b + pl.ctb0);
  s.ctb[1] = reinterpret_cast<uint32_t*>(b + pl.ctb1);
  s.stage = reinterpret_cast<unsigned long long*>(b + pl.stage);
  s.counters = reinterpret_cast<ssd::DevCounters*>(b + pl.counters);
  s.bucket_off = s.bucket_cnt = s.bucket_ent = nullptr;   // no room for the bucket index: probe hot_idx
  unsigned long long* nd = reinterpret_cast<unsigned long long*>(b + pl.n_out);
  d.touch_bits = 0;                          // no touch bits on this path
  d.dbg = SSD_DEBUG ? &s.counters->status : nullptr;

  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SSD_ECUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the counters must start at zero
  if (cudaMemsetAsync(s.counters, 0, sizeof(ssd::DevCounters), st) != cudaSuccess) return SSD_ECUDA;
  ssd::StreamArgs a{};
  a.n = 1;
  a.routers[0] = const_cast<uint16_t*>(d_recorders);
  a.global = nullptr;
  if (ssd::launch_stream(d, s, a, ssd::kHot, sms, ssd::default_tuning(), st) != cudaSuccess) return SSD_ECUDA;
  int launches = 0;
  if (ssd::launch_regain_tail(d, s, d_ips, d_rk, cap, nd, sms, st, &launches, view) != cudaSuccess)
    return SSD_ECUDA;
  ssd::DevCounters h;
  if (cudaMemcpyAsync(&h, s.counters, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SSD_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SSD_ECUDA;
  *n_out = h.n_out;
  if (h.status) return SSD_ECAPACITY;
  return SSD_OK;
}
