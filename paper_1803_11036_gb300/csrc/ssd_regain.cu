// Regaining sliding super points from the pooled hot estimators (Sec. 3.3 and
// Sec. 4.2, Algorithms 6-7 and the final test).
//
// Level 1 (pairs): every (he_0, he_1) of HSE(0) x HSE(1). With pruning, a pair
//   is kept only when the union of its two estimators still has R_k >= the
//   threshold: the union is an elementwise maximum, so R_k = popcount of the
//   AND of the "recorder < k" bitmaps, and it can only fall as rows are added;
//   a dropped tuple would fail the final test. Computed as a 32 x 32 tile of
//   AND-popcounts per block with the bitmaps staged in shared memory.
// Level i >= 2: the overlap test fixes the low q-delta bits of he_i
//   (B(i) mod 2^(q-delta) = B(i-1) >> delta with B(j) = he_0 XOR he_j), so the
//   only row-i estimators a candidate can extend to are the hot ones with those
//   low bits. The k_pairs launch also buckets each row's hot estimators by their
//   low q-delta bits, and a candidate reads its one bucket (when 2^(q-delta) is
//   too large for the index, it probes the 2^delta columns in hot_idx instead).
//   Hits are tested by the whole warp (coalesced bitmap reads) and survivors
//   are appended with warp-aggregated atomics.
// The last level applies the final test (R_k of the full union), regains the
//   host from B(1..r-1) and stages (cip, R_k); one block then sorts the staged
//   entries and writes the ascending, duplicate-free list.
#include "ssd_internal.cuh"

namespace ssd {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long warp_append(bool ok, unsigned long long* counter) {
  const unsigned mask = __ballot_sync(kFull, ok);
  if (!mask) return ~0ull;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  return ok ? base + __popc(mask & ((1u << lane) - 1u)) : ~0ull;
}

__device__ __forceinline__ uint32_t tab_hash_global(const uint32_t* T, uint32_t x) {
  return __ldg(T + (x & 255u)) ^ __ldg(T + 256u + ((x >> 8) & 255u)) ^ __ldg(T + 512u + ((x >> 16) & 255u)) ^
         __ldg(T + 768u + (x >> 24));
}

// The host whose q-bit windows (cip >> (j-1)*delta) mod 2^q are B(j) = he_0 ^ he_j,
// j = 1..r-1: bits [0, q) from B(1), then the top delta bits of each B(j) at
// (j-2)*delta + q. Consecutive windows already agree on their overlap, so the
// only way no host exists is a window bit at position 32 or beyond.
__device__ __forceinline__ bool regain_host(const Dims& d, const uint32_t* he, uint32_t* cip) {
  uint64_t v = he[0] ^ he[1];
  for (uint32_t j = 2; j < d.r; ++j) {
    const uint64_t top = (uint64_t)((he[0] ^ he[j]) >> d.low_bits);
    const uint32_t pos = (j - 2) * d.delta + d.q;
    if (pos >= 32) {
      if (top) return false;
    } else {
      v |= top << pos;
    }
  }
  if (v >> 32) return false;
  *cip = (uint32_t)v;
  return true;
}

// Row i's pooled hot estimators bucketed by the low q-delta bits of their column
// (one block; counting sort in global memory: count, exclusive scan, fill). The
// order inside a bucket is that of the fill's atomics; the levels do not depend
// on it (the list is sorted at the end).
__device__ void build_buckets(const Dims& d, const Scratch& s, uint32_t i) {
  __shared__ uint32_t part[kBlock];
  const uint32_t nb = 1u << d.low_bits;
  uint32_t* off = s.bucket_off + (uint64_t)i * (nb + 1);
  uint32_t* cnt = s.bucket_cnt + (uint64_t)i * nb;
  uint32_t* ent = s.bucket_ent + (uint64_t)i * d.hse_cap;
  const uint32_t* col = s.pool_col + (uint64_t)i * d.hse_cap;
  const uint32_t n = min(s.counters->hot[i], d.hse_cap);
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) atomicAdd(&cnt[col[j] & d.low_mask], 1u);
  __syncthreads();
  // exclusive scan: each thread sums a contiguous segment, the block scans the sums
  const uint32_t seg = (nb + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(threadIdx.x * seg, nb), hi = min(lo + seg, nb);
  uint32_t sum = 0;
  for (uint32_t b = lo; b < hi; ++b) sum += cnt[b];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (uint32_t o = 1; o < blockDim.x; o <<= 1) {   // inclusive Hillis-Steele scan of the sums
    const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (uint32_t b = lo; b < hi; ++b) {
    const uint32_t c = cnt[b];
    off[b] = run;
    cnt[b] = run;   // the fill's cursor
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) off[nb] = part[blockDim.x - 1];
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) ent[atomicAdd(&cnt[col[j] & d.low_mask], 1u)] = j;
}

constexpr int TA = 32, KW = 64;

// Blocks [0, pair_blocks) test the pairs; with the bucket index, block
// pair_blocks + m builds the buckets of row 2 + m.
__global__ void __launch_bounds__(kBlock) k_pairs(const Dims d, const Scratch s, uint32_t pair_blocks) {
  if (blockIdx.x >= pair_blocks) {
    build_buckets(d, s, 2 + (blockIdx.x - pair_blocks));
    return;
  }
  __shared__ uint32_t A[TA][KW + 1], B[TA][KW + 1];
  const uint32_t n0 = min(s.counters->hot[0], d.hse_cap);
  const uint32_t n1 = min(s.counters->hot[1], d.hse_cap);
  const uint64_t t1 = (n1 + TA - 1) / TA;
  const uint64_t ntiles = (uint64_t)((n0 + TA - 1) / TA) * t1;
  const bool prune = !(d.flags & SSD_NO_PRUNE);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const uint32_t* bm0 = s.pool_bm;
  const uint32_t* bm1 = s.pool_bm + (uint64_t)d.hse_cap * d.words;
  for (uint64_t t = blockIdx.x; t < ntiles; t += pair_blocks) {
    const uint32_t a0 = (uint32_t)(t / t1) * TA, b0 = (uint32_t)(t % t1) * TA;
    uint32_t acc[2][2] = {{0, 0}, {0, 0}};
    if (prune) {
      for (uint32_t k0 = 0; k0 < d.words; k0 += KW) {
        const uint32_t kw = d.words - k0 < (uint32_t)KW ? d.words - k0 : (uint32_t)KW;
        __syncthreads();
        for (int e = threadIdx.x; e < TA * KW; e += kBlock) {
          const int rr = e / KW, cc = e % KW;
          const bool in = cc < (int)kw;
          A[rr][cc] = (in && a0 + rr < n0) ? bm0[(uint64_t)(a0 + rr) * d.words + k0 + cc] : 0u;
          B[rr][cc] = (in && b0 + rr < n1) ? bm1[(uint64_t)(b0 + rr) * d.words + k0 + cc] : 0u;
        }
        __syncthreads();
        for (uint32_t cc = 0; cc < kw; ++cc) {
          const uint32_t x0 = A[2 * ty][cc], x1 = A[2 * ty + 1][cc];
          const uint32_t y0 = B[2 * tx][cc], y1 = B[2 * tx + 1][cc];
          acc[0][0] += __popc(x0 & y0);
          acc[0][1] += __popc(x0 & y1);
          acc[1][0] += __popc(x1 & y0);
          acc[1][1] += __popc(x1 & y1);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const uint32_t ia = a0 + 2 * ty + u, ib = b0 + 2 * tx + v;
        const bool ok = ia < n0 && ib < n1 && (!prune || acc[u][v] >= d.thr);
        const unsigned long long pos = warp_append(ok, &s.counters->level[1]);
        if (ok) {
          if (pos < d.ctb_cap) {
            s.ctb[0][pos * d.r + 0] = ia;
            s.ctb[0][pos * d.r + 1] = ib;
          } else {
            atomicOr(&s.counters->status, SSD_STATUS_CTB_OVERFLOW);
          }
        }
      }
  }
}

// One candidate tuple c of row level i extended by row-i estimator idx (pool
// index; kNone when this lane has none): the union test by the whole warp, then
// the append to the next candidate buffer or, at the last row, the final test,
// the host and its staging. Every lane of the warp makes the call.
__device__ __forceinline__ void level_hit(const Dims& d, const Scratch& s, uint32_t i, const uint32_t* rctb,
                                          uint32_t* sctb, uint64_t c, uint32_t idx, int lane) {
  const uint64_t cap = d.hse_cap;
  const bool last = (i == d.r - 1);
  const bool prune = !(d.flags & SSD_NO_PRUNE);
  const bool verify = (d.flags & SSD_VERIFY_H0) != 0;
  const bool hit = idx != kNone;
  uint32_t pc = 0;
  if (prune || last) {
    unsigned m = __ballot_sync(kFull, hit);
    while (m) {
      const int L = __ffs(m) - 1;
      m &= m - 1;
      const uint64_t cL = __shfl_sync(kFull, c, L);
      const uint32_t idxL = __shfl_sync(kFull, idx, L);
      const uint32_t* tL = rctb + cL * d.r;
      uint32_t sum = 0;
      for (uint32_t w = lane; w < d.words; w += 32) {
        uint32_t x = s.pool_bm[((uint64_t)i * cap + idxL) * d.words + w];
        for (uint32_t j = 0; j < i; ++j) x &= s.pool_bm[((uint64_t)j * cap + tL[j]) * d.words + w];
        sum += __popc(x);
      }
      sum = __reduce_add_sync(kFull, sum);
      if (lane == L) pc = sum;
    }
  }
  const bool keep = hit && (!prune || pc >= d.thr);
  if (!last) {
    const unsigned long long pos = warp_append(keep, &s.counters->level[i]);
    if (keep) {
      if (pos < d.ctb_cap) {
        const uint32_t* tup = rctb + c * d.r;
        for (uint32_t j = 0; j < i; ++j) sctb[pos * d.r + j] = tup[j];
        sctb[pos * d.r + i] = idx;
      } else {
        atomicOr(&s.counters->status, SSD_STATUS_CTB_OVERFLOW);
      }
    }
  } else {
    warp_append(keep, &s.counters->level[i]);
    bool acc = hit && pc >= d.thr;
    uint32_t cip = 0;
    if (acc) {
      const uint32_t* tup = rctb + c * d.r;
      uint32_t he[SSD_MAX_R];
      for (uint32_t j = 0; j < i; ++j) he[j] = s.pool_col[(uint64_t)j * cap + tup[j]];
      he[i] = s.pool_col[(uint64_t)i * cap + idx];
      acc = regain_host(d, he, &cip);
      if (acc && verify) acc = (tab_hash_global(s.tables + 1024, cip) & d.col_mask) == he[0];
    }
    const unsigned long long pos = warp_append(acc, &s.counters->raw);
    if (acc) {
      if (pos < d.out_cap) s.stage[pos] = ((unsigned long long)cip << 32) | pc;
      else atomicOr(&s.counters->status, SSD_STATUS_OUT_OVERFLOW);
    }
  }
}

// The low q-delta bits the overlap test fixes for row i's estimator of candidate c.
__device__ __forceinline__ uint32_t fixed_low(const Dims& d, const Scratch& s, uint32_t i, const uint32_t* tup) {
  const uint32_t he0 = s.pool_col[tup[0]];
  const uint32_t hep = s.pool_col[(uint64_t)(i - 1) * d.hse_cap + tup[i - 1]];
  const uint32_t want_low = (he0 ^ hep) >> d.delta;  // high q-delta bits of B(i-1)
  return (he0 ^ want_low) & d.low_mask;
}

__global__ void __launch_bounds__(kBlock) k_level(const Dims d, const Scratch s, const uint32_t i,
                                                  const uint32_t* __restrict__ rctb, uint32_t* __restrict__ sctb) {
  const int lane = threadIdx.x & 31;
  const unsigned long long avail = s.counters->level[i - 1];
  const uint64_t nc = avail < d.ctb_cap ? avail : d.ctb_cap;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if (s.bucket_off) {
    // one candidate per lane; round p takes each lane's p-th bucket entry
    const uint32_t nb = 1u << d.low_bits;
    const uint32_t* off = s.bucket_off + (uint64_t)i * (nb + 1);
    const uint32_t* ent = s.bucket_ent + (uint64_t)i * d.hse_cap;
    for (uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < nc; w0 += stride) {
      const uint64_t c = w0 + lane;
      uint32_t b = 0, e = 0;
      if (c < nc) {
        const uint32_t low = fixed_low(d, s, i, rctb + c * d.r);
        b = off[low];
        e = off[low + 1];
      }
      for (uint32_t p = 0; __any_sync(kFull, b + p < e); ++p)
        level_hit(d, s, i, rctb, sctb, c, b + p < e ? ent[b + p] : kNone, lane);
    }
    return;
  }
  // probes: 2^delta columns of row i per candidate, one per lane
  const uint64_t total = nc << d.delta;
  for (uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < total; w0 += stride) {
    const uint64_t item = w0 + lane;
    const uint64_t c = item >> d.delta;
    uint32_t idx = kNone;
    if (item < total) {
      const uint32_t h = (uint32_t)(item & ((1u << d.delta) - 1u));
      const uint32_t he_i = (h << d.low_bits) | fixed_low(d, s, i, rctb + c * d.r);
      idx = s.hot_idx[((uint64_t)i << d.q) | he_i];
    }
    level_hit(d, s, i, rctb, sctb, c, idx, lane);
  }
}

constexpr int kListThreads = 1024;
constexpr uint32_t kSmemKeys = 16384;

__device__ void bitonic(unsigned long long* keys, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = keys[i], b = keys[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// One block: sort the staged (cip << 32 | R_k) keys, keep the last entry of each
// cip (its largest R_k), and write the list when it fits the caller's capacity.
__global__ void __launch_bounds__(kListThreads) k_list(const Dims d, const Scratch s, uint32_t* ips, uint32_t* rk,
                                                       uint64_t cap, unsigned long long* n_out_dev) {
  extern __shared__ unsigned long long skeys[];
  __shared__ unsigned int warp_cnt[kListThreads / 32];
  __shared__ unsigned long long running;
  const unsigned long long raw = s.counters->raw;
  const uint32_t n = (uint32_t)(raw < d.out_cap ? raw : d.out_cap);
  uint32_t P = 1;
  while (P < n) P <<= 1;
  unsigned long long* keys;
  if (P <= kSmemKeys) {
    keys = skeys;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) keys[i] = i < n ? s.stage[i] : ~0ull;
  } else {
    keys = s.stage;
    for (uint32_t i = n + threadIdx.x; i < P; i += blockDim.x) keys[i] = ~0ull;
  }
  __syncthreads();
  bitonic(keys, P);
  // count unique hosts
  unsigned long long uniq = 0;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const bool f = i < n && (i + 1 == n || (keys[i] >> 32) != (keys[i + 1] >> 32));
    uniq += __syncthreads_count(f);
  }
  if (threadIdx.x == 0) {
    *n_out_dev = uniq;
    s.counters->n_out = uniq;
    if (uniq > cap) atomicOr(&s.counters->status, SSD_STATUS_LIST_OVERFLOW);
    running = 0;
  }
  if (uniq > cap) return;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const bool f = i < n && (i + 1 == n || (keys[i] >> 32) != (keys[i + 1] >> 32));
    const unsigned m = __ballot_sync(kFull, f);
    if (lane == 0) warp_cnt[wid] = __popc(m);
    __syncthreads();
    unsigned long long off = running;
    for (int w = 0; w < wid; ++w) off += warp_cnt[w];
    if (f) {
      const unsigned long long pos = off + __popc(m & ((1u << lane) - 1u));
      ips[pos] = (uint32_t)(keys[i] >> 32);
      rk[pos] = (uint32_t)keys[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kListThreads / 32; ++w) t += warp_cnt[w];
      running += t;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_regain_tail(const Dims& d, const Scratch& s, uint32_t* ips, uint32_t* rk, uint64_t cap,
                               unsigned long long* n_out_dev, int sms, cudaStream_t st, int* launches) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSmemKeys * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  static int pair_bps = 0;   // resident k_pairs blocks per SM
  if (!pair_bps) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pair_bps, k_pairs, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (pair_bps < 1) pair_bps = 1;
  }
  const uint32_t pair_blocks = (uint32_t)(sms * pair_bps);
  const uint32_t bucket_blocks = s.bucket_off && d.r > 2 ? d.r - 2 : 0;
  k_pairs<<<pair_blocks + bucket_blocks, kBlock, 0, st>>>(d, s, pair_blocks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *launches += 1;
  for (uint32_t i = 2; i < d.r; ++i) {
    // level 1 (pairs) wrote ctb[0]; level i reads ctb[i & 1] and writes ctb[(i + 1) & 1]
    const uint32_t* rctb = s.ctb[i & 1];
    uint32_t* sctb = s.ctb[(i + 1) & 1];
    k_level<<<sms * 8, kBlock, 0, st>>>(d, s, i, rctb, sctb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
  }
  k_list<<<1, kListThreads, kSmemKeys * sizeof(unsigned long long), st>>>(d, s, ips, rk, cap, n_out_dev);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace ssd
