// Streaming passes over whole RSEAs: merge (Algorithm 5), hot-estimator
// extraction (Sec. 3.3) and the distance recorder update (Sec. 4.3).
//
// One kernel serves every combination: for each recorder position it reads the
// n routers' values (16 bytes = 8 recorders per lane), optionally sets the
// recorders whose touch bit is set to distance 0 first (Algorithm 2 deferred
// from the scan of the fused slot; the bit is cleared), takes the elementwise
// minimum distance over routers (the merge), optionally writes that to the
// global RSEA, optionally counts the merged recorders below k per estimator and
// pools the hot ones with their "recorder < k" bitmap, and optionally advances
// every router by one slot. The recorders are stamps (ssd_internal.cuh): the
// advance itself is the clock's tick, so a router's vector is written back only
// when one of its recorders was set by a touch or reaches distance 65535.
// Recorders are read once per pass, in 512-byte coalesced warp accesses with
// streaming cache hints; the touch bits stay in L2.
#include "ssd_internal.cuh"

namespace ssd {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint4 min8(uint4 a, uint4 b) {
  return make_uint4(__vminu2(a.x, b.x), __vminu2(a.y, b.y), __vminu2(a.z, b.z), __vminu2(a.w, b.w));
}
__device__ __forceinline__ uint4 or8(uint4 a, uint4 b) { return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w); }
__device__ __forceinline__ bool any8(uint4 a) { return (a.x | a.y | a.z | a.w) != 0u; }
// bit i of the result = (distance i < k) for the 8 distances of v
__device__ __forceinline__ uint32_t lt2(uint32_t w, uint32_t kk) {
  const uint32_t k = kk & 0xFFFFu;
  return (uint32_t)((w & 0xFFFFu) < k) | ((uint32_t)((w >> 16) < k) << 1);
}
__device__ __forceinline__ uint32_t lt8(uint4 v, uint32_t kk) {
  return lt2(v.x, kk) | (lt2(v.y, kk) << 2) | (lt2(v.z, kk) << 4) | (lt2(v.w, kk) << 6);
}

// The clock of router j of a pass: its tm and expiry stamp in both halves (stamp recorders), or
// tm2 = 0 and `stamps` false when the pass reads distances.
struct RouterClock {
  uint32_t tm2, xe2;
};
__device__ __forceinline__ RouterClock router_clock(const uint32_t* tm) {
  RouterClock rc;
  const uint32_t t = read_tm(tm), xe = tm_next(t);
  rc.tm2 = t | (t << 16);
  rc.xe2 = xe | (xe << 16);
  return rc;
}

// Pool a hot estimator: reserve a slot in its row's pool and return it
// (kNone when the pool is full).
__device__ __forceinline__ uint32_t pool_slot(const Dims& d, const Scratch& s, uint32_t row) {
  uint32_t idx = atomicAdd(&s.counters->hot[row], 1u);
  if (idx >= d.hse_cap) {
    atomicOr(&s.counters->status, SSD_STATUS_HSE_OVERFLOW);
    idx = kNone;
  }
  return idx;
}

// Touch bits of router j for 8 recorders (one byte), cleared after reading.
__device__ __forceinline__ uint32_t take_touch(uint8_t* p) {
  const uint32_t t = *p;
  if (t) *p = 0;
  return t;
}

// Recorder vectors it0 .. it0+m-1 (m <= 8, 32 lanes x 8 recorders each) of the
// estimator at `base`. All loads of a group are issued before any store of it (a
// store in between could alias the next load and serialise them).
__device__ __forceinline__ void load_group(const uint4* r0, uint64_t base, uint32_t it0, uint32_t m, int lane,
                                           uint4 (&v)[8]) {
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (u < (int)m) v[u] = __ldcs(r0 + base + (it0 + u) * 32 + lane);
}

// kNever into the recorders of v holding the stamp xe. Out of line: a recorder expires once in
// 65535 slots, and a call keeps this from being if-converted into every vector's path.
__device__ __noinline__ uint4 expire_vec(uint4 v, uint32_t xe2) {
  return make_uint4(v.x | __vcmpeq2(v.x, xe2), v.y | __vcmpeq2(v.y, xe2), v.z | __vcmpeq2(v.z, xe2),
                    v.w | __vcmpeq2(v.w, xe2));
}

// The touch bytes of a lane's m vectors (m = 1, 2, 4 or 8; byte u of the result for its u-th
// vector), contiguous and aligned to m bytes by touch_pos, and their clearing.
__device__ __forceinline__ uint64_t load_touch(const uint8_t* p, uint32_t m) {
  if (m == 8) return __ldcg(reinterpret_cast<const unsigned long long*>(p));
  if (m == 4) return __ldcg(reinterpret_cast<const unsigned int*>(p));
  if (m == 2) return __ldcg(reinterpret_cast<const unsigned short*>(p));
  return __ldcg(p);
}
// (cleared only when `any`, by a predicated store: no branch around it)
__device__ __forceinline__ void clear_touch(uint8_t* p, uint32_t m, bool any) {
  const uint32_t c = any ? 1u : 0u;
  if (m == 8)
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %1, 0; @q st.global.u64 [%0], 0; }" :: "l"(p), "r"(c) : "memory");
  else if (m == 4)
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %1, 0; @q st.global.u32 [%0], 0; }" :: "l"(p), "r"(c) : "memory");
  else if (m == 2)
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %1, 0; @q st.global.u16 [%0], 0; }" :: "l"(p), "r"(c) : "memory");
  else
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %1, 0; @q st.global.u8 [%0], 0; }" :: "l"(p), "r"(c) : "memory");
}

// __stcs(p, v) when c: a predicated store, so the lanes that write and those that do not need no
// branch (and no reconvergence) between them.
__device__ __forceinline__ void stcs_if(uint4* p, uint4 v, bool c) {
  asm volatile("{ .reg .pred q; setp.ne.u32 q, %5, 0; @q st.global.cs.v4.u32 [%0], {%1, %2, %3, %4}; }"
               :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(c ? 1u : 0u) : "memory");
}

// The loaded group of one router's stamps: touch bits applied (tw: the group's touch bytes, from
// load_touch; those recorders take the stamp tm, distance 0, through the masks of the table tmask,
// built by touch_mask_entry; the caller clears the bytes), the state written to g, the recorders
// inside the window counted (out2), and the vectors that changed written back: a recorder set by
// a touch, or, with ADV, one whose distance reaches 65535 at this advance (it becomes kNever).
// The common path has no divergent branch: touched vectors are stored by predicated stores, and
// the expiry (any_eq8 per vector) is taken once for the group behind a warp vote, reading back the
// vectors it rewrites. No window bits are written: the caller builds them with group_bits only
// for a hot estimator. Returns the lane's count of recorders inside the window.
template <bool ADV, bool HOT, bool TOUCH, bool WRAP>
__device__ __forceinline__ uint32_t fast_group_w(uint4* r0, uint4* g, uint64_t base, uint32_t it0, uint32_t m,
                                                 int lane, const Clock& c, const uint4* tmask, uint4 (&v)[8],
                                                 uint64_t tw) {
  uint32_t out = 0;   // recorders outside the window, per half, in two 16-bit fields
  uint32_t expiring = 0;   // bit u: vector u holds a recorder with the stamp xe
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (u < (int)m) {
      const uint64_t at = base + (it0 + u) * 32 + lane;
      if (TOUCH) {
        const uint32_t t = (uint32_t)(tw >> (8 * u)) & 0xFFu;
        v[u] = set_masked(v[u], tmask[t], c.tm2);
        stcs_if(r0 + at, v[u], t != 0u);
      }
      if (g) __stcs(g + at, v[u]);
      if (HOT) out += out2<WRAP>(v[u].x, c) + out2<WRAP>(v[u].y, c) + out2<WRAP>(v[u].z, c) + out2<WRAP>(v[u].w, c);
      if (ADV) expiring |= any_eq8(v[u], c.xe2) ? 1u << u : 0u;
    }
  }
  if (ADV && __any_sync(kFull, expiring != 0u)) {   // once in 65535 slots per recorder
    for (uint32_t u = 0; u < m; ++u) {
      if ((expiring >> u) & 1u) {
        const uint64_t at = base + (it0 + u) * 32 + lane;
        __stcs(r0 + at, expire_vec(__ldcg(r0 + at), c.xe2));   // the lane's own (touched) vector
      }
    }
  }
  return 8u * m - (out & 0xFFFFu) - (out >> 16);
}
// fast_group with the window's form chosen once for the group (c.wrap is the same for the grid).
template <bool ADV, bool HOT, bool TOUCH>
__device__ __forceinline__ uint32_t fast_group(uint4* r0, uint4* g, uint64_t base, uint32_t it0, uint32_t m,
                                               int lane, const Clock& c, const uint4* tmask, uint4 (&v)[8],
                                               uint64_t tw) {
  if (HOT && c.wrap) return fast_group_w<ADV, HOT, TOUCH, true>(r0, g, base, it0, m, lane, c, tmask, v, tw);
  return fast_group_w<ADV, HOT, TOUCH, false>(r0, g, base, it0, m, lane, c, tmask, v, tw);
}

// The window bits of a group fast_group has processed, to `my`, from the recorders read again one
// vector at a time (the lane reads back the vectors it stored itself; a hot estimator is rare, so
// nothing is kept live in registers for it). A recorder the advance expired holds kNever, outside the window, as its
// stamp xe was.
__device__ __forceinline__ void group_bits(const uint4* r0, uint64_t base, uint32_t it0, uint32_t m, uint8_t* my,
                                           int lane, const Clock& c) {
#pragma unroll 1
  for (uint32_t u = 0; u < m; ++u)
    my[(it0 + u) * 32 + lane] = (uint8_t)win8(__ldcg(r0 + base + (it0 + u) * 32 + lane), c);
}

// The window bits of every group of an estimator whose warp-wide count reaches the threshold.
__device__ __forceinline__ void hot_bits(const Dims& d, const uint4* r0, uint64_t base, uint32_t cnt, uint8_t* my,
                                         int lane, const Clock& c) {
  if (__reduce_add_sync(kFull, cnt) < d.thr) return;   // warp-uniform
  const uint32_t iters = d.eta >> 8;
  for (uint32_t it0 = 0; it0 < iters; it0 += 8) group_bits(r0, base, it0, iters - it0 < 8u ? iters - it0 : 8u, my, lane, c);
}

// One estimator of one router, all eta recorders (eta >= 256), in groups of 8 vectors per lane:
// load_group then fast_group, then the window bits only when the warp's count reaches the
// threshold (pool_if_hot pools it). tb: this lane's touch bytes of the estimator (touch_pos).
template <bool ADV, bool HOT, bool TOUCH>
__device__ __forceinline__ uint32_t one_router_se(const Dims& d, uint4* r0, uint4* g, uint64_t base, uint8_t* tb,
                                                  uint8_t* my, int lane, const Clock& c, const uint4* tmask) {
  const uint32_t iters = d.eta >> 8;
  uint32_t cnt = 0;
  for (uint32_t it0 = 0; it0 < iters; it0 += 8) {
    const uint32_t m = iters - it0 < 8u ? iters - it0 : 8u;
    uint4 v[8];
    load_group(r0, base, it0, m, lane, v);
    const uint64_t tw = TOUCH ? load_touch(tb + it0, m) : 0ull;
    cnt += fast_group<ADV, HOT, TOUCH>(r0, g, base, it0, m, lane, c, tmask, v, tw);
    if (TOUCH) clear_touch(tb + it0, m, tw != 0ull);
  }
  if (HOT) hot_bits(d, r0, base, cnt, my, lane, c);
  return cnt;
}

// Pool estimator se when its warp-wide count reaches the threshold (bitmap from `my`).
__device__ __forceinline__ void pool_if_hot(const Dims& d, const Scratch& s, uint64_t se, uint32_t cnt,
                                            const uint8_t* my, int lane) {
  cnt = __reduce_add_sync(kFull, cnt);
  const uint32_t row = (uint32_t)(se >> d.q), col = (uint32_t)se & d.col_mask;
  uint32_t idx = kNone;
  if (cnt >= d.thr) {  // warp-uniform
    if (lane == 0) idx = pool_slot(d, s, row);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx != kNone) {
      __syncwarp();
      const uint32_t* mw = reinterpret_cast<const uint32_t*>(my);
      uint32_t* dst = s.pool_bm + ((uint64_t)row * d.hse_cap + idx) * d.words;
      for (uint32_t w = lane; w < d.words; w += 32) dst[w] = mw[w];
      if (lane == 0) {
        s.pool_col[(uint64_t)row * d.hse_cap + idx] = col;
        s.pool_rk[(uint64_t)row * d.hse_cap + idx] = cnt;
      }
    }
  }
  if (lane == 0 && in_bounds(d, se < ((uint64_t)d.r << d.q))) s.hot_idx[se] = idx;
  __syncwarp();
}

// eta >= 256: one warp per estimator, iters = eta/256 steps of 32 lanes x 8 recorders.
// G (several routers): routers loaded per group before any of them is stored. One router works on
// its stamps directly (window test, expiry); several routers are merged as distances (each
// router's stamps through its own clock), and the global RSEA takes router 0's clock.
template <bool ONE, bool ADV, bool HOT, bool TOUCH, int G>
__global__ void __launch_bounds__(kBlock, ONE ? 4 : 3) k_stream_large(const Dims d, const Scratch s,
                                                         const __grid_constant__ StreamArgs a) {
  extern __shared__ __align__(16) uint8_t smask[];
  __shared__ RouterClock sck[ONE ? 1 : kMaxBatch];
  __shared__ uint4 stm[ONE && TOUCH ? 256 : 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* my = smask + (size_t)wid * (d.eta >> 3);
  const uint64_t count = a.se_count ? a.se_count : ((uint64_t)d.r << d.q);
  const uint64_t se_end = a.se0 + count;
  const uint32_t iters = d.eta >> 8;
  const uint32_t kk = d.k | (d.k << 16);
  const uint64_t wstride = (uint64_t)gridDim.x * (kBlock / 32);
  const uint64_t tstride = count * (d.eta >> 3);  // touch bytes per router
  uint4* const g = reinterpret_cast<uint4*>(a.global);
  const bool stamps = a.tm[0] != nullptr;
  const uint32_t tm0 = read_tm(a.tm[0]);
  const Clock c = stamps ? make_clock(tm0, d.k) : distance_clock(d.k);
  if (a.global_tm && blockIdx.x == 0 && threadIdx.x == 0) *a.global_tm = tm0;
  if (!ONE) {
    for (int j = threadIdx.x; j < a.n; j += blockDim.x) sck[j] = router_clock(a.tm[j]);
    __syncthreads();
  }
  if (ONE && TOUCH) {
    for (int j = threadIdx.x; j < 256; j += blockDim.x) stm[j] = touch_mask_entry((uint32_t)j);
    __syncthreads();
  }

  for (uint64_t se = a.se0 + (uint64_t)blockIdx.x * (kBlock / 32) + wid; se < se_end; se += wstride) {
    const uint64_t base = (se << d.log2_eta) >> 3;  // in 8-recorder units
    uint8_t* tb = TOUCH ? a.touch + (se - a.se0) * (d.eta >> 3) + lane * iters : nullptr;   // touch_pos
    uint32_t cnt = 0;
    if (ONE) {
      uint4* const r0 = reinterpret_cast<uint4*>(a.routers[0]);
      cnt = one_router_se<ADV, HOT, TOUCH>(d, r0, g, base, tb, my, lane, c, stm);
    } else {
      for (uint32_t it = 0; it < iters; ++it) {
        const uint64_t at = base + it * 32 + lane;
        uint4 mv = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);   // distances
        // routers in groups of G: the group's loads are issued before any of its stores
        for (int n0 = 0; n0 < a.n; n0 += G) {
          const int m = a.n - n0 < G ? a.n - n0 : G;
          uint4 v[G];
          uint32_t t[G];
#pragma unroll
          for (int u = 0; u < G; ++u) {
            if (u < m) {
              v[u] = __ldcs(reinterpret_cast<uint4*>(a.routers[n0 + u]) + at);
              if (TOUCH) t[u] = tb[(uint64_t)(n0 + u) * tstride + it];
            }
          }
#pragma unroll
          for (int u = 0; u < G; ++u) {
            if (u < m) {
              const RouterClock rc = sck[n0 + u];
              bool dirty = false;
              if (TOUCH && t[u]) {
                v[u] = set8(v[u], t[u], rc.tm2);
                tb[(uint64_t)(n0 + u) * tstride + it] = 0;
                dirty = true;
              }
              mv = min8(mv, stamps ? flip8(v[u], rc.tm2) : v[u]);
              if (ADV) {
                const uint4 e = make_uint4(__vcmpeq2(v[u].x, rc.xe2), __vcmpeq2(v[u].y, rc.xe2),
                                           __vcmpeq2(v[u].z, rc.xe2), __vcmpeq2(v[u].w, rc.xe2));
                if (any8(e)) {
                  v[u] = or8(v[u], e);
                  dirty = true;
                }
              }
              if (dirty) __stcs(reinterpret_cast<uint4*>(a.routers[n0 + u]) + at, v[u]);
            }
          }
        }
        if (g) __stcs(g + at, stamps ? flip8(mv, c.tm2) : mv);
        if (HOT) {
          const uint32_t bits = lt8(mv, kk);
          cnt += __popc(bits);
          my[it * 32 + lane] = (uint8_t)bits;
        }
      }
    }
    if (HOT) pool_if_hot(d, s, se, cnt, my, lane);
  }
}

// 32 <= eta <= 128: L = eta/8 lanes per estimator, 32/L estimators per warp step. Routers are
// merged as distances (each router's stamps through its own clock).
template <bool ONE, bool ADV, bool HOT, bool TOUCH>
__global__ void __launch_bounds__(kBlock) k_stream_small(const Dims d, const Scratch s,
                                                         const __grid_constant__ StreamArgs a) {
  __shared__ RouterClock sck[ONE ? 1 : kMaxBatch];
  const int lane = threadIdx.x & 31;
  const uint32_t L = d.eta >> 3;
  const uint32_t per_warp = 32u / L;
  const uint64_t count = a.se_count ? a.se_count : ((uint64_t)d.r << d.q);
  const uint64_t u0 = a.se0 / per_warp;         // se0 and count are multiples of per_warp
  const uint64_t n_units = count / per_warp;
  const uint32_t kk = d.k | (d.k << 16);
  const uint64_t wstride = (uint64_t)gridDim.x * (kBlock / 32);
  const uint64_t tstride = count * (d.eta >> 3);
  uint4* const g = reinterpret_cast<uint4*>(a.global);
  uint8_t* const bm_bytes = reinterpret_cast<uint8_t*>(s.pool_bm);
  const bool stamps = a.tm[0] != nullptr;
  if (a.global_tm && blockIdx.x == 0 && threadIdx.x == 0) *a.global_tm = read_tm(a.tm[0]);
  for (int j = threadIdx.x; j < (ONE ? 1 : a.n); j += blockDim.x) sck[j] = router_clock(a.tm[j]);
  __syncthreads();

  // router n's vector at `at`: touch applied, written back when it changed; returns its distances
  auto one = [&](int n, uint64_t at, uint8_t* t8) {
    const RouterClock rc = sck[n];
    uint4* rp = reinterpret_cast<uint4*>(a.routers[n]);
    uint4 v = __ldcs(rp + at);
    bool dirty = false;
    if (TOUCH) {
      const uint32_t t = take_touch(t8);
      if (t) {
        v = set8(v, t, rc.tm2);
        dirty = true;
      }
    }
    const uint4 dist = stamps ? flip8(v, rc.tm2) : v;
    if (ADV) {
      const uint4 e = make_uint4(__vcmpeq2(v.x, rc.xe2), __vcmpeq2(v.y, rc.xe2), __vcmpeq2(v.z, rc.xe2),
                                 __vcmpeq2(v.w, rc.xe2));
      if (any8(e)) {
        v = or8(v, e);
        dirty = true;
      }
    }
    if (dirty) __stcs(rp + at, v);
    return dist;
  };

  for (uint64_t uu = (uint64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); uu < n_units; uu += wstride) {
    const uint64_t u = u0 + uu;
    const uint64_t at = u * 32 + lane;
    uint8_t* tb = TOUCH ? a.touch + uu * 32 + lane : nullptr;  // byte of these 8 recorders, router 0
    uint4 mv = one(0, at, tb);
    if (!ONE) {
      for (int n = 1; n < a.n; ++n) mv = min8(mv, one(n, at, TOUCH ? tb + n * tstride : nullptr));
    }
    if (g) __stcs(g + at, stamps ? flip8(mv, sck[0].tm2) : mv);
    if (HOT) {
      const uint32_t bits = lt8(mv, kk);
      uint32_t cnt = __popc(bits);
      for (uint32_t o = 1; o < L; o <<= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
      const uint64_t se = u * per_warp + lane / L;
      const uint32_t row = (uint32_t)(se >> d.q), col = (uint32_t)se & d.col_mask;
      const uint32_t leader = lane & ~(L - 1);
      uint32_t idx = kNone;
      if (lane == leader && cnt >= d.thr) idx = pool_slot(d, s, row);
      idx = __shfl_sync(kFull, idx, leader);
      if (idx != kNone) {
        bm_bytes[((uint64_t)row * d.hse_cap + idx) * (d.eta >> 3) + (lane - leader)] = (uint8_t)bits;
        if (lane == leader) {
          s.pool_col[(uint64_t)row * d.hse_cap + idx] = col;
          s.pool_rk[(uint64_t)row * d.hse_cap + idx] = cnt;
        }
      }
      if (lane == leader) s.hot_idx[se] = idx;
    }
  }
}

// Where a chunk launch finds the touches of the next chunk.
constexpr int kSrcNone = 0;     // the last chunk: nothing to collect
constexpr int kSrcRaw = 1;      // the slot's raw pairs, hashed here (tables in shared memory)
constexpr int kSrcPacked = 2;   // the slot's pre-hashed pairs (RHFG[0] | H1 << q)
constexpr int kSrcList = 3;     // the next chunk's touch list: bit indices written once per slot

// One chunk of the fused slot of one router (eta >= 256): each warp streams
// estimators of the chunk with their touch bits applied, counts and pools hot
// ones and writes back the vectors that changed (touched or expired); unless SRC is kSrcNone, between estimators each lane also
// sets a share of the next chunk's touch bits (L2 atomics that fill the gaps of
// the memory-bound stream), from the next chunk's touch list or by hashing a
// share of the slot's pairs. The pairs or list entries are walked warp by warp
// (warp e takes e*32 + lane, e*32 + lane + 32*count, ...), so every lane of a
// warp runs the same iterations, as combine mode 1 needs.
template <int SRC, int CM>
__global__ void __launch_bounds__(kBlock, 3) k_chunk(const Dims d, const Scratch s,
                                                     const __grid_constant__ ChunkArgs a) {
  constexpr bool NEXT = SRC != kSrcNone;
  constexpr bool PACKED = SRC == kSrcPacked;
  constexpr bool LIST = SRC == kSrcList;
  constexpr bool TABLES = SRC == kSrcRaw;   // raw pairs are hashed here; pre-hashed ones are not
  // Programmatic dependent launch: the next chunk's grid may be scheduled now (its blocks take
  // SM slots only as this grid's blocks exit). After the wait below, this grid reads what the
  // previous chunk wrote (this chunk's touch bits) and sets bits in the buffer the previous
  // chunk was applying and clearing (the next chunk's).
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ __align__(16) uint32_t smc[];
  uint32_t* sT = smc;                                              // 2048 table words
  uint8_t* masks = reinterpret_cast<uint8_t*>(smc + (TABLES ? 2048 : 0));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* my = masks + (size_t)wid * (d.eta >> 3);
  __shared__ uint4 stm[256];   // touch masks (touch_mask_entry)
  for (int i = threadIdx.x; i < 256; i += blockDim.x) stm[i] = touch_mask_entry((uint32_t)i);
  if (TABLES)
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) sT[i] = s.tables[i];
  __syncthreads();
  // the warp's first estimator: its recorders are loaded before the wait (no earlier grid of
  // the slot writes them), its touch bytes after it
  const uint32_t iters = d.eta >> 8;
  const uint32_t m0 = iters < 8u ? iters : 8u;
  const uint64_t tstep = d.eta >> 3;   // touch bytes per estimator
  uint4 v[8];
  const uint64_t e_first = (uint64_t)blockIdx.x * (kBlock / 32) + wid;
  if (e_first < a.count)
    load_group(reinterpret_cast<const uint4*>(a.router), ((a.se0 + e_first) << d.log2_eta) >> 3, 0, m0, lane, v);
  asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous grid has completed
  // the router's clock (moved on only after the slot's last launch)
  const uint32_t tm = *a.tm;
  const Clock c = make_clock(tm, d.k);
  if (a.global_tm && blockIdx.x == 0 && threadIdx.x == 0) *a.global_tm = tm;
  // entries of the next chunk's touch list (written by the list launch before chunk 0)
  const uint64_t n_items = LIST ? (uint64_t)*a.list_fill : a.nvec;
  const uint32_t nr0 = NEXT ? (uint32_t)(a.nx_se0 >> d.q) : 0u;
  const uint32_t nr1 = NEXT ? (uint32_t)((a.nx_se0 + a.nx_count - 1) >> d.q) : 0u;
  const uint64_t slots = a.count * 32;   // (estimator, lane) slots sharing the pairs
  uint4* const r0 = reinterpret_cast<uint4*>(a.router);
  uint4* const g = reinterpret_cast<uint4*>(a.global);
  const uint64_t wstride = (uint64_t)gridDim.x * (kBlock / 32);
  auto touch2 = [&](uint4 w, bool live) {
    if (PACKED) {
      touch_packed<CM>(a.next, w.x, w.y, live, d, nr0, nr1, a.nx_se0, a.nx_count);
      touch_packed<CM>(a.next, w.z, w.w, live, d, nr0, nr1, a.nx_se0, a.nx_count);
    } else {
      uint32_t c0, o0, c1, o1;
      const bool in0 = view_pair(a.view, w.x, w.y, c0, o0), in1 = view_pair(a.view, w.z, w.w, c1, o1);
      touch_pair<CM>(a.next, 0, c0, o0, live && in0, sT, d, nr0, nr1, a.nx_se0, a.nx_count);
      touch_pair<CM>(a.next, 0, c1, o1, live && in1, sT, d, nr0, nr1, a.nx_se0, a.nx_count);
    }
  };
  // after an estimator's pass: its share of the next chunk's touches, then its pooling
  auto finish = [&](uint64_t e, uint64_t se, uint32_t cnt, uint4 w0) {
    const uint64_t vb0 = e * 32;
    if (LIST) {
      if (vb0 < n_items)
        set_touch<CM>(a.next, w0.x, vb0 + lane < n_items && in_bounds(d, w0.x < d.touch_bits));
      for (uint64_t vb = vb0 + slots; vb < n_items; vb += slots) {
        const bool live = vb + lane < n_items;
        const uint32_t bit = live ? __ldcs(a.list + vb + lane) : 0u;
        set_touch<CM>(a.next, bit, live && in_bounds(d, bit < d.touch_bits));
      }
    } else if (NEXT) {
      if (vb0 < a.nvec) touch2(w0, vb0 + lane < a.nvec);
      for (uint64_t vb = vb0 + slots; vb < a.nvec; vb += slots) {
        const bool live = vb + lane < a.nvec;
        touch2(live ? __ldcs(a.vec + vb + lane) : make_uint4(0, 0, 0, 0), live);
      }
      if (e == 0 && lane < 2 && a.edge[lane]) {
        const uint32_t* p = a.edge[lane];
        if (PACKED) {
          touch_packed<0>(a.next, p[0], p[1], true, d, nr0, nr1, a.nx_se0, a.nx_count);
        } else {
          uint32_t c0, o0;
          const bool in = view_pair(a.view, p[0], p[1], c0, o0);
          touch_pair<0>(a.next, 0, c0, o0, in, sT, d, nr0, nr1, a.nx_se0, a.nx_count);
        }
      }
    }
    pool_if_hot(d, s, se, cnt, my, lane);
  };
  // this slot's first pair vector of an estimator is loaded before its pass so the loads overlap
  auto first_pair = [&](uint64_t e) {
    if (LIST) return make_uint4(e * 32 + lane < n_items ? __ldcs(a.list + e * 32 + lane) : 0u, 0u, 0u, 0u);
    return (NEXT && e * 32 + lane < a.nvec) ? __ldcs(a.vec + e * 32 + lane) : make_uint4(0, 0, 0, 0);
  };
  uint64_t e = e_first;
  if (e < a.count) {   // the prefetched first group, then any further groups
    const uint64_t se = a.se0 + e;
    uint8_t* tb = a.touch + e * tstep + lane * iters;   // touch_pos
    const uint4 w0 = first_pair(e);
    const uint64_t base = (se << d.log2_eta) >> 3;
    uint64_t tw = load_touch(tb, m0);
    uint32_t cnt = fast_group<true, true, true>(r0, g, base, 0, m0, lane, c, stm, v, tw);
    clear_touch(tb, m0, tw != 0ull);
    for (uint32_t it0 = 8; it0 < iters; it0 += 8) {
      const uint32_t m = iters - it0 < 8u ? iters - it0 : 8u;
      load_group(r0, base, it0, m, lane, v);
      tw = load_touch(tb + it0, m);
      cnt += fast_group<true, true, true>(r0, g, base, it0, m, lane, c, stm, v, tw);
      clear_touch(tb + it0, m, tw != 0ull);
    }
    hot_bits(d, r0, base, cnt, my, lane, c);
    finish(e, se, cnt, w0);
    e += wstride;
  }
  for (; e < a.count; e += wstride) {
    const uint64_t se = a.se0 + e;
    const uint4 w0 = first_pair(e);
    const uint64_t base = (se << d.log2_eta) >> 3;
    uint8_t* tb = a.touch + e * tstep + lane * iters;   // touch_pos
    const uint32_t cnt = one_router_se<true, true, true>(d, r0, g, base, tb, my, lane, c, stm);
    finish(e, se, cnt, w0);
  }
}

template <typename K>
int blocks_per_sm(K kernel, size_t smem, const Tuning& tn) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kBlock, smem) != cudaSuccess) return 1;
  if (tn.stream_bps && (int)tn.stream_bps < b) b = (int)tn.stream_bps;
  return b > 0 ? b : 1;
}

template <bool ONE, bool ADV, bool HOT, bool TOUCH, int G>
cudaError_t launch_large(const Dims& d, const Scratch& s, const StreamArgs& a, uint64_t count, int sms,
                         const Tuning& tn, cudaStream_t st) {
  const size_t smem = HOT ? (size_t)(kBlock / 32) * (d.eta >> 3) : 0;
  const uint64_t need = (count + (kBlock / 32) - 1) / (kBlock / 32);
  uint64_t grid = (uint64_t)sms * blocks_per_sm(k_stream_large<ONE, ADV, HOT, TOUCH, G>, smem, tn);
  if (grid > need) grid = need;
  k_stream_large<ONE, ADV, HOT, TOUCH, G><<<(unsigned)grid, kBlock, smem, st>>>(d, s, a);
  return cudaGetLastError();
}

template <bool ONE, bool ADV, bool HOT, bool TOUCH>
cudaError_t launch_variant(const Dims& d, const Scratch& s, const StreamArgs& a, int sms, const Tuning& tn,
                           cudaStream_t st) {
  const uint64_t count = a.se_count ? a.se_count : ((uint64_t)d.r << d.q);
  if (d.eta >= 256) {
    if (ONE) return launch_large<ONE, ADV, HOT, TOUCH, 1>(d, s, a, count, sms, tn, st);
    if (tn.group == 2) return launch_large<ONE, ADV, HOT, TOUCH, 2>(d, s, a, count, sms, tn, st);
    if (tn.group == 4) return launch_large<ONE, ADV, HOT, TOUCH, 4>(d, s, a, count, sms, tn, st);
    return launch_large<ONE, ADV, HOT, TOUCH, 8>(d, s, a, count, sms, tn, st);
  }
  const uint64_t n_units = count * d.eta / 256;
  const uint64_t need = (n_units + (kBlock / 32) - 1) / (kBlock / 32);
  uint64_t grid = (uint64_t)sms * blocks_per_sm(k_stream_small<ONE, ADV, HOT, TOUCH>, 0, tn);
  if (grid > need) grid = need;
  k_stream_small<ONE, ADV, HOT, TOUCH><<<(unsigned)grid, kBlock, 0, st>>>(d, s, a);
  return cudaGetLastError();
}

// The clocks of an advance move on by one slot.
__global__ void k_tick(const __grid_constant__ TickArgs a) {
  if ((int)threadIdx.x < a.n) *a.tm[threadIdx.x] = tm_next(*a.tm[threadIdx.x]);
}

// dst = flip(src) at one clock; the clock is also stored at tm_out (by one thread).
__global__ void __launch_bounds__(kBlock) k_flip(const uint16_t* __restrict__ src, uint16_t* __restrict__ dst,
                                                 uint64_t count, const uint32_t* tm_in, uint32_t tm_val,
                                                 uint32_t* tm_out) {
  const uint32_t tm = tm_in ? *tm_in : tm_val;
  const uint32_t tm2 = tm | (tm << 16);
  if (tm_out && blockIdx.x == 0 && threadIdx.x == 0) *tm_out = tm;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    dst[i] = (uint16_t)flip2(src[i], tm2);
}

}  // namespace

cudaError_t launch_tick(const TickArgs& a, cudaStream_t st) {
  if (a.n < 1 || a.n > kMaxBatch) return cudaErrorInvalidValue;
  k_tick<<<1, kMaxBatch, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_flip(const uint16_t* src, uint16_t* dst, uint64_t count, const uint32_t* tm_in, uint32_t tm_val,
                        uint32_t* tm_out, int sms, cudaStream_t st) {
  if (!count && !tm_out) return cudaSuccess;
  uint64_t grid = (count + kBlock - 1) / kBlock;
  if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
  if (grid < 1) grid = 1;
  k_flip<<<(unsigned)grid, kBlock, 0, st>>>(src, dst, count, tm_in, tm_val, tm_out);
  return cudaGetLastError();
}

cudaError_t launch_stream(const Dims& d, const Scratch& s, const StreamArgs& a, int mode, int sms,
                          const Tuning& tn, cudaStream_t st) {
  const bool one = a.n == 1, adv = (mode & kAdvance) != 0, hot = (mode & kHot) != 0, touch = a.touch != nullptr;
#define SSD_STREAM_CASE(O, A, H, T) \
  if (one == O && adv == A && hot == H && touch == T) \
    return launch_variant<O, A, H, T>(d, s, a, sms, tn, st);
  SSD_STREAM_CASE(true, true, true, false)
  SSD_STREAM_CASE(true, true, false, false)
  SSD_STREAM_CASE(true, false, true, false)
  SSD_STREAM_CASE(true, false, false, false)
  SSD_STREAM_CASE(false, true, true, false)
  SSD_STREAM_CASE(false, true, false, false)
  SSD_STREAM_CASE(false, false, true, false)
  SSD_STREAM_CASE(false, false, false, false)
  SSD_STREAM_CASE(true, true, true, true)
  SSD_STREAM_CASE(false, true, true, true)
#undef SSD_STREAM_CASE
  return cudaErrorInvalidValue;
}

template <int SRC, int CM>
cudaError_t launch_chunk_variant(const Dims& d, const Scratch& s, const ChunkArgs& a, int sms, const Tuning& tn,
                                 cudaStream_t st) {
  const size_t smem = (size_t)(kBlock / 32) * (d.eta >> 3) + (SRC == kSrcRaw ? 2048 * 4 : 0);
  const uint64_t need = (a.count + (kBlock / 32) - 1) / (kBlock / 32);
  uint64_t grid = (uint64_t)sms * blocks_per_sm(k_chunk<SRC, CM>, smem, tn);
  if (grid > need) grid = need;
  // launched as a programmatic dependent of the previous kernel on the stream (see k_chunk)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_chunk<SRC, CM>, d, s, a);
}

template <int SRC>
cudaError_t launch_chunk_cm(const Dims& d, const Scratch& s, const ChunkArgs& a, int sms, const Tuning& tn,
                            cudaStream_t st) {
  if (tn.combine == 1) return launch_chunk_variant<SRC, 1>(d, s, a, sms, tn, st);
  if (tn.combine == 2) return launch_chunk_variant<SRC, 2>(d, s, a, sms, tn, st);
  return launch_chunk_variant<SRC, 0>(d, s, a, sms, tn, st);
}

cudaError_t launch_chunk(const Dims& d, const Scratch& s, const ChunkArgs& a, int sms, const Tuning& tn,
                         cudaStream_t st) {
  if (!a.next) return launch_chunk_variant<kSrcNone, 0>(d, s, a, sms, tn, st);
  if (a.list) return launch_chunk_cm<kSrcList>(d, s, a, sms, tn, st);
  if (a.packed) return launch_chunk_cm<kSrcPacked>(d, s, a, sms, tn, st);
  return launch_chunk_cm<kSrcRaw>(d, s, a, sms, tn, st);
}

}  // namespace ssd
