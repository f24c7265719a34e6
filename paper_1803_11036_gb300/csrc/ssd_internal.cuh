// Internal declarations shared by the CUDA translation units of the detector.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssd.h"

// The debug build (nvcc -DSSD_DEBUG=1, a separate library): the kernel indices with a stated
// bound (a recorder inside its estimator, a column inside its row, a touch bit inside its buffer,
// a pool, bucket or candidate index inside its capacity) are checked before the access;
// a broken bound skips the access and records SSD_STATUS_INTERNAL instead of faulting, and guard
// words around the candidate tuple buffers are compared when the counters are read.
#ifndef SSD_DEBUG
#define SSD_DEBUG 0
#endif

namespace ssd {

constexpr uint32_t kNone = 0xFFFFFFFFu;  // "not hot" in the per-estimator pool index
constexpr int kBlock = 256;

// Device counters of one regain / slot close (zeroed before each).
struct DevCounters {
  unsigned int hot[SSD_MAX_R];              // true |HSE(i)|
  unsigned int status;                      // SSD_STATUS_* bits
  unsigned int pad_;
  unsigned long long level[SSD_MAX_R];      // candidates covering rows 0..i
  unsigned long long raw;                   // accepted full tuples (staged)
  unsigned long long n_out;                 // unique hosts
};

// Dimensions and derived constants, passed by value.
struct Dims {
  uint32_t log2_eta, q, r, delta, k, thr, flags;
  uint32_t eta;        // 2^log2_eta
  uint32_t words;      // eta / 32: bitmap words per estimator
  uint32_t col_mask;   // 2^q - 1
  uint32_t low_bits;   // q - delta
  uint32_t low_mask;   // 2^(q-delta) - 1
  uint32_t sh0;        // shift of window B(1): 0, or delta with SSD_RHFG_LITERAL (B(i) at (i-1)*delta + sh0)
  uint32_t hse_cap;    // pool entries per row
  uint64_t ctb_cap;    // tuples per candidate buffer
  uint64_t out_cap;    // staged accepted tuples (a power of two)
  uint64_t touch_bits; // bits of one touch buffer (debug bound)
  unsigned int* dbg;   // debug build: device word collecting SSD_STATUS_INTERNAL (nullptr otherwise)
};

// True when `ok`; in the debug build a false `ok` also records SSD_STATUS_INTERNAL, and the caller
// skips the access it guards. The release build compiles the check away (always true).
__device__ __forceinline__ bool in_bounds(const Dims& d, bool ok) {
#if SSD_DEBUG
  if (!ok) {
    if (d.dbg) atomicOr(d.dbg, SSD_STATUS_INTERNAL);
    return false;
  }
#else
  (void)d;
  (void)ok;
#endif
  return true;
}

// Scratch of a context (all device memory).
struct Scratch {
  const uint32_t* tables;   // 2048 words: H1 tables then RHFG[0] tables
  uint32_t* hot_idx;        // [r][2^q] pool index of a hot estimator, kNone otherwise
  uint32_t* pool_col;       // [r][hse_cap] column of each pooled hot estimator
  uint32_t* pool_rk;        // [r][hse_cap] its R_k
  uint32_t* pool_bm;        // [r][hse_cap][words] bit j = (recorder j < k)
  uint32_t* ctb[2];         // candidate tuple buffers, tuple stride r (pool indices)
  unsigned long long* stage;  // [out_cap] (cip << 32) | R_k of accepted tuples
  DevCounters* counters;
  // Per row, the pooled hot estimators bucketed by the low q-delta bits of their
  // column (the bits the overlap test fixes): bucket_off [r][2^(q-delta) + 1]
  // offsets into bucket_ent [r][hse_cap] (pool indices); bucket_cnt [r][2^(q-delta)]
  // is the build's work space. nullptr: the candidate levels probe hot_idx.
  uint32_t* bucket_off;
  uint32_t* bucket_cnt;
  uint32_t* bucket_ent;
};
// Largest q - delta for which a context keeps the bucket index.
constexpr uint32_t kMaxBucketBits = 16;

// Launch configuration (ssd_tuning without the touch buffer size). No field
// changes a result; each one only spreads the same work differently.
struct Tuning {
  uint32_t stream_bps;   // resident blocks per SM of the streaming kernels (0 = all that fit)
  uint32_t scan_bps;     // scan / touch / pre-hash grid = SMs x scan_bps at most
  uint32_t unroll;       // pair vectors per thread per step: 1, 2, 4, 8
  uint32_t group;        // routers loaded per lane before storing, multi-router pass: 2, 4, 8
  uint32_t combine;      // how same-word touch atomics are combined (set_touch's CM)
  uint32_t collect;      // one-router slot: 0 = per-chunk touch lists, 1 = pre-hashed pairs re-read per chunk
  uint32_t pair_level;   // 0 = the pair level on the tensor cores where it applies, 1 = CUDA-core tiles
};
inline Tuning default_tuning() { return Tuning{0u, 8u, 4u, 8u, 0u, 0u, 0u}; }

// ---- stamp recorders ----
// The library keeps each distance recorder of Sec. 3.2 as the slot of the last pair that set it to
// 0, modulo 65535 (a stamp in 0..65534), or kNever (0xFFFF) when its distance is 65535: never set,
// or not for 65535 slots. A sketch holds tm = its slot counter modulo 65535 in device memory, and
// the distance of a recorder x is 65535 for x = kNever, (tm - x) mod 65535 otherwise. Algorithm 2
// (set to 0) stores tm. The advance of Sec. 4.3 (every recorder + 1, saturating at 65535) is
// tm + 1 together with kNever stored into the recorders whose distance reaches 65535, the stamp
// tm + 1 mod 65535. So between those expiries a slot writes only the recorders a pair set; the
// distances, and every R_k, hot estimator and list, are those of the paper's recorders, and an
// exported sketch holds the distances themselves.
constexpr uint32_t kNever = 0xFFFFu;
__host__ __device__ __forceinline__ uint32_t tm_next(uint32_t tm) { return tm + 1u >= 65535u ? 0u : tm + 1u; }
// Two recorders (one 32-bit word): distances from stamps at clock tm2 (tm in both halves), and
// stamps from distances; the one map does both ways, kNever <-> 65535.
__device__ __forceinline__ uint32_t flip2(uint32_t v, uint32_t tm2) {
  return __vadd2(__vsub2(tm2, v), __vcmpgtu2(v, tm2)) | __vcmpeq2(v, 0xFFFFFFFFu);
}
__device__ __forceinline__ uint4 flip8(uint4 v, uint32_t tm2) {
  return make_uint4(flip2(v.x, tm2), flip2(v.y, tm2), flip2(v.z, tm2), flip2(v.w, tm2));
}
// Per-launch constants of the window test and the expiry on stamps (make_clock). A recorder is
// inside the window (distance < k) when (x - lo) mod 2^16 < klim and x is not kNever; the window
// [lo, tm] of the 65535 stamps wraps past 65534 when tm < k - 1, and then kNever lies inside the
// 16-bit range [lo, lo + k], so klim = k + 1 and kNever is excluded by `wrap`. Recorders holding
// distances (the allocation-free regain's input) use lo = 0, klim = k.
struct Clock {
  uint32_t tm2;     // tm, both halves
  uint32_t lo2;     // oldest stamp in the window, both halves
  uint32_t hi2;     // newest stamp of the window's range starting at lo (tm, or 65534 when the window
                    // wraps; k - 1 for distances), both halves
  uint32_t klim2;   // length of the window's 16-bit range, both halves
  uint32_t xe2;     // the stamp whose distance reaches 65535 at the advance, both halves
  uint32_t wrap;    // kNever lies in the 16-bit range of the window
};
__host__ __device__ __forceinline__ Clock make_clock(uint32_t tm, uint32_t k) {
  Clock c;
  const bool wrap = tm + 1u < k;
  const uint32_t lo = wrap ? tm + 65536u - k : tm + 1u - k;
  const uint32_t klim = wrap ? k + 1u : k;
  const uint32_t xe = tm_next(tm);
  c.tm2 = tm | (tm << 16);
  c.lo2 = lo | (lo << 16);
  c.hi2 = wrap ? 0xFFFEFFFEu : c.tm2;
  c.klim2 = klim | (klim << 16);
  c.xe2 = xe | (xe << 16);
  c.wrap = wrap ? 1u : 0u;
  return c;
}
__host__ __device__ __forceinline__ Clock distance_clock(uint32_t k) {
  Clock c;
  c.tm2 = 0u;
  c.lo2 = 0u;
  c.hi2 = (k - 1u) | ((k - 1u) << 16);
  c.klim2 = k | (k << 16);
  c.xe2 = 0xFFFFFFFFu;   // never matched by a stored value that is advanced (no advance on distances)
  c.wrap = 0u;
  return c;
}
// 0xFFFF in each half of a word whose recorder lies inside the window.
__device__ __forceinline__ uint32_t win2(uint32_t x, const Clock& c) {
  uint32_t m = __vcmpltu2(__vsub2(x, c.lo2), c.klim2);
  if (c.wrap) m &= ~__vcmpeq2(x, 0xFFFFFFFFu);
  return m;
}
// Bit i = recorder i of the 8 in (m0, m1, m2, m3) has 0xFFFF: the high byte of each half gathered
// by two byte permutes, each byte reduced to one bit, four bits summed into the top byte by one
// multiply (the bits are distinct, so nothing carries).
__device__ __forceinline__ uint32_t pack8(uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3) {
  const uint32_t a = __byte_perm(m0, m1, 0x7531u), b = __byte_perm(m2, m3, 0x7531u);
  return (((a & 0x08040201u) * 0x01010101u) >> 24) | (((b & 0x80402010u) * 0x01010101u) >> 24);
}
__device__ __forceinline__ uint32_t win8(uint4 v, const Clock& c) {
  return pack8(win2(v.x, c), win2(v.y, c), win2(v.z, c), win2(v.w, c));
}
// Recorders whose bit is set in t (bit i = recorder i of the 8) take the stamp tm2.
__device__ __forceinline__ uint32_t set2(uint32_t w, uint32_t t2, uint32_t tm2) {
  const uint32_t m = ((t2 & 1u) * 0xFFFFu) | ((t2 >> 1) * 0xFFFF0000u);
  return (w & ~m) | (tm2 & m);
}
__device__ __forceinline__ uint4 set8(uint4 v, uint32_t t, uint32_t tm2) {
  return make_uint4(set2(v.x, t & 3u, tm2), set2(v.y, (t >> 2) & 3u, tm2), set2(v.z, (t >> 4) & 3u, tm2),
                    set2(v.w, t >> 6, tm2));
}
// The same tests with fewer instructions: a stamp lies inside a range [lo, hi] (lo <= hi) exactly
// when clamping it into the range leaves it unchanged. The window is [lo, tm], or [lo, 65534] and
// [0, tm] when it wraps (kNever lies in neither). min/max.u16x2 are single instructions on sm_90
// and later, where the compares and subtractions of 16-bit halves above are not.
__device__ __forceinline__ uint32_t umin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t umax2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// 1 in each half of x outside [lo, hi], 0 inside.
__device__ __forceinline__ uint32_t out_range2(uint32_t x, uint32_t lo2, uint32_t hi2) {
  return umin2(umax2(umin2(x, hi2), lo2) ^ x, 0x00010001u);
}
// 1 in each half of x outside the window, 0 inside (so a sum of these words counts the recorders
// outside, per half, in 16-bit fields). WRAP = c.wrap, chosen once per group by the caller (it is
// the same for the whole grid), so the common case pays for one range only.
template <bool WRAP>
__device__ __forceinline__ uint32_t out2(uint32_t x, const Clock& c) {
  uint32_t o = out_range2(x, c.lo2, c.hi2);
  if (WRAP) o &= out_range2(x, 0u, c.tm2);
  return o;
}
// Whether any of the 8 recorders holds the stamp xe (a zero half in x ^ xe).
__device__ __forceinline__ bool any_eq8(uint4 v, uint32_t xe2) {
  const uint32_t m = umin2(umin2(v.x ^ xe2, v.y ^ xe2), umin2(v.z ^ xe2, v.w ^ xe2));
  return umin2(m, 0x00010001u) != 0x00010001u;
}
// The 16-bit masks of the recorders named by a touch byte (bit i = recorder i of 8): entry t of
// a 256-entry table, one entry per thread of a block of at least 256 threads.
__device__ __forceinline__ uint4 touch_mask_entry(uint32_t t) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w[i] = (((t >> (2 * i)) & 1u) ? 0xFFFFu : 0u) | (((t >> (2 * i + 1)) & 1u) ? 0xFFFF0000u : 0u);
  return make_uint4(w[0], w[1], w[2], w[3]);
}
// Recorders of v under the mask mk take the stamp tm2.
__device__ __forceinline__ uint4 set_masked(uint4 v, uint4 mk, uint32_t tm2) {
  return make_uint4((v.x & ~mk.x) | (tm2 & mk.x), (v.y & ~mk.y) | (tm2 & mk.y), (v.z & ~mk.z) | (tm2 & mk.z),
                    (v.w & ~mk.w) | (tm2 & mk.w));
}
// kNever (0xFFFF) in each recorder whose distance reaches 65535 at the advance, 0 elsewhere.
__device__ __forceinline__ uint4 expire8(uint4 v, const Clock& c) {
  return make_uint4(__vcmpeq2(v.x, c.xe2), __vcmpeq2(v.y, c.xe2), __vcmpeq2(v.z, c.xe2), __vcmpeq2(v.w, c.xe2));
}
// Clocks of a launch: one per sketch, read from device memory (captured work stays valid as the
// sketches advance).
__device__ __forceinline__ uint32_t read_tm(const uint32_t* tm) { return tm ? *tm : 0u; }

// ---- scan (ssd_scan.cu) ----
constexpr int kMaxBatch = SSD_MAX_ROUTERS;
struct ScanJob {
  uint16_t* dr;              // the router's recorders
  const uint4* vec;          // 16-byte aligned start of its vector body
  uint64_t nvec;             // packets / 2 in the body
  const uint32_t* head;      // a leading packet outside the body, or nullptr
  const uint32_t* tail;      // a trailing packet outside the body, or nullptr
};
struct ScanBatch {
  int n;
  uint64_t prefix[kMaxBatch + 1];  // prefix sums of nvec
  uint16_t* dr[kMaxBatch];
  const uint32_t* tm[kMaxBatch];        // each job's sketch clock (the stamp its scan stores)
  const uint4* vec[kMaxBatch];
  const uint32_t* edge[2 * kMaxBatch];  // head, tail per router (nullptr when absent)
  uint32_t view[kMaxBatch];             // each job's sketch view (view_pair)
};

// A sketch's view, packed: bit 0 = side (1: hosts are the second field of a
// pair), bits 1..5 = group bits gb, bits 16..31 = group. With gb > 0 only hosts
// whose top gb bits equal the group are counted.
__host__ __device__ __forceinline__ uint32_t view_pack(uint32_t side, uint32_t gb, uint32_t group) {
  return (side & 1u) | (gb << 1) | (group << 16);
}
__host__ __device__ __forceinline__ bool view_host_in(uint32_t view, uint32_t host) {
  const uint32_t gb = (view >> 1) & 31u;
  return gb == 0 || (host >> (32u - gb)) == (view >> 16);
}
// The (host, opposite host) a view takes from the stored pair (x, y); false when
// the host is outside the view's group.
__device__ __forceinline__ bool view_pair(uint32_t view, uint32_t x, uint32_t y, uint32_t& cip, uint32_t& oip) {
  cip = (view & 1u) ? y : x;
  oip = (view & 1u) ? x : y;
  return view_host_in(view, cip);
}
cudaError_t launch_scan(const Dims& d, const uint32_t* tables, const ScanBatch& b, int grid, const Tuning& tn,
                        cudaStream_t st);

// ---- streaming passes (ssd_stream.cu) ----
struct StreamArgs {
  int n;                               // routers
  uint16_t* routers[kMaxBatch];
  const uint32_t* tm[kMaxBatch];       // each router's clock; nullptr: the recorders hold distances
                                       // (read-only passes of the allocation-free regain)
  uint16_t* global;                    // merged output, or nullptr
  uint32_t* global_tm;                 // its clock, set to router 0's (the merged state of this slot)
  uint64_t se0;                        // first estimator of the pass
  uint64_t se_count;                   // estimators in the pass; 0 = all r * 2^q from se0 = 0
  uint8_t* touch;                      // touch bits of the pass's estimators per router, or nullptr:
                                       // router j, estimator se0 + e, recorder x at bit
                                       // (j * se_count + e) * eta + x; applied (recorder := 0) and cleared
};
// mode bits
constexpr int kAdvance = 1;   // routers advanced (expired recorders stored as kNever; the clocks are
                              // moved on by launch_tick after every launch that reads them)
constexpr int kHot = 2;       // count R_k of the merged value and pool the hot estimators
cudaError_t launch_stream(const Dims& d, const Scratch& s, const StreamArgs& a, int mode, int sms,
                          const Tuning& tn, cudaStream_t st);

// ---- touch collection for the fused slot (ssd_scan.cu) ----
// Algorithm 2 for the estimators [se0, se0 + se_count) only: instead of storing
// 0 into the recorder, set its bit in `bits` (layout of StreamArgs::touch).
cudaError_t launch_touch(const Dims& d, const uint32_t* tables, const ScanBatch& b, uint32_t* bits, uint64_t se0,
                         uint64_t se_count, int grid, const Tuning& tn, cudaStream_t st);

// ---- device helpers shared by the scan and streaming kernels ----
// Simple tabulation: four 256-word tables indexed by the bytes of x, XORed.
__device__ __forceinline__ uint32_t tab_hash(const uint32_t* T, uint32_t x) {
  return T[x & 255u] ^ T[256u + ((x >> 8) & 255u)] ^ T[512u + ((x >> 16) & 255u)] ^ T[768u + (x >> 24)];
}

// Sets bit `bit` of `bits` (an L2-resident touch buffer) when ok. CM picks how
// touches that land on one word are combined:
//  0: one atomicOr per touch;
//  1: inside the warp: lanes whose bits fall into one 32-bit word are grouped
//     (__match_any_sync on the word index), the group ORs its bits
//     (__reduce_or_sync over the group's mask) and its lowest lane issues the
//     one atomic. All 32 lanes must make the call together; a lane with
//     ok == false joins with a key no word has;
//  2: across the GPU: the word is read from L2 first (ld.global.cg) and the
//     atomic is skipped when the bit is already set. Bits are only set while a
//     buffer is collected (it was cleared by an earlier launch on the same
//     stream order), so a stale read can only cost a redundant atomic. A source
//     sending many packets to few peers sets each of its bits thousands of
//     times per slot; this drops those repeats.
template <int CM>
__device__ __forceinline__ void set_touch(uint32_t* bits, uint64_t bit, bool ok) {
  if (CM == 1) {
    const unsigned long long word = ok ? (unsigned long long)(bit >> 5) : ~0ull;
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, word);
    const unsigned v = __reduce_or_sync(grp, ok ? (1u << (bit & 31u)) : 0u);
    if (ok && (threadIdx.x & 31u) == (unsigned)(__ffs(grp) - 1)) atomicOr(bits + word, v);
  } else if (CM == 2) {
    if (ok) {
      uint32_t* w = bits + (bit >> 5);
      const uint32_t m = 1u << (bit & 31u);
      if (!(__ldcg(w) & m)) atomicOr(w, m);
    }
  } else if (ok) {
    atomicOr(bits + (bit >> 5), 1u << (bit & 31u));
  }
}

// Position of recorder x's bit among its estimator's eta touch bits. For eta >= 256 the streaming
// kernels give vector vi = x / 8 of an estimator to lane vi mod 32 as its (vi / 32)-th vector, so
// the byte of vector vi is stored at (vi mod 32) * (eta / 256) + vi / 32: a lane's bytes are
// contiguous, read with one load and cleared with one store. For eta < 256 a lane takes one
// vector and the byte stays at vi.
__device__ __forceinline__ uint32_t touch_pos(const Dims& d, uint32_t x) {
  if (d.log2_eta < 8u) return x;
  const uint32_t vi = x >> 3;
  return ((((vi & 31u) << (d.log2_eta - 8u)) | (vi >> 5)) << 3) | (x & 7u);
}

// Algorithm 2 for the estimators [se0, se0 + count) only (one chunk, inside one
// row or whole rows): the recorder a pair sets to 0 is marked in `bits` instead
// (router base jbase = router * count; estimator se0 + e, recorder x -> bit
// (jbase + e) * eta + touch_pos(x)). sT holds both table sets (2048 words). `live` = false
// makes the call a no-op (a lane past the end of the pairs; with CM == 1 every
// lane calls).
template <int CM>
__device__ __forceinline__ void touch_pair(uint32_t* bits, uint64_t jbase, uint32_t cip, uint32_t oip, bool live,
                                           const uint32_t* sT, const Dims& d, uint32_t r0, uint32_t r1,
                                           uint64_t se0, uint64_t count) {
  const uint32_t c0 = tab_hash(sT + 1024, cip) & d.col_mask;
  uint32_t x = 0xFFFFFFFFu;
  for (uint32_t i = r0; i <= r1; ++i) {
    uint32_t col = c0;
    if (i) {
      const uint32_t sh = (i - 1u) * d.delta + d.sh0;
      col = ((sh < 32u ? (cip >> sh) : 0u) ^ c0) & d.col_mask;
    }
    const uint64_t e = (((uint64_t)i << d.q) | col) - se0;
    const bool ok = live && e < count;
    if (ok && x == 0xFFFFFFFFu) x = tab_hash(sT, oip) & (d.eta - 1u);
    const uint64_t bit = ((jbase + e) << d.log2_eta) | touch_pos(d, x);
    set_touch<CM>(bits, bit, ok && in_bounds(d, bit < d.touch_bits));
  }
}

// touch_pair on a pre-hashed pair: packed = RHFG[0](cip) | H1(oip) << q (q + log2_eta <= 32).
template <int CM>
__device__ __forceinline__ void touch_packed(uint32_t* bits, uint32_t cip, uint32_t packed, bool live, const Dims& d,
                                             uint32_t r0, uint32_t r1, uint64_t se0, uint64_t count) {
  const uint32_t c0 = packed & d.col_mask;
  const uint32_t x = packed >> d.q;
  for (uint32_t i = r0; i <= r1; ++i) {
    uint32_t col = c0;
    if (i) {
      const uint32_t sh = (i - 1u) * d.delta + d.sh0;
      col = ((sh < 32u ? (cip >> sh) : 0u) ^ c0) & d.col_mask;
    }
    const uint64_t e = (((uint64_t)i << d.q) | col) - se0;
    const uint64_t bit = (e << d.log2_eta) | touch_pos(d, x);
    const bool ok = live && e < count;
    set_touch<CM>(bits, bit, ok && in_bounds(d, bit < d.touch_bits && x < d.eta));
  }
}

// ---- per-slot pre-hash of one router's pairs (ssd_scan.cu) ----
// out[m] = (cip, RHFG[0](cip) | H1(oip) << q) for every pair of the buffer described by
// job 0 of b, taken through job 0's view (its side; a grouped view is not pre-hashed):
// the body vectors first (out[2v], out[2v+1]), then the head and tail pairs.
// The result holds n_pairs entries in an order the order-free scan does not see.
cudaError_t launch_prehash(const Dims& d, const uint32_t* tables, const ScanBatch& b, uint2* out, int grid,
                           cudaStream_t st);
// Algorithm 2 for one chunk from pre-hashed pairs (one router): `vec` holds nvec
// vectors of two packed pairs, `tail` one more packed pair or nullptr.
cudaError_t launch_touch_packed(const Dims& d, const uint4* vec, uint64_t nvec, const uint2* tail, uint32_t* bits,
                                uint64_t se0, uint64_t se_count, int grid, const Tuning& tn, cudaStream_t st);

// ---- per-chunk touch lists of the fused slot (ssd_scan.cu) ----
// Algorithm 2 for every pair of the batch, once per slot, sorted by chunk: chunk c covers the
// estimators [c * count, (c + 1) * count) of every router, and the touch of router j, estimator
// se, recorder x has the bit ((j * count + se - c * count) << log2_eta) | touch_pos(x) of that
// chunk's bits.
// Chunk 0's bits are set directly in `touch0`; the bit index of every touch of chunk c >= 1 is
// appended to list c (ent + (c - 1) * cap, fill[c] entries). A pair adds at most one touch per
// row, so a list of a chunk inside one row never holds more than the batch's pairs.
constexpr uint32_t kMaxChunks = 32;
struct ListArgs {
  uint32_t log2_count;   // estimators per chunk = 2^log2_count
  uint32_t n_chunks;     // <= kMaxChunks
  uint64_t cap;          // entries per list
  uint32_t* ent;         // n_chunks - 1 lists of cap entries
  uint32_t* fill;        // kMaxChunks counters, zero before the launch
  uint32_t* touch0;      // chunk 0's touch bits
  DevCounters* counters; // SSD_STATUS_INTERNAL when a list would overflow (never, by the bound above)
};
cudaError_t launch_lists(const Dims& d, const uint32_t* tables, const ScanBatch& b, const ListArgs& a, int grid,
                         const Tuning& tn, cudaStream_t st);

// ---- one chunk of the fused slot of one router (ssd_stream.cu) ----
// The streaming pass over estimators [se0, se0 + count) with that chunk's touch
// bits applied; when `next` is set the same kernel collects the touch bits of the
// next chunk [nx_se0, nx_se0 + nx_count) from the slot's pairs.
struct ChunkArgs {
  uint16_t* router;
  const uint32_t* tm;        // the router's clock
  uint16_t* global;          // merged output, or nullptr
  uint32_t* global_tm;       // its clock (set to the router's)
  uint64_t se0, count;
  uint8_t* touch;            // this chunk's touch bits (cleared as they are applied)
  uint32_t* next;            // next chunk's touch bits, or nullptr
  uint64_t nx_se0, nx_count;
  const uint4* vec;          // the slot's pairs: 16-byte body, nvec vectors of 2 pairs
  uint64_t nvec;
  const uint32_t* edge[2];   // head / tail pair outside the body, or nullptr
  int packed;                // vec/edge[0] hold pre-hashed pairs (edge[1] unused)
  uint32_t view;             // the router's view (raw pairs; pre-hashed pairs are already in it)
  const uint32_t* list;      // the next chunk's touch list (bit indices), or nullptr: collect from vec
  const uint32_t* list_fill; // its entry count (device)
};
cudaError_t launch_chunk(const Dims& d, const Scratch& s, const ChunkArgs& a, int sms, const Tuning& tn,
                         cudaStream_t st);

// ---- sketch clocks and conversions (ssd_stream.cu) ----
// Every clock of tms moves on by one slot (tm_next), after the launches of an advance.
struct TickArgs {
  int n;
  uint32_t* tm[kMaxBatch];
};
cudaError_t launch_tick(const TickArgs& a, cudaStream_t st);
// dst[i] = flip(src[i]) for i < count at clock *tm_in (or tm_val when tm_in is nullptr): stamps to
// distances (export) or distances to stamps (import). With tm_out the clock is also stored there.
cudaError_t launch_flip(const uint16_t* src, uint16_t* dst, uint64_t count, const uint32_t* tm_in, uint32_t tm_val,
                        uint32_t* tm_out, int sms, cudaStream_t st);

// ---- reduction of a merge spread over GPUs (ssd_shard.cu) ----
// out[x] = min over j < n of in[j][x] for x < count (all 16-byte aligned; out may be an input).
cudaError_t launch_min_ranges(uint16_t* out, const uint16_t* const* in, int n, uint64_t count, int sms,
                              cudaStream_t st);

// ---- diagnostics (ssd_diag.cu) ----
// rk_sum[i] += sum over row i's estimators of R_k (recorders below k, stamps at clock *tm); eta >= 8.
cudaError_t launch_occupancy(const Dims& d, const uint16_t* dr, const uint32_t* tm, unsigned long long* rk_sum,
                             int sms, cudaStream_t st);

// ---- regain (ssd_regain.cu) ----
// Candidate levels, final test and the list; reads the pools filled by a kHot pass.
// `view`: the regained sketch's view; hosts outside its group are not listed.
// tensor_pairs: the pair level on the tensor cores when eta is a multiple of 128 and pruning is on.
cudaError_t launch_regain_tail(const Dims& d, const Scratch& s, uint32_t* ips, uint32_t* rk, uint64_t cap,
                               unsigned long long* n_out_dev, int sms, cudaStream_t st, int* launches,
                               uint32_t view = 0, bool tensor_pairs = false);

}  // namespace ssd
