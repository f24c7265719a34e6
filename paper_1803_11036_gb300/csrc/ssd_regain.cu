// Regaining sliding super points from the pooled hot estimators (Sec. 3.3 and
// Sec. 4.2, Algorithms 6-7 and the final test).
//
// Level 1 (pairs): every (he_0, he_1) of HSE(0) x HSE(1). With pruning, a pair
//   is kept only when the union of its two estimators still has R_k >= the
//   threshold: the union is an elementwise maximum, so R_k = popcount of the
//   AND of the "recorder < k" bitmaps, and it can only fall as rows are added;
//   a dropped tuple would fail the final test. Computed either as an fp8 GEMM of
//   the bitmaps expanded to bytes on the tensor cores (k_pairs_tc, the default
//   for eta a multiple of 128), or as 64 x 64 tiles of AND-popcounts on the CUDA
//   cores (4 x 4 per thread, one carry-save step per two words) with the bitmaps
//   staged in shared memory; one append per tile either way.
// Level i >= 2: the overlap test fixes the low q-delta bits of he_i
//   (B(i) mod 2^(q-delta) = B(i-1) >> delta with B(j) = he_0 XOR he_j), so the
//   only row-i estimators a candidate can extend to are the hot ones with those
//   low bits. The k_pairs launch also buckets each row's hot estimators by their
//   low q-delta bits, and a candidate reads its one bucket (when 2^(q-delta) is
//   too large for the index, it probes the 2^delta columns in hot_idx instead).
//   Hits are tested by groups of four lanes (up to eight at once per warp, all
//   loads of a group's share issued together) and survivors are appended with
//   warp-aggregated atomics.
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

// The host whose q-bit windows (cip >> ((j-1)*delta + sh0)) mod 2^q are B(j) =
// he_0 ^ he_j, j = 1..r-1: bits [sh0, sh0 + q) from B(1), then the top delta
// bits of each B(j) at (j-2)*delta + q + sh0. Consecutive windows already agree
// on their overlap, so the only way no host exists is a window bit at position
// 32 or beyond. With sh0 = delta (Eq. 2 as printed) bits 0..delta-1 stay 0: no
// window holds them.
__device__ __forceinline__ bool regain_host(const Dims& d, const uint32_t* he, uint32_t* cip) {
  const uint32_t lim = 32u - d.sh0;   // bits of cip >> sh0
  uint64_t v = he[0] ^ he[1];
  for (uint32_t j = 2; j < d.r; ++j) {
    const uint64_t top = (uint64_t)((he[0] ^ he[j]) >> d.low_bits);
    const uint32_t pos = (j - 2) * d.delta + d.q;
    if (pos >= lim) {
      if (top) return false;
    } else {
      v |= top << pos;
    }
  }
  if (v >> lim) return false;
  *cip = (uint32_t)(v << d.sh0);
  return true;
}

// Each tail kernel is launched as a programmatic dependent of the kernel before it
// on the stream: it lets its own successor be scheduled at once, then waits (in
// hardware) until its predecessor has completed - it reads the counters and
// buffers that kernel wrote - so only the launch latency is overlapped.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
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

constexpr int TA = 64, KW = 64;

// popcount(a) + popcount(b) through one carry-save step into `ones`: returns the
// carries' popcount (weight 2) and leaves the sum bits in `ones`; the total of a
// run is 2 * (sum of the returned counts) + popcount(ones).
__device__ __forceinline__ uint32_t csa_pop(uint32_t& ones, uint32_t a, uint32_t b) {
  const uint32_t carry = (ones & a) | (ones & b) | (a & b);
  ones ^= a ^ b;
  return __popc(carry);
}

// Blocks [0, pair_blocks) test the pairs in 64 x 64 tiles (4 x 4 per thread,
// output columns interleaved by 16 so the shared-memory reads are free of bank
// conflicts); with the bucket index, block pair_blocks + m builds the buckets of
// row 2 + m.
__global__ void __launch_bounds__(kBlock, 3) k_pairs(const Dims d, const Scratch s, uint32_t pair_blocks) {
  pdl_enter();
  if (blockIdx.x >= pair_blocks) {
    build_buckets(d, s, 2 + (blockIdx.x - pair_blocks));
    return;
  }
  __shared__ uint32_t A[TA][KW + 1], B[TA][KW + 1];
  __shared__ uint32_t wsum[kBlock / 32];
  __shared__ unsigned long long tile_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    uint32_t ones[4][4], twice[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) ones[u][v] = twice[u][v] = 0;
    if (prune) {
      for (uint32_t k0 = 0; k0 < d.words; k0 += KW) {
        const uint32_t kw = d.words - k0 < (uint32_t)KW ? d.words - k0 : (uint32_t)KW;
        __syncthreads();
        if ((d.words & 3u) == 0) {
          // 16-byte loads, all eight of a thread issued before any store (one round trip)
          constexpr int kVec = TA * KW / 4 / kBlock;   // 16-byte vectors per thread per operand
          uint4 va[kVec], vb[kVec];
#pragma unroll
          for (int q = 0; q < kVec; ++q) {
            const int e = threadIdx.x + q * kBlock, rr = e / (KW / 4), c4 = (e % (KW / 4)) * 4;
            const bool in = c4 < (int)kw;   // words past kw are staged as 0
            va[q] = (in && a0 + rr < n0)
                        ? *reinterpret_cast<const uint4*>(bm0 + (uint64_t)(a0 + rr) * d.words + k0 + c4)
                        : make_uint4(0, 0, 0, 0);
            vb[q] = (in && b0 + rr < n1)
                        ? *reinterpret_cast<const uint4*>(bm1 + (uint64_t)(b0 + rr) * d.words + k0 + c4)
                        : make_uint4(0, 0, 0, 0);
          }
#pragma unroll
          for (int q = 0; q < kVec; ++q) {
            const int e = threadIdx.x + q * kBlock, rr = e / (KW / 4), c4 = (e % (KW / 4)) * 4;
            A[rr][c4] = va[q].x; A[rr][c4 + 1] = va[q].y; A[rr][c4 + 2] = va[q].z; A[rr][c4 + 3] = va[q].w;
            B[rr][c4] = vb[q].x; B[rr][c4 + 1] = vb[q].y; B[rr][c4 + 2] = vb[q].z; B[rr][c4 + 3] = vb[q].w;
          }
        } else {
          for (int e = threadIdx.x; e < TA * KW; e += kBlock) {
            const int rr = e / KW, cc = e % KW;
            const bool in = cc < (int)kw;   // words past kw are staged as 0
            A[rr][cc] = (in && a0 + rr < n0) ? bm0[(uint64_t)(a0 + rr) * d.words + k0 + cc] : 0u;
            B[rr][cc] = (in && b0 + rr < n1) ? bm1[(uint64_t)(b0 + rr) * d.words + k0 + cc] : 0u;
          }
        }
        __syncthreads();
        for (uint32_t cc = 0; cc < kw; cc += 2) {
          uint32_t x0[4], x1[4], y0[4], y1[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            x0[u] = A[ty + 16 * u][cc];
            x1[u] = A[ty + 16 * u][cc + 1];
            y0[u] = B[tx + 16 * u][cc];
            y1[u] = B[tx + 16 * u][cc + 1];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) twice[u][v] += csa_pop(ones[u][v], x0[u] & y0[v], x1[u] & y1[v]);
        }
      }
    }
    // the tile's kept pairs go to the candidate buffer with one atomic per tile:
    // a block-wide scan of the threads' counts gives each its offset
    uint32_t keepm = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint32_t ia = a0 + ty + 16 * u, ib = b0 + tx + 16 * v;
        const uint32_t rk = 2 * twice[u][v] + __popc(ones[u][v]);
        if (ia < n0 && ib < n1 && (!prune || rk >= d.thr)) keepm |= 1u << (4 * u + v);
      }
    const uint32_t mine = __popc(keepm);
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int w = 0; w < kBlock / 32; ++w) {
        const uint32_t x = wsum[w];
        wsum[w] = run;
        run += x;
      }
      tile_base = run ? atomicAdd(&s.counters->level[1], (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    unsigned long long pos = tile_base + wsum[wid] + (incl - mine);
    while (keepm) {
      const int b = __ffs(keepm) - 1;
      keepm &= keepm - 1;
      const uint32_t ia = a0 + ty + 16 * (b >> 2), ib = b0 + tx + 16 * (b & 3);
      if (pos < d.ctb_cap) {
        s.ctb[0][pos * d.r + 0] = ia;
        s.ctb[0][pos * d.r + 1] = ib;
      } else {
        atomicOr(&s.counters->status, SSD_STATUS_CTB_OVERFLOW);
      }
      ++pos;
    }
    __syncthreads();   // wsum / tile_base are reused by the next tile
  }
}

// ---- the pair level on the tensor cores ----
// R_k of the union of he_0 and he_1 is the popcount of the AND of their "recorder < k" bitmaps:
// the dot product of the two bitmaps read as 0/1 vectors, so the whole pair level is one binary
// matrix product. k_pairs_tc computes it as an fp8 GEMM on tcgen05: every bit becomes an e4m3
// byte (1.0 or 0), A = the row-0 bitmaps (128 per tile), B = the row-1 bitmaps (256 per tile),
// K = eta, accumulated in f32 in tensor memory. The result is exact: every sum is at most
// eta <= 2^15 < 2^24. The bytes are expanded from the bitmaps straight into shared memory, 128
// recorders per stage with two stages in flight (the next stage's words are loaded into
// registers while the current one is expanded); one thread issues a stage's four MMAs and
// commits them to the stage's mbarrier, which frees its buffer two stages later. The epilogue
// reads the accumulator back (tcgen05.ld), applies the threshold and appends the kept pairs with
// one atomic per tile, as k_pairs does. Waits are bounded: a wait that runs out marks the call
// SSD_STATUS_INTERNAL, and the tile's memory is still released.
constexpr uint32_t kTcM = 128, kTcN = 256, kTcKc = 128;   // tile rows of row 0 / of row 1; K bytes per stage
constexpr uint32_t kTcThreads = 256;
constexpr uint32_t kTcStageA = kTcM * kTcKc, kTcStageB = kTcN * kTcKc;
constexpr uint32_t kTcSmem = 2 * (kTcStageA + kTcStageB) + 1024;   // two stages + alignment slack
constexpr uint32_t kTcCols = 256;                                   // the 128 x 256 f32 accumulator
constexpr uint32_t kTcItems = (kTcM + kTcN) * (kTcKc / 32) / kTcThreads;   // bitmap words per thread per stage
constexpr long long kTcWaitCycles = 4000000000ll;                   // about two seconds of SM clock

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of (row, k byte) in a stage tile, the canonical K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes (128 contiguous bytes), 128 bytes apart along K (the
// leading byte offset) and 8 x 128 = 1024 bytes apart along the rows (the stride byte offset).
__device__ __forceinline__ uint32_t tc_off(uint32_t row, uint32_t kbyte) {
  return (row >> 3) * 1024u + (kbyte >> 4) * 128u + (row & 7u) * 16u + (kbyte & 15u);
}

// Shared-memory matrix descriptor for that layout: start address, leading and stride byte
// offsets (each >> 4), the fixed 0b001 at bits 46-48, base offset 0, no swizzle (bits 61-63).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: D in f32 (bits 4-5 = 1), A and B e4m3 (bits 7-9 and
// 10-12 = 0), both K-major (bits 15 and 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | ((kTcN >> 3) << 17) | ((kTcM >> 4) << 24);

// 32 bits of a bitmap as 32 e4m3 bytes in bit order: 1.0 (0x38) for a set bit, 0 otherwise.
// x * 0x00204081 = x + (x << 7) + (x << 14) + (x << 21) moves bit i of a nibble x to bit 8i (the
// four copies do not overlap, so nothing carries); & 0x01010101 keeps those bits, and the
// multiply by 0x38 turns each into the byte 0x38.
__device__ __forceinline__ uint32_t nib_bytes(uint32_t nib) { return ((nib * 0x00204081u) & 0x01010101u) * 0x38u; }
__device__ __forceinline__ void expand32(uint32_t w, uint4& lo, uint4& hi) {
  lo = make_uint4(nib_bytes(w & 15u), nib_bytes((w >> 4) & 15u), nib_bytes((w >> 8) & 15u), nib_bytes((w >> 12) & 15u));
  hi = make_uint4(nib_bytes((w >> 16) & 15u), nib_bytes((w >> 20) & 15u), nib_bytes((w >> 24) & 15u),
                  nib_bytes(w >> 28));
}

__device__ __forceinline__ void mbar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
// Waits for the phase of `parity` to complete; false when about two seconds pass first.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  const uint32_t a = smem_addr(b);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(kTcIdesc), "r"((uint32_t)accumulate)
      : "memory");
}
// The MMAs issued so far by this thread arrive on `bar` when they complete.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 lanes (one row per lane), waited for.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// Blocks [0, tile_blocks) take the 128 x 256 tiles of HSE(0) x HSE(1) in turn (block b: tiles
// b, b + tile_blocks, ...), with one tensor-memory allocation for all of them; with the bucket
// index, block tile_blocks + m builds the buckets of row 2 + m (as in k_pairs). Needs eta a
// multiple of 128 and pruning on (the caller checks).
__global__ void __launch_bounds__(kTcThreads, 1) k_pairs_tc(const Dims d, const Scratch s, uint32_t tile_blocks) {
  pdl_enter();
  if (blockIdx.x >= tile_blocks) {
    build_buckets(d, s, 2 + (blockIdx.x - tile_blocks));
    return;
  }
  const uint32_t n0 = min(s.counters->hot[0], d.hse_cap);
  const uint32_t n1 = min(s.counters->hot[1], d.hse_cap);
  const uint32_t tn = (n1 + kTcN - 1) / kTcN;
  const uint32_t ntiles = ((n0 + kTcM - 1) / kTcM) * tn;
  if (blockIdx.x >= ntiles) return;   // block-uniform: nothing allocated yet
  extern __shared__ uint8_t tc_raw[];
  __shared__ __align__(8) uint64_t bar[3];   // stage buffer 0, stage buffer 1, a tile's MMAs done
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t wsum[kTcThreads / 32];
  __shared__ unsigned long long tile_base;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* const sA[2] = {sm, sm + kTcStageA};
  uint8_t* const sB[2] = {sm + 2 * kTcStageA, sm + 2 * kTcStageA + kTcStageB};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    mbar_init(&bar[2]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t* bmA = s.pool_bm;
  const uint32_t* bmB = s.pool_bm + (uint64_t)d.hse_cap * d.words;
  const uint32_t stages = d.words / 4;   // 128 recorders per stage
  const uint32_t qr = (uint32_t)warp & 3u, half = (uint32_t)warp >> 2;
  const float thr = (float)d.thr;
  uint32_t g = 0;        // stages issued by this block so far, over all its tiles
  uint32_t tiles = 0;    // tiles finished by this block
  bool ok = true;
  for (uint32_t t = blockIdx.x; t < ntiles && ok; t += tile_blocks, ++tiles) {
    const uint32_t m0 = (t / tn) * kTcM, c0 = (t % tn) * kTcN;
    // this thread's bitmap words of a stage: item threadIdx.x + 256 u, row = item / 4, word = item % 4
    auto load_stage = [&](uint32_t st, uint32_t (&w)[kTcItems]) {
#pragma unroll
      for (uint32_t u = 0; u < kTcItems; ++u) {
        const uint32_t item = threadIdx.x + u * kTcThreads, row = item >> 2, q = item & 3u;
        w[u] = 0;
        if (row < kTcM) {
          if (m0 + row < n0) w[u] = bmA[(uint64_t)(m0 + row) * d.words + st * 4 + q];
        } else if (c0 + row - kTcM < n1) {
          w[u] = bmB[(uint64_t)(c0 + row - kTcM) * d.words + st * 4 + q];
        }
      }
    };
    uint32_t cur[kTcItems], nxt[kTcItems];
    load_stage(0, cur);
    for (uint32_t st = 0; st < stages; ++st, ++g) {
      const uint32_t b = g & 1u;
      if (st + 1 < stages) load_stage(st + 1, nxt);
      // the MMAs of this block's stage g - 2 have read this buffer
      const bool free_ = g < 2 || mbar_wait(&bar[b], ((g - 2) >> 1) & 1u);
      if (!__syncthreads_and(free_)) {
        ok = false;
        break;
      }
#pragma unroll
      for (uint32_t u = 0; u < kTcItems; ++u) {
        const uint32_t item = threadIdx.x + u * kTcThreads, row = item >> 2, q = item & 3u;
        uint8_t* tile = row < kTcM ? sA[b] : sB[b];
        const uint32_t rr = row < kTcM ? row : row - kTcM;
        uint4 lo, hi;
        expand32(cur[u], lo, hi);
        *reinterpret_cast<uint4*>(tile + tc_off(rr, q * 32)) = lo;
        *reinterpret_cast<uint4*>(tile + tc_off(rr, q * 32 + 16)) = hi;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the stores, visible to the MMAs
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_addr(sA[b]), b0 = smem_addr(sB[b]);
#pragma unroll
        for (uint32_t j = 0; j < kTcKc / 32; ++j)   // K = 32 bytes per MMA: two core matrices along K
          tc_mma(tmem, tc_desc(a0 + j * 256u), tc_desc(b0 + j * 256u), (st | j) != 0);
        tc_commit(&bar[b]);
      }
#pragma unroll
      for (uint32_t u = 0; u < kTcItems; ++u) cur[u] = nxt[u];
    }
    if (!ok) break;
    if (threadIdx.x == 0) tc_commit(&bar[2]);   // this tile's MMAs, done
    if (!__syncthreads_and(mbar_wait(&bar[2], tiles & 1u))) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: warp w reads lanes 32 (w % 4) .. +31 (rows of the tile), columns 128 (w / 4) .. +127
    uint32_t masks[4];
    uint32_t mine = 0;
    const uint32_t ia = m0 + qr * 32 + lane;
#pragma unroll
    for (uint32_t cc = 0; cc < 4; ++cc) {
      const uint32_t col = half * 128 + cc * 32;
      uint32_t v[32];
      tc_ld32(tmem + ((qr * 32u) << 16) + col, v);
      uint32_t m = 0;
#pragma unroll
      for (uint32_t j = 0; j < 32; ++j)
        if (ia < n0 && c0 + col + j < n1 && __uint_as_float(v[j]) >= thr) m |= 1u << j;
      masks[cc] = m;
      mine += __popc(m);
    }
    // the accumulator has been read: the next tile's first MMA may overwrite it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int w = 0; w < kTcThreads / 32; ++w) {
        const uint32_t x = wsum[w];
        wsum[w] = run;
        run += x;
      }
      tile_base = run ? atomicAdd(&s.counters->level[1], (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    unsigned long long pos = tile_base + wsum[warp] + (incl - mine);
#pragma unroll
    for (uint32_t cc = 0; cc < 4; ++cc) {
      uint32_t m = masks[cc];
      while (m) {
        const uint32_t j = __ffs(m) - 1;
        m &= m - 1;
        if (pos < d.ctb_cap) {
          s.ctb[0][pos * d.r + 0] = ia;
          s.ctb[0][pos * d.r + 1] = c0 + half * 128 + cc * 32 + j;
        } else {
          atomicOr(&s.counters->status, SSD_STATUS_CTB_OVERFLOW);
        }
        ++pos;
      }
    }
    __syncthreads();   // wsum and tile_base are reused by the next tile
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      atomicOr(&s.counters->status, SSD_STATUS_INTERNAL);
      tc_commit(&bar[2]);   // then wait (bounded) for what is still in flight before releasing
    }
    __syncthreads();
    mbar_wait(&bar[2], tiles & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// Popcount of the AND of the "recorder < k" bitmaps of tuple tl (rows 0..i-1)
// and row-i estimator idx over words [w0, w0 + n) (n a multiple of 4): all the
// 16-byte loads of the share are issued before any is used.
__device__ __forceinline__ uint32_t union_share(const Dims& d, const Scratch& s, uint32_t i,
                                                const uint32_t (&tl)[SSD_MAX_R], uint32_t idx, uint32_t w0,
                                                uint32_t n) {
  const uint64_t cap = d.hse_cap;
  const uint32_t* mine = s.pool_bm + ((uint64_t)i * cap + idx) * d.words + w0;
  uint32_t sum = 0;
  for (uint32_t w = 0; w < n; w += 16) {
    uint4 x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = w + 4 * q < n ? *reinterpret_cast<const uint4*>(mine + w + 4 * q)
                                                      : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (uint32_t j = 0; j < SSD_MAX_R; ++j) {
      if (j < i) {
        const uint32_t* row = s.pool_bm + ((uint64_t)j * cap + tl[j]) * d.words + w0 + w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (w + 4 * q < n) {
            const uint4 y = *reinterpret_cast<const uint4*>(row + 4 * q);
            x[q].x &= y.x; x[q].y &= y.y; x[q].z &= y.z; x[q].w &= y.w;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) sum += __popc(x[q].x) + __popc(x[q].y) + __popc(x[q].z) + __popc(x[q].w);
  }
  return sum;
}

// R_k of the union for every lane with a hit (idx != kNone; tl its candidate's
// tuple), computed by the warp together. Every lane of the warp makes the call.
// With bitmaps of a multiple of 16 words, groups of 4 lanes take up to 8 hits at
// a time, each lane a quarter of the words; otherwise the whole warp takes the
// hits one after another.
__device__ __forceinline__ uint32_t union_rk(const Dims& d, const Scratch& s, uint32_t i,
                                             const uint32_t (&tl)[SSD_MAX_R], uint32_t idx, int lane) {
  const bool hit = idx != kNone;
  unsigned m = __ballot_sync(kFull, hit);
  uint32_t pc = 0;
  if ((d.words & 15u) == 0) {
    const int grp = lane >> 2;
    const uint32_t per = d.words >> 2;
    while (m) {
      unsigned mm = m;   // this group's hit: the (grp+1)-th lowest set bit of m
      for (int k = 0; k < grp; ++k) mm &= mm - 1;
      const bool busy = mm != 0;
      const int src = busy ? __ffs(mm) - 1 : lane;
      uint32_t tg[SSD_MAX_R];
#pragma unroll
      for (uint32_t j = 0; j < SSD_MAX_R; ++j) tg[j] = __shfl_sync(kFull, tl[j], src);
      const uint32_t ig = __shfl_sync(kFull, idx, src);
      uint32_t part = busy ? union_share(d, s, i, tg, ig, (lane & 3) * per, per) : 0u;
      part += __shfl_xor_sync(kFull, part, 1);
      part += __shfl_xor_sync(kFull, part, 2);
      const uint32_t rank = __popc(m & ((1u << lane) - 1u));
      const uint32_t got = __shfl_sync(kFull, part, (rank < 8 ? rank : 0) * 4);
      if (((m >> lane) & 1u) && rank < 8) pc = got;
      for (int k = 0; k < 8 && m; ++k) m &= m - 1;
    }
    return pc;
  }
  const uint64_t cap = d.hse_cap;
  while (m) {
    const int L = __ffs(m) - 1;
    m &= m - 1;
    const uint32_t idxL = __shfl_sync(kFull, idx, L);
    uint32_t tL[SSD_MAX_R];
#pragma unroll
    for (uint32_t j = 0; j < SSD_MAX_R; ++j) tL[j] = __shfl_sync(kFull, tl[j], L);
    uint32_t sum = 0;
    for (uint32_t w = lane; w < d.words; w += 32) {
      uint32_t x = s.pool_bm[((uint64_t)i * cap + idxL) * d.words + w];
#pragma unroll
      for (uint32_t j = 0; j < SSD_MAX_R; ++j)
        if (j < i) x &= s.pool_bm[((uint64_t)j * cap + tL[j]) * d.words + w];
      sum += __popc(x);
    }
    sum = __reduce_add_sync(kFull, sum);
    if (lane == L) pc = sum;
  }
  return pc;
}

// Stage an accepted host with its R_k for the list (warp-wide; ok false = no entry).
__device__ __forceinline__ void stage_host(const Dims& d, const Scratch& s, bool ok, uint32_t cip, uint32_t pc) {
  const unsigned long long pos = warp_append(ok, &s.counters->raw);
  if (ok) {
    if (pos < d.out_cap) s.stage[pos] = ((unsigned long long)cip << 32) | pc;
    else atomicOr(&s.counters->status, SSD_STATUS_OUT_OVERFLOW);
  }
}

// One candidate tuple c (its pool indices tl, rows 0..i-1) of row level i
// extended by row-i estimator idx (pool index; kNone when this lane has none):
// the union test, then the append to the next candidate buffer or, at the last
// row, the final test, the host and its staging. Every lane of the warp makes
// the call (the test and the appends are warp-wide).
__device__ __forceinline__ void level_hit(const Dims& d, const Scratch& s, uint32_t i, uint32_t* sctb,
                                          const uint32_t (&tl)[SSD_MAX_R], uint32_t idx, int lane, uint32_t view) {
  const uint64_t cap = d.hse_cap;
  const bool last = (i == d.r - 1);
  const bool prune = !(d.flags & SSD_NO_PRUNE);
  const bool verify = (d.flags & SSD_VERIFY_H0) != 0;
  const bool hit = idx != kNone;
  const uint32_t pc = (prune || last) ? union_rk(d, s, i, tl, idx, lane) : 0u;
  const bool keep = hit && (!prune || pc >= d.thr);
  if (!last) {
    const unsigned long long pos = warp_append(keep, &s.counters->level[i]);
    if (keep) {
      if (pos < d.ctb_cap) {
#pragma unroll
        for (uint32_t j = 0; j < SSD_MAX_R; ++j)
          if (j < i) sctb[pos * d.r + j] = tl[j];
        sctb[pos * d.r + i] = idx;
      } else {
        atomicOr(&s.counters->status, SSD_STATUS_CTB_OVERFLOW);
      }
    }
  } else {
    warp_append(keep, &s.counters->level[i]);
    bool acc = hit && pc >= d.thr;
    uint32_t cip = 0, he0 = 0;
    if (acc) {
      uint32_t he[SSD_MAX_R];
#pragma unroll
      for (uint32_t j = 0; j < SSD_MAX_R; ++j)
        if (j < i) he[j] = s.pool_col[(uint64_t)j * cap + tl[j]];
      he[i] = s.pool_col[(uint64_t)i * cap + idx];
      acc = regain_host(d, he, &cip);
      he0 = he[0];
    }
    if (d.sh0 == 0) {
      if (acc && verify) acc = (tab_hash_global(s.tables + 1024, cip) & d.col_mask) == he0;
      if (acc) acc = view_host_in(view, cip);   // a grouped sketch holds only its group's hosts
      stage_host(d, s, acc, cip, pc);
    } else if (__any_sync(kFull, acc)) {
      // Eq. 2 as printed: every completion of bits 0..delta-1 whose RHFG[0] is he_0
      for (uint32_t low = 0; low < (1u << d.delta); ++low) {
        const uint32_t x = cip | low;
        const bool ok = acc && (tab_hash_global(s.tables + 1024, x) & d.col_mask) == he0 && view_host_in(view, x);
        stage_host(d, s, ok, x, pc);
      }
    }
  }
}

// Candidate c's tuple (rows 0..i-1) and the low q-delta bits the overlap test
// fixes for its row-i estimator.
__device__ __forceinline__ uint32_t load_candidate(const Dims& d, const Scratch& s, uint32_t i, const uint32_t* tup,
                                                   uint32_t (&tl)[SSD_MAX_R]) {
#pragma unroll
  for (uint32_t j = 0; j < SSD_MAX_R; ++j) {
    tl[j] = j < i ? tup[j] : 0u;
    if (!in_bounds(d, tl[j] < d.hse_cap)) tl[j] = 0;   // a pool index past the pool
  }
  const uint32_t he0 = s.pool_col[tl[0]];
  uint32_t tp = 0;
#pragma unroll
  for (uint32_t j = 0; j < SSD_MAX_R; ++j)
    if (j == i - 1) tp = tl[j];
  const uint32_t hep = s.pool_col[(uint64_t)(i - 1) * d.hse_cap + tp];
  const uint32_t want_low = (he0 ^ hep) >> d.delta;  // high q-delta bits of B(i-1)
  return (he0 ^ want_low) & d.low_mask;
}

__global__ void __launch_bounds__(kBlock) k_level(const Dims d, const Scratch s, const uint32_t i,
                                                  const uint32_t* __restrict__ rctb, uint32_t* __restrict__ sctb,
                                                  const uint32_t view) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const unsigned long long avail = s.counters->level[i - 1];
  const uint64_t nc = avail < d.ctb_cap ? avail : d.ctb_cap;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t tl[SSD_MAX_R];   // the lane's candidate tuple (zero for a lane without one)
#pragma unroll
  for (uint32_t j = 0; j < SSD_MAX_R; ++j) tl[j] = 0;
  if (s.bucket_off) {
    // one candidate per lane; round p takes each lane's p-th bucket entry
    const uint32_t nb = 1u << d.low_bits;
    const uint32_t* off = s.bucket_off + (uint64_t)i * (nb + 1);
    const uint32_t* ent = s.bucket_ent + (uint64_t)i * d.hse_cap;
    for (uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < nc; w0 += stride) {
      const uint64_t c = w0 + lane;
      uint32_t b = 0, e = 0;
      if (c < nc) {
        const uint32_t low = load_candidate(d, s, i, rctb + c * d.r, tl);
        b = off[low];
        e = off[low + 1];
        if (!in_bounds(d, b <= e && e <= d.hse_cap)) b = e = 0;
      }
      for (uint32_t p = 0; __any_sync(kFull, b + p < e); ++p)
        level_hit(d, s, i, sctb, tl, b + p < e ? ent[b + p] : kNone, lane, view);
    }
    return;
  }
  // probes: 2^delta columns of row i per candidate, one per lane
  const uint64_t total = nc << d.delta;
  for (uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < total; w0 += stride) {
    const uint64_t item = w0 + lane;
    uint32_t idx = kNone;
    if (item < total) {
      const uint32_t h = (uint32_t)(item & ((1u << d.delta) - 1u));
      const uint32_t he_i = (h << d.low_bits) | load_candidate(d, s, i, rctb + (item >> d.delta) * d.r, tl);
      idx = in_bounds(d, he_i < (1u << d.q)) ? s.hot_idx[((uint64_t)i << d.q) | he_i] : kNone;
    }
    level_hit(d, s, i, sctb, tl, idx, lane, view);
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
  pdl_enter();
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
                               unsigned long long* n_out_dev, int sms, cudaStream_t st, int* launches,
                               uint32_t view, bool tensor_pairs) {
  // k_list's and k_pairs_tc's dynamic shared memory limits and k_pairs' occupancy, once per device
  constexpr int kDevices = 64;
  static bool attr[kDevices] = {};
  static bool tc_attr[kDevices] = {};
  static int pair_bps_of[kDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(k_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemKeys * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  int& pair_bps = pair_bps_of[dev];   // resident k_pairs blocks per SM
  if (!pair_bps) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pair_bps, k_pairs, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (pair_bps < 1) pair_bps = 1;
  }
  const uint32_t bucket_blocks = s.bucket_off && d.r > 2 ? d.r - 2 : 0;
  if (tensor_pairs && !(d.flags & SSD_NO_PRUNE) && (d.words & 3u) == 0) {
    if (!tc_attr[dev]) {
      e = cudaFuncSetAttribute(k_pairs_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
      if (e != cudaSuccess) return e;
      tc_attr[dev] = true;
    }
    const uint32_t tile_blocks = (uint32_t)sms;   // one resident block per SM (registers); each loops over tiles
    e = launch_pdl(k_pairs_tc, tile_blocks + bucket_blocks, kTcThreads, kTcSmem, st, d, s, tile_blocks);
  } else {
    const uint32_t pair_blocks = (uint32_t)(sms * pair_bps);
    e = launch_pdl(k_pairs, pair_blocks + bucket_blocks, kBlock, 0, st, d, s, pair_blocks);
  }
  if (e != cudaSuccess) return e;
  *launches += 1;
  for (uint32_t i = 2; i < d.r; ++i) {
    // level 1 (pairs) wrote ctb[0]; level i reads ctb[i & 1] and writes ctb[(i + 1) & 1]
    const uint32_t* rctb = s.ctb[i & 1];
    uint32_t* sctb = s.ctb[(i + 1) & 1];
    e = launch_pdl(k_level, (unsigned)(sms * 8), kBlock, 0, st, d, s, i, rctb, sctb, view);
    if (e != cudaSuccess) return e;
    *launches += 1;
  }
  e = launch_pdl(k_list, 1, kListThreads, kSmemKeys * sizeof(unsigned long long), st, d, s, ips, rk, cap, n_out_dev);
  *launches += 1;
  return e;
}

}  // namespace ssd
