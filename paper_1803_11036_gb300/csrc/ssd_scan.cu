// IP pair scanning (Algorithm 2, Sec. 4.1) for one or many routers in one launch.
//
// Each thread takes 16-byte vectors of the pair stream (two packets per
// vector), hashes both addresses with the simple-tabulation tables held in
// shared memory, and sets the r recorders RSEA[i, RHFG[i](cip)][H1(oip)] to 0,
// which for the library's stamp recorders is a store of the sketch's clock.
// Setting a recorder to 0 is idempotent and order-free (Sec. 4.1), so the
// stores need no atomics and no ordering between threads.
#include "ssd_internal.cuh"

namespace ssd {
namespace {

// Algorithm 2 for one pair: DRidx = H1(oip); RHFG[0](cip) from the second table
// set; RHFG[i](cip) = ((cip >> (i-1)*delta) ^ RHFG[0](cip)) mod 2^q for i >= 1.
// The recorders take distance 0: the stamp `now` (the sketch's clock).
__device__ __forceinline__ void scan_pair(uint16_t* __restrict__ dr, uint16_t now, uint32_t cip, uint32_t oip,
                                          const uint32_t* sT, const Dims& d) {
  const uint32_t j = tab_hash(sT, oip) & (d.eta - 1u);
  const uint32_t c0 = tab_hash(sT + 1024, cip) & d.col_mask;
  if (in_bounds(d, j < d.eta && c0 < (1u << d.q))) dr[((uint64_t)c0 << d.log2_eta) | j] = now;
#pragma unroll
  for (uint32_t i = 1; i < SSD_MAX_R; ++i) {
    if (i < d.r) {
      const uint32_t sh = (i - 1u) * d.delta + d.sh0;
      const uint32_t w = sh < 32u ? (cip >> sh) : 0u;
      const uint32_t col = (w ^ c0) & d.col_mask;
      if (in_bounds(d, col < (1u << d.q))) dr[((((uint64_t)i << d.q) | col) << d.log2_eta) | j] = now;
    }
  }
}

// scan_pair on the stored pair (x, y) through a job's view (side and group).
__device__ __forceinline__ void scan_view(uint16_t* __restrict__ dr, uint16_t now, uint32_t view, uint32_t x,
                                          uint32_t y, const uint32_t* sT, const Dims& d) {
  uint32_t cip, oip;
  if (view_pair(view, x, y, cip, oip)) scan_pair(dr, now, cip, oip, sT, d);
}

// touch_pair on the stored pair (x, y) through a job's view; every lane makes the
// call (a pair outside the view's group takes part as a no-op).
template <int CM>
__device__ __forceinline__ void touch_view(uint32_t* bits, uint64_t jbase, uint32_t view, uint32_t x, uint32_t y,
                                           bool live, const uint32_t* sT, const Dims& d, uint32_t r0, uint32_t r1,
                                           uint64_t se0, uint64_t count) {
  uint32_t cip, oip;
  const bool in = view_pair(view, x, y, cip, oip);
  touch_pair<CM>(bits, jbase, cip, oip, live && in, sT, d, r0, r1, se0, count);
}

__device__ __forceinline__ int find_router(const ScanBatch& b, uint64_t v) {
  int lo = 0, hi = b.n - 1;
  while (lo < hi) {  // last j with prefix[j] <= v
    const int mid = (lo + hi + 1) >> 1;
    if (b.prefix[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// U: 16-byte pair vectors each thread loads before it hashes any of them.
template <int U>
__global__ void __launch_bounds__(kBlock) k_scan(const Dims d, const uint32_t* __restrict__ tables,
                                                 const __grid_constant__ ScanBatch b) {
  __shared__ uint32_t sT[2048];
  __shared__ uint16_t sNow[kMaxBatch];   // each job's stamp: its sketch's clock
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) sT[i] = tables[i];
  if (threadIdx.x < b.n) sNow[threadIdx.x] = (uint16_t)read_tm(b.tm[threadIdx.x]);
  __syncthreads();

  // packets outside the 16-byte aligned bodies: a head when a buffer starts at
  // 8 mod 16, a tail when the body leaves one packet over
  if (blockIdx.x == 0 && threadIdx.x < 2 * b.n) {
    const uint32_t* e = b.edge[threadIdx.x];
    const int j = threadIdx.x >> 1;
    if (e) scan_view(b.dr[j], sNow[j], b.view[j], e[0], e[1], sT, d);
  }

  const uint64_t total = b.prefix[b.n];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b.n == 1) {
    const uint4* __restrict__ vec = b.vec[0];
    uint16_t* __restrict__ dr = b.dr[0];
    const uint32_t view = b.view[0];
    const uint16_t now = sNow[0];
    for (; v + (U - 1) * stride < total; v += U * stride) {
      uint4 w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) w[u] = __ldcs(vec + v + u * stride);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        scan_view(dr, now, view, w[u].x, w[u].y, sT, d);
        scan_view(dr, now, view, w[u].z, w[u].w, sT, d);
      }
    }
    for (; v < total; v += stride) {
      const uint4 w = __ldcs(vec + v);
      scan_view(dr, now, view, w.x, w.y, sT, d);
      scan_view(dr, now, view, w.z, w.w, sT, d);
    }
  } else {
    for (; v + (U - 1) * stride < total; v += U * stride) {
      uint4 w[U];
      int jj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t vv = v + u * stride;
        const int j = find_router(b, vv);
        w[u] = __ldcs(b.vec[j] + (vv - b.prefix[j]));
        jj[u] = j;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = jj[u];
        scan_view(b.dr[j], sNow[j], b.view[j], w[u].x, w[u].y, sT, d);
        scan_view(b.dr[j], sNow[j], b.view[j], w[u].z, w[u].w, sT, d);
      }
    }
    for (; v < total; v += stride) {
      const int j = find_router(b, v);
      const uint4 w = __ldcs(b.vec[j] + (v - b.prefix[j]));
      scan_view(b.dr[j], sNow[j], b.view[j], w.x, w.y, sT, d);
      scan_view(b.dr[j], sNow[j], b.view[j], w.z, w.w, sT, d);
    }
  }
}

// The touch kernels walk the vectors warp by warp (vb = the warp's first
// vector, a multiple of 32 because the grid stride is): every lane of a warp
// runs the same iterations, as set_touch<1> needs; a lane past the end only
// takes part.
template <int U, int CM>
__global__ void __launch_bounds__(kBlock) k_touch(const Dims d, const uint32_t* __restrict__ tables,
                                                  const __grid_constant__ ScanBatch b, uint32_t* __restrict__ bits,
                                                  uint64_t se0, uint64_t count) {
  __shared__ uint32_t sT[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) sT[i] = tables[i];
  __syncthreads();
  const uint32_t r0 = (uint32_t)(se0 >> d.q), r1 = (uint32_t)((se0 + count - 1) >> d.q);
  const uint32_t lane = threadIdx.x & 31u;
  if (blockIdx.x == 0 && threadIdx.x < 2 * b.n) {
    const uint32_t* e = b.edge[threadIdx.x];
    if (e)
      touch_view<0>(bits, (uint64_t)(threadIdx.x >> 1) * count, b.view[threadIdx.x >> 1], e[0], e[1], true, sT, d, r0,
                    r1, se0, count);
  }
  const uint64_t total = b.prefix[b.n];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t vb = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
  for (; vb + 31 + (U - 1) * stride < total; vb += U * stride) {
    uint4 w[U];
    uint64_t jb[U];
    uint32_t vw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t vv = vb + lane + u * stride;
      const int j = b.n == 1 ? 0 : find_router(b, vv);
      w[u] = __ldcs(b.vec[j] + (vv - b.prefix[j]));
      jb[u] = (uint64_t)j * count;
      vw[u] = b.view[j];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      touch_view<CM>(bits, jb[u], vw[u], w[u].x, w[u].y, true, sT, d, r0, r1, se0, count);
      touch_view<CM>(bits, jb[u], vw[u], w[u].z, w[u].w, true, sT, d, r0, r1, se0, count);
    }
  }
  for (; vb < total; vb += stride) {
    const uint64_t v = vb + lane;
    const bool live = v < total;
    uint4 w = make_uint4(0, 0, 0, 0);
    uint64_t jb = 0;
    uint32_t vw = 0;
    if (live) {
      const int j = b.n == 1 ? 0 : find_router(b, v);
      w = __ldcs(b.vec[j] + (v - b.prefix[j]));
      jb = (uint64_t)j * count;
      vw = b.view[j];
    }
    touch_view<CM>(bits, jb, vw, w.x, w.y, live, sT, d, r0, r1, se0, count);
    touch_view<CM>(bits, jb, vw, w.z, w.w, live, sT, d, r0, r1, se0, count);
  }
}

// Both hashes of every pair once per slot: packed = RHFG[0](cip) | H1(oip) << q.
__global__ void __launch_bounds__(kBlock) k_prehash(const Dims d, const uint32_t* __restrict__ tables,
                                                    const __grid_constant__ ScanBatch b, uint2* __restrict__ out) {
  __shared__ uint32_t sT[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) sT[i] = tables[i];
  __syncthreads();
  const uint64_t nvec = b.prefix[1];
  const uint32_t view = b.view[0];
  auto pack = [&](uint32_t x, uint32_t y) {
    uint32_t cip, oip;
    view_pair(view, x, y, cip, oip);   // the side only: grouped views are not pre-hashed
    return make_uint2(cip, (tab_hash(sT + 1024, cip) & d.col_mask) | ((tab_hash(sT, oip) & (d.eta - 1u)) << d.q));
  };
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
    const uint4 w = __ldcs(b.vec[0] + v);
    const uint2 p0 = pack(w.x, w.y), p1 = pack(w.z, w.w);
    reinterpret_cast<uint4*>(out)[v] = make_uint4(p0.x, p0.y, p1.x, p1.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint64_t at = 2 * nvec;
    for (int k = 0; k < 2; ++k) {
      const uint32_t* e = b.edge[k];
      if (e) out[at++] = pack(e[0], e[1]);
    }
  }
}

template <int U, int CM>
__global__ void __launch_bounds__(kBlock) k_touch_packed(const Dims d, const uint4* __restrict__ vec, uint64_t nvec,
                                                         const uint2* __restrict__ tail, uint32_t* __restrict__ bits,
                                                         uint64_t se0, uint64_t count) {
  const uint32_t r0 = (uint32_t)(se0 >> d.q), r1 = (uint32_t)((se0 + count - 1) >> d.q);
  const uint32_t lane = threadIdx.x & 31u;
  if (blockIdx.x == 0 && threadIdx.x == 0 && tail) touch_packed<0>(bits, tail->x, tail->y, true, d, r0, r1, se0, count);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t vb = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);  // as in k_touch
  for (; vb + 31 + (U - 1) * stride < nvec; vb += U * stride) {
    uint4 w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = __ldcs(vec + vb + lane + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      touch_packed<CM>(bits, w[u].x, w[u].y, true, d, r0, r1, se0, count);
      touch_packed<CM>(bits, w[u].z, w[u].w, true, d, r0, r1, se0, count);
    }
  }
  for (; vb < nvec; vb += stride) {
    const bool live = vb + lane < nvec;
    const uint4 w = live ? __ldcs(vec + vb + lane) : make_uint4(0, 0, 0, 0);
    touch_packed<CM>(bits, w.x, w.y, live, d, r0, r1, se0, count);
    touch_packed<CM>(bits, w.z, w.w, live, d, r0, r1, se0, count);
  }
}

// Per-chunk touch lists (see ListArgs). Each block owns a contiguous range of
// the batch's pair vectors and walks it twice: the first walk sets chunk 0's
// bits and counts the block's touches per chunk (warp-aggregated shared-memory
// atomics), one global atomic per chunk then reserves the block's run in each
// list, and the second walk hashes the same pairs again and writes the bit
// indices into the reserved runs. The range (about 40 KB at full size) is
// still in L2 for the second walk. Every lane of a warp runs the same
// iterations (__match_any_sync needs all 32).
template <int CM>
__global__ void __launch_bounds__(kBlock) k_lists(const Dims d, const uint32_t* __restrict__ tables,
                                                  const __grid_constant__ ScanBatch b, const ListArgs a) {
  __shared__ uint32_t sT[2048];
  __shared__ uint32_t s_cnt[kMaxChunks], s_cur[kMaxChunks];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) sT[i] = tables[i];
  if (threadIdx.x < kMaxChunks) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t count = 1ull << a.log2_count;
  const uint64_t total = b.prefix[b.n];
  uint64_t per = (total + gridDim.x - 1) / gridDim.x;
  per = (per + 31) & ~31ull;
  const uint64_t v0 = (uint64_t)blockIdx.x * per;
  const uint64_t v1 = v0 + per < total ? v0 + per : total;

  // the touches of one pair (x, y) of router j: chunk 0's set (first walk), the others counted
  // (first walk) or written (second walk)
  auto pair = [&](uint32_t x, uint32_t y, uint32_t view, uint64_t jbase, bool live, bool write) {
    uint32_t cip = 0, oip = 0;
    const bool in = live && view_pair(view, x, y, cip, oip);
    uint32_t xr = 0, c0 = 0;
    if (in) {
      xr = tab_hash(sT, oip) & (d.eta - 1u);
      c0 = tab_hash(sT + 1024, cip) & d.col_mask;
    }
#pragma unroll
    for (uint32_t i = 0; i < SSD_MAX_R; ++i) {
      if (i < d.r) {
        uint32_t col = c0;
        if (i) {
          const uint32_t sh = (i - 1u) * d.delta + d.sh0;
          col = ((sh < 32u ? (cip >> sh) : 0u) ^ c0) & d.col_mask;
        }
        const uint64_t se = ((uint64_t)i << d.q) | col;
        const uint32_t c = (uint32_t)(se >> a.log2_count);
        const uint64_t bit = ((jbase + (se & (count - 1))) << d.log2_eta) | touch_pos(d, xr);
        if (!write) set_touch<CM>(a.touch0, bit, in && c == 0 && in_bounds(d, bit < d.touch_bits));
        const uint32_t key = (in && c != 0) ? c : 0xFFFFFFFFu;
        const uint32_t grp = __match_any_sync(0xFFFFFFFFu, key);
        if (key != 0xFFFFFFFFu) {
          const uint32_t leader = __ffs(grp) - 1u;
          if (!write) {
            if (lane == leader) atomicAdd(&s_cnt[key], (uint32_t)__popc(grp));
          } else {
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&s_cur[key], (uint32_t)__popc(grp));
            base = __shfl_sync(grp, base, leader);
            const uint64_t pos = (uint64_t)base + __popc(grp & lt);
            if (pos < a.cap) a.ent[(uint64_t)(key - 1u) * a.cap + pos] = (uint32_t)bit;
            else atomicOr(&a.counters->status, SSD_STATUS_INTERNAL);
          }
        }
      }
    }
  };
  auto walk = [&](bool write) {
    for (uint64_t vb = v0 + (threadIdx.x & ~31u); vb < v1; vb += kBlock) {
      const uint64_t v = vb + lane;
      const bool live = v < v1;
      uint4 w = make_uint4(0, 0, 0, 0);
      uint64_t jb = 0;
      uint32_t vw = 0;
      if (live) {
        const int j = b.n == 1 ? 0 : find_router(b, v);
        w = write ? __ldcs(b.vec[j] + (v - b.prefix[j])) : __ldcg(b.vec[j] + (v - b.prefix[j]));
        jb = (uint64_t)j * count;
        vw = b.view[j];
      }
      pair(w.x, w.y, vw, jb, live, write);
      pair(w.z, w.w, vw, jb, live, write);
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {   // the packets outside the 16-byte bodies
      const uint32_t* e = lane < 2u * (uint32_t)b.n ? b.edge[lane] : nullptr;
      const uint32_t j = lane >> 1;
      pair(e ? e[0] : 0u, e ? e[1] : 0u, e ? b.view[j] : 0u, (uint64_t)j * count, e != nullptr, write);
    }
  };
  walk(false);
  __syncthreads();
  if (threadIdx.x >= 1 && threadIdx.x < a.n_chunks)
    s_cur[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&a.fill[threadIdx.x], s_cnt[threadIdx.x]) : 0u;
  __syncthreads();
  walk(true);
}

}  // namespace

cudaError_t launch_lists(const Dims& d, const uint32_t* tables, const ScanBatch& b, const ListArgs& a, int grid,
                         const Tuning& tn, cudaStream_t st) {
  if (a.n_chunks > kMaxChunks || b.n > 16) return cudaErrorInvalidValue;
  if (tn.combine == 1) k_lists<1><<<grid, kBlock, 0, st>>>(d, tables, b, a);
  else if (tn.combine == 2) k_lists<2><<<grid, kBlock, 0, st>>>(d, tables, b, a);
  else k_lists<0><<<grid, kBlock, 0, st>>>(d, tables, b, a);
  return cudaGetLastError();
}

cudaError_t launch_prehash(const Dims& d, const uint32_t* tables, const ScanBatch& b, uint2* out, int grid,
                           cudaStream_t st) {
  k_prehash<<<grid, kBlock, 0, st>>>(d, tables, b, out);
  return cudaGetLastError();
}

// Launches KERNEL<U, CM> for the tuning's unroll (U) and combine mode (CM).
#define SSD_TUNED_CM(KERNEL, U, GRID, ST, ...)                                             \
  do {                                                                                    \
    if (tn.combine == 1) KERNEL<U, 1><<<GRID, kBlock, 0, ST>>>(__VA_ARGS__);             \
    else if (tn.combine == 2) KERNEL<U, 2><<<GRID, kBlock, 0, ST>>>(__VA_ARGS__);        \
    else KERNEL<U, 0><<<GRID, kBlock, 0, ST>>>(__VA_ARGS__);                             \
  } while (0)
#define SSD_TUNED_LAUNCH(KERNEL, GRID, ST, ...)                                           \
  do {                                                                                    \
    switch (tn.unroll) {                                                                  \
      case 1: SSD_TUNED_CM(KERNEL, 1, GRID, ST, __VA_ARGS__); break;                      \
      case 2: SSD_TUNED_CM(KERNEL, 2, GRID, ST, __VA_ARGS__); break;                      \
      case 8: SSD_TUNED_CM(KERNEL, 8, GRID, ST, __VA_ARGS__); break;                      \
      default: SSD_TUNED_CM(KERNEL, 4, GRID, ST, __VA_ARGS__); break;                     \
    }                                                                                     \
  } while (0)

cudaError_t launch_touch_packed(const Dims& d, const uint4* vec, uint64_t nvec, const uint2* tail, uint32_t* bits,
                                uint64_t se0, uint64_t se_count, int grid, const Tuning& tn, cudaStream_t st) {
  SSD_TUNED_LAUNCH(k_touch_packed, grid, st, d, vec, nvec, tail, bits, se0, se_count);
  return cudaGetLastError();
}

cudaError_t launch_touch(const Dims& d, const uint32_t* tables, const ScanBatch& b, uint32_t* bits, uint64_t se0,
                         uint64_t se_count, int grid, const Tuning& tn, cudaStream_t st) {
  SSD_TUNED_LAUNCH(k_touch, grid, st, d, tables, b, bits, se0, se_count);
  return cudaGetLastError();
}
#undef SSD_TUNED_LAUNCH
#undef SSD_TUNED_CM

cudaError_t launch_scan(const Dims& d, const uint32_t* tables, const ScanBatch& b, int grid, const Tuning& tn,
                        cudaStream_t st) {
  static_assert(sizeof(ScanBatch) < 32000, "kernel parameter block too large");
  switch (tn.unroll) {
    case 1: k_scan<1><<<grid, kBlock, 0, st>>>(d, tables, b); break;
    case 2: k_scan<2><<<grid, kBlock, 0, st>>>(d, tables, b); break;
    case 8: k_scan<8><<<grid, kBlock, 0, st>>>(d, tables, b); break;
    default: k_scan<4><<<grid, kBlock, 0, st>>>(d, tables, b); break;
  }
  return cudaGetLastError();
}

}  // namespace ssd
