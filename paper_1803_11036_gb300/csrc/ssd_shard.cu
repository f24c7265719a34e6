// The reduction step of a merge whose routers are spread over several GPUs
// (Algorithm 5 across monitor servers, Sec. 4): each GPU folds the slices of
// one recorder range that the other GPUs sent it into that range of the global
// RSEA, with the elementwise minimum of the union reading. Collective
// libraries have no 16-bit minimum, so the wire carries bytes and this kernel
// reduces them.
#include <cstring>

#include "ssd_internal.cuh"

namespace ssd {
namespace {

struct MinArgs {
  int n;
  const uint4* in[kMaxBatch];
  uint4* out;
  uint64_t nvec;    // 16-byte vectors (8 recorders) of every input
};

__device__ __forceinline__ uint4 vmin8(uint4 a, uint4 b) {
  return make_uint4(__vminu2(a.x, b.x), __vminu2(a.y, b.y), __vminu2(a.z, b.z), __vminu2(a.w, b.w));
}

// out[v] = min over the n inputs of in[j][v], for every 16-byte vector v; the
// loads of eight inputs are issued before they are folded.
__global__ void __launch_bounds__(kBlock) k_min_ranges(const __grid_constant__ MinArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.nvec; v += stride) {
    uint4 m = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    for (int j0 = 0; j0 < a.n; j0 += 8) {
      uint4 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < a.n) x[u] = __ldcs(a.in[j0 + u] + v);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < a.n) m = vmin8(m, x[u]);
    }
    __stcs(a.out + v, m);
  }
}

// The recorders past the last whole vector (count mod 8), one thread each.
struct TailArgs {
  const uint16_t* in[kMaxBatch];
};

__global__ void k_min_tail_args(const __grid_constant__ TailArgs a, int n, uint16_t* out, uint64_t first, uint32_t m) {
  const uint32_t t = threadIdx.x;
  if (t >= m) return;
  uint16_t v = 0xFFFFu;
  for (int j = 0; j < n; ++j) {
    const uint16_t x = a.in[j][first + t];
    v = x < v ? x : v;
  }
  out[first + t] = v;
}

}  // namespace

cudaError_t launch_min_ranges(uint16_t* out, const uint16_t* const* in, int n, uint64_t count, int sms,
                              cudaStream_t st) {
  const uint64_t nvec = count >> 3;
  if (nvec) {
    MinArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    for (int j = 0; j < n; ++j) a.in[j] = reinterpret_cast<const uint4*>(in[j]);
    a.out = reinterpret_cast<uint4*>(out);
    a.nvec = nvec;
    uint64_t grid = (nvec + kBlock - 1) / kBlock;
    const uint64_t cap = (uint64_t)sms * 8;
    if (grid > cap) grid = cap;
    k_min_ranges<<<(unsigned)grid, kBlock, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const uint32_t m = (uint32_t)(count & 7u);
  if (m) {
    TailArgs t;
    std::memset(&t, 0, sizeof(t));
    for (int j = 0; j < n; ++j) t.in[j] = in[j];
    k_min_tail_args<<<1, 32, 0, st>>>(t, n, out, nvec << 3, m);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace ssd
