// Diagnostics over a whole RSEA: per-row sums of R_k (the recorders below k,
// Sec. 3.2). A row's mean R_k gives, through Eq. 1, the distinct opposite
// hosts a column holds: the realised column load that decides whether a
// parameter set is feasible for a workload (every column hot once it nears
// theta). Not on the slot path.
#include "ssd_internal.cuh"

namespace ssd {
namespace {

// Grid-stride over the RSEA's 16-byte vectors; a thread's count goes to its
// block's row total when its row changes, the block's totals to rk_sum.
__global__ void __launch_bounds__(kBlock) k_occupancy(const Dims d, const uint4* __restrict__ dr,
                                                      const uint32_t* tm, unsigned long long* rk_sum) {
  __shared__ unsigned long long part[SSD_MAX_R];
  const Clock c = make_clock(read_tm(tm), d.k);   // the recorders are stamps at this clock
  if (threadIdx.x < SSD_MAX_R) part[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t per_row = ((uint64_t)1 << (d.q + d.log2_eta)) >> 3;
  const uint64_t total = per_row * d.r;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t row = 0;
  unsigned long long cnt = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += stride) {
    const uint32_t rv = (uint32_t)(v / per_row);
    if (rv != row) {
      if (cnt) atomicAdd(&part[row], cnt);
      cnt = 0;
      row = rv;
    }
    cnt += __popc(win8(__ldcs(dr + v), c));   // the window test of the streaming passes
  }
  if (cnt) atomicAdd(&part[row], cnt);
  __syncthreads();
  if (threadIdx.x < d.r && part[threadIdx.x]) atomicAdd(&rk_sum[threadIdx.x], part[threadIdx.x]);
}

}  // namespace

cudaError_t launch_occupancy(const Dims& d, const uint16_t* dr, const uint32_t* tm, unsigned long long* rk_sum,
                             int sms, cudaStream_t st) {
  k_occupancy<<<sms * 8, kBlock, 0, st>>>(d, reinterpret_cast<const uint4*>(dr), tm, rk_sum);
  return cudaGetLastError();
}

}  // namespace ssd
