// stdp.cu -- nearest-neighbour spike-timing-dependent plasticity (Sec. 2.1,
// after Morrison et al. 2008; weight dependence of Guetig et al. 2003).
//
// A spike reaches its synapse `delay` steps after it was fired (its arrival
// step).  Depression happens at the arrival, inside the spike-buffer
// delivery of the due group (deliver_item.cuh): the synapse is depressed by
// its target's latest spike, records the arrival step and delivers the
// depressed weight.  Potentiation happens here, after the update kernels of
// step t and before the delivery of step t: every neuron that fired at step
// t and has plastic inputs (listed by the update kernels) potentiates each
// of them by that synapse's latest arrival (at or before step t, as the
// arrivals for step t + 1 are recorded only by the delivery that follows).
//
// Work: the grid's warps are spread over the listed neurons, G warps per
// neuron (G = warps / neurons, at least 1), each taking every G-th group of
// 32 of the neuron's incoming plastic synapses (the reverse index built at
// finalisation), so that a step with few firing targets still has every warp
// issuing its gathers; each lane handles two synapses per pass with both
// chains of loads in flight.  Bytes per synapse update: 8 (index word) + 8
// (weight-and-arrival word read) + 4 (weight write).
#include <cuda_runtime.h>

#include "builder.h"
#include "ngb_internal.cuh"
#include "stdp_rule.cuh"

namespace ngb {

__global__ void __launch_bounds__(256) k_stdp_post(SpikeBuf sb, StdpArgs a, const int64_t* clk) {
  griddep_wait();  // the step's update kernels have completed
  griddep_launch();
  const int64_t t = clk[1];
  const int pb = (int)(t & 1);
  const unsigned long long n = sb.post_cnt[pb];
  // the next step's list starts empty (its update kernels run after this kernel)
  if (blockIdx.x == 0 && threadIdx.x == 0) sb.post_cnt[pb ^ 1] = 0;
  const uint32_t* __restrict__ list = pb ? sb.post[1] : sb.post[0];
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  if (n == 0) return;
  const unsigned long long G = n >= nwarps ? 1ull : nwarps / n;
  const uint64_t stride = 32ull * G;
  const uint64_t kMask = (1ull << kStdpRuleShift) - 1;
  for (unsigned long long v = warp; v < n * G; v += nwarps) {
    const uint32_t gid = list[v / G];
    const uint64_t sub = v % G;
    const uint64_t lo = sb.in_ptr[gid], hi = sb.in_ptr[gid + 1];
    for (uint64_t k = lo + sub * 32 + (uint64_t)lane; k < hi; k += 2 * stride) {
      const bool two = k + stride < hi;
      const uint64_t w0 = a.in_syn[k];
      const uint64_t w1 = two ? a.in_syn[k + stride] : 0ull;
      const uint64_t j0 = w0 & kMask, j1 = w1 & kMask;
      const uint2 p0 = a.wa[j0];
      const uint2 p1 = two ? a.wa[j1] : make_uint2(0u, 0xFFFFFFFFu);
      const int32_t r0 = (int32_t)p0.y, r1 = (int32_t)p1.y;
      uint32_t* const w32 = reinterpret_cast<uint32_t*>(a.wa);
      if (r0 >= 0)
        w32[2 * j0] = __float_as_uint(
            stdp_potentiate(a.rules[w0 >> kStdpRuleShift], __uint_as_float(p0.x), (int64_t)t - (int64_t)r0));
      if (r1 >= 0)
        w32[2 * j1] = __float_as_uint(
            stdp_potentiate(a.rules[w1 >> kStdpRuleShift], __uint_as_float(p1.x), (int64_t)t - (int64_t)r1));
    }
  }
}

cudaError_t launch_stdp_post(SpikeBuf sb, StdpArgs a, const int64_t* clk, int grid, bool pdl, cudaStream_t st) {
  return launch_k(k_stdp_post, dim3((unsigned)grid), dim3(256), pdl, st, sb, a, clk);
}

namespace {
__global__ void k_init_stdp_words(const float* __restrict__ w, uint64_t K, uint2* wa) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < K; j += (uint64_t)gridDim.x * blockDim.x)
    wa[j] = make_uint2(__float_as_uint(w[j]), 0xFFFFFFFFu);
}

__global__ void k_sync_stdp_weights(const uint2* __restrict__ wa, const uint32_t* __restrict__ tgt, uint64_t first,
                                    uint64_t n, float* w) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = first + i;
    if ((tgt[j] >> kPlastShift) & kPlastMask) w[j] = __uint_as_float(wa[j].x);
  }
}
}  // namespace

cudaError_t init_stdp_words(const float* w, uint64_t K, uint2* wa, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  k_init_stdp_words<<<1024, 256, 0, st>>>(w, K, wa);
  return cudaGetLastError();
}

cudaError_t sync_stdp_weights(const uint2* wa, const uint32_t* tgt, uint64_t first, uint64_t n, float* w,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_sync_stdp_weights<<<1024, 256, 0, st>>>(wa, tgt, first, n, w);
  return cudaGetLastError();
}

// Reverse index of the plastic synapses: count per target, scan, fill.
namespace {
__global__ void k_count_plastic(const uint32_t* __restrict__ tgt, uint64_t K, unsigned long long* cnt) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < K; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t tw = tgt[j];
    if ((tw >> kPlastShift) & kPlastMask) atomicAdd(cnt + (tw & kTgtMask), 1ull);
  }
}

__global__ void k_fill_plastic(const uint32_t* __restrict__ tgt, uint64_t K, unsigned long long* cursor,
                               uint64_t* in_syn) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < K; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t tw = tgt[j];
    const uint32_t cls = (tw >> kPlastShift) & kPlastMask;
    if (!cls) continue;
    const unsigned long long pos = atomicAdd(cursor + (tw & kTgtMask), 1ull);
    in_syn[pos] = ((uint64_t)(cls - 1) << kStdpRuleShift) | j;
  }
}
}  // namespace

cudaError_t build_stdp_index(const uint32_t* tgt, uint64_t K, int64_t N, uint64_t* in_ptr, uint64_t** in_syn_out,
                             uint64_t* n_plastic_out, cudaStream_t st) {
  *in_syn_out = nullptr;
  *n_plastic_out = 0;
  unsigned long long* cnt = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  const int grid = 1024;
  cudaError_t e = cudaMalloc(&cnt, (size_t)(N + 1) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)(N + 1) * sizeof(unsigned long long), st);
  if (e == cudaSuccess && K > 0) {
    k_count_plastic<<<grid, 256, 0, st>>>(tgt, K, cnt);
    e = cudaGetLastError();
  }
  // in_ptr = exclusive scan of the counts (N + 1 entries: the last is the total)
  if (e == cudaSuccess) e = scan_scratch_bytes_u64((uint64_t)N + 1, &tmp_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 1);
  if (e == cudaSuccess)
    e = exclusive_scan_u64(cnt, reinterpret_cast<unsigned long long*>(in_ptr), (uint64_t)N + 1, tmp, tmp_bytes, st);
  uint64_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, in_ptr + N, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  uint64_t* in_syn = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&in_syn, (size_t)(total > 0 ? total : 1) * sizeof(uint64_t));
  // the counts become fill cursors starting at in_ptr
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt, in_ptr, (size_t)N * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && K > 0) {
    k_fill_plastic<<<grid, 256, 0, st>>>(tgt, K, cnt, in_syn);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(cnt);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    cudaFree(in_syn);
    return e;
  }
  *in_syn_out = in_syn;
  *n_plastic_out = total;
  return cudaSuccess;
}

}  // namespace ngb
