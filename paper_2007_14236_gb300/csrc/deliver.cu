// deliver.cu -- spike delivery kernel (K3).
//
// Sec. 2.2 of the paper: every spike of step t reaches each target of the
// source's connection groups after the group's delay.  Here the spikes of step
// t (compacted by the update kernels) are scattered into the targets' input
// ring buffer at slot (t + d) & (L - 1), one atomic add per synapse.
//
// Work decomposition (load-balanced, synapse-parallel): every spiking source
// contributes ceil((end - align4(begin)) / 128) work items of 128 consecutive
// synapses, aligned to 16 bytes; the compaction already assigned each spike
// the index of its first work item, so a warp maps a work item to its spike
// by binary search over the (monotone) work-item offsets.  Each lane then
// loads 4 target words (one 16-byte load) and 4 weights (16 or 8 bytes) with
// non-caching loads, finds each synapse's delay group by advancing from the
// work item's first group, and issues one red.global.add per synapse:
// FP32 (or int64 fixed point in deterministic mode).
//
// Reading a spike's delay groups costs two loads per work item; reading the
// synapses costs 8 (FP32) or 6 (BF16/FP16) bytes per synapse; the
// accumulation costs one 4-byte (8-byte) L2 atomic per synapse.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ngb_internal.cuh"

namespace ngb {

namespace {

template <typename WT>
struct W4;
template <>
struct W4<float> {
  static __device__ __forceinline__ void load(const void* w, uint64_t j, float out[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(w) + j));
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  }
};
template <>
struct W4<__nv_bfloat16> {
  static __device__ __forceinline__ void load(const void* w, uint64_t j, float out[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(w) + j));
    out[0] = __uint_as_float(v.x << 16);
    out[1] = __uint_as_float(v.x & 0xFFFF0000u);
    out[2] = __uint_as_float(v.y << 16);
    out[3] = __uint_as_float(v.y & 0xFFFF0000u);
  }
};
template <>
struct W4<__half> {
  static __device__ __forceinline__ void load(const void* w, uint64_t j, float out[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __half*>(w) + j));
    const __half2 a = *reinterpret_cast<const __half2*>(&v.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&v.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    out[0] = fa.x; out[1] = fa.y; out[2] = fb.x; out[3] = fb.y;
  }
};

}  // namespace

template <typename WT, bool kFixed>
__global__ void __launch_bounds__(kDeliverBlock) k_deliver(SpikeBuf sb, Csr csr, Ring ring, int64_t* clk) {
  const int64_t t = clk[1];
  const int buf = (int)(t & 1);
  const unsigned long long c = sb.ctr[buf];  // written by the update kernels of step t
  const uint32_t nspk = (uint32_t)(c >> kSpkShift);
  const uint32_t nch = (uint32_t)(c & kChunkMask);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = t + 1;        // next step for the update kernels
    sb.ctr[buf ^ 1] = 0;   // the next step's list starts empty
  }
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * (uint32_t)kDeliverBlock + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * (uint32_t)kDeliverBlock) >> 5;
  const uint32_t* __restrict__ sl = buf ? sb.src[1] : sb.src[0];
  const uint32_t* __restrict__ co = buf ? sb.choff[1] : sb.choff[0];
  for (uint32_t ch = warp; ch < nch; ch += nwarps) {
    // the spike owning work item ch: last i with co[i] <= ch
    uint32_t lo = 0, hi = nspk;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (co[mid] <= ch) lo = mid;
      else hi = mid;
    }
    const uint32_t word = sl[lo];
    const uint32_t src = word & kIdMask;
    const uint32_t mult = word >> kIdBits;
    const uint32_t local = ch - co[lo];
    const uint64_t b = __ldg(csr.src_syn + src), e = __ldg(csr.src_syn + src + 1);
    const uint64_t cbase = (b & ~3ull) + (uint64_t)local * kChunk;
    const uint64_t j0 = cbase + (uint64_t)lane * 4;
    uint4 tv = make_uint4(0, 0, 0, 0);
    float wv[4] = {0.f, 0.f, 0.f, 0.f};
    const bool any = j0 < e && j0 + 4 > b;
    if (any) {
      tv = __ldg(reinterpret_cast<const uint4*>(csr.tgt + j0));
      W4<WT>::load(csr.w, j0, wv);
    }
    // group of the work item's first synapse (uniform across the warp)
    const uint64_t jf = cbase > b ? cbase : b;
    uint32_t glo = __ldg(csr.src_grp + src), ghi = __ldg(csr.src_grp + src + 1);
    while (ghi - glo > 1) {
      const uint32_t mid = (glo + ghi) >> 1;
      if (__ldg(csr.grp_start + mid) <= jf) glo = mid;
      else ghi = mid;
    }
    const uint32_t gend = __ldg(csr.src_grp + src + 1);
    uint32_t g = glo;
    if (any) {
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t j = j0 + q;
        const uint32_t twq = q == 0 ? tv.x : q == 1 ? tv.y : q == 2 ? tv.z : tv.w;
        if (j < b || j >= e) continue;
        while (g + 1 < gend && __ldg(csr.grp_start + g + 1) <= j) ++g;
        const uint32_t d = __ldg(csr.grp_delay + g);
        const uint64_t slot = (uint64_t)((t + d) & ring.L_mask);
        const uint32_t r = twq >> 31;
        const uint64_t idx = (slot * (uint64_t)ring.R + r) * (uint64_t)ring.N + (twq & 0x7FFFFFFFu);
        if (kFixed) {
          const long long qv = __float2ll_rn(wv[q] * 4294967296.0f) * (long long)mult;
          atomicAdd(reinterpret_cast<unsigned long long*>(ring.p) + idx, (unsigned long long)qv);
        } else {
          const float v = mult == 1u ? wv[q] : wv[q] * (float)mult;
          atomicAdd(reinterpret_cast<float*>(ring.p) + idx, v);
        }
      }
    }
  }
}

cudaError_t launch_deliver(SpikeBuf sb, Csr csr, int wdtype, Ring ring, bool fixed, int64_t* clk, int grid,
                           cudaStream_t st) {
  if (fixed) {
    if (wdtype == 0) k_deliver<float, true><<<grid, kDeliverBlock, 0, st>>>(sb, csr, ring, clk);
    else if (wdtype == 1) k_deliver<__nv_bfloat16, true><<<grid, kDeliverBlock, 0, st>>>(sb, csr, ring, clk);
    else k_deliver<__half, true><<<grid, kDeliverBlock, 0, st>>>(sb, csr, ring, clk);
  } else {
    if (wdtype == 0) k_deliver<float, false><<<grid, kDeliverBlock, 0, st>>>(sb, csr, ring, clk);
    else if (wdtype == 1) k_deliver<__nv_bfloat16, false><<<grid, kDeliverBlock, 0, st>>>(sb, csr, ring, clk);
    else k_deliver<__half, false><<<grid, kDeliverBlock, 0, st>>>(sb, csr, ring, clk);
  }
  return cudaGetLastError();
}

}  // namespace ngb
