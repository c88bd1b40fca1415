// deliver_noalloc.cu -- spike delivery that allocates no memory.
//
// ngb_deliver_spikes_noalloc() delivers one step's spikes through a
// caller-owned delay-grouped CSR into a caller-owned ring buffer, like the
// delivery stage of ngb_simulate(), but for callers that cannot allocate GPU
// memory: code running under an external memory manager or a capture-only
// allocator, plugins whose host forbids cudaMalloc, or real-time loops that
// must not block on allocation.  Its working memory is a fixed array in this
// library's device image (g_noalloc_scratch below), which every GPU that
// loads the library keeps until the process exits.
//
// The work is split like the main delivery kernel: every spike contributes
// ceil((end - align4(begin)) / 128) work items of 128 synapses; a one-block
// kernel lists the spikes in input order with their work-item offsets in the
// scratch array, and the delivery kernel maps each work item to its spike by
// binary search and scatters the weights into ring slot (t + d) & (L - 1).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>
#include <string>
#include <type_traits>

#include "ngb.h"
#include "ngb_internal.cuh"

namespace ngb {
namespace {

constexpr int kNaBlock = 1024;
constexpr int64_t kNaMaxSpikes = NGB_NOALLOC_MAX_SPIKES;

// Scratch layout: [0, 8) total work items; [256, ...) per-spike work-item
// offsets (u32); then per-spike entries (2 x uint4).
constexpr size_t kNaOffChoff = 256;
constexpr size_t kNaOffEntry = kNaOffChoff + ((size_t)kNaMaxSpikes * 4 + 255) / 256 * 256;
constexpr size_t kNaBytes = kNaOffEntry + (size_t)kNaMaxSpikes * 32;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// One block: spike i gets its work-item offset by a block-wide exclusive scan
// (input order, so the result does not depend on scheduling).
__global__ void __launch_bounds__(kNaBlock) k_na_list(const uint32_t* __restrict__ spikes, int64_t n,
                                                      int64_t N, const uint64_t* __restrict__ src_syn,
                                                      const uint32_t* __restrict__ src_grp, unsigned char* scratch) {
  __shared__ uint32_t warp_tot[kNaBlock / 32];
  __shared__ unsigned long long carry;
  uint32_t* choff = reinterpret_cast<uint32_t*>(scratch + kNaOffChoff);
  uint4* entry = reinterpret_cast<uint4*>(scratch + kNaOffEntry);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += kNaBlock) {
    const int64_t i = base + threadIdx.x;
    uint32_t nch = 0;
    uint4 a = make_uint4(0, 0, 0, 0), b2 = make_uint4(0, 0, 0, 0);
    if (i < n && (int64_t)spikes[i] < N) {  // ids beyond the network are skipped
      const uint32_t s = spikes[i];
      const uint64_t b = src_syn[s], e = src_syn[s + 1];
      const uint32_t g0 = src_grp[s], g1 = src_grp[s + 1];
      if (e > b) nch = (uint32_t)((e - (b & ~3ull) + kChunk - 1) / kChunk);
      a = make_uint4(s | (1u << kIdBits), 0u, (uint32_t)b, (uint32_t)((b >> 32) & 0xFFFFu) | ((g1 - g0) << 16));
      b2 = make_uint4((uint32_t)(e - b), g0, 0u, 0u);
    }
    uint32_t inc = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    const unsigned long long off = carry + before + inc - nch;
    if (i < n) {
      choff[i] = (uint32_t)off;
      entry[2 * i] = make_uint4(a.x, (uint32_t)off, a.z, a.w);
      entry[2 * i + 1] = b2;
    }
    __syncthreads();
    if (threadIdx.x == kNaBlock - 1) carry = off + nch;
    __syncthreads();
  }
  if (threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(scratch) = carry;
}

template <typename WT>
__device__ __forceinline__ float load_w(const void* w, uint64_t j) {
  if (sizeof(WT) == 4) return reinterpret_cast<const float*>(w)[j];
  if (std::is_same<WT, __nv_bfloat16>::value) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w)[j]);
  return __half2float(reinterpret_cast<const __half*>(w)[j]);
}

template <typename WT, bool kFixed>
__global__ void __launch_bounds__(256) k_na_deliver(const unsigned char* scratch, int64_t n, ngb_csr_device csr,
                                                   void* ring, uint32_t L_mask, int32_t R, int64_t t) {
  const uint32_t* __restrict__ choff = reinterpret_cast<const uint32_t*>(scratch + kNaOffChoff);
  const uint4* __restrict__ entry = reinterpret_cast<const uint4*>(scratch + kNaOffEntry);
  const uint64_t nch = *reinterpret_cast<const unsigned long long*>(scratch);
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint64_t K = (uint64_t)csr.num_synapses;
  const uint64_t N = (uint64_t)csr.num_neurons;
  for (uint64_t ch = warp; ch < nch; ch += nwarps) {
    uint32_t lo = 0, hi = (uint32_t)n;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (choff[mid] <= ch) lo = mid;
      else hi = mid;
    }
    const uint4 a = entry[2 * lo], m2 = entry[2 * lo + 1];
    const uint64_t b = (uint64_t)a.z | ((uint64_t)(a.w & 0xFFFFu) << 32);
    const uint64_t e = b + m2.x;
    const uint32_t glo = m2.y, ngrp = a.w >> 16;
    const uint64_t cbase = (b & ~3ull) + (ch - a.y) * (uint64_t)kChunk;
    const uint64_t jf = cbase > b ? cbase : b;
    // group of the work item's first synapse
    uint32_t gl = glo, gh = glo + ngrp;
    while (gh - gl > 1 && gh <= csr.num_groups) {
      const uint32_t mid = (gl + gh) >> 1;
      if (csr.grp_start[mid] <= jf) gl = mid;
      else gh = mid;
    }
    uint32_t g = gl;
    const uint64_t G = (uint64_t)csr.num_groups;
    for (int q = 0; q < 4; ++q) {
      const uint64_t j = cbase + (uint64_t)lane * 4 + q;
      if (j < b || j >= e || j >= K || g >= G) continue;
      while (g + 1 < glo + ngrp && g + 1 < G && csr.grp_start[g + 1] <= j) ++g;
      const uint32_t d = csr.grp_delay[g];
      const uint32_t tw = csr.tgt[j];
      if ((tw & kTgtMask) >= N || (int32_t)(tw >> kRcptShift) >= R) continue;  // outside the ring: skipped
      const float w = load_w<WT>(csr.weight, j);
      const uint64_t slot = (uint64_t)((t + d) & L_mask);
      const uint64_t idx = (slot * (uint64_t)R + (tw >> kRcptShift)) * N + (tw & kTgtMask);
      if (kFixed) {
        const long long qv = __float2ll_rn(w * 4294967296.0f);
        atomicAdd(reinterpret_cast<unsigned long long*>(ring) + idx, (unsigned long long)qv);
      } else {
        atomicAdd(reinterpret_cast<float*>(ring) + idx, w);
      }
    }
  }
}

std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 64;
void* g_na_ptr[kNaMaxDevices] = {nullptr};

}  // namespace

int set_last_error(int code, const std::string& msg);  // ngb_api.cu: message for ngb_last_error()

}  // namespace ngb

using namespace ngb;

static int na_fail(int code, const std::string& m) { return set_last_error(code, m); }

extern "C" int ngb_deliver_spikes_noalloc(const ngb_csr_device* csr, const uint32_t* spikes, int64_t n_spikes,
                                          void* ring, int64_t ring_slots, int32_t receptors,
                                          int32_t fixed_point, int64_t t, void* stream) {
  if (!csr || !ring || (n_spikes > 0 && !spikes))
    return na_fail(NGB_ERR_INVALID_ARG, "ngb_deliver_spikes_noalloc: NULL argument");
  if (n_spikes < 0 || n_spikes > kNaMaxSpikes)
    return na_fail(NGB_ERR_INVALID_ARG, "ngb_deliver_spikes_noalloc: n_spikes must be in [0, " +
                                            std::to_string(kNaMaxSpikes) + "]");
  if (ring_slots < 2 || (ring_slots & (ring_slots - 1)) != 0 || receptors < 1 || receptors > kMaxPorts || t < 0)
    return na_fail(NGB_ERR_INVALID_ARG, "ngb_deliver_spikes_noalloc: ring_slots (power of two), receptors or t");
  if (csr->num_neurons <= 0 || csr->num_synapses < 0 || csr->num_groups < 0 || csr->weight_dtype < 0 ||
      csr->weight_dtype > 2 || !csr->src_syn || !csr->src_grp || !csr->grp_start || !csr->grp_delay ||
      (csr->num_synapses > 0 && (!csr->tgt || !csr->weight)))
    return na_fail(NGB_ERR_INVALID_ARG, "ngb_deliver_spikes_noalloc: CSR description");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(NGB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kNaMaxDevices) return na_fail(NGB_ERR_INVALID_ARG, "device ordinal beyond 63");
  void* ptr = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      e = cudaGetSymbolAddress(&g_na_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_na_ptr[dev] = nullptr;
        return na_fail(NGB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    ptr = g_na_ptr[dev];
  }
  if (n_spikes == 0) return NGB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* scratch = reinterpret_cast<unsigned char*>(ptr);
  k_na_list<<<1, kNaBlock, 0, st>>>(spikes, n_spikes, csr->num_neurons, csr->src_syn, csr->src_grp, scratch);
  const uint32_t mask = (uint32_t)(ring_slots - 1);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return na_fail(NGB_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
  const int grid = (sms > 0 ? sms : 1) * 4;
  const ngb_csr_device c = *csr;
  if (fixed_point) {
    if (c.weight_dtype == 0) k_na_deliver<float, true><<<grid, 256, 0, st>>>(scratch, n_spikes, c, ring, mask, receptors, t);
    else if (c.weight_dtype == 1) k_na_deliver<__nv_bfloat16, true><<<grid, 256, 0, st>>>(scratch, n_spikes, c, ring, mask, receptors, t);
    else k_na_deliver<__half, true><<<grid, 256, 0, st>>>(scratch, n_spikes, c, ring, mask, receptors, t);
  } else {
    if (c.weight_dtype == 0) k_na_deliver<float, false><<<grid, 256, 0, st>>>(scratch, n_spikes, c, ring, mask, receptors, t);
    else if (c.weight_dtype == 1) k_na_deliver<__nv_bfloat16, false><<<grid, 256, 0, st>>>(scratch, n_spikes, c, ring, mask, receptors, t);
    else k_na_deliver<__half, false><<<grid, 256, 0, st>>>(scratch, n_spikes, c, ring, mask, receptors, t);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(NGB_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return NGB_OK;
}
