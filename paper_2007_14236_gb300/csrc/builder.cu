// builder.cu -- connection builder on the device.
//
// Sec. 2.1 (connection rules fixed indegree, fixed total number, fixed
// outdegree, one-to-one and all-to-all, weights
// and delays from distributions) and Sec. 2.2 (per-source connection groups
// ordered by delay).  The paper builds connections in host RAM and copies
// them before the simulation (Sec. 3.1) and names building on the GPU as the
// way to cut the building time (Discussion); this file does that.
//
// For each source population, in population order:
//   1. k_draw: one thread per draw index q of every connect call with that
//      source population draws (source, target) from Philox (purpose
//      kPurSrc, re-drawn for excluded autapses), the weight (kPurWeight;
//      Normal by Box-Muller re-drawn until its sign equals the mean's) and the
//      delay (kPurDelay; Normal re-drawn until >= dt, or Uniform), rounds the
//      delay to steps (ties to even, at least 1) and the weight to the
//      storage precision, and writes the key (source << 12 | delay), the
//      target word and the weight in draw order;
//   2. a stable radix sort of (key, draw position) -- CUB's device radix
//      sort, a library primitive -- yields the canonical order
//      (source, delay, connect call, draw index);
//   3. k_gather writes the target words and weights into the CSR slice of
//      the population and flags the first synapse of every (source, delay)
//      group; an exclusive scan numbers the groups and k_groups records
//      their starts and delays.
// Finally per-source synapse and group counts are scanned into src_syn and
// src_grp.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "builder.h"
#include "ngb_internal.cuh"
#include "philox.cuh"

namespace ngb {

namespace {

constexpr uint32_t kMaxAttempts = 10000;  // cap of every re-draw loop

__device__ __forceinline__ double draw_weight(const CallDev& c, uint64_t q) {
  if (c.wdist == 0) return c.w0;
  for (uint32_t attempt = 0;; ++attempt) {
    if (attempt == kMaxAttempts) return c.w0;  // re-draws exhausted: the mean
    const U4 r = draw4(c.seed, q, kPurWeight, attempt, c.stream);
    if (c.wdist == 1) {
      const double v = __dadd_rn(c.w0, __dmul_rn(c.w1, gauss(r)));
      if (c.w0 > 0.0 && !(v > 0.0)) continue;
      if (c.w0 < 0.0 && !(v < 0.0)) continue;
      return v;
    }
    return __dadd_rn(c.w0, __dmul_rn(__dsub_rn(c.w1, c.w0), unit53(r.x, r.y)));
  }
}

__device__ __forceinline__ double draw_delay(const CallDev& c, uint64_t q) {
  if (c.ddist == 0) return c.d0;
  for (uint32_t attempt = 0;; ++attempt) {
    if (attempt == kMaxAttempts) return fmax(c.d0, c.dt);  // re-draws exhausted
    const U4 r = draw4(c.seed, q, kPurDelay, attempt, c.stream);
    if (c.ddist == 1) {
      const double v = __dadd_rn(c.d0, __dmul_rn(c.d1, gauss(r)));
      if (v < c.dt) continue;
      return v;
    }
    return __dadd_rn(c.d0, __dmul_rn(__dsub_rn(c.d1, c.d0), unit53(r.x, r.y)));
  }
}

__device__ __forceinline__ float round_storage(float w, int prec) {
  if (prec == 1) return __bfloat162float(__float2bfloat16_rn(w));
  if (prec == 2) return __half2float(__float2half_rn(w));
  return w;
}

__global__ void k_draw(CallDev c, uint64_t base, unsigned long long* __restrict__ keys,
                       uint32_t* __restrict__ vals, uint32_t* __restrict__ st_tgt, float* __restrict__ st_w,
                       unsigned long long* __restrict__ src_cnt, int* __restrict__ max_delay) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  int dmax = 0;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < c.nsyn; q += stride) {
    uint32_t src = 0, tgt = 0;
    if (c.rule == 3) {  // one-to-one
      src = tgt = (uint32_t)q;
    } else if (c.rule == 4) {  // all-to-all, target-major; (i, i) skipped without autapses
      if (c.no_autapse) {
        tgt = (uint32_t)(q / (uint64_t)(c.n_src - 1));
        const uint32_t r = (uint32_t)(q % (uint64_t)(c.n_src - 1));
        src = r < tgt ? r : r + 1;
      } else {
        tgt = (uint32_t)(q / (uint64_t)c.n_src);
        src = (uint32_t)(q % (uint64_t)c.n_src);
      }
    } else {
      for (uint32_t attempt = 0;; ++attempt) {
        const U4 r = draw4(c.seed, q, kPurSrc, attempt, c.stream);
        if (attempt == kMaxAttempts) break;  // keep the last draw (needs a population of one)
        if (c.rule == 0) {  // fixed indegree
          tgt = (uint32_t)(q / (uint64_t)c.K);
          src = scale_index(r.x, c.n_src);
        } else if (c.rule == 2) {  // fixed outdegree
          src = (uint32_t)(q / (uint64_t)c.K);
          tgt = scale_index(r.x, c.n_tgt);
        } else {  // fixed total number
          src = scale_index(r.x, c.n_src);
          tgt = scale_index(r.y, c.n_tgt);
        }
        if (c.no_autapse && src == tgt) continue;
        break;
      }
    }
    const float w = round_storage(__double2float_rn(draw_weight(c, q)), c.prec);
    double ds = rint(__ddiv_rn(draw_delay(c, q), c.dt));
    if (ds < 1.0) ds = 1.0;
    if (ds > (double)kMaxDelay) ds = (double)kMaxDelay;
    const uint32_t d = (uint32_t)ds;
    const uint64_t pos = base + q;
    keys[pos] = ((unsigned long long)src << kDelayBits) | d;
    vals[pos] = (uint32_t)pos;
    st_tgt[pos] = (c.tgt_off + tgt) | ((uint32_t)c.receptor << kRcptShift) | ((uint32_t)c.stdp << kPlastShift);
    st_w[pos] = w;
    atomicAdd(src_cnt + c.src_off + src, 1ull);
    dmax = d > (uint32_t)dmax ? (int)d : dmax;
  }
  if (dmax > 0) atomicMax(max_delay, dmax);
}

template <typename WT>
__device__ __forceinline__ WT to_storage(float w);
template <>
__device__ __forceinline__ float to_storage<float>(float w) { return w; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(float w) { return __float2bfloat16_rn(w); }
template <>
__device__ __forceinline__ __half to_storage<__half>(float w) { return __float2half_rn(w); }

template <typename WT>
__global__ void k_gather(uint64_t n, const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ vals,
                         const uint32_t* __restrict__ st_tgt, const float* __restrict__ st_w,
                         uint32_t* __restrict__ tgt, WT* __restrict__ w, uint32_t* __restrict__ flag,
                         unsigned long long* __restrict__ src_ngrp, uint32_t src_off) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t v = vals[i];
    tgt[i] = st_tgt[v];
    w[i] = to_storage<WT>(st_w[v]);
    const unsigned long long k = keys[i];
    const bool first = (i == 0) || (keys[i - 1] != k);
    flag[i] = first ? 1u : 0u;
    if (first) atomicAdd(src_ngrp + src_off + (uint32_t)(k >> kDelayBits), 1ull);
  }
}

__global__ void k_groups(uint64_t n, uint64_t csr_off, const unsigned long long* __restrict__ keys,
                         const uint32_t* __restrict__ flag, const uint32_t* __restrict__ gidx,
                         uint64_t* __restrict__ gstart, uint16_t* __restrict__ gdelay) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (flag[i]) {
      const uint32_t g = gidx[i];
      gstart[g] = csr_off + i;
      gdelay[g] = (uint16_t)(keys[i] & (unsigned long long)kMaxDelay);
    }
  }
}

__global__ void k_to_u32(uint64_t n, const unsigned long long* __restrict__ in, uint32_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (uint32_t)in[i];
}

int grid_for(uint64_t n) {
  const uint64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b == 0 ? 1 : b) : 152 * 32);
}

}  // namespace

#define BTRY(x)                                     \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) {                        \
      err = std::string(#x) + ": " + cudaGetErrorString(e_); \
      return e_;                                    \
    }                                               \
  } while (0)

cudaError_t sort_scratch_bytes(uint64_t n, int key_bits, size_t* sort_bytes, size_t* scan_bytes) {
  *sort_bytes = 0;
  *scan_bytes = 0;
  cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, *sort_bytes, (const unsigned long long*)nullptr,
                                                  (unsigned long long*)nullptr, (const uint32_t*)nullptr,
                                                  (uint32_t*)nullptr, (int64_t)n, 0, key_bits);
  if (e != cudaSuccess) return e;
  return cub::DeviceScan::ExclusiveSum(nullptr, *scan_bytes, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                       (int64_t)n);
}

cudaError_t build_source_population(const std::vector<CallDev>& calls, uint64_t n_total, int src_bits,
                                    uint64_t csr_off, int wdtype, BuildScratch& s, uint32_t* tgt_out, void* w_out,
                                    unsigned long long* src_cnt, unsigned long long* src_ngrp, int* max_delay,
                                    uint64_t** gstart_out, uint16_t** gdelay_out, uint64_t* ngroups_out,
                                    cudaStream_t st, std::string& err) {
  *gstart_out = nullptr;
  *gdelay_out = nullptr;
  *ngroups_out = 0;
  if (n_total == 0) return cudaSuccess;
  uint64_t base = 0;
  for (const CallDev& c : calls) {
    if (c.nsyn) {
      k_draw<<<grid_for(c.nsyn), 256, 0, st>>>(c, base, s.keys, s.vals, s.st_tgt, s.st_w, src_cnt, max_delay);
      BTRY(cudaGetLastError());
    }
    base += c.nsyn;
  }
  const int key_bits = src_bits + kDelayBits;
  size_t sb = s.sort_bytes;
  BTRY(cub::DeviceRadixSort::SortPairs(s.sort_tmp, sb, s.keys, s.keys_alt, s.vals, s.vals_alt, (int64_t)n_total, 0,
                                       key_bits, st));
  const uint32_t src_off = calls.front().src_off;
  const int g = grid_for(n_total);
  if (wdtype == 0)
    k_gather<float><<<g, 256, 0, st>>>(n_total, s.keys_alt, s.vals_alt, s.st_tgt, s.st_w, tgt_out,
                                       reinterpret_cast<float*>(w_out), s.flag, src_ngrp, src_off);
  else if (wdtype == 1)
    k_gather<__nv_bfloat16><<<g, 256, 0, st>>>(n_total, s.keys_alt, s.vals_alt, s.st_tgt, s.st_w, tgt_out,
                                               reinterpret_cast<__nv_bfloat16*>(w_out), s.flag, src_ngrp, src_off);
  else
    k_gather<__half><<<g, 256, 0, st>>>(n_total, s.keys_alt, s.vals_alt, s.st_tgt, s.st_w, tgt_out,
                                        reinterpret_cast<__half*>(w_out), s.flag, src_ngrp, src_off);
  BTRY(cudaGetLastError());
  size_t scb = s.scan_bytes;
  BTRY(cub::DeviceScan::ExclusiveSum(s.scan_tmp, scb, s.flag, s.gidx, (int64_t)n_total, st));
  uint32_t last[2] = {0, 0};
  BTRY(cudaMemcpyAsync(&last[0], s.gidx + (n_total - 1), 4, cudaMemcpyDeviceToHost, st));
  BTRY(cudaMemcpyAsync(&last[1], s.flag + (n_total - 1), 4, cudaMemcpyDeviceToHost, st));
  BTRY(cudaStreamSynchronize(st));
  const uint64_t G = (uint64_t)last[0] + last[1];
  uint64_t* gs = nullptr;
  uint16_t* gd = nullptr;
  BTRY(cudaMalloc(&gs, G * sizeof(uint64_t)));
  cudaError_t e2 = cudaMalloc(&gd, G * sizeof(uint16_t));
  if (e2 != cudaSuccess) {
    cudaFree(gs);
    err = "cudaMalloc(group delays)";
    return e2;
  }
  k_groups<<<g, 256, 0, st>>>(n_total, csr_off, s.keys_alt, s.flag, s.gidx, gs, gd);
  e2 = cudaGetLastError();
  if (e2 != cudaSuccess) {
    cudaFree(gs);
    cudaFree(gd);
    err = "k_groups";
    return e2;
  }
  *gstart_out = gs;
  *gdelay_out = gd;
  *ngroups_out = G;
  return cudaSuccess;
}

cudaError_t exclusive_scan_u64(const unsigned long long* in, unsigned long long* out, uint64_t n, void* tmp,
                               size_t tmp_bytes, cudaStream_t st) {
  size_t b = tmp_bytes;
  return cub::DeviceScan::ExclusiveSum(tmp, b, in, out, (int64_t)n, st);
}

namespace {
// Spike-record key: step << 26 | neuron (neurons < 2^26, steps < 2^38).
__global__ void k_record_keys(const uint32_t* __restrict__ ids, const int64_t* __restrict__ steps, uint64_t n,
                              unsigned long long* keys) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    keys[i] = ((unsigned long long)steps[i] << 26) | ids[i];
}
}  // namespace

cudaError_t record_sort_scratch_bytes(uint64_t n, size_t* bytes) {
  *bytes = 0;
  return cub::DeviceRadixSort::SortKeys(nullptr, *bytes, (const unsigned long long*)nullptr,
                                        (unsigned long long*)nullptr, (int64_t)n);
}

cudaError_t sort_record(const uint32_t* ids, const int64_t* steps, uint64_t n, unsigned long long* keys,
                        unsigned long long* sorted, void* tmp, size_t tmp_bytes, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, 4096);
  k_record_keys<<<grid, 256, 0, st>>>(ids, steps, n, keys);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  size_t b = tmp_bytes;
  return cub::DeviceRadixSort::SortKeys(tmp, b, keys, sorted, (int64_t)n, 0, 64, st);
}

cudaError_t scan_scratch_bytes_u64(uint64_t n, size_t* bytes) {
  *bytes = 0;
  return cub::DeviceScan::ExclusiveSum(nullptr, *bytes, (const unsigned long long*)nullptr,
                                       (unsigned long long*)nullptr, (int64_t)n);
}

// Synapses [first, first + n) decoded for introspection: target, receptor,
// weight widened to FP32 and the delay of the group containing each synapse
// (binary search over the group starts).
__global__ void k_expand(uint64_t first, uint64_t n, const uint32_t* __restrict__ tgt, const void* __restrict__ w,
                         int wdtype, const uint64_t* __restrict__ gstart, uint64_t G,
                         const uint16_t* __restrict__ gdelay, uint32_t* __restrict__ o_tgt,
                         uint8_t* __restrict__ o_rc, float* __restrict__ o_w, uint16_t* __restrict__ o_d) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t j = first + i;
    const uint32_t tw = tgt[j];
    o_tgt[i] = tw & kTgtMask;
    o_rc[i] = (uint8_t)(tw >> kRcptShift);
    float v;
    if (wdtype == 0) v = reinterpret_cast<const float*>(w)[j];
    else if (wdtype == 1) v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w)[j]);
    else v = __half2float(reinterpret_cast<const __half*>(w)[j]);
    o_w[i] = v;
    uint64_t lo = 0, hi = G;  // last g with gstart[g] <= j
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (gstart[mid] <= j) lo = mid;
      else hi = mid;
    }
    o_d[i] = gdelay[lo];
  }
}

cudaError_t expand_synapses(uint64_t first, uint64_t n, const uint32_t* tgt, const void* w, int wdtype,
                            const uint64_t* gstart, uint64_t G, const uint16_t* gdelay, uint32_t* o_tgt,
                            uint8_t* o_rc, float* o_w, uint16_t* o_d, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_expand<<<grid_for(n), 256, 0, st>>>(first, n, tgt, w, wdtype, gstart, G, gdelay, o_tgt, o_rc, o_w, o_d);
  return cudaGetLastError();
}

// Per-source metadata of one population placed at neurons [off, off + n):
// cnt_scan / grp_scan are the exclusive scans (n + 1 entries) of the
// population's per-source synapse and group counts; k_off / g_off are the
// population's ranges in the synapse and group pools.
// Per-source tables of one placed population.  The population's group
// starts and delays are already in the pool (grp_start, grp_delay).
__global__ void k_fill_meta(uint64_t n, uint64_t off, uint64_t k_off, uint64_t g_off,
                            const unsigned long long* __restrict__ cnt_scan,
                            const unsigned long long* __restrict__ grp_scan, const uint64_t* __restrict__ grp_start,
                            const uint16_t* __restrict__ grp_delay, uint4* __restrict__ meta,
                            uint64_t* __restrict__ src_syn, uint32_t* __restrict__ src_grp,
                            uint2* __restrict__ src_age, unsigned long long* __restrict__ items) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t b = k_off + cnt_scan[i];
  const uint64_t nsyn = cnt_scan[i + 1] - cnt_scan[i];
  const uint64_t g0 = g_off + grp_scan[i];
  const uint64_t ng = grp_scan[i + 1] - grp_scan[i];
  meta[off + i] = make_uint4((uint32_t)b, (uint32_t)((b >> 32) & 0xFFFFu) | ((uint32_t)ng << 16), (uint32_t)nsyn,
                             (uint32_t)g0);
  src_syn[off + i] = b;
  src_grp[off + i] = (uint32_t)g0;
  // first connection group: synapses, delay, and the delay of the second group
  uint2 ag = make_uint2(0, 0);
  if (ng > 0) {
    const uint64_t size0 = ng > 1 ? grp_start[g0 + 1] - grp_start[g0] : nsyn;
    const uint32_t d0 = grp_delay[g0], d1 = ng > 1 ? grp_delay[g0 + 1] : 0u;
    ag = make_uint2((uint32_t)size0, d0 | (d1 << 16));
  }
  src_age[off + i] = ag;
  if (nsyn) atomicAdd(items, (unsigned long long)((b + nsyn - (b & ~3ull) + kChunk - 1) / kChunk));
}

cudaError_t fill_meta(uint64_t n, uint64_t off, uint64_t k_off, uint64_t g_off, const unsigned long long* cnt_scan,
                      const unsigned long long* grp_scan, const uint64_t* grp_start, const uint16_t* grp_delay,
                      uint4* meta, uint64_t* src_syn, uint32_t* src_grp, uint2* src_age, unsigned long long* items,
                      cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_fill_meta<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, off, k_off, g_off, cnt_scan, grp_scan, grp_start,
                                                           grp_delay, meta, src_syn, src_grp, src_age, items);
  return cudaGetLastError();
}

cudaError_t narrow_u64_to_u32(const unsigned long long* in, uint32_t* out, uint64_t n, cudaStream_t st) {
  k_to_u32<<<grid_for(n), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

}  // namespace ngb
