// deliver_item.cuh -- delivery of one work item (128 consecutive synapses of
// one spiking source) into the ring buffer; shared by the per-step delivery
// kernel and the persistent step kernel.
//
// The warp reads 4 target words (one 16-byte load) and 4 weights (16 or 8
// bytes) per lane, holds the source's delay groups (up to 64) in registers,
// two per lane, finds each synapse's group with ballots over the group starts
// (a table search for sources with more groups), and issues one
// red.global.add per synapse at ring slot (t + d) & (L - 1): FP32, or int64
// fixed point (units of 2^-32) in deterministic mode.  Every lane of the warp
// must call it with the same work item.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ngb_internal.cuh"
#include "stdp_rule.cuh"

namespace ngb {

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

constexpr uint32_t kWindow = 64;  // delay groups a warp holds in registers

// a, m2: the work item's two entries ({source | multiplicity << 26, index of
// the item within the source, row start lo, row start hi | groups << 16},
// {synapses, first group, -, -}).
template <typename WT, bool kFixed>
__device__ __forceinline__ void deliver_work_item(const uint4 a, const uint4 m2, const int64_t t, const Csr& csr,
                                                  const Ring& ring, const int lane) {
  const unsigned full = 0xffffffffu;
  const uint32_t mult = a.x >> kIdBits;
  const uint32_t local = a.y;
  const uint64_t b = (uint64_t)a.z | ((uint64_t)(a.w & 0xFFFFu) << 32);
  const uint64_t e = b + m2.x;
  const uint32_t ngrp = a.w >> 16;
  const uint32_t glo = m2.y;
  const uint64_t cbase = (b & ~3ull) + (uint64_t)local * kChunk;
  const uint64_t j0 = cbase + (uint64_t)lane * 4;
  const bool any = j0 < e && j0 + 4 > b;
  uint4 tv = make_uint4(0, 0, 0, 0);
  float wv[4] = {0.f, 0.f, 0.f, 0.f};
  if (any) {
    tv = __ldg(reinterpret_cast<const uint4*>(csr.tgt + j0));
    W4<WT>::load(csr.w, j0, wv);
  }
  uint32_t g[4];
  uint32_t dA = 0, dB = 0;
  if (ngrp <= kWindow) {
    // the source's delay groups, two per lane: starts and delays in registers
    uint64_t sA = ~0ull, sB = ~0ull;
    if ((uint32_t)lane < ngrp) {
      sA = __ldg(csr.grp_start + glo + lane);
      dA = __ldg(csr.grp_delay + glo + lane);
    }
    if ((uint32_t)lane + 32 < ngrp) {
      sB = __ldg(csr.grp_start + glo + 32 + lane);
      dB = __ldg(csr.grp_delay + glo + 32 + lane);
    }
    const uint64_t jf = cbase > b ? cbase : b;             // first synapse of the work item
    const uint64_t jl = cbase + kChunk < e ? cbase + kChunk : e;
    // group of jf = (starts <= jf) - 1; the starts are sorted
    const uint32_t gf = __popc(__ballot_sync(full, sA <= jf)) + __popc(__ballot_sync(full, sB <= jf)) - 1;
    g[0] = g[1] = g[2] = g[3] = gf;
    // group boundaries strictly inside the work item
    for (unsigned mA = __ballot_sync(full, sA > jf && sA < jl); mA; mA &= mA - 1) {
      const uint64_t bk = __shfl_sync(full, sA, __ffs(mA) - 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) g[q] += (j0 + q >= bk) ? 1u : 0u;
    }
    for (unsigned mB = __ballot_sync(full, sB > jf && sB < jl); mB; mB &= mB - 1) {
      const uint64_t bk = __shfl_sync(full, sB, __ffs(mB) - 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) g[q] += (j0 + q >= bk) ? 1u : 0u;
    }
  } else {
    // many delay groups: search the group table in memory
    const uint64_t jf = cbase > b ? cbase : b;
    uint32_t l = glo, h = glo + ngrp;
    while (h - l > 1) {
      const uint32_t mid = (l + h) >> 1;
      if (__ldg(csr.grp_start + mid) <= jf) l = mid;
      else h = mid;
    }
    uint32_t gg = l;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t j = j0 + q;
      if (any && j >= jf && j < e)
        while (gg + 1 < glo + ngrp && __ldg(csr.grp_start + gg + 1) <= j) ++gg;
      g[q] = gg - glo;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t d;
    if (ngrp <= kWindow) {
      const uint32_t xa = __shfl_sync(full, dA, g[q] & 31u);
      const uint32_t xb = __shfl_sync(full, dB, g[q] & 31u);
      d = g[q] < 32u ? xa : xb;
    } else {
      d = __ldg(csr.grp_delay + glo + g[q]);
    }
    const uint64_t j = j0 + q;
    if (!any || j < b || j >= e) continue;
    const uint32_t twq = q == 0 ? tv.x : q == 1 ? tv.y : q == 2 ? tv.z : tv.w;
    const uint64_t slot = (uint64_t)((t + d) & ring.L_mask);
    const uint32_t r = twq >> kRcptShift;
    const uint64_t idx = (slot * (uint64_t)ring.R + r) * (uint64_t)ring.N + (twq & kTgtMask);
    if (kFixed) {
      const long long qv = __float2ll_rn(wv[q] * 4294967296.0f) * (long long)mult;
      atomicAdd(reinterpret_cast<unsigned long long*>(ring.p) + idx, (unsigned long long)qv);
    } else {
      const float v = mult == 1u ? wv[q] : wv[q] * (float)mult;
      atomicAdd(reinterpret_cast<float*>(ring.p) + idx, v);
    }
  }
}

// deliver_work_item with the weight storage chosen at run time (a warp-uniform branch).
template <bool kFixed>
__device__ __forceinline__ void deliver_work_item_rt(int wdtype, const uint4 a, const uint4 m2, const int64_t t,
                                                     const Csr& csr, const Ring& ring, const int lane) {
  if (wdtype == 1) deliver_work_item<__nv_bfloat16, kFixed>(a, m2, t, csr, ring, lane);
  else if (wdtype == 2) deliver_work_item<__half, kFixed>(a, m2, t, csr, ring, lane);
  else deliver_work_item<float, kFixed>(a, m2, t, csr, ring, lane);
}

// New spikes of step t in the pipelined ring scheme.  A source's first
// connection group, when its delay is one step, is delivered by this warp at
// once (into slot t + 1, which the next step's update reads); the source's
// other groups become work items of the list of step t mod 3, delivered by a
// kernel that may run beside the next step's update because their slots are
// t + 2 and later.  Spike record and event count as in the other schemes.
// Every lane of the warp must call it.
template <bool kFixed>
__device__ __forceinline__ void emit_spikes_pipe(bool spk, uint32_t gid, uint32_t mult, int64_t t, uint4 meta,
                                                 uint2 ag, const Csr& csr, const Ring& ring, const SpikeBuf& sb) {
  const unsigned full = 0xffffffffu;
  const unsigned ball = __ballot_sync(full, spk);
  if (ball == 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t ngrp = meta.y >> 16;
  const bool local = spk && ngrp > 0 && (ag.y & 0xFFFFu) == 1u;
  const uint32_t word = gid | (mult << kIdBits);
  // the delay-1 groups first (one spiking lane at a time, by the whole warp):
  // their loads are in flight while the bookkeeping below waits on atomics
  for (unsigned lm = __ballot_sync(full, local); lm; lm &= lm - 1) {
    const int l = __ffs(lm) - 1;
    const uint32_t wl = __shfl_sync(full, word, l);
    const uint32_t bx = __shfl_sync(full, meta.x, l);
    const uint32_t by = __shfl_sync(full, meta.y & 0xFFFFu, l);
    const uint32_t n0 = __shfl_sync(full, ag.x, l);
    const uint32_t g0 = __shfl_sync(full, meta.w, l);
    const uint64_t bb = (uint64_t)bx | ((uint64_t)by << 32);
    const uint32_t nc = (uint32_t)((bb + n0 - (bb & ~3ull) + kChunk - 1) / kChunk);
    for (uint32_t c = 0; c < nc; ++c)
      deliver_work_item_rt<kFixed>(csr.wdtype, make_uint4(wl, c, bx, by | (1u << 16)), make_uint4(n0, g0, 0u, 0u), t,
                                   csr, ring, lane);
  }
  const uint64_t b = (uint64_t)meta.x | ((uint64_t)(meta.y & 0xFFFFu) << 32);
  uint4 rest = meta;
  if (local) {
    const uint64_t b2 = b + ag.x;
    rest = make_uint4((uint32_t)b2, (uint32_t)((b2 >> 32) & 0xFFFFu) | ((ngrp - 1u) << 16), meta.z - ag.x,
                      meta.w + 1u);
  }
  // work items of the remaining groups and the spike record: both positions
  // reserved in one round of atomics
  uint32_t nch = 0, m = 0;
  unsigned long long nev = 0;
  if (spk) {
    if (rest.z > 0) {
      const uint64_t rb = (uint64_t)rest.x | ((uint64_t)(rest.y & 0xFFFFu) << 32);
      nch = (uint32_t)((rb + rest.z - (rb & ~3ull) + kChunk - 1) / kChunk);
    }
    m = mult;
    nev = (unsigned long long)meta.z * mult;
  }
  uint32_t inc = nch, inc_m = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(full, inc, o);
    const uint32_t y = __shfl_up_sync(full, inc_m, o);
    if (lane >= o) {
      inc += x;
      inc_m += y;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nev += __shfl_xor_sync(full, nev, o);
  const uint32_t tot = __shfl_sync(full, inc, 31);
  const uint32_t tot_m = __shfl_sync(full, inc_m, 31);
  const int q = (int)(t % 3);
  unsigned long long base = 0, rbase = 0;
  if (lane == 0) {
    if (tot) base = atomicAdd(sb.ctr3 + q, (unsigned long long)tot);
    rbase = atomicAdd(sb.rec_count, (unsigned long long)tot_m);
    atomicAdd(sb.events, nev);
  }
  base = __shfl_sync(full, base, 0);
  rbase = __shfl_sync(full, rbase, 0);
  if (nch) {
    uint4* const wi = sb.wi3[q];
    const unsigned long long first = base + inc - nch;
    for (uint32_t c = 0; c < nch; ++c) {
      wi[2 * (first + c)] = make_uint4(word, c, rest.x, rest.y);
      wi[2 * (first + c) + 1] = make_uint4(rest.z, rest.w, 0u, 0u);
    }
  }
  if (spk && sb.rec_cap > 0) {
    const unsigned long long r0 = rbase + inc_m - m;
    for (uint32_t k = 0; k < m; ++k) {
      if (r0 + k < (unsigned long long)sb.rec_cap) {
        sb.rec_id[r0 + k] = gid;
        sb.rec_step[r0 + k] = t;
      } else {
        atomicOr(sb.err, kErrRecordOverflow);
      }
    }
  }
}

// The spikes of one thread block, delivered by that block (fused step loop).
template <int kBlock>
struct BlockSpikes {
  uint4 meta[kBlock];         // source metadata of each spike
  uint32_t word[kBlock];      // neuron | multiplicity << 26
  uint32_t pre[kBlock + 1];   // first work item of each spike (prefix sum)
  int n;
};

// Compact the block's spikes into S and scatter them into the ring (slots
// t + d, ring scheme): the block's warps share the spikes' 128-synapse work
// items.  S.n must be 0 and visible to the block before the call; every
// thread of the block must call it.  Deliveries of step t land in slots
// t + 1 ... t + L - 1, never in slot t that other blocks are still reading.
template <typename WT, bool kFixed, int kBlock>
__device__ __forceinline__ void deliver_block_spikes(bool spk, uint32_t gid, uint32_t mult, uint4 meta, int64_t t,
                                                     const Csr& csr, const Ring& ring, BlockSpikes<kBlock>& S) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned ball = __ballot_sync(full, spk);
  if (ball) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&S.n, __popc(ball));
    base = __shfl_sync(full, base, 0);
    if (spk) {
      const int pos = base + __popc(ball & ((1u << lane) - 1u));
      S.meta[pos] = meta;
      S.word[pos] = gid | (mult << kIdBits);
    }
  }
  __syncthreads();
  const int n = S.n;
  if (n == 0) return;
  if (warp == 0) {
    uint32_t carry = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      uint32_t nch = 0;
      if (i < n) {
        const uint4 m = S.meta[i];
        const uint64_t b = (uint64_t)m.x | ((uint64_t)(m.y & 0xFFFFu) << 32);
        if (m.z) nch = (uint32_t)((b + m.z - (b & ~3ull) + kChunk - 1) / kChunk);
      }
      uint32_t inc = nch;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(full, inc, o);
        if (lane >= o) inc += a;
      }
      if (i < n) S.pre[i + 1] = carry + inc;
      carry += __shfl_sync(full, inc, 31);
    }
    if (lane == 0) S.pre[0] = 0;
  }
  __syncthreads();
  const uint32_t total = S.pre[n];
  for (uint32_t c = warp; c < total; c += kBlock / 32) {
    int lo = 0, hi = n;  // spike owning item c: the last with pre <= c
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (S.pre[mid] <= c) lo = mid;
      else hi = mid;
    }
    const uint4 m = S.meta[lo];
    deliver_work_item<WT, kFixed>(make_uint4(S.word[lo], c - S.pre[lo], m.x, m.y), make_uint4(m.z, m.w, 0u, 0u), t,
                                  csr, ring, lane);
  }
}

// Delivery of one due item (spike-buffer scheme): its synapses go to the
// single ring slot (the input of the next step).  it = {first synapse lo, hi
// | multiplicity << 16, synapses, -}.  The warp walks the item in aligned
// chunks of 128 synapses, two chunks per pass so that both chunks' loads are
// in flight together.  kPlastic (FP32 weights): a plastic synapse is
// depressed by its target's latest spike, records arrival step t + 1 and
// delivers the depressed weight (nearest-neighbour STDP, Sec. 2.1; each
// synapse belongs to one due item per step, so no other thread touches it).
template <typename WT, bool kFixed, bool kPlastic = false>
__device__ __forceinline__ void deliver_due_item(const uint4 it, const Csr& csr, const Ring& ring, const int lane,
                                                 int64_t t = 0, const SpikeBuf* sb = nullptr,
                                                 const StdpArgs* sa = nullptr) {
  const uint64_t b = (uint64_t)it.x | ((uint64_t)(it.y & 0xFFFFu) << 32);
  const uint32_t mult = it.y >> 16;
  const uint64_t e = b + it.z;
  for (uint64_t c = b & ~3ull; c < e; c += 2 * kChunk) {
    uint4 tv[2];
    float wv[2][4];
    uint4 pw[2][2];  // plastic synapses: the four weight-and-arrival words of the lane's synapses
    bool any[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t j0 = c + (uint64_t)u * kChunk + (uint64_t)lane * 4;
      any[u] = j0 < e && j0 + 4 > b;
      tv[u] = make_uint4(0, 0, 0, 0);
      wv[u][0] = wv[u][1] = wv[u][2] = wv[u][3] = 0.f;
      pw[u][0] = pw[u][1] = make_uint4(0, 0, 0, 0);
      if (any[u]) {
        tv[u] = __ldg(reinterpret_cast<const uint4*>(csr.tgt + j0));
        if (kPlastic) {
          // the weight-and-arrival words only where a synapse of the four is plastic, the CSR
          // weights only where one is static (a plastic synapse's weight lives in its word)
          const uint32_t pl = (tv[u].x | tv[u].y | tv[u].z | tv[u].w) >> kPlastShift & kPlastMask;
          const bool all_pl = ((tv[u].x >> kPlastShift) & kPlastMask) && ((tv[u].y >> kPlastShift) & kPlastMask) &&
                              ((tv[u].z >> kPlastShift) & kPlastMask) && ((tv[u].w >> kPlastShift) & kPlastMask);
          if (!all_pl) W4<WT>::load(csr.w, j0, wv[u]);
          if (pl) {
            pw[u][0] = *reinterpret_cast<const uint4*>(sa->wa + j0);
            pw[u][1] = *reinterpret_cast<const uint4*>(sa->wa + j0 + 2);
          }
        } else {
          W4<WT>::load(csr.w, j0, wv[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!any[u]) continue;
      const uint64_t j0 = c + (uint64_t)u * kChunk + (uint64_t)lane * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t j = j0 + q;
        if (j < b || j >= e) continue;
        const uint32_t twq = q == 0 ? tv[u].x : q == 1 ? tv[u].y : q == 2 ? tv[u].z : tv[u].w;
        float wq = wv[u][q];
        if (kPlastic) {
          const uint32_t cls = (twq >> kPlastShift) & kPlastMask;
          if (cls) {
            const uint4 pp = pw[u][q >> 1];
            wq = __uint_as_float((q & 1) ? pp.z : pp.x);  // the current plastic weight
            const int32_t arrive = (int32_t)(t + 1);
            const int32_t post = sb->last_spike[twq & kTgtMask];
            if (post >= 0) wq = stdp_depress(sa->rules[cls - 1], wq, (int64_t)arrive - (int64_t)post);
            sa->wa[j] = make_uint2(__float_as_uint(wq), (uint32_t)arrive);
          }
        }
        const uint64_t idx = (uint64_t)(twq >> kRcptShift) * (uint64_t)ring.N + (twq & kTgtMask);
        if (kFixed) {
          const long long qv = __float2ll_rn(wq * 4294967296.0f) * (long long)mult;
          atomicAdd(reinterpret_cast<unsigned long long*>(ring.p) + idx, (unsigned long long)qv);
        } else {
          const float v = mult == 1u ? wq : wq * (float)mult;
          atomicAdd(reinterpret_cast<float*>(ring.p) + idx, v);
        }
      }
    }
  }
}

}  // namespace ngb
