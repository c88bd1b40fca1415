// tiled.cu -- target-tiled spike delivery (spike-buffer scheme).
//
// Sec. 2.2 of the paper: when a spike's age reaches the delay of one of its
// source's connection groups, every synapse of the group adds its weight to
// its target's input; in the spike-buffer scheme that input is the single
// slot of the next step.  The plain delivery kernel (deliver.cu) does one L2
// atomic per synaptic event, which caps networks where every neuron receives
// about one event per step (no target-side reuse): there the L2 atomic rate,
// not HBM, bounds the step.
//
// Here the targets are cut into tiles of T consecutive neurons and each
// tile's input is accumulated in shared memory by the block, or the cluster
// of P blocks, that owns the tile (each of the P blocks takes every P-th due
// group; the cluster then sums its P partial tiles through distributed shared
// memory).  For that the synapses are stored a second time: every group's
// synapses partitioned by target tile (stable, so within a tile the storage
// order is kept), as {target word, weight bits} pairs, each tile's part padded
// to a multiple of 16 pairs (128 bytes) with filler pairs and every group
// starting on a 128-byte boundary, so that a part is whole cache lines.  A
// boundary pool holds, per group, the number of tiles its targets span and
// the (padded) offset of each tile's part within the group:
//   tile_grp[g] = {pool offset o, first tile j0, first pair of the group (lo, hi)}
//   pool[o]     = span (tiles j0 .. j0 + span - 1)
//   pool[o + 1 + k] = first pair of tile j0 + k within the group (k = 0 .. span)
// The update kernels append each due group to the bucket of its first tile
// (ngb_internal.cuh, age_emit); the blocks of tile j read the buckets of the
// tiles from lo[j] (the lowest first tile of any group reaching tile j) to j,
// take their share of the items, read the item's part for tile j and add it
// into shared memory; then the tile's slot is written once (the update kernel
// zeroed it).  No global atomic per synaptic event remains.
//
// Bytes per synaptic event: 8 (the pair) read from HBM, times the padding;
// per due group and tile block 16 (item) + 12 (pool words); per neuron and
// step 4 (slot write).  Results equal the plain kernel's: in deterministic
// mode (64-bit fixed point) bit for bit.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "builder.h"
#include "deliver_item.cuh"
#include "ngb_internal.cuh"

namespace ngb {

namespace {

constexpr int kTileBlock = 512;

// First target tile and span of every group (one warp per group).
__global__ void k_tile_span(const uint64_t* __restrict__ grp_start, uint64_t G, const uint32_t* __restrict__ tgt,
                            uint32_t T, uint32_t* tile0, unsigned long long* width, unsigned int* maxspan) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const uint64_t b = grp_start[g], e = grp_start[g + 1];
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    for (uint64_t k = b + lane; k < e; k += 32) {
      const uint32_t x = (tgt[k] & kTgtMask) / T;
      lo = min(lo, x);
      hi = max(hi, x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const uint32_t span = e > b ? hi - lo + 1 : 0;
      const uint32_t j0 = e > b ? lo : 0;
      tile0[g] = j0;
      width[g] = (unsigned long long)span + 2;
      if (span) atomicMax(maxspan + j0, span);
    }
  }
}

// Per group: the size of each tile's part, padded to 16 pairs, as offsets
// in the pool, and the group's padded size (one warp per group).
__global__ void k_tile_count(const uint64_t* __restrict__ grp_start, uint64_t G, const uint32_t* __restrict__ tgt,
                             uint32_t T, const uint32_t* __restrict__ tile0, const unsigned long long* __restrict__ off,
                             uint32_t* pool, unsigned long long* plen) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const uint64_t b = grp_start[g], e = grp_start[g + 1];
    const uint64_t o = off[g];
    const uint32_t span = (uint32_t)(off[g + 1] - o) - 2;
    const uint32_t j0 = tile0[g];
    uint32_t run = 0;  // padded pairs so far
    for (uint32_t k = 0; k < span; ++k) {
      if (lane == 0) pool[o + 1 + k] = run;
      uint32_t c = 0;
      for (uint64_t q = b; q < e; q += 32) {
        const uint64_t s = q + lane;
        c += __popc(__ballot_sync(0xffffffffu, s < e && (tgt[s] & kTgtMask) / T == j0 + k));
      }
      run += (c + 15u) & ~15u;
    }
    if (lane == 0) {
      pool[o] = span;
      pool[o + 1 + span] = run;
      plen[g] = run;
    }
  }
}

// Scatter every group's synapses into its tiles' parts (stable; the pairs
// array is pre-filled with filler pairs) and record the group's table entry.
template <typename WT>
__global__ void k_tile_fill(const uint64_t* __restrict__ grp_start, uint64_t G, const uint32_t* __restrict__ tgt,
                            const WT* __restrict__ w, uint32_t T, const uint32_t* __restrict__ tile0,
                            const unsigned long long* __restrict__ off, const unsigned long long* __restrict__ base,
                            const uint32_t* __restrict__ pool, uint2* pairs, uint4* tile_grp,
                            unsigned int* bucket_n) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const uint64_t b = grp_start[g], e = grp_start[g + 1];
    const uint64_t o = off[g], B = base[g];
    const uint32_t span = pool[o];
    const uint32_t j0 = tile0[g];
    for (uint32_t k = 0; k < span; ++k) {
      uint64_t d = B + pool[o + 1 + k];
      for (uint64_t q = b; q < e; q += 32) {
        const uint64_t s = q + lane;
        const uint32_t x = s < e ? tgt[s] : 0u;
        const bool in = s < e && (x & kTgtMask) / T == j0 + k;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          uint32_t wb;
          if constexpr (sizeof(WT) == 4) wb = __float_as_uint((float)w[s]);
          else wb = (uint32_t)w[s];
          pairs[d + __popc(m & ((1u << lane) - 1u))] = make_uint2(x, wb);
        }
        d += __popc(m);
      }
    }
    if (lane == 0) {
      tile_grp[g] = make_uint4((uint32_t)o, j0, (uint32_t)B, (uint32_t)(B >> 32));
      if (span) atomicAdd(bucket_n + j0, 1u);
    }
  }
}

__global__ void k_u32_to_u64(const unsigned int* in, unsigned long long* out, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// The weight of a pair: FP32 bits, or the 16 storage bits in the low half.
template <typename WT>
struct WBits;
template <>
struct WBits<float> {
  static __device__ __forceinline__ float get(uint32_t b) { return __uint_as_float(b); }
};
template <>
struct WBits<__nv_bfloat16> {
  static __device__ __forceinline__ float get(uint32_t b) { return __uint_as_float(b << 16); }
};
template <>
struct WBits<__half> {
  static __device__ __forceinline__ float get(uint32_t b) { return __half2float(__ushort_as_half((unsigned short)b)); }
};

// Block-wide exclusive scan of cnt[0, n) in shared memory (n <= 32 * blockDim).
__device__ void block_scan(unsigned int* cnt, int n, unsigned int* warp_tot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int a = min(n, tid * per), z = min(n, a + per);
  unsigned int s = 0;
  for (int i = a; i < z; ++i) s += cnt[i];
  unsigned int inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned int v = lane < nwarp ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nwarp) warp_tot[lane] = v;
  }
  __syncthreads();
  unsigned int run = inc - s + (warp > 0 ? warp_tot[warp - 1] : 0u);
  for (int i = a; i < z; ++i) {
    const unsigned int c = cnt[i];
    cnt[i] = run;
    run += c;
  }
  if (tid == blockDim.x - 1) cnt[n] = run;
  __syncthreads();
}

// One due item of the block's share, mapped to its group's part in tile j:
// the item (bucket prefix pre over nb buckets from b0) and then its pool words.
struct Part {
  uint64_t start;  // first synapse of the part
  uint32_t cnt;    // synapses in the part (0: none)
  uint32_t mult;   // spike multiplicity
};

// Item q of the block's buckets: among the ne non-empty ones (first items
// pre2[], bucket indices bkt_of[] relative to b0, in item order).
__device__ __forceinline__ uint4 load_item(const unsigned int* pre2, const unsigned int* bkt_of, int ne, unsigned int q,
                                           const uint4* items, const unsigned long long* boff, uint32_t b0) {
  int lo = 0, hi = ne;  // pre2[lo] <= q < pre2[lo + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre2[mid] <= q) lo = mid;
    else hi = mid;
  }
  return items[__ldg(boff + b0 + bkt_of[lo]) + (q - pre2[lo])];
}

// One block per (tile, part).  Shared memory: the tile's accumulators
// [R][T] (FP32, or int64 fixed point), then the block's bucket prefix.  Each
// warp takes batches of 32 items (one per lane) and keeps three batches in
// flight: the items of batch k + 2, the pool words of batch k + 1 and the
// synapses of batch k, in 256-byte chunks, two rounds of eight at a time.
template <typename WT, bool kFixed>
__global__ void __launch_bounds__(kTileBlock) k_deliver_tiled(SpikeBuf sb, TiledArgs A, Ring ring, int64_t* clk) {
  using Acc = typename std::conditional<kFixed, unsigned long long, float>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  Acc* acc = reinterpret_cast<Acc*>(smem);
  const uint32_t T = A.T;
  unsigned int* pre = reinterpret_cast<unsigned int*>(smem + (size_t)A.R * T * sizeof(Acc));
  __shared__ unsigned int warp_tot[32];
  griddep_wait();    // the step's update kernels have completed
  griddep_launch();  // the next step's update may start its prologue
  const uint32_t j = blockIdx.x / A.P, p = blockIdx.x % A.P;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t t = clk[1];
  const int buf = (int)(t & 1);
  if (blockIdx.x == 0 && tid == 0) {
    clk[0] = t + 1;        // next step for the update kernels
    sb.ctr[buf ^ 1] = 0;   // the plain list of the next step starts empty (shared with the plain kernel)
    sb.pcnt[buf] = 0;      // consumed by this step's scan; refilled by step t + 1's
  }
  if (p == 0 && tid == 0) sb.bcnt[(size_t)(buf ^ 1) * A.n_tiles + j] = 0;
  for (uint32_t i = tid; i < (uint32_t)A.R * T; i += blockDim.x) acc[i] = 0;
  // the buckets this tile reads: lo[j] .. j
  const uint32_t b0 = __ldg(A.lo + j);
  const int nb = (int)(j - b0 + 1);
  const unsigned int* cnts = sb.bcnt + (size_t)buf * A.n_tiles;
  for (int k = tid; k < nb; k += blockDim.x) {
    const unsigned long long cap = __ldg(sb.boff + b0 + k + 1) - __ldg(sb.boff + b0 + k);
    const unsigned int c = cnts[b0 + k];
    pre[k] = c < cap ? c : (unsigned int)cap;
  }
  __syncthreads();
  block_scan(pre, nb, warp_tot);
  const unsigned int Q = pre[nb];
  // the non-empty buckets only, in bucket order, so that an item's bucket is
  // found among them: pre2[m] (first item) and bkt_of[m] (bucket index
  // relative to b0), m < ne
  unsigned int* fl = pre + (nb + 1);
  unsigned int* pre2 = fl + (nb + 1);
  unsigned int* bkt_of = pre2 + (nb + 1);
  for (int k = tid; k < nb; k += blockDim.x) fl[k] = pre[k + 1] > pre[k] ? 1u : 0u;
  __syncthreads();
  block_scan(fl, nb, warp_tot);
  const int ne = (int)fl[nb];
  for (int k = tid; k < nb; k += blockDim.x) {
    if (pre[k + 1] > pre[k]) {
      pre2[fl[k]] = pre[k];
      bkt_of[fl[k]] = (unsigned int)k;
    }
  }
  __syncthreads();
  const uint4* __restrict__ items = buf ? sb.bkt[1] : sb.bkt[0];
  const unsigned int mine = Q > p ? (Q - p + A.P - 1) / A.P : 0u;  // items q = p + i * P
  const uint32_t tile_lo = j * T;
  // every tile starts its items at another place (all tiles read the same
  // items, and reading them in the same order would send every block to the
  // same L2 lines at once)
  const unsigned int rot = mine ? (unsigned int)(((uint64_t)j * mine) / A.n_tiles) : 0u;
  auto item_q = [&](unsigned int i) -> unsigned int {
    unsigned int k = i + rot;
    if (k >= mine) k -= mine;
    return p + k * A.P;
  };
  const int warp = tid >> 5, nwarp = blockDim.x >> 5;
  const unsigned int stride = (unsigned int)nwarp * 32;
  const uint4 none = make_uint4(0, 0, 0xFFFFFFFFu, 0);  // z = first tile: never <= j
  // pipeline: item of batch k + 2 (it2), pool words of batch k + 1 (pw), synapses of batch k
  unsigned int i0 = (unsigned int)warp * 32;
  uint4 it1 = i0 + lane < mine ? load_item(pre2, bkt_of, ne, item_q(i0 + lane), items, sb.boff, b0) : none;
  uint4 it2 = i0 + stride + lane < mine ? load_item(pre2, bkt_of, ne, item_q(i0 + stride + lane), items, sb.boff, b0)
                                        : none;
  auto pool_of = [&](const uint4& it, uint32_t& span, uint32_t& oa, uint32_t& ob) {
    const uint32_t rel = j - it.z;  // huge when the item is absent
    span = 0;
    oa = ob = 0;
    if (it.z <= j) {
      span = __ldg(A.pool + it.w);
      oa = __ldg(A.pool + it.w + 1 + rel);
      ob = __ldg(A.pool + it.w + 2 + rel);
    }
  };
  uint32_t sp1, oa1, ob1;
  pool_of(it1, sp1, oa1, ob1);
  for (; i0 < mine; i0 += stride) {
    // batch k's part from its item and pool words
    Part cur{0, 0, 0};
    if (it1.z <= j && j - it1.z < sp1) {
      cur.start = ((uint64_t)it1.x | ((uint64_t)(it1.y & 0xFFFFu) << 32)) + oa1;  // the group's first pair + part
      cur.cnt = ob1 - oa1;
      cur.mult = it1.y >> 16;
    }
    // next batches: pool words of k + 1, item of k + 2
    const uint4 it_n = it2;
    uint32_t sp_n, oa_n, ob_n;
    pool_of(it_n, sp_n, oa_n, ob_n);
    const unsigned int i2 = i0 + 2 * stride + lane;
    it2 = i2 < mine ? load_item(pre2, bkt_of, ne, item_q(i2), items, sb.boff, b0) : none;
    // batch k's synapses in chunks of 32 pairs (a part is padded to 16
    // pairs): chunk c of the batch belongs to the lane whose inclusive chunk
    // prefix first exceeds c; the warp's 32 lanes load one chunk's pairs with
    // one coalesced 256-byte load, U chunks per round, and the next round's
    // loads are issued before this round's pairs are added
    const uint32_t nch = (cur.cnt + 31u) >> 5;
    uint32_t cinc = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, cinc, o);
      if (lane >= o) cinc += v;
    }
    const uint32_t C = __shfl_sync(0xffffffffu, cinc, 31);
    constexpr int U = 4;  // chunks per round; four rounds in flight
    auto fetch = [&](uint32_t c0, uint2 pr[U], uint32_t ml[U]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t c = c0 + (uint32_t)u;  // warp-uniform
        pr[u] = make_uint2(0xFFFFFFFFu, 0u);
        ml[u] = 0;
        if (c < C) {
          int lo = 0;
#pragma unroll
          for (int stp = 16; stp > 0; stp >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, cinc, lo + stp - 1);
            if (v <= c) lo += stp;
          }
          const uint32_t first = __shfl_sync(0xffffffffu, cinc - nch, lo);
          const uint64_t s0 = __shfl_sync(0xffffffffu, cur.start, lo);
          const uint32_t cn = __shfl_sync(0xffffffffu, cur.cnt, lo);
          ml[u] = __shfl_sync(0xffffffffu, cur.mult, lo);
          const uint32_t off = (c - first) * 32u + (uint32_t)lane;
          if (off < cn) pr[u] = __ldg(A.pairs + s0 + off);
        }
      }
    };
    auto consume = [&](const uint2 pr[U], const uint32_t ml[U]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t tg = pr[u].x;
        if (tg == 0xFFFFFFFFu) continue;  // past the chunk's part, or a filler pair
        const uint32_t r = tg >> kRcptShift;
        const uint32_t loc = (tg & kTgtMask) - tile_lo;
        if (loc >= T || r >= (uint32_t)A.R) continue;  // never for a well-formed layout
        const float wv = WBits<WT>::get(pr[u].y);
        if (kFixed) {
          const long long qv = __float2ll_rn(wv * 4294967296.0f) * (long long)ml[u];
          atomicAdd(reinterpret_cast<unsigned long long*>(acc) + (size_t)r * T + loc, (unsigned long long)qv);
        } else {
          atomicAdd(reinterpret_cast<float*>(acc) + (size_t)r * T + loc, ml[u] == 1u ? wv : wv * (float)ml[u]);
        }
      }
    };
    // four register sets in rotation: rounds k + 1 .. k + 3 in flight while round k is added
    uint2 p0[U], p1[U], p2[U], p3[U];
    uint32_t m0[U], m1[U], m2[U], m3[U];
    fetch(0 * U, p0, m0);
    fetch(1 * U, p1, m1);
    fetch(2 * U, p2, m2);
    for (uint32_t c0 = 0; c0 < C; c0 += 4 * U) {
      fetch(c0 + 3 * U, p3, m3);
      consume(p0, m0);
      fetch(c0 + 4 * U, p0, m0);
      consume(p1, m1);
      fetch(c0 + 5 * U, p1, m1);
      consume(p2, m2);
      fetch(c0 + 6 * U, p2, m2);
      consume(p3, m3);
    }
    it1 = it_n;
    sp1 = sp_n;
    oa1 = oa_n;
    ob1 = ob_n;
  }
  // the tile's slot, written once: the block's own sums when it owns the
  // tile; with P blocks per tile (a thread-block cluster) block p sums its
  // slice of the tile over the P blocks' shared memory, in block order
  if (A.P == 1) {
    __syncthreads();
    for (int r = 0; r < A.R; ++r) {
      for (uint32_t loc = tid; loc < T; loc += blockDim.x) {
        const int64_t n = (int64_t)tile_lo + loc;
        const Acc v = acc[(size_t)r * T + loc];
        if (n >= A.N || v == (Acc)0) continue;
        reinterpret_cast<Acc*>(ring.p)[(size_t)r * ring.N + n] = v;
      }
    }
    return;
  }
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();  // every block's sums complete
  const uint32_t sl = (T + A.P - 1) / A.P, lo_s = p * sl, hi_s = min(T, lo_s + sl);
  for (int r = 0; r < A.R; ++r) {
    for (uint32_t loc = lo_s + tid; loc < hi_s; loc += blockDim.x) {
      const int64_t n = (int64_t)tile_lo + loc;
      if (n >= A.N) continue;
      Acc v = (Acc)0;
      for (uint32_t q = 0; q < A.P; ++q) v += cluster.map_shared_rank(acc, q)[(size_t)r * T + loc];
      if (v != (Acc)0) reinterpret_cast<Acc*>(ring.p)[(size_t)r * ring.N + n] = v;
    }
  }
  cluster.sync();  // the other blocks' shared memory stays until every slice is read
}

}  // namespace

size_t tiled_smem_bytes(bool fixed, int R, uint32_t T, uint32_t n_tiles) {
  return (size_t)R * T * (fixed ? 8 : 4) + ((size_t)n_tiles + 1) * 16;
}

cudaError_t tiled_build(const uint64_t* grp_start, uint64_t G, const uint32_t* tgt, const void* w, int wdtype,
                        uint64_t K, int64_t N, uint32_t T, uint64_t max_bytes, TiledLayout* out,
                        cudaStream_t st) {
  *out = TiledLayout{};
  if (T == 0) return cudaErrorInvalidValue;
  const uint32_t NT = (uint32_t)(((uint64_t)N + T - 1) / T);
  uint32_t* tile0 = nullptr;
  unsigned long long *width = nullptr, *off = nullptr, *plen = nullptr, *base = nullptr, *bn64 = nullptr;
  unsigned int *maxspan = nullptr, *bucket_n = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  const int grid = 2048;
  (void)K;
  cudaError_t e = cudaMalloc(&tile0, (size_t)std::max<uint64_t>(G, 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&width, (size_t)(G + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&off, (size_t)(G + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&plen, (size_t)(G + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&base, (size_t)(G + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&maxspan, (size_t)NT * 4);
  if (e == cudaSuccess) e = cudaMalloc(&bucket_n, (size_t)(NT + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&bn64, (size_t)(NT + 1) * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(maxspan, 0, (size_t)NT * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bucket_n, 0, (size_t)(NT + 1) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(width + G, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(plen + G, 0, 8, st);
  if (e == cudaSuccess && G > 0) {
    k_tile_span<<<grid, 256, 0, st>>>(grp_start, G, tgt, T, tile0, width, maxspan);
    e = cudaGetLastError();
  }
  uint64_t pool_n = 0, pairs_n = 0;
  if (e == cudaSuccess) e = scan_scratch_bytes_u64(std::max<uint64_t>(G + 1, NT + 1), &tmp_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 1);
  if (e == cudaSuccess) e = exclusive_scan_u64(width, off, G + 1, tmp, tmp_bytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&pool_n, off + G, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // the pool is read up to NT + 2 words past a group's start (a tile beyond the group's span)
  const uint64_t pool_alloc = pool_n + NT + 2;
  if (e == cudaSuccess) e = cudaMalloc(&out->pool, (size_t)pool_alloc * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(out->pool, 0, (size_t)pool_alloc * 4, st);
  if (e == cudaSuccess && G > 0) {
    k_tile_count<<<grid, 256, 0, st>>>(grp_start, G, tgt, T, tile0, off, out->pool, plen);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = exclusive_scan_u64(plen, base, G + 1, tmp, tmp_bytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&pairs_n, base + G, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const uint64_t need = (pairs_n + 64) * 8 + pool_alloc * 4 + G * (16 + 2 * 16) + (uint64_t)NT * 64;
  bool fits = e == cudaSuccess && pool_alloc < (1ull << 32) && need <= max_bytes;
  if (fits) {
    e = cudaMalloc(&out->pairs, (size_t)(pairs_n + 64) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&out->tile_grp, (size_t)std::max<uint64_t>(G, 1) * 16);
    if (e == cudaSuccess) e = cudaMalloc(&out->bkt, (size_t)std::max<uint64_t>(2 * G, 2) * 16);
    if (e == cudaSuccess) e = cudaMalloc(&out->boff, (size_t)(NT + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&out->bcnt, (size_t)2 * NT * 4);
    if (e == cudaSuccess) e = cudaMalloc(&out->lo, (size_t)NT * 4);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      fits = false;
      e = cudaSuccess;
    }
  }
  if (fits && e == cudaSuccess) e = cudaMemsetAsync(out->pairs, 0xFF, (size_t)(pairs_n + 64) * 8, st);
  if (fits && e == cudaSuccess) e = cudaMemsetAsync(out->bcnt, 0, (size_t)2 * NT * 4, st);
  if (fits && e == cudaSuccess && G > 0) {
    if (wdtype == 0)
      k_tile_fill<float><<<grid, 256, 0, st>>>(grp_start, G, tgt, (const float*)w, T, tile0, off, base, out->pool,
                                               out->pairs, out->tile_grp, bucket_n);
    else
      k_tile_fill<uint16_t><<<grid, 256, 0, st>>>(grp_start, G, tgt, (const uint16_t*)w, T, tile0, off, base,
                                                  out->pool, out->pairs, out->tile_grp, bucket_n);
    e = cudaGetLastError();
  }
  if (fits && e == cudaSuccess) {
    k_u32_to_u64<<<64, 256, 0, st>>>(bucket_n, bn64, (uint64_t)NT + 1);
    e = cudaGetLastError();
  }
  if (fits && e == cudaSuccess) e = exclusive_scan_u64(bn64, out->boff, (uint64_t)NT + 1, tmp, tmp_bytes, st);
  // lo[j]: the lowest first tile among the groups that reach tile j (j itself when none does)
  if (fits && e == cudaSuccess) {
    std::vector<unsigned int> ms((size_t)NT);
    e = cudaMemcpyAsync(ms.data(), maxspan, (size_t)NT * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<uint32_t> lo((size_t)NT);
    uint32_t cur = 0;
    for (uint32_t jj = 0; jj < NT; ++jj) {
      // the lowest j0 <= jj with j0 + maxspan[j0] > jj (jj itself when none); it never decreases with jj
      while (cur < jj && (uint64_t)cur + ms[cur] <= jj) ++cur;
      lo[jj] = cur;
    }
    uint32_t widest = 0;
    for (uint32_t jj = 0; jj < NT; ++jj) widest = std::max(widest, jj - lo[jj] + 1);
    out->max_buckets = widest;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->lo, lo.data(), (size_t)NT * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(tile0);
  cudaFree(width);
  cudaFree(off);
  cudaFree(plen);
  cudaFree(base);
  cudaFree(maxspan);
  cudaFree(bucket_n);
  cudaFree(bn64);
  cudaFree(tmp);
  if (e != cudaSuccess || !fits) {
    tiled_free(out);
    return e;
  }
  out->n_tiles = NT;
  out->T = T;
  out->pairs_n = pairs_n;
  out->bytes = need;
  return cudaSuccess;
}

void tiled_free(TiledLayout* L) {
  cudaFree(L->pairs);
  cudaFree(L->pool);
  cudaFree(L->tile_grp);
  cudaFree(L->bkt);
  cudaFree(L->boff);
  cudaFree(L->bcnt);
  cudaFree(L->lo);
  *L = TiledLayout{};
}

cudaError_t launch_deliver_tiled(SpikeBuf sb, const TiledLayout& L, uint32_t P, int wdtype, Ring ring, int R,
                                 int64_t N, bool fixed, int64_t* clk, bool pdl, cudaStream_t st) {
  TiledArgs A{};
  A.pairs = L.pairs;
  A.pool = L.pool;
  A.lo = L.lo;
  A.n_tiles = L.n_tiles;
  A.T = L.T;
  A.P = P;
  A.R = R;
  A.N = N;
  const size_t smem = tiled_smem_bytes(fixed, R, L.T, L.n_tiles);
  const dim3 g((unsigned)(L.n_tiles * P)), b(kTileBlock);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  attr[na].id = cudaLaunchAttributeClusterDimension;  // the P blocks of a tile form a cluster
  attr[na].val.clusterDim.x = P;
  attr[na].val.clusterDim.y = 1;
  attr[na].val.clusterDim.z = 1;
  ++na;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
#define NGB_TILED(T_, F_)                                                                                        \
  do {                                                                                                           \
    cudaError_t e_ = cudaFuncSetAttribute(k_deliver_tiled<T_, F_>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                          (int)smem);                                                            \
    if (e_ != cudaSuccess) return e_;                                                                            \
    return cudaLaunchKernelEx(&cfg, k_deliver_tiled<T_, F_>, sb, A, ring, clk);                                  \
  } while (0)
  if (fixed) {
    if (wdtype == 0) NGB_TILED(float, true);
    if (wdtype == 1) NGB_TILED(__nv_bfloat16, true);
    NGB_TILED(__half, true);
  }
  if (wdtype == 0) NGB_TILED(float, false);
  if (wdtype == 1) NGB_TILED(__nv_bfloat16, false);
  NGB_TILED(__half, false);
#undef NGB_TILED
}

}  // namespace ngb
