// neuron_lif.cu -- fused LIF update kernel (K1) and the state initialiser.
//
// One thread per neuron per step, for LIF neurons with exponential PSCs
// (Eqs. 1-2), integrated exactly on the dt grid (Sec. 2.1, exact integration
// after Rotter & Diesmann 1999).  The population's constants come from the
// kernel parameters, its Poisson table is staged in shared memory, and all
// independent loads are issued before the step counter is needed, so a
// thread waits on two dependent memory round trips (counter, ring slot) plus
// one more when it spikes.  Loads that do not depend on the previous kernel
// are issued before griddep_wait(), so with programmatic dependent launch
// they overlap the previous step's delivery.  In one pass each thread
//   1. reads its ring-buffer slot for step t and zeroes it in place,
//   2. adds the Poisson drive of step t (Sec. 2.1 Poisson generator): the
//      count is the inverse CDF of a Philox word, evaluated as the number of
//      integer thresholds ceil(F(k) * 2^32) not above the word,
//   3. propagates V with the current of the previous grid point unless
//      refractory, then decays the current and adds the step's input,
//   4. tests the threshold (V >= V_th -> V = V_reset, refractory counter),
//   5. joins the warp-ballot compaction of the new spikes.
// In the spike-buffer delivery scheme (Sec. 2.2) the kernel that runs first in
// the step also moves the pending spikes whose next connection group is due
// to the step's due-item list, and a new spike reads its source's group data
// only when it fires (no per-neuron metadata prefetch).
// All FP32 arithmetic uses explicit round-to-nearest intrinsics, so no FMA
// contraction changes the result: V and I are a fixed function of the input.
#include "deliver_item.cuh"
#include "neuron_step.cuh"

namespace ngb {

// kNpt neurons per thread (1, or 4 for networks that fill the GPU several
// times over): a block covers 256 * kNpt consecutive neurons of one segment,
// and each thread issues the loads of all its neurons before the first use,
// so that enough bytes are in flight to cover the memory latency.
// The body of one update block: block `blk` of a grid of `nblk` update
// blocks (the LIF update kernel's own block, or a block of the pipelined step
// kernel that also delivers).  kEarlyState: the neuron state is loaded before
// griddep_wait (the previous kernel in the stream does not write it); else
// after it.  early_clk: the previous kernel does not write the step counter
// either, so the step and the Poisson counts (which depend on nothing else)
// are computed before griddep_wait, and the state and the ring slot are then
// loaded together.
template <bool kFixed, int kMode, int kNpt, bool kEarlyState = true>
__device__ __forceinline__ void lif_update_block(const SegTable<LifSeg>& T, const uint32_t* __restrict__ thr,
                                                 float* __restrict__ y_, float* __restrict__ I_,
                                                 int32_t* __restrict__ ref_, const Ring& ring, int64_t* clk,
                                                 int64_t step_off, const Csr& csr, const SpikeBuf& sb, int scan,
                                                 int64_t blk, int64_t nblk, bool early_clk = false) {
  constexpr bool kAge = kMode == kEmitAge;
  __shared__ uint32_t s_thr[kMaxThr];
  const LifSeg sg = segment_of(T, blk);
  const int64_t k0 = (blk - sg.blk_begin) * (kLifBlock * kNpt) + threadIdx.x;
  // Prologue, overlapping the previous kernel (programmatic dependent launch):
  // state written two launches ago, static source metadata, Poisson table.
  float y[kNpt], I[kNpt];
  int32_t ref[kNpt];
  uint4 meta[kNpt];
  uint2 ag[kNpt];
#pragma unroll
  for (int j = 0; j < kNpt; ++j) {
    const int64_t k = k0 + j * kLifBlock;
    const uint32_t gid = (uint32_t)(sg.offset + k);
    y[j] = 0.0f;
    I[j] = 0.0f;
    ref[j] = 0;
    meta[j] = make_uint4(0, 0, 0, 0);
    ag[j] = make_uint2(0, 0);
    if (k < sg.n) {
      if (kEarlyState) {
        y[j] = y_[gid];
        I[j] = I_[gid];
        ref[j] = ref_[gid];
      }
      if (!kAge) meta[j] = __ldg(csr.src_meta + gid);
      if (kMode == kEmitPipe) ag[j] = __ldg(csr.src_age + gid);
    }
  }
  for (uint32_t i = threadIdx.x; i < sg.n_thr; i += kLifBlock) s_thr[i] = __ldg(thr + sg.thr_off + i);
  __syncthreads();
  int64_t t = 0;
  uint32_t kp[kNpt];
  auto draw_counts = [&]() {
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      const int64_t k = k0 + j * kLifBlock;
      kp[j] = (k < sg.n && sg.n_thr > 0)
                  ? poisson_count(sg.seed, t - sg.t0, sg.local_off + (uint32_t)k, s_thr, sg.n_thr)
                  : 0u;
    }
  };
  if (early_clk) {
    t = clk[0] + step_off;
    draw_counts();
  }
  // the previous step's delivery has completed: ring slot t and the counters are final
  griddep_wait();
  griddep_launch();
  if (!early_clk) t = clk[0] + step_off;
  if (!kEarlyState) {
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      const int64_t k = k0 + j * kLifBlock;
      if (k < sg.n) {
        const uint32_t gid = (uint32_t)(sg.offset + k);
        y[j] = y_[gid];
        I[j] = I_[gid];
        ref[j] = ref_[gid];
      }
    }
  }
  if (kMode != kEmitPipe && blk == 0 && threadIdx.x == 0) clk[1] = t;
  if (kAge && scan) scan_pending<false>(t, csr, sb, (blk * kLifBlock + threadIdx.x) >> 5, (nblk * kLifBlock) >> 5);
  const uint64_t slot_base = (uint64_t)(t & ring.L_mask) * (uint64_t)ring.R * (uint64_t)ring.N;
  float in[kNpt];
#pragma unroll
  for (int j = 0; j < kNpt; ++j) {
    const int64_t k = k0 + j * kLifBlock;
    in[j] = k < sg.n ? ring_read<kFixed, false>(ring.p, slot_base + (uint32_t)(sg.offset + k)) : 0.0f;
  }
  if (!early_clk) draw_counts();
#pragma unroll
  for (int j = 0; j < kNpt; ++j) {
    const int64_t k = k0 + j * kLifBlock;
    const uint32_t gid = (uint32_t)(sg.offset + k);
    bool spk = false;
    if (k < sg.n) {
      ring_clear<kFixed>(ring.p, slot_base + gid);
      float x = in[j];
      if (sg.n_thr > 0) x = __fadd_rn(x, __fmul_rn((float)kp[j], sg.w_ext));
      spk = lif_step(sg, y[j], I[j], ref[j], x);
      y_[gid] = y[j];
      I_[gid] = I[j];
      ref_[gid] = ref[j];
    }
    if (kMode == kEmitAge) emit_spikes_age(spk, gid, 1u, t, csr, sb);
    else if (kMode == kEmitPipe) emit_spikes_pipe<kFixed>(spk, gid, 1u, t, meta[j], ag[j], csr, ring, sb);
    else emit_spikes(spk, gid, 1u, t, meta[j], sb);
  }
}

template <bool kFixed, int kMode, int kNpt>
__global__ void __launch_bounds__(kLifBlock, kNpt > 1 ? (kMode == kEmitPipe ? 2 : 3) : (kMode == kEmitRing ? 8 : (kMode == kEmitPipe ? 5 : 6)))
    k_update_lif(const __grid_constant__ SegTable<LifSeg> T, const uint32_t* __restrict__ thr,
                 float* __restrict__ y_, float* __restrict__ I_, int32_t* __restrict__ ref_, Ring ring, int64_t* clk,
                 int64_t step_off, const Csr csr, SpikeBuf sb, int scan) {
  lif_update_block<kFixed, kMode, kNpt>(T, thr, y_, I_, ref_, ring, clk, step_off, csr, sb, scan,
                                        (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// Pipelined step kernel (ring scheme, LIF networks, one launch per step):
// blocks [0, n_upd) update step t = clk[0] + step_off (delivering each new
// spike's delay-1 group and queueing its other groups for step t mod 3), the
// other blocks deliver the queue of step t - 1 (slots t + 1 and later, so
// nothing the update reads), when deliver_prev is set.  The queue of step
// t + 1 mod 3, last read by the previous launch, is emptied here.  Launched
// one per step in a single stream with programmatic dependent launch.
template <bool kFixed, typename WT>
__global__ void __launch_bounds__(kLifBlock, 5)
    k_step_pipe(const __grid_constant__ SegTable<LifSeg> T, const uint32_t* __restrict__ thr, float* __restrict__ y_,
                float* __restrict__ I_, int32_t* __restrict__ ref_, Ring ring, int64_t* clk, int64_t step_off,
                const Csr csr, SpikeBuf sb, int64_t n_upd, int deliver_prev) {
  if ((int64_t)blockIdx.x < n_upd) {
    // the previous launch (the previous step) writes the state: loaded after the wait
    // the step counter changes only between graphs (the previous launch of a
    // graph's first step is the clock tick): known before the wait elsewhere
    lif_update_block<kFixed, kEmitPipe, 1, false>(T, thr, y_, I_, ref_, ring, clk, step_off, csr, sb, 0,
                                                  (int64_t)blockIdx.x, n_upd, step_off > 0);
    return;
  }
  griddep_wait();  // the previous step's kernel (and its queue) has completed
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  if ((int64_t)blockIdx.x == n_upd && threadIdx.x == 0) sb.ctr3[(int)((t + 1) % 3)] = 0;
  if (!deliver_prev) return;
  const uint32_t warp = (uint32_t)((((int64_t)blockIdx.x - n_upd) * kLifBlock + threadIdx.x) >> 5);
  const uint32_t nwarps = (uint32_t)((((int64_t)gridDim.x - n_upd) * kLifBlock) >> 5);
  const int lane = threadIdx.x & 31;
  const int q = (int)((t - 1) % 3);
  const uint32_t n = (uint32_t)(sb.ctr3[q] & kChunkMask);
  const uint4* __restrict__ wq = sb.wi3[q];
  for (uint32_t ch = warp; ch < n; ch += nwarps)
    deliver_work_item<WT, kFixed>(wq[2 * (uint64_t)ch], wq[2 * (uint64_t)ch + 1], t - 1, csr, ring, lane);
}

cudaError_t launch_step_pipe(const SegTable<LifSeg>& segs, int64_t upd_blocks, int del_blocks, const uint32_t* thr,
                             float* y, float* I, int32_t* ref, Ring ring, bool fixed, int wdtype, int64_t* clk,
                             int64_t step_off, const Csr& csr, SpikeBuf sb, bool deliver_prev, bool pdl,
                             cudaStream_t st) {
  const dim3 g((unsigned)(upd_blocks + del_blocks)), b(kLifBlock);
  const int dp = deliver_prev ? 1 : 0;
#define NGB_SP(F, W) \
  return launch_k(k_step_pipe<F, W>, g, b, pdl, st, segs, thr, y, I, ref, ring, clk, step_off, csr, sb, upd_blocks, dp)
  if (fixed) {
    if (wdtype == 0) NGB_SP(true, float);
    if (wdtype == 1) NGB_SP(true, __nv_bfloat16);
    NGB_SP(true, __half);
  }
  if (wdtype == 0) NGB_SP(false, float);
  if (wdtype == 1) NGB_SP(false, __nv_bfloat16);
  NGB_SP(false, __half);
#undef NGB_SP
}

// Large networks (kNpt = 2 or 4 neurons per thread, ring or spike-buffer
// scheme): a grid of resident blocks walks the tiles of kNpt x 256 neurons,
// block b taking
// tiles b, b + G, b + 2G, ...  Each thread loads the state and the ring slot
// of its next tile while it computes the current one, so two tiles' loads
// are in flight per thread.  The Poisson thresholds are read through the L1
// cache (no shared-memory staging, so no barrier when the next tile lies in
// another population).  The block's new spikes are collected in shared
// memory and compacted once at the end (or when the buffer nears capacity),
// so the list atomics leave the per-tile path and happen once per 32 spikes
// instead of once per warp with a spike; the ring scheme reads a spiking
// source's metadata only then.  Same arithmetic and spike lists as
// k_update_lif.
constexpr int kTileSpkCap = 4096;  // spikes buffered per block before a compaction

template <bool kFixed, int kMode>
__device__ __forceinline__ void flush_block_spikes(const uint32_t* s_spk, int n, int64_t t, const Csr& csr,
                                                   const SpikeBuf& sb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp * 32; c < n; c += kLifBlock) {
    const bool spk = c + lane < n;
    const uint32_t gid = spk ? s_spk[c + lane] : 0u;
    if (kMode == kEmitAge) {
      emit_spikes_age(spk, gid, 1u, t, csr, sb);
    } else {
      const uint4 meta = spk ? __ldg(csr.src_meta + gid) : make_uint4(0, 0, 0, 0);
      emit_spikes(spk, gid, 1u, t, meta, sb);
    }
  }
}

template <bool kFixed, int kMode, int kNpt>
__global__ void __launch_bounds__(kLifBlock, kNpt == 4 ? 2 : 4)
    k_update_lif_tiles(const __grid_constant__ SegTable<LifSeg> T, const uint32_t* __restrict__ thr,
                       float* __restrict__ y_, float* __restrict__ I_, int32_t* __restrict__ ref_, Ring ring,
                       int64_t* clk, int64_t step_off, const Csr csr, SpikeBuf sb, int scan, int64_t n_tiles) {
  constexpr bool kAge = kMode == kEmitAge;
  __shared__ uint32_t s_spk[kTileSpkCap];
  __shared__ int s_n;
  float y[kNpt], I[kNpt], in[kNpt], yn[kNpt], In[kNpt], inn[kNpt];
  int32_t ref[kNpt], rn[kNpt];
  auto load_state = [&](int64_t tile, const LifSeg& g, float* yy, float* ii, int32_t* rr) {
    const int64_t k0 = (tile - g.blk_begin) * (kLifBlock * kNpt) + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      const int64_t k = k0 + j * kLifBlock;
      const uint32_t gid = (uint32_t)(g.offset + k);
      yy[j] = 0.0f;
      ii[j] = 0.0f;
      rr[j] = 0;
      if (k < g.n) {
        yy[j] = y_[gid];
        ii[j] = I_[gid];
        rr[j] = ref_[gid];
      }
    }
  };
  auto load_input = [&](int64_t tile, const LifSeg& g, uint64_t slot_base, float* xx) {
    const int64_t k0 = (tile - g.blk_begin) * (kLifBlock * kNpt) + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      const int64_t k = k0 + j * kLifBlock;
      xx[j] = k < g.n ? ring_read<kFixed, false>(ring.p, slot_base + (uint32_t)(g.offset + k)) : 0.0f;
    }
  };
  int64_t tile = blockIdx.x;
  LifSeg sg = segment_of(T, tile < n_tiles ? tile : 0);
  if (tile < n_tiles) load_state(tile, sg, y, I, ref);
  if (threadIdx.x == 0) s_n = 0;
  griddep_wait();  // the previous step's delivery has completed
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  if (blockIdx.x == 0 && threadIdx.x == 0) clk[1] = t;
  const uint64_t slot_base = (uint64_t)(t & ring.L_mask) * (uint64_t)ring.R * (uint64_t)ring.N;
  if (tile < n_tiles) load_input(tile, sg, slot_base, in);
  if (kAge && scan)
    scan_pending<false>(t, csr, sb, ((int64_t)blockIdx.x * kLifBlock + threadIdx.x) >> 5,
                        ((int64_t)gridDim.x * kLifBlock) >> 5);
  __syncthreads();  // s_n initialised
  for (; tile < n_tiles; tile += gridDim.x) {
    const int64_t k0 = (tile - sg.blk_begin) * (kLifBlock * kNpt) + threadIdx.x;
    // the next tile's state and input, in flight while this tile is computed
    const int64_t nxt = tile + gridDim.x;
    LifSeg sn = sg;
    if (nxt < n_tiles) {
      sn = segment_of(T, nxt);
      load_state(nxt, sn, yn, In, rn);
      load_input(nxt, sn, slot_base, inn);
    }
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      const int64_t k = k0 + j * kLifBlock;
      if (k >= sg.n) continue;
      const uint32_t gid = (uint32_t)(sg.offset + k);
      ring_clear<kFixed>(ring.p, slot_base + gid);
      float x = in[j];
      if (sg.n_thr > 0) {
        const uint32_t kp =
            poisson_count(sg.seed, t - sg.t0, sg.local_off + (uint32_t)k, thr + sg.thr_off, sg.n_thr);
        x = __fadd_rn(x, __fmul_rn((float)kp, sg.w_ext));
      }
      const bool spk = lif_step(sg, y[j], I[j], ref[j], x);
      y_[gid] = y[j];
      I_[gid] = I[j];
      ref_[gid] = ref[j];
      if (spk) s_spk[atomicAdd(&s_n, 1)] = gid;
    }
    // compact the buffered spikes when the next tile could overflow the buffer
    __syncthreads();
    const int n_now = s_n;
    if (n_now > kTileSpkCap - kLifBlock * kNpt) {
      flush_block_spikes<kFixed, kMode>(s_spk, n_now, t, csr, sb);
      __syncthreads();
      if (threadIdx.x == 0) s_n = 0;
      __syncthreads();
    }
    sg = sn;
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      y[j] = yn[j];
      I[j] = In[j];
      ref[j] = rn[j];
      in[j] = inn[j];
    }
  }
  __syncthreads();
  flush_block_spikes<kFixed, kMode>(s_spk, s_n, t, csr, sb);
}

namespace {
// Resident blocks per SM of the tiled kernel (queried once per instantiation).
template <bool kFixed, int kMode, int kNpt>
int tiles_grid(int64_t n_tiles) {
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_lif_tiles<kFixed, kMode, kNpt>, kLifBlock,
                                                      0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return (int)std::min<int64_t>(n_tiles, (int64_t)sms * per_sm);
}

template <bool kFixed, int kMode>
cudaError_t lif_launch(const SegTable<LifSeg>& segs, dim3 g, int npt, const uint32_t* thr, float* y, float* I,
                       int32_t* ref, Ring ring, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int sc,
                       bool pdl, cudaStream_t st) {
  const dim3 b(kLifBlock);
  constexpr int kM = kMode == kEmitPipe ? kEmitRing : kMode;  // the tiled kernel has no pipelined variant
  if (npt > 1 && kMode != kEmitPipe) {
    const int64_t n_tiles = (int64_t)g.x;
    if (npt == 2)
      return launch_k(k_update_lif_tiles<kFixed, kM, 2>, dim3((unsigned)tiles_grid<kFixed, kM, 2>(n_tiles)), b, pdl,
                      st, segs, thr, y, I, ref, ring, clk, step_off, csr, sb, sc, n_tiles);
    return launch_k(k_update_lif_tiles<kFixed, kM, 4>, dim3((unsigned)tiles_grid<kFixed, kM, 4>(n_tiles)), b, pdl, st,
                    segs, thr, y, I, ref, ring, clk, step_off, csr, sb, sc, n_tiles);
  }
  if (npt == 4)
    return launch_k(k_update_lif<kFixed, kMode, 4>, g, b, pdl, st, segs, thr, y, I, ref, ring, clk, step_off, csr, sb,
                    sc);
  if (npt == 2)
    return launch_k(k_update_lif<kFixed, kMode, 2>, g, b, pdl, st, segs, thr, y, I, ref, ring, clk, step_off, csr, sb,
                    sc);
  return launch_k(k_update_lif<kFixed, kMode, 1>, g, b, pdl, st, segs, thr, y, I, ref, ring, clk, step_off, csr, sb,
                  sc);
}
}  // namespace

cudaError_t launch_update_lif(const SegTable<LifSeg>& segs, int64_t blocks, int npt, const uint32_t* thr, float* y,
                              float* I, int32_t* ref, Ring ring, bool fixed, int64_t* clk, int64_t step_off,
                              const Csr& csr, SpikeBuf sb, int emit, bool scan, bool pdl, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks);
  const int sc = scan ? 1 : 0;
#define NGB_LIF(F, M) return lif_launch<F, M>(segs, g, npt, thr, y, I, ref, ring, clk, step_off, csr, sb, sc, pdl, st)
  if (fixed) {
    if (emit == kEmitAge) NGB_LIF(true, kEmitAge);
    if (emit == kEmitPipe) NGB_LIF(true, kEmitPipe);
    NGB_LIF(true, kEmitRing);
  }
  if (emit == kEmitAge) NGB_LIF(false, kEmitAge);
  if (emit == kEmitPipe) NGB_LIF(false, kEmitPipe);
  NGB_LIF(false, kEmitRing);
#undef NGB_LIF
}

// Step counter hand-over when no update kernel runs (a network with no
// active neurons): the delivery kernel reads clk[1].
__global__ void k_tick(int64_t* clk) {
  griddep_wait();
  griddep_launch();
  clk[1] = clk[0];
}

cudaError_t launch_tick(int64_t* clk, bool pdl, cudaStream_t st) {
  return launch_k(k_tick, dim3(1), dim3(32), pdl, st, clk);
}

// ------------------------------------------------------------------ source metadata
__global__ void k_build_meta(int64_t N, const uint64_t* __restrict__ src_syn, const uint32_t* __restrict__ src_grp,
                             uint4* __restrict__ meta, unsigned long long* __restrict__ total_items) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint64_t b = src_syn[i], e = src_syn[i + 1];
  const uint32_t g0 = src_grp[i], g1 = src_grp[i + 1];
  meta[i] = make_uint4((uint32_t)b, (uint32_t)((b >> 32) & 0xFFFFu) | ((g1 - g0) << 16), (uint32_t)(e - b), g0);
  if (e > b) atomicAdd(total_items, (unsigned long long)((e - (b & ~3ull) + kChunk - 1) / kChunk));
}

cudaError_t launch_build_meta(int64_t N, const uint64_t* src_syn, const uint32_t* src_grp, uint4* meta,
                              unsigned long long* total_items, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  k_build_meta<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, src_syn, src_grp, meta, total_items);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ initial state
__global__ void k_init_state(int model, int64_t n, double mean, double sd, double E_L, double w0, double h0,
                             uint64_t seed, uint32_t local_off, float* a, float* b, float* h) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double V0 = mean;
  if (sd != 0.0) {
    const U4 r = draw4(seed, (uint64_t)(local_off + (uint64_t)i), kPurVinit, 0u, 0u);
    V0 = __dadd_rn(mean, __dmul_rn(sd, gauss(r)));
  }
  if (model == 0) {
    a[i] = __double2float_rn(__dsub_rn(V0, E_L));
  } else {
    a[i] = __double2float_rn(V0);
    b[i] = __double2float_rn(w0);
    h[i] = __double2float_rn(h0);
  }
}

cudaError_t launch_init_state(int model, int64_t n, double mean, double sd, double E_L, double w0, double h0,
                              uint64_t seed, uint32_t local_off, float* a, float* b, float* h, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_init_state<<<(unsigned)blocks, 256, 0, st>>>(model, n, mean, sd, E_L, w0, h0, seed, local_off, a, b, h);
  return cudaGetLastError();
}

}  // namespace ngb
