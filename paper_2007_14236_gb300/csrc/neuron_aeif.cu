// neuron_aeif.cu -- fused AdEx update kernel (K2).
//
// One thread per neuron per step for the AdEx model with exponential
// conductance synapses (Eqs. 3-5), integrated over the step dt by an embedded
// fifth-order Runge-Kutta method with adaptive step size (Sec. 2.1), using
// the published Cash-Karp (1990) 4(5) tableau.  State and stages are FP32;
// the step size, the time inside the step and the error-ratio test are FP64
// (the step-size control is the part that accumulates many terms).
//
// Per thread: read the two receptor slots of step t and zero them, add the
// Poisson drive, integrate with error control (error of component i relative
// to |y_i| + |h f_i| + floor_i, safety 0.9, growth exponent -1/5 capped at
// 5x, shrink exponent -1/4 capped at 10x), reset V -> V_reset, w -> w + b
// after every accepted sub-step ending at V >= V_peak (the exponential term
// is evaluated at min(V, V_peak)), then add the step's conductance input and
// join the warp-ballot spike compaction with the spike multiplicity.  In the
// spike-buffer delivery scheme the kernel that runs first in the step also
// scans the pending spikes (as the LIF kernel).  kM: the conductance model,
// exponential, alpha (the paper's balanced network, Sec. 2.4; state x_ex,
// x_in) or the beta multisynapse model of Sec. 2.1 (up to four receptor
// ports, each with g and x; the step reads one input plane per port in use).
#include <string>

#include "aeif_rk.cuh"
#include "ngb.h"
#include "deliver_item.cuh"
#include "neuron_step.cuh"

namespace ngb {

namespace {

// uint4 words of a deferred neuron's record.
template <int kM>
constexpr int kRecWords = kM == kAeifBeta ? 6 : 4;

__device__ __forceinline__ uint32_t fu(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float uf(uint32_t x) { return __uint_as_float(x); }

template <int kM>
__device__ __forceinline__ void load_state(const AeifState& S, uint32_t gid, int n_ports, St& y, float& h) {
  y.V = S.V[gid];
  y.w = S.w[gid];
  y.ge = S.g0[gid];
  y.gi = S.g1[gid];
  if (kM != kAeifExp) {
    y.xe = S.x0[gid];
    y.xi = S.x1[gid];
  }
  if (kM == kAeifBeta && n_ports > 2) {
    y.g2 = S.ext[gid];
    y.g3 = S.ext[S.N + gid];
    y.x2 = S.ext[2 * S.N + gid];
    y.x3 = S.ext[3 * S.N + gid];
  }
  h = S.h[gid];
}

template <int kM>
__device__ __forceinline__ void store_state(const AeifState& S, uint32_t gid, int n_ports, const St& y, float h) {
  S.V[gid] = y.V;
  S.w[gid] = y.w;
  S.g0[gid] = y.ge;
  S.g1[gid] = y.gi;
  if (kM != kAeifExp) {
    S.x0[gid] = y.xe;
    S.x1[gid] = y.xi;
  }
  if (kM == kAeifBeta && n_ports > 2) {
    S.ext[gid] = y.g2;
    S.ext[S.N + gid] = y.g3;
    S.ext[2 * S.N + gid] = y.x2;
    S.ext[3 * S.N + gid] = y.x3;
  }
  S.h[gid] = h;
}

// Record of a neuron whose step is unfinished: {gid, segment, spikes so far,
// attempts}, the state, the step's input and the position inside the step.
template <int kM>
__device__ __forceinline__ void pack_rec(uint4* rec, uint32_t gid, uint32_t seg, uint32_t nspk, const St& y,
                                         const RkPos& r, float4 in) {
  const unsigned long long hb = (unsigned long long)__double_as_longlong(r.h);
  const unsigned long long tb = (unsigned long long)__double_as_longlong(r.t_in);
  const uint4 pos = make_uint4((uint32_t)hb, (uint32_t)(hb >> 32), (uint32_t)tb, (uint32_t)(tb >> 32));
  rec[0] = make_uint4(gid, seg, nspk, (uint32_t)r.n);
  rec[1] = make_uint4(fu(y.V), fu(y.w), fu(y.ge), fu(y.gi));
  if constexpr (kM == kAeifBeta) {
    rec[2] = make_uint4(fu(y.g2), fu(y.g3), fu(y.xe), fu(y.xi));
    rec[3] = make_uint4(fu(y.x2), fu(y.x3), fu(in.x), fu(in.y));
    rec[4] = make_uint4(fu(in.z), fu(in.w), 0u, 0u);
    rec[5] = pos;
  } else {
    rec[2] = make_uint4(fu(y.xe), fu(y.xi), fu(in.x), fu(in.y));
    rec[3] = pos;
  }
}

template <int kM>
__device__ __forceinline__ void unpack_rec(const uint4* q, St& y, RkPos& r, float4& in) {
  const uint4 r0 = q[0], r1 = q[1];
  const uint4 pos = q[kRecWords<kM> - 1];
  y.V = uf(r1.x);
  y.w = uf(r1.y);
  y.ge = uf(r1.z);
  y.gi = uf(r1.w);
  if constexpr (kM == kAeifBeta) {
    const uint4 r2 = q[2], r3 = q[3], r4 = q[4];
    y.g2 = uf(r2.x);
    y.g3 = uf(r2.y);
    y.xe = uf(r2.z);
    y.xi = uf(r2.w);
    y.x2 = uf(r3.x);
    y.x3 = uf(r3.y);
    in = make_float4(uf(r3.z), uf(r3.w), uf(r4.x), uf(r4.y));
  } else {
    const uint4 r2 = q[2];
    y.xe = uf(r2.x);
    y.xi = uf(r2.y);
    in = make_float4(uf(r2.z), uf(r2.w), 0.f, 0.f);
  }
  r.h = __longlong_as_double((long long)((unsigned long long)pos.x | ((unsigned long long)pos.y << 32)));
  r.t_in = __longlong_as_double((long long)((unsigned long long)pos.z | ((unsigned long long)pos.w << 32)));
  r.n = (int64_t)r0.w;
}

}  // namespace

// List neuron gid (segment seg) as hot for step t + 1 when h: warp-aggregated
// append to the model's list of that step's parity, then the tag.  A full
// list drops the entry and leaves the tag, so the neuron stays with the
// neuron blocks (a list holds every neuron once, so it cannot fill).
__device__ __forceinline__ void hot_append(bool h, uint32_t gid, uint32_t seg, const SpikeBuf& sb, int kind,
                                           int64_t t) {
  const unsigned full = 0xffffffffu;
  const unsigned b = __ballot_sync(full, h);
  if (b == 0 || !sb.htag || !sb.hot[kind]) return;
  const int q = (int)((uint64_t)(t + 1) % 3u);
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(sb.hcnt + 3 * kind + q, (unsigned long long)__popc(b));
  base = __shfl_sync(full, base, 0);
  if (h) {
    const unsigned long long pos = base + __popc(b & ((1u << lane) - 1u));
    if (pos < (unsigned long long)sb.hot_cap) {
      sb.hot[kind][(uint64_t)q * (uint64_t)sb.hot_cap + pos] = make_uint2(gid, seg);
      sb.htag[gid] = (uint32_t)(t + 1);
    }
  }
}

// One neuron's step t: the receptor slots (read and zeroed), the Poisson
// drive (thresholds thr of its segment), then the integration with at most
// `budget` attempts (0: to the end of the step).  A finished step stores the
// state; an unfinished one is packed into rec for the finishing kernel.
template <bool kFixed, int kM>
__device__ __forceinline__ bool aeif_neuron_step(const AeifSeg& p, uint32_t gid, int64_t k, uint32_t seg,
                                                 const uint32_t* thr, int64_t t, Ring ring, const AeifState& S,
                                                 int n_ports, St& y, float h0, int budget, uint32_t& nspk,
                                                 unsigned long long& nsub, uint4* rec, const SpikeBuf& sb) {
  const uint64_t slot = (uint64_t)(t & ring.L_mask);
  const uint64_t i0 = (slot * (uint64_t)ring.R) * (uint64_t)ring.N + gid;
  float4 in = make_float4(0.f, 0.f, 0.f, 0.f);
  in.x = ring_take<kFixed, false>(ring.p, i0);
  in.y = ring_take<kFixed, false>(ring.p, i0 + (uint64_t)ring.N);
  if (kM == kAeifBeta) {
    if (n_ports > 2) in.z = ring_take<kFixed, false>(ring.p, i0 + 2 * (uint64_t)ring.N);
    if (n_ports > 3) in.w = ring_take<kFixed, false>(ring.p, i0 + 3 * (uint64_t)ring.N);
  }
  if (p.n_thr > 0) {
    const uint32_t kp = poisson_count(p.seed, t - p.t0, p.local_off + (uint32_t)k, thr, p.n_thr);
    const float add = __fmul_rn((float)kp, p.w_ext);
    switch (p.prec_rcpt) {
      case 0: in.x = __fadd_rn(in.x, add); break;
      case 1: in.y = __fadd_rn(in.y, add); break;
      case 2: in.z = __fadd_rn(in.z, add); break;
      default: in.w = __fadd_rn(in.w, add); break;
    }
  }
  RkPos r{(double)h0, 0.0, 0};
  bool cap_hit = false;
  const bool done = aeif_advance<kM>(p, y, r, budget, in, nspk, nsub, cap_hit);
  if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
  if (done) store_state<kM>(S, gid, n_ports, y, (float)r.h);
  else pack_rec<kM>(rec, gid, seg, nspk, y, r, in);
  return done;
}

// The warp's end of step t (every lane takes part): unfinished neurons to the
// deferred list, finished ones above V_hot to the next step's hot list, the
// attempt statistics, and the spike compaction.
template <bool kFixed, int kMode, int kM>
__device__ __forceinline__ void aeif_warp_end(bool on, bool done, const uint4* rec, uint32_t gid, uint32_t seg,
                                              uint32_t nspk, unsigned long long nsub, bool hot_next, uint4 meta,
                                              int64_t t, const Csr& csr, Ring ring, const SpikeBuf& sb) {
  constexpr int kW = kRecWords<kM>;
  defer_write<kW>(on && !done, rec, sb, kM, t);
  hot_append(on && done && hot_next, gid, seg, sb, kM, t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
  if ((threadIdx.x & 31) == 0 && nsub) atomicAdd(sb.substeps, nsub);
  const bool spk = on && done && nspk > 0;
  const uint32_t mult = nspk > 63u ? 63u : nspk;
  if (kMode == kEmitAge) emit_spikes_age(spk, gid, mult, t, csr, sb);
  else if (kMode == kEmitPipe)
    emit_spikes_pipe<kFixed>(spk, gid, mult, t, meta, spk ? __ldg(csr.src_age + gid) : make_uint2(0, 0), csr, ring,
                             sb);
  else emit_spikes(spk, gid, mult, t, meta, sb);
}

// The neurons listed hot for step t, 32 to a warp, whole steps (no attempt
// budget), in a kernel that runs beside the update kernel of the same step
// (which skips them): their tens of attempts start with the step instead of
// after it.  The previous step's kernels have completed before this one.
// One warp per block: the busy warps (the list's first entries) are spread one
// to an SM, since each attempt's FP64 step-size control queues for the SM's
// few FP64 units (16 busy warps on one SM ran their steps 1.6 times slower).
constexpr int kHotBlock = 32;

template <bool kFixed, int kMode, int kM>
__global__ void __launch_bounds__(kHotBlock) k_aeif_hot(const __grid_constant__ SegTable<AeifSeg> T,
                                                         const uint32_t* __restrict__ thr, const AeifState S,
                                                         Ring ring, const int64_t* clk, int64_t step_off,
                                                         const Csr csr, SpikeBuf sb) {
  constexpr bool kAge = kMode == kEmitAge;
  constexpr int kW = kRecWords<kM>;
  const int64_t t = clk[0] + step_off;
  const int q = (int)((uint64_t)t % 3u);
  unsigned long long n = sb.hcnt[3 * kM + q];
  if (n > (unsigned long long)sb.hot_cap) n = (unsigned long long)sb.hot_cap;
  const uint2* __restrict__ list = sb.hot[kM] + (uint64_t)q * (uint64_t)sb.hot_cap;
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * kHotBlock + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * kHotBlock) >> 5;
  for (unsigned long long base = warp * 32; base < n; base += nwarps * 32) {
    const unsigned long long i = base + lane;
    uint2 e = make_uint2(0, 0);
    bool on = i < n;
    if (on) {
      e = list[i];
      on = sb.htag[e.x] == (uint32_t)t;  // listed for this step (else a stale entry)
    }
    uint32_t nspk = 0;
    unsigned long long nsub = 0;
    bool hot_next = false;
    uint4 meta = make_uint4(0, 0, 0, 0);
    if (on) {
      const AeifSeg p = T.dev[e.y];
      const int n_ports = kM == kAeifBeta ? p.n_ports : 2;
      if (!kAge) meta = __ldg(csr.src_meta + e.x);
      St y{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float h0 = 0.f;
      uint4 rec[kW];  // unused: without a budget every step finishes
      load_state<kM>(S, e.x, n_ports, y, h0);
      aeif_neuron_step<kFixed, kM>(p, e.x, (int64_t)e.x - p.offset, e.y, thr + p.thr_off, t, ring, S, n_ports, y, h0,
                                   0, nspk, nsub, rec, sb);
      hot_next = y.V > p.V_hot;
    }
    const unsigned ran = __ballot_sync(0xffffffffu, on);
    if (lane == 0 && ran) atomicAdd(sb.hot_steps, (unsigned long long)__popc(ran));
    aeif_warp_end<kFixed, kMode, kM>(on, true, nullptr, e.x, e.y, nspk, nsub, hot_next, meta, t, csr, ring, sb);
  }
}

// hot != 0: the hot-list kernel runs this step's listed neurons beside this
// kernel; they are skipped here, and neurons ending above V_hot are listed.
template <bool kFixed, int kMode, int kM>
__global__ void __launch_bounds__(kAeifBlock) k_update_aeif(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const uint32_t* __restrict__ thr, const AeifState S,
                                                            Ring ring, int64_t* clk, int64_t step_off, const Csr csr,
                                                            SpikeBuf sb, int scan, int budget, int hot) {
  constexpr bool kAge = kMode == kEmitAge;
  constexpr int kW = kRecWords<kM>;
  __shared__ uint32_t s_thr[kMaxThr];
  const int seg = segment_index_of(T, (int64_t)blockIdx.x);
  const AeifSeg p = T.n <= kInlineSegs ? T.s[seg] : T.dev[seg];
  const int64_t k = ((int64_t)blockIdx.x - p.blk_begin) * kAeifBlock + threadIdx.x;
  const bool valid = k < p.n;
  const uint32_t gid = (uint32_t)(p.offset + k);
  const int n_ports = kM == kAeifBeta ? p.n_ports : 2;
  // prologue (overlaps the previous kernel): state, hot tag, source metadata, Poisson table
  St y{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float h0 = 0.f;
  uint4 meta = make_uint4(0, 0, 0, 0);
  uint32_t tag = 0xffffffffu;
  if (valid) {
    load_state<kM>(S, gid, n_ports, y, h0);
    if (hot) tag = sb.htag[gid];
    if (!kAge) meta = __ldg(csr.src_meta + gid);
  }
  for (uint32_t i = threadIdx.x; i < p.n_thr; i += kAeifBlock) s_thr[i] = __ldg(thr + p.thr_off + i);
  __syncthreads();
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (kMode != kEmitPipe) clk[1] = t;
    // the finishing kernel of this step starts its queue at 0; the hot list of
    // step t + 2 (last read in step t - 1) starts empty for the appends of step t + 1
    if (sb.dfetch) sb.dfetch[kM] = 0;
    if (hot) sb.hcnt[3 * kM + (int)((uint64_t)(t + 2) % 3u)] = 0;
  }
  if (kAge && scan)
    scan_pending<false>(t, csr, sb, ((int64_t)blockIdx.x * kAeifBlock + threadIdx.x) >> 5,
                        ((int64_t)gridDim.x * kAeifBlock) >> 5);
  // listed for this step: the hot-list kernel runs it (and may already have listed it for the next)
  const bool on = valid && tag != (uint32_t)t && tag != (uint32_t)(t + 1);
  uint32_t nspk = 0;
  unsigned long long nsub = 0;
  bool done = true;
  uint4 rec[kW];
  if (on) done = aeif_neuron_step<kFixed, kM>(p, gid, k, (uint32_t)seg, s_thr, t, ring, S, n_ports, y, h0, budget,
                                              nspk, nsub, rec, sb);
  aeif_warp_end<kFixed, kMode, kM>(on, done, rec, gid, (uint32_t)seg, nspk, nsub, hot && on && done && y.V > p.V_hot,
                                   meta, t, csr, ring, sb);
}

// Second part of the AdEx step: the neurons whose step did not finish within
// the update kernel's attempt budget continue from their saved position.  A
// lane takes one deferred neuron at a time from the list (a queue shared by
// the grid) and makes one attempt per pass; a lane whose neuron finished
// writes it back, joins the warp's spike compaction and takes the next one,
// so the warp's lanes stay busy however unequal the neurons' attempt counts.
template <bool kFixed, int kMode, int kM>
__global__ void __launch_bounds__(kAeifBlock) k_aeif_finish(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const AeifState S, Ring ring, int64_t* clk,
                                                            int64_t step_off, const Csr csr, SpikeBuf sb, int hot) {
  constexpr bool kAge = kMode == kEmitAge;
  constexpr int kW = kRecWords<kM>;
  const unsigned full = 0xffffffffu;
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  unsigned long long n = sb.dcnt[2 * kM + (int)(t & 1)];
  if (n > (unsigned long long)sb.dfr_cap) n = (unsigned long long)sb.dfr_cap;
  // the previous step's list is finished (this stream ran its finishing kernel
  // first) and the next step appends to it only after this kernel
  if (blockIdx.x == 0 && threadIdx.x == 0) sb.dcnt[2 * kM + (int)((t + 1) & 1)] = 0;
  const uint4* __restrict__ list = sb.dfr[kM];
  const int lane = threadIdx.x & 31;
  bool busy = false;  // this lane holds a neuron
  uint32_t gid = 0, nspk = 0, seg = 0;
  unsigned long long nsub = 0;
  St y{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  RkPos r{0.0, 0.0, 0};
  float4 in = make_float4(0.f, 0.f, 0.f, 0.f);
  bool more = true;  // the queue may hold neurons
  for (;;) {
    // idle lanes take the next neurons of the queue
    const unsigned want = __ballot_sync(full, !busy && more);
    if (want) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(sb.dfetch + kM, (unsigned long long)__popc(want));
      base = __shfl_sync(full, base, 0);
      if (!busy && more) {
        const unsigned long long i = base + __popc(want & ((1u << lane) - 1u));
        if (i < n) {
          const uint4* q = list + (unsigned long long)kW * i;
          const uint4 r0 = q[0];
          gid = r0.x;
          seg = r0.y;
          nspk = r0.z;
          unpack_rec<kM>(q, y, r, in);
          busy = true;
        }
      }
      if (base + __popc(want) >= n) more = false;  // every lane saw the queue run out
    }
    if (!__any_sync(full, busy)) break;
    bool fin = false, hot_next = false;
    uint4 meta = make_uint4(0, 0, 0, 0);
    if (busy) {
      const AeifSeg p = T.dev[seg];
      bool cap_hit = false;
      fin = aeif_advance<kM>(p, y, r, 1, in, nspk, nsub, cap_hit);
      if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
      if (fin) {
        store_state<kM>(S, gid, kM == kAeifBeta ? p.n_ports : 2, y, (float)r.h);
        hot_next = hot && y.V > p.V_hot;
        if (!kAge) meta = __ldg(csr.src_meta + gid);
        busy = false;
      }
    }
    aeif_warp_end<kFixed, kMode, kM>(fin, true, nullptr, gid, seg, nspk, 0ull, hot_next, meta, t, csr, ring, sb);
    if (fin) nspk = 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(full, nsub, o);
  if (lane == 0 && nsub) atomicAdd(sb.substeps, nsub);
}

namespace {
template <bool kFixed, int kMode>
cudaError_t aeif_launch(const SegTable<AeifSeg>& segs, dim3 g, const uint32_t* thr, const AeifState& S, int model,
                        Ring ring, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int sc, int budget,
                        int hot, bool pdl, cudaStream_t st) {
  const dim3 b(kAeifBlock);
  if (model == kAeifBeta)
    return launch_k(k_update_aeif<kFixed, kMode, kAeifBeta>, g, b, pdl, st, segs, thr, S, ring, clk, step_off, csr,
                    sb, sc, budget, hot);
  if (model == kAeifAlpha)
    return launch_k(k_update_aeif<kFixed, kMode, kAeifAlpha>, g, b, pdl, st, segs, thr, S, ring, clk, step_off, csr,
                    sb, sc, budget, hot);
  return launch_k(k_update_aeif<kFixed, kMode, kAeifExp>, g, b, pdl, st, segs, thr, S, ring, clk, step_off, csr, sb,
                  sc, budget, hot);
}

template <bool kFixed, int kMode>
cudaError_t hot_launch(const SegTable<AeifSeg>& segs, dim3 g, const uint32_t* thr, const AeifState& S, int model,
                       Ring ring, const int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, cudaStream_t st) {
  const dim3 b(kHotBlock);
  if (model == kAeifBeta)
    return launch_k(k_aeif_hot<kFixed, kMode, kAeifBeta>, g, b, false, st, segs, thr, S, ring, clk, step_off, csr,
                    sb);
  if (model == kAeifAlpha)
    return launch_k(k_aeif_hot<kFixed, kMode, kAeifAlpha>, g, b, false, st, segs, thr, S, ring, clk, step_off, csr,
                    sb);
  return launch_k(k_aeif_hot<kFixed, kMode, kAeifExp>, g, b, false, st, segs, thr, S, ring, clk, step_off, csr, sb);
}

template <bool kFixed, int kMode>
cudaError_t finish_launch(const SegTable<AeifSeg>& segs, dim3 g, const AeifState& S, int model, Ring ring,
                          int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int hot, bool pdl,
                          cudaStream_t st) {
  const dim3 b(kAeifBlock);
  if (model == kAeifBeta)
    return launch_k(k_aeif_finish<kFixed, kMode, kAeifBeta>, g, b, pdl, st, segs, S, ring, clk, step_off, csr, sb,
                    hot);
  if (model == kAeifAlpha)
    return launch_k(k_aeif_finish<kFixed, kMode, kAeifAlpha>, g, b, pdl, st, segs, S, ring, clk, step_off, csr, sb,
                    hot);
  return launch_k(k_aeif_finish<kFixed, kMode, kAeifExp>, g, b, pdl, st, segs, S, ring, clk, step_off, csr, sb, hot);
}
}  // namespace

cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr,
                               const AeifState& S, int model, Ring ring, bool fixed, int64_t* clk, int64_t step_off,
                               const Csr& csr, SpikeBuf sb, int emit, bool scan, int budget, bool hot, bool pdl,
                               cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks);
  const int sc = scan ? 1 : 0;
  const int h = hot && budget > 0 && sb.htag && sb.hot[model] ? 1 : 0;
#define NGB_AEIF(F, M) return aeif_launch<F, M>(segs, g, thr, S, model, ring, clk, step_off, csr, sb, sc, budget, h, pdl, st)
  if (fixed) {
    if (emit == kEmitAge) NGB_AEIF(true, kEmitAge);
    if (emit == kEmitPipe) NGB_AEIF(true, kEmitPipe);
    NGB_AEIF(true, kEmitRing);
  }
  if (emit == kEmitAge) NGB_AEIF(false, kEmitAge);
  if (emit == kEmitPipe) NGB_AEIF(false, kEmitPipe);
  NGB_AEIF(false, kEmitRing);
#undef NGB_AEIF
}

cudaError_t launch_hot_aeif(const SegTable<AeifSeg>& segs, int grid, const uint32_t* thr, const AeifState& S,
                            int model, Ring ring, bool fixed, const int64_t* clk, int64_t step_off, const Csr& csr,
                            SpikeBuf sb, int emit, cudaStream_t st) {
  if (grid <= 0 || !sb.htag || !sb.hot[model]) return cudaSuccess;
  const dim3 g((unsigned)grid);
#define NGB_HOT(F, M) return hot_launch<F, M>(segs, g, thr, S, model, ring, clk, step_off, csr, sb, st)
  if (fixed) {
    if (emit == kEmitAge) NGB_HOT(true, kEmitAge);
    if (emit == kEmitPipe) NGB_HOT(true, kEmitPipe);
    NGB_HOT(true, kEmitRing);
  }
  if (emit == kEmitAge) NGB_HOT(false, kEmitAge);
  if (emit == kEmitPipe) NGB_HOT(false, kEmitPipe);
  NGB_HOT(false, kEmitRing);
#undef NGB_HOT
}

cudaError_t launch_finish_aeif(const SegTable<AeifSeg>& segs, int grid, const AeifState& S, int model, Ring ring,
                               bool fixed, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int emit,
                               bool hot, bool pdl, cudaStream_t st) {
  const dim3 g((unsigned)grid);
  const int h = hot && sb.htag && sb.hot[model] ? 1 : 0;
#define NGB_FIN(F, M) return finish_launch<F, M>(segs, g, S, model, ring, clk, step_off, csr, sb, h, pdl, st)
  if (fixed) {
    if (emit == kEmitAge) NGB_FIN(true, kEmitAge);
    if (emit == kEmitPipe) NGB_FIN(true, kEmitPipe);
    NGB_FIN(true, kEmitRing);
  }
  if (emit == kEmitAge) NGB_FIN(false, kEmitAge);
  if (emit == kEmitPipe) NGB_FIN(false, kEmitPipe);
  NGB_FIN(false, kEmitRing);
#undef NGB_FIN
}

}  // namespace ngb

namespace ngb {
namespace {

__global__ void k_step_factor(const float* r, int64_t n, int k, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = k == 4 ? step_factor_root<4>(r[i]) : step_factor_root<5>(r[i]);
}

}  // namespace

int set_last_error(int code, const std::string& msg);  // ngb_api.cu: message for ngb_last_error()

}  // namespace ngb

extern "C" int ngb_eval_step_factor(const float* r, int64_t n, int32_t k, float* out) {
  using namespace ngb;
  if (n < 0 || (n > 0 && (!r || !out)) || (k != 4 && k != 5))
    return set_last_error(NGB_ERR_INVALID_ARG, "ngb_eval_step_factor: arguments");
  if (n == 0) return NGB_OK;
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, (size_t)n * 2 * sizeof(float));
  if (e != cudaSuccess) return set_last_error(NGB_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpy(d, r, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_step_factor<<<(unsigned)((n + 255) / 256), 256>>>(d, n, k, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_last_error(NGB_ERR_CUDA, std::string("ngb_eval_step_factor: ") + cudaGetErrorString(e));
  return NGB_OK;
}
