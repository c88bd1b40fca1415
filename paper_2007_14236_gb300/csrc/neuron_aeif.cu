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
// scans the pending spikes (as the LIF kernel).  kAlpha: alpha-function
// conductances (the paper's balanced network, Sec. 2.4) with state x_ex, x_in.
#include "aeif_rk.cuh"
#include "deliver_item.cuh"
#include "neuron_step.cuh"

namespace ngb {

template <bool kFixed, int kMode, bool kAlpha>
__global__ void __launch_bounds__(kAeifBlock) k_update_aeif(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const uint32_t* __restrict__ thr,
                                                            float* __restrict__ V_, float* __restrict__ w_,
                                                            float* __restrict__ ge_, float* __restrict__ gi_,
                                                            float* __restrict__ h_, float* __restrict__ xe_,
                                                            float* __restrict__ xi_, Ring ring, int64_t* clk,
                                                            int64_t step_off, const Csr csr, SpikeBuf sb, int scan,
                                                            int budget) {
  constexpr bool kAge = kMode == kEmitAge;
  __shared__ uint32_t s_thr[kMaxThr];
  const int seg = segment_index_of(T, (int64_t)blockIdx.x);
  const AeifSeg p = T.n <= kInlineSegs ? T.s[seg] : T.dev[seg];
  const int64_t k = ((int64_t)blockIdx.x - p.blk_begin) * kAeifBlock + threadIdx.x;
  const bool valid = k < p.n;
  const uint32_t gid = (uint32_t)(p.offset + k);
  // prologue (overlaps the previous kernel): state, source metadata, Poisson table
  St y{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float h0 = 0.f;
  uint4 meta = make_uint4(0, 0, 0, 0);
  if (valid) {
    y.V = V_[gid];
    y.w = w_[gid];
    y.ge = ge_[gid];
    y.gi = gi_[gid];
    if (kAlpha) {
      y.xe = xe_[gid];
      y.xi = xi_[gid];
    }
    h0 = h_[gid];
    if (!kAge) meta = __ldg(csr.src_meta + gid);
  }
  for (uint32_t i = threadIdx.x; i < p.n_thr; i += kAeifBlock) s_thr[i] = __ldg(thr + p.thr_off + i);
  __syncthreads();
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  if (kMode != kEmitPipe && blockIdx.x == 0 && threadIdx.x == 0) clk[1] = t;
  if (kAge && scan)
    scan_pending<false>(t, csr, sb, ((int64_t)blockIdx.x * kAeifBlock + threadIdx.x) >> 5,
                        ((int64_t)gridDim.x * kAeifBlock) >> 5);
  uint32_t nspk = 0;
  unsigned long long nsub = 0;
  bool done = true;
  uint4 rec[4];
  if (valid) {
    const uint64_t slot = (uint64_t)(t & ring.L_mask);
    const uint64_t i0 = (slot * (uint64_t)ring.R) * (uint64_t)ring.N + gid;
    float in0 = ring_take<kFixed, false>(ring.p, i0);
    float in1 = ring_take<kFixed, false>(ring.p, i0 + (uint64_t)ring.N);
    if (p.n_thr > 0) {
      const uint32_t kp = poisson_count(p.seed, t - p.t0, p.local_off + (uint32_t)k, s_thr, p.n_thr);
      const float add = __fmul_rn((float)kp, p.w_ext);
      if (p.prec_rcpt == 0) in0 = __fadd_rn(in0, add);
      else in1 = __fadd_rn(in1, add);
    }
    RkPos r{(double)h0, 0.0, 0};
    bool cap_hit = false;
    done = aeif_advance<kAlpha>(p, y, r, budget, in0, in1, nspk, nsub, cap_hit);
    if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
    if (done) {
      V_[gid] = y.V;
      w_[gid] = y.w;
      ge_[gid] = y.ge;
      gi_[gid] = y.gi;
      if (kAlpha) {
        xe_[gid] = y.xe;
        xi_[gid] = y.xi;
      }
      h_[gid] = (float)r.h;
    } else {
      rec[0] = make_uint4(gid, (uint32_t)seg, nspk, (uint32_t)r.n);
      rec[1] = make_uint4(__float_as_uint(y.V), __float_as_uint(y.w), __float_as_uint(y.ge), __float_as_uint(y.gi));
      rec[2] = make_uint4(__float_as_uint(y.xe), __float_as_uint(y.xi), __float_as_uint(in0), __float_as_uint(in1));
      const unsigned long long hb = (unsigned long long)__double_as_longlong(r.h);
      const unsigned long long tb = (unsigned long long)__double_as_longlong(r.t_in);
      rec[3] = make_uint4((uint32_t)hb, (uint32_t)(hb >> 32), (uint32_t)tb, (uint32_t)(tb >> 32));
    }
  }
  defer_write(!done, rec, sb, kAlpha ? 1 : 0, t);
  // sub-step statistics: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
  if ((threadIdx.x & 31) == 0 && nsub) atomicAdd(sb.substeps, nsub);
  const uint32_t mult = nspk > 63u ? 63u : nspk;
  if (kMode == kEmitAge) emit_spikes_age(done && nspk > 0, gid, mult, t, csr, sb);
  else if (kMode == kEmitPipe)
    emit_spikes_pipe<kFixed>(done && nspk > 0, gid, mult, t, meta,
                             (done && nspk > 0) ? __ldg(csr.src_age + gid) : make_uint2(0, 0), csr, ring, sb);
  else emit_spikes(done && nspk > 0, gid, mult, t, meta, sb);
}

// Second part of the AdEx step: the neurons whose step did not finish within
// the update kernel's attempt budget (mostly those crossing V_peak, whose
// step needs tens of attempts) continue from their saved position, packed
// 32 to a warp, then write their state and join the spike compaction.
template <bool kFixed, int kMode, bool kAlpha>
__global__ void __launch_bounds__(kAeifBlock) k_aeif_finish(const __grid_constant__ SegTable<AeifSeg> T,
                                                            float* __restrict__ V_, float* __restrict__ w_,
                                                            float* __restrict__ ge_, float* __restrict__ gi_,
                                                            float* __restrict__ h_, float* __restrict__ xe_,
                                                            float* __restrict__ xi_, Ring ring, int64_t* clk,
                                                            int64_t step_off, const Csr csr, SpikeBuf sb) {
  constexpr bool kAge = kMode == kEmitAge;
  griddep_wait();
  griddep_launch();
  const int kind = kAlpha ? 1 : 0;
  const int64_t t = clk[0] + step_off;
  unsigned long long n = sb.dcnt[2 * kind + (int)(t & 1)];
  if (n > (unsigned long long)sb.dfr_cap) n = (unsigned long long)sb.dfr_cap;
  // the previous step's list is finished (this stream ran its finishing kernel
  // first) and the next step appends to it only after this kernel
  if (blockIdx.x == 0 && threadIdx.x == 0) sb.dcnt[2 * kind + (int)((t + 1) & 1)] = 0;
  const uint4* __restrict__ list = sb.dfr[kind];
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * kAeifBlock + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * kAeifBlock) >> 5;
  for (unsigned long long base = warp * 32; base < n; base += nwarps * 32) {
    const unsigned long long i = base + lane;
    const bool valid = i < n;
    uint32_t gid = 0, nspk = 0;
    unsigned long long nsub = 0;
    uint4 meta = make_uint4(0, 0, 0, 0);
    if (valid) {
      const uint4 r0 = list[4 * i], r1 = list[4 * i + 1], r2 = list[4 * i + 2], r3 = list[4 * i + 3];
      gid = r0.x;
      const AeifSeg p = T.dev[r0.y];
      nspk = r0.z;
      if (!kAge) meta = __ldg(csr.src_meta + gid);
      St y{__uint_as_float(r1.x), __uint_as_float(r1.y), __uint_as_float(r1.z), __uint_as_float(r1.w),
           __uint_as_float(r2.x), __uint_as_float(r2.y)};
      RkPos r{__longlong_as_double((long long)((unsigned long long)r3.x | ((unsigned long long)r3.y << 32))),
              __longlong_as_double((long long)((unsigned long long)r3.z | ((unsigned long long)r3.w << 32))),
              (int64_t)r0.w};
      bool cap_hit = false;
      aeif_advance<kAlpha>(p, y, r, 0, __uint_as_float(r2.z), __uint_as_float(r2.w), nspk, nsub, cap_hit);
      if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
      V_[gid] = y.V;
      w_[gid] = y.w;
      ge_[gid] = y.ge;
      gi_[gid] = y.gi;
      if (kAlpha) {
        xe_[gid] = y.xe;
        xi_[gid] = y.xi;
      }
      h_[gid] = (float)r.h;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
    if (lane == 0 && nsub) atomicAdd(sb.substeps, nsub);
    const uint32_t mult = nspk > 63u ? 63u : nspk;
    if (kMode == kEmitAge) emit_spikes_age(nspk > 0, gid, mult, t, csr, sb);
    else if (kMode == kEmitPipe)
      emit_spikes_pipe<kFixed>(nspk > 0, gid, mult, t, meta, nspk > 0 ? __ldg(csr.src_age + gid) : make_uint2(0, 0),
                               csr, ring, sb);
    else emit_spikes(nspk > 0, gid, mult, t, meta, sb);
  }
}

namespace {
template <bool kFixed, int kMode>
cudaError_t aeif_launch(const SegTable<AeifSeg>& segs, dim3 g, const uint32_t* thr, float* V, float* w, float* gex,
                        float* gin, float* h, float* xe, float* xi, bool alpha, Ring ring, int64_t* clk,
                        int64_t step_off, const Csr& csr, SpikeBuf sb, int sc, int budget, bool pdl, cudaStream_t st) {
  const dim3 b(kAeifBlock);
  if (alpha)
    return launch_k(k_update_aeif<kFixed, kMode, true>, g, b, pdl, st, segs, thr, V, w, gex, gin, h, xe, xi, ring, clk,
                    step_off, csr, sb, sc, budget);
  return launch_k(k_update_aeif<kFixed, kMode, false>, g, b, pdl, st, segs, thr, V, w, gex, gin, h, xe, xi, ring, clk,
                  step_off, csr, sb, sc, budget);
}

template <bool kFixed, int kMode>
cudaError_t finish_launch(const SegTable<AeifSeg>& segs, dim3 g, float* V, float* w, float* gex, float* gin, float* h,
                          float* xe, float* xi, bool alpha, Ring ring, int64_t* clk, int64_t step_off, const Csr& csr,
                          SpikeBuf sb, bool pdl, cudaStream_t st) {
  const dim3 b(kAeifBlock);
  if (alpha)
    return launch_k(k_aeif_finish<kFixed, kMode, true>, g, b, pdl, st, segs, V, w, gex, gin, h, xe, xi, ring, clk,
                    step_off, csr, sb);
  return launch_k(k_aeif_finish<kFixed, kMode, false>, g, b, pdl, st, segs, V, w, gex, gin, h, xe, xi, ring, clk,
                  step_off, csr, sb);
}
}  // namespace

cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V,
                               float* w, float* gex, float* gin, float* h, float* xe, float* xi, bool alpha,
                               Ring ring, bool fixed, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb,
                               int emit, bool scan, int budget, bool pdl, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks);
  const int sc = scan ? 1 : 0;
#define NGB_AEIF(F, M) \
  return aeif_launch<F, M>(segs, g, thr, V, w, gex, gin, h, xe, xi, alpha, ring, clk, step_off, csr, sb, sc, budget, pdl, st)
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

cudaError_t launch_finish_aeif(const SegTable<AeifSeg>& segs, int grid, float* V, float* w, float* gex, float* gin,
                               float* h, float* xe, float* xi, bool alpha, Ring ring, bool fixed, int64_t* clk,
                               int64_t step_off, const Csr& csr, SpikeBuf sb, int emit, bool pdl, cudaStream_t st) {
  const dim3 g((unsigned)grid);
#define NGB_FIN(F, M) \
  return finish_launch<F, M>(segs, g, V, w, gex, gin, h, xe, xi, alpha, ring, clk, step_off, csr, sb, pdl, st)
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
