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
#include "neuron_step.cuh"

namespace ngb {

template <bool kFixed, bool kAge, bool kAlpha>
__global__ void __launch_bounds__(kAeifBlock) k_update_aeif(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const uint32_t* __restrict__ thr,
                                                            float* __restrict__ V_, float* __restrict__ w_,
                                                            float* __restrict__ ge_, float* __restrict__ gi_,
                                                            float* __restrict__ h_, float* __restrict__ xe_,
                                                            float* __restrict__ xi_, Ring ring, int64_t* clk,
                                                            const Csr csr, SpikeBuf sb, int scan) {
  __shared__ uint32_t s_thr[kMaxThr];
  const AeifSeg p = segment_of(T, (int64_t)blockIdx.x);
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
  const int64_t t = clk[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) clk[1] = t;
  if (kAge && scan)
    scan_pending<false>(t, csr, sb, ((int64_t)blockIdx.x * kAeifBlock + threadIdx.x) >> 5,
                        ((int64_t)gridDim.x * kAeifBlock) >> 5);
  uint32_t nspk = 0;
  unsigned long long nsub = 0;
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
    double h = (double)h0;
    bool cap_hit = false;
    aeif_step<kAlpha>(p, y, h, in0, in1, nspk, nsub, cap_hit);
    if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
    V_[gid] = y.V;
    w_[gid] = y.w;
    ge_[gid] = y.ge;
    gi_[gid] = y.gi;
    if (kAlpha) {
      xe_[gid] = y.xe;
      xi_[gid] = y.xi;
    }
    h_[gid] = (float)h;
  }
  // sub-step statistics: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
  if ((threadIdx.x & 31) == 0 && nsub) atomicAdd(sb.substeps, nsub);
  const uint32_t mult = nspk > 63u ? 63u : nspk;
  if (kAge) emit_spikes_age(nspk > 0, gid, mult, t, csr, sb);
  else emit_spikes(nspk > 0, gid, mult, t, meta, sb);
}

cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V,
                               float* w, float* gex, float* gin, float* h, float* xe, float* xi, bool alpha,
                               Ring ring, bool fixed, int64_t* clk, const Csr& csr, SpikeBuf sb, bool age, bool scan,
                               bool pdl, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks), b(kAeifBlock);
  const int sc = scan ? 1 : 0;
#define NGB_AEIF(F, A, P) \
  return launch_k(k_update_aeif<F, A, P>, g, b, pdl, st, segs, thr, V, w, gex, gin, h, xe, xi, ring, clk, csr, sb, sc)
  if (alpha) {
    if (fixed) {
      if (age) NGB_AEIF(true, true, true);
      NGB_AEIF(true, false, true);
    }
    if (age) NGB_AEIF(false, true, true);
    NGB_AEIF(false, false, true);
  }
  if (fixed) {
    if (age) NGB_AEIF(true, true, false);
    NGB_AEIF(true, false, false);
  }
  if (age) NGB_AEIF(false, true, false);
  NGB_AEIF(false, false, false);
#undef NGB_AEIF
}

}  // namespace ngb
