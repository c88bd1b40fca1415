// step_fused.cu -- fused step loop: neuron update and delivery of the block's
// own spikes in one launch per step (ring delivery scheme).
//
// The per-step path hands the step's spikes from the update kernels to a
// separate delivery kernel through a global work-item list.  Here the block
// that updated a neuron delivers that neuron's spike itself, right after the
// update: the block's spikes are compacted in shared memory and its warps
// share their 128-synapse work items (the same scatter as the delivery
// kernel, deliver_item.cuh).  No grid-wide step is needed between update and
// delivery, because a spike of step t lands in ring slots t + d with
// 1 <= d < L, never in slot t, which other blocks may still be reading; the
// launch boundary then orders the deliveries before the next step's update.
// One launch per step and model instead of two, no work-item list in HBM.
//
// The step of a launch is clk[0] + step_off: the launches of a captured graph
// carry step_off = 0, 1, ..., S-1 and one tick launch after the graph adds S.
// With programmatic dependent launch, only static data (source metadata,
// Poisson tables) is read before griddep_wait(); the state is written by the
// previous launch of the same kernel.
#include "aeif_rk.cuh"
#include "deliver_item.cuh"
#include "neuron_step.cuh"

namespace ngb {

template <bool kFixed, typename WT>
__global__ void __launch_bounds__(kLifBlock) k_step_lif(const __grid_constant__ SegTable<LifSeg> T,
                                                        const uint32_t* __restrict__ thr, float* __restrict__ y_,
                                                        float* __restrict__ I_, int32_t* __restrict__ ref_, Ring ring,
                                                        const int64_t* clk, int64_t step_off, const Csr csr,
                                                        SpikeBuf sb) {
  __shared__ uint32_t s_thr[kMaxThr];
  __shared__ BlockSpikes<kLifBlock> S;
  const LifSeg sg = segment_of(T, (int64_t)blockIdx.x);
  const int64_t k = ((int64_t)blockIdx.x - sg.blk_begin) * kLifBlock + threadIdx.x;
  const bool valid = k < sg.n;
  const uint32_t gid = (uint32_t)(sg.offset + k);
  uint4 meta = make_uint4(0, 0, 0, 0);
  if (valid) meta = __ldg(csr.src_meta + gid);
  for (uint32_t i = threadIdx.x; i < sg.n_thr; i += kLifBlock) s_thr[i] = __ldg(thr + sg.thr_off + i);
  if (threadIdx.x == 0) S.n = 0;
  __syncthreads();
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  bool spk = false;
  if (valid) {
    float y = y_[gid], I = I_[gid];
    int32_t ref = ref_[gid];
    const uint64_t slot = (uint64_t)(t & ring.L_mask);
    float in = ring_take<kFixed, false>(ring.p, slot * (uint64_t)ring.R * (uint64_t)ring.N + gid);
    if (sg.n_thr > 0) {
      const uint32_t kp = poisson_count(sg.seed, t - sg.t0, sg.local_off + (uint32_t)k, s_thr, sg.n_thr);
      in = __fadd_rn(in, __fmul_rn((float)kp, sg.w_ext));
    }
    spk = lif_step(sg, y, I, ref, in);
    y_[gid] = y;
    I_[gid] = I;
    ref_[gid] = ref;
  }
  record_spikes(spk, gid, 1u, t, spk ? (unsigned long long)meta.z : 0ull, sb);
  deliver_block_spikes<WT, kFixed, kLifBlock>(spk, gid, 1u, meta, t, csr, ring, S);
}

template <bool kFixed, typename WT, bool kAlpha>
__global__ void __launch_bounds__(kAeifBlock) k_step_aeif(const __grid_constant__ SegTable<AeifSeg> T,
                                                          const uint32_t* __restrict__ thr, float* __restrict__ V_,
                                                          float* __restrict__ w_, float* __restrict__ ge_,
                                                          float* __restrict__ gi_, float* __restrict__ h_,
                                                          float* __restrict__ xe_, float* __restrict__ xi_, Ring ring,
                                                          const int64_t* clk, int64_t step_off, const Csr csr,
                                                          SpikeBuf sb) {
  __shared__ uint32_t s_thr[kMaxThr];
  __shared__ BlockSpikes<kAeifBlock> S;
  const AeifSeg p = segment_of(T, (int64_t)blockIdx.x);
  const int64_t k = ((int64_t)blockIdx.x - p.blk_begin) * kAeifBlock + threadIdx.x;
  const bool valid = k < p.n;
  const uint32_t gid = (uint32_t)(p.offset + k);
  uint4 meta = make_uint4(0, 0, 0, 0);
  if (valid) meta = __ldg(csr.src_meta + gid);
  for (uint32_t i = threadIdx.x; i < p.n_thr; i += kAeifBlock) s_thr[i] = __ldg(thr + p.thr_off + i);
  if (threadIdx.x == 0) S.n = 0;
  __syncthreads();
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  uint32_t nspk = 0;
  unsigned long long nsub = 0;
  if (valid) {
    St y{V_[gid], w_[gid], ge_[gid], gi_[gid], 0.f, 0.f};
    if (kAlpha) {
      y.xe = xe_[gid];
      y.xi = xi_[gid];
    }
    double h = (double)h_[gid];
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
    bool cap_hit = false;
    aeif_step<kAlpha ? kAeifAlpha : kAeifExp>(p, y, h, in0, in1, nspk, nsub, cap_hit);
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
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
  if ((threadIdx.x & 31) == 0 && nsub) atomicAdd(sb.substeps, nsub);
  const uint32_t mult = nspk > 63u ? 63u : nspk;
  record_spikes(nspk > 0, gid, mult, t, nspk ? (unsigned long long)meta.z * mult : 0ull, sb);
  deliver_block_spikes<WT, kFixed, kAeifBlock>(nspk > 0, gid, mult, meta, t, csr, ring, S);
}

__global__ void k_tick_add(int64_t* clk, int64_t n, unsigned long long* ctr, unsigned long long* ctr3) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x != 0) return;
  const int64_t t = clk[0] + n;
  clk[0] = t;
  clk[1] = t - 1;
  ctr[0] = 0;
  ctr[1] = 0;
  if (ctr3) {
    ctr3[0] = 0;
    ctr3[1] = 0;
    ctr3[2] = 0;
  }
}

namespace {
template <bool kFixed, typename WT>
cudaError_t lif_t(const SegTable<LifSeg>& segs, int64_t blocks, const uint32_t* thr, float* y, float* I,
                  int32_t* ref, Ring ring, const int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb,
                  bool pdl, cudaStream_t st) {
  return launch_k(k_step_lif<kFixed, WT>, dim3((unsigned)blocks), dim3(kLifBlock), pdl, st, segs, thr, y, I, ref,
                  ring, clk, step_off, csr, sb);
}
template <bool kFixed, typename WT>
cudaError_t aeif_t(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V, float* w, float* gex,
                   float* gin, float* h, float* xe, float* xi, bool alpha, Ring ring, const int64_t* clk,
                   int64_t step_off, const Csr& csr, SpikeBuf sb, bool pdl, cudaStream_t st) {
  if (alpha)
    return launch_k(k_step_aeif<kFixed, WT, true>, dim3((unsigned)blocks), dim3(kAeifBlock), pdl, st, segs, thr, V, w,
                    gex, gin, h, xe, xi, ring, clk, step_off, csr, sb);
  return launch_k(k_step_aeif<kFixed, WT, false>, dim3((unsigned)blocks), dim3(kAeifBlock), pdl, st, segs, thr, V, w,
                  gex, gin, h, xe, xi, ring, clk, step_off, csr, sb);
}
}  // namespace

cudaError_t launch_step_lif(const SegTable<LifSeg>& segs, int64_t blocks, const uint32_t* thr, float* y, float* I,
                            int32_t* ref, Ring ring, bool fixed, int wdtype, const int64_t* clk, int64_t step_off,
                            const Csr& csr, SpikeBuf sb, bool pdl, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  if (fixed) {
    if (wdtype == 0) return lif_t<true, float>(segs, blocks, thr, y, I, ref, ring, clk, step_off, csr, sb, pdl, st);
    if (wdtype == 1)
      return lif_t<true, __nv_bfloat16>(segs, blocks, thr, y, I, ref, ring, clk, step_off, csr, sb, pdl, st);
    return lif_t<true, __half>(segs, blocks, thr, y, I, ref, ring, clk, step_off, csr, sb, pdl, st);
  }
  if (wdtype == 0) return lif_t<false, float>(segs, blocks, thr, y, I, ref, ring, clk, step_off, csr, sb, pdl, st);
  if (wdtype == 1)
    return lif_t<false, __nv_bfloat16>(segs, blocks, thr, y, I, ref, ring, clk, step_off, csr, sb, pdl, st);
  return lif_t<false, __half>(segs, blocks, thr, y, I, ref, ring, clk, step_off, csr, sb, pdl, st);
}

cudaError_t launch_step_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V, float* w,
                             float* gex, float* gin, float* h, float* xe, float* xi, bool alpha, Ring ring, bool fixed,
                             int wdtype, const int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, bool pdl,
                             cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
#define NGB_A(F, T) return aeif_t<F, T>(segs, blocks, thr, V, w, gex, gin, h, xe, xi, alpha, ring, clk, step_off, csr, sb, pdl, st)
  if (fixed) {
    if (wdtype == 0) NGB_A(true, float);
    if (wdtype == 1) NGB_A(true, __nv_bfloat16);
    NGB_A(true, __half);
  }
  if (wdtype == 0) NGB_A(false, float);
  if (wdtype == 1) NGB_A(false, __nv_bfloat16);
  NGB_A(false, __half);
#undef NGB_A
}

cudaError_t launch_tick_add(int64_t* clk, int64_t n, unsigned long long* ctr, unsigned long long* ctr3, bool pdl,
                            cudaStream_t st) {
  return launch_k(k_tick_add, dim3(1), dim3(32), pdl, st, clk, n, ctr, ctr3);
}

}  // namespace ngb
