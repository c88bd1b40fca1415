// neuron_lif.cu -- fused LIF update kernel (K1) and the state initialiser.
//
// One thread per neuron per step, for LIF neurons with exponential PSCs
// (Eqs. 1-2), integrated exactly on the dt grid (Sec. 2.1, exact integration
// after Rotter & Diesmann 1999).  In one pass each thread
//   1. reads its ring-buffer slot for step t and zeroes it in place,
//   2. adds the Poisson drive of step t (Sec. 2.1 Poisson generator): the
//      count is the inverse CDF of a Philox word, evaluated as the number of
//      integer thresholds ceil(F(k) * 2^32) not above the word,
//   3. propagates V with the current of the previous grid point unless
//      refractory, then decays the current and adds the step's input,
//   4. tests the threshold (V >= V_th -> V = V_reset, refractory counter),
//   5. joins the warp-ballot compaction of the new spikes.
// All FP32 arithmetic uses explicit round-to-nearest intrinsics, so no FMA
// contraction changes the result: V and I are a fixed function of the input.
#include "ngb_internal.cuh"
#include "philox.cuh"

namespace ngb {

template <bool kFixed>
__global__ void __launch_bounds__(kLifBlock) k_update_lif(const LifSeg* __restrict__ segs, int nseg,
                                                          const uint32_t* __restrict__ thr, float* __restrict__ y_,
                                                          float* __restrict__ I_, int32_t* __restrict__ ref_,
                                                          Ring ring, int64_t* clk,
                                                          const uint64_t* __restrict__ src_syn, SpikeBuf sb) {
  const int s = find_segment(segs, nseg, (int64_t)blockIdx.x);
  const LifSeg& sg = segs[s];
  const int64_t k = ((int64_t)blockIdx.x - sg.blk_begin) * kLifBlock + threadIdx.x;
  const int64_t t = clk[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) clk[1] = t;
  const bool valid = k < sg.n;
  bool spk = false;
  const uint32_t gid = (uint32_t)(sg.offset + k);
  if (valid) {
    const uint64_t slot = (uint64_t)(t & ring.L_mask);
    const uint64_t idx = slot * (uint64_t)ring.R * (uint64_t)ring.N + gid;
    float in;
    if (kFixed) {
      long long* rp = reinterpret_cast<long long*>(ring.p) + idx;
      const long long v = *rp;
      *rp = 0;
      in = __double2float_rn(__dmul_rn(__ll2double_rn(v), 2.3283064365386963e-10));  // x 2^-32
    } else {
      float* rp = reinterpret_cast<float*>(ring.p) + idx;
      in = *rp;
      *rp = 0.0f;
    }
    if (sg.n_thr > 0) {
      const int64_t tl = t - sg.t0;
      const U4 r = draw4(sg.seed, (uint64_t)tl, kPurPoisson, 0u, sg.local_off + (uint32_t)k);
      const uint32_t* th = thr + sg.thr_off;
      uint32_t kp = 0;
      while (kp < sg.n_thr && r.x >= __ldg(th + kp)) ++kp;
      in = __fadd_rn(in, __fmul_rn((float)kp, sg.w_ext));
    }
    float y = y_[gid];
    float I = I_[gid];
    int32_t ref = ref_[gid];
    if (ref > 0) {
      ref -= 1;
    } else {
      y = __fadd_rn(__fadd_rn(__fmul_rn(sg.P22, y), __fmul_rn(sg.P21, I)), sg.P20Ie);
    }
    I = __fadd_rn(__fmul_rn(sg.P11, I), in);
    if (y >= sg.theta) {
      y = sg.y_reset;
      ref = sg.ref_steps;
      spk = true;
    }
    y_[gid] = y;
    I_[gid] = I;
    ref_[gid] = ref;
  }
  emit_spikes(spk, gid, 1u, t, src_syn, sb);
}

cudaError_t launch_update_lif(const LifSeg* segs, int nseg, int64_t blocks, const uint32_t* thr, float* y, float* I,
                              int32_t* ref, Ring ring, bool fixed, int64_t* clk, const uint64_t* src_syn,
                              SpikeBuf sb, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  if (fixed)
    k_update_lif<true><<<(unsigned)blocks, kLifBlock, 0, st>>>(segs, nseg, thr, y, I, ref, ring, clk, src_syn, sb);
  else
    k_update_lif<false><<<(unsigned)blocks, kLifBlock, 0, st>>>(segs, nseg, thr, y, I, ref, ring, clk, src_syn, sb);
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
