// neuron_step.cuh -- per-neuron arithmetic of one simulation step, shared by
// the per-step update kernels and the persistent step kernel.
//
//  * ring_take: read the input of the step from the ring buffer and zero it
//    (FP32, or int64 fixed point in units of 2^-32 converted once to FP32).
//  * poisson_count: the Poisson drive of the step (Sec. 2.1 Poisson
//    generator): the number of inverse-CDF thresholds ceil(F(k) * 2^32) not
//    above one Philox word: word tl mod 4 of the block with key = instance
//    seed, counter = (instance-local step tl div 4, -, purpose 4,
//    instance-local neuron), so one block serves four consecutive steps.
//  * lif_step: exact integration of Eqs. 1-2 over one step (Sec. 2.1),
//    threshold, reset and refractory count, with round-to-nearest intrinsics
//    so that no FMA contraction changes the result.
//  * aeif_integrate: Cash-Karp embedded RK45 with adaptive step over one step
//    for Eqs. 3-5 (Sec. 2.1).
#pragma once
#include "ngb_internal.cuh"
#include "philox.cuh"

namespace ngb {

// kCoherent: the slot may have been written by other SMs during the same
// kernel (persistent kernel), so the load bypasses L1.
template <bool kFixed, bool kCoherent>
__device__ __forceinline__ float ring_take(void* ring, uint64_t idx) {
  if (kFixed) {
    long long* rp = reinterpret_cast<long long*>(ring) + idx;
    const long long v = kCoherent ? __ldcg(rp) : *rp;
    *rp = 0;
    return __double2float_rn(__dmul_rn(__ll2double_rn(v), 2.3283064365386963e-10));  // x 2^-32
  }
  float* rp = reinterpret_cast<float*>(ring) + idx;
  const float v = kCoherent ? __ldcg(rp) : *rp;
  *rp = 0.0f;
  return v;
}

// The same as ring_take in two parts, so that several neurons' reads can be
// issued before any slot is cleared.
template <bool kFixed, bool kCoherent>
__device__ __forceinline__ float ring_read(const void* ring, uint64_t idx) {
  if (kFixed) {
    const long long* rp = reinterpret_cast<const long long*>(ring) + idx;
    const long long v = kCoherent ? __ldcg(rp) : *rp;
    return __double2float_rn(__dmul_rn(__ll2double_rn(v), 2.3283064365386963e-10));  // x 2^-32
  }
  const float* rp = reinterpret_cast<const float*>(ring) + idx;
  return kCoherent ? __ldcg(rp) : *rp;
}

template <bool kFixed>
__device__ __forceinline__ void ring_clear(void* ring, uint64_t idx) {
  if (kFixed) reinterpret_cast<long long*>(ring)[idx] = 0;
  else reinterpret_cast<float*>(ring)[idx] = 0.0f;
}

// The Philox block of the Poisson words of steps 4q .. 4q + 3.
__device__ __forceinline__ U4 poisson_block(uint64_t seed, uint64_t q, uint32_t sid) {
  return draw4(seed, q, kPurPoisson, 0u, sid);
}

__device__ __forceinline__ uint32_t poisson_word(const U4& r, int64_t tl) {
  const uint32_t k = (uint32_t)tl & 3u;
  return k == 0 ? r.x : k == 1 ? r.y : k == 2 ? r.z : r.w;
}

__device__ __forceinline__ uint32_t poisson_from_word(uint32_t x, const uint32_t* thr, uint32_t n_thr) {
  uint32_t kp = 0;
  while (kp < n_thr && x >= thr[kp]) ++kp;
  return kp;
}

__device__ __forceinline__ uint32_t poisson_count(uint64_t seed, int64_t tl, uint32_t sid, const uint32_t* thr,
                                                  uint32_t n_thr) {
  return poisson_from_word(poisson_word(poisson_block(seed, (uint64_t)tl >> 2, sid), tl), thr, n_thr);
}

// One exact-integration step of a LIF neuron in two parts.  V is propagated
// with the current of the previous grid point, so the membrane potential of
// the step and its threshold test depend on the state after the previous
// step only, not on the step's input (lif_propagate); the input enters the
// current (lif_apply).  lif_step is the two in sequence.
__device__ __forceinline__ bool lif_propagate(const LifSeg& sg, float y, float I, int32_t ref, float& yp,
                                              int32_t& rp) {
  yp = y;
  rp = ref;
  if (rp > 0) {
    rp -= 1;  // absolute refractory period: V held at V_reset
  } else {
    yp = __fadd_rn(__fadd_rn(__fmul_rn(sg.P22, y), __fmul_rn(sg.P21, I)), sg.P20Ie);
  }
  return yp >= sg.theta;
}

__device__ __forceinline__ void lif_apply(const LifSeg& sg, float& y, float& I, int32_t& ref, float yp, int32_t rp,
                                          bool spk, float in) {
  y = yp;
  ref = rp;
  I = __fadd_rn(__fmul_rn(sg.P11, I), in);
  if (spk) {
    y = sg.y_reset;
    ref = sg.ref_steps;
  }
}

// One exact-integration step of a LIF neuron with input `in` (ring + Poisson);
// returns whether it spiked.
__device__ __forceinline__ bool lif_step(const LifSeg& sg, float& y, float& I, int32_t& ref, float in) {
  float yp;
  int32_t rp;
  const bool spk = lif_propagate(sg, y, I, ref, yp, rp);
  lif_apply(sg, y, I, ref, yp, rp, spk, in);
  return spk;
}

}  // namespace ngb
