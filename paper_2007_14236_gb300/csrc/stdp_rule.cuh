// stdp_rule.cuh -- the weight update of nearest-neighbour STDP (Sec. 2.1),
// with the power-law weight dependence of Guetig et al. (2003):
//   potentiation (lag n >= 0 from the arrival to the target's spike)
//     w <- w + lambda W_max (1 - w / W_max)^mu_plus e^(-n dt / tau_plus)
//   depression (lag n >= 1 from the target's spike to the arrival)
//     w <- w - alpha lambda W_max (w / W_max)^mu_minus e^(-n dt / tau_minus)
// each clipped to [0, W_max].  A_plus = lambda W_max and A_minus =
// alpha lambda W_max are FP32 constants; the exponentials are tabulated per
// lag (FP64, rounded once) up to 20 tau, beyond which nothing changes.  FP32
// arithmetic with explicit rounding (no contraction), so that exponents 0
// and 1 give the same bits as any other FP32 statement of the rule in this
// order; other exponents use powf.
#pragma once
#include "ngb_internal.cuh"

namespace ngb {

__device__ __forceinline__ float stdp_power(float x, float mu) {
  if (mu == 0.0f) return 1.0f;
  if (mu == 1.0f) return x;
  return powf(fmaxf(x, 0.0f), mu);
}

__device__ __forceinline__ float stdp_clip(float w, float W_max) { return fminf(fmaxf(w, 0.0f), W_max); }

__device__ __forceinline__ float stdp_potentiate(const StdpRule& r, float w, int64_t lag) {
  if (lag < 0 || lag >= (int64_t)r.n_plus) return w;
  const float f = stdp_power(__fsub_rn(1.0f, __fmul_rn(w, r.inv_W_max)), r.mu_plus);
  return stdp_clip(__fadd_rn(w, __fmul_rn(__fmul_rn(r.A_plus, f), __ldg(r.k_plus + lag))), r.W_max);
}

__device__ __forceinline__ float stdp_depress(const StdpRule& r, float w, int64_t lag) {
  if (lag < 0 || lag >= (int64_t)r.n_minus) return w;
  const float f = stdp_power(__fmul_rn(w, r.inv_W_max), r.mu_minus);
  return stdp_clip(__fsub_rn(w, __fmul_rn(__fmul_rn(r.A_minus, f), __ldg(r.k_minus + lag))), r.W_max);
}

}  // namespace ngb
