// aeif_rk.cuh -- adaptive embedded Runge-Kutta integration of one AdEx neuron
// over one step (Sec. 2.1; Eqs. 3-5), shared by the per-step AdEx kernel, the
// fused step kernel and the persistent step kernel.
//
// State y = {V, w, g_ex, g_in} for exponential conductances; with
// alpha-function conductances (the paper's balanced network, Sec. 2.4)
// also {x_ex, x_in}: g' = x - g/tau, x' = -x/tau, so that an input of weight
// W (x += W e / tau) gives g(t) = W (t/tau) e^(1 - t/tau).  The beta
// multisynapse model (Sec. 2.1) integrates four ports,
// y = {V, w, g_0..g_3, x_0..x_3} with g_k' = x_k - g_k/tau_d,k and
// x_k' = -x_k/tau_r,k; ports beyond the population's count stay zero and add
// nothing to the current or to the error.
//
// Cash & Karp (1990) 4(5) tableau; FP32 state and stages; the step size h,
// the time inside the step and the error-ratio test in FP64 (or FP32 when the
// population asks for it).  The error of component i is taken relative to
// |y_i| + |h f_i| + floor_i (floors 1 mV, 1 pA, 1e-3 nS, 1e-3 nS, 1e-3 nS/ms,
// 1e-3 nS/ms); accepted steps grow h by min(5, 0.9 r^-1/5), rejected ones
// shrink it by max(0.1, 0.9 r^-1/4), the roots taken by step_factor_root (an
// exactly specified FP32 operation sequence); h >= h_min is always accepted.  After
// every accepted sub-step ending at V >= V_peak: V -> V_reset, w -> w + b,
// and the spike is counted (the exponential term uses min(V, V_peak)).
#pragma once
#include "ngb_internal.cuh"

namespace ngb {

// Cash & Karp (1990) coefficients
constexpr float A21 = 1.0f / 5.0f;
constexpr float A31 = 3.0f / 40.0f, A32 = 9.0f / 40.0f;
constexpr float A41 = 3.0f / 10.0f, A42 = -9.0f / 10.0f, A43 = 6.0f / 5.0f;
constexpr float A51 = -11.0f / 54.0f, A52 = 5.0f / 2.0f, A53 = -70.0f / 27.0f, A54 = 35.0f / 27.0f;
constexpr float A61 = 1631.0f / 55296.0f, A62 = 175.0f / 512.0f, A63 = 575.0f / 13824.0f,
                A64 = 44275.0f / 110592.0f, A65 = 253.0f / 4096.0f;
constexpr float B1 = 37.0f / 378.0f, B3 = 250.0f / 621.0f, B4 = 125.0f / 594.0f, B6 = 512.0f / 1771.0f;
// fifth-order weights minus embedded fourth-order weights
constexpr float E1 = (float)(37.0 / 378.0 - 2825.0 / 27648.0);
constexpr float E3 = (float)(250.0 / 621.0 - 18575.0 / 48384.0);
constexpr float E4 = (float)(125.0 / 594.0 - 13525.0 / 55296.0);
constexpr float E5 = (float)(-277.0 / 14336.0);
constexpr float E6 = (float)(512.0 / 1771.0 - 1.0 / 4.0);

// Neuron state in registers: V, w, g_ex, g_in, (alpha, beta) x_ex, x_in and
// (beta ports 2-3) g_2, g_3, x_2, x_3.
struct St {
  float V, w, ge, gi, xe, xi;
  float g2, g3, x2, x3;
};

// Integrated components per conductance model.
template <int kM>
constexpr int kAeifNC = kM == kAeifExp ? 4 : kM == kAeifAlpha ? 6 : 10;

template <int NC>
__device__ __forceinline__ void deriv(const AeifSeg& p, const float y[NC], float f[NC]) {
  const float V = fminf(y[0], p.V_peak);
  const float I_spk = (p.Delta_T > 0.0f) ? p.g_L * p.Delta_T * expf((V - p.V_T) * p.inv_Delta_T) : 0.0f;
  float I_syn;
  if constexpr (NC == 10) {
    I_syn = y[2] * (p.E_p[0] - V);
#pragma unroll
    for (int k = 1; k < 4; ++k) I_syn += y[2 + k] * (p.E_p[k] - V);
  } else {
    I_syn = y[2] * (p.E_ex - V) + y[3] * (p.E_in - V);
  }
  f[0] = (-p.g_L * (V - p.E_L) + I_spk + I_syn - y[1] + p.I_e) * p.inv_C;
  f[1] = (p.a * (V - p.E_L) - y[1]) * p.inv_tau_w;
  if constexpr (NC == 10) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      f[2 + k] = y[6 + k] - y[2 + k] * p.itd_p[k];
      f[6 + k] = -y[6 + k] * p.itr_p[k];
    }
  } else if constexpr (NC == 6) {
    f[2] = y[4] - y[2] * p.inv_tau_ex;
    f[3] = y[5] - y[3] * p.inv_tau_in;
    f[4] = -y[4] * p.inv_tau_ex;
    f[5] = -y[5] * p.inv_tau_in;
  } else {
    f[2] = -y[2] * p.inv_tau_ex;
    f[3] = -y[3] * p.inv_tau_in;
  }
}

// r^(-1/K) for K = 5 (growth after an accepted sub-step) or 4 (shrink after a
// rejected one), as one fixed sequence of FP32 operations, so that every
// implementation of this definition returns the same bits: with
// r = m 2^e (m in [1, 2)) and e = K q + s (0 <= s < K),
//   r^(-1/K) = 2^(-q) * (c_K(m - 1) * 2^(-s/K)),
// 2^(-s/K) rounded to FP32 and c_K the cubic below (least-squares fit of
// m^(-1/K) on [1, 2), relative error < 2e-4) by Horner's rule with fused
// multiply-adds.  r < 2^-100 gives 2^20; r >= 2^100, infinite or NaN gives 0.
template <int K>
__device__ __forceinline__ float step_factor_root(float r) {
  if (!(r < 0x1p100f)) return 0.0f;
  if (r < 0x1p-100f) return 0x1p20f;
  const uint32_t u = __float_as_uint(r);
  const int e = (int)(u >> 23) - 127;  // sign bit is 0 here
  const float t = __uint_as_float((u & 0x7fffffu) | 0x3f800000u) - 1.0f;
  const int q = (e >= 0) ? e / K : -((K - 1 - e) / K);
  const int s = e - K * q;
  float c, ks;
  if constexpr (K == 5) {
    c = __fmaf_rn(__fmaf_rn(__fmaf_rn(-0x1.ae3294p-6f, t, 0x1.78f37cp-4f), t, -0x1.8fb646p-3f), t, 0x1.ffed6cp-1f);
    ks = s == 0 ? 0x1p+0f : s == 1 ? 0x1.bdb8cep-1f : s == 2 ? 0x1.8406p-1f : s == 3 ? 0x1.51cb46p-1f
                                                                                      : 0x1.261118p-1f;
  } else {
    c = __fmaf_rn(__fmaf_rn(__fmaf_rn(-0x1.18bd56p-5f, t, 0x1.e6677ep-4f), t, -0x1.f2b6f8p-3f), t, 0x1.ffe6dcp-1f);
    ks = s == 0 ? 0x1p+0f : s == 1 ? 0x1.ae89fap-1f : s == 2 ? 0x1.6a09e6p-1f : 0x1.306fep-1f;
  }
  return __fmul_rn(__fmul_rn(c, ks), __uint_as_float((uint32_t)(127 - q) << 23));
}

__device__ __forceinline__ float ratio_of(float err, float y, float hf, float fl) {
  return fabsf(err) / (fabsf(y) + fabsf(hf) + fl);
}

// Integrate y (NC components) over the rest of one step of p.dt, from time
// t_in inside the step after n attempts; h carries the step-size proposal in
// and out.  Adds the attempts to nsub and the spikes to nspk; cap_hit is set
// when the attempt cap (p.max_sub) ended the step early.  Returns true when
// the step is complete, false when `budget` attempts were made in this call
// first (the caller may resume later from the same y, h, t_in, n: the
// sequence of attempts is the same as without a budget).  CT is the
// precision of the step-size control (h, time inside the step, error-ratio
// test).
// a < b for the control values (step sizes, remaining time: never negative
// nor NaN); for FP64 the comparison of the bit patterns as integers, which
// orders such doubles exactly and keeps the comparison off the FP64 units.
__device__ __forceinline__ bool ctl_lt(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool ctl_lt(float a, float b) { return a < b; }

template <typename CT, int NC>
__device__ __forceinline__ bool aeif_integrate_t(const AeifSeg& p, float y[NC], CT& h, CT& t_in, int64_t& n,
                                                 int budget, uint32_t& nspk, unsigned long long& nsub,
                                                 bool& cap_hit) {
  const CT dt = (CT)p.dt, h_min = (CT)p.h_min;
  if (!(h > (CT)0)) h = dt;
  CT rem = dt - t_in;
  for (;;) {
    bool last = false;
    if (!ctl_lt(h, rem)) {  // h >= rem
      h = rem;
      last = true;
    }
    // the time reached and the time left if this attempt is accepted, computed
    // before the attempt (the same operations as after it)
    const CT t_next = t_in + h;
    const CT rem_next = dt - t_next;
    const float hf = (float)h;
    float k1[NC], k2[NC], k3[NC], k4[NC], k5[NC], k6[NC], ys[NC];
    deriv<NC>(p, y, k1);
#pragma unroll
    for (int i = 0; i < NC; ++i) ys[i] = y[i] + hf * A21 * k1[i];
    deriv<NC>(p, ys, k2);
#pragma unroll
    for (int i = 0; i < NC; ++i) ys[i] = y[i] + hf * (A31 * k1[i] + A32 * k2[i]);
    deriv<NC>(p, ys, k3);
#pragma unroll
    for (int i = 0; i < NC; ++i) ys[i] = y[i] + hf * (A41 * k1[i] + A42 * k2[i] + A43 * k3[i]);
    deriv<NC>(p, ys, k4);
#pragma unroll
    for (int i = 0; i < NC; ++i) ys[i] = y[i] + hf * (A51 * k1[i] + A52 * k2[i] + A53 * k3[i] + A54 * k4[i]);
    deriv<NC>(p, ys, k5);
#pragma unroll
    for (int i = 0; i < NC; ++i)
      ys[i] = y[i] + hf * (A61 * k1[i] + A62 * k2[i] + A63 * k3[i] + A64 * k4[i] + A65 * k5[i]);
    deriv<NC>(p, ys, k6);
    float y5[NC], er[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      y5[i] = y[i] + hf * (B1 * k1[i] + B3 * k3[i] + B4 * k4[i] + B6 * k6[i]);
      er[i] = hf * (E1 * k1[i] + E3 * k3[i] + E4 * k4[i] + E5 * k5[i] + E6 * k6[i]);
    }
    float emax = ratio_of(er[0], y[0], hf * k1[0], 1.0f);
    emax = fmaxf(emax, ratio_of(er[1], y[1], hf * k1[1], 1.0f));
#pragma unroll
    for (int i = 2; i < NC; ++i) emax = fmaxf(emax, ratio_of(er[i], y[i], hf * k1[i], 1e-3f));
    // error ratio emax / tol <= 1 in the control precision CT; the FP32
    // product rf differs from it by at most 2.4e-7 relative, so it decides
    // alone outside [0.999999, 1.000001] (same decision, fewer FP64 operations)
    const float rf = __fmul_rn(emax, p.inv_tol_f);
    bool within;
    if (rf <= 0.999999f) within = true;
    else if (rf > 1.000001f) within = false;
    else within = (CT)emax * (CT)p.inv_tol <= (CT)1;
    ++nsub;
    ++n;
    const bool cap = n >= p.max_sub;
    if (within || !ctl_lt(h_min, h) || cap) {  // h <= h_min
#pragma unroll
      for (int i = 0; i < NC; ++i) y[i] = y5[i];
      if (y[0] >= p.V_peak) {
        y[0] = p.V_reset;
        y[1] = y[1] + p.b;
        ++nspk;
      }
      float grow = 5.0f;
      if (rf > 0.0f) grow = fminf(5.0f, __fmul_rn(0.9f, step_factor_root<5>(rf)));
      h = h * (CT)grow;
      if (ctl_lt(h, h_min)) h = h_min;
      if (cap && !last) cap_hit = true;
      if (last || cap) return true;
      t_in = t_next;
      rem = rem_next;
    } else {
      const float shrink = fmaxf(0.1f, __fmul_rn(0.9f, step_factor_root<4>(rf)));
      h = h * (CT)shrink;
      if (ctl_lt(h, h_min)) h = h_min;
    }
    if (--budget == 0) return false;
  }
}

// Progress of one neuron inside a step: the step-size proposal, the time
// reached and the attempts made (FP64; FP32 control keeps FP32 values in them).
struct RkPos {
  double h, t_in;
  int64_t n;
};

template <int NC>
__device__ __forceinline__ bool aeif_integrate_nc(const AeifSeg& p, St& s, RkPos& r, int budget, uint32_t& nspk,
                                                  unsigned long long& nsub, bool& cap_hit) {
  float y[NC];
  y[0] = s.V;
  y[1] = s.w;
  y[2] = s.ge;
  y[3] = s.gi;
  if constexpr (NC == 6) {
    y[4] = s.xe;
    y[5] = s.xi;
  } else if constexpr (NC == 10) {
    y[4] = s.g2;
    y[5] = s.g3;
    y[6] = s.xe;
    y[7] = s.xi;
    y[8] = s.x2;
    y[9] = s.x3;
  }
  bool done;
  if (p.ctl32) {
    float hf = (float)r.h, tf = (float)r.t_in;
    done = aeif_integrate_t<float, NC>(p, y, hf, tf, r.n, budget, nspk, nsub, cap_hit);
    r.h = (double)hf;
    r.t_in = (double)tf;
  } else {
    done = aeif_integrate_t<double, NC>(p, y, r.h, r.t_in, r.n, budget, nspk, nsub, cap_hit);
  }
  s.V = y[0];
  s.w = y[1];
  s.ge = y[2];
  s.gi = y[3];
  if constexpr (NC == 6) {
    s.xe = y[4];
    s.xi = y[5];
  } else if constexpr (NC == 10) {
    s.g2 = y[4];
    s.g3 = y[5];
    s.xe = y[6];
    s.xi = y[7];
    s.x2 = y[8];
    s.x3 = y[9];
  }
  return done;
}

// The step's input on the receptors (in.x .. in.w: ports 0-3), after the
// integration: a conductance jump (exponential), or x += W e / tau (alpha),
// or x += W g0 (beta, g0 making the peak of g equal to W).
template <int kM>
__device__ __forceinline__ void aeif_add_input(const AeifSeg& p, St& s, float4 in) {
  if (kM == kAeifBeta) {
    s.xe = __fadd_rn(s.xe, __fmul_rn(in.x, p.jmp_p[0]));
    s.xi = __fadd_rn(s.xi, __fmul_rn(in.y, p.jmp_p[1]));
    s.x2 = __fadd_rn(s.x2, __fmul_rn(in.z, p.jmp_p[2]));
    s.x3 = __fadd_rn(s.x3, __fmul_rn(in.w, p.jmp_p[3]));
  } else if (kM == kAeifAlpha) {
    s.xe = __fadd_rn(s.xe, __fmul_rn(in.x, p.e_tau_ex));
    s.xi = __fadd_rn(s.xi, __fmul_rn(in.y, p.e_tau_in));
  } else {
    s.ge = __fadd_rn(s.ge, in.x);
    s.gi = __fadd_rn(s.gi, in.y);
  }
}

// Integrate one AdEx neuron over (the rest of) a step with at most `budget`
// attempts (0: no limit); on completion the step's input is added.  Returns
// whether the step is complete.  kM selects the conductance model.
template <int kM>
__device__ __forceinline__ bool aeif_advance(const AeifSeg& p, St& s, RkPos& r, int budget, float4 in,
                                             uint32_t& nspk, unsigned long long& nsub, bool& cap_hit) {
  const bool done = aeif_integrate_nc<kAeifNC<kM>>(p, s, r, budget, nspk, nsub, cap_hit);
  if (done) aeif_add_input<kM>(p, s, in);
  return done;
}

// A whole step (no attempt budget) of the two-receptor models.
template <int kM>
__device__ __forceinline__ void aeif_step(const AeifSeg& p, St& s, double& h, float in0, float in1, uint32_t& nspk,
                                          unsigned long long& nsub, bool& cap_hit) {
  RkPos r{h, 0.0, 0};
  aeif_advance<kM>(p, s, r, 0, make_float4(in0, in1, 0.f, 0.f), nspk, nsub, cap_hit);
  h = r.h;
}

}  // namespace ngb
