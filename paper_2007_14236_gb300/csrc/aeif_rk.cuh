// aeif_rk.cuh -- adaptive embedded Runge-Kutta integration of one AdEx neuron
// with exponential conductances over one step (Sec. 2.1; Eqs. 3-5), shared by
// the per-step AdEx kernel and the persistent step kernel.
//
// Cash & Karp (1990) 4(5) tableau; FP32 state and stages; the step size h,
// the time inside the step and the error-ratio test in FP64.  The error of
// component i is taken relative to |y_i| + |h f_i| + floor_i; accepted
// steps grow h by min(5, 0.9 r^-1/5), rejected ones shrink it by
// max(0.1, 0.9 r^-1/4); h >= h_min is always accepted.  After every
// accepted sub-step ending at V >= V_peak: V -> V_reset, w -> w + b, and
// the spike is counted (the exponential term uses min(V, V_peak)).
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

struct St {
  float V, w, ge, gi;
};

__device__ __forceinline__ St deriv(const AeifSeg& p, St y) {
  const float V = fminf(y.V, p.V_peak);
  const float I_spk = (p.Delta_T > 0.0f) ? p.g_L * p.Delta_T * expf((V - p.V_T) * p.inv_Delta_T) : 0.0f;
  const float I_syn = y.ge * (p.E_ex - V) + y.gi * (p.E_in - V);
  St f;
  f.V = (-p.g_L * (V - p.E_L) + I_spk + I_syn - y.w + p.I_e) * p.inv_C;
  f.w = (p.a * (V - p.E_L) - y.w) * p.inv_tau_w;
  f.ge = -y.ge * p.inv_tau_ex;
  f.gi = -y.gi * p.inv_tau_in;
  return f;
}

__device__ __forceinline__ St axpy(St y, float h, St k) {
  return St{y.V + h * k.V, y.w + h * k.w, y.ge + h * k.ge, y.gi + h * k.gi};
}

__device__ __forceinline__ float ratio_of(float err, float y, float hf, float fl) {
  return fabsf(err) / (fabsf(y) + fabsf(hf) + fl);
}

// Integrate y over one step of p.dt; h carries the step-size proposal in
// and out.  Adds the sub-steps to nsub and the spikes to nspk; cap_hit is set
// when the sub-step cap ended the step early.  CT is the precision of the
// step-size control (h, time inside the step, error-ratio test).
template <typename CT>
__device__ __forceinline__ void aeif_integrate_t(const AeifSeg& p, St& y, CT& h, uint32_t& nspk,
                                                 unsigned long long& nsub, bool& cap_hit) {
  const CT dt = (CT)p.dt, h_min = (CT)p.h_min;
  if (!(h > (CT)0)) h = dt;
  CT t_in = (CT)0;
  int64_t n = 0;  // sub-steps of this step (the cap applies per neuron and step)
  for (;;) {
    const CT rem = dt - t_in;
    bool last = false;
    if (h >= rem) {
      h = rem;
      last = true;
    }
    const float hf = (float)h;
    const St k1 = deriv(p, y);
    const St k2 = deriv(p, axpy(y, hf * A21, k1));
    St ys;
    ys = St{y.V + hf * (A31 * k1.V + A32 * k2.V), y.w + hf * (A31 * k1.w + A32 * k2.w),
            y.ge + hf * (A31 * k1.ge + A32 * k2.ge), y.gi + hf * (A31 * k1.gi + A32 * k2.gi)};
    const St k3 = deriv(p, ys);
    ys = St{y.V + hf * (A41 * k1.V + A42 * k2.V + A43 * k3.V), y.w + hf * (A41 * k1.w + A42 * k2.w + A43 * k3.w),
            y.ge + hf * (A41 * k1.ge + A42 * k2.ge + A43 * k3.ge),
            y.gi + hf * (A41 * k1.gi + A42 * k2.gi + A43 * k3.gi)};
    const St k4 = deriv(p, ys);
    ys = St{y.V + hf * (A51 * k1.V + A52 * k2.V + A53 * k3.V + A54 * k4.V),
            y.w + hf * (A51 * k1.w + A52 * k2.w + A53 * k3.w + A54 * k4.w),
            y.ge + hf * (A51 * k1.ge + A52 * k2.ge + A53 * k3.ge + A54 * k4.ge),
            y.gi + hf * (A51 * k1.gi + A52 * k2.gi + A53 * k3.gi + A54 * k4.gi)};
    const St k5 = deriv(p, ys);
    ys = St{y.V + hf * (A61 * k1.V + A62 * k2.V + A63 * k3.V + A64 * k4.V + A65 * k5.V),
            y.w + hf * (A61 * k1.w + A62 * k2.w + A63 * k3.w + A64 * k4.w + A65 * k5.w),
            y.ge + hf * (A61 * k1.ge + A62 * k2.ge + A63 * k3.ge + A64 * k4.ge + A65 * k5.ge),
            y.gi + hf * (A61 * k1.gi + A62 * k2.gi + A63 * k3.gi + A64 * k4.gi + A65 * k5.gi)};
    const St k6 = deriv(p, ys);
    const St y5{y.V + hf * (B1 * k1.V + B3 * k3.V + B4 * k4.V + B6 * k6.V),
                y.w + hf * (B1 * k1.w + B3 * k3.w + B4 * k4.w + B6 * k6.w),
                y.ge + hf * (B1 * k1.ge + B3 * k3.ge + B4 * k4.ge + B6 * k6.ge),
                y.gi + hf * (B1 * k1.gi + B3 * k3.gi + B4 * k4.gi + B6 * k6.gi)};
    const St er{hf * (E1 * k1.V + E3 * k3.V + E4 * k4.V + E5 * k5.V + E6 * k6.V),
                hf * (E1 * k1.w + E3 * k3.w + E4 * k4.w + E5 * k5.w + E6 * k6.w),
                hf * (E1 * k1.ge + E3 * k3.ge + E4 * k4.ge + E5 * k5.ge + E6 * k6.ge),
                hf * (E1 * k1.gi + E3 * k3.gi + E4 * k4.gi + E5 * k5.gi + E6 * k6.gi)};
    float emax = ratio_of(er.V, y.V, hf * k1.V, 1.0f);
    emax = fmaxf(emax, ratio_of(er.w, y.w, hf * k1.w, 1.0f));
    emax = fmaxf(emax, ratio_of(er.ge, y.ge, hf * k1.ge, 1e-3f));
    emax = fmaxf(emax, ratio_of(er.gi, y.gi, hf * k1.gi, 1e-3f));
    const CT ratio = (CT)emax * (CT)p.inv_tol;
    ++nsub;
    ++n;
    const bool cap = n >= p.max_sub;
    if (ratio <= (CT)1 || h <= h_min || cap) {
      y = y5;
      if (y.V >= p.V_peak) {
        y.V = p.V_reset;
        y.w = y.w + p.b;
        ++nspk;
      }
      const float rf = emax * (float)p.inv_tol;
      float grow = 5.0f;
      if (rf > 0.0f) grow = fminf(5.0f, 0.9f * exp2f(-0.2f * __log2f(rf)));
      const CT h_used = h;
      h = h * (CT)grow;
      if (h < h_min) h = h_min;
      if (cap && !last) cap_hit = true;
      if (last || cap) break;
      t_in += h_used;
    } else {
      const float shrink = fmaxf(0.1f, 0.9f * exp2f(-0.25f * __log2f(emax * (float)p.inv_tol)));
      h = h * (CT)shrink;
      if (h < h_min) h = h_min;
    }
  }
}

// FP64 step-size control by default, FP32 when the population asks for it.
__device__ __forceinline__ void aeif_integrate(const AeifSeg& p, St& y, double& h, uint32_t& nspk,
                                               unsigned long long& nsub, bool& cap_hit) {
  if (p.ctl32) {
    float hf = (float)h;
    aeif_integrate_t<float>(p, y, hf, nspk, nsub, cap_hit);
    h = (double)hf;
  } else {
    aeif_integrate_t<double>(p, y, h, nspk, nsub, cap_hit);
  }
}

}  // namespace ngb
