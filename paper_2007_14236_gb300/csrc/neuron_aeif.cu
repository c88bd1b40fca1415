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
// join the warp-ballot spike compaction with the spike multiplicity.
#include "ngb_internal.cuh"
#include "philox.cuh"

namespace ngb {

namespace {

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

}  // namespace

template <bool kFixed>
__global__ void __launch_bounds__(kAeifBlock) k_update_aeif(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const uint32_t* __restrict__ thr,
                                                            float* __restrict__ V_, float* __restrict__ w_,
                                                            float* __restrict__ ge_, float* __restrict__ gi_,
                                                            float* __restrict__ h_, Ring ring, int64_t* clk,
                                                            const uint4* __restrict__ src_meta, SpikeBuf sb) {
  __shared__ uint32_t s_thr[kMaxThr];
  const AeifSeg p = segment_of(T, (int64_t)blockIdx.x);
  const int64_t k = ((int64_t)blockIdx.x - p.blk_begin) * kAeifBlock + threadIdx.x;
  const bool valid = k < p.n;
  const uint32_t gid = (uint32_t)(p.offset + k);
  // prologue (overlaps the previous kernel): state, source metadata, Poisson table
  St y{0.f, 0.f, 0.f, 0.f};
  float h0 = 0.f;
  uint4 meta = make_uint4(0, 0, 0, 0);
  if (valid) {
    y = St{V_[gid], w_[gid], ge_[gid], gi_[gid]};
    h0 = h_[gid];
    meta = __ldg(src_meta + gid);
  }
  for (uint32_t i = threadIdx.x; i < p.n_thr; i += kAeifBlock) s_thr[i] = __ldg(thr + p.thr_off + i);
  __syncthreads();
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) clk[1] = t;
  uint32_t nspk = 0;
  unsigned long long nsub = 0;
  if (valid) {
    const uint64_t slot = (uint64_t)(t & ring.L_mask);
    const uint64_t i0 = (slot * (uint64_t)ring.R) * (uint64_t)ring.N + gid;
    const uint64_t i1 = i0 + (uint64_t)ring.N;
    float in0, in1;
    if (kFixed) {
      long long* rp = reinterpret_cast<long long*>(ring.p);
      const long long v0 = rp[i0], v1 = rp[i1];
      rp[i0] = 0;
      rp[i1] = 0;
      in0 = __double2float_rn(__dmul_rn(__ll2double_rn(v0), 2.3283064365386963e-10));
      in1 = __double2float_rn(__dmul_rn(__ll2double_rn(v1), 2.3283064365386963e-10));
    } else {
      float* rp = reinterpret_cast<float*>(ring.p);
      in0 = rp[i0];
      in1 = rp[i1];
      rp[i0] = 0.0f;
      rp[i1] = 0.0f;
    }
    if (p.n_thr > 0) {
      const int64_t tl = t - p.t0;
      const U4 r = draw4(p.seed, (uint64_t)tl, kPurPoisson, 0u, p.local_off + (uint32_t)k);
      uint32_t kp = 0;
      while (kp < p.n_thr && r.x >= s_thr[kp]) ++kp;
      const float add = __fmul_rn((float)kp, p.w_ext);
      if (p.prec_rcpt == 0) in0 = __fadd_rn(in0, add);
      else in1 = __fadd_rn(in1, add);
    }
    double h = (double)h0;
    if (!(h > 0.0)) h = p.dt;
    double t_in = 0.0;
    for (;;) {
      const double rem = p.dt - t_in;
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
      const double ratio = (double)emax * p.inv_tol;
      ++nsub;
      const bool cap = nsub >= (unsigned long long)p.max_sub;
      if (ratio <= 1.0 || h <= p.h_min || cap) {
        y = y5;
        if (y.V >= p.V_peak) {
          y.V = p.V_reset;
          y.w = y.w + p.b;
          ++nspk;
        }
        const float rf = (float)ratio;
        float grow = 5.0f;
        if (rf > 0.0f) grow = fminf(5.0f, 0.9f * exp2f(-0.2f * __log2f(rf)));
        const double h_used = h;
        h = fmax(h * (double)grow, p.h_min);
        if (cap && !last) atomicOr(sb.err, kErrSubstepCap);
        if (last || cap) break;
        t_in += h_used;
      } else {
        const float shrink = fmaxf(0.1f, 0.9f * exp2f(-0.25f * __log2f((float)ratio)));
        h = fmax(h * (double)shrink, p.h_min);
      }
    }
    y.ge = __fadd_rn(y.ge, in0);
    y.gi = __fadd_rn(y.gi, in1);
    V_[gid] = y.V;
    w_[gid] = y.w;
    ge_[gid] = y.ge;
    gi_[gid] = y.gi;
    h_[gid] = (float)h;
  }
  // sub-step statistics: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
  if ((threadIdx.x & 31) == 0 && nsub) atomicAdd(sb.substeps, nsub);
  const uint32_t mult = nspk > 63u ? 63u : nspk;
  emit_spikes(nspk > 0, gid, mult, t, meta, sb);
}

cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V,
                               float* w, float* gex, float* gin, float* h, Ring ring, bool fixed, int64_t* clk,
                               const uint4* src_meta, SpikeBuf sb, bool pdl, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks), b(kAeifBlock);
  if (fixed)
    return launch_k(k_update_aeif<true>, g, b, pdl, st, segs, thr, V, w, gex, gin, h, ring, clk, src_meta, sb);
  return launch_k(k_update_aeif<false>, g, b, pdl, st, segs, thr, V, w, gex, gin, h, ring, clk, src_meta, sb);
}

}  // namespace ngb
