// ngb_oracle.cpp -- plain, slow CPU oracle of the spiking-network hot path.
//
// TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's
// CPU-baseline leg may load this file's library.  It shares no code with the
// GPU library; every step below is written from the method's definition:
//
//   * LIF with exponential PSCs (Eqs. 1-2), integrated by exact integration
//     on the dt grid (Sec. 2.1, "The NeuronGPU library", after Rotter &
//     Diesmann 1999).
//   * AdEx with conductance synapses (Eqs. 3-5), integrated by an embedded
//     fifth-order Runge-Kutta method with adaptive step size (Sec. 2.1);
//     the tableau is the published Cash-Karp (1990) one.
//   * Poisson generators as the external drive (Sec. 2.1, devices).
//   * Connections by the rules of Sec. 2.1 (fixed indegree, fixed total
//     number, fixed outdegree, one-to-one, all-to-all), grouped per source by
//     delay (Sec. 2.2).
//   * Spike delivery: a spike of neuron s at step t adds each synapse weight
//     to its target's input at step t + delay, once (Sec. 2.2).
//
// Readings where the paper is silent or garbled (summation index of Eq. 2,
// sign of Eq. 4, step order, RNG layout, delay rounding, ...) are the ones
// listed in the design notes; each is restated next to the code using it.
// Parity status: see ngb_oracle.h.
//
// Build with -ffp-contract=off: FP32 expressions are evaluated op by op with
// round-to-nearest, in the order written.

#include "ngb_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

namespace {

thread_local std::string g_err;

int32_t fail(const std::string& m) {
  g_err = m;
  return -1;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies whose high
// halves are xored into the other two words together with the round key; the
// key is bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
void philox(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
  uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
  for (int round = 0; round < 10; ++round) {
    const uint64_t prod0 = (uint64_t)kMul0 * (uint64_t)x0;
    const uint64_t prod1 = (uint64_t)kMul1 * (uint64_t)x2;
    const uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    const uint32_t y1 = (uint32_t)prod1;
    const uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    const uint32_t y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Counter layout (design reading "RNG layout"): key = (seed low, seed high);
// counter = (index low, index high, purpose | attempt << 8, stream).
enum Purpose : uint32_t { kSrc = 1, kWeight = 2, kDelay = 3, kPoisson = 4, kVinit = 5 };

void draw(uint64_t seed, uint64_t index, uint32_t purpose, uint32_t attempt, uint32_t stream,
          uint32_t out[4]) {
  const uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), purpose | (attempt << 8), stream};
  philox(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), out);
}

// Uniform integer in [0, n): high half of the 64-bit product x * n.
uint32_t uniform_index(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * n) >> 32); }

// Uniform double in (0, 1] from two words: the top 53 bits, plus one, times 2^-53.
double uniform53(uint32_t hi, uint32_t lo) {
  const uint64_t bits = (((uint64_t)hi << 32) | lo) >> 11;
  return (double)(bits + 1) * 0x1p-53;
}

// Standard normal by the Box-Muller transform (cosine branch).
double normal_from(const uint32_t w[4]) {
  const double two_pi = 6.283185307179586;
  const double u1 = uniform53(w[0], w[1]);
  const double u2 = uniform53(w[2], w[3]);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
}

// Poisson(lambda) by inversion: the smallest k with u < F(k), u = x * 2^-32,
// F accumulated term by term from p0 = exp(-lambda), p_k = p_{k-1} * lambda / k.
const int kPoissonKmax = 255;
int poisson_inversion(double lambda, uint32_t x) {
  const double u = (double)x * 0x1p-32;
  double p = std::exp(-lambda);
  double F = p;
  int k = 0;
  while (u >= F && k < kPoissonKmax) {
    k += 1;
    p = p * lambda / (double)k;
    F = F + p;
  }
  return k;
}

// Exact-integration propagators of Eqs. 1-2 over one step h (y = V - E_L):
//   y(t+h) = P22 y + P21 I + P20 I_e,  I(t+h) = P11 I.
void lif_propagators(double tau_m, double C, double tau_s, double h, double P[4]) {
  const double P11 = std::exp(-h / tau_s);
  const double P22 = std::exp(-h / tau_m);
  double P21;
  if (tau_m == tau_s) {
    P21 = h / C * P22;
  } else {
    P21 = tau_m * tau_s / (C * (tau_m - tau_s)) * (std::expm1(-h / tau_m) - std::expm1(-h / tau_s));
  }
  const double P20 = -tau_m / C * std::expm1(-h / tau_m);
  P[0] = P11; P[1] = P21; P[2] = P22; P[3] = P20;
}

// Cash & Karp (1990) embedded 4(5) Runge-Kutta tableau.
struct Tableau {
  double c[6];
  double a[6][6];
  double b5[6];
  double b4[6];
};
Tableau cash_karp() {
  Tableau t;
  std::memset(&t, 0, sizeof(t));
  const double c[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
  for (int i = 0; i < 6; ++i) t.c[i] = c[i];
  t.a[1][0] = 1.0 / 5.0;
  t.a[2][0] = 3.0 / 40.0;        t.a[2][1] = 9.0 / 40.0;
  t.a[3][0] = 3.0 / 10.0;        t.a[3][1] = -9.0 / 10.0;   t.a[3][2] = 6.0 / 5.0;
  t.a[4][0] = -11.0 / 54.0;      t.a[4][1] = 5.0 / 2.0;     t.a[4][2] = -70.0 / 27.0;
  t.a[4][3] = 35.0 / 27.0;
  t.a[5][0] = 1631.0 / 55296.0;  t.a[5][1] = 175.0 / 512.0; t.a[5][2] = 575.0 / 13824.0;
  t.a[5][3] = 44275.0 / 110592.0; t.a[5][4] = 253.0 / 4096.0;
  const double b5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
  const double b4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                        277.0 / 14336.0, 1.0 / 4.0};
  for (int i = 0; i < 6; ++i) { t.b5[i] = b5[i]; t.b4[i] = b4[i]; }
  return t;
}

// Round an FP32 weight to the storage precision and back (round to nearest,
// ties to even).  prec 1 = bfloat16 (8-bit exponent, 7 stored mantissa bits),
// prec 2 = IEEE binary16 (5-bit exponent, 10 mantissa bits, subnormals).
float round_weight(float w, int prec) {
  if (prec == 0) return w;
  if (prec == 1) {
    uint32_t bits;
    std::memcpy(&bits, &w, 4);
    const uint32_t lsb = (bits >> 16) & 1u;
    bits += 0x7FFFu + lsb;
    bits &= 0xFFFF0000u;
    float r;
    std::memcpy(&r, &bits, 4);
    return r;
  }
  // binary16: quantum of the binade of |w| (never below the subnormal quantum 2^-24)
  const double v = (double)w;
  if (v == 0.0) return w;
  int e2;
  std::frexp(std::fabs(v), &e2);        // |v| = m * 2^e2, m in [0.5, 1)
  int exponent = e2 - 1;                // floor(log2 |v|)
  if (exponent < -14) exponent = -14;   // subnormal range shares the 2^-24 quantum
  const double quantum = std::ldexp(1.0, exponent - 10);
  double r = std::nearbyint(v / quantum) * quantum;
  if (std::fabs(r) >= 65520.0) r = std::copysign(INFINITY, v);
  return (float)r;
}

// ---------------------------------------------------------------------------
// Network description
// ---------------------------------------------------------------------------
struct LifPar {
  double tau_m, C_m, E_L, V_reset, V_th, t_ref, tau_syn, I_e, V0_mean, V0_sd;
  double pn, prate, pw;
  int precv;
};
struct AeifPar {
  double C_m, g_L, E_L, V_T, Delta_T, a, b, tau_w, V_peak, V_reset, E_ex, E_in, tau_ex, tau_in, I_e;
  double V0_mean, V0_sd, w0, tol, h_min, h_init;
  int64_t max_sub;
  double pn, prate, pw;
  int prec_rcpt;
  int fp64;
  // synaptic ports: exponential (model 1) and alpha (model 2) use two, (E_ex, tau_ex) and
  // (E_in, tau_in); the beta multisynapse model (3) up to four with their own E, rise and decay
  int n_ports;
  double E[4], tau_r[4], tau_d[4];
  double g0[4];  // jump of x per unit input weight: the peak of g equals the weight
};

struct Population {
  int model;          // 0 LIF, 1 AdEx
  int instance;
  int64_t n;
  int64_t offset;     // first global neuron id
  int64_t local_off;  // first instance-local neuron id
  LifPar lif;
  AeifPar aeif;
  // derived
  double lambda;      // Poisson mean per step
  float P11, P21, P22, P20Ie, theta, y_reset, w_ext;
  int ref_steps;
};

struct Instance {
  uint64_t seed;
  int64_t n;
  uint32_t n_calls;
};

struct Call {
  int src_pop, tgt_pop, rule, autapses, wdist, ddist, receptor;
  int64_t K;
  double w0, w1, d0, d1;
  uint32_t stream;  // connect-call index within the instance
  int stdp;         // 0: static synapses; k > 0: plastic with STDP rule k - 1
};

struct Synapse {
  uint32_t src, tgt;
  float w;
  uint16_t delay;
  uint8_t receptor;
  uint8_t stdp;
};

// Nearest-neighbour spike-timing-dependent plasticity (Sec. 2.1, after
// Morrison et al. 2008), with the weight dependence of Guetig et al. (2003).
// A spike of the source reaches the synapse `delay` steps after it was fired
// (its arrival step a).  At every arrival the weight is depressed by the
// target's latest spike p < a, and at every spike of the target at step p
// the weight is potentiated by the synapse's latest arrival a <= p
// (symmetric nearest-neighbour pairing; lags n in steps, time n * dt):
//   potentiation  w <- w + lambda W_max (1 - w / W_max)^mu_plus e^(-n dt / tau_plus)
//   depression    w <- w - alpha lambda W_max (w / W_max)^mu_minus e^(-n dt / tau_minus)
// each followed by clipping to [0, W_max].  A lag beyond 20 tau changes
// nothing (the factor e^-20 is below FP32 resolution next to the weight).
// The weight a spike delivers is the weight after the depression of its
// arrival.  Arithmetic in FP32, the exponentials tabulated in FP64 and
// rounded once.
struct StdpRule {
  float A_plus, A_minus, inv_W_max, W_max, mu_plus, mu_minus;
  std::vector<float> k_plus, k_minus;  // e^(-n dt / tau) for lags n = 0 .. 20 tau / dt
};

float stdp_power(float x, float mu) {
  if (mu == 0.0f) return 1.0f;
  if (mu == 1.0f) return x;
  return std::pow(std::max(x, 0.0f), mu);
}

float stdp_clip(float w, float W_max) { return std::min(std::max(w, 0.0f), W_max); }

float stdp_potentiate(const StdpRule& r, float w, int64_t lag) {
  if (lag < 0 || lag >= (int64_t)r.k_plus.size()) return w;
  const float f = stdp_power(1.0f - w * r.inv_W_max, r.mu_plus);
  return stdp_clip(w + (r.A_plus * f) * r.k_plus[(size_t)lag], r.W_max);
}

float stdp_depress(const StdpRule& r, float w, int64_t lag) {
  if (lag < 0 || lag >= (int64_t)r.k_minus.size()) return w;
  const float f = stdp_power(w * r.inv_W_max, r.mu_minus);
  return stdp_clip(w - (r.A_minus * f) * r.k_minus[(size_t)lag], r.W_max);
}

}  // namespace

struct ora_net {
  double dt;
  int prec;
  int deterministic;
  int track_abs;
  std::vector<Instance> inst;
  std::vector<Population> pops;
  std::vector<Call> calls;
  bool finalized = false;
  int64_t N = 0;
  // canonical CSR, source-major, ordered by (source, delay, call, draw index)
  std::vector<uint64_t> src_ptr;
  std::vector<uint32_t> tgt;
  std::vector<uint8_t> rcpt;
  std::vector<float> w;
  std::vector<uint16_t> delay;
  std::vector<uint8_t> plast;  // STDP rule + 1 of each synapse (0: static)
  int max_delay = 1;
  // STDP: rules, the latest arrival step of every synapse (-1: none), the
  // latest spike step of every neuron (-1: none), the plastic synapses of
  // every target (in_ptr[N+1] into in_syn), and the spike multiplicities of
  // the last max_delay + 1 steps (hist[(step mod H) * N + neuron])
  std::vector<StdpRule> stdp;
  std::vector<int64_t> arrival, last_spike;
  std::vector<uint64_t> in_ptr, in_syn;
  std::vector<int> hist;
  bool plastic = false;
  int64_t L = 2;
  int R = 1;
  // per-neuron state (double arrays; FP32 models keep float-representable values)
  std::vector<double> s0, s1, s2, s3, s4;  // LIF: y, I, ref | AdEx: V, w, gex, gin, h
  std::vector<double> s5, s6;              // AdEx alpha / beta: x of ports 0, 1
  std::vector<double> s7, s8, s9, s10;     // AdEx beta: g of ports 2, 3, x of ports 2, 3
  std::vector<int> pop_of;
  // ring[(slot * R + r) * N + i]
  std::vector<float> ring;
  std::vector<int64_t> ring_fx;
  std::vector<double> ring_abs, ring_exact;
  int64_t t = 0;
  int64_t events = 0;
  int64_t rk_substeps = 0;
  int64_t rk_cap_hits = 0;  // steps whose sub-step count reached the cap
  std::vector<int64_t> spk_id, spk_step;
};

namespace {

const double kFixScale = 4294967296.0;  // 2^32: fixed-point ring of the deterministic mode
const uint32_t kMaxAttempts = 10000;    // cap of every re-draw loop

uint16_t delay_steps(double d_ms, double dt) {
  double s = std::nearbyint(d_ms / dt);  // round half to even
  if (s < 1.0) s = 1.0;
  if (s > 4095.0) s = 4095.0;
  return (uint16_t)s;
}

// Draw the weight of one synapse (draw index q of call c), re-drawing a
// normal sample until its sign equals the sign of the mean.
double draw_weight(const ora_net* net, const Call& c, uint64_t seed, uint64_t q) {
  (void)net;
  if (c.wdist == 0) return c.w0;
  for (uint32_t attempt = 0;; ++attempt) {
    if (attempt == kMaxAttempts) return c.w0;  // re-draws exhausted: the mean
    uint32_t r[4];
    draw(seed, q, kWeight, attempt, c.stream, r);
    if (c.wdist == 1) {
      const double v = c.w0 + c.w1 * normal_from(r);
      if (c.w0 > 0.0 && !(v > 0.0)) continue;
      if (c.w0 < 0.0 && !(v < 0.0)) continue;
      return v;
    }
    return c.w0 + (c.w1 - c.w0) * uniform53(r[0], r[1]);
  }
}

// Draw the delay (ms) of one synapse; a normal delay is re-drawn until >= dt.
double draw_delay(const ora_net* net, const Call& c, uint64_t seed, uint64_t q) {
  if (c.ddist == 0) return c.d0;
  for (uint32_t attempt = 0;; ++attempt) {
    if (attempt == kMaxAttempts) return std::max(c.d0, net->dt);  // re-draws exhausted
    uint32_t r[4];
    draw(seed, q, kDelay, attempt, c.stream, r);
    if (c.ddist == 1) {
      const double v = c.d0 + c.d1 * normal_from(r);
      if (v < net->dt) continue;
      return v;
    }
    return c.d0 + (c.d1 - c.d0) * uniform53(r[0], r[1]);
  }
}

// Synapse of draw index q of connect call c (Sec. 2.1 connection rules).
Synapse draw_synapse(const ora_net* net, const Call& c, uint64_t q) {
  const Population& ps = net->pops[c.src_pop];
  const Population& pt = net->pops[c.tgt_pop];
  const uint64_t seed = net->inst[ps.instance].seed;
  const bool same = (c.src_pop == c.tgt_pop);
  uint32_t src = 0, tgt = 0;
  if (c.rule == 3) {
    // one-to-one: source i -> target i, no draw
    src = tgt = (uint32_t)q;
  } else if (c.rule == 4) {
    // all-to-all: pairs in target-major order, (i, i) left out without autapses
    const uint64_t per_target = (same && !c.autapses) ? (uint64_t)ps.n - 1 : (uint64_t)ps.n;
    tgt = (uint32_t)(q / per_target);
    src = (uint32_t)(q % per_target);
    if (same && !c.autapses && src >= tgt) src += 1;
  } else {
    for (uint32_t attempt = 0;; ++attempt) {
      uint32_t r[4];
      draw(seed, q, kSrc, attempt, c.stream, r);
      if (attempt == kMaxAttempts) break;  // keep the last draw (needs a population of one)
      if (c.rule == 0) {
        // fixed indegree: draw q belongs to target q / K
        tgt = (uint32_t)(q / (uint64_t)c.K);
        src = uniform_index(r[0], (uint32_t)ps.n);
      } else if (c.rule == 2) {
        // fixed outdegree: draw q belongs to source q / K
        src = (uint32_t)(q / (uint64_t)c.K);
        tgt = uniform_index(r[0], (uint32_t)pt.n);
      } else {
        src = uniform_index(r[0], (uint32_t)ps.n);
        tgt = uniform_index(r[1], (uint32_t)pt.n);
      }
      if (same && !c.autapses && src == tgt) continue;
      break;
    }
  }
  Synapse s;
  s.src = (uint32_t)(ps.offset + src);
  s.tgt = (uint32_t)(pt.offset + tgt);
  s.w = round_weight((float)draw_weight(net, c, seed, q), net->prec);
  s.delay = delay_steps(draw_delay(net, c, seed, q), net->dt);
  s.receptor = (uint8_t)c.receptor;
  s.stdp = (uint8_t)c.stdp;
  return s;
}

// Synapses of connect call c: K per target, K in all, K per source, one per
// source, or one per (source, target) pair (Sec. 2.1 connection rules).
uint64_t call_size(const ora_net* net, const Call& c) {
  const uint64_t ns = (uint64_t)net->pops[c.src_pop].n, nt = (uint64_t)net->pops[c.tgt_pop].n;
  switch (c.rule) {
    case 0: return (uint64_t)c.K * nt;
    case 2: return (uint64_t)c.K * ns;
    case 3: return ns;
    case 4: return (c.src_pop == c.tgt_pop && !c.autapses) ? ns * (ns - 1) : ns * nt;
    default: return (uint64_t)c.K;
  }
}

void generate(const ora_net* net, const Call& c, std::vector<Synapse>& out) {
  const uint64_t nsyn = call_size(net, c);
  for (uint64_t q = 0; q < nsyn; ++q) out.push_back(draw_synapse(net, c, q));
}

// The AdEx system (Eqs. 3-5) with the synaptic conductances as state:
// y = {V, w, g_0 .. g_3, x_0 .. x_3} for up to four synaptic ports (unused
// ports stay 0).  Exponential conductances (model 1): g' = -g / tau.
// Alpha-function conductances (model 2, the paper's balanced network, Sec.
// 2.4): g(t) = W (t/tau) e^(1 - t/tau) after a spike of weight W, generated
// by g' = x - g/tau, x' = -x/tau with x jumping by W e / tau at the spike.
// Beta-function conductances (model 3, the multisynapse model of the paper's
// interface example, Sec. 2.1): g' = x - g/tau_decay, x' = -x/tau_rise, x
// jumping by W g0 with g0 chosen so that the peak of g equals W.
constexpr int kAdexN = 10;
constexpr double kEuler = 2.718281828459045;  // e

template <typename T>
struct AdexSystem {
  T g_L, E_L, V_T, Delta_T, inv_Delta_T, a, inv_tau_w, V_peak, I_e, inv_C;
  int n_ports;
  bool rise;  // alpha / beta: g driven by x
  T E[4], inv_tau_r[4], inv_tau_d[4];
  void deriv(const T y[kAdexN], T f[kAdexN]) const {
    const T V = std::min(y[0], V_peak);  // the exponential is evaluated at most at V_peak
    const T I_spike = (Delta_T > T(0)) ? g_L * Delta_T * std::exp((V - V_T) * inv_Delta_T) : T(0);
    // reading of Eq. 4: I_syn = sum_i g_i (E_rev,i - V), so excitation depolarises
    T I_syn = T(0);
    for (int k = 0; k < n_ports; ++k) I_syn = I_syn + y[2 + k] * (E[k] - V);
    f[0] = (-g_L * (V - E_L) + I_spike + I_syn - y[1] + I_e) * inv_C;
    f[1] = (a * (V - E_L) - y[1]) * inv_tau_w;
    for (int k = 0; k < 4; ++k) {
      if (k >= n_ports) {
        f[2 + k] = T(0);
        f[6 + k] = T(0);
      } else if (rise) {
        f[2 + k] = y[6 + k] - y[2 + k] * inv_tau_d[k];
        f[6 + k] = -y[6 + k] * inv_tau_r[k];
      } else {
        f[2 + k] = -y[2 + k] * inv_tau_d[k];
        f[6 + k] = T(0);
      }
    }
  }
};

template <typename T>
AdexSystem<T> adex_system(const AeifPar& q, int model) {
  AdexSystem<T> s;
  s.g_L = T(q.g_L);
  s.E_L = T(q.E_L);
  s.V_T = T(q.V_T);
  s.Delta_T = T(q.Delta_T);
  s.inv_Delta_T = T(1.0 / q.Delta_T);
  s.a = T(q.a);
  s.inv_tau_w = T(1.0 / q.tau_w);
  s.V_peak = T(q.V_peak);
  s.I_e = T(q.I_e);
  s.inv_C = T(1.0 / q.C_m);
  s.n_ports = q.n_ports;
  s.rise = model != 1;
  for (int k = 0; k < 4; ++k) {
    s.E[k] = T(q.E[k]);
    s.inv_tau_r[k] = T(1.0 / q.tau_r[k]);
    s.inv_tau_d[k] = T(1.0 / q.tau_d[k]);
  }
  return s;
}

// Jump of x per unit weight so that g peaks at the weight: e / tau for equal
// rise and decay, else (1/tau_r - 1/tau_d) / (e^(-t_p/tau_d) - e^(-t_p/tau_r))
// with the time of the peak t_p = tau_d tau_r ln(tau_d / tau_r) / (tau_d - tau_r).
double beta_normalisation(double tau_r, double tau_d) {
  if (tau_r == tau_d) return kEuler / tau_d;
  const double tp = tau_d * tau_r * std::log(tau_d / tau_r) / (tau_d - tau_r);
  return (1.0 / tau_r - 1.0 / tau_d) / (std::exp(-tp / tau_d) - std::exp(-tp / tau_r));
}

// One embedded Cash-Karp step from y over h: the fifth-order solution in y5
// and its difference to the fourth-order one in err.
template <typename T>
void ck_step(const AdexSystem<T>& sys, const Tableau& tab, const T y[kAdexN], const T f0[kAdexN], double h,
             T y5[kAdexN], T err[kAdexN]) {
  T k[6][kAdexN];
  for (int i = 0; i < kAdexN; ++i) k[0][i] = f0[i];
  for (int s = 1; s < 6; ++s) {
    T ys[kAdexN];
    for (int i = 0; i < kAdexN; ++i) {
      T acc = T(0);
      for (int j = 0; j < s; ++j) acc += T(tab.a[s][j]) * k[j][i];
      ys[i] = y[i] + T(h) * acc;
    }
    sys.deriv(ys, k[s]);
  }
  for (int i = 0; i < kAdexN; ++i) {
    T acc5 = T(0), accd = T(0);
    for (int s = 0; s < 6; ++s) {
      acc5 += T(tab.b5[s]) * k[s][i];
      accd += T(tab.b5[s] - tab.b4[s]) * k[s][i];
    }
    y5[i] = y[i] + T(h) * acc5;
    err[i] = T(h) * accd;
  }
}

// Step-size factor of the FP32-state integration: r^(-1/k) for k = 5 (after
// an accepted sub-step) or k = 4 (after a rejected one), defined as a fixed
// sequence of FP32 operations so that the GPU path, which follows the same
// definition, produces the same bits.  The definition: write r = m 2^e with
// m in [1, 2) and e = k q + s, 0 <= s < k; then
//   r^(-1/k) = 2^(-q) * (c(m - 1) * K_k[s]),  K_k[s] = 2^(-s/k) rounded to FP32,
// with c the cubic below (least-squares fit of m^(-1/k) on [1, 2), relative
// error < 2e-4), evaluated by Horner's rule with fused multiply-adds.  Ratios
// below 2^-100 give 2^20 and ratios of 2^100 and above (or not finite) give 0;
// both are then clamped by the caller.
float step_factor_root(float r, int k) {
  if (!(r < 0x1p100f)) return 0.0f;
  if (r < 0x1p-100f) return 0x1p20f;
  uint32_t bits;
  std::memcpy(&bits, &r, 4);
  const int e = (int)((bits >> 23) & 0xffu) - 127;
  const uint32_t mbits = (bits & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &mbits, 4);
  const float t = m - 1.0f;  // exact
  int q = e / k;
  if (e < 0 && q * k != e) q -= 1;  // floor division
  const int s = e - q * k;
  float c, ks;
  if (k == 5) {
    static const float K5[5] = {0x1p+0f, 0x1.bdb8cep-1f, 0x1.8406p-1f, 0x1.51cb46p-1f, 0x1.261118p-1f};
    c = std::fma(std::fma(std::fma(-0x1.ae3294p-6f, t, 0x1.78f37cp-4f), t, -0x1.8fb646p-3f), t, 0x1.ffed6cp-1f);
    ks = K5[s];
  } else {
    static const float K4[4] = {0x1p+0f, 0x1.ae89fap-1f, 0x1.6a09e6p-1f, 0x1.306fep-1f};
    c = std::fma(std::fma(std::fma(-0x1.18bd56p-5f, t, 0x1.e6677ep-4f), t, -0x1.f2b6f8p-3f), t, 0x1.ffe6dcp-1f);
    ks = K4[s];
  }
  const uint32_t pbits = (uint32_t)(127 - q) << 23;  // 2^(-q), |q| <= 20
  float p2;
  std::memcpy(&p2, &pbits, 4);
  return (c * ks) * p2;
}

// Integrate one AdEx neuron over one step dt (adaptive step size, error
// relative to |y| + |h f| + floor, safety factor 0.9, growth exponent -1/5,
// shrink exponent -1/4, growth at most 5x, shrink at most 10x), resetting
// V -> V_reset and w -> w + b after every accepted sub-step that ends with
// V >= V_peak.  Returns the number of spikes; h carries the proposed step.
// The FP64 reference (T = double) tests emax / tol <= 1 and takes the factors
// with pow in FP64.  The FP32-state replica (T = float) follows the GPU's
// step control: the test (double)emax * (1 / tol) <= 1 in FP64, and the
// factors 0.9 * step_factor_root(r) in FP32 with r = emax * (float)(1 / tol).
template <typename T>
int adex_advance(const AdexSystem<T>& sys, const Tableau& tab, const AeifPar& p, double dt, double tol,
                 T y[kAdexN], double& h, int64_t& substeps, int64_t& cap_hits) {
  const T floor_[kAdexN] = {T(1.0), T(1.0), T(1e-3), T(1e-3), T(1e-3), T(1e-3), T(1e-3), T(1e-3), T(1e-3),
                            T(1e-3)};
  int spikes = 0;
  double t_in = 0.0;
  int64_t n = 0;
  if (!(h > 0.0)) h = p.h_init;
  for (;;) {
    const double rem = dt - t_in;
    bool last = false;
    if (h >= rem) {
      h = rem;
      last = true;
    }
    T f0[kAdexN], y5[kAdexN], err[kAdexN];
    sys.deriv(y, f0);
    ck_step(sys, tab, y, f0, h, y5, err);
    T emax = T(0);
    for (int i = 0; i < kAdexN; ++i) {
      const T scale = std::fabs(y[i]) + std::fabs(T(h) * f0[i]) + floor_[i];
      const T r = std::fabs(err[i]) / scale;
      if (r > emax) emax = r;
    }
    constexpr bool replica = std::is_same<T, float>::value;
    const double ratio = replica ? (double)emax * (1.0 / tol) : (double)emax / tol;
    const float rf = (float)emax * (float)(1.0 / tol);
    ++n;
    if (ratio <= 1.0 || h <= p.h_min || n >= p.max_sub) {
      for (int i = 0; i < kAdexN; ++i) y[i] = y5[i];
      if (y[0] >= T(p.V_peak)) {
        y[0] = T(p.V_reset);
        y[1] = y[1] + T(p.b);
        ++spikes;
      }
      double grow = 5.0;
      if (replica) {
        if (rf > 0.0f) grow = (double)std::min(5.0f, 0.9f * step_factor_root(rf, 5));
      } else if (ratio > 0.0) {
        grow = std::min(5.0, 0.9 * std::pow(ratio, -0.2));
      }
      const double h_used = h;
      h = std::max(h * grow, p.h_min);
      if (n >= p.max_sub && !last) cap_hits += 1;
      if (last || n >= p.max_sub) break;
      t_in += h_used;
    } else {
      const double shrink = replica ? (double)std::max(0.1f, 0.9f * step_factor_root(rf, 4))
                                    : std::max(0.1, 0.9 * std::pow(ratio, -0.25));
      h = std::max(h * shrink, p.h_min);
    }
  }
  substeps += n;
  return spikes;
}

float fx_to_float(int64_t v) { return (float)((double)v / kFixScale); }

int64_t ring_index(const ora_net* net, int64_t step, int r, int64_t i) {
  return ((step % net->L) * net->R + r) * net->N + i;
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface
// ---------------------------------------------------------------------------
extern "C" {

const char* ora_last_error(void) { return g_err.c_str(); }

ora_net* ora_create(double dt_ms, uint64_t seed, int32_t weight_prec, int32_t deterministic,
                    int32_t track_abs) {
  if (!(dt_ms > 0.0) || weight_prec < 0 || weight_prec > 2) {
    fail("ora_create: invalid dt or weight precision");
    return nullptr;
  }
  ora_net* net = new ora_net();
  net->dt = dt_ms;
  net->prec = weight_prec;
  net->deterministic = deterministic ? 1 : 0;
  net->track_abs = track_abs ? 1 : 0;
  net->inst.push_back(Instance{seed, 0, 0});
  return net;
}

void ora_destroy(ora_net* net) { delete net; }

int32_t ora_add_instance(ora_net* net, uint64_t seed) {
  if (!net || net->finalized) return fail("ora_add_instance: bad state");
  net->inst.push_back(Instance{seed, 0, 0});
  return (int32_t)net->inst.size() - 1;
}

int32_t ora_add_population(ora_net* net, int32_t instance, int32_t model, int64_t n, const double* p) {
  if (!net || net->finalized) return fail("ora_add_population: bad state");
  if (instance < 0 || instance >= (int32_t)net->inst.size()) return fail("ora_add_population: instance");
  if (n <= 0 || n > 0x7FFFFFFF || model < 0 || model > 3) return fail("ora_add_population: n/model");
  Population P;
  std::memset(&P, 0, sizeof(P));
  P.model = model;
  P.instance = instance;
  P.n = n;
  P.offset = net->N;
  P.local_off = net->inst[instance].n;
  const double dt = net->dt;
  if (model == 0) {
    LifPar& q = P.lif;
    q.tau_m = p[0]; q.C_m = p[1]; q.E_L = p[2]; q.V_reset = p[3]; q.V_th = p[4]; q.t_ref = p[5];
    q.tau_syn = p[6]; q.I_e = p[7]; q.V0_mean = p[8]; q.V0_sd = p[9];
    q.pn = p[10]; q.prate = p[11]; q.pw = p[12]; q.precv = (int)p[13];
    if (!(q.tau_m > 0 && q.C_m > 0 && q.tau_syn > 0 && q.t_ref >= 0)) return fail("ora: LIF params");
    double Pv[4];
    lif_propagators(q.tau_m, q.C_m, q.tau_syn, dt, Pv);
    P.P11 = (float)Pv[0];
    P.P21 = (float)Pv[1];
    P.P22 = (float)Pv[2];
    P.P20Ie = (float)(Pv[3] * q.I_e);
    P.theta = (float)(q.V_th - q.E_L);
    P.y_reset = (float)(q.V_reset - q.E_L);
    P.ref_steps = (int)std::nearbyint(q.t_ref / dt);
    P.lambda = q.pn * q.prate * dt * 1e-3;
    P.w_ext = (float)q.pw;
  } else {
    AeifPar& q = P.aeif;
    q.C_m = p[0]; q.g_L = p[1]; q.E_L = p[2]; q.V_T = p[3]; q.Delta_T = p[4]; q.a = p[5]; q.b = p[6];
    q.tau_w = p[7]; q.V_peak = p[8]; q.V_reset = p[9]; q.E_ex = p[10]; q.E_in = p[11];
    q.tau_ex = p[12]; q.tau_in = p[13]; q.I_e = p[14]; q.V0_mean = p[15]; q.V0_sd = p[16];
    q.w0 = p[17]; q.tol = p[18]; q.h_min = p[19]; q.h_init = p[20]; q.max_sub = (int64_t)p[21];
    q.pn = p[22]; q.prate = p[23]; q.pw = p[24]; q.prec_rcpt = (int)p[25]; q.fp64 = (int)p[26];
    if (!(q.C_m > 0 && q.tau_w > 0 && q.tau_ex > 0 && q.tau_in > 0 && q.tol > 0 && q.h_min > 0 &&
          q.h_init > 0 && q.max_sub > 0))
      return fail("ora: AdEx params");
    if (model == 3) {
      // beta multisynapse: p[27] ports, p[28..31] E_rev, p[32..35] tau_rise, p[36..39] tau_decay
      q.n_ports = (int)p[27];
      if (q.n_ports < 1 || q.n_ports > 4) return fail("ora: beta ports");
      for (int k = 0; k < 4; ++k) {
        q.E[k] = k < q.n_ports ? p[28 + k] : 0.0;
        q.tau_r[k] = k < q.n_ports ? p[32 + k] : 1.0;
        q.tau_d[k] = k < q.n_ports ? p[36 + k] : 1.0;
        if (!(q.tau_r[k] > 0 && q.tau_d[k] > 0)) return fail("ora: beta time constants");
        q.g0[k] = beta_normalisation(q.tau_r[k], q.tau_d[k]);
      }
    } else {
      q.n_ports = 2;
      q.E[0] = q.E_ex;
      q.E[1] = q.E_in;
      q.tau_r[0] = q.tau_d[0] = q.tau_ex;
      q.tau_r[1] = q.tau_d[1] = q.tau_in;
      q.E[2] = q.E[3] = 0.0;
      q.tau_r[2] = q.tau_r[3] = q.tau_d[2] = q.tau_d[3] = 1.0;
      for (int k = 0; k < 4; ++k) q.g0[k] = kEuler / q.tau_d[k];
    }
    if (q.prec_rcpt < 0 || q.prec_rcpt >= q.n_ports) return fail("ora: Poisson receptor");
    P.lambda = q.pn * q.prate * dt * 1e-3;
    P.w_ext = (float)q.pw;
    net->R = std::max(net->R, std::max(2, q.n_ports));
  }
  if (!(P.lambda >= 0.0 && P.lambda <= 100.0)) return fail("ora: Poisson mean per step must be in [0,100]");
  net->pops.push_back(P);
  net->N += n;
  net->inst[instance].n += n;
  return (int32_t)net->pops.size() - 1;
}

int32_t ora_connect(ora_net* net, int32_t src_pop, int32_t tgt_pop, int32_t rule, int64_t K,
                    int32_t allow_autapses, int32_t wdist, double w0, double w1, int32_t ddist, double d0,
                    double d1, int32_t receptor) {
  if (!net || net->finalized) return fail("ora_connect: bad state");
  const int32_t np = (int32_t)net->pops.size();
  if (src_pop < 0 || src_pop >= np || tgt_pop < 0 || tgt_pop >= np) return fail("ora_connect: pop");
  if (net->pops[src_pop].instance != net->pops[tgt_pop].instance) return fail("ora_connect: instances");
  if (K < 0 || rule < 0 || rule > 4) return fail("ora_connect: rule/K");
  if (rule == 3 && (net->pops[src_pop].n != net->pops[tgt_pop].n || (src_pop == tgt_pop && !allow_autapses)))
    return fail("ora_connect: one-to-one sizes");
  if (receptor < 0 || receptor > 3) return fail("ora_connect: receptor");
  {
    const Population& pt = net->pops[tgt_pop];
    const int ports = pt.model == 0 ? 1 : pt.aeif.n_ports;
    if (receptor >= ports) return fail("ora_connect: receptor beyond the target's synaptic ports");
  }
  if (src_pop == tgt_pop && !allow_autapses && net->pops[src_pop].n < 2 && K > 0)
    return fail("ora_connect: no admissible source without autapses");
  Instance& I = net->inst[net->pops[src_pop].instance];
  Call c{src_pop, tgt_pop, rule, allow_autapses ? 1 : 0, wdist, ddist, receptor, K, w0, w1, d0, d1, I.n_calls, 0};
  I.n_calls += 1;
  net->calls.push_back(c);
  return (int32_t)net->calls.size() - 1;
}

int32_t ora_set_stdp(ora_net* net, int32_t call, const double* p) {
  if (!net || net->finalized || call < 0 || call >= (int32_t)net->calls.size() || !p)
    return fail("ora_set_stdp: bad state or call");
  const double tau_plus = p[0], tau_minus = p[1], lambda = p[2], alpha = p[3], mu_plus = p[4], mu_minus = p[5],
               W_max = p[6];
  if (!(tau_plus > 0 && tau_minus > 0 && lambda >= 0 && alpha >= 0 && mu_plus >= 0 && mu_minus >= 0 && W_max > 0))
    return fail("ora_set_stdp: parameters");
  if (net->stdp.size() >= 15) return fail("ora_set_stdp: at most 15 rules");
  StdpRule r;
  r.A_plus = (float)(lambda * W_max);
  r.A_minus = (float)(alpha * lambda * W_max);
  r.inv_W_max = (float)(1.0 / W_max);
  r.W_max = (float)W_max;
  r.mu_plus = (float)mu_plus;
  r.mu_minus = (float)mu_minus;
  const int64_t n_plus = (int64_t)std::floor(20.0 * tau_plus / net->dt) + 1;
  const int64_t n_minus = (int64_t)std::floor(20.0 * tau_minus / net->dt) + 1;
  for (int64_t n = 0; n < n_plus; ++n) r.k_plus.push_back((float)std::exp(-(double)n * net->dt / tau_plus));
  for (int64_t n = 0; n < n_minus; ++n) r.k_minus.push_back((float)std::exp(-(double)n * net->dt / tau_minus));
  net->stdp.push_back(r);
  net->calls[(size_t)call].stdp = (int)net->stdp.size();
  return 0;
}

int32_t ora_finalize(ora_net* net) {
  if (!net) return fail("ora_finalize: null");
  if (net->finalized) return 0;
  const int64_t N = net->N;
  // 1. all synapses in (call, draw index) order
  std::vector<Synapse> syn;
  uint64_t total = 0;
  for (const Call& c : net->calls) total += call_size(net, c);
  syn.reserve((size_t)total);
  for (const Call& c : net->calls) generate(net, c, syn);
  // 2. stable counting sort by (source, delay): canonical CSR order
  int maxd = 1;
  for (const Synapse& s : syn) maxd = std::max<int>(maxd, s.delay);
  const int64_t D = maxd + 1;
  std::vector<uint64_t> bucket((size_t)(N * D + 1), 0);
  for (const Synapse& s : syn) bucket[(size_t)(s.src * D + s.delay) + 1] += 1;
  for (size_t b = 1; b < bucket.size(); ++b) bucket[b] += bucket[b - 1];
  const size_t K = syn.size();
  net->tgt.assign(K, 0);
  net->rcpt.assign(K, 0);
  net->w.assign(K, 0.0f);
  net->delay.assign(K, 0);
  net->plast.assign(K, 0);
  for (const Synapse& s : syn) {
    const size_t pos = (size_t)bucket[(size_t)(s.src * D + s.delay)]++;
    net->tgt[pos] = s.tgt;
    net->rcpt[pos] = s.receptor;
    net->w[pos] = s.w;
    net->delay[pos] = s.delay;
    net->plast[pos] = s.stdp;
  }
  net->src_ptr.assign((size_t)N + 1, 0);
  for (const Synapse& s : syn) net->src_ptr[(size_t)s.src + 1] += 1;
  for (int64_t i = 0; i < N; ++i) net->src_ptr[(size_t)i + 1] += net->src_ptr[(size_t)i];
  std::vector<Synapse>().swap(syn);
  net->max_delay = maxd;
  net->L = maxd + 1;
  // STDP bookkeeping: incoming plastic synapses of every target, in CSR order
  net->plastic = false;
  for (size_t j = 0; j < K; ++j) net->plastic = net->plastic || net->plast[j] != 0;
  if (net->plastic) {
    net->arrival.assign(K, -1);
    net->last_spike.assign((size_t)N, -1);
    net->in_ptr.assign((size_t)N + 1, 0);
    for (size_t j = 0; j < K; ++j)
      if (net->plast[j]) net->in_ptr[(size_t)net->tgt[j] + 1] += 1;
    for (int64_t i = 0; i < N; ++i) net->in_ptr[(size_t)i + 1] += net->in_ptr[(size_t)i];
    net->in_syn.assign((size_t)net->in_ptr[(size_t)N], 0);
    std::vector<uint64_t> cur(net->in_ptr.begin(), net->in_ptr.end() - 1);
    for (size_t j = 0; j < K; ++j)
      if (net->plast[j]) net->in_syn[(size_t)cur[(size_t)net->tgt[j]]++] = j;
    net->hist.assign((size_t)((maxd + 1) * N), 0);
  }
  // 3. state
  net->s0.assign((size_t)N, 0.0); net->s1.assign((size_t)N, 0.0); net->s2.assign((size_t)N, 0.0);
  net->s3.assign((size_t)N, 0.0); net->s4.assign((size_t)N, 0.0);
  net->s5.assign((size_t)N, 0.0); net->s6.assign((size_t)N, 0.0);
  net->s7.assign((size_t)N, 0.0); net->s8.assign((size_t)N, 0.0);
  net->s9.assign((size_t)N, 0.0); net->s10.assign((size_t)N, 0.0);
  net->pop_of.assign((size_t)N, 0);
  for (size_t pi = 0; pi < net->pops.size(); ++pi) {
    const Population& P = net->pops[pi];
    const uint64_t seed = net->inst[P.instance].seed;
    for (int64_t k = 0; k < P.n; ++k) {
      const int64_t i = P.offset + k;
      net->pop_of[(size_t)i] = (int)pi;
      const double mean = P.model == 0 ? P.lif.V0_mean : P.aeif.V0_mean;
      const double sd = P.model == 0 ? P.lif.V0_sd : P.aeif.V0_sd;
      double V0 = mean;
      if (sd != 0.0) {
        uint32_t r[4];
        draw(seed, (uint64_t)(P.local_off + k), kVinit, 0, 0, r);
        V0 = mean + sd * normal_from(r);
      }
      if (P.model == 0) {
        net->s0[(size_t)i] = (double)(float)(V0 - P.lif.E_L);
      } else {
        const bool f64 = P.aeif.fp64 != 0;
        net->s0[(size_t)i] = f64 ? V0 : (double)(float)V0;
        net->s1[(size_t)i] = f64 ? P.aeif.w0 : (double)(float)P.aeif.w0;
        net->s4[(size_t)i] = P.aeif.h_init;
      }
    }
  }
  const size_t ring_sz = (size_t)(net->L * net->R * N);
  if (net->deterministic) net->ring_fx.assign(ring_sz, 0);
  else net->ring.assign(ring_sz, 0.0f);
  if (net->track_abs) {
    net->ring_abs.assign(ring_sz, 0.0);
    net->ring_exact.assign(ring_sz, 0.0);
  }
  net->finalized = true;
  return 0;
}

int32_t ora_simulate(ora_net* net, int64_t steps) {
  if (!net) return fail("ora_simulate: null");
  if (!net->finalized) {
    const int32_t rc = ora_finalize(net);
    if (rc < 0) return rc;
  }
  const Tableau tab = cash_karp();
  const int64_t N = net->N;
  std::vector<int64_t> fired;
  std::vector<int> mult;
  for (int64_t s = 0; s < steps; ++s) {
    const int64_t t = net->t;
    fired.clear();
    mult.clear();
    // --- update of every neuron with the input of step t (Eqs. 1-5)
    for (size_t pi = 0; pi < net->pops.size(); ++pi) {
      const Population& P = net->pops[pi];
      const uint64_t seed = net->inst[P.instance].seed;
      for (int64_t k = 0; k < P.n; ++k) {
        const int64_t i = P.offset + k;
        float in[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int r = 0; r < net->R; ++r) {
          const int64_t idx = ring_index(net, t, r, i);
          if (net->deterministic) {
            in[r] = fx_to_float(net->ring_fx[(size_t)idx]);
            net->ring_fx[(size_t)idx] = 0;
          } else {
            in[r] = net->ring[(size_t)idx];
            net->ring[(size_t)idx] = 0.0f;
          }
          if (net->track_abs) {
            net->ring_abs[(size_t)idx] = 0.0;
            net->ring_exact[(size_t)idx] = 0.0;
          }
        }
        // Poisson drive of step t: k ~ Poisson(lambda), adds k * w_ext; the uniform word of
        // instance-local step t is word t mod 4 of the Philox block with index t div 4
        if (P.lambda > 0.0) {
          uint32_t r[4];
          draw(seed, (uint64_t)t >> 2, kPoisson, 0, (uint32_t)(P.local_off + k), r);
          const int kp = poisson_inversion(P.lambda, r[(uint64_t)t & 3u]);
          const int rc = P.model == 0 ? 0 : P.aeif.prec_rcpt;
          const float add = (float)kp * P.w_ext;
          in[rc] = in[rc] + add;
        }
        int nspk = 0;
        if (P.model == 0) {
          float y = (float)net->s0[(size_t)i];
          float I = (float)net->s1[(size_t)i];
          int ref = (int)net->s2[(size_t)i];
          if (ref > 0) {
            ref -= 1;  // absolute refractory: V is held at V_reset
          } else {
            y = P.P22 * y + P.P21 * I + P.P20Ie;  // propagate V with the current of the previous grid point
          }
          I = P.P11 * I + in[0];                  // input of step t enters after the V propagation
          if (y >= P.theta) {
            y = P.y_reset;
            ref = P.ref_steps;
            nspk = 1;
          }
          net->s0[(size_t)i] = y;
          net->s1[(size_t)i] = I;
          net->s2[(size_t)i] = ref;
        } else {
          const AeifPar& q = P.aeif;
          const bool rise = P.model != 1;
          double h = net->s4[(size_t)i];
          const size_t u = (size_t)i;
          if (q.fp64) {
            const AdexSystem<double> sys = adex_system<double>(q, P.model);
            double y[kAdexN] = {net->s0[u], net->s1[u], net->s2[u], net->s3[u], net->s7[u],
                                net->s8[u], net->s5[u], net->s6[u], net->s9[u], net->s10[u]};
            nspk = adex_advance<double>(sys, tab, q, net->dt, q.tol, y, h, net->rk_substeps, net->rk_cap_hits);
            // input of step t: a conductance jump (exponential), or a jump of x by W g0 (alpha, beta)
            for (int k = 0; k < q.n_ports; ++k) {
              if (rise) y[6 + k] += (double)in[k] * q.g0[k];
              else y[2 + k] += (double)in[k];
            }
            net->s0[u] = y[0]; net->s1[u] = y[1]; net->s2[u] = y[2]; net->s3[u] = y[3]; net->s7[u] = y[4];
            net->s8[u] = y[5]; net->s5[u] = y[6]; net->s6[u] = y[7]; net->s9[u] = y[8]; net->s10[u] = y[9];
          } else {
            const AdexSystem<float> sys = adex_system<float>(q, P.model);
            float y[kAdexN] = {(float)net->s0[u], (float)net->s1[u], (float)net->s2[u], (float)net->s3[u],
                               (float)net->s7[u], (float)net->s8[u], (float)net->s5[u], (float)net->s6[u],
                               (float)net->s9[u], (float)net->s10[u]};
            const double tol_eff = std::max(q.tol, 8.0 * 0x1p-24);
            nspk = adex_advance<float>(sys, tab, q, net->dt, tol_eff, y, h, net->rk_substeps, net->rk_cap_hits);
            for (int k = 0; k < q.n_ports; ++k) {
              if (rise) y[6 + k] = y[6 + k] + in[k] * (float)q.g0[k];
              else y[2 + k] = y[2 + k] + in[k];
            }
            net->s0[u] = y[0]; net->s1[u] = y[1]; net->s2[u] = y[2]; net->s3[u] = y[3]; net->s7[u] = y[4];
            net->s8[u] = y[5]; net->s5[u] = y[6]; net->s6[u] = y[7]; net->s9[u] = y[8]; net->s10[u] = y[9];
            h = (double)(float)h;  // the step-size proposal is carried in FP32 between steps
          }
          net->s4[(size_t)i] = h;
        }
        if (nspk > 0) {
          fired.push_back(i);
          mult.push_back(nspk);
        }
      }
    }
    // --- STDP: the targets that fired potentiate their plastic inputs with
    // the latest arrival of each (arrivals up to step t are recorded)
    if (net->plastic) {
      for (size_t f = 0; f < fired.size(); ++f) {
        const int64_t i = fired[f];
        net->last_spike[(size_t)i] = t;
        for (uint64_t k = net->in_ptr[(size_t)i]; k < net->in_ptr[(size_t)i + 1]; ++k) {
          const uint64_t j = net->in_syn[(size_t)k];
          if (net->arrival[(size_t)j] < 0) continue;
          const StdpRule& r = net->stdp[(size_t)net->plast[(size_t)j] - 1];
          net->w[(size_t)j] = stdp_potentiate(r, net->w[(size_t)j], t - net->arrival[(size_t)j]);
        }
      }
    }
    // --- delivery of the spikes of step t to the inputs of step t + delay (Sec. 2.2);
    // plastic synapses deliver when the spike arrives (below)
    for (size_t f = 0; f < fired.size(); ++f) {
      const int64_t src = fired[f];
      for (int m = 0; m < mult[f]; ++m) {
        net->spk_id.push_back(src);
        net->spk_step.push_back(t);
        for (uint64_t j = net->src_ptr[(size_t)src]; j < net->src_ptr[(size_t)src + 1]; ++j) {
          if (net->plastic && net->plast[j]) continue;
          const int64_t idx = ring_index(net, t + net->delay[j], net->rcpt[j], net->tgt[j]);
          if (net->deterministic)
            net->ring_fx[(size_t)idx] += (int64_t)std::llrint((double)net->w[j] * kFixScale);
          else
            net->ring[(size_t)idx] = net->ring[(size_t)idx] + net->w[j];
          if (net->track_abs) {
            net->ring_abs[(size_t)idx] += std::fabs((double)net->w[j]);
            net->ring_exact[(size_t)idx] += (double)net->w[j];
          }
        }
        net->events += (int64_t)(net->src_ptr[(size_t)src + 1] - net->src_ptr[(size_t)src]);
      }
    }
    // --- STDP: spikes reaching their plastic synapses at step t + 1 (fired at
    // step t + 1 - delay) depress them by the target's latest spike, then
    // deliver the depressed weight into the input of step t + 1
    if (net->plastic) {
      const int64_t H = net->max_delay + 1;
      int* row = net->hist.data() + (size_t)((t % H) * N);
      std::fill(row, row + N, 0);
      for (size_t f = 0; f < fired.size(); ++f) row[fired[f]] = mult[f];
      const int64_t a = t + 1;
      for (int64_t src = 0; src < N; ++src) {
        for (uint64_t j = net->src_ptr[(size_t)src]; j < net->src_ptr[(size_t)src + 1]; ++j) {
          if (!net->plast[j]) continue;
          const int64_t fired_at = a - net->delay[j];
          if (fired_at < 0) continue;
          const int m = net->hist[(size_t)((fired_at % H) * N + src)];
          if (m == 0) continue;
          const StdpRule& r = net->stdp[(size_t)net->plast[j] - 1];
          const int64_t post = net->last_spike[(size_t)net->tgt[j]];
          if (post >= 0) net->w[j] = stdp_depress(r, net->w[j], a - post);
          net->arrival[j] = a;
          const int64_t idx = ring_index(net, a, net->rcpt[j], net->tgt[j]);
          for (int k = 0; k < m; ++k) {
            if (net->deterministic)
              net->ring_fx[(size_t)idx] += (int64_t)std::llrint((double)net->w[j] * kFixScale);
            else
              net->ring[(size_t)idx] = net->ring[(size_t)idx] + net->w[j];
            if (net->track_abs) {
              net->ring_abs[(size_t)idx] += std::fabs((double)net->w[j]);
              net->ring_exact[(size_t)idx] += (double)net->w[j];
            }
          }
        }
      }
    }
    net->t += 1;
  }
  (void)N;
  return 0;
}

int32_t ora_inject(ora_net* net, int64_t neuron, int32_t receptor, int64_t step_offset, double value) {
  if (!net || !net->finalized) return fail("ora_inject: finalize first");
  if (neuron < 0 || neuron >= net->N || receptor < 0 || receptor >= net->R || step_offset < 0 ||
      step_offset >= net->L)
    return fail("ora_inject: range");
  const int64_t idx = ring_index(net, net->t + step_offset, receptor, neuron);
  if (net->deterministic) net->ring_fx[(size_t)idx] += (int64_t)std::llrint(value * kFixScale);
  else net->ring[(size_t)idx] = net->ring[(size_t)idx] + (float)value;
  if (net->track_abs) {
    net->ring_abs[(size_t)idx] += std::fabs(value);
    net->ring_exact[(size_t)idx] += value;
  }
  return 0;
}

int64_t ora_num_neurons(const ora_net* net) { return net ? net->N : -1; }
int64_t ora_pop_offset(const ora_net* net, int32_t pop) {
  if (!net || pop < 0 || pop >= (int32_t)net->pops.size()) return -1;
  return net->pops[pop].offset;
}
int64_t ora_num_synapses(const ora_net* net) { return net ? (int64_t)net->tgt.size() : -1; }
int64_t ora_ring_length(const ora_net* net) { return net ? net->L : -1; }
int64_t ora_steps_done(const ora_net* net) { return net ? net->t : -1; }
int64_t ora_events(const ora_net* net) { return net ? net->events : -1; }
int64_t ora_num_spikes(const ora_net* net) { return net ? (int64_t)net->spk_id.size() : -1; }
int64_t ora_rk_substeps(const ora_net* net) { return net ? net->rk_substeps : -1; }
int64_t ora_rk_cap_hits(const ora_net* net) { return net ? net->rk_cap_hits : -1; }

int32_t ora_get_csr(const ora_net* net, uint64_t* src_ptr, uint32_t* tgt, uint8_t* receptor, float* weight,
                    uint16_t* delay) {
  if (!net || !net->finalized) return fail("ora_get_csr: finalize first");
  const size_t K = net->tgt.size();
  if (src_ptr) std::memcpy(src_ptr, net->src_ptr.data(), net->src_ptr.size() * sizeof(uint64_t));
  if (tgt) std::memcpy(tgt, net->tgt.data(), K * sizeof(uint32_t));
  if (receptor) std::memcpy(receptor, net->rcpt.data(), K);
  if (weight) std::memcpy(weight, net->w.data(), K * sizeof(float));
  if (delay) std::memcpy(delay, net->delay.data(), K * sizeof(uint16_t));
  return 0;
}

int32_t ora_get_state(const ora_net* net, int32_t var, double* out) {
  if (!net || !net->finalized) return fail("ora_get_state: finalize first");
  for (int64_t i = 0; i < net->N; ++i) {
    const Population& P = net->pops[(size_t)net->pop_of[(size_t)i]];
    double v = 0.0;
    if (P.model == 0) {
      if (var == 0) v = net->s0[(size_t)i] + P.lif.E_L;
      else if (var == 1) v = net->s1[(size_t)i];
      else if (var == 4) v = net->s2[(size_t)i];
    } else {
      if (var == 0) v = net->s0[(size_t)i];
      else if (var == 1) v = net->s1[(size_t)i];
      else if (var == 2) v = net->s2[(size_t)i];
      else if (var == 3) v = net->s3[(size_t)i];
      else if (var == 5) v = net->s4[(size_t)i];
      else if (var == 6) v = net->s5[(size_t)i];
      else if (var == 7) v = net->s6[(size_t)i];
      else if (var == 8) v = net->s7[(size_t)i];   // beta: g of port 2
      else if (var == 9) v = net->s8[(size_t)i];   // g of port 3
      else if (var == 10) v = net->s9[(size_t)i];  // x of port 2
      else if (var == 11) v = net->s10[(size_t)i]; // x of port 3
    }
    out[i] = v;
  }
  return 0;
}

int32_t ora_get_input(const ora_net* net, int32_t receptor, int64_t step_offset, float* out, double* abs_out,
                      double* exact_out) {
  if (!net || !net->finalized) return fail("ora_get_input: finalize first");
  if (receptor < 0 || receptor >= net->R || step_offset < 0 || step_offset >= net->L)
    return fail("ora_get_input: range");
  for (int64_t i = 0; i < net->N; ++i) {
    const int64_t idx = ring_index(net, net->t + step_offset, receptor, i);
    if (out) out[i] = net->deterministic ? fx_to_float(net->ring_fx[(size_t)idx]) : net->ring[(size_t)idx];
    if (abs_out) abs_out[i] = net->track_abs ? net->ring_abs[(size_t)idx] : 0.0;
    if (exact_out) exact_out[i] = net->track_abs ? net->ring_exact[(size_t)idx] : 0.0;
  }
  return 0;
}

int32_t ora_get_spikes(const ora_net* net, int64_t* ids, int64_t* steps) {
  if (!net) return fail("ora_get_spikes: null");
  const size_t n = net->spk_id.size();
  if (ids) std::memcpy(ids, net->spk_id.data(), n * sizeof(int64_t));
  if (steps) std::memcpy(steps, net->spk_step.data(), n * sizeof(int64_t));
  return 0;
}

int64_t ora_rows_for_sources(const ora_net* net, int64_t n_src, const int64_t* srcs, int64_t cap,
                             uint32_t* src_out, uint32_t* tgt, uint8_t* receptor, float* weight, uint16_t* delay) {
  if (!net) return fail("ora_rows_for_sources: null");
  std::vector<int64_t> want(srcs, srcs + n_src);
  std::sort(want.begin(), want.end());
  std::vector<Synapse> rows;
  for (const Call& c : net->calls) {
    const Population& ps = net->pops[c.src_pop];
    const auto lo = std::lower_bound(want.begin(), want.end(), ps.offset);
    const auto hi = std::lower_bound(want.begin(), want.end(), ps.offset + ps.n);
    if (lo == hi) continue;
    const uint64_t nsyn = call_size(net, c);
    const uint64_t seed = net->inst[ps.instance].seed;
    for (uint64_t q = 0; q < nsyn; ++q) {
      // cheap pre-test on the source (first draw of the random-source rules); the full draw decides
      bool maybe = true;
      if (c.rule == 0 || c.rule == 1) {
        uint32_t r[4];
        draw(seed, q, kSrc, 0, c.stream, r);
        const int64_t s0 = ps.offset + uniform_index(r[0], (uint32_t)ps.n);
        maybe = std::binary_search(lo, hi, s0) || (c.src_pop == c.tgt_pop && !c.autapses);
      } else if (c.rule == 2) {
        maybe = std::binary_search(lo, hi, ps.offset + (int64_t)(q / (uint64_t)c.K));
      }
      if (!maybe) continue;
      const Synapse syn = draw_synapse(net, c, q);
      if (std::binary_search(lo, hi, (int64_t)syn.src)) rows.push_back(syn);
    }
  }
  std::stable_sort(rows.begin(), rows.end(), [](const Synapse& a, const Synapse& b) {
    if (a.src != b.src) return a.src < b.src;
    return a.delay < b.delay;
  });
  const int64_t n = (int64_t)rows.size();
  for (int64_t i = 0; i < n && i < cap; ++i) {
    if (src_out) src_out[i] = rows[(size_t)i].src;
    if (tgt) tgt[i] = rows[(size_t)i].tgt;
    if (receptor) receptor[i] = rows[(size_t)i].receptor;
    if (weight) weight[i] = rows[(size_t)i].w;
    if (delay) delay[i] = rows[(size_t)i].delay;
  }
  return n;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox(ctr, key[0], key[1], out);
}
int32_t ora_poisson_inversion(double lambda, uint32_t x) { return poisson_inversion(lambda, x); }
void ora_lif_propagators(double tau_m, double C_m, double tau_syn, double h, double out[4]) {
  lif_propagators(tau_m, C_m, tau_syn, h, out);
}
void ora_cash_karp_tableau(double c[6], double a[36], double b5[6], double b4[6]) {
  const Tableau t = cash_karp();
  for (int i = 0; i < 6; ++i) {
    c[i] = t.c[i];
    b5[i] = t.b5[i];
    b4[i] = t.b4[i];
    for (int j = 0; j < 6; ++j) a[i * 6 + j] = t.a[i][j];
  }
}
float ora_round_weight(float w, int32_t prec) { return round_weight(w, prec); }
double ora_normal_from_words(const uint32_t w[4]) { return normal_from(w); }
float ora_step_factor_root(float r, int32_t k) { return (k == 4 || k == 5) ? step_factor_root(r, k) : 0.0f; }

}  // extern "C"
