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
// scans the pending spikes (as the LIF kernel).  kM: the conductance model,
// exponential, alpha (the paper's balanced network, Sec. 2.4; state x_ex,
// x_in) or the beta multisynapse model of Sec. 2.1 (up to four receptor
// ports, each with g and x; the step reads one input plane per port in use).
#include <string>

#include "aeif_rk.cuh"
#include "ngb.h"
#include "deliver_item.cuh"
#include "neuron_step.cuh"

namespace ngb {

namespace {

// uint4 words of a deferred neuron's record.
template <int kM>
constexpr int kRecWords = kM == kAeifBeta ? 6 : 4;

__device__ __forceinline__ uint32_t fu(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float uf(uint32_t x) { return __uint_as_float(x); }

template <int kM>
__device__ __forceinline__ void load_state(const AeifState& S, uint32_t gid, int n_ports, St& y, float& h) {
  y.V = S.V[gid];
  y.w = S.w[gid];
  y.ge = S.g0[gid];
  y.gi = S.g1[gid];
  if (kM != kAeifExp) {
    y.xe = S.x0[gid];
    y.xi = S.x1[gid];
  }
  if (kM == kAeifBeta && n_ports > 2) {
    y.g2 = S.ext[gid];
    y.g3 = S.ext[S.N + gid];
    y.x2 = S.ext[2 * S.N + gid];
    y.x3 = S.ext[3 * S.N + gid];
  }
  h = S.h[gid];
}

template <int kM>
__device__ __forceinline__ void store_state(const AeifState& S, uint32_t gid, int n_ports, const St& y, float h) {
  S.V[gid] = y.V;
  S.w[gid] = y.w;
  S.g0[gid] = y.ge;
  S.g1[gid] = y.gi;
  if (kM != kAeifExp) {
    S.x0[gid] = y.xe;
    S.x1[gid] = y.xi;
  }
  if (kM == kAeifBeta && n_ports > 2) {
    S.ext[gid] = y.g2;
    S.ext[S.N + gid] = y.g3;
    S.ext[2 * S.N + gid] = y.x2;
    S.ext[3 * S.N + gid] = y.x3;
  }
  S.h[gid] = h;
}

// Record of a neuron whose step is unfinished: {gid, segment, spikes so far,
// attempts}, the state, the step's input and the position inside the step.
template <int kM>
__device__ __forceinline__ void pack_rec(uint4* rec, uint32_t gid, uint32_t seg, uint32_t nspk, const St& y,
                                         const RkPos& r, float4 in) {
  const unsigned long long hb = (unsigned long long)__double_as_longlong(r.h);
  const unsigned long long tb = (unsigned long long)__double_as_longlong(r.t_in);
  const uint4 pos = make_uint4((uint32_t)hb, (uint32_t)(hb >> 32), (uint32_t)tb, (uint32_t)(tb >> 32));
  rec[0] = make_uint4(gid, seg, nspk, (uint32_t)r.n);
  rec[1] = make_uint4(fu(y.V), fu(y.w), fu(y.ge), fu(y.gi));
  if constexpr (kM == kAeifBeta) {
    rec[2] = make_uint4(fu(y.g2), fu(y.g3), fu(y.xe), fu(y.xi));
    rec[3] = make_uint4(fu(y.x2), fu(y.x3), fu(in.x), fu(in.y));
    rec[4] = make_uint4(fu(in.z), fu(in.w), 0u, 0u);
    rec[5] = pos;
  } else {
    rec[2] = make_uint4(fu(y.xe), fu(y.xi), fu(in.x), fu(in.y));
    rec[3] = pos;
  }
}

template <int kM>
__device__ __forceinline__ void unpack_rec(const uint4* q, St& y, RkPos& r, float4& in) {
  const uint4 r0 = q[0], r1 = q[1];
  const uint4 pos = q[kRecWords<kM> - 1];
  y.V = uf(r1.x);
  y.w = uf(r1.y);
  y.ge = uf(r1.z);
  y.gi = uf(r1.w);
  if constexpr (kM == kAeifBeta) {
    const uint4 r2 = q[2], r3 = q[3], r4 = q[4];
    y.g2 = uf(r2.x);
    y.g3 = uf(r2.y);
    y.xe = uf(r2.z);
    y.xi = uf(r2.w);
    y.x2 = uf(r3.x);
    y.x3 = uf(r3.y);
    in = make_float4(uf(r3.z), uf(r3.w), uf(r4.x), uf(r4.y));
  } else {
    const uint4 r2 = q[2];
    y.xe = uf(r2.x);
    y.xi = uf(r2.y);
    in = make_float4(uf(r2.z), uf(r2.w), 0.f, 0.f);
  }
  r.h = __longlong_as_double((long long)((unsigned long long)pos.x | ((unsigned long long)pos.y << 32)));
  r.t_in = __longlong_as_double((long long)((unsigned long long)pos.z | ((unsigned long long)pos.w << 32)));
  r.n = (int64_t)r0.w;
}

}  // namespace

template <bool kFixed, int kMode, int kM>
__global__ void __launch_bounds__(kAeifBlock) k_update_aeif(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const uint32_t* __restrict__ thr, const AeifState S,
                                                            Ring ring, int64_t* clk, int64_t step_off, const Csr csr,
                                                            SpikeBuf sb, int scan, int budget) {
  constexpr bool kAge = kMode == kEmitAge;
  constexpr int kW = kRecWords<kM>;
  __shared__ uint32_t s_thr[kMaxThr];
  const int seg = segment_index_of(T, (int64_t)blockIdx.x);
  const AeifSeg p = T.n <= kInlineSegs ? T.s[seg] : T.dev[seg];
  const int64_t k = ((int64_t)blockIdx.x - p.blk_begin) * kAeifBlock + threadIdx.x;
  const bool valid = k < p.n;
  const uint32_t gid = (uint32_t)(p.offset + k);
  const int n_ports = kM == kAeifBeta ? p.n_ports : 2;
  // prologue (overlaps the previous kernel): state, source metadata, Poisson table
  St y{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float h0 = 0.f;
  uint4 meta = make_uint4(0, 0, 0, 0);
  if (valid) {
    load_state<kM>(S, gid, n_ports, y, h0);
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
  uint4 rec[kW];
  if (valid) {
    const uint64_t slot = (uint64_t)(t & ring.L_mask);
    const uint64_t i0 = (slot * (uint64_t)ring.R) * (uint64_t)ring.N + gid;
    float4 in = make_float4(0.f, 0.f, 0.f, 0.f);
    in.x = ring_take<kFixed, false>(ring.p, i0);
    in.y = ring_take<kFixed, false>(ring.p, i0 + (uint64_t)ring.N);
    if (kM == kAeifBeta) {
      if (n_ports > 2) in.z = ring_take<kFixed, false>(ring.p, i0 + 2 * (uint64_t)ring.N);
      if (n_ports > 3) in.w = ring_take<kFixed, false>(ring.p, i0 + 3 * (uint64_t)ring.N);
    }
    if (p.n_thr > 0) {
      const uint32_t kp = poisson_count(p.seed, t - p.t0, p.local_off + (uint32_t)k, s_thr, p.n_thr);
      const float add = __fmul_rn((float)kp, p.w_ext);
      switch (p.prec_rcpt) {
        case 0: in.x = __fadd_rn(in.x, add); break;
        case 1: in.y = __fadd_rn(in.y, add); break;
        case 2: in.z = __fadd_rn(in.z, add); break;
        default: in.w = __fadd_rn(in.w, add); break;
      }
    }
    RkPos r{(double)h0, 0.0, 0};
    bool cap_hit = false;
    done = aeif_advance<kM>(p, y, r, budget, in, nspk, nsub, cap_hit);
    if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
    if (done) store_state<kM>(S, gid, n_ports, y, (float)r.h);
    else pack_rec<kM>(rec, gid, (uint32_t)seg, nspk, y, r, in);
  }
  defer_write<kW>(!done, rec, sb, kM, t);
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
template <bool kFixed, int kMode, int kM>
__global__ void __launch_bounds__(kAeifBlock) k_aeif_finish(const __grid_constant__ SegTable<AeifSeg> T,
                                                            const AeifState S, Ring ring, int64_t* clk,
                                                            int64_t step_off, const Csr csr, SpikeBuf sb) {
  constexpr bool kAge = kMode == kEmitAge;
  constexpr int kW = kRecWords<kM>;
  griddep_wait();
  griddep_launch();
  const int64_t t = clk[0] + step_off;
  unsigned long long n = sb.dcnt[2 * kM + (int)(t & 1)];
  if (n > (unsigned long long)sb.dfr_cap) n = (unsigned long long)sb.dfr_cap;
  // the previous step's list is finished (this stream ran its finishing kernel
  // first) and the next step appends to it only after this kernel
  if (blockIdx.x == 0 && threadIdx.x == 0) sb.dcnt[2 * kM + (int)((t + 1) & 1)] = 0;
  const uint4* __restrict__ list = sb.dfr[kM];
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
      const uint4* q = list + (unsigned long long)kW * i;
      const uint4 r0 = q[0];
      gid = r0.x;
      const AeifSeg p = T.dev[r0.y];
      nspk = r0.z;
      if (!kAge) meta = __ldg(csr.src_meta + gid);
      St y{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      RkPos r{0.0, 0.0, 0};
      float4 in;
      unpack_rec<kM>(q, y, r, in);
      bool cap_hit = false;
      aeif_advance<kM>(p, y, r, 0, in, nspk, nsub, cap_hit);
      if (cap_hit) atomicOr(sb.err, kErrSubstepCap);
      store_state<kM>(S, gid, kM == kAeifBeta ? p.n_ports : 2, y, (float)r.h);
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
cudaError_t aeif_launch(const SegTable<AeifSeg>& segs, dim3 g, const uint32_t* thr, const AeifState& S, int model,
                        Ring ring, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int sc, int budget,
                        bool pdl, cudaStream_t st) {
  const dim3 b(kAeifBlock);
  if (model == kAeifBeta)
    return launch_k(k_update_aeif<kFixed, kMode, kAeifBeta>, g, b, pdl, st, segs, thr, S, ring, clk, step_off, csr,
                    sb, sc, budget);
  if (model == kAeifAlpha)
    return launch_k(k_update_aeif<kFixed, kMode, kAeifAlpha>, g, b, pdl, st, segs, thr, S, ring, clk, step_off, csr,
                    sb, sc, budget);
  return launch_k(k_update_aeif<kFixed, kMode, kAeifExp>, g, b, pdl, st, segs, thr, S, ring, clk, step_off, csr, sb,
                  sc, budget);
}

template <bool kFixed, int kMode>
cudaError_t finish_launch(const SegTable<AeifSeg>& segs, dim3 g, const AeifState& S, int model, Ring ring,
                          int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, bool pdl, cudaStream_t st) {
  const dim3 b(kAeifBlock);
  if (model == kAeifBeta)
    return launch_k(k_aeif_finish<kFixed, kMode, kAeifBeta>, g, b, pdl, st, segs, S, ring, clk, step_off, csr, sb);
  if (model == kAeifAlpha)
    return launch_k(k_aeif_finish<kFixed, kMode, kAeifAlpha>, g, b, pdl, st, segs, S, ring, clk, step_off, csr, sb);
  return launch_k(k_aeif_finish<kFixed, kMode, kAeifExp>, g, b, pdl, st, segs, S, ring, clk, step_off, csr, sb);
}
}  // namespace

cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr,
                               const AeifState& S, int model, Ring ring, bool fixed, int64_t* clk, int64_t step_off,
                               const Csr& csr, SpikeBuf sb, int emit, bool scan, int budget, bool pdl,
                               cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks);
  const int sc = scan ? 1 : 0;
#define NGB_AEIF(F, M) return aeif_launch<F, M>(segs, g, thr, S, model, ring, clk, step_off, csr, sb, sc, budget, pdl, st)
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

cudaError_t launch_finish_aeif(const SegTable<AeifSeg>& segs, int grid, const AeifState& S, int model, Ring ring,
                               bool fixed, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int emit,
                               bool pdl, cudaStream_t st) {
  const dim3 g((unsigned)grid);
#define NGB_FIN(F, M) return finish_launch<F, M>(segs, g, S, model, ring, clk, step_off, csr, sb, pdl, st)
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

namespace ngb {
namespace {

__global__ void k_step_factor(const float* r, int64_t n, int k, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = k == 4 ? step_factor_root<4>(r[i]) : step_factor_root<5>(r[i]);
}

}  // namespace

int set_last_error(int code, const std::string& msg);  // ngb_api.cu: message for ngb_last_error()

}  // namespace ngb

extern "C" int ngb_eval_step_factor(const float* r, int64_t n, int32_t k, float* out) {
  using namespace ngb;
  if (n < 0 || (n > 0 && (!r || !out)) || (k != 4 && k != 5))
    return set_last_error(NGB_ERR_INVALID_ARG, "ngb_eval_step_factor: arguments");
  if (n == 0) return NGB_OK;
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, (size_t)n * 2 * sizeof(float));
  if (e != cudaSuccess) return set_last_error(NGB_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpy(d, r, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_step_factor<<<(unsigned)((n + 255) / 256), 256>>>(d, n, k, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_last_error(NGB_ERR_CUDA, std::string("ngb_eval_step_factor: ") + cudaGetErrorString(e));
  return NGB_OK;
}
