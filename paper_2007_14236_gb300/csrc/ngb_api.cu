// ngb_api.cu -- C ABI of the simulator core (include/ngb.h): handle,
// construction, finalisation, the step loop with CUDA graphs, spike record
// draining and introspection.
//
// One simulation step (global step t) is three stream-ordered launches:
//   k_update_lif   (LIF populations: read+zero ring slot t, Poisson, exact
//                   integration, threshold/reset/refractory, compaction)
//   k_update_aeif  (AdEx populations: same with adaptive RK45)
//   k_deliver      (scatter of step t's spikes into ring slots t + d)
// Deliveries of step t land in slots >= t + 1 (delays are >= 1 step), so the
// update of step t never races them.  The step counter lives on the device
// (clk), so a captured graph of S steps can be replayed unchanged; host and
// device meet only at drain points (every drain_steps steps and at the end of
// ngb_simulate) to collect the spike record and error flags.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

#include "builder.h"
#include "ngb.h"
#include "ngb_internal.cuh"

using namespace ngb;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? NGB_ERR_OOM : NGB_ERR_CUDA;
  return fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                           \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);    \
  } while (0)

struct PopHost {
  int model;
  int instance;
  int64_t n;
  int64_t offset;      // global id of the first neuron
  uint32_t local_off;  // instance-local id of the first neuron
  ngb_lif_params lif;
  ngb_aeif_params aeif;
};

struct InstHost {
  uint64_t seed;
  int64_t n;
  uint32_t n_calls;
  int64_t t0;
};

struct CallHost {
  int src_pop, tgt_pop;
  ngb_conn_spec conn;
  ngb_syn_spec syn;
  uint32_t stream;
};

// Poisson(lambda) inversion thresholds: ceil(F(k) * 2^32) for the CDF F built
// term by term, p_0 = exp(-lambda), p_k = p_{k-1} * lambda / k; a count k is
// drawn from a 32-bit word x as the number of thresholds <= x.
std::vector<uint32_t> poisson_thresholds(double lambda) {
  std::vector<uint32_t> out;
  if (!(lambda > 0.0)) return out;
  double p = std::exp(-lambda);
  double F = p;
  for (int k = 0; k < kMaxThr; ++k) {
    const double th = std::ceil(F * 4294967296.0);
    if (th > 4294967295.0) break;
    out.push_back((uint32_t)th);
    p = p * lambda / (double)(k + 1);
    F = F + p;
  }
  return out;
}

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int bits_for(uint64_t n) {  // bits to represent values 0 .. n-1
  int b = 1;
  while (b < 63 && (1ull << b) < n) ++b;
  return b;
}

}  // namespace

namespace ngb {
// Error message for ngb_last_error() from other translation units.
int set_last_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace ngb

struct ngb_sim {
  ngb_sim_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<PopHost> pops;
  std::vector<InstHost> inst;
  std::vector<CallHost> calls;
  bool finalized = false;
  bool failed = false;
  int64_t N = 0;
  int R = 1;
  int64_t L = 2;
  int max_delay = 0;
  uint64_t K = 0, G = 0;
  // device memory
  std::vector<void*> allocs;
  size_t dev_bytes = 0;
  float *st0 = nullptr, *st1 = nullptr, *st2 = nullptr, *st3 = nullptr, *st4 = nullptr;
  int32_t* ref = nullptr;
  void* ring = nullptr;
  uint64_t* src_syn = nullptr;
  uint32_t* src_grp = nullptr;
  uint64_t* grp_start = nullptr;
  uint16_t* grp_delay = nullptr;
  uint32_t* tgt = nullptr;
  void* w = nullptr;
  uint4* src_meta = nullptr;
  SpikeBuf sb{};
  int64_t* clk = nullptr;
  SegTable<LifSeg> lif_tab{};
  int n_lif = 0;
  int64_t lif_blocks = 0;
  SegTable<AeifSeg> aeif_tab{};
  int n_aeif = 0;
  int64_t aeif_blocks = 0;
  uint32_t* thr = nullptr;
  int deliver_grid = 0;
  bool pdl = true;  // programmatic dependent launch between the step's kernels
  int mode = 0;     // 0: per-step kernels in CUDA graphs, 1: persistent step kernel
  bool persist_ok = false;
  int persist_grid = 0;
  int persist_max_bpsm = 0;
  size_t persist_smem = 0;
  PersistArgs pa{};
  unsigned* bar = nullptr;
  uint32_t n_thr_total = 0;
  uint64_t work_items = 0;  // delivery work items of all sources (map capacity)
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  int drain_steps = 1000;
  int64_t t = 0;  // steps done
  int64_t spikes_total = 0;
  std::vector<uint32_t> rec_ids;
  std::vector<int64_t> rec_steps;
  size_t rec_sorted_upto = 0;  // records [0, upto) are sorted by (step, id)
  std::vector<double> pop_E_L;  // per population, for V of LIF (state holds V - E_L)

  template <typename T>
  cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e == cudaSuccess) {
      allocs.push_back((void*)*p);
      dev_bytes += count * sizeof(T);
    }
    return e;
  }
};

namespace {

Ring ring_of(const ngb_sim* s) { return Ring{s->ring, s->N, (uint32_t)(s->L - 1), s->R}; }

Csr csr_of(const ngb_sim* s) {
  return Csr{s->src_meta, s->src_syn, s->src_grp, s->grp_start, s->grp_delay, s->tgt, s->w};
}

cudaError_t launch_lif(ngb_sim* s) {
  return launch_update_lif(s->lif_tab, s->lif_blocks, s->thr, s->st0, s->st1, s->ref, ring_of(s),
                           s->cfg.deterministic != 0, s->clk, s->src_meta, s->sb, s->pdl, s->stream);
}

cudaError_t launch_aeif(ngb_sim* s) {
  return launch_update_aeif(s->aeif_tab, s->aeif_blocks, s->thr, s->st0, s->st1, s->st2, s->st3, s->st4,
                            ring_of(s), s->cfg.deterministic != 0, s->clk, s->src_meta, s->sb, s->pdl,
                            s->stream);
}

cudaError_t launch_del(ngb_sim* s) {
  return launch_deliver(s->sb, csr_of(s), s->cfg.weight_dtype, ring_of(s), s->cfg.deterministic != 0, s->clk,
                        s->deliver_grid, s->pdl, s->stream);
}

cudaError_t launch_step(ngb_sim* s) {
  cudaError_t e;
  if (s->n_lif) {
    e = launch_lif(s);
    if (e != cudaSuccess) return e;
  }
  if (s->n_aeif) {
    e = launch_aeif(s);
    if (e != cudaSuccess) return e;
  }
  return launch_del(s);
}

// One persistent launch of `steps` steps.
cudaError_t launch_persistent_chunk(ngb_sim* s, int64_t steps) {
  cudaError_t e = cudaMemsetAsync(s->bar, 0, 4 * sizeof(unsigned), s->stream);
  if (e != cudaSuccess) return e;
  s->pa.steps = steps;
  s->pa.sb = s->sb;
  return launch_persistent(s->pa, s->cfg.deterministic != 0, s->cfg.weight_dtype, s->n_lif > 0, s->n_aeif > 0,
                           s->persist_grid, s->persist_smem, s->stream);
}

// Collect the device spike record and error flags; resets the record.
int drain(ngb_sim* s) {
  unsigned long long cnt = 0;
  uint32_t err = 0;
  CK(cudaMemcpyAsync(&cnt, s->sb.rec_count, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&err, s->sb.err, sizeof(err), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->spikes_total += (int64_t)cnt;
  if (s->sb.rec_cap > 0 && cnt > 0) {
    const size_t n = (size_t)std::min<unsigned long long>(cnt, (unsigned long long)s->sb.rec_cap);
    const size_t old = s->rec_ids.size();
    s->rec_ids.resize(old + n);
    s->rec_steps.resize(old + n);
    CK(cudaMemcpyAsync(s->rec_ids.data() + old, s->sb.rec_id, n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaMemcpyAsync(s->rec_steps.data() + old, s->sb.rec_step, n * sizeof(int64_t), cudaMemcpyDeviceToHost,
                       s->stream));
  }
  CK(cudaMemsetAsync(s->sb.rec_count, 0, sizeof(unsigned long long), s->stream));
  CK(cudaMemsetAsync(s->sb.err, 0, sizeof(uint32_t), s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (err & kErrBarrierTimeout) {
    s->failed = true;
    return fail(NGB_ERR_TIMEOUT, "persistent step kernel: a grid barrier wait gave up (handle unusable)");
  }
  if (err & kErrRecordOverflow)
    return fail(NGB_ERR_OVERFLOW, "spike record overflow: raise record_capacity or lower drain_steps");
  if (err & kErrSubstepCap)
    return fail(NGB_ERR_OVERFLOW, "AdEx Runge-Kutta sub-step cap reached (rk_max_substeps)");
  return NGB_OK;
}

// (Re)capture the CUDA graph of graph_steps steps with the current launch
// configuration.
int capture_graph(ngb_sim* s) {
  if (s->gexec) {
    cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
  }
  if (s->graph_steps <= 0) return NGB_OK;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < s->graph_steps && e == cudaSuccess; ++i) e = launch_step(s);
  cudaError_t e2 = cudaStreamEndCapture(s->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture (kernel launch)");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&s->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return NGB_OK;
}

int finalize_impl(ngb_sim* s) {
  if (s->finalized) return NGB_OK;
  if (s->N <= 0) return fail(NGB_ERR_STATE, "ngb_finalize: no neurons");
  if (s->N >= (int64_t)kIdMask) return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^26 neurons");
  cudaStream_t st = s->stream;
  const int64_t N = s->N;
  s->R = 1;
  for (const PopHost& p : s->pops)
    if (p.model == NGB_AEIF_COND_EXP) s->R = 2;
  const double dt = s->cfg.dt_ms;
  const int prec = s->cfg.weight_dtype;
  const size_t wsize = prec == NGB_WEIGHT_FP32 ? 4 : 2;

  // ---------------------------------------------------------------- connections
  unsigned long long *src_cnt = nullptr, *src_ngrp = nullptr, *scan_out = nullptr;
  int* dmax = nullptr;
  CK(cudaMalloc(&src_cnt, (N + 1) * sizeof(unsigned long long)));
  CK(cudaMalloc(&src_ngrp, (N + 1) * sizeof(unsigned long long)));
  CK(cudaMalloc(&scan_out, (N + 1) * sizeof(unsigned long long)));
  CK(cudaMalloc(&dmax, sizeof(int)));
  CK(cudaMemsetAsync(src_cnt, 0, (N + 1) * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(src_ngrp, 0, (N + 1) * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(dmax, 0, sizeof(int), st));

  std::vector<std::vector<CallDev>> by_src(s->pops.size());
  std::vector<uint64_t> n_by_src(s->pops.size(), 0);
  uint64_t Kmax_pop = 0;
  for (const CallHost& c : s->calls) {
    const PopHost& ps = s->pops[c.src_pop];
    const PopHost& pt = s->pops[c.tgt_pop];
    CallDev d{};
    d.seed = s->inst[ps.instance].seed;
    d.K = c.conn.K;
    d.nsyn = c.conn.rule == NGB_RULE_FIXED_INDEGREE ? (uint64_t)c.conn.K * (uint64_t)pt.n : (uint64_t)c.conn.K;
    d.w0 = c.syn.weight.p0;
    d.w1 = c.syn.weight.p1;
    d.d0 = c.syn.delay_ms.p0;
    d.d1 = c.syn.delay_ms.p1;
    d.dt = dt;
    d.stream = c.stream;
    d.rule = c.conn.rule;
    d.no_autapse = (c.src_pop == c.tgt_pop && !c.conn.allow_autapses) ? 1 : 0;
    d.wdist = c.syn.weight.dist;
    d.ddist = c.syn.delay_ms.dist;
    d.receptor = c.syn.receptor;
    d.prec = prec;
    d.n_src = (uint32_t)ps.n;
    d.n_tgt = (uint32_t)pt.n;
    d.src_off = (uint32_t)ps.offset;
    d.tgt_off = (uint32_t)pt.offset;
    by_src[c.src_pop].push_back(d);
    n_by_src[c.src_pop] += d.nsyn;
  }
  uint64_t K = 0;
  for (size_t p = 0; p < s->pops.size(); ++p) {
    K += n_by_src[p];
    Kmax_pop = std::max(Kmax_pop, n_by_src[p]);
    if (n_by_src[p] >= (1ull << 32))
      return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^32 synapses from one population");
  }
  s->K = K;
  const uint64_t Kpad = ((K + 3) & ~3ull) + kChunk;
  CK(s->dalloc(&s->tgt, Kpad));
  CK(s->dalloc((uint8_t**)&s->w, Kpad * wsize));
  CK(cudaMemsetAsync(s->tgt, 0, Kpad * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(s->w, 0, Kpad * wsize, st));

  std::vector<uint64_t*> gs_parts;
  std::vector<uint16_t*> gd_parts;
  std::vector<uint64_t> g_counts;
  if (Kmax_pop > 0) {
    BuildScratch sc;
    int max_bits = 1;
    for (size_t p = 0; p < s->pops.size(); ++p) max_bits = std::max(max_bits, bits_for((uint64_t)s->pops[p].n));
    CK(sort_scratch_bytes(Kmax_pop, max_bits + kDelayBits, &sc.sort_bytes, &sc.scan_bytes));
    CK(cudaMalloc(&sc.keys, Kmax_pop * sizeof(unsigned long long)));
    CK(cudaMalloc(&sc.keys_alt, Kmax_pop * sizeof(unsigned long long)));
    CK(cudaMalloc(&sc.vals, Kmax_pop * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.vals_alt, Kmax_pop * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.st_tgt, Kmax_pop * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.st_w, Kmax_pop * sizeof(float)));
    CK(cudaMalloc(&sc.flag, Kmax_pop * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.gidx, Kmax_pop * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.sort_tmp, std::max<size_t>(sc.sort_bytes, 16)));
    CK(cudaMalloc(&sc.scan_tmp, std::max<size_t>(sc.scan_bytes, 16)));
    uint64_t csr_off = 0;
    for (size_t p = 0; p < s->pops.size(); ++p) {
      if (n_by_src[p] == 0) continue;
      std::string err;
      uint64_t* gs = nullptr;
      uint16_t* gd = nullptr;
      uint64_t gcount = 0;
      cudaError_t e = build_source_population(by_src[p], n_by_src[p], bits_for((uint64_t)s->pops[p].n), csr_off,
                                              prec, sc, s->tgt + csr_off, (uint8_t*)s->w + csr_off * wsize, src_cnt,
                                              src_ngrp, dmax, &gs, &gd, &gcount, st, err);
      if (e != cudaSuccess) return cuda_fail(e, ("connection builder: " + err).c_str());
      gs_parts.push_back(gs);
      gd_parts.push_back(gd);
      g_counts.push_back(gcount);
      csr_off += n_by_src[p];
    }
    CK(cudaStreamSynchronize(st));
    cudaFree(sc.keys); cudaFree(sc.keys_alt); cudaFree(sc.vals); cudaFree(sc.vals_alt);
    cudaFree(sc.st_tgt); cudaFree(sc.st_w); cudaFree(sc.flag); cudaFree(sc.gidx);
    cudaFree(sc.sort_tmp); cudaFree(sc.scan_tmp);
  }
  uint64_t G = 0;
  for (uint64_t g : g_counts) G += g;
  if (G >= (1ull << 32)) return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^32 connection groups");
  s->G = G;
  CK(s->dalloc(&s->grp_start, G + 1));
  CK(s->dalloc(&s->grp_delay, G + 1));
  {
    uint64_t off = 0;
    for (size_t i = 0; i < gs_parts.size(); ++i) {
      if (g_counts[i]) {
        CK(cudaMemcpyAsync(s->grp_start + off, gs_parts[i], g_counts[i] * sizeof(uint64_t),
                           cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(s->grp_delay + off, gd_parts[i], g_counts[i] * sizeof(uint16_t),
                           cudaMemcpyDeviceToDevice, st));
      }
      off += g_counts[i];
    }
    const uint64_t Kend = K;
    CK(cudaMemcpyAsync(s->grp_start + G, &Kend, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < gs_parts.size(); ++i) {
      cudaFree(gs_parts[i]);
      cudaFree(gd_parts[i]);
    }
  }
  {
    size_t tmp_bytes = 0;
    CK(scan_scratch_bytes_u64((uint64_t)N + 1, &tmp_bytes));
    void* tmp = nullptr;
    CK(cudaMalloc(&tmp, std::max<size_t>(tmp_bytes, 16)));
    CK(s->dalloc(&s->src_syn, N + 1));
    CK(exclusive_scan_u64(src_cnt, (unsigned long long*)s->src_syn, (uint64_t)N + 1, tmp, tmp_bytes, st));
    CK(exclusive_scan_u64(src_ngrp, scan_out, (uint64_t)N + 1, tmp, tmp_bytes, st));
    CK(s->dalloc(&s->src_grp, N + 1));
    CK(narrow_u64_to_u32(scan_out, s->src_grp, (uint64_t)N + 1, st));
    CK(s->dalloc(&s->src_meta, N));
    unsigned long long* items = nullptr;
    CK(cudaMalloc(&items, sizeof(unsigned long long)));
    CK(cudaMemsetAsync(items, 0, sizeof(unsigned long long), st));
    CK(launch_build_meta(N, s->src_syn, s->src_grp, s->src_meta, items, st));
    unsigned long long items_h = 0;
    CK(cudaMemcpyAsync(&items_h, items, sizeof(items_h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(items);
    s->work_items = items_h;
    if (items_h >= (1ull << 32))
      return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^32 delivery work items per step");
    int md = 0;
    CK(cudaMemcpyAsync(&md, dmax, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(tmp);
    s->max_delay = md;
  }
  cudaFree(src_cnt);
  cudaFree(src_ngrp);
  cudaFree(scan_out);
  cudaFree(dmax);
  s->L = (int64_t)std::max<uint64_t>(2, next_pow2((uint64_t)s->max_delay + 1));

  // ---------------------------------------------------------------- state and ring
  const size_t ring_elems = (size_t)s->L * s->R * N;
  const size_t ring_esize = s->cfg.deterministic ? 8 : 4;
  CK(s->dalloc((uint8_t**)&s->ring, ring_elems * ring_esize));
  CK(cudaMemsetAsync(s->ring, 0, ring_elems * ring_esize, st));
  CK(s->dalloc(&s->st0, N));
  CK(s->dalloc(&s->st1, N));
  CK(s->dalloc(&s->ref, N));
  CK(cudaMemsetAsync(s->st1, 0, N * sizeof(float), st));
  CK(cudaMemsetAsync(s->ref, 0, N * sizeof(int32_t), st));
  if (s->R == 2) {
    CK(s->dalloc(&s->st2, N));
    CK(s->dalloc(&s->st3, N));
    CK(s->dalloc(&s->st4, N));
    CK(cudaMemsetAsync(s->st2, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(s->st3, 0, N * sizeof(float), st));
  }
  std::vector<LifSeg> lsegs;
  std::vector<AeifSeg> asegs;
  std::vector<uint32_t> thr_all;
  for (const PopHost& p : s->pops) {
    const uint64_t seed = s->inst[p.instance].seed;
    if (p.model == NGB_LIF_PSC_EXP) {
      const ngb_lif_params& q = p.lif;
      CK(launch_init_state(0, p.n, q.V_init_mean_mV, q.V_init_sd_mV, q.E_L_mV, 0.0, 0.0, seed, p.local_off,
                           s->st0 + p.offset, nullptr, nullptr, st));
      // exact-integration propagators over one step (Eqs. 1-2), y = V - E_L
      const double h = dt, tm = q.tau_m_ms, ts = q.tau_syn_ms, C = q.C_m_pF;
      const double P11 = std::exp(-h / ts);
      const double P22 = std::exp(-h / tm);
      double P21;
      if (tm == ts) P21 = h / C * P22;
      else P21 = tm * ts / (C * (tm - ts)) * (std::expm1(-h / tm) - std::expm1(-h / ts));
      const double P20 = -tm / C * std::expm1(-h / tm);
      LifSeg g{};
      g.offset = p.offset;
      g.n = p.n;
      g.blk_begin = s->lif_blocks;
      g.t0 = s->inst[p.instance].t0;
      g.seed = seed;
      g.local_off = p.local_off;
      const std::vector<uint32_t> th = poisson_thresholds(q.poisson.n_inputs * q.poisson.rate_hz * dt * 1e-3);
      g.n_thr = (uint32_t)th.size();
      g.thr_off = (uint32_t)thr_all.size();
      thr_all.insert(thr_all.end(), th.begin(), th.end());
      g.ref_steps = (int32_t)std::nearbyint(q.t_ref_ms / dt);
      g.P11 = (float)P11;
      g.P21 = (float)P21;
      g.P22 = (float)P22;
      g.P20Ie = (float)(P20 * q.I_e_pA);
      g.theta = (float)(q.V_th_mV - q.E_L_mV);
      g.y_reset = (float)(q.V_reset_mV - q.E_L_mV);
      g.w_ext = (float)q.poisson.weight;
      lsegs.push_back(g);
      s->lif_blocks += (p.n + kLifBlock - 1) / kLifBlock;
    } else {
      const ngb_aeif_params& q = p.aeif;
      CK(launch_init_state(1, p.n, q.V_init_mean_mV, q.V_init_sd_mV, q.E_L_mV, q.w_init_pA, q.rk_h_init_ms, seed,
                           p.local_off, s->st0 + p.offset, s->st1 + p.offset, s->st4 + p.offset, st));
      AeifSeg g{};
      g.offset = p.offset;
      g.n = p.n;
      g.blk_begin = s->aeif_blocks;
      g.t0 = s->inst[p.instance].t0;
      g.seed = seed;
      g.local_off = p.local_off;
      const std::vector<uint32_t> th = poisson_thresholds(q.poisson.n_inputs * q.poisson.rate_hz * dt * 1e-3);
      g.n_thr = (uint32_t)th.size();
      g.thr_off = (uint32_t)thr_all.size();
      thr_all.insert(thr_all.end(), th.begin(), th.end());
      g.prec_rcpt = q.poisson.receptor;
      g.g_L = (float)q.g_L_nS;
      g.E_L = (float)q.E_L_mV;
      g.V_T = (float)q.V_T_mV;
      g.Delta_T = (float)q.Delta_T_mV;
      g.inv_Delta_T = q.Delta_T_mV > 0 ? (float)(1.0 / q.Delta_T_mV) : 0.0f;
      g.a = (float)q.a_nS;
      g.inv_tau_w = (float)(1.0 / q.tau_w_ms);
      g.V_peak = (float)q.V_peak_mV;
      g.V_reset = (float)q.V_reset_mV;
      g.b = (float)q.b_pA;
      g.E_ex = (float)q.E_ex_mV;
      g.E_in = (float)q.E_in_mV;
      g.inv_tau_ex = (float)(1.0 / q.tau_ex_ms);
      g.inv_tau_in = (float)(1.0 / q.tau_in_ms);
      g.I_e = (float)q.I_e_pA;
      g.inv_C = (float)(1.0 / q.C_m_pF);
      g.w_ext = (float)q.poisson.weight;
      const double tol_eff = std::max(q.rk_tol, 8.0 * 5.9604644775390625e-08);  // FP32 floor 8 * 2^-24
      g.inv_tol = 1.0 / tol_eff;
      g.h_min = q.rk_h_min_ms;
      g.dt = dt;
      g.max_sub = q.rk_max_substeps;
      asegs.push_back(g);
      s->aeif_blocks += (p.n + kAeifBlock - 1) / kAeifBlock;
    }
  }
  s->n_lif = (int)lsegs.size();
  s->n_aeif = (int)asegs.size();
  if (s->n_lif) {
    LifSeg* d = nullptr;
    CK(s->dalloc(&d, lsegs.size()));
    CK(cudaMemcpyAsync(d, lsegs.data(), lsegs.size() * sizeof(LifSeg), cudaMemcpyHostToDevice, st));
    s->lif_tab.dev = d;
    s->lif_tab.n = s->n_lif;
    for (int i = 0; i < std::min(s->n_lif, kInlineSegs); ++i) s->lif_tab.s[i] = lsegs[i];
    std::vector<uint32_t> bs((size_t)s->lif_blocks);
    for (size_t i = 0; i < lsegs.size(); ++i) {
      const int64_t nb = (lsegs[i].n + kLifBlock - 1) / kLifBlock;
      for (int64_t b = 0; b < nb; ++b) bs[(size_t)(lsegs[i].blk_begin + b)] = (uint32_t)i;
    }
    uint32_t* db = nullptr;
    CK(s->dalloc(&db, bs.size()));
    CK(cudaMemcpyAsync(db, bs.data(), bs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    s->lif_tab.blk_seg = db;
  }
  if (s->n_aeif) {
    AeifSeg* d = nullptr;
    CK(s->dalloc(&d, asegs.size()));
    CK(cudaMemcpyAsync(d, asegs.data(), asegs.size() * sizeof(AeifSeg), cudaMemcpyHostToDevice, st));
    s->aeif_tab.dev = d;
    s->aeif_tab.n = s->n_aeif;
    for (int i = 0; i < std::min(s->n_aeif, kInlineSegs); ++i) s->aeif_tab.s[i] = asegs[i];
    std::vector<uint32_t> bs((size_t)s->aeif_blocks);
    for (size_t i = 0; i < asegs.size(); ++i) {
      const int64_t nb = (asegs[i].n + kAeifBlock - 1) / kAeifBlock;
      for (int64_t b = 0; b < nb; ++b) bs[(size_t)(asegs[i].blk_begin + b)] = (uint32_t)i;
    }
    uint32_t* db = nullptr;
    CK(s->dalloc(&db, bs.size()));
    CK(cudaMemcpyAsync(db, bs.data(), bs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    s->aeif_tab.blk_seg = db;
  }
  CK(s->dalloc(&s->thr, thr_all.size() + 1));
  if (!thr_all.empty())
    CK(cudaMemcpyAsync(s->thr, thr_all.data(), thr_all.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));

  // ---------------------------------------------------------------- spike lists and record
  CK(s->dalloc(&s->sb.wi[0], 2 * s->work_items + 2));
  CK(s->dalloc(&s->sb.wi[1], 2 * s->work_items + 2));
  {
    const char* env = std::getenv("NGB_PDL");
    s->pdl = !(env && env[0] == '0');
  }
  unsigned long long* ctrs = nullptr;
  CK(s->dalloc(&ctrs, 6));  // ctr[2], events, substeps, rec_count, spare
  CK(cudaMemsetAsync(ctrs, 0, 6 * sizeof(unsigned long long), st));
  s->sb.ctr = ctrs;
  s->sb.events = ctrs + 2;
  s->sb.substeps = ctrs + 3;
  s->sb.rec_count = ctrs + 4;
  CK(s->dalloc(&s->sb.err, 1));
  CK(cudaMemsetAsync(s->sb.err, 0, sizeof(uint32_t), st));
  CK(s->dalloc(&s->clk, 2));
  CK(cudaMemsetAsync(s->clk, 0, 2 * sizeof(int64_t), st));
  s->drain_steps = s->cfg.drain_steps > 0 ? s->cfg.drain_steps : 1000;
  int64_t cap = 0;
  if (s->cfg.record_spikes) {
    cap = s->cfg.record_capacity > 0 ? s->cfg.record_capacity
                                     : std::max<int64_t>(1 << 20, N * (int64_t)s->drain_steps / 100);
    CK(s->dalloc(&s->sb.rec_id, cap));
    CK(s->dalloc(&s->sb.rec_step, cap));
  }
  s->sb.rec_cap = cap;

  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  s->deliver_grid = std::max(1, sms) * 2;
  CK(cudaStreamSynchronize(st));

  // ---------------------------------------------------------------- persistent kernel set-up
  {
    std::vector<int64_t> lv(1, 0), av(1, 0);
    for (const LifSeg& g : lsegs) lv.push_back(lv.back() + g.n);
    for (const AeifSeg& g : asegs) av.push_back(av.back() + g.n);
    int64_t *dlv = nullptr, *dav = nullptr;
    CK(s->dalloc(&dlv, lv.size()));
    CK(s->dalloc(&dav, av.size()));
    CK(cudaMemcpyAsync(dlv, lv.data(), lv.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dav, av.data(), av.size() * 8, cudaMemcpyHostToDevice, st));
    CK(s->dalloc(&s->bar, 4));
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    PersistArgs& a = s->pa;
    a.lseg = s->lif_tab.dev;
    a.aseg = s->aeif_tab.dev;
    a.lvoff = dlv;
    a.avoff = dav;
    a.thr = s->thr;
    a.st0 = s->st0; a.st1 = s->st1; a.st2 = s->st2; a.st3 = s->st3; a.st4 = s->st4;
    a.ref = s->ref;
    a.src_meta = s->src_meta;
    a.ring = ring_of(s);
    a.csr = csr_of(s);
    a.sb = s->sb;
    a.clk = s->clk;
    a.bar = s->bar;
    a.n_lif = lv.back();
    a.n_aeif = av.back();
    a.n_thr = (uint32_t)thr_all.size();
    a.n_lseg = (int32_t)lsegs.size();
    a.n_aseg = (int32_t)asegs.size();
    const char* env_spin = std::getenv("NGB_BARRIER_SPIN_LIMIT");
    a.spin_limit = env_spin ? std::strtoull(env_spin, nullptr, 10) : (1ull << 24);
    const char* env_wh = std::getenv("NGB_TEST_WITHHOLD_BLOCK");
    a.withhold_block = env_wh ? std::atoi(env_wh) : -1;
    a.off_aseg = (uint32_t)a16(lsegs.size() * sizeof(LifSeg));
    a.off_lvoff = a.off_aseg + (uint32_t)a16(asegs.size() * sizeof(AeifSeg));
    a.off_avoff = a.off_lvoff + (uint32_t)a16(lv.size() * 8);
    a.off_thr = a.off_avoff + (uint32_t)a16(av.size() * 8);
    s->persist_smem = a.off_thr + a16(thr_all.size() * 4);
    s->persist_ok = false;
    if (s->persist_smem <= 200 * 1024) {
      int bpsm = 0;
      if (persistent_max_blocks_per_sm(s->cfg.deterministic != 0, s->cfg.weight_dtype, s->n_lif > 0,
                                       s->n_aeif > 0, s->persist_smem, &bpsm) == cudaSuccess && bpsm > 0) {
        s->persist_ok = true;
        s->persist_max_bpsm = bpsm;
        s->persist_grid = sms * std::min(bpsm, 2);
      }
      cudaGetLastError();
    }
    const char* env_mode = std::getenv("NGB_MODE");
    s->mode = (env_mode && std::string(env_mode) == "persistent" && s->persist_ok) ? 1 : 0;
  }

  // ---------------------------------------------------------------- step graph
  s->graph_steps = s->cfg.steps_per_graph == 0 ? 100 : std::max(0, s->cfg.steps_per_graph);
  {
    const int rc = capture_graph(s);
    if (rc != NGB_OK) return rc;
  }
  s->finalized = true;
  return NGB_OK;
}

int check_handle(ngb_sim* s) {
  if (!s) return fail(NGB_ERR_INVALID_ARG, "NULL handle");
  if (s->failed) return fail(NGB_ERR_STATE, "handle is unusable after an earlier CUDA failure");
  cudaError_t e = cudaSetDevice(s->cfg.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return NGB_OK;
}

int simulate_impl(ngb_sim* s, int64_t steps, bool profiled, double* kernel_ms, int64_t* launches) {
  if (steps < 0) return fail(NGB_ERR_INVALID_ARG, "ngb_simulate: steps < 0");
  if (!s->finalized) {
    const int rc = finalize_impl(s);
    if (rc != NGB_OK) {
      s->failed = true;
      return rc;
    }
  }
  int rc_overflow = NGB_OK;
  if (!profiled) {
    int64_t left = steps;
    while (left > 0) {
      const int64_t chunk = std::min<int64_t>(left, s->drain_steps);
      int64_t done = 0;
      if (s->mode == 1) {
        CK(launch_persistent_chunk(s, chunk));
        done = chunk;
      }
      if (s->gexec) {
        while (chunk - done >= s->graph_steps) {
          CK(cudaGraphLaunch(s->gexec, s->stream));
          done += s->graph_steps;
        }
      }
      for (; done < chunk; ++done) CK(launch_step(s));
      s->t += chunk;
      left -= chunk;
      const int rc = drain(s);
      if (rc == NGB_ERR_OVERFLOW) rc_overflow = rc;
      else if (rc != NGB_OK) return rc;
    }
    return rc_overflow;
  }
  // profiled: eager launches bracketed by events
  const int kBatch = 128;
  std::vector<cudaEvent_t> ev(4 * kBatch);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double ms[3] = {0, 0, 0};
  int64_t nl[3] = {0, 0, 0};
  int64_t left = steps;
  int rc_final = NGB_OK;
  while (left > 0 && rc_final == NGB_OK) {
    const int64_t chunk = std::min<int64_t>(left, std::min<int64_t>(kBatch, s->drain_steps));
    for (int64_t i = 0; i < chunk; ++i) {
      cudaEvent_t* e = &ev[4 * i];
      CK(cudaEventRecord(e[0], s->stream));
      if (s->n_lif) CK(launch_lif(s));
      CK(cudaEventRecord(e[1], s->stream));
      if (s->n_aeif) CK(launch_aeif(s));
      CK(cudaEventRecord(e[2], s->stream));
      CK(launch_del(s));
      CK(cudaEventRecord(e[3], s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < chunk; ++i) {
      float a = 0, b = 0, c = 0;
      CK(cudaEventElapsedTime(&a, ev[4 * i], ev[4 * i + 1]));
      CK(cudaEventElapsedTime(&b, ev[4 * i + 1], ev[4 * i + 2]));
      CK(cudaEventElapsedTime(&c, ev[4 * i + 2], ev[4 * i + 3]));
      if (s->n_lif) { ms[0] += a; nl[0] += 1; }
      if (s->n_aeif) { ms[1] += b; nl[1] += 1; }
      ms[2] += c;
      nl[2] += 1;
    }
    s->t += chunk;
    left -= chunk;
    const int rc = drain(s);
    if (rc == NGB_ERR_OVERFLOW) rc_overflow = rc;
    else if (rc != NGB_OK) rc_final = rc;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (kernel_ms)
    for (int i = 0; i < 3; ++i) kernel_ms[i] = ms[i];
  if (launches)
    for (int i = 0; i < 3; ++i) launches[i] = nl[i];
  return rc_final != NGB_OK ? rc_final : rc_overflow;
}

bool valid_dist(const ngb_dist_spec& d) { return d.dist >= NGB_DIST_CONST && d.dist <= NGB_DIST_UNIFORM; }

// Device state that a simulated step changes: neuron state, ring buffer,
// counters and the step clock.  Saved and restored around autotuning trials.
struct Snapshot {
  std::vector<std::pair<void*, size_t>> parts;
  std::vector<void*> copies;
};

int snapshot_take(ngb_sim* s, Snapshot& sn) {
  const int64_t N = s->N;
  const size_t ring_bytes = (size_t)s->L * s->R * N * (s->cfg.deterministic ? 8 : 4);
  sn.parts = {{s->st0, N * 4}, {s->st1, N * 4}, {s->ref, N * 4}, {s->ring, ring_bytes},
              {s->sb.ctr, 6 * sizeof(unsigned long long)}, {s->clk, 2 * sizeof(int64_t)},
              {s->sb.err, sizeof(uint32_t)}};
  if (s->st2) {
    sn.parts.push_back({s->st2, N * 4});
    sn.parts.push_back({s->st3, N * 4});
    sn.parts.push_back({s->st4, N * 4});
  }
  for (auto& p : sn.parts) {
    void* c = nullptr;
    CK(cudaMalloc(&c, p.second));
    sn.copies.push_back(c);
    CK(cudaMemcpyAsync(c, p.first, p.second, cudaMemcpyDeviceToDevice, s->stream));
  }
  return NGB_OK;
}

int snapshot_restore(ngb_sim* s, const Snapshot& sn) {
  for (size_t i = 0; i < sn.parts.size(); ++i)
    CK(cudaMemcpyAsync(sn.parts[i].first, sn.copies[i], sn.parts[i].second, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return NGB_OK;
}

void snapshot_free(Snapshot& sn) {
  for (void* c : sn.copies) cudaFree(c);
  sn.copies.clear();
}

std::string tune_key(ngb_sim* s) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, s->cfg.device);
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s|sm%d|N%lld|K%llu|G%llu|L%lld|R%d|w%d|det%d|lif%d|aeif%d", prop.name,
                prop.multiProcessorCount, (long long)s->N, (unsigned long long)s->K, (unsigned long long)s->G,
                (long long)s->L, s->R, s->cfg.weight_dtype, s->cfg.deterministic, s->n_lif, s->n_aeif);
  for (char* c = buf; *c; ++c)
    if (*c == ' ') *c = '_';
  return buf;
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

const char* ngb_last_error(const ngb_sim*) { return g_last_error.c_str(); }

int ngb_create(ngb_sim** out, const ngb_sim_config* cfg) {
  if (!out || !cfg) return fail(NGB_ERR_INVALID_ARG, "ngb_create: NULL argument");
  *out = nullptr;
  if (!(cfg->dt_ms > 0.0)) return fail(NGB_ERR_INVALID_ARG, "ngb_create: dt_ms must be > 0");
  if (cfg->weight_dtype < NGB_WEIGHT_FP32 || cfg->weight_dtype > NGB_WEIGHT_FP16)
    return fail(NGB_ERR_INVALID_ARG, "ngb_create: weight_dtype");
  if (cfg->record_capacity < 0 || cfg->drain_steps < 0) return fail(NGB_ERR_INVALID_ARG, "ngb_create: capacities");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (cfg->device < 0 || cfg->device >= ndev) return fail(NGB_ERR_INVALID_ARG, "ngb_create: device ordinal");
  e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  ngb_sim* s = new ngb_sim();
  s->cfg = *cfg;
  if (cfg->stream) {
    s->stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, "cudaStreamCreate");
    }
    s->own_stream = true;
  }
  s->inst.push_back(InstHost{cfg->seed, 0, 0, 0});
  *out = s;
  return NGB_OK;
}

int ngb_destroy(ngb_sim* s) {
  if (!s) return NGB_OK;
  cudaSetDevice(s->cfg.device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  for (void* p : s->allocs) cudaFree(p);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return NGB_OK;
}

int ngb_add_instance(ngb_sim* s, uint64_t seed, int32_t* instance_out) {
  if (!s) return fail(NGB_ERR_INVALID_ARG, "NULL handle");
  if (s->finalized) return fail(NGB_ERR_STATE, "ngb_add_instance: network already finalised");
  s->inst.push_back(InstHost{seed, 0, 0, 0});
  if (instance_out) *instance_out = (int32_t)s->inst.size() - 1;
  return NGB_OK;
}

int ngb_add_population_in(ngb_sim* s, int32_t instance, int32_t model, int64_t n, const void* params,
                          int32_t* pop_id_out) {
  if (!s || !params) return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: NULL argument");
  if (s->finalized) return fail(NGB_ERR_STATE, "ngb_add_population: network already finalised");
  if (instance < 0 || instance >= (int32_t)s->inst.size())
    return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: unknown instance");
  if (n <= 0 || s->N + n >= (int64_t)kIdMask) return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: n");
  PopHost p{};
  p.model = model;
  p.instance = instance;
  p.n = n;
  p.offset = s->N;
  p.local_off = (uint32_t)s->inst[instance].n;
  const double dt = s->cfg.dt_ms;
  double lambda = 0.0;
  if (model == NGB_LIF_PSC_EXP) {
    p.lif = *(const ngb_lif_params*)params;
    const ngb_lif_params& q = p.lif;
    if (!(q.tau_m_ms > 0 && q.C_m_pF > 0 && q.tau_syn_ms > 0 && q.t_ref_ms >= 0 && q.V_init_sd_mV >= 0))
      return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: LIF parameters");
    lambda = q.poisson.n_inputs * q.poisson.rate_hz * dt * 1e-3;
    s->pop_E_L.push_back(q.E_L_mV);
  } else if (model == NGB_AEIF_COND_EXP) {
    p.aeif = *(const ngb_aeif_params*)params;
    const ngb_aeif_params& q = p.aeif;
    if (!(q.C_m_pF > 0 && q.tau_w_ms > 0 && q.tau_ex_ms > 0 && q.tau_in_ms > 0 && q.rk_tol > 0 &&
          q.rk_h_min_ms > 0 && q.rk_h_init_ms > 0 && q.rk_max_substeps > 0 && q.Delta_T_mV >= 0 &&
          q.V_init_sd_mV >= 0 && (q.poisson.receptor == 0 || q.poisson.receptor == 1)))
      return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: AdEx parameters");
    lambda = q.poisson.n_inputs * q.poisson.rate_hz * dt * 1e-3;
    s->pop_E_L.push_back(0.0);
  } else {
    return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: unknown model");
  }
  if (!(lambda >= 0.0 && lambda <= 100.0))
    return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: Poisson mean per step must be in [0, 100]");
  s->pops.push_back(p);
  s->N += n;
  s->inst[instance].n += n;
  if (pop_id_out) *pop_id_out = (int32_t)s->pops.size() - 1;
  return NGB_OK;
}

int ngb_add_population(ngb_sim* s, int32_t model, int64_t n, const void* params, int32_t* pop_id_out) {
  return ngb_add_population_in(s, 0, model, n, params, pop_id_out);
}

int ngb_connect(ngb_sim* s, int32_t src_pop, int32_t tgt_pop, const ngb_conn_spec* conn, const ngb_syn_spec* syn) {
  if (!s || !conn || !syn) return fail(NGB_ERR_INVALID_ARG, "ngb_connect: NULL argument");
  if (s->finalized) return fail(NGB_ERR_STATE, "ngb_connect: network already finalised");
  const int32_t np = (int32_t)s->pops.size();
  if (src_pop < 0 || src_pop >= np || tgt_pop < 0 || tgt_pop >= np)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: population id");
  const PopHost& ps = s->pops[src_pop];
  const PopHost& pt = s->pops[tgt_pop];
  if (ps.instance != pt.instance) return fail(NGB_ERR_INVALID_ARG, "ngb_connect: populations of different instances");
  if (conn->rule != NGB_RULE_FIXED_INDEGREE && conn->rule != NGB_RULE_FIXED_TOTAL_NUMBER)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: rule");
  if (conn->K < 0) return fail(NGB_ERR_INVALID_ARG, "ngb_connect: K < 0");
  if (!valid_dist(syn->weight) || !valid_dist(syn->delay_ms))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: distribution");
  if (syn->receptor < 0 || syn->receptor > 1 || (syn->receptor == 1 && pt.model == NGB_LIF_PSC_EXP))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: receptor");
  if (syn->delay_ms.dist == NGB_DIST_NORMAL && !(syn->delay_ms.p1 >= 0))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: delay sd");
  if (syn->delay_ms.dist == NGB_DIST_CONST && !(syn->delay_ms.p0 >= 0))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: delay");
  if (syn->delay_ms.dist == NGB_DIST_UNIFORM && !(syn->delay_ms.p1 >= syn->delay_ms.p0 && syn->delay_ms.p0 >= 0))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: uniform delay bounds");
  if (syn->weight.dist == NGB_DIST_NORMAL && !(syn->weight.p1 >= 0))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: weight sd");
  if (src_pop == tgt_pop && !conn->allow_autapses && ps.n < 2 && conn->K > 0)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: no admissible source without autapses");
  const double maxd = syn->delay_ms.dist == NGB_DIST_UNIFORM ? syn->delay_ms.p1 : syn->delay_ms.p0;
  if (syn->delay_ms.dist != NGB_DIST_NORMAL && maxd / s->cfg.dt_ms > (double)kMaxDelay)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: delay beyond 4095 steps");
  CallHost c{src_pop, tgt_pop, *conn, *syn, s->inst[ps.instance].n_calls};
  s->inst[ps.instance].n_calls += 1;
  s->calls.push_back(c);
  return NGB_OK;
}

int ngb_finalize(ngb_sim* s) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  rc = finalize_impl(s);
  if (rc != NGB_OK) s->failed = true;
  return rc;
}

int ngb_simulate(ngb_sim* s, int64_t steps) {
  const int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  return simulate_impl(s, steps, false, nullptr, nullptr);
}

int ngb_simulate_profiled(ngb_sim* s, int64_t steps, double* kernel_ms, int64_t* launches) {
  const int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  return simulate_impl(s, steps, true, kernel_ms, launches);
}

int ngb_autotune(ngb_sim* s, int64_t trial_steps, int32_t* deliver_grid_out) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (trial_steps < 0) return fail(NGB_ERR_INVALID_ARG, "ngb_autotune: trial_steps < 0");
  if (!s->finalized) {
    rc = finalize_impl(s);
    if (rc != NGB_OK) {
      s->failed = true;
      return rc;
    }
  }
  if (trial_steps == 0) trial_steps = 500;
  int dev = 0, sms = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const std::string key = tune_key(s);
  const char* cache = std::getenv("NGB_AUTOTUNE_CACHE");
  if (cache && *cache) {
    std::ifstream in(cache);
    std::string k;
    int m = 0, g = 0, pg = 0;
    while (in >> k >> m >> g >> pg) {
      if (k == key && g > 0 && (m == 0 || (s->persist_ok && pg > 0))) {
        s->mode = m;
        s->deliver_grid = g;
        if (pg > 0) s->persist_grid = pg;
        rc = capture_graph(s);
        if (rc == NGB_OK && deliver_grid_out) *deliver_grid_out = m == 1 ? s->persist_grid : g;
        return rc;
      }
    }
  }
  Snapshot sn;
  rc = snapshot_take(s, sn);
  if (rc != NGB_OK) {
    snapshot_free(sn);
    return rc;
  }
  const int saved_graph_steps = s->graph_steps;
  if (s->graph_steps <= 0) s->graph_steps = 100;
  int best_mode = 0, best_grid = s->deliver_grid, best_pgrid = s->persist_grid;
  double best_ms = 1e30;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // per-step kernels in graphs: delivery blocks per SM
  for (int b : {1, 2, 4, 8}) {
    s->deliver_grid = b * sms;
    rc = capture_graph(s);
    if (rc == NGB_OK) rc = snapshot_restore(s, sn);
    if (rc != NGB_OK) break;
    const int64_t reps = std::max<int64_t>(1, trial_steps / s->graph_steps);
    CK(cudaGraphLaunch(s->gexec, s->stream));  // warm-up replay
    CK(cudaEventRecord(e0, s->stream));
    for (int64_t r = 0; r < reps; ++r) CK(cudaGraphLaunch(s->gexec, s->stream));
    CK(cudaEventRecord(e1, s->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    const double per_step = ms / (double)(reps * s->graph_steps);
    if (per_step < best_ms) {
      best_ms = per_step;
      best_mode = 0;
      best_grid = s->deliver_grid;
    }
  }
  // persistent step kernel: blocks per SM
  if (rc == NGB_OK && s->persist_ok) {
    for (int b : {1, 2, 4}) {
      if (b > s->persist_max_bpsm) break;
      s->persist_grid = b * sms;
      rc = snapshot_restore(s, sn);
      if (rc != NGB_OK) break;
      CK(launch_persistent_chunk(s, 100));  // warm-up
      CK(cudaEventRecord(e0, s->stream));
      CK(launch_persistent_chunk(s, trial_steps));
      CK(cudaEventRecord(e1, s->stream));
      CK(cudaEventSynchronize(e1));
      uint32_t err = 0;
      CK(cudaMemcpy(&err, s->sb.err, sizeof(err), cudaMemcpyDeviceToHost));
      if (err & kErrBarrierTimeout) continue;  // never chosen; the snapshot restores the flags
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      const double per_step = ms / (double)trial_steps;
      if (per_step < best_ms) {
        best_ms = per_step;
        best_mode = 1;
        best_pgrid = s->persist_grid;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == NGB_OK) rc = snapshot_restore(s, sn);
  snapshot_free(sn);
  s->graph_steps = saved_graph_steps;
  s->deliver_grid = best_grid;
  s->persist_grid = best_pgrid;
  s->mode = best_mode;
  if (rc == NGB_OK) rc = capture_graph(s);
  if (rc != NGB_OK) return rc;
  if (cache && *cache) {
    std::ofstream out(cache, std::ios::app);
    out << key << " " << best_mode << " " << best_grid << " " << (s->persist_ok ? best_pgrid : 0) << "\n";
  }
  if (deliver_grid_out) *deliver_grid_out = best_mode == 1 ? best_pgrid : best_grid;
  return NGB_OK;
}

int ngb_get_spikes(ngb_sim* s, int32_t pop, int64_t t0_step, int64_t t1_step, int32_t* ids, int64_t* steps,
                   int64_t capacity, int64_t* n_out) {
  if (!s || !n_out) return fail(NGB_ERR_INVALID_ARG, "ngb_get_spikes: NULL argument");
  if (pop < -1 || pop >= (int32_t)s->pops.size()) return fail(NGB_ERR_INVALID_ARG, "ngb_get_spikes: pop");
  if (ids && (!steps || capacity < 0)) return fail(NGB_ERR_INVALID_ARG, "ngb_get_spikes: output buffers");
  if (s->rec_sorted_upto < s->rec_ids.size()) {
    // every drain appends spikes of later steps than all earlier drains, so
    // sorting the new tail keeps the whole record sorted by (step, id)
    const size_t a = s->rec_sorted_upto, n = s->rec_ids.size() - a;
    std::vector<size_t> idx(n);
    for (size_t i = 0; i < n; ++i) idx[i] = a + i;
    std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
      if (s->rec_steps[x] != s->rec_steps[y]) return s->rec_steps[x] < s->rec_steps[y];
      return s->rec_ids[x] < s->rec_ids[y];
    });
    std::vector<uint32_t> ni(n);
    std::vector<int64_t> ns(n);
    for (size_t i = 0; i < n; ++i) {
      ni[i] = s->rec_ids[idx[i]];
      ns[i] = s->rec_steps[idx[i]];
    }
    std::copy(ni.begin(), ni.end(), s->rec_ids.begin() + a);
    std::copy(ns.begin(), ns.end(), s->rec_steps.begin() + a);
    s->rec_sorted_upto = s->rec_ids.size();
  }
  const int64_t lo = pop >= 0 ? s->pops[pop].offset : 0;
  const int64_t hi = pop >= 0 ? s->pops[pop].offset + s->pops[pop].n : s->N;
  const auto first = std::lower_bound(s->rec_steps.begin(), s->rec_steps.end(), t0_step);
  const auto last = std::lower_bound(s->rec_steps.begin(), s->rec_steps.end(), t1_step);
  int64_t n = 0;
  for (auto it = first; it < last; ++it) {
    const size_t i = (size_t)(it - s->rec_steps.begin());
    const int64_t id = s->rec_ids[i];
    if (id < lo || id >= hi) continue;
    if (ids && n < capacity) {
      ids[n] = (int32_t)(id - (pop >= 0 ? lo : 0));
      steps[n] = s->rec_steps[i];
    }
    ++n;
  }
  *n_out = n;
  return NGB_OK;
}

int ngb_get_stats(ngb_sim* s, ngb_stats* out) {
  if (!s || !out) return fail(NGB_ERR_INVALID_ARG, "ngb_get_stats: NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->steps = s->t;
  out->num_neurons = s->N;
  out->spikes = s->spikes_total;
  if (s->finalized) {
    const int rc = check_handle(s);
    if (rc != NGB_OK) return rc;
    unsigned long long c[2] = {0, 0};
    CK(cudaMemcpyAsync(c, s->sb.events, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    out->events = (int64_t)c[0];
    out->rk_substeps = (int64_t)c[1];
    out->num_synapses = (int64_t)s->K;
    out->num_groups = (int64_t)s->G;
    out->ring_slots = s->L;
    out->max_delay_steps = s->max_delay;
    out->device_bytes = (int64_t)s->dev_bytes;
    out->mode = s->mode;
    out->launch_grid = s->mode == 1 ? s->persist_grid : s->deliver_grid;
  }
  return NGB_OK;
}

int ngb_population_range(ngb_sim* s, int32_t pop, int64_t* offset_out, int64_t* n_out) {
  if (!s || pop < 0 || pop >= (int32_t)s->pops.size())
    return fail(NGB_ERR_INVALID_ARG, "ngb_population_range: pop");
  if (offset_out) *offset_out = s->pops[pop].offset;
  if (n_out) *n_out = s->pops[pop].n;
  return NGB_OK;
}

int ngb_get_state(ngb_sim* s, int32_t var, int64_t first, int64_t n, float* out) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->finalized) return fail(NGB_ERR_STATE, "ngb_get_state: not finalised");
  if (!out || first < 0 || n < 0 || first + n > s->N) return fail(NGB_ERR_INVALID_ARG, "ngb_get_state: range");
  const float* src = nullptr;
  bool is_ref = false;
  switch (var) {
    case NGB_VAR_V_M: src = s->st0; break;
    case NGB_VAR_I_SYN: src = s->st1; break;
    case NGB_VAR_G_EX: src = s->st2; break;
    case NGB_VAR_G_IN: src = s->st3; break;
    case NGB_VAR_H: src = s->st4; break;
    case NGB_VAR_REFRACT: is_ref = true; break;
    default: return fail(NGB_ERR_INVALID_ARG, "ngb_get_state: var");
  }
  if (!is_ref && !src) return fail(NGB_ERR_INVALID_ARG, "ngb_get_state: variable not present in this network");
  if (n == 0) return NGB_OK;
  if (is_ref) {
    std::vector<int32_t> tmp((size_t)n);
    CK(cudaMemcpyAsync(tmp.data(), s->ref + first, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < n; ++i) out[i] = (float)tmp[(size_t)i];
  } else {
    CK(cudaMemcpyAsync(out, src + first, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  if (var == NGB_VAR_V_M) {  // LIF keeps V - E_L
    for (size_t p = 0; p < s->pops.size(); ++p) {
      const PopHost& P = s->pops[p];
      if (P.model != NGB_LIF_PSC_EXP) continue;
      const int64_t lo = std::max(first, P.offset), hi = std::min(first + n, P.offset + P.n);
      for (int64_t i = lo; i < hi; ++i) out[i - first] = (float)((double)out[i - first] + P.lif.E_L_mV);
    }
  }
  return NGB_OK;
}

int ngb_get_input(ngb_sim* s, int32_t receptor, int64_t step_offset, int64_t first, int64_t n, float* out) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->finalized) return fail(NGB_ERR_STATE, "ngb_get_input: not finalised");
  if (!out || receptor < 0 || receptor >= s->R || step_offset < 0 || step_offset >= s->L || first < 0 || n < 0 ||
      first + n > s->N)
    return fail(NGB_ERR_INVALID_ARG, "ngb_get_input: range");
  if (n == 0) return NGB_OK;
  const uint64_t slot = (uint64_t)((s->t + step_offset) & (s->L - 1));
  const uint64_t off = (slot * (uint64_t)s->R + (uint64_t)receptor) * (uint64_t)s->N + (uint64_t)first;
  if (s->cfg.deterministic) {
    std::vector<long long> tmp((size_t)n);
    CK(cudaMemcpyAsync(tmp.data(), (long long*)s->ring + off, n * sizeof(long long), cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < n; ++i) out[i] = (float)((double)tmp[(size_t)i] * 2.3283064365386963e-10);
  } else {
    CK(cudaMemcpyAsync(out, (float*)s->ring + off, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  return NGB_OK;
}

int ngb_get_src_ptr(ngb_sim* s, uint64_t* src_ptr) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->finalized) return fail(NGB_ERR_STATE, "ngb_get_src_ptr: not finalised");
  if (!src_ptr) return fail(NGB_ERR_INVALID_ARG, "ngb_get_src_ptr: NULL");
  CK(cudaMemcpyAsync(src_ptr, s->src_syn, (s->N + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return NGB_OK;
}

int ngb_get_synapses(ngb_sim* s, int64_t first, int64_t n, uint32_t* tgt, uint8_t* receptor, float* weight,
                     uint16_t* delay) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->finalized) return fail(NGB_ERR_STATE, "ngb_get_synapses: not finalised");
  if (first < 0 || n < 0 || (uint64_t)(first + n) > s->K) return fail(NGB_ERR_INVALID_ARG, "ngb_get_synapses: range");
  if (n == 0) return NGB_OK;
  // decode on the device into a temporary buffer, then one copy per field
  const size_t bytes = (size_t)n * (4 + 1 + 4 + 2) + 64;
  uint8_t* tmp = nullptr;
  CK(cudaMalloc(&tmp, bytes));
  uint32_t* d_t = reinterpret_cast<uint32_t*>(tmp);
  float* d_w = reinterpret_cast<float*>(tmp + (size_t)n * 4);
  uint16_t* d_d = reinterpret_cast<uint16_t*>(tmp + (size_t)n * 8);
  uint8_t* d_r = tmp + (size_t)n * 10;
  cudaError_t e = expand_synapses((uint64_t)first, (uint64_t)n, s->tgt, s->w, s->cfg.weight_dtype, s->grp_start,
                                  s->G, s->grp_delay, d_t, d_r, d_w, d_d, s->stream);
  if (e == cudaSuccess && tgt) e = cudaMemcpyAsync(tgt, d_t, n * 4, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && weight) e = cudaMemcpyAsync(weight, d_w, n * 4, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && delay) e = cudaMemcpyAsync(delay, d_d, n * 2, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && receptor) e = cudaMemcpyAsync(receptor, d_r, n, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "ngb_get_synapses");
  return NGB_OK;
}

}  // extern "C"
