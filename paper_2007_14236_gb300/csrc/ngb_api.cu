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
//
// Delivery scheme (ngb_sim_config.delivery): the ring scheme scatters each
// spike at once into ring slots t + d (L slots); the spike-buffer scheme of
// Sec. 2.2 keeps spikes pending until their next connection group is due and
// scatters into one slot (the next step's input).  Automatic choice: the
// spike buffer when the L-slot ring would not fit in half the L2 cache;
// ngb_autotune may also time both while the simulation is at step 0.
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

// First-fit allocator of ranges in a pool (neurons, synapses, groups).
struct RangeAlloc {
  uint64_t cap = 0;
  std::vector<std::pair<uint64_t, uint64_t>> free_;  // (offset, length), sorted by offset
  void init(uint64_t c) {
    cap = c;
    free_.clear();
    if (c) free_.push_back({0, c});
  }
  bool alloc(uint64_t n, uint64_t* off) {
    if (n == 0) {
      *off = 0;
      return true;
    }
    for (size_t i = 0; i < free_.size(); ++i) {
      if (free_[i].second >= n) {
        *off = free_[i].first;
        free_[i].first += n;
        free_[i].second -= n;
        if (free_[i].second == 0) free_.erase(free_.begin() + i);
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    if (n == 0) return;
    auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, (uint64_t)0));
    it = free_.insert(it, {off, n});
    size_t i = (size_t)(it - free_.begin());
    if (i + 1 < free_.size() && free_[i].first + free_[i].second == free_[i + 1].first) {
      free_[i].second += free_[i + 1].second;
      free_.erase(free_.begin() + i + 1);
    }
    if (i > 0 && free_[i - 1].first + free_[i - 1].second == free_[i].first) {
      free_[i - 1].second += free_[i].second;
      free_.erase(free_.begin() + i);
    }
  }
};

struct PopHost {
  int model;
  int instance;
  int64_t n;
  int64_t offset;      // global id of the first neuron (pool position once placed)
  uint32_t local_off;  // instance-local id of the first neuron
  ngb_lif_params lif;
  ngb_aeif_params aeif;
  bool placed = false;           // neuron range allocated and initialised
  uint64_t k_off = 0, k_len = 0;  // outgoing synapses in the synapse pool
  uint64_t g_off = 0, g_len = 0;  // their delay groups in the group pool
};

// Synaptic receptors of a population's model: ports a synapse may target.
int ports_of(const PopHost& p) {
  if (p.model == NGB_LIF_PSC_EXP) return 1;
  return p.model == NGB_AEIF_COND_BETA ? p.aeif.n_ports : 2;
}
// Receptor planes the ring needs for it (AdEx kernels read at least two).
int receptors_of(const PopHost& p) { return p.model == NGB_LIF_PSC_EXP ? 1 : std::max(2, ports_of(p)); }

struct InstHost {
  uint64_t seed;
  int64_t n;
  uint32_t n_calls;
  int64_t t0;
  int state = 0;  // 0 pending, 1 active, 2 retired
};

struct CallHost {
  int src_pop, tgt_pop;
  ngb_conn_spec conn;
  ngb_syn_spec syn;
  uint32_t stream;
  int stdp = 0;  // STDP rule + 1 (0: static synapses)
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

// Synapses of one connect call (Sec. 2.1 connection rules).
uint64_t call_synapses(const ngb_conn_spec& c, int64_t ns, int64_t nt, bool same) {
  switch (c.rule) {
    case NGB_RULE_FIXED_INDEGREE: return (uint64_t)c.K * (uint64_t)nt;
    case NGB_RULE_FIXED_OUTDEGREE: return (uint64_t)c.K * (uint64_t)ns;
    case NGB_RULE_ONE_TO_ONE: return (uint64_t)ns;
    case NGB_RULE_ALL_TO_ALL:
      return same && !c.allow_autapses ? (uint64_t)ns * (uint64_t)(ns - 1) : (uint64_t)ns * (uint64_t)nt;
    default: return (uint64_t)c.K;
  }
}

// device counter words: ctr[2], events, substeps, rec_count, hot_steps, pcnt[2], dcnt[6], ctr3[3], spare,
// post_cnt[2]
constexpr int kCounters = 20;

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Jump of x per unit weight for a beta-function conductance with rise time
// tr and decay time td (Sec. 2.1 multisynapse model): after x jumps by 1, g
// follows (e^(-t/td) - e^(-t/tr)) / (1/tr - 1/td), peaking at
// t_peak = tr td ln(td / tr) / (td - tr); the jump is the reciprocal of that
// peak, so a weight-W input peaks at W.  Equal times give g = t e^(-t/td),
// peak td / e at t = td, hence the jump e / td (the alpha function).
double beta_jump(double tr, double td) {
  constexpr double kE = 2.718281828459045;
  if (tr == td) return kE / td;
  const double t_peak = tr * td * std::log(td / tr) / (td - tr);
  const double peak = (std::exp(-t_peak / td) - std::exp(-t_peak / tr)) / (1.0 / tr - 1.0 / td);
  return 1.0 / peak;
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
  float *st5 = nullptr, *st6 = nullptr;  // AdEx alpha conductances: x_ex, x_in
  float* ext = nullptr;                  // beta ports 2-3: [4][N_cap] g_2, g_3, x_2, x_3 (R > 2)
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
  uint2* src_age = nullptr;  // first-group data per source (spike-buffer scheme)
  int scheme = 1;            // 1 ring, 2 spike buffer
  SegTable<LifSeg> lif_tab{};
  int n_lif = 0;
  int64_t lif_blocks = 0;
  int lif_npt = 1;  // LIF neurons per thread of the per-step update kernel (1, 2 or 4)
  SegTable<AeifSeg> aeif_tab{};   // AdEx segments with exponential conductances
  SegTable<AeifSeg> aeifa_tab{};  // AdEx segments with alpha-function conductances
  SegTable<AeifSeg> aeifb_tab{};  // beta multisynapse AdEx segments
  int n_aeif = 0;                 // AdEx segments of all kinds
  int n_aeif_exp = 0, n_aeif_alpha = 0, n_aeif_beta = 0;
  int64_t aeif_blocks = 0, aeifa_blocks = 0, aeifb_blocks = 0;
  int aeif_budget = 8;  // RK attempts per neuron in the AdEx update kernel before deferral (0: none)
  // hot lists of the AdEx update kernels: a neuron whose step ends above V_T + hot_c * Delta_T runs its next
  // step in a warp of listed neurons from the start of the update kernel (off: budget 0 or NGB_AEIF_HOT=0)
  bool hot_on = true;   // lists allocated
  bool hot_use = true;  // and used by the step loop (the autotuner may turn them off)
  float hot_c = 4.0f;
  bool hot_kind[3] = {false, false, false};  // a list per conductance model with a finite V_hot
  uint32_t* thr = nullptr;
  int deliver_grid = 0;
  bool pdl = true;  // programmatic dependent launch between the step's kernels
  bool pdl_hold = false;  // the next kernel follows a join from another stream: launch it without PDL
  int mode = 0;  // 0: per-step kernels in CUDA graphs, 1: persistent step kernel, 2: fused update + delivery,
                 // 3: pipelined (delivery of step t beside the update of step t + 1, two streams),
                 // 4: pipelined persistent step kernel (ring scheme, one grid barrier per step),
                 // 5: pipelined, one kernel per step (LIF networks: update and delivery of the
                 //    previous step's queue in the same launch, chained by programmatic dependent launch),
                 // 6: target-owned persistent kernel (LIF networks, ring scheme: each block owns a tile
                 //    of neurons with its ring in shared memory; spikes exchanged through mailboxes),
                 // 7: per-step kernels in CUDA graphs with target-tiled delivery (spike-buffer scheme)
  cudaStream_t stream2 = nullptr;  // second stream of the pipelined loop's graphs
  cudaStream_t hstream = nullptr;  // stream of the AdEx hot-list kernels (highest priority)
  cudaEvent_t hev[2] = {nullptr, nullptr};  // fork to and join from it
  bool persist_ok = false;
  int persist_grid = 0;
  int persist_max_bpsm = 0;
  size_t persist_smem = 0;
  PersistArgs pa{};
  unsigned* bar = nullptr;
  uint32_t n_thr_total = 0;
  bool serving = false;   // pools reserved by ngb_reserve; instances committed and retired while running
  int64_t N_cap = 0;
  uint64_t K_cap = 0, G_cap = 0;
  RangeAlloc nalloc, kalloc, galloc;
  bool tables_dirty = true;
  std::vector<void*> table_allocs;  // segment and Poisson tables, rebuilt when instances change
  int64_t n_active = 0;
  int sms = 0;
  uint64_t work_items = 0;  // delivery work items of all sources (map capacity)
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  int drain_steps = 1000;
  int64_t t = 0;  // steps done
  int64_t spikes_total = 0;
  // device-side sort of each drained record (keys step << 26 | neuron) and
  // its pinned host staging buffer
  unsigned long long* rec_keys = nullptr;
  unsigned long long* rec_sorted = nullptr;
  unsigned char* rec_sort_tmp = nullptr;
  size_t rec_sort_bytes = 0;
  unsigned long long* rec_pinned = nullptr;
  std::vector<uint32_t> rec_ids;
  std::vector<int64_t> rec_steps;
  size_t rec_sorted_upto = 0;  // records [0, upto) are sorted by (step, id)
  std::vector<double> pop_E_L;  // per population, for V of LIF (state holds V - E_L)
  // STDP (Sec. 2.1): rules of the plastic connect calls, their device table,
  // the latest arrival step of every synapse and the reverse index
  std::vector<ngb_stdp_params> stdp_params;
  StdpRule* d_rules = nullptr;
  uint2* wa = nullptr;  // per synapse {FP32 weight bits, latest arrival step}
  uint64_t* in_ptr = nullptr;
  uint64_t* in_syn = nullptr;
  uint64_t n_plastic = 0;
  // target-owned loop (mode 6): tile-major synapse layout (built on first
  // use), mailboxes, overflow areas and the launch shape
  bool lif_contig = false;  // LIF segments contiguous from neuron 0 (the kernel's segment search)
  bool own_tried = false;
  // target-tiled delivery (mode 7: per-step kernels in CUDA graphs, spike-buffer
  // scheme, due groups accumulated per target tile in shared memory): the
  // layout (built on first use, for one tile size) and blocks per tile
  TiledLayout tl{};
  uint32_t tl_P = 1;
  OwnedLayout own{};
  unsigned long long* own_mb = nullptr;
  unsigned long long* own_ovf = nullptr;
  uint32_t own_T = 0;
  size_t own_smem = 0;

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

// The spike-buffer scheme uses one ring slot (L_mask 0).
Ring ring_of(const ngb_sim* s) {
  return Ring{s->ring, s->N_cap, (uint32_t)(s->scheme == 2 ? 0 : s->L - 1), s->R};
}

Csr csr_of(const ngb_sim* s) {
  return Csr{s->src_meta, s->src_syn, s->src_grp, s->grp_start, s->grp_delay, s->tgt, s->w, s->src_age,
             s->cfg.weight_dtype};
}

// How the update kernels hand the step's spikes to delivery.
int emit_of(const ngb_sim* s) {
  return s->scheme == 2 ? kEmitAge : ((s->mode == 3 || s->mode == 5) ? kEmitPipe : kEmitRing);
}

// The one-kernel pipelined loop takes LIF networks at one neuron per thread
// with the ring scheme.
bool pipe1_ok(const ngb_sim* s) {
  return s->scheme == 1 && s->n_aeif == 0 && s->n_lif > 0 && s->lif_npt == 1 && s->sb.wi3[0] != nullptr;
}

// The fused step loop takes one LIF neuron per thread and the two-receptor
// AdEx models.
bool fused_ok(const ngb_sim* s) { return s->lif_npt == 1 && s->n_aeif_beta == 0; }

// Programmatic dependent launch chains the kernels of one stream; the
// pipelined loop's kernels depend across two streams and go without it.
bool pdl_of(const ngb_sim* s) { return s->pdl && s->mode != 3 && !s->pdl_hold; }

// pdl_of for a kernel launch that consumes a pending hold (the first kernel
// after a join from another stream waits for that stream's work in full).
bool take_pdl(ngb_sim* s) {
  const bool p = pdl_of(s);
  s->pdl_hold = false;
  return p;
}

// Empty the AdEx hot lists and clear the neurons' tags: after steps run by a
// loop that does not keep them (persistent, fused), a restored snapshot or
// rebuilt tables no neuron is listed until a step of the per-step kernels
// lists it again.
cudaError_t hot_reset(ngb_sim* s) {
  if (!s->sb.htag) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(s->sb.htag, 0xFF, (size_t)s->N_cap * sizeof(uint32_t), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->sb.hcnt, 0, 9 * sizeof(unsigned long long), s->stream);
  return e;
}

// The target-owned loop takes static LIF networks with the ring scheme and
// one receptor, at most 2,048 neurons per block (one block per SM), and a
// tile ring that fits in shared memory.
bool owned_shape_ok(const ngb_sim* s, uint32_t* T_out, size_t* smem_out) {
  if (s->serving || s->scheme != 1 || s->n_aeif || !s->n_lif || s->d_rules || s->R != 1 || !s->lif_contig ||
      s->sms <= 0 || s->sms * 8 > 4 * 512 || s->n_lif > 64 || s->N <= 0)
    return false;
  const int64_t T = (s->N + s->sms - 1) / s->sms;
  if (T > 2048) return false;
  const size_t smem = owned_smem_bytes(s->cfg.deterministic != 0, (uint32_t)s->L, (uint32_t)T, s->n_lif, s->pa.n_thr);
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->cfg.device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (smem + 4096 > (size_t)optin) return false;
  *T_out = (uint32_t)T;
  *smem_out = smem;
  return true;
}

// Whether the target-owned loop can run; builds its synapse layout on the
// first call (at most half of the free device memory; a failure leaves the
// loop unavailable, not the handle).
bool owned_ready(ngb_sim* s) {
  uint32_t T = 0;
  size_t smem = 0;
  if (!owned_shape_ok(s, &T, &smem)) return false;
  if (s->own.items) return true;
  if (s->own_tried) return false;
  s->own_tried = true;
  int bpsm = 0;
  if (owned_max_blocks_per_sm(s->cfg.deterministic != 0, T, smem, 0, &bpsm) != cudaSuccess || bpsm < 1) {
    cudaGetLastError();
    return false;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  OwnedLayout L{};
  cudaError_t e = owned_build(csr_of(s), s->src_syn, s->N, s->sms, (uint32_t)s->L, (uint64_t)(free_b / 2), &L,
                              s->stream);
  if (e != cudaSuccess || !L.items) {
    cudaGetLastError();
    return false;
  }
  s->allocs.push_back(L.items);
  s->allocs.push_back(L.pub);
  s->dev_bytes += (size_t)L.G * L.S * (L.wfmt ? 4 : 8) + (size_t)s->N * sizeof(uint64_t);
  if (s->dalloc(&s->own_mb, (size_t)4 * L.G * 8) != cudaSuccess ||
      s->dalloc(&s->own_ovf, (size_t)4 * L.G * T) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s->own = L;
  s->own_T = T;
  s->own_smem = smem;
  return true;
}

// One target-owned launch per kMaxOwnedSteps steps, each with fresh
// mailboxes, overflow areas and abort word.
cudaError_t launch_owned_chunk(ngb_sim* s, int64_t steps) {
  cudaError_t e = cudaSuccess;
  while (steps > 0 && e == cudaSuccess) {
    const int64_t n = std::min<int64_t>(steps, kMaxOwnedSteps);
    e = cudaMemsetAsync(s->bar, 0, 4 * sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->own_mb, 0xFF, (size_t)4 * s->own.G * 8 * 8, s->stream);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(s->own_ovf, 0xFF, (size_t)4 * s->own.G * s->own_T * 8, s->stream);
    if (e != cudaSuccess) break;
    OwnedArgs a{};
    a.seg = s->lif_tab.dev;
    a.thr = s->thr;
    a.y = s->st0;
    a.I = s->st1;
    a.ref = s->ref;
    a.ring = s->ring;
    a.ring_N = s->N_cap;
    a.N = s->N;
    a.items = s->own.items;
    a.wfmt = s->own.wfmt;
    a.pub = s->own.pub;
    a.src_syn = s->src_syn;
    a.mb = s->own_mb;
    a.ovf = s->own_ovf;
    a.sb = s->sb;
    a.clk = s->clk;
    a.abort = s->bar + 2;
    a.steps = n;
    a.S = s->own.S;
    a.spin_limit = s->pa.spin_limit;
    a.T = s->own_T;
    a.L_mask = (uint32_t)(s->L - 1);
    a.n_thr = s->pa.n_thr;
    a.n_seg = s->n_lif;
    a.withhold_block = s->pa.withhold_block;
    e = launch_owned(a, s->cfg.deterministic != 0, s->own.G, s->stream);
    steps -= n;
  }
  return e;
}

// Target-tiled delivery takes static networks with the spike-buffer scheme
// and no plastic synapses.
bool tiled_shape_ok(const ngb_sim* s) {
  return !s->serving && s->scheme == 2 && !s->d_rules && s->G > 0 && s->N > 0 && s->R >= 1 && s->R <= kMaxPorts;
}

// Largest tile (neurons) whose accumulators fit 64 KB of shared memory.
uint32_t tiled_max_T(const ngb_sim* s) {
  return (uint32_t)(65536 / ((size_t)s->R * (s->cfg.deterministic ? 8 : 4)));
}

// Build the tiled layout for tiles of T neurons (replacing one of another
// tile size); at most half of the free device memory.  A failure leaves the
// layout absent, not the handle.
bool tiled_ready(ngb_sim* s, uint32_t T) {
  if (!tiled_shape_ok(s) || T < 32 || T > tiled_max_T(s)) return false;
  if (s->tl.pairs && s->tl.T == T) return true;
  if (s->tl.pairs) {
    s->dev_bytes -= s->tl.bytes;
    tiled_free(&s->tl);
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  TiledLayout L{};
  cudaError_t e = tiled_build(s->grp_start, s->G, s->tgt, s->w, s->cfg.weight_dtype, s->K, s->N, T,
                              (uint64_t)(free_b / 2), &L, s->stream);
  if (e != cudaSuccess || !L.pairs) {
    cudaGetLastError();
    return false;
  }
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->cfg.device) != cudaSuccess ||
      tiled_smem_bytes(s->cfg.deterministic != 0, s->R, T, L.n_tiles) + 1024 > (size_t)optin) {
    cudaGetLastError();
    tiled_free(&L);
    return false;
  }
  s->tl = L;
  s->dev_bytes += L.bytes;
  return true;
}

// Tile size for about `tiles` tiles (at least 32 neurons, within the shared-memory limit).
uint32_t tiled_T_for(const ngb_sim* s, int64_t tiles) {
  tiles = std::max<int64_t>(1, tiles);
  const int64_t T = std::max<int64_t>(32, (s->N + tiles - 1) / tiles);
  return (uint32_t)std::min<int64_t>(T, tiled_max_T(s));
}

// Point the update kernels' spike-buffer emission at the tiled buckets (mode
// 7) or at the plain due-item list; entering mode 7 starts with empty buckets.
void set_tiled(ngb_sim* s, bool on) {
  SpikeBuf& b = s->sb;
  if (on && s->tl.pairs) {
    b.tile_grp = s->tl.tile_grp;
    b.bkt[0] = s->tl.bkt;
    b.bkt[1] = s->tl.bkt + s->G;
    b.boff = s->tl.boff;
    b.bcnt = s->tl.bcnt;
    b.n_tiles = s->tl.n_tiles;
    cudaMemsetAsync(s->tl.bcnt, 0, (size_t)2 * s->tl.n_tiles * sizeof(unsigned int), s->stream);
  } else {
    b.tile_grp = nullptr;
    b.bkt[0] = b.bkt[1] = nullptr;
    b.boff = nullptr;
    b.bcnt = nullptr;
    b.n_tiles = 0;
  }
  s->pa.sb = s->sb;
}

// The first update kernel of the step scans the pending spikes (spike-buffer scheme).
cudaError_t launch_lif(ngb_sim* s, int64_t step_off = 0) {
  return launch_update_lif(s->lif_tab, s->lif_blocks, s->lif_npt, s->thr, s->st0, s->st1, s->ref, ring_of(s),
                           s->cfg.deterministic != 0, s->clk, step_off, csr_of(s), s->sb, emit_of(s), true,
                           take_pdl(s), s->stream);
}

AeifState aeif_state_of(const ngb_sim* s) {
  return AeifState{s->st0, s->st1, s->st2, s->st3, s->st4, s->st5, s->st6, s->ext, s->N_cap};
}

// AdEx update kernels: exponential-conductance segments, then alpha ones,
// then beta ones.  Each kind is an update kernel with an attempt budget, then
// the kernel that finishes the deferred neurons.
cudaError_t launch_aeif(ngb_sim* s, int64_t step_off = 0) {
  cudaError_t e = cudaSuccess;
  const bool det = s->cfg.deterministic != 0;
  const int emit = emit_of(s);
  const int fin_grid = std::max(1, s->sms) * 4;
  const AeifState S = aeif_state_of(s);
  const struct {
    int model, n;
    const SegTable<AeifSeg>* tab;
    int64_t blocks;
  } kinds[3] = {{kAeifExp, s->n_aeif_exp, &s->aeif_tab, s->aeif_blocks},
                {kAeifAlpha, s->n_aeif_alpha, &s->aeifa_tab, s->aeifa_blocks},
                {kAeifBeta, s->n_aeif_beta, &s->aeifb_tab, s->aeifb_blocks}};
  bool scan = s->n_lif == 0;  // the first update kernel of the step scans the pending spikes
  for (const auto& k : kinds) {
    if (!k.n || e != cudaSuccess) continue;
    // the hot list's kernel on its own stream, forked after the previous step, beside the update kernel
    const bool hot = s->hot_on && s->hot_use && s->hot_kind[k.model] && s->hstream && s->aeif_budget > 0;
    if (hot) {
      e = cudaEventRecord(s->hev[0], s->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->hstream, s->hev[0], 0);
      if (e == cudaSuccess)
        e = launch_hot_aeif(*k.tab, 4 * std::max(1, s->sms), s->thr, S, k.model, ring_of(s), det, s->clk, step_off,
                            csr_of(s), s->sb, emit, s->hstream);
      if (e == cudaSuccess) e = cudaEventRecord(s->hev[1], s->hstream);
    }
    if (e == cudaSuccess)
      e = launch_update_aeif(*k.tab, k.blocks, s->thr, S, k.model, ring_of(s), det, s->clk, step_off, csr_of(s),
                             s->sb, emit, scan, s->aeif_budget, hot, take_pdl(s), s->stream);
    if (e == cudaSuccess && s->aeif_budget > 0)
      e = launch_finish_aeif(*k.tab, fin_grid, S, k.model, ring_of(s), det, s->clk, step_off, csr_of(s), s->sb, emit,
                             hot, take_pdl(s), s->stream);
    // the hot neurons' spikes and state before anything that follows the step's updates
    if (e == cudaSuccess && hot) {
      e = cudaStreamWaitEvent(s->stream, s->hev[1], 0);
      s->pdl_hold = true;
    }
    scan = false;
  }
  return e;
}

StdpArgs stdp_of(const ngb_sim* s) { return StdpArgs{s->d_rules, s->wa, s->in_syn}; }

cudaError_t launch_del(ngb_sim* s, int64_t step_off = 0, cudaStream_t st = nullptr) {
  if (s->mode == 7)
    return launch_deliver_tiled(s->sb, s->tl, s->tl_P, s->cfg.weight_dtype, ring_of(s), s->R, s->N,
                                s->cfg.deterministic != 0, s->clk, take_pdl(s), st ? st : s->stream);
  const StdpArgs sa = stdp_of(s);
  return launch_deliver(s->sb, csr_of(s), s->cfg.weight_dtype, ring_of(s), s->cfg.deterministic != 0, emit_of(s),
                        s->clk, step_off, s->deliver_grid, take_pdl(s), st ? st : s->stream,
                        s->d_rules ? &sa : nullptr);
}

// STDP potentiation of the step's firing targets, between the update kernels and the delivery.
cudaError_t launch_post(ngb_sim* s) {
  if (!s->d_rules) return cudaSuccess;
  const bool pdl = s->pdl && !s->pdl_hold;
  s->pdl_hold = false;
  return launch_stdp_post(s->sb, stdp_of(s), s->clk, std::max(1, s->sms) * 4, pdl, s->stream);
}

// The update kernels of one step (step clk[0] + step_off).
cudaError_t launch_updates(ngb_sim* s, int64_t step_off) {
  cudaError_t e = cudaSuccess;
  if (s->n_lif) e = launch_lif(s, step_off);
  if (e == cudaSuccess && s->n_aeif) e = launch_aeif(s, step_off);
  return e;
}

// Switch the delivery scheme (only while no spike is in flight: step 0).
void set_scheme(ngb_sim* s, int scheme) {
  s->scheme = scheme;
  s->pa.ring = ring_of(s);
  s->pa.csr = csr_of(s);
  s->pa.age = scheme == 2 ? 1 : 0;
}

// Fused step loop (mode 2, ring scheme): update kernels that deliver their
// blocks' spikes; the step is clk[0] + step_off.
cudaError_t launch_fused_lif(ngb_sim* s, int64_t step_off) {
  if (!s->n_lif) return cudaSuccess;
  return launch_step_lif(s->lif_tab, s->lif_blocks, s->thr, s->st0, s->st1, s->ref, ring_of(s),
                         s->cfg.deterministic != 0, s->cfg.weight_dtype, s->clk, step_off, csr_of(s), s->sb, s->pdl,
                         s->stream);
}

cudaError_t launch_fused_aeif(ngb_sim* s, int64_t step_off) {
  cudaError_t e = cudaSuccess;
  const bool det = s->cfg.deterministic != 0;
  if (s->n_aeif_exp)
    e = launch_step_aeif(s->aeif_tab, s->aeif_blocks, s->thr, s->st0, s->st1, s->st2, s->st3, s->st4, s->st5, s->st6,
                         false, ring_of(s), det, s->cfg.weight_dtype, s->clk, step_off, csr_of(s), s->sb, s->pdl,
                         s->stream);
  if (e == cudaSuccess && s->n_aeif_alpha)
    e = launch_step_aeif(s->aeifa_tab, s->aeifa_blocks, s->thr, s->st0, s->st1, s->st2, s->st3, s->st4, s->st5,
                         s->st6, true, ring_of(s), det, s->cfg.weight_dtype, s->clk, step_off, csr_of(s), s->sb,
                         s->pdl, s->stream);
  return e;
}

cudaError_t launch_fused(ngb_sim* s, int64_t step_off) {
  cudaError_t e = launch_fused_lif(s, step_off);
  if (e == cudaSuccess) e = launch_fused_aeif(s, step_off);
  return e;
}

cudaError_t launch_step(ngb_sim* s) {
  cudaError_t e;
  if (s->mode == 2) {
    e = launch_fused(s, 0);
    if (e != cudaSuccess) return e;
    return launch_tick_add(s->clk, 1, s->sb.ctr, s->sb.ctr3, s->pdl, s->stream);
  }
  if (s->mode == 3 || s->mode == 5) {  // one pipelined step, serialised on the main stream
    e = launch_updates(s, 0);
    if (e == cudaSuccess) e = launch_del(s, 0);
    if (e != cudaSuccess) return e;
    return launch_tick_add(s->clk, 1, s->sb.ctr, s->sb.ctr3, false, s->stream);
  }
  if (!s->n_lif && !s->n_aeif) {
    e = launch_tick(s->clk, s->pdl, s->stream);
    if (e != cudaSuccess) return e;
  }
  if (s->n_lif) {
    e = launch_lif(s);
    if (e != cudaSuccess) return e;
  }
  if (s->n_aeif) {
    e = launch_aeif(s);
    if (e != cudaSuccess) return e;
  }
  e = launch_post(s);
  if (e != cudaSuccess) return e;
  return launch_del(s);
}

// One persistent launch of `steps` steps.
cudaError_t launch_persistent_chunk(ngb_sim* s, int64_t steps) {
  cudaError_t e = cudaMemsetAsync(s->bar, 0, 4 * sizeof(unsigned), s->stream);
  if (e != cudaSuccess) return e;
  // the pipelined variant starts with empty queue counters (every launch
  // delivers its last queue before it ends; steps run by other loops in
  // between leave the counters stale)
  if (s->mode == 4) e = cudaMemsetAsync(s->sb.ctr3, 0, 3 * sizeof(unsigned long long), s->stream);
  if (e != cudaSuccess) return e;
  s->pa.steps = steps;
  s->pa.sb = s->sb;
  return launch_persistent(s->pa, s->cfg.deterministic != 0, s->cfg.weight_dtype, s->n_lif > 0, s->n_aeif > 0,
                           s->mode == 4,
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
    // sorted by (step, neuron) on the device, then appended: every drain
    // holds later steps than the earlier ones, so the record stays sorted
    const size_t n = (size_t)std::min<unsigned long long>(cnt, (unsigned long long)s->sb.rec_cap);
    CK(sort_record(s->sb.rec_id, s->sb.rec_step, n, s->rec_keys, s->rec_sorted, s->rec_sort_tmp, s->rec_sort_bytes,
                   s->stream));
    CK(cudaMemcpyAsync(s->rec_pinned, s->rec_sorted, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const bool was_sorted = s->rec_sorted_upto == s->rec_ids.size();
    const size_t old = s->rec_ids.size();
    s->rec_ids.resize(old + n);
    s->rec_steps.resize(old + n);
    for (size_t i = 0; i < n; ++i) {
      const unsigned long long k = s->rec_pinned[i];
      s->rec_ids[old + i] = (uint32_t)(k & ((1ull << 26) - 1));
      s->rec_steps[old + i] = (int64_t)(k >> 26);
    }
    if (was_sorted) s->rec_sorted_upto = s->rec_ids.size();
  }
  CK(cudaMemsetAsync(s->sb.rec_count, 0, sizeof(unsigned long long), s->stream));
  CK(cudaMemsetAsync(s->sb.err, 0, sizeof(uint32_t), s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (err & kErrBarrierTimeout) {
    s->failed = true;
    return fail(NGB_ERR_TIMEOUT, "persistent step kernel: a grid barrier wait gave up (handle unusable)");
  }
  if (err & kErrPendingOverflow)
    return fail(NGB_ERR_OVERFLOW,
                "spike-buffer delivery: more spikes in flight than the pending list holds (use the ring scheme)");
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
  if (s->mode == 7 && !s->tl.pairs) s->mode = 0;
  set_tiled(s, s->mode == 7);
  if (s->graph_steps <= 0) return NGB_OK;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  std::vector<cudaEvent_t> events;
  if (s->mode == 2) {
    for (int i = 0; i < s->graph_steps && e == cudaSuccess; ++i) e = launch_fused(s, i);
    if (e == cudaSuccess) e = launch_tick_add(s->clk, s->graph_steps, s->sb.ctr, s->sb.ctr3, s->pdl, s->stream);
  } else if (s->mode == 5) {
    // One kernel per step: the update of step i and the delivery of step
    // i - 1's queue; then the last step's queue and the clock.
    const int S = s->graph_steps;
    const bool det = s->cfg.deterministic != 0;
    for (int i = 0; i < S && e == cudaSuccess; ++i)
      e = launch_step_pipe(s->lif_tab, s->lif_blocks, s->deliver_grid, s->thr, s->st0, s->st1, s->ref, ring_of(s), det,
                           s->cfg.weight_dtype, s->clk, i, csr_of(s), s->sb, i > 0, s->pdl, s->stream);
    if (e == cudaSuccess)
      e = launch_deliver(s->sb, csr_of(s), s->cfg.weight_dtype, ring_of(s), det, kEmitPipe, s->clk, S - 1,
                         s->deliver_grid, s->pdl, s->stream);
    if (e == cudaSuccess) e = launch_tick_add(s->clk, S, s->sb.ctr, s->sb.ctr3, s->pdl, s->stream);
  } else if (s->mode == 3) {
    // Pipelined: the updates of the steps on the main stream, their
    // deliveries on the second; the update of step i waits for the delivery
    // of step i - 2 (the delivery of step i - 1 lands in slots i + 1 and
    // later), the delivery of step i for the update of step i.
    const int S = s->graph_steps;
    events.resize((size_t)(2 * S + 1), nullptr);
    for (auto& ev : events)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(events[(size_t)(2 * S)], s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream2, events[(size_t)(2 * S)], 0);
    for (int i = 0; i < S && e == cudaSuccess; ++i) {
      cudaEvent_t eu = events[(size_t)(2 * i)], ed = events[(size_t)(2 * i + 1)];
      if (i >= 2) e = cudaStreamWaitEvent(s->stream, events[(size_t)(2 * (i - 2) + 1)], 0);
      if (e == cudaSuccess) e = launch_updates(s, i);
      if (e == cudaSuccess) e = cudaEventRecord(eu, s->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream2, eu, 0);
      if (e == cudaSuccess) e = launch_del(s, i, s->stream2);
      if (e == cudaSuccess) e = cudaEventRecord(ed, s->stream2);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, events[(size_t)(2 * (S - 1) + 1)], 0);
    if (e == cudaSuccess) e = launch_tick_add(s->clk, S, s->sb.ctr, s->sb.ctr3, false, s->stream);
  } else {
    for (int i = 0; i < s->graph_steps && e == cudaSuccess; ++i) e = launch_step(s);
  }
  cudaError_t e2 = cudaStreamEndCapture(s->stream, &graph);
  for (cudaEvent_t ev : events)
    if (ev) cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture (kernel launch)");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&s->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return NGB_OK;
}

// ---------------------------------------------------------------------------
// Network construction into pools.  A population is placed at a neuron range
// of the pool; its outgoing synapses occupy a range of the synapse pool and
// their delay groups a range of the group pool.  A static network places all
// populations in creation order at ngb_finalize (so the pools are exactly
// full and contiguous); a serving handle (ngb_reserve) places each instance
// when it is committed and frees its ranges when it is retired.
// ---------------------------------------------------------------------------
struct PopParts {
  int pop;
  uint64_t* gs;
  uint16_t* gd;
  uint64_t G;
  unsigned long long* cnt_scan;  // n + 1
  unsigned long long* grp_scan;  // n + 1
};

void free_parts(std::vector<PopParts>& parts) {
  for (PopParts& q : parts) {
    cudaFree(q.gs);
    cudaFree(q.gd);
    cudaFree(q.cnt_scan);
    cudaFree(q.grp_scan);
  }
  parts.clear();
}

// Place the population's neurons (serving handles allocate the range) and
// initialise their state; in a serving handle also clear their ring columns.
int place_population(ngb_sim* s, int pi) {
  PopHost& p = s->pops[(size_t)pi];
  cudaStream_t st = s->stream;
  uint64_t off = 0;
  if (!s->nalloc.alloc((uint64_t)p.n, &off))
    return fail(NGB_ERR_OOM, "neuron pool full (ngb_reserve max_neurons)");
  if (!s->serving && (int64_t)off != p.offset) return fail(NGB_ERR_STATE, "internal: population placement");
  p.offset = (int64_t)off;
  const uint64_t seed = s->inst[(size_t)p.instance].seed;
  CK(cudaMemsetAsync(s->st1 + off, 0, p.n * sizeof(float), st));
  CK(cudaMemsetAsync(s->ref + off, 0, p.n * sizeof(int32_t), st));
  if (p.model == NGB_LIF_PSC_EXP) {
    const ngb_lif_params& q = p.lif;
    CK(launch_init_state(0, p.n, q.V_init_mean_mV, q.V_init_sd_mV, q.E_L_mV, 0.0, 0.0, seed, p.local_off,
                         s->st0 + off, nullptr, nullptr, st));
  } else {
    const ngb_aeif_params& q = p.aeif;
    CK(cudaMemsetAsync(s->st2 + off, 0, p.n * sizeof(float), st));
    CK(cudaMemsetAsync(s->st3 + off, 0, p.n * sizeof(float), st));
    CK(cudaMemsetAsync(s->st5 + off, 0, p.n * sizeof(float), st));
    CK(cudaMemsetAsync(s->st6 + off, 0, p.n * sizeof(float), st));
    if (s->ext)
      CK(cudaMemset2DAsync(s->ext + off, (size_t)s->N_cap * sizeof(float), 0, (size_t)p.n * sizeof(float), 4, st));
    CK(launch_init_state(1, p.n, q.V_init_mean_mV, q.V_init_sd_mV, q.E_L_mV, q.w_init_pA, q.rk_h_init_ms, seed,
                         p.local_off, s->st0 + off, s->st1 + off, s->st4 + off, st));
  }
  if (s->serving && s->ring) {
    const size_t es = s->cfg.deterministic ? 8 : 4;
    CK(cudaMemset2DAsync((uint8_t*)s->ring + off * es, (size_t)s->N_cap * es, 0, (size_t)p.n * es,
                         (size_t)(s->L * s->R), st));
  }
  p.placed = true;
  return NGB_OK;
}

// Draw, sort and gather the outgoing synapses of the source populations
// `srcs` (Sec. 2.1 rules, Sec. 2.2 delay groups) into the synapse pool.
int build_populations(ngb_sim* s, const std::vector<int>& srcs, std::vector<PopParts>& parts, int* max_delay_out,
                      uint64_t* running_k) {
  cudaStream_t st = s->stream;
  const double dt = s->cfg.dt_ms;
  const int prec = s->cfg.weight_dtype;
  const size_t wsize = prec == NGB_WEIGHT_FP32 ? 4 : 2;
  std::vector<std::vector<CallDev>> by_src(srcs.size());
  std::vector<uint64_t> n_by_src(srcs.size(), 0);
  uint64_t kmax = 0;
  int max_bits = 1;
  for (size_t i = 0; i < srcs.size(); ++i) {
    const PopHost& ps = s->pops[(size_t)srcs[i]];
    for (const CallHost& c : s->calls) {
      if (c.src_pop != srcs[i]) continue;
      const PopHost& pt = s->pops[(size_t)c.tgt_pop];
      CallDev d{};
      d.seed = s->inst[(size_t)ps.instance].seed;
      d.K = c.conn.K;
      d.nsyn = call_synapses(c.conn, s->pops[(size_t)c.src_pop].n, pt.n, c.src_pop == c.tgt_pop);
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
      d.stdp = c.stdp;
      d.prec = prec;
      d.n_src = (uint32_t)ps.n;
      d.n_tgt = (uint32_t)pt.n;
      d.src_off = 0;  // per-population count arrays
      d.tgt_off = (uint32_t)pt.offset;
      by_src[i].push_back(d);
      n_by_src[i] += d.nsyn;
    }
    if (n_by_src[i] >= (1ull << 32))
      return fail(NGB_ERR_INVALID_ARG, "more than 2^32 synapses from one population");
    kmax = std::max(kmax, n_by_src[i]);
    max_bits = std::max(max_bits, bits_for((uint64_t)ps.n));
  }
  int* dmax = nullptr;
  CK(cudaMalloc(&dmax, sizeof(int)));
  CK(cudaMemsetAsync(dmax, 0, sizeof(int), st));
  BuildScratch sc;
  size_t scan_u64_bytes = 0;
  void* scan_u64_tmp = nullptr;
  int64_t nmax = 1;
  for (int p : srcs) nmax = std::max<int64_t>(nmax, s->pops[(size_t)p].n);
  CK(scan_scratch_bytes_u64((uint64_t)nmax + 1, &scan_u64_bytes));
  CK(cudaMalloc(&scan_u64_tmp, std::max<size_t>(scan_u64_bytes, 16)));
  if (kmax > 0) {
    CK(sort_scratch_bytes(kmax, max_bits + kDelayBits, &sc.sort_bytes, &sc.scan_bytes));
    CK(cudaMalloc(&sc.keys, kmax * sizeof(unsigned long long)));
    CK(cudaMalloc(&sc.keys_alt, kmax * sizeof(unsigned long long)));
    CK(cudaMalloc(&sc.vals, kmax * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.vals_alt, kmax * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.st_tgt, kmax * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.st_w, kmax * sizeof(float)));
    CK(cudaMalloc(&sc.flag, kmax * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.gidx, kmax * sizeof(uint32_t)));
    CK(cudaMalloc(&sc.sort_tmp, std::max<size_t>(sc.sort_bytes, 16)));
    CK(cudaMalloc(&sc.scan_tmp, std::max<size_t>(sc.scan_bytes, 16)));
  }
  int rc = NGB_OK;
  for (size_t i = 0; i < srcs.size() && rc == NGB_OK; ++i) {
    PopHost& ps = s->pops[(size_t)srcs[i]];
    const uint64_t n = (uint64_t)ps.n;
    uint64_t k_off = 0;
    if (!s->kalloc.alloc(n_by_src[i], &k_off)) {
      rc = fail(NGB_ERR_OOM, "synapse pool full (ngb_reserve max_synapses)");
      break;
    }
    if (!s->serving) k_off = *running_k;  // static pools are filled in order
    *running_k += n_by_src[i];
    ps.k_off = k_off;
    ps.k_len = n_by_src[i];
    PopParts q{srcs[i], nullptr, nullptr, 0, nullptr, nullptr};
    unsigned long long *cnt = nullptr, *ngrp = nullptr;
    CK(cudaMalloc(&cnt, (n + 1) * sizeof(unsigned long long)));
    CK(cudaMalloc(&ngrp, (n + 1) * sizeof(unsigned long long)));
    CK(cudaMalloc(&q.cnt_scan, (n + 1) * sizeof(unsigned long long)));
    CK(cudaMalloc(&q.grp_scan, (n + 1) * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(cnt, 0, (n + 1) * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(ngrp, 0, (n + 1) * sizeof(unsigned long long), st));
    if (n_by_src[i] > 0) {
      std::string err;
      cudaError_t e = build_source_population(by_src[i], n_by_src[i], bits_for(n), k_off, prec, sc, s->tgt + k_off,
                                              (uint8_t*)s->w + k_off * wsize, cnt, ngrp, dmax, &q.gs, &q.gd, &q.G,
                                              st, err);
      if (e != cudaSuccess) rc = cuda_fail(e, ("connection builder: " + err).c_str());
    }
    if (rc == NGB_OK) {
      cudaError_t e = exclusive_scan_u64(cnt, q.cnt_scan, n + 1, scan_u64_tmp, scan_u64_bytes, st);
      if (e == cudaSuccess) e = exclusive_scan_u64(ngrp, q.grp_scan, n + 1, scan_u64_tmp, scan_u64_bytes, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "population scans");
    }
    CK(cudaStreamSynchronize(st));
    cudaFree(cnt);
    cudaFree(ngrp);
    parts.push_back(q);
  }
  CK(cudaStreamSynchronize(st));
  cudaFree(sc.keys); cudaFree(sc.keys_alt); cudaFree(sc.vals); cudaFree(sc.vals_alt);
  cudaFree(sc.st_tgt); cudaFree(sc.st_w); cudaFree(sc.flag); cudaFree(sc.gidx);
  cudaFree(sc.sort_tmp); cudaFree(sc.scan_tmp); cudaFree(scan_u64_tmp);
  int md = 0;
  CK(cudaMemcpy(&md, dmax, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(dmax);
  *max_delay_out = md;
  return rc;
}

// Groups of the built populations into the group pool, and their per-source
// metadata (row, synapse count, group range).
int place_parts(ngb_sim* s, std::vector<PopParts>& parts, uint64_t* running_g, uint64_t* items_out) {
  cudaStream_t st = s->stream;
  unsigned long long* items = nullptr;
  CK(cudaMalloc(&items, sizeof(unsigned long long)));
  CK(cudaMemsetAsync(items, 0, sizeof(unsigned long long), st));
  int rc = NGB_OK;
  for (PopParts& q : parts) {
    PopHost& p = s->pops[(size_t)q.pop];
    uint64_t g_off = 0;
    if (!s->galloc.alloc(q.G, &g_off)) {
      rc = fail(NGB_ERR_OOM, "group pool full (ngb_reserve max_groups)");
      break;
    }
    if (!s->serving) g_off = *running_g;
    *running_g += q.G;
    p.g_off = g_off;
    p.g_len = q.G;
    if (q.G) {
      CK(cudaMemcpyAsync(s->grp_start + g_off, q.gs, q.G * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(s->grp_delay + g_off, q.gd, q.G * sizeof(uint16_t), cudaMemcpyDeviceToDevice, st));
    }
    CK(fill_meta((uint64_t)p.n, (uint64_t)p.offset, p.k_off, g_off, q.cnt_scan, q.grp_scan, s->grp_start,
                 s->grp_delay, s->src_meta, s->src_syn, s->src_grp, s->src_age, items, st));
  }
  unsigned long long ih = 0;
  CK(cudaMemcpyAsync(&ih, items, sizeof(ih), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cudaFree(items);
  free_parts(parts);
  if (items_out) *items_out = ih;
  return rc;
}

void release_instance_ranges(ngb_sim* s, int instance) {
  for (PopHost& p : s->pops) {
    if (p.instance != instance) continue;
    if (p.placed) s->nalloc.release((uint64_t)p.offset, (uint64_t)p.n);
    s->kalloc.release(p.k_off, p.k_len);
    s->galloc.release(p.g_off, p.g_len);
    p.placed = false;
    p.k_len = p.g_len = 0;
  }
}

// Serving handles: place, build and activate one pending instance at the
// current step.
int commit_impl(ngb_sim* s, int instance) {
  InstHost& I = s->inst[(size_t)instance];
  if (I.state != 0) return fail(NGB_ERR_STATE, "ngb_commit_instance: instance not pending");
  int rc = NGB_OK;
  for (size_t p = 0; p < s->pops.size() && rc == NGB_OK; ++p)
    if (s->pops[p].instance == instance) rc = place_population(s, (int)p);
  std::vector<PopParts> parts;
  int md = 0;
  uint64_t rk = 0, rg = 0, items = 0;
  std::vector<int> srcs;
  for (size_t p = 0; p < s->pops.size(); ++p)
    if (s->pops[p].instance == instance) srcs.push_back((int)p);
  if (rc == NGB_OK) rc = build_populations(s, srcs, parts, &md, &rk);
  if (rc == NGB_OK && md > s->L - 1) rc = fail(NGB_ERR_OVERFLOW, "a delay is beyond the reserved ring slots");
  if (rc == NGB_OK) rc = place_parts(s, parts, &rg, &items);
  if (rc != NGB_OK) {
    free_parts(parts);
    release_instance_ranges(s, instance);
    return rc;
  }
  s->max_delay = std::max(s->max_delay, md);
  I.t0 = s->t;
  I.state = 1;
  s->tables_dirty = true;
  return NGB_OK;
}

// Segment tables, Poisson tables, persistent-kernel arguments and the step
// graph for the active populations.
int rebuild_tables(ngb_sim* s) {
  cudaStream_t st = s->stream;
  CK(cudaStreamSynchronize(st));
  for (void* p : s->table_allocs) cudaFree(p);
  s->table_allocs.clear();
  auto talloc = [&](void** p, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) s->table_allocs.push_back(*p);
    return e;
  };
  const double dt = s->cfg.dt_ms;
  std::vector<LifSeg> lsegs;
  std::vector<AeifSeg> asegs_exp, asegs_alpha, asegs_beta;
  std::vector<uint32_t> thr_all;
  s->lif_blocks = 0;
  s->aeif_blocks = 0;
  s->aeifa_blocks = 0;
  s->aeifb_blocks = 0;
  s->n_active = 0;
  for (bool& h : s->hot_kind) h = false;
  {
    // two LIF neurons per thread (the tiled kernel: resident blocks walking
    // the tiles with the next tile's loads in flight) when the update grid
    // would fill the GPU more than twice over at one neuron per thread
    int64_t n_lif_total = 0;
    for (const PopHost& p : s->pops)
      if (p.placed && s->inst[(size_t)p.instance].state == 1 && p.model == NGB_LIF_PSC_EXP) n_lif_total += p.n;
    s->lif_npt = n_lif_total > 2 * (int64_t)std::max(1, s->sms) * 2048 ? 2 : 1;
    const char* env_npt = std::getenv("NGB_LIF_NPT");
    if (env_npt && (std::atoi(env_npt) == 1 || std::atoi(env_npt) == 2 || std::atoi(env_npt) == 4))
      s->lif_npt = std::atoi(env_npt);
  }
  const int64_t lif_tile = (int64_t)kLifBlock * s->lif_npt;
  for (const PopHost& p : s->pops) {
    if (!p.placed || s->inst[(size_t)p.instance].state != 1) continue;
    s->n_active += p.n;
    const InstHost& I = s->inst[(size_t)p.instance];
    if (p.model == NGB_LIF_PSC_EXP) {
      const ngb_lif_params& q = p.lif;
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
      g.t0 = I.t0;
      g.seed = I.seed;
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
      s->lif_blocks += (p.n + lif_tile - 1) / lif_tile;
    } else {
      const ngb_aeif_params& q = p.aeif;
      const int kind = p.model == NGB_AEIF_COND_BETA    ? kAeifBeta
                       : p.model == NGB_AEIF_COND_ALPHA ? kAeifAlpha
                                                        : kAeifExp;
      int64_t& kind_blocks = kind == kAeifBeta ? s->aeifb_blocks : kind == kAeifAlpha ? s->aeifa_blocks : s->aeif_blocks;
      AeifSeg g{};
      g.offset = p.offset;
      g.n = p.n;
      g.alpha = kind == kAeifAlpha ? 1 : 0;
      g.blk_begin = kind_blocks;
      g.t0 = I.t0;
      g.seed = I.seed;
      g.local_off = p.local_off;
      const std::vector<uint32_t> th = poisson_thresholds(q.poisson.n_inputs * q.poisson.rate_hz * dt * 1e-3);
      g.n_thr = (uint32_t)th.size();
      g.thr_off = (uint32_t)thr_all.size();
      thr_all.insert(thr_all.end(), th.begin(), th.end());
      g.prec_rcpt = q.poisson.receptor;
      g.ctl32 = q.rk_control_fp32 ? 1 : 0;
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
      g.inv_tol_f = (float)g.inv_tol;
      g.h_min = q.rk_h_min_ms;
      g.dt = dt;
      g.max_sub = q.rk_max_substeps;
      g.V_hot = s->hot_on && q.Delta_T_mV > 0 ? (float)(q.V_T_mV + s->hot_c * q.Delta_T_mV) : INFINITY;
      if (g.V_hot < INFINITY) s->hot_kind[kind] = true;
      constexpr double kEuler = 2.718281828459045;
      g.e_tau_ex = (float)(kEuler / q.tau_ex_ms);
      g.e_tau_in = (float)(kEuler / q.tau_in_ms);
      // receptor ports: the beta model's own, else the two receptors
      g.n_ports = kind == kAeifBeta ? q.n_ports : 2;
      for (int k = 0; k < kMaxPorts; ++k) {
        double E = 0.0, tr = 1.0, td = 1.0;
        bool used = k < g.n_ports;
        if (kind == kAeifBeta && used) {
          E = q.E_rev_mV[k];
          tr = q.tau_rise_ms[k];
          td = q.tau_decay_ms[k];
        } else if (kind != kAeifBeta && k < 2) {
          E = k == 0 ? q.E_ex_mV : q.E_in_mV;
          tr = td = k == 0 ? q.tau_ex_ms : q.tau_in_ms;
        }
        g.E_p[k] = (float)E;
        g.itd_p[k] = (float)(1.0 / td);
        g.itr_p[k] = (float)(1.0 / tr);
        g.jmp_p[k] = used ? (float)beta_jump(tr, td) : 0.0f;
      }
      (kind == kAeifBeta ? asegs_beta : kind == kAeifAlpha ? asegs_alpha : asegs_exp).push_back(g);
      kind_blocks += (p.n + kAeifBlock - 1) / kAeifBlock;
    }
  }
  s->n_lif = (int)lsegs.size();
  {
    int64_t next = 0;
    bool contig = true;
    for (const LifSeg& g : lsegs) {
      contig = contig && g.offset == next;
      next += g.n;
    }
    s->lif_contig = contig && next == s->N;
  }
  s->n_aeif_exp = (int)asegs_exp.size();
  s->n_aeif_alpha = (int)asegs_alpha.size();
  s->n_aeif_beta = (int)asegs_beta.size();
  s->n_aeif = s->n_aeif_exp + s->n_aeif_alpha + s->n_aeif_beta;
  // the beta model's deferred-neuron list (6 words per neuron), on first use
  if (s->n_aeif_beta && !s->sb.dfr[kAeifBeta]) CK(s->dalloc(&s->sb.dfr[kAeifBeta], 6 * (size_t)s->N_cap));
  // hot lists (both step parities) of the conductance models that list neurons, on first use
  for (int kind = 0; kind < 3; ++kind)
    if (s->hot_kind[kind] && s->sb.htag && !s->sb.hot[kind]) CK(s->dalloc(&s->sb.hot[kind], 3 * (size_t)s->N_cap));
  CK(hot_reset(s));
  // every AdEx segment of the two-receptor models, for the persistent kernel
  std::vector<AeifSeg> asegs(asegs_exp);
  asegs.insert(asegs.end(), asegs_alpha.begin(), asegs_alpha.end());
  s->lif_tab = SegTable<LifSeg>{};
  s->aeif_tab = SegTable<AeifSeg>{};
  s->aeifa_tab = SegTable<AeifSeg>{};
  s->aeifb_tab = SegTable<AeifSeg>{};
  if (s->n_lif) {
    LifSeg* d = nullptr;
    CK(talloc((void**)&d, lsegs.size() * sizeof(LifSeg)));
    CK(cudaMemcpyAsync(d, lsegs.data(), lsegs.size() * sizeof(LifSeg), cudaMemcpyHostToDevice, st));
    s->lif_tab.dev = d;
    s->lif_tab.n = s->n_lif;
    for (int i = 0; i < std::min(s->n_lif, kInlineSegs); ++i) s->lif_tab.s[i] = lsegs[(size_t)i];
    std::vector<uint32_t> bs((size_t)s->lif_blocks);
    for (size_t i = 0; i < lsegs.size(); ++i) {
      const int64_t nb = (lsegs[i].n + lif_tile - 1) / lif_tile;
      for (int64_t b = 0; b < nb; ++b) bs[(size_t)(lsegs[i].blk_begin + b)] = (uint32_t)i;
    }
    uint32_t* db = nullptr;
    CK(talloc((void**)&db, bs.size() * sizeof(uint32_t)));
    CK(cudaMemcpyAsync(db, bs.data(), bs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    s->lif_tab.blk_seg = db;
  }
  // per-step tables of the AdEx kernels, one per conductance model
  auto aeif_table = [&](const std::vector<AeifSeg>& v, int64_t blocks, SegTable<AeifSeg>& tab) -> cudaError_t {
    if (v.empty()) return cudaSuccess;
    AeifSeg* d = nullptr;
    cudaError_t e = talloc((void**)&d, v.size() * sizeof(AeifSeg));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(AeifSeg), cudaMemcpyHostToDevice, st);
    tab.dev = d;
    tab.n = (int)v.size();
    for (int i = 0; i < std::min(tab.n, kInlineSegs); ++i) tab.s[i] = v[(size_t)i];
    std::vector<uint32_t> bs((size_t)blocks);
    for (size_t i = 0; i < v.size(); ++i) {
      const int64_t nb = (v[i].n + kAeifBlock - 1) / kAeifBlock;
      for (int64_t b = 0; b < nb; ++b) bs[(size_t)(v[i].blk_begin + b)] = (uint32_t)i;
    }
    uint32_t* db = nullptr;
    if (e == cudaSuccess) e = talloc((void**)&db, bs.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, bs.data(), bs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    tab.blk_seg = db;
    return e;
  };
  CK(aeif_table(asegs_exp, s->aeif_blocks, s->aeif_tab));
  CK(aeif_table(asegs_alpha, s->aeifa_blocks, s->aeifa_tab));
  CK(aeif_table(asegs_beta, s->aeifb_blocks, s->aeifb_tab));
  AeifSeg* d_asegs = nullptr;
  if (!asegs.empty()) {
    CK(talloc((void**)&d_asegs, asegs.size() * sizeof(AeifSeg)));
    CK(cudaMemcpyAsync(d_asegs, asegs.data(), asegs.size() * sizeof(AeifSeg), cudaMemcpyHostToDevice, st));
  }
  CK(talloc((void**)&s->thr, (thr_all.size() + 1) * sizeof(uint32_t)));
  if (!thr_all.empty())
    CK(cudaMemcpyAsync(s->thr, thr_all.data(), thr_all.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));

  // persistent kernel arguments
  {
    std::vector<int64_t> lv(1, 0), av(1, 0);
    for (const LifSeg& g : lsegs) lv.push_back(lv.back() + g.n);
    for (const AeifSeg& g : asegs) av.push_back(av.back() + g.n);
    int64_t *dlv = nullptr, *dav = nullptr;
    CK(talloc((void**)&dlv, lv.size() * 8));
    CK(talloc((void**)&dav, av.size() * 8));
    CK(cudaMemcpyAsync(dlv, lv.data(), lv.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dav, av.data(), av.size() * 8, cudaMemcpyHostToDevice, st));
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    PersistArgs& a = s->pa;
    a.lseg = s->lif_tab.dev;
    a.aseg = d_asegs;
    a.lvoff = dlv;
    a.avoff = dav;
    a.thr = s->thr;
    a.st0 = s->st0; a.st1 = s->st1; a.st2 = s->st2; a.st3 = s->st3; a.st4 = s->st4;
    a.st5 = s->st5; a.st6 = s->st6;
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
    a.age = s->scheme == 2 ? 1 : 0;
    a.off_aseg = (uint32_t)a16(lsegs.size() * sizeof(LifSeg));
    a.off_lvoff = a.off_aseg + (uint32_t)a16(asegs.size() * sizeof(AeifSeg));
    a.off_avoff = a.off_lvoff + (uint32_t)a16(lv.size() * 8);
    a.off_thr = a.off_avoff + (uint32_t)a16(av.size() * 8);
    s->persist_smem = a.off_thr + a16(thr_all.size() * 4);
    const bool was_ok = s->persist_ok;
    s->persist_ok = false;
    // the persistent kernel integrates the two-receptor models only; its grid
    // fits both variants (per-step barriers, pipelined)
    if (s->persist_smem <= 200 * 1024 && s->n_aeif_beta == 0) {
      int bpsm = 0, bpsm_pipe = 0;
      if (persistent_max_blocks_per_sm(s->cfg.deterministic != 0, s->cfg.weight_dtype, s->n_lif > 0,
                                       s->n_aeif > 0, false, s->persist_smem, &bpsm) == cudaSuccess &&
          persistent_max_blocks_per_sm(s->cfg.deterministic != 0, s->cfg.weight_dtype, s->n_lif > 0,
                                       s->n_aeif > 0, true, s->persist_smem, &bpsm_pipe) == cudaSuccess &&
          std::min(bpsm, bpsm_pipe) > 0) {
        bpsm = std::min(bpsm, bpsm_pipe);
        s->persist_ok = true;
        s->persist_max_bpsm = bpsm;
        if (!was_ok || s->persist_grid <= 0 || s->persist_grid > s->sms * bpsm)
          s->persist_grid = s->sms * std::min(bpsm, 2);
      }
      cudaGetLastError();
    }
    if (!s->persist_ok && (s->mode == 1 || s->mode == 4)) s->mode = 0;
  }
  // the pipelined persistent kernel delivers with the ring scheme
  if (s->mode == 4 && (s->scheme != 1 || !s->sb.wi3[0])) s->mode = 0;
  // plastic synapses run in the per-step kernel loop (spike-buffer scheme)
  if (s->d_rules) {
    s->persist_ok = false;
    s->mode = 0;
  }
  // the fused loop runs one LIF neuron per thread, the two-receptor AdEx
  // models, and delivers with the ring scheme
  if (s->mode == 2 && (!fused_ok(s) || s->scheme != 1)) s->mode = 0;
  // the pipelined loop delivers with the ring scheme
  if (s->mode == 3 && (s->scheme != 1 || !s->stream2)) s->mode = 0;
  // target-tiled delivery: static networks, spike-buffer scheme, layout built
  if (s->mode == 7 && (!tiled_shape_ok(s) || !s->tl.pairs)) s->mode = 0;
  if (s->mode == 5 && !pipe1_ok(s)) s->mode = 0;
  if (s->mode == 6 && !owned_ready(s)) s->mode = 0;
  s->tables_dirty = false;
  return capture_graph(s);
}

// STDP state of a finalised network (Sec. 2.1): the rules' device table with
// their pair factors e^(-n dt / tau) tabulated for lags up to 20 tau (FP64,
// rounded once), the latest arrival step of every synapse and the latest
// spike step of every neuron (-1: none), the per-step lists of firing
// targets and the reverse index of the plastic synapses.
int setup_stdp(ngb_sim* s) {
  cudaStream_t st = s->stream;
  const int64_t N = s->N_cap;
  const double dt = s->cfg.dt_ms;
  std::vector<StdpRule> rules;
  for (const ngb_stdp_params& q : s->stdp_params) {
    StdpRule r{};
    r.A_plus = (float)(q.lambda * q.W_max);
    r.A_minus = (float)(q.alpha * q.lambda * q.W_max);
    r.inv_W_max = (float)(1.0 / q.W_max);
    r.W_max = (float)q.W_max;
    r.mu_plus = (float)q.mu_plus;
    r.mu_minus = (float)q.mu_minus;
    const double np = std::floor(20.0 * q.tau_plus_ms / dt) + 1.0;
    const double nm = std::floor(20.0 * q.tau_minus_ms / dt) + 1.0;
    if (np > (double)(1 << 24) || nm > (double)(1 << 24))
      return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: STDP time constant longer than 2^24 / 20 steps");
    std::vector<float> k((size_t)(np + nm));
    for (int64_t n = 0; n < (int64_t)np; ++n) k[(size_t)n] = (float)std::exp(-(double)n * dt / q.tau_plus_ms);
    for (int64_t n = 0; n < (int64_t)nm; ++n)
      k[(size_t)np + (size_t)n] = (float)std::exp(-(double)n * dt / q.tau_minus_ms);
    float* d = nullptr;
    CK(s->dalloc(&d, k.size()));
    CK(cudaMemcpy(d, k.data(), k.size() * sizeof(float), cudaMemcpyHostToDevice));
    r.n_plus = (int32_t)np;
    r.n_minus = (int32_t)nm;
    r.k_plus = d;
    r.k_minus = d + (size_t)np;
    rules.push_back(r);
  }
  CK(s->dalloc(&s->d_rules, rules.size()));
  CK(cudaMemcpy(s->d_rules, rules.data(), rules.size() * sizeof(StdpRule), cudaMemcpyHostToDevice));
  // (+4: the delivery reads the words of 4 consecutive synapses at a time)
  CK(s->dalloc(&s->wa, s->K_cap + 4));
  CK(cudaMemsetAsync(s->wa, 0, (s->K_cap + 4) * sizeof(uint2), st));
  CK(init_stdp_words((const float*)s->w, s->K_cap, s->wa, st));
  CK(s->dalloc(&s->sb.last_spike, N));
  CK(cudaMemsetAsync(s->sb.last_spike, 0xFF, N * sizeof(int32_t), st));
  CK(s->dalloc(&s->sb.post[0], N));
  CK(s->dalloc(&s->sb.post[1], N));
  CK(s->dalloc(&s->in_ptr, N + 1));
  uint64_t* in_syn = nullptr;
  CK(build_stdp_index(s->tgt, s->K_cap, N, s->in_ptr, &in_syn, &s->n_plastic, st));
  s->allocs.push_back(in_syn);
  s->dev_bytes += std::max<uint64_t>(1, s->n_plastic) * sizeof(uint64_t);
  s->in_syn = in_syn;
  s->sb.in_ptr = s->in_ptr;
  return NGB_OK;
}

int finalize_impl(ngb_sim* s) {
  if (s->finalized) return NGB_OK;
  cudaStream_t st = s->stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev));
  if (!s->serving) {
    if (s->N <= 0) return fail(NGB_ERR_STATE, "ngb_finalize: no neurons");
    s->R = 1;
    for (const PopHost& p : s->pops) s->R = std::max(s->R, receptors_of(p));
    s->N_cap = s->N;
    uint64_t K = 0;
    for (const CallHost& c : s->calls) {
      const PopHost& pt = s->pops[(size_t)c.tgt_pop];
      K += call_synapses(c.conn, s->pops[(size_t)c.src_pop].n, pt.n, c.src_pop == c.tgt_pop);
    }
    s->K_cap = K;
  }
  if (s->N_cap >= (int64_t)kIdMask) return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^26 neurons");
  const int64_t N = s->N_cap;
  const size_t wsize = s->cfg.weight_dtype == NGB_WEIGHT_FP32 ? 4 : 2;

  // neuron-indexed arrays
  CK(s->dalloc(&s->st0, N));
  CK(s->dalloc(&s->st1, N));
  CK(s->dalloc(&s->ref, N));
  CK(cudaMemsetAsync(s->st0, 0, N * sizeof(float), st));
  CK(cudaMemsetAsync(s->st1, 0, N * sizeof(float), st));
  CK(cudaMemsetAsync(s->ref, 0, N * sizeof(int32_t), st));
  if (s->R >= 2) {
    CK(s->dalloc(&s->st2, N));
    CK(s->dalloc(&s->st3, N));
    CK(s->dalloc(&s->st4, N));
    CK(s->dalloc(&s->st5, N));
    CK(s->dalloc(&s->st6, N));
    // AdEx neurons deferred to the finishing kernel: one 64-byte record per neuron and conductance model
    CK(s->dalloc(&s->sb.dfr[0], 4 * (size_t)N));
    CK(s->dalloc(&s->sb.dfr[1], 4 * (size_t)N));
    s->sb.dfr_cap = N;
    const char* env_budget = std::getenv("NGB_AEIF_BUDGET");
    if (env_budget) s->aeif_budget = std::max(0, std::atoi(env_budget));
    const char* env_hot = std::getenv("NGB_AEIF_HOT");
    if (env_hot) {
      const double c = std::atof(env_hot);
      if (c > 0.0) s->hot_c = (float)c;
      else s->hot_on = false;
    }
    if (s->aeif_budget <= 0) s->hot_on = false;  // the finishing kernel empties the lists
    CK(s->dalloc(&s->sb.dfetch, 3));
    CK(cudaMemsetAsync(s->sb.dfetch, 0, 3 * sizeof(unsigned long long), st));
    if (s->hot_on) {
      CK(s->dalloc(&s->sb.htag, N));
      CK(s->dalloc(&s->sb.hcnt, 9));
      s->sb.hot_cap = N;
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      CK(cudaStreamCreateWithPriority(&s->hstream, cudaStreamNonBlocking, hi));
      CK(cudaEventCreateWithFlags(&s->hev[0], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&s->hev[1], cudaEventDisableTiming));
    }
    CK(cudaMemsetAsync(s->st5, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(s->st6, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(s->st2, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(s->st3, 0, N * sizeof(float), st));
    CK(cudaMemsetAsync(s->st4, 0, N * sizeof(float), st));
  }
  if (s->R > 2) {  // beta ports 2-3
    CK(s->dalloc(&s->ext, 4 * (size_t)N));
    CK(cudaMemsetAsync(s->ext, 0, 4 * (size_t)N * sizeof(float), st));
  }
  CK(s->dalloc(&s->src_syn, N + 1));
  CK(s->dalloc(&s->src_grp, N + 1));
  CK(s->dalloc(&s->src_meta, N));
  CK(s->dalloc(&s->src_age, N));
  CK(cudaMemsetAsync(s->src_age, 0, N * sizeof(uint2), st));
  CK(cudaMemsetAsync(s->src_syn, 0, (N + 1) * sizeof(uint64_t), st));
  CK(cudaMemsetAsync(s->src_grp, 0, (N + 1) * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(s->src_meta, 0, N * sizeof(uint4), st));
  // synapse pool (padded for the 16-byte vector loads)
  const uint64_t Kpad = ((s->K_cap + 3) & ~3ull) + kChunk;
  CK(s->dalloc(&s->tgt, Kpad));
  CK(s->dalloc((uint8_t**)&s->w, Kpad * wsize));
  CK(cudaMemsetAsync(s->tgt, 0, Kpad * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(s->w, 0, Kpad * wsize, st));
  s->nalloc.init((uint64_t)N);
  s->kalloc.init(s->K_cap);

  // counters, clock, spike record, barrier
  unsigned long long* ctrs = nullptr;
  CK(s->dalloc(&ctrs, kCounters));  // ctr[2], events, substeps, rec_count, hot_steps, pcnt[2], dcnt[6], ctr3[3]
  CK(cudaMemsetAsync(ctrs, 0, kCounters * sizeof(unsigned long long), st));
  s->sb.ctr = ctrs;
  s->sb.events = ctrs + 2;
  s->sb.substeps = ctrs + 3;
  s->sb.hot_steps = ctrs + 5;
  s->sb.rec_count = ctrs + 4;
  s->sb.pcnt = ctrs + 6;
  s->sb.dcnt = ctrs + 8;
  s->sb.ctr3 = ctrs + 14;
  s->sb.post_cnt = ctrs + 18;
  CK(s->dalloc(&s->sb.err, 1));
  CK(cudaMemsetAsync(s->sb.err, 0, sizeof(uint32_t), st));
  CK(s->dalloc(&s->clk, 2));
  CK(cudaMemsetAsync(s->clk, 0, 2 * sizeof(int64_t), st));
  CK(s->dalloc(&s->bar, 4));
  s->drain_steps = s->cfg.drain_steps > 0 ? s->cfg.drain_steps : 1000;
  int64_t cap = 0;
  if (s->cfg.record_spikes) {
    cap = s->cfg.record_capacity > 0 ? s->cfg.record_capacity
                                     : std::max<int64_t>(1 << 20, N * (int64_t)s->drain_steps / 100);
    CK(s->dalloc(&s->sb.rec_id, cap));
    CK(s->dalloc(&s->sb.rec_step, cap));
    CK(s->dalloc(&s->rec_keys, cap));
    CK(s->dalloc(&s->rec_sorted, cap));
    CK(record_sort_scratch_bytes((uint64_t)cap, &s->rec_sort_bytes));
    CK(s->dalloc(&s->rec_sort_tmp, s->rec_sort_bytes));
    CK(cudaMallocHost((void**)&s->rec_pinned, (size_t)cap * sizeof(unsigned long long)));
  }
  s->sb.rec_cap = cap;
  {
    const char* env = std::getenv("NGB_PDL");
    s->pdl = !(env && env[0] == '0');
  }
  s->deliver_grid = std::max(1, s->sms) * 2;

  uint64_t items = 0;
  if (!s->serving) {
    // every population in creation order; groups sized after the build
    for (size_t p = 0; p < s->pops.size(); ++p) {
      const int rc = place_population(s, (int)p);
      if (rc != NGB_OK) return rc;
    }
    // sources in global id order, so the CSR is ordered by source across instances
    std::vector<PopParts> parts;
    uint64_t rk = 0;
    int md_all = 0;
    std::vector<int> srcs;
    for (size_t p = 0; p < s->pops.size(); ++p) srcs.push_back((int)p);
    {
      const int rc = build_populations(s, srcs, parts, &md_all, &rk);
      if (rc != NGB_OK) {
        free_parts(parts);
        return rc;
      }
    }
    uint64_t G = 0;
    for (const PopParts& q : parts) G += q.G;
    if (G >= (1ull << 32)) {
      free_parts(parts);
      return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^32 connection groups");
    }
    s->G_cap = G;
    CK(s->dalloc(&s->grp_start, G + 1));
    CK(s->dalloc(&s->grp_delay, G + 1));
    s->galloc.init(G);
    uint64_t rg = 0;
    int rc = place_parts(s, parts, &rg, &items);
    if (rc != NGB_OK) return rc;
    const uint64_t Kend = s->K_cap;
    CK(cudaMemcpyAsync(s->grp_start + G, &Kend, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->src_syn + N, &Kend, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    const uint32_t Gend = (uint32_t)G;
    CK(cudaMemcpyAsync(s->src_grp + N, &Gend, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    s->max_delay = md_all;
    s->L = (int64_t)std::max<uint64_t>(2, next_pow2((uint64_t)s->max_delay + 1));
    for (InstHost& I : s->inst) I.state = 1;
  } else {
    CK(s->dalloc(&s->grp_start, s->G_cap + 1));
    CK(s->dalloc(&s->grp_delay, s->G_cap + 1));
    CK(cudaMemsetAsync(s->grp_start, 0, (s->G_cap + 1) * sizeof(uint64_t), st));
    s->galloc.init(s->G_cap);
    items = s->K_cap / kChunk + 2 * (uint64_t)N + 2;
  }
  s->K = s->K_cap;
  s->G = s->G_cap;
  if (items >= (1ull << 32)) return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: more than 2^32 delivery work items");
  s->work_items = items;
  // delivery scheme (ngb_sim_config.delivery; automatic: spike buffer when the ring would not stay in L2)
  {
    int l2 = 0;
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const double ring_full = (double)s->L * s->R * (double)N * (s->cfg.deterministic ? 8 : 4);
    if (s->cfg.delivery == 1) s->scheme = 1;
    else if (s->cfg.delivery == 2) s->scheme = 2;
    else s->scheme = ring_full > 0.5 * (double)l2 ? 2 : 1;
    if (!s->stdp_params.empty()) {  // plastic synapses deliver at arrival: spike buffer
      if (s->cfg.delivery == 1)
        return fail(NGB_ERR_INVALID_ARG, "ngb_finalize: STDP synapses need the spike-buffer delivery scheme");
      s->scheme = 2;
    }
  }
  // pending-spike lists (spike-buffer scheme): a source has at most one spike
  // per refractory period + 1 steps in flight, and none older than the
  // largest delay
  uint64_t wi_entries = 2 * s->work_items + 2;
  if (s->cfg.delivery != 1) {
    uint64_t cap = 1024;
    if (s->serving) {
      cap += (uint64_t)N * (uint64_t)std::min<int64_t>(s->L, 8);
    } else {
      const int64_t D = std::max(1, s->max_delay);
      for (const PopHost& p : s->pops) {
        int64_t ref = 0;
        if (p.model == NGB_LIF_PSC_EXP) ref = std::max<int64_t>(0, (int64_t)std::nearbyint(p.lif.t_ref_ms / s->cfg.dt_ms));
        const int64_t per = std::min<int64_t>(D, (D + ref) / (ref + 1) + 1);
        cap += (uint64_t)p.n * (uint64_t)per;
      }
    }
    const char* env_cap = std::getenv("NGB_TEST_PENDING_CAP");
    if (env_cap) cap = std::strtoull(env_cap, nullptr, 10);
    s->sb.pend_cap = (int64_t)cap;
    CK(s->dalloc(&s->sb.pend[0], cap + 1));
    CK(s->dalloc(&s->sb.pend[1], cap + 1));
    // due items per step: at most one per pending or new spike plus one per 1024 synapses
    wi_entries = std::max<uint64_t>(wi_entries, cap + (uint64_t)N + s->K_cap / kAgeSpan + 2);
  }
  s->sb.wi_cap = (int64_t)wi_entries;
  CK(s->dalloc(&s->sb.wi[0], wi_entries));
  CK(s->dalloc(&s->sb.wi[1], wi_entries));
  if (s->cfg.delivery != 2) {
    // pipelined ring scheme: work-item lists by step mod 3, and its second stream
    for (int q = 0; q < 3; ++q) CK(s->dalloc(&s->sb.wi3[q], 2 * s->work_items + 2));
    CK(cudaStreamCreateWithFlags(&s->stream2, cudaStreamNonBlocking));
  }
  // ring buffer
  const size_t ring_bytes = (size_t)s->L * s->R * N * (s->cfg.deterministic ? 8 : 4);
  CK(s->dalloc((uint8_t**)&s->ring, ring_bytes));
  CK(cudaMemsetAsync(s->ring, 0, ring_bytes, st));
  if (!s->stdp_params.empty()) {
    int rc = setup_stdp(s);
    if (rc != NGB_OK) return rc;
  }
  CK(cudaStreamSynchronize(st));
  s->finalized = true;
  if (s->serving) {
    for (size_t i = 0; i < s->inst.size(); ++i) {
      if (s->inst[i].state != 0) continue;
      bool has_pop = false;
      for (const PopHost& p : s->pops) has_pop = has_pop || p.instance == (int)i;
      if (!has_pop) continue;
      const int rc = commit_impl(s, (int)i);
      if (rc != NGB_OK) return rc;
    }
  }
  const char* env_mode = std::getenv("NGB_MODE");
  s->mode = 0;
  if (env_mode && std::string(env_mode) == "persistent") s->mode = 1;
  if (env_mode && std::string(env_mode) == "persistent_pipelined" && s->scheme == 1) s->mode = 4;
  if (env_mode && std::string(env_mode) == "fused" && s->scheme == 1) s->mode = 2;
  if (env_mode && std::string(env_mode) == "pipelined" && s->scheme == 1 && s->stream2) s->mode = 3;
  if (env_mode && std::string(env_mode) == "pipelined_one_kernel" && s->scheme == 1) s->mode = 5;
  if (env_mode && std::string(env_mode) == "target_owned" && s->scheme == 1) s->mode = 6;
  if (env_mode && std::string(env_mode) == "tiled" && s->scheme == 2) {
    // tile size (neurons) and blocks per tile from NGB_TILED ("T,P"); else two tiles per SM, one block each
    uint32_t T = tiled_T_for(s, 2 * (int64_t)s->sms), P = 1;
    if (const char* tv = std::getenv("NGB_TILED")) {
      unsigned a = 0, b = 0;
      if (std::sscanf(tv, "%u,%u", &a, &b) == 2 && a >= 32 && a <= tiled_max_T(s) && b >= 1 && b <= 8) {
        T = a;
        P = b;
      }
    }
    if (tiled_ready(s, T)) {
      s->mode = 7;
      s->tl_P = P;
    }
  }
  s->graph_steps = s->cfg.steps_per_graph == 0 ? 100 : std::max(0, s->cfg.steps_per_graph);
  return rebuild_tables(s);
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
  if (!s->stdp_params.empty() && s->t + steps > (int64_t)INT32_MAX)
    return fail(NGB_ERR_OVERFLOW, "ngb_simulate: STDP synapses count steps in 31 bits");
  if (!s->finalized) {
    const int rc = finalize_impl(s);
    if (rc != NGB_OK) {
      s->failed = true;
      return rc;
    }
  }
  if (s->tables_dirty) {
    const int rc = rebuild_tables(s);
    if (rc != NGB_OK) return rc;
  }
  // loops whose AdEx update is not the per-step kernels' leave the hot lists stale
  if (s->n_aeif && (profiled ? s->mode == 2 : (s->mode == 1 || s->mode == 2 || s->mode == 4 || s->mode == 6)))
    CK(hot_reset(s));
  int rc_overflow = NGB_OK;
  if (!profiled) {
    int64_t left = steps;
    while (left > 0) {
      const int64_t chunk = std::min<int64_t>(left, s->drain_steps);
      int64_t done = 0;
      if (s->mode == 1 || s->mode == 4) {
        CK(launch_persistent_chunk(s, chunk));
        done = chunk;
      }
      if (s->mode == 6) {
        CK(launch_owned_chunk(s, chunk));
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
    const bool fused = s->mode == 2;
    for (int64_t i = 0; i < chunk; ++i) {
      cudaEvent_t* e = &ev[4 * i];
      CK(cudaEventRecord(e[0], s->stream));
      if (s->n_lif) CK(fused ? launch_fused_lif(s, 0) : launch_lif(s, 0));
      CK(cudaEventRecord(e[1], s->stream));
      if (s->n_aeif) CK(fused ? launch_fused_aeif(s, 0) : launch_aeif(s, 0));
      CK(cudaEventRecord(e[2], s->stream));
      if (!fused) CK(launch_post(s));
      CK(fused ? launch_tick_add(s->clk, 1, s->sb.ctr, s->sb.ctr3, s->pdl, s->stream) : launch_del(s, 0));
      CK(cudaEventRecord(e[3], s->stream));
      if (s->mode == 3 || s->mode == 5) CK(launch_tick_add(s->clk, 1, s->sb.ctr, s->sb.ctr3, false, s->stream));
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
  const int64_t N = s->N_cap;
  const size_t ring_bytes = (size_t)s->L * s->R * N * (s->cfg.deterministic ? 8 : 4);
  sn.parts = {{s->st0, N * 4}, {s->st1, N * 4}, {s->ref, N * 4}, {s->ring, ring_bytes},
              {s->sb.ctr, kCounters * sizeof(unsigned long long)}, {s->clk, 2 * sizeof(int64_t)},
              {s->sb.err, sizeof(uint32_t)}};
  if (s->sb.pend[0]) {
    sn.parts.push_back({s->sb.pend[0], (size_t)s->sb.pend_cap * sizeof(uint4)});
    sn.parts.push_back({s->sb.pend[1], (size_t)s->sb.pend_cap * sizeof(uint4)});
  }
  if (s->st2) {
    sn.parts.push_back({s->st2, N * 4});
    sn.parts.push_back({s->st3, N * 4});
    sn.parts.push_back({s->st4, N * 4});
    sn.parts.push_back({s->st5, N * 4});
    sn.parts.push_back({s->st6, N * 4});
  }
  if (s->ext) sn.parts.push_back({s->ext, 4 * N * 4});
  if (s->d_rules) {  // plastic weights, arrivals and latest spikes change while trial steps run
    sn.parts.push_back({s->wa, s->K_cap * 8});
    sn.parts.push_back({s->sb.last_spike, N * 4});
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
  // snapshots are taken between steps, when no due group waits in a bucket
  if (s->tl.bcnt) CK(cudaMemsetAsync(s->tl.bcnt, 0, (size_t)2 * s->tl.n_tiles * sizeof(unsigned int), s->stream));
  CK(hot_reset(s));
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
  std::snprintf(buf, sizeof(buf), "%s|sm%d|N%lld|K%llu|G%llu|L%lld|R%d|w%d|det%d|lif%d|aeif%d.%d.%d|dl%d",
                prop.name, prop.multiProcessorCount, (long long)s->N, (unsigned long long)s->K,
                (unsigned long long)s->G, (long long)s->L, s->R, s->cfg.weight_dtype, s->cfg.deterministic, s->n_lif,
                s->n_aeif_exp, s->n_aeif_alpha, s->n_aeif_beta, s->cfg.delivery);
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
  if (cfg->delivery < 0 || cfg->delivery > 2) return fail(NGB_ERR_INVALID_ARG, "ngb_create: delivery");
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
  if (s->stream2) cudaStreamDestroy(s->stream2);
  if (s->hstream) cudaStreamSynchronize(s->hstream);
  if (s->hstream) cudaStreamDestroy(s->hstream);
  for (cudaEvent_t ev : s->hev)
    if (ev) cudaEventDestroy(ev);
  for (void* p : s->allocs) cudaFree(p);
  for (void* p : s->table_allocs) cudaFree(p);
  tiled_free(&s->tl);
  if (s->rec_pinned) cudaFreeHost(s->rec_pinned);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return NGB_OK;
}

int ngb_add_instance(ngb_sim* s, uint64_t seed, int32_t* instance_out) {
  if (!s) return fail(NGB_ERR_INVALID_ARG, "NULL handle");
  if (s->finalized && !s->serving) return fail(NGB_ERR_STATE, "ngb_add_instance: network already finalised");
  s->inst.push_back(InstHost{seed, 0, 0, 0});
  if (instance_out) *instance_out = (int32_t)s->inst.size() - 1;
  return NGB_OK;
}

int ngb_add_population_in(ngb_sim* s, int32_t instance, int32_t model, int64_t n, const void* params,
                          int32_t* pop_id_out) {
  if (!s || !params) return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: NULL argument");
  if (instance < 0 || instance >= (int32_t)s->inst.size())
    return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: unknown instance");
  if ((s->finalized && !s->serving) || s->inst[(size_t)instance].state != 0)
    return fail(NGB_ERR_STATE, "ngb_add_population: network (instance) already built");
  // neuron ids (26 bits) are positions: the network's for a static handle, the pool's for a serving
  // handle (whose populations come and go, so only the pool bounds one)
  if (n <= 0 || (s->serving ? n > s->N_cap : s->N + n >= (int64_t)kIdMask))
    return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: n");
  PopHost p{};
  p.model = model;
  p.instance = instance;
  p.n = n;
  p.offset = s->serving ? -1 : s->N;  // serving handles place populations when the instance is committed
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
  } else if (model == NGB_AEIF_COND_EXP || model == NGB_AEIF_COND_ALPHA || model == NGB_AEIF_COND_BETA) {
    p.aeif = *(const ngb_aeif_params*)params;
    const ngb_aeif_params& q = p.aeif;
    const bool beta = model == NGB_AEIF_COND_BETA;
    if (beta) {
      if (q.n_ports < 1 || q.n_ports > kMaxPorts)
        return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: beta model needs 1-4 ports");
      for (int k = 0; k < q.n_ports; ++k)
        if (!(q.tau_rise_ms[k] > 0 && q.tau_decay_ms[k] > 0))
          return fail(NGB_ERR_INVALID_ARG, "ngb_add_population: beta port time constants");
    }
    const int ports = beta ? q.n_ports : 2;
    if (!(q.C_m_pF > 0 && q.tau_w_ms > 0 && (beta || (q.tau_ex_ms > 0 && q.tau_in_ms > 0)) && q.rk_tol > 0 &&
          q.rk_h_min_ms > 0 && q.rk_h_init_ms > 0 && q.rk_max_substeps > 0 && q.Delta_T_mV >= 0 &&
          q.V_init_sd_mV >= 0 && q.poisson.receptor >= 0 && q.poisson.receptor < ports))
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
  const int32_t np = (int32_t)s->pops.size();
  if (src_pop < 0 || src_pop >= np || tgt_pop < 0 || tgt_pop >= np)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: population id");
  const PopHost& ps = s->pops[src_pop];
  const PopHost& pt = s->pops[tgt_pop];
  if ((s->finalized && !s->serving) || s->inst[(size_t)ps.instance].state != 0)
    return fail(NGB_ERR_STATE, "ngb_connect: network (instance) already built");
  if (ps.instance != pt.instance) return fail(NGB_ERR_INVALID_ARG, "ngb_connect: populations of different instances");
  if (conn->rule < NGB_RULE_FIXED_INDEGREE || conn->rule > NGB_RULE_ALL_TO_ALL)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: rule");
  if (conn->rule == NGB_RULE_ONE_TO_ONE && (ps.n != pt.n || (src_pop == tgt_pop && !conn->allow_autapses)))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: one-to-one needs equal sizes (and autapses within a population)");
  if (conn->K < 0) return fail(NGB_ERR_INVALID_ARG, "ngb_connect: K < 0");
  if (!valid_dist(syn->weight) || !valid_dist(syn->delay_ms))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: distribution");
  if (syn->receptor < 0 || syn->receptor >= ports_of(pt))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect: receptor beyond the target model's ports");
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

int ngb_connect_stdp(ngb_sim* s, int32_t src_pop, int32_t tgt_pop, const ngb_conn_spec* conn, const ngb_syn_spec* syn,
                     const ngb_stdp_params* p) {
  if (!s || !p) return fail(NGB_ERR_INVALID_ARG, "ngb_connect_stdp: NULL argument");
  if (s->serving) return fail(NGB_ERR_STATE, "ngb_connect_stdp: STDP synapses are not served");
  if (s->cfg.weight_dtype != NGB_WEIGHT_FP32)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect_stdp: plastic weights need FP32 storage");
  if (s->cfg.delivery == NGB_DELIVERY_RING)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect_stdp: STDP synapses need the spike-buffer delivery scheme");
  if (!(p->tau_plus_ms > 0 && p->tau_minus_ms > 0 && p->lambda >= 0 && p->alpha >= 0 && p->mu_plus >= 0 &&
        p->mu_minus >= 0 && p->W_max > 0))
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect_stdp: STDP parameters");
  if ((int)s->stdp_params.size() >= kMaxStdpRules)
    return fail(NGB_ERR_INVALID_ARG, "ngb_connect_stdp: at most 15 STDP rules per handle");
  const size_t before = s->calls.size();
  const int rc = ngb_connect(s, src_pop, tgt_pop, conn, syn);
  if (rc != NGB_OK) return rc;
  if (s->calls.size() != before + 1) return fail(NGB_ERR_STATE, "ngb_connect_stdp: internal");
  s->stdp_params.push_back(*p);
  s->calls.back().stdp = (int)s->stdp_params.size();
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
  if (s->tables_dirty) {
    rc = rebuild_tables(s);
    if (rc != NGB_OK) return rc;
  }
  if (trial_steps == 0) trial_steps = 500;
  int dev = 0, sms = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // Both delivery schemes are candidates only while no spike is in flight
  // (step 0) and the configuration leaves the choice open.
  const bool both = s->cfg.delivery == 0 && s->t == 0 && !s->serving && s->sb.pend[0] != nullptr && !s->d_rules;
  const std::string key = tune_key(s);
  const char* cache = std::getenv("NGB_AUTOTUNE_CACHE");
  if (cache && *cache) {
    std::ifstream in(cache);
    std::string k;
    int m = 0, g = 0, pg = 0, sc = 0;
    while (in >> k >> m >> g >> pg >> sc) {
      if (k == key && g > 0 && (m == 0 || (m == 2 && sc == 1 && fused_ok(s)) || (m == 3 && sc == 1 && s->stream2) ||
                                (m == 5 && sc == 1 && pipe1_ok(s)) || (m == 6 && sc == 1 && owned_ready(s)) ||
                                (m == 1 && s->persist_ok && pg > 0) ||
                                (m == 4 && s->persist_ok && pg > 0 && sc == 1 && s->sb.wi3[0])) &&
          (sc == s->scheme || both)) {
        set_scheme(s, sc);
        s->mode = m;
        s->deliver_grid = g;
        if (pg > 0) s->persist_grid = pg;
        rc = capture_graph(s);
        if (rc == NGB_OK && deliver_grid_out)
          *deliver_grid_out = (m == 1 || m == 4) ? s->persist_grid : m == 6 ? s->own.G : g;
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
  int best_mode = 0, best_grid = s->deliver_grid, best_pgrid = s->persist_grid, best_scheme = s->scheme;
  double best_ms = 1e30;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<int> schemes;
  if (both) schemes = {1, 2};
  else schemes = {s->scheme};
  for (int scheme : schemes) {
    if (rc != NGB_OK) break;
    set_scheme(s, scheme);
    s->mode = 0;
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
        best_scheme = scheme;
      }
    }
    // pipelined loops (ring scheme): two-stream graphs, and one kernel per
    // step for LIF networks; delivery blocks per SM
    for (int pm : {3, 5}) {
      if (rc != NGB_OK || scheme != 1 || !s->stream2) break;
      s->mode = pm;
      if (pm == 5 && !pipe1_ok(s)) break;
      for (int b : {1, 2, 4, 8}) {
        s->mode = pm;
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
          best_mode = pm;
          best_grid = s->deliver_grid;
          best_scheme = scheme;
        }
      }
      s->mode = 0;
    }
    // fused update + delivery in graphs (ring scheme)
    if (rc == NGB_OK && scheme == 1 && fused_ok(s)) {
      s->mode = 2;
      rc = capture_graph(s);
      if (rc == NGB_OK) rc = snapshot_restore(s, sn);
      if (rc == NGB_OK) {
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
          best_mode = 2;
          best_scheme = scheme;
        }
      }
      s->mode = 0;
    }
    // persistent step kernel (and its pipelined variant with the ring scheme): blocks per SM
    for (int pm : {1, 4}) {
      if (rc != NGB_OK || !s->persist_ok || (pm == 4 && (scheme != 1 || !s->sb.wi3[0]))) continue;
      s->mode = pm;
      for (int b : {1, 2, 3, 4}) {
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
          best_mode = pm;
          best_pgrid = s->persist_grid;
          best_scheme = scheme;
        }
      }
      s->mode = 0;
    }
    // target-owned persistent kernel (LIF networks, ring scheme; layout built on first use)
    if (rc == NGB_OK && scheme == 1 && owned_ready(s)) {
      s->mode = 6;
      rc = snapshot_restore(s, sn);
      if (rc == NGB_OK) {
        CK(launch_owned_chunk(s, 100));  // warm-up
        CK(cudaEventRecord(e0, s->stream));
        CK(launch_owned_chunk(s, trial_steps));
        CK(cudaEventRecord(e1, s->stream));
        CK(cudaEventSynchronize(e1));
        uint32_t err = 0;
        CK(cudaMemcpy(&err, s->sb.err, sizeof(err), cudaMemcpyDeviceToHost));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double per_step = ms / (double)trial_steps;
        if (!(err & kErrBarrierTimeout) && per_step < best_ms) {
          best_ms = per_step;
          best_mode = 6;
          best_scheme = scheme;
        }
      }
      s->mode = 0;
    }
  }
  // the AdEx hot lists (on in the trials above) against none, in the chosen per-step loop
  bool best_hot = s->hot_use;
  if (rc == NGB_OK && s->hot_on && s->hot_use && s->n_aeif && (best_mode == 0 || best_mode == 3)) {
    set_scheme(s, best_scheme);
    s->mode = best_mode;
    s->deliver_grid = best_grid;
    s->hot_use = false;
    rc = capture_graph(s);
    if (rc == NGB_OK) rc = snapshot_restore(s, sn);
    if (rc == NGB_OK) {
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
        best_hot = false;
      }
    }
    s->mode = 0;
  }
  // a loop other than the per-step kernels keeps no lists (and profiled per-step runs then match it)
  s->hot_use = best_hot && (best_mode == 0 || best_mode == 3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == NGB_OK) rc = snapshot_restore(s, sn);
  snapshot_free(sn);
  s->graph_steps = saved_graph_steps;
  set_scheme(s, best_scheme);
  s->deliver_grid = best_grid;
  s->persist_grid = best_pgrid;
  if (s->tl.pairs) {  // a target-tiled layout (selected at finalisation) is no longer used
    s->dev_bytes -= s->tl.bytes;
    tiled_free(&s->tl);
  }
  s->mode = best_mode;
  if (rc == NGB_OK) rc = capture_graph(s);
  if (rc != NGB_OK) return rc;
  if (cache && *cache) {
    std::ofstream out(cache, std::ios::app);
    out << key << " " << best_mode << " " << best_grid << " "
        << (s->persist_ok ? best_pgrid : 0) << " " << best_scheme << "\n";
  }
  if (deliver_grid_out)
    *deliver_grid_out = (best_mode == 1 || best_mode == 4) ? best_pgrid : best_mode == 6 ? s->own.G : best_grid;
  return NGB_OK;
}

int ngb_reserve(ngb_sim* s, int64_t max_neurons, int64_t max_synapses, int64_t max_groups, int32_t ring_slots,
                int32_t receptors) {
  if (!s) return fail(NGB_ERR_INVALID_ARG, "NULL handle");
  if (s->finalized) return fail(NGB_ERR_STATE, "ngb_reserve: network already finalised");
  if (!s->stdp_params.empty()) return fail(NGB_ERR_STATE, "ngb_reserve: STDP synapses are not served");
  if (max_neurons <= 0 || max_neurons >= (int64_t)kIdMask || max_synapses < 0 || max_groups < 0 ||
      ring_slots < 2 || ring_slots > 4096 || (ring_slots & (ring_slots - 1)) != 0 || receptors < 1 ||
      receptors > kMaxPorts)
    return fail(NGB_ERR_INVALID_ARG, "ngb_reserve: capacities");
  if (max_neurons < s->N) return fail(NGB_ERR_INVALID_ARG, "ngb_reserve: fewer neurons than already added");
  for (const PopHost& p : s->pops)
    if (receptors_of(p) > receptors)
      return fail(NGB_ERR_INVALID_ARG, "ngb_reserve: a population needs more receptors");
  s->serving = true;
  s->N_cap = max_neurons;
  s->K_cap = (uint64_t)max_synapses;
  s->G_cap = (uint64_t)max_groups;
  s->L = ring_slots;
  s->R = receptors;
  for (PopHost& p : s->pops) p.offset = -1;
  return NGB_OK;
}

int ngb_commit_instance(ngb_sim* s, int32_t instance) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->serving) return fail(NGB_ERR_STATE, "ngb_commit_instance: needs ngb_reserve before finalising");
  if (instance < 0 || instance >= (int32_t)s->inst.size())
    return fail(NGB_ERR_INVALID_ARG, "ngb_commit_instance: instance");
  for (const PopHost& p : s->pops)
    if (p.instance == instance && receptors_of(p) > s->R)
      return fail(NGB_ERR_INVALID_ARG, "ngb_commit_instance: a population needs more receptors than reserved");
  if (!s->finalized) {
    rc = finalize_impl(s);
    if (rc != NGB_OK) {
      s->failed = true;
      return rc;
    }
    return s->inst[(size_t)instance].state == 1 ? NGB_OK : commit_impl(s, instance);
  }
  return commit_impl(s, instance);
}

int ngb_retire_instance(ngb_sim* s, int32_t instance) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->serving) return fail(NGB_ERR_STATE, "ngb_retire_instance: not a serving handle");
  if (instance < 0 || instance >= (int32_t)s->inst.size() || s->inst[(size_t)instance].state != 1)
    return fail(NGB_ERR_INVALID_ARG, "ngb_retire_instance: instance is not active");
  CK(cudaStreamSynchronize(s->stream));
  if (s->scheme == 2) {
    // spikes of the instance still waiting for a connection group are dropped
    const int pb = (int)(s->t & 1);
    for (const PopHost& p : s->pops) {
      if (p.instance != instance || !p.placed) continue;
      CK(launch_kill_pending(s->sb.pend[pb], s->sb.pcnt + pb, s->sb.pend_cap, (uint32_t)p.offset,
                             (uint32_t)(p.offset + p.n), s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
  }
  release_instance_ranges(s, instance);
  s->inst[(size_t)instance].state = 2;
  s->tables_dirty = true;
  return NGB_OK;
}

int ngb_instance_info(ngb_sim* s, int32_t instance, int64_t* t0_out, int32_t* state_out) {
  if (!s || instance < 0 || instance >= (int32_t)s->inst.size())
    return fail(NGB_ERR_INVALID_ARG, "ngb_instance_info: instance");
  if (t0_out) *t0_out = s->inst[(size_t)instance].t0;
  if (state_out) *state_out = s->inst[(size_t)instance].state;
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
    int64_t smin = s->rec_steps[a], smax = smin;
    for (size_t i = a; i < a + n; ++i) {
      smin = std::min(smin, s->rec_steps[i]);
      smax = std::max(smax, s->rec_steps[i]);
    }
    const uint64_t span = (uint64_t)(smax - smin) + 1;
    if (span <= 4 * (uint64_t)n + 4096) {
      // counting sort by step (the tail covers the steps of the last drains),
      // then the ids of each step in place
      std::vector<size_t> start(span + 1, 0);
      for (size_t i = a; i < a + n; ++i) start[(size_t)(s->rec_steps[i] - smin) + 1] += 1;
      for (size_t k = 1; k <= span; ++k) start[k] += start[k - 1];
      std::vector<uint32_t> ni(n);
      std::vector<size_t> cur(start.begin(), start.end() - 1);
      for (size_t i = a; i < a + n; ++i) ni[cur[(size_t)(s->rec_steps[i] - smin)]++] = s->rec_ids[i];
      for (size_t k = 0; k < span; ++k) {
        std::sort(ni.begin() + (ptrdiff_t)start[k], ni.begin() + (ptrdiff_t)start[k + 1]);
        std::fill(s->rec_steps.begin() + (ptrdiff_t)(a + start[k]), s->rec_steps.begin() + (ptrdiff_t)(a + start[k + 1]),
                  smin + (int64_t)k);
      }
      std::copy(ni.begin(), ni.end(), s->rec_ids.begin() + (ptrdiff_t)a);
    } else {
      std::vector<std::pair<int64_t, uint32_t>> kv(n);
      for (size_t i = 0; i < n; ++i) kv[i] = {s->rec_steps[a + i], s->rec_ids[a + i]};
      std::sort(kv.begin(), kv.end());
      for (size_t i = 0; i < n; ++i) {
        s->rec_steps[a + i] = kv[i].first;
        s->rec_ids[a + i] = kv[i].second;
      }
    }
    s->rec_sorted_upto = s->rec_ids.size();
  }
  const int64_t lo = pop >= 0 ? s->pops[pop].offset : 0;
  const int64_t hi = pop >= 0 ? s->pops[pop].offset + s->pops[pop].n : std::max<int64_t>(s->N, s->N_cap);
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
  out->num_neurons = s->finalized ? s->N_cap : s->N;
  out->spikes = s->spikes_total;
  if (s->finalized) {
    const int rc = check_handle(s);
    if (rc != NGB_OK) return rc;
    unsigned long long c[4] = {0, 0, 0, 0};  // events, substeps, rec_count, hot_steps
    CK(cudaMemcpyAsync(c, s->sb.events, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    out->events = (int64_t)c[0];
    out->rk_substeps = (int64_t)c[1];
    out->hot_steps = (int64_t)c[3];
    out->num_synapses = (int64_t)s->K;
    out->num_groups = (int64_t)s->G;
    out->ring_slots = s->L;
    out->max_delay_steps = s->max_delay;
    out->device_bytes = (int64_t)s->dev_bytes;
    out->mode = s->mode;
    out->launch_grid = (s->mode == 1 || s->mode == 4) ? s->persist_grid
                       : s->mode == 6 ? s->own.G
                       : s->mode == 7 ? (int64_t)s->tl.n_tiles * s->tl_P
                       : s->mode == 2 ? s->lif_blocks + s->aeif_blocks + s->aeifa_blocks
                                      : s->deliver_grid;  // graph and pipelined loops: the delivery grid
    out->delivery = s->scheme;
  }
  return NGB_OK;
}

int ngb_population_range(ngb_sim* s, int32_t pop, int64_t* offset_out, int64_t* n_out) {
  if (!s || pop < 0 || pop >= (int32_t)s->pops.size())
    return fail(NGB_ERR_INVALID_ARG, "ngb_population_range: pop");
  if (s->pops[pop].offset < 0) return fail(NGB_ERR_STATE, "ngb_population_range: population not placed yet");
  if (offset_out) *offset_out = s->pops[pop].offset;
  if (n_out) *n_out = s->pops[pop].n;
  return NGB_OK;
}

int ngb_get_state(ngb_sim* s, int32_t var, int64_t first, int64_t n, float* out) {
  int rc = check_handle(s);
  if (rc != NGB_OK) return rc;
  if (!s->finalized) return fail(NGB_ERR_STATE, "ngb_get_state: not finalised");
  if (!out || first < 0 || n < 0 || first + n > s->N_cap) return fail(NGB_ERR_INVALID_ARG, "ngb_get_state: range");
  const float* src = nullptr;
  bool is_ref = false;
  switch (var) {
    case NGB_VAR_V_M: src = s->st0; break;
    case NGB_VAR_I_SYN: src = s->st1; break;
    case NGB_VAR_G_EX: src = s->st2; break;
    case NGB_VAR_G_IN: src = s->st3; break;
    case NGB_VAR_H: src = s->st4; break;
    case NGB_VAR_DG_EX: src = s->st5; break;
    case NGB_VAR_DG_IN: src = s->st6; break;
    case NGB_VAR_G_2:
    case NGB_VAR_G_3:
    case NGB_VAR_X_2:
    case NGB_VAR_X_3:
      src = s->ext ? s->ext + (size_t)(var - NGB_VAR_G_2) * (size_t)s->N_cap : nullptr;
      break;
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
      first + n > s->N_cap)
    return fail(NGB_ERR_INVALID_ARG, "ngb_get_input: range");
  if (s->scheme == 2 && step_offset != 0)
    return fail(NGB_ERR_INVALID_ARG,
                "ngb_get_input: with spike-buffer delivery only the next step's input (step_offset 0) exists");
  if (n == 0) return NGB_OK;
  const uint64_t slot = s->scheme == 2 ? 0 : (uint64_t)((s->t + step_offset) & (s->L - 1));
  const uint64_t off = (slot * (uint64_t)s->R + (uint64_t)receptor) * (uint64_t)s->N_cap + (uint64_t)first;
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
  CK(cudaMemcpyAsync(src_ptr, s->src_syn, (s->N_cap + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
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
  cudaError_t e = cudaSuccess;
  if (s->wa) e = sync_stdp_weights(s->wa, s->tgt, (uint64_t)first, (uint64_t)n, (float*)s->w, s->stream);
  if (e == cudaSuccess)
    e = expand_synapses((uint64_t)first, (uint64_t)n, s->tgt, s->w, s->cfg.weight_dtype, s->grp_start, s->G,
                        s->grp_delay, d_t, d_r, d_w, d_d, s->stream);
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
