// ngb_internal.cuh -- device data layout and helpers shared by the library's
// translation units (not part of the C ABI).
//
// Data layout in HBM (N neurons, K synapses, G connection groups, L ring
// slots, R receptors):
//   state      SoA FP32 arrays of N (LIF: y = V - E_L, I, refractory counter;
//              AdEx: V, w, g_ex, g_in, h, x_ex, x_in; beta multisynapse
//              ports 0-1 in g_ex, g_in, x_ex, x_in and ports 2-3 in a
//              [4][N] block g_2, g_3, x_2, x_3)
//   ring       [L][R][N] FP32 (or int64 fixed point in deterministic mode);
//              slot (t + d) & (L - 1) receives the spikes of step t with delay d
//   CSR        src_syn[N+1] u64 (first synapse of each source),
//              src_grp[N+1] u32 (first delay group of each source),
//              grp_start[G+1] u64 and grp_delay[G] u16 (Sec. 2.2 connection
//              groups: a source's synapses with equal delay, in delay order),
//              tgt[K] u32 (bits 30-31 = receptor, bits 26-29 = STDP rule + 1
//              or 0 for a static synapse, bits 0-25 = global target),
//              w[K] FP32 / BF16 / FP16
//   src_meta   uint4 per source {row start lo, row start hi (16 bits) | groups
//              << 16, synapses, first group}: everything delivery needs about
//              a spiking source, read once by the update kernel
//   work items per step (double-buffered by step parity): 2 x uint4 per
//              work item of 128 synapses ({neuron | multiplicity << 26, index
//              of the item within its source, meta.x, meta.y}, {meta.z,
//              meta.w, 0, 0}) and one packed u64 counter (spikes << 38 |
//              work items); capacity = the work items of all sources
//
// Two delivery schemes share these arrays:
//   ring          (push at spike time) every spike of step t is scattered
//                 at once into ring slots t + d of all its groups; the ring
//                 has L slots;
//   spike buffer  (Sec. 2.2: a spike carries an age and the index of its next
//                 connection group, and reaches a group when its age equals
//                 the group's delay) the ring has one slot, the input of the
//                 next step.  Spikes whose groups are not all delivered wait
//                 in a pending list (double-buffered by step parity, one
//                 uint4 per spike: {neuron | multiplicity << 26, next group,
//                 end group, due step (low 32 bits)}).  Every step the update
//                 kernel moves the spikes whose next group is due (age + 1 =
//                 delay: delivered after step t into the input of step t+1)
//                 to the step's due-item list (one uint4 per <= 1024
//                 synapses of one group: {first synapse lo, hi | multiplicity
//                 << 16, synapses, 0}), which the delivery kernel scatters
//                 into the single slot.  The scattered-to array is N x R
//                 words instead of L x N x R, so it stays in L2 for networks
//                 whose ring would not.
//   src_age    uint2 per source {synapses of its first group, delay of the
//              first group | delay of the second group << 16}: what a new
//              spike needs to decide whether its first group is due at once
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ngb {

constexpr int kChunk = 128;          // synapses per delivery work item: 32 lanes x 4
constexpr int kSpkShift = 38;        // packed per-step counter: spikes << 38 | work items
constexpr unsigned long long kChunkMask = (1ull << kSpkShift) - 1;
constexpr int kIdBits = 26;          // spike-list word: neuron id bits
constexpr uint32_t kIdMask = (1u << kIdBits) - 1;
constexpr int kMaxThr = 255;         // Poisson inversion table length (largest count drawn)
constexpr int kDelayBits = 12;       // delays up to 4095 steps
constexpr int kMaxDelay = (1 << kDelayBits) - 1;
constexpr int kRcptShift = 30;       // synapse target word: receptor << 30 | rule << 26 | target
constexpr int kPlastShift = 26;      // STDP rule + 1 (0: static synapse), 4 bits
constexpr uint32_t kPlastMask = 15u;
constexpr uint32_t kTgtMask = (1u << kPlastShift) - 1;
constexpr int kMaxStdpRules = 15;
constexpr int kStdpRuleShift = 40;   // incoming-plastic-synapse word: rule << 40 | synapse index
constexpr int kMaxPorts = 4;         // receptor ports of the beta multisynapse AdEx

// error flags (device word)
constexpr uint32_t kErrRecordOverflow = 1u;
constexpr uint32_t kErrSubstepCap = 2u;
constexpr uint32_t kErrBarrierTimeout = 4u;
constexpr uint32_t kErrPendingOverflow = 8u;

// spike-buffer delivery
constexpr uint32_t kAgeSpan = 1024;         // synapses per due item
constexpr uint32_t kDeadWord = 0xFFFFFFFFu;  // pending entry removed (its instance was retired)

// random-stream purposes: counter word 2 = purpose | attempt << 8
enum : uint32_t { kPurSrc = 1, kPurWeight = 2, kPurDelay = 3, kPurPoisson = 4, kPurVinit = 5 };

struct LifSeg {
  int64_t offset;      // first global neuron id
  int64_t n;           // neurons
  int64_t blk_begin;   // first block of the segment in the LIF update grid
  int64_t t0;          // global step at which the instance started
  uint64_t seed;       // instance key
  uint32_t local_off;  // instance-local id of the first neuron
  uint32_t n_thr;      // Poisson thresholds in use
  uint32_t thr_off;    // offset of the thresholds in the table
  int32_t ref_steps;
  float P11, P21, P22, P20Ie, theta, y_reset, w_ext, pad_;
};

struct AeifSeg {
  int64_t offset, n, blk_begin, t0;
  uint64_t seed;
  uint32_t local_off, n_thr, thr_off;
  int32_t prec_rcpt;   // receptor of the Poisson drive
  int32_t ctl32;       // step-size control in FP32 instead of FP64
  int32_t alpha;       // alpha-function conductances (state x_ex, x_in)
  float g_L, E_L, V_T, Delta_T, inv_Delta_T, a, inv_tau_w, V_peak, V_reset, b;
  float E_ex, E_in, inv_tau_ex, inv_tau_in, I_e, inv_C, w_ext;
  float e_tau_ex, e_tau_in;  // e / tau: the jump of x per unit input weight (alpha)
  int32_t n_ports;           // beta multisynapse: ports in use (1-4)
  // beta ports (unused ports: E 0, 1/tau 1, jump 0): reversal potential, 1 / decay
  // time, 1 / rise time, jump of x per unit weight (the peak of g equals the weight)
  float E_p[4], itd_p[4], itr_p[4], jmp_p[4];
  float inv_tol_f;     // 1 / tolerance rounded to FP32 (the FP32 side of the error-ratio test)
  float V_hot;         // a step ending above this V lists the neuron as hot for the next step (+inf: never)
  double inv_tol, h_min, dt;
  int64_t max_sub;
};

struct SpikeBuf {
  uint4* wi[2];                     // 2 entries per delivery work item
  unsigned long long* ctr;          // [2] packed per-step counters
  unsigned long long* events;       // synaptic events delivered (cumulative)
  unsigned long long* substeps;     // RK sub-steps (cumulative)
  unsigned long long* hot_steps;    // AdEx neuron steps run from the hot lists (cumulative)
  uint32_t* rec_id;                 // spike record, rec_cap entries
  int64_t* rec_step;
  unsigned long long* rec_count;    // spikes since the last drain (with multiplicity)
  int64_t rec_cap;
  uint32_t* err;
  // spike-buffer delivery
  uint4* pend[2];                   // pending spikes, by step parity
  unsigned long long* pcnt;         // [2] pending-list lengths
  int64_t pend_cap;                 // entries per pending list
  int64_t wi_cap;                   // uint4 entries per work-item / due-item list
  // AdEx neurons whose step did not finish within the update kernel's attempt
  // budget (by conductance model: 0 exponential, 1 alpha, 2 beta), finished by
  // a second kernel with the neurons packed into full warps
  uint4* dfr[3];                    // 4 uint4 per neuron (beta: 6)
  unsigned long long* dcnt;         // [model * 2 + step parity]
  int64_t dfr_cap;                  // neurons per list
  // the finishing kernel's queue position in the deferred list, by model
  // (zeroed by the step's update kernel)
  unsigned long long* dfetch;
  // AdEx neurons listed as hot for a step (their previous step ended above
  // V_hot: mostly those about to cross V_peak, whose step takes tens of
  // attempts): {neuron, segment} by conductance model, three lists of hot_cap
  // entries by step mod 3, run by a kernel of their own beside the update
  // kernel, which skips them.  htag[n] holds the step (low 32 bits) neuron n was
  // last listed for; an entry counts only when its neuron's tag names the step.
  uint2* hot[3];
  unsigned long long* hcnt;         // [model * 3 + step mod 3]
  uint32_t* htag;
  int64_t hot_cap;                  // entries per list
  // pipelined ring scheme: work-item lists and counters by step mod 3
  uint4* wi3[3];
  unsigned long long* ctr3;         // [3]
  // STDP (NULL without plastic synapses): the latest spike step of every
  // neuron (-1: none), the first incoming plastic synapse of every neuron
  // (in_ptr[N+1]), and the neurons with plastic inputs that fired in the
  // step, by step parity (post[2], counts post_cnt[2], capacity N each)
  int32_t* last_spike;
  const uint64_t* in_ptr;
  uint32_t* post[2];
  unsigned long long* post_cnt;
  // target-tiled delivery (spike-buffer scheme in the graph loop, mode 7;
  // NULL otherwise): each due connection group is one item {first pair of
  // the group in the tiled copy lo, hi | multiplicity << 16, first target
  // tile, boundary-pool offset},
  // appended to the bucket of the first target tile its synapses reach
  const uint4* tile_grp;            // per group {boundary-pool offset, first target tile, first pair lo, hi}
  uint4* bkt[2];                    // bucket items by step parity (bucket j at boff[j])
  const unsigned long long* boff;   // [n_tiles + 1]: bucket j holds the groups whose first tile is j
  unsigned int* bcnt;               // [2][n_tiles] bucket fill counts by step parity
  uint32_t n_tiles;
};

// Nearest-neighbour STDP rule (Sec. 2.1): FP32 constants and the tabulated
// pair factors e^(-n dt / tau) for lags n < n_plus / n_minus.
struct StdpRule {
  float A_plus, A_minus, inv_W_max, W_max, mu_plus, mu_minus;
  int32_t n_plus, n_minus;
  const float* k_plus;
  const float* k_minus;
};

// Plastic synapses: the rules, per synapse its mutable FP32 weight and its
// latest arrival step (-1: none) side by side in one 8-byte word {weight
// bits, arrival} (a potentiation then touches one random sector, not two; the
// CSR's FP32 weight of a plastic synapse is refreshed from it only for
// introspection), and the incoming plastic synapses of every neuron
// (rule << 40 | synapse index).
struct StdpArgs {
  const StdpRule* rules;
  uint2* wa;
  const uint64_t* in_syn;
};

struct Csr {
  const uint4* src_meta;
  const uint64_t* src_syn;
  const uint32_t* src_grp;
  const uint64_t* grp_start;
  const uint16_t* grp_delay;
  const uint32_t* tgt;
  const void* w;
  const uint2* src_age;
  int32_t wdtype;  // storage of w: 0 FP32, 1 BF16, 2 FP16
};

struct Ring {
  void* p;          // float* or long long*
  int64_t N;        // neurons (plane stride)
  uint32_t L_mask;  // L - 1
  int32_t R;        // receptors per slot
};

// Warp-ballot compaction of the spikes of one warp into the step's spike
// list (Sec. 2.2 spike array, at most N entries), with one atomic per warp
// reserving both list positions and delivery work items, plus the spike
// record.  Every lane of the warp must call it (no early exit before it).
// A spiking lane writes one entry per delivery work item of its source,
// carrying the source's row and group range, so the delivery kernel maps a
// work item to its synapses with a single load.
__device__ __forceinline__ void emit_spikes(bool spk, uint32_t gid, uint32_t mult, int64_t t, uint4 meta,
                                            const SpikeBuf& sb) {
  const unsigned full = 0xffffffffu;
  const unsigned ball = __ballot_sync(full, spk);
  if (ball == 0) return;
  const int lane = threadIdx.x & 31;
  uint32_t nch = 0, m = 0;
  unsigned long long nev = 0;
  if (spk) {
    const uint64_t b = (uint64_t)meta.x | ((uint64_t)(meta.y & 0xFFFFu) << 32);
    const uint64_t e = b + meta.z;
    if (e > b) nch = (uint32_t)((e - (b & ~3ull) + kChunk - 1) / kChunk);
    m = mult;
    nev = (unsigned long long)meta.z * mult;
  }
  uint32_t inc_ch = nch, inc_m = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(full, inc_ch, o);
    const uint32_t c = __shfl_up_sync(full, inc_m, o);
    if (lane >= o) {
      inc_ch += a;
      inc_m += c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nev += __shfl_xor_sync(full, nev, o);
  const uint32_t tot_ch = __shfl_sync(full, inc_ch, 31);
  const uint32_t tot_m = __shfl_sync(full, inc_m, 31);
  const int buf = (int)(t & 1);
  unsigned long long base = 0, rbase = 0;
  if (lane == 0) {
    base = atomicAdd(sb.ctr + buf, ((unsigned long long)__popc(ball) << kSpkShift) | tot_ch);
    rbase = atomicAdd(sb.rec_count, (unsigned long long)tot_m);
    atomicAdd(sb.events, nev);
  }
  base = __shfl_sync(full, base, 0);
  rbase = __shfl_sync(full, rbase, 0);
  if (spk) {
    const uint32_t rank = __popc(ball & ((1u << lane) - 1u));
    const unsigned long long pos = (base >> kSpkShift) + rank;
    (void)pos;
    uint4* const wi = buf ? sb.wi[1] : sb.wi[0];
    const uint64_t first = (base & kChunkMask) + inc_ch - nch;
    const uint32_t word = gid | (mult << kIdBits);
    for (uint32_t c = 0; c < nch; ++c) {
      wi[2 * (first + c)] = make_uint4(word, c, meta.x, meta.y);
      wi[2 * (first + c) + 1] = make_uint4(meta.z, meta.w, 0u, 0u);
    }
    if (sb.rec_cap > 0) {
      const unsigned long long r0 = rbase + inc_m - m;
      for (uint32_t k = 0; k < m; ++k) {
        if (r0 + k < (unsigned long long)sb.rec_cap) {
          sb.rec_id[r0 + k] = gid;
          sb.rec_step[r0 + k] = t;
        } else {
          atomicOr(sb.err, kErrRecordOverflow);
        }
      }
    }
  }
}

// ------------------------------------------------------------ spike buffer
// The spike-buffer scheme (Sec. 2.2).  Every lane of the warp must call these
// (no early exit before them); lists are filled with one atomic per warp.

// Warp-aggregated output of the spike-buffer bookkeeping: lane contributes
// n_it due items covering the n synapses from b (multiplicity mult) to the
// due-item list of parity ib, and, if keep, the pending entry ent to the
// pending list of parity pb.  Positions beyond the lists' capacities are
// dropped and raise kErrPendingOverflow.
// With target-tiled delivery (sb.bkt set) the lane's due group g (n_it > 0)
// becomes one item in the bucket of its first target tile instead, with one
// atomic per bucket and warp.
__device__ __forceinline__ void age_emit(uint32_t n_it, uint64_t b, uint32_t n, uint32_t mult, bool keep, uint4 ent,
                                         int ib, int pb, const SpikeBuf& sb, uint32_t g = 0) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (sb.bkt[0]) {
    const bool has = n_it > 0;
    const unsigned act = __ballot_sync(full, has);
    if (has) {
      const uint4 tg = __ldg(sb.tile_grp + g);
      const uint32_t j = tg.y;
      const unsigned peers = __match_any_sync(act, j);
      const int leader = __ffs(peers) - 1;
      unsigned int base = 0;
      if (lane == leader) base = atomicAdd(sb.bcnt + (size_t)ib * sb.n_tiles + j, (unsigned int)__popc(peers));
      base = __shfl_sync(peers, base, leader);
      const unsigned long long slot = (unsigned long long)base + __popc(peers & ((1u << lane) - 1u));
      const unsigned long long b0 = __ldg(sb.boff + j);
      if (slot < __ldg(sb.boff + j + 1) - b0)
        (ib ? sb.bkt[1] : sb.bkt[0])[b0 + slot] = make_uint4(tg.z, (tg.w & 0xFFFFu) | (mult << 16), j, tg.x);
      else
        atomicOr(sb.err, kErrPendingOverflow);
    }
    n_it = 0;
  }
  const unsigned kb = __ballot_sync(full, keep);
  uint32_t inc = n_it;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(full, inc, o);
    if (lane >= o) inc += a;
  }
  const uint32_t tot = __shfl_sync(full, inc, 31);
  if (tot == 0 && kb == 0) return;
  unsigned long long ibase = 0, pbase = 0;
  if (lane == 0) {
    if (tot) ibase = atomicAdd(sb.ctr + ib, (unsigned long long)tot);
    if (kb) pbase = atomicAdd(sb.pcnt + pb, (unsigned long long)__popc(kb));
  }
  ibase = __shfl_sync(full, ibase, 0) & kChunkMask;
  pbase = __shfl_sync(full, pbase, 0);
  if (n_it) {
    uint4* const di = ib ? sb.wi[1] : sb.wi[0];
    const unsigned long long first = ibase + inc - n_it;
    for (uint32_t k = 0; k < n_it; ++k) {
      const uint64_t bk = b + (uint64_t)k * kAgeSpan;
      const uint32_t nk = n - k * kAgeSpan < kAgeSpan ? n - k * kAgeSpan : kAgeSpan;
      if (first + k < (unsigned long long)sb.wi_cap)
        di[first + k] = make_uint4((uint32_t)bk, (uint32_t)((bk >> 32) & 0xFFFFu) | (mult << 16), nk, 0u);
      else
        atomicOr(sb.err, kErrPendingOverflow);
    }
  }
  if (keep) {
    const unsigned long long pos = pbase + __popc(kb & ((1u << lane) - 1u));
    uint4* const pl = pb ? sb.pend[1] : sb.pend[0];
    if (pos < (unsigned long long)sb.pend_cap) pl[pos] = ent;
    else atomicOr(sb.err, kErrPendingOverflow);
  }
}

// Spike record and event count of the new spikes of one warp (spike-buffer
// scheme; the ring scheme does the same inside emit_spikes).
__device__ __forceinline__ void record_spikes(bool spk, uint32_t gid, uint32_t mult, int64_t t,
                                              unsigned long long nev, const SpikeBuf& sb) {
  const unsigned full = 0xffffffffu;
  if (__ballot_sync(full, spk) == 0) return;
  const int lane = threadIdx.x & 31;
  uint32_t m = spk ? mult : 0u, inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(full, inc, o);
    if (lane >= o) inc += a;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nev += __shfl_xor_sync(full, nev, o);
  const uint32_t tot = __shfl_sync(full, inc, 31);
  unsigned long long rbase = 0;
  if (lane == 0) {
    rbase = atomicAdd(sb.rec_count, (unsigned long long)tot);
    atomicAdd(sb.events, nev);
  }
  rbase = __shfl_sync(full, rbase, 0);
  if (spk && sb.rec_cap > 0) {
    const unsigned long long r0 = rbase + inc - m;
    for (uint32_t k = 0; k < m; ++k) {
      if (r0 + k < (unsigned long long)sb.rec_cap) {
        sb.rec_id[r0 + k] = gid;
        sb.rec_step[r0 + k] = t;
      } else {
        atomicOr(sb.err, kErrRecordOverflow);
      }
    }
  }
}

// New spikes of step t in the spike-buffer scheme: a spike whose first group
// has delay 1 is due at once (its synapses go to the due-item list of step
// t); otherwise, and while groups remain, it joins the pending list of step
// t + 1.  Synaptic events are counted at spike time, as in the ring scheme.
// STDP bookkeeping of the neurons that fired at step t: the step is recorded
// as their latest spike, and those with plastic inputs join the step's list
// for potentiation (each neuron at most once per step, so the list of
// capacity N cannot overflow).  Every lane of the warp must call it.
__device__ __forceinline__ void stdp_post_spike(bool spk, uint32_t gid, int64_t t, const SpikeBuf& sb) {
  bool listed = false;
  if (spk) {
    sb.last_spike[gid] = (int32_t)t;
    listed = __ldg(sb.in_ptr + gid + 1) > __ldg(sb.in_ptr + gid);
  }
  const unsigned b = __ballot_sync(0xffffffffu, listed);
  if (b == 0) return;
  const int lane = threadIdx.x & 31;
  const int pb = (int)(t & 1);
  const int leader = __ffs(b) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(sb.post_cnt + pb, (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (listed) (pb ? sb.post[1] : sb.post[0])[base + __popc(b & ((1u << lane) - 1u))] = gid;
}

__device__ __forceinline__ void emit_spikes_age(bool spk, uint32_t gid, uint32_t mult, int64_t t, const Csr& csr,
                                                const SpikeBuf& sb) {
  const unsigned ball = __ballot_sync(0xffffffffu, spk);
  if (ball == 0) return;
  if (sb.last_spike) stdp_post_spike(spk, gid, t, sb);
  uint4 meta = make_uint4(0, 0, 0, 0);
  uint2 ag = make_uint2(0, 0);
  if (spk) {
    meta = __ldg(csr.src_meta + gid);
    ag = __ldg(csr.src_age + gid);
  }
  const uint32_t ngrp = meta.y >> 16;
  const uint64_t bsrc = (uint64_t)meta.x | ((uint64_t)(meta.y & 0xFFFFu) << 32);
  const uint32_t d0 = ag.y & 0xFFFFu, d1 = ag.y >> 16;
  const bool has = spk && ngrp > 0;
  const bool now = has && d0 == 1u;
  const uint32_t n_it = now ? (ag.x + kAgeSpan - 1) / kAgeSpan : 0u;
  const bool keep = has && (!now || ngrp > 1u);
  const uint32_t word = gid | (mult << kIdBits);
  const uint4 ent = now ? make_uint4(word, meta.w + 1u, meta.w + ngrp, (uint32_t)(t + d1))
                        : make_uint4(word, meta.w, meta.w + ngrp, (uint32_t)(t + d0));
  record_spikes(spk, gid, mult, t, spk ? (unsigned long long)meta.z * mult : 0ull, sb);
  age_emit(n_it, bsrc, ag.x, mult, keep, ent, (int)(t & 1), (int)((t + 1) & 1), sb, meta.w);
}

// Pending spikes at the update of step t (spike-buffer scheme): a spike whose
// next group is due (due step == t + 1) sends that group to the due-item list
// of step t and advances to its next group; a spike with groups left stays
// in the pending list of step t + 1.  The warps [warp0, warp0 + nwarps) of
// the grid share the list, 32 entries per warp and pass.  kCoherent: the list
// was written by other SMs in the same launch.
template <bool kCoherent>
__device__ __forceinline__ void scan_pending(int64_t t, const Csr& csr, const SpikeBuf& sb, int64_t warp0,
                                             int64_t nwarps) {
  const int lane = threadIdx.x & 31;
  const int pb = (int)(t & 1);
  unsigned long long n = kCoherent ? __ldcg(sb.pcnt + pb) : sb.pcnt[pb];
  if (n > (unsigned long long)sb.pend_cap) n = (unsigned long long)sb.pend_cap;
  const uint4* const pl = pb ? sb.pend[1] : sb.pend[0];
  const uint32_t due_now = (uint32_t)(t + 1);
  for (unsigned long long base = (unsigned long long)warp0 * 32; base < n;
       base += (unsigned long long)nwarps * 32) {
    const unsigned long long i = base + lane;
    uint4 e = make_uint4(kDeadWord, 0, 0, 0);
    if (i < n) e = kCoherent ? __ldcg(pl + i) : pl[i];
    const bool live = e.x != kDeadWord;
    const bool due = live && e.w == due_now;
    uint32_t n_it = 0, sz = 0;
    uint64_t b = 0;
    bool keep = live;
    uint4 ent = e;
    if (due) {
      const uint32_t ig = e.y;
      const bool more = ig + 1u < e.z;
      b = __ldg(csr.grp_start + ig);
      const uint32_t dcur = __ldg(csr.grp_delay + ig);
      uint64_t end;
      uint32_t dnext = 0;
      if (more) {
        end = __ldg(csr.grp_start + ig + 1);
        dnext = __ldg(csr.grp_delay + ig + 1);
      } else {
        const uint4 m = __ldg(csr.src_meta + (e.x & kIdMask));
        end = ((uint64_t)m.x | ((uint64_t)(m.y & 0xFFFFu) << 32)) + m.z;
      }
      sz = (uint32_t)(end - b);
      n_it = (sz + kAgeSpan - 1) / kAgeSpan;
      keep = more;
      ent = make_uint4(e.x, ig + 1u, e.z, e.w - dcur + dnext);
    }
    age_emit(n_it, b, sz, e.x >> kIdBits, keep, ent, pb, pb ^ 1, sb, e.y);
  }
}

// Warp-aggregated append of the kW-entry records of the lanes whose AdEx step
// is unfinished (d) to deferred list `kind`.  Every lane of the warp must
// call it.  The list holds one record per neuron, each neuron is deferred at
// most once per step, so a position beyond the capacity is an internal error
// (flagged, record dropped).
template <int kW>
__device__ __forceinline__ void defer_write(bool d, const uint4 rec[kW], const SpikeBuf& sb, int kind, int64_t t) {
  const unsigned full = 0xffffffffu;
  const unsigned b = __ballot_sync(full, d);
  if (b == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(sb.dcnt + 2 * kind + (int)(t & 1), (unsigned long long)__popc(b));
  base = __shfl_sync(full, base, 0);
  if (d) {
    const unsigned long long pos = base + __popc(b & ((1u << lane) - 1u));
    if (pos < (unsigned long long)sb.dfr_cap) {
      uint4* q = sb.dfr[kind] + kW * pos;
#pragma unroll
      for (int i = 0; i < kW; ++i) q[i] = rec[i];
    } else {
      atomicOr(sb.err, kErrPendingOverflow);
    }
  }
}

// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialisation attribute may start while its predecessor in
// the stream finishes; griddep_wait() blocks until the predecessor grid has
// completed and its memory is visible, griddep_launch() lets the successor
// start.  Without the attribute both are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Segment tables passed by value in the kernel parameters (constant bank)
// when they are small; otherwise the kernels read the device copy.
constexpr int kInlineSegs = 12;
template <typename Seg>
struct SegTable {
  Seg s[kInlineSegs];
  const Seg* dev;           // device copy of all segments (always valid)
  const uint32_t* blk_seg;  // segment of every block (used when n > kInlineSegs)
  int n;
};

// The segment owning block `blk`: binary search over blk_begin in the inline
// copy (constant bank) or, for long tables (batched instances), the block's
// entry of the per-block segment table.
template <typename Seg>
__device__ __forceinline__ int segment_index_of(const SegTable<Seg>& T, int64_t blk) {
  if (T.n <= kInlineSegs) {
    int lo = 0, hi = T.n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (T.s[mid].blk_begin <= blk) lo = mid;
      else hi = mid;
    }
    return lo;
  }
  return (int)__ldg(T.blk_seg + blk);
}

template <typename Seg>
__device__ __forceinline__ Seg segment_of(const SegTable<Seg>& T, int64_t blk) {
  int lo = 0, hi = T.n;
  if (T.n <= kInlineSegs) {
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (T.s[mid].blk_begin <= blk) lo = mid;
      else hi = mid;
    }
    return T.s[lo];
  }
  (void)hi;
  return T.dev[__ldg(T.blk_seg + blk)];
}

// Arguments of the persistent step kernel (persistent.cu).
struct PersistArgs {
  const LifSeg* lseg;
  const AeifSeg* aseg;
  const int64_t* lvoff;  // [n_lseg + 1] first LIF-only index of each LIF segment
  const int64_t* avoff;  // [n_aseg + 1]
  const uint32_t* thr;
  float *st0, *st1, *st2, *st3, *st4, *st5, *st6;
  int32_t* ref;
  const uint4* src_meta;
  Ring ring;
  Csr csr;
  SpikeBuf sb;
  int64_t* clk;
  unsigned* bar;  // [0] arrivals, [1] generation, [2] abort
  int64_t n_lif, n_aeif, steps;
  unsigned long long spin_limit;
  uint32_t n_thr;
  int32_t n_lseg, n_aseg;
  int32_t withhold_block;  // test hook: this block never arrives at the first barrier (-1: none)
  int32_t age;             // spike-buffer delivery scheme
  uint32_t off_aseg, off_lvoff, off_avoff, off_thr;  // dynamic shared memory layout
};

// Target-owned persistent step loop (owned.cu): tile-major synapse items
// (G tiles of S items each, padded per source) and the per-neuron spike entry
// (C_s / 4) << 36 | off_s (0: no synapses).
struct OwnedLayout {
  void* items;      // uint2 items (wfmt 0) or 4-byte items (wfmt 1 BF16, 2 FP16 weights)
  int32_t wfmt;
  uint64_t* pub;
  uint64_t S;
  int G;
  uint32_t max_width;
};

constexpr int64_t kMaxOwnedSteps = 4 * 65535;  // steps per launch (mailbox stamps are 16 bits)

struct OwnedArgs {
  const LifSeg* seg;     // LIF segments in neuron order, contiguous from 0
  const uint32_t* thr;   // Poisson thresholds of all segments
  float *y, *I;
  int32_t* ref;
  void* ring;            // [L][ring_N] FP32 (int64 fixed point in deterministic mode), one receptor
  int64_t ring_N;
  int64_t N;             // neurons
  const void* items;     // [G][S] items in format wfmt
  int32_t wfmt;          // 0: {local | delay << 16, FP32 weight}; 1, 2: BF16, FP16 bits << 16 | delay << 10 | local
  const uint64_t* pub;   // [N]
  const uint64_t* src_syn;
  unsigned long long* mb;   // [4][G][4] mailboxes, by step mod 4
  unsigned long long* ovf;  // [4][G][T] overflow entries
  SpikeBuf sb;
  int64_t* clk;
  unsigned* abort;       // nonzero: a block gave up waiting
  int64_t steps;
  uint64_t S;
  unsigned long long spin_limit;
  uint32_t T;            // neurons per tile (block): ceil(N / G)
  uint32_t L_mask;
  uint32_t n_thr;
  int32_t n_seg;
  int32_t withhold_block;  // test hook: this block does not publish its first step (-1: none)
  uint32_t off_seg, off_thr, off_pub, off_ids, off_rec;  // dynamic shared memory layout (set by launch_owned)
};

// ------------------------------------------------------------------ host side
// Kernel launchers (one translation unit each).
// age: spike-buffer scheme; scan: this kernel also scans the pending list
// (the first update kernel of the step).
// Emission modes of the per-step update kernels: the ring scheme, the
// spike-buffer scheme, and the pipelined ring scheme (the delay-1 group of a
// spike delivered at once by the update kernel, the other groups queued by
// step mod 3 for a delivery kernel that runs beside the next update).
enum : int { kEmitRing = 0, kEmitAge = 1, kEmitPipe = 2 };

// npt: LIF neurons per thread (1 or 4); a block covers kLifBlock * npt neurons.
// The step is clk[0] + step_off.
cudaError_t launch_update_lif(const SegTable<LifSeg>& segs, int64_t blocks, int npt, const uint32_t* thr, float* y,
                              float* I, int32_t* ref, Ring ring, bool fixed, int64_t* clk, int64_t step_off,
                              const Csr& csr, SpikeBuf sb, int emit, bool scan, bool pdl, cudaStream_t st);
// AdEx state arrays (N_cap entries each): V, w, conductances and x of ports
// 0-1 (g_ex, g_in, x_ex, x_in), the carried RK step proposal h, and for beta
// ports 2-3 the block ext[4][N] = g_2, g_3, x_2, x_3 (NULL when no population
// has more than two ports).
struct AeifState {
  float *V, *w, *g0, *g1, *h, *x0, *x1, *ext;
  int64_t N;
};
// AdEx conductance models of the per-step kernels.
enum : int { kAeifExp = 0, kAeifAlpha = 1, kAeifBeta = 2 };
// model: kAeif*, the conductance model of every segment of the table.
// budget > 0: at most `budget` RK attempts per neuron in this kernel; the
// unfinished neurons are completed by launch_finish_aeif (same arithmetic).
// hot: the step's hot list runs in launch_hot_aeif beside this kernel, which
// skips the listed neurons and lists those ending above V_hot for the next step.
cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr,
                               const AeifState& S, int model, Ring ring, bool fixed, int64_t* clk, int64_t step_off,
                               const Csr& csr, SpikeBuf sb, int emit, bool scan, int budget, bool hot, bool pdl,
                               cudaStream_t st);
// The hot list of step clk[0] + step_off, whole steps, on a stream of its own
// forked after the previous step and joined before launch_finish_aeif.
cudaError_t launch_hot_aeif(const SegTable<AeifSeg>& segs, int grid, const uint32_t* thr, const AeifState& S,
                            int model, Ring ring, bool fixed, const int64_t* clk, int64_t step_off, const Csr& csr,
                            SpikeBuf sb, int emit, cudaStream_t st);
cudaError_t launch_finish_aeif(const SegTable<AeifSeg>& segs, int grid, const AeifState& S, int model, Ring ring,
                               bool fixed, int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, int emit,
                               bool hot, bool pdl, cudaStream_t st);
cudaError_t launch_tick(int64_t* clk, bool pdl, cudaStream_t st);
// pipe: the pipelined variant (ring scheme; one grid barrier per step).
cudaError_t persistent_max_blocks_per_sm(bool fixed, int wdtype, bool lif, bool aeif, bool pipe, size_t smem,
                                         int* out);
cudaError_t launch_persistent(const PersistArgs& a, bool fixed, int wdtype, bool lif, bool aeif, bool pipe, int grid,
                              size_t smem, cudaStream_t st);

// Per-source metadata for the update kernels' spike lists; *total_items
// (device) receives the delivery work items of all sources together.
cudaError_t launch_build_meta(int64_t N, const uint64_t* src_syn, const uint32_t* src_grp, uint4* meta,
                              unsigned long long* total_items, cudaStream_t st);

// Fused step loop (ring scheme, one launch per step and model): the update
// kernel delivers its block's own spikes.  t = clk[0] + step_off; clk[0]
// advances by a tick launch after each graph (or eager step).
cudaError_t launch_step_lif(const SegTable<LifSeg>& segs, int64_t blocks, const uint32_t* thr, float* y, float* I,
                            int32_t* ref, Ring ring, bool fixed, int wdtype, const int64_t* clk, int64_t step_off,
                            const Csr& csr, SpikeBuf sb, bool pdl, cudaStream_t st);
cudaError_t launch_step_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V, float* w,
                             float* gex, float* gin, float* h, float* xe, float* xi, bool alpha, Ring ring, bool fixed,
                             int wdtype, const int64_t* clk, int64_t step_off, const Csr& csr, SpikeBuf sb, bool pdl,
                             cudaStream_t st);
// Pipelined step kernel for LIF-only networks (ring scheme): upd_blocks update
// blocks (one LIF neuron per thread) and del_blocks blocks delivering the queue
// of the previous step when deliver_prev.
cudaError_t launch_step_pipe(const SegTable<LifSeg>& segs, int64_t upd_blocks, int del_blocks, const uint32_t* thr,
                             float* y, float* I, int32_t* ref, Ring ring, bool fixed, int wdtype, int64_t* clk,
                             int64_t step_off, const Csr& csr, SpikeBuf sb, bool deliver_prev, bool pdl,
                             cudaStream_t st);
// Target-owned loop: build the tile-major layout of a finalised CSR for G
// tiles and a ring of L slots (4-byte items with BF16 / FP16 weights when the
// tile holds at most 1,024 neurons and L <= 64, else 8-byte items; out->items
// NULL when C_s or the layout exceeds its limits or max_bytes; the caller
// frees pub and items), the dynamic shared memory of its kernel, its
// occupancy, and one cooperative launch of a.steps steps (grid G, mailboxes
// and overflow areas reset by the caller).
cudaError_t owned_build(const Csr& csr, const uint64_t* src_syn, int64_t N, int G, uint32_t L, uint64_t max_bytes,
                        OwnedLayout* out, cudaStream_t st);
size_t owned_smem_bytes(bool fixed, uint32_t L, uint32_t T, int n_seg, uint32_t n_thr);
cudaError_t owned_max_blocks_per_sm(bool fixed, uint32_t T, size_t smem, int wfmt, int* out);
cudaError_t launch_owned(OwnedArgs a, bool fixed, int grid, cudaStream_t st);
// clk[0] += n (clk[1] = clk[0] - 1); the ring scheme's step counters (both
// the per-step and the pipelined ones) are cleared.
cudaError_t launch_tick_add(int64_t* clk, int64_t n, unsigned long long* ctr, unsigned long long* ctr3, bool pdl,
                            cudaStream_t st);

// Launch `kernel` with the programmatic-serialisation attribute when pdl.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, bool pdl, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
// emit: the update kernels' emission mode; kEmitPipe delivers the list of
// step clk[0] + step_off (without advancing the clock).  stdp (spike-buffer
// scheme, FP32 weights; NULL: no plastic synapses): plastic synapses are
// depressed at their arrival and deliver the depressed weight.
cudaError_t launch_deliver(SpikeBuf sb, Csr csr, int wdtype, Ring ring, bool fixed, int emit, int64_t* clk,
                           int64_t step_off, int grid, bool pdl, cudaStream_t st, const StdpArgs* stdp = nullptr);
// STDP potentiation of the plastic inputs of the neurons that fired at step
// clk[1] (after the step's update kernels, before its delivery).
cudaError_t launch_stdp_post(SpikeBuf sb, StdpArgs a, const int64_t* clk, int grid, bool pdl, cudaStream_t st);
// The weight-and-arrival words of a CSR's K synapses: {weights[j], -1}.
cudaError_t init_stdp_words(const float* w, uint64_t K, uint2* wa, cudaStream_t st);
// The CSR weights of the plastic synapses among [first, first + n) from
// their weight-and-arrival words.
cudaError_t sync_stdp_weights(const uint2* wa, const uint32_t* tgt, uint64_t first, uint64_t n, float* w,
                              cudaStream_t st);
// Reverse index of the plastic synapses of a built CSR (N targets, K synapse
// words): in_ptr[N+1] (device, caller-owned) and a new device array of
// rule << 40 | synapse index (caller frees), grouped by target.
cudaError_t build_stdp_index(const uint32_t* tgt, uint64_t K, int64_t N, uint64_t* in_ptr, uint64_t** in_syn_out,
                             uint64_t* n_plastic_out, cudaStream_t st);
// Spike-buffer scheme, serving handles: mark the pending entries of sources
// in [lo, hi) dead (their instance was retired).
cudaError_t launch_kill_pending(uint4* list, const unsigned long long* count, int64_t cap, uint32_t lo, uint32_t hi,
                                cudaStream_t st);
// Initial state of one population: V0 = mean + sd * z (z standard normal from
// the instance's stream, purpose kPurVinit, index = instance-local id).
// LIF (model 0): a = y = V0 - E_L.  AdEx (model 1): a = V0, b = w0, h = h0.
cudaError_t launch_init_state(int model, int64_t n, double mean, double sd, double E_L, double w0, double h0,
                              uint64_t seed, uint32_t local_off, float* a, float* b, float* h, cudaStream_t st);

// Target-tiled delivery (tiled.cu): the synapses of every connection group
// partitioned by target tile (T consecutive neurons), the per-group
// boundary pool, the bucket lists of the due groups and the first bucket
// each tile reads.
struct TiledLayout {
  uint2* pairs = nullptr;             // {target word, weight bits}: groups partitioned by tile, parts padded
  uint32_t* pool = nullptr;           // per group: span, then span + 1 padded part offsets in the group
  uint4* tile_grp = nullptr;          // [G] {pool offset, first tile, first pair lo, hi}
  uint4* bkt = nullptr;               // [2][G] bucket items by step parity
  unsigned long long* boff = nullptr; // [n_tiles + 1] bucket offsets
  unsigned int* bcnt = nullptr;       // [2][n_tiles] bucket fill counts
  uint32_t* lo = nullptr;             // [n_tiles] first bucket read by each tile
  uint32_t n_tiles = 0, T = 0, max_buckets = 0;
  uint64_t pairs_n = 0, bytes = 0;
};

struct TiledArgs {
  const uint2* pairs;
  const uint32_t* pool;
  const uint32_t* lo;
  uint32_t n_tiles, T, P;
  int32_t R;
  int64_t N;
};

// Build the tiled layout of a finalised CSR (group starts grp_start[G+1],
// target words tgt, weights w in precision wdtype) for N neurons and tiles
// of T neurons; fails softly (out->pairs NULL, cudaSuccess) when it would need
// more than max_bytes or the pool exceeds 32-bit offsets.
cudaError_t tiled_build(const uint64_t* grp_start, uint64_t G, const uint32_t* tgt, const void* w, int wdtype,
                        uint64_t K, int64_t N, uint32_t T, uint64_t max_bytes, TiledLayout* out,
                        cudaStream_t st);
void tiled_free(TiledLayout* L);
size_t tiled_smem_bytes(bool fixed, int R, uint32_t T, uint32_t n_tiles);
// Deliver the step's due groups (buckets of parity clk[1] & 1) with P blocks
// per tile; advances the clock as the plain spike-buffer delivery does.
cudaError_t launch_deliver_tiled(SpikeBuf sb, const TiledLayout& L, uint32_t P, int wdtype, Ring ring, int R,
                                 int64_t N, bool fixed, int64_t* clk, bool pdl, cudaStream_t st);

constexpr int kLifBlock = 256;
constexpr int kAeifBlock = 128;
constexpr int kDeliverBlock = 256;

}  // namespace ngb
