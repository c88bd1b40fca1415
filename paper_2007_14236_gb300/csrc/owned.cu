// owned.cu -- target-owned persistent step loop (LIF networks, ring scheme).
//
// One resident block per SM for the whole launch.  Block b of the G blocks
// owns the neurons gid = b, b + G, b + 2G, ... (its tile: T = ceil(N / G)
// neurons, local index gid / G), keeps their state in registers and their
// ring buffer ([L][T] words, Sec. 2.2 ring of slots t + d) in shared memory.
// No kernel boundary and no grid barrier separate the steps: the blocks
// exchange only the step's spikes, through per-block mailboxes whose words
// carry a step stamp, so a word is valid exactly when its stamp is the
// step's.
//
// Synapses grouped by source, then tile: the synapses of source s onto the
// neurons of tile b are the items [G off_s + b C_s, G off_s + b C_s + c_bs)
// of one array, padded to C_s = max_b c_bs items per source (off_s = sum of
// C_s' over the sources before s), so that the G segments of a source lie
// back to back and the segments a spike sends the blocks to are one
// contiguous region rather than G scattered ones; each item
// {local target | delay << 16, FP32 weight} (8 bytes) or, with BF16 or FP16
// weight storage, a tile of at most 1,024 neurons and delays below 64 steps,
// weight bits << 16 | delay << 10 | local target (4 bytes, the storage
// precision kept), or the filler 0xFFFFFFFF (all ones).  The
// tile of a neuron is gid mod G, so every tile holds the same share of every
// population and C_s stays close to the mean per-tile count.  A spike thus
// needs no per-tile index lookup: the firing block publishes (off_s, C_s),
// and every block reads its own C_s items in one round of loads.
//
// The threshold test of a step depends only on the state after the previous
// step (V is propagated with the current of the previous grid point; the
// step's input enters the current), so the spikes of step t + 1 are known
// as soon as step t is updated.  Step t, in every block:
//   items     the first synapse chunks of step t's spike entries (gathered
//             during step t - 1) are loaded; the loads are in flight during
//             the next three phases
//   update    slot t of the tile's ring read and cleared, Poisson drive,
//             exact LIF step (Eqs. 1-2) with the threshold decided a step
//             ago; spike record buffered in shared memory (flushed to the
//             device record with one atomic when it could overflow, and at
//             the end of the launch); event count kept per thread
//   predict   threshold test of step t + 1; entries (off_s, C_s) of the
//             sources that will fire, collected in shared memory, and each
//             such source's item region (its G segments) prefetched into L2,
//             so that the blocks' item loads of step t + 1 find it there
//   publish   the block's mailbox for step t + 1 (buffer (t + 1) mod 4):
//             4 stamped words, 3 entries and the count, further entries in
//             the block's overflow area; then the Poisson counts of t + 1
//             (with one neuron per thread, the first thresholds of its
//             segment and the update's constants held in registers)
//   deliver   the items of step t's spikes added into the shared ring at
//             slot (t + delay) & (L - 1): FP32 atomics, or int64 fixed point
//             (units of 2^-32, as the other loops) in deterministic mode
//   gather    every block's mailbox for step t + 1 polled (one 32-byte load
//             per block; bounded spin) and its entries kept for step t + 1
// A block writes the buffer of step t + 4 only after it has gathered step
// t + 3, which needs every block's step t + 3 mailbox, which each block
// writes only after gathering step t + 2 and so after reading step t: a
// buffer is never overwritten while it is read.  The mailboxes and overflow
// areas are reset before each launch, and a launch runs at most
// kMaxOwnedSteps steps, so a stale word never carries the current stamp.
// Every wait is bounded: a block that gives up sets the timeout flag and the
// abort word, and the others stop at their next poll.
//
// The arithmetic of the update (neuron_step.cuh) and the fixed-point
// conversion are those of the per-step kernels, so deterministic runs are
// bit-identical to every other step loop.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <vector>

#include "builder.h"
#include "neuron_step.cuh"

namespace ngb {

namespace {

constexpr int kOwnedBlock = 512;
constexpr int kMbWords = 4;        // mailbox words per block and step (32 bytes): 3 entries + count
constexpr int kMaxTiles = 256;     // blocks of the launch
constexpr int kPollWords = 4;      // mailbox words polled per thread, in one 32-byte load: G * 8 <= 4 * 512
constexpr int kIdsCap = 2048;      // spike entries gathered per step in shared memory
constexpr int kRecCap = 4096;      // spike-record entries buffered per block (>= 2 x the largest tile)
constexpr uint32_t kFiller = 0xFFFFFFFFu;
constexpr int kStampShift = 48;    // word = stamp << 48 | payload
constexpr uint64_t kPayloadMask = (1ull << kStampShift) - 1;
constexpr int kOffBits = 36;       // entry payload = (C_s / 4) << 36 | off_s

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Four adjacent mailbox words in one 32-byte load (each word is validated by
// its own stamp, so the four need not be read atomically).
__device__ __forceinline__ void ld_relaxed_v4u64(const unsigned long long* p, unsigned long long v[4]) {
  asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3])
               : "l"(p)
               : "memory");
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <bool kFixed>
__device__ __forceinline__ void ring_add(void* ring_s, uint32_t idx, float w) {
  if (kFixed) {
    const long long q = __float2ll_rn(w * 4294967296.0f);
    atomicAdd(reinterpret_cast<unsigned long long*>(ring_s) + idx, (unsigned long long)q);
  } else {
    atomicAdd(reinterpret_cast<float*>(ring_s) + idx, w);
  }
}

// Item formats: kW 0 {local target | delay << 16, FP32 weight} (uint2);
// kW 1 / 2 BF16 / FP16 bits << 16 | delay << 10 | local target (uint32).
template <int kW>
struct OwnedItem {
  using T = typename std::conditional<kW == 0, uint2, uint32_t>::type;
  static __device__ __forceinline__ T filler() {
    if constexpr (kW == 0) return make_uint2(kFiller, 0u);
    else return kFiller;
  }
  static __device__ __forceinline__ bool valid(T x) {
    if constexpr (kW == 0) return x.x != kFiller;
    else return x != kFiller;
  }
  // ring index (slot of step t + delay, local target) and weight
  static __device__ __forceinline__ uint32_t index(T x, int64_t t, const OwnedArgs& a) {
    if constexpr (kW == 0) return ((uint32_t)(t + (x.x >> 16)) & a.L_mask) * a.T + (x.x & 0xFFFFu);
    else return ((uint32_t)(t + ((x >> 10) & 63u)) & a.L_mask) * a.T + (x & 0x3FFu);
  }
  static __device__ __forceinline__ float weight(T x) {
    if constexpr (kW == 0) return __uint_as_float(x.y);
    else if constexpr (kW == 1) return __uint_as_float(x & 0xFFFF0000u);
    else return __half2float(__ushort_as_half((unsigned short)(x >> 16)));
  }
};

template <bool kFixed, int kW>
__device__ __forceinline__ void add_item(typename OwnedItem<kW>::T x, const OwnedArgs& a, int64_t t, void* ring_s) {
  using IT = OwnedItem<kW>;
  if (IT::valid(x)) ring_add<kFixed>(ring_s, IT::index(x, t, a), IT::weight(x));
}

// First item of the segment of tile b of an entry's source.
__device__ __forceinline__ uint64_t seg_first(uint64_t e, uint64_t b) {
  return (e & ((1ull << kOffBits) - 1)) * (uint64_t)gridDim.x + b * ((e >> kOffBits) * 4u);
}

// The whole region of an entry's source (its G segments, back to back) into
// L2 with one bulk prefetch, issued by the block that publishes the spike a
// step before the blocks load their segments of it.  The region starts on a
// 16-byte boundary and spans a multiple of 16 bytes (4-item multiples).
template <int kW>
__device__ __forceinline__ void prefetch_region(uint64_t e, const OwnedArgs& a) {
  using IT = OwnedItem<kW>;
  const char* p = reinterpret_cast<const char*>(reinterpret_cast<const typename IT::T*>(a.items) + seg_first(e, 0));
  const uint64_t bytes = (uint64_t)gridDim.x * ((e >> kOffBits) * 4u) * sizeof(typename IT::T);
  constexpr uint64_t kChunkB = 32768;  // bytes per prefetch instruction
  for (uint64_t o = 0; o < bytes; o += kChunkB) {
    const uint32_t n = (uint32_t)(bytes - o < kChunkB ? bytes - o : kChunkB);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(n) : "memory");
  }
}

// Items of one spike entry (C_s items from seg_first), by the whole warp.
template <bool kFixed, int kW>
__device__ __forceinline__ void deliver_entry_warp(uint64_t e, const OwnedArgs& a, uint64_t tile_base, int64_t t,
                                                   void* ring_s, int lane) {
  using IT = OwnedItem<kW>;
  const uint32_t C = (uint32_t)(e >> kOffBits) * 4u;
  const typename IT::T* it = reinterpret_cast<const typename IT::T*>(a.items) + seg_first(e, tile_base);
  uint32_t k = (uint32_t)lane;
  // two chunks of 32 items in flight per pass
  for (; k < C; k += 64) {
    const typename IT::T x0 = __ldg(it + k);
    const typename IT::T x1 = k + 32 < C ? __ldg(it + k + 32) : IT::filler();
    add_item<kFixed, kW>(x0, a, t, ring_s);
    add_item<kFixed, kW>(x1, a, t, ring_s);
  }
}

// The first two 32-item chunks of an entry (lane's items lane and lane + 32;
// the filler past the entry's width), and the rest of it.
template <int kW>
__device__ __forceinline__ void load_head(uint64_t e, const OwnedArgs& a, uint64_t tile_base, int lane,
                                          typename OwnedItem<kW>::T& x0, typename OwnedItem<kW>::T& x1) {
  using IT = OwnedItem<kW>;
  const uint32_t C = (uint32_t)(e >> kOffBits) * 4u;
  const typename IT::T* it = reinterpret_cast<const typename IT::T*>(a.items) + seg_first(e, tile_base);
  x0 = (uint32_t)lane < C ? __ldg(it + lane) : IT::filler();
  x1 = (uint32_t)lane + 32 < C ? __ldg(it + lane + 32) : IT::filler();
}

template <bool kFixed, int kW>
__device__ __forceinline__ void deliver_entry_tail(uint64_t e, const OwnedArgs& a, uint64_t tile_base, int64_t t,
                                                   void* ring_s, int lane) {
  using IT = OwnedItem<kW>;
  const uint32_t C = (uint32_t)(e >> kOffBits) * 4u;
  const typename IT::T* it = reinterpret_cast<const typename IT::T*>(a.items) + seg_first(e, tile_base);
  for (uint32_t k = 64u + (uint32_t)lane; k < C; k += 32) add_item<kFixed, kW>(__ldg(it + k), a, t, ring_s);
}

// The same by one thread (entries beyond the shared-memory list).
template <bool kFixed, int kW>
__device__ __forceinline__ void deliver_entry_thread(uint64_t e, const OwnedArgs& a, uint64_t tile_base, int64_t t,
                                                     void* ring_s) {
  using IT = OwnedItem<kW>;
  const uint32_t C = (uint32_t)(e >> kOffBits) * 4u;
  const typename IT::T* it = reinterpret_cast<const typename IT::T*>(a.items) + seg_first(e, tile_base);
  for (uint32_t k = 0; k < C; ++k) add_item<kFixed, kW>(__ldg(it + k), a, t, ring_s);
}

}  // namespace

template <bool kFixed, int kNpt, int kW>
__global__ void __launch_bounds__(kOwnedBlock, 1) k_owned(OwnedArgs a) {
  using RW = typename std::conditional<kFixed, long long, float>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  RW* ring_s = reinterpret_cast<RW*>(smem);
  LifSeg* s_seg = reinterpret_cast<LifSeg*>(smem + a.off_seg);
  uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + a.off_thr);
  uint64_t* s_pub = reinterpret_cast<uint64_t*>(smem + a.off_pub);  // [T]
  uint64_t* s_ids = reinterpret_cast<uint64_t*>(smem + a.off_ids);  // [2][kIdsCap], by step parity
  uint2* s_rec = reinterpret_cast<uint2*>(smem + a.off_rec);        // [kRecCap] {neuron, step - t0}
  __shared__ int s_np[2], s_nid[2], s_novm[2];
  __shared__ int s_ovm[2][kMaxTiles];  // mailboxes with overflow (block ids)
  __shared__ int s_abort, s_rn;
  __shared__ unsigned long long s_rbase;

  const int b = (int)blockIdx.x, G = (int)gridDim.x;
  const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kOwnedBlock / 32;
  const uint32_t T = a.T;
  const int64_t N = a.N;
  const uint64_t tile_base = (uint64_t)b;  // the block's tile (seg_first)

  for (int i = tid; i < a.n_seg; i += kOwnedBlock) s_seg[i] = a.seg[i];
  for (uint32_t i = tid; i < a.n_thr; i += kOwnedBlock) s_thr[i] = a.thr[i];
  if (tid == 0) {
    s_np[0] = s_np[1] = 0;
    s_nid[0] = s_nid[1] = 0;
    s_novm[0] = s_novm[1] = 0;
    s_abort = 0;
    s_rn = 0;
  }
  // the tile's ring slots, from the global ring [L][N]
  for (uint32_t slot = 0; slot <= a.L_mask; ++slot)
    for (uint32_t lt = tid; lt < T; lt += kOwnedBlock) {
      const int64_t gid = (int64_t)lt * G + b;
      RW v = (RW)0;
      if (gid < N) v = reinterpret_cast<const RW*>(a.ring)[(uint64_t)slot * (uint64_t)a.ring_N + (uint64_t)gid];
      ring_s[slot * T + lt] = v;
    }
  __syncthreads();

  // the thread's neurons: local index lt = tid + j * 512, gid = lt * G + b
  float y[kNpt], I[kNpt];
  int32_t ref[kNpt];
  int si[kNpt];
  uint64_t pub[kNpt];
  uint32_t outdeg[kNpt], kp[kNpt];
  bool valid[kNpt];
#pragma unroll
  for (int j = 0; j < kNpt; ++j) {
    const uint32_t lt = (uint32_t)(tid + j * kOwnedBlock);
    const int64_t gid = (int64_t)lt * G + b;
    valid[j] = lt < T && gid < N;
    y[j] = I[j] = 0.f;
    ref[j] = 0;
    si[j] = 0;
    pub[j] = 0;
    outdeg[j] = 0;
    kp[j] = 0;
    if (valid[j]) {
      y[j] = a.y[gid];
      I[j] = a.I[gid];
      ref[j] = a.ref[gid];
      pub[j] = a.pub[gid];
      outdeg[j] = (uint32_t)(a.src_syn[gid + 1] - a.src_syn[gid]);
      int lo = 0, hi = a.n_seg;  // segment: the last one whose offset <= gid
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_seg[mid].offset <= gid) lo = mid;
        else hi = mid;
      }
      si[j] = lo;
    }
  }
  const int64_t t0 = a.clk[0];
  // the buffered spike record to the device record (block-wide, after a barrier)
  auto flush_record = [&]() {
    const int n = s_rn;
    if (tid == 0) s_rbase = atomicAdd(a.sb.rec_count, (unsigned long long)n);
    __syncthreads();
    const unsigned long long base = s_rbase;
    if (a.sb.rec_cap > 0)
      for (int i = tid; i < n; i += kOwnedBlock) {
        if (base + (unsigned long long)i < (unsigned long long)a.sb.rec_cap) {
          a.sb.rec_id[base + i] = s_rec[i].x;
          a.sb.rec_step[base + i] = t0 + (int64_t)s_rec[i].y;
        } else {
          atomicOr(a.sb.err, kErrRecordOverflow);
        }
      }
    __syncthreads();
    if (tid == 0) s_rn = 0;
    __syncthreads();
  };
  unsigned long long nev = 0;  // synaptic events of this thread's spikes
  // The Poisson words of four consecutive steps come from one Philox block:
  // each neuron keeps its current block in registers and draws the next one
  // every fourth step.
  U4 pblk[kNpt];
  bool pblk_ok = false;
  // With one neuron per thread, the first kThrReg Poisson thresholds of its
  // segment stay in registers: the count is the number of thresholds at or
  // below the word (they ascend), taken without the chain of dependent
  // shared-memory loads of the search; the search goes on in shared memory
  // only past them.  Thresholds past n_thr read as all ones, and the count is
  // capped at n_thr, so the result is the search's exactly.
  // (and the constants of the update in registers too: a copy of the
  // segment, of which the update reads only the propagators, threshold,
  // reset, refractory steps and drive weight)
  LifSeg sg1 = s_seg[si[0]];
  auto seg_of = [&](int j) -> const LifSeg& {
    if constexpr (kNpt == 1) return sg1;
    else return s_seg[si[j]];
  };
  constexpr int kThrReg = kNpt == 1 ? 8 : 1;
  uint32_t thr_r[kThrReg];
  if (kNpt == 1) {
    const LifSeg& sg = s_seg[si[0]];
#pragma unroll
    for (int i = 0; i < kThrReg; ++i) thr_r[i] = (uint32_t)i < sg.n_thr ? s_thr[sg.thr_off + i] : 0xFFFFFFFFu;
  }
  auto draw_counts = [&](int64_t t) {
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      kp[j] = 0;
      if (!valid[j]) continue;
      const LifSeg& sg = s_seg[si[j]];
      if (sg.n_thr > 0) {
        const int64_t gid = (int64_t)(tid + j * kOwnedBlock) * G + b;
        const int64_t tl = t - sg.t0;
        if (!pblk_ok || (tl & 3) == 0)
          pblk[j] = poisson_block(sg.seed, (uint64_t)tl >> 2, sg.local_off + (uint32_t)(gid - sg.offset));
        const uint32_t x = poisson_word(pblk[j], tl);
        if (kNpt == 1) {
          uint32_t c = 0;
#pragma unroll
          for (int i = 0; i < kThrReg; ++i) c += x >= thr_r[i] ? 1u : 0u;
          uint32_t k = c < sg.n_thr ? c : sg.n_thr;
          if (k == (uint32_t)kThrReg)
            while (k < sg.n_thr && x >= s_thr[sg.thr_off + k]) ++k;
          kp[j] = k;
        } else {
          kp[j] = poisson_from_word(x, s_thr + sg.thr_off, sg.n_thr);
        }
      }
    }
    pblk_ok = true;
  };
  draw_counts(t0);
  const int nwords = G * kMbWords;
  // mailbox buffer and stamp of the spikes of step t0 + r
  auto mb_of = [&](int64_t r) { return a.mb + (size_t)(r & 3) * nwords; };
  auto ovf_of = [&](int64_t r, int m) { return a.ovf + ((size_t)(r & 3) * G + m) * T; };
  // (a launch runs fewer than 4 x 65535 steps, so r >> 2 < 65535: never the
  // all-ones stamp of a reset word)
  auto stamp_of = [](int64_t r) { return (uint64_t)((uint32_t)r >> 2) << kStampShift; };
  // The threshold test of a step depends only on the state after the previous
  // step (lif_propagate), so the spikes of step t + 1 are known once step t is
  // updated: they are published then, and delivered during the next step.
  float yp[kNpt];
  int32_t rp[kNpt];
  bool sp[kNpt];
  auto predict = [&](int q) {  // entries of the spikes of the next step to s_pub, counted in s_np[q]
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      sp[j] = false;
      if (!valid[j]) continue;
      sp[j] = lif_propagate(seg_of(j), y[j], I[j], ref[j], yp[j], rp[j]);
      if (sp[j] && pub[j] != 0) {
        s_pub[atomicAdd(&s_np[q], 1)] = pub[j];
        prefetch_region<kW>(pub[j], a);
      }
    }
  };
  auto publish = [&](int64_t r, int np) {
    const uint64_t st = stamp_of(r);
    if (tid < kMbWords) {
      const uint64_t payload = tid < kMbWords - 1 ? (tid < np ? s_pub[tid] : 0ull) : (uint64_t)np;
      st_relaxed_u64(mb_of(r) + (size_t)b * kMbWords + tid, st | payload);
    }
    for (int k = kMbWords - 1 + tid; k < np; k += kOwnedBlock)
      st_relaxed_u64(ovf_of(r, b) + (k - (kMbWords - 1)), st | s_pub[k]);
  };
  // Entries of the spikes of step t0 + r, from every mailbox, to s_ids[q]
  // (count s_nid[q]); entries beyond the list are delivered at once by the
  // thread that read them.  Returns false when the launch must stop.
  auto gather = [&](int64_t r, int q) -> bool {
    const int64_t tr = t0 + r;
    const uint64_t stamp = stamp_of(r);
    const unsigned long long* mbp = mb_of(r);
    unsigned long long v[kPollWords];
    // one 32-byte load of four words per thread (the address clamped rather
    // than the load predicated, so that nothing consumes the values before
    // they are checked)
    const int nquads = nwords / 4;
    ld_relaxed_v4u64(mbp + 4 * min(tid, nquads - 1), v);
    auto stale = [&]() {
      return (v[0] & ~kPayloadMask) != stamp || (v[1] & ~kPayloadMask) != stamp ||
             (v[2] & ~kPayloadMask) != stamp || (v[3] & ~kPayloadMask) != stamp;
    };
    bool pend = tid < nquads && stale();
    bool gave_up = false;
    unsigned long long spins = 0;
    while (pend) {
      ld_relaxed_v4u64(mbp + 4 * tid, v);
      pend = stale();
      if (!pend) break;
      ++spins;
      if ((spins & 63u) == 0 && (ld_relaxed_u32(a.abort) != 0u || s_abort)) {
        gave_up = true;
        break;
      }
      if (spins > a.spin_limit) {
        atomicOr(a.sb.err, kErrBarrierTimeout);
        atomicExch(a.abort, 1u);
        gave_up = true;
        break;
      }
    }
    if (gave_up) s_abort = 1;
    if (!gave_up) {
#pragma unroll
      for (int i = 0; i < kPollWords; ++i) {
        const int w = 4 * tid + i;
        if (w >= nwords) continue;
        const uint64_t pl = v[i] & kPayloadMask;
        if ((w & (kMbWords - 1)) == kMbWords - 1) {
          if (pl > (uint64_t)(kMbWords - 1)) s_ovm[q][atomicAdd(&s_novm[q], 1)] = w / kMbWords;
        } else if (pl != 0) {
          const int pos = atomicAdd(&s_nid[q], 1);
          if (pos < kIdsCap) s_ids[q * kIdsCap + pos] = pl;
          else deliver_entry_thread<kFixed, kW>(pl, a, tile_base, tr, ring_s);
        }
      }
    }
    __syncthreads();
    if (s_abort) return false;
    if (s_novm[q] > 0) {
      // blocks with more than 3 spikes: their overflow words, a warp per block
      for (int k = warp; k < s_novm[q]; k += kWarps) {
        const int m = s_ovm[q][k];
        const uint64_t cnt = ld_relaxed_u64(mbp + (size_t)m * kMbWords + (kMbWords - 1)) & kPayloadMask;
        const unsigned long long* op = ovf_of(r, m);
        for (uint64_t i = (uint64_t)lane; i + (kMbWords - 1) < cnt; i += 32) {
          unsigned long long x = ld_relaxed_u64(op + i);
          unsigned long long sp2 = 0;
          while ((x & ~kPayloadMask) != stamp) {
            ++sp2;
            if ((sp2 & 63u) == 0 && ld_relaxed_u32(a.abort) != 0u) break;
            if (sp2 > a.spin_limit) {
              atomicOr(a.sb.err, kErrBarrierTimeout);
              atomicExch(a.abort, 1u);
              break;
            }
            x = ld_relaxed_u64(op + i);
          }
          if ((x & ~kPayloadMask) != stamp) {
            s_abort = 1;
            break;
          }
          const uint64_t pl = x & kPayloadMask;
          const int pos = atomicAdd(&s_nid[q], 1);
          if (pos < kIdsCap) s_ids[q * kIdsCap + pos] = pl;
          else deliver_entry_thread<kFixed, kW>(pl, a, tile_base, tr, ring_s);
        }
      }
      __syncthreads();
      if (s_abort) return false;
    }
    return true;
  };
  // the spikes of step t0, published and gathered
  predict(0);
  __syncthreads();
  if (b != a.withhold_block) publish(0, s_np[0]);
  bool aborted = !gather(0, 0);
  for (int64_t r = 0; r < a.steps && !aborted; ++r) {
    const int64_t t = t0 + r;
    const int par = (int)(r & 1);  // s_ids[par]: entries of step r (gathered during the previous step)
    if (tid == 0) {
      s_np[par] = 0;         // published during the previous step; next used by the predictions of step r + 1
      s_nid[par ^ 1] = 0;    // entries of step r + 1, gathered below
      s_novm[par ^ 1] = 0;
    }
    if (s_rn > kRecCap - (int)T) flush_record();  // room for one step's spikes of the tile
    // the first two chunks of the warp's first two entries of step r: the
    // loads are in flight during the update, the publication and the Poisson
    // draws of step t + 1
    const int n = min(s_nid[par], kIdsCap);
    const uint64_t* ids = s_ids + par * kIdsCap;
    const uint64_t e0 = warp < n ? ids[warp] : 0ull;
    const uint64_t e1 = warp + kWarps < n ? ids[warp + kWarps] : 0ull;
    typename OwnedItem<kW>::T x[4];
    load_head<kW>(e0, a, tile_base, lane, x[0], x[1]);
    load_head<kW>(e1, a, tile_base, lane, x[2], x[3]);
    // ------------------------------------------------------------ update
    const uint32_t slot = (uint32_t)t & a.L_mask;
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      if (!valid[j]) continue;
      const uint32_t lt = (uint32_t)(tid + j * kOwnedBlock);
      const LifSeg& sg = seg_of(j);
      float xin;
      if (kFixed) {
        const long long q = ring_s[slot * T + lt];
        xin = __double2float_rn(__dmul_rn(__ll2double_rn(q), 2.3283064365386963e-10));  // x 2^-32
      } else {
        xin = ring_s[slot * T + lt];
      }
      ring_s[slot * T + lt] = (RW)0;
      if (sg.n_thr > 0) xin = __fadd_rn(xin, __fmul_rn((float)kp[j], sg.w_ext));
      lif_apply(sg, y[j], I[j], ref[j], yp[j], rp[j], sp[j], xin);
      if (sp[j]) {
        s_rec[atomicAdd(&s_rn, 1)] = make_uint2((uint32_t)((int64_t)lt * G + b), (uint32_t)r);
        nev += outdeg[j];
      }
    }
    // ------------------------------------------------------------ spikes of step r + 1
    const bool more = r + 1 < a.steps;
    if (more) predict(par ^ 1);
    __syncthreads();  // s_pub complete; slot t read and cleared
    if (more) {
      publish(r + 1, s_np[par ^ 1]);
      draw_counts(t + 1);
    }
    // ------------------------------------------------------------ deliver the spikes of step r
#pragma unroll
    for (int q = 0; q < 4; ++q) add_item<kFixed, kW>(x[q], a, t, ring_s);
    deliver_entry_tail<kFixed, kW>(e0, a, tile_base, t, ring_s, lane);
    deliver_entry_tail<kFixed, kW>(e1, a, tile_base, t, ring_s, lane);
    for (int i = warp + 2 * kWarps; i < n; i += kWarps)
      deliver_entry_warp<kFixed, kW>(ids[i], a, tile_base, t, ring_s, lane);
    // ------------------------------------------------------------ entries of step r + 1
    if (more) {
      if (!gather(r + 1, par ^ 1)) aborted = true;  // ends with a barrier: slot t + 1 complete
    } else {
      __syncthreads();
    }
  }
  if (!aborted) {
    flush_record();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nev += __shfl_xor_sync(0xffffffffu, nev, o);
    if (lane == 0 && nev) atomicAdd(a.sb.events, nev);
#pragma unroll
    for (int j = 0; j < kNpt; ++j) {
      if (!valid[j]) continue;
      const int64_t gid = (int64_t)(tid + j * kOwnedBlock) * G + b;
      a.y[gid] = y[j];
      a.I[gid] = I[j];
      a.ref[gid] = ref[j];
    }
    for (uint32_t slot = 0; slot <= a.L_mask; ++slot)
      for (uint32_t lt = tid; lt < T; lt += kOwnedBlock) {
        const int64_t gid = (int64_t)lt * G + b;
        if (gid < N)
          reinterpret_cast<RW*>(a.ring)[(uint64_t)slot * (uint64_t)a.ring_N + (uint64_t)gid] = ring_s[slot * T + lt];
      }
    if (b == 0 && tid == 0) {
      a.clk[0] = t0 + a.steps;
      a.clk[1] = t0 + a.steps - 1;
    }
  }
}

namespace {

template <int kW>
void* owned_kernel_w(bool fixed, int npt) {
  if (fixed) {
    if (npt == 1) return reinterpret_cast<void*>(&k_owned<true, 1, kW>);
    if (npt == 2) return reinterpret_cast<void*>(&k_owned<true, 2, kW>);
    return reinterpret_cast<void*>(&k_owned<true, 4, kW>);
  }
  if (npt == 1) return reinterpret_cast<void*>(&k_owned<false, 1, kW>);
  if (npt == 2) return reinterpret_cast<void*>(&k_owned<false, 2, kW>);
  return reinterpret_cast<void*>(&k_owned<false, 4, kW>);
}

void* owned_kernel(bool fixed, int npt, int wfmt) {
  if (wfmt == 1) return owned_kernel_w<1>(fixed, npt);
  if (wfmt == 2) return owned_kernel_w<2>(fixed, npt);
  return owned_kernel_w<0>(fixed, npt);
}

// ----------------------------------------------------------------- layout
// Items per (source, tile): one warp per source.
__global__ void k_owned_count(const uint64_t* __restrict__ src_syn, const uint32_t* __restrict__ tgt, int64_t N,
                              int G, uint32_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = w0; s < N; s += nw) {
    const uint64_t lo = src_syn[s], hi = src_syn[s + 1];
    for (uint64_t j = lo + (uint64_t)lane; j < hi; j += 32)
      atomicAdd(cnt + (uint64_t)s * G + ((tgt[j] & kTgtMask) % (uint32_t)G), 1u);
  }
}

// C_s = max over tiles, rounded up to 4; the counts become fill cursors.
__global__ void k_owned_width(int64_t N, int G, uint32_t* cnt, unsigned long long* width) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    uint32_t m = 0;
    for (int b = 0; b < G; ++b) {
      m = max(m, cnt[(uint64_t)s * G + b]);
      cnt[(uint64_t)s * G + b] = 0;
    }
    width[s] = (m + 3u) & ~3u;
  }
}

__global__ void k_owned_pub(int64_t N, const unsigned long long* width, const unsigned long long* off,
                            uint64_t* pub) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x)
    pub[s] = width[s] ? ((width[s] / 4) << kOffBits) | off[s] : 0ull;
}

__device__ __forceinline__ float weight_at(const void* w, int wdtype, uint64_t j) {
  if (wdtype == 1) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w)[j]);
  if (wdtype == 2) return __half2float(reinterpret_cast<const __half*>(w)[j]);
  return reinterpret_cast<const float*>(w)[j];
}

__global__ void k_owned_fill(const uint64_t* __restrict__ src_syn, const uint32_t* __restrict__ src_grp,
                             const uint64_t* __restrict__ grp_start, const uint16_t* __restrict__ grp_delay,
                             const uint32_t* __restrict__ tgt, const void* w, int wdtype, int64_t N, int G,
                             const unsigned long long* __restrict__ off, uint32_t* cursor, void* items,
                             int wfmt) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = w0; s < N; s += nw) {
    for (uint32_t g = src_grp[s]; g < src_grp[s + 1]; ++g) {
      const uint32_t d = grp_delay[g];
      for (uint64_t j = grp_start[g] + (uint64_t)lane; j < grp_start[g + 1]; j += 32) {
        const uint32_t target = tgt[j] & kTgtMask;
        const uint32_t tile = target % (uint32_t)G, lt = target / (uint32_t)G;
        const uint32_t pos = atomicAdd(cursor + (uint64_t)s * G + tile, 1u);
        const uint64_t at = off[s] * (uint64_t)G + (uint64_t)tile * (off[s + 1] - off[s]) + pos;
        if (wfmt == 0) {
          reinterpret_cast<uint2*>(items)[at] = make_uint2(lt | (d << 16), __float_as_uint(weight_at(w, wdtype, j)));
        } else {  // the 16 storage bits of the weight, as stored
          const uint32_t wb = reinterpret_cast<const uint16_t*>(w)[j];
          reinterpret_cast<uint32_t*>(items)[at] = wb << 16 | d << 10 | lt;
        }
      }
    }
  }
}

}  // namespace

cudaError_t owned_build(const Csr& csr, const uint64_t* src_syn, int64_t N, int G, uint32_t L, uint64_t max_bytes,
                        OwnedLayout* out, cudaStream_t st) {
  *out = OwnedLayout{};
  const int64_t T = (N + G - 1) / G;
  const int wfmt = (csr.wdtype == 1 || csr.wdtype == 2) && T <= 1024 && L <= 64 ? csr.wdtype : 0;
  const size_t ib = wfmt ? 4 : 8;
  const uint64_t max_items = max_bytes / ib;
  uint32_t* cnt = nullptr;
  unsigned long long *width = nullptr, *off = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  uint64_t S = 0;
  const int grid = 1024;
  cudaError_t e = cudaMalloc(&cnt, (size_t)N * G * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&width, (size_t)(N + 1) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&off, (size_t)(N + 1) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&out->pub, (size_t)N * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)N * G * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(width + N, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    k_owned_count<<<grid, 256, 0, st>>>(src_syn, csr.tgt, N, G, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_owned_width<<<grid, 256, 0, st>>>(N, G, cnt, width);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_scratch_bytes_u64((uint64_t)N + 1, &tmp_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 1);
  if (e == cudaSuccess) e = exclusive_scan_u64(width, off, (uint64_t)N + 1, tmp, tmp_bytes, st);
  unsigned long long wmax = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&S, off + N, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // widest source (the entry holds C_s / 4 in 12 bits)
  if (e == cudaSuccess && N > 0) {
    std::vector<unsigned long long> wv((size_t)N);
    e = cudaMemcpy(wv.data(), width, (size_t)N * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    for (unsigned long long x : wv) wmax = x > wmax ? x : wmax;
  }
  bool fits = e == cudaSuccess && wmax / 4 < (1ull << (kStampShift - kOffBits)) && S < (1ull << kOffBits) &&
              (uint64_t)G * S <= max_items;
  if (fits) {
    e = cudaMalloc(&out->items, (size_t)((uint64_t)G * S > 0 ? (uint64_t)G * S : 1) * ib);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      fits = false;
      e = cudaSuccess;
    }
  }
  if (fits && e == cudaSuccess) e = cudaMemsetAsync(out->items, 0xFF, (size_t)G * S * ib, st);
  if (fits && e == cudaSuccess) {
    k_owned_pub<<<grid, 256, 0, st>>>(N, width, off, out->pub);
    e = cudaGetLastError();
  }
  if (fits && e == cudaSuccess) {
    k_owned_fill<<<grid, 256, 0, st>>>(src_syn, csr.src_grp, csr.grp_start, csr.grp_delay, csr.tgt, csr.w,
                                       csr.wdtype, N, G, off, cnt, out->items, wfmt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(cnt);
  cudaFree(width);
  cudaFree(off);
  cudaFree(tmp);
  if (e != cudaSuccess || !fits) {
    cudaFree(out->pub);
    cudaFree(out->items);
    *out = OwnedLayout{};
    return e;
  }
  out->S = S;
  out->G = G;
  out->max_width = (uint32_t)wmax;
  out->wfmt = wfmt;
  return cudaSuccess;
}

size_t owned_smem_bytes(bool fixed, uint32_t L, uint32_t T, int n_seg, uint32_t n_thr) {
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  return a16((size_t)L * T * (fixed ? 8 : 4)) + a16((size_t)n_seg * sizeof(LifSeg)) + a16((size_t)n_thr * 4) +
         a16((size_t)T * 8) + (size_t)2 * kIdsCap * 8 + (size_t)kRecCap * 8;
}

cudaError_t launch_owned(OwnedArgs a, bool fixed, int grid, cudaStream_t st) {
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  a.off_seg = (uint32_t)a16((size_t)(a.L_mask + 1) * a.T * (fixed ? 8 : 4));
  a.off_thr = a.off_seg + (uint32_t)a16((size_t)a.n_seg * sizeof(LifSeg));
  a.off_pub = a.off_thr + (uint32_t)a16((size_t)a.n_thr * 4);
  a.off_ids = a.off_pub + (uint32_t)a16((size_t)a.T * 8);
  a.off_rec = a.off_ids + (uint32_t)(2 * kIdsCap * 8);
  const size_t smem = a.off_rec + (size_t)kRecCap * 8;
  const int npt = a.T <= kOwnedBlock ? 1 : (a.T <= 2 * kOwnedBlock ? 2 : 4);
  if (a.T > 4 * kOwnedBlock || grid > kMaxTiles || grid * kMbWords > kPollWords * kOwnedBlock ||
      a.steps > kMaxOwnedSteps)
    return cudaErrorInvalidValue;
  void* k = owned_kernel(fixed, npt, a.wfmt);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kOwnedBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  return cudaLaunchKernelExC(&cfg, k, args);
}

cudaError_t owned_max_blocks_per_sm(bool fixed, uint32_t T, size_t smem, int wfmt, int* out) {
  const int npt = T <= kOwnedBlock ? 1 : (T <= 2 * kOwnedBlock ? 2 : 4);
  void* k = owned_kernel(fixed, npt, wfmt);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, kOwnedBlock, smem);
}

}  // namespace ngb
