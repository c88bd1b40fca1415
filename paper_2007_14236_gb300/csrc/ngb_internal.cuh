// ngb_internal.cuh -- device data layout and helpers shared by the library's
// translation units (not part of the C ABI).
//
// Data layout in HBM (N neurons, K synapses, G connection groups, L ring
// slots, R receptors):
//   state      SoA FP32 arrays of N (LIF: y = V - E_L, I, refractory counter;
//              AdEx: V, w, g_ex, g_in, h)
//   ring       [L][R][N] FP32 (or int64 fixed point in deterministic mode);
//              slot (t + d) & (L - 1) receives the spikes of step t with delay d
//   CSR        src_syn[N+1] u64 (first synapse of each source),
//              src_grp[N+1] u32 (first delay group of each source),
//              grp_start[G+1] u64 and grp_delay[G] u16 (Sec. 2.2 connection
//              groups: a source's synapses with equal delay, in delay order),
//              tgt[K] u32 (bit 31 = receptor, bits 0-30 = global target),
//              w[K] FP32 / BF16 / FP16
//   src_meta   uint4 per source {row start lo, row start hi (16 bits) | groups
//              << 16, synapses, first group}: everything delivery needs about
//              a spiking source, read once by the update kernel
//   work items per step (double-buffered by step parity): 2 x uint4 per
//              work item of 128 synapses ({neuron | multiplicity << 26, index
//              of the item within its source, meta.x, meta.y}, {meta.z,
//              meta.w, 0, 0}) and one packed u64 counter (spikes << 38 |
//              work items); capacity = the work items of all sources
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
constexpr uint32_t kRcptBit = 0x80000000u;

// error flags (device word)
constexpr uint32_t kErrRecordOverflow = 1u;
constexpr uint32_t kErrSubstepCap = 2u;
constexpr uint32_t kErrBarrierTimeout = 4u;

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
  int32_t pad2_;
  float g_L, E_L, V_T, Delta_T, inv_Delta_T, a, inv_tau_w, V_peak, V_reset, b;
  float E_ex, E_in, inv_tau_ex, inv_tau_in, I_e, inv_C, w_ext, pad_;
  double inv_tol, h_min, dt;
  int64_t max_sub;
};

struct SpikeBuf {
  uint4* wi[2];                     // 2 entries per delivery work item
  unsigned long long* ctr;          // [2] packed per-step counters
  unsigned long long* events;       // synaptic events delivered (cumulative)
  unsigned long long* substeps;     // RK sub-steps (cumulative)
  uint32_t* rec_id;                 // spike record, rec_cap entries
  int64_t* rec_step;
  unsigned long long* rec_count;    // spikes since the last drain (with multiplicity)
  int64_t rec_cap;
  uint32_t* err;
};

struct Csr {
  const uint4* src_meta;
  const uint64_t* src_syn;
  const uint32_t* src_grp;
  const uint64_t* grp_start;
  const uint16_t* grp_delay;
  const uint32_t* tgt;
  const void* w;
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
  float *st0, *st1, *st2, *st3, *st4;
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
  uint32_t off_aseg, off_lvoff, off_avoff, off_thr;  // dynamic shared memory layout
};

// ------------------------------------------------------------------ host side
// Kernel launchers (one translation unit each).
cudaError_t launch_update_lif(const SegTable<LifSeg>& segs, int64_t blocks, const uint32_t* thr, float* y,
                              float* I, int32_t* ref, Ring ring, bool fixed, int64_t* clk, const uint4* src_meta,
                              SpikeBuf sb, bool pdl, cudaStream_t st);
cudaError_t launch_update_aeif(const SegTable<AeifSeg>& segs, int64_t blocks, const uint32_t* thr, float* V,
                               float* w, float* gex, float* gin, float* h, Ring ring, bool fixed, int64_t* clk,
                               const uint4* src_meta, SpikeBuf sb, bool pdl, cudaStream_t st);
cudaError_t launch_tick(int64_t* clk, bool pdl, cudaStream_t st);
cudaError_t persistent_max_blocks_per_sm(bool fixed, int wdtype, bool lif, bool aeif, size_t smem, int* out);
cudaError_t launch_persistent(const PersistArgs& a, bool fixed, int wdtype, bool lif, bool aeif, int grid,
                              size_t smem, cudaStream_t st);

// Per-source metadata for the update kernels' spike lists; *total_items
// (device) receives the delivery work items of all sources together.
cudaError_t launch_build_meta(int64_t N, const uint64_t* src_syn, const uint32_t* src_grp, uint4* meta,
                              unsigned long long* total_items, cudaStream_t st);

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
cudaError_t launch_deliver(SpikeBuf sb, Csr csr, int wdtype, Ring ring, bool fixed, int64_t* clk, int grid,
                           bool pdl, cudaStream_t st);
// Initial state of one population: V0 = mean + sd * z (z standard normal from
// the instance's stream, purpose kPurVinit, index = instance-local id).
// LIF (model 0): a = y = V0 - E_L.  AdEx (model 1): a = V0, b = w0, h = h0.
cudaError_t launch_init_state(int model, int64_t n, double mean, double sd, double E_L, double w0, double h0,
                              uint64_t seed, uint32_t local_off, float* a, float* b, float* h, cudaStream_t st);

constexpr int kLifBlock = 256;
constexpr int kAeifBlock = 128;
constexpr int kDeliverBlock = 256;

}  // namespace ngb
