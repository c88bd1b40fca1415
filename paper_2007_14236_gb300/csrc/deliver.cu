// deliver.cu -- spike delivery kernel (K3).
//
// Sec. 2.2 of the paper: every spike of step t reaches each target of the
// source's connection groups after the group's delay.  Here the spikes of step
// t (compacted by the update kernels) are scattered into the targets' input
// ring buffer at slot (t + d) & (L - 1), one atomic add per synapse.
//
// Work decomposition (load-balanced, synapse-parallel): every spiking source
// contributes ceil((end - align4(begin)) / 128) work items of 128 consecutive
// synapses, aligned to 16 bytes.  The compaction in the update kernels wrote
// one 32-byte entry per work item (source, index within the source, row and
// group range), so a warp reads its work item with one load.  Each lane
// loads 4 target words (one 16-byte load) and 4 weights (16 or 8 bytes); the
// warp holds the source's delay groups (up to 64) in registers, two per lane,
// and finds each synapse's group with ballots over the group starts; then one
// red.global.add per synapse: FP32 (or int64 fixed point in deterministic
// mode).  Per work item the warp waits on two dependent memory round trips
// (work-item entry, then synapses + groups).
//
// Bytes: 8 (FP32) or 6 (BF16/FP16) per synapse read, one 4-byte (8-byte)
// L2 atomic per synapse, plus 32 bytes of work-item entry and 10 bytes per
// delay group of the source per work item.
//
// Pipelined ring scheme (kEmitPipe): the list of step t = clk[0] + step_off
// (by t mod 3) holds the work items of the spikes' groups with delay >= 2,
// delivered beside the update of step t + 1; the clock is not advanced here
// and the list of step t + 2 is emptied (its last reader, the delivery of
// step t - 1, ran before this one).
//
// Spike-buffer scheme (kEmitAge): the step's list holds due items (one uint4 per
// <= 1024 synapses of one connection group, written by the update kernel's
// pending-spike scan); every synapse goes to the single ring slot, the
// input of step t + 1.  The kernel also empties the pending list that the
// step's update kernel has consumed.  With plastic synapses (kPlastic) each
// one is depressed at its arrival before it delivers (nearest-neighbour
// STDP, Sec. 2.1; stdp.cu has the potentiation).
#include "deliver_item.cuh"
#include "ngb_internal.cuh"

namespace ngb {

template <typename WT, bool kFixed, int kMode, bool kPlastic = false>
__global__ void __launch_bounds__(kDeliverBlock) k_deliver(SpikeBuf sb, Csr csr, Ring ring, int64_t* clk,
                                                           int64_t step_off, StdpArgs sa) {
  constexpr bool kAge = kMode == kEmitAge;
  griddep_wait();    // the step's update kernels have completed
  griddep_launch();  // the next step's update may start its prologue
  const uint32_t warp = (blockIdx.x * (uint32_t)kDeliverBlock + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * (uint32_t)kDeliverBlock) >> 5;
  const int lane = threadIdx.x & 31;
  if (kMode == kEmitPipe) {
    const int64_t tp = clk[0] + step_off;
    const int q = (int)(tp % 3);
    const uint32_t n = (uint32_t)(sb.ctr3[q] & kChunkMask);
    if (blockIdx.x == 0 && threadIdx.x == 0) sb.ctr3[(int)((tp + 2) % 3)] = 0;
    const uint4* __restrict__ wq = sb.wi3[q];
    for (uint32_t ch = warp; ch < n; ch += nwarps)
      deliver_work_item<WT, kFixed>(wq[2 * (uint64_t)ch], wq[2 * (uint64_t)ch + 1], tp, csr, ring, lane);
    return;
  }
  // both parities' counters are read together with the step counter (one round trip)
  const unsigned long long c0 = sb.ctr[0], c1 = sb.ctr[1];
  const int64_t t = clk[1];
  const int buf = (int)(t & 1);
  const unsigned long long c = buf ? c1 : c0;
  uint32_t nch = (uint32_t)(c & kChunkMask);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = t + 1;        // next step for the update kernels
    sb.ctr[buf ^ 1] = 0;   // the next step's list starts empty
    if (kAge) sb.pcnt[buf] = 0;  // consumed by this step's scan; refilled by step t + 1's
  }
  const uint4* __restrict__ wi = buf ? sb.wi[1] : sb.wi[0];
  if (kAge) {
    if ((unsigned long long)nch > (unsigned long long)sb.wi_cap) nch = (uint32_t)sb.wi_cap;
    for (uint32_t it = warp; it < nch; it += nwarps)
      deliver_due_item<WT, kFixed, kPlastic>(wi[it], csr, ring, lane, t, &sb, &sa);
    return;
  }
  for (uint32_t ch = warp; ch < nch; ch += nwarps) {
    const uint4 a = wi[2 * (uint64_t)ch], m2 = wi[2 * (uint64_t)ch + 1];
    deliver_work_item<WT, kFixed>(a, m2, t, csr, ring, lane);
  }
}

namespace {
template <typename WT, bool kFixed>
cudaError_t launch_deliver_t(SpikeBuf sb, Csr csr, Ring ring, int emit, int64_t* clk, int64_t step_off, int grid,
                             bool pdl, cudaStream_t st) {
  const dim3 g((unsigned)grid), b(kDeliverBlock);
  const StdpArgs none{};
  if (emit == kEmitAge)
    return launch_k(k_deliver<WT, kFixed, kEmitAge>, g, b, pdl, st, sb, csr, ring, clk, step_off, none);
  if (emit == kEmitPipe)
    return launch_k(k_deliver<WT, kFixed, kEmitPipe>, g, b, pdl, st, sb, csr, ring, clk, step_off, none);
  return launch_k(k_deliver<WT, kFixed, kEmitRing>, g, b, pdl, st, sb, csr, ring, clk, step_off, none);
}
}  // namespace

cudaError_t launch_deliver(SpikeBuf sb, Csr csr, int wdtype, Ring ring, bool fixed, int emit, int64_t* clk,
                           int64_t step_off, int grid, bool pdl, cudaStream_t st, const StdpArgs* stdp) {
  if (stdp) {  // plastic synapses: FP32 weights, spike-buffer scheme
    if (wdtype != 0 || emit != kEmitAge) return cudaErrorInvalidValue;
    const dim3 g((unsigned)grid), b(kDeliverBlock);
    if (fixed)
      return launch_k(k_deliver<float, true, kEmitAge, true>, g, b, pdl, st, sb, csr, ring, clk, step_off, *stdp);
    return launch_k(k_deliver<float, false, kEmitAge, true>, g, b, pdl, st, sb, csr, ring, clk, step_off, *stdp);
  }
#define NGB_DEL(T, F) return launch_deliver_t<T, F>(sb, csr, ring, emit, clk, step_off, grid, pdl, st)
  if (fixed) {
    if (wdtype == 0) NGB_DEL(float, true);
    if (wdtype == 1) NGB_DEL(__nv_bfloat16, true);
    NGB_DEL(__half, true);
  }
  if (wdtype == 0) NGB_DEL(float, false);
  if (wdtype == 1) NGB_DEL(__nv_bfloat16, false);
  NGB_DEL(__half, false);
#undef NGB_DEL
}

// ------------------------------------------------------------------ retirement
__global__ void k_kill_pending(uint4* list, const unsigned long long* count, int64_t cap, uint32_t lo, uint32_t hi) {
  unsigned long long n = *count;
  if (n > (unsigned long long)cap) n = (unsigned long long)cap;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t w = list[i].x;
    if (w == kDeadWord) continue;
    const uint32_t gid = w & kIdMask;
    if (gid >= lo && gid < hi) list[i].x = kDeadWord;
  }
}

cudaError_t launch_kill_pending(uint4* list, const unsigned long long* count, int64_t cap, uint32_t lo, uint32_t hi,
                                cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  k_kill_pending<<<64, 256, 0, st>>>(list, count, cap, lo, hi);
  return cudaGetLastError();
}

}  // namespace ngb
