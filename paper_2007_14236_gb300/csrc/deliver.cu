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
// Spike-buffer scheme (kAge): the step's list holds due items (one uint4 per
// <= 1024 synapses of one connection group, written by the update kernel's
// pending-spike scan); every synapse goes to the single ring slot, the
// input of step t + 1.  The kernel also empties the pending list that the
// step's update kernel has consumed.
#include "deliver_item.cuh"
#include "ngb_internal.cuh"

namespace ngb {

template <typename WT, bool kFixed, bool kAge>
__global__ void __launch_bounds__(kDeliverBlock) k_deliver(SpikeBuf sb, Csr csr, Ring ring, int64_t* clk) {
  griddep_wait();    // the step's update kernels have completed
  griddep_launch();  // the next step's update may start its prologue
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
    if (sb.dcnt) {               // the step's deferred AdEx neurons are all finished
      sb.dcnt[0] = 0;
      sb.dcnt[1] = 0;
    }
  }
  const uint4* __restrict__ wi = buf ? sb.wi[1] : sb.wi[0];
  const uint32_t warp = (blockIdx.x * (uint32_t)kDeliverBlock + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * (uint32_t)kDeliverBlock) >> 5;
  const int lane = threadIdx.x & 31;
  if (kAge) {
    if ((unsigned long long)nch > (unsigned long long)sb.wi_cap) nch = (uint32_t)sb.wi_cap;
    for (uint32_t it = warp; it < nch; it += nwarps) deliver_due_item<WT, kFixed>(wi[it], csr, ring, lane);
    return;
  }
  for (uint32_t ch = warp; ch < nch; ch += nwarps) {
    const uint4 a = wi[2 * (uint64_t)ch], m2 = wi[2 * (uint64_t)ch + 1];
    deliver_work_item<WT, kFixed>(a, m2, t, csr, ring, lane);
  }
}

namespace {
template <typename WT, bool kFixed>
cudaError_t launch_deliver_t(SpikeBuf sb, Csr csr, Ring ring, bool age, int64_t* clk, int grid, bool pdl,
                             cudaStream_t st) {
  const dim3 g((unsigned)grid), b(kDeliverBlock);
  if (age) return launch_k(k_deliver<WT, kFixed, true>, g, b, pdl, st, sb, csr, ring, clk);
  return launch_k(k_deliver<WT, kFixed, false>, g, b, pdl, st, sb, csr, ring, clk);
}
}  // namespace

cudaError_t launch_deliver(SpikeBuf sb, Csr csr, int wdtype, Ring ring, bool fixed, bool age, int64_t* clk,
                           int grid, bool pdl, cudaStream_t st) {
  if (fixed) {
    if (wdtype == 0) return launch_deliver_t<float, true>(sb, csr, ring, age, clk, grid, pdl, st);
    if (wdtype == 1) return launch_deliver_t<__nv_bfloat16, true>(sb, csr, ring, age, clk, grid, pdl, st);
    return launch_deliver_t<__half, true>(sb, csr, ring, age, clk, grid, pdl, st);
  }
  if (wdtype == 0) return launch_deliver_t<float, false>(sb, csr, ring, age, clk, grid, pdl, st);
  if (wdtype == 1) return launch_deliver_t<__nv_bfloat16, false>(sb, csr, ring, age, clk, grid, pdl, st);
  return launch_deliver_t<__half, false>(sb, csr, ring, age, clk, grid, pdl, st);
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
