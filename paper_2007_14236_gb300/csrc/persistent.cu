// persistent.cu -- persistent step kernel: many simulation steps per launch.
//
// The per-step path launches three kernels per step (update LIF, update
// AdEx, deliver); at small networks (the microcircuit delivers ~1e5 synaptic
// events per step) the launch, drain and the dependent reads of the step
// counter dominate.  Here one cooperative launch runs `steps` steps:
//
//   for each step t:
//     update phase   every warp takes 32 consecutive neurons (grid-stride):
//                    ring slot t read (through L2) and zeroed, Poisson drive,
//                    exact LIF step or adaptive RK45 AdEx step, warp-ballot
//                    compaction into the work-item list of step t
//     grid barrier   the list of step t is complete
//     delivery phase every warp takes work items (grid-stride) and scatters
//                    them into ring slots t + d (as the per-step kernel)
//     grid barrier   slot t + 1 is complete
//
// In the spike-buffer delivery scheme (a.age) the update phase first moves
// the pending spikes whose next group is due to the step's due-item list, new
// spikes join that list or the pending list, and the delivery phase scatters
// the due items into the single ring slot.
//
// Pipelined variant (kPipe, ring scheme): one grid barrier per step.  The
// update phase of step t also delivers each new spike's delay-1 group into
// slot t + 1 and queues its other groups (list t mod 3); in the same phase the
// warps deliver the queue of step t - 1, whose groups land in slots t + 1 and
// later, so nothing written in the phase is read in it (slot t, read and
// cleared by the update, receives no write after the barrier that ends step
// t - 1).  After the last step the launch delivers that step's queue, so no
// queued work crosses a launch boundary; the host zeroes the queue counters
// before each launch.  The barrier is a monotonic arrival
// counter (zeroed before each launch) polled until it reaches the number of
// arrivals of the barrier: one atomic per block and no reset round trip.
//
// The step counter lives in registers.  The arithmetic is the same device
// code as the per-step kernels (neuron_step.cuh, aeif_rk.cuh,
// deliver_item.cuh), so both paths give identical results.  Data written by
// other SMs inside the launch (ring slots, work items, counters) is read with
// L1-bypassing loads.
//
// The grid barrier is an arrival counter plus a generation word in global
// memory.  Every wait is bounded: after `spin_limit` polls a block sets the
// timeout error flag and the abort word, and every block leaves the step loop
// at its next barrier, so the launch always ends.  The launch is cooperative,
// which guarantees that all blocks are resident.
#include "aeif_rk.cuh"
#include "deliver_item.cuh"
#include "neuron_step.cuh"

namespace ngb {

namespace {

constexpr int kPersistBlock = 256;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier with a bounded wait.  Returns false when the launch must
// stop (this block or another one gave up waiting).  withhold: this block does
// not arrive (test hook for the timeout path).
//
// The block's threads meet at __syncthreads; thread 0 then arrives with an
// acquire-release atomic on the arrival counter (making the block's writes,
// ordered before it by the CTA barrier, visible at GPU scope).  The last
// arriver resets the counter and publishes the next generation with a
// release store; the others poll the generation with acquire loads.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned long long spin_limit, uint32_t* err,
                                          bool withhold) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_u32(bar + 1);
    bool released = false;
    if (!withhold) {
      if (atom_add_acq_rel_u32(bar, 1u) == gridDim.x - 1) {
        st_relaxed_u32(bar, 0u);
        st_release_u32(bar + 1, gen + 1u);  // new generation: everyone may go
        released = true;
      }
    }
    if (!released) {
      unsigned long long spins = 0;
      while (ld_acquire_u32(bar + 1) == gen) {
        if ((spins & 63u) == 63u && ld_acquire_u32(bar + 2) != 0u) {  // another block gave up
          ok = 0;
          break;
        }
        if (++spins > spin_limit) {
          atomicOr(err, kErrBarrierTimeout);
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Grid barrier `k` (0, 1, ...) of the launch on a monotonic arrival counter:
// each block arrives with a release reduction and waits (bounded, acquire
// polls) until all gridDim.x * (k + 1) arrivals are in.  Returns false when the
// launch must stop (this block or another gave up).
__device__ __forceinline__ void red_add_release_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync_mono(unsigned* bar, unsigned k, unsigned long long spin_limit,
                                               uint32_t* err, bool withhold) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (!withhold) red_add_release_u32(bar, 1u);
    const unsigned target = gridDim.x * (k + 1u);
    unsigned long long spins = 0;
    while (ld_acquire_u32(bar) < target) {
      if ((spins & 63u) == 63u && ld_acquire_u32(bar + 2) != 0u) {  // another block gave up
        ok = 0;
        break;
      }
      if (++spins > spin_limit) {
        atomicOr(err, kErrBarrierTimeout);
        atomicExch(bar + 2, 1u);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename Seg>
__device__ __forceinline__ int seg_of(const int64_t* voff, int n, int64_t v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (voff[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace

template <bool kFixed, typename WT, bool kLif, bool kAeif, bool kPipe>
__global__ void __launch_bounds__(kPersistBlock) k_persistent(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  LifSeg* s_lseg = reinterpret_cast<LifSeg*>(smem);
  AeifSeg* s_aseg = reinterpret_cast<AeifSeg*>(smem + a.off_aseg);
  int64_t* s_lvoff = reinterpret_cast<int64_t*>(smem + a.off_lvoff);
  int64_t* s_avoff = reinterpret_cast<int64_t*>(smem + a.off_avoff);
  uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + a.off_thr);
  for (int i = threadIdx.x; i < a.n_lseg; i += kPersistBlock) s_lseg[i] = a.lseg[i];
  for (int i = threadIdx.x; i < a.n_aseg; i += kPersistBlock) s_aseg[i] = a.aseg[i];
  for (int i = threadIdx.x; i <= a.n_lseg; i += kPersistBlock) s_lvoff[i] = a.lvoff[i];
  for (int i = threadIdx.x; i <= a.n_aseg; i += kPersistBlock) s_avoff[i] = a.avoff[i];
  for (uint32_t i = threadIdx.x; i < a.n_thr; i += kPersistBlock) s_thr[i] = a.thr[i];
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kPersistBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kPersistBlock) >> 5;
  // pipelined variant: the last quarter of the warps delivers the previous
  // step's queue while the others update, so the two overlap within a phase
  const int64_t dwarps = kPipe ? (nwarps / 4 > 0 ? nwarps / 4 : 1) : 0;
  const int64_t uwarps = kPipe && nwarps > 1 ? nwarps - dwarps : nwarps;
  const bool updater = warp < uwarps;
  const Ring ring = a.ring;
  const uint64_t plane = (uint64_t)ring.R * (uint64_t)ring.N;
  int64_t t = a.clk[0];
  const int64_t t_first = t;  // clk[0] is rewritten by block 0 at the end of the launch
  unsigned long long nsub = 0;
  bool cap_hit = false;
  bool first_barrier = true;
  for (int64_t step = 0; step < a.steps; ++step) {
    const uint64_t slot = (uint64_t)(t & ring.L_mask);
    // ------------------------------------------------------------ update phase
    if (kPipe && blockIdx.x == 0 && threadIdx.x == 0) a.sb.ctr3[(int)((t + 1) % 3)] = 0;  // consumed in phase t - 1
    if (!kPipe && a.age) scan_pending<true>(t, a.csr, a.sb, warp, nwarps);
    if (kLif && updater) {
      for (int64_t vb = warp * 32; vb < a.n_lif; vb += uwarps * 32) {
        const int64_t v = vb + lane;
        const bool valid = v < a.n_lif;
        const int si = valid ? seg_of<LifSeg>(s_lvoff, a.n_lseg, v) : 0;
        const LifSeg& sg = s_lseg[si];
        const int64_t k = v - s_lvoff[si];
        const uint32_t gid = (uint32_t)(sg.offset + k);
        bool spk = false;
        uint4 meta = make_uint4(0, 0, 0, 0);
        if (valid) {
          float y = a.st0[gid], I = a.st1[gid];
          int32_t ref = a.ref[gid];
          if (!a.age) meta = __ldg(a.src_meta + gid);
          float in = ring_take<kFixed, true>(ring.p, slot * plane + gid);
          if (sg.n_thr > 0) {
            const uint32_t kp = poisson_count(sg.seed, t - sg.t0, sg.local_off + (uint32_t)k, s_thr + sg.thr_off,
                                              sg.n_thr);
            in = __fadd_rn(in, __fmul_rn((float)kp, sg.w_ext));
          }
          spk = lif_step(sg, y, I, ref, in);
          a.st0[gid] = y;
          a.st1[gid] = I;
          a.ref[gid] = ref;
        }
        if (kPipe)
          emit_spikes_pipe<kFixed>(spk, gid, 1u, t, meta, spk ? __ldg(a.csr.src_age + gid) : make_uint2(0, 0), a.csr,
                                   ring, a.sb);
        else if (a.age) emit_spikes_age(spk, gid, 1u, t, a.csr, a.sb);
        else emit_spikes(spk, gid, 1u, t, meta, a.sb);
      }
    }
    if (kAeif && updater) {
      for (int64_t vb = warp * 32; vb < a.n_aeif; vb += uwarps * 32) {
        const int64_t v = vb + lane;
        const bool valid = v < a.n_aeif;
        const int si = valid ? seg_of<AeifSeg>(s_avoff, a.n_aseg, v) : 0;
        const AeifSeg& p = s_aseg[si];
        const int64_t k = v - s_avoff[si];
        const uint32_t gid = (uint32_t)(p.offset + k);
        uint32_t nspk = 0;
        uint4 meta = make_uint4(0, 0, 0, 0);
        if (valid) {
          St y{a.st0[gid], a.st1[gid], a.st2[gid], a.st3[gid], 0.f, 0.f};
          if (p.alpha) {
            y.xe = a.st5[gid];
            y.xi = a.st6[gid];
          }
          double h = (double)a.st4[gid];
          if (!a.age) meta = __ldg(a.src_meta + gid);
          const uint64_t i0 = slot * plane + gid;
          float in0 = ring_take<kFixed, true>(ring.p, i0);
          float in1 = ring_take<kFixed, true>(ring.p, i0 + (uint64_t)ring.N);
          if (p.n_thr > 0) {
            const uint32_t kp = poisson_count(p.seed, t - p.t0, p.local_off + (uint32_t)k, s_thr + p.thr_off,
                                              p.n_thr);
            const float add = __fmul_rn((float)kp, p.w_ext);
            if (p.prec_rcpt == 0) in0 = __fadd_rn(in0, add);
            else in1 = __fadd_rn(in1, add);
          }
          if (p.alpha) aeif_step<kAeifAlpha>(p, y, h, in0, in1, nspk, nsub, cap_hit);
          else aeif_step<kAeifExp>(p, y, h, in0, in1, nspk, nsub, cap_hit);
          a.st0[gid] = y.V;
          a.st1[gid] = y.w;
          a.st2[gid] = y.ge;
          a.st3[gid] = y.gi;
          if (p.alpha) {
            a.st5[gid] = y.xe;
            a.st6[gid] = y.xi;
          }
          a.st4[gid] = (float)h;
        }
        const uint32_t mult = nspk > 63u ? 63u : nspk;
        if (kPipe)
          emit_spikes_pipe<kFixed>(nspk > 0, gid, mult, t, meta,
                                   nspk > 0 ? __ldg(a.csr.src_age + gid) : make_uint2(0, 0), a.csr, ring, a.sb);
        else if (a.age) emit_spikes_age(nspk > 0, gid, mult, t, a.csr, a.sb);
        else emit_spikes(nspk > 0, gid, mult, t, meta, a.sb);
      }
    }
    if (kPipe) {
      // the queue of step t - 1 (groups with delay >= 2: slots t + 1 and later)
      if (step > 0) {
        const int q = (int)((t - 1) % 3);
        const uint32_t n = (uint32_t)(__ldcg(a.sb.ctr3 + q) & kChunkMask);
        const uint4* wq = a.sb.wi3[q];
        const int64_t w0 = uwarps < nwarps ? warp - uwarps : warp;  // a one-warp grid does both
        if (w0 >= 0)
          for (int64_t ch = w0; ch < (int64_t)n; ch += (uwarps < nwarps ? dwarps : nwarps))
            deliver_work_item<WT, kFixed>(__ldcg(wq + 2 * ch), __ldcg(wq + 2 * ch + 1), t - 1, a.csr, ring, lane);
      }
      if (!grid_sync_mono(a.bar, (unsigned)step, a.spin_limit, a.sb.err,
                          first_barrier && (int)blockIdx.x == a.withhold_block))
        break;
      first_barrier = false;
      ++t;
      continue;
    }
    if (!grid_sync(a.bar, a.spin_limit, a.sb.err, first_barrier && (int)blockIdx.x == a.withhold_block)) break;
    first_barrier = false;
    // ------------------------------------------------------------ delivery phase
    const int buf = (int)(t & 1);
    const unsigned long long c = __ldcg(a.sb.ctr + buf);
    uint32_t nch = (uint32_t)(c & kChunkMask);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.sb.ctr[buf ^ 1] = 0;           // the next step's list starts empty
      if (a.age) a.sb.pcnt[buf] = 0;   // consumed by this step's scan
    }
    const uint4* wi = buf ? a.sb.wi[1] : a.sb.wi[0];
    if (a.age) {
      if ((unsigned long long)nch > (unsigned long long)a.sb.wi_cap) nch = (uint32_t)a.sb.wi_cap;
      for (int64_t it = warp; it < (int64_t)nch; it += nwarps)
        deliver_due_item<WT, kFixed>(__ldcg(wi + it), a.csr, ring, lane);
    } else {
      for (int64_t ch = warp; ch < (int64_t)nch; ch += nwarps) {
        const uint4 e0 = __ldcg(wi + 2 * ch), e1 = __ldcg(wi + 2 * ch + 1);
        deliver_work_item<WT, kFixed>(e0, e1, t, a.csr, ring, lane);
      }
    }
    if (!grid_sync(a.bar, a.spin_limit, a.sb.err, false)) break;
    ++t;
  }
  if (kPipe && t > t_first && ld_acquire_u32(a.bar + 2) == 0u) {
    // the last step's queue: delivered before the launch ends
    const int q = (int)((t - 1) % 3);
    const uint32_t n = (uint32_t)(__ldcg(a.sb.ctr3 + q) & kChunkMask);
    const uint4* wq = a.sb.wi3[q];
    for (int64_t ch = warp; ch < (int64_t)n; ch += nwarps)
      deliver_work_item<WT, kFixed>(__ldcg(wq + 2 * ch), __ldcg(wq + 2 * ch + 1), t - 1, a.csr, ring, lane);
  }
  if (kAeif) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsub += __shfl_xor_sync(0xffffffffu, nsub, o);
    if (lane == 0 && nsub) atomicAdd(a.sb.substeps, nsub);
    if (cap_hit) atomicOr(a.sb.err, kErrSubstepCap);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.clk[0] = t;
    a.clk[1] = t - 1;
  }
}

namespace {

template <bool kFixed, typename WT, bool kLif, bool kAeif>
void* pick(bool pipe) {
  if (pipe) return reinterpret_cast<void*>(&k_persistent<kFixed, WT, kLif, kAeif, true>);
  return reinterpret_cast<void*>(&k_persistent<kFixed, WT, kLif, kAeif, false>);
}

template <bool kFixed, typename WT>
void* pick_models(bool lif, bool aeif, bool pipe) {
  if (lif && aeif) return pick<kFixed, WT, true, true>(pipe);
  if (aeif) return pick<kFixed, WT, false, true>(pipe);
  return pick<kFixed, WT, true, false>(pipe);
}

void* persistent_kernel(bool fixed, int wdtype, bool lif, bool aeif, bool pipe) {
  if (fixed) {
    if (wdtype == 0) return pick_models<true, float>(lif, aeif, pipe);
    if (wdtype == 1) return pick_models<true, __nv_bfloat16>(lif, aeif, pipe);
    return pick_models<true, __half>(lif, aeif, pipe);
  }
  if (wdtype == 0) return pick_models<false, float>(lif, aeif, pipe);
  if (wdtype == 1) return pick_models<false, __nv_bfloat16>(lif, aeif, pipe);
  return pick_models<false, __half>(lif, aeif, pipe);
}

}  // namespace

cudaError_t persistent_max_blocks_per_sm(bool fixed, int wdtype, bool lif, bool aeif, bool pipe, size_t smem,
                                         int* out) {
  void* k = persistent_kernel(fixed, wdtype, lif, aeif, pipe);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, kPersistBlock, smem);
}

cudaError_t launch_persistent(const PersistArgs& a, bool fixed, int wdtype, bool lif, bool aeif, bool pipe, int grid,
                              size_t smem, cudaStream_t st) {
  void* k = persistent_kernel(fixed, wdtype, lif, aeif, pipe);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPersistBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<PersistArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace ngb
