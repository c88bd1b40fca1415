// builder.h -- host interface of the device connection builder (builder.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace ngb {

// One connect call, as the draw kernel sees it.
struct CallDev {
  uint64_t seed;       // instance key
  uint64_t nsyn;       // draws: K * n_tgt (fixed indegree) or K (fixed total)
  int64_t K;
  double w0, w1, d0, d1, dt;
  uint32_t stream;     // connect-call index within the instance
  int32_t rule;        // 0 fixed indegree, 1 fixed total number
  int32_t no_autapse;  // source == target population and autapses excluded
  int32_t wdist, ddist, receptor, prec;
  int32_t stdp;        // STDP rule + 1 of the call's synapses (0: static)
  int32_t pad_;
  uint32_t n_src, n_tgt;
  uint32_t src_off, tgt_off;  // global id of the first source / target neuron
};

// Device scratch sized for the largest source population.
struct BuildScratch {
  unsigned long long* keys = nullptr;
  unsigned long long* keys_alt = nullptr;
  uint32_t* vals = nullptr;
  uint32_t* vals_alt = nullptr;
  uint32_t* st_tgt = nullptr;
  float* st_w = nullptr;
  uint32_t* flag = nullptr;
  uint32_t* gidx = nullptr;
  void* sort_tmp = nullptr;
  size_t sort_bytes = 0;
  void* scan_tmp = nullptr;
  size_t scan_bytes = 0;
};

cudaError_t sort_scratch_bytes(uint64_t n, int key_bits, size_t* sort_bytes, size_t* scan_bytes);
cudaError_t scan_scratch_bytes_u64(uint64_t n, size_t* bytes);

// Draw, sort and gather every synapse whose source is in one population; the
// CSR slice starts at tgt_out / w_out (already offset).  Returns the
// population's group starts (global synapse index) and delays in new device
// arrays owned by the caller.
cudaError_t build_source_population(const std::vector<CallDev>& calls, uint64_t n_total, int src_bits,
                                    uint64_t csr_off, int wdtype, BuildScratch& s, uint32_t* tgt_out, void* w_out,
                                    unsigned long long* src_cnt, unsigned long long* src_ngrp, int* max_delay,
                                    uint64_t** gstart_out, uint16_t** gdelay_out, uint64_t* ngroups_out,
                                    cudaStream_t st, std::string& err);

cudaError_t exclusive_scan_u64(const unsigned long long* in, unsigned long long* out, uint64_t n, void* tmp,
                               size_t tmp_bytes, cudaStream_t st);
cudaError_t expand_synapses(uint64_t first, uint64_t n, const uint32_t* tgt, const void* w, int wdtype,
                            const uint64_t* gstart, uint64_t G, const uint16_t* gdelay, uint32_t* o_tgt,
                            uint8_t* o_rc, float* o_w, uint16_t* o_d, cudaStream_t st);
// Source tables of a placed population (meta, first synapse, first group,
// first-group data for spike-buffer delivery); *items (device) accumulates
// the ring scheme's delivery work items.
cudaError_t fill_meta(uint64_t n, uint64_t off, uint64_t k_off, uint64_t g_off, const unsigned long long* cnt_scan,
                      const unsigned long long* grp_scan, const uint64_t* grp_start, const uint16_t* grp_delay,
                      uint4* meta, uint64_t* src_syn, uint32_t* src_grp, uint2* src_age, unsigned long long* items,
                      cudaStream_t st);
// The spike record (ids, steps; n entries) as sorted keys step << 26 | neuron.
cudaError_t record_sort_scratch_bytes(uint64_t n, size_t* bytes);
cudaError_t sort_record(const uint32_t* ids, const int64_t* steps, uint64_t n, unsigned long long* keys,
                        unsigned long long* sorted, void* tmp, size_t tmp_bytes, cudaStream_t st);
cudaError_t narrow_u64_to_u32(const unsigned long long* in, uint32_t* out, uint64_t n, cudaStream_t st);

}  // namespace ngb
