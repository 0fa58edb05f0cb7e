// net.h -- the network handle behind the C ABI (host side, not exported).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/snn.h"
#include "snn_internal.cuh"

struct snn_grad;

using snn::kDCodes;
using snn::kMaxPop;
using snn::kPoisTable;
using snn::kRing;
using snn::kWCodes;

struct snn_net {
    snn_config cfg;
    uint64_t seed;
    cudaStream_t stream;
    int n, n_pop, P, ncmax, npt;
    bool smem_ring;
    size_t smem;
    int32_t pop_start[kMaxPop + 1];
    std::vector<int32_t> part_lo;
    uint64_t nnz;
    int32_t wtab[kMaxPop * kMaxPop * kWCodes];
    uint8_t dtab[kMaxPop * kDCodes];
    uint64_t pois[kMaxPop][kPoisTable];
    uint64_t conn_thr[kMaxPop][kMaxPop];
    int32_t wext_q, n_ref;
    float prop[4];
    float cdc[kMaxPop];
    int64_t step;
    uint64_t timeout_ns;
    uint32_t ras_cap;
    int32_t inject_fault;
    // device
    int32_t* d_part_lo = nullptr;
    unsigned long long* d_row_start = nullptr;
    uint32_t* d_seg = nullptr;
    uint32_t* d_words = nullptr;
    uint32_t* d_pre = nullptr;              // rows pre-decoded (weight-table index, ring offset)
    int32_t* d_wtab = nullptr;
    uint8_t* d_dtab = nullptr;
    float* d_u = nullptr;
    float* d_i = nullptr;
    int32_t* d_r = nullptr;
    int32_t* d_ring = nullptr;
    int32_t w_span = 1;                    // target populations of the widest partition
    int32_t run_max = 0;                   // longest (row, partition) run
    int32_t max_delay = kRing - 1;         // longest delay of any synapse (steps)
    std::vector<uint32_t> indeg;           // [n][8] synapses per source population
    long long in_bound = 0;                // largest |input| of one neuron-step (1/256 pA)
    bool sat_check = false;                // in_bound reaches 2^31: count wrap-arounds
    int32_t* d_wrap = nullptr;             // wrap counts, ring layout (sat_check only)
    uint32_t* step_counts = nullptr;       // caller's device buffer of per-step counts
    int64_t sc_t0 = 0, sc_cap = 0;
    unsigned long long* d_msg = nullptr;   // [4][P][msg_stride] tagged spike messages
    int32_t msg_stride = 0;
    uint32_t* d_ras_step = nullptr;
    uint32_t* d_ras_id = nullptr;
    uint32_t* d_ras_n = nullptr;
    uint32_t* d_rs_step = nullptr;          // raster read staging: every partition's entries packed
    uint32_t* d_rs_id = nullptr;
    size_t rs_cap = 0;                      // entries the staging arrays hold
    unsigned long long* d_counters = nullptr;
    uint32_t* d_sync = nullptr;   // [4] status, [5] abort
    unsigned long long* d_pop_spikes = nullptr;   // [8] spikes per population
    uint64_t rt_period = 0;                 // pacing period in ns (0: off)
    int64_t rt_t_anchor = 0;                // step whose start anchors the paced run
    unsigned long long* d_rt = nullptr;     // [3] anchor, missed deadlines, max lateness
    snn_grad* grad = nullptr;     // gradient checkpoints and adjoint state
    long long* step_times = nullptr;  // caller's device buffer of step-end clocks
    int64_t st_t0 = 0, st_cap = 0;
};

namespace snn {
// every field of the step kernel's parameters that does not depend on the
// launch (t0 and n_steps are set by the caller; trace pointers are null)
void fill_step_params(const snn_net* net, StepParams* sp);
// recompute the weight, delay, Poisson and propagator tables from net->cfg
int net_make_tables(snn_net* net);
// upload the weight table (the step kernel stages it at launch) and update
// the input bound and the saturation check
int net_upload_weights(snn_net* net);
// recompute the input bound from the weights; the first time it reaches 2^31
// the wrap-count array is allocated, and the step kernel counts wrap-arounds
int net_update_saturation(snn_net* net);
// zero the wrap counts (after the ring was replaced: load, restore)
cudaError_t net_clear_wraps(snn_net* net);
// launch the step kernel for n steps from step t0 with the given parameters
cudaError_t net_launch(snn_net* net, StepParams& sp, int64_t t0, int64_t n);
void free_grad(snn_grad* g);
int set_error(int code, const char* msg);
int set_cuda_error(cudaError_t e, const char* what);
}  // namespace snn
