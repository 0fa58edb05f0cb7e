// snn_internal.cuh -- device-side definitions shared by the kernels of the
// GB300 microcircuit library (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace snn {

constexpr int kMaxPop = 8;
constexpr int kWCodes = 128;
constexpr int kDCodes = 256;
constexpr int kPoisTable = 32;
constexpr int kRing = 64;                 // delay slots (delays 1..63)
constexpr int kStepThreads = 512;         // threads per CTA of the step kernel
constexpr int kChunk = 1024;              // spikes per delivery chunk
constexpr int kBuildThreads = 256;        // threads per CTA of the build kernels
constexpr uint32_t kTgtBits = 19;
constexpr uint32_t kTgtMask = (1u << kTgtBits) - 1u;

// Philox stream tags (third counter word)
constexpr uint32_t kStreamConn = 1u;
constexpr uint32_t kStreamSyn = 2u;
constexpr uint32_t kStreamPois = 3u;
constexpr uint32_t kStreamInit = 4u;

// status bits
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint32_t kStatusSaturated = 4u;   // a step's input left the int32 range

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the two 32x32->64-bit
// products with multipliers 0xD2511F53 (word 0) and 0xCD9E8D57 (word 2), the
// word permutation (hi1^c1^k0, lo1, hi0^c3^k1, lo0) and the Weyl key bumps
// 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t lane_of(const uint4& v, int lane) {
    return lane == 0 ? v.x : lane == 1 ? v.y : lane == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait until the device clock reaches target; bounded by 2^26 sleeps of
// about 128 ns (seconds, beyond the longest allowed pacing period)
__device__ __forceinline__ void wait_until_ns(uint64_t target) {
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (globaltimer_ns() >= target) return;
        __nanosleep(128);
    }
}

// Full grid barrier of a cooperative launch on a monotonic arrival counter
// (zeroed before the launch): barrier number `gen` completes when the counter
// reaches (gen + 1) * gridDim.x.  The wait is bounded: it gives up when
// another CTA raised the abort flag, or after timeout_ns, when it sets the
// timeout status bit and the abort flag itself.  skip_arrive withholds this
// CTA's arrival (tests of the bounded wait).  Returns false once aborted.
// The arrival is a release reduction by thread 0 after the CTA barrier (it
// publishes the writes the CTA made before it, and nothing waits for a
// returned value); the polls are acquire loads, so the CTA sees every write
// made before the other CTAs' arrivals.
__device__ __forceinline__ bool grid_barrier(uint32_t* counter, uint32_t* abort_flag,
                                             uint32_t* status, uint64_t timeout_ns,
                                             uint32_t& gen, volatile uint32_t* s_abort,
                                             bool skip_arrive) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!skip_arrive) red_release_gpu_add(counter, 1u);
        const uint32_t target = (gen + 1u) * gridDim.x;
        const uint64_t t_start = globaltimer_ns();
        uint32_t iter = 0;
        while (ld_acquire_gpu(counter) < target) {
            if ((++iter & 255u) == 0u) {
                if (ld_relaxed_gpu(abort_flag) != 0u) { *s_abort = 1u; break; }
                if (globaltimer_ns() - t_start > timeout_ns) {
                    atomicOr(status, kStatusTimeout);
                    atomicExch(abort_flag, 1u);
                    *s_abort = 1u;
                    break;
                }
            }
        }
    }
    __syncthreads();
    ++gen;
    return *s_abort == 0u;
}

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
struct BuildParams {
    int32_t n;                          // neurons
    int32_t n_pop;
    int32_t pop_start[kMaxPop + 1];
    int32_t n_part;
    uint32_t key0, key1;
    uint64_t conn_thr[kMaxPop][kMaxPop];  // [target][source], compare x < thr
    const uint8_t* dtab;                // device [8][256] delays in steps
    const int32_t* part_lo;             // device [n_part + 1]
};

// model constants and tables of one configuration, computed on the host
struct HostTables {
    int32_t n, n_pop;
    int32_t pop_start[kMaxPop + 1];
    int32_t wtab[kMaxPop * kMaxPop * kWCodes];
    uint64_t pois[kMaxPop][kPoisTable];
    float prop[4];                      // P22, P21, P11, P20
    float cdc[kMaxPop];
    float theta;
    int32_t wext_q, n_ref, mode;
    int32_t max_delay;                  // longest delay (steps) of any synapse
};

struct StepParams {
    int32_t n, n_pop, n_part, ncmax;
    int32_t pop_start[kMaxPop + 1];
    float P22, P21, P11, theta;
    float cdc[kMaxPop];                 // P20 * I_DC per population (mode 1)
    int32_t n_ref, wext_q, mode;
    uint32_t key0, key1;
    int64_t t0;
    int32_t n_steps;
    uint32_t ras_cap;                   // raster capacity per partition
    uint64_t timeout_ns;
    int32_t inject_fault;               // 1: partition 0 never publishes
    int32_t msg_stride;                 // 64-bit words per message (>= ncmax + 1)
    int32_t w_span;                     // target populations of the widest partition
    uint32_t pois_m1[kMaxPop][kPoisTable];  // Poisson thresholds minus 1 (x > T-1 -> +1)
    // network (read only)
    const int32_t* part_lo;             // [n_part + 1]
    const uint32_t* seg;                // [n][n_part + 1] absolute word offsets
    const uint32_t* words;
    const uint32_t* pre;                // pre-decoded rows, same layout as words
    const int32_t* wtab;                // [8][8][128]
    const unsigned long long* row_start;  // [n + 1] row offsets
    // state
    float* u;
    float* i_syn;
    int32_t* refr;
    int32_t* ring;                      // [n_part][kRing][ncmax]
    unsigned long long* msg;            // [4][n_part][msg_stride] tagged spike messages
    uint32_t* ras_step;                 // [n_part][ras_cap]
    uint32_t* ras_id;
    uint32_t* ras_n;                    // [n_part] spikes recorded (may exceed cap)
    unsigned long long* counters;       // [0] spikes, [1] synaptic events
    unsigned long long* pop_spikes;     // [8] spikes per population
    uint32_t* status;
    uint32_t* abort_flag;
    // optional per-step record for the gradient: for steps t in
    // [tr_t0, tr_t0 + tr_len), tr_u[(t - tr_t0) n + i] = u after the
    // membrane update (before reset), tr_f = spike | non-refractory << 1
    float* tr_u;
    uint8_t* tr_f;
    int64_t tr_t0;
    int32_t tr_len;
    // optional device clock (ns) at the end of step t, written by CTA 0 to
    // step_times[t - st_t0] for t - st_t0 in [0, st_cap)
    long long* step_times;
    int64_t st_t0, st_cap;
    // optional per-step counts (snn_record_step_counts): for steps t with
    // r = t - sc_t0 in [0, sc_cap), st_counts[4 r ..] = spikes of step t,
    // their synaptic events, the largest number of them one partition
    // processed (non-empty runs), and the (spike, partition) pairs with an
    // empty run; zeroed by the host before recording starts
    uint32_t* st_counts;
    int64_t sc_t0, sc_cap;
    // wrap-around counts of the ring cells, same layout as ring ([n_part][64]
    // [ncmax]); non-null only for networks whose input can leave the int32
    // range, which then take the kernel variant that counts wrap-arounds
    int32_t* wrap;
    // pacing to wall-clock time (0: off): step t starts no earlier than
    // rt[0] + (t - rt_t_anchor) * rt_period_ns, rt[0] being the device clock
    // when the first paced step started (0 until then); rt[1] counts steps
    // that ended after their deadline, rt[2] holds the largest lateness (ns)
    unsigned long long rt_period_ns;
    int64_t rt_t_anchor;
    unsigned long long* rt;
};

struct DeliverParams {
    int32_t n, n_pop, n_part, ncmax, n_spikes;
    int32_t pop_start[kMaxPop + 1];
    int64_t t;
    const uint32_t* spikes;
    const int32_t* part_lo;
    const uint32_t* seg;
    const uint32_t* words;
    const uint32_t* pre;          // pre-decoded rows (partition-word delivery)
    int32_t max_delay;            // longest delay of any synapse (partition-word delivery)
    const int32_t* wtab;
    int32_t* ring;
    unsigned long long* counters;
    uint32_t* status;             // ORed with the timeout bit if a bounded wait gives up
};

__device__ __forceinline__ int pop_index(const int32_t* pop_start, int n_pop, int32_t i) {
    int p = 0;
#pragma unroll
    for (int k = 1; k < kMaxPop; ++k)
        p += (k < n_pop && i >= pop_start[k]) ? 1 : 0;
    return p;
}

// host-side launchers (defined in the .cu files)
cudaError_t launch_build_count(const BuildParams& bp, uint32_t* rowlen, cudaStream_t s);
cudaError_t launch_build_scan(const uint32_t* rowlen, int n, unsigned long long* row_start,
                              cudaStream_t s);
cudaError_t launch_build_fill(const BuildParams& bp, const unsigned long long* row_start,
                              uint32_t* words, uint32_t* seg, cudaStream_t s);
cudaError_t launch_seg_from_rows(const unsigned long long* row_start, const uint32_t* words,
                                 int n, const int32_t* part_lo, int n_part, uint32_t* seg,
                                 cudaStream_t s);
// indeg[i * 8 + q] = synapses from population q onto neuron i (zeroed first)
cudaError_t launch_indegree(const unsigned long long* row_start, const uint32_t* words, int n,
                            int n_pop, const int32_t* pop_start, uint32_t* indeg, cudaStream_t s);
// largest possible |input| of one neuron in one step (1/256 pA): over neurons
// i, sum_q indeg[i][q] max_code |wtab[pop(i)][q][code]|, plus 32 |wext_q| when
// the background is Poisson (at most 32 background spikes per step)
long long input_bound(const uint32_t* indeg, int n, int n_pop, const int32_t* pop_start,
                      const int32_t* wtab, int32_t wext_q, int input_mode);
// out[c] = longest (row, partition c) segment, for every partition c
cudaError_t launch_max_segment(const uint32_t* seg, int n, int n_part, uint32_t* out,
                               cudaStream_t s);
// the raster entries of every partition (counts clamped to cap_part, then the
// first `limit` entries in partition order) packed into step_out / id_out
cudaError_t launch_pack_raster(const uint32_t* counts, int n_part, uint32_t cap_part,
                               int64_t limit, const uint32_t* ras_step, const uint32_t* ras_id,
                               uint32_t* step_out, uint32_t* id_out, cudaStream_t s);
cudaError_t launch_init_state(int n, uint32_t key0, uint32_t key1, float lo, float hi,
                              float* u, cudaStream_t s);
int step_kernel_variant(int npt, bool smem_ring);
size_t step_shared_bytes(int ncmax, int n_part, int w_span, bool smem_ring);
// target populations spanned by the widest of the partitions [part_lo[c],
// part_lo[c+1]) (the rows of the weight table a CTA of the step kernel keeps)
int partition_pop_span(const int32_t* part_lo, int n_part, const int32_t* pop_start, int n_pop);
cudaError_t step_kernel_configure(int npt, bool smem_ring, size_t smem);
cudaError_t launch_step(const StepParams& sp, int npt, bool smem_ring, size_t smem,
                        cudaStream_t s);
cudaError_t launch_deliver(const DeliverParams& dp, int tiling, cudaStream_t s);
// stand-alone delivery of the exact row segments of each partition (one CTA
// per partition, packed words cut into units of <= 32 words, weight table and,
// when it fits, the ring slice in shared memory)
cudaError_t launch_deliver_words(const DeliverParams& dp, cudaStream_t s);
// pre-decoded rows for launch_deliver_words: entry k of row j is
// (weight-table index << kPreOffBits) | (delay * ncmax + target - partition start),
// same layout as the packed words; needs kRing * ncmax < 2^kPreOffBits
constexpr uint32_t kPreOffBits = 19;
constexpr uint32_t kPreOffMask = (1u << kPreOffBits) - 1u;
cudaError_t launch_predecode(const DeliverParams& dp, const unsigned long long* row_start,
                             uint32_t* pre, cudaStream_t s);
// stand-alone delivery of the exact runs streamed into shared memory by bulk
// copies (one producer warp, consumer warps; ring slice in shared memory)
size_t deliver_stream_smem(int ncmax, int w_span);
cudaError_t launch_deliver_stream(const DeliverParams& dp, int w_span, cudaStream_t s);
// stand-alone delivery through clusters of 8 CTAs (rings in distributed
// shared memory); needs the ring slice and the weight table in shared memory
cudaError_t launch_deliver_cluster(const DeliverParams& dp, cudaStream_t s);
cudaError_t deliver_cluster_check(int ncmax, int n_part, int* max_active_clusters);
// The surrogate-gradient adjoint with its row gather done partition by
// partition in shared memory (adjoint_part.cu): the plan holds, per CTA
// (partition c, source group g), the runs of its sources into c re-packed for
// the gather.
struct AdjPartParams {
    int32_t n, n_pop, n_part, ncmax, len;
    int32_t groups, ring_r, span_max, img_max, max_lg;   // set by launch_adjoint_part
    int64_t t_first;                 // global step of trace row 0
    float P22, P21, P11, theta;
    float gs[kMaxPop];               // dL/ds per spike of each population
    int32_t pop_start[kMaxPop + 1];
    uint64_t timeout_ns;
    const int32_t* part_lo;
    const uint32_t* img;             // the CTAs' images (set by launch_adjoint_part)
    const uint32_t* img_off;
    const int32_t* wtab;             // rounded weights of the forward, 1/256 pA
    const float* wbase;              // base weights, pA
    const float* tr_u;
    const uint8_t* tr_f;
    float* lu;
    float* lI;
    float* lring;                    // [64][n] lI of the last 64 steps
    uint8_t* mnext;
    float* pds;                      // [2][n_part][n] partial spike adjoints
    double* gAc;                     // [n_part][n][8] partial weight gradients
    double* gN;
    uint32_t* barrier;
    uint32_t* status;
    uint32_t* abort_flag;
};
struct AdjPartPlan {
    int grid = 0, groups = 0, ring_r = 0, span_max = 0;
    int32_t img_max = 0;             // words of the largest CTA image
    int32_t max_lg = 0;              // most lane groups of one CTA
    size_t smem = 0;
    uint32_t* d_img = nullptr;
    uint32_t* d_img_off = nullptr;   // [grid + 1]
};
// 0: planned; 1: the network does not fit (use the global gather); < 0: error
int adjoint_part_plan(int n, int n_pop, const int32_t* pop_start, int n_part, const int32_t* part_lo,
                      int ncmax, uint64_t nnz, const unsigned long long* d_row_start,
                      const uint32_t* d_pre, const uint32_t* d_seg, AdjPartPlan* plan);
void adjoint_part_free(AdjPartPlan* plan);
cudaError_t launch_adjoint_part(const AdjPartPlan& plan, AdjPartParams& ap, cudaStream_t s);
cudaError_t launch_adjoint_part_fold(int n, int n_part, int n_pop, const int32_t* part_lo,
                                     const int32_t* pop_start, const double* gAc, double* gA,
                                     cudaStream_t s);
// stand-alone delivery through the step kernel's runs (one CTA per partition)
cudaError_t launch_deliver_part(const StepParams& sp, const uint32_t* spikes, int n, int64_t t,
                                bool smem_ring, cudaStream_t s);

}  // namespace snn
