// noalloc.cu -- snn_step_noalloc: the time-step kernel on caller-owned device
// memory, for callers that must not allocate device memory at run time.
//
// A closed-loop application that steps the network every 0.1 ms (a robot
// controller, an experiment rig driven in real time) typically reserves all
// of its device memory once, from its own pool, and may not call cudaMalloc
// or cudaFree while it runs: those calls can synchronise the whole device
// and take an unbounded time.  This entry point therefore allocates nothing.
// The caller passes the network, the state and the output buffers as device
// pointers; the kernel's scratch (spike lists, barrier and status words)
// lives in the file-scope array g_noalloc_scratch below, which every GPU that
// loads this library holds (about 1 MiB) until the process exits.
//
// The paper has no counterpart of this entry point.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/snn.h"
#include "snn_internal.cuh"

namespace snn {

int host_step_constants(const snn_config* cfg, float prop[4], float cdc[kMaxPop],
                        uint64_t pois[kMaxPop][kPoisTable], int32_t* wext_q, int32_t* n_ref);
int set_error(int code, const char* msg);
int set_cuda_error(cudaError_t e, const char* what);

namespace {

constexpr int kNaThreads = 512;
constexpr int kNaMaxDevices = 64;
// scratch words: [0..3] barrier A, [4..7] barrier B, [8] status, [9] abort,
// [16..17] spike counts of the two lists, [64 ...] two spike lists
constexpr size_t kNaHeader = 64;
constexpr size_t kNaScratchWords = kNaHeader + 2 * (size_t)SNN_NOALLOC_MAX_NEURONS;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaScratchWords];

struct NaParams {
    int32_t n, n_pop, n_part;
    int32_t pop_start[kMaxPop + 1];
    float P22, P21, P11, theta;
    float cdc[kMaxPop];
    int32_t n_ref, wext_q, mode;
    uint32_t key0, key1;
    int64_t t0;
    int32_t n_steps;
    uint64_t timeout_ns;
    uint64_t pois[kMaxPop][kPoisTable];
    const unsigned long long* row_ptr;
    const uint32_t* words;
    const int32_t* wtab;
    float* u;
    float* i_syn;
    int32_t* refr;
    int32_t* ring;                      // [64][n]
    uint32_t* ras_step;
    uint32_t* ras_id;
    uint32_t* ras_n;
    uint32_t ras_cap;
    unsigned long long* counters;
    uint32_t* status;                   // caller's word: | 1 on a timed-out wait
    uint32_t* scratch;                  // device address of g_noalloc_scratch
};

__device__ bool na_wait(const NaParams& p, const uint32_t* ctr, uint32_t target) {
    const uint64_t t_start = globaltimer_ns();
    uint32_t iter = 0;
    uint32_t* status = p.scratch + 8;
    uint32_t* abort_flag = p.scratch + 9;
    while (true) {
        if (ld_acquire_gpu(ctr) >= target) return true;
        if ((++iter & 255u) == 0u) {
            if (ld_relaxed_gpu(abort_flag) != 0u) return false;
            if (globaltimer_ns() - t_start > p.timeout_ns || iter > 0x7fffffffu) {
                atomicOr(status, kStatusTimeout);
                atomicOr(p.status, kStatusTimeout);
                atomicExch(abort_flag, 1u);
                return false;
            }
        }
    }
}

// grid barrier slot `slot` of step index s (all CTAs arrive once per step)
__device__ bool na_barrier(const NaParams& p, uint32_t* bar, int s, volatile uint32_t* s_abort) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_gpu_add(&bar[s & 3], 1u);
        if (!na_wait(p, &bar[s & 3], (uint32_t)p.n_part * (uint32_t)(s / 4 + 1))) *s_abort = 1u;
    }
    __syncthreads();
    return *s_abort == 0u;
}

__global__ void __launch_bounds__(kNaThreads, 1) k_step_noalloc(const __grid_constant__ NaParams p) {
    __shared__ uint64_t s_pois[kMaxPop * kPoisTable];
    __shared__ volatile uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31;
    const int c = blockIdx.x, P = p.n_part;
    uint32_t* barA = p.scratch;
    uint32_t* barB = p.scratch + 4;
    uint32_t* cnt = p.scratch + 16;
    uint32_t* lists = p.scratch + kNaHeader;
    for (int k = tid; k < kMaxPop * kPoisTable; k += kNaThreads)
        s_pois[k] = p.pois[k / kPoisTable][k % kPoisTable];
    if (tid == 0) s_abort = 0u;
    const int32_t lo = (int32_t)(((long long)c * p.n) / P);
    const int32_t hi = (int32_t)(((long long)(c + 1) * p.n) / P);
    unsigned long long spikes = 0, events = 0;
    __syncthreads();

    for (int s = 0; s < p.n_steps; ++s) {
        const int64_t t = p.t0 + s;
        const int lb = (int)(t & 1);
        const uint32_t slot = (uint32_t)t & (kRing - 1);
        // membrane update (uses I of step t-1), then this step's input into I
        for (int32_t i0 = lo; i0 < hi; i0 += kNaThreads) {
            const int32_t i = i0 + tid;
            bool spk = false;
            if (i < hi) {
                const int pop = pop_index(p.pop_start, p.n_pop, i);
                float u = p.u[i], isyn = p.i_syn[i];
                int32_t r = p.refr[i];
                if (r > 0) {
                    r -= 1;
                    u = 0.f;
                } else {
                    float v = __fadd_rn(__fmul_rn(p.P22, u), __fmul_rn(p.P21, isyn));
                    if (p.mode == 1) v = __fadd_rn(v, p.cdc[pop]);
                    u = v;
                }
                int32_t acc = p.ring[(size_t)slot * p.n + i];
                p.ring[(size_t)slot * p.n + i] = 0;
                if (p.mode == 0) {
                    const uint4 rnd = philox(make_uint4((uint32_t)i, (uint32_t)(t >> 2), kStreamPois,
                                                        (uint32_t)(t >> 34)), p.key0, p.key1);
                    const uint32_t x = lane_of(rnd, (int)(t & 3));
                    int kk = 0;
                    while (kk < kPoisTable && (uint64_t)x >= s_pois[pop * kPoisTable + kk]) ++kk;
                    acc += kk * p.wext_q;
                }
                isyn = __fadd_rn(__fmul_rn(p.P11, isyn), __fmul_rn(__int2float_rn(acc), 0.00390625f));
                if (u > p.theta) {
                    spk = true;
                    u = 0.f;
                    r = p.n_ref;
                }
                p.u[i] = u;
                p.i_syn[i] = isyn;
                p.refr[i] = r;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, spk);
            if (mask) {
                uint32_t base = 0, rbase = 0;
                if (lane == 0) {
                    base = atomicAdd(&cnt[lb], (uint32_t)__popc(mask));
                    rbase = atomicAdd(p.ras_n, (uint32_t)__popc(mask));
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                rbase = __shfl_sync(0xffffffffu, rbase, 0);
                if (spk) {
                    const uint32_t off = (uint32_t)__popc(mask & ((1u << lane) - 1u));
                    lists[(size_t)lb * SNN_NOALLOC_MAX_NEURONS + base + off] = (uint32_t)i;
                    if (rbase + off < p.ras_cap) {
                        p.ras_step[rbase + off] = (uint32_t)t;
                        p.ras_id[rbase + off] = (uint32_t)i;
                    }
                }
                if (lane == 0) spikes += (unsigned long long)__popc(mask);
            }
        }
        // all spikes of step t are listed
        if (!na_barrier(p, barA, s, &s_abort)) break;
        // the list of step t-1 is consumed everywhere: clear its counter for t+1
        if (c == 0 && tid == 0) cnt[lb ^ 1] = 0u;
        // deliver the spikes of step t into slots t + d, one warp per spike
        const uint32_t nsp = __ldcg(&cnt[lb]);
        const int warps = P * (kNaThreads / 32);
        for (uint32_t k = (uint32_t)(c * (kNaThreads / 32) + (tid >> 5)); k < nsp; k += (uint32_t)warps) {
            const uint32_t j = __ldcg(&lists[(size_t)lb * SNN_NOALLOC_MAX_NEURONS + k]);
            const int q = pop_index(p.pop_start, p.n_pop, (int32_t)j);
            const unsigned long long b = p.row_ptr[j], e = p.row_ptr[j + 1];
            for (unsigned long long w = b + lane; w < e; w += 32) {
                const uint32_t word = __ldg(&p.words[w]);
                const int32_t tgt = (int32_t)(word & kTgtMask);
                const uint32_t d = (word >> kTgtBits) & 63u;
                const int pp = pop_index(p.pop_start, p.n_pop, tgt);
                const int32_t wt = __ldg(&p.wtab[(pp * kMaxPop + q) * kWCodes + (word >> 25)]);
                atomicAdd(&p.ring[(size_t)(((uint32_t)t + d) & (kRing - 1)) * p.n + tgt], wt);
            }
            if (lane == 0) events += e - b;
        }
        // every ring slot of step t+1 is complete before anyone reads it
        if (!na_barrier(p, barB, s, &s_abort)) break;
    }
    if (lane == 0 && (spikes | events)) {
        atomicAdd(&p.counters[0], spikes);
        atomicAdd(&p.counters[1], events);
    }
}

// set-up of each device, done once by its first call: the scratch array's
// device address, the architecture check, the SM count and the co-resident
// CTAs per SM of the kernel (so that a call only fills parameters, clears the
// scratch header and launches)
struct NaDevice {
    uint32_t* scratch;
    cudaError_t err;
    const char* what;                   // the set-up call that failed
    bool arch_ok;
    int sms, per_sm;
};
std::once_flag g_setup_once[kNaMaxDevices];
NaDevice g_dev[kNaMaxDevices];

void setup_device(int dev) {
    NaDevice& d = g_dev[dev];
    d.what = "cudaGetSymbolAddress(g_noalloc_scratch)";
    d.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.scratch), g_noalloc_scratch);
    if (d.err != cudaSuccess) return;
    cudaDeviceProp prop;
    d.what = "cudaGetDeviceProperties";
    d.err = cudaGetDeviceProperties(&prop, dev);
    if (d.err != cudaSuccess) return;
    d.arch_ok = prop.major == 10 && prop.minor == 3;
    d.sms = prop.multiProcessorCount;
    d.what = "occupancy query";
    d.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.per_sm, k_step_noalloc, kNaThreads, 0);
}

}  // namespace
}  // namespace snn

using namespace snn;

extern "C" int snn_step_noalloc(const snn_config* cfg, uint64_t seed, const snn_noalloc_io* io,
                                int64_t t0, int64_t n_steps, void* stream) {
    if (!cfg || !io) return set_error(SNN_ERR_INVALID, "config and io are required");
    if (n_steps < 0 || n_steps > (1 << 24) || t0 < 0)
        return set_error(SNN_ERR_INVALID, "need 0 <= n_steps <= 2^24 and t0 >= 0");
    long long n = 0;
    if (cfg->n_pop >= 1 && cfg->n_pop <= kMaxPop)
        for (int q = 0; q < cfg->n_pop; ++q) n += cfg->pop_size[q];
    if (n > SNN_NOALLOC_MAX_NEURONS)
        return set_error(SNN_ERR_INVALID,
                         "snn_step_noalloc supports at most SNN_NOALLOC_MAX_NEURONS (131072) "
                         "neurons: its static scratch holds two spike lists of that length");
    NaParams p;
    std::memset(&p, 0, sizeof(p));
    float pr[4];
    int rc = host_step_constants(cfg, pr, p.cdc, p.pois, &p.wext_q, &p.n_ref);
    if (rc != SNN_OK) return rc;
    p.P22 = pr[0];
    p.P21 = pr[1];
    p.P11 = pr[2];
    if (!io->row_ptr || !io->words || !io->wtab || !io->u || !io->i_syn || !io->refr ||
        !io->ring || !io->ras_step || !io->ras_id || !io->ras_n || !io->counters || !io->status)
        return set_error(SNN_ERR_INVALID, "every io pointer is required");
    if (n_steps == 0) return SNN_OK;

    // once per device, with that device current: device address of the scratch
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(SNN_ERR_UNSUPPORTED, "device index too large");
    std::call_once(g_setup_once[dev], setup_device, dev);
    const NaDevice& d = g_dev[dev];
    if (d.err != cudaSuccess) return set_cuda_error(d.err, d.what);
    if (!d.arch_ok)
        return set_error(SNN_ERR_UNSUPPORTED, "this library is built for sm_103 (GB300) GPUs only");
    if (d.per_sm < 1) return set_error(SNN_ERR_UNSUPPORTED, "step kernel does not fit an SM");
    // one CTA per SM at most, about 256 neurons per CTA for small networks
    const int P = (int)std::min<long long>(d.sms, std::max<long long>(1, (n + 255) / 256));

    p.n = (int32_t)n;
    p.n_pop = cfg->n_pop;
    p.n_part = P;
    p.pop_start[0] = 0;
    for (int q = 0; q < kMaxPop; ++q)
        p.pop_start[q + 1] = p.pop_start[q] + (q < cfg->n_pop ? cfg->pop_size[q] : 0);
    p.theta = (float)cfg->theta;
    p.mode = cfg->input_mode;
    p.key0 = (uint32_t)(seed & 0xffffffffu);
    p.key1 = (uint32_t)(seed >> 32);
    p.t0 = t0;
    p.n_steps = (int32_t)n_steps;
    p.timeout_ns = 2000000000ull;
    p.row_ptr = reinterpret_cast<const unsigned long long*>(io->row_ptr);
    p.words = io->words;
    p.wtab = io->wtab;
    p.u = io->u;
    p.i_syn = io->i_syn;
    p.refr = io->refr;
    p.ring = io->ring;
    p.ras_step = io->ras_step;
    p.ras_id = io->ras_id;
    p.ras_n = io->ras_n;
    p.ras_cap = (uint32_t)std::min<int64_t>(std::max<int64_t>(io->ras_cap, 0), 0x7fffffff);
    p.counters = io->counters;
    p.status = io->status;
    p.scratch = d.scratch;

    // the shared scratch keeps the previous call's contents: clear the
    // barrier, status and list-counter words that must start at zero
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(p.scratch, 0, sizeof(uint32_t) * kNaHeader, s);
    if (e != cudaSuccess) return set_cuda_error(e, "clearing the scratch header");
    void* args[] = {&p};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_step_noalloc), dim3(P),
                                    dim3(kNaThreads), args, 0, s);
    if (e != cudaSuccess) return set_cuda_error(e, "launch of the allocation-free step kernel");
    return SNN_OK;
}
