// batch.cu -- many independent microcircuits of uneven size and seed in one
// persistent kernel (the same method as the single network: Sec. 2.1 Eq. 1,
// Sec. 3.1.2 ring buffers, Sec. 3.1.3 per-step processing), replayed from a
// captured CUDA graph.
//
// The neurons of all instances are concatenated: instance k owns the global
// range [goff_k, goff_k + n_k).  CTA b owns the contiguous range
// [b * chunk, (b + 1) * chunk), chunk = ceil(total / CTAs) <= 512 NPT, and keeps u, I and the refractory
// counter of its neurons in registers; the four cached background draws of
// each neuron sit in shared memory.  The ring buffers of all neurons are one
// global array [slot][global neuron] of R slots, R = the longest delay of any
// instance + 1 (38 for the benchmark's delays: the 64-instance ring, 111 MB,
// fits in L2 where 64 slots would not); step t owns slot t mod R.
//
// Per step t the work is A(t) (membrane update u_t with I_{t-1}, threshold,
// reset, refractory; spikes appended to the list of step t), D(t) (delivery
// of the spikes of step t through their rows into ring slots t + d, d >= 1)
// and C(t) (I_t = P11 I_{t-1} + ring[t] + background).  A(t + 1) needs only
// I_t, and C(t) needs the deliveries of step t - 1, so one grid barrier per
// step suffices:
//     A(t0);  for t: { barrier; C(t); A(t + 1); D(t) }
// C(t) and A(t + 1) come first: they need only slot t, filled by D(t - 1)
// before the barrier, and run while no CTA has atomics in flight; D(t) then
// writes slots t + 1 .. t + R - 1 (mod R), never slot t.  The lists and
// their counters rotate over 2 and 4 step parities, so each buffer is reset
// or rewritten only after the barrier that ends its last reader's phase.
// Every result equals the single-network path bit for bit (same fp32
// operation order, integer accumulation, same random counters).
//
// Delivery tiling per instance: one warp per spike (tiling 0), one CTA per
// row (tiling 1), or flat (tiling 2): every CTA stages the step's flat-list
// rows (start, length, instance) in shared memory with a block scan, and all
// warps of the grid stride over the concatenated words, so one row's latency
// chain is paid once per step and the work is spread evenly over the SMs.
// The autotuner (host side, at creation) times the three on each instance's
// own rows with a seeded spike list of the instance's expected size and keeps
// the fastest.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/snn.h"
#include "snn_internal.cuh"

namespace snn {

int host_tables(const snn_config* cfg, HostTables* out);
int build_rows_device(const snn_config* cfg, uint64_t seed, cudaStream_t stream,
                      unsigned long long** row_start, uint32_t** words, uint64_t* nnz);
int set_error(int code, const char* msg);
int set_cuda_error(cudaError_t e, const char* what);

namespace {

constexpr int kBThreads = 512;
constexpr int kBWarps = kBThreads / 32;
constexpr int kMaxInst = 1024;
constexpr int kGraphChunk = 1000;       // steps per captured launch
constexpr int kWarpUnroll = 8;          // words in flight per lane, warp tiling
constexpr int kBlockUnroll = 4;         // words in flight per thread, CTA tiling
constexpr int kFlatUnroll = 4;          // words in flight per lane, flat tiling
constexpr int kFlatChunk = 1024;        // flat-list rows staged at once
constexpr int kTilings = 3;
constexpr uint32_t kBatchRasterOverflow = 2u;

// per-instance constants read in the neuron phases (one 48-byte record)
struct __align__(16) InstHot {
    float4 prop;                        // P22, P21, P11, theta
    int4 misc;                          // n_ref, mode, wext_q, goff
    uint4 key;                          // key0, key1, tiling, n
};

// per-instance data read in the delivery phase
struct InstCold {
    int32_t pop_start[kMaxPop + 1];
    int32_t n_pop, goff, n, pad;
    const unsigned long long* row_start;
    const uint32_t* words;
    const int32_t* wtab;                // [8 target pops][8 source pops][128 codes]
};

struct BatchParams {
    int32_t n_inst, ntot, n_steps;
    int32_t ring_depth;                 // D: slots of the ring, the longest delay + 1
    int32_t chunk;                      // neurons per CTA (<= NPT * kBThreads)
    int32_t inject_fault;               // 1: CTA 0 never arrives at a barrier
    uint64_t timeout_ns;
    const InstHot* hot;
    const InstCold* cold;
    const uint32_t* pois;               // [n_inst][8][32] thresholds minus one
    const float* cdc;                   // [n_inst][8] P20 * I_DC
    const int32_t* goff;                // [n_inst + 1]
    const int32_t* wtab_all;            // [n_inst][8][8][128] fixed-point weights
    const int32_t* ps_all;              // [n_inst][8] population starts (unused: INT_MAX)
    float* u;
    float* i_syn;
    int32_t* refr;
    int32_t* ring;                      // [D][ntot]
    uint32_t* list;                     // [2 parity][3 tiling][ntot] global ids
    uint32_t* cnt;                      // [4 parity][3 tiling]
    uint32_t* ras_step;
    uint32_t* ras_id;
    uint32_t* ras_n;
    uint32_t ras_cap;
    unsigned long long* inst_counters;  // [n_inst][2] spikes, events
    long long* step;                    // device step counter
    uint32_t* barrier;
    uint32_t* status;
    uint32_t* abort_flag;
};

__device__ __forceinline__ int inst_of(const int32_t* s_goff, int n_inst, int32_t gi) {
    int a = 0, b = n_inst;              // s_goff[a] <= gi < s_goff[b]
    while (b - a > 1) {
        const int m = (a + b) >> 1;
        if (s_goff[m] <= gi) a = m;
        else b = m;
    }
    return a;
}

__device__ __forceinline__ bool grid_sync(const BatchParams& p, uint32_t& gen,
                                          volatile uint32_t* s_abort) {
    return grid_barrier(p.barrier, p.abort_flag, p.status, p.timeout_ns, gen, s_abort,
                        p.inject_fault == 1 && blockIdx.x == 0);
}

// Row of global neuron gi, emitted at step t, added into ring slots t + d by
// `lanes` cooperating threads (rank r among them), U words in flight each.
// tD = t mod D; a synapse of delay d (1 <= d < D) adds into slot (tD + d) mod D
__device__ __forceinline__ uint32_t ring_slot(uint32_t tD, uint32_t d, uint32_t D) {
    const uint32_t sl = tD + d;
    return sl >= D ? sl - D : sl;
}

template <int U>
__device__ __forceinline__ void deliver_row(const BatchParams& p, const int32_t* s_goff, int32_t gi,
                                            uint32_t tD, int r, int lanes, bool count) {
    const int ki = inst_of(s_goff, p.n_inst, gi);
    const InstCold& I = p.cold[ki];
    const int32_t j = gi - I.goff;
    const int n_pop = I.n_pop;
    int32_t ps[kMaxPop];
#pragma unroll
    for (int k = 1; k < kMaxPop; ++k) ps[k] = k < n_pop ? I.pop_start[k] : 0x7fffffff;
    int q = 0;
#pragma unroll
    for (int k = 1; k < kMaxPop; ++k) q += j >= ps[k] ? 1 : 0;
    const int32_t* wq = I.wtab + q * kWCodes;
    const uint32_t* words = I.words;
    int32_t* rbase = p.ring + I.goff;
    const size_t ntot = (size_t)p.ntot;
    const unsigned long long b = I.row_start[j], e = I.row_start[j + 1];
    for (unsigned long long base = b + r; base < e; base += (unsigned long long)lanes * U) {
        uint32_t w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned long long idx = base + (unsigned long long)u * lanes;
            w[u] = idx < e ? __ldg(&words[idx]) : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (base + (unsigned long long)u * lanes < e) {
                const int32_t tgt = (int32_t)(w[u] & kTgtMask);
                int pp = 0;
#pragma unroll
                for (int k = 1; k < kMaxPop; ++k) pp += tgt >= ps[k] ? 1 : 0;
                const int32_t wt = __ldg(&wq[pp * (kMaxPop * kWCodes) + (int)(w[u] >> 25)]);
                const uint32_t slot = ring_slot(tD, (w[u] >> kTgtBits) & 63u, (uint32_t)p.ring_depth);
                atomicAdd(&rbase[(size_t)slot * ntot + tgt], wt);
            }
        }
    }
    if (count && r == 0) atomicAdd(&p.inst_counters[ki * 2 + 1], e - b);
}

// shared-memory arrays of the flat tiling (after the caller's own arrays)
struct FlatSmem {
    int32_t* ps;                 // [n_inst][8] population starts
    const uint32_t** beg;        // [kFlatChunk] first word of each staged row
    uint32_t* pre;               // [kFlatChunk + 1] exclusive prefix of row lengths
    uint32_t* meta;              // [kFlatChunk] instance << 3 | source population
    uint32_t* wsum;              // [kBWarps] scan partials
    // the first chunk of a step's flat list, fetched ahead by asynchronous
    // copies (k_batch): spike ids, their row bounds, the list length
    unsigned long long* pf_rs;   // [kFlatChunk][2] row_start[j], row_start[j + 1]
    const unsigned long long** rsp;   // [n_inst] row starts of each instance
    uint32_t* pf_ids;            // [kFlatChunk]
    uint32_t* pf_nf;             // [4]
};

__host__ __device__ inline size_t flat_smem_bytes(int n_inst) {
    return (size_t)kFlatChunk * sizeof(void*) + (size_t)kFlatChunk * 16 + (size_t)n_inst * sizeof(void*) +
           (size_t)n_inst * 8 * sizeof(int32_t) + ((size_t)kFlatChunk + 1) * 4 + (size_t)kFlatChunk * 4 +
           kBWarps * 4 + (size_t)kFlatChunk * 4 + 16;
}

__device__ inline FlatSmem flat_smem(unsigned char* base, int n_inst) {
    FlatSmem F;
    F.beg = reinterpret_cast<const uint32_t**>(base);
    F.pf_rs = reinterpret_cast<unsigned long long*>(base + (size_t)kFlatChunk * sizeof(void*));
    F.rsp = reinterpret_cast<const unsigned long long**>(F.pf_rs + 2 * (size_t)kFlatChunk);
    F.ps = reinterpret_cast<int32_t*>(F.rsp + n_inst);
    F.pre = reinterpret_cast<uint32_t*>(F.ps + (size_t)n_inst * 8);
    F.meta = F.pre + kFlatChunk + 1;
    F.wsum = F.meta + kFlatChunk;
    F.pf_ids = F.wsum + kBWarps;
    F.pf_nf = F.pf_ids + kFlatChunk;
    return F;
}

__device__ inline void flat_load_ps(const BatchParams& p, const FlatSmem& F) {
    for (int k = threadIdx.x; k < p.n_inst * 8; k += kBThreads) F.ps[k] = __ldg(&p.ps_all[k]);
    for (int k = threadIdx.x; k < p.n_inst; k += kBThreads) F.rsp[k] = p.cold[k].row_start;
}

// asynchronous global -> shared copies (completed by cp_async_wait)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Flat tiling: the rows of the nf spikes in `list`, spread over every warp of
// the grid.  Every CTA stages the same rows; CTA 0 alone counts the events.
// prefetched: the first chunk's ids and row bounds are in F.pf_ids / F.pf_rs
__device__ void deliver_flat(const BatchParams& p, const int32_t* s_goff, const FlatSmem& F,
                             const uint32_t* list, uint32_t nf, uint32_t tD, bool count,
                             bool prefetched = false) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t ntot = (size_t)p.ntot;
    for (uint32_t f0 = 0; f0 < nf; f0 += kFlatChunk) {
        const uint32_t mc = min((uint32_t)kFlatChunk, nf - f0);
        const bool pf = prefetched && f0 == 0;
        // stage two rows per thread: start, length, instance and population
        uint32_t len[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t k = (uint32_t)tid * 2u + (uint32_t)h;
            if (k < mc) {
                const int32_t gi = pf ? (int32_t)F.pf_ids[k] : (int32_t)__ldcg(&list[f0 + k]);
                const int ki = inst_of(s_goff, p.n_inst, gi);
                const int32_t j = gi - s_goff[ki];
                int q = 0;
#pragma unroll
                for (int m = 1; m < kMaxPop; ++m) q += j >= F.ps[ki * 8 + m] ? 1 : 0;
                const InstCold& I = p.cold[ki];
                const unsigned long long b = pf ? F.pf_rs[2 * k] : I.row_start[j];
                const unsigned long long e = pf ? F.pf_rs[2 * k + 1] : I.row_start[j + 1];
                F.beg[k] = I.words + b;
                F.meta[k] = ((uint32_t)ki << 3) | (uint32_t)q;
                len[h] = (uint32_t)(e - b);
                if (count && blockIdx.x == 0) atomicAdd(&p.inst_counters[ki * 2 + 1], e - b);
            }
        }
        // exclusive prefix of the row lengths (block scan)
        const uint32_t v = len[0] + len[1];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) F.wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w0 = lane < kBWarps ? F.wsum[lane] : 0u;
            uint32_t z = w0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            if (lane < kBWarps) F.wsum[lane] = z - w0;
        }
        __syncthreads();
        const uint32_t excl = F.wsum[warp] + x - v;
        if ((uint32_t)tid * 2u < mc) F.pre[tid * 2] = excl;
        if ((uint32_t)tid * 2u + 1u < mc) F.pre[tid * 2 + 1] = excl + len[0];
        if (tid == kBThreads - 1) F.pre[mc] = excl + v;
        __syncthreads();
        const uint32_t W = F.pre[mc];
        // words: chunks of 32 kFlatUnroll per warp, interleaved over the SMs
        const uint32_t gw = (uint32_t)warp * gridDim.x + blockIdx.x;
        const uint32_t step_w = (uint32_t)kBWarps * gridDim.x * 32u * kFlatUnroll;
        for (uint32_t c0 = gw * 32u * kFlatUnroll; c0 < W; c0 += step_w) {
            uint32_t word[kFlatUnroll], meta[kFlatUnroll];
#pragma unroll
            for (int u = 0; u < kFlatUnroll; ++u) {
                const uint32_t w = c0 + (uint32_t)u * 32u + (uint32_t)lane;
                word[u] = 0u;
                meta[u] = 0xffffffffu;
                if (w < W) {
                    uint32_t lo = 0u, hi = mc;          // pre[lo] <= w < pre[hi]
                    while (hi - lo > 1u) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (F.pre[mid] <= w) lo = mid;
                        else hi = mid;
                    }
                    word[u] = __ldg(F.beg[lo] + (w - F.pre[lo]));
                    meta[u] = F.meta[lo];
                }
            }
#pragma unroll
            for (int u = 0; u < kFlatUnroll; ++u) {
                if (meta[u] != 0xffffffffu) {
                    const int ki = (int)(meta[u] >> 3), q = (int)(meta[u] & 7u);
                    const int32_t tgt = (int32_t)(word[u] & kTgtMask);
                    int pp = 0;
#pragma unroll
                    for (int m = 1; m < kMaxPop; ++m) pp += tgt >= F.ps[ki * 8 + m] ? 1 : 0;
                    const int32_t wt = __ldg(&p.wtab_all[(((size_t)ki * kMaxPop + pp) * kMaxPop + q) *
                                                         kWCodes + (word[u] >> 25)]);
                    const uint32_t slot = ring_slot(tD, (word[u] >> kTgtBits) & 63u, (uint32_t)p.ring_depth);
                    atomicAdd(&p.ring[(size_t)slot * ntot + s_goff[ki] + tgt], wt);
                }
            }
        }
        __syncthreads();
    }
}

template <int NPT>
__global__ void __launch_bounds__(kBThreads, 1) k_batch(const __grid_constant__ BatchParams p) {
    // dynamic shared memory: the cached background draws [NPT][4][kBThreads],
    // then the flat tiling's arrays
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_rnd = reinterpret_cast<uint32_t*>(s_dyn);
    const FlatSmem F = flat_smem(s_dyn + (size_t)NPT * 4 * kBThreads * sizeof(uint32_t), p.n_inst);
    __shared__ int32_t s_goff[kMaxInst + 1];
    __shared__ volatile uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int k = tid; k <= p.n_inst; k += kBThreads) s_goff[k] = p.goff[k];
    flat_load_ps(p, F);
    if (tid == 0) s_abort = 0u;
    __syncthreads();
    const int32_t gbase = (int32_t)blockIdx.x * p.chunk + tid;
    const long long t0 = *p.step;
    const int n = p.n_steps;
    const size_t ntot = (size_t)p.ntot;

    float u[NPT], isyn[NPT];
    int32_t refr[NPT], ip[NPT];                     // ip = instance << 3 | population
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int32_t gi = gbase + k * kBThreads;
        u[k] = 0.f; isyn[k] = 0.f; refr[k] = 0; ip[k] = -1;
        if (k * kBThreads + tid < p.chunk && gi < p.ntot) {
            u[k] = p.u[gi];
            isyn[k] = p.i_syn[gi];
            refr[k] = p.refr[gi];
            const int ki = inst_of(s_goff, p.n_inst, gi);
            const InstCold& I = p.cold[ki];
            ip[k] = (ki << 3) | pop_index(I.pop_start, I.n_pop, gi - I.goff);
        }
    }
    // per-thread cache of the constants of the last instance seen
    int cinst = -1;
    float4 pf = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 pm = make_int4(0, 0, 0, 0);
    uint4 pk = make_uint4(0u, 0u, 0u, 0u);
    auto fetch = [&](int ki) {
        if (ki != cinst) {
            cinst = ki;
            pf = p.hot[ki].prop;
            pm = p.hot[ki].misc;
            pk = p.hot[ki].key;
        }
    };

    // A(t): membrane, threshold, reset, refractory; spikes into the lists
    auto phase_a = [&](long long t) {
        const uint32_t par4 = (uint32_t)(t & 3), par2 = (uint32_t)(t & 1);
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int32_t gi = gbase + k * kBThreads;
            bool spk = false;
            int tiling = 0;
            if (ip[k] >= 0) {
                fetch(ip[k] >> 3);
                if (refr[k] > 0) {
                    refr[k] -= 1;
                    u[k] = 0.f;
                } else {
                    float v = __fadd_rn(__fmul_rn(pf.x, u[k]), __fmul_rn(pf.y, isyn[k]));
                    if (pm.y == 1) v = __fadd_rn(v, __ldg(&p.cdc[ip[k]]));
                    u[k] = v;
                }
                if (u[k] > pf.w) {
                    spk = true;
                    u[k] = 0.f;
                    refr[k] = pm.x;
                }
                tiling = (int)pk.z;
            }
            const unsigned m = __ballot_sync(0xffffffffu, spk);
            if (m) {
                unsigned mt[kTilings];
                mt[1] = __ballot_sync(0xffffffffu, spk && tiling == 1);
                mt[2] = __ballot_sync(0xffffffffu, spk && tiling == 2);
                mt[0] = m & ~mt[1] & ~mt[2];
                uint32_t bt[kTilings] = {0u, 0u, 0u}, br = 0;
                if (lane == 0) {
#pragma unroll
                    for (int tl = 0; tl < kTilings; ++tl)
                        if (mt[tl]) bt[tl] = atomicAdd(&p.cnt[par4 * kTilings + tl], (uint32_t)__popc(mt[tl]));
                    br = atomicAdd(p.ras_n, (uint32_t)__popc(m));
                }
#pragma unroll
                for (int tl = 0; tl < kTilings; ++tl) bt[tl] = __shfl_sync(0xffffffffu, bt[tl], 0);
                br = __shfl_sync(0xffffffffu, br, 0);
                if (spk) {
                    const unsigned lt = (1u << lane) - 1u;
                    const uint32_t pos = (tiling == 0 ? bt[0] : tiling == 1 ? bt[1] : bt[2]) +
                                         (uint32_t)__popc((tiling == 0 ? mt[0] : tiling == 1 ? mt[1] : mt[2]) & lt);
                    p.list[((size_t)par2 * kTilings + (uint32_t)tiling) * ntot + pos] = (uint32_t)gi;
                    const uint32_t rp = br + (uint32_t)__popc(m & lt);
                    if (rp < p.ras_cap) {
                        p.ras_step[rp] = (uint32_t)t;
                        p.ras_id[rp] = (uint32_t)gi;
                    } else {
                        atomicOr(p.status, kBatchRasterOverflow);
                    }
                    atomicAdd(&p.inst_counters[(ip[k] >> 3) * 2], 1ull);
                }
            }
        }
    };

    if (n > 0) phase_a(t0);
    uint32_t gen = 0;
    for (int s = 0; s < n; ++s) {
        const long long t = t0 + s;
        const uint32_t tD = (uint32_t)(t % p.ring_depth);
        if (!grid_sync(p, gen, &s_abort)) break;
        // counters of step t + 2: last read in D(t - 2), next written in A(t + 2)
        if (blockIdx.x == 0 && tid < kTilings) p.cnt[(uint32_t)((t + 2) & 3) * kTilings + tid] = 0u;
        // D(t)'s flat list, fetched while C(t) and A(t + 1) run: its length
        // and the first kFlatChunk ids now (past the length: unused), the
        // rows' bounds after C(t)
        const uint32_t* lf_t = p.list + ((size_t)(t & 1) * kTilings + 2) * ntot;
        {
            const uint32_t lim = (uint32_t)min((size_t)kFlatChunk, ntot);
            if (tid == 0) cp_async4(F.pf_nf, &p.cnt[(uint32_t)(t & 3) * kTilings + 2]);
            for (uint32_t k = tid; k < lim; k += kBThreads) cp_async4(&F.pf_ids[k], &lf_t[k]);
        }

        // ---- C(t): ring slot t, background, synaptic current ----
        {
            int32_t* rs = p.ring + (size_t)tD * ntot;
            int32_t acc[NPT];
#pragma unroll
            for (int k = 0; k < NPT; ++k)
                acc[k] = ip[k] >= 0 ? __ldcg(&rs[gbase + k * kBThreads]) : 0;
#pragma unroll
            for (int k = 0; k < NPT; ++k)
                if (ip[k] >= 0) __stcg(&rs[gbase + k * kBThreads], 0);
            const bool refresh = (t & 3) == 0 || s == 0;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                if (ip[k] < 0) continue;
                fetch(ip[k] >> 3);
                if (pm.y == 0) {
                    uint32_t* rr = s_rnd + (k * 4) * kBThreads + tid;
                    if (refresh) {
                        const uint32_t li = (uint32_t)(gbase + k * kBThreads - pm.w);
                        const uint4 r = philox(make_uint4(li, (uint32_t)(t >> 2), kStreamPois,
                                                          (uint32_t)(t >> 34)), pk.x, pk.y);
                        rr[0] = r.x;
                        rr[kBThreads] = r.y;
                        rr[2 * kBThreads] = r.z;
                        rr[3 * kBThreads] = r.w;
                    }
                    const uint32_t x = rr[(int)(t & 3) * kBThreads];
                    // k = #{m : x >= T_m} = #{m : x > T_m - 1}; thresholds
                    // ascend, so the tail beyond 12 matters only if all 12 pass
                    const uint4* th = reinterpret_cast<const uint4*>(p.pois) + (size_t)ip[k] * (kPoisTable / 4);
                    const uint4 a0 = __ldg(&th[0]), a1 = __ldg(&th[1]), a2 = __ldg(&th[2]);
                    int kk = (x > a0.x) + (x > a0.y) + (x > a0.z) + (x > a0.w) +
                             (x > a1.x) + (x > a1.y) + (x > a1.z) + (x > a1.w) +
                             (x > a2.x) + (x > a2.y) + (x > a2.z) + (x > a2.w);
                    if (kk == 12) {
                        const uint32_t* tt = p.pois + (size_t)ip[k] * kPoisTable;
                        for (int mm = 12; mm < kPoisTable; ++mm) kk += x > __ldg(&tt[mm]) ? 1 : 0;
                    }
                    acc[k] += kk * pm.z;
                }
                isyn[k] = __fadd_rn(__fmul_rn(pf.z, isyn[k]),
                                    __fmul_rn(__int2float_rn(acc[k]), 0.00390625f));
            }
        }
        cp_async_wait();
        __syncthreads();
        const uint32_t nf_pf = min(*F.pf_nf, (uint32_t)kFlatChunk);
        for (uint32_t k = tid; k < nf_pf; k += kBThreads) {
            const int32_t gi = (int32_t)F.pf_ids[k];
            const int ki = inst_of(s_goff, p.n_inst, gi);
            const unsigned long long* rs = F.rsp[ki] + (gi - s_goff[ki]);
            cp_async8(&F.pf_rs[2 * k], rs);
            cp_async8(&F.pf_rs[2 * k + 1], rs + 1);
        }
        // ---- A(t + 1) ----
        if (s + 1 < n) phase_a(t + 1);
        cp_async_wait();
        __syncthreads();
        // ---- D(t): spikes of step t ----
        {
            const uint32_t par4 = (uint32_t)(t & 3), par2 = (uint32_t)(t & 1);
            const uint32_t nw = __ldcg(&p.cnt[par4 * kTilings + 0]);
            const uint32_t nb = __ldcg(&p.cnt[par4 * kTilings + 1]);
            const uint32_t nf = __ldcg(&p.cnt[par4 * kTilings + 2]);
            const uint32_t* lw = p.list + ((size_t)par2 * kTilings + 0) * ntot;
            const uint32_t* lb = p.list + ((size_t)par2 * kTilings + 1) * ntot;
            const uint32_t* lf = p.list + ((size_t)par2 * kTilings + 2) * ntot;
            if (nf) deliver_flat(p, s_goff, F, lf, nf, tD, true, true);
            // warp w of CTA b takes spikes w * grid + b, spreading them over SMs
            for (uint32_t k = (uint32_t)(tid >> 5) * gridDim.x + blockIdx.x; k < nw;
                 k += (uint32_t)kBWarps * gridDim.x)
                deliver_row<kWarpUnroll>(p, s_goff, (int32_t)__ldcg(&lw[k]), tD, lane, 32, true);
            // CTA rows start from the last CTA, away from the first warp rows
            for (uint32_t k = gridDim.x - 1u - blockIdx.x; k < nb; k += gridDim.x)
                deliver_row<kBlockUnroll>(p, s_goff, (int32_t)__ldcg(&lb[k]), tD, tid, kBThreads, true);
        }
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int32_t gi = gbase + k * kBThreads;
        if (ip[k] >= 0) {
            p.u[gi] = u[k];
            p.i_syn[gi] = isyn[k];
            p.refr[gi] = refr[k];
        }
    }
    if (blockIdx.x == 0 && tid == 0 && s_abort == 0u) *p.step = t0 + n;
}

// autotuner probe: deliver `n` spikes (global ids) with one tiling at step 0
__global__ void __launch_bounds__(kBThreads) k_probe_deliver(const __grid_constant__ BatchParams p,
                                                             const uint32_t* spikes, int n,
                                                             int tiling) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const FlatSmem F = flat_smem(s_dyn, p.n_inst);
    __shared__ int32_t s_goff[kMaxInst + 1];
    for (int k = threadIdx.x; k <= p.n_inst; k += kBThreads) s_goff[k] = p.goff[k];
    flat_load_ps(p, F);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (tiling == 2) {
        deliver_flat(p, s_goff, F, spikes, (uint32_t)n, 0, false);
    } else if (tiling == 0) {
        const int warps = (int)gridDim.x * kBWarps;
        for (int k = (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x; k < n; k += warps)
            deliver_row<kWarpUnroll>(p, s_goff, (int32_t)spikes[k], 0, lane, 32, false);
    } else {
        for (int k = blockIdx.x; k < n; k += gridDim.x)
            deliver_row<kBlockUnroll>(p, s_goff, (int32_t)spikes[k], 0, threadIdx.x, kBThreads, false);
    }
}

constexpr int kNptVariants[] = {1, 2, 4, 6, 8, 12, 16};

template <int NPT>
const void* batch_fn() { return reinterpret_cast<const void*>(&k_batch<NPT>); }

const void* select_batch(int npt) {
    switch (npt) {
        case 1: return batch_fn<1>();
        case 2: return batch_fn<2>();
        case 4: return batch_fn<4>();
        case 6: return batch_fn<6>();
        case 8: return batch_fn<8>();
        case 12: return batch_fn<12>();
        case 16: return batch_fn<16>();
        default: return nullptr;
    }
}

size_t batch_smem(int npt, int n_inst) {
    return (size_t)npt * 4 * kBThreads * sizeof(uint32_t) + flat_smem_bytes(n_inst);
}

}  // namespace
}  // namespace snn

using namespace snn;

struct snn_batch {
    int n_inst = 0;
    int ntot = 0;
    int npt = 0;
    int blocks = 0;
    int ring_depth = 2;                  // ring slots: the longest delay of any instance + 1
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    std::vector<int32_t> goff;
    std::vector<InstHot> hot_h;
    std::vector<InstCold> cold_h;
    std::vector<uint64_t> nnz;
    std::vector<float> tune_us[kTilings];
    std::vector<unsigned long long*> row_start;
    std::vector<uint32_t*> words;
    int32_t* d_wtab_all = nullptr;       // [n_inst][8][8][128]
    int32_t* d_ps_all = nullptr;         // [n_inst][8]
    BatchParams p;
    InstHot* d_hot = nullptr;
    InstCold* d_cold = nullptr;
    uint32_t* d_pois = nullptr;
    float* d_cdc = nullptr;
    int32_t* d_goff = nullptr;
    float* d_u = nullptr;
    float* d_i = nullptr;
    int32_t* d_r = nullptr;
    int32_t* d_ring = nullptr;
    uint32_t* d_list = nullptr;
    uint32_t* d_cnt = nullptr;
    uint32_t* d_ras_step = nullptr;
    uint32_t* d_ras_id = nullptr;
    uint32_t* d_ras_n = nullptr;
    uint32_t ras_cap = 0;
    unsigned long long* d_ic = nullptr;
    long long* d_step = nullptr;
    uint32_t* d_sync = nullptr;          // [0] barrier, [1] status, [2] abort
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = false;
    long long step = 0;
    std::vector<std::vector<uint32_t>> host_steps, host_ids;   // drained raster per instance
    std::vector<uint16_t> inst_of;  // instance of every global neuron id (built on the first drain)
    std::vector<float2> u0_range;        // default initial potentials per instance
    float trial_us = 0.f;                // per-step time of the chosen assignment
};

namespace {

template <typename T>
int balloc(T** p, size_t n, const char* what) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(SNN_ERR_OOM, what);
    }
    return SNN_OK;
}

#define BCALL(x)                           \
    do {                                   \
        int rc_ = (x);                     \
        if (rc_ != SNN_OK) return rc_;     \
    } while (0)
#define BCK(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return set_cuda_error(e_, #call);    \
    } while (0)

void free_batch(snn_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto* x : b->row_start) cudaFree(x);
    for (auto* x : b->words) cudaFree(x);
    void* ptrs[] = {b->d_wtab_all, b->d_ps_all, b->d_hot, b->d_cold, b->d_pois, b->d_cdc, b->d_goff, b->d_u, b->d_i,
                    b->d_r, b->d_ring, b->d_list, b->d_cnt, b->d_ras_step, b->d_ras_id,
                    b->d_ras_n, b->d_ic, b->d_step, b->d_sync};
    for (void* x : ptrs)
        if (x) cudaFree(x);
    delete b;
}

cudaError_t launch_batch(snn_batch* b, int n_steps) {
    BatchParams p = b->p;
    p.n_steps = n_steps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->blocks);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {&p};
    cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync + 2, 0, sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = cudaLaunchKernelExC(&cfg, select_batch(b->npt), args);
    return e;
}

// time both tilings on each instance's own rows; keep the faster
int autotune(snn_batch* b) {
    cudaStream_t s = b->stream;
    constexpr int kMaxProbe = 1 << 14;
    uint32_t* d_spk = nullptr;
    BCALL(balloc(&d_spk, kMaxProbe, "autotune spikes"));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int tl = 0; tl < kTilings; ++tl) b->tune_us[tl].assign(b->n_inst, 0.f);
    const size_t probe_smem = flat_smem_bytes(b->n_inst);
    for (int k = 0; k < b->n_inst && e == cudaSuccess; ++k) {
        const InstCold& I = b->cold_h[k];
        // about 5 Hz of activity in one 0.1 ms step, at least 4 spikes
        const int n = std::min(kMaxProbe, std::max(4, (int)(I.n * 5e-4 + 0.5)));
        std::vector<uint32_t> spk(n);
        uint64_t x = 0x9E3779B97F4A7C15ull * (uint64_t)(k + 1);
        for (int i = 0; i < n; ++i) {
            x ^= x >> 12;
            x ^= x << 25;
            x ^= x >> 27;
            spk[i] = (uint32_t)(I.goff + (int)((x * 0x2545F4914F6CDD1Dull) % (uint64_t)I.n));
        }
        e = cudaMemcpyAsync(d_spk, spk.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s);
        for (int tl = 0; tl < kTilings && e == cudaSuccess; ++tl) {
            const int grid = tl == 0   ? std::min(b->blocks, std::max(1, (n + kBWarps - 1) / kBWarps))
                             : tl == 1 ? std::min(b->blocks, n)
                                       : b->blocks;
            float best = 1e30f;
            for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, s);
                k_probe_deliver<<<grid, kBThreads, probe_smem, s>>>(b->p, d_spk, n, tl);
                cudaEventRecord(e1, s);
                e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best = std::min(best, ms);
            }
            b->tune_us[tl][k] = best * 1000.f;
        }
        uint32_t best_tl = 0;
        for (int tl = 1; tl < kTilings; ++tl)
            if (b->tune_us[tl][k] < b->tune_us[best_tl][k]) best_tl = (uint32_t)tl;
        b->hot_h[k].key.z = best_tl;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_spk);
    if (e != cudaSuccess) return set_cuda_error(e, "autotune");
    // the probes added into the ring: clear it again
    BCK(cudaMemsetAsync(b->d_ring, 0, sizeof(int32_t) * (size_t)b->ring_depth * b->ntot, s));
    BCK(cudaMemcpyAsync(b->d_hot, b->hot_h.data(), sizeof(InstHot) * b->n_inst,
                        cudaMemcpyHostToDevice, s));
    BCK(cudaStreamSynchronize(s));
    return SNN_OK;
}

// every instance back to its initial state (after the autotuner's trials)
cudaError_t reset_state(snn_batch* b) {
    cudaStream_t s = b->stream;
    const size_t ntot = (size_t)b->ntot;
    cudaError_t e = cudaMemsetAsync(b->d_i, 0, sizeof(float) * ntot, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_r, 0, sizeof(int32_t) * ntot, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ring, 0, sizeof(int32_t) * (size_t)b->ring_depth * ntot, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cnt, 0, sizeof(uint32_t) * 4 * kTilings, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ras_n, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ic, 0, sizeof(unsigned long long) * 2 * b->n_inst, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_step, 0, sizeof(long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, sizeof(uint32_t) * 4, s);
    for (int k = 0; k < b->n_inst && e == cudaSuccess; ++k) {
        const InstHot& H = b->hot_h[k];
        e = launch_init_state((int)H.key.w, H.key.x, H.key.y, b->u0_range[k].x, b->u0_range[k].y,
                              b->d_u + H.misc.w, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

// Batch-level trials: the persistent kernel itself, 100 + 300 steps, under
// candidate tiling assignments (the per-instance probe choice, each tiling for
// every instance, and the smaller / larger half of the instances on two
// different tilings); the fastest is kept.  The probes time each instance
// alone, while in the batch all instances' spikes share the grid, so the
// trials decide.  The state is reset to the initial state afterwards.
int batch_trials(snn_batch* b) {
    cudaStream_t s = b->stream;
    const int K = b->n_inst;
    std::vector<std::vector<uint32_t>> cand;
    std::vector<uint32_t> probe(K);
    for (int k = 0; k < K; ++k) probe[k] = b->hot_h[k].key.z;
    cand.push_back(probe);
    for (uint32_t tl = 0; tl < (uint32_t)kTilings; ++tl) cand.push_back(std::vector<uint32_t>(K, tl));
    if (K > 1) {
        std::vector<int> order(K);
        for (int k = 0; k < K; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int c) { return b->cold_h[a].n < b->cold_h[c].n; });
        for (uint32_t x = 0; x < (uint32_t)kTilings; ++x)
            for (uint32_t y = 0; y < (uint32_t)kTilings; ++y) {
                if (x == y) continue;
                std::vector<uint32_t> a(K);
                for (int r = 0; r < K; ++r) a[order[r]] = r < K / 2 ? x : y;
                cand.push_back(a);
            }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    float best = 1e30f;
    size_t best_c = 0;
    cudaError_t e = cudaSuccess;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c) {
        for (int k = 0; k < K; ++k) b->hot_h[k].key.z = cand[c][k];
        e = cudaMemcpyAsync(b->d_hot, b->hot_h.data(), sizeof(InstHot) * K, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = reset_state(b);
        if (e == cudaSuccess) e = launch_batch(b, 100);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_batch(b, 300);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
            best = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_cuda_error(e, "batch autotune trials");
    uint32_t st = 0;
    BCK(cudaMemcpy(&st, b->d_sync + 1, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) return set_error(SNN_ERR_TIMEOUT, "a grid-barrier wait timed out");
    for (int k = 0; k < K; ++k) b->hot_h[k].key.z = cand[best_c][k];
    b->trial_us = best * 1000.f / 300.f;
    BCK(cudaMemcpyAsync(b->d_hot, b->hot_h.data(), sizeof(InstHot) * K, cudaMemcpyHostToDevice, s));
    BCK(reset_state(b));
    return SNN_OK;
}

int drain_raster(snn_batch* b) {
    BCK(cudaStreamSynchronize(b->stream));
    uint32_t n = 0;
    BCK(cudaMemcpy(&n, b->d_ras_n, sizeof(n), cudaMemcpyDeviceToHost));
    const uint32_t m = std::min(n, b->ras_cap);
    std::vector<uint32_t> st(m), id(m);
    if (m) {
        BCK(cudaMemcpy(st.data(), b->d_ras_step, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
        BCK(cudaMemcpy(id.data(), b->d_ras_id, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
    }
    BCK(cudaMemset(b->d_ras_n, 0, sizeof(uint32_t)));
    if (b->inst_of.empty()) {
        b->inst_of.resize((size_t)b->ntot);
        for (int k = 0; k < b->n_inst; ++k)
            std::fill(b->inst_of.begin() + b->goff[k], b->inst_of.begin() + b->goff[k + 1],
                      (uint16_t)k);
    }
    // per-instance counts first, so that each instance's buffers grow once
    std::vector<uint32_t> cnt((size_t)b->n_inst, 0u);
    for (uint32_t r = 0; r < m; ++r) ++cnt[b->inst_of[id[r]]];
    for (int k = 0; k < b->n_inst; ++k) {
        b->host_steps[k].reserve(b->host_steps[k].size() + cnt[k]);
        b->host_ids[k].reserve(b->host_ids[k].size() + cnt[k]);
    }
    for (uint32_t r = 0; r < m; ++r) {
        const int k = b->inst_of[id[r]];
        b->host_steps[k].push_back(st[r]);
        b->host_ids[k].push_back(id[r] - (uint32_t)b->goff[k]);
    }
    if (n > b->ras_cap) return set_error(SNN_ERR_OVERFLOW, "batch raster capacity exceeded");
    return SNN_OK;
}

}  // namespace

extern "C" {

int snn_batch_create(const snn_config* cfgs, const uint64_t* seeds, int32_t n_inst,
                     const snn_options* opt, void* stream, snn_batch** out) {
    if (!cfgs || !seeds || !out || n_inst < 1 || n_inst > kMaxInst)
        return set_error(SNN_ERR_INVALID, "need 1..1024 configurations, seeds and out");
    *out = nullptr;
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    BCK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return set_error(SNN_ERR_UNSUPPORTED, "this library is built for sm_103 (GB300) GPUs only");
    snn_batch* b = new snn_batch();
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t s = b->stream;
    b->n_inst = n_inst;
    b->goff.assign(n_inst + 1, 0);
    b->hot_h.resize(n_inst);
    b->cold_h.resize(n_inst);
    b->nnz.resize(n_inst);
    b->host_steps.resize(n_inst);
    b->host_ids.resize(n_inst);
    std::vector<uint32_t> pois((size_t)n_inst * kMaxPop * kPoisTable, 0xffffffffu);
    std::vector<float> cdc((size_t)n_inst * kMaxPop, 0.f);
    std::vector<int32_t> wtab_all((size_t)n_inst * kMaxPop * kMaxPop * kWCodes);
    std::vector<int32_t> ps_all((size_t)n_inst * 8);
    int rc = SNN_OK;
    long long ntot = 0;
    for (int k = 0; k < n_inst && rc == SNN_OK; ++k) {
        HostTables ht;
        rc = host_tables(&cfgs[k], &ht);
        if (rc != SNN_OK) break;
        b->ring_depth = std::max(b->ring_depth, (int)ht.max_delay + 1);
        InstHot& H = b->hot_h[k];
        InstCold& C = b->cold_h[k];
        std::memset(&H, 0, sizeof(H));
        std::memset(&C, 0, sizeof(C));
        H.prop = make_float4(ht.prop[0], ht.prop[1], ht.prop[2], ht.theta);
        H.misc = make_int4(ht.n_ref, ht.mode, ht.wext_q, (int32_t)ntot);
        H.key = make_uint4((uint32_t)(seeds[k] & 0xffffffffu), (uint32_t)(seeds[k] >> 32), 0u,
                           (uint32_t)ht.n);
        for (int q = 0; q <= kMaxPop; ++q) C.pop_start[q] = ht.pop_start[q];
        C.n_pop = ht.n_pop;
        C.goff = (int32_t)ntot;
        C.n = ht.n;
        for (int q = 0; q < kMaxPop; ++q) {
            cdc[(size_t)k * kMaxPop + q] = ht.cdc[q];
            for (int m = 0; m < kPoisTable; ++m)
                pois[((size_t)k * kMaxPop + q) * kPoisTable + m] = (uint32_t)(ht.pois[q][m] - 1u);
        }
        unsigned long long* rs = nullptr;
        uint32_t* wd = nullptr;
        uint64_t nnz = 0;
        rc = build_rows_device(&cfgs[k], seeds[k], s, &rs, &wd, &nnz);
        if (rc != SNN_OK) break;
        b->row_start.push_back(rs);
        b->words.push_back(wd);
        b->nnz[k] = nnz;
        // the batch kernel adds in plain int32: refuse an instance whose input
        // of one step could leave that range (snn_create counts wrap-arounds
        // for such networks instead)
        {
            uint32_t* d_in = nullptr;
            std::vector<uint32_t> indeg((size_t)ht.n * kMaxPop);
            cudaError_t e = cudaMalloc(&d_in, sizeof(uint32_t) * std::max<size_t>(indeg.size(), 1));
            if (e == cudaSuccess) e = launch_indegree(rs, wd, ht.n, ht.n_pop, ht.pop_start, d_in, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(indeg.data(), d_in, sizeof(uint32_t) * indeg.size(),
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (d_in) cudaFree(d_in);
            if (e != cudaSuccess) {
                rc = set_cuda_error(e, "in-degrees of a batch instance");
                break;
            }
            if (input_bound(indeg.data(), ht.n, ht.n_pop, ht.pop_start, ht.wtab, ht.wext_q,
                            ht.mode) > 2147483647ll) {
                rc = set_error(SNN_ERR_SATURATED,
                               "a batch instance's input of one step can exceed the int32 "
                               "fixed-point range; step it as a single network (snn_create), "
                               "which checks for saturation");
                break;
            }
        }
        std::memcpy(wtab_all.data() + (size_t)k * kMaxPop * kMaxPop * kWCodes, ht.wtab, sizeof(ht.wtab));
        for (int m = 0; m < 8; ++m)
            ps_all[(size_t)k * 8 + m] = m == 0 ? 0 : (m < ht.n_pop ? ht.pop_start[m] : 0x7fffffff);
        C.row_start = rs;
        C.words = wd;
        b->u0_range.push_back(make_float2((float)cfgs[k].u0_lo, (float)cfgs[k].u0_hi));
        ntot += ht.n;
        b->goff[k + 1] = (int32_t)ntot;
        if (ntot > (1ll << 30)) rc = set_error(SNN_ERR_INVALID, "too many neurons in the batch");
    }
    if (rc == SNN_OK) rc = balloc(&b->d_wtab_all, wtab_all.size(), "batch weight tables");
    if (rc == SNN_OK) rc = balloc(&b->d_ps_all, ps_all.size(), "batch population starts");
    if (rc == SNN_OK) {
        const cudaError_t ce = cudaMemcpy(b->d_wtab_all, wtab_all.data(), sizeof(int32_t) * wtab_all.size(),
                                          cudaMemcpyHostToDevice);
        const cudaError_t ce2 = cudaMemcpy(b->d_ps_all, ps_all.data(), sizeof(int32_t) * ps_all.size(),
                                           cudaMemcpyHostToDevice);
        if (ce != cudaSuccess || ce2 != cudaSuccess) rc = set_error(SNN_ERR_CUDA, "table upload");
    }
    if (rc != SNN_OK) {
        free_batch(b);
        return rc;
    }
    for (int k = 0; k < n_inst; ++k)
        b->cold_h[k].wtab = b->d_wtab_all + (size_t)k * kMaxPop * kMaxPop * kWCodes;
    b->ntot = (int)ntot;
    // launch shape: one CTA per SM, the fewest neurons per thread that cover the batch
    b->blocks = prop.multiProcessorCount;
    b->npt = 0;
    for (int npt : kNptVariants) {
        if ((long long)npt * kBThreads * b->blocks < ntot) continue;
        const size_t smem = batch_smem(npt, n_inst);
        if (cudaFuncSetAttribute(select_batch(npt), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            break;
        int ps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, select_batch(npt), kBThreads, smem) !=
                cudaSuccess ||
            ps < 1)
            break;
        b->npt = npt;
        b->smem = smem;
        break;
    }
    cudaGetLastError();
    if (b->npt == 0) {
        free_batch(b);
        return set_error(SNN_ERR_UNSUPPORTED, "batch too large for one co-resident grid");
    }
    const long long cap = (opt && opt->raster_capacity > 0) ? opt->raster_capacity : (64ll << 20);
    b->ras_cap = (uint32_t)std::min<long long>(cap, 0x7fffffff);
    if (rc == SNN_OK) rc = balloc(&b->d_hot, n_inst, "batch instance constants");
    if (rc == SNN_OK) rc = balloc(&b->d_cold, n_inst, "batch instance rows");
    if (rc == SNN_OK) rc = balloc(&b->d_pois, pois.size(), "batch background tables");
    if (rc == SNN_OK) rc = balloc(&b->d_cdc, cdc.size(), "batch DC input");
    if (rc == SNN_OK) rc = balloc(&b->d_goff, n_inst + 1, "batch offsets");
    if (rc == SNN_OK) rc = balloc(&b->d_u, ntot, "batch u");
    if (rc == SNN_OK) rc = balloc(&b->d_i, ntot, "batch I");
    if (rc == SNN_OK) rc = balloc(&b->d_r, ntot, "batch refractory counters");
    if (rc == SNN_OK) rc = balloc(&b->d_ring, (size_t)b->ring_depth * ntot, "batch ring buffers");
    if (rc == SNN_OK) rc = balloc(&b->d_list, (size_t)2 * kTilings * ntot, "batch spike lists");
    if (rc == SNN_OK) rc = balloc(&b->d_cnt, 4 * kTilings, "batch list counters");
    if (rc == SNN_OK) rc = balloc(&b->d_ras_step, b->ras_cap, "batch raster");
    if (rc == SNN_OK) rc = balloc(&b->d_ras_id, b->ras_cap, "batch raster");
    if (rc == SNN_OK) rc = balloc(&b->d_ras_n, 1, "batch raster count");
    if (rc == SNN_OK) rc = balloc(&b->d_ic, (size_t)2 * n_inst, "batch counters");
    if (rc == SNN_OK) rc = balloc(&b->d_step, 1, "batch step");
    if (rc == SNN_OK) rc = balloc(&b->d_sync, 4, "batch barrier");
    if (rc != SNN_OK) {
        free_batch(b);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_goff, b->goff.data(), sizeof(int32_t) * (n_inst + 1),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_hot, b->hot_h.data(), sizeof(InstHot) * n_inst, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_cold, b->cold_h.data(), sizeof(InstCold) * n_inst, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_pois, pois.data(), sizeof(uint32_t) * pois.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_cdc, cdc.data(), sizeof(float) * cdc.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_i, 0, sizeof(float) * ntot, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_r, 0, sizeof(int32_t) * ntot, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ring, 0, sizeof(int32_t) * (size_t)b->ring_depth * ntot, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cnt, 0, sizeof(uint32_t) * 4 * kTilings, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ras_n, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ic, 0, sizeof(unsigned long long) * 2 * n_inst, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_step, 0, sizeof(long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, sizeof(uint32_t) * 4, s);
    for (int k = 0; k < n_inst && e == cudaSuccess; ++k) {
        const InstHot& H = b->hot_h[k];
        e = launch_init_state((int)H.key.w, H.key.x, H.key.y, (float)cfgs[k].u0_lo,
                              (float)cfgs[k].u0_hi, b->d_u + H.misc.w, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_batch(b);
        return set_cuda_error(e, "batch state initialisation");
    }
    BatchParams& p = b->p;
    std::memset(&p, 0, sizeof(p));
    p.n_inst = n_inst;
    p.ntot = b->ntot;
    p.ring_depth = b->ring_depth;
    p.chunk = (int32_t)(((long long)b->ntot + b->blocks - 1) / b->blocks);
    p.timeout_ns = (uint64_t)(((opt && opt->timeout_s > 0) ? opt->timeout_s : 2.0) * 1e9);
    p.inject_fault = opt ? opt->inject_fault : 0;
    p.hot = b->d_hot;
    p.cold = b->d_cold;
    p.pois = b->d_pois;
    p.cdc = b->d_cdc;
    p.goff = b->d_goff;
    p.wtab_all = b->d_wtab_all;
    p.ps_all = b->d_ps_all;
    p.u = b->d_u;
    p.i_syn = b->d_i;
    p.refr = b->d_r;
    p.ring = b->d_ring;
    p.list = b->d_list;
    p.cnt = b->d_cnt;
    p.ras_step = b->d_ras_step;
    p.ras_id = b->d_ras_id;
    p.ras_n = b->d_ras_n;
    p.ras_cap = b->ras_cap;
    p.inst_counters = b->d_ic;
    p.step = b->d_step;
    p.barrier = b->d_sync;
    p.status = b->d_sync + 1;
    p.abort_flag = b->d_sync + 2;
    if (cudaFuncSetAttribute(k_probe_deliver, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)flat_smem_bytes(n_inst)) != cudaSuccess) {
        free_batch(b);
        return set_error(SNN_ERR_CUDA, "probe kernel shared memory");
    }
    rc = autotune(b);
    if (rc == SNN_OK && !(opt && opt->inject_fault)) rc = batch_trials(b);
    if (rc != SNN_OK) {
        free_batch(b);
        return rc;
    }
    // capture one launch of kGraphChunk steps; replays advance the device
    // step counter, so no parameter changes between replays
    // (captured on a private stream: the legacy default stream cannot be
    // captured; the graph is then launched on the batch's own stream)
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    b->graph_ok = false;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            b->stream = cs;
            const cudaError_t le = launch_batch(b, kGraphChunk);
            b->stream = s;
            const cudaError_t ce = cudaStreamEndCapture(cs, &g);
            if (le == cudaSuccess && ce == cudaSuccess && g &&
                cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess)
                b->graph_ok = true;
            if (g) cudaGraphDestroy(g);
        }
        cudaStreamDestroy(cs);
    }
    cudaGetLastError();
    *out = b;
    return SNN_OK;
}

int snn_batch_step(snn_batch* b, int64_t n_steps) {
    if (!b || n_steps < 0) return set_error(SNN_ERR_INVALID, "bad arguments");
    int64_t left = n_steps;
    while (left > 0) {
        if (b->graph_ok && left >= kGraphChunk) {
            BCK(cudaGraphLaunch(b->graph, b->stream));
            left -= kGraphChunk;
            b->step += kGraphChunk;
        } else {
            const int chunk = (int)std::min<int64_t>(left, 1 << 20);
            BCK(launch_batch(b, chunk));
            left -= chunk;
            b->step += chunk;
        }
    }
    return SNN_OK;
}

int snn_batch_sync(snn_batch* b) {
    if (!b) return set_error(SNN_ERR_INVALID, "batch is NULL");
    BCK(cudaStreamSynchronize(b->stream));
    uint32_t st = 0;
    BCK(cudaMemcpy(&st, b->d_sync + 1, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) return set_error(SNN_ERR_TIMEOUT, "a grid-barrier wait timed out");
    if (st & kBatchRasterOverflow) return set_error(SNN_ERR_OVERFLOW, "batch raster capacity exceeded");
    return SNN_OK;
}

int snn_batch_read_spikes(snn_batch* b, int32_t k, uint32_t* steps_host, uint32_t* ids_host,
                          int64_t cap, int64_t* n) {
    if (!b || k < 0 || k >= b->n_inst || !n || cap < 0)
        return set_error(SNN_ERR_INVALID, "bad arguments");
    const int rc = drain_raster(b);
    auto& st = b->host_steps[k];
    auto& id = b->host_ids[k];
    const int64_t m = std::min<int64_t>(cap, (int64_t)st.size());
    if (m > 0) {
        if (steps_host) std::memcpy(steps_host, st.data(), sizeof(uint32_t) * m);
        if (ids_host) std::memcpy(ids_host, id.data(), sizeof(uint32_t) * m);
    }
    const bool short_cap = m < (int64_t)st.size();
    st.clear();
    id.clear();
    *n = m;
    if (rc != SNN_OK) return rc;
    if (short_cap) return set_error(SNN_ERR_OVERFLOW, "cap smaller than the recorded spikes");
    return SNN_OK;
}

int snn_batch_read_state(snn_batch* b, int32_t k, float* u_host, float* i_syn_host,
                         int32_t* refr_host) {
    if (!b || k < 0 || k >= b->n_inst) return set_error(SNN_ERR_INVALID, "bad arguments");
    BCK(cudaStreamSynchronize(b->stream));
    const InstCold& C = b->cold_h[k];
    if (u_host) BCK(cudaMemcpy(u_host, b->d_u + C.goff, sizeof(float) * C.n, cudaMemcpyDeviceToHost));
    if (i_syn_host)
        BCK(cudaMemcpy(i_syn_host, b->d_i + C.goff, sizeof(float) * C.n, cudaMemcpyDeviceToHost));
    if (refr_host)
        BCK(cudaMemcpy(refr_host, b->d_r + C.goff, sizeof(int32_t) * C.n, cudaMemcpyDeviceToHost));
    return SNN_OK;
}

int snn_batch_counters(snn_batch* b, int32_t k, int64_t* step, uint64_t* spikes, uint64_t* events) {
    if (!b || k < 0 || k >= b->n_inst) return set_error(SNN_ERR_INVALID, "bad arguments");
    BCK(cudaStreamSynchronize(b->stream));
    unsigned long long c[2];
    BCK(cudaMemcpy(c, b->d_ic + 2 * k, sizeof(c), cudaMemcpyDeviceToHost));
    if (step) *step = b->step;
    if (spikes) *spikes = c[0];
    if (events) *events = c[1];
    return SNN_OK;
}

int snn_batch_get_info(snn_batch* b, int32_t k, snn_batch_info* info) {
    if (!b || !info || k < 0 || k >= b->n_inst) return set_error(SNN_ERR_INVALID, "bad arguments");
    info->n_instances = b->n_inst;
    info->n_neurons_total = b->ntot;
    info->n_neurons = b->cold_h[k].n;
    info->n_synapses = (int64_t)b->nnz[k];
    info->tiling = (int32_t)b->hot_h[k].key.z;
    info->tune_us_warp = b->tune_us[0][k];
    info->tune_us_block = b->tune_us[1][k];
    info->tune_us_flat = b->tune_us[2][k];
    info->trial_us_per_step = b->trial_us;
    info->blocks = b->blocks;
    info->threads = kBThreads;
    info->neurons_per_thread = b->npt;
    info->graph = b->graph_ok ? 1 : 0;
    info->graph_steps = kGraphChunk;
    return SNN_OK;
}

int snn_batch_set_tiling(snn_batch* b, int32_t k, int32_t tiling) {
    if (!b || k < 0 || k >= b->n_inst || tiling < 0 || tiling >= kTilings)
        return set_error(SNN_ERR_INVALID, "bad arguments");
    b->hot_h[k].key.z = (uint32_t)tiling;
    BCK(cudaMemcpyAsync(b->d_hot + k, &b->hot_h[k], sizeof(InstHot), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return SNN_OK;
}

int snn_batch_destroy(snn_batch* b) {
    if (!b) return SNN_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return SNN_OK;
}

}  // extern "C"
