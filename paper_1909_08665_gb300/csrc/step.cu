// step.cu -- the time-stepped simulation on the device (Sec. 2.1 Eq. 1,
// Sec. 3.1.2 synaptic input buffers, Sec. 3.1.3 per-step processing).
//
// One persistent cooperative launch runs n steps.  CTA c owns the neuron
// range [part_lo[c], part_lo[c+1]): their state lives in registers and their
// 64-slot synaptic-input ring buffers live in shared memory (or in a
// partition-private global block when they do not fit).  Every synaptic row
// is stored with one segment per partition, so CTA c reads only the words
// that target its own neurons and adds them with shared-memory atomics.
//
// Per step t the order is:
//   A(t)  u_t from (u_{t-1}, I_{t-1}); threshold, reset, refractory; the
//         spikes of step t are compacted with warp ballots into the CTA's
//         spike list and raster; the CTA arrives at barrier slot t mod 4.
//   wait  barrier of step t-1 (all CTAs published their spikes of t-1).
//   D     deliver the spikes of step t-1 into ring slots t-1+d (d >= 1).
//   C(t)  acc = ring[t], cleared; Poisson count; I_t = P11 I_{t-1} + acc/256.
// A(t+1) needs only I_t, and the spikes of step t reach no input before
// slot t+1, so the spike exchange of one step overlaps the next step's
// membrane update: one grid-wide wait per step, whose latency is hidden
// behind A.  All results equal the sequential order of the method (integer
// accumulation, fp32 operations in a fixed order, no FMA contraction).
#include "snn_internal.cuh"

namespace snn {

constexpr int kWarps = kStepThreads / 32;
constexpr uint32_t kStatusRasterOverflow = 2u;

// ---------------------------------------------------------------------------
// shared-memory layout (bytes), identical on host and device
// ---------------------------------------------------------------------------
struct SmemLayout {
    uint32_t wtab, pois, warp, misc, cntoff, st, wo, q, pop, ring, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int ncmax, int n_part, bool smem_ring) {
    SmemLayout L;
    uint32_t o = 0;
    L.wtab = o;   o += kMaxPop * kMaxPop * kWCodes * 4;
    L.pois = o;   o += kMaxPop * kPoisTable * 8;
    L.warp = o;   o += 32 * 4;
    L.misc = o;   o += 32 * 4;
    L.cntoff = o; o = align_up(o + (uint32_t)(n_part + 1) * 4, 16);
    L.st = o;     o += kChunk * 4;
    L.wo = o;     o = align_up(o + (kChunk + 1) * 4, 16);
    L.q = o;      o = align_up(o + kChunk, 16);
    L.pop = o;    o = align_up(o + (uint32_t)ncmax, 16);
    L.ring = o;
    if (smem_ring) o += (uint32_t)kRing * (uint32_t)ncmax * 4;
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of ITEMS consecutive values per thread
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <int ITEMS>
__device__ __forceinline__ uint32_t block_scan(uint32_t (&v)[ITEMS], uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint32_t t = v[k];
        v[k] = local;
        local += t;
    }
    const uint32_t incl = warp_incl_scan(local);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? s_warp[lane] : 0u;
        w = warp_incl_scan(w);
        if (lane < kWarps) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = (warp ? s_warp[warp - 1] : 0u) + incl - local;
    const uint32_t total = s_warp[kWarps - 1];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) v[k] += excl;
    __syncthreads();
    return total;
}

// bounded wait until *ctr >= target (thread 0 only); false on timeout/abort
__device__ bool wait_geq(const StepParams& sp, const uint32_t* ctr, uint32_t target) {
    const uint64_t t_start = globaltimer_ns();
    uint32_t iter = 0;
    while (true) {
        if (ld_acquire_gpu(ctr) >= target) return true;
        if ((++iter & 255u) == 0u) {
            if (ld_relaxed_gpu(sp.abort_flag) != 0u) return false;
            if (globaltimer_ns() - t_start > sp.timeout_ns || iter > 0x7fffffffu) {
                atomicOr(sp.status, kStatusTimeout);
                atomicExch(sp.abort_flag, 1u);
                return false;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// delivery of the spike list `list` (spikes of step tb) into this CTA's ring
// ---------------------------------------------------------------------------
__device__ __forceinline__ void deliver_list(const StepParams& sp, unsigned char* smem,
                                             const SmemLayout& L, int c, int32_t lo, int list,
                                             int64_t tb, int32_t* ring,
                                             unsigned long long& events) {
    const int tid = threadIdx.x;
    const int P = sp.n_part;
    const int32_t* s_wtab = reinterpret_cast<const int32_t*>(smem + L.wtab);
    uint32_t* s_warp = reinterpret_cast<uint32_t*>(smem + L.warp);
    uint32_t* s_cntoff = reinterpret_cast<uint32_t*>(smem + L.cntoff);
    uint32_t* s_st = reinterpret_cast<uint32_t*>(smem + L.st);
    uint32_t* s_wo = reinterpret_cast<uint32_t*>(smem + L.wo);
    uint8_t* s_q = smem + L.q;
    const uint8_t* s_pop = smem + L.pop;

    // 1. spike counts of all partitions -> offsets
    uint32_t cnt[1] = {tid < P ? __ldcg(&sp.spk_cnt[list * P + tid]) : 0u};
    const uint32_t S = block_scan<1>(cnt, s_warp);
    if (tid < P) s_cntoff[tid] = cnt[0];
    if (tid == 0) s_cntoff[P] = S;
    __syncthreads();

    for (uint32_t base = 0; base < S; base += kChunk) {
        const int m = (int)min((uint32_t)kChunk, S - base);
        // 2. spike ids -> this partition's segment of each row
        uint32_t len[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int x = tid * 2 + k;
            len[k] = 0;
            if (x < m) {
                const uint32_t g = base + (uint32_t)x;
                int a = 0, b = P;                   // s_cntoff[a] <= g < s_cntoff[b]
                while (b - a > 1) {
                    const int mid = (a + b) >> 1;
                    if (s_cntoff[mid] <= g) a = mid;
                    else b = mid;
                }
                const uint32_t id = __ldcg(&sp.spk_ids[((size_t)list * P + a) * sp.ncmax +
                                                       (g - s_cntoff[a])]);
                const uint32_t* sg = sp.seg + (size_t)id * (size_t)(P + 1) + c;
                const uint32_t st = __ldg(sg);
                const uint32_t en = __ldg(sg + 1);
                s_st[x] = st;
                s_q[x] = (uint8_t)pop_index(sp.pop_start, sp.n_pop, (int32_t)id);
                len[k] = en - st;
            }
        }
        const uint32_t W = block_scan<2>(len, s_warp);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int x = tid * 2 + k;
            if (x < m) s_wo[x] = len[k];
        }
        if (tid == 0) s_wo[m] = W;
        __syncthreads();
        // 3. words of all segments, flattened over the CTA
        for (uint32_t w = tid; w < W; w += kStepThreads) {
            int a = 0, b = m;                       // s_wo[a] <= w < s_wo[b]
            while (b - a > 1) {
                const int mid = (a + b) >> 1;
                if (s_wo[mid] <= w) a = mid;
                else b = mid;
            }
            const uint32_t word = __ldg(&sp.words[s_st[a] + (w - s_wo[a])]);
            const int32_t local = (int32_t)(word & kTgtMask) - lo;
            const uint32_t d = (word >> kTgtBits) & 63u;
            const uint32_t code = word >> 25;
            const int p = s_pop[local];
            const int32_t wt = s_wtab[(p * kMaxPop + s_q[a]) * kWCodes + code];
            const uint32_t slot = (uint32_t)(tb + d) & (kRing - 1);
            atomicAdd(&ring[slot * (uint32_t)sp.ncmax + (uint32_t)local], wt);
        }
        if (tid == 0) events += W;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// persistent step kernel
// ---------------------------------------------------------------------------
template <int NPT, bool SMEM_RING>
__global__ void __launch_bounds__(kStepThreads, 1)
k_step(const __grid_constant__ StepParams sp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int c = blockIdx.x;
    const int P = sp.n_part;
    const SmemLayout L = smem_layout(sp.ncmax, P, SMEM_RING);
    int32_t* s_wtab = reinterpret_cast<int32_t*>(smem + L.wtab);
    uint64_t* s_pois = reinterpret_cast<uint64_t*>(smem + L.pois);
    uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + L.misc);
    uint8_t* s_pop = smem + L.pop;

    const int32_t lo = sp.part_lo[c];
    const int32_t nc = sp.part_lo[c + 1] - lo;
    int32_t* ring = SMEM_RING ? reinterpret_cast<int32_t*>(smem + L.ring)
                              : sp.ring + (size_t)c * kRing * (size_t)sp.ncmax;
    int32_t* ring_g = sp.ring + (size_t)c * kRing * (size_t)sp.ncmax;

    for (int k = tid; k < kMaxPop * kMaxPop * kWCodes; k += kStepThreads) s_wtab[k] = sp.wtab[k];
    for (int k = tid; k < kMaxPop * kPoisTable; k += kStepThreads)
        s_pois[k] = sp.pois[k / kPoisTable][k % kPoisTable];
    for (int k = tid; k < nc; k += kStepThreads) s_pop[k] = (uint8_t)pop_index(sp.pop_start, sp.n_pop, lo + k);
    if (SMEM_RING)
        for (int k = tid; k < kRing * sp.ncmax; k += kStepThreads) ring[k] = ring_g[k];
    if (tid < 32) s_misc[tid] = 0u;

    float u[NPT], isyn[NPT];
    int32_t refr[NPT];
    int pop[NPT];
    uint4 rnd[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int li = tid + k * kStepThreads;
        u[k] = 0.f; isyn[k] = 0.f; refr[k] = 0; pop[k] = 0;
        rnd[k] = make_uint4(0u, 0u, 0u, 0u);
        if (li < nc) {
            u[k] = sp.u[lo + li];
            isyn[k] = sp.i_syn[lo + li];
            refr[k] = sp.refr[lo + li];
            pop[k] = pop_index(sp.pop_start, sp.n_pop, lo + li);
        }
    }
    uint32_t ras_base = sp.ras_n[c];
    unsigned long long spikes = 0, events = 0;
    bool aborted = false;
    __syncthreads();

    for (int s = 0; s < sp.n_steps; ++s) {
        const int64_t t = sp.t0 + s;
        const int list = (int)(t & 3);
        uint32_t* my_cnt = &s_misc[s & 1];
        // ---- A(t): membrane, threshold, compaction ----
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int li = tid + k * kStepThreads;
            bool spk = false;
            if (li < nc) {
                if (refr[k] > 0) {
                    refr[k] -= 1;
                    u[k] = 0.f;
                } else {
                    float v = __fadd_rn(__fmul_rn(sp.P22, u[k]), __fmul_rn(sp.P21, isyn[k]));
                    if (sp.mode == 1) v = __fadd_rn(v, sp.cdc[pop[k]]);
                    u[k] = v;
                }
                if (u[k] > sp.theta) {
                    spk = true;
                    u[k] = 0.f;
                    refr[k] = sp.n_ref;
                }
            }
            const unsigned mask = __ballot_sync(0xffffffffu, spk);
            if (mask) {
                uint32_t wbase = 0;
                if (lane == 0) wbase = atomicAdd(my_cnt, (uint32_t)__popc(mask));
                wbase = __shfl_sync(0xffffffffu, wbase, 0);
                if (spk) {
                    const uint32_t pos = wbase + (uint32_t)__popc(mask & ((1u << lane) - 1u));
                    const uint32_t id = (uint32_t)(lo + li);
                    sp.spk_ids[((size_t)list * P + c) * sp.ncmax + pos] = id;
                    const uint32_t rp = ras_base + pos;
                    if (rp < sp.ras_cap) {
                        sp.ras_step[(size_t)c * sp.ras_cap + rp] = (uint32_t)t;
                        sp.ras_id[(size_t)c * sp.ras_cap + rp] = id;
                    }
                }
            }
        }
        __syncthreads();
        const uint32_t nsp = *my_cnt;
        if (tid == 0) {
            // counter of step s+1 (last used in step s-1): its readers are all
            // past a barrier; in step 0 it is still zero from the start and is
            // left alone (no barrier separates it from step 1's adds)
            if (s > 0) s_misc[(s + 1) & 1] = 0u;
            __stcg(&sp.spk_cnt[list * P + c], nsp);
            __threadfence();
            if (!(sp.inject_fault == 1 && c == 0)) red_release_gpu_add(&sp.barrier[s & 3], 1u);
            spikes += nsp;
            if (ras_base + nsp > sp.ras_cap) atomicOr(sp.status, kStatusRasterOverflow);
        }
        ras_base += nsp;
        // ---- wait for step t-1 and deliver its spikes ----
        if (s > 0) {
            if (tid == 0) {
                const uint32_t target = (uint32_t)P * (uint32_t)((s - 1) / 4 + 1);
                if (!wait_geq(sp, &sp.barrier[(s - 1) & 3], target)) s_misc[2] = 1u;
            }
            __syncthreads();
            if (s_misc[2]) { aborted = true; break; }
            deliver_list(sp, smem, L, c, lo, (int)((t - 1) & 3), t - 1, ring, events);
        }
        // ---- C(t): ring slot t, Poisson background, synaptic current ----
        const uint32_t slot = (uint32_t)t & (kRing - 1);
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int li = tid + k * kStepThreads;
            if (li < nc) {
                int32_t* rp = &ring[slot * (uint32_t)sp.ncmax + (uint32_t)li];
                int32_t acc = *rp;
                *rp = 0;
                if (sp.mode == 0) {
                    if ((t & 3) == 0 || s == 0)
                        rnd[k] = philox(make_uint4((uint32_t)(lo + li), (uint32_t)(t >> 2),
                                                   kStreamPois, (uint32_t)(t >> 34)),
                                        sp.key0, sp.key1);
                    const uint32_t x = lane_of(rnd[k], (int)(t & 3));
                    const uint64_t* thr = s_pois + pop[k] * kPoisTable;
                    int kk = 0;
                    while (kk < kPoisTable && (uint64_t)x >= thr[kk]) ++kk;
                    acc += kk * sp.wext_q;
                }
                isyn[k] = __fadd_rn(__fmul_rn(sp.P11, isyn[k]),
                                    __fmul_rn(__int2float_rn(acc), 0.00390625f));
            }
        }
    }

    // ---- epilogue: deliver the spikes of the last step ----
    if (!aborted && sp.n_steps > 0) {
        const int s = sp.n_steps;
        if (tid == 0) {
            const uint32_t target = (uint32_t)P * (uint32_t)((s - 1) / 4 + 1);
            if (!wait_geq(sp, &sp.barrier[(s - 1) & 3], target)) s_misc[2] = 1u;
        }
        __syncthreads();
        if (!s_misc[2]) {
            const int64_t tl = sp.t0 + s - 1;
            deliver_list(sp, smem, L, c, lo, (int)(tl & 3), tl, ring, events);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int li = tid + k * kStepThreads;
        if (li < nc) {
            sp.u[lo + li] = u[k];
            sp.i_syn[lo + li] = isyn[k];
            sp.refr[lo + li] = refr[k];
        }
    }
    if (SMEM_RING)
        for (int k = tid; k < kRing * sp.ncmax; k += kStepThreads) ring_g[k] = ring[k];
    if (tid == 0) {
        sp.ras_n[c] = ras_base;
        atomicAdd(&sp.counters[0], spikes);
        atomicAdd(&sp.counters[1], events);
    }
}

// ---------------------------------------------------------------------------
// standalone delivery of one spike list (global ring, partition layout)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void deliver_word(const DeliverParams& dp, uint32_t word, int q) {
    const int32_t tgt = (int32_t)(word & kTgtMask);
    // partition of tgt: largest c with floor(c n / P) <= tgt
    const int c = (int)(((long long)(tgt + 1) * dp.n_part - 1) / dp.n);
    const int32_t local = tgt - (int32_t)(((long long)c * dp.n) / dp.n_part);
    const uint32_t d = (word >> kTgtBits) & 63u;
    const int p = pop_index(dp.pop_start, dp.n_pop, tgt);
    const int32_t wt = __ldg(&dp.wtab[(p * kMaxPop + q) * kWCodes + (word >> 25)]);
    const uint32_t slot = (uint32_t)(dp.t + d) & (kRing - 1);
    atomicAdd(&dp.ring[((size_t)c * kRing + slot) * dp.ncmax + local], wt);
}

__global__ void __launch_bounds__(256) k_deliver_warp(const __grid_constant__ DeliverParams dp) {
    const int warp = (blockIdx.x * 256 + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= dp.n_spikes) return;
    const uint32_t j = __ldg(&dp.spikes[warp]);
    const int q = pop_index(dp.pop_start, dp.n_pop, (int32_t)j);
    const uint32_t* sg = dp.seg + (size_t)j * (size_t)(dp.n_part + 1);
    const uint32_t b = __ldg(sg), e = __ldg(sg + dp.n_part);
    for (uint32_t w = b + lane; w < e; w += 32) deliver_word(dp, __ldg(&dp.words[w]), q);
    if (lane == 0) atomicAdd(&dp.counters[1], (unsigned long long)(e - b));
}

__global__ void __launch_bounds__(256) k_deliver_block(const __grid_constant__ DeliverParams dp) {
    const uint32_t j = __ldg(&dp.spikes[blockIdx.x]);
    const int q = pop_index(dp.pop_start, dp.n_pop, (int32_t)j);
    const uint32_t* sg = dp.seg + (size_t)j * (size_t)(dp.n_part + 1);
    const uint32_t b = __ldg(sg), e = __ldg(sg + dp.n_part);
    for (uint32_t w = b + threadIdx.x; w < e; w += 256) deliver_word(dp, __ldg(&dp.words[w]), q);
    if (threadIdx.x == 0) atomicAdd(&dp.counters[1], (unsigned long long)(e - b));
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
size_t step_shared_bytes(int ncmax, int n_part, bool smem_ring) {
    return smem_layout(ncmax, n_part, smem_ring).total;
}

template <int NPT, bool R>
static const void* step_fn() { return reinterpret_cast<const void*>(&k_step<NPT, R>); }

static const void* select_step(int npt, bool smem_ring) {
    switch (npt) {
        case 1: return smem_ring ? step_fn<1, true>() : step_fn<1, false>();
        case 2: return smem_ring ? step_fn<2, true>() : step_fn<2, false>();
        case 4: return smem_ring ? step_fn<4, true>() : step_fn<4, false>();
        case 8: return smem_ring ? step_fn<8, true>() : step_fn<8, false>();
        default: return nullptr;
    }
}

int step_kernel_variant(int npt, bool smem_ring) { return select_step(npt, smem_ring) != nullptr; }

cudaError_t step_kernel_configure(int npt, bool smem_ring, size_t smem) {
    const void* fn = select_step(npt, smem_ring);
    if (!fn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t step_max_blocks(int npt, bool smem_ring, size_t smem, int* blocks_per_sm) {
    const void* fn = select_step(npt, smem_ring);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kStepThreads, smem);
}

cudaError_t launch_step(const StepParams& sp, int npt, bool smem_ring, size_t smem,
                        cudaStream_t s) {
    const void* fn = select_step(npt, smem_ring);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<StepParams*>(&sp)};
    return cudaLaunchCooperativeKernel(fn, dim3(sp.n_part), dim3(kStepThreads), args, smem, s);
}

cudaError_t launch_deliver(const DeliverParams& dp, int tiling, cudaStream_t s) {
    if (dp.n_spikes <= 0) return cudaSuccess;
    if (tiling == 0) {
        const long long threads = (long long)dp.n_spikes * 32;
        k_deliver_warp<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(dp);
    } else {
        k_deliver_block<<<dp.n_spikes, 256, 0, s>>>(dp);
    }
    return cudaGetLastError();
}

}  // namespace snn
