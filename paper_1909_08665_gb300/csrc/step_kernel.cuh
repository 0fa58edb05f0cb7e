// step_kernel.cuh -- the persistent step kernel: the time-stepped simulation on the device (Sec. 2.1 Eq. 1,
// Sec. 3.1.2 synaptic input buffers, Sec. 3.1.3 per-step processing).
//
// One persistent cooperative launch runs n steps.  CTA c owns the neuron
// range [part_lo[c], part_lo[c+1]): their state lives in registers and their
// 64-slot synaptic-input ring buffers live in shared memory (or in a
// partition-private global block when they do not fit).  Rows are sorted by
// target and partitions are contiguous neuron ranges, so the synapses of row
// j onto partition c are one contiguous run of the row, [seg[j][c],
// seg[j][c+1]).  CTA c reads exactly that run of every spike's row -- 4 bytes
// per synaptic event, the algorithmic minimum -- from a pre-decoded copy of
// the rows whose entries carry the weight-table index and the offset of the
// target's ring cell in its partition's slice, and adds the weights (looked
// up in a shared-memory copy of the table rows its populations use) with
// shared-memory atomics.  The run bounds come from the segment table, which
// the CTA reads for each spike while it gathers the step's spike ids, so that
// lookup overlaps the wait for the slowest partition's message.
//
// Per step t the order is:
//   A(t)  u_t from (u_{t-1}, I_{t-1}); threshold, reset, refractory; the
//         spikes of step t are compacted with warp ballots and published as
//         a message of 64-bit words (tag = t+1, value) -- the count and the
//         neuron ids; the Poisson background count of step t is drawn.
//   D     wait for every partition's message of step t-1 (each word carries
//         its own tag, so a matching tag is both the grid-wide barrier and
//         the data; no fence, no counter), look up each spike's run for this
//         partition and deliver those spikes into ring slots t-1+d (d >= 1):
//         per warp, batches of a few spikes whose runs are all loaded
//         before the shared-memory atomics.
//   C(t)  acc = ring[t] (cleared) + background; I_t = P11 I_{t-1} + acc/256.
// A(t+1) needs only I_t, and the spikes of step t reach no input before
// slot t+1, so the spike exchange of one step overlaps the next step's
// membrane update.  All results equal the sequential order of the method
// (integer accumulation, fp32 operations in a fixed order, no FMA).
//
// Message slots rotate over 4 steps.  A partition can run at most one step
// ahead of the slowest (it waits for everyone's step t-1 message before it
// publishes step t+1), so a slot is never rewritten while it is being read.
// Tags are 32-bit: runs are limited to 2^32 - 2 steps (about 119 h).
//
// The kernel template lives in this header so that its variants compile in
// parallel: each MODE (plain, paced, wrap-counting, both) is instantiated for
// every launch shape by step_fn_mode<MODE>, one translation unit per MODE
// (step_mode_plain.cu, step_mode_paced.cu, step_mode_sat.cu,
// step_mode_sat_paced.cu).
#pragma once
#include "snn_internal.cuh"

namespace snn {

constexpr int kWarps = kStepThreads / 32;
constexpr uint32_t kStatusRasterOverflow = 2u;
constexpr int kInline = 7;              // ids read together with a message header (64 B)
// A warp takes BATCH spikes at once and loads the first 32 WAVE entries of
// each of their runs in one wave (runs: mean 26 entries at scale 1 and 4,
// rarely above 96).  At full size (one neuron per thread) the spikes are
// dealt round-robin over the warps and each warp loads its next batch before
// the adds of the current one; measured that way, 2 x 3 is fastest (2.566 us
// per step; 3 x 3: 2.618, 2 x 2: 2.658, 4 x 3: 2.695, 4 x 2: 2.725, 1 x 3:
// 2.754; two batches ahead, 2 x 3: 2.657, 1 x 3: 2.779), against 2.711 for
// 3 x 3 in contiguous batches without the early load, the fastest shape of
// those (earlier in the kernel's history 3.00 us; 4 x 4: 3.14, 2 x 3: 3.08,
// 3 x 2: 3.24, 2 x 2: 3.21).  At 4x
// (4 neurons per thread, 177 spikes per step; contiguous batches, loaded one
// at a time: the registers of that variant are spent) 8 x 3 is fastest
// (14.3 us; 4 x 4: 14.5, 3 x 3: 15.9, 6 x 4: 16.0, 8 x 4: 16.4).
template <int NPT>
struct BatchShape {
    static constexpr int kSpikes = NPT == 1 ? 2 : 8;
    static constexpr int kWave = 3;
};
constexpr uint32_t kPopWords = kMaxPop * kWCodes;   // weight-table entries per target population

// ---------------------------------------------------------------------------
// shared-memory layout (bytes), identical on host and device
// ---------------------------------------------------------------------------
struct SmemLayout {
    uint32_t pois, warp, misc, inl, rb, rl, w, ring, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// s_rb / s_rl: first entry and length of each listed spike's run; s_w: the
// weight-table rows [p][q][code] of the w_span target populations from the
// partition's first one on
__host__ __device__ inline SmemLayout smem_layout(int ncmax, int n_part, int w_span,
                                                  bool smem_ring) {
    SmemLayout L;
    uint32_t o = 0;
    L.pois = o;   o += kMaxPop * kPoisTable * 4;
    L.warp = o;   o += 32 * 4;
    L.misc = o;   o += 32 * 4;
    L.inl = o;    o += (uint32_t)n_part * kInline * 8;
    L.rb = o;     o += kChunk * 4;
    L.rl = o;     o += kChunk * 4;
    L.w = o;      o += (uint32_t)w_span * kPopWords * 4;
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

__device__ __forceinline__ uint32_t tag_of(unsigned long long w) { return (uint32_t)(w >> 32); }

// bounded-time poll of one message word until it carries `tag`
__device__ inline bool poll_word(const StepParams& sp, const unsigned long long* p, uint32_t tag,
                          unsigned long long& w) {
    uint64_t t_start = 0;
    uint32_t iter = 0;
    while (tag_of(w) != tag) {
        if (iter == 0) t_start = globaltimer_ns();
        if ((++iter & 31u) == 0u) {
            if (ld_relaxed_gpu(sp.abort_flag) != 0u) return false;
            if (globaltimer_ns() - t_start > sp.timeout_ns || iter > 0x7fffffffu) {
                atomicOr(sp.status, kStatusTimeout);
                atomicExch(sp.abort_flag, 1u);
                return false;
            }
        }
        w = __ldcg(p);
    }
    return true;
}

// ---------------------------------------------------------------------------
// the runs s_rb/s_rl[0, m) of the spikes of step tb into this CTA's ring:
// batches of kBatchSpikes spikes per warp (BatchShape).  Entry x of a run (a pre-decoded synapse) is
// the weight-table index x >> kPreOffBits and the ring offset
// x & kPreOffMask = delay * ncmax + local target; its weight, looked up in
// s_w (table rows from population p_lo on, wbase = p_lo * kPopWords), is
// added at ((tb mod 64) * ncmax + offset) wrapped into the 64-slot ring.  Each
// lane loads entries lane + 32 h (h < kRunWave) of all the batch's runs before the
// first add (all loads in flight at once); longer runs finish in a loop.  In
// the pipelined shape (PIPE) warp w's batch of round r holds the list's
// spikes r kStride + w + k kWarps (k < kBatchSpikes), so a short list spreads
// over all warps, and the next round's batch is loaded before this one's
// adds; otherwise a batch is kBatchSpikes consecutive spikes.
// ---------------------------------------------------------------------------
// SAT: the networks whose input can leave the int32 range also count, per
// ring cell, the net number of times its int32 sum wrapped around (+1 past
// the top, -1 past the bottom).  Each add's wrap follows from the value it
// replaced, so the count is exact in any order: the true sum of a cell is its
// int32 value plus 2^32 times its count.
template <bool SAT>
__device__ __forceinline__ void add_entry(uint32_t x, const int32_t* s_w, uint32_t wbase,
                                          int32_t base_t, int32_t R, int32_t* ring,
                                          int32_t* wrap) {
    const int32_t w = s_w[(x >> kPreOffBits) - wbase];
    int32_t a = base_t + (int32_t)(x & kPreOffMask);
    a -= a >= R ? R : 0;
    if (SAT) {
        const int32_t old = atomicAdd(&ring[a], w);
        const int32_t now = (int32_t)((uint32_t)old + (uint32_t)w);
        if (((old ^ now) & (w ^ now)) < 0) atomicAdd(&wrap[a], w < 0 ? -1 : 1);
    } else {
        atomicAdd(&ring[a], w);
    }
}

// s_cnt (non-null while per-step counts are recorded): the list's synaptic
// events and its non-empty runs are added into s_cnt[0], s_cnt[1]
template <bool SAT, int kBatchSpikes, int kRunWave>
__device__ __forceinline__ void deliver_batches(const StepParams& sp, const uint32_t* s_rb,
                                                const uint32_t* s_rl, const int32_t* s_w,
                                                uint32_t wbase, uint32_t m, int64_t tb,
                                                int32_t* ring, int32_t* wrap,
                                                unsigned long long& events, uint32_t* s_cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t R = kRing * sp.ncmax;                  // ring words of this CTA
    const int32_t base_t = (int32_t)(((uint32_t)tb & (kRing - 1)) * (uint32_t)sp.ncmax);
    const uint32_t* pre = sp.pre;
    // PIPE: the warp's next batch is loaded before this one's adds, so its
    // round trip overlaps them (steps with more than kStride spikes); only
    // where the registers allow it (the one-neuron-per-thread shape)
    constexpr bool PIPE = kBatchSpikes * kRunWave <= 9;
    // run bounds and first-wave entries of the batch whose first spike is
    // list position g0 (nothing past m is read)
    auto load = [&](uint32_t g0, uint32_t (&rb)[kBatchSpikes], uint32_t (&rl)[kBatchSpikes],
                    uint32_t (&ev)[kBatchSpikes][kRunWave]) {
#pragma unroll
        for (int k = 0; k < kBatchSpikes; ++k) {
            const uint32_t i = g0 + (uint32_t)k * (PIPE ? (uint32_t)kWarps : 1u);
            const bool ok = i < m;
            rb[k] = ok ? s_rb[i] : 0u;
            rl[k] = ok ? s_rl[i] : 0u;
#pragma unroll
            for (int h = 0; h < kRunWave; ++h) {
                const uint32_t e = (uint32_t)lane + 32u * (uint32_t)h;
                ev[k][h] = e < rl[k] ? __ldg(pre + ((size_t)rb[k] + e)) : 0u;
            }
        }
    };
    constexpr uint32_t kStride = (uint32_t)kWarps * kBatchSpikes;
    uint32_t g0 = (uint32_t)warp * (PIPE ? 1u : (uint32_t)kBatchSpikes);
    uint32_t rb[kBatchSpikes], rl[kBatchSpikes];
    uint32_t ev[kBatchSpikes][kRunWave];
    if (PIPE) load(g0, rb, rl, ev);
    for (; g0 < m; g0 += kStride) {
        uint32_t nrb[kBatchSpikes], nrl[kBatchSpikes];
        uint32_t nev[kBatchSpikes][kRunWave];
        if (PIPE) load(g0 + kStride, nrb, nrl, nev);
        else load(g0, rb, rl, ev);
#pragma unroll
        for (int k = 0; k < kBatchSpikes; ++k) {
#pragma unroll
            for (int h = 0; h < kRunWave; ++h)
                if ((uint32_t)lane + 32u * (uint32_t)h < rl[k])
                    add_entry<SAT>(ev[k][h], s_w, wbase, base_t, R, ring, wrap);
            // entries beyond the first wave (runs longer than 32 kRunWave)
            for (uint32_t e = 32u * kRunWave + (uint32_t)lane; e < rl[k]; e += 32u)
                add_entry<SAT>(__ldg(pre + ((size_t)rb[k] + e)), s_w, wbase, base_t, R, ring, wrap);
            if (lane == 0) events += rl[k];
        }
        if (s_cnt != nullptr && lane == 0) {
            uint32_t ev_sum = 0u, busy = 0u;
#pragma unroll
            for (int k = 0; k < kBatchSpikes; ++k) {
                ev_sum += rl[k];
                busy += rl[k] > 0u ? 1u : 0u;
            }
            atomicAdd(&s_cnt[0], ev_sum);
            atomicAdd(&s_cnt[1], busy);
        }
        if (PIPE) {
#pragma unroll
            for (int k = 0; k < kBatchSpikes; ++k) {
                rb[k] = nrb[k];
                rl[k] = nrl[k];
#pragma unroll
                for (int h = 0; h < kRunWave; ++h) ev[k][h] = nev[k][h];
            }
        }
    }
}

// Runs of this partition c for the N spike ids ids[0, cnt): both bounds of
// every id are loaded before any is stored, so the lookups are in flight
// together; a run is written as (first entry, length).
template <int N>
__device__ __forceinline__ void store_runs(const StepParams& sp, int c, const uint32_t (&ids)[N],
                                           uint32_t cnt, uint32_t* o_rb, uint32_t* o_rl) {
    uint32_t b[N], e[N];
    const size_t stride = (size_t)sp.n_part + 1;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        b[k] = e[k] = 0u;
        if ((uint32_t)k < cnt) {
            const uint32_t* sg = sp.seg + (size_t)ids[k] * stride + c;
            b[k] = __ldg(sg);
            e[k] = __ldg(sg + 1);
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
        if ((uint32_t)k < cnt) {
            o_rb[k] = b[k];
            o_rl[k] = e[k] - b[k];
        }
}

// The run bounds of one partition's first kInline spikes of step tb, looked
// up from the message head as loaded before A(tb + 1): valid (ok) only if the
// head and each of those id words already carried the tag tb + 1.
struct EarlyRuns {
    bool ok;
    uint32_t b[kInline], e[kInline];
};

__device__ __forceinline__ void early_runs(const StepParams& sp, int c, const ulonglong2 (&pre)[4],
                                           uint32_t tag, EarlyRuns& er) {
    if (tag_of(pre[0].x) != tag) return;
    const uint32_t g = min((uint32_t)pre[0].x, (uint32_t)kInline);
    const unsigned long long w[kInline] = {pre[0].y, pre[1].x, pre[1].y, pre[2].x,
                                           pre[2].y, pre[3].x, pre[3].y};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < kInline; ++i)
        if ((uint32_t)i < g && tag_of(w[i]) != tag) ok = false;
    if (!ok) return;
    const size_t stride = (size_t)sp.n_part + 1;
#pragma unroll
    for (int i = 0; i < kInline; ++i) {
        er.b[i] = er.e[i] = 0u;
        if ((uint32_t)i < g) {
            const uint32_t* sg = sp.seg + (size_t)(uint32_t)w[i] * stride + c;
            er.b[i] = __ldg(sg);
            er.e[i] = __ldg(sg + 1);
        }
    }
    er.ok = true;
}

// ---------------------------------------------------------------------------
// delivery of the spikes of step tb (message tag tb+1) into this CTA's ring;
// returns false if a wait timed out or another CTA aborted
// ---------------------------------------------------------------------------
template <bool SAT, int BATCH, int WAVE>
__device__ __forceinline__ bool deliver_list(const StepParams& sp, unsigned char* smem,
                                             const SmemLayout& L, int c, uint32_t wbase,
                                             int64_t tb, int32_t* ring, int32_t* wrap,
                                             unsigned long long& events,
                                             const ulonglong2 (&pre)[4],
                                             const EarlyRuns& early) {
    const int tid = threadIdx.x;
    const int P = sp.n_part;
    const int list = (int)(tb & 3);
    const uint32_t tag = (uint32_t)(tb + 1);
    uint32_t* s_warp = reinterpret_cast<uint32_t*>(smem + L.warp);
    volatile uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + L.misc);
    unsigned long long* s_inl = reinterpret_cast<unsigned long long*>(smem + L.inl);
    uint32_t* s_rb = reinterpret_cast<uint32_t*>(smem + L.rb);
    uint32_t* s_rl = reinterpret_cast<uint32_t*>(smem + L.rl);
    const int32_t* s_w = reinterpret_cast<const int32_t*>(smem + L.w);
    const unsigned long long* msg = sp.msg + (size_t)list * P * sp.msg_stride;
    // per-step counts of this list (s_misc[4], [5]: events, non-empty runs)
    const int64_t rec = tb - sp.sc_t0;
    const bool counting = sp.st_counts != nullptr && rec >= 0 && rec < sp.sc_cap;
    uint32_t* s_cnt = counting ? const_cast<uint32_t*>(&s_misc[4]) : nullptr;
    auto flush_counts = [&](uint32_t m_total) {
        if (counting && tid == 0) {
            uint32_t* r = sp.st_counts + 4 * rec;
            atomicAdd(&r[1], s_misc[4]);
            atomicMax(&r[2], s_misc[5]);
            atomicAdd(&r[3], m_total - s_misc[5]);
            s_misc[4] = 0u;
            s_misc[5] = 0u;
        }
    };

    // 1. every partition's 64-byte message head: the header word (the wait and
    //    the spike count at once) and the first kInline ids.  pre[] is the
    //    head as loaded by the caller, early; a stale head is polled again.
    uint32_t cnt[1] = {0u};
    const unsigned long long* m_mine = msg + (size_t)tid * sp.msg_stride;
    if (tid < P) {
        ulonglong2 h[4] = {pre[0], pre[1], pre[2], pre[3]};
        if (tag_of(h[0].x) != tag) {
            uint64_t t_start = globaltimer_ns();
            uint32_t iter = 0;
            do {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    h[q] = __ldcg(reinterpret_cast<const ulonglong2*>(m_mine + 2 * q));
                if ((++iter & 31u) == 0u) {
                    if (ld_relaxed_gpu(sp.abort_flag) != 0u ||
                        globaltimer_ns() - t_start > sp.timeout_ns) {
                        if (ld_relaxed_gpu(sp.abort_flag) == 0u) {
                            atomicOr(sp.status, kStatusTimeout);
                            atomicExch(sp.abort_flag, 1u);
                        }
                        s_misc[2] = 1u;
                        break;
                    }
                }
            } while (tag_of(h[0].x) != tag);
        }
        cnt[0] = (uint32_t)h[0].x;
        s_inl[tid * kInline + 0] = h[0].y;
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            s_inl[tid * kInline + 2 * q - 1] = h[q].x;
            s_inl[tid * kInline + 2 * q] = h[q].y;
        }
    }
    const uint32_t my_cnt = cnt[0];
    // 2a. usual case, one barrier: each header reader appends its partition's
    //     runs to the shared list at a position taken from a shared counter;
    //     ids beyond the inline ones are loaded 8 at a time, all in flight,
    //     and the run bounds of a group of ids are looked up together
    if (tid < P && my_cnt > 0u) {
        const uint32_t at = atomicAdd(const_cast<uint32_t*>(&s_misc[3]), my_cnt);
        if (at + my_cnt <= (uint32_t)kChunk) {
            if (early.ok) {                          // bounds looked up during A(tb + 1)
#pragma unroll
                for (int i = 0; i < kInline; ++i)
                    if ((uint32_t)i < my_cnt) {
                        s_rb[at + i] = early.b[i];
                        s_rl[at + i] = early.e[i] - early.b[i];
                    }
            } else {
                uint32_t ids[kInline];
#pragma unroll
                for (int i = 0; i < kInline; ++i) {
                    ids[i] = 0u;                     // in range if a wait gives up
                    if ((uint32_t)i < my_cnt) {
                        unsigned long long e = s_inl[tid * kInline + i];
                        if (poll_word(sp, m_mine + 1 + i, tag, e)) ids[i] = (uint32_t)e;
                        else s_misc[2] = 1u;
                    }
                }
                store_runs<kInline>(sp, c, ids, min(my_cnt, (uint32_t)kInline), s_rb + at,
                                    s_rl + at);
            }
            for (uint32_t i = kInline; i < my_cnt; i += 8) {
                ulonglong2 v[4];                     // entries 1+i.. are 16-B aligned
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    v[q] = i + 2 * q < my_cnt
                               ? __ldcg(reinterpret_cast<const ulonglong2*>(m_mine + 1 + i + 2 * q))
                               : make_ulonglong2(0ull, 0ull);
                uint32_t ids8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t k = i + (uint32_t)q;
                    ids8[q] = 0u;
                    if (k < my_cnt) {
                        unsigned long long e = (q & 1) ? v[q >> 1].y : v[q >> 1].x;
                        if (poll_word(sp, m_mine + 1 + k, tag, e)) ids8[q] = (uint32_t)e;
                        else s_misc[2] = 1u;
                    }
                }
                store_runs<8>(sp, c, ids8, min(my_cnt - i, 8u), s_rb + at + i, s_rl + at + i);
            }
        }
    }
    __syncthreads();
    const uint32_t S_fast = s_misc[3];
    if (s_misc[2]) return false;
    if (S_fast <= (uint32_t)kChunk) {
        deliver_batches<SAT, BATCH, WAVE>(sp, s_rb, s_rl, s_w, wbase, S_fast, tb, ring, wrap, events,
                                          s_cnt);
        __syncthreads();
        if (tid == 0) s_misc[3] = 0u;
        flush_counts(S_fast);
        return s_misc[2] == 0u;
    }
    // 2b. more than kChunk spikes: offsets by a block-wide scan, in chunks
    const uint32_t S = block_scan<1>(cnt, s_warp);   // cnt[0] <- my offset
    if (tid == 0) s_misc[3] = 0u;
    const uint32_t my_off = cnt[0];

    for (uint32_t base = 0; base < S; base += kChunk) {
        const uint32_t m = min((uint32_t)kChunk, S - base);
        // 2. the runs of this chunk into the shared list, each partition's
        //    written by the thread that read its header, 8 ids at a time
        if (tid < P) {
            // this partition's ids i with base <= my_off + i < base + m
            const uint32_t i0 = base > my_off ? base - my_off : 0u;
            const uint32_t i1 = base + m > my_off ? min(my_cnt, base + m - my_off) : 0u;
            for (uint32_t i = i0; i < i1; i += 8) {
                uint32_t ids8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t k = i + (uint32_t)q;
                    ids8[q] = 0u;                    // in range if a wait gives up
                    if (k < i1) {
                        const unsigned long long* mp = m_mine + 1 + k;
                        unsigned long long e = k < (uint32_t)kInline ? s_inl[tid * kInline + k] : __ldcg(mp);
                        if (poll_word(sp, mp, tag, e)) ids8[q] = (uint32_t)e;
                        else s_misc[2] = 1u;
                    }
                }
                const uint32_t o = my_off + i - base;
                store_runs<8>(sp, c, ids8, min(i1 - i, 8u), s_rb + o, s_rl + o);
            }
        }
        __syncthreads();
        deliver_batches<SAT, BATCH, WAVE>(sp, s_rb, s_rl, s_w, wbase, m, tb, ring, wrap, events,
                                          s_cnt);
        __syncthreads();
    }
    flush_counts(S);
    return s_misc[2] == 0u;
}

// Bulk prefetch of [addr, addr + bytes) into L2 (16-byte aligned, multiple
// of 16 bytes): fire and forget.
__device__ __forceinline__ void prefetch_l2(unsigned long long addr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(addr), "r"(bytes) : "memory");
}

// 16-byte-aligned span covering the 4-byte words [b, e) of base
__device__ __forceinline__ void span16(const uint32_t* base, unsigned long long b,
                                       unsigned long long e, unsigned long long& addr,
                                       uint32_t& bytes) {
    const unsigned long long lo = reinterpret_cast<unsigned long long>(base + b) & ~15ull;
    const unsigned long long hi = (reinterpret_cast<unsigned long long>(base + e) + 15ull) & ~15ull;
    addr = lo;
    bytes = e > b ? (uint32_t)(hi - lo) : 0u;
}

// ---------------------------------------------------------------------------
// persistent step kernel
// ---------------------------------------------------------------------------
// MODE bit kModePaced: the variant for runs paced to wall-clock time
// (snn_set_realtime); bit kModeSat: the variant for networks whose input can
// leave the int32 range, which counts wrap-arounds (sp.wrap).  Each lives
// only in its own instantiation, so the plain step loop is unchanged.
constexpr int kModePaced = 1;
constexpr int kModeSat = 2;

template <int NPT, bool SMEM_RING, int MODE>
__global__ void __launch_bounds__(kStepThreads, 1)
k_step(const __grid_constant__ StepParams sp) {
    constexpr bool PACED = (MODE & kModePaced) != 0;
    constexpr bool SAT = (MODE & kModeSat) != 0;
    // early run lookups keep 2 x kInline more registers live across the
    // background draw: only in the one-neuron-per-thread variant
    constexpr bool EARLY = NPT == 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int c = blockIdx.x;
    const int P = sp.n_part;
    const SmemLayout L = smem_layout(sp.ncmax, P, sp.w_span, SMEM_RING);
    uint32_t* s_pois = reinterpret_cast<uint32_t*>(smem + L.pois);
    uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + L.misc);
    int32_t* s_w = reinterpret_cast<int32_t*>(smem + L.w);

    const int32_t lo = sp.part_lo[c];
    const int32_t nc = sp.part_lo[c + 1] - lo;
    int32_t* ring = SMEM_RING ? reinterpret_cast<int32_t*>(smem + L.ring)
                              : sp.ring + (size_t)c * kRing * (size_t)sp.ncmax;
    int32_t* ring_g = sp.ring + (size_t)c * kRing * (size_t)sp.ncmax;
    int32_t* wrap = SAT ? sp.wrap + (size_t)c * kRing * (size_t)sp.ncmax : nullptr;
    bool saturated = false;

    for (int k = tid; k < kMaxPop * kPoisTable; k += kStepThreads)
        s_pois[k] = sp.pois_m1[k / kPoisTable][k % kPoisTable];
    // weight-table rows of the target populations of this partition: those
    // from the population of its first neuron on (at most w_span of them)
    const uint32_t wt_base = (uint32_t)pop_index(sp.pop_start, sp.n_pop, lo) * kPopWords;
    for (uint32_t k = tid; k < (uint32_t)sp.w_span * kPopWords; k += kStepThreads)
        s_w[k] = wt_base + k < (uint32_t)(kMaxPop * kPopWords) ? __ldg(&sp.wtab[wt_base + k]) : 0;
    if (SMEM_RING)
        for (int k = tid; k < kRing * sp.ncmax; k += kStepThreads) ring[k] = ring_g[k];
    if (tid < 32) s_misc[tid] = 0u;
    // pacing to wall-clock time: the first CTA to arrive fixes the anchor of
    // the paced run (the device clock at which step rt_t_anchor starts) in
    // rt[0]; the barrier before the step loop orders it before every read
    if (PACED && tid == 0) atomicCAS(sp.rt, 0ull, globaltimer_ns());

    float u[NPT], isyn[NPT];
    int32_t refr[NPT], pacc[NPT];
    int pop[NPT];
    uint4 rnd[NPT];
    // the neuron's own row of the pre-decoded rows and of the segment table,
    // prefetched into L2 when it spikes: every partition reads its run of
    // that row one step later (NPT <= 4: the registers of the widest
    // variant are spent elsewhere)
    constexpr int NPF = NPT <= 4 ? NPT : 1;
    unsigned long long pf_row[NPF], pf_seg[NPF];
    uint32_t pf_row_n[NPF], pf_seg_n[NPF];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int li = tid + k * kStepThreads;
        u[k] = 0.f; isyn[k] = 0.f; refr[k] = 0; pop[k] = 0; pacc[k] = 0;
        rnd[k] = make_uint4(0u, 0u, 0u, 0u);
        if (k < NPF) { pf_row[k] = pf_seg[k] = 0ull; pf_row_n[k] = pf_seg_n[k] = 0u; }
        if (li < nc) {
            u[k] = sp.u[lo + li];
            isyn[k] = sp.i_syn[lo + li];
            refr[k] = sp.refr[lo + li];
            pop[k] = pop_index(sp.pop_start, sp.n_pop, lo + li);
            if (NPT <= 4 && k < NPF) {
                const unsigned long long j = (unsigned long long)(lo + li);
                span16(sp.pre, sp.row_start[j], sp.row_start[j + 1], pf_row[k], pf_row_n[k]);
                const unsigned long long sw = j * (unsigned long long)(P + 1);
                span16(sp.seg, sw, sw + (unsigned long long)(P + 1), pf_seg[k], pf_seg_n[k]);
            }
        }
    }
    uint32_t ras_base = sp.ras_n[c];
    unsigned long long spikes = 0, events = 0;
    bool aborted = false;
    __syncthreads();

    for (int s = 0; s < sp.n_steps; ++s) {
        const int64_t t = sp.t0 + s;
        const unsigned long long tag = (unsigned long long)(uint32_t)(t + 1) << 32;
        // paced run: step t is released at anchor + (t - t_anchor) periods
        if (PACED)
            wait_until_ns(__ldcg(sp.rt) + (unsigned long long)(t - sp.rt_t_anchor) * sp.rt_period_ns);
        unsigned long long* my_msg = sp.msg + ((size_t)(t & 3) * P + c) * sp.msg_stride;
        uint32_t* my_cnt = &s_misc[s & 1];
        // headers of step t-1 were published one step ago: load them now so
        // the round trip overlaps A(t)
        ulonglong2 pre[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) pre[q] = make_ulonglong2(0ull, 0ull);
        if (s > 0 && tid < P) {
            const unsigned long long* m = sp.msg + ((size_t)((t - 1) & 3) * P + tid) * sp.msg_stride;
#pragma unroll
            for (int q = 0; q < 4; ++q) pre[q] = __ldcg(reinterpret_cast<const ulonglong2*>(m + 2 * q));
        }
        // ---- A(t): membrane, threshold, compaction, publication ----
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int li = tid + k * kStepThreads;
            bool spk = false;
            if (li < nc) {
                uint8_t upd = 0;
                if (refr[k] > 0) {
                    refr[k] -= 1;
                    u[k] = 0.f;
                } else {
                    float v = __fadd_rn(__fmul_rn(sp.P22, u[k]), __fmul_rn(sp.P21, isyn[k]));
                    if (sp.mode == 1) v = __fadd_rn(v, sp.cdc[pop[k]]);
                    u[k] = v;
                    upd = 2;
                }
                const float upre = u[k];
                if (u[k] > sp.theta) {
                    spk = true;
                    u[k] = 0.f;
                    refr[k] = sp.n_ref;
                    if (sp.pop_spikes) atomicAdd(&sp.pop_spikes[pop[k]], 1ull);
                }
                if (sp.tr_u != nullptr && t >= sp.tr_t0 && t < sp.tr_t0 + sp.tr_len) {
                    const size_t o = (size_t)(t - sp.tr_t0) * (size_t)sp.n + (size_t)(lo + li);
                    sp.tr_u[o] = upre;
                    sp.tr_f[o] = (uint8_t)(upd | (spk ? 1 : 0));
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
                    __stcg(&my_msg[1 + pos], tag | id);
                    if (NPT <= 4 && k < NPF) {
                        if (pf_row_n[k]) prefetch_l2(pf_row[k], pf_row_n[k]);
                        prefetch_l2(pf_seg[k], pf_seg_n[k]);
                    }
                    const uint32_t rp = ras_base + pos;
                    if (rp < sp.ras_cap) {
                        sp.ras_step[(size_t)c * sp.ras_cap + rp] = (uint32_t)t;
                        sp.ras_id[(size_t)c * sp.ras_cap + rp] = id;
                    }
                }
            }
            // background count of step t (independent of the network): drawn
            // here, added to the ring input in C(t)
            if (sp.mode == 0 && li < nc) {
                if ((t & 3) == 0 || s == 0)
                    rnd[k] = philox(make_uint4((uint32_t)(lo + li), (uint32_t)(t >> 2),
                                               kStreamPois, (uint32_t)(t >> 34)),
                                    sp.key0, sp.key1);
                // k = #{m : x >= T_m} = #{m : x > T_m - 1}; thresholds ascend,
                // so the tail beyond 12 only matters when all 12 are passed
                const uint32_t x = lane_of(rnd[k], (int)(t & 3));
                const uint32_t* thr = s_pois + pop[k] * kPoisTable;
                int kk = 0;
#pragma unroll
                for (int mm = 0; mm < 12; ++mm) kk += x > thr[mm] ? 1 : 0;
                if (kk == 12)
                    for (int mm = 12; mm < kPoisTable; ++mm) kk += x > thr[mm] ? 1 : 0;
                pacc[k] = kk * sp.wext_q;
            }
        }
        // the run bounds of the step t-1 spikes whose message words this
        // header thread already holds (the head loaded before A(t), arrived
        // by now): looked up here, so that they return while the CTA meets
        // at the barrier and the header is published
        EarlyRuns early;
        early.ok = false;
        if (EARLY && s > 0 && tid < P) early_runs(sp, c, pre, (uint32_t)t, early);
        __syncthreads();
        const uint32_t nsp = *my_cnt;
        if (tid == 0) {
            // counter of step s+1 (last used in step s-1): its readers are all
            // past a barrier; in step 0 it is still zero from the start and is
            // left alone (no barrier separates it from step 1's adds)
            if (s > 0) s_misc[(s + 1) & 1] = 0u;
            if (!(sp.inject_fault == 1 && c == 0)) __stcg(&my_msg[0], tag | nsp);
            spikes += nsp;
            if (ras_base + nsp > sp.ras_cap) atomicOr(sp.status, kStatusRasterOverflow);
            if (sp.st_counts != nullptr && nsp > 0u) {
                const int64_t r = t - sp.sc_t0;
                if (r >= 0 && r < sp.sc_cap) atomicAdd(&sp.st_counts[4 * r], nsp);
            }
        }
        ras_base += nsp;
        // ---- D: spikes of step t-1 ----
        if (s > 0) {
            if (!deliver_list<SAT, BatchShape<NPT>::kSpikes, BatchShape<NPT>::kWave>(
                    sp, smem, L, c, wt_base, t - 1, ring, wrap, events, pre, early)) {
                aborted = true;
                break;
            }
        }
        // ---- C(t): ring slot t, Poisson background, synaptic current ----
        const uint32_t slot = (uint32_t)t & (kRing - 1);
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int li = tid + k * kStepThreads;
            if (li < nc) {
                const uint32_t cell = slot * (uint32_t)sp.ncmax + (uint32_t)li;
                const int32_t r = ring[cell];
                ring[cell] = 0;
                // the input wraps modulo 2^32, as the int32 accumulation of
                // the method does; SAT: its true value r + 2^32 wraps + pacc
                // must lie in the int32 range
                const int32_t acc = (int32_t)((uint32_t)r + (uint32_t)pacc[k]);
                if (SAT) {
                    const int32_t nw = wrap[cell];
                    if (nw != 0) wrap[cell] = 0;
                    const long long exact = (long long)r + (long long)nw * 4294967296ll + (long long)pacc[k];
                    if (exact > 2147483647ll || exact < -2147483648ll) saturated = true;
                }
                isyn[k] = __fadd_rn(__fmul_rn(sp.P11, isyn[k]),
                                    __fmul_rn(__int2float_rn(acc), 0.00390625f));
            }
        }
        // optional record of the device clock at the end of every step (CTA 0)
        if (sp.step_times != nullptr && c == 0 && tid == 0) {
            const int64_t r = t - sp.st_t0;
            if (r >= 0 && r < sp.st_cap) sp.step_times[r] = (long long)globaltimer_ns();
        }
        // paced run: a step that ends after release + period missed its
        // deadline (CTA 0's view of the step end)
        if (PACED && c == 0 && tid == 0) {
            const unsigned long long now = globaltimer_ns();
            const unsigned long long deadline =
                __ldcg(sp.rt) + (unsigned long long)(t + 1 - sp.rt_t_anchor) * sp.rt_period_ns;
            if (now > deadline) {
                atomicAdd(&sp.rt[1], 1ull);
                atomicMax(&sp.rt[2], now - deadline);
            }
        }
    }

    // ---- epilogue: deliver the spikes of the last step ----
    if (!aborted && sp.n_steps > 0) {
        const int64_t tl = sp.t0 + sp.n_steps - 1;
        ulonglong2 pre[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) pre[q] = make_ulonglong2(0ull, 0ull);
        if (tid < P) {
            const unsigned long long* m = sp.msg + ((size_t)(tl & 3) * P + tid) * sp.msg_stride;
#pragma unroll
            for (int q = 0; q < 4; ++q) pre[q] = __ldcg(reinterpret_cast<const ulonglong2*>(m + 2 * q));
        }
        EarlyRuns none;
        none.ok = false;
        deliver_list<SAT, BatchShape<NPT>::kSpikes, BatchShape<NPT>::kWave>(
            sp, smem, L, c, wt_base, tl, ring, wrap, events, pre, none);
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
    }
    if (SAT && saturated) atomicOr(sp.status, kStatusSaturated);
    if (lane == 0 && events) atomicAdd(&sp.counters[1], events);   // per-warp counts
}

// the kernel of one MODE for a launch shape (neurons per thread, ring in
// shared memory or not); nullptr for an unknown shape
template <int MODE>
const void* step_fn_mode(int npt, bool smem_ring) {
    switch (npt) {
        case 1: return smem_ring ? reinterpret_cast<const void*>(&k_step<1, true, MODE>)
                                 : reinterpret_cast<const void*>(&k_step<1, false, MODE>);
        case 2: return smem_ring ? reinterpret_cast<const void*>(&k_step<2, true, MODE>)
                                 : reinterpret_cast<const void*>(&k_step<2, false, MODE>);
        case 4: return smem_ring ? reinterpret_cast<const void*>(&k_step<4, true, MODE>)
                                 : reinterpret_cast<const void*>(&k_step<4, false, MODE>);
        case 8: return smem_ring ? reinterpret_cast<const void*>(&k_step<8, true, MODE>)
                                 : reinterpret_cast<const void*>(&k_step<8, false, MODE>);
        default: return nullptr;
    }
}
extern template const void* step_fn_mode<0>(int, bool);
extern template const void* step_fn_mode<kModePaced>(int, bool);
extern template const void* step_fn_mode<kModeSat>(int, bool);
extern template const void* step_fn_mode<kModeSat | kModePaced>(int, bool);

}  // namespace snn
