// deliver_words.cu -- stand-alone delivery of one long spike list (Sec. 3.1.2:
// row fetch, word decode, ring-buffer add), partition by partition.
//
// CTA c sums the list's input to partition c in shared memory when it fits --
// only the ring slots the list can reach, t + 1 .. t + D (D the longest delay
// of the network), zeroed at the start, so nothing is read in before the adds
// -- and adds the non-zero sums into the ring slice at the end; otherwise it
// adds straight into the ring slice in global memory.  For every spike j of
// the list it reads exactly the entries of row j that
// target partition c: the run [seg[j][c], seg[j][c + 1]) of the row, which is
// contiguous because rows are sorted by target.  That is the algorithmic 4
// bytes per synaptic event and no more, and every add is a shared-memory
// atomic of the CTA's own slice, so no add crosses the L2.
//
// The rows read here are a pre-decoded copy of the packed words, built once
// (k_predecode) in the same layout: the word's target, delay and weight code
// become the weight-table index and the offset of the target's ring cell in
// its partition's slice, relative to slot 0.  The decode (source and target
// population, partition start, delay slot) is then paid once per synapse
// instead of once per synaptic event, and an event costs a table lookup, one
// add with wrap-around and the atomic.
//
// The cost that scales with the list is one (spike, partition) pair per CTA
// and spike: a few dozen words at the microcircuit's scale 1, less than a
// warp.  So a warp takes 64 spikes (a round, two per lane) at a time and
// treats their segments as one concatenated run of T entries, which it walks
// in chunks of 32 consecutive positions: every lane of a chunk but the last
// has an entry, however the entries split into segments.  A lane finds its
// segment from a bitmap of the positions where segments start (a warp scan of
// the lengths gives them): the number of starts at or before its position,
// counted with popc, ranks it among the non-empty segments, whose row offsets
// sit in a 64-entry table.  kChunkBatch chunks have their entries loaded
// before the first add; loads and adds past the end of the run are predicated
// off rather than branched around.  Rounds are handed out dynamically, and the
// next round's spike ids and segment bounds are fetched while the current one
// is processed.
#include "snn_internal.cuh"

namespace snn {
namespace {

constexpr int kWThreads = 1024;
constexpr int kWWarps = kWThreads / 32;
constexpr int kRoundSpikes = 64;      // spikes per warp round, two per lane
constexpr int kBmWords = 64;          // bitmap of segment starts: 2048 positions per window
constexpr int kChunkBatch = 8;        // chunks of 32 entries per batch; two batches in flight
constexpr uint32_t kNone = 0xffffffffu;   // no entry (offsets stay below kPreOffMask)
static_assert(kBmWords % kChunkBatch == 0, "a batch of chunks never crosses a bitmap window");
static_assert(kChunkBatch % 4 == 0, "bitmap words are read four at a time");

// entry p[0] if k < T, else kNone (a predicated load, no branch)
__device__ __forceinline__ uint32_t load_entry(const uint32_t* p, uint32_t k, uint32_t T) {
    uint32_t v = kNone;
    asm("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %2, %3;\n\t@q ld.global.nc.u32 %0, [%1];\n\t}"
        : "+r"(v)
        : "l"(p), "r"(k), "r"(T));
    return v;
}

// ring[a] += w unless e is kNone (a predicated reduction, no branch)
__device__ __forceinline__ void add_shared(uint32_t saddr, int32_t w, uint32_t e) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, -1;\n\t@q red.shared.add.s32 [%0], %1;\n\t}"
        ::"r"(saddr), "r"(w), "r"(e)
        : "memory");
}

__device__ __forceinline__ void add_global(int32_t* p, int32_t w, uint32_t e) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, -1;\n\t@q red.global.add.s32 [%0], %1;\n\t}"
        ::"l"(p), "r"(w), "r"(e)
        : "memory");
}

struct WordsSmem {
    size_t off_wt, off_info, off_bm, off_ring, total;
};

// dynamic shared memory: weight table [p][q][code], per-warp segment offsets
// and start bitmaps, then (optionally) the sums [delay - 1][ncmax] of delays
// 1 .. depth (rounded up to whole 16-byte vectors)
__host__ __device__ WordsSmem words_smem(int ncmax, bool smem_ring, int depth) {
    WordsSmem L;
    L.off_wt = 0;
    L.off_info = L.off_wt + (size_t)kMaxPop * kMaxPop * kWCodes * 4;
    L.off_bm = L.off_info + (size_t)kWWarps * kRoundSpikes * 4;
    L.off_ring = L.off_bm + (size_t)kWWarps * kBmWords * 4;
    L.total = L.off_ring + (smem_ring ? ((size_t)depth * ncmax + 3) / 4 * 16 : 0);
    return L;
}

template <bool SMEM_RING>
__global__ void __launch_bounds__(kWThreads, 1)
k_deliver_words(const __grid_constant__ DeliverParams dp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_next_round;
    const int depth = dp.max_delay;
    const WordsSmem L = words_smem(dp.ncmax, SMEM_RING, depth);
    int32_t* s_wt = reinterpret_cast<int32_t*>(smem + L.off_wt);
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* info = reinterpret_cast<uint32_t*>(smem + L.off_info) + warp * kRoundSpikes;
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem + L.off_bm) + warp * kBmWords;
    const int R = kRing * dp.ncmax;
    int32_t* ring_g = dp.ring + (size_t)c * R;
    int32_t* ring = SMEM_RING ? reinterpret_cast<int32_t*>(smem + L.off_ring) : ring_g;

    for (int k = tid; k < kMaxPop * kMaxPop * kWCodes; k += kWThreads) s_wt[k] = __ldg(&dp.wtab[k]);
    const int n_sums = (depth * dp.ncmax + 3) / 4;       // 16-byte vectors of sums
    if (SMEM_RING) {
        int4* dst = reinterpret_cast<int4*>(ring);
        for (int k = tid; k < n_sums; k += kWThreads) dst[k] = make_int4(0, 0, 0, 0);
    }
    if (tid == 0) s_next_round = kWWarps;
    __syncthreads();

    const uint32_t base_t = ((uint32_t)dp.t & (kRing - 1)) * (uint32_t)dp.ncmax;
    const uint32_t ring_s = SMEM_RING ? (uint32_t)__cvta_generic_to_shared(ring) : 0u;
    const uint32_t lanes_le = 0xffffffffu >> (31 - lane);
    const uint32_t lanes_lt = lanes_le >> 1;
    // rounds of 64 spikes, then kWWarps rounds of 32 for the last spikes of
    // the list, so that warps run out of work at nearly the same time
    const int n = dp.n_spikes;
    const int tail = min(n, kWWarps * 32);
    const int head = n - tail;
    const int r64 = (head + kRoundSpikes - 1) / kRoundSpikes;
    const int n_rounds = r64 + (tail + 31) / 32;
    const size_t seg_stride = (size_t)dp.n_part + 1;
    unsigned long long events = 0;

    auto grab = [&]() {
        int r = 0;
        if (lane == 0) r = atomicAdd(&s_next_round, 1);
        return __shfl_sync(0xffffffffu, r, 0);
    };
    // segment of row j that targets this partition
    auto bounds = [&](uint32_t j, uint32_t& b, uint32_t& len) {
        const uint32_t* sg = dp.seg + (size_t)j * seg_stride + c;
        b = __ldg(sg);
        len = __ldg(sg + 1) - b;
    };
    // spike ids of round r for this lane: list positions 64 r + 2 lane and
    // + 1 in the first r64 rounds, head + 32 (r - r64) + lane after them
    auto ids = [&](int r, uint32_t& j0, uint32_t& j1) {
        if (r < r64) {
            const int g = r * kRoundSpikes + 2 * lane;
            j0 = g < head ? __ldg(&dp.spikes[g]) : kNone;
            j1 = g + 1 < head ? __ldg(&dp.spikes[g + 1]) : kNone;
        } else {
            const int g = head + 32 * (r - r64) + lane;
            j0 = g < n ? __ldg(&dp.spikes[g]) : kNone;
            j1 = kNone;
        }
    };
    auto round_bounds = [&](uint32_t j0, uint32_t j1, uint32_t& b0, uint32_t& l0, uint32_t& b1,
                            uint32_t& l1) {
        b0 = l0 = b1 = l1 = 0u;
        if (j0 != kNone) bounds(j0, b0, l0);
        if (j1 != kNone) bounds(j1, b1, l1);
    };

    int r_cur = warp;
    int r_next = grab();
    uint32_t b0, l0, b1, l1, j0, j1;
    ids(r_cur, j0, j1);
    round_bounds(j0, j1, b0, l0, b1, l1);
    uint32_t jn0, jn1;
    ids(r_next, jn0, jn1);

    while (r_cur < n_rounds) {
        // the next round's segment bounds and the round after's spike ids are
        // in flight while this round is processed
        const int r_after = grab();
        uint32_t nb0, nl0, nb1, nl1;
        round_bounds(jn0, jn1, nb0, nl0, nb1, nl1);
        ids(r_after, jn0, jn1);

        events += l0 + l1;
        const uint32_t pair = l0 + l1;
        uint32_t inc = pair;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const uint32_t T = __shfl_sync(0xffffffffu, inc, 31);
        const uint32_t f0 = inc - pair, f1 = f0 + l0;      // run positions of both segments
        const bool nz0 = l0 > 0u, nz1 = l1 > 0u;
        // rank among the round's non-empty segments, in list order
        const uint32_t rank0 = __popc(__ballot_sync(0xffffffffu, nz0) & lanes_lt) +
                               __popc(__ballot_sync(0xffffffffu, nz1) & lanes_lt);
        const uint32_t rank1 = rank0 + (nz0 ? 1u : 0u);
        // entry at run position k of a segment: pre[info + k]
        if (nz0) info[rank0] = b0 - f0;
        if (nz1) info[rank1] = b1 - f1;
        uint32_t rbase = 0u;          // non-empty segments starting before the chunk
        for (uint32_t w0 = 0u; w0 < T; w0 += 32u * kBmWords) {
            for (int q = lane; q < kBmWords; q += 32) bm[q] = 0u;
            __syncwarp();
            if (nz0 && f0 >= w0 && f0 < w0 + 32u * kBmWords)
                atomicOr(&bm[(f0 - w0) >> 5], 1u << (f0 & 31u));
            if (nz1 && f1 >= w0 && f1 < w0 + 32u * kBmWords)
                atomicOr(&bm[(f1 - w0) >> 5], 1u << (f1 & 31u));
            __syncwarp();
            const uint32_t wend = min(T, w0 + 32u * kBmWords);
            // batches of kChunkBatch chunks; the loads of batch i + 1 are
            // issued before the adds of batch i.  A batch stays inside the
            // window; past T the bitmap is zero and loads and adds are
            // predicated off.
            auto load = [&](uint32_t c0, uint32_t (&e)[kChunkBatch]) {
                // the batch's bitmap words, four per broadcast load
                const uint4* bmv = reinterpret_cast<const uint4*>(bm + ((c0 - w0) >> 5));
                uint32_t masks[kChunkBatch];
#pragma unroll
                for (int v = 0; v < kChunkBatch / 4; ++v) {
                    const uint4 m = bmv[v];
                    masks[4 * v] = m.x;
                    masks[4 * v + 1] = m.y;
                    masks[4 * v + 2] = m.z;
                    masks[4 * v + 3] = m.w;
                }
#pragma unroll
                for (int u = 0; u < kChunkBatch; ++u) {
                    const uint32_t mask = masks[u];
                    const uint32_t o = rbase + __popc(mask & lanes_le) - 1u;
                    rbase += __popc(mask);
                    const uint32_t k = c0 + 32u * u + (uint32_t)lane;
                    e[u] = load_entry(dp.pre + (info[o & (kRoundSpikes - 1)] + k), k, T);
                }
            };
            auto add = [&](const uint32_t (&e)[kChunkBatch]) {
                int32_t wt[kChunkBatch];
                uint32_t a[kChunkBatch];
#pragma unroll
                for (int u = 0; u < kChunkBatch; ++u) {
                    wt[u] = s_wt[e[u] >> kPreOffBits];           // kNone reads the last entry
                    if (SMEM_RING) {
                        a[u] = (e[u] & kPreOffMask) - (uint32_t)dp.ncmax;   // sums cell (delay - 1, local)
                    } else {
                        a[u] = (e[u] & kPreOffMask) + base_t;    // ring slot t + delay
                        a[u] = min(a[u], a[u] - (uint32_t)R);    // wrap: a - R is huge when a < R
                    }
                }
#pragma unroll
                for (int u = 0; u < kChunkBatch; ++u) {
                    if (SMEM_RING)
                        add_shared(ring_s + 4u * a[u], wt[u], e[u]);
                    else
                        add_global(ring + a[u], wt[u], e[u]);
                }
            };
            constexpr uint32_t kBatch = 32u * kChunkBatch;
            uint32_t eA[kChunkBatch], eB[kChunkBatch];
            load(w0, eA);
            for (uint32_t c0 = w0; c0 < wend; c0 += 2u * kBatch) {
                const bool more1 = c0 + kBatch < wend, more2 = c0 + 2u * kBatch < wend;
                if (more1) load(c0 + kBatch, eB);
                add(eA);
                if (more2) load(c0 + 2u * kBatch, eA);
                if (more1) add(eB);
            }
            __syncwarp();
        }
        r_cur = r_next;
        r_next = r_after;
        b0 = nb0;
        l0 = nl0;
        b1 = nb1;
        l1 = nl1;
    }
    __syncthreads();
    if (SMEM_RING) {
        // sum of delay d into ring slot t + d (mod 64), zero sums skipped;
        // kFlush cells per thread have their ring words loaded together
        constexpr int kFlush = 8;
        const uint32_t ncm = (uint32_t)dp.ncmax, total = (uint32_t)depth * ncm;
        for (uint32_t k0 = tid; k0 < total; k0 += kWThreads * kFlush) {
            int32_t v[kFlush], old[kFlush];
            uint32_t g[kFlush];
#pragma unroll
            for (int u = 0; u < kFlush; ++u) {
                const uint32_t k = k0 + (uint32_t)u * kWThreads;
                v[u] = k < total ? ring[k] : 0;
                const uint32_t d = k / ncm + 1u, l = k - (d - 1u) * ncm;
                g[u] = (((uint32_t)dp.t + d) & (kRing - 1)) * ncm + l;
            }
#pragma unroll
            for (int u = 0; u < kFlush; ++u) old[u] = v[u] != 0 ? ring_g[g[u]] : 0;
#pragma unroll
            for (int u = 0; u < kFlush; ++u)
                if (v[u] != 0) ring_g[g[u]] = old[u] + v[u];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) events += __shfl_xor_sync(0xffffffffu, events, o);
    if (lane == 0 && events) atomicAdd(&dp.counters[1], events);
}

// One warp per row: entry k of row j from packed word k.  The partition of a
// target is the largest c with floor(c n / P) <= target, the layout the
// network's partitions follow.
__global__ void __launch_bounds__(256)
k_predecode(const __grid_constant__ DeliverParams dp, const unsigned long long* row_start,
            uint32_t* pre) {
    const int j = (int)((blockIdx.x * 256u + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= dp.n) return;
    const uint32_t q = (uint32_t)pop_index(dp.pop_start, dp.n_pop, j);
    const unsigned long long b = row_start[j], e = row_start[j + 1];
    for (unsigned long long k = b + lane; k < e; k += 32) {
        const uint32_t w = dp.words[k];
        const uint32_t tgt = w & kTgtMask;
        const uint32_t c =
            (uint32_t)((((unsigned long long)tgt + 1ull) * (unsigned)dp.n_part - 1ull) / (unsigned)dp.n);
        const uint32_t local = tgt - (uint32_t)dp.part_lo[c];
        const uint32_t d = (w >> kTgtBits) & (kRing - 1);
        const uint32_t p = (uint32_t)pop_index(dp.pop_start, dp.n_pop, (int32_t)tgt);
        const uint32_t widx = (p * kMaxPop + q) * kWCodes + (w >> 25);
        pre[k] = (widx << kPreOffBits) | (d * (uint32_t)dp.ncmax + local);
    }
}

}  // namespace

cudaError_t launch_predecode(const DeliverParams& dp, const unsigned long long* row_start,
                             uint32_t* pre, cudaStream_t s) {
    if ((long long)kRing * dp.ncmax >= (long long)kPreOffMask) return cudaErrorInvalidValue;
    const long long threads = (long long)dp.n * 32;
    if (threads > 0) k_predecode<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(dp, row_start, pre);
    return cudaGetLastError();
}

cudaError_t launch_deliver_words(const DeliverParams& dp, cudaStream_t s) {
    if (dp.n_spikes <= 0) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (dp.max_delay < 1 || dp.max_delay >= kRing) return cudaErrorInvalidValue;
    const bool smem_ring = words_smem(dp.ncmax, true, dp.max_delay).total <= (size_t)optin;
    const size_t smem = words_smem(dp.ncmax, smem_ring, dp.max_delay).total;
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    const void* fn = smem_ring ? reinterpret_cast<const void*>(&k_deliver_words<true>)
                               : reinterpret_cast<const void*>(&k_deliver_words<false>);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (smem_ring)
        k_deliver_words<true><<<dp.n_part, kWThreads, smem, s>>>(dp);
    else
        k_deliver_words<false><<<dp.n_part, kWThreads, smem, s>>>(dp);
    return cudaGetLastError();
}

}  // namespace snn
