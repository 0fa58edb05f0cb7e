// deliver_stream.cu -- stand-alone delivery of one long spike list (Sec. 3.1.2:
// row fetch, word decode, ring-buffer add), with each CTA's runs streamed
// into shared memory by the bulk-copy engine.
//
// CTA c owns partition c's ring slice (shared memory) and, as the
// partition-word tiling does, reads for every spike j of the list exactly
// the run of row j that targets partition c, [seg[j][c], seg[j][c + 1]), of
// the pre-decoded rows (weight-table index and ring-cell offset per entry).
// Here the entries do not pass through registers: warp 0 (the producer)
// looks up the runs' bounds and issues one cp.async.bulk copy per run into a
// ring of kStages shared-memory stages, each completed by an mbarrier that
// counts the copied bytes; warps 1.. (the consumers) wait for a stage, add
// every entry of its runs into the ring slice with shared-memory atomics,
// and release the stage through a second mbarrier.  A bulk copy must start
// on a 16-byte boundary and copy a multiple of 16 bytes, so each run is
// copied from its start rounded down to 4 entries to its end rounded up;
// the stage's run table records where in the stage each run's own entries
// start and how many there are.  Every wait is bounded: a wait that runs
// out sets the timeout status and the CTA's abort flag, and the producer
// then waits (bounded) for its copies in flight before the CTA returns.
#include "snn_internal.cuh"

namespace snn {
namespace {

constexpr int kSThreads = 1024;
constexpr int kSConsumers = kSThreads / 32 - 1;   // consumer warps
constexpr int kStages = 4;
constexpr uint32_t kStageEntries = 3584;        // 14 KB of entries per stage
constexpr uint32_t kStageRuns = 512;            // runs per stage (table of 2 KB)
constexpr int kProdBatch = 4;                   // 32-spike groups per producer round
constexpr uint32_t kPopWordsS = kMaxPop * kWCodes;
constexpr uint32_t kWaitLimit = 1u << 22;       // try_wait rounds before giving up
constexpr uint32_t kStatusTimeoutS = 1u;

struct StreamSmem {
    size_t ring, wt, stage, runs, info, bar, misc, total;
};

__host__ __device__ inline StreamSmem stream_smem(int ncmax, int w_span) {
    StreamSmem L;
    size_t o = 0;
    L.ring = o;  o += (size_t)kRing * ncmax * 4;
    L.wt = o;    o += (size_t)w_span * kPopWordsS * 4;
    o = (o + 127) / 128 * 128;
    L.stage = o; o += (size_t)kStages * kStageEntries * 4;
    L.runs = o;  o += (size_t)kStages * kStageRuns * 4;
    L.info = o;  o += (size_t)kStages * 4;
    o = (o + 7) / 8 * 8;
    L.bar = o;   o += (size_t)2 * kStages * 8;          // full[kStages], empty[kStages]
    L.misc = o;  o += 16;                               // abort flag
    L.total = o;
    return L;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0u;
}
// bulk copy of `bytes` (multiple of 16) from global src (16-byte aligned) to
// shared dst (16-byte aligned), completing `bytes` transactions on bar
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// bounded wait for the phase of parity `parity` of bar; false (and the abort
// flag raised) when the limit runs out or another warp raised it
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t* s_abort,
                                          uint32_t* status) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && *s_abort) return false;
    }
    *s_abort = 1u;
    if (status) atomicOr(status, kStatusTimeoutS);
    return false;
}

__global__ void __launch_bounds__(kSThreads, 1)
k_deliver_stream(const __grid_constant__ DeliverParams dp, int w_span) {
    extern __shared__ __align__(128) unsigned char smem[];
    const StreamSmem L = stream_smem(dp.ncmax, w_span);
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t* ring = reinterpret_cast<int32_t*>(smem + L.ring);
    int32_t* s_wt = reinterpret_cast<int32_t*>(smem + L.wt);
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(smem + L.stage);
    uint32_t* s_runs = reinterpret_cast<uint32_t*>(smem + L.runs);
    volatile uint32_t* s_info = reinterpret_cast<volatile uint32_t*>(smem + L.info);
    volatile uint32_t* s_abort = reinterpret_cast<volatile uint32_t*>(smem + L.misc);
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(smem + L.bar);
    auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(kStages + s); };
    const uint32_t stage0 = (uint32_t)__cvta_generic_to_shared(s_stage);

    const int R = kRing * dp.ncmax;
    int32_t* ring_g = dp.ring + (size_t)c * R;
    const uint32_t wbase = (uint32_t)pop_index(dp.pop_start, dp.n_pop, dp.part_lo[c]) * kPopWordsS;
    for (uint32_t k = tid; k < (uint32_t)w_span * kPopWordsS; k += kSThreads)
        s_wt[k] = wbase + k < (uint32_t)(kMaxPop * kPopWordsS) ? __ldg(&dp.wtab[wbase + k]) : 0;
    {   // R = 64 ncmax words: a whole number of 16-byte vectors
        const int4* src = reinterpret_cast<const int4*>(ring_g);
        int4* dst = reinterpret_cast<int4*>(ring);
        for (int k = tid; k < R / 4; k += kSThreads) dst[k] = src[k];
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full(s), 1u);
            mbar_init(empty(s), (uint32_t)kSConsumers);
        }
        *s_abort = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t base_t = ((uint32_t)dp.t & (kRing - 1)) * (uint32_t)dp.ncmax;
    const size_t seg_stride = (size_t)dp.n_part + 1;
    unsigned long long events = 0;

    if (warp == 0) {
        // ------------------------------- producer -------------------------------
        const int n = dp.n_spikes;
        int st = 0;                 // current stage
        uint32_t use = 0;           // uses of all stages so far (stage index = use mod kStages)
        uint32_t fill = 0, nrun = 0;
        bool ok = true;
        // bounds of the next round, loaded one round ahead
        uint32_t nb[kProdBatch], ne[kProdBatch];
        auto load_round = [&](int base, uint32_t (&b)[kProdBatch], uint32_t (&e)[kProdBatch]) {
            uint32_t j[kProdBatch];
#pragma unroll
            for (int u = 0; u < kProdBatch; ++u) {
                const int i = base + 32 * u + lane;
                j[u] = i < n ? __ldg(&dp.spikes[i]) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < kProdBatch; ++u) {
                b[u] = e[u] = 0u;
                if (j[u] != 0xffffffffu) {
                    const uint32_t* sg = dp.seg + (size_t)j[u] * seg_stride + c;
                    b[u] = __ldg(sg);
                    e[u] = __ldg(sg + 1);
                }
            }
        };
        // close the current stage (last: no more stages follow), move on
        auto close_stage = [&](bool last) {
            __syncwarp();
            if (lane == 0) {
                s_info[st] = nrun | (last ? 0x80000000u : 0u);
                mbar_arrive(full(st));
            }
            __syncwarp();
            ++use;
            st = (int)(use % kStages);
            fill = 0;
            nrun = 0;
            // the stage's previous use must have been released by every consumer
            if (!last && use >= (uint32_t)kStages)
                if (!mbar_wait(empty(st), ((use / kStages) - 1u) & 1u, s_abort, dp.status)) ok = false;
        };
        load_round(0, nb, ne);
        for (int base = 0; base < n && ok; base += 32 * kProdBatch) {
            uint32_t b[kProdBatch], e[kProdBatch];
#pragma unroll
            for (int u = 0; u < kProdBatch; ++u) {
                b[u] = nb[u];
                e[u] = ne[u];
            }
            if (base + 32 * kProdBatch < n) load_round(base + 32 * kProdBatch, nb, ne);
#pragma unroll
            for (int u = 0; u < kProdBatch; ++u) {
                const uint32_t len = e[u] - b[u];
                const uint32_t a0 = b[u] & ~3u, a1 = (e[u] + 3u) & ~3u;
                const uint32_t need = len > 0u ? a1 - a0 : 0u;      // entries copied
                bool pending = len > 0u;
                while (ok && __any_sync(0xffffffffu, pending)) {
                    // place the longest prefix of the pending runs that fits
                    uint32_t x = pending ? need : 0u, y = pending ? 1u : 0u;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t xs = __shfl_up_sync(0xffffffffu, x, o);
                        const uint32_t ys = __shfl_up_sync(0xffffffffu, y, o);
                        if (lane >= o) {
                            x += xs;
                            y += ys;
                        }
                    }
                    const bool fits = pending && fill + x <= kStageEntries && nrun + y <= kStageRuns;
                    if (fits) {
                        const uint32_t dst = fill + x - need;          // entry index in the stage
                        const uint32_t slot = nrun + y - 1u;
                        s_runs[(uint32_t)st * kStageRuns + slot] = ((dst + (b[u] - a0)) << 16) | len;
                        const uint32_t bytes = need * 4u;
                        mbar_expect_tx(full(st), bytes);
                        bulk_copy(stage0 + ((uint32_t)st * kStageEntries + dst) * 4u, dp.pre + a0, bytes,
                                  full(st));
                        pending = false;
                    }
                    const unsigned placed = __ballot_sync(0xffffffffu, fits);
                    if (placed) {
                        const int last_lane = 31 - __clz((int)placed);
                        fill += __shfl_sync(0xffffffffu, x, last_lane);
                        nrun += __shfl_sync(0xffffffffu, y, last_lane);
                    }
                    if (__any_sync(0xffffffffu, pending)) close_stage(false);
                }
            }
        }
        close_stage(true);
        // before returning: the copies of every stage issued must have landed
        // (normally the consumers have waited for them already)
        if (!ok && lane == 0) {
            for (uint32_t k = use > (uint32_t)kStages ? use - kStages : 0u; k < use; ++k)
                mbar_wait(full((int)(k % kStages)), (k / kStages) & 1u, s_abort, nullptr);
        }
    } else {
        // ------------------------------- consumers ------------------------------
        const int cw = warp - 1;
        const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
        for (uint32_t k = 0;; ++k) {
            const int s = (int)(k % kStages);
            if (!mbar_wait(full(s), (k / kStages) & 1u, s_abort, dp.status)) break;
            const uint32_t info = s_info[s];
            const uint32_t nr = info & 0x7fffffffu;
            const uint32_t* runs = s_runs + (uint32_t)s * kStageRuns;
            const uint32_t* ent = s_stage + (uint32_t)s * kStageEntries;
            for (uint32_t r = (uint32_t)cw; r < nr; r += kSConsumers) {
                const uint32_t pk = runs[r];
                const uint32_t off = pk >> 16, len = pk & 0xffffu;
                for (uint32_t q = (uint32_t)lane; q < len; q += 32u) {
                    const uint32_t x = ent[off + q];
                    const int32_t w = s_wt[(x >> kPreOffBits) - wbase];
                    uint32_t a = (x & kPreOffMask) + base_t;
                    a = min(a, a - (uint32_t)R);                  // wrap into the 64-slot ring
                    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(ring_s + 4u * a), "r"(w) : "memory");
                }
                if (lane == 0) events += len;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(s));
            if (info & 0x80000000u) break;
        }
    }
    __syncthreads();
    {
        const int4* src = reinterpret_cast<const int4*>(ring);
        int4* dst = reinterpret_cast<int4*>(ring_g);
        for (int k = tid; k < R / 4; k += kSThreads) dst[k] = src[k];
    }
    if (lane == 0 && events) atomicAdd(&dp.counters[1], events);
}

}  // namespace

size_t deliver_stream_smem(int ncmax, int w_span) { return stream_smem(ncmax, w_span).total; }

cudaError_t launch_deliver_stream(const DeliverParams& dp, int w_span, cudaStream_t s) {
    if (dp.n_spikes <= 0) return cudaSuccess;
    if ((long long)kRing * dp.ncmax >= (long long)kPreOffMask || (uint32_t)dp.ncmax > 0xffffu)
        return cudaErrorInvalidValue;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = stream_smem(dp.ncmax, w_span).total;
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(k_deliver_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_deliver_stream<<<dp.n_part, kSThreads, smem, s>>>(dp, w_span);
    return cudaGetLastError();
}

}  // namespace snn
