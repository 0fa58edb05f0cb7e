// adjoint_part.cu -- the surrogate-gradient adjoint (the recursion of grad.cu,
// Sec. 2.1 Eq. 1 run backwards) with its row gather done partition by
// partition, for networks whose rows fit in the SMs' shared memory.
//
// The gather of step t is ds_j = gs + sum over row j of (w / 256) lI_{i,t+d}.
// Only its delay-1 entries need step t + 1's lI; the rest ("far", delay >= 2)
// is computed while the grid barrier of step t + 1 completes (a split
// barrier: arrive, far gather of step t, wait), the near part after it.
// Gathered from a global lI ring, it costs one L2 request per synapse and
// step.  Here the targets are split into the network's partitions and the
// sources of each partition into G groups: CTA (c, g) keeps, for the whole
// launch, the lI window of partition c (slots t + 1 .. t + R - 1 of its
// neurons) and the runs of its source group into c (the pre-decoded entries,
// re-packed as weight index and window cell offset) in shared memory.  Its
// share of the gather then reads shared memory only.  Each source's partial
// sum over its run into c goes to a global array; after the step's grid
// barrier every CTA of partition c adds the partials of its partition's
// neurons over all partitions (a fixed order) and runs the membrane adjoint of
// those neurons itself -- redundantly in the G CTAs, identically -- so the
// lI_t it writes into its window needs no second barrier.  The CTA of group 0
// alone writes the outputs (the lI ring, the nu sums and, at the end, the
// adjoint state).
//
// A lane takes one source, or one chunk of a source's run when the run is
// longer than kApChunk entries (up to kApMaxChunks chunks in consecutive
// lanes, added in chunk order by the first): every sum has a fixed order.
// Sources are sorted by chunk length, dealt to the groups in snake order and
// packed 32 lanes to a lane group, their entries stored column by column
// (entry k of lane l at k * 32 + l), so that a warp walks 32 runs of similar
// length with conflict-free entry loads.  A run shorter than its group's longest is padded
// with entries of weight zero (exact: x + 0 * lI = x for the finite lI), so
// the walk has no per-entry test and its loads pipeline.  Lane groups are
// dealt to the warps longest first, each to the least loaded warp.
#include <algorithm>
#include <vector>

#include "snn_internal.cuh"

namespace snn {
namespace {

constexpr int kApThreads = 512;
constexpr int kApWarps = kApThreads / 32;
constexpr uint32_t kApNone = 0xffffffffu;
constexpr uint32_t kApWBits = 19;            // weight index << 19 | window cell offset
constexpr uint32_t kApOffMask = (1u << kApWBits) - 1u;
constexpr uint32_t kApChunk = 32;           // entries per lane before a run is split
constexpr uint32_t kApMaxChunks = 4;         // lanes one source's run is split over
constexpr int kApPre = 4;                    // neurons per thread in the membrane phase (ncmax <= 2048)
constexpr int kApHeader = 8;                 // n_lg, nc, p_lo, span, e_off, 0, 0, 0
// header, then for the entries of delay >= 2 ("far") lenmax[n_lg] and
// ebase[n_lg], for those of delay 1 ("near") lenmax[n_lg] and ebase[n_lg],
// src[32 n_lg], chunks[32 n_lg] (m on a source's first lane, else 0),
// warp_first[kApWarps + 1], lg_order[n_lg], then the entries at e_off

__global__ void __launch_bounds__(kApThreads, 1)
k_adjoint_part(const __grid_constant__ AdjPartParams p) {
    extern __shared__ __align__(16) uint32_t s_img[];
    __shared__ volatile uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = (int)blockIdx.x / p.groups, g = (int)blockIdx.x % p.groups;
    const uint32_t ncmax = (uint32_t)p.ncmax, R = (uint32_t)p.ring_r;
    // window rows padded to whole 32-word bank rounds: a cell's bank is
    // its target's, whatever the slot (the plan orders entries by it)
    const uint32_t ws = (ncmax + 31u) & ~31u;
    const size_t n = (size_t)p.n;
    // shared memory: the image [img_max], the window [R][ws], the weights
    // of the partition's target populations (forward, pA; base) and the
    // adjoint state of its neurons
    float* win = reinterpret_cast<float*>(s_img + p.img_max);
    float* wf = win + (size_t)R * ws;
    float* wb = wf + (size_t)p.span_max * kMaxPop * kWCodes + 4;
    // one zero past each table: the weight of the padding entries
    const uint32_t w_zero = (uint32_t)p.span_max * kMaxPop * kWCodes;
    float* s_lu = wb + w_zero + 4;
    float* s_lI = s_lu + ncmax;
    float* s_far = s_lI + ncmax;                 // [max_lg][32] far sums of the lanes
    // group 0: the nu sums of the partition's neurons, accumulated here in
    // the order the global ones would be, read in at the start, written at the end
    double* s_gN = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(s_far + (size_t)p.max_lg * 32) + 7) & ~uintptr_t(7));
    uint8_t* s_mn = reinterpret_cast<uint8_t*>(s_gN + ncmax);

    if (tid == 0) s_abort = 0u;
    {
        const uint32_t o0 = p.img_off[blockIdx.x], words = p.img_off[blockIdx.x + 1] - o0;
        const uint4* src = reinterpret_cast<const uint4*>(p.img + o0);   // offsets are multiples of 4
        uint4* dst = reinterpret_cast<uint4*>(s_img);
        for (uint32_t k = tid; k < words / 4; k += kApThreads) dst[k] = __ldg(&src[k]);
    }
    __syncthreads();
    const uint32_t n_lg = s_img[0], nc = s_img[1], p_lo = s_img[2], span = s_img[3];
    const uint32_t* lenmax = s_img + kApHeader;      // far columns
    const uint32_t* ebase = lenmax + n_lg;
    const uint32_t* lenmax_n = ebase + n_lg;         // near columns
    const uint32_t* ebase_n = lenmax_n + n_lg;
    const uint32_t* srcs = ebase_n + n_lg;
    const uint32_t* lens = srcs + 32 * n_lg;
    const uint32_t* warp_first = lens + 32 * n_lg;
    const uint32_t* lg_order = warp_first + kApWarps + 1;
    const uint32_t* ent = s_img + s_img[4];
    const int32_t lo = p.part_lo[c];
    for (uint32_t k = tid; k < span * kMaxPop * kWCodes; k += kApThreads) {
        const uint32_t gk = p_lo * kMaxPop * kWCodes + k;
        wf[k] = __fmul_rn(__int2float_rn(__ldg(&p.wtab[gk])), 0.00390625f);
        wb[k] = __ldg(&p.wbase[gk]);
    }
    if (tid < 4) {
        wf[w_zero + tid] = 0.f;
        wb[w_zero + tid] = 0.f;
    }
    for (uint32_t i = tid; i < nc; i += kApThreads) {
        s_lu[i] = p.lu[lo + i];
        s_lI[i] = p.lI[lo + i];
        s_mn[i] = p.mnext[lo + i];
        if (g == 0) s_gN[i] = p.gN[lo + i];
    }
    // the window of the first step processed, t_top: lI of steps t_top + d
    const int64_t t_top = p.t_first + p.len - 1;
    for (uint32_t k = tid; k < (R - 1) * nc; k += kApThreads) {
        const uint32_t d = 1 + k / nc, i = k - (d - 1) * nc;
        const int64_t tt = t_top + d;
        win[(uint32_t)(tt % R) * ws + i] = __ldcg(&p.lring[(size_t)(tt & (kRing - 1)) * n + lo + i]);
    }
    __syncthreads();

    const uint32_t RW = R * ws;               // window words
    // The gather of step tt, far (delay >= 2: window steps tt + 2 .. , all
    // final before step tt + 1's membrane phase) or near (delay 1: step tt +
    // 1).  The far sums wait in s_far; the near walk adds them, combines a
    // source's chunks and writes its partial.  Spiking sources' weight
    // partials go to gAc after each walk.
    auto walk = [&](int64_t tt, uint32_t tDt, bool far) {
        const uint8_t* flt = p.tr_f + (size_t)(tt - p.t_first) * n;
        const uint32_t base_t = tDt * ws;
        for (uint32_t wl = warp_first[warp]; wl < warp_first[warp + 1]; ++wl) {
            const uint32_t L = lg_order[wl];
            const uint32_t j = srcs[L * 32 + lane];
            const uint32_t lm = far ? lenmax[L] : lenmax_n[L];
            const uint32_t eb = far ? ebase[L] : ebase_n[L];
            const bool spk = j != kApNone && (flt[j] & 1u) != 0u;
            float acc = 0.f;
            float pa[kMaxPop];
#pragma unroll
            for (int k = 0; k < kMaxPop; ++k) pa[k] = 0.f;
            const uint32_t* ep = ent + eb + lane;
            // entry: weight index << 19 | delay * ws + target; the window
            // cell of step tt + delay is that offset plus tt's row, wrapped
#pragma unroll 4
            for (uint32_t k = 0; k < lm; ++k) {
                const uint32_t e = ep[k * 32];
                const uint32_t wi = e >> kApWBits;
                uint32_t a = base_t + (e & kApOffMask);
                a -= a >= RW ? RW : 0u;
                const float lv = win[a];
                acc = __fadd_rn(acc, __fmul_rn(wf[wi], lv));
                if (spk) {
                    const float v = __fmul_rn(wb[wi], lv);
                    const uint32_t pr = wi / (kMaxPop * kWCodes);
#pragma unroll
                    for (int kk = 0; kk < kMaxPop; ++kk) pa[kk] = __fadd_rn(pa[kk], kk == (int)pr ? v : 0.f);
                }
            }
            // the chunks of a source sit in consecutive lanes; its first lane
            // (m > 0) adds them in chunk order
            const uint32_t m = lens[L * 32 + lane];
            if (far) {
                s_far[L * 32 + lane] = acc;
            } else {
                acc = __fadd_rn(s_far[L * 32 + lane], acc);
                float tot = acc;
#pragma unroll
                for (uint32_t r = 1; r < kApMaxChunks; ++r) {
                    const float v = __shfl_down_sync(0xffffffffu, acc, r);
                    if (r < m) tot = __fadd_rn(tot, v);
                }
                if (m > 0u) {
                    float* pds = p.pds + (size_t)(tt & 1) * p.n_part * n;
                    __stcg(&pds[(size_t)c * n + j], tot);
                }
            }
            if (__any_sync(0xffffffffu, spk)) {
#pragma unroll
                for (int kk = 0; kk < kMaxPop; ++kk) {
                    float t2 = pa[kk];
#pragma unroll
                    for (uint32_t r = 1; r < kApMaxChunks; ++r) {
                        const float v = __shfl_down_sync(0xffffffffu, pa[kk], r);
                        if (r < m) t2 = __fadd_rn(t2, v);
                    }
                    pa[kk] = t2;
                }
                if (m > 0u && spk) {
                    double* ga = p.gAc + ((size_t)c * n + j) * kMaxPop;
#pragma unroll
                    for (int kk = 0; kk < kMaxPop; ++kk)
                        if ((uint32_t)kk < span) ga[kk] += (double)pa[kk];
                }
            }
        }
    };
    // split grid barrier: every CTA arrives once its partials are written,
    // does the next step's far gather, then waits
    uint32_t gen = 0;
    auto arrive = [&]() {
        __syncthreads();
        if (tid == 0) red_release_gpu_add(p.barrier, 1u);
    };
    auto wait = [&]() -> bool {
        if (tid == 0) {
            const uint32_t target = (gen + 1u) * gridDim.x;
            const uint64_t t_start = globaltimer_ns();
            uint32_t iter = 0;
            while (ld_acquire_gpu(p.barrier) < target) {
                if ((++iter & 255u) == 0u) {
                    if (ld_relaxed_gpu(p.abort_flag) != 0u) { s_abort = 1u; break; }
                    if (globaltimer_ns() - t_start > p.timeout_ns) {
                        atomicOr(p.status, kStatusTimeout);
                        atomicExch(p.abort_flag, 1u);
                        s_abort = 1u;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        ++gen;
        return s_abort == 0u;
    };

    uint32_t tD = (uint32_t)(t_top % R);      // window slot of step t
    // step t_top's gather, both parts, before the first barrier
    walk(t_top, tD, true);
    __syncwarp();
    walk(t_top, tD, false);
    arrive();
    for (int s = p.len - 1; s >= 0; --s) {
        const int64_t t = p.t_first + s;
        const uint32_t tD1 = tD == 0u ? R - 1u : tD - 1u;     // window slot of step t - 1
        // this step's trace of the partition's neurons, loaded before the wait
        const uint8_t* fl = p.tr_f + (size_t)s * n;
        const float* ut = p.tr_u + (size_t)s * n;
        float u_pre[kApPre];
        uint8_t f_pre[kApPre];
#pragma unroll
        for (int k = 0; k < kApPre; ++k) {
            const uint32_t i = (uint32_t)tid + (uint32_t)k * kApThreads;
            u_pre[k] = i < nc ? ut[lo + i] : 0.f;
            f_pre[k] = i < nc ? fl[lo + i] : (uint8_t)0;
        }
        // the far part of step t - 1's gather while the other CTAs arrive
        if (s > 0) walk(t - 1, tD1, true);
        if (!wait()) break;
        // ---- membrane and current adjoints of partition c's neurons ----
        float* pds_all = p.pds + (size_t)(t & 1) * p.n_part * n;
#pragma unroll
        for (int kp = 0; kp < kApPre; ++kp) {
            const uint32_t i = (uint32_t)tid + (uint32_t)kp * kApThreads;
            if (i >= nc) break;
            const int32_t gi = lo + (int32_t)i;
            float acc = 0.f;
            for (int cc = 0; cc < p.n_part; ++cc) acc = __fadd_rn(acc, __ldcg(&pds_all[(size_t)cc * n + gi]));
            const float ds = __fadd_rn(p.gs[pop_index(p.pop_start, p.n_pop, gi)], acc);
            const uint8_t f = f_pre[kp];
            const bool mn = s_mn[i] != 0u;
            const float lu1 = s_lu[i];
            const float lub = mn ? __fmul_rn(p.P22, lu1) : 0.f;
            const float lIt = __fadd_rn(__fmul_rn(p.P11, s_lI[i]), mn ? __fmul_rn(p.P21, lu1) : 0.f);
            const float sv = (f & 1u) ? 1.f : 0.f;
            const float x = __fsub_rn(u_pre[kp], p.theta);
            const float a = __fadd_rn(1.0f, __fmul_rn(10.0f, fabsf(x)));
            const float slope = __fdiv_rn(1.0f, __fmul_rn(a, a));
            s_lu[i] = __fadd_rn(__fmul_rn(ds, slope), __fmul_rn(__fsub_rn(1.f, sv), lub));
            s_lI[i] = lIt;
            s_mn[i] = (uint8_t)((f >> 1) & 1u);
            win[tD * ws + i] = lIt;
            if (g == 0) s_gN[i] += (double)lIt;
        }
        __syncthreads();
        // the near part of step t - 1's gather (it reads step t), its partials
        if (s > 0) {
            walk(t - 1, tD1, false);
            arrive();
        }
        tD = tD1;
    }
    if (g == 0 && s_abort == 0u) {
        for (uint32_t i = tid; i < nc; i += kApThreads) {
            p.lu[lo + i] = s_lu[i];
            p.lI[lo + i] = s_lI[i];
            p.mnext[lo + i] = s_mn[i];
            p.gN[lo + i] = s_gN[i];
        }
        // the lI ring of the next launch (the segment before): steps t_first
        // .. t_first + R - 2, which the window holds now
        for (uint32_t k = tid; k < (R - 1) * nc; k += kApThreads) {
            const uint32_t d = k / nc, i = k - d * nc;
            const int64_t tt = p.t_first + d;
            p.lring[(size_t)(tt & (kRing - 1)) * n + lo + i] = win[(uint32_t)(tt % R) * ws + i];
        }
    }
}

// gA[j][p] += the partition partials of source j, partitions in order
__global__ void __launch_bounds__(256) k_adjoint_part_fold(int32_t n, int32_t n_part, int32_t n_pop,
                                                           const int32_t* __restrict__ part_lo,
                                                           const int32_t* __restrict__ pop_start,
                                                           const double* __restrict__ gAc,
                                                           double* __restrict__ gA) {
    const int32_t j = (int32_t)(blockIdx.x * 256u + threadIdx.x);
    if (j >= n) return;
    int32_t ps[kMaxPop + 1];
    for (int k = 0; k <= kMaxPop; ++k) ps[k] = pop_start[k];
    for (int c = 0; c < n_part; ++c) {
        if (part_lo[c + 1] <= part_lo[c]) continue;
        const int p_lo = pop_index(ps, n_pop, part_lo[c]);
        const double* src = gAc + ((size_t)c * n + j) * kMaxPop;
        for (int k = 0; p_lo + k < kMaxPop; ++k) gA[(size_t)j * kMaxPop + p_lo + k] += src[k];
    }
}

}  // namespace

int adjoint_part_plan(int n, int n_pop, const int32_t* pop_start, int n_part, const int32_t* part_lo,
                      int ncmax, uint64_t nnz, const unsigned long long* d_row_start,
                      const uint32_t* d_pre, const uint32_t* d_seg, AdjPartPlan* plan) {
    *plan = AdjPartPlan();
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return -1;
    const int G = sms / std::max(1, n_part);
    if (G < 1 || ncmax > kApPre * kApThreads || n <= 0) return 1;
    // each CTA's share of the rows must fit next to the window and the tables
    if ((double)nnz * 4.0 / ((double)n_part * G) > (double)optin * 0.7) return 1;
    std::vector<unsigned long long> rs(n + 1);
    std::vector<uint32_t> pre(nnz), seg((size_t)n * (n_part + 1));
    if (cudaMemcpy(rs.data(), d_row_start, sizeof(unsigned long long) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (nnz && cudaMemcpy(pre.data(), d_pre, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        cudaMemcpy(seg.data(), d_seg, sizeof(uint32_t) * seg.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    auto pop_of = [&](int32_t i) {
        int q = 0;
        for (int k = 1; k < n_pop; ++k) q += i >= pop_start[k] ? 1 : 0;
        return q;
    };
    // target populations per partition; the padding entries index the zero
    // past the widest partition's table, which must fit the 13-bit index
    int span_max = 1;
    for (int c = 0; c < n_part; ++c)
        if (part_lo[c + 1] > part_lo[c])
            span_max = std::max(span_max, pop_of(part_lo[c + 1] - 1) - pop_of(part_lo[c]) + 1);
    const uint32_t w_zero = (uint32_t)span_max * kMaxPop * kWCodes;
    if (w_zero >= (1u << (32 - kApWBits))) return 1;
    // window rows padded to whole bank rounds (as the kernel does)
    const uint32_t wsp = ((uint32_t)ncmax + 31u) & ~31u;
    if ((size_t)kRing * wsp > kApOffMask) return 1;
    const uint32_t e_pad = (w_zero << kApWBits) | wsp;            // delay 1, target 0, weight 0
    const uint32_t e_pad_far = (w_zero << kApWBits) | (2u * wsp);  // delay 2
    std::vector<uint32_t> img;
    std::vector<uint32_t> off(1, 0u);
    int R = 2;
    size_t img_max = 0;
    uint32_t max_lg = 0;
    for (int c = 0; c < n_part; ++c) {
        const int32_t nc = part_lo[c + 1] - part_lo[c];
        const int p_lo = nc > 0 ? pop_of(part_lo[c]) : 0;
        const int span = nc > 0 ? pop_of(part_lo[c + 1] - 1) - p_lo + 1 : 1;
        auto run_len = [&](int32_t j) {
            const uint32_t* sg = seg.data() + (size_t)j * (n_part + 1) + c;
            return sg[1] - sg[0];
        };
        // a source is one unit of m <= kApMaxChunks lanes: its run in chunks
        // of at most kApChunk entries (as equal as possible), one per lane
        struct Unit {
            int32_t j;
            uint32_t m, clen;                 // chunks, entries of the longest chunk
        };
        std::vector<Unit> units(n);
        for (int32_t j = 0; j < n; ++j) {
            const uint32_t len = run_len(j);
            const uint32_t m = std::min<uint32_t>(kApMaxChunks, std::max<uint32_t>(1u, (len + kApChunk - 1) / kApChunk));
            units[j] = Unit{j, m, (len + m - 1) / m};
        }
        // longest chunks first, dealt to the G groups in snake order (0 .. G-1,
        // G-1 .. 0, ...): every group gets the same mix of chunk lengths
        std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.clen > y.clen; });
        std::vector<std::vector<Unit>> groups(G);
        for (int32_t k = 0; k < n; ++k) {
            const int r = k % G, lap = k / G;
            groups[(lap & 1) ? G - 1 - r : r].push_back(units[k]);
        }
        for (int g = 0; g < G; ++g) {
            // lanes: source, chunk, entries; a unit never straddles two lane groups
            struct Lane {
                int32_t j;
                uint32_t m, k0, len;          // m on the unit's first lane only
            };
            std::vector<Lane> lanes;
            for (const Unit& u : groups[g]) {
                if (lanes.size() % 32 + u.m > 32)
                    while (lanes.size() % 32) lanes.push_back(Lane{-1, 0u, 0u, 0u});
                const uint32_t len = run_len(u.j);
                for (uint32_t q = 0; q < u.m; ++q) {
                    const uint32_t k0 = std::min(len, q * u.clen);
                    lanes.push_back(Lane{u.j, q == 0 ? u.m : 0u, k0, std::min(len, k0 + u.clen) - k0});
                }
            }
            const uint32_t n_lg = (uint32_t)((lanes.size() + 31) / 32);
            while (lanes.size() < (size_t)n_lg * 32) lanes.push_back(Lane{-1, 0u, 0u, 0u});
            const size_t o_wf = kApHeader + 4 * (size_t)n_lg + 64 * (size_t)n_lg;
            std::vector<uint32_t> head(o_wf + kApWarps + 1 + n_lg, 0u);
            head[0] = n_lg;
            head[1] = (uint32_t)nc;
            head[2] = (uint32_t)p_lo;
            head[3] = (uint32_t)span;
            std::vector<uint32_t> ents;
            for (uint32_t L = 0; L < n_lg; ++L) {
                // each lane's entries, re-packed, far (delay >= 2) and near (1)
                std::vector<uint32_t> le[2][32];
                for (uint32_t l = 0; l < 32; ++l) {
                    const Lane& ln = lanes[L * 32 + l];
                    for (uint32_t k = 0; ln.j >= 0 && k < ln.len; ++k) {
                        const uint32_t pe = pre[seg[(size_t)ln.j * (n_part + 1) + c] + ln.k0 + k];
                        const uint32_t off_e = pe & kPreOffMask;
                        const uint32_t d = off_e / (uint32_t)ncmax, loc = off_e % (uint32_t)ncmax;
                        const uint32_t wi = (pe >> kPreOffBits) - (uint32_t)p_lo * kMaxPop * kWCodes;
                        if (d < 1 || d >= (uint32_t)kRing || (int32_t)loc >= nc ||
                            wi >= (uint32_t)span * kMaxPop * kWCodes)
                            return -2;
                        R = std::max(R, (int)d + 1);
                        le[d == 1u ? 1 : 0][l].push_back((wi << kApWBits) | (d * wsp + loc));
                    }
                }
                for (int part = 0; part < 2; ++part) {
                    uint32_t lm = 0;
                    for (uint32_t l = 0; l < 32; ++l) lm = std::max(lm, (uint32_t)le[part][l].size());
                    head[kApHeader + 2 * part * n_lg + L] = lm;
                    head[kApHeader + (2 * part + 1) * n_lg + L] = (uint32_t)ents.size();
                    // padding: weight zero, a valid window cell of the part's delays
                    const uint32_t pad = part == 0 ? e_pad_far : e_pad;
                    // The order of a lane's entries is free (its sum has a
                    // fixed order either way): column k takes from each lane
                    // an entry whose weight bank (weight index mod 32) and
                    // window bank (target mod 32) no lane of the column used
                    // yet, if it has one; a lane with spare columns may wait
                    // (a zero-weight entry) rather than collide.  Lanes with
                    // the most entries left choose first.
                    std::vector<uint32_t>* lp = le[part];
                    for (uint32_t k = 0; k < lm; ++k) {
                        uint32_t used_w = 0u, used_l = 0u;
                        uint32_t col[32];
                        int ord[32];
                        for (int l = 0; l < 32; ++l) {
                            col[l] = pad;
                            ord[l] = l;
                        }
                        std::stable_sort(ord, ord + 32, [&](int x, int y) { return lp[x].size() > lp[y].size(); });
                        for (int oi = 0; oi < 32; ++oi) {
                            const int l = ord[oi];
                            if (lp[l].empty()) continue;
                            size_t best = 0;
                            int best_cost = 3;
                            for (size_t q = 0; q < lp[l].size(); ++q) {
                                const uint32_t e = lp[l][q];
                                const int cost = (int)((used_w >> ((e >> kApWBits) & 31u)) & 1u) +
                                                 (int)((used_l >> (e & 31u)) & 1u);
                                if (cost < best_cost) {
                                    best_cost = cost;
                                    best = q;
                                    if (cost == 0) break;
                                }
                            }
                            const bool slack = lp[l].size() < (size_t)(lm - k);
                            if (best_cost > 0 && slack) continue;
                            const uint32_t e = lp[l][best];
                            lp[l][best] = lp[l].back();
                            lp[l].pop_back();
                            used_w |= 1u << ((e >> kApWBits) & 31u);
                            used_l |= 1u << (e & 31u);
                            col[l] = e;
                        }
                        for (int l = 0; l < 32; ++l) ents.push_back(col[l]);
                    }
                }
            }
            for (uint32_t l = 0; l < 32 * n_lg; ++l) {
                head[kApHeader + 4 * n_lg + l] = lanes[l].j >= 0 ? (uint32_t)lanes[l].j : kApNone;
                head[kApHeader + 4 * n_lg + 32 * n_lg + l] = lanes[l].m;
            }
            // lane groups to warps, longest first, each to the least loaded warp
            std::vector<std::vector<uint32_t>> per_warp(kApWarps);
            std::vector<unsigned long long> load(kApWarps, 0ull);
            for (uint32_t L = 0; L < n_lg; ++L) {
                const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                per_warp[w].push_back(L);
                load[w] += head[kApHeader + L] + head[kApHeader + 2 * n_lg + L] + 1ull;
            }
            uint32_t pos = 0;
            for (int w = 0; w < kApWarps; ++w) {
                head[o_wf + w] = pos;
                for (uint32_t L : per_warp[w]) head[o_wf + kApWarps + 1 + pos++] = L;
            }
            head[o_wf + kApWarps] = pos;
            while (head.size() % 4) head.push_back(0u);
            head[4] = (uint32_t)head.size();
            head.insert(head.end(), ents.begin(), ents.end());
            while (head.size() % 4) head.push_back(0u);
            img.insert(img.end(), head.begin(), head.end());
            off.push_back((uint32_t)img.size());
            img_max = std::max(img_max, head.size());
            max_lg = std::max(max_lg, n_lg);
        }
    }
    const size_t ws = ((size_t)ncmax + 31) / 32 * 32;
    const size_t smem = img_max * 4 + (size_t)R * ws * 4 + (size_t)2 * (span_max * kMaxPop * kWCodes + 4) * 4 +
                        (size_t)ncmax * 8 + (size_t)max_lg * 32 * 4 + 8 + (size_t)ncmax * 8 + (size_t)ncmax;
    if (smem > (size_t)optin) return 1;
    plan->grid = n_part * G;
    plan->groups = G;
    plan->ring_r = R;
    plan->span_max = span_max;
    plan->img_max = (int32_t)img_max;
    plan->max_lg = (int32_t)max_lg;
    plan->smem = smem;
    cudaError_t e = cudaMalloc(&plan->d_img, sizeof(uint32_t) * std::max<size_t>(img.size(), 4));
    if (e == cudaSuccess) e = cudaMalloc(&plan->d_img_off, sizeof(uint32_t) * off.size());
    if (e == cudaSuccess) e = cudaMemcpy(plan->d_img, img.data(), sizeof(uint32_t) * img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(plan->d_img_off, off.data(), sizeof(uint32_t) * off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_adjoint_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint_part, kApThreads, smem);
    if (e != cudaSuccess || per_sm * sms < plan->grid) {
        adjoint_part_free(plan);
        cudaGetLastError();
        return e != cudaSuccess ? -1 : 1;
    }
    return 0;
}

void adjoint_part_free(AdjPartPlan* plan) {
    if (plan->d_img) cudaFree(plan->d_img);
    if (plan->d_img_off) cudaFree(plan->d_img_off);
    *plan = AdjPartPlan();
}

cudaError_t launch_adjoint_part(const AdjPartPlan& plan, AdjPartParams& ap, cudaStream_t s) {
    ap.groups = plan.groups;
    ap.ring_r = plan.ring_r;
    ap.span_max = plan.span_max;
    ap.img_max = plan.img_max;
    ap.max_lg = plan.max_lg;
    ap.img = plan.d_img;
    ap.img_off = plan.d_img_off;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.grid);
    cfg.blockDim = dim3(kApThreads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {&ap};
    return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&k_adjoint_part), args);
}

cudaError_t launch_adjoint_part_fold(int n, int n_part, int n_pop, const int32_t* part_lo,
                                     const int32_t* pop_start, const double* gAc, double* gA,
                                     cudaStream_t s) {
    k_adjoint_part_fold<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, n_part, n_pop, part_lo, pop_start,
                                                                    gAc, gA);
    return cudaGetLastError();
}

}  // namespace snn
