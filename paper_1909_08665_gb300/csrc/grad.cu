// grad.cu -- gradient of a population-rate loss with respect to the 64
// projection weight scales alpha_pq and the background rate nu, by
// backpropagation through time over the step recursion of Sec. 2.1 (Eq. 1)
// with a surrogate spike derivative.  The paper trains nothing; this is the
// differentiable form of its benchmark network.
//
// Model and choices (the same as the CPU reference's hard model):
//   d s_t / d u_t := 1 / (1 + 10 |u_t - theta|)^2   (fast sigmoid, per mV)
//   reset and refractory are constants of the backward: the post-spike value
//   u (1 - s) with s held fixed, and a refractory step passes no gradient;
//   the fixed-point rounding of alpha w is passed through (d w / d alpha =
//   w_base, the unrounded weight at alpha = 1) and so is the Poisson count
//   (d k / d nu = K_ext dt).
// Adjoint recursion, last step first (lu = dL/du, lI = dL/dI, m_t = 1 when
// step t took the non-refractory update):
//   ds_{j,t} = gs[pop j] + sum over row j of (w / 256) lI_{i, t + d}
//   lu_t = ds_t s'(u_t) + (1 - s_t) m_{t+1} P22 lu_{t+1}
//   lI_t = P11 lI_{t+1} + m_{t+1} P21 lu_{t+1}
//   dL/dalpha_pq += s_{j,t} w_base lI_{i,t+d}  (words of j in q into p)
//   dL/dnu       += lI_{i,t} (w_ext K_ext,p dt)
//
// Memory: the forward keeps one checkpoint of the full state (u, I,
// refractory counters, ring buffers) every `ckpt_every` steps; the backward
// restores each segment's checkpoint, re-runs the segment with the step
// kernel recording u (before reset) and the spike / update flags, then runs
// the adjoint over the segment in one persistent cooperative kernel (one
// grid barrier per step).  When the trace of the whole forward (5 bytes per
// neuron-step) fits the trace budget (4 GiB by default) and a quarter of the
// free device memory, the forward records it directly and the backward
// re-runs nothing.  lI of the last 64 steps lives in an adjoint ring
// [64][n]; per-neuron sums are double and every reduction has a fixed order,
// so results are deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/snn.h"
#include "net.h"
#include "snn_internal.cuh"

using namespace snn;

struct snn_grad {
    int64_t t_start = 0;
    int64_t n_steps = 0;
    int32_t seg = 0;
    int32_t n_seg = 0;
    bool ready = false;
    size_t ring_words = 0;
    size_t ckpt_bytes = 0;
    size_t ckpt_cap = 0;            // checkpoints the buffer holds
    int32_t tr_cap = 0;             // steps the trace buffers hold
    bool full_trace = false;        // the forward recorded every step: no recomputation
    int64_t trace_budget = (int64_t)4 << 30;   // bytes of a whole forward's trace
    uint8_t* ckpt = nullptr;        // [n_seg + 1][u | I | refr | ring]
    float* tr_u = nullptr;          // [seg][n]
    uint8_t* tr_f = nullptr;        // [seg][n]
    float* lu = nullptr;
    float* lI = nullptr;
    float* lring = nullptr;         // [64][n]
    uint8_t* mnext = nullptr;
    double* gA = nullptr;           // [n][8] by target population
    double* gN = nullptr;           // [n]
    float* wbase = nullptr;         // [8][8][128] pA
    double* out = nullptr;          // [65]
    uint32_t* sync = nullptr;       // [0] barrier, [1] status, [2] abort
    unsigned long long* saved = nullptr;   // counters, population counters
    uint32_t* saved_ras = nullptr;  // raster counts
    uint32_t* saved_status = nullptr;
    int32_t* pop_start = nullptr;   // [9]
    int32_t* blk = nullptr;         // [grid + 1] row range of each adjoint CTA
    int32_t* order = nullptr;       // [n] each CTA's rows, longest first
    int32_t grid = 0, chunk = 0;    // CTAs of the adjoint, most rows of one CTA
    uint32_t* pre = nullptr;        // pre-decoded rows of the adjoint gather (small networks)
    bool part_planned = false;      // the partition-local adjoint was considered
    snn::AdjPartPlan* part = nullptr;   // its plan, when the network fits
    float* pds = nullptr;           // [2][P][n] its partial spike adjoints
    double* gAc = nullptr;          // [P][n][8] its partial weight gradients
};

namespace snn {

void free_grad(snn_grad* g) {
    if (!g) return;
    void* ptrs[] = {g->ckpt, g->tr_u, g->tr_f, g->lu, g->lI, g->lring, g->mnext, g->gA, g->gN,
                    g->wbase, g->out, g->sync, g->saved, g->saved_ras, g->saved_status,
                    g->pop_start, g->blk, g->order, g->pre};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->part) {
        adjoint_part_free(g->part);
        delete g->part;
    }
    if (g->pds) cudaFree(g->pds);
    if (g->gAc) cudaFree(g->gAc);
    delete g;
}

void net_base_weights(const snn_net* net, float* wb);

}  // namespace snn

namespace {

constexpr int kAdjThreads = 512;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjUnroll = 8;           // row words per lane in flight
constexpr int kAdjPopTable = 49152;     // largest network with a shared population table

// population of neuron i from the (ascending) starts s_ps[0..8]: binary search
__device__ __forceinline__ int pop_of_sorted(const int32_t* s_ps, int32_t i) {
    int pp = i >= s_ps[4] ? 4 : 0;
    pp += i >= s_ps[pp + 2] ? 2 : 0;
    pp += i >= s_ps[pp + 1] ? 1 : 0;
    return pp;
}

struct AdjParams {
    int32_t n, n_pop, len, chunk;
    const int32_t* blk;              // [grid + 1] row range of each CTA
    const int32_t* order;            // [n] rows of each CTA, longest first
    int32_t pop_start[kMaxPop + 1];
    int64_t t_first;                 // global step of trace row 0
    float P22, P21, P11, theta;
    float gs[kMaxPop];               // dL/ds per spike of each population
    uint64_t timeout_ns;
    const unsigned long long* row_start;
    const uint32_t* words;
    // entry k of row j: (weight-table index << kPreOffBits) | (delay * n + target),
    // the words pre-decoded for the gather (64 n < 2^kPreOffBits)
    const uint32_t* pre;
    const int32_t* wtab;             // rounded weights of the forward, 1/256 pA
    const float* wbase;
    const float* tr_u;
    const uint8_t* tr_f;
    float* lu;
    float* lI;
    float* lring;
    uint8_t* mnext;
    double* gA;
    double* gN;
    uint32_t* barrier;
    uint32_t* status;
    uint32_t* abort_flag;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// fast-sigmoid derivative 1 / (1 + 10 |x|)^2
__device__ __forceinline__ float surrogate_slope(float x) {
    const float a = __fadd_rn(1.0f, __fmul_rn(10.0f, fabsf(x)));
    return __fdiv_rn(1.0f, __fmul_rn(a, a));
}

// The adjoint of trace rows len-1 .. 0.  CTA b owns neurons [blk[b],
// blk[b + 1]) (ranges balanced by total row length): their rows in the spike
// phase, taken by the warps longest first, and their state in the membrane
// phase; one grid barrier per step separates the lI writes of step t from the
// row gathers of step t - 1.  PRE: the rows are read from the pre-decoded
// copy (weight-table index and ring offset per synapse), which takes the
// population lookup and the slot arithmetic off the gather; every value and
// every sum is the same as in the packed-word path.
template <bool PRE>
__global__ void __launch_bounds__(kAdjThreads, 1) k_adjoint(const __grid_constant__ AdjParams p) {
    // dynamic shared memory: the forward's weights in pA and the base weights
    // ([8][8][128] each: random lookups stay off the L1 wavefront budget), the
    // row starts of the CTA's rows [chunk + 1] (u64) and the spike adjoints of
    // the current step [chunk]
    extern __shared__ unsigned long long s_dyn[];
    float* s_wf = reinterpret_cast<float*>(s_dyn);
    float* s_wb = s_wf + kMaxPop * kMaxPop * kWCodes;
    unsigned long long* s_rs = reinterpret_cast<unsigned long long*>(s_wb + kMaxPop * kMaxPop * kWCodes);
    float* s_ds = reinterpret_cast<float*>(s_rs + p.chunk + 1);
    // population of every target neuron (one byte each) when the network is
    // small enough, else a search over the population starts
    uint8_t* s_pop = p.n <= kAdjPopTable ? reinterpret_cast<uint8_t*>(s_ds + p.chunk) : nullptr;
    __shared__ int32_t s_ps[kMaxPop + 1];
    __shared__ volatile uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t lo = p.blk[blockIdx.x];
    const int32_t hi = p.blk[blockIdx.x + 1];
    if (tid == 0) s_abort = 0u;
    for (int32_t j = lo + tid; j <= hi; j += kAdjThreads) s_rs[j - lo] = p.row_start[j];
    if (tid <= kMaxPop) s_ps[tid] = tid == 0 ? 0 : (tid < p.n_pop ? p.pop_start[tid] : 0x7fffffff);
    if (s_pop)
        for (int32_t i = tid; i < p.n; i += kAdjThreads)
            s_pop[i] = (uint8_t)pop_index(p.pop_start, p.n_pop, i);
    const uint32_t n32 = (uint32_t)p.n;
    for (int k = tid; k < kMaxPop * kMaxPop * kWCodes; k += kAdjThreads) {
        s_wf[k] = __fmul_rn(__int2float_rn(__ldg(&p.wtab[k])), 0.00390625f);
        s_wb[k] = __ldg(&p.wbase[k]);
    }
    __syncthreads();
    const size_t n = (size_t)p.n;
    uint32_t gen = 0;
    for (int s = p.len - 1; s >= 0; --s) {
        const int64_t t = p.t_first + s;
        const uint32_t t32 = (uint32_t)t;                 // only t mod 64 is used
        const uint8_t* fl = p.tr_f + (size_t)s * n;
        // ---- spike adjoints: loss term plus the rows' pull from lI(t + d) ----
        for (int32_t r = lo + warp; r < hi; r += kAdjWarps) {
            const int32_t j = __ldg(&p.order[r]);
            const int q = pop_index(p.pop_start, p.n_pop, j);
            const bool spk = (fl[j] & 1u) != 0u;
            // PRE indexes the whole table [p][q][code]; the packed path the
            // source population's block [p][code]
            const float* wq = PRE ? s_wf : s_wf + q * kWCodes;
            const float* bq = PRE ? s_wb : s_wb + q * kWCodes;
            float acc = 0.f;
            float pa[kMaxPop];
#pragma unroll
            for (int k = 0; k < kMaxPop; ++k) pa[k] = 0.f;
            const unsigned long long b = s_rs[j - lo];
            const uint32_t len = (uint32_t)(s_rs[j - lo + 1] - b);
            const uint32_t* rw = (PRE ? p.pre : p.words) + b;
            // kAdjUnroll words per lane in flight: all word loads, then all
            // lI and weight loads, then the (fixed-order) accumulation; the
            // row-relative offsets, ring index and population lookup are 32-bit
            for (uint32_t o = (uint32_t)lane; o < len; o += 32u * kAdjUnroll) {
                uint32_t word[kAdjUnroll];
#pragma unroll
                for (int u = 0; u < kAdjUnroll; ++u) {
                    const uint32_t w = o + 32u * (uint32_t)u;
                    word[u] = w < len ? __ldg(&rw[w]) : 0u;
                }
                float l[kAdjUnroll];
                int idx[kAdjUnroll];
#pragma unroll
                for (int u = 0; u < kAdjUnroll; ++u) {
                    if (PRE) {
                        // (t + d) mod 64 rows of lring: offset + (t mod 64) n, wrapped
                        idx[u] = (int)(word[u] >> kPreOffBits);
                        uint32_t a = (word[u] & kPreOffMask) + (t32 & (kRing - 1)) * n32;
                        a = min(a, a - (uint32_t)kRing * n32);
                        l[u] = o + 32u * (uint32_t)u < len ? __ldcg(&p.lring[a]) : 0.f;
                    } else {
                        const uint32_t tgt = word[u] & kTgtMask;
                        const int pp = s_pop ? (int)s_pop[tgt] : pop_of_sorted(s_ps, (int32_t)tgt);
                        idx[u] = pp * (kMaxPop * kWCodes) + (int)(word[u] >> 25);
                        const uint32_t slot = (t32 + ((word[u] >> kTgtBits) & 63u)) & (kRing - 1);
                        l[u] = o + 32u * (uint32_t)u < len ? __ldcg(&p.lring[slot * n32 + tgt]) : 0.f;
                    }
                }
                if (!spk) {
#pragma unroll
                    for (int u = 0; u < kAdjUnroll; ++u)
                        if (o + 32u * (uint32_t)u < len) acc = __fadd_rn(acc, __fmul_rn(wq[idx[u]], l[u]));
                } else {
#pragma unroll
                    for (int u = 0; u < kAdjUnroll; ++u) {
                        if (o + 32u * (uint32_t)u < len) {
                            acc = __fadd_rn(acc, __fmul_rn(wq[idx[u]], l[u]));
                            const float v = __fmul_rn(bq[idx[u]], l[u]);
                            const int pp = idx[u] / (kMaxPop * kWCodes);
#pragma unroll
                            for (int k = 0; k < kMaxPop; ++k) pa[k] = __fadd_rn(pa[k], k == pp ? v : 0.f);
                        }
                    }
                }
            }
            acc = warp_sum(acc);
            if (spk) {
#pragma unroll
                for (int k = 0; k < kMaxPop; ++k) pa[k] = warp_sum(pa[k]);
            }
            if (lane == 0) {
                s_ds[j - lo] = __fadd_rn(p.gs[q], acc);
                if (spk) {
#pragma unroll
                    for (int k = 0; k < kMaxPop; ++k)
                        if (k < p.n_pop) p.gA[(size_t)j * kMaxPop + k] += (double)pa[k];
                }
            }
        }
        __syncthreads();
        // ---- membrane and current adjoints of step t ----
        const float* ut = p.tr_u + (size_t)s * n;
        for (int32_t i = lo + tid; i < hi; i += kAdjThreads) {
            const uint8_t f = fl[i];
            const bool mn = p.mnext[i] != 0u;
            const float lu1 = p.lu[i];
            const float lub = mn ? __fmul_rn(p.P22, lu1) : 0.f;
            const float lIt = __fadd_rn(__fmul_rn(p.P11, p.lI[i]), mn ? __fmul_rn(p.P21, lu1) : 0.f);
            const float sv = (f & 1u) ? 1.f : 0.f;
            const float lut = __fadd_rn(__fmul_rn(s_ds[i - lo], surrogate_slope(__fsub_rn(ut[i], p.theta))),
                                        __fmul_rn(__fsub_rn(1.f, sv), lub));
            p.lu[i] = lut;
            p.lI[i] = lIt;
            p.mnext[i] = (uint8_t)((f >> 1) & 1u);
            __stcg(&p.lring[(size_t)((uint32_t)t & (kRing - 1)) * n + i], lIt);
            p.gN[i] += (double)lIt;
        }
        if (!grid_barrier(p.barrier, p.abort_flag, p.status, p.timeout_ns, gen, &s_abort, false))
            break;
    }
}

// One warp per row: the adjoint's pre-decoded entries from the packed words
// (source population q of the row, target population p, delay d, code).
__global__ void __launch_bounds__(256) k_adj_predecode(int32_t n, int32_t n_pop,
                                                       const int32_t* pop_start,
                                                       const unsigned long long* row_start,
                                                       const uint32_t* words, uint32_t* pre) {
    const int j = (int)((blockIdx.x * 256u + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const uint32_t q = (uint32_t)pop_index(pop_start, n_pop, j);
    const unsigned long long b = row_start[j], e = row_start[j + 1];
    for (unsigned long long k = b + (unsigned long long)lane; k < e; k += 32ull) {
        const uint32_t w = words[k];
        const uint32_t tgt = w & kTgtMask;
        const uint32_t pp = (uint32_t)pop_index(pop_start, n_pop, (int32_t)tgt);
        const uint32_t widx = (pp * kMaxPop + q) * kWCodes + (w >> 25);
        pre[k] = (widx << kPreOffBits) | (((w >> kTgtBits) & (kRing - 1)) * (uint32_t)n + tgt);
    }
}

// dL/dalpha_pq = sum over j in q of gA[j][p]; dL/dnu = sum_j gN[j] dnu[pop j].
// One CTA per output (64 scales, then nu), each reduced in a fixed order.
__global__ void __launch_bounds__(512) k_grad_reduce(int32_t n, int32_t n_pop,
                                                     const int32_t* __restrict__ pop_start_dev,
                                                     const double* __restrict__ gA,
                                                     const double* __restrict__ gN,
                                                     const double* __restrict__ dnu, double* out) {
    __shared__ double red[512];
    __shared__ int32_t ps[kMaxPop + 1];
    const int tid = threadIdx.x;
    if (tid <= kMaxPop) ps[tid] = pop_start_dev[tid];
    __syncthreads();
    {
        const int o = blockIdx.x;
        double v = 0.0;
        if (o < kMaxPop * kMaxPop) {
            const int p = o / kMaxPop, q = o % kMaxPop;
            if (p < n_pop && q < n_pop)
                for (int32_t j = ps[q] + tid; j < ps[q + 1]; j += 512) v += gA[(size_t)j * kMaxPop + p];
        } else {
            for (int32_t j = tid; j < n; j += 512) v += gN[j] * dnu[pop_index(ps, n_pop, j)];
        }
        red[tid] = v;
        __syncthreads();
        for (int w = 256; w > 0; w >>= 1) {
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        if (tid == 0) out[o] = red[0];
    }
}

#define GCK(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return set_cuda_error(e_, #call);      \
    } while (0)

template <typename T>
int galloc(T** p, size_t count, const char* what) {
    if (*p) return SNN_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(SNN_ERR_OOM, what);
    }
    return SNN_OK;
}

#define GCALL(x)                        \
    do {                                \
        int rc_ = (x);                  \
        if (rc_ != SNN_OK) return rc_;  \
    } while (0)

size_t ring_words(const snn_net* net) { return (size_t)net->P * kRing * net->ncmax; }

size_t state_bytes(const snn_net* net) {
    return (size_t)net->n * 12 + ring_words(net) * sizeof(int32_t);
}

// copy the full device state to / from one checkpoint slot
cudaError_t save_ckpt(snn_net* net, uint8_t* dst) {
    const size_t n = (size_t)net->n;
    cudaStream_t s = net->stream;
    cudaError_t e = cudaMemcpyAsync(dst, net->d_u, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + n * 4, net->d_i, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + n * 8, net->d_r, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst + n * 12, net->d_ring, ring_words(net) * 4, cudaMemcpyDeviceToDevice, s);
    return e;
}

// the spike messages carry step tags: clear them whenever the state is
// rewound, so that no message of an abandoned future can match a tag again
cudaError_t clear_messages(snn_net* net) {
    return cudaMemsetAsync(net->d_msg, 0, sizeof(unsigned long long) * 4 * net->P * net->msg_stride,
                           net->stream);
}

cudaError_t load_ckpt(snn_net* net, const uint8_t* src) {
    const size_t n = (size_t)net->n;
    cudaStream_t s = net->stream;
    cudaError_t e = cudaMemcpyAsync(net->d_u, src, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->d_i, src + n * 4, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->d_r, src + n * 8, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(net->d_ring, src + n * 12, ring_words(net) * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = clear_messages(net);
    if (e == cudaSuccess) e = net_clear_wraps(net);
    return e;
}

constexpr uint64_t kStateMagic = 0x3145544154534e53ull;   // "SNSTATE1"

}  // namespace

extern "C" {

int snn_set_params(snn_net* net, const double* scales, double nu_bg) {
    if (!net || !scales) return set_error(SNN_ERR_INVALID, "bad arguments");
    snn_config c = net->cfg;
    for (int p = 0; p < kMaxPop; ++p)
        for (int q = 0; q < kMaxPop; ++q) {
            const double a = scales[p * kMaxPop + q];
            if (!std::isfinite(a)) return set_error(SNN_ERR_INVALID, "scales must be finite");
            c.proj_scale[p][q] = a;
        }
    if (!(nu_bg >= 0) || !std::isfinite(nu_bg)) return set_error(SNN_ERR_INVALID, "nu_bg must be >= 0");
    c.nu_bg = nu_bg;
    for (int p = 0; p < c.n_pop; ++p)
        if (nu_bg * c.k_ext[p] * (c.dt / 1000.0) > 20.0)
            return set_error(SNN_ERR_INVALID, "background mean per step above 20 spikes");
    GCK(cudaStreamSynchronize(net->stream));
    const snn_config old = net->cfg;
    net->cfg = c;
    int rc = net_make_tables(net);
    if (rc != SNN_OK) {
        net->cfg = old;
        net_make_tables(net);
        return rc;
    }
    if (net->grad) net->grad->ready = false;
    return net_upload_weights(net);
}

int snn_grad_forward(snn_net* net, int64_t n_steps, int32_t ckpt_every, double* rates_host) {
    if (!net || n_steps < 1 || ckpt_every < 1 || !rates_host)
        return set_error(SNN_ERR_INVALID, "bad arguments");
    if (n_steps > (1ll << 31)) return set_error(SNN_ERR_INVALID, "n_steps too large");
    if (!net->grad) net->grad = new snn_grad();
    snn_grad* g = net->grad;
    const int n = net->n;
    // the trace of every step when it fits (one launch each way, no
    // checkpoints), else of one checkpoint segment at a time
    size_t free_b = 0, total_b = 0;
    GCK(cudaMemGetInfo(&free_b, &total_b));
    const size_t full_bytes = (size_t)n_steps * n * (sizeof(float) + 1);
    const bool full = (int64_t)full_bytes <= g->trace_budget && full_bytes <= free_b / 4;
    const int32_t seg = full ? (int32_t)n_steps : (int32_t)std::min<int64_t>(ckpt_every, n_steps);
    const int32_t n_seg = (int32_t)((n_steps + seg - 1) / seg);
    g->ready = false;
    g->ring_words = ring_words(net);
    g->ckpt_bytes = (state_bytes(net) + 255) / 256 * 256;
    if (!full) {
        if (g->ckpt && g->ckpt_cap < (size_t)n_seg + 1) {
            cudaFree(g->ckpt);
            g->ckpt = nullptr;
        }
        if (!g->ckpt) {
            GCALL(galloc(&g->ckpt, g->ckpt_bytes * ((size_t)n_seg + 1), "gradient checkpoints"));
            g->ckpt_cap = (size_t)n_seg + 1;
        }
    }
    const int32_t tr_steps = full ? (int32_t)n_steps : seg;
    if (g->tr_u && g->tr_cap < tr_steps) {
        cudaFree(g->tr_u);
        cudaFree(g->tr_f);
        g->tr_u = nullptr;
        g->tr_f = nullptr;
        g->tr_cap = 0;
    }
    GCALL(galloc(&g->tr_u, (size_t)tr_steps * n, "gradient trace"));
    GCALL(galloc(&g->tr_f, (size_t)tr_steps * n, "gradient trace"));
    g->tr_cap = std::max(g->tr_cap, tr_steps);
    g->full_trace = full;
    cudaStream_t s = net->stream;
    GCK(cudaMemsetAsync(net->d_pop_spikes, 0, sizeof(unsigned long long) * kMaxPop, s));
    StepParams sp;
    fill_step_params(net, &sp);
    const int64_t t0 = net->step;
    if (full) {
        sp.tr_u = g->tr_u;
        sp.tr_f = g->tr_f;
        sp.tr_t0 = t0;
        sp.tr_len = (int32_t)n_steps;
    }
    for (int32_t c = 0; c < n_seg; ++c) {
        if (!full) GCK(save_ckpt(net, g->ckpt + (size_t)c * g->ckpt_bytes));
        const int64_t len = std::min<int64_t>(seg, n_steps - (int64_t)c * seg);
        GCK(net_launch(net, sp, t0 + (int64_t)c * seg, len));
    }
    if (!full) GCK(save_ckpt(net, g->ckpt + (size_t)n_seg * g->ckpt_bytes));
    unsigned long long cnt[kMaxPop];
    GCK(cudaMemcpyAsync(cnt, net->d_pop_spikes, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    net->step = t0 + n_steps;
    uint32_t st = 0;
    GCK(cudaMemcpy(&st, net->d_sync + 4, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) return set_error(SNN_ERR_TIMEOUT, "a grid-barrier wait timed out");
    const double T = (double)n_steps * net->cfg.dt / 1000.0;
    for (int p = 0; p < kMaxPop; ++p)
        rates_host[p] = (p < net->n_pop && net->cfg.pop_size[p] > 0)
                            ? (double)cnt[p] / ((double)net->cfg.pop_size[p] * T)
                            : 0.0;
    g->t_start = t0;
    g->n_steps = n_steps;
    g->seg = seg;
    g->n_seg = n_seg;
    g->ready = true;
    return SNN_OK;
}

int snn_grad_set_trace_budget(snn_net* net, int64_t bytes) {
    if (!net || bytes < 0) return set_error(SNN_ERR_INVALID, "bad arguments");
    if (!net->grad) net->grad = new snn_grad();
    net->grad->trace_budget = bytes;
    return SNN_OK;
}

int snn_grad_backward(snn_net* net, const double* g_rate, double* g_alpha, double* g_nu) {
    if (!net || !g_rate || !g_alpha || !g_nu) return set_error(SNN_ERR_INVALID, "bad arguments");
    snn_grad* g = net->grad;
    if (!g || !g->ready) return set_error(SNN_ERR_INVALID, "no gradient forward to differentiate");
    if (net->step != g->t_start + g->n_steps)
        return set_error(SNN_ERR_INVALID, "the network was stepped after the gradient forward");
    const int n = net->n, P = net->P;
    cudaStream_t s = net->stream;
    GCALL(galloc(&g->lu, n, "adjoint"));
    GCALL(galloc(&g->lI, n, "adjoint"));
    GCALL(galloc(&g->lring, (size_t)kRing * n, "adjoint ring"));
    GCALL(galloc(&g->mnext, n, "adjoint"));
    GCALL(galloc(&g->gA, (size_t)n * kMaxPop, "gradient sums"));
    GCALL(galloc(&g->gN, n, "gradient sums"));
    GCALL(galloc(&g->wbase, kMaxPop * kMaxPop * kWCodes, "base weights"));
    GCALL(galloc(&g->out, kMaxPop * kMaxPop + 1 + kMaxPop, "gradient output"));
    GCALL(galloc(&g->sync, 4, "adjoint barrier"));
    GCALL(galloc(&g->saved, 2 + kMaxPop, "saved counters"));
    GCALL(galloc(&g->saved_ras, P, "saved raster counts"));
    GCALL(galloc(&g->saved_status, 1, "saved status"));
    GCALL(galloc(&g->pop_start, kMaxPop + 1, "population starts"));
    // keep the caller-visible counters, raster counts and status: the
    // recomputation re-runs steps that were already counted and recorded
    GCK(cudaMemcpyAsync(g->saved, net->d_counters, 16, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemcpyAsync(g->saved + 2, net->d_pop_spikes, 8 * kMaxPop, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemcpyAsync(g->saved_ras, net->d_ras_n, 4 * P, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemcpyAsync(g->saved_status, net->d_sync + 4, 4, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemsetAsync(g->lu, 0, sizeof(float) * n, s));
    GCK(cudaMemsetAsync(g->lI, 0, sizeof(float) * n, s));
    GCK(cudaMemsetAsync(g->lring, 0, sizeof(float) * (size_t)kRing * n, s));
    GCK(cudaMemsetAsync(g->mnext, 0, n, s));
    GCK(cudaMemsetAsync(g->gA, 0, sizeof(double) * (size_t)n * kMaxPop, s));
    GCK(cudaMemsetAsync(g->gN, 0, sizeof(double) * n, s));
    GCK(cudaMemsetAsync(g->sync, 0, sizeof(uint32_t) * 4, s));
    std::vector<float> wb(kMaxPop * kMaxPop * kWCodes);
    net_base_weights(net, wb.data());
    GCK(cudaMemcpyAsync(g->wbase, wb.data(), sizeof(float) * wb.size(), cudaMemcpyHostToDevice, s));
    // dnu per population and the population starts for the reduction
    const double dts = net->cfg.dt / 1000.0;
    double dnu[kMaxPop];
    for (int p = 0; p < kMaxPop; ++p)
        dnu[p] = (p < net->n_pop && net->cfg.input_mode == 0)
                     ? (double)net->wext_q / 256.0 * net->cfg.k_ext[p] * dts
                     : 0.0;
    GCK(cudaMemcpyAsync(g->out + kMaxPop * kMaxPop + 1, dnu, sizeof(dnu), cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(g->pop_start, net->pop_start, sizeof(int32_t) * (kMaxPop + 1), cudaMemcpyHostToDevice, s));
    // pre-decoded rows for the gather, built once (the words never change);
    // ring offsets 64 n must fit the entry's offset field
    const bool use_pre = (long long)kRing * n < (long long)kPreOffMask;
    if (use_pre && !g->pre) {
        GCALL(galloc(&g->pre, (size_t)net->nnz + 4, "pre-decoded rows"));
        k_adj_predecode<<<(unsigned)(((long long)n * 32 + 255) / 256), 256, 0, s>>>(
            n, net->n_pop, g->pop_start, net->d_row_start, net->d_words, g->pre);
        GCK(cudaGetLastError());
    }

    if (!g->part_planned) {
        // the partition-local gather when every CTA's share of the rows fits
        // in shared memory
        AdjPartPlan plan;
        const int rc = adjoint_part_plan(n, net->n_pop, net->pop_start, P, net->part_lo.data(), net->ncmax,
                                         net->nnz, net->d_row_start, net->d_pre, net->d_seg, &plan);
        if (rc < 0) return set_error(SNN_ERR_CUDA, "partition-local adjoint plan");
        if (rc == 0) {
            g->part = new AdjPartPlan(plan);
            GCALL(galloc(&g->pds, (size_t)2 * P * n, "adjoint partials"));
            GCALL(galloc(&g->gAc, (size_t)P * n * kMaxPop, "gradient partials"));
        }
        g->part_planned = true;
    }
    if (g->part) GCK(cudaMemsetAsync(g->gAc, 0, sizeof(double) * (size_t)P * n * kMaxPop, s));
    if (!g->blk) {
        // CTA row ranges with equal total row length, rows longest first
        int dev = 0, sms = 0;
        GCK(cudaGetDevice(&dev));
        GCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = std::max(1, std::min(sms, (n + 31) / 32));
        std::vector<unsigned long long> rs(n + 1);
        GCK(cudaMemcpy(rs.data(), net->d_row_start, sizeof(unsigned long long) * (n + 1),
                       cudaMemcpyDeviceToHost));
        std::vector<int32_t> blk(grid + 1, n), order(n);
        blk[0] = 0;
        const double total = (double)rs[n] + (double)n;     // + 1 per row: empty rows cost too
        int b = 1;
        for (int j = 0; j < n && b < grid; ++j)
            while (b < grid && (double)rs[j + 1] + (double)(j + 1) >= total * b / grid) blk[b++] = j + 1;
        int chunk = 1;
        for (int c = 0; c < grid; ++c) {
            for (int j = blk[c]; j < blk[c + 1]; ++j) order[j] = j;
            std::stable_sort(order.begin() + blk[c], order.begin() + blk[c + 1],
                             [&](int x, int y) { return rs[x + 1] - rs[x] > rs[y + 1] - rs[y]; });
            chunk = std::max(chunk, blk[c + 1] - blk[c]);
        }
        GCALL(galloc(&g->blk, grid + 1, "adjoint ranges"));
        GCALL(galloc(&g->order, n, "adjoint row order"));
        GCK(cudaMemcpy(g->blk, blk.data(), sizeof(int32_t) * (grid + 1), cudaMemcpyHostToDevice));
        GCK(cudaMemcpy(g->order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
        g->grid = grid;
        g->chunk = chunk;
    }
    const int grid = g->grid;
    AdjParams ap;
    std::memset(&ap, 0, sizeof(ap));
    ap.n = n;
    ap.n_pop = net->n_pop;
    ap.chunk = g->chunk;
    ap.blk = g->blk;
    ap.order = g->order;
    for (int p = 0; p <= kMaxPop; ++p) ap.pop_start[p] = net->pop_start[p];
    ap.P22 = net->prop[0];
    ap.P21 = net->prop[1];
    ap.P11 = net->prop[2];
    ap.theta = (float)net->cfg.theta;
    const double T = (double)g->n_steps * net->cfg.dt / 1000.0;
    for (int p = 0; p < kMaxPop; ++p)
        ap.gs[p] = (p < net->n_pop && net->cfg.pop_size[p] > 0)
                       ? (float)(g_rate[p] / ((double)net->cfg.pop_size[p] * T))
                       : 0.f;
    ap.timeout_ns = net->timeout_ns;
    ap.row_start = net->d_row_start;
    ap.words = net->d_words;
    ap.pre = use_pre ? g->pre : nullptr;
    ap.wtab = net->d_wtab;
    ap.wbase = g->wbase;
    ap.tr_u = g->tr_u;
    ap.tr_f = g->tr_f;
    ap.lu = g->lu;
    ap.lI = g->lI;
    ap.lring = g->lring;
    ap.mnext = g->mnext;
    ap.gA = g->gA;
    ap.gN = g->gN;
    ap.barrier = g->sync;
    ap.status = g->sync + 1;
    ap.abort_flag = g->sync + 2;
    const size_t smem = 2 * sizeof(float) * kMaxPop * kMaxPop * kWCodes +
                        sizeof(unsigned long long) * ((size_t)ap.chunk + 1) + sizeof(float) * (size_t)ap.chunk +
                        (n <= kAdjPopTable ? (size_t)n : 0);
    const void* adj_fn = use_pre ? reinterpret_cast<const void*>(&k_adjoint<true>)
                                 : reinterpret_cast<const void*>(&k_adjoint<false>);
    GCK(cudaFuncSetAttribute(adj_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));

    StepParams sp;
    fill_step_params(net, &sp);
    sp.pop_spikes = nullptr;
    sp.tr_u = g->tr_u;
    sp.tr_f = g->tr_f;
    for (int32_t c = g->n_seg - 1; c >= 0; --c) {
        const int64_t t0 = g->t_start + (int64_t)c * g->seg;
        const int32_t len = (int32_t)std::min<int64_t>(g->seg, g->n_steps - (int64_t)c * g->seg);
        // this segment's trace rows: recorded by the forward, or recomputed
        // from its checkpoint
        const size_t tr_off = g->full_trace ? (size_t)c * g->seg * n : 0;
        if (!g->full_trace) {
            GCK(load_ckpt(net, g->ckpt + (size_t)c * g->ckpt_bytes));
            sp.tr_t0 = t0;
            sp.tr_len = len;
            GCK(net_launch(net, sp, t0, len));
        }
        GCK(cudaMemsetAsync(g->sync, 0, sizeof(uint32_t), s));
        if (g->part) {
            AdjPartParams pp;
            std::memset(&pp, 0, sizeof(pp));
            pp.n = n;
            pp.n_pop = net->n_pop;
            pp.n_part = P;
            pp.ncmax = net->ncmax;
            pp.len = len;
            pp.t_first = t0;
            pp.P22 = ap.P22;
            pp.P21 = ap.P21;
            pp.P11 = ap.P11;
            pp.theta = ap.theta;
            for (int k = 0; k < kMaxPop; ++k) pp.gs[k] = ap.gs[k];
            for (int k = 0; k <= kMaxPop; ++k) pp.pop_start[k] = net->pop_start[k];
            pp.timeout_ns = ap.timeout_ns;
            pp.part_lo = net->d_part_lo;
            pp.wtab = net->d_wtab;
            pp.wbase = g->wbase;
            pp.tr_u = g->tr_u + tr_off;
            pp.tr_f = g->tr_f + tr_off;
            pp.lu = g->lu;
            pp.lI = g->lI;
            pp.lring = g->lring;
            pp.mnext = g->mnext;
            pp.pds = g->pds;
            pp.gAc = g->gAc;
            pp.gN = g->gN;
            pp.barrier = g->sync;
            pp.status = g->sync + 1;
            pp.abort_flag = g->sync + 2;
            GCK(launch_adjoint_part(*g->part, pp, s));
            continue;
        }
        ap.t_first = t0;
        ap.len = len;
        ap.tr_u = g->tr_u + tr_off;
        ap.tr_f = g->tr_f + tr_off;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kAdjThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void* args[] = {&ap};
        GCK(cudaLaunchKernelExC(&cfg, adj_fn, args));
    }
    if (g->part)
        GCK(launch_adjoint_part_fold(n, P, net->n_pop, net->d_part_lo, g->pop_start, g->gAc, g->gA, s));
    k_grad_reduce<<<kMaxPop * kMaxPop + 1, 512, 0, s>>>(n, net->n_pop, g->pop_start, g->gA, g->gN, g->out + kMaxPop * kMaxPop + 1,
                                     g->out);
    GCK(cudaGetLastError());
    // back to the state after the forward (only the recomputation changed
    // it), with the caller's counters
    if (!g->full_trace) GCK(load_ckpt(net, g->ckpt + (size_t)g->n_seg * g->ckpt_bytes));
    GCK(cudaMemcpyAsync(net->d_counters, g->saved, 16, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemcpyAsync(net->d_pop_spikes, g->saved + 2, 8 * kMaxPop, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemcpyAsync(net->d_ras_n, g->saved_ras, 4 * P, cudaMemcpyDeviceToDevice, s));
    GCK(cudaMemcpyAsync(net->d_sync + 4, g->saved_status, 4, cudaMemcpyDeviceToDevice, s));
    double out[kMaxPop * kMaxPop + 1];
    GCK(cudaMemcpyAsync(out, g->out, sizeof(out), cudaMemcpyDeviceToHost, s));
    uint32_t adj_status = 0;
    GCK(cudaMemcpyAsync(&adj_status, g->sync + 1, sizeof(adj_status), cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    if (adj_status & kStatusTimeout) return set_error(SNN_ERR_TIMEOUT, "an adjoint barrier wait timed out");
    for (int k = 0; k < kMaxPop * kMaxPop; ++k) g_alpha[k] = out[k];
    *g_nu = out[kMaxPop * kMaxPop];
    return SNN_OK;
}

int snn_save_state(snn_net* net, void* buf_host, int64_t cap, int64_t* n_bytes) {
    if (!net || !n_bytes) return set_error(SNN_ERR_INVALID, "bad arguments");
    const size_t n = (size_t)net->n;
    const size_t need = 32 + n * 12 + (size_t)kRing * n * 4;
    *n_bytes = (int64_t)need;
    if (!buf_host) return SNN_OK;
    if (cap < (int64_t)need) return set_error(SNN_ERR_INVALID, "buffer smaller than the state");
    GCK(cudaStreamSynchronize(net->stream));
    uint8_t* b = static_cast<uint8_t*>(buf_host);
    const uint64_t hdr[4] = {kStateMagic, (uint64_t)n, (uint64_t)net->step, (uint64_t)kRing};
    std::memcpy(b, hdr, 32);
    GCK(cudaMemcpy(b + 32, net->d_u, n * 4, cudaMemcpyDeviceToHost));
    GCK(cudaMemcpy(b + 32 + n * 4, net->d_i, n * 4, cudaMemcpyDeviceToHost));
    GCK(cudaMemcpy(b + 32 + n * 8, net->d_r, n * 4, cudaMemcpyDeviceToHost));
    std::vector<int32_t> tmp(ring_words(net));
    GCK(cudaMemcpy(tmp.data(), net->d_ring, tmp.size() * 4, cudaMemcpyDeviceToHost));
    int32_t* ring = reinterpret_cast<int32_t*>(b + 32 + n * 12);
    for (int c = 0; c < net->P; ++c) {
        const int lo = net->part_lo[c], nc = net->part_lo[c + 1] - lo;
        for (int slot = 0; slot < kRing; ++slot)
            std::memcpy(ring + (size_t)slot * n + lo, tmp.data() + ((size_t)c * kRing + slot) * net->ncmax,
                        sizeof(int32_t) * nc);
    }
    return SNN_OK;
}

int snn_load_state(snn_net* net, const void* buf_host, int64_t n_bytes) {
    if (!net || !buf_host) return set_error(SNN_ERR_INVALID, "bad arguments");
    const size_t n = (size_t)net->n;
    const size_t need = 32 + n * 12 + (size_t)kRing * n * 4;
    if (n_bytes != (int64_t)need) return set_error(SNN_ERR_INVALID, "state size does not match the network");
    const uint8_t* b = static_cast<const uint8_t*>(buf_host);
    uint64_t hdr[4];
    std::memcpy(hdr, b, 32);
    if (hdr[0] != kStateMagic || hdr[1] != (uint64_t)n || hdr[3] != (uint64_t)kRing)
        return set_error(SNN_ERR_INVALID, "not a state of this network");
    std::vector<int32_t> tmp(ring_words(net), 0);
    const int32_t* ring = reinterpret_cast<const int32_t*>(b + 32 + n * 12);
    for (int c = 0; c < net->P; ++c) {
        const int lo = net->part_lo[c], nc = net->part_lo[c + 1] - lo;
        for (int slot = 0; slot < kRing; ++slot)
            std::memcpy(tmp.data() + ((size_t)c * kRing + slot) * net->ncmax, ring + (size_t)slot * n + lo,
                        sizeof(int32_t) * nc);
    }
    GCK(cudaStreamSynchronize(net->stream));
    GCK(cudaMemcpy(net->d_u, b + 32, n * 4, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(net->d_i, b + 32 + n * 4, n * 4, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(net->d_r, b + 32 + n * 8, n * 4, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(net->d_ring, tmp.data(), tmp.size() * 4, cudaMemcpyHostToDevice));
    GCK(clear_messages(net));
    GCK(net_clear_wraps(net));
    GCK(cudaStreamSynchronize(net->stream));
    net->step = (int64_t)hdr[2];
    if (net->grad) net->grad->ready = false;
    return SNN_OK;
}

}  // extern "C"
