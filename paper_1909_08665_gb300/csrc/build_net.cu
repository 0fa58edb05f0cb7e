// build_net.cu -- on-device generation of the synaptic matrix (Sec. 2.1:
// connections defined by probability per population pair, normal weights
// and delays rounded to the time step; Sec. 3.1.2: the matrix is row-indexed
// by presynaptic neuron, one word per synapse).
//
// Row j is the ascending list of targets i != j that pass the Bernoulli test
// x < T[pop(i)][pop(j)], x = Philox(j, i>>2, 1, 0)[i&3].  Each synapse then
// draws (Philox(j, i, 2, 0)) a 7-bit weight code (word 0 >> 25) and an 8-bit
// delay stratum (word 1 >> 24) mapped through the source population's delay
// table.  Word = target | delay << 19 | code << 25.
//
// Two passes over the N x N pairs (count, then fill) keep the rows exact and
// contiguous; one CTA owns one row, 256 threads x 4 Philox lanes per tile of
// 1024 targets, so the write order is the target order.
#include "snn_internal.cuh"

namespace snn {

namespace {

// population boundaries passed by value to a kernel
struct PopStarts {
    int32_t pop_start[kMaxPop + 1];
};

template <int BLOCK>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp,
                                                    uint32_t& total) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t wp = warp ? s_warp[warp - 1] : 0u;
    total = s_warp[NW - 1];
    __syncthreads();
    return wp + x - v;
}

// connection bits of the 4 targets 4g .. 4g+3 of row j (bit k = target 4g+k)
__device__ __forceinline__ uint32_t conn_bits(const BuildParams& bp, const uint64_t* s_thr,
                                              int32_t j, int32_t g) {
    const uint4 r = philox(make_uint4((uint32_t)j, (uint32_t)g, kStreamConn, 0u), bp.key0,
                           bp.key1);
    uint32_t bits = 0;
#pragma unroll
    for (int lane = 0; lane < 4; ++lane) {
        const int32_t i = 4 * g + lane;
        if (i < bp.n && i != j) {
            const int p = pop_index(bp.pop_start, bp.n_pop, i);
            if ((uint64_t)lane_of(r, lane) < s_thr[p]) bits |= 1u << lane;
        }
    }
    return bits;
}

__global__ void __launch_bounds__(kBuildThreads)
k_build_count(const __grid_constant__ BuildParams bp, uint32_t* rowlen) {
    __shared__ uint32_t s_warp[kBuildThreads / 32];
    __shared__ uint64_t s_thr[kMaxPop];
    const int32_t j = blockIdx.x;
    const int q = pop_index(bp.pop_start, bp.n_pop, j);
    if (threadIdx.x < kMaxPop) s_thr[threadIdx.x] = bp.conn_thr[threadIdx.x][q];
    __syncthreads();
    uint32_t cnt = 0;
    const int32_t ngrp = (bp.n + 3) >> 2;
    for (int32_t g = threadIdx.x; g < ngrp; g += kBuildThreads)
        cnt += __popc(conn_bits(bp, s_thr, j, g));
    uint32_t total;
    block_excl_scan<kBuildThreads>(cnt, s_warp, total);
    if (threadIdx.x == 0) rowlen[j] = total;
}

// exclusive scan of the row lengths into 64-bit row starts (one CTA)
__global__ void __launch_bounds__(1024)
k_build_scan(const uint32_t* __restrict__ rowlen, int n, unsigned long long* row_start) {
    __shared__ uint32_t s_warp[32];
    unsigned long long carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < n ? rowlen[i] : 0u;
        uint32_t total;
        const uint32_t off = block_excl_scan<1024>(v, s_warp, total);
        if (i < n) row_start[i] = carry + off;
        carry += total;
    }
    if (threadIdx.x == 0) row_start[n] = carry;
}

// segment offsets of row j: seg[j][c] = first word whose target >= part_lo[c]
__device__ __forceinline__ void row_segments(const uint32_t* words, unsigned long long base,
                                             uint32_t len, const int32_t* part_lo, int n_part,
                                             uint32_t* seg_row) {
    for (int c = threadIdx.x; c <= n_part; c += blockDim.x) {
        const uint32_t lim = (uint32_t)part_lo[c];
        uint32_t a = 0, b = len;
        while (a < b) {
            const uint32_t m = (a + b) >> 1;
            if ((words[base + m] & kTgtMask) < lim) a = m + 1;
            else b = m;
        }
        seg_row[c] = (uint32_t)(base + a);
    }
}

__global__ void __launch_bounds__(kBuildThreads)
k_build_fill(const __grid_constant__ BuildParams bp, const unsigned long long* row_start,
             uint32_t* words, uint32_t* seg) {
    __shared__ uint32_t s_warp[kBuildThreads / 32];
    __shared__ uint64_t s_thr[kMaxPop];
    __shared__ uint8_t s_dtab[kDCodes];
    const int32_t j = blockIdx.x;
    const int q = pop_index(bp.pop_start, bp.n_pop, j);
    if (threadIdx.x < kMaxPop) s_thr[threadIdx.x] = bp.conn_thr[threadIdx.x][q];
    for (int k = threadIdx.x; k < kDCodes; k += kBuildThreads) s_dtab[k] = bp.dtab[q * kDCodes + k];
    __syncthreads();
    const unsigned long long base = row_start[j];
    uint32_t running = 0;
    const int32_t ngrp = (bp.n + 3) >> 2;
    for (int32_t g0 = 0; g0 < ngrp; g0 += kBuildThreads) {
        const int32_t g = g0 + threadIdx.x;
        const uint32_t bits = g < ngrp ? conn_bits(bp, s_thr, j, g) : 0u;
        uint32_t total;
        const uint32_t off = block_excl_scan<kBuildThreads>(__popc(bits), s_warp, total);
        unsigned long long pos = base + running + off;
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            if (bits & (1u << lane)) {
                const uint32_t i = (uint32_t)(4 * g + lane);
                const uint4 y = philox(make_uint4((uint32_t)j, i, kStreamSyn, 0u), bp.key0, bp.key1);
                const uint32_t code = y.x >> 25;
                const uint32_t d = s_dtab[y.y >> 24];
                words[pos++] = i | (d << kTgtBits) | (code << 25);
            }
        }
        running += total;
    }
    __syncthreads();
    row_segments(words, base, running, bp.part_lo, bp.n_part,
                 seg + (size_t)j * (size_t)(bp.n_part + 1));
}

__global__ void __launch_bounds__(kBuildThreads)
k_seg_from_rows(const unsigned long long* row_start, const uint32_t* words,
                const int32_t* part_lo, int n_part, uint32_t* seg) {
    const int32_t j = blockIdx.x;
    const unsigned long long base = row_start[j];
    const uint32_t len = (uint32_t)(row_start[j + 1] - base);
    row_segments(words, base, len, part_lo, n_part, seg + (size_t)j * (size_t)(n_part + 1));
}

// longest segment (words of one row that target one partition)
// longest (row, partition) segment of each partition: one CTA per partition
__global__ void k_max_segment(const uint32_t* seg, int n, int n_part, uint32_t* out) {
    __shared__ uint32_t red[kBuildThreads / 32];
    const int c = blockIdx.x;
    uint32_t m = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const uint32_t* r = seg + (size_t)j * (n_part + 1) + c;
        m = max(m, r[1] - r[0]);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
        out[c] = m;
    }
}


// default initial potential: uniform on [lo, hi) from 24 random bits, fp32
__global__ void k_init_u(int n, uint32_t k0, uint32_t k1, float lo, float hi, float* u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox(make_uint4((uint32_t)i, 0u, kStreamInit, 0u), k0, k1);
    const float span = __fsub_rn(hi, lo);
    const float unit = __fmul_rn(__uint2float_rn(r.x >> 8), 5.9604644775390625e-08f);
    u[i] = __fadd_rn(lo, __fmul_rn(span, unit));
}

// One CTA per partition: its offset is the sum of the clamped counts before it
// (at most a few hundred partitions), then its first entries up to `limit`.
__global__ void __launch_bounds__(256) k_pack_raster(const uint32_t* counts, int n_part,
                                                     uint32_t cap_part, long long limit,
                                                     const uint32_t* ras_step,
                                                     const uint32_t* ras_id, uint32_t* step_out,
                                                     uint32_t* id_out) {
    __shared__ long long s_off;
    const int c = blockIdx.x;
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int k = 0; k < c; ++k) o += min(counts[k], cap_part);
        s_off = o;
    }
    __syncthreads();
    const long long off = s_off;
    const long long m = min((long long)min(counts[c], cap_part), limit - off);
    const size_t base = (size_t)c * cap_part;
    for (long long i = threadIdx.x; i < m; i += 256) {
        step_out[off + i] = ras_step[base + (size_t)i];
        id_out[off + i] = ras_id[base + (size_t)i];
    }
}

// In-degree of every target neuron per source population: indeg[i][q] =
// number of synapses from population q onto neuron i.  One warp per row.
__global__ void __launch_bounds__(kBuildThreads)
k_indegree(const unsigned long long* row_start, const uint32_t* words, int n, PopStarts pops,
           int n_pop, uint32_t* indeg) {
    const long long j = ((long long)blockIdx.x * kBuildThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int q = pop_index(pops.pop_start, n_pop, (int32_t)j);
    const unsigned long long b = row_start[j], e = row_start[j + 1];
    for (unsigned long long k = b + lane; k < e; k += 32)
        atomicAdd(&indeg[(size_t)(words[k] & kTgtMask) * kMaxPop + q], 1u);
}

}  // namespace

cudaError_t launch_build_count(const BuildParams& bp, uint32_t* rowlen, cudaStream_t s) {
    k_build_count<<<bp.n, kBuildThreads, 0, s>>>(bp, rowlen);
    return cudaGetLastError();
}

cudaError_t launch_build_scan(const uint32_t* rowlen, int n, unsigned long long* row_start,
                              cudaStream_t s) {
    k_build_scan<<<1, 1024, 0, s>>>(rowlen, n, row_start);
    return cudaGetLastError();
}

cudaError_t launch_build_fill(const BuildParams& bp, const unsigned long long* row_start,
                              uint32_t* words, uint32_t* seg, cudaStream_t s) {
    k_build_fill<<<bp.n, kBuildThreads, 0, s>>>(bp, row_start, words, seg);
    return cudaGetLastError();
}

cudaError_t launch_indegree(const unsigned long long* row_start, const uint32_t* words, int n,
                            int n_pop, const int32_t* pop_start, uint32_t* indeg, cudaStream_t s) {
    PopStarts pops;
    for (int p = 0; p <= kMaxPop; ++p) pops.pop_start[p] = pop_start[p];
    cudaError_t e = cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * (size_t)n * kMaxPop, s);
    if (e != cudaSuccess || n <= 0) return e;
    const long long threads = (long long)n * 32;
    k_indegree<<<(unsigned)((threads + kBuildThreads - 1) / kBuildThreads), kBuildThreads, 0, s>>>(
        row_start, words, n, pops, n_pop, indeg);
    return cudaGetLastError();
}

cudaError_t launch_max_segment(const uint32_t* seg, int n, int n_part, uint32_t* out,
                               cudaStream_t s) {
    k_max_segment<<<n_part, kBuildThreads, 0, s>>>(seg, n, n_part, out);
    return cudaGetLastError();
}

cudaError_t launch_seg_from_rows(const unsigned long long* row_start, const uint32_t* words,
                                 int n, const int32_t* part_lo, int n_part, uint32_t* seg,
                                 cudaStream_t s) {
    k_seg_from_rows<<<n, kBuildThreads, 0, s>>>(row_start, words, part_lo, n_part, seg);
    return cudaGetLastError();
}

cudaError_t launch_pack_raster(const uint32_t* counts, int n_part, uint32_t cap_part,
                               int64_t limit, const uint32_t* ras_step, const uint32_t* ras_id,
                               uint32_t* step_out, uint32_t* id_out, cudaStream_t s) {
    if (n_part <= 0 || limit <= 0) return cudaSuccess;
    k_pack_raster<<<n_part, 256, 0, s>>>(counts, n_part, cap_part, (long long)limit, ras_step,
                                         ras_id, step_out, id_out);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int n, uint32_t key0, uint32_t key1, float lo, float hi,
                              float* u, cudaStream_t s) {
    k_init_u<<<(n + 255) / 256, 256, 0, s>>>(n, key0, key1, lo, hi, u);
    return cudaGetLastError();
}

}  // namespace snn
