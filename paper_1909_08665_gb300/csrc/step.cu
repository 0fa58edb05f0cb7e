// step.cu -- launch of the persistent step kernel (step_kernel.cuh; its
// variants are instantiated in the step_mode_*.cu files) and the stand-alone
// delivery kernels (Sec. 3.1.2: row fetch, word decode, buffer add).
#include "step_kernel.cuh"

namespace snn {

// ---------------------------------------------------------------------------
// standalone delivery of one spike list (global ring, partition layout)
// ---------------------------------------------------------------------------
// s_w: the weights wtab[p][q][code] of the row's source population q, staged
// in shared memory ([p][code]) so that a warp's 32 random lookups cost a few
// bank conflicts instead of up to 32 L1 wavefronts
__device__ __forceinline__ void deliver_word(const DeliverParams& dp, uint32_t word,
                                             const int32_t* s_w) {
    const int32_t tgt = (int32_t)(word & kTgtMask);
    // partition of tgt: largest c with floor(c n / P) <= tgt
    const int c = (int)(((long long)(tgt + 1) * dp.n_part - 1) / dp.n);
    const int32_t local = tgt - (int32_t)(((long long)c * dp.n) / dp.n_part);
    const uint32_t d = (word >> kTgtBits) & 63u;
    const int p = pop_index(dp.pop_start, dp.n_pop, tgt);
    const int32_t wt = s_w[p * kWCodes + (int)(word >> 25)];
    const uint32_t slot = (uint32_t)(dp.t + d) & (kRing - 1);
    atomicAdd(&dp.ring[((size_t)c * kRing + slot) * dp.ncmax + local], wt);
}

__device__ __forceinline__ void stage_weights(const DeliverParams& dp, int q, int32_t* s_w, int r,
                                              int lanes) {
    for (int k = r; k < kMaxPop * kWCodes; k += lanes)
        s_w[k] = __ldg(&dp.wtab[((k / kWCodes) * kMaxPop + q) * kWCodes + (k % kWCodes)]);
}

__global__ void __launch_bounds__(256) k_deliver_warp(const __grid_constant__ DeliverParams dp) {
    __shared__ int32_t s_w[8][kMaxPop * kWCodes];
    const int warp = (blockIdx.x * 256 + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= dp.n_spikes) return;
    const uint32_t j = __ldg(&dp.spikes[warp]);
    const int q = pop_index(dp.pop_start, dp.n_pop, (int32_t)j);
    int32_t* sw = s_w[threadIdx.x >> 5];
    stage_weights(dp, q, sw, lane, 32);
    __syncwarp();
    const uint32_t* sg = dp.seg + (size_t)j * (size_t)(dp.n_part + 1);
    const uint32_t b = __ldg(sg), e = __ldg(sg + dp.n_part);
    for (uint32_t w = b + lane; w < e; w += 32) deliver_word(dp, __ldg(&dp.words[w]), sw);
    if (lane == 0) atomicAdd(&dp.counters[1], (unsigned long long)(e - b));
}

__global__ void __launch_bounds__(256) k_deliver_block(const __grid_constant__ DeliverParams dp) {
    __shared__ int32_t s_w[kMaxPop * kWCodes];
    const uint32_t j = __ldg(&dp.spikes[blockIdx.x]);
    const int q = pop_index(dp.pop_start, dp.n_pop, (int32_t)j);
    stage_weights(dp, q, s_w, threadIdx.x, 256);
    __syncthreads();
    const uint32_t* sg = dp.seg + (size_t)j * (size_t)(dp.n_part + 1);
    const uint32_t b = __ldg(sg), e = __ldg(sg + dp.n_part);
    for (uint32_t w = b + threadIdx.x; w < e; w += 256) deliver_word(dp, __ldg(&dp.words[w]), s_w);
    if (threadIdx.x == 0) atomicAdd(&dp.counters[1], (unsigned long long)(e - b));
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
size_t step_shared_bytes(int ncmax, int n_part, int w_span, bool smem_ring) {
    return smem_layout(ncmax, n_part, w_span, smem_ring).total;
}

static const void* select_step(int npt, bool smem_ring, int mode) {
    switch (mode) {
        case 0: return step_fn_mode<0>(npt, smem_ring);
        case kModePaced: return step_fn_mode<kModePaced>(npt, smem_ring);
        case kModeSat: return step_fn_mode<kModeSat>(npt, smem_ring);
        case kModeSat | kModePaced: return step_fn_mode<kModeSat | kModePaced>(npt, smem_ring);
        default: return nullptr;
    }
}

int step_kernel_variant(int npt, bool smem_ring) {
    return select_step(npt, smem_ring, 0) != nullptr;
}

cudaError_t step_kernel_configure(int npt, bool smem_ring, size_t smem) {
    for (int mode = 0; mode < 4; ++mode) {
        const void* fn = select_step(npt, smem_ring, mode);
        if (!fn) return cudaErrorInvalidValue;
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// co-resident CTAs per SM: the smallest of the variants' figures
cudaError_t step_max_blocks(int npt, bool smem_ring, size_t smem, int* blocks_per_sm) {
    int best = 1 << 30;
    for (int mode = 0; mode < 4; ++mode) {
        const void* fn = select_step(npt, smem_ring, mode);
        if (!fn) return cudaErrorInvalidValue;
        int b = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kStepThreads, smem);
        if (e != cudaSuccess) return e;
        best = std::min(best, b);
    }
    *blocks_per_sm = best;
    return cudaSuccess;
}

cudaError_t launch_step(const StepParams& sp, int npt, bool smem_ring, size_t smem,
                        cudaStream_t s) {
    const int mode = (sp.rt_period_ns != 0ull ? kModePaced : 0) | (sp.wrap != nullptr ? kModeSat : 0);
    const void* fn = select_step(npt, smem_ring, mode);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<StepParams*>(&sp)};
    return cudaLaunchCooperativeKernel(fn, dim3(sp.n_part), dim3(kStepThreads), args, smem, s);
}

// Partition tiling of the stand-alone delivery: CTA c takes every spike of
// the list through its runs of the pre-decoded rows (the step kernel's
// delivery), with its ring slice staged in shared memory when it fits.
// Shared memory: run starts and lengths [kChunk] each, the weight-table rows
// of the partition's populations, then the ring slice.
__host__ __device__ inline size_t part_smem_bytes(int ncmax, int w_span, bool smem_ring) {
    return (size_t)kChunk * 8 + (size_t)w_span * kPopWords * 4 +
           (smem_ring ? (size_t)kRing * ncmax * 4 : 0);
}

template <bool SMEM_RING>
__global__ void __launch_bounds__(kStepThreads, 1)
k_deliver_part(const __grid_constant__ StepParams sp, const uint32_t* __restrict__ spikes, int n,
               int64_t t) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_rb = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_rl = s_rb + kChunk;
    int32_t* s_w = reinterpret_cast<int32_t*>(s_rl + kChunk);
    const int c = blockIdx.x, tid = threadIdx.x;
    const int R = kRing * sp.ncmax;
    int32_t* ring_g = sp.ring + (size_t)c * R;
    int32_t* ring = SMEM_RING ? s_w + (size_t)sp.w_span * kPopWords : ring_g;
    const uint32_t wbase = (uint32_t)pop_index(sp.pop_start, sp.n_pop, sp.part_lo[c]) * kPopWords;
    for (uint32_t k = tid; k < (uint32_t)sp.w_span * kPopWords; k += kStepThreads)
        s_w[k] = wbase + k < (uint32_t)(kMaxPop * kPopWords) ? __ldg(&sp.wtab[wbase + k]) : 0;
    if (SMEM_RING)
        for (int k = tid; k < R; k += kStepThreads) ring[k] = ring_g[k];
    __syncthreads();
    unsigned long long events = 0;
    const size_t stride = (size_t)sp.n_part + 1;
    for (int base = 0; base < n; base += kChunk) {
        const int m = min(kChunk, n - base);
        for (int k = tid; k < m; k += kStepThreads) {
            const uint32_t* sg = sp.seg + (size_t)__ldg(&spikes[base + k]) * stride + c;
            const uint32_t b = __ldg(sg);
            s_rb[k] = b;
            s_rl[k] = __ldg(sg + 1) - b;
        }
        __syncthreads();
        deliver_batches<false, BatchShape<1>::kSpikes, BatchShape<1>::kWave>(
            sp, s_rb, s_rl, s_w, wbase, (uint32_t)m, t, ring, nullptr, events, nullptr);
        __syncthreads();
    }
    if (SMEM_RING)
        for (int k = tid; k < R; k += kStepThreads) ring_g[k] = ring[k];
    if ((tid & 31) == 0 && events) atomicAdd(&sp.counters[1], events);
}

cudaError_t launch_deliver_part(const StepParams& sp, const uint32_t* spikes, int n, int64_t t,
                                bool smem_ring, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    smem_ring = smem_ring && part_smem_bytes(sp.ncmax, sp.w_span, true) <= (size_t)optin;
    const size_t smem = part_smem_bytes(sp.ncmax, sp.w_span, smem_ring);
    const void* fn = smem_ring ? reinterpret_cast<const void*>(&k_deliver_part<true>)
                               : reinterpret_cast<const void*>(&k_deliver_part<false>);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (smem_ring)
        k_deliver_part<true><<<sp.n_part, kStepThreads, smem, s>>>(sp, spikes, n, t);
    else
        k_deliver_part<false><<<sp.n_part, kStepThreads, smem, s>>>(sp, spikes, n, t);
    return cudaGetLastError();
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
