// deliver_cluster.cu -- stand-alone delivery of one spike list (Sec. 3.1.2:
// row fetch, word decode, ring-buffer add) through thread-block clusters.
//
// A cluster of 8 CTAs owns 8 consecutive partitions; each CTA holds its
// partition's ring slice in shared memory.  Because a row's words are sorted
// by target, the part of row j that lands in the cluster's partitions is one
// contiguous run, [seg[j][c_lo], seg[j][c_lo + 8]), so it is read exactly
// (the algorithmic 4 bytes per event, coalesced) by one warp, and every word
// is added with a shared-memory atomic into the owning CTA's ring through
// distributed shared memory.  Per spike the cost is one visit per cluster
// (19 at scale 1), not one per partition (151).
#include <cooperative_groups.h>

#include "snn_internal.cuh"

namespace cg = cooperative_groups;

namespace snn {
namespace {

constexpr int kCluster = 8;
constexpr int kCThreads = 512;
constexpr int kCWarps = kCThreads / 32;
constexpr int kCUnroll = 8;            // row words per lane in flight

__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(kCThreads, 1)
k_deliver_cluster(const __grid_constant__ DeliverParams dp) {
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t* s_wt = reinterpret_cast<int32_t*>(smem);                          // [8][8][128]
    int32_t* ring = reinterpret_cast<int32_t*>(smem + kMaxPop * kMaxPop * kWCodes * 4);
    __shared__ int32_t s_plo[kCluster + 1];   // starts of the cluster's partitions
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int c = blockIdx.x;                                  // >= n_part: no partition
    const int c_lo = c - rank;
    const int c_hi = min(dp.n_part, c_lo + kCluster);
    const int R = kRing * dp.ncmax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < kMaxPop * kMaxPop * kWCodes; k += kCThreads) s_wt[k] = __ldg(&dp.wtab[k]);
    if (c < dp.n_part) {
        const int32_t* ring_g = dp.ring + (size_t)c * R;
        for (int k = tid; k < R; k += kCThreads) ring[k] = ring_g[k];
    }
    if (tid <= kCluster) s_plo[tid] = c_lo + tid <= dp.n_part ? __ldg(&dp.part_lo[c_lo + tid])
                                                              : 0x7fffffff;
    cl.sync();      // every member's ring is staged before any remote add

    int32_t ps[kMaxPop];
#pragma unroll
    for (int k = 1; k < kMaxPop; ++k) ps[k] = k < dp.n_pop ? dp.pop_start[k] : 0x7fffffff;
    const uint32_t ncmax = (uint32_t)dp.ncmax;
    const int32_t base_t = (int32_t)(((uint32_t)dp.t & (kRing - 1)) * ncmax);
    const int nparts = c_hi - c_lo;
    unsigned long long events = 0;
    if (nparts > 0) {
        // spike i of the list is taken by warp (i mod 128) of the cluster
        for (int i = rank * kCWarps + warp; i < dp.n_spikes; i += kCluster * kCWarps) {
            const uint32_t j = __ldg(&dp.spikes[i]);
            const int32_t* wq = s_wt + pop_index(dp.pop_start, dp.n_pop, (int32_t)j) * kWCodes;
            const uint32_t* sg = dp.seg + (size_t)j * (size_t)(dp.n_part + 1);
            const uint32_t b = __ldg(&sg[c_lo]), e = __ldg(&sg[c_hi]);
            for (uint32_t o = b + (uint32_t)lane; o < e; o += 32u * kCUnroll) {
                uint32_t w[kCUnroll];
#pragma unroll
                for (int u = 0; u < kCUnroll; ++u) {
                    const uint32_t x = o + 32u * (uint32_t)u;
                    w[u] = x < e ? __ldg(&dp.words[x]) : 0u;
                }
#pragma unroll
                for (int u = 0; u < kCUnroll; ++u) {
                    if (o + 32u * (uint32_t)u < e) {
                        const int32_t tgt = (int32_t)(w[u] & kTgtMask);
                        // owning partition among the cluster's 8 (binary search)
                        int r = tgt >= s_plo[4] ? 4 : 0;
                        r += tgt >= s_plo[r + 2] ? 2 : 0;
                        r += tgt >= s_plo[r + 1] ? 1 : 0;
                        int pp = 0;
#pragma unroll
                        for (int m = 1; m < kMaxPop; ++m) pp += tgt >= ps[m] ? 1 : 0;
                        int32_t a = base_t + (int32_t)(((w[u] >> kTgtBits) & 63u) * ncmax) +
                                    (tgt - s_plo[r]);
                        a -= a >= R ? R : 0;
                        int32_t* dst = cl.map_shared_rank(ring, r);
                        atomicAdd(dst + a, wq[pp * (kMaxPop * kWCodes) + (int)(w[u] >> 25)]);
                    }
                }
            }
            if (lane == 0) events += e - b;
        }
    }
    cl.sync();      // every remote add into this CTA's ring has landed
    if (c < dp.n_part) {
        int32_t* ring_g = dp.ring + (size_t)c * R;
        for (int k = tid; k < R; k += kCThreads) ring_g[k] = ring[k];
    }
    if (lane == 0 && events) atomicAdd(&dp.counters[1], events);
}

size_t cluster_smem(int ncmax) {
    return (size_t)kMaxPop * kMaxPop * kWCodes * 4 + (size_t)kRing * ncmax * 4;
}

}  // namespace

cudaError_t deliver_cluster_check(int ncmax, int n_part, int* max_active_clusters) {
    const size_t smem = cluster_smem(ncmax);
    cudaError_t e = cudaFuncSetAttribute(k_deliver_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n_part + kCluster - 1) / kCluster * kCluster));
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = smem;
    return cudaOccupancyMaxActiveClusters(max_active_clusters, k_deliver_cluster, &cfg);
}

cudaError_t launch_deliver_cluster(const DeliverParams& dp, cudaStream_t s) {
    if (dp.n_spikes <= 0) return cudaSuccess;
    const size_t smem = cluster_smem(dp.ncmax);
    cudaError_t e = cudaFuncSetAttribute(k_deliver_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (dp.n_part + kCluster - 1) / kCluster * kCluster;
    k_deliver_cluster<<<grid, kCThreads, smem, s>>>(dp);
    return cudaGetLastError();
}

}  // namespace snn
