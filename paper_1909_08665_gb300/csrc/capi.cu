// capi.cu -- host side of the C ABI declared in include/snn.h.
//
// Parameter tables are computed here, in double precision, from the
// definitions of the method (Sec. 2.1: normal weights and delays rounded to
// the step, probabilistic connectivity; Sec. 3.1.3: Poisson background):
//   wtab[p][q][c] = llround(256 ((mu_pq + sd_pq z_c) w_scale) alpha_pq),
//       z_c = Phi^-1((c + 1/2) / 128)
//   delay[q][c]   = clamp(round((dmu_q + dsd_q z_c) / dt), 1, 63),
//       z_c = Phi^-1((c + 1/2) / 256)
//   T_pois[p][m]  = floor(2^32 F_lambda(m)), lambda_p = nu_bg K_ext,p dt/1000
//   T_conn[p][q]  = min(floor(p_pq conn_scale 2^32), 2^32)
//   P22 = e^{-dt/tau_m}, P11 = e^{-dt/tau_syn},
//   P21 = tau_m tau_syn / (C_m (tau_m - tau_syn)) (P22 - P11),
//   P20 = tau_m / C_m (1 - P22), rounded once to fp32.
// Compiled with -ffp-contract=off so that no expression is fused.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/snn.h"
#include "net.h"
#include "snn_internal.cuh"

namespace snn {
cudaError_t step_max_blocks(int npt, bool smem_ring, size_t smem, int* blocks_per_sm);
}

using namespace snn;


namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA;
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

// Standard-normal quantile: P. J. Acklam's rational approximation (2003) as
// the starting point, refined by two Halley steps on Phi(x) = erfc(-x/v2)/2;
// the upper half is taken from the lower by symmetry.
double norm_quantile(double p) {
    if (p > 0.5) return -norm_quantile(1.0 - p);
    static const double a[6] = {-3.969683028665376e+01, 2.209460984245205e+02,
                                -2.759285104469687e+02, 1.383577518672690e+02,
                                -3.066479806614716e+01, 2.506628277459239e+00};
    static const double b[5] = {-5.447609879822406e+01, 1.615858368580409e+02,
                                -1.556989798598866e+02, 6.680131188771972e+01,
                                -1.328068155288572e+01};
    static const double cc[6] = {-7.784894002430293e-03, -3.223964580411365e-01,
                                 -2.400758277161838e+00, -2.549732539343734e+00,
                                 4.374664141464968e+00, 2.938163982698783e+00};
    static const double d[4] = {7.784695709041462e-03, 3.224671290700398e-01,
                                2.445134137142996e+00, 3.754408661907416e+00};
    double x;
    if (p < 0.02425) {
        const double q = std::sqrt(-2.0 * std::log(p));
        x = (((((cc[0] * q + cc[1]) * q + cc[2]) * q + cc[3]) * q + cc[4]) * q + cc[5]) /
            ((((d[0] * q + d[1]) * q + d[2]) * q + d[3]) * q + 1.0);
    } else {
        const double q = p - 0.5, r = q * q;
        x = (((((a[0] * r + a[1]) * r + a[2]) * r + a[3]) * r + a[4]) * r + a[5]) * q /
            (((((b[0] * r + b[1]) * r + b[2]) * r + b[3]) * r + b[4]) * r + 1.0);
    }
    const double s2pi = 2.5066282746310002;  // sqrt(2 pi)
    for (int it = 0; it < 3; ++it) {
        const double e = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
        const double u = e * s2pi * std::exp(0.5 * x * x);
        x = x - u / (1.0 + 0.5 * x * u);
    }
    return x;
}

void poisson_thresholds(double lam, uint64_t* thr) {
    double term = std::exp(-lam);
    double cdf = term;
    for (int m = 0; m < kPoisTable; ++m) {
        if (m > 0) {
            term = term * lam / (double)m;
            cdf = cdf + term;
        }
        const double x = std::floor(cdf * 4294967296.0);
        thr[m] = x >= 4294967296.0 ? 4294967296ull : (uint64_t)x;
    }
}

int validate(const snn_config* c) {
    if (!c) return fail(SNN_ERR_INVALID, "config is NULL");
    if (c->n_pop < 1 || c->n_pop > kMaxPop) return fail(SNN_ERR_INVALID, "n_pop must be 1..8");
    long long n = 0;
    for (int p = 0; p < c->n_pop; ++p) {
        if (c->pop_size[p] < 0) return fail(SNN_ERR_INVALID, "negative population size");
        n += c->pop_size[p];
    }
    if (n < 1 || n > SNN_MAX_NEURONS) return fail(SNN_ERR_INVALID, "neuron count must be 1..524288");
    if (c->ring_depth != kRing) return fail(SNN_ERR_INVALID, "ring_depth must be 64");
    if (!(c->dt > 0) || !(c->tau_m > 0) || !(c->tau_syn > 0) || !(c->c_m > 0))
        return fail(SNN_ERR_INVALID, "dt, tau_m, tau_syn and C_m must be positive");
    if (c->tau_m == c->tau_syn) return fail(SNN_ERR_INVALID, "tau_m must differ from tau_syn");
    if (c->input_mode != 0 && c->input_mode != 1) return fail(SNN_ERR_INVALID, "input_mode must be 0 or 1");
    if (!(c->t_ref >= 0) || c->t_ref / c->dt > 1e6) return fail(SNN_ERR_INVALID, "bad t_ref");
    if (!(c->nu_bg >= 0)) return fail(SNN_ERR_INVALID, "nu_bg must be >= 0");
    for (int p = 0; p < c->n_pop; ++p) {
        if (!(c->k_ext[p] >= 0)) return fail(SNN_ERR_INVALID, "k_ext must be >= 0");
        if (c->nu_bg * c->k_ext[p] * (c->dt / 1000.0) > 20.0)
            return fail(SNN_ERR_INVALID, "background mean per step above 20 spikes");
        for (int q = 0; q < c->n_pop; ++q)
            if (!(c->conn_prob[p][q] >= 0)) return fail(SNN_ERR_INVALID, "negative probability");
    }
    return SNN_OK;
}

int make_tables(snn_net* net) {
    const snn_config* c = &net->cfg;
    const int np = c->n_pop;
    for (int p = 0; p < kMaxPop; ++p)
        for (int q = 0; q < kMaxPop; ++q) {
            for (int k = 0; k < kWCodes; ++k) {
                int32_t v = 0;
                if (p < np && q < np) {
                    const double z = norm_quantile(((double)k + 0.5) / (double)kWCodes);
                    double w = c->w_mean[p][q] + c->w_sd[p][q] * z;
                    w = w * c->w_scale;
                    w = w * c->proj_scale[p][q];
                    const double qv = w * 256.0;
                    if (!(std::fabs(qv) < 1073741824.0))
                        return fail(SNN_ERR_INVALID, "weight outside the fixed-point range");
                    v = (int32_t)std::llround(qv);
                }
                net->wtab[(p * kMaxPop + q) * kWCodes + k] = v;
            }
            double thr = 0.0;
            if (p < np && q < np) {
                const double pr = c->conn_prob[p][q] * c->conn_scale;
                thr = std::floor(pr * 4294967296.0);
                thr = std::min(std::max(thr, 0.0), 4294967296.0);
            }
            net->conn_thr[p][q] = (uint64_t)thr;
        }
    for (int q = 0; q < kMaxPop; ++q)
        for (int k = 0; k < kDCodes; ++k) {
            int dl = 1;
            if (q < np) {
                const double z = norm_quantile(((double)k + 0.5) / (double)kDCodes);
                const double steps = (c->d_mean[q] + c->d_sd[q] * z) / c->dt;
                double r = std::round(steps);
                r = std::min(std::max(r, 1.0), (double)(kRing - 1));
                dl = (int)r;
            }
            net->dtab[q * kDCodes + k] = (uint8_t)dl;
        }
    for (int p = 0; p < kMaxPop; ++p) {
        const double lam = p < np ? c->nu_bg * c->k_ext[p] * (c->dt / 1000.0) : 0.0;
        poisson_thresholds(lam, net->pois[p]);
    }
    const double P22 = std::exp(-c->dt / c->tau_m);
    const double P11 = std::exp(-c->dt / c->tau_syn);
    const double P21 = (c->tau_m * c->tau_syn) / (c->c_m * (c->tau_m - c->tau_syn)) * (P22 - P11);
    const double P20 = c->tau_m / c->c_m * (1.0 - P22);
    net->prop[0] = (float)P22;
    net->prop[1] = (float)P21;
    net->prop[2] = (float)P11;
    net->prop[3] = (float)P20;
    for (int p = 0; p < kMaxPop; ++p) net->cdc[p] = p < np ? (float)(P20 * c->i_dc[p]) : 0.f;
    net->wext_q = (int32_t)std::llround(c->w_ext * 256.0);
    net->n_ref = (int32_t)std::llround(c->t_ref / c->dt);
    return SNN_OK;
}

void free_net(snn_net* net) {
    if (!net) return;
    void* ptrs[] = {net->d_part_lo, net->d_row_start, net->d_seg, net->d_words, net->d_pre, net->d_wtab,
                    net->d_dtab, net->d_u, net->d_i, net->d_r, net->d_ring, net->d_msg, net->d_wrap,
                    net->d_ras_step, net->d_ras_id, net->d_ras_n, net->d_rs_step, net->d_rs_id,
                    net->d_counters, net->d_sync, net->d_pop_spikes, net->d_rt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    free_grad(net->grad);
    delete net;
}

template <typename T>
int dalloc(T** p, size_t count, const char* what) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        g_err = std::string("device allocation of ") + what + " failed: " + cudaGetErrorString(e);
        return SNN_ERR_OOM;
    }
    return SNN_OK;
}

#define CALL(x)                          \
    do {                                 \
        int rc_ = (x);                   \
        if (rc_ != SNN_OK) return rc_;   \
    } while (0)

// device check, partitioning and launch shape
int plan(snn_net* net, const snn_options* opt) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return fail(SNN_ERR_UNSUPPORTED, "this library is built for sm_103 (GB300) GPUs only");
    const int sms = prop.multiProcessorCount;
    int P = opt ? opt->n_part : 0;
    if (P <= 0) P = std::min(sms, std::max(1, (net->n + 511) / 512));
    if (P > kStepThreads) return fail(SNN_ERR_INVALID, "n_part must be <= 512");
    P = std::min(P, net->n);
    net->P = P;
    net->part_lo.resize(P + 1);
    for (int c = 0; c <= P; ++c) net->part_lo[c] = (int32_t)(((long long)c * net->n) / P);
    int ncmax = 0;
    for (int c = 0; c < P; ++c) ncmax = std::max(ncmax, net->part_lo[c + 1] - net->part_lo[c]);
    net->ncmax = ncmax;
    int npt = (ncmax + kStepThreads - 1) / kStepThreads;
    if (npt <= 1) npt = 1;
    else if (npt <= 2) npt = 2;
    else if (npt <= 4) npt = 4;
    else if (npt <= 8) npt = 8;
    else return fail(SNN_ERR_INVALID, "too many neurons per partition (raise n_part)");
    net->npt = npt;
    if ((long long)kRing * ncmax >= (long long)kPreOffMask)
        return fail(SNN_ERR_INVALID, "partition too large for the 19-bit ring offsets");
    net->w_span = partition_pop_span(net->part_lo.data(), P, net->pop_start, net->n_pop);
    int smem_max = 0;
    CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t with_ring = step_shared_bytes(ncmax, P, net->w_span, true);
    net->smem_ring = with_ring <= (size_t)smem_max;
    net->smem = step_shared_bytes(ncmax, P, net->w_span, net->smem_ring);
    CK(step_kernel_configure(npt, net->smem_ring, net->smem));
    int per_sm = 0;
    CK(step_max_blocks(npt, net->smem_ring, net->smem, &per_sm));
    if (per_sm * sms < P)
        return fail(SNN_ERR_UNSUPPORTED, "partitions exceed co-resident CTAs of the step kernel");
    const double tmo = (opt && opt->timeout_s > 0) ? opt->timeout_s : 2.0;
    net->timeout_ns = (uint64_t)(tmo * 1e9);
    const int64_t cap = (opt && opt->raster_capacity > 0) ? opt->raster_capacity : (64ll << 20);
    net->ras_cap = (uint32_t)std::min<int64_t>(std::max<int64_t>(cap / P, 1), 0x7fffffff);
    net->inject_fault = opt ? opt->inject_fault : 0;
    return SNN_OK;
}

int alloc_state(snn_net* net, const float* u0_host) {
    const int n = net->n, P = net->P;
    CALL(dalloc(&net->d_u, n, "u"));
    CALL(dalloc(&net->d_i, n, "I"));
    CALL(dalloc(&net->d_r, n, "refractory"));
    CALL(dalloc(&net->d_ring, (size_t)P * kRing * net->ncmax, "ring"));
    // header + ids, read in 16-byte pairs up to entry ncmax + 1 and as a
    // 64-byte head: a multiple of 8 entries, at least ncmax + 2
    net->msg_stride = (net->ncmax + 2 + 7) / 8 * 8;
    CALL(dalloc(&net->d_msg, (size_t)4 * P * net->msg_stride, "spike messages"));
    CALL(dalloc(&net->d_ras_step, (size_t)P * net->ras_cap, "raster"));
    CALL(dalloc(&net->d_ras_id, (size_t)P * net->ras_cap, "raster"));
    CALL(dalloc(&net->d_ras_n, P, "raster counts"));
    CALL(dalloc(&net->d_counters, 2, "counters"));
    CALL(dalloc(&net->d_sync, 8, "sync words"));
    CALL(dalloc(&net->d_pop_spikes, kMaxPop, "population spike counters"));
    cudaStream_t s = net->stream;
    CK(cudaMemsetAsync(net->d_i, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(net->d_r, 0, sizeof(int32_t) * n, s));
    CK(cudaMemsetAsync(net->d_ring, 0, sizeof(int32_t) * (size_t)P * kRing * net->ncmax, s));
    CK(cudaMemsetAsync(net->d_msg, 0, sizeof(unsigned long long) * 4 * P * net->msg_stride, s));
    CK(cudaMemsetAsync(net->d_ras_n, 0, sizeof(uint32_t) * P, s));
    CK(cudaMemsetAsync(net->d_counters, 0, sizeof(unsigned long long) * 2, s));
    CK(cudaMemsetAsync(net->d_sync, 0, sizeof(uint32_t) * 8, s));
    CK(cudaMemsetAsync(net->d_pop_spikes, 0, sizeof(unsigned long long) * kMaxPop, s));
    if (u0_host) {
        CK(cudaMemcpyAsync(net->d_u, u0_host, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    } else {
        CK(launch_init_state(n, (uint32_t)(net->seed & 0xffffffffu), (uint32_t)(net->seed >> 32),
                             (float)net->cfg.u0_lo, (float)net->cfg.u0_hi, net->d_u, s));
    }
    CK(cudaStreamSynchronize(s));
    return SNN_OK;
}

int common_setup(const snn_config* cfg, uint64_t seed, const snn_options* opt, void* stream,
                 snn_net** out_net) {
    CALL(validate(cfg));
    if (opt && (opt->inject_fault < 0 || opt->inject_fault > 1))
        return fail(SNN_ERR_INVALID, "options.inject_fault must be 0 or 1");
    snn_net* net = new snn_net();
    net->cfg = *cfg;
    net->seed = seed;
    net->stream = reinterpret_cast<cudaStream_t>(stream);
    net->n_pop = cfg->n_pop;
    net->pop_start[0] = 0;
    for (int p = 0; p < kMaxPop; ++p)
        net->pop_start[p + 1] = net->pop_start[p] + (p < cfg->n_pop ? cfg->pop_size[p] : 0);
    net->n = net->pop_start[cfg->n_pop];
    net->step = 0;
    int rc = make_tables(net);
    if (rc == SNN_OK) rc = plan(net, opt);
    if (rc != SNN_OK) {
        free_net(net);
        return rc;
    }
    *out_net = net;
    return SNN_OK;
}

// weight table upload and the pre-decoded rows the step kernel reads: entry
// k of row j is (weight-table index << 19) | (delay * ncmax + target - its
// partition's start), the same layout as the packed words
int finish_network(snn_net* net) {
    cudaStream_t s = net->stream;
    CALL(dalloc(&net->d_wtab, kMaxPop * kMaxPop * kWCodes, "wtab"));
    CK(cudaMemcpyAsync(net->d_wtab, net->wtab, sizeof(net->wtab), cudaMemcpyHostToDevice, s));
    const int P = net->P;
    uint32_t* d_max = nullptr;
    CALL(dalloc(&d_max, P, "segment maxima"));
    std::vector<uint32_t> lmax(P, 0);
    cudaError_t e = launch_max_segment(net->d_seg, net->n, P, d_max, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lmax.data(), d_max, sizeof(uint32_t) * P, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_max);
    if (e != cudaSuccess) return cuda_fail(e, "segment maxima");
    net->run_max = (int32_t)*std::max_element(lmax.begin(), lmax.end());
    CALL(dalloc(&net->d_pre, (size_t)net->nnz + 4, "pre-decoded rows"));
    DeliverParams dp;
    std::memset(&dp, 0, sizeof(dp));
    dp.n = net->n;
    dp.n_pop = net->n_pop;
    dp.n_part = P;
    dp.ncmax = net->ncmax;
    for (int p = 0; p <= kMaxPop; ++p) dp.pop_start[p] = net->pop_start[p];
    dp.part_lo = net->d_part_lo;
    dp.words = net->d_words;
    CK(launch_predecode(dp, net->d_row_start, net->d_pre, s));
    // in-degrees per source population, for the bound on one step's input
    uint32_t* d_indeg = nullptr;
    CALL(dalloc(&d_indeg, (size_t)net->n * kMaxPop, "in-degrees"));
    net->indeg.assign((size_t)net->n * kMaxPop, 0u);
    e = launch_indegree(net->d_row_start, net->d_words, net->n, net->n_pop, net->pop_start,
                        d_indeg, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(net->indeg.data(), d_indeg, sizeof(uint32_t) * net->indeg.size(),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_indeg);
    if (e != cudaSuccess) return cuda_fail(e, "in-degrees");
    return net_update_saturation(net);
}

// the synaptic rows (row starts, words, per-partition segment offsets)
int build_rows(snn_net* net) {
    cudaStream_t s = net->stream;
    const int n = net->n, P = net->P;
    CALL(dalloc(&net->d_part_lo, P + 1, "partitions"));
    CALL(dalloc(&net->d_dtab, kMaxPop * kDCodes, "delay table"));
    CK(cudaMemcpyAsync(net->d_part_lo, net->part_lo.data(), sizeof(int32_t) * (P + 1),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(net->d_dtab, net->dtab, sizeof(net->dtab), cudaMemcpyHostToDevice, s));
    BuildParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.n = n;
    bp.n_pop = net->n_pop;
    for (int p = 0; p <= kMaxPop; ++p) bp.pop_start[p] = net->pop_start[p];
    bp.n_part = P;
    bp.key0 = (uint32_t)(net->seed & 0xffffffffu);
    bp.key1 = (uint32_t)(net->seed >> 32);
    for (int p = 0; p < kMaxPop; ++p)
        for (int q = 0; q < kMaxPop; ++q) bp.conn_thr[p][q] = net->conn_thr[p][q];
    bp.dtab = net->d_dtab;
    bp.part_lo = net->d_part_lo;
    uint32_t* rowlen = nullptr;
    CALL(dalloc(&rowlen, n, "row lengths"));
    CALL(dalloc(&net->d_row_start, (size_t)n + 1, "row starts"));
    cudaError_t e = launch_build_count(bp, rowlen, s);
    if (e == cudaSuccess) e = launch_build_scan(rowlen, n, net->d_row_start, s);
    unsigned long long total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, net->d_row_start + n, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(rowlen);
    if (e != cudaSuccess) return cuda_fail(e, "network row count");
    if (total >= 0xffffffffull) return fail(SNN_ERR_INVALID, "more than 2^32-1 synapses");
    net->nnz = total;
    // + 4 words: bulk L2 prefetches of a row round its end up to 16 B
    CALL(dalloc(&net->d_words, total + 4, "synaptic words"));
    CALL(dalloc(&net->d_seg, (size_t)n * (P + 1) + 4, "row segments"));
    CK(launch_build_fill(bp, net->d_row_start, net->d_words, net->d_seg, s));
    CK(cudaStreamSynchronize(s));
    return SNN_OK;
}

int build_generated(snn_net* net) {
    net->max_delay = 1;
    for (int q = 0; q < net->n_pop; ++q)
        for (int k = 0; k < kDCodes; ++k) net->max_delay = std::max<int32_t>(net->max_delay, net->dtab[q * kDCodes + k]);
    CALL(build_rows(net));
    return finish_network(net);
}

int build_from_rows(snn_net* net, const uint64_t* row_ptr, const uint32_t* words,
                    const int32_t* wtab) {
    cudaStream_t s = net->stream;
    const int n = net->n, P = net->P;
    if (!row_ptr || !words || !wtab) return fail(SNN_ERR_INVALID, "rows, words and wtab are required");
    if (row_ptr[0] != 0) return fail(SNN_ERR_INVALID, "row_ptr[0] must be 0");
    net->max_delay = 1;
    for (int j = 0; j < n; ++j) {
        if (row_ptr[j + 1] < row_ptr[j]) return fail(SNN_ERR_INVALID, "row_ptr must not decrease");
        uint32_t prev = 0;
        for (uint64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
            const uint32_t t = words[e] & kTgtMask;
            const uint32_t d = (words[e] >> kTgtBits) & 63u;
            if ((int)t >= n) return fail(SNN_ERR_INVALID, "target index out of range");
            if (d < 1) return fail(SNN_ERR_INVALID, "delay must be 1..63 steps");
            net->max_delay = std::max<int32_t>(net->max_delay, (int32_t)d);
            if (e > row_ptr[j] && t < prev) return fail(SNN_ERR_INVALID, "targets must ascend within a row");
            prev = t;
        }
    }
    const uint64_t total = row_ptr[n];
    if (total >= 0xffffffffull) return fail(SNN_ERR_INVALID, "more than 2^32-1 synapses");
    net->nnz = total;
    std::memcpy(net->wtab, wtab, sizeof(net->wtab));
    CALL(dalloc(&net->d_part_lo, P + 1, "partitions"));
    CALL(dalloc(&net->d_row_start, (size_t)n + 1, "row starts"));
    // + 4 words: bulk L2 prefetches of a row round its end up to 16 B
    CALL(dalloc(&net->d_words, total + 4, "synaptic words"));
    CALL(dalloc(&net->d_seg, (size_t)n * (P + 1) + 4, "row segments"));
    CK(cudaMemcpyAsync(net->d_part_lo, net->part_lo.data(), sizeof(int32_t) * (P + 1),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(net->d_row_start, row_ptr, sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    if (total) CK(cudaMemcpyAsync(net->d_words, words, sizeof(uint32_t) * total, cudaMemcpyHostToDevice, s));
    CK(launch_seg_from_rows(net->d_row_start, net->d_words, n, net->d_part_lo, P, net->d_seg, s));
    CK(cudaStreamSynchronize(s));
    return finish_network(net);
}

int check_status(snn_net* net) {
    uint32_t st = 0;
    CK(cudaMemcpy(&st, net->d_sync + 4, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) return fail(SNN_ERR_TIMEOUT, "a grid-barrier wait timed out");
    if (st & 2u) return fail(SNN_ERR_OVERFLOW, "spike raster capacity exceeded; spikes were lost");
    if (st & kStatusSaturated)
        return fail(SNN_ERR_SATURATED, "a neuron's input of one step left the int32 fixed-point "
                                       "range (it wrapped modulo 2^32)");
    return SNN_OK;
}

}  // namespace

namespace snn {

// Validated model constants of a configuration (host only, no allocation).
int host_step_constants(const snn_config* cfg, float prop[4], float cdc[kMaxPop],
                        uint64_t pois[kMaxPop][kPoisTable], int32_t* wext_q, int32_t* n_ref) {
    CALL(validate(cfg));
    static thread_local snn_net tmp;   // table workspace reused by this thread
    tmp.cfg = *cfg;
    CALL(make_tables(&tmp));
    for (int k = 0; k < 4; ++k) prop[k] = tmp.prop[k];
    for (int p = 0; p < kMaxPop; ++p) {
        cdc[p] = tmp.cdc[p];
        for (int m = 0; m < kPoisTable; ++m) pois[p][m] = tmp.pois[p][m];
    }
    *wext_q = tmp.wext_q;
    *n_ref = tmp.n_ref;
    return SNN_OK;
}

int host_tables(const snn_config* cfg, HostTables* out) {
    CALL(validate(cfg));
    static thread_local snn_net tmp;
    tmp.cfg = *cfg;
    CALL(make_tables(&tmp));
    out->n_pop = cfg->n_pop;
    out->pop_start[0] = 0;
    for (int p = 0; p < kMaxPop; ++p)
        out->pop_start[p + 1] = out->pop_start[p] + (p < cfg->n_pop ? cfg->pop_size[p] : 0);
    out->n = out->pop_start[cfg->n_pop];
    std::memcpy(out->wtab, tmp.wtab, sizeof(out->wtab));
    for (int p = 0; p < kMaxPop; ++p)
        for (int m = 0; m < kPoisTable; ++m) out->pois[p][m] = tmp.pois[p][m];
    for (int k = 0; k < 4; ++k) out->prop[k] = tmp.prop[k];
    for (int p = 0; p < kMaxPop; ++p) out->cdc[p] = tmp.cdc[p];
    out->theta = (float)cfg->theta;
    out->wext_q = tmp.wext_q;
    out->n_ref = tmp.n_ref;
    out->mode = cfg->input_mode;
    out->max_delay = 1;
    for (int q = 0; q < cfg->n_pop; ++q)
        for (int k = 0; k < kDCodes; ++k) out->max_delay = std::max(out->max_delay, (int32_t)tmp.dtab[q * kDCodes + k]);
    return SNN_OK;
}

int build_rows_device(const snn_config* cfg, uint64_t seed, cudaStream_t stream,
                      unsigned long long** row_start, uint32_t** words, uint64_t* nnz) {
    CALL(validate(cfg));
    snn_net* net = new snn_net();
    net->cfg = *cfg;
    net->seed = seed;
    net->stream = stream;
    net->n_pop = cfg->n_pop;
    net->pop_start[0] = 0;
    for (int p = 0; p < kMaxPop; ++p)
        net->pop_start[p + 1] = net->pop_start[p] + (p < cfg->n_pop ? cfg->pop_size[p] : 0);
    net->n = net->pop_start[cfg->n_pop];
    int rc = make_tables(net);
    if (rc == SNN_OK) {
        net->P = 1;                                  // whole rows: one partition
        net->part_lo = {0, net->n};
        rc = build_rows(net);
    }
    if (rc == SNN_OK) {
        *row_start = net->d_row_start;
        *words = net->d_words;
        *nnz = net->nnz;
        net->d_row_start = nullptr;
        net->d_words = nullptr;
    }
    free_net(net);
    return rc;
}

void fill_step_params(const snn_net* net, StepParams* out) {
    StepParams& sp = *out;
    std::memset(&sp, 0, sizeof(sp));
    sp.n = net->n;
    sp.n_pop = net->n_pop;
    sp.n_part = net->P;
    sp.ncmax = net->ncmax;
    for (int p = 0; p <= kMaxPop; ++p) sp.pop_start[p] = net->pop_start[p];
    sp.P22 = net->prop[0];
    sp.P21 = net->prop[1];
    sp.P11 = net->prop[2];
    sp.theta = (float)net->cfg.theta;
    for (int p = 0; p < kMaxPop; ++p) sp.cdc[p] = net->cdc[p];
    sp.n_ref = net->n_ref;
    sp.wext_q = net->wext_q;
    sp.mode = net->cfg.input_mode;
    sp.key0 = (uint32_t)(net->seed & 0xffffffffu);
    sp.key1 = (uint32_t)(net->seed >> 32);
    sp.ras_cap = net->ras_cap;
    sp.timeout_ns = net->timeout_ns;
    sp.inject_fault = net->inject_fault;
    for (int p = 0; p < kMaxPop; ++p)
        for (int m = 0; m < kPoisTable; ++m)   // T >= 1 (validation bounds lambda)
            sp.pois_m1[p][m] = (uint32_t)(net->pois[p][m] - 1u);
    sp.pre = net->d_pre;
    sp.w_span = net->w_span;
    sp.part_lo = net->d_part_lo;
    sp.seg = net->d_seg;
    sp.words = net->d_words;
    sp.wtab = net->d_wtab;
    sp.u = net->d_u;
    sp.i_syn = net->d_i;
    sp.refr = net->d_r;
    sp.ring = net->d_ring;
    sp.row_start = net->d_row_start;
    sp.msg = net->d_msg;
    sp.msg_stride = net->msg_stride;
    sp.ras_step = net->d_ras_step;
    sp.ras_id = net->d_ras_id;
    sp.ras_n = net->d_ras_n;
    sp.counters = net->d_counters;
    sp.pop_spikes = net->d_pop_spikes;
    sp.status = net->d_sync + 4;
    sp.abort_flag = net->d_sync + 5;
    sp.step_times = net->step_times;
    sp.st_t0 = net->st_t0;
    sp.st_cap = net->st_cap;
    sp.st_counts = net->step_counts;
    sp.sc_t0 = net->sc_t0;
    sp.sc_cap = net->sc_cap;
    sp.wrap = net->sat_check ? net->d_wrap : nullptr;
}

cudaError_t net_launch(snn_net* net, StepParams& sp, int64_t t0, int64_t n) {
    const int64_t kMaxLaunch = 1ll << 24;
    int64_t left = n, t = t0;
    while (left > 0) {
        const int64_t chunk = std::min(left, kMaxLaunch);
        sp.t0 = t;
        sp.n_steps = (int32_t)chunk;
        cudaError_t e = cudaMemsetAsync(net->d_sync + 5, 0, sizeof(uint32_t), net->stream);
        if (e == cudaSuccess) e = launch_step(sp, net->npt, net->smem_ring, net->smem, net->stream);
        if (e != cudaSuccess) return e;
        t += chunk;
        left -= chunk;
    }
    return cudaSuccess;
}

int net_make_tables(snn_net* net) { return make_tables(net); }

// unrounded weight of every code at projection scale 1, in pA
void net_base_weights(const snn_net* net, float* wb) {
    const snn_config* c = &net->cfg;
    for (int p = 0; p < kMaxPop; ++p)
        for (int q = 0; q < kMaxPop; ++q)
            for (int k = 0; k < kWCodes; ++k) {
                double w = 0.0;
                if (p < c->n_pop && q < c->n_pop) {
                    const double z = norm_quantile(((double)k + 0.5) / (double)kWCodes);
                    w = (c->w_mean[p][q] + c->w_sd[p][q] * z) * c->w_scale;
                }
                wb[(p * kMaxPop + q) * kWCodes + k] = (float)w;
            }
}

int net_upload_weights(snn_net* net) {
    cudaStream_t s = net->stream;
    CK(cudaMemcpyAsync(net->d_wtab, net->wtab, sizeof(net->wtab), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return net_update_saturation(net);
}

long long input_bound(const uint32_t* indeg, int n, int n_pop, const int32_t* pop_start,
                      const int32_t* wtab, int32_t wext_q, int input_mode) {
    long long wmax[kMaxPop][kMaxPop];
    for (int p = 0; p < kMaxPop; ++p)
        for (int q = 0; q < kMaxPop; ++q) {
            long long m = 0;
            for (int k = 0; k < kWCodes; ++k)
                m = std::max(m, std::llabs((long long)wtab[(p * kMaxPop + q) * kWCodes + k]));
            wmax[p][q] = m;
        }
    long long best = 0;
    int p = 0;
    for (int i = 0; i < n; ++i) {
        while (p + 1 < n_pop && i >= pop_start[p + 1]) ++p;
        long long b = 0;
        for (int q = 0; q < kMaxPop; ++q) b += (long long)indeg[(size_t)i * kMaxPop + q] * wmax[p][q];
        best = std::max(best, b);
    }
    if (input_mode == 0) best += (long long)kPoisTable * std::llabs((long long)wext_q);
    return best;
}

int net_update_saturation(snn_net* net) {
    net->in_bound = input_bound(net->indeg.data(), net->n, net->n_pop, net->pop_start, net->wtab,
                                net->wext_q, net->cfg.input_mode);
    net->sat_check = net->in_bound > 2147483647ll;
    if (net->sat_check && !net->d_wrap) {
        const size_t cells = (size_t)net->P * kRing * net->ncmax;
        CALL(dalloc(&net->d_wrap, cells, "wrap counts"));
        CK(cudaMemsetAsync(net->d_wrap, 0, sizeof(int32_t) * cells, net->stream));
        CK(cudaStreamSynchronize(net->stream));
    }
    return SNN_OK;
}

cudaError_t net_clear_wraps(snn_net* net) {
    if (!net->d_wrap) return cudaSuccess;
    return cudaMemsetAsync(net->d_wrap, 0, sizeof(int32_t) * (size_t)net->P * kRing * net->ncmax,
                           net->stream);
}

int partition_pop_span(const int32_t* part_lo, int n_part, const int32_t* pop_start, int n_pop) {
    auto pop_of = [&](int32_t i) {
        int p = 0;
        while (p + 1 < n_pop && i >= pop_start[p + 1]) ++p;
        return p;
    };
    int span = 1;
    for (int c = 0; c < n_part; ++c)
        if (part_lo[c + 1] > part_lo[c])
            span = std::max(span, pop_of(part_lo[c + 1] - 1) - pop_of(part_lo[c]) + 1);
    return span;
}

int set_error(int code, const char* msg) { return fail(code, msg); }

int set_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

}  // namespace snn

extern "C" {

const char* snn_last_error(void) { return g_err.c_str(); }

int snn_create(const snn_config* cfg, uint64_t seed, const snn_options* opt,
               const float* u0_host, void* stream, snn_net** out) {
    if (!out) return fail(SNN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    snn_net* net = nullptr;
    CALL(common_setup(cfg, seed, opt, stream, &net));
    int rc = build_generated(net);
    if (rc == SNN_OK) rc = alloc_state(net, u0_host);
    if (rc != SNN_OK) {
        free_net(net);
        return rc;
    }
    *out = net;
    return SNN_OK;
}

int snn_create_from_rows(const snn_config* cfg, uint64_t seed, const snn_options* opt,
                         const uint64_t* row_ptr_host, const uint32_t* words_host,
                         const int32_t* wtab_host, const float* u0_host, void* stream,
                         snn_net** out) {
    if (!out) return fail(SNN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    snn_net* net = nullptr;
    CALL(common_setup(cfg, seed, opt, stream, &net));
    int rc = build_from_rows(net, row_ptr_host, words_host, wtab_host);
    if (rc == SNN_OK) rc = alloc_state(net, u0_host);
    if (rc != SNN_OK) {
        free_net(net);
        return rc;
    }
    *out = net;
    return SNN_OK;
}

int snn_step(snn_net* net, int64_t n_steps) {
    if (!net) return fail(SNN_ERR_INVALID, "net is NULL");
    if (n_steps < 0) return fail(SNN_ERR_INVALID, "n_steps must be >= 0");
    StepParams sp;
    fill_step_params(net, &sp);
    if (net->rt_period) {
        sp.rt_period_ns = net->rt_period;
        sp.rt_t_anchor = net->rt_t_anchor;
        sp.rt = net->d_rt;
    }
    CK(net_launch(net, sp, net->step, n_steps));
    net->step += n_steps;
    return SNN_OK;
}

int snn_set_realtime(snn_net* net, int64_t period_ns) {
    if (!net || period_ns < 0 || period_ns > 1000000000ll)
        return fail(SNN_ERR_INVALID, "period_ns must be in [0, 1e9]");
    if (!net->d_rt) CALL(dalloc(&net->d_rt, 3, "pacing state"));
    CK(cudaStreamSynchronize(net->stream));
    CK(cudaMemset(net->d_rt, 0, 3 * sizeof(unsigned long long)));
    net->rt_period = (uint64_t)period_ns;
    net->rt_t_anchor = net->step;
    return SNN_OK;
}

int snn_realtime_stats(snn_net* net, int64_t* missed, int64_t* max_late_ns) {
    if (!net || !missed || !max_late_ns) return fail(SNN_ERR_INVALID, "bad arguments");
    *missed = 0;
    *max_late_ns = 0;
    if (!net->d_rt) return SNN_OK;
    unsigned long long h[3];
    CK(cudaStreamSynchronize(net->stream));
    CK(cudaMemcpy(h, net->d_rt, sizeof(h), cudaMemcpyDeviceToHost));
    *missed = (int64_t)h[1];
    *max_late_ns = (int64_t)h[2];
    return SNN_OK;
}

int snn_record_step_times(snn_net* net, int64_t* times_dev, int64_t cap) {
    if (!net || cap < 0 || (times_dev && cap == 0)) return fail(SNN_ERR_INVALID, "bad arguments");
    net->step_times = reinterpret_cast<long long*>(times_dev);
    net->st_t0 = net->step;
    net->st_cap = times_dev ? cap : 0;
    return SNN_OK;
}

int snn_record_step_counts(snn_net* net, uint32_t* counts_dev, int64_t cap) {
    if (!net || cap < 0 || (counts_dev && cap == 0)) return fail(SNN_ERR_INVALID, "bad arguments");
    if (counts_dev)
        CK(cudaMemsetAsync(counts_dev, 0, sizeof(uint32_t) * 4 * (size_t)cap, net->stream));
    net->step_counts = counts_dev;
    net->sc_t0 = net->step;
    net->sc_cap = counts_dev ? cap : 0;
    return SNN_OK;
}

int snn_sync(snn_net* net) {
    if (!net) return fail(SNN_ERR_INVALID, "net is NULL");
    CK(cudaStreamSynchronize(net->stream));
    return check_status(net);
}

int snn_read_spikes(snn_net* net, uint32_t* steps_host, uint32_t* ids_host, int64_t cap,
                    int64_t* n) {
    if (!net || !n || cap < 0) return fail(SNN_ERR_INVALID, "bad arguments");
    CK(cudaStreamSynchronize(net->stream));
    std::vector<uint32_t> cnt(net->P);
    CK(cudaMemcpy(cnt.data(), net->d_ras_n, sizeof(uint32_t) * net->P, cudaMemcpyDeviceToHost));
    int64_t total = 0;
    bool lost = false;
    for (int c = 0; c < net->P; ++c) {
        if (cnt[c] > net->ras_cap) lost = true;
        total += std::min<uint32_t>(cnt[c], net->ras_cap);
    }
    // the first `cap` entries in partition order, packed on the device and
    // copied back in one transfer per array
    const int64_t got = std::min<int64_t>(total, cap);
    if (got > 0 && (steps_host || ids_host)) {
        if (net->rs_cap < (size_t)got) {
            cudaFree(net->d_rs_step);
            cudaFree(net->d_rs_id);
            net->d_rs_step = net->d_rs_id = nullptr;
            net->rs_cap = 0;
            CALL(dalloc(&net->d_rs_step, (size_t)got, "raster staging"));
            CALL(dalloc(&net->d_rs_id, (size_t)got, "raster staging"));
            net->rs_cap = (size_t)got;
        }
        CK(launch_pack_raster(net->d_ras_n, net->P, net->ras_cap, got, net->d_ras_step,
                              net->d_ras_id, net->d_rs_step, net->d_rs_id, net->stream));
        if (steps_host)
            CK(cudaMemcpyAsync(steps_host, net->d_rs_step, sizeof(uint32_t) * got,
                               cudaMemcpyDeviceToHost, net->stream));
        if (ids_host)
            CK(cudaMemcpyAsync(ids_host, net->d_rs_id, sizeof(uint32_t) * got,
                               cudaMemcpyDeviceToHost, net->stream));
    }
    CK(cudaMemsetAsync(net->d_ras_n, 0, sizeof(uint32_t) * net->P, net->stream));
    CK(cudaStreamSynchronize(net->stream));
    *n = got;
    if (lost) return fail(SNN_ERR_OVERFLOW, "spike raster capacity exceeded; spikes were lost");
    if (got < total) return fail(SNN_ERR_OVERFLOW, "cap smaller than the recorded spikes; the rest were dropped");
    return SNN_OK;
}

int snn_raster_size(snn_net* net, int64_t* n) {
    if (!net || !n) return fail(SNN_ERR_INVALID, "bad arguments");
    CK(cudaStreamSynchronize(net->stream));
    std::vector<uint32_t> cnt(net->P);
    CK(cudaMemcpy(cnt.data(), net->d_ras_n, sizeof(uint32_t) * net->P, cudaMemcpyDeviceToHost));
    int64_t total = 0;
    for (int c = 0; c < net->P; ++c) total += std::min<uint32_t>(cnt[c], net->ras_cap);
    *n = total;
    return SNN_OK;
}

int snn_read_state(snn_net* net, float* u_host, float* i_syn_host, int32_t* refr_host) {
    if (!net) return fail(SNN_ERR_INVALID, "net is NULL");
    CK(cudaStreamSynchronize(net->stream));
    if (u_host) CK(cudaMemcpy(u_host, net->d_u, sizeof(float) * net->n, cudaMemcpyDeviceToHost));
    if (i_syn_host) CK(cudaMemcpy(i_syn_host, net->d_i, sizeof(float) * net->n, cudaMemcpyDeviceToHost));
    if (refr_host) CK(cudaMemcpy(refr_host, net->d_r, sizeof(int32_t) * net->n, cudaMemcpyDeviceToHost));
    return SNN_OK;
}

int snn_read_ring(snn_net* net, int32_t* ring_host) {
    if (!net || !ring_host) return fail(SNN_ERR_INVALID, "bad arguments");
    CK(cudaStreamSynchronize(net->stream));
    std::vector<int32_t> tmp((size_t)net->P * kRing * net->ncmax);
    CK(cudaMemcpy(tmp.data(), net->d_ring, sizeof(int32_t) * tmp.size(), cudaMemcpyDeviceToHost));
    for (int c = 0; c < net->P; ++c) {
        const int lo = net->part_lo[c], nc = net->part_lo[c + 1] - lo;
        for (int slot = 0; slot < kRing; ++slot)
            for (int k = 0; k < nc; ++k)
                ring_host[(size_t)slot * net->n + lo + k] =
                    tmp[((size_t)c * kRing + slot) * net->ncmax + k];
    }
    return SNN_OK;
}

int snn_counters(snn_net* net, int64_t* step, uint64_t* spikes, uint64_t* events) {
    if (!net) return fail(SNN_ERR_INVALID, "net is NULL");
    CK(cudaStreamSynchronize(net->stream));
    unsigned long long c[2];
    CK(cudaMemcpy(c, net->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
    if (step) *step = net->step;
    if (spikes) *spikes = c[0];
    if (events) *events = c[1];
    return SNN_OK;
}

int snn_get_info(snn_net* net, snn_info* info) {
    if (!net || !info) return fail(SNN_ERR_INVALID, "bad arguments");
    info->n_neurons = net->n;
    info->n_synapses = (int64_t)net->nnz;
    info->n_part = net->P;
    info->threads = kStepThreads;
    info->neurons_per_thread = net->npt;
    info->ring_in_shared = net->smem_ring ? 1 : 0;
    info->max_part_neurons = net->ncmax;
    info->n_ref = net->n_ref;
    for (int k = 0; k < 4; ++k) info->propagators[k] = net->prop[k];
    info->wext_q = net->wext_q;
    info->shared_bytes = (int32_t)net->smem;
    info->slot_entries = net->run_max;
    info->slot_bytes = (int64_t)(net->nnz * sizeof(uint32_t));
    int active = 0;
    if (deliver_cluster_check(net->ncmax, net->P, &active) != cudaSuccess) {
        cudaGetLastError();
        active = 0;
    }
    info->deliver_clusters_active = active;
    info->saturation_check = net->sat_check ? 1 : 0;
    info->input_bound = (int64_t)net->in_bound;
    return SNN_OK;
}

int snn_export_network(snn_net* net, uint64_t* row_ptr_host, uint32_t* words_host,
                       int32_t* wtab_host) {
    if (!net) return fail(SNN_ERR_INVALID, "net is NULL");
    CK(cudaStreamSynchronize(net->stream));
    if (row_ptr_host)
        CK(cudaMemcpy(row_ptr_host, net->d_row_start, sizeof(uint64_t) * (net->n + 1),
                      cudaMemcpyDeviceToHost));
    if (words_host && net->nnz)
        CK(cudaMemcpy(words_host, net->d_words, sizeof(uint32_t) * net->nnz, cudaMemcpyDeviceToHost));
    if (wtab_host) std::memcpy(wtab_host, net->wtab, sizeof(net->wtab));
    return SNN_OK;
}

int snn_deliver(snn_net* net, const uint32_t* spikes_dev, int32_t n_spikes, int64_t t,
                int32_t tiling) {
    if (!net || n_spikes < 0 || (n_spikes > 0 && !spikes_dev) || tiling < 0 || tiling > 5)
        return fail(SNN_ERR_INVALID, "bad arguments");
    if (tiling == 2) {
        StepParams sp;
        fill_step_params(net, &sp);
        CK(launch_deliver_part(sp, spikes_dev, n_spikes, t, net->smem_ring, net->stream));
        return SNN_OK;
    }
    DeliverParams dp;
    std::memset(&dp, 0, sizeof(dp));
    dp.n = net->n;
    dp.n_pop = net->n_pop;
    dp.n_part = net->P;
    dp.ncmax = net->ncmax;
    dp.n_spikes = n_spikes;
    for (int p = 0; p <= kMaxPop; ++p) dp.pop_start[p] = net->pop_start[p];
    dp.t = t;
    dp.spikes = spikes_dev;
    dp.part_lo = net->d_part_lo;
    dp.seg = net->d_seg;
    dp.words = net->d_words;
    dp.wtab = net->d_wtab;
    dp.ring = net->d_ring;
    dp.counters = net->d_counters;
    dp.status = net->d_sync + 4;
    dp.pre = net->d_pre;
    dp.max_delay = net->max_delay;
    if (tiling == 5) {
        int dev = 0, optin = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (deliver_stream_smem(net->ncmax, net->w_span) > (size_t)optin)
            return fail(SNN_ERR_UNSUPPORTED, "ring slices too large for the streamed delivery");
        CK(launch_deliver_stream(dp, net->w_span, net->stream));
    } else if (tiling == 4) {
        int active = 0;
        if (deliver_cluster_check(net->ncmax, net->P, &active) != cudaSuccess || active < 1) {
            cudaGetLastError();
            return fail(SNN_ERR_UNSUPPORTED, "ring slices too large for the cluster delivery");
        }
        CK(launch_deliver_cluster(dp, net->stream));
    } else if (tiling == 3) {
        CK(launch_deliver_words(dp, net->stream));
    } else {
        CK(launch_deliver(dp, tiling, net->stream));
    }
    return SNN_OK;
}

int snn_destroy(snn_net* net) {
    if (!net) return SNN_OK;
    cudaStreamSynchronize(net->stream);
    free_net(net);
    return SNN_OK;
}

}  // extern "C"
