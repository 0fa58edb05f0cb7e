/*
 * oracle.c -- plain, slow, single-purpose CPU reference of the paper's
 * method: the 0.1 ms time-stepped simulation of the cortical microcircuit
 * (Sec. 2.1, Eq. 1), with the synaptic-input ring buffers of Sec. 3.1.2, the
 * Poisson background of Sec. 3.1.3 and spike recording (Sec. 3.1.2).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library.
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (fp32 arithmetic is
 * evaluated exactly as written, one rounding per operation, no FMA).
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *  - Eq. 1 is read as tau_m dV/dt = -(V-E) + R I_syn (+ R I_DC) and
 *    dI/dt = -I/tau_syn + sum_j w_j delta(t - t_j); u = V - E_L.
 *  - Exact integration on the time grid: u <- P22 u + P21 I (+ P20 I_DC),
 *    I <- P11 I + input; the propagators are computed in double and rounded
 *    once to fp32 (the state precision the benchmark fixes).
 *  - Threshold strict (V > V_theta), reset to rest, then n_ref steps clamped.
 *  - Input arriving in step t enters I in step t and reaches u from step t+1.
 *  - Delays "truncated to the nearest timestep": rounded half away from zero,
 *    clamped to [1, D-1].
 *  - Pairwise Bernoulli connectivity (probabilistic, Sec. 2.1), no autapses.
 *  - Normal weights and delays are drawn by inverse transform on an
 *    equiprobable grid: code c -> Phi^-1((c + 1/2) / M), M = 128 for weights
 *    and 256 for delays.
 *  - Synaptic input is accumulated as int32 fixed point with 8 fractional bits
 *    (1/256 pA) so that summation order cannot change the result; the oracle
 *    accumulates in int64 and flags any sum outside the int32 range.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed split in
 * two 32-bit words, counters
 *    connection test   (j, i>>2, 1, 0) lane i&3      source j, target i
 *    weight / delay    (j, i, 2, 0)   lane 0 >> 25, lane 1 >> 24
 *    Poisson count     (i, t>>2, 3, t>>34) lane t&3  neuron i, step t
 *    initial potential (i, 0, 4, 0)   lane 0
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4 "Philox"): ten    */
/* rounds of two 32x32->64 multiplications with the published multipliers,   */
/* a fixed permutation of the four words and a Weyl-sequence key schedule.   */
/* Pinned: against triton's independent Philox (interpreter on the CPU).     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_seed(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
}

/* ------------------------------------------------------------------------ */
/* Standard-normal quantile by bisection on Phi(x) = erfc(-x/sqrt 2)/2.      */
/* Pinned: against scipy.special.ndtri.                                      */
/* ------------------------------------------------------------------------ */
double orc_norm_quantile(double p)
{
    /* lower half: Phi(x) = p with x <= 0; upper half by symmetry on the tail
     * 1 - Phi(x) = erfc(x/sqrt 2)/2 = 1 - p, which keeps relative precision */
    int upper = p > 0.5;
    double target = upper ? 1.0 - p : p;
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (0.5 * erfc(-mid / sqrt(2.0)) < target) lo = mid;
        else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    return upper ? -x : x;
}

/* ------------------------------------------------------------------------ */
/* Exact propagators of Eq. 1 over one step dt (Sec. 2.1).                   */
/*   u' = -u/tau_m + I/C_m,  I' = -I/tau_syn                                 */
/*   P22 = exp(-dt/tau_m), P11 = exp(-dt/tau_syn),                          */
/*   P21 = tau_m tau_syn / (C_m (tau_m - tau_syn)) (P22 - P11)   [mV/pA]    */
/*   P20 = tau_m / C_m (1 - P22)                                  [mV/pA]    */
/* Pinned: against the matrix exponential of the 2x2 (3x3 with DC) system.  */
/* ------------------------------------------------------------------------ */
void orc_propagators(const orc_config* c, double out_d[4], float out_f[4])
{
    double P22 = exp(-c->dt / c->tau_m);
    double P11 = exp(-c->dt / c->tau_syn);
    double P21 = (c->tau_m * c->tau_syn) / (c->c_m * (c->tau_m - c->tau_syn)) * (P22 - P11);
    double P20 = c->tau_m / c->c_m * (1.0 - P22);
    out_d[0] = P22; out_d[1] = P21; out_d[2] = P11; out_d[3] = P20;
    for (int k = 0; k < 4; ++k) out_f[k] = (float)out_d[k];
}

/* ------------------------------------------------------------------------ */
/* Poisson background (Sec. 3.1.3, Poisson core): the number of background   */
/* spikes k in one step is Poisson(lambda), lambda = nu_bg K_ext dt.  It is   */
/* drawn from one uniform 32-bit word x by inverse transform on the integer  */
/* thresholds T_m = floor(2^32 F(m)), F the Poisson CDF summed term by term  */
/* (e^-l, then term *= l/m): k = #{m < 32 : x >= T_m}.                       */
/* Pinned: thresholds against scipy.stats.poisson.cdf, draws by chi-square.  */
/* ------------------------------------------------------------------------ */
void orc_poisson_thresholds(double lam, uint64_t thr[ORC_POIS_TABLE])
{
    double term = exp(-lam);
    double cdf = term;
    for (int m = 0; m < ORC_POIS_TABLE; ++m) {
        if (m > 0) {
            term = term * lam / (double)m;
            cdf = cdf + term;
        }
        double x = floor(cdf * 4294967296.0);
        thr[m] = (x >= 4294967296.0) ? 4294967296ull : (uint64_t)x;
    }
}

int orc_poisson_count(uint32_t x, const uint64_t thr[ORC_POIS_TABLE])
{
    int k = 0;
    for (int m = 0; m < ORC_POIS_TABLE; ++m)
        if ((uint64_t)x >= thr[m]) ++k;
    return k;
}

void orc_poisson_draws(uint64_t seed, int64_t neuron, int64_t t0, int64_t n,
                       const uint64_t thr[ORC_POIS_TABLE], int32_t* counts)
{
    uint32_t key[2], out[4];
    philox_seed(seed, key);
    for (int64_t s = 0; s < n; ++s) {
        int64_t t = t0 + s;
        uint32_t ctr[4] = {(uint32_t)neuron, (uint32_t)(t >> 2), 3u, (uint32_t)(t >> 34)};
        orc_philox4x32_10(ctr, key, out);
        counts[s] = orc_poisson_count(out[t & 3], thr);
    }
}

/* ------------------------------------------------------------------------ */
/* Parameter tables.                                                         */
/*  wtab[(p*8+q)*128+c] = llround(256 ((mu_pq + sd_pq z_c) w_scale) alpha_pq) */
/*      z_c = Phi^-1((c + 0.5)/128)   (normal weights, Sec. 2.1)             */
/*  dtab[q*256+c] = clamp(round((dmu_q + dsd_q z_c) / dt), 1, D-1)            */
/*      z_c = Phi^-1((c + 0.5)/256)   (normal delays rounded to dt, Sec. 2.1) */
/*  pois[p*32+m]  Poisson thresholds for lambda_p = nu_bg K_ext,p (dt/1000)   */
/*  conn_thr[p*8+q] = min(floor(p_pq conn_scale 2^32), 2^32)                  */
/* Returns 0, or -1 if a weight does not fit comfortably in int32.           */
/* ------------------------------------------------------------------------ */
int orc_tables(const orc_config* c, int32_t* wtab, uint8_t* dtab, uint64_t* pois,
               uint64_t* conn_thr, int32_t* wext_q, int32_t* n_ref)
{
    int np = c->n_pop;
    for (int p = 0; p < ORC_MAX_POP; ++p)
        for (int q = 0; q < ORC_MAX_POP; ++q) {
            for (int k = 0; k < ORC_WCODES; ++k) {
                int32_t v = 0;
                if (p < np && q < np) {
                    double z = orc_norm_quantile(((double)k + 0.5) / (double)ORC_WCODES);
                    double w = c->w_mean[p][q] + c->w_sd[p][q] * z;
                    w = w * c->w_scale;
                    w = w * c->proj_scale[p][q];
                    double qv = w * 256.0;
                    if (!(fabs(qv) < 1073741824.0)) return -1;
                    v = (int32_t)llround(qv);
                }
                wtab[(p * ORC_MAX_POP + q) * ORC_WCODES + k] = v;
            }
            double thr = 0.0;
            if (p < np && q < np) {
                double pr = c->conn_prob[p][q] * c->conn_scale;
                thr = floor(pr * 4294967296.0);
                if (thr < 0.0) thr = 0.0;
                if (thr > 4294967296.0) thr = 4294967296.0;
            }
            conn_thr[p * ORC_MAX_POP + q] = (uint64_t)thr;
        }
    for (int q = 0; q < ORC_MAX_POP; ++q)
        for (int k = 0; k < ORC_DCODES; ++k) {
            int d = 1;
            if (q < np) {
                double z = orc_norm_quantile(((double)k + 0.5) / (double)ORC_DCODES);
                double steps = (c->d_mean[q] + c->d_sd[q] * z) / c->dt;
                double r = round(steps);
                if (r < 1.0) r = 1.0;
                if (r > (double)(c->ring_depth - 1)) r = (double)(c->ring_depth - 1);
                d = (int)r;
            }
            dtab[q * ORC_DCODES + k] = (uint8_t)d;
        }
    for (int p = 0; p < ORC_MAX_POP; ++p) {
        double lam = (p < np) ? c->nu_bg * c->k_ext[p] * (c->dt / 1000.0) : 0.0;
        orc_poisson_thresholds(lam, pois + p * ORC_POIS_TABLE);
    }
    *wext_q = (int32_t)llround(c->w_ext * 256.0);
    *n_ref = (int32_t)llround(c->t_ref / c->dt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Network: one row per presynaptic neuron (Sec. 3.1.2: "row-indexed by      */
/* presynaptic neuron"), each word = (target, delay, weight code).  Rows are */
/* in ascending target order.                                                */
/* ------------------------------------------------------------------------ */
struct orc_net {
    int64_t n;
    int n_pop;
    int64_t pop_start[ORC_MAX_POP + 1];
    int64_t* row_ptr;
    int32_t* tgt;
    uint8_t* delay;
    uint8_t* wcode;
    int32_t wtab[ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES];
};

static int pop_of(const int64_t* pop_start, int n_pop, int64_t i)
{
    int p = 0;
    while (p + 1 < n_pop && i >= pop_start[p + 1]) ++p;
    return p;
}

typedef struct {
    int32_t wtab[ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES];
    uint8_t dtab[ORC_MAX_POP * ORC_DCODES];
    uint64_t pois[ORC_MAX_POP * ORC_POIS_TABLE];
    uint64_t conn_thr[ORC_MAX_POP * ORC_MAX_POP];
    int32_t wext_q, n_ref;
    int64_t pop_start[ORC_MAX_POP + 1];
    int n_pop;
    int64_t n;
    uint32_t key[2];
} gen_ctx;

static int gen_ctx_init(gen_ctx* g, const orc_config* c, uint64_t seed)
{
    if (orc_tables(c, g->wtab, g->dtab, g->pois, g->conn_thr, &g->wext_q, &g->n_ref)) return -1;
    g->n_pop = c->n_pop;
    g->pop_start[0] = 0;
    for (int p = 0; p < c->n_pop; ++p) g->pop_start[p + 1] = g->pop_start[p] + c->pop_size[p];
    g->n = g->pop_start[c->n_pop];
    philox_seed(seed, g->key);
    return 0;
}

/* Row of source j: every target i != j is tested once (pairwise Bernoulli). */
static int64_t gen_row(const gen_ctx* g, int64_t j, int32_t* tgt, uint8_t* delay,
                       uint8_t* wcode, int64_t cap)
{
    int q = pop_of(g->pop_start, g->n_pop, j);
    int64_t count = 0;
    uint32_t out[4], syn[4];
    for (int64_t grp = 0; 4 * grp < g->n; ++grp) {
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)grp, 1u, 0u};
        orc_philox4x32_10(ctr, g->key, out);
        for (int lane = 0; lane < 4; ++lane) {
            int64_t i = 4 * grp + lane;
            if (i >= g->n) break;
            if (i == j) continue;
            int p = pop_of(g->pop_start, g->n_pop, i);
            if ((uint64_t)out[lane] < g->conn_thr[p * ORC_MAX_POP + q]) {
                if (tgt != NULL && count < cap) {
                    uint32_t sctr[4] = {(uint32_t)j, (uint32_t)i, 2u, 0u};
                    orc_philox4x32_10(sctr, g->key, syn);
                    tgt[count] = (int32_t)i;
                    wcode[count] = (uint8_t)(syn[0] >> 25);
                    delay[count] = g->dtab[q * ORC_DCODES + (syn[1] >> 24)];
                }
                ++count;
            }
        }
    }
    return count;
}

typedef struct {
    const gen_ctx* g;
    orc_net* net;
    int64_t* counts;
    int tid, nthreads, fill;
} gen_job;

static void* gen_worker(void* arg)
{
    gen_job* jb = (gen_job*)arg;
    for (int64_t j = jb->tid; j < jb->g->n; j += jb->nthreads) {
        if (!jb->fill) {
            jb->counts[j] = gen_row(jb->g, j, NULL, NULL, NULL, 0);
        } else {
            int64_t b = jb->net->row_ptr[j];
            gen_row(jb->g, j, jb->net->tgt + b, jb->net->delay + b, jb->net->wcode + b,
                    jb->net->row_ptr[j + 1] - b);
        }
    }
    return NULL;
}

static void run_jobs(const gen_ctx* g, orc_net* net, int64_t* counts, int fill, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    gen_job* jobs = (gen_job*)calloc((size_t)nthreads, sizeof(gen_job));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].g = g; jobs[t].net = net; jobs[t].counts = counts;
        jobs[t].tid = t; jobs[t].nthreads = nthreads; jobs[t].fill = fill;
        if (nthreads == 1) gen_worker(&jobs[t]);
        else pthread_create(&th[t], NULL, gen_worker, &jobs[t]);
    }
    if (nthreads > 1)
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}

orc_net* orc_net_generate(const orc_config* c, uint64_t seed, int n_threads)
{
    gen_ctx* g = (gen_ctx*)malloc(sizeof(gen_ctx));
    if (gen_ctx_init(g, c, seed)) { free(g); return NULL; }
    orc_net* net = (orc_net*)calloc(1, sizeof(orc_net));
    net->n = g->n;
    net->n_pop = g->n_pop;
    memcpy(net->pop_start, g->pop_start, sizeof(net->pop_start));
    memcpy(net->wtab, g->wtab, sizeof(net->wtab));
    int64_t* counts = (int64_t*)calloc((size_t)g->n, sizeof(int64_t));
    run_jobs(g, net, counts, 0, n_threads);
    net->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->n + 1));
    net->row_ptr[0] = 0;
    for (int64_t j = 0; j < g->n; ++j) net->row_ptr[j + 1] = net->row_ptr[j] + counts[j];
    int64_t nnz = net->row_ptr[g->n];
    net->tgt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    net->delay = (uint8_t*)malloc((size_t)(nnz > 0 ? nnz : 1));
    net->wcode = (uint8_t*)malloc((size_t)(nnz > 0 ? nnz : 1));
    run_jobs(g, net, counts, 1, n_threads);
    free(counts);
    free(g);
    return net;
}

int64_t orc_net_row(const orc_config* c, uint64_t seed, int64_t j, int32_t* tgt,
                    uint8_t* delay, uint8_t* wcode, int64_t cap)
{
    gen_ctx* g = (gen_ctx*)malloc(sizeof(gen_ctx));
    if (gen_ctx_init(g, c, seed)) { free(g); return -1; }
    int64_t n = gen_row(g, j, tgt, delay, wcode, cap);
    free(g);
    return n;
}

orc_net* orc_net_custom(const orc_config* c, const int64_t* row_ptr, const int32_t* tgt,
                        const uint8_t* delay, const uint8_t* wcode, const int32_t* wtab)
{
    orc_net* net = (orc_net*)calloc(1, sizeof(orc_net));
    net->n_pop = c->n_pop;
    net->pop_start[0] = 0;
    for (int p = 0; p < c->n_pop; ++p) net->pop_start[p + 1] = net->pop_start[p] + c->pop_size[p];
    net->n = net->pop_start[c->n_pop];
    int64_t nnz = row_ptr[net->n];
    net->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(net->n + 1));
    memcpy(net->row_ptr, row_ptr, sizeof(int64_t) * (size_t)(net->n + 1));
    net->tgt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    net->delay = (uint8_t*)malloc((size_t)(nnz > 0 ? nnz : 1));
    net->wcode = (uint8_t*)malloc((size_t)(nnz > 0 ? nnz : 1));
    if (nnz > 0) {
        memcpy(net->tgt, tgt, sizeof(int32_t) * (size_t)nnz);
        memcpy(net->delay, delay, (size_t)nnz);
        memcpy(net->wcode, wcode, (size_t)nnz);
    }
    memcpy(net->wtab, wtab, sizeof(net->wtab));
    return net;
}

int64_t orc_net_neurons(const orc_net* n) { return n->n; }
int64_t orc_net_synapses(const orc_net* n) { return n->row_ptr[n->n]; }

void orc_net_export(const orc_net* n, int64_t* row_ptr, int32_t* tgt, uint8_t* delay,
                    uint8_t* wcode)
{
    int64_t nnz = n->row_ptr[n->n];
    memcpy(row_ptr, n->row_ptr, sizeof(int64_t) * (size_t)(n->n + 1));
    if (tgt) memcpy(tgt, n->tgt, sizeof(int32_t) * (size_t)nnz);
    if (delay) memcpy(delay, n->delay, (size_t)nnz);
    if (wcode) memcpy(wcode, n->wcode, (size_t)nnz);
}

void orc_net_free(orc_net* n)
{
    if (!n) return;
    free(n->row_ptr); free(n->tgt); free(n->delay); free(n->wcode);
    free(n);
}

/* ------------------------------------------------------------------------ */
/* Simulation (Sec. 2.1 Eq. 1; Sec. 3.1.2 ring buffers; Sec. 3.1.3 steps).   */
/* ------------------------------------------------------------------------ */
struct orc_sim {
    const orc_net* net;
    int64_t n;
    int D;
    int mode;
    float P22, P21, P11, theta;
    float cdc[ORC_MAX_POP];
    int32_t n_ref, wext_q;
    uint64_t pois[ORC_MAX_POP * ORC_POIS_TABLE];
    uint32_t key[2];
    float* u;
    float* i_syn;
    int32_t* refr;
    int64_t* ring;          /* [D][n] */
    int32_t* spk;
    int64_t step, spikes, events;
    int32_t saturated;
    int64_t* rs_step;
    int32_t* rs_id;
    int64_t rs_n, rs_cap;
    float* tr_u;            /* optional per-step trace (gradient runs) */
    uint8_t* tr_f;
    int32_t* tr_k;
};

orc_sim* orc_sim_create(const orc_net* net, const orc_config* c, uint64_t seed, const float* u0)
{
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    int32_t wtab_unused[ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES];
    uint8_t dtab_unused[ORC_MAX_POP * ORC_DCODES];
    uint64_t conn_unused[ORC_MAX_POP * ORC_MAX_POP];
    if (orc_tables(c, wtab_unused, dtab_unused, s->pois, conn_unused, &s->wext_q, &s->n_ref)) {
        free(s);
        return NULL;
    }
    double pd[4];
    float pf[4];
    orc_propagators(c, pd, pf);
    s->P22 = pf[0]; s->P21 = pf[1]; s->P11 = pf[2];
    for (int p = 0; p < ORC_MAX_POP; ++p)
        s->cdc[p] = (p < c->n_pop) ? (float)(pd[3] * c->i_dc[p]) : 0.0f;
    s->theta = (float)c->theta;
    s->mode = c->input_mode;
    s->net = net;
    s->n = net->n;
    s->D = c->ring_depth;
    philox_seed(seed, s->key);
    s->u = (float*)malloc(sizeof(float) * (size_t)s->n);
    s->i_syn = (float*)calloc((size_t)s->n, sizeof(float));
    s->refr = (int32_t*)calloc((size_t)s->n, sizeof(int32_t));
    s->ring = (int64_t*)calloc((size_t)s->D * (size_t)s->n, sizeof(int64_t));
    s->spk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->n > 0 ? s->n : 1));
    if (u0) {
        memcpy(s->u, u0, sizeof(float) * (size_t)s->n);
    } else {
        /* default initial potential: uniform on [u0_lo, u0_hi) from 24 bits */
        float lo = (float)c->u0_lo, hi = (float)c->u0_hi;
        float span = hi - lo;
        uint32_t out[4];
        for (int64_t i = 0; i < s->n; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, 0u, 4u, 0u};
            orc_philox4x32_10(ctr, s->key, out);
            float unit = (float)(out[0] >> 8) * 5.9604644775390625e-08f; /* 2^-24 */
            float m = span * unit;
            s->u[i] = lo + m;
        }
    }
    s->rs_cap = 1024;
    s->rs_step = (int64_t*)malloc(sizeof(int64_t) * (size_t)s->rs_cap);
    s->rs_id = (int32_t*)malloc(sizeof(int32_t) * (size_t)s->rs_cap);
    return s;
}

static void raster_push(orc_sim* s, int64_t t, int32_t i)
{
    if (s->rs_n == s->rs_cap) {
        s->rs_cap *= 2;
        s->rs_step = (int64_t*)realloc(s->rs_step, sizeof(int64_t) * (size_t)s->rs_cap);
        s->rs_id = (int32_t*)realloc(s->rs_id, sizeof(int32_t) * (size_t)s->rs_cap);
    }
    s->rs_step[s->rs_n] = t;
    s->rs_id[s->rs_n] = i;
    s->rs_n++;
}

/* One time step t, in the order the method defines it. */
static void sim_step(orc_sim* s)
{
    const orc_net* net = s->net;
    const int64_t n = s->n;
    const int64_t t = s->step;
    const int64_t slot = t % s->D;
    int64_t n_spk = 0;
    uint32_t out[4];
    for (int64_t i = 0; i < n; ++i) {
        int p = pop_of(net->pop_start, net->n_pop, i);
        int k = 0, updated = 0;
        /* 1. input for this step from the neuron's ring buffer; clear slot */
        int64_t acc = s->ring[slot * n + i];
        s->ring[slot * n + i] = 0;
        /* 2. Poisson background: k spikes of weight w_ext */
        if (s->mode == 0) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(t >> 2), 3u, (uint32_t)(t >> 34)};
            orc_philox4x32_10(ctr, s->key, out);
            k = orc_poisson_count(out[t & 3], s->pois + p * ORC_POIS_TABLE);
            acc += (int64_t)k * (int64_t)s->wext_q;
        }
        if (acc > 2147483647LL || acc < -2147483648LL) s->saturated = 1;
        int32_t acc32 = (int32_t)acc;
        /* 3. membrane: refractory clamp, else exact propagation with old I */
        if (s->refr[i] > 0) {
            s->refr[i] -= 1;
            s->u[i] = 0.0f;
        } else {
            float a = s->P22 * s->u[i];
            float b = s->P21 * s->i_syn[i];
            float v = a + b;
            if (s->mode == 1) v = v + s->cdc[p];
            s->u[i] = v;
            updated = 1;
        }
        if (s->tr_u) {
            s->tr_u[i] = s->u[i];
            s->tr_f[i] = (uint8_t)(updated << 1);
            s->tr_k[i] = k;
        }
        /* 4. synaptic current: decay, then this step's input (1/256 pA units) */
        float decay = s->P11 * s->i_syn[i];
        float input = (float)acc32 * 0.00390625f;
        s->i_syn[i] = decay + input;
        /* 5. threshold (strict), reset, refractory */
        if (s->u[i] > s->theta) {
            s->u[i] = 0.0f;
            s->refr[i] = s->n_ref;
            s->spk[n_spk++] = (int32_t)i;
            raster_push(s, t, (int32_t)i);
            if (s->tr_f) s->tr_f[i] |= 1u;
        }
    }
    if (s->tr_u) {
        s->tr_u += n;
        s->tr_f += n;
        s->tr_k += n;
    }
    /* 6. deliver every spike through its row into the ring slots t + d */
    for (int64_t k = 0; k < n_spk; ++k) {
        int64_t j = s->spk[k];
        int q = pop_of(net->pop_start, net->n_pop, j);
        for (int64_t e = net->row_ptr[j]; e < net->row_ptr[j + 1]; ++e) {
            int64_t i = net->tgt[e];
            int p = pop_of(net->pop_start, net->n_pop, i);
            int32_t w = net->wtab[(p * ORC_MAX_POP + q) * ORC_WCODES + net->wcode[e]];
            int64_t slot_d = (t + net->delay[e]) % s->D;
            s->ring[slot_d * n + i] += w;
        }
        s->events += net->row_ptr[j + 1] - net->row_ptr[j];
    }
    s->spikes += n_spk;
    s->step += 1;
}

/* Step 6 alone for an arbitrary spike list of step t: every word of every
 * listed row adds its weight to ring slot (t + delay) mod D of its target
 * (Sec. 3.1.2).  ring is [D][n], int64. */
void orc_deliver(const orc_net* net, const orc_config* c, const int32_t* spikes, int64_t n_spikes,
                 int64_t t, int64_t* ring)
{
    const int64_t n = net->n;
    const int D = c->ring_depth;
    for (int64_t k = 0; k < n_spikes; ++k) {
        int64_t j = spikes[k];
        int q = pop_of(net->pop_start, net->n_pop, j);
        for (int64_t e = net->row_ptr[j]; e < net->row_ptr[j + 1]; ++e) {
            int64_t i = net->tgt[e];
            int p = pop_of(net->pop_start, net->n_pop, i);
            ring[((t + net->delay[e]) % D) * n + i] +=
                net->wtab[(p * ORC_MAX_POP + q) * ORC_WCODES + net->wcode[e]];
        }
    }
}

int64_t orc_sim_run(orc_sim* s, int64_t n_steps)
{
    int64_t before = s->rs_n;
    for (int64_t k = 0; k < n_steps; ++k) sim_step(s);
    return s->rs_n - before;
}

/* orc_sim_run with a record of every step: u_trace[t][i] = u after the
 * membrane update of step t (before reset), flags[t][i] = spike (bit 0) |
 * non-refractory update (bit 1), kbg[t][i] = Poisson count of step t. */
int64_t orc_sim_run_trace(orc_sim* s, int64_t n_steps, float* u_trace, uint8_t* flags,
                          int32_t* kbg)
{
    s->tr_u = u_trace;
    s->tr_f = flags;
    s->tr_k = kbg;
    int64_t r = orc_sim_run(s, n_steps);
    s->tr_u = NULL;
    s->tr_f = NULL;
    s->tr_k = NULL;
    return r;
}

int64_t orc_sim_raster_count(const orc_sim* s) { return s->rs_n; }

void orc_sim_raster_read(orc_sim* s, int64_t* steps, int32_t* ids)
{
    memcpy(steps, s->rs_step, sizeof(int64_t) * (size_t)s->rs_n);
    memcpy(ids, s->rs_id, sizeof(int32_t) * (size_t)s->rs_n);
    s->rs_n = 0;
}

void orc_sim_state(const orc_sim* s, float* u, float* i_syn, int32_t* refr, int64_t* ring)
{
    if (u) memcpy(u, s->u, sizeof(float) * (size_t)s->n);
    if (i_syn) memcpy(i_syn, s->i_syn, sizeof(float) * (size_t)s->n);
    if (refr) memcpy(refr, s->refr, sizeof(int32_t) * (size_t)s->n);
    if (ring) memcpy(ring, s->ring, sizeof(int64_t) * (size_t)s->D * (size_t)s->n);
}

void orc_sim_set_state(orc_sim* s, const float* u, const float* i_syn, const int32_t* refr,
                       const int64_t* ring, int64_t step)
{
    if (u) memcpy(s->u, u, sizeof(float) * (size_t)s->n);
    if (i_syn) memcpy(s->i_syn, i_syn, sizeof(float) * (size_t)s->n);
    if (refr) memcpy(s->refr, refr, sizeof(int32_t) * (size_t)s->n);
    if (ring) memcpy(s->ring, ring, sizeof(int64_t) * (size_t)s->D * (size_t)s->n);
    s->step = step;
}

void orc_sim_counters(const orc_sim* s, int64_t* step, int64_t* spikes, int64_t* events,
                      int32_t* saturated)
{
    *step = s->step;
    *spikes = s->spikes;
    *events = s->events;
    *saturated = s->saturated;
}

void orc_sim_free(orc_sim* s)
{
    if (!s) return;
    free(s->u); free(s->i_syn); free(s->refr); free(s->ring); free(s->spk);
    free(s->rs_step); free(s->rs_id);
    free(s);
}

/* ======================================================================== */
/* Gradient of a population-rate loss with respect to the 64 projection      */
/* weight scales alpha_pq (cfg.proj_scale) and the background rate nu        */
/* (cfg.nu_bg).  The paper has no gradient; this is the differentiable form  */
/* of its benchmark network (Sec. 2.1, Eq. 1), by backpropagation through    */
/* time on the same step grid.  Rates r_p = (spikes of pop p) / (N_p T).     */
/*                                                                          */
/* Two models share one adjoint routine (orc_grad_backward):                */
/*  mode 0, hard model with surrogate derivative: the forward is the        */
/*    simulation above; d s / d u := 1 / (1 + 10 |u - theta|)^2 (fast        */
/*    sigmoid, slope 10 per mV); reset and refractory are treated as          */
/*    constants (u_after = u (1 - s) with s held fixed; steps clamped by the   */
/*    refractory counter pass no gradient); the fixed-point rounding of the   */
/*    weights and the Poisson count are passed straight through:              */
/*    d w / d alpha_pq = w_base, d k / d nu = K_ext dt.                       */
/*  mode 1, sigmoid-relaxed model in double: s = 1/(1 + exp(-10 (u-theta))),  */
/*    soft reset u_after = u (1 - s), no refractory period, unrounded          */
/*    weights alpha_pq w_base, background (lambda + sqrt(lambda) z) w_ext     */
/*    with fixed normal draws z; its gradient is exact.                        */
/*                                                                          */
/* Pins: mode 1 against central finite differences of orc_relaxed_forward;  */
/* mode 0 against central finite differences of orc_surrogate_forward, a     */
/* smooth model whose exact gradient at the expansion point is the surrogate */
/* gradient (spikes s* + F(u - theta) - F(u* - theta), F(x) = x/(1+10|x|),    */
/* around a recorded hard trajectory u*, s*).                                 */
/* ======================================================================== */

static double fast_sigmoid_slope(double x) { double a = 1.0 + 10.0 * fabs(x); return 1.0 / (a * a); }
static double fast_sigmoid(double x) { return x / (1.0 + 10.0 * fabs(x)); }
static double logistic10(double x) { return 1.0 / (1.0 + exp(-10.0 * x)); }

/* unrounded base weight of code k of projection q -> p, in pA */
static double base_weight(const orc_config* c, int p, int q, int k)
{
    double z = orc_norm_quantile(((double)k + 0.5) / (double)ORC_WCODES);
    return (c->w_mean[p][q] + c->w_sd[p][q] * z) * c->w_scale;
}

static void base_table(const orc_config* c, double* wb)
{
    for (int p = 0; p < ORC_MAX_POP; ++p)
        for (int q = 0; q < ORC_MAX_POP; ++q)
            for (int k = 0; k < ORC_WCODES; ++k)
                wb[(p * ORC_MAX_POP + q) * ORC_WCODES + k] =
                    (p < c->n_pop && q < c->n_pop) ? base_weight(c, p, q, k) : 0.0;
}

/* d L / d s_{j,t} of the rate loss: g_rate[p] / (N_p T_seconds) */
static void spike_loss_weights(const orc_config* c, int64_t n_steps, const double* g_rate,
                               double* gs)
{
    double T = (double)n_steps * c->dt / 1000.0;
    for (int p = 0; p < ORC_MAX_POP; ++p)
        gs[p] = (p < c->n_pop && c->pop_size[p] > 0) ? g_rate[p] / ((double)c->pop_size[p] * T) : 0.0;
}

/*
 * Adjoint pass, from the last step back to the first.  With lu_t = dL/du_t
 * (u after the update of step t, before reset), lI_t = dL/dI_t, m_t = 1 when
 * step t took the non-refractory update:
 *   ds_{j,t} = dL/ds_{j,t} = gs[p(j)] + sum over row j of  W * lI_{i,t+d}
 *   lu_t     = ds_t * s'(u_t) + R_t * lubar_t,  lubar_t = m_{t+1} P22 lu_{t+1}
 *   lI_t     = P11 lI_{t+1} + m_{t+1} P21 lu_{t+1}
 * (R_t = 1 - s_t for the detached reset, (1 - s) - u s' for the soft reset),
 *   dL/dalpha_pq += s_{j,t} w_base(p,q,code) lI_{i,t+d}   (words of j into p)
 *   dL/dnu       += lI_{i,t} d x_{i,t} / d nu.
 * u_tr, s_tr: [n_steps][n]; m_tr: [n_steps][n] (ignored in mode 1, where
 * every step updates); z: [n_steps][n] (mode 1 only).
 */
int orc_grad_backward(const orc_net* net, const orc_config* c, int mode, int64_t n_steps,
                      const double* u_tr, const double* s_tr, const uint8_t* m_tr,
                      const double* z, const double* g_rate, double* g_alpha, double* g_nu)
{
    const int64_t n = net->n;
    const int D = c->ring_depth;
    double pd[4];
    float pf[4];
    orc_propagators(c, pd, pf);
    const double P22 = mode == 0 ? (double)pf[0] : pd[0];
    const double P21 = mode == 0 ? (double)pf[1] : pd[1];
    const double P11 = mode == 0 ? (double)pf[2] : pd[2];
    const double theta = mode == 0 ? (double)(float)c->theta : c->theta;
    double* wb = (double*)malloc(sizeof(double) * ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES);
    double* weff = (double*)malloc(sizeof(double) * ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES);
    base_table(c, wb);
    for (int p = 0; p < ORC_MAX_POP; ++p)
        for (int q = 0; q < ORC_MAX_POP; ++q)
            for (int k = 0; k < ORC_WCODES; ++k) {
                int idx = (p * ORC_MAX_POP + q) * ORC_WCODES + k;
                weff[idx] = mode == 0 ? (double)net->wtab[idx] / 256.0 : c->proj_scale[p][q] * wb[idx];
            }
    double gs[ORC_MAX_POP];
    spike_loss_weights(c, n_steps, g_rate, gs);
    /* d x / d nu per population (mode 0) or its z-free part (mode 1) */
    const double dts = c->dt / 1000.0;
    double wq = mode == 0 ? (double)llround(c->w_ext * 256.0) / 256.0 : c->w_ext;
    double dnu[ORC_MAX_POP], lam[ORC_MAX_POP];
    for (int p = 0; p < ORC_MAX_POP; ++p) {
        dnu[p] = (p < c->n_pop && c->input_mode == 0) ? wq * c->k_ext[p] * dts : 0.0;
        lam[p] = (p < c->n_pop) ? c->nu_bg * c->k_ext[p] * dts : 0.0;
    }
    double* lu = (double*)calloc((size_t)n, sizeof(double));
    double* lI = (double*)calloc((size_t)n, sizeof(double));
    uint8_t* mnext = (uint8_t*)calloc((size_t)n, 1);
    double* lIr = (double*)calloc((size_t)D * (size_t)n, sizeof(double));
    double* ds = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double ga[ORC_MAX_POP * ORC_MAX_POP] = {0};
    double gnu = 0.0;
    for (int64_t t = n_steps - 1; t >= 0; --t) {
        const double* ut = u_tr + t * n;
        const double* st = s_tr + t * n;
        /* spikes: loss term plus everything they feed through the rows */
        for (int64_t j = 0; j < n; ++j) {
            int q = pop_of(net->pop_start, net->n_pop, j);
            double acc = gs[q];
            for (int64_t e = net->row_ptr[j]; e < net->row_ptr[j + 1]; ++e) {
                int64_t i = net->tgt[e];
                int p = pop_of(net->pop_start, net->n_pop, i);
                int idx = (p * ORC_MAX_POP + q) * ORC_WCODES + net->wcode[e];
                double l = lIr[((t + net->delay[e]) % D) * n + i];
                acc += weff[idx] * l;
                if (st[j] != 0.0) ga[p * ORC_MAX_POP + q] += st[j] * wb[idx] * l;
            }
            ds[j] = acc;
        }
        /* membrane and current adjoints of step t */
        for (int64_t i = 0; i < n; ++i) {
            int p = pop_of(net->pop_start, net->n_pop, i);
            double lub = mnext[i] ? P22 * lu[i] : 0.0;
            double lIt = P11 * lI[i] + (mnext[i] ? P21 * lu[i] : 0.0);
            double x = ut[i] - theta, s = st[i], lut;
            if (mode == 0) {
                lut = ds[i] * fast_sigmoid_slope(x) + (1.0 - s) * lub;
            } else {
                double sp = 10.0 * s * (1.0 - s);
                lut = ds[i] * sp + ((1.0 - s) - ut[i] * sp) * lub;
            }
            lu[i] = lut;
            lI[i] = lIt;
            mnext[i] = mode == 0 ? (uint8_t)((m_tr[t * n + i] >> 1) & 1u) : 1u;
            lIr[(t % D) * n + i] = lIt;
            double dx = dnu[p];
            if (mode == 1 && lam[p] > 0.0) dx *= 1.0 + z[t * n + i] / (2.0 * sqrt(lam[p]));
            gnu += lIt * dx;
        }
    }
    for (int k = 0; k < ORC_MAX_POP * ORC_MAX_POP; ++k) g_alpha[k] = ga[k];
    *g_nu = gnu;
    free(wb); free(weff); free(lu); free(lI); free(mnext); free(lIr); free(ds);
    return 0;
}

/* Sigmoid-relaxed model (mode 1 above), forward in double.  u0: initial
 * potentials; z: [n_steps][n] normal draws; u_tr, s_tr may be NULL. */
int orc_relaxed_forward(const orc_net* net, const orc_config* c, int64_t n_steps,
                        const double* u0, const double* z, double* u_tr, double* s_tr,
                        double* rates)
{
    const int64_t n = net->n;
    const int D = c->ring_depth;
    double pd[4];
    float pf[4];
    orc_propagators(c, pd, pf);
    double* wb = (double*)malloc(sizeof(double) * ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES);
    base_table(c, wb);
    const double dts = c->dt / 1000.0;
    double lam[ORC_MAX_POP];
    for (int p = 0; p < ORC_MAX_POP; ++p) lam[p] = (p < c->n_pop) ? c->nu_bg * c->k_ext[p] * dts : 0.0;
    double* u = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* I = (double*)calloc((size_t)n, sizeof(double));
    double* s = (double*)calloc((size_t)n, sizeof(double));
    double* ring = (double*)calloc((size_t)D * (size_t)n, sizeof(double));
    double cnt[ORC_MAX_POP] = {0};
    memcpy(u, u0, sizeof(double) * (size_t)n);
    for (int64_t t = 0; t < n_steps; ++t) {
        for (int64_t i = 0; i < n; ++i) {
            int p = pop_of(net->pop_start, net->n_pop, i);
            double x = ring[(t % D) * n + i];
            ring[(t % D) * n + i] = 0.0;
            if (c->input_mode == 0 && lam[p] > 0.0)
                x += (lam[p] + sqrt(lam[p]) * z[t * n + i]) * c->w_ext;
            double v = pd[0] * u[i] + pd[1] * I[i];
            if (c->input_mode == 1) v += pd[3] * c->i_dc[p];
            I[i] = pd[2] * I[i] + x;
            double si = logistic10(v - c->theta);
            if (u_tr) u_tr[t * n + i] = v;
            if (s_tr) s_tr[t * n + i] = si;
            s[i] = si;
            u[i] = v * (1.0 - si);
            cnt[p] += si;
        }
        for (int64_t j = 0; j < n; ++j) {
            int q = pop_of(net->pop_start, net->n_pop, j);
            for (int64_t e = net->row_ptr[j]; e < net->row_ptr[j + 1]; ++e) {
                int64_t i = net->tgt[e];
                int p = pop_of(net->pop_start, net->n_pop, i);
                int idx = (p * ORC_MAX_POP + q) * ORC_WCODES + net->wcode[e];
                ring[((t + net->delay[e]) % D) * n + i] += s[j] * c->proj_scale[p][q] * wb[idx];
            }
        }
    }
    double T = (double)n_steps * c->dt / 1000.0;
    for (int p = 0; p < ORC_MAX_POP; ++p)
        rates[p] = (p < c->n_pop && c->pop_size[p] > 0) ? cnt[p] / ((double)c->pop_size[p] * T) : 0.0;
    free(wb); free(u); free(I); free(s); free(ring);
    return 0;
}

/* Smooth model around a recorded hard trajectory (u*, s*, m*, k*) of the
 * network net0 at parameters c0, written as deviations from that trajectory:
 *   du_t = m*_t (P22 dubar_{t-1} + P21 dI_{t-1}),  dubar_t = du_t (1 - s*_t)
 *   dI_t = P11 dI_{t-1} + dx_t
 *   s_t  = s*_t + F(u*_t + du_t - theta) - F(u*_t - theta),  F(x) = x/(1+10|x|)
 *   dx_t = sum over rows of  (s - s*)_{j,t-d} W_c + s*_{j,t-d} (alpha - alpha0) w_base
 *          + (nu - nu0) K_ext dt w_ext,        W = wtab0/256 + (alpha - alpha0) w_base
 * At (alpha0, nu0) every deviation is zero, so the model is the recorded hard
 * run; its exact derivative there is the surrogate gradient of mode 0.
 * u0 is unused (the deviations start at zero); kept for a uniform signature. */
int orc_surrogate_forward(const orc_net* net0, const orc_config* c0, const double* alpha,
                          double nu, int64_t n_steps, const double* u0, const float* u_star,
                          const uint8_t* f_star, const int32_t* k_star, double* rates)
{
    (void)u0;
    (void)k_star;
    const int64_t n = net0->n;
    const int D = c0->ring_depth;
    double pd[4];
    float pf[4];
    orc_propagators(c0, pd, pf);
    const double P22 = pf[0], P21 = pf[1], P11 = pf[2];
    const double theta = (double)(float)c0->theta;
    double* wb = (double*)malloc(sizeof(double) * ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES);
    double* w = (double*)malloc(sizeof(double) * ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES);
    double* dw = (double*)malloc(sizeof(double) * ORC_MAX_POP * ORC_MAX_POP * ORC_WCODES);
    base_table(c0, wb);
    for (int p = 0; p < ORC_MAX_POP; ++p)
        for (int q = 0; q < ORC_MAX_POP; ++q)
            for (int k = 0; k < ORC_WCODES; ++k) {
                int idx = (p * ORC_MAX_POP + q) * ORC_WCODES + k;
                dw[idx] = (alpha[p * ORC_MAX_POP + q] - c0->proj_scale[p][q]) * wb[idx];
                w[idx] = (double)net0->wtab[idx] / 256.0 + dw[idx];
            }
    const double dts = c0->dt / 1000.0;
    const double wq = (double)llround(c0->w_ext * 256.0) / 256.0;
    double* du = (double*)calloc((size_t)n, sizeof(double));
    double* dI = (double*)calloc((size_t)n, sizeof(double));
    double* ds = (double*)calloc((size_t)n, sizeof(double));
    double* ring = (double*)calloc((size_t)D * (size_t)n, sizeof(double));
    double cnt[ORC_MAX_POP] = {0};
    for (int64_t t = 0; t < n_steps; ++t) {
        for (int64_t i = 0; i < n; ++i) {
            int p = pop_of(net0->pop_start, net0->n_pop, i);
            double dx = ring[(t % D) * n + i];
            ring[(t % D) * n + i] = 0.0;
            if (c0->input_mode == 0) dx += (nu - c0->nu_bg) * c0->k_ext[p] * dts * wq;
            uint8_t f = f_star[t * n + i];
            double dv = (f & 2u) ? P22 * du[i] + P21 * dI[i] : 0.0;
            dI[i] = P11 * dI[i] + dx;
            double sstar = (double)(f & 1u);
            double us = (double)u_star[t * n + i] - theta;
            ds[i] = fast_sigmoid(us + dv) - fast_sigmoid(us);
            du[i] = dv * (1.0 - sstar);
            cnt[p] += sstar + ds[i];
        }
        for (int64_t j = 0; j < n; ++j) {
            double sstar = (double)(f_star[t * n + j] & 1u);
            if (ds[j] == 0.0 && sstar == 0.0) continue;
            int q = pop_of(net0->pop_start, net0->n_pop, j);
            for (int64_t e = net0->row_ptr[j]; e < net0->row_ptr[j + 1]; ++e) {
                int64_t i = net0->tgt[e];
                int p = pop_of(net0->pop_start, net0->n_pop, i);
                int idx = (p * ORC_MAX_POP + q) * ORC_WCODES + net0->wcode[e];
                ring[((t + net0->delay[e]) % D) * n + i] += ds[j] * w[idx] + sstar * dw[idx];
            }
        }
    }
    double T = (double)n_steps * c0->dt / 1000.0;
    for (int p = 0; p < ORC_MAX_POP; ++p)
        rates[p] = (p < c0->n_pop && c0->pop_size[p] > 0) ? cnt[p] / ((double)c0->pop_size[p] * T) : 0.0;
    free(wb); free(w); free(dw); free(du); free(dI); free(ds); free(ring);
    return 0;
}
