/*
 * oracle.h -- plain CPU reference of the time-stepped LIF microcircuit.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The CUDA product path never calls
 * it, and it shares no code, header or table generator with that path.
 *
 * Parity status of each function is stated in oracle.c beside the function.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#define ORC_MAX_POP 8
#define ORC_POIS_TABLE 32
#define ORC_WCODES 128
#define ORC_DCODES 256

typedef struct orc_config {
    int32_t n_pop;
    int32_t pop_size[ORC_MAX_POP];
    int32_t pop_exc[ORC_MAX_POP];
    double conn_prob[ORC_MAX_POP][ORC_MAX_POP];   /* [target p][source q] */
    double conn_scale;
    double w_mean[ORC_MAX_POP][ORC_MAX_POP];      /* pA, [p][q], signed */
    double w_sd[ORC_MAX_POP][ORC_MAX_POP];        /* pA */
    double w_scale;
    double proj_scale[ORC_MAX_POP][ORC_MAX_POP];  /* per-projection factor */
    double d_mean[ORC_MAX_POP];                   /* ms, by source pop */
    double d_sd[ORC_MAX_POP];                     /* ms */
    double k_ext[ORC_MAX_POP];
    double nu_bg;                                 /* Hz */
    double w_ext;                                 /* pA */
    double i_dc[ORC_MAX_POP];                     /* pA */
    int32_t input_mode;                           /* 0 Poisson, 1 DC */
    double tau_m, c_m, tau_syn, t_ref, theta, dt; /* ms, pF, ms, ms, mV, ms */
    double u0_lo, u0_hi;                          /* mV */
    int32_t ring_depth;
} orc_config;

typedef struct orc_net orc_net;
typedef struct orc_sim orc_sim;

/* primitives (exposed for pins) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_norm_quantile(double p);
void orc_propagators(const orc_config* c, double out_d[4], float out_f[4]);
void orc_poisson_thresholds(double lam, uint64_t thr[ORC_POIS_TABLE]);
int orc_poisson_count(uint32_t x, const uint64_t thr[ORC_POIS_TABLE]);
int orc_tables(const orc_config* c, int32_t* wtab, uint8_t* dtab, uint64_t* pois,
               uint64_t* conn_thr, int32_t* wext_q, int32_t* n_ref);
void orc_poisson_draws(uint64_t seed, int64_t neuron, int64_t t0, int64_t n,
                       const uint64_t thr[ORC_POIS_TABLE], int32_t* counts);

/* network */
orc_net* orc_net_generate(const orc_config* c, uint64_t seed, int n_threads);
orc_net* orc_net_custom(const orc_config* c, const int64_t* row_ptr, const int32_t* tgt,
                        const uint8_t* delay, const uint8_t* wcode, const int32_t* wtab);
int64_t orc_net_neurons(const orc_net* n);
int64_t orc_net_synapses(const orc_net* n);
void orc_net_export(const orc_net* n, int64_t* row_ptr, int32_t* tgt, uint8_t* delay,
                    uint8_t* wcode);
int64_t orc_net_row(const orc_config* c, uint64_t seed, int64_t j, int32_t* tgt,
                    uint8_t* delay, uint8_t* wcode, int64_t cap);
void orc_net_free(orc_net* n);
void orc_deliver(const orc_net* net, const orc_config* c, const int32_t* spikes, int64_t n_spikes,
                 int64_t t, int64_t* ring);

/* simulation */
orc_sim* orc_sim_create(const orc_net* net, const orc_config* c, uint64_t seed,
                        const float* u0);
int64_t orc_sim_run(orc_sim* s, int64_t n_steps);
int64_t orc_sim_raster_count(const orc_sim* s);
void orc_sim_raster_read(orc_sim* s, int64_t* steps, int32_t* ids);
void orc_sim_state(const orc_sim* s, float* u, float* i_syn, int32_t* refr, int64_t* ring);
void orc_sim_set_state(orc_sim* s, const float* u, const float* i_syn, const int32_t* refr,
                       const int64_t* ring, int64_t step);
void orc_sim_counters(const orc_sim* s, int64_t* step, int64_t* spikes, int64_t* events,
                      int32_t* saturated);
void orc_sim_free(orc_sim* s);
int64_t orc_sim_run_trace(orc_sim* s, int64_t n_steps, float* u_trace, uint8_t* flags,
                          int32_t* kbg);

/* gradient of a population-rate loss (hard model with surrogate, mode 0;
 * sigmoid-relaxed model, mode 1) and the two smooth forwards that pin it */
int orc_grad_backward(const orc_net* net, const orc_config* c, int mode, int64_t n_steps,
                      const double* u_tr, const double* s_tr, const uint8_t* m_tr,
                      const double* z, const double* g_rate, double* g_alpha, double* g_nu);
int orc_relaxed_forward(const orc_net* net, const orc_config* c, int64_t n_steps,
                        const double* u0, const double* z, double* u_tr, double* s_tr,
                        double* rates);
int orc_surrogate_forward(const orc_net* net0, const orc_config* c0, const double* alpha,
                          double nu, int64_t n_steps, const double* u0, const float* u_star,
                          const uint8_t* f_star, const int32_t* k_star, double* rates);

#endif
