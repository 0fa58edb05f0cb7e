/*
 * snn.h -- C ABI of the GB300 library for the 0.1 ms time-stepped simulation
 * of the cortical microcircuit (Rhodes et al., "Real-Time Cortical Simulation
 * on Neuromorphic Hardware": Sec. 2.1 model and Eq. 1, Sec. 3.1.2 synaptic
 * matrix and ring buffers, Sec. 3.1.3 per-step processing).
 *
 * Conventions for every entry point
 *  - Return value: SNN_OK (0) or one of the SNN_ERR_* codes below; nothing
 *    is thrown across the ABI.  snn_last_error() returns a thread-local,
 *    human-readable message for the last failing call on this thread.
 *  - Pointers named *_host are host memory owned by the caller; they are read
 *    or written before the call returns.  The library owns every device
 *    allocation it makes and frees it in snn_destroy().
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Device work of a network is issued on that stream only.
 *  - The library needs an sm_103a GPU; on any other device snn_create()
 *    fails with SNN_ERR_UNSUPPORTED.  There is no CPU fallback.
 *
 * Model (Sec. 2.1, Eq. 1, read as tau_m du/dt = -u + R I, dI/dt = -I/tau_syn
 * + sum_j w_j delta(t - t_j), u = V - E_L), per step t and neuron i:
 *   1. acc = ring[t mod D][i]; ring[t mod D][i] = 0          (int32, 1/256 pA)
 *   2. Poisson background: acc += k w_ext, k ~ Poisson(nu_bg K_ext dt)
 *   3. if refr > 0: refr -= 1, u = 0; else u = P22 u + P21 I (+ P20 I_DC)
 *   4. I = P11 I + acc / 256                                  (fp32)
 *   5. if u > theta: spike, u = 0, refr = n_ref
 *   6. each spike of neuron j adds wtab[pop(i)][pop(j)][code] to
 *      ring[(t + delay) mod D][i] for every synapse (i, delay, code) of row j.
 * Integer accumulation makes every result independent of summation order,
 * so spike rasters are bit-exact and reproducible.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNN_MAX_POP 8
#define SNN_WCODES 128          /* weight codes per projection */
#define SNN_RING_DEPTH 64       /* delay slots per neuron: delays 1..63 steps */
#define SNN_MAX_NEURONS 524288  /* 19-bit target index in a synaptic word */

enum {
    SNN_OK = 0,
    SNN_ERR_INVALID = 1,      /* bad argument or configuration */
    SNN_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    SNN_ERR_OOM = 3,          /* device allocation failed */
    SNN_ERR_TIMEOUT = 4,      /* a grid-barrier wait exceeded its time limit */
    SNN_ERR_OVERFLOW = 5,     /* spike raster capacity exceeded (spikes lost) */
    SNN_ERR_UNSUPPORTED = 6,  /* device is not sm_103 or too small */
    SNN_ERR_SATURATED = 7     /* a neuron's fixed-point input of one step left the
                                 int32 range (see snn_sync) */
};

/*
 * Network and model parameters.  Field for field the same quantities the
 * paper's use case defines (Sec. 2.1): population sizes, connection
 * probabilities p[target][source], normally distributed weights (pA) and
 * delays (ms), Poisson background (K_ext x nu_bg, Sec. 3.1.3) or DC input,
 * and the neuron constants of Eq. 1.
 */
typedef struct snn_config {
    int32_t n_pop;                               /* 1..8 populations */
    int32_t pop_size[SNN_MAX_POP];               /* neurons per population */
    int32_t pop_exc[SNN_MAX_POP];                /* 1 excitatory, 0 inhibitory */
    double conn_prob[SNN_MAX_POP][SNN_MAX_POP];  /* [target][source] */
    double conn_scale;                           /* multiplies every probability */
    double w_mean[SNN_MAX_POP][SNN_MAX_POP];     /* pA, signed, [target][source] */
    double w_sd[SNN_MAX_POP][SNN_MAX_POP];       /* pA */
    double w_scale;                              /* multiplies every weight */
    double proj_scale[SNN_MAX_POP][SNN_MAX_POP]; /* per-projection weight factor */
    double d_mean[SNN_MAX_POP];                  /* ms, by source population */
    double d_sd[SNN_MAX_POP];                    /* ms */
    double k_ext[SNN_MAX_POP];                   /* background in-degree */
    double nu_bg;                                /* Hz, background rate */
    double w_ext;                                /* pA, background weight */
    double i_dc[SNN_MAX_POP];                    /* pA, DC input (input_mode 1) */
    int32_t input_mode;                          /* 0 Poisson, 1 DC */
    double tau_m, c_m, tau_syn, t_ref, theta, dt;/* ms, pF, ms, ms, mV, ms */
    double u0_lo, u0_hi;                         /* default initial u range, mV */
    int32_t ring_depth;                          /* must be SNN_RING_DEPTH */
} snn_config;

/* Execution options; a NULL pointer means all defaults. */
typedef struct snn_options {
    int32_t n_part;           /* partitions (= CTAs of the step kernel); 0 auto */
    int32_t inject_fault;     /* 0 normally.  1: partition 0 withholds its
                                 grid-barrier arrivals, so the other waits run
                                 out after timeout_s and snn_sync() returns
                                 SNN_ERR_TIMEOUT (tests of the failure path;
                                 every wait is bounded, nothing hangs) */
    int64_t raster_capacity;  /* spikes buffered on the device; 0 auto (64 Mi) */
    double timeout_s;         /* limit of one grid-barrier wait; 0 = 2 s */
} snn_options;

typedef struct snn_info {
    int64_t n_neurons;
    int64_t n_synapses;
    int32_t n_part;           /* partitions of the neuron range */
    int32_t threads;          /* threads per CTA of the step kernel */
    int32_t neurons_per_thread;
    int32_t ring_in_shared;   /* 1: ring buffers live in shared memory */
    int32_t max_part_neurons; /* largest partition */
    int32_t n_ref;            /* refractory steps */
    float propagators[4];     /* P22, P21, P11, P20 as used (fp32) */
    int32_t wext_q;           /* background weight, 1/256 pA */
    int32_t shared_bytes;     /* dynamic shared memory of the step kernel */
    int32_t slot_entries;     /* longest run of one row onto one partition (synapses) */
    int64_t slot_bytes;       /* device memory of the rows the step kernel reads
                                 (pre-decoded, 4 bytes per synapse) */
    int32_t deliver_clusters_active; /* co-resident 8-CTA clusters of snn_deliver
                                        tiling 4 (0: not available) */
    int32_t saturation_check; /* 1: the input bound below reaches the int32 range, so
                                 the step kernel counts wrap-arounds (SNN_ERR_SATURATED) */
    int64_t input_bound;      /* largest possible |input| of one neuron in one step,
                                 1/256 pA: sum over its synapses of the largest |weight|
                                 of each projection, plus the largest background count
                                 (32) times |w_ext| */
} snn_info;

typedef struct snn_net snn_net;

/*
 * snn_create -- build the network from `seed` on the device and set the
 * initial state (Sec. 2.1: probabilistic connectivity, normal weights and
 * delays; Sec. 4.1: initial conditions).
 *   cfg      host, read only.
 *   seed     Philox4x32-10 key for connectivity, weights, delays, background
 *            and the default initial potentials.
 *   opt      host or NULL.
 *   u0_host  host, n_neurons floats (mV above rest) or NULL for the default
 *            uniform draw on [u0_lo, u0_hi).
 *   stream   cudaStream_t of all later work of this network.
 *   out      receives the handle.
 * Errors: SNN_ERR_INVALID (config), SNN_ERR_UNSUPPORTED (device),
 * SNN_ERR_OOM, SNN_ERR_CUDA.  Blocks until the network is built.
 */
int snn_create(const snn_config* cfg, uint64_t seed, const snn_options* opt,
               const float* u0_host, void* stream, snn_net** out);

/*
 * snn_create_from_rows -- like snn_create, but with a caller-given synaptic
 * matrix (Sec. 3.1.2: one row per presynaptic neuron) instead of a generated
 * one.  Rows: row_ptr_host[n+1] (uint64 offsets), words_host[nnz] packed as
 * target (bits 0..18) | delay in steps (bits 19..24, 1..63) | weight code
 * (bits 25..31); targets ascending within a row.  wtab_host[8*8*128] int32
 * weights in 1/256 pA, index (target_pop*8 + source_pop)*128 + code.
 */
int snn_create_from_rows(const snn_config* cfg, uint64_t seed, const snn_options* opt,
                         const uint64_t* row_ptr_host, const uint32_t* words_host,
                         const int32_t* wtab_host, const float* u0_host, void* stream,
                         snn_net** out);

/*
 * snn_step -- advance the simulation by n_steps time steps of dt (Sec. 3.1.3:
 * every step updates all neurons, then delivers all spikes).  Asynchronous on
 * the network's stream; n_steps >= 0.  Spikes are appended to the device
 * raster.  Errors found on the device are reported by snn_sync().
 */
int snn_step(snn_net* net, int64_t n_steps);

/* snn_record_step_times -- from the next snn_step on, the step kernel
 * writes the device clock (ns, %globaltimer) at the end of every step t into
 * times_dev[t - t_first], t_first = the step count at this call, for at most
 * cap steps.  times_dev is caller-owned device memory (int64[cap]); NULL
 * stops recording.  Consecutive differences are the wall time of each step:
 * the paper's real-time criterion is every 0.1 ms step within 0.1 ms
 * (Sec. 3.1.3, Sec. 4.1).  The first step of a launch also carries the
 * launch gap. */
int snn_record_step_times(snn_net* net, int64_t* times_dev, int64_t cap);

/* snn_set_realtime -- pace snn_step to wall-clock time, the paper's "true
 * real time" (Sec. 4.1: every 0.1 ms step evaluated in 0.1 ms of wall time;
 * on SpiNNaker a 0.1 ms timer interrupt starts each step, Sec. 3.1.3).  From
 * the next snn_step on, step t starts no earlier than
 * anchor + (t - t_a) * period_ns, where t_a is the step count at this call
 * and anchor is the device clock (%globaltimer) when step t_a starts.  The
 * schedule is continuous across snn_step calls: a caller that pauses falls
 * behind it, and the late steps then run unpaced and count as missed until
 * the schedule is caught up.  A step that ends after its start time plus
 * period_ns has missed its deadline (measured at the end of the step by CTA
 * 0); snn_realtime_stats reads the count and the largest lateness.  Each
 * call resets the statistics and re-anchors; period_ns = 0 turns pacing
 * off.  period_ns in [0, 1e9], else SNN_ERR_INVALID.  Pacing changes no
 * result: rasters and state are those of an unpaced run.  Waits are bounded.
 * Only snn_step is paced (not the gradient or batch entry points). */
int snn_set_realtime(snn_net* net, int64_t period_ns);

/* snn_realtime_stats -- deadlines missed since the last snn_set_realtime,
 * and the largest lateness in ns (both 0 when pacing was never enabled).
 * Synchronises the network's stream. */
int snn_realtime_stats(snn_net* net, int64_t* missed, int64_t* max_late_ns);

/* snn_record_step_counts -- from the next snn_step on, the step kernel
 * writes one record of 4 uint32 per step t into counts_dev[4 (t - t_first)],
 * t_first = the step count at this call, for at most cap steps (the profile
 * the paper records per synapse core, Sec. 4.1, Fig. 7):
 *   [0] spikes emitted in step t;
 *   [1] synaptic events of those spikes (the sum of their row lengths);
 *   [2] the largest number of those spikes that one partition had to process
 *       (spikes with at least one synapse onto it): the busiest partition's
 *       load, the analogue of the paper's per-synapse-core count;
 *   [3] (spike, partition) pairs whose row has no synapse onto the partition:
 *       the paper's spike packets that target no neuron of a core.
 * Nothing is flushed here (every spike is delivered), so the paper's flushed
 * count is always 0 and is not recorded.  counts_dev is caller-owned device
 * memory (uint32[4 cap]); this call zeroes it on the network's stream.  NULL
 * stops recording.  Recording changes no result. */
int snn_record_step_counts(snn_net* net, uint32_t* counts_dev, int64_t cap);

/* snn_sync -- wait for the stream; returns SNN_OK, SNN_ERR_TIMEOUT if a
 * barrier wait gave up (state undefined), SNN_ERR_OVERFLOW if the raster
 * overflowed, SNN_ERR_SATURATED if some neuron's input of one step (its
 * ring-buffer slot plus background, Sec. 3.1.2) left the int32 fixed-point
 * range since the network was created, or SNN_ERR_CUDA.  Saturation is exact,
 * not a bound: the step kernel counts every int32 wrap-around of a ring cell
 * (it does so only for networks whose input bound, snn_info.input_bound,
 * reaches 2^31; others cannot saturate and pay nothing), and the simulation
 * goes on with the input wrapped modulo 2^32, as the CPU reference does.  The
 * status is sticky.  Stand-alone delivery (snn_deliver) does not count
 * wrap-arounds.  The state saved by snn_save_state does not carry pending
 * wrap counts. */
int snn_sync(snn_net* net);

/*
 * snn_read_spikes -- drain the recorded spikes (Sec. 3.1.2: output spike
 * times of all neurons are recorded) into steps_host[cap], ids_host[cap];
 * *n receives the count copied.  Order is unspecified (sort if needed).
 * Synchronises the stream.  SNN_ERR_OVERFLOW if spikes were lost on the
 * device or cap is too small (the first cap are returned).
 */
int snn_read_spikes(snn_net* net, uint32_t* steps_host, uint32_t* ids_host, int64_t cap,
                    int64_t* n);

/* snn_raster_size -- number of recorded spikes waiting to be read (the
 * capacity snn_read_spikes needs); synchronises the stream. */
int snn_raster_size(snn_net* net, int64_t* n);

/* snn_read_state -- copy u (mV), I_syn (pA) and refractory counters of all
 * neurons into host arrays of n_neurons elements; any pointer may be NULL. */
int snn_read_state(snn_net* net, float* u_host, float* i_syn_host, int32_t* refr_host);

/* snn_read_ring -- copy the ring buffers into ring_host[64 * n_neurons],
 * slot-major ([slot][neuron], slot = step mod 64), int32 in 1/256 pA. */
int snn_read_ring(snn_net* net, int32_t* ring_host);

/* snn_counters -- steps simulated, spikes emitted and synaptic events
 * delivered (one spike reaching one synapse, Sec. 3.3), since creation. */
int snn_counters(snn_net* net, int64_t* step, uint64_t* spikes, uint64_t* events);

/* snn_get_info -- sizes and launch configuration. */
int snn_get_info(snn_net* net, snn_info* info);

/* snn_export_network -- copy the synaptic matrix: row_ptr_host[n+1],
 * words_host[n_synapses] (format of snn_create_from_rows; ascending targets),
 * wtab_host[8*8*128].  Any pointer may be NULL. */
int snn_export_network(snn_net* net, uint64_t* row_ptr_host, uint32_t* words_host,
                       int32_t* wtab_host);

/*
 * snn_deliver -- deliver one arbitrary spike list into the ring buffers, as
 * step 6 does for the spikes of step t (Sec. 3.1.2: row fetch, word decode,
 * buffer add).  spikes_dev: device array of n_spikes neuron ids (duplicates
 * allowed).  tiling 0: one warp per spike; 1: one CTA per spike row; 2: one
 * CTA per partition, through the step kernel's delivery (each spike's run of
 * the pre-decoded rows onto the partition; the ring slice in shared memory
 * when it fits); 3: one CTA per partition reading exactly its run of each
 * row (the pre-decoded entries between the partition offsets: 4 bytes per
 * synapse, weight-table index and ring-cell offset, built with the network),
 * with the weights and, when they fit, the sums of the ring slots the list
 * can reach (t + 1 .. t + the longest delay) in shared memory, added into the
 * ring at the end (else straight into the ring in global memory);
 * 4: clusters of 8 CTAs,
 * one partition's ring slice in each CTA's shared memory, every row read once
 * per cluster and added through distributed shared memory
 * (SNN_ERR_UNSUPPORTED when a ring slice and the weight table do not fit);
 * 5: one CTA per partition reading the same runs as tiling 3, streamed into
 * shared memory by bulk copies (one producer warp, mbarrier-completed stages)
 * and added by the other warps (SNN_ERR_UNSUPPORTED when the ring slice and
 * the stages do not fit in shared memory).  A wait of tiling 5 that runs out
 * makes snn_sync report SNN_ERR_TIMEOUT.  Spike ids must be below n_neurons.
 * Asynchronous on the network's stream; adds to the existing ring content.
 */
int snn_deliver(snn_net* net, const uint32_t* spikes_dev, int32_t n_spikes, int64_t t,
                int32_t tiling);

/*
 * snn_step_noalloc -- advance a network held entirely in caller-owned device
 * memory by n_steps, allocating nothing.  The paper has no counterpart; it
 * exists for callers that may not allocate device memory while they run: an
 * application that steps the network in a closed real-time loop and has
 * reserved all of its device memory up front cannot call cudaMalloc or
 * cudaFree (they may synchronise the device and take unbounded time).
 *
 * The kernel's scratch (two spike lists and the barrier words) is a static
 * device array of 64 + 2 * SNN_NOALLOC_MAX_NEURONS 32-bit words (about 1 MiB)
 * that every GPU loading this library holds until the process exits.
 * Networks above SNN_NOALLOC_MAX_NEURONS neurons are rejected with
 * SNN_ERR_INVALID.  The first call on a device does that device's set-up,
 * with that device current: it looks up the array's device address
 * (cudaGetSymbolAddress) and queries the device's architecture, SM count and
 * the kernel's occupancy, and keeps them for the life of the process; make
 * that first call before any stream capture.  Do not use this entry point on
 * a device after cudaDeviceReset() of that device in the same process: the
 * kept address may no longer be the array's.  Every call shares the one array and
 * clears the words that must start at zero, so calls whose kernels overlap
 * on the GPU (on different streams, or from several threads) race and give
 * wrong results: serialise them.
 *
 *   cfg, seed  model parameters and Philox key, as for snn_create; the
 *              network's row_ptr / words / wtab must be the ones exported
 *              by snn_export_network for the same cfg (any rows in that
 *              format are accepted).
 *   io         device pointers, all required:
 *                row_ptr[n+1] (uint64), words[nnz], wtab[8*8*128]   input
 *                u[n], i_syn[n], refr[n], ring[64*n] slot-major     in/out
 *                ras_step[ras_cap], ras_id[ras_cap]                 output
 *                ras_n: spikes recorded; the kernel appends at *ras_n
 *                  and counts past ras_cap (caller zeroes it)     in/out
 *                counters[2]: spikes and synaptic events, added to  in/out
 *                status: ORed with 1 if a grid-barrier wait gave up in/out
 *   t0         index of the first step (it selects the ring slots and the
 *              background draws, so consecutive calls continue a run).
 * Asynchronous on `stream`.  Results equal snn_step on the same network.
 * Inputs wrap modulo 2^32 like snn_step's, but this entry point does not
 * check for saturation (it never sets SNN_ERR_SATURATED).
 */
#define SNN_NOALLOC_MAX_NEURONS 131072

typedef struct snn_noalloc_io {
    const uint64_t* row_ptr;
    const uint32_t* words;
    const int32_t* wtab;
    float* u;
    float* i_syn;
    int32_t* refr;
    int32_t* ring;
    uint32_t* ras_step;
    uint32_t* ras_id;
    uint32_t* ras_n;
    int64_t ras_cap;
    unsigned long long* counters;
    uint32_t* status;
} snn_noalloc_io;

int snn_step_noalloc(const snn_config* cfg, uint64_t seed, const snn_noalloc_io* io,
                     int64_t t0, int64_t n_steps, void* stream);

/*
 * ---------------------------------------------------------------------------
 * State, parameters and gradient.
 * ---------------------------------------------------------------------------
 */

/* snn_save_state -- serialise the dynamic state (u, I, refractory counters,
 * ring buffers and the step counter; Sec. 3.1.2 ring buffers) into a host
 * buffer: 32-byte header, then u[n] f32, I[n] f32, refr[n] i32 and
 * ring[64][n] i32.  With buf_host == NULL only *n_bytes is set.  Synchronises.
 * Errors: SNN_ERR_INVALID (cap smaller than *n_bytes). */
int snn_save_state(snn_net* net, void* buf_host, int64_t cap, int64_t* n_bytes);

/* snn_load_state -- restore a state saved from a network of the same size;
 * later steps continue from it exactly (bit for bit).  Synchronises. */
int snn_load_state(snn_net* net, const void* buf_host, int64_t n_bytes);

/* snn_set_params -- set the 64 projection weight scales alpha[p*8 + q]
 * (target p, source q; they multiply every weight of the projection before
 * its fixed-point rounding) and the background rate nu_bg (Hz).  The
 * connectivity, delays and weight codes are unchanged.  Synchronises.
 * Errors: SNN_ERR_INVALID (non-finite scale, negative rate, weight outside
 * the fixed-point range). */
int snn_set_params(snn_net* net, const double* scales, double nu_bg);

/*
 * snn_grad_forward -- run n_steps from the current state as snn_step does,
 * recording the trajectory when it fits the trace budget (see
 * snn_grad_set_trace_budget), else keeping a device checkpoint of the full
 * state every ckpt_every steps, and return the population rates (Hz) over
 * those steps in rates_host[8].
 * snn_grad_backward -- given g_rate[8] = dL/d rate_p of any loss of those
 * rates, return dL/d alpha (g_alpha[p*8 + q]) and dL/d nu_bg (*g_nu) by
 * backpropagation through time: each segment's trajectory (recorded by the
 * forward when it fits the trace budget, see snn_grad_set_trace_budget, else
 * recomputed from the segment's checkpoint) is differentiated in reverse.  Spike derivative: the fast-sigmoid surrogate 1/(1+10|u-theta|)^2
 * per mV; reset and refractory are held fixed; the weight rounding and the
 * Poisson count pass their derivative straight through (d w/d alpha = the
 * unrounded base weight, d k/d nu = K_ext dt).  fp32 adjoint state, double
 * accumulation, deterministic.  The paper has no gradient: this is the
 * differentiable form of its network (Sec. 2.1, Eq. 1).  The backward leaves
 * the state, counters and raster as they were after the forward.
 * Errors: SNN_ERR_INVALID (no forward, or the network was stepped since),
 * SNN_ERR_OOM, SNN_ERR_TIMEOUT.
 */
int snn_grad_forward(snn_net* net, int64_t n_steps, int32_t ckpt_every, double* rates_host);
int snn_grad_backward(snn_net* net, const double* g_rate, double* g_alpha, double* g_nu);

/*
 * snn_grad_set_trace_budget -- largest trajectory of a whole snn_grad_forward
 * kept on the device, in bytes (5 per neuron-step: u and the spike/update
 * flags; default 4 GiB, and never more than a quarter of the free device
 * memory at the forward).  A forward whose trajectory fits records it as it
 * runs, and the backward then re-runs nothing; otherwise the backward re-runs
 * each checkpoint segment to record it.  0 always re-runs.  The gradient is
 * the same bit for bit either way.  Applies from the next forward.
 * Errors: SNN_ERR_INVALID (null net, negative bytes).
 */
int snn_grad_set_trace_budget(snn_net* net, int64_t bytes);

/*
 * ---------------------------------------------------------------------------
 * Batched instances.  The paper simulates one network at a time; a batch runs
 * many independent networks of the same model (Sec. 2.1, Eq. 1) -- each with
 * its own configuration (e.g. its own scale) and seed -- in ONE persistent
 * cooperative kernel.  Neurons of all instances are concatenated; every step
 * is a neuron pass over all of them, a grid barrier, delivery of every spike
 * of the step through its own instance's rows, and a second barrier.  Every
 * instance's raster, state and counters equal those of snn_create/snn_step
 * with the same configuration and seed (default initial state), bit for bit.
 *
 * Delivery tiling per instance: at creation an autotuner times, on each
 * instance's own rows and a spike list of the size its activity gives (about
 * 5 Hz x N x 0.1 ms), one warp per spike (tiling 0), one CTA per row
 * (tiling 1) and flat (tiling 2: the rows of all flat-tiled spikes of a step
 * concatenated and spread over every warp of the grid), and keeps the
 * fastest.  Because all instances' spikes share the grid in the batch, it
 * then times the persistent kernel itself (100 + 300 steps) under candidate
 * assignments -- the probes' choices, each tiling for every instance, and the
 * smaller and larger half of the instances on two different tilings -- keeps
 * the fastest, and resets every instance to its initial state.
 * snn_batch_get_info reports the probe times and the chosen per-step time.
 *
 * Steps are issued as replays of one captured CUDA graph of 1000 steps; the
 * kernel reads its first step index from device memory and advances it, so
 * replays need no parameter update.  Remainders (n_steps mod 1000) use a
 * plain launch.
 * ---------------------------------------------------------------------------
 */
typedef struct snn_batch snn_batch;

typedef struct snn_batch_info {
    int32_t n_instances;
    int32_t n_neurons_total;     /* concatenated neurons of all instances */
    int32_t n_neurons;           /* of the queried instance */
    int64_t n_synapses;          /* of the queried instance */
    int32_t tiling;              /* 0 warp per spike, 1 CTA per row, 2 flat */
    float tune_us_warp;          /* autotuner probe times, microseconds */
    float tune_us_block;
    float tune_us_flat;
    float trial_us_per_step;     /* the chosen assignment's time per step in the
                                    autotuner's batch trials */
    int32_t blocks, threads, neurons_per_thread;
    int32_t graph;               /* 1 if the graph was captured */
    int32_t graph_steps;         /* steps per graph replay */
} snn_batch_info;

/*
 * snn_batch_create -- build n_inst networks and the batch launch.
 *   cfgs[n_inst], seeds[n_inst]   host arrays, read during the call
 *   opt                           may be NULL; raster_capacity is the total
 *                                 raster capacity of the batch (default
 *                                 64 Mi spikes), timeout_s the barrier limit,
 *                                 inject_fault = 1 makes CTA 0 skip its
 *                                 barrier arrivals (tests the bounded wait:
 *                                 snn_batch_sync then reports
 *                                 SNN_ERR_TIMEOUT); n_part is ignored
 *   stream                        cudaStream_t of all the batch's work
 * Errors: SNN_ERR_INVALID (n_inst outside 1..1024, bad configuration),
 * SNN_ERR_OOM, SNN_ERR_UNSUPPORTED (not sm_103, or too many neurons for one
 * co-resident grid), SNN_ERR_SATURATED (an instance whose input of one step
 * can leave the int32 range, snn_info.input_bound >= 2^31: the batch kernel
 * has no wrap-around count, so such an instance is refused).
 */
int snn_batch_create(const snn_config* cfgs, const uint64_t* seeds, int32_t n_inst,
                     const snn_options* opt, void* stream, snn_batch** out);

/* snn_batch_step -- advance every instance by n_steps (async on the stream). */
int snn_batch_step(snn_batch* b, int64_t n_steps);

/* snn_batch_sync -- wait; SNN_ERR_TIMEOUT if a barrier wait gave up,
 * SNN_ERR_OVERFLOW if the batch raster ran out of capacity. */
int snn_batch_sync(snn_batch* b);

/* snn_batch_read_spikes -- drain the spikes of instance k recorded since the
 * last read of that instance: (step, local neuron id) in device order (not
 * sorted).  Synchronises.  n receives the number written (<= cap). */
int snn_batch_read_spikes(snn_batch* b, int32_t k, uint32_t* steps_host, uint32_t* ids_host,
                          int64_t cap, int64_t* n);

/* snn_batch_read_state -- u, I (fp32) and refractory counters of instance k,
 * n_neurons entries each; any pointer may be NULL.  Synchronises. */
int snn_batch_read_state(snn_batch* b, int32_t k, float* u_host, float* i_syn_host,
                         int32_t* refr_host);

/* snn_batch_counters -- steps taken, spikes and synaptic events of instance k. */
int snn_batch_counters(snn_batch* b, int32_t k, int64_t* step, uint64_t* spikes,
                       uint64_t* events);

int snn_batch_get_info(snn_batch* b, int32_t k, snn_batch_info* info);

/* snn_batch_set_tiling -- override the autotuner's delivery tiling of
 * instance k (0 one warp per spike, 1 one CTA per row, 2 flat) for the steps issued
 * after the call.  Results do not depend on the tiling.  Synchronises. */
int snn_batch_set_tiling(snn_batch* b, int32_t k, int32_t tiling);

/* snn_batch_destroy -- free all device memory of the batch (synchronises). */
int snn_batch_destroy(snn_batch* b);

/* snn_destroy -- free all device memory of the network (synchronises). */
int snn_destroy(snn_net* net);

const char* snn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
