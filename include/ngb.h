/*
 * ngb.h -- C ABI of the GB300 spiking-network simulator core.
 *
 * The library simulates networks of spiking point neurons on one GPU with the
 * method of Golosio et al., "Fast simulations of highly-connected spiking
 * cortical models using GPUs" (NeuronGPU, 2020):
 *   - LIF neurons with exponential post-synaptic currents (Eqs. 1-2), updated
 *     by exact integration on the dt grid (Sec. 2.1);
 *   - AdEx neurons with exponential conductance synapses (Eqs. 3-5), updated by
 *     an embedded fifth-order Runge-Kutta method with adaptive step size
 *     (Sec. 2.1);
 *   - Poisson generators as external drive (Sec. 2.1, devices);
 *   - connections by the fixed-indegree and fixed-total-number rules (Sec. 2.1)
 *     stored per source, grouped by delay (Sec. 2.2);
 *   - spike delivery: every spike of step t adds each outgoing synapse weight to
 *     the target's input of step t + delay (Sec. 2.2), either scattered at
 *     once into a ring of future inputs, or by the paper's spike buffer (a
 *     spike waits until its age reaches the delay of its next connection
 *     group, which is then scattered into the next step's input); both give
 *     the same sums.
 *
 * Conventions shared by every entry point:
 *   - Return value 0 (NGB_OK) on success, a negative NGB_ERR_* code on failure;
 *     ngb_last_error() then returns a message (thread-local, valid until the
 *     next call on the same thread).
 *   - All pointers in this header are HOST pointers; the library owns all
 *     device memory it allocates and frees it in ngb_destroy().  Output arrays
 *     are caller-owned and must hold the stated number of elements.
 *   - A handle is not thread-safe: use one handle per thread.
 *   - Units: ms, mV, pF, pA, nS, Hz.
 *   - A spike reported at step s crossed threshold during step s, i.e. in the
 *     interval [s*dt, (s+1)*dt); its time is (s+1)*dt.
 *   - Neuron ids are global (creation order over all populations) unless a call
 *     says population-local.
 */
#ifndef NGB_H
#define NGB_H

#include <stdint.h>

#if defined(__GNUC__)
#define NGB_API __attribute__((visibility("default")))
#else
#define NGB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- errors */
#define NGB_OK 0
#define NGB_ERR_INVALID_ARG (-1) /* an argument is out of range or inconsistent */
#define NGB_ERR_STATE (-2)       /* call not allowed now (e.g. connect after the first simulate) */
#define NGB_ERR_OOM (-3)         /* a device or host allocation failed */
#define NGB_ERR_CUDA (-4)        /* a CUDA call failed; the message names it */
#define NGB_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */
#define NGB_ERR_OVERFLOW (-6)    /* spike record full, delay beyond the ring, or RK sub-step cap hit */

/* ----------------------------------------------------------------- enums */
typedef enum { NGB_WEIGHT_FP32 = 0, NGB_WEIGHT_BF16 = 1, NGB_WEIGHT_FP16 = 2 } ngb_weight_dtype;
/* Neuron models: LIF with exponential PSCs (Eqs. 1-2); AdEx (Eqs. 3-5) with
 * exponential conductances; AdEx with alpha-function conductances (the
 * paper's balanced network, Sec. 2.4: an input of weight W gives
 * g(t) = W (t/tau) e^(1 - t/tau), peak W at t = tau); the multisynapse AdEx
 * of the paper's interface example (Sec. 2.1) with 1-4 receptor ports of
 * beta-function conductances: port k has reversal potential E_k, rise time
 * tau_r,k and decay time tau_d,k, g_k' = x_k - g_k / tau_d,k,
 * x_k' = -x_k / tau_r,k, and an input of weight W raises x_k by W g0_k with
 * g0_k set so that g_k peaks at W (the alpha function when tau_r = tau_d).
 * Beta populations run in the per-step kernel loops (graph, pipelined); a
 * handle holding one never uses the persistent or fused loop. */
typedef enum {
  NGB_LIF_PSC_EXP = 0,
  NGB_AEIF_COND_EXP = 1,
  NGB_AEIF_COND_ALPHA = 2,
  NGB_AEIF_COND_BETA = 3
} ngb_model;
typedef enum {
  NGB_RULE_FIXED_INDEGREE = 0,
  NGB_RULE_FIXED_TOTAL_NUMBER = 1,
  NGB_RULE_FIXED_OUTDEGREE = 2,
  NGB_RULE_ONE_TO_ONE = 3,
  NGB_RULE_ALL_TO_ALL = 4
} ngb_rule;
typedef enum { NGB_DIST_CONST = 0, NGB_DIST_NORMAL = 1, NGB_DIST_UNIFORM = 2 } ngb_dist;
/* Spike delivery scheme (results are the same; memory traffic differs):
 *   RING          every spike is scattered at once into ring slots t + delay
 *                 (L slots of N x receptors words);
 *   SPIKE_BUFFER  Sec. 2.2: a spike waits in a pending list until its age
 *                 equals the delay of its next connection group, which is
 *                 then scattered into the next step's input (one slot), so
 *                 the scattered-to array stays in L2 on large networks.
 *                 With it, at most (refractory steps + 1)-spaced spikes per
 *                 source can be in flight; an overflow is NGB_ERR_OVERFLOW.
 *   AUTO          spike buffer when the L-slot ring would exceed half of the
 *                 L2 cache, else ring; ngb_autotune at step 0 times both. */
typedef enum { NGB_DELIVERY_AUTO = 0, NGB_DELIVERY_RING = 1, NGB_DELIVERY_SPIKE_BUFFER = 2 } ngb_delivery;
typedef enum {
  NGB_VAR_V_M = 0,     /* membrane potential, mV (both models) */
  NGB_VAR_I_SYN = 1,   /* LIF: synaptic current, pA.  AdEx: adaptation current w, pA */
  NGB_VAR_G_EX = 2,    /* AdEx: excitatory conductance, nS */
  NGB_VAR_G_IN = 3,    /* AdEx: inhibitory conductance, nS */
  NGB_VAR_REFRACT = 4, /* LIF: refractory steps left */
  NGB_VAR_H = 5,       /* AdEx: carried Runge-Kutta step proposal, ms */
  NGB_VAR_DG_EX = 6,   /* AdEx alpha: x_ex with g_ex' = x_ex - g_ex / tau_ex, nS/ms (beta: x_0) */
  NGB_VAR_DG_IN = 7,   /* AdEx alpha: x_in, nS/ms (beta: x_1) */
  NGB_VAR_G_2 = 8,     /* AdEx beta: conductance of port 2, nS (ports 0, 1: G_EX, G_IN) */
  NGB_VAR_G_3 = 9,     /* AdEx beta: conductance of port 3, nS */
  NGB_VAR_X_2 = 10,    /* AdEx beta: x of port 2, nS/ms */
  NGB_VAR_X_3 = 11     /* AdEx beta: x of port 3, nS/ms */
} ngb_state_var;

/* ------------------------------------------------------------ structures */
/* Simulation-wide settings (ngb_create). */
typedef struct {
  double dt_ms;            /* time step, > 0 */
  uint64_t seed;           /* key of instance 0's random streams */
  int32_t weight_dtype;    /* ngb_weight_dtype: storage of synapse weights; accumulation is FP32 */
  int32_t device;          /* CUDA device ordinal */
  void* stream;            /* cudaStream_t to run on, or NULL for a library-owned stream */
  int32_t deterministic;   /* 1: accumulate inputs in 64-bit fixed point (2^-32 units), so the
                              result does not depend on the order of the atomic additions */
  int32_t record_spikes;   /* 1: keep every spike for ngb_get_spikes */
  int64_t record_capacity; /* device spike-record entries between drains; 0 = default */
  int32_t steps_per_graph; /* steps captured in one CUDA graph; 0 = default, <0 = no graph */
  int32_t drain_steps;     /* steps between spike-record drains; 0 = default */
  int32_t delivery;        /* ngb_delivery: 0 automatic, 1 ring, 2 spike buffer */
  int32_t pad_;
} ngb_sim_config;

/* External Poisson drive of a population (Sec. 2.1, Poisson generator device):
 * every neuron independently receives k ~ Poisson(n_inputs * rate_hz * dt)
 * input spikes per step, each of weight `weight` (pA for LIF, nS for AdEx),
 * on receptor `receptor` (AdEx: 0 excitatory, 1 inhibitory; beta: the port). */
typedef struct {
  double n_inputs;
  double rate_hz;
  double weight;
  int32_t receptor;
  int32_t pad_;
} ngb_poisson_drive;

/* LIF with exponential PSC (Eqs. 1-2).  Initial V ~ Normal(V_init_mean, V_init_sd). */
typedef struct {
  double tau_m_ms, C_m_pF, E_L_mV, V_reset_mV, V_th_mV, t_ref_ms, tau_syn_ms, I_e_pA;
  double V_init_mean_mV, V_init_sd_mV;
  ngb_poisson_drive poisson;
} ngb_lif_params;

/* AdEx (Eqs. 3-5), for the three conductance models.  NGB_AEIF_COND_EXP,
 * NGB_AEIF_COND_ALPHA: receptors 0 (E_ex, tau_ex) and 1 (E_in, tau_in), the
 * taus being the decay or alpha time constants.  NGB_AEIF_COND_BETA: ports
 * 0 .. n_ports-1 with E_rev_mV, tau_rise_ms, tau_decay_ms (E_ex, E_in,
 * tau_ex, tau_in are not used then; the other two models ignore the port
 * fields).  No refractory period.
 * rk_tol: relative tolerance of the adaptive Runge-Kutta step; with FP32 state
 * the effective tolerance is max(rk_tol, 8 * 2^-24).  The step size, the time
 * inside the step and the error-ratio test are FP64 unless rk_control_fp32 is
 * 1 (then FP32: faster on parts with few FP64 units, same state precision). */
typedef struct {
  double C_m_pF, g_L_nS, E_L_mV, V_T_mV, Delta_T_mV, a_nS, b_pA, tau_w_ms, V_peak_mV, V_reset_mV;
  double E_ex_mV, E_in_mV, tau_ex_ms, tau_in_ms, I_e_pA;
  double V_init_mean_mV, V_init_sd_mV, w_init_pA;
  double rk_tol, rk_h_min_ms, rk_h_init_ms;
  int64_t rk_max_substeps;
  int32_t rk_control_fp32;
  int32_t pad_;
  ngb_poisson_drive poisson;
  int32_t n_ports; /* NGB_AEIF_COND_BETA: 1..4 */
  int32_t pad2_;
  double E_rev_mV[4], tau_rise_ms[4], tau_decay_ms[4];
} ngb_aeif_params;

/* Connection rule (Sec. 2.1).  FIXED_INDEGREE: every target draws K sources
 * uniformly with replacement.  FIXED_TOTAL_NUMBER: K (source, target) pairs
 * drawn uniformly with replacement.  FIXED_OUTDEGREE: every source draws K
 * targets uniformly with replacement.  ONE_TO_ONE: source i -> target i
 * (equal sizes; K unused).  ALL_TO_ALL: every (source, target) pair once
 * (K unused).  Multapses are allowed; autapses only when allow_autapses is set
 * (and only matter when source == target pop; ONE_TO_ONE within one
 * population then needs them).  Draw index q numbers the synapses of a call:
 * target-major for FIXED_INDEGREE and ALL_TO_ALL, source-major for
 * FIXED_OUTDEGREE, the source for ONE_TO_ONE. */
typedef struct {
  int32_t rule;
  int32_t allow_autapses;
  int64_t K;
} ngb_conn_spec;

/* Distribution of a synapse parameter.  CONST: p0.  NORMAL(mean p0, sd p1):
 * for weights re-drawn until the sign equals the sign of the mean; for delays
 * re-drawn until >= dt.  UNIFORM on (p0, p1]. */
typedef struct {
  int32_t dist;
  int32_t pad_;
  double p0, p1;
} ngb_dist_spec;

/* Synapse parameters: weight (pA for LIF targets, nS for AdEx targets; an
 * inhibitory AdEx synapse has a positive weight on receptor 1), delay in ms
 * (rounded to the nearest step, ties to even, at least one step), receptor
 * (LIF 0; AdEx 0, 1; beta 0 .. n_ports-1). */
typedef struct {
  ngb_dist_spec weight;
  ngb_dist_spec delay_ms;
  int32_t receptor;
  int32_t pad_;
} ngb_syn_spec;

/* Nearest-neighbour STDP (Sec. 2.1, after Morrison et al. 2008) with the
 * power-law weight dependence of Guetig et al. (2003).  A spike reaches a
 * synapse `delay` steps after it was fired (its arrival).  At an arrival the
 * synapse is depressed by the target's latest spike at an earlier step (lag
 * n >= 1 steps): w -= alpha lambda W_max (w / W_max)^mu_minus e^(-n dt / tau_minus),
 * and delivers the depressed weight; at a spike of the target every plastic
 * input is potentiated by its latest arrival at or before that step (lag
 * n >= 0): w += lambda W_max (1 - w / W_max)^mu_plus e^(-n dt / tau_plus).
 * Each update is clipped to [0, W_max]; a lag beyond 20 tau changes nothing;
 * FP32 arithmetic with the exponentials tabulated per lag. */
typedef struct {
  double tau_plus_ms, tau_minus_ms; /* > 0 */
  double lambda, alpha;             /* learning rate, depression / potentiation ratio, >= 0 */
  double mu_plus, mu_minus;         /* weight exponents: 0 additive, 1 multiplicative, >= 0 */
  double W_max;                     /* weight bound, > 0 */
} ngb_stdp_params;

/* Counters accumulated since ngb_create. */
typedef struct {
  int64_t steps;        /* steps simulated */
  int64_t spikes;       /* spikes emitted (with multiplicity) */
  int64_t events;       /* synaptic events delivered (spikes x out-degree) */
  int64_t rk_substeps;  /* accepted + rejected Runge-Kutta sub-steps of all AdEx neurons */
  int64_t num_neurons;
  int64_t num_synapses;
  int64_t num_groups;   /* (source, delay) connection groups */
  int64_t ring_slots;   /* L, a power of two > max delay in steps */
  int64_t max_delay_steps;
  int64_t device_bytes; /* device memory held by the handle */
  int64_t mode;         /* step loop: 0 per-step kernels in CUDA graphs, 1 persistent step kernel, 2 fused
                           update + delivery, 3 pipelined (delivery of step t beside the update of t + 1),
                           4 pipelined persistent step kernel (one grid barrier per step), 5 pipelined
                           with one kernel per step (LIF networks), 6 target-owned persistent kernel
                           (LIF networks: one block per SM owns every G-th neuron, with the ring of its
                           neurons in shared memory; spikes exchanged through step-stamped mailboxes),
                           7 per-step kernels in CUDA graphs with target-tiled delivery (spike-buffer
                           scheme: the due groups' synapses, stored a second time partitioned by target
                           tile, are summed per tile in shared memory and each tile's input written once,
                           instead of one global atomic per synaptic event) */
  int64_t launch_grid;  /* blocks of the delivery kernel (modes 0, 3, 5, 7) or of the persistent kernel
                           (modes 1, 4, 6) */
  int64_t delivery;     /* delivery scheme in use: 1 ring, 2 spike buffer */
  int64_t hot_steps;    /* AdEx neuron steps run by the hot-list kernel (per-step kernels: a neuron whose
                           step ended above V_T + c Delta_T runs its next step, whole, in a warp of such
                           neurons beside the update kernel; c = 4, environment NGB_AEIF_HOT = c, 0 off;
                           the arithmetic of each step is the same either way) */
} ngb_stats;

typedef struct ngb_sim ngb_sim;

/* ------------------------------------------------------------ lifecycle */
/* Create an empty simulation on cfg->device.  *out receives the handle. */
NGB_API int ngb_create(ngb_sim** out, const ngb_sim_config* cfg);

/* Free every resource of the handle; NULL is a no-op. */
NGB_API int ngb_destroy(ngb_sim* sim);

/* Message of the last failed call on this thread ("" if none).  `sim` may be NULL. */
NGB_API const char* ngb_last_error(const ngb_sim* sim);

/* -------------------------------------------------------- construction */
/* Add a network instance with its own random key (batched execution: several
 * independent networks advance in the same kernels; instance 0 exists from
 * ngb_create with cfg->seed).  Random streams use instance-local neuron ids
 * and connect-call indices, so an instance's result does not depend on what
 * else is batched with it.  NGB_ERR_STATE after the first simulate. */
NGB_API int ngb_add_instance(ngb_sim* sim, uint64_t seed, int32_t* instance_out);

/* Add n neurons of `model` (params: ngb_lif_params* or ngb_aeif_params*) to
 * instance 0.  Population ids count from 0 over the whole handle. */
NGB_API int ngb_add_population(ngb_sim* sim, int32_t model, int64_t n, const void* params, int32_t* pop_id_out);

/* As ngb_add_population, into the given instance. */
NGB_API int ngb_add_population_in(ngb_sim* sim, int32_t instance, int32_t model, int64_t n, const void* params,
                          int32_t* pop_id_out);

/* Connect src_pop -> tgt_pop (same instance) with rule `conn` and synapse
 * parameters `syn` (Sec. 2.1).  Synapses are drawn on the device when the
 * network is finalised (first ngb_simulate or ngb_finalize). */
NGB_API int ngb_connect(ngb_sim* sim, int32_t src_pop, int32_t tgt_pop, const ngb_conn_spec* conn,
                const ngb_syn_spec* syn);

/* As ngb_connect, with plastic synapses (ngb_stdp_params; each call is its
 * own rule, at most 15 per handle).  Plastic synapses need FP32 weight
 * storage and the spike-buffer delivery scheme (NGB_DELIVERY_AUTO chooses
 * it; NGB_DELIVERY_RING is NGB_ERR_INVALID_ARG), run in the per-step kernel
 * loop, and are not available in serving handles (NGB_ERR_STATE).  Steps are
 * counted in 31 bits for them: simulating beyond step 2^31 - 1 is
 * NGB_ERR_OVERFLOW.  ngb_get_synapses returns the current weights. */
NGB_API int ngb_connect_stdp(ngb_sim* sim, int32_t src_pop, int32_t tgt_pop, const ngb_conn_spec* conn,
                             const ngb_syn_spec* syn, const ngb_stdp_params* stdp);

/* ----------------------------------------------------- continuous batching */
/* Make the handle a serving handle: reserve pools for max_neurons neurons,
 * max_synapses synapses and max_groups (source, delay) connection groups, a
 * ring of ring_slots (power of two, > every delay in steps) slots and
 * `receptors` receptors (1-4: at least 2 if any AdEx instance will come,
 * at least n_ports for beta instances).  Call before the
 * handle is finalised.  Afterwards instances may be added (ngb_add_instance,
 * ngb_add_population_in, ngb_connect) and committed or retired between
 * simulate calls, while the other instances keep running in the same kernels.
 * Population ids and global neuron ids then refer to pool positions, valid
 * once the instance is committed. */
NGB_API int ngb_reserve(ngb_sim* sim, int64_t max_neurons, int64_t max_synapses, int64_t max_groups,
                        int32_t ring_slots, int32_t receptors);

/* Serving handles: build a pending instance's connections on the device
 * into the pools (Sec. 2.1 rules, Sec. 2.2 groups) and make it active from
 * the current step on (its instance-local step 0).  NGB_ERR_OOM when a pool
 * lacks room (nothing is changed then); NGB_ERR_OVERFLOW when a delay does
 * not fit the reserved ring. */
NGB_API int ngb_commit_instance(ngb_sim* sim, int32_t instance);

/* Serving handles: stop an active instance and return its pool ranges.  Its
 * recorded spikes stay readable until another instance reuses the neurons. */
NGB_API int ngb_retire_instance(ngb_sim* sim, int32_t instance);

/* The step at which an instance became active and its state (0 pending,
 * 1 active, 2 retired). */
NGB_API int ngb_instance_info(ngb_sim* sim, int32_t instance, int64_t* t0_out, int32_t* state_out);

/* Build the delay-grouped CSR on the device (Sec. 2.2 connection groups),
 * allocate state, ring buffer and spike lists, and capture the step graph.
 * Called implicitly by the first ngb_simulate. */
NGB_API int ngb_finalize(ngb_sim* sim);

/* ----------------------------------------------------------- simulation */
/* Advance every instance by `steps` steps; returns when done (blocking).
 * The step's kernels are chained with programmatic dependent launch unless
 * the environment variable NGB_PDL is "0" when the network is finalised. */
NGB_API int ngb_simulate(ngb_sim* sim, int64_t steps);

/* As ngb_simulate, without CUDA graphs, with CUDA events around every kernel
 * launch.  kernel_ms[3] receives the summed device time of the LIF update,
 * AdEx update and delivery kernels; launches[3] their launch counts.  In the
 * fused step loop (ngb_stats.mode 2) the update kernels include the delivery
 * of their own spikes and entry 2 is the step-counter launch. */
NGB_API int ngb_simulate_profiled(ngb_sim* sim, int64_t steps, double* kernel_ms, int64_t* launches);

/* Autotune the step loop on this network: the per-step kernels in CUDA
 * graphs with the delivery kernel at 1, 2, 4 or 8 blocks per SM; the
 * pipelined loop (ring scheme: a spike's delay-1 group delivered by the
 * update kernel at once, its other groups by a delivery kernel that runs
 * beside the next step's update, in two-stream CUDA graphs; for LIF
 * networks also with one kernel per step whose extra blocks deliver the
 * previous step's queue) at the same delivery grids; the fused
 * loop (ring scheme: each update block delivers its own spikes, one launch
 * per step and model, in CUDA graphs); the persistent step kernel (one
 * cooperative launch for many steps, grid barriers between its phases) and,
 * with the ring scheme, its pipelined variant (one grid barrier per step: the
 * update phase delivers delay-1 groups and the queued groups of the previous
 * step) at 1 to 4 blocks per SM; for static LIF networks with the ring
 * scheme whose per-block ring fits in shared memory, the target-owned
 * persistent kernel (its tile-major synapse layout, about 1.5 - 2 times the
 * CSR's bytes, is built on first use; deterministic mode gives bit-identical
 * results to every other loop); at step 0 with delivery AUTO, under both delivery
 * schemes (ngb_stats.delivery); for AdEx networks, the chosen per-step or
 * pipelined loop also without the hot lists (ngb_stats.hot_steps).  Each candidate is
 * timed over trial_steps steps (0 = 500); the simulation state is saved
 * before and restored after the trials, so the simulation does not advance.
 * The fastest candidate is kept (see ngb_stats.mode / launch_grid).  With the
 * environment variable NGB_AUTOTUNE_CACHE naming a file, results are looked up
 * and appended there per (GPU, network shape) key.  *deliver_grid_out (may be
 * NULL) receives the chosen grid.  The environment variable NGB_MODE
 * ("persistent", "persistent_pipelined", "fused", "pipelined", "pipelined_one_kernel", "target_owned" or
 * "tiled") selects that step loop at finalisation without tuning (networks the loop does not take keep the
 * per-step kernels); "tiled" selects target-tiled delivery with the spike-buffer scheme (stats mode 7;
 * its layout, another copy of the synapses partitioned by target tile, is built at finalisation; the
 * autotuner does not consider it, being slower than the plain delivery kernel on the networks measured),
 * with NGB_TILED = "T,P" setting the tile size (neurons) and the blocks per tile (1-8, a thread-block
 * cluster when above 1). */
NGB_API int ngb_autotune(ngb_sim* sim, int64_t trial_steps, int32_t* deliver_grid_out);

/* Spikes recorded in steps [t0_step, t1_step) of population `pop` (-1 = all,
 * then ids are global; else population-local), sorted by (step, id).  With
 * ids == NULL only *n_out is set.  Otherwise up to `capacity` entries are
 * written and *n_out is the number available. */
NGB_API int ngb_get_spikes(ngb_sim* sim, int32_t pop, int64_t t0_step, int64_t t1_step, int32_t* ids,
                   int64_t* steps, int64_t capacity, int64_t* n_out);

/* --------------------------------------------------------- introspection */
NGB_API int ngb_get_stats(ngb_sim* sim, ngb_stats* out);

/* Global id of the first neuron of `pop` and its size. */
NGB_API int ngb_population_range(ngb_sim* sim, int32_t pop, int64_t* offset_out, int64_t* n_out);

/* Copy state variable `var` (ngb_state_var) of neurons [first, first+n) into out[n]. */
NGB_API int ngb_get_state(ngb_sim* sim, int32_t var, int64_t first, int64_t n, float* out);

/* Copy the input accumulated so far for step (current step + step_offset),
 * receptor `receptor`, neurons [first, first+n), as FP32 (offset 0 is the
 * complete synaptic input the next update consumes; the Poisson drive is not
 * included).  0 <= step_offset < ring slots; with the spike-buffer delivery
 * scheme only step_offset 0 exists (NGB_ERR_INVALID_ARG otherwise). */
NGB_API int ngb_get_input(ngb_sim* sim, int32_t receptor, int64_t step_offset, int64_t first, int64_t n, float* out);

/* Number of synapses of sources [0, N) before each source: src_ptr[N+1]. */
NGB_API int ngb_get_src_ptr(ngb_sim* sim, uint64_t* src_ptr);

/* Synapses [first, first+n) of the CSR in storage order (source, delay,
 * connect call, draw index): global target id, receptor, weight widened to
 * FP32, delay in steps. Any output pointer may be NULL. */
NGB_API int ngb_get_synapses(ngb_sim* sim, int64_t first, int64_t n, uint32_t* tgt, uint8_t* receptor, float* weight,
                     uint16_t* delay);

/* Evaluate, on the current device, the factor r^(-1/k) (k = 5 or 4) that
 * sizes the next sub-step of the adaptive Runge-Kutta integration of AdEx
 * neurons (Sec. 2.1: fifth-order Runge-Kutta with adaptive step size), for
 * the n ratios r[n] (error / tolerance) into out[n] (host arrays).  The
 * factor is an exactly specified sequence of FP32 operations (r = m 2^e,
 * e = k q + s; 2^-q * (c(m - 1) * 2^(-s/k)) with a fixed cubic c), so an
 * implementation on another processor can reproduce it bit for bit; ratios
 * below 2^-100 give 2^20, those of 2^100 and above or not finite give 0.
 * Blocking; allocates a temporary device buffer. */
NGB_API int ngb_eval_step_factor(const float* r, int64_t n, int32_t k, float* out);

/* --------------------------------------------------- allocation-free entry */
/* Device-resident CSR described by caller-owned DEVICE pointers (the layout
 * ngb_finalize builds): src_syn[N+1] first synapse of each source,
 * src_grp[N+1] first delay group of each source, grp_start[G+1] first synapse
 * of each group, grp_delay[G] its delay in steps, tgt[K] target id in bits
 * 0-25 with the receptor in bits 30-31 (bits 26-29 zero), weight[K] in
 * weight_dtype. */
typedef struct {
  const uint64_t* src_syn;
  const uint32_t* src_grp;
  const uint64_t* grp_start;
  const uint16_t* grp_delay;
  const uint32_t* tgt;
  const void* weight;
  int64_t num_neurons, num_synapses, num_groups;
  int32_t weight_dtype;
  int32_t pad_;
} ngb_csr_device;

/* Largest spike count one ngb_deliver_spikes_noalloc call accepts. */
#define NGB_NOALLOC_MAX_SPIKES 4096

/* Deliver the spikes of step t -- spikes[n_spikes], global source ids, a
 * DEVICE array -- through the CSR into the DEVICE ring buffer
 * ring[ring_slots][receptors][num_neurons] (FP32, or int64 in units of 2^-32
 * when fixed_point is 1), adding each synapse's weight at slot
 * (t + delay) & (ring_slots - 1), on `stream` (a cudaStream_t, NULL = the
 * legacy default stream).  Asynchronous: returns after enqueueing.
 *
 * Counterpart in the paper: none -- this is a library convenience.  It exists
 * for callers that cannot allocate device memory (a host application that
 * owns all GPU memory through its own allocator, a plugin that is not allowed
 * to call cudaMalloc, a latency-critical loop that must never block in the
 * allocator): it calls no cudaMalloc, cudaFree or allocating library routine.
 * Its working memory is a fixed array of about 150 KB compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits; it limits a call to NGB_NOALLOC_MAX_SPIKES spikes (more is
 * NGB_ERR_INVALID_ARG).  The first call on each device looks up that array's
 * device address (with that device current); make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU (different streams, or devices sharing it) race, so serialise them.
 * Spike ids >= num_neurons and targets outside the ring are skipped. */
NGB_API int ngb_deliver_spikes_noalloc(const ngb_csr_device* csr, const uint32_t* spikes, int64_t n_spikes,
                                       void* ring, int64_t ring_slots, int32_t receptors, int32_t fixed_point,
                                       int64_t t, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NGB_H */
