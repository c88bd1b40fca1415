/*
 * ngb_oracle.h -- C interface of the plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is the slow, obviously-correct CPU
 * statement of the method of Golosio et al., "Fast simulations of highly-
 * connected spiking cortical models using GPUs" (NeuronGPU): the clock-driven
 * update of LIF neurons with exponential PSCs by exact integration (Sec. 2.1,
 * Eqs. 1-2), AdEx neurons with conductance synapses by adaptive fifth-order
 * Runge-Kutta (Sec. 2.1, Eqs. 3-5), Poisson drive (Sec. 2.1, devices),
 * delay-exact spike delivery (Sec. 2.2) and nearest-neighbour STDP synapses
 * (Sec. 2.1).  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header or constant with the GPU library.
 *
 * Parity status: every function is pinned by a test against something other
 * than itself (closed forms, cuRAND's host Philox generator, scipy's DOP853,
 * numpy/torch format conversions, brute-force dense delivery, exact counts),
 * except the network-level firing rates, which are "parity unpinned" beyond
 * agreement between this oracle and the GPU path.
 *
 * All functions return >= 0 on success and a negative value on error; the
 * message of the last error is returned by ora_last_error().
 */
#ifndef NGB_ORACLE_H
#define NGB_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_net ora_net;

/* Parameter vector layouts (doubles), in this order.
 * LIF (ORA_LIF_NPARAM = 14):
 *   tau_m_ms, C_m_pF, E_L_mV, V_reset_mV, V_th_mV, t_ref_ms, tau_syn_ms, I_e_pA,
 *   V_init_mean_mV, V_init_sd_mV, poisson_n_inputs, poisson_rate_hz,
 *   poisson_weight, poisson_receptor
 * AdEx (ORA_AEIF_NPARAM = 27):
 *   C_m_pF, g_L_nS, E_L_mV, V_T_mV, Delta_T_mV, a_nS, b_pA, tau_w_ms,
 *   V_peak_mV, V_reset_mV, E_ex_mV, E_in_mV, tau_ex_ms, tau_in_ms, I_e_pA,
 *   V_init_mean_mV, V_init_sd_mV, w_init_pA, rk_tol, rk_h_min_ms,
 *   rk_h_init_ms, rk_max_substeps, poisson_n_inputs, poisson_rate_hz,
 *   poisson_weight, poisson_receptor, precision (0 = FP32 state as the GPU
 *   specification, 1 = FP64 reference at the full tolerance)
 */
#define ORA_LIF_NPARAM 14
#define ORA_AEIF_NPARAM 27

const char* ora_last_error(void);

ora_net* ora_create(double dt_ms, uint64_t seed, int32_t weight_prec /*0 fp32,1 bf16,2 fp16*/,
                    int32_t deterministic, int32_t track_abs);
void ora_destroy(ora_net* net);
int32_t ora_add_instance(ora_net* net, uint64_t seed);
int32_t ora_add_population(ora_net* net, int32_t instance, int32_t model /*0 LIF, 1 AdEx exp, 2 AdEx alpha*/,
                           int64_t n, const double* params);
int32_t ora_connect(ora_net* net, int32_t src_pop, int32_t tgt_pop, int32_t rule /*0 indeg, 1 total, 2 outdeg, 3 one-to-one, 4 all-to-all*/,
                    int64_t K, int32_t allow_autapses, int32_t wdist, double w0, double w1,
                    int32_t ddist, double d0, double d1, int32_t receptor);  /* returns the call index */
/* Make the synapses of connect call `call` plastic: nearest-neighbour STDP
 * (Sec. 2.1, after Morrison et al. 2008) with p = {tau_plus_ms, tau_minus_ms,
 * lambda, alpha, mu_plus, mu_minus, W_max}; at most 15 rules per network. */
int32_t ora_set_stdp(ora_net* net, int32_t call, const double* p);
int32_t ora_finalize(ora_net* net);
int32_t ora_simulate(ora_net* net, int64_t steps);
int32_t ora_inject(ora_net* net, int64_t neuron, int32_t receptor, int64_t step_offset, double value);

int64_t ora_num_neurons(const ora_net* net);
int64_t ora_pop_offset(const ora_net* net, int32_t pop);
int64_t ora_num_synapses(const ora_net* net);
int64_t ora_ring_length(const ora_net* net);
int64_t ora_steps_done(const ora_net* net);
int64_t ora_events(const ora_net* net);
int64_t ora_num_spikes(const ora_net* net);
int32_t ora_get_csr(const ora_net* net, uint64_t* src_ptr, uint32_t* tgt, uint8_t* receptor,
                    float* weight, uint16_t* delay);
int32_t ora_get_state(const ora_net* net, int32_t var, double* out);
int32_t ora_get_input(const ora_net* net, int32_t receptor, int64_t step_offset, float* out,
                      double* abs_out, double* exact_out);
int32_t ora_get_spikes(const ora_net* net, int64_t* ids, int64_t* steps);
int64_t ora_rk_substeps(const ora_net* net);
int64_t ora_rk_cap_hits(const ora_net* net);

/* Synapses of the given global source ids in canonical order (source, delay,
 * call, draw index), computed draw by draw without building the network (the
 * network need not be finalised).  Returns the number of synapses; at most cap
 * are written. */
int64_t ora_rows_for_sources(const ora_net* net, int64_t n_src, const int64_t* srcs, int64_t cap,
                             uint32_t* src_out, uint32_t* tgt, uint8_t* receptor, float* weight, uint16_t* delay);

/* Building blocks exposed for the pins. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int32_t ora_poisson_inversion(double lambda, uint32_t x);
void ora_lif_propagators(double tau_m, double C_m, double tau_syn, double h, double out[4]);
void ora_cash_karp_tableau(double c[6], double a[36], double b5[6], double b4[6]);
float ora_round_weight(float w, int32_t prec);
double ora_normal_from_words(const uint32_t w[4]);
/* r^(-1/k) (k = 4 or 5) by the fixed FP32 operation sequence that sizes the
 * next Runge-Kutta sub-step of the FP32-state AdEx integration (Sec. 2.1). */
float ora_step_factor_root(float r, int32_t k);

#ifdef __cplusplus
}
#endif
#endif
