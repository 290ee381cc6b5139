/*
 * qaoa.h - C ABI of the GB300 (sm_103a) statevector library for depth-p QAOA
 * on random NAE-k-SAT (arXiv 2401.02852).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Assignment index x = sum_l x_l 2^l: variable l is bit l of x.  X_j flips
 *    bit j.  (The paper's decimal representation in Appendix A.3 is garbled;
 *    this is the reading used throughout.)
 *  - A literal (v, neg) takes the value of bit v of x, complemented when
 *    neg = 1 (negated literal, Eq. for the literal Hamiltonian, Appendix A.2).
 *  - State vectors are device arrays of 2^n complex amplitudes, interleaved
 *    (re, im): QAOA_C64 = 2 x float (8 bytes), QAOA_C128 = 2 x double (16 bytes).
 *  - Cost tables are device uint8 arrays of 2^n entries, C(x) exact.
 *  - Angles are host float64 arrays in radians; layer 0 (gamma[0], beta[0])
 *    acts first on |+>^n (the product of the QAOA output state, Sec. "QAOA
 *    Procedure", read right to left).
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Device pointers are owned by the caller; the library never frees them.
 *    The library keeps its own small per-(device, stream) scratch (reduction
 *    partials, counters, pinned result slots), allocated on first use on that
 *    stream and released by qaoa_release_scratch().
 *  - Host result pointers (p_succ, norm, n_sol, ...) are written before the
 *    call returns: such calls synchronise the stream.  Passing NULL skips the
 *    result (and the reduction that produces it) where documented.
 *  - Every entry point returns an int status (QAOA_OK = 0, QAOA_PENDING > 0,
 *    errors < 0); no exception crosses the ABI.  qaoa_last_error() gives a
 *    thread-local message for the last failing call of the calling thread.
 *  - Arguments are validated on the host before any device work; an invalid
 *    call changes no device memory.
 */
#ifndef QAOA_NAESAT_H
#define QAOA_NAESAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QAOA_OK 0
#define QAOA_PENDING 1     /* serving: request not finished yet                */
#define QAOA_EINVAL (-1)   /* malformed argument (NULL, bad enum, bad clause)   */
#define QAOA_ERANGE (-2)   /* size out of range (n > 32, m > 8191, k > n,
                              max C > 255 for the uint8 table, tile limits)     */
#define QAOA_ENOMEM (-3)   /* device or host allocation failed / over budget    */
#define QAOA_ECUDA (-4)    /* a CUDA runtime call failed (message has details)  */
#define QAOA_ETIMEOUT (-5) /* serving: wait deadline passed                     */
#define QAOA_ECANCELLED (-6) /* serving: request cancelled                      */
#define QAOA_ENOTFOUND (-7)  /* serving: unknown ticket                         */

/* ---- element types and flags ------------------------------------------- */
#define QAOA_C64 0  /* complex64 state, FP32 butterflies, FP64 reductions   */
#define QAOA_C128 1 /* complex128 state, FP64 throughout                    */

/* Mixer sign.  The paper writes U_B(beta) = exp(-i beta H_B) in Sec. 2.1 but
 * uses U_B(beta) = exp(+i beta sum_j X_j) = prod_j [cos(beta) I + i sin(beta)
 * X_j] for the NAE problem (Sec. "Efficient Classical Simulation", Appendix
 * A.3: the sign flips because the problem is posed as a minimisation).  The
 * default is the latter.  QAOA_MIXER_RX2B selects exp(-i beta sum_j X_j) =
 * prod_j RX(2 beta). */
#define QAOA_MIXER_PAPER 0x0
#define QAOA_MIXER_RX2B 0x1

/* Halved state.  NAE-SAT is symmetric under the global bit flip (Sec. 2.2):
 * C(x) = C(not x), and |+>, U_C and U_B commute with the flip, so
 * psi(x) = psi(not x) at every layer.  With QAOA_Z2_HALF the state buffer holds
 * only the 2^(n-1) amplitudes with bit n-1 clear and the cost table only
 * C(x) for those x (naesat_cost_table_half); the mixer's factor on qubit n-1
 * then pairs x with 2^(n-1) - 1 - x.  Results (p_succ, norm) are those of the
 * full state.  Exact: the same numbers as the full evolution, half the bytes. */
#define QAOA_Z2_HALF 0x2

/* QAOA_DF64 (complex128 evolutions only, full state, not for the gradient):
 * the state stays complex128 in memory and in the result, but between passes
 * it is held as double-float pairs (hi + lo floats, about 48 significant bits)
 * and the butterflies and phases run in that arithmetic on the FP32 pipes,
 * which on GB300 are far faster than the FP64 pipe.  Per-operation error about
 * 2^-45 of the operands instead of 2^-53 (n = 30, p = 10: p_succ within about
 * 1e-13 of FP64).  Small n (the one-CTA path) takes it too. */
#define QAOA_DF64 0x4

#define QAOA_MAX_N 32
/* Clause counts up to 8191 cover the threshold densities of k = 3..10 at the
 * paper's sizes (Sec. "Random Problems": m ~ Poisson(r n), r near the
 * satisfiability threshold, about 350 n at k = 10). */
#define QAOA_MAX_M 8191

/* One NAE-k-SAT instance, host memory.  var[i*k + j] in [0, n) is the variable
 * of literal j of clause i (distinct within a clause); neg[i*k + j] in {0, 1}
 * marks a negated literal.  Sec. "Random Problems" / Def. of CNF(n, k, r). */
typedef struct {
    int32_t n, m, k;
    const int32_t *var;
    const uint8_t *neg;
} naesat_instance;

/* Thread-local text of the last error of the calling thread ("" if none). */
const char *qaoa_last_error(void);

/* ABI version (major * 100 + minor). */
int qaoa_version(void);

/* Releases the library's scratch on every device (call with no work in
 * flight).  Returns QAOA_OK. */
int qaoa_release_scratch(void);

/* ---- cost table (Eq. for C^NAE, Sec. "Problem Hamiltonian") ----------------
 * C(x) = number of clauses whose k literals are all false or all true
 * (De Morgan form, Appendix A.2), for every x in [0, 2^n).
 *   inst      host instance (validated: 1 <= n <= 32, 0 <= m <= 8191,
 *             1 <= k <= n, variables distinct within a clause).
 *   d_cost    device uint8 [2^n], written.
 *   n_sol     host, nullable: number of x with C(x) = 0 (exact brute force).
 *   max_cost  host, nullable: max_x C(x).
 * Returns QAOA_ERANGE (and leaves d_cost with every entry taken mod 256) when
 * some C(x) > 255; n_sol and max_cost are still exact in that case.
 * Synchronises the stream when n_sol or max_cost is requested. */
int naesat_cost_table(const naesat_instance *inst, uint8_t *d_cost, uint64_t *n_sol,
                      uint32_t *max_cost, void *stream);

/* Half table for the QAOA_Z2_HALF mode: C(x) for x in [0, 2^(n-1)) only
 * (d_cost_half device uint8 [2^(n-1)], n >= 6).  C(not x) = C(x) under NAE, so
 * this determines the full table; n_sol and max_cost are those of the full
 * table (n_sol = 2 x the half count).  Same errors as naesat_cost_table. */
int naesat_cost_table_half(const naesat_instance *inst, uint8_t *d_cost_half, uint64_t *n_sol,
                           uint32_t *max_cost, void *stream);

/* Same for `batch` instances of one n: d_costs is device uint8 [batch][2^n];
 * n_sol / max_cost are host arrays [batch] (nullable). */
int naesat_cost_table_batch(int batch, const naesat_instance *insts, uint8_t *d_costs,
                            uint64_t *n_sol, uint32_t *max_cost, void *stream);

/* ---- state evolution (Eq. for the QAOA output state) -----------------------
 * d_state <- prod_{l=0}^{p-1} U_B(beta_l) U_C(gamma_l) |+>^n, with
 * U_C(gamma) = diag(exp(-i gamma C(x))) (Eq. for U_C) and the mixer of `flags`.
 *   n        1..32 (C64) / 1..31 (C128); the state must fit in device memory.
 *   d_cost   device uint8 [2^n] from naesat_cost_table.
 *   m        number of clauses, 0 <= m <= 8191 (bounds C; the phase tables
 *            have min(m, 255) + 1 entries, the uint8 costs index no more).
 *   p        depth >= 0 (p = 0 returns |+>^n).
 *   gamma, beta  host float64 [p].
 *   dtype    QAOA_C64 or QAOA_C128.
 *   d_state  device [2^n] of dtype, written (no input is read from it).
 *   p_succ, norm  host, nullable: p_succ = sum_{C(x)=0} |psi(x)|^2 (Def. of the
 *            success probability, unnormalised) and sum_x |psi(x)|^2, reduced
 *            in FP64 inside the last pass.
 * Synchronises the stream when p_succ or norm is requested. */
int qaoa_evolve(int n, const uint8_t *d_cost, int m, int p, const double *gamma, const double *beta,
                int dtype, int flags, void *d_state, double *p_succ, double *norm, void *stream);

/* `batch` independent instances of one n sharing the angles:
 * d_costs [batch][2^n], d_states [batch][2^n], m_max = max clause count,
 * p_succ / norm host [batch] (nullable). */
int qaoa_evolve_batch(int batch, int n, const uint8_t *d_costs, int m_max, int p, const double *gamma,
                      const double *beta, int dtype, int flags, void *d_states, double *p_succ,
                      double *norm, void *stream);

/* ---- success probability (Def. of the k-NAE-SAT success probability) -------
 * p_succ = sum_{x: C(x)=0} |psi(x)|^2 and norm = sum_x |psi(x)|^2 of a given
 * device state (FP64 accumulation, deterministic order).  Both host outputs
 * are required.  Synchronises the stream. */
int qaoa_success_prob(int n, const uint8_t *d_cost, const void *d_state, int dtype, double *p_succ,
                      double *norm, void *stream);

/* Same result as qaoa_success_prob, for callers that cannot allocate device
 * memory at the point of the call: hosts whose own allocator has reserved the
 * whole device, or paths (real-time loops, signal handlers) that must not risk
 * the implicit device synchronisation of cudaMalloc.  The paper has no
 * counterpart; this is an interface variant of the reduction above.
 *   Scratch: a fixed device array inside the library (2 x 4096 + 2 doubles,
 *   about 64 KiB), held by every GPU that loads the library until exit.  The
 *   call uses at most 4096 blocks, each striding over the state, so every n in
 *   [1, 32] fits; other n return QAOA_ERANGE.  No cudaMalloc, cudaFree or other
 *   allocating routine is called; the result is copied into a local host buffer.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, which also loads the
 *   library's device code on that device if nothing of the library has run
 *   there yet (CUDA loads modules lazily by default): that load allocates the
 *   module and its fixed array.  So make one warm-up call per device at
 *   start-up, before the caller's own allocator reserves the device and before
 *   any stream capture (or run with CUDA_MODULE_LOADING=EAGER, which loads
 *   the module when the context is created).  The address is kept for the
 *   life of the process: a device reset (cudaDeviceReset) between calls is
 *   not supported.
 *   Sharing: all calls share the array, which keeps the last call's contents;
 *   every entry a call reads is written earlier in the same call, so nothing
 *   needs clearing.  Calls whose work overlaps on the GPU (other streams or
 *   threads) race on the array: serialise them.
 * Synchronises the stream. */
int qaoa_success_prob_noalloc(int n, const uint8_t *d_cost, const void *d_state, int dtype, double *p_succ,
                              double *norm, void *stream);

/* ---- sampling and running times ------------------------------------------------
 * Bitstrings measured from a state (Sec. "Running Times": a measurement of the
 * output state yields x with probability |Psi(x)|^2, and the running time of an
 * instance is the number of measured bitstrings up to and including the first
 * that satisfies it).  The caller supplies the randomness: one uniform u_j in
 * [0, 1) per draw, device float64 [k] (per instance [batch][k]).  Draw j is
 *   x_j = min { x : F(x) > u_j F_total },   F(x) = sum_{y <= x} |psi(y)|^2
 * (inverse CDF in index order; within each block of 2^13 amplitudes the
 * probabilities are integer weights on a binary scale, about 2^-44 of the
 * block's largest probability, summed exactly; the block totals are summed
 * in FP64; so it differs from a sequential FP64 scan only for u_j within
 * about 2^-40 F_total of a step of F; a probability below about 2^-44 of
 * its block's largest, or below about 1e-45, weighs 0).  An x of probability
 * zero is never drawn; a u_j <= 0 yields the first and a u_j >= 1 the last x
 * of nonzero weight; a state of norm zero draws 0.  With QAOA_Z2_HALF the state and table are the
 * halved ones (the x with bit n-1 clear, psi(not x) = psi(x)) and draws cover
 * all 2^n assignments: u_j < 1/2 draws the stored x at 2 u_j, u_j >= 1/2 the
 * complement of the stored x drawn at 2 u_j - 1 (the same distribution; u_j
 * >= 1 then gives the complement of the last stored x of nonzero
 * probability).  k in [1, 2^30].
 *
 * qaoa_sample: d_x device uint64 [k], written.  Asynchronous on the stream.
 */
int qaoa_sample(int n, const void *d_state, int dtype, int flags, int k, const double *d_u, uint64_t *d_x,
                void *stream);

/* Running time over the draws of d_u: *running_time = 1 + the index of the
 * first draw with C(x_j) = 0, or 0 when none of the k draws satisfies (draw
 * again with fresh uniforms and add k).  d_x: device uint64 [k] receiving the
 * draws, nullable (library scratch).  Synchronises the stream. */
int qaoa_running_time(int n, const uint8_t *d_cost, const void *d_state, int dtype, int flags, int k,
                      const double *d_u, int64_t *running_time, uint64_t *d_x, void *stream);

/* Batched running times for `batch` instances of one n: d_costs [batch][2^n]
 * (halved: [batch][2^(n-1)]), d_states likewise, d_u [batch][k],
 * running_time host int64 [batch].  batch in [1, 65535].  Synchronises. */
int qaoa_running_time_batch(int batch, int n, const uint8_t *d_costs, const void *d_states, int dtype, int flags,
                            int k, const double *d_u, int64_t *running_time, void *stream);

/* ---- gradient ----------------------------------------------------------------
 * dp_succ/dgamma_l and dp_succ/dbeta_l by a reverse sweep that recomputes the
 * states backward with inverse layers (no stored intermediate states).  The
 * paper trains the fixed angles by gradient ascent on p_succ (Sec. "QAOA
 * Procedure"); this is the adjoint form of that derivative.
 *   d_state, d_adj  device scratch [2^n] of dtype each (overwritten; on
 *            return d_state holds |+>^n up to rounding, d_adj the adjoint).
 *   p_succ   host, nullable; dgamma, dbeta host float64 [p], written.
 * Synchronises the stream. */
int qaoa_grad(int n, const uint8_t *d_cost, int m, int p, const double *gamma, const double *beta,
              int dtype, int flags, void *d_state, void *d_adj, double *p_succ, double *dgamma,
              double *dbeta, void *stream);

/* Batched gradient for `batch` instances of one n sharing the angles.
 * d_costs [batch][2^n]; d_states, d_adjs [batch][2^n] scratch;
 * p_succ host [batch] (nullable); dgamma, dbeta host [batch][p]. */
int qaoa_grad_batch(int batch, int n, const uint8_t *d_costs, int m_max, int p, const double *gamma,
                    const double *beta, int dtype, int flags, void *d_states, void *d_adjs,
                    double *p_succ, double *dgamma, double *dbeta, void *stream);

/* ---- serving: continuous batching of whole requests ---------------------------
 * A server owns a scheduler thread, device memory for resident cost tables and
 * states (bounded by hbm_budget_bytes) and a few CUDA streams.  Requests of any
 * n (1..max_n) and depth arrive through qaoa_serve_submit; each is admitted
 * when its footprint fits the budget and a slot is free, packed with other
 * small-n requests into one launch when n <= small_n_max, and otherwise run as
 * a multi-pass evolution on one of the streams, batched with the waiting
 * requests of the same shape (same n, m, p and angles: one pass plan and one
 * set of phase tables), up to max_batch.  Small requests behind a large one
 * that is over the budget are still admitted.  Results are read with
 * qaoa_serve_poll / qaoa_serve_wait; each request's result is the same whether
 * it runs alone, packed or batched (its arithmetic depends on its own inputs
 * only).  (Not in the paper: a serving pattern around its simulation.) */
typedef struct qaoa_server qaoa_server;

typedef struct {
    size_t hbm_budget_bytes; /* admission budget for resident tables + states (0 = 50% of free) */
    int max_batch;           /* max requests per packed small-n launch or same-shape batch (0 = 256) */
    int n_streams;           /* CUDA streams for large requests (0 = 4)                       */
    int dtype;               /* QAOA_C64 or QAOA_C128                                          */
    int small_n_max;         /* n at or below which requests are packed (0 = default)         */
    int flags;               /* mixer sign flags as for qaoa_evolve; QAOA_Z2_HALF runs the
                                unpacked requests on the halved state (half the memory);
                                QAOA_DF64 (QAOA_C128 without QAOA_Z2_HALF) runs every request
                                in double-float arithmetic                                    */
    int device;              /* CUDA device ordinal                                            */
    int max_n;               /* largest n accepted (0 = 30)                                    */
} qaoa_server_opts;

typedef struct {
    double p_succ, norm;     /* as qaoa_evolve                                                 */
    uint64_t n_sol;          /* number of x with C(x) = 0                                       */
    uint32_t max_cost;       /* max_x C(x)                                                     */
    int32_t status;          /* QAOA_OK, or the error of this request                          */
    uint64_t t_submit_ns, t_start_ns, t_done_ns; /* CLOCK_MONOTONIC nanoseconds                */
} qaoa_result;

int qaoa_server_create(const qaoa_server_opts *opts, qaoa_server **out);
/* Copies the instance and angles; returns at once with a ticket. */
int qaoa_serve_submit(qaoa_server *s, const naesat_instance *inst, int p, const double *gamma,
                      const double *beta, uint64_t *ticket);
/* QAOA_OK with *out filled (the ticket is then retired), QAOA_PENDING, or an error. */
int qaoa_serve_poll(qaoa_server *s, uint64_t ticket, qaoa_result *out);
/* Blocks until the ticket finishes or timeout_s passes (QAOA_ETIMEOUT); timeout_s
 * must be finite and >= 0 (QAOA_EINVAL otherwise). */
int qaoa_serve_wait(qaoa_server *s, uint64_t ticket, qaoa_result *out, double timeout_s);
/* Cancels a request that has not started; QAOA_OK or QAOA_PENDING if running. */
int qaoa_serve_cancel(qaoa_server *s, uint64_t ticket);
/* Counters: submitted, completed, packed launches, single launches, peak bytes,
 * cancelled, errors, requests run in same-shape batches of two or more. */
int qaoa_server_stats(qaoa_server *s, uint64_t *counters /* [8] */);
/* Host time the scheduler thread has spent issuing work (staging uploads,
 * stream-ordered allocations, kernel launches and result copies, for all
 * slots), the number of issues (one per packed batch, same-shape batch or
 * single request) and the time since the first admission, all in ns: the
 * share of the scheduler's time that launches take. */
int qaoa_server_issue_time(qaoa_server *s, uint64_t *issue_ns, uint64_t *issues, uint64_t *span_ns);
/* Drains running work, joins the scheduler, frees device memory. */
int qaoa_server_destroy(qaoa_server *s);

/* ---- pass planning and instrumentation (host only, no device work) ----------
 * qaoa_plan describes how one layer of an n-qubit evolution in dtype (and
 * flags: QAOA_Z2_HALF, where pass 0 mixes qubits [0, T - 1) and qubit n - 1 and
 * the high passes work on n - 1 index bits) is split into HBM passes.  Pass 0 streams contiguous tiles and mixes qubits
 * [0, row_bits[0]).  Pass i > 0 streams tiles of 2^row_bits[i] contiguous
 * amplitudes times 2^G rows strided by 2^group_lo[i] (G = tile bits -
 * row_bits[i]) and mixes the top group_bits[i] qubits of its group.  Returns
 * the number of passes per layer (>= 1) or an error; arrays hold up to 8. */
int qaoa_plan(int n, int dtype, int flags, int *group_lo, int *group_bits, int *row_bits);

/* The launch sequence of a depth-p evolution: for launch i, the pass of
 * qaoa_plan it runs, its layer l and its mode (0: first pass of layer 0, which
 * generates |+> from the phase table; 1: butterflies of layer l; 2: butterflies
 * of layer l, then the phase and butterflies of layer l + 1 on the same tile;
 * 3: the phase of layer l at load, then its butterflies).  The qubit groups
 * commute within a layer, so their order alternates between layers and a
 * layer boundary on a strided group costs one pass instead of two.  Returns
 * the number of launches (p * (passes - 1) + 1 when every boundary fuses) or
 * an error; at most max_launches entries are written. */
int qaoa_pass_schedule(int n, int p, int dtype, int flags, int max_launches, int *pass_index, int *layer,
                       int *mode);

/* The launch sequence of the gradient's backward sweep (layers p-1 down to 0;
 * the passes are those of the backward plan: 2^12-amplitude tiles of both
 * states, groups of at most 8 bits).  For launch i: its pass (0 = low), its
 * layer l and its mode (0: undo the butterflies of layer l on the group;
 * 1: then take the phase term of layer l and undo its phase; 2: then also
 * undo the butterflies of layer l - 1 on the same group).  The phase of a
 * layer is undone only after all its butterflies (every qubit factor
 * commutes with the others, not with the phase).  Returns the number of
 * launches (P + (p - 1)(P - 1) for P passes per layer when every boundary
 * fuses) or an error; host only. */
int qaoa_adjoint_schedule(int n, int p, int dtype, int max_launches, int *pass_index, int *layer, int *mode);

/* Per-kernel timing: when enabled, every kernel the library launches is
 * bracketed by CUDA events on its stream.  qaoa_profile_read synchronises the
 * device, then returns for kernel kind i (names via qaoa_kernel_name) the
 * launch count and summed milliseconds; it resets the accumulators. */
int qaoa_profile_enable(int on);
int qaoa_profile_read(int max_kinds, uint64_t *launches, double *ms);
const char *qaoa_kernel_name(int kind);
/* Total kernels launched by this library in this process. */
uint64_t qaoa_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* QAOA_NAESAT_H */
