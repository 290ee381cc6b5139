// Internal declarations of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "qaoa.h"

namespace qaoa {

// ---------------------------------------------------------------------------
// Errors: every ABI entry point returns a status; the message is thread-local.
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
#define QAOA_CUDA_TRY(call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ::qaoa::cuda_error(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Device facts, queried once per device.
struct DeviceInfo {
    int device = -1;
    int sms = 0;
    size_t smem_optin = 0;
};
int device_info(DeviceInfo *out);

// ---------------------------------------------------------------------------
// Per-(device, stream) scratch owned by the library.  Grows on demand; the
// pinned host block receives results of device reductions.
struct Scratch {
    void *dev = nullptr;   // device bytes
    size_t dev_bytes = 0;
    void *host = nullptr;  // pinned host bytes
    size_t host_bytes = 0;
};
// Returns scratch for `stream` on the current device with at least the given
// capacities (device, pinned host).  Not thread-safe per stream: one caller
// thread per stream at a time, as for any CUDA stream.
int scratch_for(cudaStream_t stream, size_t dev_bytes, size_t host_bytes, Scratch **out);
// Kernel attributes (the dynamic shared-memory limit) belong to a device:
// the current device's ordinal for per-device set-up state, or -1 with the
// error recorded when it is out of [0, MAX_DEVICES).
constexpr int MAX_DEVICES = 64;
int current_device_slot();

// ---------------------------------------------------------------------------
// Instrumentation: kernel kinds, launch counting and optional event timing.
enum KernelKind {
    K_COST_TABLE = 0,
    K_PASS_LOW,
    K_PASS_HIGH,
    K_SMALL_N,
    K_REDUCE,
    K_PSUCC,
    K_ADJ_LOW,
    K_ADJ_HIGH,
    K_ADJ_SEED,
    K_SERVE_SMALL,
    K_SAMPLE,
    K_NUM_KINDS
};
// Call before / after a launch on `stream`.  `after` checks the launch status.
void profile_before(int kind, cudaStream_t stream);
int profile_after(int kind, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Pass plan: how one layer's mixer is split into HBM passes.  Pass 0 is the
// "low" pass over the contiguous tile bits [0, T); each further pass is a
// "high" pass whose tile is 2^row contiguous elements times 2^G rows strided
// by 2^lo (G = T - row, state bits [lo, lo + G)); it butterflies the top `bits`
// of those G bits (the others were mixed by an earlier pass).
struct Pass {
    int lo;    // lowest state bit of the tile's strided group
    int bits;  // qubits butterflied by this pass (the low pass: T)
    int row;   // contiguous low bits per tile row (the low pass: T)
};
struct Plan {
    int n = 0;
    int state_bits = 0;  // index bits of the stored state (n, or n - 1 when halved)
    int z2 = 0;          // halved by the global-flip symmetry
    int tile_bits = 0;   // T
    int n_passes = 0;
    Pass pass[8];
};
constexpr int T_C64 = 13;   // 2^13 complex64 = 64 KiB tile
constexpr int T_C128 = 12;  // 2^12 complex128 = 64 KiB tile
constexpr int G_MAX_C64 = 9;
constexpr int G_MAX_C128 = 8;
int make_plan(int n, int dtype, Plan *plan, bool z2 = false);
// Plan for a tile of 2^T amplitudes and high groups of at most gmax bits.
// With `wide`, groups that can spare a bit take gmax - 1 bits and rows of
// T - gmax + 1 bits instead (twice the contiguous bytes per row, which the
// HBM streams more efficiently at large strides); the top groups go wide first.
int make_plan_geo(int n, int T, int gmax, Plan *plan, bool z2 = false, bool wide = false);

// One launch of the forward evolution: pass `pass` of the plan for layer `la`.
// Modes: 0 = first pass of layer 0 (the state |+> is generated from the phase
// table), 1 = butterflies of one layer, 2 = butterflies of layer la, the phase
// of layer la + 1 and the butterflies of layer la + 1 on the same tile,
// 3 = the phase of layer la applied at load, then its butterflies.
// The qubit groups of a layer commute, so their order alternates between
// layers and the last pass of a layer fuses with the first of the next; the
// low pass always sits inside a layer (its fused form would be bound by the
// SMs rather than by HBM), so only high passes fuse.
struct Launch {
    int pass, la, mode;
};
enum PassMode { MODE_INIT = 0, MODE_PLAIN = 1, MODE_FUSED = 2, MODE_PHASE = 3 };
std::vector<Launch> make_schedule(int n_passes, int p);

// The backward (adjoint) sweep, layers p-1 down to 0.  Each launch undoes the
// butterflies of layer la on one group; the last pass of a layer also takes
// the phase term and undoes D_la (A_PHASE), and when layer la - 1 starts with
// the same group it goes on to undo that layer's butterflies too (A_FUSED).
// With two or more high groups the orders alternate ([1, 0, 2, ..., k] and
// [k, 0, k-1, ..., 1]) so every layer boundary fuses on a high group; with one
// high group each layer is [1, 0] with the phase in the low pass.
enum AdjMode { A_PLAIN = 0, A_PHASE = 1, A_FUSED = 2 };
std::vector<Launch> make_adj_schedule(int n_passes, int p);

// ---------------------------------------------------------------------------
// Host-side per-layer coefficients.  One mixer layer is
//   prod_j [c I + i S X_j] = sigma^n prod_j [A I + i B X_j]
// with (sigma, A, B) chosen so that A = 1 or B = 1 (one FMA per component).
// `arith` is the arithmetic of the kernels that take A and B: the non-unit
// coefficient is returned already rounded to it (exactly representable there)
// and sigma is derived from that rounded value.
enum Arith { ARITH_F32 = 0, ARITH_F64 = 1, ARITH_DF = 2 };
struct LayerCoef {
    double sigma, A, B;
    bool unit_a;  // true: A == 1, else B == 1
};
LayerCoef layer_coef(double beta, int sign, int arith);
inline int arith_of(int dtype, int flags) {
    return dtype == QAOA_C64 ? ARITH_F32 : ((flags & QAOA_DF64) ? ARITH_DF : ARITH_F64);
}

// Phase table of one layer: T[c] = scale * exp(-i gamma c), c = 0..m (FP64 on
// the host; cast to the state's element type by the caller).
void phase_table(double gamma, double scale, int m, double *re, double *im);

// Largest cost a phase table indexes.  The cost table is uint8, so
// C(x) <= 255 whatever m is: a table holds entries 0..table_top(m).
inline int table_top(int m) { return m < 255 ? m : 255; }
// Number of clause-count entries a phase table must hold.
constexpr int MAX_TABLE = 256;

// ---------------------------------------------------------------------------
// Cost-table internals shared by the cost-table and serving code.
struct ClauseRec {
    uint32_t hi_mask;  // mask of the clause's variables >= 5 (as bits of x)
    uint32_t hi_neg;   // negation pattern on those variables
    uint32_t all_true; // bit b: every literal on a variable < 5 is true at x = b (mod 32)
    uint32_t all_false;// bit b: every such literal is false at x = b (mod 32)
};
int encode_instance(const naesat_instance *inst, ClauseRec *out);
int validate_instance(const naesat_instance *inst);
// Launches the batched cost-table kernel: recs [batch][m_stride] on the device,
// m per instance on the device, results into d_stats [batch][2] (uint64 n_sol,
// uint64 max C) which must be zeroed first.  With d_ns == nullptr all
// instances have n qubits and consecutive tables; otherwise instance b has
// d_ns[b] <= n qubits and its table at d_costs + d_offs[b].  `mirror`: the
// tables are full ones (2^n entries), counted on their lower half and
// completed by the global-flip symmetry; false for the lower-half tables of
// the halved state (n then counts their index bits).
int launch_cost_table_batch(int batch, int n, const int *d_ns, const uint64_t *d_offs, const ClauseRec *d_recs,
                            const int *d_m, int m_stride, uint8_t *d_costs, unsigned long long *d_stats,
                            cudaStream_t stream, bool mirror);
// One table.  Up to 1023 clauses the records go as kernel parameters (no
// staging); a longer list is copied to d_big (device, cost_table_big_bytes(m)
// bytes, 16-byte aligned) and counted chunk by chunk.
int launch_cost_table_one(const naesat_instance *inst, uint8_t *d_cost, unsigned long long *d_stats,
                          cudaStream_t stream, bool half, void *d_big);
size_t cost_table_big_bytes(int m);

// Multi-pass evolution of `batch` states (device side only, no host sync).
// `tables` holds p layers x (m + 1) complex FP64 entries (interleaved).
struct EvolveReq {
    int batch, n, m, p, dtype, flags;  // flags & QAOA_Z2_HALF: halved state and half cost tables
    const uint8_t *cost;
    void *state;
    void *adj;          // nullable: if set, the last pass also writes P psi into it
    const double *gamma, *beta;
    double *d_result;   // nullable: device [batch][2] (p_succ, norm)
};
// Runs the passes of `r` on `stream`; d_partials holds batch x gx x 2 doubles
// (gx from pass_grid_x); r.d_result (if set) receives [batch][2].
int evolve_device_impl(const EvolveReq &r, cudaStream_t stream, double *d_partials, int gx);
int pass_grid_x(int dtype, int n, int batch);
// Grid width per instance for `batch` instances of `tiles` tiles on `slots`
// resident CTAs (the wave-balanced choice; 1 <= result <= min(slots, tiles)).
int balanced_grid_x(int slots, int batch, uint64_t tiles);
// Fixed-order sums: out[g][k] = sum_j part[g][j][k] for g < groups, k < nv <= 4.
int launch_reduce(const double *part, int groups, int nblk, int nv, double *out, cudaStream_t stream);

// Small-n whole-evolution kernel for a packed batch (serving and n <= T).
struct SmallJob {
    const uint8_t *cost;  // device [2^n]
    void *state;          // device [2^n] (may be null: state not kept)
    double *result;       // device [2] (p_succ, norm)
    int n, m, p;
    int table_off;        // offset (in complex entries) of this job's tables
    int coef_off;         // offset (in layers) of this job's coefficients
};
int launch_small_batch(int dtype, int n_jobs, const SmallJob *d_jobs, const double *d_tables,
                       const double *d_coefs, int max_n, int flags, cudaStream_t stream);
// Largest n that the single-instance evolution runs in one CTA (the pass path
// needs n > T), and the largest n the packed small-n kernel accepts.
int small_n_limit(int dtype);
int small_n_pack_limit(int dtype);

}  // namespace qaoa
