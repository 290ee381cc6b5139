// K5: gradient of p_succ with respect to the angles by a reverse (adjoint)
// sweep that recomputes the states backward with inverse layers.
//
// Forward: phi_l = D_l psi_{l-1}, psi_l = M_l phi_l, D_l = exp(-i gamma_l C),
// M_l = exp(i s beta_l B), B = sum_j X_j, f = <psi_p| P |psi_p>, P the
// projector on C = 0 (Def. of the success probability).  With
// lam_p = P psi_p and, going backward,
//   df/dbeta_l  = 2 Re <lam_l| i s B |psi_l> = -2 s Im <lam_l| B |psi_l>,
//   (phi_l, mu_l) = M_l^dagger (psi_l, lam_l),
//   df/dgamma_l = 2 Re <mu_l| -i C |phi_l> = 2 sum_x C(x) Im(conj(mu_x) phi_x),
//   (psi_{l-1}, lam_{l-1}) = D_l^dagger (phi_l, mu_l).
// Every X_j commutes with every single-qubit factor of M_l, so the term of qubit
// j, Im(conj(a') b + conj(b') a) over the pairs (x, x xor 2^j), is taken at the
// moment qubit j's inverse butterfly runs; the inverse butterflies are the
// normalised ones (c a - i S b, c b - i S a), so the states stay unit-norm.
//
// The paper differentiates through its simulator with automatic
// differentiation (Sec. "QAOA Procedure", training of the fixed angles); this
// computes the same derivative without storing the p intermediate states.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "pass_common.cuh"
#include "qaoa_internal.cuh"

namespace qaoa {

template <typename R>
using AGeo = Geo<R, 12, 4>;  // 2 tiles (psi, lam) of 2^12 amplitudes

template <typename R>
struct AdjArgs {
    typename AGeo<R>::V *psi, *lam;
    const uint8_t *cost;
    double *partials;   // layer l's slice: [batch][p][gx][2], base at layer l
    double *partials2;  // A_FUSED: layer l - 1's slice (nullable: no second layer)
    int n, row, lo, m, p;
    uint32_t active;
    R c, S;             // inverse butterfly coefficients of layer l
    R c2, S2;           // A_FUSED: those of layer l - 1
    uint64_t tiles;
};

template <typename R, int NT>
struct AdjTab {
    typename AGeo<R>::V t[NT];  // exp(+i gamma c)
};

// Inverse butterfly on psi and lam for the pair (i, j), with the mixer term.
template <typename V, typename R>
__device__ __forceinline__ void inv_pair(V &a, V &b, V &la, V &lb, R c, R S, R &term) {
    term += la.x * b.y - la.y * b.x + lb.x * a.y - lb.y * a.x;
    V na, nb;
    na.x = fma(c, a.x, S * b.y);
    na.y = fma(c, a.y, -S * b.x);
    nb.x = fma(c, b.x, S * a.y);
    nb.y = fma(c, b.y, -S * a.x);
    a = na;
    b = nb;
    na.x = fma(c, la.x, S * lb.y);
    na.y = fma(c, la.y, -S * lb.x);
    nb.x = fma(c, lb.x, S * la.y);
    nb.y = fma(c, lb.y, -S * la.x);
    la = na;
    lb = nb;
}

template <typename G, int LO, int BELOW>
__device__ __forceinline__ void inv_round(typename G::V *vp, typename G::V *vl, uint32_t mask, typename G::Real c,
                                          typename G::Real S, typename G::Real &term) {
    constexpr int RB = G::RB, NR = G::NR;
#pragma unroll
    for (int q = 0; q < RB; ++q) {
        if (LO + q < BELOW && ((mask >> (LO + q)) & 1u)) {
#pragma unroll
            for (int i = 0; i < NR; ++i)
                if (!(i & (1 << q))) inv_pair(vp[i], vp[i | (1 << q)], vl[i], vl[i | (1 << q)], c, S, term);
        }
    }
}

// Mapping change of both states.  complex64 amplitudes of psi and lam are
// packed into one 16-byte element per tile position and moved in one exchange
// over both buffers (half the shared-memory instructions and barriers of two
// 8-byte exchanges; the 16-byte padded layout is the complex128 one, conflict
// free for the same mappings); complex128 states are exchanged one by one.
template <typename G, int FROM, int TO>
__device__ __forceinline__ void exchange_pair(typename G::V *vp, typename G::V *vl, typename G::V *tp,
                                              typename G::V *tl) {
    if constexpr (sizeof(typename G::V) == 8) {
        using G4 = Geo<dfloat, G::T, G::RB>;  // 16-byte elements, same tile shape
        static_assert(G4::TILE_ELEMS == G::TILE_ELEMS, "tile shapes differ");
        float4 w[G::NR];
#pragma unroll
        for (int r = 0; r < G::NR; ++r) w[r] = make_float4(vp[r].x, vp[r].y, vl[r].x, vl[r].y);
        exchange<G4, FROM, TO>(w, reinterpret_cast<float4 *>(tp));  // tp and tl are adjacent
#pragma unroll
        for (int r = 0; r < G::NR; ++r) {
            vp[r] = make_float2(w[r].x, w[r].y);
            vl[r] = make_float2(w[r].z, w[r].w);
        }
    } else {
        exchange<G, FROM, TO>(vp, tp);
        exchange<G, FROM, TO>(vl, tl);
    }
}

// State offset of register r's tile element in mapping LO: its row part plus
// its group part times gstride = 2^lo (ROW: the tile's contiguous bits).
template <int LO, int ROW>
__device__ __forceinline__ uint32_t reg_off(int r, uint32_t gstride) {
    const uint32_t u = (uint32_t)r << LO;
    return (u & ((1u << ROW) - 1u)) + (u >> ROW) * gstride;
}

// One backward pass over the tiles of both states.  The tile pair (psi, lam)
// and, when the pass undoes a phase, the tile's cost bytes arrive by cp.async
// into dense shared buffers; the next pair is copied as soon as the last
// exchange has been read out, overlapping the last round, the phase and the
// stores.  MODE (AdjMode): A_PLAIN undoes layer l's butterflies on the group;
// A_PHASE then takes the phase term and undoes D_l; A_FUSED (high passes) also
// undoes layer l-1's butterflies on the same group, in the mapping it ends in
// and back (with c2 = 1, S2 = 0 and no partials2 it is A_PHASE for a high
// group).  HROW: row bits of a high pass; FULL: 1 = every group bit of the
// tile is undone here (a compile-time mask, straight-line stages), 0 = the
// runtime mask, 2 = (high passes) the runtime mask with every undone bit among
// the load mapping's register bits, so the pass needs no exchange: the next
// pair is copied as soon as this one is in registers, and the phase is taken
// in the load mapping.
template <typename R, bool LOW, int MODE, int NT, int HROW, int FULL>
__global__ void __launch_bounds__(PT, sizeof(R) == 4 ? 2 : 1) adj_kernel(const __grid_constant__ AdjArgs<R> a,
                                                                        const __grid_constant__ AdjTab<R, NT> tab) {
    static_assert(!LOW || MODE != A_FUSED, "the low pass never fuses");
    static_assert(LOW || MODE != A_PHASE, "a high pass undoes a phase in its fused form");
    constexpr bool PH = MODE != A_PLAIN;  // the pass undoes a phase
    using G = AGeo<R>;
    using V = typename G::V;
    constexpr int T = G::T, NR = G::NR;
    constexpr int LD = 8;  // load mapping: the registers on the top tile bits
    constexpr int LC = LOW ? G::LC_LOW : G::LC_HIGH;
    constexpr int row = LOW ? T : HROW;
    constexpr uint32_t full_mask = ((1u << T) - 1u) & ~(LOW ? 0u : (1u << row) - 1u);
    constexpr bool TOP = !LOW && FULL == 2;
    const uint32_t active = FULL == 1 ? full_mask : a.active;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tp = reinterpret_cast<V *>(smem_raw);
    V *tl = tp + G::TILE_ELEMS;
    // phase passes: two dense cost-byte buffers.  (The forward high passes pad
    // theirs so that the cost loads in mapping 4 take one wavefront instead of
    // two; here the extra per-thread offset made the fused kernels, which hold
    // both states in registers, spill, so the backward passes keep the dense
    // layout and its second wavefront.)
    uint8_t *scs = reinterpret_cast<uint8_t *>(tl + G::TILE_ELEMS);
    V *stab = reinterpret_cast<V *>(scs + (PH ? (2 << T) : 0));
    if (PH) {  // 256 entries at least: any uint8 cost indexes inside the table
        for (int i = threadIdx.x; i < 256 || i <= a.m; i += PT) {
            V z;
            z.x = z.y = 0;
            stab[i] = i <= a.m ? tab.t[i] : z;
        }
    }
    const uint32_t tid = threadIdx.x;
    const size_t inst = blockIdx.y;
    V *psi = a.psi + (inst << a.n);
    V *lam = a.lam + (inst << a.n);
    const uint8_t *cs = a.cost + (inst << a.n);
    constexpr int SM = (MODE == A_FUSED || TOP) ? LD : LC;  // store mapping
    const uint32_t st_t = elem_offset32(tile_elem<G, SM>(tid, 0), row, a.lo);
    const uint32_t gstride = LOW ? 0u : (1u << a.lo);
    const uint32_t tiles = (uint32_t)a.tiles;
    auto issue = [&](uint32_t tt, uint8_t *scb) {
        const uint32_t bb = tile_base32(tt, row, a.lo, T);
        issue_tile<G>(psi, cs, bb, row, a.lo, true, PH, tp, scb);
        issue_tile<G>(lam, cs, bb, row, a.lo, true, false, tl, scb);
    };
    double acc[3] = {0.0, 0.0, 0.0};  // mixer term, phase term (layer l), mixer term (layer l - 1)
    uint32_t t = blockIdx.x;
    if (t < tiles) issue(t, scs);
    cp_async_commit();
    for (int i = 0; t < tiles; ++i, t += gridDim.x) {
        const int b = i & 1;
        const uint8_t *sc = scs + ((size_t)b << T);
        const uint32_t base = tile_base32(t, row, a.lo, T);
        const uint32_t tn = t + gridDim.x;
        cp_async_wait_all();
        __syncthreads();
        V vp[NR], vl[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {  // dense buffers, consecutive lanes: no conflicts
            const uint32_t u = tile_elem<G, LD>(tid, r);
            vp[r] = tp[u];
            vl[r] = tl[u];
        }
        R term = 0, gterm = 0, term2 = 0;
        auto prefetch = [&]() {  // both buffers are read out: copy the next pair into them
            __syncthreads();
            if (tn < tiles) issue(tn, scs + ((size_t)(b ^ 1) << T));
            cp_async_commit();
        };
        // all of M_l undone on this tile: phase term, then D_l^dagger (registers
        // in mapping MP)
        auto undo_phase = [&](auto mp) {
            constexpr int MP = decltype(mp)::value;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int cst = sc[tile_elem<G, MP>(tid, r)];
                gterm += (R)cst * (vl[r].x * vp[r].y - vl[r].y * vp[r].x);
                const V ph = stab[cst];
                vp[r] = cmul(vp[r], ph);
                vl[r] = cmul(vl[r], ph);
            }
        };
        if constexpr (TOP) prefetch();  // the pair is in registers for good
        inv_round<G, LD, T>(vp, vl, active, a.c, a.S, term);
        if constexpr (TOP) {
            if constexpr (MODE == A_FUSED) {
                undo_phase(std::integral_constant<int, LD>{});
                inv_round<G, LD, T>(vp, vl, active, a.c2, a.S2, term2);
            }
        } else if (LOW) {
            exchange_pair<G, LD, 0>(vp, vl, tp, tl);
            inv_round<G, 0, T>(vp, vl, active, a.c, a.S, term);
            exchange_pair<G, 0, LC>(vp, vl, tp, tl);
            prefetch();
            inv_round<G, LC, LD>(vp, vl, active, a.c, a.S, term);
            if (PH) undo_phase(std::integral_constant<int, LC>{});
        } else if (MODE == A_FUSED) {
            exchange_pair<G, LD, LC>(vp, vl, tp, tl);
            inv_round<G, LC, LD>(vp, vl, active, a.c, a.S, term);
            undo_phase(std::integral_constant<int, LC>{});
            inv_round<G, LC, LD>(vp, vl, active, a.c2, a.S2, term2);
            exchange_pair<G, LC, LD>(vp, vl, tp, tl);
            prefetch();
            inv_round<G, LD, T>(vp, vl, active, a.c2, a.S2, term2);
        } else {
            exchange_pair<G, LD, LC>(vp, vl, tp, tl);
            prefetch();
            inv_round<G, LC, LD>(vp, vl, active, a.c, a.S, term);
        }
        V *pp = psi + (base + st_t);
        V *pl = lam + (base + st_t);
        uint32_t gs = gstride;
        asm volatile("" : "+l"(pp), "+l"(pl), "+r"(gs));  // keep the store addresses out of the load phase
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const uint32_t o = reg_off<SM, row>(r, gs);
            pp[o] = vp[r];
            pl[o] = vl[r];
        }
        acc[0] += (double)term;
        acc[1] += (double)gterm;
        acc[2] += (double)term2;
    }
    block_sum<3>(acc);
    if (threadIdx.x == 0) {
        const size_t slot = 2 * ((inst * a.p) * gridDim.x + blockIdx.x);
        a.partials[slot] += acc[0];
        a.partials[slot + 1] += acc[1];
        if (MODE == A_FUSED && a.partials2) a.partials2[slot] += acc[2];
    }
}

// ---------------------------------------------------------------------------
// Small n: the whole forward and reverse sweep of one instance per CTA, both
// states resident in shared memory.  tables: FP64 exp(-i gamma_l c) [p][m+1];
// coefs: (c, S) per layer.  out: [batch][1 + p][2] = (p_succ, norm), then
// (mixer sum, phase sum) per layer.
template <typename R>
__global__ void __launch_bounds__(PT) small_grad_kernel(const uint8_t *costs, int n, int m, int p, const double *tables,
                                                        const double *coefs, double *out) {
    using V = typename Cx<R>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t N = 1u << n;
    V *sp = reinterpret_cast<V *>(smem_raw);
    V *sl = sp + N;
    uint8_t *sc = reinterpret_cast<uint8_t *>(sl + N);
    const size_t inst = blockIdx.x;
    const uint8_t *cost = costs + (inst << n);
    double *o = out + inst * 2 * (1 + p);
    for (uint32_t x = threadIdx.x; x < N; x += PT) sc[x] = cost[x];
    const R amp = (R)(1.0 / sqrt((double)N));
    for (uint32_t x = threadIdx.x; x < N; x += PT) sp[x] = V{amp, (R)0};
    __syncthreads();
    for (int l = 0; l < p; ++l) {
        const double *tb = tables + 2 * (size_t)l * (m + 1);
        for (uint32_t x = threadIdx.x; x < N; x += PT) {
            const int cx = min((int)sc[x], m);
            const V ph{(R)tb[2 * cx], (R)tb[2 * cx + 1]};
            sp[x] = cmul(sp[x], ph);
        }
        const R c = (R)coefs[2 * l], S = (R)coefs[2 * l + 1];
        for (int j = 0; j < n; ++j) {
            __syncthreads();
            for (uint32_t g = threadIdx.x; g < N / 2; g += PT) {
                const uint32_t x0 = ((g >> j) << (j + 1)) | (g & ((1u << j) - 1u)), x1 = x0 | (1u << j);
                const V a = sp[x0], b = sp[x1];
                sp[x0] = V{fma(c, a.x, -S * b.y), fma(c, a.y, S * b.x)};
                sp[x1] = V{fma(c, b.x, -S * a.y), fma(c, b.y, S * a.x)};
            }
        }
        __syncthreads();
    }
    double acc[2] = {0.0, 0.0};
    for (uint32_t x = threadIdx.x; x < N; x += PT) {
        const V v = sp[x];
        const double w = (double)v.x * v.x + (double)v.y * v.y;
        acc[1] += w;
        const bool sol = sc[x] == 0;
        if (sol) acc[0] += w;
        sl[x] = sol ? v : V{(R)0, (R)0};
    }
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
        o[0] = acc[0];
        o[1] = acc[1];
    }
    for (int l = p - 1; l >= 0; --l) {
        const R c = (R)coefs[2 * l], S = (R)coefs[2 * l + 1];
        R term = 0;
        for (int j = 0; j < n; ++j) {
            __syncthreads();
            for (uint32_t g = threadIdx.x; g < N / 2; g += PT) {
                const uint32_t x0 = ((g >> j) << (j + 1)) | (g & ((1u << j) - 1u)), x1 = x0 | (1u << j);
                V a = sp[x0], b = sp[x1], la = sl[x0], lb = sl[x1];
                inv_pair(a, b, la, lb, c, S, term);
                sp[x0] = a;
                sp[x1] = b;
                sl[x0] = la;
                sl[x1] = lb;
            }
        }
        __syncthreads();
        const double *tb = tables + 2 * (size_t)l * (m + 1);
        R gterm = 0;
        for (uint32_t x = threadIdx.x; x < N; x += PT) {
            const int cst = min((int)sc[x], m);
            const V vp = sp[x], vl = sl[x];
            gterm += (R)cst * (vl.x * vp.y - vl.y * vp.x);
            const V ph{(R)tb[2 * cst], (R)(-tb[2 * cst + 1])};
            sp[x] = cmul(vp, ph);
            sl[x] = cmul(vl, ph);
        }
        double g2[2] = {(double)term, (double)gterm};
        block_sum<2>(g2);
        if (threadIdx.x == 0) {
            o[2 * (1 + l)] = g2[0];
            o[2 * (1 + l) + 1] = g2[1];
        }
    }
}

// Dynamic shared memory of a backward pass: the two tile buffers, then (low
// pass, m >= 0) two cost-byte buffers and the phase table.
template <typename R>
static size_t adj_smem(int m) {
    using G = AGeo<R>;
    size_t b = sizeof(typename G::V) * 2 * (size_t)G::TILE_ELEMS;
    if (m >= 0) b += 2 * (size_t(1) << G::T) + sizeof(typename G::V) * (size_t)(m < 255 ? 256 : m + 1);
    return b;
}

// Rows of a wide high group (complex64: 32 amplitudes, 256 B); complex128 rows
// of 16 are 256 B already and take no wide groups.
template <typename R>
constexpr int adj_wrow() {
    return sizeof(R) == 4 ? HIGH_ROW + 1 : HIGH_ROW;
}

template <typename R>
struct AdjKernels {
    using KF = void (*)(AdjArgs<R>, AdjTab<R, MAX_TABLE>);
    using KN = void (*)(AdjArgs<R>, AdjTab<R, 1>);
    static constexpr int W = adj_wrow<R>();
    KN low = adj_kernel<R, true, A_PLAIN, 1, HIGH_ROW, 1>;
    KF low_phase = adj_kernel<R, true, A_PHASE, MAX_TABLE, HIGH_ROW, 1>;
    // [wide][FULL: runtime mask, full, top bits only]
    KN high[2][3] = {{adj_kernel<R, false, A_PLAIN, 1, HIGH_ROW, 0>, adj_kernel<R, false, A_PLAIN, 1, HIGH_ROW, 1>,
                      adj_kernel<R, false, A_PLAIN, 1, HIGH_ROW, 2>},
                     {adj_kernel<R, false, A_PLAIN, 1, W, 0>, adj_kernel<R, false, A_PLAIN, 1, W, 1>,
                      adj_kernel<R, false, A_PLAIN, 1, W, 2>}};
    KF fused[2][3] = {{adj_kernel<R, false, A_FUSED, MAX_TABLE, HIGH_ROW, 0>,
                       adj_kernel<R, false, A_FUSED, MAX_TABLE, HIGH_ROW, 1>,
                       adj_kernel<R, false, A_FUSED, MAX_TABLE, HIGH_ROW, 2>},
                      {adj_kernel<R, false, A_FUSED, MAX_TABLE, W, 0>, adj_kernel<R, false, A_FUSED, MAX_TABLE, W, 1>,
                       adj_kernel<R, false, A_FUSED, MAX_TABLE, W, 2>}};
};

template <typename R>
static int adj_init(AdjKernels<R> **out) {
    static std::mutex mu;
    static int state[MAX_DEVICES] = {};  // per device: 0 = not yet, 1 = ok
    static AdjKernels<R> ks;
    const int dev = current_device_slot();
    if (dev < 0) return QAOA_ECUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (!state[dev]) {
        cudaError_t e = cudaFuncSetAttribute(ks.low, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)adj_smem<R>(-1));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ks.low_phase, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)adj_smem<R>(MAX_TABLE - 1));
        for (int w = 0; w < 2 && e == cudaSuccess; ++w)
            for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
                e = cudaFuncSetAttribute(ks.high[w][f], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)adj_smem<R>(-1));
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(ks.fused[w][f], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)adj_smem<R>(MAX_TABLE - 1));
            }
        const int small = (int)(2 * sizeof(typename Cx<R>::V) * (size_t(1) << Cx<R>::T) + (size_t(1) << Cx<R>::T));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(small_grad_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, small);
        if (e != cudaSuccess) return cuda_error(e, "adjoint kernel attributes");
        state[dev] = 1;
    }
    *out = &ks;
    return QAOA_OK;
}

template <typename R>
static int grad_passes(int batch, int n, const uint8_t *cost, int m, int p, const double *gamma, const double *beta,
                       int dtype, int flags, void *state, void *adj, double *d_scr, double *h_scr,
                       cudaStream_t stream, double *p_succ, double *dgamma, double *dbeta) {
    using V = typename AGeo<R>::V;
    AdjKernels<R> *ks = nullptr;
    int rc = adj_init<R>(&ks);
    if (rc) return rc;
    const int sign = (flags & QAOA_MIXER_RX2B) ? -1 : 1;
    // forward with the adjoint seed lam_p = P psi_p written by the last pass
    const int gxf = pass_grid_x(dtype, n, batch);
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    const uint64_t tiles = 1ull << (n - AGeo<R>::T);
    const int gxa = balanced_grid_x(di.sms * (sizeof(R) == 4 ? 2 : 1), batch, tiles);
    double *d_fpart = d_scr;                                  // batch * gxf * 2
    double *d_fres = d_fpart + (size_t)batch * gxf * 2;       // batch * 2
    double *d_apart = d_fres + (size_t)batch * 2;             // batch * p * gxa * 2
    double *d_ares = d_apart + (size_t)batch * p * gxa * 2;   // batch * p * 2
    EvolveReq r{batch, n, m, p, dtype, flags, cost, state, adj, gamma, beta, d_fres};
    if ((rc = evolve_device_impl(r, stream, d_fpart, gxf))) return rc;
    QAOA_CUDA_TRY(cudaMemsetAsync(d_apart, 0, (size_t)batch * p * gxa * 2 * sizeof(double), stream));
    Plan pl;
    if ((rc = make_plan_geo(n, AGeo<R>::T, 8, &pl, false, adj_wrow<R>() != HIGH_ROW))) return rc;
    std::vector<char> tbuf(sizeof(AdjTab<R, MAX_TABLE>));
    auto *tab = reinterpret_cast<AdjTab<R, MAX_TABLE> *>(tbuf.data());
    AdjTab<R, 1> none{};
    const std::vector<Launch> seq = make_adj_schedule(pl.n_passes, p);
    for (const Launch &L : seq) {
        const int l = L.la;
        const Pass &ps = pl.pass[L.pass];
        const double c = std::cos(beta[l]), S = sign * std::sin(beta[l]);
        AdjArgs<R> a;
        a.psi = reinterpret_cast<V *>(state);
        a.lam = reinterpret_cast<V *>(adj);
        a.cost = cost;
        a.partials = d_apart + (size_t)l * gxa * 2;
        a.partials2 = nullptr;
        a.n = n;
        a.m = m;
        a.p = p;
        a.c = (R)c;
        a.S = (R)S;
        a.c2 = (R)1;  // identity second half unless the pass fuses layer l - 1
        a.S2 = (R)0;
        a.tiles = tiles;
        if (L.mode != A_PLAIN) {
            for (int k = 0; k <= m; ++k) {  // D_l^dagger = exp(+i gamma_l C)
                tab->t[k].x = (R)std::cos(gamma[l] * k);
                tab->t[k].y = (R)std::sin(gamma[l] * k);
            }
        }
        if (L.mode == A_FUSED) {
            a.c2 = (R)std::cos(beta[l - 1]);
            a.S2 = (R)(sign * std::sin(beta[l - 1]));
            a.partials2 = d_apart + (size_t)(l - 1) * gxa * 2;
        }
        if (L.pass == 0) {
            a.row = AGeo<R>::T;
            a.lo = AGeo<R>::T;
            a.active = (1u << AGeo<R>::T) - 1u;
            if (L.mode == A_FUSED) return set_error(QAOA_ECUDA, "adjoint schedule: fused low pass");
            profile_before(K_ADJ_LOW, stream);
            if (L.mode == A_PHASE)
                ks->low_phase<<<dim3(gxa, batch), PT, adj_smem<R>(m), stream>>>(a, *tab);
            else
                ks->low<<<dim3(gxa, batch), PT, adj_smem<R>(-1), stream>>>(a, none);
            rc = profile_after(K_ADJ_LOW, stream);
        } else {
            a.row = ps.row;
            a.lo = ps.lo;
            a.active = ((1u << ps.bits) - 1u) << (pl.tile_bits - ps.bits);
            if (ps.row != HIGH_ROW && ps.row != adj_wrow<R>())
                return set_error(QAOA_ECUDA, "adjoint plan: rows of %d bits", ps.row);
            // the undone bits are the tile's top ps.bits; the load mapping holds
            // the top RB in registers
            const int wide = ps.row != HIGH_ROW ? 1 : 0;
            const int full = ps.bits == pl.tile_bits - ps.row ? 1 : (ps.bits <= AGeo<R>::RB ? 2 : 0);
            profile_before(K_ADJ_HIGH, stream);
            if (L.mode == A_PLAIN)
                ks->high[wide][full]<<<dim3(gxa, batch), PT, adj_smem<R>(-1), stream>>>(a, none);
            else  // A_FUSED, or A_PHASE as the fused kernel with an identity second layer
                ks->fused[wide][full]<<<dim3(gxa, batch), PT, adj_smem<R>(m), stream>>>(a, *tab);
            rc = profile_after(K_ADJ_HIGH, stream);
        }
        if (rc) return rc;
    }
    if ((rc = launch_reduce(d_apart, batch * p, gxa, 2, d_ares, stream))) return rc;
    QAOA_CUDA_TRY(cudaMemcpyAsync(h_scr, d_fres, (size_t)batch * 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaMemcpyAsync(h_scr + 2 * batch, d_ares, (size_t)batch * p * 2 * sizeof(double),
                                  cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    for (int b = 0; b < batch; ++b) {
        if (p_succ) p_succ[b] = h_scr[2 * b];
        for (int l = 0; l < p; ++l) {
            const double *g = h_scr + 2 * batch + 2 * ((size_t)b * p + l);
            dbeta[(size_t)b * p + l] = -2.0 * sign * g[0];
            dgamma[(size_t)b * p + l] = 2.0 * g[1];
        }
    }
    return QAOA_OK;
}

template <typename R>
static int grad_small(int batch, int n, const uint8_t *cost, int m, int p, const double *gamma, const double *beta,
                      int flags, double *d_scr, double *h_scr, cudaStream_t stream, double *p_succ, double *dgamma,
                      double *dbeta) {
    AdjKernels<R> *ks = nullptr;
    int rc = adj_init<R>(&ks);
    if (rc) return rc;
    const int sign = (flags & QAOA_MIXER_RX2B) ? -1 : 1;
    const size_t tab_n = (size_t)p * (m + 1);
    double *h_tab = h_scr;
    double *h_coef = h_tab + 2 * tab_n;
    for (int l = 0; l < p; ++l) {
        for (int k = 0; k <= m; ++k) {
            h_tab[2 * ((size_t)l * (m + 1) + k)] = std::cos(gamma[l] * k);
            h_tab[2 * ((size_t)l * (m + 1) + k) + 1] = -std::sin(gamma[l] * k);
        }
        h_coef[2 * l] = std::cos(beta[l]);
        h_coef[2 * l + 1] = sign * std::sin(beta[l]);
    }
    const size_t in_bytes = (2 * tab_n + 2 * (size_t)p) * sizeof(double);
    double *d_tab = d_scr, *d_coef = d_scr + 2 * tab_n;
    double *d_out = d_scr + 2 * tab_n + 2 * p;
    const size_t out_n = (size_t)batch * 2 * (1 + p);
    QAOA_CUDA_TRY(cudaMemcpyAsync(d_scr, h_scr, in_bytes, cudaMemcpyHostToDevice, stream));
    const size_t smem = 2 * sizeof(typename Cx<R>::V) * (size_t(1) << n) + (size_t(1) << n);
    profile_before(K_SMALL_N, stream);
    small_grad_kernel<R><<<batch, PT, smem, stream>>>(cost, n, m, p, d_tab, d_coef, d_out);
    if ((rc = profile_after(K_SMALL_N, stream))) return rc;
    double *h_out = h_scr + 2 * tab_n + 2 * p;
    QAOA_CUDA_TRY(cudaMemcpyAsync(h_out, d_out, out_n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    for (int b = 0; b < batch; ++b) {
        const double *o = h_out + (size_t)b * 2 * (1 + p);
        if (p_succ) p_succ[b] = o[0];
        for (int l = 0; l < p; ++l) {
            dbeta[(size_t)b * p + l] = -2.0 * sign * o[2 * (1 + l)];
            dgamma[(size_t)b * p + l] = 2.0 * o[2 * (1 + l) + 1];
        }
    }
    return QAOA_OK;
}

static int grad_common(int batch, int n, const uint8_t *cost, int m, int p, const double *gamma, const double *beta,
                       int dtype, int flags, void *state, void *adj, double *p_succ, double *dgamma, double *dbeta,
                       void *stream_) {
    if (batch < 1) return set_error(QAOA_EINVAL, "batch=%d", batch);
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", dtype);
    if (flags & ~QAOA_MIXER_RX2B)
        return set_error(QAOA_EINVAL, "flags=0x%x: the gradient takes the full state in native arithmetic", flags);
    const int nmax = dtype == QAOA_C64 ? QAOA_MAX_N : QAOA_MAX_N - 1;
    if (n < 1 || n > nmax) return set_error(QAOA_ERANGE, "n=%d outside [1, %d]", n, nmax);
    if (m < 0 || m > QAOA_MAX_M) return set_error(QAOA_ERANGE, "m=%d", m);
    if (p < 1) return set_error(QAOA_EINVAL, "gradient needs p >= 1 (p=%d)", p);
    if (!cost || !state || !adj || !gamma || !beta || !dgamma || !dbeta) return set_error(QAOA_EINVAL, "NULL argument");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l])) return set_error(QAOA_EINVAL, "angle %d not finite", l);
    m = table_top(m);  // from here m bounds the phase tables only
    cudaStream_t stream = (cudaStream_t)stream_;
    Scratch *sc = nullptr;
    int rc;
    if (n <= small_n_limit(dtype)) {
        const size_t words = 2 * (size_t)p * (m + 1) + 2 * (size_t)p + (size_t)batch * 2 * (1 + p) + 16;
        if ((rc = scratch_for(stream, words * sizeof(double), words * sizeof(double), &sc))) return rc;
        if (dtype == QAOA_C64)
            return grad_small<float>(batch, n, cost, m, p, gamma, beta, flags, (double *)sc->dev, (double *)sc->host,
                                     stream, p_succ, dgamma, dbeta);
        return grad_small<double>(batch, n, cost, m, p, gamma, beta, flags, (double *)sc->dev, (double *)sc->host,
                                  stream, p_succ, dgamma, dbeta);
    }
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    const int gxf = pass_grid_x(dtype, n, batch);
    const size_t gxa = (size_t)di.sms * 2 + 1;
    const size_t words = (size_t)batch * gxf * 2 + (size_t)batch * 2 + (size_t)batch * p * gxa * 2 +
                         (size_t)batch * p * 2 + 64;
    const size_t hwords = (size_t)batch * 2 + (size_t)batch * p * 2 + 16;
    if ((rc = scratch_for(stream, words * sizeof(double), hwords * sizeof(double), &sc))) return rc;
    if (dtype == QAOA_C64)
        return grad_passes<float>(batch, n, cost, m, p, gamma, beta, dtype, flags, state, adj, (double *)sc->dev,
                                  (double *)sc->host, stream, p_succ, dgamma, dbeta);
    return grad_passes<double>(batch, n, cost, m, p, gamma, beta, dtype, flags, state, adj, (double *)sc->dev,
                               (double *)sc->host, stream, p_succ, dgamma, dbeta);
}

}  // namespace qaoa

using namespace qaoa;

extern "C" int qaoa_grad(int n, const uint8_t *d_cost, int m, int p, const double *gamma, const double *beta, int dtype,
                         int flags, void *d_state, void *d_adj, double *p_succ, double *dgamma, double *dbeta,
                         void *stream) {
    return grad_common(1, n, d_cost, m, p, gamma, beta, dtype, flags, d_state, d_adj, p_succ, dgamma, dbeta, stream);
}

extern "C" int qaoa_grad_batch(int batch, int n, const uint8_t *d_costs, int m_max, int p, const double *gamma,
                               const double *beta, int dtype, int flags, void *d_states, void *d_adjs, double *p_succ,
                               double *dgamma, double *dbeta, void *stream) {
    return grad_common(batch, n, d_costs, m_max, p, gamma, beta, dtype, flags, d_states, d_adjs, p_succ, dgamma, dbeta,
                       stream);
}
