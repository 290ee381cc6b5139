// K2/K3/K4/K6: the QAOA layers U_B(beta) U_C(gamma) on a state in HBM.
//
//  * U_C(gamma) = diag(exp(-i gamma C(x))) (Eq. for U_C; Appendix A.3's
//    diagonalisation): C(x) takes at most m + 1 values, so the phase is a lookup
//    in a per-layer table T[c] (FP64 on the host, cast to the state's type),
//    fused into the load of the layer's first pass.
//  * U_B(beta) = prod_j [cos(beta) I + i sin(beta) X_j] (Appendix A.3): one
//    butterfly per qubit over the pairs (x, x xor 2^j).  The qubit factors
//    commute, so a layer is split into HBM passes over groups of qubits: the
//    low pass (tile bits = state bits [0, T)) and high passes over strided rows.
//  * p_succ = sum_{C(x)=0} |psi(x)|^2 and the norm (Def. of the success
//    probability): accumulated in the store of the last pass, per-block FP64
//    partials, then a fixed-order reduction (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "pass_common.cuh"
#include "qaoa_internal.cuh"

namespace qaoa {

template <typename R>
struct PassArgs {
    typename Cx<R>::V *state;  // instance 0; instance b at state + b 2^n
    typename Cx<R>::V *adj;    // nullable: receives P psi in the store
    const uint8_t *cost;
    double *partials;          // [batch][gridDim.x][2] when reduce
    int n, row, lo, m;
    uint32_t active;           // tile bits to butterfly
    int reduce;
    int ua1, ua2;              // butterfly forms of the two layers (fused: l, l+1)
    R A1, B1, A2, B2;
    uint64_t tiles;            // tiles per instance
};

template <typename R, int NT>
struct PhaseTab {
    typename Cx<R>::V t[NT];
};

// Pass modes (MODE_* in the internal header): INIT generates layer 0's state
// from the phase table, PHASE multiplies by a layer's phase at load, PLAIN only
// butterflies, FUSED butterflies layer l, applies the phase of layer l + 1 in
// the tile and butterflies layer l + 1 (the pass is the last of layer l and the
// first of layer l + 1; the qubit factors commute, so the group order
// alternates between layers).

// Mapping of the last round of a pass (its stores are coalesced too).
template <typename G, bool LOW>
struct LastLO {
    static constexpr int value = PassRounds<G, LOW>::LAST;
};

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// The rounds of one layer from the load mapping to the last mapping...  `hook`
// runs right after the last exchange (the tile buffer is free from then on).
template <typename G, bool LOW, bool UA, class Hook>
__device__ __forceinline__ void rounds_up(typename G::V *v, typename G::V *tile, uint32_t active, typename G::Real A,
                                          typename G::Real B, const Hook &hook) {
    using P = PassRounds<G, LOW>;
    mask_butterflies<G, UA, P::R0::LO, P::R0::MASK>(v, active, A, B);
    exchange<G, P::R0::LO, P::R1::LO>(v, tile);
    if constexpr (P::N == 2) hook();
    mask_butterflies<G, UA, P::R1::LO, P::R1::MASK>(v, active, A, B);
    if constexpr (P::N > 2) {
        exchange<G, P::R1::LO, P::R2::LO>(v, tile);
        if constexpr (P::N == 3) hook();
        mask_butterflies<G, UA, P::R2::LO, P::R2::MASK>(v, active, A, B);
    }
    if constexpr (P::N > 3) {
        exchange<G, P::R2::LO, P::R3::LO>(v, tile);
        hook();
        mask_butterflies<G, UA, P::R3::LO, P::R3::MASK>(v, active, A, B);
    }
}

// ... and back from the last mapping to the load mapping (same qubits).
template <typename G, bool LOW, bool UA, class Hook>
__device__ __forceinline__ void rounds_down(typename G::V *v, typename G::V *tile, uint32_t active,
                                            typename G::Real A, typename G::Real B, const Hook &hook) {
    using P = PassRounds<G, LOW>;
    if constexpr (P::N > 3) {
        mask_butterflies<G, UA, P::R3::LO, P::R3::MASK>(v, active, A, B);
        exchange<G, P::R3::LO, P::R2::LO>(v, tile);
    }
    if constexpr (P::N > 2) {
        mask_butterflies<G, UA, P::R2::LO, P::R2::MASK>(v, active, A, B);
        exchange<G, P::R2::LO, P::R1::LO>(v, tile);
    }
    mask_butterflies<G, UA, P::R1::LO, P::R1::MASK>(v, active, A, B);
    exchange<G, P::R1::LO, P::R0::LO>(v, tile);
    hook();
    mask_butterflies<G, UA, P::R0::LO, P::R0::MASK>(v, active, A, B);
}

// Halved state (low pass): tile element u with bit T-1 set is the mirror
// 2^(n-1) - 1 - x of the element x = u with that bit clear; its data and cost
// bytes land in reverse memory order at position 2^T - 1 - (u mod 2^(T-1)).
template <int T>
__host__ __device__ __forceinline__ constexpr uint32_t land(uint32_t u) {
    return (u >> (T - 1)) ? ((1u << T) - 1u - (u & ((1u << (T - 1)) - 1u))) : u;
}

// Stores the tile from mapping LO, fusing the p_succ / norm partials and the
// adjoint seed P psi when this is the evolution's last pass.  sp: the thread's
// first element; register r adds the state offset of tile element r << LO,
// i.e. its row part plus its group part times gstride = 2^lo (ROW: the
// tile's row bits).  In the halved state's mirror half (low pass) the offsets
// run downwards.  Indices inside one instance fit in 32 bits (n <= 32).
// sc: the tile's cost bytes in shared memory, indexed by tile element (by
// landing position when Z2).
// |v|^2 and a zero amplitude for each arithmetic (double-float: in FP64).
__device__ __forceinline__ float amp_prob(const float2 &v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double amp_prob(const double2 &v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double amp_prob(const float4 &v) {
    const double re = (double)v.x + (double)v.y, im = (double)v.z + (double)v.w;
    return re * re + im * im;
}
template <typename V>
__device__ __forceinline__ V zero_amp() {
    V z;
    memset(&z, 0, sizeof z);
    return z;
}

// A double-float evolution keeps its state as (re.hi, re.lo, im.hi, im.lo)
// floats in the complex128 buffer; its last pass (always a reducing one)
// writes FP64 (re, im) back, 16 bytes for 16 bytes.
template <typename R>
constexpr bool is_df() {
    return std::is_same<R, dfloat>::value;
}

template <typename R, int LO, int ROW, bool Z2, bool RED, bool PADC>
__device__ __forceinline__ void store_tile(const typename Cx<R>::V *v, typename Cx<R>::V *sp, const uint8_t *sc,
                                           typename Cx<R>::V *sa, uint32_t gstride, bool mirror, bool reduce,
                                           double acc[2]) {
    using V = typename Cx<R>::V;
    using P = decltype(amp_prob(v[0]));  // probability accumulation type
    constexpr int NR = Cx<R>::NR;
    // Opaque to the compiler: otherwise it keeps the load phase's 32 offsets
    // live across the whole tile to reuse them here.
    asm volatile("" : "+l"(sp), "+r"(gstride));
    auto off = [&](int r) -> int64_t {
        const uint32_t u = (uint32_t)r << LO;
        const uint32_t o = (u & ((1u << ROW) - 1u)) + (u >> ROW) * gstride;
        return (Z2 && mirror) ? -(int64_t)o : (int64_t)o;
    };
    if (is_df<R>() && RED && reduce) {  // the evolution's last pass: FP64 out
        double2 *sd = reinterpret_cast<double2 *>(sp);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float4 w = *reinterpret_cast<const float4 *>(&v[r]);
            sd[off(r)] = make_double2((double)w.x + (double)w.y, (double)w.z + (double)w.w);
        }
    } else if constexpr (is_df<R>()) {  // pairs renormalised between passes
#pragma unroll
        for (int r = 0; r < NR; ++r) sp[off(r)] = df_renorm(v[r]);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) sp[off(r)] = v[r];
    }
    if (RED && reduce) {
        // The thread's NR probabilities are summed pairwise in P (FP32 for
        // complex64: relative error at most 7 u = 4.2e-7 with the two roundings
        // of each |v|^2), then everything above the thread in FP64.
        PairwiseSum<NR, P> ps, nm;
        const uint32_t tid = threadIdx.x;
        const uint32_t cb = PADC ? cost_base<Cx<R>, LO>(tid) : 0u;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const P w = amp_prob(v[r]);
            nm.add(r, w);
            const uint32_t u = tile_elem<Cx<R>, LO>(tid, r);
            const bool sol = sc[PADC ? cb + Cx<R>::cidx((uint32_t)r << LO) : (Z2 ? land<Cx<R>::T>(u) : u)] == 0;
            ps.add(r, sol ? w : P(0));
            if (sa) sa[off(r)] = sol ? v[r] : zero_amp<V>();
        }
        acc[0] += (double)ps.total();
        acc[1] += (double)nm.total();
    }
}

// Halved state, low pass: the tile is the half-tile [base, base + H) and its
// mirror block [mbase, mbase + H), H = 2^(T-1), each copied in memory order
// (the mirror block lands at positions [H, 2H)).
template <typename R>
__device__ __forceinline__ void issue_tile_z2(const typename Cx<R>::V *st, const uint8_t *cs, uint32_t base,
                                              uint32_t mbase, bool state, bool cost, typename Cx<R>::V *buf,
                                              uint8_t *sc) {
    using V = typename Cx<R>::V;
    constexpr int T = Cx<R>::T;
    constexpr int EPC = 16 / (int)sizeof(V);
    constexpr int NT = Cx<R>::PT;
    constexpr int NCH = (1 << T) / EPC / NT;
    constexpr int CCH = (1 << T) / 16 / NT;
    constexpr uint32_t HC = (1u << (T - 1)) / 16;  // cost chunks per half
    const uint32_t tid = threadIdx.x;
    if (state) {
        char *dst = reinterpret_cast<char *>(buf) + 16 * tid;
        const V *reg = st + base + EPC * tid;
        const V *mir = st + mbase + EPC * tid;
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const V *src = j < NCH / 2 ? reg + (size_t)EPC * NT * j : mir + (size_t)EPC * NT * (j - NCH / 2);
            cp_async16(dst + (size_t)16 * NT * j, src);
        }
    }
    if (cost) {
#pragma unroll
        for (int j = 0; j < CCH; ++j) {
            const uint32_t q = tid + NT * j;
            const uint8_t *src = q < HC ? cs + base + 16 * q : cs + mbase + 16 * (q - HC);
            cp_async16(sc + 16 * q, src);
        }
    }
}

// Early landing (complex64 fused high passes): the next tile's elements
// u < EARLY_ELEMS and all its cost bytes are copied into buffers of their own
// right after the current tile's first exchange, i.e. about half a tile of
// compute before the tile buffer frees at the last exchange and takes the
// rest.  In the load mapping u = tid + (r << LOAD), so those elements are
// exactly registers r < EARLY_ELEMS >> LOAD (12 of 32), and every thread's
// copy chunks j < EARLY_ELEMS / (2 PT) (6 of 16): both splits are compile-time.
// 24 KiB more per CTA (108.5 KiB), still two CTAs per SM.
constexpr int EARLY_ELEMS = 3072;
template <typename R, bool LOW, int MODE, int NB>
__host__ __device__ constexpr bool early_landing() {
    return !LOW && MODE == MODE_FUSED && NB == 1 && std::is_same<R, float>::value;
}

// NB = 1: one tile buffer per CTA, two CTAs per SM; the next tile's copies
// start once the current tile's last exchange is read out.  NB = 3: three tile
// (and cost) buffers, one CTA per SM; tile i + 2's copies are issued when tile
// i starts, so two tiles are always in flight while one is computed (a
// cp.async commit-group pipeline: wait_group 2 completes the oldest).
template <typename R, bool LOW, int MODE, bool UA1, bool UA2, bool Z2, bool RED, int HROW, bool FULL, int NB>
__device__ __forceinline__ void pass_tiles(const PassArgs<R> &a, const typename Cx<R>::V *stab,
                                           typename Cx<R>::V *tiles_buf, uint8_t *scs, typename Cx<R>::V *ebuf) {
    using G = Cx<R>;
    using V = typename G::V;
    constexpr int T = G::T, NR = G::NR;
    constexpr int LD = G::LOAD;                // first round's mapping
    constexpr int LC = LastLO<G, LOW>::value;  // last round's mapping
    const uint32_t tid = threadIdx.x;
    const size_t inst = blockIdx.y;
    V *st = a.state + (inst << a.n);
    V *adj = a.adj ? a.adj + (inst << a.n) : nullptr;
    const uint8_t *cs = a.cost + (inst << a.n);
    // Only the evolution's last pass reduces (a plain pass, or the initial one
    // when p = 0); RED compiles that path in.
    const bool red = RED && a.reduce;
    const bool need_c = MODE != MODE_PLAIN || red;
    constexpr int row = LOW ? T : HROW;  // contiguous tile bits
    // FULL: every group bit of the tile is butterflied (a compile-time mask, so
    // the stages are straight-line code); otherwise the pass's runtime mask
    // (a last group that re-covers mixed bits, or no butterflies when p = 0).
    constexpr uint32_t full_mask = ((1u << T) - 1u) & ~(LOW ? 0u : (1u << row) - 1u);
    const uint32_t active = FULL ? full_mask : a.active;
    const bool need_s = MODE != MODE_INIT;
    // Stores go straight from registers: thread pointer + the register's offset.
    static_assert(!Z2 || (LOW && MODE != MODE_FUSED), "the halved state changes the low pass only");
    // State indices of one instance fit in 32 bits (n <= 32).
    const uint32_t ld_t = elem_offset32(tile_elem<G, LD>(tid, 0), row, a.lo);
    const uint32_t st_t = elem_offset32(tile_elem<G, LC>(tid, 0), row, a.lo);
    const uint32_t gstride = LOW ? 0u : (1u << a.lo);
    // halved state: the mirror of element x of the stored half is M - x
    const uint32_t M = (uint32_t)((1ull << a.n) - 1);
    constexpr uint32_t H = 1u << (T - 1);
    const uint32_t z_u0 = tile_elem<G, LC>(tid, 0);  // its bit T - 1 is a thread bit in every store mapping
    const bool z_mir = Z2 && (z_u0 >> (T - 1));
    auto base_of = [&](uint32_t tt) { return Z2 ? (tt << (T - 1)) : tile_base32(tt, row, a.lo, T); };
    auto issue = [&](uint32_t tt, V *tb, uint8_t *scb) {
        const uint32_t bb = base_of(tt);
        if (Z2)
            issue_tile_z2<R>(st, cs, bb, M - bb - (H - 1), need_s, need_c, tb, scb);
        else
            issue_tile<Cx<R>, !LOW>(st, cs, bb, row, a.lo, need_s, need_c, tb, scb);
    };
    auto tbuf = [&](int b) { return tiles_buf + (size_t)b * G::TILE_ELEMS; };
    auto cbuf = [&](int b) { return scs + (size_t)b * G::CS_BYTES; };
    constexpr bool EARLY = early_landing<R, LOW, MODE, NB>();
    constexpr int JE = EARLY_ELEMS / ((16 / (int)sizeof(V)) * G::PT);  // early copy chunks per thread
    constexpr int RE = EARLY_ELEMS >> LD;                              // early load-mapping registers
    static_assert(!EARLY || ((RE << LD) == EARLY_ELEMS && JE * (16 / (int)sizeof(V)) * G::PT == EARLY_ELEMS),
                  "the early part must be whole registers and whole copy chunks");
    auto issue_early = [&](uint32_t tt, uint8_t *scb) {  // elements below EARLY_ELEMS and the cost bytes
        if constexpr (EARLY)
            issue_tile<Cx<R>, true, 0, JE>(st, cs, base_of(tt), row, a.lo, true, true, ebuf, scb);
    };
    auto issue_late = [&](uint32_t tt, V *tb) {  // the other elements, into the tile buffer
        if constexpr (EARLY)
            issue_tile<Cx<R>, true, JE, -1>(st, cs, base_of(tt), row, a.lo, true, false, tb, nullptr);
    };
    double acc[2] = {0.0, 0.0};  // p_succ, norm
    const uint32_t tiles = (uint32_t)a.tiles;
    // High passes that read both the state and the cost bytes take tiles in
    // groups of GT = 64 B / (cost bytes per row): tiles GT q .. GT q + GT - 1,
    // q = blockIdx.x + k gridDim.x.  Their rows are neighbours in memory, so the
    // cost bytes of GT rows (one 64-byte DRAM burst) are fetched once and the
    // group's later tiles find them in L2.  (The initial pass reads no state
    // and keeps the plain order, in which concurrent tiles write neighbouring
    // rows.)
    constexpr uint32_t GT = (LOW || MODE == MODE_INIT) ? 1u : (row >= 6 ? 1u : 64u >> row);
    const bool grouped = GT > 1 && tiles % GT == 0;
    auto tile_at = [&](uint32_t i) -> uint32_t {
        return grouped ? GT * (blockIdx.x + (i / GT) * gridDim.x) + (i % GT) : blockIdx.x + i * gridDim.x;
    };
    uint32_t t = tile_at(0);
    if (t < tiles) {
        if constexpr (EARLY) {
            issue_early(t, cbuf(0));
            issue_late(t, tbuf(0));
        } else {
            issue(t, tbuf(0), cbuf(0));
        }
    }
    cp_async_commit();
    if (NB == 3) {
        const uint32_t t1 = tile_at(1);
        if (t1 < tiles) issue(t1, tbuf(1), cbuf(1));
        cp_async_commit();
    }
    for (uint32_t i = 0; t < tiles; ++i, t = tile_at(i)) {
        const int b = NB == 3 ? (int)(i % 3u) : (int)(i & 1u);
        V *tile = NB == 3 ? tbuf(b) : tbuf(0);
        uint8_t *sc = cbuf(b);
        const uint32_t base = base_of(t);
        const uint32_t tn = tile_at(i + 1);
        // NB = 1: once the tile's last exchange is read out the buffer is free:
        // copy the next tile into it (and its cost bytes into the other cost
        // buffer) while this tile finishes its last round and its stores.
        auto prefetch = [&]() {
            if constexpr (NB == 1) {
                __syncthreads();
                if (tn < tiles) {
                    if constexpr (EARLY)
                        issue_late(tn, tbuf(0));
                    else
                        issue(tn, tbuf(0), cbuf(b ^ 1));
                }
                cp_async_commit();
            }
        };
        // EARLY: after the first exchange every thread has read its registers out
        // of the early buffer, and the other cost buffer held the previous tile's
        auto early_hook = [&]() {
            if constexpr (EARLY) {
                if (tn < tiles) issue_early(tn, cbuf(b ^ 1));
                cp_async_commit();
            }
        };
        if constexpr (NB == 3) {
            // every thread is done with tile i - 1, whose buffers take tile i + 2
            __syncthreads();
            const uint32_t t2 = tile_at(i + 2);
            const int b2 = (int)((i + 2) % 3u);
            if (t2 < tiles) issue(t2, tbuf(b2), cbuf(b2));
            cp_async_commit();
            asm volatile("cp.async.wait_group 2;\n" ::: "memory");  // tile i's copies are done
        } else {
            cp_async_wait_all();  // this tile's copies are done
        }
        __syncthreads();
        V v[NR];
        const uint32_t cbl = LOW ? 0u : cost_base<G, LD>(tid);  // high passes: padded cost bytes
#pragma unroll
        for (int r = 0; r < NR; ++r) {  // load mapping on the dense buffer: consecutive lanes, no conflicts
            const uint32_t u0 = tile_elem<G, LD>(tid, r);
            const uint32_t u = Z2 ? land<T>(u0) : u0;
            const uint8_t c = LOW ? sc[u] : sc[cbl + G::cidx((uint32_t)r << LD)];
            if (MODE == MODE_INIT)
                v[r] = stab[c];
            else if (MODE == MODE_PHASE)
                v[r] = cmul(tile[u], stab[c]);
            else
                v[r] = (EARLY && r < RE) ? ebuf[u] : tile[u];
        }
        if (MODE == MODE_FUSED) {
            rounds_up<G, LOW, UA1>(v, tile, active, a.A1, a.B1, early_hook);
            const uint32_t cb = cost_base<G, LC>(tid);
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = cmul(v[r], stab[sc[cb + G::cidx((uint32_t)r << LC)]]);
            rounds_down<G, LOW, UA2>(v, tile, active, a.A2, a.B2, prefetch);
            store_tile<R, LD, row, false, false, !LOW>(v, st + (base + ld_t), sc, nullptr, gstride, false, false, acc);
        } else {
            rounds_up<G, LOW, UA1>(v, tile, active, a.A1, a.B1, prefetch);
            if (Z2) {  // the mirror half stores in descending order
                const uint32_t ul0 = z_u0 & (H - 1);
                V *sp = z_mir ? st + (M - base - ul0) : st + (base + ul0);
                store_tile<R, LC, row, true, RED, false>(v, sp, sc, nullptr, gstride, z_mir, red, acc);
            } else {
                store_tile<R, LC, row, false, RED, !LOW>(v, st + (base + st_t), sc, adj ? adj + (base + st_t) : nullptr,
                                                   gstride, false, red, acc);
            }
        }
    }
    if (red) {
        block_sum<2, G::PT>(acc);
        if (threadIdx.x == 0) {
            double *out = a.partials + 2 * (inst * gridDim.x + blockIdx.x);
            out[0] = acc[0];
            out[1] = acc[1];
        }
    }
}

// Shared-memory phase table length: at least 256 entries (any uint8 cost
// indexes inside it), a multiple of 16 so what follows stays aligned.
__host__ __device__ __forceinline__ int table_entries(int m) {
    const int e = m < 255 ? 256 : m + 1;
    return (e + 15) & ~15;
}

// Persistent over tiles.  NB = 1: two CTAs per SM, one (padded) tile buffer
// and two cost-byte buffers each; NB = 3: one CTA per SM, three of each.  Then
// the phase table.  Cost bytes are padded in high passes.
// UA1 / UA2: butterfly forms (A = 1 or B = 1) of the pass's one or two layers,
// chosen on the host per layer.
template <typename R, bool LOW, int MODE, bool UA1, bool UA2, int NT, bool Z2 = false, bool RED = false,
          int HROW = HIGH_ROW, bool FULL = true, int NB = 1>
__global__ void __launch_bounds__(Cx<R>::PT, NB == 3 ? 1 : 2) pass_kernel(const __grid_constant__ PassArgs<R> a,
                                                                          const __grid_constant__ PhaseTab<R, NT> tab) {
    using V = typename Cx<R>::V;
    constexpr int T = Cx<R>::T;
    constexpr int NCB = NB == 3 ? 3 : 2;  // cost buffers
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tile = reinterpret_cast<V *>(smem_raw);
    uint8_t *scs = reinterpret_cast<uint8_t *>(tile + (size_t)NB * Cx<R>::TILE_ELEMS);
    constexpr bool EARLY = early_landing<R, LOW, MODE, NB>();
    V *ebuf = EARLY ? reinterpret_cast<V *>(scs + (size_t)NCB * Cx<R>::CS_BYTES) : nullptr;
    V *stab = reinterpret_cast<V *>(scs + (size_t)NCB * Cx<R>::CS_BYTES + (EARLY ? EARLY_ELEMS * sizeof(V) : 0));
    if (MODE != MODE_PLAIN) {  // 256 entries at least: any uint8 cost indexes inside the table
        for (int i = threadIdx.x; i < 256 || i <= a.m; i += Cx<R>::PT) stab[i] = i <= a.m ? tab.t[i] : zero_amp<V>();
        __syncthreads();
    }
    pass_tiles<R, LOW, MODE, UA1, UA2, Z2, RED, HROW, FULL, NB>(a, stab, tile, scs, ebuf);
}

// Fixed-order reduction of per-block partials: out[b][k] = sum_j part[b][j][k].
__global__ void __launch_bounds__(PT) reduce_partials_kernel(const double *part, int nblk, int nv, double *out) {
    const size_t b = blockIdx.x;
    double x[4] = {0, 0, 0, 0};
    for (int j = threadIdx.x; j < nblk; j += PT)
        for (int k = 0; k < nv; ++k) x[k] += part[(b * nblk + j) * nv + k];
    block_sum<4>(x);
    if (threadIdx.x == 0)
        for (int k = 0; k < nv; ++k) out[b * nv + k] = x[k];
}

int launch_reduce(const double *part, int groups, int nblk, int nv, double *out, cudaStream_t stream) {
    profile_before(K_REDUCE, stream);
    reduce_partials_kernel<<<groups, PT, 0, stream>>>(part, nblk, nv, out);
    return profile_after(K_REDUCE, stream);
}

// Standalone p_succ / norm of a state (Def. of the success probability).
template <typename R>
__global__ void __launch_bounds__(PT) psucc_kernel(const typename Cx<R>::V *st, const uint8_t *cs, int n,
                                                   double *partials) {
    // elements per thread per chunk, summed pairwise in R (complex64: FP32,
    // relative error at most 7 u = 4.2e-7); chunks and threads in FP64
    constexpr int CH = 32;
    const uint64_t N = 1ull << n;
    const uint64_t chunk = (uint64_t)PT * CH;
    double acc[2] = {0.0, 0.0};
    for (uint64_t c0 = (uint64_t)blockIdx.x * chunk; c0 < N; c0 += (uint64_t)gridDim.x * chunk) {
        PairwiseSum<CH, R> ps, nm;
#pragma unroll
        for (int r = 0; r < CH; ++r) {
            const uint64_t g = c0 + (uint64_t)r * PT + threadIdx.x;
            R w = 0, wsol = 0;
            if (g < N) {
                const typename Cx<R>::V v = st[g];
                w = v.x * v.x + v.y * v.y;
                wsol = cs[g] == 0 ? w : R(0);
            }
            nm.add(r, w);
            ps.add(r, wsol);
        }
        acc[0] += (double)ps.total();
        acc[1] += (double)nm.total();
    }
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = acc[0];
        partials[2 * blockIdx.x + 1] = acc[1];
    }
}

// ---------------------------------------------------------------------------
// K6: whole evolution of one small instance per CTA, state resident in shared
// memory.  Tables are FP64 complex [p][m+1] and coefficients [p][4]
// (A, B, unit_a, unused) in device memory.
template <typename R>
__device__ __forceinline__ void smem_butterfly_pass(typename Cx<R>::V *s, int n, int j, int two, R A, R B,
                                                    bool ua) {
    using V = typename Cx<R>::V;
    const uint32_t groups = 1u << (n - 1 - two);
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        if (two) {
            const uint32_t x0 = ((g >> j) << (j + 2)) | (g & ((1u << j) - 1u));
            const uint32_t h1 = 1u << j, h2 = 2u << j;
            V a = s[x0], b = s[x0 | h1], c = s[x0 | h2], d = s[x0 | h1 | h2];
            if (ua) {
                bfly<true>(a, b, A, B);
                bfly<true>(c, d, A, B);
                bfly<true>(a, c, A, B);
                bfly<true>(b, d, A, B);
            } else {
                bfly<false>(a, b, A, B);
                bfly<false>(c, d, A, B);
                bfly<false>(a, c, A, B);
                bfly<false>(b, d, A, B);
            }
            s[x0] = a;
            s[x0 | h1] = b;
            s[x0 | h2] = c;
            s[x0 | h1 | h2] = d;
        } else {
            const uint32_t x0 = ((g >> j) << (j + 1)) | (g & ((1u << j) - 1u));
            V a = s[x0], b = s[x0 | (1u << j)];
            if (ua)
                bfly<true>(a, b, A, B);
            else
                bfly<false>(a, b, A, B);
            s[x0] = a;
            s[x0 | (1u << j)] = b;
        }
    }
}

// Device conversions of FP64 inputs to each arithmetic (double-float: the
// nearest float, then the nearest float to the remainder).
template <typename R>
__device__ __forceinline__ R real_dev(double x) {
    if constexpr (is_df<R>()) {
        const float hi = __double2float_rn(x);
        return dfloat{hi, __double2float_rn(x - (double)hi)};
    } else {
        return (R)x;
    }
}
template <typename R>
__device__ __forceinline__ typename Cx<R>::V amp_dev(double re, double im) {
    if constexpr (is_df<R>()) {
        const dfloat r = real_dev<dfloat>(re), i = real_dev<dfloat>(im);
        return make_float4(r.hi, r.lo, i.hi, i.lo);
    } else {
        typename Cx<R>::V z;
        z.x = (R)re;
        z.y = (R)im;
        return z;
    }
}

// One CTA per job: the whole evolution in shared memory.  complex128 runs in
// FP64, or with QAOA_DF64 in double-float arithmetic (R = dfloat: float4
// amplitudes in shared memory, FP64 (re, im) written out).
template <typename R>
__global__ void __launch_bounds__(PT) small_kernel(const SmallJob *jobs, const double *tables, const double *coefs,
                                                   int max_n) {
    using V = typename Cx<R>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmallJob jb = jobs[blockIdx.x];
    const int n = jb.n;
    const uint32_t N = 1u << n;
    V *s = reinterpret_cast<V *>(smem_raw);
    V *stab = s + (1u << max_n);
    uint8_t *sc = reinterpret_cast<uint8_t *>(stab + MAX_TABLE);
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) sc[x] = jb.cost[x];
    for (int l = 0; l < jb.p; ++l) {
        const double *tb = tables + 2 * ((size_t)jb.table_off + (size_t)l * (jb.m + 1));
        __syncthreads();
        for (int c = threadIdx.x; c <= jb.m; c += blockDim.x) stab[c] = amp_dev<R>(tb[2 * c], tb[2 * c + 1]);
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) s[x] = l == 0 ? stab[sc[x]] : cmul(s[x], stab[sc[x]]);
        const double *cf = coefs + 4 * ((size_t)jb.coef_off + l);
        const R A = real_dev<R>(cf[0]), B = real_dev<R>(cf[1]);
        const bool ua = cf[2] != 0.0;
        for (int j = 0; j < n; j += 2) {
            __syncthreads();
            smem_butterfly_pass<R>(s, n, j, (j + 1 < n) ? 1 : 0, A, B, ua);
        }
    }
    if (jb.p == 0) {  // |+>: the table of "layer 0" holds the amplitude
        const double *tb = tables + 2 * (size_t)jb.table_off;
        const V z = amp_dev<R>(tb[0], tb[1]);
        for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) s[x] = z;
    }
    __syncthreads();
    double acc[2] = {0.0, 0.0};
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
        const V v = s[x];
        double w;
        if constexpr (is_df<R>()) {
            w = amp_prob(v);
            if (jb.state)
                reinterpret_cast<double2 *>(jb.state)[x] =
                    make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
        } else {
            w = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            if (jb.state) reinterpret_cast<V *>(jb.state)[x] = v;
        }
        acc[1] += w;
        if (sc[x] == 0) acc[0] += w;
    }
    block_sum<2>(acc);
    if (threadIdx.x == 0 && jb.result) {
        jb.result[0] = acc[0];
        jb.result[1] = acc[1];
    }
}

int small_n_limit(int dtype) { return dtype == QAOA_C64 ? Cx<float>::T : Cx<double>::T; }
int small_n_pack_limit(int dtype) { return dtype == QAOA_C64 ? 14 : 13; }

static size_t small_smem(int dtype, int max_n) {
    const size_t es = dtype == QAOA_C64 ? sizeof(float2) : sizeof(double2);
    return es * ((size_t(1) << max_n) + MAX_TABLE) + (size_t(1) << max_n);
}

int launch_small_batch(int dtype, int n_jobs, const SmallJob *d_jobs, const double *d_tables, const double *d_coefs,
                       int max_n, int flags, cudaStream_t stream) {
    const size_t smem = small_smem(dtype, max_n);
    {
        static std::mutex mu;
        static int state[MAX_DEVICES] = {};  // per device: 0 = not yet, 1 = ok
        const int dev = current_device_slot();
        if (dev < 0) return QAOA_ECUDA;
        std::lock_guard<std::mutex> lk(mu);
        if (!state[dev]) {
            const int big = (int)small_smem(QAOA_C128, small_n_pack_limit(QAOA_C128));
            cudaError_t e = cudaFuncSetAttribute(small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)small_smem(QAOA_C64, small_n_pack_limit(QAOA_C64)));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(small_kernel<dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
            if (e != cudaSuccess) return cuda_error(e, "small_kernel attributes");
            state[dev] = 1;
        }
    }
    profile_before(K_SMALL_N, stream);
    if (dtype == QAOA_C64)
        small_kernel<float><<<n_jobs, PT, smem, stream>>>(d_jobs, d_tables, d_coefs, max_n);
    else if (flags & QAOA_DF64)
        small_kernel<dfloat><<<n_jobs, PT, smem, stream>>>(d_jobs, d_tables, d_coefs, max_n);
    else
        small_kernel<double><<<n_jobs, PT, smem, stream>>>(d_jobs, d_tables, d_coefs, max_n);
    return profile_after(K_SMALL_N, stream);
}

// ---------------------------------------------------------------------------
// Host side of the multi-pass evolution.

// Dynamic shared memory of a pass: the tile buffer, two cost-byte buffers and
// the phase table (modes that apply a phase).
template <typename R>
static size_t pass_smem(bool phase, int m, int nb = 1, bool early = false) {
    return sizeof(typename Cx<R>::V) * Cx<R>::TILE_ELEMS * (size_t)nb + (nb == 3 ? 3 : 2) * (size_t)Cx<R>::CS_BYTES +
           (early ? sizeof(typename Cx<R>::V) * EARLY_ELEMS : 0) +
           (phase ? sizeof(typename Cx<R>::V) * table_entries(m) : 0);
}

using KPtr = const void *;

// The kernels of one kind of high pass: rows of HROW bits; FULL: every group
// bit is butterflied.  [ua1] for init / plain, [ua1][ua2] for fused.
template <typename R, int HROW, bool FULL>
struct HighSet {
    using Full = PhaseTab<R, MAX_TABLE>;
    using None = PhaseTab<R, 1>;
    void (*init[2])(PassArgs<R>, Full) = {pass_kernel<R, false, MODE_INIT, false, false, MAX_TABLE, false, false, HROW, FULL>,
                                          pass_kernel<R, false, MODE_INIT, true, false, MAX_TABLE, false, false, HROW, FULL>};
    void (*plain[2])(PassArgs<R>, None) = {pass_kernel<R, false, MODE_PLAIN, false, false, 1, false, false, HROW, FULL>,
                                           pass_kernel<R, false, MODE_PLAIN, true, false, 1, false, false, HROW, FULL>};
    void (*plain_red[2])(PassArgs<R>, None) = {pass_kernel<R, false, MODE_PLAIN, false, false, 1, false, true, HROW, FULL>,
                                               pass_kernel<R, false, MODE_PLAIN, true, false, 1, false, true, HROW, FULL>};
    void (*fused[2][2])(PassArgs<R>, Full) = {
        {pass_kernel<R, false, MODE_FUSED, false, false, MAX_TABLE, false, false, HROW, FULL>,
         pass_kernel<R, false, MODE_FUSED, false, true, MAX_TABLE, false, false, HROW, FULL>},
        {pass_kernel<R, false, MODE_FUSED, true, false, MAX_TABLE, false, false, HROW, FULL>,
         pass_kernel<R, false, MODE_FUSED, true, true, MAX_TABLE, false, false, HROW, FULL>}};
    void all(std::vector<KPtr> &ks) const {
        for (int i = 0; i < 2; ++i) {
            ks.push_back((KPtr)init[i]);
            ks.push_back((KPtr)plain[i]);
            ks.push_back((KPtr)plain_red[i]);
            for (int j = 0; j < 2; ++j) ks.push_back((KPtr)fused[i][j]);
        }
    }
};

// The kernels of the low pass (Z2: the halved state's mirror variant; NB:
// tile buffers per CTA); all butterfly every tile bit, except init0 (p = 0:
// the initial state alone).
template <typename R, bool Z2, int NB = 1>
struct LowSet {
    using Full = PhaseTab<R, MAX_TABLE>;
    using None = PhaseTab<R, 1>;
    void (*init[2])(PassArgs<R>, Full) = {pass_kernel<R, true, MODE_INIT, false, false, MAX_TABLE, Z2, true, HIGH_ROW, true, NB>,
                                          pass_kernel<R, true, MODE_INIT, true, false, MAX_TABLE, Z2, true, HIGH_ROW, true, NB>};
    void (*init0)(PassArgs<R>, Full) = pass_kernel<R, true, MODE_INIT, true, false, MAX_TABLE, Z2, true, HIGH_ROW, false, NB>;
    void (*phase[2])(PassArgs<R>, Full) = {pass_kernel<R, true, MODE_PHASE, false, false, MAX_TABLE, Z2, false, HIGH_ROW, true, NB>,
                                           pass_kernel<R, true, MODE_PHASE, true, false, MAX_TABLE, Z2, false, HIGH_ROW, true, NB>};
    void (*plain[2])(PassArgs<R>, None) = {pass_kernel<R, true, MODE_PLAIN, false, false, 1, Z2, false, HIGH_ROW, true, NB>,
                                           pass_kernel<R, true, MODE_PLAIN, true, false, 1, Z2, false, HIGH_ROW, true, NB>};
    void (*plain_red[2])(PassArgs<R>, None) = {pass_kernel<R, true, MODE_PLAIN, false, false, 1, Z2, true, HIGH_ROW, true, NB>,
                                               pass_kernel<R, true, MODE_PLAIN, true, false, 1, Z2, true, HIGH_ROW, true, NB>};
    void all(std::vector<KPtr> &ks) const {
        ks.push_back((KPtr)init0);
        for (int i = 0; i < 2; ++i) {
            ks.push_back((KPtr)init[i]);
            ks.push_back((KPtr)phase[i]);
            ks.push_back((KPtr)plain[i]);
            ks.push_back((KPtr)plain_red[i]);
        }
    }
};

// Stand-in for the halved-state kernels where an arithmetic has none
// (double-float evolutions take the full state only).
template <typename R>
struct NoLowSet {
    void all(std::vector<KPtr> &) const {}
};

template <typename R>
struct PassKernels {
    using Full = PhaseTab<R, MAX_TABLE>;
    using None = PhaseTab<R, 1>;
    // high passes with rows of WROW bits (complex64: 32 amplitudes, 256 B);
    // complex128 has no wide rows and those are the narrow kernels again
    static constexpr int WROW = sizeof(R) == 4 ? HIGH_ROW + 1 : HIGH_ROW;
    LowSet<R, false> low;
    typename std::conditional<is_df<R>(), NoLowSet<R>, LowSet<R, true>>::type low_z2;
    // One CTA per SM, three tile buffers: the complex64 low passes of a single
    // instance (full and halved state).  (Measured in same-box A/Bs: the
    // strided high passes, the double-float and complex128 low passes and
    // batched low passes all run slower with one CTA per SM.)
    static constexpr bool NB3 = std::is_same<R, float>::value;
    typename std::conditional<NB3, LowSet<R, false, 3>, NoLowSet<R>>::type low3;
    typename std::conditional<NB3, LowSet<R, true, 3>, NoLowSet<R>>::type low_z2_3;
    HighSet<R, HIGH_ROW, true> high;     // [wide][full] below
    HighSet<R, HIGH_ROW, false> high_part;
    HighSet<R, WROW, true> wide;
    HighSet<R, WROW, false> wide_part;
    bool nb3_ok = false;  // the three-buffer kernels' shared memory fits the device
    cudaError_t init(size_t smem_optin) {
        const int big = (int)pass_smem<R>(true, MAX_TABLE - 1, 1, std::is_same<R, float>::value);
        std::vector<KPtr> ks;
        low.all(ks);
        low_z2.all(ks);
        high.all(ks);
        high_part.all(ks);
        wide.all(ks);
        wide_part.all(ks);
        for (KPtr k : ks) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
            if (e != cudaSuccess) return e;
        }
        const size_t big3 = pass_smem<R>(true, MAX_TABLE - 1, 3);
        nb3_ok = big3 + 1024 <= smem_optin;  // 1 KB for the static reduction buffers
        if (nb3_ok) {
            std::vector<KPtr> k3;
            low3.all(k3);
            low_z2_3.all(k3);
            for (KPtr k : k3) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big3);
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
};

template <typename R>
static int pass_kernels(PassKernels<R> **out) {
    static std::mutex mu;
    static PassKernels<R> pk;
    static int state[MAX_DEVICES] = {};  // per device: 0 = not yet, 1 = ok
    const int dev = current_device_slot();
    if (dev < 0) return QAOA_ECUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (!state[dev]) {
        DeviceInfo di;
        if (device_info(&di)) return QAOA_ECUDA;
        const cudaError_t e = pk.init(di.smem_optin);
        if (e != cudaSuccess) return cuda_error(e, "pass kernel attributes");
        state[dev] = 1;
    }
    *out = &pk;
    return QAOA_OK;
}

// Grid width per instance (CTAs gx x batch, CTA (x, y) takes tiles x, x + gx,
// ... of instance y).  The CTAs run in waves of `slots` resident ones and a
// CTA lasts about its tile count plus half a tile (its first copy overlaps
// nothing), so gx minimises
//   ceil(gx batch / slots) (ceil(tiles / gx) + 1/2)
// over 1 <= gx <= min(slots, tiles), the widest on ties.  One instance gets
// min(slots, tiles); a batch gets a width whose last wave is not left
// part-empty for the length of a whole CTA (256 instances of 2^10 tiles on
// 304 slots: gx = 19, 16 full waves of 54 tiles, where a width of 2 gave two
// waves of 512 tiles, the second with 208 CTAs).
int balanced_grid_x(int slots, int batch, uint64_t tiles) {
    if (slots < 1) slots = 1;
    if (batch < 1) batch = 1;
    const uint64_t cap = tiles < (uint64_t)slots ? (tiles > 0 ? tiles : 1) : (uint64_t)slots;
    uint64_t best = 1, best_cost = ~0ull;
    for (uint64_t gx = 1; gx <= cap; ++gx) {
        const uint64_t waves = (gx * (uint64_t)batch + slots - 1) / slots;
        const uint64_t cost = waves * (2 * ((tiles + gx - 1) / gx) + 1);  // in half tiles
        if (cost <= best_cost) {
            best_cost = cost;
            best = gx;
        }
    }
    return (int)best;
}

int pass_grid_x(int dtype, int n, int batch) {
    DeviceInfo di;
    if (device_info(&di)) return -1;
    const int T = dtype == QAOA_C64 ? Cx<float>::T : Cx<double>::T;
    return balanced_grid_x(di.sms * 2, batch, 1ull << (n - T));  // two persistent CTAs per SM
}

// Host conversions of FP64 values to each arithmetic (double-float: the
// nearest float, then the nearest float to the remainder).
template <typename R>
static R real_from(double x) {
    return (R)x;
}
template <>
dfloat real_from<dfloat>(double x) {
    const float hi = (float)x;
    return dfloat{hi, (float)(x - (double)hi)};
}
static float2 amp_from(float2 *, double re, double im) { return make_float2((float)re, (float)im); }
static double2 amp_from(double2 *, double re, double im) { return make_double2(re, im); }
static float4 amp_from(float4 *, double re, double im) {
    const dfloat r = real_from<dfloat>(re), i = real_from<dfloat>(im);
    return make_float4(r.hi, r.lo, i.hi, i.lo);
}

template <typename R>
static void fill_table(typename PassKernels<R>::Full *tab, const EvolveReq &r, int l, int sign) {
    std::vector<double> re(r.m + 1), im(r.m + 1);
    const LayerCoef k = r.p > 0 ? layer_coef(r.beta[l], sign, arith_of(r.dtype, r.flags)) : LayerCoef{1.0, 1.0, 0.0, true};
    double scale = std::pow(k.sigma, r.n);
    if (l == 0) scale *= std::pow(2.0, -0.5 * r.n);
    phase_table(r.p > 0 ? r.gamma[l] : 0.0, scale, r.m, re.data(), im.data());
    for (int c = 0; c <= r.m; ++c) tab->t[c] = amp_from(&tab->t[c], re[c], im[c]);
}

template <typename R>
static int evolve_passes(const EvolveReq &r, double *d_partials, int gx, cudaStream_t stream) {
    using V = typename Cx<R>::V;
    PassKernels<R> *pk = nullptr;
    int rc = pass_kernels<R>(&pk);
    if (rc) return rc;
    const bool z2 = (r.flags & QAOA_Z2_HALF) != 0;
    Plan pl;
    rc = make_plan(r.n, r.dtype, &pl, z2);
    if (rc) return rc;
    constexpr int T = Cx<R>::T;
    const int sign = (r.flags & QAOA_MIXER_RX2B) ? -1 : 1;
    const int arith = arith_of(r.dtype, r.flags);
    const bool want = r.d_result != nullptr;
    // The phase table is large: keep it off the stack.
    std::vector<char> tbuf(sizeof(typename PassKernels<R>::Full));
    auto *tab = reinterpret_cast<typename PassKernels<R>::Full *>(tbuf.data());
    typename PassKernels<R>::None none{};
    const std::vector<Launch> seq = make_schedule(pl.n_passes, r.p);
    const dim3 block(Cx<R>::PT), grid(gx, r.batch);
    // The complex64 low passes of a single instance take the three-buffer
    // kernels (one CTA per SM) when they fit the device: their grid is one CTA
    // per SM (never wider than gx, the partials buffer's width).
    DeviceInfo di;
    if (device_info(&di)) return QAOA_ECUDA;
    const bool use3 = PassKernels<R>::NB3 && pk->nb3_ok && r.batch == 1;
    const uint64_t tiles_one = 1ull << (pl.state_bits - T);
    const int gx3 = std::min(balanced_grid_x(di.sms, r.batch, tiles_one), gx);
    const dim3 grid3(gx3, r.batch);
    int last_gx = gx;  // grid width of the pass that writes the p_succ partials
    for (size_t i = 0; i < seq.size(); ++i) {
        const Launch &L = seq[i];
        const Pass &ps = pl.pass[L.pass];
        const bool low = L.pass == 0;
        PassArgs<R> a;
        a.state = reinterpret_cast<V *>(r.state);
        a.cost = r.cost;
        a.partials = d_partials;
        a.n = pl.state_bits;  // index bits of the stored state (and of the cost table)
        a.m = r.m;
        if (low) {  // the whole tile is one contiguous row
            a.row = T;
            a.lo = T;
            a.active = r.p > 0 ? ((1u << T) - 1u) : 0u;
        } else {
            if (ps.row != HIGH_ROW && ps.row != PassKernels<R>::WROW)
                return set_error(QAOA_ECUDA, "plan: high pass rows of %d bits", ps.row);
            a.row = ps.row;
            a.lo = ps.lo;
            a.active = ((1u << ps.bits) - 1u) << (T - ps.bits);
        }
        const bool last = i + 1 == seq.size();
        // a double-float evolution's last pass always reduces: it writes FP64 out
        a.reduce = (last && (want || r.adj || is_df<R>())) ? 1 : 0;
        if (a.reduce && !(L.mode == MODE_PLAIN || (L.mode == MODE_INIT && low)))
            return set_error(QAOA_ECUDA, "schedule: the last pass has mode %d", L.mode);
        a.adj = (last && r.adj) ? reinterpret_cast<V *>(r.adj) : nullptr;
        const LayerCoef k1 = r.p > 0 ? layer_coef(r.beta[L.la], sign, arith) : LayerCoef{1.0, 1.0, 0.0, true};
        a.ua1 = k1.unit_a;
        a.A1 = real_from<R>(k1.A);
        a.B1 = real_from<R>(k1.B);
        a.ua2 = 1;
        a.A2 = a.B2 = real_from<R>(0.0);
        if (L.mode == MODE_FUSED) {
            const LayerCoef k2 = layer_coef(r.beta[L.la + 1], sign, arith);
            a.ua2 = k2.unit_a;
            a.A2 = real_from<R>(k2.A);
            a.B2 = real_from<R>(k2.B);
        }
        a.tiles = 1ull << (pl.state_bits - T);
        const int kind = low ? K_PASS_LOW : K_PASS_HIGH;
        profile_before(kind, stream);
        const int u1 = a.ua1 ? 1 : 0, u2 = a.ua2 ? 1 : 0;
        const size_t smem_phase = pass_smem<R>(true, r.m), smem_plain = pass_smem<R>(false, 0);
        if (low) {
            // the full-state or the halved-state set (double-float has only the former)
            auto launch_low = [&](const auto &ls, dim3 g, size_t sm_phase, size_t sm_plain) -> int {
                if (L.mode == MODE_INIT) {
                    fill_table<R>(tab, r, 0, sign);
                    (r.p == 0 ? ls.init0 : ls.init[u1])<<<g, block, sm_phase, stream>>>(a, *tab);
                } else if (L.mode == MODE_PHASE) {
                    fill_table<R>(tab, r, L.la, sign);
                    ls.phase[u1]<<<g, block, sm_phase, stream>>>(a, *tab);
                } else if (L.mode == MODE_PLAIN) {
                    (a.reduce ? ls.plain_red[u1] : ls.plain[u1])<<<g, block, sm_plain, stream>>>(a, none);
                } else {
                    return set_error(QAOA_ECUDA, "schedule: fused low pass");
                }
                if (a.reduce) last_gx = (int)g.x;
                return QAOA_OK;
            };
            int lrc = QAOA_OK;
            if constexpr (PassKernels<R>::NB3) {
                const size_t p3 = pass_smem<R>(true, r.m, 3), q3 = pass_smem<R>(false, 0, 3);
                if (use3)
                    lrc = z2 ? launch_low(pk->low_z2_3, grid3, p3, q3) : launch_low(pk->low3, grid3, p3, q3);
                else
                    lrc = z2 ? launch_low(pk->low_z2, grid, smem_phase, smem_plain)
                             : launch_low(pk->low, grid, smem_phase, smem_plain);
            } else if (z2) {
                if constexpr (is_df<R>())
                    lrc = set_error(QAOA_EINVAL, "double-float takes the full state");
                else
                    lrc = launch_low(pk->low_z2, grid, smem_phase, smem_plain);
            } else {
                lrc = launch_low(pk->low, grid, smem_phase, smem_plain);
            }
            if (lrc) return lrc;
        } else {
            // rows of HIGH_ROW or WROW bits; FULL kernels when no bit of the group is a carried one
            const bool wide = ps.row != HIGH_ROW, full = ps.bits == T - ps.row;
            const HighSet<R, HIGH_ROW, true> &hn = pk->high;
            const HighSet<R, HIGH_ROW, false> &hp = pk->high_part;
            const HighSet<R, PassKernels<R>::WROW, true> &wn = pk->wide;
            const HighSet<R, PassKernels<R>::WROW, false> &wp = pk->wide_part;
            if (L.mode == MODE_INIT) {
                fill_table<R>(tab, r, 0, sign);
                auto k = wide ? (full ? wn.init[u1] : wp.init[u1]) : (full ? hn.init[u1] : hp.init[u1]);
                k<<<grid, block, smem_phase, stream>>>(a, *tab);
            } else if (L.mode == MODE_FUSED) {
                fill_table<R>(tab, r, L.la + 1, sign);
                auto k = wide ? (full ? wn.fused[u1][u2] : wp.fused[u1][u2])
                              : (full ? hn.fused[u1][u2] : hp.fused[u1][u2]);
                const size_t smem_fused = pass_smem<R>(true, r.m, 1, early_landing<R, false, MODE_FUSED, 1>());
                k<<<grid, block, smem_fused, stream>>>(a, *tab);
            } else if (L.mode == MODE_PLAIN) {
                auto k = a.reduce ? (wide ? (full ? wn.plain_red[u1] : wp.plain_red[u1])
                                          : (full ? hn.plain_red[u1] : hp.plain_red[u1]))
                                  : (wide ? (full ? wn.plain[u1] : wp.plain[u1])
                                          : (full ? hn.plain[u1] : hp.plain[u1]));
                k<<<grid, block, smem_plain, stream>>>(a, none);
            } else {
                return set_error(QAOA_ECUDA, "schedule: phase-at-load on a strided pass");
            }
        }
        rc = profile_after(kind, stream);
        if (rc) return rc;
    }
    if (want) rc = launch_reduce(d_partials, r.batch, last_gx, 2, r.d_result, stream);
    return rc;
}

// Small-n path of evolve_device: tables and coefficients through scratch.
static int evolve_small(const EvolveReq &r, Scratch *sc, size_t off, cudaStream_t stream) {
    const int sign = (r.flags & QAOA_MIXER_RX2B) ? -1 : 1;
    const int pl = r.p > 0 ? r.p : 1;
    const size_t tab_n = (size_t)pl * (r.m + 1);
    char *hb = reinterpret_cast<char *>(sc->host) + off;
    char *db = reinterpret_cast<char *>(sc->dev) + off;
    double *h_tab = reinterpret_cast<double *>(hb);
    double *h_coef = h_tab + 2 * tab_n;
    SmallJob *h_jobs = reinterpret_cast<SmallJob *>(h_coef + 4 * pl);
    std::vector<double> re(r.m + 1), im(r.m + 1);
    for (int l = 0; l < pl; ++l) {
        LayerCoef k = r.p > 0 ? layer_coef(r.beta[l], sign, arith_of(r.dtype, r.flags)) : LayerCoef{1.0, 1.0, 0.0, true};
        double scale = std::pow(k.sigma, r.n);
        if (l == 0) scale *= std::pow(2.0, -0.5 * r.n);
        phase_table(r.p > 0 ? r.gamma[l] : 0.0, scale, r.m, re.data(), im.data());
        for (int c = 0; c <= r.m; ++c) {
            h_tab[2 * ((size_t)l * (r.m + 1) + c)] = re[c];
            h_tab[2 * ((size_t)l * (r.m + 1) + c) + 1] = im[c];
        }
        h_coef[4 * l] = k.A;
        h_coef[4 * l + 1] = k.B;
        h_coef[4 * l + 2] = k.unit_a ? 1.0 : 0.0;
        h_coef[4 * l + 3] = 0.0;
    }
    const size_t es = r.dtype == QAOA_C64 ? 8 : 16;
    for (int b = 0; b < r.batch; ++b) {
        SmallJob j;
        j.cost = r.cost + ((size_t)b << r.n);
        j.state = reinterpret_cast<char *>(r.state) + ((size_t)b << r.n) * es;
        j.result = r.d_result ? r.d_result + 2 * b : nullptr;
        j.n = r.n;
        j.m = r.m;
        j.p = r.p;
        j.table_off = 0;
        j.coef_off = 0;
        h_jobs[b] = j;
    }
    const size_t bytes = (2 * tab_n + 4 * (size_t)pl) * sizeof(double) + (size_t)r.batch * sizeof(SmallJob);
    QAOA_CUDA_TRY(cudaMemcpyAsync(db, hb, bytes, cudaMemcpyHostToDevice, stream));
    int rc = launch_small_batch(r.dtype, r.batch, reinterpret_cast<SmallJob *>(db + (2 * tab_n + 4 * pl) * sizeof(double)),
                                reinterpret_cast<double *>(db), reinterpret_cast<double *>(db) + 2 * tab_n, r.n, r.flags,
                                stream);
    if (rc) return rc;
    // the pinned staging block is reused by the next call on this stream
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    return QAOA_OK;
}

// Validates an evolution request (shared by the ABI entry points).
static int validate_evolve(int batch, int n, const uint8_t *cost, int m, int p, const double *gamma,
                           const double *beta, int dtype, void *state) {
    if (batch < 1) return set_error(QAOA_EINVAL, "batch=%d", batch);
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", dtype);
    const int nmax = dtype == QAOA_C64 ? QAOA_MAX_N : QAOA_MAX_N - 1;
    if (n < 1 || n > nmax) return set_error(QAOA_ERANGE, "n=%d outside [1, %d]", n, nmax);
    if (m < 0 || m > QAOA_MAX_M) return set_error(QAOA_ERANGE, "m=%d outside [0, %d]", m, QAOA_MAX_M);
    if (p < 0) return set_error(QAOA_EINVAL, "p=%d", p);
    if (p > 0 && (!gamma || !beta)) return set_error(QAOA_EINVAL, "gamma/beta NULL");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l]))
            return set_error(QAOA_EINVAL, "angle %d is not finite", l);
    if (!cost || !state) return set_error(QAOA_EINVAL, "d_cost/d_state NULL");
    return QAOA_OK;
}

int evolve_device_impl(const EvolveReq &r, cudaStream_t stream, double *d_partials, int gx) {
    if (r.dtype == QAOA_C64) return evolve_passes<float>(r, d_partials, gx, stream);
    if (r.flags & QAOA_DF64) return evolve_passes<dfloat>(r, d_partials, gx, stream);
    return evolve_passes<double>(r, d_partials, gx, stream);
}

}  // namespace qaoa

using namespace qaoa;

// Runs an evolution and (optionally) copies the FP64 results to the host.
static int evolve_common(int batch, int n, const uint8_t *d_cost, int m, int p, const double *gamma,
                         const double *beta, int dtype, int flags, void *d_state, double *p_succ, double *norm,
                         void *adj, void *stream_) {
    int rc = validate_evolve(batch, n, d_cost, m, p, gamma, beta, dtype, d_state);
    if (rc) return rc;
    const bool z2 = (flags & QAOA_Z2_HALF) != 0;
    if ((flags & QAOA_DF64) && (dtype != QAOA_C128 || z2 || adj))
        return set_error(QAOA_EINVAL, "QAOA_DF64 takes a complex128 full-state evolution (no halved state, no gradient)");
    if (z2 && n <= small_n_limit(dtype))
        return set_error(QAOA_ERANGE, "halved state needs n > %d (n=%d)", small_n_limit(dtype), n);
    if (z2 && adj) return set_error(QAOA_EINVAL, "the gradient does not take the halved state");
    const double scale = z2 ? 2.0 : 1.0;  // each stored amplitude stands for x and not x
    cudaStream_t stream = (cudaStream_t)stream_;
    const bool want = p_succ || norm;
    m = table_top(m);  // from here m bounds the phase tables only
    EvolveReq r{batch, n, m, p, dtype, flags, d_cost, d_state, adj, gamma, beta, nullptr};
    Scratch *sc = nullptr;
    if (n <= small_n_limit(dtype) && !adj) {
        const int pl = p > 0 ? p : 1;
        const size_t stage = (2 * (size_t)pl * (m + 1) + 4 * (size_t)pl) * sizeof(double) +
                             (size_t)batch * sizeof(SmallJob) + 256;
        const size_t res = (size_t)batch * 2 * sizeof(double);
        rc = scratch_for(stream, stage + res, stage + res, &sc);
        if (rc) return rc;
        if (want) r.d_result = reinterpret_cast<double *>(reinterpret_cast<char *>(sc->dev) + stage);
        rc = evolve_small(r, sc, 0, stream);
        if (rc || !want) return rc;
        double *h = reinterpret_cast<double *>(reinterpret_cast<char *>(sc->host) + stage);
        QAOA_CUDA_TRY(cudaMemcpyAsync(h, r.d_result, res, cudaMemcpyDeviceToHost, stream));
        QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
        for (int b = 0; b < batch; ++b) {
            if (p_succ) p_succ[b] = h[2 * b];
            if (norm) norm[b] = h[2 * b + 1];
        }
        return QAOA_OK;
    }
    if (n <= small_n_limit(dtype)) return set_error(QAOA_ERANGE, "n=%d too small for the pass path", n);
    const int gx = pass_grid_x(dtype, z2 ? n - 1 : n, batch);
    if (gx < 0) return QAOA_ECUDA;
    const size_t part = (size_t)batch * gx * 2 * sizeof(double);
    const size_t res = (size_t)batch * 2 * sizeof(double);
    rc = scratch_for(stream, part + res + 256, res + 64, &sc);
    if (rc) return rc;
    double *d_part = reinterpret_cast<double *>(sc->dev);
    if (want) r.d_result = reinterpret_cast<double *>(reinterpret_cast<char *>(sc->dev) + part);
    rc = evolve_device_impl(r, stream, d_part, gx);
    if (rc || !want) return rc;
    double *h = reinterpret_cast<double *>(sc->host);
    QAOA_CUDA_TRY(cudaMemcpyAsync(h, r.d_result, res, cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    for (int b = 0; b < batch; ++b) {
        if (p_succ) p_succ[b] = scale * h[2 * b];
        if (norm) norm[b] = scale * h[2 * b + 1];
    }
    return QAOA_OK;
}

namespace qaoa {
int evolve_with_adjoint_seed(int batch, int n, const uint8_t *d_cost, int m, int p, const double *gamma,
                             const double *beta, int dtype, int flags, void *d_state, void *d_adj, double *p_succ,
                             void *stream) {
    return evolve_common(batch, n, d_cost, m, p, gamma, beta, dtype, flags, d_state, p_succ, nullptr, d_adj, stream);
}
}  // namespace qaoa

extern "C" int qaoa_evolve(int n, const uint8_t *d_cost, int m, int p, const double *gamma, const double *beta,
                           int dtype, int flags, void *d_state, double *p_succ, double *norm, void *stream) {
    return evolve_common(1, n, d_cost, m, p, gamma, beta, dtype, flags, d_state, p_succ, norm, nullptr, stream);
}

extern "C" int qaoa_evolve_batch(int batch, int n, const uint8_t *d_costs, int m_max, int p, const double *gamma,
                                 const double *beta, int dtype, int flags, void *d_states, double *p_succ,
                                 double *norm, void *stream) {
    return evolve_common(batch, n, d_costs, m_max, p, gamma, beta, dtype, flags, d_states, p_succ, norm, nullptr,
                         stream);
}

extern "C" int qaoa_success_prob(int n, const uint8_t *d_cost, const void *d_state, int dtype, double *p_succ,
                                 double *norm, void *stream_) {
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", dtype);
    if (n < 1 || n > QAOA_MAX_N) return set_error(QAOA_ERANGE, "n=%d", n);
    if (!d_cost || !d_state || !p_succ || !norm) return set_error(QAOA_EINVAL, "NULL argument");
    cudaStream_t stream = (cudaStream_t)stream_;
    DeviceInfo di;
    int rc = device_info(&di);
    if (rc) return rc;
    const uint64_t chunks = ((1ull << n) + (uint64_t)PT * 32 - 1) / ((uint64_t)PT * 32);
    uint64_t g = (uint64_t)di.sms * 8;
    const int grid = (int)(chunks < g ? chunks : g);
    const size_t part = (size_t)grid * 2 * sizeof(double);
    Scratch *sc = nullptr;
    rc = scratch_for(stream, part + 64, 64, &sc);
    if (rc) return rc;
    double *d_part = reinterpret_cast<double *>(sc->dev);
    double *d_res = reinterpret_cast<double *>(reinterpret_cast<char *>(sc->dev) + part);
    profile_before(K_PSUCC, stream);
    if (dtype == QAOA_C64)
        psucc_kernel<float><<<grid, PT, 0, stream>>>(reinterpret_cast<const float2 *>(d_state), d_cost, n, d_part);
    else
        psucc_kernel<double><<<grid, PT, 0, stream>>>(reinterpret_cast<const double2 *>(d_state), d_cost, n, d_part);
    rc = profile_after(K_PSUCC, stream);
    if (rc) return rc;
    profile_before(K_REDUCE, stream);
    reduce_partials_kernel<<<1, PT, 0, stream>>>(d_part, grid, 2, d_res);
    rc = profile_after(K_REDUCE, stream);
    if (rc) return rc;
    double *h = reinterpret_cast<double *>(sc->host);
    QAOA_CUDA_TRY(cudaMemcpyAsync(h, d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    *p_succ = h[0];
    *norm = h[1];
    return QAOA_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of qaoa_success_prob.  Some callers cannot allocate
// device memory at the moment they need a result: hosts that pre-reserve the
// whole device for their own allocator, or signal-safe / real-time paths where
// a cudaMalloc (which may synchronise the device) is not allowed.  For them the
// per-block partial sums and the final pair live in this fixed device array,
// part of the library's image: every GPU that loads the library holds it
// (2 x 4096 + 2 doubles, about 64 KiB) until the process exits.
constexpr int NOALLOC_MAX_BLOCKS = 4096;
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 2];

static std::mutex g_noalloc_mu;
static double *g_noalloc_addr[256];  // device address of the array, per device ordinal

// Host code cannot use g_noalloc_scratch's name as a device address; the
// address is looked up once per device with that device current.
static int noalloc_scratch(double **out) {
    int dev = 0;
    QAOA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(QAOA_ERANGE, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[dev];
    return QAOA_OK;
}

extern "C" int qaoa_success_prob_noalloc(int n, const uint8_t *d_cost, const void *d_state, int dtype,
                                         double *p_succ, double *norm, void *stream_) {
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", dtype);
    if (n < 1 || n > QAOA_MAX_N)
        return set_error(QAOA_ERANGE, "n=%d outside [1, %d] (the fixed scratch serves states of up to 2^%d amplitudes)",
                         n, QAOA_MAX_N, QAOA_MAX_N);
    if (!d_cost || !d_state || !p_succ || !norm) return set_error(QAOA_EINVAL, "NULL argument");
    cudaStream_t stream = (cudaStream_t)stream_;
    int dev = 0, sms = 0;
    QAOA_CUDA_TRY(cudaGetDevice(&dev));
    QAOA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double *scr = nullptr;
    int rc = noalloc_scratch(&scr);
    if (rc) return rc;
    // Each block strides over the state and writes one partial pair, so the
    // grid (never above NOALLOC_MAX_BLOCKS) bounds the scratch it uses.
    const uint64_t chunks = ((1ull << n) + (uint64_t)PT * 32 - 1) / ((uint64_t)PT * 32);
    uint64_t g = (uint64_t)sms * 8;
    if (g > (uint64_t)NOALLOC_MAX_BLOCKS) g = NOALLOC_MAX_BLOCKS;
    const int grid = (int)(chunks < g ? chunks : g);
    double *d_part = scr;                             // [grid][2], all written before they are read
    double *d_res = scr + 2 * NOALLOC_MAX_BLOCKS;     // [2]
    profile_before(K_PSUCC, stream);
    if (dtype == QAOA_C64)
        psucc_kernel<float><<<grid, PT, 0, stream>>>(reinterpret_cast<const float2 *>(d_state), d_cost, n, d_part);
    else
        psucc_kernel<double><<<grid, PT, 0, stream>>>(reinterpret_cast<const double2 *>(d_state), d_cost, n, d_part);
    rc = profile_after(K_PSUCC, stream);  // counts the launch, checks its status
    if (rc) return rc;
    profile_before(K_REDUCE, stream);
    reduce_partials_kernel<<<1, PT, 0, stream>>>(d_part, grid, 2, d_res);
    rc = profile_after(K_REDUCE, stream);
    if (rc) return rc;
    double h[2];  // pageable host copy: the runtime stages it, nothing is allocated here
    QAOA_CUDA_TRY(cudaMemcpyAsync(h, d_res, sizeof h, cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    *p_succ = h[0];
    *norm = h[1];
    return QAOA_OK;
}
