// Device building blocks of the HBM butterfly passes (forward and adjoint).
//
// A pass streams the state through shared memory one tile at a time.  A tile
// holds 2^T amplitudes: 2^row contiguous ones (a row) times 2^(T - row) rows
// strided by 2^lo, so its tile bits [row, T) are the state bits
// [lo, lo + T - row) that the pass butterflies ("the group"); the low pass has
// row = lo = T and butterflies state bits [0, T).
//
// 256 threads own the tile in registers, 2^RB amplitudes each.  A "mapping"
// (parameter LO) gives thread tid and register r the tile element
//   u = (tid & (2^LO - 1)) | ((tid >> LO) << (LO + RB)) | (r << LO),
// so the registers of a thread span tile bits [LO, LO + RB) and the butterflies
// on those bits run in registers.  Moving between mappings goes through shared
// memory with an XOR swizzle that keeps every round free of bank conflicts.
//   mapping 8       : lanes run along tile bits 0..4 -> coalesced loads/stores
//   mapping 0       : the low pass's tile bits [0, RB)
//   mapping LC      : the rest, also coalesced (lanes along bits 0..3 or 0..4)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace qaoa {

constexpr int PT = 256;  // threads per pass CTA (8 thread bits)
// Row width (bits) of every high-pass tile: 16 contiguous amplitudes.
constexpr int HIGH_ROW = 4;

// Double-float number: the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits (Dekker 1971; the arithmetic
// below is Knuth's TwoSum, Dekker's Fast2Sum and the FMA form of Dekker's
// TwoProduct).  On GB300 the FP32 pipes are 64 times as fast as the FP64 pipe,
// so complex128 evolutions can run their butterflies and phases in this
// arithmetic (QAOA_DF64) and stay accurate to about 1e-14 per operation.
struct dfloat {
    float hi, lo;
};

// Register/shared-memory amplitude of each arithmetic: (re, im), or for
// double-float (re.hi, re.lo, im.hi, im.lo).
template <typename R>
struct VecOf;
template <>
struct VecOf<float> {
    using type = float2;
};
template <>
struct VecOf<double> {
    using type = double2;
};
template <>
struct VecOf<dfloat> {
    using type = float4;
};

// Tile geometry: element type R, 2^T amplitudes per tile, 2^RB per thread,
// 2^(T - RB) threads.  The load mapping (LO = T - RB) puts the registers on the
// top RB tile bits, so lanes run along tile bits 0..4 (coalesced, and dense in
// shared memory).  The swizzle spreads the bits that lanes run along in the
// other mappings over the shared-memory banks (checked conflict-free for every
// mapping used).
template <typename R, int T_, int RB_>
struct Geo {
    using V = typename VecOf<R>::type;
    using Real = R;
    static constexpr int T = T_;
    static constexpr int RB = RB_;
    static constexpr int NR = 1 << RB_;
    static constexpr int TB = T_ - RB_;
    static constexpr int PT = 1 << TB;
    static constexpr int LOAD = TB;
    static constexpr int LC_LOW = RB_;  // adjoint passes: rounds at 8, 0, RB
    static constexpr int LC_HIGH = 4;
    // Padded layout: one spare amplitude after every 2^RB, which keeps every
    // mapping used free of bank conflicts.  It is additive over the disjoint
    // thread and register bit fields of a tile element, so an exchange address
    // is a per-thread base plus a compile-time offset.
    static constexpr int PADSH = RB_;
    static constexpr int TILE_ELEMS = (1 << T_) + (1 << (T_ - RB_));
    __host__ __device__ static constexpr uint32_t swz(uint32_t u) { return u + (u >> PADSH); }
    // Cost bytes of a high-pass tile: 16 spare bytes after every 2^(4 + RB).  In
    // the passes' last mapping (4) lanes 0..15 read 16 consecutive bytes and
    // lanes 16..31 the 16 bytes 2^(4 + RB) further on, which the dense layout
    // puts in the same four banks (one extra wavefront per load); the padding
    // moves them to the next four.  The load mapping reads 32 consecutive bytes
    // inside one period either way.  Low passes keep the dense layout.
    static constexpr int CPAD = 4 + RB_;
    static constexpr int CS_BYTES = (1 << T_) + ((1 << T_) >> RB_);  // one cost buffer, padded
    // Additive over disjoint bit fields, so a mapping's cost index is the
    // thread part's plus a compile-time constant per register.
    __host__ __device__ static constexpr uint32_t cidx(uint32_t u) { return u + ((u >> CPAD) << 4); }
};

// The thread's cost bytes in mapping LO on the padded layout: register r's
// byte is at sc[returned offset + G::cidx(r << LO)] (a compile-time offset).
// The offset passes through an opaque asm, so it is formed where it is used
// instead of being kept live across the tile loop.
template <typename G, int LO>
__device__ __forceinline__ uint32_t cost_base(uint32_t tid) {
    uint32_t o = G::cidx((tid & ((1u << LO) - 1u)) | ((tid >> LO) << (LO + G::RB)));
    asm volatile("" : "+r"(o));
    return o;
}

// Forward geometry: 64 KiB tiles, 256 threads; complex64 with 32 amplitudes
// per thread, complex128 with 16.
template <typename R>
struct FwdGeoT;
template <>
struct FwdGeoT<float> {
    using type = Geo<float, 13, 5>;
};
template <>
struct FwdGeoT<double> {
    using type = Geo<double, 12, 4>;
};
template <>
struct FwdGeoT<dfloat> {  // complex128 storage, double-float arithmetic: 16 B per amplitude
    using type = Geo<dfloat, 12, 4>;
};
template <typename R>
using Cx = typename FwdGeoT<R>::type;

// A round: the mapping LO and the tile bits it butterflies (compile time; the
// pass's runtime mask of active bits is applied on top).
template <int LO_, uint32_t MASK_>
struct Round {
    static constexpr int LO = LO_;
    static constexpr uint32_t MASK = MASK_;
};

// The rounds of the low pass (all T tile bits) and of a high pass (tile bits
// [4, T): rows of 16 contiguous amplitudes), per forward geometry.  The first
// round is the load mapping; the last round's mapping is also coalesced.
template <int T, int RB, bool LOW>
struct RoundsFor;
template <>
struct RoundsFor<13, 5, true> {
    static constexpr int N = 3, LAST = 5;
    using R0 = Round<8, 0x1F00>;
    using R1 = Round<0, 0x001F>;
    using R2 = Round<5, 0x00E0>;
};
template <>
struct RoundsFor<13, 5, false> {
    static constexpr int N = 2, LAST = 4;
    using R0 = Round<8, 0x1F00>;
    using R1 = Round<4, 0x00F0>;
};
template <>
struct RoundsFor<12, 4, true> {
    static constexpr int N = 3, LAST = 4;
    using R0 = Round<8, 0xF00>;
    using R1 = Round<0, 0x00F>;
    using R2 = Round<4, 0x0F0>;
};
template <>
struct RoundsFor<12, 4, false> {
    static constexpr int N = 2, LAST = 4;
    using R0 = Round<8, 0xF00>;
    using R1 = Round<4, 0x0F0>;
};
// The rounds depend only on the tile shape (T, RB), not on the arithmetic.
template <typename G, bool LOW>
struct PassRounds : RoundsFor<G::T, G::RB, LOW> {};

template <typename G, int LO>
__device__ __forceinline__ uint32_t tile_elem(uint32_t tid, uint32_t r) {
    constexpr int RB = G::RB;
    return (tid & ((1u << LO) - 1u)) | ((tid >> LO) << (LO + RB)) | (r << LO);
}

// State index of tile element u relative to the tile base, in 32 bits (the
// indices of one instance fit, n <= 32).
__device__ __forceinline__ uint32_t elem_offset32(uint32_t u, int row, int lo) {
    return (u & ((1u << row) - 1u)) | ((u >> row) << lo);
}

// State index of the first element of tile t: the tile id fills the free bits
// [row, lo) and [lo + G, n), G = T - row.
__device__ __forceinline__ uint64_t tile_base(uint64_t t, int row, int lo, int T) {
    const int G = T - row;
    const int span = lo - row;
    return ((t & ((1ull << span) - 1ull)) << row) | ((t >> span) << (lo + G));
}
__device__ __forceinline__ uint32_t tile_base32(uint32_t t, int row, int lo, int T) {
    return (uint32_t)tile_base(t, row, lo, T);
}

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// ---- double-float arithmetic (no contraction: every step rounds once) -------
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float &s, float &e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// x + c y for double-floats (the lo x lo product is below the format's
// precision and dropped), left unrenormalised: hi + lo carries the same value
// with |lo| a few ulp(hi).  The butterflies chain these; the pass renormalises
// each pair with Fast2Sum before it stores the tile.
__device__ __forceinline__ dfloat df_axpy_raw(dfloat c, float y_hi, float y_lo, float x_hi, float x_lo) {
    const float p = __fmul_rn(c.hi, y_hi);
    const float pe = __fmaf_rn(c.hi, y_hi, -p);  // c.hi y.hi = p + pe exactly
    float s, se;
    df_two_sum(x_hi, p, s, se);
    float lo = __fadd_rn(__fadd_rn(se, pe), x_lo);
    lo = __fmaf_rn(c.hi, y_lo, lo);
    lo = __fmaf_rn(c.lo, y_hi, lo);
    return dfloat{s, lo};
}
// x + c y, renormalised (|lo| <= ulp(hi) / 2).
__device__ __forceinline__ dfloat df_axpy(dfloat c, float y_hi, float y_lo, float x_hi, float x_lo) {
    const dfloat t = df_axpy_raw(c, y_hi, y_lo, x_hi, x_lo);
    dfloat r;
    df_fast_two_sum(t.hi, t.lo, r.hi, r.lo);
    return r;
}
// A pair renormalised (|hi| >= |lo|, or hi = 0).
__device__ __forceinline__ float4 df_renorm(float4 v) {
    float4 r;
    df_fast_two_sum(v.x, v.y, r.x, r.y);
    df_fast_two_sum(v.z, v.w, r.z, r.w);
    return r;
}
__device__ __forceinline__ dfloat df_neg(dfloat c) { return dfloat{-c.hi, -c.lo}; }

// Complex product in double-float: (a.re b.re - a.im b.im, a.re b.im + a.im b.re).
__device__ __forceinline__ float4 cmul(float4 a, float4 b) {
    const dfloat are{a.x, a.y}, aim{a.z, a.w};
    const dfloat t = df_axpy(are, b.x, b.y, 0.f, 0.f);
    const dfloat re = df_axpy(df_neg(aim), b.z, b.w, t.hi, t.lo);
    const dfloat u = df_axpy(are, b.z, b.w, 0.f, 0.f);
    const dfloat im = df_axpy(aim, b.x, b.y, u.hi, u.lo);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// Mixer butterfly in factored form: (a, b) <- (A a + i B b, i B a + A b) with
// A = 1 (UA) or B = 1; the dropped scalar sigma^n is folded into the phase table.
template <bool UA, typename V, typename R>
__device__ __forceinline__ void bfly(V &a, V &b, R A, R B) {
    V na, nb;
    if (UA) {
        na.x = fma(-B, b.y, a.x);
        na.y = fma(B, b.x, a.y);
        nb.x = fma(-B, a.y, b.x);
        nb.y = fma(B, a.x, b.y);
    } else {
        na.x = fma(A, a.x, -b.y);
        na.y = fma(A, a.y, b.x);
        nb.x = fma(A, b.x, -a.y);
        nb.y = fma(A, b.y, a.x);
    }
    a = na;
    b = nb;
}

// The factored butterfly in double-float arithmetic (float4 amplitudes; the
// results are left unrenormalised, see df_axpy_raw).
template <bool UA>
__device__ __forceinline__ void bfly(float4 &a, float4 &b, dfloat A, dfloat B) {
    float4 na, nb;
    if (UA) {  // (a + i B b, b + i B a)
        const dfloat nB = df_neg(B);
        dfloat t = df_axpy_raw(nB, b.z, b.w, a.x, a.y);
        na.x = t.hi, na.y = t.lo;
        t = df_axpy_raw(B, b.x, b.y, a.z, a.w);
        na.z = t.hi, na.w = t.lo;
        t = df_axpy_raw(nB, a.z, a.w, b.x, b.y);
        nb.x = t.hi, nb.y = t.lo;
        t = df_axpy_raw(B, a.x, a.y, b.z, b.w);
        nb.z = t.hi, nb.w = t.lo;
    } else {  // (A a + i b, A b + i a)
        dfloat t = df_axpy_raw(A, a.x, a.y, -b.z, -b.w);
        na.x = t.hi, na.y = t.lo;
        t = df_axpy_raw(A, a.z, a.w, b.x, b.y);
        na.z = t.hi, na.w = t.lo;
        t = df_axpy_raw(A, b.x, b.y, -a.z, -a.w);
        nb.x = t.hi, nb.y = t.lo;
        t = df_axpy_raw(A, b.z, b.w, a.x, a.y);
        nb.z = t.hi, nb.w = t.lo;
    }
    a = na;
    b = nb;
}

// Butterflies on the register bits of mapping LO that are in MASK and active.
template <typename G, bool UA, int LO, uint32_t MASK>
__device__ __forceinline__ void mask_butterflies(typename G::V *v, uint32_t active, typename G::Real A,
                                                 typename G::Real B) {
    constexpr int RB = G::RB;
    constexpr int NR = 1 << RB;
#pragma unroll
    for (int q = 0; q < RB; ++q) {
        if (((MASK >> (LO + q)) & 1u) && ((active >> (LO + q)) & 1u)) {
#pragma unroll
            for (int i = 0; i < NR; ++i)
                if (!(i & (1 << q))) bfly<UA>(v[i], v[i | (1 << q)], A, B);
        }
    }
}

// Butterflies on the register bits of mapping LO whose tile bits are in `mask`
// (bits LO + q, q = 0..RB-1) and below `below` (compile-time exclusion of bits
// done in an earlier round).
template <typename G, bool UA, int LO, int BELOW>
__device__ __forceinline__ void reg_butterflies(typename G::V *v, uint32_t mask, typename G::Real A,
                                                typename G::Real B) {
    constexpr int RB = G::RB;
    constexpr int NR = 1 << RB;
#pragma unroll
    for (int q = 0; q < RB; ++q) {
        if (LO + q < BELOW && ((mask >> (LO + q)) & 1u)) {
#pragma unroll
            for (int i = 0; i < NR; ++i)
                if (!(i & (1 << q))) bfly<UA>(v[i], v[i | (1 << q)], A, B);
        }
    }
}

// Re-distribute the tile from mapping FROM to mapping TO through shared memory
// (padded layout: per-thread base + compile-time offset per register).  The
// thread parts pass through an opaque asm so that the compiler recomputes them
// per tile instead of hoisting them out of the tile loop.
template <typename G, int FROM, int TO>
__device__ __forceinline__ void exchange(typename G::V *v, typename G::V *tile) {
    constexpr int NR = G::NR;
    const uint32_t tid = threadIdx.x;
    uint32_t bf = G::swz(tile_elem<G, FROM>(tid, 0)), bt = G::swz(tile_elem<G, TO>(tid, 0));
    asm volatile("" : "+r"(bf), "+r"(bt));
    typename G::V *pf = tile + bf;
    typename G::V *pt = tile + bt;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) pf[G::swz((uint32_t)r << FROM)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = pt[G::swz((uint32_t)r << TO)];
}

// cp.async (LDGSTS) helpers: 16-byte global -> shared copies that complete in
// the background; completion is a hardware wait on the thread's commit groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issues the copies of tile `base` into (buf, sc): the state as 16-byte chunks
// (the tile's rows of 2^row amplitudes are whole numbers of chunks) and, when
// needed, its cost bytes (one 16-byte chunk per row of 16 amplitudes).  Chunk q
// of the tile lands at byte 16 q of the buffer, i.e. tile element u sits at
// buf[u] (with PADC the cost byte of u at sc[G::cidx(u)]); thread tid takes
// chunks tid + PT j, whose addresses are a thread base plus j times a stride.
// Indices inside one instance fit in 32 bits.
// Chunks j in [J0, J1) of each thread only (J1 < 0: all), so that a tile can
// land in two parts: the chunks of elements below a bound, and the rest.
template <typename G, bool PADC = false, int J0 = 0, int J1 = -1>
__device__ __forceinline__ void issue_tile(const typename G::V *st, const uint8_t *cs, uint32_t base, int row, int lo,
                                           bool state, bool cost, typename G::V *buf, uint8_t *sc) {
    using V = typename G::V;
    constexpr int T = G::T;
    constexpr int EPC = 16 / (int)sizeof(V);            // amplitudes per 16-byte chunk
    constexpr int NT = G::PT;
    constexpr int NCH = (1 << T) / EPC / NT;             // state chunks per thread
    constexpr int CCH = (1 << T) / 16 / NT;              // cost chunks per thread
    constexpr int JE = J1 < 0 ? NCH : J1;
    const uint32_t tid = threadIdx.x;
    if (state) {
        // chunk q = tid + PT j covers tile elements [EPC q, EPC q + EPC)
        // the bits of EPC * NT * j lie above those of EPC * tid and above the row
        // bits, so the offset is linear in j
        const uint32_t off0 = base + elem_offset32((uint32_t)EPC * tid, row, lo);
        const uint32_t step = elem_offset32((uint32_t)(EPC * NT), row, lo);
        char *dst = reinterpret_cast<char *>(buf) + 16 * tid;
#pragma unroll
        for (int j = J0; j < JE; ++j) cp_async16(dst + (size_t)16 * NT * j, st + (off0 + step * j));
    }
    if (cost) {
        const uint32_t off0 = base + elem_offset32(16u * tid, row, lo);
        const uint32_t step = elem_offset32(16u * NT, row, lo);
#pragma unroll
        for (int j = 0; j < CCH; ++j) {
            const uint32_t q = tid + NT * j;  // 16-byte chunk q: bytes [16 q, 16 q + 16) of the tile
            cp_async16(sc + 16 * q + (PADC ? 16 * (q >> G::RB) : 0), cs + (off0 + step * j));
        }
    }
}

// Pairwise sum of NR values fed in index order (NR a power of two; the index
// must be a compile-time constant after unrolling, so the levels stay in
// registers): element r joins the partial sums of the completed blocks below it,
// giving the perfectly balanced tree ((x0 + x1) + (x2 + x3)) + ... with only
// log2(NR) + 1 values live.  For NR = 32 non-negative FP32 terms the relative
// error is at most 5 u (u = 2^-24), against 31 u for a running sum.
template <int NR, typename P>
struct PairwiseSum {
    static constexpr int LOG = NR <= 1 ? 0 : (NR <= 2 ? 1 : (NR <= 4 ? 2 : (NR <= 8 ? 3 : (NR <= 16 ? 4 : (NR <= 32 ? 5 : 6)))));
    static_assert((1 << LOG) == NR, "NR must be a power of two up to 64");
    P lvl[LOG + 1];
    __device__ __forceinline__ void add(int r, P x) {
        int k = 0;
#pragma unroll
        for (; k < LOG && ((r >> k) & 1); ++k) x = lvl[k] + x;
        lvl[k] = x;
    }
    __device__ __forceinline__ P total() const { return lvl[LOG]; }
};

// FP64 block reduction of NV values per thread (NT threads); thread 0 gets
// the sums.
template <int NV, int NT = PT>
__device__ __forceinline__ void block_sum(double (&x)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_xor_sync(0xFFFFFFFFu, x[k], o);
    __shared__ double s_red[NT / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) s_red[wid][k] = x[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += s_red[w][k];
            x[k] = s;
        }
    }
}

}  // namespace qaoa
