// K1: the NAE cost table C(x) (Eq. for C^NAE, Sec. "Problem Hamiltonian"; its
// De Morgan form in Appendix A.2: a clause is violated when its literals are
// all false or all true).
//
// Bit-sliced design.  A thread owns one 32-bit word of assignments,
// x = 32 X + b for b = 0..31.  Variables 0..4 vary inside the word, variables
// >= 5 are constant across it.  Per clause the host precomputes
//   hi_mask / hi_neg : the clause's variables >= 5 and their negations,
//   all_true  : bit b set iff every literal on a variable < 5 is true at b,
//   all_false : bit b set iff every such literal is false at b.
// With t = ((32 X) ^ hi_neg) & hi_mask (the literal values on the high
// variables) the clause's violation word is
//   V = (t == 0 ? all_false : 0) | (t == hi_mask ? all_true : 0),
// i.e. all literals false, or all true.  The 32 per-x counts are kept as
// bit planes by a carry-save (Harley-Seal) adder over chunks of 16 clauses,
// then transposed to bytes with 8x8 bit-matrix transposes.  The clause records
// sit in shared memory (one broadcast 16-byte load per clause) and each thread
// counts two words per record load.  The number of
// solutions (count 0) and the largest count come out of the same pass.
//
// Large clause counts.  The records are staged CT_CHUNK at a time: the block
// filters and counts one chunk, then the next, accumulating into the same
// counters.  Up to 1023 clauses 10 bit planes count exactly; beyond that 13
// planes do (m <= 8191).  Only the counts <= 255 go into the table; a larger
// one makes the call fail with the exact maximum.
//
// Global-flip symmetry.  Flipping every bit of x flips every literal, so a
// clause's literals stay all equal or not: C(not x) = C(x) (Sec. 2.2).  The
// complement of x = 32 X + b is 32 (W - 1 - X) + (31 - b) (W = 2^(n - 5)
// words), so a full table is counted on its lower half only: each counted
// word is written twice, the second time byte-reversed at word W - 1 - X.
//
// Clause filtering.  A block takes 512 consecutive words at a time, so the
// variables >= 14 (SUB_BITS) are constant over them.  A clause whose literals
// on those variables are neither all true nor all false is violated nowhere in
// the block; the block first keeps only the others, each reduced to its
// variables 5..13 and to the one or two patterns still possible (for random
// 5-literal clauses over 30 variables about 40% survive), then counts against
// that list.  Counts are sums of 0/1 terms, so the list order is immaterial.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "qaoa_internal.cuh"

namespace qaoa {

constexpr int CT_THREADS = 256;
constexpr int CT_CHUNK = 1024;     // clause records staged in shared memory at a time
constexpr int CT_PARAM_M = 1023;   // largest m passed as kernel parameters
constexpr int NPL_SMALL = 10;      // bit planes for m <= 1023
constexpr int NPL_LARGE = 13;      // bit planes for m <= 8191
static_assert(QAOA_MAX_M < (1 << NPL_LARGE), "counts must fit the planes");

struct CostParams {
    int n, m;
    int mirror;  // count the lower half, write both (full tables, n >= 6)
    ClauseRec rec[CT_PARAM_M];
};

__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

__device__ __forceinline__ uint32_t violation_word(uint32_t xh, const ClauseRec &r) {
    const uint32_t t = (xh ^ r.hi_neg) & r.hi_mask;
    return (t == 0u ? r.all_false : 0u) | (t == r.hi_mask ? r.all_true : 0u);
}

// Carry-save counter of the violated clauses of one 32-assignment word:
// bit plane q holds bit q of every count (q = 0..NPL-1, counts < 2^NPL).
template <int NPL>
struct WordCounter {
    uint32_t ones = 0, twos = 0, fours = 0, eights = 0;
    uint32_t up[NPL - 4] = {};
    // Adds 16 violation words (a Harley-Seal chunk).
    __device__ __forceinline__ void add16(const uint32_t v[16]) {
        uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
        csa(twosA, ones, ones, v[0], v[1]);
        csa(twosB, ones, ones, v[2], v[3]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, v[4], v[5]);
        csa(twosB, ones, ones, v[6], v[7]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eightsA, fours, fours, foursA, foursB);
        csa(twosA, ones, ones, v[8], v[9]);
        csa(twosB, ones, ones, v[10], v[11]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, v[12], v[13]);
        csa(twosB, ones, ones, v[14], v[15]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eightsB, fours, fours, foursA, foursB);
        csa(sixteens, eights, eights, eightsA, eightsB);
        uint32_t carry = sixteens;
#pragma unroll
        for (int q = 0; q < NPL - 4; ++q) {
            const uint32_t t = up[q] & carry;
            up[q] ^= carry;
            carry = t;
        }
    }
    __device__ __forceinline__ void planes(uint32_t p[NPL]) const {
        p[0] = ones;
        p[1] = twos;
        p[2] = fours;
        p[3] = eights;
#pragma unroll
        for (int q = 0; q < NPL - 4; ++q) p[4 + q] = up[q];
    }
};

// Adds to c0, c1 the counts of words X0, X1 against the clause records in
// shared memory (m16 = record count rounded up to 16; the padding records are
// all zero, which are never violated: t = 0 = hi_mask selects
// all_false | all_true = 0).
template <int NPL>
__device__ __forceinline__ void count_words2(uint32_t X0, uint32_t X1, int m16, const uint4 *srec,
                                             WordCounter<NPL> &c0, WordCounter<NPL> &c1) {
    const uint32_t xh0 = X0 << 5, xh1 = X1 << 5;
    for (int i0 = 0; i0 < m16; i0 += 16) {
        uint32_t v0[16], v1[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint4 r4 = srec[i0 + j];
            const ClauseRec r{r4.x, r4.y, r4.z, r4.w};
            v0[j] = violation_word(xh0, r);
            v1[j] = violation_word(xh1, r);
        }
        c0.add16(v0);
        c1.add16(v1);
    }
}

// 8x8 bit transpose of a 64-bit word (byte j = row j, bit i = column i).
__device__ __forceinline__ uint64_t transpose8(uint64_t w) {
    uint64_t t;
    t = (w ^ (w >> 7)) & 0x00AA00AA00AA00AAull;
    w ^= t ^ (t << 7);
    t = (w ^ (w >> 14)) & 0x0000CCCC0000CCCCull;
    w ^= t ^ (t << 14);
    t = (w ^ (w >> 28)) & 0x00000000F0F0F0F0ull;
    w ^= t ^ (t << 28);
    return w;
}

// Byte b of the result (b = 0..31) = bits 0..7 of the count of x = 32 X + b.
__device__ __forceinline__ void planes_to_bytes(const uint32_t *planes, uint32_t out[8]) {
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        // row j of the 8x8 block = byte g of plane j
        const uint32_t lo = __byte_perm(__byte_perm(planes[0], planes[1], 0x0040 + g * 0x0011),
                                        __byte_perm(planes[2], planes[3], 0x0040 + g * 0x0011), 0x5410);
        const uint32_t hi = __byte_perm(__byte_perm(planes[4], planes[5], 0x0040 + g * 0x0011),
                                        __byte_perm(planes[6], planes[7], 0x0040 + g * 0x0011), 0x5410);
        const uint64_t w = transpose8(((uint64_t)hi << 32) | lo);
        out[2 * g] = (uint32_t)w;
        out[2 * g + 1] = (uint32_t)(w >> 32);
    }
}

// Writes the 32 counts of word X (bytes) and folds its solution count and max.
// With `mirror` (n >= 6) the same counts also go, byte-reversed, to the
// complement word W - 1 - X, and they count twice.
template <int NPL>
__device__ __forceinline__ void emit_word(int n, uint64_t X, const uint32_t planes[NPL], uint8_t *cost,
                                          unsigned long long &nsol, uint32_t &mx, bool mirror) {
    const uint32_t valid = n >= 5 ? 0xFFFFFFFFu : ((1u << (1u << n)) - 1u);
    uint32_t bytes[8];
    planes_to_bytes(planes, bytes);
    uint32_t any = 0;
    uint32_t over = 0;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
        any |= planes[q];
        if (q >= 8) over |= planes[q];
    }
    nsol += (mirror ? 2u : 1u) * __popc(~any & valid);
    over &= valid;
    uint32_t bm = 0;
    if (n >= 5) {
#pragma unroll
        for (int q = 0; q < 8; ++q) bm = __vmaxu4(bm, bytes[q]);
        bm = max(max(bm & 0xFF, (bm >> 8) & 0xFF), max((bm >> 16) & 0xFF, bm >> 24));
    } else {
        for (uint32_t b = 0; b < (1u << n); ++b) bm = max(bm, (bytes[b >> 2] >> (8 * (b & 3))) & 0xFFu);
    }
    if (over) {  // some count >= 256: take those lanes exactly
        for (uint32_t b = 0; b < 32; ++b)
            if ((over >> b) & 1u) {
                uint32_t c = 0;
                for (int q = 0; q < NPL; ++q) c |= ((planes[q] >> b) & 1u) << q;
                bm = max(bm, c);
            }
    }
    mx = max(mx, bm);
    if (n >= 5) {
        uint4 *dst = reinterpret_cast<uint4 *>(cost + 32 * X);
        dst[0] = make_uint4(bytes[0], bytes[1], bytes[2], bytes[3]);
        dst[1] = make_uint4(bytes[4], bytes[5], bytes[6], bytes[7]);
        if (mirror) {  // byte 31 - b of the complement word holds the count of byte b
            const uint64_t Xm = (1ull << (n - 5)) - 1ull - X;
            uint4 *dm = reinterpret_cast<uint4 *>(cost + 32 * Xm);
            dm[0] = make_uint4(__byte_perm(bytes[7], 0, 0x0123), __byte_perm(bytes[6], 0, 0x0123),
                               __byte_perm(bytes[5], 0, 0x0123), __byte_perm(bytes[4], 0, 0x0123));
            dm[1] = make_uint4(__byte_perm(bytes[3], 0, 0x0123), __byte_perm(bytes[2], 0, 0x0123),
                               __byte_perm(bytes[1], 0, 0x0123), __byte_perm(bytes[0], 0, 0x0123));
        }
    } else {
        for (uint32_t b = 0; b < (1u << n); ++b) cost[b] = (uint8_t)((bytes[b >> 2] >> (8 * (b & 3))) & 0xFFu);
    }
}

constexpr int SUB_WORDS = 2 * CT_THREADS;  // words per block step
constexpr int SUB_BITS = 14;                // log2(32 SUB_WORDS): variables >= 14 are constant over a step

// Keeps the clauses of recs[0, m) (m <= CT_CHUNK; shared or global memory)
// that can be violated somewhere in the words [base, base + SUB_WORDS),
// reduced to variables 5..13, in alive[0, *count), zero-padded to a multiple
// of 16.  Called by all threads of the block.
__device__ __forceinline__ int filter_clauses(uint32_t base, int m, const uint4 *recs, uint4 *alive, int *count) {
    constexpr uint32_t MID = (1u << SUB_BITS) - 32u;  // variables 5..13
    const uint32_t xu = base << 5;                     // x bits >= 14 of the step (bits < 14 are zero)
    if (threadIdx.x == 0) *count = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < m; i0 += CT_THREADS) {
        const int i = i0 + threadIdx.x;
        uint4 r = make_uint4(0, 0, 0, 0);
        bool keep = false;
        if (i < m) {
            r = recs[i];
            const uint32_t umask = r.x & ~MID & ~31u;
            const uint32_t tu = (xu ^ r.y) & umask;
            const bool at = tu == umask, af = tu == 0u;  // uniform literals all true / all false
            keep = at || af;
            r = make_uint4(r.x & MID, r.y & MID, at ? r.z : 0u, af ? r.w : 0u);
        }
        const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, keep);
        int pos = 0;
        if (lane == 0 && ballot) pos = atomicAdd(count, __popc(ballot));
        pos = __shfl_sync(0xFFFFFFFFu, pos, 0) + __popc(ballot & ((1u << lane) - 1u));
        if (keep) alive[pos] = r;
    }
    __syncthreads();
    const int c = *count, c16 = (c + 15) & ~15;
    for (int i = c + threadIdx.x; i < c16; i += CT_THREADS) alive[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    return c16;
}

// One table: each block steps through SUB_WORDS consecutive words at a time;
// thread t takes words base + t and base + CT_THREADS + t, so every clause
// record loaded from shared memory serves 64 assignments.  recs holds the m
// records (shared memory when m <= CT_CHUNK, else global), taken CT_CHUNK at a
// time.
template <int NPL>
__device__ __forceinline__ void cost_table_body(int n, int m, const uint4 *recs, uint4 *alive, int *acount,
                                                uint8_t *cost, unsigned long long *stats, bool mirror) {
    mirror = mirror && n >= 6;  // the lower half is then a whole number of words
    const uint64_t words = n >= 5 ? (1ull << (n - 5)) >> (mirror ? 1 : 0) : 1ull;  // words counted
    const uint64_t steps = (words + SUB_WORDS - 1) / SUB_WORDS;
    unsigned long long nsol = 0;
    uint32_t mx = 0;
    for (uint64_t sb = blockIdx.x; sb < steps; sb += gridDim.x) {
        const uint32_t base = (uint32_t)(sb * SUB_WORDS);
        const uint64_t X0 = base + threadIdx.x, X1 = X0 + CT_THREADS;
        WordCounter<NPL> c0, c1;
        for (int k0 = 0; k0 < m || k0 == 0; k0 += CT_CHUNK) {
            const int mc = m - k0 < CT_CHUNK ? m - k0 : CT_CHUNK;
            const int c16 = filter_clauses(base, mc, recs + k0, alive, acount);
            if (X0 < words) count_words2<NPL>((uint32_t)X0, (uint32_t)(X1 < words ? X1 : X0), c16, alive, c0, c1);
            __syncthreads();  // the list is rebuilt for the next chunk or step
        }
        if (X0 < words) {
            uint32_t p0[NPL], p1[NPL];
            c0.planes(p0);
            c1.planes(p1);
            emit_word<NPL>(n, X0, p0, cost, nsol, mx, mirror);
            if (X1 < words) emit_word<NPL>(n, X1, p1, cost, nsol, mx, mirror);
        }
    }
    // warp then block reduction, one atomic pair per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nsol += __shfl_xor_sync(0xFFFFFFFFu, nsol, o);
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    __shared__ unsigned long long s_sol[CT_THREADS / 32];
    __shared__ uint32_t s_max[CT_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_sol[wid] = nsol;
        s_max[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0;
        uint32_t b = 0;
        for (int w = 0; w < CT_THREADS / 32; ++w) {
            a += s_sol[w];
            b = max(b, s_max[w]);
        }
        if (a) atomicAdd(&stats[0], a);
        atomicMax(&stats[1], (unsigned long long)b);
    }
}

// One table, m <= CT_PARAM_M, the records passed as kernel parameters and
// copied to shared memory once.
__global__ void __launch_bounds__(CT_THREADS) cost_table_kernel(const __grid_constant__ CostParams prm, uint8_t *cost,
                                                                unsigned long long *stats) {
    __shared__ uint4 srec[CT_CHUNK];
    __shared__ uint4 alive[CT_CHUNK];
    __shared__ int acount;
    for (int i = threadIdx.x; i < prm.m; i += CT_THREADS) {
        const ClauseRec r = prm.rec[i];
        srec[i] = make_uint4(r.hi_mask, r.hi_neg, r.all_true, r.all_false);
    }
    __syncthreads();
    cost_table_body<NPL_SMALL>(prm.n, prm.m, srec, alive, &acount, cost, stats, prm.mirror != 0);
}

// Batched tables.  With ns == nullptr every instance has n qubits and its table
// at costs + inst 2^n; otherwise instance inst has ns[inst] qubits and its table
// at costs + offs[inst].  Records of up to CT_CHUNK clauses are copied to
// shared memory once; longer lists are read from global memory chunk by chunk.
template <int NPL>
__global__ void __launch_bounds__(CT_THREADS) cost_table_batch_kernel(int n, const int *ns, const uint64_t *offs,
                                                                      const ClauseRec *recs, const int *ms,
                                                                      int m_stride, uint8_t *costs,
                                                                      unsigned long long *stats, int mirror) {
    static_assert(sizeof(ClauseRec) == sizeof(uint4), "a clause record is one 16-byte load");
    __shared__ uint4 srec[CT_CHUNK];
    __shared__ uint4 alive[CT_CHUNK];
    __shared__ int acount;
    const int inst = blockIdx.y;
    const int m = ms[inst];
    const ClauseRec *g = recs + (size_t)inst * m_stride;
    const uint4 *src = reinterpret_cast<const uint4 *>(g);
    if (m <= CT_CHUNK) {
        for (int i = threadIdx.x; i < m; i += CT_THREADS) {
            const ClauseRec r = g[i];
            srec[i] = make_uint4(r.hi_mask, r.hi_neg, r.all_true, r.all_false);
        }
        __syncthreads();
        src = srec;
    }
    const int ni = ns ? ns[inst] : n;
    uint8_t *dst = ns ? costs + offs[inst] : costs + ((size_t)inst << n);
    cost_table_body<NPL>(ni, m, src, alive, &acount, dst, stats + 2 * inst, mirror != 0);
}

// ---------------------------------------------------------------------------
int validate_instance(const naesat_instance *inst) {
    if (!inst) return set_error(QAOA_EINVAL, "instance is NULL");
    const int n = inst->n, m = inst->m, k = inst->k;
    if (n < 1 || n > QAOA_MAX_N) return set_error(QAOA_ERANGE, "n=%d outside [1, %d]", n, QAOA_MAX_N);
    if (m < 0 || m > QAOA_MAX_M) return set_error(QAOA_ERANGE, "m=%d outside [0, %d]", m, QAOA_MAX_M);
    if (m == 0) return QAOA_OK;
    if (k < 1 || k > n) return set_error(QAOA_ERANGE, "k=%d outside [1, n=%d]", k, n);
    if (!inst->var || !inst->neg) return set_error(QAOA_EINVAL, "var/neg is NULL");
    for (int i = 0; i < m; ++i) {
        uint64_t seen = 0;
        for (int j = 0; j < k; ++j) {
            const int v = inst->var[(size_t)i * k + j];
            const int s = inst->neg[(size_t)i * k + j];
            if (v < 0 || v >= n) return set_error(QAOA_EINVAL, "clause %d: variable %d outside [0, %d)", i, v, n);
            if (s != 0 && s != 1) return set_error(QAOA_EINVAL, "clause %d: negation flag %d not 0/1", i, s);
            if ((seen >> v) & 1ull) return set_error(QAOA_EINVAL, "clause %d: variable %d repeated", i, v);
            seen |= 1ull << v;
        }
    }
    return QAOA_OK;
}

int encode_instance(const naesat_instance *inst, ClauseRec *out) {
    // bit b of COL[v] = bit v of b: the value of variable v < 5 at x = b (mod 32)
    static const uint32_t COL[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    const int m = inst->m, k = inst->k;
    for (int i = 0; i < m; ++i) {
        uint32_t mask = 0, negp = 0, at = 0xFFFFFFFFu, af = 0xFFFFFFFFu;
        for (int j = 0; j < k; ++j) {
            const int v = inst->var[(size_t)i * k + j];
            const uint32_t s = inst->neg[(size_t)i * k + j];
            mask |= 1u << v;
            negp |= s << v;
            if (v < 5) {
                const uint32_t lit = s ? ~COL[v] : COL[v];  // bit b: the literal is true at b
                at &= lit;
                af &= ~lit;
            }
        }
        out[i] = ClauseRec{mask & ~31u, negp & ~31u, at, af};
    }
    return QAOA_OK;
}

static int grid_for(uint64_t words, int batch) {
    DeviceInfo di;
    if (device_info(&di)) return -1;
    const uint64_t need = ((words + 1) / 2 + CT_THREADS - 1) / CT_THREADS;
    uint64_t cap = (uint64_t)di.sms * 8 * 4;
    cap = cap / (uint64_t)batch + 1;
    return (int)(need < cap ? need : cap);
}

int launch_cost_table_batch(int batch, int n, const int *d_ns, const uint64_t *d_offs, const ClauseRec *d_recs,
                            const int *d_m, int m_stride, uint8_t *d_costs, unsigned long long *d_stats,
                            cudaStream_t stream, bool mirror) {
    const uint64_t words = n >= 5 ? (1ull << (n - 5)) >> (mirror && n >= 6 ? 1 : 0) : 1ull;
    const int gx = grid_for(words, batch);
    if (gx < 0) return QAOA_ECUDA;
    const int mi = mirror ? 1 : 0;
    profile_before(K_COST_TABLE, stream);
    if (m_stride <= CT_PARAM_M)
        cost_table_batch_kernel<NPL_SMALL><<<dim3(gx, batch), CT_THREADS, 0, stream>>>(n, d_ns, d_offs, d_recs, d_m,
                                                                                     m_stride, d_costs, d_stats, mi);
    else
        cost_table_batch_kernel<NPL_LARGE><<<dim3(gx, batch), CT_THREADS, 0, stream>>>(n, d_ns, d_offs, d_recs, d_m,
                                                                                     m_stride, d_costs, d_stats, mi);
    return profile_after(K_COST_TABLE, stream);
}

int launch_cost_table_one(const naesat_instance *inst, uint8_t *d_cost, unsigned long long *d_stats,
                          cudaStream_t stream, bool half, void *d_big) {
    // the kernel uses n only for the number of assignments: the half table is
    // the first 2^(n-1) of them (variable n - 1 is 0 there)
    const int n = half ? inst->n - 1 : inst->n;
    if (inst->m > CT_PARAM_M) {
        // records in global memory: d_big holds the m records then the count
        if (!d_big) return set_error(QAOA_EINVAL, "m=%d needs device space for the clause records", inst->m);
        std::vector<ClauseRec> rec((size_t)inst->m);
        encode_instance(inst, rec.data());
        ClauseRec *d_rec = reinterpret_cast<ClauseRec *>(d_big);
        int *d_m = reinterpret_cast<int *>(d_rec + inst->m);
        // pageable sources: the copies return once the data is staged
        QAOA_CUDA_TRY(cudaMemcpyAsync(d_rec, rec.data(), rec.size() * sizeof(ClauseRec), cudaMemcpyHostToDevice, stream));
        QAOA_CUDA_TRY(cudaMemcpyAsync(d_m, &inst->m, sizeof(int), cudaMemcpyHostToDevice, stream));
        return launch_cost_table_batch(1, n, nullptr, nullptr, d_rec, d_m, inst->m, d_cost, d_stats, stream, !half);
    }
    std::vector<char> buf(sizeof(CostParams));
    CostParams *prm = reinterpret_cast<CostParams *>(buf.data());
    prm->n = n;
    prm->m = inst->m;
    prm->mirror = (!half && n >= 6) ? 1 : 0;  // a full table: count its lower half
    encode_instance(inst, prm->rec);
    const uint64_t words = prm->n >= 5 ? (1ull << (prm->n - 5)) >> prm->mirror : 1ull;
    const int gx = grid_for(words, 1);
    if (gx < 0) return QAOA_ECUDA;
    profile_before(K_COST_TABLE, stream);
    cost_table_kernel<<<gx, CT_THREADS, 0, stream>>>(*prm, d_cost, d_stats);
    return profile_after(K_COST_TABLE, stream);
}

size_t cost_table_big_bytes(int m) { return m > CT_PARAM_M ? (size_t)m * sizeof(ClauseRec) + 16 : 0; }

}  // namespace qaoa

using namespace qaoa;

static int cost_table_common(const naesat_instance *inst, uint8_t *d_cost, uint64_t *n_sol, uint32_t *max_cost,
                             void *stream_, bool half) {
    int rc = validate_instance(inst);
    if (rc) return rc;
    if (!d_cost) return set_error(QAOA_EINVAL, "d_cost is NULL");
    if (half && inst->n < 6) return set_error(QAOA_ERANGE, "half table needs n >= 6 (n=%d)", inst->n);
    cudaStream_t stream = (cudaStream_t)stream_;
    Scratch *sc = nullptr;
    rc = scratch_for(stream, 256 + cost_table_big_bytes(inst->m), 64, &sc);
    if (rc) return rc;
    unsigned long long *d_stats = reinterpret_cast<unsigned long long *>(sc->dev);
    QAOA_CUDA_TRY(cudaMemsetAsync(d_stats, 0, 2 * sizeof(unsigned long long), stream));
    rc = launch_cost_table_one(inst, d_cost, d_stats, stream, half, reinterpret_cast<char *>(sc->dev) + 256);
    if (rc) return rc;
    if (!n_sol && !max_cost && inst->m <= 255) return QAOA_OK;
    unsigned long long *h = reinterpret_cast<unsigned long long *>(sc->host);
    QAOA_CUDA_TRY(cudaMemcpyAsync(h, d_stats, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    if (n_sol) *n_sol = half ? 2 * h[0] : h[0];  // C(not x) = C(x): each half solution has its complement
    if (max_cost) *max_cost = (uint32_t)h[1];
    if (h[1] > 255) return set_error(QAOA_ERANGE, "max C = %llu does not fit the uint8 table", h[1]);
    return QAOA_OK;
}

extern "C" int naesat_cost_table(const naesat_instance *inst, uint8_t *d_cost, uint64_t *n_sol, uint32_t *max_cost,
                                 void *stream) {
    return cost_table_common(inst, d_cost, n_sol, max_cost, stream, false);
}

extern "C" int naesat_cost_table_half(const naesat_instance *inst, uint8_t *d_cost_half, uint64_t *n_sol,
                                      uint32_t *max_cost, void *stream) {
    return cost_table_common(inst, d_cost_half, n_sol, max_cost, stream, true);
}

extern "C" int naesat_cost_table_batch(int batch, const naesat_instance *insts, uint8_t *d_costs, uint64_t *n_sol,
                                       uint32_t *max_cost, void *stream_) {
    if (batch < 1 || !insts || !d_costs) return set_error(QAOA_EINVAL, "batch/insts/d_costs");
    const int n = insts[0].n;
    int m_stride = 1;
    for (int b = 0; b < batch; ++b) {
        int rc = validate_instance(&insts[b]);
        if (rc) return rc;
        if (insts[b].n != n) return set_error(QAOA_EINVAL, "batch instances differ in n");
        m_stride = insts[b].m > m_stride ? insts[b].m : m_stride;
    }
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t rec_bytes = (size_t)batch * m_stride * sizeof(ClauseRec);
    const size_t m_bytes = ((size_t)batch * sizeof(int) + 255) & ~(size_t)255;
    const size_t stat_bytes = (size_t)batch * 2 * sizeof(unsigned long long);
    Scratch *sc = nullptr;
    int rc = scratch_for(stream, rec_bytes + m_bytes + stat_bytes + 512, rec_bytes + m_bytes + stat_bytes + 512, &sc);
    if (rc) return rc;
    char *hbase = reinterpret_cast<char *>(sc->host);
    char *dbase = reinterpret_cast<char *>(sc->dev);
    ClauseRec *h_recs = reinterpret_cast<ClauseRec *>(hbase);
    int *h_m = reinterpret_cast<int *>(hbase + rec_bytes);
    for (int b = 0; b < batch; ++b) {
        encode_instance(&insts[b], h_recs + (size_t)b * m_stride);
        h_m[b] = insts[b].m;
    }
    QAOA_CUDA_TRY(cudaMemcpyAsync(dbase, hbase, rec_bytes + m_bytes, cudaMemcpyHostToDevice, stream));
    unsigned long long *d_stats = reinterpret_cast<unsigned long long *>(dbase + rec_bytes + m_bytes);
    QAOA_CUDA_TRY(cudaMemsetAsync(d_stats, 0, stat_bytes, stream));
    rc = launch_cost_table_batch(batch, n, nullptr, nullptr, reinterpret_cast<const ClauseRec *>(dbase),
                                 reinterpret_cast<const int *>(dbase + rec_bytes), m_stride, d_costs, d_stats, stream,
                                 true);
    if (rc) return rc;
    unsigned long long *h_stats = reinterpret_cast<unsigned long long *>(hbase + rec_bytes + m_bytes);
    QAOA_CUDA_TRY(cudaMemcpyAsync(h_stats, d_stats, stat_bytes, cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));  // the pinned staging block is reused by the next call
    int status = QAOA_OK;
    for (int b = 0; b < batch; ++b) {
        if (n_sol) n_sol[b] = h_stats[2 * b];
        if (max_cost) max_cost[b] = (uint32_t)h_stats[2 * b + 1];
        if (h_stats[2 * b + 1] > 255 && status == QAOA_OK)
            status = set_error(QAOA_ERANGE, "instance %d: max C = %llu does not fit the uint8 table", b, h_stats[2 * b + 1]);
    }
    return status;
}
