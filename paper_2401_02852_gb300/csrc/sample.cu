// K7: bitstrings drawn from the output state, and instance running times
// (Sec. "Running Times": measuring the final state yields x with probability
// |Psi(x)|^2; the running time of an instance is the number of draws up to and
// including the first one that satisfies it).
//
// Inverse-CDF sampling with caller-supplied uniforms u_j in [0, 1): draw j is
// the smallest x with F(x) > u_j F_total, F(x) = sum_{y <= x} |psi(y)|^2.
//
// Two-level prefix: an entry is 32 amplitudes, a group 256 entries (2^13
// amplitudes).  Within a group the probabilities are integer weights on a
// per-group binary scale (see weight()), so the entry prefix Q of a group is
// exact and a draw's scan of its entry re-forms the same integers: the entry
// and amplitude levels agree to the unit, in any summation order.  Only the
// group totals are FP64, and their prefix P is formed serially (fixed order).
//   1. entry_scan_kernel: one CTA per group: the group's largest probability
//      sets its scale E_g; each thread sums its entry's weights; an exact
//      warp/block scan gives Q; the group total goes to FP64;
//   2. block_prefix_kernel: inclusive prefix P of the group totals;
//   3. draw_kernel: one warp per draw: a 32-way search over P (doubles >= +0
//      compared as integers), the remainder in the group's units, a 32-way
//      search over Q, then an integer warp scan over the entry's 32 weights.
// The draws differ from a sequential FP64 scan of the probabilities only for
// a u_j within about 2^-40 of a step of F (the weights' quantisation).
// GB300's FP64 pipe is narrow: apart from a few operations per draw and per
// group, the sampler runs on the FP32 pipes and the integer ALUs.
// With QAOA_Z2_HALF the stored half holds the x with bit n-1 clear and
// |psi(not x)| = |psi(x)| (Sec. 2.2's global flip): t = u 2 F_half picks the
// stored x (t < F_half) or the complement of the x drawn at t - F_half.
#include <cuda_runtime.h>

#include <cmath>

#include "pass_common.cuh"
#include "qaoa_internal.cuh"

namespace qaoa {

constexpr int ENTRY_BITS = 5;    // log2 amplitudes per entry
constexpr int GROUP_BITS = 8;    // log2 entries per group
constexpr int GROUP = 1 << GROUP_BITS;
constexpr int PREFIX_PT = 1024;  // threads of the group-prefix kernel
constexpr int DRAW_WARPS = 8;    // draws per CTA of the draw kernel
constexpr int W_TOP = 44;        // a group's largest probability scales into [2^44, 2^46)

// Entry and group counts of a stored state of 2^ns amplitudes.
__host__ __device__ __forceinline__ uint64_t entry_count(int ns) {
    return ns > ENTRY_BITS ? 1ull << (ns - ENTRY_BITS) : 1ull;
}
__host__ __device__ __forceinline__ uint64_t group_count(int ns) {
    return (entry_count(ns) + GROUP - 1) >> GROUP_BITS;
}

// ---- fixed-point weights ------------------------------------------------------
// In group g every probability is taken as the integer
//   W(x) = |psi(x)|^2 2^E_g, to about 2^-44 of the group's largest one,
// with E_g even and set by that largest probability (it lands in
// [2^44, 2^46)), so an entry (32 amplitudes) sums below 2^51 and a group below
// 2^59.  Integer sums are exact in any order: the entry prefix of a group is
// the exact running sum of its entries' W, and a draw re-forms the same W of
// its entry's 32 amplitudes, so the levels agree to the unit.  complex64:
// the components are scaled by 2^(E/2) (exact), squared exactly as p + e (the
// FMA form of Dekker's TwoProduct), p_re + p_im split by Knuth's TwoSum, and
// W = trunc(s) + trunc(rest of the sum): FP32 and integer operations.
// complex128: |psi|^2 in FP64, scaled and truncated by integer operations.

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }       // e in [-126, 127]
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// trunc(f) for |f| < 2^63 from the float's bits with integer operations (the
// float-to-int64 conversion instruction runs on the FP64 pipe).
__device__ __forceinline__ long long trunc_ll(float f) {
    const uint32_t b = __float_as_uint(f);
    const int ex = (int)((b >> 23) & 0xFFu);
    const uint32_t mant = (b & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
    const int sh = (ex ? ex : 1) - 150;  // |f| = mant 2^sh
    const long long v = sh >= 0 ? (long long)((unsigned long long)mant << sh) : (sh > -24 ? (long long)(mant >> -sh) : 0);
    return (b >> 31) ? -v : v;
}

// trunc(v 2^E) for a double v from its bits with integer operations: the
// scaling only moves the exponent, so this is exact; v <= 0 (and a subnormal
// v, whose v 2^E is below 1 for |E| <= 200) gives 0, and results at or above
// 2^62 (beyond any group total) saturate there.
__device__ __forceinline__ long long scaled_trunc(double v, int E) {
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (b <= 0 || ex == 0) return 0;
    const long long mant = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);  // v = mant 2^(ex - 1075)
    const int sh = ex - 1075 + E;
    if (sh >= 10) return 1LL << 62;  // mant >= 2^52
    return sh >= 0 ? mant << sh : (sh > -53 ? mant >> -sh : 0);
}

__device__ __forceinline__ long long weight(float2 z, int E) {
    const float sc = pow2f(E / 2);
    const float re = __fmul_rn(z.x, sc), im = __fmul_rn(z.y, sc);
    const float pr = __fmul_rn(re, re), er = __fmaf_rn(re, re, -pr);
    const float pi = __fmul_rn(im, im), ei = __fmaf_rn(im, im, -pi);
    float s, e;
    df_two_sum(pr, pi, s, e);
    const float t = __fadd_rn(__fadd_rn(e, er), ei);
    return trunc_ll(s) + trunc_ll(t);
}
__device__ __forceinline__ long long weight(double2 z, int E) {
    return scaled_trunc(z.x * z.x + z.y * z.y, E);
}
// |psi(x)|^2 as a float (to choose E) and the exponent that scales a maximum m.
__device__ __forceinline__ float prob_f(float2 z) { return z.x * z.x + z.y * z.y; }
__device__ __forceinline__ float prob_f(double2 z) { return (float)(z.x * z.x + z.y * z.y); }
__device__ __forceinline__ int scale_exp(float m) {
    if (!(m > 0.f)) return 0;
    const int e = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 127;  // m in [2^e, 2^(e+1)) (normal m)
    int E = W_TOP - (e > -127 ? e : -126);
    E &= ~1;  // even: the components take 2^(E/2)
    return E < -200 ? -200 : (E > 200 ? 200 : E);
}

// Group g = blockIdx.x of instance blockIdx.y: E[g], the inclusive prefix Q
// (int64) of its entries' weights, and the group total G[g] = Q_last 2^-E_g
// in FP64.  With STAGED (complex64 states at 16-byte aligned addresses) the
// group is first staged in shared memory (dynamic, STAGE_BYTES) with
// coalesced 16-byte loads, pair j of entry e at float4 slot
// 16 e + ((j + e) & 15): the loads' and the entry reads' quarter-warps hit
// eight distinct bank quads.
constexpr int STAGE_PAIRS = 1 << (GROUP_BITS + ENTRY_BITS - 1);
constexpr size_t STAGE_BYTES = sizeof(float4) * STAGE_PAIRS;
template <typename V, bool STAGED>
__global__ void __launch_bounds__(GROUP) entry_scan_kernel(const V *states, int ns, long long *Q, int *Eg,
                                                           double *G) {
    __shared__ long long wsum[GROUP / 32];
    __shared__ unsigned int smax;
    const uint64_t N = 1ull << ns, ne = entry_count(ns), ng = group_count(ns);
    const uint64_t inst = blockIdx.y;
    const V *st = states + (inst << ns);
    const uint32_t el = threadIdx.x;
    const uint64_t e = ((uint64_t)blockIdx.x << GROUP_BITS) + el;
    const uint64_t x0 = e << ENTRY_BITS;
    const uint32_t cnt = e < ne ? (uint32_t)(N - x0 < 32 ? N - x0 : 32) : 0u;  // amplitudes of this entry
    if (el == 0) smax = 0u;
    const float4 *stage = nullptr;
    if constexpr (STAGED) {
        static_assert(sizeof(V) == 8, "complex64 only");
        extern __shared__ float4 stage_buf[];
        const uint64_t gx0 = (uint64_t)blockIdx.x << (GROUP_BITS + ENTRY_BITS);  // first amplitude (even)
        const uint64_t left = (N - gx0) / 2;  // N even: ns >= 1
        const uint32_t np = left < (uint64_t)STAGE_PAIRS ? (uint32_t)left : (uint32_t)STAGE_PAIRS;
        const float4 *src = reinterpret_cast<const float4 *>(st + gx0);
        for (uint32_t q = threadIdx.x; q < np; q += GROUP) {
            const uint32_t qe = q >> (ENTRY_BITS - 1), qj = q & 15u;
            stage_buf[16 * qe + ((qj + qe) & 15u)] = src[q];
        }
        stage = stage_buf;
    }
    // amplitude i (< cnt) of this thread's entry
    auto amp = [&](uint32_t i) -> V {
        if constexpr (STAGED) {
            const float4 w = stage[16 * el + (((i >> 1) + el) & 15u)];
            return (i & 1u) ? make_float2(w.z, w.w) : make_float2(w.x, w.y);
        } else {
            return st[x0 + i];
        }
    };
    __syncthreads();  // staged tile and smax
    float m = 0.f;
    for (uint32_t i = 0; i < cnt; ++i) m = fmaxf(m, prob_f(amp(i)));
    atomicMax(&smax, __float_as_uint(m));  // nonnegative floats order as their bits
    __syncthreads();
    const int E = scale_exp(__uint_as_float(smax));
    long long wv = 0;
    for (uint32_t i = 0; i < cnt; ++i) wv += weight(amp(i), E);
    // inclusive scan over the group's 256 entries (exact integer sums)
    const int lane = el & 31, w = el >> 5;
    long long incl = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    long long off = 0;
    for (int i = 0; i < w; ++i) off += wsum[i];
    incl += off;
    if (e < ne) Q[inst * ne + e] = incl;
    const uint64_t gl = ne - ((uint64_t)blockIdx.x << GROUP_BITS);  // entries of this group
    if ((uint64_t)el == (gl < (uint64_t)GROUP ? gl : (uint64_t)GROUP) - 1) {
        G[inst * ng + blockIdx.x] = (double)incl * pow2d(-E);
        Eg[inst * ng + blockIdx.x] = E;
    }
}

// In place, per instance (one CTA each): sums[b] <- sums[0] + ... + sums[b].
// Each thread forms serial running sums over a contiguous chunk, thread 0
// turns the chunk totals into offsets in order, then each thread adds its
// offset; the last value of a chunk equals the next chunk's offset, so the
// result is nondecreasing and rises only where a sum is nonzero.
__global__ void __launch_bounds__(PREFIX_PT) block_prefix_kernel(double *sums, uint64_t nb) {
    __shared__ double chunk[PREFIX_PT];
    double *s = sums + (uint64_t)blockIdx.x * nb;
    const uint64_t per = (nb + PREFIX_PT - 1) / PREFIX_PT;
    const uint64_t lo = threadIdx.x * per < nb ? threadIdx.x * per : nb;
    const uint64_t hi = lo + per < nb ? lo + per : nb;
    double r = 0.0;
    for (uint64_t i = lo; i < hi; ++i) {
        r += s[i];
        s[i] = r;
    }
    chunk[threadIdx.x] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int t = 0; t < PREFIX_PT; ++t) {
            const double v = chunk[t];
            chunk[t] = acc;
            acc = acc + v;
        }
    }
    __syncthreads();
    const double o = chunk[threadIdx.x];
    for (uint64_t i = lo; i < hi; ++i) s[i] = o + s[i];
}

// Doubles >= +0 compare as their bit patterns do (as signed 64-bit integers),
// which keeps the group search off the FP64 pipe.
__device__ __forceinline__ long long ord(double v) { return __double_as_longlong(v); }

// Smallest i in [0, len) with key(A[i]) > kb (A nondecreasing, the last one
// qualifies), or >= kb when `ge`; a 32-way search by the whole warp
// (len < 2^31: at most 2^19 groups, 256 entries).
template <typename T, typename K>
__device__ __forceinline__ uint32_t warp_search(const T *A, uint32_t len, long long kb, bool ge, K key) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = len;  // the answer is in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t stride = (hi - lo + 31) / 32;
        uint32_t i = lo + (lane + 1) * stride - 1;
        if (i > hi - 1) i = hi - 1;
        const long long v = key(A[i]);
        const unsigned ok = __ballot_sync(0xFFFFFFFFu, ge ? v >= kb : v > kb);
        const uint32_t f = (uint32_t)(__ffs(ok) - 1);  // A[hi - 1] qualifies, so ok != 0
        const uint32_t nlo = lo + f * stride;
        hi = nlo + stride < hi ? nlo + stride : hi;
        lo = nlo;
    }
    return lo;
}

// One warp per draw j of instance blockIdx.y: x_j = min { x : F(x) > t } with
// t = u_j F_total.  The group comes from the FP64 prefix P; within it the
// remainder becomes the group's integer units and the rest is exact: the
// entry from Q, then the first amplitude whose running weight passes it.
// When t is at F_total, or the remainder at or past the group's integer total
// (the FP64 group totals are rounded), the last x of nonzero weight of the
// group is taken; a state of norm zero draws 0.
template <typename V>
__global__ void __launch_bounds__(DRAW_WARPS * 32) draw_kernel(const V *states, int ns, int z2, const long long *Q,
                                                                 const int *Eg, const double *P, int k,
                                                                 const double *u, uint64_t *xs) {
    const int lane = threadIdx.x & 31;
    const uint64_t j = (uint64_t)blockIdx.x * DRAW_WARPS + (threadIdx.x >> 5);
    if (j >= (uint64_t)k) return;  // whole warps leave together
    const uint64_t inst = blockIdx.y;
    const uint64_t N = 1ull << ns, ne = entry_count(ns), ng = group_count(ns);
    const V *st = states + (inst << ns);
    const double *Pi = P + inst * ng;
    const double total = Pi[ng - 1];
    double uj = u[inst * (uint64_t)k + j];
    // u <= 0 (or NaN) draws the first x of nonzero probability; the test on the
    // bits keeps it off the FP64 pipe (+inf and below are the non-NaN doubles)
    const long long ub = ord(uj);
    uj = ub > 0 && ub <= 0x7FF0000000000000LL ? uj : 0.0;
    double t = uj * total;
    if (z2) t += t;  // u 2 F_half
    bool flip = false;
    if (z2 && ord(total) > 0 && ord(t) >= ord(total)) {
        flip = true;
        t -= total;
    }
    // group (t and the sums are >= +0)
    bool edge = ord(t) >= ord(total);
    auto dkey = [](double v) { return ord(v); };
    const uint64_t g = warp_search(Pi, (uint32_t)ng, ord(edge ? total : t), edge, dkey);
    const int E = Eg[inst * ng + g];
    // the remainder in the group's integer units
    const uint64_t e0 = g << GROUP_BITS;
    const uint64_t glen = ne - e0 < (uint64_t)GROUP ? ne - e0 : (uint64_t)GROUP;
    const long long *Qg = Q + inst * ne + e0;
    const long long Ig = Qg[glen - 1];
    long long R = 0;
    if (!edge) {
        R = scaled_trunc(t - (g > 0 ? Pi[g - 1] : 0.0), E);  // P[g-1] <= t
        edge = R >= Ig;
    }
    auto ikey = [](long long v) { return v; };
    const uint64_t e = warp_search(Qg, (uint32_t)glen, edge ? Ig : R, edge, ikey);
    R -= e > 0 ? Qg[e - 1] : 0;
    // amplitude within the entry: exact integer running weights
    const uint64_t x = ((e0 + e) << ENTRY_BITS) + (uint64_t)lane;
    const long long wv = x < N ? weight(st[x], E) : 0;
    long long incl = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned hit = __ballot_sync(0xFFFFFFFFu, !edge && incl > R);
    const unsigned nz = __ballot_sync(0xFFFFFFFFu, wv > 0);
    const int pick = hit ? __ffs(hit) - 1 : (nz ? 31 - __clz(nz) : 0);
    if (lane == 0) {
        const uint64_t found = ((e0 + e) << ENTRY_BITS) + (uint64_t)pick;
        const uint64_t full = (1ull << (ns + (z2 ? 1 : 0))) - 1ull;
        xs[inst * (uint64_t)k + j] = flip ? (~found & full) : found;
    }
}

// first[inst] = min j with C(x_j) = 0 (left untouched when no draw satisfies).
// With a half table (z2) an x with bit n-1 set is looked up as its complement,
// C(not x) = C(x).
__global__ void first_hit_kernel(const uint8_t *costs, int nc, int z2, int k, const uint64_t *xs, int *first) {
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t inst = blockIdx.y;
    if (j >= (uint64_t)k) return;
    const uint64_t mask = (1ull << nc) - 1ull;
    uint64_t x = xs[inst * (uint64_t)k + j];
    if (z2 && ((x >> nc) & 1ull)) x = ~x;
    if (costs[(inst << nc) + (x & mask)] == 0) atomicMin(first + inst, (int)j);
}

// ---------------------------------------------------------------------------
static int sample_impl(int batch, int n, const uint8_t *d_costs, const void *d_states, int dtype, int flags, int k,
                       const double *d_u, uint64_t *d_x, int64_t *running_time, cudaStream_t stream) {
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", dtype);
    const bool z2 = (flags & QAOA_Z2_HALF) != 0;
    if (flags & ~(QAOA_Z2_HALF | QAOA_MIXER_RX2B)) return set_error(QAOA_EINVAL, "flags=0x%x", flags);
    if (n < (z2 ? 2 : 1) || n > QAOA_MAX_N) return set_error(QAOA_ERANGE, "n=%d", n);
    if (batch < 1 || batch > 65535) return set_error(QAOA_ERANGE, "batch=%d", batch);
    if (k < 1 || k > (1 << 30)) return set_error(QAOA_ERANGE, "k=%d", k);
    if (!d_states || !d_u) return set_error(QAOA_EINVAL, "NULL state or uniforms");
    if (running_time && !d_costs) return set_error(QAOA_EINVAL, "running time needs the cost table");
    if (!running_time && !d_x) return set_error(QAOA_EINVAL, "nowhere to put the draws");
    const int ns = z2 ? n - 1 : n;  // index bits of the stored state and of its table
    const uint64_t ne = entry_count(ns), ng = group_count(ns);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t qb = al(sizeof(long long) * ne * (size_t)batch);
    const size_t eb = al(sizeof(int) * ng * (size_t)batch);
    const size_t pre = qb + eb + al(sizeof(double) * ng * (size_t)batch);
    const size_t xb = d_x ? 0 : sizeof(uint64_t) * (size_t)k * batch;
    const size_t fb = sizeof(int) * (size_t)batch;
    Scratch *sc = nullptr;
    int rc = scratch_for(stream, pre + xb + fb + 64, fb + 64, &sc);
    if (rc) return rc;
    char *dev = reinterpret_cast<char *>(sc->dev);
    long long *d_q = reinterpret_cast<long long *>(dev);
    int *d_e = reinterpret_cast<int *>(dev + qb);
    double *d_pre = reinterpret_cast<double *>(dev + qb + eb);
    uint64_t *xs = d_x ? d_x : reinterpret_cast<uint64_t *>(dev + pre);
    int *d_first = reinterpret_cast<int *>(dev + pre + xb);
    const dim3 draw_grid((unsigned)((k + DRAW_WARPS - 1) / DRAW_WARPS), batch);
    profile_before(K_SAMPLE, stream);
    if (dtype == QAOA_C64) {
        const float2 *st = reinterpret_cast<const float2 *>(d_states);
        if ((reinterpret_cast<uintptr_t>(d_states) & 15u) == 0) {
            // per call: the attribute belongs to the current device
            const cudaError_t attr = cudaFuncSetAttribute(
                entry_scan_kernel<float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STAGE_BYTES);
            if (attr != cudaSuccess) return cuda_error(attr, "entry scan shared memory");
            entry_scan_kernel<float2, true><<<dim3((unsigned)ng, batch), GROUP, STAGE_BYTES, stream>>>(st, ns, d_q,
                                                                                                      d_e, d_pre);
        } else {
            entry_scan_kernel<float2, false><<<dim3((unsigned)ng, batch), GROUP, 0, stream>>>(st, ns, d_q, d_e, d_pre);
        }
        block_prefix_kernel<<<batch, PREFIX_PT, 0, stream>>>(d_pre, ng);
        draw_kernel<float2><<<draw_grid, DRAW_WARPS * 32, 0, stream>>>(st, ns, z2 ? 1 : 0, d_q, d_e, d_pre, k, d_u,
                                                                       xs);
    } else {
        const double2 *st = reinterpret_cast<const double2 *>(d_states);
        entry_scan_kernel<double2, false><<<dim3((unsigned)ng, batch), GROUP, 0, stream>>>(st, ns, d_q, d_e, d_pre);
        block_prefix_kernel<<<batch, PREFIX_PT, 0, stream>>>(d_pre, ng);
        draw_kernel<double2><<<draw_grid, DRAW_WARPS * 32, 0, stream>>>(st, ns, z2 ? 1 : 0, d_q, d_e, d_pre, k, d_u,
                                                                        xs);
    }
    rc = profile_after(K_SAMPLE, stream);
    if (rc || !running_time) return rc;
    QAOA_CUDA_TRY(cudaMemsetAsync(d_first, 0x7F, fb, stream));  // 0x7F7F7F7F > any draw index
    first_hit_kernel<<<dim3((unsigned)((k + 255) / 256), batch), 256, 0, stream>>>(d_costs, ns, z2 ? 1 : 0, k, xs,
                                                                                    d_first);
    QAOA_CUDA_TRY(cudaGetLastError());
    int *h = reinterpret_cast<int *>(sc->host);
    QAOA_CUDA_TRY(cudaMemcpyAsync(h, d_first, fb, cudaMemcpyDeviceToHost, stream));
    QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
    for (int i = 0; i < batch; ++i) running_time[i] = h[i] >= k ? 0 : (int64_t)h[i] + 1;
    return QAOA_OK;
}

}  // namespace qaoa

using namespace qaoa;

extern "C" int qaoa_sample(int n, const void *d_state, int dtype, int flags, int k, const double *d_u, uint64_t *d_x,
                           void *stream) {
    if (!d_x) return set_error(QAOA_EINVAL, "d_x is NULL");
    return sample_impl(1, n, nullptr, d_state, dtype, flags, k, d_u, d_x, nullptr, (cudaStream_t)stream);
}

extern "C" int qaoa_running_time(int n, const uint8_t *d_cost, const void *d_state, int dtype, int flags, int k,
                                 const double *d_u, int64_t *running_time, uint64_t *d_x, void *stream) {
    if (!running_time) return set_error(QAOA_EINVAL, "running_time is NULL");
    return sample_impl(1, n, d_cost, d_state, dtype, flags, k, d_u, d_x, running_time, (cudaStream_t)stream);
}

extern "C" int qaoa_running_time_batch(int batch, int n, const uint8_t *d_costs, const void *d_states, int dtype,
                                       int flags, int k, const double *d_u, int64_t *running_time, void *stream) {
    if (!running_time) return set_error(QAOA_EINVAL, "running_time is NULL");
    return sample_impl(batch, n, d_costs, d_states, dtype, flags, k, d_u, nullptr, running_time,
                       (cudaStream_t)stream);
}
