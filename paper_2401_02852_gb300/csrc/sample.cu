// K7: bitstrings drawn from the output state, and instance running times
// (Sec. "Running Times": measuring the final state yields x with probability
// |Psi(x)|^2; the running time of an instance is the number of draws up to and
// including the first one that satisfies it).
//
// Inverse-CDF sampling with caller-supplied uniforms u_j in [0, 1): draw j is
// the smallest x with F(x) > u_j F_total, F(x) = sum_{y <= x} |psi(y)|^2.  The
// sums are formed in FP64 (complex64 entry sums in double-float arithmetic
// with exact squares, about 2^-44 relative), so the result differs from a
// sequential FP64 scan only through rounding, i.e. only for a u_j within
// rounding of a step of F.
//
// Two-level prefix.  An entry is 32 consecutive amplitudes, a group 256
// entries (2^13 amplitudes).
//   1. entry_scan_kernel: one CTA per group: each thread sums one entry in
//      index order (complex64: on the FP32 pipes, see entry_sum), then the CTA
//      forms the inclusive prefix Q of its 256 entry sums (fixed order) and
//      writes the group total;
//   2. block_prefix_kernel: inclusive prefix P of the group totals, fixed order;
//   3. draw_kernel: one warp per draw: 32-way searches over P and over the
//      group's Q, then one FP64 warp scan over the chosen entry's 32
//      amplitudes.
// GB300's FP64 pipe is narrow, so a draw forms only those 32 probabilities in
// FP64; the searches compare the stored nonnegative sums as integers (the bit
// patterns of doubles >= +0 order as the values do).
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

template <typename V>
__device__ __forceinline__ double prob(const V &z) {
    const double re = (double)z.x, im = (double)z.y;
    return re * re + im * im;
}

// Sum of |psi(x)|^2 over x in [x0, x1), in index order.  complex64: the
// squares are exact as p + e (FMA form of Dekker's TwoProduct), each p is
// added to a double-float accumulator with Knuth's TwoSum and the rounding
// errors collect in its low word, all on the FP32 pipes; complex128: FP64.
__device__ __forceinline__ double entry_sum(const float2 *st, uint64_t x0, uint64_t x1) {
    float hi = 0.f, lo = 0.f;
    for (uint64_t x = x0; x < x1; ++x) {
        const float2 z = st[x];
        const float pr = __fmul_rn(z.x, z.x), er = __fmaf_rn(z.x, z.x, -pr);
        const float pi = __fmul_rn(z.y, z.y), ei = __fmaf_rn(z.y, z.y, -pi);
        float s, e;
        df_two_sum(hi, pr, s, e);
        lo = __fadd_rn(lo, __fadd_rn(e, er));
        df_two_sum(s, pi, hi, e);
        lo = __fadd_rn(lo, __fadd_rn(e, ei));
    }
    return (double)hi + (double)lo;  // exact: hi + lo fits a double
}
// complex64, from a staged group: entry el's amplitudes 2j, 2j + 1 sit in the
// float4 at stage[16 el + ((j + el) & 15)] (see entry_scan_kernel); `pairs`
// of them, summed as above in index order.
__device__ __forceinline__ double entry_sum_staged(const float4 *stage, uint32_t el, uint32_t pairs) {
    float hi = 0.f, lo = 0.f;
    auto add = [&](float zx, float zy) {
        const float pr = __fmul_rn(zx, zx), er = __fmaf_rn(zx, zx, -pr);
        const float pi = __fmul_rn(zy, zy), ei = __fmaf_rn(zy, zy, -pi);
        float s, e;
        df_two_sum(hi, pr, s, e);
        lo = __fadd_rn(lo, __fadd_rn(e, er));
        df_two_sum(s, pi, hi, e);
        lo = __fadd_rn(lo, __fadd_rn(e, ei));
    };
    for (uint32_t j = 0; j < pairs; ++j) {
        const float4 w = stage[16 * el + ((j + el) & 15)];
        add(w.x, w.y);
        add(w.z, w.w);
    }
    return (double)hi + (double)lo;
}
__device__ __forceinline__ double entry_sum(const double2 *st, uint64_t x0, uint64_t x1) {
    double s = 0.0;
    for (uint64_t x = x0; x < x1; ++x) s += prob(st[x]);
    return s;
}

// |z|^2 of a complex64 amplitude as a normalised double-float (hi, lo): the
// squares exact by FMA, their sum by TwoSum.
__device__ __forceinline__ void prob_df(float2 z, float &hi, float &lo) {
    const float pr = __fmul_rn(z.x, z.x), er = __fmaf_rn(z.x, z.x, -pr);
    const float pi = __fmul_rn(z.y, z.y), ei = __fmaf_rn(z.y, z.y, -pi);
    float s, e;
    df_two_sum(pr, pi, s, e);
    df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(er, ei)), hi, lo);
}
// (ah, al) + (bh, bl), normalised.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &h, float &l) {
    float s, e;
    df_two_sum(ah, bh, s, e);
    df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(al, bl)), h, l);
}
// x > y for normalised double-floats (hi decides unless equal).
__device__ __forceinline__ bool df_greater(float xh, float xl, float yh, float yl) {
    return xh > yh || (xh == yh && xl > yl);
}

// The chosen entry's draw: the first lane x with w(x) > 0 whose inclusive
// prefix exceeds rest (a warp scan), or when none does (edge, or the
// remainder at the entry's rounded sum) the last lane with w > 0; -1 when
// every w is 0.  complex64: probabilities and scan in double-float on the
// FP32 pipes, rest split into a double-float; complex128: FP64.
__device__ __forceinline__ int entry_pick(float2 z, bool valid, double rest, bool edge) {
    const int lane = threadIdx.x & 31;
    float wh = 0.f, wl = 0.f;
    if (valid) prob_df(z, wh, wl);
    float ih = wh, il = wl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float yh = __shfl_up_sync(0xFFFFFFFFu, ih, o), yl = __shfl_up_sync(0xFFFFFFFFu, il, o);
        if (lane >= o) df_add(ih, il, yh, yl, ih, il);
    }
    const float rh = __double2float_rn(rest);
    const float rl = __double2float_rn(rest - (double)rh);
    const unsigned hit = __ballot_sync(0xFFFFFFFFu, !edge && wh > 0.f && df_greater(ih, il, rh, rl));
    const unsigned nz = __ballot_sync(0xFFFFFFFFu, wh > 0.f);
    return hit ? __ffs(hit) - 1 : (nz ? 31 - __clz(nz) : -1);
}
__device__ __forceinline__ int entry_pick(double2 z, bool valid, double rest, bool edge) {
    const int lane = threadIdx.x & 31;
    const double w = valid ? prob(z) : 0.0;
    double incl = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned hit = __ballot_sync(0xFFFFFFFFu, !edge && w > 0.0 && incl > rest);
    const unsigned nz = __ballot_sync(0xFFFFFFFFu, w > 0.0);
    return hit ? __ffs(hit) - 1 : (nz ? 31 - __clz(nz) : -1);
}

// Entry and group counts of a stored state of 2^ns amplitudes.
__host__ __device__ __forceinline__ uint64_t entry_count(int ns) {
    return ns > ENTRY_BITS ? 1ull << (ns - ENTRY_BITS) : 1ull;
}
__host__ __device__ __forceinline__ uint64_t group_count(int ns) {
    return (entry_count(ns) + GROUP - 1) >> GROUP_BITS;
}

// Group g = blockIdx.x of instance blockIdx.y: Q[e] = sum of the entry sums of
// the group up to entry e (inclusive), G[g] = the group's total (= Q at its
// last entry).  The running sums are serial within each warp's 32 entries and
// offset by the serial sums of the earlier warps' totals, so Q is
// nondecreasing and Q[e] > Q[e - 1] only where entry e has a nonzero sum.
// With STAGED (complex64 states at 16-byte aligned addresses) the group is
// first staged in shared memory (dynamic, STAGE_BYTES) with coalesced 16-byte
// loads, pair j of entry e at float4 slot 16 e + ((j + e) & 15): the loads'
// quarter-warps write, and the entry reads' quarter-warps read, eight
// distinct bank quads.
constexpr int STAGE_PAIRS = 1 << (GROUP_BITS + ENTRY_BITS - 1);
constexpr size_t STAGE_BYTES = sizeof(float4) * STAGE_PAIRS;
template <typename V, bool STAGED>
__global__ void __launch_bounds__(GROUP) entry_scan_kernel(const V *states, int ns, double *Q, double *G) {
    __shared__ double run[GROUP];
    __shared__ double off[GROUP / 32];
    const uint64_t N = 1ull << ns, ne = entry_count(ns), ng = group_count(ns);
    const uint64_t inst = blockIdx.y;
    const V *st = states + (inst << ns);
    const uint64_t e = ((uint64_t)blockIdx.x << GROUP_BITS) + threadIdx.x;
    double s = 0.0;
    if constexpr (STAGED) {
        static_assert(sizeof(V) == 8, "complex64 only");
        extern __shared__ float4 stage[];
        const uint64_t gx0 = (uint64_t)blockIdx.x << (GROUP_BITS + ENTRY_BITS);  // first amplitude (even)
        const uint64_t left = (N - gx0) / 2;  // N even: ns >= 1
        const uint32_t np = left < (uint64_t)STAGE_PAIRS ? (uint32_t)left : (uint32_t)STAGE_PAIRS;
        const float4 *src = reinterpret_cast<const float4 *>(st + gx0);
        for (uint32_t q = threadIdx.x; q < np; q += GROUP) {
            const uint32_t qe = q >> (ENTRY_BITS - 1), qj = q & 15u;
            stage[16 * qe + ((qj + qe) & 15u)] = src[q];
        }
        __syncthreads();
        if (e < ne) {
            const uint32_t el = threadIdx.x;
            const uint32_t pairs = np > 16 * el ? (np - 16 * el < 16u ? np - 16 * el : 16u) : 0u;
            s = entry_sum_staged(stage, el, pairs);
        }
    } else if (e < ne) {
        const uint64_t x0 = e << ENTRY_BITS, x1 = x0 + 32 < N ? x0 + 32 : N;
        s = entry_sum(st, x0, x1);
    }
    run[threadIdx.x] = s;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {  // serial running sums of this warp's entries
        double r = 0.0;
        for (int i = 0; i < 32; ++i) {
            r += run[32 * w + i];
            run[32 * w + i] = r;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // warp totals -> offsets, in order
        double r = 0.0;
        for (int i = 0; i < GROUP / 32; ++i) {
            off[i] = r;
            r = r + run[32 * i + 31];
        }
    }
    __syncthreads();
    const double q = off[w] + run[threadIdx.x];
    if (e < ne) Q[inst * ne + e] = q;
    const uint64_t left = ne - ((uint64_t)blockIdx.x << GROUP_BITS);  // entries of this group
    if ((uint64_t)threadIdx.x == (left < (uint64_t)GROUP ? left : (uint64_t)GROUP) - 1) G[inst * ng + blockIdx.x] = q;
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
// which keeps the searches off the FP64 pipe.
__device__ __forceinline__ long long ord(double v) { return __double_as_longlong(v); }

// Smallest i in [0, len) with A[i] > key (A nondecreasing, A[len - 1] > key),
// or with A[i] >= A[len - 1] when `edge`; a 32-way search by the whole warp.
// Every A[i] and key are >= +0.
__device__ __forceinline__ uint64_t warp_search(const double *A, uint64_t len, double key, bool edge) {
    const int lane = threadIdx.x & 31;
    const long long kb = ord(edge ? A[len - 1] : key);
    uint64_t lo = 0, hi = len;  // the answer is in [lo, hi)
    while (hi - lo > 1) {
        const uint64_t stride = (hi - lo + 31) / 32;
        uint64_t i = lo + (uint64_t)(lane + 1) * stride - 1;
        if (i > hi - 1) i = hi - 1;
        const long long v = ord(A[i]);
        const unsigned ok = __ballot_sync(0xFFFFFFFFu, edge ? v >= kb : v > kb);
        const uint64_t f = (uint64_t)(__ffs(ok) - 1);  // A[hi - 1] qualifies, so ok != 0
        const uint64_t nlo = lo + f * stride;
        hi = nlo + stride < hi ? nlo + stride : hi;
        lo = nlo;
    }
    return lo;
}

// One warp per draw j of instance blockIdx.y: x_j = min { x : F(x) > t } with
// t = u_j F_total; an x of probability zero never wins.  When rounding leaves
// no x qualifying at some level (t at F_total, or the remainder at a group's or
// an entry's rounded total) the last x of nonzero probability under the
// chosen group and entry is taken.
template <typename V>
__global__ void __launch_bounds__(DRAW_WARPS * 32) draw_kernel(const V *states, int ns, int z2, const double *Q,
                                                                 const double *P, int k, const double *u,
                                                                 uint64_t *xs) {
    const int lane = threadIdx.x & 31;
    const uint64_t j = (uint64_t)blockIdx.x * DRAW_WARPS + (threadIdx.x >> 5);
    if (j >= (uint64_t)k) return;  // whole warps leave together
    const uint64_t inst = blockIdx.y;
    const uint64_t N = 1ull << ns, ne = entry_count(ns), ng = group_count(ns);
    const V *st = states + (inst << ns);
    const double *Pi = P + inst * ng;
    const double total = Pi[ng - 1];
    double uj = u[inst * (uint64_t)k + j];
    uj = uj > 0.0 ? uj : 0.0;  // u <= 0 (or NaN) draws the first x of nonzero probability
    double t = uj * (z2 ? 2.0 * total : total);
    bool flip = false;
    if (z2 && total > 0.0 && ord(t) >= ord(total)) {
        flip = true;
        t -= total;
    }
    // group (t, the sums and every remainder below are >= +0)
    bool edge = ord(t) >= ord(total);
    const uint64_t g = warp_search(Pi, ng, t, edge);
    double rest = t - (g > 0 ? Pi[g - 1] : 0.0);
    // entry within the group
    const uint64_t e0 = g << GROUP_BITS;
    const uint64_t glen = ne - e0 < (uint64_t)GROUP ? ne - e0 : (uint64_t)GROUP;
    const double *Qg = Q + inst * ne + e0;
    edge = edge || ord(rest) >= ord(Qg[glen - 1]);
    const uint64_t e = warp_search(Qg, glen, rest, edge);
    rest -= e > 0 ? Qg[e - 1] : 0.0;
    // amplitude within the entry; the chosen entry has a nonzero sum unless
    // the state's norm is 0 (then x = 0)
    const uint64_t x = ((e0 + e) << ENTRY_BITS) + (uint64_t)lane;
    V z{};
    if (x < N) z = st[x];
    const int pk = entry_pick(z, x < N, rest, edge);
    const int pick = pk >= 0 ? pk : 0;
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
    const size_t qb = sizeof(double) * ne * (size_t)batch;
    const size_t pre = qb + ((sizeof(double) * ng * (size_t)batch + 255) & ~(size_t)255);
    const size_t xb = d_x ? 0 : sizeof(uint64_t) * (size_t)k * batch;
    const size_t fb = sizeof(int) * (size_t)batch;
    Scratch *sc = nullptr;
    int rc = scratch_for(stream, pre + xb + fb + 64, fb + 64, &sc);
    if (rc) return rc;
    char *dev = reinterpret_cast<char *>(sc->dev);
    double *d_q = reinterpret_cast<double *>(dev);
    double *d_pre = reinterpret_cast<double *>(dev + qb);
    uint64_t *xs = d_x ? d_x : reinterpret_cast<uint64_t *>(dev + pre);
    int *d_first = reinterpret_cast<int *>(dev + pre + xb);
    const dim3 draw_grid((unsigned)((k + DRAW_WARPS - 1) / DRAW_WARPS), batch);
    profile_before(K_SAMPLE, stream);
    if (dtype == QAOA_C64) {
        const float2 *st = reinterpret_cast<const float2 *>(d_states);
        if ((reinterpret_cast<uintptr_t>(d_states) & 15u) == 0) {
            static const cudaError_t attr = cudaFuncSetAttribute(
                entry_scan_kernel<float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STAGE_BYTES);
            if (attr != cudaSuccess) return cuda_error(attr, "entry scan shared memory");
            entry_scan_kernel<float2, true><<<dim3((unsigned)ng, batch), GROUP, STAGE_BYTES, stream>>>(st, ns, d_q,
                                                                                                      d_pre);
        } else {
            entry_scan_kernel<float2, false><<<dim3((unsigned)ng, batch), GROUP, 0, stream>>>(st, ns, d_q, d_pre);
        }
        block_prefix_kernel<<<batch, PREFIX_PT, 0, stream>>>(d_pre, ng);
        draw_kernel<float2><<<draw_grid, DRAW_WARPS * 32, 0, stream>>>(st, ns, z2 ? 1 : 0, d_q, d_pre, k, d_u, xs);
    } else {
        const double2 *st = reinterpret_cast<const double2 *>(d_states);
        entry_scan_kernel<double2, false><<<dim3((unsigned)ng, batch), GROUP, 0, stream>>>(st, ns, d_q, d_pre);
        block_prefix_kernel<<<batch, PREFIX_PT, 0, stream>>>(d_pre, ng);
        draw_kernel<double2><<<draw_grid, DRAW_WARPS * 32, 0, stream>>>(st, ns, z2 ? 1 : 0, d_q, d_pre, k, d_u, xs);
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
