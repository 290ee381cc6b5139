// K7: bitstrings drawn from the output state, and instance running times
// (Sec. "Running Times": measuring the final state yields x with probability
// |Psi(x)|^2; the running time of an instance is the number of draws up to and
// including the first one that satisfies it).
//
// Inverse-CDF sampling with caller-supplied uniforms u_j in [0, 1): draw j is
// the smallest x with F(x) > u_j F_total, F(x) = sum_{y <= x} |psi(y)|^2.  The
// probabilities are formed in FP64 from the stored amplitudes, so the result
// differs from a sequential FP64 scan only through the summation order, i.e.
// only for a u_j within rounding of a step of F.
//
//   1. block_sums_kernel: one FP64 sum per block of 2^SB amplitudes;
//   2. block_prefix_kernel: inclusive prefix of the block sums, fixed order;
//   3. draw_kernel: one warp per draw: binary search over the block prefix,
//      then a warp-wide FP64 scan through the chosen block.
// With QAOA_Z2_HALF the stored half holds the x with bit n-1 clear and
// |psi(not x)| = |psi(x)| (Sec. 2.2's global flip): t = u 2 F_half picks the
// stored x (t < F_half) or the complement of the x drawn at t - F_half.
#include <cuda_runtime.h>

#include <cmath>

#include "pass_common.cuh"
#include "qaoa_internal.cuh"

namespace qaoa {

constexpr int SB = 13;           // log2 amplitudes per block
constexpr int SUM_PT = 256;      // threads of the block-sum kernel
constexpr int PREFIX_PT = 1024;  // threads of the prefix kernel
constexpr int DRAW_WARPS = 8;    // draws per CTA of the draw kernel

template <typename V>
__device__ __forceinline__ double prob(const V &z) {
    const double re = (double)z.x, im = (double)z.y;
    return re * re + im * im;
}

// sums[inst][b] = sum of |psi|^2 over block b (2^SB amplitudes, or the whole
// stored state when it is smaller) of instance inst = blockIdx.y.
template <typename V>
__global__ void __launch_bounds__(SUM_PT) block_sums_kernel(const V *states, int ns, uint64_t nb, double *sums) {
    const uint64_t N = 1ull << ns;
    const V *st = states + ((uint64_t)blockIdx.y << ns);
    const uint64_t lo = (uint64_t)blockIdx.x << SB;
    const uint64_t hi = lo + (1ull << SB) < N ? lo + (1ull << SB) : N;
    double s = 0.0;
    for (uint64_t x = lo + threadIdx.x; x < hi; x += SUM_PT) s += prob(st[x]);
    double v[1] = {s};
    block_sum<1, SUM_PT>(v);
    if (threadIdx.x == 0) sums[(uint64_t)blockIdx.y * nb + blockIdx.x] = v[0];
}

// In place, per instance (one CTA each): sums[b] <- sums[0] + ... + sums[b].
// Each thread adds a contiguous chunk in order, thread 0 turns the chunk
// totals into offsets in order, then each thread writes its running sums.
__global__ void __launch_bounds__(PREFIX_PT) block_prefix_kernel(double *sums, uint64_t nb) {
    __shared__ double chunk[PREFIX_PT];
    double *s = sums + (uint64_t)blockIdx.x * nb;
    const uint64_t per = (nb + PREFIX_PT - 1) / PREFIX_PT;
    const uint64_t lo = threadIdx.x * per < nb ? threadIdx.x * per : nb;
    const uint64_t hi = lo + per < nb ? lo + per : nb;
    double c = 0.0;
    for (uint64_t i = lo; i < hi; ++i) c += s[i];
    chunk[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int t = 0; t < PREFIX_PT; ++t) {
            const double v = chunk[t];
            chunk[t] = run;
            run += v;
        }
    }
    __syncthreads();
    double run = chunk[threadIdx.x];
    for (uint64_t i = lo; i < hi; ++i) {
        run += s[i];
        s[i] = run;
    }
}

// One warp per draw j of instance blockIdx.y: x_j = min { x : F(x) > t } with
// t = u_j F_total; an x of probability zero never wins.  When no x qualifies
// (t at F_total by rounding, or inside a block past its rounded sum) the last
// x of nonzero probability of the block is taken.
template <typename V>
__global__ void __launch_bounds__(DRAW_WARPS * 32) draw_kernel(const V *states, int ns, int z2, const double *prefix,
                                                                 uint64_t nb, int k, const double *u, uint64_t *xs) {
    const int lane = threadIdx.x & 31;
    const uint64_t j = (uint64_t)blockIdx.x * DRAW_WARPS + (threadIdx.x >> 5);
    if (j >= (uint64_t)k) return;  // whole warps leave together
    const uint64_t inst = blockIdx.y;
    const uint64_t N = 1ull << ns;
    const V *st = states + (inst << ns);
    const double *P = prefix + inst * nb;
    const double total = P[nb - 1];
    double t = u[inst * (uint64_t)k + j] * (z2 ? 2.0 * total : total);
    bool flip = false;
    if (z2 && t >= total) {
        flip = true;
        t -= total;
    }
    // smallest block b with P[b] > t; when rounding left t at F_total, the
    // block holding the last x of nonzero probability (smallest P[b] >= total)
    const bool edge = !(t < total);
    uint64_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (edge ? P[mid] >= total : P[mid] > t)
            hi = mid;
        else
            lo = mid + 1;
    }
    double rest = edge ? HUGE_VAL : t - (lo > 0 ? P[lo - 1] : 0.0);
    const uint64_t x0 = lo << SB, x1 = x0 + (1ull << SB) < N ? x0 + (1ull << SB) : N;
    uint64_t found = ~0ull, last_nz = x0;
    for (uint64_t c = x0; c < x1 && found == ~0ull; c += 32) {
        const uint64_t x = c + lane;
        const double w = x < x1 ? prob(st[x]) : 0.0;
        double incl = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, w > 0.0 && incl > rest);
        const unsigned nz = __ballot_sync(0xFFFFFFFFu, w > 0.0);
        if (hit) found = c + (uint64_t)(__ffs(hit) - 1);
        if (nz) last_nz = c + (uint64_t)(31 - __clz(nz));
        rest -= __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (found == ~0ull) found = last_nz;
    if (lane == 0) {
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
    const uint64_t nb = ((1ull << ns) + (1ull << SB) - 1) >> SB;
    const size_t pre = sizeof(double) * nb * (size_t)batch;
    const size_t xb = d_x ? 0 : sizeof(uint64_t) * (size_t)k * batch;
    const size_t fb = sizeof(int) * (size_t)batch;
    Scratch *sc = nullptr;
    int rc = scratch_for(stream, pre + xb + fb + 64, fb + 64, &sc);
    if (rc) return rc;
    char *dev = reinterpret_cast<char *>(sc->dev);
    double *d_pre = reinterpret_cast<double *>(dev);
    uint64_t *xs = d_x ? d_x : reinterpret_cast<uint64_t *>(dev + pre);
    int *d_first = reinterpret_cast<int *>(dev + pre + xb);
    profile_before(K_SAMPLE, stream);
    if (dtype == QAOA_C64) {
        const float2 *st = reinterpret_cast<const float2 *>(d_states);
        block_sums_kernel<float2><<<dim3((unsigned)nb, batch), SUM_PT, 0, stream>>>(st, ns, nb, d_pre);
        block_prefix_kernel<<<batch, PREFIX_PT, 0, stream>>>(d_pre, nb);
        draw_kernel<float2><<<dim3((unsigned)((k + DRAW_WARPS - 1) / DRAW_WARPS), batch), DRAW_WARPS * 32, 0, stream>>>(
            st, ns, z2 ? 1 : 0, d_pre, nb, k, d_u, xs);
    } else {
        const double2 *st = reinterpret_cast<const double2 *>(d_states);
        block_sums_kernel<double2><<<dim3((unsigned)nb, batch), SUM_PT, 0, stream>>>(st, ns, nb, d_pre);
        block_prefix_kernel<<<batch, PREFIX_PT, 0, stream>>>(d_pre, nb);
        draw_kernel<double2><<<dim3((unsigned)((k + DRAW_WARPS - 1) / DRAW_WARPS), batch), DRAW_WARPS * 32, 0, stream>>>(
            st, ns, z2 ? 1 : 0, d_pre, nb, k, d_u, xs);
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
