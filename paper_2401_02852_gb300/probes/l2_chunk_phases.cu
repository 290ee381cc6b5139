// Measurement behind a design choice of the mixer passes (not part of the
// library; built and run on its own).  Could the low pass and the first high
// group run on chunks of the state that stay in L2 (three read-modify-write
// phases per chunk: low qubits, the high group, the next layer's low qubits),
// so that three passes cost one HBM round trip?  This measures the memory side
// alone: a state of 2^30 complex64 (2^29 float4), chunks of 2^C float4, each
// thread keeping 8 float4 loads in flight.  Phase 0 walks a chunk
// contiguously (a low-pass tile order), phase 1 in rows of 8 float4 strided
// by 2^12 (a high group's tile order), phase 2 contiguously again.  Between
// phases all CTAs meet at a grid barrier: a monotonic counter with a bounded
// spin (error flag and exit after LIMIT polls); the launch is cooperative (all
// CTAs resident).  The chunk permutation is a bijection for C >= 21.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o l2_chunk_phases paper_2401_02852_gb300/probes/l2_chunk_phases.cu && ./l2_chunk_phases
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstdint>

constexpr int NT = 256;
constexpr int ITEMS = 8;  // float4 per thread in flight; every chunk is a multiple of NT * ITEMS
constexpr unsigned long long LIMIT = 1ull << 24;  // polls (~ seconds) before giving up

struct Bar {
    unsigned int count;
    unsigned int error;
};

__device__ __forceinline__ bool grid_barrier(Bar *bar, unsigned int target) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&bar->count, 1u);
        unsigned long long it = 0;
        volatile unsigned int *c = &bar->count;
        volatile unsigned int *e = &bar->error;
        while (*c < target && *e == 0 && it < LIMIT) ++it;
        if (it >= LIMIT) atomicExch(&bar->error, 1u);
        __threadfence();
        ok = (*e == 0);
    }
    __syncthreads();
    return ok;
}

// float4 index inside a chunk for position j of phase ph (0 <= j < 2^C)
__device__ __forceinline__ uint32_t perm(uint32_t j, int ph, int C) {
    if (ph != 1) return j;
    // tiles of 2^12 float4: 8 contiguous x 2^9 rows strided by 2^12; tile id fills bits 3..11 and 21..C-1
    const uint32_t q = j & 4095u, t = j >> 12;
    const uint32_t row = q & 7u, grp = q >> 3;                    // grp: 9 bits -> index bits 12..20
    const uint32_t tlo = t & 511u, thi = t >> 9;                  // tlo -> bits 3..11, thi -> bits 21..
    return row | (tlo << 3) | (grp << 12) | (thi << 21);
}

__global__ void __launch_bounds__(NT) chunk_kernel(float4 *x, int total_log2, int C, int phases, Bar *bar) {
    const uint32_t chunk = 1u << C;
    const uint64_t nchunks = 1ull << (total_log2 - C);
    const uint32_t stride = gridDim.x * NT;
    unsigned int epoch = 0;
    for (uint64_t c = 0; c < nchunks; ++c) {
        float4 *base = x + c * chunk;
        for (int ph = 0; ph < phases; ++ph) {
            // ITEMS loads in flight per thread (coalesced: item k of thread t is j0 + k * NT + t)
            for (uint32_t j0 = blockIdx.x * NT * ITEMS; j0 < chunk; j0 += stride * ITEMS) {
                float4 v[ITEMS];
                uint32_t idx[ITEMS];
#pragma unroll
                for (int k = 0; k < ITEMS; ++k) {
                    idx[k] = perm(j0 + k * NT + threadIdx.x, ph, C);
                    v[k] = __ldcg(base + idx[k]);
                }
#pragma unroll
                for (int k = 0; k < ITEMS; ++k) {
                    v[k].x += 1.f;
                    base[idx[k]] = v[k];
                }
            }
            if (phases > 1) {
                ++epoch;
                if (!grid_barrier(bar, epoch * gridDim.x)) return;
            }
        }
    }
}

int main() {
    const int total_log2 = 29;  // float4 count: 2^29 (8 GiB)
    float4 *x = nullptr;
    if (cudaMalloc(&x, (size_t)sizeof(float4) << total_log2) != cudaSuccess) {
        printf("alloc failed\n");
        return 1;
    }
    cudaMemset(x, 0, (size_t)sizeof(float4) << total_log2);
    Bar *bar = nullptr;
    cudaMalloc(&bar, sizeof(Bar));
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chunk_kernel, NT, 0);
    struct Case {
        int C, phases, blocks_per_sm;
    } cases[] = {{29, 1, 2}, {29, 1, 4}, {21, 1, 2}, {21, 2, 2}, {21, 3, 2}, {22, 3, 2}, {21, 3, 4}, {22, 3, 4}};
    double plain_ms = 0.0;
    for (const Case &k : cases) {
        const int bps = k.blocks_per_sm < per_sm ? k.blocks_per_sm : per_sm;
        int grid = sms * bps;
        int C = k.C, phases = k.phases, tl = total_log2;
        void *args[] = {&x, &tl, &C, &phases, &bar};
        cudaMemset(bar, 0, sizeof(Bar));
        cudaLaunchCooperativeKernel((void *)chunk_kernel, grid, NT, args, 0, 0);  // warm-up
        cudaMemset(bar, 0, sizeof(Bar));
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a);
        cudaError_t e = cudaLaunchCooperativeKernel((void *)chunk_kernel, grid, NT, args, 0, 0);
        cudaEventRecord(b);
        cudaError_t e2 = cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        Bar hb{};
        cudaMemcpy(&hb, bar, sizeof hb, cudaMemcpyDeviceToHost);
        const double bytes = 2.0 * ((double)sizeof(float4) * (1ull << total_log2));  // one read + one write of the state
        if (plain_ms == 0.0) plain_ms = ms;  // the first case is the plain pass
        printf("chunk 2^%d float4 (%6.1f MB) phases %d grid %d: %8.3f ms = %.2f x the plain pass; "
               "one read + write of the state per %.0f GB/s; barrier error %u; launch %s / %s\n",
               k.C, (double)(sizeof(float4) << k.C) / 1e6, k.phases, grid, ms, ms / plain_ms, bytes / ms / 1e6,
               hb.error, cudaGetErrorString(e), cudaGetErrorString(e2));
        if (e != cudaSuccess || e2 != cudaSuccess) return 1;
    }
    return 0;
}
