// Measurement behind a design choice of the mixer passes (not part of the
// library; built and run on its own).  A pass over a group of more than 13
// qubits would need a tile larger than one CTA holds, spread over the CTAs of
// a thread-block cluster and exchanged once or twice per tile.  This measures
// that exchange: an all-to-all between the CTAs of a cluster through
// distributed shared memory (cluster sizes 2..16), against a local
// shared-memory copy and against a round trip through global memory (L2).
// Each CTA (512 threads, one per SM) owns SRC and DST buffers of 64 KiB; one
// round sends block d of SRC (64 KiB / CS) to CTA d's DST slot r (r = its own
// rank), then a cluster barrier, as a pass would per tile.  No waits other
// than cluster barriers; every index stays inside its 64 KiB buffer.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o dsmem_exchange paper_2401_02852_gb300/probes/dsmem_exchange.cu && ./dsmem_exchange
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

namespace cg = cooperative_groups;

constexpr int ELEMS = 4096;  // float4 per buffer = 64 KiB
constexpr int NT = 512;

template <int CS, int MODE>  // MODE 0: DSMEM all-to-all, 1: local copy, 2: global round trip
__global__ void __launch_bounds__(NT, 1) xchg(int rounds, float4 *gbuf, float *sink) {
    extern __shared__ float4 sm[];
    float4 *src = sm, *dst = sm + ELEMS;
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    for (int i = threadIdx.x; i < ELEMS; i += NT) src[i] = make_float4(i, r, 0, 1);
    constexpr int BLK = ELEMS / CS;  // float4 per destination
    float4 *g = gbuf + (size_t)blockIdx.x * ELEMS;
    float4 *gcl = gbuf + (size_t)(blockIdx.x - r) * ELEMS;  // this cluster's first CTA's region
    cl.sync();
    for (int it = 0; it < rounds; ++it) {
        if (MODE == 0) {
            for (int i = threadIdx.x; i < ELEMS; i += NT) {
                const int d = i / BLK, o = i % BLK;
                float4 *rd = cl.map_shared_rank(dst, d);
                rd[r * BLK + o] = src[i];
            }
            cl.sync();
        } else if (MODE == 1) {
            for (int i = threadIdx.x; i < ELEMS; i += NT) dst[i] = src[i];
            __syncthreads();
        } else {
            for (int i = threadIdx.x; i < ELEMS; i += NT) g[i] = src[i];
            cl.sync();
            // read block r of every CTA of the cluster
            for (int i = threadIdx.x; i < ELEMS; i += NT) {
                const int c = i / BLK, o = i % BLK;
                dst[i] = gcl[(size_t)c * ELEMS + r * BLK + o];
            }
            cl.sync();
        }
        float4 *t = src;  // swap roles so the compiler cannot drop rounds
        src = dst;
        dst = t;
    }
    float acc = 0.f;
    for (int i = threadIdx.x; i < ELEMS; i += NT) acc += src[i].x;
    if (acc == 12345.f) sink[0] = acc;
}

template <int CS, int MODE>
static void run(const char *name, int sms) {
    auto k = xchg<CS, MODE>;
    const size_t smem = 2 * ELEMS * sizeof(float4);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (CS > 8) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    cfg.gridDim = dim3(CS * 64);
    cudaError_t e = cudaOccupancyMaxActiveClusters(&max_clusters, (void *)k, &cfg);
    if (e != cudaSuccess || max_clusters < 1) {
        printf("%-28s CS=%2d occupancy query failed: %s (%d)\n", name, CS, cudaGetErrorString(e), max_clusters);
        cudaGetLastError();
        return;
    }
    const int ctas = max_clusters * CS;
    cfg.gridDim = dim3(ctas);
    float4 *gbuf = nullptr;
    float *sink = nullptr;
    cudaMalloc(&gbuf, (size_t)ctas * ELEMS * sizeof(float4));
    cudaMalloc(&sink, 4);
    const int rounds = 4000;
    cudaLaunchKernelEx(&cfg, k, 10, gbuf, sink);  // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    cudaLaunchKernelEx(&cfg, k, rounds, gbuf, sink);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
        printf("%s failed: %s\n", name, cudaGetErrorString(e));
        exit(1);
    }
    // bytes written per round by all CTAs (the exchange volume)
    const double bytes = (double)ctas * ELEMS * sizeof(float4) * rounds;
    printf("%-28s CS=%2d clusters=%3d ctas=%3d (sms %d)  %.3f ms  %.1f GB/s written (%.1f GB/s per SM), %.2f us/round\n",
           name, CS, max_clusters, ctas, sms, ms, bytes / ms / 1e6, bytes / ms / 1e6 / ctas, 1000.0 * ms / rounds);
    cudaFree(gbuf);
    cudaFree(sink);
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    run<1, 1>("local smem copy", sms);
    run<2, 0>("dsmem all-to-all", sms);
    run<4, 0>("dsmem all-to-all", sms);
    run<8, 0>("dsmem all-to-all", sms);
    run<16, 0>("dsmem all-to-all", sms);
    run<2, 2>("global round trip", sms);
    run<8, 2>("global round trip", sms);
    return 0;
}
