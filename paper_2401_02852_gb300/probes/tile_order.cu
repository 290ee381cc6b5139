// Measurement behind a design choice of the mixer passes (not part of the
// library; built and run on its own).  In which order should the persistent
// CTAs of a high pass take their tiles?  One read-modify-write pass over a
// 2^30-amplitude complex64 state (8 GiB) plus its 1-byte cost table (1 GiB),
// in the two strided tile orders of n = 30 (tiles of 2^13 amplitudes):
//   rows16   512 rows of 16 amplitudes (128 B) at stride 2^13; the tile index
//            fills bits 4..12 and 22..29; cost rows of 16 B
//   rows32   256 rows of 32 amplitudes (256 B) at stride 2^22; the tile index
//            fills bits 5..21; cost rows of 32 B
// with the movers of the high passes (cp.async 16-byte copies of the tile and
// its cost bytes into one buffer, two CTAs per SM, stores from registers) and
// three assignments of tiles to CTAs:
//   plain    CTA b takes tiles b, b + G, b + 2G, ... (G CTAs)
//   grouped  CTA b takes GT consecutive tiles at a time (GT = 64 B of cost
//            bytes / the cost bytes of a row: 4 for rows16, 2 for rows32):
//            GT (b + k G) + j, j < GT
//   dynamic  every CTA takes the next unclaimed tile from a counter in global
//            memory (one atomicAdd per tile), so the tiles in flight are
//            always a window of consecutive indices
// The counter is zeroed before every launch; every claimed index is checked
// against the tile count before use.  Afterwards every sampled amplitude must
// have been modified exactly once per launch.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o tile_order paper_2401_02852_gb300/probes/tile_order.cu && ./tile_order
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>

constexpr int NQ = 30;
constexpr int T = 13;
constexpr int NT = 256;
constexpr int PER = (1 << T) / NT;     // amplitudes per thread (32)
constexpr int CH = (1 << T) / 2 / NT;  // state 16-byte chunks per thread (16)
constexpr int CC = (1 << T) / 16 / NT; // cost 16-byte chunks per thread (2)
constexpr uint32_t NTILES = 1u << (NQ - T);

struct Geo {
    int R, lo, G, mid;
};

__host__ __device__ inline uint32_t tile_base(const Geo &g, uint32_t t) {
    const uint32_t tm = t & ((1u << g.mid) - 1u), tt = t >> g.mid;
    return (tm << g.R) | (tt << (g.lo + g.G));
}
__host__ __device__ inline uint32_t elem_addr(const Geo &g, uint32_t base, uint32_t u) {
    return base + (u & ((1u << g.R) - 1u)) + ((u >> g.R) << g.lo);
}

__device__ __forceinline__ void cp_async16(void *s, const void *gm) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gm) : "memory");
}

__device__ __forceinline__ void issue(const Geo &g, const float2 *st, const uint8_t *cs, uint32_t t, float2 *buf,
                                      uint8_t *cbuf) {
    const uint32_t base = tile_base(g, t);
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        const uint32_t q = threadIdx.x + NT * j;
        cp_async16(buf + 2 * q, st + elem_addr(g, base, 2 * q));
    }
#pragma unroll
    for (int j = 0; j < CC; ++j) {
        const uint32_t q = threadIdx.x + NT * j;  // cost bytes [16 q, 16 q + 16) of the tile
        cp_async16(cbuf + 16 * q, cs + elem_addr(g, base, 16 * q));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// ORDER: 0 plain, 1 grouped, 2 dynamic
template <int ORDER>
__global__ void __launch_bounds__(NT, 2) mover(Geo g, int gt, float2 *st, const uint8_t *cs, unsigned *ctr) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *buf = reinterpret_cast<float2 *>(smraw);
    uint8_t *cbuf = smraw + (8u << T);
    __shared__ uint32_t claimed;
    auto tile_at = [&](uint32_t i) -> uint32_t {
        if (ORDER == 0) return blockIdx.x + i * gridDim.x;
        return gt * (blockIdx.x + (i / gt) * gridDim.x) + (i % gt);
    };
    uint32_t t;
    if (ORDER == 2) {
        if (threadIdx.x == 0) claimed = atomicAdd(ctr, 1u);
        __syncthreads();
        t = claimed;
    } else {
        t = tile_at(0);
    }
    if (t < NTILES) issue(g, st, cs, t, buf, cbuf);
    for (uint32_t i = 0; t < NTILES; ++i) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        float2 v[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t u = threadIdx.x + NT * j;
            v[j] = buf[u];
            v[j].x += 1.0f + (float)cbuf[u];
        }
        if (ORDER == 2 && threadIdx.x == 0) claimed = atomicAdd(ctr, 1u);
        __syncthreads();  // the buffer is read out (and the next index claimed)
        const uint32_t tn = ORDER == 2 ? claimed : tile_at(i + 1);
        if (tn < NTILES) issue(g, st, cs, tn, buf, cbuf);
        const uint32_t base = tile_base(g, t);
#pragma unroll
        for (int j = 0; j < PER; ++j) st[elem_addr(g, base, threadIdx.x + NT * j)] = v[j];
        t = tn;
    }
}

#define CK(x)                                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) {                                                               \
            fprintf(stderr, "%s:%d %s: %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
            exit(1);                                                                           \
        }                                                                                      \
    } while (0)

// Host check: the grouped order visits every tile once for the grid sizes used
// (the tile count is a multiple of GT), and tile_base/elem_addr cover the state
// once (sampled tiles; the probe's sampled-amplitude check covers the rest).
static bool check(const Geo &g, int gt, int grid) {
    if (NTILES % gt) return false;
    unsigned char *seen = (unsigned char *)calloc(NTILES, 1);
    for (uint32_t b = 0; b < (uint32_t)grid; ++b)
        for (uint32_t i = 0;; ++i) {
            const uint32_t t = gt * (b + (i / gt) * grid) + (i % gt);
            if (t >= NTILES) break;
            if (seen[t]++) {
                free(seen);
                return false;
            }
        }
    for (uint32_t t = 0; t < NTILES; ++t)
        if (seen[t] != 1) {
            free(seen);
            return false;
        }
    free(seen);
    for (uint32_t t = 0; t < NTILES; t += 4093)
        for (uint32_t u = 0; u < (1u << T); ++u)
            if (elem_addr(g, tile_base(g, t), u) >= (1u << NQ)) return false;
    return true;
}

int main() {
    const Geo geos[2] = {{4, 13, 9, 9}, {5, 22, 8, 17}};
    const int gts[2] = {4, 2};
    const char *gname[2] = {"rows16 @ 2^13", "rows32 @ 2^22"};
    const char *oname[3] = {"plain", "grouped", "dynamic"};
    int sms = 0;
    CK(cudaSetDevice(0));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const int grid = 2 * sms;
    for (int k = 0; k < 2; ++k)
        if (!check(geos[k], gts[k], grid) || !check(geos[k], 1, grid)) {
            fprintf(stderr, "host check failed for %s\n", gname[k]);
            return 1;
        }
    printf("host checks passed (static orders visit every tile once; addresses inside the state)\n");
    const size_t n = (size_t)1 << NQ;
    float2 *st = nullptr;
    uint8_t *cs = nullptr;
    unsigned *ctr = nullptr;
    CK(cudaMalloc(&st, n * sizeof(float2)));
    CK(cudaMalloc(&cs, n));
    CK(cudaMalloc(&ctr, sizeof(unsigned)));
    CK(cudaMemset(st, 0, n * sizeof(float2)));
    CK(cudaMemset(cs, 0, n));
    const int smem = (8 << T) + (1 << T);
    CK(cudaFuncSetAttribute(mover<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(mover<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(mover<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int WARM = 2, REPS = 5;
    int launches = 0;
    const double bytes = 2.0 * n * 8 + n;  // state read and written, cost read
    printf("| tile order | assignment | ms per pass (mean of %d) | TB/s (state + cost) |\n|---|---|---:|---:|\n", REPS);
    for (int k = 0; k < 2; ++k)
        for (int o = 0; o < 3; ++o) {
            const Geo g = geos[k];
            auto launch = [&]() {
                CK(cudaMemsetAsync(ctr, 0, sizeof(unsigned)));
                if (o == 0) mover<0><<<grid, NT, smem>>>(g, 1, st, cs, ctr);
                if (o == 1) mover<1><<<grid, NT, smem>>>(g, gts[k], st, cs, ctr);
                if (o == 2) mover<2><<<grid, NT, smem>>>(g, 1, st, cs, ctr);
                ++launches;
            };
            for (int w = 0; w < WARM; ++w) launch();
            CK(cudaGetLastError());
            CK(cudaDeviceSynchronize());
            CK(cudaEventRecord(e0));
            for (int r = 0; r < REPS; ++r) launch();
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ms /= REPS;
            printf("| %s | %s | %.3f | %.2f |\n", gname[k], oname[o], ms, bytes / (ms * 1e-3) / 1e12);
        }
    const size_t SAMPLE = 1 << 20;
    float2 *h = (float2 *)malloc(SAMPLE * sizeof(float2));
    size_t bad = 0;
    for (int part = 0; part < 4; ++part) {
        CK(cudaMemcpy(h, st + (n / 4) * part, SAMPLE * sizeof(float2), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < SAMPLE; ++i)
            if (h[i].x != (float)launches || h[i].y != 0.0f) ++bad;
    }
    printf("check: %zu of %zu sampled amplitudes differ from %d\n", bad, 4 * SAMPLE, launches);
    free(h);
    CK(cudaFree(st));
    CK(cudaFree(cs));
    CK(cudaFree(ctr));
    return bad ? 1 : 0;
}
