// Measurement behind a design choice of the mixer passes (not part of the
// library; built and run on its own).  How fast can one read-modify-write pass
// over a 2^30-amplitude complex64 state (8 GiB) stream, in the three tile
// orders the passes use at n = 30, with four ways of moving a tile?
//
// Tile orders (every tile is 2^13 amplitudes = 64 KiB):
//   contiguous   the low pass: tile t is amplitudes [2^13 t, 2^13 (t + 1))
//   rows16       the 9-bit group 13..21: 512 rows of 16 amplitudes (128 B)
//                at stride 2^13; the tile index fills bits 4..12 and 22..29
//   rows32       the 8-bit group 22..29: 256 rows of 32 amplitudes (256 B)
//                at stride 2^22; the tile index fills bits 5..21
// Tile element u sits at base + (u mod 2^R) + (u >> R) 2^lo (R = row bits).
//
// Movers (each thread modifies its 32 amplitudes u = tid + 256 j):
//   A  cp.async 16-byte copies into one buffer, two CTAs per SM; the next
//      tile's copies are issued once the buffer is read into registers;
//      stores from registers (8 bytes per thread)
//   B  cp.async, three buffers, one CTA per SM (tile i + 3 issued when tile
//      i has been read out), stores from registers
//   C  one TMA tensor load per tile (mbarrier completion), three buffers,
//      one CTA per SM, stores from registers
//   D  TMA loads and TMA stores: the modified tile goes back to its buffer
//      and leaves by one bulk tensor store; tile i + 2 is loaded as soon as
//      the store of tile i - 1 has read its buffer
// Every mbarrier wait is bounded (LIMIT polls); a CTA that gives up sets an
// error flag and stops taking tiles.  The coordinates of every TMA copy are
// inside the tensor map's extents (checked by the host before the launches),
// and the innermost coordinate is always 0.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o strided_rows_pipeline paper_2401_02852_gb300/probes/strided_rows_pipeline.cu && ./strided_rows_pipeline
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>

constexpr int NQ = 30;
constexpr int T = 13;                       // tile bits
constexpr int NT = 256;                     // threads per CTA
constexpr int PER = (1 << T) / NT;          // amplitudes per thread (32)
constexpr int CH = (1 << T) / 2 / NT;       // 16-byte chunks per thread (16)
constexpr uint32_t TILE_BYTES = 8u << T;    // 64 KiB
constexpr uint32_t NTILES = 1u << (NQ - T);
constexpr unsigned long long LIMIT = 1ull << 22;

struct Geo {
    int R, lo;       // row bits; lowest bit of the group
    int G;           // group bits (T - R)
    int mid;         // tile-index bits placed at R..lo-1
};

__host__ __device__ inline uint32_t tile_base(const Geo &g, uint32_t t) {
    if (g.R == T) return t << T;
    const uint32_t tm = t & ((1u << g.mid) - 1u), tt = t >> g.mid;
    return (tm << g.R) | (tt << (g.lo + g.G));
}
__host__ __device__ inline uint32_t elem_addr(const Geo &g, uint32_t base, uint32_t u) {
    if (g.R == T) return base + u;
    return base + (u & ((1u << g.R) - 1u)) + ((u >> g.R) << g.lo);
}
// TMA coordinates of tile t (5-d map; see make_map)
__host__ __device__ inline void tile_coords(const Geo &g, uint32_t t, int c[5]) {
    c[0] = 0;
    if (g.R == T) {  // 2-d view {32, 2^25}, box {32, 256}
        c[1] = (int)(t << (T - 5));
        c[2] = c[3] = c[4] = 0;
        return;
    }
    c[1] = (int)(t & ((1u << g.mid) - 1u));
    c[2] = 0;
    c[3] = 0;
    c[4] = (int)(t >> g.mid);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *s, const void *gm) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    const uint32_t a = smem_u32(b);
    for (unsigned long long it = 0; it < LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, const int c[5], uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap *map, const int c[5], const void *src) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n" ::"l"(
                     map),
                 "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void issue_cp(const Geo &g, const float2 *st, uint32_t t, float2 *buf) {
    const uint32_t base = tile_base(g, t);
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        const uint32_t q = threadIdx.x + NT * j;
        cp_async16(buf + 2 * q, st + elem_addr(g, base, 2 * q));
    }
}
__device__ __forceinline__ void read_modify(const float2 *buf, float2 v[PER]) {
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = buf[threadIdx.x + NT * j];
        v[j].x += 1.0f;
    }
}
__device__ __forceinline__ void store_regs(const Geo &g, float2 *st, uint32_t t, const float2 v[PER]) {
    const uint32_t base = tile_base(g, t);
#pragma unroll
    for (int j = 0; j < PER; ++j) st[elem_addr(g, base, threadIdx.x + NT * j)] = v[j];
}

__global__ void __launch_bounds__(NT, 2) mover_a(Geo g, float2 *st) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    uint32_t t = blockIdx.x;
    if (t >= NTILES) return;
    issue_cp(g, st, t, sm);
    cp_commit();
    for (; t < NTILES; t += gridDim.x) {
        cp_wait<0>();
        __syncthreads();
        float2 v[PER];
        read_modify(sm, v);
        __syncthreads();
        const uint32_t tn = t + gridDim.x;
        if (tn < NTILES) {
            issue_cp(g, st, tn, sm);
            cp_commit();
        }
        store_regs(g, st, t, v);
    }
}

__global__ void __launch_bounds__(NT, 1) mover_b(Geo g, float2 *st) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const uint32_t t0 = blockIdx.x, step = gridDim.x;
    for (int s = 0; s < 3; ++s) {
        const uint32_t t = t0 + s * step;
        if (t < NTILES) issue_cp(g, st, t, sm + (s << T));
        cp_commit();
    }
    int s = 0;
    for (uint32_t t = t0; t < NTILES; t += step) {
        cp_wait<2>();  // the groups of tiles up to this one are complete
        __syncthreads();
        float2 v[PER];
        read_modify(sm + (s << T), v);
        __syncthreads();
        const uint32_t tn = t + 3 * step;
        if (tn < NTILES) issue_cp(g, st, tn, sm + (s << T));
        cp_commit();
        store_regs(g, st, t, v);
        s = s == 2 ? 0 : s + 1;
    }
    cp_wait<0>();
}

// Loads issued into stage s so far and loads already waited for: after a
// failed wait, thread 0 waits (bounded) for the ones still in flight.
struct Stages {
    uint32_t issued[3] = {0, 0, 0}, done[3] = {0, 0, 0};
};
__device__ __forceinline__ void drain(uint64_t *bar, Stages &sg) {
    for (int s = 0; s < 3; ++s)
        while (sg.done[s] < sg.issued[s]) {
            if (!mbar_wait(bar + s, sg.done[s] & 1u)) return;
            ++sg.done[s];
        }
}

__global__ void __launch_bounds__(NT, 1) mover_c(const __grid_constant__ CUtensorMap map, Geo g, float2 *st,
                                                 unsigned *err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + 3 * TILE_BYTES);
    const uint32_t t0 = blockIdx.x, step = gridDim.x;
    Stages sg;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 3; ++s) mbar_init(bar + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    for (int s = 0; s < 3; ++s) {
        const uint32_t t = t0 + s * step;
        if (t < NTILES) {
            if (threadIdx.x == 0) {
                int c[5];
                tile_coords(g, t, c);
                mbar_expect_tx(bar + s, TILE_BYTES);
                tma_load(sm + (s << T), &map, c, bar + s);
            }
            ++sg.issued[s];
        }
    }
    int s = 0;
    for (uint32_t t = t0; t < NTILES; t += step) {
        const bool ok = mbar_wait(bar + s, sg.done[s] & 1u);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1u);
                drain(bar, sg);
            }
            return;
        }
        ++sg.done[s];
        float2 v[PER];
        read_modify(sm + (s << T), v);
        __syncthreads();
        const uint32_t tn = t + 3 * step;
        if (tn < NTILES) {
            if (threadIdx.x == 0) {
                int c[5];
                tile_coords(g, tn, c);
                fence_async_shared();
                mbar_expect_tx(bar + s, TILE_BYTES);
                tma_load(sm + (s << T), &map, c, bar + s);
            }
            ++sg.issued[s];
        }
        store_regs(g, st, t, v);
        s = s == 2 ? 0 : s + 1;
    }
}

__global__ void __launch_bounds__(NT, 1) mover_d(const __grid_constant__ CUtensorMap map, Geo g, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + 3 * TILE_BYTES);
    const uint32_t t0 = blockIdx.x, step = gridDim.x;
    Stages sg;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 3; ++s) mbar_init(bar + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
        const uint32_t t = t0 + s * step;
        if (t < NTILES) {
            if (threadIdx.x == 0) {
                int c[5];
                tile_coords(g, t, c);
                mbar_expect_tx(bar + s, TILE_BYTES);
                tma_load(sm + (s << T), &map, c, bar + s);
            }
            ++sg.issued[s];
        }
    }
    int s = 0;
    for (uint32_t t = t0; t < NTILES; t += step) {
        const bool ok = mbar_wait(bar + s, sg.done[s] & 1u);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1u);
                drain(bar, sg);
                asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
            }
            return;
        }
        ++sg.done[s];
        float2 *buf = sm + (s << T);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            float2 x = buf[threadIdx.x + NT * j];
            x.x += 1.0f;
            buf[threadIdx.x + NT * j] = x;
        }
        fence_async_shared();
        __syncthreads();
        const int s2 = s == 0 ? 2 : s - 1;  // (s + 2) mod 3: the buffer of tile i - 1
        const uint32_t tn = t + 2 * step;
        if (threadIdx.x == 0) {
            int c[5];
            tile_coords(g, t, c);
            tma_store(&map, c, buf);
            asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
            // the store of tile i - 1 has finished reading its buffer
            asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
            if (tn < NTILES) {
                tile_coords(g, tn, c);
                mbar_expect_tx(bar + s2, TILE_BYTES);
                tma_load(sm + (s2 << T), &map, c, bar + s2);
            }
        }
        if (tn < NTILES) ++sg.issued[s2];
        s = s == 2 ? 0 : s + 1;
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------- host side
#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            fprintf(stderr, "%s:%d %s: %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
            exit(1);                                                                       \
        }                                                                                  \
    } while (0)

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct MapShape {
    cuuint64_t dim[5];
    cuuint64_t stride[5];  // bytes; stride[0] is the element size
    cuuint32_t box[5];
};

// The 5-d view of the state that makes one tile one box.
static MapShape shape_of(const Geo &g) {
    MapShape m;
    if (g.R == T) {
        const cuuint64_t d[5] = {32, 1ull << (NQ - 5), 1, 1, 1};
        const cuuint32_t b[5] = {32, 1u << (T - 5), 1, 1, 1};
        for (int k = 0; k < 5; ++k) m.dim[k] = d[k], m.box[k] = b[k];
    } else {
        const int top = NQ - g.lo - g.G;
        const cuuint64_t d[5] = {1ull << g.R, 1ull << g.mid, 1ull << (g.G - 1), 2, 1ull << top};
        const cuuint32_t b[5] = {1u << g.R, 1, 1u << (g.G - 1), 2, 1};
        for (int k = 0; k < 5; ++k) m.dim[k] = d[k], m.box[k] = b[k];
    }
    m.stride[0] = 8;
    if (g.R == T) {
        for (int k = 1; k < 5; ++k) m.stride[k] = m.stride[k - 1] * m.dim[k - 1];
    } else {
        m.stride[1] = 8ull << g.R;                    // next row: bits R..lo-1
        m.stride[2] = 8ull << g.lo;                   // group bits lo..lo+G-2
        m.stride[3] = 8ull << (g.lo + g.G - 1);       // group bit lo+G-1
        m.stride[4] = 8ull << (g.lo + g.G);           // bits above the group
    }
    return m;
}

// Host check: every TMA box lies inside the map, its elements are the tile's
// elements in tile order (box element u is at elem_addr(base, u)), and the
// tiles cover the state once.
static bool check_geometry(const Geo &g, const char *name, bool full) {
    const MapShape m = shape_of(g);
    uint32_t boxel = 1;
    for (int k = 0; k < 5; ++k) boxel *= m.box[k];
    if (boxel != (1u << T)) {
        fprintf(stderr, "%s: box holds %u elements\n", name, boxel);
        return false;
    }
    unsigned char *seen = (unsigned char *)calloc((size_t)1 << (NQ - 3), 1);
    for (uint32_t t = 0; t < NTILES; ++t) {
        int c[5];
        tile_coords(g, t, c);
        for (int k = 0; k < 5; ++k)
            if (c[k] < 0 || (cuuint64_t)c[k] + m.box[k] > m.dim[k]) {
                fprintf(stderr, "%s: tile %u coordinate %d out of range\n", name, t, k);
                free(seen);
                return false;
            }
        // element order and coverage on every tile with `full`, else on 1 tile in 509
        if (!full && t % 509u != 0 && t != NTILES - 1) continue;
        const uint32_t base = tile_base(g, t);
        for (uint32_t u = 0; u < (1u << T); ++u) {
            uint32_t r = u, i[5];
            for (int k = 0; k < 5; ++k) i[k] = r % m.box[k], r /= m.box[k];
            uint64_t byte = 0;
            for (int k = 0; k < 5; ++k) byte += (uint64_t)(c[k] + i[k]) * m.stride[k];
            const uint64_t a = elem_addr(g, base, u);
            if (byte != 8 * a || a >= (1ull << NQ)) {
                fprintf(stderr, "%s: tile %u element %u: box at %llu, tile order at %llu\n", name, t, u,
                        (unsigned long long)byte / 8, (unsigned long long)a);
                free(seen);
                return false;
            }
            if (seen[a >> 3] & (1u << (a & 7))) {
                fprintf(stderr, "%s: amplitude %llu covered twice\n", name, (unsigned long long)a);
                free(seen);
                return false;
            }
            seen[a >> 3] |= (unsigned char)(1u << (a & 7));
        }
    }
    for (size_t b = 0; full && b < ((size_t)1 << (NQ - 3)); ++b)
        if (seen[b] != 0xff) {
            fprintf(stderr, "%s: amplitudes near %zu never covered\n", name, b * 8);
            free(seen);
            return false;
        }
    free(seen);
    return true;
}

static CUtensorMap make_map(EncodeTiled enc, const Geo &g, void *st) {
    const MapShape m = shape_of(g);
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUtensorMap map;
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, st, m.dim, m.stride + 1, m.box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        fprintf(stderr, "cuTensorMapEncodeTiled failed: %d\n", (int)r);
        exit(1);
    }
    return map;
}

int main(int argc, char **argv) {
    const Geo geos[3] = {{T, 0, 0, 0}, {4, 13, 9, 9}, {5, 22, 8, 17}};
    const char *gname[3] = {"contiguous", "rows16 @ 2^13", "rows32 @ 2^22"};
    // "--check-only": the whole host check (every element of every tile) and exit
    const bool full = argc > 1;
    for (int k = 0; k < 3; ++k)
        if (!check_geometry(geos[k], gname[k], full)) return 1;
    printf("geometry checks passed (%s)\n", full ? "every tile: boxes inside their maps, box order = tile order, "
                                               "state covered once"
                                             : "every tile's box inside its map; box order = tile order on sampled tiles");
    if (full) return 0;

    int dev = 0, sms = 0;
    CK(cudaSetDevice(dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess) {
        fprintf(stderr, "cuTensorMapEncodeTiled not found\n");
        return 1;
    }
    const EncodeTiled enc = (EncodeTiled)fn;

    const size_t n = (size_t)1 << NQ;
    float2 *st = nullptr;
    unsigned *err = nullptr;
    CK(cudaMalloc(&st, n * sizeof(float2)));
    CK(cudaMalloc(&err, sizeof(unsigned)));
    CK(cudaMemset(st, 0, n * sizeof(float2)));
    CK(cudaMemset(err, 0, sizeof(unsigned)));
    const int smem1 = TILE_BYTES, smem3 = 3 * TILE_BYTES + 64;
    CK(cudaFuncSetAttribute(mover_a, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    CK(cudaFuncSetAttribute(mover_b, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3));
    CK(cudaFuncSetAttribute(mover_c, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3));
    CK(cudaFuncSetAttribute(mover_d, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3));

    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int WARM = 2, REPS = 5;
    int launches = 0;
    printf("| tile order | mover | CTAs | ms per pass (mean of %d) | TB/s (read + write) |\n|---|---|---:|---:|---:|\n", REPS);
    for (int k = 0; k < 3; ++k) {
        const Geo g = geos[k];
        const CUtensorMap map = make_map(enc, g, st);
        for (int mv = 0; mv < 4; ++mv) {
            const int grid = mv == 0 ? 2 * sms : sms;
            auto launch = [&]() {
                if (mv == 0) mover_a<<<grid, NT, smem1>>>(g, st);
                if (mv == 1) mover_b<<<grid, NT, smem3>>>(g, st);
                if (mv == 2) mover_c<<<grid, NT, smem3>>>(map, g, st, err);
                if (mv == 3) mover_d<<<grid, NT, smem3>>>(map, g, err);
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
            unsigned herr = 0;
            CK(cudaMemcpy(&herr, err, sizeof herr, cudaMemcpyDeviceToHost));
            if (herr) {
                fprintf(stderr, "%s mover %c: an mbarrier wait gave up\n", gname[k], 'A' + mv);
                return 1;
            }
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ms /= REPS;
            printf("| %s | %c | %d | %.3f | %.2f |\n", gname[k], 'A' + mv, grid, ms, 2.0 * n * 8 / (ms * 1e-3) / 1e12);
        }
    }
    // every launch added 1 to every amplitude's real part exactly once
    const size_t SAMPLE = 1 << 20;
    float2 *h = (float2 *)malloc(SAMPLE * sizeof(float2));
    size_t bad = 0;
    for (int part = 0; part < 4; ++part) {
        const size_t off = (n / 4) * part;
        CK(cudaMemcpy(h, st + off, SAMPLE * sizeof(float2), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < SAMPLE; ++i)
            if (h[i].x != (float)launches || h[i].y != 0.0f) ++bad;
    }
    printf("check: %zu of %zu sampled amplitudes differ from %d\n", bad, 4 * SAMPLE, launches);
    free(h);
    CK(cudaFree(st));
    CK(cudaFree(err));
    return bad ? 1 : 0;
}
