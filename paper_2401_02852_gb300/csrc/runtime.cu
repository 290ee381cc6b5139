// Host runtime of the library: errors, device facts, scratch, instrumentation,
// pass planning and the FP64 per-layer coefficients.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "qaoa_internal.cuh"

namespace qaoa {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    return set_error(QAOA_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// ---------------------------------------------------------------------------
static std::mutex g_dev_mu;
static std::map<int, DeviceInfo> g_devs;

int device_info(DeviceInfo *out) {
    int dev = 0;
    QAOA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_devs.find(dev);
    if (it == g_devs.end()) {
        DeviceInfo d;
        d.device = dev;
        QAOA_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        int optin = 0;
        QAOA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        d.smem_optin = (size_t)optin;
        it = g_devs.emplace(dev, d).first;
    }
    *out = it->second;
    return QAOA_OK;
}

// ---------------------------------------------------------------------------
static std::mutex g_scratch_mu;
static std::map<std::pair<int, cudaStream_t>, Scratch> g_scratch;

int current_device_slot() {
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cuda_error(e, "cudaGetDevice");
        return -1;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error(QAOA_ERANGE, "device ordinal %d", dev);
        return -1;
    }
    return dev;
}

int scratch_for(cudaStream_t stream, size_t dev_bytes, size_t host_bytes, Scratch **out) {
    int dev = 0;
    QAOA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    Scratch &s = g_scratch[{dev, stream}];
    if (s.dev_bytes < dev_bytes) {
        // The stream may still use the old block: wait for it before freeing.
        QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
        if (s.dev) cudaFree(s.dev);
        s.dev = nullptr;
        s.dev_bytes = 0;
        size_t want = dev_bytes < (1u << 20) ? (1u << 20) : dev_bytes + dev_bytes / 4;
        if (cudaMalloc(&s.dev, want) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QAOA_ENOMEM, "scratch: cudaMalloc(%zu) failed", want);
        }
        s.dev_bytes = want;
    }
    if (s.host_bytes < host_bytes) {
        QAOA_CUDA_TRY(cudaStreamSynchronize(stream));
        if (s.host) cudaFreeHost(s.host);
        s.host = nullptr;
        s.host_bytes = 0;
        size_t want = host_bytes < 4096 ? 4096 : host_bytes;
        if (cudaMallocHost(&s.host, want) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QAOA_ENOMEM, "scratch: cudaMallocHost(%zu) failed", want);
        }
        s.host_bytes = want;
    }
    *out = &s;
    return QAOA_OK;
}

static int release_all_scratch() {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_scratch) {
        cudaSetDevice(kv.first.first);
        cudaDeviceSynchronize();
        if (kv.second.dev) cudaFree(kv.second.dev);
        if (kv.second.host) cudaFreeHost(kv.second.host);
    }
    g_scratch.clear();
    cudaSetDevice(cur);
    return QAOA_OK;
}

// ---------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
static std::atomic<bool> g_profile{false};
static std::mutex g_prof_mu;
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;
static thread_local cudaEvent_t t_pending = nullptr;

static const char *k_names[K_NUM_KINDS] = {
    "cost_table", "pass_low", "pass_high", "small_n", "reduce",
    "success_prob", "adjoint_low", "adjoint_high", "adjoint_seed", "serve_small", "sample"};

static cudaEvent_t take_event() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void profile_before(int kind, cudaStream_t stream) {
    (void)kind;
    if (!g_profile.load(std::memory_order_relaxed)) return;
    t_pending = take_event();
    cudaEventRecord(t_pending, stream);
}

int profile_after(int kind, cudaStream_t stream) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, k_names[kind]);
    if (g_profile.load(std::memory_order_relaxed) && t_pending) {
        cudaEvent_t b = take_event();
        cudaEventRecord(b, stream);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.push_back({kind, t_pending, b});
        t_pending = nullptr;
    }
    return QAOA_OK;
}

// ---------------------------------------------------------------------------
int make_plan_geo(int n, int T, int G, Plan *plan, bool z2, bool wide) {
    // In the halved representation the stored state has n - 1 index bits and
    // the low pass covers T - 1 of them plus the mirror (the top qubit).
    const int nb = z2 ? n - 1 : n;
    const int low = z2 ? T - 1 : T;
    if (nb < T || n > QAOA_MAX_N || (!z2 && n < T + 1))
        return set_error(QAOA_ERANGE, "plan: n=%d outside [%d, %d]", n, T + 1, QAOA_MAX_N);
    plan->n = n;
    plan->state_bits = nb;
    plan->z2 = z2 ? 1 : 0;
    plan->tile_bits = T;
    plan->pass[0] = {0, T, T};
    // k high groups cover the R bits above the low pass: narrow groups span G
    // bits with rows of T - G contiguous amplitudes, wide ones G - 1 bits with
    // rows of T - G + 1; as many groups go wide (top first) as the k G - R spare
    // bits allow.  The last group ends at bit nb, so when the groups have room
    // to spare it re-covers already mixed bits, which it carries without
    // butterflies (`bits` counts only the new ones).
    const int R = nb - low;
    const int k = R > 0 ? (R + G - 1) / G : 0;
    if (1 + k > 8) return set_error(QAOA_ERANGE, "plan: n=%d needs too many passes", n);
    const int w = wide ? std::min(k, k * G - R) : 0;
    int lo = low;
    for (int i = 0; i < k; ++i) {
        const int g = i >= k - w ? G - 1 : G;
        const int glo = lo + g <= nb ? lo : nb - g;
        plan->pass[1 + i] = {glo, lo + g <= nb ? g : nb - lo, T - g};
        lo += g;
    }
    plan->n_passes = 1 + k;
    return QAOA_OK;
}

int make_plan(int n, int dtype, Plan *plan, bool z2) {
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype %d", dtype);
    // complex64 rows of 16 amplitudes are 128 B: take wide groups (256 B rows)
    // where the bit count allows; complex128 rows are 256 B already.
    return dtype == QAOA_C64 ? make_plan_geo(n, T_C64, G_MAX_C64, plan, z2, true)
                             : make_plan_geo(n, T_C128, G_MAX_C128, plan, z2);
}

std::vector<Launch> make_schedule(int n_passes, int p) {
    std::vector<Launch> out;
    if (p == 0) {
        out.push_back({0, 0, MODE_INIT});
        return out;
    }
    // Pass orders of even and odd layers.  With two or more high groups the low
    // pass (index 0) is second, so both ends of every layer are high groups and
    // each layer boundary fuses.  With one high group the orders are [0, 1] and
    // [1, 0]: the boundary on group 1 fuses, the one on the low pass does not.
    const int k = n_passes - 1;
    std::vector<int> even, odd;
    if (k >= 2) {
        even.push_back(1);
        even.push_back(0);
        for (int g = 2; g <= k; ++g) even.push_back(g);
        odd.push_back(k);
        odd.push_back(0);
        for (int g = k - 1; g >= 1; --g) odd.push_back(g);
    } else {
        even = {0, 1};
        odd = {1, 0};
    }
    for (int l = 0; l < p; ++l) {
        const std::vector<int> &ord = (l % 2 == 0) ? even : odd;
        for (int j = 0; j < n_passes; ++j) {
            const int ps = ord[j];
            const bool first = j == 0, last = j == n_passes - 1;
            if (l > 0 && first && ps != 0) continue;  // fused into the previous layer's last pass
            int mode = MODE_PLAIN;
            if (first) mode = (l == 0) ? MODE_INIT : MODE_PHASE;
            if (last && l + 1 < p && ps != 0) mode = MODE_FUSED;
            out.push_back({ps, l, mode});
        }
    }
    return out;
}

std::vector<Launch> make_adj_schedule(int n_passes, int p) {
    std::vector<Launch> out;
    const int k = n_passes - 1;
    std::vector<int> even, odd;
    if (k >= 2) {
        even.push_back(1);
        even.push_back(0);
        for (int g = 2; g <= k; ++g) even.push_back(g);
        odd.push_back(k);
        odd.push_back(0);
        for (int g = k - 1; g >= 1; --g) odd.push_back(g);
    } else {
        even = {1, 0};
        odd = {1, 0};
    }
    for (int j = 0; j < p; ++j) {  // j-th layer undone: la = p - 1 - j
        const int la = p - 1 - j;
        const std::vector<int> &ord = (j % 2 == 0) ? even : odd;
        for (int q = 0; q < n_passes; ++q) {
            if (k >= 2 && j > 0 && q == 0) continue;  // undone by the previous layer's fused pass
            int mode = A_PLAIN;
            if (q == n_passes - 1) mode = (k >= 2 && la > 0) ? A_FUSED : A_PHASE;
            out.push_back({ord[q], la, mode});
        }
    }
    return out;
}

// The non-unit coefficient as the kernels' arithmetic holds it: FP32, FP64,
// or a double-float pair (the nearest float, then the nearest float to the
// remainder; hi + lo is exact in FP64).
static double coef_in_arith(double x, int arith) {
    if (arith == ARITH_F32) return (double)(float)x;
    if (arith == ARITH_DF) {
        const float hi = (float)x;
        const float lo = (float)(x - (double)hi);
        return (double)hi + (double)lo;
    }
    return x;
}

LayerCoef layer_coef(double beta, int sign, int arith) {
    const double c = std::cos(beta), sn = std::sin(beta);
    const double S = sign * sn;  // butterfly: a' = c a + i S b, b' = i S a + c b
    // sigma [x I + i y X] is unitary iff sigma^2 (x^2 + y^2) = 1.  sigma is taken
    // from the coefficient as rounded to the kernels' arithmetic, so the product
    // the kernels apply is unitary up to their own rounding: an FP64 sigma = cos
    // beta beside an FP32 S / c would scale the norm by the same factor on every
    // qubit of a layer (about 1e-6 over an n = 30, p = 10 evolution).
    LayerCoef k;
    if (std::fabs(c) >= std::fabs(S)) {
        k.A = 1.0;
        k.B = coef_in_arith(S / c, arith);
        k.sigma = std::copysign(1.0 / std::sqrt(1.0 + k.B * k.B), c);
        k.unit_a = true;
    } else {
        k.A = coef_in_arith(c / S, arith);
        k.B = 1.0;
        k.sigma = std::copysign(1.0 / std::sqrt(1.0 + k.A * k.A), S);
        k.unit_a = false;
    }
    return k;
}

void phase_table(double gamma, double scale, int m, double *re, double *im) {
    for (int c = 0; c <= m; ++c) {
        re[c] = scale * std::cos(gamma * (double)c);
        im[c] = -scale * std::sin(gamma * (double)c);
    }
}

}  // namespace qaoa

using namespace qaoa;

extern "C" {

const char *qaoa_last_error(void) { return g_err; }

int qaoa_version(void) { return 100; }

int qaoa_release_scratch(void) { return release_all_scratch(); }

int qaoa_plan(int n, int dtype, int flags, int *group_lo, int *group_bits, int *row_bits) {
    Plan pl;
    int rc = make_plan(n, dtype, &pl, (flags & QAOA_Z2_HALF) != 0);
    if (rc) return rc;
    for (int i = 0; i < pl.n_passes; ++i) {
        if (group_lo) group_lo[i] = pl.pass[i].lo;
        if (group_bits) group_bits[i] = pl.pass[i].bits;
        if (row_bits) row_bits[i] = pl.pass[i].row;
    }
    return pl.n_passes;
}

int qaoa_pass_schedule(int n, int p, int dtype, int flags, int max_launches, int *pass_index, int *layer,
                       int *mode) {
    Plan pl;
    if (p < 0) return set_error(QAOA_EINVAL, "p=%d", p);
    int rc = make_plan(n, dtype, &pl, (flags & QAOA_Z2_HALF) != 0);
    if (rc) return rc;
    const std::vector<Launch> seq = make_schedule(pl.n_passes, p);
    for (size_t i = 0; i < seq.size() && (int)i < max_launches; ++i) {
        if (pass_index) pass_index[i] = seq[i].pass;
        if (layer) layer[i] = seq[i].la;
        if (mode) mode[i] = seq[i].mode;
    }
    return (int)seq.size();
}

extern "C" int qaoa_adjoint_schedule(int n, int p, int dtype, int max_launches, int *pass_index, int *layer,
                                     int *mode) {
    if (p < 1) return set_error(QAOA_EINVAL, "p=%d", p);
    if (dtype != QAOA_C64 && dtype != QAOA_C128) return set_error(QAOA_EINVAL, "dtype=%d", dtype);
    Plan pl;
    // the backward passes tile both states in 2^12-amplitude tiles, groups of
    // at most 8 bits (complex64 also takes 7-bit groups with 256-byte rows)
    int rc = make_plan_geo(n, 12, 8, &pl, false, dtype == QAOA_C64);
    if (rc) return rc;
    const std::vector<Launch> seq = make_adj_schedule(pl.n_passes, p);
    for (size_t i = 0; i < seq.size() && (int)i < max_launches; ++i) {
        if (pass_index) pass_index[i] = seq[i].pass;
        if (layer) layer[i] = seq[i].la;
        if (mode) mode[i] = seq[i].mode;
    }
    return (int)seq.size();
}

int qaoa_profile_enable(int on) {
    g_profile.store(on != 0);
    return QAOA_OK;
}

int qaoa_profile_read(int max_kinds, uint64_t *launches, double *ms) {
    for (int i = 0; i < max_kinds; ++i) {
        if (launches) launches[i] = 0;
        if (ms) ms[i] = 0.0;
    }
    QAOA_CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof) {
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        if (r.kind < max_kinds) {
            if (launches) launches[r.kind] += 1;
            if (ms) ms[r.kind] += t;
        }
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_prof.clear();
    return K_NUM_KINDS;
}

const char *qaoa_kernel_name(int kind) {
    if (kind < 0 || kind >= K_NUM_KINDS) return "";
    return k_names[kind];
}

uint64_t qaoa_launch_count(void) { return g_launches.load(); }

}  // extern "C"
