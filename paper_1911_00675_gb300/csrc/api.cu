// Host side of libpmh.so: handle, argument validation, per-m tables, the
// device work queue, the launch planner, CUDA-graph caching, and the
// estimation / merge entry points.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "launch.h"

using namespace pmh;

namespace {

thread_local std::string g_create_error;

struct TableBuf {
    void *dev = nullptr;
    Tables t{};
};

struct GraphKey {
    const void *ids, *weights, *offsets, *out_ids, *out_q, *status, *counters;
    int64_t num_sets;
    uint32_t m;
    int32_t variants[8];
    int32_t num_variants, precision, profiling;
    uint64_t seed;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

}  // namespace

struct pmh_handle_s {
    int device = 0;
    int sm_count = 0;
    std::string err;
    std::map<uint32_t, TableBuf> tables;
    // work queue
    uint64_t *queue = nullptr;
    int64_t queue_cap = 0;
    unsigned int *qmeta = nullptr;   // histogram, running starts, per-family heads
    SetStat *stats = nullptr;        // per-set statistics
    int64_t stats_cap = 0;
    cudaStream_t cap_stream = nullptr;
    bool graph_valid = false;
    GraphKey gkey{};
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    // planner knobs (tunable)
    float t_c = 4.0f;
    int rounds = 5;
    // profiling events
    bool profiling = false;
    bool prof_recorded = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

static pmh_status fail(pmh_handle h, pmh_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return code;
}

#define CUDA_TRY(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail((h), PMH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ tables
// Per-m constants of Sec. ProbMinHash2/3/4 in FP64 (host libm), plus FP32
// copies for the filter.
static pmh_status get_tables(pmh_handle h, uint32_t m, Tables *out) {
    auto it = h->tables.find(m);
    if (it != h->tables.end()) { *out = it->second.t; return PMH_OK; }
    const size_t n = (size_t)m + 1;
    std::vector<double> beta(n, 0.0), gamma(n, 0.0), dgamma(n, 0.0), c4(n, 0.0), inv4(n, 0.0);
    for (uint32_t i = 1; i <= m; i++) beta[i] = (double)m / (double)(m - i + 1);
    double lambda1 = 0.0, c3 = 0.0, inv3 = 0.0, delta = 0.0;
    if (m >= 2) {
        lambda1 = std::log1p(1.0 / (double)(m - 1));
        c3 = std::expm1(-lambda1);
        inv3 = 1.0 / lambda1;
        delta = 1.0 / lambda1;
        for (uint32_t i = 1; i < m; i++) {
            const double li = std::log1p(1.0 / (double)(m - i));
            c4[i] = std::expm1(-li);
            inv4[i] = 1.0 / li;
            gamma[i] = std::log1p((double)i / (double)(m - i)) / lambda1;
            dgamma[i] = gamma[i] - gamma[i - 1];
        }
    }
    std::vector<float> f[5];
    const std::vector<double> *src[5] = {&beta, &gamma, &dgamma, &c4, &inv4};
    for (int a = 0; a < 5; a++) {
        f[a].resize(n);
        for (size_t i = 0; i < n; i++) f[a][i] = (float)(*src[a])[i];
    }
    const size_t bytes = 5 * n * sizeof(double) + 5 * n * sizeof(float);
    TableBuf tb;
    CUDA_TRY(h, cudaMalloc(&tb.dev, bytes));
    char *d = (char *)tb.dev;
    std::vector<char> host(bytes);
    for (int a = 0; a < 5; a++) std::memcpy(host.data() + a * n * sizeof(double), src[a]->data(), n * sizeof(double));
    for (int a = 0; a < 5; a++)
        std::memcpy(host.data() + 5 * n * sizeof(double) + a * n * sizeof(float), f[a].data(), n * sizeof(float));
    cudaError_t e = cudaMemcpy(tb.dev, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(tb.dev); return fail(h, PMH_ERR_CUDA, "table upload: %s", cudaGetErrorString(e)); }
    Tables &t = tb.t;
    t.m = m;
    t.beta = (const double *)(d);
    t.gamma = (const double *)(d + 1 * n * sizeof(double));
    t.dgamma = (const double *)(d + 2 * n * sizeof(double));
    t.c4 = (const double *)(d + 3 * n * sizeof(double));
    t.inv4 = (const double *)(d + 4 * n * sizeof(double));
    const char *fb = d + 5 * n * sizeof(double);
    t.beta32 = (const float *)(fb);
    t.gamma32 = (const float *)(fb + 1 * n * sizeof(float));
    t.dgamma32 = (const float *)(fb + 2 * n * sizeof(float));
    t.c4_32 = (const float *)(fb + 3 * n * sizeof(float));
    t.inv4_32 = (const float *)(fb + 4 * n * sizeof(float));
    t.c3 = c3;
    t.inv3 = inv3;
    t.delta = delta;
    t.c3_32 = (float)c3;
    t.inv3_32 = (float)inv3;
    t.delta32 = (float)delta;
    // Exp(lambda_1;0,1) >= U * (1-e^-lambda_1)/lambda_1 (since -log1p(-a) >= a); round the factor down
    double lo = (m >= 2) ? -c3 / lambda1 : 1.0;
    float lo32 = (float)lo;
    if ((double)lo32 > lo) lo32 = std::nextafterf(lo32, 0.0f);
    t.te_lo = lo32;
    t.lambda1_32 = (float)lambda1;
    h->tables[m] = tb;
    *out = t;
    return PMH_OK;
}

// ------------------------------------------------------------------ queue
// Items (variant, set) in family-major order (ProbMinHash1/1a, 2, 3/3a, 4),
// each family sorted by decreasing floor(log2(n+1)) (largest sets first).
// Meta layout: [0, 256) histogram per (family, bucket), [256, 512) running
// starts, [512, 516) per-family head counters of the persistent kernels.
constexpr int kQHist = 0, kQStart = 256, kQHead = 512, kQMetaWords = 520;

struct FamOfVariant {
    int f[8];
};

__device__ __forceinline__ int queue_bucket(const int64_t *off, int64_t s) {
    int64_t n = off[s + 1] - off[s];
    if (n < 0) n = 0;
    return 63 - __clzll((long long)(n + 1));
}

__global__ void queue_count(const int64_t *off, int64_t num_sets, int32_t nv, FamOfVariant fv, unsigned int *meta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < num_sets * nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i % num_sets;
        const int v = (int)(i / num_sets);
        atomicAdd(&meta[kQHist + (fv.f[v] - 1) * 64 + queue_bucket(off, s)], 1u);
    }
}
__global__ void queue_starts(unsigned int *meta) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned int acc = 0;
        for (int f = 0; f < 4; ++f)
            for (int b = 63; b >= 0; --b) { meta[kQStart + f * 64 + b] = acc; acc += meta[kQHist + f * 64 + b]; }
        for (int f = 0; f < 4; ++f) meta[kQHead + f] = 0;
    }
}
__global__ void queue_scatter(const int64_t *off, int64_t num_sets, int32_t nv, FamOfVariant fv, unsigned int *meta,
                              uint64_t *queue) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < num_sets * nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i % num_sets;
        const int64_t v = i / num_sets;
        const unsigned int pos = atomicAdd(&meta[kQStart + (fv.f[v] - 1) * 64 + queue_bucket(off, s)], 1u);
        queue[pos] = ((uint64_t)v << 40) | (uint64_t)s;
    }
}

// Per-set statistics, computed once per set for all variants: the weight sum
// (FP64; it only sets the threshold T), the number of positive weights, and a
// bad-weight flag (negative, NaN, +-inf, or a subnormal whose reciprocal
// overflows).  One block per set, grid-stride over sets.
__global__ void __launch_bounds__(256) set_stats_kernel(const int64_t *off, const double *w, int64_t num_sets,
                                                        SetStat *out) {
    __shared__ double ssum[8];
    __shared__ int snp[8], sbad[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = blockIdx.x; s < num_sets; s += gridDim.x) {
        const int64_t b = off[s], e = off[s + 1];
        double sum = 0.0;
        int np = 0, bad = 0;
        for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            const double x = w[i];
            const uint64_t bits = (uint64_t)__double_as_longlong(x);
            const int ex = (int)(bits >> 52) & 0x7FF;
            const bool neg = (bits >> 63) != 0;
            if (ex == 0x7FF || (neg && (bits << 1) != 0)) { bad = 1; continue; }
            if (neg || (bits << 1) == 0) continue;
            if (ex == 0 && isinf(__drcp_rn(x))) { bad = 1; continue; }
            sum += x;
            np++;
        }
        for (int o = 16; o; o >>= 1) {
            sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
            np += __shfl_xor_sync(0xFFFFFFFFu, np, o);
            bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, o);
        }
        if (lane == 0) { ssum[warp] = sum; snp[warp] = np; sbad[warp] = bad; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double S = 0.0;
            int N = 0, B = 0;
            for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { S += ssum[j]; N += snp[j]; B |= sbad[j]; }
            SetStat r;
            r.wsum = S;
            r.npos = N;
            r.bad = B;
            out[s] = r;
        }
        __syncthreads();
    }
}

static pmh_status ensure_queue(pmh_handle h, int64_t items) {
    if (!h->qmeta) CUDA_TRY(h, cudaMalloc(&h->qmeta, kQMetaWords * sizeof(unsigned int)));
    if (items > h->queue_cap) {
        if (h->queue) cudaFree(h->queue);
        h->queue = nullptr;
        h->queue_cap = 0;
        int64_t cap = items < 1024 ? 1024 : items;
        cudaError_t e = cudaMalloc(&h->queue, (size_t)cap * sizeof(uint64_t));
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "queue allocation (%lld items): %s", (long long)cap, cudaGetErrorString(e));
        h->queue_cap = cap;
        h->graph_valid = false;
    }
    return PMH_OK;
}

static pmh_status ensure_stats(pmh_handle h, int64_t num_sets) {
    if (num_sets > h->stats_cap) {
        if (h->stats) cudaFree(h->stats);
        h->stats = nullptr;
        h->stats_cap = 0;
        int64_t cap = num_sets < 1024 ? 1024 : num_sets;
        cudaError_t e = cudaMalloc(&h->stats, (size_t)cap * sizeof(SetStat));
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "set statistics (%lld sets): %s", (long long)cap, cudaGetErrorString(e));
        h->stats_cap = cap;
        h->graph_valid = false;
    }
    return PMH_OK;
}

static uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Launch plan per family present: warp teams when at least 12 warps per SM
// fit, else CTA teams.  Computed outside any stream capture (it sets kernel
// attributes).
struct Plan {
    int nfam;
    int fam[4];
    int64_t qbase[4], qlen[4];
    LaunchShape shape[4];
    int grid[4];
};

static pmh_status plan_sketch(pmh_handle h, const SketchParams &p, int precision, Plan *out) {
    const bool f32 = precision == PMH_FP32_RECHECK;
    const bool perm = false;   // the permutation arrays are part of the ProbMinHash2/4 kernels' layout
    int64_t per_fam[4] = {0, 0, 0, 0};
    for (int v = 0; v < p.num_variants; v++) per_fam[family_of(p.variants[v]) - 1] += p.num_sets;
    out->nfam = 0;
    int64_t base = 0;
    for (int f = 1; f <= 4; f++) {
        const int64_t items = per_fam[f - 1];
        if (items == 0) continue;
        LaunchShape warp_s{}, cta_s{};
        cudaError_t e = sketch_shape_any(f32, f, false, p.m, perm, &warp_s);
        if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
        LaunchShape shape = warp_s;
        if (warp_s.blocks_per_sm * 4 < 12) {
            e = sketch_shape_any(f32, f, true, p.m, perm, &cta_s);
            if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
            if (cta_s.blocks_per_sm > 0) shape = cta_s;
        }
        if (shape.blocks_per_sm <= 0) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u does not fit in shared memory", p.m);
        int grid = h->sm_count * shape.blocks_per_sm;
        const int64_t teams_needed = shape.cta_team ? items : (items + 3) / 4;
        if (teams_needed < grid) grid = (int)std::max<int64_t>(1, teams_needed);
        const int j = out->nfam++;
        out->fam[j] = f;
        out->qbase[j] = base;
        out->qlen[j] = items;
        out->shape[j] = shape;
        out->grid[j] = grid;
        base += items;
    }
    return PMH_OK;
}

// Enqueues the whole batch (queue build + one persistent kernel per family) on `st`.
static pmh_status enqueue_sketch(pmh_handle h, const SketchParams &p0, const Plan &plan, int precision,
                                 cudaStream_t st) {
    SketchParams p = p0;
    const int64_t items = p.num_sets * p.num_variants;
    FamOfVariant fv{};
    for (int v = 0; v < p.num_variants; v++) fv.f[v] = family_of(p.variants[v]);
    const int qb = 256;
    int qg = (int)std::min<int64_t>((items + qb - 1) / qb, (int64_t)h->sm_count * 8);
    if (qg < 1) qg = 1;
    if (h->profiling) CUDA_TRY(h, cudaEventRecord(h->ev[0], st));
    CUDA_TRY(h, cudaMemsetAsync(h->qmeta, 0, kQMetaWords * sizeof(unsigned int), st));
    queue_count<<<qg, qb, 0, st>>>(p.offsets, p.num_sets, p.num_variants, fv, h->qmeta);
    queue_starts<<<1, 32, 0, st>>>(h->qmeta);
    queue_scatter<<<qg, qb, 0, st>>>(p.offsets, p.num_sets, p.num_variants, fv, h->qmeta, h->queue);
    const int sg = (int)std::min<int64_t>(p.num_sets, (int64_t)h->sm_count * 8);
    set_stats_kernel<<<sg, 256, 0, st>>>(p.offsets, p.weights, p.num_sets, h->stats);
    CUDA_TRY(h, cudaGetLastError());
    p.stats = h->stats;
    if (h->profiling) CUDA_TRY(h, cudaEventRecord(h->ev[1], st));
    for (int j = 0; j < plan.nfam; j++) {
        p.queue = h->queue + plan.qbase[j];
        p.queue_len = plan.qlen[j];
        p.head = h->qmeta + kQHead + (plan.fam[j] - 1);
        cudaError_t e = sketch_launch_any(precision == PMH_FP32_RECHECK, plan.fam[j], plan.shape[j], plan.grid[j], p, st);
        if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "sketch launch: %s", cudaGetErrorString(e));
    }
    if (h->profiling) CUDA_TRY(h, cudaEventRecord(h->ev[2], st));
    return PMH_OK;
}

// ------------------------------------------------------------------ ABI
extern "C" pmh_status pmh_create(pmh_handle *out, int device) {
    if (!out) return fail(nullptr, PMH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return fail(nullptr, PMH_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= count) return fail(nullptr, PMH_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, count);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, PMH_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    pmh_handle h = new pmh_handle_s();
    h->device = device;
    e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, PMH_ERR_CUDA, "device setup: %s", cudaGetErrorString(e));
    }
    const char *ng = std::getenv("PMH_NO_GRAPH");
    h->use_graph = !(ng && ng[0] == '1');
    *out = h;
    return PMH_OK;
}

extern "C" void pmh_destroy(pmh_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    for (int i = 0; i < 3; i++) if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (auto &kv : h->tables) cudaFree(kv.second.dev);
    if (h->queue) cudaFree(h->queue);
    if (h->qmeta) cudaFree(h->qmeta);
    if (h->stats) cudaFree(h->stats);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

extern "C" const char *pmh_last_error(pmh_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

extern "C" pmh_status pmh_set_profiling(pmh_handle h, int32_t enable) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    CUDA_TRY(h, cudaSetDevice(h->device));
    if (enable && !h->ev[0])
        for (int i = 0; i < 3; i++) CUDA_TRY(h, cudaEventCreate(&h->ev[i]));
    h->profiling = enable != 0;
    return PMH_OK;
}

extern "C" pmh_status pmh_last_kernel_ms(pmh_handle h, float *queue_ms, float *sketch_ms) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (!h->prof_recorded || !h->ev[0]) return fail(h, PMH_ERR_INVALID_ARG, "profiling was off for the last call");
    CUDA_TRY(h, cudaEventSynchronize(h->ev[2]));
    float a = 0.0f, b = 0.0f;
    CUDA_TRY(h, cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    CUDA_TRY(h, cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
    if (queue_ms) *queue_ms = a;
    if (sketch_ms) *sketch_ms = b;
    return PMH_OK;
}

extern "C" pmh_status pmh_sketch_batch(pmh_handle h, const uint64_t *ids, const double *weights, const int64_t *offsets,
                                       int64_t num_sets, uint32_t m, const int32_t *variants, int32_t num_variants,
                                       int32_t precision, uint64_t seed, uint64_t *out_ids, double *out_q,
                                       int32_t *set_status, uint64_t *counters, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_sets < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_sets < 0");
    if (num_sets >= (1ll << 40)) return fail(h, PMH_ERR_UNSUPPORTED, "num_sets >= 2^40");
    if (num_variants >= 1 && num_variants <= 8 && num_sets * num_variants > 0x7FFFFFFFll - (1ll << 24))
        return fail(h, PMH_ERR_UNSUPPORTED, "num_sets * num_variants too large for one call");
    if (m < 1 || m > PMH_MAX_M) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, %u]", m, PMH_MAX_M);
    if (!variants || num_variants < 1 || num_variants > 8) return fail(h, PMH_ERR_INVALID_ARG, "need 1..8 variants");
    if (precision != PMH_FP64 && precision != PMH_FP32_RECHECK) return fail(h, PMH_ERR_INVALID_ARG, "bad precision %d", precision);
    bool has_perm = false;
    for (int v = 0; v < num_variants; v++) {
        if (variants[v] < PMH_V1 || variants[v] > PMH_V4) return fail(h, PMH_ERR_INVALID_ARG, "bad variant %d", variants[v]);
        if ((variants[v] == PMH_V3 || variants[v] == PMH_V3A || variants[v] == PMH_V4) && m < 2)
            return fail(h, PMH_ERR_INVALID_ARG, "variant %d requires m >= 2", variants[v]);
        has_perm |= (variants[v] == PMH_V2 || variants[v] == PMH_V4);
    }
    if (num_sets == 0) return PMH_OK;
    if (!ids || !weights || !offsets || !out_ids) return fail(h, PMH_ERR_INVALID_ARG, "NULL ids/weights/offsets/out_ids");
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t st = (cudaStream_t)stream;
    Tables tab;
    pmh_status rc = get_tables(h, m, &tab);
    if (rc) return rc;
    rc = ensure_queue(h, num_sets * num_variants);
    if (rc) return rc;
    rc = ensure_stats(h, num_sets);
    if (rc) return rc;

    SketchParams p{};
    p.ids = ids;
    p.weights = weights;
    p.offsets = offsets;
    p.num_sets = num_sets;
    p.m = m;
    p.mixed_seed = host_mix64(seed);
    for (int v = 0; v < num_variants; v++) p.variants[v] = variants[v];
    p.num_variants = num_variants;
    p.tab = tab;
    p.out_ids = out_ids;
    p.out_q = out_q;
    p.status = set_status;
    p.counters = (unsigned long long *)counters;
    p.t_factor = (float)(std::log((double)m) + h->t_c);
    p.rounds = h->rounds;
    p.cap_points = (uint32_t)(64.0 * m * std::log((double)m + 1.0)) + 4096;
    (void)has_perm;

    Plan plan;
    rc = plan_sketch(h, p, precision, &plan);
    if (rc) return rc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st) CUDA_TRY(h, cudaStreamIsCapturing(st, &cs));
    if (!h->use_graph || cs != cudaStreamCaptureStatusNone || !st) {
        h->prof_recorded = h->profiling;
        return enqueue_sketch(h, p, plan, precision, st);
    }

    GraphKey key{};
    key.ids = ids; key.weights = weights; key.offsets = offsets; key.out_ids = out_ids; key.out_q = out_q;
    key.status = set_status; key.counters = counters; key.num_sets = num_sets; key.m = m;
    for (int v = 0; v < num_variants; v++) key.variants[v] = variants[v];
    key.num_variants = num_variants; key.precision = precision; key.seed = seed;
    key.profiling = h->profiling ? 1 : 0;
    h->prof_recorded = h->profiling;
    if (!(h->graph_valid && h->gkey == key)) {
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
        h->graph_valid = false;
        CUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_sketch(h, p, plan, precision, h->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        h->gkey = key;
        h->graph_valid = true;
    }
    CUDA_TRY(h, cudaGraphLaunch(h->gexec, st));
    return PMH_OK;
}

// ------------------------------------------------------------------ estimation
// All-pairs equal-component counts, Eq. jaccard_estimator.  64x64 tile of
// pairs per CTA, 16 components per shared-memory stage, 4x4 pairs per thread
// (rows ty + 16i, columns tx + 16j: conflict-free shared reads).
constexpr int kTile = 64, kKc = 16;

__global__ void __launch_bounds__(256) allpairs_kernel(const uint64_t *__restrict__ sig, int64_t n, uint32_t m,
                                                       int upper_only, uint16_t *__restrict__ out) {
    __shared__ uint64_t As[kKc][kTile + 1];
    __shared__ uint64_t Bs[kKc][kTile + 1];
    const int64_t ta = blockIdx.y, tb = blockIdx.x;
    if (upper_only && ta > tb) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t a0 = ta * kTile, b0 = tb * kTile;
    uint32_t cnt[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) cnt[i][j] = 0;
    for (uint32_t kc = 0; kc < m; kc += kKc) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int idx = threadIdx.x + 256 * q;
            const int r = idx >> 4, kk = idx & 15;
            const uint32_t k = kc + kk;
            const int64_t ra = a0 + r, rb = b0 + r;
            // out-of-range rows/components load two different sentinels so they never match
            As[kk][r] = (ra < n && k < m) ? sig[ra * m + k] : 0xFFFFFFFFFFFFFFFFull;
            Bs[kk][r] = (rb < n && k < m) ? sig[rb * m + k] : 0xFFFFFFFFFFFFFFFEull;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKc; kk++) {
            uint64_t a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) cnt[i][j] += (a[i] == b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int64_t a = a0 + ty + 16 * i;
        if (a >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t b = b0 + tx + 16 * j;
            if (b >= n || (upper_only && a > b)) continue;
            out[a * n + b] = (uint16_t)cnt[i][j];
        }
    }
}

__global__ void pairs_kernel(const uint64_t *__restrict__ sa, const uint64_t *__restrict__ sb,
                             const int64_t *__restrict__ pa, const int64_t *__restrict__ pb, int64_t np, uint32_t m,
                             uint32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < np; i += nw) {
        const uint64_t *x = sa + pa[i] * (int64_t)m;
        const uint64_t *y = sb + pb[i] * (int64_t)m;
        uint32_t c = 0;
        for (uint32_t k = lane; k < m; k += 32) c += (x[k] == y[k]);
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) out[i] = c;
    }
}

__global__ void merge_kernel(const double *__restrict__ q, const uint64_t *__restrict__ z, int64_t parts, uint32_t m,
                             double *__restrict__ oq, uint64_t *__restrict__ oz) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        double bq = __longlong_as_double(0x7FF0000000000000ll);
        uint64_t bz = 0;
        for (int64_t p = 0; p < parts; p++) {
            const double x = q[p * m + k];
            const uint64_t d = z[p * m + k];
            if (x < bq || (x == bq && !isinf(x) && d < bz)) { bq = x; bz = d; }
        }
        oq[k] = bq;
        oz[k] = isinf(bq) ? 0 : bz;
    }
}

extern "C" pmh_status pmh_estimate_allpairs(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m,
                                            int32_t upper_only, uint16_t *counts, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_sigs < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_sigs < 0");
    if (m < 1 || m > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, 65535]", m);
    if (num_sigs == 0) return PMH_OK;
    if (!sigs || !counts) return fail(h, PMH_ERR_INVALID_ARG, "NULL sigs/counts");
    const int64_t tiles = (num_sigs + kTile - 1) / kTile;
    if (tiles > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "num_sigs too large for one launch");
    CUDA_TRY(h, cudaSetDevice(h->device));
    dim3 grid((unsigned)tiles, (unsigned)tiles);
    allpairs_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(sigs, num_sigs, m, upper_only ? 1 : 0, counts);
    CUDA_TRY(h, cudaGetLastError());
    return PMH_OK;
}

extern "C" pmh_status pmh_estimate_pairs(pmh_handle h, const uint64_t *sig_a, const uint64_t *sig_b,
                                         const int64_t *pairs_a, const int64_t *pairs_b, int64_t num_pairs, uint32_t m,
                                         uint32_t *counts, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_pairs < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_pairs < 0");
    if (m < 1) return fail(h, PMH_ERR_INVALID_ARG, "m < 1");
    if (num_pairs == 0) return PMH_OK;
    if (!sig_a || !sig_b || !pairs_a || !pairs_b || !counts) return fail(h, PMH_ERR_INVALID_ARG, "NULL pointer");
    CUDA_TRY(h, cudaSetDevice(h->device));
    int grid = (int)std::min<int64_t>((num_pairs + 7) / 8, (int64_t)h->sm_count * 16);
    pairs_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(sig_a, sig_b, pairs_a, pairs_b, num_pairs, m, counts);
    CUDA_TRY(h, cudaGetLastError());
    return PMH_OK;
}

extern "C" pmh_status pmh_merge(pmh_handle h, const double *q, const uint64_t *z, int64_t parts, uint32_t m,
                                double *out_q, uint64_t *out_z, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (parts < 0 || m < 1) return fail(h, PMH_ERR_INVALID_ARG, "parts < 0 or m < 1");
    if (!out_q || !out_z || (parts > 0 && (!q || !z))) return fail(h, PMH_ERR_INVALID_ARG, "NULL pointer");
    CUDA_TRY(h, cudaSetDevice(h->device));
    int grid = (int)std::min<uint32_t>((m + 255) / 256, 1024u);
    merge_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(q, z, parts, m, out_q, out_z);
    CUDA_TRY(h, cudaGetLastError());
    return PMH_OK;
}
