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

#include "batch_common.cuh"

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
    int32_t variants[PMH_MAX_VARIANTS];
    int32_t num_variants, precision, profiling;
    uint64_t seed;
    int32_t kinds[4];
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

// Autotuning key: the batch shape as the host sees it (the set sizes live on
// the device), per family.
struct TuneKey {
    uint32_t m;
    int32_t precision, family, items_log2;
    bool operator<(const TuneKey &o) const {
        return std::memcmp(this, &o, sizeof(*this)) < 0;
    }
};

}  // namespace

// Device workspace of one sketch call in flight: work queue, queue metadata,
// per-set statistics, grid-mode state.
struct Workspace {
    uint64_t *queue = nullptr;
    uint64_t *redo = nullptr;        // FP32 items redone in FP64, per family segment (capacity queue_cap)
    int64_t queue_cap = 0;
    unsigned int *qmeta = nullptr;   // histogram, running starts, per-family heads, big-set list
    SetStat *stats = nullptr;
    int64_t stats_cap = 0;
    void *grid = nullptr;
    size_t grid_bytes = 0;
    ulonglong2 *list = nullptr;      // prefilter lists (list_cap entries) and per-set entry counts
    int64_t list_cap = 0;
    uint32_t *list_n = nullptr;      // and, behind the counts, the sets the prefilter pass takes
    int64_t list_n_cap = 0;
};

// Buffers and streams of pmh_sketch_batch_host.
struct HostPipe {
    void *ids = nullptr, *w = nullptr, *off = nullptr;
    size_t ids_cap = 0, w_cap = 0, off_cap = 0;
    void *z[2] = {nullptr, nullptr}, *q[2] = {nullptr, nullptr}, *st[2] = {nullptr, nullptr};
    size_t z_cap[2] = {0, 0}, q_cap[2] = {0, 0}, st_cap[2] = {0, 0};
    cudaStream_t s[4] = {nullptr, nullptr, nullptr, nullptr};   // copy in, compute (two), copy out
    std::vector<cudaEvent_t> ev;
    cudaEvent_t span[2] = {nullptr, nullptr};   // device-side span of the last call (timing events)
    bool span_valid = false;
};

struct pmh_handle_s {
    int device = 0;
    int sm_count = 0;
    std::string err;
    std::map<uint32_t, TableBuf> tables;
    // per-stream workspaces: [0] for pmh_sketch_batch (and its graph), [1] for the
    // second compute stream of pmh_sketch_batch_host
    Workspace ws[2];
    cudaStream_t cap_stream = nullptr;
    bool graph_valid = false;
    GraphKey gkey{};
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    // planner knobs (tunable)
    Thresholds th;
    int last_launches = 0;
    int last_chunks = 0;
    HostPipe hp;
    FamilyFork ff[2];            // family kernels side by side, per workspace
#ifndef PMH_FAMILY_FORK
#define PMH_FAMILY_FORK 1
#endif
#ifndef PMH_PIPE_FORK
#define PMH_PIPE_FORK 1          // the host-buffer pipeline's ranges fork their family kernels too
#endif
    bool concurrent_families = PMH_FAMILY_FORK;
    int force_shape[4] = {-1, -1, -1, -1};   // per family: TeamShape, or -1
    int last_shape[4] = {-1, -1, -1, -1};    // shapes of the most recent call (-1: family absent)
    bool autotune = true;
    std::map<TuneKey, int> tuned;            // best TeamShape per key
    cudaEvent_t tev[3 + 4] = {};             // autotuning: queue/sketch brackets + one per family
    unsigned long long *status_scratch = nullptr;   // pmh_sync_status: 8 counts + the first failing (index, code)
    unsigned int *pm_counter = nullptr;              // pmh_pminhash_batch: the blocks' set counter
    // element counts of recent batches read back (they size the prefilter lists), keyed by their arrays
    struct NCount {
        const void *ids, *w, *off;
        int64_t sets, n;
    };
    std::vector<NCount> ncache;   // most recent last, at most 16
    // profiling events
    bool profiling = false;
    bool prof_recorded = false;        // the most recent call was profiled
    // profiled calls take the next slot of a ring of event triplets (no graph replay for them)
    static constexpr int kRing = 256;
    std::vector<cudaEvent_t> ring;     // kRing * 3 events, created by pmh_set_profiling
    int64_t prof_calls = 0;            // profiled calls so far (slot = (prof_calls - 1) % kRing)
};

void pmh::set_thread_error(const char *msg) { g_create_error = msg; }

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
// Per-m constant tables, built on the host and uploaded once per (handle, m).
static pmh_status get_tables(pmh_handle h, uint32_t m, Tables *out) {
    auto it = h->tables.find(m);
    if (it != h->tables.end()) { *out = it->second.t; return PMH_OK; }
    const size_t bytes = table_bytes(m);
    TableBuf tb;
    CUDA_TRY(h, cudaMalloc(&tb.dev, bytes));
    std::vector<unsigned char> host(bytes);
    build_tables(m, host.data(), tb.dev, &tb.t);
    cudaError_t e = cudaMemcpy(tb.dev, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(tb.dev); return fail(h, PMH_ERR_CUDA, "table upload: %s", cudaGetErrorString(e)); }
    h->tables[m] = tb;
    *out = tb.t;
    return PMH_OK;
}

static pmh_status ensure_queue(pmh_handle h, Workspace &w, int64_t items) {
    if (!w.qmeta) CUDA_TRY(h, cudaMalloc(&w.qmeta, kQMetaWords * sizeof(unsigned int)));
    if (items > w.queue_cap) {
        if (w.queue) cudaFree(w.queue);
        w.queue = nullptr;
        w.redo = nullptr;
        w.queue_cap = 0;
        int64_t cap = items < 1024 ? 1024 : items;
        // the work queue and, behind it, the FP64 redo list of the same capacity
        cudaError_t e = cudaMalloc(&w.queue, (size_t)cap * 2 * sizeof(uint64_t));
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "queue allocation (%lld items): %s", (long long)cap, cudaGetErrorString(e));
        w.redo = w.queue + cap;
        w.queue_cap = cap;
        h->graph_valid = false;
    }
    return PMH_OK;
}

static pmh_status ensure_grid(pmh_handle h, Workspace &w, uint32_t m) {
    const size_t need = grid_scratch_bytes(m);
    if (need > w.grid_bytes) {
        if (w.grid) cudaFree(w.grid);
        w.grid = nullptr;
        w.grid_bytes = 0;
        cudaError_t e = cudaMalloc(&w.grid, need);
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "grid workspace (%zu bytes): %s", need, cudaGetErrorString(e));
        w.grid_bytes = need;
        h->graph_valid = false;
    }
    return PMH_OK;
}

static pmh_status ensure_stats(pmh_handle h, Workspace &w, int64_t num_sets) {
    if (num_sets > w.stats_cap) {
        if (w.stats) cudaFree(w.stats);
        w.stats = nullptr;
        w.stats_cap = 0;
        int64_t cap = num_sets < 1024 ? 1024 : num_sets;
        cudaError_t e = cudaMalloc(&w.stats, (size_t)cap * sizeof(SetStat));
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "set statistics (%lld sets): %s", (long long)cap, cudaGetErrorString(e));
        w.stats_cap = cap;
        h->graph_valid = false;
    }
    return PMH_OK;
}

// Prefilter lists for a call of `elements` elements (offsets[num_sets] - offsets[0]) and num_sets sets.
static pmh_status ensure_list(pmh_handle h, Workspace &w, int64_t elements, int64_t num_sets) {
    const int64_t need = elements / 2 + 1;
    if (need > w.list_cap) {
        if (w.list) cudaFree(w.list);
        w.list = nullptr;
        w.list_cap = 0;
        cudaError_t e = cudaMalloc(&w.list, (size_t)need * sizeof(ulonglong2));
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "prefilter lists (%lld entries): %s", (long long)need, cudaGetErrorString(e));
        w.list_cap = need;
        h->graph_valid = false;
    }
    if (num_sets > w.list_n_cap) {
        if (w.list_n) cudaFree(w.list_n);
        w.list_n = nullptr;
        w.list_n_cap = 0;
        const int64_t cap = num_sets < 1024 ? 1024 : num_sets;
        cudaError_t e = cudaMalloc(&w.list_n, (size_t)cap * 2 * sizeof(uint32_t));
        if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "prefilter list counts (%lld sets): %s", (long long)cap, cudaGetErrorString(e));
        w.list_n_cap = cap;
        h->graph_valid = false;
    }
    return PMH_OK;
}

// Sets of list_min..list_max elements get prefilter lists (list_min from the first round's threshold),
// when some variant of the call reads them: a weighted one whose first point the filter bounds
// without the rejection sampler.
static bool list_bounds(const Thresholds &th, uint32_t m, float t_factor, const int32_t *variants, int32_t nv,
                        int64_t *lo, int64_t *hi) {
    if (!kListing || !(th.list_factor > 0.0) || th.rounds <= 0) return false;
    bool used = false;
    for (int v = 0; v < nv; v++)
        used |= !variant_unweighted(variants[v]) && !(th.te_rej && family_of(variants[v]) >= 3);
    if (!used) return false;
    const double lmin = std::ceil(th.list_factor * (double)m * (double)t_factor);
    *lo = lmin < 2.0 ? 2 : (lmin > 9e18 ? INT64_MAX : (int64_t)lmin);
    *hi = th.list_max;
    return *lo <= *hi;
}

// The element count offsets[num_sets] - offsets[0] of a device batch: read back (waiting for `st`)
// the first time a batch (ids, weights, offsets, num_sets) is seen, then taken from the handle.
// -1 when it cannot be read (during a stream capture).  A stale count costs speed only: the
// prefilter kernel lists only the sets that fit in the lists.
static pmh_status element_count(pmh_handle h, const void *ids, const void *weights, const int64_t *offsets,
                                int64_t num_sets, cudaStream_t st, cudaStreamCaptureStatus cs, int64_t *n) {
    *n = -1;
    for (size_t i = 0; i < h->ncache.size(); i++) {
        const pmh_handle_s::NCount c = h->ncache[i];
        if (c.off == offsets && c.ids == ids && c.w == weights && c.sets == num_sets) {
            h->ncache.erase(h->ncache.begin() + (std::ptrdiff_t)i);   // most recent last
            h->ncache.push_back(c);
            *n = c.n;
            return PMH_OK;
        }
    }
    if (cs != cudaStreamCaptureStatusNone) return PMH_OK;
    int64_t v[2] = {0, 0};
    CUDA_TRY(h, cudaMemcpyAsync(&v[0], offsets, sizeof(int64_t), cudaMemcpyDefault, st));
    CUDA_TRY(h, cudaMemcpyAsync(&v[1], offsets + num_sets, sizeof(int64_t), cudaMemcpyDefault, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    if (h->ncache.size() >= 16) h->ncache.erase(h->ncache.begin());
    h->ncache.push_back({ids, weights, offsets, num_sets, v[1] > v[0] ? v[1] - v[0] : 0});
    *n = h->ncache.back().n;
    return PMH_OK;
}

static pmh_status ensure_workspace(pmh_handle h, Workspace &w, int64_t num_sets, int64_t items, uint32_t m) {
    pmh_status rc = ensure_queue(h, w, items);
    if (!rc) rc = ensure_stats(h, w, num_sets);
    if (!rc) rc = ensure_grid(h, w, m);
    return rc;
}

// Streams and events of workspace wsi's family fork, created on first use.
static pmh_status ensure_fork(pmh_handle h, int wsi) {
    FamilyFork &ff = h->ff[wsi];
    if (ff.fork) return PMH_OK;
    for (int i = 0; i < 4; i++) {
        CUDA_TRY(h, cudaStreamCreateWithFlags(&ff.s[i], cudaStreamNonBlocking));
        CUDA_TRY(h, cudaEventCreateWithFlags(&ff.join[i], cudaEventDisableTiming));
    }
    CUDA_TRY(h, cudaEventCreateWithFlags(&ff.fork, cudaEventDisableTiming));
    return PMH_OK;
}

// Enqueues the whole batch on `st` with workspace wsi; with `fork`, the family
// kernels run side by side on that workspace's fork streams.
static pmh_status enqueue_sketch(pmh_handle h, int wsi, const SketchParams &p, const Plan &plan, int precision,
                                 cudaStream_t st, cudaEvent_t *prof_ev, cudaEvent_t *fam_ev, bool fork,
                                 const ListSpec &ls) {
    if (fork) {
        pmh_status rc = ensure_fork(h, wsi);
        if (rc) return rc;
    }
    Workspace &w = h->ws[wsi];
    cudaError_t e = enqueue_batch(p, plan, precision, h->sm_count, w.queue, w.redo, w.qmeta, w.stats, st, prof_ev, fam_ev,
                                  fork ? &h->ff[wsi] : nullptr, ls);
    if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "sketch launch: %s", cudaGetErrorString(e));
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
    for (cudaEvent_t e : h->ring) cudaEventDestroy(e);
    for (int i = 0; i < 7; i++) if (h->tev[i]) cudaEventDestroy(h->tev[i]);
    for (auto &kv : h->tables) cudaFree(kv.second.dev);
    if (h->status_scratch) cudaFree(h->status_scratch);
    if (h->pm_counter) cudaFree(h->pm_counter);
    for (Workspace &w : h->ws) {
        if (w.queue) cudaFree(w.queue);
        if (w.qmeta) cudaFree(w.qmeta);
        if (w.stats) cudaFree(w.stats);
        if (w.grid) cudaFree(w.grid);
    }
    for (Workspace &w : h->ws) {
        if (w.list) cudaFree(w.list);
        if (w.list_n) cudaFree(w.list_n);
    }
    for (void *ptr : {h->hp.ids, h->hp.w, h->hp.off, h->hp.z[0], h->hp.z[1], h->hp.q[0], h->hp.q[1], h->hp.st[0], h->hp.st[1]})
        if (ptr) cudaFree(ptr);
    for (int i = 0; i < 4; i++) if (h->hp.s[i]) cudaStreamDestroy(h->hp.s[i]);
    for (cudaEvent_t e : h->hp.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->hp.span) if (e) cudaEventDestroy(e);
    for (FamilyFork &ff : h->ff) {
        for (int i = 0; i < 4; i++) {
            if (ff.s[i]) cudaStreamDestroy(ff.s[i]);
            if (ff.join[i]) cudaEventDestroy(ff.join[i]);
        }
        if (ff.fork) cudaEventDestroy(ff.fork);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

extern "C" const char *pmh_last_error(pmh_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

extern "C" pmh_status pmh_set_profiling(pmh_handle h, int32_t enable) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    CUDA_TRY(h, cudaSetDevice(h->device));
    while (enable && (int)h->ring.size() < 3 * pmh_handle_s::kRing) {
        cudaEvent_t e;
        CUDA_TRY(h, cudaEventCreate(&e));
        h->ring.push_back(e);
    }
    h->profiling = enable != 0;
    return PMH_OK;
}

extern "C" pmh_status pmh_set_thresholds(pmh_handle h, double t_c, double t_c_grid, int32_t rounds, int64_t grid_min) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (!std::isfinite(t_c) || !std::isfinite(t_c_grid)) return fail(h, PMH_ERR_INVALID_ARG, "t_c and t_c_grid must be finite");
    if (rounds < 0 || rounds > 64) return fail(h, PMH_ERR_INVALID_ARG, "rounds = %d outside [0, 64]", rounds);
    h->th.t_c = t_c;
    h->th.t_c_grid = t_c_grid;
    h->th.rounds = rounds;
    h->th.grid_min = grid_min;
    h->graph_valid = false;
    return PMH_OK;
}

extern "C" pmh_status pmh_set_prefilter(pmh_handle h, double list_factor) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (!std::isfinite(list_factor)) return fail(h, PMH_ERR_INVALID_ARG, "list_factor must be finite");
    h->th.list_factor = list_factor;
    h->graph_valid = false;
    return PMH_OK;
}

extern "C" pmh_status pmh_set_limits(pmh_handle h, uint32_t cap_points, int32_t max_contenders) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (max_contenders < -1 || max_contenders > kGridCont)
        return fail(h, PMH_ERR_INVALID_ARG, "max_contenders = %d outside [-1, %d]", max_contenders, kGridCont);
    h->th.cap_points = cap_points;
    h->th.max_cont = max_contenders;
    h->graph_valid = false;
    return PMH_OK;
}

extern "C" pmh_status pmh_set_te_sampler(pmh_handle h, int32_t sampler) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (sampler != PMH_TE_INVERSION && sampler != PMH_TE_REJECTION)
        return fail(h, PMH_ERR_INVALID_ARG, "sampler %d is neither PMH_TE_INVERSION nor PMH_TE_REJECTION", sampler);
    h->th.te_rej = sampler == PMH_TE_REJECTION;
    h->graph_valid = false;
    return PMH_OK;
}

extern "C" pmh_status pmh_set_team_shape(pmh_handle h, int32_t family, int32_t shape) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (family < 0 || family > 4) return fail(h, PMH_ERR_INVALID_ARG, "family %d outside [0, 4]", family);
    if (shape < -1 || shape >= kNumShapes) return fail(h, PMH_ERR_INVALID_ARG, "shape %d outside [-1, %d]", shape, kNumShapes - 1);
    for (int f = 1; f <= 4; f++)
        if (family == 0 || family == f) h->force_shape[f - 1] = shape;
    h->graph_valid = false;
    return PMH_OK;
}

extern "C" pmh_status pmh_set_autotune(pmh_handle h, int32_t enable) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    h->autotune = enable != 0;
    if (enable < 0) h->tuned.clear();
    h->graph_valid = false;
    return PMH_OK;
}

extern "C" pmh_status pmh_last_team_shapes(pmh_handle h, int32_t *shapes) {
    if (!h || !shapes) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    for (int f = 0; f < 4; f++) shapes[f] = h->last_shape[f];
    return PMH_OK;
}

extern "C" pmh_status pmh_last_launches(pmh_handle h, int32_t *launches) {
    if (!h || !launches) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    *launches = h->last_launches;
    return PMH_OK;
}

extern "C" pmh_status pmh_last_kernel_ms(pmh_handle h, float *queue_ms, float *sketch_ms) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (!h->prof_recorded || h->prof_calls == 0) return fail(h, PMH_ERR_INVALID_ARG, "profiling was off for the last call");
    int32_t n = 0;
    return pmh_kernel_ms_history(h, 1, queue_ms, sketch_ms, &n);
}

extern "C" pmh_status pmh_kernel_ms_history(pmh_handle h, int32_t max_calls, float *queue_ms, float *sketch_ms,
                                            int32_t *count) {
    if (!h || !count || max_calls < 0) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    const int64_t n = std::min<int64_t>({(int64_t)max_calls, h->prof_calls, (int64_t)pmh_handle_s::kRing});
    *count = 0;
    if (n == 0) return PMH_OK;
    const int64_t last = (h->prof_calls - 1) % pmh_handle_s::kRing;
    CUDA_TRY(h, cudaEventSynchronize(h->ring[3 * last + 2]));
    for (int64_t j = 0; j < n; j++) {
        const int64_t slot = (h->prof_calls - n + j) % pmh_handle_s::kRing;
        float a = 0.0f, b = 0.0f;
        CUDA_TRY(h, cudaEventElapsedTime(&a, h->ring[3 * slot], h->ring[3 * slot + 1]));
        CUDA_TRY(h, cudaEventElapsedTime(&b, h->ring[3 * slot + 1], h->ring[3 * slot + 2]));
        if (queue_ms) queue_ms[j] = a;
        if (sketch_ms) sketch_ms[j] = b;
    }
    *count = (int32_t)n;
    return PMH_OK;
}

// Times every team shape on this batch (one full run each, on `st`, blocking)
// and records the fastest per family.  All runs write the same results.
static pmh_status autotune_shapes(pmh_handle h, Workspace &w, SketchParams p, uint32_t m, const int32_t *variants,
                                  int32_t num_variants, int64_t num_sets, int precision, cudaStream_t st,
                                  int *kinds, const TuneKey *tkey, const ListSpec &ls) {
    if (!h->tev[0])
        for (int i = 0; i < 7; i++) CUDA_TRY(h, cudaEventCreate(&h->tev[i]));
    float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    int best_kind[4] = {-1, -1, -1, -1};
    // two passes over the shapes, keeping each one's faster trial: a first launch of a kernel
    // (module loading, cold caches) would otherwise decide between shapes within a few percent
    for (int trial = 0; trial < 2 * kNumShapes; trial++) {
        const int cand = trial % kNumShapes;
        int ck[4];
        for (int f = 0; f < 4; f++) ck[f] = kinds[f] >= 0 ? kinds[f] : cand;
        Plan plan;
        bool fits = true;
        cudaError_t e = plan_batch(h->sm_count, precision, m, variants, num_variants, num_sets, ck, &plan, &fits);
        if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
        if (!fits) continue;
        SketchParams q = p;
        q.counters = nullptr;   // the trials are not the call's work
        for (int j = 0; j < plan.nfam && q.gctl; j++)
            if (plan.ggrid[j] <= 0) { q.gctl = nullptr; q.gstate = nullptr; q.gsig = nullptr; }
        e = enqueue_batch(q, plan, precision, h->sm_count, w.queue, w.redo, w.qmeta, w.stats, st, h->tev, h->tev + 3,
                          nullptr, ls);
        if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
        CUDA_TRY(h, cudaEventSynchronize(h->tev[2]));
        for (int j = 0; j < plan.nfam; j++) {
            const int f = plan.fam[j] - 1;
            if (kinds[f] >= 0 || plan.shape[j].kind != cand) continue;   // forced, or the candidate did not fit
            float ms = 0.0f;
            CUDA_TRY(h, cudaEventElapsedTime(&ms, j == 0 ? h->tev[1] : h->tev[3 + j - 1], h->tev[3 + j]));
            if (ms < best[f]) { best[f] = ms; best_kind[f] = cand; }
        }
    }
    for (int f = 0; f < 4; f++)
        if (kinds[f] < 0 && best_kind[f] >= 0) {
            kinds[f] = best_kind[f];
            h->tuned[tkey[f]] = best_kind[f];
        }
    h->graph_valid = false;
    return PMH_OK;
}

// Argument checks shared by the device and the host-buffer entry points.
static pmh_status check_sketch_args(pmh_handle h, int64_t num_sets, uint32_t m, const int32_t *variants,
                                    int32_t num_variants, int32_t precision) {
    if (num_sets < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_sets < 0");
    if (num_sets >= (1ll << 40)) return fail(h, PMH_ERR_UNSUPPORTED, "num_sets >= 2^40");
    if (num_variants >= 1 && num_variants <= PMH_MAX_VARIANTS && num_sets * num_variants > 0x7FFFFFFFll - (1ll << 24))
        return fail(h, PMH_ERR_UNSUPPORTED, "num_sets * num_variants too large for one call");
    if (m < 1 || m > PMH_MAX_M) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, %u]", m, PMH_MAX_M);
    if (!variants || num_variants < 1 || num_variants > PMH_MAX_VARIANTS)
        return fail(h, PMH_ERR_INVALID_ARG, "need 1..%d variants", PMH_MAX_VARIANTS);
    if (precision != PMH_FP64 && precision != PMH_FP32_RECHECK) return fail(h, PMH_ERR_INVALID_ARG, "bad precision %d", precision);
    bool has_perm = false;
    for (int v = 0; v < num_variants; v++) {
        if (variants[v] < PMH_V1 || variants[v] > PMH_V4U) return fail(h, PMH_ERR_INVALID_ARG, "bad variant %d", variants[v]);
        if ((variants[v] == PMH_V3 || variants[v] == PMH_V3A || variants[v] == PMH_V4) && m < 2)
            return fail(h, PMH_ERR_INVALID_ARG, "variant %d requires m >= 2", variants[v]);
        has_perm |= (variants[v] == PMH_V2 || variants[v] == PMH_V4);
    }
    (void)has_perm;
    return PMH_OK;
}

// The sketch of a CSR batch already in device memory, enqueued on `st`
// (replayed from a cached CUDA graph when allow_graph and the arguments repeat).
static TuneKey tune_key(uint32_t m, int32_t precision, int family, int64_t items) {
    return TuneKey{m, precision, family, items > 0 ? 63 - __builtin_clzll((unsigned long long)items) : -1};
}

static pmh_status sketch_device(pmh_handle h, int wsi, const uint64_t *ids, const double *weights,
                                const int64_t *offsets, int64_t num_sets, uint32_t m, const int32_t *variants,
                                int32_t num_variants, int32_t precision, uint64_t seed, uint64_t *out_ids,
                                double *out_q, int32_t *set_status, uint64_t *counters, cudaStream_t st,
                                bool allow_graph, cudaEvent_t *fam_ev, const int *kinds_in = nullptr,
                                int64_t n_hint = -1) {
    CUDA_TRY(h, cudaSetDevice(h->device));
    Workspace &w = h->ws[wsi];
    Tables tab;
    pmh_status rc = get_tables(h, m, &tab);
    if (rc) return rc;
    rc = ensure_workspace(h, w, num_sets, num_sets * num_variants, m);
    if (rc) return rc;

    SketchParams p;
    fill_params(&p, ids, weights, offsets, num_sets, m, variants, num_variants, seed, out_ids, out_q, set_status, counters,
                h->th);
    p.tab = tab;
    if (h->th.grid_min > 0) bind_grid_scratch(&p, w.grid);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st) CUDA_TRY(h, cudaStreamIsCapturing(st, &cs));
    // prefilter lists, sized by the call's element count
    ListSpec ls;
    if (list_bounds(h->th, m, p.t_factor, variants, num_variants, &ls.list_min, &ls.list_max)) {
        int64_t n_el = n_hint;
        if (n_el < 0 && (rc = element_count(h, ids, weights, offsets, num_sets, st, cs, &n_el))) return rc;
        if (n_el > 0) {
            rc = ensure_list(h, w, n_el, num_sets);
            if (rc == PMH_ERR_NO_MEMORY) {
                // the lists only save work: without room for them every element is filtered in full
                (void)cudaGetLastError();
                h->err.clear();
                rc = PMH_OK;
            } else if (rc) {
                return rc;
            } else {
                ls.list = w.list;
                ls.list_n = w.list_n;
                ls.sel = w.list_n + w.list_n_cap;
                ls.list_cap = w.list_cap;
            }
        }
    }
    // team shape per family: given by the caller (host pipeline), else forced, else tuned, else
    // (tuning off or impossible) the default rule
    int kinds[4];
    TuneKey tkey[4];
    bool need_tune = false;
    if (kinds_in) {
        for (int f = 0; f < 4; f++) kinds[f] = kinds_in[f];
    } else {
        int64_t per_fam[4] = {0, 0, 0, 0};
        for (int v = 0; v < num_variants; v++) per_fam[family_of(variants[v]) - 1] += num_sets;
        for (int f = 0; f < 4; f++) {
            tkey[f] = tune_key(m, precision, f + 1, per_fam[f]);
            kinds[f] = h->force_shape[f];
            if (kinds[f] < 0 && per_fam[f] > 0) {
                auto it = h->tuned.find(tkey[f]);
                if (it != h->tuned.end()) kinds[f] = it->second;
                else need_tune = true;
            }
        }
    }
    if (need_tune && h->autotune && cs == cudaStreamCaptureStatusNone) {
        rc = autotune_shapes(h, w, p, m, variants, num_variants, num_sets, precision, st, kinds, tkey, ls);
        if (rc) return rc;
    }
    Plan plan;
    bool fits = true;
    cudaError_t pe = plan_batch(h->sm_count, precision, m, variants, num_variants, num_sets, kinds, &plan, &fits);
    if (pe != cudaSuccess) return fail(h, PMH_ERR_CUDA, "occupancy: %s", cudaGetErrorString(pe));
    if (!fits) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u does not fit in shared memory", m);
    // grid mode only when every family's grid kernel can be resident (items it
    // takes are skipped by the ordinary kernels)
    for (int j = 0; j < plan.nfam && p.gctl; j++)
        if (plan.ggrid[j] <= 0) { p.gctl = nullptr; p.gstate = nullptr; p.gsig = nullptr; }
    h->last_launches = launch_count(plan, p.gctl != nullptr, precision == PMH_FP32_RECHECK, ls.list != nullptr);
    for (int f = 0; f < 4; f++) h->last_shape[f] = -1;
    for (int j = 0; j < plan.nfam; j++) h->last_shape[plan.fam[j] - 1] = plan.shape[j].kind;
    cudaEvent_t *prof_ev = nullptr;
    if (h->profiling && cs == cudaStreamCaptureStatusNone && (int)h->ring.size() == 3 * pmh_handle_s::kRing) {
        prof_ev = h->ring.data() + 3 * (h->prof_calls % pmh_handle_s::kRing);
        h->prof_calls++;
    }
    h->prof_recorded = prof_ev != nullptr;
    // the family kernels side by side; the host-buffer pipeline's ranges (fam_ev: their outputs go
    // back family by family) fork on their own workspace's streams
    const bool fork = h->concurrent_families && (!fam_ev || PMH_PIPE_FORK);
    if (fork && (rc = ensure_fork(h, wsi))) return rc;   // before any capture begins
    if (!allow_graph || wsi != 0 || fam_ev || prof_ev || !h->use_graph || cs != cudaStreamCaptureStatusNone || !st)
        return enqueue_sketch(h, wsi, p, plan, precision, st, prof_ev, fam_ev, fork, ls);

    GraphKey key{};
    key.ids = ids; key.weights = weights; key.offsets = offsets; key.out_ids = out_ids; key.out_q = out_q;
    key.status = set_status; key.counters = counters; key.num_sets = num_sets; key.m = m;
    for (int v = 0; v < num_variants; v++) key.variants[v] = variants[v];
    key.num_variants = num_variants; key.precision = precision; key.seed = seed;
    key.profiling = 0;
    for (int f = 0; f < 4; f++) key.kinds[f] = kinds[f];
    if (!(h->graph_valid && h->gkey == key)) {
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
        h->graph_valid = false;
        CUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_sketch(h, wsi, p, plan, precision, h->cap_stream, nullptr, nullptr, fork, ls);
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

extern "C" pmh_status pmh_sketch_batch(pmh_handle h, const uint64_t *ids, const double *weights, const int64_t *offsets,
                                       int64_t num_sets, uint32_t m, const int32_t *variants, int32_t num_variants,
                                       int32_t precision, uint64_t seed, uint64_t *out_ids, double *out_q,
                                       int32_t *set_status, uint64_t *counters, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    pmh_status rc = check_sketch_args(h, num_sets, m, variants, num_variants, precision);
    if (rc) return rc;
    if (num_sets == 0) return PMH_OK;
    if (!ids || !weights || !offsets || !out_ids) return fail(h, PMH_ERR_INVALID_ARG, "NULL ids/weights/offsets/out_ids");
    return sketch_device(h, 0, ids, weights, offsets, num_sets, m, variants, num_variants, precision, seed, out_ids,
                         out_q, set_status, counters, (cudaStream_t)stream, true, nullptr);
}

// ------------------------------------------------------------------ host buffers
// Device mirror of a host batch plus double-buffered chunk outputs, and the
// three streams of the copy / compute / copy-back pipeline.
static pmh_status ensure_dev(pmh_handle h, void **ptr, size_t *cap, size_t need, const char *what) {
    if (need <= *cap) return PMH_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(ptr, need);
    if (e != cudaSuccess) return fail(h, PMH_ERR_NO_MEMORY, "%s (%zu bytes): %s", what, need, cudaGetErrorString(e));
    *cap = need;
    return PMH_OK;
}

// Contiguous set ranges by work (n + m H_m ln(n+1) per set, the element
// hashing plus the early-stop points of Sec. ProbMinHash1): the first range
// gets half the share of the others, so that the first kernels start after a
// shorter copy.
static void chunk_bounds(const int64_t *off, int64_t num_sets, uint32_t m, int k, std::vector<int64_t> *b) {
    double hm = 0.0;
    for (uint32_t i = 1; i <= m; i++) hm += 1.0 / i;
    std::vector<double> cum((size_t)num_sets + 1, 0.0);
    for (int64_t s = 0; s < num_sets; s++) {
        const double n = (double)(off[s + 1] - off[s]);
        cum[s + 1] = cum[s] + n + m * hm * std::log1p(n);
    }
    b->assign(1, 0);
    int64_t s = 0;
    const double shares = 2.0 * k - 1.0;   // weights 1, 2, 2, ..., 2
    for (int c = 1; c < k; c++) {
        const double t = cum[num_sets] * (2.0 * c - 1.0) / shares;
        while (s < num_sets && cum[s + 1] < t) s++;
        if (s > b->back()) b->push_back(s);
    }
    if (b->back() != num_sets) b->push_back(num_sets);
}

extern "C" pmh_status pmh_sketch_batch_host(pmh_handle h, const uint64_t *ids, const double *weights,
                                            const int64_t *offsets, int64_t num_sets, uint32_t m,
                                            const int32_t *variants, int32_t num_variants, int32_t precision,
                                            uint64_t seed, uint64_t *out_ids, double *out_q, int32_t *set_status,
                                            int32_t chunks) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    pmh_status rc = check_sketch_args(h, num_sets, m, variants, num_variants, precision);
    if (rc) return rc;
    if (num_sets == 0) return PMH_OK;
    if (!ids || !weights || !offsets || !out_ids) return fail(h, PMH_ERR_INVALID_ARG, "NULL ids/weights/offsets/out_ids");
    if (offsets[0] < 0) return fail(h, PMH_ERR_INVALID_ARG, "offsets[0] < 0");
    for (int64_t s = 0; s < num_sets; s++)
        if (offsets[s + 1] < offsets[s]) return fail(h, PMH_ERR_INVALID_ARG, "offsets decrease at set %lld", (long long)s);
    CUDA_TRY(h, cudaSetDevice(h->device));
    const int64_t N = offsets[num_sets];
    // 4: measured best on c2 with the prefilter (median step 3: 27.2 ms, 4: 26.2 ms, 6: 28.3 ms)
    int k = chunks > 0 ? chunks : (N >= (1ll << 22) ? 4 : 1);
    std::vector<int64_t> b;
    chunk_bounds(offsets, num_sets, m, k, &b);
    k = (int)b.size() - 1;
    int64_t smax = 0;
    for (int c = 0; c < k; c++) smax = std::max<int64_t>(smax, b[c + 1] - b[c]);
    const int64_t V = num_variants;
    // families present, in the order the sketch runs them (ascending)
    int fam_rank[5] = {-1, -1, -1, -1, -1};
    {
        bool present[5] = {false, false, false, false, false};
        for (int v = 0; v < num_variants; v++) present[family_of(variants[v])] = true;
        int r = 0;
        for (int f = 1; f <= 4; f++) if (present[f]) fam_rank[f] = r++;
    }
    // workspace for every chunk first: no allocation while the pipeline runs
    Tables tab;
    if ((rc = get_tables(h, m, &tab))) return rc;
    int64_t lmin = 0, lmax = 0, nmax = 0;
    for (int c = 0; c < k; c++) nmax = std::max<int64_t>(nmax, offsets[b[c + 1]] - offsets[b[c]]);
    bool lists = list_bounds(h->th, m, (float)(std::log((double)m) + h->th.t_c), variants, num_variants, &lmin, &lmax) &&
                 nmax > 0;
    for (Workspace &w : h->ws) {
        if ((rc = ensure_workspace(h, w, smax, smax * V, m))) return rc;
        if (lists && (rc = ensure_list(h, w, nmax, smax))) {
            if (rc != PMH_ERR_NO_MEMORY) return rc;
            (void)cudaGetLastError();   // no room for the lists: the ranges filter every element in full
            h->err.clear();
            rc = PMH_OK;
            lists = false;
        }
    }
    HostPipe &hp = h->hp;
    if ((rc = ensure_dev(h, &hp.ids, &hp.ids_cap, (size_t)N * 8, "device ids"))) return rc;
    if ((rc = ensure_dev(h, &hp.w, &hp.w_cap, (size_t)N * 8, "device weights"))) return rc;
    if ((rc = ensure_dev(h, &hp.off, &hp.off_cap, (size_t)(num_sets + 1) * 8, "device offsets"))) return rc;
    for (int i = 0; i < 2; i++) {
        if ((rc = ensure_dev(h, &hp.z[i], &hp.z_cap[i], (size_t)(V * smax * m) * 8, "chunk ids"))) return rc;
        if (out_q && (rc = ensure_dev(h, &hp.q[i], &hp.q_cap[i], (size_t)(V * smax * m) * 8, "chunk q"))) return rc;
        if (set_status && (rc = ensure_dev(h, &hp.st[i], &hp.st_cap[i], (size_t)(V * smax) * 4, "chunk status"))) return rc;
    }
    if (!hp.s[0])
        for (int i = 0; i < 4; i++) CUDA_TRY(h, cudaStreamCreateWithFlags(&hp.s[i], cudaStreamNonBlocking));
    constexpr int kEvPerChunk = 6;   // inputs in, four families done, outputs out
    while ((int)hp.ev.size() < kEvPerChunk * k) {
        cudaEvent_t e;
        CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        hp.ev.push_back(e);
    }
    cudaStream_t s_in = hp.s[0], s_out = hp.s[3];
    unsigned char *dids = (unsigned char *)hp.ids, *dw = (unsigned char *)hp.w;
    int64_t *doff = (int64_t *)hp.off;
    auto ev_in = [&](int c) { return hp.ev[kEvPerChunk * c]; };
    auto ev_fam = [&](int c) { return hp.ev.data() + kEvPerChunk * c + 1; };
    auto ev_out = [&](int c) { return hp.ev[kEvPerChunk * c + 5]; };
    if (!hp.span[0])
        for (int i = 0; i < 2; i++) CUDA_TRY(h, cudaEventCreate(&hp.span[i]));
    hp.span_valid = false;
    CUDA_TRY(h, cudaEventRecord(hp.span[0], s_in));
    // inputs: offsets, then each chunk's elements in place
    CUDA_TRY(h, cudaMemcpyAsync(doff, offsets, (size_t)(num_sets + 1) * 8, cudaMemcpyHostToDevice, s_in));
    for (int c = 0; c < k; c++) {
        const int64_t e0 = c == 0 ? 0 : offsets[b[c]], e1 = offsets[b[c + 1]];
        if (e1 > e0) {
            CUDA_TRY(h, cudaMemcpyAsync(dids + e0 * 8, ids + e0, (size_t)(e1 - e0) * 8, cudaMemcpyHostToDevice, s_in));
            CUDA_TRY(h, cudaMemcpyAsync(dw + e0 * 8, weights + e0, (size_t)(e1 - e0) * 8, cudaMemcpyHostToDevice, s_in));
        }
        CUDA_TRY(h, cudaEventRecord(ev_in(c), s_in));
    }
    // team shapes: the ones tuned for the whole batch's size (or forced), else the default rule; the
    // ranges are not tuned on their own (their timings would overlap each other)
    int kinds[4];
    {
        int64_t per_fam[4] = {0, 0, 0, 0};
        for (int v = 0; v < num_variants; v++) per_fam[family_of(variants[v]) - 1] += num_sets;
        for (int f = 0; f < 4; f++) {
            kinds[f] = h->force_shape[f];
            if (kinds[f] < 0 && per_fam[f] > 0) {
                auto it = h->tuned.find(tune_key(m, precision, f + 1, per_fam[f]));
                if (it != h->tuned.end()) kinds[f] = it->second;
            }
        }
    }
    // chunks alternate between two compute streams (each with its own workspace), so that one
    // chunk's kernels fill the SMs the other's tail leaves idle; each family's rows go back as
    // soon as that family's kernel is done
    for (int c = 0; c < k; c++) {
        const int64_t s0 = b[c], sc = b[c + 1] - b[c];
        const int r = c & 1;
        cudaStream_t s_run = hp.s[1 + r];
        CUDA_TRY(h, cudaStreamWaitEvent(s_run, ev_in(c), 0));
        if (c >= 2) CUDA_TRY(h, cudaStreamWaitEvent(s_run, ev_out(c - 2), 0));   // chunk outputs are double-buffered
        rc = sketch_device(h, r, (const uint64_t *)dids, (const double *)dw, doff + s0, sc, m, variants, num_variants,
                           precision, seed, (uint64_t *)hp.z[r], out_q ? (double *)hp.q[r] : nullptr,
                           set_status ? (int32_t *)hp.st[r] : nullptr, nullptr, s_run, false, ev_fam(c), kinds,
                           lists ? offsets[b[c + 1]] - offsets[b[c]] : 0);
        if (rc) {
            for (int i = 0; i < 4; i++) cudaStreamSynchronize(hp.s[i]);
            return rc;
        }
        for (int f = 1; f <= 4; f++) {
            if (fam_rank[f] < 0) continue;
            CUDA_TRY(h, cudaStreamWaitEvent(s_out, ev_fam(c)[fam_rank[f]], 0));
            for (int64_t v = 0; v < V; v++) {
                if (family_of(variants[v]) != f) continue;
                CUDA_TRY(h, cudaMemcpyAsync(out_ids + (v * num_sets + s0) * m, (const uint64_t *)hp.z[r] + v * sc * m,
                                            (size_t)(sc * m) * 8, cudaMemcpyDeviceToHost, s_out));
                if (out_q)
                    CUDA_TRY(h, cudaMemcpyAsync(out_q + (v * num_sets + s0) * m, (const double *)hp.q[r] + v * sc * m,
                                                (size_t)(sc * m) * 8, cudaMemcpyDeviceToHost, s_out));
                if (set_status)
                    CUDA_TRY(h, cudaMemcpyAsync(set_status + v * num_sets + s0, (const int32_t *)hp.st[r] + v * sc,
                                                (size_t)sc * 4, cudaMemcpyDeviceToHost, s_out));
            }
        }
        CUDA_TRY(h, cudaEventRecord(ev_out(c), s_out));
    }
    for (int i = 1; i < 3; i++) {   // the copy-out stream ends after both compute streams
        CUDA_TRY(h, cudaEventRecord(hp.ev[kEvPerChunk * (k - 1) + 5], hp.s[i]));
        CUDA_TRY(h, cudaStreamWaitEvent(s_out, hp.ev[kEvPerChunk * (k - 1) + 5], 0));
    }
    CUDA_TRY(h, cudaEventRecord(hp.span[1], s_out));
    for (int i = 0; i < 4; i++) CUDA_TRY(h, cudaStreamSynchronize(hp.s[i]));
    hp.span_valid = true;
    h->last_chunks = k;
    return PMH_OK;
}

extern "C" pmh_status pmh_last_host_span_ms(pmh_handle h, float *ms, int32_t *chunks) {
    if (!h || !ms) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (!h->hp.span_valid) return fail(h, PMH_ERR_INVALID_ARG, "no completed pmh_sketch_batch_host call");
    CUDA_TRY(h, cudaEventElapsedTime(ms, h->hp.span[0], h->hp.span[1]));
    if (chunks) *chunks = h->last_chunks;
    return PMH_OK;
}

// ------------------------------------------------------------------ verification
static __global__ void check_exp1_kernel(const uint64_t *__restrict__ w, int64_t n, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = exp1_32(w[i]);
}

static __global__ void check_texp_kernel(const uint64_t *__restrict__ w, int64_t n, float c, float inv,
                                         float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = texp_32(w[i], c, inv);
}

extern "C" pmh_status pmh_check_texp(const uint64_t *words, int64_t n, float c, float inv, float *out, void *stream) {
    if (n < 0 || (n > 0 && (!words || !out))) return PMH_ERR_INVALID_ARG;
    if (n == 0) return PMH_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    check_texp_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(words, n, c, inv, out);
    return cudaGetLastError() == cudaSuccess ? PMH_OK : PMH_ERR_CUDA;
}

extern "C" pmh_status pmh_check_exp1(const uint64_t *words, int64_t n, float *out, void *stream) {
    if (n < 0 || (n > 0 && (!words || !out))) return PMH_ERR_INVALID_ARG;
    if (n == 0) return PMH_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    check_exp1_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(words, n, out);
    return cudaGetLastError() == cudaSuccess ? PMH_OK : PMH_ERR_CUDA;
}

// ------------------------------------------------------------------ estimation
// Equal-component counts of every pair (a, b) of rows of two signature tables,
// Eq. jaccard_estimator: out[a * ldo + b].  128x128 tile of pairs per CTA, 16
// components per shared-memory stage, 8x8 pairs per thread (rows ty + 16i,
// columns tx + 16j: conflict-free shared reads, 16 shared loads per 64 pairs).
// With upper_only (one table against itself) only b >= a is written.
constexpr int kTile = 64, kKc = 16;   // the b-bit kernel's tile
constexpr int kApTile = 128, kApR = kApTile / 16;

__global__ void __launch_bounds__(256, 2) allpairs_kernel(const uint64_t *__restrict__ sa, int64_t na,
                                                          const uint64_t *__restrict__ sb, int64_t nb, uint32_t m,
                                                          int upper_only, uint16_t *__restrict__ out, int64_t ldo) {
    __shared__ uint64_t As[kKc][kApTile + 1];
    __shared__ uint64_t Bs[kKc][kApTile + 1];
    const int64_t ta = blockIdx.y, tb = blockIdx.x;
    if (upper_only && ta > tb) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t a0 = ta * kApTile, b0 = tb * kApTile;
    uint32_t cnt[kApR][kApR];
#pragma unroll
    for (int i = 0; i < kApR; i++)
#pragma unroll
        for (int j = 0; j < kApR; j++) cnt[i][j] = 0;
    for (uint32_t kc = 0; kc < m; kc += kKc) {
#pragma unroll
        for (int q = 0; q < kApTile * kKc / 256; q++) {
            const int idx = threadIdx.x + 256 * q;
            const int r = idx >> 4, kk = idx & 15;
            const uint32_t k = kc + kk;
            const int64_t ra = a0 + r, rb = b0 + r;
            // out-of-range rows/components load two different sentinels so they never match
            As[kk][r] = (ra < na && k < m) ? sa[ra * m + k] : 0xFFFFFFFFFFFFFFFFull;
            Bs[kk][r] = (rb < nb && k < m) ? sb[rb * m + k] : 0xFFFFFFFFFFFFFFFEull;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKc; kk++) {
            uint64_t a[kApR], b[kApR];
#pragma unroll
            for (int i = 0; i < kApR; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < kApR; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < kApR; i++)
#pragma unroll
                for (int j = 0; j < kApR; j++) cnt[i][j] += (a[i] == b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < kApR; i++) {
        const int64_t a = a0 + ty + 16 * i;
        if (a >= na) continue;
#pragma unroll
        for (int j = 0; j < kApR; j++) {
            const int64_t b = b0 + tx + 16 * j;
            if (b >= nb || (upper_only && a > b)) continue;
            out[a * ldo + b] = (uint16_t)cnt[i][j];
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

// Component minima are non-negative doubles or +inf, which order like their
// bit patterns as unsigned integers: the comparison runs on the integer pipe
// (an FP64 comparison would make this HBM-bound kernel FP64-pipe bound).
__global__ void merge_kernel(const double *__restrict__ q, const uint64_t *__restrict__ z, int64_t parts, uint32_t m,
                             double *__restrict__ oq, uint64_t *__restrict__ oz) {
    const unsigned long long *qb = (const unsigned long long *)q;
    constexpr unsigned long long kInf = 0x7FF0000000000000ull;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        unsigned long long bq = kInf;
        uint64_t bz = 0;
#pragma unroll 8
        for (int64_t p = 0; p < parts; p++) {
            const unsigned long long x = __ldcs(qb + p * m + k);
            const uint64_t d = __ldcs(z + p * m + k);
            if (x < bq || (x == bq && x != kInf && d < bz)) { bq = x; bz = d; }
        }
        oq[k] = __longlong_as_double((long long)bq);
        oz[k] = bq == kInf ? 0 : bz;
    }
}

extern "C" pmh_status pmh_estimate_jp(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m,
                                      int32_t upper_only, uint16_t *counts, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_sigs < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_sigs < 0");
    if (m < 1 || m > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, 65535]", m);
    if (num_sigs == 0) return PMH_OK;
    if (!sigs || !counts) return fail(h, PMH_ERR_INVALID_ARG, "NULL sigs/counts");
    const int64_t tiles = (num_sigs + kApTile - 1) / kApTile;
    if (tiles > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "num_sigs too large for one launch");
    CUDA_TRY(h, cudaSetDevice(h->device));
    dim3 grid((unsigned)tiles, (unsigned)tiles);
    allpairs_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(sigs, num_sigs, sigs, num_sigs, m, upper_only ? 1 : 0,
                                                            counts, num_sigs);
    CUDA_TRY(h, cudaGetLastError());
    return PMH_OK;
}

extern "C" pmh_status pmh_estimate_jp_block(pmh_handle h, const uint64_t *sig_a, int64_t num_a, const uint64_t *sig_b,
                                            int64_t num_b, uint32_t m, uint16_t *counts, int64_t ld_counts,
                                            void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_a < 0 || num_b < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_a < 0 or num_b < 0");
    if (m < 1 || m > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, 65535]", m);
    if (num_a == 0 || num_b == 0) return PMH_OK;
    if (!sig_a || !sig_b || !counts) return fail(h, PMH_ERR_INVALID_ARG, "NULL sig_a/sig_b/counts");
    if (ld_counts < num_b) return fail(h, PMH_ERR_INVALID_ARG, "ld_counts < num_b");
    const int64_t ta = (num_a + kApTile - 1) / kApTile, tb = (num_b + kApTile - 1) / kApTile;
    if (ta > 65535 || tb > 2147483647ll) return fail(h, PMH_ERR_UNSUPPORTED, "tables too large for one launch");
    CUDA_TRY(h, cudaSetDevice(h->device));
    dim3 grid((unsigned)tb, (unsigned)ta);
    allpairs_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(sig_a, num_a, sig_b, num_b, m, 0, counts, ld_counts);
    CUDA_TRY(h, cudaGetLastError());
    return PMH_OK;
}

extern "C" pmh_status pmh_estimate_allpairs(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m,
                                            int32_t upper_only, uint16_t *counts, void *stream) {
    return pmh_estimate_jp(h, sigs, num_sigs, m, upper_only, counts, stream);
}

// ------------------------------------------------------------------ P-MinHash
extern "C" pmh_status pmh_pminhash_batch(pmh_handle h, const uint64_t *ids, const double *weights,
                                         const int64_t *offsets, int64_t num_sets, uint32_t m, uint64_t seed,
                                         uint64_t *out_ids, double *out_q, int32_t *set_status, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_sets < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_sets < 0");
    if (m < 1 || m > PMH_MAX_M) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, %u]", m, PMH_MAX_M);
    if (num_sets == 0) return PMH_OK;
    if (!ids || !weights || !offsets || !out_ids) return fail(h, PMH_ERR_INVALID_ARG, "NULL ids/weights/offsets/out_ids");
    CUDA_TRY(h, cudaSetDevice(h->device));
    if (!h->pm_counter) CUDA_TRY(h, cudaMalloc(&h->pm_counter, sizeof(unsigned int)));
    bool fits = true;
    cudaError_t e = pminhash_launch(ids, weights, offsets, num_sets, m, seed, out_ids, out_q, set_status, h->pm_counter,
                                    h->sm_count, (cudaStream_t)stream, &fits);
    if (e != cudaSuccess) return fail(h, PMH_ERR_CUDA, "P-MinHash launch: %s", cudaGetErrorString(e));
    if (!fits) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u does not fit in shared memory", m);
    return PMH_OK;
}

// ------------------------------------------------------------------ status reduction
// Per-code item counts (codes outside 0..6 in slot 7) and the minimum of
// (index << 8 | code) over the items that are not PMH_OK.  Each thread counts
// in registers, warps add their counts with one reduction per code, and each
// warp adds to the global totals once per code (a shared or global atomic per
// item would serialise on the one code nearly every item has).
static __global__ void status_reduce_kernel(const int32_t *__restrict__ st, int64_t n, unsigned long long *out) {
    unsigned int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long first = ~0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = st[i];
        const int slot = (c >= 0 && c <= 6) ? c : 7;
#pragma unroll
        for (int j = 0; j < 8; ++j) cnt[j] += (slot == j) ? 1u : 0u;
        if (c != PMH_OK) first = min(first, ((unsigned long long)i << 8) | (unsigned long long)(slot == 7 ? 255 : c));
    }
    for (int o = 16; o; o >>= 1) first = min(first, __shfl_xor_sync(0xFFFFFFFFu, first, o));
    const int lane = threadIdx.x & 31;
    if (lane == 0 && first != ~0ull) atomicMin(&out[8], first);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const unsigned int t = __reduce_add_sync(0xFFFFFFFFu, cnt[j]);
        if (lane == 0 && t) atomicAdd(&out[j], (unsigned long long)t);
    }
}

extern "C" pmh_status pmh_sync_status(pmh_handle h, const int32_t *set_status, int64_t n, int64_t *counts,
                                      int64_t *first_bad, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (n < 0 || (n > 0 && !set_status)) return fail(h, PMH_ERR_INVALID_ARG, "n < 0 or NULL set_status");
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long host[9];
    for (int i = 0; i < 8; i++) host[i] = 0;
    host[8] = ~0ull;
    if (n > 0) {
        if (!h->status_scratch) CUDA_TRY(h, cudaMalloc(&h->status_scratch, 9 * sizeof(unsigned long long)));
        CUDA_TRY(h, cudaMemcpyAsync(h->status_scratch, host, sizeof(host), cudaMemcpyHostToDevice, st));
        const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)h->sm_count * 4);
        status_reduce_kernel<<<grid, 256, 0, st>>>(set_status, n, h->status_scratch);
        CUDA_TRY(h, cudaGetLastError());
        CUDA_TRY(h, cudaMemcpyAsync(host, h->status_scratch, sizeof(host), cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(h, cudaStreamSynchronize(st));
    if (counts)
        for (int i = 0; i < 8; i++) counts[i] = (int64_t)host[i];
    if (first_bad) *first_bad = host[8] == ~0ull ? -1 : (int64_t)(host[8] >> 8);
    if (host[8] == ~0ull) return PMH_OK;
    const int code = (int)(host[8] & 0xFF);
    return code == 255 ? PMH_ERR_INVALID_ARG : (pmh_status)code;
}

// ------------------------------------------------------------------ b-bit signatures
// Algorithm "Reduction to a b-bit signature": component k keeps the low b bits
// of mix(z_k ^ key_k), key_k = mix(mix(seed) + (k+1) phi) (output k+1 of
// SplitMix64 seeded with mix(seed)), packed little-endian: field k occupies
// bits (k b) mod 64 .. +b of word (k b) / 64 of its signature's
// ceil(m b / 64) words; unused high bits of the last word are zero.
__device__ __forceinline__ uint64_t bbit_code(uint64_t z, uint32_t k, uint64_t mseed, uint32_t b) {
    const uint64_t h = mix64(z ^ mix64(mseed + ((uint64_t)k + 1) * kPhi));
    return b >= 64 ? h : (h & ((1ull << b) - 1));
}

static __global__ void bbit_reduce_kernel(const uint64_t *__restrict__ sig, int64_t n, uint32_t m, uint32_t b,
                                          uint64_t mseed, uint32_t words, uint64_t *__restrict__ out) {
    const uint32_t per = 64 / b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * words; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = t / words;
        const uint32_t wd = (uint32_t)(t - a * words);
        uint64_t acc = 0;
        for (uint32_t j = 0; j < per; j++) {
            const uint32_t k = wd * per + j;
            if (k >= m) break;
            acc |= bbit_code(sig[a * m + k], k, mseed, b) << (j * b);
        }
        out[t] = acc;
    }
}

// Number of all-zero b-bit fields of a 32-bit word (b <= 32): fold each field's
// bits into its lowest bit, then count the lowest bits left clear.
template <int B>
__device__ __forceinline__ uint32_t zero_fields32(uint32_t x) {
    if constexpr (B == 1) {
        return 32u - __popc(x);
    } else {
        constexpr uint32_t low = B == 2 ? 0x55555555u : B == 4 ? 0x11111111u : B == 8 ? 0x01010101u
                               : B == 16 ? 0x00010001u : 0x00000001u;
#pragma unroll
        for (int s = 1; s < B; s <<= 1) x |= x >> s;
        return __popc(~x & low);
    }
}

template <int B>
__device__ __forceinline__ uint32_t zero_fields64(uint64_t x) {
    if constexpr (B == 64) return x == 0 ? 1u : 0u;
    else return zero_fields32<B>((uint32_t)x) + zero_fields32<B>((uint32_t)(x >> 32));
}

// Equal-field counts of all pairs of packed b-bit signatures: the tiling of
// allpairs_kernel, over words instead of components; the zero padding of the
// last word is counted as equal in every pair and subtracted at the end.
template <int B>
__global__ void __launch_bounds__(256) bbit_allpairs_kernel(const uint64_t *__restrict__ sig, int64_t n, uint32_t words,
                                                            uint32_t pad, int upper_only, uint16_t *__restrict__ out) {
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
    for (uint32_t kc = 0; kc < words; kc += kKc) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int idx = threadIdx.x + 256 * q;
            const int r = idx >> 4, kk = idx & 15;
            const uint32_t k = kc + kk;
            const int64_t ra = a0 + r, rb = b0 + r;
            // outside the arrays: all ones against all zeros, no field equal
            As[kk][r] = (ra < n && k < words) ? sig[ra * words + k] : 0xFFFFFFFFFFFFFFFFull;
            Bs[kk][r] = (rb < n && k < words) ? sig[rb * words + k] : 0ull;
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
                for (int j = 0; j < 4; j++) cnt[i][j] += zero_fields64<B>(a[i] ^ b[j]);
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
            out[a * n + b] = (uint16_t)(cnt[i][j] - pad);
        }
    }
}

static bool bbit_width_ok(uint32_t b) { return b >= 1 && b <= 64 && (b & (b - 1)) == 0; }

extern "C" pmh_status pmh_bbit_reduce(pmh_handle h, const uint64_t *sigs, int64_t num_sigs, uint32_t m, uint32_t b,
                                      uint64_t seed, uint64_t *packed, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_sigs < 0 || m < 1) return fail(h, PMH_ERR_INVALID_ARG, "num_sigs < 0 or m < 1");
    if (!bbit_width_ok(b)) return fail(h, PMH_ERR_INVALID_ARG, "b = %u is not a power of two in [1, 64]", b);
    if (num_sigs == 0) return PMH_OK;
    if (!sigs || !packed) return fail(h, PMH_ERR_INVALID_ARG, "NULL sigs/packed");
    CUDA_TRY(h, cudaSetDevice(h->device));
    const uint32_t words = (uint32_t)(((uint64_t)m * b + 63) / 64);
    const int64_t total = num_sigs * words;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)h->sm_count * 16);
    bbit_reduce_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(sigs, num_sigs, m, b, host_mix64(seed), words, packed);
    CUDA_TRY(h, cudaGetLastError());
    return PMH_OK;
}

extern "C" pmh_status pmh_bbit_allpairs(pmh_handle h, const uint64_t *packed, int64_t num_sigs, uint32_t m, uint32_t b,
                                        int32_t upper_only, uint16_t *counts, void *stream) {
    if (!h) return PMH_ERR_INVALID_ARG;
    h->err.clear();
    if (num_sigs < 0) return fail(h, PMH_ERR_INVALID_ARG, "num_sigs < 0");
    if (m < 1 || m > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "m = %u outside [1, 65535]", m);
    if (!bbit_width_ok(b)) return fail(h, PMH_ERR_INVALID_ARG, "b = %u is not a power of two in [1, 64]", b);
    if (num_sigs == 0) return PMH_OK;
    if (!packed || !counts) return fail(h, PMH_ERR_INVALID_ARG, "NULL packed/counts");
    const int64_t tiles = (num_sigs + kTile - 1) / kTile;
    if (tiles > 65535) return fail(h, PMH_ERR_UNSUPPORTED, "num_sigs too large for one launch");
    CUDA_TRY(h, cudaSetDevice(h->device));
    const uint32_t words = (uint32_t)(((uint64_t)m * b + 63) / 64);
    const uint32_t pad = b == 64 ? 0u : words * (64 / b) - m;
    dim3 grid((unsigned)tiles, (unsigned)tiles);
    cudaStream_t st = (cudaStream_t)stream;
    const int up = upper_only ? 1 : 0;
    switch (b) {
        case 1: bbit_allpairs_kernel<1><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
        case 2: bbit_allpairs_kernel<2><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
        case 4: bbit_allpairs_kernel<4><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
        case 8: bbit_allpairs_kernel<8><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
        case 16: bbit_allpairs_kernel<16><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
        case 32: bbit_allpairs_kernel<32><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
        default: bbit_allpairs_kernel<64><<<grid, 256, 0, st>>>(packed, num_sigs, words, pad, up, counts); break;
    }
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
