// pmh_sketch_batch_noalloc: the batch sketch for callers that cannot allocate
// GPU memory (for example code running inside another runtime's memory
// budget, or under a framework that forbids cudaMalloc on its hot path).  It
// runs the same kernels as pmh_sketch_batch, but its scratch memory (constant
// tables, work queue and per-set statistics) lives in one file-scope device
// array of fixed size that every GPU holds from the moment the library is
// loaded until the process exits.  No call here allocates or frees device
// memory, and no CUDA graph is built.  Grid mode (all SMs on one huge set)
// needs workspace sized by m and is off here: a set of 2^20 elements or more
// runs on one team, with the same result but far more slowly.
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "batch_common.cuh"

using namespace pmh;

namespace {

// Scratch layout: tables for m <= PMH_MAX_M | queue metadata | work queue | FP64 redo list (items whose
// contender log overflowed) | per-set statistics.
constexpr size_t kTableRegion = 1024u * 1024u;                                 // >= table_bytes(PMH_MAX_M)
static_assert(kTableRegion >= table_bytes(PMH_MAX_M), "table region too small");
constexpr size_t kMetaRegion = 16384;                                           // >= kQMetaWords * 4
constexpr size_t kQueueRegion = (size_t)PMH_NOALLOC_MAX_ITEMS * sizeof(uint64_t);
constexpr size_t kStatsRegion = (size_t)PMH_NOALLOC_MAX_SETS * 16;
constexpr size_t kScratchBytes = kTableRegion + kMetaRegion + 2 * kQueueRegion + kStatsRegion;
static_assert(kMetaRegion >= kQMetaWords * sizeof(unsigned int), "queue metadata region too small");
static_assert(sizeof(SetStat) == 16, "per-set statistics entry is 16 bytes");

// Lives in every GPU's memory while the library is loaded.  In host code this
// name is only a stand-in: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceState {
    int sm_count = 0;                // 0 until the first call on this device
};
DeviceState g_state[kMaxDevices];
std::mutex g_mu;
unsigned char g_host_tables[kTableRegion];   // staging for table uploads (static: no allocation)

pmh_status fail_na(pmh_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_thread_error(buf);
    return code;
}

}  // namespace

extern "C" pmh_status pmh_sketch_batch_noalloc(const uint64_t *ids, const double *weights, const int64_t *offsets,
                                               int64_t num_sets, uint32_t m, const int32_t *variants,
                                               int32_t num_variants, int32_t precision, uint64_t seed,
                                               uint64_t *out_ids, double *out_q, int32_t *set_status,
                                               uint64_t *counters, void *stream) {
    set_thread_error("");
    if (num_sets < 0) return fail_na(PMH_ERR_INVALID_ARG, "num_sets < 0");
    if (m < 1 || m > PMH_MAX_M) return fail_na(PMH_ERR_UNSUPPORTED, "m = %u outside [1, %u]", m, PMH_MAX_M);
    if (!variants || num_variants < 1 || num_variants > PMH_MAX_VARIANTS)
        return fail_na(PMH_ERR_INVALID_ARG, "need 1..%d variants", PMH_MAX_VARIANTS);
    if (precision != PMH_FP64 && precision != PMH_FP32_RECHECK) return fail_na(PMH_ERR_INVALID_ARG, "bad precision %d", precision);
    for (int v = 0; v < num_variants; v++) {
        if (variants[v] < PMH_V1 || variants[v] > PMH_V4U) return fail_na(PMH_ERR_INVALID_ARG, "bad variant %d", variants[v]);
        if ((variants[v] == PMH_V3 || variants[v] == PMH_V3A || variants[v] == PMH_V4) && m < 2)
            return fail_na(PMH_ERR_INVALID_ARG, "variant %d requires m >= 2", variants[v]);
    }
    if (num_sets > PMH_NOALLOC_MAX_SETS)
        return fail_na(PMH_ERR_UNSUPPORTED, "num_sets = %lld exceeds the allocation-free limit of %d sets",
                       (long long)num_sets, PMH_NOALLOC_MAX_SETS);
    if (num_sets * num_variants > PMH_NOALLOC_MAX_ITEMS)
        return fail_na(PMH_ERR_UNSUPPORTED, "num_sets * num_variants = %lld exceeds the allocation-free limit of %d items",
                       (long long)(num_sets * num_variants), PMH_NOALLOC_MAX_ITEMS);
    if (num_sets == 0) return PMH_OK;
    if (!ids || !weights || !offsets || !out_ids) return fail_na(PMH_ERR_INVALID_ARG, "NULL ids/weights/offsets/out_ids");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_na(PMH_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_na(PMH_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    cudaStream_t st = (cudaStream_t)stream;
    // The tables are staged through one static host buffer that later calls rewrite, so a call
    // recorded into a CUDA graph would replay with whatever the buffer holds then: refused.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return fail_na(PMH_ERR_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    if (cs != cudaStreamCaptureStatusNone)
        return fail_na(PMH_ERR_UNSUPPORTED, "pmh_sketch_batch_noalloc cannot be called while its stream is being captured");
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &ds = g_state[dev];
    if (!ds.sm_count) {
        e = cudaDeviceGetAttribute(&ds.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) { ds.sm_count = 0; return fail_na(PMH_ERR_CUDA, "device attribute: %s", cudaGetErrorString(e)); }
    }
    // the array's device address on the current device, resolved on every call (cheap, and still
    // right after a cudaDeviceReset has replaced the context)
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_na(PMH_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    unsigned char *base = (unsigned char *)ptr;
    unsigned char *tables = base;
    unsigned int *qmeta = (unsigned int *)(base + kTableRegion);
    uint64_t *queue = (uint64_t *)(base + kTableRegion + kMetaRegion);
    uint64_t *redo = (uint64_t *)(base + kTableRegion + kMetaRegion + kQueueRegion);
    SetStat *stats = (SetStat *)(base + kTableRegion + kMetaRegion + 2 * kQueueRegion);

    // The tables of this m are uploaded on every call (120 KiB at m = 1024), in stream order before
    // the kernels: nothing on the host has to know what the array held before.  The copy from this
    // pageable buffer has read it by the time cudaMemcpyAsync returns, so the next call may refill it.
    Tables tab;
    build_tables(m, g_host_tables, tables, &tab);
    e = cudaMemcpyAsync(tables, g_host_tables, table_bytes(m), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail_na(PMH_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
    SketchParams p;
    Thresholds th;
    th.grid_min = 0;   // grid mode needs workspace sized by m: off here
    fill_params(&p, ids, weights, offsets, num_sets, m, variants, num_variants, seed, out_ids, out_q, set_status,
                counters, th);
    p.tab = tab;
    Plan plan;
    bool fits = true;
    e = plan_batch(ds.sm_count, precision, m, variants, num_variants, num_sets, nullptr, &plan, &fits);
    if (e != cudaSuccess) return fail_na(PMH_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
    if (!fits) return fail_na(PMH_ERR_UNSUPPORTED, "m = %u does not fit in shared memory", m);
    // enqueue_batch clears the queue metadata; the queue and the statistics are rewritten in full
    e = enqueue_batch(p, plan, precision, ds.sm_count, queue, redo, qmeta, stats, st, nullptr);
    if (e != cudaSuccess) return fail_na(PMH_ERR_CUDA, "sketch launch: %s", cudaGetErrorString(e));
    return PMH_OK;
}
