// Pieces of pmh_sketch_batch shared by the allocating entry point (api.cu)
// and the allocation-free one (noalloc.cu): per-m constant tables, the device
// work queue, per-set statistics, the launch plan and the launch sequence.
// Kernels here are static: each translation unit that includes the header
// owns its copy.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "launch.h"

namespace pmh {

// ------------------------------------------------------------------ tables
// Per-m constants of Sec. ProbMinHash2/3/4 in FP64 (host libm), plus FP32
// copies for the filter: five FP64 arrays then five FP32 arrays of m+1 entries,
// then (16-byte aligned) the ProbMinHash4 FP32 constants of each point packed
// in one float4, then the rejection sampler's constants per rate (Sec.
// Truncated Exponential Sampling): k1, k2 (u64), c1, c3, lambda (FP64) and c1
// in FP32, m+1 entries each.
constexpr size_t table_f4_off(uint32_t m) { return ((5 * ((size_t)m + 1) * (sizeof(double) + sizeof(float))) + 15) & ~(size_t)15; }
constexpr size_t table_rej_off(uint32_t m) { return table_f4_off(m) + ((size_t)m + 1) * 16; }
constexpr size_t table_bytes(uint32_t m) { return table_rej_off(m) + ((size_t)m + 1) * (5 * 8 + 4); }

// Fills `host` (table_bytes(m) bytes) and sets `out` to point into the same
// layout at device address `dev`.
inline void build_tables(uint32_t m, unsigned char *host, const void *dev, Tables *out) {
    const size_t n = (size_t)m + 1;
    double *beta = (double *)host, *gamma = beta + n, *dgamma = gamma + n, *c4 = dgamma + n, *inv4 = c4 + n;
    for (size_t i = 0; i < 5 * n; i++) beta[i] = 0.0;
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
    float *f = (float *)(host + 5 * n * sizeof(double));
    for (size_t i = 0; i < 5 * n; i++) f[i] = (float)beta[i];
    {
        const float *g32 = f + n, *dg32 = f + 2 * n, *c432 = f + 3 * n, *i432 = f + 4 * n;
        float *q = (float *)(host + table_f4_off(m));
        for (size_t i = 0; i < 4 * n; i++) q[i] = 0.0f;
        for (uint32_t i = 1; i <= m; i++) {
            q[4 * i + 0] = g32[i - 1];
            if (i < m) {
                q[4 * i + 1] = dg32[i];
                q[4 * i + 2] = c432[i];
                q[4 * i + 3] = i432[i];
            }
        }
    }
    const char *d = (const char *)dev;
    Tables &t = *out;
    t.m = m;
    t.beta = (const double *)d;
    t.gamma = (const double *)(d + 1 * n * sizeof(double));
    t.dgamma = (const double *)(d + 2 * n * sizeof(double));
    t.c4 = (const double *)(d + 3 * n * sizeof(double));
    t.inv4 = (const double *)(d + 4 * n * sizeof(double));
    const char *fb = d + 5 * n * sizeof(double);
    t.beta32 = (const float *)fb;
    t.gamma32 = (const float *)(fb + 1 * n * sizeof(float));
    t.dgamma32 = (const float *)(fb + 2 * n * sizeof(float));
    t.c4_32 = (const float *)(fb + 3 * n * sizeof(float));
    t.inv4_32 = (const float *)(fb + 4 * n * sizeof(float));
    t.p4 = (const float4 *)(d + table_f4_off(m));
    t.c3 = c3;
    t.inv3 = inv3;
    t.delta = delta;
    t.c3_32 = (float)c3;
    t.inv3_32 = (float)inv3;
    t.delta32 = (float)delta;
    // Exp(lambda_1;0,1) >= U * (1-e^-lambda_1)/lambda_1 (since -log1p(-a) >= a); round the factor down
    const double lo = (m >= 2) ? -c3 / lambda1 : 1.0;
    float lo32 = (float)lo;
    if ((double)lo32 > lo) lo32 = std::nextafterf(lo32, 0.0f);
    t.te_lo = lo32;
    t.lambda1_32 = (float)lambda1;

    // rejection sampler constants, i = 1..m-1 (entry i for the rate lambda_i; ProbMinHash3 uses i = 1)
    uint64_t *k1 = (uint64_t *)(host + table_rej_off(m)), *k2 = k1 + n;
    double *rc1 = (double *)(k2 + n), *rc3 = rc1 + n, *rlam = rc3 + n;
    float *rc1f = (float *)(rlam + n);
    for (size_t i = 0; i < n; i++) { k1[i] = 0; k2[i] = 0; rc1[i] = 0.0; rc3[i] = 0.0; rlam[i] = 0.0; rc1f[i] = 0.0f; }
    for (uint32_t i = 1; i < m; i++) {
        const double l = std::log1p(1.0 / (double)(m - i));
        const double c1 = std::expm1(l) / l;
        const double c2 = std::log(2.0 / (1.0 + std::exp(-l))) / l;
        const double c3 = -std::expm1(-l) / l;
        // smallest k with fl(fl(k 2^-53) c1) >= 1: the product is monotone in k
        uint64_t lo_k = 0, hi_k = 1ull << 53;
        while (lo_k < hi_k) {
            const uint64_t mid = lo_k + (hi_k - lo_k) / 2;
            const double u = (double)mid * 0x1p-53;
            if (c1 * u >= 1.0) hi_k = mid; else lo_k = mid + 1;
        }
        k1[i] = lo_k;
        k2[i] = (uint64_t)std::ceil(std::ldexp(c2, 53));
        rc1[i] = c1;
        rc3[i] = c3;
        rlam[i] = l;
        rc1f[i] = (float)c1;
    }
    t.rej_k1 = (const uint64_t *)(d + table_rej_off(m));
    t.rej_k2 = t.rej_k1 + n;
    t.rej_c1 = (const double *)(t.rej_k2 + n);
    t.rej_c3 = t.rej_c1 + n;
    t.rej_lam = t.rej_c3 + n;
    t.rej_c1_32 = (const float *)(t.rej_lam + n);
    // filter at point 1: a 23-bit lower bound ulo of U with ulo < u1 guarantees U < k1 2^-53
    // (U < ulo + 2^-23); u1 = the largest float at most k1 2^-53 - 2^-23
    t.rej_u1_32 = 0.0f;
    if (m >= 2) {
        const double lim = (double)k1[1] * 0x1p-53 - 0x1p-23;
        float u1 = (float)lim;
        if ((double)u1 > lim) u1 = std::nextafterf(u1, 0.0f);
        t.rej_u1_32 = lim > 0.0 ? u1 : 0.0f;
    }
}

inline uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------------ queue
// Items (variant, set) in family-major order (ProbMinHash1/1a, 2, 3/3a, 4),
// each family sorted by decreasing floor(log2(n+1)) (largest sets first).
// Meta layout: [0, 256) histogram per (family, bucket), [256, 512) running
// starts, [512, 516) per-family head counters of the persistent kernels.
// [516] counts the sets whose statistics are split over all blocks, [518, 520)
// is the statistics kernel's set counter (u64), [520, 524) the per-family
// lengths of the FP64 redo lists, [524, 528) the head counters of the redo
// kernels, [528, 530) the prefilter kernel's counter (u64), [530] the number
// of sets it lists and [531] a flag set when the offsets decrease somewhere;
// [532, ...) lists the split sets (u64 set indices, kBigCap of them).
constexpr int kQHist = 0, kQStart = 256, kQHead = 512, kQBigCount = 516, kQStatNext = 518, kQRedoCount = 520,
              kQRedoHead = 524, kQListNext = 528, kQListCount = 530, kQListBad = 531, kQBigList = 532;
constexpr int kBigCap = 1024;
constexpr int kQMetaWords = kQBigList + 2 * kBigCap;
constexpr int kQMetaClearWords = kQBigList;     // words cleared per call
#ifndef PMH_STAT_CHUNK
#define PMH_STAT_CHUNK 16384   // measured on one set of 1e8: 16384 0.193 ms, 65536 0.221, 4096 0.215 (queue + statistics)
#endif
constexpr int64_t kStatChunk = PMH_STAT_CHUNK;  // elements per statistics chunk of a split set
constexpr int64_t kStatBig = 262144;            // sets longer than this are split over all blocks

struct FamOfVariant {
    int f[PMH_MAX_VARIANTS];
};

__device__ __forceinline__ int queue_bucket(const int64_t *off, int64_t s) {
    int64_t n = off[s + 1] - off[s];
    if (n < 0) n = 0;
    return 63 - __clzll((long long)(n + 1));
}

static __global__ void queue_count(const int64_t *off, int64_t num_sets, int32_t nv, FamOfVariant fv, unsigned int *meta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < num_sets * nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i % num_sets;
        const int v = (int)(i / num_sets);
        atomicAdd(&meta[kQHist + (fv.f[v] - 1) * 64 + queue_bucket(off, s)], 1u);
    }
}
static __global__ void queue_starts(unsigned int *meta) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned int acc = 0;
        for (int f = 0; f < 4; ++f)
            for (int b = 63; b >= 0; --b) { meta[kQStart + f * 64 + b] = acc; acc += meta[kQHist + f * 64 + b]; }
        for (int f = 0; f < 4; ++f) meta[kQHead + f] = 0;
    }
}
// Items of sets with at least grid_min elements also go to the per-family grid
// list (first kMaxGrid of them); their queue entries are then marked skipped.
static __global__ void queue_scatter(const int64_t *off, int64_t num_sets, int32_t nv, FamOfVariant fv,
                                     unsigned int *meta, uint64_t *queue, GridCtl *gctl, int64_t grid_min) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < num_sets * nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i % num_sets;
        const int64_t v = i / num_sets;
        const int f = fv.f[v] - 1;
        const unsigned int pos = atomicAdd(&meta[kQStart + f * 64 + queue_bucket(off, s)], 1u);
        uint64_t item = ((uint64_t)v << 40) | (uint64_t)s;
        if (gctl && off[s + 1] - off[s] >= grid_min && off[s + 1] - off[s] <= (int64_t)PMH_MAX_SET_ELEMENTS) {
            const unsigned int slot = atomicAdd(&gctl->count[f], 1u);
            if (slot < (unsigned int)kMaxGrid) {
                gctl->list[f][slot] = item;
                item |= kSkipBit;
            }
        }
        queue[pos] = item;
    }
}

// Per-set statistics, computed once per set for all variants: the weight sum
// (it only sets the threshold T, so a ~1e-3 relative error is harmless), the
// number of positive weights, and a bad-weight flag (negative, NaN, +-inf, or
// a subnormal whose reciprocal overflows).  One block per set, grid-stride
// over sets, four loads in flight per thread.
//
// The sum avoids FP64 arithmetic (a slow pipe on this GPU): each thread keeps
// an FP32 accumulator `acc` scaled by 2^-(me-1023), me = the largest biased
// FP64 exponent it has seen; a weight enters as the FP32 number with its top
// 23 mantissa bits and exponent shifted by -me (integer operations only), and
// a larger exponent rescales acc by a power of two.  Weights below 2^-126 of
// the running maximum (and subnormals) add nothing.  Weights in [2^-100, 2^90)
// (nearly all in practice) skip the rescaling: they go to a plain FP32 sum
// (two integer operations and an add), folded into the scaled one at the end.
struct ScaledSum {
    int me = -1000;   // running maximum biased exponent (none yet)
    float acc = 0.0f;
};
__device__ __forceinline__ float pow2f(int d) {   // 2^d for d in [-126, 0], else 0 below
    return d >= -126 ? __int_as_float((127 + d) << 23) : 0.0f;
}
__device__ __forceinline__ void scaled_add(ScaledSum &s, uint64_t bits) {
    const int ex = (int)(bits >> 52) & 0x7FF;
    if (ex > s.me) {
        s.acc = __fmul_rn(s.acc, pow2f(s.me - ex));
        s.me = ex;
    }
    const int d = ex - s.me;
    if (d >= -126) s.acc = __fadd_rn(s.acc, __int_as_float(((127 + d) << 23) | (int)((bits >> 29) & 0x7FFFFFu)));
}
__device__ __forceinline__ void scaled_merge(ScaledSum &s, int me2, float acc2) {
    const int M = max(s.me, me2);
    s.acc = __fadd_rn(__fmul_rn(s.acc, pow2f(s.me - M)), __fmul_rn(acc2, pow2f(me2 - M)));
    s.me = M;
}

// Statistics of the elements [b, e) of one set by one block; the totals are
// valid in thread 0.
struct StatPart {
    ScaledSum sum;
    float fsum = 0.0f;   // the weights in [2^-100, 2^90), summed as plain FP32
    unsigned int np = 0;
    int bad = 0;
};
// Biased FP64 exponents of the plain FP32 sum: [kFastLo, kFastHi) (2^-100 <= w < 2^90, so a
// thread's sum of at most 2^20 of them stays finite).
constexpr uint32_t kFastLo = 923, kFastHi = 1113;
__device__ __forceinline__ void stat_one(StatPart &r, uint64_t x) {
    // common case: a positive weight in the fast range enters as the FP32 number with its top 23
    // mantissa bits (bits 29..60 of the double, exponent re-biased from 1023 to 127)
    if ((uint32_t)(x >> 32) - (kFastLo << 20) < ((kFastHi - kFastLo) << 20)) {
        r.fsum = __fadd_rn(r.fsum, __uint_as_float((uint32_t)(x >> 29) - (896u << 23)));
        r.np++;
        return;
    }
    const int ex = (int)(x >> 52) & 0x7FF;
    const bool neg = (x >> 63) != 0;
    const bool zero = (x << 1) == 0;
    if (ex == 0x7FF || (neg && !zero)) { r.bad = 1; return; }
    if (zero) return;
    if (ex == 0) {   // subnormal: counted, adds nothing to the sum; bad if 1/w overflows
        if (isinf(__drcp_rn(__longlong_as_double((long long)x)))) r.bad = 1;
        else r.np++;
        return;
    }
    scaled_add(r.sum, x);
    r.np++;
}
__device__ __forceinline__ StatPart block_stats(const unsigned long long *wb, int64_t b, int64_t e) {
    __shared__ float sacc[8];
    __shared__ int sme[8], sbad[8];
    __shared__ unsigned int snp[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    StatPart r;
    // 16-byte loads of two weights each: a first weight off the 16-byte grid and a last odd one
    // are read alone (a zero pair, used as padding, counts as two skipped weights)
    int64_t a = b;
    if (a < e && ((uintptr_t)(wb + a) & 15u) != 0) {
        if (threadIdx.x == 0) stat_one(r, __ldcs(wb + a));
        a++;
    }
    const int64_t np2 = (e - a) / 2;
    const ulonglong2 *w2 = (const ulonglong2 *)(wb + a);
    for (int64_t p0 = threadIdx.x; p0 < np2; p0 += 4 * (int64_t)blockDim.x) {
        ulonglong2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + (int64_t)u * blockDim.x;
            v[u] = p < np2 ? __ldcs(w2 + p) : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            stat_one(r, v[u].x);
            stat_one(r, v[u].y);
        }
    }
    if (a + 2 * np2 < e && threadIdx.x == 0) stat_one(r, __ldcs(wb + e - 1));
    if (r.fsum != 0.0f) scaled_add(r.sum, (uint64_t)__double_as_longlong((double)r.fsum));
    for (int o = 16; o; o >>= 1) {
        const int me2 = __shfl_xor_sync(0xFFFFFFFFu, r.sum.me, o);
        const float acc2 = __shfl_xor_sync(0xFFFFFFFFu, r.sum.acc, o);
        scaled_merge(r.sum, me2, acc2);
        r.np += __shfl_xor_sync(0xFFFFFFFFu, r.np, o);
        r.bad |= __shfl_xor_sync(0xFFFFFFFFu, r.bad, o);
    }
    if (lane == 0) { sacc[warp] = r.sum.acc; sme[warp] = r.sum.me; snp[warp] = r.np; sbad[warp] = r.bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        StatPart t;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { scaled_merge(t.sum, sme[j], sacc[j]); t.np += snp[j]; t.bad |= sbad[j]; }
        r = t;
    }
    __syncthreads();
    return r;
}
__device__ __forceinline__ double scaled_value(const ScaledSum &s) {
    return s.me < 0 ? 0.0 : ldexp((double)s.acc, s.me - 1023);
}

// Pass 1: one block per set, the blocks taking sets from a shared counter (set
// sizes vary by orders of magnitude, so a fixed deal leaves blocks idle).  A
// set longer than kStatBig is listed (up to kBigCap of them) and only its
// first chunk is summed here; pass 2 adds the rest with all blocks.
static __global__ void __launch_bounds__(256) set_stats_kernel(const int64_t *off, const double *w, int64_t num_sets,
                                                               SetStat *out, unsigned int *meta) {
    __shared__ int s_listed;
    __shared__ long long s_next;
    const unsigned long long *wb = (const unsigned long long *)w;
    for (;;) {
        if (threadIdx.x == 0) s_next = (long long)atomicAdd((unsigned long long *)(meta + kQStatNext), 1ull);
        __syncthreads();
        const int64_t s = s_next;
        if (s >= num_sets) break;
        const int64_t b = off[s], e = off[s + 1];
        int64_t end = e;
        if (threadIdx.x == 0) {
            s_listed = 0;
            if (e - b > kStatBig) {
                const unsigned int slot = atomicAdd(&meta[kQBigCount], 1u);
                if (slot < (unsigned int)kBigCap) {
                    ((unsigned long long *)(meta + kQBigList))[slot] = (unsigned long long)s;
                    s_listed = 1;
                }
            }
        }
        __syncthreads();
        if (s_listed) end = b + kStatChunk;
        const StatPart r = block_stats(wb, b, end);
        if (threadIdx.x == 0) {
            SetStat o;
            o.wsum = scaled_value(r.sum);
            o.npos = r.np;
            o.bad = r.bad;
            out[s] = o;
        }
    }
}

// Pass 2: the chunks after the first of every listed set, numbered across the
// listed sets and dealt round-robin to all blocks; partial results are added
// atomically (one FP64 add per chunk).
static __global__ void __launch_bounds__(256) set_stats_big_kernel(const int64_t *off, const double *w, SetStat *out,
                                                                   const unsigned int *meta) {
    const unsigned long long *wb = (const unsigned long long *)w;
    const int nbig = min((int)meta[kQBigCount], kBigCap);
    const int64_t G = gridDim.x;
    int64_t base = 0;   // global number of the entry's chunk 1
    for (int j = 0; j < nbig; ++j) {
        const int64_t s = (int64_t)((const unsigned long long *)(meta + kQBigList))[j];
        const int64_t b = off[s], e = off[s + 1];
        const int64_t nch = (e - b + kStatChunk - 1) / kStatChunk;
        const int64_t first = 1 + (((int64_t)blockIdx.x - base) % G + G) % G;   // (base + c - 1) = blockIdx.x mod G
        base += nch - 1;
        for (int64_t c = first; c < nch; c += G) {
            const int64_t cb = b + c * kStatChunk;
            const StatPart r = block_stats(wb, cb, min(e, cb + kStatChunk));
            if (threadIdx.x == 0) {
                atomicAdd(&out[s].wsum, scaled_value(r.sum));
                atomicAdd(&out[s].npos, r.np);
                if (r.bad) atomicOr(&out[s].bad, 1);
            }
        }
    }
}

// ------------------------------------------------------------------ prefilter lists
#ifndef PMH_LIST_BLOCK
#define PMH_LIST_BLOCK 512     // threads per block of the prefilter kernel
#endif
#ifndef PMH_LIST_UNROLL
#define PMH_LIST_UNROLL 8      // elements per thread and step (their loads in flight together)
#endif
// One pass over the elements of every set of list_min..list_max elements that
// keeps the elements whose first point can lie below the first round's bound
// in some family: U te_lo (1 - 16 ulp) <= t_s (w 2^-sigma), the sketch kernels'
// own filter test with the smallest lower-bound factor of any family (te_lo of
// Exp(lambda;0,1) <= 1 of Exp(1)) and the first round's bound t_s, which the
// running bound of every later point of that round only undercuts.  Each kept
// element is written as (key, index | scaled weight << 32), so that the first
// round of every weighted variant of the set visits only these entries, with
// one SplitMix64 word to compute per entry (point 1's value word) instead of
// two per element (the key and that word).  The sets that profit are those much
// larger than m (ln m + c), where most elements fail the first point's test;
// the elements are hashed here once for all variants instead of once per
// variant.  Set s may use list[(offsets[s] - offsets[0]) / 2, + n/2) and
// list_cap entries in all; a set whose survivors exceed n/2, or that does not
// fit, stays unlisted (list_n = kUnlisted) and is filtered in full.
// The sets of list_min..list_max elements are gathered first (list_select:
// one thread per set; every other set is marked unlisted; offsets that
// decrease anywhere, whose sets' ranges may overlap, turn the lists off for the
// call), then list_kernel
// gives one block to each gathered set, the blocks taking them from a shared
// counter; each thread keeps kListUnroll elements' loads in flight (1,024
// threads per SM at <= 64 registers).
constexpr int kListBlock = PMH_LIST_BLOCK, kListUnroll = PMH_LIST_UNROLL;
static __global__ void __launch_bounds__(256) list_select(const int64_t *off, int64_t num_sets, uint32_t *sel,
                                                          uint32_t *list_n, int64_t list_min, int64_t list_max,
                                                          unsigned int *meta) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < num_sets; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = off[s + 1] - off[s];
        if (n < 0) atomicOr(&meta[kQListBad], 1u);
        if (n >= list_min && n <= list_max) sel[atomicAdd(&meta[kQListCount], 1u)] = (uint32_t)s;
        else list_n[s] = kUnlisted;
    }
}

static __global__ void __launch_bounds__(kListBlock, 1024 / kListBlock) list_kernel(const SketchParams p, ulonglong2 *list, uint32_t *list_n,
                                                          const uint32_t *sel, int64_t list_cap, unsigned int *meta) {
    __shared__ long long s_next;
    __shared__ unsigned int s_cnt;
    const int lane = threadIdx.x & 31;
    const unsigned long long *wb = (const unsigned long long *)p.weights;
    const int64_t off0 = p.offsets[0];
    const float te_lo = p.tab.te_lo;
    const int64_t nsel = (int64_t)ld_volatile((const int *)&meta[kQListCount]);
    const bool disjoint = ld_volatile((const int *)&meta[kQListBad]) == 0;   // the sets' ranges do not overlap
    for (;;) {
        if (threadIdx.x == 0) {
            s_next = (long long)atomicAdd((unsigned long long *)(meta + kQListNext), 1ull);
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t j = s_next;
        if (j >= nsel) break;
        const int64_t s = sel[j];
        const int64_t b = p.offsets[s], n = p.offsets[s + 1] - b;
        const int64_t lb = (b - off0) >> 1, cap = n >> 1;
        const SetStat st = p.stats[s];
        float t_s;
        int sigma;
        first_threshold(p.m, p.t_factor, st.wsum, st.npos, &t_s, &sigma);
        const bool ok = disjoint && b >= off0 && !st.bad && st.npos > 0 && lb + cap <= list_cap && !isinf(t_s);
        if (ok) {
            // 32-bit offsets within the set (n <= list_max < 2^32)
            const unsigned long long *wset = wb + b, *iset = (const unsigned long long *)p.ids + b;
            ulonglong2 *lset = list + lb;
            const uint32_t n32 = (uint32_t)n;
            for (uint32_t e0 = 0; e0 < n32; e0 += kListUnroll * kListBlock) {
                uint64_t wv[kListUnroll], iv[kListUnroll];
#pragma unroll
                for (int u = 0; u < kListUnroll; ++u) {
                    const uint32_t e = e0 + u * kListBlock + threadIdx.x;
                    wv[u] = 0;
                    iv[u] = 0;
                    if (e < n32) {
                        wv[u] = __ldcs(wset + e);
                        iv[u] = __ldcs(iset + e);
                    }
                }
#pragma unroll
                for (int u = 0; u < kListUnroll; ++u) {
                    const uint32_t e = e0 + u * kListBlock + threadIdx.x;
                    const double w = __longlong_as_double((long long)wv[u]);
                    bool keep = false;
                    uint64_t key = 0;
                    float ws = 0.0f;
                    if (e < n32 && weight_positive(w)) {
                        key = mix64(iv[u] ^ p.mixed_seed);
                        ws = ws_scaled(w, sigma);
                        const float ulo = __fmul_rn(unif_lo(value_word(key, 1)), te_lo);
                        keep = !(__fmul_rn(ulo, 1.0f - 16.0f * 0x1p-24f) > __fmul_rn(t_s, ws));
                    }
                    const unsigned msk = __ballot_sync(0xFFFFFFFFu, keep);
                    unsigned int wbase = 0;
                    if (lane == 0 && msk) wbase = atomicAdd(&s_cnt, (unsigned int)__popc(msk));
                    wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
                    const unsigned int pos = wbase + __popc(msk & ((1u << lane) - 1u));
                    if (keep && pos < (uint64_t)cap)
                        lset[pos] = make_ulonglong2(key, (uint64_t)e | ((uint64_t)__float_as_uint(ws) << 32));
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            list_n[s] = (ok && (int64_t)s_cnt <= cap) ? s_cnt : kUnlisted;
            if (ok && p.counters) atomicAdd(&p.counters[PMH_CNT_LIST_HASHED], (unsigned long long)st.npos);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ plan
// Launch plan per family present: warp teams when at least 12 warps per SM
// fit, else CTA teams.  Computed outside any stream capture (it sets kernel
// attributes).
struct Plan {
    int nfam;
    int fam[4];
    int64_t qbase[4], qlen[4];
    LaunchShape shape[4];
    int grid[4];
    LaunchShape gshape[4];   // grid-mode kernel (blocks_per_sm = 0: grid mode off for this family)
    int ggrid[4];
    LaunchShape rshape[4];   // FP32 calls: the FP64 kernel that redoes items whose contender log overflowed
    int rgrid[4];
};

// Default team shape of a family: teams of 2 warps when 16 warps per SM fit,
// else warp teams when 12 fit, else CTA teams of 8; when none of these fits in
// shared memory (FP64 signatures at m = 8192), the shape with the most
// resident warps among those that fit (blocks_per_sm = 0: nothing fits).
inline cudaError_t default_shape(bool f32, int f, uint32_t m, LaunchShape *out) {
    LaunchShape pair_s{}, warp_s{}, cta_s{};
    cudaError_t e = sketch_shape_any(f32, f, kShapePair, m, &pair_s);
    if (e != cudaSuccess) return e;
    e = sketch_shape_any(f32, f, kShapeWarp, m, &warp_s);
    if (e != cudaSuccess) return e;
    LaunchShape shape = pair_s.blocks_per_sm * 8 >= 16 ? pair_s : warp_s;
    if (shape.blocks_per_sm * (shape.block / 32) < 12) {
        e = sketch_shape_any(f32, f, kShapeCta8, m, &cta_s);
        if (e != cudaSuccess) return e;
        if (cta_s.blocks_per_sm > 0) shape = cta_s;
    }
    if (shape.blocks_per_sm <= 0) {
        for (int k = 0; k < kNumShapes; k++) {
            LaunchShape t{};
            e = sketch_shape_any(f32, f, k, m, &t);
            if (e != cudaSuccess) return e;
            if (t.blocks_per_sm * (t.block / 32) > shape.blocks_per_sm * (shape.block / 32)) shape = t;
        }
    }
    *out = shape;
    return cudaSuccess;
}

// Returns cudaSuccess and sets *fits = false when m does not fit in shared memory.
// kinds[f-1]: team shape for family f (TeamShape), or -1 for the default
// rule: teams of 2 warps when 16 warps per SM fit, else warp teams when 12
// fit, else CTA teams of 8 (the autotuner picks among all shapes).
inline cudaError_t plan_batch(int sm_count, int precision, uint32_t m, const int32_t *variants, int nv,
                              int64_t num_sets, const int *kinds, Plan *out, bool *fits) {
    const bool f32 = precision == PMH_FP32_RECHECK;
    int64_t per_fam[4] = {0, 0, 0, 0};
    for (int v = 0; v < nv; v++) per_fam[family_of(variants[v]) - 1] += num_sets;
    out->nfam = 0;
    *fits = true;
    int64_t base = 0;
    for (int f = 1; f <= 4; f++) {
        const int64_t items = per_fam[f - 1];
        if (items == 0) continue;
        LaunchShape shape{};
        cudaError_t e;
        const int want = kinds ? kinds[f - 1] : -1;
        if (want >= 0 && want < kNumShapes) {
            e = sketch_shape_any(f32, f, want, m, &shape);
            if (e != cudaSuccess) return e;
        }
        if (shape.blocks_per_sm <= 0) {
            e = default_shape(f32, f, m, &shape);
            if (e != cudaSuccess) return e;
        }
        if (shape.blocks_per_sm <= 0) { *fits = false; return cudaSuccess; }
        int grid = sm_count * shape.blocks_per_sm;
        const int teams_per_block = shape.block / 32 / shape.team_warps;
        const int64_t blocks_needed = (items + teams_per_block - 1) / teams_per_block;
        if (blocks_needed < grid) grid = (int)std::max<int64_t>(1, blocks_needed);
        const int j = out->nfam++;
        out->fam[j] = f;
        out->qbase[j] = base;
        out->qlen[j] = items;
        out->shape[j] = shape;
        out->grid[j] = grid;
        LaunchShape gs{};
        e = grid_shape_any(f32, f, m, &gs);
        if (e != cudaSuccess) return e;
        out->gshape[j] = gs;
        out->ggrid[j] = sm_count * gs.blocks_per_sm;
        // the FP64 redo kernel: one block per SM at most (redone items are rare), none when it does not fit
        LaunchShape rs{};
        if (f32) {
            e = default_shape(false, f, m, &rs);
            if (e != cudaSuccess) return e;
        }
        out->rshape[j] = rs;
        out->rgrid[j] = rs.blocks_per_sm > 0 ? sm_count : 0;
        base += items;
    }
    return cudaSuccess;
}

// Enqueues queue build, set statistics and one persistent kernel per family
// on `st`.  `ev` (optional) receives records before the queue build, before
// the sketch kernels and after them; `fam_ev` (optional) one record after
// each family's kernels, in plan order.
// Streams and events that let the family kernels of one call run side by side
// (forked from and joined back into the caller's stream), so that the SMs one
// family's kernel leaves idle in its tail start the next family's items.
struct FamilyFork {
    cudaStream_t s[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[4] = {nullptr, nullptr, nullptr, nullptr};
};

// Prefilter lists of a call (list == null: none): list_cap entries, list_n and sel of num_sets
// entries, for the sets of list_min..list_max elements.
struct ListSpec {
    ulonglong2 *list = nullptr;
    uint32_t *list_n = nullptr;
    uint32_t *sel = nullptr;
    int64_t list_cap = 0, list_min = 0, list_max = 0;
};

inline cudaError_t enqueue_batch(SketchParams p, const Plan &plan, int precision, int sm_count, uint64_t *queue,
                                 uint64_t *redo, unsigned int *qmeta, SetStat *stats, cudaStream_t st, cudaEvent_t *ev,
                                 cudaEvent_t *fam_ev = nullptr, const FamilyFork *ff = nullptr,
                                 const ListSpec &ls = ListSpec()) {
    const int64_t items = p.num_sets * p.num_variants;
    FamOfVariant fv{};
    for (int v = 0; v < p.num_variants; v++) fv.f[v] = family_of(p.variants[v]);
    const int qb = 256;
    int qg = (int)std::min<int64_t>((items + qb - 1) / qb, (int64_t)sm_count * 8);
    if (qg < 1) qg = 1;
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(qmeta, 0, kQMetaClearWords * sizeof(unsigned int), st)) != cudaSuccess) return e;
    queue_count<<<qg, qb, 0, st>>>(p.offsets, p.num_sets, p.num_variants, fv, qmeta);
    queue_starts<<<1, 32, 0, st>>>(qmeta);
    if (p.gctl && (e = cudaMemsetAsync(p.gctl, 0, sizeof(unsigned int) * 4, st)) != cudaSuccess) return e;
    queue_scatter<<<qg, qb, 0, st>>>(p.offsets, p.num_sets, p.num_variants, fv, qmeta, queue, p.gctl, p.grid_min);
    if (p.gctl) grid_init_kernel<<<4 * kMaxGrid, 256, 0, st>>>(p.gctl, p.gstate, p.gsig, p.m, precision == PMH_FP32_RECHECK);
    const int sg = (int)std::max<int64_t>(1, std::min<int64_t>(p.num_sets, (int64_t)sm_count * 8));
    set_stats_kernel<<<sg, 256, 0, st>>>(p.offsets, p.weights, p.num_sets, stats, qmeta);
    set_stats_big_kernel<<<sm_count * 8, 256, 0, st>>>(p.offsets, p.weights, stats, qmeta);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    p.stats = stats;
    // the prefilter pass counts as sketching work: it runs after the second event
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    p.list = nullptr;
    p.list_n = nullptr;
    if (kListing && ls.list && ls.list_n && ls.sel && p.rounds > 0) {
        const int lg = (int)std::max<int64_t>(1, std::min<int64_t>((p.num_sets + 255) / 256, (int64_t)sm_count * 8));
        list_select<<<lg, 256, 0, st>>>(p.offsets, p.num_sets, ls.sel, ls.list_n, ls.list_min, ls.list_max, qmeta);
        list_kernel<<<sm_count * (1024 / kListBlock), kListBlock, 0, st>>>(p, ls.list, ls.list_n, ls.sel, ls.list_cap, qmeta);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        p.list = ls.list;
        p.list_n = ls.list_n;
    }
    const bool forked = ff && plan.nfam > 1;
    if (forked) {
        if ((e = cudaEventRecord(ff->fork, st)) != cudaSuccess) return e;
        for (int j = 0; j < plan.nfam; j++)
            if ((e = cudaStreamWaitEvent(ff->s[j], ff->fork, 0)) != cudaSuccess) return e;
    }
    const bool f32 = precision == PMH_FP32_RECHECK;
    for (int j = 0; j < plan.nfam; j++) {
        cudaStream_t sj = forked ? ff->s[j] : st;
        const int f = plan.fam[j];
        SketchParams pj = p;
        pj.queue = queue + plan.qbase[j];
        pj.queue_len = plan.qlen[j];
        pj.head = qmeta + kQHead + (f - 1);
        if (f32 && redo && plan.rgrid[j] > 0) {
            pj.redo = redo + plan.qbase[j];
            pj.redo_count = qmeta + kQRedoCount + (f - 1);
            pj.redo_cap = plan.qlen[j];
        }
        e = sketch_launch_any(f32, f, plan.shape[j], plan.grid[j], pj, sj);
        if (e != cudaSuccess) return e;
        if (pj.gctl && plan.ggrid[j] > 0) {
            e = grid_launch_any(f32, f, plan.gshape[j], plan.ggrid[j], pj, sj);
            if (e != cudaSuccess) return e;
        }
        if (pj.redo) {
            // items whose contender log overflowed, sketched again in FP64 (the list is usually empty)
            SketchParams pr = pj;
            pr.queue = pj.redo;
            pr.queue_len = pj.redo_cap;
            pr.queue_len_dev = pj.redo_count;
            pr.head = qmeta + kQRedoHead + (f - 1);
            pr.redo = nullptr;
            pr.redo_count = nullptr;
            pr.redo_cap = 0;
            e = sketch_launch_any(false, f, plan.rshape[j], plan.rgrid[j], pr, sj);
            if (e != cudaSuccess) return e;
        }
        if (fam_ev && (e = cudaEventRecord(fam_ev[j], sj)) != cudaSuccess) return e;
    }
    if (forked) {
        for (int j = 0; j < plan.nfam; j++) {
            if ((e = cudaEventRecord(ff->join[j], ff->s[j])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, ff->join[j], 0)) != cudaSuccess) return e;
        }
    }
    if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Work-only parameters of a sketch call: first-round threshold
// T = m (ln m + t_c) / sum(w) (t_c_grid for grid items), number of finite
// threshold rounds, and the set size from which grid mode is used (<= 0: off).
struct Thresholds {
    double t_c = 3.0;          // measured on c2 with the prefilter: 3: 19.35, 4: 19.73, 5: 20.21 ms per step
    double t_c_grid = 8.0;
    int rounds = 5;
    int64_t grid_min = kGridMinDefault;
    uint32_t cap_points = 0;   // points per element in warp-cooperative expansion (0: 64 m ln(m+1) + 4096)
    int max_cont = -1;         // contender records per team / grid item (-1: kMaxCont / kGridCont)
    bool te_rej = false;       // ProbMinHash3/3a/4: Exp(lambda;0,1) by the rejection sampler instead of inversion
    // prefilter lists for sets of at least list_factor * m (ln m + t_c) elements (<= 0: off) and at most
    // list_max (one block of the prefilter kernel hashes a whole set)
    double list_factor = 2.0;   // measured on c2: 1.5 19.93, 2.0 19.86, 2.5 20.04, 3.5 20.58 ms per step
    int64_t list_max = 262144;
};

// Kernel launches of one enqueue_batch call (fixed by the plan).
inline int launch_count(const Plan &plan, bool grid, bool redo, bool listed = false) {
    int n = 5 + plan.nfam + (grid ? 1 : 0) + (listed ? 2 : 0);
    for (int j = 0; j < plan.nfam; j++) n += ((grid && plan.ggrid[j] > 0) ? 1 : 0) + ((redo && plan.rgrid[j] > 0) ? 1 : 0);
    return n;
}

// Fills the fields of SketchParams common to both entry points.
inline void fill_params(SketchParams *p, const uint64_t *ids, const double *weights, const int64_t *offsets,
                        int64_t num_sets, uint32_t m, const int32_t *variants, int32_t nv, uint64_t seed,
                        uint64_t *out_ids, double *out_q, int32_t *set_status, uint64_t *counters, const Thresholds &th) {
    std::memset(p, 0, sizeof(*p));
    p->ids = ids;
    p->weights = weights;
    p->offsets = offsets;
    p->num_sets = num_sets;
    p->m = m;
    p->mixed_seed = host_mix64(seed);
    for (int v = 0; v < nv; v++) p->variants[v] = variants[v];
    p->num_variants = nv;
    p->out_ids = out_ids;
    p->out_q = out_q;
    p->status = set_status;
    p->counters = (unsigned long long *)counters;
    p->t_factor = (float)(std::log((double)m) + th.t_c);
    p->rounds = th.rounds;
    p->cap_points = th.cap_points ? th.cap_points : (uint32_t)(64.0 * m * std::log((double)m + 1.0)) + 4096;
    p->max_cont = th.max_cont < 0 ? kMaxCont : std::min(th.max_cont, kMaxCont);
    p->max_cont_grid = th.max_cont < 0 ? kGridCont : std::min(th.max_cont, kGridCont);
    p->redo = nullptr;
    p->redo_count = nullptr;
    p->redo_cap = 0;
    p->queue_len_dev = nullptr;
    p->te_rej = th.te_rej;
    p->t_factor_grid = (float)(std::log((double)m) + th.t_c_grid);
    p->grid_min = th.grid_min;
    p->gctl = nullptr;
    p->gstate = nullptr;
    p->gsig = nullptr;
}

// Device bytes of the grid-mode workspace for signature size m.
inline size_t grid_scratch_bytes(uint32_t m) {
    return align16(sizeof(GridCtl)) + align16(sizeof(GridState) * 4 * kMaxGrid) + (size_t)4 * kMaxGrid * m * 16;
}
inline void bind_grid_scratch(SketchParams *p, void *base) {
    unsigned char *b = (unsigned char *)base;
    p->gctl = (GridCtl *)b;
    p->gstate = (GridState *)(b + align16(sizeof(GridCtl)));
    p->gsig = b + align16(sizeof(GridCtl)) + align16(sizeof(GridState) * 4 * kMaxGrid);
}

}  // namespace pmh
