// Persistent ProbMinHash sketch kernel (template over precision, team shape
// and algorithm family).
//
// GPU design (replaces the paper's sequential element loop, Algorithm
// "Basic structure of ProbMinHash algorithms"):
//   * A team (one warp, or a whole CTA) owns one work item = (set, variant) at
//     a time; its signature lives in shared memory.  Items come from a global
//     queue, one segment per family, ordered by decreasing set size; each
//     family has its own persistent kernel so a launch carries only that
//     family's code.
//   * Threshold rounds.  The sequential algorithm lets q_max fall element by
//     element; a data-parallel pass cannot wait for that.  Round r instead
//     stops every element at min(T*4^r, q_max) with T = m(ln m + c)/sum(w):
//     the merged point process of the set has density sum(w), so all m labels
//     have appeared below T except with probability ~e^-c (coupon collector).
//     Every point <= the final q_max is still generated (q_max only decreases),
//     so the signature is exactly that of the paper; a round that leaves a
//     component empty is repeated with a larger T (offers are idempotent), and
//     the last round has T = +inf.  sum(w) comes from a per-set statistics
//     kernel that runs once per set for all variants.
//   * Filter: each lane takes two elements per step and rejects the first
//     point without a logarithm (Exp(1) >= U, Exp(lambda;0,1) >=
//     U(1-e^-lambda)/lambda).  Survivors are compacted into a per-warp buffer
//     and expanded lane-sequentially with work stealing: each lane owns one
//     element and computes one point of it per step (the uncorrelated running
//     sum of Eq. uncorrelated_recursion term by term; the lazy Fisher-Yates
//     permutation of Algorithm "Lazy generation of random permutation
//     elements" through a per-lane write list).  Elements with long sequences
//     are expanded warp-cooperatively instead (deep mode): 32 points per step,
//     a warp scan of the spacings, and 32 Fisher-Yates steps resolved at once
//     with match/shuffle.
//   * q_max (Sec. Stop Limit Update) is a warp max-reduction over the shared
//     signature, refreshed after updates, instead of the binary tree.
//   * FP64 path: each component holds (q, id), updated with a 128-bit CAS
//     (lexicographic minimum).
//   * FP32 path: each component holds key = (float bits of x32 << 32 | element
//     index), updated with a 64-bit atomicMin.  Whenever an offer lands within
//     the error bound of the holder, both are logged as contenders; the true
//     minimum is always the final holder or a logged contender, and the
//     contenders are re-evaluated exactly in FP64 at the end of the item.
#pragma once

#include "pmh_device.cuh"
#include "../../include/pmh.h"

namespace pmh {

constexpr int kMaxCont = 64;       // contender records per team (overflow: the item is redone in FP64)
constexpr int kCasLimit = 1 << 16; // CAS retries per offer (each failure means another offer succeeded)
constexpr int kSurvCap = 128;      // survivor buffer per warp: < 64 left over + <= 64 new per filter step
#ifndef PMH_SURV_BATCH
#define PMH_SURV_BATCH 64
#endif
constexpr int kSurvBatch = PMH_SURV_BATCH;   // survivors expanded together (keeps the lanes of the expansion busy)
static_assert(kSurvBatch >= 1 && kSurvBatch <= 64, "the buffer holds < kSurvBatch left over + 64 new");

struct __align__(16) Rec64 {
    double q;
    unsigned long long id;
};

// Grid mode: items of sets with at least SketchParams::grid_min elements are
// processed by every CTA of a launch, each CTA with its own shared signature,
// merged into a global one per item.  With 16-byte aligned inputs every warp
// claims runs of 128-element blocks (grid_pass); otherwise the CTAs take chunks
// of kGridChunkMin..kGridChunk elements, about four per CTA (run_range).
constexpr int64_t kGridMinDefault = 1ll << 20;
constexpr uint32_t kGridChunk = 1u << 16;
constexpr uint32_t kGridChunkMin = 1u << 11;
constexpr int kMaxGrid = 16;            // grid items per family and call (further ones use one team)
constexpr int kGridCont = 1024;         // contender records per grid item
constexpr uint64_t kSkipBit = 1ull << 63;   // queue entry taken by grid mode

struct GridState {
    unsigned int next_chunk;       // next chunk (general pass) or 128-element block (aligned inputs) to claim
    unsigned int done;             // CTAs finished with the item
    unsigned int bound32;          // shared stop bound (float bits, scaled)
    int status;
    unsigned long long bound64;    // FP64 path: shared stop bound (double bits)
    int cont_n;
    int redo;                      // a CTA's contender log overflowed: the item goes to the FP64 redo
    unsigned int cont_k[kGridCont];
    unsigned int cont_e[kGridCont];
};

struct GridCtl {
    unsigned int count[4];         // grid-eligible items per family (entries beyond kMaxGrid stay in the team queue)
    unsigned long long list[4][kMaxGrid];
};

// Per-set statistics (one entry per set, computed once for all variants).
struct SetStat {
    double wsum;   // sum of the positive weights
    uint32_t npos; // elements with w > 0 (a set has < 2^32 elements)
    int bad;       // a weight is negative, NaN, infinite, or has no finite reciprocal
};

struct SketchParams {
    const uint64_t *ids;
    const double *weights;
    const int64_t *offsets;
    const SetStat *stats;
    int64_t num_sets;
    uint32_t m;
    uint64_t mixed_seed;          // mix64(seed)
    int32_t variants[PMH_MAX_VARIANTS];
    int32_t num_variants;
    Tables tab;
    uint64_t *out_ids;
    double *out_q;
    int32_t *status;
    unsigned long long *counters;
    const uint64_t *queue;        // this family's segment: (variant index << 40) | set index
    int64_t queue_len;
    unsigned int *head;           // next queue position of this family
    float t_factor;               // ln m + c
    int rounds;                   // finite-T rounds before the T = +inf round
    uint32_t cap_points;          // iteration cap (with replacement)
    int32_t max_cont;             // contender records kept per team (<= kMaxCont)
    int32_t max_cont_grid;        // contender records kept per grid item (<= kGridCont)
    // FP32 path: items whose contender log overflowed are listed here (this family's segment, of
    // redo_cap entries) and sketched again by the FP64 kernel; null: overflow fails the item
    uint64_t *redo;
    unsigned int *redo_count;
    int64_t redo_cap;
    const unsigned int *queue_len_dev;   // FP64 redo launch: the queue's length in device memory (else null)
    bool te_rej;                  // ProbMinHash3/3a/4: Exp(lambda;0,1) by the rejection sampler
    // grid mode (null when disabled)
    GridCtl *gctl;
    GridState *gstate;            // [4][kMaxGrid]
    void *gsig;                   // [4][kMaxGrid][m] records of 16 bytes
    float t_factor_grid;          // ln m + c for grid items (larger c: a failed round costs a full pass)
    int64_t grid_min;             // sets with at least this many elements use grid mode
    // Prefilter lists (null: none).  list_n[s] is kUnlisted, or the number of entries of set s
    // from list[(offsets[s] - offsets[0]) / 2]: the elements whose first point can pass the first
    // round's bound in some family, a superset of each variant's survivors (list_kernel).
    const ulonglong2 *list;
    const uint32_t *list_n;
};

constexpr uint32_t kUnlisted = 0xFFFFFFFFu;
// Prefilter lists need the filter that compares U against bound * w (PMH_FILTER_WS)
#ifndef PMH_FILTER_WS
#define PMH_FILTER_WS 1         // filter compares U against bound * w (no reciprocal for rejected elements)
#endif
constexpr bool kListing = PMH_FILTER_WS != 0;

// Threshold of the first round of an item: T = m t_factor / wsum = t_s 2^-sigma with t_s in
// [1, 2), or t_s = +inf and sigma = 0 (a single unbounded round) when the sum gives no usable
// estimate.  The sketch kernels and the prefilter take it from here alike.
__device__ __forceinline__ void first_threshold(uint32_t m, float t_factor, double wsum, uint32_t npos, float *t_s,
                                                int *sigma) {
    *sigma = 0;
    *t_s = __int_as_float(0x7F800000);
    const double T = (double)m * (double)t_factor / wsum;
    if (npos > 0 && T > 0.0 && T < 1e300) {
        int ex;
        const double fr = frexp(T, &ex);      // T = fr * 2^ex, fr in [0.5, 1)
        *t_s = (float)(2.0 * fr);
        *sigma = -(ex - 1);
    }
}

struct TeamShared {
    int item_idx;
    int unfilled;
    int status;
    int cont_n;
    int redo;           // FP32: the item was handed to the FP64 redo (outputs are written there)
    float bound32;      // stop bound in scaled FP32 units (x * 2^sigma)
    int sigma;
    double bound64;     // FP64 path: exact stop bound
    float t_s;          // T * 2^sigma
    unsigned long long next;   // next unclaimed element of the current pass (warps claim 64 at a time)
    uint32_t cont_k[kMaxCont];
    uint32_t cont_e[kMaxCont];
};

struct WarpShared {
    unsigned long long cnt[PMH_NUM_COUNTERS];   // work counters of this warp (lane 0 adds)
    int dq_n;                  // deep-mode queue length (the queue reuses sb_e, see process_survivors)
    int slot[32];              // Fisher-Yates scratch (deep mode)
    uint32_t sb_e[32 + kSurvCap];   // prefilter survivors: element index, from sb_e[32] (deep queue from sb_e[0])
    uint64_t sb_key[kSurvCap]; //   stream key
    float sb_winv[kSurvCap];   //   and scaled FP32 weight (its reciprocal once the batch is expanded)
    int sb_n;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// ProbMinHash2/4 per-warp region, used in turn by the two expansion modes:
// the per-lane Fisher-Yates write lists of lane-sequential expansion
// (kFyCap x 32 x u32, live while a lane walks one element) and the dense
// permutation of deep mode (m x u16, rebuilt for every element it expands).
// A warp runs its deep elements only after its lane-sequential loop has ended,
// so the two share the bytes.
constexpr int kFyCap = 16;
__host__ __device__ inline size_t perm_bytes(uint32_t m) {
    const size_t dense = align16((size_t)m * 2), lists = (size_t)kFyCap * 32 * 4;
    return dense > lists ? dense : lists;
}

struct SmemLayout {
    size_t team_off, sig_off, warp_off, perm_off, total;
    __host__ __device__ SmemLayout(int teams, int warps, uint32_t m, bool f32, bool perm) {
        team_off = 0;
        sig_off = align16(team_off + (size_t)teams * align16(sizeof(TeamShared)));
        warp_off = align16(sig_off + (size_t)teams * m * (f32 ? 8 : 16));
        perm_off = align16(warp_off + (size_t)warps * align16(sizeof(WarpShared)));
        total = align16(perm_off + (perm ? (size_t)warps * perm_bytes(m) : 0));
    }
};

// ------------------------------------------------------------------------
// Per-item context (registers).
template <bool F32>
struct Ctx {
    const SketchParams *p;
    TeamShared *ts;
    void *sig;
    WarpShared *ws;
    uint16_t *perm;     // this warp's permutation array (ProbMinHash2/4), else null
    uint32_t *fy;       // this warp's Fisher-Yates write lists [kFyCap][32] (ProbMinHash2/4)
    int64_t beg;
    int64_t off0;       // offsets[0] of the call (prefilter list positions count from it)
    uint32_t n;
    int sigma;
    unsigned int *gbound32;        // grid mode: the item's bound shared by all CTAs (float bits), else null
    unsigned long long *gbound64;  //   and its FP64 bound (double bits)
    bool unw;                      // binary-weight variant: w_inv = 1, uniform variates, gamma_i = i
    bool rej;                      // weighted ProbMinHash3/3a/4 with Exp(lambda;0,1) by the rejection sampler
};

__device__ __forceinline__ float ld_volatile(const float *p) { return *(volatile const float *)p; }
__device__ __forceinline__ double ld_volatile(const double *p) { return *(volatile const double *)p; }
__device__ __forceinline__ int ld_volatile(const int *p) { return *(volatile const int *)p; }
__device__ __forceinline__ uint64_t ld_volatile(const uint64_t *p) { return *(volatile const uint64_t *)p; }

__device__ __forceinline__ void atomic_min_pos_float(float *addr, float v) {
    atomicMin((int *)addr, __float_as_int(v));   // positive floats order like their bit patterns
}
__device__ __forceinline__ void atomic_min_pos_double(double *addr, double v) {
    atomicMin((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}
// Warp-uniform counter update (lane 0 adds; nothing when the call has no counters).
template <bool F32>
__device__ __forceinline__ void count(Ctx<F32> &c, int idx, unsigned long long v) {
    if (c.p->counters && (threadIdx.x & 31) == 0) c.ws->cnt[idx] += v;
}
__device__ __forceinline__ unsigned popc_ballot(bool b) { return __popc(__ballot_sync(kFull, b)); }
// Per-phase cycle counters (PMH_CNT_CYC_*): a diagnostic, compiled in only with
// PMH_CYCLE_COUNTERS=1.  The clock reads and the 64-bit stamps they keep live
// cost about 6 % of the sketch kernels' time on c2 (more register spills).
#ifndef PMH_CYCLE_COUNTERS
#define PMH_CYCLE_COUNTERS 0
#endif
__device__ __forceinline__ long long cyc_now() {
#if PMH_CYCLE_COUNTERS
    return clock64();
#else
    return 0;
#endif
}
template <bool F32>
__device__ __forceinline__ void count_cyc(Ctx<F32> &c, int idx, long long t0) {
#if PMH_CYCLE_COUNTERS
    count(c, idx, (unsigned long long)(clock64() - t0));
#else
    (void)c; (void)idx; (void)t0;
#endif
}

// ------------------------------------------------------------ offers
template <bool F32> struct Offer;

template <> struct Offer<true> {
    // x32: scaled FP32 value, e: element index in the set.
    static __device__ __forceinline__ bool run(Ctx<true> &c, uint32_t k, float x32, uint32_t e) {
        uint64_t *sig = (uint64_t *)c.sig;
        uint64_t key = ((uint64_t)__float_as_uint(x32) << 32) | e;
        uint64_t cur = ld_volatile(&sig[k]);
        if (cur != kEmptyKey) {
            float xc = __uint_as_float((uint32_t)(cur >> 32));
            if (xc < x32 * (1.0f - 2.0f * kEta)) return false;   // loses and is not near
        }
        uint64_t old = atomicMin((unsigned long long *)&sig[k], (unsigned long long)key);
        if (old == kEmptyKey) {
            atomicSub(&c.ts->unfilled, 1);
            return true;
        }
        float xo = __uint_as_float((uint32_t)(old >> 32));
        // an element never contends with itself: h_k(e) is a single value, and its
        // re-offers (deep mode restarts from point 1, later rounds repeat) are idempotent
        if ((uint32_t)(old & 0xFFFFFFFFu) != e && fabsf(x32 - xo) <= kEta * (x32 + xo)) {
            int at = atomicAdd(&c.ts->cont_n, 2);
            if (at + 1 < c.p->max_cont) {
                c.ts->cont_k[at] = k;
                c.ts->cont_e[at] = e;
                c.ts->cont_k[at + 1] = k;
                c.ts->cont_e[at + 1] = (uint32_t)(old & 0xFFFFFFFFu);
            }
            atomicAdd(&c.ws->cnt[PMH_CNT_CONTENDERS], 1ull);
        }
        return key < old;
    }
};

template <> struct Offer<false> {
    static __device__ __forceinline__ bool run(Ctx<false> &c, uint32_t k, double x, uint64_t id) {
        Rec64 *sig = (Rec64 *)c.sig;
        double qc = ld_volatile(&sig[k].q);
        if (x > qc) return false;
        Rec64 expected;
        expected.q = qc;
        expected.id = ld_volatile((const uint64_t *)&sig[k].id);
        for (int it = 0; it < kCasLimit; ++it) {
            if (!(x < expected.q || (x == expected.q && id < expected.id))) return false;
            Rec64 desired;
            desired.q = x;
            desired.id = id;
            Rec64 old = atomicCAS(&sig[k], expected, desired);
            if (__double_as_longlong(old.q) == __double_as_longlong(expected.q) && old.id == expected.id) {
                if (isinf(old.q)) atomicSub(&c.ts->unfilled, 1);
                return true;
            }
            expected = old;
        }
        c.ts->status = PMH_ERR_ITER_LIMIT;
        return false;
    }
};

// ------------------------------------------------------------ q_max refresh
// Warp-wide maximum over the team's signature; lowers the shared bound.
template <bool F32>
__device__ void refresh_bound(Ctx<F32> &c) {
    const int lane = threadIdx.x & 31;
    const uint32_t m = c.p->m;
    const long long t0 = cyc_now();
    if constexpr (F32) {
        const uint64_t *sig = (const uint64_t *)c.sig;
        uint32_t mx = 0;
        for (uint32_t k = lane; k < m; k += 32) mx = max(mx, (uint32_t)(ld_volatile(&sig[k]) >> 32));
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        if (lane == 0 && mx != 0xFFFFFFFFu) atomic_min_pos_float(&c.ts->bound32, __uint_as_float(mx) * (1.0f + 2.0f * kEta));
    } else {
        const Rec64 *sig = (const Rec64 *)c.sig;
        double mx = 0.0;
        for (uint32_t k = lane; k < m; k += 32) mx = fmax(mx, ld_volatile(&sig[k].q));
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        if (lane == 0 && !isinf(mx)) {
            atomic_min_pos_double(&c.ts->bound64, mx);
            atomic_min_pos_float(&c.ts->bound32, __double2float_ru(ldexp(mx, c.sigma)));
        }
    }
    count_cyc(c, PMH_CNT_CYC_REFRESH, t0);
}

// ------------------------------------------------------------ Fisher-Yates group
// 32 consecutive steps t0..t0+31 (0-based) of the lazy permutation of one
// element, whose state before the group is perm[t0..m).  Step t draws
// r_t = t + floor(L * (m-t) / 2^64), returns label P[r_t] and sets P[r_t] = P[t]
// (Algorithm "Lazy generation of random permutation elements", 0-based).
// In-group dependencies: the value at position p before step t is the value
// moved there by the latest earlier step u with r_u = p, else perm[p]; chains
// of such moves are resolved by pointer jumping over lanes.  A step never
// targets the position of an earlier step (r_u >= u), so the latest earlier
// writer of position t0 + j is the highest lane below j among the lanes that
// target it.
__device__ __forceinline__ uint32_t fy_group(uint16_t *perm, int *slot, uint32_t m, uint32_t t0, uint64_t lw, bool act) {
    const int lane = threadIdx.x & 31;
    const uint32_t t = t0 + lane;
    const uint32_t r = act ? t + uniform_int(lw, m - t) : 0xFFFFFFFFu;
    const uint32_t same = __match_any_sync(kFull, r);   // lanes with the same target
    slot[lane] = -1;
    __syncwarp();
    const uint32_t j = r - t0;                           // target inside the group: j in (lane, 32)
    if (act && j < 32u && j != (uint32_t)lane) {
        const uint32_t below = same & ((1u << j) - 1u);
        if (lane == 31 - __clz(below)) slot[j] = lane;
    }
    __syncwarp();
    int ptr = act ? slot[lane] : -1;
    uint32_t val = (act && ptr < 0) ? (uint32_t)perm[t] : 0u;
    // chains are short: most groups need no jump at all
    for (int it = 0; it < 5 && __any_sync(kFull, ptr >= 0); ++it) {
        int src = ptr >= 0 ? ptr : lane;
        uint32_t v2 = __shfl_sync(kFull, val, src);
        int p2 = __shfl_sync(kFull, ptr, src);
        if (ptr >= 0) {
            if (p2 < 0) { val = v2; ptr = -1; } else ptr = p2;
        }
    }
    const uint32_t moved = val;   // value at position t just before step t
    const uint32_t earlier = same & ((1u << lane) - 1u);
    const int w2 = earlier ? 31 - __clz(earlier) : -1;
    const uint32_t from_lane = __shfl_sync(kFull, moved, w2 >= 0 ? w2 : lane);
    uint32_t label = 0;
    if (act) label = (w2 >= 0) ? from_lane : (uint32_t)perm[r];
    const uint32_t later = (lane == 31) ? 0u : (same & ~((2u << lane) - 1u));
    __syncwarp();
    if (act && later == 0 && r >= t0 + 32) perm[r] = (uint16_t)moved;
    __syncwarp();
    return label;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src);
    uint32_t hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ double shfl_d(double v, int src) {
    return __longlong_as_double((long long)shfl64((uint64_t)__double_as_longlong(v), src));
}

// ------------------------------------------------------------ deep mode
// Warp-cooperative expansion of one element from point 1, 32 points per step.
// EXACT = false: offer points <= bound.  EXACT = true (exact search): stop at
// the first point with label `want` and return its canonical FP64 value.
template <int FAM, bool F32, bool EXACT, bool REJ>
__device__ double deep(Ctx<F32> &c, uint32_t e, uint32_t want) {
    const SketchParams &P = *c.p;
    const Tables &T = P.tab;
    const uint32_t m = P.m;
    const int lane = threadIdx.x & 31;
    const uint64_t id = P.ids[c.beg + e];
    const double w = P.weights[c.beg + e];
    const uint64_t key = mix64(id ^ P.mixed_seed);
    const double w_inv = (EXACT || !F32) ? (c.unw ? 1.0 : __drcp_rn(w)) : 0.0;
    const float winv32 = winv_scaled(c.unw ? 1.0 : w, c.sigma);
    if (FAM == 2 || FAM == 4) {
        // identity permutation, eight 16-bit entries per 16-byte store (the region
        // holds align16(2m) bytes, so the last store stays inside it)
        uint4 *p4 = (uint4 *)c.perm;
        for (uint32_t q = lane; q * 8 < m; q += 32) {
            const uint32_t a = q * 8;
            p4[q] = make_uint4(a | (a + 1) << 16, (a + 2) | (a + 3) << 16, (a + 4) | (a + 5) << 16, (a + 6) | (a + 7) << 16);
        }
        __syncwarp();
    }
    if (!EXACT) count(c, PMH_CNT_DEEP, 1);
    double carry64 = 0.0;
    float c_hi = 0.0f, c_lo = 0.0f;
    bool refreshed = false;
    const uint32_t limit = (FAM == 2 || FAM == 4) ? m : P.cap_points;
#pragma unroll 1
    for (uint32_t base = 1;; base += 32) {
        if (base > limit) {
            if (FAM == 1 || FAM == 3) { if (lane == 0) c.ts->status = PMH_ERR_ITER_LIMIT; }
            return __longlong_as_double(0x7FF0000000000001ll);
        }
        // correlated: the group starts beyond the bound?
        if (!EXACT && FAM >= 3) {
            bool stop;
            if constexpr (F32) {
                float lb = (FAM == 3 || c.unw) ? winv32 * (float)(base - 1) : winv32 * T.gamma32[base - 1];
                stop = lb * (1.0f - kEta) > ld_volatile(&c.ts->bound32);
            } else {
                double lb = (FAM == 3 || c.unw) ? lower3_64(base, w_inv) : lower4_64(T, base, w_inv);
                stop = lb > ld_volatile(&c.ts->bound64);
            }
            if (__shfl_sync(kFull, (int)stop, 0)) return 0.0;
        }
        const uint32_t i = base + lane;
        const bool act = i <= limit;
        const uint64_t vw = act ? value_word(key, i) : 0;
        const uint64_t lw = act ? label_word(key, i) : 0;
        uint32_t k;
        if (FAM == 1 || FAM == 3) k = uniform_int(lw, m);
        else k = fy_group(c.perm, c.ws->slot, m, base - 1, lw, act);
        if constexpr (EXACT) {
            const unsigned hit = __ballot_sync(kFull, act && k == want);
            // canonical FP64 values of this group (the uncorrelated families need the carry)
            double x = 0.0;
            if (FAM == 1 || FAM == 2) {
                double t = act ? (FAM == 1 ? term1_64(vw, w_inv) : term2_64(T, vw, i, w_inv)) : 0.0;
                double run = carry64;
                for (int s = 0; s < 32; ++s) {
                    double ts = __shfl_sync(kFull, t, s);
                    run = __dadd_rn(run, ts);
                    if (lane == s) x = run;
                }
                carry64 = run;
            } else if (hit) {
                int src = __ffs(hit) - 1;
                if (lane == src) x = c.unw ? point_unw_64(vw, i, w_inv)
                                     : (REJ && c.rej) ? ((FAM == 3) ? point3r_64(T, key, vw, i, w_inv) : point4r_64(T, key, vw, i, w_inv))
                                           : (FAM == 3) ? point3_64(T, vw, i, w_inv) : point4_64(T, vw, i, w_inv);
            }
            if (hit) return __shfl_sync(kFull, x, __ffs(hit) - 1);
            continue;
        }
        bool last_beyond, any_win;
        if constexpr (F32) {
            float x32;
            if (FAM == 1 || FAM == 2) {
                float t = act ? (FAM == 1 ? exp1_32(vw) : __fmul_rn(T.beta32[i], exp1_32(vw))) : 0.0f;
                float s = t;
                for (int o = 1; o < 32; o <<= 1) {
                    float y = __shfl_up_sync(kFull, s, o);
                    if (lane >= o) s = __fadd_rn(s, y);
                }
                x32 = __fmul_rn(winv32, __fadd_rn(c_hi, __fadd_rn(c_lo, s)));
                // error-free carry (TwoSum): c_hi + c_lo = sum of all earlier groups exactly
                float tot = __shfl_sync(kFull, s, 31);
                float sh = __fadd_rn(c_hi, tot);
                float bb = __fsub_rn(sh, c_hi);
                float err = __fadd_rn(__fsub_rn(c_hi, __fsub_rn(sh, bb)), __fsub_rn(tot, bb));
                c_hi = sh;
                c_lo = __fadd_rn(c_lo, err);
            } else if (c.unw) {
                x32 = act ? __fmul_rn(winv32, __fadd_rn((float)(i - 1), u53_to_float(vw >> 11))) : 0.0f;
            } else if (FAM == 3) {
                const float te = (REJ && c.rej) ? texp_rej_32(T, 1, key, i, vw) : texp_32(vw, T.c3_32, T.inv3_32);
                x32 = act ? __fmul_rn(winv32, __fadd_rn((float)(i - 1), te)) : 0.0f;
            } else {
                float sv = 0.0f;
                if (act) {
                    const float4 q = T.p4[i];
                    if (i < m) sv = __fadd_rn(q.x, __fmul_rn(q.y, (REJ && c.rej) ? texp_rej_32(T, i, key, i, vw) : texp_32(vw, q.z, q.w)));
                    else sv = __fadd_rn(q.x, __fmul_rn(T.delta32, exp1_32(vw)));
                }
                x32 = __fmul_rn(winv32, sv);
            }
            if (P.counters) count(c, PMH_CNT_POINTS32, popc_ballot(act));
            const bool beyond = x32 * (1.0f - kEta) > ld_volatile(&c.ts->bound32);
            bool wi = false;
            if (act && !beyond) wi = Offer<true>::run(c, k, x32, e);
            any_win = __any_sync(kFull, wi);
            last_beyond = __shfl_sync(kFull, (int)beyond, (int)min((uint32_t)31, limit - base));
        } else {
            double x;
            if (FAM == 1 || FAM == 2) {
                double t = act ? (FAM == 1 ? term1_64(vw, w_inv) : term2_64(T, vw, i, w_inv)) : 0.0;
                double run = carry64;
                x = 0.0;
                for (int s = 0; s < 32; ++s) {   // canonical left-to-right sum
                    double ts = __shfl_sync(kFull, t, s);
                    run = __dadd_rn(run, ts);
                    if (lane == s) x = run;
                }
                carry64 = run;
            } else if (c.unw) {
                x = act ? point_unw_64(vw, i, w_inv) : 0.0;
            } else if (FAM == 3) {
                x = act ? ((REJ && c.rej) ? point3r_64(T, key, vw, i, w_inv) : point3_64(T, vw, i, w_inv)) : 0.0;
            } else {
                x = act ? ((REJ && c.rej) ? point4r_64(T, key, vw, i, w_inv) : point4_64(T, vw, i, w_inv)) : 0.0;
            }
            if (P.counters) count(c, PMH_CNT_POINTS64, popc_ballot(act));
            const bool beyond = x > ld_volatile(&c.ts->bound64);
            bool wi = false;
            if (act && !beyond) wi = Offer<false>::run(c, k, x, id);
            any_win = __any_sync(kFull, wi);
            last_beyond = __shfl_sync(kFull, (int)beyond, (int)min((uint32_t)31, limit - base));
        }
        if (base + 31 >= limit && (FAM == 2 || FAM == 4)) return 0.0;
        if ((FAM == 1 || FAM == 2) && last_beyond) return 0.0;
        // keep q_max fresh while expanding: after groups that changed a minimum, and
        // once as soon as the signature is full (another warp of the team may have
        // filled it, and this element's later points may never win again)
        const int uf = __shfl_sync(kFull, lane == 0 ? ld_volatile(&c.ts->unfilled) : 1, 0);
        if (uf == 0 && (any_win || !refreshed)) {
            refresh_bound<F32>(c);
            refreshed = true;
        }
    }
}

// Exact FP64 value of h_k(e) (the first point of element e with label k).
// Cold path (contender resolution, exact q output): kept out of line.
template <int FAM, bool F32, bool REJ>
__device__ __noinline__ double exact_h(Ctx<F32> c, uint32_t e, uint32_t k) {
    return deep<FAM, F32, true, REJ>(c, e, k);
}

// FP32 path: re-evaluates every logged contender (and the holder of its
// component) exactly in FP64 and installs the lexicographic (value, id)
// minimum in `sig`.  Runs in one warp.  Returns the number of exact
// evaluations.
template <int FAM, bool REJ>
__device__ __noinline__ uint32_t resolve_list(Ctx<true> c, const uint32_t *ck, const uint32_t *ce, int ncont,
                                              uint64_t *sig) {
    const SketchParams &P = *c.p;
    const int lane = threadIdx.x & 31;
    uint32_t evals = 0;
    for (int a = 0; a < ncont; ++a) {
        const uint32_t k = ck[a];
        bool seen = false;
        for (int b = 0; b < a; ++b) seen |= (ck[b] == k);
        if (seen) continue;
        const uint64_t hk = ld_volatile(&sig[k]);
        uint32_t best_e = (uint32_t)(hk & 0xFFFFFFFFu);
        double best_x = exact_h<FAM, true, REJ>(c, best_e, k);
        uint64_t best_id = P.ids[c.beg + best_e];
        evals++;
        for (int b = a; b < ncont; ++b) {
            if (ck[b] != k) continue;
            const uint32_t e = ce[b];
            if (e == best_e) continue;
            double x = exact_h<FAM, true, REJ>(c, e, k);
            evals++;
            uint64_t cid = P.ids[c.beg + e];
            if (x < best_x || (x == best_x && cid < best_id)) { best_x = x; best_id = cid; best_e = e; }
        }
        if (lane == 0) sig[k] = (hk & 0xFFFFFFFF00000000ull) | best_e;
        __syncwarp();
    }
    return evals;
}

template <int FAM, bool REJ>
__device__ __forceinline__ uint32_t resolve_contenders(Ctx<true> &c) {
    TeamShared *ts = c.ts;
    const int ncont = min(ld_volatile(&ts->cont_n), c.p->max_cont);   // the caller redoes an item that overflowed
    return resolve_list<FAM, REJ>(c, ts->cont_k, ts->cont_e, ncont, (uint64_t *)c.sig);
}

// FP32 path: hands an item whose contender log overflowed to the FP64 kernel
// that runs after this family's kernels (its queue is the redo list).  Returns
// false when there is no list or it is full; the item then fails with
// PMH_ERR_ITER_LIMIT.  Called by one thread.
__device__ __forceinline__ bool push_redo(const SketchParams &P, int item_v, int64_t set) {
    if (!P.redo) return false;
    const unsigned int at = atomicAdd(P.redo_count, 1u);
    if ((int64_t)at >= P.redo_cap) return false;
    P.redo[at] = ((uint64_t)item_v << 40) | (uint64_t)set;
    return true;
}

// ------------------------------------------------------------ survivors
// Elements whose first point passed the log-free lower bound are expanded
// lane-sequentially with work stealing: every lane owns one survivor, computes
// one point of it per step (value word, label word, value, label, offer), and
// takes the next buffered survivor when its sequence ends.  Sequential
// per-lane sums follow the uncorrelated recursion exactly as written, and the
// lazy Fisher-Yates permutation of ProbMinHash2/4 keeps a per-lane list of its
// writes.  At the first point the number of further points below the bound is
// estimated:
//   ProbMinHash3: points i >= 2 with lower bound w_inv*(i-1) <= bound, i.e.
//     i-1 <= bound*w;
//   ProbMinHash4: lower bound w_inv*gamma_{i-1} with
//     gamma_j = log(m/(m-j))/lambda_1 <= bound*w, i.e. j <= m(1-e^{-lambda_1 bound w});
//   ProbMinHash1/2: after x_1 a Poisson count of mean w*(bound - x_1)
//     (ProbMinHash1's spacings are Exp(1)/w; ProbMinHash2's are longer).
// Long sequences go to warp-cooperative deep mode instead; so does a
// sequence that outgrows the lane-sequential cap (the FP32 running sum's error
// bound holds for at most kSeqCap terms, the write list has kFyCap entries).
// Tuning constants (compile-time; the defaults are the measured best on c2).
#ifndef PMH_PREF_STEPS
#define PMH_PREF_STEPS 0     // off: measured 1 % faster on c2 once the kernels became issue-bound
#endif
#ifndef PMH_SEQ_CAP
#define PMH_SEQ_CAP 32
#endif
#ifndef PMH_SEQ_CAP3
#define PMH_SEQ_CAP3 64
#endif
#ifndef PMH_SEQ_KEEP
#define PMH_SEQ_KEEP 8
#endif
#ifndef PMH_GRID_LEAN
#define PMH_GRID_LEAN 1         // grid mode: the trimmed filter pass (grid_pass) for 16-byte aligned inputs
#endif
#ifndef PMH_EST_SIGMAS
#define PMH_EST_SIGMAS 0.0f     // ProbMinHash1/2: deep mode when mean + this many sd of the point count (+2) reach the cap
#endif
#ifndef PMH_SEQ_KEEP_FAMS
#define PMH_SEQ_KEEP_FAMS 3     // families whose busy lanes carry over (bit f-1: ProbMinHash f); the measured best on c2
#endif
constexpr int kPrefSteps = PMH_PREF_STEPS;  // filter: L2 prefetch distance in 64-element steps of a warp (0: none)
constexpr int kSeqKeep = PMH_SEQ_KEEP;      // idle lanes at which a dry buffer hands the rest to the next call (0: never)
static_assert(kSeqKeep >= 0 && kSeqKeep <= 32, "a count of lanes");
constexpr int kSeqCap = PMH_SEQ_CAP;        // lane-sequential points (ProbMinHash1)
constexpr int kSeqCap3 = PMH_SEQ_CAP3;      // lane-sequential points (ProbMinHash3)
static_assert(kSeqCap <= 32, "the FP32 running-sum error bound holds for at most 32 terms");

// Lane-sequential state of one lane: the survivor it is expanding.  In the
// families that carry lanes over (PMH_SEQ_KEEP_FAMS: ProbMinHash1 and 2 by
// default) it outlives a call of process_survivors: when the buffer runs dry
// while a few lanes are still busy, those lanes keep their elements and resume
// them in the next call, together with the survivors that the filter buffered
// meanwhile (the bound only falls in between, so a resumed sequence stops no
// later than it would have).  ProbMinHash2/4 lanes keep their Fisher-Yates
// write lists in place meanwhile; since those share bytes with the deep-mode
// permutation, their deep queue waits for a call that ends with every lane
// idle.
template <bool F32>
struct SeqLane {
    bool has;
    uint32_t e, i;
    uint64_t key, id;
    float winv32, s32;
    double w_inv, x64;
    int fyn;
};

// Expands the n buffered survivors (ws->sb_e[32 + j], sb_key[j], sb_winv[j];
// the filter leaves w * 2^-sigma in sb_winv, replaced by its scaled reciprocal
// on entry).  fin: the last call of the pass (every sequence ends in it).
template <int FAM, bool F32, bool REJ>
__device__ __forceinline__ bool process_survivors(Ctx<F32> &c, SeqLane<F32> &L, int n, bool fin) {
    const long long t_sv = cyc_now();
    const SketchParams &P = *c.p;
    const Tables &T = P.tab;
    const uint32_t m = P.m;
    const int lane = threadIdx.x & 31;
    WarpShared *ws = c.ws;
    constexpr bool kPerm = (FAM == 2 || FAM == 4);
    constexpr int kCap = (FAM == 3) ? kSeqCap3 : (kPerm ? kFyCap : kSeqCap);   // the write list bounds ProbMinHash2/4
    constexpr bool kKeep = kSeqKeep > 0 && ((PMH_SEQ_KEEP_FAMS >> (FAM - 1)) & 1);
    bool won = false;
    int next = 0;
    uint32_t npts = 0;
    int nsteps = 0;
#if PMH_FILTER_WS
    // the filter buffered w * 2^-sigma: the scaled reciprocal weight of every new survivor
    for (int j = lane; j < n; j += 32) ws->sb_winv[j] = winv_from_ws(ws->sb_winv[j]);
    __syncwarp();
#endif
#pragma unroll 1
    for (;; ++nsteps) {
        // idle lanes take the next survivors
        const unsigned idle = __ballot_sync(kFull, !L.has);
        const int avail = n - next;
        if (avail > 0 && idle) {
            const int rank = __popc(idle & ((1u << lane) - 1u));
            if (!L.has && rank < avail) {
                const int j = next + rank;
                L.e = ws->sb_e[32 + j];
                L.key = ws->sb_key[j];
                L.winv32 = ws->sb_winv[j];
                if constexpr (!F32) {
                    L.w_inv = c.unw ? 1.0 : __drcp_rn(P.weights[c.beg + L.e]);
                    L.id = P.ids[c.beg + L.e];
                }
                L.i = 1;
                L.s32 = 0.0f;
                L.x64 = 0.0;
                L.fyn = 0;
                L.has = true;
            }
            next += min(__popc(idle), avail);
        } else if (kKeep && !fin && avail <= 0 && __popc(idle) >= kSeqKeep) {
            if (!kPerm) break;   // the buffer is dry: the busy lanes carry on in the next call
            __syncwarp();
            if (ld_volatile(&ws->dq_n) + 32 - __popc(idle) <= 32) break;
        }
        // every taken slot has been read.  The deep queue fills sb_e[0, 32 + next):
        // it holds at most one entry per survivor taken here or carried in (< 32),
        // plus, for ProbMinHash2/4, the entries left waiting (with the carried lanes <= 32)
        __syncwarp();
        if (!__any_sync(kFull, L.has)) break;
        if (L.has) {
            bool done = false, to_deep = false;
            // correlated families: point i lies above its lower bound
            if (FAM >= 3 && L.i >= 2) {
                if constexpr (F32) {
                    const float lb = (FAM == 3 || c.unw) ? L.winv32 * (float)(L.i - 1) : L.winv32 * T.p4[L.i].x;
                    done = lb * (1.0f - kEta) > ld_volatile(&c.ts->bound32);
                } else {
                    const double lb = (FAM == 3 || c.unw) ? lower3_64(L.i, L.w_inv) : lower4_64(T, L.i, L.w_inv);
                    done = lb > ld_volatile(&c.ts->bound64);
                }
            }
            if (!done) {
                const uint64_t vw = value_word(L.key, L.i);
                const uint64_t lw = label_word(L.key, L.i);
                uint32_t k;
                if constexpr (kPerm) {
                    // step t = i-1 of the lazy Fisher-Yates permutation; list entry = (position << 16) | value
                    const uint32_t t = L.i - 1;
                    const uint32_t r = t + uniform_int(lw, m - t);
                    uint32_t moved = t, lab = r;   // untouched positions hold their own index
                    // the latest write wins: one backward scan, keeping the first match of each
                    bool ft = false, fr = false;
                    for (int j = L.fyn - 1; j >= 0; --j) {
                        const uint32_t ent = c.fy[j * 32 + lane];
                        const uint32_t pos = ent >> 16;
                        if (!ft && pos == t) { moved = ent & 0xFFFFu; ft = true; }
                        if (!fr && pos == r) { lab = ent & 0xFFFFu; fr = true; }
                    }
                    if (L.fyn < kFyCap) c.fy[L.fyn * 32 + lane] = (r << 16) | moved;
                    L.fyn++;
                    k = lab;
                } else {
                    k = uniform_int(lw, m);
                }
                bool beyond;
                float y = 0.0f;
                if constexpr (F32) {
                    float x32;
                    if (FAM == 1) { L.s32 = __fadd_rn(L.s32, exp1_32(vw)); x32 = __fmul_rn(L.winv32, L.s32); }
                    else if (FAM == 2) { L.s32 = __fadd_rn(L.s32, __fmul_rn(T.beta32[L.i], exp1_32(vw))); x32 = __fmul_rn(L.winv32, L.s32); }
                    else if (c.unw) x32 = __fmul_rn(L.winv32, __fadd_rn((float)(L.i - 1), u53_to_float(vw >> 11)));
                    else if (FAM == 3) {
                        const float te = (REJ && c.rej) ? texp_rej_32(T, 1, L.key, L.i, vw) : texp_32(vw, T.c3_32, T.inv3_32);
                        x32 = __fmul_rn(L.winv32, __fadd_rn((float)(L.i - 1), te));
                    } else {
                        float sv;
                        const float4 q = T.p4[L.i];
                        if (L.i < m) sv = __fadd_rn(q.x, __fmul_rn(q.y, (REJ && c.rej) ? texp_rej_32(T, L.i, L.key, L.i, vw) : texp_32(vw, q.z, q.w)));
                        else sv = __fadd_rn(q.x, __fmul_rn(T.delta32, exp1_32(vw)));
                        x32 = __fmul_rn(L.winv32, sv);
                    }
                    const float b32 = ld_volatile(&c.ts->bound32);
                    beyond = x32 * (1.0f - kEta) > b32;
                    if (!beyond) won |= Offer<true>::run(c, k, x32, L.e);
                    if (L.i == 1) {
                        // bound * w (minus x_1 * w): only chooses the expansion mode, so approximate
                        y = __fdividef(b32, L.winv32);
                        if (FAM == 1 || FAM == 2) y -= L.s32;
                    }
                } else {
                    if (FAM == 1) L.x64 = __dadd_rn(L.x64, term1_64(vw, L.w_inv));
                    else if (FAM == 2) L.x64 = __dadd_rn(L.x64, term2_64(T, vw, L.i, L.w_inv));
                    else if (c.unw) L.x64 = point_unw_64(vw, L.i, L.w_inv);
                    else if (FAM == 3) L.x64 = (REJ && c.rej) ? point3r_64(T, L.key, vw, L.i, L.w_inv) : point3_64(T, vw, L.i, L.w_inv);
                    else L.x64 = (REJ && c.rej) ? point4r_64(T, L.key, vw, L.i, L.w_inv) : point4_64(T, vw, L.i, L.w_inv);
                    const double b64 = ld_volatile(&c.ts->bound64);
                    beyond = L.x64 > b64;
                    if (!beyond) won |= Offer<false>::run(c, k, L.x64, L.id);
                    if (L.i == 1)
                        y = (FAM == 1 || FAM == 2) ? (float)((b64 - L.x64) * (1.0 / L.w_inv))
                                                   : __fdiv_rn(ld_volatile(&c.ts->bound32), L.winv32);
                    if (L.i == 1) y *= (1.0f + 4.0f * kEta);
                }
                npts++;
                if ((FAM == 1 || FAM == 2) && beyond) done = true;                 // uncorrelated: points increase
                if (kPerm && L.i >= m) done = true;                                // the sequence has m points
                if (!done && L.i == 1) {
                    // estimated number of further points below the bound
                    int est;
                    if (!(y < 1e9f)) est = 1 << 30;
                    else if (FAM == 1 || FAM == 2) {
                        const float mu = fmaxf(y, 0.0f);
                        float sd_part = 0.0f;   // the standard deviation's share, only when asked for
                        if constexpr (PMH_EST_SIGMAS != 0.0f) sd_part = PMH_EST_SIGMAS * (mu > 0.0f ? mu * rsqrtf(mu) : 0.0f);
                        est = (int)(mu + sd_part + 2.0f);
                    }
                    else if (FAM == 3 || c.unw) est = (int)y;
                    else est = (int)((float)m * (1.0f - __expf(-T.lambda1_32 * y)) * 1.001f) + 1;
                    if (est >= kCap) to_deep = true;
                }
                if (!done && !to_deep && (int)L.i >= kCap) to_deep = true;            // outgrew the lane-sequential cap
                L.i++;
            }
            if (to_deep) {
                // queued for deep mode; at < 32 + next: the slot is slack or was read already
                const int at = atomicAdd(&ws->dq_n, 1);
                if (at < 32 + kSurvCap) ws->sb_e[at] = L.e;
                done = true;
            }
            if (done) L.has = false;
        }
    }
    {
        uint32_t tot = npts;
        for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(kFull, tot, o);
        if (lane == 0 && tot) {
            ws->cnt[F32 ? PMH_CNT_POINTS32 : PMH_CNT_POINTS64] += tot;
            ws->cnt[PMH_CNT_SEQ_POINTS] += tot;
            ws->cnt[PMH_CNT_SEQ_STEPS] += (unsigned long long)nsteps;
        }
    }
    __syncwarp();
    // ---- deep mode for the long sequences (ProbMinHash2/4: once no lane holds a write list)
    const int total_deep = min(ws->dq_n, 32 + kSurvCap);
    if (total_deep && (!kPerm || !__any_sync(kFull, L.has))) {
        const long long td = cyc_now();
        for (int j = 0; j < total_deep; ++j) deep<FAM, F32, false, REJ>(c, ws->sb_e[j], 0);
        count_cyc(c, PMH_CNT_CYC_DEEP, td);
        __syncwarp();
        if (lane == 0) ws->dq_n = 0;
        __syncwarp();
    }
    count_cyc(c, PMH_CNT_CYC_SURV, t_sv);
    return __any_sync(kFull, won);
}

// ------------------------------------------------------------ team helpers
// Barrier of a team of TW warps: the warp itself, or named barrier 1 + team
// index over the team's TW * 32 threads (barrier 0 stays free for
// __syncthreads).
template <int TW>
__device__ __forceinline__ void team_sync() {
    if constexpr (TW == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x >> 5) / TW), "n"(TW * 32) : "memory");
    }
}

// One pass over the elements [lo, hi) of the current item with the team's
// current bound: filter, compacted survivors, q_max refreshes.  Every warp of
// the team takes 64-element steps.  listed: [lo, hi) are entries of the
// item's prefilter list instead, which carry the key and scaled weight.
template <int FAM, bool F32, int TW, bool REJ>
__device__ void run_range(Ctx<F32> &c, uint32_t lo, uint32_t hi, bool listed = false) {
    const SketchParams &P = *c.p;
    const int lane = threadIdx.x & 31;
    constexpr int team_warps = TW;
    TeamShared *ts = c.ts;
    WarpShared *ws = c.ws;
    // Lower bound of the first point's variate: Exp(1) >= U and, by inversion, Exp(lambda;0,1) >=
    // U (1-e^-lambda)/lambda.  With the rejection sampler (REJ) the first draw c1 U >= U holds when
    // U's 53-bit integer is below k1 and nothing is known otherwise; u1: a 23-bit U below it has k < k1.
    const bool rej = REJ && c.rej;
    const float te_lo = (FAM >= 3 && !c.unw && !rej) ? P.tab.te_lo : 1.0f;
    const float u1 = rej ? P.tab.rej_u1_32 : 2.0f;
    if (lane == 0) { ws->sb_n = 0; ws->dq_n = 0; }
    __syncwarp();
    bool refreshed = false;
    int steps = 0;
    SeqLane<F32> L;
    L.has = false;
    // claim size: 64 elements, or less for short ranges so that every warp of the
    // team gets a share of the survivors (about four claims per warp)
    const unsigned long long csz = TW == 1 ? 64ull
        : min(64ull, max(1ull, ((unsigned long long)(hi - lo) + 4ull * TW - 1ull) / (4ull * TW)));
    for (;;) {
        // dynamic claim of the next csz elements of the pass (ts->next starts at lo)
        unsigned long long claim = 0;
        if (lane == 0) claim = TW == 1 ? ts->next : atomicAdd(&ts->next, csz);
        if (TW == 1 && lane == 0) ts->next = claim + csz;
        claim = __shfl_sync(kFull, claim, 0);
        const bool fin = claim >= (unsigned long long)hi;   // the pass is over for this warp
        int n = ws->sb_n;
        if (!fin) {
            const uint32_t base = (uint32_t)claim;
            const uint32_t end = (uint32_t)min((unsigned long long)hi, claim + csz);
            if (c.gbound32 && (steps++ & 15) == 0) {
                // grid mode: adopt the bound published by the other CTAs of this item
                if (lane == 0) {
                    atomic_min_pos_float(&ts->bound32, __uint_as_float(ld_volatile((const int *)c.gbound32)));
                    if constexpr (!F32)
                        atomic_min_pos_double(&ts->bound64, __longlong_as_double((long long)ld_volatile((const uint64_t *)c.gbound64)));
                }
                __syncwarp();
            }
            // L2 prefetch of this warp's step kPrefSteps ahead (ids and weights: up to
            // five 128-byte lines each), so that its loads find L2 instead of HBM
            if (kPrefSteps > 0) {
                const uint32_t pb = base + (uint32_t)(kPrefSteps * team_warps * 64);
                const int pl = lane < 5 ? lane : lane - 5;
                const uint32_t pe = pb + (uint32_t)min(pl * 16, 63);
                if (lane < 10 && pe < hi) {
                    const void *a = lane < 5 ? (const void *)(P.ids + c.beg + pe) : (const void *)(P.weights + c.beg + pe);
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                }
            }
            // filter two elements per lane: the log-free lower bound of the first point.
            // Weights and ids are loaded together (the id does not wait for the weight); a
            // list entry is (key, element index | scaled weight << 32).
            const float b32 = ld_volatile(&ts->bound32);
            bool surv[2];
            uint64_t key[2];
            uint32_t ev[2];
            float winv[2];
            bool valid[2];
            uint64_t wv[2];
            uint64_t idv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t e = base + 32 * h + lane;
                wv[h] = 0;
                idv[h] = 0;
                if (e < end) {
                    if (kListing && listed) {
                        const ulonglong2 v = P.list[((c.beg - c.off0) >> 1) + e];
                        idv[h] = v.x;
                        wv[h] = v.y;
                    } else {
                        wv[h] = (uint64_t)__double_as_longlong(P.weights[c.beg + e]);
                        idv[h] = P.ids[c.beg + e];
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t e = base + 32 * h + lane;
                ev[h] = e;
                surv[h] = false;
                key[h] = 0;
                winv[h] = 0.0f;
                valid[h] = false;
                if (kListing && listed) {
                    valid[h] = e < end;
                    key[h] = idv[h];
                    ev[h] = (uint32_t)wv[h];
                    winv[h] = __uint_as_float((uint32_t)(wv[h] >> 32));
                } else if (e < end && weight_positive(__longlong_as_double((long long)wv[h]))) {
                    valid[h] = true;
                    key[h] = mix64(idv[h] ^ P.mixed_seed);
#if PMH_FILTER_WS
                    winv[h] = ws_scaled(c.unw ? 1.0 : __longlong_as_double((long long)wv[h]), c.sigma);
#endif
                }
                if (valid[h]) {
#if PMH_FILTER_WS
                    // w * 2^-sigma instead of its reciprocal: U te_lo > bound w rejects, and the
                    // reciprocal is taken only for the buffered survivors (process_survivors).
                    // Conservative: the products' roundings and the truncated mantissa are
                    // within the 16-ulp slack.
                    const float u = unif_lo(value_word(key[h], 1));
                    const float ulo = __fmul_rn(u, te_lo);
                    surv[h] = !(__fmul_rn(ulo, 1.0f - 16.0f * 0x1p-24f) > __fmul_rn(b32, winv[h]));
                    if constexpr (REJ) surv[h] = surv[h] || !(u < u1);
#else
                    winv[h] = winv_scaled(c.unw ? 1.0 : __longlong_as_double((long long)wv[h]), c.sigma);
                    const float u = unif_lo(value_word(key[h], 1));
                    const float xlo = winv[h] * u * te_lo;
                    surv[h] = !(xlo * (1.0f - 8.0f * 0x1p-24f) > b32);
                    if constexpr (REJ) surv[h] = surv[h] || !(u < u1);
#endif
                }
            }
            unsigned nvalid = 0, nsurv = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned msk = __ballot_sync(kFull, surv[h]);
                if (surv[h]) {
                    const int pos = n + __popc(msk & ((1u << lane) - 1u));
                    if (pos < kSurvCap) {   // always true: n <= kSurvBatch - 1 before the two appends of <= 32
                        ws->sb_e[32 + pos] = ev[h];
                        ws->sb_key[pos] = key[h];
                        ws->sb_winv[pos] = winv[h];
                    } else {
                        ts->status = PMH_ERR_ITER_LIMIT;
                    }
                }
                n = min(n + __popc(msk), kSurvCap);
                nsurv += __popc(msk);
                if (P.counters) nvalid += popc_ballot(valid[h]);
            }
            if (P.counters) {
                count(c, PMH_CNT_ELEMENTS, nvalid);
                count(c, PMH_CNT_PREFILTERED, nvalid - nsurv);
                if (listed) count(c, PMH_CNT_LISTED, nvalid);
            }
            __syncwarp();
        }
        // expand a full batch of survivors; at the end of the pass, whatever is left
        bool any_win = false;
        if (fin ? (n > 0 || __any_sync(kFull, L.has)) : n >= kSurvBatch) {
            any_win = process_survivors<FAM, F32, REJ>(c, L, n, fin);
            n = 0;
        }
        if (lane == 0) ws->sb_n = n;
        __syncwarp();
        if (fin) break;
        // refresh q_max once everything is filled
        const int uf = __shfl_sync(kFull, lane == 0 ? ld_volatile(&ts->unfilled) : 1, 0);
        if (uf == 0 && (!refreshed || any_win)) {
            refresh_bound<F32>(c);
            refreshed = true;
            if (c.gbound32 && lane == 0) {   // grid mode: publish this CTA's q_max bound
                atomicMin((int *)c.gbound32, __float_as_int(ld_volatile(&ts->bound32)));
                if constexpr (!F32) atomicMin(c.gbound64, (unsigned long long)__double_as_longlong(ld_volatile(&ts->bound64)));
            }
        }
    }
}

// ------------------------------------------------------------ one item
template <int FAM, bool F32, int TW, bool REJ>
__device__ void process_item(Ctx<F32> &c, int item_v, int64_t set) {
    const SketchParams &P = *c.p;
    const uint32_t m = P.m;
    const int lane = threadIdx.x & 31;
    const int tw = (int)(threadIdx.x >> 5) % TW;
    constexpr int team_warps = TW;
    const int tt = tw * 32 + lane;
    const int team_threads = team_warps * 32;
    TeamShared *ts = c.ts;
    WarpShared *ws = c.ws;
    const bool leader = (tt == 0);
    const int64_t out_row = (int64_t)item_v * P.num_sets + set;
    long long t_ph = cyc_now();
    count(c, PMH_CNT_ITEMS, tw == 0);

    // ---- init: empty signature; T = m (ln m + c) / sum(w) = t_s * 2^-sigma, t_s in [1, 2)
    for (uint32_t k = tt; k < m; k += team_threads) {
        if constexpr (F32) ((uint64_t *)c.sig)[k] = kEmptyKey;
        else { ((Rec64 *)c.sig)[k].q = __longlong_as_double(0x7FF0000000000000ll); ((Rec64 *)c.sig)[k].id = 0; }
    }
    c.unw = variant_unweighted(P.variants[item_v]);
    c.rej = REJ && FAM >= 3 && !c.unw;
    SetStat st0 = P.stats[set];
    if (c.unw) st0.wsum = (double)st0.npos;   // binary weights: each element counts 1
    if (leader) {
        ts->status = st0.bad ? PMH_ERR_BAD_WEIGHT : PMH_OK;
        ts->unfilled = (int)m;
        ts->cont_n = 0;
        ts->redo = 0;
        int sigma;
        float t_s;
        first_threshold(m, P.t_factor, st0.wsum, st0.npos, &t_s, &sigma);
        ts->sigma = sigma;
        ts->t_s = t_s;
    }
    team_sync<TW>();
    c.sigma = ts->sigma;
    if (st0.bad || st0.npos == 0) {
        // bad weights or empty set: zero ids, +inf q
        for (uint32_t k = tt; k < m; k += team_threads) {
            P.out_ids[out_row * m + k] = 0;
            if (P.out_q) P.out_q[out_row * m + k] = __longlong_as_double(0x7FF0000000000000ll);
        }
        if (leader && P.status) P.status[out_row] = st0.bad ? PMH_ERR_BAD_WEIGHT : PMH_OK;
        return;
    }
    count_cyc(c, PMH_CNT_CYC_PASS0, t_ph);
    t_ph = cyc_now();

    // ---- rounds.  A listed set's first round (whose bound is the list's) visits only its list
    // entries; the elements the prefilter rejected count as visited and prefiltered here.
    uint32_t listed_n = kUnlisted;
    if (kListing && P.list_n && !c.unw && !c.rej && P.rounds > 0) listed_n = P.list_n[set];
    if (listed_n != kUnlisted) {
        count(c, PMH_CNT_ELEMENTS, leader ? st0.npos - listed_n : 0);
        count(c, PMH_CNT_PREFILTERED, leader ? st0.npos - listed_n : 0);
        count(c, PMH_CNT_LIST_SKIPPED, leader ? st0.npos - listed_n : 0);
    }
    for (int round = 0; round <= P.rounds; ++round) {
        if (leader) {
            ts->next = 0ull;
            if (round < P.rounds && !isinf(ts->t_s)) {
                ts->bound32 = ldexpf(ts->t_s, 2 * round);
                ts->bound64 = ldexp((double)ts->t_s, 2 * round - c.sigma);
            } else {
                ts->bound32 = __int_as_float(0x7F800000);
                ts->bound64 = __longlong_as_double(0x7FF0000000000000ll);
            }
        }
        if (round > 0) count(c, PMH_CNT_ROUNDS, leader);
        team_sync<TW>();
        const bool listed = round == 0 && listed_n != kUnlisted;
        run_range<FAM, F32, TW, REJ>(c, 0, listed ? listed_n : c.n, listed);
        const long long t_bar = cyc_now();
        team_sync<TW>();
        count_cyc(c, PMH_CNT_CYC_BARRIER, t_bar);
        count_cyc(c, PMH_CNT_CYC_FIRST, t_ph);
        t_ph = cyc_now();
        if (ld_volatile(&ts->unfilled) == 0 || ld_volatile(&ts->status) != PMH_OK) break;
        team_sync<TW>();
    }
    team_sync<TW>();

    // ---- FP32: resolve contenders exactly, or redo the item in FP64 when they overflowed the log
    if constexpr (F32) {
        if (leader && ld_volatile(&ts->cont_n) > P.max_cont && ld_volatile(&ts->status) == PMH_OK) {
            if (push_redo(P, item_v, set)) ts->redo = 1;
            else ts->status = PMH_ERR_ITER_LIMIT;
        }
        team_sync<TW>();
        if (ld_volatile(&ts->redo)) {
            count(c, PMH_CNT_REDO, leader);
            count_cyc(c, PMH_CNT_CYC_FINISH, t_ph);
            return;   // the FP64 kernel writes this item's outputs
        }
        if (tw == 0 && ld_volatile(&ts->cont_n) > 0) {
            const uint32_t ev = resolve_contenders<FAM, REJ>(c);
            count(c, PMH_CNT_RESOLVED, ev);
        }
    }
    team_sync<TW>();

    // ---- write out
    const int st = ld_volatile(&ts->status);
    if constexpr (F32) {
        const uint64_t *sig = (const uint64_t *)c.sig;
        for (uint32_t k = tt; k < m; k += team_threads) {
            uint64_t key = sig[k];
            P.out_ids[out_row * m + k] = (key == kEmptyKey || st != PMH_OK) ? 0 : P.ids[c.beg + (uint32_t)(key & 0xFFFFFFFFu)];
        }
        if (P.out_q) {
            // exact FP64 minima: one exact evaluation per component, warps split the components
            for (uint32_t k = tw; k < m; k += team_warps) {
                uint64_t key = sig[k];
                double q = __longlong_as_double(0x7FF0000000000000ll);
                if (key != kEmptyKey && st == PMH_OK) q = exact_h<FAM, F32, REJ>(c, (uint32_t)(key & 0xFFFFFFFFu), k);
                if (lane == 0) P.out_q[out_row * m + k] = q;
            }
        }
    } else {
        const Rec64 *sig = (const Rec64 *)c.sig;
        for (uint32_t k = tt; k < m; k += team_threads) {
            Rec64 r = sig[k];
            bool ok = st == PMH_OK && !isinf(r.q);
            P.out_ids[out_row * m + k] = ok ? r.id : 0;
            if (P.out_q) P.out_q[out_row * m + k] = ok ? r.q : __longlong_as_double(0x7FF0000000000000ll);
        }
    }
    if (leader && P.status) P.status[out_row] = st;
    count_cyc(c, PMH_CNT_CYC_FINISH, t_ph);
}

// ------------------------------------------------------------ grid mode
// Merges a CTA-local FP32 key into the item's global signature (atomicMin),
// logging both sides as contenders when they are within the error bound of
// each other (same rule as an offer).
__device__ __forceinline__ void merge_key_global(uint64_t *gsig, uint32_t k, uint64_t key, GridState *g, int max_cont) {
    const uint64_t cur = ld_volatile(&gsig[k]);
    const float x32 = __uint_as_float((uint32_t)(key >> 32));
    if (cur != kEmptyKey && __uint_as_float((uint32_t)(cur >> 32)) < x32 * (1.0f - 2.0f * kEta)) return;
    const uint64_t old = atomicMin((unsigned long long *)&gsig[k], (unsigned long long)key);
    if (old == kEmptyKey) return;
    const float xo = __uint_as_float((uint32_t)(old >> 32));
    const uint32_t e = (uint32_t)(key & 0xFFFFFFFFu), eo = (uint32_t)(old & 0xFFFFFFFFu);
    if (eo != e && fabsf(x32 - xo) <= kEta * (x32 + xo)) {
        const int at = atomicAdd(&g->cont_n, 2);
        if (at + 1 < max_cont) {
            g->cont_k[at] = k; g->cont_e[at] = e;
            g->cont_k[at + 1] = k; g->cont_e[at + 1] = eo;
        }
    }
}

// Merges a CTA-local (q, id) record into the item's global FP64 signature
// (lexicographic minimum by 128-bit CAS).
__device__ __forceinline__ void merge_rec_global(Rec64 *gsig, uint32_t k, Rec64 r, GridState *g) {
    if (isinf(r.q)) return;
    Rec64 expected;
    expected.q = ld_volatile(&gsig[k].q);
    if (r.q > expected.q) return;
    expected.id = ld_volatile((const uint64_t *)&gsig[k].id);
    for (int it = 0; it < kCasLimit; ++it) {
        if (!(r.q < expected.q || (r.q == expected.q && r.id < expected.id))) return;
        Rec64 old = atomicCAS(&gsig[k], expected, r);
        if (__double_as_longlong(old.q) == __double_as_longlong(expected.q) && old.id == expected.id) return;
        expected = old;
    }
    g->status = PMH_ERR_ITER_LIMIT;
}

// Finalisation by the last CTA of a grid item: exact resolution of the logged
// contenders (FP32), write-out, and a single-CTA rerun with growing
// thresholds if a component is still empty (probability ~e^-c per item).
template <int FAM, bool F32, bool REJ>
__device__ void grid_finalize(Ctx<F32> &c, GridState *g, void *gsig_v, int item_v, int64_t set) {
    const SketchParams &P = *c.p;
    const uint32_t m = P.m;
    const int lane = threadIdx.x & 31;
    const int tw = threadIdx.x >> 5;
    const int team_warps = blockDim.x >> 5;
    const int64_t out_row = (int64_t)item_v * P.num_sets + set;
    TeamShared *ts = c.ts;
    int st = ld_volatile(&g->status);
    if constexpr (F32) {
        uint64_t *gsig = (uint64_t *)gsig_v;
        const int nc = ld_volatile(&g->cont_n);
        if ((nc > P.max_cont_grid || ld_volatile(&g->redo)) && st == PMH_OK) {
            // a contender log overflowed: the FP64 kernel of this family redoes the item
            if (threadIdx.x == 0) {
                if (push_redo(P, item_v, set)) ts->redo = 1;
                else { ts->redo = 0; g->status = PMH_ERR_ITER_LIMIT; }
            }
            __syncthreads();
            if (ts->redo) {
                count(c, PMH_CNT_REDO, threadIdx.x == 0);
                return;
            }
            st = PMH_ERR_ITER_LIMIT;
        }
        if (tw == 0 && nc > 0 && st == PMH_OK) {
            const uint32_t ev = resolve_list<FAM, REJ>(c, g->cont_k, g->cont_e, nc, gsig);
            count(c, PMH_CNT_RESOLVED, ev);
        }
    }
    __syncthreads();
    // a component left empty: redo the item in this CTA with growing thresholds
    int empty = 0;
#pragma unroll 4
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
        if constexpr (F32) empty |= __ldcg(&((const unsigned long long *)gsig_v)[k]) == kEmptyKey;
        else empty |= isinf(__ldcg(&((const Rec64 *)gsig_v)[k].q));
    }
    empty = __syncthreads_or(empty);
    if (empty && st == PMH_OK) {
        c.gbound32 = nullptr;
        c.gbound64 = nullptr;
        process_item<FAM, F32, 8, REJ>(c, item_v, set);
        return;
    }
    if constexpr (F32) {
        // L2 loads: other CTAs wrote the global signature
        const unsigned long long *gsig = (const unsigned long long *)gsig_v;
        // eight components per thread in flight: the id gathers of one thread do not wait on each other
        constexpr int kU = 8;
        for (uint32_t k0 = threadIdx.x; k0 < m; k0 += kU * blockDim.x) {
            uint64_t idv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t k = k0 + u * blockDim.x;
                const uint64_t key = k < m ? __ldcg(&gsig[k]) : kEmptyKey;
                idv[u] = (key == kEmptyKey || st != PMH_OK) ? 0 : P.ids[c.beg + (uint32_t)(key & 0xFFFFFFFFu)];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t k = k0 + u * blockDim.x;
                if (k < m) P.out_ids[out_row * m + k] = idv[u];
            }
        }
        if (P.out_q) {
            for (uint32_t k = tw; k < m; k += team_warps) {
                const uint64_t key = __ldcg(&gsig[k]);
                double q = __longlong_as_double(0x7FF0000000000000ll);
                if (key != kEmptyKey && st == PMH_OK) q = exact_h<FAM, F32, REJ>(c, (uint32_t)(key & 0xFFFFFFFFu), k);
                if (lane == 0) P.out_q[out_row * m + k] = q;
            }
        }
    } else {
        const Rec64 *gsig = (const Rec64 *)gsig_v;
        for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
            Rec64 r;
            r.q = __ldcg(&gsig[k].q);
            r.id = __ldcg((const unsigned long long *)&gsig[k].id);
            const bool ok = st == PMH_OK && !isinf(r.q);
            P.out_ids[out_row * m + k] = ok ? r.id : 0;
            if (P.out_q) P.out_q[out_row * m + k] = ok ? r.q : __longlong_as_double(0x7FF0000000000000ll);
        }
    }
    if (threadIdx.x == 0 && P.status) P.status[out_row] = st;
    (void)ts;
}

// Expansion of a grid-mode warp's buffered survivors to the end of their
// sequences.  (Kept inline: out of line, with the call's register saves, the
// grid kernel on one set of 1e8 took 0.678 ms instead of 0.614.)
template <int FAM, bool F32, bool REJ>
__device__ __forceinline__ bool grid_expand(Ctx<F32> &c, int n) {
    SeqLane<F32> L;
    L.has = false;
    return process_survivors<FAM, F32, REJ>(c, L, n, true);
}

// One lane's pairs of a grid-mode block starting at element gb of the whole input: pairs
// (gb >> 1) + lane and + 32; a pair whose second element lies at or past g_hi is read as its
// first element alone, and one wholly past it as zeros.
__device__ __forceinline__ void grid_load_pairs(const ulonglong2 *w2, const ulonglong2 *ids2, uint64_t gb, uint64_t g_hi,
                                                int lane, ulonglong2 &w0, ulonglong2 &w1, ulonglong2 &i0, ulonglong2 &i1) {
    const uint64_t pe = gb + 2 * (uint64_t)lane;
    w0 = w1 = i0 = i1 = make_ulonglong2(0ull, 0ull);
    if (pe + 1 < g_hi) { w0 = __ldcs(w2 + (pe >> 1)); i0 = __ldcs(ids2 + (pe >> 1)); }
    else if (pe < g_hi) { w0.x = __ldcs(&w2[pe >> 1].x); i0.x = __ldcs(&ids2[pe >> 1].x); }
    if (pe + 65 < g_hi) { w1 = __ldcs(w2 + (pe >> 1) + 32); i1 = __ldcs(ids2 + (pe >> 1) + 32); }
    else if (pe + 64 < g_hi) { w1.x = __ldcs(&w2[(pe >> 1) + 32].x); i1.x = __ldcs(&ids2[(pe >> 1) + 32].x); }
}

// Grid mode's pass over all elements of one item by this warp, which claims
// runs of 128-element blocks from the item's counter (no barrier of the CTA
// until the pass ends).  A huge set's elements almost all fail the filter (the
// survivors number about m (ln m + c) per item, against 1e6 and more
// elements), so the common path is the filter alone: every lane takes four
// elements of a block from two 16-byte loads of ids and two of weights (ids and
// weights 16-byte aligned; blocks start at an even element of the whole
// input), and a block without survivors costs one vote.  A block with
// survivors appends them to the warp's buffer (their keys and scaled weights
// computed again there) and expands it as run_range does, except that every
// expansion runs its sequences to the end (no lane state outlives it, so none
// is live in the common path).
template <int FAM, bool F32, bool REJ>
__device__ void grid_pass(Ctx<F32> &c, GridState *gs) {
    const SketchParams &P = *c.p;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = blockDim.x >> 5;
    TeamShared *ts = c.ts;
    WarpShared *ws = c.ws;
    const bool rej = REJ && c.rej;
    const float te_lo = (FAM >= 3 && !c.unw && !rej) ? P.tab.te_lo : 1.0f;
    const float u1 = rej ? P.tab.rej_u1_32 : 2.0f;
    const uint64_t mseed = P.mixed_seed;
    const int sigma = c.sigma;
    const bool unw = c.unw;
    const float ws1 = ws_scaled(1.0, sigma);   // binary weights: every element counts 1
    const bool counting = P.counters != nullptr;
    if (lane == 0) { ws->sb_n = 0; ws->dq_n = 0; }
    __syncwarp();
    int n = 0;
    const uint64_t g_lo = (uint64_t)c.beg, g_hi = (uint64_t)c.beg + c.n;
    const uint64_t g0 = g_lo & ~1ull;
    const uint32_t nblk = (uint32_t)((g_hi - g0 + 127) / 128);
    const ulonglong2 *ids2 = (const ulonglong2 *)P.ids;
    const ulonglong2 *w2 = (const ulonglong2 *)P.weights;
    // claims of kb blocks: about eight per warp of the launch, at most 16 blocks (2048 elements;
    // claims shrinking towards the end measured no faster on one set of 1e8)
    const uint32_t warps_all = gridDim.x * nwarps;
    const uint32_t kb = max(1u, min(16u, nblk / (8u * warps_all)));
    auto claim = [&](uint32_t &x, uint32_t &xend) {
        unsigned cl = 0;
        if (lane == 0) cl = atomicAdd(&gs->next_chunk, kb);
        cl = __shfl_sync(kFull, cl, 0);
        x = cl;
        xend = cl < nblk ? min(cl + kb, nblk) : cl;
    };
    uint32_t b = 0, bend = 0, step = 0;
    for (;;) {
        if (b >= bend) claim(b, bend);
        const bool fin = b >= nblk;
        const uint64_t gb = g0 + (uint64_t)b * 128;
        ulonglong2 wp[2], ip[2];   // this lane's pairs: elements gb + 64 h + 2 lane + {0, 1}
        unsigned sm = 0;           // bit j: element j of this lane (j = 2 h + s) survives
        if (!fin) {
            // every 16 blocks the bound published by the other CTAs of the item (read here,
            // adopted after the filter, so that the load's latency hides behind it)
            const bool adopt = c.gbound32 && (step & 15) == 0 && lane == 0;
            unsigned gb32 = 0;
            unsigned long long gb64 = 0;
            if (adopt) {
                gb32 = (unsigned)ld_volatile((const int *)c.gbound32);
                if constexpr (!F32) gb64 = ld_volatile((const uint64_t *)c.gbound64);
            }
            const float b32 = ld_volatile(&ts->bound32);
            // the item's elements relative to the block: [rlo, rhi) within [0, 128]
            const uint32_t rlo = gb < g_lo ? (uint32_t)(g_lo - gb) : 0u;
            const uint32_t rhi = g_hi - gb < 128 ? (uint32_t)(g_hi - gb) : 128u;
            grid_load_pairs(w2, ids2, gb, g_hi, lane, wp[0], wp[1], ip[0], ip[1]);
            unsigned nvalid = 0, nsurv = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t r = 64 * (j >> 1) + 2 * lane + (j & 1);   // element gb + r
                const uint64_t wb = (j & 1) ? wp[j >> 1].y : wp[j >> 1].x;
                const double w = __longlong_as_double((long long)wb);
                const bool valid = r >= rlo && r < rhi && weight_positive(w);
                bool surv = false;
                if (valid) {
                    const uint64_t key = mix64(((j & 1) ? ip[j >> 1].y : ip[j >> 1].x) ^ mseed);
                    const float u = unif_lo(value_word(key, 1));
                    const float ulo = __fmul_rn(u, te_lo);
                    surv = !(__fmul_rn(ulo, 1.0f - 16.0f * 0x1p-24f) > __fmul_rn(b32, unw ? ws1 : ws_scaled(w, sigma)));
                    if constexpr (REJ) surv = surv || !(u < u1);
                }
                sm |= (unsigned)surv << j;
                if (counting) {
                    nvalid += popc_ballot(valid);
                    nsurv += popc_ballot(surv);
                }
            }
            if (counting) {
                count(c, PMH_CNT_ELEMENTS, nvalid);
                count(c, PMH_CNT_PREFILTERED, nvalid - nsurv);
            }
            if (adopt) {
                atomic_min_pos_float(&ts->bound32, __uint_as_float(gb32));
                if constexpr (!F32) atomic_min_pos_double(&ts->bound64, __longlong_as_double((long long)gb64));
            }
        }
        // rare path: this block has survivors, or the pass ends with some buffered
        if (fin ? n > 0 : __any_sync(kFull, sm != 0)) {
            bool pending = !fin;   // this block's survivors are not in the buffer yet
            bool any_win = false;
            for (;;) {
                if (pending) {
                    unsigned msk[4];
                    int cnt = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        msk[j] = __ballot_sync(kFull, (sm >> j) & 1u);
                        cnt += __popc(msk[j]);
                    }
                    if (n + cnt <= kSurvCap) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if ((sm >> j) & 1u) {
                                const int pos = n + __popc(msk[j] & ((1u << lane) - 1u));
                                const uint64_t g = gb + 64 * (j >> 1) + 2 * lane + (j & 1);
                                const double w = __longlong_as_double((long long)((j & 1) ? wp[j >> 1].y : wp[j >> 1].x));
                                ws->sb_e[32 + pos] = (uint32_t)(g - (uint64_t)c.beg);
                                ws->sb_key[pos] = mix64(((j & 1) ? ip[j >> 1].y : ip[j >> 1].x) ^ mseed);
                                ws->sb_winv[pos] = unw ? ws1 : ws_scaled(w, sigma);
                            }
                            n += __popc(msk[j]);
                        }
                        pending = false;
                        __syncwarp();
                    }
                }
                // expand when the buffer holds a batch, cannot take this block, or the pass ends
                if (!pending && !(fin ? n > 0 : n >= kSurvBatch)) break;
                any_win |= grid_expand<FAM, F32, REJ>(c, n);
                n = 0;
            }
            if (any_win) {
                const int uf = __shfl_sync(kFull, lane == 0 ? ld_volatile(&ts->unfilled) : 1, 0);
                if (uf == 0) {
                    refresh_bound<F32>(c);
                    if (c.gbound32 && lane == 0) {   // publish this CTA's q_max bound
                        atomicMin((int *)c.gbound32, __float_as_int(ld_volatile(&ts->bound32)));
                        if constexpr (!F32) atomicMin(c.gbound64, (unsigned long long)__double_as_longlong(ld_volatile(&ts->bound64)));
                    }
                }
            }
        }
        if (fin) break;
        ++b;
        ++step;
    }
    if (lane == 0) ws->sb_n = 0;
    __syncwarp();
}

// One CTA's share of a grid item: its warps' part of the filter pass with a
// local signature, then the merge into the global signature; the last CTA to
// finish finalises the item.
template <int FAM, bool F32, bool REJ>
__device__ void grid_participate(Ctx<F32> &c, GridState *g, void *gsig_v, int item_v, int64_t set) {
    const SketchParams &P = *c.p;
    const uint32_t m = P.m;
    TeamShared *ts = c.ts;
    const bool leader = threadIdx.x == 0;
    c.unw = variant_unweighted(P.variants[item_v]);
    c.rej = REJ && FAM >= 3 && !c.unw;
    SetStat st0 = P.stats[set];
    if (c.unw) st0.wsum = (double)st0.npos;   // binary weights: each element counts 1
    const bool live = !st0.bad && st0.npos > 0;
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
        if constexpr (F32) ((uint64_t *)c.sig)[k] = kEmptyKey;
        else { ((Rec64 *)c.sig)[k].q = __longlong_as_double(0x7FF0000000000000ll); ((Rec64 *)c.sig)[k].id = 0; }
    }
    if (leader) {
        ts->status = PMH_OK;
        ts->unfilled = (int)m;
        ts->cont_n = 0;
        int sigma = 0;
        float t_s = __int_as_float(0x7F800000);
        const double T = (double)m * (double)P.t_factor_grid / st0.wsum;
        if (live && T > 0.0 && T < 1e300) {
            int ex;
            const double fr = frexp(T, &ex);
            t_s = (float)(2.0 * fr);
            sigma = -(ex - 1);
        }
        ts->sigma = sigma;
        ts->t_s = t_s;
        ts->bound32 = t_s;
        ts->bound64 = isinf(t_s) ? __longlong_as_double(0x7FF0000000000000ll) : ldexp((double)t_s, -sigma);
        if (st0.bad && g->status == PMH_OK) g->status = PMH_ERR_BAD_WEIGHT;
    }
    __syncthreads();
    c.sigma = ts->sigma;
    c.gbound32 = &g->bound32;
    c.gbound64 = &g->bound64;
    if (live) {
        // the trimmed filter needs 16-byte aligned ids and weights (else run_range's, chunk by chunk)
        const bool lean = PMH_GRID_LEAN && ((((uintptr_t)P.ids) | ((uintptr_t)P.weights)) & 15u) == 0;
        const long long t_pass = cyc_now();
        uint64_t chunk = (uint64_t)c.n / (4ull * gridDim.x);
        chunk = chunk < kGridChunkMin ? kGridChunkMin : (chunk > kGridChunk ? kGridChunk : chunk);
        if (lean) {
            grid_pass<FAM, F32, REJ>(c, g);
            __syncthreads();
        }
        for (; !lean;) {
            if (leader) {
                const unsigned int idx = atomicAdd(&g->next_chunk, 1u);
                ts->item_idx = (int)idx;
                ts->next = (unsigned long long)idx * chunk;
            }
            __syncthreads();
            const uint64_t lo = (uint64_t)(uint32_t)ts->item_idx * chunk;
            __syncthreads();
            if (lo >= c.n) break;
            const uint32_t hi = (uint32_t)min((uint64_t)c.n, lo + chunk);
            run_range<FAM, F32, 8, REJ>(c, (uint32_t)lo, hi);
            __syncthreads();
        }
        count_cyc(c, PMH_CNT_CYC_FIRST, t_pass);
        // merge the local signature into the item's global one
        for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
            if constexpr (F32) {
                const uint64_t key = ((const uint64_t *)c.sig)[k];
                if (key != kEmptyKey) merge_key_global((uint64_t *)gsig_v, k, key, g, P.max_cont_grid);
            } else {
                merge_rec_global((Rec64 *)gsig_v, k, ((const Rec64 *)c.sig)[k], g);
            }
        }
        if (leader) {
            // local contenders join the item's list
            const int nl = ts->cont_n;
            if (nl > P.max_cont) g->redo = 1;
            const int nk = min(nl, P.max_cont);
            if (nk > 0) {
                const int at = atomicAdd(&g->cont_n, nk);
                for (int j = 0; j < nk && at + j < P.max_cont_grid; ++j) { g->cont_k[at + j] = ts->cont_k[j]; g->cont_e[at + j] = ts->cont_e[j]; }
            }
            if (ts->status != PMH_OK) g->status = ts->status;
        }
    }
    __syncthreads();
    __threadfence();
    if (leader) ts->item_idx = (atomicAdd(&g->done, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    const bool last = ts->item_idx == 1;
    __syncthreads();
    if (last) {
        __threadfence();
        const long long t_f = cyc_now();
        grid_finalize<FAM, F32, REJ>(c, g, gsig_v, item_v, set);
        count_cyc(c, PMH_CNT_CYC_FINISH, t_f);
    }
    c.gbound32 = nullptr;
    c.gbound64 = nullptr;
}

// Persistent grid-mode kernel of one family: every CTA takes part in every
// grid item of that family, in list order.  Registers are budgeted for three
// 8-warp CTAs per SM in FP32 (80 registers) and two in FP64 (128): the filter
// that dominates a huge set issues fewer instructions with fewer spills, and
// the FP64 expansion needs the registers.
#ifndef PMH_GRID_MINB32
#define PMH_GRID_MINB32 3
#endif
#ifndef PMH_GRID_MINB64
#define PMH_GRID_MINB64 2
#endif
template <bool F32, int FAM, bool REJ = false>
__global__ void __launch_bounds__(256, F32 ? PMH_GRID_MINB32 : PMH_GRID_MINB64) grid_kernel(const __grid_constant__ SketchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool kPerm = (FAM == 2 || FAM == 4);
    constexpr int NW = 8;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (!p.gctl) return;
    const int count_all = (int)ld_volatile((const int *)&p.gctl->count[FAM - 1]);
    const int nitems = min(count_all, kMaxGrid);
    if (nitems == 0) return;
    SmemLayout L(1, NW, p.m, F32, kPerm);
    Ctx<F32> c;
    c.p = &p;
    c.ts = (TeamShared *)(smem + L.team_off);
    c.sig = smem + L.sig_off;
    c.ws = (WarpShared *)(smem + L.warp_off + (size_t)warp * align16(sizeof(WarpShared)));
    c.perm = kPerm ? (uint16_t *)(smem + L.perm_off + (size_t)warp * perm_bytes(p.m)) : nullptr;
    c.fy = kPerm ? (uint32_t *)(smem + L.perm_off + (size_t)warp * perm_bytes(p.m)) : nullptr;   // shares the bytes of perm
    c.gbound32 = nullptr;
    c.gbound64 = nullptr;
    if (lane < PMH_NUM_COUNTERS) c.ws->cnt[lane] = 0;
    __syncwarp();
    for (int j = 0; j < nitems; ++j) {
        const uint64_t it = p.gctl->list[FAM - 1][j];
        const int v = (int)(it >> 40);
        const int64_t set = (int64_t)(it & ((1ull << 40) - 1));
        const int slot = (FAM - 1) * kMaxGrid + j;
        c.beg = p.offsets[set];
        c.off0 = p.offsets[0];
        c.n = (uint32_t)(p.offsets[set + 1] - c.beg);
        grid_participate<FAM, F32, REJ>(c, &p.gstate[slot], (unsigned char *)p.gsig + (size_t)slot * p.m * 16, v, set);
        __syncthreads();
    }
    __syncwarp();
    if (p.counters && lane < PMH_NUM_COUNTERS && c.ws->cnt[lane]) atomicAdd(&p.counters[lane], c.ws->cnt[lane]);
}

// Resets the state and global signature of the grid items of this call.
static __global__ void grid_init_kernel(GridCtl *ctl, GridState *gs, void *gsig, uint32_t m, int f32) {
    const int slot = blockIdx.x;   // [4][kMaxGrid]
    const int fam = slot / kMaxGrid, j = slot % kMaxGrid;
    if (j >= min((int)ctl->count[fam], kMaxGrid)) return;
    GridState *g = &gs[slot];
    if (threadIdx.x == 0) {
        g->next_chunk = 0;
        g->done = 0;
        g->bound32 = 0x7F800000u;
        g->status = PMH_OK;
        g->bound64 = 0x7FF0000000000000ull;
        g->cont_n = 0;
        g->redo = 0;
    }
    unsigned char *sig = (unsigned char *)gsig + (size_t)slot * m * 16;
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
        if (f32) ((uint64_t *)sig)[k] = kEmptyKey;
        else { ((Rec64 *)sig)[k].q = __longlong_as_double(0x7FF0000000000000ll); ((Rec64 *)sig)[k].id = 0; }
    }
}

// ------------------------------------------------------------ kernel
// NW warps per block in teams of TW warps (TW = 1: every warp sketches its own
// items; TW = NW: the whole block shares one signature); MINB = the blocks per
// SM the register budget is sized for.
template <bool F32, int NW, int TW, int MINB, int FAM, bool REJ = false>
__global__ void __launch_bounds__(NW * 32, MINB) sketch_kernel(const __grid_constant__ SketchParams p) {
    static_assert(NW % TW == 0 && NW / TW <= 15, "teams must tile the block (named barriers 1..15)");
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool kPerm = (FAM == 2 || FAM == 4);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    constexpr int teams = NW / TW;
    const int team = warp / TW;
    SmemLayout L(teams, NW, p.m, F32, kPerm);
    TeamShared *ts = (TeamShared *)(smem + L.team_off + (size_t)team * align16(sizeof(TeamShared)));
    Ctx<F32> c;
    c.p = &p;
    c.ts = ts;
    c.sig = smem + L.sig_off + (size_t)team * p.m * (F32 ? 8 : 16);
    c.ws = (WarpShared *)(smem + L.warp_off + (size_t)warp * align16(sizeof(WarpShared)));
    c.perm = kPerm ? (uint16_t *)(smem + L.perm_off + (size_t)warp * perm_bytes(p.m)) : nullptr;
    c.fy = kPerm ? (uint32_t *)(smem + L.perm_off + (size_t)warp * perm_bytes(p.m)) : nullptr;   // shares the bytes of perm
    c.gbound32 = nullptr;
    c.gbound64 = nullptr;
    if (lane < PMH_NUM_COUNTERS) c.ws->cnt[lane] = 0;
    __syncwarp();
    const int tt = (warp % TW) * 32 + lane;   // thread index within the team
    const bool team_leader = tt == 0;
    const long long t_warp = cyc_now();
    // the FP64 redo launch reads its queue's length (the FP32 kernels' redo count) from the device
    const int64_t qlen = p.queue_len_dev ? min(p.queue_len, (int64_t)ld_volatile((const int *)p.queue_len_dev)) : p.queue_len;
    for (;;) {
        const long long t_item = cyc_now();
        if (team_leader) ts->item_idx = (int)atomicAdd(p.head, 1u);
        team_sync<TW>();
        const int64_t qi = ts->item_idx;
        team_sync<TW>();
        if (qi >= qlen) break;
        const uint64_t it = p.queue[qi];
        if (it & kSkipBit) continue;     // processed in grid mode
        const int v = (int)(it >> 40);
        const int64_t set = (int64_t)(it & ((1ull << 40) - 1));
        const int64_t b = p.offsets[set], e = p.offsets[set + 1];
        const int64_t out_row = (int64_t)v * p.num_sets + set;
        if (e < b || e - b > (int64_t)PMH_MAX_SET_ELEMENTS) {
            const int code = e < b ? PMH_ERR_INVALID_ARG : PMH_ERR_UNSUPPORTED;
            for (uint32_t k = tt; k < p.m; k += TW * 32) {
                p.out_ids[out_row * p.m + k] = 0;
                if (p.out_q) p.out_q[out_row * p.m + k] = __longlong_as_double(0x7FF0000000000000ll);
            }
            if (team_leader && p.status) p.status[out_row] = code;
            continue;
        }
        c.beg = b;
        c.off0 = p.offsets[0];
        c.n = (uint32_t)(e - b);
        process_item<FAM, F32, TW, REJ>(c, v, set);
        team_sync<TW>();
        count_cyc(c, PMH_CNT_CYC_ITEM, t_item);
    }
    count_cyc(c, PMH_CNT_CYC_WARP, t_warp);
    __syncwarp();
    if (p.counters && lane < PMH_NUM_COUNTERS && c.ws->cnt[lane]) atomicAdd(&p.counters[lane], c.ws->cnt[lane]);
}

}  // namespace pmh
