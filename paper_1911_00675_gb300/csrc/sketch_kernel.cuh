// Persistent ProbMinHash sketch kernel (template over precision and team shape).
//
// GPU design (replaces the paper's sequential element loop, Algorithm
// "Basic structure of ProbMinHash algorithms"):
//   * A team (one warp, or a whole CTA) owns one work item = (set, variant) at
//     a time; its signature lives in shared memory.  Items come from a global
//     queue ordered by decreasing set size.
//   * Threshold rounds.  The sequential algorithm lets q_max fall element by
//     element; a data-parallel pass cannot wait for that.  Round r instead
//     stops every element at min(T*4^r, q_max) with T = m(ln m + c)/sum(w):
//     the merged point process of the set has density sum(w), so all m labels
//     have appeared below T except with probability ~e^-c (coupon collector).
//     Every point <= the final q_max is still generated (q_max only decreases),
//     so the signature is exactly that of the paper; a round that leaves a
//     component empty is repeated with a larger T (offers are idempotent), and
//     the last round has T = +inf.
//   * First points: one lane per element, with a log-free prefilter
//     (Exp(1) >= U, Exp(lambda;0,1) >= U*(1-e^-lambda)/lambda).  Survivors
//     continue lane-sequentially for a few points; longer sequences go to a
//     warp queue and are expanded 32 points at a time (warp scan of the
//     uncorrelated spacings, Eq. uncorrelated_recursion; the lazy
//     Fisher-Yates permutation of Algorithm "Lazy generation of random
//     permutation elements" resolved inside the group with match/shuffle).
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

constexpr int kMaxCont = 64;     // contender records per team (overflow -> PMH_ERR_ITER_LIMIT)
constexpr int kLSeq = 4;         // points generated lane-sequentially before the warp queue
constexpr int kCasLimit = 1 << 16;

struct __align__(16) Rec64 {
    double q;
    unsigned long long id;
};

struct SketchParams {
    const uint64_t *ids;
    const double *weights;
    const int64_t *offsets;
    int64_t num_sets;
    uint32_t m;
    uint64_t mixed_seed;          // mix64(seed)
    int32_t variants[8];
    int32_t num_variants;
    Tables tab;
    uint64_t *out_ids;
    double *out_q;
    int32_t *status;
    unsigned long long *counters;
    const uint64_t *queue;        // (variant index << 40) | set index
    int64_t queue_len;
    unsigned int *head;           // next queue position
    float t_factor;               // ln m + c
    int rounds;                   // finite-T rounds before the T = +inf round
    uint32_t cap_points;          // iteration cap (with replacement)
    int has_perm;                 // shared permutation arrays allocated
};

struct TeamShared {
    int item_idx;
    int unfilled;
    int status;
    int cont_n;
    float bound32;      // stop bound in scaled FP32 units (x * 2^sigma)
    int sigma;
    double bound64;     // FP64 path: exact stop bound
    float t_s;          // T * 2^sigma
    int n_pos;
    float red_s[32];
    int red_e[32];
    int red_i[32];
    uint32_t cont_k[kMaxCont];
    uint32_t cont_e[kMaxCont];
};

struct WarpShared {
    uint32_t dq[32];
    int dq_n;
    int slot[32];
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct SmemLayout {
    size_t team_off, sig_off, warp_off, perm_off, total;
    __host__ __device__ SmemLayout(int teams, int warps, uint32_t m, bool f32, bool perm) {
        team_off = 0;
        sig_off = align16(team_off + (size_t)teams * align16(sizeof(TeamShared)));
        warp_off = align16(sig_off + (size_t)teams * m * (f32 ? 8 : 16));
        perm_off = align16(warp_off + (size_t)warps * align16(sizeof(WarpShared)));
        total = align16(perm_off + (perm ? (size_t)warps * m * 2 : 0));
    }
};

// Work counters kept in registers and flushed once per item.
struct Counters {
    unsigned long long c[PMH_NUM_COUNTERS];
};

// ------------------------------------------------------------------------
// Per-item context.
template <bool F32>
struct Ctx {
    const SketchParams *p;
    TeamShared *ts;
    void *sig;
    WarpShared *ws;
    uint16_t *perm;     // this warp's permutation array (or null)
    int64_t beg;
    uint32_t n;
    int sigma;
    int fam;
    Counters cnt;
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
            if (at + 1 < kMaxCont) {
                c.ts->cont_k[at] = k;
                c.ts->cont_e[at] = e;
                c.ts->cont_k[at + 1] = k;
                c.ts->cont_e[at + 1] = (uint32_t)(old & 0xFFFFFFFFu);
            }
            c.cnt.c[PMH_CNT_CONTENDERS] += 1;
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
    if constexpr (F32) {
        const uint64_t *sig = (const uint64_t *)c.sig;
        uint32_t mx = 0;
        for (uint32_t k = lane; k < m; k += 32) {
            uint32_t hi = (uint32_t)(ld_volatile(&sig[k]) >> 32);
            mx = max(mx, hi);
        }
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
}

// ------------------------------------------------------------ Fisher-Yates group
// 32 consecutive steps t0..t0+31 (0-based) of the lazy permutation of one
// element, whose state before the group is perm[t0..m).  Step t draws
// r_t = t + floor(L * (m-t) / 2^64), returns label P[r_t] and sets P[r_t] = P[t]
// (Algorithm "Lazy generation of random permutation elements", 0-based).
// In-group dependencies: the value at position p before step t is the value
// moved there by the latest earlier step u with r_u = p, else perm[p]; chains
// of such moves are resolved by pointer jumping over lanes.
__device__ __forceinline__ uint32_t fy_group(uint16_t *perm, int *slot, uint32_t m, uint32_t t0, uint64_t lw, bool act) {
    const int lane = threadIdx.x & 31;
    const uint32_t t = t0 + lane;
    const uint32_t r = act ? t + uniform_int(lw, m - t) : 0xFFFFFFFFu;
    slot[lane] = -1;
    __syncwarp();
    if (act && r != t && r - t0 < 32u) atomicMax(&slot[r - t0], lane);
    __syncwarp();
    int ptr = slot[lane];
    uint32_t val = (act && ptr < 0) ? (uint32_t)perm[t] : 0u;
    for (int it = 0; it < 5; ++it) {
        int src = ptr >= 0 ? ptr : lane;
        uint32_t v2 = __shfl_sync(kFull, val, src);
        int p2 = __shfl_sync(kFull, ptr, src);
        if (ptr >= 0) {
            if (p2 < 0) { val = v2; ptr = -1; } else ptr = p2;
        }
    }
    const uint32_t moved = val;   // value at position t just before step t
    const uint32_t same = __match_any_sync(kFull, r);
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

// Sparse Fisher-Yates for the first kLSeq steps of one element (registers).
struct SparseFY {
    uint32_t r[kLSeq], mv[kLSeq];
    __device__ __forceinline__ uint32_t lookup(uint32_t pos, int t) const {
        uint32_t v = pos;
#pragma unroll
        for (int s = 0; s < kLSeq; ++s)
            if (s < t && r[s] == pos) v = mv[s];
        return v;
    }
    __device__ __forceinline__ uint32_t step(int t, uint64_t lw, uint32_t m) {
        uint32_t rt = (uint32_t)t + uniform_int(lw, m - (uint32_t)t);
        uint32_t moved = lookup((uint32_t)t, t);
        uint32_t label = lookup(rt, t);
#pragma unroll
        for (int s = 0; s < kLSeq; ++s)
            if (s == t) { r[s] = rt; mv[s] = moved; }
        return label;
    }
};

// ------------------------------------------------------------ element weights
struct ElemW {
    double w_inv;    // FP64 path
    float winv32;    // scaled FP32 reciprocal (both paths: prefilter)
};

// ------------------------------------------------------------ stage A
// One lane, one element: first point (with prefilter) and up to kLSeq points
// sequentially.  Returns kNeedDeep if the element needs the warp queue, plus
// kWon if one of its offers became a component minimum.
constexpr int kNeedDeep = 1, kWon = 2;
template <int FAM, bool F32>
__device__ int stage_a(Ctx<F32> &c, uint32_t e, uint64_t id, double w) {
    const SketchParams &P = *c.p;
    const Tables &T = P.tab;
    const uint32_t m = P.m;
    ElemW ew;
    ew.winv32 = winv_scaled(w, c.sigma);
    ew.w_inv = F32 ? 0.0 : __drcp_rn(w);
    const uint64_t key = mix64(id ^ P.mixed_seed);
    c.cnt.c[PMH_CNT_ELEMENTS] += 1;
    uint64_t vw = value_word(key, 1);
    // log-free prefilter on the first point: x_1 >= w_inv * U (* te_lo for the correlated families)
    {
        float b32 = ld_volatile(&c.ts->bound32);
        float xlo = ew.winv32 * unif_lo(vw);
        if (FAM >= 3) xlo *= T.te_lo;
        if (xlo * (1.0f - 8.0f * 0x1p-24f) > b32) {
            c.cnt.c[PMH_CNT_PREFILTERED] += 1;
            return 0;
        }
    }
    int won = 0;
    SparseFY fy;
    float s32 = 0.0f;      // F1/F2: running unscaled sum (FP32)
    double x64 = 0.0;      // F1/F2: running value (FP64)
#pragma unroll 1
    for (int i = 1; i <= kLSeq; ++i) {
        if ((FAM == 2 || FAM == 4) && (uint32_t)i > m) return won;
        if (FAM == 1 || FAM == 3) {
            if ((uint32_t)i > P.cap_points) { c.ts->status = PMH_ERR_ITER_LIMIT; return won; }
        }
        if (i > 1) vw = value_word(key, (uint64_t)i);
        // correlated: lower bound of point i
        if (FAM >= 3 && i > 1) {
            if constexpr (F32) {
                float lb = (FAM == 3) ? ew.winv32 * (float)(i - 1) : ew.winv32 * T.gamma32[i - 1];
                if (lb * (1.0f - kEta) > ld_volatile(&c.ts->bound32)) return won;
            } else {
                double lb = (FAM == 3) ? lower3_64((uint64_t)i, ew.w_inv) : lower4_64(T, (uint32_t)i, ew.w_inv);
                if (lb > ld_volatile(&c.ts->bound64)) return won;
            }
        }
        // point value
        bool beyond;
        float x32 = 0.0f;
        if constexpr (F32) {
            if (FAM == 1) { s32 = __fadd_rn(s32, exp1_32(vw)); x32 = __fmul_rn(ew.winv32, s32); }
            else if (FAM == 2) { s32 = __fadd_rn(s32, __fmul_rn(T.beta32[i], exp1_32(vw))); x32 = __fmul_rn(ew.winv32, s32); }
            else if (FAM == 3) { x32 = __fmul_rn(ew.winv32, __fadd_rn((float)(i - 1), texp_32(vw, T.c3_32, T.inv3_32))); }
            else {
                float sv;
                if ((uint32_t)i < m) sv = __fadd_rn(T.gamma32[i - 1], __fmul_rn(T.dgamma32[i], texp_32(vw, T.c4_32[i], T.inv4_32[i])));
                else sv = __fadd_rn(T.gamma32[m - 1], __fmul_rn(T.delta32, exp1_32(vw)));
                x32 = __fmul_rn(ew.winv32, sv);
            }
            c.cnt.c[PMH_CNT_POINTS32] += 1;
            beyond = x32 * (1.0f - kEta) > ld_volatile(&c.ts->bound32);
        } else {
            if (FAM == 1) x64 = __dadd_rn(x64, term1_64(vw, ew.w_inv));
            else if (FAM == 2) x64 = __dadd_rn(x64, term2_64(T, vw, (uint32_t)i, ew.w_inv));
            else if (FAM == 3) x64 = point3_64(T, vw, (uint64_t)i, ew.w_inv);
            else x64 = point4_64(T, vw, (uint32_t)i, ew.w_inv);
            c.cnt.c[PMH_CNT_POINTS64] += 1;
            beyond = x64 > ld_volatile(&c.ts->bound64);
        }
        if ((FAM == 1 || FAM == 2) && beyond) return won;   // uncorrelated: points increase
        // label
        uint64_t lw = label_word(key, (uint64_t)i);
        uint32_t k;
        if (FAM == 1 || FAM == 3) k = uniform_int(lw, m);
        else k = fy.step(i - 1, lw, m);
        if (!beyond) {
            bool wi;
            if constexpr (F32) wi = Offer<true>::run(c, k, x32, e);
            else wi = Offer<false>::run(c, k, x64, id);
            if (wi) won = kWon;
        }
        if ((FAM == 2 || FAM == 4) && (uint32_t)i == m) return won;   // the sequence has m points
    }
    // still going after kLSeq points?
    if (FAM == 1 || FAM == 2) return won | kNeedDeep;   // the last point was <= bound
    if (FAM == 4 && (uint32_t)kLSeq >= m) return won;
    bool more;
    if constexpr (F32) {
        float lb = (FAM == 3) ? ew.winv32 * (float)kLSeq : ew.winv32 * T.gamma32[kLSeq];
        more = !(lb * (1.0f - kEta) > ld_volatile(&c.ts->bound32));
    } else {
        double lb = (FAM == 3) ? lower3_64((uint64_t)kLSeq + 1, ew.w_inv) : lower4_64(T, (uint32_t)kLSeq + 1, ew.w_inv);
        more = !(lb > ld_volatile(&c.ts->bound64));
    }
    return won | (more ? kNeedDeep : 0);
}

// ------------------------------------------------------------ deep mode
// Warp-cooperative expansion of one element from point 1, 32 points per step.
// mode 0: offer points <= bound.  mode 1 (exact search): stop at the first
// point with label `want` and return its canonical FP64 value in *out.
template <int FAM, bool F32, bool EXACT>
__device__ void deep(Ctx<F32> &c, uint32_t e, uint32_t want, double *out) {
    const SketchParams &P = *c.p;
    const Tables &T = P.tab;
    const uint32_t m = P.m;
    const int lane = threadIdx.x & 31;
    const uint64_t id = P.ids[c.beg + e];
    const double w = P.weights[c.beg + e];
    const uint64_t key = mix64(id ^ P.mixed_seed);
    const double w_inv = (EXACT || !F32) ? __drcp_rn(w) : 0.0;
    const float winv32 = winv_scaled(w, c.sigma);
    if (FAM == 2 || FAM == 4) {
        for (uint32_t p = lane; p < m; p += 32) c.perm[p] = (uint16_t)p;
        __syncwarp();
    }
    if (!EXACT) c.cnt.c[PMH_CNT_DEEP] += (lane == 0);
    double carry64 = 0.0;
    float c_hi = 0.0f, c_lo = 0.0f;
    const uint32_t limit = (FAM == 2 || FAM == 4) ? m : P.cap_points;
#pragma unroll 1
    for (uint32_t base = 1;; base += 32) {
        if (base > limit) {
            if (FAM == 1 || FAM == 3) { if (lane == 0) c.ts->status = PMH_ERR_ITER_LIMIT; }
            if (EXACT && lane == 0) *out = __longlong_as_double(0x7FF0000000000001ll);
            return;
        }
        // correlated: the group starts beyond the bound?
        if (!EXACT && FAM >= 3) {
            bool stop;
            if constexpr (F32) {
                float lb = (FAM == 3) ? winv32 * (float)(base - 1) : winv32 * T.gamma32[base - 1];
                stop = lb * (1.0f - kEta) > ld_volatile(&c.ts->bound32);
            } else {
                double lb = (FAM == 3) ? lower3_64(base, w_inv) : lower4_64(T, base, w_inv);
                stop = lb > ld_volatile(&c.ts->bound64);
            }
            if (__shfl_sync(kFull, (int)stop, 0)) return;
        }
        const uint32_t i = base + lane;
        const bool act = i <= limit;
        const uint64_t vw = act ? value_word(key, i) : 0;
        const uint64_t lw = act ? label_word(key, i) : 0;
        // labels
        uint32_t k;
        if (FAM == 1 || FAM == 3) k = uniform_int(lw, m);
        else k = fy_group(c.perm, c.ws->slot, m, base - 1, lw, act);
        if constexpr (EXACT) {
            unsigned hit = __ballot_sync(kFull, act && k == want);
            // FP64 canonical values of this group (needed for the carry and the hit)
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
                if (lane == src) x = (FAM == 3) ? point3_64(T, vw, i, w_inv) : point4_64(T, vw, i, w_inv);
            }
            if (hit) {
                int src = __ffs(hit) - 1;
                double v = __shfl_sync(kFull, x, src);
                if (lane == 0) *out = v;
                c.cnt.c[PMH_CNT_RESOLVED] += (lane == 0);
                return;
            }
            continue;
        }
        // values and offers
        bool last_beyond;
        bool any_win;
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
                float tot = __shfl_sync(kFull, s, 31);
                float sh = __fadd_rn(c_hi, tot);
                float bb = __fsub_rn(sh, c_hi);
                float err = __fadd_rn(__fsub_rn(c_hi, __fsub_rn(sh, bb)), __fsub_rn(tot, bb));
                c_hi = sh;
                c_lo = __fadd_rn(c_lo, err);
            } else if (FAM == 3) {
                x32 = act ? __fmul_rn(winv32, __fadd_rn((float)(i - 1), texp_32(vw, T.c3_32, T.inv3_32))) : 0.0f;
            } else {
                float sv = 0.0f;
                if (act) {
                    if (i < m) sv = __fadd_rn(T.gamma32[i - 1], __fmul_rn(T.dgamma32[i], texp_32(vw, T.c4_32[i], T.inv4_32[i])));
                    else sv = __fadd_rn(T.gamma32[m - 1], __fmul_rn(T.delta32, exp1_32(vw)));
                }
                x32 = __fmul_rn(winv32, sv);
            }
            c.cnt.c[PMH_CNT_POINTS32] += act;
            const float b32 = ld_volatile(&c.ts->bound32);
            const bool beyond = x32 * (1.0f - kEta) > b32;
            bool wi = false;
            if (act && !beyond) wi = Offer<true>::run(c, k, x32, e);
            any_win = __any_sync(kFull, wi);
            const int last = (int)min((uint32_t)31, limit - base);
            last_beyond = __shfl_sync(kFull, (int)beyond, last);
        } else {
            double x;
            if (FAM == 1 || FAM == 2) {
                double t = act ? (FAM == 1 ? term1_64(vw, w_inv) : term2_64(T, vw, i, w_inv)) : 0.0;
                double run = carry64;
                x = 0.0;
                for (int s = 0; s < 32; ++s) {
                    double ts = __shfl_sync(kFull, t, s);
                    run = __dadd_rn(run, ts);
                    if (lane == s) x = run;
                }
                carry64 = run;
            } else if (FAM == 3) {
                x = act ? point3_64(T, vw, i, w_inv) : 0.0;
            } else {
                x = act ? point4_64(T, vw, i, w_inv) : 0.0;
            }
            c.cnt.c[PMH_CNT_POINTS64] += act;
            const double b64 = ld_volatile(&c.ts->bound64);
            const bool beyond = x > b64;
            bool wi = false;
            if (act && !beyond) wi = Offer<false>::run(c, k, x, id);
            any_win = __any_sync(kFull, wi);
            const int last = (int)min((uint32_t)31, limit - base);
            last_beyond = __shfl_sync(kFull, (int)beyond, last);
        }
        if (base + 31 >= limit && (FAM == 2 || FAM == 4)) return;
        if ((FAM == 1 || FAM == 2) && last_beyond) return;
        // keep q_max fresh while expanding (after groups that changed a minimum)
        int uf = __shfl_sync(kFull, lane == 0 ? ld_volatile(&c.ts->unfilled) : 1, 0);
        if (uf == 0 && any_win) refresh_bound<F32>(c);
    }
}

// Exact FP64 value of h_k(e) (the first point of element e with label k).
template <int FAM, bool F32>
__device__ double exact_h(Ctx<F32> &c, uint32_t e, uint32_t k) {
    __shared__ double xs[32];   // per warp slot (the warp's index)
    const int warp = threadIdx.x >> 5;
    deep<FAM, F32, true>(c, e, k, &xs[warp]);
    __syncwarp();
    double v = xs[warp];
    __syncwarp();
    return v;
}

// ------------------------------------------------------------ team helpers
template <bool CTA_TEAM>
__device__ __forceinline__ void team_sync() {
    if (CTA_TEAM) __syncthreads(); else __syncwarp();
}

// Combines two scaled sums s1*2^e1 + s2*2^e2.
__device__ __forceinline__ void combine_sum(float &s, int &e, float s2, int e2) {
    if (s2 == 0.0f) return;
    if (s == 0.0f) { s = s2; e = e2; return; }
    if (e2 > e) { s = ldexpf(s, max(e - e2, -200)); e = e2; }
    else s2 = ldexpf(s2, max(e2 - e, -200));
    s += s2;
}

// ------------------------------------------------------------ one item
template <int FAM, bool F32, bool CTA_TEAM>
__device__ void process_item(Ctx<F32> &c, int item_v, int64_t set) {
    const SketchParams &P = *c.p;
    const uint32_t m = P.m;
    const int lane = threadIdx.x & 31;
    const int tw = CTA_TEAM ? (threadIdx.x >> 5) : 0;
    const int team_warps = CTA_TEAM ? (blockDim.x >> 5) : 1;
    const int tt = tw * 32 + lane;
    const int team_threads = team_warps * 32;
    TeamShared *ts = c.ts;
    const bool leader = (tt == 0);
    const int64_t out_row = (int64_t)item_v * P.num_sets + set;

    // ---- init
    for (uint32_t k = tt; k < m; k += team_threads) {
        if constexpr (F32) ((uint64_t *)c.sig)[k] = kEmptyKey;
        else { ((Rec64 *)c.sig)[k].q = __longlong_as_double(0x7FF0000000000000ll); ((Rec64 *)c.sig)[k].id = 0; }
    }
    // ---- pass 0: validate weights, scaled weight sum
    float s = 0.0f;
    int se = -100000, bad = 0, npos = 0;
    for (uint32_t e = tt; e < c.n; e += team_threads) {
        double w = P.weights[c.beg + e];
        uint64_t b = (uint64_t)__double_as_longlong(w);
        uint32_t ex = (uint32_t)(b >> 52) & 0x7FF;
        uint64_t mant = b & 0xFFFFFFFFFFFFFull;
        bool neg = (b >> 63) != 0;
        if (ex == 0x7FF) { bad = 1; continue; }
        if (neg) { if (ex != 0 || mant != 0) bad = 1; continue; }
        if (ex == 0 && mant == 0) continue;
        if (ex == 0) {
            double r = __drcp_rn(w);
            if (isinf(r)) { bad = 1; continue; }
        }
        npos++;
        int ew = (ex == 0) ? -1075 : (int)ex - 1023;
        float mf = __uint_as_float(0x3F800000u | (uint32_t)(mant >> 29));   // [1,2)
        combine_sum(s, se, mf, ew);
    }
    for (int o = 16; o; o >>= 1) {
        float s2 = __shfl_xor_sync(kFull, s, o);
        int e2 = __shfl_xor_sync(kFull, se, o);
        combine_sum(s, se, s2, e2);
        bad |= __shfl_xor_sync(kFull, bad, o);
        npos += __shfl_xor_sync(kFull, npos, o);
    }
    if (lane == 0) { ts->red_s[tw] = s; ts->red_e[tw] = se; ts->red_i[tw] = bad | (npos << 1); }
    team_sync<CTA_TEAM>();
    if (leader) {
        float S = 0.0f;
        int E = -100000, B = 0, NP = 0;
        for (int w = 0; w < team_warps; ++w) {
            combine_sum(S, E, ts->red_s[w], ts->red_e[w]);
            B |= ts->red_i[w] & 1;
            NP += ts->red_i[w] >> 1;
        }
        ts->status = B ? PMH_ERR_BAD_WEIGHT : PMH_OK;
        ts->n_pos = NP;
        ts->unfilled = (int)m;
        ts->cont_n = 0;
        // T = m (ln m + c) / sum(w) = t_s * 2^-sigma with t_s in [1, 2)
        int sigma = 0;
        float t_s = 1.0f;
        if (NP > 0) {
            float num = (float)m * P.t_factor / S;
            int en;
            float fr = frexpf(num, &en);   // num = fr * 2^en, fr in [0.5, 1)
            t_s = 2.0f * fr;
            sigma = E - (en - 1);
        }
        ts->sigma = sigma;
        ts->t_s = t_s;
    }
    team_sync<CTA_TEAM>();
    const int st0 = ts->status;
    const int np = ts->n_pos;
    c.sigma = ts->sigma;
    if (st0 != PMH_OK || np == 0) {
        // bad weights or empty set: zero ids, +inf q
        for (uint32_t k = tt; k < m; k += team_threads) {
            P.out_ids[out_row * m + k] = 0;
            if (P.out_q) P.out_q[out_row * m + k] = __longlong_as_double(0x7FF0000000000000ll);
        }
        if (leader && P.status) P.status[out_row] = st0;
        return;
    }

    // ---- rounds
    WarpShared *ws = c.ws;
    for (int round = 0; round <= P.rounds; ++round) {
        if (leader) {
            if (round < P.rounds) {
                float b = ldexpf(ts->t_s, 2 * round);
                ts->bound32 = b;
                ts->bound64 = ldexp((double)ts->t_s, 2 * round - c.sigma);
            } else {
                ts->bound32 = __int_as_float(0x7F800000);
                ts->bound64 = __longlong_as_double(0x7FF0000000000000ll);
            }
            if (round > 0) c.cnt.c[PMH_CNT_ROUNDS] += 1;
        }
        team_sync<CTA_TEAM>();
        bool refreshed = false;
        for (uint32_t base = tw * 32; base < c.n; base += team_warps * 32) {
            const uint32_t e = base + lane;
            int r = 0;
            if (e < c.n) {
                const double w = P.weights[c.beg + e];
                if (w > 0.0) {
                    const uint64_t id = P.ids[c.beg + e];
                    r = stage_a<FAM, F32>(c, e, id, w);
                }
            }
            const bool need = (r & kNeedDeep) != 0;
            const bool any_win = __any_sync(kFull, (r & kWon) != 0);
            // warp queue of long sequences
            unsigned msk = __ballot_sync(kFull, need);
            if (msk) {
                if (need) ws->dq[__popc(msk & ((1u << lane) - 1u))] = e;
                __syncwarp();
                const int cnt = __popc(msk);
                for (int j = 0; j < cnt; ++j) {
                    const uint32_t de = ws->dq[j];
                    deep<FAM, F32, false>(c, de, 0, nullptr);
                }
                __syncwarp();
            }
            // refresh q_max once everything is filled
            int uf = __shfl_sync(kFull, lane == 0 ? ld_volatile(&ts->unfilled) : 1, 0);
            if (uf == 0 && (!refreshed || msk || any_win)) {
                refresh_bound<F32>(c);
                refreshed = true;
            }
        }
        team_sync<CTA_TEAM>();
        if (ld_volatile(&ts->unfilled) == 0 || ld_volatile(&ts->status) != PMH_OK) break;
        team_sync<CTA_TEAM>();
    }
    team_sync<CTA_TEAM>();

    // ---- FP32: resolve contenders exactly
    if constexpr (F32) if (tw == 0) {
        Ctx<F32> &cc = c;
        const int ncont_all = ld_volatile(&ts->cont_n);
        if (ncont_all > kMaxCont) { if (lane == 0) ts->status = PMH_ERR_ITER_LIMIT; }
        const int ncont = min(ncont_all, kMaxCont);
        uint64_t *sig = (uint64_t *)cc.sig;
        for (int a = 0; a < ncont; ++a) {
            const uint32_t k = ts->cont_k[a];
            bool seen = false;
            for (int b = 0; b < a; ++b) seen |= (ts->cont_k[b] == k);
            if (seen) continue;
            const uint64_t hk = sig[k];
            uint32_t best_e = (uint32_t)(hk & 0xFFFFFFFFu);
            double best_x = exact_h<FAM, F32>(cc, best_e, k);
            uint64_t best_id = P.ids[c.beg + best_e];
            for (int b = a; b < ncont; ++b) {
                if (ts->cont_k[b] != k) continue;
                const uint32_t ce = ts->cont_e[b];
                if (ce == best_e) continue;
                double x = exact_h<FAM, F32>(cc, ce, k);
                uint64_t cid = P.ids[c.beg + ce];
                if (x < best_x || (x == best_x && cid < best_id)) { best_x = x; best_id = cid; best_e = ce; }
            }
            if (lane == 0) sig[k] = (hk & 0xFFFFFFFF00000000ull) | best_e;
            __syncwarp();
        }
    }
    team_sync<CTA_TEAM>();

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
                if (key != kEmptyKey && st == PMH_OK) q = exact_h<FAM, F32>(c, (uint32_t)(key & 0xFFFFFFFFu), k);
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
}

// ------------------------------------------------------------ kernel
template <bool F32, int NW, bool CTA_TEAM>
__global__ void __launch_bounds__(NW * 32) sketch_kernel(SketchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int teams = CTA_TEAM ? 1 : NW;
    const int team = CTA_TEAM ? 0 : warp;
    SmemLayout L(teams, NW, p.m, F32, p.has_perm != 0);
    TeamShared *ts = (TeamShared *)(smem + L.team_off + (size_t)team * align16(sizeof(TeamShared)));
    Ctx<F32> c;
    c.p = &p;
    c.ts = ts;
    c.sig = smem + L.sig_off + (size_t)team * p.m * (F32 ? 8 : 16);
    c.ws = (WarpShared *)(smem + L.warp_off + (size_t)warp * align16(sizeof(WarpShared)));
    c.perm = p.has_perm ? (uint16_t *)(smem + L.perm_off + (size_t)warp * p.m * 2) : nullptr;
    for (int j = 0; j < PMH_NUM_COUNTERS; ++j) c.cnt.c[j] = 0;
    const bool team_leader = CTA_TEAM ? (threadIdx.x == 0) : (lane == 0);
    for (;;) {
        if (team_leader) ts->item_idx = (int)atomicAdd(p.head, 1u);
        team_sync<CTA_TEAM>();
        const int64_t qi = ts->item_idx;
        team_sync<CTA_TEAM>();
        if (qi >= p.queue_len) break;
        const uint64_t it = p.queue[qi];
        const int v = (int)(it >> 40);
        const int64_t set = (int64_t)(it & ((1ull << 40) - 1));
        const int64_t b = p.offsets[set], e = p.offsets[set + 1];
        const int64_t out_row = (int64_t)v * p.num_sets + set;
        if (e < b || e - b > (int64_t)PMH_MAX_SET_ELEMENTS) {
            const int code = e < b ? PMH_ERR_INVALID_ARG : PMH_ERR_UNSUPPORTED;
            const int tt = CTA_TEAM ? threadIdx.x : lane;
            const int nthr = CTA_TEAM ? blockDim.x : 32;
            for (uint32_t k = tt; k < p.m; k += nthr) {
                p.out_ids[out_row * p.m + k] = 0;
                if (p.out_q) p.out_q[out_row * p.m + k] = __longlong_as_double(0x7FF0000000000000ll);
            }
            if (team_leader && p.status) p.status[out_row] = code;
            continue;
        }
        c.beg = b;
        c.n = (uint32_t)(e - b);
        const int fam = family_of(p.variants[v]);
        switch (fam) {
            case 1: process_item<1, F32, CTA_TEAM>(c, v, set); break;
            case 2: process_item<2, F32, CTA_TEAM>(c, v, set); break;
            case 3: process_item<3, F32, CTA_TEAM>(c, v, set); break;
            default: process_item<4, F32, CTA_TEAM>(c, v, set); break;
        }
        team_sync<CTA_TEAM>();
    }
    if (p.counters) {
        for (int j = 0; j < PMH_NUM_COUNTERS; ++j) {
            unsigned long long v = c.cnt.c[j];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0 && v) atomicAdd(&p.counters[j], v);
        }
    }
}

}  // namespace pmh
