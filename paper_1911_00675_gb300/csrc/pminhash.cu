// P-MinHash on the GPU (Algorithm P-MinHash, the paper's state of the art for
// J_P before ProbMinHash): every element d with w(d) > 0 gets m independent
// values h_k(d) = Exp(1) / w(d), and component k keeps the element with the
// lexicographically smallest (h_k(d), d) (Eq. signature_def).  There is no
// early stop: O(n m) hash values per set, against ProbMinHash's O(n + m log m)
// for large n, which is the comparison the paper's experiments draw.
//
// Stream: h_k(d) uses word k (0-based) of the element's counter-based stream,
// key(d) = mix(d ^ mix(seed)), word_j = mix(key + (j+1) phi).
//
// GPU design: one 256-thread block per set (blocks take sets from a counter);
// each thread owns the components k = tid, tid + 256, ..., keeps their current
// holder in shared memory (its FP32 value, its index in the set, and its exact
// FP64 value once computed), and walks the set's elements in tiles of 256
// staged in shared memory (key, FP32 scaled 1/w, FP64 1/w, id, index).
// Candidates are compared in FP32 (within kEta of the exact values): one
// clearly below the holder replaces it, one clearly above is dropped, and only
// the rare candidate within the error margin of the holder is compared exactly
// in FP64 (lexicographically with the id).  The output therefore equals the
// all-FP64 computation, while FP64 work stays proportional to the near ties
// (plus one exact value per component when out_q is asked for).
#include "batch_common.cuh"

using namespace pmh;

namespace {

constexpr int kPmBlock = 256;
constexpr int kPmTile = 256;
constexpr uint32_t kNoHolder = 0xFFFFFFFFu;

// One staged element.  winv32 = 2^sigma / w in FP32 (0: empty slot).  exact: the
// scaled weight is below the FP32 range, so the element's values are always
// compared in FP64 (its FP32 values carry no error bound).
struct __align__(16) PmElem {
    uint64_t key;
    uint64_t id;
    double w_inv;
    float winv32;
    uint32_t idx;      // index in the set
    int exact;
};

__device__ __forceinline__ double pm_exact(uint64_t key, double w_inv, uint64_t ctr) {
    return __dmul_rn(w_inv, exp1_64(mix64(key + ctr)));
}
// Exact value of component k's current holder (element `idx` of the set at b).
__device__ __forceinline__ double pm_holder_exact(const uint64_t *ids, const double *weights, int64_t b, uint32_t idx,
                                                  uint64_t mixed_seed, uint64_t ctr) {
    return pm_exact(mix64(ids[b + idx] ^ mixed_seed), __drcp_rn(weights[b + idx]), ctr);
}

__global__ void __launch_bounds__(kPmBlock) pminhash_kernel(const uint64_t *__restrict__ ids,
                                                            const double *__restrict__ weights,
                                                            const int64_t *__restrict__ offsets, int64_t num_sets,
                                                            uint32_t m, uint64_t mixed_seed, unsigned int *next_set,
                                                            uint64_t *__restrict__ out_ids, double *__restrict__ out_q,
                                                            int32_t *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *bx = (double *)smem;                 // holder's exact value (NaN: not computed yet)
    uint32_t *bi = (uint32_t *)(bx + m);         // holder's index in the set (kNoHolder: none)
    float *b32 = (float *)(bi + m);              // holder's FP32 value; sign bit set: an exact-only holder
    PmElem *tile = (PmElem *)(smem + (((size_t)m * 16 + 15) & ~(size_t)15));
    __shared__ long long s_set;
    __shared__ int s_bad, s_maxexp;
    const double kNaN = __longlong_as_double(0x7FF8000000000000ll);
    for (;;) {
        if (threadIdx.x == 0) s_set = (long long)atomicAdd(next_set, 1u);
        __syncthreads();
        const int64_t s = s_set;
        if (s >= num_sets) break;
        const int64_t b = offsets[s], e = offsets[s + 1];
        if (threadIdx.x == 0) { s_bad = 0; s_maxexp = 0; }
        for (uint32_t k = threadIdx.x; k < m; k += kPmBlock) {
            bx[k] = kNaN;
            bi[k] = kNoHolder;
            b32[k] = __int_as_float(0x7F800000);
        }
        __syncthreads();
        if (e < b) {
            for (uint32_t k = threadIdx.x; k < m; k += kPmBlock) {
                out_ids[s * m + k] = 0;
                if (out_q) out_q[s * m + k] = __longlong_as_double(0x7FF0000000000000ll);
            }
            if (threadIdx.x == 0 && status) status[s] = PMH_ERR_INVALID_ARG;
            __syncthreads();
            continue;
        }
        // weight check and the largest exponent: FP32 values are scaled by 2^-sigma so that the
        // heaviest element's scaled weight lies in [1, 2)
        int bad = 0, mx = 0;
        for (int64_t j = b + threadIdx.x; j < e; j += kPmBlock) {
            const uint64_t x = (uint64_t)__double_as_longlong(weights[j]);
            const int ex = (int)(x >> 52) & 0x7FF;
            const bool neg = (x >> 63) != 0, zero = (x << 1) == 0;
            if (ex == 0x7FF || (neg && !zero)) bad = 1;
            else if (!zero && ex == 0 && isinf(__drcp_rn(__longlong_as_double((long long)x)))) bad = 1;
            else if (!zero) mx = max(mx, ex);
        }
        if (bad) atomicOr(&s_bad, 1);
        atomicMax(&s_maxexp, mx);
        __syncthreads();
        const bool set_bad = s_bad != 0;
        const int sigma = s_maxexp - 1023;     // w 2^-sigma < 2 for every weight
        for (int64_t t0 = b; t0 < e && !set_bad; t0 += kPmTile) {
            const int64_t j = t0 + threadIdx.x;
            if (threadIdx.x < kPmTile) {
                PmElem el{};
                el.winv32 = 0.0f;   // empty slot: never a candidate
                if (j < e) {
                    const double w = weights[j];
                    if (weight_positive(w)) {
                        el.id = ids[j];
                        el.key = mix64(el.id ^ mixed_seed);
                        el.w_inv = __drcp_rn(w);
                        el.idx = (uint32_t)(j - b);
                        el.exact = ws_scaled(w, sigma) == 0.0f;
                        el.winv32 = el.exact ? 1.0f : winv_scaled(w, sigma);
                    }
                }
                tile[threadIdx.x] = el;
            }
            __syncthreads();
            const int cnt = (int)min((int64_t)kPmTile, e - t0);
            for (uint32_t k = threadIdx.x; k < m; k += kPmBlock) {
                double hx = bx[k];
                uint32_t hi = bi[k];
                float h32 = b32[k];
                const uint64_t ctr = ((uint64_t)k + 1) * kPhi;
                for (int q = 0; q < cnt; ++q) {
                    const PmElem el = tile[q];
                    if (el.winv32 == 0.0f) continue;
                    const uint64_t word = mix64(el.key + ctr);
                    const float x32 = __fmul_rn(el.winv32, exp1_32(word));
                    // both FP32 values lie within kEta of the exact scaled ones; 4 kEta also covers
                    // the products' rounding.  An exact-only element or holder is compared in FP64.
                    const bool exact_path = el.exact || __float_as_int(h32) < 0;
                    if (!exact_path && x32 < __fmul_rn(h32, 1.0f - 4.0f * kEta)) {
                        h32 = x32;             // clearly below the holder (or no holder yet)
                        hi = el.idx;
                        hx = kNaN;
                    } else if (exact_path || __fmul_rn(x32, 1.0f - 4.0f * kEta) <= h32) {
                        // within the margin: compare the exact values, then the ids
                        const double x = __dmul_rn(el.w_inv, exp1_64(word));
                        bool take = hi == kNoHolder;
                        if (!take) {
                            if (isnan(hx)) hx = pm_holder_exact(ids, weights, b, hi, mixed_seed, ctr);
                            take = x < hx || (x == hx && el.id < ids[b + hi]);
                        }
                        if (take) {
                            hx = x;
                            hi = el.idx;
                            // an exact-only holder keeps its scaled value rounded up, marked by the sign bit
                            h32 = el.exact ? -__double2float_ru(ldexp(x, sigma)) : x32;
                        }
                    }
                }
                bx[k] = hx;
                bi[k] = hi;
                b32[k] = h32;
            }
            __syncthreads();
        }
        for (uint32_t k = threadIdx.x; k < m; k += kPmBlock) {
            const uint32_t hi = bi[k];
            const bool ok = !set_bad && hi != kNoHolder;
            out_ids[s * m + k] = ok ? ids[b + hi] : 0;
            if (out_q) {
                double q = __longlong_as_double(0x7FF0000000000000ll);
                if (ok) q = isnan(bx[k]) ? pm_holder_exact(ids, weights, b, hi, mixed_seed, ((uint64_t)k + 1) * kPhi) : bx[k];
                out_q[s * m + k] = q;
            }
        }
        if (threadIdx.x == 0 && status) status[s] = set_bad ? PMH_ERR_BAD_WEIGHT : PMH_OK;
        __syncthreads();
    }
}

}  // namespace

// Launches the P-MinHash kernel on `st`: one block per set at a time, blocks
// taking sets from *set_counter (device, reset here).  Returns the CUDA error
// of the set-up or launch; *fits = false when m's shared memory does not fit.
cudaError_t pmh::pminhash_launch(const uint64_t *ids, const double *weights, const int64_t *offsets, int64_t num_sets,
                                 uint32_t m, uint64_t seed, uint64_t *out_ids, double *out_q, int32_t *set_status,
                                 unsigned int *set_counter, int sm_count, cudaStream_t st, bool *fits) {
    const size_t smem = (((size_t)m * 16 + 15) & ~(size_t)15) + (size_t)kPmTile * sizeof(PmElem);
    *fits = true;
    cudaError_t e = cudaFuncSetAttribute(pminhash_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pminhash_kernel, kPmBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) { *fits = false; return cudaSuccess; }
    if ((e = cudaMemsetAsync(set_counter, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(num_sets, (int64_t)sm_count * per_sm);
    pminhash_kernel<<<grid, kPmBlock, smem, st>>>(ids, weights, offsets, num_sets, m, host_mix64(seed), set_counter,
                                                  out_ids, out_q, set_status);
    return cudaGetLastError();
}
