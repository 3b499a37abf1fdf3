// Internal launch interface between the host API and the per-precision
// kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "sketch_kernel.cuh"

namespace pmh {

// Team shapes of the persistent sketch kernel: warps per block, warps per
// team (sharing one signature) and the blocks per SM its registers are sized
// for (65,536 / (minb * threads) registers per thread).
enum TeamShape : int {
    kShapeWarp = 0,    // 4 warps per block, every warp its own team (96 registers)
    kShapeCta8 = 1,    // 8 warps per block, one team (128 registers)
    kShapeQuad = 2,    // 4 warps per block, one team (64 registers)
    kShapePair = 3,    // 8 warps per block, teams of 2 warps (64 registers)
    kShapeQuad8 = 4,   // 8 warps per block, teams of 4 warps (64 registers)
    kShapeQuad8L = 5,  // 8 warps per block, teams of 4 warps (48 registers)
    kNumShapes = 6
};
struct ShapeDims {
    int nw, tw, minb;
};
constexpr ShapeDims kShapeDims[kNumShapes] = {{4, 1, 5}, {8, 8, 2}, {4, 4, 8}, {8, 2, 4}, {8, 4, 4}, {8, 4, 5}};
constexpr int shape_nw(int s) { return kShapeDims[s].nw; }
constexpr int shape_tw(int s) { return kShapeDims[s].tw; }
constexpr int shape_minb(int s) { return kShapeDims[s].minb; }

struct LaunchShape {
    int kind;           // TeamShape
    int block;          // threads per block
    int team_warps;     // warps per team
    size_t smem;        // dynamic shared memory per block
    int blocks_per_sm;  // occupancy (0 = does not fit)
};

// One persistent kernel per (precision, team shape, family): each launch holds
// only its own family's code.  Defined in sketch_<precision>_f<family>.cu.
template <bool F32, int FAM>
cudaError_t sketch_shape(int kind, uint32_t m, LaunchShape *out);
template <bool F32, int FAM>
cudaError_t sketch_launch(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);

// Records the message returned by pmh_last_error(NULL) on this host thread.
void set_thread_error(const char *msg);

// Algorithm P-MinHash over a CSR batch (pminhash.cu).
cudaError_t pminhash_launch(const uint64_t *ids, const double *weights, const int64_t *offsets, int64_t num_sets,
                            uint32_t m, uint64_t seed, uint64_t *out_ids, double *out_q, int32_t *set_status,
                            unsigned int *set_counter, int sm_count, cudaStream_t st, bool *fits);

// Grid-mode kernel of one (precision, family): a CTA-team launch shape.
template <bool F32, int FAM>
cudaError_t grid_shape(uint32_t m, LaunchShape *out);
template <bool F32, int FAM>
cudaError_t grid_launch(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);
cudaError_t grid_shape_any(bool f32, int fam, uint32_t m, LaunchShape *out);
cudaError_t grid_launch_any(bool f32, int fam, const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);

// Dispatch on (precision, family) at run time.
cudaError_t sketch_shape_any(bool f32, int fam, int kind, uint32_t m, LaunchShape *out);
cudaError_t sketch_launch_any(bool f32, int fam, const LaunchShape &s, int grid, const SketchParams &p,
                              cudaStream_t st);

}  // namespace pmh
