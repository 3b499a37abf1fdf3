// Internal launch interface between the host API and the per-precision
// kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "sketch_kernel.cuh"

namespace pmh {

struct LaunchShape {
    bool cta_team;      // true: one CTA of 8 warps per item; false: 4 independent warp teams per CTA
    int block;          // threads per block
    size_t smem;        // dynamic shared memory per block
    int blocks_per_sm;  // occupancy (0 = does not fit)
};

// Occupancy of the sketch kernel for (precision, team shape, m, permutation arrays).
cudaError_t sketch_shape_f32(bool cta_team, uint32_t m, bool has_perm, LaunchShape *out);
cudaError_t sketch_shape_f64(bool cta_team, uint32_t m, bool has_perm, LaunchShape *out);
cudaError_t sketch_launch_f32(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);
cudaError_t sketch_launch_f64(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);

}  // namespace pmh
