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

// One persistent kernel per (precision, team shape, family): each launch holds
// only its own family's code.  Defined in sketch_<precision>_f<family>.cu.
template <bool F32, int FAM>
cudaError_t sketch_shape(bool cta_team, uint32_t m, bool has_perm, LaunchShape *out);
template <bool F32, int FAM>
cudaError_t sketch_launch(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);

// Records the message returned by pmh_last_error(NULL) on this host thread.
void set_thread_error(const char *msg);

// Grid-mode kernel of one (precision, family): a CTA-team launch shape.
template <bool F32, int FAM>
cudaError_t grid_shape(uint32_t m, LaunchShape *out);
template <bool F32, int FAM>
cudaError_t grid_launch(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);
cudaError_t grid_shape_any(bool f32, int fam, uint32_t m, LaunchShape *out);
cudaError_t grid_launch_any(bool f32, int fam, const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st);

// Dispatch on (precision, family) at run time.
cudaError_t sketch_shape_any(bool f32, int fam, bool cta_team, uint32_t m, bool has_perm, LaunchShape *out);
cudaError_t sketch_launch_any(bool f32, int fam, const LaunchShape &s, int grid, const SketchParams &p,
                              cudaStream_t st);

}  // namespace pmh
