// Run-time dispatch to the per-(precision, family) sketch kernels.
#include "launch.h"

namespace pmh {

cudaError_t sketch_shape_any(bool f32, int fam, int kind, uint32_t m, LaunchShape *out) {
    if (f32) {
        switch (fam) {
            case 1: return sketch_shape<true, 1>(kind, m, out);
            case 2: return sketch_shape<true, 2>(kind, m, out);
            case 3: return sketch_shape<true, 3>(kind, m, out);
            default: return sketch_shape<true, 4>(kind, m, out);
        }
    }
    switch (fam) {
        case 1: return sketch_shape<false, 1>(kind, m, out);
        case 2: return sketch_shape<false, 2>(kind, m, out);
        case 3: return sketch_shape<false, 3>(kind, m, out);
        default: return sketch_shape<false, 4>(kind, m, out);
    }
}

cudaError_t sketch_launch_any(bool f32, int fam, const LaunchShape &s, int grid, const SketchParams &p,
                              cudaStream_t st) {
    if (f32) {
        switch (fam) {
            case 1: return sketch_launch<true, 1>(s, grid, p, st);
            case 2: return sketch_launch<true, 2>(s, grid, p, st);
            case 3: return sketch_launch<true, 3>(s, grid, p, st);
            default: return sketch_launch<true, 4>(s, grid, p, st);
        }
    }
    switch (fam) {
        case 1: return sketch_launch<false, 1>(s, grid, p, st);
        case 2: return sketch_launch<false, 2>(s, grid, p, st);
        case 3: return sketch_launch<false, 3>(s, grid, p, st);
        default: return sketch_launch<false, 4>(s, grid, p, st);
    }
}

cudaError_t grid_shape_any(bool f32, int fam, uint32_t m, LaunchShape *out) {
    if (f32) {
        switch (fam) {
            case 1: return grid_shape<true, 1>(m, out);
            case 2: return grid_shape<true, 2>(m, out);
            case 3: return grid_shape<true, 3>(m, out);
            default: return grid_shape<true, 4>(m, out);
        }
    }
    switch (fam) {
        case 1: return grid_shape<false, 1>(m, out);
        case 2: return grid_shape<false, 2>(m, out);
        case 3: return grid_shape<false, 3>(m, out);
        default: return grid_shape<false, 4>(m, out);
    }
}

cudaError_t grid_launch_any(bool f32, int fam, const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    if (f32) {
        switch (fam) {
            case 1: return grid_launch<true, 1>(s, grid, p, st);
            case 2: return grid_launch<true, 2>(s, grid, p, st);
            case 3: return grid_launch<true, 3>(s, grid, p, st);
            default: return grid_launch<true, 4>(s, grid, p, st);
        }
    }
    switch (fam) {
        case 1: return grid_launch<false, 1>(s, grid, p, st);
        case 2: return grid_launch<false, 2>(s, grid, p, st);
        case 3: return grid_launch<false, 3>(s, grid, p, st);
        default: return grid_launch<false, 4>(s, grid, p, st);
    }
}

}  // namespace pmh
