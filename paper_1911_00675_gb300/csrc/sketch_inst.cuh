// Instantiation of the persistent sketch kernel for one (precision, family);
// included by sketch_<precision>_f<family>.cu with PMH_F32 and PMH_FAM defined.
// ProbMinHash3/3a/4 also get kernels drawing Exp(lambda;0,1) with the
// rejection sampler (REJ = true), launched when the call asks for it, so that
// the default kernels carry none of its code.
#include "launch.h"

namespace pmh {

namespace {
template <int S>
cudaError_t shape_impl(uint32_t m, LaunchShape *out) {
    constexpr int NW = shape_nw(S), TW = shape_tw(S), MINB = shape_minb(S);
    SmemLayout L(NW / TW, NW, m, PMH_F32, PMH_FAM == 2 || PMH_FAM == 4);
    out->kind = S;
    out->block = NW * 32;
    out->team_warps = TW;
    out->smem = L.total;
    out->blocks_per_sm = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (L.total > (size_t)optin) return cudaSuccess;
    auto kern = sketch_kernel<PMH_F32, NW, TW, MINB, PMH_FAM, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    if constexpr (PMH_FAM >= 3) {
        e = cudaFuncSetAttribute(sketch_kernel<PMH_F32, NW, TW, MINB, PMH_FAM, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->blocks_per_sm, kern, NW * 32, L.total);
}
template <int S>
void launch_impl(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    if constexpr (PMH_FAM >= 3) {
        if (p.te_rej) {
            sketch_kernel<PMH_F32, shape_nw(S), shape_tw(S), shape_minb(S), PMH_FAM, true><<<grid, s.block, s.smem, st>>>(p);
            return;
        }
    }
    sketch_kernel<PMH_F32, shape_nw(S), shape_tw(S), shape_minb(S), PMH_FAM, false><<<grid, s.block, s.smem, st>>>(p);
}
}  // namespace

template <>
cudaError_t sketch_shape<PMH_F32, PMH_FAM>(int kind, uint32_t m, LaunchShape *out) {
    switch (kind) {
        case kShapeWarp: return shape_impl<kShapeWarp>(m, out);
        case kShapeCta8: return shape_impl<kShapeCta8>(m, out);
        case kShapeQuad: return shape_impl<kShapeQuad>(m, out);
        case kShapePair: return shape_impl<kShapePair>(m, out);
        case kShapeQuad8: return shape_impl<kShapeQuad8>(m, out);
        default: return shape_impl<kShapeQuad8L>(m, out);
    }
}

template <>
cudaError_t sketch_launch<PMH_F32, PMH_FAM>(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    switch (s.kind) {
        case kShapeWarp: launch_impl<kShapeWarp>(s, grid, p, st); break;
        case kShapeCta8: launch_impl<kShapeCta8>(s, grid, p, st); break;
        case kShapeQuad: launch_impl<kShapeQuad>(s, grid, p, st); break;
        case kShapePair: launch_impl<kShapePair>(s, grid, p, st); break;
        case kShapeQuad8: launch_impl<kShapeQuad8>(s, grid, p, st); break;
        default: launch_impl<kShapeQuad8L>(s, grid, p, st); break;
    }
    return cudaGetLastError();
}

template <>
cudaError_t grid_shape<PMH_F32, PMH_FAM>(uint32_t m, LaunchShape *out) {
    SmemLayout L(1, 8, m, PMH_F32, PMH_FAM == 2 || PMH_FAM == 4);
    out->kind = kShapeCta8;
    out->block = 256;
    out->team_warps = 8;
    out->smem = L.total;
    out->blocks_per_sm = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (L.total > (size_t)optin) return cudaSuccess;
    auto kern = grid_kernel<PMH_F32, PMH_FAM, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    if constexpr (PMH_FAM >= 3) {
        e = cudaFuncSetAttribute(grid_kernel<PMH_F32, PMH_FAM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.total);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->blocks_per_sm, kern, 256, L.total);
}

template <>
cudaError_t grid_launch<PMH_F32, PMH_FAM>(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    if constexpr (PMH_FAM >= 3) {
        if (p.te_rej) {
            grid_kernel<PMH_F32, PMH_FAM, true><<<grid, s.block, s.smem, st>>>(p);
            return cudaGetLastError();
        }
    }
    grid_kernel<PMH_F32, PMH_FAM, false><<<grid, s.block, s.smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace pmh
