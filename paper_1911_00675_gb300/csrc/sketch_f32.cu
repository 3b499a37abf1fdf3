// Instantiation of the persistent sketch kernel for the FP32 candidate + FP64 recheck path.
#include "launch.h"

namespace pmh {

namespace {
template <bool CTA>
cudaError_t shape_impl(uint32_t m, bool has_perm, LaunchShape *out) {
    constexpr int NW = CTA ? 8 : 4;
    const int teams = CTA ? 1 : NW;
    SmemLayout L(teams, NW, m, true, has_perm);
    out->cta_team = CTA;
    out->block = NW * 32;
    out->smem = L.total;
    out->blocks_per_sm = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (L.total > (size_t)optin) return cudaSuccess;
    e = cudaFuncSetAttribute(sketch_kernel<true, NW, CTA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->blocks_per_sm, sketch_kernel<true, NW, CTA>, NW * 32,
                                                         L.total);
}
}  // namespace

cudaError_t sketch_shape_f32(bool cta_team, uint32_t m, bool has_perm, LaunchShape *out) {
    return cta_team ? shape_impl<true>(m, has_perm, out) : shape_impl<false>(m, has_perm, out);
}

cudaError_t sketch_launch_f32(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    if (s.cta_team) sketch_kernel<true, 8, true><<<grid, s.block, s.smem, st>>>(p);
    else sketch_kernel<true, 4, false><<<grid, s.block, s.smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace pmh
