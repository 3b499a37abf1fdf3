// Instantiation of the persistent sketch kernel for one (precision, family);
// included by sketch_<precision>_f<family>.cu with PMH_F32 and PMH_FAM defined.
#include "launch.h"

namespace pmh {

namespace {
template <bool CTA>
cudaError_t shape_impl(uint32_t m, bool has_perm, LaunchShape *out) {
    constexpr int NW = CTA ? 8 : 4;
    const int teams = CTA ? 1 : NW;
    (void)has_perm;
    SmemLayout L(teams, NW, m, PMH_F32, PMH_FAM == 2 || PMH_FAM == 4);
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
    auto kern = sketch_kernel<PMH_F32, NW, CTA, PMH_FAM>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->blocks_per_sm, kern, NW * 32, L.total);
}
}  // namespace

template <>
cudaError_t sketch_shape<PMH_F32, PMH_FAM>(bool cta_team, uint32_t m, bool has_perm, LaunchShape *out) {
    return cta_team ? shape_impl<true>(m, has_perm, out) : shape_impl<false>(m, has_perm, out);
}

template <>
cudaError_t sketch_launch<PMH_F32, PMH_FAM>(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    if (s.cta_team) sketch_kernel<PMH_F32, 8, true, PMH_FAM><<<grid, s.block, s.smem, st>>>(p);
    else sketch_kernel<PMH_F32, 4, false, PMH_FAM><<<grid, s.block, s.smem, st>>>(p);
    return cudaGetLastError();
}

template <>
cudaError_t grid_shape<PMH_F32, PMH_FAM>(uint32_t m, LaunchShape *out) {
    SmemLayout L(1, 8, m, PMH_F32, PMH_FAM == 2 || PMH_FAM == 4);
    out->cta_team = true;
    out->block = 256;
    out->smem = L.total;
    out->blocks_per_sm = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (L.total > (size_t)optin) return cudaSuccess;
    auto kern = grid_kernel<PMH_F32, PMH_FAM>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->blocks_per_sm, kern, 256, L.total);
}

template <>
cudaError_t grid_launch<PMH_F32, PMH_FAM>(const LaunchShape &s, int grid, const SketchParams &p, cudaStream_t st) {
    grid_kernel<PMH_F32, PMH_FAM><<<grid, s.block, s.smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace pmh
