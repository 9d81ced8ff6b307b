// Instantiations and launcher of the 3D stencil kernel, mode: fwd.
#include "kernels.cuh"
#include "stencil3d.cuh"

namespace wp {

template <int R>
static cudaError_t launch_t(dim3 grid, cudaStream_t st, const CUtensorMap *maps, const Stencil3dArgs &a) {
  constexpr int bytes = Smem3d<R, kModeFwd>::BYTES;
  stencil3d_kernel<R, kModeFwd><<<grid, kThreads3d, bytes, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4],
                                                            maps[5], a);
  return cudaGetLastError();
}

template <int R>
static cudaError_t prepare_t(int *smem_bytes, int *blocks_per_sm) {
  constexpr int bytes = Smem3d<R, kModeFwd>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(stencil3d_kernel<R, kModeFwd>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  *smem_bytes = bytes;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stencil3d_kernel<R, kModeFwd>,
                                                       kThreads3d, bytes);
}

#define WP_DISPATCH(F, ...)                 \
  switch (R) {                              \
    case 1: return F<1>(__VA_ARGS__);       \
    case 2: return F<2>(__VA_ARGS__);       \
    case 3: return F<3>(__VA_ARGS__);       \
    case 4: return F<4>(__VA_ARGS__);       \
    case 5: return F<5>(__VA_ARGS__);       \
    case 6: return F<6>(__VA_ARGS__);       \
    case 7: return F<7>(__VA_ARGS__);       \
    case 8: return F<8>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;  \
  }

cudaError_t launch_stencil3d_fwd(int R, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                  const Stencil3dArgs &a) {
  WP_DISPATCH(launch_t, grid, st, maps, a)
}

cudaError_t prepare_stencil3d_fwd(int R, int *smem_bytes, int *blocks_per_sm) {
  WP_DISPATCH(prepare_t, smem_bytes, blocks_per_sm)
}

}  // namespace wp
