// Instantiations and launcher of the 3D stencil kernel, mode: fwd.
#include "kernels.cuh"
#include "stencil3d.cuh"

namespace wp {

template <int R>
static cudaError_t launch_t(dim3 grid, cudaStream_t st, const CUtensorMap *m, const Stencil3dArgs &a) {
  return launch_kernel(stencil3d_kernel<R, kModeFwd>, grid, dim3(kThreads3d), Cfg3d<R, kModeFwd>::SMEM, st, a.pdl != 0, m[0],
                       m[1], m[2], m[3], m[4], m[5], a);
}

template <int R>
static cudaError_t prepare_t(int *smem_bytes, int *blocks_per_sm, int *tile_y) {
  constexpr int bytes = Cfg3d<R, kModeFwd>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(stencil3d_kernel<R, kModeFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  *smem_bytes = bytes;
  *tile_y = Cfg3d<R, kModeFwd>::TY;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stencil3d_kernel<R, kModeFwd>, kThreads3d, bytes);
}

#define WP_DISPATCH(F, ...)                 \
  switch (R) {                              \
    case 1: return F<1>(__VA_ARGS__);       \
    case 2: return F<2>(__VA_ARGS__);       \
    case 3: return F<3>(__VA_ARGS__);       \
    case 4: return F<4>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;  \
  }

cudaError_t launch_stencil3d_fwd(int R, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                  const Stencil3dArgs &a) {
  if (R > 4) return launch_stencil3d_hi(R, kModeFwd, grid, st, maps, a);
  WP_DISPATCH(launch_t, grid, st, maps, a)
}

template <int R>
static int tile_x_t() {
  return Cfg3d<R, kModeFwd>::TX;
}

int stencil3d_tile_x_fwd(int R) {
  switch (R) {
    case 1: return tile_x_t<1>();
    case 2: return tile_x_t<2>();
    case 3: return tile_x_t<3>();
    case 4: return tile_x_t<4>();
    default: return stencil3d_hi_tile_x(R, kModeFwd);
  }
}

template <int R>
static int tile_y_t() {
  return Cfg3d<R, kModeFwd>::TY;
}

int stencil3d_tile_y_fwd(int R) {
  switch (R) {
    case 1: return tile_y_t<1>();
    case 2: return tile_y_t<2>();
    case 3: return tile_y_t<3>();
    case 4: return tile_y_t<4>();
    default: return stencil3d_hi_tile_y(R, kModeFwd);
  }
}

cudaError_t prepare_stencil3d_fwd(int R, int *smem_bytes, int *blocks_per_sm, int *tile_y) {
  if (R > 4) return prepare_stencil3d_hi(R, kModeFwd, smem_bytes, blocks_per_sm, tile_y);
  WP_DISPATCH(prepare_t, smem_bytes, blocks_per_sm, tile_y)
}

}  // namespace wp
