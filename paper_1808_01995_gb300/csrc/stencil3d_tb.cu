// Instantiations and launcher of the two-step (temporally blocked) 3D stencil.
#include "kernels.cuh"
#include "stencil3d_tb.cuh"

namespace wp {

template <int R>
static cudaError_t launch_tb_t(dim3 grid, cudaStream_t st, const CUtensorMap *m, const Stencil3dTbArgs &a) {
  stencil3d_tb_kernel<R><<<grid, kThreadsTb, CfgTb<R>::SMEM, st>>>(m[0], m[1], m[2], m[3], m[4], m[5], a);
  return cudaGetLastError();
}

template <int R>
static cudaError_t prepare_tb_t(int *smem_bytes, int *blocks_per_sm) {
  constexpr int bytes = CfgTb<R>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(stencil3d_tb_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  *smem_bytes = bytes;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stencil3d_tb_kernel<R>, kThreadsTb, bytes);
}

template <int R>
static void tb_shape_t(TbShape *s) {
  using C = CfgTb<R>;
  s->region_w = C::W;
  s->region_h = C::H;
  s->core_w = C::CW;
  s->core_h = C::CH;
  s->rim_x = C::RX;
  s->plane_w = C::UPW;
  s->plane_h = C::UPH;
}

cudaError_t launch_stencil3d_tb(int R, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                const Stencil3dTbArgs &a) {
  switch (R) {
    case 1: return launch_tb_t<1>(grid, st, maps, a);
    case 2: return launch_tb_t<2>(grid, st, maps, a);
    case 3: return launch_tb_t<3>(grid, st, maps, a);
    case 4: return launch_tb_t<4>(grid, st, maps, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_stencil3d_tb(int R, int *smem_bytes, int *blocks_per_sm) {
  switch (R) {
    case 1: return prepare_tb_t<1>(smem_bytes, blocks_per_sm);
    case 2: return prepare_tb_t<2>(smem_bytes, blocks_per_sm);
    case 3: return prepare_tb_t<3>(smem_bytes, blocks_per_sm);
    case 4: return prepare_tb_t<4>(smem_bytes, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

bool stencil3d_tb_shape(int R, TbShape *s) {
  switch (R) {
    case 1: tb_shape_t<1>(s); return true;
    case 2: tb_shape_t<2>(s); return true;
    case 3: tb_shape_t<3>(s); return true;
    case 4: tb_shape_t<4>(s); return true;
    default: return false;
  }
}

}  // namespace wp
