// Instantiations and launcher of the 3D stencil, mode: pair (two steps by two CTA
// roles in one cooperative launch).
#include "kernels.cuh"
#include "stencil3d.cuh"

namespace wp {

template <int R>
static cudaError_t launch_pair_t(dim3 grid, cudaStream_t st, const CUtensorMap *m, const Stencil3dArgs &a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads3d);
  cfg.dynamicSmemBytes = Cfg3d<R, kModePair>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: role 1 waits on role 0
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, stencil3d_kernel<R, kModePair>, m[0], m[1], m[2], m[3], m[4], m[5], a);
}

template <int R>
static cudaError_t prepare_pair_t(int *smem_bytes, int *blocks_per_sm) {
  constexpr int bytes = Cfg3d<R, kModePair>::SMEM;
  cudaError_t e =
      cudaFuncSetAttribute(stencil3d_kernel<R, kModePair>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  *smem_bytes = bytes;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stencil3d_kernel<R, kModePair>, kThreads3d,
                                                       bytes);
}

cudaError_t launch_stencil3d_pair(int R, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                  const Stencil3dArgs &a) {
  switch (R) {
    case 1: return launch_pair_t<1>(grid, st, maps, a);
    case 2: return launch_pair_t<2>(grid, st, maps, a);
    case 3: return launch_pair_t<3>(grid, st, maps, a);
    case 4: return launch_pair_t<4>(grid, st, maps, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_stencil3d_pair(int R, int *smem_bytes, int *blocks_per_sm) {
  switch (R) {
    case 1: return prepare_pair_t<1>(smem_bytes, blocks_per_sm);
    case 2: return prepare_pair_t<2>(smem_bytes, blocks_per_sm);
    case 3: return prepare_pair_t<3>(smem_bytes, blocks_per_sm);
    case 4: return prepare_pair_t<4>(smem_bytes, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wp
