// Instantiations and launchers of the 3D stencil kernel for half-orders 5..8
// (space orders 10..16), forward and adjoint+gradient modes.
#include "kernels.cuh"
#include "stencil3d_hi.cuh"

namespace wp {

// equal spacing on every axis: the Laplacian's three coefficient sets coincide
static bool isotropic(const LapCoef &c) {
#ifdef WP_HI_NO_ISO
  (void)c;
  return false;
#endif
  for (int j = 0; j < 9; ++j)
    if (c.cx[j] != c.cy[j] || c.cx[j] != c.cz[j]) return false;
  return true;
}

template <int R, int MODE>
static cudaError_t launch_t(dim3 grid, cudaStream_t st, const CUtensorMap *m, const Stencil3dArgs &a) {
  using C = CfgHi<R, MODE>;
  if (isotropic(a.c))
    return launch_kernel(stencil3d_hi_kernel<R, MODE, true>, grid, dim3(C::THREADS), C::SMEM, st, a.pdl != 0, m[0],
                         m[1], m[2], m[3], m[4], m[5], m[6], a);
  return launch_kernel(stencil3d_hi_kernel<R, MODE, false>, grid, dim3(C::THREADS), C::SMEM, st, a.pdl != 0, m[0],
                       m[1], m[2], m[3], m[4], m[5], m[6], a);
}

template <int R, int MODE, bool ISO>
static cudaError_t prepare_one(int *blocks_per_sm) {
  using C = CfgHi<R, MODE>;
  if constexpr (C::SPLIT_REGS) {
    // the register split must fit the block's launch allocation exactly as
    // planned, else a setmaxnreg.inc would wait for registers that never come:
    // refuse to use the kernel instead
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, stencil3d_hi_kernel<R, MODE, ISO>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != C::LAUNCH_REGS || fa.maxThreadsPerBlock < C::THREADS) return cudaErrorInvalidConfiguration;
  }
  cudaError_t e = cudaFuncSetAttribute(stencil3d_hi_kernel<R, MODE, ISO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stencil3d_hi_kernel<R, MODE, ISO>, C::THREADS,
                                                       C::SMEM);
}

template <int R, int MODE>
static cudaError_t prepare_t(int *smem_bytes, int *blocks_per_sm, int *tile_y) {
  using C = CfgHi<R, MODE>;
  int occ_iso = 0, occ = 0;
  cudaError_t e = prepare_one<R, MODE, true>(&occ_iso);
  if (e != cudaSuccess) return e;
  e = prepare_one<R, MODE, false>(&occ);
  if (e != cudaSuccess) return e;
  *smem_bytes = C::SMEM;
  *tile_y = C::TY;
  *blocks_per_sm = occ < occ_iso ? occ : occ_iso;
  return cudaSuccess;
}

#define WP_HI_DISPATCH(F, ...)                                                          \
  switch (R * 2 + (mode == kModeAdjGrad ? 1 : 0)) {                                     \
    case 10: return F<5, kModeFwd>(__VA_ARGS__);                                        \
    case 11: return F<5, kModeAdjGrad>(__VA_ARGS__);                                    \
    case 12: return F<6, kModeFwd>(__VA_ARGS__);                                        \
    case 13: return F<6, kModeAdjGrad>(__VA_ARGS__);                                    \
    case 14: return F<7, kModeFwd>(__VA_ARGS__);                                        \
    case 15: return F<7, kModeAdjGrad>(__VA_ARGS__);                                    \
    case 16: return F<8, kModeFwd>(__VA_ARGS__);                                        \
    case 17: return F<8, kModeAdjGrad>(__VA_ARGS__);                                    \
    default: return cudaErrorInvalidValue;                                              \
  }

cudaError_t launch_stencil3d_hi(int R, int mode, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                const Stencil3dArgs &a) {
  WP_HI_DISPATCH(launch_t, grid, st, maps, a)
}

cudaError_t prepare_stencil3d_hi(int R, int mode, int *smem_bytes, int *blocks_per_sm, int *tile_y) {
  WP_HI_DISPATCH(prepare_t, smem_bytes, blocks_per_sm, tile_y)
}

int stencil3d_hi_tile_x(int R, int mode) {
  (void)R;
  return mode == kModeAdjGrad ? CfgHi<8, kModeAdjGrad>::TX : CfgHi<8, kModeFwd>::TX;
}

int stencil3d_hi_tile_y(int R, int mode) {
  (void)R;
  return mode == kModeAdjGrad ? CfgHi<8, kModeAdjGrad>::TY : CfgHi<8, kModeFwd>::TY;
}

}  // namespace wp
