// Declarations of the kernel launchers (one translation unit per kernel family).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "wp_device.cuh"

namespace wp {

struct Stencil3dArgs;

// Launch k<<<grid, block, smem, st>>>(args...), with programmatic stream
// serialization when pdl is set (the kernel must call grid_dependency_wait()
// before touching memory the previous kernel on the stream reads or writes).
template <class... KArgs, class... Args>
inline cudaError_t launch_kernel(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                                 Args &&...args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args &&>(args)...);
}

// ---- K1, 3D (stencil3d_fwd.cu / stencil3d_adj.cu; half-orders above 4: stencil3d_hi.cu) ----
// maps: u^n (halo'd plane box of the mode), u^{n-1}, b, s, u^j, g, u^n (tile boxes of the mode)
cudaError_t launch_stencil3d_fwd(int R, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                 const Stencil3dArgs &a);
cudaError_t launch_stencil3d_adj(int R, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                 const Stencil3dArgs &a);
// sets the dynamic shared-memory limit; reports the CTA footprint, occupancy and tile height
cudaError_t prepare_stencil3d_fwd(int R, int *smem_bytes, int *blocks_per_sm, int *tile_y);
cudaError_t prepare_stencil3d_adj(int R, int *smem_bytes, int *blocks_per_sm, int *tile_y);
// tile width (x) and height (y) of the work tiles of each mode
int stencil3d_tile_x_fwd(int R);
int stencil3d_tile_x_adj(int R);
int stencil3d_tile_y_fwd(int R);
int stencil3d_tile_y_adj(int R);
inline int stencil3d_tile_x(int R, int mode) {
  return mode == 1 ? stencil3d_tile_x_adj(R) : stencil3d_tile_x_fwd(R);
}
inline int stencil3d_tile_y(int R, int mode) {
  return mode == 1 ? stencil3d_tile_y_adj(R) : stencil3d_tile_y_fwd(R);
}
// the kernel of half-orders 5..8 (mode 0 forward, 1 adjoint+gradient)
cudaError_t launch_stencil3d_hi(int R, int mode, dim3 grid, cudaStream_t st, const CUtensorMap *maps,
                                const Stencil3dArgs &a);
cudaError_t prepare_stencil3d_hi(int R, int mode, int *smem_bytes, int *blocks_per_sm, int *tile_y);
int stencil3d_hi_tile_x(int R, int mode);
int stencil3d_hi_tile_y(int R, int mode);

// ---- K1, 2D (kernels.cu) ----
struct Stencil2dArgs {
  FieldGeom g;        // 2D fields use nz rows of `pitch` elements (ny = 1)
  LapCoef c;
  const float *u;     // u^n
  const float *um;    // u^{n-1}
  const float *b;
  const float *s;
  float *out;         // u^{n+1} (may alias um)
  float *grad;        // adjoint+gradient mode
  const float *uj;    // adjoint+gradient mode: forward field u^j
  float neg_inv_dt2;
  int pdl;            // launch with programmatic stream serialization
};
cudaError_t launch_stencil2d(int R, int mode, cudaStream_t st, const Stencil2dArgs &a);

// ---- A1: coefficients b, s, damping flags, input checks (kernels.cu) ----
struct CoefArgs {
  const float *m;          // contiguous (nz, ny, nx) / (nz, nx)
  const float *eta;
  FieldGeom g;
  double dt;
  float dt_hi, dt_lo, dt2_hi, dt2_lo, hdt_hi, hdt_lo;  // dt, dt^2, dt/2 as float pairs (hi + lo)
  float *b;                // pitched
  float *s;                // pitched
  unsigned char *tflag;    // 3D only: [nz][tiles_y][tiles_x] bytes, 1 where eta != 0, pre-zeroed
  unsigned *tbits;         // 3D only: [tiles_y][tiles_x][nzw] z bitmasks packed from tflag
  int nzw;
  int tiles_x, tiles_y, tile_w, tile_h;
  unsigned int *max_inv_m_bits;  // float bits of max(1/m), pre-zeroed
  int *bad;                // bit 0: non-finite input, bit 1: m <= 0 or eta < 0
};
cudaError_t launch_coef(cudaStream_t st, const CoefArgs &a);

// ---- K2: injection, deterministic CSR gather (kernels.cu) ----
struct InjectArgs {
  int ntarget;
  const long long *target;   // pitched flat index of each distinct target point
  const int *rowptr;         // [ntarget + 1]
  const int *pid;            // point id of each entry
  const float *w;            // weight of each entry
  const float *data;         // [nt][npts]
  int npts;
  const long long *row_base; // optional device row base (graph replays); row is added to it
  long long row;             // time row of `data` (offset from *row_base if set)
  float *u;                  // field receiving dt^2/(m + eta dt/2) * sum w q
  const float *b;
  float *grad;               // optional: gradient correction at the targets
  const float *uj;
  float neg_inv_dt2;
  long long nfield;          // elements of a pitched field (debug bounds checks)
  int *err;                  // error word (debug bounds checks)
  int pdl;                   // launch with programmatic stream serialization
};
cudaError_t launch_inject(cudaStream_t st, const InjectArgs &a);

// ---- K3: interpolation, gather (kernels.cu) ----
struct InterpArgs {
  int npts;
  int ncorner;               // 4 (2D) or 8 (3D)
  const long long *idx;      // [npts][ncorner] pitched flat indices
  const float *w;            // [npts][ncorner]
  const float *u;
  float *out;                // [nt][npts]
  const long long *row_base; // optional device row base (graph replays); row is added to it
  long long row;
  long long nfield;          // elements of a pitched field (debug bounds checks)
  int *err;                  // error word (debug bounds checks)
  int pdl;                   // launch with programmatic stream serialization
};
cudaError_t launch_interp(cudaStream_t st, const InterpArgs &a);

// Debug builds: record kErrBounds if any pitch padding element (x in [nx, pitch))
// of a pitched field is nonzero (nothing may write there).  Release builds: no-op.
cudaError_t launch_check_padding(cudaStream_t st, const float *f, FieldGeom g, int *err);

// *p = v / *p += d (row bases of graph replays), one thread
cudaError_t launch_set_row(cudaStream_t st, long long *p, long long v, bool pdl);
cudaError_t launch_add_row(cudaStream_t st, long long *p, long long d, bool pdl);

// ---- misc ----
// r = d - d_obs over n samples; partial[b] = sum over block b's samples of r^2
// (double), blocks of 256 threads; returns the number of blocks used (<= max_blocks)
cudaError_t launch_residual(cudaStream_t st, const float *d, const float *d_obs, float *r, long long n,
                            double *partial, int max_blocks, int *blocks_used);

// y[i] += alpha x[i], i < n
cudaError_t launch_axpy(cudaStream_t st, long long n, float alpha, const float *x, float *y);
// m[i] = min(max(m[i] - step g[i], lo), hi), i < n
cudaError_t launch_update_model(cudaStream_t st, long long n, float step, const float *g, float *m, float lo,
                                float hi);

// ---- boundary-wavefield reconstruction (kernels.cu) ----
// An axis-aligned box of grid points, [z0, z1) x [y0, y1) x [x0, x1).
struct Box {
  int z0, z1, y0, y1, x0, x1;
};
// box[0..5] = (min z, max z, min y, max y, min x, max x) over the points of the
// contiguous field eta (nz, ny, nx) where eta == 0; box must hold
// (INT_MAX, -1, INT_MAX, -1, INT_MAX, -1) on entry.
cudaError_t launch_zero_bbox(cudaStream_t st, const float *eta, FieldGeom g, int *box);
// *count += number of points inside `b` where eta != 0
cudaError_t launch_count_nonzero(cudaStream_t st, const float *eta, FieldGeom g, Box b, int *count);
// Up to six boxes of a pitched field, concatenated in order (each in z, y, x order)
// in a contiguous buffer: gather (to_buffer) or scatter back.
struct RingBoxes {
  int n;
  Box b[6];
  long long start[7];  // prefix sums of the box sizes
};
cudaError_t launch_ring_copy(cudaStream_t st, float *field, FieldGeom g, float *buf, const RingBoxes &rb,
                             bool to_buffer);
// field = 0 at every point outside `b` (pitched field)
cudaError_t launch_zero_outside(cudaStream_t st, float *field, FieldGeom g, Box b);

// ---- CFD examples of Sec. 5 (kernels.cu): one step / iteration on (ny, nx) fields,
// interior updated, edges copied (Dirichlet data) ----
// convection (Eq. convection_fd), sx = c dt/dx, sy = c dt/dy
cudaError_t launch_convection(cudaStream_t st, const float *u, float *out, int nx, int ny, float sx, float sy);
// Burgers' equation (Eq. Burger): rdx = 1/dx, rdy = 1/dy, nudx2 = nu/dx^2, nudy2 = nu/dy^2
cudaError_t launch_burgers(cudaStream_t st, const float *u, const float *v, float *uo, float *vo, int nx, int ny,
                           float rdx, float rdy, float dt, float nudx2, float nudy2);
// Poisson (Eq. Poisson_fd), one Jacobi iteration; inv_den = 1 / (2 (dx^2 + dy^2))
cudaError_t launch_poisson(cudaStream_t st, const float *p, const float *b, float *out, int nx, int ny, float dx2,
                           float dy2, float inv_den);

// bit 0 of *bad set if any of x[0..n) is NaN or Inf
cudaError_t launch_check_finite(cudaStream_t st, const float *x, long long n, int *bad);

}  // namespace wp
