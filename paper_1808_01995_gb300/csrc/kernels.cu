// 2D stencil (K1 in 2D), coefficient setup (A1), injection (K2), interpolation
// (K3) and input checks.
#include <limits.h>
#include <math.h>

#include "kernels.cuh"
#include "stencil3d.cuh"

namespace wp {

// ---------------------------------------------------------------------------
// K1, 2D: same update as the 3D kernel (see stencil3d.cuh) on (nz, nx) fields.
// A 32 x 16 output tile per CTA; the halo'd tile of u^n is staged in shared
// memory with zero values outside the grid; each thread computes two points.
// ---------------------------------------------------------------------------
template <int R, int MODE>
__global__ void __launch_bounds__(256) stencil2d_kernel(const Stencil2dArgs a) {
  constexpr int TW = 32, TH = 16, SW = TW + 2 * R, SH = TH + 2 * R;
  __shared__ float tile[SH][SW];
  grid_dependents_launch();
  grid_dependency_wait();
  const int x0 = blockIdx.x * TW, z0 = blockIdx.y * TH;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int nx = a.g.nx, nz = a.g.nz, pitch = a.g.pitch;
  for (int i = tid; i < SH * SW; i += 256) {
    const int lz = i / SW, lx = i % SW;
    const int gz = z0 - R + lz, gx = x0 - R + lx;
    tile[lz][lx] = (gz >= 0 && gz < nz && gx >= 0 && gx < nx)
                       ? __ldg(a.u + static_cast<long long>(gz) * pitch + gx)
                       : 0.f;
  }
  __syncthreads();
  const int lx = threadIdx.x + R;
  const int gx = x0 + threadIdx.x;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int lz = threadIdx.y + 8 * r + R;
    const int gz = z0 + threadIdx.y + 8 * r;
    if (gx >= nx || gz >= nz) continue;
    const float c = tile[lz][lx];
    float lap = a.c.c0 * c;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      lap = fmaf(a.c.cx[j], tile[lz][lx + j] + tile[lz][lx - j], lap);
      lap = fmaf(a.c.cz[j], tile[lz + j][lx] + tile[lz - j][lx], lap);
    }
    const long long gi = static_cast<long long>(gz) * pitch + gx;
    const float um = a.um[gi];
    const float bb = a.b[gi];
    const float sv = a.s[gi];
    const float dd = c - um;
    const float bl = bb * lap;
    a.out[gi] = fmaf(sv, dd, c + dd) + bl;
    if (MODE == kModeAdjGrad) a.grad[gi] = fmaf(a.neg_inv_dt2 * a.uj[gi], fmaf(sv, dd, bl), a.grad[gi]);
  }
}

template <int R, int MODE>
static cudaError_t launch2d_t(cudaStream_t st, const Stencil2dArgs &a) {
  dim3 grid((a.g.nx + 31) / 32, (a.g.nz + 15) / 16);
  return launch_kernel(stencil2d_kernel<R, MODE>, grid, dim3(32, 8), 0, st, a.pdl != 0, a);
}

template <int MODE>
static cudaError_t launch2d_m(int R, cudaStream_t st, const Stencil2dArgs &a) {
  switch (R) {
    case 1: return launch2d_t<1, MODE>(st, a);
    case 2: return launch2d_t<2, MODE>(st, a);
    case 3: return launch2d_t<3, MODE>(st, a);
    case 4: return launch2d_t<4, MODE>(st, a);
    case 5: return launch2d_t<5, MODE>(st, a);
    case 6: return launch2d_t<6, MODE>(st, a);
    case 7: return launch2d_t<7, MODE>(st, a);
    case 8: return launch2d_t<8, MODE>(st, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stencil2d(int R, int mode, cudaStream_t st, const Stencil2dArgs &a) {
  return mode == kModeAdjGrad ? launch2d_m<kModeAdjGrad>(R, st, a) : launch2d_m<kModeFwd>(R, st, a);
}

// ---------------------------------------------------------------------------
// A1: b = dt^2 / (m + eta dt/2) and s = -eta dt / (m + eta dt/2), evaluated in
// double and stored as float in the pitched layout; per-(plane, tile) damping
// flags (bytes, then packed into per-tile z bitmasks by a second kernel);
// max(1/m) for the CFL check; non-finite / sign checks of the inputs.
// ---------------------------------------------------------------------------
// Double-float arithmetic (a value as an unevaluated sum hi + lo of two floats),
// from the error-free transformations of Dekker (product, with an FMA) and Knuth
// (sum): about 44 significant bits in FP32 instructions, where this GPU's FP64
// rate would make a per-point FP64 division the kernel's bottleneck.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_norm(float hi, float lo) {  // |lo| small against hi
  const float s = __fadd_rn(hi, lo);
  return DF{s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
// a (double-float) times a float
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  DF p = df_two_prod(a.hi, b);
  return df_norm(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// n / d rounded once to float: the float quotient q1 plus a correction from the
// exact remainder n - q1 d (Dekker's division step)
__device__ __forceinline__ float df_div_to_float(DF n, DF d) {
  const float q1 = __fdiv_rn(n.hi, d.hi);
  const DF t = df_two_prod(q1, d.hi);
  float r = __fsub_rn(n.hi, t.hi);  // exact: t.hi is within a factor 2 of n.hi
  r = __fsub_rn(r, t.lo);
  r = __fadd_rn(r, n.lo);
  r = __fmaf_rn(-q1, d.lo, r);
  return __fadd_rn(q1, __fdiv_rn(r, d.hi));
}

// A1: b = dt^2 / D, s = -eta dt / D, D = m + eta dt/2 (double-float, rounded once to
// float), damping flags per (plane, flag tile), input checks and max(1/m).  One
// grid row (z, y) per block iteration: no 64-bit index division per point.
__global__ void coef_kernel(const CoefArgs a) {
  const int nx = a.g.nx, ny = a.g.ny;
  const long long nrows = static_cast<long long>(ny) * a.g.nz;
  const DF dt = {a.dt_hi, a.dt_lo};
  const DF dt2 = {a.dt2_hi, a.dt2_lo};
  const DF hdt = {a.hdt_hi, a.hdt_lo};
  float local_max = 0.f;
  int bad = 0;
  for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int y = static_cast<int>(row % ny);
    const long long z = row / ny;
    const long long ci = row * nx;                       // contiguous input row
    const long long gi = z * a.g.plane + static_cast<long long>(y) * a.g.pitch;  // pitched row
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const float mf = a.m[ci + x], ef = a.eta[ci + x];
      if (!isfinite(mf) || !isfinite(ef)) bad |= 1;
      if (!(mf > 0.f) || !(ef >= 0.f)) bad |= 2;
      // D = m + eta (dt/2)
      const DF eh = df_mul_f(hdt, ef);
      const DF s0 = df_two_sum(mf, eh.hi);
      const DF D = df_norm(s0.hi, __fadd_rn(s0.lo, eh.lo));
      a.b[gi + x] = df_div_to_float(dt2, D);
      a.s[gi + x] = ef != 0.f ? -df_div_to_float(df_mul_f(dt, ef), D) : -0.f;
      if (a.tflag && ef != 0.f)
        a.tflag[(z * a.tiles_y + y / a.tile_h) * a.tiles_x + x / a.tile_w] = 1;
      if (mf > 0.f) local_max = fmaxf(local_max, __frcp_rn(mf));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (isfinite(local_max)) atomicMax(a.max_inv_m_bits, __float_as_uint(local_max));
    else atomicOr(a.bad, 1);
    if (bad) atomicOr(a.bad, bad);
  }
}

// Pack the (plane, tile) damping bytes into one z bitmask per tile:
// tbits[(ty * tiles_x + tx) * nzw + w] bit b  <=>  tflag[(32 w + b) * tiles_y * tiles_x + ty * tiles_x + tx].
__global__ void pack_flags_kernel(const CoefArgs a) {
  const long long nword = static_cast<long long>(a.tiles_y) * a.tiles_x * a.nzw;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < nword;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long tile = i / a.nzw;
    const int w = static_cast<int>(i - tile * a.nzw);
    unsigned bits = 0;
    for (int b = 0; b < 32; ++b) {
      const long long z = 32ll * w + b;
      if (z >= a.g.nz) break;
      if (a.tflag[z * a.tiles_y * a.tiles_x + tile]) bits |= 1u << b;
    }
    a.tbits[i] = bits;
  }
}

cudaError_t launch_coef(cudaStream_t st, const CoefArgs &a) {
  const long long nrows = static_cast<long long>(a.g.ny) * a.g.nz;
  long long blocks = nrows;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  coef_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !a.tbits) return e;
  const long long nword = static_cast<long long>(a.tiles_y) * a.tiles_x * a.nzw;
  long long pb = (nword + 255) / 256;
  if (pb > 152 * 8) pb = 152 * 8;
  pack_flags_kernel<<<static_cast<unsigned>(pb), 256, 0, st>>>(a);
  return cudaGetLastError();
}

__global__ void check_finite_kernel(const float *x, long long n, int *bad) {
  int b = 0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    if (!isfinite(x[i])) b = 1;
  if (b) atomicOr(bad, 1);
}

cudaError_t launch_check_finite(cudaStream_t st, const float *x, long long n, int *bad) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  check_finite_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(x, n, bad);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Boundary-wavefield reconstruction helpers: the box where eta vanishes, the
// ring of stored boundary values around it, and the mask of the gradient.
// ---------------------------------------------------------------------------
__global__ void zero_bbox_kernel(const float *eta, FieldGeom g, int *box) {
  const long long n = static_cast<long long>(g.nz) * g.ny * g.nx;
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (eta[i] != 0.f) continue;
    const int x = static_cast<int>(i % g.nx);
    const long long zy = i / g.nx;
    const int y = static_cast<int>(zy % g.ny);
    const int z = static_cast<int>(zy / g.ny);
    const int c[3] = {z, y, x};
    for (int a = 0; a < 3; ++a) {
      lo[a] = min(lo[a], c[a]);
      hi[a] = max(hi[a], c[a]);
    }
  }
  for (int a = 0; a < 3; ++a) {
    const int l = __reduce_min_sync(0xffffffffu, lo[a]);
    const int h = __reduce_max_sync(0xffffffffu, hi[a]);
    if ((threadIdx.x & 31) == 0 && h >= 0) {
      atomicMin(box + 2 * a, l);
      atomicMax(box + 2 * a + 1, h);
    }
  }
}

cudaError_t launch_zero_bbox(cudaStream_t st, const float *eta, FieldGeom g, int *box) {
  const long long n = static_cast<long long>(g.nz) * g.ny * g.nx;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  zero_bbox_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(eta, g, box);
  return cudaGetLastError();
}

__global__ void count_nonzero_kernel(const float *eta, FieldGeom g, Box b, int *count) {
  const int bx = b.x1 - b.x0, by = b.y1 - b.y0;
  const long long n = static_cast<long long>(b.z1 - b.z0) * by * bx;
  unsigned c = 0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = b.x0 + static_cast<int>(i % bx);
    const long long zy = i / bx;
    const int y = b.y0 + static_cast<int>(zy % by);
    const int z = b.z0 + static_cast<int>(zy / by);
    c += eta[(static_cast<long long>(z) * g.ny + y) * g.nx + x] != 0.f;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, static_cast<int>(c));
}

cudaError_t launch_count_nonzero(cudaStream_t st, const float *eta, FieldGeom g, Box b, int *count) {
  const long long n = static_cast<long long>(b.z1 - b.z0) * (b.y1 - b.y0) * (b.x1 - b.x0);
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_nonzero_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(eta, g, b, count);
  return cudaGetLastError();
}

__global__ void ring_copy_kernel(float *field, FieldGeom g, float *buf, RingBoxes rb, int to_buffer) {
  const long long n = rb.start[rb.n];
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    int k = 0;
    while (i >= rb.start[k + 1]) ++k;
    const Box b = rb.b[k];
    const long long l = i - rb.start[k];
    const int bx = b.x1 - b.x0, by = b.y1 - b.y0;
    const int x = b.x0 + static_cast<int>(l % bx);
    const long long zy = l / bx;
    const int y = b.y0 + static_cast<int>(zy % by);
    const int z = b.z0 + static_cast<int>(zy / by);
    const long long f = z * g.plane + static_cast<long long>(y) * g.pitch + x;
    if (to_buffer)
      buf[i] = field[f];
    else
      field[f] = buf[i];
  }
}

cudaError_t launch_ring_copy(cudaStream_t st, float *field, FieldGeom g, float *buf, const RingBoxes &rb,
                             bool to_buffer) {
  const long long n = rb.start[rb.n];
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  ring_copy_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(field, g, buf, rb, to_buffer ? 1 : 0);
  return cudaGetLastError();
}

__global__ void zero_outside_kernel(float *field, FieldGeom g, Box b) {
  const long long n = static_cast<long long>(g.nz) * g.ny * g.nx;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(i % g.nx);
    const long long zy = i / g.nx;
    const int y = static_cast<int>(zy % g.ny);
    const int z = static_cast<int>(zy / g.ny);
    if (z < b.z0 || z >= b.z1 || y < b.y0 || y >= b.y1 || x < b.x0 || x >= b.x1)
      field[z * g.plane + static_cast<long long>(y) * g.pitch + x] = 0.f;
  }
}

cudaError_t launch_zero_outside(cudaStream_t st, float *field, FieldGeom g, Box b) {
  const long long n = static_cast<long long>(g.nz) * g.ny * g.nx;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  zero_outside_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(field, g, b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K2: injection u[t] += b[t] * sum_k w_k q[row][pid_k], one thread per distinct
// target point, entries summed in a fixed order (deterministic, no atomics).
// With grad set, also applies the injected part of the gradient bracket:
// grad[t] -= dt^-2 u^j[t] * b[t] * sum_k w_k q_k.
// ---------------------------------------------------------------------------
__global__ void inject_kernel(const InjectArgs a) {
  grid_dependents_launch();
  grid_dependency_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.ntarget) return;
  const long long row = a.row + (a.row_base ? *a.row_base : 0);
  const float *q = a.data + row * a.npts;
  float acc = 0.f;
  for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) acc = fmaf(a.w[k], q[a.pid[k]], acc);
  const long long t = a.target[i];
  if (!WP_IN_BOUNDS(t >= 0 && t < a.nfield, a.err)) return;
  // explicit roundings (no contraction), so the result does not depend on how the
  // compiler fuses this expression
  const float inc = __fmul_rn(a.b[t], acc);
  a.u[t] = __fadd_rn(a.u[t], inc);
  if (a.grad) a.grad[t] = fmaf(a.neg_inv_dt2 * a.uj[t], inc, a.grad[t]);
}

cudaError_t launch_inject(cudaStream_t st, const InjectArgs &a) {
  if (a.ntarget <= 0) return cudaSuccess;
  return launch_kernel(inject_kernel, dim3((a.ntarget + 127) / 128), dim3(128), 0, st, a.pdl != 0, a);
}

// K3: out[row][i] = sum_c w[i][c] u[idx[i][c]].
__global__ void interp_kernel(const InterpArgs a) {
  grid_dependents_launch();
  grid_dependency_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.npts) return;
  float acc = 0.f;
  for (int c = 0; c < a.ncorner; ++c) {
    const long long k = static_cast<long long>(i) * a.ncorner + c;
    if (!WP_IN_BOUNDS(a.idx[k] >= 0 && a.idx[k] < a.nfield, a.err)) return;
    acc = fmaf(a.w[k], a.u[a.idx[k]], acc);
  }
  const long long row = a.row + (a.row_base ? *a.row_base : 0);
  a.out[row * a.npts + i] = acc;
}

#ifdef WP_DEBUG_BOUNDS
__global__ void check_padding_kernel(const float *f, FieldGeom g, int *err) {
  const int pad = g.pitch - g.nx;
  const long long rows = static_cast<long long>(g.ny) * g.nz;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < rows * pad;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long row = i / pad;
    const int x = g.nx + static_cast<int>(i - row * pad);
    if (f[row * g.pitch + x] != 0.f) {
      atomicCAS(err, 0, static_cast<int>(kErrBounds));
      return;
    }
  }
}
#endif

cudaError_t launch_check_padding(cudaStream_t st, const float *f, FieldGeom g, int *err) {
#ifdef WP_DEBUG_BOUNDS
  if (g.pitch == g.nx) return cudaSuccess;
  check_padding_kernel<<<152 * 4, 256, 0, st>>>(f, g, err);
  return cudaGetLastError();
#else
  (void)st;
  (void)f;
  (void)g;
  (void)err;
  return cudaSuccess;
#endif
}

cudaError_t launch_interp(cudaStream_t st, const InterpArgs &a) {
  if (a.npts <= 0) return cudaSuccess;
  return launch_kernel(interp_kernel, dim3((a.npts + 127) / 128), dim3(128), 0, st, a.pdl != 0, a);
}

// Residual of the misfit J = 1/2 ||d - d_obs||^2 (Eq. AS): r = d - d_obs, and one
// double partial sum of r^2 per block, reduced in a fixed order (deterministic).
__global__ void residual_kernel(const float *d, const float *d_obs, float *r, long long n, double *partial) {
  __shared__ double warp_sum[8];
  double acc = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float v = d[i] - d_obs[i];
    r[i] = v;
    acc += static_cast<double>(v) * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += warp_sum[w];
    partial[blockIdx.x] = t;
  }
}

cudaError_t launch_residual(cudaStream_t st, const float *d, const float *d_obs, float *r, long long n,
                            double *partial, int max_blocks, int *blocks_used) {
  long long blocks = (n + 255) / 256;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  *blocks_used = static_cast<int>(blocks);
  residual_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(d, d_obs, r, n, partial);
  return cudaGetLastError();
}

// Gradient sum over shots (Sec. 3.4): y += alpha x.
__global__ void axpy_kernel(long long n, float alpha, const float *x, float *y) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = fmaf(alpha, x[i], y[i]);
}

cudaError_t launch_axpy(cudaStream_t st, long long n, float alpha, const float *x, float *y) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  axpy_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(n, alpha, x, y);
  return cudaGetLastError();
}

// Fixed-step gradient update with bounds (Sec. 3.4): m = clamp(m - step g, lo, hi).
__global__ void update_model_kernel(long long n, float step, const float *g, float *m, float lo, float hi) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    m[i] = fminf(fmaxf(fmaf(-step, g[i], m[i]), lo), hi);
}

cudaError_t launch_update_model(cudaStream_t st, long long n, float step, const float *g, float *m, float lo,
                                float hi) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  update_model_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(n, step, g, m, lo, hi);
  return cudaGetLastError();
}

__global__ void set_row_kernel(long long *p, long long v) {
  grid_dependents_launch();
  grid_dependency_wait();
  *p = v;
}
__global__ void add_row_kernel(long long *p, long long d) {
  grid_dependents_launch();
  grid_dependency_wait();
  *p += d;
}

cudaError_t launch_set_row(cudaStream_t st, long long *p, long long v, bool pdl) {
  return launch_kernel(set_row_kernel, dim3(1), dim3(1), 0, st, pdl, p, v);
}

cudaError_t launch_add_row(cudaStream_t st, long long *p, long long d, bool pdl) {
  return launch_kernel(add_row_kernel, dim3(1), dim3(1), 0, st, pdl, p, d);
}

}  // namespace wp

namespace wp {

// ---------------------------------------------------------------------------
// CFD examples (Sec. 5), 2D fields (ny, nx), x fastest; the interior points are
// updated, the edge values (Dirichlet data) are copied through.
// ---------------------------------------------------------------------------
__global__ void convection_kernel(const float *__restrict__ u, float *__restrict__ out, int nx, int ny, float sx,
                                  float sy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    const long long k = static_cast<long long>(j) * nx + i;
    const float c = u[k];
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) {
      out[k] = c;
      continue;
    }
    // Eq. convection_fd: backward differences in x and y
    out[k] = c - sx * (c - __ldg(u + k - 1)) - sy * (c - __ldg(u + k - nx));
  }
}

__global__ void burgers_kernel(const float *__restrict__ u, const float *__restrict__ v, float *__restrict__ uo,
                               float *__restrict__ vo, int nx, int ny, float rdx, float rdy, float dt, float nudx2,
                               float nudy2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    const long long k = static_cast<long long>(j) * nx + i;
    const float uc = u[k], vc = v[k];
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) {
      uo[k] = uc;
      vo[k] = vc;
      continue;
    }
    const float uw = __ldg(u + k - 1), ue = __ldg(u + k + 1), us = __ldg(u + k - nx), un = __ldg(u + k + nx);
    const float vw = __ldg(v + k - 1), ve = __ldg(v + k + 1), vs = __ldg(v + k - nx), vn = __ldg(v + k + nx);
    // Eq. Burger: upwind (backward) advection, central diffusion, forward Euler
    const float adv_u = uc * (uc - uw) * rdx + vc * (uc - us) * rdy;
    const float adv_v = uc * (vc - vw) * rdx + vc * (vc - vs) * rdy;
    const float lap_u = (ue - 2.f * uc + uw) * nudx2 + (un - 2.f * uc + us) * nudy2;
    const float lap_v = (ve - 2.f * vc + vw) * nudx2 + (vn - 2.f * vc + vs) * nudy2;
    uo[k] = uc - dt * adv_u + dt * lap_u;
    vo[k] = vc - dt * adv_v + dt * lap_v;
  }
}

__global__ void poisson_kernel(const float *__restrict__ p, const float *__restrict__ b, float *__restrict__ out,
                               int nx, int ny, float dx2, float dy2, float inv_den) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    const long long k = static_cast<long long>(j) * nx + i;
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) {
      out[k] = p[k];
      continue;
    }
    // Eq. Poisson_fd (Jacobi)
    const float sx = __ldg(p + k + 1) + __ldg(p + k - 1), sy = __ldg(p + k + nx) + __ldg(p + k - nx);
    out[k] = (sx * dy2 + sy * dx2 - __ldg(b + k) * dx2 * dy2) * inv_den;
  }
}

static dim3 cfd_grid(int nx, int ny) {
  return dim3(static_cast<unsigned>((nx + 255) / 256), static_cast<unsigned>(ny < 65535 ? ny : 65535));
}

// Streaming forms (nx a multiple of 4): a thread owns four x points (16-byte
// loads and stores) and walks a strip of kStrip rows, keeping the rows above and
// below in registers; x neighbours come from the adjacent lanes (shuffles), the
// warp's outer ones from a scalar load.  Every value is read from DRAM about once.
constexpr int kStrip = 32;

struct Row4 {
  float4 v;
  float w, e;  // x neighbours of the first and last point
};

__device__ __forceinline__ Row4 load_row4(const float *f, long long row, int x4, int nx, bool in) {
  Row4 r;
  r.v = in ? __ldg(reinterpret_cast<const float4 *>(f + row + x4)) : make_float4(0.f, 0.f, 0.f, 0.f);
  const int lane = threadIdx.x & 31;
  float w = __shfl_up_sync(0xffffffffu, r.v.w, 1);
  float e = __shfl_down_sync(0xffffffffu, r.v.x, 1);
  if (lane == 0) w = (in && x4 > 0) ? __ldg(f + row + x4 - 1) : 0.f;
  if (lane == 31) e = (in && x4 + 4 < nx) ? __ldg(f + row + x4 + 4) : 0.f;
  r.w = w;
  r.e = e;
  return r;
}

__device__ __forceinline__ float get4(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ void set4(float4 &v, int k, float a) {
  if (k == 0) v.x = a; else if (k == 1) v.y = a; else if (k == 2) v.z = a; else v.w = a;
}

__global__ void convection4_kernel(const float *__restrict__ u, float *__restrict__ out, int nx, int ny, float sx,
                                   float sy) {
  const int x4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const bool in = x4 < nx;
  const int j0 = blockIdx.y * kStrip, j1 = min(j0 + kStrip, ny);
  float4 up = (in && j0 > 0) ? __ldg(reinterpret_cast<const float4 *>(u + static_cast<long long>(j0 - 1) * nx + x4))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = j0; j < j1; ++j) {
    const long long row = static_cast<long long>(j) * nx;
    const Row4 c = load_row4(u, row, x4, nx, in);
    float4 o = c.v;
    if (j > 0 && j < ny - 1) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x4 + k;
        if (x == 0 || x == nx - 1) continue;
        const float cc = get4(c.v, k), wv = k == 0 ? c.w : get4(c.v, k - 1);
        set4(o, k, cc - sx * (cc - wv) - sy * (cc - get4(up, k)));
      }
    }
    if (in) *reinterpret_cast<float4 *>(out + row + x4) = o;
    up = c.v;
  }
}

__global__ void burgers4_kernel(const float *__restrict__ u, const float *__restrict__ v, float *__restrict__ uo,
                                float *__restrict__ vo, int nx, int ny, float rdx, float rdy, float dt, float nudx2,
                                float nudy2) {
  const int x4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const bool in = x4 < nx;
  const int j0 = blockIdx.y * kStrip, j1 = min(j0 + kStrip, ny);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto ld = [&](const float *f, int j) -> float4 {
    return (in && j >= 0 && j < ny) ? __ldg(reinterpret_cast<const float4 *>(f + static_cast<long long>(j) * nx + x4)) : z4;
  };
  float4 us = ld(u, j0 - 1), vs = ld(v, j0 - 1);
  Row4 uc = load_row4(u, static_cast<long long>(j0) * nx, x4, nx, in && j0 < ny);
  Row4 vc = load_row4(v, static_cast<long long>(j0) * nx, x4, nx, in && j0 < ny);
  for (int j = j0; j < j1; ++j) {
    const long long row = static_cast<long long>(j) * nx;
    const bool has_n = j + 1 < ny;
    const Row4 un = load_row4(u, row + nx, x4, nx, in && has_n), vn = load_row4(v, row + nx, x4, nx, in && has_n);
    float4 ou = uc.v, ov = vc.v;
    if (j > 0 && j < ny - 1) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x4 + k;
        if (x == 0 || x == nx - 1) continue;
        const float ucc = get4(uc.v, k), vcc = get4(vc.v, k);
        const float uw = k == 0 ? uc.w : get4(uc.v, k - 1), ue = k == 3 ? uc.e : get4(uc.v, k + 1);
        const float vw = k == 0 ? vc.w : get4(vc.v, k - 1), ve = k == 3 ? vc.e : get4(vc.v, k + 1);
        const float uss = get4(us, k), unn = get4(un.v, k), vss = get4(vs, k), vnn = get4(vn.v, k);
        const float adv_u = ucc * (ucc - uw) * rdx + vcc * (ucc - uss) * rdy;
        const float adv_v = ucc * (vcc - vw) * rdx + vcc * (vcc - vss) * rdy;
        const float lap_u = (ue - 2.f * ucc + uw) * nudx2 + (unn - 2.f * ucc + uss) * nudy2;
        const float lap_v = (ve - 2.f * vcc + vw) * nudx2 + (vnn - 2.f * vcc + vss) * nudy2;
        set4(ou, k, ucc - dt * adv_u + dt * lap_u);
        set4(ov, k, vcc - dt * adv_v + dt * lap_v);
      }
    }
    if (in) {
      *reinterpret_cast<float4 *>(uo + row + x4) = ou;
      *reinterpret_cast<float4 *>(vo + row + x4) = ov;
    }
    us = uc.v;
    vs = vc.v;
    uc = un;
    vc = vn;
  }
}

__global__ void poisson4_kernel(const float *__restrict__ p, const float *__restrict__ b, float *__restrict__ out,
                                int nx, int ny, float dx2, float dy2, float inv_den) {
  const int x4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const bool in = x4 < nx;
  const int j0 = blockIdx.y * kStrip, j1 = min(j0 + kStrip, ny);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 ps = (in && j0 > 0) ? __ldg(reinterpret_cast<const float4 *>(p + static_cast<long long>(j0 - 1) * nx + x4)) : z4;
  Row4 pc = load_row4(p, static_cast<long long>(j0) * nx, x4, nx, in && j0 < ny);
  const float dxy = dx2 * dy2;
  for (int j = j0; j < j1; ++j) {
    const long long row = static_cast<long long>(j) * nx;
    const Row4 pn = load_row4(p, row + nx, x4, nx, in && j + 1 < ny);
    float4 o = pc.v;
    if (j > 0 && j < ny - 1) {
      const float4 bb = in ? __ldg(reinterpret_cast<const float4 *>(b + row + x4)) : z4;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x4 + k;
        if (x == 0 || x == nx - 1) continue;
        const float pw = k == 0 ? pc.w : get4(pc.v, k - 1), pe = k == 3 ? pc.e : get4(pc.v, k + 1);
        const float sxx = pe + pw, syy = get4(pn.v, k) + get4(ps, k);
        set4(o, k, (sxx * dy2 + syy * dx2 - get4(bb, k) * dxy) * inv_den);
      }
    }
    if (in) *reinterpret_cast<float4 *>(out + row + x4) = o;
    ps = pc.v;
    pc = pn;
  }
}

static dim3 cfd_grid4(int nx, int ny) {
  return dim3(static_cast<unsigned>((nx / 4 + 127) / 128), static_cast<unsigned>((ny + kStrip - 1) / kStrip));
}

cudaError_t launch_convection(cudaStream_t st, const float *u, float *out, int nx, int ny, float sx, float sy) {
  if (nx % 4 == 0 && (ny + kStrip - 1) / kStrip <= 65535)
    convection4_kernel<<<cfd_grid4(nx, ny), 128, 0, st>>>(u, out, nx, ny, sx, sy);
  else
    convection_kernel<<<cfd_grid(nx, ny), 256, 0, st>>>(u, out, nx, ny, sx, sy);
  return cudaGetLastError();
}

cudaError_t launch_burgers(cudaStream_t st, const float *u, const float *v, float *uo, float *vo, int nx, int ny,
                           float rdx, float rdy, float dt, float nudx2, float nudy2) {
  if (nx % 4 == 0 && (ny + kStrip - 1) / kStrip <= 65535)
    burgers4_kernel<<<cfd_grid4(nx, ny), 128, 0, st>>>(u, v, uo, vo, nx, ny, rdx, rdy, dt, nudx2, nudy2);
  else
    burgers_kernel<<<cfd_grid(nx, ny), 256, 0, st>>>(u, v, uo, vo, nx, ny, rdx, rdy, dt, nudx2, nudy2);
  return cudaGetLastError();
}

cudaError_t launch_poisson(cudaStream_t st, const float *p, const float *b, float *out, int nx, int ny, float dx2,
                           float dy2, float inv_den) {
  if (nx % 4 == 0 && (ny + kStrip - 1) / kStrip <= 65535)
    poisson4_kernel<<<cfd_grid4(nx, ny), 128, 0, st>>>(p, b, out, nx, ny, dx2, dy2, inv_den);
  else
    poisson_kernel<<<cfd_grid(nx, ny), 256, 0, st>>>(p, b, out, nx, ny, dx2, dy2, inv_den);
  return cudaGetLastError();
}

}  // namespace wp
