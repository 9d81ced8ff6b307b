// K1 (3D): one leapfrog step of the damped acoustic equation on a pitched grid,
//
//   u^{n+1} = u^n + (1 + s) (u^n - u^{n-1}) + b Lap u^n,
//   b = dt^2 / (m + eta dt/2),  s = -eta dt / (m + eta dt/2),
//
// which is the solved form of Eq. fdWE-abc with the order-k central Laplacian of
// Eq. fdSpace (centre once), Eq. fdTime in time and a central damping
// difference.  In adjoint+gradient mode the same update produces w^j from
// (w^{j+1}, w^{j+2}) and, fused, accumulates the adjoint-state gradient of
// Eq. Grad:  g -= dt^-2 u^j [s (w^{j+1} - w^{j+2}) + b Lap w^{j+1}]  (the
// injected part is added by the injection kernel).
//
// Design (GB300): each CTA owns a 32 x 16 (x, y) tile and a chunk of z-planes and
// streams up z.  One thread issues TMA (cp.async.bulk.tensor) loads of
//   - the halo'd u^n plane (32 + 2RX) x (16 + 2R) into an (R + 1 + P)-deep ring,
//   - the u^{n-1}, b, s (and u^j, g) tiles into a (P + 1)-deep ring,
// P planes ahead of the compute, completing on mbarriers.  TMA's zero fill
// outside the tensor supplies the Dirichlet ghosts.  x/y neighbours are read from
// the shared plane, z neighbours from a per-thread register queue of 2R + 1
// values.  s is loaded only for (tile, plane) pairs flagged as damped.
#pragma once

#include "wp_device.cuh"

namespace wp {

constexpr int kTX = 32;                 // tile width (x)
constexpr int kTY = 16;                 // tile height (y)
constexpr int kWarps = 8;               // warps per CTA
constexpr int kRows = kTY / kWarps;     // tile rows per thread
constexpr int kThreads3d = kWarps * 32;

enum StencilMode : int { kModeFwd = 0, kModeAdjGrad = 1 };

template <int R>
struct Cfg3d {
  static constexpr int RX = (R + 3) / 4 * 4;          // x halo rounded to 16 bytes
  static constexpr int PW = kTX + 2 * RX;             // halo'd plane width
  static constexpr int PH = kTY + 2 * R;              // halo'd plane height
  static constexpr int P = 2;                         // planes in flight ahead
  static constexpr int NSU = R + 1 + P;               // u ring depth
  static constexpr int NS2 = P + 1;                   // pointwise-stream ring depth
  static constexpr int USLOT = ((PW * PH * 4 + 127) / 128) * 128;  // bytes per u slot
  static constexpr int TSLOT = kTX * kTY * 4;         // bytes per tile slot
};

template <int R, int MODE>
struct Smem3d {
  using C = Cfg3d<R>;
  static constexpr int NSTREAM = MODE == kModeAdjGrad ? 5 : 3;  // um, b, s [, uj, g]
  static constexpr int OFF_T = C::NSU * C::USLOT;
  static constexpr int OFF_BAR = OFF_T + NSTREAM * C::NS2 * C::TSLOT;
  static constexpr int BYTES = OFF_BAR + (C::NSU + C::NS2) * 8 + 16;
};

struct Stencil3dArgs {
  FieldGeom g;
  LapCoef c;
  const float *u;               // u^n (plain loads of the z-halo below a chunk)
  float *out;                   // u^{n+1} (may alias u^{n-1})
  float *grad;                  // gradient (adjoint+gradient mode)
  float neg_inv_dt2;            // -1 / dt^2
  const unsigned char *tflag;   // [nz][tiles_y][tiles_x], 1 where the tile has eta != 0
  int tiles_x, tiles_y;
  int zchunk;                   // planes per CTA
  int *err;                     // device error word
};

template <int R, int MODE>
__global__ void __launch_bounds__(kThreads3d)
    stencil3d_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_um,
                     const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_s,
                     const __grid_constant__ CUtensorMap tm_uj, const __grid_constant__ CUtensorMap tm_g,
                     const Stencil3dArgs a) {
  using C = Cfg3d<R>;
  using S = Smem3d<R, MODE>;
  constexpr int TT = kTX * kTY;
  extern __shared__ __align__(128) unsigned char smem[];
  float *uring = reinterpret_cast<float *>(smem);
  float *t_um = reinterpret_cast<float *>(smem + S::OFF_T);
  float *t_b = t_um + C::NS2 * TT;
  float *t_s = t_b + C::NS2 * TT;
  float *t_uj = t_s + C::NS2 * TT;  // adjoint+gradient only
  float *t_g = t_uj + C::NS2 * TT;  // adjoint+gradient only
  uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + S::OFF_BAR);
  uint64_t *full_t = full_u + C::NSU;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(full_t + C::NS2);

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int tile_x = blockIdx.x, tile_y = blockIdx.y;
  const int x0 = tile_x * kTX, y0 = tile_y * kTY;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.g.nz);
  if (z0 >= z1) return;  // uniform over the CTA
  const int last_u = z1 + R;  // u planes z0 .. z1+R-1 are streamed

  if (tid == 0) {
    for (int i = 0; i < C::NSU; ++i) mbar_init(&full_u[i], 1);
    for (int i = 0; i < C::NS2; ++i) mbar_init(&full_t[i], 1);
    *abort_flag = 0;
    mbar_init_fence();
    prefetch_tensormap(&tm_u);
    prefetch_tensormap(&tm_um);
    prefetch_tensormap(&tm_b);
    prefetch_tensormap(&tm_s);
    if (MODE == kModeAdjGrad) {
      prefetch_tensormap(&tm_uj);
      prefetch_tensormap(&tm_g);
    }
  }
  __syncthreads();

  auto damped = [&](int z) -> bool {
    return a.tflag[(static_cast<long long>(z) * a.tiles_y + tile_y) * a.tiles_x + tile_x] != 0;
  };
  // Producer side (thread 0 only).
  auto issue_u = [&](int p) {
    const int slot = (p - z0) % C::NSU;
    mbar_arrive_expect_tx(&full_u[slot], C::PW * C::PH * 4);
    tma_load_3d(uring + slot * (C::USLOT / 4), &tm_u, x0 - C::RX, y0 - R, p, &full_u[slot]);
  };
  auto issue_t = [&](int z) {
    const int slot = (z - z0) % C::NS2;
    const bool d = damped(z);
    const int n = (MODE == kModeAdjGrad ? 4 : 2) + (d ? 1 : 0);
    mbar_arrive_expect_tx(&full_t[slot], n * C::TSLOT);
    tma_load_3d(t_um + slot * TT, &tm_um, x0, y0, z, &full_t[slot]);
    tma_load_3d(t_b + slot * TT, &tm_b, x0, y0, z, &full_t[slot]);
    if (d) tma_load_3d(t_s + slot * TT, &tm_s, x0, y0, z, &full_t[slot]);
    if (MODE == kModeAdjGrad) {
      tma_load_3d(t_uj + slot * TT, &tm_uj, x0, y0, z, &full_t[slot]);
      tma_load_3d(t_g + slot * TT, &tm_g, x0, y0, z, &full_t[slot]);
    }
  };
  int issued_u = z0, issued_t = z0;  // next plane to issue (thread 0)
  if (tid == 0) {
    for (; issued_u < min(z0 + R + C::P, last_u); ++issued_u) issue_u(issued_u);
    for (; issued_t < min(z0 + C::P, z1); ++issued_t) issue_t(issued_t);
  }

  // Register queues: q[r][j] = u^n at plane z - R + j of this thread's point r.
  float q[kRows][2 * R + 1];
  int ty[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) ty[r] = warp + r * kWarps;
  const int gx = x0 + lane;
  // z-halo below the chunk: plain loads (zero outside the grid)
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int p = z0 - R + j;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int gy = y0 + ty[r];
      q[r][j] = (p >= 0 && gx < a.g.nx && gy < a.g.ny)
                    ? __ldg(a.u + p * a.g.plane + static_cast<long long>(gy) * a.g.pitch + gx)
                    : 0.f;
    }
  }
  // planes z0 .. z0+R-1 from the ring
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int p = z0 + j;
    const int slot = (p - z0) % C::NSU;
    const float *P = uring + slot * (C::USLOT / 4);
    if (p < last_u) mbar_wait_bounded(&full_u[slot], ((p - z0) / C::NSU) & 1, abort_flag);
#pragma unroll
    for (int r = 0; r < kRows; ++r) q[r][R + j] = P[(ty[r] + R) * C::PW + lane + C::RX];
  }

  for (int z = z0; z < z1; ++z) {
    if (tid == 0 && !*abort_flag) {
      // slots of plane z-1 were released by the barrier ending the last iteration
      if (issued_u < last_u) issue_u(issued_u++);
      if (issued_t < z1) issue_t(issued_t++);
    }
    // centre of plane z+R into the queue
    {
      const int p = z + R;
      const int slot = (p - z0) % C::NSU;
      mbar_wait_bounded(&full_u[slot], ((p - z0) / C::NSU) & 1, abort_flag);
      const float *P = uring + slot * (C::USLOT / 4);
#pragma unroll
      for (int r = 0; r < kRows; ++r) q[r][2 * R] = P[(ty[r] + R) * C::PW + lane + C::RX];
    }
    const int tslot = (z - z0) % C::NS2;
    mbar_wait_bounded(&full_t[tslot], ((z - z0) / C::NS2) & 1, abort_flag);
    const bool d = damped(z);
    const float *P = uring + ((z - z0) % C::NSU) * (C::USLOT / 4);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const float *pc = P + (ty[r] + R) * C::PW + lane + C::RX;
      const float c = q[r][R];
      float lap = a.c.c0 * c;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        lap = fmaf(a.c.cx[j], pc[j] + pc[-j], lap);
        lap = fmaf(a.c.cy[j], pc[j * C::PW] + pc[-j * C::PW], lap);
        lap = fmaf(a.c.cz[j], q[r][R + j] + q[r][R - j], lap);
      }
      const int ti = tslot * TT + ty[r] * kTX + lane;
      const float um = t_um[ti];
      const float bb = t_b[ti];
      const float sv = d ? t_s[ti] : 0.f;
      const float dd = c - um;
      const float bl = bb * lap;
      const float un = fmaf(sv, dd, c + dd) + bl;
      const int gy = y0 + ty[r];
      if (gx < a.g.nx && gy < a.g.ny && !*abort_flag) {
        const long long gi = z * a.g.plane + static_cast<long long>(gy) * a.g.pitch + gx;
        a.out[gi] = un;
        if (MODE == kModeAdjGrad) {
          const float br = fmaf(sv, dd, bl);
          a.grad[gi] = fmaf(a.neg_inv_dt2 * t_uj[ti], br, t_g[ti]);
        }
      }
    }
    __syncthreads();  // every thread is done with plane z's u slot and tile slot
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
      for (int j = 0; j < 2 * R; ++j) q[r][j] = q[r][j + 1];
  }

  if (*abort_flag) {
    // Let the copies this CTA issued land (bounded) before shared memory goes away.
    if (tid == 0) {
      const uint64_t t0 = global_timer_ns();
      for (int p = max(z0, issued_u - C::NSU); p < issued_u; ++p) {
        const int slot = (p - z0) % C::NSU;
        while (!mbar_try_wait(&full_u[slot], ((p - z0) / C::NSU) & 1) &&
               global_timer_ns() - t0 < kWaitLimitNs) {
        }
      }
      for (int p = max(z0, issued_t - C::NS2); p < issued_t; ++p) {
        const int slot = (p - z0) % C::NS2;
        while (!mbar_try_wait(&full_t[slot], ((p - z0) / C::NS2) & 1) &&
               global_timer_ns() - t0 < kWaitLimitNs) {
        }
      }
      atomicCAS(a.err, 0, static_cast<int>(kErrWaitFull));
    }
  }
}

}  // namespace wp
