// K1 (3D): one leapfrog step of the damped acoustic equation on a pitched grid,
//
//   u^{n+1} = u^n + (1 + s) (u^n - u^{n-1}) + b Lap u^n,
//   b = dt^2 / (m + eta dt/2),  s = -eta dt / (m + eta dt/2),
//
// the solved form of Eq. fdWE-abc with the order-k central Laplacian of
// Eq. fdSpace (centre once), Eq. fdTime in time and a central damping
// difference.  In adjoint+gradient mode the same update produces w^j from
// (w^{j+1}, w^{j+2}) and, fused, accumulates the adjoint-state gradient of
// Eq. Grad:  g -= dt^-2 u^j [s (w^{j+1} - w^{j+2}) + b Lap w^{j+1}]  (the
// injected part is added by the injection kernel).
//
// GB300 design.  Persistent CTAs walk (32 x TY tile, z-chunk) work items in a
// static round-robin order and stream each chunk up z.  A producer warp issues
// TMA (cp.async.bulk.tensor) loads, P planes ahead of the compute, into two
// shared rings guarded by full/empty mbarriers:
//   - the halo'd u^n plane, (32 + 2 RX) x (TY + 2R), ring depth R + 1 + P (TMA's
//     zero fill outside the tensor supplies the Dirichlet ghosts);
//   - the pointwise tiles u^{n-1}, b, s (and u^j, g), ring depth P + 1; s only for
//     planes whose tile holds damping (per-tile z bitmask, one word per 32 planes).
// 8 consumer warps compute; each thread owns NY consecutive rows of one column:
// it loads that column of the plane once for all y neighbours, reads x
// neighbours from the plane and keeps z neighbours in a register queue, so the
// shared-memory traffic per point stays well under the SM's bandwidth.
// Every wait is bounded (%globaltimer); a timeout sets an abort flag, the
// producer lets its copies land, and the error word reports it.
#pragma once

#include "wp_device.cuh"

namespace wp {

constexpr int kTX = 32;                     // tile width (x), one warp
constexpr int kConsumerWarps = 8;
constexpr int kThreads3d = (kConsumerWarps + 1) * 32;
constexpr int kTileFlagTY = 16;             // y extent of a damping-flag tile

enum StencilMode : int { kModeFwd = 0, kModeAdjGrad = 1 };

// Tile parameters of the high orders (R > 4), chosen by measurement; the -D
// overrides exist for tuning sweeps.
#ifndef WP_NY_HI
#define WP_NY_HI 2
#endif
#ifndef WP_P_HI
#define WP_P_HI 2
#endif
#ifndef WP_MINB_HI
#define WP_MINB_HI 2
#endif

template <int R, int MODE>
struct Cfg3d {
  static constexpr int NY = MODE == kModeFwd ? (R <= 4 ? 4 : WP_NY_HI) : 2;  // rows per consumer thread
  static constexpr int TY = kConsumerWarps * NY;                               // tile height
  static constexpr int RX = (R + 3) / 4 * 4;                                   // x halo rounded to 16 bytes
  static constexpr int PW = kTX + 2 * RX;
  static constexpr int PH = TY + 2 * R;
  static constexpr int P = R <= 4 ? 3 : WP_P_HI;                               // planes in flight ahead
  static constexpr int MINB = (R <= 4 || MODE != kModeFwd) ? 2 : WP_MINB_HI;   // CTAs per SM to fit
  static constexpr int NSU = R + 1 + P;                              // u ring depth
  static constexpr int NST = P + 1;                                  // tile ring depth
  static constexpr int NSTREAM = MODE == kModeAdjGrad ? 5 : 3;       // um, b, s [, uj, g]
  static constexpr int USLOT = ((PW * PH * 4 + 127) / 128) * 128;    // bytes per u slot
  static constexpr int TSLOT = kTX * TY * 4;                         // bytes per tile
  static constexpr int T_OFF = NSU * USLOT;
  static constexpr int BAR_OFF = T_OFF + NST * NSTREAM * TSLOT;
  static constexpr int SMEM = BAR_OFF + 2 * (NSU + NST) * 8 + NST * 4 + 16;
};

struct Stencil3dArgs {
  FieldGeom g;
  LapCoef c;
  const float *u;               // u^n (plain loads of the z-halo below a chunk)
  float *out;                   // u^{n+1} (may alias u^{n-1})
  float *grad;                  // adjoint+gradient: gradient (read-modify-write)
  float neg_inv_dt2;            // -1 / dt^2
  const unsigned *tbits;        // [flag_tiles_y][tiles_x][nzw]: bit z set where the tile row has eta != 0
  int nzw;                      // 32-bit words per tile (ceil(nz / 32))
  int tiles_x, tiles_y;         // work tiles (32 x TY)
  int flag_tiles_y;
  int zchunk, nzc;              // planes per item, chunks per column
  int nitems;                   // tiles_x * tiles_y * nzc
  int *err;
};

// tm: [0] u^n (halo'd plane box), [1] u^{n-1}, [2] b, [3] s, [4] u^j, [5] g (tile boxes)
template <int R, int MODE>
__global__ void __launch_bounds__(kThreads3d, Cfg3d<R, MODE>::MINB)
    stencil3d_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_um,
                     const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_s,
                     const __grid_constant__ CUtensorMap tm_uj, const __grid_constant__ CUtensorMap tm_g,
                     const Stencil3dArgs a) {
  using C = Cfg3d<R, MODE>;
  constexpr int NY = C::NY, TY = C::TY, TT = kTX * TY;
  extern __shared__ __align__(128) unsigned char smem[];
  float *uring = reinterpret_cast<float *>(smem);
  float *tring = reinterpret_cast<float *>(smem + C::T_OFF);  // [NST][NSTREAM][TT]
  uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + C::BAR_OFF);
  uint64_t *empty_u = full_u + C::NSU;
  uint64_t *full_t = empty_u + C::NSU;
  uint64_t *empty_t = full_t + C::NST;
  volatile int *sflag = reinterpret_cast<volatile int *>(empty_t + C::NST);  // [NST]: s loaded
  volatile int *abort_flag = sflag + C::NST;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < C::NSU; ++i) {
      mbar_init(&full_u[i], 1);
      mbar_init(&empty_u[i], kConsumerWarps);
    }
    for (int i = 0; i < C::NST; ++i) {
      mbar_init(&full_t[i], 1);
      mbar_init(&empty_t[i], kConsumerWarps);
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();

  auto item_geom = [&](int item, int &tx, int &ty, int &z0, int &z1) {
    const int tile = item / a.nzc, zc = item - tile * a.nzc;
    tx = tile % a.tiles_x;
    ty = tile / a.tiles_x;
    z0 = zc * a.zchunk;
    z1 = min(z0 + a.zchunk, a.g.nz);
  };

  if (warp == kConsumerWarps) {
    // ---------------- producer (one lane) ----------------
    if (lane == 0) {
      prefetch_tensormap(&tm_u);
      prefetch_tensormap(&tm_um);
      prefetch_tensormap(&tm_b);
      prefetch_tensormap(&tm_s);
      if (MODE == kModeAdjGrad) {
        prefetch_tensormap(&tm_uj);
        prefetch_tensormap(&tm_g);
      }
      uint32_t iu = 0, itt = 0;  // planes issued into each ring
      bool ok = true;
      // A TMA copy needs a 128-byte aligned shared destination and an x start whose
      // byte offset is a multiple of 16; refuse (and report) anything else.
      auto aligned = [&](const float *dst, int x) -> bool {
        if ((smem_u32(dst) & 127u) == 0 && (x & 3) == 0) return true;
        atomicCAS(a.err, 0, static_cast<int>(kErrLaunch));
        *abort_flag = 1;
        ok = false;
        return false;
      };
      auto issue_u = [&](int x0, int y0, int p) {
        const uint32_t slot = iu % C::NSU;
        if (iu >= C::NSU && !mbar_wait_bounded(&empty_u[slot], ((iu / C::NSU) - 1) & 1, abort_flag)) {
          ok = false;
          return;
        }
        float *dst = uring + slot * (C::USLOT / 4);
        if (!aligned(dst, x0 - C::RX)) return;
        mbar_arrive_expect_tx(&full_u[slot], C::PW * C::PH * 4);
        tma_load_3d(dst, &tm_u, x0 - C::RX, y0 - R, p, &full_u[slot]);
        ++iu;
      };
      auto issue_t = [&](int x0, int y0, int z, bool d) {
        const uint32_t slot = itt % C::NST;
        if (itt >= C::NST && !mbar_wait_bounded(&empty_t[slot], ((itt / C::NST) - 1) & 1, abort_flag)) {
          ok = false;
          return;
        }
        float *t = tring + slot * (C::NSTREAM * TT);
        if (!aligned(t, x0)) return;
        sflag[slot] = d ? 1 : 0;  // published by the arrive below (release) to the waiters (acquire)
        const int n = (MODE == kModeAdjGrad ? 4 : 2) + (d ? 1 : 0);
        mbar_arrive_expect_tx(&full_t[slot], n * C::TSLOT);
        tma_load_3d(t + 0 * TT, &tm_um, x0, y0, z, &full_t[slot]);
        tma_load_3d(t + 1 * TT, &tm_b, x0, y0, z, &full_t[slot]);
        if (d) tma_load_3d(t + 2 * TT, &tm_s, x0, y0, z, &full_t[slot]);
        if (MODE == kModeAdjGrad) {
          tma_load_3d(t + 3 * TT, &tm_uj, x0, y0, z, &full_t[slot]);
          tma_load_3d(t + 4 * TT, &tm_g, x0, y0, z, &full_t[slot]);
        }
        ++itt;
      };
      for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
        int tx, ty, z0, z1;
        item_geom(item, tx, ty, z0, z1);
        if (z0 >= z1) continue;
        const int x0 = tx * kTX, y0 = ty * TY;
        // damping bits of the flag rows covered by this work tile
        const int fy0 = y0 / kTileFlagTY;
        const int fy1 = min(fy0 + TY / kTileFlagTY, a.flag_tiles_y);
        auto word = [&](int w) -> unsigned {
          unsigned v = 0;
          if (w < a.nzw)
            for (int fy = fy0; fy < fy1; ++fy)
              v |= __ldg(a.tbits + (static_cast<long long>(fy) * a.tiles_x + tx) * a.nzw + w);
          return v;
        };
        int wcur = z0 >> 5;
        unsigned bits = word(wcur), bits_next = word(wcur + 1);
        for (int p = z0; p < min(z0 + R, z1 + R) && ok; ++p) issue_u(x0, y0, p);
        for (int z = z0; z < z1 && ok; ++z) {
          if (z + R < z1 + R) issue_u(x0, y0, z + R);
          if ((z >> 5) != wcur) {
            wcur = z >> 5;
            bits = bits_next;
            bits_next = word(wcur + 1);
          }
          if (ok) issue_t(x0, y0, z, (bits >> (z & 31)) & 1u);
        }
      }
      if (*abort_flag) {
        // let issued copies land (bounded) before shared memory goes away
        const uint64_t t0 = global_timer_ns();
        for (uint32_t j = iu > C::NSU ? iu - C::NSU : 0; j < iu; ++j)
          while (!mbar_try_wait(&full_u[j % C::NSU], (j / C::NSU) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
          }
        for (uint32_t j = itt > C::NST ? itt - C::NST : 0; j < itt; ++j)
          while (!mbar_try_wait(&full_t[j % C::NST], (j / C::NST) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
          }
        atomicCAS(a.err, 0, static_cast<int>(kErrWaitFull));
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  const int ty0 = warp * NY;  // first tile row of this thread
  uint32_t ub = 0;            // u-ring position of the current item's first plane
  uint32_t tpos = 0;          // tile-ring position of the next plane
  auto release = [&](uint64_t *bar) {
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
  };
  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    int tx, ty, z0, z1;
    item_geom(item, tx, ty, z0, z1);
    if (z0 >= z1) continue;
    const int gx = tx * kTX + lane;
    const int y0 = ty * TY;
    const bool xin = gx < a.g.nx;
    bool yin[NY];
    long long roff[NY];  // in-plane offset of each row (clamped inside the grid)
#pragma unroll
    for (int r = 0; r < NY; ++r) {
      const int gy = y0 + ty0 + r;
      yin[r] = xin && gy < a.g.ny;
      roff[r] = static_cast<long long>(min(gy, a.g.ny - 1)) * a.g.pitch + min(gx, a.g.nx - 1);
    }

    // z queue: q[r][j] = u^n at plane z - R + j
    float q[NY][2 * R + 1];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int p = z0 - R + j;
#pragma unroll
      for (int r = 0; r < NY; ++r)
        q[r][j] = (p >= 0 && yin[r]) ? __ldg(a.u + p * a.g.plane + roff[r]) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const uint32_t pos = ub + j;
      const uint32_t slot = pos % C::NSU;
      mbar_wait_bounded(&full_u[slot], (pos / C::NSU) & 1, abort_flag);
      const float *P = uring + slot * (C::USLOT / 4);
#pragma unroll
      for (int r = 0; r < NY; ++r) q[r][R + j] = P[(ty0 + r + R) * C::PW + lane + C::RX];
      if (z0 + j >= z1) release(&empty_u[slot]);  // trailing plane of a short chunk: centre only
    }

    for (int z = z0; z < z1; ++z) {
      // centre of plane z + R into the queue
      {
        const uint32_t pos = ub + (z + R - z0);
        const uint32_t slot = pos % C::NSU;
        mbar_wait_bounded(&full_u[slot], (pos / C::NSU) & 1, abort_flag);
        const float *P = uring + slot * (C::USLOT / 4);
#pragma unroll
        for (int r = 0; r < NY; ++r) q[r][2 * R] = P[(ty0 + r + R) * C::PW + lane + C::RX];
        if (z + R >= z1) release(&empty_u[slot]);
      }
      // x / y neighbours from the halo'd plane z (waited for as a centre plane)
      const uint32_t zslot = (ub + (z - z0)) % C::NSU;
      const float *P = uring + zslot * (C::USLOT / 4);
      float lap[NY];
      {
        float col[NY + 2 * R];
#pragma unroll
        for (int i = 0; i < NY + 2 * R; ++i) col[i] = P[(ty0 + i) * C::PW + lane + C::RX];
#pragma unroll
        for (int r = 0; r < NY; ++r) {
          const float *pc = P + (ty0 + r + R) * C::PW + lane + C::RX;
          float l = a.c.c0 * q[r][R];
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            l = fmaf(a.c.cx[j], pc[j] + pc[-j], l);
            l = fmaf(a.c.cy[j], col[R + r + j] + col[R + r - j], l);
            l = fmaf(a.c.cz[j], q[r][R + j] + q[r][R - j], l);
          }
          lap[r] = l;
        }
      }
      release(&empty_u[zslot]);

      // pointwise tiles of plane z
      const uint32_t tslot = tpos % C::NST;
      mbar_wait_bounded(&full_t[tslot], (tpos / C::NST) & 1, abort_flag);
      ++tpos;
      const float *T = tring + tslot * (C::NSTREAM * TT);
      const bool d = sflag[tslot] != 0;
      const long long po = static_cast<long long>(z) * a.g.plane;
      const bool live = !*abort_flag;
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        const int ti = (ty0 + r) * kTX + lane;
        const float c = q[r][R];
        const float dd = c - T[ti];
        const float sv = d ? T[2 * TT + ti] : 0.f;
        const float bl = T[TT + ti] * lap[r];
        const float un = fmaf(sv, dd, c + dd) + bl;
        if (yin[r] && live) {
          a.out[po + roff[r]] = un;
          if (MODE == kModeAdjGrad)
            a.grad[po + roff[r]] = fmaf(a.neg_inv_dt2 * T[3 * TT + ti], fmaf(sv, dd, bl), T[4 * TT + ti]);
        }
      }
      release(&empty_t[tslot]);
#pragma unroll
      for (int r = 0; r < NY; ++r)
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) q[r][j] = q[r][j + 1];
    }
    ub += static_cast<uint32_t>(z1 + R - z0);
  }
}

}  // namespace wp
