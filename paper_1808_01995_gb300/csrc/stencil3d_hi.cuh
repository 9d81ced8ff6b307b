// K1 (3D) for space orders above 8 (half-order R = 5..8): the same update as
// stencil3d_kernel (Eq. fdWE-abc solved for u^{n+1}, the order-k Laplacian of
// Eq. fdSpace, and in adjoint+gradient mode the fused correlation of Eq. Grad),
// with a memory layout made for the wide stencils.
//
// Differences from the kernel of orders up to 8:
//   - The z register queue of a lane needs the centre value of plane z + R when
//     plane z is computed.  Here that value comes from a centre-only tile
//     (TX x TY, no halo) of plane z + R that travels in the pointwise tile ring
//     with plane z's u^{n-1}, b, s tiles, so the halo'd plane ring only holds the
//     planes in flight (NH slots) instead of R + 1 + P planes.  The planes above
//     a chunk are therefore streamed as centre tiles, not halo'd planes.
//   - Ring depths are powers of two and ring positions are plain counters, so a
//     plane's slot and phase cost a mask and a shift.
//   - The first 2R queue entries of a chunk (planes z0 - R .. z0 + R - 1) are
//     read with plain loads, all issued together.
// Lanes own two adjacent x points (packed FP32x2 arithmetic) in NY consecutive
// rows, as in the lower-order kernel; the Laplacian is accumulated in x, y and z
// partial sums.  Every wait is bounded (%globaltimer); a timeout sets the abort
// flag, the producer lets its copies land, and the error word reports it.
// The wait limit is a.wait_ns.
#pragma once

#include "stencil3d.cuh"

namespace wp {

#ifndef WP_HI_W
#define WP_HI_W 12       // consumer warps
#endif
#ifndef WP_HI_NX
#define WP_HI_NX 2       // x points per lane (2 or 4)
#endif
#ifndef WP_HI_NY
#define WP_HI_NY 2       // rows per lane, forward
#endif
#ifndef WP_HI_NY_ADJ
#define WP_HI_NY_ADJ 2   // rows per lane, adjoint+gradient
#endif
#ifndef WP_HI_NH
#define WP_HI_NH 4       // halo'd plane ring depth (power of two)
#endif
#ifndef WP_HI_NT
#define WP_HI_NT 4       // pointwise tile ring depth (power of two), forward
#endif
#ifndef WP_HI_NT_ADJ
#define WP_HI_NT_ADJ 4   // the same, adjoint+gradient (six streams per slot)
#endif
#ifndef WP_HI_ZU
#define WP_HI_ZU 4       // planes per unrolled z step
#endif
#ifndef WP_HI_DEC
#define WP_HI_DEC 40        // registers per thread left to the producer warpgroup
#endif
#ifndef WP_HI_ZALT
#define WP_HI_ZALT 1        // odd z-chunks of a column swept downward
#endif
#ifndef WP_HI_SPLIT_REGS
#define WP_HI_SPLIT_REGS 1  // producer warpgroup gives its registers to the consumer warpgroups (setmaxnreg)
#endif

template <int R, int MODE>
struct CfgHi {
  static constexpr int W = WP_HI_W;
  static constexpr int NX = WP_HI_NX;
  static constexpr int NP = NX / 2;  // packed pairs of a lane in a row
  static constexpr int NY = MODE == kModeAdjGrad ? WP_HI_NY_ADJ : WP_HI_NY;
  static constexpr int TX = 32 * NX;
  static constexpr int TY = W * NY;
  static constexpr int TT = TX * TY;
  static constexpr int RX = (R + 3) / 4 * 4;  // x halo rounded to 16 bytes
  static constexpr int RE = (R + 1) / 2 * 2;  // x window half-width (even)
  // a lane's x window: WL columns from WB before its first point (16-byte aligned
  // loads when NX = 4, 8-byte ones when NX = 2)
  static constexpr int WB = NX == 4 ? RX : RE;
  static constexpr int WL = NX == 4 ? NX + 2 * RX : NX + 2 * RE;
  static constexpr int PW = TX + 2 * RX;
  static constexpr int PH = TY + 2 * R;
  static constexpr int NH = WP_HI_NH;
  static constexpr int NT = MODE == kModeAdjGrad ? WP_HI_NT_ADJ : WP_HI_NT;
  static constexpr int ZU = WP_HI_ZU;
  // streams of a tile slot: u^{n-1}, b, s, centre of u^n at plane z + R [, u^j, g]
  static constexpr int S_UM = 0, S_B = 1, S_S = 2, S_UC = 3, S_UJ = 4, S_G = 5;
  static constexpr int NSTREAM = MODE == kModeAdjGrad ? 6 : 4;
  static constexpr int HSLOT = ((PW * PH * 4 + 127) / 128) * 128;
  static constexpr int TSLOT = TT * 4;
  static constexpr int T_OFF = NH * HSLOT;
  static constexpr int BAR_OFF = T_OFF + NT * NSTREAM * TSLOT;
  static constexpr int SMEM = BAR_OFF + (2 * (NH + NT) + 1) * 8 + NT * 4 + 16;
  // Without the register split: W consumer warps and one producer warp.  With it
  // (W a multiple of 4): W/4 consumer warpgroups and one producer warpgroup whose
  // first lane issues the copies; the producer warpgroup drops to DEC registers per
  // thread and the consumers rise to INC, within the block's launch allocation
  // (THREADS x LAUNCH_REGS, LAUNCH_REGS being what the launch bound lets ptxas use:
  // 65536 / THREADS rounded down to 8 after rounding THREADS up to whole warpgroups).
  static constexpr bool SPLIT_REGS = WP_HI_SPLIT_REGS != 0 && W % 4 == 0;
  static constexpr int THREADS = SPLIT_REGS ? (W + 4) * 32 : (W + 1) * 32;
  static constexpr int LAUNCH_REGS = (65536 / ((THREADS + 127) / 128 * 128)) / 8 * 8;
  static constexpr int DEC = WP_HI_DEC;
  static constexpr int INC_RAW = (THREADS * LAUNCH_REGS - 128 * DEC) / (W * 32) / 8 * 8;
  static constexpr int INC = INC_RAW > 248 ? 248 : INC_RAW;
  static_assert(!SPLIT_REGS || W * 32 * INC + 128 * DEC <= THREADS * LAUNCH_REGS, "register split over the launch");
  static_assert((NH & (NH - 1)) == 0 && (NT & (NT - 1)) == 0, "ring depths must be powers of two");
  static_assert(TSLOT % 128 == 0, "tile slots must stay 128-byte aligned");
  static_assert(RX >= RE, "x halo must cover the x window");
  static_assert(NX == 2 || NX == 4, "lanes own two or four x points");
  static_assert(WL % NX == 0 && WB >= R, "x window");
};

// f(integral_constant<int, I>) for I = 0 .. N - 1, unrolled at compile time
template <class F, int... I>
__device__ __forceinline__ void hi_unroll(F &&f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}

// tm: [0] u^n halo'd plane box, [1] u^{n-1}, [2] b, [3] s, [4] u^j, [5] g, [6] u^n (tile boxes)
// ISO: the three axes have the same spacing (cx = cy = cz): one coefficient per
// distance j multiplies the sum of the six neighbours at that distance.
template <int R, int MODE, bool ISO>
__global__ void __launch_bounds__(CfgHi<R, MODE>::THREADS, 1)
    stencil3d_hi_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_um,
                        const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_s,
                        const __grid_constant__ CUtensorMap tm_uj, const __grid_constant__ CUtensorMap tm_g,
                        const __grid_constant__ CUtensorMap tm_uc, const Stencil3dArgs a) {
  using C = CfgHi<R, MODE>;
  constexpr int NX = C::NX, NY = C::NY, TX = C::TX, TY = C::TY, TT = C::TT, W = C::W;
  using V = float2;
  extern __shared__ __align__(128) unsigned char smem[];
  float *hring = reinterpret_cast<float *>(smem);
  float *tring = reinterpret_cast<float *>(smem + C::T_OFF);  // [NT][NSTREAM][TT]
  uint64_t *full_h = reinterpret_cast<uint64_t *>(smem + C::BAR_OFF);
  uint64_t *empty_h = full_h + C::NH;
  uint64_t *full_t = empty_h + C::NH;
  uint64_t *empty_t = full_t + C::NT;
  uint64_t *never = empty_t + C::NT;  // completed by nothing: the zero wait limit's first wait
  volatile int *sflag = reinterpret_cast<volatile int *>(never + 1);  // [NT]: s loaded
  volatile int *abort_flag = sflag + C::NT;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < C::NH; ++i) {
      mbar_init(&full_h[i], 1);
      mbar_init(&empty_h[i], W);
    }
    for (int i = 0; i < C::NT; ++i) {
      mbar_init(&full_t[i], 1);
      mbar_init(&empty_t[i], W);
    }
    mbar_init(never, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();
  // Under a programmatic launch the kernel before this one on the stream may still
  // be running: it writes fields read here (and reads the one written here).  The
  // stencil itself does not let the next kernel launch early: measured, that
  // kernel's blocks then take SM room in the stencil's last round (SO16 shots
  // 2 us per step slower; without the early launch 1.5 us faster than no
  // programmatic launch at all).
  grid_dependency_wait();

  const int ncta = static_cast<int>(gridDim.x);
  const int cta = static_cast<int>(blockIdx.x);
  // With WP_HI_ZALT, odd chunks of a column are swept downward, so that two
  // adjacent chunks read the planes around their common face at about the same
  // time (both at the end of their sweeps) and the second read hits L2.  Loops run
  // over a sweep index z in [z0, z1) (halos z0 - R .. z1 - 1 + R); phys() maps it
  // to the plane.  The z neighbours' sums are symmetric, so results do not depend
  // on the direction.
  auto item_geom = [&](int item, int &tx, int &ty, int &z0, int &z1, int &dir) {
    const int tile = item / a.nzc, zc = item - tile * a.nzc;
    tx = tile % a.tiles_x;
    ty = tile / a.tiles_x;
    z0 = a.bz0 + zc * a.zchunk;
    z1 = min(z0 + a.zchunk, a.bz1);
    dir = (WP_HI_ZALT && (zc & 1)) ? -1 : 1;
  };

  if (warp >= W) {
    // ---------------- producer (one lane) ----------------
    if constexpr (C::SPLIT_REGS) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::DEC) : "memory");
    if (warp == W && lane == 0) {
      prefetch_tensormap(&tm_u);
      prefetch_tensormap(&tm_um);
      prefetch_tensormap(&tm_b);
      prefetch_tensormap(&tm_s);
      prefetch_tensormap(&tm_uc);
      if (MODE == kModeAdjGrad) {
        prefetch_tensormap(&tm_uj);
        prefetch_tensormap(&tm_g);
      }
      uint32_t ih = 0, it_ = 0;  // planes issued into each ring
      bool ok = true;
      auto aligned = [&](const float *dst, int x) -> bool {
        if ((smem_u32(dst) & 127u) == 0 && (x & 3) == 0) return true;
        atomicCAS(a.err, 0, static_cast<int>(kErrLaunch));
        *abort_flag = 1;
        ok = false;
        return false;
      };
      for (int item = cta; item < a.nitems && ok; item += ncta) {
        int tx, ty, z0, z1, dir;
        item_geom(item, tx, ty, z0, z1, dir);
        if (z0 >= z1) continue;
        auto phys = [&](int p) -> int { return dir > 0 ? p : z0 + z1 - 1 - p; };
        const int x0 = a.bx0 + tx * TX, y0 = a.by0 + ty * TY;
        const int fx0 = x0 / kFlagTX, fx1 = min((x0 + TX - 1) / kFlagTX + 1, a.flag_tiles_x);
        const int fy0 = y0 / kTileFlagTY, fy1 = min((y0 + TY - 1) / kTileFlagTY + 1, a.flag_tiles_y);
        auto word = [&](int w) -> unsigned {
          unsigned v = 0;
          if (w >= 0 && w < a.nzw)
            for (int fy = fy0; fy < fy1; ++fy)
              for (int fx = fx0; fx < fx1; ++fx)
                v |= __ldg(a.tbits + (static_cast<long long>(fy) * a.flag_tiles_x + fx) * a.nzw + w);
          return v;
        };
        int wcur = phys(z0) >> 5;
        unsigned bits = word(wcur);
        for (int zs = z0; zs < z1 && ok; ++zs) {
          const int z = phys(zs);  // the plane updated at this step of the sweep
          if ((z >> 5) != wcur) {
            wcur = z >> 5;
            bits = word(wcur);
          }
          const bool d = (bits >> (z & 31)) & 1u;
          // tile slot of plane z: u^{n-1}, b, [s], centre of plane z + R [, u^j, g]
          {
            const uint32_t slot = it_ & (C::NT - 1);
            if (it_ >= C::NT && !mbar_wait_bounded(&empty_t[slot], ((it_ / C::NT) - 1) & 1, abort_flag, a.wait_ns)) {
              ok = false;
              break;
            }
            float *t = tring + slot * (C::NSTREAM * TT);
            if (!aligned(t, x0)) break;
            sflag[slot] = d ? 1 : 0;  // published by the arrive below (release) to the waiters (acquire)
            const int n = (MODE == kModeAdjGrad ? 5 : 3) + (d ? 1 : 0);
            mbar_arrive_expect_tx(&full_t[slot], n * C::TSLOT);
            tma_load_3d(t + C::S_UM * TT, &tm_um, x0, y0, z, &full_t[slot]);
            tma_load_3d(t + C::S_B * TT, &tm_b, x0, y0, z, &full_t[slot]);
            if (d) tma_load_3d(t + C::S_S * TT, &tm_s, x0, y0, z, &full_t[slot]);
            tma_load_3d(t + C::S_UC * TT, &tm_uc, x0, y0, phys(zs + R), &full_t[slot]);
            if (MODE == kModeAdjGrad) {
              tma_load_3d(t + C::S_UJ * TT, &tm_uj, x0, y0, z, &full_t[slot]);
              tma_load_3d(t + C::S_G * TT, &tm_g, x0, y0, z, &full_t[slot]);
            }
            ++it_;
          }
          // halo'd plane z of u^n
          {
            const uint32_t slot = ih & (C::NH - 1);
            if (ih >= C::NH && !mbar_wait_bounded(&empty_h[slot], ((ih / C::NH) - 1) & 1, abort_flag, a.wait_ns)) {
              ok = false;
              break;
            }
            float *dst = hring + slot * (C::HSLOT / 4);
            if (!aligned(dst, x0 - C::RX)) break;
            mbar_arrive_expect_tx(&full_h[slot], C::PW * C::PH * 4);
            tma_load_3d(dst, &tm_u, x0 - C::RX, y0 - R, z, &full_h[slot]);
            ++ih;
          }
        }
      }
      if (*abort_flag) {
        // let issued copies land (bounded) before shared memory goes away
        const uint64_t t0 = global_timer_ns();
        for (uint32_t j = ih > C::NH ? ih - C::NH : 0; j < ih; ++j)
          while (!mbar_try_wait(&full_h[j & (C::NH - 1)], (j / C::NH) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
          }
        for (uint32_t j = it_ > C::NT ? it_ - C::NT : 0; j < it_; ++j)
          while (!mbar_try_wait(&full_t[j & (C::NT - 1)], (j / C::NT) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
          }
        atomicCAS(a.err, 0, static_cast<int>(kErrWaitFull));
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  if constexpr (C::SPLIT_REGS) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::INC) : "memory");
  constexpr int NP = C::NP;           // packed pairs of a lane in a row
  const int ty0 = warp * NY;          // first tile row of this lane
  const int cx0 = C::RX + NX * lane;  // this lane's first column in a halo'd plane row
  uint32_t hpos = 0, tpos = 0;        // ring positions of the next plane
  auto release = [&](uint64_t *bar) {
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
  };
  const V nidt2 = make_float2(a.neg_inv_dt2, a.neg_inv_dt2);
  // the lane's NX consecutive values at p (one 16-byte load when NX = 4) as NP pairs
  auto ldp = [](const float *p, V *out) {
    if constexpr (NX == 4) {
      const float4 v = *reinterpret_cast<const float4 *>(p);
      out[0] = make_float2(v.x, v.y);
      out[1] = make_float2(v.z, v.w);
    } else {
      out[0] = vld<V>(p);
    }
  };
  auto stp = [](float *p, const V *v) {
    if constexpr (NX == 4)
      *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    else
      *reinterpret_cast<V *>(p) = v[0];
  };

  for (int item = cta; item < a.nitems; item += ncta) {
    int tx, ty, z0, z1, dir;
    item_geom(item, tx, ty, z0, z1, dir);
    if (z0 >= z1) continue;
    // a zero wait limit gives up here, on a barrier that nothing completes
    if (a.wait_ns == 0) mbar_wait_first(never, 0, abort_flag, 0);
    auto phys = [&](int p) -> int { return dir > 0 ? p : z0 + z1 - 1 - p; };
    const int gx = a.bx0 + tx * TX + NX * lane;
    const int y0 = a.by0 + ty * TY;
    int nin = 0;  // this lane's points inside the box: a prefix of its NX points
#pragma unroll
    for (int i = 0; i < NX; ++i) nin += gx + i < a.bx1 ? 1 : 0;
    bool yin[NY];
    int rofs[NY];  // in-plane offset of each row (row clamped inside the grid)
    // this lane's first point of each row in plane 0 of the output (and gradient):
    // a plane's store address is then one 64-bit add
    float *obase[NY];
    float *gbase[NY];
#pragma unroll
    for (int r = 0; r < NY; ++r) {
      const int gy = y0 + ty0 + r;
      yin[r] = gy < a.by1;
      rofs[r] = min(gy, a.g.ny - 1) * a.g.pitch;
      obase[r] = a.out + rofs[r] + gx;
      gbase[r] = MODE == kModeAdjGrad ? a.grad + rofs[r] + gx : nullptr;
    }

    // z queue: q[r][p][o + j] = u^n at plane z - R + j (o = offset of the plane in an
    // unrolled step); planes z0 - R .. z0 + R - 1 first, with plain loads
    V q[NY][NP][2 * R + C::ZU];
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      const int pl = phys(z0 - R + j);
      const bool pin = pl >= 0 && pl < a.g.nz;
      const float *src = a.u + static_cast<long long>(pin ? pl : 0) * a.g.plane;
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        const bool ok = pin && yin[r];
        float v[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) v[i] = ok && i < nin ? __ldg(src + rofs[r] + min(gx + i, a.g.nx - 1)) : 0.f;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) q[r][pp][j] = make_float2(v[2 * pp], v[2 * pp + 1]);
      }
    }

    auto plane = [&](int z, auto oc) {
      constexpr int o = decltype(oc)::value;
      // pointwise tiles of plane z (and the centre of plane z + R)
      const uint32_t tslot = tpos & (C::NT - 1);
      mbar_wait_bounded(&full_t[tslot], (tpos / C::NT) & 1, abort_flag, a.wait_ns);
      ++tpos;
      const float *T = tring + tslot * (C::NSTREAM * TT);
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        V t[NP];
        ldp(T + C::S_UC * TT + (ty0 + r) * TX + NX * lane, t);
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) q[r][pp][2 * R + o] = t[pp];
      }
      // x / y neighbours from the halo'd plane z
      const uint32_t hslot = hpos & (C::NH - 1);
      mbar_wait_bounded(&full_h[hslot], (hpos / C::NH) & 1, abort_flag, a.wait_ns);
      ++hpos;
      const float *P = hring + hslot * (C::HSLOT / 4);
      V lap[NY][NP];
      {
        V col[NY + 2 * R][NP];
#pragma unroll
        for (int i = 0; i < NY + 2 * R; ++i) ldp(P + (ty0 + i) * C::PW + cx0, col[i]);
#pragma unroll
        for (int r = 0; r < NY; ++r) {
          // window w = columns cx0 - WB .. cx0 - WB + WL - 1 of the row, as pairs
          const float *pc = P + (ty0 + r + R) * C::PW + cx0 - C::WB;
          V w[C::WL / 2];
#pragma unroll
          for (int k = 0; k < C::WL / NX; ++k) ldp(pc + NX * k, &w[NP * k]);
          auto win = [&](int i) -> float { return (i & 1) ? w[i >> 1].y : w[i >> 1].x; };
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) {
            const int c0 = C::WB + 2 * pp;  // window index of the pair's first point
            auto xsum = [&](int j) -> V {
              if ((j & 1) == 0) return vadd(w[(c0 + j) >> 1], w[(c0 - j) >> 1]);
              return make_float2(win(c0 + j) + win(c0 - j), win(c0 + 1 + j) + win(c0 + 1 - j));
            };
            auto ysum = [&](int j) -> V { return vadd(col[R + r + j][pp], col[R + r - j][pp]); };
            auto zsum = [&](int j) -> V { return vadd(q[r][pp][o + R + j], q[r][pp][o + R - j]); };
            if constexpr (ISO) {
              // two chains (odd and even distances) of the six-neighbour sums
              auto nsum = [&](int j) -> V { return vadd(vadd(xsum(j), ysum(j)), zsum(j)); };
              V la = vfma(a.c.px[1], nsum(1), vmul(a.c.p0, q[r][pp][o + R]));
              V lb = vmul(a.c.px[2], nsum(2));
#pragma unroll
              for (int j = 3; j <= R; ++j) {
                if (j & 1)
                  la = vfma(a.c.px[j], nsum(j), la);
                else
                  lb = vfma(a.c.px[j], nsum(j), lb);
              }
              lap[r][pp] = vadd(la, lb);
            } else {
              // three partial sums (x, y, z) keep every chain of dependent FMAs at most R long
              V lx = vmul(a.c.p0, q[r][pp][o + R]);
              V ly = vmul(a.c.py[1], ysum(1));
              V lz = vmul(a.c.pz[1], zsum(1));
#pragma unroll
              for (int j = 1; j <= R; ++j) {
                lx = vfma(a.c.px[j], xsum(j), lx);
                if (j > 1) {
                  ly = vfma(a.c.py[j], ysum(j), ly);
                  lz = vfma(a.c.pz[j], zsum(j), lz);
                }
              }
              lap[r][pp] = vadd(lx, vadd(ly, lz));
            }
          }
        }
      }
      release(&empty_h[hslot]);

      const bool d = sflag[tslot] != 0;
      const int pz = phys(z);
      const long long po = static_cast<long long>(pz) * a.g.plane;
      const bool live = !*abort_flag;
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        const int ti = (ty0 + r) * TX + NX * lane;
        V um[NP], bv[NP], sv[NP], uj[NP], gv[NP], un[NP], gn[NP];
        ldp(T + C::S_UM * TT + ti, um);
        ldp(T + C::S_B * TT + ti, bv);
        if (d) {
          ldp(T + C::S_S * TT + ti, sv);
        } else {
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) sv[pp] = make_float2(0.f, 0.f);
        }
        if (MODE == kModeAdjGrad) {
          ldp(T + C::S_UJ * TT + ti, uj);
          ldp(T + C::S_G * TT + ti, gv);
        }
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
          const V c = q[r][pp][o + R];
          const V dd = vsub(c, um[pp]);
          const V bl = vmul(bv[pp], lap[r][pp]);
          un[pp] = vadd(vfma(sv[pp], dd, vadd(c, dd)), bl);
          if (MODE == kModeAdjGrad) gn[pp] = vfma(vmul(nidt2, uj[pp]), vfma(sv[pp], dd, bl), gv[pp]);
        }
        if (yin[r] && nin > 0 && live &&
            WP_IN_BOUNDS(pz >= 0 && pz < a.g.nz && y0 + ty0 + r < a.g.ny && gx >= 0 && gx + nin - 1 < a.g.nx,
                         a.err)) {
          float *op = obase[r] + po;
          float *gp = gbase[r] + po;
          if (nin == NX) {
            stp(op, un);
            if (MODE == kModeAdjGrad) stp(gp, gn);
          } else {
#pragma unroll
            for (int i = 0; i < NX - 1; ++i) {
              if (i < nin) {
                op[i] = (i & 1) ? un[i >> 1].y : un[i >> 1].x;
                if (MODE == kModeAdjGrad) gp[i] = (i & 1) ? gn[i >> 1].y : gn[i >> 1].x;
              }
            }
          }
        }
      }
      release(&empty_t[tslot]);
    };
    auto rotate = [&](auto nc) {
      constexpr int n = decltype(nc)::value;
#pragma unroll
      for (int r = 0; r < NY; ++r)
#pragma unroll
        for (int pp = 0; pp < NP; ++pp)
#pragma unroll
          for (int j = 0; j < 2 * R; ++j) q[r][pp][j] = q[r][pp][j + n];
    };
    int z = z0;
    for (; z + C::ZU <= z1; z += C::ZU) {
      hi_unroll([&](auto oc) { plane(z + decltype(oc)::value, oc); }, std::make_integer_sequence<int, C::ZU>{});
      rotate(std::integral_constant<int, C::ZU>{});
    }
    for (; z < z1; ++z) {
      plane(z, std::integral_constant<int, 0>{});
      rotate(std::integral_constant<int, 1>{});
    }
  }
}

}  // namespace wp
