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
// This file holds the kernel of space orders up to 8 (half-order R <= 4); the
// wider stencils have their own layout (stencil3d_hi.cuh).
//
// GB300 design.  Persistent CTAs walk (TX x TY tile, z-chunk) work items in a
// static round-robin order and stream each chunk along z.  A producer warp issues
// TMA (cp.async.bulk.tensor) loads, P planes ahead of the compute, into two
// shared rings guarded by full/empty mbarriers:
//   - the halo'd u^n plane, (TX + 2 RX) x (TY + 2R), ring depth R + 1 + P (TMA's
//     zero fill outside the tensor supplies the Dirichlet ghosts);
//   - the pointwise tiles u^{n-1}, b, s (and u^j, g), ring depth P + 1; s only for
//     planes whose tile holds damping (per-tile z bitmask, one word per 32 planes).
// 8 consumer warps compute.  Each lane owns NX adjacent x points (NX = 2: packed
// FP32x2 arithmetic, FFMA2/FADD2, and 8-byte shared loads) in NY consecutive
// rows: it loads its column of the plane once for all y neighbours, reads x
// neighbours from the plane and keeps z neighbours in a register queue.  This
// keeps both the shared-memory traffic and the instructions issued per point
// low enough for HBM to be the bound.
// Every wait is bounded (%globaltimer, limit a.wait_ns); a timeout sets an abort
// flag, the producer lets its copies land, and the error word reports it.
#pragma once

#include <type_traits>

#include "wp_device.cuh"

namespace wp {

constexpr int kConsumerWarps = 8;
constexpr int kThreads3d = (kConsumerWarps + 1) * 32;
constexpr int kFlagTX = 32;                 // x extent of a damping-flag tile
constexpr int kTileFlagTY = 16;             // y extent of a damping-flag tile

enum StencilMode : int { kModeFwd = 0, kModeAdjGrad = 1 };

// Tile parameters, chosen by measurement; the -D overrides exist for sweeps.
#ifndef WP_NX
#define WP_NX 2          // x points per lane
#endif
#ifndef WP_NY_LO
#define WP_NY_LO 2       // rows per lane
#endif
#ifndef WP_MINB_LO
#define WP_MINB_LO 2     // CTAs per SM the compiler must fit
#endif
#ifndef WP_ZU
#define WP_ZU 2          // planes per unrolled z step (1..4)
#endif
#ifndef WP_P_ADJ
#define WP_P_ADJ 2       // planes in flight, adjoint+gradient mode (two CTAs per SM)
#endif
#ifndef WP_ZALT
#define WP_ZALT 1        // odd z-chunks of a column swept downward
#endif


template <int R, int MODE>
struct Cfg3d {
  static_assert(R >= 1 && R <= 4, "half-orders above 4 use stencil3d_hi_kernel");
  static constexpr int NX = WP_NX;
  static constexpr int NY = WP_NY_LO;
  static constexpr int TX = 32 * NX;                                 // tile width
  static constexpr int TY = kConsumerWarps * NY;                     // tile height
  static constexpr int RX = (R + 3) / 4 * 4;                         // x halo rounded to 16 bytes
  static constexpr int RE = (R + 1) / 2 * 2;                         // x window half-width (even)
  static constexpr int PW = TX + 2 * RX;
  static constexpr int PH = TY + 2 * R;
  static constexpr int P = MODE == kModeAdjGrad ? WP_P_ADJ : 3;      // planes in flight ahead
  static constexpr int MINB = WP_MINB_LO;                            // CTAs per SM to fit
  static constexpr int ZU = WP_ZU;                                   // planes per unrolled z step
  static constexpr bool ZALT = WP_ZALT != 0;                         // alternate sweep directions
  static constexpr int NSU = R + 1 + P;                              // u ring depth
  static constexpr int NST = P + 1;                                  // tile ring depth
  static constexpr int NSTREAM = MODE == kModeAdjGrad ? 5 : 3;       // um, b, s [, uj, g]
  static constexpr int USLOT = ((PW * PH * 4 + 127) / 128) * 128;    // bytes per u slot
  static constexpr int TSLOT = TX * TY * 4;                          // bytes per tile
  static constexpr int T_OFF = NSU * USLOT;
  static constexpr int BAR_OFF = T_OFF + NST * NSTREAM * TSLOT;
  static constexpr int SMEM = BAR_OFF + (2 * (NSU + NST) + 1) * 8 + NST * 4 + 16;
  static_assert(RX >= RE, "x halo must cover the x window");
};

struct Stencil3dArgs {
  FieldGeom g;
  LapCoef c;
  const float *u;               // u^n (plain loads of the z-halo below a chunk)
  float *out;                   // u^{n+1} (may alias u^{n-1})
  float *grad;                  // adjoint+gradient: gradient (read-modify-write)
  float neg_inv_dt2;            // -1 / dt^2
  const unsigned *tbits;        // [flag_tiles_y][flag_tiles_x][nzw]: bit z set where the flag tile has eta != 0
  int nzw;                      // 32-bit words per flag tile (ceil(nz / 32))
  int flag_tiles_x, flag_tiles_y;
  int tiles_x, tiles_y;         // work tiles (TX x TY)
  int zchunk, nzc;              // planes per item, chunks per column
  int nitems;                   // tiles_x * tiles_y * nzc
  int *err;
  // updated box [bx0, bx1) x [by0, by1) x [bz0, bz1) (the whole grid normally; bx0 a
  // multiple of 4); neighbours outside it are read, only points inside are written
  int bx0, by0, bz0, bx1, by1, bz1;
  unsigned long long wait_ns;   // a wait gives up after this long (0: at each item's start, see wp_set_wait_limit)
  int pdl;                      // launch with programmatic stream serialization
};



// ---- scalar / packed-pair arithmetic -------------------------------------
template <int NX> struct Vec;
template <> struct Vec<1> { typedef float T; };
template <> struct Vec<2> { typedef float2 T; };

__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
template <class V> __device__ __forceinline__ V vsplat(float c);
template <> __device__ __forceinline__ float vsplat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 vsplat<float2>(float c) { return make_float2(c, c); }
template <class V> __device__ __forceinline__ V vld(const float *p) { return *reinterpret_cast<const V *>(p); }

// tm: [0] u^n (halo'd plane box), [1] u^{n-1}, [2] b, [3] s, [4] u^j, [5] g (tile boxes)
template <int R, int MODE>
__global__ void __launch_bounds__(kThreads3d, Cfg3d<R, MODE>::MINB)
    stencil3d_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_um,
                     const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_s,
                     const __grid_constant__ CUtensorMap tm_uj, const __grid_constant__ CUtensorMap tm_g,
                     const Stencil3dArgs a) {
  using C = Cfg3d<R, MODE>;
  constexpr int NX = C::NX, NY = C::NY, TX = C::TX, TY = C::TY, TT = TX * TY;
  using V = typename Vec<NX>::T;
  extern __shared__ __align__(128) unsigned char smem[];
  float *uring = reinterpret_cast<float *>(smem);
  float *tring = reinterpret_cast<float *>(smem + C::T_OFF);  // [NST][NSTREAM][TT]
  uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + C::BAR_OFF);
  uint64_t *empty_u = full_u + C::NSU;
  uint64_t *full_t = empty_u + C::NSU;
  uint64_t *empty_t = full_t + C::NST;
  uint64_t *never = empty_t + C::NST;  // completed by nothing: the zero wait limit's first wait
  volatile int *sflag = reinterpret_cast<volatile int *>(never + 1);  // [NST]: s loaded
  volatile int *abort_flag = sflag + C::NST;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int cta = static_cast<int>(blockIdx.x);
  const int ncta = static_cast<int>(gridDim.x);
  const CUtensorMap *map_u = &tm_u;
  const CUtensorMap *map_um = &tm_um;
  float *const outp = a.out;
  if (tid == 0) {
    for (int i = 0; i < C::NSU; ++i) {
      mbar_init(&full_u[i], 1);
      mbar_init(&empty_u[i], kConsumerWarps);
    }
    for (int i = 0; i < C::NST; ++i) {
      mbar_init(&full_t[i], 1);
      mbar_init(&empty_t[i], kConsumerWarps);
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

  // Items of this CTA, round-robin: in every round the CTAs hold consecutive items
  // (neighbouring tiles and a tile's adjacent z-chunks), so halos meet in L2.
  const int item_end = a.nitems;
  auto first_item = [&](int i) -> int { return cta + i * ncta; };
  // With ZALT, odd chunks of a column are swept downward: two adjacent chunks then
  // read the planes around their common face at about the same time (both at the
  // start or both at the end of the chunk), so the second read hits L2 (measured at
  // SO8 on 336^3: 21 MB less DRAM read per launch, the z-halo re-reads).  Loops run
  // over a sweep index z in [z0, z1) (halos z0 - R .. z1 - 1 + R); phys() maps it to
  // the plane.  The z neighbours' sums are symmetric, so results do not depend on
  // the direction.  Orders above 8 are not HBM-bound and keep upward sweeps.
  auto item_geom = [&](int item, int &tx, int &ty, int &z0, int &z1, int &dir) {
    const int tile = item / a.nzc, zc = item - tile * a.nzc;
    tx = tile % a.tiles_x;
    ty = tile / a.tiles_x;
    z0 = a.bz0 + zc * a.zchunk;
    z1 = min(z0 + a.zchunk, a.bz1);
    dir = (C::ZALT && (zc & 1)) ? -1 : 1;
  };

  if (warp == kConsumerWarps) {
    // ---------------- producer (one lane) ----------------
    if (lane == 0) {
      prefetch_tensormap(map_u);
      prefetch_tensormap(map_um);
      prefetch_tensormap(&tm_b);
      prefetch_tensormap(&tm_s);
      if (MODE == kModeAdjGrad) {
        prefetch_tensormap(&tm_uj);
        prefetch_tensormap(&tm_g);
      }
      uint32_t iu = 0, itt = 0;  // planes issued into each ring
      int cz0 = 0, cz1 = 0, cdir = 1;  // current item's chunk and sweep direction
      auto phys = [&](int p) -> int { return cdir > 0 ? p : cz0 + cz1 - 1 - p; };
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
        if (iu >= C::NSU && !mbar_wait_bounded(&empty_u[slot], ((iu / C::NSU) - 1) & 1, abort_flag, a.wait_ns)) {
          ok = false;
          return;
        }
        float *dst = uring + slot * (C::USLOT / 4);
        if (!aligned(dst, x0 - C::RX)) return;
        mbar_arrive_expect_tx(&full_u[slot], C::PW * C::PH * 4);
        tma_load_3d(dst, map_u, x0 - C::RX, y0 - R, phys(p), &full_u[slot]);
        ++iu;
      };
      auto issue_t = [&](int x0, int y0, int zs, bool d) {
        const int z = phys(zs);
        const uint32_t slot = itt % C::NST;
        if (itt >= C::NST && !mbar_wait_bounded(&empty_t[slot], ((itt / C::NST) - 1) & 1, abort_flag, a.wait_ns)) {
          ok = false;
          return;
        }
        float *t = tring + slot * (C::NSTREAM * TT);
        if (!aligned(t, x0)) return;
        sflag[slot] = d ? 1 : 0;  // published by the arrive below (release) to the waiters (acquire)
        const int n = (MODE == kModeAdjGrad ? 4 : 2) + (d ? 1 : 0);
        mbar_arrive_expect_tx(&full_t[slot], n * C::TSLOT);
        tma_load_3d(t + 0 * TT, map_um, x0, y0, z, &full_t[slot]);
        tma_load_3d(t + 1 * TT, &tm_b, x0, y0, z, &full_t[slot]);
        if (d) tma_load_3d(t + 2 * TT, &tm_s, x0, y0, z, &full_t[slot]);
        if (MODE == kModeAdjGrad) {
          tma_load_3d(t + 3 * TT, &tm_uj, x0, y0, z, &full_t[slot]);
          tma_load_3d(t + 4 * TT, &tm_g, x0, y0, z, &full_t[slot]);
        }
        ++itt;
      };
      for (int it = 0, item = first_item(0); item < item_end && ok; item = first_item(++it)) {
        int tx, ty, z0, z1, dir;
        item_geom(item, tx, ty, z0, z1, dir);
        if (z0 >= z1) continue;
        cz0 = z0;
        cz1 = z1;
        cdir = dir;
        const int x0 = a.bx0 + tx * TX, y0 = a.by0 + ty * TY;
        // damping bits of the flag tiles covered by this work tile
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
        unsigned bits = word(wcur), bits_next = word(wcur + dir);
        for (int p = z0; p < z0 + R && ok; ++p) issue_u(x0, y0, p);
        for (int z = z0; z < z1 && ok; ++z) {
          issue_u(x0, y0, z + R);
          const int pz = phys(z);
          if ((pz >> 5) != wcur) {
            wcur = pz >> 5;
            bits = bits_next;
            bits_next = word(wcur + dir);
          }
          if (ok) issue_t(x0, y0, z, (bits >> (pz & 31)) & 1u);
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
  const int ty0 = warp * NY;          // first tile row of this lane
  const int cx0 = C::RX + NX * lane;  // this lane's first column in a plane row
  uint32_t ub = 0;                    // u-ring position of the current item's first plane
  uint32_t tpos = 0;                  // tile-ring position of the next plane
  auto release = [&](uint64_t *bar) {
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
  };
  for (int it = 0, item = first_item(0); item < item_end; item = first_item(++it)) {
    int tx, ty, z0, z1, dir;
    item_geom(item, tx, ty, z0, z1, dir);
    if (z0 >= z1) continue;
    // a zero wait limit gives up here, on a barrier that nothing completes
    if (a.wait_ns == 0) mbar_wait_first(never, 0, abort_flag, 0);
    auto phys = [&](int p) -> int { return dir > 0 ? p : z0 + z1 - 1 - p; };
    const int gx = a.bx0 + tx * TX + NX * lane;
    const int y0 = a.by0 + ty * TY;
    const bool xin0 = gx < a.bx1;
    const bool xin1 = NX == 2 && gx + 1 < a.bx1;
    bool yin[NY];
    long long rbase[NY];  // in-plane offset of each row (row clamped inside the grid)
#pragma unroll
    for (int r = 0; r < NY; ++r) {
      const int gy = y0 + ty0 + r;
      yin[r] = gy < a.by1;
      rbase[r] = static_cast<long long>(min(gy, a.g.ny - 1)) * a.g.pitch;
    }
    const int gxc0 = min(gx, a.g.nx - 1), gxc1 = min(gx + 1, a.g.nx - 1);

    // z queue: q[r][o + j] = u^n at plane z - R + j (o = offset of the plane in an unrolled step)
    V q[NY][2 * R + C::ZU];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int p = phys(z0 - R + j);
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        const float *src = a.u + p * a.g.plane + rbase[r];
        const bool ok = p >= 0 && p < a.g.nz && yin[r];
        if constexpr (NX == 2) {
          q[r][j] = make_float2(ok && xin0 ? __ldg(src + gxc0) : 0.f, ok && xin1 ? __ldg(src + gxc1) : 0.f);
        } else {
          q[r][j] = ok && xin0 ? __ldg(src + gxc0) : 0.f;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const uint32_t pos = ub + j;
      const uint32_t slot = pos % C::NSU;
      if (j == 0)  // the item's first wait
        mbar_wait_first(&full_u[slot], (pos / C::NSU) & 1, abort_flag, a.wait_ns);
      else
        mbar_wait_bounded(&full_u[slot], (pos / C::NSU) & 1, abort_flag, a.wait_ns);
      const float *P = uring + slot * (C::USLOT / 4);
#pragma unroll
      for (int r = 0; r < NY; ++r) q[r][R + j] = vld<V>(P + (ty0 + r + R) * C::PW + cx0);
      if (z0 + j >= z1) release(&empty_u[slot]);  // trailing plane of a short chunk: centre only
    }

    // One plane of the sweep; o (a compile-time offset) is where plane z - R sits
    // in the queue, so an unrolled step of U planes rotates the queue only once.
    auto plane = [&](int z, auto oc) {
      constexpr int o = decltype(oc)::value;
        // centre of plane z + R into the queue
        {
          const uint32_t pos = ub + (z + R - z0);
          const uint32_t slot = pos % C::NSU;
          mbar_wait_bounded(&full_u[slot], (pos / C::NSU) & 1, abort_flag, a.wait_ns);
          const float *P = uring + slot * (C::USLOT / 4);
#pragma unroll
          for (int r = 0; r < NY; ++r) q[r][2 * R + o] = vld<V>(P + (ty0 + r + R) * C::PW + cx0);
          if (z + R >= z1) release(&empty_u[slot]);
        }
        // x / y neighbours from the halo'd plane z (waited for as a centre plane)
        const uint32_t zslot = (ub + (z - z0)) % C::NSU;
        const float *P = uring + zslot * (C::USLOT / 4);
        V lap[NY];
        {
          V col[NY + 2 * R];
#pragma unroll
          for (int i = 0; i < NY + 2 * R; ++i) col[i] = vld<V>(P + (ty0 + i) * C::PW + cx0);
#pragma unroll
          for (int r = 0; r < NY; ++r) {
            const float *pc = P + (ty0 + r + R) * C::PW + cx0;
            // sums of the symmetric neighbour pairs at distance j along x, y, z
            auto ysum = [&](int j) -> V { return vadd(col[R + r + j], col[R + r - j]); };
            auto zsum = [&](int j) -> V { return vadd(q[r][o + R + j], q[r][o + R - j]); };
            V l = vmul(vsplat<V>(a.c.c0), q[r][o + R]);
            if constexpr (NX == 2) {
              // window w[k] = columns (cx0 - RE + 2k, +1): point 0 sits at RE, point 1 at RE + 1
              float2 w[C::RE + 1];
#pragma unroll
              for (int k = 0; k <= C::RE; ++k) w[k] = vld<float2>(pc - C::RE + 2 * k);
              auto win = [&](int i) -> float { return (i & 1) ? w[i >> 1].y : w[i >> 1].x; };
              auto xsum = [&](int j) -> float2 {
                if ((j & 1) == 0) return __fadd2_rn(w[(C::RE + j) >> 1], w[(C::RE - j) >> 1]);
                return make_float2(win(C::RE + j) + win(C::RE - j), win(C::RE + 1 + j) + win(C::RE + 1 - j));
              };
#pragma unroll
              for (int j = 1; j <= R; ++j) {
                l = vfma(vsplat<V>(a.c.cx[j]), xsum(j), l);
                l = vfma(vsplat<V>(a.c.cy[j]), ysum(j), l);
                l = vfma(vsplat<V>(a.c.cz[j]), zsum(j), l);
              }
            } else {
#pragma unroll
              for (int j = 1; j <= R; ++j) {
                l = vfma(vsplat<V>(a.c.cx[j]), vadd(vld<V>(pc + j), vld<V>(pc - j)), l);
                l = vfma(vsplat<V>(a.c.cy[j]), ysum(j), l);
                l = vfma(vsplat<V>(a.c.cz[j]), zsum(j), l);
              }
            }
            lap[r] = l;
          }
        }
        release(&empty_u[zslot]);

        // pointwise tiles of plane z
        const uint32_t tslot = tpos % C::NST;
        mbar_wait_bounded(&full_t[tslot], (tpos / C::NST) & 1, abort_flag, a.wait_ns);
        ++tpos;
        const float *T = tring + tslot * (C::NSTREAM * TT);
        const bool d = sflag[tslot] != 0;
        const long long po = static_cast<long long>(phys(z)) * a.g.plane;
        const bool live = !*abort_flag;
#pragma unroll
        for (int r = 0; r < NY; ++r) {
          const int ti = (ty0 + r) * TX + NX * lane;
          const V c = q[r][o + R];
          const V dd = vsub(c, vld<V>(T + ti));
          const V sv = d ? vld<V>(T + 2 * TT + ti) : vsplat<V>(0.f);
          const V bl = vmul(vld<V>(T + TT + ti), lap[r]);
          V un = vadd(vfma(sv, dd, vadd(c, dd)), bl);
          V gn = vsplat<V>(0.f);
          if (MODE == kModeAdjGrad)
            gn = vfma(vmul(vsplat<V>(a.neg_inv_dt2), vld<V>(T + 3 * TT + ti)), vfma(sv, dd, bl),
                      vld<V>(T + 4 * TT + ti));
          if (yin[r] && live &&
              WP_IN_BOUNDS(phys(z) >= 0 && phys(z) < a.g.nz && y0 + ty0 + r < a.g.ny && (!xin0 || gx < a.g.nx) &&
                               (!xin1 || gx + 1 < a.g.nx) && gx >= 0,
                           a.err)) {
            float *o = outp + po + rbase[r] + gx;
            float *gp = a.grad + po + rbase[r] + gx;
            if constexpr (NX == 2) {
              if (xin1) {
                *reinterpret_cast<float2 *>(o) = un;
                if (MODE == kModeAdjGrad) *reinterpret_cast<float2 *>(gp) = gn;
              } else if (xin0) {
                o[0] = un.x;
                if (MODE == kModeAdjGrad) gp[0] = gn.x;
              }
            } else {
              if (xin0) {
                o[0] = un;
                if (MODE == kModeAdjGrad) gp[0] = gn;
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
        for (int j = 0; j < 2 * R; ++j) q[r][j] = q[r][j + n];
    };
    int z = z0;
    for (; z + C::ZU <= z1; z += C::ZU) {
      plane(z, std::integral_constant<int, 0>{});
      if constexpr (C::ZU > 1) plane(z + 1, std::integral_constant<int, 1>{});
      if constexpr (C::ZU > 2) plane(z + 2, std::integral_constant<int, 2>{});
      if constexpr (C::ZU > 3) plane(z + 3, std::integral_constant<int, 3>{});
      rotate(std::integral_constant<int, C::ZU>{});
    }
    for (; z < z1; ++z) {
      plane(z, std::integral_constant<int, 0>{});
      rotate(std::integral_constant<int, 1>{});
    }
    ub += static_cast<uint32_t>(z1 + R - z0);
  }
}

}  // namespace wp
