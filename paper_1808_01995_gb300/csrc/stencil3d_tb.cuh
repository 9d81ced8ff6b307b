// K1 (3D), two time steps per pass (temporal blocking): from (u^{n-1}, u^n) the
// kernel produces u^{n+1} and u^{n+2} of the same leapfrog update as
// stencil3d_kernel, with the injection of q^n into u^{n+1} done in between:
//
//   u^{n+1} = u^n + (1 + s)(u^n - u^{n-1}) + b Lap u^n        (+ b P_s^T q^n)
//   u^{n+2} = u^{n+1} + (1 + s)(u^{n+1} - u^n) + b Lap u^{n+1}
//
// Each work item is a core tile of CW x CH points and a z-chunk.  Step 1 runs on
// the region = core grown by R (RX = 4 in x for TMA alignment) and by R planes in
// z, so that step 2 finds every neighbour of u^{n+1} it needs in shared memory;
// the region's rim is computed redundantly by the neighbouring items.  HBM sees
// u^{n-1}, u^n, b, s read once and u^{n+1}, u^{n+2} written once per two steps
// (halo re-reads meet in L2), about 0.6 of the bytes of two single steps.
//
// The per-point arithmetic (operand order included) is that of stencil3d_kernel
// and of the injection kernel, so the two-step path reproduces the single-step
// path bit for bit.  u^{n+1} and u^{n+2} go to buffers other than the inputs:
// neighbouring items read the inputs' halos while this one writes.
//
// Pipeline: lane 0 of warp 0 issues TMA loads into four mbarrier rings (the
// halo'd u^n plane; region tiles u^{n-1}, b, s; core tiles b, s of the step-2
// plane); step-1 output planes live in a ring of R + 1 region planes.  Eight
// warps (no separate producer warp, so that the register file allows the two z
// queues without spills): each lane owns two adjacent x points (packed FP32x2) in NY
// rows, for step 1 on the region and for step 2 on its core part, with z
// neighbours of u^n and of u^{n+1} in register queues.  Two named barriers per
// plane order the u^{n+1} ring.  Waits are bounded as in stencil3d_kernel.
#pragma once

#include <type_traits>

#include "stencil3d.cuh"

namespace wp {

#ifndef WP_TB_NY
#define WP_TB_NY 4       // rows per lane, R > 2 (one CTA per SM)
#endif
#ifndef WP_TB_WARPS
#define WP_TB_WARPS 8    // warps per CTA (each lane: two x points in NY rows)
#endif
#ifndef WP_TB_ZU
#define WP_TB_ZU 1       // planes per unrolled z step (1 or 2; 1 measured faster: smaller code)
#endif
#ifndef WP_TB_NY_LO
#define WP_TB_NY_LO 4    // rows per lane, R <= 2 (2: two CTAs per SM, measured slower)
#endif

constexpr int kTbMaxTargets = 64;  // injection targets handled inside the kernel

template <int R>
struct CfgTb {
  static_assert(R >= 1 && R <= 4, "the two-step kernel covers space orders 2..8");
  static constexpr int NX = 2;
  static constexpr int NY = R <= 2 ? WP_TB_NY_LO : WP_TB_NY;
  static constexpr int MINB = NY <= 2 && WP_TB_WARPS <= 8 ? 2 : 1;  // CTAs per SM the registers must allow
  static constexpr int W = 32 * NX;                // region width (step 1)
  static constexpr int WARPS = WP_TB_WARPS;
  static constexpr int H = WARPS * NY;             // region height
  static constexpr int RX = 4;                     // x rim, 16 bytes for TMA
  static constexpr int RE = (R + 1) / 2 * 2;       // x window half-width (even)
  static constexpr int CW = W - 2 * RX;            // core width (step 2)
  static constexpr int CH = H - 2 * R;             // core height
  static constexpr int UPW = W + 2 * RX;           // u^n plane box
  static constexpr int UPH = H + 2 * R;
  static constexpr int P = 2;                      // planes in flight ahead
  static constexpr int ZU = WP_TB_ZU;              // planes per unrolled z step
  static constexpr int NSU = R + 1 + P;            // u^n ring depth
  static constexpr int NST = P + 1;                // region tile ring depth
  static constexpr int NSC = P + 1;                // core tile ring depth
  static constexpr int NV = R + 1;                 // u^{n+1} ring depth
  static constexpr int USLOT = ((UPW * UPH * 4 + 127) / 128) * 128;
  static constexpr int TSLOT = W * H * 4;
  static constexpr int CSLOT = ((CW * CH * 4 + 127) / 128) * 128;
  static constexpr int VSLOT = W * H * 4;
  static constexpr int T_OFF = NSU * USLOT;
  static constexpr int C_OFF = T_OFF + NST * 3 * TSLOT;
  static constexpr int V_OFF = C_OFF + NSC * 2 * CSLOT;
  static constexpr int TGT_OFF = V_OFF + NV * VSLOT;                // injection targets (z, y, x)
  static constexpr int BAR_OFF = TGT_OFF + kTbMaxTargets * 16;
  static constexpr int SMEM = BAR_OFF + 2 * (NSU + NST + NSC) * 8 + (NST + NSC) * 4 + 16;
  static_assert(RX >= RE && RX >= R, "x rim must cover the x window");
  static_assert(CW > 0 && CH > 0, "empty core");
  static_assert((CW * 4) % 16 == 0, "core tile rows must be whole 16-byte units");
  static_assert(SMEM <= 232448, "shared memory of the two-step kernel exceeds 227 KB");
};

struct Stencil3dTbArgs {
  FieldGeom g;
  LapCoef c;
  float *out1;                  // u^{n+1}
  float *out2;                  // u^{n+2}
  const uint2 *tile_bits;       // [tile][nzw]: damping words of the tile's region (x) and core (y)
  int nzw;
  int tiles_x, tiles_y;         // core tiles
  int zchunk, nzc, nitems;
  int *err;
  // injection of data row `row` (+ *row_base) into u^{n+1}, arithmetic of inject_kernel
  int ntarget;                  // <= kTbMaxTargets
  const long long *target;      // pitched flat index of each target
  const int *rowptr, *pid;
  const float *w;
  const float *data;
  int npts;
  const long long *row_base;
  long long row;
  const float *b;               // pitched b (the injection weight)
};

constexpr int kThreadsTb = WP_TB_WARPS * 32;

// tm: [0] u^n (plane box UPW x UPH), [1] u^{n-1}, [2] b, [3] s (region boxes W x H),
//     [4] b, [5] s (core boxes CW x CH)
template <int R>
__global__ void __launch_bounds__(kThreadsTb, CfgTb<R>::MINB)
    stencil3d_tb_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_um,
                        const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_s,
                        const __grid_constant__ CUtensorMap tm_bc, const __grid_constant__ CUtensorMap tm_sc,
                        const Stencil3dTbArgs a) {
  using C = CfgTb<R>;
  constexpr int NX = C::NX, NY = C::NY, W = C::W, H = C::H, TT = W * H, CT = C::CSLOT / 4;
  using V = float2;
  extern __shared__ __align__(128) unsigned char smem[];
  float *uring = reinterpret_cast<float *>(smem);
  float *tring = reinterpret_cast<float *>(smem + C::T_OFF);  // [NST][3][TT]: u^{n-1}, b, s
  float *cring = reinterpret_cast<float *>(smem + C::C_OFF);  // [NSC][2][CT]: b, s (core)
  float *vring = reinterpret_cast<float *>(smem + C::V_OFF);  // [NV][TT]: u^{n+1} on the region
  uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + C::BAR_OFF);
  uint64_t *empty_u = full_u + C::NSU;
  uint64_t *full_t = empty_u + C::NSU;
  uint64_t *empty_t = full_t + C::NST;
  uint64_t *full_c = empty_t + C::NST;
  uint64_t *empty_c = full_c + C::NSC;
  volatile int *sflag_t = reinterpret_cast<volatile int *>(empty_c + C::NSC);  // [NST]
  volatile int *sflag_c = sflag_t + C::NST;                                    // [NSC]
  volatile int *abort_flag = sflag_c + C::NSC;
  int4 *tgt = reinterpret_cast<int4 *>(smem + C::TGT_OFF);  // (z, y, x, -) of each injection target

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < a.ntarget; i += blockDim.x) {
    const long long t = a.target[i];
    const int z = static_cast<int>(t / a.g.plane);
    const long long rem = t - static_cast<long long>(z) * a.g.plane;
    const int y = static_cast<int>(rem / a.g.pitch);
    tgt[i] = make_int4(z, y, static_cast<int>(rem - static_cast<long long>(y) * a.g.pitch), 0);
  }
  if (tid == 0) {
    for (int i = 0; i < C::NSU; ++i) {
      mbar_init(&full_u[i], 1);
      mbar_init(&empty_u[i], C::WARPS);
    }
    for (int i = 0; i < C::NST; ++i) {
      mbar_init(&full_t[i], 1);
      mbar_init(&empty_t[i], C::WARPS);
    }
    for (int i = 0; i < C::NSC; ++i) {
      mbar_init(&full_c[i], 1);
      mbar_init(&empty_c[i], C::WARPS);
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();

  const int item_end = a.nitems;
  auto first_item = [&](int i) -> int { return blockIdx.x + i * gridDim.x; };
  auto item_geom = [&](int item, int &tx, int &ty, int &z0, int &z1) {
    const int tile = item / a.nzc, zc = item - tile * a.nzc;
    tx = tile % a.tiles_x;
    ty = tile / a.tiles_x;
    z0 = zc * a.zchunk;
    z1 = min(z0 + a.zchunk, a.g.nz);
  };

  // ---------------- producer: lane 0 of warp 0, never blocking ----------------
  // The loads of this CTA's items form one sequence, consumed in the same order:
  // per item the 2R u^n planes below the region, then for every step-1 plane t
  // the u^n plane t + R, the region tiles of t and (once t - R >= z0) the core
  // tiles of t - R.  pump() issues the next loads while their ring slots are free;
  // warp 0 pumps before and while it waits, and every load that any warp waits
  // for is waited for by warp 0 in the same plane iteration.
  const bool producer = warp == 0 && lane == 0;
  struct Cursor {
    int it, item, tx, ty, z0, z1;
    int k;        // prologue plane (0 .. 2R-1), then 2R + (t - (z0 - R)) * 3 + sub
    bool done;
  } cur;
  uint32_t iu = 0, itt = 0, ic = 0;  // loads issued into each ring
  cur.it = 0;
  cur.item = first_item(0);
  cur.k = 0;
  cur.done = cur.item >= item_end;
  if (!cur.done) item_geom(cur.item, cur.tx, cur.ty, cur.z0, cur.z1);
  // damping words of the cursor's tile: the current 32-plane word of each kind and
  // the next one, loaded one word ahead so that the lookup rarely waits
  int dw[2] = {-2, -2};
  unsigned dcur[2] = {0u, 0u}, dnext[2] = {0u, 0u};
  auto tile_word = [&](int tile, int w, int kind) -> unsigned {
    if (w < 0 || w >= a.nzw) return 0u;
    const uint2 v = __ldg(a.tile_bits + static_cast<long long>(tile) * a.nzw + w);
    return kind == 0 ? v.x : v.y;
  };
  auto damped = [&](int z, int kind) -> bool {  // kind 0: region, 1: core
    if (z < 0 || z >= a.g.nz) return false;
    const int w = z >> 5, tile = cur.ty * a.tiles_x + cur.tx;
    if (w != dw[kind]) {
      dcur[kind] = w == dw[kind] + 1 ? dnext[kind] : tile_word(tile, w, kind);
      dw[kind] = w;
      dnext[kind] = tile_word(tile, w + 1, kind);
    }
    return (dcur[kind] >> (z & 31)) & 1u;
  };
  auto fail_align = [&]() {
    atomicCAS(a.err, 0, static_cast<int>(kErrLaunch));
    *abort_flag = 1;
  };
  auto pump = [&]() {
    while (!cur.done && !*abort_flag) {
      const int z0 = cur.z0, z1 = cur.z1;
      const int gx0 = cur.tx * C::CW, gy0 = cur.ty * C::CH;
      const int rx0 = gx0 - C::RX, ry0 = gy0 - R;
      int kind, z;  // 0: u^n plane z, 1: region tiles z, 2: core tiles z
      if (cur.k < 2 * R) {
        kind = 0;
        z = z0 - 2 * R + cur.k;
      } else {
        const int e = cur.k - 2 * R, t = z0 - R + e / 3, sub = e % 3;
        kind = sub;
        z = sub == 0 ? t + R : sub == 1 ? t : t - R;
        if (sub == 2 && t - R < z0) {  // no core tiles yet
          ++cur.k;
          continue;
        }
      }
      if (kind == 0) {
        const uint32_t slot = iu % C::NSU;
        if (iu >= C::NSU && !mbar_test_wait(&empty_u[slot], ((iu / C::NSU) - 1) & 1)) return;
        float *dst = uring + slot * (C::USLOT / 4);
        if ((smem_u32(dst) & 127u) || ((rx0 - C::RX) & 3)) {
          fail_align();
          return;
        }
        mbar_arrive_expect_tx(&full_u[slot], C::UPW * C::UPH * 4);
        tma_load_3d(dst, &tm_u, rx0 - C::RX, ry0 - R, z, &full_u[slot]);
        ++iu;
      } else if (kind == 1) {
        const uint32_t slot = itt % C::NST;
        if (itt >= C::NST && !mbar_test_wait(&empty_t[slot], ((itt / C::NST) - 1) & 1)) return;
        float *t = tring + slot * (3 * TT);
        if ((smem_u32(t) & 127u) || (rx0 & 3)) {
          fail_align();
          return;
        }
        const bool d = damped(z, 0);
        sflag_t[slot] = d ? 1 : 0;
        mbar_arrive_expect_tx(&full_t[slot], (d ? 3 : 2) * C::TSLOT);
        tma_load_3d(t + 0 * TT, &tm_um, rx0, ry0, z, &full_t[slot]);
        tma_load_3d(t + 1 * TT, &tm_b, rx0, ry0, z, &full_t[slot]);
        if (d) tma_load_3d(t + 2 * TT, &tm_s, rx0, ry0, z, &full_t[slot]);
        ++itt;
      } else {
        const uint32_t slot = ic % C::NSC;
        if (ic >= C::NSC && !mbar_test_wait(&empty_c[slot], ((ic / C::NSC) - 1) & 1)) return;
        float *t = cring + slot * (2 * CT);
        if ((smem_u32(t) & 127u) || (smem_u32(t + CT) & 127u) || (gx0 & 3)) {
          fail_align();
          return;
        }
        const bool d = damped(z, 1);
        sflag_c[slot] = d ? 1 : 0;
        mbar_arrive_expect_tx(&full_c[slot], (d ? 2 : 1) * C::CW * C::CH * 4);
        tma_load_3d(t, &tm_bc, gx0, gy0, z, &full_c[slot]);
        if (d) tma_load_3d(t + CT, &tm_sc, gx0, gy0, z, &full_c[slot]);
        ++ic;
      }
      // advance
      ++cur.k;
      if (cur.k >= 2 * R + 3 * (z1 - z0 + 2 * R)) {
        cur.item = first_item(++cur.it);
        cur.k = 0;
        cur.done = cur.item >= item_end;
        if (!cur.done) item_geom(cur.item, cur.tx, cur.ty, cur.z0, cur.z1);
        dw[0] = dw[1] = -2;  // new tile: the cached words no longer apply
      }
    }
  };
  // bounded wait on a full barrier; the producer lane issues loads while it waits
  // and probes without suspending (test_wait)
  auto wait_full = [&](uint64_t *bar, uint32_t parity) {
    if (producer) {
      pump();
      const uint64_t t0 = global_timer_ns();
      while (!mbar_test_wait(bar, parity)) {
        if (*abort_flag) return;
        pump();
        if (global_timer_ns() - t0 > kWaitLimitNs) {
          *abort_flag = 1;
          return;
        }
      }
    } else {
      mbar_wait_bounded(bar, parity, abort_flag);
    }
  };

  // ---------------- consumers ----------------
  const int ry = warp * NY;       // this lane's first region row
  const int rc = NX * lane;       // this lane's first region column
  const bool core_lane = rc >= C::RX && rc < W - C::RX;
  uint32_t ub = 0, tpos = 0, cpos = 0;
  auto release = [&](uint64_t *bar) {
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
  };
  auto cbar = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(C::WARPS * 32) : "memory"); };
  const long long drow = a.ntarget ? a.row + (a.row_base ? *a.row_base : 0) : 0;

  for (int it = 0, item = first_item(0); item < item_end; item = first_item(++it)) {
    int tx, ty, z0, z1;
    item_geom(item, tx, ty, z0, z1);
    if (z0 >= z1) continue;
    const int gx0 = tx * C::CW, gy0 = ty * C::CH;
    const int rx0 = gx0 - C::RX, ry0 = gy0 - R;
    const int gx = rx0 + rc;  // global column of this lane's first point
    const bool xin0 = gx >= 0 && gx < a.g.nx;
    const bool xin1 = gx + 1 >= 0 && gx + 1 < a.g.nx;
    // planes of this item's region that hold injection targets
    int inj_lo = 1 << 30, inj_hi = -(1 << 30);
    for (int i = 0; i < a.ntarget; ++i) {
      const int4 p = tgt[i];
      const int z = p.x, y = p.y, x = p.z;
      if (x >= rx0 && x < rx0 + W && y >= ry0 && y < ry0 + H && z >= z0 - R && z < z1 + R) {
        inj_lo = min(inj_lo, z);
        inj_hi = max(inj_hi, z);
      }
    }

    // q: u^n z queue (q[r][o + j] = plane t - R + j); v: u^{n+1} z queue (v[r][o + j] = plane t - 2R + j)
    V q[NY][2 * R + C::ZU];
    V v[NY][2 * R + C::ZU];
#pragma unroll
    for (int r = 0; r < NY; ++r)
#pragma unroll
      for (int j = 0; j < 2 * R + C::ZU; ++j) v[r][j] = make_float2(0.f, 0.f);
    // prologue: centres of planes z0 - 2R .. z0 - 1
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      const uint32_t pos = ub + j;
      const uint32_t slot = pos % C::NSU;
      wait_full(&full_u[slot], (pos / C::NSU) & 1);
      const float *Pl = uring + slot * (C::USLOT / 4);
#pragma unroll
      for (int r = 0; r < NY; ++r) q[r][j] = vld<V>(Pl + (ry + r + R) * C::UPW + rc + C::RX);
      if (j < R) release(&empty_u[slot]);  // below the region: centre only
    }

    auto plane = [&](int t, auto oc) {
      constexpr int o = decltype(oc)::value;
      // centre of u^n plane t + R into the queue
      {
        const uint32_t pos = ub + (t + 3 * R - z0);
        const uint32_t slot = pos % C::NSU;
        wait_full(&full_u[slot], (pos / C::NSU) & 1);
        const float *Pl = uring + slot * (C::USLOT / 4);
#pragma unroll
        for (int r = 0; r < NY; ++r) q[r][2 * R + o] = vld<V>(Pl + (ry + r + R) * C::UPW + rc + C::RX);
        if (t >= z1) release(&empty_u[slot]);  // above the region: centre only
      }
      // ---- step 1 on the region, plane t ----
      const uint32_t zslot = (ub + (t + 2 * R - z0)) % C::NSU;
      const float *Pl = uring + zslot * (C::USLOT / 4);
      V lap[NY];
      {
        V col[NY + 2 * R];
#pragma unroll
        for (int i = 0; i < NY + 2 * R; ++i) col[i] = vld<V>(Pl + (ry + i) * C::UPW + rc + C::RX);
#pragma unroll
        for (int r = 0; r < NY; ++r) {
          const float *pc = Pl + (ry + r + R) * C::UPW + rc + C::RX;
          V l = vmul(vsplat<V>(a.c.c0), q[r][o + R]);
          float2 w[C::RE + 1];
#pragma unroll
          for (int k = 0; k <= C::RE; ++k) w[k] = vld<float2>(pc - C::RE + 2 * k);
          auto win = [&](int i) -> float { return (i & 1) ? w[i >> 1].y : w[i >> 1].x; };
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            float2 xs;
            if ((j & 1) == 0) {
              xs = __fadd2_rn(w[(C::RE + j) >> 1], w[(C::RE - j) >> 1]);
            } else {
              xs = make_float2(win(C::RE + j) + win(C::RE - j), win(C::RE + 1 + j) + win(C::RE + 1 - j));
            }
            l = vfma(vsplat<V>(a.c.cx[j]), xs, l);
            l = vfma(vsplat<V>(a.c.cy[j]), vadd(col[R + r + j], col[R + r - j]), l);
            l = vfma(vsplat<V>(a.c.cz[j]), vadd(q[r][o + R + j], q[r][o + R - j]), l);
          }
          lap[r] = l;
        }
      }
      release(&empty_u[zslot]);
      const uint32_t tslot = tpos % C::NST;
      wait_full(&full_t[tslot], (tpos / C::NST) & 1);
      ++tpos;
      const float *T = tring + tslot * (3 * TT);
      const bool d1 = sflag_t[tslot] != 0;
      float *Vt = vring + (static_cast<uint32_t>(t + 2 * R) % C::NV) * TT;  // t + 2R >= 0
      V un1[NY];
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        const int ti = (ry + r) * W + rc;
        const V c = q[r][o + R];
        const V dd = vsub(c, vld<V>(T + ti));
        const V sv = d1 ? vld<V>(T + 2 * TT + ti) : vsplat<V>(0.f);
        const V bl = vmul(vld<V>(T + TT + ti), lap[r]);
        un1[r] = vadd(vfma(sv, dd, vadd(c, dd)), bl);
        *reinterpret_cast<V *>(Vt + ti) = un1[r];
      }
      release(&empty_t[tslot]);
      cbar();  // plane t of u^{n+1} complete
      if (t >= inj_lo && t <= inj_hi) {
        if (warp == 0) {
          for (int i = lane; i < a.ntarget; i += 32) {
            const int4 p = tgt[i];
            const int z = p.x, y = p.y, x = p.z;
            const long long tg = a.target[i];
            if (z == t && x >= rx0 && x < rx0 + W && y >= ry0 && y < ry0 + H) {
              const float *qd = a.data + drow * a.npts;
              float acc = 0.f;
              for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) acc = fmaf(a.w[k], qd[a.pid[k]], acc);
              const float inc = __fmul_rn(a.b[tg], acc);
              float *vp = Vt + (y - ry0) * W + (x - rx0);
              *vp = __fadd_rn(*vp, inc);
            }
          }
        }
        cbar();
#pragma unroll
        for (int r = 0; r < NY; ++r) un1[r] = vld<V>(Vt + (ry + r) * W + rc);
      }
#pragma unroll
      for (int r = 0; r < NY; ++r) v[r][2 * R + o] = un1[r];

      // ---- step 2 on the core, plane z2 = t - R ----
      const int z2 = t - R;
      if (z2 >= z0) {
        const uint32_t cslot = cpos % C::NSC;
        wait_full(&full_c[cslot], (cpos / C::NSC) & 1);
        ++cpos;
        const float *Cb = cring + cslot * (2 * CT);
        const bool d2 = sflag_c[cslot] != 0;
        const float *Vz = vring + (static_cast<uint32_t>(z2 + 2 * R) % C::NV) * TT;
        const bool any_row = ry + NY > R && ry < H - R;
        if (any_row && core_lane) {
          const long long po = static_cast<long long>(z2) * a.g.plane;
          const bool live = !*abort_flag;
          V col[NY + 2 * R];
#pragma unroll
          for (int i = 0; i < NY + 2 * R; ++i) {
            const int row = ry - R + i;
            col[i] = (row >= 0 && row < H) ? vld<V>(Vz + row * W + rc) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int r = 0; r < NY; ++r) {
            const int row = ry + r;
            if (row < R || row >= H - R) continue;
            const float *pc = Vz + row * W + rc;
            V l = vmul(vsplat<V>(a.c.c0), v[r][o + R]);
            float2 w[C::RE + 1];
#pragma unroll
            for (int k = 0; k <= C::RE; ++k) w[k] = vld<float2>(pc - C::RE + 2 * k);
            auto win = [&](int i) -> float { return (i & 1) ? w[i >> 1].y : w[i >> 1].x; };
#pragma unroll
            for (int j = 1; j <= R; ++j) {
              float2 xs;
              if ((j & 1) == 0) {
                xs = __fadd2_rn(w[(C::RE + j) >> 1], w[(C::RE - j) >> 1]);
              } else {
                xs = make_float2(win(C::RE + j) + win(C::RE - j), win(C::RE + 1 + j) + win(C::RE + 1 - j));
              }
              l = vfma(vsplat<V>(a.c.cx[j]), xs, l);
              l = vfma(vsplat<V>(a.c.cy[j]), vadd(col[R + r + j], col[R + r - j]), l);
              l = vfma(vsplat<V>(a.c.cz[j]), vadd(v[r][o + R + j], v[r][o + R - j]), l);
            }
            const int ci = (row - R) * C::CW + (rc - C::RX);
            const V c = v[r][o + R];
            const V dd = vsub(c, q[r][o]);
            const V sv = d2 ? vld<V>(Cb + CT + ci) : vsplat<V>(0.f);
            const V bl = vmul(vld<V>(Cb + ci), l);
            const V un2 = vadd(vfma(sv, dd, vadd(c, dd)), bl);
            const int gy = ry0 + row;
            if (gy < a.g.ny && live) {
              const long long off = po + static_cast<long long>(gy) * a.g.pitch + gx;
              if (xin1) {
                *reinterpret_cast<V *>(a.out1 + off) = c;
                *reinterpret_cast<V *>(a.out2 + off) = un2;
              } else if (xin0) {
                a.out1[off] = c.x;
                a.out2[off] = un2.x;
              }
            }
          }
        }
        release(&empty_c[cslot]);
      }
      cbar();  // step-2 reads of the u^{n+1} ring done before the next plane overwrites a slot
    };
    auto rotate = [&](auto nc) {
      constexpr int n = decltype(nc)::value;
#pragma unroll
      for (int r = 0; r < NY; ++r)
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) {
          q[r][j] = q[r][j + n];
          v[r][j] = v[r][j + n];
        }
    };
    int t = z0 - R;
    for (; t + C::ZU <= z1 + R; t += C::ZU) {
      plane(t, std::integral_constant<int, 0>{});
      if constexpr (C::ZU > 1) plane(t + 1, std::integral_constant<int, 1>{});
      rotate(std::integral_constant<int, C::ZU>{});
    }
    for (; t < z1 + R; ++t) {
      plane(t, std::integral_constant<int, 0>{});
      rotate(std::integral_constant<int, 1>{});
    }
    ub += static_cast<uint32_t>(z1 - z0 + 4 * R);
  }
  if (producer && *abort_flag) {
    // let issued copies land (bounded) before shared memory goes away
    const uint64_t t0 = global_timer_ns();
    for (uint32_t j = iu > C::NSU ? iu - C::NSU : 0; j < iu; ++j)
      while (!mbar_try_wait(&full_u[j % C::NSU], (j / C::NSU) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
      }
    for (uint32_t j = itt > C::NST ? itt - C::NST : 0; j < itt; ++j)
      while (!mbar_try_wait(&full_t[j % C::NST], (j / C::NST) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
      }
    for (uint32_t j = ic > C::NSC ? ic - C::NSC : 0; j < ic; ++j)
      while (!mbar_try_wait(&full_c[j % C::NSC], (j / C::NSC) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
      }
    atomicCAS(a.err, 0, static_cast<int>(kErrWaitFull));
  }
}

}  // namespace wp
