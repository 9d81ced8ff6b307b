// Device helpers for the sm_103a kernels: mbarrier and TMA (cp.async.bulk.tensor)
// wrappers in inline PTX, bounded waits that report through an error flag, and
// the argument structs shared by the stencil, injection and interpolation
// kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wp {

// Device error codes written to the context's error word (first error wins).
enum DeviceError : int {
  kErrNone = 0,
  kErrWaitFull = 1,   // a wait on a ring barrier gave up (its limit ran out)
  kErrLaunch = 2,     // a kernel was launched with an unsupported shape
  kErrBounds = 4,     // debug builds: an index outside its array, or a nonzero pitch padding value
};

// Debug builds (-DWP_DEBUG_BOUNDS): WP_IN_BOUNDS(cond, err) records kErrBounds in
// the error word and is false when cond fails, so that the access it guards is
// skipped; release builds compile it to `true`.
#ifdef WP_DEBUG_BOUNDS
#define WP_IN_BOUNDS(cond, err) ((cond) ? true : (atomicCAS((err), 0, static_cast<int>(::wp::kErrBounds)), false))
#else
#define WP_IN_BOUNDS(cond, err) true
#endif

// Default limit of a wait, in nanoseconds of %globaltimer (kernels take theirs
// from an argument; a context may set another one).  Letting copies that were
// already issued land before a CTA exits always uses this limit.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while the kernel before it on the stream still runs:
// grid_dependency_wait() returns once that kernel has completed and its memory
// operations are visible, so nothing that kernel writes or reads may be touched
// before it.  grid_dependents_launch() lets the next such kernel start launching.
// Both are no-ops for kernels launched the ordinary way.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of phase `parity` of `bar` (try_wait may suspend the thread
// for a while when the phase is not complete; test_wait returns at once).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar`; false (and *abort set) once limit_ns has
// passed, or when another thread of the block has already aborted.  The fast path
// is a single try_wait; the limit is read only when that fails (limit_ns = 0: give
// up at once).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  if (limit_ns == 0) {
    *abort_flag = 1;
    return false;
  }
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_timer_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}

// As mbar_wait_bounded, but with limit_ns = 0 the look does not block (a try_wait
// may suspend until the phase completes): a phase not complete at once gives up.
__device__ __forceinline__ bool mbar_wait_first(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                                uint64_t limit_ns) {
  if (limit_ns == 0 && !mbar_test_wait(bar, parity)) {
    *abort_flag = 1;
    return false;
  }
  return mbar_wait_bounded(bar, parity, abort_flag, limit_ns);
}

// 3D tiled TMA load of a box at element coordinates (x, y, z) into shared memory,
// completing `bytes` on `bar`.  x * 4 bytes must be a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Laplacian coefficients of one space order on one grid: c0 = a_0 sum_a h_a^-2,
// c[a][j] = a_j / h_a^2 (a = 0: z, 1: y, 2: x).
struct LapCoef {
  float c0;
  float cz[9];
  float cy[9];
  float cx[9];
  // the same coefficients as packed pairs (c, c), operands of FP32x2 arithmetic
  float2 p0;
  float2 pz[9];
  float2 py[9];
  float2 px[9];
};

// Geometry of a pitched field: element (z, y, x) at z*plane + y*pitch + x.
struct FieldGeom {
  int nx, ny, nz;
  int pitch;        // elements per row (multiple of 32)
  long long plane;  // elements per z-plane (ny * pitch)
};

}  // namespace wp
