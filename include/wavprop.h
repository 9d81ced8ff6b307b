/*
 * wavprop.h -- C ABI of the GB300 (sm_103a) propagator for the damped isotropic
 * acoustic wave equation
 *
 *      m u_tt - Lap u + eta u_t = q,      m = 1 / c^2            (Eq. acoustic, Eq. fdWE-abc)
 *
 * discretised with a space-order-k central Laplacian (Eq. fdSpace), the
 * second-order leapfrog in time (Eq. fdTime, Eq. eulerfwd) and a central
 * difference for the damping term, i.e. per time step
 *
 *      (m + eta dt/2) u^{n+1} = (2m + dt^2 Lap) u^n - (m - eta dt/2) u^{n-1} + dt^2 P_s^T q^n,
 *      d^n = P_r u^{n+1},      u^{-1} = u^0 = 0,
 *
 * with zero values outside the grid (Sec. 3.2), multilinear injection P_s^T and
 * interpolation P_r inside the containing cell (Sec. 2.2.4), the adjoint as
 * backward substitution with the transposed system (Sec. 2.2.2, Eq. Adj) and the
 * adjoint-state gradient of J(m) = 1/2 ||F(m) q - d_obs||^2 (Eq. AS, Eq. Grad).
 *
 * Conventions shared by every call
 *   - Fields are C-ordered arrays of float: (nz, ny, nx) in 3D, (nz, nx) in 2D,
 *     x fastest.  The grid is the computational grid (physical interior plus any
 *     damping layer).
 *   - spacing[], origin[] and point coordinates use the same axis order as
 *     shape[] (z, y, x) / (z, x); origin is the coordinate of index 0.
 *   - A point must lie in [origin, origin + (n-1) h] on every axis (points within
 *     1e-9 cells outside are clamped onto the grid).  Its cell is
 *     i = min(floor((c - o)/h), n - 2), computed in double precision.
 *   - Time series are row-major [nt][npoints] float arrays; sample n of a
 *     receiver trace is u^{n+1} (time (n+1) dt).
 *   - The injected source is weighted by dt^2 / (m + eta dt/2) at each corner
 *     (equal to the paper's dt^2/m where eta = 0).
 *
 * Ownership: the caller owns every array passed in or out; the library reads or
 * writes them during the call and keeps no reference.  A context owns its device
 * memory, stream and kernels' scratch; a wp_state owns its snapshots.
 *
 * Errors: every int-returning call returns WP_OK (0) or a negative status and
 * sets a thread-local message readable with wp_last_error().  No call throws.
 * Calls are synchronous: they return after their device work has finished.
 * A context may be used by one thread at a time; distinct contexts may run
 * concurrently from different threads (each has its own stream).
 */
#ifndef WAVPROP_H
#define WAVPROP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WP_OK 0
#define WP_EINVAL (-1)      /* bad shape/order/count/coordinate, m <= 0 or eta < 0 */
#define WP_ECFL (-2)        /* dt above the stability limit of the scheme */
#define WP_ENOMEM (-3)      /* request exceeds the context's HBM budget or device memory */
#define WP_ENONFINITE (-4)  /* NaN or Inf in an input array */
#define WP_ECUDA (-5)       /* a CUDA runtime or driver call failed */
#define WP_ETIMEOUT (-6)    /* device work did not finish within the context's deadline */
#define WP_EDEVICE (-7)     /* a kernel reported an internal error (e.g. a wait that timed out) */

/* hbm_budget_bytes value meaning "90 % of the device memory free at creation" */
#define WP_BUDGET_AUTO ((size_t)-1)

typedef struct wp_ctx wp_ctx;
typedef struct wp_state wp_state;

typedef struct {
  int ndim;            /* 2 or 3 */
  int64_t shape[3];    /* (nz, ny, nx) or (nz, nx); every used entry >= 2 */
  double spacing[3];   /* > 0, same axis order */
  double origin[3];    /* coordinate of index 0, same axis order */
  int space_order;     /* k, even, 2..16 */
  double dt;           /* time step, 0 < dt <= wp_cfl_dt(...) */
  int nt;              /* number of time steps, >= 0 */
} wp_grid;

/* Create a context on CUDA device `device` that may hold at most
 * hbm_budget_bytes of device memory (WP_BUDGET_AUTO: 90 % of free memory).
 * *out receives the context; release it with wp_destroy. */
int wp_create(wp_ctx **out, int device, size_t hbm_budget_bytes);
void wp_destroy(wp_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *wp_last_error(void);

/* Seconds after which a call gives up waiting for its device work and returns
 * WP_ETIMEOUT (default 600).  The context must not be reused after a timeout
 * (every later call on it returns WP_ETIMEOUT).  The work it had queued keeps
 * running and may still write the call's output arrays: synchronise the device
 * (cudaDeviceSynchronize) before reading, reusing or freeing them, and before
 * wp_destroy. */
int wp_set_timeout(wp_ctx *ctx, double seconds);

/* Weights a_0..a_{k/2} of the order-k central second derivative
 * (Eq. fdSpace, centre counted once): closed form
 * a_j = 2 (-1)^{j+1} (p!)^2 / (j^2 (p-j)! (p+j)!), p = k/2, a_0 = -2 sum a_j.
 * alpha must hold k/2 + 1 doubles. */
int wp_fd_weights(int space_order, double *alpha);

/* Largest stable dt of the scheme for velocity vmax (von Neumann bound of the
 * undamped leapfrog: dt_max = 2 / (vmax sqrt(sum_a A_k / h_a^2)), A_k = |a_0| + 2 sum |a_j|). */
int wp_cfl_dt(const wp_grid *grid, double vmax, double *dt_max);

/* Device bytes a call would hold for this grid: mode 0 forward/adjoint,
 * 1 gradient with the given snapshot interval, 2 checkpointed gradient with
 * snap_interval stored states, 3 gradient by boundary reconstruction (an upper
 * bound; snap_interval unused). */
int wp_estimate_bytes(const wp_grid *grid, int nsrc, int nrec, int mode, int snap_interval,
                      size_t *bytes);

/* ---- forward, adjoint, gradient: HOST arrays ---------------------------- */

/* Forward modelling (Sec. 3.2): rec_out[nt][nrec] = P_r u^{n+1}.
 * m, eta: fields (host, float); wavelet[nt][nsrc]; src_coords[nsrc][ndim] and
 * rec_coords[nrec][ndim] (double).  nsrc, nrec >= 0. */
int wp_forward(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
               const float *wavelet, int nsrc, const double *src_coords, int nrec,
               const double *rec_coords, float *rec_out);

/* Adjoint modelling (Sec. 3.3, Eq. Adj): the exact transpose of the forward map
 * wavelet -> rec_out.  rec_data[nt][nrec] is injected at the receivers backward in
 * time; src_out[nt][nsrc] samples the adjoint field at the sources. */
int wp_adjoint(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
               const float *rec_data, int nrec, const double *rec_coords, int nsrc,
               const double *src_coords, float *src_out);

/* Gradient of J(m) = 1/2 ||F(m) q - d_obs||^2 (Eq. AS, Eq. Grad) given the
 * residual F(m) q - d_obs [nt][nrec]:
 *   grad = -dt^-2 sum_{j=1}^{nt} u^j (w^j - 2 w^{j+1} + w^{j+2}),
 * w the adjoint field driven by the residual.  The forward field is kept as
 * snapshot pairs every snap_interval steps in device memory and recomputed
 * between them (Sec. 3.3, checkpointing); snap_interval = 1 keeps the whole
 * history instead (each level stored once, nt fields, written by the forward
 * step itself) and recomputes nothing; snap_interval = 0 chooses: the whole
 * history if it fits the context's remaining budget, else the smallest interval
 * that fits (WP_ENOMEM if none does).  The gradient is the same whichever
 * interval is used.  grad_out has the field's shape. */
int wp_gradient(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                const float *wavelet, int nsrc, const double *src_coords,
                const float *residual, int nrec, const double *rec_coords, int snap_interval,
                float *grad_out);

/* Gradient as wp_gradient, with binomial checkpointing instead of periodic
 * snapshots (Sec. 3.3: partial time history plus recomputation, as Revolve):
 * `checkpoints` stored states (2 fields each) and the optimal reversal schedule
 * for that number minimise the recomputed forward steps.  Memory: about
 * 2 checkpoints + 7 fields instead of 2 nt/snap_interval + snap_interval + 5.
 * The result is identical to wp_gradient's. */
int wp_gradient_checkpointed(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                             const float *wavelet, int nsrc, const double *src_coords,
                             const float *residual, int nrec, const double *rec_coords,
                             int checkpoints, float *grad_out);

/* Gradient by boundary-wavefield reconstruction (Sec. 3.3): the forward pass
 * keeps only the values on a ring of width space_order/2 around the box Z where
 * eta = 0 (for every time level), and the backward pass rebuilds u^j on Z by
 * running the time-symmetric undamped update backward, beside the adjoint.
 * Memory: O(surface x nt) instead of snapshots; cost: the same passes as
 * wp_gradient.  grad_out receives the gradient on Z and 0 in the damping layer
 * (where the forward field is not reversible); on Z it equals wp_gradient's up
 * to FP32 rounding of the reversal.  WP_EINVAL if eta vanishes nowhere or the
 * set where it vanishes is not an axis-aligned box. */
int wp_gradient_reconstruct(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                            const float *wavelet, int nsrc, const double *src_coords,
                            const float *residual, int nrec, const double *rec_coords,
                            float *grad_out);

/* The reversal schedule used by wp_gradient_checkpointed: 4 ints per op
 * (kind, a, b, slot) with kind 0 = advance from the state a held in `slot` to
 * state b, 1 = store the current state a in `slot`, 2 = adjoint step j = a;
 * state k is (u^{k-1}, u^k) and slot 0 holds state 0.  *nops receives the
 * number of ops (ops may be NULL to query it), *forward_steps the number of
 * forward steps the schedule recomputes. */
int wp_checkpoint_schedule(int nt, int checkpoints, int *ops, int max_ops, int *nops,
                           long long *forward_steps);

/* ---- DEVICE-array variants ------------------------------------------------
 * Same contracts; m, eta, wavelet, rec/src data and outputs are device pointers
 * (contiguous, float), coordinates stay on the host.  Work is ordered after
 * everything already queued on `stream` (a cudaStream_t, NULL = legacy default
 * stream), and later work on `stream` is ordered after it.  Every device-array
 * argument (and those of the CFD, axpy and model-update _dev calls) must be
 * device or managed memory of the context's device: a host pointer or memory of
 * another GPU is refused with WP_EINVAL before anything is launched. */
int wp_forward_dev(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                   const float *wavelet, int nsrc, const double *src_coords, int nrec,
                   const double *rec_coords, float *rec_out, void *stream);
int wp_adjoint_dev(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                   const float *rec_data, int nrec, const double *rec_coords, int nsrc,
                   const double *src_coords, float *src_out, void *stream);
int wp_gradient_dev(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                    const float *wavelet, int nsrc, const double *src_coords,
                    const float *residual, int nrec, const double *rec_coords,
                    int snap_interval, float *grad_out, void *stream);
int wp_gradient_reconstruct_dev(wp_ctx *ctx, const wp_grid *grid, const float *m,
                                const float *eta, const float *wavelet, int nsrc,
                                const double *src_coords, const float *residual, int nrec,
                                const double *rec_coords, float *grad_out, void *stream);
int wp_gradient_checkpointed_dev(wp_ctx *ctx, const wp_grid *grid, const float *m,
                                 const float *eta, const float *wavelet, int nsrc,
                                 const double *src_coords, const float *residual, int nrec,
                                 const double *rec_coords, int checkpoints, float *grad_out,
                                 void *stream);

/* nsteps source-free updates of (u_prev, u) = (u^{n-1}, u^n) in place (device
 * fields, contiguous): on return they hold (u^{n+nsteps-1}, u^{n+nsteps}). */
int wp_propagate_dev(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                     float *u_prev, float *u, int nsteps, void *stream);

/* FWI objective and gradient of one shot (Eq. AS, Eq. Grad; the per-source
 * function of Sec. 3.4): forward with snapshots, residual r = d - d_obs,
 * *misfit = 1/2 ||r||^2 (summed in double, deterministic order), and
 * grad_out = J^T r.  d_obs[nt][nrec]; the _dev variant takes device arrays. */
int wp_fwi_gradient(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                    const float *wavelet, int nsrc, const double *src_coords, const float *d_obs,
                    int nrec, const double *rec_coords, int snap_interval, float *grad_out,
                    double *misfit);
int wp_fwi_gradient_dev(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                        const float *wavelet, int nsrc, const double *src_coords,
                        const float *d_obs, int nrec, const double *rec_coords, int snap_interval,
                        float *grad_out, double *misfit, void *stream);

/* Multi-shot FWI (Sec. 3.4): the gradient of the objective summed over source
 * experiments, and the fixed-step gradient update with bounds.
 *   wp_axpy_dev:         y[i] += alpha x[i] for i < n (device arrays);
 *   wp_update_model_dev: m[i] = min(max(m[i] - step grad[i], m_min), m_max),
 *                        with 0 < m_min <= m_max (squared-slowness bounds). */
int wp_axpy_dev(wp_ctx *ctx, long long n, float alpha, const float *x, float *y, void *stream);

/* Misfit of one shot (Eq. AS): r_out[i] = d[i] - d_obs[i] for i < n and
 * *misfit = 1/2 sum r_i^2, summed in double in a fixed order (the same kernel and
 * order as wp_fwi_gradient's misfit, so the two agree bitwise).  Device arrays;
 * WP_ENONFINITE if the sum is not finite. */
int wp_misfit_dev(wp_ctx *ctx, long long n, const float *d, const float *d_obs, float *r_out,
                  double *misfit, void *stream);
int wp_update_model_dev(wp_ctx *ctx, long long n, float step, const float *grad, float *m,
                        float m_min, float m_max, void *stream);

/* Release cached (not live) device blocks of the context until it holds at most
 * keep_bytes.  Waits for the context's stream first. */
int wp_trim(wp_ctx *ctx, size_t keep_bytes);

/* Change the context's device-memory budget (later allocations release cached
 * blocks first and fail with WP_ENOMEM beyond it). */
int wp_set_budget(wp_ctx *ctx, size_t hbm_budget_bytes);

/* ---- split forward / backward (autograd, serving) ---------------------------
 * wp_forward_save runs the forward (device arrays) and keeps its snapshots
 * resident in *state; wp_backward(state, residual, grad) then returns
 * J^T residual = dJ/dm for J = 1/2 ||d - d_obs||^2 with residual = d - d_obs
 * (or any upstream gradient dL/dd).  A state may be back-propagated more than
 * once; wp_state_free releases its memory.  The state borrows ctx (its memory
 * counts against ctx's budget).  If ctx is destroyed first, wp_destroy releases
 * the state's device memory and detaches it: wp_backward on it then returns
 * WP_EINVAL, and wp_state_free only frees the handle. */
int wp_forward_save(wp_ctx *ctx, const wp_grid *grid, const float *m, const float *eta,
                    const float *wavelet, int nsrc, const double *src_coords, int nrec,
                    const double *rec_coords, int snap_interval, float *rec_out, void *stream,
                    wp_state **state);
int wp_backward(wp_state *state, const float *residual, float *grad_out, void *stream);
void wp_state_free(wp_state *state);

/* Limit, in seconds, of every wait inside the context's stencil kernels (a
 * kernel waits for its own TMA copies and ring slots; default 2 s, at most 60).
 * A wait that runs out makes the kernel skip its remaining stores and the call
 * return WP_EDEVICE; the context stays usable (set a larger limit and call
 * again).  0 makes every stencil kernel give up at the start of its first work
 * item (a wait on a barrier that nothing completes), and any later wait that is
 * not complete at once: it exists to exercise that error path deterministically. */
int wp_set_wait_limit(wp_ctx *ctx, double seconds);

/* ---- The computational-fluid-dynamics examples of Sec. 5 (2D, FP32) --------
 * Fields are (ny, nx) arrays in C order (x fastest).  Each call advances the
 * interior points 1 <= i <= nx-2, 1 <= j <= ny-2 and keeps the edge values of the
 * initial field (Dirichlet data; the paper's examples set them to 1, 1 and 0).
 * Inputs are read, outputs written by the call; errors as for the propagator
 * (WP_EINVAL, WP_ENONFINITE for NaN/Inf inputs, WP_ENOMEM, WP_ECUDA).
 *
 * Convection (Eq. convection_fd): nt steps of
 *   u_{i,j} <- u_{i,j} - c dt/dx (u_{i,j} - u_{i-1,j}) - c dt/dy (u_{i,j} - u_{i,j-1});
 * WP_ECFL unless c >= 0 and c dt/dx + c dt/dy <= 1 (the upwind scheme's limit). */
int wp_convection_2d(wp_ctx *ctx, int nx, int ny, double dx, double dy, double dt, double c, int nt,
                     const float *u0, float *u_out);
/* Burgers' equation (Eq. Burger): nt forward-Euler steps of the coupled system with
 * upwind (backward) first derivatives and central second derivatives, viscosity nu. */
int wp_burgers_2d(wp_ctx *ctx, int nx, int ny, double dx, double dy, double dt, double nu, int nt,
                  const float *u0, const float *v0, float *u_out, float *v_out);
/* Poisson (Eq. Poisson_fd): nit Jacobi iterations for Lap p = b from p0. */
int wp_poisson_2d(wp_ctx *ctx, int nx, int ny, double dx, double dy, int nit, const float *p0,
                  const float *b, float *p_out);
/* Device-array variants (stream-ordered like the other *_dev calls). */
int wp_convection_2d_dev(wp_ctx *ctx, int nx, int ny, double dx, double dy, double dt, double c,
                         int nt, const float *u0, float *u_out, void *stream);
int wp_burgers_2d_dev(wp_ctx *ctx, int nx, int ny, double dx, double dy, double dt, double nu,
                      int nt, const float *u0, const float *v0, float *u_out, float *v_out,
                      void *stream);
int wp_poisson_2d_dev(wp_ctx *ctx, int nx, int ny, double dx, double dy, int nit, const float *p0,
                      const float *b, float *p_out, void *stream);

/* Device bytes currently held by the context (including live states). */
size_t wp_bytes_in_use(const wp_ctx *ctx);

/* Number of kernels this context has launched (graph replays count every node). */
uint64_t wp_kernel_launches(const wp_ctx *ctx);

/* Profiling: with every = N > 0, every N-th stencil (K1) launch is bracketed by
 * CUDA events on the context's stream (0 turns it off); wp_profile_read returns
 * the summed device time (ms) of the bracketed launches and their number since
 * the last reset.  Sampling (N > 1) keeps the event nodes out of most steps. */
int wp_set_profiling(wp_ctx *ctx, int every);
int wp_profile_read(wp_ctx *ctx, double *stencil_ms, uint64_t *stencil_launches, int reset);

/* ---- forward modelling without any device allocation -----------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory: code that runs inside a host application which owns
 * every device byte through its own pool or arena and forbids cudaMalloc /
 * cudaFree from libraries, or that has budgeted its device memory up front.
 * It computes exactly what wp_forward_dev computes (same kernels, same
 * arguments, device pointers for m, eta, wavelet and rec_out, host coordinates)
 * but needs no wp_ctx and allocates nothing: its work space (coefficients, the
 * two wavefields, damping flags, source and receiver tables) is one fixed
 * device array of WP_NOALLOC_MAX_BYTES declared by the library, which every GPU
 * that loads the library holds until the process exits.
 *   - A problem whose work space would exceed WP_NOALLOC_MAX_BYTES is rejected
 *     with WP_ENOMEM before any device work (3D grids up to about 4 million
 *     points fit).
 *   - The first call on a device looks the array's device address up there
 *     (this may make CUDA load the library's device code on that device); make
 *     that first call before any stream capture.
 *   - Every call uses the same array, which keeps the previous call's contents
 *     (the call clears what must start at zero).  Calls that overlap on the GPU,
 *     from several streams or host threads, race on it and corrupt each other's
 *     results: serialise them.
 * Work runs on the current device, on `stream` (NULL = legacy default stream),
 * and the call returns after it has finished.  m, eta, wavelet and rec_out must
 * be device memory of the current device and `stream` must belong to it, else
 * WP_EINVAL (nothing launched).  After an error the call also waits for any
 * work it had already queued, so the array is idle when it returns. */
#define WP_NOALLOC_MAX_BYTES ((size_t)64 << 20)
int wp_forward_noalloc(const wp_grid *grid, const float *m, const float *eta,
                       const float *wavelet, int nsrc, const double *src_coords, int nrec,
                       const double *rec_coords, float *rec_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WAVPROP_H */
