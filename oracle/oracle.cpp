/*
 * FP64 CPU oracle for the damped isotropic acoustic propagator
 *
 *     m u_tt - Lap u + eta u_t = q                          (Eq. acoustic, Eq. fdWE-abc)
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline / reference legs may load and call this library; the GPU product
 * path never does, and this file shares no code, header or table with it.
 *
 * Everything is plain nested loops in double precision (or std::complex<double>
 * for the complex-step derivative check), written from the paper's definitions:
 *
 *   - space-order-k central second derivative (Eq. fdSpace), with the centre
 *     term counted once:  d2u/dx2 ~ h^-2 [a_0 u + sum_{j=1}^{k/2} a_j (u_{+j} + u_{-j})]
 *   - second-order time difference (Eq. fdTime) and a central first difference
 *     for the damping term, solved for the next time level (Eq. eulerfwd, the
 *     "solve(eqn, u.forward)" derivation of Sec. 2.2.2):
 *        (m + eta dt/2) u+ = dt^2 Lap u + m (2u - u-) + (eta dt/2) u- + dt^2 P_s^T q
 *   - zero Dirichlet values outside the grid (Sec. 3.2, "zero Dirichlet boundary")
 *   - multilinear injection / interpolation inside the containing cell (Sec. 2.2.4)
 *   - the adjoint as backward substitution with the transposed system (Sec. 2.2.2,
 *     Eq. Adj) and the adjoint-state gradient sum_t u v_tt (Eq. Grad).
 *
 * Readings where the paper is silent or garbled (all listed in the design notes):
 *   - Eq. fdSpace sums j = 0..k/2 of a_j (u_{+j} + u_{-j}); the j = 0 term is read
 *     as a_0 u (centre once).
 *   - the damping term uses a central difference in time.
 *   - the injected source is scaled by dt^2/(m + eta dt/2), i.e. the source enters
 *     the right-hand side before the division; equal to dt^2/m wherever eta = 0.
 *   - receiver sample n is taken from u^{n+1}, after injection of q^n.
 *   - coefficients a_j: the standard closed form
 *        a_j = 2 (-1)^{j+1} (p!)^2 / (j^2 (p-j)! (p+j)!),  p = k/2,  a_0 = -2 sum a_j.
 *
 * Layout: fields are C-ordered (nz, ny, nx), x fastest (2D: (nz, nx)).  Point
 * coordinates are given in the same axis order (z, y, x) / (z, x), in the same
 * physical units as spacing and origin; origin is the coordinate of index 0.
 */
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::complex<double> cplx;

struct Grid {
  int ndim;
  int64_t n[3];     // internal axes (z, y, x); 2D problems use ny = 1
  bool active[3];   // axes that carry a second derivative
  double h[3];
  double o[3];
  int k;            // space order
  int r;            // k / 2
  double dt;
  int nt;
};

// Closed-form central second-derivative weights (Eq. fdSpace), k even in [2, 16].
bool fd_weights(int k, double *alpha) {
  if (k < 2 || k > 16 || (k % 2) != 0) return false;
  const int p = k / 2;
  double sum = 0.0;
  for (int j = 1; j <= p; ++j) {
    // (p!)^2 / ((p-j)! (p+j)!) = prod_{i=1..j} (p - i + 1) / (p + i)
    double ratio = 1.0;
    for (int i = 1; i <= j; ++i) ratio *= double(p - i + 1) / double(p + i);
    const double sgn = (j % 2 == 1) ? 1.0 : -1.0;
    alpha[j] = 2.0 * sgn * ratio / double(j * j);
    sum += alpha[j];
  }
  alpha[0] = -2.0 * sum;
  return true;
}

// A padded field: r ghost cells on each side of every active axis.  Ghosts stay
// zero (Dirichlet) unless a test asks for odd reflection.
template <class T>
struct Field {
  int64_t n[3], pad[3], p[3], s[3];
  std::vector<T> a;
  explicit Field(const Grid &g) {
    for (int d = 0; d < 3; ++d) {
      n[d] = g.n[d];
      pad[d] = g.active[d] ? g.r : 0;
      p[d] = n[d] + 2 * pad[d];
    }
    s[2] = 1;
    s[1] = p[2];
    s[0] = p[1] * p[2];
    a.assign(size_t(p[0] * p[1] * p[2]), T(0));
  }
  int64_t idx(int64_t z, int64_t y, int64_t x) const {
    return (z + pad[0]) * s[0] + (y + pad[1]) * s[1] + (x + pad[2]);
  }
  T &at(int64_t z, int64_t y, int64_t x) { return a[size_t(idx(z, y, x))]; }
  const T &at(int64_t z, int64_t y, int64_t x) const { return a[size_t(idx(z, y, x))]; }
  void zero() { std::fill(a.begin(), a.end(), T(0)); }
};

// Odd reflection about the first and last node of every active axis (test-only
// boundary used by the exact standing-wave check; the method itself uses zeros).
template <class T>
void fill_odd_ghosts(Field<T> &f, const Grid &g) {
  for (int d = 0; d < 3; ++d) {
    if (!g.active[d]) continue;
    const int64_t nd = g.n[d];
    int64_t ext[3] = {g.n[0], g.n[1], g.n[2]};
    ext[d] = 1;  // walk every line along axis d
    for (int64_t a0 = 0; a0 < ext[0]; ++a0)
      for (int64_t a1 = 0; a1 < ext[1]; ++a1)
        for (int64_t a2 = 0; a2 < ext[2]; ++a2)
          for (int j = 1; j <= g.r; ++j) {
            int64_t src_lo[3] = {a0, a1, a2}, dst_lo[3] = {a0, a1, a2};
            int64_t src_hi[3] = {a0, a1, a2}, dst_hi[3] = {a0, a1, a2};
            src_lo[d] = j;
            dst_lo[d] = -j;
            src_hi[d] = nd - 1 - j;
            dst_hi[d] = nd - 1 + j;
            f.at(dst_lo[0], dst_lo[1], dst_lo[2]) = -f.at(src_lo[0], src_lo[1], src_lo[2]);
            f.at(dst_hi[0], dst_hi[1], dst_hi[2]) = -f.at(src_hi[0], src_hi[1], src_hi[2]);
          }
  }
}

// Discrete Laplacian at (z, y, x): sum over active axes of Eq. fdSpace.
template <class T>
inline T laplacian(const Field<T> &u, const Grid &g, const double *alpha, int64_t z, int64_t y,
                   int64_t x) {
  const int64_t c = u.idx(z, y, x);
  const T uc = u.a[size_t(c)];
  T lap = T(0);
  for (int d = 0; d < 3; ++d) {
    if (!g.active[d]) continue;
    T s = alpha[0] * uc;
    for (int j = 1; j <= g.r; ++j)
      s += alpha[j] * (u.a[size_t(c + j * u.s[d])] + u.a[size_t(c - j * u.s[d])]);
    lap += s / (g.h[d] * g.h[d]);
  }
  return lap;
}

// One leapfrog step: solve the discretised damped wave equation for u+ (no source).
template <class T>
void step(const Grid &g, const double *alpha, const T *m, const double *eta, const Field<T> &uprev,
          const Field<T> &u, Field<T> &unext) {
  const double dt = g.dt;
  const double dt2 = dt * dt;
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        const int64_t i = (z * g.n[1] + y) * g.n[2] + x;
        const T lap = laplacian(u, g, alpha, z, y, x);
        const T mm = m[i];
        const double half_damp = eta[i] * dt / 2.0;
        const T un = u.at(z, y, x), um = uprev.at(z, y, x);
        unext.at(z, y, x) = (dt2 * lap + mm * (2.0 * un - um) + half_damp * um) / (mm + half_damp);
      }
}

// Multilinear weights of an off-grid point inside its containing cell.
// t_a = (c_a - o_a) / h_a (points within 1e-9 cells of the grid are clamped onto
// it), i_a = floor(t_a) clamped to n_a - 2 so the last node is reached with
// fractional part 1.  Returns false for a point outside the grid.
struct Stencil {
  int64_t idx[8];  // flat unpadded index of each corner
  int64_t zyx[8][3];
  double w[8];
  int ncorner;
};

bool interp_stencil(const Grid &g, const double *coord, Stencil &st) {
  int64_t base[3] = {0, 0, 0};
  double frac[3] = {0.0, 0.0, 0.0};
  int ci = 0;
  for (int d = 0; d < 3; ++d) {
    if (!g.active[d]) continue;
    double t = (coord[ci] - g.o[d]) / g.h[d];
    ++ci;
    // accept points up to 1e-9 cells outside (rounding of on-node coordinates)
    if (!(t >= -1e-9) || !(t <= double(g.n[d] - 1) + 1e-9)) return false;
    t = std::min(std::max(t, 0.0), double(g.n[d] - 1));
    int64_t i = int64_t(std::floor(t));
    if (i > g.n[d] - 2) i = g.n[d] - 2;
    if (i < 0) i = 0;
    base[d] = i;
    frac[d] = t - double(i);
  }
  st.ncorner = 0;
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const int cc[3] = {cz, cy, cx};
        bool skip = false;
        double w = 1.0;
        int64_t p[3];
        for (int d = 0; d < 3; ++d) {
          if (!g.active[d]) {
            if (cc[d] != 0) skip = true;
            p[d] = 0;
            continue;
          }
          p[d] = base[d] + cc[d];
          w *= cc[d] ? frac[d] : (1.0 - frac[d]);
        }
        if (skip) continue;
        Stencil &s = st;
        s.zyx[s.ncorner][0] = p[0];
        s.zyx[s.ncorner][1] = p[1];
        s.zyx[s.ncorner][2] = p[2];
        s.idx[s.ncorner] = (p[0] * g.n[1] + p[1]) * g.n[2] + p[2];
        s.w[s.ncorner] = w;
        ++s.ncorner;
      }
  return true;
}

bool make_grid(Grid &g, int ndim, const int64_t *shape, const double *spacing, const double *origin,
               int k, double dt, int nt) {
  if (ndim != 2 && ndim != 3) return false;
  if (k < 2 || k > 16 || k % 2) return false;
  g.ndim = ndim;
  g.k = k;
  g.r = k / 2;
  g.dt = dt;
  g.nt = nt;
  if (ndim == 3) {
    for (int d = 0; d < 3; ++d) {
      g.n[d] = shape[d];
      g.h[d] = spacing[d];
      g.o[d] = origin[d];
      g.active[d] = true;
    }
  } else {
    g.n[0] = shape[0]; g.h[0] = spacing[0]; g.o[0] = origin[0]; g.active[0] = true;
    g.n[1] = 1;        g.h[1] = 1.0;        g.o[1] = 0.0;       g.active[1] = false;
    g.n[2] = shape[1]; g.h[2] = spacing[1]; g.o[2] = origin[1]; g.active[2] = true;
  }
  for (int d = 0; d < 3; ++d)
    if (g.active[d] && g.n[d] < 2) return false;
  return true;
}

bool make_stencils(const Grid &g, int npts, const double *coords, std::vector<Stencil> &out) {
  out.resize(size_t(std::max(npts, 0)));
  for (int i = 0; i < npts; ++i)
    if (!interp_stencil(g, coords + size_t(i) * g.ndim, out[size_t(i)])) return false;
  return true;
}

// Add dt^2 / (m + eta dt/2) * w * value at each corner (the P^T term of the
// right-hand side, divided by the same factor as the rest of the update).
template <class T>
void inject(const Grid &g, Field<T> &u, const T *m, const double *eta,
            const std::vector<Stencil> &pts, const double *values) {
  const double dt2 = g.dt * g.dt;
  for (size_t s = 0; s < pts.size(); ++s)
    for (int c = 0; c < pts[s].ncorner; ++c) {
      const int64_t i = pts[s].idx[c];
      const T denom = m[i] + eta[i] * g.dt / 2.0;
      u.at(pts[s].zyx[c][0], pts[s].zyx[c][1], pts[s].zyx[c][2]) +=
          dt2 * pts[s].w[c] * values[s] / denom;
    }
}

template <class T>
void sample(const Field<T> &u, const std::vector<Stencil> &pts, T *out) {
  for (size_t i = 0; i < pts.size(); ++i) {
    T acc = T(0);
    for (int c = 0; c < pts[i].ncorner; ++c)
      acc += pts[i].w[c] * u.at(pts[i].zyx[c][0], pts[i].zyx[c][1], pts[i].zyx[c][2]);
    out[i] = acc;
  }
}

// Forward: u^{-1} = u^0 = 0; for n = 0..nt-1 solve for u^{n+1}, inject q^n,
// record d^n = P_r u^{n+1}.  Optionally return u^{nt} and u^{nt-1}.
template <class T>
int forward_impl(const Grid &g, const T *m, const double *eta, const double *wavelet, int nsrc,
                 const double *src, int nrec, const double *rec, T *rec_out, T *u_last,
                 T *u_prev_last) {
  double alpha[9];
  fd_weights(g.k, alpha);
  std::vector<Stencil> sp, rp;
  if (!make_stencils(g, nsrc, src, sp) || !make_stencils(g, nrec, rec, rp)) return -1;
  Field<T> a(g), b(g), c(g);
  Field<T> *uprev = &a, *u = &b, *unext = &c;
  for (int n = 0; n < g.nt; ++n) {
    step(g, alpha, m, eta, *uprev, *u, *unext);
    inject(g, *unext, m, eta, sp, wavelet + size_t(n) * nsrc);
    sample(*unext, rp, rec_out + size_t(n) * nrec);
    Field<T> *t = uprev;
    uprev = u;
    u = unext;
    unext = t;
  }
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        const int64_t i = (z * g.n[1] + y) * g.n[2] + x;
        if (u_last) u_last[i] = u->at(z, y, x);
        if (u_prev_last) u_prev_last[i] = uprev->at(z, y, x);
      }
  return 0;
}

// Adjoint (Eq. Adj): backward substitution with A^T.  w^{nt+1} = w^{nt+2} = 0;
// for j = nt..1 solve for w^j from w^{j+1}, w^{j+2}, inject the data d^{j-1} at
// the receivers, and sample q_hat^{j-1} = P_s w^j at the sources.
int adjoint_impl(const Grid &g, const double *m, const double *eta, const double *rec_data,
                 int nrec, const double *rec, int nsrc, const double *src, double *src_out) {
  double alpha[9];
  fd_weights(g.k, alpha);
  std::vector<Stencil> sp, rp;
  if (!make_stencils(g, nsrc, src, sp) || !make_stencils(g, nrec, rec, rp)) return -1;
  Field<double> a(g), b(g), c(g);
  Field<double> *w2 = &a, *w1 = &b, *w0 = &c;  // w^{j+2}, w^{j+1}, w^j
  for (int j = g.nt; j >= 1; --j) {
    step(g, alpha, m, eta, *w2, *w1, *w0);
    inject(g, *w0, m, eta, rp, rec_data + size_t(j - 1) * nrec);
    sample(*w0, sp, src_out + size_t(j - 1) * nsrc);
    Field<double> *t = w2;
    w2 = w1;
    w1 = w0;
    w0 = t;
  }
  return 0;
}

// Gradient of J(m) = 1/2 || F(m) q - d_obs ||^2 (Eq. AS) by the adjoint-state
// method (Eq. Grad):  g = -dt^-2 sum_{j=1}^{nt} u^j (w^j - 2 w^{j+1} + w^{j+2}),
// i.e. "grad = grad - u * v.dt2", where w is the adjoint field driven by the
// residual.  The forward field is kept as (u^{s-1}, u^s) pairs every `ckpt`
// steps and recomputed segment by segment (checkpointing, Sec. 3.3).
int gradient_impl(const Grid &g, const double *m, const double *eta, const double *wavelet,
                  int nsrc, const double *src, const double *residual, int nrec,
                  const double *rec, int ckpt, double *grad) {
  double alpha[9];
  fd_weights(g.k, alpha);
  std::vector<Stencil> sp, rp;
  if (!make_stencils(g, nsrc, src, sp) || !make_stencils(g, nrec, rec, rp)) return -1;
  if (ckpt < 1) ckpt = 1;
  const int nt = g.nt;
  const int nseg = (nt + ckpt - 1) / ckpt;
  // checkpoint s holds (u^{s*ckpt - 1}, u^{s*ckpt})
  std::vector<Field<double>> ck_prev, ck_cur;
  ck_prev.reserve(size_t(nseg));
  ck_cur.reserve(size_t(nseg));
  {
    Field<double> a(g), b(g), c(g);
    Field<double> *uprev = &a, *u = &b, *unext = &c;
    for (int n = 0; n < nt; ++n) {
      if (n % ckpt == 0) {
        ck_prev.push_back(*uprev);
        ck_cur.push_back(*u);
      }
      step(g, alpha, m, eta, *uprev, *u, *unext);
      inject(g, *unext, m, eta, sp, wavelet + size_t(n) * nsrc);
      Field<double> *t = uprev;
      uprev = u;
      u = unext;
      unext = t;
    }
  }
  const int64_t N = g.n[0] * g.n[1] * g.n[2];
  std::fill(grad, grad + N, 0.0);
  const double inv_dt2 = 1.0 / (g.dt * g.dt);
  Field<double> a(g), b(g), c(g);
  Field<double> *w2 = &a, *w1 = &b, *w0 = &c;  // w^{j+2}, w^{j+1}, w^j
  std::vector<Field<double>> seg;               // u^{s0+1} .. u^{s0+len}
  for (int s = nseg - 1; s >= 0; --s) {
    const int s0 = s * ckpt;
    const int len = std::min(ckpt, nt - s0);
    seg.clear();
    {
      Field<double> uprev = ck_prev[size_t(s)], u = ck_cur[size_t(s)], unext(g);
      for (int n = s0; n < s0 + len; ++n) {
        step(g, alpha, m, eta, uprev, u, unext);
        inject(g, unext, m, eta, sp, wavelet + size_t(n) * nsrc);
        seg.push_back(unext);
        uprev = u;
        u = unext;
      }
    }
    for (int j = s0 + len; j >= s0 + 1; --j) {
      step(g, alpha, m, eta, *w2, *w1, *w0);
      inject(g, *w0, m, eta, rp, residual + size_t(j - 1) * nrec);
      const Field<double> &uj = seg[size_t(j - s0 - 1)];
#pragma omp parallel for schedule(static)
      for (int64_t z = 0; z < g.n[0]; ++z)
        for (int64_t y = 0; y < g.n[1]; ++y)
          for (int64_t x = 0; x < g.n[2]; ++x) {
            const int64_t i = (z * g.n[1] + y) * g.n[2] + x;
            const double vtt = (w0->at(z, y, x) - 2.0 * w1->at(z, y, x) + w2->at(z, y, x)) * inv_dt2;
            grad[i] -= uj.at(z, y, x) * vtt;
          }
      Field<double> *t = w2;
      w2 = w1;
      w1 = w0;
      w0 = t;
    }
  }
  return 0;
}

}  // namespace

extern "C" {

typedef struct {
  int ndim;
  int64_t shape[3];
  double spacing[3];
  double origin[3];
  int space_order;
  double dt;
  int nt;
} or_grid;

static bool grid_from(const or_grid *gi, Grid &g) {
  return make_grid(g, gi->ndim, gi->shape, gi->spacing, gi->origin, gi->space_order, gi->dt, gi->nt);
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_fd_weights(int k, double *alpha) { return fd_weights(k, alpha) ? 0 : -1; }

// Largest stable dt of the undamped leapfrog scheme (von Neumann): the symbol of
// -Lap peaks at the Nyquist wavenumber, where it equals sum_a A_k / h_a^2 with
// A_k = |a_0| + 2 sum_j |a_j|; leapfrog needs v^2 dt^2 * that <= 4.
int or_cfl_dt(int ndim, const double *spacing, int k, double vmax, double *dt_max) {
  double alpha[9];
  if (!fd_weights(k, alpha) || (ndim != 2 && ndim != 3) || !(vmax > 0)) return -1;
  double A = std::fabs(alpha[0]);
  for (int j = 1; j <= k / 2; ++j) A += 2.0 * std::fabs(alpha[j]);
  double s = 0.0;
  for (int d = 0; d < ndim; ++d) s += A / (spacing[d] * spacing[d]);
  *dt_max = 2.0 / (vmax * std::sqrt(s));
  return 0;
}

// Corner indices (flat, unpadded) and weights of each point; 2^ndim per point.
int or_interp(const or_grid *gi, int npts, const double *coords, int64_t *idx, double *w) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  const int nc = 1 << g.ndim;
  for (int i = 0; i < npts; ++i) {
    Stencil st;
    if (!interp_stencil(g, coords + size_t(i) * g.ndim, st)) return -2;
    for (int c = 0; c < nc; ++c) {
      idx[size_t(i) * nc + c] = st.idx[c];
      w[size_t(i) * nc + c] = st.w[c];
    }
  }
  return 0;
}

int or_forward(const or_grid *gi, const double *m, const double *eta, const double *wavelet,
               int nsrc, const double *src, int nrec, const double *rec, double *rec_out,
               double *u_last, double *u_prev_last) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  return forward_impl<double>(g, m, eta, wavelet, nsrc, src, nrec, rec, rec_out, u_last,
                              u_prev_last);
}

// Same forward map with complex squared slowness (complex-step derivatives).
int or_forward_cplx(const or_grid *gi, const double *m_re, const double *m_im, const double *eta,
                    const double *wavelet, int nsrc, const double *src, int nrec, const double *rec,
                    double *rec_re, double *rec_im) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  const int64_t N = g.n[0] * g.n[1] * g.n[2];
  std::vector<cplx> m(static_cast<size_t>(N));
  for (int64_t i = 0; i < N; ++i) m[size_t(i)] = cplx(m_re[i], m_im[i]);
  std::vector<cplx> out(size_t(g.nt) * size_t(std::max(nrec, 0)));
  const int rc = forward_impl<cplx>(g, m.data(), eta, wavelet, nsrc, src, nrec, rec, out.data(),
                                    nullptr, nullptr);
  for (size_t i = 0; i < out.size(); ++i) {
    rec_re[i] = out[i].real();
    rec_im[i] = out[i].imag();
  }
  return rc;
}

int or_adjoint(const or_grid *gi, const double *m, const double *eta, const double *rec_data,
               int nrec, const double *rec, int nsrc, const double *src, double *src_out) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  return adjoint_impl(g, m, eta, rec_data, nrec, rec, nsrc, src, src_out);
}

int or_gradient(const or_grid *gi, const double *m, const double *eta, const double *wavelet,
                int nsrc, const double *src, const double *residual, int nrec, const double *rec,
                int ckpt, double *grad) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  return gradient_impl(g, m, eta, wavelet, nsrc, src, residual, nrec, rec, ckpt, grad);
}

// One step of the update from (u^{n-1}, u^n) without sources.  halo_mode 0 keeps
// zero values outside the grid (the method); 1 uses odd reflection about the
// first and last node of each axis (test-only, for the exact standing wave).
int or_step(const or_grid *gi, const double *m, const double *eta, const double *u_prev,
            const double *u, double *u_next, int halo_mode) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  double alpha[9];
  fd_weights(g.k, alpha);
  Field<double> fp(g), fu(g), fn(g);
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        const int64_t i = (z * g.n[1] + y) * g.n[2] + x;
        fp.at(z, y, x) = u_prev[i];
        fu.at(z, y, x) = u[i];
      }
  if (halo_mode == 1) {
    for (int d = 0; d < 3; ++d)
      if (g.active[d] && g.n[d] <= g.r) return -2;
    fill_odd_ghosts(fu, g);
  }
  step(g, alpha, m, eta, fp, fu, fn);
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) u_next[(z * g.n[1] + y) * g.n[2] + x] = fn.at(z, y, x);
  return 0;
}

// nsteps of the update with halo_mode as in or_step (no sources); (u_prev, u) in,
// (u^{n+nsteps-1}, u^{n+nsteps}) out, in place.
int or_run(const or_grid *gi, const double *m, const double *eta, double *u_prev, double *u,
           int nsteps, int halo_mode) {
  Grid g;
  if (!grid_from(gi, g)) return -1;
  double alpha[9];
  fd_weights(g.k, alpha);
  if (halo_mode == 1)
    for (int d = 0; d < 3; ++d)
      if (g.active[d] && g.n[d] <= g.r) return -2;
  Field<double> a(g), b(g), c(g);
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        const int64_t i = (z * g.n[1] + y) * g.n[2] + x;
        a.at(z, y, x) = u_prev[i];
        b.at(z, y, x) = u[i];
      }
  Field<double> *fp = &a, *fu = &b, *fn = &c;
  for (int n = 0; n < nsteps; ++n) {
    if (halo_mode == 1) fill_odd_ghosts(*fu, g);
    step(g, alpha, m, eta, *fp, *fu, *fn);
    Field<double> *t = fp;
    fp = fu;
    fu = fn;
    fn = t;
  }
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        const int64_t i = (z * g.n[1] + y) * g.n[2] + x;
        u_prev[i] = fp->at(z, y, x);
        u[i] = fu->at(z, y, x);
      }
  return 0;
}

}  // extern "C"
