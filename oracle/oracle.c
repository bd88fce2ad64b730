/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, FP64 CPU restatement of the HISQ staggered operator on an
 * even/odd-split lattice and of the Krylov solvers it is used in. Only the tests,
 * the package's smoke check and the CPU-baseline leg of the benchmark may load it;
 * the CUDA library never calls it, and the two share no code (no headers, no
 * helpers, no tables).
 *
 * What the method computes (the paper names the operator, the CG variants and
 * RHMC but writes none of them out, so the textbook definitions are used):
 *   - the HISQ Dslash, the stencil whose cost dominates the CG that in turn takes
 *     about 60% of RHMC time (Sec. 3);
 *   - CG on M^dag M with multi-RHS, multi-shift and mixed-precision variants (Sec. 2,
 *     list of modules; Sec. 3);
 *   - HISQ fermions in RHMC (Sec. 1, Sec. 2).
 *
 * Conventions (readings of a paper that is silent on them):
 *   lattice   extents L[0..3] = Lx, Ly, Lz, Lt, all even;
 *             idx = x + Lx (y + Ly (z + Lz t)); parity = (x+y+z+t) mod 2, even = 0;
 *             cb = idx / 2 numbers the sites of one parity; periodic index wrap.
 *   phases    eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z).
 *   boundary  antiperiodic in t: F_t(x) *= -1 at t = Lt-1, L_t(x) *= -1 at t >= Lt-3,
 *             so every hop across the t boundary carries exactly one -1.
 *   operator  (D chi)(x) = sum_mu [ F_mu(x) chi(x+mu) - F_mu(x-mu)^dag chi(x-mu)
 *                                 + L_mu(x) chi(x+3mu) - L_mu(x-3mu)^dag chi(x-3mu) ]
 *             with phases and boundary signs folded into F and L, the Naik
 *             coefficient inside L, and no factor 1/2, so that
 *             M = 2m + D and M^dag M restricted to even sites is A = 4m^2 - D_eo D_oe.
 *             D_eo maps odd-site vectors to even sites, D_oe even to odd.
 *   layouts   links [idx][mu][row][col] complex; vectors [cb][color] complex.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ORACLE_APPLY_PHASES = 1, ORACLE_ANTIPERIODIC_T = 2 };

/* ------------------------------------------------------------------ indexing */

static int64_t volume(const int L[4]) { return (int64_t)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int L[4], int64_t idx, int c[4]) {
  c[0] = (int)(idx % L[0]);
  idx /= L[0];
  c[1] = (int)(idx % L[1]);
  idx /= L[1];
  c[2] = (int)(idx % L[2]);
  c[3] = (int)(idx / L[2]);
}

static int64_t index_of(const int L[4], const int c[4]) {
  int w[4];
  for (int m = 0; m < 4; ++m) w[m] = ((c[m] % L[m]) + L[m]) % L[m];
  return (int64_t)w[0] + (int64_t)L[0] * ((int64_t)w[1] + (int64_t)L[1] * ((int64_t)w[2] + (int64_t)L[2] * w[3]));
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* Lexicographic index of the site of parity p numbered cb. */
static int64_t site_of_cb(const int L[4], int p, int64_t cb) {
  int c[4];
  int64_t idx = 2 * cb;
  coords_of(L, idx, c);
  if (parity_of(c) != p) idx += 1;
  return idx;
}

/* The neighbour of site c at offset k along direction mu. */
static int64_t shifted(const int L[4], const int c[4], int mu, int k) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  d[mu] += k;
  return index_of(L, d);
}

/* ------------------------------------------------------------------ 3x3 algebra */

static const cplx* link_at(const double* links, int64_t idx, int mu) {
  return (const cplx*)links + (idx * 4 + mu) * 9;
}

/* out += s * U v */
static void add_mat_vec(cplx* out, const cplx* U, const cplx* v, double s) {
  for (int i = 0; i < 3; ++i) {
    cplx a = 0;
    for (int j = 0; j < 3; ++j) a += U[3 * i + j] * v[j];
    out[i] += s * a;
  }
}

/* out += s * U^dag v */
static void add_dag_mat_vec(cplx* out, const cplx* U, const cplx* v, double s) {
  for (int i = 0; i < 3; ++i) {
    cplx a = 0;
    for (int j = 0; j < 3; ++j) a += conj(U[3 * j + i]) * v[j];
    out[i] += s * a;
  }
}

/* ------------------------------------------------------------------ link folding */

/*
 * Multiply the staggered phases eta_mu(x) and the antiperiodic-t sign into the fat
 * and long links (either may be NULL). in and out may alias.
 */
void oracle_fold_links(const int L[4], unsigned flags, const double* fat_in, const double* long_in,
                       double* fat_out, double* long_out) {
  const int64_t V = volume(L);
  for (int64_t idx = 0; idx < V; ++idx) {
    int c[4];
    coords_of(L, idx, c);
    for (int mu = 0; mu < 4; ++mu) {
      double eta = 1.0;
      if (flags & ORACLE_APPLY_PHASES) {
        int sum = 0;
        for (int nu = 0; nu < mu; ++nu) sum += c[nu];
        eta = (sum & 1) ? -1.0 : 1.0;
      }
      double sf = eta, sl = eta;
      if ((flags & ORACLE_ANTIPERIODIC_T) && mu == 3) {
        if (c[3] == L[3] - 1) sf = -sf;
        if (c[3] >= L[3] - 3) sl = -sl;
      }
      for (int k = 0; k < 9; ++k) {
        int64_t o = (idx * 4 + mu) * 9 + k;
        if (fat_in) ((cplx*)fat_out)[o] = sf * ((const cplx*)fat_in)[o];
        if (long_in) ((cplx*)long_out)[o] = sl * ((const cplx*)long_in)[o];
      }
    }
  }
}

/* ------------------------------------------------------------------ the operator */

/*
 * (D chi)(x) at one site x, accumulating all 16 terms: on small extents two hops can
 * land on the same neighbour (x+3mu == x-mu when L_mu = 4) and both terms count.
 * `chi_at(idx)` returns the colour vector at lexicographic site idx.
 */
typedef const cplx* (*vec_lookup)(const void* ctx, int64_t idx);

static void dslash_site(const int L[4], const double* fat, const double* lng, int64_t idx, vec_lookup chi_at,
                        const void* ctx, cplx out[3]) {
  int c[4];
  coords_of(L, idx, c);
  out[0] = out[1] = out[2] = 0;
  for (int mu = 0; mu < 4; ++mu) {
    int64_t fwd1 = shifted(L, c, mu, +1), bwd1 = shifted(L, c, mu, -1);
    int64_t fwd3 = shifted(L, c, mu, +3), bwd3 = shifted(L, c, mu, -3);
    if (fat) {
      add_mat_vec(out, link_at(fat, idx, mu), chi_at(ctx, fwd1), +1.0);
      add_dag_mat_vec(out, link_at(fat, bwd1, mu), chi_at(ctx, bwd1), -1.0);
    }
    if (lng) {
      add_mat_vec(out, link_at(lng, idx, mu), chi_at(ctx, fwd3), +1.0);
      add_dag_mat_vec(out, link_at(lng, bwd3, mu), chi_at(ctx, bwd3), -1.0);
    }
  }
}

typedef struct {
  const cplx* v;
} full_ctx;

static const cplx* full_lookup(const void* ctx, int64_t idx) { return ((const full_ctx*)ctx)->v + idx * 3; }

typedef struct {
  const cplx* v;
  int parity;
  const int* L;
} half_ctx;

/* Half-lattice vectors hold only sites of one parity; every hop of D lands on the
 * opposite parity, so the lookup never sees the other one. */
static const cplx* half_lookup(const void* ctx, int64_t idx) {
  const half_ctx* h = (const half_ctx*)ctx;
  return h->v + (idx >> 1) * 3;
}

/*
 * D on the full lattice: out[idx][c] = (D in)(idx). Links are folded. fat or long
 * may be NULL to drop that part.
 */
void oracle_dslash_full(const int L[4], const double* fat, const double* lng, const double* in, double* out) {
  const int64_t V = volume(L);
  full_ctx ctx = {(const cplx*)in};
#pragma omp parallel for schedule(static)
  for (int64_t idx = 0; idx < V; ++idx) dslash_site(L, fat, lng, idx, full_lookup, &ctx, (cplx*)out + idx * 3);
}

/*
 * The even/odd halves: out_parity 0 gives out = D_eo in (in on odd sites),
 * out_parity 1 gives out = D_oe in (in on even sites). Vectors [cb][3] complex.
 */
void oracle_dslash(const int L[4], const double* fat, const double* lng, int out_parity, const double* in,
                   double* out) {
  const int64_t half = volume(L) / 2;
  half_ctx ctx = {(const cplx*)in, 1 - out_parity, L};
#pragma omp parallel for schedule(static)
  for (int64_t cb = 0; cb < half; ++cb) {
    int64_t idx = site_of_cb(L, out_parity, cb);
    dslash_site(L, fat, lng, idx, half_lookup, &ctx, (cplx*)out + cb * 3);
  }
}

/* The same operator evaluated only at the listed output sites (cb numbers of parity
 * out_parity); out holds n * 3 complex. For sampled checks on large lattices. */
void oracle_dslash_sites(const int L[4], const double* fat, const double* lng, int out_parity, const double* in,
                         int64_t n, const int64_t* cb_list, double* out) {
  half_ctx ctx = {(const cplx*)in, 1 - out_parity, L};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t idx = site_of_cb(L, out_parity, cb_list[i]);
    dslash_site(L, fat, lng, idx, half_lookup, &ctx, (cplx*)out + i * 3);
  }
}

/* ------------------------------------------------------------------ A = M^dag M on even sites */

static int64_t n_half(const int L[4]) { return volume(L) / 2 * 3; } /* complex entries */

/* out = (4 m^2 + sigma) in - D_eo D_oe in, all on even sites. */
void oracle_apply_A(const int L[4], const double* fat, const double* lng, double mass, double sigma,
                    const double* in, double* out) {
  const int64_t n = n_half(L);
  cplx* tmp = malloc(sizeof(cplx) * n);
  cplx* dd = malloc(sizeof(cplx) * n);
  oracle_dslash(L, fat, lng, 1, in, (double*)tmp);
  oracle_dslash(L, fat, lng, 0, (const double*)tmp, (double*)dd);
  const cplx* x = (const cplx*)in;
  cplx* y = (cplx*)out;
  for (int64_t i = 0; i < n; ++i) y[i] = (4.0 * mass * mass + sigma) * x[i] - dd[i];
  free(tmp);
  free(dd);
}

static double re_dot(const cplx* a, const cplx* b, int64_t n) {
  double s = 0;
  for (int64_t i = 0; i < n; ++i) s += creal(conj(a[i]) * b[i]);
  return s;
}

/* ||b - (A + sigma) x|| / ||b|| */
double oracle_true_residual(const int L[4], const double* fat, const double* lng, double mass, double sigma,
                            const double* b, const double* x) {
  const int64_t n = n_half(L);
  cplx* Ax = malloc(sizeof(cplx) * n);
  oracle_apply_A(L, fat, lng, mass, sigma, x, (double*)Ax);
  double num = 0, den = 0;
  for (int64_t i = 0; i < n; ++i) {
    cplx r = ((const cplx*)b)[i] - Ax[i];
    num += creal(r * conj(r));
    den += creal(((const cplx*)b)[i] * conj(((const cplx*)b)[i]));
  }
  free(Ax);
  return den > 0 ? sqrt(num / den) : sqrt(num);
}

/* ------------------------------------------------------------------ CG (Hestenes-Stiefel) */

/*
 * Textbook CG on (A + sigma) x = b. x holds the initial guess on entry (zero for the
 * usual start) and the solution on exit. Stops when the iterated residual satisfies
 * ||r|| <= tol ||b||. Returns the iteration count, or -1 if maxiter was reached.
 */
int oracle_cg(const int L[4], const double* fat, const double* lng, double mass, double sigma, const double* b,
              double* x_io, double tol, int maxiter) {
  const int64_t n = n_half(L);
  cplx* x = (cplx*)x_io;
  cplx* r = malloc(sizeof(cplx) * n);
  cplx* p = malloc(sizeof(cplx) * n);
  cplx* Ap = malloc(sizeof(cplx) * n);
  oracle_apply_A(L, fat, lng, mass, sigma, x_io, (double*)Ap);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = ((const cplx*)b)[i] - Ap[i];
    p[i] = r[i];
  }
  const double bb = re_dot((const cplx*)b, (const cplx*)b, n);
  double rr = re_dot(r, r, n);
  int it = 0;
  while (rr > tol * tol * bb && it < maxiter) {
    oracle_apply_A(L, fat, lng, mass, sigma, (const double*)p, (double*)Ap);
    double alpha = rr / re_dot(p, Ap, n);
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    double rr_new = re_dot(r, r, n);
    double beta = rr_new / rr;
    rr = rr_new;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  free(r);
  free(p);
  free(Ap);
  return rr > tol * tol * bb ? -1 : it;
}

/* ------------------------------------------------------------------ multi-shift CG */

/*
 * Multi-shift CG for (A + sigma_k) x_k = b, k = 0..ns-1, from one Krylov space
 * (Jegerlehner, hep-lat/9612014; the shifted residuals stay collinear with the
 * base residual, r_k = zeta_k r). The base system is the one with the smallest
 * shift. x (ns vectors back to back) starts from zero. Shift k is frozen once
 * |zeta_k| ||r|| <= tol[k] ||b||. iters_out[k] receives the iteration at which shift
 * k converged (-1 if it did not within maxiter). Returns the base iteration count.
 */
int oracle_multishift_cg(const int L[4], const double* fat, const double* lng, double mass, int ns,
                         const double* sigma, const double* b, double* x_out, const double* tol, int maxiter,
                         int* iters_out) {
  const int64_t n = n_half(L);
  int base = 0;
  for (int k = 1; k < ns; ++k)
    if (sigma[k] < sigma[base]) base = k;
  const double s0 = sigma[base];

  cplx* r = malloc(sizeof(cplx) * n);
  cplx* Ap = malloc(sizeof(cplx) * n);
  cplx* p = malloc(sizeof(cplx) * n * ns);
  cplx* x = (cplx*)x_out;
  double* zeta = malloc(sizeof(double) * ns);      /* zeta_k at step i   */
  double* zeta_old = malloc(sizeof(double) * ns);  /* zeta_k at step i-1 */
  int* active = malloc(sizeof(int) * ns);

  for (int64_t i = 0; i < n; ++i) r[i] = ((const cplx*)b)[i];
  for (int k = 0; k < ns; ++k) {
    for (int64_t i = 0; i < n; ++i) {
      p[k * n + i] = r[i];
      x[k * n + i] = 0;
    }
    zeta[k] = zeta_old[k] = 1.0;
    active[k] = 1;
    iters_out[k] = -1;
  }
  const double bb = re_dot(r, r, n);
  double rr = bb;
  double alpha_old = 1.0, beta_old = 0.0;
  int it = 0;
  for (; it < maxiter; ++it) {
    int any = 0;
    for (int k = 0; k < ns; ++k) {
      if (active[k] && fabs(zeta[k]) * sqrt(rr) <= tol[k] * sqrt(bb)) {
        active[k] = 0;
        iters_out[k] = it;
      }
      any |= active[k];
    }
    if (!any) break;
    /* base system (A + s0) */
    oracle_apply_A(L, fat, lng, mass, s0, (const double*)(p + base * n), (double*)Ap);
    const double alpha = rr / re_dot(p + base * n, Ap, n);
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * Ap[i];
    const double rr_new = re_dot(r, r, n);
    const double beta = rr_new / rr;
    for (int k = 0; k < ns; ++k) {
      if (!active[k]) continue;
      double zeta_new, alpha_k, beta_k;
      if (k == base) {
        zeta_new = 1.0;
        alpha_k = alpha;
        beta_k = beta;
      } else {
        const double dk = sigma[k] - s0;
        zeta_new = zeta[k] * zeta_old[k] * alpha_old /
                   (alpha * beta_old * (zeta_old[k] - zeta[k]) + zeta_old[k] * alpha_old * (1.0 + dk * alpha));
        alpha_k = alpha * zeta_new / zeta[k];
        beta_k = beta * (zeta_new / zeta[k]) * (zeta_new / zeta[k]);
      }
      cplx* pk = p + k * n;
      cplx* xk = x + k * n;
      for (int64_t i = 0; i < n; ++i) {
        xk[i] += alpha_k * pk[i];
        pk[i] = zeta_new * r[i] + beta_k * pk[i];
      }
      zeta_old[k] = zeta[k];
      zeta[k] = zeta_new;
    }
    alpha_old = alpha;
    beta_old = beta;
    rr = rr_new;
  }
  for (int k = 0; k < ns; ++k)
    if (active[k] && fabs(zeta[k]) * sqrt(rr) <= tol[k] * sqrt(bb)) iters_out[k] = it;
  free(r);
  free(Ap);
  free(p);
  free(zeta);
  free(zeta_old);
  free(active);
  return it;
}
