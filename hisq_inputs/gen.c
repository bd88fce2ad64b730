/*
 * Seeded synthetic inputs for the HISQ even/odd operator and its solvers.
 *
 * This module only draws inputs: gauge links and source vectors. It holds none of
 * the operator's arithmetic (no staggered phases, no boundary signs, no hopping
 * terms): both the CPU oracle and the CUDA library receive its output as plain
 * arrays and fold phases and boundary conditions themselves.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from its published definition:
 * ten rounds of two 32x32->64-bit multiplies with the Weyl key schedule. It is
 * counter based, so any link of any lattice can be regenerated on its own from
 * (seed, site, direction, kind, draw), which lets a test rebuild the few links a
 * sampled output site needs.
 *
 * Gaussians: Box-Muller on pairs of uniforms in the open interval (0,1).
 *
 * Link recipe (the synthetic stand-in for thermalised HotQCD ensembles):
 *   thin   U_mu(x) = exp(i eps H),  H = sum_a h_a lambda_a / 2,  h_a ~ N(0,1)
 *          (lambda_a the eight Gell-Mann matrices), exp in FP64 by scaling and
 *          squaring of a Taylor series;
 *   fat    F_mu(x) = U_mu(x) + noise * G,  G_ij complex Gaussian, Re, Im ~ N(0, 1/2);
 *   long   L_mu(x) = -(1/24) U_mu(x) U_mu(x+mu) U_mu(x+2mu)  (periodic wrap).
 * Source vectors: complex Gaussian entries with Re, Im ~ N(0, 1/2).
 *
 * Layouts (host, complex128 interleaved re,im):
 *   links   [t][z][y][x][mu][row][col], x fastest, mu = 0..3 = x,y,z,t
 *   vectors [cb][color] over the sites of one parity, cb = lexicographic index / 2
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox4x32-10 */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void hin_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(PHILOX_M0, c0, &hi0, &lo0);
    mulhilo32(PHILOX_M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream kinds: each kind of draw owns its own counter space. */
enum { KIND_THIN = 1, KIND_FAT_NOISE = 2, KIND_SOURCE = 3, KIND_GAUGE_XFORM = 4, KIND_UNIFORM = 5 };

static double u32_to_open01(uint32_t v) { return ((double)v + 0.5) * (1.0 / 4294967296.0); }

/* Four standard normals from one Philox block: counter (site lo, site hi, tag, block). */
static void normals4(uint64_t seed, uint64_t site, uint32_t tag, uint32_t block, double g[4]) {
  uint32_t ctr[4] = {(uint32_t)site, (uint32_t)(site >> 32), tag, block};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  hin_philox4x32_10(ctr, key, r);
  for (int k = 0; k < 2; ++k) {
    double u1 = u32_to_open01(r[2 * k]), u2 = u32_to_open01(r[2 * k + 1]);
    double rad = sqrt(-2.0 * log(u1));
    g[2 * k] = rad * cos(2.0 * M_PI * u2);
    g[2 * k + 1] = rad * sin(2.0 * M_PI * u2);
  }
}

/* n normals for (site, tag), drawn block by block. */
static void normals(uint64_t seed, uint64_t site, uint32_t tag, int n, double* g) {
  double tmp[4];
  for (int b = 0; 4 * b < n; ++b) {
    normals4(seed, site, tag, (uint32_t)b, tmp);
    for (int k = 0; k < 4 && 4 * b + k < n; ++k) g[4 * b + k] = tmp[k];
  }
}

/* ---------------------------------------------------------------- 3x3 complex helpers */
typedef struct { double re, im; } cpx;

static void mat_mul(const cpx* a, const cpx* b, cpx* c) {
  cpx t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double re = 0, im = 0;
      for (int k = 0; k < 3; ++k) {
        re += a[3 * i + k].re * b[3 * k + j].re - a[3 * i + k].im * b[3 * k + j].im;
        im += a[3 * i + k].re * b[3 * k + j].im + a[3 * i + k].im * b[3 * k + j].re;
      }
      t[3 * i + j].re = re;
      t[3 * i + j].im = im;
    }
  memcpy(c, t, sizeof t);
}

/* Hermitian traceless H = sum_a h_a lambda_a / 2 (Gell-Mann basis). */
static void hermitian_from_coeffs(const double h[8], cpx* H) {
  const double s3 = 1.0 / sqrt(3.0);
  for (int k = 0; k < 9; ++k) H[k].re = H[k].im = 0.0;
  /* lambda_1, lambda_2: (0,1) block */
  H[1].re += h[0]; H[3].re += h[0];
  H[1].im += -h[1]; H[3].im += h[1];
  /* lambda_3 */
  H[0].re += h[2]; H[4].re += -h[2];
  /* lambda_4, lambda_5: (0,2) block */
  H[2].re += h[3]; H[6].re += h[3];
  H[2].im += -h[4]; H[6].im += h[4];
  /* lambda_6, lambda_7: (1,2) block */
  H[5].re += h[5]; H[7].re += h[5];
  H[5].im += -h[6]; H[7].im += h[6];
  /* lambda_8 */
  H[0].re += h[7] * s3; H[4].re += h[7] * s3; H[8].re += -2.0 * h[7] * s3;
  for (int k = 0; k < 9; ++k) { H[k].re *= 0.5; H[k].im *= 0.5; }
}

/* U = exp(i a H) for Hermitian H: scaling and squaring with a degree-18 Taylor series. */
static void expi_hermitian(const cpx* H, double a, cpx* U) {
  cpx Q[9];
  double norm = 0.0;
  for (int k = 0; k < 9; ++k) {
    Q[k].re = -a * H[k].im;  /* i a H */
    Q[k].im = a * H[k].re;
    norm += Q[k].re * Q[k].re + Q[k].im * Q[k].im;
  }
  norm = sqrt(norm);
  int s = 0;
  while (norm > 0.25) { norm *= 0.5; ++s; }
  double scale = ldexp(1.0, -s);
  for (int k = 0; k < 9; ++k) { Q[k].re *= scale; Q[k].im *= scale; }
  /* Horner: U = I + Q(I + Q/2 (I + Q/3 (...))) */
  cpx acc[9];
  for (int k = 0; k < 9; ++k) acc[k].re = acc[k].im = 0.0;
  for (int k = 0; k < 3; ++k) acc[4 * k].re = 1.0;
  for (int n = 18; n >= 1; --n) {
    cpx t[9];
    mat_mul(Q, acc, t);
    for (int k = 0; k < 9; ++k) {
      acc[k].re = t[k].re / n;
      acc[k].im = t[k].im / n;
    }
    for (int k = 0; k < 3; ++k) acc[4 * k].re += 1.0;
  }
  for (int i = 0; i < s; ++i) mat_mul(acc, acc, acc);
  memcpy(U, acc, sizeof acc);
}

/* ---------------------------------------------------------------- lattice indexing */
static int64_t lex(const int L[4], int x, int y, int z, int t) {
  return (int64_t)x + (int64_t)L[0] * ((int64_t)y + (int64_t)L[1] * ((int64_t)z + (int64_t)L[2] * (int64_t)t));
}

static void thin_link(uint64_t seed, double eps, const int L[4], int64_t site, int mu, cpx* U) {
  double h[8];
  cpx H[9];
  normals(seed, (uint64_t)site, (uint32_t)(KIND_THIN << 8 | mu), 8, h);
  hermitian_from_coeffs(h, H);
  expi_hermitian(H, eps, U);
  (void)L;
}

/*
 * Fat and long links for the sites with t in [t0, t0 + nt): out arrays hold
 * nt * Lz*Ly*Lx * 4 * 9 complex numbers each, in the link layout above, starting at t = t0.
 * Either output may be NULL. Returns 0, or -1 on bad arguments.
 */
int hin_gen_links(const int L[4], uint64_t seed, double eps, double noise, int t0, int nt, double* fat,
                  double* lng) {
  for (int m = 0; m < 4; ++m)
    if (L[m] < 1) return -1;
  if (t0 < 0 || nt < 0 || t0 + nt > L[3]) return -1;
  const int64_t slab = (int64_t)L[0] * L[1] * L[2];
  const int64_t n = slab * nt;
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; ++s) {
    int x = (int)(s % L[0]);
    int y = (int)((s / L[0]) % L[1]);
    int z = (int)((s / ((int64_t)L[0] * L[1])) % L[2]);
    int t = t0 + (int)(s / slab);
    int64_t site = lex(L, x, y, z, t);
    for (int mu = 0; mu < 4; ++mu) {
      cpx U[9];
      thin_link(seed, eps, L, site, mu, U);
      if (fat) {
        double g[18];
        normals(seed, (uint64_t)site, (uint32_t)(KIND_FAT_NOISE << 8 | mu), 18, g);
        double* f = fat + ((s * 4 + mu) * 9) * 2;
        for (int k = 0; k < 9; ++k) {
          f[2 * k] = U[k].re + noise * g[2 * k] * M_SQRT1_2;
          f[2 * k + 1] = U[k].im + noise * g[2 * k + 1] * M_SQRT1_2;
        }
      }
      if (lng) {
        int c[4] = {x, y, z, t};
        cpx U1[9], U2[9], P[9];
        c[mu] = (c[mu] + 1) % L[mu];
        thin_link(seed, eps, L, lex(L, c[0], c[1], c[2], c[3]), mu, U1);
        c[mu] = (c[mu] + 1) % L[mu];
        thin_link(seed, eps, L, lex(L, c[0], c[1], c[2], c[3]), mu, U2);
        mat_mul(U, U1, P);
        mat_mul(P, U2, P);
        double* l = lng + ((s * 4 + mu) * 9) * 2;
        for (int k = 0; k < 9; ++k) {
          l[2 * k] = -P[k].re / 24.0;
          l[2 * k + 1] = -P[k].im / 24.0;
        }
      }
    }
  }
  return 0;
}

/* Thin links only (all sites), for tests of the generator itself. */
int hin_gen_thin(const int L[4], uint64_t seed, double eps, double* thin) {
  const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < V; ++s)
    for (int mu = 0; mu < 4; ++mu) {
      cpx U[9];
      thin_link(seed, eps, L, s, mu, U);
      memcpy(thin + (s * 4 + mu) * 18, U, sizeof U);
    }
  return 0;
}

/* The Hermitian generator H of one thin link (for tests: exp(i eps H) == U). */
void hin_thin_generator(const int L[4], uint64_t seed, int64_t site, int mu, double* H_out) {
  double h[8];
  cpx H[9];
  normals(seed, (uint64_t)site, (uint32_t)(KIND_THIN << 8 | mu), 8, h);
  hermitian_from_coeffs(h, H);
  memcpy(H_out, H, sizeof H);
  (void)L;
}

/*
 * nvec complex Gaussian vectors of n_sites * 3 entries each (one parity), written
 * back to back; vector v uses counter stream (seed, v).
 */
int hin_gen_source(uint64_t seed, int64_t n_sites, int nvec, double* out) {
  if (n_sites < 0 || nvec < 0) return -1;
  for (int v = 0; v < nvec; ++v) {
    double* o = out + (int64_t)v * n_sites * 6;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n_sites; ++s) {
      double g[6];
      normals(seed, (uint64_t)s, (uint32_t)(KIND_SOURCE << 8 | (v & 0xff)) | ((uint32_t)(v >> 8) << 16), 6, g);
      for (int k = 0; k < 6; ++k) o[s * 6 + k] = g[k] * M_SQRT1_2;
    }
  }
  return 0;
}

/* A random SU(3) matrix per site, exp(i a H), for gauge-transformation tests. */
int hin_gen_gauge_xform(const int L[4], uint64_t seed, double a, double* omega) {
  const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < V; ++s) {
    double h[8];
    cpx H[9], U[9];
    normals(seed, (uint64_t)s, (uint32_t)(KIND_GAUGE_XFORM << 8), 8, h);
    hermitian_from_coeffs(h, H);
    expi_hermitian(H, a, U);
    memcpy(omega + s * 18, U, sizeof U);
  }
  return 0;
}

/* n uniforms in (0,1) from stream (seed, index) -- for per-lattice parameters of batches. */
void hin_uniforms(uint64_t seed, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)(KIND_UNIFORM << 8), 0};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    hin_philox4x32_10(ctr, key, r);
    out[i] = u32_to_open01(r[0]);
  }
}
