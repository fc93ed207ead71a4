/*
 * gf_inputs.c -- seeded synthetic link fields (the only code shared by the
 * CUDA path's tests/benchmarks and the oracle's).  It holds none of the
 * gauge-fixing arithmetic: it only produces the starting configurations.
 *
 * Every number is a pure function of (seed, link index, word), so any slab
 * of time-slices can be generated on its own and in parallel:
 *   word(seed, l, k) = SplitMix64 finaliser of
 *                      seed * 0x9E3779B97F4A7C15 + (8 l + k) * 0xD1B54A32D192ED03
 * (SplitMix64: Steele, Lea, Flood, OOPSLA 2014).
 *
 * Fields (StandardPattern t,x,y,z,mu,i,j,re/im; 18 doubles per link):
 *   smooth: U = exp(i eps H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0,1)
 *           (Gell-Mann lambda_a; Box-Muller normals), exponential by
 *           scaling and squaring of a degree-18 Taylor series;
 *   hot:    Haar-random SU(3) links (Gram-Schmidt of two complex Gaussian
 *           rows, third row conj(row0 x row1)).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef double complex cplx;

static uint64_t word(uint64_t seed, uint64_t l, uint64_t k) {
  uint64_t z = seed * 0x9E3779B97F4A7C15ull + (8 * l + k) * 0xD1B54A32D192ED03ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double unif(uint64_t w) { return ((double)(w >> 12) + 0.5) * 0x1p-52; }

/* eight N(0,1) numbers for link l */
static void normals8(uint64_t seed, uint64_t l, double h[8]) {
  for (int k = 0; k < 4; ++k) {
    double u1 = unif(word(seed, l, 2 * k)), u2 = unif(word(seed, l, 2 * k + 1));
    double r = sqrt(-2.0 * log(u1));
    h[2 * k] = r * cos(2.0 * M_PI * u2);
    h[2 * k + 1] = r * sin(2.0 * M_PI * u2);
  }
}

static void matmul3(const cplx a[3][3], const cplx b[3][3], cplx c[3][3]) {
  cplx t[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = 0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      t[i][j] = s;
    }
  memcpy(c, t, sizeof t);
}

static void smooth_link(uint64_t seed, uint64_t l, double eps, double* out) {
  double h[8];
  normals8(seed, l, h);
  const double r3 = 1.0 / sqrt(3.0);
  /* H = sum_a h_a lambda_a / 2 (Hermitian, traceless) */
  cplx H[3][3];
  H[0][0] = 0.5 * (h[2] + h[7] * r3);
  H[1][1] = 0.5 * (-h[2] + h[7] * r3);
  H[2][2] = 0.5 * (-2.0 * h[7] * r3);
  H[0][1] = 0.5 * (h[0] - I * h[1]);
  H[1][0] = conj(H[0][1]);
  H[0][2] = 0.5 * (h[3] - I * h[4]);
  H[2][0] = conj(H[0][2]);
  H[1][2] = 0.5 * (h[5] - I * h[6]);
  H[2][1] = conj(H[1][2]);
  /* A = i eps H, scaled by 2^-s so that its Frobenius norm is below 1/4 */
  double nrm = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) nrm += creal(H[i][j] * conj(H[i][j]));
  nrm = fabs(eps) * sqrt(nrm);
  int s = 0;
  while (nrm > 0.25) {
    nrm *= 0.5;
    ++s;
  }
  double scale = eps * ldexp(1.0, -s);
  cplx A[3][3], E[3][3], T[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i][j] = I * scale * H[i][j];
      E[i][j] = (i == j) ? 1.0 : 0.0;
      T[i][j] = E[i][j];
    }
  for (int n = 1; n <= 18; ++n) {
    matmul3(T, A, T);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T[i][j] /= (double)n;
        E[i][j] += T[i][j];
      }
  }
  for (int k = 0; k < s; ++k) matmul3(E, E, E);
  memcpy(out, E, sizeof E);
}

static void hot_link(uint64_t seed, uint64_t l, double* out) {
  double z[16];
  normals8(seed, 2 * l, z);
  normals8(seed, 2 * l + 1, z + 8);
  cplx a[3], b[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = z[2 * k] + I * z[2 * k + 1];
    b[k] = z[6 + 2 * k] + I * z[6 + 2 * k + 1];
  }
  double na = 0;
  for (int k = 0; k < 3; ++k) na += creal(a[k] * conj(a[k]));
  for (int k = 0; k < 3; ++k) a[k] /= sqrt(na);
  cplx ab = 0;
  for (int k = 0; k < 3; ++k) ab += conj(a[k]) * b[k];
  for (int k = 0; k < 3; ++k) b[k] -= ab * a[k];
  double nb = 0;
  for (int k = 0; k < 3; ++k) nb += creal(b[k] * conj(b[k]));
  for (int k = 0; k < 3; ++k) b[k] /= sqrt(nb);
  cplx U[3][3];
  for (int k = 0; k < 3; ++k) {
    U[0][k] = a[k];
    U[1][k] = b[k];
  }
  U[2][0] = conj(a[1] * b[2] - a[2] * b[1]);
  U[2][1] = conj(a[2] * b[0] - a[0] * b[2]);
  U[2][2] = conj(a[0] * b[1] - a[1] * b[0]);
  memcpy(out, U, sizeof U);
}

/* Fill links of time-slices [t0, t0 + nt) of a lattice dims = {Nt,Nx,Ny,Nz}.
 * kind: 0 = unit field, 1 = smooth exp(i eps H), 2 = hot (Haar).
 * out holds nt * Nx*Ny*Nz * 4 links of 18 doubles. */
void gfin_links(const int dims[4], int t0, int nt, int kind, double eps,
                uint64_t seed, double* out) {
  long V3 = (long)dims[1] * dims[2] * dims[3];
  long first = (long)t0 * V3 * 4, count = (long)nt * V3 * 4;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < count; ++q) {
    double* o = out + 18 * q;
    uint64_t l = (uint64_t)(first + q);
    if (kind == 1) {
      smooth_link(seed, l, eps, o);
    } else if (kind == 2) {
      hot_link(seed, l, o);
    } else {
      memset(o, 0, 18 * sizeof(double));
      o[0] = o[8] = o[16] = 1.0;
    }
  }
}
