/*
 * gf_oracle.c -- plain, slow FP64 CPU oracle for lattice gauge fixing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path; the two meet only in
 * the seeded synthetic inputs and in the published Philox4x32-10 definition
 * (Salmon et al., SC'11), which each side implements on its own.
 *
 * Everything follows Schroeck & Vogt, "Coulomb, Landau and Maximally Abelian
 * Gauge Fixing in Lattice QCD with Multi-GPUs" (arXiv:1212.5221):
 *   - gauge functionals and theta: Sec. 2.1 (Eqs. landau_functional,
 *     MAG_functional, the theta definitions of Secs. 2.1.1 and 2.1.2);
 *   - local relaxation: Sec. 2.2 (Eqs. landau_loc, Kx, localsolution), with
 *     the three Cabibbo-Marinari SU(2) subgroups;
 *   - MAG local maximum: Sec. 2.2.2 (Eqs. up, upMatrix);
 *   - overrelaxation / microcanonical / stochastic relaxation: Secs. 2.2.3-5;
 *   - simulated annealing with heatbath + 3 microcanonical steps: Sec. 2.3;
 *   - the checkerboard sweep: Sec. 2.4, Alg. 1;
 *   - unitarity measure: Sec. 4.5.
 * Readings of passages the paper leaves open are marked READING below.
 *
 * Links are full 3x3 complex matrices in FP64, stored in the natural order
 * ("StandardPattern", Sec. 4.2.1): t, x, y, z, mu, i, j, re/im -- 18 doubles
 * per link.  mu = 0 is the temporal direction.  Boundaries are periodic
 * (READING: the paper does not state them).  Sites of the active parity are
 * visited in lexicographic order; the order does not matter because sites of
 * one parity touch disjoint links (Sec. 2.2).
 *
 * Parity pinned by tests/test_oracle_pins.py; the SA heat-bath samplers and
 * Philox are pinned statistically and against an independent Philox
 * implementation.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;
typedef struct { cplx m[3][3]; } su3;
typedef struct { cplx m[2][2]; } su2;

enum { OR_LANDAU = 0, OR_COULOMB = 1, OR_MAG = 2 };
enum { OR_ALGO_RELAX = 0, OR_ALGO_OR = 1, OR_ALGO_MICRO = 2, OR_ALGO_SR = 3,
       OR_ALGO_SA = 4 };

/* Philox counter word 2 carries a stream tag, the subgroup and a draw index
 * (READING: the paper only says Philox is used; the counter layout is ours). */
#define TAG_SR 1u
#define TAG_SA 2u
#define TAG_HAAR 3u
#define KP_MAX_TRIALS 64

static const int SUBGROUP[3][2] = {{0, 1}, {0, 2}, {1, 2}};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the definition in Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two
 * 32x32->64 multiplications with the round multipliers, xor with the other
 * counter words and the key, and a Weyl increment of the key between rounds. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  memcpy(out, c, sizeof c);
}

/* Uniform in the open interval (0,1) from two 32-bit words: the top 52 bits
 * of hi:lo, plus one half, times 2^-52.  Every value is exact in IEEE double.
 * READING: the paper gives no mapping. */
double or_u01(uint32_t hi, uint32_t lo) {
  uint64_t bits = ((uint64_t)hi << 32) | lo;
  return ((double)(bits >> 12) + 0.5) * 0x1p-52;
}

/* One Philox call for (seed, site, sweep, tag/subgroup/draw, copy); returns
 * two uniforms. */
static void draw2(uint64_t seed, uint32_t site, uint32_t sweep, uint32_t tag,
                  uint32_t sub, uint32_t draw, uint32_t copy, double u[2]) {
  uint32_t ctr[4] = {site, sweep, (tag << 24) | (sub << 8) | draw, copy};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  u[0] = or_u01(r[0], r[1]);
  u[1] = or_u01(r[2], r[3]);
}

/* ------------------------------------------------------------------------ */
/* Matrix algebra (plain loops). */

static su3 su3_mul(const su3* a, const su3* b) {
  su3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = 0;
      for (int k = 0; k < 3; ++k) s += a->m[i][k] * b->m[k][j];
      c.m[i][j] = s;
    }
  return c;
}

static su3 su3_dag(const su3* a) {
  su3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.m[i][j] = conj(a->m[j][i]);
  return c;
}

static cplx su3_det(const su3* a) {
  const cplx(*m)[3] = a->m;
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
         m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
         m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* Cayley-Klein embedding of a quaternion (Sec. 2.2.2):
 *   [[g0 + i g3, g2 + i g1], [-g2 + i g1, g0 - i g3]]. */
static su2 su2_from_quaternion(const double g[4]) {
  su2 h;
  h.m[0][0] = g[0] + I * g[3];
  h.m[0][1] = g[2] + I * g[1];
  h.m[1][0] = -g[2] + I * g[1];
  h.m[1][1] = g[0] - I * g[3];
  return h;
}

static su2 su2_mul(const su2* a, const su2* b) {
  su2 c;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      c.m[i][j] = a->m[i][0] * b->m[0][j] + a->m[i][1] * b->m[1][j];
  return c;
}

/* The SU(3) matrix that acts as h on rows/columns (i, j) and as 1 on the
 * third index (Cabibbo-Marinari, Sec. 2.2.1). */
static su3 embed(const su2* h, int i, int j) {
  su3 g;
  memset(&g, 0, sizeof g);
  for (int k = 0; k < 3; ++k) g.m[k][k] = 1;
  g.m[i][i] = h->m[0][0];
  g.m[i][j] = h->m[0][1];
  g.m[j][i] = h->m[1][0];
  g.m[j][j] = h->m[1][1];
  return g;
}

/* ------------------------------------------------------------------------ */
/* Lattice indexing: dims = {Nt, Nx, Ny, Nz}; site index
 * s = ((t*Nx + x)*Ny + y)*Nz + z; direction mu moves coordinate mu. */

typedef struct {
  int n[4];
  long V;
} lattice;

static lattice make_lattice(const int dims[4]) {
  lattice L;
  L.V = 1;
  for (int d = 0; d < 4; ++d) {
    L.n[d] = dims[d];
    L.V *= dims[d];
  }
  return L;
}

static void coords(const lattice* L, long s, int c[4]) {
  for (int d = 3; d >= 0; --d) {
    c[d] = (int)(s % L->n[d]);
    s /= L->n[d];
  }
}

static long site_of(const lattice* L, const int c[4]) {
  long s = 0;
  for (int d = 0; d < 4; ++d) s = s * L->n[d] + c[d];
  return s;
}

static long neighbour(const lattice* L, long s, int mu, int step) {
  int c[4];
  coords(L, s, c);
  c[mu] = (c[mu] + step + L->n[mu]) % L->n[mu];
  return site_of(L, c);
}

static int parity_of(const lattice* L, long s) {
  int c[4];
  coords(L, s, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

static su3 get_link(const double* U, long s, int mu) {
  su3 u;
  memcpy(&u, U + ((size_t)s * 4 + mu) * 18, sizeof u);
  return u;
}

static void put_link(double* U, long s, int mu, const su3* u) {
  memcpy(U + ((size_t)s * 4 + mu) * 18, u, sizeof *u);
}

/* ------------------------------------------------------------------------ */
/* Gauge transformation (Sec. 1): U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger.
 * g holds V matrices of 18 doubles in site order. */
void or_gauge_transform(const int dims[4], double* U, const double* g) {
  lattice L = make_lattice(dims);
  for (long s = 0; s < L.V; ++s)
    for (int mu = 0; mu < 4; ++mu) {
      su3 gx, gy, u;
      memcpy(&gx, g + (size_t)s * 18, sizeof gx);
      memcpy(&gy, g + (size_t)neighbour(&L, s, mu, +1) * 18, sizeof gy);
      u = get_link(U, s, mu);
      su3 t = su3_mul(&gx, &u);
      su3 gyd = su3_dag(&gy);
      u = su3_mul(&t, &gyd);
      put_link(U, s, mu, &u);
    }
}

/* A Haar-random SU(3) matrix for one site: twelve Gaussians (Box-Muller on
 * Philox uniforms) form two complex rows; Gram-Schmidt makes them
 * orthonormal and the third row is conj(row0 x row1), so det = 1.  Rows of a
 * complex Ginibre matrix orthonormalised this way are Haar on U(3); fixing
 * the third row's phase by right-invariance gives Haar on SU(3).
 * READING: the paper only says "random starting points on the gauge orbit"
 * (Sec. 6.5-6.6). */
void or_haar_su3(uint64_t seed, uint32_t site, uint32_t copy, double out[18]) {
  double z[12];
  for (int k = 0; k < 6; ++k) {
    double u[2];
    draw2(seed, site, 0, TAG_HAAR, 0, (uint32_t)k, copy, u);
    double r = sqrt(-2.0 * log(u[0]));
    z[2 * k] = r * cos(2.0 * M_PI * u[1]);
    z[2 * k + 1] = r * sin(2.0 * M_PI * u[1]);
  }
  cplx a[3], b[3], c[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = z[2 * k] + I * z[2 * k + 1];
    b[k] = z[6 + 2 * k] + I * z[6 + 2 * k + 1];
  }
  double na = 0;
  for (int k = 0; k < 3; ++k) na += creal(a[k] * conj(a[k]));
  na = sqrt(na);
  for (int k = 0; k < 3; ++k) a[k] /= na;
  cplx ab = 0; /* <a, b> = sum conj(a_k) b_k */
  for (int k = 0; k < 3; ++k) ab += conj(a[k]) * b[k];
  for (int k = 0; k < 3; ++k) b[k] -= ab * a[k];
  double nb = 0;
  for (int k = 0; k < 3; ++k) nb += creal(b[k] * conj(b[k]));
  nb = sqrt(nb);
  for (int k = 0; k < 3; ++k) b[k] /= nb;
  c[0] = conj(a[1] * b[2] - a[2] * b[1]);
  c[1] = conj(a[2] * b[0] - a[0] * b[2]);
  c[2] = conj(a[0] * b[1] - a[1] * b[0]);
  su3 g;
  for (int k = 0; k < 3; ++k) {
    g.m[0][k] = a[k];
    g.m[1][k] = b[k];
    g.m[2][k] = c[k];
  }
  memcpy(out, &g, sizeof g);
}

/* Random gauge transformation with g(x) = or_haar_su3(seed, x, copy). */
void or_random_gauge_transform(const int dims[4], double* U, uint64_t seed,
                               uint32_t copy) {
  lattice L = make_lattice(dims);
  double* g = malloc(sizeof(double) * 18 * (size_t)L.V);
  for (long s = 0; s < L.V; ++s) or_haar_su3(seed, (uint32_t)s, copy, g + 18 * s);
  or_gauge_transform(dims, U, g);
  free(g);
}

/* Reprojection onto SU(3) (Sec. 4.5: "reproject the links to SU(3)").
 * READING: the method is not given; normalise row 0, Gram-Schmidt row 1
 * against it, normalise, and set row 2 = conj(row0 x row1). */
static void reunitarize_one(su3* u) {
  cplx* a = u->m[0];
  cplx* b = u->m[1];
  double na = 0;
  for (int k = 0; k < 3; ++k) na += creal(a[k] * conj(a[k]));
  na = sqrt(na);
  for (int k = 0; k < 3; ++k) a[k] /= na;
  cplx ab = 0;
  for (int k = 0; k < 3; ++k) ab += conj(a[k]) * b[k];
  for (int k = 0; k < 3; ++k) b[k] -= ab * a[k];
  double nb = 0;
  for (int k = 0; k < 3; ++k) nb += creal(b[k] * conj(b[k]));
  nb = sqrt(nb);
  for (int k = 0; k < 3; ++k) b[k] /= nb;
  u->m[2][0] = conj(a[1] * b[2] - a[2] * b[1]);
  u->m[2][1] = conj(a[2] * b[0] - a[0] * b[2]);
  u->m[2][2] = conj(a[0] * b[1] - a[1] * b[0]);
}

void or_reunitarize(const int dims[4], double* U) {
  lattice L = make_lattice(dims);
  for (long s = 0; s < L.V; ++s)
    for (int mu = 0; mu < 4; ++mu) {
      su3 u = get_link(U, s, mu);
      reunitarize_one(&u);
      put_link(U, s, mu, &u);
    }
}

/* ------------------------------------------------------------------------ */
/* Observables. */

/* Which directions enter the Landau/Coulomb sums (Sec. 2.1.1): all four for
 * Landau, the spatial ones for Coulomb. */
static int mu_first(int gauge) { return gauge == OR_COULOMB ? 1 : 0; }

/* K(x) = sum_mu [U_mu(x) + U_mu(x - mu)^dagger] on the current links
 * (Eq. Kx with the neighbours' g already applied in place). */
static su3 gather_K(const lattice* L, const double* U, long s, int gauge) {
  su3 K;
  memset(&K, 0, sizeof K);
  for (int mu = mu_first(gauge); mu < 4; ++mu) {
    su3 up = get_link(U, s, mu);
    su3 dn = get_link(U, neighbour(L, s, mu, -1), mu);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) K.m[i][j] += up.m[i][j] + conj(dn.m[j][i]);
  }
  return K;
}

/* tr[Delta Delta^dagger] at one site, where Delta(x) = sum_mu (A_mu(x) -
 * A_mu(x - mu)) and A_mu = traceless part of (U - U^dagger)/(2i)
 * (Sec. 2.1.1).  READING: the lattice A_mu is not defined in the paper; with
 * this definition Delta is the traceless part of (K - K^dagger)/(2i). */
static double theta_site_landau(const lattice* L, const double* U, long s,
                                int gauge) {
  su3 K = gather_K(L, U, s, gauge);
  cplx D[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = (K.m[i][j] - conj(K.m[j][i])) / (2.0 * I);
  cplx tr3 = (D[0][0] + D[1][1] + D[2][2]) / 3.0;
  for (int i = 0; i < 3; ++i) D[i][i] -= tr3;
  double t = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t += creal(D[i][j] * conj(D[i][j]));
  return t;
}

/* Pauli vector of X = sum_mu (W_mu s3 W_mu^dag + D_mu^dag s3 D_mu) for the
 * subgroup (i,j) at site s, W/D the (i,j) blocks of U_mu(x) / U_mu(x-mu)
 * (Sec. 2.1.2, the matrix X(x)).  X = x0 + x.sigma; returns (x1, x2, x3) =
 * (Re X01, -Im X01, (X00 - X11)/2).  READING: Sec. 2.2.2 writes the
 * down-link term with U sigma3 U^dagger; X(x) of Sec. 2.1.2 and the
 * derivation of the local functional give D^dagger sigma3 D, used here. */
static void mag_vector(const lattice* L, const double* U, long s, int i, int j,
                       double x[3]) {
  cplx X[2][2] = {{0, 0}, {0, 0}};
  const int idx[2] = {i, j};
  const double s3[2] = {1.0, -1.0};
  for (int mu = 0; mu < 4; ++mu) {
    su3 up = get_link(U, s, mu);
    su3 dn = get_link(U, neighbour(L, s, mu, -1), mu);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c) {
          /* (W s3 W^dag)_ab = sum_c W_ac s3_c conj(W_bc) */
          X[a][b] += up.m[idx[a]][idx[c]] * s3[c] * conj(up.m[idx[b]][idx[c]]);
          /* (D^dag s3 D)_ab = sum_c conj(D_ca) s3_c D_cb */
          X[a][b] += conj(dn.m[idx[c]][idx[a]]) * s3[c] * dn.m[idx[c]][idx[b]];
        }
  }
  x[0] = creal(X[0][1]);
  x[1] = -cimag(X[0][1]);
  x[2] = 0.5 * creal(X[0][0] - X[1][1]);
}

/* Functional F and gauge precision theta (Sec. 2.1).
 *  Landau:  F = (1/(Nc Nd V)) Re sum_{x,mu} tr U_mu(x),
 *           theta = (1/(Nc V)) sum_x tr[Delta Delta^dag].
 *  Coulomb: per time-slice t with V3 sites, F_t uses mu = 1..3 and
 *           1/(Nc 3 V3), theta_t uses 1/(Nc V3); F and theta are the means
 *           over slices.  F_t / theta_t may be NULL.
 *  MAG:     F = (1/(Nc Nd V)) sum |U_ii|^2 (Eq. MAG_functional),
 *           theta = (1/(Nc V)) sum_x sum_subgroups |X_01|^2.
 *           READING: the SU(3) theta of Sec. 2.1.2 adds off-diagonal
 *           elements of different subgroups; we sum their squares. */
void or_observables(const int dims[4], const double* U, int gauge, double* F,
                    double* theta, double* F_t, double* theta_t) {
  lattice L = make_lattice(dims);
  int Nt = L.n[0];
  long V3 = L.V / Nt;
  double* ft = calloc((size_t)Nt, sizeof(double));
  double* tt = calloc((size_t)Nt, sizeof(double));
  for (long s = 0; s < L.V; ++s) {
    int t = (int)(s / V3);
    for (int mu = 0; mu < 4; ++mu) {
      su3 u = get_link(U, s, mu);
      if (gauge == OR_MAG) {
        for (int i = 0; i < 3; ++i) ft[t] += creal(u.m[i][i] * conj(u.m[i][i]));
      } else if (mu >= mu_first(gauge)) {
        ft[t] += creal(u.m[0][0] + u.m[1][1] + u.m[2][2]);
      }
    }
    if (gauge == OR_MAG) {
      for (int sub = 0; sub < 3; ++sub) {
        double x[3];
        mag_vector(&L, U, s, SUBGROUP[sub][0], SUBGROUP[sub][1], x);
        tt[t] += x[0] * x[0] + x[1] * x[1];
      }
    } else {
      tt[t] += theta_site_landau(&L, U, s, gauge);
    }
  }
  int nd = (gauge == OR_COULOMB) ? 3 : 4;
  double Fsum = 0, Tsum = 0;
  for (int t = 0; t < Nt; ++t) {
    ft[t] /= 3.0 * nd * (double)V3;
    tt[t] /= 3.0 * (double)V3;
    Fsum += ft[t];
    Tsum += tt[t];
    if (F_t) F_t[t] = ft[t];
    if (theta_t) theta_t[t] = tt[t];
  }
  *F = Fsum / Nt;
  *theta = Tsum / Nt;
  free(ft);
  free(tt);
}

/* Average plaquette (1/(18 V)) sum_{x, mu<nu} Re tr[U_mu(x) U_nu(x+mu)
 * U_mu(x+nu)^dag U_nu(x)^dag].  The standard Wilson form; the paper does not
 * use it, it serves as a gauge-invariant check. */
double or_plaquette(const int dims[4], const double* U) {
  lattice L = make_lattice(dims);
  double sum = 0;
  for (long s = 0; s < L.V; ++s)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        su3 a = get_link(U, s, mu);
        su3 b = get_link(U, neighbour(&L, s, mu, +1), nu);
        su3 c = get_link(U, neighbour(&L, s, nu, +1), mu);
        su3 d = get_link(U, s, nu);
        su3 cd = su3_dag(&c), dd = su3_dag(&d);
        su3 ab = su3_mul(&a, &b);
        su3 abc = su3_mul(&ab, &cd);
        su3 p = su3_mul(&abc, &dd);
        sum += creal(p.m[0][0] + p.m[1][1] + p.m[2][2]);
      }
  return sum / (18.0 * (double)L.V);
}

/* Unitarity measure of Sec. 4.5: mean and max over links of |1 - det U|. */
void or_unitarity(const int dims[4], const double* U, double* mean,
                  double* maxdev) {
  lattice L = make_lattice(dims);
  double sum = 0, mx = 0;
  for (long s = 0; s < L.V; ++s)
    for (int mu = 0; mu < 4; ++mu) {
      su3 u = get_link(U, s, mu);
      double d = cabs(1.0 - su3_det(&u));
      sum += d;
      if (d > mx) mx = d;
    }
  *mean = sum / (4.0 * (double)L.V);
  *maxdev = mx;
}

/* ------------------------------------------------------------------------ */
/* Step 1: the local SU(2) update for one subgroup. */

/* The maximiser direction for Landau/Coulomb.  For the Cayley-Klein g and
 * the (i,j) block W of K, expanding the trace gives Re tr(g W) = g0 a0 - g.a
 * with a = (Re W00 + Re W11, Im W01 + Im W10, Re W01 - Re W10,
 * Im W00 - Im W11) (the same four sums as App. A), so the maximiser is the
 * conjugate (a0, -a1, -a2, -a3) normalised (Eq. localsolution for SU(2)). */
static void landau_maximiser(const su3* K, int i, int j, double m[4]) {
  cplx W00 = K->m[i][i], W01 = K->m[i][j], W10 = K->m[j][i], W11 = K->m[j][j];
  double a0 = creal(W00) + creal(W11);
  double a1 = cimag(W01) + cimag(W10);
  double a2 = creal(W01) - creal(W10);
  double a3 = cimag(W00) - cimag(W11);
  m[0] = a0;
  m[1] = -a1;
  m[2] = -a2;
  m[3] = -a3;
}

/* The MAG maximiser (Sec. 2.2.2): with g3 = 0 the local functional is
 * const + g^T M g with M = [[D, E, F], [E, -D, 0], [F, 0, -D]], whose top
 * eigenvector is (D + sqrt(D^2 + E^2 + F^2), E, F).  In terms of the Pauli
 * vector of X: D = x3, E = -x2, F = x1.  For x3 < 0 the first component is
 * written as (x1^2 + x2^2)/(|x| - x3) to avoid cancellation.  Degenerate
 * cases (READING): x = 0 gives the identity, x along -z gives i sigma1. */
static void mag_maximiser(const double x[3], double m[4]) {
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  m[3] = 0;
  if (r == 0) {
    m[0] = 1; m[1] = 0; m[2] = 0;
    return;
  }
  double top = x[2] >= 0 ? x[2] + r : (x[0] * x[0] + x[1] * x[1]) / (r - x[2]);
  double v0 = top, v1 = -x[1], v2 = x[0];
  double n = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  if (n == 0) {
    m[0] = 0; m[1] = 1; m[2] = 0;
    return;
  }
  m[0] = v0 / n;
  m[1] = v1 / n;
  m[2] = v2 / n;
}

/* Overrelaxation (Sec. 2.2.3): the relaxation update g is replaced by its
 * power g^w, taken to first order in the rotation angle.  With q = m/|m| =
 * (q0, v) the unit maximiser, the vector part is stretched by
 * s = 1 + (w - 1) q0^2 and the result normalised, g = (q0, s v)/|(q0, s v)|:
 * for the small rotations near convergence q0 -> 1 and s -> w, so the angle
 * grows by w (g^w to first order); for a rotation by pi (q0 = 0) s = 1.
 * READING: Sec. 2.2.3 does not write the first-order form out; App. A's update
 * uses this stretch factor.  w = 1 is plain relaxation; a zero quaternion
 * gives the identity. */
static void or_update(const double m[4], double omega, double g[4]) {
  double nm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
  if (nm == 0) {
    g[0] = 1; g[1] = g[2] = g[3] = 0;
    return;
  }
  double q[4];
  for (int k = 0; k < 4; ++k) q[k] = m[k] / nm;
  double s = 1.0 + (omega - 1.0) * q[0] * q[0];
  double h[4] = {q[0], s * q[1], s * q[2], s * q[3]};
  double nh = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2] + h[3] * h[3]);
  for (int k = 0; k < 4; ++k) g[k] = h[k] / nh;
}

/* Microcanonical step (Sec. 2.2.4): the square of the normalised maximiser,
 * g^2 = (2 g0^2 - 1, 2 g0 g).  READING: the exact square, which leaves the
 * local functional invariant; the OR formula at w = 2 does not. */
static void micro_update(const double m[4], double g[4]) {
  double n = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
  if (n == 0) {
    g[0] = 1; g[1] = g[2] = g[3] = 0;
    return;
  }
  double q0 = m[0] / n;
  g[0] = 2 * q0 * q0 - 1;
  for (int k = 1; k < 4; ++k) g[k] = 2 * q0 * (m[k] / n);
}

/* Kennedy-Pendleton (Phys. Lett. B 156 (1985) 393) sample of x0 in [-1,1]
 * with density proportional to sqrt(1 - x0^2) exp(alpha x0).  With
 * x0 = 1 - 2 delta the proposal delta ~ Gamma(3/2, rate 2 alpha) is
 * -(ln r1 + cos^2(2 pi r2) ln r3)/(2 alpha), accepted when
 * r4^2 <= 1 - delta.  READING: the heat-bath algorithm is not named in
 * Sec. 2.3; trials are capped at 64 and x0 = 1 is kept if none is accepted.
 * Returns the number of trials used (0 = cap hit).  margin (may be NULL)
 * receives the smallest |r4^2 - (1 - delta)| over the trials taken: how close
 * the nearest accept/reject decision came to its threshold. */
static int kp_sample(double alpha, uint64_t seed, uint32_t site, uint32_t sweep,
                     uint32_t sub, uint32_t copy, double* x0, double* margin) {
  double closest = INFINITY;
  for (int trial = 0; trial < KP_MAX_TRIALS; ++trial) {
    double ua[2], ub[2];
    draw2(seed, site, sweep, TAG_SA, sub, (uint32_t)(2 * trial), copy, ua);
    draw2(seed, site, sweep, TAG_SA, sub, (uint32_t)(2 * trial + 1), copy, ub);
    double c = cos(2.0 * M_PI * ua[1]);
    double delta = -(log(ua[0]) + c * c * log(ub[0])) / (2.0 * alpha);
    double gap = fabs(ub[1] * ub[1] - (1.0 - delta));
    if (gap < closest) closest = gap;
    if (ub[1] * ub[1] <= 1.0 - delta) {
      *x0 = 1.0 - 2.0 * delta;
      if (margin) *margin = closest;
      return trial + 1;
    }
  }
  *x0 = 1.0;
  if (margin) *margin = closest;
  return 0;
}

int or_kp_sample(double alpha, uint64_t seed, uint32_t site, uint32_t sweep,
                 uint32_t sub, uint32_t copy, double* x0) {
  return kp_sample(alpha, seed, site, sweep, sub, copy, x0, NULL);
}

/* Direction draw used by the Landau heat bath (draw index 128). */
#define KP_DIRECTION_DRAW 128u

/* Heat bath for Landau/Coulomb (Sec. 2.3): the subgroup weight is
 * exp(Re tr(g W)/T) = exp(|m| (g.n)/T) with n = m/|m|.  Draw h with
 * h0 ~ sqrt(1-h0^2) exp(alpha h0), alpha = |m|/T, and a uniform direction,
 * then g = h n, so that g.n = h0. */
static int sa_landau_update(const double m[4], double T, uint64_t seed,
                            uint32_t site, uint32_t sweep, uint32_t sub,
                            uint32_t copy, double g[4], double* margin) {
  double nm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
  if (margin) *margin = INFINITY;
  if (nm == 0) {
    g[0] = 1; g[1] = g[2] = g[3] = 0;
    return 1;
  }
  double x0;
  int trials = kp_sample(nm / T, seed, site, sweep, sub, copy, &x0, margin);
  double u[2];
  draw2(seed, site, sweep, TAG_SA, sub, KP_DIRECTION_DRAW, copy, u);
  double cth = 2.0 * u[0] - 1.0;
  double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
  double phi = 2.0 * M_PI * u[1];
  double r = sqrt(fmax(0.0, 1.0 - x0 * x0));
  double h[4] = {x0, r * sth * cos(phi), r * sth * sin(phi), r * cth};
  double n[4] = {m[0] / nm, m[1] / nm, m[2] / nm, m[3] / nm};
  su2 H = su2_from_quaternion(h), N = su2_from_quaternion(n);
  su2 G = su2_mul(&H, &N);
  /* read the quaternion back from the Cayley-Klein form */
  g[0] = creal(G.m[0][0]);
  g[3] = cimag(G.m[0][0]);
  g[2] = creal(G.m[0][1]);
  g[1] = cimag(G.m[0][1]);
  return trials;
}

/* cos(beta) with density proportional to exp(kappa cos(beta)) on [-1,1], by
 * inversion of its distribution function. */
double or_mag_cosbeta(double kappa, double u) {
  double c = 1.0 + log1p(u * expm1(-2.0 * kappa)) / kappa;
  return fmin(1.0, fmax(-1.0, c));
}

/* Heat bath for MAG: the local functional is const + |x| cos(beta), beta
 * the angle between R(g) x and +z; under Haar g the rotated direction is
 * uniform on the sphere, so cos(beta) ~ exp(kappa cos(beta)), kappa = |x|/T,
 * and the azimuth is uniform.  g = r h1 with h1 the maximiser (x -> +z) and
 * r the g3 = 0 rotation taking +z to that direction.  READING: Sec. 2.3
 * does not give the MAG heat bath; the U(1) phase left free by the sigma3
 * symmetry is not drawn. */
static void sa_mag_update(const double x[3], double T, uint64_t seed,
                          uint32_t site, uint32_t sweep, uint32_t sub,
                          uint32_t copy, double g[4]) {
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  if (r == 0) {
    g[0] = 1; g[1] = g[2] = g[3] = 0;
    return;
  }
  double h1[4];
  mag_maximiser(x, h1);
  double u[2];
  draw2(seed, site, sweep, TAG_SA, sub, 0, copy, u);
  double cb = or_mag_cosbeta(r / T, u[0]);
  double phi = 2.0 * M_PI * u[1];
  double ch = sqrt(0.5 * (1.0 + cb)), sh = sqrt(0.5 * (1.0 - cb));
  double rq[4] = {ch, sh * sin(phi), -sh * cos(phi), 0.0};
  su2 R = su2_from_quaternion(rq), H = su2_from_quaternion(h1);
  su2 G = su2_mul(&R, &H);
  g[0] = creal(G.m[0][0]);
  g[3] = cimag(G.m[0][0]);
  g[2] = creal(G.m[0][1]);
  g[1] = cimag(G.m[0][1]);
}

/* ------------------------------------------------------------------------ */
/* One subgroup step at one site: Step 1 (find g) and Step 2 (apply it to
 * the eight links U_mu(x) and U_mu(x - mu)) of Alg. 1.  For Coulomb the
 * local functional uses the spatial links only but g is applied to all four
 * directions, so the temporal links follow the gauge transformation.  For the
 * Landau/Coulomb heat bath, trials/margin (may be NULL) receive the
 * Kennedy-Pendleton trial count and decision margin of this update. */
static void site_subgroup_update(const int dims[4], double* U, long s, int sub,
                                 int gauge, int algo, double param,
                                 uint32_t sweep, uint64_t seed, uint32_t copy,
                                 int* trials, double* margin) {
  lattice L = make_lattice(dims);
  int i = SUBGROUP[sub][0], j = SUBGROUP[sub][1];
  double m[4], g[4], x[3] = {0, 0, 0};
  if (gauge == OR_MAG) {
    mag_vector(&L, U, s, i, j, x);
    mag_maximiser(x, m);
  } else {
    su3 K = gather_K(&L, U, s, gauge);
    landau_maximiser(&K, i, j, m);
  }
  switch (algo) {
    case OR_ALGO_RELAX:
      or_update(m, 1.0, g);
      break;
    case OR_ALGO_OR:
      or_update(m, param, g);
      break;
    case OR_ALGO_MICRO:
      micro_update(m, g);
      break;
    case OR_ALGO_SR: {
      /* Stochastic relaxation (Sec. 2.2.5): the microcanonical step with
       * probability p, plain relaxation otherwise.  READING: one draw per
       * site and subgroup. */
      double u[2];
      draw2(seed, (uint32_t)s, sweep, TAG_SR, (uint32_t)sub, 0, copy, u);
      if (u[0] < param)
        micro_update(m, g);
      else
        or_update(m, 1.0, g);
      break;
    }
    case OR_ALGO_SA: {
      int n = 1;
      double gap = INFINITY;
      if (gauge == OR_MAG)
        sa_mag_update(x, param, seed, (uint32_t)s, sweep, (uint32_t)sub, copy, g);
      else
        n = sa_landau_update(m, param, seed, (uint32_t)s, sweep, (uint32_t)sub, copy, g, &gap);
      if (trials) *trials = n;
      if (margin) *margin = gap;
      break;
    }
    default:
      return;
  }
  su2 h = su2_from_quaternion(g);
  su3 G = embed(&h, i, j);
  su3 Gd = su3_dag(&G);
  for (int mu = 0; mu < 4; ++mu) {
    su3 up = get_link(U, s, mu);
    up = su3_mul(&G, &up);
    put_link(U, s, mu, &up);
    long sd = neighbour(&L, s, mu, -1);
    su3 dn = get_link(U, sd, mu);
    dn = su3_mul(&dn, &Gd);
    put_link(U, sd, mu, &dn);
  }
}

void or_site_subgroup_update(const int dims[4], double* U, long s, int sub,
                             int gauge, int algo, double param, uint32_t sweep,
                             uint64_t seed, uint32_t copy) {
  site_subgroup_update(dims, U, s, sub, gauge, algo, param, sweep, seed, copy,
                       NULL, NULL);
}

/* Checkerboard sweeps (Alg. 1): for each sweep, the even sublattice, then
 * the odd one; at each site the three subgroups in the order (0,1), (0,2),
 * (1,2) (READING: the order is not stated).  Random draws use the sweep
 * index sweep0 + k.  For Coulomb, slice_active (Nt flags, NULL = all) skips
 * time-slices that have stopped.  or_sweep_trace also records, for the last
 * sweep and every (site, subgroup) in the order s*3 + sub, the heat-bath
 * trial count (1 for MAG and for the other rules) and decision margin
 * (infinite where no accept/reject decision was taken). */
/* One half of a sweep: the sites of parity p (Alg. 1's inner loop). */
static void half_sweep(const lattice* L, const int dims[4], double* U, int gauge,
                       int algo, double param, int p, uint32_t sweep,
                       uint64_t seed, uint32_t copy, const int* slice_active,
                       int* trials, double* margin) {
  long V3 = L->V / L->n[0];
  /* sites of one parity touch disjoint links (Sec. 2.2): a build with
   * -fopenmp may visit them in parallel with the same result; the plain
   * build ignores the pragma */
#pragma omp parallel for schedule(static)
  for (long s = 0; s < L->V; ++s) {
    if (parity_of(L, s) != p) continue;
    if (slice_active && !slice_active[s / V3]) continue;
    for (int sub = 0; sub < 3; ++sub) {
      int n = 1;
      double gap = INFINITY;
      site_subgroup_update(dims, U, s, sub, gauge, algo, param, sweep, seed,
                           copy, &n, &gap);
      if (trials) trials[s * 3 + sub] = n;
      if (margin) margin[s * 3 + sub] = gap;
    }
  }
}

void or_sweep_trace(const int dims[4], double* U, int gauge, int algo,
                    double param, int n_sweeps, uint32_t sweep0, uint64_t seed,
                    uint32_t copy, const int* slice_active, int* trials,
                    double* margin) {
  lattice L = make_lattice(dims);
  for (int k = 0; k < n_sweeps; ++k)
    for (int p = 0; p < 2; ++p)
      half_sweep(&L, dims, U, gauge, algo, param, p, sweep0 + (uint32_t)k,
                 seed, copy, slice_active, trials, margin);
}

/* The sites of parity p only, with the draws of sweep index `sweep` (the
 * half-sweeps of Alg. 1 one at a time, as a time-slab decomposition over
 * several processes runs them, Sec. 5). */
void or_half_sweep(const int dims[4], double* U, int gauge, int algo,
                   double param, int parity, uint32_t sweep, uint64_t seed,
                   uint32_t copy, const int* slice_active) {
  lattice L = make_lattice(dims);
  half_sweep(&L, dims, U, gauge, algo, param, parity & 1, sweep, seed, copy,
             slice_active, NULL, NULL);
}

void or_sweep(const int dims[4], double* U, int gauge, int algo, double param,
              int n_sweeps, uint32_t sweep0, uint64_t seed, uint32_t copy,
              const int* slice_active) {
  or_sweep_trace(dims, U, gauge, algo, param, n_sweeps, sweep0, seed, copy,
                 slice_active, NULL, NULL);
}

/* Simulated annealing (Sec. 2.3): n heat-bath sweeps at temperatures
 * falling linearly from T0 to T1, each followed by three microcanonical
 * sweeps.  READING: the schedule shape is not given ("from 4 down to 1e-4",
 * Sec. 6.6); we take it linear in T.  The sweep counter advances by four per
 * step. */
void or_anneal(const int dims[4], double* U, int gauge, double T0, double T1,
               int n, uint32_t sweep0, uint64_t seed, uint32_t copy) {
  uint32_t sw = sweep0;
  for (int k = 0; k < n; ++k) {
    double T = n > 1 ? T0 + (T1 - T0) * (double)k / (double)(n - 1) : T0;
    or_sweep(dims, U, gauge, OR_ALGO_SA, T, 1, sw, seed, copy, NULL);
    or_sweep(dims, U, gauge, OR_ALGO_MICRO, 0.0, 3, sw + 1, seed, copy, NULL);
    sw += 4;
  }
}

/* The deterministic update rules on a maximiser quaternion m (relaxation,
 * overrelaxation with w = param, microcanonical), exposed for the pins. */
void or_step_quaternion(const double m[4], int algo, double param, double g[4]) {
  if (algo == OR_ALGO_MICRO)
    micro_update(m, g);
  else
    or_update(m, algo == OR_ALGO_OR ? param : 1.0, g);
}

/* The complete heat-bath update of one subgroup, exposed for the pins:
 * Landau/Coulomb from the maximiser direction v = m (4 entries, unnormalised),
 * MAG from the Pauli vector v = x (3 entries), at temperature T with the
 * draws of (seed, site, sweep, sub, copy).  Returns the Kennedy-Pendleton
 * trial count (Landau/Coulomb; 0 = cap hit) or 1 (MAG). */
int or_sa_update(int gauge, const double v[4], double T, uint64_t seed,
                 uint32_t site, uint32_t sweep, uint32_t sub, uint32_t copy,
                 double g[4]) {
  if (gauge == OR_MAG) {
    sa_mag_update(v, T, seed, site, sweep, sub, copy, g);
    return 1;
  }
  return sa_landau_update(v, T, seed, site, sweep, sub, copy, g, NULL);
}

/* The MAG maximiser for a Pauli vector x, exposed for the pins. */
void or_mag_maximiser(const double x[3], double m[4]) { mag_maximiser(x, m); }

/* g(x) = or_haar_su3(seed, site, copy) for the n sites site0 .. site0+n-1,
 * written as n consecutive 3x3 matrices (for building the transformation of
 * a sub-lattice cut out of a larger one). */
void or_haar_field(uint64_t seed, uint32_t site0, long n, uint32_t copy, double* out) {
  for (long k = 0; k < n; ++k) or_haar_su3(seed, site0 + (uint32_t)k, copy, out + 18 * k);
}
