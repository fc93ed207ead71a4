// gf_device.cuh -- device-side building blocks of the gauge-fixing kernels.
//
// Storage ("parity-split structure of arrays", the GB300 form of the
// GpuPatternParityPriority layout of Sec. 4.2.1): for copy c, parity p, slot
// mu, chunk k and site index sp within the parity,
//     element((c*2 + p)*NS + mu)*NC + k)*Vh + sp
// holds one 16-byte vector.  A link keeps its first two rows only (the
// 12-parameter representation of Sec. 4.2); the third row is conj(row0 x
// row1).  FP32: NC = 3 float4 (u00 u01 | u02 u10 | u11 u12).  FP64: NC = 6
// double2, one complex entry each.  Slots: mu = 0..3 are the links U_mu(x);
// Coulomb adds slot 4, the accumulated gauge transformation g(x) of the
// time-slice sweeps.  A site's index is s = ((t*Nx + x)*Ny + y)*Nz + z; its
// index within its parity is s >> 1 (all extents even).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gfk {

enum Gauge { LANDAU = 0, COULOMB = 1, MAG = 2 };
enum Algo { ALG_OR = 0, ALG_MICRO = 1, ALG_SR = 2, ALG_SA = 3 };

// Philox counter word 2: stream tag << 24 | subgroup << 8 | draw.
constexpr uint32_t TAG_SR = 1u, TAG_SA = 2u, TAG_HAAR = 3u;
constexpr int KP_TRIALS = 64;
constexpr uint32_t KP_DIR_DRAW = 128u;

// ---------------------------------------------------------------------------
// Division by a runtime constant: q = (umulhi(n, m) + n) >> l for n < 2^31
// (the round-up multiplier of Granlund & Montgomery, PLDI 1994).
struct FastDiv {
  uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return FastDiv{d, (uint32_t)m, l};
}

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  uint32_t t = __umulhi(n, f.m);
#else
  uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (t + n) >> f.l;
}

struct Geom {
  int n[4];            // Nt, Nx, Ny, Nz
  uint32_t V, Vh, V3;  // sites, sites per parity, sites per time-slice
  uint32_t stride[4];  // V3, Ny*Nz, Nz, 1
  FastDiv dz, dy, dx;
};

// Coordinates of the site with parity p and parity index sp.
__device__ __forceinline__ void site_coords(const Geom& g, uint32_t sp, int p, int c[4],
                                            uint32_t& s) {
  uint32_t s0 = 2u * sp;
  uint32_t q1 = fdiv(s0, g.dz);
  uint32_t z0 = s0 - q1 * (uint32_t)g.n[3];
  uint32_t q2 = fdiv(q1, g.dy);
  uint32_t y = q1 - q2 * (uint32_t)g.n[2];
  uint32_t t = fdiv(q2, g.dx);
  uint32_t x = q2 - t * (uint32_t)g.n[1];
  uint32_t b = ((t + x + y) ^ (uint32_t)p) & 1u;
  c[0] = (int)t;
  c[1] = (int)x;
  c[2] = (int)y;
  c[3] = (int)(z0 + b);
  s = s0 + b;
}

// Lexicographic index of x - mu (periodic).
__device__ __forceinline__ uint32_t site_minus(const Geom& g, uint32_t s, const int c[4], int mu) {
  return c[mu] > 0 ? s - g.stride[mu] : s + (uint32_t)(g.n[mu] - 1) * g.stride[mu];
}
__device__ __forceinline__ uint32_t site_plus(const Geom& g, uint32_t s, const int c[4], int mu) {
  return c[mu] < g.n[mu] - 1 ? s + g.stride[mu] : s - (uint32_t)(g.n[mu] - 1) * g.stride[mu];
}

// ---------------------------------------------------------------------------
// Complex numbers and 3x3 matrices in registers.
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * b + c * d
template <typename R>
__device__ __forceinline__ cx<R> cmul2(cx<R> a, cx<R> b, cx<R> c, cx<R> d) {
  return {a.re * b.re - a.im * b.im + c.re * d.re - c.im * d.im,
          a.re * b.im + a.im * b.re + c.re * d.im + c.im * d.re};
}
// a * conj(b) + c * conj(d)
template <typename R>
__device__ __forceinline__ cx<R> cmul2c(cx<R> a, cx<R> b, cx<R> c, cx<R> d) {
  return {a.re * b.re + a.im * b.im + c.re * d.re + c.im * d.im,
          a.im * b.re - a.re * b.im + c.im * d.re - c.re * d.im};
}
// conj(a*b - c*d)
template <typename R>
__device__ __forceinline__ cx<R> cross_conj(cx<R> a, cx<R> b, cx<R> c, cx<R> d) {
  return {a.re * b.re - a.im * b.im - (c.re * d.re - c.im * d.im),
          -(a.re * b.im + a.im * b.re - (c.re * d.im + c.im * d.re))};
}

template <typename R>
struct mat3 {
  cx<R> e[3][3];
};

// Third row of an SU(3) matrix from its first two: conj(row0 x row1).
template <typename R>
__device__ __forceinline__ void reconstruct_row2(mat3<R>& u) {
  u.e[2][0] = cross_conj(u.e[0][1], u.e[1][2], u.e[0][2], u.e[1][1]);
  u.e[2][1] = cross_conj(u.e[0][2], u.e[1][0], u.e[0][0], u.e[1][2]);
  u.e[2][2] = cross_conj(u.e[0][0], u.e[1][1], u.e[0][1], u.e[1][0]);
}

// ---------------------------------------------------------------------------
// Link storage: NC vectors of 16 bytes per link.
template <typename R>
struct store_traits;
template <>
struct store_traits<float> {
  using vec = float4;
  static constexpr int NC = 3;
};
template <>
struct store_traits<double> {
  using vec = double2;
  static constexpr int NC = 6;
};

__device__ __forceinline__ void load_rows(const float4* __restrict__ p, size_t stride, mat3<float>& u) {
  float4 a = p[0], b = p[stride], c = p[2 * stride];
  u.e[0][0] = {a.x, a.y};
  u.e[0][1] = {a.z, a.w};
  u.e[0][2] = {b.x, b.y};
  u.e[1][0] = {b.z, b.w};
  u.e[1][1] = {c.x, c.y};
  u.e[1][2] = {c.z, c.w};
}
__device__ __forceinline__ void store_rows(float4* __restrict__ p, size_t stride, const mat3<float>& u) {
  p[0] = make_float4(u.e[0][0].re, u.e[0][0].im, u.e[0][1].re, u.e[0][1].im);
  p[stride] = make_float4(u.e[0][2].re, u.e[0][2].im, u.e[1][0].re, u.e[1][0].im);
  p[2 * stride] = make_float4(u.e[1][1].re, u.e[1][1].im, u.e[1][2].re, u.e[1][2].im);
}
__device__ __forceinline__ void load_rows(const double2* __restrict__ p, size_t stride, mat3<double>& u) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double2 v = p[k * stride];
    u.e[k / 3][k % 3] = {v.x, v.y};
  }
}
__device__ __forceinline__ void store_rows(double2* __restrict__ p, size_t stride, const mat3<double>& u) {
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k * stride] = make_double2(u.e[k / 3][k % 3].re, u.e[k / 3][k % 3].im);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), this file's own implementation.
struct u4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u4 philox10(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = u4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// (0,1) uniform: top 52 bits of hi:lo, plus one half, times 2^-52 (exact).
__device__ __forceinline__ double u01(uint32_t hi, uint32_t lo) {
  uint64_t b = ((uint64_t)hi << 32) | lo;
  return ((double)(b >> 12) + 0.5) * 0x1p-52;
}

struct Rng {
  uint32_t k0, k1, site, sweep, copy;
  __device__ __forceinline__ void draw2(uint32_t tag, uint32_t sub, uint32_t draw, double& a,
                                        double& b) const {
    u4 r = philox10(u4{site, sweep, (tag << 24) | (sub << 8) | draw, copy}, k0, k1);
    a = u01(r.x, r.y);
    b = u01(r.z, r.w);
  }
};

// ---------------------------------------------------------------------------
// Math wrappers per precision.
__device__ __forceinline__ float rsqrt_(float x) { return 1.0f / sqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
// the math library's reciprocal square root (a few ulp, no division)
__device__ __forceinline__ float rsq_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq_(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double log_(double x) { return log(x); }
__device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_(double x) { return log1p(x); }
__device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_(double x) { return expm1(x); }
__device__ __forceinline__ void sincos2pi(float u, float& s, float& c) { sincospif(2.0f * u, &s, &c); }
__device__ __forceinline__ void sincos2pi(double u, double& s, double& c) { sincospi(2.0 * u, &s, &c); }
__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }

// ---------------------------------------------------------------------------
// Quaternions q = (q0, q1, q2, q3) <-> q0 + i(q1 s1 + q2 s2 + q3 s3)
//   = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]  (Sec. 2.2.2).
template <typename R>
struct quat {
  R q0, q1, q2, q3;
};

// Product matching the matrix product Q(a) Q(b):
// (a0 b0 - a.b, a0 b + b0 a - a x b).
template <typename R>
__device__ __forceinline__ quat<R> qmul(quat<R> a, quat<R> b) {
  return {a.q0 * b.q0 - a.q1 * b.q1 - a.q2 * b.q2 - a.q3 * b.q3,
          a.q0 * b.q1 + b.q0 * a.q1 - (a.q2 * b.q3 - a.q3 * b.q2),
          a.q0 * b.q2 + b.q0 * a.q2 - (a.q3 * b.q1 - a.q1 * b.q3),
          a.q0 * b.q3 + b.q0 * a.q3 - (a.q1 * b.q2 - a.q2 * b.q1)};
}

template <typename R>
__device__ __forceinline__ quat<R> qidentity() {
  return {R(1), R(0), R(0), R(0)};
}

// Overrelaxation (Sec. 2.2.3): g^w to first order in the rotation angle.  On
// the maximiser direction m = (a0, a), the vector part is stretched by
// b = 1 + (w - 1) a0^2/|m|^2 and the result normalised; w = 1 is relaxation,
// a zero m gives the identity.
template <typename R>
__device__ __forceinline__ quat<R> rule_or(quat<R> m, R omega) {
  // x0, xi: the squared parts of the normalised quaternion, so that two
  // reciprocal square roots replace the division and the square root
  R a0 = m.q0 * m.q0;
  R ai = m.q1 * m.q1 + m.q2 * m.q2 + m.q3 * m.q3;
  R den = a0 + ai;
  if (den == R(0)) return qidentity<R>();
  const R s = rsq_(den);
  const R s2 = s * s;
  const R x0 = a0 * s2, xi = ai * s2;
  const R b = omega * x0 + xi;
  const R c = rsq_(x0 + b * b * xi) * s;
  const R bc = b * c;
  return {c * m.q0, bc * m.q1, bc * m.q2, bc * m.q3};
}

// Microcanonical step (Sec. 2.2.4): the square of the normalised maximiser.
template <typename R>
__device__ __forceinline__ quat<R> rule_micro(quat<R> m) {
  R n2 = m.q0 * m.q0 + m.q1 * m.q1 + m.q2 * m.q2 + m.q3 * m.q3;
  if (n2 == R(0)) return qidentity<R>();
  R inv = rsq_(n2);
  R h0 = m.q0 * inv;
  R f = R(2) * h0 * inv;
  return {R(2) * h0 * h0 - R(1), f * m.q1, f * m.q2, f * m.q3};
}

// MAG maximiser from the Pauli vector x of X (Sec. 2.2.2, Eq. upMatrix):
// the top eigenvector (D + sqrt(D^2+E^2+F^2), E, F) with D = x3, E = -x2,
// F = x1, normalised; for x3 < 0 its first entry is (x1^2+x2^2)/(|x| - x3).
template <typename R>
__device__ __forceinline__ quat<R> mag_max(R x1, R x2, R x3, R& r) {
  r = sqrt_(x1 * x1 + x2 * x2 + x3 * x3);
  if (r == R(0)) return qidentity<R>();
  R top = x3 >= R(0) ? x3 + r : (x1 * x1 + x2 * x2) / (r - x3);
  R v1 = -x2, v2 = x1;
  R n2 = top * top + v1 * v1 + v2 * v2;
  if (n2 == R(0)) return {R(0), R(1), R(0), R(0)};
  R inv = R(1) / sqrt_(n2);
  return {top * inv, v1 * inv, v2 * inv, R(0)};
}

// MAG microcanonical step: the square of the maximiser above.  With h the
// rotation by the angle a between x and +z about an axis in the xy-plane,
// h^2 is the rotation by 2a, whose quaternion is (x3, -x2, x1, 0)/|x|; this
// form needs no half angles and loses no accuracy when x3 < 0.
template <typename R>
__device__ __forceinline__ quat<R> mag_micro(R x1, R x2, R x3, R r) {
  if (r == R(0)) return qidentity<R>();
  R inv = R(1) / r;
  return {x3 * inv, -x2 * inv, x1 * inv, R(0)};
}

// Kennedy-Pendleton heat bath for x0 ~ sqrt(1-x0^2) exp(alpha x0), at most
// KP_TRIALS trials (x0 = 1 if none is accepted); trials receives the number
// of trials used (0 if none was accepted).
template <typename R>
__device__ __forceinline__ R kp_sample(R alpha, const Rng& rng, uint32_t sub, int& trials) {
  for (int t = 0; t < KP_TRIALS; ++t) {
    double a1, a2, b1, b2;
    rng.draw2(TAG_SA, sub, (uint32_t)(2 * t), a1, a2);
    rng.draw2(TAG_SA, sub, (uint32_t)(2 * t + 1), b1, b2);
    R s, c;
    sincos2pi((R)a2, s, c);
    R delta = -(log_((R)a1) + c * c * log_((R)b1)) / (R(2) * alpha);
    R r4 = (R)b2;
    if (r4 * r4 <= R(1) - delta) {
      trials = t + 1;
      return R(1) - R(2) * delta;
    }
  }
  trials = 0;
  return R(1);
}

// Landau/Coulomb heat bath: g = h m/|m| with h0 from Kennedy-Pendleton at
// alpha = |m|/T and a uniform direction for the vector part.
template <typename R>
__device__ __forceinline__ quat<R> rule_sa_landau(quat<R> m, R T, const Rng& rng, uint32_t sub, int& trials) {
  R n2 = m.q0 * m.q0 + m.q1 * m.q1 + m.q2 * m.q2 + m.q3 * m.q3;
  trials = 1;
  if (n2 == R(0)) return qidentity<R>();
  R nm = sqrt_(n2);
  R x0 = kp_sample<R>(nm / T, rng, sub, trials);
  double ua, ub;
  rng.draw2(TAG_SA, sub, KP_DIR_DRAW, ua, ub);
  R cth = R(2) * (R)ua - R(1);
  R sth = sqrt_(fmax_(R(0), R(1) - cth * cth));
  R sp, cp;
  sincos2pi((R)ub, sp, cp);
  R rr = sqrt_(fmax_(R(0), R(1) - x0 * x0));
  quat<R> h{x0, rr * sth * cp, rr * sth * sp, rr * cth};
  R inv = R(1) / nm;
  quat<R> n{m.q0 * inv, m.q1 * inv, m.q2 * inv, m.q3 * inv};
  return qmul(h, n);
}

// MAG heat bath: cos(beta) ~ exp(kappa cos(beta)) by inversion, kappa = |x|/T,
// uniform azimuth; g = r h1 with h1 the maximiser and r the g3 = 0 rotation
// taking +z to the drawn direction.
template <typename R>
__device__ __forceinline__ quat<R> rule_sa_mag(quat<R> h1, R r, R T, const Rng& rng, uint32_t sub) {
  if (r == R(0)) return qidentity<R>();
  double ua, ub;
  rng.draw2(TAG_SA, sub, 0, ua, ub);
  R kappa = r / T;
  R cb = R(1) + log1p_((R)ua * expm1_(R(-2) * kappa)) / kappa;
  cb = fmin_(R(1), fmax_(R(-1), cb));
  R sp, cp;
  sincos2pi((R)ub, sp, cp);
  R ch = sqrt_(R(0.5) * (R(1) + cb)), sh = sqrt_(R(0.5) * (R(1) - cb));
  quat<R> rq{ch, sh * sp, -sh * cp, R(0)};
  return qmul(rq, h1);
}

// Haar-random SU(3) for one site (twelve Box-Muller normals on Philox draws,
// Gram-Schmidt of two complex rows, third row conj(row0 x row1)).
template <typename R>
__device__ __forceinline__ void haar_su3(const Rng& rng, mat3<R>& g) {
  R z[12];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double a, b;
    rng.draw2(TAG_HAAR, 0, (uint32_t)k, a, b);
    R r = sqrt_(R(-2) * log_((R)a));
    R s, c;
    sincos2pi((R)b, s, c);
    z[2 * k] = r * c;
    z[2 * k + 1] = r * s;
  }
  R na = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) na += z[2 * k] * z[2 * k] + z[2 * k + 1] * z[2 * k + 1];
  na = rsqrt_(na);
#pragma unroll
  for (int k = 0; k < 3; ++k) g.e[0][k] = {z[2 * k] * na, z[2 * k + 1] * na};
  // <row0, b> = sum conj(row0_k) b_k
  cx<R> ip{R(0), R(0)};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cx<R> b{z[6 + 2 * k], z[7 + 2 * k]};
    ip.re += g.e[0][k].re * b.re + g.e[0][k].im * b.im;
    ip.im += g.e[0][k].re * b.im - g.e[0][k].im * b.re;
  }
  R nb = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cx<R> b{z[6 + 2 * k], z[7 + 2 * k]};
    cx<R> p = cmul(ip, g.e[0][k]);
    g.e[1][k] = {b.re - p.re, b.im - p.im};
    nb += g.e[1][k].re * g.e[1][k].re + g.e[1][k].im * g.e[1][k].im;
  }
  nb = rsqrt_(nb);
#pragma unroll
  for (int k = 0; k < 3; ++k) g.e[1][k] = {g.e[1][k].re * nb, g.e[1][k].im * nb};
  reconstruct_row2(g);
}

// Re-projection of the two stored rows at load: row 0 normalised, row 1
// made orthogonal to it and normalised.  With 12-real storage the third row
// is rebuilt as conj(row0 x row1), and a subgroup rotation in (0,2) or (1,2)
// mixes it back into the stored rows: a norm error d0, d1 of the rows then
// grows as d0 -> d0 + sin^2 d1, i.e. exponentially under large rotations
// (heat bath, microcanonical steps, early sweeps), and rounding kicks
// accumulate in the rows' inner product.  Re-projecting at every load keeps
// the stored matrices unitary to rounding.
__device__ __forceinline__ float rnorm_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rnorm_(double x) { return 1.0 / sqrt(x); }
template <typename R>
__device__ __forceinline__ void reproject_rows(mat3<R>& u) {
  R n0 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) n0 += u.e[0][k].re * u.e[0][k].re + u.e[0][k].im * u.e[0][k].im;
  const R i0 = rnorm_(n0);
#pragma unroll
  for (int k = 0; k < 3; ++k) u.e[0][k] = {u.e[0][k].re * i0, u.e[0][k].im * i0};
  cx<R> ip{R(0), R(0)};  // <row0, row1>
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ip.re += u.e[0][k].re * u.e[1][k].re + u.e[0][k].im * u.e[1][k].im;
    ip.im += u.e[0][k].re * u.e[1][k].im - u.e[0][k].im * u.e[1][k].re;
  }
  R n1 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cx<R> p = cmul(ip, u.e[0][k]);
    u.e[1][k] = {u.e[1][k].re - p.re, u.e[1][k].im - p.im};
    n1 += u.e[1][k].re * u.e[1][k].re + u.e[1][k].im * u.e[1][k].im;
  }
  const R i1 = rnorm_(n1);
#pragma unroll
  for (int k = 0; k < 3; ++k) u.e[1][k] = {u.e[1][k].re * i1, u.e[1][k].im * i1};
}

// Re-unitarisation: normalise row 0, Gram-Schmidt row 1 against it,
// normalise (the third row stays implicit).
template <typename R>
__device__ __forceinline__ void gram_schmidt_rows(mat3<R>& u) {
  R na = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) na += u.e[0][k].re * u.e[0][k].re + u.e[0][k].im * u.e[0][k].im;
  na = R(1) / sqrt_(na);
#pragma unroll
  for (int k = 0; k < 3; ++k) u.e[0][k] = {u.e[0][k].re * na, u.e[0][k].im * na};
  cx<R> ip{R(0), R(0)};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ip.re += u.e[0][k].re * u.e[1][k].re + u.e[0][k].im * u.e[1][k].im;
    ip.im += u.e[0][k].re * u.e[1][k].im - u.e[0][k].im * u.e[1][k].re;
  }
  R nb = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cx<R> p = cmul(ip, u.e[0][k]);
    u.e[1][k] = {u.e[1][k].re - p.re, u.e[1][k].im - p.im};
    nb += u.e[1][k].re * u.e[1][k].re + u.e[1][k].im * u.e[1][k].im;
  }
  nb = R(1) / sqrt_(nb);
#pragma unroll
  for (int k = 0; k < 3; ++k) u.e[1][k] = {u.e[1][k].re * nb, u.e[1][k].im * nb};
}

}  // namespace gfk
