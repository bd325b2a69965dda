// su3_device.cuh -- device arithmetic for the checkerboard SU(3) heatbath:
// complex 3x3 algebra, link storage formats, Philox4x32-10, the
// Kennedy-Pendleton SU(2) draw and the Cabibbo-Marinari link update.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "su3_engine.h"

namespace su3g {

// ------------------------------------------------------------------ debug bounds checks
// Built with SU3_DEBUG_BOUNDS, every link access and every scratch index is
// checked against its extent before the access.  The first violation is
// recorded in g_bounds (site code, index, extent) and the access is skipped
// (a load gives zeros); nothing traps, so the context stays usable and the
// host reports the violation (su3_bounds_status, su3_synchronize).  Without
// the flag the checks compile to nothing.
#ifdef SU3_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds[3];
#endif
enum BoundsSite : unsigned {
  kBoundsPlane = 1,    // (layer, colour, direction) of a link plane
  kBoundsIndex = 2,    // checkerboard index within a plane
  kBoundsLink = 3,     // plane offset of a precomputed link index
  kBoundsPartial = 4,  // measurement partial-sum slot
  kBoundsSlot = 5,     // action bookkeeping slot
  kBoundsSelfTest = 9  // the self-test's deliberate out-of-range index (never accessed)
};

__device__ __forceinline__ bool in_bounds(long long i, long long n, unsigned site) {
#ifdef SU3_DEBUG_BOUNDS
  if (i >= 0 && i < n) return true;
  if (atomicCAS(&g_bounds[0], 0ull, (unsigned long long)site) == 0ull) {
    g_bounds[1] = (unsigned long long)i;
    g_bounds[2] = (unsigned long long)n;
  }
  return false;
#else
  (void)i;
  (void)n;
  (void)site;
  return true;
#endif
}

// ------------------------------------------------------------------ complex 3x3

template <typename R>
struct C {
  R re, im;
};

template <typename R>
struct M3 {
  C<R> e[3][3];
};

template <typename R>
__device__ __forceinline__ M3<R> m3_zero() {
  M3<R> m;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m.e[i][j] = {R(0), R(0)};
  return m;
}

// Fused multiply-add in the working precision.  The complex algebra below
// is written as explicit FMA chains: `s += a*b - c*d` would otherwise be
// compiled as FMUL + FFMA + FADD (C semantics forbid the reassociation).
__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fm(double a, double b, double c) { return __fma_rn(a, b, c); }

// s += a b
template <typename R>
__device__ __forceinline__ void cmac(C<R> &s, const C<R> &a, const C<R> &b) {
  s.re = fm(a.re, b.re, s.re);
  s.re = fm(-a.im, b.im, s.re);
  s.im = fm(a.re, b.im, s.im);
  s.im = fm(a.im, b.re, s.im);
}
// s += a conj(b)
template <typename R>
__device__ __forceinline__ void cmac_nc(C<R> &s, const C<R> &a, const C<R> &b) {
  s.re = fm(a.re, b.re, s.re);
  s.re = fm(a.im, b.im, s.re);
  s.im = fm(a.im, b.re, s.im);
  s.im = fm(-a.re, b.im, s.im);
}
// s += conj(a) b
template <typename R>
__device__ __forceinline__ void cmac_cn(C<R> &s, const C<R> &a, const C<R> &b) {
  s.re = fm(a.re, b.re, s.re);
  s.re = fm(a.im, b.im, s.re);
  s.im = fm(a.re, b.im, s.im);
  s.im = fm(-a.im, b.re, s.im);
}
template <typename R>
__device__ __forceinline__ C<R> cmul(const C<R> &a, const C<R> &b) {
  return {fm(-a.im, b.im, a.re * b.re), fm(a.im, b.re, a.re * b.im)};
}
template <typename R>
__device__ __forceinline__ C<R> cmul_nc(const C<R> &a, const C<R> &b) {
  return {fm(a.im, b.im, a.re * b.re), fm(-a.re, b.im, a.im * b.re)};
}
template <typename R>
__device__ __forceinline__ C<R> cmul_cn(const C<R> &a, const C<R> &b) {
  return {fm(a.im, b.im, a.re * b.re), fm(-a.im, b.re, a.re * b.im)};
}

// c = a b (rows 0..NR-1)
template <int NR = 3, typename R>
__device__ __forceinline__ M3<R> mul_nn(const M3<R> &a, const M3<R> &b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C<R> s = cmul(a.e[i][0], b.e[0][j]);
      cmac(s, a.e[i][1], b.e[1][j]);
      cmac(s, a.e[i][2], b.e[2][j]);
      c.e[i][j] = s;
    }
  return c;
}

// c = a b^+ (rows 0..NR-1)
template <int NR = 3, typename R>
__device__ __forceinline__ M3<R> mul_nd(const M3<R> &a, const M3<R> &b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C<R> s = cmul_nc(a.e[i][0], b.e[j][0]);
      cmac_nc(s, a.e[i][1], b.e[j][1]);
      cmac_nc(s, a.e[i][2], b.e[j][2]);
      c.e[i][j] = s;
    }
  return c;
}

// c = a^+ b (rows 0..NR-1)
template <int NR = 3, typename R>
__device__ __forceinline__ M3<R> mul_dn(const M3<R> &a, const M3<R> &b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C<R> s = cmul_cn(a.e[0][i], b.e[0][j]);
      cmac_cn(s, a.e[1][i], b.e[1][j]);
      cmac_cn(s, a.e[2][i], b.e[2][j]);
      c.e[i][j] = s;
    }
  return c;
}

// Two-row forms: a product of SU(3) factors is SU(3), so only rows 0, 1 are
// computed and row 2 is completed by third_row (24 FMA instead of 36).
template <typename R>
__device__ __forceinline__ M3<R> mul_nn_2(const M3<R> &a, const M3<R> &b) { return mul_nn<2>(a, b); }
template <typename R>
__device__ __forceinline__ M3<R> mul_nd_2(const M3<R> &a, const M3<R> &b) { return mul_nd<2>(a, b); }
template <typename R>
__device__ __forceinline__ M3<R> mul_dn_2(const M3<R> &a, const M3<R> &b) { return mul_dn<2>(a, b); }

// conj(p q - r s)
template <typename R>
__device__ __forceinline__ C<R> conj_cross(const C<R> &p, const C<R> &q, const C<R> &r, const C<R> &s) {
  R re = p.re * q.re;
  re = fm(-p.im, q.im, re);
  re = fm(-r.re, s.re, re);
  re = fm(r.im, s.im, re);
  R im = -(p.re * q.im);
  im = fm(-p.im, q.re, im);
  im = fm(r.re, s.im, im);
  im = fm(r.im, s.re, im);
  return {re, im};
}

// Third row of an SU(3) matrix from the first two: conj(row1 x row2).
template <typename R>
__device__ __forceinline__ void third_row(M3<R> &m) {
  const C<R> *a = m.e[0], *b = m.e[1];
  m.e[2][0] = conj_cross(a[1], b[2], a[2], b[1]);
  m.e[2][1] = conj_cross(a[2], b[0], a[0], b[2]);
  m.e[2][2] = conj_cross(a[0], b[1], a[1], b[0]);
}

// A += m for an SU(3) matrix m given by rows 0, 1: row 2 of m is
// accumulated straight from the cross product.
template <typename R>
__device__ __forceinline__ void acc_su3_2rows(M3<R> &A, const M3<R> &m) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.e[i][j].re += m.e[i][j].re;
      A.e[i][j].im += m.e[i][j].im;
    }
  const C<R> *a = m.e[0], *b = m.e[1];
  const int P[3][4] = {{1, 2, 2, 1}, {2, 0, 0, 2}, {0, 1, 1, 0}};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const C<R> &p = a[P[j][0]], &q = b[P[j][1]], &r = a[P[j][2]], &t = b[P[j][3]];
    // A_2j += conj(p q - r t)
    R re = fm(p.re, q.re, A.e[2][j].re);
    re = fm(-p.im, q.im, re);
    re = fm(-r.re, t.re, re);
    re = fm(r.im, t.im, re);
    R im = fm(-p.re, q.im, A.e[2][j].im);
    im = fm(-p.im, q.re, im);
    im = fm(r.re, t.im, im);
    im = fm(r.im, t.re, im);
    A.e[2][j] = {re, im};
  }
}

// ------------------------------------------------------------------ float <-> double by bits
// On this GPU the FP64 pipe also executes the float <-> double conversion
// instructions, and in the FP64 stages (re-unitarisation) that pipe is the
// bottleneck.  These two conversions move the IEEE-754 fields with integer
// operations instead (sign; exponent rebias 1023 - 127 = 896; mantissa
// shifted by 52 - 23 = 29 bits), bit for bit the round-to-nearest-even
// conversions for every normal input.  Subnormal values (below 2^-126 in
// magnitude) flush to signed zero; infinities and NaNs are preserved.

__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sg = u & 0x80000000u, a = u & 0x7FFFFFFFu, e = u & 0x7F800000u;
  uint32_t hi = sg | ((a >> 3) + (896u << 20));
  hi = e == 0x7F800000u ? (sg | 0x7FF00000u | ((a >> 3) & 0x000FFFFFu)) : hi;
  hi = e == 0u ? sg : hi;
  const uint32_t lo = e == 0u ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_bits(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t sg = hi & 0x80000000u, a = hi & 0x7FFFFFFFu;
  // in range: double exponent 897..1150 (float exponent 1..254); the
  // 29 dropped mantissa bits decide the rounding, ties to even; a carry
  // out of the mantissa steps the exponent (to infinity above the range)
  uint32_t f = ((a - (896u << 20)) << 3) | (lo >> 29);
  const uint32_t r = lo & 0x1FFFFFFFu;
  f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
  f = a < (897u << 20) ? 0u : f;
  const bool nan = a > 0x7FF00000u || (a == 0x7FF00000u && lo != 0u);
  f = a >= (1151u << 20) ? (nan ? 0x7FC00000u : 0x7F800000u) : f;
  return __uint_as_float(sg | f);
}

// 1/sqrt(n) in double: a float seed refined by NEWTON Newton steps,
// y <- y (3 - n y^2) / 2; each roughly squares the relative error
// (~2e-7 -> ~1e-13 -> rounding level).  One step is ample for links stored
// in FP32 (rounded to ~6e-8 afterwards), two reach double rounding.
template <int NEWTON = 2>
__device__ __forceinline__ double rsqrt_d(double n) {
  double y = f2d_bits(rsqrtf(d2f_bits(n)));
  const double h = 0.5 * n;
#pragma unroll
  for (int k = 0; k < NEWTON; ++k) y = y * __fma_rn(-h * y, y, 1.5);
  return y;
}

// Gram-Schmidt of rows 1, 2 in double, row 3 from the cross product
// (ROW3 = false: rows 1, 2 only, for storage that keeps two rows).  Written
// as explicit FMA chains: FP64 is the scarce pipe on this GPU, and
// `s += a*b + c*d` would cost a multiply, an FMA and an add.
template <int NEWTON = 2, bool ROW3 = true>
__device__ __forceinline__ void reunit_d(M3<double> &m) {
  C<double> *r1 = m.e[0], *r2 = m.e[1];
  double n1 = r1[0].re * r1[0].re;
  n1 = fm(r1[0].im, r1[0].im, n1);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    n1 = fm(r1[k].re, r1[k].re, n1);
    n1 = fm(r1[k].im, r1[k].im, n1);
  }
  const double i1 = rsqrt_d<NEWTON>(n1);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r1[k].re *= i1;
    r1[k].im *= i1;
  }
  // <r1, r2> = sum_k conj(r1_k) r2_k
  double pr = r1[0].re * r2[0].re, pi = r1[0].re * r2[0].im;
  pr = fm(r1[0].im, r2[0].im, pr);
  pi = fm(-r1[0].im, r2[0].re, pi);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    pr = fm(r1[k].re, r2[k].re, pr);
    pr = fm(r1[k].im, r2[k].im, pr);
    pi = fm(r1[k].re, r2[k].im, pi);
    pi = fm(-r1[k].im, r2[k].re, pi);
  }
  // r2 -= <r1, r2> r1
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double re = r1[k].re, im = r1[k].im;
    r2[k].re = fm(-pr, re, fm(pi, im, r2[k].re));
    r2[k].im = fm(-pr, im, fm(-pi, re, r2[k].im));
  }
  double n2 = r2[0].re * r2[0].re;
  n2 = fm(r2[0].im, r2[0].im, n2);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    n2 = fm(r2[k].re, r2[k].re, n2);
    n2 = fm(r2[k].im, r2[k].im, n2);
  }
  const double i2 = rsqrt_d<NEWTON>(n2);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r2[k].re *= i2;
    r2[k].im *= i2;
  }
  if constexpr (ROW3) third_row(m);
}

// A double-precision link in the storage precision R (float: by bits).
template <typename R>
__device__ __forceinline__ M3<R> to_storage(const M3<double> &b) {
  M3<R> a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if constexpr (sizeof(R) == 4)
        a.e[i][j] = {d2f_bits(b.e[i][j].re), d2f_bits(b.e[i][j].im)};
      else
        a.e[i][j] = {b.e[i][j].re, b.e[i][j].im};
    }
  return a;
}

template <typename A, typename B>
__device__ __forceinline__ M3<A> m3_cast(const M3<B> &b) {
  M3<A> a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a.e[i][j] = {A(b.e[i][j].re), A(b.e[i][j].im)};
  return a;
}

// A += w m for an SU(3) matrix m given by rows 0, 1 (row 2 from the cross
// product), w a real weight (a plaquette's coupling).
template <typename R>
__device__ __forceinline__ void acc_su3_2rows_w(M3<R> &A, const M3<R> &m, R w) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.e[i][j].re = fm(w, m.e[i][j].re, A.e[i][j].re);
      A.e[i][j].im = fm(w, m.e[i][j].im, A.e[i][j].im);
    }
  const C<R> *a = m.e[0], *b = m.e[1];
  const C<R> r2[3] = {conj_cross(a[1], b[2], a[2], b[1]), conj_cross(a[2], b[0], a[0], b[2]),
                      conj_cross(a[0], b[1], a[1], b[0])};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    A.e[2][j].re = fm(w, r2[j].re, A.e[2][j].re);
    A.e[2][j].im = fm(w, r2[j].im, A.e[2][j].im);
  }
}

// ------------------------------------------------------------------ storage
//
// Links of one chain: Vec planes [layer][colour][mu][q][jj], jj the
// checkerboard index (i_s - 1) / 2 of the site within its layer, so a warp
// of consecutive sites reads each q-vector as one contiguous line (512
// bytes of 128-bit loads; the float2 plane of the 18-real float form 256).

// Every form has load (3 rows), load2 (rows 1, 2; row 3 left unset), store
// and copy (one link between two planes, for halo and box copies).

struct StoreF32x12 {
  using R = float;
  using Vec = float4;
  static constexpr int NQ = 3;  // rows 1, 2: six complex numbers
  static constexpr bool kTwoRows = true;
  // rows 0, 1 only (row 2 left unset)
  __device__ static __forceinline__ M3<float> load2(const Vec *plane, int Vh, int jj) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return m3_zero<float>();
    const Vec *p = plane + jj;
    const float4 q0 = __ldg(p), q1 = __ldg(p + Vh), q2 = __ldg(p + 2 * Vh);
    M3<float> m;
    m.e[0][0] = {q0.x, q0.y};
    m.e[0][1] = {q0.z, q0.w};
    m.e[0][2] = {q1.x, q1.y};
    m.e[1][0] = {q1.z, q1.w};
    m.e[1][1] = {q2.x, q2.y};
    m.e[1][2] = {q2.z, q2.w};
    return m;
  }
  __device__ static __forceinline__ M3<float> load(const Vec *plane, int Vh, int jj) {
    M3<float> m = load2(plane, Vh, jj);
    third_row(m);
    return m;
  }
  __device__ static __forceinline__ void store(Vec *plane, int Vh, int jj, const M3<float> &m) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return;
    Vec *p = plane + jj;
    p[0] = make_float4(m.e[0][0].re, m.e[0][0].im, m.e[0][1].re, m.e[0][1].im);
    p[Vh] = make_float4(m.e[0][2].re, m.e[0][2].im, m.e[1][0].re, m.e[1][0].im);
    p[2 * Vh] = make_float4(m.e[1][1].re, m.e[1][1].im, m.e[1][2].re, m.e[1][2].im);
  }
  __device__ static __forceinline__ void copy(Vec *dst, int dVh, int dj, const Vec *src, int sVh, int sj) {
    if (!(in_bounds(dj, dVh, kBoundsIndex) && in_bounds(sj, sVh, kBoundsIndex))) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) dst[(size_t)q * dVh + dj] = src[(size_t)q * sVh + sj];
  }
};

// All 18 reals in float: the 12-real planes (rows 1, 2 as three 128-bit
// vectors) followed by row 3 as one 128-bit and one 64-bit vector.  In units
// of Vec = float2 a (layer, colour, mu) plane group spans 9 Vh: float4 plane
// k (k = 0..3) starts at 2 k Vh, the float2 plane at 8 Vh.  Plane groups
// start on 16-byte boundaries because Vh is even (all extents are even).
// Loads of rows 1, 2 are those of the 12-real form; row 3 costs two more
// loads instead of the cross product.
struct StoreF32x18 {
  using R = float;
  using Vec = float2;
  static constexpr int NQ = 9;  // float2 units per link
  static constexpr bool kTwoRows = false;
  __device__ static __forceinline__ M3<float> load2(const Vec *plane, int Vh, int jj) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return m3_zero<float>();
    const float4 *p = reinterpret_cast<const float4 *>(plane) + jj;
    const float4 q0 = __ldg(p), q1 = __ldg(p + Vh), q2 = __ldg(p + 2 * Vh);
    M3<float> m;
    m.e[0][0] = {q0.x, q0.y};
    m.e[0][1] = {q0.z, q0.w};
    m.e[0][2] = {q1.x, q1.y};
    m.e[1][0] = {q1.z, q1.w};
    m.e[1][1] = {q2.x, q2.y};
    m.e[1][2] = {q2.z, q2.w};
    return m;
  }
  __device__ static __forceinline__ M3<float> load(const Vec *plane, int Vh, int jj) {
    M3<float> m = load2(plane, Vh, jj);
    if (!in_bounds(jj, Vh, kBoundsIndex)) return m;
    const float4 q3 = __ldg(reinterpret_cast<const float4 *>(plane) + 3 * Vh + jj);
    const float2 q4 = __ldg(plane + 8 * Vh + jj);
    m.e[2][0] = {q3.x, q3.y};
    m.e[2][1] = {q3.z, q3.w};
    m.e[2][2] = {q4.x, q4.y};
    return m;
  }
  __device__ static __forceinline__ void store(Vec *plane, int Vh, int jj, const M3<float> &m) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return;
    float4 *p = reinterpret_cast<float4 *>(plane) + jj;
    p[0] = make_float4(m.e[0][0].re, m.e[0][0].im, m.e[0][1].re, m.e[0][1].im);
    p[Vh] = make_float4(m.e[0][2].re, m.e[0][2].im, m.e[1][0].re, m.e[1][0].im);
    p[2 * Vh] = make_float4(m.e[1][1].re, m.e[1][1].im, m.e[1][2].re, m.e[1][2].im);
    p[3 * Vh] = make_float4(m.e[2][0].re, m.e[2][0].im, m.e[2][1].re, m.e[2][1].im);
    plane[8 * Vh + jj] = make_float2(m.e[2][2].re, m.e[2][2].im);
  }
  __device__ static __forceinline__ void copy(Vec *dst, int dVh, int dj, const Vec *src, int sVh, int sj) {
    if (!(in_bounds(dj, dVh, kBoundsIndex) && in_bounds(sj, sVh, kBoundsIndex))) return;
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int k = 0; k < 4; ++k) d4[(size_t)k * dVh + dj] = s4[(size_t)k * sVh + sj];
    dst[(size_t)8 * dVh + dj] = src[(size_t)8 * sVh + sj];
  }
};

struct StoreF64x18 {
  using R = double;
  using Vec = double2;
  static constexpr int NQ = 9;  // one complex number per 128-bit vector
  static constexpr bool kTwoRows = false;
  __device__ static __forceinline__ M3<double> load(const Vec *plane, int Vh, int jj) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return m3_zero<double>();
    const Vec *p = plane + jj;
    M3<double> m;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const double2 v = __ldg(p + q * Vh);
      m.e[q / 3][q % 3] = {v.x, v.y};
    }
    return m;
  }
  __device__ static __forceinline__ M3<double> load2(const Vec *plane, int Vh, int jj) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return m3_zero<double>();
    const Vec *p = plane + jj;
    M3<double> m;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double2 v = __ldg(p + q * Vh);
      m.e[q / 3][q % 3] = {v.x, v.y};
    }
    return m;
  }
  __device__ static __forceinline__ void store(Vec *plane, int Vh, int jj, const M3<double> &m) {
    if (!in_bounds(jj, Vh, kBoundsIndex)) return;
    Vec *p = plane + jj;
#pragma unroll
    for (int q = 0; q < 9; ++q) p[q * Vh] = make_double2(m.e[q / 3][q % 3].re, m.e[q / 3][q % 3].im);
  }
  __device__ static __forceinline__ void copy(Vec *dst, int dVh, int dj, const Vec *src, int sVh, int sj) {
    if (!(in_bounds(dj, dVh, kBoundsIndex) && in_bounds(sj, sVh, kBoundsIndex))) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) dst[(size_t)q * dVh + dj] = src[(size_t)q * sVh + sj];
  }
};

// The (layer, colour, mu) plane of a chain's links.  Offsets stay in 32 bits
// (the host rejects chains with 2^31 vectors or more).
template <class S>
__device__ __forceinline__ typename S::Vec *plane_ptr(const ChainDesc &d, int layer, int colour, int mu) {
  typename S::Vec *base = reinterpret_cast<typename S::Vec *>(d.links);
  // (virtual) layers: nlayers x nb sublattice boxes (nb = 1 undivided)
  if (!(in_bounds(layer, d.nlayers * d.nb, kBoundsPlane) && in_bounds(colour, 2, kBoundsPlane) &&
        in_bounds(mu, d.D, kBoundsPlane)))
    return base;
  return base + ((layer * 2 + colour) * d.D + mu) * (S::NQ * d.Vh);
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC11): ten rounds; round constants
// 0xD2511F53 / 0xCD9E8D57, key increments 0x9E3779B9 / 0xBB67AE85.

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniforms (w + 1/2) / 2^32 in (0,1].  In float the word is rounded to 24
// bits first, which keeps ln(u) within ~6e-8 of the double value for every
// u (truncating to the top 24 bits instead would quantise u near 0 and make
// ln(u) there far less accurate).  u can round up to 1.0f, where ln(u) = 0.
__device__ __forceinline__ float unif_f(uint32_t w) { return __fmaf_rn(__uint2float_rn(w), 0x1p-32f, 0x1p-33f); }
__device__ __forceinline__ double unif_d(uint32_t w) { return __fma_rn((double)w, 0x1p-32, 0x1p-33); }

// Approximate (SFU) square root and reciprocal for the FP32 draw: their
// relative errors (a few 1e-7) stay inside the FP32 rounding of the link.
// sqrt.approx of 0 is 0.
__device__ __forceinline__ float sqrt_sfu(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_sfu(float x) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// |a| and 1/|a| of the projection: IEEE sqrt and division in double; in
// float one SFU reciprocal square root gives both.
__device__ __forceinline__ void norm_and_inverse(double n, double &k, double &ik) {
  k = sqrt(n);
  ik = 1.0 / k;
}
__device__ __forceinline__ void norm_and_inverse(float n, float &k, float &ik) {
  float r;
  asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(n));
  ik = r;
  k = n * r;
}

__device__ __forceinline__ uint32_t heatbath_tag(int colour, int mu, int subgroup) {
  return ((uint32_t)subgroup << 8) | ((uint32_t)mu << 10) | ((uint32_t)colour << 14);
}

// The two uniforms of a subgroup's direction are two words of a direction
// block: subgroups 0 and 1 share the block of subgroup 0 (words x, y and
// z, w), subgroup 2 takes words x, y of its own.  Five blocks per link
// update when every first proposal is accepted, not six.
__device__ __forceinline__ uint2 direction_words(uint2 key, uint32_t c0, uint32_t c1, uint32_t tag) {
  const uint32_t sg = (tag >> 8) & 3u;
  const uint32_t block_tag = (tag & ~(3u << 8)) | ((sg & 2u) << 8) | kHitDirection;
  const uint4 v = philox4x32_10(make_uint4(c0, c1, block_tag, kPurposeHeatbath), key);
  return sg == 1 ? make_uint2(v.z, v.w) : make_uint2(v.x, v.y);
}

// ------------------------------------------------------------------ SU(2) heatbath
// Kennedy-Pendleton with the Fredenhagen-Marcu hit limit: per hit
// X = -(ln u1 + cos^2(2 pi u2) ln u3) / alpha, accepted when
// u4^2 <= 1 - X/2; x0 = 1 - X and (x1, x2, x3) isotropic with length
// sqrt(X (2 - X)).  Returns false (subgroup kept) after `hits` rejections.

__device__ __forceinline__ bool su2_draw_d(double alpha, int hits, uint2 key, uint32_t c0, uint32_t c1,
                                           uint32_t tag, double x[4], uint32_t &nprop) {
  double X = 0.0;
  bool acc = false;
  for (int h = 0; h < hits; ++h) {
    const uint4 w = philox4x32_10(make_uint4(c0, c1, tag | (uint32_t)h, kPurposeHeatbath), key);
    ++nprop;
    const double cs = cospi(2.0 * unif_d(w.y));
    X = -(log(unif_d(w.x)) + cs * cs * log(unif_d(w.z))) / alpha;
    const double u4 = unif_d(w.w);
    if (u4 * u4 <= 1.0 - 0.5 * X) {
      acc = true;
      break;
    }
  }
  if (!acc) return false;
  const uint2 w = direction_words(key, c0, c1, tag);
  const double costh = 2.0 * unif_d(w.x) - 1.0;
  const double sinth = sqrt(1.0 - costh * costh);
  double sphi, cphi;
  sincospi(2.0 * unif_d(w.y), &sphi, &cphi);
  const double rho = sqrt(X * (2.0 - X));
  x[0] = 1.0 - X;
  x[1] = rho * sinth * cphi;
  x[2] = rho * sinth * sphi;
  x[3] = rho * costh;
  return true;
}

__device__ __forceinline__ bool su2_draw(double alpha, int hits, uint2 key, uint32_t c0, uint32_t c1, uint32_t tag,
                                         double x[4], uint32_t &nprop) {
  return su2_draw_d(alpha, hits, key, c0, c1, tag, x, nprop);
}

// ln u of the uniform (w + 1/2) / 2^32, accurate relative to ln u for
// every word: for u above 1/2 from the exact small complement,
// ln u = log1p(-(2^32 - 1 - w + 1/2) / 2^32), so that u near 1 keeps its
// digits (the float u itself is quantised there to ~6e-8).
__device__ __forceinline__ float log_unif_accurate(uint32_t w) {
  if (w & 0x80000000u) return log1pf(-__fmaf_rn(__uint2float_rn(0xFFFFFFFFu - w), 0x1p-32f, 0x1p-33f));
  return logf(unif_f(w));
}

// The float draw.  ACCURATE = false: the SFU forms of ln and cos, whose
// absolute errors (~3.6e-7 for ln on [0.5, 1], ~4e-7 for cos on [-pi, pi])
// enter X = -(ln u1 + cos^2 ln u3) / alpha divided by alpha: inside the FP32
// storage rounding for alpha >= 2.  ACCURATE = true (small alpha, strong
// coupling): cosf and a logarithm accurate relative to ln u even for u near
// 1 (log_unif_accurate), which keep X to ~1e-7 relative for any alpha.  Angles 2 pi u are taken as 2 pi (u - 1/2) - the sign flip
// is absorbed - to stay on [-pi, pi].
template <bool ACCURATE>
__device__ __forceinline__ bool su2_draw_f(float alpha, int hits, uint2 key, uint32_t c0, uint32_t c1, uint32_t tag,
                                           float x[4], uint32_t &nprop) {
  float X = 0.0f;
  bool acc = false;
  const float ia = rcp_sfu(alpha);
  for (int h = 0; h < hits; ++h) {
    const uint4 w = philox4x32_10(make_uint4(c0, c1, tag | (uint32_t)h, kPurposeHeatbath), key);
    ++nprop;
    const float ang = __fmaf_rn(unif_f(w.y), 6.28318530717958648f, -3.14159265358979324f);
    const float cs = ACCURATE ? cosf(ang) : __cosf(ang);
    const float l1 = ACCURATE ? log_unif_accurate(w.x) : __logf(unif_f(w.x));
    const float l3 = ACCURATE ? log_unif_accurate(w.z) : __logf(unif_f(w.z));
    X = -(l1 + cs * cs * l3) * ia;
    const float u4 = unif_f(w.w);
    if (u4 * u4 <= 1.0f - 0.5f * X) {
      acc = true;
      break;
    }
  }
  if (!acc) return false;
  const uint2 w = direction_words(key, c0, c1, tag);
  const float costh = 2.0f * unif_f(w.x) - 1.0f;
  const float sinth = sqrt_sfu(1.0f - costh * costh);
  float sphi, cphi;
  __sincosf(__fmaf_rn(unif_f(w.y), 6.28318530717958648f, -3.14159265358979324f), &sphi, &cphi);
  sphi = -sphi;  // sin(2 pi u) = -sin(2 pi (u - 1/2)), likewise cos
  cphi = -cphi;
  const float rho = sqrt_sfu(X * (2.0f - X));
  x[0] = 1.0f - X;
  x[1] = rho * sinth * cphi;
  x[2] = rho * sinth * sphi;
  x[3] = rho * costh;
  return true;
}

__device__ __forceinline__ bool su2_draw(float alpha, int hits, uint2 key, uint32_t c0, uint32_t c1, uint32_t tag,
                                         float x[4], uint32_t &nprop) {
  if (alpha >= kAlphaFp64) {
    double xd[4];
    const bool a = su2_draw_d((double)alpha, hits, key, c0, c1, tag, xd, nprop);
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = (float)xd[i];
    return a;
  }
  if (alpha < kAlphaAccurateLog) return su2_draw_f<true>(alpha, hits, key, c0, c1, tag, x, nprop);
  return su2_draw_f<false>(alpha, hits, key, c0, c1, tag, x, nprop);
}

// ------------------------------------------------------------------ Cabibbo-Marinari
// W = U A; for the subgroups (1,2), (1,3), (2,3): project the 2x2 block of
// W on the quaternions a, k = |a|, alpha = 2 beta k / 3, draw x from
// exp(alpha x0), r = x v^+ with v = a / k, and rotate rows i, j of U and W
// by r.  Weight exp((beta/3) Re Tr(U A)).

template <typename R>
__device__ __forceinline__ void rotate_rows(M3<R> &m, int i, int j, R r0, R r1, R r2, R r3) {
  // r = [[r0 + i r3, r2 + i r1], [-r2 + i r1, r0 - i r3]]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const C<R> a = m.e[i][c], b = m.e[j][c];
    m.e[i][c] = {r0 * a.re - r3 * a.im + r2 * b.re - r1 * b.im, r0 * a.im + r3 * a.re + r2 * b.im + r1 * b.re};
    m.e[j][c] = {-r2 * a.re - r1 * a.im + r0 * b.re + r3 * b.im, -r2 * a.im + r1 * a.re + r0 * b.im - r3 * b.re};
  }
}

// The quaternion projection a of the (i, j) block of W = U A, taken from
// the current (already rotated) U and the staple sum A: four sums of six
// products each.  a0 = Re(w_ii + w_jj)/2, a1 = Im(w_ij + w_ji)/2,
// a2 = Re(w_ij - w_ji)/2, a3 = Im(w_ii - w_jj)/2 with w_ab = sum_k U_ak A_kb.
template <typename R>
__device__ __forceinline__ void block_projection(const M3<R> &U, const M3<R> &A, int i, int j, R &a0, R &a1, R &a2,
                                                 R &a3) {
  R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const C<R> ui = U.e[i][k], uj = U.e[j][k], ai = A.e[k][i], aj = A.e[k][j];
    // Re(u_ik a_ki + u_jk a_kj)
    s0 = fm(ui.re, ai.re, s0);
    s0 = fm(-ui.im, ai.im, s0);
    s0 = fm(uj.re, aj.re, s0);
    s0 = fm(-uj.im, aj.im, s0);
    // Im(u_ik a_kj + u_jk a_ki)
    s1 = fm(ui.re, aj.im, s1);
    s1 = fm(ui.im, aj.re, s1);
    s1 = fm(uj.re, ai.im, s1);
    s1 = fm(uj.im, ai.re, s1);
    // Re(u_ik a_kj - u_jk a_ki)
    s2 = fm(ui.re, aj.re, s2);
    s2 = fm(-ui.im, aj.im, s2);
    s2 = fm(-uj.re, ai.re, s2);
    s2 = fm(uj.im, ai.im, s2);
    // Im(u_ik a_ki - u_jk a_kj)
    s3 = fm(ui.re, ai.im, s3);
    s3 = fm(ui.im, ai.re, s3);
    s3 = fm(-uj.re, aj.im, s3);
    s3 = fm(-uj.im, aj.re, s3);
  }
  a0 = R(0.5) * s0;
  a1 = R(0.5) * s1;
  a2 = R(0.5) * s2;
  a3 = R(0.5) * s3;
}

// dretr (out): the change of Re Tr(U A) = Re Tr W.  An accepted subgroup
// replaces Re(w_ii + w_jj) = 2 a0 = 2 k v0 by 2 k x0 and leaves the third
// diagonal element alone, so the change is the sum of 2 (k x0 - a0).
// W itself is never formed: each subgroup projects the block of the current
// U times A (block_projection), which equals the block of the rotated W.
template <typename R>
__device__ __forceinline__ void cm_update(M3<R> &U, const M3<R> &A, R beta, int hits, uint2 key, uint32_t c0,
                                          uint32_t c1, int colour, int mu, uint32_t &nprop, uint32_t &nacc,
                                          R &dretr) {
  dretr = R(0);
  const R ca = R(2) * beta / R(3);  // alpha = (2 beta / 3) k
#pragma unroll
  for (int sg = 0; sg < 3; ++sg) {
    const int i = (sg == 2) ? 1 : 0;
    const int j = (sg == 0) ? 1 : 2;
    R a0, a1, a2, a3;
    block_projection(U, A, i, j, a0, a1, a2, a3);
    R k, ik;
    norm_and_inverse(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3, k, ik);
    if (!(k > (sizeof(R) == 4 ? R(1e-30) : R(1e-300)))) continue;
    const R alpha = ca * k;
    R x[4];
    if (!su2_draw(alpha, hits, key, c0, c1, heatbath_tag(colour, mu, sg), x, nprop)) continue;
    ++nacc;
    dretr += R(2) * (k * x[0] - a0);
    const R v0 = a0 * ik, v1 = a1 * ik, v2 = a2 * ik, v3 = a3 * ik;
    // r = x v^+ as quaternions: r0 = x0 v0 + x.v, r = -x0 v + v0 x + x cross v
    const R r0 = x[0] * v0 + x[1] * v1 + x[2] * v2 + x[3] * v3;
    const R r1 = -x[0] * v1 + v0 * x[1] + (x[2] * v3 - x[3] * v2);
    const R r2 = -x[0] * v2 + v0 * x[2] + (x[3] * v1 - x[1] * v3);
    const R r3 = -x[0] * v3 + v0 * x[3] + (x[1] * v2 - x[2] * v1);
    rotate_rows(U, i, j, r0, r1, r2, r3);
  }
}

// ------------------------------------------------------------------ Cabibbo-Marinari, float, draws first
// The random numbers of the first proposal and of the direction of every
// subgroup do not depend on the staple: they are functions of the counter
// alone.  So are the parts of the proposal and of the direction that do not
// involve alpha: L = ln u1 + cos^2(2 pi u2) ln u3 (X = -L / alpha), u4^2,
// and cos(theta), sin(theta), cos(phi), sin(phi).  cm_update_f computes
// them for all three subgroups before the sequential part, as five
// independent Philox chains that the scheduler can interleave; each
// subgroup then runs only the alpha-dependent steps.  The arithmetic and its
// order are those of su2_draw_f<false>; rejected first proposals (further
// hits) and the rare alpha ranges (alpha < 2: accurate logarithms,
// alpha >= 32: double precision) take su2_draw as before.
struct DrawPre {
  float L, u4sq, costh, sinth, cphi, sphi;
};

__device__ __forceinline__ void proposal_pre_f(DrawPre &p, uint2 key, uint32_t c0, uint32_t c1, uint32_t tag) {
  const uint4 w = philox4x32_10(make_uint4(c0, c1, tag, kPurposeHeatbath), key);
  const float ang = __fmaf_rn(unif_f(w.y), 6.28318530717958648f, -3.14159265358979324f);
  const float cs = __cosf(ang);
  const float l1 = __logf(unif_f(w.x));
  const float l3 = __logf(unif_f(w.z));
  p.L = l1 + cs * cs * l3;
  const float u4 = unif_f(w.w);
  p.u4sq = u4 * u4;
}

// The direction from its two words (those direction_words returns).
__device__ __forceinline__ void direction_pre_f(DrawPre &p, uint32_t wx, uint32_t wy) {
  p.costh = 2.0f * unif_f(wx) - 1.0f;
  p.sinth = sqrt_sfu(1.0f - p.costh * p.costh);
  float sphi, cphi;
  __sincosf(__fmaf_rn(unif_f(wy), 6.28318530717958648f, -3.14159265358979324f), &sphi, &cphi);
  p.sphi = -sphi;  // sin(2 pi u) = -sin(2 pi (u - 1/2)), likewise cos
  p.cphi = -cphi;
}

// The float draw of one subgroup from its precomputed first proposal.
__device__ __forceinline__ bool su2_draw_pre(float alpha, int hits, uint2 key, uint32_t c0, uint32_t c1, uint32_t tag,
                                             const DrawPre &p, float x[4], uint32_t &nprop) {
  if (alpha >= kAlphaFp64 || alpha < kAlphaAccurateLog) return su2_draw(alpha, hits, key, c0, c1, tag, x, nprop);
  const float ia = rcp_sfu(alpha);
  ++nprop;
  float X = -p.L * ia;
  bool acc = p.u4sq <= 1.0f - 0.5f * X;
  for (int h = 1; h < hits && !acc; ++h) {
    const uint4 w = philox4x32_10(make_uint4(c0, c1, tag | (uint32_t)h, kPurposeHeatbath), key);
    ++nprop;
    const float ang = __fmaf_rn(unif_f(w.y), 6.28318530717958648f, -3.14159265358979324f);
    const float cs = __cosf(ang);
    const float l1 = __logf(unif_f(w.x));
    const float l3 = __logf(unif_f(w.z));
    X = -(l1 + cs * cs * l3) * ia;
    const float u4 = unif_f(w.w);
    acc = u4 * u4 <= 1.0f - 0.5f * X;
  }
  if (!acc) return false;
  const float rho = sqrt_sfu(X * (2.0f - X));
  x[0] = 1.0f - X;
  x[1] = rho * p.sinth * p.cphi;
  x[2] = rho * p.sinth * p.sphi;
  x[3] = rho * p.costh;
  return true;
}

// cm_update for float links with the draws' counter-only parts first.
__device__ __forceinline__ void cm_update_f(M3<float> &U, const M3<float> &A, float beta, int hits, uint2 key,
                                            uint32_t c0, uint32_t c1, int colour, int mu, uint32_t &nprop,
                                            uint32_t &nacc, float &dretr) {
  DrawPre pre[3];
#pragma unroll
  for (int sg = 0; sg < 3; ++sg) proposal_pre_f(pre[sg], key, c0, c1, heatbath_tag(colour, mu, sg));
  // the two direction blocks, split as direction_words splits them
  const uint4 d01 = philox4x32_10(make_uint4(c0, c1, heatbath_tag(colour, mu, 0) | kHitDirection, kPurposeHeatbath), key);
  const uint4 d2 = philox4x32_10(make_uint4(c0, c1, heatbath_tag(colour, mu, 2) | kHitDirection, kPurposeHeatbath), key);
  direction_pre_f(pre[0], d01.x, d01.y);
  direction_pre_f(pre[1], d01.z, d01.w);
  direction_pre_f(pre[2], d2.x, d2.y);
  dretr = 0.0f;
  const float ca = 2.0f * beta / 3.0f;
#pragma unroll
  for (int sg = 0; sg < 3; ++sg) {
    const int i = (sg == 2) ? 1 : 0;
    const int j = (sg == 0) ? 1 : 2;
    float a0, a1, a2, a3;
    block_projection(U, A, i, j, a0, a1, a2, a3);
    float k, ik;
    norm_and_inverse(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3, k, ik);
    if (!(k > 1e-30f)) continue;
    const float alpha = ca * k;
    float x[4];
    if (!su2_draw_pre(alpha, hits, key, c0, c1, heatbath_tag(colour, mu, sg), pre[sg], x, nprop)) continue;
    ++nacc;
    dretr += 2.0f * (k * x[0] - a0);
    const float v0 = a0 * ik, v1 = a1 * ik, v2 = a2 * ik, v3 = a3 * ik;
    const float r0 = x[0] * v0 + x[1] * v1 + x[2] * v2 + x[3] * v3;
    const float r1 = -x[0] * v1 + v0 * x[1] + (x[2] * v3 - x[3] * v2);
    const float r2 = -x[0] * v2 + v0 * x[2] + (x[3] * v1 - x[1] * v3);
    const float r3 = -x[0] * v3 + v0 * x[3] + (x[1] * v2 - x[2] * v1);
    rotate_rows(U, i, j, r0, r1, r2, r3);
  }
}

}  // namespace su3g
