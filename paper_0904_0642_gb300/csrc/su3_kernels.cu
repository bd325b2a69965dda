// su3_kernels.cu -- CUDA kernels of the checkerboard SU(3) heatbath (sm_103a).
//
// k_tick: one persistent launch advances every resident chain by one stage
//   (a (colour, direction) update phase, a re-unitarisation or a
//   measurement).  One thread per site of the tile (tile = CTA width); tiles
//   of all chains are spread over a grid of CTAs sized to the SM count.
//   The chains' stage machines advance at the end of the launch (one
//   chain: by the last warp to finish; several: by the first, into a second
//   state slot, with the last one flipping the slot parity), and the last
//   warp reduces measurement partial sums in a fixed order.
// k_start, k_convert, k_measure*: start configurations, canonical-layout
//   conversion and stand-alone measurements.
#include <cstdio>
#include <mutex>
#include <type_traits>

#include <cuda.h>  // CUcontext / CUresult for the two driver calls reached through the runtime

#include "su3_device.cuh"
#include "su3_launch.h"

namespace su3g {

// ------------------------------------------------------------------ geometry

struct SiteGeo {
  int x[kMaxD];
  int s;      // i_s - 1 within the layer
  int layer;
};

// Coordinates of the site of colour `colour` at checkerboard index jj
// (eqs. xD, x^i, i_c): the even lexicographic index 2 jj shares its row
// with the odd one, and the colour fixes which of the two it is.
// SUB (sublattice boxes): jj counts the interior sites of the box; the
// returned coordinates and index are those of the padded box.  Sublattice
// origins are even, so the colour is the colour of the undivided lattice.
template <bool SUB = false>
__device__ __forceinline__ SiteGeo site_of(const ChainDesc &d, int layer, int colour, int jj) {
  SiteGeo g;
  if constexpr (SUB) {
    int r = 2 * jj, par = colour;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
      if (i < d.D) {
        const int n = d.idims[i];
        const int q = r / n;
        g.x[i] = r - q * n;
        r = q;
        if (i > 0) par += g.x[i];
      } else {
        g.x[i] = 0;
      }
    }
    g.x[0] += par & 1;
    int sp = 0;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i)
      if (i < d.D) {
        g.x[i] += d.hpad[i];
        sp += g.x[i] * d.stride[i];
      }
    g.s = sp;
    g.layer = layer;
    return g;
  }
  int r = 2 * jj;
  int par = colour;
  if (d.pow2) {
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
      if (i < d.D) {
        g.x[i] = r & (d.dims[i] - 1);
        r >>= d.shift[i];
        if (i > 0) par += g.x[i];
      } else {
        g.x[i] = 0;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
      if (i < d.D) {
        const int n = d.dims[i];
        const int q = r / n;
        g.x[i] = r - q * n;
        r = q;
        if (i > 0) par += g.x[i];
      } else {
        g.x[i] = 0;
      }
    }
  }
  par &= 1;
  g.x[0] += par;
  g.s = 2 * jj + par;
  g.layer = layer;
  return g;
}

// Lexicographic offset and layer flip of one step in direction nu.
__device__ __forceinline__ void step_fwd(const ChainDesc &d, int xnu, int nu, int &off, int &flip) {
  const int n = d.dims[nu], st = d.stride[nu];
  if (xnu == n - 1) {
    off = -(n - 1) * st;
    flip = (d.nlayers == 2) ? ((d.glue_mask >> nu) & 1) : 0;
  } else {
    off = st;
    flip = 0;
  }
}
__device__ __forceinline__ void step_bwd(const ChainDesc &d, int xnu, int nu, int &off, int &flip) {
  const int n = d.dims[nu], st = d.stride[nu];
  if (xnu == 0) {
    off = (n - 1) * st;
    flip = (d.nlayers == 2) ? ((d.glue_mask >> nu) & 1) : 0;
  } else {
    off = -st;
    flip = 0;
  }
}

// The layer reached by a step with layer flip f: for sublattice boxes the
// virtual layer of the same sublattice in the other layer.
template <bool SUB>
__device__ __forceinline__ int lflip(const ChainDesc &d, int l, int f) {
  if constexpr (SUB)
    return f ? (l < d.nb ? l + d.nb : l - d.nb) : l;
  else
    return l ^ f;
}

// 1 when (virtual) layer l belongs to layer 1 of the double-layered torus.
template <bool SUB>
__device__ __forceinline__ int in_layer1(const ChainDesc &d, int l) {
  if constexpr (SUB)
    return l >= d.nb ? 1 : 0;
  else
    return l;
}

// Random-number site key: layer * V + i_s - 1, or the site number of
// (x mod period) on the period lattice (identical numbers on sublattices).
// SUB: from the coordinates in the undivided lattice, so that a divided
// lattice draws the same numbers as the undivided one.
template <bool SUB = false>
__device__ __forceinline__ uint32_t site_key(const ChainDesc &d, const SiteGeo &g) {
  if constexpr (SUB) {
    const int L = g.layer / d.nb;
    int b = g.layer - L * d.nb;
    const int lay = (d.nlayers == 2 && !d.layer_blind) ? L : 0;
    int key = 0;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i)
      if (i < d.D) {
        const int bc = b % d.bdiv[i];
        b /= d.bdiv[i];
        const int gx = bc * d.idims[i] + g.x[i] - d.hpad[i];
        key += d.custom_period ? (gx % d.period[i]) * d.pstride[i] : gx * d.gstride[i];
      }
    return (uint32_t)(lay * (d.custom_period ? d.Vp : d.V) + key);
  }
  const int lay = (d.nlayers == 2 && !d.layer_blind) ? g.layer : 0;
  if (!d.custom_period) return (uint32_t)(lay * d.V + g.s);
  int key = 0;
#pragma unroll
  for (int i = 0; i < kMaxD; ++i)
    if (i < d.D) key += (g.x[i] % d.period[i]) * d.pstride[i];
  return (uint32_t)(lay * d.Vp + key);
}

__device__ __forceinline__ int sel(const int (&x)[kMaxD], int i) {
  int v = 0;
#pragma unroll
  for (int k = 0; k < kMaxD; ++k)
    if (k == i) v = x[k];
  return v;
}

// ------------------------------------------------------------------ one link update

// The staples of one direction nu added to A.
template <class S, bool WT, bool SUB>
__device__ __forceinline__ void add_staples(const ChainDesc &d, const SiteGeo &g, int colour, int mu, int nu, int xnu,
                                            int sp, int lp, M3<typename S::R> &A) {
  using R = typename S::R;
  const int Vh = d.Vh, layer = g.layer, jj = g.s >> 1, oc = colour ^ 1;
  int offn, fln, offm, flm;
  step_fwd(d, xnu, nu, offn, fln);
  step_bwd(d, xnu, nu, offm, flm);
  const int sn = g.s + offn, ln = lflip<SUB>(d, layer, fln);  // x + nu
  const int sm = g.s + offm, lm = lflip<SUB>(d, layer, flm);  // x - nu
  const int spm = sp + offm, lpm = lflip<SUB>(d, lp, flm);    // x + mu - nu
  // upper staple U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ = a (c b)^+, all factors SU(3):
  // two rows of each product, the third from the cross product
  const M3<R> b = S::load(plane_ptr<S>(d, ln, oc, mu), Vh, sn >> 1);       // U_mu(x+nu)
  const M3<R> c = S::load2(plane_ptr<S>(d, layer, colour, nu), Vh, jj);    // U_nu(x)
  M3<R> cb = mul_nn_2(c, b);
  third_row(cb);
  const M3<R> a = S::load2(plane_ptr<S>(d, lp, oc, nu), Vh, sp >> 1);      // U_nu(x+mu)
  // WT (a kernel compiled for two-coupling chains) and a two-coupling chain:
  // each staple enters with the coupling of its plaquette, beta1 when any of
  // its links lies in layer 1, so A carries the betas and the heatbath runs
  // with beta = 1.  Otherwise plain sums (beta enters the heatbath).
  const bool weighted = WT && d.weighted;
  const R b0 = sizeof(R) == 4 ? (R)d.beta_f : (R)d.beta_d, b1 = sizeof(R) == 4 ? (R)d.beta1_f : (R)d.beta1_d;
  if (weighted)
    acc_su3_2rows_w(A, mul_nd_2(a, cb), (in_layer1<SUB>(d, layer) | in_layer1<SUB>(d, lp) | in_layer1<SUB>(d, ln)) ? b1 : b0);
  else
    acc_su3_2rows(A, mul_nd_2(a, cb));
  // lower staple U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) = (e f)^+ h
  const M3<R> f = S::load(plane_ptr<S>(d, lpm, colour, nu), Vh, spm >> 1); // U_nu(x+mu-nu)
  const M3<R> e = S::load2(plane_ptr<S>(d, lm, oc, mu), Vh, sm >> 1);      // U_mu(x-nu)
  M3<R> ef = mul_nn_2(e, f);
  third_row(ef);
  const M3<R> h = S::load(plane_ptr<S>(d, lm, oc, nu), Vh, sm >> 1);       // U_nu(x-nu)
  if (weighted)
    acc_su3_2rows_w(A, mul_dn_2(ef, h), (in_layer1<SUB>(d, lm) | in_layer1<SUB>(d, lpm) | in_layer1<SUB>(d, layer)) ? b1 : b0);
  else
    acc_su3_2rows(A, mul_dn_2(ef, h));
}

// The staples of one direction nu from precomputed plane offsets (p*, in
// vectors from the chain's link base) and checkerboard indices (j*) of the
// six links: the arithmetic and its order are those of add_staples.  Plane
// offset and index stay separate because the 18-real float form addresses a
// plane's 16-byte vectors from its (16-byte aligned) start.
// Where a form's vectors are its addressing unit (every form but the 18-real
// float one) offset and index are summed first: one index per link.
template <class S>
__device__ __forceinline__ M3<typename S::R> load_at(const ChainDesc &d, const typename S::Vec *base, int Vh, int p,
                                                     int j, bool rows2) {
  // the plane offset lies within the (virtual) layers' planes
  if (!in_bounds(p, (long long)d.nlayers * d.nb * 2 * d.D * S::NQ * Vh, kBoundsLink)) return m3_zero<typename S::R>();
  if constexpr (std::is_same<S, StoreF32x18>::value)
    return rows2 ? S::load2(base + p, Vh, j) : S::load(base + p, Vh, j);
  else
  {
    if (!in_bounds(j, Vh, kBoundsIndex)) return m3_zero<typename S::R>();
    return rows2 ? S::load2(base + (p + j), Vh, 0) : S::load(base + (p + j), Vh, 0);
  }
}

template <class S, bool WT>
__device__ __forceinline__ void add_staples_idx(const ChainDesc &d, const typename S::Vec *base, int Vh, int pb, int jb,
                                                int pc, int jc, int pa, int ja, int pf, int jf, int pe, int je, int ph,
                                                int jh, int wu, int wl, M3<typename S::R> &A) {
  using R = typename S::R;
  const M3<R> b = load_at<S>(d, base, Vh, pb, jb, false);  // U_mu(x+nu)
  const M3<R> c = load_at<S>(d, base, Vh, pc, jc, true);   // U_nu(x)
  M3<R> cb = mul_nn_2(c, b);
  third_row(cb);
  const M3<R> a = load_at<S>(d, base, Vh, pa, ja, true);   // U_nu(x+mu)
  const bool weighted = WT && d.weighted;
  const R b0 = sizeof(R) == 4 ? (R)d.beta_f : (R)d.beta_d, b1 = sizeof(R) == 4 ? (R)d.beta1_f : (R)d.beta1_d;
  if (weighted)
    acc_su3_2rows_w(A, mul_nd_2(a, cb), wu ? b1 : b0);
  else
    acc_su3_2rows(A, mul_nd_2(a, cb));
  const M3<R> f = load_at<S>(d, base, Vh, pf, jf, false);  // U_nu(x+mu-nu)
  const M3<R> e = load_at<S>(d, base, Vh, pe, je, true);   // U_mu(x-nu)
  M3<R> ef = mul_nn_2(e, f);
  third_row(ef);
  const M3<R> h = load_at<S>(d, base, Vh, ph, jh, false);  // U_nu(x-nu)
  if (weighted)
    acc_su3_2rows_w(A, mul_dn_2(ef, h), wl ? b1 : b0);
  else
    acc_su3_2rows(A, mul_dn_2(ef, h));
}

// update_site for an undivided lattice with the neighbour geometry computed
// once per site: forward and backward site offsets and layer flips in every
// direction, and the plane offsets as multiples of one plane stride.  Same
// arithmetic, same order as update_site.
template <class S, bool WT, int DF = 0>
__device__ __forceinline__ void update_site_lean(const ChainDesc &d, uint32_t sweep, int colour, int mu, int layer,
                                                 int jj, uint32_t &nprop, uint32_t &nacc, typename S::R &dretr) {
  using R = typename S::R;
  using Vec = typename S::Vec;
  // DF > 0: every chain of the launch is a periodic torus (one layer) of
  // dimension DF, undivided, with one coupling and the default random-number
  // site key (no layer flips, no layer offsets, D known to the compiler)
  constexpr bool kTorus = DF > 0;
  if constexpr (kTorus) layer = 0;
  const int Vh = d.Vh, D = kTorus ? DF : d.D;
  const SiteGeo g = site_of<false>(d, layer, colour, jj);
  const int PS = S::NQ * Vh, CS = D * PS, LS = 2 * CS;
  const int oc = colour ^ 1;
  const Vec *base = reinterpret_cast<const Vec *>(d.links);
  const int s = g.s;
  int of[kMaxD], ob[kMaxD], ff[kMaxD], fb[kMaxD];
#pragma unroll
  for (int k = 0; k < kMaxD; ++k) {
    of[k] = ob[k] = ff[k] = fb[k] = 0;
    if (k < D) {
      step_fwd(d, g.x[k], k, of[k], ff[k]);
      step_bwd(d, g.x[k], k, ob[k], fb[k]);
      if constexpr (kTorus) ff[k] = fb[k] = 0;
    }
  }
  int ofm = 0, ffm = 0;
#pragma unroll
  for (int k = 0; k < kMaxD; ++k)
    if (k == mu) {
      ofm = of[k];
      ffm = ff[k];
    }
  const int lp = layer ^ ffm;            // layer of x + mu
  const int sp = s + ofm;                // x + mu
  const int pmu_oc = oc * CS + mu * PS;  // plane (oc, mu) within a layer
  const uint2 key = make_uint2(d.seed_lo, d.seed_hi);
  const uint32_t skey = kTorus ? (uint32_t)s : site_key<false>(d, g);  // the torus form has the default key
  M3<R> A = m3_zero<R>();
#pragma unroll
  for (int nu = 0; nu < kMaxD; ++nu) {
    if (nu < D && nu != mu) {
      const int lb = layer ^ ff[nu], lm = layer ^ fb[nu], lf = lp ^ fb[nu];
      const int sm = s + ob[nu];
      add_staples_idx<S, WT>(d, base, Vh,
                             lb * LS + pmu_oc, (s + of[nu]) >> 1,                   // U_mu(x+nu)
                             layer * LS + colour * CS + nu * PS, jj,                // U_nu(x)
                             lp * LS + oc * CS + nu * PS, sp >> 1,                  // U_nu(x+mu)
                             lf * LS + colour * CS + nu * PS, (sp + ob[nu]) >> 1,   // U_nu(x+mu-nu)
                             lm * LS + pmu_oc, sm >> 1,                             // U_mu(x-nu)
                             lm * LS + oc * CS + nu * PS, sm >> 1,                  // U_nu(x-nu)
                             layer | lp | lb, lm | lf | layer, A);
    }
  }
  typename S::Vec *pu = plane_ptr<S>(d, layer, colour, mu);
  M3<R> U = S::load(pu, Vh, jj);
  const R beta = (WT && d.weighted) ? R(1) : (sizeof(R) == 4 ? (R)d.beta_f : (R)d.beta_d);
  if constexpr (sizeof(R) == 4)
    cm_update_f(U, A, beta, d.hits, key, skey, sweep, colour, mu, nprop, nacc, dretr);
  else
    cm_update(U, A, beta, d.hits, key, skey, sweep, colour, mu, nprop, nacc, dretr);
  S::store(pu, Vh, jj, U);
}

// ROLLED: the loop over staple directions stays a loop (no unrolling), so the
// compiler cannot hoist later directions' loads; fewer registers, less code.
template <class S, bool ROLLED, bool WT, bool SUB>
__device__ __forceinline__ void update_site(const ChainDesc &d, uint32_t sweep, int colour, int mu, int layer, int jj,
                                            uint32_t &nprop, uint32_t &nacc, typename S::R &dretr) {
  using R = typename S::R;
  const int Vh = d.Vh;
  const SiteGeo g = site_of<SUB>(d, layer, colour, jj);
  int offp, flp;
  step_fwd(d, sel(g.x, mu), mu, offp, flp);
  const int sp = g.s + offp, lp = lflip<SUB>(d, layer, flp);  // x + mu
  const uint2 key = make_uint2(d.seed_lo, d.seed_hi);
  const uint32_t skey = site_key<SUB>(d, g);

  M3<R> A = m3_zero<R>();
  if constexpr (ROLLED) {
#pragma unroll 1
    for (int nu = 0; nu < d.D; ++nu)
      if (nu != mu) add_staples<S, WT, SUB>(d, g, colour, mu, nu, sel(g.x, nu), sp, lp, A);
  } else {
#pragma unroll
    for (int nu = 0; nu < kMaxD; ++nu)
      if (nu < d.D && nu != mu) add_staples<S, WT, SUB>(d, g, colour, mu, nu, g.x[nu], sp, lp, A);
  }
  typename S::Vec *pu = plane_ptr<S>(d, layer, colour, mu);
  const int ju = g.s >> 1;  // jj itself unless the site sits in a padded box
  M3<R> U = S::load(pu, Vh, ju);
  const R beta = (WT && d.weighted) ? R(1) : (sizeof(R) == 4 ? (R)d.beta_f : (R)d.beta_d);
  if constexpr (sizeof(R) == 4)
    cm_update_f(U, A, beta, d.hits, key, skey, sweep, colour, mu, nprop, nacc, dretr);
  else
    cm_update(U, A, beta, d.hits, key, skey, sweep, colour, mu, nprop, nacc, dretr);
  S::store(pu, Vh, ju, U);
}


// ------------------------------------------------------------------ re-unitarisation

__device__ __forceinline__ double to_double(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_double(double x) { return x; }

// Rows 1, 2 of a stored link in double (row 3 is rebuilt by reunit_d, or
// not kept at all by two-row storage).
template <class S>
__device__ __forceinline__ M3<double> load_rows2_d(const typename S::Vec *p, int Vh, int js) {
  const M3<typename S::R> f = S::load2(p, Vh, js);
  M3<double> m;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      m.e[i][j] = i < 2 ? C<double>{to_double(f.e[i][j].re), to_double(f.e[i][j].im)} : C<double>{0.0, 0.0};
  return m;
}

// The double-precision Gram-Schmidt of two float rows r1, r2, applied in
// float.  The norms and the inner product are summed in double from the
// float elements (products of floats are exact in double):
//   n1 = |r1|^2, s1 = n1^(-1/2), q = <r1, r2>, p = s1 q = <r1', r2>,
//   n2 = |r2 - p r1'|^2 = |r2|^2 - |p|^2 (as |r1'| = 1), s2 = n2^(-1/2).
// The results r1' = r1 s1 and r2'' = (r2 - p r1') s2 differ from the stored
// rows by corrections of the rows' departure from orthonormality (~1e-7
// between re-unitarisations): r1' = r1 + r1 e1 with e1 = s1 - 1, and
// r2'' = r2 + (c (1 + e2) + r2 e2) with c = -p r1' and e2 = s2 - 1.  Each
// correction is formed in float (the factors e1, p, e2 rounded to float:
// relative errors 2^-24 of small quantities) and added with a single
// rounding, so the stored floats are the double computation's rounded
// result except where that result lies within ~1e-14 of a rounding boundary
// (1e-12 for departures of 1e-4).  38 double operations per link instead of
// 56, on a pipe that runs at 1/64 of the float rate here.
__device__ __forceinline__ void reunit_rows2_f(M3<float> &m) {
  C<float> *r1 = m.e[0], *r2 = m.e[1];
  double n1 = f2d_bits(r1[0].re) * f2d_bits(r1[0].re);
  n1 = fm(f2d_bits(r1[0].im), f2d_bits(r1[0].im), n1);
  double n2 = f2d_bits(r2[0].re) * f2d_bits(r2[0].re);
  n2 = fm(f2d_bits(r2[0].im), f2d_bits(r2[0].im), n2);
  // q = sum_k conj(r1_k) r2_k
  double qr = f2d_bits(r1[0].re) * f2d_bits(r2[0].re), qi = f2d_bits(r1[0].re) * f2d_bits(r2[0].im);
  qr = fm(f2d_bits(r1[0].im), f2d_bits(r2[0].im), qr);
  qi = fm(-f2d_bits(r1[0].im), f2d_bits(r2[0].re), qi);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    const double ar = f2d_bits(r1[k].re), ai = f2d_bits(r1[k].im), br = f2d_bits(r2[k].re), bi = f2d_bits(r2[k].im);
    n1 = fm(ar, ar, n1);
    n1 = fm(ai, ai, n1);
    n2 = fm(br, br, n2);
    n2 = fm(bi, bi, n2);
    qr = fm(ar, br, qr);
    qr = fm(ai, bi, qr);
    qi = fm(ar, bi, qi);
    qi = fm(-ai, br, qi);
  }
  const double s1 = rsqrt_d<1>(n1);
  const double pdr = s1 * qr, pdi = s1 * qi;
  n2 = fm(-pdr, pdr, n2);
  n2 = fm(-pdi, pdi, n2);
  const double s2 = rsqrt_d<1>(n2);
  const float e1 = d2f_bits(s1 - 1.0), e2 = d2f_bits(s2 - 1.0);
  const float pr = d2f_bits(pdr), pi = d2f_bits(pdi);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const C<float> a = r1[k];
    r1[k] = {fm(a.re, e1, a.re), fm(a.im, e1, a.im)};
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // c = -p r1'_k, then r2''_k = r2_k + (c (1 + e2) + r2_k e2), one rounding
    const C<float> a = r1[k], b = r2[k];
    const float cr = fm(pi, a.im, -pr * a.re), ci = fm(-pi, a.re, -pr * a.im);
    r2[k] = {b.re + fm(b.re, e2, fm(cr, e2, cr)), b.im + fm(b.im, e2, fm(ci, e2, ci))};
  }
}

// Two links per step: their Gram-Schmidt chains are independent.
template <class S, bool SUB = false>
__device__ __forceinline__ void reunit_site(const ChainDesc &d, int layer, int jj) {
  constexpr bool kTwoRows = S::kTwoRows;  // the 12-real form keeps rows 1, 2 only
  constexpr int kNewton = sizeof(typename S::R) == 4 ? 1 : 2;  // float storage: one Newton step suffices
  const int Vh = d.Vh;
  if constexpr (std::is_same<S, StoreF32x12>::value) {
    // two-row float storage: the double Gram-Schmidt applied in float
    for (int colour = 0; colour < 2; ++colour) {
      const int js = SUB ? (site_of<true>(d, layer, colour, jj).s >> 1) : jj;
      int mu = 0;
#pragma unroll 1
      for (; mu + 1 < d.D; mu += 2) {
        typename S::Vec *p0 = plane_ptr<S>(d, layer, colour, mu), *p1 = plane_ptr<S>(d, layer, colour, mu + 1);
        M3<float> m0 = S::load2(p0, Vh, js), m1 = S::load2(p1, Vh, js);
        reunit_rows2_f(m0);
        reunit_rows2_f(m1);
        S::store(p0, Vh, js, m0);
        S::store(p1, Vh, js, m1);
      }
      if (mu < d.D) {
        typename S::Vec *p = plane_ptr<S>(d, layer, colour, mu);
        M3<float> m = S::load2(p, Vh, js);
        reunit_rows2_f(m);
        S::store(p, Vh, js, m);
      }
    }
  } else {
    for (int colour = 0; colour < 2; ++colour) {
      const int js = SUB ? (site_of<true>(d, layer, colour, jj).s >> 1) : jj;
      int mu = 0;
#pragma unroll 1
      for (; mu + 1 < d.D; mu += 2) {
        typename S::Vec *p0 = plane_ptr<S>(d, layer, colour, mu), *p1 = plane_ptr<S>(d, layer, colour, mu + 1);
        M3<double> m0 = load_rows2_d<S>(p0, Vh, js);
        M3<double> m1 = load_rows2_d<S>(p1, Vh, js);
        reunit_d<kNewton, !kTwoRows>(m0);
        reunit_d<kNewton, !kTwoRows>(m1);
        S::store(p0, Vh, js, to_storage<typename S::R>(m0));
        S::store(p1, Vh, js, to_storage<typename S::R>(m1));
      }
      if (mu < d.D) {
        typename S::Vec *p = plane_ptr<S>(d, layer, colour, mu);
        M3<double> m = load_rows2_d<S>(p, Vh, js);
        reunit_d<kNewton, !kTwoRows>(m);
        S::store(p, Vh, js, to_storage<typename S::R>(m));
      }
    }
  }
}

// ------------------------------------------------------------------ measurements
// Per thread: the two sites of checkerboard index jj (both colours).  Sums
// in double: plaquettes split space/time, and Polyakov lines started at
// x^D = 0 (the line follows the forward time neighbour until it closes).

// Re Tr(U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+) = Re Tr(P Q^+) with
// P = U_mu(x) U_nu(x+mu), Q = U_nu(x) U_mu(x+nu), both in SU(3): rows 1, 2
// of P and Q come from rows 1, 2 of U_mu(x) and U_nu(x) (um2, un2) and the
// full U_nu(x+mu), U_mu(x+nu); their third rows contribute
// sum_j P_3j conj(Q_3j) = <P_1 x P_2, Q_1 x Q_2> = G_11 G_22 - G_12 G_21
// (the Binet-Cauchy identity; row 3 of an SU(3) matrix is the conjugated
// cross product of rows 1, 2) with G_kl = <P_k, Q_l> = sum_j conj(P_kj) Q_lj.
// The factor 1/3 is applied to the sums.
template <class S, bool SUB = false>
__device__ __forceinline__ typename S::R plaquette_at(const ChainDesc &d, const SiteGeo &g, int colour, int mu, int nu,
                                                      int xmu, int xnu, const M3<typename S::R> &um2) {
  using R = typename S::R;
  const int Vh = d.Vh, layer = g.layer, jj = g.s >> 1, oc = colour ^ 1;
  int offp, flp, offn, fln;
  step_fwd(d, xmu, mu, offp, flp);
  step_fwd(d, xnu, nu, offn, fln);
  const M3<R> a = S::load(plane_ptr<S>(d, lflip<SUB>(d, layer, flp), oc, nu), Vh, (g.s + offp) >> 1);  // U_nu(x+mu)
  const M3<R> b = S::load(plane_ptr<S>(d, lflip<SUB>(d, layer, fln), oc, mu), Vh, (g.s + offn) >> 1);  // U_mu(x+nu)
  const M3<R> un2 = S::load2(plane_ptr<S>(d, layer, colour, nu), Vh, jj);                // U_nu(x), rows 1, 2
  const M3<R> P = mul_nn_2(um2, a), Q = mul_nn_2(un2, b);
  C<R> G[2][2];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      C<R> x = cmul_cn(P.e[k][0], Q.e[l][0]);
      cmac_cn(x, P.e[k][1], Q.e[l][1]);
      cmac_cn(x, P.e[k][2], Q.e[l][2]);
      G[k][l] = x;
    }
  R tr = G[0][0].re + G[1][1].re;
  tr = fm(G[0][0].re, G[1][1].re, tr);
  tr = fm(-G[0][0].im, G[1][1].im, tr);
  tr = fm(-G[0][1].re, G[1][0].re, tr);
  tr = fm(G[0][1].im, G[1][0].im, tr);
  return tr;
}

// Per thread: the two sites of checkerboard index jj (both colours).  Sums
// of Re Tr and Tr (the 1/3 is applied by finalize_measure): plaquettes split
// space/time, summed per site in the storage precision and accumulated in
// double; Polyakov lines started at x^D = 0 (the line follows the forward
// time neighbour until it closes).  The loop over mu is unrolled so that
// the loads of several plaquettes are in flight together.
// SUB: plaquettes read the forward halos; a Polyakov line stays inside its
// sublattice box only when time is undivided, so it is taken only then.
template <class S, bool SUB = false>
__device__ __forceinline__ void measure_site(const ChainDesc &d, int layer, int jj, double acc[kPartVals]) {
  using R = typename S::R;
  const int Vh = d.Vh;
  const int D = d.D;
#pragma unroll 1
  for (int colour = 0; colour < 2; ++colour) {
    const SiteGeo g = site_of<SUB>(d, layer, colour, jj);
    R ps = R(0), pt = R(0);
#pragma unroll
    for (int mu = 0; mu + 1 < kMaxD; ++mu) {
      if (mu + 1 >= D) continue;
      const int xmu = sel(g.x, mu);
      const M3<R> um2 = S::load2(plane_ptr<S>(d, layer, colour, mu), Vh, g.s >> 1);  // U_mu(x), rows 1, 2
#pragma unroll
      for (int nu = 1; nu < kMaxD; ++nu) {
        if (nu <= mu || nu >= D) continue;
        const R p = plaquette_at<S, SUB>(d, g, colour, mu, nu, xmu, g.x[nu], um2);
        if (nu == D - 1) pt += p; else ps += p;
      }
    }
    acc[0] += to_double(ps);
    acc[1] += to_double(pt);
    const int t = D - 1;
    if (sel(g.x, t) == 0 && !(SUB && d.hpad[t])) {
      // Polyakov line through (layer, x, x^D = 0): rows 1, 2 of the running
      // product (SU(3)), the next link's load issued before the product
      M3<R> P = S::load2(plane_ptr<S>(d, layer, colour, t), Vh, g.s >> 1);
      int cs = g.s, cl = layer, cc = colour, xt = 0;
      auto advance = [&]() {
        int off, fl;
        step_fwd(d, xt, t, off, fl);
        cs += off;
        cl = lflip<SUB>(d, cl, fl);
        cc ^= 1;
        xt = (xt == d.dims[t] - 1) ? 0 : xt + 1;
        return !(cs == g.s && cl == layer);
      };
      bool more = advance();
      M3<R> nxt = more ? S::load(plane_ptr<S>(d, cl, cc, t), Vh, cs >> 1) : m3_zero<R>();
#pragma unroll 1
      while (more) {
        const M3<R> cur = nxt;
        more = advance();
        if (more) nxt = S::load(plane_ptr<S>(d, cl, cc, t), Vh, cs >> 1);
        P = mul_nn_2(P, cur);
      }
      // trace: P_11 + P_22 + P_33 with P_33 = conj(P_11 P_22 - P_12 P_21)
      const C<R> p33 = conj_cross(P.e[0][0], P.e[1][1], P.e[0][1], P.e[1][0]);
      acc[2] += to_double(P.e[0][0].re + P.e[1][1].re + p33.re);
      acc[3] += to_double(P.e[0][0].im + P.e[1][1].im + p33.im);
    }
  }
}

// Block reduction of kPartVals doubles in a fixed order (warp shuffles, then
// warp 0 over the warp sums).  Result valid in thread 0.
__device__ __forceinline__ void block_reduce(double v[kPartVals], double *smem /* [32][kPartVals] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < kPartVals; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kPartVals; ++k) smem[warp * kPartVals + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kPartVals; ++k) {
      double x = lane < nw ? smem[lane * kPartVals + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
  __syncthreads();
}

// Sum the tile partials of one chain per layer (one warp, fixed order) and
// write [total, space, time, poly_re, poly_im] for each layer and the whole.
__device__ void finalize_measure(const ChainDesc &d, const double *partials, double *out) {
  const int lane = threadIdx.x & 31;
  double whole[kPartVals] = {0, 0, 0, 0};
  const int D = d.D;
  // the partial sums hold Re Tr and Tr: the counts carry the factor 3
  const double np_s = 3.0 * d.V * (D - 1) * (D - 2) / 2, np_t = 3.0 * d.V * (D - 1);
  // Polyakov lines are not taken inside sublattice boxes with divided time
  const double nl = d.hpad[D - 1] ? __longlong_as_double(0x7ff8000000000000ll) : 3.0 * d.spatial_per_layer;
  for (int layer = 0; layer < d.nlayers; ++layer) {
    double v[kPartVals] = {0, 0, 0, 0};
    for (int t = lane; t < d.tiles_per_layer; t += 32)
#pragma unroll
      for (int k = 0; k < kPartVals; ++k) v[k] += __ldcg(partials + (size_t)(layer * d.tiles_per_layer + t) * kPartVals + k);
#pragma unroll
    for (int k = 0; k < kPartVals; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = __shfl_sync(0xffffffffu, v[k], 0);
      whole[k] += v[k];
    }
    if (lane == 0) {
      double *o = out + layer * kMeasVals;
      o[0] = (v[0] + v[1]) / (np_s + np_t);
      o[1] = np_s > 0 ? v[0] / np_s : 0.0;
      o[2] = v[1] / np_t;
      o[3] = v[2] / nl;  // NaN when nl is
      o[4] = v[3] / nl;
    }
  }
  if (lane == 0) {
    const double L = (double)d.nlayers;
    double *o = out + d.nlayers * kMeasVals;
    o[0] = (whole[0] + whole[1]) / (L * (np_s + np_t));
    o[1] = np_s > 0 ? whole[0] / (L * np_s) : 0.0;
    o[2] = whole[1] / (L * np_t);
    o[3] = whole[2] / (L * nl);
    o[4] = whole[3] / (L * nl);
  }
}

// The action bookkeeping restarts at this measurement (a chain whose links
// were replaced asks for it): the measurement becomes the reference and
// the booked changes restart from zero.  Warp-collective; the measurement
// was written by lane 0 of this warp.
__device__ __forceinline__ void restart_bookkeeping(const ChainDesc &d, const double *out) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < (d.nlayers + 1) * kMeasVals; i += 32) d.ref_meas[i] = out[i];
  for (int i = lane; i < d.n_action_slots; i += 32) d.action_slots[i] = 0.0;
}

// ------------------------------------------------------------------ tick kernel

// Copy a chain's descriptor and its current state (of its two state slots,
// the one the launch's parity names; the parity is the same for the whole
// launch) into the CTA's shared memory.  Both slots and the parity are
// loaded together and the current one selected, so that no load waits for
// another.
__device__ __forceinline__ void load_chain(const EngineArgs &ea, int c, ChainDesc &sd, ChainState &ss, int &s_par) {
  const int n1 = sizeof(ChainDesc) / 4, n2 = sizeof(ChainState) / 4;
  const uint32_t *src1 = reinterpret_cast<const uint32_t *>(ea.desc + c);
  const uint32_t *src2 = reinterpret_cast<const uint32_t *>(ea.state + 2 * (size_t)c);
  uint32_t *dst1 = reinterpret_cast<uint32_t *>(&sd), *dst2 = reinterpret_cast<uint32_t *>(&ss);
  for (int i = threadIdx.x; i < n1; i += blockDim.x) dst1[i] = src1[i];
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    const uint32_t w0 = __ldcg(src2 + i), w1 = __ldcg(src2 + n2 + i);
    const int par = __ldcg(&ea.hdr->parity);
    dst2[i] = par ? w1 : w0;
    if (i == 0) s_par = par;
  }
}

// The next chain of a CTA, staged in shared memory (multi-chain form).
struct ChainStaging {
  ChainDesc d;
  ChainState s;
};
struct NoStaging {};

// Start asynchronous copies (cp.async, one 4-byte word per thread at a
// time) of chain c's descriptor and current state into the CTA's staging
// buffer.  The CTA's next chain switch waits for them (cp.async.wait_all,
// then the barrier) and copies them over the current ones, instead of
// waiting behind that barrier for a round trip to L2.
__device__ __forceinline__ void stage_chain(const EngineArgs &ea, int c, int par, ChainStaging &stg) {
  const int n1 = sizeof(ChainDesc) / 4, n2 = sizeof(ChainState) / 4;
  const uint32_t *src1 = reinterpret_cast<const uint32_t *>(ea.desc + c);
  const uint32_t *src2 = reinterpret_cast<const uint32_t *>(ea.state + 2 * (size_t)c + par);
  uint32_t *dst1 = reinterpret_cast<uint32_t *>(&stg.d), *dst2 = reinterpret_cast<uint32_t *>(&stg.s);
  for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
    const uint32_t *src = i < n1 ? src1 + i : src2 + (i - n1);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(i < n1 ? dst1 + i : dst2 + (i - n1));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Copy the staged descriptor and state over the current ones (shared to
// shared, one word per thread at a time).
__device__ __forceinline__ void take_staged(ChainDesc &sd, ChainState &ss, const ChainStaging &stg) {
  const int n1 = sizeof(ChainDesc) / 4, n2 = sizeof(ChainState) / 4;
  const uint32_t *src1 = reinterpret_cast<const uint32_t *>(&stg.d), *src2 = reinterpret_cast<const uint32_t *>(&stg.s);
  uint32_t *dst1 = reinterpret_cast<uint32_t *>(&sd), *dst2 = reinterpret_cast<uint32_t *>(&ss);
  for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
    if (i < n1)
      dst1[i] = src1[i];
    else
      dst2[i - n1] = src2[i - n1];
  }
}

// Warp-sum the FHKP counters and add them to the chain's totals.
__device__ __forceinline__ void flush_counters(const ChainDesc &d, uint32_t &np, uint32_t &na) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    np += __shfl_down_sync(0xffffffffu, np, o);
    na += __shfl_down_sync(0xffffffffu, na, o);
  }
  if ((threadIdx.x & 31) == 0 && np) {
    atomicAdd(d.counters + 0, (unsigned long long)np);
    atomicAdd(d.counters + 1, (unsigned long long)na);
  }
  np = 0;
  na = 0;
}

// Next stage of a chain's stage machine (the host keeps an identical mirror):
// the 2D update phases of a sweep, then a re-unitarisation and/or a
// measurement when the completed-sweep count is a multiple of their
// cadence; the chain goes idle when a sweep would start at its target.
struct StageParams {
  int D, reunit_every, measure_every;
};

__device__ __host__ inline void advance_stage(const StageParams &d, ChainState &s) {
  s.prev_stage = s.stage;
  if (s.stage < 2 * d.D) {
    s.stage += 1;
    if (s.stage == 2 * d.D) {
      s.sweep += 1;
      const bool r = d.reunit_every > 0 && (s.sweep % (uint32_t)d.reunit_every) == 0;
      const bool m = d.measure_every > 0 && (s.sweep % (uint32_t)d.measure_every) == 0;
      s.stage = r ? kStageReunit : (m ? kStageMeasure : 0);
    }
  } else if (s.stage == kStageReunit) {
    const bool m = d.measure_every > 0 && (s.sweep % (uint32_t)d.measure_every) == 0;
    s.stage = m ? kStageMeasure : 0;
  } else {
    s.stage = 0;
  }
  if (s.stage == 0 && s.sweep >= s.target) s.active = 0;
}

__device__ __host__ inline void advance_stage(const ChainDesc &d, ChainState &s) {
  advance_stage(StageParams{d.D, d.reunit_every, d.measure_every}, s);
}

// The state of a chain after this launch's tick.
__device__ __forceinline__ ChainState next_state(const StageParams &p, ChainState s) {
  if (!s.active) {
    s.prev_stage = -1;  // nothing ran: no halo refresh
    return s;
  }
  if (s.stage == kStageMeasure) {
    s.n_meas += 1;
    s.anchor = 0;  // the measurement restarts the bookkeeping if it was set
  }
  advance_stage(p, s);
  return s;
}

__device__ __forceinline__ bool measures(const ChainState &s) { return s.active && s.stage == kStageMeasure; }

// The end of a one-chain launch, by its last warp: finish the measurement
// and advance the chain's state in place (every other warp has read it).
__device__ __forceinline__ void finish_single_chain(const EngineArgs &ea, const ChainDesc &d, const ChainState &cs,
                                                    int par, int lane) {
  if (measures(cs)) {
    __threadfence();  // acquire the partials of every tile
    double *out = d.results + (size_t)(cs.n_meas % (uint32_t)d.result_cap) * (d.nlayers + 1) * kMeasVals;
    finalize_measure(d, d.partials, out);
    if (cs.anchor) restart_bookkeeping(d, out);
  }
  const ChainState st = next_state(StageParams{d.D, d.reunit_every, d.measure_every}, cs);
  if (lane == 0) {
    ea.state[par] = st;
    ea.hdr->done = 0u;
  }
}

// Register variants of the tick kernel: __launch_bounds__(threads, CTAs per
// SM) caps registers at 65536 / (threads x CTAs).  The autotuner times them.
// kRolled: the update keeps its loop over staple directions rolled.
// On the 32^4 workload (one update phase, fresh re-unitarised lattice per
// shape) the best shapes are within 5 % of each other: 128 registers at
// 16 warps per SM is fastest; 96 and 85 registers (spills) are 3-10 % and
// the unconstrained 156 registers (12 warps) 14 % slower.  Dropped after
// measuring: a split into a staple kernel and a heatbath kernel (30 %
// slower), an L1 prefetch of the next staple direction's links (8 %).
template <int V> struct TickBounds;
template <> struct TickBounds<0> { static constexpr int kThreads = 256, kMinBlocks = 2; static constexpr bool kRolled = false; };   // FP32, 128 regs
template <> struct TickBounds<1> { static constexpr int kThreads = 128, kMinBlocks = 5; static constexpr bool kRolled = false; };   // FP32, 96 regs
template <> struct TickBounds<2> { static constexpr int kThreads = 128, kMinBlocks = 5; static constexpr bool kRolled = true; };    // FP32, rolled, 96 regs
template <> struct TickBounds<3> { static constexpr int kThreads = 256, kMinBlocks = 2; static constexpr bool kRolled = true; };    // FP32, rolled, 128 regs
template <> struct TickBounds<4> { static constexpr int kThreads = 256, kMinBlocks = 3; static constexpr bool kRolled = true; };    // FP32, rolled, 85 regs
template <> struct TickBounds<10> { static constexpr int kThreads = 256, kMinBlocks = 1; static constexpr bool kRolled = false; };  // FP64

// WT: compiled for engines holding a two-coupling DLT chain (any chain with
// beta1 != beta); unweighted chains compute identically in both forms.
// SUB: compiled for a chain divided into sublattice boxes (one chain per
// engine); a halo refresh follows every launch.
// MC (with TOR, FP32 12-real variant 0 only): compiled for such engines with
// several chains.  A CTA's tiles then belong to a new chain almost every
// time (tiles are dealt out in grid-stride order), and each switch waited
// behind a CTA barrier for the new descriptor's round trip to L2; this form
// stages the chain of the CTA's next tile in shared memory with cp.async
// while the current tile runs.  It is a form of its own because the
// staging code, even when not executed, slowed the single-chain update by
// 0.6 %.
// TOR: compiled for engines whose chains are all undivided periodic 4-D tori
// with one coupling and the default random-number key (the benchmark's
// lattices and most ensembles): the unrolled update with D, the layer and
// the site key fixed at compile time.
template <class S, int V, bool WT, bool SUB = false, bool TOR = false, bool MC = false>
__global__ void __launch_bounds__(TickBounds<V>::kThreads, TickBounds<V>::kMinBlocks) k_tick(EngineArgs ea) {
  __shared__ std::conditional_t<MC, ChainStaging, NoStaging> stg;
  __shared__ ChainDesc sd;
  __shared__ ChainState ss;  // the current chain's current state
  __shared__ int s_par;      // the state slot that holds the current states
  __shared__ double s_red[32 * kPartVals];
  // Launched as a programmatic dependent (pdl), this tick may be scheduled
  // before the previous kernel of the stream has finished: wait for its
  // completion and memory before touching anything, then let the next tick
  // be scheduled.  Both are no-ops for an ordinary launch.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int total = ea.hdr->total_tiles;
  const int nchains = ea.hdr->nchains;
  int cur = -1;
  uint32_t np = 0, na = 0;  // FHKP counters of the current chain, flushed per warp
  bool wrote_partials = false;  // this thread wrote data that the last warp reads
  bool staged = false;  // (MC) stg holds the chain of this CTA's next tile
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int c = __ldg(ea.tile_chain + t);  // the same for every thread of the CTA
    int cn = -1;  // (MC) the chain of the CTA's next tile
    if constexpr (MC) cn = t + (int)gridDim.x < total ? __ldg(ea.tile_chain + t + gridDim.x) : -1;
    if (c != cur) {
      if (cur >= 0) flush_counters(sd, np, na);
      if constexpr (MC)
        if (staged) asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();  // every warp is done with the previous descriptor (MC: staged copies visible)
      if constexpr (MC) {
        if (staged)
          take_staged(sd, ss, stg);
        else
          load_chain(ea, c, sd, ss, s_par);
      } else {
        load_chain(ea, c, sd, ss, s_par);
      }
      __syncthreads();
      cur = c;
    }
    if constexpr (MC) {
      // the next tile belongs to another chain: stage it now (its buffer was
      // last read between the barriers above)
      staged = cn >= 0 && cn != c;
      if (staged) stage_chain(ea, cn, s_par, stg);
    }
    if (!ss.active) continue;
    const int lt = t - sd.tile_base;
    const int layer = lt / sd.tiles_per_vl;  // a layer, or a sublattice box of one
    const int jj = (lt - layer * sd.tiles_per_vl) * blockDim.x + threadIdx.x;
    const bool valid = jj < sd.Vn;
    if (ss.stage < 2 * sd.D) {
      const int colour = ss.stage / sd.D, mu = ss.stage - colour * sd.D;
      typename S::R dr = 0;  // change of Re Tr(U A), in the kernel's precision
      if (valid) {
        if constexpr (TOR)
          update_site_lean<S, false, 4>(sd, ss.sweep, colour, mu, layer, jj, np, na, dr);
        else if constexpr (!TickBounds<V>::kRolled && !SUB)
          update_site_lean<S, WT>(sd, ss.sweep, colour, mu, layer, jj, np, na, dr);
        else
          update_site<S, TickBounds<V>::kRolled, WT, SUB>(sd, ss.sweep, colour, mu, layer, jj, np, na, dr);
      }
      // book the action change S = sum_p beta_p (1 - Re Tr U_p / 3): each warp
      // owns the slot of its 32 sites, so the one fire-and-forget add per warp
      // meets no other add in this launch and the order of adds is fixed
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dr += __shfl_down_sync(0xffffffffu, dr, o);
      // (a warp of the ragged last tile with no valid site has no slot)
      if ((threadIdx.x & 31) == 0 && valid && sd.action_slots) {
        const int slot = layer * ((sd.Vn + 31) >> 5) + (jj >> 5);
        if (in_bounds(slot, sd.n_action_slots, kBoundsSlot))
          atomicAdd(sd.action_slots + slot, sd.action_factor * (double)dr);
      }
    } else if (ss.stage == kStageReunit) {
      if (valid) reunit_site<S, SUB>(sd, layer, jj);
    } else {
      double v[kPartVals] = {0, 0, 0, 0};
      if (valid) measure_site<S, SUB>(sd, layer, jj, v);
      block_reduce(v, s_red);
      if (threadIdx.x == 0 && in_bounds(lt, sd.nlayers * sd.tiles_per_layer, kBoundsPartial)) {
        for (int k = 0; k < kPartVals; ++k) sd.partials[(size_t)lt * kPartVals + k] = v[k];
        wrote_partials = true;
      }
    }
  }
  if (cur >= 0) flush_counters(sd, np, na);
  // The end of the launch's stage machine.  Counting warps, not CTAs, lets a
  // warp leave as soon as its own work is done (no CTA-wide barrier at the
  // end).  Writers of what a later warp of this launch reads (measurement
  // partials; with several chains also next states and the measuring list)
  // fence before counting (release); link stores and counter adds are
  // ordered for the next launch by the launch boundary.
  // One chain: the last warp to finish advances it in place, from its CTA's
  // shared copies (no global reads); the parity stays.  Every warp of a
  // one-chain launch takes this path, so that exactly one count per warp
  // is made.
  // Several chains: the first warp to finish writes every chain's next state
  // into the chain's other state slot (the current slot is only read during
  // a launch, so this overlaps the tiles still running) and lists the chains
  // that measure in this tick; then it counts itself a second time.  The
  // warp whose count completes the grid's warps + 1 finishes those
  // measurements and flips the parity.  (Reading and advancing hundreds of
  // chain states at the end of the launch, by the last warp, had kept the
  // rest of the GPU idle for several microseconds per tick.)
  const int lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  constexpr uint32_t kMeasFlag = 0x80000000u;
  uint32_t prev = 0;
  if (lane == 0) {
    if (wrote_partials) __threadfence();
    prev = atomicAdd(&ea.hdr->done, 1u);
  }
  prev = __shfl_sync(0xffffffffu, prev, 0);
  const int par = cur >= 0 ? s_par : __ldcg(&ea.hdr->parity);
  if (nchains == 1) {
    if (prev != nwarps - 1) return;
    // (a CTA of a grid captured for more tiles than the engine now has can
    // have run no tile: it reads the chain from global memory)
    if (cur == 0)
      finish_single_chain(ea, sd, ss, par, lane);
    else
      finish_single_chain(ea, ea.desc[0], ea.state[par], par, lane);
    return;
  }
  int nmeas = -1;  // known to the first warp; the others read it when flagged
  if (prev == 0) {
    nmeas = 0;
    {
      // every chain's state read once, four per lane in flight; the
      // measuring chains listed in chain order (ballot prefix)
      constexpr int kU = 4;
      for (int base = 0; base < nchains; base += 32 * kU) {
        ChainState st[kU];
        StageParams sp[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int c = base + 32 * u + lane;
          if (c < nchains) {
            st[u] = ea.state[2 * (size_t)c + par];
            const ChainDesc &d = ea.desc[c];
            sp[u] = StageParams{d.D, d.reunit_every, d.measure_every};
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int c = base + 32 * u + lane;
          const bool m = c < nchains && measures(st[u]);
          const unsigned mask = __ballot_sync(0xffffffffu, m);
          if (m) {
            const int slot = nmeas + __popc(mask & ((1u << lane) - 1u));
            if (in_bounds(slot, nchains, kBoundsSlot)) ea.meas_list[slot] = c;
          }
          nmeas += __popc(mask);
          if (c < nchains) ea.state[2 * (size_t)c + (par ^ 1)] = next_state(sp[u], st[u]);
        }
      }
    }
    if (lane == 0) ea.hdr->n_meas = nmeas;
    __threadfence();  // each lane's next states and list entries before the count
    __syncwarp();
    if (lane == 0) prev = atomicAdd(&ea.hdr->done, 1u | (nmeas ? kMeasFlag : 0u));
    prev = __shfl_sync(0xffffffffu, prev, 0);
  }
  if ((prev & ~kMeasFlag) != nwarps) return;
  // The last count: finish the listed measurements, flip the parity.
  if (nmeas < 0) nmeas = (prev & kMeasFlag) ? -2 : 0;
  if (nmeas != 0) {
    __threadfence();  // acquire the tiles' partials, the list and its length
    if (nmeas < 0) nmeas = __ldcg(&ea.hdr->n_meas);
    for (int i = 0; i < nmeas && i < nchains; ++i) {
      const int c = __ldcg(ea.meas_list + i);
      if (!in_bounds(c, nchains, kBoundsSlot)) continue;
      const ChainDesc &d = ea.desc[c];
      // the current slot: this tick's measurement count and anchor
      const ChainState &s = ea.state[2 * (size_t)c + par];
      double *out = d.results + (size_t)(s.n_meas % (uint32_t)d.result_cap) * (d.nlayers + 1) * kMeasVals;
      finalize_measure(d, d.partials, out);
      if (s.anchor) restart_bookkeeping(d, out);
    }
  }
  if (lane == 0) {
    ea.hdr->parity = par ^ 1;
    ea.hdr->done = 0u;
  }
}

// ------------------------------------------------------------------ stand-alone measurement

// The CTA's shared copy of a chain descriptor (a per-thread copy of the
// struct would live in local memory).
__device__ __forceinline__ void desc_to_shared(ChainDesc &dst, const ChainDesc *src) {
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(ChainDesc) / 4); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

template <class S>
__global__ void __launch_bounds__(256) k_measure(ChainDesc *desc_dev) {
  __shared__ double s_red[32 * kPartVals];
  __shared__ ChainDesc d;
  desc_to_shared(d, desc_dev);
  const int total = d.tiles_per_layer * d.nlayers;
  for (int lt = blockIdx.x; lt < total; lt += gridDim.x) {
    const int layer = lt / d.tiles_per_layer;
    const int jj = (lt - layer * d.tiles_per_layer) * blockDim.x + threadIdx.x;
    double v[kPartVals] = {0, 0, 0, 0};
    if (jj < d.Vh) measure_site<S>(d, layer, jj, v);
    block_reduce(v, s_red);
    if (threadIdx.x == 0 && in_bounds(lt, total, kBoundsPartial))
      for (int k = 0; k < kPartVals; ++k) d.partials[(size_t)lt * kPartVals + k] = v[k];
  }
}

__global__ void k_measure_finalize(ChainDesc *desc_dev, double *out) {
  const ChainDesc d = *desc_dev;
  finalize_measure(d, d.partials, out);
}

// Sum of a chain's booked action changes, one warp, fixed order.
__global__ void k_action_sum(const double *slots, int n, double *out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) v += slots[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

// Arm every chain of an engine for n more sweeps, in stream order (the host
// mirror does the same): no host buffer, so nothing to synchronise on.
// Both state slots of a chain hold its current state between launches
// as far as the host-visible fields go: arm them both (the next launch
// overwrites the one that is not current).
__global__ void k_arm(ChainState *state, int nchains, uint32_t n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * nchains; i += gridDim.x * blockDim.x) {
    ChainState s = state[i];
    s.target = s.sweep + n;
    s.active = 1;
    state[i] = s;
  }
}

// Set the bookkeeping-restart flag of one chain (both state slots), in
// stream order.
__global__ void k_set_anchor(ChainState *state, int value) {
  state[0].anchor = value;
  state[1].anchor = value;
}

cudaError_t launch_set_anchor(ChainState *state, int value, cudaStream_t st) {
  k_set_anchor<<<1, 1, 0, st>>>(state, value);
  return cudaGetLastError();
}

cudaError_t launch_arm(ChainState *state, int nchains, uint32_t n, cudaStream_t st) {
  if (nchains <= 0) return cudaSuccess;
  const int grid = (nchains + 255) / 256 < 1024 ? (nchains + 255) / 256 : 1024;
  k_arm<<<grid, 256, 0, st>>>(state, nchains, n);
  return cudaGetLastError();
}

cudaError_t launch_action_sum(const double *slots, int n, double *out, cudaStream_t st) {
  k_action_sum<<<1, 32, 0, st>>>(slots, n, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ start configurations

template <class S>
__global__ void k_start(ChainDesc *desc_dev, int hot) {
  __shared__ ChainDesc d;
  desc_to_shared(d, desc_dev);
  const size_t nl = (size_t)d.nlayers * 2 * d.D * d.Vh;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nl; i += (size_t)gridDim.x * blockDim.x) {
    const int jj = (int)(i % d.Vh);
    size_t r = i / d.Vh;
    const int mu = (int)(r % d.D);
    r /= d.D;
    const int colour = (int)(r % 2);
    const int layer = (int)(r / 2);
    M3<double> m = m3_zero<double>();
    if (!hot) {
      m.e[0][0].re = m.e[1][1].re = m.e[2][2].re = 1.0;
    } else {
      // Haar SU(3): Gaussian rows 1, 2 (Box-Muller), Gram-Schmidt, cross product.
      const SiteGeo g = site_of(d, layer, colour, jj);
      const uint32_t key = site_key(d, g);
      double gs[12];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const uint4 w = philox4x32_10(make_uint4(key, (uint32_t)mu, (uint32_t)b, kPurposeStart),
                                      make_uint2(d.seed_lo, d.seed_hi));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const double rad = sqrt(-2.0 * log(unif_d(ws[2 * p])));
          double sn, cs;
          sincospi(2.0 * unif_d(ws[2 * p + 1]), &sn, &cs);
          gs[4 * b + 2 * p] = rad * cs;
          gs[4 * b + 2 * p + 1] = rad * sn;
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        m.e[0][k] = {gs[2 * k], gs[2 * k + 1]};
        m.e[1][k] = {gs[6 + 2 * k], gs[6 + 2 * k + 1]};
      }
      reunit_d(m);
    }
    S::store(plane_ptr<S>(d, layer, colour, mu), d.Vh, jj, m3_cast<typename S::R>(m));
  }
}

// ------------------------------------------------------------------ canonical layout <-> storage

template <class S>
__global__ void k_convert(ChainDesc *desc_dev, double *canon, int to_canonical) {
  __shared__ ChainDesc d;
  desc_to_shared(d, desc_dev);
  const size_t nlinks = (size_t)d.nlayers * d.V * d.D;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nlinks; i += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(i % d.D);
    const size_t ls = i / d.D;
    const int s = (int)(ls % d.V);
    const int layer = (int)(ls / d.V);
    // colour of site s: parity of its coordinate sum
    int r = s, sum = 0;
    for (int k = 0; k < d.D; ++k) {
      const int n = d.dims[k];
      sum += r % n;
      r /= n;
    }
    const int colour = sum & 1;
    typename S::Vec *p = plane_ptr<S>(d, layer, colour, mu);
    double *c = canon + i * 18;
    if (to_canonical) {
      const M3<typename S::R> m = S::load(p, d.Vh, s >> 1);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          c[(a * 3 + b) * 2] = (double)m.e[a][b].re;
          c[(a * 3 + b) * 2 + 1] = (double)m.e[a][b].im;
        }
    } else {
      M3<typename S::R> m;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m.e[a][b] = {(typename S::R)c[(a * 3 + b) * 2], (typename S::R)c[(a * 3 + b) * 2 + 1]};
      S::store(p, d.Vh, s >> 1, m);
    }
  }
}

// ------------------------------------------------------------------ sublattice boxes
// The paper's boundary exchange (Sec. 2.4: faces, and corners when two or
// more directions are divided) restated as device copies: every halo site
// of every box takes its links from the interior site that owns it in the
// undivided lattice (periodic wrap; a wrap across a glued boundary of the
// double-layered torus lands in the other layer).  Halo sites are never
// sources, so the copies do not race.

// Refresh the halos of a divided chain: all links (all = 1, after a start,
// set_links or re-unitarisation) or, after an update tick, only the
// (colour, direction) that the tick changed.  Threads run over the box's
// list of halo sites of that colour (blockIdx.y = box): the owner is the
// same padded site of the neighbouring box given by the entry's offset
// code, whose box coordinate wraps periodically; a wrap across a glued
// boundary of the double-layered torus lands in the other layer.
template <class S>
__global__ void k_halo(const ChainDesc *desc_dev, const ChainState *state_dev, const EngineHeader *hdr, int all) {
  const ChainDesc &d = *desc_dev;
  int c0 = 0, c1 = 2, m0 = 0, m1 = d.D;
  if (!all) {
    const int ps = state_dev[hdr->parity].prev_stage;  // the chain's current state slot
    if (ps >= 0 && ps < 2 * d.D) {
      c0 = ps / d.D;
      c1 = c0 + 1;
      m0 = ps - c0 * d.D;
      m1 = m0 + 1;
    } else if (ps != kStageReunit) {
      return;  // a measurement, or nothing ran: no link changed
    }
  }
  const int vl = blockIdx.y;
  const int L = vl / d.nb;
  int bc[kMaxD], rest = vl - L * d.nb;
#pragma unroll
  for (int k = 0; k < kMaxD; ++k) {
    bc[k] = 0;
    if (k < d.D) {
      bc[k] = rest % d.bdiv[k];
      rest /= d.bdiv[k];
    }
  }
  const int first = c0 == 0 ? 0 : d.halo_n[0];
  const int count = (c0 == 0 ? d.halo_n[0] : 0) + (c1 == 2 ? d.halo_n[1] : 0);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const int4 h = d.halo[first + e];
    const int colour = (first + e) < d.halo_n[0] ? 0 : 1;
    int bsrc = 0, bmul = 1, flip = 0;
#pragma unroll
    for (int k = 0; k < kMaxD; ++k)
      if (k < d.D) {
        const int code = (h.z >> (2 * k)) & 3;
        int o = bc[k] + (code == 1 ? -1 : (code == 2 ? 1 : 0));
        if (o < 0 || o >= d.bdiv[k]) {
          o = o < 0 ? o + d.bdiv[k] : o - d.bdiv[k];
          if (d.nlayers == 2) flip ^= (d.glue_mask >> k) & 1;
        }
        bsrc += o * bmul;
        bmul *= d.bdiv[k];
      }
    const int vsrc = (L ^ flip) * d.nb + bsrc;
    for (int mu = m0; mu < m1; ++mu)
      S::copy(plane_ptr<S>(d, vl, colour, mu), d.Vh, h.x >> 1, plane_ptr<S>(d, vsrc, colour, mu), d.Vh, h.y >> 1);
  }
}

// Copy links between the undivided layout (plain) and the sublattice boxes
// (sub): to_sub = 1 scatters into the box interiors, 0 gathers from them.
template <class S>
__global__ void k_sub_copy(const ChainDesc *sub_dev, const ChainDesc *plain_dev, int to_sub) {
  const ChainDesc &d = *sub_dev;
  const ChainDesc &p = *plain_dev;
  const size_t nlinks = (size_t)p.nlayers * p.V * p.D;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nlinks; i += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(i % p.D);
    const size_t ls = i / p.D;
    const int s = (int)(ls % p.V);
    const int L = (int)(ls / p.V);
    int r = s, par = 0, b = 0, bmul = 1, sp = 0;
    for (int k = 0; k < p.D; ++k) {
      const int gx = r % p.dims[k];
      r /= p.dims[k];
      par += gx;
      const int bo = gx / d.idims[k];
      b += bo * bmul;
      bmul *= d.bdiv[k];
      sp += (gx - bo * d.idims[k] + d.hpad[k]) * d.stride[k];
    }
    const int colour = par & 1;
    typename S::Vec *pv = plane_ptr<S>(p, L, colour, mu);
    typename S::Vec *sv = plane_ptr<S>(d, L * d.nb + b, colour, mu);
    if (to_sub)
      S::copy(sv, d.Vh, sp >> 1, pv, p.Vh, s >> 1);
    else
      S::copy(pv, p.Vh, s >> 1, sv, d.Vh, sp >> 1);
  }
}

// Links given as rows 1 and 2 in float (12 per link, canonical site order:
// [layer][i_s - 1][mu][row][col][re, im]); row 3 = conj(row1 x row2).
template <class S>
__global__ void k_convert_rows2(ChainDesc *desc_dev, const float *src) {
  __shared__ ChainDesc d;
  desc_to_shared(d, desc_dev);
  const size_t nlinks = (size_t)d.nlayers * d.V * d.D;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nlinks; i += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(i % d.D);
    const size_t ls = i / d.D;
    const int s = (int)(ls % d.V);
    const int layer = (int)(ls / d.V);
    int r = s, sum = 0;
    for (int k = 0; k < d.D; ++k) {
      const int n = d.dims[k];
      sum += r % n;
      r /= n;
    }
    const float4 *c = reinterpret_cast<const float4 *>(src + i * 12);
    const float4 q0 = c[0], q1 = c[1], q2 = c[2];
    using R = typename S::R;
    M3<R> m;
    m.e[0][0] = {(R)q0.x, (R)q0.y};
    m.e[0][1] = {(R)q0.z, (R)q0.w};
    m.e[0][2] = {(R)q1.x, (R)q1.y};
    m.e[1][0] = {(R)q1.z, (R)q1.w};
    m.e[1][1] = {(R)q2.x, (R)q2.y};
    m.e[1][2] = {(R)q2.z, (R)q2.w};
    third_row(m);
    S::store(plane_ptr<S>(d, layer, sum & 1, mu), d.Vh, s >> 1, m);
  }
}

// ------------------------------------------------------------------ measurement without allocation
// For callers that cannot allocate device memory (see su3_measure_noalloc):
// the per-tile partial sums go to a fixed array in the library's own device
// memory instead of a buffer from cudaMalloc.  Every tile writes its own
// slots before the finishing kernel reads them, so nothing has to start at
// zero; calls that overlap on the GPU share the array and race.

constexpr int kNoAllocTiles = 32768;  // 32768 tiles x 4 doubles = 1 MiB
static __device__ __align__(256) double g_noalloc_partials[kNoAllocTiles * kPartVals];

template <class S>
__global__ void __launch_bounds__(256) k_measure_noalloc(ChainDesc d, double *partials) {
  __shared__ double s_red[32 * kPartVals];
  const int total = d.tiles_per_layer * d.nlayers;
  for (int lt = blockIdx.x; lt < total; lt += gridDim.x) {
    const int layer = lt / d.tiles_per_layer;
    const int jj = (lt - layer * d.tiles_per_layer) * blockDim.x + threadIdx.x;
    double v[kPartVals] = {0, 0, 0, 0};
    if (jj < d.Vh) measure_site<S>(d, layer, jj, v);
    block_reduce(v, s_red);
    if (threadIdx.x == 0 && in_bounds(lt, kNoAllocTiles, kBoundsPartial))
      for (int k = 0; k < kPartVals; ++k) partials[(size_t)lt * kPartVals + k] = v[k];
  }
}

__global__ void k_measure_finalize_noalloc(ChainDesc d, const double *partials, double *out) {
  finalize_measure(d, partials, out);
}

int noalloc_max_tiles() { return kNoAllocTiles; }

// The unique id of the current context (cuCtxGetId), or 0 when there is no
// current context or the driver cannot say.  The two driver calls are
// reached through the runtime's entry-point table, so the library does not
// link the driver library itself.
static unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(p);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array in the current context.  Host code
// cannot use the symbol itself (it names a host-side stand-in), so the
// address is looked up with cudaGetSymbolAddress.  It is kept per device
// together with the id of the context it was taken in: a device reset
// (cudaDeviceReset) or any other teardown of the context unloads the
// library's module, and the next call then sees a new context id and looks
// the address up again instead of using a stale one.  Without a context id
// the address is looked up on every call.
static cudaError_t noalloc_scratch(double **ptr) {
  static std::mutex mu;
  static double *addr[64] = {nullptr};
  static unsigned long long ctx_of[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  const unsigned long long id = current_context_id();
  if (id && ctx_of[dev] == id && addr[dev]) {
    *ptr = addr[dev];
    return cudaSuccess;
  }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // also makes the device's context current
  if (e != cudaSuccess) return e;
  addr[dev] = static_cast<double *>(p);
  ctx_of[dev] = current_context_id();
  *ptr = addr[dev];
  return cudaSuccess;
}

// Run f with a value of the storage form of `storage` (0: FP64 18-real,
// 1: FP32 12-real, 2: FP32 18-real); f launches the kernels of that form.
template <class F>
static cudaError_t by_storage(int storage, F &&f) {
  switch (storage) {
    case 0: return f(StoreF64x18{});
    case 2: return f(StoreF32x18{});
    default: return f(StoreF32x12{});
  }
}

cudaError_t launch_measure_noalloc(int storage, const ChainDesc &d, int block, double *out, cudaStream_t st) {
  double *partials = nullptr;
  cudaError_t e = noalloc_scratch(&partials);
  if (e != cudaSuccess) return e;
  const int tiles = d.tiles_per_layer * d.nlayers;
  const int grid = tiles < 4096 ? tiles : 4096;
  return by_storage(storage, [&](auto s) {
    k_measure_noalloc<decltype(s)><<<grid, block, 0, st>>>(d, partials);
    k_measure_finalize_noalloc<<<1, 32, 0, st>>>(d, partials, out);
    return cudaGetLastError();
  });
}

// ------------------------------------------------------------------ debug bounds checks (host side)

// A deliberate out-of-range index checked by the device predicate; nothing
// is accessed, only the violation record is written.
__global__ void k_bounds_selftest() { (void)in_bounds(1, 1, kBoundsSelfTest); }

bool debug_bounds_build() {
#ifdef SU3_DEBUG_BOUNDS
  return true;
#else
  return false;
#endif
}

cudaError_t bounds_record(unsigned long long out[3]) {
  out[0] = out[1] = out[2] = 0;
#ifdef SU3_DEBUG_BOUNDS
  return cudaMemcpyFromSymbol(out, g_bounds, 3 * sizeof(unsigned long long));
#else
  return cudaSuccess;
#endif
}

cudaError_t launch_bounds_selftest() {
  k_bounds_selftest<<<1, 1>>>();
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : cudaDeviceSynchronize();
}

// ------------------------------------------------------------------ launchers
// Tick kernel forms: FP32 12-real has variants 0..4 (TickBounds), FP32
// 18-real variant 0 only, FP64 its one form (10).  A chain divided into
// sublattice boxes runs one form: FP32 the rolled 128-register variant (3).

constexpr int kSubVariant = 3;

int tick_variants(int storage) { return storage == 1 ? 5 : 1; }

// pdl: launch as a programmatic dependent of the previous kernel in the
// stream (the tick waits for that kernel's completion and memory at its
// first instruction, so only the launch itself overlaps the previous tick).
template <class S, int V, bool WT, bool SUB = false, bool TOR = false, bool MC = false>
static cudaError_t tick_v(const EngineArgs &ea, int grid, int block, cudaStream_t st, bool pdl) {
  if (!pdl) {
    k_tick<S, V, WT, SUB, TOR, MC><<<grid, block, 0, st>>>(ea);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tick<S, V, WT, SUB, TOR, MC>, ea);
}

template <class S, int V, bool WT, bool SUB = false, bool TOR = false, bool MC = false>
static cudaError_t occ_v(int block, int *ctas) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_tick<S, V, WT, SUB, TOR, MC>, block, 0);
}

int tick_max_threads(int storage, int variant) {
  if (storage == 0) return TickBounds<10>::kThreads;
  if (storage == 2) return TickBounds<0>::kThreads;
  switch (variant) {
    case 0: return TickBounds<0>::kThreads;
    case 1: return TickBounds<1>::kThreads;
    case 2: return TickBounds<2>::kThreads;
    case 3: return TickBounds<3>::kThreads;
    default: return TickBounds<4>::kThreads;
  }
}

// One switch for launching and for occupancy queries: OP<S, V, WT, SUB, TOR, MC>.
// torus: 0 none, 1 the torus form, 2 the torus form for several chains.
// The torus form exists for the unrolled float variants (FP32 12-real 0 and
// 1, FP32 18-real 0), its multi-chain form for FP32 12-real variant 0 (the
// others run the plain torus form); the remaining forms ignore `torus`.
template <template <class, int, bool, bool, bool, bool> class OP, bool WT, class... A>
static cudaError_t tick_dispatch(int storage, int variant, bool sub, int torus, A... a) {
  const bool tor = torus != 0 && !sub && !WT, mc = tor && torus == 2;
  if (storage == 0) return sub ? OP<StoreF64x18, 10, WT, true, false, false>::run(a...) : OP<StoreF64x18, 10, WT, false, false, false>::run(a...);
  if (storage == 2) {
    if (sub) return OP<StoreF32x18, kSubVariant, WT, true, false, false>::run(a...);
    return tor ? OP<StoreF32x18, 0, false, false, true, false>::run(a...) : OP<StoreF32x18, 0, WT, false, false, false>::run(a...);
  }
  if (sub) return OP<StoreF32x12, kSubVariant, WT, true, false, false>::run(a...);
  switch (variant) {
    case 0:
      if (mc) return OP<StoreF32x12, 0, false, false, true, true>::run(a...);
      return tor ? OP<StoreF32x12, 0, false, false, true, false>::run(a...) : OP<StoreF32x12, 0, WT, false, false, false>::run(a...);
    case 1: return tor ? OP<StoreF32x12, 1, false, false, true, false>::run(a...) : OP<StoreF32x12, 1, WT, false, false, false>::run(a...);
    case 2: return OP<StoreF32x12, 2, WT, false, false, false>::run(a...);
    case 3: return OP<StoreF32x12, 3, WT, false, false, false>::run(a...);
    default: return OP<StoreF32x12, 4, WT, false, false, false>::run(a...);
  }
}

template <class S, int V, bool WT, bool SUB, bool TOR, bool MC = false>
struct TickLaunch {
  static cudaError_t run(const EngineArgs *ea, int grid, int block, cudaStream_t st, bool pdl) {
    return tick_v<S, V, WT, SUB, TOR, MC>(*ea, grid, block, st, pdl);
  }
};

template <class S, int V, bool WT, bool SUB, bool TOR, bool MC = false>
struct TickOccupancy {
  static cudaError_t run(int block, int *ctas) { return occ_v<S, V, WT, SUB, TOR, MC>(block, ctas); }
};

cudaError_t launch_tick(int storage, int variant, bool weighted, bool sub, int torus, const EngineArgs &ea, int grid,
                        int block, cudaStream_t st, bool pdl) {
  if (sub) variant = storage == 0 ? 0 : kSubVariant;
  if (block > tick_max_threads(storage, variant)) return cudaErrorInvalidConfiguration;
  const EngineArgs *pa = &ea;
  return weighted ? tick_dispatch<TickLaunch, true>(storage, variant, sub, torus, pa, grid, block, st, pdl)
                  : tick_dispatch<TickLaunch, false>(storage, variant, sub, torus, pa, grid, block, st, pdl);
}

cudaError_t launch_halo(int storage, const ChainDesc *desc_dev, const ChainState *state_dev, const EngineHeader *hdr,
                        int all, int boxes, int halo_sites, cudaStream_t st) {
  const int block = 256;
  const dim3 grid((unsigned)((halo_sites + block - 1) / block > 0 ? (halo_sites + block - 1) / block : 1),
                  (unsigned)boxes);
  return by_storage(storage, [&](auto s) {
    k_halo<decltype(s)><<<grid, block, 0, st>>>(desc_dev, state_dev, hdr, all);
    return cudaGetLastError();
  });
}

static int copy_grid(size_t nlinks, int block) {
  return (int)((nlinks + block - 1) / block < 65536 ? (nlinks + block - 1) / block : 65536);
}

cudaError_t launch_sub_copy(int storage, const ChainDesc *sub_dev, const ChainDesc *plain_dev, size_t nlinks,
                            int to_sub, cudaStream_t st) {
  const int block = 256, grid = copy_grid(nlinks, block);
  return by_storage(storage, [&](auto s) {
    k_sub_copy<decltype(s)><<<grid, block, 0, st>>>(sub_dev, plain_dev, to_sub);
    return cudaGetLastError();
  });
}

cudaError_t launch_measure(int storage, ChainDesc *desc_dev, int tiles_total, int block, double *out, cudaStream_t st) {
  const int grid = tiles_total < 4096 ? tiles_total : 4096;
  return by_storage(storage, [&](auto s) {
    k_measure<decltype(s)><<<grid, block, 0, st>>>(desc_dev);
    k_measure_finalize<<<1, 32, 0, st>>>(desc_dev, out);
    return cudaGetLastError();
  });
}

cudaError_t launch_start(int storage, ChainDesc *desc_dev, size_t nlinks, int hot, cudaStream_t st) {
  const int block = 256, grid = copy_grid(nlinks, block);
  return by_storage(storage, [&](auto s) {
    k_start<decltype(s)><<<grid, block, 0, st>>>(desc_dev, hot);
    return cudaGetLastError();
  });
}

cudaError_t launch_convert_rows2(int storage, ChainDesc *desc_dev, size_t nlinks, const float *src, cudaStream_t st) {
  const int block = 256, grid = copy_grid(nlinks, block);
  return by_storage(storage, [&](auto s) {
    k_convert_rows2<decltype(s)><<<grid, block, 0, st>>>(desc_dev, src);
    return cudaGetLastError();
  });
}

cudaError_t launch_convert(int storage, ChainDesc *desc_dev, size_t nlinks, double *canon, int to_canonical,
                           cudaStream_t st) {
  const int block = 256, grid = copy_grid(nlinks, block);
  return by_storage(storage, [&](auto s) {
    k_convert<decltype(s)><<<grid, block, 0, st>>>(desc_dev, canon, to_canonical);
    return cudaGetLastError();
  });
}

cudaError_t tick_occupancy(int storage, int variant, bool weighted, bool sub, int torus, int block, int *ctas_per_sm) {
  *ctas_per_sm = 0;
  if (sub) variant = storage == 0 ? 0 : kSubVariant;
  if (block > tick_max_threads(storage, variant)) return cudaSuccess;
  return weighted ? tick_dispatch<TickOccupancy, true>(storage, variant, sub, torus, block, ctas_per_sm)
                  : tick_dispatch<TickOccupancy, false>(storage, variant, sub, torus, block, ctas_per_sm);
}

void host_advance_stage(const ChainDesc &d, ChainState &s) { advance_stage(d, s); }

}  // namespace su3g
