/*
 * su3_oracle.c -- plain, slow, double-precision CPU oracle for the
 * checkerboard Cabibbo-Marinari heatbath of pure SU(3) Wilson-action lattice
 * gauge theory (B. A. Berg, "Fortran MPI Checkerboard Code for SU(3) Lattice
 * Gauge Theory I", arXiv:0904.0642).
 *
 * TEST INFRASTRUCTURE.  This file is the checker that the CUDA library is
 * compared against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA path, and it imports nothing from it.
 *
 * Every function follows the paper's definitions in the paper's order, with
 * no blocking, fusion or reordering:
 *   - site numbering, coordinates and colour: Sec. 2, eqs. (i_s), (xD),
 *     (x^i), (i_c);
 *   - the checkerboard sweep: Sec. 2 and Sec. 2.1 (sequential order, colour by
 *     colour, one link direction at a time);
 *   - Cabibbo-Marinari updating over the three SU(2) subgroups with the
 *     Fabricius-Haan / Kennedy-Pendleton heatbath in the multi-hit
 *     accept/reject form of Fredenhagen-Marcu: Sec. 2.1;
 *   - the double-layered torus (DLT): Sec. 2.2 (two identical lattices, each
 *     the other's boundary in all or only some directions);
 *   - plaquette measurements split into space- and time-like: Sec. 2.4
 *     (the wloops routine) and Table 2.
 * Where the paper is silent (staple orientation, subgroup order, the SU(2)
 * formulas it only cites, the random number generator), the readings used
 * are stated at the function that needs them.
 *
 * Storage ("canonical layout"): links as doubles
 *     U[layer][site][mu][row][col][re,im],
 * site = i_s - 1 with x^1 running fastest (eq. i_s), 18 doubles per matrix.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC11), written here from its published
 * definition.  The paper's Marsaglia generator cannot be reproduced bitwise
 * (the paper itself notes that results are platform dependent, Sec. 3), so
 * the generator is a free choice shared, by definition only, with the GPU.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 8
#define ORC_TWO_PI 6.283185307179586476925286766559

typedef struct {
  int32_t D;                      /* lattice dimension, 2..8 */
  int32_t dims[ORC_MAXD];         /* extents n^1..n^D, all even */
  int32_t nlayers;                /* 1: torus with PBC, 2: double-layered torus */
  int32_t glue_mask;              /* DLT: bit mu set -> the mu boundary leads to the other layer */
  int32_t rng_period[ORC_MAXD];   /* random-number site key uses x^i mod period (0 -> n^i) */
  int32_t layer_blind;            /* 1: both layers draw identical random numbers */
} orc_geom;

typedef double complex cplx;
typedef struct { cplx m[3][3]; } mat3;

/* ------------------------------------------------------------------ */
/* Geometry: Sec. 2, eqs. (i_s), (xD), (x^i), (i_c).                   */
/* ------------------------------------------------------------------ */

int64_t orc_nsites(const orc_geom *g) {
  int64_t v = 1;
  for (int i = 0; i < g->D; ++i) v *= g->dims[i];
  return v;
}

/* n_a^i of eq. (i_s): 1 for the first direction, prod_{j<i} n^j after. */
static int64_t orc_stride(const orc_geom *g, int i) {
  int64_t s = 1;
  for (int j = 0; j < i; ++j) s *= g->dims[j];
  return s;
}

/* eq. (i_s), returned zero-based: i_s - 1 = sum_i x^i n_a^i. */
int64_t orc_site_index(const orc_geom *g, const int32_t *x) {
  int64_t s = 0;
  for (int i = 0; i < g->D; ++i) s += (int64_t)x[i] * orc_stride(g, i);
  return s;
}

/* eqs. (xD) and (x^i): peel the coordinates off from the last direction
 * down, by integer division with n_a^i. */
void orc_site_coords(const orc_geom *g, int64_t s, int32_t *x) {
  int64_t js = s; /* j_s^i - 1 */
  for (int i = g->D - 1; i >= 0; --i) {
    int64_t na = orc_stride(g, i);
    x[i] = (int32_t)(js / na);
    js -= (int64_t)x[i] * na;
  }
}

/* eq. (i_c), returned zero-based: i_c - 1 = mod(sum_i x^i, 2). */
int orc_colour(const orc_geom *g, const int32_t *x) {
  int sum = 0;
  for (int i = 0; i < g->D; ++i) sum += x[i];
  return sum % 2;
}

/* One step from (layer, x) in direction mu, forward (dir=+1) or backward
 * (dir=-1).  On a torus (Sec. 2) the coordinate wraps periodically.  On the
 * DLT (Sec. 2.2) a step that crosses the boundary of a glued direction wraps
 * the coordinate and lands on the other layer; unglued directions stay
 * periodic within the layer. */
void orc_neighbour(const orc_geom *g, int layer, int64_t s, int mu, int dir,
                   int32_t *layer_out, int64_t *s_out) {
  int32_t x[ORC_MAXD];
  orc_site_coords(g, s, x);
  int n = g->dims[mu];
  int crossed = 0;
  if (dir > 0) {
    x[mu] += 1;
    if (x[mu] == n) { x[mu] = 0; crossed = 1; }
  } else {
    x[mu] -= 1;
    if (x[mu] < 0) { x[mu] = n - 1; crossed = 1; }
  }
  int l = layer;
  if (crossed && g->nlayers == 2 && ((g->glue_mask >> mu) & 1)) l = 1 - layer;
  *layer_out = l;
  *s_out = orc_site_index(g, x);
}

/* Every neighbour at once: out[((layer*V + s)*D + mu)*2 + (dir>0)] holds
 * layer'*V + s'.  Used by the tests to check the geometry by brute force. */
void orc_neighbour_table(const orc_geom *g, int64_t *out) {
  int64_t V = orc_nsites(g);
  for (int l = 0; l < g->nlayers; ++l)
    for (int64_t s = 0; s < V; ++s)
      for (int mu = 0; mu < g->D; ++mu)
        for (int d = 0; d < 2; ++d) {
          int32_t l2; int64_t s2;
          orc_neighbour(g, l, s, mu, d ? +1 : -1, &l2, &s2);
          out[(((int64_t)l * V + s) * g->D + mu) * 2 + d] = (int64_t)l2 * V + s2;
        }
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC11), from its published definition: */
/* ten rounds of two 32x32->64 multiplies with the round constants     */
/* M0 = 0xD2511F53, M1 = 0xCD9E8D57 and Weyl key bumps                 */
/* W0 = 0x9E3779B9, W1 = 0xBB67AE85.                                    */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A uniform deviate in (0,1) from one 32-bit word: (w + 1/2) / 2^32.
 * Never 0 or 1, so the logarithms below are always finite. */
static double orc_uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Purposes of a random-number block (fourth counter word). */
#define ORC_PURPOSE_HEATBATH 0u
#define ORC_PURPOSE_START 1u
/* Heatbath tag (third counter word): hit index (255 = the direction draw),
 * SU(2) subgroup, link direction and checkerboard colour. */
#define ORC_HIT_DIRECTION 255u
static uint32_t orc_tag(int colour, int mu, int subgroup, unsigned hit) {
  return (uint32_t)hit | ((uint32_t)subgroup << 8) | ((uint32_t)mu << 10) | ((uint32_t)colour << 14);
}

/* Site key (first counter word): the zero-based site number of
 * (x^i mod period^i) in a lattice of extents period^i, plus layer times that
 * volume on the DLT unless both layers draw the same numbers.  With the
 * default period = n^i this is layer*V + i_s - 1.  A smaller period makes
 * every sublattice of that size draw identical numbers, which is the test of
 * Sec. 3.1 (identical random numbers on sublattices). */
static uint32_t orc_site_key(const orc_geom *g, int layer, int64_t s) {
  int32_t x[ORC_MAXD];
  orc_site_coords(g, s, x);
  int64_t key = 0, stride = 1;
  for (int i = 0; i < g->D; ++i) {
    int p = g->rng_period[i] > 0 ? g->rng_period[i] : g->dims[i];
    key += (int64_t)(x[i] % p) * stride;
    stride *= p;
  }
  if (g->nlayers == 2 && !g->layer_blind) key += (int64_t)layer * stride;
  return (uint32_t)key;
}

static void orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double u[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  for (int i = 0; i < 4; ++i) u[i] = orc_uniform(w[i]);
}

/* ------------------------------------------------------------------ */
/* 3x3 complex matrices (the paper's su3mult routine and friends).      */
/* ------------------------------------------------------------------ */

static mat3 m_load(const double *p) {
  mat3 a;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a.m[i][j] = p[(i * 3 + j) * 2] + I * p[(i * 3 + j) * 2 + 1];
  return a;
}
static void m_store(double *p, const mat3 *a) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      p[(i * 3 + j) * 2] = creal(a->m[i][j]);
      p[(i * 3 + j) * 2 + 1] = cimag(a->m[i][j]);
    }
}
static mat3 m_mul(const mat3 *a, const mat3 *b) {
  mat3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = 0;
      for (int k = 0; k < 3; ++k) s += a->m[i][k] * b->m[k][j];
      c.m[i][j] = s;
    }
  return c;
}
static mat3 m_dag(const mat3 *a) {
  mat3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.m[i][j] = conj(a->m[j][i]);
  return c;
}
static mat3 m_add(const mat3 *a, const mat3 *b) {
  mat3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.m[i][j] = a->m[i][j] + b->m[i][j];
  return c;
}
static mat3 m_zero(void) { mat3 c; memset(&c, 0, sizeof c); return c; }
static mat3 m_unit(void) { mat3 c = m_zero(); for (int i = 0; i < 3; ++i) c.m[i][i] = 1; return c; }
static double m_retr(const mat3 *a) { return creal(a->m[0][0] + a->m[1][1] + a->m[2][2]); }
static cplx m_tr(const mat3 *a) { return a->m[0][0] + a->m[1][1] + a->m[2][2]; }

static const double *link_ptr(const orc_geom *g, const double *U, int layer, int64_t s, int mu) {
  return U + (((int64_t)layer * orc_nsites(g) + s) * g->D + mu) * 18;
}

/* Third row of an SU(3) matrix from its first two: r3 = conj(r1 x r2),
 * which makes the rows orthonormal with determinant one. */
static void m_third_row(mat3 *a) {
  a->m[2][0] = conj(a->m[0][1] * a->m[1][2] - a->m[0][2] * a->m[1][1]);
  a->m[2][1] = conj(a->m[0][2] * a->m[1][0] - a->m[0][0] * a->m[1][2]);
  a->m[2][2] = conj(a->m[0][0] * a->m[1][1] - a->m[0][1] * a->m[1][0]);
}

/* Re-unitarisation (the paper's su3reunit, Sec. 2.4): Gram-Schmidt on the
 * first two rows, then the third row from the cross product. */
static void m_reunit(mat3 *a) {
  double n1 = 0;
  for (int k = 0; k < 3; ++k) n1 += creal(a->m[0][k] * conj(a->m[0][k]));
  n1 = sqrt(n1);
  for (int k = 0; k < 3; ++k) a->m[0][k] /= n1;
  cplx p = 0; /* <r1, r2> = sum_k conj(r1_k) r2_k */
  for (int k = 0; k < 3; ++k) p += conj(a->m[0][k]) * a->m[1][k];
  for (int k = 0; k < 3; ++k) a->m[1][k] -= p * a->m[0][k];
  double n2 = 0;
  for (int k = 0; k < 3; ++k) n2 += creal(a->m[1][k] * conj(a->m[1][k]));
  n2 = sqrt(n2);
  for (int k = 0; k < 3; ++k) a->m[1][k] /= n2;
  m_third_row(a);
}

void orc_reunitarize_matrix(double *u18) {
  mat3 a = m_load(u18);
  m_reunit(&a);
  m_store(u18, &a);
}

void orc_reunitarize(const orc_geom *g, double *U) {
  int64_t n = (int64_t)g->nlayers * orc_nsites(g) * g->D;
  for (int64_t i = 0; i < n; ++i) orc_reunitarize_matrix(U + i * 18);
}

/* ------------------------------------------------------------------ */
/* Start configurations (the paper's istart: 1 ordered, 2 disordered).  */
/* ------------------------------------------------------------------ */

void orc_cold_start(const orc_geom *g, double *U) {
  int64_t n = (int64_t)g->nlayers * orc_nsites(g) * g->D;
  mat3 one = m_unit();
  for (int64_t i = 0; i < n; ++i) m_store(U + i * 18, &one);
}

/* Disordered start, read as Haar-random SU(3): two rows of independent
 * complex Gaussians (Box-Muller from Philox uniforms), Gram-Schmidt, and the
 * third row from the cross product.  Each link draws three Philox blocks with
 * counter (site key, mu, block, START). */
void orc_hot_start(const orc_geom *g, uint64_t seed, double *U) {
  int64_t V = orc_nsites(g);
  for (int l = 0; l < g->nlayers; ++l)
    for (int64_t s = 0; s < V; ++s)
      for (int mu = 0; mu < g->D; ++mu) {
        uint32_t key = orc_site_key(g, l, s);
        double gauss[12];
        for (int b = 0; b < 3; ++b) {
          double u[4];
          orc_draw(seed, key, (uint32_t)mu, (uint32_t)b, ORC_PURPOSE_START, u);
          for (int pair = 0; pair < 2; ++pair) {
            double r = sqrt(-2.0 * log(u[2 * pair]));
            double phi = ORC_TWO_PI * u[2 * pair + 1];
            gauss[4 * b + 2 * pair] = r * cos(phi);
            gauss[4 * b + 2 * pair + 1] = r * sin(phi);
          }
        }
        mat3 a = m_zero();
        for (int k = 0; k < 3; ++k) {
          a.m[0][k] = gauss[2 * k] + I * gauss[2 * k + 1];
          a.m[1][k] = gauss[6 + 2 * k] + I * gauss[6 + 2 * k + 1];
        }
        m_reunit(&a);
        m_store((double *)link_ptr(g, U, l, s, mu), &a);
      }
}

/* ------------------------------------------------------------------ */
/* Staple sum.  The paper's bstaple routines are not printed; this is   */
/* the standard Wilson-action staple, chosen so that the sum of          */
/* Re Tr U_p over the 2(D-1) plaquettes that contain U_mu(x) equals      */
/* Re Tr(U_mu(x) A):                                                     */
/*   A = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+              */
/*                      + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ].     */
/* ------------------------------------------------------------------ */

static mat3 link_at(const orc_geom *g, const double *U, int layer, int64_t s, int mu) {
  return m_load(link_ptr(g, U, layer, s, mu));
}

static mat3 orc_staple_m(const orc_geom *g, const double *U, int layer, int64_t s, int mu) {
  mat3 A = m_zero();
  int32_t lp; int64_t sp;  /* x + mu */
  orc_neighbour(g, layer, s, mu, +1, &lp, &sp);
  for (int nu = 0; nu < g->D; ++nu) {
    if (nu == mu) continue;
    int32_t ln; int64_t sn;    /* x + nu */
    int32_t lm; int64_t sm;    /* x - nu */
    int32_t lpm; int64_t spm;  /* x + mu - nu */
    orc_neighbour(g, layer, s, nu, +1, &ln, &sn);
    orc_neighbour(g, layer, s, nu, -1, &lm, &sm);
    orc_neighbour(g, lp, sp, nu, -1, &lpm, &spm);
    /* upper staple */
    mat3 a = link_at(g, U, lp, sp, nu);
    mat3 b = link_at(g, U, ln, sn, mu); b = m_dag(&b);
    mat3 c = link_at(g, U, layer, s, nu); c = m_dag(&c);
    mat3 t = m_mul(&a, &b);
    mat3 up = m_mul(&t, &c);
    /* lower staple */
    mat3 d = link_at(g, U, lpm, spm, nu); d = m_dag(&d);
    mat3 e = link_at(g, U, lm, sm, mu); e = m_dag(&e);
    mat3 f = link_at(g, U, lm, sm, nu);
    mat3 t2 = m_mul(&d, &e);
    mat3 dn = m_mul(&t2, &f);
    A = m_add(&A, &up);
    A = m_add(&A, &dn);
  }
  return A;
}

void orc_staple(const orc_geom *g, const double *U, int layer, int64_t s, int mu, double *A18) {
  mat3 A = orc_staple_m(g, U, layer, s, mu);
  m_store(A18, &A);
}

/* DLT with two couplings (Sec. 2.2): every link carries the tag of its
 * layer (0 or 1); a plaquette whose tag sum is zero has beta0, any other
 * beta1.  The Wilson weight of a link is then exp((1/3) Re Tr(U A_w)) with
 * the weighted staple A_w = sum over its plaquettes of beta_p times the
 * staple of that plaquette.  Upper staple of nu: plaquette at x with links
 * based at x, x+mu, x+nu, x; lower staple: plaquette at x-nu with links
 * based at x-nu, x+mu-nu, x, x-nu. */
static mat3 orc_staple_weighted_m(const orc_geom *g, const double *U, int layer, int64_t s, int mu, double beta0,
                                  double beta1) {
  mat3 A = m_zero();
  int32_t lp; int64_t sp;
  orc_neighbour(g, layer, s, mu, +1, &lp, &sp);
  for (int nu = 0; nu < g->D; ++nu) {
    if (nu == mu) continue;
    int32_t ln; int64_t sn;
    int32_t lm; int64_t sm;
    int32_t lpm; int64_t spm;
    orc_neighbour(g, layer, s, nu, +1, &ln, &sn);
    orc_neighbour(g, layer, s, nu, -1, &lm, &sm);
    orc_neighbour(g, lp, sp, nu, -1, &lpm, &spm);
    double b_up = (layer + lp + ln + layer) ? beta1 : beta0;
    double b_dn = (lm + lpm + layer + lm) ? beta1 : beta0;
    mat3 a = link_at(g, U, lp, sp, nu);
    mat3 b = link_at(g, U, ln, sn, mu); b = m_dag(&b);
    mat3 c = link_at(g, U, layer, s, nu); c = m_dag(&c);
    mat3 t = m_mul(&a, &b);
    mat3 up = m_mul(&t, &c);
    mat3 d = link_at(g, U, lpm, spm, nu); d = m_dag(&d);
    mat3 e = link_at(g, U, lm, sm, mu); e = m_dag(&e);
    mat3 f = link_at(g, U, lm, sm, nu);
    mat3 t2 = m_mul(&d, &e);
    mat3 dn = m_mul(&t2, &f);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A.m[i][j] += b_up * up.m[i][j] + b_dn * dn.m[i][j];
  }
  return A;
}

void orc_staple_weighted(const orc_geom *g, const double *U, int layer, int64_t s, int mu, double beta0, double beta1,
                         double *A18) {
  mat3 A = orc_staple_weighted_m(g, U, layer, s, mu, beta0, beta1);
  m_store(A18, &A);
}

/* ------------------------------------------------------------------ */
/* SU(2) heatbath (Sec. 2.1: FHKP, multi-hit accept/reject).            */
/* The paper cites the algorithm without formulas; this follows          */
/* Kennedy-Pendleton.  For a subgroup with weight exp(alpha * x0) on      */
/* Haar SU(2), x = (x0, x1, x2, x3):                                      */
/*   per hit, four uniforms u1..u4:                                       */
/*     X = -(ln u1 + cos^2(2 pi u2) ln u3) / alpha   (density ~ sqrt(X) e^{-alpha X}) */
/*     accept when u4^2 <= 1 - X/2, then x0 = 1 - X;                      */
/*   after `hits` rejections the subgroup is left unchanged               */
/*   (Fredenhagen-Marcu, Sec. 2.1);                                       */
/*   on acceptance two more uniforms u5, u6 give the direction of         */
/*   (x1,x2,x3), of length sqrt(1 - x0^2) = sqrt(X (2 - X)):              */
/*     cos(theta) = 2 u5 - 1, phi = 2 pi u6.                              */
/*   u5, u6 are two words of a direction block: subgroups 1 and 2 (of the */
/*   three, counted from 0: subgroups 0 and 1) share the block of         */
/*   subgroup 0, the first taking its words 1, 2 and the second words     */
/*   3, 4; subgroup 2 takes words 1, 2 of its own block.                  */
/* ------------------------------------------------------------------ */

typedef struct {
  int accepted;
  int proposals;
  double x[4];
  double margin; /* smallest |u4^2 - (1 - X/2)| over the hits evaluated */
} orc_su2_draw_t;

static orc_su2_draw_t orc_su2_draw(double alpha, int hits, uint64_t seed, uint32_t c0, uint32_t c1,
                                   int colour, int mu, int subgroup) {
  orc_su2_draw_t r;
  r.accepted = 0;
  r.proposals = 0;
  r.margin = INFINITY;
  r.x[0] = 1; r.x[1] = r.x[2] = r.x[3] = 0;
  double X = 0;
  for (int h = 0; h < hits; ++h) {
    double u[4];
    orc_draw(seed, c0, c1, orc_tag(colour, mu, subgroup, (unsigned)h), ORC_PURPOSE_HEATBATH, u);
    r.proposals++;
    double c = cos(ORC_TWO_PI * u[1]);
    X = -(log(u[0]) + c * c * log(u[2])) / alpha;
    double lhs = u[3] * u[3], rhs = 1.0 - 0.5 * X;
    double m = fabs(lhs - rhs);
    if (m < r.margin) r.margin = m;
    if (lhs <= rhs) { r.accepted = 1; break; }
  }
  if (!r.accepted) return r;
  double u[4];
  orc_draw(seed, c0, c1, orc_tag(colour, mu, subgroup == 1 ? 0 : subgroup, ORC_HIT_DIRECTION), ORC_PURPOSE_HEATBATH,
           u);
  double u5 = subgroup == 1 ? u[2] : u[0], u6 = subgroup == 1 ? u[3] : u[1];
  double costh = 2.0 * u5 - 1.0;
  double sinth = sqrt(1.0 - costh * costh);
  double phi = ORC_TWO_PI * u6;
  double rho = sqrt(X * (2.0 - X));
  r.x[0] = 1.0 - X;
  r.x[1] = rho * sinth * cos(phi);
  r.x[2] = rho * sinth * sin(phi);
  r.x[3] = rho * costh;
  return r;
}

/* The SU(2) matrix of a quaternion a: [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]]. */
static void su2_matrix(const double a[4], cplx m[2][2]) {
  m[0][0] = a[0] + I * a[3];
  m[0][1] = a[2] + I * a[1];
  m[1][0] = -a[2] + I * a[1];
  m[1][1] = a[0] - I * a[3];
}

/* Test hook: n independent draws (counter (i, 0, tag(0,0,subgroup,h))) of the
 * SU(2) heatbath of one subgroup at fixed alpha, with the same routine the
 * sweep uses. */
void orc_su2_samples(double alpha, int hits, uint64_t seed, int64_t n, int subgroup, double *x, int32_t *accepted) {
  for (int64_t i = 0; i < n; ++i) {
    orc_su2_draw_t r = orc_su2_draw(alpha, hits, seed, (uint32_t)i, (uint32_t)(i >> 32), 0, 0, subgroup);
    for (int k = 0; k < 4; ++k) x[4 * i + k] = r.x[k];
    accepted[i] = r.accepted;
  }
}

/* ------------------------------------------------------------------ */
/* Cabibbo-Marinari update of one link (Sec. 2.1).                      */
/* The Wilson weight of the link is exp((beta/3) Re Tr(U A)), beta = 6/g^2 */
/* (the normalisation that gives the plaquette values of Table 2).       */
/* With W = U A, for each subgroup (i,j) in the order (1,2),(1,3),(2,3): */
/*   w = 2x2 block of W on rows/columns (i,j), projected on the          */
/*   quaternions: a0 = Re(w11+w22)/2, a1 = Im(w12+w21)/2,                 */
/*                a2 = Re(w12-w21)/2, a3 = Im(w11-w22)/2;                 */
/*   k = |a|, v = a/k, alpha = 2 beta k / 3, so that                      */
/*   (beta/3) Re Tr(R W) = alpha (r v)_0 + const for R = r embedded;      */
/*   draw x from exp(alpha x0) (above), r = x v^+, U <- R U, W <- R W.    */
/* A subgroup with k below 1e-300 is skipped (the weight is flat there).  */
/* ------------------------------------------------------------------ */

static const int orc_pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};

typedef struct {
  uint64_t proposals, accepts;
  double margin;
  double kmin; /* smallest subgroup norm k seen (how well v = a/k is determined) */
} orc_link_stats;

static void orc_cm_update(mat3 *U, const mat3 *A, double beta, int hits, uint64_t seed, uint32_t site_key,
                          uint32_t sweep, int colour, int mu, orc_link_stats *st) {
  mat3 W = m_mul(U, A);
  for (int sg = 0; sg < 3; ++sg) {
    int i = orc_pairs[sg][0], j = orc_pairs[sg][1];
    double a[4];
    a[0] = 0.5 * (creal(W.m[i][i]) + creal(W.m[j][j]));
    a[1] = 0.5 * (cimag(W.m[i][j]) + cimag(W.m[j][i]));
    a[2] = 0.5 * (creal(W.m[i][j]) - creal(W.m[j][i]));
    a[3] = 0.5 * (cimag(W.m[i][i]) - cimag(W.m[j][j]));
    double k = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
    if (k < st->kmin) st->kmin = k;
    if (k < 1e-300) continue;
    double v[4] = {a[0] / k, a[1] / k, a[2] / k, a[3] / k};
    double alpha = 2.0 * beta * k / 3.0;
    orc_su2_draw_t d = orc_su2_draw(alpha, hits, seed, site_key, sweep, colour, mu, sg);
    st->proposals += (uint64_t)d.proposals;
    st->accepts += (uint64_t)d.accepted;
    if (d.margin < st->margin) st->margin = d.margin;
    if (!d.accepted) continue;
    cplx xm[2][2], vm[2][2], r[2][2];
    su2_matrix(d.x, xm);
    su2_matrix(v, vm);
    for (int p = 0; p < 2; ++p)      /* r = x v^+ */
      for (int q = 0; q < 2; ++q) r[p][q] = xm[p][0] * conj(vm[q][0]) + xm[p][1] * conj(vm[q][1]);
    for (int col = 0; col < 3; ++col) { /* rows i, j of U and W <- r * (rows i, j) */
      cplx ui = U->m[i][col], uj = U->m[j][col];
      U->m[i][col] = r[0][0] * ui + r[0][1] * uj;
      U->m[j][col] = r[1][0] * ui + r[1][1] * uj;
      cplx wi = W.m[i][col], wj = W.m[j][col];
      W.m[i][col] = r[0][0] * wi + r[0][1] * wj;
      W.m[j][col] = r[1][0] * wi + r[1][1] * wj;
    }
  }
}

/* Test hook: one CM update of a single link with a given staple and RNG
 * coordinates, exactly as inside the sweep. */
void orc_link_heatbath(double *u18, const double *A18, double beta, int hits, uint64_t seed, uint32_t site_key,
                       uint32_t sweep, int colour, int mu, uint64_t stats[2]) {
  mat3 U = m_load(u18), A = m_load(A18);
  orc_link_stats st = {0, 0, INFINITY, INFINITY};
  orc_cm_update(&U, &A, beta, hits, seed, site_key, sweep, colour, mu, &st);
  m_store(u18, &U);
  if (stats) { stats[0] += st.proposals; stats[1] += st.accepts; }
}

/* Test hook: n CM updates of one link in a frozen staple A (sweep counter
 * 0..n-1), recording Re Tr(U A) after each. */
void orc_link_chain(double *u18, const double *A18, double beta, int hits, uint64_t seed, int64_t n,
                    double *retr_ua) {
  mat3 U = m_load(u18), A = m_load(A18);
  orc_link_stats st = {0, 0, INFINITY, INFINITY};
  for (int64_t t = 0; t < n; ++t) {
    orc_cm_update(&U, &A, beta, hits, seed, 0u, (uint32_t)t, 0, 0, &st);
    mat3 UA = m_mul(&U, &A);
    retr_ua[t] = m_retr(&UA);
  }
  m_store(u18, &U);
}

/* ------------------------------------------------------------------ */
/* The checkerboard sweep (Sec. 2, Sec. 2.1, the updating routine of    */
/* Sec. 2.4): for colour i_c = 1, 2 and, inside, for each link direction  */
/* mu, every link U_mu(x) with colour(x) = i_c is updated.  Its staple    */
/* touches only links of the other colour or of other directions, so the  */
/* order of sites inside one (colour, direction) phase does not matter;   */
/* here it is increasing i_s, layer by layer.                             */
/* stats (may be NULL): [proposals, accepts] accumulated.                 */
/* margins, kmins (may be NULL): per link, the smallest accept-test margin */
/* and the smallest subgroup norm k seen in these sweeps (canonical link  */
/* order, initialised by the caller).                                     */
/* ------------------------------------------------------------------ */

/* Threads for the sites of one phase (1 unless set).  The links updated in
 * one phase are independent -- each staple reads only links of the other
 * colour or of other directions (Sec. 2) -- and every random number is a
 * function of its counter, so any number of threads gives the same links
 * bit for bit. */
static int orc_threads = 1;

void orc_set_threads(int n) { orc_threads = n < 1 ? 1 : n; }

int orc_available_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

/* One (colour, direction) phase over the sites s_begin <= i_s - 1 < s_end
 * of every layer (the whole phase for [0, V)). */
void orc_phase(const orc_geom *g, double *U, double beta, double beta1, int hits, uint64_t seed, int64_t sweep,
               int colour, int mu, int64_t s_begin, int64_t s_end, uint64_t *stats, double *margins, double *kmins) {
  int64_t V = orc_nsites(g);
  if (s_end > V) s_end = V;
  const int weighted = g->nlayers == 2 && beta1 != beta; /* Sec. 2.2, two couplings */
  for (int l = 0; l < g->nlayers; ++l) {
    uint64_t nprop = 0, nacc = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(orc_threads) schedule(static) reduction(+ : nprop, nacc) if (orc_threads > 1)
#endif
    for (int64_t s = s_begin; s < s_end; ++s) {
      int32_t x[ORC_MAXD];
      orc_site_coords(g, s, x);
      if (orc_colour(g, x) != colour) continue;
      mat3 A = weighted ? orc_staple_weighted_m(g, U, l, s, mu, beta, beta1) : orc_staple_m(g, U, l, s, mu);
      double *p = (double *)link_ptr(g, U, l, s, mu);
      mat3 Ul = m_load(p);
      orc_link_stats st = {0, 0, INFINITY, INFINITY};
      /* with two couplings the staple already carries beta_p */
      orc_cm_update(&Ul, &A, weighted ? 1.0 : beta, hits, seed, orc_site_key(g, l, s), (uint32_t)sweep, colour, mu,
                    &st);
      m_store(p, &Ul);
      nprop += st.proposals;
      nacc += st.accepts;
      int64_t idx = ((int64_t)l * V + s) * g->D + mu;
      if (margins && st.margin < margins[idx]) margins[idx] = st.margin;
      if (kmins && st.kmin < kmins[idx]) kmins[idx] = st.kmin;
    }
    if (stats) { stats[0] += nprop; stats[1] += nacc; }
  }
}

void orc_sweep(const orc_geom *g, double *U, double beta, double beta1, int hits, uint64_t seed, int64_t sweep0,
               int nsweeps, uint64_t *stats, double *margins, double *kmins) {
  int64_t V = orc_nsites(g);
  for (int64_t sw = sweep0; sw < sweep0 + nsweeps; ++sw)
    for (int colour = 0; colour < 2; ++colour)
      for (int mu = 0; mu < g->D; ++mu)
        orc_phase(g, U, beta, beta1, hits, seed, sw, colour, mu, 0, V, stats, margins, kmins);
}

/* ------------------------------------------------------------------ */
/* Observables.                                                          */
/* Plaquette (Sec. 2.4 wloops, Table 2): (1/3) Re Tr of                  */
/*   U_p = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+,  mu < nu,          */
/* averaged over the V D(D-1)/2 plaquettes whose base site x lies in the   */
/* layer; time-like planes contain direction D (V (D-1) of them, the       */
/* paper's mptime), space-like planes do not.  layer < 0 averages over    */
/* all layers.  out = [total, space, time]; space is 0 when D = 2.        */
/* ------------------------------------------------------------------ */

static double orc_plaq_one(const orc_geom *g, const double *U, int l, int64_t s, int mu, int nu) {
  int32_t lp, ln; int64_t sp, sn;
  orc_neighbour(g, l, s, mu, +1, &lp, &sp);
  orc_neighbour(g, l, s, nu, +1, &ln, &sn);
  mat3 a = link_at(g, U, l, s, mu);
  mat3 b = link_at(g, U, lp, sp, nu);
  mat3 c = link_at(g, U, ln, sn, mu); c = m_dag(&c);
  mat3 d = link_at(g, U, l, s, nu); d = m_dag(&d);
  mat3 ab = m_mul(&a, &b);
  mat3 abc = m_mul(&ab, &c);
  mat3 p = m_mul(&abc, &d);
  return m_retr(&p) / 3.0;
}

void orc_plaquette(const orc_geom *g, const double *U, int layer, double out[3]) {
  int64_t V = orc_nsites(g);
  int D = g->D;
  double sum_s = 0, sum_t = 0;
  int64_t n_s = 0, n_t = 0;
  for (int l = 0; l < g->nlayers; ++l) {
    if (layer >= 0 && l != layer) continue;
    for (int64_t s = 0; s < V; ++s)
      for (int mu = 0; mu < D; ++mu)
        for (int nu = mu + 1; nu < D; ++nu) {
          double p = orc_plaq_one(g, U, l, s, mu, nu);
          if (nu == D - 1) { sum_t += p; n_t++; } else { sum_s += p; n_s++; }
        }
  }
  out[0] = (sum_s + sum_t) / (double)(n_s + n_t);
  out[1] = n_s ? sum_s / (double)n_s : 0.0;
  out[2] = sum_t / (double)n_t;
}

/* sum over plaquettes of beta_p (1/3) Re Tr U_p, with beta_p from the tags
 * (layers) of the plaquette's four links: beta1 if any is in layer 1 (Sec.
 * 2.2).  Links of U_p = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ are based at
 * x, x+mu, x+nu and x. */
double orc_action_weighted(const orc_geom *g, const double *U, double beta0, double beta1) {
  int64_t V = orc_nsites(g);
  double sum = 0;
  for (int l = 0; l < g->nlayers; ++l)
    for (int64_t s = 0; s < V; ++s)
      for (int mu = 0; mu < g->D; ++mu)
        for (int nu = mu + 1; nu < g->D; ++nu) {
          int32_t lp, ln; int64_t sp, sn;
          orc_neighbour(g, l, s, mu, +1, &lp, &sp);
          orc_neighbour(g, l, s, nu, +1, &ln, &sn);
          int tags[4] = {l, lp, ln, l};
          int any = 0;
          for (int k = 0; k < 4; ++k) any |= tags[k];
          sum += (any ? beta1 : beta0) * orc_plaq_one(g, U, l, s, mu, nu);
        }
  return sum;
}

/* Polyakov loop (not in the paper): (1/3) Tr of the ordered product of
 * U_D along the closed line that starts at (layer, x, x^D = 0) and follows
 * the forward D neighbour until it returns (length n^D, or 2 n^D on a DLT
 * glued in direction D), averaged over the spatial sites of the layer.
 * layer < 0 averages over all layers.  out = [Re, Im]. */
void orc_polyakov(const orc_geom *g, const double *U, int layer, double out[2]) {
  int64_t V = orc_nsites(g);
  int D = g->D;
  cplx sum = 0;
  int64_t count = 0;
  for (int l = 0; l < g->nlayers; ++l) {
    if (layer >= 0 && l != layer) continue;
    for (int64_t s = 0; s < V; ++s) {
      int32_t x[ORC_MAXD];
      orc_site_coords(g, s, x);
      if (x[D - 1] != 0) continue;
      mat3 P = m_unit();
      int32_t cl = l; int64_t cs = s;
      do {
        mat3 u = link_at(g, U, cl, cs, D - 1);
        P = m_mul(&P, &u);
        int32_t nl; int64_t ns;
        orc_neighbour(g, cl, cs, D - 1, +1, &nl, &ns);
        cl = nl; cs = ns;
      } while (!(cl == l && cs == s));
      sum += m_tr(&P) / 3.0;
      count++;
    }
  }
  out[0] = creal(sum) / (double)count;
  out[1] = cimag(sum) / (double)count;
}
