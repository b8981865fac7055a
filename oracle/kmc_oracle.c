/*
 * kmc_oracle.c -- plain FP64 CPU oracle of the kinetic Monte-Carlo hysteresis
 * method of Tan, Carrey & Respaud (arXiv:1407.2737, Sec. II).
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library. It shares nothing with the
 * CUDA library. It follows the paper's steps i)-viii) in the paper's order:
 *
 *   i)    the moment of every NP is known from the previous step;
 *   ii)   total field = applied field + dipolar field of all others (Eq. 1);
 *   iii)  working plane through the easy axis and the total field; the
 *         previous moment is projected onto it and renormalised;
 *   iv)   200-point scan of dE/dtheta (derivative of Eq. 2), each sign change
 *         refined by Newton's method: minima theta1, theta2 and the lower
 *         maximum theta3 with energies E1, E2, E3;
 *   v)    the moment falls into the minimum whose basin holds it;
 *   vi)   switching rates (Eqs. 3-4) and jump probability over t_step (Eq. 5);
 *   vii)  a uniform draw decides the jump; T = 0 skips vi) and vii);
 *   viii) next step.
 *
 * Readings where the paper is silent or garbled (each is listed with its
 * reason in the design notes of the repository):
 *   - Eq. 1 sums over j != i (the printed index "i != j" is a typo);
 *     the prefactor mu0 M_S V / 4 pi takes the source's own volume V_j.
 *   - Grid nodes sit at theta_j = 2 pi (j + 1/2) / 200 so that theta = 0,
 *     pi/2, pi are never nodes; a sign change between consecutive nodes
 *     (cyclically) brackets one extremum.
 *   - With two minima, the lower of the two maxima is the barrier top for both
 *     directions (Eqs. 3-4); with one minimum no jump is possible.
 *   - Eq. 5 is written for a start in well 2; by symmetry the jump probability
 *     out of well a is nu_a / (nu_1 + nu_2) (1 - exp(-(nu_1 + nu_2) t_step)).
 *   - Step vii: the moment jumps iff u < P.
 *   - Applied field mu0 H_ext,k = mu0 H_max cos(2 pi k / S), constant over
 *     step k; every period starts at +H_max (Sec. III.1).
 *   - Initial moments lie along +/- easy axis with m_z >= 0.
 *   - Loop area of one NP: mu0 M_S V sum_k H_ext,k (m_z,k+1 - m_z,k) over the
 *     recorded periods (parity unpinned at the level of one NP; the
 *     lysosome total is the hysteresis area of Sec. III.2.a).
 */
#include "kmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559
#define PI 3.14159265358979323846264338327950288
#define ORACLE_MU0 (4.0e-7 * 3.14159265358979323846264338327950288)
#define ORACLE_KB 1.380649e-23 /* J/K, exact in the 2019 SI */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11). Each round multiplies counter words 0 and 2 by the two Philox
 * multipliers, swaps the halves and mixes in the key; the key is advanced by
 * the two Weyl increments between rounds. */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void kmc_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                              uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

double kmc_oracle_uniform(uint64_t seed, int64_t step, int32_t np, int32_t lys) {
  const uint64_t s = (uint64_t)step;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)np,
                           (uint32_t)lys};
  uint32_t w[4];
  kmc_oracle_philox4x32_10(ctr, key, w);
  const uint64_t bits = ((uint64_t)w[0] << 21) ^ (uint64_t)(w[1] >> 11);
  return (double)bits * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* ------------------------------------------------------------------------ */
/* Sample regeneration between loops (Sec. II.4). Two 53-bit uniforms per
 * Philox call, from words (w0, w1) and (w2, w3) like kmc_oracle_uniform, with
 * counter (loop, 0x80000000 | sub, NP, lys): the set top bit of word 1 keeps
 * these counters apart from the kMC draws (word 1 = high half of a step index,
 * below 2^31). */
static void regen_uniforms(uint64_t seed, uint32_t loop, uint32_t sub, int32_t np,
                           int32_t lys, double u[2]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {loop, 0x80000000u | sub, (uint32_t)np, (uint32_t)lys};
  uint32_t w[4];
  kmc_oracle_philox4x32_10(ctr, key, w);
  u[0] = (double)(((uint64_t)w[0] << 21) ^ (uint64_t)(w[1] >> 11)) * (1.0 / 9007199254740992.0);
  u[1] = (double)(((uint64_t)w[2] << 21) ^ (uint64_t)(w[3] >> 11)) * (1.0 / 9007199254740992.0);
}

/* A direction uniform on the sphere from two uniforms: z uniform on [-1, 1]
 * (Archimedes) and the azimuth uniform on [0, 2 pi). */
static void sphere_point(const double u[2], double out[3]) {
  const double z = 1.0 - 2.0 * u[0];
  const double ph = TWO_PI * u[1];
  const double r2 = 1.0 - z * z;
  const double r = r2 > 0.0 ? sqrt(r2) : 0.0;
  out[0] = r * cos(ph);
  out[1] = r * sin(ph);
  out[2] = z;
}

/* RSA candidate c: direction from sub 3, radius (R - d/2) max(u0, u1, u2)
 * from subs 4 and 5 (the maximum of three uniforms has density 3 x^2, the
 * radial density of a uniform ball). */
void kmc_oracle_rsa_candidate(double radius, double d, uint64_t seed, uint32_t loop, int64_t c,
                              int32_t lys, double out[3]) {
  double u[2], v[2], w[2], e[3];
  regen_uniforms(seed, loop, 3u, (int32_t)(uint32_t)c, lys, u);
  regen_uniforms(seed, loop, 4u, (int32_t)(uint32_t)c, lys, v);
  regen_uniforms(seed, loop, 5u, (int32_t)(uint32_t)c, lys, w);
  sphere_point(u, e);
  double x = v[0] > v[1] ? v[0] : v[1];
  if (w[0] > x) x = w[0];
  const double r = (radius - 0.5 * d) * x;
  for (int q = 0; q < 3; ++q) out[q] = r * e[q];
}

int64_t kmc_oracle_rsa(int32_t n, double radius, double d, uint64_t seed, uint32_t loop,
                       int32_t lys, int64_t max_candidates, double *pos) {
  const double d2 = d * d;
  int32_t kept = 0;
  int64_t c = 0;
  while (kept < n) {
    if (c >= max_candidates) return -1;
    double p[3];
    kmc_oracle_rsa_candidate(radius, d, seed, loop, c, lys, p);
    ++c;
    int ok = 1;
    for (int32_t j = 0; j < kept && ok; ++j) {
      const double dx = p[0] - pos[3 * j], dy = p[1] - pos[3 * j + 1], dz = p[2] - pos[3 * j + 2];
      if ((dx * dx + dy * dy) + dz * dz < d2) ok = 0;
    }
    if (ok) {
      for (int q = 0; q < 3; ++q) pos[3 * kept + q] = p[q];
      ++kept;
    }
  }
  return c;
}

void kmc_oracle_regen_axes(int32_t n, uint64_t seed, uint32_t loop, int32_t lys, double *axis) {
  for (int32_t i = 0; i < n; ++i) {
    double u[2];
    regen_uniforms(seed, loop, 0u, i, lys, u);
    sphere_point(u, &axis[3 * i]);
  }
}

void kmc_oracle_regen_positions(int32_t n, const double *nodes, double disorder, uint64_t seed,
                                uint32_t loop, int32_t lys, double *pos) {
  for (int32_t i = 0; i < n; ++i) {
    double u[2], v[2], dir[3];
    regen_uniforms(seed, loop, 1u, i, lys, u);
    regen_uniforms(seed, loop, 2u, i, lys, v);
    sphere_point(u, dir);
    const double rho = disorder * v[0];  /* distance uniform on [0, disorder] */
    for (int q = 0; q < 3; ++q) pos[3 * i + q] = nodes[3 * i + q] + rho * dir[q];
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: mu0 H_dip,i = sum_{j != i} (mu0 M_S V_j / 4 pi)
 *                      [3 (m_j . e_ij) e_ij - m_j] / r_ij^3. */
static void dipolar_on(int32_t i, int32_t n, const double *pos, const double *vol,
                       double Ms, const double *m, double *Bi) {
  double bx = 0.0, by = 0.0, bz = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    if (j == i) continue;
    const double rx = pos[3 * j + 0] - pos[3 * i + 0];
    const double ry = pos[3 * j + 1] - pos[3 * i + 1];
    const double rz = pos[3 * j + 2] - pos[3 * i + 2];
    const double r = sqrt(rx * rx + ry * ry + rz * rz);
    const double ex = rx / r, ey = ry / r, ez = rz / r;
    const double mx = m[3 * j + 0], my = m[3 * j + 1], mz = m[3 * j + 2];
    const double me = mx * ex + my * ey + mz * ez;
    const double pref = ORACLE_MU0 * Ms * vol[j] / (4.0 * 3.14159265358979323846);
    const double r3 = r * r * r;
    bx += pref * (3.0 * me * ex - mx) / r3;
    by += pref * (3.0 * me * ey - my) / r3;
    bz += pref * (3.0 * me * ez - mz) / r3;
  }
  Bi[0] = bx;
  Bi[1] = by;
  Bi[2] = bz;
}

void kmc_oracle_dipolar_field(int32_t n, const double *pos, const double *vol,
                              double Ms, const double *m, double *B) {
  for (int32_t i = 0; i < n; ++i) dipolar_on(i, n, pos, vol, Ms, m, &B[3 * i]);
}

void kmc_oracle_dipolar_field_at(int32_t n, const double *pos, const double *vol,
                                 double Ms, const double *m, int32_t n_t,
                                 const int32_t *idx, double *B) {
  for (int32_t t = 0; t < n_t; ++t) dipolar_on(idx[t], n, pos, vol, Ms, m, &B[3 * t]);
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 and its first two derivatives in theta. */
typedef struct {
  double KV;   /* K_eff V, J        */
  double MVB;  /* M_S V mu0 H, J    */
  double phi;
} sw_energy;

static double sw_E(const sw_energy *s, double th) {
  const double st = sin(th);
  return s->KV * st * st - s->MVB * cos(th - s->phi);
}
static double sw_dE(const sw_energy *s, double th) {
  return s->KV * sin(2.0 * th) + s->MVB * sin(th - s->phi);
}
static double sw_d2E(const sw_energy *s, double th) {
  return 2.0 * s->KV * cos(2.0 * th) + s->MVB * cos(th - s->phi);
}

/* Newton's method on dE/dtheta inside a bracket [lo, hi] whose ends have
 * derivatives of opposite sign; a step that leaves the bracket is replaced by
 * bisection, and the bracket shrinks around the sign change every iteration. */
static double refine_extremum(const sw_energy *s, double lo, double hi, double dlo) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double d = sw_dE(s, x);
    if (d == 0.0) return x;
    if ((d < 0.0) == (dlo < 0.0)) {
      lo = x;
      dlo = d;
    } else {
      hi = x;
    }
    const double d2 = sw_d2E(s, x);
    double xn = (d2 != 0.0) ? x - d / d2 : 0.5 * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) < 1e-14 || hi - lo < 1e-14) return xn;
    x = xn;
  }
  return x;
}

int32_t kmc_oracle_extrema(double Keff, double Ms, double V, double B, double phi,
                           double *theta, double *E, int32_t *is_min) {
  sw_energy s;
  s.KV = Keff * V;
  s.MVB = Ms * V * B;
  s.phi = phi;
  double grid[KMC_ORACLE_GRID], d[KMC_ORACLE_GRID];
  for (int j = 0; j < KMC_ORACLE_GRID; ++j) {
    grid[j] = TWO_PI * ((double)j + 0.5) / (double)KMC_ORACLE_GRID;
    d[j] = sw_dE(&s, grid[j]);
  }
  int32_t count = 0;
  for (int j = 0; j < KMC_ORACLE_GRID; ++j) {
    const int jn = (j + 1) % KMC_ORACLE_GRID;
    const double a = grid[j];
    const double b = (jn == 0) ? grid[0] + TWO_PI : grid[jn];
    const int neg_a = d[j] < 0.0, neg_b = d[jn] < 0.0;
    if (neg_a == neg_b) continue;
    if (count == 4) return -1;
    double th = refine_extremum(&s, a, b, d[j]);
    if (th >= TWO_PI) th -= TWO_PI;
    theta[count] = th;
    E[count] = sw_E(&s, th);
    is_min[count] = neg_a && !neg_b; /* dE/dtheta rises through zero */
    ++count;
  }
  return count;
}

/* ------------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* 1 if x lies on the arc that runs counter-clockwise from just after `from`
 * up to and including `to`. */
static int on_arc(double x, double from, double to) {
  double dx = fmod(x - from, TWO_PI);
  if (dx < 0.0) dx += TWO_PI;
  double dt = fmod(to - from, TWO_PI);
  if (dt < 0.0) dt += TWO_PI;
  return dx > 0.0 && dx <= dt;
}

int32_t kmc_oracle_np_update(const double axis[3], const double m_old[3],
                             const double Btot[3], double Keff, double Ms, double V,
                             double T, double tau0, double t_step, double u,
                             kmc_oracle_np_result *res) {
  memset(res, 0, sizeof(*res));
  res->u = u;
  /* iii) working plane spanned by the easy axis a and the total field. */
  const double *a = axis;
  double ep[3];
  double phi = 0.0;
  int degenerate = 0;
  const double Bmag = sqrt(dot3(Btot, Btot));
  if (Bmag > 0.0) {
    const double bh[3] = {Btot[0] / Bmag, Btot[1] / Bmag, Btot[2] / Bmag};
    double cphi = dot3(a, bh);
    const double perp[3] = {bh[0] - cphi * a[0], bh[1] - cphi * a[1],
                            bh[2] - cphi * a[2]};
    const double sp = sqrt(dot3(perp, perp));
    if (sp >= 1e-12) {
      ep[0] = perp[0] / sp;
      ep[1] = perp[1] / sp;
      ep[2] = perp[2] / sp;
      phi = atan2(sp, cphi);
    } else {
      degenerate = 1;
      phi = (cphi >= 0.0) ? 0.0 : 3.14159265358979323846;
    }
  } else {
    degenerate = 1;
  }
  if (degenerate) {
    const double ma = dot3(m_old, a);
    double perp[3] = {m_old[0] - ma * a[0], m_old[1] - ma * a[1], m_old[2] - ma * a[2]};
    double sp = sqrt(dot3(perp, perp));
    if (sp < 1e-12) {
      /* a x x-hat, or a x y-hat when a is close to x-hat */
      if (fabs(a[0]) > 0.9) {
        perp[0] = -a[2];
        perp[1] = 0.0;
        perp[2] = a[0];
      } else {
        perp[0] = 0.0;
        perp[1] = a[2];
        perp[2] = -a[1];
      }
      sp = sqrt(dot3(perp, perp));
    }
    ep[0] = perp[0] / sp;
    ep[1] = perp[1] / sp;
    ep[2] = perp[2] / sp;
  }
  res->degenerate = degenerate;
  /* projection of the previous moment onto the plane, as an angle from a */
  double th0 = atan2(dot3(m_old, ep), dot3(m_old, a));
  if (th0 < 0.0) th0 += TWO_PI;

  /* iv) extrema of Eq. 2 */
  double th[4], E[4];
  int32_t ismin[4];
  const int32_t cnt = kmc_oracle_extrema(Keff, Ms, V, Bmag, phi, th, E, ismin);
  if (cnt < 0) return -1;
  int32_t nmin = 0, nmax = 0, imin[2] = {0, 0}, imax[2] = {0, 0};
  for (int32_t q = 0; q < cnt; ++q) {
    if (ismin[q]) {
      if (nmin == 2) return -1;
      imin[nmin++] = q;
    } else {
      if (nmax == 2) return -1;
      imax[nmax++] = q;
    }
  }
  res->n_min = nmin;
  double th_new = th0;
  if (nmin == 1) {
    th_new = th[imin[0]];
  } else if (nmin == 2) {
    /* v) the basin of a minimum is the arc between the two maxima holding it */
    const double M1 = th[imax[0]], M2 = th[imax[1]];
    const int arc0 = on_arc(th0, M1, M2);
    const int arcA = on_arc(th[imin[0]], M1, M2);
    const int wa = (arc0 == arcA) ? imin[0] : imin[1]; /* current well */
    const int wb = (wa == imin[0]) ? imin[1] : imin[0];
    const double E3 = (E[imax[0]] < E[imax[1]]) ? E[imax[0]] : E[imax[1]];
    res->dE[0] = E3 - E[wa];
    res->dE[1] = E3 - E[wb];
    th_new = th[wa];
    if (T > 0.0) {
      /* vi) Eqs. 3-5 */
      const double nu0 = 1.0 / tau0;
      const double kT = ORACLE_KB * T;
      const double nua = nu0 * exp(-res->dE[0] / kT);
      const double nub = nu0 * exp(-res->dE[1] / kT);
      const double sum = nua + nub;
      res->P = (sum > 0.0) ? (nua / sum) * (-expm1(-sum * t_step)) : 0.0;
      /* vii) */
      res->near = fabs(u - res->P) < 1e-9;
      if (u < res->P) {
        res->flipped = 1;
        th_new = th[wb];
      }
    }
  }
  const double c = cos(th_new), sn = sin(th_new);
  for (int q = 0; q < 3; ++q) res->m_new[q] = c * a[q] + sn * ep[q];
  return 0;
}

/* ------------------------------------------------------------------------ */
int32_t kmc_oracle_step(const kmc_oracle_lysosome *lys, int32_t lys_index,
                        const double *m_in, double mu0Hext, double t_step,
                        uint64_t seed, int64_t step, double *m_out, double *B_dip,
                        double *dE, double *P, double *u, int32_t *flags) {
  const int32_t n = lys->n;
  double *B = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  if (!B) return -2;
  kmc_oracle_dipolar_field(n, lys->pos, lys->vol, lys->Ms, m_in, B);
  int32_t rc = 0;
  for (int32_t i = 0; i < n; ++i) {
    const double Bt[3] = {B[3 * i + 0], B[3 * i + 1], B[3 * i + 2] + mu0Hext};
    const double ui = kmc_oracle_uniform(seed, step, i, lys_index);
    kmc_oracle_np_result r;
    if (kmc_oracle_np_update(&lys->axis[3 * i], &m_in[3 * i], Bt, lys->Keff, lys->Ms,
                             lys->vol[i], lys->T, lys->tau0, t_step, ui, &r) != 0)
      rc = -1;
    if (m_out) memcpy(&m_out[3 * i], r.m_new, sizeof(r.m_new));
    if (B_dip) memcpy(&B_dip[3 * i], &B[3 * i], 3 * sizeof(double));
    if (dE) {
      dE[2 * i + 0] = r.dE[0];
      dE[2 * i + 1] = r.dE[1];
    }
    if (P) P[i] = r.P;
    if (u) u[i] = ui;
    if (flags)
      flags[i] = r.n_min | (r.flipped << 2) | (r.near << 3) | (r.degenerate << 4);
  }
  free(B);
  return rc;
}

int32_t kmc_oracle_run(const kmc_oracle_lysosome *lys, int32_t lys_index, double *m,
                       double mu0Hmax, double f, int32_t S, int32_t periods,
                       int32_t discard, uint64_t seed, int64_t step0, int32_t nthreads,
                       double *E_diss, double *dHdip, double *loop_H, double *loop_M,
                       int64_t *counters) {
  const int32_t n = lys->n;
  if (n < 0 || S <= 0 || periods < 0 || discard < 0 || f <= 0.0) return -3;
  const double t_step = 1.0 / (f * (double)S);
  double *B = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double *mn = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int32_t *fl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!B || !mn || !fl) {
    free(B);
    free(mn);
    free(fl);
    return -2;
  }
  double vsum = 0.0;
  for (int32_t i = 0; i < n; ++i) vsum += lys->vol[i];
  if (E_diss)
    for (int32_t i = 0; i < n; ++i) E_diss[i] = 0.0;
  if (dHdip)
    for (int32_t i = 0; i < n; ++i) dHdip[i] = 0.0;
  /* Eq. 6 compares the dipolar field at the two extremes of the applied
   * field: +mu0Hmax at step 0 of a period and -mu0Hmax at step S/2 (for odd
   * S the first of the two most negative steps, (S-1)/2). */
  const int32_t k_minus = S / 2;
  int32_t n_rec_periods = 0;
  int64_t cnt[4] = {0, 0, 0, 0};
  int32_t rc = 0;
  int64_t rec = 0;
  if (nthreads < 1) nthreads = 1;
  (void)nthreads;
  for (int32_t p = 0; p < periods; ++p) {
    for (int32_t k = 0; k < S; ++k) {
      const int64_t step = step0 + (int64_t)p * S + k;
      const double H = mu0Hmax * cos(TWO_PI * (double)k / (double)S);
      const int record = p >= discard;
      /* ii) dipolar field from the moments at the start of the step */
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
      for (int32_t i = 0; i < n; ++i)
        dipolar_on(i, n, lys->pos, lys->vol, lys->Ms, m, &B[3 * i]);
      /* Eq. 6: z component (the applied field's direction) of the dipolar
       * field acting during the steps at +mu0Hmax and -mu0Hmax */
      if (record && dHdip) {
        if (k == 0)
          for (int32_t i = 0; i < n; ++i) dHdip[i] += B[3 * i + 2];
        if (k == k_minus)
          for (int32_t i = 0; i < n; ++i) dHdip[i] -= B[3 * i + 2];
      }
      /* iii)-vii) for every NP; all NPs see the start-of-step field */
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
      for (int32_t i = 0; i < n; ++i) {
        const double Bt[3] = {B[3 * i + 0], B[3 * i + 1], B[3 * i + 2] + H};
        const double ui = kmc_oracle_uniform(seed, step, i, lys_index);
        kmc_oracle_np_result r;
        int bad = kmc_oracle_np_update(&lys->axis[3 * i], &m[3 * i], Bt, lys->Keff,
                                       lys->Ms, lys->vol[i], lys->T, lys->tau0,
                                       t_step, ui, &r) != 0;
        memcpy(&mn[3 * i], r.m_new, sizeof(r.m_new));
        fl[i] = r.flipped | (r.near << 1) | ((r.n_min == 1) << 2) |
                (r.degenerate << 3) | (bad << 4);
        if (record && E_diss)
          E_diss[i] += lys->Ms * lys->vol[i] * H * (r.m_new[2] - m[3 * i + 2]);
      }
      double msum = 0.0;
      for (int32_t i = 0; i < n; ++i) {
        cnt[0] += fl[i] & 1;
        cnt[1] += (fl[i] >> 1) & 1;
        cnt[2] += (fl[i] >> 2) & 1;
        cnt[3] += (fl[i] >> 3) & 1;
        if ((fl[i] >> 4) & 1) rc = -1;
        m[3 * i + 0] = mn[3 * i + 0];
        m[3 * i + 1] = mn[3 * i + 1];
        m[3 * i + 2] = mn[3 * i + 2];
        msum += lys->vol[i] * m[3 * i + 2];
      }
      if (record) {
        if (loop_H) loop_H[rec] = H;
        if (loop_M) loop_M[rec] = (vsum > 0.0) ? msum / vsum : 0.0;
        ++rec;
      }
    }
    if (p >= discard) ++n_rec_periods;
  }
  /* Eq. 6 averaged over the recorded periods */
  if (dHdip && n_rec_periods > 0)
    for (int32_t i = 0; i < n; ++i) dHdip[i] /= (double)n_rec_periods;
  if (counters) memcpy(counters, cnt, sizeof(cnt));
  free(B);
  free(mn);
  free(fl);
  return rc;
}

double kmc_oracle_area(int32_t n, const double *vol, const double *E_diss,
                       int32_t n_periods) {
  double e = 0.0, v = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    e += E_diss[i];
    v += vol[i];
  }
  if (v <= 0.0 || n_periods <= 0) return 0.0;
  return e / ((double)n_periods * v);
}

double kmc_oracle_sar(double area, double f, double rho) { return area * f / rho; }

/* ------------------------------------------------------------------------ */
/* Eq. 8 (Sec. III.5): local volume concentration around NP i from the
 * distance r_N to its N-th nearest neighbour, phi_N = 3 N V / (4 pi r_N^3),
 * V taken as the volume of NP i. Every distance is listed and sorted. */
static int cmp_double(const void *a, const void *b) {
  const double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* phi_N of NP i; d2 is scratch for n - 1 values */
static double phi_of(int32_t i, int32_t n, const double *pos, const double *vol, int32_t N,
                     double *d2) {
  int32_t q = 0;
  for (int32_t j = 0; j < n; ++j) {
    if (j == i) continue;
    const double dx = pos[3 * j + 0] - pos[3 * i + 0];
    const double dy = pos[3 * j + 1] - pos[3 * i + 1];
    const double dz = pos[3 * j + 2] - pos[3 * i + 2];
    d2[q++] = (dx * dx + dy * dy) + dz * dz;
  }
  qsort(d2, (size_t)(n - 1), sizeof(double), cmp_double);
  const double rN = sqrt(d2[N - 1]);
  return (3.0 * (double)N * vol[i]) / (4.0 * PI * (rN * rN * rN));
}

int32_t kmc_oracle_local_concentration(int32_t n, const double *pos, const double *vol,
                                       int32_t N, double *phi) {
  if (n < 2 || N < 1 || N > n - 1) return -3;
  double *d2 = (double *)malloc(sizeof(double) * (size_t)(n - 1));
  if (!d2) return -2;
  for (int32_t i = 0; i < n; ++i) phi[i] = phi_of(i, n, pos, vol, N, d2);
  free(d2);
  return 0;
}

int32_t kmc_oracle_local_concentration_at(int32_t n, const double *pos, const double *vol,
                                          int32_t N, int32_t n_t, const int32_t *idx,
                                          double *phi) {
  if (n < 2 || N < 1 || N > n - 1 || n_t < 0) return -3;
  for (int32_t t = 0; t < n_t; ++t)
    if (idx[t] < 0 || idx[t] >= n) return -3;
  double *d2 = (double *)malloc(sizeof(double) * (size_t)(n - 1));
  if (!d2) return -2;
  for (int32_t t = 0; t < n_t; ++t) phi[t] = phi_of(idx[t], n, pos, vol, N, d2);
  free(d2);
  return 0;
}

/* Radial profile (Sec. III.4, Fig. 8): NP i lies in shell
 * s = floor(n_shells |r_i - c| / R), the last shell also taking |r_i - c| >= R.
 * R <= 0 selects the radius of the smallest sphere about c that holds every
 * NP whole, max_i (|r_i - c| + (3 V_i / 4 pi)^(1/3)). For each shell: count[s]
 * NPs and, for each of the n_val per-NP columns of val ([n][n_val]), the
 * volume-weighted mean sum V_i val_i / sum V_i in mean[s][n_val] (0 for an
 * empty shell). Returns the radius used, or a negative value on bad input. */
double kmc_oracle_shell_profile(int32_t n, const double *pos, const double *vol,
                                const double center[3], double R, int32_t n_shells,
                                int32_t n_val, const double *val, double *count,
                                double *mean) {
  if (n < 0 || n_shells < 1 || n_val < 0) return -1.0;
  double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *vs = (double *)calloc((size_t)n_shells, sizeof(double));
  if (!r || !vs) {
    free(r);
    free(vs);
    return -2.0;
  }
  double Rmax = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double dx = pos[3 * i + 0] - center[0];
    const double dy = pos[3 * i + 1] - center[1];
    const double dz = pos[3 * i + 2] - center[2];
    r[i] = sqrt((dx * dx + dy * dy) + dz * dz);
    const double a = cbrt(3.0 * vol[i] / (4.0 * PI));
    if (r[i] + a > Rmax) Rmax = r[i] + a;
  }
  if (R <= 0.0) R = Rmax;
  for (int32_t s = 0; s < n_shells; ++s) {
    count[s] = 0.0;
    for (int32_t q = 0; q < n_val; ++q) mean[s * n_val + q] = 0.0;
  }
  for (int32_t i = 0; i < n; ++i) {
    int32_t s = n_shells - 1;
    if (R > 0.0) {
      const double x = floor((double)n_shells * r[i] / R);
      if (x < (double)(n_shells - 1)) s = (int32_t)x;
    }
    count[s] += 1.0;
    vs[s] += vol[i];
    for (int32_t q = 0; q < n_val; ++q) mean[s * n_val + q] += vol[i] * val[i * n_val + q];
  }
  for (int32_t s = 0; s < n_shells; ++s)
    if (vs[s] > 0.0)
      for (int32_t q = 0; q < n_val; ++q) mean[s * n_val + q] /= vs[s];
  free(r);
  free(vs);
  return R;
}

/* ------------------------------------------------------------------------ */
/* Ref. [8] mode (Sec. II.3): probabilities instead of samples. The applied
 * field stays along z, so each NP keeps one working plane spanned by its axis
 * a and e_perp = normalise(z - (z.a) a); the signed field enters Eq. 2 through
 * the angle phi_z of z (or phi_z + pi when the field is negative). */
int32_t kmc_oracle_mean_run(int32_t n, const double *axis, const double *vol,
                            double Ms, double Keff, double T, double tau0,
                            double mu0Hmax, double f, int32_t S, int32_t periods,
                            int32_t discard, double *loop_M) {
  if (n < 0 || S <= 0 || f <= 0.0) return -3;
  const double t_step = 1.0 / (f * (double)S);
  double *thw = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  double *pw = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  int32_t *nw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  double *ep = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double *phz = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!thw || !pw || !nw || !ep || !phz) {
    free(thw);
    free(pw);
    free(nw);
    free(ep);
    free(phz);
    return -2;
  }
  double vsum = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double *a = &axis[3 * i];
    double perp[3] = {-a[2] * a[0], -a[2] * a[1], 1.0 - a[2] * a[2]};
    double sp = sqrt(dot3(perp, perp));
    if (sp >= 1e-12) {
      phz[i] = atan2(sp, a[2]);
    } else {
      if (fabs(a[0]) > 0.9) {
        perp[0] = -a[2];
        perp[1] = 0.0;
        perp[2] = a[0];
      } else {
        perp[0] = 0.0;
        perp[1] = a[2];
        perp[2] = -a[1];
      }
      sp = sqrt(dot3(perp, perp));
      phz[i] = (a[2] >= 0.0) ? 0.0 : 3.14159265358979323846;
    }
    for (int q = 0; q < 3; ++q) ep[3 * i + q] = perp[q] / sp;
    nw[i] = 1;
    thw[2 * i] = (a[2] >= 0.0) ? 0.0 : 3.14159265358979323846;
    pw[2 * i] = 1.0;
    vsum += vol[i];
  }
  int64_t rec = 0;
  int32_t rc = 0;
  for (int32_t p = 0; p < periods; ++p) {
    for (int32_t k = 0; k < S; ++k) {
      const double H = mu0Hmax * cos(TWO_PI * (double)k / (double)S);
      double msum = 0.0;
      for (int32_t i = 0; i < n; ++i) {
        double phi = phz[i];
        if (H < 0.0) phi += 3.14159265358979323846;
        double th[4], E[4];
        int32_t ismin[4];
        const int32_t cnt =
            kmc_oracle_extrema(Keff, Ms, vol[i], fabs(H), phi, th, E, ismin);
        if (cnt < 0) {
          rc = -1;
          continue;
        }
        int32_t nmin = 0, nmax = 0, imin[2] = {0, 0}, imax[2] = {0, 0};
        for (int32_t q = 0; q < cnt; ++q) {
          if (ismin[q]) {
            if (nmin < 2) imin[nmin] = q;
            ++nmin;
          } else {
            if (nmax < 2) imax[nmax] = q;
            ++nmax;
          }
        }
        if (nmin > 2 || nmax > 2) {
          rc = -1;
          continue;
        }
        if (nmin == 1) {
          nw[i] = 1;
          thw[2 * i] = th[imin[0]];
          pw[2 * i] = 1.0;
        } else if (nmin == 2) {
          const double M1 = th[imax[0]], M2 = th[imax[1]];
          const int arcA = on_arc(th[imin[0]], M1, M2);
          double pnew[2] = {0.0, 0.0};
          for (int32_t w = 0; w < nw[i]; ++w) {
            const int target = (on_arc(thw[2 * i + w], M1, M2) == arcA) ? 0 : 1;
            pnew[target] += pw[2 * i + w];
          }
          if (T > 0.0) {
            const double E3 = (E[imax[0]] < E[imax[1]]) ? E[imax[0]] : E[imax[1]];
            const double kT = ORACLE_KB * T;
            const double nuA = exp(-(E3 - E[imin[0]]) / kT) / tau0;
            const double nuB = exp(-(E3 - E[imin[1]]) / kT) / tau0;
            const double sum = nuA + nuB;
            if (sum > 0.0) {
              const double decay = exp(-sum * t_step);
              const double pAinf = nuB / sum;
              const double pA = pAinf + (pnew[0] - pAinf) * decay;
              pnew[1] = 1.0 - pA;
              pnew[0] = pA;
            }
          }
          nw[i] = 2;
          thw[2 * i] = th[imin[0]];
          thw[2 * i + 1] = th[imin[1]];
          pw[2 * i] = pnew[0];
          pw[2 * i + 1] = pnew[1];
        }
        double mz = 0.0;
        for (int32_t w = 0; w < nw[i]; ++w)
          mz += pw[2 * i + w] *
                (cos(thw[2 * i + w]) * axis[3 * i + 2] + sin(thw[2 * i + w]) * ep[3 * i + 2]);
        msum += vol[i] * mz;
      }
      if (p >= discard) {
        if (loop_M) loop_M[rec] = (vsum > 0.0) ? msum / vsum : 0.0;
        ++rec;
      }
    }
  }
  free(thw);
  free(pw);
  free(nw);
  free(ep);
  free(phz);
  return rc;
}
