/*
 * kmc_oracle.h -- plain FP64 CPU oracle of the kinetic Monte-Carlo (kMC)
 * hysteresis step of Tan, Carrey & Respaud, "Magnetic hyperthermia properties
 * of nanoparticles inside lysosomes using kinetic Monte-Carlo simulations"
 * (arXiv:1407.2737).
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it. It shares no code, header, table or constant with the CUDA library, and
 * it is slow on purpose: every loop is written the way the paper states the
 * method, with no blocking, fusion or reordering.
 *
 * Units are SI throughout: positions in m, volumes in m^3, M_S in A/m,
 * K_eff in J/m^3, fields as mu0*H in tesla, energies in J, times in s.
 *
 * Parity status of each entry point (what pins it is listed in the tests):
 *   philox / uniform ........ pinned (published known-answer vectors, an
 *                              independent library implementation)
 *   dipolar_field ........... pinned (closed forms, lattice symmetry,
 *                              potential gradient)
 *   extrema ................. pinned (brute-force scan, astroid, h = 0)
 *   np_update, step, run .... pinned (Fig. 1b example, Neel statistics,
 *                              two-state equilibrium, T = 0 Stoner-Wohlfarth
 *                              limits, A/K_eff = 2)
 *   per-NP split of the loop area (E_diss of one NP): pinned for isolated NPs
 *                              (discrete square Stoner-Wohlfarth loops); for
 *                              interacting NPs parity unpinned: only the
 *                              lysosome total is fixed by the paper.
 *   mean_run (Ref. [8] mode) . pinned (two-state Boltzmann equilibrium)
 *   run: dHdip (Eq. 6) ....... pinned (closed forms for a saturated pair,
 *                              re-derivation from a stepped trajectory)
 *   local_concentration ...... pinned (cubic lattices: neighbour shells in
 *                              closed form)
 *   shell_profile ............ pinned (hand-placed NPs with known shells)
 *   regen_axes, regen_positions  pinned (moments of the uniform sphere
 *                              distribution, KS tests of z, azimuth and
 *                              displacement length, no overlap at maximal
 *                              disorder by brute force)
 *   rsa_candidate, rsa ....... pinned (candidates uniform in the ball: KS of
 *                              the radius and the direction; every accept and
 *                              reject re-derived by brute force; the dilute
 *                              limit keeps the first n candidates)
 */
#ifndef KMC_ORACLE_H
#define KMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of grid points of the energy-profile scan (Sec. II.1, step iv). */
#define KMC_ORACLE_GRID 200

/* One lysosome: monodisperse or not, one parameter set (Sec. II.1). */
typedef struct {
  int32_t n;            /* number of nanoparticles                          */
  const double *pos;    /* [n][3] centres, m                                */
  const double *axis;   /* [n][3] unit easy axes                            */
  const double *vol;    /* [n] magnetic volumes, m^3                        */
  double Ms;            /* saturation magnetisation, A/m                    */
  double Keff;          /* uniaxial anisotropy, J/m^3                       */
  double T;             /* temperature, K; 0 skips steps vi-vii             */
  double tau0;          /* 1/nu0 with nu1^0 = nu2^0 = nu0 (Eqs. 3-4), s      */
} kmc_oracle_lysosome;

/* Result of steps iii-vii for one nanoparticle. */
typedef struct {
  double m_new[3];      /* unit moment after the step                        */
  double dE[2];         /* E3 - E_a (current well a), E3 - E_b, J; 0 if one well */
  double P;             /* probability of jumping a -> b during t_step (Eq. 5) */
  double u;             /* the uniform draw used (copied from the input)     */
  int32_t n_min;        /* number of minima found (1 or 2; 0 if none)        */
  int32_t flipped;      /* 1 if the moment jumped to the other well          */
  int32_t near;         /* 1 if |u - P| < 1e-9 (near-threshold draw)         */
  int32_t degenerate;   /* 1 if the working plane needed the fallback        */
} kmc_oracle_np_result;

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11). */
void kmc_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                              uint32_t out[4]);

/* Uniform draw in [0,1) with 53 random bits for (seed, step, NP, lysosome):
 * key = (seed low, seed high), counter = (step low, step high, np, lys),
 * u = ((w0 << 21) ^ (w1 >> 11)) * 2^-53 from output words w0, w1. */
double kmc_oracle_uniform(uint64_t seed, int64_t step, int32_t np, int32_t lys);

/* Sample regeneration between loops (Sec. II.4): between loops the paper
 * draws fresh easy axes and, around fixed mean positions (the nodes of a cubic
 * lattice), fresh positions. Draws: Philox4x32-10, key (seed lo, seed hi),
 * counter (loop, 0x80000000 | sub, NP, lys), two 53-bit uniforms per call as
 * in kmc_oracle_uniform. Axes (sub 0): uniform on the sphere, z = 1 - 2 u0,
 * azimuth 2 pi u1. Positions: node + rho e with e uniform on the sphere from
 * sub 1 and rho = disorder * (first uniform of sub 2), uniform on
 * [0, disorder] as the paper states it. axis, pos are [n][3]. */
void kmc_oracle_regen_axes(int32_t n, uint64_t seed, uint32_t loop, int32_t lys, double *axis);
void kmc_oracle_regen_positions(int32_t n, const double *nodes, double disorder, uint64_t seed,
                                uint32_t loop, int32_t lys, double *pos);

/* Random sequential addition (Sec. II.4 names it as the alternative to the
 * lattice; the configs place lysosomes by it): candidate c is a point uniform
 * in the ball of radius R - d/2 about the origin, with direction from sub 3
 * (as the axes) and radius (R - d/2) * max(u0, u1, u2), whose density grows as
 * r^2, from sub 4 (u0, u1) and sub 5 (u0); NP slot of the counter = c.
 * Candidates are taken in order c = 0, 1, ...; one is kept iff its squared
 * distance to every kept one is at least d^2, until n are kept. Returns the
 * number of candidates used, or -1 if max_candidates ran out first (pos then
 * holds the ones kept so far). pos is [n][3], m, about the lysosome centre. */
void kmc_oracle_rsa_candidate(double radius, double d, uint64_t seed, uint32_t loop, int64_t c,
                              int32_t lys, double out[3]);
int64_t kmc_oracle_rsa(int32_t n, double radius, double d, uint64_t seed, uint32_t loop,
                       int32_t lys, int64_t max_candidates, double *pos);

/* Eq. 1: mu0*H_dip on every NP from the moments of all the others, exact sum
 * over j != i with per-source volume V_j. B is [n][3] in tesla. */
void kmc_oracle_dipolar_field(int32_t n, const double *pos, const double *vol,
                              double Ms, const double *m, double *B);

/* Eq. 1 at n_t listed targets only (idx[t] in [0, n)); B is [n_t][3]. */
void kmc_oracle_dipolar_field_at(int32_t n, const double *pos, const double *vol,
                                 double Ms, const double *m, int32_t n_t,
                                 const int32_t *idx, double *B);

/* Step iv: extrema of Eq. 2 for field magnitude B = mu0*H_tot (T) at angle phi
 * (rad) from the easy axis. Writes up to 4 extrema in scan order: angle in
 * [0, 2 pi), energy (J) and 1 for a minimum / 0 for a maximum. Returns the
 * count. */
int32_t kmc_oracle_extrema(double Keff, double Ms, double V, double B, double phi,
                           double *theta, double *E, int32_t *is_min);

/* Steps iii-vii for one NP with total field Btot (T) and draw u. T = 0 skips
 * vi-vii. Returns 0, or -1 if more than four extrema were found. */
int32_t kmc_oracle_np_update(const double axis[3], const double m_old[3],
                             const double Btot[3], double Keff, double Ms, double V,
                             double T, double tau0, double t_step, double u,
                             kmc_oracle_np_result *res);

/* One synchronous step of one lysosome (steps i-vii for every NP, Sec. II.2):
 * applied field mu0Hext along z (T). Any of the outputs may be NULL.
 * flags[i] = n_min | flipped << 2 | near << 3 | degenerate << 4. */
int32_t kmc_oracle_step(const kmc_oracle_lysosome *lys, int32_t lys_index,
                        const double *m_in, double mu0Hext, double t_step,
                        uint64_t seed, int64_t step, double *m_out, double *B_dip,
                        double *dE, double *P, double *u, int32_t *flags);

/* A whole run of `periods` field periods with S steps each; the first
 * `discard` periods are not recorded (Sec. III.1). m is [n][3], updated in
 * place; step0 is the global index of the first step (Philox counter).
 * Outputs (any may be NULL):
 *   E_diss [n]: sum over recorded steps of mu0 M_S V_i H_ext,k (m_z,new - m_z,old), J
 *   loop_H, loop_M [S*(periods-discard)]: mu0*H_ext,k (T) and the
 *   volume-weighted mean m_z after step k
 *   dHdip [n]: Eq. 6 per NP, mu0 H_dip,z at the step of +mu0Hmax (step 0 of
 *   a period) minus mu0 H_dip,z at the step of -mu0Hmax (step S/2; (S-1)/2
 *   for odd S), both from the moments at the start of the step, averaged
 *   over the recorded periods, T
 *   counters [4]: flips, near-threshold draws, monostable NP-steps,
 *   degenerate working planes.
 * nthreads > 1 runs the per-NP loops with OpenMP, as the paper did. */
int32_t kmc_oracle_run(const kmc_oracle_lysosome *lys, int32_t lys_index, double *m,
                       double mu0Hmax, double f, int32_t S, int32_t periods,
                       int32_t discard, uint64_t seed, int64_t step0, int32_t nthreads,
                       double *E_diss, double *dHdip, double *loop_H, double *loop_M,
                       int64_t *counters);

/* Hysteresis area A (J/m^3 per cycle) from the per-NP recorded energies, and
 * the SAR A*f/rho in W/kg (Sec. III.2.a). */
double kmc_oracle_area(int32_t n, const double *vol, const double *E_diss,
                       int32_t n_periods);
double kmc_oracle_sar(double area, double f, double rho);

/* Eq. 8 (Sec. III.5): phi_N,i = 3 N V_i / (4 pi r_N^3) with r_N the distance
 * from NP i to its N-th nearest neighbour. phi is [n]. Returns 0, or -3
 * unless 1 <= N <= n - 1. */
int32_t kmc_oracle_local_concentration(int32_t n, const double *pos, const double *vol,
                                       int32_t N, double *phi);

/* Eq. 8 at n_t listed NPs only (idx[t] in [0, n)); phi is [n_t]. */
int32_t kmc_oracle_local_concentration_at(int32_t n, const double *pos, const double *vol,
                                          int32_t N, int32_t n_t, const int32_t *idx,
                                          double *phi);

/* Radial profile (Sec. III.4, Fig. 8): n_shells shells of equal thickness
 * R / n_shells about `center`; NP i goes to floor(n_shells |r_i - c| / R),
 * clamped to the last shell. R <= 0 selects max_i (|r_i - c| + radius_i).
 * count [n_shells]; mean [n_shells][n_val] = volume-weighted mean of each
 * column of val [n][n_val] over the shell (0 if empty). Returns R used. */
double kmc_oracle_shell_profile(int32_t n, const double *pos, const double *vol,
                                const double center[3], double R, int32_t n_shells,
                                int32_t n_val, const double *val, double *count,
                                double *mean);

/* The Ref. [8] program's mode used for validation (Sec. II.3): no sampling and
 * no interactions; each NP carries the probability of each well, moved with
 * the wells and relaxed with Eqs. 3-5. Writes the volume-weighted mean m_z
 * after every recorded step into loop_M. */
int32_t kmc_oracle_mean_run(int32_t n, const double *axis, const double *vol,
                            double Ms, double Keff, double T, double tau0,
                            double mu0Hmax, double f, int32_t S, int32_t periods,
                            int32_t discard, double *loop_M);

#ifdef __cplusplus
}
#endif
#endif
