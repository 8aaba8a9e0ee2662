/*
 * vcsgc_oracle.h -- serial FP64 CPU oracle for the parallel VC-SGC Monte Carlo
 * method of Sadigh, Erhart, Stukowski, Caro, Martinez and Zepeda-Ruiz,
 * "A scalable parallel Monte Carlo algorithm for atomistic simulations of
 * precipitation in alloys".
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Every function follows the paper's statement of the method:
 *   - target distribution pi_V (Sec. II C, Eq. pi_vcsgc; Appendix, Eq. vprob)
 *   - serial VC-SGC rule (Sec. II C, Eqs. cbar and trans_vcsgc)
 *   - modified two-factor serial rule (Sec. III B 2, Eq. mod, with the factor
 *     2 that the printed equation drops restored)
 *   - parallel composite move: local stage (Eq. trans_vcsgc_par1) and global
 *     stage (Eq. trans_vcsgc_par2, with the sign of the (c - c0) term taken
 *     from pi_V, i.e. exponent -beta*kappa_p*dn*(dn + 2(n - n0)))
 *   - domain decomposition into non-interacting domains, one colour per step
 *     chosen from a synchronised random stream (Sec. III A, Fig. decompos1)
 *   - hybrid MC/MD (Sec. IV A) with an EAM potential (Daw-Baskes form).
 *
 * Units: Angstrom, eV, K, fs, amu.
 */
#ifndef VCSGC_ORACLE_H
#define VCSGC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* EAM tables on uniform grids.  pair[0..2] = AA, AB, BB pair energy phi(r);
 * dens[0..1] = electron density contribution f_A(r), f_B(r); embed[0..1] =
 * embedding energy F_A(rho), F_B(rho).  r grid: r_j = j*dr, j = 0..nr-1;
 * rho grid: rho_j = j*drho, j = 0..nrho-1.  d* arrays hold the derivative at
 * each knot; NULL means "estimate it by finite differences of the values". */
typedef struct {
  int32_t nr;
  double dr;
  int32_t nrho;
  double drho;
  double rc;
  const double* pair[3];
  const double* dpair[3];
  const double* dens[2];
  const double* ddens[2];
  const double* embed[2];
  const double* dembed[2];
} orc_eam_in;

typedef struct orc_sys orc_sys;

#define ORC_MAX_SHELLS 8
#define ORC_MLP_IN 10
#define ORC_MLP_H 64
#define ORC_MLP_NPARAM (ORC_MLP_H * ORC_MLP_IN + ORC_MLP_H + ORC_MLP_H * ORC_MLP_H + ORC_MLP_H + ORC_MLP_H + 1)

/* Observables of Sec. II C: B count n, energy, acceptance counters and
 * running moments of the concentration (sampled once per composite step). */
typedef struct {
  int64_t n_sites;
  int64_t n_b;
  double energy;         /* incrementally tracked total energy (eV) */
  int64_t steps;         /* composite (colour) steps done */
  int64_t trials;        /* local trial moves proposed */
  int64_t local_accepts; /* trials accepted by the local stage */
  int64_t global_trials; /* composite steps with at least one local accept */
  int64_t global_accepts;/* of those, steps accepted by the global stage */
  int64_t flips;         /* site flips committed */
  int64_t near_ties;     /* decisions with |u - p| <= 1e-9 p */
  double sum_c;          /* sum over steps of c after the step */
  double sum_c2;
  int64_t stage1_accepts;/* delayed acceptance: trials that passed stage 1 */
} orc_obs;

/* Build a system from explicit positions (SoA) in an orthorhombic periodic
 * box.  The full neighbour list (every periodic image within rc) is built by
 * brute force when brute != 0, else by binning into cells of side >= rc. */
orc_sys* orc_create(int64_t n, const double* x, const double* y, const double* z,
                    const double box[3], const uint8_t* types, const orc_eam_in* eam,
                    int brute);
void orc_free(orc_sys* s);

/* Ensemble parameters (Eq. pi_vcsgc).  kappa_units = 0: kappa is
 * dimensionless and kappa_p = kappa*kB*T/N (eV); kappa_units = 1: kappa_p =
 * kappa in eV.  c0 < 0 selects the current concentration. */
int orc_set_params(orc_sys* s, double phi, double kappa, double T, int kappa_units,
                   double c0, uint64_t seed);

/* Colour schedules (Sec. III A).  Lattice schedules use the rigid BCC cell
 * indices: site i = ((cz*ny + cy)*nx + cx)*2 + b.
 *  blocks:     domains are bx*by*bz-cell blocks; colour = (block index mod p)
 *              per axis; one random site per domain per step.
 *  sublattice: colour = (cx mod qx, cy mod qy, cz mod qz, b); every site of
 *              the colour is trialled each step.
 *  spatial:    domains are nbx*nby*nbz boxes of the periodic cell (explicit
 *              positions); colour = (block index mod p) per axis.
 * Each returns 0, or -1 if the sizes do not divide. */
int orc_schedule_blocks(orc_sys* s, int nx, int ny, int nz, int bx, int by, int bz,
                        int px, int py, int pz);
int orc_schedule_sublattice(orc_sys* s, int nx, int ny, int nz, int qx, int qy, int qz);
int orc_schedule_spatial(orc_sys* s, int nbx, int nby, int nbz, int px, int py, int pz);
/* Overlapping, position-weighted domains (Sec. III A): cells of lx*ly*lz
 * lattice cells, eight colours (one bit per axis); along each axis the
 * domain of bit b covers lattice cells [b g, b g + l - g) of its cell, so
 * same-colour domains of neighbouring cells are g lattice cells apart and
 * the eight domains of a cell overlap where 2 g < l.  Each listed site has
 * the pick weight 8 / (number of the cell's domains that contain it); a
 * domain lists its sites by decreasing weight, ascending index within one
 * weight.  Needs l | n and 0 <= 2 g <= l per axis; returns 0 or -1. */
int orc_schedule_overlap(orc_sys* s, int nx, int ny, int nz, int lx, int ly, int lz,
                         int gx, int gy, int gz);
/* Pick weights of the dom_sites entries (dom_start[n_domains] values) when
 * the schedule is weighted: returns 1 and fills wt (may be NULL), else 0. */
int orc_schedule_weights(const orc_sys* s, int64_t* wt);
/* Count the trials of each site in parallel steps (on != 0), or stop. */
int orc_track_trials(orc_sys* s, int on);
void orc_trial_counts(const orc_sys* s, int64_t* out);
/* Smallest distance between two sites of distinct domains of one colour. */
double orc_schedule_min_separation(const orc_sys* s);
int64_t orc_schedule_info(const orc_sys* s, int64_t* n_colours, int64_t* domains_per_colour);
/* Export domain tables: col_start[n_colours+1], dom_start[n_domains+1],
 * dom_sites[dom_start[n_domains]] (N, or more for overlapping domains; each
 * may be NULL). */
void orc_schedule_export(const orc_sys* s, int64_t* col_start, int64_t* dom_start,
                         int64_t* dom_sites);

/* Parallel composite steps (Sec. III B 2).  Returns 0. */
int orc_parallel_steps(orc_sys* s, int64_t n_steps);
/* Serial single-site steps: mode 0 = Eq. trans_vcsgc, mode 1 = Eq. mod,
 * mode 2 = Eq. mod with a delayed-acceptance local factor (needs a
 * surrogate; returns -1 otherwise). */
int orc_serial_steps(orc_sys* s, int64_t n_steps, int mode);

/* Run n_steps steps (mode -1: parallel composite; 0, 1: serial as above)
 * and add one count per step to hist[n_B] (hist has N+1 entries) and the
 * energy after each step to *sum_e.  Used for distribution tests. */
int orc_run_histogram(orc_sys* s, int64_t n_steps, int mode, int64_t* hist, double* sum_e);

/* Delayed acceptance (Christen and Fox 2005) of the local stage.  Stage 1
 * accepts the move of site i (sign s = +1 for A->B, -1 for B->A) with
 * min{1, exp[-beta (s g_i + s dmu0)]}, stage 2 with min{1, exp[-beta (dE_i -
 * s g_i)]}; g_i predicts E(i = B) - E(i = A) from the environment of i only,
 * so the two stages together keep the ratio of the plain local rule and the
 * sampled distribution is unchanged.  Stage 2 draws its uniform from tag 5
 * (parallel steps, counter (step, trial, 5)) or counter (step, 2, 2) (serial
 * mode 2).
 *
 * Shells: n_shells radii (Angstrom); a neighbour at distance r is in shell q
 * when |r - radii[q]| <= tol.
 * Descriptor of site i (needs 5 shells): out[q] = B sites j != i in shell q
 * of i; out[5 + q] = sum over the first-shell neighbours k of i of the B
 * sites j != i in shell q of k (raw counts).
 * MLP parameters (ORC_MLP_NPARAM doubles): W1[64][10], b1[64], W2[64][64],
 * b2[64], w3[64], b3; inputs are count_c / max_c with max = (8, 6, 12, 24,
 * 8, 56, 48, 96, 192, 64); SiLU activations; output g in eV.
 * Surrogate kind: 0 off, 1 the MLP, 2 the exact energy change (a perfect
 * surrogate, for tests). */
int orc_set_shells(orc_sys* s, int n_shells, const double* radii, double tol);
int orc_descriptor(const orc_sys* s, int64_t i, double out[ORC_MLP_IN]);
double orc_mlp_eval(const double* params, const double x[ORC_MLP_IN]);
int orc_set_surrogate(orc_sys* s, int kind, const double* params);
double orc_surrogate(const orc_sys* s, int64_t i);

/* Energy change for flipping site i (Sec. III A; EAM energy difference with
 * pair, own-embedding and neighbour re-embedding terms). */
double orc_delta_e(const orc_sys* s, int64_t i);
/* Same, by recomputing the full energy before and after the flip. */
double orc_delta_e_full(orc_sys* s, int64_t i);
double orc_energy_full(const orc_sys* s);
void orc_flip(orc_sys* s, int64_t i);

void orc_get_types(const orc_sys* s, uint8_t* out);
void orc_set_types(orc_sys* s, const uint8_t* in);
void orc_get_rho(const orc_sys* s, double* out);
void orc_get_obs(const orc_sys* s, orc_obs* out);
void orc_reset_counters(orc_sys* s);
int64_t orc_neighbour_count(const orc_sys* s, int64_t i);
/* Neighbour j, distance and separation vector (x_j - x_i) of slot k of site i,
 * slots ordered by (distance, j, image). */
void orc_neighbour(const orc_sys* s, int64_t i, int64_t k, int64_t* j, double* r, double d[3]);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the derived draws. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t lo, uint32_t hi);
uint64_t orc_below(uint32_t lo, uint32_t hi, uint64_t m);

/* Cubic Hermite spline of a table: value and derivative at x.  which: 0..2
 * pair, 3..4 density, 5..6 embedding.  Returns 0, or -1 out of range. */
int orc_spline(const orc_sys* s, int which, double x, double* v, double* dv);

/* Molecular dynamics (Sec. IV A): forces -dU/dx and BAOAB Langevin
 * velocity Verlet.  Velocities in Angstrom/fs, masses in amu. */
void orc_forces(orc_sys* s, double* fx, double* fy, double* fz);
void orc_set_md(orc_sys* s, const double* vx, const double* vy, const double* vz,
                double mass_a, double mass_b, double dt, double gamma, double T_md,
                uint64_t seed);
int orc_md_steps(orc_sys* s, int64_t n_steps);
void orc_get_md(const orc_sys* s, double* x, double* y, double* z, double* vx, double* vy,
                double* vz);
double orc_kinetic_energy(const orc_sys* s);
/* Hybrid cycle: n_md MD steps then a MC phase of n_mc composite steps on the
 * current positions; when a site flips its velocity is scaled by
 * sqrt(m_old/m_new). */
int orc_hybrid_cycles(orc_sys* s, int64_t n_cycles, int64_t n_md, int64_t n_mc);

/* The paper's MD ensemble (Sec. IV B: Nose-Hoover thermostat and barostat)
 * in the isotropic form of Martyna, Tobias, Klein (J. Chem. Phys. 101, 4177
 * (1994)) with Nose-Hoover chains (Martyna, Klein, Tuckerman, J. Chem.
 * Phys. 97, 2635 (1992)), integrated by a Trotter splitting (Martyna,
 * Tuckerman, Tobias, Klein, Mol. Phys. 87, 1117 (1996)).
 *   kind 0: Langevin (orc_set_md's gamma), 1: NVT, 2: NPT.
 *   t_damp, p_damp: relaxation times (fs); p_ext in bar; chain: M <= 4.
 * Masses: Q_1 = N_f kT t_damp^2, Q_k = kT t_damp^2 (k > 1); barostat
 * W = (N_f + 3) kT p_damp^2 and its chain kT p_damp^2; N_f = 3 N.
 * Returns 0 or -1. */
#define ORC_MAX_CHAIN 4
int orc_set_ensemble(orc_sys* s, int kind, double t_damp, double p_damp, double p_ext_bar, int chain);
/* Virial sum over pairs r_ij . F_ij (eV) at the current positions. */
double orc_virial(orc_sys* s);
/* out[0..8]: kinetic energy, potential energy, temperature (K), pressure
 * (bar), volume (A^3), conserved extended energy (eV), box x, y, z. */
void orc_md_state(orc_sys* s, double out[9]);
/* Polak-Ribiere conjugate-gradient minimisation of the potential energy in
 * the positions (box and species fixed) until max |F_i| < ftol (eV/A) or
 * max_iter iterations; the line search finds a zero of the directional
 * derivative by secant steps.  Returns 0 (converged), 1 (max_iter) or -1. */
int orc_minimize(orc_sys* s, double ftol, int64_t max_iter, int64_t* iters, double* fmax);

#ifdef __cplusplus
}
#endif
#endif
