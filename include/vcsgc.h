/*
 * vcsgc.h -- C ABI of the GB300 (sm_103a) implementation of the parallel
 * variance-constrained semi-grandcanonical (VC-SGC) Monte Carlo method of
 * Sadigh, Erhart, Stukowski, Caro, Martinez and Zepeda-Ruiz, "A scalable
 * parallel Monte Carlo algorithm for atomistic simulations of precipitation
 * in alloys", with the EAM molecular-dynamics step of its hybrid MC/MD scheme.
 *
 * Conventions
 *   - Units: Angstrom, eV, K, fs, amu.  Species 0 = A, 1 = B; the
 *     concentration c is the fraction of B sites (Sec. II: n = sum sigma_i).
 *   - Every function returns an int status: VCSGC_OK (0) or a negative
 *     VCSGC_ERR_* code; vcsgc_last_error() gives a text for the last failure.
 *     No function traps, aborts or exits the process.
 *   - Pointer arguments are HOST pointers unless stated otherwise.  Inputs are
 *     copied during the call; the caller keeps ownership of its buffers.
 *   - A context owns all device memory it allocates and releases it in
 *     vcsgc_free().  Work is issued on the stream given in the options (the
 *     legacy default stream when NULL); calls that return host data
 *     synchronise that stream.
 *   - A context may hold R >= 1 independent replicas (chains) of one lattice,
 *     each with its own species array, phi, kappa, T and seed.  Replicas are
 *     advanced together, one composite step each per colour step.
 *   - Multi-GPU: none.  One context drives one GPU; replicas are the only
 *     data-parallel axis.
 */
#ifndef VCSGC_H
#define VCSGC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define VCSGC_OK 0
#define VCSGC_ERR_INVALID_ARG (-1) /* argument out of its documented range  */
#define VCSGC_ERR_CUDA (-2)        /* a CUDA runtime call failed            */
#define VCSGC_ERR_TABLE_RANGE (-3) /* r or rho left an EAM table's grid     */
#define VCSGC_ERR_NONFINITE (-4)   /* NaN or Inf met in an energy or force  */
#define VCSGC_ERR_SCHEDULE (-5)    /* domains of one colour closer than the
                                      independence radius 2 r_c, or sizes
                                      that do not divide                    */
#define VCSGC_ERR_TIMEOUT (-6)     /* a bounded device wait ran out         */
#define VCSGC_ERR_NOMEM (-7)       /* device or host allocation failed      */
#define VCSGC_ERR_STATE (-8)       /* call not valid in the context's state
                                      (e.g. md_steps without velocities)    */
#define VCSGC_ERR_OVERFLOW (-9)    /* neighbour list capacity exceeded      */

/* ------------------------------------------------------------- lattices */
/* The periodic cell the species live on (Sec. II: positions x^{3N}).
 * kind 0: rigid BCC lattice of nx*ny*nz cubic cells of side a; site
 *         i = ((cz*ny + cy)*nx + cx)*2 + b sits at a*(cx+b/2, cy+b/2, cz+b/2);
 *         box = a*(nx, ny, nz); x, y, z, n, box are ignored.
 * kind 1: n explicit positions (host SoA arrays x, y, z, each length n) in
 *         the orthorhombic periodic box box[0..2]; each box length must
 *         exceed 2 (r_c + skin). */
typedef struct {
  int32_t kind;
  int32_t nx, ny, nz;
  double a;
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  double box[3];
} vcsgc_lattice;

/* EAM potential (Daw-Baskes form, the many-body short-range potential the
 * paper's method targets, Sec. I and III A):
 *   U = sum_i [ 1/2 sum_j phi_{t_i t_j}(r_ij) + F_{t_i}(rho_i) ],
 *   rho_i = sum_j f_{t_j}(r_ij).
 * Tables on uniform grids: r_j = j*dr (j < nr, covering [0, rc]) for
 * pair[0..2] = phi_AA, phi_AB, phi_BB and dens[0..1] = f_A, f_B; rho_j =
 * j*drho (j < nrho) for embed[0..1] = F_A, F_B.  d* arrays give the exact
 * derivative at each knot; NULL selects central finite differences of the
 * values (one-sided at the two ends).  Interpolation is cubic Hermite, so
 * energies are C^1 and forces are the exact derivative of the interpolant. */
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
} vcsgc_eam_tables;

/* ------------------------------------------------------------ schedules */
/* Colour schedules: the domain decomposition of Sec. III A.  Each colour
 * step draws one colour from the synchronised random stream; every domain of
 * that colour proposes one flip at once.  Domains of one colour must be more
 * than 2 r_c apart (many-body independence radius), which vcsgc_init checks.
 *   BLOCKS:     (kind 0) domains = blocks of sched[0..2] = bx,by,bz cells,
 *               colour = (block index mod p) per axis with sched[3..5] =
 *               px,py,pz; one uniformly chosen site per domain per step.
 *               The paper's octant scheme is p = (2,2,2).
 *   SUBLATTICE: (kind 0) colour = (cx mod qx, cy mod qy, cz mod qz, basis)
 *               with sched[0..2] = qx,qy,qz; every site of the colour is a
 *               domain of its own, so all of them are trialled at once.
 *   SPATIAL:    (kind 0 or 1) domains = sched[0..2] = nbx,nby,nbz boxes of
 *               the periodic cell, colour as for BLOCKS with sched[3..5].
 *   OVERLAP:    (kind 0) overlapping, position-weighted domains (Sec. III A):
 *               cells of sched[0..2] = lx,ly,lz lattice cells, eight colours
 *               (one bit per axis); along each axis the domain of bit b
 *               covers cell-local lattice cells [b g, b g + l - g), g =
 *               sched[3..5], so same-colour domains are g cells apart and the
 *               eight domains of a cell overlap where 2 g < l.  A site in m of
 *               its cell's domains is picked with weight 8 / m, which makes
 *               every site's pick probability 1 / (2 lx ly lz) per step; a
 *               domain lists its sites by decreasing weight, ascending index
 *               within one weight.  Needs l | n and 2 g <= l per axis. */
#define VCSGC_SCHED_BLOCKS 0
#define VCSGC_SCHED_SUBLATTICE 1
#define VCSGC_SCHED_SPATIAL 2
#define VCSGC_SCHED_OVERLAP 3

#define VCSGC_PREC_FP64 0
#define VCSGC_PREC_MIXED 1

typedef struct {
  uint64_t seed;        /* Philox key of replica 0 (replica r: seed_r[r] or seed + r) */
  double c0;            /* reference concentration of Eq. trans_vcsgc_par1; < 0: initial c */
  int32_t kappa_units;  /* 0: kappa dimensionless, kappa_p = kappa kB T / N (eV)
                           1: kappa_p = kappa in eV, Eq. pi_vcsgc as printed */
  int32_t schedule;     /* VCSGC_SCHED_* */
  int32_t sched[6];
  int32_t precision;    /* VCSGC_PREC_FP64, or VCSGC_PREC_MIXED: pair, density and
                           embedding-table interpolation in FP32 (coefficients
                           rounded to float, FP32 separations from fixed-point
                           copies of the positions, exact minimum image); rho
                           sums, embedding differences, dE and force sums in FP64 */
  int32_t n_replicas;   /* >= 1 */
  const double* phi_r;  /* per-replica phi, kappa, T, seed, c0 (n_replicas each) or NULL */
  const double* kappa_r;
  const double* T_r;
  const uint64_t* seed_r;
  const double* c0_r;
  /* molecular dynamics (hybrid scheme, Sec. IV A); used by md_steps */
  double mass[2];       /* amu; default 55.845, 63.546 */
  double dt;            /* fs; default 2 */
  double gamma;         /* Langevin friction (1/fs); 0 = NVE; default 0.01 */
  double T_md;          /* thermostat temperature (K); default = T */
  double skin;          /* neighbour-list skin (Angstrom); default 0.3 */
  uint64_t md_seed;     /* Philox key of the thermostat noise */
  void* stream;         /* cudaStream_t; NULL: the context creates its own stream */
  int32_t device;       /* CUDA device ordinal; < 0: the calling thread's current device */
} vcsgc_options;

/* Observables (Sec. II C): B count, concentration, energy, acceptance and
 * the chemical-potential estimate dmu = phi + 2 kappa_p N <c> (Eq. gforce). */
typedef struct {
  int64_t n_sites;
  int64_t n_b;
  double c;
  double energy;          /* total energy (eV): tracked step by step, or
                             recomputed by this call (rigid lattice with
                             species-dependent densities) */
  double energy_per_atom;
  int64_t steps;          /* colour (composite) steps */
  int64_t trials;         /* local trial moves */
  int64_t local_accepts;
  int64_t global_trials;  /* steps with >= 1 local accept */
  int64_t global_accepts;
  int64_t flips;
  int64_t near_ties;      /* decisions with |u - p| <= 1e-9 p */
  double acc_local;       /* local_accepts / trials */
  double acc_global;      /* global_accepts / global_trials */
  double mean_c;          /* <c> over steps */
  double var_c;
  double dmu_est;         /* phi + 2 kappa_p N <c> */
  double sweeps;          /* trials / N */
  double kappa_p;         /* eV */
  double dmu0;            /* phi + 2 kappa_p N c0 (eV) */
  int64_t stage1_accepts; /* delayed acceptance: trials that passed stage 1
                             (the exact dE was evaluated for these only) */
} vcsgc_observables;

/* Fill *opt with the defaults: seed 1, c0 = -1, kappa_units 0, SUBLATTICE
 * (4,4,4), FP64, one replica, masses 55.845/63.546 amu, dt 2 fs, gamma
 * 0.01/fs, skin 0.3 A, NULL stream. */
int vcsgc_default_options(vcsgc_options* opt);

/* Create a context: copy the lattice, species (n_replicas * N bytes,
 * replica-major; 0 = A, 1 = B), EAM tables and ensemble parameters to the
 * device, build the neighbour list (A1), rho and U (A2) and the colour
 * schedule (A3).  phi (eV), kappa and T (K) follow Eq. pi_vcsgc:
 * pi_V ~ exp[-beta (U + phi n + kappa_p n^2)].  opt may be NULL.
 * With species-dependent densities on a rigid lattice the local decision is
 * taken on an FP32 dE within a proven error bound (FP64 where the bound
 * cannot decide), so every decision is the FP64 one; the energy is then
 * recomputed when observables or a checkpoint read it.  With the period-q
 * sublattice schedule, the five-shell BCC neighbourhood, FP64 precision and
 * kappa_units 0, such a context advances its replicas through the
 * multicomponent kernels with K = 2 (the same chain step for step, see
 * vcsgc_multi_init) and mirrors their species and counters when read.
 * Errors: INVALID_ARG (bad sizes, N >= 2^30 sites, species other than 0/1,
 * T <= 0), SCHEDULE, TABLE_RANGE, NOMEM, CUDA. */
int vcsgc_init(void** ctx, const vcsgc_lattice* lattice, const uint8_t* types,
               const vcsgc_eam_tables* eam, double phi, double kappa, double T,
               const vcsgc_options* opt);

/* Batch of rigid BCC lattices of different sizes in one context: replica r
 * has cells[3r..3r+2] = (nx, ny, nz) cells of side a, its species at
 * types[sum_{q<r} N_q .. + N_r) (N_r = 2 nx ny nz, concatenated), and its own
 * phi[r], kappa[r], T[r] (n_rep each; opt->seed_r / c0_r per replica as in
 * vcsgc_init).  Every replica must use the SUBLATTICE schedule with the same
 * period (each size divisible by it) and the same a and tables, with one
 * density function.  All replicas advance together: one fused launch per
 * colour step serves the whole batch.  Calls taking a replica index work on
 * batches; md_steps, forces and neighbours do not (VCSGC_ERR_STATE).
 * Errors: INVALID_ARG, SCHEDULE, NOMEM, CUDA. */
int vcsgc_batch_init(void** ctx, int32_t n_rep, const int32_t* cells, double a, const uint8_t* types,
                     const vcsgc_eam_tables* eam, const double* phi, const double* kappa,
                     const double* T, const vcsgc_options* opt);

/* Pick the launch shape of the fused colour step by timing `steps` colour
 * steps with each candidate (these are real steps of the chain): form 0
 * with thread-block size 64, 128 or 256, each with and without loading the
 * trial's neighbour rows ahead of the block barrier (shorter dependent
 * chain, more registers), and form 1 with every cluster size the lattices
 * allow at 256 and 512 threads (see vcsgc_set_launch).  The fastest is kept
 * for later launches (vcsgc_get_launch reports it); *best_block receives its
 * block size.  A context outside the fused form reports its fixed block
 * size. */
int vcsgc_autotune(void* ctx, int64_t steps, int32_t* best_block);

/* Change the colour schedule of a rigid single-lattice context between two
 * colour steps (kind and sched[6] as in vcsgc_options; BLOCKS, SUBLATTICE or
 * OVERLAP).  Each schedule leaves pi_V invariant (Sec. III A-B: the
 * decomposition only chooses which independent trials a composite move
 * holds), so the chain stays exact; the step counter and the random streams
 * continue.  Errors: INVALID_ARG, SCHEDULE (domains closer than 2 r_c, sizes
 * that do not divide; the old schedule is kept), STATE (explicit positions,
 * batches, or a context run through the multicomponent kernels). */
int vcsgc_set_schedule(void* ctx, int32_t kind, const int32_t* sched);

/* Pick a colour schedule by the sampling it delivers: for each of n_cand
 * candidates (kinds[q], scheds[6 q .. 6 q + 5]) the chain, started from its
 * state at the call (species, counters, step counter), runs `sweeps` sweeps
 * under the candidate to settle, then `sweeps` timed sweeps; scores[q]
 * receives the accepted flips per second of all replicas over the timed
 * sweeps (-1 for a schedule the lattices refuse).  These trial runs are
 * discarded: the chain then resumes from its state at the call under the
 * best candidate, as if they had not been run; *best receives its index.
 * Errors: INVALID_ARG, STATE as vcsgc_set_schedule, SCHEDULE (no candidate
 * applies). */
int vcsgc_autotune_schedule(void* ctx, int32_t n_cand, const int32_t* kinds, const int32_t* scheds, int64_t sweeps,
                            double* scores, int32_t* best);

/* Advance every replica by n_steps colour steps (composite moves of
 * Sec. III B 2: site pick, dE gather, local Metropolis test with
 * dmu0 = phi + 2 kappa_p N c0, reduction of dn, global test with exponent
 * -beta kappa_p dn (dn + 2 (n - n0)), commit).  Asynchronous on the stream. */
int vcsgc_steps(void* ctx, int64_t n_steps);

/* n_sweeps sweeps: one sweep = N trial moves = N / (domains per colour)
 * colour steps (the paper's MC cycle of N_at trials, Sec. IV B). */
int vcsgc_sweep(void* ctx, int64_t n_sweeps);

/* Colour steps per sweep for this context's schedule. */
int vcsgc_steps_per_sweep(void* ctx, int64_t* out);

/* n_steps MD steps (EAM forces, BAOAB Langevin velocity Verlet) on replica 0.
 * Needs kind 1 (explicit positions), n_replicas = 1 and velocities set by
 * vcsgc_set_velocities.  The neighbour list is rebuilt when an atom moved
 * more than skin/2 since the last build. */
int md_steps(void* ctx, int64_t n_steps);

/* Hybrid MC/MD (Sec. IV A): n_cycles times (n_md MD steps, then n_mc colour
 * steps on the frozen positions; a flipped atom's velocity is scaled by
 * sqrt(m_old/m_new)).  SPATIAL schedules are rebuilt from the positions at
 * the start of each MC phase. */
int vcsgc_hybrid(void* ctx, int64_t n_cycles, int64_t n_md, int64_t n_mc);

/* Observables of one replica (synchronises the stream). */
int observables(void* ctx, int32_t replica, vcsgc_observables* out);
/* Observables of every replica: out[R] (one synchronisation). */
int vcsgc_observables_all(void* ctx, vcsgc_observables* out);

/* Species of one replica: N bytes to/from host memory.  set_types
 * recomputes rho and the energy and keeps the counters.  Errors:
 * INVALID_ARG when a byte is neither 0 nor 1 (nothing is changed). */
int vcsgc_get_types(void* ctx, int32_t replica, uint8_t* out);
int vcsgc_set_types(void* ctx, int32_t replica, const uint8_t* in);
/* Species of every replica at once: the replicas' arrays back to back
 * (replica 0 first; sum of the replica sizes bytes), one transfer per
 * replica and one synchronisation in all.  Same errors as above. */
int vcsgc_get_types_all(void* ctx, uint8_t* out);
int vcsgc_set_types_all(void* ctx, const uint8_t* in);
/* Electron density rho_i of one replica, N doubles. */
int vcsgc_get_rho(void* ctx, int32_t replica, double* out);
/* Energy change of flipping each of sites[0..n) of one replica on its current
 * state, evaluated by the sweep's own device code (A4); out: n doubles. */
int vcsgc_delta_e(void* ctx, int32_t replica, const int64_t* sites, int64_t n, double* out);
/* Total energy of one replica recomputed from scratch on the device. */
int vcsgc_energy(void* ctx, int32_t replica, double* out);
/* Forces of replica 0 (3 x N doubles, SoA fx, fy, fz). */
int vcsgc_forces(void* ctx, double* fx, double* fy, double* fz);
/* Positions and velocities of replica 0 (each N doubles; any may be NULL). */
int vcsgc_get_md(void* ctx, double* x, double* y, double* z, double* vx, double* vy,
                 double* vz);
int vcsgc_set_velocities(void* ctx, const double* vx, const double* vy, const double* vz);
/* Kinetic energy of replica 0 (eV). */
int vcsgc_kinetic_energy(void* ctx, double* out);

/* Run n colour steps with a CUDA event after each launch on the context's
 * stream and return the summed device time (ms) of the propose kernels and
 * of the commit kernels.  Same work as vcsgc_steps(n); for profiling. */
int vcsgc_profile_steps(void* ctx, int64_t n, double* ms_propose, double* ms_commit);

/* Launch shape of the fused colour step.  Any shape advances the same chain
 * (the random numbers are keyed by step and trial, not by thread).
 *   form 0: one launch per colour step for every replica, `block` threads
 *           per thread block (64, 128 or 256), variant = 1 loads the
 *           trial's neighbour rows ahead of the block barrier, 0 does not.
 *   form 1: cluster-resident: one launch runs many colour steps; each
 *           replica is one thread-block cluster of `variant` CTAs (1, 2, 4,
 *           8 or 16) of `block` threads (256 or 512) that holds the
 *           replica's bit-packed species in shared memory, tiled in (y, z)
 *           with a two-row halo, and separates colour steps by cluster
 *           barriers (the paper's allgather of dc_i, Sec. III B 2, becomes a
 *           reduction in the cluster's distributed shared memory).  Needs
 *           the period-q sublattice schedule, the five-shell BCC table, one
 *           density function and no surrogate; vcsgc_cluster_sizes lists
 *           the sizes these lattices allow.
 * vcsgc_autotune picks a shape by timing; this call sets one explicitly.
 * Errors: INVALID_ARG (unknown form or shape), STATE (not the fused form,
 * or a form-1 size these lattices or this GPU do not allow). */
int vcsgc_set_launch(void* ctx, int32_t form, int32_t block, int32_t variant);
/* The current launch shape (HOST outputs; any may be NULL). */
int vcsgc_get_launch(void* ctx, int32_t* form, int32_t* block, int32_t* variant);
/* Cluster sizes of launch form 1 available for this context: bit q of *mask
 * set for size 2^q (q = 0..4). */
int vcsgc_cluster_sizes(void* ctx, int32_t* mask);

/* Philox4x32-10 words of the device generator every kernel draws from
 * (Salmon, Moraes, Dror and Shaw, SC'11), for checks against the
 * generator's published known-answer values: out[4q..4q+3] = Philox4x32-10
 * of counter ctr[4q..4q+3] under key key[2q..2q+1], q < n.  HOST arrays;
 * one launch on the current device, which the call waits for.
 * Errors: INVALID_ARG (null pointer, n < 1 or n > 2^20), NOMEM, CUDA. */
int vcsgc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n);

/* Neighbour list of replica 0's lattice: capacity K per site and, for site
 * i, the neighbour indices in out[0..count) (count <= K).  For tests. */
int vcsgc_neighbours(void* ctx, int64_t i, int32_t* out, int32_t cap, int32_t* count);

/* Neighbour-list build that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc when they need a list, for example code that runs while another
 * framework's caching allocator holds nearly all device memory, or code with
 * a fixed memory budget.  It builds the same cell-binned full list as a
 * context does for explicit positions.
 *   In:  n positions as DEVICE arrays d_x, d_y, d_z (doubles; a position
 *        outside the periodic box box[0..2], a HOST array, is taken at its
 *        periodic image inside), list radius rl (Angstrom).
 *   Out: DEVICE arrays owned by the caller: d_nbr[n][K] (int32, row i lists
 *        every atom within rl of atom i under the minimum image, and may
 *        also list atoms up to rl + 0.01 A + 1e-6 max(box) away, the margin
 *        of the list's FP32 distance test; cell order, -1 padded) and
 *        d_cnt[n] (row lengths).
 * Work runs on `stream` (NULL: legacy default stream); the call waits for it.
 * Its working space is one static device array of about 6 MB that every
 * GPU loading this library holds until the process exits.  The first call on
 * a device looks up that array's address (make it before any stream
 * capture).  All calls share the array, so calls that overlap on the GPU
 * race.  Limits: n <= 262144; each box length > 2 rl with at least 3 and, in
 * total, at most 65536 binning cells of side >= rl.
 * Errors: INVALID_ARG beyond those limits or for null pointers; OVERFLOW when
 * a row had more than K neighbours (that row is truncated to K); CUDA. */
int vcsgc_neighbour_list_noalloc(int64_t n, const double* d_x, const double* d_y,
                                 const double* d_z, const double box[3], double rl, int32_t K,
                                 int32_t* d_nbr, int32_t* d_cnt, void* stream);

/* ---- Delayed acceptance with a learned surrogate of dE.
 * The local stage of the composite move (Sec. III B 2, Eq.
 * trans_vcsgc_par1) split into two stages (Christen and Fox, J. Comput.
 * Graph. Stat. 14 (2005) 795): a trial of site i (s = +1 for A->B, -1 for
 * B->A) passes stage 1 when u < min{1, exp[-beta (s g_i + s dmu0)]} and is
 * accepted when it also passes stage 2, u2 < min{1, exp[-beta (dE_i - s
 * g_i)]}, where g_i is the surrogate's prediction of E(i = B) - E(i = A) and
 * dE_i the exact energy change, evaluated only after stage 1.  g_i depends
 * on the environment of i only (every site but i), so the product of the two
 * stages has the ratio exp(-X) of the plain rule and the sampled
 * distribution is unchanged, whatever the surrogate's error.  u is the
 * plain rule's uniform; u2 comes from Philox counter (step, trial, 5).
 *
 * Environment descriptor of site i (ten counts): own[s] = B neighbours of i
 * in shell s = 1..5; nb[s] = sum over the 8 first-shell neighbours k of i of
 * the B sites other than i in shell s of k.  Only the rigid BCC lattice with
 * r_c between sqrt(3) a and sqrt(19) a / 2 (five shells: 8, 6, 12, 24, 8
 * sites) has it: in the fused form, and, with species-dependent densities,
 * in a context that runs its steps through the two-species multicomponent
 * kernels (vcsgc_init; the calls go to vcsgc_multi_set_surrogate and
 * vcsgc_multi_features).
 *
 * Surrogate network (VCSGC_MLP_NPARAM FP32 parameters, in this order):
 * W1[64][10], b1[64], W2[64][64], b2[64], w3[64], b3.  x_c = count_c / max_c
 * with max = (8, 6, 12, 24, 8, 56, 48, 96, 192, 64); z1 = W1 x + b1;
 * h1 = SiLU(z1); z2 = W2 h1 + b2; h2 = SiLU(z2); g = w3 . h2 + b3 (eV).
 * On the GPU x, W1, W2 and h1 enter the tensor cores as BF16 with FP32
 * accumulation, and SiLU(z) = z (1 + tanh(z / 2)) / 2 uses the hardware
 * tanh approximation. */
#define VCSGC_MLP_IN 10
#define VCSGC_MLP_NPARAM 4929

/* Descriptors and exact targets of every site of every replica, on the
 * current (committed) species.  DEVICE outputs owned by the caller:
 * d_X[rows][10] (float, raw counts own[1..5], nb[1..5]) and d_Y[rows]
 * (float, E(i = B) - E(i = A) in eV), rows = sum of the replica sizes,
 * replica after replica in site order.  Errors: STATE when the context has
 * neither form of the five-shell rigid lattice above; CUDA. */
int vcsgc_features(void* ctx, float* d_X, float* d_Y);

/* A surrogate network on the current device: FP32 master parameters (copied
 * from the HOST array params[VCSGC_MLP_NPARAM]), Adam moments (zero) and
 * packed BF16 fragments.  Work runs on `stream` (NULL: a stream of its own).
 * Errors: INVALID_ARG, NONFINITE (a parameter is NaN or Inf), NOMEM, CUDA. */
int vcsgc_mlp_create(void** mlp, const float* params, void* stream);
/* Replace the parameters (HOST array); the Adam state restarts. */
int vcsgc_mlp_set_params(void* mlp, const float* params);
/* Copy the current FP32 parameters to the HOST array params. */
int vcsgc_mlp_get_params(void* mlp, float* params);
/* g for n raw descriptors: DEVICE d_X[n][10] in, DEVICE d_out[n] out (the
 * same arithmetic as stage 1 of the colour step).  Waits for the result. */
int vcsgc_mlp_forward(void* mlp, const float* d_X, int64_t n, float* d_out);
/* Gradient of the mean squared error (1/n) sum (g - y)^2 over all n rows
 * (DEVICE d_X[n][10], d_Y[n]): HOST grad[VCSGC_MLP_NPARAM] and *loss. */
int vcsgc_mlp_grad(void* mlp, const float* d_X, const float* d_Y, int64_t n, float* grad, double* loss);
/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8; learning rate lr
 * decaying by a half cosine to lr / 100 over the call's steps) on
 * minibatches of `batch` rows drawn with replacement from the n rows
 * (Philox keyed by seed, counter = Adam step).  loss_hist (HOST, `steps`
 * entries, or NULL) receives each minibatch's mean squared error before its
 * update.  Runs as a CUDA graph of 32 steps on the surrogate's stream. */
int vcsgc_mlp_train(void* mlp, const float* d_X, const float* d_Y, int64_t n, int64_t batch, int64_t steps,
                    double lr, uint64_t seed, double* loss_hist);
const char* vcsgc_mlp_last_error(void* mlp);
void vcsgc_mlp_free(void* mlp);

/* Turn delayed acceptance on with a copy of the surrogate's current weights
 * (later changes to mlp do not reach the context), or off when mlp is NULL.
 * Applies to every replica from the next colour step.  Errors: STATE as for
 * vcsgc_features; CUDA. */
int vcsgc_set_surrogate(void* ctx, void* mlp);

/* The paper's MD ensemble (Sec. IV B: Nose-Hoover thermostat and
 * barostat) for md_steps and vcsgc_hybrid: kind 0 Langevin (BAOAB with the
 * options' gamma, the default), 1 NVT with a Nose-Hoover chain of `chain`
 * links (<= 4), 2 NPT with the isotropic MTK barostat at p_ext_bar (bar),
 * its own chain, and the box scaled uniformly (Martyna, Tobias, Klein, J.
 * Chem. Phys. 101, 4177 (1994); the Trotter-split step of Martyna,
 * Tuckerman, Tobias, Klein, Mol. Phys. 87, 1117 (1996)).  t_damp, p_damp:
 * relaxation times (fs); masses Q_1 = N_f kT t_damp^2, Q_k = kT t_damp^2,
 * W = (N_f + 3) kT p_damp^2, barostat chain kT p_damp^2, N_f = 3 N, T the
 * options' T_md.  Resets the chains and the barostat velocity.  Errors:
 * INVALID_ARG; STATE (not explicit positions with one replica, or NPT with
 * precision MIXED: the barostat needs the FP64 virial). */
int vcsgc_set_ensemble(void* ctx, int32_t kind, double t_damp, double p_damp, double p_ext_bar, int32_t chain);
/* HOST out[9]: kinetic energy (eV), potential energy (eV), temperature (K),
 * pressure (bar, from the virial), volume (A^3), the extended energy the
 * Nose-Hoover steps conserve (eV), box lengths (A).  Synchronises; evaluates
 * the forces.  Errors: STATE, CUDA, device error bits. */
int vcsgc_md_state(void* ctx, double* out);
/* Conjugate-gradient relaxation of the explicit positions at fixed box and
 * species (the pre-relaxation of Sec. IV B): Polak-Ribiere directions with
 * restarts, a line search for a zero of the directional derivative
 * (extension, then regula falsi), until max_i |F_i| < ftol (eV/A) or
 * max_iter iterations.  *iters and *fmax (HOST, may be NULL) report the
 * iterations taken and the final max |F_i|; the tracked energy restarts from
 * the relaxed positions.  Errors: INVALID_ARG, STATE, CUDA, device bits. */
int vcsgc_minimize(void* ctx, double ftol, int64_t max_iter, int64_t* iters, double* fmax);

/* Checkpoint and resume.  vcsgc_save applies the pending commit and writes
 * to `path` every replica's species, its running state (step counters, B
 * count, tracked energy, acceptance counters, concentration sums), the
 * fused form's step base, and for explicit positions the positions, box,
 * velocities, MD step and Nose-Hoover state.  vcsgc_load restores them into
 * a context created from the same lattice, tables and options (checked:
 * sizes, replica count, schedule, form); the Philox streams are counters, so
 * n sweeps, save, load into a new context and m sweeps give the species of
 * n + m sweeps bit for bit.  The surrogate (vcsgc_set_surrogate) is not
 * saved.  Positions read back are reduced into [0, L) per axis.  Errors:
 * INVALID_ARG (path, mismatch, or a box that is not finite or not longer
 * than 2 r_c), CUDA. */
int vcsgc_save(void* ctx, const char* path);
int vcsgc_load(void* ctx, const char* path);

/* Text of the last error of ctx (or of the last failed vcsgc_init when ctx
 * is NULL).  Valid until the next call on the same context. */
const char* vcsgc_last_error(void* ctx);

/* Release the context and all its device memory.  NULL is a no-op. */
void vcsgc_free(void* ctx);

/* ------------------------------------------------------ multicomponent
 * K-species form (2 <= K <= 4) of the parallel transmutation step on a
 * rigid BCC lattice.  The paper derives the method for binary alloys and
 * notes that more species follow directly (Sec. II); this form keeps one
 * variance constraint per solute species alpha = 1..K-1 (species 0 is the
 * solvent):
 *   pi_V ~ exp{-beta [U + sum_alpha (phi_alpha n_alpha + kappa_p,alpha n_alpha^2)]},
 *   kappa_p,alpha = kappa_alpha kB T / N (kappa dimensionless).
 * A trial at site i of species a proposes b uniformly among the other K-1
 * species (Philox (step, domain rank, 6)); the local stage (Eq.
 * trans_vcsgc_par1 per solute) accepts with
 *   min{1, exp[-beta (dE_i + dmu0_b - dmu0_a)]},
 *   dmu0_alpha = phi_alpha + 2 kappa_p,alpha N c0_alpha, dmu0_0 = 0,
 * and the global stage (Eq. trans_vcsgc_par2 per solute) with
 *   min{1, exp[-beta sum_alpha kappa_p,alpha dn_alpha (dn_alpha + 2 (n_alpha - N c0_alpha))]}.
 * Schedule: the period-q sublattice (colour (cx mod qx, cy mod qy, cz mod
 * qz, basis), every site of the colour trialled at once); q a > 2 r_c is
 * required.  For K = 2 the chain is the binary one of vcsgc_init with the
 * SUBLATTICE schedule. */
#define VCSGC_MULTI_MAX_K 4

/* EAM tables of K species, grids as for vcsgc_eam_tables: pair[p] for the
 * unordered pair p = tri(a, b), a <= b, in the order (0,0), (0,1), ...,
 * (0,K-1), (1,1), ..., (K-1,K-1); dens[a]; embed[a].  Derivative arrays may
 * be NULL (central differences). */
typedef struct {
  int32_t K;
  int32_t nr;
  double dr;
  int32_t nrho;
  double drho;
  double rc;
  const double* pair[10];
  const double* dpair[10];
  const double* dens[4];
  const double* ddens[4];
  const double* embed[4];
  const double* dembed[4];
} vcsgc_multi_tables;

typedef struct {
  int64_t n_sites;
  int32_t K;
  int32_t pad;
  int64_t n[4];           /* sites of each species */
  double c[4];
  double energy;          /* total energy (eV): tracked step by step, or, with
                             re-embedding (the screened form), recomputed in
                             full by this call */
  double energy_per_atom;
  int64_t steps, trials, local_accepts, global_trials, global_accepts, flips, near_ties;
  double acc_local, acc_global;
  double mean_c[4];       /* <c_alpha> over steps */
  double var_c[4];
  double dmu_est[4];      /* phi_alpha + 2 kappa_p,alpha N <c_alpha> (Eq. gforce per solute) */
  double kappa_p[4];      /* eV */
  double dmu0[4];         /* eV */
  double sweeps;          /* trials / N */
  int64_t stage1_accepts; /* delayed acceptance: trials that passed stage 1 */
} vcsgc_multi_obs;

/* Create a K-species context of n_replicas copies of one rigid lattice
 * (lattice->kind 0; each edge at least 2 r_c long).  HOST inputs, copied:
 * types[n_replicas][N] (values < K), phi, kappa, c0 [n_replicas][K-1]
 * (replica-major; c0 < 0: the replica's initial concentration of that
 * species), T[n_replicas], seed_r[n_replicas] (Philox keys; NULL: r + 1).
 * period[3] = (qx, qy, qz) divides the cell counts.  stream: a cudaStream_t
 * or NULL (the context makes its own); device < 0: the current device.
 * With species-dependent densities on the five-shell neighbourhood (and at
 * most 1024 replicas) the local decision is taken on an FP32 dE within a
 * proven error bound, FP64 where the bound cannot decide: every decision is
 * the FP64 one; the energy is then recomputed by vcsgc_multi_observables.
 * Errors: INVALID_ARG (sizes, species, K, period), SCHEDULE (q a <= 2 r_c),
 * NOMEM, CUDA, TABLE_RANGE (a shell outside the grids). */
int vcsgc_multi_init(void** out, const vcsgc_lattice* lattice, const uint8_t* types, const vcsgc_multi_tables* tables,
                     int32_t n_replicas, const double* phi, const double* kappa, const double* T, const double* c0,
                     const uint64_t* seed_r, const int32_t period[3], void* stream, int32_t device);
/* n sweeps (N / (sites per colour) colour steps each) or n colour steps on
 * every replica; asynchronous on the context's stream.  Errors: CUDA. */
int vcsgc_multi_sweep(void* m, int64_t n);
int vcsgc_multi_steps(void* m, int64_t n);
int vcsgc_multi_steps_per_sweep(void* m, int64_t* out);
/* Synchronises; fills *out for replica r.  Errors: INVALID_ARG, CUDA, and
 * the device error bits (TABLE_RANGE, NONFINITE). */
int vcsgc_multi_observables(void* m, int32_t r, vcsgc_multi_obs* out);
/* Species of replica r, HOST buffers of N bytes.  set_types recomputes the
 * densities, counts and energy and keeps the counters.  Errors: INVALID_ARG
 * (r, a value >= K), CUDA. */
int vcsgc_multi_get_types(void* m, int32_t r, uint8_t* out);
int vcsgc_multi_set_types(void* m, int32_t r, const uint8_t* in);
/* dE of site sites[q] becoming species to[q] in replica r (HOST arrays of
 * n; out HOST).  Errors: INVALID_ARG, CUDA, device error bits. */
int vcsgc_multi_delta_e(void* m, int32_t r, const int64_t* sites, const uint8_t* to, int64_t n, double* out);
/* Full energy of replica r from its species and densities (eV). */
int vcsgc_multi_energy(void* m, int32_t r, double* out);
/* Delayed acceptance (the two stages of vcsgc_set_surrogate) for K = 2 with
 * species-dependent densities on the five-shell table (the screened form):
 * stage 1 on the surrogate's g from the descriptor, stage 2 on the exact
 * dE - s g (FP32-screened, FP64 where the bound cannot decide).  The
 * descriptor comes from per-site B counts by shell (4 bytes per site),
 * built from the species when delayed acceptance is turned on or the
 * species were set, and updated by the commit of every accepted step.  The
 * context keeps a copy of the surrogate's current weights; mlp NULL turns
 * it off.  Errors: STATE (K != 2 or not the screened form), INVALID_ARG,
 * NOMEM, CUDA. */
int vcsgc_multi_set_surrogate(void* m, void* mlp);
/* Descriptors and exact targets of every site of every replica (the rows
 * and units of vcsgc_features: DEVICE d_X[R N][10] raw counts, d_Y[R N]
 * E(i = B) - E(i = A) in eV, replica after replica in site order), from the
 * per-site counts and the FP64 dE.  Synchronises.  Errors: as
 * vcsgc_multi_set_surrogate, and the device error bits. */
int vcsgc_multi_features(void* m, float* d_X, float* d_Y);
const char* vcsgc_multi_last_error(void* m);
void vcsgc_multi_free(void* m);

#ifdef __cplusplus
}
#endif
#endif
