/* Multicomponent VC-SGC oracle: serial FP64 reference of the K-species
 * generalisation of the parallel transmutation step (K <= 4).
 * TEST INFRASTRUCTURE ONLY (see vcsgc_multi.c). */
#ifndef VCSGC_MULTI_ORACLE_H
#define VCSGC_MULTI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORCM_MAX_K 4
#define ORCM_MAX_PAIRS (ORCM_MAX_K * (ORCM_MAX_K + 1) / 2)

/* EAM tables of K species on uniform grids (values and knot derivatives):
 * pair[p] for the unordered species pair p = tri(a, b), a <= b, in the order
 * (0,0), (0,1), ..., (0,K-1), (1,1), ..., (K-1,K-1); dens[a] on the same
 * grid r_j = j dr; embed[a] on rho_j = j drho. */
typedef struct {
  int32_t K;
  int32_t nr;
  double dr;
  int32_t nrho;
  double drho;
  double rc;
  const double* pair[ORCM_MAX_PAIRS];
  const double* dpair[ORCM_MAX_PAIRS];
  const double* dens[ORCM_MAX_K];
  const double* ddens[ORCM_MAX_K];
  const double* embed[ORCM_MAX_K];
  const double* dembed[ORCM_MAX_K];
} orcm_eam_in;

typedef struct orcm_sys orcm_sys;

/* Observables: counts n[alpha] of every species, energy, counters, and the
 * running sums of c_alpha and c_alpha^2 (sampled after every step). */
typedef struct {
  int64_t n_sites;
  int32_t K;
  int32_t pad;
  int64_t n[ORCM_MAX_K];
  double energy;
  int64_t steps, trials, local_accepts, global_trials, global_accepts, flips, near_ties;
  double sum_c[ORCM_MAX_K];
  double sum_c2[ORCM_MAX_K];
} orcm_obs;

int orcm_tri(int K, int a, int b);
/* Positions x, y, z in a periodic box (every image within r_c is listed);
 * types in [0, K).  NULL on bad input. */
orcm_sys* orcm_create(int64_t n, const double* x, const double* y, const double* z,
                      const double box[3], const uint8_t* types, const orcm_eam_in* eam);
void orcm_free(orcm_sys* s);
/* phi, kappa, c0: K - 1 values each, for the solute species 1..K-1; kappa
 * is dimensionless, kappa_p = kappa kB T / N; c0 < 0 takes the current
 * concentration of that species.  Returns 0 or -1. */
int orcm_set_params(orcm_sys* s, const double* phi, const double* kappa, double T, const double* c0,
                    uint64_t seed);
int orcm_schedule_sublattice(orcm_sys* s, int nx, int ny, int nz, int qx, int qy, int qz);
int orcm_schedule_blocks(orcm_sys* s, int nx, int ny, int nz, int bx, int by, int bz, int px, int py,
                         int pz);
int orcm_parallel_steps(orcm_sys* s, int64_t n_steps);
/* Joint histogram of the solute counts over n_steps steps: bin n_1 + (N+1)
 * (n_2 + (N+1) n_3) (K - 1 solutes), plus the sum of the energy. */
int orcm_run_histogram(orcm_sys* s, int64_t n_steps, int64_t* hist, double* sum_e);
double orcm_energy_full(const orcm_sys* s);
/* Energy change of site i becoming species b: incremental and by two full
 * evaluations. */
double orcm_delta_e(const orcm_sys* s, int64_t i, int b);
double orcm_delta_e_full(orcm_sys* s, int64_t i, int b);
void orcm_get_types(const orcm_sys* s, uint8_t* out);
void orcm_set_types(orcm_sys* s, const uint8_t* in);
void orcm_get_rho(const orcm_sys* s, double* out);
void orcm_get_obs(const orcm_sys* s, orcm_obs* o);

#ifdef __cplusplus
}
#endif
#endif
