/*
 * vcsgc_multi.c -- serial FP64 CPU oracle for the K-species (multicomponent)
 * generalisation of the parallel VC-SGC transmutation step.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow reference the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library.
 *
 * The paper derives the ensemble and the algorithms for a binary alloy and
 * states that the generalisation to any number of species is
 * straightforward (Sec. II).  This file takes the following reading of it:
 *
 *   Ensemble.  Species 0 is the reference (solvent); for each solute
 *   alpha = 1..K-1 with n_alpha sites, one variance constraint of the form of
 *   Eq. pi_vcsgc:
 *     pi_V ~ exp{-beta [U + sum_alpha (phi_alpha n_alpha + kappa_p,alpha n_alpha^2)]},
 *   kappa_p,alpha = kappa_alpha kB T / N (kappa dimensionless).
 *
 *   Trial move.  Site i of species a becomes species b, drawn uniformly from
 *   the K - 1 others (a symmetric proposal): dn_alpha = [b = alpha] - [a = alpha].
 *
 *   Composite move (Sec. III B 2, Eqs. trans_vcsgc_par1 and _par2 per
 *   solute).  With n0_alpha = N c0_alpha and dmu0_alpha = phi_alpha +
 *   2 kappa_p,alpha n0_alpha (dmu0_0 = 0), the ratio of pi_V between the
 *   configurations after and before a composite move with changes dn_alpha is
 *     exp{-beta [dU + sum_alpha dmu0_alpha dn_alpha
 *                 + sum_alpha kappa_p,alpha dn_alpha (dn_alpha + 2 (n_alpha - n0_alpha))]}.
 *   The first two terms are sums over the trial sites of
 *   dE_i + dmu0_b - dmu0_a (the local stage, one factor per domain); the
 *   last is the global stage.  For K = 2 both reduce to the binary rules.
 *
 * Random numbers (Philox, key = seed): the colour from (step, 0xFFFFFFFF,
 * tag 1); per domain rank d, the site and the local u from (step, d, tag 0),
 * the new species from (step, d, tag 6) as b = (a + 1 + below(K - 1)) mod K;
 * the global u from the colour draw's second word pair.  For K = 2 the
 * species draw is not needed and the chain is the binary one.
 */
#include "vcsgc_multi.h"
#include "orc_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KB_EV 8.617333262e-5

typedef struct {
  int64_t j;
  double r;
  int sx, sy, sz;
} mnbr_t;

struct orcm_sys {
  int64_t n;
  int K, P;
  double box[3];
  double *x, *y, *z;
  uint8_t* t;
  double* rho;
  spline_t pair[ORCM_MAX_PAIRS], dens[ORCM_MAX_K], embed[ORCM_MAX_K];
  double rc;
  int64_t* nstart;
  mnbr_t* nb;
  /* ensemble (index alpha = 0..K-1; entry 0 unused: the solvent) */
  double T, beta;
  double phi[ORCM_MAX_K], kappa[ORCM_MAX_K], kappa_p[ORCM_MAX_K], n0[ORCM_MAX_K], dmu0[ORCM_MAX_K];
  uint32_t key[2];
  uint64_t step;
  int64_t cnt[ORCM_MAX_K];
  double energy;
  /* counters */
  int64_t trials, local_acc, global_trials, global_acc, flips, near_ties, steps_done;
  double sum_c[ORCM_MAX_K], sum_c2[ORCM_MAX_K];
  /* schedule: col_start[n_colours+1] -> domains, dom_start -> dom_sites */
  int64_t n_colours, n_domains;
  int64_t *col_start, *dom_start, *dom_sites;
};

int orcm_tri(int K, int a, int b) {
  if (a > b) { int q = a; a = b; b = q; }
  return a * K - a * (a - 1) / 2 + (b - a);
}

static double phi_of(const orcm_sys* s, int a, int b, double r) {
  double v;
  if (orc_hermite_eval(&s->pair[orcm_tri(s->K, a, b)], r, &v, NULL)) return NAN;
  return v;
}
static double dens_of(const orcm_sys* s, int a, double r) {
  double v;
  if (orc_hermite_eval(&s->dens[a], r, &v, NULL)) return NAN;
  return v;
}
static double embed_of(const orcm_sys* s, int a, double rho) {
  double v;
  if (orc_hermite_eval(&s->embed[a], rho, &v, NULL)) return NAN;
  return v;
}

/* --------------------------------------------------------- neighbour list */
static int cmp_mnbr(const void* pa, const void* pb) {
  const mnbr_t* a = (const mnbr_t*)pa;
  const mnbr_t* b = (const mnbr_t*)pb;
  if (a->r != b->r) return a->r < b->r ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->sx != b->sx) return a->sx < b->sx ? -1 : 1;
  if (a->sy != b->sy) return a->sy < b->sy ? -1 : 1;
  if (a->sz != b->sz) return a->sz < b->sz ? -1 : 1;
  return 0;
}

/* Every j and every periodic image within r_c, sorted by (r, j, image). */
static int build_neighbours(orcm_sys* s) {
  int m[3];
  for (int a = 0; a < 3; ++a) m[a] = (int)ceil(s->rc / s->box[a]) + 1;
  const double rc2 = s->rc * s->rc;
  int64_t cap = 1024, used = 0;
  mnbr_t* v = (mnbr_t*)malloc(sizeof(mnbr_t) * cap);
  s->nstart = (int64_t*)malloc(sizeof(int64_t) * (s->n + 1));
  if (!v || !s->nstart) { free(v); return -1; }
  for (int64_t i = 0; i < s->n; ++i) {
    s->nstart[i] = used;
    for (int64_t j = 0; j < s->n; ++j)
      for (int sx = -m[0]; sx <= m[0]; ++sx)
        for (int sy = -m[1]; sy <= m[1]; ++sy)
          for (int sz = -m[2]; sz <= m[2]; ++sz) {
            if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
            double dx = s->x[j] + sx * s->box[0] - s->x[i];
            double dy = s->y[j] + sy * s->box[1] - s->y[i];
            double dz = s->z[j] + sz * s->box[2] - s->z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= rc2) continue;
            if (used == cap) {
              cap *= 2;
              mnbr_t* p = (mnbr_t*)realloc(v, sizeof(mnbr_t) * cap);
              if (!p) { free(v); return -1; }
              v = p;
            }
            mnbr_t e = {j, sqrt(r2), sx, sy, sz};
            v[used++] = e;
          }
    qsort(v + s->nstart[i], (size_t)(used - s->nstart[i]), sizeof(mnbr_t), cmp_mnbr);
  }
  s->nstart[s->n] = used;
  s->nb = v;
  return 0;
}

static void compute_rho(orcm_sys* s) {
  for (int64_t i = 0; i < s->n; ++i) {
    double r = 0.0;
    for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k) r += dens_of(s, s->t[s->nb[k].j], s->nb[k].r);
    s->rho[i] = r;
  }
}

/* ---------------------------------------------------------------- energy */
typedef struct { double s, c; } ksum;
static void kadd(ksum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

/* U = sum_i [ 1/2 sum_j phi_{t_i t_j}(r_ij) + F_{t_i}(rho_i) ],
 * rho_i = sum_j f_{t_j}(r_ij). */
double orcm_energy_full(const orcm_sys* s) {
  ksum acc = {0, 0};
  for (int64_t i = 0; i < s->n; ++i) {
    int ti = s->t[i];
    double rho = 0.0;
    for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k) {
      const mnbr_t* e = &s->nb[k];
      kadd(&acc, 0.5 * phi_of(s, ti, s->t[e->j], e->r));
      rho += dens_of(s, s->t[e->j], e->r);
    }
    kadd(&acc, embed_of(s, ti, rho));
  }
  return acc.s + acc.c;
}

/* Energy change of site i going from a = t_i to b:
 *   pair:     sum_k [phi_{b t_k}(r_ik) - phi_{a t_k}(r_ik)]
 *   own:      F_b(rho_i) - F_a(rho_i)        (rho_i does not depend on t_i)
 *   re-embed: sum over distinct neighbours j of
 *             F_{t_j}(rho_j + drho_j) - F_{t_j}(rho_j),
 *             drho_j = sum over the slots of j of f_b(r) - f_a(r). */
double orcm_delta_e(const orcm_sys* s, int64_t i, int b) {
  int a = s->t[i];
  if (a == b) return 0.0;
  int64_t lo = s->nstart[i], hi = s->nstart[i + 1];
  double pair = 0.0;
  int any_drho = 0;
  for (int64_t k = lo; k < hi; ++k) {
    const mnbr_t* e = &s->nb[k];
    int tk = s->t[e->j];
    pair += phi_of(s, b, tk, e->r) - phi_of(s, a, tk, e->r);
    if (dens_of(s, b, e->r) - dens_of(s, a, e->r) != 0.0) any_drho = 1;
  }
  double own = embed_of(s, b, s->rho[i]) - embed_of(s, a, s->rho[i]);
  double reembed = 0.0;
  if (any_drho) {
    for (int64_t k = lo; k < hi; ++k) {
      int64_t j = s->nb[k].j;
      int seen = 0;
      for (int64_t q = lo; q < k; ++q)
        if (s->nb[q].j == j) { seen = 1; break; }
      if (seen) continue;
      double drho = 0.0;
      for (int64_t q = k; q < hi; ++q)
        if (s->nb[q].j == j) drho += dens_of(s, b, s->nb[q].r) - dens_of(s, a, s->nb[q].r);
      int tj = s->t[j];
      reembed += embed_of(s, tj, s->rho[j] + drho) - embed_of(s, tj, s->rho[j]);
    }
  }
  return pair + own + reembed;
}

/* site i becomes species b: scatter the density change, update the counts */
static void set_species(orcm_sys* s, int64_t i, int b) {
  int a = s->t[i];
  for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k) {
    const mnbr_t* e = &s->nb[k];
    s->rho[e->j] += dens_of(s, b, e->r) - dens_of(s, a, e->r);
  }
  s->t[i] = (uint8_t)b;
  s->cnt[a]--;
  s->cnt[b]++;
}

double orcm_delta_e_full(orcm_sys* s, int64_t i, int b) {
  double e0 = orcm_energy_full(s);
  uint8_t a = s->t[i];
  s->t[i] = (uint8_t)b;
  double e1 = orcm_energy_full(s);
  s->t[i] = a;
  return e1 - e0;
}

/* ---------------------------------------------------------------- create */
orcm_sys* orcm_create(int64_t n, const double* x, const double* y, const double* z,
                      const double box[3], const uint8_t* types, const orcm_eam_in* eam) {
  if (n <= 0 || !eam || eam->K < 2 || eam->K > ORCM_MAX_K || eam->nr < 2 || eam->nrho < 2) return NULL;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > eam->rc)) return NULL;
  for (int64_t i = 0; i < n; ++i)
    if (types[i] >= eam->K) return NULL;
  orcm_sys* s = (orcm_sys*)calloc(1, sizeof(orcm_sys));
  if (!s) return NULL;
  s->n = n;
  s->K = eam->K;
  s->P = eam->K * (eam->K + 1) / 2;
  memcpy(s->box, box, sizeof(double) * 3);
  s->x = (double*)malloc(sizeof(double) * n);
  s->y = (double*)malloc(sizeof(double) * n);
  s->z = (double*)malloc(sizeof(double) * n);
  s->t = (uint8_t*)malloc(n);
  s->rho = (double*)malloc(sizeof(double) * n);
  if (!s->x || !s->y || !s->z || !s->t || !s->rho) { orcm_free(s); return NULL; }
  for (int64_t i = 0; i < n; ++i) {
    s->x[i] = x[i] - floor(x[i] / box[0]) * box[0];
    s->y[i] = y[i] - floor(y[i] / box[1]) * box[1];
    s->z[i] = z[i] - floor(z[i] / box[2]) * box[2];
    if (s->x[i] >= box[0]) s->x[i] = 0.0;
    if (s->y[i] >= box[1]) s->y[i] = 0.0;
    if (s->z[i] >= box[2]) s->z[i] = 0.0;
  }
  memcpy(s->t, types, n);
  s->rc = eam->rc;
  for (int p = 0; p < s->P; ++p)
    if (orc_hermite_init(&s->pair[p], eam->nr, eam->dr, eam->pair[p], eam->dpair[p])) { orcm_free(s); return NULL; }
  for (int a = 0; a < s->K; ++a) {
    if (orc_hermite_init(&s->dens[a], eam->nr, eam->dr, eam->dens[a], eam->ddens[a])) { orcm_free(s); return NULL; }
    if (orc_hermite_init(&s->embed[a], eam->nrho, eam->drho, eam->embed[a], eam->dembed[a])) { orcm_free(s); return NULL; }
  }
  if (build_neighbours(s)) { orcm_free(s); return NULL; }
  compute_rho(s);
  for (int64_t i = 0; i < n; ++i) s->cnt[s->t[i]]++;
  s->energy = orcm_energy_full(s);
  return s;
}

void orcm_free(orcm_sys* s) {
  if (!s) return;
  free(s->x); free(s->y); free(s->z); free(s->t); free(s->rho);
  for (int p = 0; p < ORCM_MAX_PAIRS; ++p) { free(s->pair[p].y); free(s->pair[p].m); }
  for (int a = 0; a < ORCM_MAX_K; ++a) {
    free(s->dens[a].y); free(s->dens[a].m); free(s->embed[a].y); free(s->embed[a].m);
  }
  free(s->nstart); free(s->nb);
  free(s->col_start); free(s->dom_start); free(s->dom_sites);
  free(s);
}

int orcm_set_params(orcm_sys* s, const double* phi, const double* kappa, double T, const double* c0,
                    uint64_t seed) {
  if (!(T > 0.0)) return -1;
  s->T = T;
  s->beta = 1.0 / (KB_EV * T);
  s->phi[0] = s->kappa[0] = s->kappa_p[0] = s->n0[0] = s->dmu0[0] = 0.0;
  for (int al = 1; al < s->K; ++al) {
    s->phi[al] = phi[al - 1];
    s->kappa[al] = kappa[al - 1];
    s->kappa_p[al] = kappa[al - 1] * KB_EV * T / (double)s->n;
    double c = c0[al - 1] < 0.0 ? (double)s->cnt[al] / (double)s->n : c0[al - 1];
    s->n0[al] = (double)s->n * c;
    s->dmu0[al] = s->phi[al] + 2.0 * s->kappa_p[al] * s->n0[al];
  }
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->step = 0;
  s->trials = s->local_acc = s->global_trials = s->global_acc = s->flips = s->near_ties = 0;
  s->steps_done = 0;
  for (int al = 0; al < ORCM_MAX_K; ++al) s->sum_c[al] = s->sum_c2[al] = 0.0;
  return 0;
}

/* -------------------------------------------------------------- schedule */
static int sched_alloc(orcm_sys* s, int64_t n_colours, int64_t n_domains) {
  free(s->col_start); free(s->dom_start); free(s->dom_sites);
  s->col_start = (int64_t*)calloc(n_colours + 1, sizeof(int64_t));
  s->dom_start = (int64_t*)calloc(n_domains + 1, sizeof(int64_t));
  s->dom_sites = (int64_t*)calloc(s->n, sizeof(int64_t));
  s->n_colours = n_colours;
  s->n_domains = n_domains;
  return (s->col_start && s->dom_start && s->dom_sites) ? 0 : -1;
}

/* colour (cx mod qx, cy mod qy, cz mod qz, basis): every site of the colour
 * is a domain of its own, in ascending site index */
int orcm_schedule_sublattice(orcm_sys* s, int nx, int ny, int nz, int qx, int qy, int qz) {
  if ((int64_t)2 * nx * ny * nz != s->n) return -1;
  if (qx < 1 || qy < 1 || qz < 1 || nx % qx || ny % qy || nz % qz) return -1;
  int64_t ncol = (int64_t)qx * qy * qz * 2;
  if (sched_alloc(s, ncol, s->n)) return -1;
  int64_t dom = 0;
  for (int64_t c = 0; c < ncol; ++c) {
    s->col_start[c] = dom;
    for (int64_t i = 0; i < s->n; ++i) {
      int64_t b = i % 2, cell = i / 2;
      int64_t cx = cell % nx, cy = (cell / nx) % ny, cz = cell / ((int64_t)nx * ny);
      if ((((cz % qz) * qy + (cy % qy)) * qx + (cx % qx)) * 2 + b != c) continue;
      s->dom_start[dom] = dom;
      s->dom_sites[dom] = i;
      ++dom;
    }
  }
  s->col_start[ncol] = dom;
  s->dom_start[dom] = dom;
  return 0;
}

/* blocks of bx*by*bz cells; colour = block index mod p per axis */
int orcm_schedule_blocks(orcm_sys* s, int nx, int ny, int nz, int bx, int by, int bz, int px, int py,
                         int pz) {
  if ((int64_t)2 * nx * ny * nz != s->n) return -1;
  if (bx < 1 || by < 1 || bz < 1 || px < 1 || py < 1 || pz < 1) return -1;
  if (nx % bx || ny % by || nz % bz) return -1;
  int nbx = nx / bx, nby = ny / by, nbz = nz / bz;
  if (nbx % px || nby % py || nbz % pz) return -1;
  int64_t ncol = (int64_t)px * py * pz;
  if (sched_alloc(s, ncol, (int64_t)nbx * nby * nbz)) return -1;
  int64_t dom = 0, site = 0;
  for (int64_t c = 0; c < ncol; ++c) {
    s->col_start[c] = dom;
    for (int ibz = 0; ibz < nbz; ++ibz)
      for (int iby = 0; iby < nby; ++iby)
        for (int ibx = 0; ibx < nbx; ++ibx) {
          if (((int64_t)(ibz % pz) * py + (iby % py)) * px + (ibx % px) != c) continue;
          s->dom_start[dom++] = site;
          for (int lz = 0; lz < bz; ++lz)
            for (int ly = 0; ly < by; ++ly)
              for (int lx = 0; lx < bx; ++lx)
                for (int b = 0; b < 2; ++b) {
                  int64_t cx = (int64_t)ibx * bx + lx, cy = (int64_t)iby * by + ly, cz = (int64_t)ibz * bz + lz;
                  s->dom_sites[site++] = ((cz * ny + cy) * nx + cx) * 2 + b;
                }
        }
  }
  s->col_start[ncol] = dom;
  s->dom_start[dom] = site;
  return 0;
}

/* ------------------------------------------------------------- sampling */
static void draw(const orcm_sys* s, uint64_t k, uint32_t d, uint32_t tag, uint32_t w[4]) {
  uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(k >> 32), d, tag};
  orc_philox(ctr, s->key, w);
}

/* accept with probability min{1, exp(-X)}; flag |u - p| <= 1e-9 p */
static int metropolis(orcm_sys* s, double X, double u) {
  if (X <= 0.0) {
    if (X > -1e-9 && u >= 1.0 - 1e-9) s->near_ties++;
    return 1;
  }
  double p = exp(-X);
  if (fabs(u - p) <= 1e-9 * p) s->near_ties++;
  return u < p;
}

static void sample_c(orcm_sys* s) {
  for (int al = 0; al < s->K; ++al) {
    double c = (double)s->cnt[al] / (double)s->n;
    s->sum_c[al] += c;
    s->sum_c2[al] += c * c;
  }
  s->steps_done++;
}

/* One composite step: colour c; in every domain of c one site i (species
 * a) proposes species b; local stage min{1, exp[-beta (dE_i + dmu0_b -
 * dmu0_a)]}; dn_alpha summed over the local accepts; global stage
 * min{1, exp[-beta sum_alpha kappa_p,alpha dn_alpha (dn_alpha + 2 (n_alpha
 * - n0_alpha))]}; if accepted every local accept is applied. */
static void parallel_step(orcm_sys* s, int64_t* acc_site, int* acc_to, double* acc_de) {
  uint64_t k = s->step;
  uint32_t w[4], w6[4];
  draw(s, k, 0xFFFFFFFFu, 1u, w);
  int64_t c = (int64_t)orc_below(w[0], w[1], (uint64_t)s->n_colours);
  double ug = orc_u01(w[2], w[3]);
  int64_t d0 = s->col_start[c], d1 = s->col_start[c + 1];
  int64_t nacc = 0;
  int64_t dn[ORCM_MAX_K] = {0, 0, 0, 0};
  for (int64_t g = d0; g < d1; ++g) {
    int64_t size = s->dom_start[g + 1] - s->dom_start[g];
    if (size == 0) continue;
    draw(s, k, (uint32_t)(g - d0), 0u, w);
    int64_t site = s->dom_sites[s->dom_start[g] + orc_below(w[0], w[1], (uint64_t)size)];
    double u = orc_u01(w[2], w[3]);
    int a = s->t[site], b;
    if (s->K == 2) {
      b = 1 - a;
    } else {
      draw(s, k, (uint32_t)(g - d0), 6u, w6);
      b = (int)((a + 1 + (int)orc_below(w6[0], w6[1], (uint64_t)(s->K - 1))) % s->K);
    }
    s->trials++;
    double de = orcm_delta_e(s, site, b);
    if (metropolis(s, s->beta * (de + (s->dmu0[b] - s->dmu0[a])), u)) {
      acc_site[nacc] = site;
      acc_to[nacc] = b;
      acc_de[nacc] = de;
      nacc++;
      dn[b]++;
      dn[a]--;
    }
  }
  s->local_acc += nacc;
  if (nacc > 0) {
    s->global_trials++;
    double Y = 0.0;
    for (int al = 1; al < s->K; ++al)
      Y += s->beta * s->kappa_p[al] * (double)dn[al] * ((double)dn[al] + 2.0 * ((double)s->cnt[al] - s->n0[al]));
    if (metropolis(s, Y, ug)) {
      s->global_acc++;
      for (int64_t q = 0; q < nacc; ++q) {
        set_species(s, acc_site[q], acc_to[q]);
        s->energy += acc_de[q];
      }
      s->flips += nacc;
    }
  }
  s->step++;
  sample_c(s);
}

int orcm_parallel_steps(orcm_sys* s, int64_t n_steps) {
  if (!s->n_colours) return -1;
  int64_t maxd = 1;
  for (int64_t c = 0; c < s->n_colours; ++c)
    if (s->col_start[c + 1] - s->col_start[c] > maxd) maxd = s->col_start[c + 1] - s->col_start[c];
  int64_t* sites = (int64_t*)malloc(sizeof(int64_t) * maxd);
  int* to = (int*)malloc(sizeof(int) * maxd);
  double* des = (double*)malloc(sizeof(double) * maxd);
  if (!sites || !to || !des) { free(sites); free(to); free(des); return -1; }
  for (int64_t q = 0; q < n_steps; ++q) parallel_step(s, sites, to, des);
  free(sites); free(to); free(des);
  return 0;
}

int orcm_run_histogram(orcm_sys* s, int64_t n_steps, int64_t* hist, double* sum_e) {
  for (int64_t q = 0; q < n_steps; ++q) {
    if (orcm_parallel_steps(s, 1)) return -1;
    int64_t bin = 0;
    for (int al = s->K - 1; al >= 1; --al) bin = bin * (s->n + 1) + s->cnt[al];
    hist[bin]++;
    *sum_e += s->energy;
  }
  return 0;
}

/* ------------------------------------------------------------- accessors */
void orcm_get_types(const orcm_sys* s, uint8_t* out) { memcpy(out, s->t, s->n); }

void orcm_set_types(orcm_sys* s, const uint8_t* in) {
  memcpy(s->t, in, s->n);
  for (int al = 0; al < ORCM_MAX_K; ++al) s->cnt[al] = 0;
  for (int64_t i = 0; i < s->n; ++i) s->cnt[s->t[i]]++;
  compute_rho(s);
  s->energy = orcm_energy_full(s);
}

void orcm_get_rho(const orcm_sys* s, double* out) { memcpy(out, s->rho, sizeof(double) * s->n); }

void orcm_get_obs(const orcm_sys* s, orcm_obs* o) {
  memset(o, 0, sizeof(*o));
  o->n_sites = s->n;
  o->K = s->K;
  for (int al = 0; al < s->K; ++al) {
    o->n[al] = s->cnt[al];
    o->sum_c[al] = s->sum_c[al];
    o->sum_c2[al] = s->sum_c2[al];
  }
  o->energy = s->energy;
  o->steps = s->steps_done;
  o->trials = s->trials;
  o->local_accepts = s->local_acc;
  o->global_trials = s->global_trials;
  o->global_accepts = s->global_acc;
  o->flips = s->flips;
  o->near_ties = s->near_ties;
}
