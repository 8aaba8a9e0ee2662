/*
 * vcsgc_oracle.c -- serial FP64 CPU oracle for the parallel VC-SGC method.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow reference the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library.
 *
 * Written from the paper (Sadigh et al., "A scalable parallel Monte Carlo
 * algorithm for atomistic simulations of precipitation in alloys"):
 *   Sec. II C, Eq. pi_vcsgc ...... target distribution
 *           pi_V ~ exp[-beta (U + phi n + kappa_p n^2)], n = N c
 *   Sec. II C, Eq. trans_vcsgc ... serial acceptance rule
 *   Sec. III B 2, Eq. mod ........ two-factor serial rule (factor 2 restored)
 *   Sec. III B 2, Eq. trans_vcsgc_par1 .. local stage of the composite move
 *   Sec. III B 2, Eq. trans_vcsgc_par2 .. global stage; the sign inside the
 *           bracket is fixed by pi_V: exponent -beta kappa_p dn (dn + 2(n-n0))
 *   Sec. III A ................... non-interacting domains, one colour per
 *           step chosen with a synchronised random stream
 *   Sec. IV A .................... hybrid MD + transmutation MC
 *
 * The only numerical shortcut is none: every energy difference is evaluated
 * neighbour by neighbour from the spline tables, in slot order.
 */
#include "vcsgc_oracle.h"
#include "orc_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KB_EV 8.617333262e-5       /* Boltzmann constant, eV/K */
#define FTM 9.648533212331e-3      /* eV/(Angstrom amu) -> Angstrom/fs^2 */


typedef struct {
  int64_t j;
  double r;
  double d[3];
  int sx, sy, sz;
} nbr_t;

struct orc_sys {
  int64_t n;
  double box[3];
  double *x, *y, *z;
  uint8_t* t;
  double* rho;
  spline_t sp[7]; /* 0..2 pair AA AB BB, 3..4 dens A B, 5..6 embed A B */
  double rc;
  int brute;
  /* neighbour list, CSR */
  int64_t* nstart;
  nbr_t* nb;
  /* ensemble */
  double phi, kappa, T, beta, kappa_p, c0, n0, dmu0;
  uint32_t key[2];
  uint64_t step;
  int64_t nb_count;
  double energy;
  /* counters */
  int64_t trials, local_acc, global_acc, global_trials, flips, near_ties;
  double sum_c, sum_c2;
  int64_t steps_done;
  /* schedule */
  int64_t n_colours, n_domains;
  int64_t *col_start, *dom_start, *dom_sites;
  int64_t* dom_wt;       /* pick weight of each dom_sites entry, or NULL (uniform) */
  int64_t* site_trials;  /* trials per site, or NULL (not counted) */
  int sched_kind; /* 0 none, 1 blocks, 2 sublattice, 3 spatial, 4 overlapping */
  int sched_args[9];
  /* delayed acceptance: stage-1 surrogate of the energy change */
  int sur_kind;          /* 0 off, 1 MLP, 2 the exact energy change */
  double* mlp;           /* ORC_MLP_NPARAM parameters */
  int n_shells;
  double shell_r[ORC_MAX_SHELLS];
  double shell_tol;
  int64_t s1_accepts;    /* trials that passed stage 1 */
  /* md */
  double *vx, *vy, *vz, *fx, *fy, *fz;
  double mass[2], dt, gamma, T_md;
  uint32_t md_key[2];
  uint64_t md_step;
  /* Nose-Hoover ensembles: 0 Langevin (BAOAB), 1 NVT, 2 NPT (isotropic) */
  int ens;
  int chain;                               /* thermostat chain length M */
  double t_damp, p_damp, p_ext;            /* fs, fs, eV/A^3 */
  double xi[ORC_MAX_CHAIN], eta[ORC_MAX_CHAIN], Q[ORC_MAX_CHAIN];
  double xib[ORC_MAX_CHAIN], etab[ORC_MAX_CHAIN], Qb[ORC_MAX_CHAIN];
  double veps, W;                          /* barostat velocity (1/fs) and mass */
  double virial;                           /* sum over pairs r_ij . F_ij (eV) */
};

/* ---------------------------------------------------------------- Philox */
/* Philox4x32-10 as published by Salmon et al. (SC'11): ten rounds of two
 * 32x32->64 multiplies with the bijection (c0,c1,c2,c3) ->
 * (hi1^c1^k0, lo1, hi0^c3^k1, lo0), key bumped by the Weyl constants. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in [0,1) from the top 53 bits of the 64-bit word hi:lo. */
double orc_u01(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

/* floor(w * m / 2^64): an index in [0, m) from the 64-bit word hi:lo. */
uint64_t orc_below(uint32_t lo, uint32_t hi, uint64_t m) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  unsigned __int128 p = (unsigned __int128)w * (unsigned __int128)m;
  return (uint64_t)(p >> 64);
}

static void draw(const orc_sys* s, uint64_t k, uint32_t d, uint32_t tag, uint32_t w[4]) {
  uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(k >> 32), d, tag};
  orc_philox(ctr, s->key, w);
}

/* ---------------------------------------------------------------- spline */
/* Cubic Hermite interpolation on a uniform grid with given (or central
 * finite-difference) knot derivatives. */
int orc_hermite_init(spline_t* sp, int n, double h, const double* y, const double* m) {
  sp->n = n;
  sp->h = h;
  sp->y = (double*)malloc(sizeof(double) * n);
  sp->m = (double*)malloc(sizeof(double) * n);
  if (!sp->y || !sp->m) return -1;
  memcpy(sp->y, y, sizeof(double) * n);
  if (m) {
    memcpy(sp->m, m, sizeof(double) * n);
  } else {
    for (int j = 0; j < n; ++j) {
      if (j == 0) sp->m[j] = (y[1] - y[0]) / h;
      else if (j == n - 1) sp->m[j] = (y[n - 1] - y[n - 2]) / h;
      else sp->m[j] = (y[j + 1] - y[j - 1]) / (2.0 * h);
    }
  }
  return 0;
}

int orc_hermite_eval(const spline_t* sp, double x, double* v, double* dv) {
  double xmax = (sp->n - 1) * sp->h;
  if (!(x >= 0.0) || x > xmax) return -1;
  int j = (int)floor(x / sp->h);
  if (j > sp->n - 2) j = sp->n - 2;
  double h = sp->h;
  double t = (x - j * h) / h;
  double y0 = sp->y[j], y1 = sp->y[j + 1];
  double m0 = sp->m[j] * h, m1 = sp->m[j + 1] * h;
  double t2 = t * t, t3 = t2 * t;
  double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t;
  double h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  if (v) *v = h00 * y0 + h10 * m0 + h01 * y1 + h11 * m1;
  if (dv) {
    double d00 = 6 * t2 - 6 * t, d10 = 3 * t2 - 4 * t + 1;
    double d01 = -6 * t2 + 6 * t, d11 = 3 * t2 - 2 * t;
    *dv = (d00 * y0 + d10 * m0 + d01 * y1 + d11 * m1) / h;
  }
  return 0;
}

int orc_spline(const orc_sys* s, int which, double x, double* v, double* dv) {
  if (which < 0 || which > 6) return -1;
  return orc_hermite_eval(&s->sp[which], x, v, dv);
}

/* table accessors: abort-free, out-of-range yields NaN so it shows up */
static double phi_ab(const orc_sys* s, int a, int b, double r) {
  double v;
  if (orc_hermite_eval(&s->sp[a + b], r, &v, NULL)) return NAN;
  return v;
}
static double dens_of(const orc_sys* s, int a, double r) {
  double v;
  if (orc_hermite_eval(&s->sp[3 + a], r, &v, NULL)) return NAN;
  return v;
}
static double embed_of(const orc_sys* s, int a, double rho) {
  double v;
  if (orc_hermite_eval(&s->sp[5 + a], rho, &v, NULL)) return NAN;
  return v;
}

/* --------------------------------------------------------- neighbour list */
static int cmp_nbr(const void* pa, const void* pb) {
  const nbr_t* a = (const nbr_t*)pa;
  const nbr_t* b = (const nbr_t*)pb;
  if (a->r != b->r) return a->r < b->r ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->sx != b->sx) return a->sx < b->sx ? -1 : 1;
  if (a->sy != b->sy) return a->sy < b->sy ? -1 : 1;
  if (a->sz != b->sz) return a->sz < b->sz ? -1 : 1;
  return 0;
}

typedef struct {
  nbr_t* v;
  int64_t n, cap;
} nbr_vec;

static int vec_push(nbr_vec* a, nbr_t e) {
  if (a->n == a->cap) {
    int64_t cap = a->cap ? 2 * a->cap : 1024;
    nbr_t* p = (nbr_t*)realloc(a->v, sizeof(nbr_t) * cap);
    if (!p) return -1;
    a->v = p;
    a->cap = cap;
  }
  a->v[a->n++] = e;
  return 0;
}

/* Brute force: every j and every periodic image shift within reach. */
static int build_brute(orc_sys* s, nbr_vec* all, int64_t* start) {
  int m[3];
  for (int a = 0; a < 3; ++a) m[a] = (int)ceil(s->rc / s->box[a]) + 1;
  double rc2 = s->rc * s->rc;
  for (int64_t i = 0; i < s->n; ++i) {
    start[i] = all->n;
    int64_t first = all->n;
    for (int64_t j = 0; j < s->n; ++j)
      for (int sx = -m[0]; sx <= m[0]; ++sx)
        for (int sy = -m[1]; sy <= m[1]; ++sy)
          for (int sz = -m[2]; sz <= m[2]; ++sz) {
            if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
            double dx = s->x[j] + sx * s->box[0] - s->x[i];
            double dy = s->y[j] + sy * s->box[1] - s->y[i];
            double dz = s->z[j] + sz * s->box[2] - s->z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2) {
              nbr_t e = {j, sqrt(r2), {dx, dy, dz}, sx, sy, sz};
              if (vec_push(all, e)) return -1;
            }
          }
    qsort(all->v + first, (size_t)(all->n - first), sizeof(nbr_t), cmp_nbr);
  }
  start[s->n] = all->n;
  return 0;
}

/* Cell binning (at least 3 cells of side >= rc per axis, so the minimum
 * image is the only image within rc). */
static int build_cells(orc_sys* s, nbr_vec* all, int64_t* start) {
  int nc[3];
  for (int a = 0; a < 3; ++a) nc[a] = (int)floor(s->box[a] / s->rc);
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * ncell);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * s->n);
  int* cell = (int*)malloc(sizeof(int) * 3 * s->n);
  if (!head || !next || !cell) { free(head); free(next); free(cell); return -1; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  const double* xs[3] = {s->x, s->y, s->z};
  for (int64_t i = s->n - 1; i >= 0; --i) {
    int c3[3];
    for (int a = 0; a < 3; ++a) {
      int c = (int)floor(xs[a][i] / s->box[a] * nc[a]);
      if (c < 0) c = 0;
      if (c >= nc[a]) c = nc[a] - 1;
      c3[a] = c;
      cell[3 * i + a] = c;
    }
    int64_t lin = ((int64_t)c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
    next[i] = head[lin];
    head[lin] = i;
  }
  double rc2 = s->rc * s->rc;
  for (int64_t i = 0; i < s->n; ++i) {
    start[i] = all->n;
    int64_t first = all->n;
    for (int ox = -1; ox <= 1; ++ox)
      for (int oy = -1; oy <= 1; ++oy)
        for (int oz = -1; oz <= 1; ++oz) {
          int cx = (cell[3 * i] + ox + nc[0]) % nc[0];
          int cy = (cell[3 * i + 1] + oy + nc[1]) % nc[1];
          int cz = (cell[3 * i + 2] + oz + nc[2]) % nc[2];
          int64_t lin = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
          for (int64_t j = head[lin]; j >= 0; j = next[j]) {
            if (j == i) continue;
            double d[3];
            int sh[3];
            for (int a = 0; a < 3; ++a) {
              double v = xs[a][j] - xs[a][i];
              int k = (int)lround(v / s->box[a]);
              d[a] = v - k * s->box[a];
              sh[a] = -k;
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rc2) {
              nbr_t e = {j, sqrt(r2), {d[0], d[1], d[2]}, sh[0], sh[1], sh[2]};
              if (vec_push(all, e)) { free(head); free(next); free(cell); return -1; }
            }
          }
        }
    qsort(all->v + first, (size_t)(all->n - first), sizeof(nbr_t), cmp_nbr);
  }
  start[s->n] = all->n;
  free(head);
  free(next);
  free(cell);
  return 0;
}

static int build_neighbours(orc_sys* s) {
  nbr_vec all = {NULL, 0, 0};
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (s->n + 1));
  if (!start) return -1;
  int use_cells = !s->brute;
  for (int a = 0; a < 3; ++a)
    if (floor(s->box[a] / s->rc) < 3) use_cells = 0;
  int rc = use_cells ? build_cells(s, &all, start) : build_brute(s, &all, start);
  if (rc) { free(all.v); free(start); return -1; }
  free(s->nstart);
  free(s->nb);
  s->nstart = start;
  s->nb = all.v;
  return 0;
}

static void compute_rho(orc_sys* s) {
  for (int64_t i = 0; i < s->n; ++i) {
    double r = 0.0;
    for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k)
      r += dens_of(s, s->t[s->nb[k].j], s->nb[k].r);
    s->rho[i] = r;
  }
}

/* ---------------------------------------------------------------- energy */
/* Neumaier-compensated running sum. */
typedef struct { double s, c; } ksum;
static void kadd(ksum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

/* U = sum_i [ 1/2 sum_j phi_{t_i t_j}(r_ij) + F_{t_i}(rho_i) ]  (EAM). */
double orc_energy_full(const orc_sys* s) {
  ksum acc = {0, 0};
  for (int64_t i = 0; i < s->n; ++i) {
    int ti = s->t[i];
    double rho = 0.0;
    for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k) {
      const nbr_t* e = &s->nb[k];
      kadd(&acc, 0.5 * phi_ab(s, ti, s->t[e->j], e->r));
      rho += dens_of(s, s->t[e->j], e->r);
    }
    kadd(&acc, embed_of(s, ti, rho));
  }
  return acc.s + acc.c;
}

/* Energy change for flipping site i from t to t' = 1 - t:
 *   pair:     sum_k [phi_{t' t_k}(r_ik) - phi_{t t_k}(r_ik)]
 *   own:      F_{t'}(rho_i) - F_t(rho_i)   (rho_i does not depend on t_i)
 *   re-embed: sum over distinct neighbours k of
 *             F_{t_k}(rho_k + drho_k) - F_{t_k}(rho_k),
 *             drho_k = sum over the slots of k of f_{t'}(r) - f_t(r). */
double orc_delta_e(const orc_sys* s, int64_t i) {
  int t = s->t[i], tp = 1 - t;
  int64_t b = s->nstart[i], e = s->nstart[i + 1];
  double pair = 0.0;
  int any_drho = 0;
  for (int64_t k = b; k < e; ++k) {
    const nbr_t* nb = &s->nb[k];
    int tk = s->t[nb->j];
    pair += phi_ab(s, tp, tk, nb->r) - phi_ab(s, t, tk, nb->r);
    if (dens_of(s, tp, nb->r) - dens_of(s, t, nb->r) != 0.0) any_drho = 1;
  }
  double own = embed_of(s, tp, s->rho[i]) - embed_of(s, t, s->rho[i]);
  double reembed = 0.0;
  if (any_drho) {
    for (int64_t k = b; k < e; ++k) {
      int64_t j = s->nb[k].j;
      int seen = 0;
      for (int64_t q = b; q < k; ++q)
        if (s->nb[q].j == j) { seen = 1; break; }
      if (seen) continue;
      double drho = 0.0;
      for (int64_t q = k; q < e; ++q)
        if (s->nb[q].j == j) drho += dens_of(s, tp, s->nb[q].r) - dens_of(s, t, s->nb[q].r);
      int tj = s->t[j];
      reembed += embed_of(s, tj, s->rho[j] + drho) - embed_of(s, tj, s->rho[j]);
    }
  }
  return pair + own + reembed;
}

void orc_flip(orc_sys* s, int64_t i) {
  int t = s->t[i], tp = 1 - t;
  for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k) {
    const nbr_t* nb = &s->nb[k];
    s->rho[nb->j] += dens_of(s, tp, nb->r) - dens_of(s, t, nb->r);
  }
  s->t[i] = (uint8_t)tp;
  s->nb_count += tp ? 1 : -1;
}

double orc_delta_e_full(orc_sys* s, int64_t i) {
  double e0 = orc_energy_full(s);
  uint8_t t = s->t[i];
  s->t[i] = 1 - t;
  double e1 = orc_energy_full(s);
  s->t[i] = t;
  return e1 - e0;
}

/* ---------------------------------------------------------------- create */
orc_sys* orc_create(int64_t n, const double* x, const double* y, const double* z,
                    const double box[3], const uint8_t* types, const orc_eam_in* eam,
                    int brute) {
  if (n <= 0 || !eam || eam->nr < 2 || eam->nrho < 2) return NULL;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > eam->rc)) return NULL; /* no self-images within rc */
  orc_sys* s = (orc_sys*)calloc(1, sizeof(orc_sys));
  if (!s) return NULL;
  s->n = n;
  memcpy(s->box, box, sizeof(double) * 3);
  s->x = (double*)malloc(sizeof(double) * n);
  s->y = (double*)malloc(sizeof(double) * n);
  s->z = (double*)malloc(sizeof(double) * n);
  s->t = (uint8_t*)malloc(n);
  s->rho = (double*)malloc(sizeof(double) * n);
  if (!s->x || !s->y || !s->z || !s->t || !s->rho) { orc_free(s); return NULL; }
  /* positions are periodic: keep them in [0, L) */
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
  s->brute = brute;
  for (int p = 0; p < 3; ++p)
    if (orc_hermite_init(&s->sp[p], eam->nr, eam->dr, eam->pair[p], eam->dpair[p])) { orc_free(s); return NULL; }
  for (int a = 0; a < 2; ++a) {
    if (orc_hermite_init(&s->sp[3 + a], eam->nr, eam->dr, eam->dens[a], eam->ddens[a])) { orc_free(s); return NULL; }
    if (orc_hermite_init(&s->sp[5 + a], eam->nrho, eam->drho, eam->embed[a], eam->dembed[a])) { orc_free(s); return NULL; }
  }
  if (build_neighbours(s)) { orc_free(s); return NULL; }
  compute_rho(s);
  s->nb_count = 0;
  for (int64_t i = 0; i < n; ++i) s->nb_count += s->t[i];
  s->energy = orc_energy_full(s);
  return s;
}

void orc_free(orc_sys* s) {
  if (!s) return;
  free(s->x); free(s->y); free(s->z); free(s->t); free(s->rho);
  for (int p = 0; p < 7; ++p) { free(s->sp[p].y); free(s->sp[p].m); }
  free(s->nstart); free(s->nb);
  free(s->col_start); free(s->dom_start); free(s->dom_sites); free(s->dom_wt);
  free(s->site_trials);
  free(s->vx); free(s->vy); free(s->vz); free(s->fx); free(s->fy); free(s->fz);
  free(s->mlp);
  free(s);
}

int orc_set_params(orc_sys* s, double phi, double kappa, double T, int kappa_units,
                   double c0, uint64_t seed) {
  if (!(T > 0) || !(kappa >= 0)) return -1;
  s->phi = phi;
  s->kappa = kappa;
  s->T = T;
  s->beta = 1.0 / (KB_EV * T);
  s->kappa_p = kappa_units == 1 ? kappa : kappa * KB_EV * T / (double)s->n;
  s->c0 = c0 < 0 ? (double)s->nb_count / (double)s->n : c0;
  s->n0 = (double)s->n * s->c0;
  /* Delta mu_0 = phi + 2 kappa N c0 (Eq. trans_vcsgc_par1) */
  s->dmu0 = phi + 2.0 * s->kappa_p * s->n0;
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->step = 0;
  orc_reset_counters(s);
  return 0;
}

void orc_reset_counters(orc_sys* s) {
  s->trials = s->local_acc = s->global_acc = s->global_trials = 0;
  s->flips = s->near_ties = 0;
  s->s1_accepts = 0;
  s->sum_c = s->sum_c2 = 0.0;
  s->steps_done = 0;
}

/* -------------------------------------------------------------- schedule */
static int sched_alloc(orc_sys* s, int64_t n_colours, int64_t n_domains) {
  free(s->col_start); free(s->dom_start); free(s->dom_sites); free(s->dom_wt);
  s->dom_wt = NULL;
  s->col_start = (int64_t*)calloc(n_colours + 1, sizeof(int64_t));
  s->dom_start = (int64_t*)calloc(n_domains + 1, sizeof(int64_t));
  s->dom_sites = (int64_t*)calloc(s->n, sizeof(int64_t));
  s->n_colours = n_colours;
  s->n_domains = n_domains;
  return (s->col_start && s->dom_start && s->dom_sites) ? 0 : -1;
}

int orc_schedule_blocks(orc_sys* s, int nx, int ny, int nz, int bx, int by, int bz,
                        int px, int py, int pz) {
  if ((int64_t)2 * nx * ny * nz != s->n) return -1;
  if (bx < 1 || by < 1 || bz < 1 || px < 1 || py < 1 || pz < 1) return -1;
  if (nx % bx || ny % by || nz % bz) return -1;
  int nbx = nx / bx, nby = ny / by, nbz = nz / bz;
  if (nbx % px || nby % py || nbz % pz) return -1;
  int64_t ncol = (int64_t)px * py * pz, nblk = (int64_t)nbx * nby * nbz;
  if (sched_alloc(s, ncol, nblk)) return -1;
  int64_t dom = 0, site = 0;
  for (int64_t c = 0; c < ncol; ++c) {
    s->col_start[c] = dom;
    for (int ibz = 0; ibz < nbz; ++ibz)
      for (int iby = 0; iby < nby; ++iby)
        for (int ibx = 0; ibx < nbx; ++ibx) {
          int64_t col = ((int64_t)(ibz % pz) * py + (iby % py)) * px + (ibx % px);
          if (col != c) continue;
          s->dom_start[dom] = site;
          for (int lz = 0; lz < bz; ++lz)
            for (int ly = 0; ly < by; ++ly)
              for (int lx = 0; lx < bx; ++lx)
                for (int b = 0; b < 2; ++b) {
                  int64_t cx = (int64_t)ibx * bx + lx, cy = (int64_t)iby * by + ly,
                          cz = (int64_t)ibz * bz + lz;
                  s->dom_sites[site++] = ((cz * ny + cy) * nx + cx) * 2 + b;
                }
          ++dom;
        }
  }
  s->col_start[ncol] = dom;
  s->dom_start[dom] = site;
  s->sched_kind = 1;
  return 0;
}

int orc_schedule_sublattice(orc_sys* s, int nx, int ny, int nz, int qx, int qy, int qz) {
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
      int64_t col = (((cz % qz) * qy + (cy % qy)) * qx + (cx % qx)) * 2 + b;
      if (col != c) continue;
      s->dom_start[dom] = dom;
      s->dom_sites[dom] = i;
      ++dom;
    }
  }
  s->col_start[ncol] = dom;
  s->dom_start[dom] = dom;
  s->sched_kind = 2;
  return 0;
}

int orc_schedule_spatial(orc_sys* s, int nbx, int nby, int nbz, int px, int py, int pz) {
  if (nbx < 1 || nby < 1 || nbz < 1 || px < 1 || py < 1 || pz < 1) return -1;
  if (nbx % px || nby % py || nbz % pz) return -1;
  int64_t ncol = (int64_t)px * py * pz, nblk = (int64_t)nbx * nby * nbz;
  int64_t* blk = (int64_t*)malloc(sizeof(int64_t) * s->n);
  if (!blk) return -1;
  int nb3[3] = {nbx, nby, nbz};
  const double* xs[3] = {s->x, s->y, s->z};
  for (int64_t i = 0; i < s->n; ++i) {
    int c3[3];
    for (int a = 0; a < 3; ++a) {
      int c = (int)floor(xs[a][i] / s->box[a] * nb3[a]);
      if (c < 0) c = 0;
      if (c >= nb3[a]) c = nb3[a] - 1;
      c3[a] = c;
    }
    blk[i] = ((int64_t)c3[2] * nby + c3[1]) * nbx + c3[0];
  }
  if (sched_alloc(s, ncol, nblk)) { free(blk); return -1; }
  int64_t dom = 0, site = 0;
  for (int64_t c = 0; c < ncol; ++c) {
    s->col_start[c] = dom;
    for (int64_t b = 0; b < nblk; ++b) {
      int64_t ibx = b % nbx, iby = (b / nbx) % nby, ibz = b / ((int64_t)nbx * nby);
      int64_t col = ((ibz % pz) * py + (iby % py)) * px + (ibx % px);
      if (col != c) continue;
      s->dom_start[dom] = site;
      for (int64_t i = 0; i < s->n; ++i)
        if (blk[i] == b) s->dom_sites[site++] = i;
      ++dom;
    }
  }
  s->col_start[ncol] = dom;
  s->dom_start[dom] = site;
  free(blk);
  s->sched_kind = 3;
  s->sched_args[0] = nbx; s->sched_args[1] = nby; s->sched_args[2] = nbz;
  s->sched_args[3] = px; s->sched_args[4] = py; s->sched_args[5] = pz;
  return 0;
}

/* Overlapping, position-weighted domains (Sec. III A, the optimal
 * decomposition): the lattice is cut into cells of lx*ly*lz lattice cells;
 * along each axis a domain covers either the first l - g or the last l - g
 * lattice cells of its cell, so the eight domains of a cell (colour bits
 * bx, by, bz) overlap in the middle and domains of one colour in
 * neighbouring cells are g lattice cells apart.  A site covered by m_x m_y
 * m_z domains (m = 1 or 2 per axis) has the pick weight 8 / (m_x m_y m_z):
 * with the domain's site drawn in proportion to weight, every site is picked
 * with probability 1 / (2 lx ly lz) per step.  Within a domain the sites are
 * listed by decreasing weight, ascending index within one weight. */
int orc_schedule_overlap(orc_sys* s, int nx, int ny, int nz, int lx, int ly, int lz,
                         int gx, int gy, int gz) {
  if ((int64_t)2 * nx * ny * nz != s->n) return -1;
  int n3[3] = {nx, ny, nz}, l3[3] = {lx, ly, lz}, g3[3] = {gx, gy, gz}, nc[3], ld[3];
  for (int q = 0; q < 3; ++q) {
    if (l3[q] < 1 || g3[q] < 0 || n3[q] % l3[q] || 2 * g3[q] > l3[q]) return -1;
    nc[q] = n3[q] / l3[q];
    ld[q] = l3[q] - g3[q];
  }
  int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t per_dom = (int64_t)2 * ld[0] * ld[1] * ld[2];
  if (sched_alloc(s, 8, 8 * ncells)) return -1;
  free(s->dom_sites);
  s->dom_sites = (int64_t*)calloc(8 * ncells * per_dom, sizeof(int64_t));
  s->dom_wt = (int64_t*)calloc(8 * ncells * per_dom, sizeof(int64_t));
  int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * per_dom);
  int64_t* tw = (int64_t*)malloc(sizeof(int64_t) * per_dom);
  if (!s->dom_sites || !s->dom_wt || !tmp || !tw) { free(tmp); free(tw); return -1; }
  int64_t dom = 0, pos = 0;
  for (int c = 0; c < 8; ++c) {
    int bit[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    s->col_start[c] = dom;
    for (int icz = 0; icz < nc[2]; ++icz)
      for (int icy = 0; icy < nc[1]; ++icy)
        for (int icx = 0; icx < nc[0]; ++icx) {
          int ic[3] = {icx, icy, icz};
          int64_t k = 0;
          for (int tz = 0; tz < ld[2]; ++tz)
            for (int ty = 0; ty < ld[1]; ++ty)
              for (int tx = 0; tx < ld[0]; ++tx) {
                int t3[3] = {tx, ty, tz}, X[3];
                int cover = 1;
                for (int q = 0; q < 3; ++q) {
                  int local = bit[q] * g3[q] + t3[q]; /* position inside the cell */
                  int m = 0;
                  for (int b = 0; b < 2; ++b)
                    if (local >= b * g3[q] && local < b * g3[q] + ld[q]) ++m;
                  cover *= m;
                  X[q] = ic[q] * l3[q] + local;
                }
                for (int b = 0; b < 2; ++b) {
                  tmp[k] = (((int64_t)X[2] * ny + X[1]) * nx + X[0]) * 2 + b;
                  tw[k] = 8 / cover;
                  ++k;
                }
              }
          s->dom_start[dom] = pos;
          for (int64_t w = 8; w >= 1; w /= 2)
            for (int64_t q = 0; q < per_dom; ++q)
              if (tw[q] == w) {
                s->dom_sites[pos] = tmp[q];
                s->dom_wt[pos] = w;
                ++pos;
              }
          ++dom;
        }
  }
  s->col_start[8] = dom;
  s->dom_start[dom] = pos;
  free(tmp);
  free(tw);
  s->sched_kind = 4;
  return 0;
}

int orc_schedule_weights(const orc_sys* s, int64_t* wt) {
  if (!s->dom_wt) return 0;
  if (wt) memcpy(wt, s->dom_wt, sizeof(int64_t) * s->dom_start[s->n_domains]);
  return 1;
}

int orc_track_trials(orc_sys* s, int on) {
  free(s->site_trials);
  s->site_trials = on ? (int64_t*)calloc(s->n, sizeof(int64_t)) : NULL;
  return on && !s->site_trials ? -1 : 0;
}

void orc_trial_counts(const orc_sys* s, int64_t* out) {
  for (int64_t i = 0; i < s->n; ++i) out[i] = s->site_trials ? s->site_trials[i] : 0;
}

int64_t orc_schedule_info(const orc_sys* s, int64_t* n_colours, int64_t* domains_per_colour) {
  if (n_colours) *n_colours = s->n_colours;
  if (domains_per_colour) *domains_per_colour = s->n_colours ? s->col_start[1] - s->col_start[0] : 0;
  return s->n_domains;
}

void orc_schedule_export(const orc_sys* s, int64_t* col_start, int64_t* dom_start,
                         int64_t* dom_sites) {
  if (col_start) memcpy(col_start, s->col_start, sizeof(int64_t) * (s->n_colours + 1));
  if (dom_start) memcpy(dom_start, s->dom_start, sizeof(int64_t) * (s->n_domains + 1));
  if (dom_sites) memcpy(dom_sites, s->dom_sites, sizeof(int64_t) * s->dom_start[s->n_domains]);
}

static double min_image_dist(const orc_sys* s, int64_t i, int64_t j) {
  double best = INFINITY;
  for (int sx = -1; sx <= 1; ++sx)
    for (int sy = -1; sy <= 1; ++sy)
      for (int sz = -1; sz <= 1; ++sz) {
        double dx = s->x[j] + sx * s->box[0] - s->x[i];
        double dy = s->y[j] + sy * s->box[1] - s->y[i];
        double dz = s->z[j] + sz * s->box[2] - s->z[i];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r < best) best = r;
      }
  return best;
}

double orc_schedule_min_separation(const orc_sys* s) {
  double best = INFINITY;
  for (int64_t c = 0; c < s->n_colours; ++c)
    for (int64_t d1 = s->col_start[c]; d1 < s->col_start[c + 1]; ++d1)
      for (int64_t d2 = d1 + 1; d2 < s->col_start[c + 1]; ++d2)
        for (int64_t a = s->dom_start[d1]; a < s->dom_start[d1 + 1]; ++a)
          for (int64_t b = s->dom_start[d2]; b < s->dom_start[d2 + 1]; ++b) {
            double r = min_image_dist(s, s->dom_sites[a], s->dom_sites[b]);
            if (r < best) best = r;
          }
  return best;
}

/* ------------------------------------------------- surrogate (stage 1) */
/* The delayed-acceptance form replaces the local Metropolis factor by two
 * stages (Christen and Fox, J. Comput. Graph. Stat. 14, 795 (2005)): a cheap
 * prediction g_i of E(sigma with i = B) - E(sigma with i = A) is tested
 * first, and only a move that passes is tested again with the exact energy
 * change.  g_i is a function of the environment of i alone (every site but
 * i), so the predicted change of the reverse move is exactly -s g_i and the
 * product of the two stages keeps the ratio exp(-X) of the plain local rule.
 *
 * Environment descriptor of site i (ten counts, shells identified by their
 * radii):
 *   own[s] = number of B sites j != i in shell s of i;
 *   nb[s]  = sum over the first-shell neighbours k of i of the number of B
 *            sites j != i in shell s of k.
 * MLP: x_c = count_c / max_c (max_c = the count when every site is B on the
 * BCC lattice), z1 = W1 x + b1, h1 = SiLU(z1), z2 = W2 h1 + b2,
 * h2 = SiLU(z2), g = w3 . h2 + b3, SiLU(z) = z / (1 + exp(-z)). */
static const double k_desc_max[ORC_MLP_IN] = {8, 6, 12, 24, 8, 56, 48, 96, 192, 64};

int orc_set_shells(orc_sys* s, int n_shells, const double* radii, double tol) {
  if (n_shells < 1 || n_shells > ORC_MAX_SHELLS || !(tol > 0)) return -1;
  s->n_shells = n_shells;
  for (int q = 0; q < n_shells; ++q) s->shell_r[q] = radii[q];
  s->shell_tol = tol;
  return 0;
}

static int shell_of(const orc_sys* s, double r) {
  for (int q = 0; q < s->n_shells; ++q)
    if (fabs(r - s->shell_r[q]) <= s->shell_tol) return q;
  return -1;
}

int orc_descriptor(const orc_sys* s, int64_t i, double out[ORC_MLP_IN]) {
  if (s->n_shells != ORC_MLP_IN / 2) return -1;
  for (int q = 0; q < ORC_MLP_IN; ++q) out[q] = 0.0;
  for (int64_t a = s->nstart[i]; a < s->nstart[i + 1]; ++a) {
    const int64_t j = s->nb[a].j;
    const int q = shell_of(s, s->nb[a].r);
    if (j == i || q < 0) continue;
    out[q] += s->t[j];
    if (q != 0) continue;
    /* j is a first-shell neighbour k of i: add its shell counts */
    for (int64_t b = s->nstart[j]; b < s->nstart[j + 1]; ++b) {
      const int64_t j2 = s->nb[b].j;
      const int q2 = shell_of(s, s->nb[b].r);
      if (j2 == i || q2 < 0) continue;
      out[ORC_MLP_IN / 2 + q2] += s->t[j2];
    }
  }
  return 0;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }

double orc_mlp_eval(const double* p, const double x[ORC_MLP_IN]) {
  const double* W1 = p;
  const double* b1 = W1 + ORC_MLP_H * ORC_MLP_IN;
  const double* W2 = b1 + ORC_MLP_H;
  const double* b2 = W2 + ORC_MLP_H * ORC_MLP_H;
  const double* w3 = b2 + ORC_MLP_H;
  const double b3 = w3[ORC_MLP_H];
  double h1[ORC_MLP_H], h2[ORC_MLP_H];
  for (int o = 0; o < ORC_MLP_H; ++o) {
    double z = b1[o];
    for (int c = 0; c < ORC_MLP_IN; ++c) z += W1[o * ORC_MLP_IN + c] * (x[c] / k_desc_max[c]);
    h1[o] = silu(z);
  }
  for (int o = 0; o < ORC_MLP_H; ++o) {
    double z = b2[o];
    for (int c = 0; c < ORC_MLP_H; ++c) z += W2[o * ORC_MLP_H + c] * h1[c];
    h2[o] = silu(z);
  }
  double y = b3;
  for (int o = 0; o < ORC_MLP_H; ++o) y += w3[o] * h2[o];
  return y;
}

int orc_set_surrogate(orc_sys* s, int kind, const double* params) {
  if (kind < 0 || kind > 2) return -1;
  if (kind == 1) {
    if (!params || s->n_shells != ORC_MLP_IN / 2) return -1;
    if (!s->mlp) s->mlp = (double*)malloc(sizeof(double) * ORC_MLP_NPARAM);
    if (!s->mlp) return -1;
    memcpy(s->mlp, params, sizeof(double) * ORC_MLP_NPARAM);
  }
  s->sur_kind = kind;
  return 0;
}

double orc_surrogate(const orc_sys* s, int64_t i) {
  if (s->sur_kind == 2) {
    const double de = orc_delta_e(s, i);
    return s->t[i] == 0 ? de : -de;
  }
  double x[ORC_MLP_IN];
  orc_descriptor(s, i, x);
  return orc_mlp_eval(s->mlp, x);
}

/* ------------------------------------------------------------- sampling */
/* Metropolis decision u < min{1, exp(-X)}; counts decisions within 1e-9
 * (relative) of the boundary, where CPU and GPU exp may round differently. */
static int metropolis(orc_sys* s, double X, double u) {
  if (X <= 0.0) {
    if (X > -1e-9 && u >= 1.0 - 1e-9) s->near_ties++;
    return 1;
  }
  double p = exp(-X);
  if (fabs(u - p) <= 1e-9 * p) s->near_ties++;
  return u < p;
}

/* Local decision of trial site i with sign s_i = sg, drawn with u (stage 1
 * or the plain rule) and, for delayed acceptance, u2 (stage 2).  Returns the
 * decision; *de gets the exact energy change when it was evaluated.
 *   plain:   u  < min{1, exp(-beta (dE + s dmu0))}                 (Eq. trans_vcsgc_par1)
 *   stage 1: u  < min{1, exp(-beta (s g + s dmu0))}
 *   stage 2: u2 < min{1, exp(-beta (dE - s g))}                    */
static int local_decision(orc_sys* s, int64_t site, int sg, double u, double u2, double* de) {
  if (!s->sur_kind) {
    *de = orc_delta_e(s, site);
    return metropolis(s, s->beta * (*de + sg * s->dmu0), u);
  }
  const double g = orc_surrogate(s, site);
  if (!metropolis(s, s->beta * (sg * g + sg * s->dmu0), u)) return 0;
  s->s1_accepts++;
  *de = orc_delta_e(s, site);
  return metropolis(s, s->beta * (*de - sg * g), u2);
}

static void sample_c(orc_sys* s) {
  double c = (double)s->nb_count / (double)s->n;
  s->sum_c += c;
  s->sum_c2 += c * c;
  s->steps_done++;
}

static void flip_commit(orc_sys* s, int64_t i) {
  if (s->vx) {
    /* keep the Maxwell distribution: v scaled by sqrt(m_old / m_new) */
    double f = sqrt(s->mass[s->t[i]] / s->mass[1 - s->t[i]]);
    s->vx[i] *= f; s->vy[i] *= f; s->vz[i] *= f;
  }
  orc_flip(s, i);
}

/* One composite step of the parallel algorithm (Sec. III B 2):
 *  1. colour c drawn from the step's synchronised stream;
 *  2. every domain d of colour c picks one of its sites uniformly and
 *     proposes t -> 1 - t; the local stage accepts it with
 *     min{1, exp[-beta (dE_i + s_i dmu0)]}, s_i = N dc_i = +-1;
 *  3. dn = sum of s_i over the locally accepted moves;
 *  4. the global stage accepts the whole composite move with
 *     min{1, exp[-beta kappa_p dn (dn + 2 (n - n0))]};
 *  5. if accepted every locally accepted site flips. */
static void parallel_step(orc_sys* s, int64_t* acc_sites, double* acc_de) {
  uint64_t k = s->step;
  uint32_t w[4];
  draw(s, k, 0xFFFFFFFFu, 1u, w);
  int64_t c = (int64_t)orc_below(w[0], w[1], (uint64_t)s->n_colours);
  double ug = orc_u01(w[2], w[3]);
  int64_t d0 = s->col_start[c], d1 = s->col_start[c + 1];
  int64_t nacc = 0, dn = 0;
  for (int64_t g = d0; g < d1; ++g) {
    int64_t size = s->dom_start[g + 1] - s->dom_start[g];
    if (size == 0) continue;
    draw(s, k, (uint32_t)(g - d0), 0u, w);
    int64_t site;
    if (s->dom_wt) {
      /* weighted pick: r uniform on [0, total weight), the first site whose
       * running weight exceeds r */
      int64_t total = 0;
      for (int64_t q = s->dom_start[g]; q < s->dom_start[g + 1]; ++q) total += s->dom_wt[q];
      int64_t r = (int64_t)orc_below(w[0], w[1], (uint64_t)total), run = 0, q = s->dom_start[g];
      for (;; ++q) {
        run += s->dom_wt[q];
        if (r < run) break;
      }
      site = s->dom_sites[q];
    } else {
      site = s->dom_sites[s->dom_start[g] + orc_below(w[0], w[1], (uint64_t)size)];
    }
    if (s->site_trials) s->site_trials[site]++;
    double u = orc_u01(w[2], w[3]), u2 = 0.0;
    if (s->sur_kind) {
      uint32_t w2[4];
      draw(s, k, (uint32_t)(g - d0), 5u, w2);
      u2 = orc_u01(w2[0], w2[1]);
    }
    int sg = s->t[site] == 0 ? 1 : -1;
    double de = 0.0;
    s->trials++;
    if (local_decision(s, site, sg, u, u2, &de)) {
      acc_sites[nacc] = site;
      acc_de[nacc] = de;
      nacc++;
      dn += sg;
    }
  }
  s->local_acc += nacc;
  if (nacc > 0) {
    s->global_trials++;
    double Y = s->beta * s->kappa_p * (double)dn * ((double)dn + 2.0 * ((double)s->nb_count - s->n0));
    if (metropolis(s, Y, ug)) {
      s->global_acc++;
      for (int64_t a = 0; a < nacc; ++a) {
        flip_commit(s, acc_sites[a]);
        s->energy += acc_de[a];
      }
      s->flips += nacc;
    }
  }
  s->step++;
  sample_c(s);
}

int orc_parallel_steps(orc_sys* s, int64_t n_steps) {
  if (!s->n_colours) return -1;
  int64_t maxd = 0;
  for (int64_t c = 0; c < s->n_colours; ++c) {
    int64_t d = s->col_start[c + 1] - s->col_start[c];
    if (d > maxd) maxd = d;
  }
  int64_t* sites = (int64_t*)malloc(sizeof(int64_t) * (maxd + 1));
  double* des = (double*)malloc(sizeof(double) * (maxd + 1));
  if (!sites || !des) { free(sites); free(des); return -1; }
  for (int64_t k = 0; k < n_steps; ++k) parallel_step(s, sites, des);
  free(sites);
  free(des);
  return 0;
}

/* Serial single-site steps.
 * mode 0, Eq. trans_vcsgc: X = beta (dE + N dc (phi + 2 kappa_p N c~)),
 *         with N dc = s and 2 N c~ = n + n' = 2n + s.
 * mode 1, Eq. mod: local factor with dmu0 times global factor with
 *         exponent beta kappa_p s (s + 2 (n - n0)).
 * mode 2: mode 1 with the local factor taken in the two delayed-acceptance
 *         stages of the surrogate (orc_set_surrogate). */
int orc_serial_steps(orc_sys* s, int64_t n_steps, int mode) {
  if (mode == 2 && !s->sur_kind) return -1;
  for (int64_t q = 0; q < n_steps; ++q) {
    uint64_t k = s->step;
    uint32_t w[4], w2[4];
    draw(s, k, 0u, 2u, w);
    int64_t site = (int64_t)orc_below(w[0], w[1], (uint64_t)s->n);
    double u = orc_u01(w[2], w[3]);
    int sg = s->t[site] == 0 ? 1 : -1;
    double n = (double)s->nb_count;
    double de = 0.0;
    int acc;
    s->trials++;
    if (mode == 0) {
      de = orc_delta_e(s, site);
      double X = s->beta * (de + sg * (s->phi + s->kappa_p * (2.0 * n + sg)));
      acc = metropolis(s, X, u);
      if (acc) s->local_acc++;
    } else {
      double u2 = 0.0;
      if (mode == 2) {
        draw(s, k, 2u, 2u, w2);
        u2 = orc_u01(w2[0], w2[1]);
      }
      const int kind = s->sur_kind;
      if (mode == 1) s->sur_kind = 0;
      acc = local_decision(s, site, sg, u, u2, &de);
      s->sur_kind = kind;
      if (acc) {
        s->local_acc++;
        s->global_trials++;
        draw(s, k, 1u, 2u, w2);
        double ug = orc_u01(w2[0], w2[1]);
        double Y = s->beta * s->kappa_p * (double)sg * ((double)sg + 2.0 * (n - s->n0));
        acc = metropolis(s, Y, ug);
        if (acc) s->global_acc++;
      }
    }
    if (acc) {
      flip_commit(s, site);
      s->energy += de;
      s->flips++;
    }
    s->step++;
    sample_c(s);
  }
  return 0;
}

int orc_run_histogram(orc_sys* s, int64_t n_steps, int mode, int64_t* hist, double* sum_e) {
  for (int64_t q = 0; q < n_steps; ++q) {
    int rc = mode < 0 ? orc_parallel_steps(s, 1) : orc_serial_steps(s, 1, mode);
    if (rc) return rc;
    hist[s->nb_count]++;
    *sum_e += s->energy;
  }
  return 0;
}

/* ------------------------------------------------------------- accessors */
void orc_get_types(const orc_sys* s, uint8_t* out) { memcpy(out, s->t, s->n); }

void orc_set_types(orc_sys* s, const uint8_t* in) {
  memcpy(s->t, in, s->n);
  s->nb_count = 0;
  for (int64_t i = 0; i < s->n; ++i) s->nb_count += s->t[i];
  compute_rho(s);
  s->energy = orc_energy_full(s);
}

void orc_get_rho(const orc_sys* s, double* out) { memcpy(out, s->rho, sizeof(double) * s->n); }

void orc_get_obs(const orc_sys* s, orc_obs* o) {
  o->n_sites = s->n;
  o->n_b = s->nb_count;
  o->energy = s->energy;
  o->steps = s->steps_done;
  o->trials = s->trials;
  o->local_accepts = s->local_acc;
  o->global_trials = s->global_trials;
  o->global_accepts = s->global_acc;
  o->flips = s->flips;
  o->near_ties = s->near_ties;
  o->sum_c = s->sum_c;
  o->sum_c2 = s->sum_c2;
  o->stage1_accepts = s->s1_accepts;
}

int64_t orc_neighbour_count(const orc_sys* s, int64_t i) { return s->nstart[i + 1] - s->nstart[i]; }

void orc_neighbour(const orc_sys* s, int64_t i, int64_t k, int64_t* j, double* r, double d[3]) {
  const nbr_t* e = &s->nb[s->nstart[i] + k];
  if (j) *j = e->j;
  if (r) *r = e->r;
  if (d) { d[0] = e->d[0]; d[1] = e->d[1]; d[2] = e->d[2]; }
}

/* -------------------------------------------------------------------- MD */
/* F_i = sum_j [phi'_{t_i t_j}(r) + F'_{t_i}(rho_i) f'_{t_j}(r)
 *              + F'_{t_j}(rho_j) f'_{t_i}(r)] (x_j - x_i) / r */
void orc_forces(orc_sys* s, double* fx, double* fy, double* fz) {
  double* dF = (double*)malloc(sizeof(double) * s->n);
  for (int64_t i = 0; i < s->n; ++i) {
    double v;
    orc_hermite_eval(&s->sp[5 + s->t[i]], s->rho[i], NULL, &v);
    dF[i] = v;
  }
  /* the pair (i, j) pulls i along d_ij = r_j - r_i with g = dU/dr_ij; its
   * virial term r_ij . F_ij = -g r, each pair seen from both ends */
  double vir = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    int ti = s->t[i];
    double f[3] = {0, 0, 0};
    for (int64_t k = s->nstart[i]; k < s->nstart[i + 1]; ++k) {
      const nbr_t* e = &s->nb[k];
      int tj = s->t[e->j];
      double dphi, dfj, dfi;
      orc_hermite_eval(&s->sp[ti + tj], e->r, NULL, &dphi);
      orc_hermite_eval(&s->sp[3 + tj], e->r, NULL, &dfj);
      orc_hermite_eval(&s->sp[3 + ti], e->r, NULL, &dfi);
      double g = dphi + dF[i] * dfj + dF[e->j] * dfi;
      for (int a = 0; a < 3; ++a) f[a] += g * e->d[a] / e->r;
      vir -= 0.5 * g * e->r;
    }
    fx[i] = f[0]; fy[i] = f[1]; fz[i] = f[2];
  }
  s->virial = vir;
  free(dF);
}

void orc_set_md(orc_sys* s, const double* vx, const double* vy, const double* vz,
                double mass_a, double mass_b, double dt, double gamma, double T_md,
                uint64_t seed) {
  if (!s->vx) {
    s->vx = (double*)malloc(sizeof(double) * s->n);
    s->vy = (double*)malloc(sizeof(double) * s->n);
    s->vz = (double*)malloc(sizeof(double) * s->n);
    s->fx = (double*)malloc(sizeof(double) * s->n);
    s->fy = (double*)malloc(sizeof(double) * s->n);
    s->fz = (double*)malloc(sizeof(double) * s->n);
  }
  memcpy(s->vx, vx, sizeof(double) * s->n);
  memcpy(s->vy, vy, sizeof(double) * s->n);
  memcpy(s->vz, vz, sizeof(double) * s->n);
  s->mass[0] = mass_a;
  s->mass[1] = mass_b;
  s->dt = dt;
  s->gamma = gamma;
  s->T_md = T_md;
  s->md_key[0] = (uint32_t)seed;
  s->md_key[1] = (uint32_t)(seed >> 32);
  s->md_step = 0;
  orc_forces(s, s->fx, s->fy, s->fz);
}

static double wrap(double x, double L) {
  double y = x - floor(x / L) * L;
  if (y >= L) y -= L;
  if (y < 0) y = 0;
  return y;
}

/* Two standard normals by the Box-Muller transform of two uniforms. */
static void box_muller(uint32_t w[4], double* z0, double* z1) {
  double u1 = orc_u01(w[0], w[1]), u2 = orc_u01(w[2], w[3]);
  double r = sqrt(-2.0 * log(1.0 - u1));
  double th = 2.0 * M_PI * u2;
  *z0 = r * cos(th);
  *z1 = r * sin(th);
}

static int nh_steps(orc_sys* s, int64_t n_steps);

/* BAOAB Langevin velocity Verlet (gamma = 0 gives plain velocity Verlet). */
int orc_md_steps(orc_sys* s, int64_t n_steps) {
  if (!s->vx) return -1;
  if (s->ens) return nh_steps(s, n_steps);
  double dt = s->dt;
  double c1 = exp(-s->gamma * dt), c2 = sqrt(1.0 - c1 * c1);
  for (int64_t q = 0; q < n_steps; ++q) {
    for (int64_t i = 0; i < s->n; ++i) {
      double im = FTM / s->mass[s->t[i]];
      s->vx[i] += 0.5 * dt * s->fx[i] * im;
      s->vy[i] += 0.5 * dt * s->fy[i] * im;
      s->vz[i] += 0.5 * dt * s->fz[i] * im;
      s->x[i] += 0.5 * dt * s->vx[i];
      s->y[i] += 0.5 * dt * s->vy[i];
      s->z[i] += 0.5 * dt * s->vz[i];
      if (s->gamma > 0) {
        double sig = sqrt(KB_EV * s->T_md * FTM / s->mass[s->t[i]]);
        uint32_t ctr[4] = {(uint32_t)s->md_step, (uint32_t)(s->md_step >> 32), (uint32_t)i, 3u};
        uint32_t w[4];
        double z0, z1, z2, z3;
        orc_philox(ctr, s->md_key, w);
        box_muller(w, &z0, &z1);
        ctr[3] = 4u;
        orc_philox(ctr, s->md_key, w);
        box_muller(w, &z2, &z3);
        s->vx[i] = c1 * s->vx[i] + c2 * sig * z0;
        s->vy[i] = c1 * s->vy[i] + c2 * sig * z1;
        s->vz[i] = c1 * s->vz[i] + c2 * sig * z2;
      }
      s->x[i] = wrap(s->x[i] + 0.5 * dt * s->vx[i], s->box[0]);
      s->y[i] = wrap(s->y[i] + 0.5 * dt * s->vy[i], s->box[1]);
      s->z[i] = wrap(s->z[i] + 0.5 * dt * s->vz[i], s->box[2]);
    }
    if (build_neighbours(s)) return -1;
    compute_rho(s);
    orc_forces(s, s->fx, s->fy, s->fz);
    for (int64_t i = 0; i < s->n; ++i) {
      double im = FTM / s->mass[s->t[i]];
      s->vx[i] += 0.5 * dt * s->fx[i] * im;
      s->vy[i] += 0.5 * dt * s->fy[i] * im;
      s->vz[i] += 0.5 * dt * s->fz[i] * im;
    }
    s->md_step++;
  }
  s->energy = orc_energy_full(s);
  return 0;
}

/* ------------------------------------------------ Nose-Hoover ensembles */
#define BAR_EV_A3 6.241509074460763e-07 /* 1 bar in eV / A^3 */

int orc_set_ensemble(orc_sys* s, int kind, double t_damp, double p_damp, double p_ext_bar, int chain) {
  if (kind < 0 || kind > 2 || chain < 1 || chain > ORC_MAX_CHAIN) return -1;
  if (kind && !(t_damp > 0.0)) return -1;
  if (kind == 2 && !(p_damp > 0.0)) return -1;
  s->ens = kind;
  s->chain = chain;
  s->t_damp = t_damp;
  s->p_damp = p_damp;
  s->p_ext = p_ext_bar * BAR_EV_A3;
  double kT = KB_EV * s->T_md, nf = 3.0 * (double)s->n;
  for (int k = 0; k < ORC_MAX_CHAIN; ++k) {
    s->xi[k] = s->eta[k] = s->xib[k] = s->etab[k] = 0.0;
    s->Q[k] = (k == 0 ? nf : 1.0) * kT * t_damp * t_damp;
    s->Qb[k] = kT * p_damp * p_damp;
  }
  s->veps = 0.0;
  s->W = (nf + 3.0) * kT * p_damp * p_damp;
  return 0;
}

double orc_virial(orc_sys* s) {
  double* f = (double*)malloc(sizeof(double) * 3 * s->n);
  orc_forces(s, f, f + s->n, f + 2 * s->n);
  free(f);
  return s->virial;
}

/* sum_i m_i v_i^2 (eV), twice the kinetic energy */
static double twice_ke(const orc_sys* s) {
  double k2 = 0.0;
  for (int64_t i = 0; i < s->n; ++i)
    k2 += s->mass[s->t[i]] / FTM * (s->vx[i] * s->vx[i] + s->vy[i] * s->vy[i] + s->vz[i] * s->vz[i]);
  return k2;
}

/* Propagate a Nose-Hoover chain (M links, masses Q, velocities xi,
 * positions eta) for a time h, driven by K2 = sum m v^2 of the g degrees
 * of freedom it couples to (target g kT).  Symmetric splitting: the last
 * link a half step, the links down to the first with the next link's
 * friction applied as exp factors around each half kick, the coupled
 * velocities scaled by exp(-h xi_1), the positions eta advanced, and the
 * mirror sequence back up.  Returns the velocity scale factor. */
static double nhc_propagate(int M, const double* Q, double* xi, double* eta, double K2, double gkT, double kT,
                            double h) {
  double scale = 1.0;
  for (int pass = 0; pass < 2; ++pass) {
    /* pass 0: links M..1; pass 1 (after the scaling): links 1..M */
    for (int q = 0; q < M; ++q) {
      int k = pass == 0 ? M - 1 - q : q;
      double G = k == 0 ? (K2 * scale * scale - gkT) / Q[0] : (Q[k - 1] * xi[k - 1] * xi[k - 1] - kT) / Q[k];
      double e = k + 1 < M ? exp(-0.25 * h * xi[k + 1]) : 1.0;
      xi[k] = (xi[k] * e + 0.5 * h * G) * e;
    }
    if (pass == 0) {
      scale = exp(-h * xi[0]);
      for (int k = 0; k < M; ++k) eta[k] += h * xi[k];
    }
  }
  return scale;
}

static double sinhc(double x) {
  /* sinh(x) / x; the Taylor series where x is small */
  if (fabs(x) < 1e-4) return 1.0 + x * x / 6.0 + x * x * x * x / 120.0;
  return sinh(x) / x;
}

/* One half kick of the particle velocities with the barostat coupling
 * alpha v_eps: v <- v e^{-a h} + h (F/m) e^{-a h/2} sinhc(a h/2). */
static void kick(orc_sys* s, double h, double a) {
  double e1 = exp(-a * h), e2 = exp(-0.5 * a * h) * sinhc(0.5 * a * h);
  for (int64_t i = 0; i < s->n; ++i) {
    double im = FTM / s->mass[s->t[i]];
    s->vx[i] = s->vx[i] * e1 + h * s->fx[i] * im * e2;
    s->vy[i] = s->vy[i] * e1 + h * s->fy[i] * im * e2;
    s->vz[i] = s->vz[i] * e1 + h * s->fz[i] * im * e2;
  }
}

static void scale_v(orc_sys* s, double f) {
  for (int64_t i = 0; i < s->n; ++i) {
    s->vx[i] *= f;
    s->vy[i] *= f;
    s->vz[i] *= f;
  }
}

/* barostat force: [alpha K2 + W_vir - 3 V P_ext] / W, alpha = 1 + 3 / N_f */
static double baro_force(const orc_sys* s, double K2) {
  double nf = 3.0 * (double)s->n, V = s->box[0] * s->box[1] * s->box[2];
  return ((1.0 + 3.0 / nf) * K2 + s->virial - 3.0 * V * s->p_ext) / s->W;
}

/* Trotter-split MTK step: thermostats, barostat velocity, particle
 * velocities, positions and box, forces, and the mirror sequence. */
static int nh_steps(orc_sys* s, int64_t n_steps) {
  double dt = s->dt, h = 0.5 * dt, kT = KB_EV * s->T_md, nf = 3.0 * (double)s->n;
  int npt = s->ens == 2;
  for (int64_t q = 0; q < n_steps; ++q) {
    for (int half = 0; half < 2; ++half) {
      if (half == 1) {
        /* positions and box: r e^{v dt} + dt v e^{v dt/2} sinhc(v dt/2) */
        double ve = npt ? s->veps : 0.0;
        double e1 = exp(ve * dt), e2 = dt * exp(0.5 * ve * dt) * sinhc(0.5 * ve * dt);
        for (int a = 0; a < 3; ++a) s->box[a] *= e1;
        for (int64_t i = 0; i < s->n; ++i) {
          s->x[i] = wrap(s->x[i] * e1 + s->vx[i] * e2, s->box[0]);
          s->y[i] = wrap(s->y[i] * e1 + s->vy[i] * e2, s->box[1]);
          s->z[i] = wrap(s->z[i] * e1 + s->vz[i] * e2, s->box[2]);
        }
        if (build_neighbours(s)) return -1;
        compute_rho(s);
        orc_forces(s, s->fx, s->fy, s->fz);
        kick(s, h, npt ? (1.0 + 3.0 / nf) * s->veps : 0.0);
        if (npt) {
          s->veps += h * baro_force(s, twice_ke(s));
          s->veps *= nhc_propagate(s->chain, s->Qb, s->xib, s->etab, s->W * s->veps * s->veps, kT, kT, h);
        }
        scale_v(s, nhc_propagate(s->chain, s->Q, s->xi, s->eta, twice_ke(s), nf * kT, kT, h));
      } else {
        scale_v(s, nhc_propagate(s->chain, s->Q, s->xi, s->eta, twice_ke(s), nf * kT, kT, h));
        if (npt) {
          s->veps *= nhc_propagate(s->chain, s->Qb, s->xib, s->etab, s->W * s->veps * s->veps, kT, kT, h);
          s->veps += h * baro_force(s, twice_ke(s));
        }
        kick(s, h, npt ? (1.0 + 3.0 / nf) * s->veps : 0.0);
      }
    }
    s->md_step++;
  }
  s->energy = orc_energy_full(s);
  return 0;
}

void orc_md_state(orc_sys* s, double out[9]) {
  double K2 = s->vx ? twice_ke(s) : 0.0, nf = 3.0 * (double)s->n, kT = KB_EV * s->T_md;
  double V = s->box[0] * s->box[1] * s->box[2];
  double pe = orc_energy_full(s);
  double vir = orc_virial(s);
  double H = 0.5 * K2 + pe;
  if (s->ens) {
    for (int k = 0; k < s->chain; ++k) H += 0.5 * s->Q[k] * s->xi[k] * s->xi[k] + (k == 0 ? nf : 1.0) * kT * s->eta[k];
    if (s->ens == 2) {
      H += s->p_ext * V + 0.5 * s->W * s->veps * s->veps;
      for (int k = 0; k < s->chain; ++k) H += 0.5 * s->Qb[k] * s->xib[k] * s->xib[k] + kT * s->etab[k];
    }
  }
  out[0] = 0.5 * K2;
  out[1] = pe;
  out[2] = K2 / (nf * KB_EV);
  out[3] = (K2 + vir) / (3.0 * V) / BAR_EV_A3;
  out[4] = V;
  out[5] = H;
  out[6] = s->box[0];
  out[7] = s->box[1];
  out[8] = s->box[2];
}

/* ------------------------------------------------- conjugate gradients */
static double dot3(const orc_sys* s, const double* a, const double* b) {
  double t = 0.0;
  for (int64_t i = 0; i < 3 * s->n; ++i) t += a[i] * b[i];
  (void)s;
  return t;
}

/* energy and forces at x0 + alpha d (positions wrapped), into f */
static double eval_at(orc_sys* s, const double* x0, const double* d, double alpha, double* f) {
  for (int64_t i = 0; i < s->n; ++i) {
    s->x[i] = wrap(x0[i] + alpha * d[i], s->box[0]);
    s->y[i] = wrap(x0[s->n + i] + alpha * d[s->n + i], s->box[1]);
    s->z[i] = wrap(x0[2 * s->n + i] + alpha * d[2 * s->n + i], s->box[2]);
  }
  build_neighbours(s);
  compute_rho(s);
  orc_forces(s, f, f + s->n, f + 2 * s->n);
  return orc_energy_full(s);
}

int orc_minimize(orc_sys* s, double ftol, int64_t max_iter, int64_t* iters, double* fmax_out) {
  int64_t n3 = 3 * s->n;
  double* x0 = (double*)malloc(sizeof(double) * n3);
  double* f = (double*)malloc(sizeof(double) * n3);
  double* g = (double*)malloc(sizeof(double) * n3);
  double* d = (double*)malloc(sizeof(double) * n3);
  if (!x0 || !f || !g || !d) { free(x0); free(f); free(g); free(d); return -1; }
  memcpy(x0, s->x, sizeof(double) * s->n);
  memcpy(x0 + s->n, s->y, sizeof(double) * s->n);
  memcpy(x0 + 2 * s->n, s->z, sizeof(double) * s->n);
  eval_at(s, x0, x0, 0.0, f);
  memcpy(d, f, sizeof(double) * n3);
  double ff = dot3(s, f, f), step = 0.0;
  int64_t it = 0;
  int rc = 1;
  double fmax = 0.0;
  for (; it < max_iter; ++it) {
    fmax = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
      double a = sqrt(f[i] * f[i] + f[s->n + i] * f[s->n + i] + f[2 * s->n + i] * f[2 * s->n + i]);
      if (a > fmax) fmax = a;
    }
    if (fmax < ftol) { rc = 0; break; }
    /* line search: a zero of phi'(alpha) = -F(x0 + alpha d) . d by secant
     * steps from 0 and a first step that moves no atom more than 0.05 A */
    double dmax = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
      double a = sqrt(d[i] * d[i] + d[s->n + i] * d[s->n + i] + d[2 * s->n + i] * d[2 * s->n + i]);
      if (a > dmax) dmax = a;
    }
    double a0 = 0.0, p0 = -dot3(s, f, d), pstart = fabs(p0);
    double a1 = step > 0.0 ? step : 0.05 / dmax;
    if (a1 * dmax > 0.2) a1 = 0.2 / dmax;
    eval_at(s, x0, d, a1, g);
    double p1 = -dot3(s, g, d);
    /* extend until the derivative changes sign */
    for (int ls = 0; ls < 30 && p1 < 0.0 && fabs(p1) > 1e-3 * pstart; ++ls) {
      a0 = a1;
      p0 = p1;
      a1 *= 2.0;
      eval_at(s, x0, d, a1, g);
      p1 = -dot3(s, g, d);
    }
    /* regula falsi inside [a0, a1] (p0 < 0 < p1) */
    for (int ls = 0; ls < 40 && fabs(p1) > 1e-3 * pstart && p1 > 0.0; ++ls) {
      double a2 = a0 - p0 * (a1 - a0) / (p1 - p0);
      eval_at(s, x0, d, a2, g);
      double p2 = -dot3(s, g, d);
      if (p2 < 0.0) {
        a0 = a2;
        p0 = p2;
        if (fabs(p2) <= 1e-3 * pstart) {
          a1 = a2;
          p1 = p2;
        }
      } else {
        a1 = a2;
        p1 = p2;
      }
    }
    if (p1 > 0.0 && fabs(p1) > 1e-3 * pstart) eval_at(s, x0, d, a1, g); /* positions at a1 */
    step = a1;
    for (int64_t i = 0; i < s->n; ++i) {
      x0[i] = s->x[i];
      x0[s->n + i] = s->y[i];
      x0[2 * s->n + i] = s->z[i];
    }
    /* Polak-Ribiere with restart */
    double gg = dot3(s, g, g), gf = dot3(s, g, f);
    double beta = (gg - gf) / ff;
    if (beta < 0.0) beta = 0.0;
    for (int64_t k = 0; k < n3; ++k) d[k] = g[k] + beta * d[k];
    if (dot3(s, g, d) <= 0.0) memcpy(d, g, sizeof(double) * n3);
    memcpy(f, g, sizeof(double) * n3);
    ff = gg;
  }
  if (s->fx) memcpy(s->fx, f, sizeof(double) * s->n), memcpy(s->fy, f + s->n, sizeof(double) * s->n),
      memcpy(s->fz, f + 2 * s->n, sizeof(double) * s->n);
  s->energy = orc_energy_full(s);
  if (iters) *iters = it;
  if (fmax_out) *fmax_out = fmax;
  free(x0); free(f); free(g); free(d);
  return rc;
}

void orc_get_md(const orc_sys* s, double* x, double* y, double* z, double* vx, double* vy,
                double* vz) {
  if (x) memcpy(x, s->x, sizeof(double) * s->n);
  if (y) memcpy(y, s->y, sizeof(double) * s->n);
  if (z) memcpy(z, s->z, sizeof(double) * s->n);
  if (vx && s->vx) memcpy(vx, s->vx, sizeof(double) * s->n);
  if (vy && s->vy) memcpy(vy, s->vy, sizeof(double) * s->n);
  if (vz && s->vz) memcpy(vz, s->vz, sizeof(double) * s->n);
}

double orc_kinetic_energy(const orc_sys* s) {
  if (!s->vx) return 0.0;
  double ke = 0.0;
  for (int64_t i = 0; i < s->n; ++i)
    ke += 0.5 * s->mass[s->t[i]] / FTM *
          (s->vx[i] * s->vx[i] + s->vy[i] * s->vy[i] + s->vz[i] * s->vz[i]);
  return ke;
}

/* Hybrid MC/MD (Sec. IV A): n_md MD steps, then n_mc composite steps on the
 * frozen positions.  Spatial schedules are rebuilt from the new positions. */
int orc_hybrid_cycles(orc_sys* s, int64_t n_cycles, int64_t n_md, int64_t n_mc) {
  for (int64_t c = 0; c < n_cycles; ++c) {
    if (orc_md_steps(s, n_md)) return -1;
    if (s->sched_kind == 3 &&
        orc_schedule_spatial(s, s->sched_args[0], s->sched_args[1], s->sched_args[2],
                             s->sched_args[3], s->sched_args[4], s->sched_args[5]))
      return -1;
    if (orc_parallel_steps(s, n_mc)) return -1;
    /* forces follow the new types */
    orc_forces(s, s->fx, s->fy, s->fz);
  }
  return 0;
}
