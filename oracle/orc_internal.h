/* Primitives shared by the two oracle files (binary and multicomponent):
 * the Philox counter generator and cubic Hermite interpolation on a uniform
 * grid.  TEST INFRASTRUCTURE, like the rest of oracle/: only the tests, the
 * smoke check and the benchmark's CPU baseline use it. */
#ifndef ORC_INTERNAL_H
#define ORC_INTERNAL_H

#include <stdint.h>

typedef struct {
  int n;
  double h;
  double* y;
  double* m; /* knot derivatives */
} spline_t;

/* Copy n samples y (and knot derivatives m, or central differences when m
 * is NULL) on the grid x_j = j h.  Returns 0, or -1 when out of memory. */
int orc_hermite_init(spline_t* sp, int n, double h, const double* y, const double* m);
/* Value (and derivative) at x in [0, (n-1) h]; returns -1 outside. */
int orc_hermite_eval(const spline_t* sp, double x, double* v, double* dv);

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t lo, uint32_t hi);
uint64_t orc_below(uint32_t lo, uint32_t hi, uint64_t m);

#endif
