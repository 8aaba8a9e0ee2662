// Error bound of the FP32 screen with re-embedding (host side, shared by the
// binary and the multicomponent contexts).
//
// For one embedding cubic p_j(t) = c0 + t (c1 + t (c2 + t c3)) on interval j
// (t = x / h - j), an FP32 evaluation at an argument carried in float differs
// from the FP64 one by at most 2^-24 [5 G + 4 P + 2 dmax S] to first order:
//   G = max_j sum_k |c_jk|: coefficient rounding and three FMAs;
//   P = max_j (j + 2) max(D_j-1, D_j, D_j+1), D_j = |c1| + 2|c2| + 3|c3|:
//       |x F'| near interval j (the argument rho + (f_b - f_a) and x / h
//       carry relative errors 2^-24 (|rho| + |f_b - f_a| + 3|x|));
//   S = max_j D_j / h, dmax = max |f_b(r_s) - f_a(r_s)|: the part of that
//       argument error that scales with |f_b - f_a|.
// The bound taken is 2^-24 [6 G + 5 P + 3 dmax S] over the species and the
// intervals of the screened range [x_lo, x_max (1 - 10^-6)], x_lo = max(h,
// x_max / 20): the FP64 evaluation is in range there, and below x_lo (a
// nearly isolated atom) the slope of a sqrt-like embedding would dominate.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace vcsgc {

struct ScreenBound {
  double err;  // eV per evaluation
  double lo, hi;
};

// cubics[t][j]: the FP64 coefficients of species t's embedding on a grid of
// spacing h (all species on one grid); dmax as above
inline ScreenBound screen_bound(const std::vector<std::vector<Cubic>>& cubics, double h, double dmax) {
  const int n = (int)cubics[0].size();
  const double xmax = n * h;
  const double lo = std::max(h, xmax / 20.0);
  const int jlo = std::max(0, (int)std::floor(lo / h) - 1);
  double G = 0.0, P = 0.0, S = 0.0;
  for (const std::vector<Cubic>& hc : cubics) {
    std::vector<double> D((size_t)n, 0.0);
    for (int j = jlo; j < n; ++j) {
      const Cubic& c = hc[j];
      G = std::max(G, std::fabs(c.x) + std::fabs(c.y) + std::fabs(c.z) + std::fabs(c.w));
      D[j] = std::fabs(c.y) + 2.0 * std::fabs(c.z) + 3.0 * std::fabs(c.w);
      S = std::max(S, D[j] / h);
    }
    for (int j = jlo + 1; j < n; ++j) {
      const double dn = std::max(D[j], std::max(D[j - 1], j + 1 < n ? D[j + 1] : 0.0));
      P = std::max(P, (double)(j + 2) * dn);
    }
  }
  ScreenBound b;
  b.err = std::ldexp(6.0 * G + 5.0 * P + 3.0 * dmax * S, -24) * (1.0 + 1e-6);
  b.lo = lo;
  b.hi = xmax * (1.0 - 1e-6);
  return b;
}

// The same bound for arguments confined to [lo, hi] (the intervals that
// reach them, and their neighbours in P), for cubics offset by a constant
// per species.  The offset changes c0 only, so it shrinks G where the
// function is far from zero; an evaluation of the offset table differs
// from the FP64 offset cubic by at most the bound returned.
inline double screen_bound_in(const std::vector<std::vector<Cubic>>& cubics, double h, double dmax, double lo,
                              double hi) {
  const int n = (int)cubics[0].size();
  const int j0 = std::max(0, (int)std::floor(lo / h) - 1);
  const int j1 = std::min(n - 1, (int)std::floor(hi / h) + 1);
  double G = 0.0, P = 0.0, S = 0.0;
  for (const std::vector<Cubic>& hc : cubics) {
    auto D = [&](int j) {
      if (j < 0 || j >= n) return 0.0;
      const Cubic& c = hc[j];
      return std::fabs(c.y) + 2.0 * std::fabs(c.z) + 3.0 * std::fabs(c.w);
    };
    for (int j = j0; j <= j1; ++j) {
      const Cubic& c = hc[j];
      G = std::max(G, std::fabs(c.x) + std::fabs(c.y) + std::fabs(c.z) + std::fabs(c.w));
      S = std::max(S, D(j) / h);
      P = std::max(P, (double)(j + 2) * std::max(D(j), std::max(D(j - 1), D(j + 1))));
    }
  }
  return std::ldexp(6.0 * G + 5.0 * P + 3.0 * dmax * S, -24) * (1.0 + 1e-6);
}

}  // namespace vcsgc
