// kernels_nbr.cu -- table set-up, neighbour lists, electron density and
// total energy (EAM, Daw-Baskes form; the short-range many-body potential of
// Sec. III A of Sadigh et al.).
#include "common.cuh"
#include "kernels.h"

namespace vcsgc {

// ------------------------------------------------------------ splines
// Hermite data (y_j, m_j) on [x_j, x_j + h] -> power-form cubic in t:
//   c0 = y0, c1 = h m0, c2 = 3 (y1 - y0) - h (2 m0 + m1), c3 = 2 (y0 - y1) + h (m0 + m1).
// Missing derivatives: central differences, one-sided at the ends.
__global__ void k_spline_coeffs(const double* y, const double* m, int n, double h, Cubic* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n - 1) return;
  auto slope = [&](int q) -> double {
    if (m) return m[q];
    if (q == 0) return (y[1] - y[0]) / h;
    if (q == n - 1) return (y[n - 1] - y[n - 2]) / h;
    return (y[q + 1] - y[q - 1]) / (2.0 * h);
  };
  const double y0 = y[j], y1 = y[j + 1];
  const double m0 = h * slope(j), m1 = h * slope(j + 1);
  out[j] = Cubic{y0, m0, 3.0 * (y1 - y0) - 2.0 * m0 - m1, 2.0 * (y0 - y1) + m0 + m1};
}

void launch_spline_coeffs(const double* y, const double* m, int n, double h, Cubic* out,
                          cudaStream_t st) {
  k_spline_coeffs<<<(n + 255) / 256, 256, 0, st>>>(y, m, n, h, out);
}

__global__ void k_spline_derivs(const Cubic* c, int n_int, double inv_h, Cubic* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_int) return;
  const Cubic q = c[j];
  out[j] = Cubic{q.y * inv_h, 2.0 * q.z * inv_h, 3.0 * q.w * inv_h, 0.0};
}

void launch_spline_derivs(const Cubic* c, int n_int, double h, Cubic* out, cudaStream_t st) {
  k_spline_derivs<<<(n_int + 255) / 256, 256, 0, st>>>(c, n_int, 1.0 / h, out);
}

__global__ void k_to_cubic32(const Cubic* c, int n_int, Cubic32* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_int) return;
  const Cubic q = c[j];
  out[j] = Cubic32{(float)q.x, (float)q.y, (float)q.z, (float)q.w};
}

void launch_to_cubic32(const Cubic* c, int n_int, Cubic32* out, cudaStream_t st) {
  k_to_cubic32<<<(n_int + 255) / 256, 256, 0, st>>>(c, n_int, out);
}

// ------------------------------------------------------- shell tables
// Rigid lattice: the pair part of dE(A->B) is
//   sum_s [ (z_s - b_s) (phi_BA - phi_AA)(r_s) + b_s (phi_BB - phi_AB)(r_s) ]
//   = C_A + sum_s b_s G_A[s],
// C_A = sum_s z_s (phi_AB - phi_AA)(r_s), G_A[s] = (phi_BB - 2 phi_AB + phi_AA)(r_s).
// value of table q at r: FP64, or FP32 interpolation widened (mixed form)
__device__ __forceinline__ double tab_val(const Tables& tab, const Tables32* t32, int q, double r,
                                          unsigned* err) {
  if (t32) {
    float t;
    const int j = spline32_locate(t32->sp[q], (float)r, t, err);
    return (double)spline32_val_at(t32->sp[q], j, t);
  }
  return spline_val(tab.sp[q], r, err);
}

__global__ void k_shell_tables(Tables tab, Tables32 tab32, int mixed, const int* h2, const int* z,
                               int S, double a, double* out, unsigned* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Tables32* t32 = mixed ? &tab32 : nullptr;
  double C = 0.0;
  for (int s = 0; s < S; ++s) {
    const double r = 0.5 * a * sqrt((double)h2[s]);
    const double pAA = tab_val(tab, t32, 0, r, err);
    const double pAB = tab_val(tab, t32, 1, r, err);
    const double pBB = tab_val(tab, t32, 2, r, err);
    C += (double)z[s] * (pAB - pAA);
    out[1 + s] = (pBB - pAB) - (pAB - pAA);
    out[1 + S + s] = tab_val(tab, t32, 4, r, err) - tab_val(tab, t32, 3, r, err);
    out[1 + 2 * S + s] = r;
  }
  out[0] = C;
}

// Energy table of the rigid lattice with one density function (uniform
// rho0): etab[s], etab[S + s], etab[2S + s] = phi_AA, phi_AB, phi_BB at r_s
// (r_s = shell_tab[1 + 2S + s]), etab[3S] = F_A(rho0), etab[3S + 1] =
// F_B(rho0), etab[3S + 2 + s] = z_s.  Site energy: F_t(rho0) + 1/2 sum_s
// [(z_s - b_s) phi_{tA}(r_s) + b_s phi_{tB}(r_s)].
__global__ void k_lattice_energy_table(Tables tab, Tables32 tab32, int mixed, const double* shell_tab, int S,
                                       LatZ z, const double* rho, double* etab, unsigned* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Tables32* t32 = mixed ? &tab32 : nullptr;
  for (int s = 0; s < S; ++s) {
    const double r = shell_tab[1 + 2 * S + s];
    etab[s] = tab_val(tab, t32, 0, r, err);
    etab[S + s] = tab_val(tab, t32, 1, r, err);
    etab[2 * S + s] = tab_val(tab, t32, 2, r, err);
    etab[3 * S + 2 + s] = (double)z.z[s];
  }
  etab[3 * S] = tab_val(tab, t32, 5, rho[0], err);
  etab[3 * S + 1] = tab_val(tab, t32, 6, rho[0], err);
}

void launch_lattice_energy_table(Tables tab, const Tables32* tab32, const double* shell_tab, int S, LatZ z,
                                 const double* rho, double* etab, unsigned* err, cudaStream_t st) {
  Tables32 t{};
  if (tab32) t = *tab32;
  k_lattice_energy_table<<<1, 32, 0, st>>>(tab, t, tab32 ? 1 : 0, shell_tab, S, z, rho, etab, err);
}

void launch_shell_tables(Tables tab, const int* h2, const int* z, int S, double a, double* out,
                         unsigned* err, cudaStream_t st, const Tables32* tab32) {
  Tables32 t{};
  if (tab32) t = *tab32;
  k_shell_tables<<<1, 32, 0, st>>>(tab, t, tab32 ? 1 : 0, h2, z, S, a, out, err);
}

// --------------------------------------------------- lattice neighbours
// Site (cx, cy, cz, b) has half-lattice coordinates H = 2 c + b; the
// neighbour at offset h has coordinates H + h (periodic in 2 n), basis
// (H + h) mod 2 and cell (H + h) / 2.
__global__ void k_lattice_nbr(int nx, int ny, int nz, const int3* hoff, int K, int* nbr, int* cnt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = 2LL * nx * ny * nz;
  if (i >= N) return;
  const int b = (int)(i & 1);
  const long long cell = i >> 1;
  const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((long long)nx * ny));
  const int X = 2 * cx + b, Y = 2 * cy + b, Z = 2 * cz + b;
  for (int k = 0; k < K; ++k) {
    const int3 h = hoff[k];
    int hx = (X + h.x) % (2 * nx); if (hx < 0) hx += 2 * nx;
    int hy = (Y + h.y) % (2 * ny); if (hy < 0) hy += 2 * ny;
    int hz = (Z + h.z) % (2 * nz); if (hz < 0) hz += 2 * nz;
    const int bb = hx & 1;
    const long long j = (((long long)(hz >> 1) * ny + (hy >> 1)) * nx + (hx >> 1)) * 2 + bb;
    nbr[i * K + k] = (int)j;
  }
  cnt[i] = K;
}

void launch_lattice_neighbours(int nx, int ny, int nz, const int3* hoff, int K, int* nbr, int* cnt,
                               cudaStream_t st) {
  const long long N = 2LL * nx * ny * nz;
  k_lattice_nbr<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(nx, ny, nz, hoff, K, nbr, cnt);
}

// ------------------------------------------------------ cell neighbours
// periodic image of v in [0, L): positions outside the box (a caller's, or
// one rounding step past an edge) are binned where their image lies
__device__ __forceinline__ double wrap_into(double v, double L) {
  const double w = v - L * floor(v / L);
  return w < L ? w : 0.0;  // v a hair below a multiple of L rounds up to L
}

__device__ __forceinline__ int cell_index(double w, double L, int n) {
  const int c = (int)(w / L * n);
  return c < n ? c : n - 1;
}

__global__ void k_cell_assign(long long N, const double* x, const double* y, const double* z,
                              double bx, double by, double bz, int nx, int ny, int nz,
                              int* cell_of, int* count, float* x32, float* y32, float* z32) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double wx = wrap_into(x[i], bx), wy = wrap_into(y[i], by), wz = wrap_into(z[i], bz);
  const int c = (cell_index(wz, bz, nz) * ny + cell_index(wy, by, ny)) * nx + cell_index(wx, bx, nx);
  cell_of[i] = c;
  atomicAdd(&count[c], 1);
  x32[i] = (float)wx;
  y32[i] = (float)wy;
  z32[i] = (float)wz;
}

// exclusive scan of count[0..n) into start[0..n], one block
__global__ void k_scan(const int* count, int n, int* start) {
  __shared__ int carry;
  __shared__ int warp_sum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < n ? count[i] : 0;
    int s = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int q = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += q;
    }
    if (lane == 31) warp_sum[w] = s;
    __syncthreads();
    if (w == 0) {
      int ws = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int q = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += q;
      }
      warp_sum[lane] = ws;
    }
    __syncthreads();
    const int prefix = carry + (w ? warp_sum[w - 1] : 0) + s - v;
    if (i < n) start[i] = prefix;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = prefix + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_cell_scatter(long long N, const int* cell_of, const int* start, int* cursor, int* sorted) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int c = cell_of[i];
  sorted[start[c] + atomicAdd(&cursor[c], 1)] = (int)i;
}

// order each cell's members by index so the neighbour order is reproducible
__global__ void k_cell_sort(int ncell, const int* start, int* sorted) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int b = start[c], e = start[c + 1];
  for (int p = b + 1; p < e; ++p) {
    const int v = sorted[p];
    int q = p - 1;
    while (q >= b && sorted[q] > v) {
      sorted[q + 1] = sorted[q];
      --q;
    }
    sorted[q + 1] = v;
  }
}

// Candidates are tested in FP32 against (rl + m)^2, m = 0.01 A + 1e-6 L_max:
// the wrapped coordinates lie in [0, L), so the FP32 minimum-image distance
// is within about 7 L 2^-24 < 1e-6 L of the exact one, and every pair within
// rl is listed; the few extra pairs in [rl, rl + m) are skipped where the
// list is used (r >= r_c).
__global__ void k_cell_nbr(long long N, const float* x, const float* y, const float* z, float bx,
                           float by, float bz, int nx, int ny, int nz, const int* cell_of,
                           const int* start, const int* sorted, float rl2, int K, int* nbr, int* cnt,
                           unsigned* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int c = cell_of[i];
  const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
  const float xi = x[i], yi = y[i], zi = z[i];
  const float ibx = 1.0f / bx, iby = 1.0f / by, ibz = 1.0f / bz;
  int m = 0;
  for (int oz = -1; oz <= 1; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        const int qx = (cx + ox + nx) % nx, qy = (cy + oy + ny) % ny, qz = (cz + oz + nz) % nz;
        const int q = (qz * ny + qy) * nx + qx;
        for (int p = start[q]; p < start[q + 1]; ++p) {
          const int j = sorted[p];
          if (j == i) continue;
          float dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
          dx -= bx * rintf(dx * ibx);
          dy -= by * rintf(dy * iby);
          dz -= bz * rintf(dz * ibz);
          if (dx * dx + dy * dy + dz * dz < rl2) {
            if (m < K) nbr[i * K + m] = j;
            ++m;
          }
        }
      }
  if (m > K) atomicOr(err, ERRF_OVERFLOW);
  const int mm = m < K ? m : K;
  for (int k = mm; k < K; ++k) nbr[i * K + k] = -1;
  cnt[i] = mm;
}

void launch_cell_neighbours(long long N, const double* x, const double* y, const double* z,
                            const double box[3], double rl, CellList cl, int K, int* nbr, int* cnt,
                            unsigned* err, cudaStream_t st) {
  const int ncell = cl.nc[0] * cl.nc[1] * cl.nc[2];
  const unsigned g = (unsigned)((N + 127) / 128);
  cudaMemsetAsync(cl.cell_count, 0, sizeof(int) * ncell, st);
  cudaMemsetAsync(cl.cell_cursor, 0, sizeof(int) * ncell, st);
  k_cell_assign<<<g, 128, 0, st>>>(N, x, y, z, box[0], box[1], box[2], cl.nc[0], cl.nc[1], cl.nc[2],
                                   cl.cell_of, cl.cell_count, cl.x32, cl.y32, cl.z32);
  k_scan<<<1, 1024, 0, st>>>(cl.cell_count, ncell, cl.cell_start);
  k_cell_scatter<<<g, 128, 0, st>>>(N, cl.cell_of, cl.cell_start, cl.cell_cursor, cl.sorted);
  k_cell_sort<<<(ncell + 127) / 128, 128, 0, st>>>(ncell, cl.cell_start, cl.sorted);
  const float rlm = (float)(rl + cell_list_margin(box));
  k_cell_nbr<<<g, 128, 0, st>>>(N, cl.x32, cl.y32, cl.z32, (float)box[0], (float)box[1], (float)box[2],
                                cl.nc[0], cl.nc[1], cl.nc[2], cl.cell_of, cl.cell_start, cl.sorted,
                                rlm * rlm, K, nbr, cnt, err);
}

// ------------------------------------------------- spatial colour schedule
// Domain of every atom for the SPATIAL schedule (boxes of the periodic cell,
// Sec. III A): box index from floor(v / L * n) clamped to the grid -- the
// host's rule, so the tables are the same -- mapped to its domain rank
// (colour-major, then box index) by dom_of_block.
__device__ __forceinline__ int spatial_box(double v, double L, int n) {
  const int q = (int)floor(v / L * n);
  return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

__global__ void k_spatial_assign(long long N, const double* x, const double* y, const double* z, double bx,
                                 double by, double bz, int nbx, int nby, int nbz, const int* dom_of_block,
                                 int* dom_of, int* count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = (spatial_box(z[i], bz, nbz) * nby + spatial_box(y[i], by, nby)) * nbx + spatial_box(x[i], bx, nbx);
  const int d = dom_of_block[b];
  dom_of[i] = d;
  atomicAdd(&count[d], 1);
}

void launch_spatial_schedule(long long N, const double* x, const double* y, const double* z, const double box[3],
                             const int nb[3], const int* dom_of_block, int ndom, int* dom_of, int* count,
                             int* cursor, int* dom_start, int* dom_sites, cudaStream_t st) {
  const unsigned g = (unsigned)((N + 127) / 128);
  cudaMemsetAsync(count, 0, sizeof(int) * ndom, st);
  cudaMemsetAsync(cursor, 0, sizeof(int) * ndom, st);
  k_spatial_assign<<<g, 128, 0, st>>>(N, x, y, z, box[0], box[1], box[2], nb[0], nb[1], nb[2], dom_of_block, dom_of,
                                      count);
  // counting sort by domain, ascending atom index within a domain (the
  // cell-list kernels with domains as bins)
  k_scan<<<1, 1024, 0, st>>>(count, ndom, dom_start);
  k_cell_scatter<<<g, 128, 0, st>>>(N, dom_of, dom_start, cursor, dom_sites);
  k_cell_sort<<<(ndom + 127) / 128, 128, 0, st>>>(ndom, dom_start, dom_sites);
}

__global__ void k_half_list(long long N, int K, const int* nbr, const int* cnt, int* nbr_h, int* cnt_h) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int* row = nbr + i * K;
  int* out = nbr_h + i * K;
  int m = 0;
  for (int k = 0; k < cnt[i]; ++k) {
    const int j = row[k];
    if (j > i) out[m++] = j;
  }
  cnt_h[i] = m;
}

void launch_half_list(long long N, int K, const int* nbr, const int* cnt, int* nbr_h, int* cnt_h,
                      cudaStream_t st) {
  k_half_list<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(N, K, nbr, cnt, nbr_h, cnt_h);
}

// ------------------------------------------------------ density, energy
__device__ __forceinline__ double pair_r(const McArgs& a, bool shell, int i, int k, int j, int s) {
  if (shell) return a.shell_tab[1 + 2 * a.n_shells + s];
  double dx = a.x[j] - a.x[i], dy = a.y[j] - a.y[i], dz = a.z[j] - a.z[i];
  dx -= a.box[0] * rint(dx / a.box[0]);
  dy -= a.box[1] * rint(dy / a.box[1]);
  dz -= a.box[2] * rint(dz / a.box[2]);
  const double r2 = dx * dx + dy * dy + dz * dz;
  return r2 * rsqrt_nr(r2);
}

// FP32 distance of pair (i, j) for the mixed form (r_s on the rigid lattice)
__device__ __forceinline__ float pair_r32(const McArgs& a, bool shell, int i, int j, int s) {
  if (shell) return (float)a.shell_tab[1 + 2 * a.n_shells + s];
  const float dx = fix_diff(a.ux[j], a.ux[i], a.ul[0]);
  const float dy = fix_diff(a.uy[j], a.uy[i], a.ul[1]);
  const float dz = fix_diff(a.uz[j], a.uz[i], a.ul[2]);
  return sqrtf(dx * dx + dy * dy + dz * dz);
}

// table q at the pair distance: FP64, or FP32 widened to FP64 (mixed)
template <bool MIXED>
__device__ __forceinline__ double pair_tab(const McArgs& a, int q, double r64, float r32) {
  if constexpr (MIXED) {
    float t;
    const int j = spline32_locate(a.tab32.sp[q], r32, t, a.err);
    return (double)spline32_val_at(a.tab32.sp[q], j, t);
  } else {
    return spline_val(a.tab.sp[q], r64, a.err);
  }
}

// rho_i = sum_k f_{t_k}(r_ik) (FP64 sum); dF_i = F_B(rho_i) - F_A(rho_i) (FP64)
template <bool SHELL, bool MIXED>
__global__ void k_rho(McArgs a, int r, double* dF) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t* ty = a.types + (long long)r * a.N;
  const int* row = a.nbr + i * a.K;
  const int cnt = a.nbr_cnt[i];
  double rho = 0.0;
  int s = 0;
  for (int k = 0; k < cnt; ++k) {
    if (SHELL) while (k >= a.shell_end[s]) ++s;
    const int j = row[k];
    double rr = 0.0;
    float rf = 0.0f;
    if (MIXED) {
      rf = pair_r32(a, SHELL, (int)i, j, s);
      if (rf >= (float)a.rc) continue;
    } else {
      rr = pair_r(a, SHELL, (int)i, k, j, s);
      if (rr >= a.rc) continue;
    }
    rho += pair_tab<MIXED>(a, 3 + ty[j], rr, rf);
  }
  double* out = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
  out[i] = rho;
  if (dF) dF[i] = spline_val(a.tab.sp[6], rho, a.err) - spline_val(a.tab.sp[5], rho, a.err);
}

void launch_rho(const McArgs& a, bool shell, int r, cudaStream_t st) {
  const unsigned g = (unsigned)((a.N + 127) / 128);
  double* dF = const_cast<double*>(a.dF);
  if (a.mixed && !shell) launch_fix_positions(a.N, a.x, a.y, a.z, a.box, a.ux, a.uy, a.uz, st);
  if (a.mixed) {
    if (shell) k_rho<true, true><<<g, 128, 0, st>>>(a, r, dF);
    else k_rho<false, true><<<g, 128, 0, st>>>(a, r, dF);
  } else {
    if (shell) k_rho<true, false><<<g, 128, 0, st>>>(a, r, dF);
    else k_rho<false, false><<<g, 128, 0, st>>>(a, r, dF);
  }
}

constexpr int E_BLOCK = 256;
int energy_blocks(long long N) { return (int)((N + E_BLOCK - 1) / E_BLOCK); }

// e_i = 1/2 sum_k phi_{t_i t_k}(r_ik) + F_{t_i}(rho_i), block partial sums
template <bool SHELL, bool MIXED>
__global__ void __launch_bounds__(E_BLOCK) k_energy(McArgs a, int r, double* part) {
  const long long i = (long long)blockIdx.x * E_BLOCK + threadIdx.x;
  double e = 0.0;
  if (i < a.N) {
    const uint8_t* ty = a.types + (long long)r * a.N;
    const int* row = a.nbr + i * a.K;
    const int cnt = a.nbr_cnt[i];
    const int ti = ty[i];
    double rho = 0.0, ph = 0.0;
    int s = 0;
    for (int k = 0; k < cnt; ++k) {
      if (SHELL) while (k >= a.shell_end[s]) ++s;
      const int j = row[k];
      double rr = 0.0;
      float rf = 0.0f;
      if (MIXED) {
        rf = pair_r32(a, SHELL, (int)i, j, s);
        if (rf >= (float)a.rc) continue;
      } else {
        rr = pair_r(a, SHELL, (int)i, k, j, s);
        if (rr >= a.rc) continue;
      }
      const int tj = ty[j];
      ph += pair_tab<MIXED>(a, ti + tj, rr, rf);
      rho += pair_tab<MIXED>(a, 3 + tj, rr, rf);
    }
    e = 0.5 * ph + spline_val(a.tab.sp[5 + ti], rho, a.err);
  }
  __shared__ double sh[E_BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < E_BLOCK / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

void launch_energy(const McArgs& a, bool shell, int r, double* part, cudaStream_t st) {
  const int g = energy_blocks(a.N);
  if (a.mixed && !shell) launch_fix_positions(a.N, a.x, a.y, a.z, a.box, a.ux, a.uy, a.uz, st);
  if (a.mixed) {
    if (shell) k_energy<true, true><<<g, E_BLOCK, 0, st>>>(a, r, part);
    else k_energy<false, true><<<g, E_BLOCK, 0, st>>>(a, r, part);
  } else {
    if (shell) k_energy<true, false><<<g, E_BLOCK, 0, st>>>(a, r, part);
    else k_energy<false, false><<<g, E_BLOCK, 0, st>>>(a, r, part);
  }
}

}  // namespace vcsgc
