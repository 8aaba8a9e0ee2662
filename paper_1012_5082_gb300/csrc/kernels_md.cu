// kernels_md.cu -- EAM forces and BAOAB Langevin velocity Verlet, the MD half
// of the hybrid MC/MD scheme (Sec. IV A of Sadigh et al.).
//   rho pass:   rho_i = sum_j f_{t_j}(r_ij), F'(rho_i), F_B(rho_i) - F_A(rho_i)
//   force pass: F_i = sum_j [phi'_{t_i t_j} + F'_i f'_{t_j} + F'_j f'_{t_i}](r_ij) (x_j - x_i)/r_ij
//   B A O A B:  half kick, half drift, Ornstein-Uhlenbeck velocity update with
//               Philox normals, half drift, (forces), half kick.
#include "common.cuh"
#include "kernels.h"

namespace vcsgc {

__device__ __forceinline__ double mimg(double d, double L, double iL) { return d - L * rint(d * iL); }

template <bool MIXED>
__global__ void k_md_rho(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int* row = m.nbr + i * m.K;
  const int cnt = m.nbr_cnt[i];
  const double xi = m.x[i], yi = m.y[i], zi = m.z[i];
  const uint32_t uxi = MIXED ? m.ux[i] : 0u, uyi = MIXED ? m.uy[i] : 0u, uzi = MIXED ? m.uz[i] : 0u;
  const double ix = 1.0 / m.box[0], iy = 1.0 / m.box[1], iz = 1.0 / m.box[2];
  const double rc2 = m.rc * m.rc;
  double rho = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int j = row[k];
    if constexpr (MIXED) {
      const float dx = fix_diff(m.ux[j], uxi, m.ul[0]);
      const float dy = fix_diff(m.uy[j], uyi, m.ul[1]);
      const float dz = fix_diff(m.uz[j], uzi, m.ul[2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= (float)rc2) continue;
      float t;
      const Spline32& sp = m.tab32.sp[3 + m.types[j]];
      const int q = spline32_locate(sp, sqrtf(r2), t, m.err);
      rho += (double)spline32_val_at(sp, q, t);
    } else {
      const double dx = mimg(m.x[j] - xi, m.box[0], ix);
      const double dy = mimg(m.y[j] - yi, m.box[1], iy);
      const double dz = mimg(m.z[j] - zi, m.box[2], iz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= rc2) continue;
      rho += spline_val(m.tab.sp[3 + m.types[j]], r2 * rsqrt_nr(r2), m.err);
    }
  }
  m.rho[i] = rho;
  double t;
  const int ti = m.types[i];
  const int q = spline_locate(m.tab.sp[5 + ti], rho, t, m.err);
  m.dFp[i] = spline_der_at(m.tab.sp[5 + ti], q, t);
  if (MIXED) m.dFp32[i] = (float)m.dFp[i];
  m.dF[i] = spline_val_at(m.tab.sp[6], q, t) - spline_val_at(m.tab.sp[5], q, t);
}

// interval and offset of r on a table grid when 0 <= r < r_c <= the grid's
// end is already known (no range test)
__device__ __forceinline__ int locate_in(const Spline& s, double r, double& t) {
  const double u = r * s.inv_h;
  int j = (int)u;
  j = j < s.n_int - 1 ? j : s.n_int - 1;
  t = u - (double)j;
  return j;
}

// FP64 form on the half list (each pair once, j > i): rho_i and rho_j both
// receive the pair's density (atomic adds into rho, zeroed before); with one
// density function (same_dens) one table value serves both ends.
__global__ void k_md_rho_half(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int* row = m.nbr_h + i * m.K;
  const int cnt = m.cnt_h[i];
  const double xi = m.x[i], yi = m.y[i], zi = m.z[i];
  const double ix = 1.0 / m.box[0], iy = 1.0 / m.box[1], iz = 1.0 / m.box[2];
  const double rc2 = m.rc * m.rc;
  const int ti = m.types[i];
  double rho = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int j = row[k];
    const double dx = mimg(m.x[j] - xi, m.box[0], ix);
    const double dy = mimg(m.y[j] - yi, m.box[1], iy);
    const double dz = mimg(m.z[j] - zi, m.box[2], iz);
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2) continue;
    const double r = r2 * rsqrt_nr(r2);
    const int tj = m.types[j];
    double t;
    const int q = locate_in(m.tab.sp[3], r, t);
    const double fj = spline_val_at(m.tab.sp[3 + tj], q, t);  // density of j at i
    const double fi = m.same_dens ? fj : spline_val_at(m.tab.sp[3 + ti], q, t);
    rho += fj;
    atomicAdd(m.rho + j, fi);
  }
  atomicAdd(m.rho + i, rho);
}

// mixed form on the half list: FP32 geometry and tables, FP64 sums
__global__ void k_md_rho_half32(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int* row = m.nbr_h + i * m.K;
  const int cnt = m.cnt_h[i];
  const uint32_t uxi = m.ux[i], uyi = m.uy[i], uzi = m.uz[i];
  const float rc2 = (float)(m.rc * m.rc);
  const int ti = m.types[i];
  double rho = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int j = row[k];
    const float dx = fix_diff(m.ux[j], uxi, m.ul[0]);
    const float dy = fix_diff(m.uy[j], uyi, m.ul[1]);
    const float dz = fix_diff(m.uz[j], uzi, m.ul[2]);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2) continue;
    const int tj = m.types[j];
    float t;
    const int q = spline32_locate(m.tab32.sp[3], sqrtf(r2), t, m.err);
    const float fj = spline32_val_at(m.tab32.sp[3 + tj], q, t);
    const float fi = m.same_dens ? fj : spline32_val_at(m.tab32.sp[3 + ti], q, t);
    rho += (double)fj;
    atomicAdd(m.rho + j, (double)fi);
  }
  atomicAdd(m.rho + i, rho);
}

__global__ void k_md_force_half32(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int* row = m.nbr_h + i * m.K;
  const int cnt = m.cnt_h[i];
  const uint32_t uxi = m.ux[i], uyi = m.uy[i], uzi = m.uz[i];
  const int ti = m.types[i];
  const float Fi = m.dFp32[i];
  const float rc2 = (float)(m.rc * m.rc);
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int j = row[k];
    const float dx = fix_diff(m.ux[j], uxi, m.ul[0]);
    const float dy = fix_diff(m.uy[j], uyi, m.ul[1]);
    const float dz = fix_diff(m.uz[j], uzi, m.ul[2]);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2) continue;
    const float ir = rsqrtf(r2);
    const int tj = m.types[j];
    float t;
    const int q = spline32_locate(m.tab32.sp[0], r2 * ir, t, m.err);
    const float Fj = m.dFp32[j];
    float g;
    if (m.same_dens) {
      g = fmaf(Fi + Fj, spline32_dval_at(m.tab32.dsp[3], q, t), spline32_dval_at(m.tab32.dsp[ti + tj], q, t));
    } else {
      g = fmaf(Fj, spline32_dval_at(m.tab32.dsp[3 + ti], q, t),
               fmaf(Fi, spline32_dval_at(m.tab32.dsp[3 + tj], q, t), spline32_dval_at(m.tab32.dsp[ti + tj], q, t)));
    }
    const float gr = g * ir;
    const double gx = (double)(gr * dx), gy = (double)(gr * dy), gz = (double)(gr * dz);
    fx += gx;
    fy += gy;
    fz += gz;
    atomicAdd(m.fx + j, -gx);
    atomicAdd(m.fy + j, -gy);
    atomicAdd(m.fz + j, -gz);
  }
  if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(m.err, ERRF_NONFINITE);
  atomicAdd(m.fx + i, fx);
  atomicAdd(m.fy + i, fy);
  atomicAdd(m.fz + i, fz);
}

// F'(rho_i) and F_B(rho_i) - F_A(rho_i) once rho is complete
__global__ void k_md_embed(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const double rho = m.rho[i];
  double t;
  const int ti = m.types[i];
  const int q = spline_locate(m.tab.sp[5 + ti], rho, t, m.err);
  m.dFp[i] = spline_der_at(m.tab.sp[5 + ti], q, t);
  m.dF[i] = spline_val_at(m.tab.sp[6], q, t) - spline_val_at(m.tab.sp[5], q, t);
  if (m.mixed) m.dFp32[i] = (float)m.dFp[i];
}

// warp sum of the per-thread virial terms, one atomic per warp (every lane
// of the warp reaches this point)
__device__ __forceinline__ void add_virial(const MdArgs& m, double vir) {
  if (!m.vir) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vir += __shfl_xor_sync(0xffffffffu, vir, o);
  if ((threadIdx.x & 31) == 0 && vir != 0.0) atomicAdd(m.vir, vir);
}

// FP64 forces on the half list: F_i += g (x_j - x_i) / r, F_j -= the same,
// g = phi'_{ti tj} + F'_i f'_{tj} + F'_j f'_{ti} (one density derivative
// when same_dens); force arrays zeroed before.  The virial term of the
// pair, r_ij . F_ij = -g r, goes to *m.vir when it is set.
__device__ __forceinline__ void force_half_row(const MdArgs& m, long long i, double& vir) {
  const int* row = m.nbr_h + i * m.K;
  const int cnt = m.cnt_h[i];
  const double xi = m.x[i], yi = m.y[i], zi = m.z[i];
  const int ti = m.types[i];
  const double Fi = m.dFp[i];
  const double ix = 1.0 / m.box[0], iy = 1.0 / m.box[1], iz = 1.0 / m.box[2];
  const double rc2 = m.rc * m.rc;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int j = row[k];
    const double dx = mimg(m.x[j] - xi, m.box[0], ix);
    const double dy = mimg(m.y[j] - yi, m.box[1], iy);
    const double dz = mimg(m.z[j] - zi, m.box[2], iz);
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2) continue;
    const double ir = rsqrt_nr(r2);
    const int tj = m.types[j];
    double t;
    const int q = locate_in(m.tab.sp[0], r2 * ir, t);
    const double Fj = m.dFp[j];
    double g;
    if (m.same_dens) {
      g = fma(Fi + Fj, spline_dval_at(m.tab.dsp[3], q, t), spline_dval_at(m.tab.dsp[ti + tj], q, t));
    } else {
      g = fma(Fj, spline_dval_at(m.tab.dsp[3 + ti], q, t),
              fma(Fi, spline_dval_at(m.tab.dsp[3 + tj], q, t), spline_dval_at(m.tab.dsp[ti + tj], q, t)));
    }
    const double gr = g * ir;
    const double gx = gr * dx, gy = gr * dy, gz = gr * dz;
    fx += gx;
    fy += gy;
    fz += gz;
    vir -= gr * r2;
    atomicAdd(m.fx + j, -gx);
    atomicAdd(m.fy + j, -gy);
    atomicAdd(m.fz + j, -gz);
  }
  if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(m.err, ERRF_NONFINITE);
  atomicAdd(m.fx + i, fx);
  atomicAdd(m.fy + i, fy);
  atomicAdd(m.fz + i, fz);
}

__global__ void k_md_force_half(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double vir = 0.0;
  if (i < m.N) force_half_row(m, i, vir);
  add_virial(m, vir);
}

template <bool MIXED>
__device__ __forceinline__ void force_row(const MdArgs& m, long long i, double& vir) {
  const int* row = m.nbr + i * m.K;
  const int cnt = m.nbr_cnt[i];
  const double xi = m.x[i], yi = m.y[i], zi = m.z[i];
  const int ti = m.types[i];
  const double Fi = m.dFp[i];
  const double ix = 1.0 / m.box[0], iy = 1.0 / m.box[1], iz = 1.0 / m.box[2];
  const double rc2 = m.rc * m.rc;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  const float Fi32 = (float)Fi;
  const uint32_t uxi = MIXED ? m.ux[i] : 0u, uyi = MIXED ? m.uy[i] : 0u, uzi = MIXED ? m.uz[i] : 0u;
  for (int k = 0; k < cnt; ++k) {
    const int j = row[k];
    if constexpr (MIXED) {
      // FP32 geometry and table derivatives, FP64 force sums
      const float dx = fix_diff(m.ux[j], uxi, m.ul[0]);
      const float dy = fix_diff(m.uy[j], uyi, m.ul[1]);
      const float dz = fix_diff(m.uz[j], uzi, m.ul[2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= (float)rc2) continue;
      const float ir = rsqrtf(r2);
      const int tj = m.types[j];
      float t;
      const int q = spline32_locate(m.tab32.sp[0], r2 * ir, t, m.err);
      const float g = fmaf(m.dFp32[j], spline32_dval_at(m.tab32.dsp[3 + ti], q, t),
                           fmaf(Fi32, spline32_dval_at(m.tab32.dsp[3 + tj], q, t),
                                spline32_dval_at(m.tab32.dsp[ti + tj], q, t)));
      const float gr = g * ir;
      fx += (double)(gr * dx);
      fy += (double)(gr * dy);
      fz += (double)(gr * dz);
      continue;
    }
    const double dx = mimg(m.x[j] - xi, m.box[0], ix);
    const double dy = mimg(m.y[j] - yi, m.box[1], iy);
    const double dz = mimg(m.z[j] - zi, m.box[2], iz);
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2) continue;
    const double ir = rsqrt_nr(r2);
    const int tj = m.types[j];
    double t;
    const int q = spline_locate(m.tab.sp[0], r2 * ir, t, m.err);
    const double g = fma(m.dFp[j], spline_dval_at(m.tab.dsp[3 + ti], q, t),
                         fma(Fi, spline_dval_at(m.tab.dsp[3 + tj], q, t),
                             spline_dval_at(m.tab.dsp[ti + tj], q, t)));
    const double gr = g * ir;
    fx = fma(gr, dx, fx);
    fy = fma(gr, dy, fy);
    fz = fma(gr, dz, fz);
    vir -= 0.5 * gr * r2;  // each pair is seen from both ends
  }
  if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(m.err, ERRF_NONFINITE);
  m.fx[i] = fx;
  m.fy[i] = fy;
  m.fz[i] = fz;
}

template <bool MIXED>
__global__ void k_md_force(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double vir = 0.0;
  if (i < m.N) force_row<MIXED>(m, i, vir);
  if (!MIXED) add_virial(m, vir);
}

__device__ __forceinline__ double wrap_box(double v, double L) {
  double w = v - L * floor(v / L);
  if (w >= L) w -= L;
  if (w < 0.0) w = 0.0;
  return w;
}

// Box-Muller: two standard normals from two uniforms
__device__ __forceinline__ void normals(uint4 w, double& z0, double& z1) {
  const double u1 = (double)top53(w.x, w.y) * 0x1p-53;
  const double u2 = (double)top53(w.z, w.w) * 0x1p-53;
  const double rr = sqrt(-2.0 * log(1.0 - u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = rr * c;
  z1 = rr * s;
}

__global__ void k_md_first_half(MdArgs m, long long step) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const int ti = m.types[i];
  const double im = FTM / m.mass[ti];
  const double h = 0.5 * m.dt;
  double vx = m.vx[i] + h * m.fx[i] * im;
  double vy = m.vy[i] + h * m.fy[i] * im;
  double vz = m.vz[i] + h * m.fz[i] * im;
  double x = m.x[i] + h * vx, y = m.y[i] + h * vy, z = m.z[i] + h * vz;
  if (m.c2 > 0.0) {
    const double sig = m.c2 * sqrt(m.kT * im);
    const uint4 c0 = make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)i, TAG_NOISE0);
    const uint4 c1 = make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)i, TAG_NOISE1);
    double z0, z1, z2, z3;
    normals(philox4x32_10(c0, m.key), z0, z1);
    normals(philox4x32_10(c1, m.key), z2, z3);
    vx = m.c1 * vx + sig * z0;
    vy = m.c1 * vy + sig * z1;
    vz = m.c1 * vz + sig * z2;
  }
  x = wrap_box(x + h * vx, m.box[0]);
  y = wrap_box(y + h * vy, m.box[1]);
  z = wrap_box(z + h * vz, m.box[2]);
  m.vx[i] = vx;
  m.vy[i] = vy;
  m.vz[i] = vz;
  m.x[i] = x;
  m.y[i] = y;
  m.z[i] = z;
  const double dx = mimg(x - m.x0[i], m.box[0], 1.0 / m.box[0]);
  const double dy = mimg(y - m.y0[i], m.box[1], 1.0 / m.box[1]);
  const double dz = mimg(z - m.z0[i], m.box[2], 1.0 / m.box[2]);
  const double d2 = dx * dx + dy * dy + dz * dz;
  // non-negative doubles order like their bit patterns
  atomicMax(m.max_disp2_bits, (unsigned long long)__double_as_longlong(d2));
}

__global__ void k_md_second_half(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const double im = FTM / m.mass[m.types[i]];
  const double h = 0.5 * m.dt;
  m.vx[i] += h * m.fx[i] * im;
  m.vy[i] += h * m.fy[i] * im;
  m.vz[i] += h * m.fz[i] * im;
}

__global__ void k_md_snapshot(MdArgs m) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *m.max_disp2_bits = 0ull;
  if (i >= m.N) return;
  m.x0[i] = m.x[i];
  m.y0[i] = m.y[i];
  m.z0[i] = m.z[i];
}

// Nose-Hoover / MTK sub-flows (the step's scalars are integrated on the
// host): v <- v s e1 + (F/m) he2, and r <- wrap(r e1 + v e2dt) in the
// current box with the displacement from the last neighbour build measured
// against the snapshot scaled by lam = L / L_build.
__global__ void k_nh_kick(MdArgs m, double s, double e1, double he2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const double im = FTM / m.mass[m.types[i]];
  const double se = s * e1, ke = he2 * im;
  m.vx[i] = fma(m.vx[i], se, m.fx[i] * ke);
  m.vy[i] = fma(m.vy[i], se, m.fy[i] * ke);
  m.vz[i] = fma(m.vz[i], se, m.fz[i] * ke);
}

__global__ void k_nh_drift(MdArgs m, double e1, double e2dt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const double x = wrap_box(fma(m.x[i], e1, m.vx[i] * e2dt), m.box[0]);
  const double y = wrap_box(fma(m.y[i], e1, m.vy[i] * e2dt), m.box[1]);
  const double z = wrap_box(fma(m.z[i], e1, m.vz[i] * e2dt), m.box[2]);
  m.x[i] = x;
  m.y[i] = y;
  m.z[i] = z;
  const double dx = mimg(x - m.x0[i] * m.lam, m.box[0], 1.0 / m.box[0]);
  const double dy = mimg(y - m.y0[i] * m.lam, m.box[1], 1.0 / m.box[1]);
  const double dz = mimg(z - m.z0[i] * m.lam, m.box[2], 1.0 / m.box[2]);
  atomicMax(m.max_disp2_bits, (unsigned long long)__double_as_longlong(dx * dx + dy * dy + dz * dz));
}

// positions x0 + alpha d (conjugate-gradient line search), wrapped, with the
// displacement check of the MD step
__global__ void k_cg_place(MdArgs m, const double* x0, const double* d, double alpha) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.N) return;
  const long long N = m.N;
  const double x = wrap_box(fma(alpha, d[i], x0[i]), m.box[0]);
  const double y = wrap_box(fma(alpha, d[N + i], x0[N + i]), m.box[1]);
  const double z = wrap_box(fma(alpha, d[2 * N + i], x0[2 * N + i]), m.box[2]);
  m.x[i] = x;
  m.y[i] = y;
  m.z[i] = z;
  const double dx = mimg(x - m.x0[i], m.box[0], 1.0 / m.box[0]);
  const double dy = mimg(y - m.y0[i], m.box[1], 1.0 / m.box[1]);
  const double dz = mimg(z - m.z0[i], m.box[2], 1.0 / m.box[2]);
  atomicMax(m.max_disp2_bits, (unsigned long long)__double_as_longlong(dx * dx + dy * dy + dz * dz));
}

constexpr int DOT_BLOCK = 256;
int dot_blocks(long long n) { return (int)((n + DOT_BLOCK - 1) / DOT_BLOCK); }

// block partials of sum_k a[k] b[k], k < n
__global__ void __launch_bounds__(DOT_BLOCK) k_dot(const double* a, const double* b, long long n, double* part) {
  const long long k = (long long)blockIdx.x * DOT_BLOCK + threadIdx.x;
  double v = k < n ? a[k] * b[k] : 0.0;
  __shared__ double sh[DOT_BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < DOT_BLOCK / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// max over atoms of |v_i|^2 for a 3N SoA vector, as double bits
__global__ void k_max_norm2(const double* a, long long N, unsigned long long* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double v = a[i] * a[i] + a[N + i] * a[N + i] + a[2 * N + i] * a[2 * N + i];
  atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

constexpr int KE_BLOCK = 256;
int kinetic_blocks(long long N) { return (int)((N + KE_BLOCK - 1) / KE_BLOCK); }

__global__ void __launch_bounds__(KE_BLOCK) k_kinetic(MdArgs m, double* part) {
  const long long i = (long long)blockIdx.x * KE_BLOCK + threadIdx.x;
  double e = 0.0;
  if (i < m.N) {
    const double v2 = m.vx[i] * m.vx[i] + m.vy[i] * m.vy[i] + m.vz[i] * m.vz[i];
    e = 0.5 * m.mass[m.types[i]] / FTM * v2;
  }
  __shared__ double sh[KE_BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < KE_BLOCK / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

static unsigned grid_of(long long N) { return (unsigned)((N + 127) / 128); }

__global__ void k_fix_positions(long long N, const double* x, const double* y, const double* z, double sx, double sy,
                                double sz, uint32_t* ux, uint32_t* uy, uint32_t* uz) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // x 2^32 / L rounded to an integer, reduced mod 2^32 (two's complement
  // wrap of a negative or >= 2^32 value is the periodic reduction)
  ux[i] = (uint32_t)(unsigned long long)llrint(x[i] * sx);
  uy[i] = (uint32_t)(unsigned long long)llrint(y[i] * sy);
  uz[i] = (uint32_t)(unsigned long long)llrint(z[i] * sz);
}

void launch_fix_positions(long long N, const double* x, const double* y, const double* z, const double box[3],
                          uint32_t* ux, uint32_t* uy, uint32_t* uz, cudaStream_t st) {
  if (N < 1 || !ux || !uy || !uz) return;
  const double two32 = 4294967296.0;
  k_fix_positions<<<grid_of(N), 128, 0, st>>>(N, x, y, z, two32 / box[0], two32 / box[1], two32 / box[2], ux, uy,
                                              uz);
}

void launch_md_rho(const MdArgs& m, cudaStream_t st) {
  if (m.mixed) launch_fix_positions(m.N, m.x, m.y, m.z, m.box, m.ux, m.uy, m.uz, st);
  if (m.nbr_h) {
    cudaMemsetAsync(m.rho, 0, sizeof(double) * m.N, st);
    if (m.mixed) k_md_rho_half32<<<grid_of(m.N), 128, 0, st>>>(m);
    else k_md_rho_half<<<grid_of(m.N), 128, 0, st>>>(m);
    k_md_embed<<<grid_of(m.N), 128, 0, st>>>(m);
  } else if (m.mixed) {
    k_md_rho<true><<<grid_of(m.N), 128, 0, st>>>(m);
  } else {
    k_md_rho<false><<<grid_of(m.N), 128, 0, st>>>(m);
  }
}
void launch_md_force(const MdArgs& m, cudaStream_t st) {
  if (m.nbr_h) {
    cudaMemsetAsync(m.fx, 0, sizeof(double) * m.N, st);
    cudaMemsetAsync(m.fy, 0, sizeof(double) * m.N, st);
    cudaMemsetAsync(m.fz, 0, sizeof(double) * m.N, st);
    if (m.mixed) k_md_force_half32<<<grid_of(m.N), 128, 0, st>>>(m);
    else k_md_force_half<<<grid_of(m.N), 128, 0, st>>>(m);
  } else if (m.mixed) {
    k_md_force<true><<<grid_of(m.N), 128, 0, st>>>(m);
  } else {
    k_md_force<false><<<grid_of(m.N), 128, 0, st>>>(m);
  }
}
void launch_md_first_half(const MdArgs& m, long long step, cudaStream_t st) {
  k_md_first_half<<<grid_of(m.N), 128, 0, st>>>(m, step);
}
void launch_md_second_half(const MdArgs& m, cudaStream_t st) {
  k_md_second_half<<<grid_of(m.N), 128, 0, st>>>(m);
}
void launch_md_snapshot(const MdArgs& m, cudaStream_t st) { k_md_snapshot<<<grid_of(m.N), 128, 0, st>>>(m); }
void launch_nh_kick(const MdArgs& m, double s, double e1, double he2, cudaStream_t st) {
  k_nh_kick<<<grid_of(m.N), 128, 0, st>>>(m, s, e1, he2);
}
void launch_nh_drift(const MdArgs& m, double e1, double e2dt, cudaStream_t st) {
  k_nh_drift<<<grid_of(m.N), 128, 0, st>>>(m, e1, e2dt);
}
void launch_cg_place(const MdArgs& m, const double* x0, const double* d, double alpha, cudaStream_t st) {
  k_cg_place<<<grid_of(m.N), 128, 0, st>>>(m, x0, d, alpha);
}
void launch_dot(const double* a, const double* b, long long n, double* part, cudaStream_t st) {
  k_dot<<<dot_blocks(n), DOT_BLOCK, 0, st>>>(a, b, n, part);
}
void launch_max_norm2(const double* a, long long N, unsigned long long* out, cudaStream_t st) {
  k_max_norm2<<<grid_of(N), 128, 0, st>>>(a, N, out);
}
__global__ void k_axpby(double* d, const double* g, double beta, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) d[k] = fma(beta, d[k], g[k]);
}
void launch_axpby(double* d, const double* g, double beta, long long n, cudaStream_t st) {
  k_axpby<<<grid_of(n), 128, 0, st>>>(d, g, beta, n);
}
void launch_kinetic(const MdArgs& m, double* part, cudaStream_t st) {
  k_kinetic<<<kinetic_blocks(m.N), KE_BLOCK, 0, st>>>(m, part);
}

}  // namespace vcsgc
