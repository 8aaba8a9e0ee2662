// Multicomponent form of the colour step: K <= 4 species on a rigid BCC
// lattice, one variance constraint per solute species.  Device structures
// shared by kernels_multi.cu and vcsgc_multi_capi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace vcsgc {

constexpr int MK_MAX = 4;         // species
constexpr int MK_MAX_SH = 8;      // neighbour shells
constexpr int MK_MAX_OFF = 96;    // neighbour offsets (5 BCC shells: 58)
constexpr int MK_BLOCK = 128;
constexpr uint32_t TAG_SPECIES = 6u;  // (step, domain rank): the proposed species

// Per-replica parameters: index alpha = 0..K-1, entry 0 (the solvent) zero.
struct MRepParams {
  double beta;
  double kappa_p[MK_MAX];
  double n0[MK_MAX];
  double dmu0[MK_MAX];  // phi_alpha + 2 kappa_p,alpha n0_alpha
  double phi[MK_MAX];
  uint2 key;
};

struct MRepState {
  long long cnt[MK_MAX];
  long long step;
  double energy;
  long long trials, local_acc, global_trials, global_acc, flips, near_ties, steps;
  double sum_c[MK_MAX], sum_c2[MK_MAX];
};

// accumulator of one colour step (two per replica, by step parity)
struct MStepAcc {
  int dn[MK_MAX];
  int nacc;
  int ties;
  unsigned done;
  int accept;
  double sum_de;
};

struct MultiArgs {
  int R, K;
  int nx, ny, nz;
  long long N;
  // sublattice schedule: colour ((pz qy + py) qx + px) 2 + b
  int qx, qy, qz;
  int nxq, nyq, nzq;   // n / q per axis
  int n_colours;
  int D;               // trials per colour step (sites of one colour)
  // neighbour offsets in half-lattice units, sorted by shell
  int n_off, n_sh;
  int4 off[MK_MAX_OFF];  // (hx, hy, hz, shell)
  // shell tables: V[(s K + a) K + b] = phi_ab(r_s), Fd[s K + a] = f_a(r_s)
  const double* V;
  const double* Fd;
  int reembed;          // f_a(r_s) differs between species at some shell
  Spline embed[MK_MAX];
  uint8_t* types;       // [R][N]
  double* rho;          // [R][N]
  const MRepParams* rp;
  MRepState* rs;
  MStepAcc* acc;        // [R][2]
  int2* pend;           // [R][D] (site, new species) of the local accepts
  unsigned* err;
};

// site index of trial d of colour c (ascending site index within a colour)
__device__ __forceinline__ int multi_site(const MultiArgs& a, int c, int d) {
  const int b = c & 1;
  const int pc = c >> 1;
  const int px = pc % a.qx, py = (pc / a.qx) % a.qy, pz = pc / (a.qx * a.qy);
  const int kx = d % a.nxq, ky = (d / a.nxq) % a.nyq, kz = d / (a.nxq * a.nyq);
  const int cx = px + a.qx * kx, cy = py + a.qy * ky, cz = pz + a.qz * kz;
  return ((cz * a.ny + cy) * a.nx + cx) * 2 + b;
}

// neighbour of site i along half-lattice offset h (periodic)
__device__ __forceinline__ int multi_nbr(const MultiArgs& a, int i, int4 h) {
  const int b = i & 1;
  const int cell = i >> 1;
  const int cx = cell % a.nx, cy = (cell / a.nx) % a.ny, cz = cell / (a.nx * a.ny);
  const int qx = 2 * cx + b + h.x, qy = 2 * cy + b + h.y, qz = 2 * cz + b + h.z;
  const int bb = qx & 1;
  int X = (qx - bb) >> 1, Y = (qy - bb) >> 1, Z = (qz - bb) >> 1;
  X += X < 0 ? a.nx : (X >= a.nx ? -a.nx : 0);
  Y += Y < 0 ? a.ny : (Y >= a.ny ? -a.ny : 0);
  Z += Z < 0 ? a.nz : (Z >= a.nz ? -a.nz : 0);
  return ((Z * a.ny + Y) * a.nx + X) * 2 + bb;
}

void launch_multi_shell_tables(const Spline* pair, const Spline* dens, int K, const double* r_s, int n_sh,
                               double* V, double* Fd, unsigned* err, cudaStream_t st);
void launch_multi_rho(const MultiArgs& a, int r0, int nrep, cudaStream_t st);
// per-site energies summed into block partials part[r][blocks]
int multi_energy_blocks(long long N);
void launch_multi_energy(const MultiArgs& a, int r0, int nrep, double* part, cudaStream_t st);
void launch_multi_delta_e(const MultiArgs& a, int r, const long long* sites, const uint8_t* to, int n,
                          double* out, cudaStream_t st);
void launch_multi_step(const MultiArgs& a, cudaStream_t st);

}  // namespace vcsgc
