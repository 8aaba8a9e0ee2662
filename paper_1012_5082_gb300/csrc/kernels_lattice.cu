// kernels_lattice.cu -- fused colour step for the rigid BCC lattice with one
// density function (the production form of the parallel VC-SGC sweep,
// Sec. III B 2 of Sadigh et al.).
//
// Species are bit-packed: each periodic x-row (cy, cz) of a replica holds
// 2 nx sites as bits p = 4 + H (H = 2 cx + b is the half-lattice x
// coordinate) plus 4 halo bits on each side that mirror the far end of the
// row, in 64-bit words whose low half carries 32 species bits and whose high
// half carries the matching "pending flip" bits.  Every neighbour of a site
// lies in one of 13 rows at half-lattice x offsets -3..3, so a trial reads a
// 7-bit window from each row and counts the B neighbours of each shell with
// popc against per-row shell masks (dE of the rigid lattice is affine in
// those counts).  Lanes of a warp are consecutive trial sites of one row of
// the colour, so their windows come from the same words.
//
// One kernel per colour step k:
//   1. every block derives the global decision G_{k-1} of the previous step
//      (its dn was reduced by the previous launch);
//   2. each thread commits its own pending flip of step k-1 with one atomic
//      XOR that clears the pending bit and flips the species bit if G_{k-1};
//   3. block (0, r) finalises step k-1 for replica r (n, energy, counters);
//   4. the thread proposes trial d of step k: it reads effective species
//      t ^ (pending & G_{k-1}), so it never waits for other blocks' commits;
//      an accepted move sets its pending bit(s) and joins the dn reduction.
// Same-colour sites are > 2 r_c apart, so no trial of step k reads a bit that
// another trial of step k sets; a pending bit is only ever read under the
// decision of its own step.
#include "common.cuh"
#include "kernels.h"

namespace vcsgc {

__device__ __forceinline__ void decode_site(const LatArgs& a, int i, int& X, int& Y, int& Z, int& b) {
  b = i & 1;
  const int cell = i >> 1;
  X = cell % a.nx;
  const int q = cell / a.nx;
  Y = q % a.ny;
  Z = q / a.ny;
}

__device__ __forceinline__ unsigned long long* row_ptr(const LatArgs& a, int r, int Y, int Z) {
  return a.bits + (long long)r * a.rep_words + ((long long)Z * a.ny + Y) * a.W;
}

// effective 32 species bits of a word under the pending decision mask gm
__device__ __forceinline__ uint32_t eff32(unsigned long long w, uint32_t gm) {
  return (uint32_t)w ^ ((uint32_t)(w >> 32) & gm);
}

// window of half-lattice x offsets -hmax..hmax around half-coordinate H
__device__ __forceinline__ uint32_t window(const unsigned long long* row, int H, int hmax, uint32_t gm) {
  const int q = LAT_HALO + H - hmax;
  const int wq = q >> 5;
  const unsigned long long w0 = __ldcg(row + wq);
  const unsigned long long w1 = __ldcg(row + wq + 1);
  return __funnelshift_r(eff32(w0, gm), eff32(w1, gm), q & 31);
}

__device__ __forceinline__ int own_bit(const unsigned long long* row, int H, uint32_t gm) {
  const int p = LAT_HALO + H;
  return (eff32(__ldcg(row + (p >> 5)), gm) >> (p & 31)) & 1;
}

// the (up to two) bit copies of site H in its row: main p = 4 + H, halo
// p - 2 nx (for H >= 2 nx - 4) and p + 2 nx (for H < 4)
__device__ __forceinline__ void xor_copies(const LatArgs& a, unsigned long long* row, int H,
                                           bool flip_species, bool flip_pending) {
  int pos[3];
  int n = 0;
  pos[n++] = LAT_HALO + H;
  if (H >= 2 * a.nx - LAT_HALO) pos[n++] = LAT_HALO + H - 2 * a.nx;
  if (H < LAT_HALO) pos[n++] = LAT_HALO + H + 2 * a.nx;
  for (int q = 0; q < n; ++q) {
    const int p = pos[q];
    unsigned long long m = 0;
    if (flip_species) m |= 1ull << (p & 31);
    if (flip_pending) m |= 1ull << (32 + (p & 31));
    atomicXor(row + (p >> 5), m);
  }
}

// dE of flipping site i of replica r on the effective state
__device__ __forceinline__ double lattice_delta_e(const LatArgs& a, int r, int i, uint32_t gm, int& t) {
  int X, Y, Z, b;
  decode_site(a, i, X, Y, Z, b);
  const int H = 2 * X + b;
  int cnt[LAT_MAX_SH];
#pragma unroll
  for (int s = 0; s < LAT_MAX_SH; ++s) cnt[s] = 0;
  const int nr = a.n_rows[b];
  for (int q = 0; q < nr; ++q) {
    const LatRow& rw = a.rows[b][q];
    int yy = Y + rw.dy, zz = Z + rw.dz;
    yy = yy < 0 ? yy + a.ny : (yy >= a.ny ? yy - a.ny : yy);
    zz = zz < 0 ? zz + a.nz : (zz >= a.nz ? zz - a.nz : zz);
    const uint32_t win = window(row_ptr(a, r, yy, zz), H, a.hmax, gm);
#pragma unroll
    for (int s = 0; s < LAT_MAX_SH; ++s) cnt[s] += __popc(win & rw.mask[s]);
  }
  t = own_bit(row_ptr(a, r, Y, Z), H, gm);
  double de = a.C;
#pragma unroll
  for (int s = 0; s < LAT_MAX_SH; ++s) de = fma((double)cnt[s], a.G[s], de);
  const double dfi = a.dF[i];
  de += dfi;
  return t ? -de : de;
}

__device__ __forceinline__ int lat_colour(const LatArgs& a, uint2 key, long long step, uint64_t* ug53) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0xFFFFFFFFu, TAG_STEP), key);
  if (ug53) *ug53 = top53(w.z, w.w);
  return (int)below64(w.x, w.y, (uint64_t)a.n_colours);
}

template <bool PROPOSE>
__global__ void __launch_bounds__(LAT_BLOCK) k_lattice_step(LatArgs a, int j) {
  const int r = blockIdx.y;
  const long long k = a.ctl->base_step + j;
  const long long kp = k - 1;
  const RepParams p = a.rp[r];
  const int d = blockIdx.x * LAT_BLOCK + threadIdx.x;

  // 1. global decision of step k-1
  bool Gp = false;
  int tie_p = 0, dnp = 0, naccp = 0, cp = 0;
  long long np = 0;
  if (kp >= 0) {
    const StepAcc* Ap = a.acc + r * 3 + (int)(kp % 3);
    naccp = *(volatile const int*)&Ap->nacc;
    dnp = *(volatile const int*)&Ap->dn;
    np = a.n_start[r * 2 + (int)(kp & 1)];
    uint64_t ug53;
    cp = lat_colour(a, p.key, kp, &ug53);
    if (naccp > 0) {
      const double Y = p.beta * p.kappa_p * (double)dnp * ((double)dnp + 2.0 * ((double)np - p.n0));
      Gp = metropolis(Y, ug53, &tie_p);
    }
  }
  const uint32_t gm = Gp ? 0xFFFFFFFFu : 0u;

  // 2. commit this thread's pending flip of step k-1
  if (d < a.dmax) {
    int* slot = a.pend + (long long)r * a.dmax + d;
    const int ps = *slot;
    if (ps >= 0) {
      int X, Y, Z, b;
      decode_site(a, ps, X, Y, Z, b);
      xor_copies(a, row_ptr(a, r, Y, Z), 2 * X + b, Gp, true);
      *slot = -1;
    }
  }

  // 3. finalise step k-1 and clear the accumulator of step k+1
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    RepState* S = a.rs + r;
    if (kp >= 0 && S->fin_step < kp) {
      const StepAcc* Ap = a.acc + r * 3 + (int)(kp % 3);
      const int D = a.col_start[cp + 1] - a.col_start[cp];
      S->trials += D;
      S->local_acc += naccp;
      S->near_ties += *(volatile const int*)&Ap->ties + tie_p;
      long long nn = np;
      if (naccp > 0) {
        S->global_trials += 1;
        if (Gp) {
          S->global_acc += 1;
          S->flips += naccp;
          nn = np + dnp;
          S->energy += *(volatile const double*)&Ap->sum_de;
        }
      }
      S->n = nn;
      a.n_start[r * 2 + (int)(k & 1)] = nn;
      const double cc = (double)nn / (double)a.N;
      S->sum_c += cc;
      S->sum_c2 += cc * cc;
      S->steps += 1;
      S->step = k;
      S->fin_step = kp;
    }
    if (PROPOSE) {
      StepAcc* An = a.acc + r * 3 + (int)((k + 1) % 3);
      An->dn = 0;
      An->nacc = 0;
      An->sum_de = 0.0;
      An->ties = 0;
    }
  }
  if (!PROPOSE) return;

  // 4. propose trial d of step k
  const int c = lat_colour(a, p.key, k, nullptr);
  const int g0 = a.col_start[c];
  const int D = a.col_start[c + 1] - g0;
  int dn = 0, acc = 0, tie = 0;
  double sde = 0.0;
  if (d < D) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)d, TAG_TRIAL), p.key);
    int site;
    if (a.sublattice) {
      // colour c = (((pz qy + py) qx + px) 2 + b); trial d runs over the
      // colour's sites in ascending index: d = (kz nyq + ky) nxq + kx
      const int b = c & 1;
      const int pc = c >> 1;
      const int px = pc % a.qx, py = (pc / a.qx) % a.qy, pz = pc / (a.qx * a.qy);
      const int nxq = a.nx / a.qx, nyq = a.ny / a.qy;
      const int kx = d % nxq, ky = (d / nxq) % nyq, kz = d / (nxq * nyq);
      const int X = px + a.qx * kx, Y = py + a.qy * ky, Z = pz + a.qz * kz;
      site = ((Z * a.ny + Y) * a.nx + X) * 2 + b;
    } else {
      const int g = g0 + d;
      const int base = a.dom_start[g];
      const int size = a.dom_start[g + 1] - base;
      site = a.dom_sites[base + (int)below64(w.x, w.y, (uint64_t)size)];
    }
    int t;
    const double de = lattice_delta_e(a, r, site, gm, t);
    if (!isfinite(de)) atomicOr(a.err, ERRF_NONFINITE);
    const double sg = t ? -1.0 : 1.0;
    const double X = p.beta * fma(sg, p.dmu0, de);
    if (metropolis(X, top53(w.z, w.w), &tie)) {
      int XX, YY, ZZ, bb;
      decode_site(a, site, XX, YY, ZZ, bb);
      xor_copies(a, row_ptr(a, r, YY, ZZ), 2 * XX + bb, false, true);  // set pending
      a.pend[(long long)r * a.dmax + d] = site;
      acc = 1;
      dn = t ? -1 : 1;
      sde = de;
    }
  }
  // reduction of dn, accepts and sum dE (the paper's allgather of dc_i)
  __shared__ int s_dn[LAT_BLOCK / 32], s_acc[LAT_BLOCK / 32], s_tie[LAT_BLOCK / 32];
  __shared__ double s_de[LAT_BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    tie += __shfl_xor_sync(0xffffffffu, tie, o);
    sde += __shfl_xor_sync(0xffffffffu, sde, o);
  }
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s_dn[wi] = dn; s_acc[wi] = acc; s_tie[wi] = tie; s_de[wi] = sde; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tdn = 0, tacc = 0, ttie = 0;
    double tde = 0.0;
    for (int q = 0; q < LAT_BLOCK / 32; ++q) {
      tdn += s_dn[q];
      tacc += s_acc[q];
      ttie += s_tie[q];
      tde += s_de[q];
    }
    if (tacc) {
      StepAcc* A = a.acc + r * 3 + (int)(k % 3);
      atomicAdd(&A->dn, tdn);
      atomicAdd(&A->nacc, tacc);
      atomicAdd(&A->sum_de, tde);
    }
    if (ttie) atomicAdd(&a.acc[r * 3 + (int)(k % 3)].ties, ttie);
  }
}

__global__ void k_lattice_advance(LatCtl* ctl, int n) { ctl->base_step += n; }

// species bytes <-> bit rows (pending bits cleared)
__global__ void k_lattice_pack(LatArgs a, const uint8_t* types, int r) {
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long long)a.ny * a.nz) return;
  unsigned long long* w = a.bits + (long long)r * a.rep_words + row * a.W;
  const uint8_t* t = types + (long long)r * a.N + row * 2 * a.nx;
  for (int q = 0; q < a.W; ++q) w[q] = 0ull;
  const int L = 2 * a.nx;
  for (int p = 0; p < L + 2 * LAT_HALO; ++p) {
    int H = p - LAT_HALO;
    H = H < 0 ? H + L : (H >= L ? H - L : H);
    if (t[H]) w[p >> 5] |= 1ull << (p & 31);
  }
}

__global__ void k_lattice_unpack(LatArgs a, uint8_t* types, int r) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  int X, Y, Z, b;
  decode_site(a, (int)i, X, Y, Z, b);
  types[(long long)r * a.N + i] = (uint8_t)own_bit(row_ptr(a, r, Y, Z), 2 * X + b, 0u);
}

__global__ void k_lattice_delta_e(LatArgs a, int r, const int* sites, int n, double* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  int t;
  if (q < n) out[q] = lattice_delta_e(a, r, sites[q], 0u, t);
}

void launch_lattice_step(const LatArgs& a, int j, bool propose, cudaStream_t st) {
  const dim3 g((a.dmax + LAT_BLOCK - 1) / LAT_BLOCK, a.R);
  if (propose) k_lattice_step<true><<<g, LAT_BLOCK, 0, st>>>(a, j);
  else k_lattice_step<false><<<g, LAT_BLOCK, 0, st>>>(a, j);
}

void launch_lattice_advance(const LatArgs& a, int n, cudaStream_t st) {
  k_lattice_advance<<<1, 1, 0, st>>>(a.ctl, n);
}

void launch_lattice_pack(const LatArgs& a, const uint8_t* types, int r, cudaStream_t st) {
  const long long rows = (long long)a.ny * a.nz;
  k_lattice_pack<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(a, types, r);
}

void launch_lattice_unpack(const LatArgs& a, uint8_t* types, int r, cudaStream_t st) {
  k_lattice_unpack<<<(unsigned)((a.N + 255) / 256), 256, 0, st>>>(a, types, r);
}

void launch_lattice_delta_e(const LatArgs& a, int r, const int* sites, int n, double* out, cudaStream_t st) {
  if (n > 0) k_lattice_delta_e<<<(n + 127) / 128, 128, 0, st>>>(a, r, sites, n, out);
}

}  // namespace vcsgc
