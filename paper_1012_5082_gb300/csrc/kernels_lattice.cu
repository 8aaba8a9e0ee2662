// kernels_lattice.cu -- fused colour step for rigid BCC lattices with one
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
// One kernel per colour step k, for every replica at once (replicas may have
// different lattice sizes; each has a geometry record):
//   1. one thread per block derives the global decision G_{k-1} of the
//      previous step (its dn was reduced by the previous launch);
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
#include "lattice.cuh"
#include "multi.cuh"

namespace vcsgc {

__device__ __forceinline__ void decode_site(const LatGeom& g, int i, int& X, int& Y, int& Z, int& b) {
  b = i & 1;
  const int cell = i >> 1;
  const int q = fdiv(cell, g.nx, g.rcp_nx);
  X = cell - q * g.nx;
  Z = fdiv(q, g.ny, g.rcp_ny);
  Y = q - Z * g.ny;
}

__device__ __forceinline__ unsigned long long* row_ptr(const LatArgs& a, const LatGeom& g, int Y, int Z) {
  return a.bits + g.bits_off + ((long long)Z * g.ny + Y) * g.W;
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
__device__ __forceinline__ void xor_copies(int nx, unsigned long long* row, int H, bool flip_species,
                                           bool flip_pending) {
  int pos[3];
  int n = 0;
  pos[n++] = LAT_HALO + H;
  if (H >= 2 * nx - LAT_HALO) pos[n++] = LAT_HALO + H - 2 * nx;
  if (H < LAT_HALO) pos[n++] = LAT_HALO + H + 2 * nx;
  for (int q = 0; q < n; ++q) {
    const int p = pos[q];
    unsigned long long m = 0;
    if (flip_species) m |= 1ull << (p & 31);
    if (flip_pending) m |= 1ull << (32 + (p & 31));
    atomicXor(row + (p >> 5), m);
  }
}

// Per-shell B counts of site (X, Y, Z, b) on the effective state and its
// species t.  NR > 0: exactly NR rows per basis, unrolled so that every row
// load is in flight at once; NR = 0: runtime row count.
template <int NS, int NR>
__device__ __forceinline__ void lattice_counts_at(const LatArgs& a, const LatGeom& g, int X, int Y, int Z,
                                                  int b, uint32_t gm, int (&cnt)[NS], int& t) {
  const int H = 2 * X + b;
#pragma unroll
  for (int s = 0; s < NS; ++s) cnt[s] = 0;
  const LatRow* rows = a.rows[b];
  const int nr = NR > 0 ? NR : a.n_rows[b];
#pragma unroll
  for (int q = 0; q < (NR > 0 ? NR : LAT_MAX_ROWS); ++q) {
    if (NR == 0 && q >= nr) break;
    const LatRow& rw = rows[q];
    int yy = Y + rw.dy, zz = Z + rw.dz;
    yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
    zz = zz < 0 ? zz + g.nz : (zz >= g.nz ? zz - g.nz : zz);
    const uint32_t win = window(row_ptr(a, g, yy, zz), H, a.hmax, gm);
#pragma unroll
    for (int s = 0; s < NS; ++s) cnt[s] += __popc(win & rw.mask[s]);
  }
  t = own_bit(row_ptr(a, g, Y, Z), H, gm);
}

// raw words of a site's neighbour rows (w0, w1: the two words holding its
// window in row q) and of its own word
template <int NR>
struct RowWords {
  unsigned long long w0[NR], w1[NR], own;
};

template <int B>
__device__ __forceinline__ void bcc5_rows_load(const LatArgs& a, const LatGeom& g, int X, int Y, int Z,
                                               RowWords<13>& rw) {
  const int q0 = LAT_HALO + 2 * X + B - 3;
  // word offsets of the wrapped rows Y + dy and planes Z + dz (dy, dz in
  // -2..2; the unrolled loop below uses only those its rows need)
  int yo[5], zo[5];
#pragma unroll
  for (int d = -2; d <= 2; ++d) {
    yo[d + 2] = wrap_add(Y, d, g.ny) * g.W;
    zo[d + 2] = wrap_add(Z, d, g.nz) * g.ny * g.W;
  }
  const unsigned long long* base = a.bits + g.bits_off + (q0 >> 5);
#pragma unroll
  for (int q = 0; q < 13; ++q) {
    const unsigned long long code = bcc5_row(B, q);
    const int dy = (int)((code >> 40) & 15) - 2, dz = (int)((code >> 44) & 15) - 2;
    const unsigned long long* row = base + zo[dz + 2] + yo[dy + 2];
    rw.w0[q] = __ldcg(row);
    rw.w1[q] = __ldcg(row + 1);
  }
  rw.own = __ldcg(a.bits + g.bits_off + zo[2] + yo[2] + ((LAT_HALO + 2 * X + B) >> 5));
}

template <int B>
__device__ __forceinline__ void bcc5_counts_from(int X, const RowWords<13>& rw, uint32_t gm, int (&cnt)[5],
                                                 int& t) {
  const int H = 2 * X + B;
  const int sh = (LAT_HALO + H - 3) & 31;
#pragma unroll
  for (int s = 0; s < 5; ++s) cnt[s] = 0;
#pragma unroll
  for (int q = 0; q < 13; ++q) {
    const unsigned long long code = bcc5_row(B, q);
    const uint32_t win = __funnelshift_r(eff32(rw.w0[q], gm), eff32(rw.w1[q], gm), sh);
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const uint32_t m = (uint32_t)(code >> (7 * s)) & 0x7Fu;
      if (m) cnt[s] += __popc(win & m);
    }
  }
  t = (eff32(rw.own, gm) >> ((LAT_HALO + H) & 31)) & 1;
}

template <int B>
__device__ __forceinline__ void bcc5_counts_at(const LatArgs& a, const LatGeom& g, int X, int Y, int Z,
                                               uint32_t gm, int (&cnt)[5], int& t) {
  RowWords<13> rw;
  bcc5_rows_load<B>(a, g, X, Y, Z, rw);
  bcc5_counts_from<B>(X, rw, gm, cnt, t);
}

// first-shell neighbours' summed counts (as lattice_nb_counts) on the
// compile-time rows; B is the basis of the site, the neighbours have 1 - B
template <int B>
__device__ __forceinline__ void bcc5_nb_counts(const LatArgs& a, const LatGeom& g, int X, int Y, int Z,
                                               uint32_t gm, int ti, int (&nb)[5]) {
#pragma unroll
  for (int s = 0; s < 5; ++s) nb[s] = 0;
  const int lo = B ? 0 : -1;
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    const int xx = wrap_add(X, lo + (q & 1), g.nx);
    const int yy = wrap_add(Y, lo + ((q >> 1) & 1), g.ny);
    const int zz = wrap_add(Z, lo + (q >> 2), g.nz);
    int c[5], tk;
    bcc5_counts_at<1 - B>(a, g, xx, yy, zz, gm, c, tk);
#pragma unroll
    for (int s = 0; s < 5; ++s) nb[s] += c[s];
  }
  nb[0] -= 8 * ti;
}

// Summed per-shell B counts of the 8 first-shell neighbours k of site
// (X, Y, Z, b), each without the site itself (species ti, in shell 1 of k):
// the second half of the surrogate's environment descriptor.  The
// neighbours of a corner site (b = 0) are the body centres of the cells at
// offsets {-1, 0}^3, those of a body centre the corners at {0, 1}^3.
template <int NS, int NR>
__device__ __forceinline__ void lattice_nb_counts(const LatArgs& a, const LatGeom& g, int X, int Y, int Z,
                                                  int b, uint32_t gm, int ti, int (&nb)[NS]) {
#pragma unroll
  for (int s = 0; s < NS; ++s) nb[s] = 0;
  const int lo = b ? 0 : -1;
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    int xx = X + lo + (q & 1), yy = Y + lo + ((q >> 1) & 1), zz = Z + lo + (q >> 2);
    xx = xx < 0 ? xx + g.nx : (xx >= g.nx ? xx - g.nx : xx);
    yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
    zz = zz < 0 ? zz + g.nz : (zz >= g.nz ? zz - g.nz : zz);
    int c[NS], tk;
    lattice_counts_at<NS, NR>(a, g, xx, yy, zz, 1 - b, gm, c, tk);
#pragma unroll
    for (int s = 0; s < NS; ++s) nb[s] += c[s];
  }
  nb[0] -= 8 * ti;
}

// The ten scaled descriptor inputs as BF16 pairs (mlp_pairs)
template <int NS>
__device__ __forceinline__ void descriptor_pairs(const int (&cnt)[NS], const int (&nb)[NS], uint32_t (&p)[5]) {
  static_assert(NS == 5, "the descriptor has five shells");
  mlp_pairs(cnt, nb, p);
}

// The same counts in two phases: the raw words of the NR rows (and of the
// site's own word) are loaded first -- they do not depend on the decision
// mask -- so the loads overlap the derivation of G_{k-1}; the counts are
// formed once gm is known.  A word read before another thread's commit of
// step k-1 and one read after it give the same effective species.

template <int NR>
__device__ __forceinline__ void lattice_rows_load(const LatArgs& a, const LatGeom& g, int X, int Y, int Z, int b,
                                                  RowWords<NR>& rw) {
  const int H = 2 * X + b;
  const LatRow* rows = a.rows[b];
  const int q0 = LAT_HALO + H - a.hmax;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    int yy = Y + rows[q].dy, zz = Z + rows[q].dz;
    yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
    zz = zz < 0 ? zz + g.nz : (zz >= g.nz ? zz - g.nz : zz);
    const unsigned long long* row = row_ptr(a, g, yy, zz);
    rw.w0[q] = __ldcg(row + (q0 >> 5));
    rw.w1[q] = __ldcg(row + (q0 >> 5) + 1);
  }
  rw.own = __ldcg(row_ptr(a, g, Y, Z) + ((LAT_HALO + H) >> 5));
}

template <int NS, int NR>
__device__ __forceinline__ void lattice_counts_from(const LatArgs& a, int H, int b, const RowWords<NR>& rw,
                                                    uint32_t gm, int (&cnt)[NS], int& t) {
  const LatRow* rows = a.rows[b];
  const int sh = (LAT_HALO + H - a.hmax) & 31;
#pragma unroll
  for (int s = 0; s < NS; ++s) cnt[s] = 0;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const uint32_t win = __funnelshift_r(eff32(rw.w0[q], gm), eff32(rw.w1[q], gm), sh);
#pragma unroll
    for (int s = 0; s < NS; ++s) cnt[s] += __popc(win & rows[q].mask[s]);
  }
  t = (eff32(rw.own, gm) >> ((LAT_HALO + H) & 31)) & 1;
}

// Programmatic dependent launch: within a chain of colour steps every launch
// after the first is made with programmatic stream serialization, so the
// next step's blocks are scheduled, and draw their random numbers and pick
// their sites, while this step drains.  What a step reads that the previous
// step writes (accumulators, bits, pending slots, states) is read after
// griddepcontrol.wait, which returns once the preceding grid has completed
// and its memory is visible.  Before it a step reads only host-written
// tables and the step base, which only k_lattice_advance writes: that
// kernel and the first step after it are ordinary launches, so the base is
// final before any step of the chain starts.  Without the attribute both
// instructions are no-ops.
// (pdl_wait and pdl_trigger are in common.cuh)

template <bool PROPOSE, int NS, int NR, int BS, bool DA, bool B5, bool PF>
__global__ void __launch_bounds__(BS) k_lattice_step(LatArgs a, int j) {
  pdl_trigger();
  // block -> (replica, first trial): only the blocks a replica needs
  const int2 bk = a.blk[blockIdx.x];
  const int r = bk.x;
  const LatGeom g = a.geom[r];
  const RepParams p = a.rp[r];
  const int d = bk.y + threadIdx.x;
  const long long k = a.ctl->base_step + j;
  const long long kp = k - 1;
  __shared__ int s_g[2];  // [0] = G_{k-1}, [1] = near-tie of that decision

  // inputs that depend on no earlier launch: the global uniform of step k-1
  // (thread 0), the colour, site and random word of trial d of step k.
  // Colours and global uniforms of the chain's steps come from the table
  // the advance kernel filled (entry j + 1 for step base + j).
  const bool tab = j < LAT_CTAB - 1;
  const int* ctab = a.ctab + r * LAT_CTAB;
  uint64_t ug53 = 0;
  if (threadIdx.x == 0 && kp >= 0) {
    if (tab) ug53 = a.ugtab[r * LAT_CTAB + j];
    else lat_colour(a, p.key, kp, &ug53);
  }
  int site = -1, sX = 0, sY = 0, sZ = 0, sb_ = 0;
  uint4 w = make_uint4(0, 0, 0, 0);
  if (PROPOSE) {
    const int c = tab ? ctab[j + 1] : lat_colour(a, p.key, k, nullptr);
    const int D = a.sublattice ? g.d : a.col_start[c + 1] - a.col_start[c];
    if (d < D) {
      w = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)d, TAG_TRIAL), p.key);
      if (a.sublattice) {
        // colour c = (((pz qy + py) qx + px) 2 + b); trial d runs over the
        // colour's sites in ascending index: d = (kz nyq + ky) nxq + kx
        const int b = c & 1;
        const int pc = c >> 1;
        const int pq = fdiv(pc, a.qx, a.rcp_qx);
        const int px = pc - pq * a.qx;
        const int pz = fdiv(pq, a.qy, a.rcp_qy);
        const int py = pq - pz * a.qy;
        const int dq = fdiv(d, g.nxq, g.rcp_nxq);
        const int kx = d - dq * g.nxq;
        const int kz = fdiv(dq, g.nyq, g.rcp_nyq);
        const int ky = dq - kz * g.nyq;
        sX = px + a.qx * kx;
        sY = py + a.qy * ky;
        sZ = pz + a.qz * kz;
        sb_ = b;
        site = ((sZ * g.ny + sY) * g.nx + sX) * 2 + b;
      } else {
        const int gg = a.col_start[c] + d;
        const int base = a.dom_start[gg];
        const int size = a.dom_start[gg + 1] - base;
        site = a.dom_sites[base + pick_index(a.pick, w.x, w.y, size)];
        decode_site(g, site, sX, sY, sZ, sb_);
      }
    }
  }
  pdl_wait();

  // loads of what step k-1 wrote, all issued before the block barrier: the
  // pending slot this thread commits, and (second warp of the replica's
  // first block) the replica state and step k-1's accumulator, staged in
  // shared memory for the finalisation
  int* const slot = a.pend + g.pend_off + d;
  const int ps = d < g.dmax ? __ldcg(slot) : -1;
  __shared__ RepState s_rs;
  __shared__ StepAcc s_acc;
  __shared__ long long s_np;
  const bool fin_warp = bk.y == 0 && (threadIdx.x >> 5) == 1;
  if (fin_warp) {
    const int l = threadIdx.x & 31;
    static_assert(sizeof(RepState) <= 128 && sizeof(StepAcc) <= 128, "one word per lane");
    if (l < (int)(sizeof(RepState) / 4))
      reinterpret_cast<uint32_t*>(&s_rs)[l] = __ldcg(reinterpret_cast<const uint32_t*>(a.rs + r) + l);
    if (kp >= 0) {
      if (l < (int)(sizeof(StepAcc) / 4))
        reinterpret_cast<uint32_t*>(&s_acc)[l] =
            __ldcg(reinterpret_cast<const uint32_t*>(a.acc + r * 3 + (int)(kp % 3)) + l);
      if (l == 0) s_np = __ldcg(a.n_start + r * 2 + (int)(kp & 1));
    }
  }

  // 1. global decision of step k-1: one thread per block, FP64
  if (threadIdx.x == 0) {
    int G = 0, tie = 0;
    if (kp >= 0) {
      // dn and nacc of step k-1 in one 8-byte load, n at its start beside it
      const unsigned long long dn_nacc =
          __ldcg(reinterpret_cast<const unsigned long long*>(&a.acc[r * 3 + (int)(kp % 3)].dn));
      const long long np = __ldcg(a.n_start + r * 2 + (int)(kp & 1));
      const int dnp = (int)(uint32_t)dn_nacc, naccp = (int)(uint32_t)(dn_nacc >> 32);
      if (naccp > 0) G = global_accept(a.lrep[r], p, dnp, np, ug53, &tie) ? 1 : 0;
    }
    s_g[0] = G;
    s_g[1] = tie;
  }

  // rows of the trial site, loaded before the decision of step k-1 is known
  RowWords<(NR > 0 ? NR : 1)> rw;
  if constexpr (PF && PROPOSE && !DA && NR > 0) {
    if (site >= 0) {
      if constexpr (B5) {
        if (sb_) bcc5_rows_load<1>(a, g, sX, sY, sZ, rw);
        else bcc5_rows_load<0>(a, g, sX, sY, sZ, rw);
      } else {
        lattice_rows_load<NR>(a, g, sX, sY, sZ, sb_, rw);
      }
    }
  }
  __syncthreads();
  const bool Gp = s_g[0] != 0;
  const uint32_t gm = Gp ? 0xFFFFFFFFu : 0u;

  // 3. commit this thread's pending flip of step k-1 (slot = row * 2048 +
  //    H, row = Z ny + Y, H = 2 X + b).  The slot itself is rewritten at the
  //    end with this step's pending flip, if any.
  if (ps >= 0) xor_copies(g.nx, a.bits + g.bits_off + (long long)(ps >> 11) * g.W, ps & 2047, Gp, true);

  // 4. finalise step k-1 (second warp of the replica's first block, off the
  //    first warp's path) and clear the accumulator of step k+1
  if (fin_warp && threadIdx.x == 32) {
    RepState S = s_rs;
    if (kp >= 0 && S.fin_step < kp) {
      const StepAcc A = s_acc;
      const long long np = s_np;
      const int cp = tab ? ctab[j] : lat_colour(a, p.key, kp, nullptr);
      const int D = a.sublattice ? g.d : a.col_start[cp + 1] - a.col_start[cp];
      S.trials += D;
      S.local_acc += A.nacc;
      S.s1_acc += A.s1;
      S.near_ties += A.ties + s_g[1];
      long long nn = np;
      if (A.nacc > 0) {
        S.global_trials += 1;
        if (Gp) {
          S.global_acc += 1;
          S.flips += A.nacc;
          nn = np + A.dn;
          // sum over the accepted moves of s_i (C + sum_s b_s G_s + dF_i)
          double e = a.C * (double)A.dn;
          for (int q = 0; q < NS; ++q) e = fma((double)A.sb[q], a.G[q], e);
          e += a.df_uniform ? a.dF0 * (double)A.dn : A.sum_de;
          S.energy += e;
        }
      }
      S.n = nn;
      a.n_start[r * 2 + (int)(k & 1)] = nn;
      const double cc = (double)nn / (double)g.n_sites;
      S.sum_c += cc;
      S.sum_c2 += cc * cc;
      S.steps += 1;
      S.step = k;
      S.fin_step = kp;
      a.rs[r] = S;
    }
    if (PROPOSE) {
      StepAcc* An = a.acc + r * 3 + (int)((k + 1) % 3);
      An->dn = 0;
      An->nacc = 0;
      An->sum_de = 0.0;
      An->ties = 0;
      An->s1 = 0;
      for (int q = 0; q < NS; ++q) An->sb[q] = 0;
    }
  }
  if (!PROPOSE) {
    if (ps >= 0) *slot = -1;
    return;
  }

  // 5. propose trial d of step k on the effective species
  int dn = 0, acc = 0, tie = 0, s1 = 0;
  int sb[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) sb[q] = 0;
  double sdf = 0.0;
  int cnt[NS], t = 0;
  bool accepted = false;
  if constexpr (DA) {
    // delayed acceptance: every lane of the warp takes part in the
    // surrogate's evaluation (lanes without a trial feed zeros)
    uint32_t P[5] = {0u, 0u, 0u, 0u, 0u};
    if (site >= 0) {
      int nb[NS];
      if constexpr (B5) {
        if (sb_) {
          bcc5_counts_at<1>(a, g, sX, sY, sZ, gm, cnt, t);
          bcc5_nb_counts<1>(a, g, sX, sY, sZ, gm, t, nb);
        } else {
          bcc5_counts_at<0>(a, g, sX, sY, sZ, gm, cnt, t);
          bcc5_nb_counts<0>(a, g, sX, sY, sZ, gm, t, nb);
        }
      } else {
        lattice_counts_at<NS, NR>(a, g, sX, sY, sZ, sb_, gm, cnt, t);
        lattice_nb_counts<NS, NR>(a, g, sX, sY, sZ, sb_, gm, t, nb);
      }
      descriptor_pairs<NS>(cnt, nb, P);
    }
    const float gnn = mlp_warp_eval(a.mlp, P);
    if (site >= 0) {
      // stage 1: u < min{1, exp[-beta (s g + s dmu0)]}
      const double sg = t ? -1.0 : 1.0, gd = (double)gnn;
      if (metropolis(p.beta * fma(sg, p.dmu0, sg * gd), top53(w.z, w.w), &tie)) {
        // stage 2: u2 < min{1, exp[-beta (dE - s g)]}
        s1 = 1;
        const double de = lattice_de64<NS>(a, cnt, site, t);
        const uint4 w2 =
            philox4x32_10(make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)d, TAG_STAGE2), p.key);
        accepted = metropolis(p.beta * fma(-sg, gd, de), top53(w2.x, w2.y), &tie);
      }
    }
  } else if (site >= 0) {
    if constexpr (B5 && PF) {
      if (sb_) bcc5_counts_from<1>(sX, rw, gm, cnt, t);
      else bcc5_counts_from<0>(sX, rw, gm, cnt, t);
    } else if constexpr (B5) {
      if (sb_) bcc5_counts_at<1>(a, g, sX, sY, sZ, gm, cnt, t);
      else bcc5_counts_at<0>(a, g, sX, sY, sZ, gm, cnt, t);
    } else if constexpr (NR > 0 && PF) {
      lattice_counts_from<NS, NR>(a, 2 * sX + sb_, sb_, rw, gm, cnt, t);
    } else {
      lattice_counts_at<NS, NR>(a, g, sX, sY, sZ, sb_, gm, cnt, t);
    }
    accepted = lattice_accept<NS>(a, a.lrep[r], p, cnt, site, t, top53(w.z, w.w), &tie);
  }
  if (accepted) {
    const int H = 2 * sX + sb_;
    xor_copies(g.nx, row_ptr(a, g, sY, sZ), H, false, true);  // set pending
    *slot = (sZ * g.ny + sY) * 2048 + H;
    acc = 1;
    dn = t ? -1 : 1;
#pragma unroll
    for (int q = 0; q < NS; ++q) sb[q] = t ? -cnt[q] : cnt[q];
    if (!a.df_uniform) sdf = t ? -a.dF[site] : a.dF[site];
  } else if (ps >= 0) {
    *slot = -1;
  }
  // reduction of dn, accepts, per-shell sums and ties (the paper's
  // allgather of dc_i); warps without an accept or a tie skip the shuffles
  __shared__ int s_red[BS / 32][NS + 4];
  __shared__ double s_df[BS / 32];
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  const bool any = __ballot_sync(0xffffffffu, acc | tie | s1) != 0u;
  if (any) {
    // integer sums with one redux.sync each; the FP64 sum by shuffles
    dn = __reduce_add_sync(0xffffffffu, dn);
    acc = __reduce_add_sync(0xffffffffu, acc);
    tie = __reduce_add_sync(0xffffffffu, tie);
    if constexpr (DA) s1 = __reduce_add_sync(0xffffffffu, s1);
#pragma unroll
    for (int q = 0; q < NS; ++q) sb[q] = __reduce_add_sync(0xffffffffu, sb[q]);
    if (!a.df_uniform) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sdf += __shfl_xor_sync(0xffffffffu, sdf, o);
    }
  }
  if (l == 0) {
    s_red[wi][0] = dn;
    s_red[wi][1] = acc;
    s_red[wi][2] = tie;
#pragma unroll
    for (int q = 0; q < NS; ++q) s_red[wi][3 + q] = sb[q];
    s_red[wi][3 + NS] = s1;
    s_df[wi] = sdf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot[NS + 4];
#pragma unroll
    for (int q = 0; q < NS + 4; ++q) tot[q] = 0;
    double tdf = 0.0;
    for (int w2 = 0; w2 < BS / 32; ++w2) {
#pragma unroll
      for (int q = 0; q < NS + 4; ++q) tot[q] += s_red[w2][q];
      if (!a.df_uniform) tdf += s_df[w2];
    }
    StepAcc* A = a.acc + r * 3 + (int)(k % 3);
    if (tot[1]) {
      atomicAdd(&A->dn, tot[0]);
      atomicAdd(&A->nacc, tot[1]);
#pragma unroll
      for (int q = 0; q < NS; ++q)
        if (tot[3 + q]) atomicAdd(&A->sb[q], tot[3 + q]);
      if (!a.df_uniform) atomicAdd(&A->sum_de, tdf);
    }
    if (tot[2]) atomicAdd(&A->ties, tot[2]);
    if (DA && tot[3 + NS]) atomicAdd(&A->s1, tot[3 + NS]);
  }
}

__global__ void k_lattice_advance(LatCtl* ctl, int n) { ctl->base_step += n; }

// colours and global uniforms of steps base - 1 .. base + LAT_CTAB - 2 of
// every replica (one block per replica); entries for steps < 0 are zero
__global__ void k_colour_table(LatArgs a) {
  const int r = blockIdx.x, t = threadIdx.x;
  if (t >= LAT_CTAB) return;
  const long long k = a.ctl->base_step + t - 1;
  int c = 0;
  uint64_t ug = 0;
  if (k >= 0) c = lat_colour(a, a.rp[r].key, k, &ug);
  a.ctab[r * LAT_CTAB + t] = c;
  a.ugtab[r * LAT_CTAB + t] = ug;
}

void launch_colour_table(const LatArgs& a, cudaStream_t st) {
  k_colour_table<<<a.R, 96, 0, st>>>(a);
}

// species bytes of replica r <-> its bit rows (pending bits cleared)
// species bytes set from the host: any byte other than 0 or 1 sets
// ERRF_SPECIES (16 bytes per thread)
__global__ void k_species_check(const uint8_t* t, long long n, unsigned* err) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long i = 16 * q;
  if (i >= n) return;
  unsigned bad = 0u;
  if (i + 16 <= n && ((uintptr_t)(t + i) & 15) == 0) {
    const uint4 w = *reinterpret_cast<const uint4*>(t + i);
    bad = (w.x | w.y | w.z | w.w) & 0xFEFEFEFEu;
  } else {
    for (long long k = i; k < n && k < i + 16; ++k) bad |= t[k] & 0xFEu;
  }
  if (bad) atomicOr(err, ERRF_SPECIES);
}

void launch_species_check(const uint8_t* t, long long n, unsigned* err, cudaStream_t st) {
  const long long threads = (n + 15) / 16;
  if (threads > 0) k_species_check<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(t, n, err);
}

// one thread per 64-bit word of the rows: 32 species bits (halo included),
// pending half zero; nothing is written after a failed species check.
// Replica r0 + blockIdx.y, species bytes at tptr[r].
__global__ void k_lattice_pack(LatArgs a, uint8_t* const* tptr, int r0) {
  if (*(volatile unsigned*)a.err & ERRF_SPECIES) return;
  const int r = r0 + blockIdx.y;
  const LatGeom g = a.geom[r];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)g.ny * g.nz * g.W) return;
  const long long row = idx / g.W;
  const int q = (int)(idx - row * g.W);
  const uint8_t* t = tptr[r] + row * 2 * g.nx;
  const int L = 2 * g.nx;
  uint32_t bits = 0u;
  for (int k = 0; k < 32; ++k) {
    const int p = 32 * q + k;
    if (p >= L + 2 * LAT_HALO) break;
    int H = p - LAT_HALO;
    H = H < 0 ? H + L : (H >= L ? H - L : H);
    bits |= (uint32_t)(t[H] & 1u) << k;
  }
  a.bits[g.bits_off + idx] = (unsigned long long)bits;
}

__global__ void k_lattice_unpack(LatArgs a, uint8_t* const* tptr, int r0) {
  const int r = r0 + blockIdx.y;
  uint8_t* types_r = tptr[r];
  const LatGeom g = a.geom[r];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_sites) return;
  int X, Y, Z, b;
  decode_site(g, (int)i, X, Y, Z, b);
  types_r[i] = (uint8_t)own_bit(row_ptr(a, g, Y, Z), 2 * X + b, 0u);
}

// four sites per thread when nx is even: sites 4u .. 4u + 3 share a row and
// a 4-bit window of one species word (row positions are multiples of 4 plus
// the even halo), written as one 32-bit store of four bytes
__global__ void k_lattice_unpack4(LatArgs a, uint8_t* const* tptr, int r0) {
  const int r = r0 + blockIdx.y;
  const LatGeom g = a.geom[r];
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * u >= g.n_sites) return;
  const int i = (int)(4 * u);
  const int row = fdiv(i >> 1, g.nx, g.rcp_nx);  // (Z ny + Y)
  const int p = LAT_HALO + (i - 2 * g.nx * row);
  const uint32_t w = (uint32_t)__ldcg(a.bits + g.bits_off + (long long)row * g.W + (p >> 5));
  const uint32_t f = (w >> (p & 31)) & 15u;
  const uint32_t v = (f & 1u) | ((f & 2u) << 7) | ((f & 4u) << 14) | ((f & 8u) << 21);
  *reinterpret_cast<uint32_t*>(tptr[r] + i) = v;
}

template <int NS>
__global__ void k_lattice_delta_e(LatArgs a, int r, const int* sites, int n, double* out) {
  const LatGeom g = a.geom[r];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int X, Y, Z, b, t;
  decode_site(g, sites[q], X, Y, Z, b);
  int cnt[NS];
  lattice_counts_at<NS, 0>(a, g, X, Y, Z, b, 0u, cnt, t);
  out[q] = lattice_de64<NS>(a, cnt, sites[q], t);
}

// Descriptor counts and exact A->B energy change of every site (all
// replicas; blockIdx.y = replica), species as stored (no pending flips)
template <bool B5>
__global__ void k_lattice_features(LatArgs a, float* X, float* Y) {
  const int r = blockIdx.y;
  const LatGeom g = a.geom[r];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_sites) return;
  int sX, sY, sZ, b, t;
  decode_site(g, (int)i, sX, sY, sZ, b);
  int cnt[5], nb[5];
  if constexpr (B5) {
    if (b) {
      bcc5_counts_at<1>(a, g, sX, sY, sZ, 0u, cnt, t);
      bcc5_nb_counts<1>(a, g, sX, sY, sZ, 0u, t, nb);
    } else {
      bcc5_counts_at<0>(a, g, sX, sY, sZ, 0u, cnt, t);
      bcc5_nb_counts<0>(a, g, sX, sY, sZ, 0u, t, nb);
    }
  } else {
    lattice_counts_at<5, 13>(a, g, sX, sY, sZ, b, 0u, cnt, t);
    lattice_nb_counts<5, 13>(a, g, sX, sY, sZ, b, 0u, t, nb);
  }
  const long long row = g.site_off + i;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    X[row * MLP_IN + s] = (float)cnt[s];
    X[row * MLP_IN + 5 + s] = (float)nb[s];
  }
  Y[row] = (float)lattice_de64<5>(a, cnt, (int)i, 0);
}

void launch_lattice_features(const LatArgs& a, long long max_sites, float* X, float* Y, cudaStream_t st) {
  const dim3 grid((unsigned)((max_sites + 127) / 128), (unsigned)a.R);
  if (a.bcc5) k_lattice_features<true><<<grid, 128, 0, st>>>(a, X, Y);
  else k_lattice_features<false><<<grid, 128, 0, st>>>(a, X, Y);
}

// Energy and B count of replica r = r0 + blockIdx.y from its packed species.
// With phi_ab(r_s) the pair values at the shell radii, G_s = phi_BB - 2
// phi_AB + phi_AA and one uniform density rho0,
//   E = N F_A + n_B (F_B - F_A) + 1/2 sum_s z_s [N phi_AA + 2 n_B (phi_AB - phi_AA)]
//       + 1/2 sum_s G_s P_s,   P_s = sum over B sites i of b_s(i),
// (expand phi_{t_i t_j} in t_i, t_j and sum over ordered neighbour pairs), so
// only B sites are visited: one thread per 32-bit species word of the rows,
// a loop over its set bits (halo bits excluded).  Block partial sums of
// (P_1 .. P_S, n_B): part[r - r0][b][LAT_E_W], stride pstride blocks.
constexpr int LAT_E_BLOCK = 256;
constexpr int LAT_E_W = LAT_MAX_SH + 1;
template <bool B5>
__global__ void __launch_bounds__(LAT_E_BLOCK)
    k_lattice_energy(LatArgs a, int r0, double* part, int pstride) {
  if (*(volatile unsigned*)a.err & ERRF_SPECIES) return;
  const int r = r0 + blockIdx.y;
  part += (long long)LAT_E_W * pstride * blockIdx.y;
  const LatGeom g = a.geom[r];
  const long long nw = (long long)g.ny * g.nz * g.W;
  if ((long long)blockIdx.x * LAT_E_BLOCK >= nw) return;
  const long long idx = (long long)blockIdx.x * LAT_E_BLOCK + threadIdx.x;
  int acc[LAT_E_W];
#pragma unroll
  for (int s = 0; s < LAT_E_W; ++s) acc[s] = 0;
  if (idx < nw) {
    const long long row = idx / g.W;
    const int q = (int)(idx - row * g.W);
    const int Y = (int)(row % g.ny), Z = (int)(row / g.ny);
    uint32_t w = (uint32_t)a.bits[g.bits_off + idx];
    // keep bits p = 32 q + k with LAT_HALO <= p < LAT_HALO + 2 nx
    const int lo = LAT_HALO - 32 * q, hi = LAT_HALO + 2 * g.nx - 32 * q;
    if (lo > 0) w &= lo >= 32 ? 0u : ~((1u << lo) - 1u);
    if (hi < 32) w &= hi <= 0 ? 0u : ((1u << hi) - 1u);
    while (w) {
      const int k = __ffs(w) - 1;
      w &= w - 1u;
      const int H = 32 * q + k - LAT_HALO;
      const int X = H >> 1, b = H & 1;
      int t;
      if constexpr (B5) {
        int cnt[5];
        if (b) bcc5_counts_at<1>(a, g, X, Y, Z, 0u, cnt, t);
        else bcc5_counts_at<0>(a, g, X, Y, Z, 0u, cnt, t);
#pragma unroll
        for (int s = 0; s < 5; ++s) acc[s] += cnt[s];
      } else {
        int cnt[LAT_MAX_SH];
        lattice_counts_at<LAT_MAX_SH, 0>(a, g, X, Y, Z, b, 0u, cnt, t);
#pragma unroll
        for (int s = 0; s < LAT_MAX_SH; ++s) acc[s] += cnt[s];
      }
      acc[LAT_MAX_SH] += 1;
    }
  }
  __shared__ int s_acc[LAT_E_BLOCK / 32][LAT_E_W];
#pragma unroll
  for (int s = 0; s < LAT_E_W; ++s) acc[s] = __reduce_add_sync(0xffffffffu, acc[s]);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int s = 0; s < LAT_E_W; ++s) s_acc[threadIdx.x >> 5][s] = acc[s];
  }
  __syncthreads();
  if (threadIdx.x < LAT_E_W) {
    long long tot = 0;
    for (int w2 = 0; w2 < LAT_E_BLOCK / 32; ++w2) tot += s_acc[w2][threadIdx.x];
    // integer totals of the replica: one atomic per block and counter
    if (tot) atomicAdd(reinterpret_cast<unsigned long long*>(part) + threadIdx.x, (unsigned long long)tot);
  }
}

// The same totals bit-parallel for the five-shell table: one thread per
// word of 32 row positions, whose B sites are summed against the neighbour
// offsets of one sign at once (twice that is the ordered-pair count).  For own basis b and offset h (half-lattice
// units) the neighbours sit in row (Y + dy, Z + dz) at row position H + hx,
// so a 32-bit window of that row shifted by hx, ANDed with the word's B
// sites of basis b, counts the ordered B-B pairs of shell s(h) in popc.
// The rows' halo copies make the windows of valid positions periodic.
__device__ __forceinline__ uint32_t spec_word(const LatArgs& a, const LatGeom& g, int Y, int Z, int q) {
  return (q < 0 || q >= g.W) ? 0u : (uint32_t)__ldcg(a.bits + g.bits_off + ((long long)Z * g.ny + Y) * g.W + q);
}

__global__ void __launch_bounds__(LAT_E_BLOCK) k_lattice_pairs_bcc5(LatArgs a, int r0, double* part, int pstride) {
  if (*(volatile unsigned*)a.err & ERRF_SPECIES) return;
  const int r = r0 + blockIdx.y;
  part += (long long)LAT_E_W * pstride * blockIdx.y;
  const LatGeom g = a.geom[r];
  const long long nw = (long long)g.ny * g.nz * g.W;
  if ((long long)blockIdx.x * LAT_E_BLOCK >= nw) return;
  const long long idx = (long long)blockIdx.x * LAT_E_BLOCK + threadIdx.x;
  int acc[LAT_E_W];
#pragma unroll
  for (int s = 0; s < LAT_E_W; ++s) acc[s] = 0;
  if (idx < nw) {
    const long long row = idx / g.W;
    const int q = (int)(idx - row * g.W);
    const int Y = (int)(row % g.ny), Z = (int)(row / g.ny);
    uint32_t w = spec_word(a, g, Y, Z, q);
    // own positions p = 32 q + k with LAT_HALO <= p < LAT_HALO + 2 nx
    const int lo = LAT_HALO - 32 * q, hi = LAT_HALO + 2 * g.nx - 32 * q;
    if (lo > 0) w &= lo >= 32 ? 0u : ~((1u << lo) - 1u);
    if (hi < 32) w &= hi <= 0 ? 0u : ((1u << hi) - 1u);
    acc[LAT_MAX_SH] = __popc(w);
    if (w) {
      int yw[5], zw[5];
#pragma unroll
      for (int d = -2; d <= 2; ++d) {
        yw[d + 2] = wrap_add(Y, d, g.ny);
        zw[d + 2] = wrap_add(Z, d, g.nz);
      }
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        // row position parity = basis (LAT_HALO is even)
        const uint32_t wb = w & (b ? 0xAAAAAAAAu : 0x55555555u);
        if (!wb) continue;
#pragma unroll
        for (int k = 0; k < MK_BCC5_N; ++k) {
          const int code = mk_bcc5_code(k);
          const int hx = (code & 15) - 4, hy = ((code >> 4) & 15) - 4, hz = ((code >> 8) & 15) - 4;
          // the table holds h and -h: pairs along offsets of one sign, each
          // unordered pair once (doubled below)
          if (!(hx > 0 || (hx == 0 && (hy > 0 || (hy == 0 && hz > 0))))) continue;
          const int bb = b ^ (hx & 1);
          const int Yn = yw[((b + hy - bb) >> 1) + 2], Zn = zw[((b + hz - bb) >> 1) + 2];
          const uint32_t win = hx >= 0 ? __funnelshift_r(spec_word(a, g, Yn, Zn, q), spec_word(a, g, Yn, Zn, q + 1), hx)
                                       : __funnelshift_r(spec_word(a, g, Yn, Zn, q - 1), spec_word(a, g, Yn, Zn, q),
                                                         32 + hx);
          acc[code >> 12] += __popc(wb & win);
        }
      }
#pragma unroll
      for (int sh = 0; sh < 5; ++sh) acc[sh] *= 2;  // ordered pairs
    }
  }
  __shared__ int s_acc[LAT_E_BLOCK / 32][LAT_E_W];
#pragma unroll
  for (int s = 0; s < LAT_E_W; ++s) acc[s] = __reduce_add_sync(0xffffffffu, acc[s]);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int s = 0; s < LAT_E_W; ++s) s_acc[threadIdx.x >> 5][s] = acc[s];
  }
  __syncthreads();
  if (threadIdx.x < LAT_E_W) {
    long long tot = 0;
    for (int w2 = 0; w2 < LAT_E_BLOCK / 32; ++w2) tot += s_acc[w2][threadIdx.x];
    if (tot) atomicAdd(reinterpret_cast<unsigned long long*>(part) + threadIdx.x, (unsigned long long)tot);
  }
}

// Sums of the block partials (one block per replica r0 + blockIdx.x), the
// energy, written to the replica's state and to the B count at the start of
// the next step.  etab: phi_AA, phi_AB, phi_BB per shell, F_A, F_B, z_s.
__global__ void k_lattice_energy_final(LatArgs a, int r0, const double* etab, const double* part, int pstride,
                                       int parity) {
  if (*(volatile unsigned*)a.err & ERRF_SPECIES) return;
  const int r = r0 + blockIdx.x;
  part += (long long)LAT_E_W * pstride * blockIdx.x;
  const LatGeom g = a.geom[r];
  __shared__ double s_tot[LAT_E_W];
  if (threadIdx.x < LAT_E_W) s_tot[threadIdx.x] = (double)reinterpret_cast<const unsigned long long*>(part)[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int S = a.n_shells;
    const double N = (double)g.n_sites, nB = s_tot[LAT_MAX_SH];
    double pair = 0.0;
    for (int s = 0; s < S; ++s) {
      const double pAA = etab[s], pAB = etab[S + s], pBB = etab[2 * S + s], z = etab[3 * S + 2 + s];
      pair += z * (N * pAA + 2.0 * nB * (pAB - pAA)) + (pBB - 2.0 * pAB + pAA) * s_tot[s];
    }
    const double e = N * etab[3 * S] + nB * (etab[3 * S + 1] - etab[3 * S]) + 0.5 * pair;
    const long long nb = (long long)nB;
    a.rs[r].n = nb;
    a.rs[r].energy = e;
    a.n_start[2 * r + parity] = nb;
  }
}

int lattice_energy_blocks(long long max_words) { return (int)((max_words + LAT_E_BLOCK - 1) / LAT_E_BLOCK); }
int lattice_energy_width() { return LAT_E_W; }

void launch_lattice_energy(const LatArgs& a, int r0, int nrep, long long max_words, const double* etab,
                           double* part, int pstride, int parity, cudaStream_t st) {
  const dim3 grid(lattice_energy_blocks(max_words), nrep);
  // the first LAT_E_W words of each replica's region take integer totals
  cudaMemsetAsync(part, 0, sizeof(double) * LAT_E_W * pstride * nrep, st);
  if (a.bcc5) k_lattice_pairs_bcc5<<<grid, LAT_E_BLOCK, 0, st>>>(a, r0, part, pstride);
  else k_lattice_energy<false><<<grid, LAT_E_BLOCK, 0, st>>>(a, r0, part, pstride);
  k_lattice_energy_final<<<nrep, 32, 0, st>>>(a, r0, etab, part, pstride, parity);
}

__global__ void k_to_float(const double* in, float* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

void launch_to_float(const double* in, float* out, long long n, cudaStream_t st) {
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
}

// launch, with programmatic stream serialization when pdl (see pdl_wait)
template <typename K>
static void launch_step(K kern, dim3 grid, int block, cudaStream_t st, const LatArgs& a, int j, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, a, j);
}

// PF: the trial's row words are loaded before the block barrier (fewer
// dependent steps, more registers); the autotuner picks it or not
template <int NS, int NR, int BS, bool B5>
static void step_b5(const LatArgs& a, int j, bool propose, cudaStream_t st) {
  const dim3 g(a.n_blk);
  const bool pdl = j > 0;  // the first step of a chain is an ordinary launch
  constexpr bool DA_OK = NS == 5 && NR == 13;
  if (!propose) launch_step(k_lattice_step<false, NS, NR, BS, false, B5, false>, g, BS, st, a, j, pdl);
  else if (DA_OK && a.da) launch_step(k_lattice_step<true, NS, NR, BS, DA_OK, B5, false>, g, BS, st, a, j, pdl);
  else if (a.prefetch) launch_step(k_lattice_step<true, NS, NR, BS, false, B5, true>, g, BS, st, a, j, pdl);
  else launch_step(k_lattice_step<true, NS, NR, BS, false, B5, false>, g, BS, st, a, j, pdl);
}

template <int NS, int NR, int BS>
static void step_bs(const LatArgs& a, int j, bool propose, cudaStream_t st) {
  if constexpr (NS == 5 && NR == 13) {
    if (a.bcc5) {
      step_b5<NS, NR, BS, true>(a, j, propose, st);
      return;
    }
  }
  step_b5<NS, NR, BS, false>(a, j, propose, st);
}

template <int NS, int NR>
static void step_ns(const LatArgs& a, int j, bool propose, cudaStream_t st) {
  switch (a.block) {
    case 64: step_bs<NS, NR, 64>(a, j, propose, st); break;
    case 256: step_bs<NS, NR, 256>(a, j, propose, st); break;
    default: step_bs<NS, NR, 128>(a, j, propose, st); break;
  }
}

// shells and neighbour rows as compile-time constants: the 5-shell, 13-row
// BCC neighbourhood within r_c < sqrt(19) a/2 and the first-shell form are
// unrolled; any other neighbourhood takes the runtime-count variant
void launch_lattice_step(const LatArgs& a, int j, bool propose, cudaStream_t st) {
  const int nr = a.n_rows[0] == a.n_rows[1] ? a.n_rows[0] : -1;
  if (a.n_shells == 5 && nr == 13) step_ns<5, 13>(a, j, propose, st);
  else if (a.n_shells == 1 && nr == 2) step_ns<1, 2>(a, j, propose, st);
  else step_ns<LAT_MAX_SH, 0>(a, j, propose, st);
}

bool lattice_rows_bcc5(const LatArgs& a) {
  if (a.n_shells != 5 || a.hmax != 3 || a.n_rows[0] != 13 || a.n_rows[1] != 13) return false;
  for (int b = 0; b < 2; ++b)
    for (int q = 0; q < 13; ++q) {
      const unsigned long long code = bcc5_row(b, q);
      const LatRow& rw = a.rows[b][q];
      if (rw.dy != (int)((code >> 40) & 15) - 2 || rw.dz != (int)((code >> 44) & 15) - 2) return false;
      for (int s = 0; s < LAT_MAX_SH; ++s)
        if (rw.mask[s] != (s < 5 ? (uint32_t)(code >> (7 * s)) & 0x7Fu : 0u)) return false;
    }
  return true;
}

void launch_lattice_advance(const LatArgs& a, int n, cudaStream_t st) {
  k_lattice_advance<<<1, 1, 0, st>>>(a.ctl, n);
  launch_colour_table(a, st);
}

void launch_lattice_pack(const LatArgs& a, uint8_t* const* tptr, int r0, int nrep, long long max_words,
                         cudaStream_t st) {
  k_lattice_pack<<<dim3((unsigned)((max_words + 255) / 256), nrep), 256, 0, st>>>(a, tptr, r0);
}

void launch_lattice_unpack(const LatArgs& a, uint8_t* const* tptr, int r0, int nrep, long long max_sites,
                           cudaStream_t st) {
  if (a.unpack4) {
    const long long groups = (max_sites + 3) / 4;
    k_lattice_unpack4<<<dim3((unsigned)((groups + 255) / 256), nrep), 256, 0, st>>>(a, tptr, r0);
  } else {
    k_lattice_unpack<<<dim3((unsigned)((max_sites + 255) / 256), nrep), 256, 0, st>>>(a, tptr, r0);
  }
}

void launch_lattice_delta_e(const LatArgs& a, int r, const int* sites, int n, double* out, cudaStream_t st) {
  if (n > 0) k_lattice_delta_e<LAT_MAX_SH><<<(n + 127) / 128, 128, 0, st>>>(a, r, sites, n, out);
}

}  // namespace vcsgc
