// kernels_cluster.cu -- the fused colour step of the rigid BCC lattice
// (period-q sublattice schedule, five-shell neighbourhood, one density
// function) as one persistent launch: one thread-block cluster per replica
// runs many colour steps (composite moves of Sec. III B 2) back to back.
//
// The replica's bit-packed species rows (the layout of kernels_lattice.cu:
// per (y, z) row, 32 species bits and 32 pending bits per 64-bit word, four
// halo bits at each end) are tiled over the cluster's CTAs in (y, z): CTA
// (ty, tz) of a TY x TZ grid owns rows [ty Ty, (ty + 1) Ty) x [tz Tz, (tz +
// 1) Tz) and keeps them in shared memory together with a halo of two rows on
// each side (every neighbour of a site lies within dy, dz in -2..2), so the
// dE gather of a trial reads only its own shared memory.
//
// Only a row's owner changes it, with shared-memory atomics on its own
// copies.  At the end of each colour step, after a block barrier, the owner
// stores the final value of every word it changed in that step into the
// halo copies the other CTAs hold (plain st.shared::cluster: all stores of
// one word in one step carry the same value, so their order is free).  A
// first form that XOR-ed the halo copies with red.shared::cluster lost
// updates when two XORs of one word met, so no distributed-shared atomics
// are used.  The dn reduction works the same way: each CTA leaves its
// partial sums in its own shared memory and every warp reads all of them
// after the barrier.
//
// Colour step k, every CTA:
//   1. draws its trials' uniforms (Philox keyed by step and trial: the same
//      numbers as the per-step launch) while the previous step's barrier
//      completes;
//   2. after barrier.cluster.wait, sums the CTAs' partials of step k-1 and
//      takes the global decision G_{k-1} (Eq. trans_vcsgc_par2) -- every warp
//      the same, no second barrier;
//   3. commits its own accepted trials of step k-1 (one XOR per copy that
//      clears the pending bit and flips the species if G_{k-1});
//   4. proposes step k on the effective species t ^ (pending & G_{k-1}) and
//      sets the pending bit of each locally accepted trial;
//   5. reduces dn, accepts, ties and per-shell sums into its partial, pushes
//      the words it changed to the halo copies, and arrives at the cluster
//      barrier (release).
// The leader CTA (rank 0) also finalises step k-1 (counters, B count,
// energy, <c> sums) as the per-step launch does.  A word read before or
// after a commit or push of step k-1 gives the same effective species, and
// no trial of step k reads a bit that another trial of step k sets
// (same-colour sites are more than 2 r_c apart), exactly as in the per-step
// form.  After the last step the kernel commits it, finalises it and writes
// the owned rows, the replica state and the bookkeeping the per-step launch
// expects back to global memory, so the two forms can follow each other in
// one chain.
//
// Every CTA of a cluster runs the same number of cluster barriers (uniform
// control flow, no early exit, a last barrier before any CTA exits so that
// no CTA reads the shared memory of one that has finished); clusters of
// different replicas never wait on each other.
#include "common.cuh"
#include "kernels.h"
#include "lattice.cuh"

namespace vcsgc {

namespace {

constexpr int CL_NF = 8;                      // partial sums: dn, nacc, ties, sb[0..4]

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_nctas() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared::cluster address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st_u64(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ int4 cl_ld_v4(uint32_t a) {
  int4 v;
  asm volatile("ld.shared::cluster.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
// cluster barrier, split: arrive (release: this thread's earlier shared and
// distributed-shared writes become visible) and wait (acquire)
__device__ __forceinline__ void cl_arrive() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
  __syncwarp();
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the CTA's tile of one replica
struct TileView {
  int ty, tz;  // tile indices
  int RY;      // rows per plane in shared memory (Ty + 4)
  int Y0, Z0;  // first owned row, plane
};

// positions (row bit indices) of the copies of site H in its row: the main
// one and, near the ends, the halo copy at the other end
__device__ __forceinline__ int site_positions(int nx, int H, int (&pos)[3]) {
  int n = 0;
  pos[n++] = LAT_HALO + H;
  if (H >= 2 * nx - LAT_HALO) pos[n++] = LAT_HALO + H - 2 * nx;
  if (H < LAT_HALO) pos[n++] = LAT_HALO + H + 2 * nx;
  return n;
}

// XOR the species (flip_species) and pending (flip_pending) bits of site H
// of row (Y, Z) -- owned by this CTA -- into every copy of the row this CTA
// holds: local row Y - (Y0 - 2) (mod ny) below Ty + 4, more than once when
// the tile with its halo spans the whole period
__device__ __forceinline__ void flip_local(unsigned long long* rows, const ClTile& T, const LatGeom& g,
                                           const TileView& v, int Y, int Z, int H, bool flip_species,
                                           bool flip_pending) {
  int pos[3];
  const int n = site_positions(g.nx, H, pos);
  int ly0 = (Y - (v.Y0 - 2)) % g.ny;
  ly0 = ly0 < 0 ? ly0 + g.ny : ly0;
  int lz0 = (Z - (v.Z0 - 2)) % g.nz;
  lz0 = lz0 < 0 ? lz0 + g.nz : lz0;
  for (int q = 0; q < n; ++q) {
    const int p = pos[q];
    unsigned long long m = 0;
    if (flip_species) m |= 1ull << (p & 31);
    if (flip_pending) m |= 1ull << (32 + (p & 31));
    for (int lz = lz0; lz < T.Tz + 4; lz += g.nz)
      for (int ly = ly0; ly < T.Ty + 4; ly += g.ny) atomicXor(rows + (lz * v.RY + ly) * g.W + (p >> 5), m);
  }
}

// store the current value of the words of site H of row (Y, Z) (owned by
// this CTA) into every copy of the row the other CTAs of the cluster hold:
// the tiles at tile offsets -1..1 in y and z (distinct ones, this one left
// out) whose rows with halo cover (Y, Z)
__device__ __forceinline__ void push_remote(const unsigned long long* rows, uint32_t rows_addr, const ClTile& T,
                                            const LatGeom& g, const TileView& v, int Y, int Z, int H) {
  int pos[3];
  const int n = site_positions(g.nx, H, pos);
  const int own = ((Z - v.Z0 + 2) * v.RY + (Y - v.Y0 + 2)) * g.W;
  const int me = v.tz * T.TY + v.ty;
  int seen_y[3], ny_seen = 0;
  for (int a = -1; a <= 1; ++a) {
    int tyn = v.ty + a;
    tyn = tyn < 0 ? tyn + T.TY : (tyn >= T.TY ? tyn - T.TY : tyn);
    bool dup = false;
    for (int q = 0; q < ny_seen; ++q) dup |= seen_y[q] == tyn;
    if (dup) continue;
    seen_y[ny_seen++] = tyn;
    int seen_z[3], nz_seen = 0;
    for (int b = -1; b <= 1; ++b) {
      int tzn = v.tz + b;
      tzn = tzn < 0 ? tzn + T.TZ : (tzn >= T.TZ ? tzn - T.TZ : tzn);
      bool dz = false;
      for (int q = 0; q < nz_seen; ++q) dz |= seen_z[q] == tzn;
      if (dz) continue;
      seen_z[nz_seen++] = tzn;
      const int rank = tzn * T.TY + tyn;
      if (rank == me) continue;
      int ly0 = (Y - (tyn * T.Ty - 2)) % g.ny;
      ly0 = ly0 < 0 ? ly0 + g.ny : ly0;
      int lz0 = (Z - (tzn * T.Tz - 2)) % g.nz;
      lz0 = lz0 < 0 ? lz0 + g.nz : lz0;
      for (int lz = lz0; lz < T.Tz + 4; lz += g.nz)
        for (int ly = ly0; ly < T.Ty + 4; ly += g.ny)
          for (int q = 0; q < n; ++q) {
            const int w = pos[q] >> 5;
            const uint32_t la = rows_addr + (uint32_t)(((lz * v.RY + ly) * g.W + w) * 8);
            cl_st_u64(cl_map(la, (uint32_t)rank), rows[own + w]);
          }
    }
  }
}

// per-shell B counts and own species of site (X, ly, lz, basis B) from the
// shared-memory rows (local row ly, plane lz of the tile with halo)
template <int B>
__device__ __forceinline__ void cl_counts(const unsigned long long* rows, int RY, int W, int X, int ly, int lz,
                                          uint32_t gm, int (&cnt)[5], int& t) {
  const int H = 2 * X + B;
  const int q0 = LAT_HALO + H - 3;
  const int sh = q0 & 31;
  const unsigned long long* base = rows + (q0 >> 5);
  unsigned long long w0[13], w1[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) {
    const unsigned long long code = bcc5_row(B, q);
    const int dy = (int)((code >> 40) & 15) - 2, dz = (int)((code >> 44) & 15) - 2;
    const unsigned long long* row = base + ((lz + dz) * RY + (ly + dy)) * W;
    w0[q] = row[0];
    w1[q] = row[1];
  }
  const unsigned long long own = rows[(lz * RY + ly) * W + ((LAT_HALO + H) >> 5)];
#pragma unroll
  for (int s = 0; s < 5; ++s) cnt[s] = 0;
#pragma unroll
  for (int q = 0; q < 13; ++q) {
    const unsigned long long code = bcc5_row(B, q);
    const uint32_t win = __funnelshift_r(eff32(w0[q], gm), eff32(w1[q], gm), sh);
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const uint32_t m = (uint32_t)(code >> (7 * s)) & 0x7Fu;
      if (m) cnt[s] += __popc(win & m);
    }
  }
  t = (eff32(own, gm) >> ((LAT_HALO + H) & 31)) & 1;
}

// sums over the cluster's CTAs of four consecutive partial fields at
// part_addr (lane c < nctas loads CTA c's; every lane returns the totals)
__device__ __forceinline__ int4 cluster_sum4(uint32_t part_addr, int nctas, int lane) {
  int4 v = make_int4(0, 0, 0, 0);
  if (lane < nctas) v = cl_ld_v4(cl_map(part_addr, (uint32_t)lane));
  v.x = __reduce_add_sync(0xffffffffu, v.x);
  v.y = __reduce_add_sync(0xffffffffu, v.y);
  v.z = __reduce_add_sync(0xffffffffu, v.z);
  v.w = __reduce_add_sync(0xffffffffu, v.w);
  return v;
}

}  // namespace

// One cluster per replica (replica = cluster index).  Dynamic shared memory:
// the tile's rows with halo, one pad word, the uniforms of a step's trials,
// two lists of accepted trials.
template <int BS>
__global__ void __launch_bounds__(BS, 1) k_cluster_steps(LatArgs a, const ClTile* tiles, long long base, int n) {
  extern __shared__ __align__(16) unsigned long long cl_smem[];
  __shared__ int s_cnt[2];
  __shared__ int s_red[BS / 32][CL_NF];
  __shared__ __align__(16) int s_part[2][CL_NF];  // this CTA's sums of a step, by step parity
  __shared__ RepState s_rs;                        // the replica's running state (leader only)

  const int r = (int)cl_id();
  const uint32_t rank = cl_rank();
  const int nctas = (int)cl_nctas();
  const ClTile T = tiles[r];
  const LatGeom g = a.geom[r];
  const RepParams p = a.rp[r];
  const LatRep lr = a.lrep[r];
  TileView v;
  v.ty = (int)rank % T.TY;
  v.tz = (int)rank / T.TY;
  v.RY = T.Ty + 4;
  v.Y0 = v.ty * T.Ty;
  v.Z0 = v.tz * T.Tz;
  const int W = g.W;
  const int RZ = T.Tz + 4;
  unsigned long long* rows = cl_smem;
  const int lcap = T.lcap;
  unsigned long long* s_u53 = cl_smem + (size_t)RZ * v.RY * W + 1;  // the trials' uniforms of a step
  int* list = reinterpret_cast<int*>(s_u53 + lcap);
  const uint32_t rows_addr = smem_addr(rows);
  const uint32_t part_addr = smem_addr(&s_part[0][0]);
  const bool leader = rank == 0;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;

  // ---- load the tile with halo (pending bits are clear: the host applied
  //      any pending commit before this launch)
  {
    const int nwords = RZ * v.RY * W;
    const unsigned long long* src = a.bits + g.bits_off;
    for (int q = threadIdx.x; q < nwords; q += BS) {
      const int w = q % W;
      const int rr = q / W;
      const int ly = rr % v.RY, lz = rr / v.RY;
      int Y = (v.Y0 - 2 + ly) % g.ny;
      Y = Y < 0 ? Y + g.ny : Y;
      int Z = (v.Z0 - 2 + lz) % g.nz;
      Z = Z < 0 ? Z + g.nz : Z;
      rows[q] = __ldcg(src + ((long long)Z * g.ny + Y) * W + w);
    }
  }
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  if (leader && threadIdx.x == 0) s_rs = a.rs[r];
  // B count at the start of the previous step (tracked alike by every warp)
  long long n_prev = __ldcg(&a.rs[r].n);
  cl_arrive();
  cl_wait();

  uint64_t ug_prev = 0;  // global uniform of step k - 1 (lane 0 of each warp)

  for (int j = 0; j <= n; ++j) {
    const long long k = base + j;
    const bool propose = j < n;
    // ---- 1. colour of step k, its trials and their uniforms (no state read)
    int c = 0;
    uint64_t ug_k = 0;
    if (lane == 0 && propose) c = lat_colour(a, p.key, k, &ug_k);
    c = __shfl_sync(0xffffffffu, c, 0);
    const int b = c & 1, pc = c >> 1;
    const int px = pc % a.qx, pq = pc / a.qx;
    const int py = pq % a.qy, pz = pq / a.qy;
    const int kyb = (v.Y0 - py + a.qy - 1) / a.qy, kzb = (v.Z0 - pz + a.qz - 1) / a.qz;
    const int cy = (v.Y0 + T.Ty - py + a.qy - 1) / a.qy - kyb;
    const int cz = (v.Z0 + T.Tz - pz + a.qz - 1) / a.qz - kzb;
    const int ntr = propose ? cy * cz * g.nxq : 0;
    const float rcp_cy = 1.0f / (float)(cy > 0 ? cy : 1);
    // (the previous step's reads of s_u53 ended before its last block barrier)
    for (int t = threadIdx.x; t < ntr; t += BS) {
      const int tq = fdiv(t, g.nxq, g.rcp_nxq);
      const int kx = t - tq * g.nxq;
      const int kzl = fdiv(tq, cy, rcp_cy);
      const int ky = kyb + tq - kzl * cy, kz = kzb + kzl;
      const int d = (kz * g.nyq + ky) * g.nxq + kx;
      const uint4 w =
          philox4x32_10(make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)d, TAG_TRIAL), p.key);
      s_u53[t] = top53(w.z, w.w);
    }
    if (j > 0) cl_wait();  // barrier of step k - 1

    // ---- 2. global decision of step k - 1 (every warp alike)
    int G = 0, gtie = 0;
    int4 s_lo = make_int4(0, 0, 0, 0), s_hi = make_int4(0, 0, 0, 0);
    if (j > 0) {
      const uint32_t pa = part_addr + (uint32_t)(((k - 1) & 1) * CL_NF * 4);
      s_lo = cluster_sum4(pa, nctas, lane);  // dn, nacc, ties, sb[0]
      if (lane == 0 && s_lo.y > 0) G = global_accept(lr, p, s_lo.x, n_prev, ug_prev, &gtie) ? 1 : 0;
      G = __shfl_sync(0xffffffffu, G, 0);
      if (leader && wi == 0) s_hi = cluster_sum4(pa + 16, nctas, lane);  // sb[1..4]
    }
    ug_prev = ug_k;
    const uint32_t gm = G ? 0xFFFFFFFFu : 0u;

    // ---- 3. commit this CTA's accepted trials of step k - 1 (its own copies)
    int na_prev = 0;
    if (j > 0) {
      const int* lp = list + ((k - 1) & 1) * lcap;
      na_prev = s_cnt[(k - 1) & 1];
      for (int q = threadIdx.x; q < na_prev; q += BS) {
        const int e = lp[q];  // (Y * nz + Z) * 2048 + H
        const int H = e & 2047, yz = e >> 11;
        flip_local(rows, T, g, v, yz / g.nz, yz % g.nz, H, G != 0, true);
      }
      // leader: finalise step k - 1
      if (leader && threadIdx.x == 0) {
        RepState S = s_rs;
        const int dn = s_lo.x, nacc = s_lo.y, ties = s_lo.z;
        S.trials += g.d;
        S.local_acc += nacc;
        S.near_ties += ties + gtie;
        long long nn = n_prev;
        if (nacc > 0) {
          S.global_trials += 1;
          if (G) {
            S.global_acc += 1;
            S.flips += nacc;
            nn = n_prev + dn;
            const int sbv[5] = {s_lo.w, s_hi.x, s_hi.y, s_hi.z, s_hi.w};
            double e = a.C * (double)dn;
            for (int q = 0; q < 5; ++q) e = fma((double)sbv[q], a.G[q], e);
            e += a.dF0 * (double)dn;
            S.energy += e;
          }
        }
        S.n = nn;
        const double cc = (double)nn / (double)g.n_sites;
        S.sum_c += cc;
        S.sum_c2 += cc * cc;
        S.steps += 1;
        S.step = k;
        S.fin_step = k - 1;
        s_rs = S;
      }
      if (G) n_prev += s_lo.x;  // B count at the start of step k
    }
    if (!propose) break;

    // ---- 4. propose step k
    int dn = 0, acc = 0, tie = 0;
    int sb[5] = {0, 0, 0, 0, 0};
#pragma unroll 1
    for (int t0 = 0; t0 < ntr; t0 += BS) {  // warp-uniform trip count
      const int t = t0 + threadIdx.x;
      if (t < ntr) {
        const int tq = fdiv(t, g.nxq, g.rcp_nxq);
        const int kx = t - tq * g.nxq;
        const int kzl = fdiv(tq, cy, rcp_cy);
        const int kyl = tq - kzl * cy;
        const int X = px + a.qx * kx;
        const int Y = py + a.qy * (kyb + kyl), Z = pz + a.qz * (kzb + kzl);
        const int ly = Y - v.Y0 + 2, lz = Z - v.Z0 + 2;
        int cnt[5], ts;
        if (b) cl_counts<1>(rows, v.RY, W, X, ly, lz, gm, cnt, ts);
        else cl_counts<0>(rows, v.RY, W, X, ly, lz, gm, cnt, ts);
        int tie1 = 0;
        const bool ok = lattice_accept<5>(a, lr, p, cnt, 0, ts, s_u53[t], &tie1);
        tie += tie1;
        if (ok) {
          const int H = 2 * X + b;
          flip_local(rows, T, g, v, Y, Z, H, false, true);
          const int slot = atomicAdd(&s_cnt[k & 1], 1);
          list[(k & 1) * lcap + slot] = (Y * g.nz + Z) * 2048 + H;
          acc += 1;
          dn += ts ? -1 : 1;
#pragma unroll
          for (int q = 0; q < 5; ++q) sb[q] += ts ? -cnt[q] : cnt[q];
        }
      }
    }
    // ---- 5. this CTA's sums of step k
    const bool any = __ballot_sync(0xffffffffu, acc | tie) != 0u;
    if (any) {
      dn = __reduce_add_sync(0xffffffffu, dn);
      acc = __reduce_add_sync(0xffffffffu, acc);
      tie = __reduce_add_sync(0xffffffffu, tie);
#pragma unroll
      for (int q = 0; q < 5; ++q) sb[q] = __reduce_add_sync(0xffffffffu, sb[q]);
    }
    if (lane == 0) {
      s_red[wi][0] = dn;
      s_red[wi][1] = acc;
      s_red[wi][2] = tie;
#pragma unroll
      for (int q = 0; q < 5; ++q) s_red[wi][3 + q] = sb[q];
    }
    __syncthreads();  // every change this CTA makes to its rows in step k is done
    if (threadIdx.x < CL_NF) {
      int tot = 0;
#pragma unroll
      for (int w2 = 0; w2 < BS / 32; ++w2) tot += s_red[w2][threadIdx.x];
      s_part[k & 1][threadIdx.x] = tot;
    }
    // the final values of the words changed in step k (the commits of step
    // k - 1 and the pending bits of step k) into the other CTAs' halo copies
    {
      const int na_k = s_cnt[k & 1];
      const int* lp = list + ((k - 1) & 1) * lcap;
      const int* lk = list + (k & 1) * lcap;
      for (int q = threadIdx.x; q < na_prev + na_k; q += BS) {
        const int e = q < na_prev ? lp[q] : lk[q - na_prev];
        const int H = e & 2047, yz = e >> 11;
        push_remote(rows, rows_addr, T, g, v, yz / g.nz, yz % g.nz, H);
      }
    }
    __syncthreads();  // every push issued and every read of the old list done
    if (threadIdx.x == 0) s_cnt[(k - 1) & 1] = 0;  // the list of step k + 1
    cl_arrive();
  }

  // ---- write back the owned rows (this CTA's own commits of the last step
  //      are done), then a last cluster barrier: no CTA leaves while another
  //      may still read its partial sums
  __syncthreads();
  {
    unsigned long long* dst = a.bits + g.bits_off;
    const int nwords = T.Tz * T.Ty * W;
    for (int q = threadIdx.x; q < nwords; q += BS) {
      const int w = q % W;
      const int rr = q / W;
      const int oy = rr % T.Ty, oz = rr / T.Ty;
      const int Y = v.Y0 + oy, Z = v.Z0 + oz;
      dst[((long long)Z * g.ny + Y) * W + w] = rows[((oz + 2) * v.RY + (oy + 2)) * W + w];
    }
  }
  if (leader && threadIdx.x == 0) {
    const long long kn = base + n;  // next step of the chain
    a.rs[r] = s_rs;
    a.n_start[r * 2 + (int)(kn & 1)] = s_rs.n;
    // nothing is pending: a following per-step launch finds step kn - 1
    // finalised and no accepts to decide, and a zero accumulator for kn
    StepAcc* A = a.acc + r * 3;
    for (int q = 0; q < 3; ++q) {
      A[q].dn = 0;
      A[q].nacc = 0;
      A[q].sum_de = 0.0;
      A[q].ties = 0;
      A[q].s1 = 0;
      for (int f = 0; f < 8; ++f) A[q].sb[f] = 0;
    }
  }
  cl_arrive();
  cl_wait();
}

template <int BS>
static cudaError_t cluster_launch_bs(const LatArgs& a, const ClTile* d_tiles, size_t smem, int csize, long long base,
                                     int n, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_cluster_steps<BS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cluster_steps<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.R * csize));
  cfg.blockDim = dim3(BS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cluster_steps<BS>, a, d_tiles, base, n);
}

cudaError_t launch_cluster_steps(const LatArgs& a, const ClTile* d_tiles, size_t smem, int csize, int block,
                                 long long base, int n, cudaStream_t st) {
  if (block == 256) return cluster_launch_bs<256>(a, d_tiles, smem, csize, base, n, st);
  return cluster_launch_bs<512>(a, d_tiles, smem, csize, base, n, st);
}

template <int BS>
static int cluster_capacity_bs(int csize, size_t smem) {
  if (cudaFuncSetAttribute(k_cluster_steps<BS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(k_cluster_steps<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3(BS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_cluster_steps<BS>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int cluster_capacity(int csize, int block, size_t smem) {
  return block == 256 ? cluster_capacity_bs<256>(csize, smem) : cluster_capacity_bs<512>(csize, smem);
}

}  // namespace vcsgc
