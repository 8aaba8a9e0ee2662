// common.cuh -- device-side building blocks shared by the VC-SGC kernels:
// the counter-based random stream, EAM table interpolation, the Metropolis
// test, and the argument blocks passed to the kernels by value.
//
// Method: Sadigh et al., "A scalable parallel Monte Carlo algorithm for
// atomistic simulations of precipitation in alloys" (Sec. III).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vcsgc {

constexpr double KB_EV = 8.617333262e-5;      // Boltzmann constant, eV/K
constexpr double FTM = 9.648533212331e-3;     // eV/(A amu) -> A/fs^2
constexpr int MAX_SHELLS = 16;
constexpr int MAX_OFFSETS = 256;

// device error bits, OR-ed into a context-wide status word
enum : unsigned {
  ERRF_TABLE = 1u,      // r or rho outside a table grid
  ERRF_NONFINITE = 2u,  // NaN/Inf energy difference or force
  ERRF_OVERFLOW = 4u,   // neighbour row longer than its capacity
  ERRF_TIMEOUT = 8u,    // bounded wait ran out
  ERRF_SPECIES = 16u,   // a species byte set from the host is neither 0 nor 1
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter-based: each
// (key, counter) pair gives four independent 32-bit words, so every trial of
// every colour step draws its numbers without state or communication -- the
// "synchronised seed" of Sec. III A taken to the limit.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// stream tags in the fourth counter word
constexpr uint32_t TAG_TRIAL = 0u;   // (step, domain rank): site pick + local u
constexpr uint32_t TAG_STEP = 1u;    // (step, 0xFFFFFFFF): colour + global u
constexpr uint32_t TAG_NOISE0 = 3u;  // (md step, atom): thermostat normals
constexpr uint32_t TAG_NOISE1 = 4u;
constexpr uint32_t TAG_STAGE2 = 5u;  // (step, domain rank): delayed-acceptance stage-2 u

__device__ __forceinline__ uint64_t word64(uint32_t lo, uint32_t hi) {
  return ((uint64_t)hi << 32) | lo;
}
// index in [0, m): floor(w * m / 2^64)
__device__ __forceinline__ uint64_t below64(uint32_t lo, uint32_t hi, uint64_t m) {
  return __umul64hi(word64(lo, hi), m);
}
// Site pick inside a domain (Sec. III A).  Uniform domains (n == 0): the
// index below(size).  Position-weighted domains list their sites in n <= 4
// classes of equal weight 2^sh[k], class k starting at index beg[k], with
// cum[k] the weight of classes 0..k; a draw r = below(cum[n-1]) falls in the
// class with cum[k-1] <= r < cum[k] and picks index beg[k] + (r - cum[k-1])
// / 2^sh[k], the first site whose running weight exceeds r.
struct PickTab {
  int n;
  int cum[4], beg[4], sh[4];
};
__device__ __forceinline__ int pick_index(const PickTab& t, uint32_t lo, uint32_t hi, int size) {
  if (t.n == 0) return (int)below64(lo, hi, (uint64_t)size);
  const int r = (int)below64(lo, hi, (uint64_t)t.cum[t.n - 1]);
  int k = 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) k += (q + 1 < t.n && r >= t.cum[q]) ? 1 : 0;
  const int prev = k ? t.cum[k - 1] : 0;
  return t.beg[k] + ((r - prev) >> t.sh[k]);
}
// programmatic dependent launch: wait for the preceding grid (and its
// memory), and let the next grid be scheduled; no-ops without the launch
// attribute
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// top 53 bits of the word; u = u53 * 2^-53 in [0, 1)
__device__ __forceinline__ uint64_t top53(uint32_t lo, uint32_t hi) {
  return word64(lo, hi) >> 11;
}

// --------------------------------------------------------------- splines
// Cubic on each grid interval in power form: v(t) = c0 + t(c1 + t(c2 + t c3)),
// t = x/h - j in [0, 1]; the coefficients are derived on the device from the
// caller's knot values and derivatives (Hermite data).
struct __align__(32) Cubic {
  double x, y, z, w;  // c0, c1, c2, c3
};

struct Spline {
  const Cubic* c;
  double inv_h;
  double xmax;
  int n_int;
};

struct Tables {
  Spline sp[7];   // 0..2 pair AA AB BB, 3..4 density A B, 5..6 embedding A B
  Spline dsp[7];  // derivatives d/dx of the same cubics, as quadratics (x, y, z)
};

__device__ __forceinline__ int spline_locate(const Spline& s, double x, double& t, unsigned* err) {
  if (!(x >= 0.0) || x > s.xmax) {
    atomicOr(err, ERRF_TABLE);
    t = 0.0;
    return 0;
  }
  const double u = x * s.inv_h;
  int j = (int)u;
  if (j > s.n_int - 1) j = s.n_int - 1;
  t = u - (double)j;
  return j;
}

__device__ __forceinline__ double spline_val(const Spline& s, double x, unsigned* err) {
  double t;
  const int j = spline_locate(s, x, t, err);
  const Cubic c = s.c[j];
  return fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
}

__device__ __forceinline__ double spline_val_at(const Spline& s, int j, double t) {
  const Cubic c = s.c[j];
  return fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
}

// derivative d/dx at a located point
__device__ __forceinline__ double spline_der_at(const Spline& s, int j, double t) {
  const Cubic c = s.c[j];
  return fma(t, fma(t, 3.0 * c.w, 2.0 * c.z), c.y) * s.inv_h;
}

// derivative from the derivative table: d0 + t (d1 + t d2)
__device__ __forceinline__ double spline_dval_at(const Spline& ds, int j, double t) {
  const Cubic c = ds.c[j];
  return fma(t, fma(t, c.z, c.y), c.x);
}

// 1/sqrt(r2): FP32 estimate refined by two Newton-Raphson steps in FP64,
// y <- y + y (1 - r2 y^2) / 2; each step squares the relative error, so the
// 2^-22 estimate reaches full double precision.
__device__ __forceinline__ double rsqrt_nr(double r2) {
  double y = (double)rsqrtf((float)r2);
  double e = fma(-r2 * y, y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-r2 * y, y, 1.0);
  return fma(0.5 * y, e, y);
}

// ------------------------------------------------- FP32 tables (mixed form)
// The mixed-precision form evaluates pair, density and embedding-table
// interpolants in FP32 from the same coefficients rounded to float; sums
// (rho, dE, forces) and embedding differences stay FP64.
struct __align__(16) Cubic32 {
  float x, y, z, w;
};

struct Spline32 {
  const Cubic32* c;
  float inv_h;
  float xmax;
  int n_int;
};

struct Tables32 {
  Spline32 sp[7];
  Spline32 dsp[7];
};

__device__ __forceinline__ int spline32_locate(const Spline32& s, float x, float& t, unsigned* err) {
  if (!(x >= 0.0f) || x > s.xmax) {
    atomicOr(err, ERRF_TABLE);
    t = 0.0f;
    return 0;
  }
  const float u = x * s.inv_h;
  int j = (int)u;
  if (j > s.n_int - 1) j = s.n_int - 1;
  t = u - (float)j;
  return j;
}

__device__ __forceinline__ float spline32_val_at(const Spline32& s, int j, float t) {
  const Cubic32 c = s.c[j];
  return fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x);
}

__device__ __forceinline__ float spline32_dval_at(const Spline32& ds, int j, float t) {
  const Cubic32 c = ds.c[j];
  return fmaf(t, fmaf(t, c.z, c.y), c.x);
}

// minimum-image separation in FP32 of two FP64 coordinates (difference in FP64)
// Minimum image of d = x_j - x_i for positions kept in [0, L) (so |d| < L):
// the image shift is -sign(d) L exactly when |d| > L/2, decided on the bit
// pattern of d (a non-negative double orders like its bits; hb = the bits of
// L/2), so a pair costs one FP64 FMA per axis instead of a multiply (or a
// division), a rounding and an FMA.  For every pair within a cutoff below
// L/2 it gives the double d - L rint(d / L) gives.
__device__ __forceinline__ double mimg_w(double d, double L, long long hb) {
  const long long b = __double_as_longlong(d);
  const double s = (b & 0x7fffffffffffffffLL) > hb ? (b < 0 ? 1.0 : -1.0) : 0.0;
  return fma(s, L, d);
}
__device__ __forceinline__ long long half_bits(double L) { return __double_as_longlong(0.5 * L); }

// Explicit positions of the mixed form as fixed-point fractions of the box,
// u = x / L 2^32 mod 2^32 per axis.  The difference of two words read as a
// signed 32-bit integer is the minimum-image separation in units of L 2^-32,
// exactly (wrap-around of the integer is the periodic image), so the FP32
// separation carries only the int-to-float and scale roundings (3 2^-24
// relative) and the quantisation (L 2^-33; 2.9e-8 A in a 250 A box)
// whatever the box size, with no FP64 arithmetic per pair.  ul = L 2^-32.
__device__ __forceinline__ float fix_diff(uint32_t uj, uint32_t ui, float ul) {
  return (float)(int32_t)(uj - ui) * ul;
}

// ------------------------------------------------------------ Metropolis
// Decision u < min{1, exp(-X)} with u = u53 * 2^-53, exactly as an FP64
// evaluation decides it.  GB300 runs FP32 ~60x faster than FP64, so the
// exponential is first taken in FP32 with an error margin that covers the
// rounding of X to float (|X| 2^-24 relative), expf's documented 2-ulp bound
// and the float products; only decisions inside that margin (about one in
// 10^5) fall through to the FP64 exp.  For X > 80 the FP64 p is below
// 2^-53 <= u whenever u53 >= 1, so such moves are rejected without exp.
// *tie is set when |u - p| <= 1e-9 p, where CPU and GPU exp may disagree.
// u53 as a float from two 32-bit conversions and one FMA (a 64-bit integer
// conversion would occupy the slow FP64 pipe): within 2^-23 relative
__device__ __forceinline__ float u53_float(uint64_t u53) {
  return fmaf(__uint2float_rn((uint32_t)(u53 >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)u53));
}

// u >= 1 - 1e-9 (the near-tie test at X = 0) on the integer u53: the FP64
// value nearest 1 - 1e-9 times 2^53 is an integer, computed at compile time
constexpr uint64_t U53_NEAR_ONE = (uint64_t)((1.0 - 1e-9) * 9007199254740992.0);

// FP32 screen of u < min{1, exp(-X)} given x32 with |x32 - X| <= dx:
// 1 accept, 0 reject, -1 undecided (decide in FP64).  exp(-x32) is within a
// factor exp(+-dx) of exp(-X); the relative margin dx + dx^2 covers
// exp(dx) - 1 for dx <= 1 (the second-order term matters once dx exceeds
// about 1e-3, as in the re-embedding screens), 2^-20 the expf bound and the
// float products.  Past dx = 0.5 (steep tables at low T) the screen leaves
// every decision to FP64: dx + dx^2 stops covering exp(dx) - 1 near 1.79.
__device__ __forceinline__ int screen32(float x32, float dx, uint64_t u53) {
  if (!(dx <= 0.5f)) return -1;
  if (x32 <= -2.0f * dx) return 1;
  if (u53 == 0) return -1;
  if (x32 >= 80.0f + dx) return 0;
  const float pf = expf(-x32) * 9007199254740992.0f;  // p * 2^53
  const float uf = u53_float(u53);
  const float m = fmaf(dx, dx, dx) + 9.5367431640625e-07f;
  if (uf * (1.0f + 2.384185791015625e-07f) < pf * (1.0f - m)) return 1;
  if (uf * (1.0f - 2.384185791015625e-07f) > pf * (1.0f + m)) return 0;
  return -1;
}

__device__ __forceinline__ bool metropolis(double X, uint64_t u53, int* tie) {
  if (X <= 0.0) {
    if (X > -1e-9 && u53 >= U53_NEAR_ONE) *tie = 1;
    return true;
  }
  if (u53 != 0) {
    if (X > 80.0) return false;
    const float xf = (float)X;
    const float pf = expf(-xf) * 9007199254740992.0f;  // p * 2^53
    const float uf = u53_float(u53);
    const float m = 9.5367431640625e-07f + xf * 2.384185791015625e-07f;  // 2^-20 + X 2^-22
    if (uf * (1.0f + 2.384185791015625e-07f) < pf * (1.0f - m)) return true;
    if (uf * (1.0f - 2.384185791015625e-07f) > pf * (1.0f + m)) return false;
  }
  const double p = exp(-X);
  const double u = (double)u53 * 0x1p-53;
  if (fabs(u - p) <= 1e-9 * p) *tie = 1;
  return u < p;
}

// --------------------------------------------------------- state blocks
// Per-replica ensemble parameters (Eq. pi_vcsgc, Eq. trans_vcsgc_par1).
struct RepParams {
  double beta;     // 1/(kB T)
  double kappa_p;  // eV
  double n0;       // N c0
  double dmu0;     // phi + 2 kappa_p N c0
  double phi;
  uint2 key;       // Philox key
};

// Per-replica running state, advanced by the last block of each commit.
struct RepState {
  long long n;  // B count
  long long step;
  long long fin_step;  // last finalised step (fused lattice form)
  double energy;
  long long trials, local_acc, global_trials, global_acc, flips, near_ties, steps;
  double sum_c, sum_c2;
  long long s1_acc;  // delayed acceptance: trials that passed stage 1
};

// Per-replica accumulator of one colour step (the paper's allgather of dc_i).
struct StepAcc {
  int dn;
  int nacc;
  double sum_de;
  unsigned done;
  int ties;
  int sb[8];  // fused lattice form: sum over accepted moves of s_i b_s (per shell)
  int s1;     // delayed acceptance: trials that passed stage 1
};

// Everything the colour-step kernels read, passed by value.
// FP32 embedding value of species t at x for the screened forms (Args: the
// binary or multicomponent launch arguments, with emb32 [K][emb_n] float
// cubics on one grid of 1/h = emb_ih).  Callers check x's range with
// emb32_in; j is clamped so that the load stays inside the table anyway.
template <class Args>
__device__ __forceinline__ float emb32_val(const Args& a, int t, float x) {
  const float u = x * a.emb_ih;
  int j = (int)u;
  j = j < 0 ? 0 : (j > a.emb_n - 1 ? a.emb_n - 1 : j);
  const float tt = u - (float)j;
  const float4 c = __ldg(a.emb32 + t * a.emb_n + j);
  return fmaf(tt, fmaf(tt, fmaf(tt, c.w, c.z), c.y), c.x);
}

template <class Args>
__device__ __forceinline__ bool emb32_in(const Args& a, float x) {
  return x >= a.emb_lo && x <= a.emb_hi;
}

struct McArgs {
  long long N;
  int R;
  int K;                 // neighbour row stride
  const int* nbr;        // [N][K], -1 padded
  const int* nbr_cnt;    // [N] row lengths
  uint8_t* types;        // [R][N]
  double* rho;           // [R][N] when rho_per_rep, else [N]
  int rho_per_rep;
  const double* dF;      // [N] F_B(rho_i) - F_A(rho_i) (static-density forms)
  double* vel[3];        // velocities of replica 0 or null (hybrid MC/MD)
  double mass[2];
  // shell form (rigid lattice): slots sorted by shell
  int n_shells;
  int shell_end[MAX_SHELLS];
  const double* shell_tab;  // [0] = C_A, [1+s] = G_A[s], [1+S+s] = f_B - f_A at r_s,
                            // [1+2S+s] = r_s
  // general form (explicit positions)
  const double* x;
  const double* y;
  const double* z;
  uint32_t *ux, *uy, *uz;  // fixed-point copies (mixed form; fix_diff)
  float ul[3];             // L 2^-32 per axis
  double box[3];
  double rc;
  Tables tab;
  Tables32 tab32;
  int mixed;             // FP32 table evaluation (VCSGC_PREC_MIXED)
  // schedule
  int n_colours;
  const int* col_start;
  const int* dom_start;
  const int* dom_sites;
  PickTab pick;          // site weights of overlapping domains (n = 0: uniform)
  int dmax;
  // replicas
  const RepParams* rp;
  RepState* rs;
  StepAcc* acc;
  int* acc_list;  // [R][dmax]
  unsigned* err;
  // screened re-embedding (rigid lattice, shell form): the local decision on
  // an FP32 dE within a proven bound.  Per site (rho as float, F32_t(rho)),
  // [R][N]; the embedding cubics as floats [2][emb_n]; the bound per
  // evaluation (eV) and the argument range where it holds.
  int screen;
  float2* rf;
  const float4* emb32;
  int emb_n;
  float emb_ih, emb_lo, emb_hi, emb_err;
};

}  // namespace vcsgc
