// hevi_internal.cuh -- device-side building blocks of the HEVI column solver.
//
// One column: Nez elements of LGL order N, n_z = Nez N + 1 points, n = 3 n_z
// unknowns (rho, m = rho w, Theta = rho theta), point-major (Sec. 3; set 2C
// of App. A.1 restricted to the vertical).  Band half-width K = 3(N+1) - 1
// (Sec. 4.2.3).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hevi.h"

namespace hevi {

constexpr int kMaxOrder = 5;
constexpr int kTile = 32;  // columns per tile (one warp, one column per lane)

// Band sizes and factor record layout for order N.  Per pivot step j a
// column stores a forward record F_j = {l_1..l_K, pivot offset, 1/u_jj}
// (unit-lower multipliers of Sec. 4.2.3's band LU, dgbtrf semantics) and a
// backward record B_j = {U[j-1][j], U[j-2][j], .., U[j-2K][j]}, column j of U
// above the diagonal (partial pivoting fills U to k_l + k_u = 2K
// super-diagonals); both padded to a multiple of 4.
template <int N>
struct Band {
  static constexpr int K = 3 * (N + 1) - 1;
  static constexpr int WR = K + 1;          // active window rows (forward window)
  static constexpr int WC = 2 * K + 1;      // active window columns (backward window)
  static constexpr int FR = ((K + 2) + 3) / 4 * 4;
  static constexpr int BR = ((2 * K) + 3) / 4 * 4;
  static constexpr int RL = FR + BR;        // record length per pivot step
};

// Record layout of the FP32 factors (no pivoting, equilibrated band; the L
// factor has K sub-diagonals and U has K super-diagonals).  Per pivot step j
// a column stores a forward record F_j = {l_1 .. l_K} (unit-lower multipliers
// of rows j+1 .. j+K) and a backward record B_j = {1/u_jj, u_j,j+1, ..,
// u_j,j+K} (row j of U), each padded to whole float4 vectors.  A tile keeps all F records, then all B records, each interleaved
// [step][vector][lane][4]: one step of a 32-column tile is one contiguous
// block of FV (or BV) x 512 bytes.
template <int N>
struct NpBand {
  static constexpr int K = 3 * (N + 1) - 1;
  static constexpr int FV = (K + 3) / 4;      // float4 vectors of F_j
  static constexpr int BV = (K + 1 + 3) / 4;  // float4 vectors of B_j
  static constexpr int RL = 4 * (FV + BV);    // floats per step and column
  static constexpr int WR = K + 1;            // rows of the active window
};
inline int np_record_floats(int N) {  // floats per step and column (host)
  const int K = 3 * (N + 1) - 1;
  return 4 * ((K + 3) / 4 + (K + 4) / 4);
}

// Physical constants of the isothermal reference atmosphere.
constexpr int kEosTerms = 9;
struct Phys {
  double T0, p0, R, cp, g;
  double cv, gamma, cs;   // cp - R, cp / cv, sqrt(gamma R T0)
  double bin[kEosTerms];  // C(gamma, k), k = 1 .. kEosTerms
  float binhi[kEosTerms], binlo[kEosTerms];  // the same as double-float pairs
  // FP32 constants of the equilibration scales of the FP32 path:
  // rho_bar = rho0f exp(-za z), theta_bar = T0f exp(zb z), c_s = csf
  float rho0f, za, zb, T0f, csf;
  float cvT0f, gf;  // c_v T0 and g: the set-3C energy scale rho_bar (c_v T0 + g z)
  // equation set: 0 = set 2C (rho, m, Theta), 1 = set 3C (rho, m, E; FP64 path)
  int eqset;
};
// Fill the derived fields of a Phys from T0, p0, R, cp, g (host).
inline void phys_derive(Phys& ph);

// One tile = up to 32 columns of the same size class.
struct TileDesc {
  int32_t order;      // N
  int32_t nez;        // elements
  int32_t count;      // columns in this tile (<= 32)
  int32_t first;      // index into the class-sorted column permutation
  int64_t fac_off;    // offset of the tile's factor records (elements of T)
  int64_t scr_off;    // offset of the tile's Newton scratch (floats)
  int64_t y_off;      // offset of the tile's solve vectors (floats, (n + 2K) x 32)
};

// LGL tables per order (host fills them at setup): weights w_k, Dhat_kj =
// h_j'(xi_k), and wD_kj = w_k Dhat_kj, in FP64 and FP32.
// Even-odd form of wD: LGL points are symmetric, so wD[N-k][N-j] = -wD[k][j];
// for pair rows k < P = (N+1)/2, with e_j = f_j + f_{N-j}, o_j = f_j - f_{N-j}:
//   sE_k = sum_{j<P} ep[k][j] e_j + (N even) wD[k][N/2] f_{N/2},
//   sO_k = sum_{j<P} op[k][j] o_j,   c_k = sE_k + sO_k,  c_{N-k} = sO_k - sE_k,
// and for N even the middle row c_{N/2} = sum_{j<P} om[j] o_j.
struct LglTables {
  double xi[kMaxOrder + 1][kMaxOrder + 1];
  double w[kMaxOrder + 1][kMaxOrder + 1];
  double wD[kMaxOrder + 1][(kMaxOrder + 1) * (kMaxOrder + 1)];
  float wDf[kMaxOrder + 1][(kMaxOrder + 1) * (kMaxOrder + 1)];
  float iwf[kMaxOrder + 1][kMaxOrder + 1];  // 1 / w_k
  double iw[kMaxOrder + 1][kMaxOrder + 1];  // 1 / w_k (FP64)
  // Row coefficients of the DSS'd derivative: for a point of class cls
  // (0 bottom end, 1 top end, 2 shared element boundary, 2 + k interior
  // local index k) and dJ = J - I in [-N, N], G = sum_e w_k Dhat_kj / W_I.
  float gcoef[kMaxOrder + 1][kMaxOrder + 2][2 * kMaxOrder + 1];
  double ep[kMaxOrder + 1][3][3];
  double op[kMaxOrder + 1][3][3];
  double om[kMaxOrder + 1][3];
  // the same FP64 values split into double-float pairs (hi, lo) for the
  // refinement residual: wD, 1/w and the even-odd halves
  float2 wD2[kMaxOrder + 1][(kMaxOrder + 1) * (kMaxOrder + 1)];
  float2 iw2[kMaxOrder + 1][kMaxOrder + 1];
  float2 ep2[kMaxOrder + 1][3][3];
  float2 op2[kMaxOrder + 1][3][3];
  float2 om2[kMaxOrder + 1][3];
  float xh[kMaxOrder + 1][kMaxOrder + 1];  // (xi_k + 1) / 2 in FP32
};

// Device view of a context's buffers (passed to kernels by value).
struct DevView {
  Phys ph;
  int64_t ncols;
  const int64_t* col_off;   // [ncols + 1] state offsets
  const int32_t* perm;      // [ncols] class-sorted column index
  const double* col_dz;     // [ncols] element height
  const double* ref;        // state layout: (rho_bar, P_bar, X) per point, X = Theta_bar (set
                            // 2C), E_bar (3C) or theta_bar (2NC)
  double* ithb;             // per point (index off/3 + I): 1 / X (X as in ref), or null
  double* lin;              // state layout: set 2C (w0, theta0, c0 = gamma P0 / Theta0),
                            // set 3C (w0, h0, z), set 2NC (w0, rho0, theta0)
  double* lin2;             // set 2NC only, 6 per point at 2 off + 6 I: (P_rho, P_theta,
                            // Dcal w0, Dcal[P0 - P_bar] + g (rho0 - rho_bar), Dcal theta0, 0)
  const TileDesc* tiles;
  int32_t ntiles;
  int32_t tile_begin;       // tiles [tile_begin, tile_begin + tile_count) of one order, or
  int32_t tile_count;       // entries of tile_list (the single-launch FP32 stage solve)
  const int32_t* tile_list; // if set: tile indices in decreasing column length (FP32 solve)
  int32_t* tile_next;       // [1] next tile to take (FP32 solve; zeroed before each launch)
  void* fac;                // factor records (float or double)
  float* scr;               // Newton scratch (U records)
  float* ysc;               // per tile: FP64 point coefficients of L(q0), [row][lane] (FP32 path)
  int32_t* fac_status;      // [ncols] status of the last factorisation
  int32_t* col_status;      // [ncols] status of the last call
  int32_t* col_iters;       // [ncols]
  int32_t* fail_count;      // [1]
  int32_t solve_wps;        // resident stage-solve warps per SM (0: default)
  const int32_t* gate;      // if set and *gate == 0, the factor and solve kernels do nothing
  int32_t drop_copy;        // test hook: > 0 = the record ring leaves out the copy of the
                            // chunk holding forward step drop_copy - 1 of a tile's first sweep
};

// Per-column geometry in a kernel.
struct Col {
  int64_t col;
  int64_t off;
  int nez, nz, n;
  double s;  // 2 / dz: d(xi)/dz of every element
};

// Point weight sum W_I: M_I = (dz/2) W_I (DSS of the diagonal LGL mass).
template <int N>
__device__ __forceinline__ double wsum(const double* w, int I, int nz) {
  if (I == 0 || I == nz - 1) return w[0];
  int k = I % N;
  return k == 0 ? 2.0 * w[0] : w[k];
}

// Element pass: visits the elements of a column bottom to top, asks `flux`
// for the NC (default 3) flux components at every point (once per point, in increasing
// order), forms the strong-form element derivative weighted by the LGL
// weights, sums the two contributions of shared points (DSS), and hands each
// completed point I to `out` with D_I = (Dcal f)_I =
// (1/M_I) sum_{(e,k)->I} w_k J_e (dxi/dz) sum_j Dhat_kj f_(e,j)   (Sec. 3).
// `out(I, D)` is called in increasing I, always after flux(J) for every J
// of the element holding I.
// Weighted element derivative cc[k] = sum_j w_k Dhat_kj f_j (NC components)
// in the even-odd form; reads the tables from constant memory.
template <int N, int NC>
__device__ __forceinline__ void elem_deriv(const double (&f)[N + 1][NC], double (&cc)[N + 1][NC]);

template <int N, int NC = 3, class FluxF, class OutF>
__device__ __forceinline__ void element_pass(const Col& c, const double* w, const double* iw,
                                             FluxF&& flux, OutF&& out) {
  (void)w;
  double f[N + 1][NC];
  double carry[NC] = {};
  flux(0, f[0]);
  for (int e = 0; e < c.nez; ++e) {
    const int I0 = e * N;
#pragma unroll
    for (int k = 1; k <= N; ++k) flux(I0 + k, f[k]);
    double cc[N + 1][NC];
    elem_deriv<N, NC>(f, cc);
    {
      double D[NC];
      const double sc = c.s * (e == 0 ? iw[0] : 0.5 * iw[0]);
#pragma unroll
      for (int v = 0; v < NC; ++v) D[v] = (carry[v] + cc[0][v]) * sc;
      out(I0, D);
    }
#pragma unroll
    for (int k = 1; k < N; ++k) {
      double D[NC];
      const double sc = c.s * iw[k];
#pragma unroll
      for (int v = 0; v < NC; ++v) D[v] = cc[k][v] * sc;
      out(I0 + k, D);
    }
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      carry[v] = cc[N][v];
      f[0][v] = f[N][v];
    }
  }
  double D[NC];
  const double sc = c.s * iw[0];
#pragma unroll
  for (int v = 0; v < NC; ++v) D[v] = carry[v] * sc;
  out(c.nz - 1, D);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic for the refinement residual.  A value is an
// unevaluated sum hi + lo of two floats (|lo| < ulp(hi)), about 48
// significant bits, computed on the FP32 pipes, which on this part issue at
// many times the FP64 rate.  The building blocks are the error-free
// transformations of Dekker (1971) and Knuth (TAOCP vol. 2, "TwoSum") and
// the FMA-based exact product of Ogita, Rump and Oishi (2005); additions use
// the "sloppy" double-word sum, whose error is bounded relative to |x| + |y|
// (Joldes, Muller and Popescu, 2017), which is the bound a residual
// b - A x needs.  Every operation below is written with explicit fmaf so
// that contraction cannot change it.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, {-y.hi, -y.lo}); }
__device__ __forceinline__ df df_add_f(df x, float f) {
  const df s = df_two_sum(x.hi, f);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ df df_of(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 df_pack(df v) { return make_float2(v.hi, v.lo); }
// float -> double with integer operations only (no FP64 conversion):
// exact for zero, normal, infinite and NaN values; FP32 subnormals (below
// 1.2e-38, only ever a low part here) go to zero.  hi + lo then takes one
// FP64 add.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long mant = (unsigned long long)(u & 0x7fffffu) << 29;
  if (e == 0u) return __longlong_as_double((long long)sign);
  const unsigned long long ed = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (ed << 52) | mant));
}
__device__ __forceinline__ double df_to_double(df v) { return f2d(v.hi) + f2d(v.lo); }

// Split an FP64 value into a double-float pair with integer operations only
// (no FP64 conversion): hi keeps the top 24 significand bits, lo the next 29
// (rounded to 24 by the integer-to-float conversion).  Outside 2^-63 .. 2^127
// in magnitude: below it lo is dropped (24 bits kept, an error under 1e-26)
// and below FP32's normal range (2^-126) the value goes to zero; above it
// the pair is +-Inf, and NaN stays NaN.
__device__ __forceinline__ df df_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ffu);
  const unsigned long long M = b & 0xfffffffffffffull;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (E < 897) return {__uint_as_float(sign), 0.0f};
  if (E > 1150)
    return {__uint_as_float(sign | 0x7f800000u | (E == 2047 && M ? 0x400000u : 0u)), 0.0f};
  const float hi = __uint_as_float(sign | ((unsigned)(E - 1023 + 127) << 23) | (unsigned)(M >> 29));
  if (E < 960) return {hi, 0.0f};
  const float lo = __fmul_rn(__uint2float_rn((unsigned)(M & 0x1fffffffu)),
                             __uint_as_float((unsigned)(E - 1075 + 127) << 23));
  return {hi, sign ? -lo : lo};
}

// 1/x in FP64 from an FP32 reciprocal seed and two Newton-Raphson steps
// r <- r + r (1 - x r) (quadratic: relative error ~1e-7, ~1e-14, then
// rounding), for positive x within the FP32 range; a few FP64 operations
// instead of a division.
__device__ __forceinline__ double rcp64(double x) {
  double r = (double)(1.0f / (float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Equation of state of set 2C (App. A.1): P = p0 (R Theta / p0)^gamma.
__device__ __forceinline__ double eos(const Phys& ph, double Theta) {
  return ph.p0 * pow(ph.R * Theta / ph.p0, ph.gamma);
}

// Pressure perturbation about the reference state, from the same equation of
// state: P(Theta) - P_bar = P_bar ((1 + x)^gamma - 1), x = (Theta - Theta_bar) /
// Theta_bar, exactly zero at Theta = Theta_bar and free of the cancellation of
// two O(1e5 Pa) numbers.  For |x| <= 0.02 the binomial series replaces the
// FP64 log1p/expm1 pair, which costs several times more on this part's FP64
// pipe: its first three terms in FP64, the rest (kEosTerms in all; below |x|^3
// of the leading term, truncation below 1e-19 relative) in FP32, whose
// rounding then stays below 2e-14 of the perturbation.
__device__ __forceinline__ double eos_perturbation(const Phys& ph, double Theta, double Theta_bar,
                                                   double P_bar, const double* inv_theta_bar = nullptr) {
  const double x = inv_theta_bar ? (Theta - Theta_bar) * *inv_theta_bar : (Theta - Theta_bar) / Theta_bar;
  const float xf = df_from_double(x).hi;
  if (fabsf(xf) <= 0.02f) {
    float t = ph.binhi[kEosTerms - 1];
#pragma unroll
    for (int k = kEosTerms - 2; k >= 3; --k) t = fmaf(t, xf, ph.binhi[k]);
    double s = fma(f2d(t), x, ph.bin[2]);
    s = fma(s, x, ph.bin[1]);
    s = fma(s, x, ph.bin[0]);
    return P_bar * (s * x);
  }
  return P_bar * expm1(ph.gamma * log1p(x));
}

inline void phys_derive(Phys& ph) {
  ph.eqset = 0;
  ph.cv = ph.cp - ph.R;
  ph.gamma = ph.cp / ph.cv;
  ph.cs = std::sqrt(ph.gamma * ph.R * ph.T0);
  double coef = 1.0;  // C(gamma, k) = C(gamma, k-1) (gamma - k + 1) / k
  for (int k = 1; k <= kEosTerms; ++k) {
    coef *= (ph.gamma - k + 1.0) / k;
    ph.bin[k - 1] = coef;
    ph.binhi[k - 1] = (float)coef;
    ph.binlo[k - 1] = (float)(coef - (double)ph.binhi[k - 1]);
  }
  ph.rho0f = (float)(ph.p0 / (ph.R * ph.T0));
  ph.za = (float)(ph.g / (ph.R * ph.T0));
  ph.zb = (float)(ph.g / (ph.cp * ph.T0));
  ph.T0f = (float)ph.T0;
  ph.cvT0f = (float)(ph.cv * ph.T0);
  ph.gf = (float)ph.g;
  ph.csf = (float)ph.cs;
}

// Launch helpers (host side, defined in hevi_kernels.cu).
// Reference state (and element heights' consequences) of the columns
// [first, first + count) (count < 0: to the last column).
void launch_setup_ref(const DevView& v, const int32_t* col_order, const int32_t* col_nez,
                      cudaStream_t st, int64_t first = 0, int64_t count = -1);
// The column launchers below process the tiles [v.tile_begin, v.tile_begin +
// v.tile_count), all of order `order`; ylen is the longest n + 2K among them.
void launch_factor(const DevView& v, int order, hevi_precision prec, double lam, const double* q0,
                   int ylen, cudaStream_t st);
// launch_solve: one stage solve, FP64 factors (plain) or FP32 factors with
// iterative refinement, for the tiles of one order.
void launch_solve(const DevView& v, int order, hevi_precision prec, double lam, const double* b,
                  double* x, double tol, int max_sweeps, int ylen, cudaStream_t st);
// The FP32 path (hevi_np.cu): no-pivot factorisation of the equilibrated band
// and the refined stage solve.
void launch_factor_np(const DevView& v, int order, double lam, const double* q0, int ylen,
                      cudaStream_t st);
// launch_solve_np: one persistent launch over the tiles [tile_begin,
// tile_begin + tile_count) (or, with tile_list set, over the tiles
// tile_list[tile_begin ..]); order = N when every tile has order N, else 0
// with nmax the largest order among them.  v.tile_next must be device memory.
void launch_solve_np(const DevView& v, int order, int nmax, double lam, const double* b,
                     double* x, double tol, int max_sweeps, cudaStream_t st);
// Most stage-solve warps per SM the FP32 kernel's resources allow.
int solve_np_max_warps_per_sm(int order, int nmax);
void launch_apply(const DevView& v, int order, const double* x, double* y, int nonlinear,
                  cudaStream_t st);
void launch_apply_stage(const DevView& v, int order, const double* Q, const double* H, double* E,
                        double* LQ, cudaStream_t st);
// The stage combinations an LHEVI step folds into the tendency pass of stage
// i (Sec. 4.3, Eq. lhevi-ark-final-3), every vector in the state layout.  With
// qtt set, the stage value is formed at each point as
//   Q_i = qtt + sum_t cq[t] q[t]
// (and stored to qout when set) instead of being read from Q.  With rout
// set, after S_i = H + V(Q_i) the pass writes
//   rout = rbase + sum_t cr[t] r[t] (+ cs S_i if has_s) (+ cqs Q_i if has_q),
// each sum an FMA chain in this order, as the stand-alone combination kernel
// evaluates it, so the fused step gives the same bits as the unfused one.
constexpr int kFuseQ = 8, kFuseR = 16;
struct StageFuse {
  const double* qtt = nullptr;
  int nq = 0;
  const double* q[kFuseQ] = {};
  double cq[kFuseQ] = {};
  double* qout = nullptr;
  const double* rbase = nullptr;
  double* rout = nullptr;
  int nr = 0;
  const double* r[kFuseR] = {};
  double cr[kFuseR] = {};
  int has_s = 0, has_q = 0;
  double cs = 0.0, cqs = 0.0;
};
// S = H + V(Q) in double-float arithmetic (hevi_np.cu): the FP32 path's
// explicit tendency; with fz (may be null) also the stage combinations above.
// S may be null when only rout is wanted.
void launch_apply_rhs_df(const DevView& v, int order, const double* Q, const double* H, double* S,
                         cudaStream_t st, const StageFuse* fz = nullptr);
void launch_apply_rhs(const DevView& v, int order, const double* Q, const double* H, double* S,
                      cudaStream_t st);
// The fused one-column-per-thread Newton kernel (the allocation-free entry
// point); returns the launch's error.
cudaError_t launch_newton(const DevView& v, int order, double lam, double* q, const double* R,
                          double rtol, int max_iter, int ylen, cudaStream_t st);
// Arguments of the NHEVI-GMRES column solve (Krylov scratch per tile:
// kstride = (kmax + 1) nmax 32, hstride = kmax (kmax + 3) / 2 32,
// astride = (4 kmax + 1) 32 doubles).
struct GmArgs {
  double lam, eps, rtol, gtol;
  int max_newton, kmax, nmax;
  int64_t kstride, hstride, astride;
  double* q;
  const double* R;
  double* F;
  double* Qp;
  double* Vp;
  double* Kb;
  double* Hb;
  double* Ab;
  int32_t* kits;  // per column Krylov iterations, or null
};
void launch_newton_gmres(const DevView& v, int order, const GmArgs& a, cudaStream_t st);
// NHEVI-LU as a sequence of kernels (Sec. 4.2.3): an F pass (FP64) before the
// first iteration and after each Newton update, with the band factorisation
// of J(q_m) and the refined solve J delta = -F in between.
struct NewtonArgs {
  double lam, rtol;
  int max_iter, iter;        // iter 0: the pass at the initial guess; m >= 1: after update m
  double* q;                 // state (updated in place)
  const double* R;
  const double* q0;          // initial guess
  double* rhs;               // -F(q), the next right-hand side
  const double* delta;       // the update of iteration iter (iter >= 1)
  double* f0;                // [ncols] |S^-1 F(q_0)|
  int32_t* conv;             // [ncols] 0 iterating, 1 converged, 2 stopped (status says why)
  int32_t* iters;            // [ncols]
  int32_t* status;           // [ncols]
  const int32_t* active_in;  // columns still iterating before this pass (null: all)
  int32_t* active_out;       // the pass counts the columns still iterating after it
};
void launch_newton_fpass(const DevView& v, int order, const NewtonArgs& a, cudaStream_t st);
void launch_newton_finish(const DevView& v, const NewtonArgs& a, cudaStream_t st);
void launch_combine(int64_t count, const double* base, int nterms, const double* const* vec,
                    const double* coef, double* out, cudaStream_t st);
// Reference state of the columns [first, first + count) (count < 0: to the
// last column) into q (state layout).
void launch_reference_state(const DevView& v, double* q, cudaStream_t st, int64_t first = 0,
                            int64_t count = -1);
// Copy the LGL tables into the constant memory of every kernel translation
// unit (the current device); returns the first CUDA error.
cudaError_t upload_tables(const LglTables& t);
cudaError_t upload_tables_np(const LglTables& t);
// The LGL tables of every order (built once on the host, FP64).
const LglTables& lgl_tables();

}  // namespace hevi
