// hevi_kernels.cu -- CUDA kernels of the HEVI vertical column solver (sm_103a).
//
// Work decomposition: 32 columns of one size class form a tile.  Factor
// records are interleaved per tile
//   [step j][record vector][lane][vector lane]
// so that the 32 lanes of a warp read or write one contiguous 512-byte line
// (float4 / double2) per record vector, and one pivot step of a whole tile is
// one contiguous block (what the solve's bulk copies move).  The FP32 band LU
// (k_factor_r) gives each row of a column's active window, (K+1) rows x
// (2K+1) columns (Sec. 4.2.3: partial pivoting fills U to k_l + k_u
// super-diagonals), its own thread; the FP64 LU (k_factor), the solves and
// the operator applies take one column per thread (lane of the tile's warp),
// with the exceptions each kernel states.
#include <algorithm>
#include <cstdio>

#include "hevi_internal.cuh"

namespace hevi {

__constant__ LglTables c_tab;

void upload_tables(const LglTables& t) { cudaMemcpyToSymbol(c_tab, &t, sizeof(LglTables)); }

template <int N>
__device__ __forceinline__ void elem_deriv(const double (&f)[N + 1][3], double (&cc)[N + 1][3]) {
  constexpr int P = (N + 1) / 2;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    double e[P], o[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      e[j] = f[j][v] + f[N - j][v];
      o[j] = f[j][v] - f[N - j][v];
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      double sE = (N % 2 == 0) ? c_tab.wD[N][k * (N + 1) + N / 2] * f[N / 2][v] : 0.0;
      double sO = 0.0;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        sE = fma(c_tab.ep[N][k][j], e[j], sE);
        sO = fma(c_tab.op[N][k][j], o[j], sO);
      }
      cc[k][v] = sE + sO;
      cc[N - k][v] = sO - sE;
    }
    if (N % 2 == 0) {
      double sm = 0.0;
#pragma unroll
      for (int j = 0; j < P; ++j) sm = fma(c_tab.om[N][j], o[j], sm);
      cc[N / 2][v] = sm;
    }
  }
}

// One field of elem_deriv_df.
template <int N>
__device__ __forceinline__ void elem_deriv_df1(const df (&f)[N + 1], df (&cc)[N + 1]) {
  constexpr int P = (N + 1) / 2;
  df e[P], o[P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    e[j] = df_add(f[j], f[N - j]);
    o[j] = df_sub(f[j], f[N - j]);
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    df sE = df_mul(df_of(c_tab.ep2[N][k][0]), e[0]);
    df sO = df_mul(df_of(c_tab.op2[N][k][0]), o[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) {
      sE = df_fma(df_of(c_tab.ep2[N][k][j]), e[j], sE);
      sO = df_fma(df_of(c_tab.op2[N][k][j]), o[j], sO);
    }
    if (N % 2 == 0) sE = df_fma(df_of(c_tab.wD2[N][k * (N + 1) + N / 2]), f[N / 2], sE);
    cc[k] = df_add(sE, sO);
    cc[N - k] = df_sub(sO, sE);
  }
  if (N % 2 == 0) {
    df sm = df_mul(df_of(c_tab.om2[N][0]), o[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) sm = df_fma(df_of(c_tab.om2[N][j]), o[j], sm);
    cc[N / 2] = sm;
  }
}

// element_pass in double-float arithmetic for one thread's column, with the
// element's point fluxes and derivatives parked in the thread's own slots of
// shared memory (sm: (2N + 1) x 3 pairs per lane, lane fastest) so that one
// field at a time is live in registers.  flux(I, f[3]) gives the point
// fluxes, out(I, D[3]) receives the DSS'd derivative; cs = 2 / dz.
template <int N, class FluxF, class OutF>
__device__ __forceinline__ void element_pass_df(int nez, df cs, float2* sm, int lane, FluxF&& flux,
                                                OutF&& out) {
  auto FS = [&](int k, int v) -> float2& { return sm[(k * 3 + v) * kTile + lane]; };
  auto DS = [&](int k, int v) -> float2& { return sm[((N + 1 + k) * 3 + v) * kTile + lane]; };
  df carry[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  {
    df f[3];
    flux(0, f);
#pragma unroll
    for (int v = 0; v < 3; ++v) FS(0, v) = df_pack(f[v]);
  }
  const df iw0 = df_of(c_tab.iw2[N][0]);
  for (int e = 0; e < nez; ++e) {
    const int I0 = e * N;
#pragma unroll
    for (int k = 1; k <= N; ++k) {
      df f[3];
      flux(I0 + k, f);
#pragma unroll
      for (int v = 0; v < 3; ++v) FS(k, v) = df_pack(f[v]);
    }
    const df sc0 = df_mul(cs, e == 0 ? iw0 : df{0.5f * iw0.hi, 0.5f * iw0.lo});
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      df fv[N + 1], cc[N + 1];
#pragma unroll
      for (int k = 0; k <= N; ++k) fv[k] = df_of(FS(k, v));
      elem_deriv_df1<N>(fv, cc);
      DS(0, v) = df_pack(df_mul(df_add(carry[v], cc[0]), sc0));
#pragma unroll
      for (int k = 1; k < N; ++k) DS(k, v) = df_pack(df_mul(cc[k], df_mul(cs, df_of(c_tab.iw2[N][k]))));
      carry[v] = cc[N];
      FS(0, v) = FS(N, v);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const df D[3] = {df_of(DS(k, 0)), df_of(DS(k, 1)), df_of(DS(k, 2))};
      out(I0 + k, D);
    }
  }
  const df sc = df_mul(cs, iw0);
  const df D[3] = {df_mul(carry[0], sc), df_mul(carry[1], sc), df_mul(carry[2], sc)};
  out(nez * N, D);
}

// ---------------------------------------------------------------------------
// Record addressing
// ---------------------------------------------------------------------------
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int W = 2;
};

// A tile's records: the F block (n steps x FR values x 32 lanes) followed by
// the B block (n steps x BR values x 32 lanes), each [j][vector][lane][W].
template <int N, typename T>
__device__ __forceinline__ T* frec_vec(T* tile_base, int j, int e, int lane) {
  constexpr int W = Vec<T>::W;
  constexpr int NV = Band<N>::FR / W;
  return tile_base + ((int64_t)(j * NV + e / W) * kTile + lane) * W;
}
template <int N, typename T>
__device__ __forceinline__ T* brec_vec(T* tile_base, int n, int j, int e, int lane) {
  constexpr int W = Vec<T>::W;
  constexpr int NV = Band<N>::BR / W;
  return tile_base + (int64_t)n * Band<N>::FR * kTile + ((int64_t)(j * NV + e / W) * kTile + lane) * W;
}

// Record a per-column failure; counters: [0] any, [1] singular, [2] not
// converged, [3] bad input, [4] a device wait past its limit.
__device__ __forceinline__ void fail(const DevView& v, int64_t col, int code) {
  v.col_status[col] = code;
  atomicAdd(v.fail_count, 1);
  atomicAdd(v.fail_count + (code == HEVI_COL_SINGULAR        ? 1
                            : code == HEVI_COL_NOT_CONVERGED ? 2
                            : code == HEVI_COL_WAIT_TIMEOUT  ? 4
                                                             : 3),
            1);
}

__device__ __forceinline__ Col make_col(const DevView& v, const TileDesc& t, int lane, int N) {
  Col c;
  c.col = v.perm[t.first + lane];
  c.off = v.col_off[c.col];
  c.nez = t.nez;
  c.nz = t.nez * N + 1;
  c.n = 3 * c.nz;
  c.s = 2.0 / v.col_dz[c.col];
  return c;
}

// A tile's refinement scratch, every array interleaved [row][lane] so that a
// warp's 32 columns read and write one contiguous line per row: the work
// vector y (FP32, n + 2K + 4 rows), the iterate x, the right-hand side b and
// the point coefficients (w, theta, c) of L(q0) (FP64, n rows each), and the
// scales S, S^-1 (FP32, n rows each).
struct TileScr {
  float* y;
  double *x, *b, *lin;
  float *s, *is;
};
__device__ __forceinline__ TileScr tile_scratch(const DevView& v, const TileDesc& t) {
  const int64_t n = 3 * ((int64_t)t.nez * t.order + 1), K = 3 * (t.order + 1) - 1;
  TileScr r;
  r.y = v.ysc + t.y_off;
  r.x = reinterpret_cast<double*>(r.y + (n + 2 * K + 4) * kTile);
  r.b = r.x + n * kTile;
  r.lin = r.b + n * kTile;
  r.s = reinterpret_cast<float*>(r.lin + n * kTile);
  r.is = r.s + n * kTile;
  return r;
}

// ---------------------------------------------------------------------------
// Setup: reference state per point (isothermal, hydrostatic) and rest state
// ---------------------------------------------------------------------------
__global__ void k_setup_ref(DevView v, const int32_t* col_order, const int32_t* col_nez) {
  int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= v.ncols) return;
  const int N = col_order[col], nez = col_nez[col], nz = nez * N + 1;
  const double dz = v.col_dz[col];
  const Phys ph = v.ph;
  const double Hs = ph.R * ph.T0 / ph.g;
  double* r = const_cast<double*>(v.ref) + v.col_off[col];
  for (int I = 0; I < nz; ++I) {
    int e = I / N;
    if (e == nez) e = nez - 1;
    const int k = I - e * N;
    double z = e * dz + (c_tab.xi[N][k] + 1.0) * 0.5 * dz;
    if (I == 0) z = 0.0;
    if (I == nz - 1) z = nez * dz;
    const double rho = ph.p0 / (ph.R * ph.T0) * exp(-z / Hs);
    const double th = ph.T0 * exp(ph.g * z / (ph.cp * ph.T0));
    const double Th = rho * th;
    r[3 * I + 0] = rho;
    r[3 * I + 1] = eos(ph, Th);
    r[3 * I + 2] = Th;
    if (v.ithb) v.ithb[v.col_off[col] / 3 + I] = 1.0 / Th;
    if (v.s32) {
      const int64_t a = v.col_off[col] + 3 * I;
      const double sc[3] = {rho, rho * ph.cs, Th};
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        v.s32[a + u] = (float)sc[u];
        v.is32[a + u] = (float)(1.0 / sc[u]);
      }
    }
  }
}

// Interleaved copies of S and S^-1 in each tile's refinement scratch.
__global__ void k_setup_tile_scales(DevView v) {
  const TileDesc t = v.tiles[blockIdx.x];
  const int lane = threadIdx.x;
  if (lane >= t.count) return;
  const TileScr sc = tile_scratch(v, t);
  const int64_t off = v.col_off[v.perm[t.first + lane]];
  const int n = 3 * (t.nez * t.order + 1);
  for (int i = 0; i < n; ++i) {
    sc.s[(int64_t)i * kTile + lane] = v.s32[off + i];
    sc.is[(int64_t)i * kTile + lane] = v.is32[off + i];
  }
}

void launch_setup_ref(const DevView& v, const int32_t* col_order, const int32_t* col_nez,
                      cudaStream_t st) {
  int blk = 128;
  k_setup_ref<<<(unsigned)((v.ncols + blk - 1) / blk), blk, 0, st>>>(v, col_order, col_nez);
  if (v.ysc && v.ntiles > 0) k_setup_tile_scales<<<(unsigned)v.ntiles, kTile, 0, st>>>(v);
}

__global__ void k_reference_state(DevView v, double* q) {
  int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= v.ncols) return;
  const int64_t a = v.col_off[col], b = v.col_off[col + 1];
  for (int64_t i = a; i < b; i += 3) {
    q[i] = v.ref[i];
    q[i + 1] = 0.0;
    q[i + 2] = v.ref[i + 2];
  }
}

void launch_reference_state(const DevView& v, double* q, cudaStream_t st) {
  int blk = 128;
  k_reference_state<<<(unsigned)((v.ncols + blk - 1) / blk), blk, 0, st>>>(v, q);
}

// ---------------------------------------------------------------------------
// Linearisation coefficients per point: w = m/rho, theta = Theta/rho and
// c = dP/dTheta = gamma P / Theta; these are the entries of the flux
// Jacobian K (App. A.3 restricted to the vertical):
//   rho-flux (0, 1, 0);  m-flux (-w^2, 2w, c);  Theta-flux (-theta w, theta, w)
// Returns false on a non-physical state.
// ---------------------------------------------------------------------------
// dP receives P(Theta) - P_bar; ithb (optional) points at 1 / Theta_bar.
__device__ __forceinline__ bool lin_coefs(const Phys& ph, double rho, double m, double Th,
                                          double Th_bar, double P_bar, double* w, double* th,
                                          double* c, double* dP, const double* ithb = nullptr) {
  if (!(rho > 0.0) || !(Th > 0.0) || !isfinite(m)) return false;
  const double ir = rcp64(rho);
  *w = m * ir;
  *th = Th * ir;
  *dP = eos_perturbation(ph, Th, Th_bar, P_bar, ithb);
  *c = ph.gamma * (P_bar + *dP) * rcp64(Th);
  return true;
}

// ---------------------------------------------------------------------------
// Band assembly of one row of A = I + Lambda Dcal K(q0) + Lambda G into the
// shared-memory window (Sec. 4.2.3, App. A.3):
//   A[(I,v),(J,u)] = delta + Lambda (2/dz)/W_I sum_{e containing I and J}
//                    w_k(I) Dhat_k(I),j(J) K_vu(J) + Lambda g [v=m, u=rho, I=J],
// m-rows of the two end points replaced by identity rows (w = 0).
// With SCALED the row is equilibrated: A_hat = S^-1 A S with the reference
// scales S = (rho_bar, rho_bar c_s, Theta_bar).
// ---------------------------------------------------------------------------
template <int N, typename T, bool SCALED>
__device__ __forceinline__ void assemble_row(const DevView& v, const Col& c, double lam, int i,
                                             T* win, int stride, int rs, int col0, int cs0) {
  constexpr int K = Band<N>::K, WC = Band<N>::WC;
  T* row = win + (rs * WC) * stride;
#pragma unroll
  for (int s = 0; s < WC; ++s) row[s * stride] = T(0);
  auto slot = [&](int col) {
    int s = cs0 + (col - col0);
    return s >= WC ? s - WC : s;
  };
  const int I = i / 3, vv = i - 3 * I;
  if (vv == 1 && (I == 0 || I == c.nz - 1)) {
    row[slot(i) * stride] = T(1);
    return;
  }
  const double* w = c_tab.w[N];
  const double* lin = v.lin + c.off;
  const double* ref = v.ref + c.off;
  const double cs = v.ph.cs;
  auto scale = [&](int idx) -> double {  // S entry of unknown idx
    const int P = idx / 3, u = idx - 3 * P;
    const double rb = ref[3 * P];
    return u == 0 ? rb : (u == 1 ? rb * cs : ref[3 * P + 2]);
  };
  const T inv_si = SCALED ? T(1.0 / scale(i)) : T(1);
  const T fac = T(lam * c.s / wsum<N>(w, I, c.nz));
  // elements containing point I and I's local index in each
  int e_lo, e_hi;
  if (I % N == 0) {
    e_lo = I / N - 1;
    e_hi = I / N;
  } else {
    e_lo = e_hi = I / N;
  }
  if (e_lo < 0) e_lo = 0;
  if (e_hi > c.nez - 1) e_hi = c.nez - 1;
  for (int e = e_lo; e <= e_hi; ++e) {
    const int kI = I - e * N;
#pragma unroll
    for (int j = 0; j <= N; ++j) {
      const int J = e * N + j;
      T g;
      if constexpr (sizeof(T) == 4)
        g = fac * c_tab.wDf[N][kI * (N + 1) + j];
      else
        g = fac * c_tab.wD[N][kI * (N + 1) + j];
      const T wJ = T(lin[3 * J]), thJ = T(lin[3 * J + 1]), cJ = T(lin[3 * J + 2]);
      T kv0, kv1, kv2;
      if (vv == 0) {
        kv0 = T(0); kv1 = T(1); kv2 = T(0);
      } else if (vv == 1) {
        kv0 = -wJ * wJ; kv1 = T(2) * wJ; kv2 = cJ;
      } else {
        kv0 = -thJ * wJ; kv1 = thJ; kv2 = wJ;
      }
      if (SCALED) {
        kv0 *= T(scale(3 * J)) * inv_si;
        kv1 *= T(scale(3 * J + 1)) * inv_si;
        kv2 *= T(scale(3 * J + 2)) * inv_si;
      }
      const int b = 3 * J;
      row[slot(b) * stride] += g * kv0;
      row[slot(b + 1) * stride] += g * kv1;
      row[slot(b + 2) * stride] += g * kv2;
    }
  }
  row[slot(i) * stride] += T(1);
  if (vv == 1) {
    T gg = T(lam * v.ph.g);
    if (SCALED) gg *= T(scale(i - 1)) * inv_si;
    row[slot(i - 1) * stride] += gg;
  }
  (void)K;
}

// ---------------------------------------------------------------------------
// Band LU with partial pivoting of one column in the shared-memory window
// (LAPACK dgbtrf semantics: pivot = first row of maximal |a| among rows
// j..j+k_l; swap over the fill extent; unit-lower multipliers; rank-1 update).
// The assembly of row j+K+1 happens as the window advances.  `emit(j, l[],
// invd, piv, u[])` receives the finished pivot step; with FWD the L part is
// also applied right away to the right-hand side y (Newton).
// Returns info (0, or 1 + first zero-pivot step).
// ---------------------------------------------------------------------------
template <int N, typename T, bool SCALED, class Emit>
__device__ int band_lu(const DevView& v, const Col& c, double lam, T* win, int stride,
                       Emit&& emit) {
  constexpr int K = Band<N>::K, WR = Band<N>::WR, WC = Band<N>::WC;
  const int n = c.n;
  for (int i = 0; i <= K && i < n; ++i) assemble_row<N, T, SCALED>(v, c, lam, i, win, stride, i, 0, 0);
  for (int i = n; i <= K; ++i) {  // rows past the end of a tiny column
    T* row = win + (i * WC) * stride;
    for (int s = 0; s < WC; ++s) row[s * stride] = T(0);
  }
  int info = 0;
  int rb = 0, cb = 0;
  auto W = [&](int r, int cc) -> T& {
    int rs = rb + r;
    rs = rs >= WR ? rs - WR : rs;
    int cs = cb + cc;
    cs = cs >= WC ? cs - WC : cs;
    return win[(rs * WC + cs) * stride];
  };
  for (int j = 0; j < n; ++j) {
    const int nr = min(K, n - 1 - j);
    const int ncol = min(2 * K, n - 1 - j);
    // pivot search: first maximal |a|
    int p = 0;
    T amax = fabs(W(0, 0));
#pragma unroll
    for (int r = 1; r <= K; ++r) {
      if (r <= nr) {
        const T a = fabs(W(r, 0));
        if (a > amax) {
          amax = a;
          p = r;
        }
      }
    }
    T l[K];
    T invd;
    if (amax == T(0)) {
      if (info == 0) info = j + 1;
      invd = T(0);
#pragma unroll
      for (int r = 0; r < K; ++r) l[r] = T(0);
    } else {
      if (p != 0) {
#pragma unroll
        for (int cc = 0; cc <= 2 * K; ++cc) {
          if (cc <= ncol) {
            T t = W(0, cc);
            W(0, cc) = W(p, cc);
            W(p, cc) = t;
          }
        }
      }
      invd = T(1) / W(0, 0);
#pragma unroll
      for (int r = 1; r <= K; ++r) l[r - 1] = (r <= nr) ? W(r, 0) * invd : T(0);
#pragma unroll 4
      for (int cc = 1; cc <= 2 * K; ++cc) {
        if (cc <= ncol) {
          const T u = W(0, cc);
#pragma unroll
          for (int r = 1; r <= K; ++r)
            if (r <= nr) W(r, cc) -= l[r - 1] * u;
        }
      }
    }
    emit(j, l, invd, p, [&](int cc) -> T { return cc <= ncol ? W(0, cc) : T(0); });
    // advance: column j leaves, column j+2K+1 enters (zero fill for rows
    // j+1..j+K); row j leaves, row j+K+1 enters (assembled).
#pragma unroll
    for (int r = 1; r <= K; ++r) W(r, 0) = T(0);
    const int inew = j + K + 1;
    const int rs_new = rb, cs_next = (cb + 1 == WC) ? 0 : cb + 1;
    if (inew < n) {
      assemble_row<N, T, SCALED>(v, c, lam, inew, win, stride, rs_new, j + 1, cs_next);
    } else {
      T* row = win + (rs_new * WC) * stride;
      for (int s = 0; s < WC; ++s) row[s * stride] = T(0);
    }
    rb = (rb + 1 == WR) ? 0 : rb + 1;
    cb = cs_next;
  }
  return info;
}

// ---------------------------------------------------------------------------
// Factor kernel: linearisation coefficients, assembly, band LU, records out.
// ---------------------------------------------------------------------------
template <int N, typename T, bool SCALED>
__device__ void factor_column(const DevView& v, const TileDesc& t, int lane, double lam,
                              const double* q0, T* win, int stride) {
  constexpr int K = Band<N>::K;
  constexpr int W = Vec<T>::W;
  using V = typename Vec<T>::type;
  const Col c = make_col(v, t, lane, N);
  const Phys ph = v.ph;
  bool ok = true;
  for (int I = 0; I < c.nz; ++I) {
    const int64_t a = c.off + 3 * I;
    double rho, m, Th;
    if (q0) {
      rho = q0[a]; m = q0[a + 1]; Th = q0[a + 2];
    } else {
      rho = v.ref[a]; m = 0.0; Th = v.ref[a + 2];
    }
    double w, th, cc, dP;
    if (!lin_coefs(ph, rho, m, Th, v.ref[a + 2], v.ref[a + 1], &w, &th, &cc, &dP)) {
      ok = false;
      w = 0.0; th = 0.0; cc = 0.0;
    }
    v.lin[a] = w;
    v.lin[a + 1] = th;
    v.lin[a + 2] = cc;
  }
  T* base = reinterpret_cast<T*>(v.fac) + t.fac_off;
  constexpr int FR = Band<N>::FR;
  const int n = c.n;
  const int info = band_lu<N, T, SCALED>(
      v, c, lam, win, stride, [&](int j, const T* l, T invd, int p, auto&& U) {
        // forward record {l_1..l_K, p, 1/u_jj}
        T rec[FR];
#pragma unroll
        for (int r = 0; r < K; ++r) rec[r] = l[r];
        rec[K] = T(p);
        rec[K + 1] = invd;
#pragma unroll
        for (int r = K + 2; r < FR; ++r) rec[r] = T(0);
#pragma unroll
        for (int q = 0; q < FR; q += W) {
          V* dst = reinterpret_cast<V*>(frec_vec<N, T>(base, j, q, lane));
          if constexpr (W == 4)
            *dst = make_float4(rec[q], rec[q + 1], rec[q + 2], rec[q + 3]);
          else
            *dst = make_double2(rec[q], rec[q + 1]);
        }
        // row j of U goes to the backward records of columns j+1..j+2K
#pragma unroll
        for (int cc = 1; cc <= 2 * K; ++cc) {
          if (j + cc < n) brec_vec<N, T>(base, n, j + cc, cc - 1, lane)[(cc - 1) % W] = U(cc);
        }
        // entries of B_j that no row reaches (rows j-c < 0) and the padding
#pragma unroll
        for (int cc = 1; cc <= Band<N>::BR; ++cc) {
          if (cc > j || cc > 2 * K) brec_vec<N, T>(base, n, j, cc - 1, lane)[(cc - 1) % W] = T(0);
        }
      });
  int st = HEVI_COL_OK;
  if (!ok)
    st = HEVI_COL_BAD_INPUT;
  else if (info)
    st = HEVI_COL_SINGULAR;
  v.fac_status[c.col] = st;
  if (st != HEVI_COL_OK)
    fail(v, c.col, st);
  else
    v.col_status[c.col] = HEVI_COL_OK;
  v.col_iters[c.col] = 0;
}

template <int N, typename T, bool SCALED>
__global__ void __launch_bounds__(64) k_factor(DevView v, double lam, const double* q0) {
  extern __shared__ unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  T* win = smem + threadIdx.x;
  const int stride = blockDim.x;
  factor_column<N, T, SCALED>(v, t, lane, lam, q0, win, stride);
}

// shared-memory floats reserved for the row coefficient table
constexpr int kGSz = (kMaxOrder + 2) * (2 * kMaxOrder + 1) + 3;

// Row data of A_hat = S^-1 (I + Lambda Dcal K(q0) + Lambda G) S for row i:
// point I, variable v, point class (0 bottom end, 1 top end, 2 shared element
// boundary, 2 + k interior local index k), 1/s_i, identity row (m at an end).
struct RowInfo {
  int i, I, v, cls;
  float isi;
  bool ident;
};

template <int N>
__device__ __forceinline__ RowInfo row_info(const Col& c, const float* is32, int i) {
  RowInfo r;
  r.i = i;
  r.I = i / 3;
  r.v = i - 3 * r.I;
  const int k = r.I % N;
  r.cls = (r.I == 0) ? 0 : (r.I == c.nz - 1 ? 1 : (k == 0 ? 2 : 2 + k));
  r.ident = (r.v == 1) && (r.I == 0 || r.I == c.nz - 1);
  r.isi = is32[i];
  return r;
}

// Entry (i, col) of A_hat in FP32 (Sec. 4.2.3, App. A.3): delta + Lambda (2/dz)
// G[cls][J-I] K_vu(q0_J) s_col / s_i + Lambda g [v=m, u=rho, J=I] s_col / s_i,
// with the point coefficients (w, theta, gamma P / Theta) of q0 in lin32.
template <int N>
__device__ __forceinline__ float ahat_entry(const RowInfo& ri, int col, const float* lin32,
                                            const float* s32, const float* G, float lam_s,
                                            float lam_g) {
  if (ri.ident) return col == ri.i ? 1.0f : 0.0f;
  const int J = col / 3, u = col - 3 * J, dJ = J - ri.I;
  float a = (col == ri.i) ? 1.0f : 0.0f;
  const float sr = s32[col] * ri.isi;
  if (ri.v == 1 && u == 0 && dJ == 0) a = fmaf(lam_g, sr, a);
  if (dJ < -N || dJ > N) return a;
  const float g = G[ri.cls * (2 * N + 1) + dJ + N];
  const float w = lin32[3 * J], th = lin32[3 * J + 1];
  float kvu;
  if (ri.v == 0)
    kvu = (u == 1) ? 1.0f : 0.0f;
  else if (ri.v == 1)
    kvu = (u == 0) ? -w * w : (u == 1 ? 2.0f * w : lin32[3 * J + 2]);
  else
    kvu = (u == 0) ? -th * w : (u == 1 ? th : w);
  return fmaf(lam_s * g * kvu, sr, a);
}

// ---------------------------------------------------------------------------
// Row-per-thread FP32 factorisation (Sec. 4.2.3 band LU, dgbtrf semantics).
//
// One thread per row of the column's active window ((K+1) rows, 2K+1
// columns of A_hat = S^-1 A S): GW threads per column (the power of two >=
// K+1), 32/GW columns per warp.  A thread keeps its row's 2K+1 entries in
// registers at positions relative to the pivot column (a[s] = column j+s),
// so every position is a compile-time register and the window's shift by one
// column per step is folded into the update (a[s] <- a[s+1] - l u[s]).
// Interchanges swap row labels between threads instead of moving entries.  At step j: a width-GW shuffle argmax over (|a_ij|, row label)
// finds the pivot (first maximal |a|); the pivot row publishes its 2K entries
// of U's row j through shared memory; every other row forms its multiplier
// and updates its 2K entries from registers; the pivot row's thread retires
// and takes the row that enters the window, which the group assembled during
// the step (entries of S^-1 A S from FP64 point coefficients).  Records are
// written in the layout of the solves: per step an L record {l_1..l_K, pivot
// offset, 1/u_jj} and column-oriented U records.
// ---------------------------------------------------------------------------
template <int N>
struct FRow {
  static constexpr int K = Band<N>::K, WR = Band<N>::WR, WC = Band<N>::WC;
  static constexpr int GW = WR <= 8 ? 8 : (WR <= 16 ? 16 : 32);  // threads per column
  static constexpr int CPW = 32 / GW;                              // columns per warp
  static constexpr int CPB = CPW * 4;                              // columns per 4-warp block
  static constexpr int UB = ((2 * K + 3) / 4) * 4;                 // U row buffer (floats)
  static constexpr int RB = ((WC + 3) / 4) * 4;                    // entering-row buffer
};
constexpr int kGSzA = (kGSz + 3) / 4 * 4;  // coefficient table, 16-byte aligned

template <int N>
__global__ void __launch_bounds__(128) k_factor_r(DevView v, double lam, const double* q0,
                                                  int linstride) {
  using P = FRow<N>;
  constexpr int K = P::K, WR = P::WR, WC = P::WC, GW = P::GW, FRn = Band<N>::FR;
  constexpr int BR = Band<N>::BR;
  constexpr int NG = (N + 2) * (2 * N + 1);
  extern __shared__ __align__(16) float fr_smem[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int sub = lane / GW, r = lane % GW;
  constexpr int bpt = kTile / P::CPB;  // blocks per tile
  const int64_t tile = v.tile_begin + blockIdx.x / bpt;
  const TileDesc t = v.tiles[tile];
  const int cl0 = (blockIdx.x % bpt) * P::CPB;
  float* G = fr_smem;
  for (int k = threadIdx.x; k < NG; k += blockDim.x)
    G[k] = c_tab.gcoef[N][k / (2 * N + 1)][k % (2 * N + 1)];
  __syncthreads();
  if (cl0 + warp * P::CPW >= t.count) return;  // warp-uniform: no column for this warp
  const int colw = warp * P::CPW + sub;
  const bool active = cl0 + colw < t.count;
  // groups past the tile's last column shadow it without writing anything
  const int cl = active ? cl0 + colw : t.count - 1;
  const Col c = make_col(v, t, cl, N);
  const Phys ph = v.ph;
  float* ubuf = fr_smem + kGSzA + (int64_t)colw * (2 * P::UB + 2 * P::RB + linstride);
  float* rbuf = ubuf + 2 * P::UB;
  float* lin32 = rbuf + 2 * P::RB;
  const float* s32 = v.s32 + c.off;
  const float* is32 = v.is32 + c.off;
  float* tb = reinterpret_cast<float*>(v.fac) + t.fac_off;
  float* bb = tb + (int64_t)c.n * FRn * kTile;
  const int n = c.n;
  double* lin_t = tile_scratch(v, t).lin;

  // point coefficients of L(q0) (FP64): w, theta, c = gamma P / Theta
  bool ok = true;
  for (int I = r; I < c.nz; I += GW) {
    const int64_t a = c.off + 3 * I;
    double rho, m, Th;
    if (q0) {
      rho = q0[a]; m = q0[a + 1]; Th = q0[a + 2];
    } else {
      rho = v.ref[a]; m = 0.0; Th = v.ref[a + 2];
    }
    double w, th, cc, dP;
    if (!lin_coefs(ph, rho, m, Th, v.ref[a + 2], v.ref[a + 1], &w, &th, &cc, &dP,
                   v.ithb ? v.ithb + c.off / 3 + I : nullptr)) {
      ok = false;
      w = th = cc = 0.0;
    }
    if (active) {
      v.lin[a] = w;
      v.lin[a + 1] = th;
      v.lin[a + 2] = cc;
      double* lt = lin_t + (int64_t)(3 * I) * kTile + cl;
      lt[0] = w;
      lt[kTile] = th;
      lt[2 * kTile] = cc;
    }
    lin32[3 * I] = (float)w;
    lin32[3 * I + 1] = (float)th;
    lin32[3 * I + 2] = (float)cc;
  }
  {  // AND over the group's lanes (every lane of the warp takes part)
    int okv = ok ? 1 : 0;
#pragma unroll
    for (int off = 1; off < GW; off <<= 1) okv &= __shfl_xor_sync(0xffffffffu, okv, off, GW);
    ok = okv != 0;
  }
  __syncwarp();
  const float lam_s = (float)(lam * c.s), lam_g = (float)(lam * ph.g);

  // initial window: thread r holds row r; a[s] is the entry of column j + s
  float a[WC];
  int label = r < WR ? r : -1;
  {
    const bool has = r < WR && r < n;
    const RowInfo ri = row_info<N>(c, is32, has ? r : 0);
#pragma unroll
    for (int cc = 0; cc < WC; ++cc)
      a[cc] = (has && cc < n && cc <= r + K) ? ahat_entry<N>(ri, cc, lin32, s32, G, lam_s, lam_g)
                                             : 0.0f;
  }

  int info = 0;
  for (int j = 0; j < n; ++j) {
    const int buf = j & 1;
    float* ub = ubuf + buf * P::UB;
    float* rb = rbuf + buf * P::RB;
    // the row that enters after this step, j+K+1, entries of columns j+1+s:
    // lane r <= 2N takes the three columns of point J = I + r - N (they share
    // the coefficient G[cls][J-I] and J's linearisation); lane 2N+1 clears the
    // two slots of the band that no point within N of I reaches
    {
      const int inew = j + K + 1;
      const bool live = inew < n;
      const RowInfo ri = row_info<N>(c, is32, live ? inew : 0);
      if (r <= 2 * N) {
        const int dJ = r - N, J = ri.I + dJ;
        const int s0 = 3 * dJ - ri.v + K;  // slot of (J, u = 0), in [2 - v, 2K - v - 2]
        float e[3] = {0.0f, 0.0f, 0.0f};
        if (live && J >= 0 && J < c.nz) {
          if (ri.ident) {
#pragma unroll
            for (int u = 0; u < 3; ++u) e[u] = (3 * J + u == inew) ? 1.0f : 0.0f;
          } else {
            const float g = G[ri.cls * (2 * N + 1) + dJ + N];
            const float w = lin32[3 * J], th = lin32[3 * J + 1];
            float kv[3];
            if (ri.v == 0) {
              kv[0] = 0.0f; kv[1] = 1.0f; kv[2] = 0.0f;
            } else if (ri.v == 1) {
              kv[0] = -w * w; kv[1] = 2.0f * w; kv[2] = lin32[3 * J + 2];
            } else {
              kv[0] = -th * w; kv[1] = th; kv[2] = w;
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              const int col = 3 * J + u;
              float a0 = (col == inew) ? 1.0f : 0.0f;
              const float sr = s32[col] * ri.isi;
              if (ri.v == 1 && u == 0 && dJ == 0) a0 = fmaf(lam_g, sr, a0);
              e[u] = fmaf(lam_s * g * kv[u], sr, a0);
            }
          }
        }
        rb[s0] = e[0];
        rb[s0 + 1] = e[1];
        rb[s0 + 2] = e[2];
      } else if (r == 2 * N + 1) {
        // uncovered slots: s < 2 - v and s > 2K - v
        const int v0 = live ? ri.v : 0;
        for (int s = 0; s < 2 - v0; ++s) rb[s] = 0.0f;
        for (int s = 2 * K - v0 + 1; s < WC; ++s) rb[s] = 0.0f;
      }
    }
    // pivot: first row of maximal |a| among window rows j .. j+nr of column j
    const int nr = min(K, n - 1 - j);
    // one 64-bit key per lane, larger is better: |a| (the bit pattern of a
    // non-negative float orders like its value), then the smaller label, then
    // the lane; rows that are not candidates have key 0 and never win
    const bool cand = label >= j && label <= j + nr;
    unsigned long long key =
        cand ? ((unsigned long long)__float_as_uint(fabsf(a[0])) << 32) |
                   ((unsigned long long)(0xffffu - (unsigned)label) << 8) | (unsigned)lane
             : 0ull;
#pragma unroll
    for (int off = 1; off < GW; off <<= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off, GW);
      key = o > key ? o : key;
    }
    const int pl = (int)(0xffffu - (unsigned)((key >> 8) & 0xffffu));
    const float kv = __shfl_sync(0xffffffffu, a[0], (int)(key & 0xffu));
    const bool sing = !(__uint_as_float((unsigned)(key >> 32)) > 0.0f);
    if (sing && info == 0) info = j + 1;
    const float invd = sing ? 0.0f : 1.0f / kv;
    const int p = pl - j;
    // interchange rows j and j+p: the labels swap
    const bool piv = label == pl;
    if (p != 0) {
      if (label == j)
        label = pl;
      else if (piv)
        label = j;
    }
    // U's row j from the pivot row (float4 stores; entries past 2K are 0)
    if (piv) {
#pragma unroll
      for (int q4 = 0; q4 < P::UB / 4; ++q4) {
        float4 u4;
        u4.x = (4 * q4 + 1 <= 2 * K) ? a[4 * q4 + 1] : 0.0f;
        u4.y = (4 * q4 + 2 <= 2 * K) ? a[4 * q4 + 2] : 0.0f;
        u4.z = (4 * q4 + 3 <= 2 * K) ? a[4 * q4 + 3] : 0.0f;
        u4.w = (4 * q4 + 4 <= 2 * K) ? a[4 * q4 + 4] : 0.0f;
        reinterpret_cast<float4*>(ub)[q4] = u4;
      }
    }
    __syncwarp();
    // multiplier, then update and shift by one column (a[s] <- column j+1+s)
    const int rr = label - j;  // position of my row after the interchange
    const bool below = rr >= 1 && rr <= K;
    const float l = (below && rr <= nr && !sing) ? a[0] * invd : 0.0f;
#pragma unroll
    for (int q4 = 0; q4 < P::UB / 4; ++q4) {
      const float4 u4 = reinterpret_cast<const float4*>(ub)[q4];
      const float uu[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int s = 4 * q4 + e;
        if (s < 2 * K) a[s] = fmaf(-l, uu[e], a[s + 1]);
      }
    }
    a[2 * K] = 0.0f;
    if (active) {
      const int64_t fj = (int64_t)j * (FRn / 4);
      if (below) tb[((fj + (rr - 1) / 4) * kTile + cl) * 4 + ((rr - 1) & 3)] = l;
      if (r == 0) {
        tb[((fj + K / 4) * kTile + cl) * 4 + (K & 3)] = (float)p;
        tb[((fj + (K + 1) / 4) * kTile + cl) * 4 + ((K + 1) & 3)] = invd;
#pragma unroll
        for (int e = K + 2; e < FRn; ++e) tb[((fj + e / 4) * kTile + cl) * 4 + (e & 3)] = 0.0f;
      }
      // U[j][j+cc] is entry cc-1 of column j+cc's backward record
      const int ncol = min(2 * K, n - 1 - j);
      for (int cc = 1 + r; cc <= ncol; cc += GW)
        bb[((int64_t)((j + cc) * (BR / 4) + (cc - 1) / 4) * kTile + cl) * 4 + ((cc - 1) & 3)] =
            ub[cc - 1];
      // entries of B_j that no row reaches (rows j - 1 - d < 0) and the padding
      if (j < BR)
        for (int d = r; d < BR; d += GW)
          if (d >= j || d >= 2 * K)
            bb[((int64_t)(j * (BR / 4) + d / 4) * kTile + cl) * 4 + (d & 3)] = 0.0f;
    }
    // the pivot row retires; its thread takes row j+K+1
    if (label == j) {
#pragma unroll
      for (int q4 = 0; q4 < P::RB / 4; ++q4) {
        const float4 r4 = reinterpret_cast<const float4*>(rb)[q4];
        if (4 * q4 < WC) a[4 * q4] = r4.x;
        if (4 * q4 + 1 < WC) a[4 * q4 + 1] = r4.y;
        if (4 * q4 + 2 < WC) a[4 * q4 + 2] = r4.z;
        if (4 * q4 + 3 < WC) a[4 * q4 + 3] = r4.w;
      }
      label = j + K + 1;
    }
  }
#pragma unroll
  for (int off = 1; off < GW; off <<= 1) info = max(info, __shfl_xor_sync(0xffffffffu, info, off, GW));
  if (r == 0 && active) {
    const int st = !ok ? HEVI_COL_BAD_INPUT : (info ? HEVI_COL_SINGULAR : HEVI_COL_OK);
    v.fac_status[c.col] = st;
    if (st != HEVI_COL_OK)
      fail(v, c.col, st);
    else
      v.col_status[c.col] = HEVI_COL_OK;
    v.col_iters[c.col] = 0;
  }
}

static int pick_block(int bytes, int max_blk);
static unsigned col_grid(const DevView& v, int blk);
static int window_slots(int N) {
  const int K = 3 * (N + 1) - 1;
  return (K + 1) * (2 * K + 1);
}

template <int N>
static void launch_factor_n(const DevView& v, hevi_precision prec, double lam, const double* q0,
                            int ylen, cudaStream_t st) {
  const int esz = prec == HEVI_FP64 ? (int)sizeof(double) : (int)sizeof(float);
  const int blk = pick_block(window_slots(N) * esz, 64), tiles_per_blk = blk / kTile;
  const unsigned grid = (unsigned)((v.tile_count + tiles_per_blk - 1) / tiles_per_blk);
  const int smem = window_slots(N) * blk * esz;
  if (prec == HEVI_FP64) {
    cudaFuncSetAttribute(k_factor<N, double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_factor<N, double, false><<<grid, blk, smem, st>>>(v, lam, q0);
  } else {
    // row-per-thread: blocks of four warps, 32/GW columns per warp
    constexpr int K = Band<N>::K;
    using P = FRow<N>;
    const int nmax = ylen - 2 * K;  // longest n of these tiles
    const int linstride = (3 * (nmax / 3) + 3) / 4 * 4;
    const int rsmem = (kGSzA + P::CPB * (2 * P::UB + 2 * P::RB + linstride)) * (int)sizeof(float);
    cudaFuncSetAttribute(k_factor_r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, rsmem);
    k_factor_r<N><<<(unsigned)(v.tile_count * (kTile / P::CPB)), 128, rsmem, st>>>(v, lam, q0,
                                                                                 linstride);
    (void)grid;
    (void)smem;
  }
}

void launch_factor(const DevView& v, int order, hevi_precision prec, double lam, const double* q0,
                   int ylen, cudaStream_t st) {
  switch (order) {
    case 1: launch_factor_n<1>(v, prec, lam, q0, ylen, st); break;
    case 2: launch_factor_n<2>(v, prec, lam, q0, ylen, st); break;
    case 3: launch_factor_n<3>(v, prec, lam, q0, ylen, st); break;
    case 4: launch_factor_n<4>(v, prec, lam, q0, ylen, st); break;
    case 5: launch_factor_n<5>(v, prec, lam, q0, ylen, st); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// Triangular solves with the records of one column (dgbtrs semantics:
// interchanges and unit-lower multipliers in factorisation order, then the
// upper triangle with 2K super-diagonals, column by column).  The active
// window of the sweep lives in registers: the loop over pivot steps is
// unrolled by the window length so that every ring position is a
// compile-time register.  y is the column's work vector with element stride
// `stride` (shared memory, or the tile's interleaved global scratch), length
// n + 2K with a zero tail; the forward sweep leaves the intermediate vector
// in y, the backward sweep the solution.  PD > 0 prefetches the records of
// step j +/- PD into L1 while step j computes: the sweep is a dependent chain
// of n steps per thread, and without it every step waits for its record.
// ---------------------------------------------------------------------------
template <int N, typename T>
__device__ __forceinline__ void load_vecs(const T* src, T* dst, int count) {
  constexpr int W = Vec<T>::W;
  using V = typename Vec<T>::type;
#pragma unroll
  for (int q = 0; q < count; q += W) {
    const V x = *reinterpret_cast<const V*>(src + (int64_t)(q / W) * kTile * W);
    if constexpr (W == 4) {
      dst[q] = x.x; dst[q + 1] = x.y; dst[q + 2] = x.z; dst[q + 3] = x.w;
    } else {
      dst[q] = x.x; dst[q + 1] = x.y;
    }
  }
}

// Cache-line prefetch of one 16-byte record vector (no registers held).
__device__ __forceinline__ void prefetch_line(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <int N, typename T, typename Y, int PD = 0>
__device__ __forceinline__ void forward_sweep(const T* base, int lane, int n, Y* y, int stride) {
  constexpr int K = Band<N>::K, WR = Band<N>::WR, FR = Band<N>::FR;
  constexpr int NVF = FR / Vec<T>::W;
  if constexpr (PD > 0) {
    for (int jj = 0; jj < PD && jj < n; ++jj)
#pragma unroll
      for (int vv = 0; vv < NVF; ++vv) prefetch_line(frec_vec<N, T>(const_cast<T*>(base), jj, vv * Vec<T>::W, lane));
  }
  Y w[WR];
#pragma unroll
  for (int r = 0; r < WR; ++r) w[r] = y[r * stride];
  for (int j0 = 0; j0 < n; j0 += WR) {
#pragma unroll
    for (int t = 0; t < WR; ++t) {
      const int j = j0 + t;
      if (j < n) {
        if constexpr (PD > 0) {
          if (j + PD < n) {
#pragma unroll
            for (int vv = 0; vv < NVF; ++vv)
              prefetch_line(frec_vec<N, T>(const_cast<T*>(base), j + PD, vv * Vec<T>::W, lane));
          }
          // and the work-vector row that enters the window PD steps later
          if (j + WR + PD < n + 2 * K) prefetch_line(&y[(j + WR + PD) * stride]);
        }
        T f[FR];
        load_vecs<N, T>(frec_vec<N, T>(const_cast<T*>(base), j, 0, lane), f, FR);
        const int p = (int)f[K];
        // interchange rows j and j+p, then eliminate below the pivot
        Y yp = w[t];
#pragma unroll
        for (int r = 1; r <= K; ++r)
          if (p == r) yp = w[(t + r) % WR];
#pragma unroll
        for (int r = 1; r <= K; ++r)
          if (p == r) w[(t + r) % WR] = w[t];
        y[j * stride] = yp;
#pragma unroll
        for (int r = 1; r <= K; ++r) w[(t + r) % WR] -= Y(f[r - 1]) * yp;
        w[t] = y[(j + WR) * stride];
      }
    }
  }
}

// Backward substitution; returns the sum of squares of the solution.
template <int N, typename T, typename Y, int PD = 0>
__device__ __forceinline__ Y backward_sweep(const T* base, int lane, int n, Y* y, int stride) {
  constexpr int K = Band<N>::K, WB = Band<N>::WC, BR = Band<N>::BR, FR = Band<N>::FR;
  constexpr int W = Vec<T>::W;
  constexpr int NVB = BR / W;
  using V = typename Vec<T>::type;
  auto prefetch_step = [&](int jj) {
#pragma unroll
    for (int vv = 0; vv < NVB; ++vv) prefetch_line(brec_vec<N, T>(const_cast<T*>(base), n, jj, vv * W, lane));
    prefetch_line(frec_vec<N, T>(const_cast<T*>(base), jj, K + 1, lane));
  };
  if constexpr (PD > 0) {
    for (int jj = n - 1; jj > n - 1 - PD && jj >= 0; --jj) prefetch_step(jj);
  }
  Y w[WB];
#pragma unroll
  for (int cc = 0; cc < WB; ++cc) {
    const int i = n - 1 - cc;
    w[cc] = i >= 0 ? y[i * stride] : Y(0);
  }
  Y ss = Y(0);
  for (int j0 = n - 1; j0 >= 0; j0 -= WB) {
#pragma unroll
    for (int t = 0; t < WB; ++t) {
      const int j = j0 - t;
      if (j >= 0) {
        if constexpr (PD > 0) {
          if (j - PD >= 0) prefetch_step(j - PD);
          if (j - WB - PD >= 0) prefetch_line(&y[(j - WB - PD) * stride]);
        }
        T u[BR];
        load_vecs<N, T>(brec_vec<N, T>(const_cast<T*>(base), n, j, 0, lane), u, BR);
        const V dv = *reinterpret_cast<const V*>(frec_vec<N, T>(const_cast<T*>(base), j, K + 1, lane));
        T invd;
        if constexpr (W == 4)
          invd = ((K + 1) % 4 == 0) ? dv.x : ((K + 1) % 4 == 1) ? dv.y : ((K + 1) % 4 == 2) ? dv.z : dv.w;
        else
          invd = ((K + 1) % 2 == 0) ? dv.x : dv.y;
        const Y x = w[t] * Y(invd);
        y[j * stride] = x;
        ss += x * x;
#pragma unroll
        for (int cc = 1; cc <= 2 * K; ++cc) w[(t + cc) % WB] -= Y(u[cc - 1]) * x;
        const int jn = j - WB;
        w[t] = jn >= 0 ? y[jn * stride] : Y(0);
      }
    }
  }
  (void)FR;
  return ss;
}

// ---------------------------------------------------------------------------
// Record ring for the FP32 solve: the warp's records stream through a small
// shared-memory ring filled by bulk asynchronous copies (cp.async.bulk, the
// TMA engine's linear mode) that complete on one mbarrier per slot.  One lane
// issues the copies of step j + D while the warp computes step j; the 32
// lanes' records of a step are one contiguous block of the tile, so a step is
// one (forward) or two (backward: B record + the 1/u_jj vector) copies.
// Every wait is bounded: past the limit the ring records the failure, stops
// issuing, and the caller drains what is still in flight before returning.
// ---------------------------------------------------------------------------
constexpr int kRingWaitTries = 1 << 16;  // x the suspend hint below: ~1.3 s bound
constexpr unsigned kRingSuspendNs = 20000;
// A sweep in which at least kRingLanes lanes still refine streams the whole
// tile's records through the ring (the stopped lanes compute on their own
// scratch, which is no longer read); with at most kWarpSweepLanes the warp
// solves those columns one at a time (warp_sweeps and the warp_* passes).
constexpr int kRingLanes = 3;
constexpr int kWarpSweepLanes = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// true once the phase of the given parity has completed, false past the limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < kRingWaitTries; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kRingSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

template <int N>
struct RingCfg {
  static constexpr int FB = Band<N>::FR * kTile * 4;        // forward step: F record
  static constexpr int BB = (Band<N>::BR + 4) * kTile * 4;  // backward: B record + 1/u_jj vector
  static constexpr int BYTES = 2 * BB;                      // ring size
  static constexpr int DF = BYTES / FB;                     // forward slots (>= 3)
  static constexpr int DB = 2;                              // backward slots
  static constexpr int NBAR = DF > DB ? DF : DB;
  static constexpr int TRANSPOSE = kTile * 17 * 8;          // b / x transpose tile
  static constexpr int YST = 512;                           // warp_sweeps' vector (floats)
  static constexpr int SMEM = (BYTES > TRANSPOSE ? BYTES : TRANSPOSE) + YST * 4;  // barriers follow
  static_assert(DF >= 3, "forward ring too shallow");
};

// Dynamic shared memory of the solve kernel: the ring, then its barriers.
extern __shared__ __align__(128) unsigned char g_ring[];

// Lane-uniform state of one warp's ring; the buffer and the barriers are the
// kernel's dynamic shared memory (RingCfg<N>::SMEM bytes of ring, then NBAR
// barriers).
template <int N>
struct Ring {
  unsigned phase;    // expected parity per barrier (bit s)
  unsigned pending;  // barriers with a copy in flight (bit s)
  bool ok;
  int drop;          // test hook: forward step + 1 whose copy is announced but not issued
  __device__ __forceinline__ static unsigned char* buf() { return g_ring; }
  __device__ __forceinline__ static uint64_t* bar() {
    return reinterpret_cast<uint64_t*>(g_ring + RingCfg<N>::SMEM);
  }
  __device__ __forceinline__ bool wait(int s) {
    bool good = ok;
    if (good) good = mbar_wait(&bar()[s], (phase >> s) & 1u);
    good = __all_sync(0xffffffffu, good);
    if (good) {
      phase ^= 1u << s;
      pending &= ~(1u << s);
    }
    ok = good;
    return good;
  }
  // wait (bounded) for every copy still in flight; the ring is idle after
  __device__ __forceinline__ void drain() {
    for (int s = 0; s < RingCfg<N>::NBAR; ++s)
      if (pending & (1u << s)) {
        mbar_wait(&bar()[s], (phase >> s) & 1u);
        phase ^= 1u << s;
      }
    pending = 0;
    __syncwarp();
  }
};

template <int N>
__device__ __forceinline__ void ring_issue_f(Ring<N>& rg, const float* base, int j, int slot,
                                             int lane) {
  using C = RingCfg<N>;
  rg.pending |= 1u << slot;
  if (lane == 0) {
    uint64_t* bar = &Ring<N>::bar()[slot];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, C::FB);
    if (rg.drop != j + 1)
      bulk_g2s(Ring<N>::buf() + slot * C::FB, frec_vec<N, float>(const_cast<float*>(base), j, 0, 0),
               C::FB, bar, evict_first_policy());
  }
}
template <int N>
__device__ __forceinline__ void ring_issue_b(Ring<N>& rg, const float* base, int n, int j,
                                             int slot, int lane) {
  using C = RingCfg<N>;
  constexpr int K = Band<N>::K;
  rg.pending |= 1u << slot;
  if (lane == 0) {
    uint64_t* bar = &Ring<N>::bar()[slot];
    const uint64_t pol = evict_first_policy();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, C::BB);
    unsigned char* dst = Ring<N>::buf() + slot * C::BB;
    bulk_g2s(dst, brec_vec<N, float>(const_cast<float*>(base), n, j, 0, 0), Band<N>::BR * kTile * 4,
             bar, pol);
    bulk_g2s(dst + Band<N>::BR * kTile * 4, frec_vec<N, float>(const_cast<float*>(base), j, K + 1, 0),
             4 * kTile * 4, bar, pol);
  }
}

// Forward sweep of forward_sweep with the F records taken from the ring.
template <int N>
__device__ __forceinline__ void forward_sweep_ring(Ring<N>& rg, const float* base, int lane, int n,
                                                   float* y, int stride) {
  using C = RingCfg<N>;
  constexpr int K = Band<N>::K, WR = Band<N>::WR, FR = Band<N>::FR;
  if (rg.ok)
    for (int s = 0; s < C::DF && s < n; ++s) ring_issue_f<N>(rg, base, s, s, lane);
  float w[WR];
#pragma unroll
  for (int r = 0; r < WR; ++r) w[r] = y[r * stride];
  int slot = 0;
  for (int j0 = 0; j0 < n; j0 += WR) {
#pragma unroll
    for (int t = 0; t < WR; ++t) {
      const int j = j0 + t;
      if (j < n) {
        rg.wait(slot);
        float f[FR];
        const float4* src = reinterpret_cast<const float4*>(Ring<N>::buf() + slot * C::FB) + lane;
#pragma unroll
        for (int q = 0; q < FR; q += 4) {
          const float4 x = src[(q / 4) * kTile];
          f[q] = x.x; f[q + 1] = x.y; f[q + 2] = x.z; f[q + 3] = x.w;
        }
        const int p = (int)f[K];
        float yp = w[t];
#pragma unroll
        for (int r = 1; r <= K; ++r)
          if (p == r) yp = w[(t + r) % WR];
#pragma unroll
        for (int r = 1; r <= K; ++r)
          if (p == r) w[(t + r) % WR] = w[t];
#pragma unroll
        for (int r = 1; r <= K; ++r) w[(t + r) % WR] -= f[r - 1] * yp;
        // refill the slot just read with step j + D
        __syncwarp();
        if (j + C::DF < n && rg.ok) ring_issue_f<N>(rg, base, j + C::DF, slot, lane);
        slot = slot + 1 == C::DF ? 0 : slot + 1;
        y[j * stride] = yp;
        w[t] = y[(j + WR) * stride];
      }
    }
  }
}

// Backward sweep of backward_sweep with the B records and 1/u_jj from the ring.
template <int N>
__device__ __forceinline__ float backward_sweep_ring(Ring<N>& rg, const float* base, int lane, int n,
                                                     float* y, int stride) {
  using C = RingCfg<N>;
  constexpr int K = Band<N>::K, WB = Band<N>::WC, BR = Band<N>::BR;
  if (rg.ok)  // after a wait ran out nothing more is issued
    for (int s = 0; s < C::DB && s < n; ++s) ring_issue_b<N>(rg, base, n, n - 1 - s, s, lane);
  float w[WB];
#pragma unroll
  for (int cc = 0; cc < WB; ++cc) {
    const int i = n - 1 - cc;
    w[cc] = i >= 0 ? y[i * stride] : 0.0f;
  }
  float ss = 0.0f;
  int slot = 0;
  for (int j0 = n - 1; j0 >= 0; j0 -= WB) {
#pragma unroll
    for (int t = 0; t < WB; ++t) {
      const int j = j0 - t;
      if (j >= 0) {
        rg.wait(slot);
        float u[BR];
        const float4* src = reinterpret_cast<const float4*>(Ring<N>::buf() + slot * C::BB) + lane;
#pragma unroll
        for (int q = 0; q < BR; q += 4) {
          const float4 x = src[(q / 4) * kTile];
          u[q] = x.x; u[q + 1] = x.y; u[q + 2] = x.z; u[q + 3] = x.w;
        }
        const float4 dv = src[(BR / 4) * kTile];
        const float invd = ((K + 1) % 4 == 0)   ? dv.x
                           : ((K + 1) % 4 == 1) ? dv.y
                           : ((K + 1) % 4 == 2) ? dv.z
                                                : dv.w;
        const float x = w[t] * invd;
        ss += x * x;
#pragma unroll
        for (int cc = 1; cc <= 2 * K; ++cc) w[(t + cc) % WB] -= u[cc - 1] * x;
        // refill the slot just read with step j - D
        __syncwarp();
        if (j - C::DB >= 0 && rg.ok) ring_issue_b<N>(rg, base, n, j - C::DB, slot, lane);
        slot ^= 1;
        y[j * stride] = x;
        const int jn = j - WB;
        w[t] = jn >= 0 ? y[jn * stride] : 0.0f;
      }
    }
  }
  return ss;
}

// Copy `count` 16-byte vectors src(q), q = 0..count-1, into dst[q] with the
// warp, four loads in flight per lane before their stores.
template <class Src>
__device__ __forceinline__ void stage_vecs(float* dst, int count, int lane, Src&& src) {
  float4* d = reinterpret_cast<float4*>(dst);
  for (int q0 = 0; q0 < count; q0 += 4 * 32) {
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = q0 + k * 32 + lane;
      if (q < count) v[k] = *src(q);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = q0 + k * 32 + lane;
      if (q < count) d[q] = v[k];
    }
  }
}

// Forward and backward substitution of ONE column (tile lane c) by the whole
// warp.  Lane l carries the window rows i = l (mod 32) and the row 32 below
// (forward: above) it, so a pivot step is two shuffles and one FMA per lane
// instead of a per-thread chain of loads; the column's records are staged
// into the (idle) ring a chunk of steps at a time.  Same arithmetic as
// forward_sweep / backward_sweep.  Used for the few lanes that still refine
// after the ring sweeps, which would otherwise set the kernel's tail.
template <int N>
__device__ __noinline__ void warp_sweeps(const float* base, int c, int n, float* ytile, int lane) {
  constexpr int K = Band<N>::K, FR = Band<N>::FR, BR = Band<N>::BR;
  constexpr int NVF = FR / 4, NVB = BR / 4, RS = BR + 4;
  constexpr int CAP = RingCfg<N>::SMEM / 4 - RingCfg<N>::YST;  // floats of staging space
  constexpr unsigned FULL = 0xffffffffu;
  float* sm = reinterpret_cast<float*>(Ring<N>::buf());
  float* yc = sm + CAP;  // the column's work vector, rows 0 .. n + 2K - 1
  const int ylen = n + 2 * K;
  float* fb = const_cast<float*>(base);
  for (int i = lane; i < ylen; i += 32) yc[i] = ytile[(int64_t)i * kTile + c];
  __syncwarp();
  {  // forward: L y = P b
    constexpr int CH = CAP / FR;
    float yw = lane < ylen ? yc[lane] : 0.0f;
    float yn = lane + 32 < ylen ? yc[lane + 32] : 0.0f;
    for (int j0 = 0; j0 < n; j0 += CH) {
      const int cnt = min(CH, n - j0);
      __syncwarp();
      stage_vecs(sm, cnt * NVF, lane, [&](int q) {
        return reinterpret_cast<const float4*>(frec_vec<N, float>(fb, j0 + q / NVF, (q % NVF) * 4, c));
      });
      __syncwarp();
      for (int jj = 0; jj < cnt; ++jj) {
        const int j = j0 + jj;
        const float* f = sm + jj * FR;
        const int p = (int)f[K];
        const int l0 = j & 31, lp = (j + p) & 31;
        const int rel = (lane - j) & 31;  // this lane's row is j + rel
        const float lr = f[rel >= 1 && rel <= K ? rel - 1 : K + 1];
        const float ynext = j + 64 < ylen ? yc[j + 64] : 0.0f;
        const float yj = __shfl_sync(FULL, yw, lp);  // row j after the interchange
        const float yo = __shfl_sync(FULL, yw, l0);
        yw = lane == lp ? yo : yw;
        yw = rel >= 1 && rel <= K ? yw - lr * yj : yw;
        if (lane == l0) yc[j] = yj;
        yw = lane == l0 ? yn : yw;
        yn = lane == l0 ? ynext : yn;
      }
    }
  }
  {  // backward: U x = y
    constexpr int CH = CAP / RS;
    __syncwarp();
    const int il = n - 1 - ((n - 1 - lane) & 31);  // the lane's row nearest below n
    float yw = il >= 0 ? yc[il] : 0.0f;
    float yn = il - 32 >= 0 ? yc[il - 32] : 0.0f;
    for (int j1 = n - 1; j1 >= 0; j1 -= CH) {
      const int cnt = min(CH, j1 + 1);  // steps j1, j1 - 1, .., j1 - cnt + 1
      __syncwarp();
      stage_vecs(sm, cnt * (NVB + 1), lane, [&](int q) {
        const int jj = q / (NVB + 1), vv = q % (NVB + 1);
        return reinterpret_cast<const float4*>(vv < NVB ? brec_vec<N, float>(fb, n, j1 - jj, vv * 4, c)
                                                        : frec_vec<N, float>(fb, j1 - jj, K + 1, c));
      });
      __syncwarp();
      for (int jj = 0; jj < cnt; ++jj) {
        const int j = j1 - jj;
        const float* u = sm + jj * RS;
        const int l0 = j & 31;
        const int rel = (j - lane) & 31;  // this lane's row is j - rel
        const float ur = u[rel >= 1 && rel <= 2 * K ? rel - 1 : BR];
        const float ynext = j - 64 >= 0 ? yc[j - 64] : 0.0f;
        const float xj = __shfl_sync(FULL, yw, l0) * u[BR + (K + 1) % 4];
        yw = rel >= 1 && rel <= 2 * K ? yw - ur * xj : yw;
        if (lane == l0) yc[j] = xj;
        yw = lane == l0 ? yn : yw;
        yn = lane == l0 ? ynext : yn;
      }
    }
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) ytile[(int64_t)i * kTile + c] = yc[i];
  __syncwarp();
}

// The other refinement passes of ONE column (tile lane c) by the whole warp,
// lanes over the column's rows / points; same arithmetic as the per-thread
// passes of solve_ir_column except the order of the sums.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// |S y|^2 of column c.
__device__ __noinline__ float warp_d2(const TileScr& sc, int c, int n, int lane) {
  float d2 = 0.0f;
  for (int i = lane; i < n; i += 32) {
    const float d = sc.y[(int64_t)i * kTile + c] * sc.s[(int64_t)i * kTile + c];
    d2 = fmaf(d, d, d2);
  }
  return warp_sum(d2);
}

// x += S y (x = S y on the first sweep) of column c (x as double-float pairs).
__device__ __noinline__ void warp_update_x(const TileScr& sc, int c, int n, bool fst, int lane) {
  float2* xd = reinterpret_cast<float2*>(sc.x);
  for (int i = lane; i < n; i += 32) {
    const int64_t a = (int64_t)i * kTile + c;
    const float d = sc.y[a] * sc.s[a];
    xd[a] = df_pack(fst ? df{d, 0.0f} : df_add_f(df_of(xd[a]), d));
  }
  __syncwarp();
}

// Fused pass of column c: x += S y, r = b - A x, y = S^-1 r (double-float
// arithmetic, as the per-thread pass); returns |x|^2 (FP32).  The point
// fluxes K x go through shared memory so that each lane can form the element
// derivative (and the direct-stiffness sum at element ends) of its own points.
template <int N>
__device__ __noinline__ float warp_residual(const TileScr& sc, int c, int nez, double cs,
                                            double lam, double g, bool fst, int lane) {
  const int nz = nez * N + 1;
  float2* F = reinterpret_cast<float2*>(Ring<N>::buf());  // [nz][3], then the tables
  float2* Dm = F + 3 * nz;                                 // wD (lane-dependent rows)
  float2* iw = Dm + (N + 1) * (N + 1);
  float2* xd = reinterpret_cast<float2*>(sc.x);
  const float2* bd = reinterpret_cast<const float2*>(sc.b);
  const df lamd = df_from_double(lam), gd = df_from_double(g), csd = df_from_double(cs);
  float xsq = 0.0f;
  __syncwarp();
  for (int k = lane; k < (N + 1) * (N + 1); k += 32) Dm[k] = c_tab.wD2[N][k];
  if (lane <= N) iw[lane] = c_tab.iw2[N][lane];
  for (int I = lane; I < nz; I += 32) {
    df xi[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int64_t a = (int64_t)(3 * I + u) * kTile + c;
      const float d = sc.y[a] * sc.s[a];
      xi[u] = fst ? df{d, 0.0f} : df_add_f(df_of(xd[a]), d);
      xd[a] = df_pack(xi[u]);
      xsq = fmaf(xi[u].hi, xi[u].hi, xsq);
    }
    const int64_t a0 = (int64_t)(3 * I) * kTile + c;
    const df wI = df_from_double(sc.lin[a0]), thI = df_from_double(sc.lin[a0 + kTile]),
             cI = df_from_double(sc.lin[a0 + 2 * kTile]);
    F[3 * I] = df_pack(xi[1]);
    F[3 * I + 1] = df_pack(df_sub(df_fma({2.0f * wI.hi, 2.0f * wI.lo}, xi[1], df_mul(cI, xi[2])),
                                  df_mul(df_mul(wI, wI), xi[0])));
    F[3 * I + 2] = df_pack(df_sub(df_fma(thI, xi[1], df_mul(wI, xi[2])), df_mul(df_mul(thI, wI), xi[0])));
  }
  __syncwarp();
  auto cc = [&](int e, int k, int v) {  // element e's derivative row k of field v
    df sum = df_mul(df_of(Dm[k * (N + 1)]), df_of(F[3 * (e * N) + v]));
#pragma unroll
    for (int j = 1; j <= N; ++j) sum = df_fma(df_of(Dm[k * (N + 1) + j]), df_of(F[3 * (e * N + j) + v]), sum);
    return sum;
  };
  for (int I = lane; I < nz; I += 32) {
    const int e = I == nz - 1 ? nez - 1 : I / N, k = I - e * N;
    const df iw0 = df_of(iw[0]);
    df D[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      if (k != 0 && k != N) {
        D[v] = df_mul(cc(e, k, v), df_mul(csd, df_of(iw[k])));
      } else if (I == 0) {
        D[v] = df_mul(cc(0, 0, v), df_mul(csd, iw0));
      } else if (I == nz - 1) {
        D[v] = df_mul(cc(nez - 1, N, v), df_mul(csd, iw0));
      } else {
        D[v] = df_mul(df_add(cc(e - 1, N, v), cc(e, 0, v)), df_mul(csd, {0.5f * iw0.hi, 0.5f * iw0.lo}));
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int64_t a = (int64_t)(3 * I + u) * kTile + c;
      const df xv = df_of(xd[a]), bv = df_of(bd[a]);
      df r;
      if (u == 1 && (I == 0 || I == nz - 1)) {
        r = df_sub(bv, xv);
      } else {
        df ax = D[u];
        if (u == 1) ax = df_fma(gd, df_of(xd[(int64_t)(3 * I) * kTile + c]), ax);
        r = df_sub(bv, df_fma(lamd, ax, xv));
      }
      sc.y[a] = __fadd_rn(r.hi, r.lo) * sc.is[a];
    }
  }
  __syncwarp();
  return warp_sum(xsq);
}

// Plain FP64 solve (K = one column per thread, FP64 factors).
template <int N>
__device__ void solve_fp64_column(const DevView& v, const TileDesc& t, int lane, const double* b,
                                  double* x, double* y, int stride) {
  constexpr int K = Band<N>::K;
  const Col c = make_col(v, t, lane, N);
  const double* base = reinterpret_cast<const double*>(v.fac) + t.fac_off;
  if (v.fac_status[c.col] != HEVI_COL_OK) {  // no usable factors for this column
    for (int i = 0; i < c.n; ++i) x[c.off + i] = __longlong_as_double(0x7ff8000000000000LL);
    v.col_iters[c.col] = 0;
    fail(v, c.col, v.fac_status[c.col]);
    return;
  }
  v.col_status[c.col] = HEVI_COL_OK;
  for (int i = 0; i < c.n; ++i) y[i * stride] = b[c.off + i];
  for (int i = c.n; i < c.n + 2 * K; ++i) y[i * stride] = 0.0;
  forward_sweep<N, double, double>(base, lane, c.n, y, stride);
  backward_sweep<N, double, double>(base, lane, c.n, y, stride);
  for (int i = 0; i < c.n; ++i) x[c.off + i] = y[i * stride];
  v.col_iters[c.col] = 1;
}

// Scales S = (rho_bar, rho_bar c_s, Theta_bar) of unknown (I, u).
__device__ __forceinline__ double ref_scale(const double* ref, double cs, int64_t a, int u) {
  return u == 0 ? ref[a] : (u == 1 ? ref[a] * cs : ref[a + 2]);
}

// Fused refinement pass of one thread's column (rows kTile apart): x += S y
// (skipped when !update), r = b - A x, y = S^-1 r, in double-float
// arithmetic; slots are the thread's shared-memory slots for element_pass_df.
// Returns |x|^2 (FP32: it only scales the stop test).
template <int N>
__device__ __forceinline__ float lane_residual(float* y, const float* s32, float2* xs_,
                                               const float2* bs_, const double* lin,
                                               const float* is32, int nez, double lam, double g,
                                               double cs, bool fst, bool update, float2* slots,
                                               int slot_lane) {
  constexpr int stride = kTile;
  const int nz = nez * N + 1;
  float xs = 0.0f;
  const df lamd = df_from_double(lam), gd = df_from_double(g), csd = df_from_double(cs);
  // Each call loads the next point's values of y and x (flux) or x and b
  // (out) before it stores its own, so that the loads are not held back
  // behind the stores; lin and the scales are read-only here (__ldg).
  const int nzc = 3 * nz;
  float py[3];
  float2 px[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    py[u] = y[u * stride];
    px[u] = xs_[u * stride];
  }
  auto flux = [&](int I, df* f) {
    float yc3[3];
    float2 xc3[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      yc3[u] = py[u];
      xc3[u] = px[u];
    }
    if (3 * I + 3 < nzc) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        py[u] = y[(3 * I + 3 + u) * stride];
        px[u] = xs_[(3 * I + 3 + u) * stride];
      }
    }
    df xi[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = 3 * I + u;
      const float d = update ? yc3[u] * __ldg(&s32[i * stride]) : 0.0f;
      xi[u] = !update ? df_of(xc3[u]) : fst ? df{d, 0.0f} : df_add_f(df_of(xc3[u]), d);
      xs_[i * stride] = df_pack(xi[u]);
      xs = fmaf(xi[u].hi, xi[u].hi, xs);
    }
    const df wI = df_from_double(__ldg(&lin[(3 * I) * stride]));
    const df thI = df_from_double(__ldg(&lin[(3 * I + 1) * stride]));
    const df cI = df_from_double(__ldg(&lin[(3 * I + 2) * stride]));
    f[0] = xi[1];
    // f1 = -w^2 rho + 2 w m + c Theta,  f2 = -theta w rho + theta m + w Theta
    f[1] = df_sub(df_fma({2.0f * wI.hi, 2.0f * wI.lo}, xi[1], df_mul(cI, xi[2])),
                  df_mul(df_mul(wI, wI), xi[0]));
    f[2] = df_sub(df_fma(thI, xi[1], df_mul(wI, xi[2])), df_mul(df_mul(thI, wI), xi[0]));
  };
  float2 qx[3], qb[3];
  bool qfirst = true;
  auto out = [&](int I, const df* D) {
    // A x = x + Lambda (Dcal[K x] + G x);  r = b - A x
    if (qfirst) {  // x of point 0 is final once flux(0) has run
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        qx[u] = xs_[u * stride];
        qb[u] = bs_[u * stride];
      }
      qfirst = false;
    }
    float2 xc3[3], bc3[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      xc3[u] = qx[u];
      bc3[u] = qb[u];
    }
    if (3 * I + 3 < nzc) {  // flux has already run for point I + 1
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        qx[u] = xs_[(3 * I + 3 + u) * stride];
        qb[u] = bs_[(3 * I + 3 + u) * stride];
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = 3 * I + u;
      const df xv = df_of(xc3[u]), bv = df_of(bc3[u]);
      df r;
      if (u == 1 && (I == 0 || I == nz - 1)) {
        r = df_sub(bv, xv);
      } else {
        df ax = D[u];
        if (u == 1) ax = df_fma(gd, df_of(xc3[0]), ax);
        r = df_sub(bv, df_fma(lamd, ax, xv));
      }
      y[i * stride] = __fadd_rn(r.hi, r.lo) * __ldg(&is32[i * stride]);
    }
  };
  element_pass_df<N>(nez, csd, slots, slot_lane, flux, out);
  return xs;
}

// FP32 factors + iterative refinement.
//   y0 = S^-1 b (FP32), solve; then repeat: x += S y; r = b - A x (double-
//   float, matrix-free from the point coefficients of L(q0)); y = S^-1 r
//   (FP32); solve; until the predicted relative error |d_k|^2/|d_{k-1}| / |x|
//   (plain 2-norms) is below tol, or max_sweeps.
// The loop is warp-uniform: a sweep in which at least kRingLanes lanes still
// refine streams the tile's records through the ring; with at most
// kWarpSweepLanes the warp takes those columns one at a time; otherwise each
// active lane loads its own records.  With `tail`, a column that would need a
// third sweep is updated and handed to k_solve_tail instead.
template <int N>
__device__ void solve_ir_column(const DevView& v, const TileDesc& t, int lane, double lam,
                                const double* b, double* x, double tol, int max_sweeps,
                                bool tail, Ring<N>& rg) {
  constexpr int stride = kTile;
  const TileScr sc = tile_scratch(v, t);
  float* y = sc.y + lane;
  float2* xs_ = reinterpret_cast<float2*>(sc.x) + lane;  // double-float pairs
  float2* bs_ = reinterpret_cast<float2*>(sc.b) + lane;
  const double* lin = sc.lin + lane;
  const float* s32 = sc.s + lane;
  const float* is32 = sc.is + lane;
  constexpr int K = Band<N>::K;
  const bool valid = lane < t.count;
  const int n = 3 * (t.nez * N + 1);
  const float* base = reinterpret_cast<const float*>(v.fac) + t.fac_off;
  Col c{};
  bool active = false;
  if (valid) {
    c = make_col(v, t, lane, N);
    if (v.fac_status[c.col] != HEVI_COL_OK) {  // no usable factors for this column
      for (int i = 0; i < c.n; ++i) x[c.off + i] = __longlong_as_double(0x7ff8000000000000LL);
      v.col_iters[c.col] = 0;
      fail(v, c.col, v.fac_status[c.col]);
    } else {
      active = true;
    }
  }
  double* xc = x + c.off;
  const double g = v.ph.g;
  // b enters the tile's interleaved scratch (bs_) through a transpose in the
  // idle ring, 16 rows x 32 columns a round, so that both the caller's
  // column-contiguous b and the scratch are accessed in whole lines; x is
  // refined in xs_ and leaves the same way at the end.
  const int64_t myoff = valid ? c.off : 0;
  double* tr = reinterpret_cast<double*>(Ring<N>::buf());  // [32 columns][17]
  for (int r0 = 0; r0 < n; r0 += 16) {
#pragma unroll 4
    for (int cc = 0; cc < kTile; cc += 2) {
      const int col = cc + (lane >> 4), k = lane & 15;
      const int64_t o = __shfl_sync(0xffffffffu, myoff, col);
      if (col < t.count && r0 + k < n) tr[col * 17 + k] = b[o + r0 + k];
    }
    __syncwarp();
    for (int k = 0; k < 16 && r0 + k < n; ++k) {
      const df bi = df_from_double(tr[lane * 17 + k]);
      bs_[(r0 + k) * stride] = df_pack(bi);
      y[(r0 + k) * stride] = __fadd_rn(bi.hi, bi.lo) * is32[(r0 + k) * stride];
    }
    __syncwarp();
  }
  for (int i = n; i < n + 2 * K; ++i) y[i * stride] = 0.0f;
  bool ran = active;  // the lanes whose x leaves through the final transpose

  int sweeps = 0, status = HEVI_COL_NOT_CONVERGED;
  double dprev = 0.0, xnorm = 0.0;
  bool first = true;
  const bool coop_ok = 2 * K < kTile && n + 2 * K <= RingCfg<N>::YST;
  while (true) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (act == 0) break;
    // few lanes left: the warp works on their columns together
    const bool coop = coop_ok && __popc(act) <= kWarpSweepLanes;
    if (__popc(act) >= kRingLanes && rg.ok) {
      forward_sweep_ring<N>(rg, base, lane, n, y, stride);
      backward_sweep_ring<N>(rg, base, lane, n, y, stride);
      if (!rg.ok) {  // a copy did not arrive within the wait limit
        rg.drain();
        if (active) {
          for (int i = 0; i < n; ++i) xc[i] = __longlong_as_double(0x7ff8000000000000LL);
          v.col_iters[c.col] = sweeps;
          fail(v, c.col, HEVI_COL_WAIT_TIMEOUT);
          ran = false;
          active = false;
        }
        break;
      }
    } else if (coop) {
      // a few straggling lanes: the warp solves their columns one at a time
      // (its 32 lanes hold the 2K + 1 rows of the backward window for N <= 4)
      if constexpr (2 * K < kTile)
        for (unsigned m = act; m; m &= m - 1) warp_sweeps<N>(base, __ffs(m) - 1, n, sc.y, lane);
    } else if (active) {
      // records of step j+2 are prefetched into L1 while step j computes
      forward_sweep<N, float, float, 2>(base, lane, n, y, stride);
      backward_sweep<N, float, float, 2>(base, lane, n, y, stride);
    }
    // size of the correction d = S y in the caller's (unscaled) norm
    float d2 = 0.0f;
    if (coop) {
      for (unsigned m = act; m; m &= m - 1) {
        const float t2 = warp_d2(sc, __ffs(m) - 1, n, lane);
        if (lane == __ffs(m) - 1) d2 = t2;
      }
    } else if (active) {
      for (int i = 0; i < n; ++i) {
        const float d = y[i * stride] * s32[i * stride];
        d2 = fmaf(d, d, d2);
      }
    }
    bool stop = false;
    const double dn = sqrt((double)d2);
    if (active) {
      ++sweeps;
      const double xref = first ? dn : xnorm;
      if (dn <= tol * xref) {
        stop = true;
        status = HEVI_COL_OK;
      } else if (!first) {
        const double pred = dn * (dn / dprev);  // error left after applying d
        if (pred <= tol * xref) {
          stop = true;
          status = HEVI_COL_OK;
        } else if (dn > 0.5 * dprev) {
          stop = true;  // refinement is not contracting
        }
      }
      if (sweeps >= max_sweeps) stop = true;
    }
    const bool stopping = active && stop;
    bool more = active && !stop;
    // stopping lanes: x += S y, and the column is done
    if (coop) {
      for (unsigned m = __ballot_sync(0xffffffffu, stopping); m; m &= m - 1)
        warp_update_x(sc, __ffs(m) - 1, n, __shfl_sync(0xffffffffu, first, __ffs(m) - 1), lane);
    } else if (stopping) {
      for (int i = 0; i < n; ++i) {
        const float d = y[i * stride] * s32[i * stride];
        xs_[i * stride] = df_pack(first ? df{d, 0.0f} : df_add_f(df_of(xs_[i * stride]), d));
      }
    }
    if (stopping) {
      active = false;
      v.col_iters[c.col] = sweeps;
      if (status != HEVI_COL_OK)
        fail(v, c.col, status);
      else
        v.col_status[c.col] = HEVI_COL_OK;
    }
    // a third sweep is left to the tail kernel: x += S y now, hand over
    if (more && !first && tail) {
      for (int i = 0; i < n; ++i) {
        const float d = y[i * stride] * s32[i * stride];
        xs_[i * stride] = df_pack(df_add_f(df_of(xs_[i * stride]), d));
      }
      v.tail_dprev[c.col] = dn;
      v.tail_list[v.tile_begin * kTile + atomicAdd(&v.tail_count[N], 1)] =
          (int32_t)(((v.tile_begin + blockIdx.x) << 5) | lane);
      more = false;
      active = false;
    }
    // refining lanes, fused pass: x += S y, r = b - A x, y = S^-1 r, |S^-1 x|
    const unsigned mm = __ballot_sync(0xffffffffu, more);
    if (coop_ok && __popc(mm) <= kWarpSweepLanes) {
      for (unsigned m = mm; m; m &= m - 1) {
        const int cl = __ffs(m) - 1;
        const float xsq = warp_residual<N>(sc, cl, t.nez, __shfl_sync(0xffffffffu, c.s, cl), lam, g,
                                           __shfl_sync(0xffffffffu, first, cl), lane);
        if (lane == cl) xnorm = sqrt((double)xsq);
      }
    } else if (more) {
      const float xs = lane_residual<N>(y, s32, xs_, bs_, lin, is32, t.nez, lam, g, c.s, first, true,
                                        reinterpret_cast<float2*>(Ring<N>::buf()), lane);
      xnorm = sqrt((double)xs);
    }
    if (more) {
      dprev = dn;
      first = false;
    }
  }
  const unsigned ranmask = __ballot_sync(0xffffffffu, ran);
  for (int r0 = 0; r0 < n; r0 += 16) {
    for (int k = 0; k < 16 && r0 + k < n; ++k) tr[lane * 17 + k] = df_to_double(df_of(xs_[(r0 + k) * stride]));
    __syncwarp();
#pragma unroll 4
    for (int cc = 0; cc < kTile; cc += 2) {
      const int col = cc + (lane >> 4), k = lane & 15;
      const int64_t o = __shfl_sync(0xffffffffu, myoff, col);
      if (((ranmask >> col) & 1u) && r0 + k < n) x[o + r0 + k] = tr[col * 17 + k];
    }
    __syncwarp();
  }
}

// FP32 + refinement solve: one warp per block, one column per thread, the
// work vectors in the tile's interleaved global scratch, the factor records
// streamed through the block's shared-memory ring.  Each sweep is a dependent
// chain of 2n pivot steps per thread, so what matters is that every column is
// resident at once: with 96 registers and 10 KB of shared memory (a ring of 2
// backward steps plus the straggler staging), 20 one-warp blocks fit an SM,
// i.e. 97k columns in one wave on 152 SMs.
template <int N>
__global__ void __launch_bounds__(32, 20) k_solve_ir(DevView v, double lam, const double* b,
                                                     double* x, double tol, int max_sweeps) {
  const int lane = threadIdx.x;
  const TileDesc t = v.tiles[v.tile_begin + blockIdx.x];
  if (lane == 0) {
    for (int s = 0; s < RingCfg<N>::NBAR; ++s) mbar_init(&Ring<N>::bar()[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  Ring<N> rg{0u, 0u, true, v.drop_copy};
  solve_ir_column<N>(v, t, lane, lam, b, x, tol, max_sweeps, true, rg);
}

// Tail of the FP32 + refinement solve: one thread per column that needed a
// third sweep (handed over by k_solve_ir with x updated after its second
// sweep): residual, sweep, stop test, as in solve_ir_column, then x.  The
// columns come from many tiles, so each thread reads its own records (one
// column per thread, the L1-prefetched per-thread sweeps); handing them over
// keeps k_solve_ir's warps at two uniform sweeps.
template <int N>
__global__ void __launch_bounds__(128) k_solve_tail(DevView v, double lam, double* x, double tol,
                                                    int max_sweeps) {
  constexpr int stride = kTile;
  extern __shared__ __align__(16) float2 tail_slots[];  // (2N + 1) x 3 pairs per lane, per warp
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= v.tail_count[N]) return;
  const int32_t e = v.tail_list[v.tile_begin * kTile + idx];
  const TileDesc t = v.tiles[e >> 5];
  const int lane = e & 31;
  const Col c = make_col(v, t, lane, N);
  const TileScr sc = tile_scratch(v, t);
  float* y = sc.y + lane;
  float2* xs_ = reinterpret_cast<float2*>(sc.x) + lane;
  const float2* bs_ = reinterpret_cast<const float2*>(sc.b) + lane;
  const double* lin = sc.lin + lane;
  const float* s32 = sc.s + lane;
  const float* is32 = sc.is + lane;
  const float* base = reinterpret_cast<const float*>(v.fac) + t.fac_off;
  float2* slots = tail_slots + (threadIdx.x / 32) * (2 * N + 1) * 3 * kTile;
  const int n = c.n;
  double dprev = v.tail_dprev[c.col];
  int sweeps = 2, status = HEVI_COL_NOT_CONVERGED;
  bool update = false;  // x already holds the second sweep's correction
  while (true) {
    const double xnorm =
        sqrt((double)lane_residual<N>(y, s32, xs_, bs_, lin, is32, t.nez, lam, v.ph.g, c.s, false,
                                      update, slots, threadIdx.x & 31));
    update = true;
    forward_sweep<N, float, float, 2>(base, lane, n, y, stride);
    backward_sweep<N, float, float, 2>(base, lane, n, y, stride);
    ++sweeps;
    float d2 = 0.0f;
    for (int i = 0; i < n; ++i) {
      const float d = y[i * stride] * s32[i * stride];
      d2 = fmaf(d, d, d2);
    }
    const double dn = sqrt((double)d2);
    bool stop = false;
    if (dn <= tol * xnorm || dn * (dn / dprev) <= tol * xnorm) {
      stop = true;
      status = HEVI_COL_OK;
    } else if (dn > 0.5 * dprev || sweeps >= max_sweeps) {
      stop = true;
    }
    if (stop) {
      double* xc = x + c.off;
      for (int i = 0; i < n; ++i) {
        const float d = y[i * stride] * s32[i * stride];
        xc[i] = df_to_double(df_add_f(df_of(xs_[i * stride]), d));
      }
      break;
    }
    dprev = dn;
  }
  v.col_iters[c.col] = sweeps;
  if (status != HEVI_COL_OK)
    fail(v, c.col, status);
  else
    v.col_status[c.col] = HEVI_COL_OK;
}

// Plain FP64 solve; the work vectors live in shared memory.
template <int N>
__global__ void __launch_bounds__(128) k_solve_fp64(DevView v, const double* b, double* x) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  double* y = reinterpret_cast<double*>(smem_raw) + threadIdx.x;
  solve_fp64_column<N>(v, t, lane, b, x, y, blockDim.x);
}

// Threads per block for a per-thread shared-memory footprint of `bytes`.
static int pick_block(int bytes, int max_blk) {
  int blk = max_blk;
  while (blk > kTile && bytes * blk > 200 * 1024) blk /= 2;
  return blk;
}

template <int N>
static void launch_solve_n(const DevView& v, hevi_precision prec, double lam, const double* b,
                           double* x, double tol, int max_sweeps, int ylen, int part,
                           cudaStream_t st) {
  if (part == 1) {  // the tail of the FP32 + refinement solve
    if (prec == HEVI_FP64) return;
    // the handed-over columns: one thread each (the grid covers every column
    // of this order; threads past the count return at once)
    constexpr int tail_smem = 4 * (2 * N + 1) * 3 * kTile * (int)sizeof(float2);
    static bool tail_configured = false;
    if (!tail_configured) {
      cudaFuncSetAttribute(k_solve_tail<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, tail_smem);
      tail_configured = true;
    }
    k_solve_tail<N><<<(unsigned)((v.tile_count * kTile + 127) / 128), 128, tail_smem, st>>>(
        v, lam, x, tol, max_sweeps);
    return;
  }
  if (prec == HEVI_FP64) {
    const int esz = (int)sizeof(double);
    const int blk = pick_block(ylen * esz, 128), tiles_per_blk = blk / kTile;
    const unsigned grid = (unsigned)((v.tile_count + tiles_per_blk - 1) / tiles_per_blk);
    const int smem = ylen * blk * esz;
    cudaFuncSetAttribute(k_solve_fp64<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_solve_fp64<N><<<grid, blk, smem, st>>>(v, b, x);
  } else {
    constexpr int smem = RingCfg<N>::SMEM + RingCfg<N>::NBAR * 8;
    static bool configured = false;
    if (!configured) {
      cudaFuncSetAttribute(k_solve_ir<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      // carve enough shared memory for 20 resident blocks; the rest stays L1
      cudaFuncSetAttribute(k_solve_ir<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           std::min(100, (20 * (smem + 1024 + 64) * 100 + 232447) / 232448));
      configured = true;
    }
    cudaMemsetAsync(v.tail_count + N, 0, sizeof(int32_t), st);
    k_solve_ir<N><<<(unsigned)v.tile_count, kTile, smem, st>>>(v, lam, b, x, tol, max_sweeps);
  }
}

void launch_solve(const DevView& v, int order, hevi_precision prec, double lam, const double* b,
                  double* x, double tol, int max_sweeps, int ylen, int part, cudaStream_t st) {
  switch (order) {
    case 1: launch_solve_n<1>(v, prec, lam, b, x, tol, max_sweeps, ylen, part, st); break;
    case 2: launch_solve_n<2>(v, prec, lam, b, x, tol, max_sweeps, ylen, part, st); break;
    case 3: launch_solve_n<3>(v, prec, lam, b, x, tol, max_sweeps, ylen, part, st); break;
    case 4: launch_solve_n<4>(v, prec, lam, b, x, tol, max_sweeps, ylen, part, st); break;
    case 5: launch_solve_n<5>(v, prec, lam, b, x, tol, max_sweeps, ylen, part, st); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// Operator applies (FP64): V(x) (App. A.2 with the reference subtracted) and
// L(q0) x (Sec. 4.3.1).
// ---------------------------------------------------------------------------
template <int N>
__device__ void apply_V_column(const DevView& v, const Col& c, const double* q, double* out,
                               double scale_lq, const double* add, const double* sub,
                               bool report = true) {
  // out = add + V(q) - sub (add / sub may be null)
  const Phys ph = v.ph;
  const double* ref = v.ref + c.off;
  const double* qc = q + c.off;
  bool ok = true;
  auto flux = [&](int I, double* f) {
    const double rho = qc[3 * I], m = qc[3 * I + 1], Th = qc[3 * I + 2];
    if (!(rho > 0.0) || !(Th > 0.0)) ok = false;
    const double ir = rcp64(rho);
    f[0] = m;
    f[1] = fma(m * m, ir, eos_perturbation(ph, Th, ref[3 * I + 2], ref[3 * I + 1],
                                           v.ithb ? v.ithb + c.off / 3 + I : nullptr));
    f[2] = Th * m * ir;
  };
  auto o = [&](int I, const double* D) {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int64_t i = c.off + 3 * I + u;
      double val;
      if (u == 1 && (I == 0 || I == c.nz - 1))
        val = 0.0;
      else
        val = (u == 1) ? -D[1] - ph.g * (qc[3 * I] - ref[3 * I]) : -D[u];
      if (add) val += add[i];
      if (sub) val -= sub[i];
      out[i] = val;
    }
  };
  element_pass<N>(c, c_tab.w[N], c_tab.iw[N], flux, o);
  if (!ok && report) fail(v, c.col, HEVI_COL_BAD_INPUT);
  (void)scale_lq;
}

template <int N>
__device__ void apply_L_column(const DevView& v, const Col& c, const double* x, double* out) {
  const double* lin = v.lin + c.off;
  const double* xc = x + c.off;
  const double g = v.ph.g;
  auto flux = [&](int I, double* f) {
    const double x0 = xc[3 * I], x1 = xc[3 * I + 1], x2 = xc[3 * I + 2];
    const double wI = lin[3 * I], thI = lin[3 * I + 1], cI = lin[3 * I + 2];
    f[0] = x1;
    f[1] = fma(-wI * wI, x0, fma(2.0 * wI, x1, cI * x2));
    f[2] = fma(-thI * wI, x0, fma(thI, x1, wI * x2));
  };
  auto o = [&](int I, const double* D) {
    const int64_t a = c.off + 3 * I;
    out[a] = -D[0];
    out[a + 1] = (I == 0 || I == c.nz - 1) ? 0.0 : -D[1] - g * xc[3 * I];
    out[a + 2] = -D[2];
  };
  element_pass<N>(c, c_tab.w[N], c_tab.iw[N], flux, o);
}

template <int N>
__device__ void apply_dispatch(const DevView& v, const TileDesc& t, int lane, const double* x,
                               double* y, int nonlinear) {
  const Col c = make_col(v, t, lane, N);
  if (nonlinear)
    apply_V_column<N>(v, c, x, y, 0.0, nullptr, nullptr);
  else
    apply_L_column<N>(v, c, x, y);
}

template <int N>
__global__ void __launch_bounds__(128) k_apply(DevView v, const double* x, double* y, int nonlinear) {
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  apply_dispatch<N>(v, t, lane, x, y, nonlinear);
}

#define HEVI_ORDER_SWITCH(order, CALL) \
  switch (order) {                       \
    case 1: CALL(1); break;              \
    case 2: CALL(2); break;              \
    case 3: CALL(3); break;              \
    case 4: CALL(4); break;              \
    case 5: CALL(5); break;              \
    default: break;                      \
  }

static unsigned col_grid(const DevView& v, int blk) {
  const int tiles_per_blk = blk / kTile;
  return (unsigned)((v.tile_count + tiles_per_blk - 1) / tiles_per_blk);
}

void launch_apply(const DevView& v, int order, const double* x, double* y, int nonlinear,
                  cudaStream_t st) {
#define HEVI_CALL(NN) k_apply<NN><<<col_grid(v, 128), 128, 0, st>>>(v, x, y, nonlinear)
  HEVI_ORDER_SWITCH(order, HEVI_CALL)
#undef HEVI_CALL
}

// Full right-hand side S(Q) = H + V(Q) of a stage value (Sec. 4.1, 4.3).
template <int N>
__device__ void apply_rhs_dispatch(const DevView& v, const TileDesc& t, int lane, const double* Q,
                                   const double* H, double* S) {
  const Col c = make_col(v, t, lane, N);
  apply_V_column<N>(v, c, Q, S, 0.0, H, nullptr);
}

template <int N>
__global__ void __launch_bounds__(128) k_apply_rhs(DevView v, const double* Q, const double* H,
                                                   double* S) {
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  apply_rhs_dispatch<N>(v, t, lane, Q, H, S);
}

void launch_apply_rhs(const DevView& v, int order, const double* Q, const double* H, double* S,
                      cudaStream_t st) {
#define HEVI_CALL(NN) k_apply_rhs<NN><<<col_grid(v, 128), 128, 0, st>>>(v, Q, H, S)
  HEVI_ORDER_SWITCH(order, HEVI_CALL)
#undef HEVI_CALL
}

// ARK stage tendencies of the LHEVI split (Sec. 4.3):
//   LQ = L(q0) Q,   E = H + V(Q) - L Q.
template <int N>
__device__ void apply_stage_dispatch(const DevView& v, const TileDesc& t, int lane,
                                     const double* Q, const double* H, double* E, double* LQ) {
  const Col c = make_col(v, t, lane, N);
  apply_L_column<N>(v, c, Q, LQ);
  apply_V_column<N>(v, c, Q, E, 0.0, H, LQ);
}

template <int N>
__global__ void __launch_bounds__(128) k_apply_stage(DevView v, const double* Q, const double* H,
                                                     double* E, double* LQ) {
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  apply_stage_dispatch<N>(v, t, lane, Q, H, E, LQ);
}

void launch_apply_stage(const DevView& v, int order, const double* Q, const double* H, double* E,
                        double* LQ, cudaStream_t st) {
#define HEVI_CALL(NN) k_apply_stage<NN><<<col_grid(v, 128), 128, 0, st>>>(v, Q, H, E, LQ)
  HEVI_ORDER_SWITCH(order, HEVI_CALL)
#undef HEVI_CALL
}

// Rounding floor of the Newton stop: |S^-1 F| <= 512 eps |S^-1 q|, eps = 2^-52
// (a residual evaluated in FP64 stalls at 60-90 eps |S^-1 q| on the stiffest
// columns of the workloads, acoustic Courant number ~500).
constexpr double kNewtonFloor = 512.0 * 2.220446049250313e-16;

// ---------------------------------------------------------------------------
// NHEVI-LU Newton solve (Sec. 4.2.3), one column per thread, fused:
//   F(q) = q - Lambda V(q) - R (FP64), y = -S^-1 F (FP32);
//   J(q) assembled from FP64 point coefficients, equilibrated, LU-factored in
//   FP32 with the L part applied to y on the fly; U records to scratch;
//   backward sweep; q += S y (FP64); repeat until
//   |S^-1 F(q_m)| <= max(rtol |S^-1 F(q_0)|, 512 eps |S^-1 q_m|) or max_iter updates.
// ---------------------------------------------------------------------------
template <int N>
__device__ void newton_column(const DevView& v, const TileDesc& t, int lane, double lam, double* q,
                              const double* R, double rtol, int max_iter, float* win, float* y,
                              int stride) {
  constexpr int K = Band<N>::K;
  constexpr int UR2 = ((2 * K + 1) + 3) / 4 * 4;  // {1/u_jj, u_j,j+1 .. u_j,j+2K}
  const Col c = make_col(v, t, lane, N);
  const Phys ph = v.ph;
  const double* ref = v.ref + c.off;
  double* lin = v.lin + c.off;
  double* qc = q + c.off;
  const double* Rc = R + c.off;
  const double cs = ph.cs;
  float* scr = v.scr + t.scr_off;
  auto urec = [&](int j, int e) -> float* {
    return scr + ((int64_t)(j * (UR2 / 4) + e / 4) * kTile + lane) * 4 + (e & 3);
  };
  bool ok = true;

  // F pass with the pending update q += S y (when `update`); returns |S^-1 F|
  // and leaves |S^-1 q| in qnorm.
  double qnorm = 0.0;
  auto fpass = [&](bool update) -> double {
    double fn = 0.0, qn = 0.0;
    auto flux = [&](int I, double* f) {
      double qi[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = 3 * I + u;
        qi[u] = qc[i];
        if (update) {
          qi[u] += (double)y[i * stride] * ref_scale(ref, cs, 3 * I, u);
          qc[i] = qi[u];
        }
      }
      double w, th, cc, dP;
      if (!lin_coefs(ph, qi[0], qi[1], qi[2], ref[3 * I + 2], ref[3 * I + 1], &w, &th, &cc, &dP,
                     v.ithb ? v.ithb + c.off / 3 + I : nullptr)) {
        ok = false;
        w = th = cc = dP = 0.0;
      }
      lin[3 * I] = w;
      lin[3 * I + 1] = th;
      lin[3 * I + 2] = cc;
      f[0] = qi[1];
      f[1] = fma(qi[1], w, dP);
      f[2] = qi[2] * w;
    };
    auto out = [&](int I, const double* D) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = 3 * I + u;
        double F;
        if (u == 1 && (I == 0 || I == c.nz - 1)) {
          F = qc[i] - Rc[i];
        } else {
          // F = q - Lambda V - R,  V = -D - g (rho - rho_bar) e_m
          double vterm = D[u];
          if (u == 1) vterm = fma(ph.g, qc[3 * I] - ref[3 * I], vterm);
          F = fma(lam, vterm, qc[i]) - Rc[i];
        }
        const double sc = ref_scale(ref, cs, 3 * I, u);
        const double sF = F / sc, sq = qc[i] / sc;
        fn += sF * sF;
        qn += sq * sq;
        y[i * stride] = (float)(-sF);
      }
    };
    element_pass<N>(c, c_tab.w[N], c_tab.iw[N], flux, out);
    qnorm = sqrt(qn);
    return sqrt(fn);
  };
  // converged: the relative test of Sec. 4.2.3, or the residual at the
  // rounding level of its own FP64 evaluation (where the relative test cannot
  // be met: |F(q_0)| itself within 1/rtol of that level)
  auto converged = [&](double fn, double f0) {
    return fn <= rtol * f0 || fn <= kNewtonFloor * qnorm;
  };

  for (int i = c.n; i < c.n + 2 * K; ++i) y[i * stride] = 0.0f;
  const double f0 = fpass(false);
  int it = 0, status = HEVI_COL_OK;
  if (!ok) status = HEVI_COL_BAD_INPUT;
  if (ok && !converged(f0, f0) && max_iter > 0) {
    status = HEVI_COL_NOT_CONVERGED;
    for (it = 1; it <= max_iter; ++it) {
      // factor J(q_m) with the forward substitution applied to y on the fly
      const int info = band_lu<N, float, true>(
          v, c, lam, win, stride, [&](int j, const float* l, float invd, int p, auto&& U) {
            float yj = y[j * stride];
            if (p) {
              const float tt = y[(j + p) * stride];
              y[(j + p) * stride] = yj;
              yj = tt;
              y[j * stride] = yj;
            }
#pragma unroll
            for (int r = 1; r <= K; ++r) y[(j + r) * stride] -= l[r - 1] * yj;
            *urec(j, 0) = invd;
#pragma unroll
            for (int cc = 1; cc <= 2 * K; ++cc) *urec(j, cc) = U(cc);
          });
      if (info) {
        status = HEVI_COL_SINGULAR;
        break;
      }
      for (int j = c.n - 1; j >= 0; --j) {
        float s = y[j * stride];
#pragma unroll
        for (int cc = 1; cc <= 2 * K; ++cc) s -= *urec(j, cc) * y[(j + cc) * stride];
        y[j * stride] = s * *urec(j, 0);
      }
      const double fn = fpass(true);
      if (!ok) {
        status = HEVI_COL_BAD_INPUT;
        break;
      }
      if (converged(fn, f0)) {
        status = HEVI_COL_OK;
        break;
      }
    }
    if (it > max_iter) it = max_iter;
  }
  v.col_iters[c.col] = it;
  if (status != HEVI_COL_OK)
    fail(v, c.col, status);
  else
    v.col_status[c.col] = HEVI_COL_OK;
}

template <int N>
__global__ void __launch_bounds__(64) k_newton(DevView v, double lam, double* q, const double* R,
                                               double rtol, int max_iter, int win_slots) {
  extern __shared__ unsigned char smem_raw[];
  float* smem = reinterpret_cast<float*>(smem_raw);
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  const int stride = blockDim.x;
  float* win = smem + threadIdx.x;
  float* y = smem + (int64_t)win_slots * stride + threadIdx.x;
  newton_column<N>(v, t, lane, lam, q, R, rtol, max_iter, win, y, stride);
}

template <int N>
static void launch_newton_n(const DevView& v, double lam, double* q, const double* R, double rtol,
                            int max_iter, int ylen, cudaStream_t st) {
  const int slots = window_slots(N);
  const int blk = pick_block((slots + ylen) * (int)sizeof(float), 64);
  const int smem = (slots + ylen) * blk * (int)sizeof(float);
  cudaFuncSetAttribute(k_newton<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_newton<N><<<col_grid(v, blk), blk, smem, st>>>(v, lam, q, R, rtol, max_iter, slots);
}

void launch_newton(const DevView& v, int order, double lam, double* q, const double* R,
                   double rtol, int max_iter, int ylen, cudaStream_t st) {
#define HEVI_CALL(NN) launch_newton_n<NN>(v, lam, q, R, rtol, max_iter, ylen, st)
  HEVI_ORDER_SWITCH(order, HEVI_CALL)
#undef HEVI_CALL
}

// ---------------------------------------------------------------------------
// out = base + sum_t coef[t] vec[t]  (ARK stage right-hand sides and update)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// NHEVI-GMRES (Sec. 4.2.1): Jacobian-free Newton-Krylov, one column per
// thread.  Newton on F(q) = q - Lambda V(q) - R; each Newton system is solved
// by unrestarted GMRES (modified Gram-Schmidt Arnoldi, Givens rotations) on
// the equilibrated system J^ y = -S^-1 F, J^ = S^-1 J S, with the Frechet
// difference J^ v ~ S^-1 [F(q + eps S v) - F(q)] / eps (diagonal perturbation
// eps S).  FP64 throughout.  The Krylov basis, the Hessenberg columns (column
// k keeps its k+2 entries at k (k+3) / 2) and the rotations live in per-tile
// scratch interleaved over the tile's 32 lanes; F, the perturbed state and
// its V use three state-size scratch vectors.
// ---------------------------------------------------------------------------
template <int N>
__device__ void gmres_column(const DevView& v, const TileDesc& t, int64_t tile, int lane,
                             const GmArgs& a) {
  const Col c = make_col(v, t, lane, N);
  const int n = c.n, kmax = a.kmax;
  const double cs0 = v.ph.cs, lam = a.lam, eps = a.eps;
  const double* ref = v.ref + c.off;
  auto scl = [&](int i) { return ref_scale(ref, cs0, 3 * (i / 3), i % 3); };
  double* qc = a.q + c.off;
  const double* Rc = a.R + c.off;
  double* F = a.F + c.off;
  double* Qp = a.Qp + c.off;
  const double* Vp = a.Vp + c.off;
  double* K = a.Kb + tile * a.kstride + lane;  // element (k, i) at 32 (k nmax + i)
  double* H = a.Hb + tile * a.hstride + lane;  // element e at 32 e
  double* rc = a.Ab + tile * a.astride + lane;
  double* rs = rc + 32 * (int64_t)kmax;
  double* g = rs + 32 * (int64_t)kmax;
  double* y = g + 32 * (int64_t)(kmax + 1);
  auto Ke = [&](int k, int i) -> double& { return K[32 * ((int64_t)k * a.nmax + i)]; };
  auto He = [&](int k, int j) -> double& { return H[32 * ((int64_t)k * (k + 3) / 2 + j)]; };
  // F(q) from V(q); returns |S^-1 F|^2 and |S^-1 q|^2
  auto residual = [&](double& f2, double& q2) {
    apply_V_column<N>(v, c, a.q, a.Vp, 0.0, nullptr, nullptr, false);
    f2 = 0.0;
    q2 = 0.0;
    for (int i = 0; i < n; ++i) {
      const double fi = qc[i] - lam * Vp[i] - Rc[i];
      F[i] = fi;
      const double si = scl(i);
      f2 += (fi / si) * (fi / si);
      q2 += (qc[i] / si) * (qc[i] / si);
    }
  };
  double f2, q2;
  residual(f2, q2);
  const double f0 = sqrt(f2);
  int it = 0, kit = 0, status = HEVI_COL_OK;
  if (!(f0 == f0)) status = HEVI_COL_BAD_INPUT;
  else if (f0 > kNewtonFloor * sqrt(q2)) {
    status = HEVI_COL_NOT_CONVERGED;
    for (int m = 1; m <= a.max_newton; ++m) {
      double beta = 0.0;
      for (int i = 0; i < n; ++i) {
        const double bi = -F[i] / scl(i);
        Ke(0, i) = bi;
        beta += bi * bi;
      }
      beta = sqrt(beta);
      for (int i = 0; i < n; ++i) Ke(0, i) /= beta;
      for (int k = 0; k <= kmax; ++k) g[32 * k] = 0.0;
      g[0] = beta;
      int kk = 0;
      for (int k = 0; k < kmax; ++k) {
        // w = S^-1 [F(q + eps S V_k) - F(q)] / eps into slot k+1
        for (int i = 0; i < n; ++i) Qp[i] = qc[i] + eps * scl(i) * Ke(k, i);
        apply_V_column<N>(v, c, a.Qp, a.Vp, 0.0, nullptr, nullptr, false);
        for (int i = 0; i < n; ++i) {
          const double fp = Qp[i] - lam * Vp[i] - Rc[i];
          Ke(k + 1, i) = (fp - F[i]) / eps / scl(i);
        }
        for (int j = 0; j <= k; ++j) {  // modified Gram-Schmidt
          double h = 0.0;
          for (int i = 0; i < n; ++i) h += Ke(k + 1, i) * Ke(j, i);
          He(k, j) = h;
          for (int i = 0; i < n; ++i) Ke(k + 1, i) -= h * Ke(j, i);
        }
        double hn = 0.0;
        for (int i = 0; i < n; ++i) hn += Ke(k + 1, i) * Ke(k + 1, i);
        hn = sqrt(hn);
        He(k, k + 1) = hn;
        for (int i = 0; i < n; ++i) Ke(k + 1, i) = hn > 0.0 ? Ke(k + 1, i) / hn : 0.0;
        for (int j = 0; j < k; ++j) {
          const double t0 = rc[32 * j] * He(k, j) + rs[32 * j] * He(k, j + 1);
          He(k, j + 1) = -rs[32 * j] * He(k, j) + rc[32 * j] * He(k, j + 1);
          He(k, j) = t0;
        }
        const double r = hypot(He(k, k), He(k, k + 1));
        rc[32 * k] = r > 0.0 ? He(k, k) / r : 1.0;
        rs[32 * k] = r > 0.0 ? He(k, k + 1) / r : 0.0;
        He(k, k) = r;
        He(k, k + 1) = 0.0;
        g[32 * (k + 1)] = -rs[32 * k] * g[32 * k];
        g[32 * k] = rc[32 * k] * g[32 * k];
        kk = k + 1;
        if (fabs(g[32 * (k + 1)]) <= a.gtol * beta || hn == 0.0) break;
      }
      kit += kk;
      for (int j = kk - 1; j >= 0; --j) {  // R y = g
        double tj = g[32 * j];
        for (int l = j + 1; l < kk; ++l) tj -= He(l, j) * y[32 * l];
        y[32 * j] = tj / He(j, j);
      }
      for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int j = 0; j < kk; ++j) d += y[32 * j] * Ke(j, i);
        qc[i] += scl(i) * d;
      }
      it = m;
      residual(f2, q2);
      const double fn = sqrt(f2);
      if (!(fn == fn)) {
        status = HEVI_COL_BAD_INPUT;
        break;
      }
      if (fn <= a.rtol * f0 || fn <= kNewtonFloor * sqrt(q2)) {
        status = HEVI_COL_OK;
        break;
      }
    }
  }
  v.col_iters[c.col] = it;
  if (a.kits) a.kits[c.col] = kit;
  if (status != HEVI_COL_OK)
    fail(v, c.col, status);
  else
    v.col_status[c.col] = HEVI_COL_OK;
}

template <int N>
__global__ void __launch_bounds__(64) k_newton_gmres(DevView v, GmArgs a) {
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  gmres_column<N>(v, t, tile, lane, a);
}

void launch_newton_gmres(const DevView& v, int order, const GmArgs& a, cudaStream_t st) {
#define HEVI_CALL(NN) k_newton_gmres<NN><<<col_grid(v, 64), 64, 0, st>>>(v, a)
  HEVI_ORDER_SWITCH(order, HEVI_CALL)
#undef HEVI_CALL
}

constexpr int kMaxTerms = 16;
struct CombineArgs {
  const double* vec[kMaxTerms];
  double coef[kMaxTerms];
  int n;
};

__global__ void k_combine(int64_t count, const double* base, CombineArgs a, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = base ? base[i] : 0.0;
    for (int t = 0; t < a.n; ++t) s = fma(a.coef[t], a.vec[t][i], s);
    out[i] = s;
  }
}

void launch_combine(int64_t count, const double* base, int nterms, const double* const* vec,
                    const double* coef, double* out, cudaStream_t st) {
  CombineArgs a;
  a.n = nterms;
  for (int t = 0; t < nterms && t < kMaxTerms; ++t) {
    a.vec[t] = vec[t];
    a.coef[t] = coef[t];
  }
  const int blk = 256;
  int64_t grid = (count + blk - 1) / blk;
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  k_combine<<<(unsigned)grid, blk, 0, st>>>(count, base, a, out);
}

}  // namespace hevi

// ---------------------------------------------------------------------------
// Newton solve without any device allocation.
//
// For callers that cannot call cudaMalloc (code running inside another
// framework's memory pool or allocator lock, or plugins that must not touch
// the device heap), hevi_newton_solve_noalloc runs the same Newton kernel as
// hevi_newton_solve with all of its scratch -- column table, reference
// state, linearisation coefficients and the U records of the factorisation --
// in one file-scope device array of kNoAllocBytes.  Every GPU that loads this
// library holds that array until the process exits.  All calls share it and
// it keeps the last call's contents, so calls that overlap on the GPU race;
// the failure counters are cleared by every call.
// ---------------------------------------------------------------------------
namespace hevi {
namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
bool g_noalloc_tables[kMaxDevices] = {false};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Fill the column table, tiles and reference state of `ncols` uniform
// columns inside the scratch array, and clear the failure counters.
__global__ void k_noalloc_init(DevView v, int order, int nez, double dz, int64_t n,
                               TileDesc* tiles, int64_t* col_off, int32_t* perm, double* col_dz,
                               int32_t* col_order, int32_t* col_nez) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    for (int k = 0; k < 4; ++k) v.fail_count[k] = 0;
  }
  if (i <= v.ncols) col_off[i] = i * n;
  if (i < v.ncols) {
    perm[i] = (int32_t)i;
    col_dz[i] = dz;
    col_order[i] = order;
    col_nez[i] = nez;
  }
  if (i < v.ntiles) {
    const int K = 3 * (order + 1) - 1;
    const int ur2 = ((2 * K + 1) + 3) / 4 * 4;
    TileDesc t;
    t.order = order;
    t.nez = nez;
    t.first = (int32_t)(i * kTile);
    t.count = (int32_t)min((int64_t)kTile, v.ncols - i * kTile);
    t.fac_off = 0;
    t.scr_off = i * n * ur2 * kTile;
    tiles[i] = t;
  }
}

}  // namespace
}  // namespace hevi

extern "C" hevi_status hevi_newton_solve_noalloc(int32_t nez, int32_t order, double z_top,
                                                 int64_t ncols, double gamma_dt, double* state,
                                                 const double* R, double rtol, int32_t max_iter,
                                                 int32_t* status, int32_t* iters, void* stream) {
  using namespace hevi;
  if (nez < 1 || nez > 4096 || order < 1 || order > kMaxOrder || !(z_top > 0.0) || ncols < 1 ||
      !state || !R || state == R || !status || !iters || !(gamma_dt >= 0.0) || !(rtol >= 0.0) ||
      max_iter < 0 || max_iter > 1000)
    return HEVI_ERR_INVALID_ARG;
  const int64_t nz = (int64_t)nez * order + 1, n = 3 * nz;
  const int K = 3 * (order + 1) - 1, ur2 = ((2 * K + 1) + 3) / 4 * 4;
  const int64_t ntiles = (ncols + kTile - 1) / kTile;
  // scratch layout: fail counters | tiles | col_off | perm | col_dz | order | nez | ref | lin |
  // U records
  size_t off = 0;
  const size_t o_fail = off;
  off = align256(off + 4 * sizeof(int32_t));
  const size_t o_tiles = off;
  off = align256(off + ntiles * sizeof(TileDesc));
  const size_t o_off = off;
  off = align256(off + (ncols + 1) * sizeof(int64_t));
  const size_t o_perm = off;
  off = align256(off + ncols * sizeof(int32_t));
  const size_t o_dz = off;
  off = align256(off + ncols * sizeof(double));
  const size_t o_ord = off;
  off = align256(off + ncols * sizeof(int32_t));
  const size_t o_nez = off;
  off = align256(off + ncols * sizeof(int32_t));
  const size_t o_ref = off;
  off = align256(off + ncols * n * sizeof(double));
  const size_t o_lin = off;
  off = align256(off + ncols * n * sizeof(double));
  const size_t o_scr = off;
  off = align256(off + ntiles * n * ur2 * kTile * sizeof(float));
  if (off > kNoAllocBytes) return HEVI_ERR_INVALID_ARG;  // columns do not fit the scratch array

  // once per device, with that device current: the device address of the
  // scratch array and the LGL tables in constant memory
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HEVI_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HEVI_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  if (!g_noalloc_tables[dev]) {
    upload_tables(lgl_tables());
    if (cudaGetLastError() != cudaSuccess) return HEVI_ERR_CUDA;
    g_noalloc_tables[dev] = true;
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  DevView v{};
  Phys ph;
  ph.T0 = 300.0;
  ph.p0 = 1.0e5;
  ph.R = 287.17;
  ph.cp = 1004.67;
  ph.g = 9.80616;
  ph.cv = ph.cp - ph.R;
  ph.gamma = ph.cp / ph.cv;
  ph.cs = sqrt(ph.gamma * ph.R * ph.T0);
  {
    double coef = 1.0;  // C(gamma, k)
    for (int k = 1; k <= kEosTerms; ++k) {
      coef *= (ph.gamma - k + 1.0) / k;
      ph.bin[k - 1] = coef;
    }
  }
  v.ph = ph;
  v.ncols = ncols;
  v.ntiles = (int32_t)ntiles;
  v.tile_begin = 0;
  v.tile_count = (int32_t)ntiles;
  v.fail_count = reinterpret_cast<int32_t*>(base + o_fail);
  TileDesc* tiles = reinterpret_cast<TileDesc*>(base + o_tiles);
  int64_t* col_off = reinterpret_cast<int64_t*>(base + o_off);
  int32_t* perm = reinterpret_cast<int32_t*>(base + o_perm);
  double* col_dz = reinterpret_cast<double*>(base + o_dz);
  v.tiles = tiles;
  v.col_off = col_off;
  v.perm = perm;
  v.col_dz = col_dz;
  v.ref = reinterpret_cast<double*>(base + o_ref);
  v.lin = reinterpret_cast<double*>(base + o_lin);
  v.scr = reinterpret_cast<float*>(base + o_scr);
  v.fac = nullptr;
  v.fac_status = nullptr;  // not used by the Newton kernel
  v.col_status = status;
  v.col_iters = iters;
  const double dz = z_top / nez;
  const int64_t items = ncols + 1 > ntiles ? ncols + 1 : ntiles;
  int32_t* col_order = reinterpret_cast<int32_t*>(base + o_ord);
  int32_t* col_nez = reinterpret_cast<int32_t*>(base + o_nez);
  k_noalloc_init<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(v, order, nez, dz, n, tiles,
                                                                   col_off, perm, col_dz,
                                                                   col_order, col_nez);
  launch_setup_ref(v, col_order, col_nez, st);
  launch_newton(v, order, gamma_dt, state, R, rtol, max_iter, (int)(n + 2 * K), st);
  int32_t h_fail[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h_fail, v.fail_count, sizeof(h_fail), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return HEVI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return HEVI_ERR_CUDA;
  if (h_fail[0] == 0) return HEVI_OK;
  if (h_fail[3]) return HEVI_ERR_BAD_INPUT;
  if (h_fail[1]) return HEVI_ERR_SINGULAR;
  return HEVI_ERR_NOT_CONVERGED;
}
