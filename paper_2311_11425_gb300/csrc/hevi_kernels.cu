// hevi_kernels.cu -- CUDA kernels of the HEVI vertical column solver (sm_103a):
// the plain FP64 path (band LU with partial pivoting and its solves, one column
// per thread), the operator applies, the NHEVI Newton and GMRES column solves,
// the setup kernels and the allocation-free Newton entry point.  The FP32 path
// (no-pivot factorisation of the equilibrated band and the refined stage
// solve) is in hevi_np.cu.
//
// Work decomposition: 32 columns of one size class form a tile.  FP64 factor
// records are interleaved per tile
//   [step j][record vector][lane][vector lane]
// so that the 32 lanes of a warp read or write one contiguous 512-byte line
// (double2) per record vector.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "hevi_dev.cuh"

namespace hevi {

cudaError_t upload_tables(const LglTables& t) {
  cudaError_t e = cudaMemcpyToSymbol(c_tab, &t, sizeof(LglTables));
  if (e != cudaSuccess) return e;
  return upload_tables_np(t);
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

// ---------------------------------------------------------------------------
// Setup: reference state per point (isothermal, hydrostatic) and rest state
// ---------------------------------------------------------------------------
__global__ void k_setup_ref(DevView v, const int32_t* col_order, const int32_t* col_nez,
                            int64_t first, int64_t last) {
  const int64_t col = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= last) return;
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
    const double P = eos(ph, Th);
    // set 3C keeps the reference energy E_bar = P_bar / (gamma - 1) + rho_bar g z,
    // set 2NC the potential temperature theta_bar
    const double X = ph.eqset == 1 ? P / (ph.gamma - 1.0) + rho * ph.g * z
                     : ph.eqset == 2 ? th
                                     : Th;
    r[3 * I + 0] = rho;
    r[3 * I + 1] = P;
    r[3 * I + 2] = X;
    if (v.ithb) v.ithb[v.col_off[col] / 3 + I] = 1.0 / X;
  }
}

void launch_setup_ref(const DevView& v, const int32_t* col_order, const int32_t* col_nez,
                      cudaStream_t st, int64_t first, int64_t count) {
  if (count < 0) count = v.ncols - first;
  if (count <= 0) return;
  int blk = 128;
  k_setup_ref<<<(unsigned)((count + blk - 1) / blk), blk, 0, st>>>(v, col_order, col_nez, first,
                                                                   first + count);
}

__global__ void k_reference_state(DevView v, double* q, int64_t first, int64_t last) {
  const int64_t col = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= last) return;
  const int64_t a = v.col_off[col], b = v.col_off[col + 1];
  for (int64_t i = a; i < b; i += 3) {
    q[i] = v.ref[i];
    q[i + 1] = 0.0;
    q[i + 2] = v.ref[i + 2];
  }
}

void launch_reference_state(const DevView& v, double* q, cudaStream_t st, int64_t first,
                            int64_t count) {
  if (count < 0) count = v.ncols - first;
  if (count <= 0) return;
  int blk = 128;
  k_reference_state<<<(unsigned)((count + blk - 1) / blk), blk, 0, st>>>(v, q, first,
                                                                         first + count);
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
  const bool nc = v.ph.eqset == 2;
  auto scale = [&](int idx) -> double {  // S entry of unknown idx (set 2NC: c_s for w)
    const int P = idx / 3, u = idx - 3 * P;
    const double rb = ref[3 * P];
    return u == 0 ? rb : (u == 1 ? (nc ? cs : rb * cs) : ref[3 * P + 2]);
  };
  // set 2NC: lin = (w0, rho0, theta0), lin2 = (P_rho, P_theta, Dcal w0, X0, Dcal theta0);
  // the w- and theta-rows carry coefficients of the row's own point
  const double* l2 = nc ? v.lin2 + 2 * c.off : nullptr;
  const double irI = nc ? 1.0 / lin[3 * I + 1] : 0.0, w0I = nc ? lin[3 * I] : 0.0;
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
      if (v.ph.eqset == 1) {  // set 3C: lin = (w, h, z)
        double k0, k1, k2;
        k_row_3c(v.ph, vv, lin[3 * J], lin[3 * J + 1], lin[3 * J + 2], k0, k1, k2);
        kv0 = T(k0); kv1 = T(k1); kv2 = T(k2);
      } else if (nc) {  // set 2NC: Dcal_IJ times these, the w-, theta-rows scaled at I
        if (vv == 0) {
          kv0 = T(lin[3 * J]); kv1 = T(lin[3 * J + 1]); kv2 = T(0);
        } else if (vv == 1) {
          kv0 = T(l2[6 * J] * irI); kv1 = T(w0I); kv2 = T(l2[6 * J + 1] * irI);
        } else {
          kv0 = T(0); kv1 = T(0); kv2 = T(w0I);
        }
      } else if (vv == 0) {
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
  if (nc) {  // set 2NC: the point-local terms of the derivative (gravity among them)
    if (vv == 1) {
      T gr = T(lam * (v.ph.g * irI - l2[6 * I + 3] * irI * irI));
      T gw = T(lam * l2[6 * I + 2]);
      if (SCALED) {
        gr *= T(scale(i - 1)) * inv_si;
        gw *= T(scale(i)) * inv_si;
      }
      row[slot(i - 1) * stride] += gr;
      row[slot(i) * stride] += gw;
    } else if (vv == 2) {
      T gw = T(lam * l2[6 * I + 4]);
      if (SCALED) gw *= T(scale(i - 1)) * inv_si;
      row[slot(i - 1) * stride] += gw;
    }
  } else if (vv == 1) {
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

// Set 2NC: P(rho theta) - P_bar at a point, ref = (rho_bar, P_bar, theta_bar)
// there.  Both products are rounded as written (never fused into a
// multiply-add with the subtraction inside), so that the rest state gives
// exactly zero.
__device__ __forceinline__ double dp_2nc(const Phys& ph, double rho, double th, const double* ref) {
  return eos_perturbation(ph, __dmul_rn(rho, th), __dmul_rn(ref[0], ref[2]), ref[1]);
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
    if (ph.eqset == 2) {  // set 2NC: lin = (w0, rho0, theta0); lin2[0..1] = (P_rho, P_theta)
      if (!(rho > 0.0) || !(Th > 0.0) || !isfinite(m)) ok = false;
      const double P = v.ref[a + 1] + dp_2nc(ph, rho, Th, v.ref + a);
      double* l2 = v.lin2 + 2 * a;
      l2[0] = ph.gamma * P / rho;
      l2[1] = ph.gamma * P / Th;
      l2[5] = 0.0;
      v.lin[a] = m;
      v.lin[a + 1] = rho;
      v.lin[a + 2] = Th;
      continue;
    }
    if (ph.eqset == 1) {  // set 3C: (w, h, z)
      const double z = point_z<N>(1.0 / (0.5 * c.s), I, c.nz);
      double h;
      if (!lin_coefs_3c(ph, rho, m, Th, v.ref[a], v.ref[a + 2], v.ref[a + 1], z, &w, &h, &dP)) {
        ok = false;
        w = h = 0.0;
      }
      th = h;
      cc = z;
    } else if (!lin_coefs(ph, rho, m, Th, v.ref[a + 2], v.ref[a + 1], &w, &th, &cc, &dP)) {
      ok = false;
      w = 0.0; th = 0.0; cc = 0.0;
    }
    v.lin[a] = w;
    v.lin[a + 1] = th;
    v.lin[a + 2] = cc;
  }
  if (ph.eqset == 2) {  // set 2NC: the derivatives of q0 its Jacobian needs at each point
    const double* lc = v.lin + c.off;
    const double* ref = v.ref + c.off;
    double* l2 = v.lin2 + 2 * c.off;
    auto flux = [&](int I, double* f) {
      const double rho = lc[3 * I + 1], th = lc[3 * I + 2];
      f[0] = lc[3 * I];
      f[1] = dp_2nc(ph, rho, th, ref + 3 * I);
      f[2] = th;
    };
    auto out = [&](int I, const double* D) {
      l2[6 * I + 2] = D[0];
      l2[6 * I + 3] = D[1] + ph.g * (lc[3 * I + 1] - ref[3 * I]);
      l2[6 * I + 4] = D[2];
    };
    element_pass<N>(c, c_tab.w[N], c_tab.iw[N], flux, out);
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
  if (v.gate && *v.gate == 0) return;  // nothing left to do (Newton sequence)
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

static int pick_block(int bytes, int max_blk);
static unsigned col_grid(const DevView& v, int blk);
static int window_slots(int N) {
  const int K = 3 * (N + 1) - 1;
  return (K + 1) * (2 * K + 1);
}

template <int N>
static void launch_factor_n(const DevView& v, double lam, const double* q0, cudaStream_t st) {
  const int esz = (int)sizeof(double);
  const int blk = pick_block(window_slots(N) * esz, 64), tiles_per_blk = blk / kTile;
  const unsigned grid = (unsigned)((v.tile_count + tiles_per_blk - 1) / tiles_per_blk);
  const int smem = window_slots(N) * blk * esz;
  if (v.ph.eqset != 0) {
    // sets 3C and 2NC: the band equilibrated with the reference scales (their
    // unknowns differ by orders of magnitude); the solve scales b and x to match
    cudaFuncSetAttribute(k_factor<N, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    k_factor<N, double, true><<<grid, blk, smem, st>>>(v, lam, q0);
    return;
  }
  cudaFuncSetAttribute(k_factor<N, double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_factor<N, double, false><<<grid, blk, smem, st>>>(v, lam, q0);
}

void launch_factor(const DevView& v, int order, hevi_precision prec, double lam, const double* q0,
                   int ylen, cudaStream_t st) {
  if (prec == HEVI_FP32_IR) {  // no-pivot FP32 factorisation (hevi_np.cu)
    launch_factor_np(v, order, lam, q0, ylen, st);
    return;
  }
  switch (order) {
    case 1: launch_factor_n<1>(v, lam, q0, st); break;
    case 2: launch_factor_n<2>(v, lam, q0, st); break;
    case 3: launch_factor_n<3>(v, lam, q0, st); break;
    case 4: launch_factor_n<4>(v, lam, q0, st); break;
    case 5: launch_factor_n<5>(v, lam, q0, st); break;
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
  // sets 3C and 2NC factor S^-1 A S (S: rho_bar, rho_bar c_s or, in set 2NC, c_s,
  // and the third unknown's reference): y = S^-1 b, x = S y
  const bool eq = v.ph.eqset != 0, nc = v.ph.eqset == 2;
  const double* ref = v.ref + c.off;
  auto scale = [&](int i) {
    const int P = i / 3, u = i - 3 * P;
    return u == 0 ? ref[3 * P] : (u == 1 ? (nc ? v.ph.cs : ref[3 * P] * v.ph.cs) : ref[3 * P + 2]);
  };
  for (int i = 0; i < c.n; ++i) y[i * stride] = eq ? b[c.off + i] / scale(i) : b[c.off + i];
  for (int i = c.n; i < c.n + 2 * K; ++i) y[i * stride] = 0.0;
  forward_sweep<N, double, double>(base, lane, c.n, y, stride);
  backward_sweep<N, double, double>(base, lane, c.n, y, stride);
  for (int i = 0; i < c.n; ++i) x[c.off + i] = eq ? y[i * stride] * scale(i) : y[i * stride];
  v.col_iters[c.col] = 1;
}

// Plain FP64 solve; the work vectors live in shared memory.
template <int N>
__global__ void __launch_bounds__(128) k_solve_fp64(DevView v, const double* b, double* x) {
  extern __shared__ unsigned char smem_raw[];
  if (v.gate && *v.gate == 0) return;  // nothing left to do (Newton sequence)
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
static void launch_solve_n(const DevView& v, const double* b, double* x, int ylen, cudaStream_t st) {
  const int esz = (int)sizeof(double);
  const int blk = pick_block(ylen * esz, 128), tiles_per_blk = blk / kTile;
  const unsigned grid = (unsigned)((v.tile_count + tiles_per_blk - 1) / tiles_per_blk);
  const int smem = ylen * blk * esz;
  cudaFuncSetAttribute(k_solve_fp64<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_solve_fp64<N><<<grid, blk, smem, st>>>(v, b, x);
}

void launch_solve(const DevView& v, int order, hevi_precision prec, double lam, const double* b,
                  double* x, double tol, int max_sweeps, int ylen, cudaStream_t st) {
  if (prec == HEVI_FP32_IR) {  // FP32 factors + refinement (hevi_np.cu)
    launch_solve_np(v, order, order, lam, b, x, tol, max_sweeps, st);
    return;
  }
  switch (order) {
    case 1: launch_solve_n<1>(v, b, x, ylen, st); break;
    case 2: launch_solve_n<2>(v, b, x, ylen, st); break;
    case 3: launch_solve_n<3>(v, b, x, ylen, st); break;
    case 4: launch_solve_n<4>(v, b, x, ylen, st); break;
    case 5: launch_solve_n<5>(v, b, x, ylen, st); break;
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
  if (ph.eqset == 2) {
    // set 2NC, unknowns (rho, w, theta):  V_rho = -Dcal[rho w],
    // V_w = -(w Dcal[w] + (Dcal[P - P_bar] + g (rho - rho_bar)) / rho), V_theta = -w Dcal[theta]
    auto flux4 = [&](int I, double* f) {
      const double rho = qc[3 * I], w = qc[3 * I + 1], th = qc[3 * I + 2];
      if (!(rho > 0.0) || !(th > 0.0)) ok = false;
      f[0] = rho * w;
      f[1] = w;
      f[2] = dp_2nc(ph, rho, th, ref + 3 * I);
      f[3] = th;
    };
    auto o4 = [&](int I, const double* D) {
      const double rho = qc[3 * I], w = qc[3 * I + 1];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int64_t i = c.off + 3 * I + u;
        double val;
        if (u == 0)
          val = -D[0];
        else if (u == 1)
          val = (I == 0 || I == c.nz - 1) ? 0.0
                                          : -(w * D[1] + (D[2] + ph.g * (rho - ref[3 * I])) / rho);
        else
          val = -(w * D[3]);
        if (add) val += add[i];
        if (sub) val -= sub[i];
        out[i] = val;
      }
    };
    element_pass<N, 4>(c, c_tab.w[N], c_tab.iw[N], flux4, o4);
    if (!ok && report) fail(v, c.col, HEVI_COL_BAD_INPUT);
    return;
  }
  auto flux = [&](int I, double* f) {
    const double rho = qc[3 * I], m = qc[3 * I + 1], Th = qc[3 * I + 2];
    if (ph.eqset == 1) {  // set 3C: fluxes (m, m^2/rho + P - P_bar, (E + P) m / rho)
      double w, h, dP;
      if (!lin_coefs_3c(ph, rho, m, Th, ref[3 * I], ref[3 * I + 2], ref[3 * I + 1],
                        point_z<N>(1.0 / (0.5 * c.s), I, c.nz), &w, &h, &dP)) {
        ok = false;
        w = h = dP = 0.0;
      }
      f[0] = m;
      f[1] = fma(m, w, dP);
      f[2] = h * m;
      return;
    }
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
  if (v.ph.eqset == 2) {
    // set 2NC: the Frechet derivative of V at q0 (lin = (w0, rho0, theta0), lin2 =
    // (P_rho, P_theta, Dcal w0, X0, Dcal theta0)) applied to x = (r, u, t):
    //   L_rho = -Dcal[w0 r + rho0 u],
    //   L_w   = -(u Dcal w0 + w0 Dcal u - r X0 / rho0^2 + (Dcal[P_rho r + P_theta t] + g r) / rho0),
    //   L_theta = -(u Dcal theta0 + w0 Dcal t)
    const double* l2 = v.lin2 + 2 * c.off;
    auto flux4 = [&](int I, double* f) {
      const double r = xc[3 * I], u = xc[3 * I + 1], t = xc[3 * I + 2];
      f[0] = lin[3 * I] * r + lin[3 * I + 1] * u;
      f[1] = u;
      f[2] = l2[6 * I] * r + l2[6 * I + 1] * t;
      f[3] = t;
    };
    auto o4 = [&](int I, const double* D) {
      const int64_t a = c.off + 3 * I;
      const double r = xc[3 * I], u = xc[3 * I + 1];
      const double w0 = lin[3 * I], r0 = lin[3 * I + 1];
      out[a] = -D[0];
      out[a + 1] = (I == 0 || I == c.nz - 1)
                       ? 0.0
                       : -(u * l2[6 * I + 2] + w0 * D[1] - r * l2[6 * I + 3] / (r0 * r0) +
                           (D[2] + g * r) / r0);
      out[a + 2] = -(u * l2[6 * I + 4] + w0 * D[3]);
    };
    element_pass<N, 4>(c, c_tab.w[N], c_tab.iw[N], flux4, o4);
    return;
  }
  auto flux = [&](int I, double* f) {
    const double x0 = xc[3 * I], x1 = xc[3 * I + 1], x2 = xc[3 * I + 2];
    const double wI = lin[3 * I], thI = lin[3 * I + 1], cI = lin[3 * I + 2];
    if (v.ph.eqset == 1) {  // set 3C: lin = (w, h, z)
      f[0] = x1;
#pragma unroll
      for (int r = 1; r < 3; ++r) {
        double k0, k1, k2;
        k_row_3c(v.ph, r, wI, thI, cI, k0, k1, k2);
        f[r] = fma(k0, x0, fma(k1, x1, k2 * x2));
      }
      return;
    }
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
#define HEVI_CALL(NN) k_apply<NN><<<col_grid(v, kTile), kTile, 0, st>>>(v, x, y, nonlinear)
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
#define HEVI_CALL(NN) k_apply_rhs<NN><<<col_grid(v, kTile), kTile, 0, st>>>(v, Q, H, S)
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
#define HEVI_CALL(NN) k_apply_stage<NN><<<col_grid(v, kTile), kTile, 0, st>>>(v, Q, H, E, LQ)
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
static cudaError_t launch_newton_n(const DevView& v, double lam, double* q, const double* R,
                                   double rtol, int max_iter, int ylen, cudaStream_t st) {
  const int slots = window_slots(N);
  const int blk = pick_block((slots + ylen) * (int)sizeof(float), 64);
  const int smem = (slots + ylen) * blk * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_newton<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_newton<N><<<col_grid(v, blk), blk, smem, st>>>(v, lam, q, R, rtol, max_iter, slots);
  return cudaGetLastError();
}

// Dynamic shared memory the fused Newton kernel needs per block at its
// smallest block (one warp), for columns of n unknowns and order N.
size_t newton_smem_min(int order, int64_t n) {
  const int K = 3 * (order + 1) - 1;
  return (size_t)((K + 1) * (2 * K + 1) + n + 2 * K) * kTile * sizeof(float);
}

// ---------------------------------------------------------------------------
// NHEVI-LU F pass (Sec. 4.2.3), one column per thread, FP64: for a column
// still iterating, apply the update q += delta of iteration m (m >= 1), then
// evaluate F(q) = q - Lambda V(q) - R, write rhs = -F (the right-hand side of
// the next Newton system) and take the stop test
//   |S^-1 F(q_m)| <= rtol |S^-1 F(q_0)|  and  |S^-1 delta_m| <= rtol |S^-1 (q_m - q_0)|,
// or |S^-1 F(q_m)| at the rounding floor of its FP64 evaluation (512 eps
// |S^-1 q_m|); S = (rho_bar, rho_bar c_s, Theta_bar).  The second half of the
// first test (the last update small against the whole update) makes the
// solution agree with the root to about rtol in the update's norm whatever
// the rate of the iteration.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_newton_fpass(DevView v, NewtonArgs a) {
  if (a.active_in && *a.active_in == 0) return;
  const int warp = threadIdx.x / kTile, lane = threadIdx.x % kTile;
  const int64_t tile = v.tile_begin + (int64_t)blockIdx.x * (blockDim.x / kTile) + warp;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;
  const TileDesc t = v.tiles[tile];
  if (lane >= t.count) return;
  const Col c = make_col(v, t, lane, N);
  const Phys ph = v.ph;
  const int64_t col = c.col;
  if (a.iter > 0) {
    if (a.conv[col] != 0) return;
    const int fs = v.fac_status[col];
    if (fs != HEVI_COL_OK) {  // J(q_m) could not be factored
      a.conv[col] = 2;
      a.status[col] = fs;
      return;
    }
  }
  const double* ref = v.ref + c.off;
  double* qc = a.q + c.off;
  const double* Rc = a.R + c.off;
  const double* q0c = a.q0 + c.off;
  double* rc = a.rhs + c.off;
  // The norms of the stop test only compare magnitudes (relative accuracy
  // 1e-7 is ample), so they run in FP32 on values rounded toward zero by
  // integer operations, with S^-1 of point I = 1/rho_bar, 1/(rho_bar c_s),
  // 1/Theta_bar in FP32; F itself is FP64.
  const float ics = 1.0f / ph.csf;
  auto f32 = [](double x) { return df_from_double(x).hi; };
  const bool nc = ph.eqset == 2;  // set 2NC: w is scaled by c_s alone
  auto inv_scales = [&](int I, float (&is)[3]) {
    const float ir = __frcp_rn(f32(ref[3 * I]));
    is[0] = ir;
    is[1] = nc ? ics : ir * ics;
    is[2] = v.ithb ? f32(v.ithb[c.off / 3 + I]) : __frcp_rn(f32(ref[3 * I + 2]));
  };
  float dn2 = 0.0f;
  if (a.iter > 0) {
    const double* dc = a.delta + c.off;
    for (int I = 0; I < c.nz; ++I) {
      float is[3];
      inv_scales(I, is);
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = 3 * I + u;
        const double d = dc[i];
        qc[i] += d;
        const float sd = f32(d) * is[u];
        dn2 = fmaf(sd, sd, dn2);
      }
    }
  }
  const double dn = sqrt((double)dn2);
  bool ok = true;
  float fn2 = 0.0f, qn2 = 0.0f, un2 = 0.0f;
  auto flux = [&](int I, double* f) {
    const double rho = qc[3 * I], m = qc[3 * I + 1], Th = qc[3 * I + 2];
    double w, th, cc, dP;
    if (ph.eqset == 1) {  // set 3C: E-flux (E + P) m / rho = h m
      double h;
      if (!lin_coefs_3c(ph, rho, m, Th, ref[3 * I], ref[3 * I + 2], ref[3 * I + 1],
                        point_z<N>(1.0 / (0.5 * c.s), I, c.nz), &w, &h, &dP)) {
        ok = false;
        w = h = dP = 0.0;
      }
      f[0] = m;
      f[1] = fma(m, w, dP);
      f[2] = h * m;
      return;
    }
    if (!lin_coefs(ph, rho, m, Th, ref[3 * I + 2], ref[3 * I + 1], &w, &th, &cc, &dP,
                   v.ithb ? v.ithb + c.off / 3 + I : nullptr)) {
      ok = false;
      w = dP = 0.0;
    }
    f[0] = m;
    f[1] = fma(m, w, dP);
    f[2] = Th * w;
  };
  auto out = [&](int I, const double* D) {
    float is[3];
    inv_scales(I, is);
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
        F = fma(a.lam, vterm, qc[i]) - Rc[i];
      }
      rc[i] = -F;
      const float isc = is[u];
      const float sF = f32(F) * isc, sq = f32(qc[i]) * isc, su = f32(qc[i] - q0c[i]) * isc;
      fn2 = fmaf(sF, sF, fn2);
      qn2 = fmaf(sq, sq, qn2);
      un2 = fmaf(su, su, un2);
    }
  };
  if (nc) {
    // set 2NC: V_rho = -Dcal[rho w], V_w = -(w Dcal[w] + (Dcal[P - P_bar] + g (rho -
    // rho_bar)) / rho), V_theta = -w Dcal[theta]
    auto flux4 = [&](int I, double* f) {
      const double rho = qc[3 * I], w = qc[3 * I + 1], th = qc[3 * I + 2];
      if (!(rho > 0.0) || !(th > 0.0)) ok = false;
      f[0] = rho * w;
      f[1] = w;
      f[2] = dp_2nc(ph, rho, th, ref + 3 * I);
      f[3] = th;
    };
    auto out4 = [&](int I, const double* D) {
      float is[3];
      inv_scales(I, is);
      const double rho = qc[3 * I], w = qc[3 * I + 1];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = 3 * I + u;
        double F;
        if (u == 1 && (I == 0 || I == c.nz - 1)) {
          F = qc[i] - Rc[i];
        } else {
          // F = q - Lambda V - R with -V as below
          double vterm;
          if (u == 0)
            vterm = D[0];
          else if (u == 1)
            vterm = w * D[1] + (D[2] + ph.g * (rho - ref[3 * I])) / rho;
          else
            vterm = w * D[3];
          F = fma(a.lam, vterm, qc[i]) - Rc[i];
        }
        rc[i] = -F;
        const float isc = is[u];
        const float sF = f32(F) * isc, sq = f32(qc[i]) * isc, su = f32(qc[i] - q0c[i]) * isc;
        fn2 = fmaf(sF, sF, fn2);
        qn2 = fmaf(sq, sq, qn2);
        un2 = fmaf(su, su, un2);
      }
    };
    element_pass<N, 4>(c, c_tab.w[N], c_tab.iw[N], flux4, out4);
  } else {
    element_pass<N>(c, c_tab.w[N], c_tab.iw[N], flux, out);
  }
  const double fn = sqrt((double)fn2), qn = sqrt((double)qn2), un = sqrt((double)un2);
  const double floor_ok = kNewtonFloor * qn;
  int cv = 0, st = HEVI_COL_OK;
  if (!ok || !(fn == fn)) {
    cv = 2;
    st = HEVI_COL_BAD_INPUT;
  } else if (a.iter == 0) {
    a.f0[col] = fn;
    a.iters[col] = 0;
    if (fn == 0.0 || fn <= floor_ok) cv = 1;
  } else {
    a.iters[col] = a.iter;
    if ((fn <= a.rtol * a.f0[col] && dn <= a.rtol * un) || fn <= floor_ok)
      cv = 1;
    else if (a.iter >= a.max_iter) {
      cv = 2;
      st = HEVI_COL_NOT_CONVERGED;
    }
  }
  if (a.iter == 0 && a.max_iter == 0 && cv == 0) {
    cv = 2;
    st = HEVI_COL_NOT_CONVERGED;
  }
  a.conv[col] = cv;
  a.status[col] = st;
  if (cv == 0) atomicAdd(a.active_out, 1);
}

// One warp per block: at 106 registers a thread, blocks of four warps fit four
// to an SM and the launch would spill into a second, nearly empty wave.
void launch_newton_fpass(const DevView& v, int order, const NewtonArgs& a, cudaStream_t st) {
#define HEVI_CALL(NN) k_newton_fpass<NN><<<col_grid(v, kTile), kTile, 0, st>>>(v, a)
  HEVI_ORDER_SWITCH(order, HEVI_CALL)
#undef HEVI_CALL
}

// The per-column result of the Newton sequence into the context's status.
__global__ void k_newton_finish(DevView v, NewtonArgs a) {
  const int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (col >= v.ncols) return;
  const int st = a.status[col];
  v.col_iters[col] = a.iters[col];
  if (st != HEVI_COL_OK)
    fail(v, col, st);
  else
    v.col_status[col] = HEVI_COL_OK;
}

void launch_newton_finish(const DevView& v, const NewtonArgs& a, cudaStream_t st) {
  k_newton_finish<<<(unsigned)((v.ncols + 127) / 128), 128, 0, st>>>(v, a);
}

cudaError_t launch_newton(const DevView& v, int order, double lam, double* q, const double* R,
                          double rtol, int max_iter, int ylen, cudaStream_t st) {
  switch (order) {
    case 1: return launch_newton_n<1>(v, lam, q, R, rtol, max_iter, ylen, st);
    case 2: return launch_newton_n<2>(v, lam, q, R, rtol, max_iter, ylen, st);
    case 3: return launch_newton_n<3>(v, lam, q, R, rtol, max_iter, ylen, st);
    case 4: return launch_newton_n<4>(v, lam, q, R, rtol, max_iter, ylen, st);
    case 5: return launch_newton_n<5>(v, lam, q, R, rtol, max_iter, ylen, st);
    default: return cudaErrorInvalidValue;
  }
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
constexpr int kNoAllocFailSlots = 5;            // the failure counters fail() writes
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
bool g_noalloc_tables[kMaxDevices] = {false};
std::mutex g_noalloc_init;  // the per-device lookups above, made once per device

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Fill the column table, tiles and reference state of `ncols` uniform
// columns inside the scratch array, and clear the failure counters.
__global__ void k_noalloc_init(DevView v, int order, int nez, double dz, int64_t n,
                               TileDesc* tiles, int64_t* col_off, int32_t* perm, double* col_dz,
                               int32_t* col_order, int32_t* col_nez) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    for (int k = 0; k < kNoAllocFailSlots; ++k) v.fail_count[k] = 0;
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
  // every column needs at least its reference state and coefficients (2 n
  // doubles): bound ncols before any offset arithmetic
  if (ncols > (int64_t)(kNoAllocBytes / (2 * (size_t)n * sizeof(double)))) return HEVI_ERR_INVALID_ARG;
  const int64_t ntiles = (ncols + kTile - 1) / kTile;
  // scratch layout: fail counters | tiles | col_off | perm | col_dz | order | nez | ref | lin |
  // U records
  size_t off = 0;
  const size_t o_fail = off;
  off = align256(off + kNoAllocFailSlots * sizeof(int32_t));
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
  // scratch array and the LGL tables in constant memory (serialised, so that
  // first calls from several host threads do not race)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HEVI_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_init);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return HEVI_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    if (!g_noalloc_tables[dev]) {
      if (upload_tables(lgl_tables()) != cudaSuccess) {
        cudaGetLastError();
        return HEVI_ERR_CUDA;
      }
      g_noalloc_tables[dev] = true;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }
  // the Newton kernel's shared memory at its smallest block must fit the device
  {
    int smax = 0;
    if (cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return HEVI_ERR_CUDA;
    }
    if (newton_smem_min(order, n) > (size_t)smax) return HEVI_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  DevView v{};
  Phys ph;
  ph.T0 = 300.0;
  ph.p0 = 1.0e5;
  ph.R = 287.17;
  ph.cp = 1004.67;
  ph.g = 9.80616;
  phys_derive(ph);
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
  if (launch_newton(v, order, gamma_dt, state, R, rtol, max_iter, (int)(n + 2 * K), st) !=
      cudaSuccess) {
    cudaGetLastError();
    return HEVI_ERR_CUDA;
  }
  int32_t h_fail[kNoAllocFailSlots] = {0, 0, 0, 0, 0};
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
