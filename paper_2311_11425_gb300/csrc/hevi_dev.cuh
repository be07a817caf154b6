// hevi_dev.cuh -- device building blocks shared by the kernel translation
// units of the HEVI column solver: the LGL tables in constant memory (one copy
// per translation unit, filled by upload_tables), the element pass of the
// continuous-Galerkin column operator in double-float arithmetic, the
// refinement residual, the linearisation coefficients, the band-entry
// formula of the equilibrated FP32 matrix and the mbarrier / bulk-copy
// primitives.
#pragma once
#include <cstdint>

#include "hevi_internal.cuh"

namespace hevi {

// The LGL tables of every order; each translation unit holds its own copy
// and uploads it in its upload function (upload_tables calls all of them).
static __constant__ LglTables c_tab;

// Height of point I of a column of nez = (nz - 1) / N elements of height dz
// (the ends exact).
template <int N>
__device__ __forceinline__ double point_z(double dz, int I, int nz) {
  if (I == 0) return 0.0;
  if (I == nz - 1) return (double)((nz - 1) / N) * dz;
  const int e = I / N, k = I - e * N;
  return e * dz + (c_tab.xi[N][k] + 1.0) * 0.5 * dz;
}

// Set 3C (App. A.1, Eq. set3c, in a column without horizontal momentum):
// from (rho, m, E) at height z, w = m / rho, the pressure perturbation
// P - P_bar = (gamma - 1)((E - E_bar) - m w / 2 - (rho - rho_bar) g z) (the
// differences to the reference first) and h = (E + P) / rho; false for a
// non-physical state (rho <= 0 or P <= 0).
__device__ __forceinline__ bool lin_coefs_3c(const Phys& ph, double rho, double m, double E,
                                             double rho_bar, double E_bar, double P_bar, double z,
                                             double* w, double* h, double* dP) {
  if (!(rho > 0.0) || !isfinite(m) || !isfinite(E)) return false;
  const double ir = rcp64(rho);
  *w = m * ir;
  *dP = (ph.gamma - 1.0) * ((E - E_bar) - 0.5 * m * *w - (rho - rho_bar) * ph.g * z);
  const double P = P_bar + *dP;
  if (!(P > 0.0)) return false;
  *h = (E + P) * ir;
  return true;
}

// Row v of the set-3C flux Jacobian (App. A.3, Eq. set3c_jacobian without
// horizontal momentum) at a point with w, h = (E + P) / rho and height z:
//   rho-flux (0, 1, 0); m-flux (-w^2 + P_rho, 2w + P_m, P_E);
//   E-flux (w P_rho - h w, h + w P_m, w (1 + P_E)),
// P_rho = (gamma - 1)(w^2/2 - g z), P_m = -(gamma - 1) w, P_E = gamma - 1.
__device__ __forceinline__ void k_row_3c(const Phys& ph, int v, double w, double h, double z,
                                         double& k0, double& k1, double& k2) {
  const double gm = ph.gamma - 1.0, Pr = gm * (0.5 * w * w - ph.g * z), Pm = -gm * w;
  if (v == 0) {
    k0 = 0.0; k1 = 1.0; k2 = 0.0;
  } else if (v == 1) {
    k0 = -w * w + Pr; k1 = 2.0 * w + Pm; k2 = gm;
  } else {
    k0 = w * Pr - h * w; k1 = h + w * Pm; k2 = w * ph.gamma;
  }
}

template <int N, int NC>
__device__ __forceinline__ void elem_deriv(const double (&f)[N + 1][NC], double (&cc)[N + 1][NC]) {
  constexpr int P = (N + 1) / 2;
#pragma unroll
  for (int v = 0; v < NC; ++v) {
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
// shared memory (sm: (2N + 2) x 3 pairs per lane, lane fastest: N + 1 fluxes,
// N derivatives and the carried boundary row) so that one field at a time is
// live in registers.  flux(I, f[3]) gives the point fluxes, out(I, D[3])
// receives the DSS'd derivative; cs = 2 / dz.  The loops over points and
// fields are kept rolled (their data live in the slots): the code stays small
// enough for the instruction cache beside the sweeps it runs with.
template <int N, class FluxF, class OutF>
__device__ __forceinline__ void element_pass_df(int nez, df cs, float2* sm, int lane, FluxF&& flux,
                                                OutF&& out) {
  auto FS = [&](int k, int v) -> float2& { return sm[(k * 3 + v) * kTile + lane]; };
  auto DS = [&](int k, int v) -> float2& { return sm[((N + 1 + k) * 3 + v) * kTile + lane]; };
  auto CS = [&](int v) -> float2& { return sm[((2 * N + 1) * 3 + v) * kTile + lane]; };
#pragma unroll
  for (int v = 0; v < 3; ++v) CS(v) = make_float2(0.0f, 0.0f);
  {
    df f[3];
    flux(0, f);
#pragma unroll
    for (int v = 0; v < 3; ++v) FS(0, v) = df_pack(f[v]);
  }
  const df iw0 = df_of(c_tab.iw2[N][0]);
  for (int e = 0; e < nez; ++e) {
    const int I0 = e * N;
#pragma unroll 1
    for (int k = 1; k <= N; ++k) {
      df f[3];
      flux(I0 + k, f);
#pragma unroll
      for (int v = 0; v < 3; ++v) FS(k, v) = df_pack(f[v]);
    }
    const df sc0 = df_mul(cs, e == 0 ? iw0 : df{0.5f * iw0.hi, 0.5f * iw0.lo});
#pragma unroll 1
    for (int v = 0; v < 3; ++v) {
      df fv[N + 1], cc[N + 1];
#pragma unroll
      for (int k = 0; k <= N; ++k) fv[k] = df_of(FS(k, v));
      elem_deriv_df1<N>(fv, cc);
      DS(0, v) = df_pack(df_mul(df_add(df_of(CS(v)), cc[0]), sc0));
#pragma unroll
      for (int k = 1; k < N; ++k) DS(k, v) = df_pack(df_mul(cc[k], df_mul(cs, df_of(c_tab.iw2[N][k]))));
      CS(v) = df_pack(cc[N]);
      FS(0, v) = FS(N, v);
    }
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      const df D[3] = {df_of(DS(k, 0)), df_of(DS(k, 1)), df_of(DS(k, 2))};
      out(I0 + k, D);
    }
  }
  const df sc = df_mul(cs, iw0);
  const df D[3] = {df_mul(df_of(CS(0)), sc), df_mul(df_of(CS(1)), sc), df_mul(df_of(CS(2)), sc)};
  out(nez * N, D);
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

// A tile's point coefficients (w, theta, c) of L(q0) for the refinement
// residual, FP64, interleaved [row][lane] so that a warp's 32 columns read
// one contiguous 256-byte line per row.
__device__ __forceinline__ double* tile_lin(const DevView& v, const TileDesc& t) {
  return reinterpret_cast<double*>(v.ysc + t.y_off);
}

// Height of point I of a column with element height dz (FP32).
template <int N>
__device__ __forceinline__ float np_point_z(float dz, int I, int nz) {
  int e = I / N;
  if (I == nz - 1) e = (nz - 1) / N - 1;
  const int k = I - e * N;
  return dz * ((float)e + c_tab.xh[N][k]);
}

// Equilibration scales of the FP32 path at height z: S = (rho_bar, rho_bar c_s,
// Theta_bar) of the isothermal reference state, evaluated in FP32 (the factor
// and the solve use the same formula, so the scaling is consistent; it only
// conditions the FP32 factors and does not enter the FP64 residual).
__device__ __forceinline__ void np_scales(const Phys& ph, float z, float (&s)[3]) {
  const float rho = ph.rho0f * __expf(-ph.za * z);
  s[0] = rho;
  s[1] = rho * ph.csf;
  if (ph.eqset == 1)
    s[2] = rho * (ph.cvT0f + ph.gf * z);  // set 3C: E_bar = rho_bar (c_v T0 + g z)
  else
    s[2] = rho * (ph.T0f * __expf(ph.zb * z));  // Theta_bar
}

// Prefetch the line holding p into L1 (no registers held).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// cp.async (8-byte, L1-allocating) from global to shared memory, and its
// group completion.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
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
// mbarrier and bulk-copy primitives (cp.async.bulk: the TMA engine's linear
// mode).  Every wait is bounded: mbar_wait waits with try_wait (the thread
// may be suspended up to kWaitHintNs per try, and resumes when the phase
// completes) and gives up after kWaitCycles SM clock cycles, about a second.
// ---------------------------------------------------------------------------
constexpr long long kWaitCycles = 2000000000ll;
constexpr unsigned kWaitHintNs = 2000;

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
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}
__device__ __forceinline__ uint64_t evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
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

// Scales S = (rho_bar, rho_bar c_s, Theta_bar) of unknown (I, u).
__device__ __forceinline__ double ref_scale(const double* ref, double cs, int64_t a, int u) {
  return u == 0 ? ref[a] : (u == 1 ? ref[a] * cs : ref[a + 2]);
}

}  // namespace hevi
