// hevi_np.cu -- the FP32 path of the HEVI stage solve (sm_103a): LU
// factorisation of the equilibrated band without pivoting, and the stage
// solve with iterative refinement.
//
// The band A = I + Lambda Dcal K(q0) + Lambda G (Sec. 4.2.3, App. A.3) is
// equilibrated with the reference-state scales S = (rho_bar, rho_bar c_s,
// Theta_bar), A_hat = S^-1 A S, rounded to FP32 and factored A_hat = L U
// without interchanges: L keeps K = k_l sub-diagonals and U keeps K = k_u
// super-diagonals, so a pivot step stores 2K + 1 numbers instead of the 3K + 2
// of partial pivoting, and neither triangular sweep has a data-dependent
// interchange.  The refinement residual b - A x is evaluated in double-float
// arithmetic from the FP64 point coefficients of L(q0), so the factors only
// precondition the iteration: the solution matches the partially pivoted FP64
// solve of the same system to the refinement tolerance.  A pivot that is
// exactly zero marks the column SINGULAR.
//
// Record layout (NpBand<N>): per tile of 32 columns all forward records
// F_j = {l_(j+1)j .. l_(j+K)j} (column j of L), then all backward records
// B_j = {1/u_jj, u_j,j+1 .. u_j,j+K} (row j of U), each [step][float4
// vector][lane][4], so one step of a tile is one contiguous block and a run
// of steps is one bulk copy.
#include <algorithm>
#include <cstdio>

#include "hevi_dev.cuh"

namespace hevi {

cudaError_t upload_tables_np(const LglTables& t) {
  return cudaMemcpyToSymbol(c_tab, &t, sizeof(LglTables));
}

namespace {

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

}  // namespace

// ---------------------------------------------------------------------------
// Factorisation: one thread per row of the column's active window
// ((K+1) rows x (K+1) columns of A_hat), GW threads per column (the power of
// two >= K+1), 32/GW columns per warp, blocks of four warps.  Without
// interchanges thread r always holds the rows r, r + (K+1), r + 2(K+1), ...
// At step j:
//  - every thread forms one entry of the row that replaces row j (row
//    j+K+1, columns j+1 .. j+K+1) and, for its own row, the entry of the
//    column that enters the window (column j+K+1);
//  - the thread holding row j (the pivot) publishes {1/u_jj, u_j,j+1 ..
//    u_j,j+K} as whole float4 vectors to shared memory, writes the same
//    vectors as the backward record B_j, and loads the replacement row;
//  - the other threads form their multiplier, write it to the forward record
//    F_j and update their K entries in registers (a[s] <- a[s+1] - l u[s+1]:
//    the window moves one column per step).
// Row and column indices advance by one per step, so their point, variable
// and point class are carried along instead of divided out.
// ---------------------------------------------------------------------------
template <int N>
struct NpF {
  using B = NpBand<N>;
  static constexpr int K = B::K, WR = B::WR;
  static constexpr int GW = WR <= 8 ? 8 : (WR <= 16 ? 16 : 32);  // threads per column
  static constexpr int CPW = 32 / GW;                              // columns per warp
  static constexpr int CPB = CPW * 4;                              // columns per block
  static constexpr int UBW = 4 * B::BV;                            // published pivot row
  static constexpr int RBW = (K + 1 + 3) / 4 * 4;                  // replacement row
  // per column in shared memory: UBW + RBW, then per point the scaled K(q0)
  // table (9 floats), the gravity entries (1) and per unknown 1/s (1)
  static constexpr int fixed = UBW + RBW;
};
constexpr int kGSzA = (kGSz + 3) / 4 * 4;  // coefficient table, 16-byte aligned

// A row of A_hat while a thread holds it: index i, point I, variable v (0 rho,
// 1 m, 2 Theta), I mod N, gi = cls (2N+1) + N - I (the coefficient row of its
// point class cls, offset so that gi + J indexes point J), 1/s_i, identity
// row (m at an end: w = 0), and i < n.
struct NpRowF {
  int i, I, v, k, gi;
  float isi;
  bool ident, live;
};

template <int N>
__device__ __forceinline__ void np_row_derive(NpRowF& R, int nz, int n, const float* is32) {
  const int cls = (R.I == 0) ? 0 : (R.I == nz - 1 ? 1 : (R.k == 0 ? 2 : 2 + R.k));
  R.gi = cls * (2 * N + 1) + N - R.I;
  R.live = R.i < n;
  R.isi = R.live ? is32[R.i] : 0.0f;
  R.ident = (R.v == 1) && (R.I == 0 || R.I == nz - 1);
}

template <int N>
__device__ __forceinline__ NpRowF np_row_at(int i, int nz, int n, const float* is32) {
  NpRowF R;
  R.i = i;
  R.I = i / 3;
  R.v = i - 3 * R.I;
  R.k = R.I % N;
  np_row_derive<N>(R, nz, n, is32);
  return R;
}

template <int N>
__device__ __forceinline__ void np_row_next(NpRowF& R, int nz, int n, const float* is32) {
  ++R.i;
  if (++R.v == 3) {
    R.v = 0;
    ++R.I;
    R.k = (R.k + 1 == N) ? 0 : R.k + 1;
  }
  np_row_derive<N>(R, nz, n, is32);
}

// Set 3C point of the FP32 factor (App. A.1, A.3): the linearisation
// coefficients (w, h) of q0 at height z, and the point's scaled Jacobian rows
// ks[3 v + u] = lam_s K~_vu s_u with K~ = K T: the band is factored in the
// variables (rho, m, E - g z rho), T the identity but for g z at (E, rho), so
// the rho column of K gains g z times its E column and the identity part of
// the band gains the entry g z s_rho at (E, rho) (*kz; divided by s_E in the
// row).  False for a non-physical q0 (w = h = 0 then).
__device__ __forceinline__ bool np_point_3c(const Phys& ph, double rho, double m, double E,
                                          double rho_bar, double E_bar, double P_bar, double z,
                                          float s0, float s1, float s2, float lam_s, float* ks,
                                          float* kz, double* wh) {
  double w, h, dP;
  const bool ok = lin_coefs_3c(ph, rho, m, E, rho_bar, E_bar, P_bar, z, &w, &h, &dP);
  if (!ok) w = h = 0.0;
  const double zeta = ph.g * z;
  for (int r = 0; r < 3; ++r) {
    double k0, k1, k2;
    k_row_3c(ph, r, w, h, z, k0, k1, k2);
    ks[3 * r] = lam_s * ((float)(k0 + zeta * k2) * s0);
    ks[3 * r + 1] = lam_s * ((float)k1 * s1);
    ks[3 * r + 2] = lam_s * ((float)k2 * s2);
  }
  *kz = (float)zeta * s0;
  wh[0] = w;
  wh[1] = h;
  return ok;
}

// Entry (i, col) of A_hat = S^-1 (I + Lambda Dcal K(q0) + Lambda G) S (Sec.
// 4.2.3, App. A.3), col = 3J + u, from the column's tables
//   KSp[9 J + 3 v + u] = Lambda (2/dz) K_vu(q0_J) s_(3J+u),  KG[J] = Lambda g s_(3J):
//   delta + G[cls][J - I] KSp / s_i + KG / s_i [v = m, u = rho, J = I]
//   + KZ / s_i [v = E, u = rho, J = I] (set 3C, EQ3),
// identity rows at the ends' m unknowns, 0 outside the band or past the last
// unknown (colok: col < n).
template <int N, bool EQ3>
__device__ __forceinline__ float np_ent(const NpRowF& R, int col, int J, int u, bool colok,
                                        const float* G, const float* KSp, const float* KG,
                                        const float* KZ) {
  const int dJ = J - R.I;
  const bool live = R.live && colok;
  const bool inb = live && (unsigned)(dJ + N) <= 2u * N;
  const float g = G[inb ? R.gi + J : 0];
  const float ks = KSp[inb ? 9 * J + 3 * R.v + u : 0];
  const float one = (col == R.i && live) ? 1.0f : 0.0f;
  float a = fmaf(inb ? g * ks : 0.0f, R.isi, one);
  if (R.v == 1 && u == 0 && dJ == 0 && live) a = fmaf(KG[J], R.isi, a);
  if (EQ3 && R.v == 2 && u == 0 && dJ == 0 && live) a = fmaf(KZ[J], R.isi, a);
  return R.ident ? one : a;
}

template <int N, bool EQ3>
__global__ void __launch_bounds__(128) k_factor_np(DevView v, double lam, const double* q0,
                                                   int linstride) {
  using P = NpF<N>;
  using B = NpBand<N>;
  constexpr int K = P::K, WR = P::WR, GW = P::GW, FV = B::FV, BV = B::BV;
  constexpr int NG = (N + 2) * (2 * N + 1);
  extern __shared__ __align__(16) float np_smem[];
  if (v.gate && *v.gate == 0) return;  // nothing left to do (Newton sequence)
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int sub = lane / GW, r = lane % GW;
  constexpr int bpt = kTile / P::CPB;  // blocks per tile
  const int64_t tile = v.tile_begin + blockIdx.x / bpt;
  const TileDesc t = v.tiles[tile];
  const int cl0 = (blockIdx.x % bpt) * P::CPB;
  float* G = np_smem;
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
  float* ub = np_smem + kGSzA + (int64_t)colw * (P::fixed + 5 * linstride);
  float* rb = ub + P::UBW;
  float* KSp = rb + P::RBW;          // per point: 9 floats
  float* KG = KSp + 3 * linstride;   // per point: gravity entry
  float* KZ = KG + c.nz;             // per point: set 3C's E-row entry at rho (after KG)
  float* is32 = KG + linstride;      // per unknown: 1 / s
  const int n = c.n, nz = c.nz;
  float* fb = reinterpret_cast<float*>(v.fac) + t.fac_off;                   // F records
  float4* bb4 = reinterpret_cast<float4*>(fb + (int64_t)n * FV * 4 * kTile);  // B records
  double* lin_t = tile_lin(v, t);
  const float dzf = (float)v.col_dz[c.col];
  const float lam_s = (float)(lam * c.s), lam_g = (float)(lam * ph.g);

  // point coefficients of L(q0) (FP64): w, theta, c = gamma P / Theta, and the
  // equilibration scales of the point
  bool ok = true;
  for (int I = r; I < nz; I += GW) {
    float sc[3];
    np_scales(ph, np_point_z<N>(dzf, I, nz), sc);
#pragma unroll
    for (int u = 0; u < 3; ++u) is32[3 * I + u] = 1.0f / sc[u];
    KG[I] = lam_g * sc[0];
    const int64_t a = c.off + 3 * I;
    double rho, m, Th;
    if (q0) {
      rho = q0[a]; m = q0[a + 1]; Th = q0[a + 2];
    } else {
      rho = v.ref[a]; m = 0.0; Th = v.ref[a + 2];
    }
    double w, th, cc, dP;
    float* ks = KSp + 9 * I;
    if (EQ3) {  // lin = (w, h, z)
      const double z = point_z<N>((double)v.col_dz[c.col], I, nz);
      double wh[2];
      if (!np_point_3c(ph, rho, m, Th, v.ref[a], v.ref[a + 2], v.ref[a + 1], z, sc[0], sc[1],
                       sc[2], lam_s, ks, KZ + I, wh))
        ok = false;
      w = wh[0];
      th = wh[1];
      cc = z;
    } else if (!lin_coefs(ph, rho, m, Th, v.ref[a + 2], v.ref[a + 1], &w, &th, &cc, &dP,
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
    if (EQ3) continue;
    // K(q0) at point I (App. A.3 restricted to the vertical), scaled by the
    // column scales and Lambda (2/dz): rho-flux (0, 1, 0), m-flux
    // (-w^2, 2w, c), Theta-flux (-theta w, theta, w)
    const float wf = (float)w, tf = (float)th, cf = (float)cc;
    ks[0] = 0.0f;
    ks[1] = lam_s * sc[1];
    ks[2] = 0.0f;
    ks[3] = lam_s * (-wf * wf * sc[0]);
    ks[4] = lam_s * (2.0f * wf * sc[1]);
    ks[5] = lam_s * (cf * sc[2]);
    ks[6] = lam_s * (-tf * wf * sc[0]);
    ks[7] = lam_s * (tf * sc[1]);
    ks[8] = lam_s * (wf * sc[2]);
  }
  {  // AND over the group's lanes (every lane of the warp takes part)
    int okv = ok ? 1 : 0;
#pragma unroll
    for (int off = 1; off < GW; off <<= 1) okv &= __shfl_xor_sync(0xffffffffu, okv, off, GW);
    ok = okv != 0;
  }
  __syncwarp();

  // initial window: thread r < WR holds row r, a[s] = A_hat[r][s]
  const bool mine = r < WR;
  NpRowF my = np_row_at<N>(mine ? r : n, nz, n, is32);
  float a[WR];
#pragma unroll
  for (int s = 0; s < WR; ++s)
    a[s] = mine ? np_ent<N, EQ3>(my, s, s / 3, s % 3, s < n, G, KSp, KG, KZ) : 0.0f;

  // The main loop keeps, for a row, pointers to its coefficient row in G and
  // its variable's slice of KSp and its effective 1/s (0 for identity rows
  // and rows past the last unknown): entry (i, 3J + u) = gp[J] kp[9J + u] isx.
  // Row j+K+1 (the same for every thread) replaces row j; thread r
  // assembles its column j+1+r (point Jr, variable ur, kr = 9 Jr + ur); the
  // column entering the window is col = j+K+1 (Jc, kc = 9 Jc + uc).
  struct Lean {
    const float* gp;
    const float* kp;
    float isx;
    int I;
  };
  auto lean = [&](const NpRowF& R) {
    Lean L;
    L.gp = G + R.gi;
    L.kp = KSp + 3 * R.v;
    L.isx = (R.live && !R.ident) ? R.isi : 0.0f;
    L.I = R.I;
    return L;
  };
  Lean me = lean(my);
  NpRowF nr = np_row_at<N>(K + 1, nz, n, is32);
  int Jr = (1 + r) / 3, ur = (1 + r) % 3;
  int kr = 9 * Jr + ur;
  int Jc = (K + 1) / 3, uc = (K + 1) % 3;
  int kc = 9 * Jc + uc;
  const bool diag = r == K;  // thread K assembles the diagonal entry of the new row
  const float4* ub4 = reinterpret_cast<const float4*>(ub);
  float* fcol = fb + (int64_t)cl * 4;  // F records of this column, step 0
  int info = 0;
  int pos = r;  // position of this thread's row in the window: row j + pos
  for (int j = 0; j < n; ++j) {
    const int col = j + K + 1;
    if (mine) {
      // entry (j+K+1, j+1+r) (Jr <= I): in the band unless Jr < I - N; the diagonal;
      // gravity at the m row's own rho unknown (Sec. 4.2.3, App. A.3)
      const Lean ln = lean(nr);
      float e = 0.0f;
      if (nr.live && Jr >= ln.I - N) e = ln.gp[Jr] * ln.kp[kr] * ln.isx;
      if (diag && nr.live) e += 1.0f;
      if (nr.v == 1 && ur == 0 && Jr == ln.I && ln.isx != 0.0f) e = fmaf(KG[Jr], ln.isx, e);
      if (EQ3 && nr.v == 2 && ur == 0 && Jr == ln.I && ln.isx != 0.0f) e = fmaf(KZ[Jr], ln.isx, e);
      rb[r] = e;
    }
    // this row's entry in the entering column (above the diagonal: neither
    // the identity nor the gravity entry)
    float ecol = 0.0f;
    if (mine && pos >= 1 && col < n && Jc <= me.I + N) ecol = me.gp[Jc] * me.kp[kc] * me.isx;
    __syncwarp();
    if (mine && pos == 0) {
      const float u = a[0];
      const bool sing = !(fabsf(u) > 0.0f) || !isfinite(u);
      if (sing && info == 0) info = j + 1;
      float row[4 * BV];
      row[0] = sing ? 0.0f : __frcp_rn(u);
#pragma unroll
      for (int s = 1; s < 4 * BV; ++s) row[s] = s <= K ? a[s] : 0.0f;
#pragma unroll
      for (int q = 0; q < BV; ++q)
        reinterpret_cast<float4*>(ub)[q] =
            make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
      // row j retires; this thread takes row j+K+1
#pragma unroll
      for (int q = 0; q < P::RBW / 4; ++q) {
        const float4 x4 = reinterpret_cast<const float4*>(rb)[q];
        if (4 * q < WR) a[4 * q] = x4.x;
        if (4 * q + 1 < WR) a[4 * q + 1] = x4.y;
        if (4 * q + 2 < WR) a[4 * q + 2] = x4.z;
        if (4 * q + 3 < WR) a[4 * q + 3] = x4.w;
      }
      me = lean(nr);
    }
    __syncwarp();
    if (mine && pos >= 1) {
      float uj[4 * BV];
#pragma unroll
      for (int q = 0; q < BV; ++q) {
        const float4 x4 = ub4[q];
        uj[4 * q] = x4.x; uj[4 * q + 1] = x4.y; uj[4 * q + 2] = x4.z; uj[4 * q + 3] = x4.w;
      }
      const float l = (j + pos < n) ? a[0] * uj[0] : 0.0f;
#pragma unroll
      for (int s = 0; s < K; ++s) a[s] = fmaf(-l, uj[s + 1], a[s + 1]);
      a[K] = ecol;
      if (active) {
        const int e = pos - 1;  // 0 .. K-1: vector e / 4, element e % 4
        fcol[(e >> 2) * (kTile * 4) + (e & 3)] = l;
      }
    }
    // B_j = the published row j of U, one float4 vector per thread q < BV
    if (active && r < BV) bb4[((int64_t)j * BV + r) * kTile + cl] = ub4[r];
    pos = (pos == 0) ? K : pos - 1;
    fcol += FV * kTile * 4;
    np_row_next<N>(nr, nz, n, is32);
    if (++ur == 3) { ur = 0; ++Jr; kr += 7; } else { ++kr; }
    if (++uc == 3) { uc = 0; ++Jc; kc += 7; } else { ++kc; }
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

template <int N>
static void launch_factor_np_n(const DevView& v, double lam, const double* q0, int ylen,
                               cudaStream_t st) {
  using P = NpF<N>;
  constexpr int K = NpBand<N>::K;
  const int nmax = ylen - 2 * K;  // longest n of these tiles
  const int linstride = (3 * (nmax / 3) + 3) / 4 * 4;
  const int smem = (kGSzA + P::CPB * (P::fixed + 5 * linstride)) * (int)sizeof(float);
  const unsigned grid = (unsigned)(v.tile_count * (kTile / P::CPB));
  if (v.ph.eqset == 1) {
    cudaFuncSetAttribute(k_factor_np<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_factor_np<N, true><<<grid, 128, smem, st>>>(v, lam, q0, linstride);
  } else {
    cudaFuncSetAttribute(k_factor_np<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_factor_np<N, false><<<grid, 128, smem, st>>>(v, lam, q0, linstride);
  }
}

void launch_factor_np(const DevView& v, int order, double lam, const double* q0, int ylen,
                      cudaStream_t st) {
  switch (order) {
    case 1: launch_factor_np_n<1>(v, lam, q0, ylen, st); break;
    case 2: launch_factor_np_n<2>(v, lam, q0, ylen, st); break;
    case 3: launch_factor_np_n<3>(v, lam, q0, ylen, st); break;
    case 4: launch_factor_np_n<4>(v, lam, q0, ylen, st); break;
    case 5: launch_factor_np_n<5>(v, lam, q0, ylen, st); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// Stage solve with FP32 factors and iterative refinement.
//
// A persistent kernel of one-warp blocks; each warp takes tiles of 32 columns
// (one column per lane) in turn.  Per tile: b is read through a shared-memory
// transpose; then sweeps (forward with L, backward with U, in FP32, the work
// vector y in shared memory) alternate with the fused refinement pass
// x += S y, r = b - A x, y = S^-1 r (double-float, from the FP64 point
// coefficients of L(q0)) until every column's predicted error |d_k|^2 /
// |d_(k-1)| is below tol |x| (or the iteration stops contracting, or
// max_sweeps); x leaves through the transpose.  The factor records stream
// through a shared-memory ring filled by bulk copies (one lane issues the
// copy of a chunk of kChunk steps; completion on the slot's mbarrier).  The
// grid keeps a few warps per SM, so the records of the tiles in flight (their
// first sweep reads them from HBM) are still in L2 when the next sweeps read
// them again.
// ---------------------------------------------------------------------------
// Record ring: D slots of C steps' records each.  A launch lays the ring out
// for the largest order among its tiles (the slot holds the larger of F_j
// and B_j, BV >= FV), so that one ring serves tiles of every smaller order;
// the same bytes hold element_pass_df's slots before the sweeps.
constexpr int kNpC = 2;  // steps per chunk (a power of two)
constexpr int kNpD = 2;  // ring slots
__host__ __device__ constexpr int np_slot_bytes(int n) {
  return kNpC * ((3 * (n + 1) - 1 + 1 + 3) / 4) * 512;
}
__host__ __device__ constexpr int np_elem_slot_bytes(int n) {  // element_pass_df's slots
  return ((2 * n + 2) * 3) * kTile * 8;
}
__host__ __device__ constexpr int np_ring_bytes(int n) {
  return kNpD * np_slot_bytes(n) > np_elem_slot_bytes(n) ? kNpD * np_slot_bytes(n)
                                                         : np_elem_slot_bytes(n);
}
template <int N>
struct NpS {
  using B = NpBand<N>;
  static constexpr int K = B::K, WR = B::WR, FV = B::FV, BV = B::BV;
  static constexpr int C = kNpC, D = kNpD;
  static_assert(C * (FV > BV ? FV : BV) * 512 <= np_slot_bytes(N), "ring slot too small");
  static_assert(np_elem_slot_bytes(N) <= np_ring_bytes(N), "element slots do not fit");
};

// Points per round of the loops that move a tile's vectors: their loads are
// issued together (the warps of an SM hide the latency of one round each).
constexpr int kPts = 4;

// Warp-uniform state of the record ring.  Chunks are numbered continuously
// over the warp's life: chunk k sits in slot k % D and completes the phase of
// parity (k / D) & 1 of that slot's barrier.
struct NpRing {
  unsigned char* buf;
  uint64_t* bar;
  uint32_t slot;              // bytes per slot
  uint32_t issued, consumed;  // chunks issued / consumed so far
  bool ok;
};

// keep: the records will be read again (L2 evict-last), else evict-first.
template <int N>
__device__ __forceinline__ void np_issue(NpRing& rg, const float* src, unsigned bytes, bool drop,
                                         bool keep, int lane) {
  using S = NpS<N>;
  const uint32_t k = rg.issued++;
  if (lane == 0) {
    uint64_t* bar = &rg.bar[k % S::D];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    if (!drop)
      bulk_g2s(rg.buf + (k % S::D) * rg.slot, src, bytes, bar,
               keep ? evict_last_policy() : evict_first_policy());
  }
}

// Wait (bounded) for the next chunk; false once a wait has run out.
template <int N>
__device__ __forceinline__ bool np_wait(NpRing& rg) {
  using S = NpS<N>;
  const uint32_t k = rg.consumed;
  bool good = rg.ok && mbar_wait(&rg.bar[k % S::D], (k / S::D) & 1u);
  good = __all_sync(0xffffffffu, good);
  rg.ok = good;
  return good;
}

// After a wait ran out: wait (bounded) for the copies still in flight, then
// re-arm every barrier so that the ring can serve the next tile.
template <int N>
__device__ void np_reset(NpRing& rg, int lane) {
  using S = NpS<N>;
  for (uint32_t k = rg.consumed; k < rg.issued; ++k) mbar_wait(&rg.bar[k % S::D], (k / S::D) & 1u);
  __syncwarp();
  if (lane == 0) {
    for (int s = 0; s < S::D; ++s) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&rg.bar[s])) : "memory");
      mbar_init(&rg.bar[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  rg.issued = rg.consumed = 0;
  rg.ok = true;
}

// Forward sweep L y = y (unit lower, K sub-diagonals), the window of K+1 rows
// in registers, shifted by one row per step (the shift rides on the update:
// w[r-1] = w[r] - l_r y_j), so the loop body is one step of code; ys is this
// lane's column of the work vector (rows kTile apart), rows n .. n+K zero.
// Rows enter the window two steps ahead of use; lane 0 prefetches the row
// line (one 128-byte line holds the row for the warp) two windows ahead.
// drop_step >= 0 leaves out the copy of the chunk holding that step (test
// hook).
template <int N>
__device__ __forceinline__ void np_forward(NpRing& rg, const float* fb, int n, float* ys, int lane,
                                           int drop_step, bool keep) {
  using S = NpS<N>;
  constexpr int K = S::K, WR = S::WR, FV = S::FV, C = S::C, D = S::D;
  const int nch = (n + C - 1) / C;
  auto issue = [&](int ci) {
    const int cnt = min(C, n - ci * C);
    np_issue<N>(rg, fb + (int64_t)ci * C * FV * 4 * kTile, (unsigned)(cnt * FV * 512),
                drop_step >= ci * C && drop_step < ci * C + cnt, keep, lane);
  };
  for (int ci = 0; ci < D && ci < nch; ++ci) issue(ci);
  float w[WR];
#pragma unroll
  for (int r = 0; r < WR; ++r) w[r] = ys[r * kTile];
  float q0 = ys[WR * kTile], q1 = ys[(WR + 1) * kTile];  // rows j+K+1, j+K+2
  const float* yrow = ys - lane;
#pragma unroll 1
  for (int j = 0; j < n && rg.ok; ++j) {
    const int k = j & (C - 1), ci = j / C;
    if (k == 0 && !np_wait<N>(rg)) break;
    if (lane == 0 && j + 2 * WR <= n + K) prefetch_l1(yrow + (j + 2 * WR) * kTile);
    const float4* rec =
        reinterpret_cast<const float4*>(rg.buf + (rg.consumed % D) * rg.slot) + k * FV * kTile +
        lane;
    float l[4 * FV];
#pragma unroll
    for (int q = 0; q < FV; ++q) {
      const float4 x4 = rec[q * kTile];
      l[4 * q] = x4.x; l[4 * q + 1] = x4.y; l[4 * q + 2] = x4.z; l[4 * q + 3] = x4.w;
    }
    const float yj = w[0];
    ys[j * kTile] = yj;
#pragma unroll
    for (int r = 1; r <= K; ++r) w[r - 1] = fmaf(-l[r - 1], yj, w[r]);
    w[K] = q0;
    q0 = q1;
    q1 = (j + WR + 2 <= n + K) ? ys[(j + WR + 2) * kTile] : 0.0f;
    if (k == C - 1 || j == n - 1) {  // chunk consumed: refill its slot
      __syncwarp();
      rg.consumed++;
      if (ci + D < nch) issue(ci + D);
    }
  }
}

// Backward sweep U x = y (K super-diagonals, row-oriented records B_j =
// {1/u_jj, u_j,j+1 .. u_j,j+K}): x_j = (y_j - sum_s u_j,j+s x_(j+s)) / u_jj
// with the K latest x in registers (shifted by one per step); x overwrites y;
// returns |x|^2.
template <int N>
__device__ __forceinline__ float np_backward(NpRing& rg, const float* bb, int n, float* ys,
                                            int lane, bool keep) {
  using S = NpS<N>;
  constexpr int K = S::K, WR = S::WR, BV = S::BV, C = S::C, D = S::D;
  const int nch = (n + C - 1) / C;
  auto issue = [&](int ci) {  // steps hi = n-1-ci C down to lo
    const int hi = n - 1 - ci * C, lo = max(0, hi - C + 1);
    np_issue<N>(rg, bb + (int64_t)lo * BV * 4 * kTile, (unsigned)((hi - lo + 1) * BV * 512), false,
                keep, lane);
  };
  for (int ci = 0; ci < D && ci < nch; ++ci) issue(ci);
  float xw[K];  // xw[s - 1] = x_(j+s)
#pragma unroll
  for (int s = 0; s < K; ++s) xw[s] = 0.0f;
  float q0 = ys[(n - 1) * kTile], q1 = n >= 2 ? ys[(n - 2) * kTile] : 0.0f;  // y_j, y_(j-1)
  const float* yrow = ys - lane;
  float ss = 0.0f;
#pragma unroll 1
  for (int j = n - 1; j >= 0 && rg.ok; --j) {
    const int i = n - 1 - j, k = i & (C - 1), ci = i / C;
    if (k == 0 && !np_wait<N>(rg)) break;
    if (lane == 0 && j - 2 * WR >= 0) prefetch_l1(yrow + (j - 2 * WR) * kTile);
    const int lo = max(0, n - 1 - ci * C - C + 1);
    const float4* rec = reinterpret_cast<const float4*>(rg.buf + (rg.consumed % D) * rg.slot) +
                        (j - lo) * BV * kTile + lane;
    float u[4 * BV];
#pragma unroll
    for (int q = 0; q < BV; ++q) {
      const float4 x4 = rec[q * kTile];
      u[4 * q] = x4.x; u[4 * q + 1] = x4.y; u[4 * q + 2] = x4.z; u[4 * q + 3] = x4.w;
    }
    float acc0 = q0, acc1 = 0.0f;
#pragma unroll
    for (int s = 1; s <= K; ++s) {
      if (s & 1)
        acc0 = fmaf(-u[s], xw[s - 1], acc0);
      else
        acc1 = fmaf(-u[s], xw[s - 1], acc1);
    }
    const float xj = (acc0 + acc1) * u[0];
    ss = fmaf(xj, xj, ss);
    ys[j * kTile] = xj;
#pragma unroll
    for (int s = K - 1; s >= 1; --s) xw[s] = xw[s - 1];
    xw[0] = xj;
    q0 = q1;
    q1 = j >= 2 ? ys[(j - 2) * kTile] : 0.0f;
    if (k == C - 1 || j == 0) {
      __syncwarp();
      rg.consumed++;
      if (ci + D < nch) issue(ci + D);
    }
  }
  return ss;
}

// Refinement residual of the tile's columns (one per lane), point by point
// through the element pass in double-float arithmetic:
//   v' = S v (v = y, the last sweep's solution in the scaled variables;
//   the product of two floats is exact as a double-float pair; in set 3C
//   v' = T S v, the band having been factored in (rho, m, E - g z rho)),
//   r = base - A v',  A v' = v' + Lambda (Dcal[K(q0) v'] + G v'),
// with base = b (the pair rr + zz) on the first call and the stored residual
// afterwards (r_k+1 = r_k - A d_k).  Then rr = fl(r) and y = S^-1 rr, the
// next right-hand side.  The stored residual is rr alone in set 2C; in set 3C
// it is the pair rr + rl (rl = r - fl(r)): there the first FP32 solve leaves a
// residual of about 2^-24 |A||x| times the LU's growth, and rounding it to
// FP32 bounds the refined solution at about 2^-48 |A||x| times that growth
// times kappa, past 1e-10 on the worst columns.  The first call keeps v in y1 (the first solution),
// later calls add it to zz (zz = v on the call after the second sweep; in set
// 3C that call makes (y1, zz) the normalised pair of y1 + v instead).  The
// point coefficients of L(q0) are read from the tile's scratch (one contiguous
// line per row for the warp).  Writes are predicated on w (the lanes whose
// column goes on).
template <int N>
__device__ void np_residual(const double* lint, int nez, const Phys& ph, float dzf, double cs,
                            double lam, int sweep, float* y, float* y1, float* zz, float* rr,
                            float* rl, float2* slots, int lane, bool w) {
  const int nz = nez * N + 1;
  const bool first = sweep == 1, eq3 = ph.eqset == 1;
  const double* lc0 = lint + lane;
  const df lamd = df_from_double(lam), gd = df_from_double(ph.g), csd = df_from_double(cs);
  auto scaled = [&](int I, float (&v)[3], df (&xp)[3], float (&sc)[3]) {
    np_scales(ph, np_point_z<N>(dzf, I, nz), sc);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      v[u] = y[(3 * I + u) * kTile];
      const float p = sc[u] * v[u];
      xp[u] = {p, fmaf(sc[u], v[u], -p)};
    }
    if (eq3)  // set 3C: x = T S v, E = (E - g z rho) + g z rho
      xp[2] = df_fma(df_mul(gd, df_from_double(lc0[(int64_t)(3 * I + 2) * kTile])), xp[0], xp[2]);
  };
  auto flux = [&](int I, df* f) {
    const double* lc = lc0 + (int64_t)(3 * I) * kTile;
    {  // the rows of the point one element ahead: one line per lane
      const int Ip = I + N;
      if (Ip < nz) {
        const int q = lane % 3, h = lane / 3;  // row 3 Ip + q; lanes 0-8
        const int64_t row = 3 * Ip + q;
        if (h == 0) prefetch_l1(y - lane + row * kTile);
        if (h == 1) prefetch_l1(lc0 - lane + row * kTile);
        if (h == 2) prefetch_l1(lc0 - lane + row * kTile + 16);
        if (h == 3) prefetch_l1(rr - lane + row * kTile);
        if (h == 4 && first) prefetch_l1(zz - lane + row * kTile);
      }
    }
    float v[3], sc[3];
    df xp[3];
    scaled(I, v, xp, sc);
    if (w) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = (3 * I + u) * kTile;
        if (first) {
          y1[i] = v[u];
        } else if (sweep == 2 && eq3) {
          // set 3C: the first FP32 solve is poorer there, so the first
          // correction can be a sizeable part of y1, and zz rounded to FP32
          // would hold x to only 2^-24 of it; y1 + zz becomes a normalised
          // pair, so the later corrections add to a zz below ulp(y1)
          const df p2 = df_two_sum(y1[i], v[u]);
          y1[i] = p2.hi;
          zz[i] = p2.lo;
        } else {
          zz[i] = sweep == 2 ? v[u] : zz[i] + v[u];
        }
      }
    }
    const df wI = df_from_double(lc[0]), thI = df_from_double(lc[kTile]),
             cI = df_from_double(lc[2 * kTile]);
    f[0] = xp[1];
    if (ph.eqset == 1) {  // set 3C: lin = (w, h, z); rows of the flux Jacobian
      const df gm = df_from_double(ph.gamma - 1.0);
      const df w2 = df_mul(wI, wI);
      const df Pr = df_mul(gm, df_sub(df{0.5f * w2.hi, 0.5f * w2.lo}, df_mul(gd, cI)));
      const df Pm = df_mul(gm, df{-wI.hi, -wI.lo});
      const df k10 = df_add(df{-w2.hi, -w2.lo}, Pr), k11 = df_add(df{2.0f * wI.hi, 2.0f * wI.lo}, Pm);
      const df k20 = df_mul(wI, df_sub(Pr, thI)), k21 = df_fma(wI, Pm, thI);
      const df k22 = df_mul(wI, df_from_double(ph.gamma));
      f[1] = df_fma(k10, xp[0], df_fma(k11, xp[1], df_mul(gm, xp[2])));
      f[2] = df_fma(k20, xp[0], df_fma(k21, xp[1], df_mul(k22, xp[2])));
      return;
    }
    // f1 = -w^2 rho + 2 w m + c Theta,  f2 = -theta w rho + theta m + w Theta
    f[1] = df_sub(df_fma({2.0f * wI.hi, 2.0f * wI.lo}, xp[1], df_mul(cI, xp[2])),
                  df_mul(df_mul(wI, wI), xp[0]));
    f[2] = df_sub(df_fma(thI, xp[1], df_mul(wI, xp[2])), df_mul(df_mul(thI, wI), xp[0]));
  };
  auto out = [&](int I, const df* Dv) {
    float v[3], sc[3];
    df xp[3];
    scaled(I, v, xp, sc);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = (3 * I + u) * kTile;
      const df base = first ? df{rr[i], zz[i]} : df{rr[i], eq3 ? rl[i] : 0.0f};
      df r;
      if (u == 1 && (I == 0 || I == nz - 1)) {
        r = df_sub(base, xp[1]);  // identity rows: w = 0 at the ends
      } else {
        df ax = Dv[u];
        if (u == 1) ax = df_fma(gd, xp[0], ax);
        r = df_sub(base, df_fma(lamd, ax, xp[u]));
      }
      if (w) {
        const float rf = __fadd_rn(r.hi, r.lo);
        rr[i] = rf;
        if (eq3) rl[i] = __fadd_rn(__fsub_rn(r.hi, rf), r.lo);
        y[i] = rf * (1.0f / sc[u]);
      }
    }
  };
  element_pass_df<N>(nez, csd, slots, lane, flux, out);
  __syncwarp();
}

// Shared memory of one solve warp: the record ring and its barriers; the
// element pass of the residual parks its slots in the ring's memory (the ring
// is idle between sweeps).  The tile's vectors live in its global scratch,
// [row][lane]: the work vector y (n + K + 1 rows, the rows past n zero), the
// first sweep's solution y1, the sum zz of the later corrections, the
// stored residual rr and its low part rl (set 3C); x = S (y1 + zz).
struct NpWarpMem {
  float2* slots;
};

// The tile's FP32 vectors after its point coefficients in the scratch.
__device__ __forceinline__ float* np_tile_vectors(const DevView& v, const TileDesc& t) {
  const int64_t n = 3 * ((int64_t)t.nez * t.order + 1);
  return v.ysc + t.y_off + 2 * n * kTile;
}

// One tile: 32 columns, one per lane.
template <int N>
__device__ void np_solve_tile(const DevView& v, const TileDesc& t, int lane, double lam,
                              const double* b, double* x, double tol, int max_sweeps, NpRing& rg,
                              const NpWarpMem& wm) {
  using S = NpS<N>;
  constexpr int K = S::K;
  constexpr unsigned FULL = 0xffffffffu;
  const bool valid = lane < t.count;
  const int nz = t.nez * N + 1, n = 3 * nz;
  const float* fb = reinterpret_cast<const float*>(v.fac) + t.fac_off;
  const float* bb = fb + (int64_t)n * S::FV * 4 * kTile;
  const double* lint = tile_lin(v, t);
  const int yr = (n + K + 1 + 3) / 4 * 4;
  float* y = np_tile_vectors(v, t) + lane;
  float* y1 = y + (int64_t)yr * kTile;
  float* zz = y1 + (int64_t)n * kTile;
  float* rr = zz + (int64_t)n * kTile;
  float* rl = rr + (int64_t)n * kTile;
  const bool eq3 = v.ph.eqset == 1;
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
  const float dzf = valid ? (float)v.col_dz[c.col] : 1.0f;
  const double cs = valid ? c.s : 1.0;
  // b, read by each lane from its own column: rr + zz = b as a double-float
  // pair, y = S^-1 b
  // (kPts points a round, their loads issued together)
  const double* bc = b + (valid ? c.off : 0);
  for (int I0 = 0; I0 < nz; I0 += kPts) {
    double bv[3 * kPts];
#pragma unroll
    for (int q = 0; q < 3 * kPts; ++q)
      bv[q] = (valid && 3 * I0 + q < n) ? __ldg(bc + 3 * I0 + q) : 0.0;
#pragma unroll
    for (int p = 0; p < kPts; ++p) {
      const int I = I0 + p;
      if (I < nz) {
        float sc[3];
        np_scales(v.ph, np_point_z<N>(dzf, I, nz), sc);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int i = 3 * I + u;
          const df bi = df_from_double(bv[3 * p + u]);
          rr[i * kTile] = bi.hi;
          zz[i * kTile] = bi.lo;
          y[i * kTile] = __fadd_rn(bi.hi, bi.lo) * (1.0f / sc[u]);
        }
      }
    }
  }
  for (int i = n; i <= n + K; ++i) y[i * kTile] = 0.0f;
  __syncwarp();
  bool ran = active;  // the lanes whose x leaves through the final transpose
  int status = HEVI_COL_NOT_CONVERGED;
  double dprev = 0.0, xnorm = 0.0;
  const int drop = v.drop_copy - 1;
  // sweeps: every lane takes part (the waits are warp-wide); the stop test,
  // the folding of the correction and the residual act on the active lanes.
  // Norms are 2-norms of the scaled variables (the correction |y_k| against
  // the solution |y_1|).
  for (int k = 1; __any_sync(FULL, active); ++k) {
    // the first sweep's records are read again by the next sweep (keep them in L2)
    np_forward<N>(rg, fb, n, y, lane, k == 1 ? drop : -1, k == 1);
    float d2 = 0.0f;
    if (rg.ok) d2 = np_backward<N>(rg, bb, n, y, lane, k == 1);
    bool more = false;
    if (rg.ok && active) {
      const double dn = sqrt((double)d2);
      bool stop = false;
      if (k == 1) {
        xnorm = dn;
        if (dn <= tol * xnorm) {  // zero right-hand side, or tol >= 1: one sweep
          stop = true;
          status = HEVI_COL_OK;
        }
      } else {
        // error left after applying d, from the last contraction; in set 3C
        // only from the third sweep on: there the first ratio |d_2| / |y_1|
        // can understate the contraction of the later corrections (whose
        // right-hand sides are rounding residuals, not the smooth b), and a
        // prediction from it stopped columns at 1e-10 after two sweeps
        const double pred = dn * (dn / dprev);
        if (dn <= tol * xnorm || (pred <= tol * xnorm && (k > 2 || !eq3))) {
          stop = true;
          status = HEVI_COL_OK;
        } else if (dn > 0.5 * dprev) {
          stop = true;  // refinement is not contracting
        }
      }
      if (k >= max_sweeps) stop = true;
      if (stop) {  // fold this sweep's correction: x = S (y1 + zz)
        for (int i0 = 0; i0 < n; i0 += 16) {
          float yv[16], zv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int i = min(i0 + q, n - 1);
            yv[q] = y[i * kTile];
            zv[q] = k > 2 ? zz[i * kTile] : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int i = i0 + q;
            if (i < n) {
              if (k == 1) {
                y1[i * kTile] = yv[q];
                zz[i * kTile] = 0.0f;
              } else {
                zz[i * kTile] = zv[q] + yv[q];
              }
            }
          }
        }
        active = false;
        v.col_iters[c.col] = k;
        if (status != HEVI_COL_OK)
          fail(v, c.col, status);
        else
          v.col_status[c.col] = HEVI_COL_OK;
      } else {
        more = true;
        dprev = dn;
      }
    }
    // the columns that go on: r = base - A S y, y = S^-1 r
    if (rg.ok && __any_sync(FULL, more))
      np_residual<N>(lint, t.nez, v.ph, dzf, cs, lam, k, y, y1, zz, rr, rl, wm.slots, lane, more);
    if (!rg.ok) {  // a copy did not arrive within the wait limit
      np_reset<N>(rg, lane);
      if (active) {
        for (int i = 0; i < n; ++i) x[c.off + i] = __longlong_as_double(0x7ff8000000000000LL);
        v.col_iters[c.col] = k;
        fail(v, c.col, HEVI_COL_WAIT_TIMEOUT);
      }
      ran = false;
      active = false;
    }
    __syncwarp();
  }
  // x = S (y1 + zz) (set 3C: T S (y1 + zz)), written by each lane into its own column
  if (ran) {
    double* xc = x + c.off;
    const df gd3 = df_from_double(v.ph.g);
    df x0 = {0.0f, 0.0f};
    for (int I0 = 0; I0 < nz; I0 += kPts) {
      float a1[3 * kPts], a2[3 * kPts];
#pragma unroll
      for (int q = 0; q < 3 * kPts; ++q) {
        const int i = min(3 * I0 + q, n - 1);
        a1[q] = y1[i * kTile];
        a2[q] = zz[i * kTile];
      }
#pragma unroll
      for (int p = 0; p < kPts; ++p) {
        const int I = I0 + p;
        if (I < nz) {
          float sc[3];
          np_scales(v.ph, np_point_z<N>(dzf, I, nz), sc);
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            // S (y1 + zz) as a double-float pair on the FP32 pipes, one FP64 add
            // (set 3C: T S (y1 + zz), E gaining g z rho)
            df xi = df_mul(df_two_sum(a1[3 * p + u], a2[3 * p + u]), df{sc[u], 0.0f});
            if (u == 0) x0 = xi;
            if (u == 2 && eq3)
              xi = df_fma(df_mul(gd3, df_from_double(lint[(int64_t)(3 * I + 2) * kTile + lane])), x0, xi);
            xc[3 * I + u] = (double)xi.hi + (double)xi.lo;
          }
        }
      }
    }
  }
  __syncwarp();
}

// One persistent launch solves every tile of the launch's range: each warp
// takes the next tile from a device counter (with a tile list, in the list's
// order: the costliest tiles first, so that short ones fill the end of the
// launch) and solves it with the routine of its order.  NO = 1..5: every tile
// has order NO (ring and code for that order alone); NO = 0: tiles of any
// order up to nmax, the ring laid out for nmax.
template <int NO>
__global__ void __launch_bounds__(32, 18) k_solve_np(DevView v, double lam, const double* b,
                                                     double* x, double tol, int max_sweeps,
                                                     int nmax) {
  extern __shared__ __align__(128) unsigned char np_dyn[];
  if (v.gate && *v.gate == 0) return;  // nothing left to do (Newton sequence)
  const int lane = threadIdx.x;
  const int nr = NO ? NO : nmax;
  NpRing rg;
  rg.buf = np_dyn;
  rg.bar = reinterpret_cast<uint64_t*>(np_dyn + np_ring_bytes(nr));
  rg.slot = (uint32_t)np_slot_bytes(nr);
  rg.issued = rg.consumed = 0;
  rg.ok = true;
  NpWarpMem wm;
  wm.slots = reinterpret_cast<float2*>(np_dyn);
  if (lane == 0) {
    for (int s = 0; s < kNpD; ++s) mbar_init(&rg.bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  while (true) {
    int tt = 0;
    if (lane == 0) tt = atomicAdd(v.tile_next, 1);
    tt = __shfl_sync(0xffffffffu, tt, 0);
    if (tt >= v.tile_count) break;
    const int tile = v.tile_list ? v.tile_list[v.tile_begin + tt] : v.tile_begin + tt;
    const TileDesc t = v.tiles[tile];
    if constexpr (NO > 0) {
      if (t.order == NO) np_solve_tile<NO>(v, t, lane, lam, b, x, tol, max_sweeps, rg, wm);
    } else {
      if (t.order > nr) continue;  // outside the ring's layout (not in a valid launch)
      switch (t.order) {
        case 1: np_solve_tile<1>(v, t, lane, lam, b, x, tol, max_sweeps, rg, wm); break;
        case 2: np_solve_tile<2>(v, t, lane, lam, b, x, tol, max_sweeps, rg, wm); break;
        case 3: np_solve_tile<3>(v, t, lane, lam, b, x, tol, max_sweeps, rg, wm); break;
        case 4: np_solve_tile<4>(v, t, lane, lam, b, x, tol, max_sweeps, rg, wm); break;
        case 5: np_solve_tile<5>(v, t, lane, lam, b, x, tol, max_sweeps, rg, wm); break;
        default: break;
      }
    }
  }
}

// Most resident solve warps per SM (the register budget of the launch
// bounds): the sweeps and the double-float residual are chains of dependent
// instructions, and only many warps per SM hide their latency.
constexpr int kNpWarpsPerSm = 18;

using SolveNpKernel = void (*)(DevView, double, const double*, double*, double, int, int);

static SolveNpKernel solve_np_kernel(int order) {
  switch (order) {
    case 1: return k_solve_np<1>;
    case 2: return k_solve_np<2>;
    case 3: return k_solve_np<3>;
    case 4: return k_solve_np<4>;
    case 5: return k_solve_np<5>;
    default: return k_solve_np<0>;
  }
}

int solve_np_max_warps_per_sm(int order, int nmax) {
  const int nr = order ? order : nmax;
  const int smem = np_ring_bytes(nr) + kNpD * 8;
  SolveNpKernel k = solve_np_kernel(order);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTile, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::min(per_sm, kNpWarpsPerSm);
}

void launch_solve_np(const DevView& v, int order, int nmax, double lam, const double* b,
                     double* x, double tol, int max_sweeps, cudaStream_t st) {
  if (order < 0 || order > kMaxOrder || nmax < 1 || nmax > kMaxOrder) return;
  const int nr = order ? order : nmax;
  const int smem = np_ring_bytes(nr) + kNpD * 8;
  int per_sm = solve_np_max_warps_per_sm(order, nmax);
  const int sms = sm_count();
  if (v.solve_wps > 0) {
    per_sm = std::min(per_sm, v.solve_wps);
  } else {
    // each warp solves whole tiles, so the launch takes about ceil(tiles /
    // warps) rounds of one tile's latency: take the fewest rounds the
    // occupancy allows, then the fewest warps per SM that keep that many
    const int rounds = (v.tile_count + per_sm * sms - 1) / (per_sm * sms);
    per_sm = std::min(per_sm, (v.tile_count + rounds * sms - 1) / (rounds * sms));
  }
  const int grid = std::max(1, std::min(v.tile_count, per_sm * sms));
  cudaMemsetAsync(v.tile_next, 0, sizeof(int32_t), st);
  solve_np_kernel(order)<<<(unsigned)grid, kTile, smem, st>>>(v, lam, b, x, tol, max_sweeps, nmax);
}

// ---------------------------------------------------------------------------
// Explicit tendency of the FP32 path: S = H + V(Q) (Sec. 4.1, 4.3; the
// vertical operator of App. A.2 with the reference state subtracted) in
// double-float arithmetic on the FP32 pipes.  Point fluxes
//   f = (m, m^2 / rho + (P - P_bar), Theta m / rho),
// 1 / rho from an FP32 reciprocal and one double-float Newton step, the
// pressure perturbation P_bar ((1 + x)^gamma - 1), x = (Theta - Theta_bar) /
// Theta_bar, from its binomial series (the first three terms in double-float,
// the rest, below |x|^3 of the leading term, in FP32); the differences
// Theta - Theta_bar and rho - rho_bar are taken in FP64 first, where they are
// exact, so that perturbations keep their relative accuracy.  The element
// derivative, the DSS and the output S = H - Dcal f - g (rho - rho_bar) e_m
// (w = 0 rows: H) run in double-float and round once to FP64.  About 48
// significant bits where the FP64 kernel has 53, and a few FP64 operations
// per point instead of a few dozen.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df eos_perturbation_df(const Phys& ph, double dTh, double ithb,
                                                  double P_bar) {
  const df x = df_mul(df_from_double(dTh), df_from_double(ithb));
  if (!(fabsf(x.hi) <= 0.02f))  // far from the reference: the FP64 form
    return df_from_double(P_bar * expm1(ph.gamma * log1p(dTh * ithb)));
  float t = ph.binhi[kEosTerms - 1];
#pragma unroll
  for (int k = kEosTerms - 2; k >= 3; --k) t = fmaf(t, x.hi, ph.binhi[k]);
  df s = df_fma(x, df{t, 0.0f}, df{ph.binhi[2], ph.binlo[2]});
  s = df_fma(x, s, df{ph.binhi[1], ph.binlo[1]});
  s = df_fma(x, s, df{ph.binhi[0], ph.binlo[0]});
  return df_mul(df_mul(df_from_double(P_bar), x), s);
}

// One warp per column, N + 1 lanes per element: lane (el, k) of a round
// holds local point k of element e = e0 + el (the points shared by two
// elements are held twice), evaluates its point flux, gathers its element's
// N + 1 fluxes by shuffles and forms its row of the weighted element
// derivative, cc_k = sum_j w_k Dhat_kj f_j.  Shared points add their two
// rows (the lane of row 0 takes the row N of the lane before it, or, at the
// first element of a round, the last row carried from the previous round)
// and scale by (2/dz) / W_I; every point's output is written by one lane.
// Loads and stores of a round touch consecutive points of the column.
// acc[u] = fma(c[t], v[t][g0 + u], acc[u]) for t = 0 .. n-1 in order (u = 0..2);
// the loads of two terms are issued before their FMAs, so their latencies
// overlap (n is uniform across the warp).
template <int MAXT>
__device__ __forceinline__ void fuse_chain(int n, const double* const (&v)[MAXT],
                                           const double (&c)[MAXT], int64_t g0, double (&acc)[3]) {
#pragma unroll
  for (int t0 = 0; t0 < MAXT; t0 += 2) {
    if (t0 < n) {
      double x[2][3];
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int u = 0; u < 3; ++u) x[d][u] = t0 + d < n ? v[t0 + d][g0 + u] : 0.0;
#pragma unroll
      for (int d = 0; d < 2; ++d)
        if (t0 + d < n)
#pragma unroll
          for (int u = 0; u < 3; ++u) acc[u] = fma(c[t0 + d], x[d][u], acc[u]);
    }
  }
}

template <int N, bool EQ3>
__global__ void __launch_bounds__(128) k_apply_rhs_df(DevView v, const double* Q, const double* H,
                                                      double* S, StageFuse fz) {
  constexpr int P = N + 1;      // lanes per element
  constexpr int EPR = 32 / P;   // elements per round
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t gw = (int64_t)blockIdx.x * 4 + warp;
  const int64_t tile = v.tile_begin + gw / kTile;
  if (tile >= (int64_t)v.tile_begin + v.tile_count) return;  // warp-uniform
  const TileDesc t = v.tiles[tile];
  const int cl = (int)(gw % kTile);
  if (cl >= t.count) return;  // warp-uniform
  const Col c = make_col(v, t, cl, N);
  const Phys ph = v.ph;
  const int el = lane / P, k = lane % P;
  const bool lane_ok = el < EPR;
  // this lane's row of w_k Dhat_kj and its scale factors
  df wd[P];
#pragma unroll
  for (int jj = 0; jj < P; ++jj) wd[jj] = df_of(c_tab.wD2[N][(lane_ok ? k : 0) * P + jj]);
  const df cs = df_from_double(c.s);
  const df iw0 = df_of(c_tab.iw2[N][0]);
  const df sc_k = df_mul(cs, df_of(c_tab.iw2[N][lane_ok ? k : 0]));   // interior
  const df sc_sh = df_mul(cs, df{0.5f * iw0.hi, 0.5f * iw0.lo});      // shared point
  const df sc_end = df_mul(cs, iw0);                                  // bottom, top
  const df gd = df_from_double(ph.g);
  const double* ref = v.ref + c.off;
  const double* ith = v.ithb + c.off / 3;
  const double* hc = H + c.off;
  bool ok = true;
  df carry[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  for (int e0 = 0; e0 < c.nez; e0 += EPR) {
    const int e = e0 + el;
    const bool act = lane_ok && e < c.nez;
    const int I = e * N + k;
    df f[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    double rho = 0.0, dTh = 0.0, ithb = 0.0, Pb = 0.0, rb = 0.0;
    double q[3] = {0.0, 0.0, 0.0};   // Q_i at point I
    double rp[3] = {0.0, 0.0, 0.0};  // memory part of the next right-hand side at point I
    if (act) {
      const int64_t g0 = c.off + 3 * I;
      if (fz.qtt) {  // Q_i = qtt + sum_t cq[t] q[t]
#pragma unroll
        for (int u = 0; u < 3; ++u) q[u] = fz.qtt[g0 + u];
        fuse_chain<kFuseQ>(fz.nq, fz.q, fz.cq, g0, q);
      } else {
#pragma unroll
        for (int u = 0; u < 3; ++u) q[u] = Q[g0 + u];
      }
      if (fz.rout && (k < N || e == c.nez - 1)) {
        // the memory terms of the right-hand side at the point this lane
        // writes (the chain's first part: rbase, then the r[t] in order)
#pragma unroll
        for (int u = 0; u < 3; ++u) rp[u] = fz.rbase[g0 + u];
        fuse_chain<kFuseR>(fz.nr, fz.r, fz.cr, g0, rp);
      }
      rho = q[0];
      const double m = q[1], Th = q[2];
      rb = ref[3 * I];
      Pb = ref[3 * I + 1];
      dTh = Th - ref[3 * I + 2];
      ithb = ith[I];
      const df r = df_from_double(rho), md = df_from_double(m), T = df_from_double(Th);
      if (!(r.hi > 0.0f) || !(T.hi > 0.0f)) ok = false;
      const float r0 = __frcp_rn(r.hi);
      const df ee = df_sub(df{1.0f, 0.0f}, df_mul(r, df{r0, 0.0f}));
      const df ir = df_add_f(df_mul(df{r0, 0.0f}, ee), r0);
      const df w = df_mul(md, ir);
      f[0] = md;
      if (EQ3) {
        // set 3C: P - P_bar = (gamma - 1)((E - E_bar) - m w / 2 - (rho - rho_bar) g z),
        // fluxes (m, m w + P - P_bar, (E + P) w)
        const double z = point_z<N>(1.0 / (0.5 * c.s), I, c.nz);
        const df gm = df_from_double(ph.gamma - 1.0);
        const df mw2 = df_mul(md, w);
        const df dP = df_mul(gm, df_sub(df_sub(df_from_double(dTh), df{0.5f * mw2.hi, 0.5f * mw2.lo}),
                                        df_from_double((rho - rb) * ph.g * z)));
        if (!((float)Pb + dP.hi > 0.0f)) ok = false;
        f[1] = df_add(mw2, dP);
        f[2] = df_mul(df_add(df_from_double(Th + Pb), dP), w);
      } else {
        f[1] = df_add(df_mul(md, w), eos_perturbation_df(ph, dTh, ithb, Pb));
        f[2] = df_mul(T, w);
      }
    }
    // this lane's row of the element derivative from its element's fluxes
    const int base = (lane_ok ? el : 0) * P;
    df R[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
    for (int jj = 0; jj < P; ++jj) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const df fj = {__shfl_sync(0xffffffffu, f[u].hi, base + jj),
                       __shfl_sync(0xffffffffu, f[u].lo, base + jj)};
        R[u] = jj == 0 ? df_mul(wd[0], fj) : df_fma(wd[jj], fj, R[u]);
      }
    }
    // row N of the element before: from the lane before, or carried
    df left[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      left[u] = {__shfl_up_sync(0xffffffffu, R[u].hi, 1), __shfl_up_sync(0xffffffffu, R[u].lo, 1)};
      if (el == 0) left[u] = carry[u];
    }
    {  // the last row of this round goes to the next round's first point
      const int src = (EPR - 1) * P + N;
#pragma unroll
      for (int u = 0; u < 3; ++u)
        carry[u] = {__shfl_sync(0xffffffffu, R[u].hi, src), __shfl_sync(0xffffffffu, R[u].lo, src)};
    }
    const bool top = k == N && e == c.nez - 1;
    if (act && (k < N || top)) {
      df D[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if (k == 0 && e == 0)
          D[u] = df_mul(R[u], sc_end);  // bottom
        else if (k == 0)
          D[u] = df_mul(df_add(R[u], left[u]), sc_sh);  // shared point
        else if (top)
          D[u] = df_mul(R[u], sc_end);
        else
          D[u] = df_mul(R[u], sc_k);
      }
      const int nzl = c.nz - 1;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = 3 * I + u;
        df val;
        if (u == 1 && (I == 0 || I == nzl)) {
          val = df_from_double(hc[i]);
        } else {
          val = df_sub(df_from_double(hc[i]), D[u]);
          if (u == 1) val = df_sub(val, df_mul(gd, df_from_double(rho - rb)));
        }
        const double sv = df_to_double(val);
        const int64_t gi = c.off + i;
        if (S) S[gi] = sv;
        if (fz.qout) fz.qout[gi] = q[u];
        if (fz.rout) {
          double rs = rp[u];
          if (fz.has_s) rs = fma(fz.cs, sv, rs);
          if (fz.has_q) rs = fma(fz.cqs, q[u], rs);
          fz.rout[gi] = rs;
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, !ok) && lane == 0) fail(v, c.col, HEVI_COL_BAD_INPUT);
}

template <int N>
void launch_apply_df_n(bool eq3, unsigned grid, cudaStream_t st, const DevView& v, const double* Q,
                       const double* H, double* S, const StageFuse& fz) {
  if (eq3)
    k_apply_rhs_df<N, true><<<grid, 128, 0, st>>>(v, Q, H, S, fz);
  else
    k_apply_rhs_df<N, false><<<grid, 128, 0, st>>>(v, Q, H, S, fz);
}

void launch_apply_rhs_df(const DevView& v, int order, const double* Q, const double* H, double* S,
                         cudaStream_t st, const StageFuse* fzp) {
  const StageFuse fz = fzp ? *fzp : StageFuse{};
  const unsigned grid = (unsigned)(v.tile_count * (kTile / 4));  // a warp per column slot
  const bool e3 = v.ph.eqset == 1;
  switch (order) {
    case 1: launch_apply_df_n<1>(e3, grid, st, v, Q, H, S, fz); break;
    case 2: launch_apply_df_n<2>(e3, grid, st, v, Q, H, S, fz); break;
    case 3: launch_apply_df_n<3>(e3, grid, st, v, Q, H, S, fz); break;
    case 4: launch_apply_df_n<4>(e3, grid, st, v, Q, H, S, fz); break;
    case 5: launch_apply_df_n<5>(e3, grid, st, v, Q, H, S, fz); break;
    default: break;
  }
}

}  // namespace hevi
