/*
 * hevi_oracle.c -- plain, slow, FP64 CPU oracle for the vertically implicit
 * column solve of Giraldo, Alves, Kelly, Kang & Reinecke, "A Performance Study
 * of Horizontally Explicit Vertically Implicit (HEVI) Time-Integrators for
 * Non-Hydrostatic Atmospheric Models" (arXiv:2311.11425).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header,
 * table or constant with the CUDA library; everything here is written out
 * from the definitions in the paper, one step at a time, with no blocking,
 * fusion or reordering beyond what those definitions state.
 *
 * Conventions (one column; n_z = Nez*N + 1 CG points, n = 3*n_z unknowns):
 *   unknown index = 3*I + v, I = global point, v = 0 (rho), 1 (m = rho*w),
 *   2 (Theta = rho*theta)   -- set 2C restricted to the vertical (App. A.1).
 *   Band half-widths k_l = k_u = n_var(N+1) - 1 (Sec. 4.2.3, "Lapack Banded
 *   Matrix Routines"); band storage is LAPACK's, column-major, with
 *   ldab >= 2 k_l + k_u + 1 and AB[k_l + k_u + i - j, j] = A[i, j].
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *   R1  flat column, uniform elements dz = z_top / Nez, zeta parallel to z;
 *   R2  the hydrostatic reference (rho_bar, Theta_bar) is isothermal and
 *       P_bar := EOS(Theta_bar) is subtracted inside the vertical pressure
 *       flux together with g*rho_bar in the gravity term, so the rest state
 *       is an exact discrete equilibrium;
 *   R3  w = 0 at the bottom and top point: the m-rows there are identity rows
 *       of the Jacobian and V_m := 0 there;
 *   R4  the gravity entry of the Jacobian (App. A.3, matrix P) couples the
 *       m-row to the rho-column at the same point (it is printed as a
 *       diagonal entry);
 *   R5  the Theta-row, rho-column entry of K_2C is -theta*w (the printed
 *       entry lacks a factor Theta);
 *   R6  pivot tie-break: the first row of maximal |a| (LAPACK semantics);
 *   R7  Newton: initial guess supplied by the caller, stop when
 *       ||S^-1 F(q_m)||_2 <= rtol ||S^-1 F(q_0)||_2 with S the reference
 *       scales (rho_bar, rho_bar*c_s, Theta_bar), or when
 *       ||S^-1 F(q_m)||_2 <= 512 eps ||S^-1 q_m||_2 (eps = 2^-52): the
 *       residual is then at the rounding level of its own FP64 evaluation and
 *       the relative test cannot be met when ||F(q_0)|| is itself within
 *       1/rtol of that level (a column already near its stage solution).
 *       Both tests are applied to q_0 as well (m = 0 updates).
 *   R14 NHEVI-GMRES: the Frechet perturbation E of Eq. Frechet-derivative is
 *       diagonal, eps S with the reference scales S (per-variable magnitudes),
 *       applied to the equilibrated system; GMRES starts at zero and is not
 *       restarted (restarted GMRES(30..60) stagnates on these columns).
 *   R16 set 3C (App. A.1, Eq. set3c; Jacobian Eq. set3c_jacobian) in a flat
 *       column without horizontal momentum, unknowns (rho, m = rho w, E): the
 *       horizontal momenta are only advected by the vertical operator, so zero
 *       horizontal momentum is an invariant subspace and the coupled system
 *       keeps three unknowns per point.  Phi = g z; the reference energy is
 *       E_bar = P_bar / (gamma - 1) + rho_bar g z (P_bar as in R2), the
 *       pressure flux carries P - P_bar with P = (gamma - 1)(E - m^2/(2 rho) -
 *       rho g z); the flux Jacobian is that of the fluxes (m, m^2/rho + P,
 *       (E + P) m / rho), whose printed momentum-row energy entry carries a
 *       stray 1/rho.  Scales for the Newton norm: (rho_bar, rho_bar c_s,
 *       E_bar); the band LU solves the system equilibrated with the same
 *       scales (E and rho differ by five orders of magnitude).  Selected by
 *       or_set_equation_set(1); 0 (default) is set 2C.
 *   R17 set 2NC (Sec. 2.1, Eq. set2nc) in the same column, unknowns (rho, w,
 *       theta): zero horizontal velocity is invariant under the vertical
 *       operator.  V follows Eq. (hevi/vertical_operators) with the reference
 *       subtracted as in R2,
 *         V_rho = -Dcal[rho w],
 *         V_w   = -(w Dcal[w] + (Dcal[P - P_bar] + g (rho - rho_bar)) / rho),
 *         V_th  = -w Dcal[theta],
 *       P = EOS(rho theta), V_w = 0 at both ends (R3).  With w = 0 at both
 *       ends the weak-form continuity derivative of Sec. 4.2.3 equals the
 *       strong form after DSS (the element boundary terms cancel in pairs and
 *       vanish at the ends), so Dcal serves all three equations.  L is the
 *       Frechet derivative of this V (the printed K_2NC is not: its advection
 *       and pressure entries put the point-j factor where the derivative has
 *       the point-i one); the band is A = I - Lambda L assembled column by
 *       column from L applied to unit vectors.  Scales (rho_bar, c_s,
 *       theta_bar).  Selected by or_set_equation_set(2).
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* reading R7: rounding floor of the Newton stop */
#define OR_NEWTON_FLOOR (512.0 * DBL_EPSILON)

/* physical constants of the isothermal reference atmosphere */
#define OR_T0 300.0
#define OR_P0 1.0e5
#define OR_R 287.17
#define OR_CP 1004.67
#define OR_G 9.80616

static double or_cv(void) { return OR_CP - OR_R; }
static double or_gamma(void) { return OR_CP / or_cv(); }

/* ------------------------------------------------------------------ */
/* Sec. 3, Eq. (space/basis): Legendre-Gauss-Lobatto points of order N  */
/* are the end points +-1 and the roots of P_N'; the co-located weights */
/* are w_k = 2 / (N (N+1) P_N(xi_k)^2).                                 */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_N and its first two derivatives by the three-term
 * recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}. */
static void legendre(int N, double x, double* p, double* dp, double* ddp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, dd0 = 0.0, dd1 = 0.0;
  if (N == 0) { *p = 1.0; *dp = 0.0; *ddp = 0.0; return; }
  for (int n = 1; n < N; ++n) {
    double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
    double d2 = d0 + (2.0 * n + 1.0) * p1;   /* P'_{n+1} = P'_{n-1} + (2n+1) P_n */
    double dd2 = dd0 + (2.0 * n + 1.0) * d1; /* differentiate the line above */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; dd0 = dd1; dd1 = dd2;
  }
  *p = p1; *dp = d1; *ddp = dd1;
}

int or_lgl(int N, double* xi, double* w) {
  if (N < 1 || N > 32) return 1;
  xi[0] = -1.0;
  xi[N] = 1.0;
  for (int k = 1; k < N; ++k) {
    /* Newton's method on P_N'(x) = 0 from the Chebyshev-Lobatto guess */
    double x = -cos(3.14159265358979323846 * k / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre(N, x, &p, &dp, &ddp);
      double dx = dp / ddp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    xi[k] = x;
  }
  for (int k = 0; k <= N; ++k) {
    double p, dp, ddp;
    legendre(N, xi[k], &p, &dp, &ddp);
    w[k] = 2.0 / (N * (N + 1.0) * p * p);
  }
  return 0;
}

/* Sec. 3: derivative of the cardinal Lagrange basis, Dhat[k][j] = h_j'(xi_k),
 * written literally from h_j(x) = prod_{m != j} (x - xi_m) / (xi_j - xi_m).
 * (The paper indexes D_ij = h_i'(xi_j), the transpose of Dhat.) */
int or_dmatrix(int N, const double* xi, double* D) {
  for (int k = 0; k <= N; ++k) {
    for (int j = 0; j <= N; ++j) {
      double s = 0.0;
      for (int l = 0; l <= N; ++l) {
        if (l == j) continue;
        double t = 1.0 / (xi[j] - xi[l]);
        for (int m = 0; m <= N; ++m) {
          if (m == j || m == l) continue;
          t *= (xi[k] - xi[m]) / (xi[j] - xi[m]);
        }
        s += t;
      }
      D[k * (N + 1) + j] = s;
    }
  }
  return 0;
}

/* Sec. 3: column grid.  Element e covers [e dz, (e+1) dz] (reading R1); the
 * local node k of element e is the global point I = e N + k; the diagonal
 * mass is M_I = DSS of w_k J_e with J_e = dz / 2. */
int or_column_grid(int nez, int N, double ztop, double* z, double* M) {
  double xi[33], w[33];
  if (nez < 1 || or_lgl(N, xi, w)) return 1;
  int nz = nez * N + 1;
  double dz = ztop / nez;
  for (int I = 0; I < nz; ++I) M[I] = 0.0;
  for (int e = 0; e < nez; ++e) {
    for (int k = 0; k <= N; ++k) {
      int I = e * N + k;
      z[I] = e * dz + (xi[k] + 1.0) * 0.5 * dz;
      M[I] += w[k] * 0.5 * dz;
    }
  }
  z[0] = 0.0;
  z[nz - 1] = ztop;
  return 0;
}

/* The equation set of every call: 0 = set 2C (unknowns rho, m, Theta),
 * 1 = set 3C (rho, m, E; reading R16), 2 = set 2NC (rho, w, theta; R17). */
static int or_set = 0;
int or_set_equation_set(int s) {
  if (s != 0 && s != 1 && s != 2) return 1;
  or_set = s;
  return 0;
}

/* App. A.1, Eq. (set2c_pressure): P = P_A (R Theta / P_A)^gamma. */
static double eos(double Theta) { return OR_P0 * pow(OR_R * Theta / OR_P0, or_gamma()); }

/* Reading R2: isothermal hydrostatic reference state at height z. */
void or_reference_state(int nz, const double* z, double* rho, double* theta, double* Theta,
                        double* P) {
  double H = OR_R * OR_T0 / OR_G;
  for (int I = 0; I < nz; ++I) {
    double r = OR_P0 / (OR_R * OR_T0) * exp(-z[I] / H);
    double th = OR_T0 * exp(OR_G * z[I] / (OR_CP * OR_T0));
    rho[I] = r;
    theta[I] = th;
    Theta[I] = r * th;
    P[I] = eos(r * th);
  }
}

/* Scales used for the Newton norm (reading R7): rho_bar, rho_bar * c_s and
 * Theta_bar at each point, with c_s = sqrt(gamma R T0); set 3C: E_bar for the
 * third; set 2NC: c_s and theta_bar for the second and third. */
void or_scales(int nz, const double* z, double* s) {
  double* rho = (double*)malloc(sizeof(double) * 4 * nz);
  double *th = rho + nz, *Th = th + nz, *P = Th + nz;
  or_reference_state(nz, z, rho, th, Th, P);
  double cs = sqrt(or_gamma() * OR_R * OR_T0);
  for (int I = 0; I < nz; ++I) {
    s[3 * I + 0] = rho[I];
    s[3 * I + 1] = or_set == 2 ? cs : rho[I] * cs;
    s[3 * I + 2] = or_set == 1   ? P[I] / (or_gamma() - 1.0) + rho[I] * OR_G * z[I]
                   : or_set == 2 ? th[I]
                                 : Th[I];
  }
  free(rho);
}

/* ------------------------------------------------------------------ */
/* Column geometry bundle (recomputed per call: the oracle is slow on   */
/* purpose and keeps no state).                                         */
/* ------------------------------------------------------------------ */
typedef struct {
  int nez, N, nz, n;
  double xi[33], w[33];
  double* D;   /* (N+1)^2 */
  double* z;   /* nz */
  double* M;   /* nz */
  double *rho_b, *theta_b, *Theta_b, *P_b;
  double* E_b;  /* set 3C reference energy P_bar / (gamma - 1) + rho_bar g z */
  double* X_b;  /* reference value of the third unknown: Theta_b (2C), E_b (3C), theta_b (2NC) */
} column_t;

static int column_init(column_t* c, int nez, int N, double ztop) {
  c->nez = nez; c->N = N; c->nz = nez * N + 1; c->n = 3 * c->nz;
  if (or_lgl(N, c->xi, c->w)) return 1;
  c->D = (double*)malloc(sizeof(double) * ((N + 1) * (N + 1) + 7 * c->nz));
  c->z = c->D + (N + 1) * (N + 1);
  c->M = c->z + c->nz;
  c->rho_b = c->M + c->nz;
  c->theta_b = c->rho_b + c->nz;
  c->Theta_b = c->theta_b + c->nz;
  c->P_b = c->Theta_b + c->nz;
  or_dmatrix(N, c->xi, c->D);
  or_column_grid(nez, N, ztop, c->z, c->M);
  or_reference_state(c->nz, c->z, c->rho_b, c->theta_b, c->Theta_b, c->P_b);
  c->E_b = c->P_b + c->nz;
  for (int I = 0; I < c->nz; ++I)
    c->E_b[I] = c->P_b[I] / (or_gamma() - 1.0) + c->rho_b[I] * OR_G * c->z[I];
  c->X_b = or_set == 1 ? c->E_b : (or_set == 2 ? c->theta_b : c->Theta_b);
  return 0;
}
static void column_free(column_t* c) { free(c->D); }

/* (Dcal f)_I = (1/M_I) DSS_e [ w_k J_e (dxi/dz) sum_j Dhat_kj f_(e,j) ]
 *            = (1/M_I) sum_{(e,k) -> I} w_k sum_j Dhat_kj f_(e,j)
 * Sec. 3 (strong-form derivative on each element, diagonal mass, DSS);
 * with J_e = dz/2 and dxi/dz = 2/dz the metric factors cancel. */
static void dss_derivative(const column_t* c, const double* f, double* out) {
  int N = c->N;
  for (int I = 0; I < c->nz; ++I) out[I] = 0.0;
  for (int e = 0; e < c->nez; ++e) {
    for (int k = 0; k <= N; ++k) {
      double s = 0.0;
      for (int j = 0; j <= N; ++j) s += c->D[k * (N + 1) + j] * f[e * N + j];
      out[e * N + k] += c->w[k] * s;
    }
  }
  for (int I = 0; I < c->nz; ++I) out[I] /= c->M[I];
}

/* App. A.2 (vertical operator V of set 2C restricted to the vertical):
 *   V_rho   = -Dcal[m]
 *   V_m     = -Dcal[m^2/rho + P(Theta) - P_bar] - g (rho - rho_bar)
 *   V_Theta = -Dcal[Theta m / rho]
 * with readings R2 (reference subtraction) and R3 (V_m = 0 at both ends). */
static void apply_V_2nc(const column_t* c, const double* q, double* v);
static void apply_V(const column_t* c, const double* q, double* v) {
  if (or_set == 2) {
    apply_V_2nc(c, q, v);
    return;
  }
  int nz = c->nz;
  double* f = (double*)malloc(sizeof(double) * 6 * nz);
  double *fr = f, *fm = f + nz, *ft = f + 2 * nz, *dr = f + 3 * nz, *dm = f + 4 * nz,
         *dt = f + 5 * nz;
  for (int I = 0; I < nz; ++I) {
    double rho = q[3 * I], m = q[3 * I + 1], Th = q[3 * I + 2];
    fr[I] = m;
    if (or_set == 1) {
      /* set 3C (R16): Th holds E; P - P_bar from the differences to the reference */
      double E = Th;
      double dP = (or_gamma() - 1.0) *
                  ((E - c->E_b[I]) - m * m / (2.0 * rho) - (rho - c->rho_b[I]) * OR_G * c->z[I]);
      fm[I] = m * m / rho + dP;
      ft[I] = (E + c->P_b[I] + dP) * m / rho;
    } else {
      fm[I] = m * m / rho + (eos(Th) - c->P_b[I]);
      ft[I] = Th * m / rho;
    }
  }
  dss_derivative(c, fr, dr);
  dss_derivative(c, fm, dm);
  dss_derivative(c, ft, dt);
  for (int I = 0; I < nz; ++I) {
    v[3 * I + 0] = -dr[I];
    v[3 * I + 1] = -dm[I] - OR_G * (q[3 * I] - c->rho_b[I]);
    v[3 * I + 2] = -dt[I];
  }
  v[1] = 0.0;
  v[3 * (nz - 1) + 1] = 0.0;
  free(f);
}

/* Set 2NC (reading R17), unknowns (rho, w, theta):
 *   V_rho = -Dcal[rho w]
 *   V_w   = -( w Dcal[w] + (Dcal[P - P_bar] + g (rho - rho_bar)) / rho ),  P = EOS(rho theta)
 *   V_th  = -w Dcal[theta]
 * and V_w = 0 at both ends (R3). */
static void apply_V_2nc(const column_t* c, const double* q, double* v) {
  int nz = c->nz;
  double* f = (double*)malloc(sizeof(double) * 8 * nz);
  double *fr = f, *fw = f + nz, *fp = f + 2 * nz, *ft = f + 3 * nz;
  double *dr = f + 4 * nz, *dw = f + 5 * nz, *dp = f + 6 * nz, *dt = f + 7 * nz;
  for (int I = 0; I < nz; ++I) {
    double rho = q[3 * I], w = q[3 * I + 1], th = q[3 * I + 2];
    fr[I] = rho * w;
    fw[I] = w;
    fp[I] = eos(rho * th) - c->P_b[I];
    ft[I] = th;
  }
  dss_derivative(c, fr, dr);
  dss_derivative(c, fw, dw);
  dss_derivative(c, fp, dp);
  dss_derivative(c, ft, dt);
  for (int I = 0; I < nz; ++I) {
    double rho = q[3 * I], w = q[3 * I + 1];
    v[3 * I + 0] = -dr[I];
    v[3 * I + 1] = -(w * dw[I] + (dp[I] + OR_G * (rho - c->rho_b[I])) / rho);
    v[3 * I + 2] = -w * dt[I];
  }
  v[1] = 0.0;
  v[3 * (nz - 1) + 1] = 0.0;
  free(f);
}

/* Set 2NC (reading R17): L = dV/dq at q0 = (rho0, w0, theta0) applied to
 * x = (r, u, t), with P0 = EOS(rho0 theta0), P_rho = gamma P0 / rho0,
 * P_theta = gamma P0 / theta0 and X0 = Dcal[P0 - P_bar] + g (rho0 - rho_bar):
 *   L_rho = -Dcal[w0 r + rho0 u]
 *   L_w   = -( u Dcal[w0] + w0 Dcal[u] - r X0 / rho0^2
 *              + (Dcal[P_rho r + P_theta t] + g r) / rho0 )
 *   L_th  = -( u Dcal[theta0] + w0 Dcal[t] )
 * and L_w = 0 at both ends (R3). */
static void apply_L_2nc(const column_t* c, const double* q0, const double* x, double* y) {
  int nz = c->nz;
  double* f = (double*)malloc(sizeof(double) * 14 * nz);
  double *fr = f, *fu = f + nz, *fp = f + 2 * nz, *ft = f + 3 * nz;
  double *gw = f + 4 * nz, *gp = f + 5 * nz, *gt = f + 6 * nz;
  double *dr = f + 7 * nz, *du = f + 8 * nz, *dp = f + 9 * nz, *dt = f + 10 * nz;
  double *Dw0 = f + 11 * nz, *Dp0 = f + 12 * nz, *Dt0 = f + 13 * nz;
  for (int I = 0; I < nz; ++I) {
    double r0 = q0[3 * I], w0 = q0[3 * I + 1], t0 = q0[3 * I + 2];
    double P0 = eos(r0 * t0);
    double r = x[3 * I], u = x[3 * I + 1], t = x[3 * I + 2];
    fr[I] = w0 * r + r0 * u;
    fu[I] = u;
    fp[I] = or_gamma() * P0 / r0 * r + or_gamma() * P0 / t0 * t;
    ft[I] = t;
    gw[I] = w0;
    gp[I] = P0 - c->P_b[I];
    gt[I] = t0;
  }
  dss_derivative(c, fr, dr);
  dss_derivative(c, fu, du);
  dss_derivative(c, fp, dp);
  dss_derivative(c, ft, dt);
  dss_derivative(c, gw, Dw0);
  dss_derivative(c, gp, Dp0);
  dss_derivative(c, gt, Dt0);
  for (int I = 0; I < nz; ++I) {
    double r0 = q0[3 * I], w0 = q0[3 * I + 1];
    double r = x[3 * I], u = x[3 * I + 1];
    double X0 = Dp0[I] + OR_G * (r0 - c->rho_b[I]);
    y[3 * I + 0] = -dr[I];
    y[3 * I + 1] = -(u * Dw0[I] + w0 * du[I] - r * X0 / (r0 * r0) + (dp[I] + OR_G * r) / r0);
    y[3 * I + 2] = -(u * Dt0[I] + w0 * dt[I]);
  }
  y[1] = 0.0;
  y[3 * (nz - 1) + 1] = 0.0;
  free(f);
}

/* App. A.3, Eq. (set2c_jacobian) restricted to the vertical (zeta_x = zeta_y
 * = 0, zeta_z = 1 after the metric cancellation above): the 3x3 flux
 * Jacobian at a point, rows = flux of (rho, m, Theta), columns = d/d(rho, m,
 * Theta).  With w = m/rho, theta = Theta/rho, P' = gamma P / Theta:
 *   rho-flux   : ( 0,        1,      0  )
 *   m-flux     : ( -w^2,     2w,     P' )
 *   Theta-flux : ( -theta w, theta,  w  )       (reading R5) */
static void flux_jacobian(const double* q, double z, double K[3][3]) {
  double rho = q[0], m = q[1], Th = q[2];
  if (or_set == 1) {
    /* set 3C (R16): fluxes (m, m^2/rho + P, (E + P) m / rho), P = (gamma - 1)
     * (E - m^2/(2 rho) - rho g z): with w = m/rho, h = (E + P)/rho,
     *   dP/drho = (gamma - 1)(w^2/2 - g z), dP/dm = -(gamma - 1) w, dP/dE = gamma - 1 */
    double gm = or_gamma() - 1.0, E = Th, w = m / rho;
    double P = gm * (E - m * w / 2.0 - rho * OR_G * z), h = (E + P) / rho;
    double Pr = gm * (w * w / 2.0 - OR_G * z), Pm = -gm * w, PE = gm;
    K[0][0] = 0.0;               K[0][1] = 1.0;         K[0][2] = 0.0;
    K[1][0] = -w * w + Pr;       K[1][1] = 2 * w + Pm;  K[1][2] = PE;
    K[2][0] = w * Pr - h * w;    K[2][1] = h + w * Pm;  K[2][2] = w * (1.0 + PE);
    return;
  }
  double w = m / rho, th = Th / rho, dP = or_gamma() * eos(Th) / Th;
  K[0][0] = 0.0;     K[0][1] = 1.0; K[0][2] = 0.0;
  K[1][0] = -w * w;  K[1][1] = 2 * w; K[1][2] = dP;
  K[2][0] = -th * w; K[2][1] = th;  K[2][2] = w;
}

/* Sec. 4.3.1: L = dV/dq at q0 (LHEVI-PS linearisation), applied to x:
 *   (L x) = -Dcal[K(q0) x] - G x,   G[m, rho] = g   (reading R4),
 * and (L x)_m = 0 at both ends (reading R3). */
static void apply_L(const column_t* c, const double* q0, const double* x, double* y) {
  if (or_set == 2) {
    apply_L_2nc(c, q0, x, y);
    return;
  }
  int nz = c->nz;
  double* f = (double*)malloc(sizeof(double) * 6 * nz);
  double *fr = f, *fm = f + nz, *ft = f + 2 * nz, *dr = f + 3 * nz, *dm = f + 4 * nz,
         *dt = f + 5 * nz;
  for (int I = 0; I < nz; ++I) {
    double K[3][3];
    flux_jacobian(q0 + 3 * I, c->z[I], K);
    const double* xi = x + 3 * I;
    fr[I] = K[0][0] * xi[0] + K[0][1] * xi[1] + K[0][2] * xi[2];
    fm[I] = K[1][0] * xi[0] + K[1][1] * xi[1] + K[1][2] * xi[2];
    ft[I] = K[2][0] * xi[0] + K[2][1] * xi[1] + K[2][2] * xi[2];
  }
  dss_derivative(c, fr, dr);
  dss_derivative(c, fm, dm);
  dss_derivative(c, ft, dt);
  for (int I = 0; I < nz; ++I) {
    y[3 * I + 0] = -dr[I];
    y[3 * I + 1] = -dm[I] - OR_G * x[3 * I];
    y[3 * I + 2] = -dt[I];
  }
  y[1] = 0.0;
  y[3 * (nz - 1) + 1] = 0.0;
  free(f);
}

/* Sec. 4.2.3 and App. A.3: A = I - Lambda L(q0) = I + Lambda Dcal K(q0) +
 * Lambda G, assembled entry by entry into LAPACK band storage:
 *   A[(I,v),(J,u)] = delta + Lambda/M_I sum_{e containing I and J}
 *                    w_{k(I)} Dhat_{k(I), j(J)} K_vu(q0_J) + Lambda g [v=m,u=rho,I=J]
 * The m-rows of the two end points are identity rows (reading R3). */
static void assemble_band(const column_t* c, double lam, const double* q0, double* ab, int ldab) {
  int N = c->N, n = c->n, kl = 3 * (N + 1) - 1, ku = kl;
  memset(ab, 0, sizeof(double) * (size_t)ldab * n);
#define AB(i, j) ab[(size_t)(j) * ldab + (kl + ku + (i) - (j))]
  if (or_set == 2) {
    /* set 2NC (R17): column j of A = I - Lambda L is e_j - Lambda L e_j; L
     * couples the points of one element only, so the column lies in the band */
    double* e = (double*)calloc((size_t)n, sizeof(double));
    double* y = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < n; ++j) {
      e[j] = 1.0;
      apply_L(c, q0, e, y);
      e[j] = 0.0;
      int i0 = j - ku < 0 ? 0 : j - ku, i1 = j + kl > n - 1 ? n - 1 : j + kl;
      for (int i = i0; i <= i1; ++i) AB(i, j) = (i == j ? 1.0 : 0.0) - lam * y[i];
    }
    free(e);
    free(y);
    return;
  }
  for (int e = 0; e < c->nez; ++e) {
    for (int k = 0; k <= N; ++k) {
      int I = e * N + k;
      for (int j = 0; j <= N; ++j) {
        int J = e * N + j;
        double K[3][3];
        flux_jacobian(q0 + 3 * J, c->z[J], K);
        double coef = lam * c->w[k] * c->D[k * (N + 1) + j] / c->M[I];
        for (int v = 0; v < 3; ++v)
          for (int u = 0; u < 3; ++u) AB(3 * I + v, 3 * J + u) += coef * K[v][u];
      }
    }
  }
  for (int I = 0; I < c->nz; ++I) {
    for (int v = 0; v < 3; ++v) AB(3 * I + v, 3 * I + v) += 1.0;
    AB(3 * I + 1, 3 * I + 0) += lam * OR_G;
  }
  int ends[2] = {0, c->nz - 1};
  for (int t = 0; t < 2; ++t) {
    int row = 3 * ends[t] + 1;
    for (int col = row - kl; col <= row + ku; ++col)
      if (col >= 0 && col < n) AB(row, col) = (col == row) ? 1.0 : 0.0;
  }
#undef AB
}

/* ------------------------------------------------------------------ */
/* Sec. 4.2.3: LAPACK band LU with partial pivoting (dgbtrf semantics,  */
/* unblocked) and the matching solve (dgbtrs, no transpose).            */
/* ------------------------------------------------------------------ */
int or_gbtrf(int n, int kl, int ku, double* ab, int ldab, int* ipiv) {
  int kv = ku + kl, info = 0;
#define AB(i, j) ab[(size_t)(j) * ldab + (kv + (i) - (j))]
  for (int j = 0; j < n; ++j) {
    int last = j + kl < n - 1 ? j + kl : n - 1;
    /* pivot: first row of maximal |a| in column j (reading R6) */
    int p = j;
    double amax = fabs(AB(j, j));
    for (int i = j + 1; i <= last; ++i)
      if (fabs(AB(i, j)) > amax) { amax = fabs(AB(i, j)); p = i; }
    ipiv[j] = p;
    int cend = j + kv < n - 1 ? j + kv : n - 1;  /* U row j reaches column j+kl+ku */
    if (AB(p, j) == 0.0) {
      if (info == 0) info = j + 1;
      continue;
    }
    if (p != j)
      for (int col = j; col <= cend; ++col) {
        double t = AB(j, col); AB(j, col) = AB(p, col); AB(p, col) = t;
      }
    for (int i = j + 1; i <= last; ++i) AB(i, j) /= AB(j, j);
    for (int col = j + 1; col <= cend; ++col)
      for (int i = j + 1; i <= last; ++i) AB(i, col) -= AB(i, j) * AB(j, col);
  }
#undef AB
  return info;
}

void or_gbtrs(int n, int kl, int ku, const double* ab, int ldab, const int* ipiv, double* b) {
  int kv = ku + kl;
#define AB(i, j) ab[(size_t)(j) * ldab + (kv + (i) - (j))]
  /* forward: interchanges and unit-lower multipliers, in factorisation order */
  for (int j = 0; j < n; ++j) {
    int p = ipiv[j];
    if (p != j) { double t = b[j]; b[j] = b[p]; b[p] = t; }
    int last = j + kl < n - 1 ? j + kl : n - 1;
    for (int i = j + 1; i <= last; ++i) b[i] -= AB(i, j) * b[j];
  }
  /* backward: upper triangle with kl+ku super-diagonals */
  for (int j = n - 1; j >= 0; --j) {
    int cend = j + kv < n - 1 ? j + kv : n - 1;
    double s = b[j];
    for (int col = j + 1; col <= cend; ++col) s -= AB(j, col) * b[col];
    b[j] = s / AB(j, j);
  }
#undef AB
}

/* ------------------------------------------------------------------ */
/* Batched entry points over columns of one size class.  q, x, b, ... */
/* are [col][point][var] arrays with n = 3 (Nez N + 1) doubles/column;  */
/* ztop is per column.                                                  */
/* ------------------------------------------------------------------ */
int or_apply_V(int ncols, int nez, int N, const double* ztop, const double* q, double* v) {
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    apply_V(&col, q + (size_t)c * col.n, v + (size_t)c * col.n);
    column_free(&col);
  }
  return 0;
}

int or_apply_L(int ncols, int nez, int N, const double* ztop, const double* q0, const double* x,
               double* y) {
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    size_t o = (size_t)c * col.n;
    apply_L(&col, q0 + o, x + o, y + o);
    column_free(&col);
  }
  return 0;
}

/* A = I - Lambda L(q0) in band storage, ldab rows per column (ldab >= 2kl+ku+1). */
int or_assemble_band(int ncols, int nez, int N, const double* ztop, double lam, const double* q0,
                     double* ab, int ldab) {
  int n = 3 * (nez * N + 1), kl = 3 * (N + 1) - 1;
  if (ldab < 3 * kl + 1) return 1;
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    assemble_band(&col, lam, q0 + (size_t)c * n, ab + (size_t)c * ldab * n, ldab);
    column_free(&col);
  }
  return 0;
}

/* Reference state q_bar = (rho_bar, 0, Theta_bar) for each column (set 3C:
 * (rho_bar, 0, E_bar)). */
int or_reference_q(int ncols, int nez, int N, const double* ztop, double* q) {
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    double* qc = q + (size_t)c * col.n;
    for (int I = 0; I < col.nz; ++I) {
      qc[3 * I] = col.rho_b[I];
      qc[3 * I + 1] = 0.0;
      qc[3 * I + 2] = col.X_b[I];
    }
    column_free(&col);
  }
  return 0;
}

/* Column heights and masses for each column ([col][nz] arrays). */
int or_grid(int ncols, int nez, int N, const double* ztop, double* z, double* M) {
  int nz = nez * N + 1;
  for (int c = 0; c < ncols; ++c)
    if (or_column_grid(nez, N, ztop[c], z + (size_t)c * nz, M + (size_t)c * nz)) return 1;
  return 0;
}

/* The band LU of a column's stage matrix, and the solve with it.  Set 3C
 * (reading R16) is solved equilibrated, (S^-1 A S)(S^-1 x) = S^-1 b with the
 * reference scales S = (rho_bar, rho_bar c_s, E_bar): its unknowns differ by
 * five orders of magnitude and the unscaled band's condition number (~1e14)
 * would put the FP64 LU's error near 1e-10; set 2NC likewise with (rho_bar,
 * c_s, theta_bar); set 2C is factored as assembled. */
static double unknown_scale(const column_t* c, int i);
static int factor_band(const column_t* c, double lam, const double* q0, double* ab, int ldab,
                       int* ipiv) {
  int n = c->n, kl = 3 * (c->N + 1) - 1;
  assemble_band(c, lam, q0, ab, ldab);
  if (or_set) {
    for (int j = 0; j < n; ++j) {
      int i0 = j - kl < 0 ? 0 : j - kl, i1 = j + kl > n - 1 ? n - 1 : j + kl;
      for (int i = i0; i <= i1; ++i)
        ab[(size_t)j * ldab + (2 * kl + i - j)] *= unknown_scale(c, j) / unknown_scale(c, i);
    }
  }
  return or_gbtrf(n, kl, kl, ab, ldab, ipiv);
}
static void solve_band(const column_t* c, const double* ab, int ldab, const int* ipiv, double* x) {
  int n = c->n, kl = 3 * (c->N + 1) - 1;
  if (or_set)
    for (int i = 0; i < n; ++i) x[i] /= unknown_scale(c, i);
  or_gbtrs(n, kl, kl, ab, ldab, ipiv, x);
  if (or_set)
    for (int i = 0; i < n; ++i) x[i] *= unknown_scale(c, i);
}

/* Sec. 4.3, Eq. (lhevi-ark-final-2): solve (I - Lambda L(q0)) x = b for each
 * column with the band LU above.  info[c] is dgbtrf's info for column c. */
int or_stage_solve(int ncols, int nez, int N, const double* ztop, double lam, const double* q0,
                   const double* b, double* x, int* info) {
  int n = 3 * (nez * N + 1), kl = 3 * (N + 1) - 1, ldab = 3 * kl + 1;
  double* ab = (double*)malloc(sizeof(double) * (size_t)ldab * n);
  int* ipiv = (int*)malloc(sizeof(int) * n);
  int bad = 0;
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) { bad = 1; break; }
    size_t o = (size_t)c * n;
    info[c] = factor_band(&col, lam, q0 + o, ab, ldab, ipiv);
    memcpy(x + o, b + o, sizeof(double) * n);
    if (info[c] == 0) solve_band(&col, ab, ldab, ipiv, x + o);
    column_free(&col);
  }
  free(ab);
  free(ipiv);
  return bad;
}

/* Sec. 4.2.2, Eq. (nl_function): F(q) = q - Lambda V(q) - R. */
static void residual_F(const column_t* c, double lam, const double* q, const double* R, double* F) {
  apply_V(c, q, F);
  for (int i = 0; i < c->n; ++i) F[i] = q[i] - lam * F[i] - R[i];
}

static double scaled_norm(const column_t* c, const double* F) {
  double s2 = 0.0, cs = sqrt(or_gamma() * OR_R * OR_T0);
  for (int I = 0; I < c->nz; ++I) {
    double a = F[3 * I] / c->rho_b[I];
    double b = F[3 * I + 1] / (or_set == 2 ? cs : c->rho_b[I] * cs);
    double d = F[3 * I + 2] / c->X_b[I];
    s2 += a * a + b * b + d * d;
  }
  return sqrt(s2);
}

/* Reference scale of unknown i (rho_bar, rho_bar c_s, Theta_bar at point i/3;
 * set 3C: E_bar third; set 2NC: c_s second, theta_bar third). */
static double unknown_scale(const column_t* c, int i) {
  int I = i / 3, u = i - 3 * I;
  if (u == 0) return c->rho_b[I];
  if (u == 1) return (or_set == 2 ? 1.0 : c->rho_b[I]) * sqrt(or_gamma() * OR_R * OR_T0);
  return c->X_b[I];
}

/* Sec. 4.2.1 (NHEVI-GMRES): Jacobian-free Newton-Krylov.  Newton on
 * F(q) = q - Lambda V(q) - R; each Newton system J(q_m) dq = -F(q_m) is
 * solved by unpreconditioned GMRES (zero start, no restart: modified
 * Gram-Schmidt Arnoldi, Givens rotations) on the equilibrated system
 * J^ y = -S^-1 F(q_m), J^ = S^-1 J S, dq = S y, with the Frechet
 * difference (Eq. Frechet-derivative) J^ v ~ S^-1 [F(q_m + eps S v) - F(q_m)]
 * / eps, i.e. the diagonal perturbation E = eps S (reading R14: per-variable
 * magnitudes from the reference scales).  GMRES stops when its residual
 * estimate is <= gtol |S^-1 F(q_m)| or after kmax iterations; Newton stops
 * as in or_newton (reading R7).  iters[c] = Newton updates, kits[c] = Krylov
 * iterations in all, status 0 / 5 (Newton not converged) / 6 (non-physical
 * state met). */
int or_newton_gmres(int ncols, int nez, int N, const double* ztop, double lam, const double* R,
                    double* q, double eps, double rtol, double gtol, int max_newton, int kmax,
                    int* iters, int* kits, int* status) {
  int n = 3 * (nez * N + 1);
  double* F = (double*)malloc(sizeof(double) * n);
  double* qp = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* sc = (double*)malloc(sizeof(double) * n);
  double* Vb = (double*)malloc(sizeof(double) * (size_t)n * (kmax + 1));
  double* H = (double*)malloc(sizeof(double) * (size_t)(kmax + 1) * kmax);
  double* cs = (double*)malloc(sizeof(double) * kmax);
  double* sn = (double*)malloc(sizeof(double) * kmax);
  double* g = (double*)malloc(sizeof(double) * (kmax + 1));
  double* y = (double*)malloc(sizeof(double) * kmax);
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    size_t o = (size_t)c * n;
    double* qc = q + o;
    const double* Rc = R + o;
    for (int i = 0; i < n; ++i) sc[i] = unknown_scale(&col, i);
    residual_F(&col, lam, qc, Rc, F);
    double f0 = scaled_norm(&col, F);
    iters[c] = 0;
    kits[c] = 0;
    status[c] = 0;
    if (!(f0 > OR_NEWTON_FLOOR * scaled_norm(&col, qc))) {
      column_free(&col);
      continue;
    }
    status[c] = 5;
    for (int m = 1; m <= max_newton; ++m) {
      /* b = -S^-1 F, V_0 = b / beta */
      double beta = 0.0;
      for (int i = 0; i < n; ++i) {
        double bi = -F[i] / sc[i];
        Vb[i] = bi;
        beta += bi * bi;
      }
      beta = sqrt(beta);
      for (int i = 0; i < n; ++i) Vb[i] /= beta;
      for (int k = 0; k <= kmax; ++k) g[k] = 0.0;
      g[0] = beta;
      int kk = 0;
      for (int k = 0; k < kmax; ++k) {
        double* Vk = Vb + (size_t)k * n;
        /* w = S^-1 [F(q + eps S V_k) - F(q)] / eps */
        for (int i = 0; i < n; ++i) qp[i] = qc[i] + eps * sc[i] * Vk[i];
        residual_F(&col, lam, qp, Rc, w);
        for (int i = 0; i < n; ++i) w[i] = (w[i] - F[i]) / eps / sc[i];
        /* modified Gram-Schmidt */
        double* Hk = H + (size_t)k * (kmax + 1);
        for (int j = 0; j <= k; ++j) {
          const double* Vj = Vb + (size_t)j * n;
          double h = 0.0;
          for (int i = 0; i < n; ++i) h += w[i] * Vj[i];
          Hk[j] = h;
          for (int i = 0; i < n; ++i) w[i] -= h * Vj[i];
        }
        double hn = 0.0;
        for (int i = 0; i < n; ++i) hn += w[i] * w[i];
        hn = sqrt(hn);
        Hk[k + 1] = hn;
        double* Vn = Vb + (size_t)(k + 1) * n;
        for (int i = 0; i < n; ++i) Vn[i] = hn > 0.0 ? w[i] / hn : 0.0;
        /* previous rotations, then the one that zeroes H[k+1][k] */
        for (int j = 0; j < k; ++j) {
          double t = cs[j] * Hk[j] + sn[j] * Hk[j + 1];
          Hk[j + 1] = -sn[j] * Hk[j] + cs[j] * Hk[j + 1];
          Hk[j] = t;
        }
        double r = hypot(Hk[k], Hk[k + 1]);
        cs[k] = r > 0.0 ? Hk[k] / r : 1.0;
        sn[k] = r > 0.0 ? Hk[k + 1] / r : 0.0;
        Hk[k] = r;
        Hk[k + 1] = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        kk = k + 1;
        if (fabs(g[k + 1]) <= gtol * beta || hn == 0.0) break;
      }
      kits[c] += kk;
      /* R y = g (back substitution), dq = S sum_j y_j V_j */
      for (int j = kk - 1; j >= 0; --j) {
        double t = g[j];
        for (int l = j + 1; l < kk; ++l) t -= H[(size_t)l * (kmax + 1) + j] * y[l];
        y[j] = t / H[(size_t)j * (kmax + 1) + j];
      }
      for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int j = 0; j < kk; ++j) d += y[j] * Vb[(size_t)j * n + i];
        qc[i] += sc[i] * d;
      }
      iters[c] = m;
      residual_F(&col, lam, qc, Rc, F);
      double fn = scaled_norm(&col, F);
      if (!(fn == fn)) { status[c] = 6; break; }
      if (fn <= rtol * f0 || fn <= OR_NEWTON_FLOOR * scaled_norm(&col, qc)) {
        status[c] = 0;
        break;
      }
    }
    column_free(&col);
  }
  free(F); free(qp); free(w); free(sc); free(Vb); free(H); free(cs); free(sn); free(g); free(y);
  return 0;
}

/* Sec. 4.2.3 (NHEVI-LU): Newton-Raphson, Eqs. (Newton-system-update) and
 * (Newton-system), with the analytic Jacobian J(q_m) = I - Lambda L(q_m)
 * rebuilt in band storage and LU-factored at every iteration.
 * q holds the initial guess on entry and the root on exit.  iters[c] is the
 * number of Newton updates taken; status[c] = 0 converged, 4 singular
 * Jacobian, 5 not converged within max_iter.  Stop (reading R7; the paper
 * gives the tolerance, not the test): after update m,
 *   |S^-1 F(q_m)| <= rtol |S^-1 F(q_0)|  and  |S^-1 dq_m| <= rtol |S^-1 (q_m - q_0)|
 * (the residual small against the first, and the last update small against
 * the whole update, so that the iterate agrees with the root to about rtol in
 * the update's norm), or |S^-1 F(q_m)| at the rounding floor of its FP64
 * evaluation; S = (rho_bar, rho_bar c_s, Theta_bar). */
int or_newton(int ncols, int nez, int N, const double* ztop, double lam, const double* R,
              double* q, double rtol, int max_iter, int* iters, int* status) {
  int n = 3 * (nez * N + 1), kl = 3 * (N + 1) - 1, ldab = 3 * kl + 1;
  double* ab = (double*)malloc(sizeof(double) * (size_t)ldab * n);
  double* F = (double*)malloc(sizeof(double) * n);
  double* qi = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  int* ipiv = (int*)malloc(sizeof(int) * n);
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    size_t o = (size_t)c * n;
    double* qc = q + o;
    for (int i = 0; i < n; ++i) qi[i] = qc[i];
    residual_F(&col, lam, qc, R + o, F);
    double f0 = scaled_norm(&col, F);
    iters[c] = 0;
    status[c] = 0;
    if (f0 > OR_NEWTON_FLOOR * scaled_norm(&col, qc)) {
      status[c] = 5;
      for (int m = 1; m <= max_iter; ++m) {
        if (factor_band(&col, lam, qc, ab, ldab, ipiv) != 0) { status[c] = 4; break; }
        for (int i = 0; i < n; ++i) F[i] = -F[i];
        solve_band(&col, ab, ldab, ipiv, F);
        for (int i = 0; i < n; ++i) qc[i] += F[i];
        const double dn = scaled_norm(&col, F);
        for (int i = 0; i < n; ++i) t[i] = qc[i] - qi[i];
        const double un = scaled_norm(&col, t);
        iters[c] = m;
        residual_F(&col, lam, qc, R + o, F);
        double fn = scaled_norm(&col, F);
        if ((fn <= rtol * f0 && dn <= rtol * un) || fn <= OR_NEWTON_FLOOR * scaled_norm(&col, qc)) {
          status[c] = 0;
          break;
        }
      }
    }
    column_free(&col);
  }
  free(ab);
  free(F);
  free(qi);
  free(t);
  free(ipiv);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1 and 4.3: one IMEX ARK step with the HEVI split.  The       */
/* tableau is (s, A explicit, At implicit, b), row-major s x s, ESDIRK */
/* (first stage explicit, constant diagonal gamma = At[1][1], b = bt).  */
/* H is the explicit tendency, held constant over the step.            */
/* ------------------------------------------------------------------ */

/* LHEVI (Sec. 4.3), in the ARK form of Eq. (lhevi-ark-final-3): with
 * S(Q) = H + V(Q) the full right-hand side and w_ij = (at_ij - a_ij)/at_ii,
 *   q^E   = q^n + dt sum_{j<i} a_ij S(Q_j),
 *   q_hat = q^E + sum_{j<i} w_ij Q_j,
 *   (I - gamma dt L) q_tt = q_hat                    (Eq. lhevi-ark-final-2),
 *   Q_i   = q_tt - sum_{j<i} w_ij Q_j,
 * and q^{n+1} = q^n + dt sum_i b_i S(Q_i) (Sec. 4.1 with b = bt).  Since the
 * rows of A and At have equal sums, sum_j w_ij = -1 and q_tt is a difference
 * of states.
 * lin = 0: L linearised about q^n (LHEVI-PS, Sec. 4.3.1); lin = 1: about
 * the reference state (LHEVI-RS); lin = 2: V itself replaced by the
 * reference-state linear operator V(q) := L_RS (q - q_bar), the linear test
 * problem.  info[c] = band-LU info of the step's factorisation. */
/* One LHEVI step with L linearised about qlin (per column, state layout)
 * when qlin != NULL: a Jacobian kept from an earlier step (the update
 * interval of Sec. 4.3 and the timing table of Sec. 7.1, R10); otherwise as
 * or_lhevi_step. */
static int lhevi_step_impl(int ncols, int nez, int N, const double* ztop, int s, const double* A,
                           const double* At, const double* b, double dt, int lin,
                           const double* qlin, const double* qn, const double* H, double* qout,
                           int* info) {
  int n = 3 * (nez * N + 1), kl = 3 * (N + 1) - 1, ldab = 3 * kl + 1;
  double gam = At[1 * s + 1], lam = gam * dt;
  double* ab = (double*)malloc(sizeof(double) * (size_t)ldab * n);
  int* ipiv = (int*)malloc(sizeof(int) * n);
  double* Q = (double*)malloc(sizeof(double) * (size_t)n * (2 * s + 3));
  double *S = Q + (size_t)n * s, *q0 = S + (size_t)n * s, *qbar = q0 + n, *tmp = qbar + n;
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    size_t o = (size_t)c * n;
    const double *qnc = qn + o, *Hc = H + o;
    for (int I = 0; I < col.nz; ++I) {
      qbar[3 * I] = col.rho_b[I];
      qbar[3 * I + 1] = 0.0;
      qbar[3 * I + 2] = col.X_b[I];
    }
    memcpy(q0, qlin ? qlin + o : (lin == 0 ? qnc : qbar), sizeof(double) * n);
    info[c] = factor_band(&col, lam, q0, ab, ldab, ipiv);
    for (int i = 0; i < s; ++i) {
      double* Qi = Q + (size_t)n * i;
      if (i == 0) {
        memcpy(Qi, qnc, sizeof(double) * n);
      } else {
        /* q_hat = q^n + dt sum_j a_ij S_j + sum_j w_ij Q_j, solved in place */
        for (int r = 0; r < n; ++r) {
          double acc = 0.0, wq = 0.0;
          for (int j = 0; j < i; ++j) {
            acc += A[i * s + j] * S[(size_t)n * j + r];
            wq += (At[i * s + j] - A[i * s + j]) / gam * Q[(size_t)n * j + r];
          }
          Qi[r] = qnc[r] + dt * acc + wq;
        }
        if (info[c] == 0) solve_band(&col, ab, ldab, ipiv, Qi);
        /* Q_i = q_tt - sum_j w_ij Q_j */
        for (int r = 0; r < n; ++r) {
          double wq = 0.0;
          for (int j = 0; j < i; ++j) wq += (At[i * s + j] - A[i * s + j]) / gam * Q[(size_t)n * j + r];
          Qi[r] -= wq;
        }
      }
      /* S(Q_i) = H + V(Q_i) */
      double* Si = S + (size_t)n * i;
      if (lin == 2) {
        for (int r = 0; r < n; ++r) tmp[r] = Qi[r] - qbar[r];
        apply_L(&col, qbar, tmp, Si);  /* V(Q) = L_RS (Q - q_bar) */
      } else {
        apply_V(&col, Qi, Si);
      }
      for (int r = 0; r < n; ++r) Si[r] += Hc[r];
    }
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int i = 0; i < s; ++i) acc += b[i] * S[(size_t)n * i + r];
      qout[o + r] = qnc[r] + dt * acc;
    }
    column_free(&col);
  }
  free(ab);
  free(ipiv);
  free(Q);
  return 0;
}

int or_lhevi_step(int ncols, int nez, int N, const double* ztop, int s, const double* A,
                  const double* At, const double* b, double dt, int lin, const double* qn,
                  const double* H, double* qout, int* info) {
  return lhevi_step_impl(ncols, nez, N, ztop, s, A, At, b, dt, lin, NULL, qn, H, qout, info);
}

/* LHEVI step with the Jacobian linearised about a given state qlin; lin = 0
 * for V itself, 2 for the linear test problem V := L_RS (q - q_bar). */
int or_lhevi_step_about(int ncols, int nez, int N, const double* ztop, int s, const double* A,
                        const double* At, const double* b, double dt, int lin, const double* qlin,
                        const double* qn, const double* H, double* qout, int* info) {
  return lhevi_step_impl(ncols, nez, N, ztop, s, A, At, b, dt, lin, qlin, qn, H, qout, info);
}

/* NHEVI-LU (Sec. 4.2): stage i solves F(Q_i) = Q_i - gamma dt V(Q_i) - R_i = 0,
 *   R_i = q^n + dt sum_{j<i} [ a_ij H + at_ij V(Q_j) ],
 * by Newton from the guess Q_{i-1}; then
 *   q^{n+1} = q^n + dt sum_i b_i [ H + V(Q_i) ].
 * iters[c] = total Newton updates over the step; status[c] as or_newton. */
int or_nhevi_step(int ncols, int nez, int N, const double* ztop, int s, const double* A,
                  const double* At, const double* b, double dt, const double* qn, const double* H,
                  double rtol, int max_iter, double* qout, int* iters, int* status) {
  int n = 3 * (nez * N + 1);
  double lam = At[1 * s + 1] * dt;
  double* Q = (double*)malloc(sizeof(double) * (size_t)n * (2 * s + 1));
  double *VQ = Q + (size_t)n * s, *R = VQ + (size_t)n * s;
  for (int c = 0; c < ncols; ++c) {
    column_t col;
    if (column_init(&col, nez, N, ztop[c])) return 1;
    size_t o = (size_t)c * n;
    const double *qnc = qn + o, *Hc = H + o;
    iters[c] = 0;
    status[c] = 0;
    for (int i = 0; i < s; ++i) {
      double* Qi = Q + (size_t)n * i;
      if (i == 0) {
        memcpy(Qi, qnc, sizeof(double) * n);
      } else {
        for (int r = 0; r < n; ++r) {
          double acc = 0.0;
          for (int j = 0; j < i; ++j) acc += A[i * s + j] * Hc[r] + At[i * s + j] * VQ[(size_t)n * j + r];
          R[r] = qnc[r] + dt * acc;
        }
        memcpy(Qi, Q + (size_t)n * (i - 1), sizeof(double) * n);
        int it = 0, st = 0;
        or_newton(1, nez, N, ztop + c, lam, R, Qi, rtol, max_iter, &it, &st);
        iters[c] += it;
        if (st && !status[c]) status[c] = st;
      }
      apply_V(&col, Qi, VQ + (size_t)n * i);
    }
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int i = 0; i < s; ++i) acc += b[i] * (Hc[r] + VQ[(size_t)n * i + r]);
      qout[o + r] = qnc[r] + dt * acc;
    }
    column_free(&col);
  }
  free(Q);
  return 0;
}
