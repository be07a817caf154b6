// hevi_capi.cu -- host side of the C ABI declared in include/hevi.h.
//
// Setup (Sec. 3): LGL nodes and weights of each order and the derivative of
// the cardinal Lagrange basis are built here in FP64; columns are grouped by
// size class into tiles of 32; the reference state of every column is
// computed on the device.  Calls launch kernels on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hevi_internal.cuh"

using hevi::Band;
using hevi::DevView;
using hevi::kMaxOrder;
using hevi::kTile;
using hevi::TileDesc;

namespace {

// Failure counters on the device: [0] any, [1] singular, [2] not converged,
// [3] bad input.
constexpr int kFailSlots = 5;

// Factor record length per pivot step and column: FP64 band LU with partial
// pivoting (L record {l_1..l_K, pivot, 1/u_jj}, U record of 2K entries) or
// the FP32 no-pivot factors (K multipliers; 1/u_jj and K entries of U).
int rl_of(int N, hevi_precision prec) {
  if (prec == HEVI_FP32_IR) return hevi::np_record_floats(N);
  const int K = 3 * (N + 1) - 1;
  return ((K + 2) + 3) / 4 * 4 + ((2 * K) + 3) / 4 * 4;
}
int ur2_of(int N) {  // Newton scratch record {1/u_jj, u_j,j+1..j+2K}
  const int K = 3 * (N + 1) - 1;
  return ((2 * K + 1) + 3) / 4 * 4;
}

// Legendre P_n(x) by the three-term recurrence.
double legendre_p(int n, double x) {
  if (n == 0) return 1.0;
  double a = 1.0, b = x;
  for (int k = 2; k <= n; ++k) {
    const double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  return b;
}

// LGL points of order N: the roots of P_{N+1} - P_{N-1} (which include +-1),
// found by Newton's method with q' = (2N+1) P_N; weights 2/(N(N+1) P_N^2).
void lgl_points(int N, double* x, double* w) {
  for (int k = 0; k <= N; ++k) {
    double t = -std::cos(M_PI * k / N);
    if (k > 0 && k < N) {
      for (int it = 0; it < 200; ++it) {
        const double q = legendre_p(N + 1, t) - legendre_p(N - 1, t);
        const double dq = (2.0 * N + 1.0) * legendre_p(N, t);
        const double d = q / dq;
        t -= d;
        if (std::fabs(d) <= 1e-17) break;
      }
    }
    x[k] = t;
  }
  for (int k = 0; k <= N; ++k) {
    const double p = legendre_p(N, x[k]);
    w[k] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

// Derivative of the cardinal Lagrange basis by barycentric weights:
// Dhat_kj = h_j'(x_k) = (b_j / b_k) / (x_k - x_j), k != j; the diagonal makes
// each row sum to zero.
void lagrange_derivative(int N, const double* x, double* D) {
  double b[kMaxOrder + 1];
  for (int j = 0; j <= N; ++j) {
    double p = 1.0;
    for (int m = 0; m <= N; ++m)
      if (m != j) p *= (x[j] - x[m]);
    b[j] = 1.0 / p;
  }
  for (int k = 0; k <= N; ++k) {
    double diag = 0.0;
    for (int j = 0; j <= N; ++j) {
      if (j == k) continue;
      const double d = (b[j] / b[k]) / (x[k] - x[j]);
      D[k * (N + 1) + j] = d;
      diag -= d;
    }
    D[k * (N + 1) + k] = diag;
  }
}

hevi::LglTables make_tables() {
  hevi::LglTables t{};
  std::memset(&t, 0, sizeof(t));
  for (int N = 1; N <= kMaxOrder; ++N) {
    double D[(kMaxOrder + 1) * (kMaxOrder + 1)];
    lgl_points(N, t.xi[N], t.w[N]);
    lagrange_derivative(N, t.xi[N], D);
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N; ++j) {
        const double v = t.w[N][k] * D[k * (N + 1) + j];
        t.wD[N][k * (N + 1) + j] = v;
        t.wDf[N][k * (N + 1) + j] = (float)v;
      }
    for (int k = 0; k <= N; ++k) t.iwf[N][k] = (float)(1.0 / t.w[N][k]);
    for (int k = 0; k <= N; ++k) t.iw[N][k] = 1.0 / t.w[N][k];
    for (int k = 0; k <= N; ++k) t.xh[N][k] = (float)(0.5 * (t.xi[N][k] + 1.0));
    {
      auto wD = [&](int k, int j) { return t.wD[N][k * (N + 1) + j]; };
      for (int dJ = -N; dJ <= N; ++dJ) {
        const int o = dJ + N;
        t.gcoef[N][0][o] = dJ >= 0 ? (float)(wD(0, dJ) / t.w[N][0]) : 0.0f;            // bottom
        t.gcoef[N][1][o] = dJ <= 0 ? (float)(wD(N, N + dJ) / t.w[N][0]) : 0.0f;        // top
        double sh = 0.0;                                                              // shared
        if (dJ <= 0) sh += wD(N, N + dJ);
        if (dJ >= 0) sh += wD(0, dJ);
        t.gcoef[N][2][o] = (float)(sh / (2.0 * t.w[N][0]));
        for (int k = 1; k < N; ++k)                                                   // interior
          t.gcoef[N][2 + k][o] =
              (k + dJ >= 0 && k + dJ <= N) ? (float)(wD(k, k + dJ) / t.w[N][k]) : 0.0f;
      }
    }
    // even-odd halves (LGL symmetry: wD[N-k][N-j] = -wD[k][j])
    const int P = (N + 1) / 2;
    for (int k = 0; k < P; ++k)
      for (int j = 0; j < P; ++j) {
        t.ep[N][k][j] = 0.5 * (t.wD[N][k * (N + 1) + j] + t.wD[N][k * (N + 1) + N - j]);
        t.op[N][k][j] = 0.5 * (t.wD[N][k * (N + 1) + j] - t.wD[N][k * (N + 1) + N - j]);
      }
    if (N % 2 == 0)
      for (int j = 0; j < P; ++j)
        t.om[N][j] = 0.5 * (t.wD[N][(N / 2) * (N + 1) + j] - t.wD[N][(N / 2) * (N + 1) + N - j]);
    // double-float pairs: hi = v rounded to FP32, lo = the remainder rounded
    auto split = [](double v) {
      const float hi = (float)v;
      return float2{hi, (float)(v - (double)hi)};
    };
    for (int k = 0; k < (N + 1) * (N + 1); ++k) t.wD2[N][k] = split(t.wD[N][k]);
    for (int k = 0; k <= N; ++k) t.iw2[N][k] = split(t.iw[N][k]);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) {
        t.ep2[N][k][j] = split(t.ep[N][k][j]);
        t.op2[N][k][j] = split(t.op[N][k][j]);
      }
    for (int j = 0; j < 3; ++j) t.om2[N][j] = split(t.om[N][j]);
  }
  return t;
}

}  // namespace

namespace hevi {
const LglTables& lgl_tables() {
  static const LglTables t = make_tables();
  return t;
}
}  // namespace hevi

struct hevi_ctx {
  DevView v{};
  hevi_precision prec = HEVI_FP64;
  cudaStream_t stream = nullptr;
  int64_t ncols = 0, state_size = 0, ntiles = 0;
  std::vector<int64_t> h_off;
  std::vector<TileDesc> h_tiles;
  int max_order = 0, max_ylen = 0;
  // tiles of each order N occupy [order_begin[N], order_begin[N] + order_count[N])
  int32_t order_begin[kMaxOrder + 1] = {0}, order_count[kMaxOrder + 1] = {0};
  int order_ylen[kMaxOrder + 1] = {0};
  // FP32 stage solve: the tiles in decreasing cost (records per tile) for the
  // single launch over all orders (null with one order: tiles in place), and
  // the launch's tile counter
  int32_t* d_tile_list = nullptr;
  int32_t* d_tile_next = nullptr;
  // per column: order and element count (device), for re-topping columns
  int32_t* d_col_order = nullptr;
  int32_t* d_col_nez = nullptr;
  std::vector<int32_t> h_col_nez;
  // NHEVI-LU: read the count of iterating columns on the host after each
  // Newton iteration (and stop enqueuing at zero), else gate on the device only
  bool newton_host_check = true;
  bool fuse_stages = true;
  double lam = 0.0;
  bool factored = false;
  double ir_tol = 1e-11;
  int ir_max = 10;
  int64_t scr_floats = 0;
  int64_t fac_elems = 0;
  int64_t ysc_floats = 0;
  // device allocations
  std::vector<void*> allocs;
  // NHEVI-LU sequence: q0, -F and the update (state vectors); per column
  // |S^-1 F(q0)|, convergence, iterations, status, and the status and
  // iterations the inner factor / solve calls write; per iteration the count
  // of columns still iterating; failure counters of the inner calls
  double* nw_vec = nullptr;
  double* nw_f0 = nullptr;
  int32_t* nw_int = nullptr;
  int32_t* nw_active = nullptr;
  int32_t* nw_fail = nullptr;
  // NHEVI-GMRES scratch: three state vectors and per-tile Krylov storage
  double* gm_vec = nullptr;
  double* gm_tile = nullptr;
  int gm_kmax = 0;
  float* scr = nullptr;
  double* work = nullptr;
  int64_t work_vecs = 0;
  int32_t* h_fail = nullptr;  // pinned mirror of the failure counters
  int64_t launches = 0;
  int64_t dev_bytes = 0;
  // opt-in per-kernel timing with CUDA events on the context's stream
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[8] = {0};
  int64_t prof_n[8] = {0};
  // fork/join of per-order launches when several orders are present: the
  // kernels of each order run on their own stream, concurrently
  int norders = 0;
  cudaStream_t aux[kMaxOrder + 1] = {nullptr};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kMaxOrder + 1] = {nullptr};

  template <typename T>
  hevi_status alloc(T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return HEVI_ERR_OOM;
    }
    allocs.push_back(q);
    dev_bytes += (int64_t)(count * sizeof(T));
    *p = static_cast<T*>(q);
    return HEVI_OK;
  }
};

namespace {

enum Kind { kSetup = 0, kFactor, kSolve, kApply, kApplyStage, kNewton, kCombine, kNumKinds };
const char* kKindNames[kNumKinds] = {"setup", "factor", "stage_solve", "apply",
                                     "apply_stage", "newton_fpass", "combine"};

cudaEvent_t get_event(hevi_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events when timing is on (and the stream is
// not being captured into a graph).
struct Scope {
  hevi_ctx* c;
  int kind;
  cudaEvent_t a = nullptr;
  Scope(hevi_ctx* ctx, int k) : c(ctx), kind(k) {
    if (!c->prof) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &cs);
    if (cs != cudaStreamCaptureStatusNone) return;
    a = get_event(c);
    cudaEventRecord(a, c->stream);
  }
  ~Scope() {
    if (!a) return;
    cudaEvent_t b = get_event(c);
    cudaEventRecord(b, c->stream);
    c->prof_recs.push_back({kind, a, b});
  }
};

void fold_profile(hevi_ctx* c) {
  if (c->prof_recs.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->prof_recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.kind] += ms;
      c->prof_n[r.kind] += 1;
    }
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof_recs.clear();
  cudaGetLastError();
}

hevi_status check_launch(hevi_ctx* c, int n = 0) {
  c->launches += n;
  return cudaGetLastError() == cudaSuccess ? HEVI_OK : HEVI_ERR_CUDA;
}

// Run f(view, order, ylen, stream) for every order present, with the view's
// tile range set to that order's tiles.  With one order the launch goes to
// the context's stream.  With several, each order's launch goes to its own
// stream, forked from and joined back into the context's stream by events,
// so that the orders' kernels share the GPU instead of running one after
// the other (each with its own partial last wave).  Fork and join are plain
// event record/wait pairs and so are also valid under stream capture.
template <class F>
void for_orders(hevi_ctx* c, const DevView& base, F&& f) {
  const bool fork = c->norders > 1;
  if (fork) cudaEventRecord(c->fork_ev, c->stream);
  for (int N = 1; N <= kMaxOrder; ++N) {
    if (!c->order_count[N]) continue;
    DevView v = base;
    v.tile_begin = c->order_begin[N];
    v.tile_count = c->order_count[N];
    v.tile_list = nullptr;
    cudaStream_t sk = c->stream;
    if (fork) {
      sk = c->aux[N];
      cudaStreamWaitEvent(sk, c->fork_ev, 0);
    }
    f(v, N, c->order_ylen[N], sk);
    if (fork) {
      cudaEventRecord(c->join_ev[N], sk);
      cudaStreamWaitEvent(c->stream, c->join_ev[N], 0);
    }
    c->launches += 1;
  }
}

// One stage solve x = A^-1 b over every tile.  The FP32 path is a single
// persistent launch whose warps take the tiles of all orders, longest first,
// from a shared counter; the FP64 path launches per order.
void stage_solve_all(hevi_ctx* c, const DevView& base, double lam, const double* b, double* x) {
  if (c->prec == HEVI_FP32_IR) {
    DevView v = base;
    v.tile_begin = 0;
    v.tile_count = (int32_t)c->ntiles;
    v.tile_list = c->d_tile_list;
    v.tile_next = c->d_tile_next;
    hevi::launch_solve_np(v, c->norders > 1 ? 0 : c->max_order, c->max_order, lam, b, x,
                          c->ir_tol, c->ir_max, c->stream);
    c->launches += 1;
    return;
  }
  for_orders(c, base, [&](const DevView& v, int N, int ylen, cudaStream_t sk) {
    hevi::launch_solve(v, N, c->prec, lam, b, x, c->ir_tol, c->ir_max, ylen, sk);
  });
}

// S = H + V(Q): in double-float arithmetic on an FP32 context (its solves
// are refined to about the same accuracy), in FP64 on an FP64 context.
void apply_rhs(hevi_ctx* c, const DevView& v, int N, const double* Q, const double* H, double* S,
               cudaStream_t sk, const hevi::StageFuse* fz = nullptr) {
  if (c->prec == HEVI_FP32_IR)
    hevi::launch_apply_rhs_df(v, N, Q, H, S, sk, fz);
  else
    hevi::launch_apply_rhs(v, N, Q, H, S, sk);
}

void reset_fail(hevi_ctx* c) {
  cudaMemsetAsync(c->v.fail_count, 0, kFailSlots * sizeof(int32_t), c->stream);
}

// Wait for the stream and turn the failure counters into a status.
hevi_status wait_status(hevi_ctx* c) {
  if (cudaMemcpyAsync(c->h_fail, c->v.fail_count, kFailSlots * sizeof(int32_t),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return HEVI_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HEVI_ERR_CUDA;
  if (c->h_fail[0] == 0) return HEVI_OK;
  if (c->h_fail[4]) return HEVI_ERR_WAIT_TIMEOUT;
  if (c->h_fail[3]) return HEVI_ERR_BAD_INPUT;
  if (c->h_fail[1]) return HEVI_ERR_SINGULAR;
  return HEVI_ERR_NOT_CONVERGED;
}

hevi_status ensure_work(hevi_ctx* c, int64_t vecs) {
  if (c->work_vecs >= vecs) return HEVI_OK;
  if (c->work) {
    cudaStreamSynchronize(c->stream);
    auto it = std::find(c->allocs.begin(), c->allocs.end(), (void*)c->work);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(c->work);
    c->dev_bytes -= c->work_vecs * c->state_size * (int64_t)sizeof(double);
    c->work = nullptr;
    c->work_vecs = 0;
  }
  hevi_status s = c->alloc(&c->work, (size_t)(vecs * c->state_size));
  if (s == HEVI_OK) c->work_vecs = vecs;
  return s;
}

constexpr int kNewtonMaxIter = 1000;

hevi_status ensure_newton(hevi_ctx* c) {
  if (c->nw_vec) return HEVI_OK;
  hevi_status s;
  if ((s = c->alloc(&c->nw_vec, (size_t)(3 * c->state_size))) ||
      (s = c->alloc(&c->nw_f0, (size_t)c->ncols)) ||
      (s = c->alloc(&c->nw_int, (size_t)(5 * c->ncols))) ||
      (s = c->alloc(&c->nw_active, (size_t)(kNewtonMaxIter + 1))) ||
      (s = c->alloc(&c->nw_fail, (size_t)kFailSlots)))
    return s;
  return HEVI_OK;
}

// NHEVI-LU (Sec. 4.2.3) as a sequence of launches: an F pass at the initial
// guess, then per iteration the factorisation of J(q_m) (hevi_factor's
// kernels with q_m as the linearisation state), the refined solve
// J delta = -F(q_m) (hevi_stage_solve's kernels) and the F pass that applies
// the update and takes the stop test.  The launches of an iteration do
// nothing once no column is left iterating (a device-side count gates them),
// so the sequence needs no host synchronisation and can be captured into a
// graph; `sync` lets the host stop launching as soon as every column is done.
hevi_status newton_sequence(hevi_ctx* c, double lam, double* q, const double* R, double rtol,
                            int32_t max_iter, bool sync) {
  hevi_status s = ensure_newton(c);
  if (s != HEVI_OK) return s;
  const int64_t n = c->state_size, nc = c->ncols;
  hevi::NewtonArgs a;
  a.lam = lam;
  a.rtol = rtol;
  a.max_iter = max_iter;
  a.q = q;
  a.R = R;
  a.q0 = c->nw_vec;
  a.rhs = c->nw_vec + n;
  a.delta = c->nw_vec + 2 * n;
  a.f0 = c->nw_f0;
  a.conv = c->nw_int;
  a.iters = c->nw_int + nc;
  a.status = c->nw_int + 2 * nc;
  // the inner factor / solve calls report into scratch, not the context
  DevView in = c->v;
  in.col_status = c->nw_int + 3 * nc;
  in.col_iters = c->nw_int + 4 * nc;
  in.fail_count = c->nw_fail;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &cap);
  if (cap != cudaStreamCaptureStatusNone) sync = false;
  cudaMemcpyAsync(c->nw_vec, q, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemsetAsync(c->nw_active, 0, (max_iter + 1) * sizeof(int32_t), c->stream);
  a.iter = 0;
  a.active_in = nullptr;
  a.active_out = c->nw_active;
  {
    Scope sc(c, kNewton);
    for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
      hevi::launch_newton_fpass(v, N, a, sk);
    });
  }
  for (int m = 1; m <= max_iter; ++m) {
    const int32_t* gate = c->nw_active + (m - 1);
    if (sync) {
      int32_t h = 0;
      if (cudaMemcpyAsync(c->h_fail + kFailSlots, gate, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return HEVI_ERR_CUDA;
      h = c->h_fail[kFailSlots];
      if (h == 0) break;
    }
    DevView g = in;
    g.gate = gate;
    {
      Scope sc(c, kFactor);
      for_orders(c, g, [&](const DevView& v, int N, int ylen, cudaStream_t sk) {
        hevi::launch_factor(v, N, c->prec, lam, q, ylen, sk);
      });
    }
    {
      Scope sc(c, kSolve);
      stage_solve_all(c, g, lam, a.rhs, const_cast<double*>(a.delta));
    }
    a.iter = m;
    a.active_in = gate;
    a.active_out = c->nw_active + m;
    {
      Scope sc(c, kNewton);
      for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
        hevi::launch_newton_fpass(v, N, a, sk);
      });
    }
  }
  hevi::launch_newton_finish(c->v, a, c->stream);
  c->launches += 1;
  c->factored = false;  // the factors now belong to J(q), not to the last hevi_factor
  return check_launch(c);
}

// Longest column of the context (unknowns).
int64_t max_unknowns(const hevi_ctx* c) {
  int64_t m = 0;
  for (const TileDesc& t : c->h_tiles) m = std::max<int64_t>(m, 3 * ((int64_t)t.nez * t.order + 1));
  return m;
}

hevi_status ensure_gmres(hevi_ctx* c, int kmax) {
  if (c->gm_kmax >= kmax && c->gm_vec) return HEVI_OK;
  cudaStreamSynchronize(c->stream);
  for (double** p : {&c->gm_vec, &c->gm_tile}) {
    if (*p) {
      auto it = std::find(c->allocs.begin(), c->allocs.end(), (void*)*p);
      if (it != c->allocs.end()) c->allocs.erase(it);
      cudaFree(*p);
      *p = nullptr;
    }
  }
  const int64_t nmax = max_unknowns(c);
  const int64_t per_tile = ((int64_t)(kmax + 1) * nmax + (int64_t)kmax * (kmax + 3) / 2 +
                            4 * (int64_t)kmax + 1) * kTile;
  hevi_status s = c->alloc(&c->gm_vec, (size_t)(3 * c->state_size));
  if (s != HEVI_OK) return s;
  s = c->alloc(&c->gm_tile, (size_t)(per_tile * c->ntiles));
  if (s != HEVI_OK) return s;
  c->gm_kmax = kmax;
  return HEVI_OK;
}

}  // namespace

extern "C" {

const char* hevi_status_string(hevi_status s) {
  switch (s) {
    case HEVI_OK: return "ok";
    case HEVI_ERR_INVALID_ARG: return "invalid argument";
    case HEVI_ERR_CUDA: return "CUDA error";
    case HEVI_ERR_OOM: return "out of device memory";
    case HEVI_ERR_SINGULAR: return "singular column";
    case HEVI_ERR_NOT_CONVERGED: return "not converged";
    case HEVI_ERR_BAD_INPUT: return "non-physical input state";
    case HEVI_ERR_WAIT_TIMEOUT: return "device wait past its limit";
  }
  return "unknown status";
}

hevi_status hevi_setup(hevi_ctx** out, const hevi_column_grid* grid, const hevi_ref_params* ref,
                       hevi_precision precision, void* stream) {
  if (!out || !grid || grid->ncols <= 0 || !grid->classes || grid->nclasses <= 0 || !grid->z_top)
    return HEVI_ERR_INVALID_ARG;
  if (grid->nclasses > 1 && !grid->class_of_col) return HEVI_ERR_INVALID_ARG;
  if (precision != HEVI_FP64 && precision != HEVI_FP32_IR) return HEVI_ERR_INVALID_ARG;
  if (grid->ncols > (int64_t)INT32_MAX) return HEVI_ERR_INVALID_ARG;
  for (int c = 0; c < grid->nclasses; ++c) {
    const hevi_size_class& k = grid->classes[c];
    if (k.order < 1 || k.order > kMaxOrder || k.nez < 1 || k.nez > 4096) return HEVI_ERR_INVALID_ARG;
  }
  const int64_t ncols = grid->ncols;
  std::vector<int32_t> cls(ncols), order(ncols), nez(ncols);
  std::vector<double> dz(ncols);
  for (int64_t i = 0; i < ncols; ++i) {
    const int32_t k = grid->class_of_col ? grid->class_of_col[i] : 0;
    if (k < 0 || k >= grid->nclasses) return HEVI_ERR_INVALID_ARG;
    const double zt = grid->z_top[i];
    if (!(zt > 0.0) || !std::isfinite(zt)) return HEVI_ERR_INVALID_ARG;
    cls[i] = k;
    order[i] = grid->classes[k].order;
    nez[i] = grid->classes[k].nez;
    dz[i] = zt / nez[i];
  }
  hevi_ctx* c = new (std::nothrow) hevi_ctx();
  if (!c) return HEVI_ERR_OOM;
  c->prec = precision;
  c->stream = static_cast<cudaStream_t>(stream);
  c->ncols = ncols;
  hevi::Phys ph;
  ph.T0 = ref ? ref->T0 : 300.0;
  ph.p0 = ref ? ref->p0 : 1.0e5;
  ph.R = ref ? ref->R : 287.17;
  ph.cp = ref ? ref->cp : 1004.67;
  ph.g = ref ? ref->g : 9.80616;
  hevi::phys_derive(ph);
  c->v.ph = ph;
  c->v.ncols = ncols;

  // state offsets
  c->h_off.resize(ncols + 1);
  c->h_off[0] = 0;
  for (int64_t i = 0; i < ncols; ++i) c->h_off[i + 1] = c->h_off[i] + 3 * ((int64_t)nez[i] * order[i] + 1);
  c->state_size = c->h_off[ncols];

  // class-sorted permutation and tiles of 32 columns of one class
  std::vector<int32_t> perm(ncols);
  for (int64_t i = 0; i < ncols; ++i) perm[i] = (int32_t)i;
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
    return order[a] != order[b] ? order[a] < order[b] : cls[a] < cls[b];
  });
  int64_t fac_off = 0, scr_off = 0, y_off = 0;
  const int esz = precision == HEVI_FP64 ? 8 : 4;
  for (int64_t i = 0; i < ncols;) {
    const int32_t k = cls[perm[i]];
    int64_t j = i;
    while (j < ncols && j - i < kTile && cls[perm[j]] == k) ++j;
    TileDesc t;
    t.order = grid->classes[k].order;
    t.nez = grid->classes[k].nez;
    t.count = (int32_t)(j - i);
    t.first = (int32_t)i;
    t.fac_off = fac_off;
    t.scr_off = scr_off;
    t.y_off = y_off;
    const int64_t n = 3 * ((int64_t)t.nez * t.order + 1);
    // the FP32 solve's scratch, [row][lane]: the point coefficients of L(q0)
    // (FP64, n rows), the work vector (n + K + 1 rows, rounded to 4) and the
    // first solution, the correction sum and the residual's two parts (n rows each)
    y_off += (2 * n + (n + 3 * (t.order + 1) + 3) / 4 * 4 + 4 * n) * kTile;
    fac_off += n * rl_of(t.order, precision) * kTile;
    scr_off += n * ur2_of(t.order) * kTile;
    if (c->order_count[t.order] == 0) c->order_begin[t.order] = (int32_t)c->h_tiles.size();
    c->order_count[t.order] += 1;
    c->h_tiles.push_back(t);
    c->max_order = std::max(c->max_order, (int)t.order);
    const int K = 3 * (t.order + 1) - 1;
    c->max_ylen = std::max(c->max_ylen, (int)(n + 2 * K));
    c->order_ylen[t.order] = std::max(c->order_ylen[t.order], (int)(n + 2 * K));
    i = j;
  }
  c->ntiles = (int64_t)c->h_tiles.size();
  c->fac_elems = fac_off;
  c->scr_floats = scr_off;
  c->ysc_floats = y_off;
  (void)esz;

  static bool tables_done = false;
  static hevi::LglTables tables;
  if (!tables_done) {
    tables = make_tables();
    tables_done = true;
  }
  if (hevi::upload_tables(tables) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return HEVI_ERR_CUDA;
  }

  hevi_status s = HEVI_OK;
  int64_t* d_off;
  int32_t *d_perm, *d_order, *d_nez;
  double *d_dz, *d_ref;
  TileDesc* d_tiles;
  int32_t *d_fs, *d_cs, *d_it, *d_fail;
  void* d_fac;
  if ((s = c->alloc(&d_off, ncols + 1)) || (s = c->alloc(&d_perm, ncols)) ||
      (s = c->alloc(&d_order, ncols)) || (s = c->alloc(&d_nez, ncols)) ||
      (s = c->alloc(&d_dz, ncols)) || (s = c->alloc(&d_ref, c->state_size)) ||
      (s = c->alloc(&c->v.lin, c->state_size)) || (s = c->alloc(&d_tiles, c->ntiles)) ||
      (s = c->alloc(&c->v.ithb, c->state_size / 3)) ||
      (s = precision == HEVI_FP32_IR ? c->alloc(&c->v.ysc, c->ysc_floats) : HEVI_OK) ||
      (s = c->alloc(&d_fs, ncols)) || (s = c->alloc(&d_cs, ncols)) || (s = c->alloc(&d_it, ncols)) ||
      (s = c->alloc(&d_fail, kFailSlots)) || (s = c->alloc(&c->d_tile_next, 1)) ||
      (s = precision == HEVI_FP64 ? c->alloc((double**)&d_fac, c->fac_elems)
                                  : c->alloc((float**)&d_fac, c->fac_elems))) {
    hevi_destroy(c);
    return s;
  }
  if (cudaMallocHost(&c->h_fail, (kFailSlots + 1) * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    hevi_destroy(c);
    return HEVI_ERR_OOM;
  }
  for (int N = 1; N <= kMaxOrder; ++N) c->norders += c->order_count[N] ? 1 : 0;
  if (c->norders > 1) {
    // the single-launch solve takes the costliest tiles first, so that the
    // short ones fill the end of the launch
    std::vector<int32_t> list(c->ntiles);
    for (int64_t i = 0; i < c->ntiles; ++i) list[i] = (int32_t)i;
    auto cost = [&](int32_t i) {
      const TileDesc& t = c->h_tiles[i];
      return 3 * ((int64_t)t.nez * t.order + 1) * (int64_t)hevi::np_record_floats(t.order);
    };
    std::stable_sort(list.begin(), list.end(),
                     [&](int32_t a, int32_t b) { return cost(a) > cost(b); });
    if ((s = c->alloc(&c->d_tile_list, c->ntiles))) {
      hevi_destroy(c);
      return s;
    }
    cudaMemcpy(c->d_tile_list, list.data(), c->ntiles * sizeof(int32_t), cudaMemcpyHostToDevice);
    bool ok = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int N = 1; N <= kMaxOrder && ok; ++N) {
      if (!c->order_count[N]) continue;
      ok = cudaStreamCreateWithFlags(&c->aux[N], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->join_ev[N], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      hevi_destroy(c);
      return HEVI_ERR_CUDA;
    }
  }
  cudaMemcpy(d_off, c->h_off.data(), (ncols + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d_perm, perm.data(), ncols * sizeof(int32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d_order, order.data(), ncols * sizeof(int32_t), cudaMemcpyHostToDevice);
  c->d_col_order = d_order;
  c->d_col_nez = d_nez;
  c->h_col_nez = nez;
  cudaMemcpy(d_nez, nez.data(), ncols * sizeof(int32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d_dz, dz.data(), ncols * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(d_tiles, c->h_tiles.data(), c->ntiles * sizeof(TileDesc), cudaMemcpyHostToDevice);
  // the records' padding is never written by the factor kernels: zero it once
  cudaMemset(d_fac, 0, c->fac_elems * (precision == HEVI_FP64 ? 8 : 4));
  cudaMemset(d_fs, 0xff, ncols * sizeof(int32_t));  // no factorisation yet
  cudaMemset(d_cs, 0, ncols * sizeof(int32_t));
  cudaMemset(d_it, 0, ncols * sizeof(int32_t));
  cudaMemset(d_fail, 0, kFailSlots * sizeof(int32_t));
  c->v.col_off = d_off;
  c->v.perm = d_perm;
  c->v.col_dz = d_dz;
  c->v.ref = d_ref;
  c->v.tiles = d_tiles;
  c->v.ntiles = (int32_t)c->ntiles;
  c->v.fac = d_fac;
  c->v.scr = nullptr;
  c->v.fac_status = d_fs;
  c->v.col_status = d_cs;
  c->v.col_iters = d_it;
  c->v.fail_count = d_fail;
  c->v.tile_next = c->d_tile_next;
  hevi::launch_setup_ref(c->v, d_order, d_nez, c->stream);
  c->launches += 1;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    hevi_destroy(c);
    return HEVI_ERR_CUDA;
  }
  *out = c;
  return HEVI_OK;
}

void hevi_destroy(hevi_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  fold_profile(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (int N = 0; N <= kMaxOrder; ++N) {
    if (c->aux[N]) {
      cudaStreamSynchronize(c->aux[N]);
      cudaStreamDestroy(c->aux[N]);
    }
    if (c->join_ev[N]) cudaEventDestroy(c->join_ev[N]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_fail) cudaFreeHost(c->h_fail);
  delete c;
}

int64_t hevi_estimate_bytes(const hevi_column_grid* grid, hevi_precision precision, int32_t kind,
                            int32_t stages) {
  if (!grid || grid->ncols <= 0 || !grid->classes || grid->nclasses <= 0 ||
      grid->ncols > (int64_t)INT32_MAX || (grid->nclasses > 1 && !grid->class_of_col))
    return -1;
  if (precision != HEVI_FP64 && precision != HEVI_FP32_IR) return -1;
  if (kind < 0 || kind > 2 || (kind > 0 && (stages < 2 || stages > 8))) return -1;
  std::vector<int64_t> count(grid->nclasses, 0);
  for (int c = 0; c < grid->nclasses; ++c) {
    const hevi_size_class& k = grid->classes[c];
    if (k.order < 1 || k.order > kMaxOrder || k.nez < 1 || k.nez > 4096) return -1;
  }
  for (int64_t i = 0; i < grid->ncols; ++i) {
    const int32_t k = grid->class_of_col ? grid->class_of_col[i] : 0;
    if (k < 0 || k >= grid->nclasses) return -1;
    count[k] += 1;
  }
  // the same sizes as hevi_setup: tiles of up to 32 columns of one class
  const int64_t ncols = grid->ncols;
  int64_t state = 0, ntiles = 0, fac = 0, scr = 0, ysc = 0;
  bool has_order[kMaxOrder + 1] = {false};
  for (int c = 0; c < grid->nclasses; ++c) {
    if (!count[c]) continue;
    const int N = grid->classes[c].order;
    has_order[N] = true;
    const int64_t n = 3 * ((int64_t)grid->classes[c].nez * N + 1);
    const int64_t tiles = (count[c] + kTile - 1) / kTile;
    state += n * count[c];
    ntiles += tiles;
    ysc += tiles * (2 * n + (n + 3 * (N + 1) + 3) / 4 * 4 + 4 * n) * kTile;
    fac += tiles * n * rl_of(N, precision) * kTile;
    scr += tiles * n * ur2_of(N) * kTile;
  }
  const int64_t esz = precision == HEVI_FP64 ? 8 : 4;
  int64_t b = (ncols + 1) * 8 + 3 * ncols * 4 + ncols * 8 + 2 * state * 8 +
              ntiles * (int64_t)sizeof(TileDesc) + (state / 3) * 8 +
              (precision == HEVI_FP32_IR ? ysc * 4 : 0) +
              3 * ncols * 4 + kFailSlots * 4 + 4 +
              fac * esz;
  // the single-launch solve's tile list when several orders are present
  int norders = 0;
  for (int N = 1; N <= kMaxOrder; ++N) norders += has_order[N] ? 1 : 0;
  if (norders > 1) b += ntiles * 4;
  if (kind == 1) b += (2 * (int64_t)stages + 1) * state * 8;
  // NHEVI step: stage work vectors, then the Newton sequence's workspace
  if (kind == 2)
    b += ((int64_t)stages + 2) * state * 8 + 3 * state * 8 + ncols * 8 + 5 * ncols * 4 +
         (kNewtonMaxIter + 1) * 4 + kFailSlots * 4;
  (void)scr;
  return b;
}

hevi_status hevi_set_stream(hevi_ctx* c, void* stream) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return HEVI_OK;
}

int64_t hevi_state_size(const hevi_ctx* c) { return c ? c->state_size : -1; }

int64_t hevi_column_offset(const hevi_ctx* c, int64_t i) {
  if (!c || i < 0 || i > c->ncols) return -1;
  return c->h_off[i];
}

int64_t hevi_device_bytes(const hevi_ctx* c) { return c ? c->dev_bytes : -1; }

int64_t hevi_launch_count(const hevi_ctx* c) { return c ? c->launches : -1; }

hevi_status hevi_reference_state(hevi_ctx* c, double* q) {
  if (!c || !q) return HEVI_ERR_INVALID_ARG;
  hevi::launch_reference_state(c->v, q, c->stream);
  return check_launch(c, 1);
}

hevi_status hevi_reference_columns(hevi_ctx* c, int64_t first, int64_t count, double* q) {
  if (!c || !q || first < 0 || count < 0 || first + count > c->ncols) return HEVI_ERR_INVALID_ARG;
  if (count == 0) return HEVI_OK;
  hevi::launch_reference_state(c->v, q, c->stream, first, count);
  return check_launch(c, 1);
}

hevi_status hevi_set_column_tops(hevi_ctx* c, int64_t first, int64_t count, const double* z_top) {
  if (!c || first < 0 || count < 0 || first + count > c->ncols || (count > 0 && !z_top))
    return HEVI_ERR_INVALID_ARG;
  if (count == 0) return HEVI_OK;
  std::vector<double> dz(count);
  for (int64_t i = 0; i < count; ++i) {
    const double zt = z_top[i];
    if (!(zt > 0.0) || !std::isfinite(zt)) return HEVI_ERR_INVALID_ARG;
    dz[i] = zt / c->h_col_nez[first + i];
  }
  // from pageable memory: the copy is staged before the call returns
  if (cudaMemcpyAsync(const_cast<double*>(c->v.col_dz) + first, dz.data(), count * sizeof(double),
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return HEVI_ERR_CUDA;
  }
  hevi::launch_setup_ref(c->v, c->d_col_order, c->d_col_nez, c->stream, first, count);
  c->factored = false;
  return check_launch(c, 1);
}

hevi_status hevi_set_equation_set(hevi_ctx* c, int32_t set) {
  if (!c || (set != HEVI_SET_2C && set != HEVI_SET_3C && set != HEVI_SET_2NC))
    return HEVI_ERR_INVALID_ARG;
  if (set == HEVI_SET_2NC) {
    if (c->prec != HEVI_FP64) return HEVI_ERR_INVALID_ARG;
    if (!c->v.lin2) {
      const hevi_status s = c->alloc(&c->v.lin2, 2 * (size_t)c->state_size);
      if (s != HEVI_OK) return s;
    }
  }
  c->v.ph.eqset = set;
  hevi::launch_setup_ref(c->v, c->d_col_order, c->d_col_nez, c->stream);
  c->factored = false;
  return check_launch(c, 1);
}

hevi_status hevi_set_fused_stages(hevi_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return HEVI_ERR_INVALID_ARG;
  c->fuse_stages = on != 0;
  return HEVI_OK;
}

hevi_status hevi_set_newton_host_check(hevi_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return HEVI_ERR_INVALID_ARG;
  c->newton_host_check = on != 0;
  return HEVI_OK;
}

hevi_status hevi_set_refinement(hevi_ctx* c, double tol, int32_t max_sweeps) {
  if (!c || !(tol > 0.0) || max_sweeps < 1 || max_sweeps > 100) return HEVI_ERR_INVALID_ARG;
  c->ir_tol = tol;
  c->ir_max = max_sweeps;
  return HEVI_OK;
}

hevi_status hevi_set_solve_warps(hevi_ctx* c, int32_t warps_per_sm) {
  if (!c || warps_per_sm < 0 || warps_per_sm > 32) return HEVI_ERR_INVALID_ARG;
  c->v.solve_wps = warps_per_sm;
  return HEVI_OK;
}

hevi_status hevi_test_drop_record_copy(hevi_ctx* c, int32_t step) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  c->v.drop_copy = step >= 0 ? step + 1 : 0;
  return HEVI_OK;
}

hevi_status hevi_factor(hevi_ctx* c, double gamma_dt, const double* lin_state) {
  if (!c || !(gamma_dt >= 0.0) || !std::isfinite(gamma_dt)) return HEVI_ERR_INVALID_ARG;
  {
    Scope sc(c, kFactor);
    for_orders(c, c->v, [&](const DevView& v, int N, int ylen, cudaStream_t sk) {
      hevi::launch_factor(v, N, c->prec, gamma_dt, lin_state, ylen, sk);
    });
  }
  c->lam = gamma_dt;
  c->factored = true;
  return check_launch(c);
}

hevi_status hevi_stage_solve_async(hevi_ctx* c, const double* rhs, double* x) {
  if (!c || !rhs || !x || rhs == x || !c->factored) return HEVI_ERR_INVALID_ARG;
  {
    Scope sc(c, kSolve);
    stage_solve_all(c, c->v, c->lam, rhs, x);
  }
  return check_launch(c);
}

hevi_status hevi_autotune_solve(hevi_ctx* c, const double* rhs, double* x, int32_t reps,
                                int32_t* warps_per_sm, double* ms, double* ms_default) {
  if (!c || !rhs || !x || rhs == x || !c->factored || c->prec != HEVI_FP32_IR || reps < 1 ||
      reps > 1000)
    return HEVI_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &cap);
  if (cap != cudaStreamCaptureStatusNone) return HEVI_ERR_INVALID_ARG;
  cudaEvent_t e0 = get_event(c), e1 = get_event(c);
  const int32_t saved = c->v.solve_wps;
  // mean time of one solve with the given warps per SM (0: default shape)
  auto time_at = [&](int32_t w, float* t) {
    c->v.solve_wps = w;
    stage_solve_all(c, c->v, c->lam, rhs, x);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps; ++r) stage_solve_all(c, c->v, c->lam, rhs, x);
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(t, e0, e1) != cudaSuccess)
      return false;
    *t /= (float)reps;
    return true;
  };
  reset_fail(c);
  bool ok = true;
  float t_default = 0.f, best = 0.f;
  int32_t best_w = 0;
  ok = time_at(0, &t_default);
  const int maxw = hevi::solve_np_max_warps_per_sm(c->norders > 1 ? 0 : c->max_order, c->max_order);
  for (int32_t w = 1; ok && w <= maxw; ++w) {
    float t = 0.f;
    ok = time_at(w, &t);
    if (ok && (best_w == 0 || t < 0.99f * best)) {
      best = t;
      best_w = w;
    }
  }
  c->ev_pool.push_back(e0);
  c->ev_pool.push_back(e1);
  if (!ok || cudaGetLastError() != cudaSuccess) {
    c->v.solve_wps = saved;
    return HEVI_ERR_CUDA;
  }
  c->v.solve_wps = best_w;
  if (warps_per_sm) *warps_per_sm = best_w;
  if (ms) *ms = best;
  if (ms_default) *ms_default = t_default;
  return HEVI_OK;
}

hevi_status hevi_stage_solve(hevi_ctx* c, const double* rhs, double* x) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  reset_fail(c);
  hevi_status s = hevi_stage_solve_async(c, rhs, x);
  if (s != HEVI_OK) return s;
  return wait_status(c);
}

hevi_status hevi_newton_solve_async(hevi_ctx* c, double gamma_dt, double* state, const double* R,
                                    double rtol, int32_t max_iter) {
  if (!c || !state || !R || state == R || !(gamma_dt >= 0.0) || !(rtol >= 0.0) || max_iter < 0 ||
      max_iter > 1000)
    return HEVI_ERR_INVALID_ARG;
  return newton_sequence(c, gamma_dt, state, R, rtol, max_iter, false);
}

hevi_status hevi_newton_solve(hevi_ctx* c, double gamma_dt, double* state, const double* R,
                              double rtol, int32_t max_iter) {
  if (!c || !state || !R || state == R || !(gamma_dt >= 0.0) || !(rtol >= 0.0) || max_iter < 0 ||
      max_iter > 1000)
    return HEVI_ERR_INVALID_ARG;
  reset_fail(c);
  hevi_status s = newton_sequence(c, gamma_dt, state, R, rtol, max_iter, true);
  if (s != HEVI_OK) return s;
  return wait_status(c);
}

hevi_status hevi_newton_gmres_solve_async(hevi_ctx* c, double gamma_dt, double* state,
                                          const double* R, double eps, double rtol, double gtol,
                                          int32_t max_newton, int32_t kmax, int32_t* krylov) {
  if (c && c->v.ph.eqset != 0) return HEVI_ERR_INVALID_ARG;  // the JFNK path is set 2C only
  if (!c || !state || !R || state == R || !(gamma_dt >= 0.0) || !(eps > 0.0) || !(rtol >= 0.0) ||
      !(gtol > 0.0) || max_newton < 0 || max_newton > 1000 || kmax < 0)
    return HEVI_ERR_INVALID_ARG;
  const int64_t nmax = max_unknowns(c);
  if (kmax == 0 || kmax > nmax) kmax = (int32_t)nmax;  // GMRES is exact after n iterations
  hevi_status s = ensure_gmres(c, kmax);
  if (s != HEVI_OK) return s;
  hevi::GmArgs a;
  a.lam = gamma_dt;
  a.eps = eps;
  a.rtol = rtol;
  a.gtol = gtol;
  a.max_newton = max_newton;
  a.kmax = kmax;
  a.nmax = (int)nmax;
  a.kstride = (int64_t)(kmax + 1) * nmax * kTile;
  a.hstride = (int64_t)kmax * (kmax + 3) / 2 * kTile;
  a.astride = (4 * (int64_t)kmax + 1) * kTile;
  a.q = state;
  a.R = R;
  a.F = c->gm_vec;
  a.Qp = c->gm_vec + c->state_size;
  a.Vp = c->gm_vec + 2 * c->state_size;
  a.Kb = c->gm_tile;
  a.Hb = c->gm_tile + a.kstride * c->ntiles;
  a.Ab = a.Hb + a.hstride * c->ntiles;
  a.kits = krylov;
  {
    Scope sc(c, kNewton);
    for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
      hevi::launch_newton_gmres(v, N, a, sk);
    });
  }
  return check_launch(c);
}

hevi_status hevi_newton_gmres_solve(hevi_ctx* c, double gamma_dt, double* state, const double* R,
                                    double eps, double rtol, double gtol, int32_t max_newton,
                                    int32_t kmax, int32_t* krylov) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  reset_fail(c);
  hevi_status s = hevi_newton_gmres_solve_async(c, gamma_dt, state, R, eps, rtol, gtol,
                                                max_newton, kmax, krylov);
  if (s != HEVI_OK) return s;
  return wait_status(c);
}

hevi_status hevi_apply_Lv(hevi_ctx* c, const double* x, double* y, int nonlinear) {
  if (!c || !x || !y || x == y) return HEVI_ERR_INVALID_ARG;
  if (!nonlinear && !c->factored) return HEVI_ERR_INVALID_ARG;
  {
    Scope sc(c, kApply);
    for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
      hevi::launch_apply(v, N, x, y, nonlinear, sk);
    });
  }
  return check_launch(c);
}

hevi_status hevi_column_status(hevi_ctx* c, int32_t* status, int32_t* iters) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  if (status &&
      cudaMemcpyAsync(status, c->v.col_status, c->ncols * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                      c->stream) != cudaSuccess)
    return HEVI_ERR_CUDA;
  if (iters &&
      cudaMemcpyAsync(iters, c->v.col_iters, c->ncols * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                      c->stream) != cudaSuccess)
    return HEVI_ERR_CUDA;
  return HEVI_OK;
}

hevi_status hevi_sync(hevi_ctx* c) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  hevi_status s = wait_status(c);
  reset_fail(c);
  cudaStreamSynchronize(c->stream);
  return s;
}

hevi_status hevi_profile(hevi_ctx* c, int32_t enable) {
  if (!c) return HEVI_ERR_INVALID_ARG;
  fold_profile(c);
  if (enable) {
    for (int k = 0; k < kNumKinds; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_n[k] = 0;
    }
  }
  c->prof = enable != 0;
  return HEVI_OK;
}

int32_t hevi_profile_kinds(void) { return kNumKinds; }

const char* hevi_profile_kind_name(int32_t kind) {
  return (kind >= 0 && kind < kNumKinds) ? kKindNames[kind] : "";
}

hevi_status hevi_profile_read(hevi_ctx* c, int32_t kind, double* total_ms, int64_t* launches) {
  if (!c || kind < 0 || kind >= kNumKinds || !total_ms || !launches) return HEVI_ERR_INVALID_ARG;
  fold_profile(c);
  *total_ms = c->prof_ms[kind];
  *launches = c->prof_n[kind];
  return HEVI_OK;
}

static bool tableau_ok(int32_t s, const double* A, const double* At, const double* b) {
  if (s < 2 || s > 8 || !A || !At || !b) return false;
  if (At[0] != 0.0) return false;
  const double g = At[1 * s + 1];
  if (!(g > 0.0)) return false;
  for (int i = 1; i < s; ++i)
    if (At[i * s + i] != g) return false;
  for (int i = 0; i < s; ++i)
    for (int j = i; j < s; ++j)
      if (A[i * s + j] != 0.0 || (j > i && At[i * s + j] != 0.0)) return false;
  return true;
}

hevi_status hevi_lhevi_step(hevi_ctx* c, int32_t s, const double* A, const double* At,
                            const double* b, double dt, const double* q_in, const double* H,
                            double* q_out, int32_t lin_about_rest) {
  if (!c || !q_in || !H || !q_out || q_in == q_out || !(dt > 0.0) || !tableau_ok(s, A, At, b) ||
      lin_about_rest < 0 || lin_about_rest > 2)
    return HEVI_ERR_INVALID_ARG;
  // ARK form of LHEVI (Sec. 4.3, Eq. lhevi-ark-final-3), S(Q) = H + V(Q),
  // w_ij = (at_ij - a_ij) / gamma:
  //   q_hat = q^n + dt sum_j a_ij S_j + sum_j w_ij Q_j;  (I - gamma dt L) q_tt = q_hat;
  //   Q_i = q_tt - sum_j w_ij Q_j;  q^{n+1} = q^n + dt sum_i b_i S_i.
  // The solve is for q_tt, a difference of states (sum_j w_ij = -1 when the
  // two tableaux share their stage times), so the refinement tolerance
  // applies to the stage increment.
  hevi_status st = ensure_work(c, 2 * s + 1);
  if (st != HEVI_OK) return st;
  const int64_t n = c->state_size;
  double* Qb = c->work;            // stage values Q_1 .. Q_{s-1} (Q_0 = q_in)
  double* S = c->work + s * n;     // s vectors
  double* rhs = c->work + 2 * s * n;
  const double gam = At[1 * s + 1], lam = gam * dt;
  auto Qp = [&](int j) -> const double* { return j == 0 ? q_in : Qb + j * n; };
  if (lin_about_rest == 2) {
    // Jacobian kept from the last factorisation (update interval > 1 step)
    if (!c->factored || c->lam != lam) return HEVI_ERR_INVALID_ARG;
  } else if ((st = hevi_factor(c, lam, lin_about_rest ? nullptr : q_in))) {
    return st;
  }
  if (c->fuse_stages && c->prec == HEVI_FP32_IR && c->v.ph.eqset == 0 &&
      2 * s <= hevi::kFuseR) {
    // The same sequence with every stage combination folded into the
    // tendency pass of the stage before it: the pass of stage i forms Q_i
    // from the solve's q_tt, then S_i, then the next stage's right-hand side
    // (the last stage's pass: q^{n+1}).  Same operations in the same order,
    // so the same bits; no combination launches.  Set 2C only: set 3C's
    // tendency pass has less room for the extra loads (measured: 0.48 ms per
    // fused pass against 0.29 ms plus the separate combinations' 0.15 ms).
    for (int i = 0; i < s; ++i) {
      hevi::StageFuse fz;
      double* Qi = Qb + i * n;
      if (i > 0) {  // Q_i = q_tt - sum_j w_ij Q_j
        fz.qtt = Qi;
        for (int j = 0; j < i; ++j) {
          fz.q[fz.nq] = Qp(j);
          fz.cq[fz.nq++] = -(At[i * s + j] - A[i * s + j]) / gam;
        }
      }
      const bool last = i == s - 1;
      fz.rbase = q_in;
      if (!last) {  // rhs of stage i + 1 (its terms j < i from memory, then S_i, Q_i)
        fz.qout = i > 0 ? Qi : nullptr;
        fz.rout = rhs;
        for (int j = 0; j < i; ++j) {
          fz.r[fz.nr] = S + j * n;
          fz.cr[fz.nr++] = dt * A[(i + 1) * s + j];
          fz.r[fz.nr] = Qp(j);
          fz.cr[fz.nr++] = (At[(i + 1) * s + j] - A[(i + 1) * s + j]) / gam;
        }
        fz.has_s = fz.has_q = 1;
        fz.cs = dt * A[(i + 1) * s + i];
        fz.cqs = (At[(i + 1) * s + i] - A[(i + 1) * s + i]) / gam;
      } else {  // q^{n+1} = q^n + dt sum_j b_j S_j
        fz.rout = q_out;
        for (int j = 0; j < i; ++j) {
          fz.r[fz.nr] = S + j * n;
          fz.cr[fz.nr++] = dt * b[j];
        }
        fz.has_s = 1;
        fz.cs = dt * b[i];
      }
      {
        Scope sc(c, kApply);
        for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
          apply_rhs(c, v, N, i == 0 ? q_in : nullptr, H, last ? nullptr : S + i * n, sk, &fz);
        });
      }
      if (!last) {
        Scope sc(c, kSolve);
        stage_solve_all(c, c->v, lam, rhs, Qb + (i + 1) * n);
      }
    }
    return cudaGetLastError() == cudaSuccess ? HEVI_OK : HEVI_ERR_CUDA;
  }
  {
    Scope sc(c, kApply);
    for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
      apply_rhs(c, v, N, q_in, H, S, sk);
    });
  }
  for (int i = 1; i < s; ++i) {
    const double* vec[16];
    double coef[16];
    int nt = 0;
    for (int j = 0; j < i; ++j) {
      vec[nt] = S + j * n;
      coef[nt++] = dt * A[i * s + j];
      vec[nt] = Qp(j);
      coef[nt++] = (At[i * s + j] - A[i * s + j]) / gam;
    }
    double* Qi = Qb + i * n;
    {
      Scope sc(c, kCombine);
      hevi::launch_combine(n, q_in, nt, vec, coef, rhs, c->stream);
    }
    {
      Scope sc(c, kSolve);
      stage_solve_all(c, c->v, lam, rhs, Qi);
    }
    nt = 0;
    for (int j = 0; j < i; ++j) {
      vec[nt] = Qp(j);
      coef[nt++] = -(At[i * s + j] - A[i * s + j]) / gam;
    }
    {
      Scope sc(c, kCombine);
      hevi::launch_combine(n, Qi, nt, vec, coef, Qi, c->stream);
    }
    {
      Scope sc(c, kApply);
      for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
        apply_rhs(c, v, N, Qi, H, S + i * n, sk);
      });
    }
    c->launches += 2;  // the two combines
  }
  {
    const double* vec[16];
    double coef[16];
    int nt = 0;
    for (int i = 0; i < s; ++i) {
      vec[nt] = S + i * n;
      coef[nt++] = dt * b[i];
    }
    {
      Scope sc(c, kCombine);
      hevi::launch_combine(n, q_in, nt, vec, coef, q_out, c->stream);
    }
    c->launches += 1;
  }
  return cudaGetLastError() == cudaSuccess ? HEVI_OK : HEVI_ERR_CUDA;
}

hevi_status hevi_nhevi_step(hevi_ctx* c, int32_t s, const double* A, const double* At,
                            const double* b, double dt, const double* q_in, const double* H,
                            double* q_out, double rtol, int32_t max_iter) {
  if (!c || !q_in || !H || !q_out || q_in == q_out || !(dt > 0.0) || !tableau_ok(s, A, At, b))
    return HEVI_ERR_INVALID_ARG;
  hevi_status st = ensure_work(c, s + 2);
  if (st != HEVI_OK) return st;
  if ((st = ensure_newton(c))) return st;
  const int64_t n = c->state_size;
  double* VQ = c->work;  // s vectors
  double* R = c->work + s * n;
  double* Q = R + n;
  const double lam = At[1 * s + 1] * dt;
  {
    Scope sc(c, kApply);
    for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
      hevi::launch_apply(v, N, q_in, VQ, 1, sk);
    });
  }
  cudaMemcpyAsync(Q, q_in, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  for (int i = 1; i < s; ++i) {
    const double* vec[16];
    double coef[16];
    int nt = 0;
    double ah = 0.0;
    for (int j = 0; j < i; ++j) {
      ah += A[i * s + j];
      vec[nt] = VQ + j * n;
      coef[nt++] = dt * At[i * s + j];
    }
    vec[nt] = H;
    coef[nt++] = dt * ah;
    {
      Scope sc(c, kCombine);
      hevi::launch_combine(n, q_in, nt, vec, coef, R, c->stream);
    }
    if ((st = newton_sequence(c, lam, Q, R, rtol, max_iter, c->newton_host_check))) return st;
    {
      Scope sc(c, kApply);
      for_orders(c, c->v, [&](const DevView& v, int N, int, cudaStream_t sk) {
        hevi::launch_apply(v, N, Q, VQ + i * n, 1, sk);
      });
    }
    c->launches += 1;  // the combine
  }
  {
    const double* vec[16];
    double coef[16];
    int nt = 0;
    double bs = 0.0;
    for (int i = 0; i < s; ++i) {
      bs += b[i];
      vec[nt] = VQ + i * n;
      coef[nt++] = dt * b[i];
    }
    vec[nt] = H;
    coef[nt++] = dt * bs;
    {
      Scope sc(c, kCombine);
      hevi::launch_combine(n, q_in, nt, vec, coef, q_out, c->stream);
    }
    c->launches += 1;
  }
  return cudaGetLastError() == cudaSuccess ? HEVI_OK : HEVI_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Named ESDIRK tableaux (Sec. 6).  Coefficients of the cited constructions,
// stored as ratios of integers.
// ---------------------------------------------------------------------------
namespace {
struct Ratio {
  double p, q;
};
double r(const Ratio& x) { return x.p / x.q; }
}  // namespace

extern "C" hevi_status hevi_tableau(const char* name, int32_t* s_out, double* A, double* At,
                                    double* b) {
  if (!name || !s_out || !A || !At || !b) return HEVI_ERR_INVALID_ARG;
  std::string nm(name);
  int s = 0;
  std::fill(A, A + 64, 0.0);
  std::fill(At, At + 64, 0.0);
  std::fill(b, b + 8, 0.0);
  auto a = [&](double* M, int i, int j) -> double& { return M[i * s + j]; };
  if (nm == "ARK2") {
    // ARK(2,3,2)b: gamma = 1 - 1/sqrt(2), a32 = 1/2 (Sec. 4.1)
    s = 3;
    const double g = 1.0 - 1.0 / std::sqrt(2.0), d = 1.0 / (2.0 * std::sqrt(2.0));
    a(A, 1, 0) = 2.0 * g;
    a(A, 2, 0) = 0.5;
    a(A, 2, 1) = 0.5;
    a(At, 1, 0) = g; a(At, 1, 1) = g;
    a(At, 2, 0) = d; a(At, 2, 1) = d; a(At, 2, 2) = g;
    b[0] = d; b[1] = d; b[2] = g;
  } else if (nm == "ARK3") {
    s = 4;
    const double g = r({1767732205903.0, 4055673282236.0});
    const double b0 = r({1471266399579.0, 7840856788654.0});
    const double b1 = r({-4482444167858.0, 7529755066697.0});
    const double b2 = r({11266239266428.0, 11593286722821.0});
    a(At, 1, 0) = g; a(At, 1, 1) = g;
    a(At, 2, 0) = r({2746238789719.0, 10658868560708.0});
    a(At, 2, 1) = r({-640167445237.0, 6845629431997.0});
    a(At, 2, 2) = g;
    a(At, 3, 0) = b0; a(At, 3, 1) = b1; a(At, 3, 2) = b2; a(At, 3, 3) = g;
    a(A, 1, 0) = r({1767732205903.0, 2027836641118.0});
    a(A, 2, 0) = r({5535828885825.0, 10492691773637.0});
    a(A, 2, 1) = r({788022342437.0, 10882634858940.0});
    a(A, 3, 0) = r({6485989280629.0, 16251701735622.0});
    a(A, 3, 1) = r({-4246266847089.0, 9704473918619.0});
    a(A, 3, 2) = r({10755448449292.0, 10357097424841.0});
    b[0] = b0; b[1] = b1; b[2] = b2; b[3] = g;
  } else if (nm == "ARK4") {
    s = 6;
    const double g = 0.25;
    const double bb[6] = {r({82889.0, 524892.0}), 0.0, r({15625.0, 83664.0}),
                          r({69875.0, 102672.0}), r({-2260.0, 8211.0}), g};
    a(At, 1, 0) = g; a(At, 1, 1) = g;
    a(At, 2, 0) = r({8611.0, 62500.0}); a(At, 2, 1) = r({-1743.0, 31250.0}); a(At, 2, 2) = g;
    a(At, 3, 0) = r({5012029.0, 34652500.0}); a(At, 3, 1) = r({-654441.0, 2922500.0});
    a(At, 3, 2) = r({174375.0, 388108.0}); a(At, 3, 3) = g;
    a(At, 4, 0) = r({15267082809.0, 155376265600.0}); a(At, 4, 1) = r({-71443401.0, 120774400.0});
    a(At, 4, 2) = r({730878875.0, 902184768.0}); a(At, 4, 3) = r({2285395.0, 8070912.0});
    a(At, 4, 4) = g;
    for (int j = 0; j < 6; ++j) a(At, 5, j) = bb[j];
    a(A, 1, 0) = 0.5;
    a(A, 2, 0) = r({13861.0, 62500.0}); a(A, 2, 1) = r({6889.0, 62500.0});
    a(A, 3, 0) = r({-116923316275.0, 2393684061468.0});
    a(A, 3, 1) = r({-2731218467317.0, 15368042101831.0});
    a(A, 3, 2) = r({9408046702089.0, 11113171139209.0});
    a(A, 4, 0) = r({-451086348788.0, 2902428689909.0});
    a(A, 4, 1) = r({-2682348792572.0, 7519795681897.0});
    a(A, 4, 2) = r({12662868775082.0, 11960479115383.0});
    a(A, 4, 3) = r({3355817975965.0, 11060851509271.0});
    a(A, 5, 0) = r({647845179188.0, 3216320057751.0});
    a(A, 5, 1) = r({73281519250.0, 8382639484533.0});
    a(A, 5, 2) = r({552539513391.0, 3454668386233.0});
    a(A, 5, 3) = r({3354512671639.0, 8306763924573.0});
    a(A, 5, 4) = r({4040.0, 17871.0});
    for (int j = 0; j < 6; ++j) b[j] = bb[j];
  } else if (nm == "ARS3") {
    // ARK(3,4,3) of Ascher, Ruuth & Spiteri: gamma solves 6g^3 - 18g^2 + 9g - 1
    // = 0 in (1/6, 1/2); the free explicit coefficients a42 = a43; a31, a32
    // from the construction's closed forms; implicit first column zero
    s = 4;
    double g = 0.4358665215;
    for (int it = 0; it < 4; ++it)
      g -= (6.0 * g * g * g - 18.0 * g * g + 9.0 * g - 1.0) / (18.0 * g * g - 36.0 * g + 9.0);
    const double e42 = 0.5529291480359398, e43 = e42, g2 = g * g;
    const double b1 = -1.5 * g2 + 4.0 * g - 0.25, b2 = 1.5 * g2 - 5.0 * g + 1.25;
    a(A, 1, 0) = g;
    a(A, 2, 0) = (1.0 - 4.5 * g + 1.5 * g2) * e42 + (2.75 - 10.5 * g + 3.75 * g2) * e43 - 3.5 +
                 13.0 * g - 4.5 * g2;
    a(A, 2, 1) = (-1.0 + 4.5 * g - 1.5 * g2) * e42 + (-2.75 + 10.5 * g - 3.75 * g2) * e43 + 4.0 -
                 12.5 * g + 4.5 * g2;
    a(A, 3, 0) = 1.0 - e42 - e43;
    a(A, 3, 1) = e42;
    a(A, 3, 2) = e43;
    a(At, 1, 1) = g;
    a(At, 2, 1) = 0.5 * (1.0 - g); a(At, 2, 2) = g;
    a(At, 3, 1) = b1; a(At, 3, 2) = b2; a(At, 3, 3) = g;
    b[0] = 0.0; b[1] = b1; b[2] = b2; b[3] = g;
  } else {
    return HEVI_ERR_INVALID_ARG;
  }
  *s_out = s;
  return HEVI_OK;
}

// ---------------------------------------------------------------------------
// Step loops captured into CUDA graphs.
// ---------------------------------------------------------------------------
struct hevi_graph {
  hevi_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches_per_replay = 0;
};

namespace {

// Capture nsteps calls of `step(q_in, q_out)` ping-ponging between q_a and
// q_b on a private stream, then instantiate.  The context's stream is swapped
// for the capture stream while capturing and restored afterwards.
template <class Step>
hevi_status capture_steps(hevi_ctx* c, double* q_a, double* q_b, int32_t nsteps, Step&& step,
                          hevi_graph** out) {
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return HEVI_ERR_CUDA;
  }
  // the capture must not start before earlier work on the caller's stream
  cudaStreamSynchronize(c->stream);
  cudaStream_t user = c->stream;
  c->stream = cap;
  const int64_t l0 = c->launches;
  hevi_status st = HEVI_OK;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    st = HEVI_ERR_CUDA;
  } else {
    for (int32_t k = 0; k < nsteps && st == HEVI_OK; ++k)
      st = (k % 2 == 0) ? step(q_a, q_b) : step(q_b, q_a);
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess && st == HEVI_OK) st = HEVI_ERR_CUDA;
  }
  c->stream = user;
  const int64_t per = c->launches - l0;
  c->launches = l0;
  cudaGraphExec_t exec = nullptr;
  if (st == HEVI_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) st = HEVI_ERR_CUDA;
  cudaStreamDestroy(cap);
  if (st != HEVI_OK) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  hevi_graph* g = new hevi_graph;
  g->ctx = c;
  g->graph = graph;
  g->exec = exec;
  g->launches_per_replay = per;
  *out = g;
  return HEVI_OK;
}

}  // namespace

extern "C" {

hevi_status hevi_lhevi_graph_create(hevi_ctx* c, int32_t s, const double* A, const double* At,
                                    const double* b, double dt, double* q_a, double* q_b,
                                    const double* H, int32_t nsteps, int32_t lin_about_rest,
                                    hevi_graph** out) {
  if (!out) return HEVI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!c || !q_a || !q_b || !H || q_a == q_b || nsteps < 1 || !(dt > 0.0) ||
      !tableau_ok(s, A, At, b))
    return HEVI_ERR_INVALID_ARG;
  hevi_status st = ensure_work(c, 2 * s + 1);  // no allocation inside the capture
  if (st != HEVI_OK) return st;
  std::vector<double> a(A, A + s * s), at(At, At + s * s), w(b, b + s);
  return capture_steps(c, q_a, q_b, nsteps, [&](const double* qi, double* qo) {
    return hevi_lhevi_step(c, s, a.data(), at.data(), w.data(), dt, qi, H, qo, lin_about_rest);
  }, out);
}

hevi_status hevi_nhevi_graph_create(hevi_ctx* c, int32_t s, const double* A, const double* At,
                                    const double* b, double dt, double* q_a, double* q_b,
                                    const double* H, int32_t nsteps, double rtol,
                                    int32_t max_iter, hevi_graph** out) {
  if (!out) return HEVI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!c || !q_a || !q_b || !H || q_a == q_b || nsteps < 1 || !(dt > 0.0) ||
      !tableau_ok(s, A, At, b) || !(rtol > 0.0) || max_iter < 1)
    return HEVI_ERR_INVALID_ARG;
  hevi_status st = ensure_work(c, s + 2);
  if (st != HEVI_OK) return st;
  if ((st = ensure_newton(c))) return st;
  std::vector<double> a(A, A + s * s), at(At, At + s * s), w(b, b + s);
  return capture_steps(c, q_a, q_b, nsteps, [&](const double* qi, double* qo) {
    return hevi_nhevi_step(c, s, a.data(), at.data(), w.data(), dt, qi, H, qo, rtol, max_iter);
  }, out);
}

hevi_status hevi_graph_launch(hevi_graph* g) {
  if (!g || !g->exec || !g->ctx) return HEVI_ERR_INVALID_ARG;
  if (cudaGraphLaunch(g->exec, g->ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return HEVI_ERR_CUDA;
  }
  g->ctx->launches += g->launches_per_replay;
  return HEVI_OK;
}

void hevi_graph_destroy(hevi_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

}  // extern "C"
