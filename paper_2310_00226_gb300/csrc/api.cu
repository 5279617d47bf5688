// C ABI of libsem3d: plan construction, workspace, and the orchestration of
// one solve (Section 2.4, Eq. 13) plus FP64 iterative refinement.
#include "sem3d_internal.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

using namespace sem3d;

namespace {

thread_local std::string g_last_error;

sem3d_status fail(sem3d_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

sem3d_status cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? SEM3D_ERR_OOM : SEM3D_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                                 \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr); \
  } while (0)

// Host-side cache of 1D axis data: identical (n, k, L) axes share one eigen-
// decomposition within a process.
std::mutex g_axis_mu;
std::map<std::tuple<int, int, double, int>, std::shared_ptr<const Axis1D>> g_axis_cache;

std::shared_ptr<const Axis1D> get_axis(int n, int k, double L, int bc) {
  const auto key = std::make_tuple(n, k, L, bc);
  {
    std::lock_guard<std::mutex> lk(g_axis_mu);
    auto it = g_axis_cache.find(key);
    if (it != g_axis_cache.end()) return it->second;
  }
  auto ax = std::make_shared<const Axis1D>(build_axis(n, k, L, bc));
  std::lock_guard<std::mutex> lk(g_axis_mu);
  g_axis_cache[key] = ax;
  return ax;
}

}  // namespace

struct sem3d_plan {
  int device = 0;
  int num_sms = 0;
  Geom g{};
  int k = 0;
  double L[3] = {0, 0, 0};
  std::shared_ptr<const Axis1D> ax[3];
  DevAxis dev[3];
  sem3d_precision prec = SEM3D_FP64;
  int sweeps = 1;
  int residual = SEM3D_RESIDUAL_MIXED;  // arithmetic of the refinement residuals (BF16X3 tier)
  // FP64-accurate residuals of the split tiers: 64-bit fixed point on the
  // integer pipe (fix_ok: Dirichlet, k <= 8) unless exact_kind says FP64
  FixCoef fix{};
  bool fix_ok = false;
  int exact_kind = SEM3D_EXACT_FIXED;
  int* d_fix = nullptr;  // 2 ints: max exponents of u and f
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  int* d_err = nullptr;
  F16State* d_f16 = nullptr;  // scale state of the F16X3 tier
  float div_bound = 1.f;      // 1 / (lambda_x,1 + lambda_y,1 + lambda_z,1 + c)
  std::vector<void*> owned;  // device allocations made at setup
  // launch accounting and optional per-kernel timing
  unsigned long long launches = 0;
  bool profiling = false;
  struct EvPair { int kind, sub, count; cudaEvent_t a, b; };
  std::vector<EvPair> pending;
  std::vector<cudaEvent_t> pool;
  // PCG: six FP64 n^3 vectors, scalars, an internal stream (allocated on first use)
  double* pcg_buf = nullptr;
  PcgScalars* pcg_sc = nullptr;
  double* ch_buf = nullptr;  // third phi buffer of sem3d_ch_run
  cudaStream_t pcg_stream = nullptr;
  // sem3d_solve_host: two device (f, u) pairs used in turn, copy streams and events.
  struct HostIo {
    double* f[2] = {nullptr, nullptr};
    double* u[2] = {nullptr, nullptr};
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t copied_in[2] = {nullptr, nullptr}, solved[2] = {nullptr, nullptr}, copied_out[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    long long calls = 0;
  } io;
  double prof_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long prof_n[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

template <class T>
sem3d_status dev_upload(sem3d_plan* p, T** dst, const T* src, size_t count) {
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, count * sizeof(T) + 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(setup)");
  p->owned.push_back(d);
  e = cudaMemcpy(d, src, count * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(setup)");
  *dst = static_cast<T*>(d);
  return SEM3D_OK;
}

// Split W (n x n row-major FP64) into bf16 hi + lo with row pitch Kp.
void split_matrix(const std::vector<double>& W, int n, int Kp, std::vector<__nv_bfloat16>& hi,
                  std::vector<__nv_bfloat16>& lo) {
  hi.assign((size_t)n * Kp, __float2bfloat16_rn(0.f));
  lo.assign((size_t)n * Kp, __float2bfloat16_rn(0.f));
  for (int o = 0; o < n; ++o)
    for (int t = 0; t < n; ++t) {
      const float x = (float)W[(size_t)o * n + t];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      hi[(size_t)o * Kp + t] = h;
      lo[(size_t)o * Kp + t] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Kernel classes for sem3d_profile_read; tensor-core launches are also
// counted per pass (x / y / z, and the last pass that writes FP64 u).
enum { K_TC = 0, K_F64 = 1, K_STENCIL = 2, K_SPLIT = 3, K_TC_X = 4, K_TC_Y = 5, K_TC_Z = 6, K_TC_F64OUT = 7, K_F32 = 8 };

cudaEvent_t take_event(sem3d_plan* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Bracket one launch site (`count` kernels) with events when profiling.
struct LaunchScope {
  sem3d_plan* p;
  int kind, sub, count;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  LaunchScope(sem3d_plan* p_, int kind_, int sub_, int count_, cudaStream_t s_)
      : p(p_), kind(kind_), sub(sub_), count(count_), s(s_) {
    if (p->profiling && (a = take_event(p)) != nullptr) cudaEventRecord(a, s);
  }
  void done() {
    p->launches += (unsigned long long)count;
    if (!a) return;
    cudaEvent_t b = take_event(p);
    if (!b) { p->pool.push_back(a); return; }
    cudaEventRecord(b, s);
    p->pending.push_back({kind, sub, count, a, b});
  }
};

#define LAUNCH_SUB(plan, kind, sub, count, stream, expr)  \
  do {                                                    \
    LaunchScope _ls((plan), (kind), (sub), (count), (stream)); \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);   \
    _ls.done();                                           \
  } while (0)
#define LAUNCH(plan, kind, count, stream, expr) LAUNCH_SUB(plan, kind, -1, count, stream, expr)

// Workspace layout per mode.
//   FP64   : two FP64 n^3 arrays (ping-pong) + one FP64 residual array.
//   FP32   : two FP32 n^3 arrays (ping-pong) + one FP64 residual array.
//   TF32   : two FP32 arrays holding the largest of the rotated layouts
//            (x, y, z)/(y, z, x)/(z, x, y), each at its padded pitch, + one
//            FP64 residual array.
//   BF16X3 / BF16 : three split arrays {hi, lo} of Px*ny*nz bf16 each (the
//            third serves the Cahn-Hilliard step), and the double-FP32
//            solution (two FP32 n^3 arrays) used between sweeps.
// Elements of the largest rotated TF32 layout: pitch pad16 of the fastest axis.
size_t tf32_elems(const Geom& g) {
  const size_t a = (size_t)pad16(g.nx) * g.ny * g.nz, b = (size_t)pad16(g.ny) * g.nz * g.nx,
               c = (size_t)pad16(g.nz) * g.nx * g.ny;
  return std::max(a, std::max(b, c));
}

size_t workspace_bytes(const sem3d_plan* p) {
  const size_t N = (size_t)p->g.nx * p->g.ny * p->g.nz;
  if (p->prec == SEM3D_FP64) return 3 * align256(N * sizeof(double));
  if (p->prec == SEM3D_FP32) return 2 * align256(N * sizeof(float)) + align256(N * sizeof(double));
  if (p->prec == SEM3D_TF32) return 2 * align256(tf32_elems(p->g) * sizeof(float)) + align256(N * sizeof(double));
  const size_t Ns = (size_t)p->g.Px * p->g.ny * p->g.nz;
  return 6 * align256(Ns * sizeof(__nv_bfloat16)) + 2 * align256(Ns * sizeof(float));
}

sem3d_status ensure_workspace(sem3d_plan* p) {
  const size_t need = workspace_bytes(p);
  if (p->ws && p->ws_bytes >= need) return SEM3D_OK;
  if (p->ws && !p->ws_owned) return fail(SEM3D_ERR_INVALID_ARG, "caller workspace smaller than sem3d_workspace_size");
  if (p->ws) { cudaFree(p->ws); p->ws = nullptr; p->ws_bytes = 0; }
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, need);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
  p->ws = d;
  p->ws_bytes = need;
  p->ws_owned = true;
  return SEM3D_OK;
}


// ---- FP64 path: one solve of (c + H (+) H (+) H) out = in, paper order z, y, x.
sem3d_status solve_once_f64(sem3d_plan* p, const double* in, double* out, bool accumulate, cudaStream_t s) {
  const size_t N = (size_t)p->g.nx * p->g.ny * p->g.nz;
  double* A = static_cast<double*>(p->ws);
  double* B = reinterpret_cast<double*>(static_cast<char*>(p->ws) + align256(N * sizeof(double)));
  const Geom& g = p->g;
  const DevAxis* d = p->dev;
  LAUNCH(p, K_F64, 1, s, launch_mode_product_f64(g, 2, d[2].Tinv, in, A, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH(p, K_F64, 1, s, launch_mode_product_f64(g, 1, d[1].Tinv, A, B, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH(p, K_F64, 1, s, launch_mode_product_f64(g, 0, d[0].Tinv, B, A, EPI_DIV, d[0].lam, d[1].lam, d[2].lam, s));
  LAUNCH(p, K_F64, 1, s, launch_mode_product_f64(g, 2, d[2].T, A, B, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH(p, K_F64, 1, s, launch_mode_product_f64(g, 1, d[1].T, B, A, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH(p, K_F64, 1, s, launch_mode_product_f64(g, 0, d[0].T, A, out, accumulate ? EPI_ACCUM : EPI_STORE, nullptr, nullptr,
                                   nullptr, s));
  return SEM3D_OK;
}

// ---- FP32 path: FP64 in -> FP64 out (store or accumulate), FP32 ping-pong.
sem3d_status solve_once_f32(sem3d_plan* p, const double* in, double* out, bool accumulate, cudaStream_t s) {
  const size_t N = (size_t)p->g.nx * p->g.ny * p->g.nz;
  float* A = static_cast<float*>(p->ws);
  float* B = reinterpret_cast<float*>(static_cast<char*>(p->ws) + align256(N * sizeof(float)));
  const Geom& g = p->g;
  const DevAxis* d = p->dev;
  const double *lx = d[0].lam, *ly = d[1].lam, *lz = d[2].lam;
  LAUNCH(p, K_F32, 1, s, launch_mode_product_f32(g, 2, d[2].Wf[0], in, true, A, false, EPI_STORE, lx, ly, lz, s));
  LAUNCH(p, K_F32, 1, s, launch_mode_product_f32(g, 1, d[1].Wf[0], A, false, B, false, EPI_STORE, lx, ly, lz, s));
  LAUNCH(p, K_F32, 1, s, launch_mode_product_f32(g, 0, d[0].Wf[0], B, false, A, false, EPI_DIV, lx, ly, lz, s));
  LAUNCH(p, K_F32, 1, s, launch_mode_product_f32(g, 0, d[0].Wf[1], A, false, B, false, EPI_STORE, lx, ly, lz, s));
  LAUNCH(p, K_F32, 1, s, launch_mode_product_f32(g, 1, d[1].Wf[1], B, false, A, false, EPI_STORE, lx, ly, lz, s));
  LAUNCH(p, K_F32, 1, s, launch_mode_product_f32(g, 2, d[2].Wf[1], A, false, out, true,
                                                 accumulate ? EPI_ACCUM : EPI_STORE, lx, ly, lz, s));
  return SEM3D_OK;
}

// ---- TF32 path (rotating layouts, see tf32_kernels.cu): FP64 in -> FP64 out
// (store or accumulate).  Passes x, y, z (forward, division fused into the z
// pass) then x, y, z (backward); the arrays alternate between A and B.
sem3d_status solve_once_tf32(sem3d_plan* p, const double* in, double* out, bool accumulate, cudaStream_t s) {
  const Geom& g = p->g;
  float* A = static_cast<float*>(p->ws);
  float* B = reinterpret_cast<float*>(static_cast<char*>(p->ws) + align256(tf32_elems(g) * sizeof(float)));
  const DevAxis* d = p->dev;
  const int n3[3] = {g.nx, g.ny, g.nz};
  const int P3[3] = {pad16(g.nx), pad16(g.ny), pad16(g.nz)};
  LAUNCH(p, K_SPLIT, 1, s, launch_to_tf32(g, in, A, s));
  float* bufs[2] = {A, B};
  for (int q = 0; q < 6; ++q) {
    const int ax = q % 3, a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;  // contracted axis, then the two row axes
    Tf32Pass t;
    t.nK = n3[ax]; t.d1 = n3[a1]; t.d2 = n3[a2]; t.P0 = P3[ax];
    t.in = bufs[q & 1];
    t.W = d[ax].Wt32[q < 3 ? 0 : 1];
    t.Wpitch = d[ax].Kp;
    if (q < 5) {
      t.out32 = bufs[(q + 1) & 1];
      t.P1 = P3[a1];
      t.epi = q == 2 ? EPI_DIV : EPI_STORE;
      // pass 3 rows (a, b), output c: lam_x[a] + lam_y[b] + lam_z[c]
      t.lam1 = d[0].lamf; t.lam2 = d[1].lamf; t.lam3 = d[2].lamf;
      t.c = (float)g.c;
    } else {
      t.out64 = out;
      t.P1 = g.nx;  // dense FP64 solution, x fastest
      t.epi = accumulate ? EPI_ACCUM : EPI_STORE;
    }
    const int sub = ax == 0 ? K_TC_X : ax == 1 ? K_TC_Y : K_TC_Z;
    LAUNCH_SUB(p, K_TC, q == 5 ? K_TC_F64OUT : sub, 1, s, launch_mode_product_tf32(t, p->d_err, p->num_sms, s));
  }
  return SEM3D_OK;
}

// ---- BF16x3 path: the split input is in buffer S0.  The last (z) pass
// writes the result with epilogue `epi_last` into out64 and/or the
// double-FP32 solution df.
sem3d_status solve_once_bf16x3(sem3d_plan* p, TcBuffers S0, TcBuffers S1, double* out64, int epi_last, DfBuffers df,
                               cudaStream_t s) {
  const int np = (p->prec == SEM3D_BF16) ? 1 : 3;
  const DfBuffers none{nullptr, nullptr};
  // F16X3: pass q reads scale slot q-1 and writes slot q (slot 0 = split input).
  const bool f16 = p->prec == SEM3D_F16X3;
  F16Pass fp[6];
  for (int q = 0; q < 6; ++q) fp[q] = F16Pass{p->d_f16, q, q + 1, q == 2 ? p->div_bound : 1.f};
  const F16Pass* F[6];
  for (int q = 0; q < 6; ++q) F[q] = f16 ? &fp[q] : nullptr;
  const Geom& g = p->g;
  const DevAxis* d = p->dev;
  const float *lx = d[0].lamf, *ly = d[1].lamf, *lz = d[2].lamf;
  const int sms = p->num_sms;
  int* e = p->d_err;
  // Forward: z, y, x with the division fused into the x pass (Eq. 13).
  LAUNCH_SUB(p, K_TC, K_TC_Z, 1, s, launch_mode_product_bf16x3(g, 2, d[2], 0, S0, S1, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np, F[0]));
  LAUNCH_SUB(p, K_TC, K_TC_Y, 1, s, launch_mode_product_bf16x3(g, 1, d[1], 0, S1, S0, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np, F[1]));
  LAUNCH_SUB(p, K_TC, K_TC_X, 1, s, launch_mode_product_bf16x3(g, 0, d[0], 0, S0, S1, nullptr, EPI_DIV, lx, ly, lz, e, sms, s, none, np, F[2]));
  // Backward: x, y, z.  The mode products commute, so the order is free; the
  // z pass goes last because its TMEM lanes run along the contiguous index,
  // which makes the read-modify-write of the solution coalesced.
  LAUNCH_SUB(p, K_TC, K_TC_X, 1, s, launch_mode_product_bf16x3(g, 0, d[0], 1, S1, S0, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np, F[3]));
  LAUNCH_SUB(p, K_TC, K_TC_Y, 1, s, launch_mode_product_bf16x3(g, 1, d[1], 1, S0, S1, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np, F[4]));
  LAUNCH_SUB(p, K_TC, K_TC_F64OUT, 1, s,
             launch_mode_product_bf16x3(g, 2, d[2], 1, S1, S0, out64, epi_last, lx, ly, lz, e, sms, s, df, np, F[5]));
  return SEM3D_OK;
}

sem3d_status run_solve(sem3d_plan* h, const double* f, double* u, cudaStream_t s);

}  // namespace

extern "C" {

const char* sem3d_last_error(void) { return g_last_error.c_str(); }

sem3d_status sem3d_setup(int nx, int ny, int nz, int k, double Lx, double Ly, double Lz, double c,
                         sem3d_handle* out) {
  return sem3d_setup_bc(nx, ny, nz, k, Lx, Ly, Lz, c, SEM3D_BC_DIRICHLET, out);
}

sem3d_status sem3d_setup_bc(int nx, int ny, int nz, int k, double Lx, double Ly, double Lz, double c, sem3d_bc bc,
                            sem3d_handle* out) {
  if (!out) return fail(SEM3D_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > 24) return fail(SEM3D_ERR_INVALID_ARG, "k must be in [1, 24]");
  if (bc != SEM3D_BC_DIRICHLET && bc != SEM3D_BC_NEUMANN) return fail(SEM3D_ERR_INVALID_ARG, "unknown boundary condition");
  const int n3[3] = {nx, ny, nz};
  const double L3[3] = {Lx, Ly, Lz};
  for (int a = 0; a < 3; ++a) {
    if (bc == SEM3D_BC_DIRICHLET && (n3[a] < 1 || (n3[a] + 1) % k != 0))
      return fail(SEM3D_ERR_INVALID_ARG, "Dirichlet: each n must be >= 1 with (n+1) % k == 0");
    if (bc == SEM3D_BC_NEUMANN && (n3[a] < k + 1 || (n3[a] - 1) % k != 0))
      return fail(SEM3D_ERR_INVALID_ARG, "Neumann: each n must be > k with (n-1) % k == 0");
    if (!(L3[a] > 0.0) || !std::isfinite(L3[a])) return fail(SEM3D_ERR_INVALID_ARG, "box lengths must be > 0");
  }
  if ((double)nx * ny * nz >= 1099511627776.0) return fail(SEM3D_ERR_INVALID_ARG, "grid too large");
  if (!std::isfinite(c)) return fail(SEM3D_ERR_INVALID_ARG, "c must be finite");
  // With Neumann data the constant is in the kernel of -Lap (lambda = 0 on every axis).
  if (bc == SEM3D_BC_NEUMANN && !(c > 0.0)) return fail(SEM3D_ERR_INVALID_ARG, "Neumann: c must be > 0");
  std::unique_ptr<sem3d_plan> p(new (std::nothrow) sem3d_plan());
  if (!p) return fail(SEM3D_ERR_OOM, "host allocation failed");
  try {
    for (int a = 0; a < 3; ++a) p->ax[a] = get_axis(n3[a], k, L3[a], (int)bc);
  } catch (const std::exception& ex) {
    return fail(SEM3D_ERR_INVALID_ARG, std::string("axis setup failed: ") + ex.what());
  }
  const double lmin = p->ax[0]->lam[0] + p->ax[1]->lam[0] + p->ax[2]->lam[0];
  if (!(c > -lmin)) return fail(SEM3D_ERR_INVALID_ARG, "c <= -(lambda_x1 + lambda_y1 + lambda_z1): not definite");
  CUDA_TRY(cudaGetDevice(&p->device));
  CUDA_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  p->g.nx = nx; p->g.ny = ny; p->g.nz = nz; p->g.Px = pad16(nx); p->g.c = c; p->g.bc = (int)bc;
  p->k = k;
  for (int a = 0; a < 3; ++a) p->L[a] = L3[a];
  std::vector<double> hq_rows[3];
  for (int a = 0; a < 3; ++a) {
    const Axis1D& A = *p->ax[a];
    DevAxis& D = p->dev[a];
    D.n = A.n; D.k = k; D.Kp = pad16(A.n);
    sem3d_status st;
    if ((st = dev_upload(p.get(), &D.M, A.M.data(), A.M.size())) != SEM3D_OK) return st;
    if ((st = dev_upload(p.get(), &D.T, A.T.data(), A.T.size())) != SEM3D_OK) return st;
    if ((st = dev_upload(p.get(), &D.Tinv, A.Tinv.data(), A.Tinv.size())) != SEM3D_OK) return st;
    if ((st = dev_upload(p.get(), &D.lam, A.lam.data(), A.lam.size())) != SEM3D_OK) return st;
    std::vector<float> lf(A.lam.begin(), A.lam.end());
    if ((st = dev_upload(p.get(), &D.lamf, lf.data(), lf.size())) != SEM3D_OK) return st;
    if ((st = dev_upload(p.get(), &D.Hband, A.Hband.data(), A.Hband.size())) != SEM3D_OK) return st;
    {
      std::vector<double>& hq = hq_rows[a];
      hq = A.Hq;  // the shift c joins the x operator's diagonal
      if (a == 0)
        for (int q = 0; q < k; ++q) hq[(size_t)q * (2 * k + 1) + k] += c;
      if ((st = dev_upload(p.get(), &D.Hq, hq.data(), hq.size())) != SEM3D_OK) return st;
      // Three FP32 terms: hi + lo holds 48 bits; the remainder lo2 makes the
      // sum exact (53 bits need at most three 24-bit pieces).
      std::vector<float> hh(hq.size()), hl(hq.size()), hl2(hq.size());
      for (size_t q = 0; q < hq.size(); ++q) {
        hh[q] = (float)hq[q];
        hl[q] = (float)(hq[q] - (double)hh[q]);
        hl2[q] = (float)(hq[q] - (double)hh[q] - (double)hl[q]);
      }
      if (k <= 4)
        for (size_t q = 0; q < hq.size(); ++q) {
          D.Hq_hi_host[q] = hh[q];
          D.Hq_lo_host[q] = hl[q];
          D.Hq_lo2_host[q] = hl2[q];
        }
      if ((st = dev_upload(p.get(), &D.Hq_hi, hh.data(), hh.size())) != SEM3D_OK) return st;
      if ((st = dev_upload(p.get(), &D.Hq_lo, hl.data(), hl.size())) != SEM3D_OK) return st;
      if ((st = dev_upload(p.get(), &D.Hq_lo2, hl2.data(), hl2.size())) != SEM3D_OK) return st;
    }
    if ((st = dev_upload(p.get(), &D.band_lo, A.band_lo.data(), A.band_lo.size())) != SEM3D_OK) return st;
    if ((st = dev_upload(p.get(), &D.band_hi, A.band_hi.data(), A.band_hi.size())) != SEM3D_OK) return st;
    for (int w = 0; w < 2; ++w) {
      const std::vector<double>& Wd = (w == 0) ? A.Tinv : A.T;
      std::vector<float> wf(Wd.begin(), Wd.end());
      if ((st = dev_upload(p.get(), &D.Wf[w], wf.data(), wf.size())) != SEM3D_OK) return st;
    }
    for (int w = 0; w < 2; ++w) {  // TF32-rounded W for the TF32 tier, row pitch Kp
      const std::vector<double>& Wd = (w == 0) ? A.Tinv : A.T;
      std::vector<float> wt((size_t)A.n * D.Kp, 0.f);
      for (int o = 0; o < A.n; ++o)
        for (int t = 0; t < A.n; ++t) wt[(size_t)o * D.Kp + t] = tf32_round((float)Wd[(size_t)o * A.n + t]);
      if ((st = dev_upload(p.get(), &D.Wt32[w], wt.data(), wt.size())) != SEM3D_OK) return st;
    }
    for (int w = 0; w < 2; ++w) {  // fp16 pairs of W * 2^eW for the F16X3 tier
      const std::vector<double>& Wd = (w == 0) ? A.Tinv : A.T;
      const int n = A.n;
      double mx = 0.0, norm = 0.0;
      for (int o = 0; o < n; ++o) {
        double rs = 0.0;
        for (int t = 0; t < n; ++t) {
          const double v = std::fabs(Wd[(size_t)o * n + t]);
          mx = std::max(mx, v);
          rs += v;
        }
        norm = std::max(norm, rs);
      }
      const int eW = mx > 0.0 ? std::ilogb(16384.0 / mx) : 0;
      D.eW16[w] = eW;
      D.normW[w] = (float)norm;
      std::vector<__half> h16((size_t)n * D.Kp, __float2half_rn(0.f)), l16((size_t)n * D.Kp, __float2half_rn(0.f));
      for (int o = 0; o < n; ++o)
        for (int t = 0; t < n; ++t) {
          const float x = (float)std::ldexp(Wd[(size_t)o * n + t], eW);
          const __half hh = __float2half_rn(x);
          h16[(size_t)o * D.Kp + t] = hh;
          l16[(size_t)o * D.Kp + t] = __float2half_rn(x - __half2float(hh));
        }
      if ((st = dev_upload(p.get(), &D.W16_hi[w], h16.data(), h16.size())) != SEM3D_OK) return st;
      if ((st = dev_upload(p.get(), &D.W16_lo[w], l16.data(), l16.size())) != SEM3D_OK) return st;
    }
    std::vector<__nv_bfloat16> hi, lo;
    for (int w = 0; w < 2; ++w) {
      split_matrix(w == 0 ? A.Tinv : A.T, A.n, D.Kp, hi, lo);
      if ((st = dev_upload(p.get(), &D.W_hi[w], hi.data(), hi.size())) != SEM3D_OK) return st;
      if ((st = dev_upload(p.get(), &D.W_lo[w], lo.data(), lo.size())) != SEM3D_OK) return st;
    }
  }
  {
    void* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, 256));
    p->owned.push_back(d);
    CUDA_TRY(cudaMemset(d, 0, 256));
    p->d_err = static_cast<int*>(d);
    p->d_f16 = reinterpret_cast<F16State*>(static_cast<char*>(d) + 128);
    p->d_fix = reinterpret_cast<int*>(static_cast<char*>(d) + 192);
  }
  if (p->g.bc == 0) {
    const double* rows[3] = {hq_rows[0].data(), hq_rows[1].data(), hq_rows[2].data()};
    p->fix_ok = build_fix_coef(rows, k, p->fix);
  }
  p->div_bound = (float)(1.0 / (lmin + c));
  *out = p.release();
  return SEM3D_OK;
}

sem3d_status sem3d_set_precision(sem3d_handle h, sem3d_precision prec, int sweeps) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  if (prec != SEM3D_FP64 && prec != SEM3D_FP32 && prec != SEM3D_TF32 && prec != SEM3D_BF16 && prec != SEM3D_BF16X3 &&
      prec != SEM3D_F16X3)
    return fail(SEM3D_ERR_INVALID_ARG, "unknown precision");
  if (prec == SEM3D_F16X3 && (h->k > 8 || h->g.bc != 0))
    return fail(SEM3D_ERR_UNSUPPORTED, "F16X3 needs k <= 8 and Dirichlet data");
  if (sweeps < 0 || sweeps > 16) return fail(SEM3D_ERR_INVALID_ARG, "sweeps must be in [0, 16]");
  if (prec == SEM3D_BF16X3 || prec == SEM3D_BF16 || prec == SEM3D_F16X3 || prec == SEM3D_TF32) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device);
    if (major != 10 || minor != 3) return fail(SEM3D_ERR_UNSUPPORTED, "tensor-core tiers need an sm_103 GPU");
  }
  if (prec == SEM3D_FP32) {
    const cudaError_t e = f32_autotune(h->g, h->dev);
    if (e != cudaSuccess) return fail(SEM3D_ERR_CUDA, std::string("FP32 autotuning: ") + cudaGetErrorString(e));
  }
  if (prec == SEM3D_BF16X3 || prec == SEM3D_BF16) {
    const cudaError_t e = tc_autotune(h->g, h->dev, prec == SEM3D_BF16 ? 1 : 3, h->d_err, h->num_sms);
    if (e != cudaSuccess) return fail(SEM3D_ERR_CUDA, std::string("tensor-core autotuning: ") + cudaGetErrorString(e));
  }
  if (prec == SEM3D_TF32) {
    const cudaError_t e = tf32_autotune(h->g, h->dev, h->d_err, h->num_sms);
    if (e != cudaSuccess) return fail(SEM3D_ERR_CUDA, std::string("TF32 autotuning: ") + cudaGetErrorString(e));
  }
  h->prec = prec;
  h->sweeps = sweeps;
  return SEM3D_OK;
}

sem3d_status sem3d_inject_stall(sem3d_handle h, int launches) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  if (launches < 0 || launches > 64) return fail(SEM3D_ERR_INVALID_ARG, "launches must be in [0, 64]");
  tc_inject_stall(launches);
  return SEM3D_OK;
}

sem3d_status sem3d_set_tuned_config(sem3d_handle h, int axis, int config) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  if (axis < 0 || axis > 2) return fail(SEM3D_ERR_INVALID_ARG, "axis must be 0, 1 or 2");
  if (config < 0 || config > 5) return fail(SEM3D_ERR_INVALID_ARG, "config must be in [0, 5]");
  f32_set_config(axis, h->g, config);
  return SEM3D_OK;
}

sem3d_status sem3d_tuned_config(sem3d_handle h, int axis, int* config) {
  if (!h || !config) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  if (axis < 0 || axis > 2) return fail(SEM3D_ERR_INVALID_ARG, "axis must be 0, 1 or 2");
  *config = f32_config(axis, h->g);
  return SEM3D_OK;
}

sem3d_status sem3d_set_tc_config(sem3d_handle h, int axis, int config) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  if (axis < 0 || axis > 2) return fail(SEM3D_ERR_INVALID_ARG, "axis must be 0, 1 or 2");
  if (config != TC_SINGLE && config != TC_PAIR) return fail(SEM3D_ERR_INVALID_ARG, "config must be 0 or 1");
  tc_set_config(axis, h->g, 1, config);
  tc_set_config(axis, h->g, 3, config);
  const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
  tf32_set_config(n3[axis], n3[(axis + 1) % 3], n3[(axis + 2) % 3], config);
  return SEM3D_OK;
}

sem3d_status sem3d_tc_config(sem3d_handle h, int axis, int* config) {
  if (!h || !config) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  if (axis < 0 || axis > 2) return fail(SEM3D_ERR_INVALID_ARG, "axis must be 0, 1 or 2");
  if (h->prec == SEM3D_TF32) {
    const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
    *config = tf32_config(n3[axis], n3[(axis + 1) % 3], n3[(axis + 2) % 3]);
  } else {
    *config = tc_config(axis, h->g, h->prec == SEM3D_BF16 ? 1 : 3);
  }
  return SEM3D_OK;
}

sem3d_status sem3d_set_residual(sem3d_handle h, sem3d_residual mode) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  if (mode != SEM3D_RESIDUAL_FP64 && mode != SEM3D_RESIDUAL_MIXED && mode != SEM3D_RESIDUAL_DF)
    return fail(SEM3D_ERR_INVALID_ARG, "unknown mode");
  h->residual = mode;
  return SEM3D_OK;
}

}  // extern "C"

namespace {
bool use_fixed_residual(const sem3d_plan* h);  // FP64-accurate residuals in fixed point (defined below)
}  // namespace

extern "C" {

sem3d_status sem3d_set_exact_residual(sem3d_handle h, sem3d_exact_residual kind) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  if (kind != SEM3D_EXACT_FIXED && kind != SEM3D_EXACT_FP64) return fail(SEM3D_ERR_INVALID_ARG, "unknown kind");
  h->exact_kind = kind;
  return SEM3D_OK;
}

sem3d_status sem3d_exact_residual_kind(sem3d_handle h, int* kind) {
  if (!h || !kind) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  *kind = use_fixed_residual(h) ? SEM3D_EXACT_FIXED : SEM3D_EXACT_FP64;
  return SEM3D_OK;
}

sem3d_status sem3d_workspace_size(sem3d_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  *bytes = workspace_bytes(h);
  return SEM3D_OK;
}

sem3d_status sem3d_set_workspace(sem3d_handle h, void* dptr, size_t bytes) {
  if (!h || !dptr) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(dptr) & 255) != 0) return fail(SEM3D_ERR_INVALID_ARG, "workspace not 256-B aligned");
  if (bytes < workspace_bytes(h)) return fail(SEM3D_ERR_INVALID_ARG, "workspace too small");
  if (h->ws && h->ws_owned) cudaFree(h->ws);
  h->ws = dptr;
  h->ws_bytes = bytes;
  h->ws_owned = false;
  return SEM3D_OK;
}

sem3d_status sem3d_solve(sem3d_handle h, const double* f, double* u, void* stream) {
  if (!h || !f || !u) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  if (f == u || (f < u + N && u < f + N)) return fail(SEM3D_ERR_INVALID_ARG, "f and u overlap");
  sem3d_status st = ensure_workspace(h);
  if (st != SEM3D_OK) return st;
  return run_solve(h, f, u, static_cast<cudaStream_t>(stream));
}

sem3d_status sem3d_solve_host(sem3d_handle h, const double* f_host, double* u_host, void* stream) {
  if (!h || !f_host || !u_host) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  sem3d_status st = ensure_workspace(h);
  if (st != SEM3D_OK) return st;
  auto& io = h->io;
  if (!io.h2d) {
    for (int b = 0; b < 2; ++b) {
      CUDA_TRY(cudaMalloc(&io.f[b], N * sizeof(double)));
      CUDA_TRY(cudaMalloc(&io.u[b], N * sizeof(double)));
      CUDA_TRY(cudaEventCreateWithFlags(&io.copied_in[b], cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&io.solved[b], cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&io.copied_out[b], cudaEventDisableTiming));
    }
    CUDA_TRY(cudaStreamCreateWithFlags(&io.h2d, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&io.d2h, cudaStreamNonBlocking));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int b = (int)(io.calls++ & 1);
  // f into buffer b once the solve that last read it is done.
  if (io.used[b]) CUDA_TRY(cudaStreamWaitEvent(io.h2d, io.solved[b], 0));
  CUDA_TRY(cudaMemcpyAsync(io.f[b], f_host, N * sizeof(double), cudaMemcpyHostToDevice, io.h2d));
  CUDA_TRY(cudaEventRecord(io.copied_in[b], io.h2d));
  // Solve on the caller's stream once f is in and u[b] has been copied out.
  CUDA_TRY(cudaStreamWaitEvent(s, io.copied_in[b], 0));
  if (io.used[b]) CUDA_TRY(cudaStreamWaitEvent(s, io.copied_out[b], 0));
  if ((st = run_solve(h, io.f[b], io.u[b], s)) != SEM3D_OK) return st;
  CUDA_TRY(cudaEventRecord(io.solved[b], s));
  // u back to the host on the other copy stream.
  CUDA_TRY(cudaStreamWaitEvent(io.d2h, io.solved[b], 0));
  CUDA_TRY(cudaMemcpyAsync(u_host, io.u[b], N * sizeof(double), cudaMemcpyDeviceToHost, io.d2h));
  CUDA_TRY(cudaEventRecord(io.copied_out[b], io.d2h));
  io.used[b] = true;
  return SEM3D_OK;
}

sem3d_status sem3d_solve_host_wait(sem3d_handle h, void* stream) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  auto& io = h->io;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int b = 0; b < 2; ++b)
    if (io.used[b]) CUDA_TRY(cudaStreamWaitEvent(s, io.copied_out[b], 0));
  return SEM3D_OK;
}

}  // extern "C"

namespace {

// The solve itself (arguments already checked, workspace present).
// FP64-accurate residuals of the split tiers in 64-bit fixed point (see fix_kernels.cu)
bool use_fixed_residual(const sem3d_plan* h) {
  return h->fix_ok && h->exact_kind == SEM3D_EXACT_FIXED &&
         (h->prec == SEM3D_BF16X3 || h->prec == SEM3D_BF16 || h->prec == SEM3D_TF32);
}

sem3d_status run_solve(sem3d_plan* h, const double* f, double* u, cudaStream_t s) {
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  sem3d_status st = SEM3D_OK;
  if (h->prec == SEM3D_FP64) {
    double* r = reinterpret_cast<double*>(static_cast<char*>(h->ws) + 2 * align256(N * sizeof(double)));
    if ((st = solve_once_f64(h, f, u, false, s)) != SEM3D_OK) return st;
    for (int sw = 0; sw < h->sweeps; ++sw) {
      LAUNCH(h, K_STENCIL, 1, s, launch_stencil(h->g, h->k, h->dev, u, f, r, nullptr, nullptr, 1, s));
      if ((st = solve_once_f64(h, r, u, true, s)) != SEM3D_OK) return st;
    }
  } else if (h->prec == SEM3D_FP32) {
    double* r = reinterpret_cast<double*>(static_cast<char*>(h->ws) + 2 * align256(N * sizeof(float)));
    if ((st = solve_once_f32(h, f, u, false, s)) != SEM3D_OK) return st;
    for (int sw = 0; sw < h->sweeps; ++sw) {
      LAUNCH(h, K_STENCIL, 1, s, launch_stencil(h->g, h->k, h->dev, u, f, r, nullptr, nullptr, 1, s));
      if ((st = solve_once_f32(h, r, u, true, s)) != SEM3D_OK) return st;
    }
  } else if (h->prec == SEM3D_TF32) {
    double* r = reinterpret_cast<double*>(static_cast<char*>(h->ws) + 2 * align256(tf32_elems(h->g) * sizeof(float)));
    if ((st = solve_once_tf32(h, f, u, false, s)) != SEM3D_OK) return st;
    // between solves the two ping-pong buffers (>= Px ny nz floats each) are
    // free: they hold u in fixed point for the fixed-point residual
    int* Uh = static_cast<int*>(h->ws);
    int* Ul = reinterpret_cast<int*>(static_cast<char*>(h->ws) + align256(tf32_elems(h->g) * sizeof(float)));
    const bool fixed = use_fixed_residual(h);
    for (int sw = 0; sw < h->sweeps; ++sw) {
      if (fixed)
        LAUNCH(h, K_STENCIL, sw == 0 ? 4 : 3, s,
               launch_residual_fixed(h->g, h->k, h->fix, u, f, h->d_fix, sw > 0, Uh, Ul, nullptr, nullptr,
                                     h->num_sms, s, r));
      else
        LAUNCH(h, K_STENCIL, 1, s, launch_stencil(h->g, h->k, h->dev, u, f, r, nullptr, nullptr, 1, s));
      if ((st = solve_once_tf32(h, r, u, true, s)) != SEM3D_OK) return st;
    }
  } else {
    const size_t Ns = align256((size_t)h->g.Px * h->g.ny * h->g.nz * sizeof(__nv_bfloat16));
    const size_t Nf = align256((size_t)h->g.Px * h->g.ny * h->g.nz * sizeof(float));  // double-FP32 u, pitch Px
    char* w = static_cast<char*>(h->ws);
    TcBuffers S0{reinterpret_cast<__nv_bfloat16*>(w), reinterpret_cast<__nv_bfloat16*>(w + Ns)};
    TcBuffers S1{reinterpret_cast<__nv_bfloat16*>(w + 2 * Ns), reinterpret_cast<__nv_bfloat16*>(w + 3 * Ns)};
    DfBuffers D{reinterpret_cast<float*>(w + 6 * Ns), reinterpret_cast<float*>(w + 6 * Ns + Nf)};
    const DfBuffers none{nullptr, nullptr};
    const int sw = h->sweeps;
    // Double-FP32 sweeps (the solution held as a double-FP32 pair between
    // them): SEM3D_RESIDUAL_MIXED runs sweeps 1 .. sw-1 so and the last one in
    // FP64 on the FP64 solution; SEM3D_RESIDUAL_DF runs every sweep so.
    const bool df_ok = h->k <= 8 && h->g.bc == 0 && (h->prec == SEM3D_BF16X3 || h->prec == SEM3D_F16X3);
    const int ndf = !df_ok ? 0
                           : (h->residual == SEM3D_RESIDUAL_MIXED && sw >= 2) ? sw - 1
                           : (h->residual == SEM3D_RESIDUAL_DF) ? sw : 0;
    const bool mixed = ndf > 0;
    // Every residual in double-FP32: the operator's rows must then be exact
    // (three FP32 terms), or the sweeps converge to the 48-bit operator's
    // solution.  With a final FP64 sweep the 48-bit rows suffice.
    const bool exact_coef = h->residual == SEM3D_RESIDUAL_DF;
    const bool f16 = h->prec == SEM3D_F16X3;
    // F16X3: the residual is written as FP32 into S1's storage (4 bytes per
    // entry at pitch Px fit in its hi + lo arrays) and then split with a
    // power-of-two scale chosen from its maximum.
    float* r32 = reinterpret_cast<float*>(S1.hi);
    __half* S0h = reinterpret_cast<__half*>(S0.hi);
    __half* S0l = reinterpret_cast<__half*>(S0.lo);
    auto reset_scales = [&]() -> sem3d_status {
      CUDA_TRY(cudaMemsetAsync(h->d_f16, 0, sizeof(F16State), s));
      return SEM3D_OK;
    };
    const bool fixed = use_fixed_residual(h);
    if (f16) {
      if ((st = reset_scales()) != SEM3D_OK) return st;
      LAUNCH(h, K_SPLIT, 1, s, launch_absmax_f64(h->g, f, h->d_f16, s));
      LAUNCH(h, K_SPLIT, 1, s, launch_split_f16(h->g, f, true, S0h, S0l, h->d_f16, s));
    } else {
      // the fixed-point residuals' scale of f comes with the split
      if (fixed) CUDA_TRY(cudaMemsetAsync(h->d_fix + 1, 0, sizeof(int), s));
      LAUNCH(h, K_SPLIT, 1, s, launch_split(h->g, f, S0.hi, S0.lo, s, fixed ? h->d_fix + 1 : nullptr));
    }
    if (!mixed) {
      if ((st = solve_once_bf16x3(h, S0, S1, u, EPI_STORE, none, s)) != SEM3D_OK) return st;
    } else {
      if ((st = solve_once_bf16x3(h, S0, S1, nullptr, EPI_DF_STORE, D, s)) != SEM3D_OK) return st;
      for (int q = 1; q <= ndf; ++q) {
        if (f16) {
          if ((st = reset_scales()) != SEM3D_OK) return st;
          LAUNCH(h, K_STENCIL, 1, s,
                 launch_stencil_df(h->g, h->k, h->dev, D, f, nullptr, nullptr, s, r32, h->d_f16, exact_coef, q == 1));
          LAUNCH(h, K_SPLIT, 1, s, launch_split_f16(h->g, r32, false, S0h, S0l, h->d_f16, s));
        } else {
          // k in {1, 2, 4}: one vector kernel that also writes the pads; otherwise
          // the element kernel plus a pad-zeroing kernel when Px > nx
          const int df_launches = (h->k == 1 || h->k == 2 || h->k == 4 || h->g.Px == h->g.nx) ? 1 : 2;
          LAUNCH(h, K_STENCIL, df_launches, s,
                 launch_stencil_df(h->g, h->k, h->dev, D, f, S0.hi, S0.lo, s, nullptr, nullptr, exact_coef, q == 1));
        }
        const bool last_df = (q == ndf);
        if ((st = solve_once_bf16x3(h, S0, S1, last_df ? u : nullptr, last_df ? EPI_DF_ACCUM_F64 : EPI_DF_ACCUM, D,
                                    s)) != SEM3D_OK)
          return st;
      }
    }
    for (int q = ndf; q < sw; ++q) {
      if (f16) {
        if ((st = reset_scales()) != SEM3D_OK) return st;
        LAUNCH(h, K_STENCIL, 1, s, launch_stencil_f32out(h->g, h->k, h->dev, u, f, r32, h->d_f16, s));
        LAUNCH(h, K_SPLIT, 1, s, launch_split_f16(h->g, r32, false, S0h, S0l, h->d_f16, s));
      } else if (fixed) {
        // the double-FP32 solution buffers are free by now: they hold u in fixed point
        LAUNCH(h, K_STENCIL, 3, s,
               launch_residual_fixed(h->g, h->k, h->fix, u, f, h->d_fix, true, reinterpret_cast<int*>(D.hi),
                                     reinterpret_cast<int*>(D.lo), S0.hi, S0.lo, h->num_sms, s));
      } else {
        LAUNCH(h, K_STENCIL, h->g.Px != h->g.nx ? 2 : 1, s,
               launch_stencil(h->g, h->k, h->dev, u, f, nullptr, S0.hi, S0.lo, 2, s));
      }
      if ((st = solve_once_bf16x3(h, S0, S1, u, EPI_ACCUM, none, s)) != SEM3D_OK) return st;
    }
  }
  return SEM3D_OK;
}

}  // namespace

extern "C" {

sem3d_status sem3d_apply(sem3d_handle h, const double* u, double* Au, void* stream) {
  if (!h || !u || !Au) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  if (u < Au + N && Au < u + N) return fail(SEM3D_ERR_INVALID_ARG, "u and Au overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LAUNCH(h, K_STENCIL, 1, s, launch_stencil(h->g, h->k, h->dev, u, nullptr, Au, nullptr, nullptr, 0, s));
  return SEM3D_OK;
}

sem3d_status sem3d_get_nodes(sem3d_handle h, int axis, double* x_host) {
  if (!h || !x_host || axis < 0 || axis > 2) return fail(SEM3D_ERR_INVALID_ARG, "bad argument");
  std::memcpy(x_host, h->ax[axis]->x.data(), h->ax[axis]->x.size() * sizeof(double));
  return SEM3D_OK;
}

sem3d_status sem3d_get_eigs(sem3d_handle h, int axis, double* lambda_host, double* T_host) {
  if (!h || axis < 0 || axis > 2) return fail(SEM3D_ERR_INVALID_ARG, "bad argument");
  const Axis1D& A = *h->ax[axis];
  if (lambda_host) std::memcpy(lambda_host, A.lam.data(), A.lam.size() * sizeof(double));
  if (T_host) {
    const int n = A.n;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) T_host[(size_t)j * n + i] = A.T[(size_t)i * n + j];  // column-major
  }
  return SEM3D_OK;
}

sem3d_status sem3d_axis_info(int n, int k, double L, double* x, double* M, double* lambda, double* T) {
  if (k < 1 || k > 24 || n < 1 || (n + 1) % k != 0 || !(L > 0.0))
    return fail(SEM3D_ERR_INVALID_ARG, "need k in [1,24], n >= 1, (n+1) % k == 0, L > 0");
  std::shared_ptr<const Axis1D> ax;
  try {
    ax = get_axis(n, k, L, 0);
  } catch (const std::exception& ex) {
    return fail(SEM3D_ERR_INVALID_ARG, std::string("axis setup failed: ") + ex.what());
  }
  if (x) std::memcpy(x, ax->x.data(), n * sizeof(double));
  if (M) std::memcpy(M, ax->M.data(), n * sizeof(double));
  if (lambda) std::memcpy(lambda, ax->lam.data(), n * sizeof(double));
  if (T)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) T[(size_t)j * n + i] = ax->T[(size_t)i * n + j];
  return SEM3D_OK;
}

sem3d_status sem3d_sync_check(sem3d_handle h, void* stream) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int flags = 0;
  CUDA_TRY(cudaMemcpy(&flags, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flags != 0) {
    CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
    if (flags & (1 << SEM3D_ERR_TIMEOUT)) {
      // bits 8-15: where the wait ran out (role and kernel family, see tc_ptx.cuh)
      static const char* names[8] = {"producer", "MMA (operands)", "MMA (accumulator)", "epilogue",
                                     "split kernel", "split CTA-pair kernel", "TF32 kernel", "TF32 CTA-pair kernel"};
      std::string where;
      for (int b = 0; b < 8; ++b)
        if (flags & (1 << (8 + b))) where += std::string(where.empty() ? "" : ", ") + names[b];
      return fail(SEM3D_ERR_TIMEOUT, "a tensor-core kernel's bounded wait expired" +
                                         (where.empty() ? std::string() : " (" + where + ")"));
    }
    return fail(SEM3D_ERR_CUDA, "device error flag set");
  }
  return SEM3D_OK;
}

sem3d_status sem3d_profile(sem3d_handle h, int enable) {
  if (!h) return fail(SEM3D_ERR_INVALID_ARG, "handle is NULL");
  for (auto& ev : h->pending) {
    cudaEventSynchronize(ev.b);
    h->pool.push_back(ev.a);
    h->pool.push_back(ev.b);
  }
  h->pending.clear();
  for (int q = 0; q < 9; ++q) { h->prof_ms[q] = 0.0; h->prof_n[q] = 0; }
  h->profiling = enable != 0;
  return SEM3D_OK;
}

sem3d_status sem3d_profile_read(sem3d_handle h, int kind, long long* launches, double* total_ms) {
  if (!h || kind < 0 || kind > 8) return fail(SEM3D_ERR_INVALID_ARG, "bad argument");
  for (auto& ev : h->pending) {
    CUDA_TRY(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
    h->prof_ms[ev.kind] += ms;
    h->prof_n[ev.kind] += ev.count;
    if (ev.sub >= 0) {
      h->prof_ms[ev.sub] += ms;
      h->prof_n[ev.sub] += ev.count;
    }
    h->pool.push_back(ev.a);
    h->pool.push_back(ev.b);
  }
  h->pending.clear();
  if (launches) *launches = h->prof_n[kind];
  if (total_ms) *total_ms = h->prof_ms[kind];
  return SEM3D_OK;
}

sem3d_status sem3d_launch_count(sem3d_handle h, unsigned long long* count) {
  if (!h || !count) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  *count = h->launches;
  return SEM3D_OK;
}

sem3d_status sem3d_pcg(sem3d_handle h, const double* V, const double* f, double* u, double rtol, int maxit,
                       int* iters, double* relres, void* stream) {
  if (!h || !V || !f || !u) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  if (!(rtol > 0.0) || maxit < 1) return fail(SEM3D_ERR_INVALID_ARG, "need rtol > 0 and maxit >= 1");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  if (u < f + N && f < u + N) return fail(SEM3D_ERR_INVALID_ARG, "f and u overlap");
  if (u < V + N && V < u + N) return fail(SEM3D_ERR_INVALID_ARG, "V and u overlap");
  sem3d_status st = ensure_workspace(h);
  if (st != SEM3D_OK) return st;
  if (!h->pcg_buf) {
    void* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, 6 * align256(N * sizeof(double))));
    h->pcg_buf = static_cast<double*>(d);
    CUDA_TRY(cudaMalloc(&d, sizeof(PcgScalars)));
    h->pcg_sc = static_cast<PcgScalars*>(d);
    CUDA_TRY(cudaStreamCreateWithFlags(&h->pcg_stream, cudaStreamNonBlocking));
  }
  const size_t stride = align256(N * sizeof(double)) / sizeof(double);
  PcgArgs a{};
  a.N = (long long)N;
  a.nx = h->g.nx; a.ny = h->g.ny; a.nz = h->g.nz;
  a.Mx = h->dev[0].M; a.My = h->dev[1].M; a.Mz = h->dev[2].M;
  a.c = h->g.c;
  a.V = V; a.f = f; a.u = u;
  a.r = h->pcg_buf; a.z = a.r + stride; a.p = a.z + stride; a.q = a.p + stride; a.M3 = a.q + stride;
  a.Vmc = a.M3 + stride;
  a.sc = h->pcg_sc;
  // The iteration runs on the plan's own stream, joined to the caller's
  // stream by events at both ends (the caller's stream may be the legacy
  // default stream, which cannot be captured into a graph).
  cudaStream_t cs = static_cast<cudaStream_t>(stream), s = h->pcg_stream;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  CUDA_TRY(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{ev0, ev1};
  CUDA_TRY(cudaEventRecord(ev0, cs));
  CUDA_TRY(cudaStreamWaitEvent(s, ev0, 0));
  CUDA_TRY(cudaMemsetAsync(a.sc, 0, sizeof(PcgScalars), s));
  LAUNCH(h, K_STENCIL, 1, s, launch_pcg(PCG_INIT, a, s));
  // One iteration: z = P r, beta, p = z + beta p, q = A_V p, alpha, u and r.
  auto body = [&](cudaStream_t bs) -> sem3d_status {
    sem3d_status bst = run_solve(h, a.r, a.z, bs);
    if (bst != SEM3D_OK) return bst;
    LAUNCH(h, K_STENCIL, 1, bs, launch_pcg(PCG_DOT_RZ, a, bs));
    LAUNCH(h, K_STENCIL, 1, bs, launch_pcg(PCG_BETA, a, bs));
    LAUNCH(h, K_STENCIL, 1, bs, launch_pcg(PCG_P, a, bs));
    LAUNCH(h, K_STENCIL, 1, bs, launch_stencil(h->g, h->k, h->dev, a.p, nullptr, a.q, nullptr, nullptr, 0, bs));
    LAUNCH(h, K_STENCIL, 1, bs, launch_pcg(PCG_Q, a, bs));
    LAUNCH(h, K_STENCIL, 1, bs, launch_pcg(PCG_UPDATE, a, bs));
    LAUNCH(h, K_STENCIL, 1, bs, launch_pcg(PCG_COUNT, a, bs));
    return SEM3D_OK;
  };
  PcgScalars host{};
  auto read = [&]() -> sem3d_status {
    CUDA_TRY(cudaMemcpyAsync(&host, a.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SEM3D_OK;
  };
  // First iteration runs eagerly (it also performs one-time launch set-up),
  // the rest replay a captured graph of the same body.
  if ((st = body(s)) != SEM3D_OK) return st;
  if ((st = read()) != SEM3D_OK) return st;
  double rr = host.bnorm2 > 0.0 ? std::sqrt(host.rnorm2 / host.bnorm2) : 0.0;
  int it = 1;
  cudaGraphExec_t exec = nullptr;
  if (rr > rtol && std::isfinite(rr) && it < maxit) {
    const bool prof = h->profiling;
    h->profiling = false;  // no event records inside the captured body
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    st = body(s);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    h->profiling = prof;
    if (st != SEM3D_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture(pcg)");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate(pcg)");
  }
  struct ExecGuard {
    cudaGraphExec_t e;
    ~ExecGuard() { if (e) cudaGraphExecDestroy(e); }
  } eg{exec};
  while (rr > rtol && std::isfinite(rr) && it < maxit) {
    CUDA_TRY(cudaGraphLaunch(exec, s));
    // kernels in the graph: one solve + 7 PCG launches
    if ((st = read()) != SEM3D_OK) return st;
    rr = host.bnorm2 > 0.0 ? std::sqrt(host.rnorm2 / host.bnorm2) : 0.0;
    ++it;
  }
  CUDA_TRY(cudaEventRecord(ev1, s));
  CUDA_TRY(cudaStreamWaitEvent(cs, ev1, 0));
  if (iters) *iters = it;
  if (relres) *relres = rr;
  if (!std::isfinite(rr)) return fail(SEM3D_ERR_NOT_CONVERGED, "PCG residual is not finite");
  if (rr > rtol) return fail(SEM3D_ERR_NOT_CONVERGED, "PCG reached maxit before rtol");
  return SEM3D_OK;
}

}  // extern "C"

namespace {

// One Cahn-Hilliard BDF2 step in the plan's arithmetic tier (see
// csrc/ch_kernels.cu for the formula): prep, two forward transforms (z, y, x
// with T^{-1}), pointwise combination in the eigenbasis, backward transform
// (x, y, z with T) writing FP64 phi_{n+1}.
sem3d_status ch_step_core(sem3d_plan* h, const double* phi_n, const double* phi_nm1, double* phi_np1,
                          const ChParams& c, cudaStream_t s) {
  const Geom& g = h->g;
  const DevAxis* d = h->dev;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  char* w = static_cast<char*>(h->ws);
  const TcBuffers nb{nullptr, nullptr};
  if (h->prec == SEM3D_FP64) {
    double* A = reinterpret_cast<double*>(w);
    double* B = reinterpret_cast<double*>(w + align256(N * sizeof(double)));
    double* R = reinterpret_cast<double*>(w + 2 * align256(N * sizeof(double)));
    LAUNCH(h, K_STENCIL, 1, s, launch_ch_prep(SEM3D_FP64, g, phi_n, phi_nm1, A, B, nb, nb, c, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 2, d[2].Tinv, A, R, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 1, d[1].Tinv, R, A, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 0, d[0].Tinv, A, R, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 2, d[2].Tinv, B, A, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 1, d[1].Tinv, A, B, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 0, d[0].Tinv, B, A, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_STENCIL, 1, s, launch_ch_combine(SEM3D_FP64, g, d, R, A, B, nb, nb, nb, c, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 0, d[0].T, B, A, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 1, d[1].T, A, R, EPI_STORE, nullptr, nullptr, nullptr, s));
    LAUNCH(h, K_F64, 1, s, launch_mode_product_f64(g, 2, d[2].T, R, phi_np1, EPI_STORE, nullptr, nullptr, nullptr, s));
  } else if (h->prec == SEM3D_FP32) {
    float* A = reinterpret_cast<float*>(w);
    float* B = reinterpret_cast<float*>(w + align256(N * sizeof(float)));
    float* C = reinterpret_cast<float*>(w + 2 * align256(N * sizeof(float)));
    const double *lx = d[0].lam, *ly = d[1].lam, *lz = d[2].lam;
    LAUNCH(h, K_STENCIL, 1, s, launch_ch_prep(SEM3D_FP32, g, phi_n, phi_nm1, A, B, nb, nb, c, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 2, d[2].Wf[0], A, false, C, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 1, d[1].Wf[0], C, false, A, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 0, d[0].Wf[0], A, false, C, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 2, d[2].Wf[0], B, false, A, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 1, d[1].Wf[0], A, false, B, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 0, d[0].Wf[0], B, false, A, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_STENCIL, 1, s, launch_ch_combine(SEM3D_FP32, g, d, C, A, B, nb, nb, nb, c, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 0, d[0].Wf[1], B, false, A, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 1, d[1].Wf[1], A, false, C, false, EPI_STORE, lx, ly, lz, s));
    LAUNCH(h, K_F32, 1, s, launch_mode_product_f32(g, 2, d[2].Wf[1], C, false, phi_np1, true, EPI_STORE, lx, ly, lz, s));
  } else {
    const size_t Ns = align256((size_t)g.Px * g.ny * g.nz * sizeof(__nv_bfloat16));
    TcBuffers S0{reinterpret_cast<__nv_bfloat16*>(w), reinterpret_cast<__nv_bfloat16*>(w + Ns)};
    TcBuffers S1{reinterpret_cast<__nv_bfloat16*>(w + 2 * Ns), reinterpret_cast<__nv_bfloat16*>(w + 3 * Ns)};
    TcBuffers S2{reinterpret_cast<__nv_bfloat16*>(w + 4 * Ns), reinterpret_cast<__nv_bfloat16*>(w + 5 * Ns)};
    const float *lx = d[0].lamf, *ly = d[1].lamf, *lz = d[2].lamf;
    const int sms = h->num_sms, np = (h->prec == SEM3D_BF16) ? 1 : 3;
    int* e = h->d_err;
    const DfBuffers none{nullptr, nullptr};
    LAUNCH(h, K_SPLIT, 1, s, launch_ch_prep(SEM3D_BF16X3, g, phi_n, phi_nm1, nullptr, nullptr, S0, S2, c, s));
    LAUNCH_SUB(h, K_TC, K_TC_Z, 1, s, launch_mode_product_bf16x3(g, 2, d[2], 0, S0, S1, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_Y, 1, s, launch_mode_product_bf16x3(g, 1, d[1], 0, S1, S0, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_X, 1, s, launch_mode_product_bf16x3(g, 0, d[0], 0, S0, S1, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_Z, 1, s, launch_mode_product_bf16x3(g, 2, d[2], 0, S2, S0, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_Y, 1, s, launch_mode_product_bf16x3(g, 1, d[1], 0, S0, S2, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_X, 1, s, launch_mode_product_bf16x3(g, 0, d[0], 0, S2, S0, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH(h, K_SPLIT, 1, s, launch_ch_combine(SEM3D_BF16X3, g, d, nullptr, nullptr, nullptr, S1, S0, S2, c, s));
    LAUNCH_SUB(h, K_TC, K_TC_X, 1, s, launch_mode_product_bf16x3(g, 0, d[0], 1, S2, S0, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_Y, 1, s, launch_mode_product_bf16x3(g, 1, d[1], 1, S0, S1, nullptr, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
    LAUNCH_SUB(h, K_TC, K_TC_F64OUT, 1, s, launch_mode_product_bf16x3(g, 2, d[2], 1, S1, S0, phi_np1, EPI_STORE, lx, ly, lz, e, sms, s, none, np));
  }
  return SEM3D_OK;
}

sem3d_status ch_check(sem3d_plan* h, double eps, double m, double dt, double S) {
  if (!(eps > 0.0) || !(m > 0.0) || !(dt > 0.0) || !(S >= 0.0) || !std::isfinite(eps + m + dt + S))
    return fail(SEM3D_ERR_INVALID_ARG, "need eps, m, dt > 0 and S >= 0");
  if (h->prec == SEM3D_TF32) return fail(SEM3D_ERR_UNSUPPORTED, "the Cahn-Hilliard step has no TF32 tier");
  return ensure_workspace(h);
}

}  // namespace

extern "C" {

sem3d_status sem3d_ch_step(sem3d_handle h, const double* phi_n, const double* phi_nm1, double* phi_np1, double eps,
                           double m, double dt, double S, void* stream) {
  if (!h || !phi_n || !phi_nm1 || !phi_np1) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  if ((phi_np1 < phi_n + N && phi_n < phi_np1 + N) || (phi_np1 < phi_nm1 + N && phi_nm1 < phi_np1 + N))
    return fail(SEM3D_ERR_INVALID_ARG, "phi_np1 overlaps an input");
  sem3d_status st = ch_check(h, eps, m, dt, S);
  if (st != SEM3D_OK) return st;
  return ch_step_core(h, phi_n, phi_nm1, phi_np1, ChParams{eps, m, dt, S}, static_cast<cudaStream_t>(stream));
}

sem3d_status sem3d_ch_run(sem3d_handle h, double* phi_nm1, double* phi_n, int nsteps, double eps, double m, double dt,
                          double S, void* stream) {
  if (!h || !phi_nm1 || !phi_n) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  if (nsteps < 0) return fail(SEM3D_ERR_INVALID_ARG, "nsteps must be >= 0");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  if (phi_nm1 < phi_n + N && phi_n < phi_nm1 + N) return fail(SEM3D_ERR_INVALID_ARG, "phi arrays overlap");
  sem3d_status st = ch_check(h, eps, m, dt, S);
  if (st != SEM3D_OK) return st;
  if (nsteps == 0) return SEM3D_OK;
  if (!h->ch_buf) {
    void* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, N * sizeof(double)));
    h->ch_buf = static_cast<double*>(d);
  }
  if (!h->pcg_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->pcg_stream, cudaStreamNonBlocking));
  const ChParams c{eps, m, dt, S};
  // Buffers rotate: step q reads B[q%3] (phi_{n-1}) and B[(q+1)%3] (phi_n) and
  // writes B[(q+2)%3]; three steps restore the roles, so a graph of three
  // steps is replayed.  The run is on the plan's own stream, joined to the
  // caller's by events (the caller's stream may be the uncapturable legacy one).
  double* B[3] = {phi_nm1, phi_n, h->ch_buf};
  cudaStream_t cs = static_cast<cudaStream_t>(stream), s = h->pcg_stream;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  CUDA_TRY(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{ev0, ev1};
  CUDA_TRY(cudaEventRecord(ev0, cs));
  CUDA_TRY(cudaStreamWaitEvent(s, ev0, 0));
  int q = 0;
  // first step eagerly (one-time launch set-up must not happen inside a capture)
  if ((st = ch_step_core(h, B[1], B[0], B[2], c, s)) != SEM3D_OK) return st;
  q = 1;
  const int full = (nsteps - q) / 3;
  if (full > 0) {
    const bool prof = h->profiling;
    h->profiling = false;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int t = 0; t < 3 && st == SEM3D_OK; ++t) {
      const int qq = q + t;
      st = ch_step_core(h, B[(qq + 1) % 3], B[qq % 3], B[(qq + 2) % 3], c, s);
    }
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    h->profiling = prof;
    if (st != SEM3D_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture(ch)");
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate(ch)");
    for (int r = 0; r < full; ++r) {
      ce = cudaGraphLaunch(exec, s);
      if (ce != cudaSuccess) { cudaGraphExecDestroy(exec); return cuda_fail(ce, "cudaGraphLaunch(ch)"); }
    }
    cudaGraphExecDestroy(exec);
    q += 3 * full;
  }
  for (; q < nsteps; ++q)
    if ((st = ch_step_core(h, B[(q + 1) % 3], B[q % 3], B[(q + 2) % 3], c, s)) != SEM3D_OK) return st;
  // phi_N is in B[(nsteps+1)%3], phi_{N-1} in B[nsteps%3]; move them home.
  const size_t bytes = N * sizeof(double);
  if (nsteps % 3 == 1) {         // (prev, last) = (phi_n, buf)
    CUDA_TRY(cudaMemcpyAsync(phi_nm1, phi_n, bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(phi_n, h->ch_buf, bytes, cudaMemcpyDeviceToDevice, s));
  } else if (nsteps % 3 == 2) {  // (prev, last) = (buf, phi_nm1)
    CUDA_TRY(cudaMemcpyAsync(phi_n, phi_nm1, bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(phi_nm1, h->ch_buf, bytes, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(cudaEventRecord(ev1, s));
  CUDA_TRY(cudaStreamWaitEvent(cs, ev1, 0));
  return SEM3D_OK;
}

}  // extern "C"

namespace {

// Process-wide state of batched solves: a pool of streams for independent
// problems and a staging area for the grouped launches' descriptor tables.
struct BatchState {
  std::mutex mu;
  int device = -1;
  cudaStream_t streams[8] = {};
  void* host_table = nullptr;   // pinned
  void* dev_table = nullptr;
  size_t table_bytes = 0;
  cudaEvent_t done = nullptr;   // last use of the staging area
};
BatchState g_batch;

constexpr size_t kStageTableBytes = 64 * 1024;  // per grouped launch (>= 64 problems)

sem3d_status batch_resources(int device, size_t stages) {
  if (g_batch.device != device) {
    // first use (or another device): streams and staging on this device
    for (auto& st : g_batch.streams)
      if (st) { cudaStreamDestroy(st); st = nullptr; }
    if (g_batch.host_table) { cudaFreeHost(g_batch.host_table); g_batch.host_table = nullptr; }
    if (g_batch.dev_table) { cudaFree(g_batch.dev_table); g_batch.dev_table = nullptr; }
    if (g_batch.done) { cudaEventDestroy(g_batch.done); g_batch.done = nullptr; }
    g_batch.table_bytes = 0;
    for (auto& st : g_batch.streams) CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&g_batch.done, cudaEventDisableTiming));
    g_batch.device = device;
  }
  const size_t need = stages * kStageTableBytes;
  if (g_batch.table_bytes < need) {
    CUDA_TRY(cudaEventSynchronize(g_batch.done));
    if (g_batch.host_table) cudaFreeHost(g_batch.host_table);
    if (g_batch.dev_table) cudaFree(g_batch.dev_table);
    g_batch.host_table = g_batch.dev_table = nullptr;
    CUDA_TRY(cudaMallocHost(&g_batch.host_table, need));
    CUDA_TRY(cudaMalloc(&g_batch.dev_table, need));
    g_batch.table_bytes = need;
  }
  // the staging area is reused: wait until the previous batch's copies ran
  CUDA_TRY(cudaEventSynchronize(g_batch.done));
  return SEM3D_OK;
}

// Marks the last use of the staging area on s when a grouped batch returns,
// on its error paths too, so that the next batch waits for every table copy
// this one queued before it rewrites the pinned host tables.
struct StagingRelease {
  cudaStream_t s;
  bool recorded = false;
  sem3d_status record() {
    recorded = true;
    CUDA_TRY(cudaEventRecord(g_batch.done, s));
    return SEM3D_OK;
  }
  ~StagingRelease() {
    if (!recorded) cudaEventRecord(g_batch.done, s);
  }
};

// Grouped FP32 solves: each of the six passes of all problems is one launch.
sem3d_status batched_f32(int count, const sem3d_handle* hs, const double* const* f, double* const* u,
                         cudaStream_t s) {
  const int sweeps = hs[0]->sweeps;
  const size_t stages = 6 * (size_t)(1 + sweeps);
  sem3d_status st = batch_resources(hs[0]->device, stages);
  if (st != SEM3D_OK) return st;
  StagingRelease release{s};
  std::vector<Geom> geo(count);
  std::vector<const float*> W(count);
  std::vector<const void*> in(count);
  std::vector<void*> out(count);
  std::vector<const double*> lx(count), ly(count), lz(count);
  std::vector<float*> A(count), B(count);
  std::vector<double*> R(count);
  for (int q = 0; q < count; ++q) {
    sem3d_plan* h = hs[q];
    const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
    geo[q] = h->g;
    lx[q] = h->dev[0].lam; ly[q] = h->dev[1].lam; lz[q] = h->dev[2].lam;
    A[q] = static_cast<float*>(h->ws);
    B[q] = reinterpret_cast<float*>(static_cast<char*>(h->ws) + align256(N * sizeof(float)));
    R[q] = reinterpret_cast<double*>(static_cast<char*>(h->ws) + 2 * align256(N * sizeof(float)));
  }
  size_t stage = 0;
  auto pass = [&](int axis, int which, bool in64, bool out64, int epi, auto in_of, auto out_of) -> sem3d_status {
    for (int q = 0; q < count; ++q) {
      W[q] = hs[q]->dev[axis].Wf[which];
      in[q] = in_of(q);
      out[q] = out_of(q);
    }
    char* ht = static_cast<char*>(g_batch.host_table) + stage * kStageTableBytes;
    char* dt = static_cast<char*>(g_batch.dev_table) + stage * kStageTableBytes;
    ++stage;
    LAUNCH(hs[0], K_F32, 1, s,
           launch_mode_product_f32_grouped(count, geo.data(), axis, W.data(), in.data(), in64, out.data(), out64, epi,
                                           lx.data(), ly.data(), lz.data(), dt, kStageTableBytes, ht, s));
    return SEM3D_OK;
  };
  auto solve_group = [&](auto src, bool accumulate) -> sem3d_status {
    sem3d_status r;
    if ((r = pass(2, 0, true, false, EPI_STORE, src, [&](int q) -> void* { return A[q]; })) != SEM3D_OK) return r;
    if ((r = pass(1, 0, false, false, EPI_STORE, [&](int q) -> const void* { return A[q]; },
                  [&](int q) -> void* { return B[q]; })) != SEM3D_OK) return r;
    if ((r = pass(0, 0, false, false, EPI_DIV, [&](int q) -> const void* { return B[q]; },
                  [&](int q) -> void* { return A[q]; })) != SEM3D_OK) return r;
    if ((r = pass(0, 1, false, false, EPI_STORE, [&](int q) -> const void* { return A[q]; },
                  [&](int q) -> void* { return B[q]; })) != SEM3D_OK) return r;
    if ((r = pass(1, 1, false, false, EPI_STORE, [&](int q) -> const void* { return B[q]; },
                  [&](int q) -> void* { return A[q]; })) != SEM3D_OK) return r;
    return pass(2, 1, false, true, accumulate ? EPI_ACCUM : EPI_STORE, [&](int q) -> const void* { return A[q]; },
                [&](int q) -> void* { return u[q]; });
  };
  if ((st = solve_group([&](int q) -> const void* { return f[q]; }, false)) != SEM3D_OK) return st;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int q = 0; q < count; ++q) {
      sem3d_plan* h = hs[q];
      LAUNCH(h, K_STENCIL, 1, s, launch_stencil(h->g, h->k, h->dev, u[q], f[q], R[q], nullptr, nullptr, 1, s));
    }
    if ((st = solve_group([&](int q) -> const void* { return R[q]; }, true)) != SEM3D_OK) return st;
  }
  return release.record();
}

// Any tiers: each problem's own solve on a pool of streams, forked from and
// joined back to the caller's stream.
// Double-FP32 sweeps of a plan's split-tier solve (see run_solve): 0 when its
// residuals are all FP64.
int df_sweeps(const sem3d_plan* h) {
  const bool df_ok = h->k <= 8 && h->g.bc == 0 && (h->prec == SEM3D_BF16X3 || h->prec == SEM3D_F16X3);
  const int sw = h->sweeps;
  return !df_ok ? 0 : (h->residual == SEM3D_RESIDUAL_MIXED && sw >= 2) ? sw - 1
                    : (h->residual == SEM3D_RESIDUAL_DF) ? sw : 0;
}

// Fork `count` per-problem tasks from s onto the batch's stream pool and join
// them back into s (events created once per batched call).
struct StreamFan {
  cudaStream_t s;
  int ns;
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[8] = {};
  ~StreamFan() {
    if (fork) cudaEventDestroy(fork);
    for (auto e : join)
      if (e) cudaEventDestroy(e);
  }
  sem3d_status init(cudaStream_t s_, int count) {
    s = s_;
    ns = count < 8 ? count : 8;
    CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int k = 0; k < ns; ++k) CUDA_TRY(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
    return SEM3D_OK;
  }
  sem3d_status begin() {
    CUDA_TRY(cudaEventRecord(fork, s));
    for (int k = 0; k < ns; ++k) CUDA_TRY(cudaStreamWaitEvent(g_batch.streams[k], fork, 0));
    return SEM3D_OK;
  }
  cudaStream_t stream(int q) const { return g_batch.streams[q % ns]; }
  sem3d_status end() {
    for (int k = 0; k < ns; ++k) {
      CUDA_TRY(cudaEventRecord(join[k], g_batch.streams[k]));
      CUDA_TRY(cudaStreamWaitEvent(s, join[k], 0));
    }
    return SEM3D_OK;
  }
};

// All plans in a split tier (BF16x3 or BF16) with the same sweeps and the same
// residual schedule: each of the six mode-product passes of every solve of the
// refinement runs as ONE persistent CTA-pair launch over all problems (a queue
// of pair tiles with prefix offsets; per-problem tensor maps and epilogue
// arguments in a device table).  The splits and residuals, which are
// element-wise per problem, run on the stream pool between them.
sem3d_status batched_tc(int count, const sem3d_handle* hs, const double* const* f, double* const* u, cudaStream_t s) {
  const int sweeps = hs[0]->sweeps;
  const int ndf = df_sweeps(hs[0]);
  const int nprod = hs[0]->prec == SEM3D_BF16 ? 1 : 3;
  sem3d_status st = batch_resources(hs[0]->device, 6 * (size_t)(1 + sweeps));
  if (st != SEM3D_OK) return st;
  StagingRelease release{s};
  StreamFan fan;
  if ((st = fan.init(s, count)) != SEM3D_OK) return st;
  std::vector<TcBuffers> S0(count), S1(count);
  std::vector<DfBuffers> D(count);
  for (int q = 0; q < count; ++q) {
    sem3d_plan* h = hs[q];
    const size_t Ns = align256((size_t)h->g.Px * h->g.ny * h->g.nz * sizeof(__nv_bfloat16));
    const size_t Nf = align256((size_t)h->g.Px * h->g.ny * h->g.nz * sizeof(float));
    char* w = static_cast<char*>(h->ws);
    S0[q] = TcBuffers{reinterpret_cast<__nv_bfloat16*>(w), reinterpret_cast<__nv_bfloat16*>(w + Ns)};
    S1[q] = TcBuffers{reinterpret_cast<__nv_bfloat16*>(w + 2 * Ns), reinterpret_cast<__nv_bfloat16*>(w + 3 * Ns)};
    D[q] = DfBuffers{reinterpret_cast<float*>(w + 6 * Ns), reinterpret_cast<float*>(w + 6 * Ns + Nf)};
  }
  const DfBuffers none{nullptr, nullptr};
  std::vector<TcGroupItem> items(count);
  size_t stage = 0;
  // One grouped pass: problem q reads in(q), writes out(q) / out64(q) / df(q).
  auto pass = [&](int axis, int which, int epi, int sub, auto in_of, auto out_of, auto out64_of,
                  bool use_df) -> sem3d_status {
    for (int q = 0; q < count; ++q) {
      const sem3d_plan* h = hs[q];
      items[q] = TcGroupItem{&h->g, &h->dev[axis], in_of(q), out_of(q), out64_of(q), use_df ? D[q] : none,
                             h->dev[0].lamf, h->dev[1].lamf, h->dev[2].lamf};
    }
    char* ht = static_cast<char*>(g_batch.host_table) + stage * kStageTableBytes;
    char* dt = static_cast<char*>(g_batch.dev_table) + stage * kStageTableBytes;
    ++stage;
    LAUNCH_SUB(hs[0], K_TC, sub, 1, s,
               launch_mode_product_bf16x3_grouped(count, items.data(), axis, which, epi, nprod, hs[0]->d_err, dt, ht,
                                                  kStageTableBytes, hs[0]->num_sms, s));
    return SEM3D_OK;
  };
  auto s0 = [&](int q) { return S0[q]; };
  auto s1 = [&](int q) { return S1[q]; };
  auto no64 = [&](int) -> double* { return nullptr; };
  // Forward z, y, x (division fused), backward x, y, then the last z pass with
  // the epilogue epi_last into u / the double-FP32 solution.
  auto solve_group = [&](int epi_last, bool out_u, bool use_df) -> sem3d_status {
    sem3d_status r;
    if ((r = pass(2, 0, EPI_STORE, K_TC_Z, s0, s1, no64, false)) != SEM3D_OK) return r;
    if ((r = pass(1, 0, EPI_STORE, K_TC_Y, s1, s0, no64, false)) != SEM3D_OK) return r;
    if ((r = pass(0, 0, EPI_DIV, K_TC_X, s0, s1, no64, false)) != SEM3D_OK) return r;
    if ((r = pass(0, 1, EPI_STORE, K_TC_X, s1, s0, no64, false)) != SEM3D_OK) return r;
    if ((r = pass(1, 1, EPI_STORE, K_TC_Y, s0, s1, no64, false)) != SEM3D_OK) return r;
    return pass(2, 1, epi_last, K_TC_F64OUT, s1, s0, [&](int q) -> double* { return out_u ? u[q] : nullptr; },
                use_df);
  };
  // f -> split input of every problem
  if ((st = fan.begin()) != SEM3D_OK) return st;
  for (int q = 0; q < count; ++q) {
    int* fexp = use_fixed_residual(hs[q]) ? hs[q]->d_fix + 1 : nullptr;  // the fixed-point residuals' scale of f
    if (fexp) CUDA_TRY(cudaMemsetAsync(fexp, 0, sizeof(int), fan.stream(q)));
    LAUNCH(hs[q], K_SPLIT, 1, fan.stream(q), launch_split(hs[q]->g, f[q], S0[q].hi, S0[q].lo, fan.stream(q), fexp));
  }
  if ((st = fan.end()) != SEM3D_OK) return st;
  if (ndf == 0) {
    if ((st = solve_group(EPI_STORE, true, false)) != SEM3D_OK) return st;
  } else {
    if ((st = solve_group(EPI_DF_STORE, false, true)) != SEM3D_OK) return st;
    const bool exact_coef = hs[0]->residual == SEM3D_RESIDUAL_DF;
    for (int sw = 1; sw <= ndf; ++sw) {
      if ((st = fan.begin()) != SEM3D_OK) return st;
      for (int q = 0; q < count; ++q) {
        sem3d_plan* h = hs[q];
        const int launches = (h->k == 1 || h->k == 2 || h->k == 4 || h->g.Px == h->g.nx) ? 1 : 2;
        LAUNCH(h, K_STENCIL, launches, fan.stream(q),
               launch_stencil_df(h->g, h->k, h->dev, D[q], f[q], S0[q].hi, S0[q].lo, fan.stream(q), nullptr, nullptr,
                                 exact_coef, sw == 1));
      }
      if ((st = fan.end()) != SEM3D_OK) return st;
      const bool last_df = sw == ndf;
      if ((st = solve_group(last_df ? EPI_DF_ACCUM_F64 : EPI_DF_ACCUM, last_df, true)) != SEM3D_OK) return st;
    }
  }
  for (int sw = ndf; sw < sweeps; ++sw) {
    if ((st = fan.begin()) != SEM3D_OK) return st;
    for (int q = 0; q < count; ++q) {
      sem3d_plan* h = hs[q];
      if (use_fixed_residual(h)) {
        LAUNCH(h, K_STENCIL, 3, fan.stream(q),
               launch_residual_fixed(h->g, h->k, h->fix, u[q], f[q], h->d_fix, true, reinterpret_cast<int*>(D[q].hi),
                                     reinterpret_cast<int*>(D[q].lo), S0[q].hi, S0[q].lo, h->num_sms, fan.stream(q)));
      } else {
        LAUNCH(h, K_STENCIL, h->g.Px != h->g.nx ? 2 : 1, fan.stream(q),
               launch_stencil(h->g, h->k, h->dev, u[q], f[q], nullptr, S0[q].hi, S0[q].lo, 2, fan.stream(q)));
      }
    }
    if ((st = fan.end()) != SEM3D_OK) return st;
    if ((st = solve_group(EPI_ACCUM, true, false)) != SEM3D_OK) return st;
  }
  return release.record();
}

sem3d_status batched_streams(int count, const sem3d_handle* hs, const double* const* f, double* const* u,
                             cudaStream_t s) {
  sem3d_status st = batch_resources(hs[0]->device, 1);
  if (st != SEM3D_OK) return st;
  cudaEvent_t fork = nullptr;
  CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  std::vector<cudaEvent_t> joins(8, nullptr);
  struct Guard {
    cudaEvent_t f;
    std::vector<cudaEvent_t>& j;
    ~Guard() {
      cudaEventDestroy(f);
      for (auto e : j)
        if (e) cudaEventDestroy(e);
    }
  } guard{fork, joins};
  CUDA_TRY(cudaEventRecord(fork, s));
  const int ns = count < 8 ? count : 8;
  for (int k = 0; k < ns; ++k) {
    CUDA_TRY(cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming));
    CUDA_TRY(cudaStreamWaitEvent(g_batch.streams[k], fork, 0));
  }
  for (int q = 0; q < count; ++q)
    if ((st = run_solve(hs[q], f[q], u[q], g_batch.streams[q % ns])) != SEM3D_OK) return st;
  for (int k = 0; k < ns; ++k) {
    CUDA_TRY(cudaEventRecord(joins[k], g_batch.streams[k]));
    CUDA_TRY(cudaStreamWaitEvent(s, joins[k], 0));
  }
  return SEM3D_OK;
}

}  // namespace

extern "C" {

sem3d_status sem3d_solve_batched(int count, const sem3d_handle* hs, const double* const* f, double* const* u,
                                 void* stream) {
  if (count < 1 || count > 1024 || !hs || !f || !u) return fail(SEM3D_ERR_INVALID_ARG, "bad batch arguments");
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  for (int q = 0; q < count; ++q) {
    if (!hs[q] || !f[q] || !u[q]) return fail(SEM3D_ERR_INVALID_ARG, "NULL entry in batch");
    if (hs[q]->device != cur) return fail(SEM3D_ERR_INVALID_ARG, "all plans must be on the current device");
    for (int r = 0; r < q; ++r)
      if (hs[r] == hs[q]) return fail(SEM3D_ERR_INVALID_ARG, "a plan appears twice in the batch");
    const size_t N = (size_t)hs[q]->g.nx * hs[q]->g.ny * hs[q]->g.nz;
    if (f[q] < u[q] + N && u[q] < f[q] + N) return fail(SEM3D_ERR_INVALID_ARG, "f and u overlap");
    sem3d_status st = ensure_workspace(hs[q]);
    if (st != SEM3D_OK) return st;
  }
  std::lock_guard<std::mutex> lk(g_batch.mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool grouped_f32 = count <= 64, grouped_tc = count <= 64;
  for (int q = 0; q < count; ++q) {
    const sem3d_plan* h = hs[q];
    grouped_f32 = grouped_f32 && h->prec == SEM3D_FP32 && h->sweeps == hs[0]->sweeps;
    grouped_tc = grouped_tc && (h->prec == SEM3D_BF16X3 || h->prec == SEM3D_BF16) && h->prec == hs[0]->prec &&
                 h->sweeps == hs[0]->sweeps && df_sweeps(h) == df_sweeps(hs[0]) &&
                 h->residual == hs[0]->residual;
  }
  if (grouped_f32) return batched_f32(count, hs, f, u, s);
  if (grouped_tc) return batched_tc(count, hs, f, u, s);
  return batched_streams(count, hs, f, u, s);
}

sem3d_status sem3d_destroy(sem3d_handle h) {
  if (!h) return SEM3D_OK;
  if (h->ch_buf) cudaFree(h->ch_buf);
  cudaError_t e = cudaDeviceSynchronize();
  if (h->pcg_buf) cudaFree(h->pcg_buf);
  if (h->pcg_sc) cudaFree(h->pcg_sc);
  if (h->pcg_stream) cudaStreamDestroy(h->pcg_stream);
  for (int b = 0; b < 2; ++b) {
    if (h->io.f[b]) cudaFree(h->io.f[b]);
    if (h->io.u[b]) cudaFree(h->io.u[b]);
    if (h->io.copied_in[b]) cudaEventDestroy(h->io.copied_in[b]);
    if (h->io.solved[b]) cudaEventDestroy(h->io.solved[b]);
    if (h->io.copied_out[b]) cudaEventDestroy(h->io.copied_out[b]);
  }
  if (h->io.h2d) cudaStreamDestroy(h->io.h2d);
  if (h->io.d2h) cudaStreamDestroy(h->io.d2h);
  for (auto& ev : h->pending) { h->pool.push_back(ev.a); h->pool.push_back(ev.b); }
  for (cudaEvent_t ev : h->pool) cudaEventDestroy(ev);
  if (h->ws && h->ws_owned) cudaFree(h->ws);
  for (void* d : h->owned) cudaFree(d);
  delete h;
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize(destroy)");
  return SEM3D_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve without any allocation.
//
// Some callers cannot let the library call cudaMalloc on their behalf: a
// program whose device memory is owned by another allocator (a framework's
// caching allocator that must account for every byte), one that reserves all
// device memory when it starts, or one that must not pay the implicit device
// synchronisation that cudaMalloc and cudaFree may perform in the middle of
// its work.  sem3d_solve_fp64_static serves them: its scratch (the two
// ping-pong arrays of the mode products and the residual array) is a fixed
// file-scope device array that every GPU loading this library holds until the
// process exits.  The caller still passes f and u.
namespace {

constexpr size_t kStaticMaxDofs = 524288;  // nx*ny*nz limit: 3 * 8 B * 524288 = 12 MiB
static __device__ __align__(256) double g_static_scratch[3 * kStaticMaxDofs];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
struct StaticAddr {
  CUcontext ctx = nullptr;  // context the address belongs to
  double* ptr = nullptr;
};
StaticAddr g_static_addr[kMaxDevices];

// The CUDA driver API's cuCtxGetCurrent, reached through the runtime's entry-point
// query (the library links no driver library).
CUresult current_context(CUcontext* ctx) {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &q, 4000, cudaEnableDefault, &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(q);
  });
  return fn ? fn(ctx) : CUDA_ERROR_NOT_FOUND;
}

// Device address of g_static_scratch on device `dev` (which must be the
// current device).  In host code the array's name is only a host-side
// stand-in, so the address is asked from the runtime: once per device and
// CUDA context (after a cudaDeviceReset the device's new primary context
// holds the array at a new address, which is looked up again).
sem3d_status static_scratch(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SEM3D_ERR_UNSUPPORTED, "device ordinal too large");
  CUcontext ctx = nullptr;
  if (current_context(&ctx) != CUDA_SUCCESS || ctx == nullptr)
    return fail(SEM3D_ERR_CUDA, "sem3d_solve_fp64_static: no current CUDA context");
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticAddr& a = g_static_addr[dev];
  if (a.ptr == nullptr || a.ctx != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    a.ptr = static_cast<double*>(p);
    a.ctx = ctx;
  }
  *out = a.ptr;
  return SEM3D_OK;
}

// Launches of the allocation-free path are counted but never bracketed with
// profiling events (creating an event may allocate).
#define LAUNCH_COUNTED(plan, count, expr)                 \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);   \
    (plan)->launches += (unsigned long long)(count);      \
  } while (0)

sem3d_status solve_once_f64_into(sem3d_plan* p, const double* in, double* out, bool accumulate, double* A, double* B,
                                 cudaStream_t s) {
  const Geom& g = p->g;
  const DevAxis* d = p->dev;
  LAUNCH_COUNTED(p, 1, launch_mode_product_f64(g, 2, d[2].Tinv, in, A, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH_COUNTED(p, 1, launch_mode_product_f64(g, 1, d[1].Tinv, A, B, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH_COUNTED(p, 1, launch_mode_product_f64(g, 0, d[0].Tinv, B, A, EPI_DIV, d[0].lam, d[1].lam, d[2].lam, s));
  LAUNCH_COUNTED(p, 1, launch_mode_product_f64(g, 2, d[2].T, A, B, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH_COUNTED(p, 1, launch_mode_product_f64(g, 1, d[1].T, B, A, EPI_STORE, nullptr, nullptr, nullptr, s));
  LAUNCH_COUNTED(p, 1,
         launch_mode_product_f64(g, 0, d[0].T, A, out, accumulate ? EPI_ACCUM : EPI_STORE, nullptr, nullptr, nullptr, s));
  return SEM3D_OK;
}

}  // namespace

extern "C" sem3d_status sem3d_solve_fp64_static(sem3d_handle h, const double* f, double* u, void* stream) {
  if (!h || !f || !u) return fail(SEM3D_ERR_INVALID_ARG, "NULL argument");
  const size_t N = (size_t)h->g.nx * h->g.ny * h->g.nz;
  if (N > kStaticMaxDofs)
    return fail(SEM3D_ERR_INVALID_ARG, "sem3d_solve_fp64_static: nx*ny*nz = " + std::to_string(N) +
                                           " exceeds the static scratch limit of " + std::to_string(kStaticMaxDofs));
  if (f < u + N && u < f + N) return fail(SEM3D_ERR_INVALID_ARG, "f and u overlap");
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != h->device) return fail(SEM3D_ERR_INVALID_ARG, "current device is not the plan's device");
  double* base = nullptr;
  sem3d_status st = static_scratch(cur, &base);
  if (st != SEM3D_OK) return st;
  // Every pass writes its whole output before anything reads it, so no part
  // of the shared scratch has to start at zero.
  double* A = base;
  double* B = base + N;
  double* r = base + 2 * N;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = solve_once_f64_into(h, f, u, false, A, B, s)) != SEM3D_OK) return st;
  for (int sw = 0; sw < h->sweeps; ++sw) {
    LAUNCH_COUNTED(h, 1, launch_stencil(h->g, h->k, h->dev, u, f, r, nullptr, nullptr, 1, s));
    if ((st = solve_once_f64_into(h, r, u, true, A, B, s)) != SEM3D_OK) return st;
  }
  return SEM3D_OK;
}
