// FP32 CUDA-core mode product (the SEM3D_FP32 tier): FFMA with FP32 operands
// and accumulation, no tensor cores.  Same strided formulation as the FP64
// DMMA kernel (Section 2.4, Eq. 11-13: one Kronecker factor at a time, no
// transposes): C[row, o] = sum_t A[row, t] * W[o, t], rows enumerated by two
// loops (p < R1 stride s1, q < R2 stride s2), axis stride sm.
//
// A CTA of 256 threads computes a BM x BN output tile; each thread owns a
// TM x TN register tile.  K advances in chunks of 16 staged in shared memory,
// with one buffer (load, sync, compute, sync) or two (the next chunk's global
// loads are in flight in registers while the current chunk is multiplied).
// Which of the configurations runs is decided per pass shape by measuring
// them (f32_autotune), since the best one depends on n and on the number of
// rows: a 63-wide output axis wastes half of a 128-wide tile, while large
// passes want the larger register tiles.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "sem3d_internal.h"

namespace sem3d {

namespace {

struct F32Pass {
  const void* in;         // float or double (first pass of a solve)
  void* out;              // float, or double for the last pass
  const float* W;         // n x n row-major
  long long s1, s2, sm;
  int R1, R2, n;
  int epi;                // EPI_STORE / EPI_DIV / EPI_ACCUM (double output only)
  int cfg;                // configuration index (F32Cfg below)
  int nx, ny;
  const double *lamx, *lamy, *lamz;
  double c;
};

template <int BM_, int BN_, int TM_, int TN_, int STAGES_>
struct F32Cfg {
  static constexpr int BM = BM_, BN = BN_, BK = 16, TM = TM_, TN = TN_, STAGES = STAGES_;
  static constexpr int TX = BN / TN, TY = BM / TM;  // threads along outputs / rows
  static_assert(TX * TY == 256, "256 threads");
  static_assert(TM % 4 == 0 && TN % 4 == 0, "float4 shared-memory reads");
  static constexpr int LA = BM * BK / 256, LW = BN * BK / 256;
  static constexpr int A_LD = BM + 4, W_LD = BN + 4;  // padded rows of the staged tiles
  static constexpr int SMEM_FLOATS = STAGES * BK * (A_LD + W_LD);
};

// Configurations: tile shape x {two stages, one stage}.  Indexes 0..2 are the
// double-buffered ones (the grouped launch uses those).
using Cfg0 = F32Cfg<128, 128, 8, 8, 2>;
using Cfg1 = F32Cfg<128, 64, 8, 4, 2>;
using Cfg2 = F32Cfg<64, 64, 4, 4, 2>;
using Cfg3 = F32Cfg<128, 128, 8, 8, 1>;
using Cfg4 = F32Cfg<128, 64, 8, 4, 1>;
using Cfg5 = F32Cfg<64, 64, 4, 4, 1>;
constexpr int F32_NCFG = 6;
constexpr int F32_SMEM_MAX = Cfg0::SMEM_FLOATS;  // the largest

__host__ __device__ constexpr int cfg_bm(int c) { return (c % 3 == 2) ? 64 : 128; }
__host__ __device__ constexpr int cfg_bn(int c) { return (c % 3 == 0) ? 128 : 64; }

// One BM x BN output tile (row tile bx, output tile by) of pass p.
template <class C, typename TIN, typename TOUT, bool KCONTIG>
__device__ __forceinline__ void f32_tile(const F32Pass& p, long long bx, int by, float* smem) {
  float* As = smem;                                     // [STAGES][BK][A_LD]
  float* Ws = smem + C::STAGES * C::BK * C::A_LD;       // [STAGES][BK][W_LD]
  const int tid = threadIdx.x;
  const int tx = tid % C::TX, ty = tid / C::TX;  // outputs tx*TN.., rows ty*TM..
  const long long rows = (long long)p.R1 * p.R2;
  const long long row0 = bx * C::BM;
  const int o0 = by * C::BN;
  const TIN* in = static_cast<const TIN*>(p.in);

  float acc[C::TM][C::TN];
#pragma unroll
  for (int r = 0; r < C::TM; ++r)
#pragma unroll
    for (int c = 0; c < C::TN; ++c) acc[r][c] = 0.f;

  // The rows this thread loads are the same in every K chunk: decode them once.
  long long abase[C::LA];
  int akk[C::LA], ar[C::LA];
#pragma unroll
  for (int it = 0; it < C::LA; ++it) {
    const int e = tid + it * 256;
    int r, kk;
    if (KCONTIG) { kk = e % C::BK; r = e / C::BK; }
    else { r = e % C::BM; kk = e / C::BM; }
    const long long row = row0 + r;
    akk[it] = kk;
    ar[it] = r;
    abase[it] = -1;
    if (row < rows) {
      const long long pp = row % p.R1, qq = row / p.R1;
      abase[it] = pp * p.s1 + qq * p.s2;
    }
  }
  float ra[C::LA], rw[C::LW];
  auto load = [&](int t0) {
#pragma unroll
    for (int it = 0; it < C::LA; ++it) {
      const int t = t0 + akk[it];
      ra[it] = (abase[it] >= 0 && t < p.n) ? (float)in[abase[it] + (long long)t * p.sm] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < C::LW; ++it) {
      const int e = tid + it * 256;
      const int kk = e % C::BK, o = e / C::BK;
      const int oo = o0 + o, t = t0 + kk;
      rw[it] = (oo < p.n && t < p.n) ? __ldg(p.W + (long long)oo * p.n + t) : 0.f;
    }
  };
  auto store = [&](int st) {
    float* a = As + st * C::BK * C::A_LD;
    float* w = Ws + st * C::BK * C::W_LD;
#pragma unroll
    for (int it = 0; it < C::LA; ++it) a[akk[it] * C::A_LD + ar[it]] = ra[it];
#pragma unroll
    for (int it = 0; it < C::LW; ++it) {
      const int e = tid + it * 256;
      w[(e % C::BK) * C::W_LD + e / C::BK] = rw[it];
    }
  };
  auto compute = [&](int st) {
    const float* a = As + st * C::BK * C::A_LD + ty * C::TM;
    const float* w = Ws + st * C::BK * C::W_LD + tx * C::TN;
#pragma unroll
    for (int kk = 0; kk < C::BK; ++kk) {
      float av[C::TM], bv[C::TN];
#pragma unroll
      for (int r = 0; r < C::TM; r += 4) {
        const float4 v = *reinterpret_cast<const float4*>(a + kk * C::A_LD + r);
        av[r] = v.x; av[r + 1] = v.y; av[r + 2] = v.z; av[r + 3] = v.w;
      }
#pragma unroll
      for (int c = 0; c < C::TN; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(w + kk * C::W_LD + c);
        bv[c] = v.x; bv[c + 1] = v.y; bv[c + 2] = v.z; bv[c + 3] = v.w;
      }
#pragma unroll
      for (int r = 0; r < C::TM; ++r)
#pragma unroll
        for (int c = 0; c < C::TN; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
  };

  const int nch = (p.n + C::BK - 1) / C::BK;
  load(0);
  store(0);
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    if (C::STAGES == 2) {
      // The other buffer was last read in the previous chunk, before the
      // barrier that ended it: it can be refilled while this one is used.
      const int cur = ch & 1;
      if (ch + 1 < nch) load((ch + 1) * C::BK);
      compute(cur);
      if (ch + 1 < nch) store(cur ^ 1);
      __syncthreads();
    } else {
      compute(0);
      __syncthreads();
      if (ch + 1 < nch) {
        load((ch + 1) * C::BK);
        store(0);
        __syncthreads();
      }
    }
  }
  TOUT* out = static_cast<TOUT*>(p.out);
#pragma unroll
  for (int r = 0; r < C::TM; ++r) {
    const long long row = row0 + ty * C::TM + r;
    if (row >= rows) continue;
    const long long pp = row % p.R1, qq = row / p.R1;
    const long long base = pp * p.s1 + qq * p.s2;
#pragma unroll
    for (int c = 0; c < C::TN; ++c) {
      const int o = o0 + tx * C::TN + c;
      if (o >= p.n) continue;
      const long long idx = base + (long long)o * p.sm;
      float v = acc[r][c];
      if (p.epi == EPI_DIV) {
        const long long i = idx % p.nx, jl = idx / p.nx;
        const long long j = jl % p.ny, l = jl / p.ny;
        v = v / (float)(p.lamx[i] + p.lamy[j] + p.lamz[l] + p.c);
      }
      if (p.epi == EPI_ACCUM) out[idx] += (TOUT)v;
      else out[idx] = (TOUT)v;
    }
  }
}

template <int CFG, typename TIN, typename TOUT, bool KCONTIG>
__global__ void __launch_bounds__(256, 2) mode_product_f32_kernel(F32Pass p) {
  __shared__ __align__(16) float smem[F32_SMEM_MAX];
  if constexpr (CFG == 0) f32_tile<Cfg0, TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y, smem);
  else if constexpr (CFG == 1) f32_tile<Cfg1, TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y, smem);
  else if constexpr (CFG == 2) f32_tile<Cfg2, TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y, smem);
  else if constexpr (CFG == 3) f32_tile<Cfg3, TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y, smem);
  else if constexpr (CFG == 4) f32_tile<Cfg4, TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y, smem);
  else f32_tile<Cfg5, TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y, smem);
}

// Grouped launch: one pass (the same axis and operand types) of many
// independent problems in a single grid.  Block b belongs to the problem q
// with block_begin[q] <= b < block_begin[q+1]; its tiles are numbered row
// tile fastest, with that problem's own (double-buffered) configuration.
struct F32Group {
  int count;
  const F32Pass* passes;
  const long long* block_begin;  // count + 1 entries
};

template <typename TIN, typename TOUT, bool KCONTIG>
__global__ void __launch_bounds__(256, 2) mode_product_f32_grouped_kernel(F32Group g) {
  __shared__ __align__(16) float smem[F32_SMEM_MAX];
  __shared__ int prob;
  if (threadIdx.x == 0) {
    int q = 0;
    while (q + 1 < g.count && g.block_begin[q + 1] <= (long long)blockIdx.x) ++q;
    prob = q;
  }
  __syncthreads();
  const F32Pass p = g.passes[prob];
  const long long lb = (long long)blockIdx.x - g.block_begin[prob];
  const long long rows = (long long)p.R1 * p.R2;
  const int cfg = p.cfg % 3;
  const long long rt = (rows + cfg_bm(cfg) - 1) / cfg_bm(cfg);
  if (cfg == 0) f32_tile<Cfg0, TIN, TOUT, KCONTIG>(p, lb % rt, (int)(lb / rt), smem);
  else if (cfg == 1) f32_tile<Cfg1, TIN, TOUT, KCONTIG>(p, lb % rt, (int)(lb / rt), smem);
  else f32_tile<Cfg2, TIN, TOUT, KCONTIG>(p, lb % rt, (int)(lb / rt), smem);
}

template <int CFG, typename TIN, typename TOUT>
cudaError_t launch_cfg(const F32Pass& p, bool kcontig, cudaStream_t s) {
  const long long rows = (long long)p.R1 * p.R2;
  const long long bx = (rows + cfg_bm(CFG) - 1) / cfg_bm(CFG);
  if (bx >= (1LL << 31)) return cudaErrorInvalidValue;
  dim3 grid((unsigned)bx, (unsigned)((p.n + cfg_bn(CFG) - 1) / cfg_bn(CFG)));
  if (kcontig) mode_product_f32_kernel<CFG, TIN, TOUT, true><<<grid, 256, 0, s>>>(p);
  else mode_product_f32_kernel<CFG, TIN, TOUT, false><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename TIN, typename TOUT>
cudaError_t launch_f32(const F32Pass& p, bool kcontig, cudaStream_t s) {
  switch (p.cfg) {
    case 0: return launch_cfg<0, TIN, TOUT>(p, kcontig, s);
    case 1: return launch_cfg<1, TIN, TOUT>(p, kcontig, s);
    case 2: return launch_cfg<2, TIN, TOUT>(p, kcontig, s);
    case 3: return launch_cfg<3, TIN, TOUT>(p, kcontig, s);
    case 4: return launch_cfg<4, TIN, TOUT>(p, kcontig, s);
    default: return launch_cfg<5, TIN, TOUT>(p, kcontig, s);
  }
}

template <typename TIN, typename TOUT>
cudaError_t launch_f32_grouped(const F32Group& grp, long long blocks, bool kcontig, cudaStream_t s) {
  if (kcontig) mode_product_f32_grouped_kernel<TIN, TOUT, true><<<(unsigned)blocks, 256, 0, s>>>(grp);
  else mode_product_f32_grouped_kernel<TIN, TOUT, false><<<(unsigned)blocks, 256, 0, s>>>(grp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- autotuner
// Pass shape -> configuration, filled by f32_autotune from measurements.
// Rows are capped at the tuning size: beyond a few waves of tiles the ranking
// no longer changes with the row count.
constexpr long long TUNE_ROWS = 65536;
using TuneKey = std::tuple<int, int, long long>;  // (K contiguous, n, min(rows, TUNE_ROWS))
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

TuneKey tune_key(bool kcontig, int n, long long rows) {
  return TuneKey{kcontig ? 1 : 0, n, rows < TUNE_ROWS ? rows : TUNE_ROWS};
}

int tuned_cfg(bool kcontig, int n, long long rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(kcontig, n, rows));
  return it == g_tune.end() ? 0 : it->second;
}

F32Pass make_pass(const Geom& g, int axis, const float* W, const void* in, void* out, int epi, const double* lamx,
                  const double* lamy, const double* lamz, bool* kcontig) {
  F32Pass p{};
  p.in = in;
  p.out = out;
  p.W = W;
  p.epi = epi;
  p.nx = g.nx;
  p.ny = g.ny;
  p.lamx = lamx;
  p.lamy = lamy;
  p.lamz = lamz;
  p.c = g.c;
  const long long nxy = (long long)g.nx * g.ny;
  *kcontig = false;
  if (axis == 0) {
    p.R1 = g.ny * g.nz; p.R2 = 1; p.s1 = g.nx; p.s2 = 0; p.sm = 1; p.n = g.nx; *kcontig = true;
  } else if (axis == 1) {
    p.R1 = g.nx; p.R2 = g.nz; p.s1 = 1; p.s2 = nxy; p.sm = g.nx; p.n = g.ny;
  } else {
    p.R1 = (int)nxy; p.R2 = 1; p.s1 = 1; p.s2 = 0; p.sm = nxy; p.n = g.nz;
  }
  p.cfg = tuned_cfg(*kcontig, p.n, (long long)p.R1 * p.R2);
  return p;
}

}  // namespace

cudaError_t f32_autotune(const Geom& g, const DevAxis* ax) {
  // The three pass shapes of this grid, each timed on a synthetic pass with
  // the same K extent, output length and access pattern and min(rows, TUNE_ROWS)
  // rows, on scratch buffers of this device.
  struct Shape { bool kcontig; int n; long long rows; const float* W; };
  const Shape shapes[3] = {{true, g.nx, (long long)g.ny * g.nz, ax[0].Wf[0]},
                           {false, g.ny, (long long)g.nx * g.nz, ax[1].Wf[0]},
                           {false, g.nz, (long long)g.nx * g.ny, ax[2].Wf[0]}};
  std::vector<int> todo;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int a = 0; a < 3; ++a)
      if (!g_tune.count(tune_key(shapes[a].kcontig, shapes[a].n, shapes[a].rows))) todo.push_back(a);
  }
  if (todo.empty()) return cudaSuccess;
  size_t need = 0;
  for (int a : todo) {
    const long long r = shapes[a].rows < TUNE_ROWS ? shapes[a].rows : TUNE_ROWS;
    need = std::max(need, (size_t)r * shapes[a].n * sizeof(float));
  }
  float *in = nullptr, *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&in, need);
  if (err == cudaSuccess) err = cudaMalloc(&out, need);
  if (err == cudaSuccess) err = cudaMemset(in, 0, need);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  for (size_t q = 0; q < todo.size() && err == cudaSuccess; ++q) {
    const Shape& sh = shapes[todo[q]];
    const long long r = sh.rows < TUNE_ROWS ? sh.rows : TUNE_ROWS;
    F32Pass p{};
    p.in = in; p.out = out; p.W = sh.W; p.epi = EPI_STORE; p.n = sh.n;
    p.R1 = (int)r; p.R2 = 1; p.s2 = 0;
    if (sh.kcontig) { p.s1 = sh.n; p.sm = 1; }
    else { p.s1 = 1; p.sm = r; }
    int best = 0;
    float best_ms = 0.f;
    for (int c = 0; c < F32_NCFG && err == cudaSuccess; ++c) {
      p.cfg = c;
      err = launch_f32<float, float>(p, sh.kcontig, s);  // warm-up
      if (err == cudaSuccess) err = cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) err = launch_f32<float, float>(p, sh.kcontig, s);
      if (err == cudaSuccess) err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess && (c == 0 || ms < best_ms)) { best = c; best_ms = ms; }
    }
    if (err == cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[tune_key(sh.kcontig, sh.n, sh.rows)] = best;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (in) cudaFree(in);
  if (out) cudaFree(out);
  return err;
}

void f32_set_config(int axis, const Geom& g, int cfg) {
  const bool kc = axis == 0;
  const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
  const long long rows = axis == 0 ? (long long)g.ny * g.nz : (axis == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(kc, n, rows)] = cfg;
}

int f32_config(int axis, const Geom& g) {
  if (axis == 0) return tuned_cfg(true, g.nx, (long long)g.ny * g.nz);
  if (axis == 1) return tuned_cfg(false, g.ny, (long long)g.nx * g.nz);
  return tuned_cfg(false, g.nz, (long long)g.nx * g.ny);
}

cudaError_t launch_mode_product_f32_grouped(int count, const Geom* geoms, int axis, const float* const* W,
                                            const void* const* in, bool in_f64, void* const* out, bool out_f64,
                                            int epi, const double* const* lamx, const double* const* lamy,
                                            const double* const* lamz, void* dev_table, size_t table_bytes,
                                            void* host_table, cudaStream_t s) {
  // Table layout: count passes, then count + 1 block offsets.
  const size_t need = (size_t)count * sizeof(F32Pass) + (size_t)(count + 1) * sizeof(long long);
  if (count < 1 || need > table_bytes) return cudaErrorInvalidValue;
  if (epi == EPI_ACCUM && !out_f64) return cudaErrorInvalidValue;
  F32Pass* passes = static_cast<F32Pass*>(host_table);
  long long* begin = reinterpret_cast<long long*>(static_cast<char*>(host_table) + (size_t)count * sizeof(F32Pass));
  bool kcontig = false;
  begin[0] = 0;
  for (int q = 0; q < count; ++q) {
    passes[q] = make_pass(geoms[q], axis, W[q], in[q], out[q], epi, lamx[q], lamy[q], lamz[q], &kcontig);
    passes[q].cfg %= 3;  // the grouped kernel holds the double-buffered shapes
    const long long rows = (long long)passes[q].R1 * passes[q].R2;
    const int c = passes[q].cfg;
    begin[q + 1] = begin[q] + ((rows + cfg_bm(c) - 1) / cfg_bm(c)) * ((passes[q].n + cfg_bn(c) - 1) / cfg_bn(c));
  }
  if (begin[count] >= (1LL << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(dev_table, host_table, need, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  F32Group grp{count, static_cast<const F32Pass*>(dev_table),
               reinterpret_cast<const long long*>(static_cast<const char*>(dev_table) + (size_t)count * sizeof(F32Pass))};
  if (in_f64 && out_f64) return launch_f32_grouped<double, double>(grp, begin[count], kcontig, s);
  if (in_f64) return launch_f32_grouped<double, float>(grp, begin[count], kcontig, s);
  if (out_f64) return launch_f32_grouped<float, double>(grp, begin[count], kcontig, s);
  return launch_f32_grouped<float, float>(grp, begin[count], kcontig, s);
}

cudaError_t launch_mode_product_f32(const Geom& g, int axis, const float* W, const void* in, bool in_f64, void* out,
                                    bool out_f64, int epi, const double* lamx, const double* lamy, const double* lamz,
                                    cudaStream_t s) {
  if (epi == EPI_ACCUM && !out_f64) return cudaErrorInvalidValue;
  bool kcontig = false;
  const F32Pass p = make_pass(g, axis, W, in, out, epi, lamx, lamy, lamz, &kcontig);
  if (in_f64 && out_f64) return launch_f32<double, double>(p, kcontig, s);
  if (in_f64) return launch_f32<double, float>(p, kcontig, s);
  if (out_f64) return launch_f32<float, double>(p, kcontig, s);
  return launch_f32<float, float>(p, kcontig, s);
}

}  // namespace sem3d
