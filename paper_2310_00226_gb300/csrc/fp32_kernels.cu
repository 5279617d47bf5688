// FP32 CUDA-core mode product (the SEM3D_FP32 tier): FFMA with FP32 operands
// and accumulation, no tensor cores.  Same strided formulation as the FP64
// DMMA kernel (Section 2.4, Eq. 11-13: one Kronecker factor at a time, no
// transposes): C[row, o] = sum_t A[row, t] * W[o, t], rows enumerated by two
// loops (p < R1 stride s1, q < R2 stride s2), axis stride sm.
//
// CTA tile 128 rows x 128 outputs, K chunk 16, 256 threads with 8 x 8 outputs
// each (register tiling), operands staged in shared memory.
#include "sem3d_internal.h"

namespace sem3d {

namespace {

constexpr int F32_BM = 128, F32_BN = 128, F32_BK = 16;

struct F32Pass {
  const void* in;         // float or double (first pass of a solve)
  void* out;              // float, or double for the last pass
  const float* W;         // n x n row-major
  long long s1, s2, sm;
  int R1, R2, n;
  int epi;                // EPI_STORE / EPI_DIV / EPI_ACCUM (double output only)
  int nx, ny;
  const double *lamx, *lamy, *lamz;
  double c;
};

// One 128 x 128 output tile (row tile bx, output tile by) of pass p.
template <typename TIN, typename TOUT, bool KCONTIG>
__device__ __forceinline__ void f32_tile(const F32Pass& p, long long bx, int by) {
  __shared__ __align__(16) float As[F32_BK][F32_BM + 4];
  __shared__ __align__(16) float Ws[F32_BK][F32_BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // outputs tx*8.., rows ty*8..
  const long long rows = (long long)p.R1 * p.R2;
  const long long row0 = bx * F32_BM;
  const int o0 = by * F32_BN;
  const TIN* in = static_cast<const TIN*>(p.in);

  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  // The rows this thread loads are the same in every K chunk: decode them once.
  constexpr int LOADS = (F32_BM * F32_BK) / 256;
  long long abase[LOADS];
  int akk[LOADS], ar[LOADS];
#pragma unroll
  for (int it = 0; it < LOADS; ++it) {
    const int e = tid + it * 256;
    int r, kk;
    if (KCONTIG) { kk = e % F32_BK; r = e / F32_BK; }
    else { r = e % F32_BM; kk = e / F32_BM; }
    const long long row = row0 + r;
    akk[it] = kk;
    ar[it] = r;
    abase[it] = -1;
    if (row < rows) {
      const long long pp = row % p.R1, qq = row / p.R1;
      abase[it] = pp * p.s1 + qq * p.s2;
    }
  }

  for (int t0 = 0; t0 < p.n; t0 += F32_BK) {
#pragma unroll
    for (int it = 0; it < LOADS; ++it) {
      const int t = t0 + akk[it];
      float v = 0.f;
      if (abase[it] >= 0 && t < p.n) v = (float)in[abase[it] + (long long)t * p.sm];
      As[akk[it]][ar[it]] = v;
    }
#pragma unroll
    for (int it = 0; it < (F32_BN * F32_BK) / 256; ++it) {
      const int e = tid + it * 256;
      const int kk = e % F32_BK, o = e / F32_BK;
      const int oo = o0 + o, t = t0 + kk;
      Ws[kk][o] = (oo < p.n && t < p.n) ? p.W[(long long)oo * p.n + t] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < F32_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Ws[kk][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Ws[kk][tx * 8 + 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
  TOUT* out = static_cast<TOUT*>(p.out);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const long long row = row0 + ty * 8 + r;
    if (row >= rows) continue;
    const long long pp = row % p.R1, qq = row / p.R1;
    const long long base = pp * p.s1 + qq * p.s2;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int o = o0 + tx * 8 + c;
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

template <typename TIN, typename TOUT, bool KCONTIG>
__global__ void __launch_bounds__(256) mode_product_f32_kernel(F32Pass p) {
  f32_tile<TIN, TOUT, KCONTIG>(p, blockIdx.x, blockIdx.y);
}

// Grouped launch: one pass (the same axis and operand types) of many
// independent problems in a single grid.  Block b belongs to the problem q
// with block_begin[q] <= b < block_begin[q+1]; its tiles are numbered row
// tile fastest.
struct F32Group {
  int count;
  const F32Pass* passes;
  const long long* block_begin;  // count + 1 entries
};

template <typename TIN, typename TOUT, bool KCONTIG>
__global__ void __launch_bounds__(256) mode_product_f32_grouped_kernel(F32Group g) {
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
  const long long rt = (rows + F32_BM - 1) / F32_BM;
  f32_tile<TIN, TOUT, KCONTIG>(p, lb % rt, (int)(lb / rt));
}

template <typename TIN, typename TOUT>
cudaError_t launch_f32(const F32Pass& p, bool kcontig, cudaStream_t s) {
  const long long rows = (long long)p.R1 * p.R2;
  dim3 grid((unsigned)((rows + F32_BM - 1) / F32_BM), (unsigned)((p.n + F32_BN - 1) / F32_BN));
  if (kcontig) mode_product_f32_kernel<TIN, TOUT, true><<<grid, 256, 0, s>>>(p);
  else mode_product_f32_kernel<TIN, TOUT, false><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
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
  return p;
}

template <typename TIN, typename TOUT>
cudaError_t launch_f32_grouped(const F32Group& grp, long long blocks, bool kcontig, cudaStream_t s) {
  if (kcontig) mode_product_f32_grouped_kernel<TIN, TOUT, true><<<(unsigned)blocks, 256, 0, s>>>(grp);
  else mode_product_f32_grouped_kernel<TIN, TOUT, false><<<(unsigned)blocks, 256, 0, s>>>(grp);
  return cudaGetLastError();
}

}  // namespace

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
    const long long rows = (long long)passes[q].R1 * passes[q].R2;
    begin[q + 1] = begin[q] + ((rows + F32_BM - 1) / F32_BM) * ((passes[q].n + F32_BN - 1) / F32_BN);
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
  if (epi == EPI_ACCUM && !out_f64) return cudaErrorInvalidValue;
  const long long nxy = (long long)g.nx * g.ny;
  bool kcontig = false;
  if (axis == 0) {
    p.R1 = g.ny * g.nz; p.R2 = 1; p.s1 = g.nx; p.s2 = 0; p.sm = 1; p.n = g.nx; kcontig = true;
  } else if (axis == 1) {
    p.R1 = g.nx; p.R2 = g.nz; p.s1 = 1; p.s2 = nxy; p.sm = g.nx; p.n = g.ny;
  } else {
    p.R1 = (int)nxy; p.R2 = 1; p.s1 = 1; p.s2 = 0; p.sm = nxy; p.n = g.nz;
  }
  if (in_f64 && out_f64) return launch_f32<double, double>(p, kcontig, s);
  if (in_f64) return launch_f32<double, float>(p, kcontig, s);
  if (out_f64) return launch_f32<float, double>(p, kcontig, s);
  return launch_f32<float, float>(p, kcontig, s);
}

}  // namespace sem3d
