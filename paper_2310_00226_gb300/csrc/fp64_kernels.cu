// FP64 kernels: the plain-FP64 mode product (mma.sync DMMA), the banded
// FP64 operator / residual, and the FP64 -> split-bf16 conversion.
#include "sem3d_internal.h"

namespace sem3d {

namespace {

// ------------------------------------------------------------------ DMMA GEMM
//
// A mode product along one axis is a GEMM C[row, o] = sum_t A[row, t] W[o, t]
// where `row` enumerates the grid lines along that axis.  Rows are described
// by two loops (p < R1 with stride s1, q < R2 with stride s2) and the axis
// index has stride sm, so the same kernel serves x, y and z without
// transposes (Section 2.4, Eq. 11: the paper's tensorprod / pagemtimes).
//
// CTA tile: 64 rows x 64 outputs, K chunk 16; 8 warps, each owning 32 rows x
// 16 outputs = 4 x 2 fragments of mma.m8n8k4.f64.

constexpr int F64_BM = 64, F64_BN = 64, F64_BK = 16;

struct F64Pass {
  const double* in;
  double* out;
  const double* W;        // n x n row-major
  long long s1, s2, sm;   // strides of p, q and the axis index
  int R1, R2, n;          // row loops and axis length
  int epi;
  int nx, ny;             // to decode (i, j, l) for the division epilogue
  const double *lamx, *lamy, *lamz;
  double c;
};

template <bool KCONTIG>
__global__ void __launch_bounds__(256) mode_product_f64_kernel(F64Pass p) {
  __shared__ double As[F64_BK][F64_BM + 1];
  __shared__ double Bs[F64_BK][F64_BN + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long rows = (long long)p.R1 * p.R2;
  const long long row0 = (long long)blockIdx.x * F64_BM;
  const int o0 = blockIdx.y * F64_BN;
  const int wr = (warp & 1) * 32, wc = (warp >> 1) * 16;

  double acc[4][2][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

  for (int t0 = 0; t0 < p.n; t0 += F64_BK) {
    // A tile: 64 rows x 16 t.
#pragma unroll
    for (int it = 0; it < (F64_BM * F64_BK) / 256; ++it) {
      const int e = tid + it * 256;
      int r, kk;
      if (KCONTIG) { kk = e % F64_BK; r = e / F64_BK; }
      else { r = e % F64_BM; kk = e / F64_BM; }
      const long long row = row0 + r;
      const int t = t0 + kk;
      double v = 0.0;
      if (row < rows && t < p.n) {
        const long long pp = row % p.R1, qq = row / p.R1;
        v = p.in[pp * p.s1 + qq * p.s2 + (long long)t * p.sm];
      }
      As[kk][r] = v;
    }
    // W tile: 64 outputs x 16 t (row-major W, t contiguous).
#pragma unroll
    for (int it = 0; it < (F64_BN * F64_BK) / 256; ++it) {
      const int e = tid + it * 256;
      const int kk = e % F64_BK, o = e / F64_BK;
      const int oo = o0 + o, t = t0 + kk;
      Bs[kk][o] = (oo < p.n && t < p.n) ? p.W[(long long)oo * p.n + t] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k4 = 0; k4 < F64_BK; k4 += 4) {
      double afr[4], bfr[2];
#pragma unroll
      for (int a = 0; a < 4; ++a) afr[a] = As[k4 + (lane & 3)][wr + a * 8 + (lane >> 2)];
#pragma unroll
      for (int b = 0; b < 2; ++b) bfr[b] = Bs[k4 + (lane & 3)][wc + b * 8 + (lane >> 2)];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
          asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                       : "+d"(acc[a][b][0]), "+d"(acc[a][b][1])
                       : "d"(afr[a]), "d"(bfr[b]));
    }
    __syncthreads();
  }
  // Epilogue: fragment (a, b) holds rows wr + a*8 + lane/4, outputs
  // wc + b*8 + 2*(lane%4) + {0,1}.
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const long long row = row0 + wr + a * 8 + (lane >> 2);
    if (row >= rows) continue;
    const long long pp = row % p.R1, qq = row / p.R1;
    const long long base = pp * p.s1 + qq * p.s2;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int o = o0 + wc + b * 8 + 2 * (lane & 3) + h;
        if (o >= p.n) continue;
        const long long idx = base + (long long)o * p.sm;
        double v = acc[a][b][h];
        if (p.epi == EPI_DIV) {
          const long long i = idx % p.nx, jl = idx / p.nx;
          const long long j = jl % p.ny, l = jl / p.ny;
          v = v / (p.lamx[i] + p.lamy[j] + p.lamz[l] + p.c);
          p.out[idx] = v;
        } else if (p.epi == EPI_ACCUM) {
          p.out[idx] += v;
        } else {
          p.out[idx] = v;
        }
      }
  }
}

// ------------------------------------------------------------------ stencil
//
// (H_x (+) H_y (+) H_z) u with the banded H = M^{-1} S of each axis
// (Eq. 12): row i of H couples the nodes of the one or two elements that
// contain node i, stored as H[i][i+d], d in [-k, k].  One thread per node.

struct StencilArgs {
  const double* u;
  const double* f;
  double* out64;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  const double *Hx, *Hy, *Hz;
  const int *lox, *hix, *loy, *hiy, *loz, *hiz;
  int nx, ny, nz, k, Px, mode;
  double c;
  float* out32;        // MODE 3: FP32 residual at pitch Px, max |r| -> st slot 0
  F16State* st;
};

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

__global__ void __launch_bounds__(256) stencil_kernel(StencilArgs a) {
  const long long N = (long long)a.nx * a.ny * a.nz;
  const int bw = 2 * a.k + 1;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % a.nx);
    const long long jl = idx / a.nx;
    const int j = (int)(jl % a.ny), l = (int)(jl / a.ny);
    const double* u = a.u;
    double s = a.c * u[idx];
    // x: the band of row i (lanes of a warp sit on different rows of H_x).
    {
      const double* h = a.Hx + (long long)i * bw;
      const long long base = idx - i;
      for (int t = a.lox[i]; t <= a.hix[i]; ++t) s += h[t - i + a.k] * u[base + t];
    }
    // y
    {
      const double* h = a.Hy + (long long)j * bw;
      const long long base = idx - (long long)j * a.nx;
      for (int t = a.loy[j]; t <= a.hiy[j]; ++t) s += h[t - j + a.k] * u[base + (long long)t * a.nx];
    }
    // z
    {
      const double* h = a.Hz + (long long)l * bw;
      const long long pl = (long long)a.nx * a.ny;
      const long long base = idx - (long long)l * pl;
      for (int t = a.loz[l]; t <= a.hiz[l]; ++t) s += h[t - l + a.k] * u[base + (long long)t * pl];
    }
    if (a.mode == 0) {
      a.out64[idx] = s;
    } else {
      const double r = a.f[idx] - s;
      if (a.mode == 1) {
        a.out64[idx] = r;
      } else {
        const float rf = (float)r;
        const __nv_bfloat16 h16 = __float2bfloat16_rn(rf);
        const __nv_bfloat16 l16 = __float2bfloat16_rn(rf - __bfloat162float(h16));
        const long long o = (long long)i + (long long)a.Px * jl;
        a.hi[o] = h16;
        a.lo[o] = l16;
      }
    }
  }
}

// Element-wise variant of the same operator for a uniform mesh and
// 1 <= K <= 8.  Along x, one thread owns the K global nodes g = ex*K + q
// (q = 0..K-1) of element ex: node q = 0 is the vertex shared with element
// ex-1 (row of 2K+1 entries), q > 0 are the element's other nodes (K+1
// entries each).  The thread keeps the 2K+1 node values of elements ex-1 and
// ex in registers, and every thread runs the same fully unrolled loops, so
// the lanes of a warp never wait on each other's band lengths.  The rows of
// H depend only on q (table Hq, x table with c added on its diagonal).  The
// y and z bands are uniform across a warp (its lanes share j and l).
// Work per node: k+2 FMAs per axis on average (6 at k = 4), accumulated from
// f in residual modes.
template <int K, int MODE>
__global__ void __launch_bounds__(256) stencil_elem_kernel(StencilArgs a, const double* __restrict__ Hqx,
                                                           const double* __restrict__ Hqy,
                                                           const double* __restrict__ Hqz, int nex) {
  constexpr int BW = 2 * K + 1;
  const long long lines = (long long)a.ny * a.nz;
  const long long total = (long long)nex * lines;
  const long long plane = (long long)a.nx * a.ny;
  float rmax = 0.f;  // MODE 3: max |r| of this thread's nodes
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(t % nex);
    const long long jl = t / nex;
    const int j = (int)(jl % a.ny), l = (int)(jl / a.ny);
    const long long line = jl * a.nx;
    const int i0 = ex * K - 1;  // unknown index of node q = 0 (g = ex*K)
    // x window: global nodes (ex-1)K .. (ex+1)K -> unknowns i0-K .. i0+K
    double w[BW];
#pragma unroll
    for (int d = 0; d < BW; ++d) {
      const int i = i0 - K + d;
      w[d] = (i >= 0 && i < a.nx) ? __ldg(a.u + line + i) : 0.0;
    }
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int i = i0 + q;
      acc[q] = (MODE != 0 && i >= 0) ? __ldg(a.f + line + i) : 0.0;
    }
    // x part
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int dlo = (q == 0) ? -K : -q, dhi = (q == 0) ? K : K - q;
#pragma unroll
      for (int d = dlo; d <= dhi; ++d) {
        const double hv = __ldg(Hqx + q * BW + d + K);
        if (MODE == 0) acc[q] += hv * w[K + q + d];
        else acc[q] -= hv * w[K + q + d];
      }
    }
    // y part: row j of H_y, local index qy = (j+1) % K
    {
      const int qy = (j + 1) % K;
      const int dlo = (qy == 0) ? -K : -qy, dhi = (qy == 0) ? K : K - qy;
      for (int d = dlo; d <= dhi; ++d) {
        const int jj = j + d;
        if (jj < 0 || jj >= a.ny) continue;
        const double hv = __ldg(Hqy + qy * BW + d + K);
        const double* src = a.u + ((long long)l * a.ny + jj) * a.nx;
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int i = i0 + q;
          const double uv = (i >= 0) ? __ldg(src + i) : 0.0;
          if (MODE == 0) acc[q] += hv * uv;
          else acc[q] -= hv * uv;
        }
      }
    }
    // z part
    {
      const int qz = (l + 1) % K;
      const int dlo = (qz == 0) ? -K : -qz, dhi = (qz == 0) ? K : K - qz;
      for (int d = dlo; d <= dhi; ++d) {
        const int ll = l + d;
        if (ll < 0 || ll >= a.nz) continue;
        const double hv = __ldg(Hqz + qz * BW + d + K);
        const double* src = a.u + (long long)ll * plane + (long long)j * a.nx;
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int i = i0 + q;
          const double uv = (i >= 0) ? __ldg(src + i) : 0.0;
          if (MODE == 0) acc[q] += hv * uv;
          else acc[q] -= hv * uv;
        }
      }
    }
    if (MODE == 3) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const int i = i0 + q;
        if (i < 0) continue;
        const float rf = (float)acc[q];
        a.out32[(long long)i + (long long)a.Px * jl] = rf;
        rmax = fmaxf(rmax, fabsf(rf));
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int i = i0 + q;
      if (i < 0) continue;
      if (MODE != 2) {
        a.out64[line + i] = acc[q];
      } else {
        const float rf = (float)acc[q];
        const __nv_bfloat16 h16 = __float2bfloat16_rn(rf);
        const __nv_bfloat16 l16 = __float2bfloat16_rn(rf - __bfloat162float(h16));
        const long long o = (long long)i + (long long)a.Px * jl;
        a.hi[o] = h16;
        a.lo[o] = l16;
      }
    }
  }
  if (MODE == 3) {  // every lane of the warp gets here (after the loop)
    rmax = warp_max(rmax);
    if ((threadIdx.x & 31) == 0 && rmax > 0.f) atomicMax(&a.st->maxbits[0], __float_as_uint(rmax));
  }
}

template <int K>
cudaError_t launch_elem(const StencilArgs& a, const DevAxis* ax, int mode, cudaStream_t s) {
  const int nex = (a.nx + 1) / K;
  const long long total = (long long)nex * a.ny * a.nz;
  long long b = (total + 255) / 256;
  // One thread per work item (no grid-stride wrap): blocks are issued in
  // order, so the resident set sweeps the grid plane by plane and the z
  // neighbours of a plane are still in L2 when they are read again.
  if (b > 0x7FFFFFFFLL) b = 0x7FFFFFFFLL;
  const int grid = (int)(b < 1 ? 1 : b);
  if (mode == 0) stencil_elem_kernel<K, 0><<<grid, 256, 0, s>>>(a, ax[0].Hq, ax[1].Hq, ax[2].Hq, nex);
  else if (mode == 1) stencil_elem_kernel<K, 1><<<grid, 256, 0, s>>>(a, ax[0].Hq, ax[1].Hq, ax[2].Hq, nex);
  else if (mode == 2) stencil_elem_kernel<K, 2><<<grid, 256, 0, s>>>(a, ax[0].Hq, ax[1].Hq, ax[2].Hq, nex);
  else stencil_elem_kernel<K, 3><<<grid, 256, 0, s>>>(a, ax[0].Hq, ax[1].Hq, ax[2].Hq, nex);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ double-FP32 residual
//
// The same element-wise operator evaluated in double-FP32 arithmetic: every
// value is a pair hi + lo of FP32 numbers (about 48 significant bits).  FP32
// runs at ~70x the FP64 rate on this GPU, so a refinement sweep whose only
// job is to bring the error down to the level the final FP64 sweep removes
// can use it.  Products use the FMA error-free transformation
// (p = a*b, e = fma(a, b, -p)), sums the two-sum of the leading parts.

// Exact split of an FP64 value into hi (first 24 significant bits, truncated)
// and lo (the next 24, rounded) with integer operations only.  |x| < 2^-126
// gives (0, 0); 2^-126 <= |x| < 2^-74 gives lo = 0.
__device__ __forceinline__ void f64_to_df(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126) { hi = 0.f; lo = 0.f; return; }
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  hi = __uint_as_float(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29));
  if (e < -74) { lo = 0.f; return; }
  const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);  // value rem * 2^(e-52)
  const float scale = __uint_as_float((unsigned int)(e - 52 + 127) << 23);
  lo = __uint_as_float(__float_as_uint(__uint2float_rn(rem) * scale) | sign);
}

// (ah, al) -= (ch + cl [+ cl2]) * (uh + ul), dropping cl*ul and cl2*ul; the
// third coefficient term cl2 enters only when EXACT (else the 48-bit ch + cl).
// LO0: ul is zero (the solution right after the first solve), and the ch*ul
// term, exactly 0 there, is not formed (the same result).
template <bool EXACT = false, bool LO0 = false>
__device__ __forceinline__ void df_sub_prod(float& ah, float& al, float ch, float cl, float uh, float ul,
                                            float cl2 = 0.f) {
  const float p = ch * uh;
  const float e = fmaf(ch, uh, -p);
  const float t0 = fmaf(cl, uh, EXACT ? fmaf(cl2, uh, e) : e);
  const float t = LO0 ? t0 : fmaf(ch, ul, t0);
  const float s = ah - p;
  const float bb = s - ah;
  const float err = (ah - (s - bb)) - (p + bb);
  ah = s;
  al = al + (err - t);
}

struct DfArgs {
  const float* uh;
  const float* ul;
  const double* f;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  float* out32;        // if set: FP32 residual at pitch Px, max |r| -> st slot 0
  F16State* st;
  const float *Hxh, *Hxl, *Hyh, *Hyl, *Hzh, *Hzl;
  const float *Hxl2, *Hyl2, *Hzl2;  // third coefficient terms (read when EXACT)
  int nx, ny, nz, Px, nex;
};

template <int K, bool EXACT>
__global__ void __launch_bounds__(256) stencil_df_kernel(DfArgs a) {
  constexpr int BW = 2 * K + 1;
  const long long lines = (long long)a.ny * a.nz;
  const long long total = (long long)a.nex * lines;
  float rmax = 0.f;  // FP32 output: max |r| of this thread's nodes
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(t % a.nex);
    const long long jl = t / a.nex;
    const int j = (int)(jl % a.ny), l = (int)(jl / a.ny);
    const long long line = jl * a.nx;    // f (pitch nx)
    const long long uline = jl * a.Px;   // u (pitch Px)
    const int i0 = ex * K - 1;
    float wh[BW], wl[BW];
#pragma unroll
    for (int d = 0; d < BW; ++d) {
      const int i = i0 - K + d;
      const bool ok = i >= 0 && i < a.nx;
      wh[d] = ok ? __ldg(a.uh + uline + i) : 0.f;
      wl[d] = ok ? __ldg(a.ul + uline + i) : 0.f;
    }
    float ah[K], al[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int i = i0 + q;
      if (i >= 0) f64_to_df(__ldg(a.f + line + i), ah[q], al[q]);
      else { ah[q] = 0.f; al[q] = 0.f; }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int dlo = (q == 0) ? -K : -q, dhi = (q == 0) ? K : K - q;
#pragma unroll
      for (int d = dlo; d <= dhi; ++d)
        df_sub_prod<EXACT>(ah[q], al[q], __ldg(a.Hxh + q * BW + d + K), __ldg(a.Hxl + q * BW + d + K), wh[K + q + d],
                    wl[K + q + d], EXACT ? __ldg(a.Hxl2 + q * BW + d + K) : 0.f);
    }
    {
      const int qy = (j + 1) % K;
      const int dlo = (qy == 0) ? -K : -qy, dhi = (qy == 0) ? K : K - qy;
      for (int d = dlo; d <= dhi; ++d) {
        const int jj = j + d;
        if (jj < 0 || jj >= a.ny) continue;
        const float ch = __ldg(a.Hyh + qy * BW + d + K), cl = __ldg(a.Hyl + qy * BW + d + K);
        const float cl2 = EXACT ? __ldg(a.Hyl2 + qy * BW + d + K) : 0.f;
        const long long off = ((long long)l * a.ny + jj) * a.Px;
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int i = i0 + q;
          if (i < 0) continue;
          df_sub_prod<EXACT>(ah[q], al[q], ch, cl, __ldg(a.uh + off + i), __ldg(a.ul + off + i), cl2);
        }
      }
    }
    {
      const int qz = (l + 1) % K;
      const int dlo = (qz == 0) ? -K : -qz, dhi = (qz == 0) ? K : K - qz;
      for (int d = dlo; d <= dhi; ++d) {
        const int ll = l + d;
        if (ll < 0 || ll >= a.nz) continue;
        const float ch = __ldg(a.Hzh + qz * BW + d + K), cl = __ldg(a.Hzl + qz * BW + d + K);
        const float cl2 = EXACT ? __ldg(a.Hzl2 + qz * BW + d + K) : 0.f;
        const long long off = ((long long)ll * a.ny + j) * a.Px;
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int i = i0 + q;
          if (i < 0) continue;
          df_sub_prod<EXACT>(ah[q], al[q], ch, cl, __ldg(a.uh + off + i), __ldg(a.ul + off + i), cl2);
        }
      }
    }
    if (a.out32) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const int i = i0 + q;
        if (i < 0) continue;
        const float rf = ah[q] + al[q];
        a.out32[(long long)i + (long long)a.Px * jl] = rf;
        rmax = fmaxf(rmax, fabsf(rf));
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int i = i0 + q;
      if (i < 0) continue;
      const float rf = ah[q] + al[q];
      const __nv_bfloat16 h16 = __float2bfloat16_rn(rf);
      const __nv_bfloat16 l16 = __float2bfloat16_rn(rf - __bfloat162float(h16));
      const long long o = (long long)i + (long long)a.Px * jl;
      a.hi[o] = h16;
      a.lo[o] = l16;
    }
  }
  if (a.out32) {  // every lane of the warp gets here (after the loop)
    rmax = warp_max(rmax);
    if ((threadIdx.x & 31) == 0 && rmax > 0.f) atomicMax(&a.st->maxbits[0], __float_as_uint(rmax));
  }
}

// Rows of H per local index for the vector residual (k <= 4), as kernel
// parameters: the x rows are read at compile-time offsets (no load
// instructions), the y and z rows at warp-uniform offsets.
struct DfCoef {
  float h[3][4 * 9];
  float l[3][4 * 9];
  float l2[3][4 * 9];  // third terms (used when EXACT)
};

// Double-FP32 residual for k in {1, 2, 4}.  A lane handles the 4 consecutive
// nodes i = 4c .. 4c+3 of one (j, l) line -- one float4 of each of u_hi and
// u_lo, whose rows (pitch Px, a multiple of 16) are 16-byte aligned and whose
// pad columns are zero -- and a warp handles one line, its lanes striding over
// the line's Px/4 chunks.  Since 4 % k == 0, node 4c+p has the local index
// (p+1) % k for every c: each position's x row of H is known at compile time
// and only its band is summed.  The y and z rows depend on the warp's (j, l).
template <int K, bool EXACT, bool LO0>
__global__ void __launch_bounds__(256, 4) stencil_df4_kernel(DfArgs a, const __grid_constant__ DfCoef cf) {
  constexpr int BW = 2 * K + 1;
  const int lane = threadIdx.x & 31;
  const long long lines = (long long)a.ny * a.nz;
  const int chunks = a.Px >> 2;
  const long long splane = (long long)a.ny * chunks;  // float4 per z-plane
  const float4* UH = reinterpret_cast<const float4*>(a.uh);
  const float4* UL = reinterpret_cast<const float4*>(a.ul);
  float rmax = 0.f;
  for (long long line = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); line < lines;
       line += (long long)gridDim.x * 8) {  // warp-uniform
    const int j = (int)(line % a.ny), l = (int)(line / a.ny);
    const int qy = (j + 1) % K, qz = (l + 1) % K;
    const int ylo = (qy == 0) ? -K : -qy, yhi = (qy == 0) ? K : K - qy;
    const int zlo = (qz == 0) ? -K : -qz, zhi = (qz == 0) ? K : K - qz;
    const long long row4 = line * chunks;
    const double* frow = a.f + line * a.nx;
    for (int c = lane; c < chunks; c += 32) {
      const int i0 = 4 * c;
      float ah[4], al[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (i0 + p < a.nx) f64_to_df(__ldg(frow + i0 + p), ah[p], al[p]);
        else { ah[p] = 0.f; al[p] = 0.f; }
      }
      // x: nodes i0-4 .. i0+7 (the neighbouring chunks; zero outside the line)
      float wh[12], wl[12];
      {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 ph = c > 0 ? __ldg(UH + row4 + c - 1) : z4, pl = (c > 0 && !LO0) ? __ldg(UL + row4 + c - 1) : z4;
        const float4 ch = __ldg(UH + row4 + c), cl = LO0 ? z4 : __ldg(UL + row4 + c);
        const float4 nh = c + 1 < chunks ? __ldg(UH + row4 + c + 1) : z4;
        const float4 nl = (c + 1 < chunks && !LO0) ? __ldg(UL + row4 + c + 1) : z4;
        wh[0] = ph.x; wh[1] = ph.y; wh[2] = ph.z; wh[3] = ph.w; wh[4] = ch.x; wh[5] = ch.y;
        wh[6] = ch.z; wh[7] = ch.w; wh[8] = nh.x; wh[9] = nh.y; wh[10] = nh.z; wh[11] = nh.w;
        wl[0] = pl.x; wl[1] = pl.y; wl[2] = pl.z; wl[3] = pl.w; wl[4] = cl.x; wl[5] = cl.y;
        wl[6] = cl.z; wl[7] = cl.w; wl[8] = nl.x; wl[9] = nl.y; wl[10] = nl.z; wl[11] = nl.w;
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int q = (p + 1) % K;
        const int dlo = (q == 0) ? -K : -q, dhi = (q == 0) ? K : K - q;
#pragma unroll
        for (int d = -K; d <= K; ++d)
          if (d >= dlo && d <= dhi)  // compile-time after unrolling
            df_sub_prod<EXACT, LO0>(ah[p], al[p], cf.h[0][q * BW + d + K], cf.l[0][q * BW + d + K], wh[4 + p + d], wl[4 + p + d],
                        EXACT ? cf.l2[0][q * BW + d + K] : 0.f);
      }
      // y and z: the rows of the neighbouring lines, one float4 pair per row
#pragma unroll
      for (int d = -K; d <= K; ++d) {
        if (d < ylo || d > yhi || j + d < 0 || j + d >= a.ny) continue;  // warp-uniform
        const float chh = cf.h[1][qy * BW + d + K], cll = cf.l[1][qy * BW + d + K];
        const float cl2 = EXACT ? cf.l2[1][qy * BW + d + K] : 0.f;
        const float4 vh = __ldg(UH + row4 + (long long)d * chunks + c);
        const float4 vl = LO0 ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(UL + row4 + (long long)d * chunks + c);
        df_sub_prod<EXACT, LO0>(ah[0], al[0], chh, cll, vh.x, vl.x, cl2);
        df_sub_prod<EXACT, LO0>(ah[1], al[1], chh, cll, vh.y, vl.y, cl2);
        df_sub_prod<EXACT, LO0>(ah[2], al[2], chh, cll, vh.z, vl.z, cl2);
        df_sub_prod<EXACT, LO0>(ah[3], al[3], chh, cll, vh.w, vl.w, cl2);
      }
#pragma unroll
      for (int d = -K; d <= K; ++d) {
        if (d < zlo || d > zhi || l + d < 0 || l + d >= a.nz) continue;  // warp-uniform
        const float chh = cf.h[2][qz * BW + d + K], cll = cf.l[2][qz * BW + d + K];
        const float cl2 = EXACT ? cf.l2[2][qz * BW + d + K] : 0.f;
        const float4 vh = __ldg(UH + row4 + (long long)d * splane + c);
        const float4 vl = LO0 ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(UL + row4 + (long long)d * splane + c);
        df_sub_prod<EXACT, LO0>(ah[0], al[0], chh, cll, vh.x, vl.x, cl2);
        df_sub_prod<EXACT, LO0>(ah[1], al[1], chh, cll, vh.y, vl.y, cl2);
        df_sub_prod<EXACT, LO0>(ah[2], al[2], chh, cll, vh.z, vl.z, cl2);
        df_sub_prod<EXACT, LO0>(ah[3], al[3], chh, cll, vh.w, vl.w, cl2);
      }
      float r[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) r[p] = (i0 + p < a.nx) ? ah[p] + al[p] : 0.f;  // pads stay zero
      const long long o = line * a.Px + i0;
      if (a.out32) {
        *reinterpret_cast<float4*>(a.out32 + o) = make_float4(r[0], r[1], r[2], r[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) rmax = fmaxf(rmax, fabsf(r[p]));
      } else {
        uint32_t hw[2], lw[2];
#pragma unroll
        for (int p = 0; p < 4; p += 2) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(r[p]), h1 = __float2bfloat16_rn(r[p + 1]);
          const __nv_bfloat16 l0 = __float2bfloat16_rn(r[p] - __bfloat162float(h0));
          const __nv_bfloat16 l1 = __float2bfloat16_rn(r[p + 1] - __bfloat162float(h1));
          hw[p / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
          lw[p / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        *reinterpret_cast<uint2*>(a.hi + o) = make_uint2(hw[0], hw[1]);
        *reinterpret_cast<uint2*>(a.lo + o) = make_uint2(lw[0], lw[1]);
      }
    }
  }
  if (a.out32) {  // every lane of the warp gets here
    rmax = warp_max(rmax);
    if ((threadIdx.x & 31) == 0 && rmax > 0.f) atomicMax(&a.st->maxbits[0], __float_as_uint(rmax));
  }
}

template <int K>
cudaError_t launch_df4(const DfArgs& a, const DevAxis* ax, bool exact, bool lo_zero, cudaStream_t s) {
  DfCoef cf{};
  for (int w = 0; w < 3; ++w)
    for (int e = 0; e < K * (2 * K + 1); ++e) {
      cf.h[w][e] = ax[w].Hq_hi_host[e];
      cf.l[w][e] = ax[w].Hq_lo_host[e];
      cf.l2[w][e] = ax[w].Hq_lo2_host[e];
    }
  // One block per 8 consecutive lines and no grid stride: the resident blocks
  // then sweep the grid plane by plane, so the rows 1..K planes away that a
  // warp reads were read moments earlier by other warps and are still in L2.
  const long long lines = (long long)a.ny * a.nz;
  long long blocks = (lines + 7) / 8;
  if (blocks > 0x7FFFFFFFLL) blocks = 0x7FFFFFFFLL;
  const unsigned g = (unsigned)(blocks < 1 ? 1 : blocks);
  if (exact) {
    if (lo_zero) stencil_df4_kernel<K, true, true><<<g, 256, 0, s>>>(a, cf);
    else stencil_df4_kernel<K, true, false><<<g, 256, 0, s>>>(a, cf);
  } else {
    if (lo_zero) stencil_df4_kernel<K, false, true><<<g, 256, 0, s>>>(a, cf);
    else stencil_df4_kernel<K, false, false><<<g, 256, 0, s>>>(a, cf);
  }
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_df(const DfArgs& a, bool exact, cudaStream_t s) {
  const long long total = (long long)a.nex * a.ny * a.nz;
  long long b = (total + 255) / 256;
  if (b > 0x7FFFFFFFLL) b = 0x7FFFFFFFLL;  // one thread per work item (see launch_elem)
  if (exact) stencil_df_kernel<K, true><<<(int)(b < 1 ? 1 : b), 256, 0, s>>>(a);
  else stencil_df_kernel<K, false><<<(int)(b < 1 ? 1 : b), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// Zero the pad columns i in [nx, Px) of a split array (the stencil writes
// only i < nx).
__global__ void zero_pads_kernel(__nv_bfloat16* hi, __nv_bfloat16* lo, int nx, int Px, long long lines) {
  const int w = Px - nx;
  const long long total = lines * w;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long line = e / w;
    const long long o = line * Px + nx + (e % w);
    hi[o] = __float2bfloat16_rn(0.f);
    lo[o] = __float2bfloat16_rn(0.f);
  }
}

// FP64 (dense, pitch nx) -> bf16 hi + lo (pitch Px, zero pads):
// hi = bf16(x), lo = bf16(x - hi), x rounded to FP32 first.  Blocks walk the
// (j, l) lines; a lane converts 4 consecutive entries and writes them as one
// 8-byte store per array (rows of pitch Px, a multiple of 16, are aligned).
// With emax set, the largest biased FP64 exponent of the input also goes to
// *emax (atomicMax; the fixed-point residual's scale of f).
__global__ void __launch_bounds__(256) split_kernel(const double* in, __nv_bfloat16* hi, __nv_bfloat16* lo, int nx,
                                                    int Px, long long lines, int* emax) {
  const int chunks = Px >> 2;
  unsigned int m = 0;
  for (long long line = blockIdx.x; line < lines; line += gridDim.x) {
    const double* row = in + line * nx;
    uint2* hrow = reinterpret_cast<uint2*>(hi + line * Px);
    uint2* lrow = reinterpret_cast<uint2*>(lo + line * Px);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
      uint32_t hw[2], lw[2];
#pragma unroll
      for (int p = 0; p < 4; p += 2) {
        const int i = 4 * c + p;
        const double d0 = i < nx ? row[i] : 0.0, d1 = i + 1 < nx ? row[i + 1] : 0.0;
        m = max(m, max((unsigned int)(__double_as_longlong(d0) >> 52) & 0x7FFu,
                       (unsigned int)(__double_as_longlong(d1) >> 52) & 0x7FFu));
        const float x0 = f64_to_f32_rn(d0), x1 = f64_to_f32_rn(d1);
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
        hw[p / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        lw[p / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
      }
      hrow[c] = make_uint2(hw[0], hw[1]);
      lrow[c] = make_uint2(lw[0], lw[1]);
    }
  }
  if (emax) {  // every lane of the block gets here
    m = __reduce_max_sync(0xFFFFFFFFu, m);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(emax, (int)m);
  }
}

// Grid of a streaming (grid-stride) kernel: enough blocks to fill the GPU a
// few times over; each thread then walks the arrays in order.
int grid_for(long long work, int per_block) {
  long long b = (work + per_block - 1) / per_block;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_mode_product_f64(const Geom& g, int axis, const double* W, const double* in, double* out, int epi,
                                    const double* lamx, const double* lamy, const double* lamz, cudaStream_t s) {
  F64Pass p{};
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
  bool kcontig = false;
  if (axis == 0) {         // rows = (j,l) lines, t = i contiguous
    p.R1 = g.ny * g.nz; p.R2 = 1; p.s1 = g.nx; p.s2 = 0; p.sm = 1; p.n = g.nx; kcontig = true;
  } else if (axis == 1) {  // rows = (i, l), t = j
    p.R1 = g.nx; p.R2 = g.nz; p.s1 = 1; p.s2 = nxy; p.sm = g.nx; p.n = g.ny;
  } else {                 // rows = (i,j) plane, t = l
    p.R1 = (int)nxy; p.R2 = 1; p.s1 = 1; p.s2 = 0; p.sm = nxy; p.n = g.nz;
  }
  const long long rows = (long long)p.R1 * p.R2;
  dim3 grid((unsigned)((rows + F64_BM - 1) / F64_BM), (unsigned)((p.n + F64_BN - 1) / F64_BN));
  if (kcontig) mode_product_f64_kernel<true><<<grid, 256, 0, s>>>(p);
  else mode_product_f64_kernel<false><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_stencil(const Geom& g, int k, const DevAxis* ax, const double* u, const double* f, double* out64,
                           __nv_bfloat16* out_hi, __nv_bfloat16* out_lo, int mode, cudaStream_t s) {
  StencilArgs a{};
  a.u = u; a.f = f; a.out64 = out64; a.hi = out_hi; a.lo = out_lo;
  a.Hx = ax[0].Hband; a.Hy = ax[1].Hband; a.Hz = ax[2].Hband;
  a.lox = ax[0].band_lo; a.hix = ax[0].band_hi;
  a.loy = ax[1].band_lo; a.hiy = ax[1].band_hi;
  a.loz = ax[2].band_lo; a.hiz = ax[2].band_hi;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.k = k; a.Px = g.Px; a.mode = mode; a.c = g.c;
  const long long N = (long long)g.nx * g.ny * g.nz;
  cudaError_t e;
  switch (g.bc == 0 ? k : 0) {  // the element-pattern kernels assume Dirichlet rows
    case 1: e = launch_elem<1>(a, ax, mode, s); break;
    case 2: e = launch_elem<2>(a, ax, mode, s); break;
    case 3: e = launch_elem<3>(a, ax, mode, s); break;
    case 4: e = launch_elem<4>(a, ax, mode, s); break;
    case 5: e = launch_elem<5>(a, ax, mode, s); break;
    case 6: e = launch_elem<6>(a, ax, mode, s); break;
    case 7: e = launch_elem<7>(a, ax, mode, s); break;
    case 8: e = launch_elem<8>(a, ax, mode, s); break;
    default:  // higher degrees and Neumann data: one thread per node, per-row band ranges
      stencil_kernel<<<(int)((N + 255) / 256 < 0x7FFFFFFF ? (N + 255) / 256 : 0x7FFFFFFF), 256, 0, s>>>(a);
      e = cudaGetLastError();
  }
  if (e != cudaSuccess || mode != 2 || g.Px == g.nx) return e;
  const long long lines = (long long)g.ny * g.nz;
  zero_pads_kernel<<<grid_for(lines * (g.Px - g.nx), 256), 256, 0, s>>>(out_hi, out_lo, g.nx, g.Px, lines);
  return cudaGetLastError();
}

cudaError_t launch_stencil_df(const Geom& g, int k, const DevAxis* ax, DfBuffers u, const double* f,
                              __nv_bfloat16* out_hi, __nv_bfloat16* out_lo, cudaStream_t s, float* out32,
                              F16State* st, bool exact_coef, bool lo_zero) {
  if (g.bc != 0) return cudaErrorInvalidValue;  // element-pattern rows (Dirichlet) only
  DfArgs a{};
  a.uh = u.hi; a.ul = u.lo; a.f = f; a.hi = out_hi; a.lo = out_lo;
  a.out32 = out32; a.st = st;
  a.Hxh = ax[0].Hq_hi; a.Hxl = ax[0].Hq_lo;
  a.Hyh = ax[1].Hq_hi; a.Hyl = ax[1].Hq_lo;
  a.Hzh = ax[2].Hq_hi; a.Hzl = ax[2].Hq_lo;
  if (exact_coef) { a.Hxl2 = ax[0].Hq_lo2; a.Hyl2 = ax[1].Hq_lo2; a.Hzl2 = ax[2].Hq_lo2; }
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.Px = g.Px;
  a.nex = (g.nx + 1) / k;
  cudaError_t e;
  switch (k) {
    case 1: return launch_df4<1>(a, ax, exact_coef, lo_zero, s);  // pads written as zeros
    case 2: return launch_df4<2>(a, ax, exact_coef, lo_zero, s);
    case 4: return launch_df4<4>(a, ax, exact_coef, lo_zero, s);
    case 3: e = launch_df<3>(a, exact_coef, s); break;
    case 5: e = launch_df<5>(a, exact_coef, s); break;
    case 6: e = launch_df<6>(a, exact_coef, s); break;
    case 7: e = launch_df<7>(a, exact_coef, s); break;
    case 8: e = launch_df<8>(a, exact_coef, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || g.Px == g.nx || out32) return e;
  const long long lines = (long long)g.ny * g.nz;
  zero_pads_kernel<<<grid_for(lines * (g.Px - g.nx), 256), 256, 0, s>>>(out_hi, out_lo, g.nx, g.Px, lines);
  return cudaGetLastError();
}

cudaError_t launch_stencil_f32out(const Geom& g, int k, const DevAxis* ax, const double* u, const double* f,
                                  float* out32, F16State* st, cudaStream_t s) {
  if (k < 1 || k > 8 || g.bc != 0) return cudaErrorInvalidValue;
  StencilArgs a{};
  a.u = u; a.f = f; a.out32 = out32; a.st = st;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.k = k; a.Px = g.Px; a.mode = 3; a.c = g.c;
  switch (k) {
    case 1: return launch_elem<1>(a, ax, 3, s);
    case 2: return launch_elem<2>(a, ax, 3, s);
    case 3: return launch_elem<3>(a, ax, 3, s);
    case 4: return launch_elem<4>(a, ax, 3, s);
    case 5: return launch_elem<5>(a, ax, 3, s);
    case 6: return launch_elem<6>(a, ax, 3, s);
    case 7: return launch_elem<7>(a, ax, 3, s);
    default: return launch_elem<8>(a, ax, 3, s);
  }
}

// ------------------------------------------------------------------ F16X3 split
__global__ void __launch_bounds__(256) absmax_f64_kernel(const double* in, long long N, F16State* st) {
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, (float)fabs(in[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&st->maxbits[0], __float_as_uint(m));
}

// hi + lo = fp16 split of x * 2^e, e from slot 0's max (largest |x 2^e| near
// 2^15 < 65504); fp16 subnormals keep the absolute error below 2^-24 of 2^e.
template <bool IN64>
__global__ void __launch_bounds__(256) split_f16_kernel(const void* in, __half* hi, __half* lo, int nx, int Px,
                                                        long long lines, F16State* st) {
  const float mx = __uint_as_float(st->maxbits[0]);
  int e = 0;
  if (mx > 0.f && isfinite(mx)) {
    e = ilogbf(32768.f / mx);
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->e[0] = e;
  const float sc = __int_as_float((e + 127) << 23);
  const long long total = lines * Px;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long line = idx / Px;
    const int i = (int)(idx - line * Px);
    float x = 0.f;
    if (i < nx) x = IN64 ? f64_to_f32_rn(static_cast<const double*>(in)[line * nx + i]) : static_cast<const float*>(in)[idx];
    x *= sc;
    const __half h = __float2half_rn(x);
    hi[idx] = h;
    lo[idx] = __float2half_rn(x - __half2float(h));
  }
}

cudaError_t launch_absmax_f64(const Geom& g, const double* in, F16State* st, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  absmax_f64_kernel<<<grid_for(N, 256), 256, 0, s>>>(in, N, st);
  return cudaGetLastError();
}

cudaError_t launch_split_f16(const Geom& g, const void* in, bool in_f64, __half* hi, __half* lo, F16State* st,
                             cudaStream_t s) {
  const long long lines = (long long)g.ny * g.nz;
  if (in_f64) split_f16_kernel<true><<<grid_for(lines * g.Px, 256), 256, 0, s>>>(in, hi, lo, g.nx, g.Px, lines, st);
  else split_f16_kernel<false><<<grid_for(lines * g.Px, 256), 256, 0, s>>>(in, hi, lo, g.nx, g.Px, lines, st);
  return cudaGetLastError();
}

cudaError_t launch_split(const Geom& g, const double* in, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s,
                         int* emax) {
  const long long lines = (long long)g.ny * g.nz;
  const long long blocks = lines < 152LL * 16 ? (lines < 1 ? 1 : lines) : 152LL * 16;
  split_kernel<<<(int)blocks, 256, 0, s>>>(in, hi, lo, g.nx, g.Px, lines, emax);
  return cudaGetLastError();
}

}  // namespace sem3d
