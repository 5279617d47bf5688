// Refinement residual r = f - (c + H_x (+) H_y (+) H_z) u (Eq. 12, the
// banded operator of each axis) evaluated exactly in 64-bit integer fixed
// point on the integer pipe instead of the FP64 pipe.
//
// Why: on this GPU an FP64 FMA issues at ~1.7 lanes per clock per SM and a
// 32 x 32 -> 64-bit integer multiply-add (mad.wide.s32) at ~14, while the
// FP64 residual needs 18 FMAs per node (k = 4) and keeps the FP64 pipe
// saturated.
//
// Representation.  With one power-of-two scale for the whole field, u is held
// as U = round(u 2^s) with |U| <= 2^57 and every row of H (all three axes and
// c, sharing one scale) as C + E 2^-14 with integers C = round(H 2^t),
// whose magnitudes over the terms of any node sum to about 2^58, and E the
// rounded fraction H 2^t - C.  U and C are split into balanced chunks
// X = Xh 2^28 + Xl, Xl in [-2^27, 2^27):
//   C U = Ch Uh 2^56 + (Ch Ul + Cl Uh) 2^28 + Cl Ul.
// Per node, two int64 sums take the first two parts exactly (three
// mad.wide.s32 per term; they stay below 2^60 and 2^62) and an int32 sum Q
// the fraction correction E round(Uh 2^-17) (full-rate 32-bit multiply-adds);
// the last part, below 2^54 per term and of mean zero, is dropped.  The
// correction joins the 2^28 sum before its one rounding, f is rounded to the
// same fixed point, the difference F - T is exact, and the residual is
// converted to FP32 and split to bf16 (the split tiers' next solve reads it
// so) or to FP64 (the TF32 tier's).
//
// Every rounding is to nearest: the operator's conditioning amplifies the
// smooth (low-frequency) part of a residual error by up to 1/lambda_min, so a
// rounding that is biased, or one applied to a quantity that changes slowly
// from node to node (the small correction sum rounded on its own), leaves a
// coherent error that grows with the grid; the rows' fractions matter for
// the same reason (an error in a row sum acts like a change of c).  An exact-
// integer model of this arithmetic (tests/test_fixed_point_model_cpu.py),
// against exact rational residuals and propagated through the solve: the
// result's error is no larger than that of FP64 residuals, also with
// lambda_min + c a thousandth of lambda_min.
// The error is absolute (one scale per field): nodes where |u| is far below
// max |u| get the field's resolution, not FP64's relative one.
//
// Mirror symmetry: on a uniform mesh the row of H at an element vertex is
// symmetric in the offset d, and so is the row of the element's midpoint
// (even k).  Those rows are applied as C_d (U_{+d} + U_{-d}) + (C_{-d} - C_d)
// U_{-d}: the correction C_{-d} - C_d (a few units: the FP64 rows are
// symmetric up to rounding) costs one multiply-add instead of three and keeps
// the operator exactly that of the FP64 rows.
#include "sem3d_internal.h"

#include <cmath>

namespace sem3d {

namespace {

constexpr int kChunk = 28;
constexpr long long kHalf = 1LL << (kChunk - 1);

constexpr int kFracBits = 14;   // E = round((H 2^t - C) 2^14)
constexpr int kCorrShift = 17;  // the correction multiplies E by round(Uh 2^-17)

// round(x 2^s) (halves away from zero) for |x| 2^s < 2^62 (the callers keep
// it below 2^61); zero and subnormal inputs give 0.  Integer operations only.
__device__ __forceinline__ long long f64_to_fixed(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = e - 1075 + s;
  unsigned long long v;
  if (e == 0 || sh <= -64) v = 0;
  else if (sh >= 0) v = sh < 10 ? m << sh : 0;  // sh <= 8 under the callers' bounds
  else v = (m + (1ull << (-sh - 1))) >> (-sh);
  return (b >> 63) ? -(long long)v : (long long)v;
}

__device__ __forceinline__ int corr_u(int uh) { return (uh + (1 << (kCorrShift - 1))) >> kCorrShift; }

// R 2^X as FP32, truncated to 24 bits; below the normal range: signed zero.
__device__ __forceinline__ float fixed_to_f32(long long R, int X) {
  if (R == 0) return 0.f;
  const unsigned int sign = R < 0 ? 0x80000000u : 0u;
  const unsigned long long mag = R < 0 ? (unsigned long long)(-R) : (unsigned long long)R;
  const int lz = __clzll((long long)mag);
  const unsigned int mant = (unsigned int)((mag << lz) >> 40);  // leading one at bit 23
  const int be = 63 - lz + X + 127;
  if (be <= 0) return __uint_as_float(sign);
  if (be >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned int)be << 23) | (mant & 0x7FFFFFu));
}

__device__ __forceinline__ int biased_exp(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

// Largest biased FP64 exponent of |in[0 .. N)| -> atomicMax(*slot): an upper
// bound |x| < 2^(e - 1022) for every element (2047 flags Inf / NaN).
__global__ void __launch_bounds__(256) max_exponent_kernel(const double* __restrict__ in, long long N, int* slot) {
  int m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    m = max(m, biased_exp(__ldg(in + i)));
  m = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned int)m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(slot, m);
}

// The scale exponent s of U = round(u 2^s): |U| <= 2^57 and
// |F| = |round(f 2^(s+t-56))| <= 2^61 (state[0], state[1]: the max biased
// exponents of u and f, so |u| < 2^(state[0] - 1022)).
__device__ __forceinline__ int fixed_scale(const int* state, int t) {
  const int eu = state[0], ef = state[1];
  return min(1079 - eu, 1139 - t - ef);
}

// u (pitch nx) -> Uh, Ul (pitch Px, 16-byte rows, pad columns zero).  A
// thread converts 4 consecutive nodes of one line.
__global__ void __launch_bounds__(256) to_fixed_kernel(const double* __restrict__ u, int* __restrict__ Uh,
                                                       int* __restrict__ Ul, int nx, int Px, long long lines,
                                                       const int* __restrict__ state, int t) {
  const int chunks = Px >> 2;
  const long long total = lines * chunks;
  const int s = fixed_scale(state, t);
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    const long long line = w / chunks;
    const int i0 = (int)(w - line * chunks) * 4;
    const double* src = u + line * nx;
    int h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const long long U = (i0 + p < nx) ? f64_to_fixed(__ldg(src + i0 + p), s) : 0;
      const long long hh = (U + kHalf) >> kChunk;  // |Uh| <= 2^29
      h[p] = (int)hh;
      l[p] = (int)(U - (hh << kChunk));
    }
    const long long o = line * Px + i0;
    *reinterpret_cast<int4*>(Uh + o) = make_int4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<int4*>(Ul + o) = make_int4(l[0], l[1], l[2], l[3]);
  }
}

// P2 += Ch Uh, P1 += Ch Ul + Cl Uh for the 4 nodes of a lane.
__device__ __forceinline__ void fx_term(long long (&P2)[4], long long (&P1)[4], int ch, int cl, const int4& uh,
                                        const int4& ul) {
  P2[0] += (long long)ch * uh.x; P1[0] += (long long)ch * ul.x; P1[0] += (long long)cl * uh.x;
  P2[1] += (long long)ch * uh.y; P1[1] += (long long)ch * ul.y; P1[1] += (long long)cl * uh.y;
  P2[2] += (long long)ch * uh.z; P1[2] += (long long)ch * ul.z; P1[2] += (long long)cl * uh.z;
  P2[3] += (long long)ch * uh.w; P1[3] += (long long)ch * ul.w; P1[3] += (long long)cl * uh.w;
}

__device__ __forceinline__ int4 add4(const int4& a, const int4& b) {
  return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// One node's scalar term (x part): P2 += Ch uh, P1 += Ch ul + Cl uh.
__device__ __forceinline__ void fx1(long long& P2, long long& P1, int ch, int cl, int uh, int ul) {
  P2 += (long long)ch * uh;
  P1 += (long long)ch * ul;
  P1 += (long long)cl * uh;
}

// Fixed-point residual for k in {1, 2, 4} with Dirichlet rows.  Layout as
// the double-FP32 vector residual: a warp per (j, l) line, a lane per 4
// consecutive nodes i = 4c .. 4c+3 (one int4 of Uh and one of Ul); since
// 4 % k == 0 node 4c+p has local index (p+1) % k, so the x rows and their
// folding are known at compile time.  The y and z rows depend on the warp's
// (j, l) and are read from the term tables.
template <int K>
__global__ void __launch_bounds__(256, 4) stencil_fix4_kernel(FixArgs a, const __grid_constant__ FixCoef cf) {
  constexpr int BW = 2 * K + 1;
  const int lane = threadIdx.x & 31;
  const long long lines = (long long)a.ny * a.nz;
  const int chunks = a.Px >> 2;
  const long long splane = (long long)a.ny * chunks;  // int4 per z-plane
  const int4* UH = reinterpret_cast<const int4*>(a.Uh);
  const int4* UL = reinterpret_cast<const int4*>(a.Ul);
  const int s = fixed_scale(a.state, cf.t);
  const int sF = s + cf.t - 56;  // F = trunc(f 2^sF), in the units of T
  const int X = -sF;             // r = R 2^X
  const bool finite = a.state[0] < 2047 && a.state[1] < 2047;
  for (long long line = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); line < lines;
       line += (long long)gridDim.x * 8) {  // warp-uniform
    const int j = (int)(line % a.ny), l = (int)(line / a.ny);
    const int qy = (j + 1) % K, qz = (l + 1) % K;
    const long long row4 = line * chunks;
    const double* frow = a.f + line * a.nx;
    for (int c = lane; c < chunks; c += 32) {
      const int i0 = 4 * c;
      long long P2[4] = {0, 0, 0, 0}, P1[4] = {0, 0, 0, 0};
      int Q[4] = {0, 0, 0, 0};  // fraction corrections (units of 2^31)
      // x: nodes i0-4 .. i0+7 (the neighbouring chunks; zero outside the line)
      int wh[12], wl[12];
      {
        const int4 z4 = make_int4(0, 0, 0, 0);
        const int4 ph = c > 0 ? __ldg(UH + row4 + c - 1) : z4, pl = c > 0 ? __ldg(UL + row4 + c - 1) : z4;
        const int4 ch = __ldg(UH + row4 + c), cl = __ldg(UL + row4 + c);
        const int4 nh = c + 1 < chunks ? __ldg(UH + row4 + c + 1) : z4;
        const int4 nl = c + 1 < chunks ? __ldg(UL + row4 + c + 1) : z4;
        wh[0] = ph.x; wh[1] = ph.y; wh[2] = ph.z; wh[3] = ph.w; wh[4] = ch.x; wh[5] = ch.y;
        wh[6] = ch.z; wh[7] = ch.w; wh[8] = nh.x; wh[9] = nh.y; wh[10] = nh.z; wh[11] = nh.w;
        wl[0] = pl.x; wl[1] = pl.y; wl[2] = pl.z; wl[3] = pl.w; wl[4] = cl.x; wl[5] = cl.y;
        wl[6] = cl.z; wl[7] = cl.w; wl[8] = nl.x; wl[9] = nl.y; wl[10] = nl.z; wl[11] = nl.w;
      }
      int ws[12];
#pragma unroll
      for (int d = 0; d < 12; ++d) ws[d] = corr_u(wh[d]);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int q = (p + 1) % K;
        const int nt = fix_terms(K, q);
#pragma unroll
        for (int e = 0; e < K + 1; ++e) {
          if (e >= nt) break;  // compile-time after unrolling
          const int dA = fix_da(K, q, e), dB = fix_db(K, q, e);
          const int ch = cf.ch[0][q * BW + e], cl = cf.cl[0][q * BW + e];
          Q[p] += cf.e[0][q * BW + e] * ws[4 + p + dA];
          if (dB == kNoRow) {
            fx1(P2[p], P1[p], ch, cl, wh[4 + p + dA], wl[4 + p + dA]);
          } else {
            fx1(P2[p], P1[p], ch, cl, wh[4 + p + dA] + wh[4 + p + dB], wl[4 + p + dA] + wl[4 + p + dB]);
            P1[p] += (long long)cf.dc[0][q * BW + e] * wh[4 + p + dB];
            Q[p] += cf.eb[0][q * BW + e] * ws[4 + p + dB];
          }
        }
      }
      // y and z: whole rows of the neighbouring lines, one int4 pair per row;
      // the local index is warp-uniform, each case unrolled at compile time
#pragma unroll
      for (int ax = 1; ax < 3; ++ax) {
        const int q = ax == 1 ? qy : qz;
        const int pos = ax == 1 ? j : l;
        const int lim = ax == 1 ? a.ny : a.nz;
        const long long stride = ax == 1 ? (long long)chunks : splane;
        const int nt = fix_terms(K, q);
        for (int e = 0; e < nt; ++e) {  // warp-uniform
          const int dA = fix_da(K, q, e), dB = fix_db(K, q, e);
          const int ch = cf.ch[ax][q * BW + e], cl = cf.cl[ax][q * BW + e];
          const bool okA = pos + dA >= 0 && pos + dA < lim;
          const int4 z4 = make_int4(0, 0, 0, 0);
          int4 vh = okA ? __ldg(UH + row4 + dA * stride + c) : z4;
          int4 vl = okA ? __ldg(UL + row4 + dA * stride + c) : z4;
          const int ea = cf.e[ax][q * BW + e];
          Q[0] += ea * corr_u(vh.x); Q[1] += ea * corr_u(vh.y); Q[2] += ea * corr_u(vh.z); Q[3] += ea * corr_u(vh.w);
          if (dB != kNoRow) {
            const bool okB = pos + dB >= 0 && pos + dB < lim;
            const int4 bh = okB ? __ldg(UH + row4 + dB * stride + c) : z4;
            const int4 bl = okB ? __ldg(UL + row4 + dB * stride + c) : z4;
            const int dc = cf.dc[ax][q * BW + e], eb = cf.eb[ax][q * BW + e];
            P1[0] += (long long)dc * bh.x; P1[1] += (long long)dc * bh.y;
            P1[2] += (long long)dc * bh.z; P1[3] += (long long)dc * bh.w;
            Q[0] += eb * corr_u(bh.x); Q[1] += eb * corr_u(bh.y); Q[2] += eb * corr_u(bh.z); Q[3] += eb * corr_u(bh.w);
            vh = add4(vh, bh);
            vl = add4(vl, bl);
          }
          fx_term(P2, P1, ch, cl, vh, vl);
        }
      }
      long long R[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        // sum (C + E 2^-14) U / 2^56, rounded once (Q E-units are 2^31 = 8 x 2^28)
        const long long T = P2[p] + ((P1[p] + ((long long)Q[p] << 3) + kHalf) >> kChunk);
        R[p] = (i0 + p < a.nx) ? f64_to_fixed(__ldg(frow + i0 + p), sF) - T : 0;
      }
      if (a.out64) {  // FP64 r at pitch nx
        double* orow = a.out64 + line * a.nx;
#pragma unroll
        for (int p = 0; p < 4; ++p)
          if (i0 + p < a.nx) orow[i0 + p] = finite ? ldexp((double)R[p], X) : __longlong_as_double(0x7FF8000000000000LL);
        continue;
      }
      float r[4];
#pragma unroll
      for (int p = 0; p < 4; ++p)  // pads stay zero
        r[p] = (i0 + p >= a.nx) ? 0.f : finite ? fixed_to_f32(R[p], X) : __int_as_float(0x7FC00000);
      const long long o = line * a.Px + i0;
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

// Fixed-point residual for the other k <= 8 (Dirichlet rows), in the element
// layout of the FP64 residual: a thread owns the K nodes g = ex*K + q of
// element ex of one (j, l) line (unknowns i0 + q, i0 = ex*K - 1; q = 0 is the
// vertex shared with element ex-1), keeps the 2K+1 x-neighbours in registers
// with every node's x row known at compile time, and reads the y and z rows
// from the term tables at its (j, l).  The thread of a line's last element
// also writes the line's pad columns (zeros).  Same arithmetic as
// stencil_fix4_kernel.
template <int K>
__global__ void __launch_bounds__(256) stencil_fix_elem_kernel(FixArgs a, const __grid_constant__ FixCoef cf,
                                                               int nex) {
  constexpr int BW = 2 * K + 1;
  const long long lines = (long long)a.ny * a.nz;
  const long long total = (long long)nex * lines;
  const int s = fixed_scale(a.state, cf.t);
  const int sF = s + cf.t - 56;
  const int X = -sF;
  const bool finite = a.state[0] < 2047 && a.state[1] < 2047;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(t % nex);
    const long long jl = t / nex;
    const int j = (int)(jl % a.ny), l = (int)(jl / a.ny);
    const long long row = jl * a.Px;  // this line in Uh, Ul and the output (pitch Px)
    const int i0 = ex * K - 1;
    int wh[BW], wl[BW], ws[BW];
#pragma unroll
    for (int d = 0; d < BW; ++d) {
      const int i = i0 - K + d;
      const bool ok = i >= 0 && i < a.nx;
      wh[d] = ok ? __ldg(a.Uh + row + i) : 0;
      wl[d] = ok ? __ldg(a.Ul + row + i) : 0;
      ws[d] = corr_u(wh[d]);
    }
    long long P2[K], P1[K];
    int Q[K];
#pragma unroll
    for (int q = 0; q < K; ++q) { P2[q] = 0; P1[q] = 0; Q[q] = 0; }
    // x: the rows of the element's nodes, known at compile time
#pragma unroll
    for (int q = 0; q < K; ++q) {
#pragma unroll
      for (int e = 0; e < K + 1; ++e) {
        if (e >= fix_terms(K, q)) break;
        const int dA = fix_da(K, q, e), dB = fix_db(K, q, e);
        const int ch = cf.ch[0][q * BW + e], cl = cf.cl[0][q * BW + e];
        Q[q] += cf.e[0][q * BW + e] * ws[K + q + dA];
        if (dB == kNoRow) {
          fx1(P2[q], P1[q], ch, cl, wh[K + q + dA], wl[K + q + dA]);
        } else {
          fx1(P2[q], P1[q], ch, cl, wh[K + q + dA] + wh[K + q + dB], wl[K + q + dA] + wl[K + q + dB]);
          P1[q] += (long long)cf.dc[0][q * BW + e] * wh[K + q + dB];
          Q[q] += cf.eb[0][q * BW + e] * ws[K + q + dB];
        }
      }
    }
    // y and z: the rows of the neighbouring lines
#pragma unroll
    for (int ax = 1; ax < 3; ++ax) {
      const int pos = ax == 1 ? j : l;
      const int lim = ax == 1 ? a.ny : a.nz;
      const long long stride = ax == 1 ? (long long)a.Px : (long long)a.ny * a.Px;
      const int qa = (pos + 1) % K;
      const int nt = fix_terms(K, qa);
      for (int e = 0; e < nt; ++e) {
        const int dA = fix_da(K, qa, e), dB = fix_db(K, qa, e);
        const int ch = cf.ch[ax][qa * BW + e], cl = cf.cl[ax][qa * BW + e], ea = cf.e[ax][qa * BW + e];
        const bool okA = pos + dA >= 0 && pos + dA < lim;
        const bool okB = dB != kNoRow && pos + dB >= 0 && pos + dB < lim;
        const int dc = dB != kNoRow ? cf.dc[ax][qa * BW + e] : 0, eb = dB != kNoRow ? cf.eb[ax][qa * BW + e] : 0;
        const long long ra = row + dA * stride, rb = row + (dB != kNoRow ? dB : 0) * stride;
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int i = i0 + q;
          if (i < 0) continue;
          int uh = okA ? __ldg(a.Uh + ra + i) : 0, ul = okA ? __ldg(a.Ul + ra + i) : 0;
          Q[q] += ea * corr_u(uh);
          if (dB != kNoRow) {
            const int bh = okB ? __ldg(a.Uh + rb + i) : 0, bl = okB ? __ldg(a.Ul + rb + i) : 0;
            P1[q] += (long long)dc * bh;
            Q[q] += eb * corr_u(bh);
            uh += bh;
            ul += bl;
          }
          fx1(P2[q], P1[q], ch, cl, uh, ul);
        }
      }
    }
    const double* frow = a.f + jl * a.nx;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int i = i0 + q;
      if (i < 0) continue;
      const long long T = P2[q] + ((P1[q] + ((long long)Q[q] << 3) + kHalf) >> kChunk);
      const long long R = f64_to_fixed(__ldg(frow + i), sF) - T;
      if (a.out64) {  // FP64 r at pitch nx
        a.out64[jl * a.nx + i] = finite ? ldexp((double)R, X) : __longlong_as_double(0x7FF8000000000000LL);
        continue;
      }
      const float r = finite ? fixed_to_f32(R, X) : __int_as_float(0x7FC00000);
      const __nv_bfloat16 h16 = __float2bfloat16_rn(r);
      a.hi[row + i] = h16;
      a.lo[row + i] = __float2bfloat16_rn(r - __bfloat162float(h16));
    }
    if (ex == nex - 1 && !a.out64)
      for (int i = a.nx; i < a.Px; ++i) {
        a.hi[row + i] = __float2bfloat16_rn(0.f);
        a.lo[row + i] = __float2bfloat16_rn(0.f);
      }
  }
}

template <int K>
cudaError_t launch_fix_elem(const FixArgs& a, const FixCoef& cf, cudaStream_t s) {
  const int nex = (a.nx + 1) / K;
  const long long total = (long long)nex * a.ny * a.nz;
  long long b = (total + 255) / 256;  // one thread per element and line, in order (see launch_fix4)
  if (b > 0x7FFFFFFFLL) b = 0x7FFFFFFFLL;
  stencil_fix_elem_kernel<K><<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(a, cf, nex);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_fix4(const FixArgs& a, const FixCoef& cf, cudaStream_t s) {
  // one block per 8 consecutive lines, no grid stride (the resident blocks
  // sweep the grid plane by plane; z neighbours are still in L2)
  const long long lines = (long long)a.ny * a.nz;
  long long blocks = (lines + 7) / 8;
  if (blocks > 0x7FFFFFFFLL) blocks = 0x7FFFFFFFLL;
  stencil_fix4_kernel<K><<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(a, cf);
  return cudaGetLastError();
}

}  // namespace

bool build_fix_coef(const double* const hq[3], int k, FixCoef& cf) {
  if (k < 1 || k > 8) return false;
  const int bw = 2 * k + 1;
  // one scale for all axes: the largest sum of |H| over the terms of a node
  double rsum = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    double m = 0.0;
    for (int q = 0; q < k; ++q) {
      double sq = 0.0;
      for (int d = 0; d < bw; ++d) sq += std::fabs(hq[ax][q * bw + d]);
      m = std::max(m, sq);
    }
    rsum += m;
  }
  if (!(rsum > 0.0) || !std::isfinite(rsum)) return false;
  const int t = (int)std::floor(58.0 - std::log2(rsum));
  cf = FixCoef{};
  cf.t = t;
  auto fixed = [&](double h) { return (long long)std::llround(std::ldexp(h, t)); };
  // the rounded fraction of h 2^t in units of 2^-14 (h 2^t - C is exact in FP64)
  auto frac = [&](double h, long long C) {
    return (int)std::llround(std::ldexp(std::ldexp(h, t) - (double)C, kFracBits));
  };
  for (int ax = 0; ax < 3; ++ax)
    for (int q = 0; q < k; ++q) {
      const double* row = hq[ax] + q * bw;  // entry d at row[d + k]
      const int nt = fix_terms(k, q);
      for (int e = 0; e < nt; ++e) {
        const int dA = fix_da(k, q, e), dB = fix_db(k, q, e);
        const long long C = fixed(row[dA + k]);
        const long long hh = (C + kHalf) >> kChunk;
        cf.ch[ax][q * bw + e] = (int)hh;
        cf.cl[ax][q * bw + e] = (int)(C - (hh << kChunk));
        cf.e[ax][q * bw + e] = frac(row[dA + k], C);
        if (dB != kNoRow) {
          const long long CB = fixed(row[dB + k]);
          const long long dc = CB - C;
          if (dc < -(1LL << 20) || dc > (1LL << 20)) return false;  // not mirror-symmetric
          cf.dc[ax][q * bw + e] = (int)dc;
          cf.eb[ax][q * bw + e] = frac(row[dB + k], CB);
        }
      }
      // every entry of the row outside the terms must be zero
      for (int d = -k; d <= k; ++d) {
        bool used = false;
        for (int e = 0; e < nt; ++e) used = used || fix_da(k, q, e) == d || fix_db(k, q, e) == d;
        if (!used && row[d + k] != 0.0) return false;
      }
    }
  return true;
}

cudaError_t launch_residual_fixed(const Geom& g, int k, const FixCoef& cf, const double* u, const double* f,
                                  int* state, bool f_exponent_known, int* Uh, int* Ul, __nv_bfloat16* out_hi,
                                  __nv_bfloat16* out_lo, int num_sms, cudaStream_t s, double* out64) {
  if (g.bc != 0 || k < 1 || k > 8) return cudaErrorInvalidValue;
  const long long N = (long long)g.nx * g.ny * g.nz;
  const long long lines = (long long)g.ny * g.nz;
  const int red_grid = num_sms * 8;
  cudaError_t e = cudaMemsetAsync(state, 0, f_exponent_known ? sizeof(int) : 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  max_exponent_kernel<<<red_grid, 256, 0, s>>>(u, N, state);
  if (!f_exponent_known) max_exponent_kernel<<<red_grid, 256, 0, s>>>(f, N, state + 1);
  const long long conv = lines * (g.Px / 4);
  long long cb = (conv + 255) / 256;
  if (cb > (long long)num_sms * 16) cb = (long long)num_sms * 16;
  to_fixed_kernel<<<(unsigned)(cb < 1 ? 1 : cb), 256, 0, s>>>(u, Uh, Ul, g.nx, g.Px, lines, state, cf.t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  FixArgs a{};
  a.Uh = Uh; a.Ul = Ul; a.f = f; a.hi = out_hi; a.lo = out_lo; a.state = state; a.out64 = out64;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.Px = g.Px;
  switch (k) {
    case 1: return launch_fix4<1>(a, cf, s);  // 4 % k == 0: the vector layout
    case 2: return launch_fix4<2>(a, cf, s);
    case 4: return launch_fix4<4>(a, cf, s);
    case 3: return launch_fix_elem<3>(a, cf, s);
    case 5: return launch_fix_elem<5>(a, cf, s);
    case 6: return launch_fix_elem<6>(a, cf, s);
    case 7: return launch_fix_elem<7>(a, cf, s);
    default: return launch_fix_elem<8>(a, cf, s);
  }
}

}  // namespace sem3d
