// Shared by the tcgen05 split-precision mode-product kernels (BF16x3, BF16,
// F16X3): tc_kernels.cu holds the one-CTA-per-tile kernel, the pass set-up,
// the kernel-variant table and its autotuner; tc_pair_kernels.cu holds the
// CTA-pair (cta_group::2) kernel and its one-problem and grouped launches.
// This header has the tile constants, the kernel arguments, the instruction
// descriptor, the output modes and the epilogue that both use.
#pragma once

#include "sem3d_internal.h"
#include "tc_ptx.cuh"

namespace sem3d {
namespace tcx {

constexpr int BM = 128;           // tile rows = TMEM lanes
constexpr int BN = 256;           // tile outputs = TMEM columns per accumulator
constexpr int BK = 32;            // K per stage: one 64-byte swizzle row of bf16 (K-major tiles)
constexpr int STAGES = 4;
constexpr int A_TILE_BYTES = BM * BK * 2;  // 8 KB
constexpr int B_TILE_BYTES = BN * BK * 2;  // 16 KB
constexpr int STAGE_BYTES = 2 * A_TILE_BYTES + 2 * B_TILE_BYTES;
// x-pass split outputs are staged per epilogue warp (32 rows x 64 bytes, rows
// padded to 80 bytes so that 16-byte accesses of 8 lanes hit distinct banks)
// and written back row-contiguously; see epilogue_chunk.
constexpr int XSTAGE_ROW = 80, XSTAGE_BYTES = 32 * XSTAGE_ROW;
__host__ __device__ constexpr int smem_bytes(int pass) {
  return STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/ + (pass == 0 ? 8 * XSTAGE_BYTES : 0);
}
constexpr int TMEM_COLS = 2 * BN;  // 512
// Epilogue warps: two per TMEM lane quadrant for the split-bf16 outputs; four
// for the outputs that read and write FP64 / double-FP32 solution arrays
// (12-16 more bytes per element), which need more loads in flight to keep up
// with the MMAs.  Threads: producer warp, MMA warp, epilogue warps.
__host__ __device__ constexpr int epi_warps(int mode) { return mode >= 2 ? 16 : 8; }
__host__ __device__ constexpr int num_threads(int mode) { return 64 + 32 * epi_warps(mode); }

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B format at bits 7-9 and 10-12 (0 = fp16, 1 = bf16; both operands of one
// MMA always share the format), A major-ness at bit 15 (1 = MN-major),
// B K-major, N>>3 at bits 17-22, M>>4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(int m, int n, bool a_mn_major, int fmt) {
  return (1u << 4) | ((fmt == 1 ? 0u : 1u) << 7) | ((fmt == 1 ? 0u : 1u) << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// ---------------------------------------------------------------- kernel

struct TcArgs {
  int m_tiles, n_tiles, batches, k_blocks;
  int kc;              // K blocks per TMEM accumulation chunk (see the kernel)
  int rows;            // valid tile rows per batch (x: ny*nz, y: Px, z: Px*ny)
  int nout;            // valid outputs (length of the output axis)
  int nx, ny, nz, Px;
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;
  double* out64;
  float* df_hi;        // solution in double-FP32 form (hi + lo), dense n-pitch
  float* df_lo;
  const float *lamx, *lamy, *lamz;
  float c;
  int* err;
  // F16X3 scaling (FMT = 1): state slots read / written, W scale exponent,
  // infinity norm of W and the division bound (see F16Pass).
  F16State* st;
  int pin, pout, eW;
  float normW, div_bound;
  int stall;           // failure-detection test: the producer issues no loads, so the waits expire
};

// One problem of a grouped pass (device table entry).
struct TcGroupEntry {
  CUtensorMap A_hi, A_lo, B_hi, B_lo;  // 64-byte aligned (CUtensorMap's alignment)
  TcArgs a;
  int tile0;            // first pair tile of this problem in the launch
  int tiles_per_batch;  // pair tiles per batch (page) of this problem
};

// Output modes of the epilogue.  The DF modes (y and z passes only) keep the
// solution as a double-FP32 pair u = hi + lo between refinement sweeps:
//   OUT_DF_STORE     : (hi, lo) = (acc, 0)
//   OUT_DF_ACCUM     : (hi, lo) += acc           (compensated FP32 addition)
//   OUT_DF_ACCUM_F64 : out64 = (double)hi + (double)lo, (hi, lo) = (hi, lo) + acc
enum : int {
  OUT_SPLIT = 0, OUT_DIV_SPLIT = 1, OUT_F64 = 2, OUT_F64_ACCUM = 3,
  OUT_DF_STORE = 4, OUT_DF_ACCUM = 5, OUT_DF_ACCUM_F64 = 6
};

// Split two FP32 values into bf16 hi + lo pairs (packed bf16x2: element 0 in
// the low half).  hi = rn(v), lo = rn(v - hi).
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(v1), "f"(v0));
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(v1 - h1), "f"(v0 - h0));
}

// Split two FP32 values into fp16 hi + lo pairs (packed f16x2, element 0 in
// the low half): hi = rn(v), lo = rn(v - hi).
__device__ __forceinline__ void split_pair_f16(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(v1), "f"(v0));
  const float h0 = __half2float(__ushort_as_half((unsigned short)(hi & 0xFFFFu)));
  const float h1 = __half2float(__ushort_as_half((unsigned short)(hi >> 16)));
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(v1 - h1), "f"(v0 - h0));
}

template <int FMT>
__device__ __forceinline__ void split_any(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  if (FMT == 1) split_pair_f16(v0, v1, hi, lo);
  else split_pair(v0, v1, hi, lo);
}

// Scale 2^e that maps a bound B of |values| to at most 2^15 (fp16 max 65504).
__device__ __forceinline__ int f16_exponent(float bound) {
  if (!(bound > 0.f) || !isfinite(bound)) return 0;
  int e = ilogbf(32768.f / bound);
  return e < -120 ? -120 : (e > 120 ? 120 : e);
}

__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ void st_b16(__nv_bfloat16* p, uint32_t v) {
  asm volatile("st.global.b16 [%0], %1;" ::"l"(p), "h"((unsigned short)(v & 0xFFFFu)) : "memory");
}

// Epilogue of one 32-column chunk held by this thread: TMEM lane = `row`,
// registers v[0..31] = columns col0 .. col0+31 of the output axis.
//
// x pass (PASS 0): row = (j,l) line, the output axis is contiguous in memory,
//   so each thread writes 16-byte vectors of its own line.
// y / z passes: row = contiguous index (i, or i + Px*j), the output axis has
//   a stride, and the 32 lanes of a warp write 32 consecutive elements.
// sc_in: accumulator -> true value (2^-(e_in + eW), 1 for bf16); sc_out: true
// value -> stored split value (2^e_out, 1 for bf16); vmax: running max |true|.
template <int PASS, int MODE, int NP, int FMT>
__device__ __forceinline__ void epilogue_chunk(const TcArgs& a, int row, int col0, int batch, float (&v)[32],
                                               float sc_in, float sc_out, float& vmax, uint8_t* xstage) {
  const bool full = col0 + 32 <= a.nout;
  // Read-modify-write batches: loads of HB elements are issued before their
  // stores (independent, but the compiler cannot prove it through one
  // pointer); 16 with 8 epilogue warps, 8 with 16 (the register budget halves).
  constexpr int HB = epi_warps(MODE) > 8 ? (MODE == OUT_DF_ACCUM ? 4 : 8) : 16;
  if (FMT == 1) {
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] *= sc_in;
  }
  if (PASS == 0) {
    // Split outputs are stored by the whole warp (staged); the other outputs per lane.
    if (row >= a.rows && !(MODE == OUT_SPLIT || MODE == OUT_DIV_SPLIT)) return;
    if (MODE == OUT_DIV_SPLIT) {
      const int rr = row < a.rows ? row : 0;  // rows past the end (not stored) read valid entries
      const int j = rr % a.ny, l = rr / a.ny;
      const float s = __ldg(a.lamy + j) + __ldg(a.lamz + l) + a.c;
      // lambda_x of the chunk's 32 outputs: one coalesced load (lane q holds
      // output col0 + q), broadcast by shuffles; every lane of the warp is here
      const int lane = threadIdx.x & 31;
      const float lx = __ldg(a.lamx + min(col0 + lane, a.nout - 1));
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float d = __shfl_sync(0xFFFFFFFFu, lx, q) + s;
        v[q] = __fdividef(v[q], (full || col0 + q < a.nout) ? d : 1.0f);
      }
    }
    if (FMT == 1 && (MODE == OUT_SPLIT || MODE == OUT_DIV_SPLIT)) {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        if (row < a.rows && (full || col0 + q < a.nout)) vmax = fmaxf(vmax, fabsf(v[q]));
        v[q] *= sc_out;
      }
    }
    if (MODE == OUT_F64 || MODE == OUT_F64_ACCUM) {
      double* dst = a.out64 + (size_t)row * a.nx + col0;
      // Loads first, 16 at a time: the read-modify-writes are independent, but
      // the compiler cannot prove it through one pointer and would otherwise
      // serialise one memory round trip per element.
#pragma unroll
      for (int h = 0; h < 32; h += HB) {
        double old[HB];
#pragma unroll
        for (int q = 0; q < HB; ++q)
          old[q] = (MODE == OUT_F64_ACCUM && (full || col0 + h + q < a.nout)) ? dst[h + q] : 0.0;
#pragma unroll
        for (int q = 0; q < HB; ++q)
          if (full || col0 + h + q < a.nout) dst[h + q] = old[q] + f32_to_f64(v[h + q]);
      }
    } else {
      // Each lane holds 32 consecutive outputs of its own row (line).  Written
      // directly, every 16-byte store of the warp would touch 32 rows; instead
      // the warp stages its 32 x 32 block in shared memory and writes it back
      // with 4 lanes per row: each store instruction covers 8 full 64-byte row
      // segments.  All 32 lanes take part (rows past the end are not stored).
      const int lane = threadIdx.x & 31;
      const int row0 = row - lane;
      uint4 hh[4], ll[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        split_any<FMT>(v[8 * g + 0], v[8 * g + 1], hh[g].x, ll[g].x);
        split_any<FMT>(v[8 * g + 2], v[8 * g + 3], hh[g].y, ll[g].y);
        split_any<FMT>(v[8 * g + 4], v[8 * g + 5], hh[g].z, ll[g].z);
        split_any<FMT>(v[8 * g + 6], v[8 * g + 7], hh[g].w, ll[g].w);
      }
#pragma unroll
      for (int part = 0; part < (NP == 3 ? 2 : 1); ++part) {
        __nv_bfloat16* dst = part == 0 ? a.out_hi : a.out_lo;
#pragma unroll
        for (int g = 0; g < 4; ++g)
          *reinterpret_cast<uint4*>(xstage + lane * XSTAGE_ROW + 16 * g) = part == 0 ? hh[g] : ll[g];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int r = 8 * k + (lane >> 2), seg = lane & 3;
          const uint4 val = *reinterpret_cast<const uint4*>(xstage + r * XSTAGE_ROW + 16 * seg);
          if (row0 + r < a.rows && col0 + 8 * seg + 8 <= a.Px)  // Px is a multiple of 16
            *reinterpret_cast<uint4*>(dst + (size_t)(row0 + r) * a.Px + col0 + 8 * seg) = val;
        }
        __syncwarp();
      }
    }
    return;
  }
  if (row >= a.rows) return;
  int i, j = 0;
  uint32_t rowoff, cs;
  if (PASS == 1) {  // row = i, column = j, batch = l
    i = row;
    rowoff = (uint32_t)row + (uint32_t)a.Px * (uint32_t)a.ny * (uint32_t)batch;
    cs = (uint32_t)a.Px;
  } else {          // row = i + Px*j, column = l
    i = row % a.Px;
    j = row / a.Px;
    rowoff = (uint32_t)row;
    cs = (uint32_t)a.Px * (uint32_t)a.ny;
  }
  if (MODE == OUT_DIV_SPLIT) {
    const float li = __ldg(a.lamx + (i < a.nx ? i : 0)) + a.c;
    const float fixed = (PASS == 1) ? __ldg(a.lamz + batch) : __ldg(a.lamy + j);
    const float* lv = (PASS == 1) ? a.lamy : a.lamz;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int o = col0 + q;
      const float d = (full || o < a.nout) ? li + fixed + __ldg(lv + o) : 1.0f;
      v[q] = __fdividef(v[q], d);
    }
  }
  if (FMT == 1 && (MODE == OUT_SPLIT || MODE == OUT_DIV_SPLIT)) {
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      if (full || col0 + q < a.nout) vmax = fmaxf(vmax, fabsf(v[q]));
      v[q] *= sc_out;
    }
  }
  if (MODE == OUT_DF_STORE || MODE == OUT_DF_ACCUM || MODE == OUT_DF_ACCUM_F64) {
    // z pass only: row = i + Px*j is also the index of (i, j, 0) in the
    // double-FP32 arrays (pitch Px); the FP64 solution has pitch nx.  The
    // store writes zeros into the pad columns i >= nx (the residual stencil
    // reads them as the zero boundary values); the updates leave them alone.
    if (MODE != OUT_DF_STORE && i >= a.nx) return;
    const size_t dcs = (size_t)a.Px * a.ny;
    const size_t d0 = (size_t)row + (size_t)col0 * dcs;
    const size_t cs64 = (size_t)a.nx * a.ny;
    const size_t o0 = (size_t)i + (size_t)a.nx * j + (size_t)col0 * cs64;
#pragma unroll
    for (int h = 0; h < 32; h += HB) {
      float oh[HB], ol[HB];
#pragma unroll
      for (int q = 0; q < HB; ++q) {
        const bool ok = full || col0 + h + q < a.nout;
        oh[q] = (MODE != OUT_DF_STORE && ok) ? a.df_hi[d0 + (size_t)(h + q) * dcs] : 0.f;
        ol[q] = (MODE != OUT_DF_STORE && ok) ? a.df_lo[d0 + (size_t)(h + q) * dcs] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < HB; ++q) {
        if (!(full || col0 + h + q < a.nout)) continue;
        const size_t d = d0 + (size_t)(h + q) * dcs;
        if (MODE == OUT_DF_STORE) {
          a.df_hi[d] = i < a.nx ? v[h + q] : 0.f;
          a.df_lo[d] = 0.f;
        } else {
          // (oh + ol) + v: two-sum of the leading parts, then renormalise.
          const float sum = oh[q] + v[h + q];
          const float bb = sum - oh[q];
          const float err = (oh[q] - (sum - bb)) + (v[h + q] - bb);
          const float t = ol[q] + err;
          const float nh = sum + t;
          const float nl = t - (nh - sum);
          if (MODE == OUT_DF_ACCUM) {
            a.df_hi[d] = nh;
            a.df_lo[d] = nl;
          } else {
            a.out64[o0 + (size_t)(h + q) * cs64] = f32_to_f64(nh) + f32_to_f64(nl);
          }
        }
      }
    }
  } else if (MODE == OUT_F64 || MODE == OUT_F64_ACCUM) {
    if (i >= a.nx) return;
    size_t base, cs64;
    if (PASS == 1) { base = (size_t)i + (size_t)a.nx * a.ny * batch; cs64 = (size_t)a.nx; }
    else { base = (size_t)i + (size_t)a.nx * j; cs64 = (size_t)a.nx * a.ny; }
    double* p = a.out64 + base + (size_t)col0 * cs64;
    // Loads first, 16 at a time (see the x pass).
#pragma unroll
    for (int h = 0; h < 32; h += HB) {
      double old[HB];
#pragma unroll
      for (int q = 0; q < HB; ++q)
        old[q] = (MODE == OUT_F64_ACCUM && (full || col0 + h + q < a.nout)) ? p[(size_t)(h + q) * cs64] : 0.0;
#pragma unroll
      for (int q = 0; q < HB; ++q)
        if (full || col0 + h + q < a.nout) p[(size_t)(h + q) * cs64] = old[q] + f32_to_f64(v[h + q]);
    }
  } else {
    __nv_bfloat16* ph = a.out_hi + rowoff + (size_t)col0 * cs;
    __nv_bfloat16* pl = a.out_lo + rowoff + (size_t)col0 * cs;
#pragma unroll
    for (int q = 0; q < 32; q += 2) {
      uint32_t hh, ll;
      split_any<FMT>(v[q], v[q + 1], hh, ll);
      if (full || col0 + q < a.nout) { st_b16(ph, hh); if (NP == 3) st_b16(pl, ll); }
      ph += cs; pl += cs;
      if (full || col0 + q + 1 < a.nout) { st_b16(ph, hh >> 16); if (NP == 3) st_b16(pl, ll >> 16); }
      ph += cs; pl += cs;
    }
  }
}


// Tensor maps, arguments and epilogue mode of one pass, prepared on the host.
struct PassSetup {
  CUtensorMap mAh, mAl, mBh, mBl;
  TcArgs a;
  int mode;
};

// Build the TMA maps (A for the pass's axis; W with boxes of BN/2 rows for the
// pair kernel, BN/4 for the one-CTA kernel's clusters of 4) and the arguments
// of one pass; a.stall is left 0.  cudaErrorInvalidValue for inconsistent
// arguments or a map the driver rejects.  (tc_kernels.cu)
cudaError_t prepare_pass(const Geom& g, int axis, const DevAxis& W, int which, TcBuffers in, TcBuffers out,
                         double* out64, int epi, const float* lamx, const float* lamy, const float* lamz, int* err_flag,
                         DfBuffers df, int nprod, const F16Pass* f16, bool pair, PassSetup& ps);

// Launch the CTA-pair kernel for one prepared pass over `work_pairs` pair
// tiles (tc_pair_kernels.cu).
cudaError_t launch_pair_pass(int axis, int nprod, const PassSetup& ps, long long work_pairs, int num_sms,
                             cudaStream_t s);

}  // namespace tcx
}  // namespace sem3d
