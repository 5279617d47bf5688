// tcgen05 tensor-core mode product in TF32 (kind::tf32): operands rounded to
// TF32 (8-bit exponent, 10-bit mantissa), products accumulated in FP32 tensor
// memory.  This is the single-precision tensor-core arithmetic whose effect on
// the Q^k method Section 3.7 (Table 10) measures against plain FP32.
//
// Rotating layout.  Every pass contracts the FASTEST axis of its input and
// stores its output with the next contracted axis fastest, so both operands of
// every MMA are K-major (128-byte swizzle rows of 32 fp32) and no pass needs a
// transposed operand.  An input array has dims (d0, d1, d2), d0 fastest with
// row pitch P0, and is read as a matrix of R = d1*d2 rows (row r = i1 + d1*i2
// at offset P0*r).  The pass computes
//     D[r, o] = sum_t A[r, t] * W[o, t]          (W = T^{-1} or T, n x n)
// and stores element (i1, i2, o) at i1 + P1*(i2 + d2*o): the output's fastest
// axis is i1, which the next pass contracts.  Starting from (x, y, z) the six
// passes of a solve run x, y, z, x, y, z and visit the layouts
//     (x,y,z) -> (y,z,a) -> (z,a,b) -> (a,b,c) -> (b,c,i) -> (c,i,j) -> (i,j,l)
// so the last pass writes the FP64 solution in the caller's x-fastest order.
// TMEM lane = row, so the 32 lanes of an epilogue warp store 32 consecutive
// elements of one output column.
//
// Kernel structure (as the split-bf16 kernel): one CTA per SM in clusters of
// four that share the W tile by TMA multicast; warp 0 issues the TMA loads,
// warp 1 owns TMEM and issues the MMAs, the remaining warps run the epilogue
// on two 128 x 256 FP32 accumulators in turn.  Every wait is bounded (1 s);
// on expiry the kernel records SEM3D_ERR_TIMEOUT, drains and returns.
#include "sem3d_internal.h"
#include "tc_ptx.cuh"

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

namespace sem3d {

namespace {

constexpr int T_BM = 128;        // tile rows = TMEM lanes
constexpr int T_BN = 256;        // tile outputs = TMEM columns per accumulator
constexpr int T_BK = 32;         // K per stage: one 128-byte swizzle row of fp32
constexpr int T_STAGES = 4;
constexpr int T_A_BYTES = T_BM * T_BK * 4;  // 16 KB
constexpr int T_B_BYTES = T_BN * T_BK * 4;  // 32 KB
constexpr int T_STAGE_BYTES = T_A_BYTES + T_B_BYTES;
constexpr int T_SMEM = T_STAGES * T_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int T_TMEM_COLS = 2 * T_BN;  // 512
constexpr int T_CL = 4;                // cluster size of the W multicast

// Output modes: TF32 intermediate (optionally divided by the eigenvalue sum),
// or the FP64 solution (stored, or added to).
enum : int { T_OUT_T32 = 0, T_OUT_T32_DIV = 1, T_OUT_F64 = 2, T_OUT_F64_ACCUM = 3 };
// Epilogue warps: two per TMEM lane quadrant, four for the FP64 outputs
// (8-16 bytes per element instead of 4).
__host__ __device__ constexpr int t_epi_warps(int mode) { return mode >= 2 ? 16 : 8; }
__host__ __device__ constexpr int t_threads(int mode) { return 64 + 32 * t_epi_warps(mode); }

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B format TF32 (2) at bits 7-9 and 10-12, both operands K-major (bits 15 and
// 16 clear), N>>3 at bits 17-22, M>>4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

struct Tf32Args {
  int m_tiles, n_tiles, k_blocks;
  int rows;             // R = d1 * d2
  int d1, d2;           // row r = i1 + d1 * i2
  int nout;             // length of the output axis
  long long P1;         // output element (i1, i2, o) at i1 + P1 * (i2 + d2 * o)
  float* out32;         // TF32 intermediate, or
  double* out64;        // the FP64 solution
  const float *lam1, *lam2, *lam3;  // division: lam1[i1] + lam2[i2] + lam3[o] + c
  float c;
  int* err;
  int stall;            // failure-detection test: the producer issues no loads
};

// Epilogue of one 32-column chunk: TMEM lane = `row`, v[q] = column col0 + q.
// Every lane of the warp calls this (rows past the end return after the
// division, whose shuffles need the whole warp).
template <int MODE>
__device__ __forceinline__ void tf32_epilogue(const Tf32Args& a, int row, int col0, float (&v)[32]) {
  const bool row_ok = row < a.rows;
  const bool full = col0 + 32 <= a.nout;
  const int rowc = row_ok ? row : 0;
  const int i1 = rowc % a.d1, i2 = rowc / a.d1;
  if (MODE == T_OUT_T32_DIV) {
    const float s = __ldg(a.lam1 + i1) + __ldg(a.lam2 + i2) + a.c;
    // lam3 of the chunk's 32 outputs: one coalesced load, broadcast by shuffles
    const int lane = threadIdx.x & 31;
    const float l3 = __ldg(a.lam3 + min(col0 + lane, a.nout - 1));
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const float d = s + __shfl_sync(0xFFFFFFFFu, l3, q);
      v[q] = __fdividef(v[q], (full || col0 + q < a.nout) ? d : 1.0f);
    }
  }
  if (!row_ok) return;
  const size_t cs = (size_t)a.P1 * (size_t)a.d2;
  const size_t base = (size_t)i1 + (size_t)a.P1 * (size_t)i2 + (size_t)col0 * cs;
  if (MODE == T_OUT_T32 || MODE == T_OUT_T32_DIV) {
    float* p = a.out32 + base;
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (full || col0 + q < a.nout) p[(size_t)q * cs] = tf32_round(v[q]);
  } else {
    // Read-modify-write in batches: all loads of a batch before its stores.
    constexpr int HB = 8;
    double* p = a.out64 + base;
#pragma unroll
    for (int h = 0; h < 32; h += HB) {
      double old[HB];
#pragma unroll
      for (int q = 0; q < HB; ++q)
        old[q] = (MODE == T_OUT_F64_ACCUM && (full || col0 + h + q < a.nout)) ? p[(size_t)(h + q) * cs] : 0.0;
#pragma unroll
      for (int q = 0; q < HB; ++q)
        if (full || col0 + h + q < a.nout) p[(size_t)(h + q) * cs] = old[q] + f32_to_f64(v[h + q]);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(t_threads(MODE), 1)
    mode_product_tf32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                             const Tf32Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + T_STAGES * T_STAGE_BYTES);
  // bars: full[T_STAGES], empty[T_STAGES], tfull[2], tempty[2], drain[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * T_STAGES + 5);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (T_STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * T_STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * T_STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * T_STAGES + 4);
  constexpr uint16_t kMask = (uint16_t)((1u << T_CL) - 1u);
  constexpr int WROWS = T_BN / T_CL;  // rows of the W tile this CTA loads and multicasts

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_ctarank();
  const int cid = blockIdx.x / T_CL, ncl = gridDim.x / T_CL;

  if (threadIdx.x == 0) {
    for (int s = 0; s < T_STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), T_CL); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull_bar(b), 1); mbar_init(tempty_bar(b), t_epi_warps(MODE)); }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(T_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // peers' barriers are initialised before any multicast
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  // Cluster tile ct -> (M group mg, N tile nt); this CTA's M tile is
  // mg*T_CL + rank (past the last M tile TMA reads zeros and nothing is stored).
  const int m_groups = (a.m_tiles + T_CL - 1) / T_CL;
  const int total_ct = m_groups * a.n_tiles;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int it = 0;
    bool ok = true;
    for (int ct = cid; ct < total_ct && ok && !a.stall; ct += ncl) {
      const int mg = ct / a.n_tiles, nt = ct - mg * a.n_tiles;
      const int m0 = (mg * T_CL + rank) * T_BM, n0 = nt * T_BN;
      for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
        const int s = it % T_STAGES;
        if (!mbar_wait(empty_bar(s), ((it / T_STAGES) & 1) ^ 1, a.err, KERN_TF32 | WAIT_PRODUCER)) { ok = false; break; }
        const uint32_t st = smem_u32(smem + s * T_STAGE_BYTES);
        mbar_arrive_expect_tx(full_bar(s), T_STAGE_BYTES);
        const int k0 = kb * T_BK;
        tma_load_2d(st, &tmA, full_bar(s), k0, m0);
        tma_load_2d_mc(st + T_A_BYTES + (uint32_t)(rank * WROWS * T_BK * 4), &tmB, full_bar(s), k0,
                       n0 + rank * WROWS, kMask);
      }
    }
    // Drain: the last fill of every stage has landed here and has been
    // released by every CTA of the cluster, so nothing targets this CTA later.
    const int armed = it;
    for (int q = (armed > T_STAGES ? armed - T_STAGES : 0); q < armed; ++q) {
      mbar_wait(full_bar(q % T_STAGES), (q / T_STAGES) & 1, nullptr);
      mbar_wait(empty_bar(q % T_STAGES), (q / T_STAGES) & 1, nullptr);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    // K-major 128-byte-swizzled tiles (rows of 32 fp32 = 128 B): SBO 1024 B
    // (next 8-row group); each MMA covers K = 8, i.e. 32 B inside the row.
    constexpr uint32_t idesc = make_idesc_tf32(T_BM, T_BN);
    int it = 0, cc = 0;
    bool ok = true;
    for (int ct = cid; ct < total_ct && ok; ct += ncl, ++cc) {
      const int buf = cc & 1;
      if (!mbar_wait(tempty_bar(buf), ((cc >> 1) & 1) ^ 1, a.err, KERN_TF32 | WAIT_MMA_TMEM)) break;
      tc_fence_after();
      const uint32_t tmem_d = tmem_base + (uint32_t)(buf * T_BN);
      for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
        const int s = it % T_STAGES;
        if (!mbar_wait(full_bar(s), (it / T_STAGES) & 1, a.err, KERN_TF32 | WAIT_MMA_FULL)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * T_STAGE_BYTES);
#pragma unroll
        for (int k8 = 0; k8 < T_BK / 8; ++k8) {
          const uint64_t da = smem_desc(st + k8 * 32u, 16u, 1024u, LAYOUT_SW128);
          const uint64_t db = smem_desc(st + T_A_BYTES + k8 * 32u, 16u, 1024u, LAYOUT_SW128);
          mma_tf32(tmem_d, da, db, idesc, (kb | k8) ? 1u : 0u);
        }
        mma_commit_mc(empty_bar(s), kMask);  // the stage is free in every CTA once these finish
      }
      if (!ok) break;
      mma_commit(tfull_bar(buf));
    }
    mma_commit(drain_bar);  // every MMA issued has finished before TMEM is freed
    mbar_wait(drain_bar, 0, nullptr);
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue
    const int quad = warp & 3;             // TMEM lane quadrant (hardware rule: warp % 4)
    const int slice = (warp - 2) >> 2;     // column slice of the tile
    constexpr int COLS = T_BN / (t_epi_warps(MODE) / 4);
    int cc = 0;
    for (int ct = cid; ct < total_ct; ct += ncl, ++cc) {
      const int mg = ct / a.n_tiles, nt = ct - mg * a.n_tiles;
      const int mt = mg * T_CL + rank;
      const int buf = cc & 1;
      if (!mbar_wait(tfull_bar(buf), (cc >> 1) & 1, a.err, KERN_TF32 | WAIT_EPILOGUE)) break;
      tc_fence_after();
      const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * T_BN + slice * COLS);
      const int row = mt * T_BM + quad * 32 + lane;
#pragma unroll 1
      for (int ch = 0; ch < COLS / 32; ++ch) {
        const int col0 = nt * T_BN + slice * COLS + ch * 32;
        if (col0 >= a.nout || mt >= a.m_tiles) break;  // warp-uniform
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)(ch * 32), v);
        tf32_epilogue<MODE>(a, row, col0, v);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(buf));
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no peer copy or arrival can target this CTA any more
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(T_TMEM_COLS));
  }
}

// ---------------------------------------------------------------- CTA-pair kernel
//
// The same pass with one kind::tf32 MMA per pair of SMs (cta_group::2, M =
// 256): CTA r of a cluster of 2 stages rows [128 r, 128 r + 128) of the A tile
// and of the W tile, 32 KB per stage, 6 stages (the one-CTA kernel holds 4 of
// 48 KB).  The protocol is that of the split-bf16 pair kernel: both CTAs' TMA
// loads complete on the leader's full barrier, which the leader arms with the
// pair's bytes; the leader's MMA commits arrive on both CTAs' empty / tfull
// barriers (multicast); both CTAs' epilogue warps release an accumulator on
// the leader's tempty barrier; every wait is bounded.
constexpr int TP_STAGES = 6;
constexpr int TP_B_BYTES = (T_BN / 2) * T_BK * 4;    // 16 KB: this CTA's half of W
constexpr int TP_STAGE_BYTES = T_A_BYTES + TP_B_BYTES;  // 32 KB
constexpr int TP_SMEM = TP_STAGES * TP_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

__device__ __forceinline__ void mma_tf32_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(t_threads(MODE), 1)
    mode_product_tf32_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                  const Tf32Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TP_STAGES * TP_STAGE_BYTES);
  // bars: full[TP_STAGES], empty[TP_STAGES], tfull[2], tempty[2], drain[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TP_STAGES + 5);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (TP_STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * TP_STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * TP_STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * TP_STAGES + 4);
  constexpr uint16_t kPair = 3;
  constexpr int ROWS_B = T_BN / 2;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_ctarank();
  const int pid = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TP_STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull_bar(b), 1); mbar_init(tempty_bar(b), 2 * t_epi_warps(MODE)); }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(T_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers are initialised before any cross-CTA signal
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  // Pair tile pt -> (M pair mp, N tile nt); this CTA's M tile is 2 mp + rank.
  const int m_pairs = (a.m_tiles + 1) / 2;
  const int total_pt = m_pairs * a.n_tiles;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer (each CTA)
    const uint32_t full_leader0 = mapa_shared(full_bar(0), 0);
    int it = 0;
    bool ok = true;
    for (int pt = pid; pt < total_pt && ok && !a.stall; pt += npairs) {
      const int mp = pt / a.n_tiles, nt = pt - mp * a.n_tiles;
      const int m0 = (2 * mp + rank) * T_BM, n0 = nt * T_BN + rank * ROWS_B;
      for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
        const int s = it % TP_STAGES;
        if (!mbar_wait(empty_bar(s), ((it / TP_STAGES) & 1) ^ 1, a.err, KERN_TF32_PAIR | WAIT_PRODUCER)) {
          ok = false;
          break;
        }
        const uint32_t st = smem_u32(smem + s * TP_STAGE_BYTES);
        const uint32_t fb = full_leader0 + 8u * s;
        if (rank == 0) mbar_arrive_expect_tx(full_bar(s), 2 * TP_STAGE_BYTES);
        const int k0 = kb * T_BK;
        tma_load_2d_pair(st, &tmA, fb, k0, m0);
        tma_load_2d_pair(st + T_A_BYTES, &tmB, fb, k0, n0);
      }
    }
    // Drain (see the split-bf16 pair kernel): the last fill of each stage has
    // landed and its MMAs have completed before this CTA may exit.
    const int armed = it;
    for (int q = (armed > TP_STAGES ? armed - TP_STAGES : 0); q < armed; ++q) {
      if (rank == 0) mbar_wait(full_bar(q % TP_STAGES), (q / TP_STAGES) & 1, nullptr);
      mbar_wait(empty_bar(q % TP_STAGES), (q / TP_STAGES) & 1, nullptr);
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------ MMA issuer (leader only)
    constexpr uint32_t idesc = make_idesc_tf32(2 * T_BM, T_BN);
    int it = 0, cc = 0;
    bool ok = true;
    for (int pt = pid; pt < total_pt && ok; pt += npairs, ++cc) {
      const int buf = cc & 1;
      if (!mbar_wait_cluster(tempty_bar(buf), ((cc >> 1) & 1) ^ 1, a.err, KERN_TF32_PAIR | WAIT_MMA_TMEM)) break;
      tc_fence_after();
      const uint32_t tmem_d = tmem_base + (uint32_t)(buf * T_BN);
      for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
        const int s = it % TP_STAGES;
        if (!mbar_wait(full_bar(s), (it / TP_STAGES) & 1, a.err, KERN_TF32_PAIR | WAIT_MMA_FULL)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * TP_STAGE_BYTES);
#pragma unroll
        for (int k8 = 0; k8 < T_BK / 8; ++k8) {
          const uint64_t da = smem_desc(st + k8 * 32u, 16u, 1024u, LAYOUT_SW128);
          const uint64_t db = smem_desc(st + T_A_BYTES + k8 * 32u, 16u, 1024u, LAYOUT_SW128);
          mma_tf32_pair(tmem_d, da, db, idesc, (kb | k8) ? 1u : 0u);
        }
        mma_commit_pair_mc(empty_bar(s), kPair);
      }
      if (!ok) break;
      mma_commit_pair_mc(tfull_bar(buf), kPair);
    }
    mma_commit_pair_mc(drain_bar, 1);
    mbar_wait(drain_bar, 0, nullptr);
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue (each CTA, its own 128 rows)
    const int quad = warp & 3;
    const int slice = (warp - 2) >> 2;
    constexpr int COLS = T_BN / (t_epi_warps(MODE) / 4);
    const uint32_t tempty_leader0 = mapa_shared(tempty_bar(0), 0);
    int cc = 0;
    for (int pt = pid; pt < total_pt; pt += npairs, ++cc) {
      const int mp = pt / a.n_tiles, nt = pt - mp * a.n_tiles;
      const int mt = 2 * mp + rank;
      const int buf = cc & 1;
      if (!mbar_wait(tfull_bar(buf), (cc >> 1) & 1, a.err, KERN_TF32_PAIR | WAIT_EPILOGUE)) break;
      tc_fence_after();
      const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * T_BN + slice * COLS);
      const int row = mt * T_BM + quad * 32 + lane;
#pragma unroll 1
      for (int ch = 0; ch < COLS / 32; ++ch) {
        const int col0 = nt * T_BN + slice * COLS + ch * 32;
        if (col0 >= a.nout || mt >= a.m_tiles) break;  // warp-uniform
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)(ch * 32), v);
        tf32_epilogue<MODE>(a, row, col0, v);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty_leader0 + 8u * buf);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(T_TMEM_COLS));
  }
}

// FP64 array (x fastest, pitch nx) -> TF32-rounded FP32 array at pitch Px.
// Blocks walk the (j, l) lines; a lane converts 4 consecutive entries and
// writes them as one 16-byte store (rows of pitch Px, a multiple of 16, are
// 64-byte aligned); the pad entries i >= nx are written as zeros.
__global__ void __launch_bounds__(256) to_tf32_kernel(const double* __restrict__ in, float* __restrict__ out, int nx,
                                                      int Px, long long lines) {
  const int chunks = Px >> 2;
  for (long long line = blockIdx.x; line < lines; line += gridDim.x) {
    const double* row = in + line * nx;
    float4* orow = reinterpret_cast<float4*>(out + line * Px);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
      const int i = 4 * c;
      float4 v;
      v.x = i < nx ? tf32_round(f64_to_f32_rn(row[i])) : 0.f;
      v.y = i + 1 < nx ? tf32_round(f64_to_f32_rn(row[i + 1])) : 0.f;
      v.z = i + 2 < nx ? tf32_round(f64_to_f32_rn(row[i + 2])) : 0.f;
      v.w = i + 3 < nx ? tf32_round(f64_to_f32_rn(row[i + 3])) : 0.f;
      orow[c] = v;
    }
  }
}

template <int MODE>
cudaError_t launch_tf32(const CUtensorMap& mA, const CUtensorMap& mB, const Tf32Args& a, long long work_clusters,
                        int num_sms, cudaStream_t s) {
  auto kern = mode_product_tf32_kernel<MODE>;
  static std::atomic<int> max_clusters_cache{0};  // co-resident clusters of this instantiation
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = T_CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(t_threads(MODE));
  cfg.dynamicSmemBytes = T_SMEM;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_clusters = max_clusters_cache.load(std::memory_order_relaxed);
  if (max_clusters == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T_SMEM);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(T_CL * (num_sms / T_CL));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_clusters = n;
    max_clusters_cache.store(n, std::memory_order_relaxed);
  }
  const long long clusters = work_clusters < max_clusters ? work_clusters : max_clusters;
  cfg.gridDim = dim3((unsigned)(clusters * T_CL));
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, kern, mA, mB, a);
}

template <int MODE>
cudaError_t launch_tf32_pair(const CUtensorMap& mA, const CUtensorMap& mB, const Tf32Args& a, long long work_pairs,
                             int num_sms, cudaStream_t s) {
  auto kern = mode_product_tf32_pair_kernel<MODE>;
  static std::atomic<int> max_pairs_cache{0};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(t_threads(MODE));
  cfg.dynamicSmemBytes = TP_SMEM;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_pairs = max_pairs_cache.load(std::memory_order_relaxed);
  if (max_pairs == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TP_SMEM);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2 * (num_sms / 2));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_pairs = n;
    max_pairs_cache.store(n, std::memory_order_relaxed);
  }
  const long long pairs = work_pairs < max_pairs ? work_pairs : max_pairs;
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, kern, mA, mB, a);
}

// Kernel variant per TF32 pass shape (nK, d1, d2), process-wide: TC_SINGLE
// (one CTA per tile, W multicast in clusters of 4) or TC_PAIR.
std::mutex g_tf32_cfg_mu;
std::map<std::tuple<int, int, int>, int> g_tf32_cfg;

int tf32_variant(int nK, int d1, int d2) {
  std::lock_guard<std::mutex> lk(g_tf32_cfg_mu);
  auto it = g_tf32_cfg.find(std::make_tuple(nK, d1, d2));
  return it == g_tf32_cfg.end() ? TC_SINGLE : it->second;
}

}  // namespace

bool tf32_config_known(int nK, int d1, int d2) {
  std::lock_guard<std::mutex> lk(g_tf32_cfg_mu);
  return g_tf32_cfg.count(std::make_tuple(nK, d1, d2)) != 0;
}

void tf32_set_config(int nK, int d1, int d2, int cfg) {
  std::lock_guard<std::mutex> lk(g_tf32_cfg_mu);
  g_tf32_cfg[std::make_tuple(nK, d1, d2)] = cfg;
}

int tf32_config(int nK, int d1, int d2) { return tf32_variant(nK, d1, d2); }

cudaError_t launch_to_tf32(const Geom& g, const double* in, float* out, cudaStream_t s) {
  const long long lines = (long long)g.ny * g.nz;
  const long long blocks = lines < 152LL * 16 ? (lines < 1 ? 1 : lines) : 152LL * 16;
  to_tf32_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, g.nx, g.Px, lines);
  return cudaGetLastError();
}

cudaError_t launch_mode_product_tf32(const Tf32Pass& p, int* err_flag, int num_sms, cudaStream_t s) {
  // Shapes: K-major TMA rows need a pitch of a multiple of 16 bytes and a
  // 16-byte aligned base; the row count and tile counts must fit in int.
  if (p.nK < 1 || p.d1 < 1 || p.d2 < 1 || p.P0 < p.nK || (p.P0 & 3) || p.Wpitch < p.nK || (p.Wpitch & 3) ||
      !p.in || !p.W || (reinterpret_cast<uintptr_t>(p.in) & 15) || (reinterpret_cast<uintptr_t>(p.W) & 15))
    return cudaErrorInvalidValue;
  const long long rows = (long long)p.d1 * p.d2;
  if (rows >= (1LL << 31)) return cudaErrorInvalidValue;
  int mode;
  if (p.out64) {
    if (p.out32 || p.epi == EPI_DIV || p.P1 < p.d1) return cudaErrorInvalidValue;
    mode = p.epi == EPI_ACCUM ? T_OUT_F64_ACCUM : T_OUT_F64;
  } else {
    if (!p.out32 || p.epi == EPI_ACCUM || p.P1 < p.d1) return cudaErrorInvalidValue;
    if (p.epi == EPI_DIV && (!p.lam1 || !p.lam2 || !p.lam3)) return cudaErrorInvalidValue;
    mode = p.epi == EPI_DIV ? T_OUT_T32_DIV : T_OUT_T32;
  }
  Tf32Args a{};
  a.stall = tc_take_stall();
  a.rows = (int)rows;
  a.d1 = p.d1;
  a.d2 = p.d2;
  a.nout = p.nK;
  a.P1 = p.P1;
  a.out32 = p.out32;
  a.out64 = p.out64;
  a.lam1 = p.lam1; a.lam2 = p.lam2; a.lam3 = p.lam3;
  a.c = p.c;
  a.err = err_flag;
  a.m_tiles = (int)((rows + T_BM - 1) / T_BM);
  a.n_tiles = (p.nK + T_BN - 1) / T_BN;
  a.k_blocks = (p.nK + T_BK - 1) / T_BK;
  CUtensorMap mA, mB;
  {
    // A: dims {t: nK, row: R}, row stride P0*4 B; box {T_BK, T_BM}
    const uint64_t dims[2] = {(uint64_t)p.nK, (uint64_t)rows};
    const uint64_t str[1] = {(uint64_t)p.P0 * 4};
    const uint32_t box[2] = {T_BK, T_BM};
    if (!make_map(&mA, p.in, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_DATA_TYPE_FLOAT32))
      return cudaErrorInvalidValue;
  }
  const bool pair = tf32_variant(p.nK, p.d1, p.d2) == TC_PAIR;
  {
    // W: dims {t: nK, o: nK}, row stride Wpitch*4 B; box {T_BK, T_BN / T_CL}
    // (pair kernel: T_BN / 2 rows, each CTA of the pair stages half of the tile)
    const uint64_t dims[2] = {(uint64_t)p.nK, (uint64_t)p.nK};
    const uint64_t str[1] = {(uint64_t)p.Wpitch * 4};
    const uint32_t box[2] = {T_BK, (uint32_t)(pair ? T_BN / 2 : T_BN / T_CL)};
    if (!make_map(&mB, p.W, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_DATA_TYPE_FLOAT32))
      return cudaErrorInvalidValue;
  }
  if (pair) {
    const long long work = (long long)((a.m_tiles + 1) / 2) * a.n_tiles;
    if (work >= (1LL << 31)) return cudaErrorInvalidValue;
    switch (mode) {
      case T_OUT_T32: return launch_tf32_pair<T_OUT_T32>(mA, mB, a, work, num_sms, s);
      case T_OUT_T32_DIV: return launch_tf32_pair<T_OUT_T32_DIV>(mA, mB, a, work, num_sms, s);
      case T_OUT_F64: return launch_tf32_pair<T_OUT_F64>(mA, mB, a, work, num_sms, s);
      default: return launch_tf32_pair<T_OUT_F64_ACCUM>(mA, mB, a, work, num_sms, s);
    }
  }
  const long long work = (long long)((a.m_tiles + T_CL - 1) / T_CL) * a.n_tiles;
  if (work >= (1LL << 31)) return cudaErrorInvalidValue;
  switch (mode) {
    case T_OUT_T32: return launch_tf32<T_OUT_T32>(mA, mB, a, work, num_sms, s);
    case T_OUT_T32_DIV: return launch_tf32<T_OUT_T32_DIV>(mA, mB, a, work, num_sms, s);
    case T_OUT_F64: return launch_tf32<T_OUT_F64>(mA, mB, a, work, num_sms, s);
    default: return launch_tf32<T_OUT_F64_ACCUM>(mA, mB, a, work, num_sms, s);
  }
}

// Measure both kernel variants on the three TF32 pass shapes of g (along x,
// y and z: nK = that axis, rows = the other two) that the process has not
// measured: a synthetic pass with the real nK, d1 and output layout and d2
// truncated so that an array holds at most 2^26 elements; inputs are zeros;
// one warm-up and three timed launches per variant.
cudaError_t tf32_autotune(const Geom& g, const DevAxis* ax, int* err_flag, int num_sms) {
  const int n3[3] = {g.nx, g.ny, g.nz};
  bool need = false;
  for (int a = 0; a < 3; ++a) need = need || !tf32_config_known(n3[a], n3[(a + 1) % 3], n3[(a + 2) % 3]);
  if (!need) return cudaSuccess;
  constexpr size_t kCap = size_t(1) << 26;
  Tf32Pass ps[3];
  size_t in_elems = 0, out_elems = 0;
  for (int a = 0; a < 3; ++a) {
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    Tf32Pass& t = ps[a];
    t.nK = n3[a]; t.d1 = n3[a1]; t.P0 = pad16(n3[a]); t.P1 = pad16(n3[a1]);
    const size_t per = (size_t)t.P0 * t.d1 > (size_t)t.P1 * t.nK ? (size_t)t.P0 * t.d1 : (size_t)t.P1 * t.nK;
    t.d2 = (int)std::min<size_t>(n3[a2], std::max<size_t>(1, kCap / per));
    in_elems = std::max(in_elems, (size_t)t.P0 * t.d1 * t.d2);
    out_elems = std::max(out_elems, (size_t)t.P1 * t.d2 * t.nK);
    t.W = ax[a].Wt32[0];
    t.Wpitch = ax[a].Kp;
    t.epi = EPI_STORE;
  }
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaEventCreate(&ev[q]);
  float* buf = nullptr;
  const size_t in_bytes = (in_elems * sizeof(float) + 255) & ~size_t(255);
  const size_t out_bytes = (out_elems * sizeof(float) + 255) & ~size_t(255);
  const int stalls = tc_swap_stall(0);  // measurement launches take no injected stall
  if (e == cudaSuccess) e = cudaMalloc(&buf, in_bytes + out_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, in_bytes + out_bytes, s);
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    Tf32Pass t = ps[a];
    const int d2 = n3[(a + 2) % 3];
    if (tf32_config_known(t.nK, t.d1, d2)) continue;
    t.in = buf;
    t.out32 = reinterpret_cast<float*>(reinterpret_cast<char*>(buf) + in_bytes);
    float best_ms = 0.f;
    int best = TC_SINGLE;
    for (int variant : {TC_SINGLE, TC_PAIR}) {
      tf32_set_config(t.nK, t.d1, t.d2, variant);
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess) e = launch_mode_product_tf32(t, err_flag, num_sms, s);
      }
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (e == cudaSuccess && (variant == TC_SINGLE || ms < best_ms)) { best_ms = ms; best = variant; }
    }
    if (e == cudaSuccess) tf32_set_config(t.nK, t.d1, d2, best);
  }
  if (buf) cudaFree(buf);
  for (int q = 0; q < 2; ++q)
    if (ev[q]) cudaEventDestroy(ev[q]);
  cudaStreamDestroy(s);
  tc_swap_stall(stalls);
  return e;
}

}  // namespace sem3d
