// tcgen05 tensor-core mode product in split-bf16 arithmetic (BF16x3).
//
// One mode product of the solve (Section 2.4, Eq. 13: the tensorprod /
// pagemtimes steps) is a GEMM  D[row, o] = sum_t A[row, t] * W[o, t]  where
// `row` enumerates the grid lines along the contracted axis, t runs along the
// axis and W is T^{-1} (forward) or T (backward).  Operands are split into two
// bfloat16 numbers, x = x_hi + x_lo, and the product is accumulated in FP32
// tensor memory as A_hi W_hi + A_hi W_lo + A_lo W_hi (the dropped lo*lo term
// is below FP32 rounding of the sum).
//
// Layout (bf16 working arrays, x pitch Px = pad16(nx), element (i,j,l) at
// i + Px*(j + ny*l)):
//   x pass: rows = (j,l) lines, t = i is contiguous      -> A is K-major
//   y pass: rows = i (contiguous), t = j, batch = l      -> A is MN-major
//   z pass: rows = i + Px*j (contiguous), t = l           -> A is MN-major
// TMA tensor maps stride along the contracted axis directly, so no pass ever
// transposes data.  TMEM lane = row, so for y and z the epilogue stores of a
// warp are 32 consecutive addresses.
//
// Kernel structure (one CTA per SM, persistent over output tiles of
// 128 rows x 256 outputs):
//   warp 0      : TMA producer (one thread)
//   warp 1      : TMEM allocator + MMA issuer (one thread)
//   warps 2..9  : epilogue (TMEM -> registers -> global), two warps per TMEM
//                 lane quadrant, each on half of the tile's columns
// Shared memory holds STAGES = 4 stages of {A_hi, A_lo, W_hi, W_lo} K-slices of 32;
// TMEM holds two 128 x 256 FP32 accumulators so the epilogue of one tile
// overlaps the MMAs of the next.  Every wait is bounded: on expiry the kernel
// records SEM3D_ERR_TIMEOUT in *err, drains its own copies and MMAs, frees
// TMEM and returns.
#include "tc_common.cuh"

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

namespace sem3d {


namespace {

using namespace tcx;

// Thread-block clusters of CL CTAs (CL = 1, 2 or 4) work on CL consecutive M
// tiles that share one N tile, so they need the same W tile: each CTA loads
// BN/CL of its rows and multicasts them into the shared memory of all CL CTAs,
// which cuts the L2 -> SM traffic of W (2/3 of all operand traffic at
// BM = 128, BN = 256) by CL.  A stage may be refilled only when every CTA of
// the cluster has finished the MMAs that read it: each CTA's MMA completion
// arrives on the "empty" barrier of all CL CTAs (count CL).
// NP = 3: BF16x3 (A_hi W_hi + A_hi W_lo + A_lo W_hi); NP = 1: single bf16
// product A_hi W_hi (the lo arrays are neither loaded nor written).
//
// Accumulation chunks: the tensor core adds each MMA's products into its FP32
// accumulator with an error of about 2^-24 of the accumulator per K = 16 step
// that does not average out, so a K = 1000 contraction loses ~60 such steps.
// The MMA warp therefore fills the two TMEM buffers in turn with partial sums
// over a.kc K blocks each.  With FMT = 1 (fp16 hi/lo operands, whose own
// rounding is ~2^-22) the epilogue adds the chunks with FP32 round-to-nearest
// additions, so no tensor-core accumulation runs longer than a.kc * BK; with
// bf16 operands (rounding ~2^-17, which dominates) a.kc covers the whole K and
// each TMEM buffer holds one finished tile as before.
template <int PASS, int MODE, int CL, int NP, int FMT>
__global__ void __launch_bounds__(num_threads(MODE), 1)
    mode_product_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                               const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
                               const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
  constexpr int WROWS = BN / CL;  // rows of the W tile this CTA loads

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool a_mn = (PASS != 0);
  const int rank = (CL > 1) ? (int)cluster_ctarank() : 0;
  const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), CL); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull_bar(b), 1); mbar_init(tempty_bar(b), epi_warps(MODE)); }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  if (CL > 1) cluster_sync_all();  // peers' barriers are initialised before any multicast
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  // Cluster tile ct -> (batch b, M group mg, N tile nt); this CTA's M tile is
  // mg*CL + rank (it may lie past the last M tile: TMA then reads zeros and
  // the epilogue stores nothing).
  const int m_groups = (a.m_tiles + CL - 1) / CL;
  const int tiles_per_batch = m_groups * a.n_tiles;
  const int total_ct = tiles_per_batch * a.batches;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int it = 0;
    bool ok = true;
    for (int ct = cid; ct < total_ct && ok && !a.stall; ct += ncl) {
      const int b = ct / tiles_per_batch;
      const int rem = ct - b * tiles_per_batch;
      const int mg = rem / a.n_tiles, nt = rem - mg * a.n_tiles;
      const int m0 = (mg * CL + rank) * BM, n0 = nt * BN;
      for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
        const int s = it % STAGES;
        const uint32_t par = ((it / STAGES) & 1) ^ 1;
        if (!mbar_wait(empty_bar(s), par, a.err, KERN_SPLIT | WAIT_PRODUCER)) { ok = false; break; }
        const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t a_hi = st, a_lo = st + A_TILE_BYTES;
        const uint32_t b_hi = st + 2 * A_TILE_BYTES, b_lo = b_hi + B_TILE_BYTES;
        mbar_arrive_expect_tx(full_bar(s), NP == 3 ? STAGE_BYTES : A_TILE_BYTES + B_TILE_BYTES);
        const int k0 = kb * BK;
        if (PASS == 0) {
          tma_load_2d(a_hi, &tmA_hi, full_bar(s), k0, m0);
          if (NP == 3) tma_load_2d(a_lo, &tmA_lo, full_bar(s), k0, m0);
        } else if (PASS == 1) {
          tma_load_3d(a_hi, &tmA_hi, full_bar(s), m0, k0, b);
          tma_load_3d(a_hi + A_TILE_BYTES / 2, &tmA_hi, full_bar(s), m0 + 64, k0, b);
          if (NP == 3) {
            tma_load_3d(a_lo, &tmA_lo, full_bar(s), m0, k0, b);
            tma_load_3d(a_lo + A_TILE_BYTES / 2, &tmA_lo, full_bar(s), m0 + 64, k0, b);
          }
        } else {
          tma_load_2d(a_hi, &tmA_hi, full_bar(s), m0, k0);
          tma_load_2d(a_hi + A_TILE_BYTES / 2, &tmA_hi, full_bar(s), m0 + 64, k0);
          if (NP == 3) {
            tma_load_2d(a_lo, &tmA_lo, full_bar(s), m0, k0);
            tma_load_2d(a_lo + A_TILE_BYTES / 2, &tmA_lo, full_bar(s), m0 + 64, k0);
          }
        }
        const uint32_t woff = (uint32_t)(rank * WROWS * BK * 2);
        if (CL == 1) {
          tma_load_2d(b_hi, &tmB_hi, full_bar(s), k0, n0);
          if (NP == 3) tma_load_2d(b_lo, &tmB_lo, full_bar(s), k0, n0);
        } else {
          tma_load_2d_mc(b_hi + woff, &tmB_hi, full_bar(s), k0, n0 + rank * WROWS, kMask);
          if (NP == 3) tma_load_2d_mc(b_lo + woff, &tmB_lo, full_bar(s), k0, n0 + rank * WROWS, kMask);
        }
      }
    }
    // Drain: every stage this thread armed must have landed, and (clusters)
    // every CTA must have released the last fill of each stage, so that no
    // copy or remote arrival targets this CTA after it exits.
    const int armed = it;
    for (int q = (armed > STAGES ? armed - STAGES : 0); q < armed; ++q) {
      mbar_wait(full_bar(q % STAGES), (q / STAGES) & 1, nullptr);
      if (CL > 1) mbar_wait(empty_bar(q % STAGES), (q / STAGES) & 1, nullptr);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    constexpr uint32_t idesc = make_idesc(BM, BN, a_mn, FMT);
    // K-major tiles (rows of BK = 32 bf16 = 64 B, 64-byte swizzle): SBO 512
    //   (next 8-row group), advance 32 B per K = 16 inside the swizzled row.
    // MN-major A (64 rows = 128 B per K row, 128-byte swizzle): LBO 4096 (next
    //   64-row half of the tile), SBO 1024 (next 8 K rows), advance 2048 B per
    //   K = 16.
    constexpr uint32_t a_lbo = a_mn ? 4096u : 16u, a_sbo = a_mn ? 1024u : 512u, a_kstep = a_mn ? 2048u : 32u;
    constexpr uint32_t a_layout = a_mn ? LAYOUT_SW128 : LAYOUT_SW64;
    int it = 0, cc = 0;  // cc: accumulation chunks issued (TMEM buffer cc & 1)
    bool ok = true;
    for (int ct = cid; ct < total_ct && ok; ct += ncl) {
      for (int kb0 = 0; kb0 < a.k_blocks; kb0 += a.kc, ++cc) {
        const int buf = cc & 1;
        if (!mbar_wait(tempty_bar(buf), ((cc >> 1) & 1) ^ 1, a.err, KERN_SPLIT | WAIT_MMA_TMEM)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tmem_d = tmem_base + (uint32_t)(buf * BN);
        const int kb1 = kb0 + a.kc < a.k_blocks ? kb0 + a.kc : a.k_blocks;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(full_bar(s), (it / STAGES) & 1, a.err, KERN_SPLIT | WAIT_MMA_FULL)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
          const uint32_t a_hi = st, a_lo = st + A_TILE_BYTES;
          const uint32_t b_hi = st + 2 * A_TILE_BYTES, b_lo = b_hi + B_TILE_BYTES;
#pragma unroll
          for (int k16 = 0; k16 < BK / 16; ++k16) {
            const uint64_t dah = smem_desc(a_hi + k16 * a_kstep, a_lbo, a_sbo, a_layout);
            const uint64_t dal = smem_desc(a_lo + k16 * a_kstep, a_lbo, a_sbo, a_layout);
            const uint64_t dbh = smem_desc(b_hi + k16 * 32u, 16u, 512u, LAYOUT_SW64);
            const uint64_t dbl = smem_desc(b_lo + k16 * 32u, 16u, 512u, LAYOUT_SW64);
            const uint32_t acc = ((kb - kb0) | k16) ? 1u : 0u;
            mma_bf16(tmem_d, dah, dbh, idesc, acc);
            if (NP == 3) {
              mma_bf16(tmem_d, dah, dbl, idesc, 1u);
              mma_bf16(tmem_d, dal, dbh, idesc, 1u);
            }
          }
          // The stage is free (in every CTA of the cluster) once these MMAs finish.
          if (CL == 1) mma_commit(empty_bar(s));
          else mma_commit_mc(empty_bar(s), kMask);
        }
        if (!ok) break;
        mma_commit(tfull_bar(buf));  // chunk ready for the epilogue
      }
    }
    // Drain: wait for every MMA this thread issued before TMEM is freed.
    mma_commit(drain_bar);
    mbar_wait(drain_bar, 0, nullptr);
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue (epi_warps(MODE) warps)
    // Warp w reads TMEM lane quadrant w % 4 (hardware rule) and one of
    // epi_warps(MODE)/4 column slices of the tile.
    const int quad = warp & 3;
    const int slice = (warp - 2) >> 2;
    uint8_t* xstage = PASS == 0 ? smem + STAGES * STAGE_BYTES + 256 + (warp - 2) * XSTAGE_BYTES : nullptr;
    constexpr int COLS = BN / (epi_warps(MODE) / 4);
    // F16X3: scales from the state the previous kernels left (every CTA
    // computes the same values; one thread publishes this pass's exponent).
    float sc_in = 1.f, sc_out = 1.f;
    if (FMT == 1) {
      const int e_in = a.st->e[a.pin];
      const float max_in = __uint_as_float(a.st->maxbits[a.pin]);
      sc_in = exp2i(-(e_in + a.eW));
      const int e_out = f16_exponent(a.normW * max_in * a.div_bound);
      sc_out = exp2i(e_out);
      if (blockIdx.x == 0 && warp == 2 && lane == 0) a.st->e[a.pout] = e_out;
    }
    float vmax = 0.f;
    int cc = 0;
    bool ok = true;
    for (int ct = cid; ct < total_ct && ok; ct += ncl) {
      const int b = ct / tiles_per_batch;
      const int rem = ct - b * tiles_per_batch;
      const int mg = rem / a.n_tiles, nt = rem - mg * a.n_tiles;
      const int mt = mg * CL + rank;
      const int row = mt * BM + quad * 32 + lane;
      const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(slice * COLS);
      if constexpr (FMT == 1) {
        // Sum the tile's chunks with round-to-nearest FP32 additions.  The
        // running sum moves with the chunks: consuming chunk c adds the sum so
        // far (in the previous chunk's buffer) into chunk c's buffer and
        // releases the previous one, so the MMA always has a buffer to fill.
        int prev = -1;
        for (int kb0 = 0; kb0 < a.k_blocks; kb0 += a.kc, ++cc) {
          const int buf = cc & 1;
          if (!mbar_wait(tfull_bar(buf), (cc >> 1) & 1, a.err, KERN_SPLIT | WAIT_EPILOGUE)) { ok = false; break; }
          tc_fence_after();
          if (prev >= 0) {
#pragma unroll 1
            for (int g = 0; g < COLS / 32; ++g) {
              float x[32], y[32];
              tmem_ld32(lane_addr + (uint32_t)(buf * BN + g * 32), x);
              tmem_ld32(lane_addr + (uint32_t)(prev * BN + g * 32), y);
#pragma unroll
              for (int q = 0; q < 32; ++q) x[q] += y[q];
              tmem_st32(lane_addr + (uint32_t)(buf * BN + g * 32), x);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(prev));
          }
          prev = buf;
        }
        if (!ok) break;
#pragma unroll 1
        for (int ch = 0; ch < COLS / 32; ++ch) {
          const int col0 = nt * BN + slice * COLS + ch * 32;
          if (col0 >= a.nout || mt >= a.m_tiles) break;  // warp-uniform
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(prev * BN + ch * 32), v);
          epilogue_chunk<PASS, MODE, NP, FMT>(a, row, col0, b, v, sc_in, sc_out, vmax, xstage);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(prev));
      } else {
        const int c = cc++;  // one chunk per tile (a.kc >= a.k_blocks)
        const int buf = c & 1;
        if (!mbar_wait(tfull_bar(buf), (c >> 1) & 1, a.err, KERN_SPLIT | WAIT_EPILOGUE)) break;
        tc_fence_after();
#pragma unroll 1
        for (int ch = 0; ch < COLS / 32; ++ch) {
          const int col0 = nt * BN + slice * COLS + ch * 32;
          if (col0 >= a.nout || mt >= a.m_tiles) break;  // warp-uniform
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(buf * BN + ch * 32), v);
          epilogue_chunk<PASS, MODE, NP, FMT>(a, row, col0, b, v, sc_in, sc_out, vmax, xstage);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(buf));
      }
    }
    if (FMT == 1 && (MODE == OUT_SPLIT || MODE == OUT_DIV_SPLIT)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, o));
      if (lane == 0 && vmax > 0.f) atomicMax(&a.st->maxbits[a.pout], __float_as_uint(vmax));
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (CL > 1) cluster_sync_all();  // no peer copy or arrival can target this CTA any more
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
  }
}

}  // namespace

using namespace tcx;

namespace {

// Cluster size of the W multicast (1 = none).
#ifndef SEM3D_TC_CLUSTER
#define SEM3D_TC_CLUSTER 4
#endif
constexpr int CLUSTER = SEM3D_TC_CLUSTER;

// K blocks (of BK) per tensor-core accumulation chunk with fp16 hi/lo operands.
#ifndef SEM3D_TC_CHUNK_KBLOCKS
#define SEM3D_TC_CHUNK_KBLOCKS 8
#endif

template <int PASS, int MODE, int NP, int FMT = 0>
cudaError_t launch_tc(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0, const CUtensorMap& b1,
                      const TcArgs& a, long long work_clusters, int num_sms, cudaStream_t s) {
  auto kern = mode_product_bf16x3_kernel<PASS, MODE, CLUSTER, NP, FMT>;
  static std::atomic<int> max_clusters_cache{0};  // per instantiation: co-resident clusters of CLUSTER CTAs
  int max_clusters = max_clusters_cache.load(std::memory_order_relaxed);
  if (max_clusters == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(PASS));
    if (e != cudaSuccess) return e;
    if (CLUSTER > 1) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CLUSTER;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(CLUSTER * (num_sms / CLUSTER));
      cfg.blockDim = dim3(num_threads(MODE));
      cfg.dynamicSmemBytes = smem_bytes(PASS);
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
      if (e != cudaSuccess) return e;
      if (n < 1) return cudaErrorInvalidConfiguration;
      max_clusters = n;
    } else {
      max_clusters = num_sms;
    }
    max_clusters_cache.store(max_clusters, std::memory_order_relaxed);
  }
  const long long clusters = work_clusters < max_clusters ? work_clusters : max_clusters;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(clusters * CLUSTER));
  cfg.blockDim = dim3(num_threads(MODE));
  cfg.dynamicSmemBytes = smem_bytes(PASS);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a0, a1, b0, b1, a);
}

template <int PASS>
cudaError_t launch_tc_mode(int mode, int nprod, int fmt, const CUtensorMap& a0, const CUtensorMap& a1,
                           const CUtensorMap& b0, const CUtensorMap& b1, const TcArgs& a, long long work, int num_sms,
                           cudaStream_t s) {
  if (fmt == 1) {
    switch (mode) {
      case OUT_SPLIT: return launch_tc<PASS, OUT_SPLIT, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_DIV_SPLIT: return launch_tc<PASS, OUT_DIV_SPLIT, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_F64: return launch_tc<PASS, OUT_F64, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_F64_ACCUM: return launch_tc<PASS, OUT_F64_ACCUM, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      default:
        if constexpr (PASS == 2) {
          if (mode == OUT_DF_STORE) return launch_tc<PASS, OUT_DF_STORE, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
          if (mode == OUT_DF_ACCUM) return launch_tc<PASS, OUT_DF_ACCUM, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
          return launch_tc<PASS, OUT_DF_ACCUM_F64, 3, 1>(a0, a1, b0, b1, a, work, num_sms, s);
        }
        return cudaErrorInvalidValue;
    }
  }
  if (nprod == 1) {
    switch (mode) {
      case OUT_SPLIT: return launch_tc<PASS, OUT_SPLIT, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_DIV_SPLIT: return launch_tc<PASS, OUT_DIV_SPLIT, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_F64: return launch_tc<PASS, OUT_F64, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_F64_ACCUM: return launch_tc<PASS, OUT_F64_ACCUM, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (mode) {
    case OUT_SPLIT: return launch_tc<PASS, OUT_SPLIT, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    case OUT_DIV_SPLIT: return launch_tc<PASS, OUT_DIV_SPLIT, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    case OUT_F64: return launch_tc<PASS, OUT_F64, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    case OUT_F64_ACCUM: return launch_tc<PASS, OUT_F64_ACCUM, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    default:
      if constexpr (PASS == 2) {
        if (mode == OUT_DF_STORE) return launch_tc<PASS, OUT_DF_STORE, 3>(a0, a1, b0, b1, a, work, num_sms, s);
        if (mode == OUT_DF_ACCUM) return launch_tc<PASS, OUT_DF_ACCUM, 3>(a0, a1, b0, b1, a, work, num_sms, s);
        return launch_tc<PASS, OUT_DF_ACCUM_F64, 3>(a0, a1, b0, b1, a, work, num_sms, s);
      }
      return cudaErrorInvalidValue;
  }
}

}  // namespace

// K-major tiles are BK = 32 bf16 = 64 B wide (64-byte swizzle); MN-major
// tiles are 64 elements = 128 B wide (128-byte swizzle).
static constexpr CUtensorMapSwizzle SWZ_K = CU_TENSOR_MAP_SWIZZLE_64B;
static constexpr CUtensorMapSwizzle SWZ_MN = CU_TENSOR_MAP_SWIZZLE_128B;

// Launches that still have to run with the producer stalled (sem3d_inject_stall).
std::atomic<int> g_stall_launches{0};

// Kernel variant per pass shape (process-wide): TC_SINGLE = one CTA per
// 128 x 256 tile, W multicast in clusters of 4, 4 stages; TC_PAIR = one
// cta_group::2 MMA per pair of SMs on 256 x 256 tiles, 6 stages.  Chosen by
// tc_autotune (measured) or pinned by tc_set_config; unmeasured shapes use
// TC_SINGLE.
std::mutex g_tc_cfg_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tc_cfg;

std::tuple<int, int, int, int, int> tc_key(int axis, const Geom& g, int nprod) {
  return std::make_tuple(axis, g.nx, g.ny, g.nz, nprod);
}

int tc_config(int axis, const Geom& g, int nprod) {
  std::lock_guard<std::mutex> lk(g_tc_cfg_mu);
  auto it = g_tc_cfg.find(tc_key(axis, g, nprod));
  return it == g_tc_cfg.end() ? TC_SINGLE : it->second;
}

bool tc_config_known(int axis, const Geom& g, int nprod) {
  std::lock_guard<std::mutex> lk(g_tc_cfg_mu);
  return g_tc_cfg.count(tc_key(axis, g, nprod)) != 0;
}

void tc_set_config(int axis, const Geom& g, int nprod, int cfg) {
  std::lock_guard<std::mutex> lk(g_tc_cfg_mu);
  g_tc_cfg[tc_key(axis, g, nprod)] = cfg;
}

void tc_inject_stall(int launches) { g_stall_launches.store(launches); }

int tc_swap_stall(int launches) { return g_stall_launches.exchange(launches); }

int tc_take_stall() {
  int left = g_stall_launches.load();
  while (left > 0 && !g_stall_launches.compare_exchange_weak(left, left - 1)) {
  }
  return left > 0 ? 1 : 0;
}

namespace tcx {

cudaError_t prepare_pass(const Geom& g, int axis, const DevAxis& W, int which, TcBuffers in, TcBuffers out,
                         double* out64, int epi, const float* lamx, const float* lamy, const float* lamz, int* err_flag,
                         DfBuffers df, int nprod, const F16Pass* f16, bool pair, PassSetup& ps) {
  if (nprod != 1 && nprod != 3) return cudaErrorInvalidValue;
  const int fmt = f16 ? 1 : 0;
  if (fmt == 1 && (nprod != 3 || pair)) return cudaErrorInvalidValue;
  int mode;
  if (epi == EPI_DF_STORE || epi == EPI_DF_ACCUM || epi == EPI_DF_ACCUM_F64) {
    if (axis != 2 || !df.hi || !df.lo || (epi == EPI_DF_ACCUM_F64 && !out64)) return cudaErrorInvalidValue;
    mode = epi == EPI_DF_STORE ? OUT_DF_STORE : (epi == EPI_DF_ACCUM ? OUT_DF_ACCUM : OUT_DF_ACCUM_F64);
  } else if (out64) {
    mode = (epi == EPI_ACCUM) ? OUT_F64_ACCUM : OUT_F64;
  } else {
    mode = (epi == EPI_DIV) ? OUT_DIV_SPLIT : OUT_SPLIT;
  }
  if (out64 && epi == EPI_DIV) return cudaErrorInvalidValue;
  TcArgs& a = ps.a;
  a = TcArgs{};
  ps.mode = mode;
  a.df_hi = df.hi;
  a.df_lo = df.lo;
  if (f16) {
    a.st = f16->st;
    a.pin = f16->pin;
    a.pout = f16->pout;
    a.eW = W.eW16[which];
    a.normW = W.normW[which];
    a.div_bound = f16->div_bound;
  }
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.Px = g.Px;
  a.out_hi = out.hi; a.out_lo = out.lo; a.out64 = out64;
  a.lamx = lamx; a.lamy = lamy; a.lamz = lamz; a.c = (float)g.c;
  a.err = err_flag;
  const uint64_t Px = (uint64_t)g.Px, ny = (uint64_t)g.ny, nz = (uint64_t)g.nz;
  bool ok = true;
  int nin = 0;
  if (axis == 0) {
    // A: dims {i: nx, line: ny*nz}, line stride Px*2 B; box {BK (K), 128 rows}
    const uint64_t dims[2] = {(uint64_t)g.nx, ny * nz};
    const uint64_t str[1] = {Px * 2};
    const uint32_t box[2] = {BK, 128};
    ok = ok && make_map(&ps.mAh, in.hi, 2, dims, str, box, SWZ_K) && make_map(&ps.mAl, in.lo, 2, dims, str, box, SWZ_K);
    a.rows = g.ny * g.nz; a.batches = 1; nin = g.nx;
  } else if (axis == 1) {
    // A: dims {i: Px, j: ny, l: nz}; box {64 rows, BK K, 1}
    const uint64_t dims[3] = {Px, ny, nz};
    const uint64_t str[2] = {Px * 2, Px * ny * 2};
    const uint32_t box[3] = {64, BK, 1};
    ok = ok && make_map(&ps.mAh, in.hi, 3, dims, str, box, SWZ_MN) &&
         make_map(&ps.mAl, in.lo, 3, dims, str, box, SWZ_MN);
    a.rows = g.Px; a.batches = g.nz; nin = g.ny;
  } else {
    // A: dims {m = i + Px*j: Px*ny, l: nz}; box {64 rows, BK K}
    const uint64_t dims[2] = {Px * ny, nz};
    const uint64_t str[1] = {Px * ny * 2};
    const uint32_t box[2] = {64, BK};
    ok = ok && make_map(&ps.mAh, in.hi, 2, dims, str, box, SWZ_MN) &&
         make_map(&ps.mAl, in.lo, 2, dims, str, box, SWZ_MN);
    a.rows = g.Px * g.ny; a.batches = 1; nin = g.nz;
  }
  {
    // W: dims {t: n, o: n}, row pitch Kp*2 B; box {BK (K), BN/CLUSTER rows}
    // (pair kernel: BN/2 rows, each CTA of the pair stages half of the tile)
    const uint64_t dims[2] = {(uint64_t)W.n, (uint64_t)W.n};
    const uint64_t str[1] = {(uint64_t)W.Kp * 2};
    const uint32_t box[2] = {BK, (uint32_t)(pair ? BN / 2 : BN / CLUSTER)};
    const void* wh = fmt ? (const void*)W.W16_hi[which] : (const void*)W.W_hi[which];
    const void* wl = fmt ? (const void*)W.W16_lo[which] : (const void*)W.W_lo[which];
    ok = ok && make_map(&ps.mBh, wh, 2, dims, str, box, SWZ_K) && make_map(&ps.mBl, wl, 2, dims, str, box, SWZ_K);
  }
  if (!ok) return cudaErrorInvalidValue;
  a.nout = W.n;
  a.m_tiles = (a.rows + BM - 1) / BM;
  a.n_tiles = (W.n + BN - 1) / BN;
  a.k_blocks = (nin + BK - 1) / BK;
  a.kc = (fmt == 1 && SEM3D_TC_CHUNK_KBLOCKS > 0) ? SEM3D_TC_CHUNK_KBLOCKS : a.k_blocks;
  return cudaSuccess;
}

}  // namespace tcx

cudaError_t launch_mode_product_bf16x3(const Geom& g, int axis, const DevAxis& W, int which, TcBuffers in,
                                       TcBuffers out, double* out64, int epi, const float* lamx, const float* lamy,
                                       const float* lamz, int* err_flag, int num_sms, cudaStream_t s,
                                       DfBuffers df, int nprod, const F16Pass* f16) {
  const int fmt = f16 ? 1 : 0;
  const bool pair = fmt == 0 && tc_config(axis, g, nprod) == TC_PAIR;
  PassSetup ps;
  cudaError_t e = prepare_pass(g, axis, W, which, in, out, out64, epi, lamx, lamy, lamz, err_flag, df, nprod, f16,
                               pair, ps);
  if (e != cudaSuccess) return e;
  TcArgs& a = ps.a;
  a.stall = tc_take_stall();
  if (pair) {
    const long long work = (long long)((a.m_tiles + 1) / 2) * a.n_tiles * a.batches;
    if (work >= (1LL << 31)) return cudaErrorInvalidValue;
    return launch_pair_pass(axis, nprod, ps, work, num_sms, s);
  }
  const long long work = (long long)((a.m_tiles + CLUSTER - 1) / CLUSTER) * a.n_tiles * a.batches;
  if (work >= (1LL << 31)) return cudaErrorInvalidValue;
  const int mode = ps.mode;
  if (axis == 0) return launch_tc_mode<0>(mode, nprod, fmt, ps.mAh, ps.mAl, ps.mBh, ps.mBl, a, work, num_sms, s);
  if (axis == 1) return launch_tc_mode<1>(mode, nprod, fmt, ps.mAh, ps.mAl, ps.mBh, ps.mBl, a, work, num_sms, s);
  return launch_tc_mode<2>(mode, nprod, fmt, ps.mAh, ps.mAl, ps.mBh, ps.mBl, a, work, num_sms, s);
}

// Measure both kernel variants on each pass shape of g not measured before.
// The synthetic pass keeps the contracted extent, the output extent and the
// access pattern of the real one and truncates the grid so that a split array
// holds at most 2^26 elements (nz for the x and y passes, ny for the z pass);
// inputs are zeros.  One warm-up and three timed launches per variant (CUDA
// events on a private stream); the faster variant is recorded for g.
cudaError_t tc_autotune(const Geom& g, const DevAxis* ax, int nprod, int* err_flag, int num_sms) {
  bool need = false;
  for (int axis = 0; axis < 3; ++axis) need = need || !tc_config_known(axis, g, nprod);
  if (!need) return cudaSuccess;
  constexpr size_t kCap = size_t(1) << 26;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  __nv_bfloat16* buf = nullptr;
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaEventCreate(&ev[q]);
  const size_t plane = (size_t)g.Px * g.ny;
  size_t elems = 0;
  Geom gs[3];
  for (int axis = 0; axis < 3; ++axis) {
    gs[axis] = g;
    if (axis < 2) {
      gs[axis].nz = (int)std::min<size_t>(g.nz, std::max<size_t>(1, kCap / plane));
    } else {
      gs[axis].ny = (int)std::min<size_t>(g.ny, std::max<size_t>(1, kCap / ((size_t)g.Px * g.nz)));
    }
    elems = std::max(elems, (size_t)gs[axis].Px * gs[axis].ny * gs[axis].nz);
  }
  const size_t bytes = (elems * sizeof(__nv_bfloat16) + 255) & ~size_t(255);
  const int stalls = g_stall_launches.exchange(0);  // measurement launches take no injected stall
  if (e == cudaSuccess) e = cudaMalloc(&buf, 4 * bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 4 * bytes, s);
  for (int axis = 0; axis < 3 && e == cudaSuccess; ++axis) {
    if (tc_config_known(axis, g, nprod)) continue;
    uint8_t* b8 = reinterpret_cast<uint8_t*>(buf);
    TcBuffers in{reinterpret_cast<__nv_bfloat16*>(b8), reinterpret_cast<__nv_bfloat16*>(b8 + bytes)};
    TcBuffers out{reinterpret_cast<__nv_bfloat16*>(b8 + 2 * bytes), reinterpret_cast<__nv_bfloat16*>(b8 + 3 * bytes)};
    float best_ms = 0.f;
    int best = TC_SINGLE;
    for (int variant : {TC_SINGLE, TC_PAIR}) {
      tc_set_config(axis, gs[axis], nprod, variant);
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess)
          e = launch_mode_product_bf16x3(gs[axis], axis, ax[axis], 0, in, out, nullptr, EPI_STORE, nullptr, nullptr,
                                         nullptr, err_flag, num_sms, s, DfBuffers{nullptr, nullptr}, nprod);
      }
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (e == cudaSuccess && (variant == TC_SINGLE || ms < best_ms)) { best_ms = ms; best = variant; }
    }
    if (e == cudaSuccess) tc_set_config(axis, g, nprod, best);
  }
  if (buf) cudaFree(buf);
  for (int q = 0; q < 2; ++q)
    if (ev[q]) cudaEventDestroy(ev[q]);
  cudaStreamDestroy(s);
  g_stall_launches.store(stalls);
  return e;
}

}  // namespace sem3d
