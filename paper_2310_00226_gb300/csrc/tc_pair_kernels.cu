// tcgen05 split-precision mode product with one MMA per pair of SMs
// (cta_group::2), for one problem or for a group of independent problems in
// one persistent launch.  The arithmetic is that of tc_kernels.cu (the same
// MMAs in the same K order: results are bit-identical); see the comment at
// the kernel for the division of work between the two CTAs of a pair.
#include "tc_common.cuh"

#include <algorithm>
#include <atomic>

namespace sem3d {

namespace {

using namespace tcx;

// ---------------------------------------------------------------- CTA-pair kernel
//
// The same mode product with one MMA per pair of SMs (tcgen05 cta_group::2):
// a cluster of 2 CTAs owns a 256-row x 256-output tile.  CTA r of the pair
// stages rows [128 r, 128 r + 128) of the A tile and rows [128 r, 128 r + 128)
// of the W tile, so a stage holds 32 KB per CTA instead of 48 KB (6 stages fit
// where 4 did) and each SM loads half of W without multicast.  The leader CTA
// (rank 0) issues M = 256 MMAs that read A and W from both CTAs' shared memory
// at the same offsets and accumulate rows 128 r .. 128 r + 127 of the tile in
// CTA r's tensor memory.  Both CTAs' TMA loads complete on the leader's "full"
// barrier (armed by the leader with the pair's bytes); MMA completion arrives
// on the "empty" and "tfull" barriers of both CTAs (commit multicast); the
// epilogue warps of both CTAs release a TMEM buffer on the leader's "tempty"
// barrier.  Pairs of clusters pack every SM (clusters of 4 leave SMs idle on
// GPCs whose SM count is not a multiple of 4).
constexpr int P_STAGES = 6;
constexpr int P_B_TILE_BYTES = (BN / 2) * BK * 2;  // 8 KB: this CTA's half of W
constexpr int P_STAGE_BYTES = 2 * A_TILE_BYTES + 2 * P_B_TILE_BYTES;  // 32 KB
__host__ __device__ constexpr int pair_smem_bytes(int pass) {
  return P_STAGES * P_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/ + (pass == 0 ? 8 * XSTAGE_BYTES : 0);
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One pair tile handed to the kernel body: the problem's arguments and tensor
// maps, and the tile's (batch, M pair, N tile) within that problem.
struct PairTile {
  const TcArgs* a;
  const CUtensorMap *Ah, *Al, *Bh, *Bl;
  int b, mp, nt;
};

// Tile source of a launch for one problem: the kernel's own parameters.
struct OneProblem {
  const CUtensorMap *Ah, *Al, *Bh, *Bl;
  const TcArgs* a;
  int tiles_per_batch, total;
  __device__ __forceinline__ void at(int pt, int& /*cursor*/, PairTile& t) const {
    t.a = a; t.Ah = Ah; t.Al = Al; t.Bh = Bh; t.Bl = Bl;
    t.b = pt / tiles_per_batch;
    const int rem = pt - t.b * tiles_per_batch;
    t.mp = rem / a->n_tiles;
    t.nt = rem - t.mp * a->n_tiles;
  }
};

// Tile source of a grouped launch: problem q owns pair tiles [tile0, tile0 +
// its count) of the launch (prefix offsets, ascending).  Each thread walks its
// tiles in ascending order, so its cursor into the table only moves forward.
struct ProblemGroup {
  const TcGroupEntry* tab;
  int count, total;
  __device__ __forceinline__ void at(int pt, int& cursor, PairTile& t) const {
    while (cursor + 1 < count && tab[cursor + 1].tile0 <= pt) ++cursor;
    const TcGroupEntry& e = tab[cursor];
    t.a = &e.a; t.Ah = &e.A_hi; t.Al = &e.A_lo; t.Bh = &e.B_hi; t.Bl = &e.B_lo;
    const int local = pt - e.tile0;
    t.b = local / e.tiles_per_batch;
    const int rem = local - t.b * e.tiles_per_batch;
    t.mp = rem / e.a.n_tiles;
    t.nt = rem - t.mp * e.a.n_tiles;
  }
};

template <int PASS, int MODE, int NP, class Src>
__device__ __forceinline__ void pair_body(const Src& src, int* err, int stall) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P_STAGES * P_STAGE_BYTES);
  // bars: full[P_STAGES], empty[P_STAGES], tfull[2], tempty[2], drain[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * P_STAGES + 5);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (P_STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * P_STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * P_STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * P_STAGES + 4);
  constexpr uint16_t kPair = 3;  // both CTAs of the pair
  constexpr int ROWS_B = BN / 2;  // rows of the W tile this CTA stages

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool a_mn = (PASS != 0);
  const int rank = (int)cluster_ctarank();
  const int pid = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull_bar(b), 1); mbar_init(tempty_bar(b), 2 * epi_warps(MODE)); }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers are initialised before any cross-CTA signal
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  // Pair tile pt -> (problem, batch b, M pair mp, N tile nt); this CTA's M
  // tile is 2 mp + rank (past the problem's last M tile, TMA reads zeros and
  // nothing is stored).
  const int total_pt = src.total;
  PairTile t;
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer (each CTA)
    const uint32_t full_leader0 = mapa_shared(full_bar(0), 0);
    int it = 0, cursor = 0;
    bool ok = true;
    for (int pt = pid; pt < total_pt && ok && !stall; pt += npairs) {
      src.at(pt, cursor, t);
      const int m0 = (2 * t.mp + rank) * BM, n0 = t.nt * BN + rank * ROWS_B;
      const int k_blocks = t.a->k_blocks;
      for (int kb = 0; kb < k_blocks; ++kb, ++it) {
        const int s = it % P_STAGES;
        const uint32_t par = ((it / P_STAGES) & 1) ^ 1;
        if (!mbar_wait(empty_bar(s), par, err, KERN_SPLIT_PAIR | WAIT_PRODUCER)) { ok = false; break; }
        const uint32_t st = smem_u32(smem + s * P_STAGE_BYTES);
        const uint32_t a_hi = st, a_lo = st + A_TILE_BYTES;
        const uint32_t b_hi = st + 2 * A_TILE_BYTES, b_lo = b_hi + P_B_TILE_BYTES;
        const uint32_t fb = full_leader0 + 8u * s;  // the leader's full barrier of stage s
        if (rank == 0)
          mbar_arrive_expect_tx(full_bar(s), 2 * (NP == 3 ? P_STAGE_BYTES : A_TILE_BYTES + P_B_TILE_BYTES));
        const int k0 = kb * BK;
        if (PASS == 0) {
          tma_load_2d_pair(a_hi, t.Ah, fb, k0, m0);
          if (NP == 3) tma_load_2d_pair(a_lo, t.Al, fb, k0, m0);
        } else if (PASS == 1) {
          tma_load_3d_pair(a_hi, t.Ah, fb, m0, k0, t.b);
          tma_load_3d_pair(a_hi + A_TILE_BYTES / 2, t.Ah, fb, m0 + 64, k0, t.b);
          if (NP == 3) {
            tma_load_3d_pair(a_lo, t.Al, fb, m0, k0, t.b);
            tma_load_3d_pair(a_lo + A_TILE_BYTES / 2, t.Al, fb, m0 + 64, k0, t.b);
          }
        } else {
          tma_load_2d_pair(a_hi, t.Ah, fb, m0, k0);
          tma_load_2d_pair(a_hi + A_TILE_BYTES / 2, t.Ah, fb, m0 + 64, k0);
          if (NP == 3) {
            tma_load_2d_pair(a_lo, t.Al, fb, m0, k0);
            tma_load_2d_pair(a_lo + A_TILE_BYTES / 2, t.Al, fb, m0 + 64, k0);
          }
        }
        tma_load_2d_pair(b_hi, t.Bh, fb, k0, n0);
        if (NP == 3) tma_load_2d_pair(b_lo, t.Bl, fb, k0, n0);
      }
    }
    // Drain: the last fill of each stage has landed (leader: its full barrier
    // counts both CTAs' bytes) and the MMAs reading it have completed (both:
    // the commit arrived on this CTA's empty barrier), so no copy, MMA read or
    // remote arrival targets this CTA after it exits.
    const int armed = it;
    for (int q = (armed > P_STAGES ? armed - P_STAGES : 0); q < armed; ++q) {
      if (rank == 0) mbar_wait(full_bar(q % P_STAGES), (q / P_STAGES) & 1, nullptr);
      mbar_wait(empty_bar(q % P_STAGES), (q / P_STAGES) & 1, nullptr);
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------ MMA issuer (leader CTA only)
    constexpr uint32_t idesc = make_idesc(2 * BM, BN, a_mn, 0);
    constexpr uint32_t a_lbo = a_mn ? 4096u : 16u, a_sbo = a_mn ? 1024u : 512u, a_kstep = a_mn ? 2048u : 32u;
    constexpr uint32_t a_layout = a_mn ? LAYOUT_SW128 : LAYOUT_SW64;
    int it = 0, cc = 0, cursor = 0;
    bool ok = true;
    for (int pt = pid; pt < total_pt && ok; pt += npairs, ++cc) {
      src.at(pt, cursor, t);
      const int k_blocks = t.a->k_blocks;
      const int buf = cc & 1;
      if (!mbar_wait_cluster(tempty_bar(buf), ((cc >> 1) & 1) ^ 1, err, KERN_SPLIT_PAIR | WAIT_MMA_TMEM)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t tmem_d = tmem_base + (uint32_t)(buf * BN);
      for (int kb = 0; kb < k_blocks; ++kb, ++it) {
        const int s = it % P_STAGES;
        if (!mbar_wait(full_bar(s), (it / P_STAGES) & 1, err, KERN_SPLIT_PAIR | WAIT_MMA_FULL)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * P_STAGE_BYTES);
        const uint32_t a_hi = st, a_lo = st + A_TILE_BYTES;
        const uint32_t b_hi = st + 2 * A_TILE_BYTES, b_lo = b_hi + P_B_TILE_BYTES;
#pragma unroll
        for (int k16 = 0; k16 < BK / 16; ++k16) {
          const uint64_t dah = smem_desc(a_hi + k16 * a_kstep, a_lbo, a_sbo, a_layout);
          const uint64_t dal = smem_desc(a_lo + k16 * a_kstep, a_lbo, a_sbo, a_layout);
          const uint64_t dbh = smem_desc(b_hi + k16 * 32u, 16u, 512u, LAYOUT_SW64);
          const uint64_t dbl = smem_desc(b_lo + k16 * 32u, 16u, 512u, LAYOUT_SW64);
          const uint32_t acc = (kb | k16) ? 1u : 0u;
          mma_bf16_pair(tmem_d, dah, dbh, idesc, acc);
          if (NP == 3) {
            mma_bf16_pair(tmem_d, dah, dbl, idesc, 1u);
            mma_bf16_pair(tmem_d, dal, dbh, idesc, 1u);
          }
        }
        mma_commit_pair_mc(empty_bar(s), kPair);  // the stage is free in both CTAs once these finish
      }
      if (!ok) break;
      mma_commit_pair_mc(tfull_bar(buf), kPair);  // accumulator ready for both CTAs' epilogues
    }
    mma_commit_pair_mc(drain_bar, 1);  // every pair MMA issued so far has completed
    mbar_wait(drain_bar, 0, nullptr);
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue (each CTA, its own 128 rows)
    const int quad = warp & 3;
    const int slice = (warp - 2) >> 2;
    uint8_t* xstage = PASS == 0 ? smem + P_STAGES * P_STAGE_BYTES + 256 + (warp - 2) * XSTAGE_BYTES : nullptr;
    constexpr int COLS = BN / (epi_warps(MODE) / 4);
    const uint32_t tempty_leader0 = mapa_shared(tempty_bar(0), 0);
    float vmax = 0.f;
    int cc = 0, cursor = 0;
    for (int pt = pid; pt < total_pt; pt += npairs, ++cc) {
      src.at(pt, cursor, t);
      const TcArgs& a = *t.a;
      const int mt = 2 * t.mp + rank;
      const int row = mt * BM + quad * 32 + lane;
      const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(slice * COLS);
      const int buf = cc & 1;
      if (!mbar_wait(tfull_bar(buf), (cc >> 1) & 1, err, KERN_SPLIT_PAIR | WAIT_EPILOGUE)) break;
      tc_fence_after();
#pragma unroll 1
      for (int ch = 0; ch < COLS / 32; ++ch) {
        const int col0 = t.nt * BN + slice * COLS + ch * 32;
        if (col0 >= a.nout || mt >= a.m_tiles) break;  // warp-uniform
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)(buf * BN + ch * 32), v);
        epilogue_chunk<PASS, MODE, NP, 0>(a, row, col0, t.b, v, 1.f, 1.f, vmax, xstage);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty_leader0 + 8u * buf);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no copy, MMA or arrival of the pair targets this CTA any more
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
  }
}

template <int PASS, int MODE, int NP>
__global__ void __launch_bounds__(num_threads(MODE), 1)
    mode_product_bf16x3_pair_kernel(const __grid_constant__ CUtensorMap tmA_hi,
                                    const __grid_constant__ CUtensorMap tmA_lo,
                                    const __grid_constant__ CUtensorMap tmB_hi,
                                    const __grid_constant__ CUtensorMap tmB_lo, const __grid_constant__ TcArgs a) {
  const int m_pairs = (a.m_tiles + 1) / 2;
  const OneProblem src{&tmA_hi, &tmA_lo, &tmB_hi, &tmB_lo, &a, m_pairs * a.n_tiles, m_pairs * a.n_tiles * a.batches};
  pair_body<PASS, MODE, NP>(src, a.err, a.stall);
}

// The same pass for many problems in one persistent launch (grouped batched
// solve): pair tiles of all problems form one queue, problem q's tiles
// starting at tab[q].tile0; each problem brings its own tensor maps and
// epilogue arguments in the device table (64-byte aligned).
template <int PASS, int MODE, int NP>
__global__ void __launch_bounds__(num_threads(MODE), 1)
    mode_product_bf16x3_pair_group_kernel(const TcGroupEntry* __restrict__ tab, int count, int total, int* err,
                                          int stall) {
  const ProblemGroup src{tab, count, total};
  pair_body<PASS, MODE, NP>(src, err, stall);
}

// CTA-pair launch: clusters of 2, one pair per pair of SMs, persistent over
// pair tiles.
template <int PASS, int MODE, int NP>
cudaError_t launch_tc_pair(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0, const CUtensorMap& b1,
                           const TcArgs& a, long long work_pairs, int num_sms, cudaStream_t s) {
  auto kern = mode_product_bf16x3_pair_kernel<PASS, MODE, NP>;
  static std::atomic<int> max_pairs_cache{0};  // per instantiation: co-resident clusters of 2 CTAs
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(num_threads(MODE));
  cfg.dynamicSmemBytes = pair_smem_bytes(PASS);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_pairs = max_pairs_cache.load(std::memory_order_relaxed);
  if (max_pairs == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pair_smem_bytes(PASS));
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
  return cudaLaunchKernelEx(&cfg, kern, a0, a1, b0, b1, a);
}

template <int PASS>
cudaError_t launch_tc_pair_mode(int mode, int nprod, const CUtensorMap& a0, const CUtensorMap& a1,
                                const CUtensorMap& b0, const CUtensorMap& b1, const TcArgs& a, long long work,
                                int num_sms, cudaStream_t s) {
  if (nprod == 1) {
    switch (mode) {
      case OUT_SPLIT: return launch_tc_pair<PASS, OUT_SPLIT, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_DIV_SPLIT: return launch_tc_pair<PASS, OUT_DIV_SPLIT, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_F64: return launch_tc_pair<PASS, OUT_F64, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      case OUT_F64_ACCUM: return launch_tc_pair<PASS, OUT_F64_ACCUM, 1>(a0, a1, b0, b1, a, work, num_sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (mode) {
    case OUT_SPLIT: return launch_tc_pair<PASS, OUT_SPLIT, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    case OUT_DIV_SPLIT: return launch_tc_pair<PASS, OUT_DIV_SPLIT, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    case OUT_F64: return launch_tc_pair<PASS, OUT_F64, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    case OUT_F64_ACCUM: return launch_tc_pair<PASS, OUT_F64_ACCUM, 3>(a0, a1, b0, b1, a, work, num_sms, s);
    default:
      if constexpr (PASS == 2) {
        if (mode == OUT_DF_STORE) return launch_tc_pair<PASS, OUT_DF_STORE, 3>(a0, a1, b0, b1, a, work, num_sms, s);
        if (mode == OUT_DF_ACCUM) return launch_tc_pair<PASS, OUT_DF_ACCUM, 3>(a0, a1, b0, b1, a, work, num_sms, s);
        return launch_tc_pair<PASS, OUT_DF_ACCUM_F64, 3>(a0, a1, b0, b1, a, work, num_sms, s);
      }
      return cudaErrorInvalidValue;
  }
}

// Grouped launch: the same pass of `count` problems, one persistent launch.
template <int PASS, int MODE, int NP>
cudaError_t launch_pair_group_t(const TcGroupEntry* tab, int count, int total, int* err, int stall, int num_sms,
                                cudaStream_t s) {
  auto kern = mode_product_bf16x3_pair_group_kernel<PASS, MODE, NP>;
  static std::atomic<int> max_pairs_cache{0};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(num_threads(MODE));
  cfg.dynamicSmemBytes = pair_smem_bytes(PASS);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_pairs = max_pairs_cache.load(std::memory_order_relaxed);
  if (max_pairs == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pair_smem_bytes(PASS));
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2 * (num_sms / 2));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_pairs = n;
    max_pairs_cache.store(n, std::memory_order_relaxed);
  }
  const int pairs = total < max_pairs ? total : max_pairs;
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, kern, tab, count, total, err, stall);
}

cudaError_t launch_pair_group(int axis, int mode, int nprod, const TcGroupEntry* tab, int count, int total, int* err,
                              int stall, int num_sms, cudaStream_t s) {
  // The modes a grouped solve uses: forward z, y (split), x (division); backward
  // x, y (split) and z (split, FP64 store / accumulate, double-FP32 modes).
  if (nprod == 3) {
    if (axis == 0 && mode == OUT_SPLIT) return launch_pair_group_t<0, OUT_SPLIT, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 0 && mode == OUT_DIV_SPLIT) return launch_pair_group_t<0, OUT_DIV_SPLIT, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 1 && mode == OUT_SPLIT) return launch_pair_group_t<1, OUT_SPLIT, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_SPLIT) return launch_pair_group_t<2, OUT_SPLIT, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_F64) return launch_pair_group_t<2, OUT_F64, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_F64_ACCUM) return launch_pair_group_t<2, OUT_F64_ACCUM, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_DF_STORE) return launch_pair_group_t<2, OUT_DF_STORE, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_DF_ACCUM) return launch_pair_group_t<2, OUT_DF_ACCUM, 3>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_DF_ACCUM_F64) return launch_pair_group_t<2, OUT_DF_ACCUM_F64, 3>(tab, count, total, err, stall, num_sms, s);
  } else if (nprod == 1) {
    if (axis == 0 && mode == OUT_SPLIT) return launch_pair_group_t<0, OUT_SPLIT, 1>(tab, count, total, err, stall, num_sms, s);
    if (axis == 0 && mode == OUT_DIV_SPLIT) return launch_pair_group_t<0, OUT_DIV_SPLIT, 1>(tab, count, total, err, stall, num_sms, s);
    if (axis == 1 && mode == OUT_SPLIT) return launch_pair_group_t<1, OUT_SPLIT, 1>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_SPLIT) return launch_pair_group_t<2, OUT_SPLIT, 1>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_F64) return launch_pair_group_t<2, OUT_F64, 1>(tab, count, total, err, stall, num_sms, s);
    if (axis == 2 && mode == OUT_F64_ACCUM) return launch_pair_group_t<2, OUT_F64_ACCUM, 1>(tab, count, total, err, stall, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

size_t tc_group_table_bytes(int count) { return ((size_t)count * sizeof(TcGroupEntry) + 255) & ~size_t(255); }

cudaError_t launch_mode_product_bf16x3_grouped(int count, const TcGroupItem* items, int axis, int which, int epi,
                                               int nprod, int* err_flag, void* dev_table, void* host_table,
                                               size_t table_bytes, int num_sms, cudaStream_t s) {
  if (count < 1 || !items || tc_group_table_bytes(count) > table_bytes) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(dev_table) | reinterpret_cast<uintptr_t>(host_table)) & 63)
    return cudaErrorInvalidValue;
  TcGroupEntry* tab = static_cast<TcGroupEntry*>(host_table);
  long long total = 0;
  int mode = -1;
  for (int q = 0; q < count; ++q) {
    const TcGroupItem& it = items[q];
    PassSetup ps;
    cudaError_t e = prepare_pass(*it.g, axis, *it.W, which, it.in, it.out, it.out64, epi, it.lamx, it.lamy, it.lamz,
                                 err_flag, it.df, nprod, nullptr, true, ps);
    if (e != cudaSuccess) return e;
    if (mode >= 0 && ps.mode != mode) return cudaErrorInvalidValue;  // one epilogue mode per launch
    mode = ps.mode;
    TcGroupEntry& en = tab[q];
    en.A_hi = ps.mAh; en.A_lo = ps.mAl; en.B_hi = ps.mBh; en.B_lo = ps.mBl;
    en.a = ps.a;
    en.tiles_per_batch = ((ps.a.m_tiles + 1) / 2) * ps.a.n_tiles;
    en.tile0 = (int)total;
    total += (long long)en.tiles_per_batch * ps.a.batches;
    if (total >= (1LL << 31)) return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaMemcpyAsync(dev_table, host_table, (size_t)count * sizeof(TcGroupEntry), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (total == 0) return cudaSuccess;
  return launch_pair_group(axis, mode, nprod, static_cast<const TcGroupEntry*>(dev_table), count, (int)total, err_flag,
                           tc_take_stall(), num_sms, s);
}

namespace tcx {

cudaError_t launch_pair_pass(int axis, int nprod, const PassSetup& ps, long long work_pairs, int num_sms,
                             cudaStream_t s) {
  if (axis == 0) return launch_tc_pair_mode<0>(ps.mode, nprod, ps.mAh, ps.mAl, ps.mBh, ps.mBl, ps.a, work_pairs, num_sms, s);
  if (axis == 1) return launch_tc_pair_mode<1>(ps.mode, nprod, ps.mAh, ps.mAl, ps.mBh, ps.mBl, ps.a, work_pairs, num_sms, s);
  return launch_tc_pair_mode<2>(ps.mode, nprod, ps.mAh, ps.mAl, ps.mBh, ps.mBl, ps.a, work_pairs, num_sms, s);
}

}  // namespace tcx

}  // namespace sem3d
