// Internal declarations of libsem3d (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sem3d.h"

namespace sem3d {

#ifdef __CUDACC__
// FP64 -> FP32 with round-to-nearest-even, entirely in integer arithmetic
// from the IEEE 754 binary64/binary32 formats (the hardware conversion runs on
// the FP64 pipe, 1/64 of the FP32 rate on this GPU).  Covers normal and
// subnormal results, overflow to infinity, zeros, infinities and NaN (quieted).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ex == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u | (unsigned int)(m >> 29) : 0u));
  const int e = ex - 1023 + 127;  // biased FP32 exponent
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  if (e >= 1) {
    unsigned int r = ((unsigned int)e << 23) | (unsigned int)(m >> 29);  // truncated
    const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull), half = 0x10000000u;
    r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;  // a carry rounds into the exponent
    return __uint_as_float(sign | r);
  }
  // Subnormal (or zero) result: significand 1.m (53 bits) scaled to units of
  // 2^-149, i.e. shifted right by s = 30 - e >= 30 bits, then rounded.
  if (ex == 0) return __uint_as_float(sign);  // FP64 zero or subnormal: below half of 2^-149
  const int sh = 30 - e;
  if (sh > 54) return __uint_as_float(sign);
  const unsigned long long sig = m | (1ull << 52);
  const unsigned int q = (unsigned int)(sig >> sh);
  const unsigned long long rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  return __uint_as_float(sign | (q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u)));
}

// Round an FP32 value to TF32 (10 explicit mantissa bits) to nearest, ties to
// even, on the binary32 bit pattern; the result is an FP32 number whose 13 low
// mantissa bits are zero.  Infinities and NaN pass through; finite values
// that round past the largest TF32 number become infinity.
__host__ __device__ inline float tf32_round(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  if ((b & 0x7F800000u) != 0x7F800000u) {
    b += 0xFFFu + ((b >> 13) & 1u);
    b &= 0xFFFFE000u;
  }
  float y;
  memcpy(&y, &b, 4);
  return y;
}
#endif


// ---------------------------------------------------------------- host setup

// 1D data of one axis of degree k on [0, L]: with homogeneous Dirichlet data
// (bc = 0) the n = Ne*k - 1 interior nodes, with homogeneous Neumann data
// (bc = 1) all n = Ne*k + 1 nodes (Section 2.2).
struct Axis1D {
  int n = 0, k = 0, Ne = 0, bc = 0;
  double L = 0.0;
  std::vector<double> x;        // interior node coordinates
  std::vector<double> M;        // lumped mass diagonal
  std::vector<double> S;        // stiffness, n x n row-major
  std::vector<double> lam;      // eigenvalues of H = M^{-1} S, ascending
  std::vector<double> T;        // n x n row-major, T[i*n+j] = component i of eigenvector j
  std::vector<double> Tinv;     // n x n row-major, T^{-1}
  std::vector<double> Hband;    // n x (2k+1): H[i][i+d] at [i*(2k+1) + d + k]
  std::vector<int> band_lo, band_hi;  // nonzero column range of row i of H
  // Uniform mesh: the row of H at global node g depends only on q = g % k.
  // Hq[q*(2k+1) + d + k] = H[g][g+d], including the columns of the two
  // boundary nodes (their values are zero, so those entries are never used).
  std::vector<double> Hq;
};

void gll_rule(int N, std::vector<double>& r, std::vector<double>& w);
void gll_diff(int N, const std::vector<double>& r, std::vector<double>& D);
Axis1D build_axis(int n, int k, double L, int bc = 0);

// ---------------------------------------------------------------- device data

// Pitch (elements) of the x dimension of the tensor-core working arrays and
// of the bf16 matrices: a multiple of 16 so that every bf16 row starts on a
// 32-byte boundary (TMA needs 16; 32 keeps row segments sector-aligned).
inline int pad16(int n) { return (n + 15) & ~15; }

struct DevAxis {
  int n = 0, k = 0, Kp = 0;     // Kp = pad16(n): row pitch of the bf16 matrices
  double* M = nullptr;          // FP64 lumped mass diagonal (n)
  double* T = nullptr;          // FP64 n x n row-major (W[out][in] for the backward pass)
  double* Tinv = nullptr;       // FP64 n x n row-major (W[out][in] for the forward pass)
  double* lam = nullptr;        // FP64 eigenvalues
  float* lamf = nullptr;        // FP32 copy for the low-precision epilogues
  double* Hband = nullptr;      // FP64 n x (2k+1)
  double* Hq = nullptr;         // FP64 k x (2k+1) per-local-index rows of H (x axis: + c on the diagonal)
  float* Hq_hi = nullptr;       // the same table as FP32 terms: Hq = Hq_hi + Hq_lo (48 bits) + Hq_lo2 (exact)
  float* Hq_lo = nullptr;
  float* Hq_lo2 = nullptr;
  float Hq_hi_host[4 * 9] = {}; // host copies for k <= 4 (kernel parameters of the vector residual)
  float Hq_lo_host[4 * 9] = {};
  float Hq_lo2_host[4 * 9] = {};
  int* band_lo = nullptr;
  int* band_hi = nullptr;
  float* Wf[2] = {nullptr, nullptr};            // FP32 copies: [0] = T^{-1}, [1] = T; n x n row-major
  float* Wt32[2] = {nullptr, nullptr};          // TF32-rounded copies, n rows x Kp (TF32 tier)
  __nv_bfloat16* W_hi[2] = {nullptr, nullptr};  // [0] = T^{-1}, [1] = T; n rows x Kp
  // F16X3 tier: W * 2^eW16 split into fp16 hi + lo (same layout), and the
  // infinity norm of W (largest row sum of |W|) for the scale bounds.
  __half* W16_hi[2] = {nullptr, nullptr};
  __half* W16_lo[2] = {nullptr, nullptr};
  int eW16[2] = {0, 0};
  float normW[2] = {0.f, 0.f};
  __nv_bfloat16* W_lo[2] = {nullptr, nullptr};
};

// Epilogues of a mode-product pass.
enum Epi : int {
  EPI_STORE = 0,       // out = acc
  EPI_DIV = 1,         // out = acc / (lam_x,i + lam_y,j + lam_z,l + c)
  EPI_ACCUM = 2,       // out += acc (FP64 outputs only)
  EPI_DF_STORE = 3,    // double-FP32 solution (hi, lo) = (acc, 0)            [z pass]
  EPI_DF_ACCUM = 4,    // (hi, lo) += acc                                     [z pass]
  EPI_DF_ACCUM_F64 = 5 // FP64 out = (hi, lo) + acc                           [z pass]
};

// Power-of-two scaling of the fp16 split arrays of the F16X3 tier, kept on
// the device so a solve needs no host round trip.  Slot 0 describes the split
// input of a solve, slot p the output of its p-th mode product: e[p] is the
// exponent of the scale 2^e the array is stored with, maxbits[p] the FP32 bit
// pattern of the largest |value| (unscaled) written to it (atomicMax on the
// bits orders non-negative floats correctly).
struct F16State {
  int e[8];
  unsigned int maxbits[8];
};

// F16X3 operands: the pass reads state slot pin and writes slot pout; the
// division bound is 1 / min(lambda_x + lambda_y + lambda_z + c) for the
// pass with the lambda-sum division (1 otherwise).
struct F16Pass {
  F16State* st;
  int pin, pout;
  float div_bound;
};

// Solution in double-FP32 form between refinement sweeps: u = hi + lo, both
// at pitch Px (x fastest) with zero pad columns i >= nx.
struct DfBuffers {
  float* hi;
  float* lo;
};

// Grid geometry of one solve.
struct Geom {
  int nx, ny, nz;
  int Px;              // pitch of x in the bf16 working arrays
  double c;
  int bc = 0;          // 0: Dirichlet (element-pattern stencils), 1: Neumann (per-row stencil)
};

// ---- FP64 kernels (fp64_kernels.cu)
// One mode product along `axis` (0 = x, 1 = y, 2 = z) on dense n-pitch FP64
// arrays: out[.., o, ..] (=|+=|/=) sum_t W[o*n + t] * in[.., t, ..].
cudaError_t launch_mode_product_f64(const Geom& g, int axis, const double* W, const double* in, double* out,
                                    int epi, const double* lamx, const double* lamy, const double* lamz,
                                    cudaStream_t s);
// ---- FP32 CUDA-core kernels (fp32_kernels.cu)
// One mode product in FP32 arithmetic; `in` is FP64 (first pass) or FP32,
// `out` FP64 (last pass, EPI_STORE or EPI_ACCUM) or FP32.
cudaError_t launch_mode_product_f32(const Geom& g, int axis, const float* W, const void* in, bool in_f64, void* out,
                                    bool out_f64, int epi, const double* lamx, const double* lamy, const double* lamz,
                                    cudaStream_t s);
// Measure the FP32 kernel configurations on the three pass shapes of grid g
// (once per shape per process; synchronous) and record the fastest; later
// launches of those shapes use it.  f32_config reports the choice for an axis.
cudaError_t f32_autotune(const Geom& g, const DevAxis* ax);
int f32_config(int axis, const Geom& g);
void f32_set_config(int axis, const Geom& g, int cfg);  // pin a configuration
// The same pass for `count` independent problems in one grouped launch.
// The per-problem descriptor table (count * ~160 B) is staged through
// host_table (pinned, >= table_bytes) into dev_table with an async copy on s.
cudaError_t launch_mode_product_f32_grouped(int count, const Geom* geoms, int axis, const float* const* W,
                                            const void* const* in, bool in_f64, void* const* out, bool out_f64,
                                            int epi, const double* const* lamx, const double* const* lamy,
                                            const double* const* lamz, void* dev_table, size_t table_bytes,
                                            void* host_table, cudaStream_t s);
// Au = c u + (H_x (+) H_y (+) H_z) u            (mode 0)
// r  = f - c u - (H_x (+) H_y (+) H_z) u        (mode 1, FP64 r)
// r  = same, written as bf16 hi/lo at pitch Px   (mode 2)
cudaError_t launch_stencil(const Geom& g, int k, const DevAxis* ax, const double* u, const double* f, double* out64,
                           __nv_bfloat16* out_hi, __nv_bfloat16* out_lo, int mode, cudaStream_t s);
// r = f - (c + H_x (+) H_y (+) H_z) u in double-FP32 arithmetic (about 48
// significant bits), u given as a double-FP32 pair (pitch Px, zero pads), f as
// FP64 (pitch nx); r written as bf16 hi/lo at pitch Px with zero pads, or as
// FP32 (out32).  Needs 1 <= k <= 8 and Dirichlet rows (returns
// cudaErrorInvalidValue otherwise).  The rows of H enter as hi + lo FP32 pairs
// (48 bits); with exact_coef also the third term lo2, which makes them exact:
// a 48-bit operator is a different operator, whose solution a refinement with
// only these residuals would converge to (off by ~kappa * 2^-48).
// lo_zero: u's low parts are all zero (right after the first solve); the
// vector kernel (k in {1, 2, 4}) then skips them (the same result).
cudaError_t launch_stencil_df(const Geom& g, int k, const DevAxis* ax, DfBuffers u, const double* f,
                              __nv_bfloat16* out_hi, __nv_bfloat16* out_lo, cudaStream_t s,
                              float* out32 = nullptr, F16State* st = nullptr, bool exact_coef = false,
                              bool lo_zero = false);
// FP64 residual written as FP32 at pitch Px with its max |r| in state slot 0
// (the F16X3 tier then splits it with launch_split_f16).  1 <= k <= 8.
cudaError_t launch_stencil_f32out(const Geom& g, int k, const DevAxis* ax, const double* u, const double* f,
                                  float* out32, F16State* st, cudaStream_t s);
// ---- fixed-point residual (fix_kernels.cu)
// Terms of the row of H with local index q (0 = element vertex) for k in
// {1, 2, 4}: the vertex row and, for even k, the midpoint row are mirror-
// symmetric and enter as C (U_{+d} + U_{-d}) plus a correction for the
// rounding difference of the two FP64 entries; the other rows term by term.
// Term e reads offset fix_da (and fix_db for a mirrored pair, else kNoRow).
constexpr int kNoRow = -100;
__host__ __device__ constexpr bool fix_folded(int K, int q) { return q == 0 || (K % 2 == 0 && 2 * q == K); }
__host__ __device__ constexpr int fix_terms(int K, int q) { return q == 0 ? K + 1 : fix_folded(K, q) ? K / 2 + 1 : K + 1; }
__host__ __device__ constexpr int fix_da(int K, int q, int e) { return fix_folded(K, q) ? e : e - q; }
__host__ __device__ constexpr int fix_db(int K, int q, int e) { return (fix_folded(K, q) && e > 0) ? -e : kNoRow; }
// Rows of (c +) H per axis as fixed-point integers C = round(H 2^t) (one t
// for all axes: the terms of any node sum to about 2^58 in magnitude),
// in balanced 28-bit chunks C = ch 2^28 + cl, entry [q * (2k+1) + e] for term
// e; e = round((H 2^t - C) 2^14), the rounded fraction; for a mirrored pair
// dc = C_{-d} - C_{+d} and eb the fraction of C_{-d}.  A kernel parameter.
struct FixCoef {  // 8 KB: a kernel parameter (CUDA 12.1+ allows 32 KB)
  int ch[3][8 * 17];
  int cl[3][8 * 17];
  int dc[3][8 * 17];
  int e[3][8 * 17];
  int eb[3][8 * 17];
  int t;
};
struct FixArgs {
  const int* Uh;
  const int* Ul;
  const double* f;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  const int* state;  // [0]: max biased exponent of u, [1]: of f
  double* out64;     // if set: r in FP64 at pitch nx (hi / lo unused)
  int nx, ny, nz, Px;
};
// Build the tables from the FP64 rows hq[axis] (k x (2k+1), x with c on its
// diagonal).  False for k > 8 or rows that are not mirror-symmetric up to
// rounding (the fixed-point residual is then not used).
bool build_fix_coef(const double* const hq[3], int k, FixCoef& cf);
// r = f - (c + H_x (+) H_y (+) H_z) u evaluated exactly in 64-bit integer
// fixed point (error below FP64 rounding of the terms), written as bf16 hi/lo
// at pitch Px with zero pads, like launch_stencil mode 2.  Dirichlet rows and
// 1 <= k <= 8 only (cudaErrorInvalidValue otherwise).  state: 2 device ints
// (the max exponents of u and f; f's is taken as given when f_exponent_known,
// e.g. from launch_split's emax); Uh,
// Ul: two int32 arrays of Px * ny * nz (the fixed-point u, 16-byte aligned).
// With out64 set, r is written in FP64 at pitch nx instead (the TF32 tier's
// refinement reads it so).
cudaError_t launch_residual_fixed(const Geom& g, int k, const FixCoef& cf, const double* u, const double* f,
                                  int* state, bool f_exponent_known, int* Uh, int* Ul, __nv_bfloat16* out_hi,
                                  __nv_bfloat16* out_lo, int num_sms, cudaStream_t s, double* out64 = nullptr);
// FP64 dense n-pitch -> bf16 hi/lo at pitch Px with zero pads; with emax
// set, also atomicMax(*emax, largest biased FP64 exponent of the input).
cudaError_t launch_split(const Geom& g, const double* in, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s,
                         int* emax = nullptr);

// ---- tcgen05 kernels (tc_kernels.cu)
struct TcBuffers {
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
};
// Tensor maps and launch data of one BF16x3 mode product, prepared on the host.
struct TcPassPlan;
// One BF16x3 mode product along `axis` reading the split array `in` and
// writing either the split array `out` (EPI_STORE / EPI_DIV) or the FP64
// dense n-pitch array out64 (EPI_STORE / EPI_ACCUM).
// Failure-detection testing: the next `launches` tensor-core launches of the
// process issue no operand loads, so their bounded waits expire.
void tc_inject_stall(int launches);
// Takes one launch from the pending sem3d_inject_stall count: 1 if this
// launch must run with its producer stalled, else 0.
int tc_take_stall();
// Replace the pending stall count (returns the old one): autotuners measure
// with no stall pending and put the count back afterwards.
int tc_swap_stall(int launches);
// Tensor-core kernel variant of the BF16x3 / BF16 mode products, per pass
// shape (process-wide): TC_SINGLE = one CTA per 128 x 256 tile with W
// multicast in clusters of 4; TC_PAIR = one cta_group::2 MMA per pair of SMs
// on 256 x 256 tiles.  Keyed by (axis, grid shape, products per pass: 3 for
// BF16x3, 1 for BF16).  tc_autotune measures both on each pass shape of g not
// measured before (synchronous; scratch of up to 2^26 elements per split
// array) and keeps the faster; tc_set_config pins one.
enum { TC_SINGLE = 0, TC_PAIR = 1 };
int tc_config(int axis, const Geom& g, int nprod);
bool tc_config_known(int axis, const Geom& g, int nprod);
void tc_set_config(int axis, const Geom& g, int nprod, int cfg);
cudaError_t tc_autotune(const Geom& g, const DevAxis* ax, int nprod, int* err_flag, int num_sms);
// One problem of a grouped BF16x3 / BF16 pass (tc_pair_kernels.cu): its grid,
// the axis data of the pass's axis, split input / output (or FP64 out64, or
// the double-FP32 solution df for the double-FP32 modes) and lambda vectors.
struct TcGroupItem {
  const Geom* g;
  const DevAxis* W;
  TcBuffers in, out;
  double* out64;
  DfBuffers df;
  const float *lamx, *lamy, *lamz;
};
// Bytes of the device (and pinned host) table of a grouped launch.
size_t tc_group_table_bytes(int count);
// The same mode product (axis, which = 0: T^{-1}, 1: T; one epilogue mode for
// all) of `count` problems as ONE persistent CTA-pair launch: the problems'
// tensor maps and arguments are written to host_table (pinned, 64-byte
// aligned, >= tc_group_table_bytes(count)), copied to dev_table on s, and the
// kernel walks one queue of pair tiles over all problems.
cudaError_t launch_mode_product_bf16x3_grouped(int count, const TcGroupItem* items, int axis, int which, int epi,
                                               int nprod, int* err_flag, void* dev_table, void* host_table,
                                               size_t table_bytes, int num_sms, cudaStream_t s);

// One TF32 mode product of the rotating-layout solve (tf32_kernels.cu): the
// input has dims (nK, d1, d2), nK fastest at row pitch P0 (a multiple of 4);
// W is nK x nK, row o at W + o*Wpitch (TF32-rounded FP32).  The output element
// (i1, i2, o) goes to i1 + P1*(i2 + d2*o) of out32 (TF32-rounded; epi
// EPI_STORE or EPI_DIV with lam1[i1] + lam2[i2] + lam3[o] + c) or of out64
// (EPI_STORE or EPI_ACCUM).
struct Tf32Pass {
  int nK = 0, d1 = 0, d2 = 0, P0 = 0;
  const float* in = nullptr;
  const float* W = nullptr;
  int Wpitch = 0;
  float* out32 = nullptr;
  double* out64 = nullptr;
  long long P1 = 0;
  int epi = EPI_STORE;
  const float *lam1 = nullptr, *lam2 = nullptr, *lam3 = nullptr;
  float c = 0.f;
};
cudaError_t launch_mode_product_tf32(const Tf32Pass& p, int* err_flag, int num_sms, cudaStream_t s);
// Kernel variant (TC_SINGLE / TC_PAIR) of the TF32 pass of shape (nK, d1, d2),
// process-wide, as for the split tiers; tf32_autotune measures the three pass
// shapes of g not measured before (synchronous; up to 512 MB scratch).
int tf32_config(int nK, int d1, int d2);
bool tf32_config_known(int nK, int d1, int d2);
void tf32_set_config(int nK, int d1, int d2, int cfg);
cudaError_t tf32_autotune(const Geom& g, const DevAxis* ax, int* err_flag, int num_sms);
// FP64 x-fastest array (pitch nx) -> TF32-rounded FP32 at pitch g.Px.
cudaError_t launch_to_tf32(const Geom& g, const double* in, float* out, cudaStream_t s);
cudaError_t launch_mode_product_bf16x3(const Geom& g, int axis, const DevAxis& W, int which, TcBuffers in,
                                       TcBuffers out, double* out64, int epi, const float* lamx, const float* lamy,
                                       const float* lamz, int* err_flag, int num_sms, cudaStream_t s,
                                       DfBuffers df = DfBuffers{nullptr, nullptr}, int nprod = 3,
                                       const F16Pass* f16 = nullptr);
// F16X3 split input: fp16 hi + lo of x * 2^e at pitch Px (zero pads), with e
// chosen from state slot 0's max so the largest |x * 2^e| is near 2^15.
// in is FP64 (pitch nx) or FP32 (pitch Px).
cudaError_t launch_absmax_f64(const Geom& g, const double* in, F16State* st, cudaStream_t s);
cudaError_t launch_split_f16(const Geom& g, const void* in, bool in_f64, __half* hi, __half* lo, F16State* st,
                             cudaStream_t s);

// ---- Cahn-Hilliard pointwise kernels (ch_kernels.cu)
struct ChParams {
  double eps, m, dt, S;
};
// tier: SEM3D_FP64 / SEM3D_FP32 (dense arrays ghat, gg of that type) or the
// split tiers (sh, sg split arrays at pitch Px).
cudaError_t launch_ch_prep(int tier, const Geom& g, const double* phi_n, const double* phi_nm1, void* ghat, void* gg,
                           TcBuffers sh, TcBuffers sg, const ChParams& c, cudaStream_t s);
cudaError_t launch_ch_combine(int tier, const Geom& g, const DevAxis* ax, const void* a1, const void* a2, void* out,
                              TcBuffers s1, TcBuffers s2, TcBuffers so, const ChParams& c, cudaStream_t s);

// ---- PCG vector kernels (pcg_kernels.cu)
struct PcgScalars {
  double rz_old, rz_new, pq, beta, rnorm2, bnorm2;
  long long iter;
};
struct PcgArgs {
  long long N;
  int nx, ny, nz;
  const double *Mx, *My, *Mz;
  double c;                 // shift of the preconditioner (inside the stencil's H table)
  const double* V;
  const double* f;
  double *u, *r, *z, *p, *q, *M3, *Vmc;
  PcgScalars* sc;
};
enum { PCG_INIT = 0, PCG_DOT_RZ, PCG_BETA, PCG_P, PCG_Q, PCG_UPDATE, PCG_COUNT };
cudaError_t launch_pcg(int op, const PcgArgs& a, cudaStream_t s);

}  // namespace sem3d
