/*
 * libsem3d -- fast-diagonalisation direct solver for Q^k spectral-element
 * discretisations of (-Lap + c) u = f on a box, homogeneous Dirichlet data.
 *
 * Method: Liu, Shen, Zhang, "A simple GPU implementation of spectral-element
 * methods for solving 3D Poisson type equations on rectangular domains and its
 * applications", arXiv 2310.00226.
 *   - Section 2.1, Eq. (2)-(4): Q^k SEM = continuous Q^k FEM with (k+1)-point
 *     Gauss-Lobatto quadrature; the 1D mass matrix M is diagonal.
 *   - Section 2.2, Eq. (6)-(9): H = M^{-1} S = T Lambda T^{-1} from the
 *     generalised eigenproblem S v = lambda M v.
 *   - Section 2.3: robust form S1 = M^{-1/2} S M^{-1/2} = Q Lambda Q^T,
 *     T = M^{-1/2} Q, T^{-1} = Q^T M^{1/2}.
 *   - Section 2.4, Eq. (12)-(13): (c + H_x (+) H_y (+) H_z) u = f is solved by
 *     three mode products with T^{-1}, an entrywise division by
 *     lambda_x,i + lambda_y,j + lambda_z,l + c, and three mode products with T.
 *
 * Conventions shared by every call:
 *   - Grid functions are dense FP64 arrays of the interior nodes, x fastest:
 *     u[i + nx*(j + ny*l)], 0 <= i < nx, ... (the paper's vec(U), Section 2.4).
 *     Boundary values are zero and not stored.  n_axis = Ne_axis * k - 1.
 *   - Device pointers are CUDA global-memory pointers of the current device;
 *     the caller owns them.  Host pointers are ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *     Work is enqueued on it; calls return without synchronising the host
 *     unless stated otherwise.
 *   - Every call returns a sem3d_status; on failure sem3d_last_error() gives a
 *     message (thread-local).  Asynchronous CUDA faults surface as
 *     SEM3D_ERR_CUDA on a later call.  No C++ exception crosses this boundary.
 *   - A handle is not thread-safe; calls on one handle must be serialised by
 *     the caller (they may target different streams one after another).
 */
#ifndef SEM3D_H
#define SEM3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem3d_plan* sem3d_handle;

typedef enum {
  SEM3D_OK = 0,
  SEM3D_ERR_INVALID_ARG = 1,   /* bad size, pointer, axis, shift or mode     */
  SEM3D_ERR_CUDA = 2,          /* a CUDA runtime/driver call failed          */
  SEM3D_ERR_OOM = 3,           /* device or host allocation failed           */
  SEM3D_ERR_NOT_CONVERGED = 4, /* refinement residual grew or became NaN/Inf */
  SEM3D_ERR_TIMEOUT = 5,       /* a kernel's bounded wait expired            */
  SEM3D_ERR_UNSUPPORTED = 6    /* mode not available for this size / device  */
} sem3d_status;

/* Arithmetic of the six mode products of one solve (Section 2.4, Eq. 13).
 *   SEM3D_FP64   : FP64 operands and accumulation (mma.sync DMMA).
 *   SEM3D_FP32   : FP32 operands and accumulation on the CUDA cores (FFMA).
 *   SEM3D_TF32   : operands rounded to TF32 (10-bit mantissa), one product
 *                  per element pair, FP32 accumulation on tcgen05 tensor
 *                  cores: the single-precision tensor-core arithmetic of
 *                  Section 3.7 (Table 10).  Each pass contracts the fastest
 *                  axis of its input and writes its output transposed, so
 *                  all operands are K-major.  Not available to the
 *                  Cahn-Hilliard step (SEM3D_ERR_UNSUPPORTED).
 *   SEM3D_BF16   : operands rounded to bfloat16, one product per element pair,
 *                  FP32 accumulation on tcgen05 tensor cores (~8 bits).
 *   SEM3D_BF16X3 : operands split x = hi + lo into two bfloat16 numbers;
 *                  hi*hi + hi*lo + lo*hi accumulated in FP32 on tcgen05
 *                  tensor cores (about 16 significant bits per pass).
 *   SEM3D_F16X3  : the same three products on fp16 hi + lo pairs (about 22
 *                  significant bits per pass) of arrays scaled by powers of
 *                  two chosen on the device from tracked maxima (fp16's
 *                  range is small); needs k <= 8.
 * FP64 accuracy is recovered by iterative refinement (sem3d_set_precision). */
typedef enum {
  SEM3D_FP64 = 0,
  SEM3D_FP32 = 1,
  SEM3D_TF32 = 2,
  SEM3D_BF16 = 4,
  SEM3D_BF16X3 = 5,
  SEM3D_F16X3 = 6
} sem3d_precision;

/* Build a plan: 1D GLL nodes, stiffness S, lumped mass M and the robust
 * eigenbasis T, T^{-1}, lambda of each axis in FP64 on the host (Section 2.3,
 * Appendix), then upload them to the current device.
 *   nx, ny, nz : interior nodes per axis; each must satisfy (n+1) % k == 0,
 *                n >= 1, and nx*ny*nz < 2^40.
 *   k          : polynomial degree, 1 <= k <= 24.
 *   Lx, Ly, Lz : box [0,Lx] x [0,Ly] x [0,Lz], each > 0.
 *   c          : shift of -Lap + c; requires c > -(lambda_x,1 + lambda_y,1 +
 *                lambda_z,1) so that the operator is positive definite.
 *   out        : receives the handle (owned by the caller, freed by
 *                sem3d_destroy).
 * Synchronous with respect to the host.  Default mode: SEM3D_FP64, 1 sweep. */
sem3d_status sem3d_setup(int nx, int ny, int nz, int k, double Lx, double Ly, double Lz, double c,
                         sem3d_handle* out);

/* Homogeneous boundary data of a plan (Section 2.2 treats Dirichlet data by
 * dropping the boundary nodes; the appendix assembles the Neumann problem,
 * whose natural boundary condition keeps every node; Table 1 has both). */
typedef enum { SEM3D_BC_DIRICHLET = 0, SEM3D_BC_NEUMANN = 1 } sem3d_bc;

/* sem3d_setup with a choice of boundary condition.  SEM3D_BC_DIRICHLET is
 * sem3d_setup.  SEM3D_BC_NEUMANN: homogeneous Neumann data du/dn = 0 on every
 * face; the unknowns are all n = Ne*k + 1 GLL nodes of each axis, so each n
 * must satisfy (n-1) % k == 0 and n > k, nodes run from 0 to L inclusive,
 * and c > 0 is required (lambda = 0 belongs to the constant mode).  Neumann
 * plans compute every refinement residual in FP64 with the per-row banded
 * operator (SEM3D_RESIDUAL_MIXED acts as SEM3D_RESIDUAL_FP64) and do not
 * support SEM3D_F16X3 (SEM3D_ERR_UNSUPPORTED). */
sem3d_status sem3d_setup_bc(int nx, int ny, int nz, int k, double Lx, double Ly, double Lz, double c, sem3d_bc bc,
                            sem3d_handle* out);

/* Select the arithmetic of the mode products and the number of FP64
 * iterative-refinement sweeps (each sweep: FP64 residual r = f - (c + H_x (+)
 * H_y (+) H_z) u with the banded operator of Eq. 12, a solve of the correction
 * in the selected arithmetic, u += correction).  sweeps in [0, 16].
 * With a fixed sweep count the solve performs no host synchronisation.
 * Errors: SEM3D_ERR_INVALID_ARG for an unknown precision or sweep count;
 * SEM3D_ERR_UNSUPPORTED for the tensor-core tiers (TF32, BF16, BF16X3,
 * F16X3) on a GPU other than sm_103, and for F16X3 with k > 8 or Neumann
 * data.  A plan-owned workspace grows on the next solve if the new tier
 * needs more (sem3d_workspace_size); with a caller-owned workspace that is
 * too small the next solve fails with SEM3D_ERR_INVALID_ARG. */
sem3d_status sem3d_set_precision(sem3d_handle h, sem3d_precision p, int sweeps);

/* Arithmetic of the refinement residuals in the SEM3D_BF16X3 / F16X3 tiers.
 *   SEM3D_RESIDUAL_FP64  : every sweep computes r = f - (c + H_x (+) H_y (+)
 *                          H_z) u in FP64 with the banded operator of Eq. 12.
 *   SEM3D_RESIDUAL_MIXED : (default) sweeps 1 .. s-1 compute it in double-FP32
 *                          arithmetic (pairs of FP32 numbers, ~48 significant
 *                          bits; products by the FMA error-free transform)
 *                          with the solution held as a double-FP32 pair; the
 *                          last sweep computes it in FP64 on the FP64
 *                          solution.  The final accuracy is that of the last
 *                          (FP64) residual.  Applies for k <= 8 and s >= 2;
 *                          otherwise every sweep is FP64.
 *   SEM3D_RESIDUAL_DF    : every sweep in double-FP32 arithmetic, the last one
 *                          writing the FP64 solution; the rows of H enter as
 *                          exact three-term FP32 sums (a 48-bit operator
 *                          would be a different operator: 8e-11 at n=999).
 *                          Not FP64 refinement: the residual carries ~2^-48
 *                          of the operator's terms, amplified by the
 *                          conditioning of the operator: measured 1.5e-12 at
 *                          n=383 and 7e-12 at n=999 from the FP64-residual
 *                          result (against 9e-15 with the FP64 last sweep),
 *                          in 11% less time; for k <= 8 with Dirichlet data,
 *                          else every sweep is FP64.
 * The FP64 tier always uses FP64 residuals. */
typedef enum { SEM3D_RESIDUAL_FP64 = 0, SEM3D_RESIDUAL_MIXED = 1, SEM3D_RESIDUAL_DF = 2 } sem3d_residual;
sem3d_status sem3d_set_residual(sem3d_handle h, sem3d_residual mode);

/* How the split tiers (SEM3D_BF16X3, SEM3D_BF16) and the TF32 tier evaluate
 * their FP64-accurate residuals (split tiers: every sweep of
 * SEM3D_RESIDUAL_FP64, the last sweep of SEM3D_RESIDUAL_MIXED; TF32: every
 * sweep) -- the same r = f - (c + H_x (+) H_y (+) H_z) u of Eq. 12 either way:
 *   SEM3D_EXACT_FIXED : (default) exactly in 64-bit integer fixed point on
 *                       the integer pipe: u and f scaled by one power of two
 *                       per field (found on the device from their largest
 *                       exponents) to 58 / 61-bit integers, the rows of H to
 *                       integers whose magnitudes over a node's terms sum to
 *                       ~2^58; products and sums are exact, and the
 *                       truncations and dropped low partial products leave
 *                       an absolute error below 2^-53 of the largest
 *                       sum of |H||u| over the grid -- within one FP64
 *                       rounding of that sum (normwise: nodes where |u| is
 *                       far below max |u| get the field's absolute
 *                       resolution).
 *                       Dirichlet plans with k <= 8; other plans use
 *                       FP64 arithmetic.  Inf or NaN in u or f gives a NaN
 *                       residual.
 *   SEM3D_EXACT_FP64  : FP64 fused multiply-adds.
 * sem3d_exact_residual_kind reports the arithmetic the plan's current tier
 * and geometry use (SEM3D_EXACT_FP64 for the FP64, FP32 and F16X3 tiers).
 * Errors: SEM3D_ERR_INVALID_ARG for a NULL handle / pointer or unknown kind. */
typedef enum { SEM3D_EXACT_FIXED = 0, SEM3D_EXACT_FP64 = 1 } sem3d_exact_residual;
sem3d_status sem3d_set_exact_residual(sem3d_handle h, sem3d_exact_residual kind);
sem3d_status sem3d_exact_residual_kind(sem3d_handle h, int* kind);

/* Bytes of device workspace that sem3d_solve needs in the current mode. */
sem3d_status sem3d_workspace_size(sem3d_handle h, size_t* bytes);

/* Hand the plan a caller-owned device workspace of at least
 * sem3d_workspace_size bytes (256-byte aligned); it stays owned by the caller
 * and must outlive every solve that uses it.  Without this call the plan
 * allocates its own workspace on the first solve (cudaMalloc). */
sem3d_status sem3d_set_workspace(sem3d_handle h, void* dptr, size_t bytes);

/* Solve (c + H_x (+) H_y (+) H_z) u = f, equivalently the weak form
 * A u = (M (x) M (x) M) f of Eq. 12 with the alpha term c M (x) M (x) M.
 *   f, u : device FP64 arrays of nx*ny*nz values (layout above); f and u must
 *          not overlap.  u is fully overwritten.
 * Enqueued on `stream`; no host synchronisation. */
sem3d_status sem3d_solve(sem3d_handle h, const double* f, double* u, void* stream);

/* sem3d_solve with the data in HOST memory, pipelined across calls.  Each
 * call copies f_host to the device, solves in the plan's mode on `stream` and
 * copies the result to u_host, all asynchronously: the copies use the plan's
 * own host->device and device->host streams and two device (f, u) pairs used in
 * turn, so consecutive calls overlap one call's copies with another's solve
 * (the copy engines run both directions at once).  The first call allocates the
 * two pairs (4 * nx*ny*nz doubles).  f_host and u_host should be pinned
 * (cudaHostAlloc / cudaHostRegister) for the copies to be asynchronous; f_host
 * must stay unchanged and u_host unread until sem3d_solve_host_wait's stream
 * work has completed.  Calls on one plan must come from one host thread. */
sem3d_status sem3d_solve_host(sem3d_handle h, const double* f_host, double* u_host, void* stream);

/* Make `stream` wait for the device->host copies of every earlier
 * sem3d_solve_host call of this plan (the results are in host memory once the
 * stream's work up to this point has completed; synchronise it or record an
 * event). */
sem3d_status sem3d_solve_host_wait(sem3d_handle h, void* stream);

/* Many independent solves (a batch of Helmholtz problems; each problem is
 * Section 2.4's solve on its own box, grid, degree and shift).
 *   count : number of problems, 1 <= count <= 1024.
 *   hs    : count distinct plans on the current device; each keeps its own
 *           precision, sweeps and workspace.
 *   f, u  : host arrays of count device pointers (as in sem3d_solve).
 * When every plan is SEM3D_FP32 with the same sweep count (and count <= 64),
 * each of the six mode-product passes of all problems runs as ONE grouped
 * launch (per-problem descriptors in a device table); the FP64 residuals run
 * per problem.  Otherwise the problems' solves run concurrently on a pool of
 * streams forked from and joined to `stream`.  Asynchronous; the library's
 * batch staging area is shared, so concurrent batched calls from several host
 * threads are serialised internally. */
sem3d_status sem3d_solve_batched(int count, const sem3d_handle* hs, const double* const* f, double* const* u,
                                 void* stream);

/* Apply the discrete operator in H form: Au = c u + (H_x (+) H_y (+) H_z) u
 * (Eq. 12 with H = M^{-1} S, banded, at most 2k+1 entries per row and axis),
 * in FP64.  u, Au: device FP64 arrays, must not overlap. */
sem3d_status sem3d_apply(sem3d_handle h, const double* u, double* Au, void* stream);

/* Preconditioned conjugate gradient for -Lap u + V(x) u = f (Section 3.3,
 * Eq. 15: the SEM operator with a variable potential, preconditioned by the
 * fast solver of a constant-coefficient operator; the paper uses
 * (alpha + beta/2) - Lap).  The preconditioner is this plan's solve: its shift
 * c (sem3d_setup) is the constant (e.g. the mean of V), its precision and
 * sweeps (sem3d_set_precision) its arithmetic.  Operator apply (banded FP64
 * stencil plus V u), dot products and vector updates are FP64.  The inner
 * product is weighted by the lumped GLL mass M (x) M (x) M, which makes the
 * iteration CG on the symmetric weak form S(+)S(+)S + (M(x)M(x)M) diag(V).
 *   V, f   : device FP64 nodal arrays (layout as in sem3d_solve).
 *   u      : device FP64 solution, overwritten; the iteration starts at u = 0.
 *   rtol   : stop when ||M3 r||_2 <= rtol * ||M3 f||_2 (weak-form residual).
 *   maxit  : iteration limit, >= 1.
 *   iters, relres : host outputs (may be NULL): iterations run, final ratio.
 * Every iteration after the first replays a CUDA graph of the iteration body
 * on a plan-owned stream joined to `stream` by events; the host reads the
 * residual norm after each iteration, so the call is synchronous.  Uses six
 * FP64 arrays of nx*ny*nz plan-owned device memory (allocated on first use).
 * Returns SEM3D_ERR_NOT_CONVERGED when maxit is reached or the residual
 * becomes non-finite (iters and relres are still written). */
sem3d_status sem3d_pcg(sem3d_handle h, const double* V, const double* f, double* u, double rtol, int maxit,
                       int* iters, double* relres, void* stream);

/* One BDF2 time step of the Cahn-Hilliard equation (Section 3.5, Eqs. 17-20):
 * phi_t = m Lap mu, mu = -eps Lap phi + F'(phi)/eps, F(phi) = (phi^2-1)^2/4,
 * with homogeneous Dirichlet data for phi and Lap phi.  With a = 3/2,
 * phi_hat = 2 phi_n - phi_{n-1}/2, phi_bar = 2 phi_n - phi_{n-1}:
 *   (a + dt m (eps Lap^2 - (S/eps) Lap)) phi_{n+1}
 *        = phi_hat + (dt m / eps) Lap (F'(phi_bar) - S phi_bar),
 * solved in the plan's eigenbasis (the paper's Eq. 20: the two operators
 * share T): prep, two forward transforms, a pointwise combination, one
 * backward transform (9 mode products).  S is a stabilisation constant (the
 * paper borrows one without printing it; this reading adds
 * (S/eps)(phi_{n+1} - phi_bar) to mu; S = 0 is the printed scheme).
 * Arithmetic: the plan's precision (FP64 DMMA, FP32, BF16X3 or BF16 tensor
 * cores; no refinement), the plan's shift c is not used.
 *   phi_n, phi_nm1 : device FP64 arrays (layout as in sem3d_solve).
 *   phi_np1        : device FP64 output, must not overlap the inputs.
 *   eps, m, dt > 0, S >= 0. */
sem3d_status sem3d_ch_step(sem3d_handle h, const double* phi_n, const double* phi_nm1, double* phi_np1, double eps,
                           double m, double dt, double S, void* stream);

/* nsteps BDF2 steps in place: on entry phi_nm1, phi_n hold phi_{-1}, phi_0
 * (pass the same values twice for a cold start), on return phi_{N-1}, phi_N.
 * Steps run on a plan-owned stream joined to `stream` by events; after the
 * first step, groups of three steps are replayed from one CUDA graph (three
 * steps rotate the three phi buffers back to their roles).  Uses one extra
 * plan-owned FP64 array (allocated on first use).  Asynchronous. */
sem3d_status sem3d_ch_run(sem3d_handle h, double* phi_nm1, double* phi_n, int nsteps, double eps, double m, double dt,
                          double S, void* stream);

/* Axis data (axis 0 = x, 1 = y, 2 = z), copied to host memory; synchronous.
 *   x_host      : n_axis node coordinates of the interior nodes.
 *   lambda_host : n_axis eigenvalues of H, ascending (may be NULL).
 *   T_host      : n_axis*n_axis FP64, column-major, column j = eigenvector of
 *                 lambda_j (T of Section 2.3); may be NULL. */
sem3d_status sem3d_get_nodes(sem3d_handle h, int axis, double* x_host);
sem3d_status sem3d_get_eigs(sem3d_handle h, int axis, double* lambda_host, double* T_host);

/* Host only (no device needed): the 1D data of one axis exactly as
 * sem3d_setup builds it for n interior nodes of degree k on [0, L] (GLL
 * nodes by Newton's method, closed-form GLL differentiation matrix, assembled
 * S and lumped M, Householder + implicit-QR eigen-decomposition of
 * S1 = M^{-1/2} S M^{-1/2}; Section 2.3 and the Appendix of the paper).
 * Output arrays (host, caller-allocated, any may be NULL):
 *   x[n] nodes, M[n] mass diagonal, lambda[n] ascending eigenvalues,
 *   T[n*n] column-major eigenvectors (column j <-> lambda_j, T = M^{-1/2} Q,
 *   sign fixed so that the largest |entry| of each column is positive). */
sem3d_status sem3d_axis_info(int n, int k, double L, double* x, double* M, double* lambda, double* T);

/* Wait for the work enqueued on `stream` and report errors that kernels of
 * this plan recorded on the device: SEM3D_ERR_TIMEOUT if a bounded wait inside
 * a tensor-core kernel expired (the kernel then stopped early and its output
 * is invalid), SEM3D_ERR_CUDA for an asynchronous CUDA error.  Clears the
 * recorded flags.  Synchronous with respect to the host. */
sem3d_status sem3d_sync_check(sem3d_handle h, void* stream);

/* Per-kernel timing for measurement tools.  sem3d_profile(h, 1) discards
 * earlier records and, from then on, brackets every kernel launch of this plan
 * with CUDA events recorded on the launch's stream; sem3d_profile(h, 0) stops.
 * sem3d_profile_read synchronises on the recorded events and returns, for one
 * kernel class, the number of kernels launched and their summed device time
 * in milliseconds.  Kernel classes: 0 = tensor-core (tcgen05) mode product,
 * 1 = FP64 (DMMA) mode product, 2 = FP64 stencil / residual, 3 = FP64 ->
 * split-bf16 conversion; the tensor-core launches of class 0 are also counted
 * by pass: 4 = x pass, 5 = y pass, 6 = z pass writing split-bf16 output,
 * 7 = the last pass of a solve (writes or accumulates FP64 u); 8 = FP32
 * CUDA-core mode product. */
sem3d_status sem3d_profile(sem3d_handle h, int enable);
sem3d_status sem3d_profile_read(sem3d_handle h, int kind, long long* launches, double* total_ms);

/* The FP32 mode-product configuration the autotuner chose for this plan's
 * pass along `axis` (0 = x, 1 = y, 2 = z).  sem3d_set_precision(h, SEM3D_FP32,
 * ...) measures six configurations of the FP32 CUDA-core kernel on each pass
 * shape of the plan that the process has not measured before (synchronous;
 * scratch buffers of up to 65536 * n floats twice) and keeps the fastest:
 *   0 = 128 x 128 output tile, 8 x 8 per thread, two shared-memory stages,
 *   1 = 128 x 64, 8 x 4, two stages,   2 = 64 x 64, 4 x 4, two stages,
 *   3..5 = the same three tiles with one stage.
 * Shapes never measured report 0 (the default).  The grouped launch of
 * sem3d_solve_batched uses the two-stage tile of the same shape. */
sem3d_status sem3d_tuned_config(sem3d_handle h, int axis, int* config);
/* Pin `config` (0..5) for the pass shape of this plan's `axis`, replacing the
 * measured choice for every plan of the process with that pass shape (until
 * the next pin; sem3d_set_precision does not re-measure a known shape). */
sem3d_status sem3d_set_tuned_config(sem3d_handle h, int axis, int config);

/* Tensor-core kernel of this plan's mode product along `axis` (0 = x, 1 = y,
 * 2 = z) in the SEM3D_BF16X3, SEM3D_BF16 and SEM3D_TF32 tiers (SEM3D_F16X3
 * always uses 0):
 *   0 = one CTA per 128-row x 256-output tile, the W tile multicast by TMA
 *       across clusters of 4 CTAs, 4 pipeline stages;
 *   1 = one cta_group::2 MMA per pair of SMs on 256 x 256 tiles, each CTA of
 *       the pair staging its 128 rows and half of the W tile, 6 stages.
 * Both compute the same products in the same order (bit-identical results).
 * sem3d_set_precision(h, SEM3D_BF16X3, SEM3D_BF16 or SEM3D_TF32, ...) times
 * both on a synthetic pass of each pass shape the process has not measured
 * before (synchronous; up to 512 MB of scratch, freed again) and keeps the
 * faster one in a process-wide table (split tiers: keyed by axis, nx, ny, nz
 * and products per pass; TF32: by the pass's contracted length and its two
 * row extents).  sem3d_tc_config reports the choice for the plan's current
 * tier (0 for a shape never measured); sem3d_set_tc_config pins `config` (0
 * or 1) for this plan's pass along `axis` in all three tiers, for every plan
 * of the process with that shape (sem3d_set_precision does not re-measure a
 * known shape). */
sem3d_status sem3d_tc_config(sem3d_handle h, int axis, int* config);
sem3d_status sem3d_set_tc_config(sem3d_handle h, int axis, int config);

/* Failure-detection testing (no counterpart in the paper).  The next
 * `launches` tensor-core kernel launches of the process (any plan) issue no
 * operand loads: their bounded waits (1 s each, on mbarriers that nothing then
 * arms) expire, the kernels record SEM3D_ERR_TIMEOUT, release their tensor
 * memory and return, and the next sem3d_sync_check reports the timeout.  No
 * GPU fault is raised; the plan and the CUDA context stay usable, and later
 * solves are correct.  0 cancels.  launches in [0, 64]; h only validates. */
sem3d_status sem3d_inject_stall(sem3d_handle h, int launches);

/* Total number of kernels this plan has launched since sem3d_setup. */
sem3d_status sem3d_launch_count(sem3d_handle h, unsigned long long* count);

/* Release the plan and every device buffer it allocated (not caller-owned
 * workspace).  Synchronises the device first.  NULL is accepted. */
sem3d_status sem3d_destroy(sem3d_handle h);

/* FP64 solve that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library call cudaMalloc,
 * for example a program whose device memory belongs to another allocator, one
 * that reserves all device memory up front, or one that must avoid the
 * implicit device synchronisation cudaMalloc and cudaFree may cause.
 *   Computes the same result as sem3d_solve in SEM3D_FP64 mode (DMMA mode
 *   products and the plan's number of FP64 refinement sweeps, whatever
 *   precision the plan is set to), with its scratch in one fixed device array
 *   of 3 * 524288 doubles (12 MiB) compiled into the library: every GPU that
 *   loads the library holds that array until the process exits.
 *   Limit: nx*ny*nz <= 524288 (e.g. 63^3 or 80^3); larger grids return
 *   SEM3D_ERR_INVALID_ARG with a message naming the limit.
 *   f, u : device FP64 arrays as in sem3d_solve; must not overlap.
 *   The current device must be the plan's device.  The first call on a device
 *   (and the first after a cudaDeviceReset, which gives the array a new
 *   address) looks up the array's device address (cudaGetSymbolAddress), so
 *   make that first call before any stream capture.  No cudaMalloc, cudaFree,
 *   event creation or other allocating call is made: the plan's own workspace
 *   is neither allocated nor used, and sem3d_profile does not time these
 *   launches (they are counted by sem3d_launch_count).
 *   All calls share the one array and leave their intermediates in it; calls
 *   whose work overlaps on the GPU (other streams, other threads, other plans
 *   on the same device) race on it and must be serialised by the caller. */
sem3d_status sem3d_solve_fp64_static(sem3d_handle h, const double* f, double* u, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* sem3d_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM3D_H */
