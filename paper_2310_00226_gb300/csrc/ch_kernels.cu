// Pointwise kernels of the Cahn-Hilliard BDF2 step (Section 3.5, Eqs. 19-20).
//
// With -Lap -> H3 = T3 diag(L) T3^{-1} (L = lambda_x,i + lambda_y,j +
// lambda_z,l), one step is
//   phi_{n+1} = T3 [ (T3^{-1} phi_hat - dt m L * T3^{-1} g)
//                    / (a + dt m (eps L^2 + (S/eps) L)) ]
// phi_hat = 2 phi_n - phi_{n-1}/2, g = (F'(phi_bar) - S phi_bar)/eps,
// phi_bar = 2 phi_n - phi_{n-1}, F'(phi) = phi^3 - phi, a = 3/2.  The two
// forward transforms and the backward one are the solver's mode products;
// these kernels do the pointwise parts (prep before, combine in between).
#include "sem3d_internal.h"

namespace sem3d {

namespace {

constexpr int CH_THREADS = 256;

int ch_grid(long long n) {
  long long b = (n + CH_THREADS - 1) / CH_THREADS;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)(b < 1 ? 1 : b);
}

// Grid of the line kernels: a block walks lines blockIdx.x, + gridDim.x, ...;
// 16 blocks per SM (two waves of 8 resident), so that block launches are few
// against the work (a line of Px elements is only 2-4 elements per thread).
int line_grid(long long lines) { return (int)(lines < 152LL * 16 ? (lines < 1 ? 1 : lines) : 152LL * 16); }

__device__ __forceinline__ void split2f(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// FP64 / FP32 inputs: phi_hat and g at pitch nx.
template <typename T>
__global__ void __launch_bounds__(CH_THREADS) ch_prep_kernel(const double* phi_n, const double* phi_nm1, T* ghat,
                                                             T* g, long long N, ChParams c) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double pn = phi_n[i], pm = phi_nm1[i];
    const double bar = 2.0 * pn - pm;
    ghat[i] = (T)(2.0 * pn - 0.5 * pm);
    g[i] = (T)((bar * bar * bar - bar - c.S * bar) / c.eps);
  }
}

// Split-bf16 inputs (pitch Px, zero pads), FP32 arithmetic.  Blocks walk the
// (j, l) lines, their threads along i.
__global__ void __launch_bounds__(CH_THREADS) ch_prep_split_kernel(const double* phi_n, const double* phi_nm1,
                                                                   __nv_bfloat16* gh_hi, __nv_bfloat16* gh_lo,
                                                                   __nv_bfloat16* g_hi, __nv_bfloat16* g_lo, int nx,
                                                                   int Px, long long lines, ChParams c) {
  const float S = (float)c.S, inv_eps = (float)(1.0 / c.eps);
  for (long long line = blockIdx.x; line < lines; line += gridDim.x) {
    const double* pn_row = phi_n + line * nx;
    const double* pm_row = phi_nm1 + line * nx;
    const long long o = line * Px;
    for (int i = threadIdx.x; i < Px; i += blockDim.x) {
      float gh = 0.f, gg = 0.f;
      if (i < nx) {
        const float pn = f64_to_f32_rn(pn_row[i]), pm = f64_to_f32_rn(pm_row[i]);
        const float bar = 2.f * pn - pm;
        gh = 2.f * pn - 0.5f * pm;
        gg = (bar * bar * bar - bar - S * bar) * inv_eps;
      }
      split2f(gh, gh_hi[o + i], gh_lo[o + i]);
      split2f(gg, g_hi[o + i], g_lo[o + i]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(CH_THREADS) ch_combine_kernel(const T* a1, const T* a2, T* out, const double* lx,
                                                                const double* ly, const double* lz, int nx, int ny,
                                                                long long N, ChParams c) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % nx, jl = idx / nx;
    const double L = lx[i] + ly[jl % ny] + lz[jl / ny];
    const double num = (double)a1[idx] - c.dt * c.m * L * (double)a2[idx];
    const double den = 1.5 + c.dt * c.m * (c.eps * L * L + (c.S / c.eps) * L);
    out[idx] = (T)(num / den);
  }
}

__global__ void __launch_bounds__(CH_THREADS) ch_combine_split_kernel(
    const __nv_bfloat16* a1h, const __nv_bfloat16* a1l, const __nv_bfloat16* a2h, const __nv_bfloat16* a2l,
    __nv_bfloat16* oh, __nv_bfloat16* ol, const float* lx, const float* ly, const float* lz, int nx, int ny, int Px,
    long long lines, ChParams c) {
  const float dtm = (float)(c.dt * c.m), eps = (float)c.eps, s_eps = (float)(c.S / c.eps);
  for (long long line = blockIdx.x; line < lines; line += gridDim.x) {
    const float lyz = ly[line % ny] + lz[line / ny];  // block-uniform
    const long long o = line * Px;
    for (int i = threadIdx.x; i < Px; i += blockDim.x) {
      float v = 0.f;
      if (i < nx) {
        const float L = lx[i] + lyz;
        const float x1 = __bfloat162float(a1h[o + i]) + __bfloat162float(a1l[o + i]);
        const float x2 = __bfloat162float(a2h[o + i]) + __bfloat162float(a2l[o + i]);
        v = (x1 - dtm * L * x2) / (1.5f + dtm * (eps * L * L + s_eps * L));
      }
      split2f(v, oh[o + i], ol[o + i]);
    }
  }
}

}  // namespace

cudaError_t launch_ch_prep(int tier, const Geom& g, const double* phi_n, const double* phi_nm1, void* ghat, void* gg,
                           TcBuffers sh, TcBuffers sg, const ChParams& c, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  if (tier == SEM3D_FP64) {
    ch_prep_kernel<double><<<ch_grid(N), CH_THREADS, 0, s>>>(phi_n, phi_nm1, static_cast<double*>(ghat),
                                                               static_cast<double*>(gg), N, c);
  } else if (tier == SEM3D_FP32) {
    ch_prep_kernel<float><<<ch_grid(N), CH_THREADS, 0, s>>>(phi_n, phi_nm1, static_cast<float*>(ghat),
                                                              static_cast<float*>(gg), N, c);
  } else {
    const long long lines = (long long)g.ny * g.nz;
    ch_prep_split_kernel<<<line_grid(lines), CH_THREADS, 0, s>>>(phi_n, phi_nm1, sh.hi, sh.lo, sg.hi, sg.lo, g.nx,
                                                                  g.Px, lines, c);
  }
  return cudaGetLastError();
}

cudaError_t launch_ch_combine(int tier, const Geom& g, const DevAxis* ax, const void* a1, const void* a2, void* out,
                              TcBuffers s1, TcBuffers s2, TcBuffers so, const ChParams& c, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  if (tier == SEM3D_FP64) {
    ch_combine_kernel<double><<<ch_grid(N), CH_THREADS, 0, s>>>(
        static_cast<const double*>(a1), static_cast<const double*>(a2), static_cast<double*>(out), ax[0].lam,
        ax[1].lam, ax[2].lam, g.nx, g.ny, N, c);
  } else if (tier == SEM3D_FP32) {
    ch_combine_kernel<float><<<ch_grid(N), CH_THREADS, 0, s>>>(
        static_cast<const float*>(a1), static_cast<const float*>(a2), static_cast<float*>(out), ax[0].lam,
        ax[1].lam, ax[2].lam, g.nx, g.ny, N, c);
  } else {
    const long long lines = (long long)g.ny * g.nz;
    ch_combine_split_kernel<<<line_grid(lines), CH_THREADS, 0, s>>>(
        s1.hi, s1.lo, s2.hi, s2.lo, so.hi, so.lo, ax[0].lamf, ax[1].lamf, ax[2].lamf, g.nx, g.ny, g.Px, lines, c);
  }
  return cudaGetLastError();
}

}  // namespace sem3d
