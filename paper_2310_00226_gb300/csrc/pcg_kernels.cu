// Vector kernels of the preconditioned conjugate gradient for
// -Lap u + V(x) u = f (Section 3.3 of the paper, Eq. 15: PCG on the SEM
// operator with the fast solver of a constant-coefficient operator as the
// preconditioner).  All arithmetic is FP64.
//
// The iteration works on H-form vectors (nodal values).  The operator
// A_V = H_x (+) H_y (+) H_z + diag(V), H = M^{-1} S, is self-adjoint in the
// inner product <a, b> = sum M3 a b with M3 = M_x (x) M_y (x) M_z (the lumped
// GLL mass), so every dot product carries that weight; with it the iteration
// is exactly CG on the symmetric weak form S(+)S(+)S + M3 diag(V).
// Scalars (alpha, beta, dot products) live in device memory, so an iteration
// needs no host round trip and can be captured in a CUDA graph.
#include "sem3d_internal.h"

namespace sem3d {

namespace {

constexpr int PCG_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[PCG_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) warp_part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < PCG_THREADS / 32 ? warp_part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  }
  return s;  // valid in thread 0
}

__device__ __forceinline__ double weight(const PcgArgs& a, long long idx) {
  const long long i = idx % a.nx, jl = idx / a.nx;
  return a.Mx[i] * a.My[jl % a.ny] * a.Mz[jl / a.ny];
}

// M3 = Mx (x) My (x) Mz, Vmc = V - c (the preconditioner's shift c is inside
// the stencil's H table), u = 0, r = f, p = 0; bnorm2 = sum (M3 f)^2.
__global__ void __launch_bounds__(PCG_THREADS) pcg_init_kernel(PcgArgs a) {
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const double w = weight(a, idx);
    a.M3[idx] = w;
    a.Vmc[idx] = a.V[idx] - a.c;
    a.u[idx] = 0.0;
    a.p[idx] = 0.0;
    const double f = a.f[idx];
    a.r[idx] = f;
    const double wf = w * f;
    acc += wf * wf;
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(&a.sc->bnorm2, s);
}

// rz_new = <r, z>
__global__ void __launch_bounds__(PCG_THREADS) pcg_dot_rz_kernel(PcgArgs a) {
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.N;
       idx += (long long)gridDim.x * blockDim.x)
    acc += a.M3[idx] * a.r[idx] * a.z[idx];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(&a.sc->rz_new, s);
}

// beta = rz_new / rz_old (0 on the first iteration), rz_old = rz_new; clear
// the accumulators of this iteration's remaining dot products.
__global__ void pcg_beta_kernel(PcgScalars* sc) {
  sc->beta = (sc->iter == 0 || sc->rz_old == 0.0) ? 0.0 : sc->rz_new / sc->rz_old;
  sc->rz_old = sc->rz_new;
  sc->rz_new = 0.0;
  sc->pq = 0.0;
  sc->rnorm2 = 0.0;
}

// p = z + beta p
__global__ void __launch_bounds__(PCG_THREADS) pcg_p_kernel(PcgArgs a) {
  const double beta = a.sc->beta;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.N;
       idx += (long long)gridDim.x * blockDim.x)
    a.p[idx] = a.z[idx] + beta * a.p[idx];
}

// q += (V - c) p (q holds (c + H (+) H (+) H) p), pq = <p, q>
__global__ void __launch_bounds__(PCG_THREADS) pcg_q_kernel(PcgArgs a) {
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const double p = a.p[idx];
    const double q = a.q[idx] + a.Vmc[idx] * p;
    a.q[idx] = q;
    acc += a.M3[idx] * p * q;
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(&a.sc->pq, s);
}

// alpha = rz_old / pq, u += alpha p, r -= alpha q, rnorm2 = sum (M3 r)^2
__global__ void __launch_bounds__(PCG_THREADS) pcg_update_kernel(PcgArgs a) {
  const double alpha = a.sc->pq != 0.0 ? a.sc->rz_old / a.sc->pq : 0.0;
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.N;
       idx += (long long)gridDim.x * blockDim.x) {
    a.u[idx] += alpha * a.p[idx];
    const double r = a.r[idx] - alpha * a.q[idx];
    a.r[idx] = r;
    const double wr = a.M3[idx] * r;
    acc += wr * wr;
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(&a.sc->rnorm2, s);
}

__global__ void pcg_count_kernel(PcgScalars* sc) { sc->iter += 1; }

int pcg_grid(long long N) {
  long long b = (N + PCG_THREADS - 1) / PCG_THREADS;
  if (b > 152LL * 16) b = 152LL * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_pcg(int op, const PcgArgs& a, cudaStream_t s) {
  const int g = pcg_grid(a.N);
  switch (op) {
    case PCG_INIT: pcg_init_kernel<<<g, PCG_THREADS, 0, s>>>(a); break;
    case PCG_DOT_RZ: pcg_dot_rz_kernel<<<g, PCG_THREADS, 0, s>>>(a); break;
    case PCG_BETA: pcg_beta_kernel<<<1, 1, 0, s>>>(a.sc); break;
    case PCG_P: pcg_p_kernel<<<g, PCG_THREADS, 0, s>>>(a); break;
    case PCG_Q: pcg_q_kernel<<<g, PCG_THREADS, 0, s>>>(a); break;
    case PCG_UPDATE: pcg_update_kernel<<<g, PCG_THREADS, 0, s>>>(a); break;
    case PCG_COUNT: pcg_count_kernel<<<1, 1, 0, s>>>(a.sc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sem3d
