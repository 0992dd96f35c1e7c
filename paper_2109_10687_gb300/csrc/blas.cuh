// Reduction machinery, the per-right-hand-side scalar record and the fused
// BLAS-1 kernels of the BiCGStab iteration (Algorithm 5 of
// arXiv:2109.10687), shared by the single-lattice solver and the ragged
// batch solver.
//
// Reductions: every reducing kernel accumulates per thread in float32,
// combines warps and blocks in float64 and lets the last block to finish sum
// the per-block partials in a fixed order, so results do not depend on
// scheduling.  Kernels run on a grid (blocks, k) with blockIdx.y = k the
// right-hand side (or, in a ragged batch, the lattice); a Seg says where
// element k of a stacked vector lives.
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

constexpr int RED_THREADS = 256;
constexpr int MAX_RED_OUT = 4;

// The scalars of one right-hand side's BiCGStab iteration, in device memory.
struct Scal {
  double rho0_re, rho0_im;
  double alpha_re, alpha_im;
  double omega_re, omega_im;
  double beta_re, beta_im;
  double rnorm2, bnorm2;
  double tol2;  // stop when rnorm2 < tol2 * bnorm2
  double aux;
  int done;     // 1: converged or failed; no further updates
  int status;   // QCD_OK, QCD_ERR_BREAKDOWN, QCD_ERR_NONFINITE
  int conv;     // 1: converged
  int iters;   // iterations begun (counted by k_alpha)
  int xpend;   // 1: x += alpha z_p of this iteration not yet applied (k_update2 or k_xfinal does it)
};

// Where element k of a stacked vector lives: uniform stacking (element k at
// k n, n entries) or ragged (off[k], len[k] entries; off and len in device
// memory).
struct Seg {
  size_t n;
  const size_t* off = nullptr;
  const size_t* len = nullptr;
  __device__ __forceinline__ size_t at(int k) const { return off ? __ldg(off + k) : (size_t)k * n; }
  __device__ __forceinline__ size_t size(int k) const { return off ? __ldg(len + k) : n; }
};

// ---------------------------------------------------------------------------
// reduction machinery
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void block_sum(double v[N], double* sh /* [32][N] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sh[warp * N + k] = v[k];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      v[k] = lane < nw ? sh[lane * N + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
  }
  __syncthreads();
}

// Writes this block's partials; returns true (in every thread) in the block
// that finished last, which then holds the totals in tot[] (all threads).
template <int N>
__device__ bool grid_reduce(double v[N], double* partials, unsigned* counter, double tot[N]) {
  __shared__ double sh[32 * N];
  __shared__ bool is_last;
  block_sum<N>(v, sh);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) partials[blockIdx.x * N + k] = v[k];
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    is_last = prev == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double w[N];
#pragma unroll
  for (int k = 0; k < N; ++k) w[k] = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] += __ldcg(partials + i * N + k);
  block_sum<N>(w, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) sh[k] = w[k];
    *counter = 0;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) tot[k] = sh[k];
  __syncthreads();
  return true;
}

// complex (a.x + i a.y) * (b.x + i b.y) for the two complex numbers of a float4
__device__ __forceinline__ float4 caxpy4(float ar, float ai, float4 xv, float4 y) {
  y.x = fmaf(ar, xv.x, fmaf(-ai, xv.y, y.x));
  y.y = fmaf(ar, xv.y, fmaf(ai, xv.x, y.y));
  y.z = fmaf(ar, xv.z, fmaf(-ai, xv.w, y.z));
  y.w = fmaf(ar, xv.w, fmaf(ai, xv.z, y.w));
  return y;
}
__device__ __forceinline__ void cdot_acc(float4 a, float4 b, float& re, float& im) {
  re = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, re))));
  im = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, im))));
}
__device__ __forceinline__ float norm4(float4 a) { return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w; }

// kernels of Algorithm 5 (defined in solver.cu): grid (blocks, k), RED_THREADS threads
__global__ void k_init(const float4* __restrict__ b, float4* x, float4* r, float4* p, float4* rt, Seg seg,
                       double tol2, Scal* scal, double* partials, unsigned* counters, int* ctrl);
__global__ void k_alpha(const float4* __restrict__ rt, const float4* __restrict__ q, Seg seg, Scal* scal,
                        double* partials, unsigned* counters, int* ctrl);
__global__ void k_update1(float4* x, float4* r, const float4* __restrict__ z, const float4* __restrict__ q, Seg seg,
                          Scal* scal, double* partials, unsigned* counters, int* ctrl);
__global__ void k_omega(const float4* __restrict__ t, const float4* __restrict__ r, Seg seg, Scal* scal,
                        double* partials, unsigned* counters, int* ctrl);
__global__ void k_update2(float4* x, float4* r, const float4* __restrict__ zp, const float4* __restrict__ z,
                          const float4* __restrict__ t, const float4* __restrict__ rt, Seg seg, Scal* scal,
                          double* partials, unsigned* counters, int* ctrl);
__global__ void k_update_p(float4* p, const float4* __restrict__ r, const float4* __restrict__ q, Seg seg,
                           Scal* scal);
__global__ void k_xfinal(float4* x, const float4* __restrict__ z, Seg seg, const Scal* scal);
__global__ void k_loop_cond(cudaGraphConditionalHandle handle, int* ctrl);

}  // namespace qcd
