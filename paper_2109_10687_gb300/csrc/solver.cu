// BiCGStab (Algorithm 5) on A M_SAP, the float64 defect-correction loop
// (Algorithm 4) and the fused BLAS-1 kernels they use (arXiv:2109.10687,
// Sec. 3).
//
// Reductions: every reducing kernel accumulates per thread in float32,
// combines warps and blocks in float64 and lets the last block to finish sum
// the per-block partials in a fixed order, so results do not depend on
// scheduling.  The scalars of the iteration (rho_0, alpha, omega, beta,
// |r|^2) live in device memory, one record per right-hand side, and are
// computed by the last block of the reduction that produces them; the host
// only reads the per-rhs "done" flags to decide when to leave the loop.
//
// Solution accumulation: Algorithm 5 iterates y and finishes with
// x = M_SAP y.  Here every A M_SAP p also yields z = M_SAP p, and the solution
// is accumulated as x += alpha z_p + omega z_r, which equals M_SAP y by the
// linearity of M_SAP and keeps the recursive residual tied to the true one
// when the preconditioner runs in reduced precision.

#include <algorithm>
#include <chrono>
#include <complex>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "blas.cuh"

namespace qcd {


struct Workspace {
  int nrhs = 0;
  size_t v4 = 0;  // float4 per rhs
  float4 *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *t = nullptr, *zp = nullptr, *zr = nullptr,
         *rt = nullptr, *tmp32 = nullptr;
  void *sap_s = nullptr, *sap_x16 = nullptr, *sap_b16 = nullptr;
  double2 *x64 = nullptr, *r64 = nullptr, *b64 = nullptr, *t64 = nullptr;
  double* partials = nullptr;
  double* dres = nullptr;   // small device results: 4 doubles per rhs
  unsigned* counters = nullptr;
  Scal* scal = nullptr;
  Scal* h_scal = nullptr;  // pinned
  double* h_red = nullptr; // pinned
  int* ctrl = nullptr;     // device: [0] rhs still iterating, [1] iterations, [2] iteration limit
  int* h_ctrl = nullptr;   // pinned
  int nblocks = 0;
  // flexible GMRES: basis V (m + 1 vectors), preconditioned directions Z
  // (m vectors), float64 internal layout, and its Hessenberg column scratch
  double2* fg = nullptr;
  double* fg_h = nullptr;
  int fg_m = 0;
  // instantiated CUDA graphs of the inner loop, reused while the key matches
  struct Graphs {
    int nrhs = -1, n_sap = -1, n_jac = -1, sap_prec = -1, mode = -1;
    double kappa = 0.0;
    cudaGraphExec_t half1 = nullptr, half2 = nullptr, loop = nullptr;
    long long n1 = 0, n2 = 0, nloop = 0;  // kernels per replay
    void reset() {
      if (half1) cudaGraphExecDestroy(half1);
      if (half2) cudaGraphExecDestroy(half2);
      if (loop) cudaGraphExecDestroy(loop);
      half1 = half2 = loop = nullptr;
      nrhs = -1;
    }
  } graphs;
};

// drop the captured inner-loop graphs (their kernels depend on settings
// such as the SAP domains)
void workspace_reset_graphs(qcd_ctx* ctx) {
  if (ctx->ws) ctx->ws->graphs.reset();
}

void workspace_free(qcd_ctx* ctx) {
  Workspace* w = ctx->ws;
  if (!w) return;
  void* ptrs[] = {w->x, w->r, w->p, w->q, w->t, w->zp, w->zr, w->rt, w->tmp32, w->sap_s, w->sap_x16, w->sap_b16,
                  w->x64, w->r64, w->b64, w->t64, w->partials, w->dres, w->counters, w->scal};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (w->fg) cudaFree(w->fg);
  if (w->fg_h) cudaFree(w->fg_h);
  if (w->h_scal) cudaFreeHost(w->h_scal);
  if (w->h_red) cudaFreeHost(w->h_red);
  if (w->ctrl) cudaFree(w->ctrl);
  if (w->h_ctrl) cudaFreeHost(w->h_ctrl);
  w->graphs.reset();
  delete w;
  ctx->ws = nullptr;
}


// Allocate (or grow) the workspace for nrhs right-hand sides.  The reduction
// buffers are always present; the solver vectors only with `solver`.
static Workspace* workspace(qcd_ctx* ctx, int nrhs, bool solver) {
  Workspace* w = ctx->ws;
  const bool have_solver = w && w->x;
  if (w && w->nrhs >= nrhs && (have_solver || !solver)) return w;
  const int keep_nrhs = w ? std::max(w->nrhs, nrhs) : nrhs;
  const bool want_solver = solver || have_solver;
  workspace_free(ctx);
  w = new Workspace();
  ctx->ws = w;
  const Geom& g = ctx->geom;
  w->nrhs = keep_nrhs;
  w->v4 = (size_t)g.vol * 6;
  int dev = 0, sms = 0;
  QCD_CUDA_CHECK(cudaGetDevice(&dev));
  QCD_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  w->nblocks = std::max(1, std::min(4 * sms, (int)((w->v4 + RED_THREADS - 1) / RED_THREADS)));
  QCD_CUDA_CHECK(cudaMalloc(&w->partials, sizeof(double) * MAX_RED_OUT * w->nblocks * keep_nrhs));
  QCD_CUDA_CHECK(cudaMalloc(&w->dres, sizeof(double) * 4 * keep_nrhs));
  QCD_CUDA_CHECK(cudaMalloc(&w->counters, sizeof(unsigned) * keep_nrhs));
  QCD_CUDA_CHECK(cudaMemset(w->counters, 0, sizeof(unsigned) * keep_nrhs));
  QCD_CUDA_CHECK(cudaMalloc(&w->scal, sizeof(Scal) * keep_nrhs));
  QCD_CUDA_CHECK(cudaMemset(w->scal, 0, sizeof(Scal) * keep_nrhs));
  QCD_CUDA_CHECK(cudaMallocHost(&w->h_scal, sizeof(Scal) * keep_nrhs));
  QCD_CUDA_CHECK(cudaMallocHost(&w->h_red, sizeof(double) * MAX_RED_OUT * keep_nrhs));
  QCD_CUDA_CHECK(cudaMalloc(&w->ctrl, sizeof(int) * 4));
  QCD_CUDA_CHECK(cudaMemset(w->ctrl, 0, sizeof(int) * 4));
  QCD_CUDA_CHECK(cudaMallocHost(&w->h_ctrl, sizeof(int) * 4));
  if (want_solver) {
    const size_t b32 = w->v4 * sizeof(float4) * keep_nrhs;
    float4** vecs[] = {&w->x, &w->r, &w->p, &w->q, &w->t, &w->zp, &w->zr, &w->rt, &w->tmp32};
    for (auto v : vecs) QCD_CUDA_CHECK(cudaMalloc(v, b32));
    const size_t b64 = (size_t)g.vol * 12 * sizeof(double2) * keep_nrhs;
    double2** v64[] = {&w->x64, &w->r64, &w->b64, &w->t64};
    for (auto v : v64) QCD_CUDA_CHECK(cudaMalloc(v, b64));
    QCD_CUDA_CHECK(cudaMalloc(&w->sap_s, spinor_bytes(g, QCD_PREC_SINGLE) * keep_nrhs));
    // float16 x of the generic SAP kernel, or the shared-memory kernel's halo (96 B per site)
    QCD_CUDA_CHECK(cudaMalloc(&w->sap_x16, spinor_bytes(g, QCD_PREC_SINGLE) * keep_nrhs));
    QCD_CUDA_CHECK(cudaMalloc(&w->sap_b16, spinor_bytes(g, QCD_PREC_HALF) * keep_nrhs));
  }
  return w;
}

#define RHS_SETUP                                                     \
  const int rhs = blockIdx.y;                                         \
  Scal& sc = scal[rhs];                                               \
  const size_t off = seg.at(rhs);                                     \
  const size_t n4 = seg.size(rhs);                                    \
  double* part = partials + (size_t)rhs * MAX_RED_OUT * gridDim.x;    \
  unsigned* cnt = counters + rhs;

// |a|^2 -> out[rhs]
__global__ void k_norm2(const float4* __restrict__ a, size_t n4, double* out, double* partials, unsigned* counters) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n4;
  double* part = partials + (size_t)rhs * MAX_RED_OUT * gridDim.x;
  unsigned* cnt = counters + rhs;
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    s += norm4(a[off + i]);
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, part, cnt, tot) && threadIdx.x == 0) out[rhs] = tot[0];
}

// <a|b> -> out[2 rhs], out[2 rhs + 1]
__global__ void k_cdot(const float4* __restrict__ a, const float4* __restrict__ b, size_t n, double* out,
                       double* partials, unsigned* counters, Scal* scal) {
  const Seg seg{n, nullptr, nullptr};
  RHS_SETUP
  (void)sc;
  float re = 0.f, im = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    cdot_acc(a[off + i], b[off + i], re, im);
  double v[2] = {re, im}, tot[2];
  if (grid_reduce<2>(v, part, cnt, tot) && threadIdx.x == 0) {
    out[2 * rhs] = tot[0];
    out[2 * rhs + 1] = tot[1];
  }
}

// BiCGStab initialisation: x = 0, r = p = rt = b, bnorm2 = |b|^2, rho_0 = bnorm2
__global__ void k_init(const float4* __restrict__ b, float4* x, float4* r, float4* p, float4* rt, Seg seg,
                       double tol2, Scal* scal, double* partials, unsigned* counters, int* ctrl) {
  RHS_SETUP
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = b[off + i];
    x[off + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    r[off + i] = v;
    p[off + i] = v;
    rt[off + i] = v;
    s += norm4(v);
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, part, cnt, tot) && threadIdx.x == 0) {
    sc.bnorm2 = tot[0];
    sc.rnorm2 = tot[0];
    sc.rho0_re = tot[0];
    sc.rho0_im = 0.0;
    sc.tol2 = tol2;
    sc.iters = 0;
    sc.xpend = 0;
    sc.status = QCD_OK;
    sc.conv = tot[0] == 0.0;
    sc.done = tot[0] == 0.0;
    if (!isfinite(tot[0])) {
      sc.status = QCD_ERR_NONFINITE;
      sc.done = 1;
    }
    if (!sc.done) atomicAdd(ctrl, 1);  // one more right-hand side iterating
  }
}

// alpha = rho_0 / <rt|q>
__global__ void k_alpha(const float4* __restrict__ rt, const float4* __restrict__ q, Seg seg, Scal* scal,
                        double* partials, unsigned* counters, int* ctrl) {
  RHS_SETUP
  if (sc.done) return;
  float re = 0.f, im = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    cdot_acc(rt[off + i], q[off + i], re, im);
  double v[2] = {re, im}, tot[2];
  if (grid_reduce<2>(v, part, cnt, tot) && threadIdx.x == 0) {
    ++sc.iters;
    const double dn = tot[0] * tot[0] + tot[1] * tot[1];
    if (!(dn > 0.0) || !isfinite(dn)) {
      sc.status = isfinite(dn) ? QCD_ERR_BREAKDOWN : QCD_ERR_NONFINITE;
      sc.done = 1;
      atomicSub(ctrl, 1);
    } else {
      sc.alpha_re = (sc.rho0_re * tot[0] + sc.rho0_im * tot[1]) / dn;
      sc.alpha_im = (sc.rho0_im * tot[0] - sc.rho0_re * tot[1]) / dn;
    }
  }
}

// r -= alpha q; rnorm2 = |r|^2; first exit test.  The solution's share
// x += alpha z_p is left pending and applied with the second one in
// k_update2 (one pass over x instead of two), or by k_xfinal when the
// iteration stops here.
__global__ void k_update1(float4* x, float4* r, const float4* __restrict__ z, const float4* __restrict__ q, Seg seg,
                          Scal* scal, double* partials, unsigned* counters, int* ctrl) {
  RHS_SETUP
  if (sc.done) return;
  (void)x;
  (void)z;
  const float ar = (float)sc.alpha_re, ai = (float)sc.alpha_im;
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 rv = caxpy4(-ar, -ai, q[off + i], r[off + i]);
    r[off + i] = rv;
    s += norm4(rv);
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, part, cnt, tot) && threadIdx.x == 0) {
    sc.xpend = 1;
    sc.rnorm2 = tot[0];
    if (!isfinite(tot[0])) {
      sc.status = QCD_ERR_NONFINITE;
      sc.done = 1;
      atomicSub(ctrl, 1);
    } else if (tot[0] < sc.tol2 * sc.bnorm2) {
      sc.conv = 1;
      sc.done = 1;
      atomicSub(ctrl, 1);
    }
  }
}

// omega = <t|r> / |t|^2
__global__ void k_omega(const float4* __restrict__ t, const float4* __restrict__ r, Seg seg, Scal* scal,
                        double* partials, unsigned* counters, int* ctrl) {
  RHS_SETUP
  if (sc.done) return;
  float re = 0.f, im = 0.f, tt = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 tv = t[off + i];
    cdot_acc(tv, r[off + i], re, im);
    tt += norm4(tv);
  }
  double v[3] = {re, im, tt}, tot[3];
  if (grid_reduce<3>(v, part, cnt, tot) && threadIdx.x == 0) {
    if (!(tot[2] > 0.0) || !isfinite(tot[2])) {
      sc.status = isfinite(tot[2]) ? QCD_ERR_BREAKDOWN : QCD_ERR_NONFINITE;
      sc.done = 1;
      atomicSub(ctrl, 1);
    } else {
      sc.omega_re = tot[0] / tot[2];
      sc.omega_im = tot[1] / tot[2];
    }
  }
}

// x += alpha z_p + omega z_r (z_p: zp, z_r: z); r -= omega t;
// rnorm2 = |r|^2, rho = <rt|r>; second exit test;
// beta = alpha rho / (rho_0 omega); rho_0 = rho.  A right-hand side that
// stopped after k_update1 (converged or broken down since) gets only its
// pending x += alpha z_p.
__global__ void k_update2(float4* x, float4* r, const float4* __restrict__ zp, const float4* __restrict__ z,
                          const float4* __restrict__ t, const float4* __restrict__ rt, Seg seg, Scal* scal,
                          double* partials, unsigned* counters, int* ctrl) {
  RHS_SETUP
  const float ar = (float)sc.alpha_re, ai = (float)sc.alpha_im;
  if (sc.done) {
    if (!sc.xpend) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
      x[off + i] = caxpy4(ar, ai, zp[off + i], x[off + i]);
    return;
  }
  const float wr = (float)sc.omega_re, wi = (float)sc.omega_im;
  float s = 0.f, re = 0.f, im = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    x[off + i] = caxpy4(wr, wi, z[off + i], caxpy4(ar, ai, zp[off + i], x[off + i]));
    const float4 rv = caxpy4(-wr, -wi, t[off + i], r[off + i]);
    r[off + i] = rv;
    s += norm4(rv);
    cdot_acc(rt[off + i], rv, re, im);
  }
  double v[3] = {s, re, im}, tot[3];
  if (grid_reduce<3>(v, part, cnt, tot) && threadIdx.x == 0) {
    sc.rnorm2 = tot[0];
    if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
      sc.status = QCD_ERR_NONFINITE;
      sc.done = 1;
      atomicSub(ctrl, 1);
    } else if (tot[0] < sc.tol2 * sc.bnorm2) {
      sc.conv = 1;
      sc.done = 1;
      atomicSub(ctrl, 1);
    } else {
      // beta = (alpha rho) / (rho_0 omega)
      const double nr = sc.alpha_re * tot[1] - sc.alpha_im * tot[2];
      const double ni = sc.alpha_re * tot[2] + sc.alpha_im * tot[1];
      const double dr = sc.rho0_re * sc.omega_re - sc.rho0_im * sc.omega_im;
      const double di = sc.rho0_re * sc.omega_im + sc.rho0_im * sc.omega_re;
      const double dn = dr * dr + di * di;
      if (!(dn > 0.0) || (tot[1] == 0.0 && tot[2] == 0.0)) {
        sc.status = QCD_ERR_BREAKDOWN;
        sc.done = 1;
      atomicSub(ctrl, 1);
      } else {
        sc.beta_re = (nr * dr + ni * di) / dn;
        sc.beta_im = (ni * dr - nr * di) / dn;
        sc.rho0_re = tot[1];
        sc.rho0_im = tot[2];
      }
    }
  }
}

// p = r + beta (p - omega q); the pending x update has been applied by k_update2
__global__ void k_update_p(float4* p, const float4* __restrict__ r, const float4* __restrict__ q, Seg seg,
                           Scal* scal) {
  const int rhs = blockIdx.y;
  Scal& sc = scal[rhs];
  if (blockIdx.x == 0 && threadIdx.x == 0) sc.xpend = 0;  // no block of this kernel reads it
  if (sc.done) return;
  const size_t off = seg.at(rhs);
  const size_t n4 = seg.size(rhs);
  const float br = (float)sc.beta_re, bi = (float)sc.beta_im;
  const float wr = (float)sc.omega_re, wi = (float)sc.omega_im;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 tmp = caxpy4(-wr, -wi, q[off + i], p[off + i]);
    p[off + i] = caxpy4(br, bi, tmp, r[off + i]);
  }
}

// x += alpha z_p for a right-hand side whose iteration stopped after
// k_update1 (the loop left before k_update2); no-op otherwise
__global__ void k_xfinal(float4* x, const float4* __restrict__ z, Seg seg, const Scal* scal) {
  const int rhs = blockIdx.y;
  const Scal& sc = scal[rhs];
  if (!sc.xpend) return;
  const size_t off = seg.at(rhs);
  const size_t n4 = seg.size(rhs);
  const float ar = (float)sc.alpha_re, ai = (float)sc.alpha_im;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    x[off + i] = caxpy4(ar, ai, z[off + i], x[off + i]);
}

// ---------------------------------------------------------------------------
// float64 helpers for Algorithm 4 (two doubles per complex, 12 complex/site)
// ---------------------------------------------------------------------------
// out[rhs] = |a|^2 (float64 accumulation throughout)
__global__ void k_norm2_f64(const double2* __restrict__ a, size_t n2, double* out, double* partials,
                            unsigned* counters) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n2;
  double* part = partials + (size_t)rhs * MAX_RED_OUT * gridDim.x;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = a[off + i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, part, counters + rhs, tot) && threadIdx.x == 0) out[rhs] = tot[0];
}

// r = b - r (r holds D x on entry); out[rhs] = |r|^2
__global__ void k_residual_f64(const double2* __restrict__ b, double2* r, size_t n2, double* out, double* partials,
                               unsigned* counters) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n2;
  double* part = partials + (size_t)rhs * MAX_RED_OUT * gridDim.x;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = b[off + i], dv = r[off + i];
    const double2 v = make_double2(bv.x - dv.x, bv.y - dv.y);
    r[off + i] = v;
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, part, counters + rhs, tot) && threadIdx.x == 0) out[rhs] = tot[0];
}

// ---------------------------------------------------------------------------
// float64 vector kernels of the flexible GMRES outer solver (one right-hand
// side; a vector is n2 complex numbers in the internal float64 layout, whose
// inner product does not depend on the site order)
// ---------------------------------------------------------------------------
// <a|b> = sum conj(a) b -> out[0] (re), out[1] (im)
__global__ void k_cdot_f64(const double2* __restrict__ a, const double2* __restrict__ b, size_t n2, double* out,
                           double* partials, unsigned* counters) {
  double re = 0.0, im = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 u = a[i], v = b[i];
    re = fma(u.x, v.x, fma(u.y, v.y, re));
    im = fma(u.x, v.y, fma(-u.y, v.x, im));
  }
  double v[2] = {re, im}, tot[2];
  if (grid_reduce<2>(v, partials, counters, tot) && threadIdx.x == 0) {
    out[0] = tot[0];
    out[1] = tot[1];
  }
}

// y -= s x with the complex s = (s[0], s[1]) read from device memory
__global__ void k_caxmy_f64(double2* y, const double2* __restrict__ x, size_t n2, const double* s) {
  const double sr = s[0], si = s[1];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 u = x[i];
    double2 v = y[i];
    v.x -= sr * u.x - si * u.y;
    v.y -= sr * u.y + si * u.x;
    y[i] = v;
  }
}

// y += (sr + i si) x, scalar from the host
__global__ void k_caxpy_f64(double2* y, const double2* __restrict__ x, size_t n2, double sr, double si) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 u = x[i];
    double2 v = y[i];
    v.x += sr * u.x - si * u.y;
    v.y += sr * u.y + si * u.x;
    y[i] = v;
  }
}

// v *= f with f = 1 / sqrt(n2[0]) read from device memory (v / |v|); no-op for a zero norm
__global__ void k_normalize_f64(double2* v, size_t n2, const double* norm2) {
  const double q = norm2[0];
  if (!(q > 0.0)) return;
  const double f = 1.0 / sqrt(q);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 u = v[i];
    v[i] = make_double2(u.x * f, u.y * f);
  }
}

// v = f w (real f from the host)
__global__ void k_scale_f64(double2* v, const double2* __restrict__ w, size_t n2, double f) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 u = w[i];
    v[i] = make_double2(u.x * f, u.y * f);
  }
}

// float32 p = R_SP(r / err): same internal site order, float64 complex ->
// float32 pairs (the float64 and float32 layouts order components alike
// within a domain: float4 group k holds complex components 2k, 2k+1)
__global__ void k_f64_to_f32_scaled(Geom g, const double2* __restrict__ r, float4* p, const double* scale) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int rhs = blockIdx.y;
  const int dom = (int)(gid >> g.logvd) + rhs * g.ndom, s = (int)(gid & (g.vd - 1));
  const double f = scale[rhs];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 a = r[((size_t)(dom * 12 + 2 * k) << g.logvd) + s];
    const double2 b = r[((size_t)(dom * 12 + 2 * k + 1) << g.logvd) + s];
    p[((size_t)(dom * 6 + k) << g.logvd) + s] = make_float4((float)(a.x * f), (float)(a.y * f), (float)(b.x * f),
                                                            (float)(b.y * f));
  }
}

// x64 += err * P_DP(q32)
__global__ void k_f64_axpy_f32(Geom g, double2* x, const float4* __restrict__ q, const double* scale) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int rhs = blockIdx.y;
  const int dom = (int)(gid >> g.logvd) + rhs * g.ndom, s = (int)(gid & (g.vd - 1));
  const double f = scale[rhs];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = q[((size_t)(dom * 6 + k) << g.logvd) + s];
    double2& a = x[((size_t)(dom * 12 + 2 * k) << g.logvd) + s];
    double2& b = x[((size_t)(dom * 12 + 2 * k + 1) << g.logvd) + s];
    a.x = fma(f, (double)v.x, a.x);
    a.y = fma(f, (double)v.y, a.y);
    b.x = fma(f, (double)v.z, b.x);
    b.y = fma(f, (double)v.w, b.y);
  }
}

// ---------------------------------------------------------------------------
// double-float versions of the Algorithm-4 vector kernels (float4 per
// complex: re.hi, re.lo, im.hi, im.lo; same element order as float64)
// ---------------------------------------------------------------------------
// A double-float number has the exponent range of float32, so b, x and r
// are held scaled by a power of two 2^k (exact), with k chosen from |b|^2
// (b2, computed in float64) so that b's components are of order one; the
// residual norms are reported unscaled.  D is linear, so the scaled system
// has the same solution, scaled.
__device__ __forceinline__ int df_scale_exp(const double* b2, int rhs, size_t n2) { return df_scale_exp(b2[rhs], n2); }
// float64 -> scaled double-float, one right-hand side per grid row; in
// place allowed (the conversions are integer operations on the bits)
__global__ void k_df_from_f64(const double2* in, float4* out, size_t n2, const double* b2) {
  const int rhs = blockIdx.y;
  const int k = df_scale_exp(b2, rhs, n2);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[rhs * n2 + i];
    const df64 re = df64_from_double_scaled(v.x, k), im = df64_from_double_scaled(v.y, k);
    out[rhs * n2 + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}
// scaled double-float -> float64, in place allowed
__global__ void k_f64_from_df(const float4* in, double2* out, size_t n2, const double* b2) {
  const int rhs = blockIdx.y;
  const int k = df_scale_exp(b2, rhs, n2);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = in[rhs * n2 + i];
    out[rhs * n2 + i] =
        make_double2(df64_to_double_scaled(df64(v.x, v.y), k), df64_to_double_scaled(df64(v.z, v.w), k));
  }
}
// r = b - r (r holds D x on entry), in double-float; out[rhs] = |r|^2,
// unscaled.  The arithmetic stays on the float32 pipes (the float64 pipe of
// this GPU is a small fraction of their width): squares of each component's
// high part (the scaled components are of order one, their squares well
// inside the float32 range), float32 sums over each thread's elements
// (relative error about 1e-6, far below what the stopping test at 1e-10
// and the reported residual need), float64 across threads.
__global__ void k_residual_df(const float4* __restrict__ b, float4* r, size_t n2, const double* b2, double* out,
                              double* partials, unsigned* counters) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n2;
  double* part = partials + (size_t)rhs * MAX_RED_OUT * gridDim.x;
  const int k = df_scale_exp(b2, rhs, n2);
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const float4 bv = b[off + i], dv = r[off + i];
    const df64 re = df64(bv.x, bv.y) - df64(dv.x, dv.y);
    const df64 im = df64(bv.z, bv.w) - df64(dv.z, dv.w);
    r[off + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    s = fmaf(re.hi, re.hi, fmaf(im.hi, im.hi, s));
  }
  double v[1] = {ldexp((double)s, -2 * k)}, tot[1];
  if (grid_reduce<1>(v, part, counters + rhs, tot) && threadIdx.x == 0) out[rhs] = tot[0];
}
// float32 p = R_SP(r / err) from the scaled double-float r (err unscaled),
// in float32 arithmetic: (hi + lo) f as hi f + lo f with one rounding
__global__ void k_df_to_f32_scaled(Geom g, const float4* __restrict__ r, float4* p, const double* scale,
                                   const double* b2) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int rhs = blockIdx.y;
  const int dom = (int)(gid >> g.logvd) + rhs * g.ndom, s = (int)(gid & (g.vd - 1));
  const float f = (float)ldexp(scale[rhs], -df_scale_exp(b2, rhs, (size_t)g.vol * 12));
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 a = r[((size_t)(dom * 12 + 2 * k) << g.logvd) + s];
    const float4 b = r[((size_t)(dom * 12 + 2 * k + 1) << g.logvd) + s];
    p[((size_t)(dom * 6 + k) << g.logvd) + s] = make_float4(fmaf(a.x, f, a.y * f), fmaf(a.z, f, a.w * f),
                                                            fmaf(b.x, f, b.y * f), fmaf(b.z, f, b.w * f));
  }
}
// scaled double-float x += err * P_DP(q32) (err unscaled)
__global__ void k_df_axpy_f32(Geom g, float4* x, const float4* __restrict__ q, const double* scale,
                              const double* b2) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int rhs = blockIdx.y;
  const int dom = (int)(gid >> g.logvd) + rhs * g.ndom, s = (int)(gid & (g.vd - 1));
  const df64 f(ldexp(scale[rhs], df_scale_exp(b2, rhs, (size_t)g.vol * 12)));
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = q[((size_t)(dom * 6 + k) << g.logvd) + s];
    float4& a = x[((size_t)(dom * 12 + 2 * k) << g.logvd) + s];
    float4& b = x[((size_t)(dom * 12 + 2 * k + 1) << g.logvd) + s];
    const df64 ar = fma(f, df64(v.x), df64(a.x, a.y)), ai = fma(f, df64(v.y), df64(a.z, a.w));
    const df64 br = fma(f, df64(v.z), df64(b.x, b.y)), bi = fma(f, df64(v.w), df64(b.z, b.w));
    a = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
    b = make_float4(br.hi, br.lo, bi.hi, bi.lo);
  }
}

// Condition of the device-side inner loop: one more iteration while some
// right-hand side iterates and the limit is not reached.
__global__ void k_loop_cond(cudaGraphConditionalHandle handle, int* ctrl) {
  const int it = ++ctrl[1];
  cudaGraphSetConditional(handle, (ctrl[0] > 0 && it < ctrl[2]) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
struct Launcher {
  qcd_ctx* ctx;
  Workspace* w;
  cudaStream_t st;
  int nrhs;
  dim3 grid() const { return dim3(w->nblocks, nrhs); }
};

static void am_sap(qcd_ctx* ctx, Workspace* w, float4* z, float4* out, const float4* in, int nrhs, int n_sap, int n_jac,
                   int sap_prec, cudaStream_t st) {
  sap_apply_launch(ctx, z, in, nrhs, n_sap, n_jac, sap_prec, w->sap_s, w->sap_x16, w->sap_b16, st);
  dslash_launch(ctx, out, z, QCD_PREC_SINGLE, MODE_A, nrhs, st);
}

static bool all_done(Workspace* w, int nrhs, cudaStream_t st) {
  QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r)
    if (!w->h_scal[r].done) return false;
  return true;
}

// One iteration of Algorithm 5 (both half-steps); usable for graph capture.
static void bicg_half1(qcd_ctx* ctx, Workspace* w, int nrhs, const qcd_solve_params& P, cudaStream_t st) {
  const dim3 grid(w->nblocks, nrhs);
  am_sap(ctx, w, w->zp, w->q, w->p, nrhs, P.n_sap, P.n_jac, P.sap_prec, st);
  LaunchScope ls(ctx, QCD_KC_BLAS, st);
  k_alpha<<<grid, RED_THREADS, 0, st>>>(w->rt, w->q, Seg{w->v4}, w->scal, w->partials, w->counters, w->ctrl);
  k_update1<<<grid, RED_THREADS, 0, st>>>(w->x, w->r, w->zp, w->q, Seg{w->v4}, w->scal, w->partials, w->counters,
                                         w->ctrl);
  ctx->launches++;
  check_launch();
}
static void bicg_half2(qcd_ctx* ctx, Workspace* w, int nrhs, const qcd_solve_params& P, cudaStream_t st) {
  const dim3 grid(w->nblocks, nrhs);
  am_sap(ctx, w, w->zr, w->t, w->r, nrhs, P.n_sap, P.n_jac, P.sap_prec, st);
  LaunchScope ls(ctx, QCD_KC_BLAS, st);
  k_omega<<<grid, RED_THREADS, 0, st>>>(w->t, w->r, Seg{w->v4}, w->scal, w->partials, w->counters, w->ctrl);
  k_update2<<<grid, RED_THREADS, 0, st>>>(w->x, w->r, w->zp, w->zr, w->t, w->rt, Seg{w->v4}, w->scal, w->partials,
                                         w->counters,
                                         w->ctrl);
  k_update_p<<<grid, RED_THREADS, 0, st>>>(w->p, w->r, w->q, Seg{w->v4}, w->scal);
  ctx->launches += 2;
  check_launch();
}

// Algorithm 5 on A M_SAP z = b32 (float32 internal fields, nrhs stacked);
// solution accumulated in w->x.  Returns iterations; fills per-rhs status.
//   use_graph 0: kernels launched one by one, the host reads the exit flags
//                after each half-iteration;
//   use_graph 1: each half-iteration replayed as a CUDA graph, same host checks;
//   use_graph 2: the whole loop is one CUDA graph with a conditional WHILE
//                node: a one-thread kernel sets the condition from the count
//                of right-hand sides still iterating, and every operator
//                kernel of an iteration returns at once when that count is
//                zero, so the host waits only for the finished loop.
// Graphs are cached in the workspace and reused while nrhs, n_sap, n_jac,
// sap_prec and kappa are unchanged.
static int bicgstab_sap(qcd_ctx* ctx, Workspace* w, const float4* b32, int nrhs, const qcd_solve_params& P,
                        cudaStream_t st, int* worst_status) {
  const dim3 grid(w->nblocks, nrhs);
  w->h_ctrl[0] = 0;
  w->h_ctrl[1] = 0;
  w->h_ctrl[2] = P.max_inner;
  QCD_CUDA_CHECK(cudaMemcpyAsync(w->ctrl, w->h_ctrl, sizeof(int) * 3, cudaMemcpyHostToDevice, st));
  {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    k_init<<<grid, RED_THREADS, 0, st>>>(b32, w->x, w->r, w->p, w->rt, Seg{w->v4}, P.inner_tol * P.inner_tol, w->scal,
                                         w->partials, w->counters, w->ctrl);
    check_launch();
  }
  const int mode = P.use_graph < 0 ? 0 : (P.use_graph > 2 ? 2 : P.use_graph);
  Workspace::Graphs& G = w->graphs;
  if (mode > 0 && (G.nrhs != nrhs || G.n_sap != P.n_sap || G.n_jac != P.n_jac || G.sap_prec != P.sap_prec ||
                   G.mode != mode || G.kappa != ctx->kappa)) {
    G.reset();
    // the autotuner cannot time launch shapes inside a capture: run the
    // operator and SAP kernels of the loop once beforehand (into scratch
    // buffers the loop overwrites before reading; p holds the source here)
    dslash_launch(ctx, w->t, w->zp, QCD_PREC_SINGLE, MODE_A, nrhs, st);
    sap_apply_launch(ctx, w->zr, w->p, nrhs, P.n_sap, P.n_jac, P.sap_prec, w->sap_s, w->sap_x16, w->sap_b16, st);
    cudaGraph_t gr;
    const long long c_start = ctx->launches;
    long long c0 = c_start;
    if (mode == 1) {
      QCD_CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      bicg_half1(ctx, w, nrhs, P, st);
      QCD_CUDA_CHECK(cudaStreamEndCapture(st, &gr));
      QCD_CUDA_CHECK(cudaGraphInstantiate(&G.half1, gr, 0));
      cudaGraphDestroy(gr);
      G.n1 = ctx->launches - c0;
      c0 = ctx->launches;
      QCD_CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      bicg_half2(ctx, w, nrhs, P, st);
      QCD_CUDA_CHECK(cudaStreamEndCapture(st, &gr));
      QCD_CUDA_CHECK(cudaGraphInstantiate(&G.half2, gr, 0));
      cudaGraphDestroy(gr);
      G.n2 = ctx->launches - c0;
    } else {
      QCD_CUDA_CHECK(cudaGraphCreate(&gr, 0));
      cudaGraphConditionalHandle handle;
      QCD_CUDA_CHECK(cudaGraphConditionalHandleCreate(&handle, gr, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      QCD_CUDA_CHECK(cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      // operator kernels of the body return at once when no rhs iterates
      ctx->geom.run_flag = w->ctrl;
      QCD_CUDA_CHECK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      bicg_half1(ctx, w, nrhs, P, st);
      bicg_half2(ctx, w, nrhs, P, st);
      k_loop_cond<<<1, 1, 0, st>>>(handle, w->ctrl);
      ctx->launches++;
      const cudaError_t ce = cudaStreamEndCapture(st, &body);
      ctx->geom.run_flag = nullptr;
      QCD_CUDA_CHECK(ce);
      QCD_CUDA_CHECK(cudaGraphInstantiate(&G.loop, gr, 0));
      cudaGraphDestroy(gr);
      G.nloop = ctx->launches - c0;
    }
    ctx->launches = c_start;  // captured kernels are counted when replayed
    G.nrhs = nrhs;
    G.n_sap = P.n_sap;
    G.n_jac = P.n_jac;
    G.sap_prec = P.sap_prec;
    G.mode = mode;
    G.kappa = ctx->kappa;
  }
  int it = 0;
  // x += alpha z_p of a right-hand side whose iteration stopped after the
  // first half (k_update1); the loop leaves that share to k_update2
  auto xfinal = [&]() {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    k_xfinal<<<grid, RED_THREADS, 0, st>>>(w->x, w->zp, Seg{w->v4}, w->scal);
    check_launch();
  };
  if (mode == 2) {
    QCD_CUDA_CHECK(cudaGraphLaunch(G.loop, st));
    xfinal();
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_ctrl, w->ctrl, sizeof(int) * 3, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    it = w->h_ctrl[1];
    ctx->launches += (long long)it * G.nloop;
  } else {
    bool finished = all_done(w, nrhs, st);
    while (!finished && it < P.max_inner) {
      ++it;
      if (mode == 1) {
        QCD_CUDA_CHECK(cudaGraphLaunch(G.half1, st));
        ctx->launches += G.n1;
      } else {
        bicg_half1(ctx, w, nrhs, P, st);
      }
      if (all_done(w, nrhs, st)) break;
      if (mode == 1) {
        QCD_CUDA_CHECK(cudaGraphLaunch(G.half2, st));
        ctx->launches += G.n2;
      } else {
        bicg_half2(ctx, w, nrhs, P, st);
      }
      finished = all_done(w, nrhs, st);
    }
    xfinal();
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  }
  int worst = QCD_OK;
  for (int r = 0; r < nrhs; ++r) {
    const Scal& sc = w->h_scal[r];
    if (sc.status != QCD_OK) worst = sc.status;
    else if (!sc.conv && worst == QCD_OK) worst = QCD_ERR_NOT_CONVERGED;
  }
  *worst_status = worst;
  return it;
}

// ---------------------------------------------------------------------------
// |a|^2 without any allocation (qcd_norm2_noalloc)
// ---------------------------------------------------------------------------
// Scratch of the reduction (per-block partial sums, completion counters and
// the results) in a file-scope device array instead of the context's
// workspace.  Every GPU that loads the library holds it (about 514 KB) until
// the process exits; all calls share it.
constexpr int NOALLOC_MAX_RHS = 16;
constexpr int NOALLOC_MAX_BLOCKS = 1024;
struct NoAllocScratch {
  double partials[MAX_RED_OUT * NOALLOC_MAX_BLOCKS * NOALLOC_MAX_RHS];
  double result[NOALLOC_MAX_RHS];
  unsigned counters[NOALLOC_MAX_RHS];
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol itself is only a host-side stand-in, never a device address; the
// address is looked up once per device with that device current.
static NoAllocScratch* noalloc_scratch_address() {
  static std::mutex mu;
  static NoAllocScratch* addr[256] = {nullptr};
  int dev = 0;
  QCD_CUDA_CHECK(cudaGetDevice(&dev));
  QCD_REQUIRE(dev >= 0 && dev < 256, QCD_ERR_ARG, "qcd_norm2_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      throw Error{QCD_ERR_CUDA, std::string("qcd_norm2_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    addr[dev] = static_cast<NoAllocScratch*>(p);
  }
  return addr[dev];
}

}  // namespace qcd

using namespace qcd;

#define API_BEGIN try {
#define API_END(ctx)                          \
  }                                           \
  catch (const qcd::Error& e) {               \
    (ctx)->err = e.msg;                       \
    return e.code;                            \
  }                                           \
  catch (...) {                               \
    (ctx)->err = "unknown error";             \
    return QCD_ERR_CUDA;                      \
  }                                           \
  return QCD_OK;

static void require_operator(qcd_ctx* ctx) {
  QCD_REQUIRE(ctx->have_gauge, QCD_ERR_STATE, "no gauge field set");
  QCD_REQUIRE(ctx->have_clover, QCD_ERR_STATE, "clover term not built (qcd_build_clover)");
}

extern "C" int qcd_solve_params_default(qcd_solve_params* p) {
  if (!p) return QCD_ERR_ARG;
  p->tol = 1e-10;
  p->inner_tol = 1e-6;
  p->max_outer = 20;
  p->max_inner = 500;
  p->n_sap = 4;
  p->n_jac = 4;
  p->sap_prec = QCD_PREC_SINGLE;
  p->use_graph = 0;
  p->x_is_guess = 0;
  p->residual_prec = 0;
  p->outer_restart = 0;
  return QCD_OK;
}

extern "C" int qcd_sap_apply_nrhs(qcd_ctx* ctx, void* out, const void* in, int nrhs, int n_sap, int n_jac,
                                  int sap_prec, int with_A, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  require_operator(ctx);
  QCD_REQUIRE(out && in && out != in, QCD_ERR_ARG, "qcd_sap_apply: bad buffers");
  QCD_REQUIRE(nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_sap_apply: 1 <= nrhs <= 65535");
  QCD_REQUIRE(n_sap >= 0 && n_jac >= 1, QCD_ERR_ARG, "qcd_sap_apply: n_sap >= 0 and n_jac >= 1");
  QCD_REQUIRE(sap_prec == QCD_PREC_SINGLE || sap_prec == QCD_PREC_HALF || sap_prec == QCD_PREC_HALF_GAUGE,
              QCD_ERR_ARG, "qcd_sap_apply: sap_prec must be SINGLE, HALF or HALF_GAUGE");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace* w = workspace(ctx, nrhs, true);
  if (with_A) {
    am_sap(ctx, w, w->tmp32, (float4*)out, (const float4*)in, nrhs, n_sap, n_jac, sap_prec, st);
  } else {
    sap_apply_launch(ctx, (float4*)out, (const float4*)in, nrhs, n_sap, n_jac, sap_prec, w->sap_s, w->sap_x16,
                     w->sap_b16, st);
  }
  API_END(ctx)
}

extern "C" int qcd_sap_apply(qcd_ctx* ctx, void* out, const void* in, int n_sap, int n_jac, int sap_prec, int with_A,
                             void* stream) {
  return qcd_sap_apply_nrhs(ctx, out, in, 1, n_sap, n_jac, sap_prec, with_A, stream);
}

extern "C" int qcd_norm2(qcd_ctx* ctx, double* result, const void* a, int prec, int nrhs, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  QCD_REQUIRE(result && a && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_norm2: bad arguments");
  QCD_REQUIRE(prec == QCD_PREC_SINGLE || prec == QCD_PREC_DOUBLE, QCD_ERR_ARG, "qcd_norm2: SINGLE or DOUBLE");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace* w = workspace(ctx, nrhs, false);
  double* res = w->dres;
  {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    if (prec == QCD_PREC_SINGLE)
      k_norm2<<<dim3(w->nblocks, nrhs), RED_THREADS, 0, st>>>((const float4*)a, w->v4, res, w->partials,
                                                             w->counters);
    else
      k_norm2_f64<<<dim3(w->nblocks, nrhs), RED_THREADS, 0, st>>>((const double2*)a, (size_t)ctx->geom.vol * 12, res,
                                                                 w->partials, w->counters);
    check_launch();
  }
  QCD_CUDA_CHECK(cudaMemcpyAsync(result, res, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  API_END(ctx)
}

// Same result as qcd_norm2, computed with the library's static scratch so that
// the call allocates nothing (no cudaMalloc, no workspace growth).  For
// callers that cannot allocate device memory at this point.
extern "C" int qcd_norm2_noalloc(qcd_ctx* ctx, double* result, const void* a, int prec, int nrhs, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  QCD_REQUIRE(result && a, QCD_ERR_ARG, "qcd_norm2_noalloc: null pointer");
  QCD_REQUIRE(nrhs >= 1 && nrhs <= NOALLOC_MAX_RHS, QCD_ERR_ARG,
              "qcd_norm2_noalloc: nrhs must be between 1 and 16 (size of the static scratch)");
  QCD_REQUIRE(prec == QCD_PREC_SINGLE || prec == QCD_PREC_DOUBLE, QCD_ERR_ARG,
              "qcd_norm2_noalloc: SINGLE or DOUBLE");
  cudaStream_t st = (cudaStream_t)stream;
  NoAllocScratch* scr = noalloc_scratch_address();
  int dev = 0, sms = 0;
  QCD_CUDA_CHECK(cudaGetDevice(&dev));
  QCD_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t v4 = (size_t)ctx->geom.vol * 6;
  const int nblocks = std::max(1, std::min({4 * sms, NOALLOC_MAX_BLOCKS, (int)((v4 + RED_THREADS - 1) / RED_THREADS)}));
  // the completion counters must start at zero; a previous call may have
  // been interrupted, so clear them every time
  QCD_CUDA_CHECK(cudaMemsetAsync(scr->counters, 0, sizeof(unsigned) * nrhs, st));
  {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    if (prec == QCD_PREC_SINGLE)
      k_norm2<<<dim3(nblocks, nrhs), RED_THREADS, 0, st>>>((const float4*)a, v4, scr->result, scr->partials,
                                                          scr->counters);
    else
      k_norm2_f64<<<dim3(nblocks, nrhs), RED_THREADS, 0, st>>>((const double2*)a, (size_t)ctx->geom.vol * 12,
                                                              scr->result, scr->partials, scr->counters);
    check_launch();
  }
  QCD_CUDA_CHECK(cudaMemcpyAsync(result, scr->result, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  API_END(ctx)
}

extern "C" int qcd_cdot(qcd_ctx* ctx, double result[2], const void* a, const void* b, int prec, int nrhs,
                        void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  QCD_REQUIRE(result && a && b && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_cdot: bad arguments");
  QCD_REQUIRE(prec == QCD_PREC_SINGLE, QCD_ERR_ARG, "qcd_cdot: SINGLE only");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace* w = workspace(ctx, nrhs, false);
  double* res = w->dres;
  {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    k_cdot<<<dim3(w->nblocks, nrhs), RED_THREADS, 0, st>>>((const float4*)a, (const float4*)b, w->v4, res, w->partials,
                                                          w->counters, w->scal);
    check_launch();
  }
  QCD_CUDA_CHECK(cudaMemcpyAsync(result, res, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  API_END(ctx)
}

extern "C" int qcd_solve(qcd_ctx* ctx, double* x, const double* b, int nrhs, int on_device,
                         const qcd_solve_params* params, qcd_solve_info* info, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  int result = QCD_OK;
  API_BEGIN
  require_operator(ctx);
  QCD_REQUIRE(x && b && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_solve: bad arguments");
  qcd_solve_params P;
  if (params) P = *params;
  else qcd_solve_params_default(&P);
  QCD_REQUIRE(P.tol > 0 && P.inner_tol > 0 && P.max_outer >= 1 && P.max_inner >= 1 && P.n_sap >= 0 && P.n_jac >= 1,
              QCD_ERR_ARG, "qcd_solve: bad parameters");
  QCD_REQUIRE(P.sap_prec == QCD_PREC_SINGLE || P.sap_prec == QCD_PREC_HALF || P.sap_prec == QCD_PREC_HALF_GAUGE,
              QCD_ERR_ARG, "qcd_solve: sap_prec must be SINGLE, HALF or HALF_GAUGE");
  QCD_REQUIRE(P.outer_restart >= 0 && P.outer_restart <= 64, QCD_ERR_ARG, "qcd_solve: outer_restart in [0, 64]");
  QCD_REQUIRE(P.residual_prec == 0 || P.residual_prec == 1, QCD_ERR_ARG, "qcd_solve: residual_prec must be 0 or 1");
  QCD_REQUIRE(P.outer_restart == 0 || nrhs == 1, QCD_ERR_ARG, "qcd_solve: flexible GMRES needs nrhs = 1");
  cudaStream_t st = (cudaStream_t)stream;
  if (P.use_graph) {
    // stream capture is not possible on the legacy default stream: run the
    // solve on a private stream, ordered after the caller's stream
    if (!ctx->aux_stream) QCD_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    st = ctx->aux_stream;
    stream = (void*)st;
  }
  const Geom& g = ctx->geom;
  Workspace* w = workspace(ctx, nrhs, true);
  const size_t n2 = (size_t)g.vol * 12;
  const size_t canon_bytes = (size_t)g.vol * 24 * sizeof(double) * nrhs;
  const dim3 rgrid(w->nblocks, nrhs);
  const dim3 sgrid(grid_for(g.vol, 128), nrhs);
  double* d_red = w->dres;  // [0, nrhs): |b|^2, [nrhs, 2 nrhs): |r|^2, [2 nrhs, 3 nrhs): scale
  std::vector<double> h_b2(nrhs), h_r2(nrhs), h_scale(nrhs);

  // import b (and the guess), r = b - D x
  int rc = qcd_import_spinor(ctx, w->b64, b, QCD_PREC_DOUBLE, nrhs, on_device, stream);
  if (rc != QCD_OK) throw Error{rc, ctx->err};
  {
    LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
    k_norm2_f64<<<rgrid, RED_THREADS, 0, st>>>(w->b64, n2, d_red, w->partials, w->counters);
    check_launch();
  }
  // residual precision: double-float on the float32 pipes (default) or native
  // float64; the flexible GMRES outer iteration is float64 throughout
  const bool df = P.residual_prec == 0 && P.outer_restart == 0;
  float4* bdf = reinterpret_cast<float4*>(w->t64);
  float4* xdf = reinterpret_cast<float4*>(w->x64);
  float4* rdf = reinterpret_cast<float4*>(w->r64);
  if (df) {
    LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
    k_df_from_f64<<<dim3(1024, nrhs), 256, 0, st>>>(w->b64, bdf, n2, d_red);
    check_launch();
  }
  if (P.x_is_guess) {
    rc = qcd_import_spinor(ctx, w->x64, x, QCD_PREC_DOUBLE, nrhs, on_device, stream);
    if (rc != QCD_OK) throw Error{rc, ctx->err};
    if (df) {
      LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
      k_df_from_f64<<<dim3(1024, nrhs), 256, 0, st>>>(w->x64, xdf, n2, d_red);
      check_launch();
    }
  } else {
    QCD_CUDA_CHECK(cudaMemsetAsync(w->x64, 0, n2 * sizeof(double2) * nrhs, st));
  }
  // device-side failures (a bounded wait that gave up) are read with every residual
  int dev_status = QCD_OK;
  QCD_CUDA_CHECK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  auto residual = [&]() {
    if (df) {
      dslash_launch(ctx, rdf, xdf, PREC_DF64, MODE_D, nrhs, st);
      LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
      k_residual_df<<<rgrid, RED_THREADS, 0, st>>>(bdf, rdf, n2, d_red, d_red + nrhs, w->partials, w->counters);
      check_launch();
    } else {
      dslash_launch(ctx, w->r64, w->x64, QCD_PREC_DOUBLE, MODE_D, nrhs, st);
      LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
      k_residual_f64<<<rgrid, RED_THREADS, 0, st>>>(w->b64, w->r64, n2, d_red + nrhs, w->partials, w->counters);
      check_launch();
    }
    QCD_CUDA_CHECK(cudaMemcpyAsync(h_r2.data(), d_red + nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(&dev_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  };
  if (P.x_is_guess) {
    residual();
  } else {
    // x = 0: r = b exactly, no operator application needed
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->r64, df ? (const void*)bdf : (const void*)w->b64, n2 * sizeof(double2) * nrhs,
                                   cudaMemcpyDeviceToDevice, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(d_red + nrhs, d_red, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(h_r2.data(), d_red, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  }
  QCD_CUDA_CHECK(cudaMemcpyAsync(h_b2.data(), d_red, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));

  int outer = 0, inner_total = 0, last_inner_status = QCD_OK, breakdowns = 0;
  double worst_rel = 0.0;
  auto rel = [&](int r) { return h_b2[r] > 0 ? std::sqrt(h_r2[r] / h_b2[r]) : 0.0; };
  if (P.outer_restart > 0) {
    // ---- flexible GMRES(m) in float64 (one right-hand side) ----------------
    // Arnoldi on D with the inner SAP-BiCGStab solve z_j ~ D^-1 v_j as a
    // preconditioner that may differ from step to step, so the directions
    // z_j are kept and x += Z y at the end of each cycle; modified
    // Gram-Schmidt in float64; complex Givens rotations on the host give the
    // residual estimate |g_{j+1}| after every step.  Each cycle ends with
    // the true residual r = b - D x.
    using cplx = std::complex<double>;
    const int m = P.outer_restart;
    if (w->fg_m < m) {
      if (w->fg) cudaFree(w->fg);
      if (w->fg_h) cudaFree(w->fg_h);
      w->fg = nullptr;
      w->fg_h = nullptr;
      w->fg_m = 0;
      QCD_CUDA_CHECK(cudaMalloc(&w->fg, sizeof(double2) * n2 * (2 * (size_t)m + 1)));
      QCD_CUDA_CHECK(cudaMalloc(&w->fg_h, sizeof(double) * 2 * (m + 2)));
      w->fg_m = m;
    }
    double2* V = w->fg;                        // v_i = V + i n2, i = 0..m
    double2* Z = w->fg + (size_t)(m + 1) * n2;  // z_j = Z + j n2, j < m
    const dim3 vgrid(w->nblocks, 1);
    std::vector<cplx> H((size_t)(m + 1) * m), sn(m), gv(m + 1), y(m);
    std::vector<double> cs(m), hcol(2 * (m + 2));
    const double bnorm = std::sqrt(h_b2[0]);
    h_scale[0] = 1.0;
    QCD_CUDA_CHECK(cudaMemcpyAsync(d_red + 2 * nrhs, h_scale.data(), sizeof(double), cudaMemcpyHostToDevice, st));
    bool stop = false;
    while (!stop) {
      if (dev_status == QCD_ERR_TIMEOUT) {
        result = QCD_ERR_TIMEOUT;
        break;
      }
      worst_rel = rel(0);
      if (!std::isfinite(h_r2[0])) {
        result = QCD_ERR_NONFINITE;
        break;
      }
      if (worst_rel < P.tol) break;
      if (outer >= P.max_outer) {
        result = last_inner_status == QCD_ERR_BREAKDOWN ? QCD_ERR_BREAKDOWN : QCD_ERR_NOT_CONVERGED;
        break;
      }
      const double beta = std::sqrt(h_r2[0]);
      {
        LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
        k_scale_f64<<<vgrid, RED_THREADS, 0, st>>>(V, w->r64, n2, 1.0 / beta);
        check_launch();
      }
      std::fill(gv.begin(), gv.end(), cplx(0.0));
      gv[0] = beta;
      int j = 0;
      while (j < m && outer < P.max_outer) {
        ++outer;
        double2* vj = V + (size_t)j * n2;
        double2* vn = V + (size_t)(j + 1) * n2;
        double2* zj = Z + (size_t)j * n2;
        // z_j: the inner solve of A q = C_inv R_SP(v_j), i.e. D q = v_j
        {
          LaunchScope ls(ctx, QCD_KC_BLAS, st);
          k_f64_to_f32_scaled<<<sgrid, 128, 0, st>>>(g, vj, w->tmp32, d_red + 2 * nrhs);
          check_launch();
        }
        clover_apply_launch(ctx, w->tmp32, w->tmp32, QCD_PREC_SINGLE, 1, 1, st);
        int st_inner = QCD_OK;
        inner_total += bicgstab_sap(ctx, w, w->tmp32, 1, P, st, &st_inner);
        last_inner_status = st_inner;
        if (st_inner == QCD_ERR_BREAKDOWN) ++breakdowns;
        QCD_CUDA_CHECK(cudaMemcpyAsync(&dev_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        QCD_CUDA_CHECK(cudaStreamSynchronize(st));
        if (dev_status == QCD_ERR_TIMEOUT) {
          result = QCD_ERR_TIMEOUT;
          stop = true;
          break;
        }
        if (st_inner == QCD_ERR_NONFINITE) {
          result = QCD_ERR_NONFINITE;
          stop = true;
          break;
        }
        QCD_CUDA_CHECK(cudaMemsetAsync(zj, 0, sizeof(double2) * n2, st));
        {
          LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
          k_f64_axpy_f32<<<sgrid, 128, 0, st>>>(g, zj, w->x, d_red + 2 * nrhs);
          check_launch();
        }
        // v_{j+1} = D z_j orthogonalised against v_0 .. v_j, then normalised
        dslash_launch(ctx, vn, zj, QCD_PREC_DOUBLE, MODE_D, 1, st);
        {
          LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
          for (int i = 0; i <= j; ++i) {
            const double2* vi = V + (size_t)i * n2;
            k_cdot_f64<<<vgrid, RED_THREADS, 0, st>>>(vi, vn, n2, w->fg_h + 2 * i, w->partials, w->counters);
            k_caxmy_f64<<<vgrid, RED_THREADS, 0, st>>>(vn, vi, n2, w->fg_h + 2 * i);
          }
          k_norm2_f64<<<vgrid, RED_THREADS, 0, st>>>(vn, n2, w->fg_h + 2 * (j + 1), w->partials, w->counters);
          k_normalize_f64<<<vgrid, RED_THREADS, 0, st>>>(vn, n2, w->fg_h + 2 * (j + 1));
          check_launch();
          ctx->launches += 2 * j + 3;  // 2 (j + 1) + 2 kernels in this scope
        }
        QCD_CUDA_CHECK(cudaMemcpyAsync(hcol.data(), w->fg_h, sizeof(double) * 2 * (j + 2), cudaMemcpyDeviceToHost, st));
        QCD_CUDA_CHECK(cudaStreamSynchronize(st));
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = cplx(hcol[2 * i], hcol[2 * i + 1]);
        const double hn = std::sqrt(std::max(hcol[2 * (j + 1)], 0.0));
        // earlier rotations on column j, then the one that zeroes H[j+1][j]
        for (int i = 0; i < j; ++i) {
          const cplx a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
          H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * b;
        }
        const cplx a = H[(size_t)j * m + j];
        const double nu = std::sqrt(std::norm(a) + hn * hn);
        if (std::abs(a) == 0.0) {
          cs[j] = 0.0;
          sn[j] = 1.0;
        } else {
          cs[j] = std::abs(a) / nu;
          sn[j] = (a / std::abs(a)) * hn / nu;
        }
        H[(size_t)j * m + j] = cs[j] * a + sn[j] * hn;
        gv[j + 1] = -std::conj(sn[j]) * gv[j];
        gv[j] = cs[j] * gv[j];
        ++j;
        if (!std::isfinite(std::abs(gv[j]))) {
          result = QCD_ERR_NONFINITE;
          stop = true;
          break;
        }
        if (std::abs(gv[j]) < P.tol * bnorm || hn == 0.0) break;
      }
      if (stop || j == 0) break;
      // y from the triangular system R y = g, then x += Z y
      for (int k = j - 1; k >= 0; --k) {
        cplx acc = gv[k];
        for (int l = k + 1; l < j; ++l) acc -= H[(size_t)k * m + l] * y[l];
        y[k] = acc / H[(size_t)k * m + k];
      }
      {
        LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
        for (int k = 0; k < j; ++k)
          k_caxpy_f64<<<vgrid, RED_THREADS, 0, st>>>(w->x64, Z + (size_t)k * n2, n2, y[k].real(), y[k].imag());
        check_launch();
        ctx->launches += j - 1;
      }
      residual();
    }
  } else {
  for (;;) {
    if (dev_status == QCD_ERR_TIMEOUT) {
      result = QCD_ERR_TIMEOUT;
      break;
    }
    worst_rel = 0.0;
    bool finite = true;
    for (int r = 0; r < nrhs; ++r) {
      worst_rel = std::max(worst_rel, rel(r));
      finite = finite && std::isfinite(h_r2[r]);
    }
    if (!finite) {
      result = QCD_ERR_NONFINITE;
      break;
    }
    if (worst_rel < P.tol) break;
    if (outer >= P.max_outer) {
      result = last_inner_status == QCD_ERR_BREAKDOWN ? QCD_ERR_BREAKDOWN : QCD_ERR_NOT_CONVERGED;
      break;
    }
    ++outer;
    // p = R_SP(r / err); the inner right-hand side of A q = C_inv p
    for (int r = 0; r < nrhs; ++r) h_scale[r] = h_r2[r] > 0 ? 1.0 / std::sqrt(h_r2[r]) : 0.0;
    QCD_CUDA_CHECK(cudaMemcpyAsync(d_red + 2 * nrhs, h_scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls(ctx, QCD_KC_BLAS, st);
      if (df) k_df_to_f32_scaled<<<sgrid, 128, 0, st>>>(g, rdf, w->tmp32, d_red + 2 * nrhs, d_red);
      else k_f64_to_f32_scaled<<<sgrid, 128, 0, st>>>(g, w->r64, w->tmp32, d_red + 2 * nrhs);
      check_launch();
    }
    clover_apply_launch(ctx, w->tmp32, w->tmp32, QCD_PREC_SINGLE, 1, nrhs, st);
    int st_inner = QCD_OK;
    inner_total += bicgstab_sap(ctx, w, w->tmp32, nrhs, P, st, &st_inner);
    last_inner_status = st_inner;
    if (st_inner == QCD_ERR_BREAKDOWN) ++breakdowns;
    QCD_CUDA_CHECK(cudaMemcpyAsync(&dev_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    if (dev_status == QCD_ERR_TIMEOUT) {
      result = QCD_ERR_TIMEOUT;
      break;
    }
    if (st_inner == QCD_ERR_NONFINITE) {
      result = QCD_ERR_NONFINITE;
      break;
    }
    // x += err * P_DP(q)
    for (int r = 0; r < nrhs; ++r) h_scale[r] = std::sqrt(h_r2[r]);
    QCD_CUDA_CHECK(cudaMemcpyAsync(d_red + 2 * nrhs, h_scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
      if (df) k_df_axpy_f32<<<sgrid, 128, 0, st>>>(g, xdf, w->x, d_red + 2 * nrhs, d_red);
      else k_f64_axpy_f32<<<sgrid, 128, 0, st>>>(g, w->x64, w->x, d_red + 2 * nrhs);
      check_launch();
    }
    residual();
  }
  }
  if (df) {
    LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
    k_f64_from_df<<<dim3(1024, nrhs), 256, 0, st>>>(xdf, w->x64, n2, d_red);
    check_launch();
  }
  rc = qcd_export_spinor(ctx, x, w->x64, QCD_PREC_DOUBLE, nrhs, on_device, stream);
  if (rc != QCD_OK) throw Error{rc, ctx->err};
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  (void)canon_bytes;
  (void)breakdowns;
  if (info) {
    info->outer_iters = outer;
    info->inner_iters = inner_total;
    info->status = result;
    info->true_resid = worst_rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (result != QCD_OK) {
    ctx->err = result == QCD_ERR_NOT_CONVERGED ? "qcd_solve: tolerance not reached"
               : result == QCD_ERR_BREAKDOWN   ? "qcd_solve: BiCGStab breakdown"
               : result == QCD_ERR_TIMEOUT     ? "qcd_solve: a bounded device-side wait gave up"
                                               : "qcd_solve: non-finite residual";
    return result;
  }
  API_END(ctx)
}
