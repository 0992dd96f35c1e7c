// Gradients of L = Re(eta^dag D^-1 b) (differentiation of the solve of
// App. A's operator): d/db by the gamma_5-adjoint solve and d/dU from the
// hopping term and the clover leaves, float32 kernels.
//
// With x = D^-1 b and lambda = D^-dag eta = gamma_5 D^-1 gamma_5 eta,
// dL = -Re(lambda^dag dD x).  Written as dL = sum Re tr(G^dag dU):
//   hopping: G_mu(y) += kappa sum_s [(1 - g_mu) lambda(y)]_s x(y+mu)_s^dag
//                     + kappa sum_s x(y)_s [(1 + g_mu) lambda(y+mu)]_s^dag
//   clover:  per site n and plane p = (mu < nu),
//            Z_p = sum_{alpha,beta} sigma_p[alpha,beta] x_beta lambda_alpha^dag,
//            V_p = (W - W^dag) / 8,  W = -i kappa c_SW Z_p,
//            and every link factor A_k of every leaf of Q_p(n) receives
//            R_k = A_{k+1} .. A_4 V_p(n) A_1 .. A_{k-1} (R_k^dag for an
//            undaggered factor).
// The clover part is gathered per link (no atomics): each thread owns one
// link U_d(y) and visits the 24 (plane, leaf, factor) slots where it occurs.

#include "qcd_internal.cuh"

namespace qcd {

using C32 = cx<float>;
using M3f = SU3<float>;

__device__ __forceinline__ void mm(const M3f& a, const M3f& b, M3f& c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C32 acc = a.m[i][0] * b.m[0][j];
      acc = cmac(acc, a.m[i][1], b.m[1][j]);
      acc = cmac(acc, a.m[i][2], b.m[2][j]);
      c.m[i][j] = acc;
    }
}
__device__ __forceinline__ M3f dg(const M3f& a) {
  M3f r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[i][j] = conjg(a.m[j][i]);
  return r;
}

__device__ __forceinline__ void coords_of(const Geom& g, long long n, int x[4]) { site_coords(g, n, x); }

// periodic wrap of a coordinate at most one period outside [0, L)
__device__ __forceinline__ int wrap1(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// internal (domain, site) of x + off, |off_k| <= 1
__device__ __forceinline__ void at_coords(const Geom& g, const int x[4], const int off[4], int& dom, int& s) {
  int y[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) y[k] = wrap1(x[k] + off[k], g.L[k]);
  coords_to_internal(g, y, dom, s);
}

// leaves of Q_{mu nu}(n): (direction: 0 = mu, 1 = nu; offset along mu; offset
// along nu; daggered)
struct LeafFactor {
  signed char dir, om, on, dag;
};
__constant__ LeafFactor c_leaf[4][4] = {
    {{0, 0, 0, 0}, {1, 1, 0, 0}, {0, 0, 1, 1}, {1, 0, 0, 1}},
    {{1, 0, 0, 0}, {0, -1, 1, 1}, {1, -1, 0, 1}, {0, -1, 0, 0}},
    {{0, -1, 0, 1}, {1, -1, -1, 1}, {0, -1, -1, 0}, {1, 0, -1, 0}},
    {{1, 0, -1, 1}, {0, 0, -1, 0}, {1, 1, -1, 0}, {0, 0, 0, 1}},
};

// plane index of (mu < nu): 0 xy, 1 xz, 2 xt, 3 yz, 4 yt, 5 zt
__host__ __device__ __forceinline__ int plane_index(int mu, int nu) {
  return mu == 0 ? nu - 1 : (mu == 1 ? nu + 1 : 5);
}

// sigma_{mu nu} in the chiral basis, block b (0 upper, 1 lower) as a 2x2
// complex matrix: xy -s3, xz +s2, yz -s1 on both blocks; xt, yt, zt =
// +/- s1, s2, s3 (upper +, lower -).
__device__ void sigma_block(int p, int b, C32 s[2][2]) {
  const float sgn = b == 0 ? 1.f : -1.f;
  int k;       // Pauli index 1..3
  float f;     // prefactor
  switch (p) {
    case 0: k = 3; f = -1.f; break;       // xy
    case 1: k = 2; f = 1.f; break;        // xz
    case 2: k = 1; f = sgn; break;        // xt
    case 3: k = 1; f = -1.f; break;       // yz
    case 4: k = 2; f = sgn; break;        // yt
    default: k = 3; f = sgn; break;       // zt
  }
  const C32 z = make_cx(0.f, 0.f);
  if (k == 1) { s[0][0] = z; s[0][1] = make_cx(f, 0.f); s[1][0] = make_cx(f, 0.f); s[1][1] = z; }
  else if (k == 2) { s[0][0] = z; s[0][1] = make_cx(0.f, -f); s[1][0] = make_cx(0.f, f); s[1][1] = z; }
  else { s[0][0] = make_cx(f, 0.f); s[0][1] = z; s[1][0] = z; s[1][1] = make_cx(-f, 0.f); }
}

// V_p(n) for the six planes, stored as float2 [6][9][site] (canonical site order)
__global__ void clover_v_kernel(Geom g, F32Spinor xs, F32Spinor ls, float kc, float2* V) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.vol) return;
  int x[4];
  coords_of(g, n, x);
  int dom, s;
  coords_to_internal(g, x, dom, s);
  Spinor<float> xv, lv;
  xs.load(g, dom, s, xv);
  ls.load(g, dom, s, lv);
  for (int p = 0; p < 6; ++p) {
    // Z[b][a] = sum_{alpha beta} sigma[alpha][beta] x[beta][b] conj(lambda[alpha][a])
    C32 z[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) z[i][j] = make_cx(0.f, 0.f);
    for (int blk = 0; blk < 2; ++blk) {
      C32 sg[2][2];
      sigma_block(p, blk, sg);
      for (int al = 0; al < 2; ++al)
        for (int be = 0; be < 2; ++be) {
          const C32 sab = sg[al][be];
          if (sab.re == 0.f && sab.im == 0.f) continue;
          for (int b = 0; b < 3; ++b) {
            const C32 t = sab * xv.v[2 * blk + be][b];
            for (int a = 0; a < 3; ++a) z[b][a] = cmacc(z[b][a], lv.v[2 * blk + al][a], t);
          }
        }
    }
    // W = -i kc Z; V = (W - W^dag) / 8
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const C32 wij = make_cx(kc * z[i][j].im, -kc * z[i][j].re);
        const C32 wji = make_cx(kc * z[j][i].im, -kc * z[j][i].re);
        const C32 v = make_cx(0.125f * (wij.re - wji.re), 0.125f * (wij.im + wji.im));
        V[((size_t)(p * 9 + i * 3 + j)) * g.vol + n] = make_float2(v.re, v.im);
      }
  }
}

__device__ __forceinline__ M3f load_v(const Geom& g, const float2* V, int p, long long n) {
  M3f r;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const float2 v = V[((size_t)(p * 9 + e)) * g.vol + n];
    r.m[e / 3][e % 3] = make_cx(v.x, v.y);
  }
  return r;
}

// canonical index of the coordinates x (each in [0, L))
__device__ __forceinline__ long long canon_index(const Geom& g, const int x[4]) {
  return ((long long)(x[3] * g.L[2] + x[2]) * g.L[1] + x[1]) * g.L[0] + x[0];
}

template <int MU>
__device__ void hop_force(const Geom& g, const F32Spinor& xs, const F32Spinor& ls, int dom, int s, float kappa,
                          M3f& G) {
  int nd, ns;
  const int sign = nbr_site(g, dom, s, MU, true, nd, ns);
  Spinor<float> x0, xf, l0, lf;
  xs.load(g, dom, s, x0);
  xs.load(g, nd, ns, xf);
  ls.load(g, dom, s, l0);
  ls.load(g, nd, ns, lf);
  // w1 = (1 - g_mu) lambda(y), w2 = (1 + g_mu) lambda(y + mu)
  HalfSpinor<float> h1, h2;
  Spinor<float> w1, w2;
  project<MU, -1>(l0, h1);
  zero(w1);
  accumulate<MU, -1>(w1, h1);
  project<MU, +1>(lf, h2);
  zero(w2);
  accumulate<MU, +1>(w2, h2);
  const float f = kappa * (float)sign;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      C32 acc = make_cx(0.f, 0.f);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) {
        acc = cmacc(acc, xf.v[sp][b], w1.v[sp][a]);   // w1_a conj(xf_b)
        acc = cmacc(acc, w2.v[sp][b], x0.v[sp][a]);   // x0_a conj(w2_b)
      }
      G.m[a][b] = G.m[a][b] + f * acc;
    }
}

// one thread per link (y, d): G = G_hop + G_clover; project: TA(G U^dag)
__global__ void __launch_bounds__(128) force_kernel(Geom g, F32Spinor xs, F32Spinor ls, LinkPtr<float> U,
                                                    const float2* V, float kappa, int with_clover, int project,
                                                    double* out) {
  // a block takes 32 sites, warp d their links in direction d: the
  // direction, and with it every branch and loop bound below, is uniform
  // across a warp
  const int d = threadIdx.x >> 5;
  const long long n = blockIdx.x * 32LL + (threadIdx.x & 31);
  if (n >= g.vol) return;
  int y[4];
  coords_of(g, n, y);
  int dom, s;
  coords_to_internal(g, y, dom, s);
  M3f G;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G.m[i][j] = make_cx(0.f, 0.f);
  switch (d) {
    case 0: hop_force<0>(g, xs, ls, dom, s, kappa, G); break;
    case 1: hop_force<1>(g, xs, ls, dom, s, kappa, G); break;
    case 2: hop_force<2>(g, xs, ls, dom, s, kappa, G); break;
    default: hop_force<3>(g, xs, ls, dom, s, kappa, G); break;
  }
  if (with_clover) {
    for (int other = 0; other < 4; ++other) {
      if (other == d) continue;
      const int mu = d < other ? d : other, nu = d < other ? other : d;
      const int p = plane_index(mu, nu);
      const int my_dir = d == mu ? 0 : 1;
      for (int leaf = 0; leaf < 4; ++leaf)
        for (int k = 0; k < 4; ++k) {
          const LeafFactor fk = c_leaf[leaf][k];
          if (fk.dir != my_dir) continue;
          // site n of the leaf: y = n + offset_k
          int base[4] = {0, 0, 0, 0};
          base[mu] -= fk.om;
          base[nu] -= fk.on;
          int xn[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) xn[q] = wrap1(y[q] + base[q], g.L[q]);
          const long long nn = canon_index(g, xn);
          // R_k = A_{k+1} .. A_4 V A_1 .. A_{k-1}
          M3f r;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) r.m[i][j] = make_cx(i == j ? 1.f : 0.f, 0.f);
          auto factor = [&](int j) {
            const LeafFactor f = c_leaf[leaf][j];
            int off[4] = {0, 0, 0, 0};
            off[mu] += f.om;
            off[nu] += f.on;
            int fd, fs;
            at_coords(g, xn, off, fd, fs);
            M3f u;
            U.load(g, fd, f.dir == 0 ? mu : nu, fs, u);
            return f.dag ? dg(u) : u;
          };
          M3f tmp;
          for (int j = k + 1; j < 4; ++j) {
            const M3f a = factor(j);
            mm(r, a, tmp);
            r = tmp;
          }
          const M3f v = load_v(g, V, p, nn);
          mm(r, v, tmp);
          r = tmp;
          for (int j = 0; j < k; ++j) {
            const M3f a = factor(j);
            mm(r, a, tmp);
            r = tmp;
          }
          const M3f c = fk.dag ? r : dg(r);
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) G.m[i][j] = G.m[i][j] + c.m[i][j];
        }
    }
  }
  if (project) {
    // M = G U^dag; TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6
    M3f u, m;
    U.load(g, dom, d, s, u);
    mm(G, dg(u), m);
    C32 tr = make_cx(0.f, 0.f);
    for (int i = 0; i < 3; ++i) tr = tr + (m.m[i][i] - conjg(m.m[i][i]));
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        C32 a = 0.5f * (m.m[i][j] - conjg(m.m[j][i]));
        if (i == j) a = a - (1.f / 6.f) * tr;
        G.m[i][j] = a;
      }
  }
  double* o = out + (n * 4 + d) * 18;
  for (int e = 0; e < 9; ++e) {
    o[2 * e] = (double)G.m[e / 3][e % 3].re;
    o[2 * e + 1] = (double)G.m[e / 3][e % 3].im;
  }
}

// gamma_5 on a canonical float64 field in the context's basis
__global__ void gamma5_canonical_kernel(long long vol, double* f, int paper_basis) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= vol) return;
  double* p = f + n * 24;
  for (int c = 0; c < 3; ++c) {
    double* q = p + c * 8;  // spins 0..3 of colour c: (re, im) pairs
    if (paper_basis) {
      // gamma_5 = [[0, 1], [1, 0]] on (upper, lower) spin pairs
      for (int k = 0; k < 4; ++k) {
        const double t = q[k];
        q[k] = q[k + 4];
        q[k + 4] = t;
      }
    } else {
      for (int k = 4; k < 8; ++k) q[k] = -q[k];
    }
  }
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_grad(qcd_ctx* ctx, const double* eta, const double* b, const double* x, const double* lam,
                        double* grad_b, double* grad_U, int project, const qcd_solve_params* params, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  try {
    QCD_REQUIRE(ctx->have_gauge && ctx->have_clover, QCD_ERR_STATE, "qcd_grad: operator not ready");
    QCD_REQUIRE(grad_U || grad_b, QCD_ERR_ARG, "qcd_grad: nothing to compute");
    QCD_REQUIRE((x || b) && (lam || eta), QCD_ERR_ARG, "qcd_grad: need b or x, and eta or lambda");
    const Geom& g = ctx->geom;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cbytes = (size_t)g.vol * 24 * sizeof(double);
    double *xs = nullptr, *ls = nullptr;
    float4 *x32 = nullptr, *l32 = nullptr;
    float2* V = nullptr;
    struct Guard {
      void* p[6];
      ~Guard() {
        for (void* q : p)
          if (q) cudaFree(q);
      }
    } guard{{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}};
    QCD_CUDA_CHECK(cudaMalloc(&xs, cbytes));
    guard.p[0] = xs;
    QCD_CUDA_CHECK(cudaMalloc(&ls, cbytes));
    guard.p[1] = ls;
    qcd_solve_params P;
    if (params) P = *params;
    else qcd_solve_params_default(&P);
    P.x_is_guess = 0;
    qcd_solve_info info;
    const int pb = ctx->basis == QCD_BASIS_PAPER;
    if (!x && !lam && P.outer_restart == 0) {
      // both solves at once: D [x, y] = [b, gamma_5 eta] as two right-hand
      // sides of one batched solve (every launch serves both), lambda = gamma_5 y
      double *rhs2 = nullptr, *sol2 = nullptr;
      QCD_CUDA_CHECK(cudaMalloc(&rhs2, 2 * cbytes));
      guard.p[4] = rhs2;
      QCD_CUDA_CHECK(cudaMalloc(&sol2, 2 * cbytes));
      guard.p[5] = sol2;
      QCD_CUDA_CHECK(cudaMemcpyAsync(rhs2, b, cbytes, cudaMemcpyDeviceToDevice, st));
      QCD_CUDA_CHECK(cudaMemcpyAsync(rhs2 + (size_t)g.vol * 24, eta, cbytes, cudaMemcpyDeviceToDevice, st));
      gamma5_canonical_kernel<<<grid_for(g.vol, 256), 256, 0, st>>>(g.vol, rhs2 + (size_t)g.vol * 24, pb);
      check_launch();
      ctx->launches++;
      const int rc = qcd_solve(ctx, sol2, rhs2, 2, 1, &P, &info, stream);
      if (rc != QCD_OK) throw Error{rc, "qcd_grad: solve failed: " + ctx->err};
      QCD_CUDA_CHECK(cudaMemcpyAsync(xs, sol2, cbytes, cudaMemcpyDeviceToDevice, st));
      QCD_CUDA_CHECK(cudaMemcpyAsync(ls, sol2 + (size_t)g.vol * 24, cbytes, cudaMemcpyDeviceToDevice, st));
      gamma5_canonical_kernel<<<grid_for(g.vol, 256), 256, 0, st>>>(g.vol, ls, pb);
      check_launch();
      ctx->launches++;
      cudaFree(rhs2);
      cudaFree(sol2);
      guard.p[4] = guard.p[5] = nullptr;
    } else {
    if (x) {
      QCD_CUDA_CHECK(cudaMemcpyAsync(xs, x, cbytes, cudaMemcpyDeviceToDevice, st));
    } else {
      const int rc = qcd_solve(ctx, xs, b, 1, 1, &P, &info, stream);
      if (rc != QCD_OK) throw Error{rc, "qcd_grad: forward solve failed: " + ctx->err};
    }
    if (lam) {
      QCD_CUDA_CHECK(cudaMemcpyAsync(ls, lam, cbytes, cudaMemcpyDeviceToDevice, st));
    } else {
      double* e5 = nullptr;
      QCD_CUDA_CHECK(cudaMalloc(&e5, cbytes));
      guard.p[4] = e5;
      QCD_CUDA_CHECK(cudaMemcpyAsync(e5, eta, cbytes, cudaMemcpyDeviceToDevice, st));
      gamma5_canonical_kernel<<<grid_for(g.vol, 256), 256, 0, st>>>(g.vol, e5, pb);
      check_launch();
      ctx->launches++;
      const int rc = qcd_solve(ctx, ls, e5, 1, 1, &P, &info, stream);
      if (rc != QCD_OK) throw Error{rc, "qcd_grad: adjoint solve failed: " + ctx->err};
      gamma5_canonical_kernel<<<grid_for(g.vol, 256), 256, 0, st>>>(g.vol, ls, pb);
      check_launch();
      ctx->launches++;
    }
    }
    if (grad_b) QCD_CUDA_CHECK(cudaMemcpyAsync(grad_b, ls, cbytes, cudaMemcpyDeviceToDevice, st));
    if (grad_U) {
      const size_t b32 = spinor_bytes(g, QCD_PREC_SINGLE);
      QCD_CUDA_CHECK(cudaMalloc(&x32, b32));
      guard.p[2] = x32;
      QCD_CUDA_CHECK(cudaMalloc(&l32, b32));
      guard.p[3] = l32;
      int rc = qcd_import_spinor(ctx, x32, xs, QCD_PREC_SINGLE, 1, 1, stream);
      if (rc != QCD_OK) throw Error{rc, ctx->err};
      rc = qcd_import_spinor(ctx, l32, ls, QCD_PREC_SINGLE, 1, 1, stream);
      if (rc != QCD_OK) throw Error{rc, ctx->err};
      const int with_clover = ctx->csw != 0.0;
      if (with_clover) {
        QCD_CUDA_CHECK(cudaMalloc(&V, (size_t)g.vol * 54 * sizeof(float2)));
        guard.p[5] = V;
        LaunchScope ls_(ctx, QCD_KC_OTHER, st);
        clover_v_kernel<<<grid_for(g.vol, 128), 128, 0, st>>>(g, F32Spinor{x32}, F32Spinor{l32},
                                                              (float)(ctx->kappa * ctx->csw), V);
        check_launch();
      }
      {
        LaunchScope ls_(ctx, QCD_KC_OTHER, st);
        force_kernel<<<grid_for(g.vol, 32), 128, 0, st>>>(g, F32Spinor{x32}, F32Spinor{l32},
                                                              LinkPtr<float>{ctx->u32}, V, (float)ctx->kappa,
                                                              with_clover, project, grad_U);
        check_launch();
      }
    }
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  } catch (const qcd::Error& e) {
    ctx->err = e.msg;
    return e.code;
  } catch (...) {
    ctx->err = "unknown error";
    return QCD_ERR_CUDA;
  }
  return QCD_OK;
}
