// Clover term and its inverse (App. A of arXiv:2109.10687), float64.
//
// F_mu,nu(n) = (Q_mu,nu - Q_mu,nu^dag) / 8 with Q the sum of the four
// plaquettes ("leaves") in the mu-nu plane through n, all oriented the same
// way; C = i kappa c_SW sum_{mu<nu} sigma_mu,nu F_mu,nu.  In the chiral basis
// sigma_mu,nu is block diagonal, so 1 + C splits into two 6x6 Hermitian
// blocks per site:
//   upper: sigma_1 (F_xt - F_yz) + sigma_2 (F_xz + F_yt) + sigma_3 (F_zt - F_xy)
//   lower: sigma_1 (-F_xt - F_yz) + sigma_2 (F_xz - F_yt) + sigma_3 (-F_zt - F_xy)
// (sigma_k (x) A = [[A_3, A_1 - i A_2], [A_1 + i A_2, -A_3]] on (spin, colour)),
// each multiplied by i kappa c_SW.  C_inv = (1 + C)^-1 is taken per block by
// Gauss-Jordan elimination with partial pivoting in float64.

#include "qcd_internal.cuh"

namespace qcd {

using C64 = cx<double>;
using M3 = SU3<double>;

__device__ __forceinline__ void mat_mul(const M3& a, const M3& b, M3& c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C64 acc = a.m[i][0] * b.m[0][j];
      acc = cmac(acc, a.m[i][1], b.m[1][j]);
      acc = cmac(acc, a.m[i][2], b.m[2][j]);
      c.m[i][j] = acc;
    }
}

__device__ __forceinline__ M3 dagger(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[i][j] = conjg(a.m[j][i]);
  return r;
}

// U_mu at site x + off (periodic wrap; links carry no boundary sign)
__device__ __forceinline__ M3 link_at(const Geom& g, const LinkPtr<double>& U, const int x[4], const int off[4],
                                      int mu) {
  int y[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) y[k] = (x[k] + off[k] + g.L[k]) % g.L[k];
  int dom, s;
  coords_to_internal(g, y, dom, s);
  M3 u;
  U.load(g, dom, mu, s, u);
  return u;
}

__device__ M3 prod4(const M3& a, const M3& b, const M3& c, const M3& d) {
  M3 t1, t2, r;
  mat_mul(a, b, t1);
  mat_mul(t1, c, t2);
  mat_mul(t2, d, r);
  return r;
}

// anti-Hermitian F_mu,nu = (Q - Q^dag) / 8
__device__ M3 field_strength(const Geom& g, const LinkPtr<double>& U, const int x[4], int mu, int nu) {
  auto at = [&](int dm, int dn, int dir) {
    int off[4] = {0, 0, 0, 0};
    off[mu] += dm;
    off[nu] += dn;
    return link_at(g, U, x, off, dir);
  };
  const M3 um = at(0, 0, mu), un = at(0, 0, nu);
  M3 q1 = prod4(um, at(1, 0, nu), dagger(at(0, 1, mu)), dagger(un));
  M3 q2 = prod4(un, dagger(at(-1, 1, mu)), dagger(at(-1, 0, nu)), at(-1, 0, mu));
  M3 q3 = prod4(dagger(at(-1, 0, mu)), dagger(at(-1, -1, nu)), at(-1, -1, mu), at(0, -1, nu));
  M3 q4 = prod4(dagger(at(0, -1, nu)), at(0, -1, mu), at(1, -1, nu), dagger(um));
  M3 f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const C64 q = q1.m[i][j] + q2.m[i][j] + q3.m[i][j] + q4.m[i][j];
      const C64 qt = conjg(q1.m[j][i] + q2.m[j][i] + q3.m[j][i] + q4.m[j][i]);
      f.m[i][j] = 0.125 * (q - qt);
    }
  return f;
}

// 6x6 matrix (1 + i kappa csw [[A3, A1 - i A2], [A1 + i A2, -A3]])
__device__ void build_block(const M3& a1, const M3& a2, const M3& a3, double kc, C64 m[6][6]) {
  const C64 ikc = make_cx(0.0, kc);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const C64 tl = a3.m[i][j];
      const C64 tr = a1.m[i][j] - times_i(a2.m[i][j]);
      const C64 bl = a1.m[i][j] + times_i(a2.m[i][j]);
      const C64 br = -a3.m[i][j];
      m[i][j] = ikc * tl;
      m[i][j + 3] = ikc * tr;
      m[i + 3][j] = ikc * bl;
      m[i + 3][j + 3] = ikc * br;
    }
  for (int i = 0; i < 6; ++i) m[i][i].re += 1.0;
}

// inverse by Gauss-Jordan with partial pivoting; returns false if singular
__device__ bool invert6(C64 a[6][6], C64 inv[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) inv[i][j] = make_cx(i == j ? 1.0 : 0.0, 0.0);
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    double best = 0.0;
    for (int r = col; r < 6; ++r) {
      const double v = a[r][col].re * a[r][col].re + a[r][col].im * a[r][col].im;
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > 1e-200)) return false;
    if (piv != col)
      for (int j = 0; j < 6; ++j) {
        C64 t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
        t = inv[col][j]; inv[col][j] = inv[piv][j]; inv[piv][j] = t;
      }
    const C64 p = a[col][col];
    const double pn = p.re * p.re + p.im * p.im;
    const C64 pinv = make_cx(p.re / pn, -p.im / pn);
    for (int j = 0; j < 6; ++j) {
      a[col][j] = a[col][j] * pinv;
      inv[col][j] = inv[col][j] * pinv;
    }
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      const C64 f = a[r][col];
      for (int j = 0; j < 6; ++j) {
        a[r][j] = a[r][j] - f * a[col][j];
        inv[r][j] = inv[r][j] - f * inv[col][j];
      }
    }
  }
  return true;
}

// pack a (numerically) Hermitian block into 36 reals: diag, then i<j row-major
__device__ void pack_block(const C64 m[6][6], double r[36]) {
  for (int i = 0; i < 6; ++i) r[i] = m[i][i].re;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      // average with the conjugate of the mirrored entry
      const int k = herm_off(i, j);
      r[6 + 2 * k] = 0.5 * (m[i][j].re + m[j][i].re);
      r[7 + 2 * k] = 0.5 * (m[i][j].im - m[j][i].im);
    }
}

__global__ void __launch_bounds__(64) clover_build_kernel(Geom g, LinkPtr<double> U, double kc, double2* clov64,
                                                          double2* cinv64, float4* clov32, float4* cinv32,
                                                          __half2* cinv16, int* status) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.vol) return;
  int x[4];
  site_coords(g, n, x);
  int dom, s;
  coords_to_internal(g, x, dom, s);
  // planes: 0 xy, 1 xz, 2 xt, 3 yz, 4 yt, 5 zt
  const M3 fxy = field_strength(g, U, x, 0, 1), fxz = field_strength(g, U, x, 0, 2);
  const M3 fxt = field_strength(g, U, x, 0, 3), fyz = field_strength(g, U, x, 1, 2);
  const M3 fyt = field_strength(g, U, x, 1, 3), fzt = field_strength(g, U, x, 2, 3);
  double packed[2][36], packed_inv[2][36];
  for (int b = 0; b < 2; ++b) {
    M3 a1, a2, a3;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        if (b == 0) {
          a1.m[i][j] = fxt.m[i][j] - fyz.m[i][j];
          a2.m[i][j] = fxz.m[i][j] + fyt.m[i][j];
          a3.m[i][j] = fzt.m[i][j] - fxy.m[i][j];
        } else {
          a1.m[i][j] = -(fxt.m[i][j] + fyz.m[i][j]);
          a2.m[i][j] = fxz.m[i][j] - fyt.m[i][j];
          a3.m[i][j] = -(fzt.m[i][j] + fxy.m[i][j]);
        }
      }
    C64 m[6][6], inv[6][6];
    build_block(a1, a2, a3, kc, m);
    pack_block(m, packed[b]);
    if (!invert6(m, inv)) {
      atomicExch(status, 1);
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) inv[i][j] = make_cx(0.0, 0.0);
    }
    pack_block(inv, packed_inv[b]);
  }
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 18; ++k) {
      const size_t idx = (((size_t)(dom * 36 + 18 * b + k)) << g.logvd) + s;
      clov64[idx] = make_double2(packed[b][2 * k], packed[b][2 * k + 1]);
      cinv64[idx] = make_double2(packed_inv[b][2 * k], packed_inv[b][2 * k + 1]);
      cinv16[idx] = __floats2half2_rn((float)packed_inv[b][2 * k], (float)packed_inv[b][2 * k + 1]);
      if (!isfinite(packed_inv[b][2 * k]) || !isfinite(packed_inv[b][2 * k + 1])) atomicExch(status, 1);
    }
  for (int k = 0; k < 18; ++k) {
    const int f0 = 4 * k;
    const double* src = f0 < 36 ? &packed[0][f0] : &packed[1][f0 - 36];
    const double* srci = f0 < 36 ? &packed_inv[0][f0] : &packed_inv[1][f0 - 36];
    const size_t idx = (((size_t)(dom * 18 + k)) << g.logvd) + s;
    clov32[idx] = make_float4((float)src[0], (float)src[1], (float)src[2], (float)src[3]);
    cinv32[idx] = make_float4((float)srci[0], (float)srci[1], (float)srci[2], (float)srci[3]);
  }
}

void build_clover_launch(qcd_ctx* ctx, cudaStream_t st) {
  const Geom& g = ctx->geom;
  LaunchScope ls(ctx, QCD_KC_OTHER, st);
  clover_build_kernel<<<grid_for(g.vol, 64), 64, 0, st>>>(g, LinkPtr<double>{ctx->u64}, ctx->kappa * ctx->csw,
                                                          ctx->clov64, ctx->cinv64, ctx->clov32, ctx->cinv32,
                                                          ctx->cinv16, ctx->d_status);
  check_launch();
}

}  // namespace qcd
