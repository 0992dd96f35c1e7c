// Internal types shared by the CUDA translation units of libqcd_gb300.
//
// Device layout ("internal layout"): the lattice is cut into domains of
// d = (dx, dy, dz, dt) sites (powers of two, at most 256 sites).  Domains are
// coloured by the parity of the sum of their domain coordinates (Sec. 3,
// red/black domain decomposition); all even (E) domains come first, then all
// odd (O) ones, each half in lexicographic domain order.  Inside a domain the
// site index is s = ((t dz + z) dy + y) dx + x.  Every field is a structure of
// arrays per domain so that a warp touching consecutive sites of a domain
// issues one coalesced 128-bit (or 64-bit) access per component group:
//
//   quark float32 : float4  [rhs][domain][6 groups][vd]   (24 floats / site)
//   quark float64 : double2 [rhs][domain][12 comps][vd]   (12 complex / site)
//   quark float16 : uint4   [rhs][domain][3 groups][vd]   (24 halves / site)
//                 + float   [rhs][domain][vd]            (per-site norm)
//   links  float32: float2  [domain][mu][9][vd]           (3x3 complex)
//   links  float64: double2 [domain][mu][9][vd]
//   links  float16: __half2 [domain][mu][9][vd]
//   clover float32: float4  [domain][18][vd]  (two packed 6x6 Hermitian blocks)
//   clover float64: double2 [domain][36][vd]
//   clover float16: __half2 [domain][36][vd]
//
// Quark components inside a site are ordered (spin, colour, re/im) in the
// chiral gamma basis; the upper chirality (spins 0, 1) occupies float4
// groups 0-2, the lower (spins 2, 3) groups 3-5, matching the two clover
// blocks.  A packed Hermitian 6x6 block holds its 6 real diagonal entries
// followed by the 15 complex entries (i < j) in row-major order; its index i
// is (spin within the block) * 3 + colour.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>
#include <utility>

#include "qcd_gb300.h"
#include "df64.cuh"

namespace qcd {

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Geom {
  int L[4];        // lattice extents x, y, z, t
  int d[4];        // domain extents
  int nd[4];       // domains per direction
  int logd[4];     // log2 d_mu
  int shift[4];    // bit offset of local coordinate mu inside s
  int vd;          // sites per domain
  int logvd;
  int ndom;        // domains in total
  int nhalf;       // domains per colour
  long long vol;   // sites
  int bc_t;        // +1 periodic, -1 antiperiodic in t
  const int* nbr;  // [ndom][8]: neighbour domain across face 2 mu (+) / 2 mu + 1 (-)
  const unsigned char* tflag;  // [ndom]: bit k set when face k crosses t = Lt-1 <-> 0
  const int* lex2dom;          // [ndom]: lexicographic domain index -> storage index
  const int* run_flag;         // if set: operator kernels return at once when *run_flag == 0
};

// true when a kernel launched inside the device-side solver loop has nothing
// left to do (every right-hand side has stopped iterating)
__device__ __forceinline__ bool loop_idle(const Geom& g) {
  return g.run_flag != nullptr && *(volatile const int*)g.run_flag == 0;
}

// Neighbouring site of (dom, s) in direction mu, forward (fwd) or backward.
// Returns the sign of the boundary condition carried by the hop.
__device__ __forceinline__ int nbr_site(const Geom& g, int dom, int s, int mu, bool fwd,
                                        int& ndom_out, int& ns_out) {
  const int c = (s >> g.shift[mu]) & (g.d[mu] - 1);
  const int step = 1 << g.shift[mu];
  if (fwd) {
    if (c < g.d[mu] - 1) {
      ndom_out = dom;
      ns_out = s + step;
      return 1;
    }
    ndom_out = __ldg(g.nbr + dom * 8 + 2 * mu);
    ns_out = s - (g.d[mu] - 1) * step;
    return ((__ldg(g.tflag + dom) >> (2 * mu)) & 1) ? g.bc_t : 1;
  }
  if (c > 0) {
    ndom_out = dom;
    ns_out = s - step;
    return 1;
  }
  ndom_out = __ldg(g.nbr + dom * 8 + 2 * mu + 1);
  ns_out = s + (g.d[mu] - 1) * step;
  return ((__ldg(g.tflag + dom) >> (2 * mu + 1)) & 1) ? g.bc_t : 1;
}

// true when the hop (dom, s) -> direction mu stays inside the domain
__device__ __forceinline__ bool hop_is_intra(const Geom& g, int s, int mu, bool fwd) {
  const int c = (s >> g.shift[mu]) & (g.d[mu] - 1);
  return fwd ? (c < g.d[mu] - 1) : (c > 0);
}

// Global coordinates -> (domain, local site).
__device__ __forceinline__ void coords_to_internal(const Geom& g, const int x[4], int& dom, int& s) {
  int dc[4];
  s = 0;
  int lex = 0;
#pragma unroll
  for (int mu = 3; mu >= 0; --mu) {
    dc[mu] = x[mu] >> g.logd[mu];
    lex = lex * g.nd[mu] + dc[mu];
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) s |= (x[mu] & (g.d[mu] - 1)) << g.shift[mu];
  const int colour = (dc[0] + dc[1] + dc[2] + dc[3]) & 1;
  dom = colour * g.nhalf + (lex >> 1);
}

// canonical site index n = ((t Lz + z) Ly + y) Lx + x -> coordinates
__device__ __forceinline__ void site_coords(const Geom& g, long long n, int x[4]) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    x[mu] = (int)(n % g.L[mu]);
    n /= g.L[mu];
  }
}

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> make_cx(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return make_cx(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return make_cx(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return make_cx(-a.re, -a.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return make_cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R a, cx<R> b) { return make_cx(a * b.re, a * b.im); }
template <typename R>
__device__ __forceinline__ cx<R> conjg(cx<R> a) { return make_cx(a.re, -a.im); }
template <typename R>
__device__ __forceinline__ cx<R> times_i(cx<R> a) { return make_cx(-a.im, a.re); }
template <typename R>
__device__ __forceinline__ cx<R> times_mi(cx<R> a) { return make_cx(a.im, -a.re); }
// acc + a * b
template <typename R>
__device__ __forceinline__ cx<R> cmac(cx<R> acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cmacc(cx<R> acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}

template <typename R>
struct Spinor {
  cx<R> v[4][3];  // [spin][colour], chiral basis
};
template <typename R>
struct HalfSpinor {
  cx<R> h[2][3];
};
template <typename R>
struct SU3 {
  cx<R> m[3][3];
};

template <typename R>
__device__ __forceinline__ void zero(Spinor<R>& a) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) a.v[s][c] = make_cx<R>(0, 0);
}

// ---------------------------------------------------------------------------
// spin projection in the chiral basis
//   gamma_4 = [[0, 1], [1, 0]],  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]].
// PM = -1 selects (1 - gamma_mu), PM = +1 selects (1 + gamma_mu).  project()
// returns the two independent spin rows h (the upper half of the projected
// spinor); accumulate() adds the full projected spinor rebuilt from U h.
// ---------------------------------------------------------------------------
// one colour: (u0, u1, l0, l1) are the four spins of that colour
template <int MU, int PM, typename R>
__device__ __forceinline__ void project1(cx<R> u0, cx<R> u1, cx<R> l0, cx<R> l1, cx<R>& h0, cx<R>& h1) {
  if (MU == 0) {
    if (PM < 0) { h0 = u0 + times_i(l1); h1 = u1 + times_i(l0); }
    else        { h0 = u0 - times_i(l1); h1 = u1 - times_i(l0); }
  } else if (MU == 1) {
    if (PM < 0) { h0 = u0 + l1; h1 = u1 - l0; }
    else        { h0 = u0 - l1; h1 = u1 + l0; }
  } else if (MU == 2) {
    if (PM < 0) { h0 = u0 + times_i(l0); h1 = u1 - times_i(l1); }
    else        { h0 = u0 - times_i(l0); h1 = u1 + times_i(l1); }
  } else {
    if (PM < 0) { h0 = u0 - l0; h1 = u1 - l1; }
    else        { h0 = u0 + l0; h1 = u1 + l1; }
  }
}

template <int MU, int PM, typename R>
__device__ __forceinline__ void project(const Spinor<R>& p, HalfSpinor<R>& h) {
#pragma unroll
  for (int c = 0; c < 3; ++c) project1<MU, PM>(p.v[0][c], p.v[1][c], p.v[2][c], p.v[3][c], h.h[0][c], h.h[1][c]);
}

// a + f x for a real factor f
template <typename R>
__device__ __forceinline__ cx<R> cfma(R f, const cx<R>& x, const cx<R>& a) {
  return make_cx<R>(fma(f, x.re, a.re), fma(f, x.im, a.im));
}

// one colour: a[sp] += f * (spin sp of the spinor rebuilt from (h0, h1))
template <int MU, int PM, typename R>
__device__ __forceinline__ void accumulate1(cx<R>& a0, cx<R>& a1, cx<R>& a2, cx<R>& a3, cx<R> h0, cx<R> h1, R f) {
  a0 = cfma(f, h0, a0);
  a1 = cfma(f, h1, a1);
  if (MU == 0) {
    if (PM < 0) { a2 = cfma(f, times_mi(h1), a2); a3 = cfma(f, times_mi(h0), a3); }
    else        { a2 = cfma(f, times_i(h1), a2);  a3 = cfma(f, times_i(h0), a3); }
  } else if (MU == 1) {
    if (PM < 0) { a2 = cfma(-f, h1, a2); a3 = cfma(f, h0, a3); }
    else        { a2 = cfma(f, h1, a2);  a3 = cfma(-f, h0, a3); }
  } else if (MU == 2) {
    if (PM < 0) { a2 = cfma(f, times_mi(h0), a2); a3 = cfma(f, times_i(h1), a3); }
    else        { a2 = cfma(f, times_i(h0), a2);  a3 = cfma(f, times_mi(h1), a3); }
  } else {
    if (PM < 0) { a2 = cfma(-f, h0, a2); a3 = cfma(-f, h1, a3); }
    else        { a2 = cfma(f, h0, a2);  a3 = cfma(f, h1, a3); }
  }
}

// acc = the projected spinor rebuilt from h (the first hop of a sum: no
// additions to zero)
template <int MU, int PM, typename R>
__device__ __forceinline__ void rebuild(Spinor<R>& acc, const HalfSpinor<R>& h) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<R> h0 = h.h[0][c], h1 = h.h[1][c];
    acc.v[0][c] = h0;
    acc.v[1][c] = h1;
    if (MU == 0) {
      if (PM < 0) { acc.v[2][c] = times_mi(h1); acc.v[3][c] = times_mi(h0); }
      else        { acc.v[2][c] = times_i(h1);  acc.v[3][c] = times_i(h0); }
    } else if (MU == 1) {
      if (PM < 0) { acc.v[2][c] = -h1; acc.v[3][c] = h0; }
      else        { acc.v[2][c] = h1;  acc.v[3][c] = -h0; }
    } else if (MU == 2) {
      if (PM < 0) { acc.v[2][c] = times_mi(h0); acc.v[3][c] = times_i(h1); }
      else        { acc.v[2][c] = times_i(h0);  acc.v[3][c] = times_mi(h1); }
    } else {
      if (PM < 0) { acc.v[2][c] = -h0; acc.v[3][c] = -h1; }
      else        { acc.v[2][c] = h0;  acc.v[3][c] = h1; }
    }
  }
}

// acc += f * (projected spinor rebuilt from h); f = 1 unless a hop carries
// the antiperiodic sign (a constant 1 folds to plain additions)
template <int MU, int PM, typename R>
__device__ __forceinline__ void accumulate(Spinor<R>& acc, const HalfSpinor<R>& h, R f = R(1.0f)) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
    accumulate1<MU, PM>(acc.v[0][c], acc.v[1][c], acc.v[2][c], acc.v[3][c], h.h[0][c], h.h[1][c], f);
}

// y = U h (both spin rows) or y = U^dag h
template <typename R>
__device__ __forceinline__ void su3_mul(const SU3<R>& u, const HalfSpinor<R>& h, HalfSpinor<R>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = u.m[a][0] * h.h[s][0];
      acc = cmac(acc, u.m[a][1], h.h[s][1]);
      acc = cmac(acc, u.m[a][2], h.h[s][2]);
      y.h[s][a] = acc;
    }
}
template <typename R>
__device__ __forceinline__ void su3_dag_mul(const SU3<R>& u, const HalfSpinor<R>& h, HalfSpinor<R>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = make_cx<R>(0, 0);
      acc = cmacc(acc, u.m[0][a], h.h[s][0]);
      acc = cmacc(acc, u.m[1][a], h.h[s][1]);
      acc = cmacc(acc, u.m[2][a], h.h[s][2]);
      y.h[s][a] = acc;
    }
}

template <typename R>
__device__ __forceinline__ void scale_half(HalfSpinor<R>& h, R f) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) h.h[s][c] = f * h.h[s][c];
}

// offset of packed Hermitian entry (i, j), i < j, in a 6x6 block
__host__ __device__ __forceinline__ int herm_off(int i, int j) { return 5 * i - (i * (i - 1)) / 2 + (j - i - 1); }

// y = M x for one packed Hermitian 6x6 block given as 36 reals
template <typename R, typename Load>
__device__ __forceinline__ void herm6_mul(Load blk, const cx<R> x[6], cx<R> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = blk.diagv(i) * x[i];  // real diagonal: 2 multiplies, not 4
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      const cx<R> a = blk.off(herm_off(i, j));
      y[i] = cmac(y[i], a, x[j]);
      y[j] = cmacc(y[j], a, x[i]);
    }
}

// ---------------------------------------------------------------------------
// field accessors
// ---------------------------------------------------------------------------
struct F32Spinor {
  float4* p;
  __device__ __forceinline__ size_t idx(const Geom& g, int dom, int grp, int s) const {
    return ((size_t)(dom * 6 + grp) << g.logvd) + s;
  }
  __device__ __forceinline__ void load(const Geom& g, int dom, int s, Spinor<float>& a) const {
    float f[24];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 v = __ldg(p + idx(g, dom, k, s));
      f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) a.v[sp][c] = make_cx(f[(sp * 3 + c) * 2], f[(sp * 3 + c) * 2 + 1]);
  }
  __device__ __forceinline__ void store(const Geom& g, int dom, int s, const Spinor<float>& a) const {
    float f[24];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) { f[(sp * 3 + c) * 2] = a.v[sp][c].re; f[(sp * 3 + c) * 2 + 1] = a.v[sp][c].im; }
#pragma unroll
    for (int k = 0; k < 6; ++k) p[idx(g, dom, k, s)] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
  }
  // store with the streaming cache operator (evict first)
  __device__ __forceinline__ void store_stream(const Geom& g, int dom, int s, const Spinor<float>& a) const {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const cx<float> a0 = a.v[(2 * k) / 3][(2 * k) % 3], a1 = a.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
      __stcs(p + idx(g, dom, k, s), make_float4(a0.re, a0.im, a1.re, a1.im));
    }
  }
};

struct F64Spinor {
  double2* p;
  __device__ __forceinline__ size_t idx(const Geom& g, int dom, int comp, int s) const {
    return ((size_t)(dom * 12 + comp) << g.logvd) + s;
  }
  __device__ __forceinline__ void load(const Geom& g, int dom, int s, Spinor<double>& a) const {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double2 v = __ldg(p + idx(g, dom, sp * 3 + c, s));
        a.v[sp][c] = make_cx(v.x, v.y);
      }
  }
  __device__ __forceinline__ void store(const Geom& g, int dom, int s, const Spinor<double>& a) const {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) p[idx(g, dom, sp * 3 + c, s)] = make_double2(a.v[sp][c].re, a.v[sp][c].im);
  }
};

// float16 storage: 24 halves scaled by a per-site float32 norm (max |component|)
struct F16Spinor {
  uint4* p;
  float* nrm;
  __device__ __forceinline__ size_t idx(const Geom& g, int dom, int grp, int s) const {
    return ((size_t)(dom * 3 + grp) << g.logvd) + s;
  }
  __device__ __forceinline__ void load(const Geom& g, int dom, int s, Spinor<float>& a) const {
    const float n = __ldg(nrm + ((size_t)dom << g.logvd) + s);
    float f[24];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint4 v = __ldg(p + idx(g, dom, k, s));
      const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __half2 h2 = *reinterpret_cast<const __half2*>(&w[j]);
        const float2 ff = __half22float2(h2);
        f[8 * k + 2 * j] = ff.x * n;
        f[8 * k + 2 * j + 1] = ff.y * n;
      }
    }
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) a.v[sp][c] = make_cx(f[(sp * 3 + c) * 2], f[(sp * 3 + c) * 2 + 1]);
  }
  __device__ __forceinline__ void store(const Geom& g, int dom, int s, const Spinor<float>& a) const {
    float f[24];
    float m = 0.f;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f[(sp * 3 + c) * 2] = a.v[sp][c].re;
        f[(sp * 3 + c) * 2 + 1] = a.v[sp][c].im;
        m = fmaxf(m, fmaxf(fabsf(a.v[sp][c].re), fabsf(a.v[sp][c].im)));
      }
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    nrm[((size_t)dom << g.logvd) + s] = m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __half2 h2 = __floats2half2_rn(f[8 * k + 2 * j] * inv, f[8 * k + 2 * j + 1] * inv);
        w[j] = *reinterpret_cast<unsigned*>(&h2);
      }
      p[idx(g, dom, k, s)] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
};

template <typename R>
struct LinkPtr;
template <>
struct LinkPtr<float> {
  const float2* p;
  __device__ __forceinline__ void load(const Geom& g, int dom, int mu, int s, SU3<float>& u) const {
    const size_t base = ((size_t)((dom * 4 + mu) * 9)) << g.logvd;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 v = __ldg(p + base + ((size_t)e << g.logvd) + s);
      u.m[e / 3][e % 3] = make_cx(v.x, v.y);
    }
  }
};
template <>
struct LinkPtr<double> {
  const double2* p;
  __device__ __forceinline__ void load(const Geom& g, int dom, int mu, int s, SU3<double>& u) const {
    const size_t base = ((size_t)((dom * 4 + mu) * 9)) << g.logvd;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double2 v = __ldg(p + base + ((size_t)e << g.logvd) + s);
      u.m[e / 3][e % 3] = make_cx(v.x, v.y);
    }
  }
};
// float32 links stored as their first two rows, 12 reals in three float4
// per link ([dom][mu][3][vd]: (u00, u01), (u02, u10), (u11, u12)).  For an
// SU(3) matrix the third row is the complex conjugate of the cross product
// of the first two (unit determinant and unitarity), which the load rebuilds.
struct LinkPtr12 {
  const float4* p;
  __device__ __forceinline__ void load(const Geom& g, int dom, int mu, int s, SU3<float>& u) const {
    const size_t base = ((size_t)((dom * 4 + mu) * 3)) << g.logvd;
    const float4 a = __ldg(p + base + s);
    const float4 b = __ldg(p + base + ((size_t)1 << g.logvd) + s);
    const float4 c = __ldg(p + base + ((size_t)2 << g.logvd) + s);
    u.m[0][0] = make_cx(a.x, a.y);
    u.m[0][1] = make_cx(a.z, a.w);
    u.m[0][2] = make_cx(b.x, b.y);
    u.m[1][0] = make_cx(b.z, b.w);
    u.m[1][1] = make_cx(c.x, c.y);
    u.m[1][2] = make_cx(c.z, c.w);
    // conj(p q - r t) for the three cofactors
    auto cof = [](cx<float> p, cx<float> q, cx<float> r, cx<float> t) {
      const float re = fmaf(p.re, q.re, fmaf(-p.im, q.im, fmaf(-r.re, t.re, r.im * t.im)));
      const float im = fmaf(p.re, q.im, fmaf(p.im, q.re, fmaf(-r.re, t.im, -r.im * t.re)));
      return make_cx(re, -im);
    };
    u.m[2][0] = cof(u.m[0][1], u.m[1][2], u.m[0][2], u.m[1][1]);
    u.m[2][1] = cof(u.m[0][2], u.m[1][0], u.m[0][0], u.m[1][2]);
    u.m[2][2] = cof(u.m[0][0], u.m[1][1], u.m[0][1], u.m[1][0]);
  }
};

struct LinkPtrHalf {
  const __half2* p;
  __device__ __forceinline__ void load(const Geom& g, int dom, int mu, int s, SU3<float>& u) const {
    const size_t base = ((size_t)((dom * 4 + mu) * 9)) << g.logvd;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 v = __half22float2(__ldg(p + base + ((size_t)e << g.logvd) + s));
      u.m[e / 3][e % 3] = make_cx(v.x, v.y);
    }
  }
};

// double-float storage (the float64 residual of the solve): float4 =
// (re.hi, re.lo, im.hi, im.lo) per complex, same element order as float64
struct DF64Spinor {
  float4* p;
  __device__ __forceinline__ size_t idx(const Geom& g, int dom, int comp, int s) const {
    return ((size_t)(dom * 12 + comp) << g.logvd) + s;
  }
  __device__ __forceinline__ void load(const Geom& g, int dom, int s, Spinor<df64>& a) const {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 v = __ldg(p + idx(g, dom, sp * 3 + c, s));
        a.v[sp][c] = make_cx(df64(v.x, v.y), df64(v.z, v.w));
      }
  }
  __device__ __forceinline__ void store(const Geom& g, int dom, int s, const Spinor<df64>& a) const {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        p[idx(g, dom, sp * 3 + c, s)] =
            make_float4(a.v[sp][c].re.hi, a.v[sp][c].re.lo, a.v[sp][c].im.hi, a.v[sp][c].im.lo);
  }
};
template <>
struct LinkPtr<df64> {
  const float4* p;
  __device__ __forceinline__ void load(const Geom& g, int dom, int mu, int s, SU3<df64>& u) const {
    const size_t base = ((size_t)((dom * 4 + mu) * 9)) << g.logvd;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float4 v = __ldg(p + base + ((size_t)e << g.logvd) + s);
      u.m[e / 3][e % 3] = make_cx(df64(v.x, v.y), df64(v.z, v.w));
    }
  }
};

// packed clover block readers (block b = 0 upper, 1 lower)
struct CloverBlockF32 {
  float r[36];
  __device__ __forceinline__ float diagv(int i) const { return r[i]; }
  __device__ __forceinline__ cx<float> diag(int i) const { return make_cx(r[i], 0.f); }
  __device__ __forceinline__ cx<float> off(int k) const { return make_cx(r[6 + 2 * k], r[7 + 2 * k]); }
};
struct CloverBlockF64 {
  double r[36];
  __device__ __forceinline__ double diagv(int i) const { return r[i]; }
  __device__ __forceinline__ cx<double> diag(int i) const { return make_cx(r[i], 0.0); }
  __device__ __forceinline__ cx<double> off(int k) const { return make_cx(r[6 + 2 * k], r[7 + 2 * k]); }
};

struct CloverBlockDF64 {
  df64 r[36];
  __device__ __forceinline__ df64 diagv(int i) const { return r[i]; }
  __device__ __forceinline__ cx<df64> diag(int i) const { return make_cx(r[i], df64(0.f)); }
  __device__ __forceinline__ cx<df64> off(int k) const { return make_cx(r[6 + 2 * k], r[7 + 2 * k]); }
};
struct CloverPtrDF64 {
  const float4* p;  // [dom][36][vd]: two reals of the packed block per float4
  __device__ __forceinline__ void load_block(const Geom& g, int dom, int s, int b, CloverBlockDF64& blk) const {
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const float4 v = __ldg(p + (((size_t)(dom * 36 + 18 * b + k)) << g.logvd) + s);
      blk.r[2 * k] = df64(v.x, v.y);
      blk.r[2 * k + 1] = df64(v.z, v.w);
    }
  }
};

struct CloverPtrF32 {
  const float4* p;
  __device__ __forceinline__ void load_block(const Geom& g, int dom, int s, int b, CloverBlockF32& blk) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = __ldg(p + (((size_t)(dom * 18 + 9 * b + k)) << g.logvd) + s);
      blk.r[4 * k] = v.x; blk.r[4 * k + 1] = v.y; blk.r[4 * k + 2] = v.z; blk.r[4 * k + 3] = v.w;
    }
  }
};
// the same rows read with the streaming cache operator (evict first)
struct CloverPtrF32Stream {
  const float4* p;
  __device__ __forceinline__ void load_block(const Geom& g, int dom, int s, int b, CloverBlockF32& blk) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = __ldcs(p + (((size_t)(dom * 18 + 9 * b + k)) << g.logvd) + s);
      blk.r[4 * k] = v.x; blk.r[4 * k + 1] = v.y; blk.r[4 * k + 2] = v.z; blk.r[4 * k + 3] = v.w;
    }
  }
};
struct CloverPtrF64 {
  const double2* p;
  __device__ __forceinline__ void load_block(const Geom& g, int dom, int s, int b, CloverBlockF64& blk) const {
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const double2 v = __ldg(p + (((size_t)(dom * 36 + 18 * b + k)) << g.logvd) + s);
      blk.r[2 * k] = v.x; blk.r[2 * k + 1] = v.y;
    }
  }
};
struct CloverPtrF16 {
  const __half2* p;
  __device__ __forceinline__ void load_block(const Geom& g, int dom, int s, int b, CloverBlockF32& blk) const {
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const float2 v = __half22float2(__ldg(p + (((size_t)(dom * 36 + 18 * b + k)) << g.logvd) + s));
      blk.r[2 * k] = v.x; blk.r[2 * k + 1] = v.y;
    }
  }
};

// psi <- M psi with the two chiral blocks of a clover field
template <typename R, typename Ptr, typename Blk>
__device__ __forceinline__ void clover_mul(const Ptr& cp, const Geom& g, int dom, int s, Spinor<R>& psi) {
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    Blk blk;
    cp.load_block(g, dom, s, b, blk);
    cx<R> x[6], y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = psi.v[2 * b + i / 3][i % 3];
    herm6_mul<R>(blk, x, y);
#pragma unroll
    for (int i = 0; i < 6; ++i) psi.v[2 * b + i / 3][i % 3] = y[i];
  }
}

// ---------------------------------------------------------------------------
// programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor drains; it must call
// pdl_wait() before touching anything the predecessor writes.  pdl_trigger()
// lets the next such kernel start early.  Both are no-ops otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// context (host side)
// ---------------------------------------------------------------------------
struct Workspace;
struct Profiler;
struct Tuner;

}  // namespace qcd

struct qcd_ctx {
  qcd::Geom geom;
  int basis = QCD_BASIS_CHIRAL;
  int device = 0;
  double kappa = 0.125, csw = 1.0;
  bool have_gauge = false, have_clover = false;
  // device arrays owned by the context
  int* d_nbr = nullptr;
  int* d_lex2dom = nullptr;
  unsigned char* d_tflag = nullptr;
  double2* u64 = nullptr;
  float2* u32 = nullptr;
  __half2* u16 = nullptr;
  float4* u32c = nullptr;          // float32 links as their first two rows (12 reals, three float4)
  bool su3_links = false;          // every link is SU(3) to 1e-9: the third row follows from the first two
  int link12 = -1;                 // float32 D with links as 12 reals: -1 when SU(3), 0 never, 1 always
  double2* clov64 = nullptr;     // 1 + C
  float4* clov32 = nullptr;
  double2* cinv64 = nullptr;     // (1 + C)^-1
  float4* cinv32 = nullptr;
  __half2* cinv16 = nullptr;
  float4* udf = nullptr;         // links in double-float
  float4* clovdf = nullptr;      // 1 + C in double-float
  int* d_status = nullptr;       // device status word (non-finite, ...)
  cudaStream_t aux_stream = nullptr;  // private stream for graph capture
  // staging layouts of the shared-memory SAP kernel (4^4 domains only)
  void* st_link16 = nullptr;
  void* st_link32 = nullptr;
  void* st_clov16 = nullptr;
  void* st_clov32 = nullptr;
  int* flow_state = nullptr;       // one-launch M_SAP: 2 counters, then one flag per domain (zero at rest)
  bool force_generic_sap = false;  // testing: use the generic SAP kernel
  int sap_shape = -1;              // SAP block-kernel shape: -1 autotuned, else an index of the shapes
  bool sap_general = false;        // SAP on domains sap_dom, independent of the storage blocking
  int sap_dom[4] = {0, 0, 0, 0};
  int clover_gen = 0;              // counts clover builds (staging copies follow it)
  void* cl_link = nullptr;         // staging of the cluster SAP kernel (domains sap_dom)
  void* cl_clov = nullptr;
  int cl_gen = -1;
  int cl_dom[4] = {0, 0, 0, 0};
  int inject = 0;                  // testing: QCD_INJECT_* fault (host-side, bounded)
  qcd::Workspace* ws = nullptr;
  qcd::Profiler* prof = nullptr;
  qcd::Tuner* tuner = nullptr;
  long long launches = 0;
  std::string err;
};

namespace qcd {
// whether a context's float32 operator reads its links as 12 reals (its
// links are SU(3) and qcd_set_link_compression does not forbid it, or asks
// for it)
inline bool uses_links12(const qcd_ctx* ctx) {
  return ctx->link12 == 1 || (ctx->link12 == -1 && ctx->su3_links);
}
}  // namespace qcd

namespace qcd {

// error helpers used by the C entry points
struct Error {
  int code;
  std::string msg;
};

#define QCD_CUDA_CHECK(call)                                                            \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::qcd::Error{e_ == cudaErrorMemoryAllocation ? QCD_ERR_OOM : QCD_ERR_CUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_)};            \
  } while (0)

#define QCD_REQUIRE(cond, code, msg)                  \
  do {                                                \
    if (!(cond)) throw ::qcd::Error{(code), (msg)};   \
  } while (0)

// launch bookkeeping: profiling events and the launch counter
void launch_begin(qcd_ctx* ctx, int kclass, cudaStream_t st);
void launch_end(qcd_ctx* ctx, int kclass, cudaStream_t st);

struct LaunchScope {
  qcd_ctx* ctx;
  int kc;
  cudaStream_t st;
  LaunchScope(qcd_ctx* c, int k, cudaStream_t s) : ctx(c), kc(k), st(s) { launch_begin(c, k, s); }
  ~LaunchScope() { launch_end(ctx, kc, st); }
};

inline void check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error{QCD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

inline size_t spinor_bytes(const Geom& g, int prec) {
  const size_t v = (size_t)g.vol;
  if (prec == QCD_PREC_DOUBLE) return v * 24 * sizeof(double);
  if (prec == QCD_PREC_SINGLE) return v * 24 * sizeof(float);
  return v * (24 * sizeof(__half) + sizeof(float));
}

inline int grid_for(long long n, int block) { return (int)((n + block - 1) / block); }

// Autotuner: returns the launch variant to use for `key`.  The first call per
// key with tuning on (and outside stream capture) times every variant with
// CUDA events -- run(v) must be an out-of-place launch whose repetition is
// harmless -- and remembers the fastest; later calls return it.
int tune_pick(qcd_ctx* ctx, const char* key, int nvariants, const char* const* names,
              const std::function<void(int)>& run, cudaStream_t st);
void tuner_free(qcd_ctx* ctx);

// internal entry points implemented in the other translation units
// pdl: launch the float32/float64 operator with programmatic stream
// serialization (back-to-back applications overlap their tails); off inside
// the solver, where it measured slower
void dslash_launch(qcd_ctx* ctx, void* out, const void* in, int prec, int mode, int nrhs, cudaStream_t st,
                   bool pdl = false);
void clover_apply_launch(qcd_ctx* ctx, void* out, const void* in, int prec, int inverse, int nrhs,
                         cudaStream_t st);
void ablock_launch(qcd_ctx* ctx, float4* out, const float4* in, int row, int col, cudaStream_t st);
void build_clover_launch(qcd_ctx* ctx, cudaStream_t st);
void build_sap_staging(qcd_ctx* ctx, cudaStream_t st);
bool sap_staged_available(const qcd_ctx* ctx);
// halo: face halo of the shared-memory SAP kernel, 96 bytes per site and right-hand side
void sap_staged_sequence_f32(qcd_ctx* ctx, F32Spinor s_first_in, F32Spinor s, F32Spinor x, F32Spinor b,
                             float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st);
void sap_staged_sequence_f16(qcd_ctx* ctx, F32Spinor s_first_in, F16Spinor s, F32Spinor b, F32Spinor x_out,
                             float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st);
void sap_staged_sequence_h16g(qcd_ctx* ctx, F32Spinor s_first_in, F32Spinor s, F32Spinor x, F32Spinor b,
                              float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st);
// ws_x16 holds 96 bytes per site and right-hand side: the float16 x of the
// generic kernel, or the face halo of the shared-memory kernel
void sap_apply_launch(qcd_ctx* ctx, float4* x, const float4* b, int nrhs, int n_sap, int n_jac, int sap_prec,
                      void* ws_s, void* ws_x16, void* ws_b16, cudaStream_t st);
void workspace_reset_graphs(qcd_ctx* ctx);
// SAP on the context's general domains (sap_dom, any extents; up to 1152
// sites on the one-CTA kernel, larger ones on the cluster kernel)
bool sap_domain_valid(const int dims[4], const int sdom[4]);
void sap_general_apply(qcd_ctx* ctx, float4* x, const float4* b, int nrhs, int n_sap, int n_jac, int sap_prec,
                       void* ws_s, cudaStream_t st);
// the same with one thread-block cluster per domain (float16 links and C_inv staged in shared memory)
bool sap_cluster_eligible(const qcd_ctx* ctx, int sap_prec);
bool sap_cluster_fits(const int sdom[4]);
bool sap_general_fits(const int sdom[4]);  // the one-CTA kernel: at most 1152 sites
void sap_cluster_apply(qcd_ctx* ctx, float4* x, const float4* b, int nrhs, int n_sap, int n_jac, void* ws_s,
                       cudaStream_t st);
void gauge_import_launch(qcd_ctx* ctx, const double* u, cudaStream_t st);

// dslash modes
enum { MODE_D = 0, MODE_DDAG = 1, MODE_A = 2 };
// internal precision code of the double-float operator (not part of the ABI)
constexpr int PREC_DF64 = 7;
void build_df64_copies(qcd_ctx* ctx, bool links, bool clover, cudaStream_t st);

// one lattice of a ragged batch (device copy, rebuilt for every batched call)
struct BatchDesc {
  Geom g;
  float4* out;
  const float4* in;
  const float2* u;
  const float4* u12;      // the links as 12 reals, when this lattice's operator uses them (else null)
  const float4* clov;
  float kappa;
  long long block_begin;  // first block of this lattice in the batched launch
};
void dslash_batch_launch(const BatchDesc* d_desc, const int* d_block_lat, long long total_blocks, int dagger,
                         cudaStream_t st);

// One lattice of a ragged batch solve, as the shared launches see it: its
// geometry and operator, and where its vectors lie in the batch's ragged
// buffers (built once per batch).
struct LatDesc {
  Geom g;
  float kappa;
  double kappa64;
  const float2* u32;
  const float4* u32c;                  // the links as 12 reals, or null (as uses_links12)
  const float4* cinv32;
  const double2* u64;
  const double2* clov64;
  float4 *x, *q, *t, *zp, *zr, *b32;   // float32 internal fields of Algorithm 5
  double2 *x64, *r64, *b64;            // float64 internal fields of Algorithm 4
  const float4* udf;                   // links and 1 + C in double-float
  const float4* clovdf;
  float4* xdf;                         // scaled double-float copy of x64
  const int* done;                     // this lattice's BiCGStab stop flag
  long long block_begin;               // first 128-thread block of this lattice
  long long df_tile_begin;             // first 64-site double-float tile of this lattice
};
// which: 0 q = A zp, 1 t = A zr (float32; lattices whose done flag is set
// are skipped), 2 r64 = D x64 (float64)
void lat_dslash_launch(const LatDesc* d_lat, const int* d_block_lat, long long blocks, int which, cudaStream_t st);
// r64 = D x of every lattice in double-float, from the copy xdf scaled by
// the power of two of its lattice's |b|^2 (b2), written unscaled in float64
void lat_dslash_df64_launch(const LatDesc* d_lat, const int* d_tile_lat, long long tiles, const double* d_b2,
                            cudaStream_t st);

// M_SAP (Algorithm 1) of every lattice of a ragged batch in shared launches:
// one launch per half-sweep covers every lattice's domains of that colour.
struct SapLat {
  const qcd_ctx* ctx;
  F32Spinor in, out;   // source and result (float32 internal layout)
  float4* s32;         // the s vector in float32 ...
  uint4* s16;          // ... or in float16 storage (values, per-site norms)
  float* s16n;
  float4* halo;        // face halo, 96 bytes per site
  const int* skip;     // nonzero: the lattice has stopped iterating
};
struct SapBatchPlan;
struct RaggedWS;
bool ragged_eligible(const std::vector<qcd_ctx*>& ctx, const qcd_solve_params& P);
int ragged_solve(const std::vector<qcd_ctx*>& ctx, RaggedWS*& ws, double* const* x, const double* const* b,
                 int on_device, const qcd_solve_params& P, qcd_solve_info* infos, cudaStream_t user_st,
                 std::string& err);
void ragged_free(RaggedWS* ws);
SapBatchPlan* sap_batch_plan(const std::vector<SapLat>& lats, int sap_prec, int n_sap, int n_jac, int* status,
                             const int* run_flag);
void sap_batch_run(const SapBatchPlan* plan, qcd_ctx* count_ctx, cudaStream_t st);
void sap_batch_free(SapBatchPlan* plan);

// launch with programmatic stream serialization (see pdl_wait)
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  QCD_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

}  // namespace qcd
