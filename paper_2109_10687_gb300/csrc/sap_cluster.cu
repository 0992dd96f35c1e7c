// SAP half-sweep on large domains of any extents (the paper's 16x6x4x3 and
// 16x6x4x6, Sec. 4.3, Tables 2-3) with one thread-block cluster per domain
// (Sec. 3, Algorithms 1 and 2; float16 links and C_inv, float32 vectors).
//
// A domain d0 x d1 x d2 x d3 is cut into its d3 time slices; CTA t of the
// cluster (cluster rank t) holds slice t, d0 d1 d2 sites, one thread per
// site.  At entry a CTA brings its slice's links (float16, 40 B per link)
// and C_inv (float16, 144 B per site) into shared memory with two bulk
// copies on an mbarrier (bounded wait), from a staging layout built for this
// kernel.  Its shared memory also holds two buffers of the slice's float32
// iterate x.  A Jacobi sweep reads x from the current buffer and writes the
// other: hops in x, y and z stay inside the slice; the t hops read the
// neighbouring slice's x, and for a backward hop its link, from that CTA's
// shared memory through the cluster's distributed shared memory.  One
// cluster barrier per sweep separates the reads of a buffer from the next
// writes to it.  The surface term (hops that leave the domain) reads the
// other colour's x and the neighbouring domains' links from memory.
// Before a CTA leaves, a last cluster barrier keeps its shared memory alive
// while its neighbours may still read it.

#include <cooperative_groups.h>

#include <cstdio>

#include "qcd_internal.cuh"

namespace cg = cooperative_groups;

namespace qcd {

constexpr int CS_MAX_K = 8;            // slices (CTAs) per cluster, the portable maximum
constexpr int CS_MAX_SLICE = 448;      // sites per slice: 496 B of shared memory each
constexpr int CS_LINK_H2 = 10;         // half2 per staged link (9 + 1 pad)
constexpr int CS_CLOV_U4 = 9;          // uint4 per site of staged C_inv
constexpr int CS_BYTES_PER_SITE = 2 * 96 + 4 * CS_LINK_H2 * 4 + CS_CLOV_U4 * 16;  // 496

struct ClusterSapArgs {
  Geom g;
  int sd[4];     // SAP domain extents; sd[3] slices per domain = cluster size
  int snd[4];    // SAP domains per direction
  int slice;     // sites per slice
  int colour, n_jac, do_surface, do_update;
  float kappa;
  F32Spinor s_in, s_out, x, b;
  LinkPtrHalf U16;             // links in the internal layout (backward hops that enter the domain)
  const unsigned char* links;  // staging: [domain][slice][mu][site][10 half2]
  const unsigned char* clov;   // staging: [domain][slice][site][9 uint4]
  int* status;
  int extra_tx;                // testing: bytes the staging wait expects beyond its copies
};

__device__ __forceinline__ SU3<float> cs_link(const unsigned char* base, int slice, int mu, int site) {
  const uint2* p = reinterpret_cast<const uint2*>(base) + (mu * slice + site) * (CS_LINK_H2 / 2);
  SU3<float> u;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint2 w = p[k];
    const float2 v0 = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
    u.m[(2 * k) / 3][(2 * k) % 3] = make_cx(v0.x, v0.y);
    if (2 * k + 1 < 9) {
      const float2 v1 = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
      u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v1.x, v1.y);
    }
  }
  return u;
}

// C_inv of a site: two blocks of 36 halves back to back in 9 uint4
__device__ __forceinline__ void cs_clover(const unsigned char* base, int site, Spinor<float>& psi) {
  const uint4* p = reinterpret_cast<const uint4*>(base) + site * CS_CLOV_U4;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    unsigned w[18];
    const uint2 mid = reinterpret_cast<const uint2*>(p + 4)[b];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 v = p[b == 0 ? k : 5 + k];
      const int o = b == 0 ? 4 * k : 2 + 4 * k;
      w[o] = v.x; w[o + 1] = v.y; w[o + 2] = v.z; w[o + 3] = v.w;
    }
    w[b == 0 ? 16 : 0] = mid.x;
    w[b == 0 ? 17 : 1] = mid.y;
    CloverBlockF32 blk;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
      blk.r[2 * k] = v.x;
      blk.r[2 * k + 1] = v.y;
    }
    cx<float> xin[6], y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) xin[i] = psi.v[2 * b + i / 3][i % 3];
    herm6_mul<float>(blk, xin, y);
#pragma unroll
    for (int i = 0; i < 6; ++i) psi.v[2 * b + i / 3][i % 3] = y[i];
  }
}

__device__ __forceinline__ void cs_load_x(const float4* buf, int slice, int s, Spinor<float>& a) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = buf[k * slice + s];
    a.v[(2 * k) / 3][(2 * k) % 3] = make_cx(v.x, v.y);
    a.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v.z, v.w);
  }
}
__device__ __forceinline__ void cs_store_x(float4* buf, int slice, int s, const Spinor<float>& a) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const cx<float> a0 = a.v[(2 * k) / 3][(2 * k) % 3], a1 = a.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
    buf[k * slice + s] = make_float4(a0.re, a0.im, a1.re, a1.im);
  }
}

template <int MU, int PM>
__device__ __forceinline__ void cs_hop(const SU3<float>& u, const Spinor<float>& p, float sign, Spinor<float>& acc) {
  HalfSpinor<float> h, uh;
  project<MU, PM>(p, h);
  if (PM < 0) su3_mul(u, h, uh);
  else su3_dag_mul(u, h, uh);
  accumulate<MU, PM>(acc, uh, sign);
}

// hops of direction MU (0..2) that stay in the slice
template <int MU>
__device__ __forceinline__ void cs_intra_space(const ClusterSapArgs& a, const float4* xb, const unsigned char* sl,
                                               const int lc[4], int s, Spinor<float>& acc) {
  const int stride = MU == 0 ? 1 : (MU == 1 ? a.sd[0] : a.sd[0] * a.sd[1]);
  if (lc[MU] < a.sd[MU] - 1) {
    Spinor<float> p;
    cs_load_x(xb, a.slice, s + stride, p);
    cs_hop<MU, -1>(cs_link(sl, a.slice, MU, s), p, 1.f, acc);
  }
  if (lc[MU] > 0) {
    Spinor<float> p;
    cs_load_x(xb, a.slice, s - stride, p);
    cs_hop<MU, +1>(cs_link(sl, a.slice, MU, s - stride), p, 1.f, acc);
  }
}

// hops that leave the domain (surface term): x of the other colour and the
// neighbouring domain's links from memory
template <int MU>
__device__ __forceinline__ void cs_inter(const ClusterSapArgs& a, const unsigned char* sl, const int X[4],
                                         const int lc[4], int s, Spinor<float>& acc) {
  const Geom& g = a.g;
  int Y[4] = {X[0], X[1], X[2], X[3]};
  if (lc[MU] == a.sd[MU] - 1) {
    Y[MU] = X[MU] + 1 == g.L[MU] ? 0 : X[MU] + 1;
    const float sign = (MU == 3 && X[3] + 1 == g.L[3]) ? (float)g.bc_t : 1.f;
    int nd, ns;
    coords_to_internal(g, Y, nd, ns);
    Spinor<float> p;
    a.x.load(g, nd, ns, p);
    cs_hop<MU, -1>(cs_link(sl, a.slice, MU, s), p, sign, acc);
    Y[MU] = X[MU];
  }
  if (lc[MU] == 0) {
    Y[MU] = X[MU] == 0 ? g.L[MU] - 1 : X[MU] - 1;
    const float sign = (MU == 3 && X[3] == 0) ? (float)g.bc_t : 1.f;
    int nd, ns;
    coords_to_internal(g, Y, nd, ns);
    Spinor<float> p;
    a.x.load(g, nd, ns, p);
    SU3<float> u;
    a.U16.load(g, nd, MU, ns, u);
    cs_hop<MU, +1>(u, p, sign, acc);
  }
}

__device__ __forceinline__ bool cs_wait(uint64_t* bar) {
  unsigned ok = 0;
  const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(bar));
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int i = 0; i < (1 << 24); ++i) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr)
        : "memory");
    if (ok) return true;
    if ((i & 255) == 255) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 500000000ull) return false;
    }
  }
  return false;
}

__global__ void __launch_bounds__(CS_MAX_SLICE, 1) sap_cluster_kernel(ClusterSapArgs a) {
  extern __shared__ __align__(128) unsigned char csm[];
  const Geom& g = a.g;
  cg::cluster_group cl = cg::this_cluster();
  const int K = a.sd[3];
  const int lt = (int)cl.block_rank();  // time slice of this CTA
  const int S = a.slice;
  float4* xbuf0 = reinterpret_cast<float4*>(csm);
  float4* xbuf1 = xbuf0 + 6 * S;
  unsigned char* sl = csm + 2 * 96 * S;          // links
  unsigned char* sc = sl + 4 * CS_LINK_H2 * 4 * S;  // C_inv
  uint64_t* bar = reinterpret_cast<uint64_t*>(sc + CS_CLOV_U4 * 16 * S);
  int* bad = reinterpret_cast<int*>(bar + 1);
  // the same decision in every CTA of the cluster: the flag was written before this launch
  if (loop_idle(g)) return;
  const int tid = threadIdx.x;
  const bool live = tid < S;
  const int s = live ? tid : 0;
  // this cluster's domain: the k-th domain of colour a.colour (see sap_general.cu)
  int D[4];
  {
    const int per = a.snd[0] / 2, k = (int)blockIdx.x / K;
    const int row = k / per, i = k - row * per;
    D[1] = row % a.snd[1];
    D[2] = (row / a.snd[1]) % a.snd[2];
    D[3] = row / (a.snd[1] * a.snd[2]);
    D[0] = 2 * i + ((a.colour + D[1] + D[2] + D[3]) & 1);
  }
  const long long jd = ((long long)(D[3] * a.snd[2] + D[2]) * a.snd[1] + D[1]) * a.snd[0] + D[0];
  const size_t slice_id = (size_t)jd * K + lt;
  if (tid == 0) {
    const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(bar));
    const unsigned lbytes = 4 * CS_LINK_H2 * 4 * S, cbytes = CS_CLOV_U4 * 16 * S;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(addr) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr),
                 "r"(lbytes + cbytes + a.extra_tx)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(sl))),
                 "l"(a.links + slice_id * lbytes), "r"(lbytes), "r"(addr)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(sc))),
                 "l"(a.clov + slice_id * cbytes), "r"(cbytes), "r"(addr)
                 : "memory");
  }
  int lc[4], X[4];
  lc[0] = s % a.sd[0];
  lc[1] = (s / a.sd[0]) % a.sd[1];
  lc[2] = s / (a.sd[0] * a.sd[1]);
  lc[3] = lt;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) X[mu] = D[mu] * a.sd[mu] + lc[mu];
  int dom, st;
  coords_to_internal(g, X, dom, st);
  Spinor<float> src;
  if (live) a.s_in.load(g, dom, st, src);
  __syncthreads();  // barrier initialisation visible to every thread
  {
    // every CTA of the cluster takes the same decision on a wait that gave up
    const bool ok = cs_wait(bar);
    const int cta_bad = __syncthreads_or(!ok);
    if (tid == 0) *bad = cta_bad;
    cl.sync();
    int any = 0;
    for (int r = 0; r < K; ++r) any |= *cl.map_shared_rank(bad, r);
    if (any) {
      if (tid == 0) atomicExch(a.status, QCD_ERR_TIMEOUT);
      if (cta_bad) cs_wait(bar);
      cl.sync();
      return;
    }
  }
  Spinor<float> acc;
  if (a.do_surface && live) {
    zero(acc);
    cs_inter<0>(a, sl, X, lc, s, acc);
    cs_inter<1>(a, sl, X, lc, s, acc);
    cs_inter<2>(a, sl, X, lc, s, acc);
    if (lt == K - 1 || lt == 0) cs_inter<3>(a, sl, X, lc, s, acc);
    cs_clover(sc, s, acc);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        src.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, src.v[sp][c].re);
        src.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, src.v[sp][c].im);
      }
  }
  if (live) cs_store_x(xbuf0, S, s, src);
  cl.sync();  // every slice holds x_0
  int cur = 0;
  Spinor<float> xk = src;  // this site's current iterate
  const int napp = a.n_jac + (a.do_update ? 1 : 0);
  for (int it = 0; it < napp; ++it) {
    float4* xb = cur ? xbuf1 : xbuf0;
    float4* xnb = cur ? xbuf0 : xbuf1;
    if (live) {
      zero(acc);
      cs_intra_space<0>(a, xb, sl, lc, s, acc);
      cs_intra_space<1>(a, xb, sl, lc, s, acc);
      cs_intra_space<2>(a, xb, sl, lc, s, acc);
      // t hops: the neighbouring slices' x (and, backward, their links)
      // through distributed shared memory
      if (lt < K - 1) {
        const float4* rx = cl.map_shared_rank(xb, lt + 1);
        Spinor<float> p;
        cs_load_x(rx, S, s, p);
        cs_hop<3, -1>(cs_link(sl, S, 3, s), p, 1.f, acc);
      }
      if (lt > 0) {
        const float4* rx = cl.map_shared_rank(xb, lt - 1);
        const unsigned char* rl = cl.map_shared_rank(sl, lt - 1);
        Spinor<float> p;
        cs_load_x(rx, S, s, p);
        cs_hop<3, +1>(cs_link(rl, S, 3, s), p, 1.f, acc);
      }
      cs_clover(sc, s, acc);
      if (it < a.n_jac) {
        // x_k = s + kappa C_inv H_cc x_{k-1}
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            xk.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, src.v[sp][c].re);
            xk.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, src.v[sp][c].im);
          }
        cs_store_x(xnb, S, s, xk);
      } else {
        // s + b - x + kappa C_inv H_cc x
        Spinor<float> b;
        a.b.load(g, dom, st, b);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float re = src.v[sp][c].re + b.v[sp][c].re - xk.v[sp][c].re;
            const float im = src.v[sp][c].im + b.v[sp][c].im - xk.v[sp][c].im;
            acc.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, re);
            acc.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, im);
          }
        a.s_out.store(g, dom, st, acc);
      }
    }
    if (it < a.n_jac) {
      cl.sync();  // every slice has read the old buffer and written the new one
      cur ^= 1;
    }
  }
  if (live) a.x.store(g, dom, st, xk);
  cl.sync();  // the neighbours' last reads of this CTA's shared memory are done
}

// ---------------------------------------------------------------------------
// staging layout and launches
// ---------------------------------------------------------------------------
// one thread per site: its links and C_inv, float16, into the domain-slice
// staging layout [domain][slice][mu][site][10 half2] and [domain][slice][site][9 uint4]
__global__ void build_cluster_stage_kernel(Geom g, int sd0, int sd1, int sd2, int sd3, int snd0, int snd1,
                                           int snd2, const double2* u64, const double2* cinv64, __half2* l16,
                                           __half2* c16) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.vol) return;
  int X[4];
  site_coords(g, n, X);
  int dom, s;
  coords_to_internal(g, X, dom, s);
  const int sd[4] = {sd0, sd1, sd2, sd3};
  int D[4], l[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    D[mu] = X[mu] / sd[mu];
    l[mu] = X[mu] - D[mu] * sd[mu];
  }
  const int S = sd0 * sd1 * sd2;
  const long long jd = ((long long)(D[3] * snd2 + D[2]) * snd1 + D[1]) * snd0 + D[0];
  const size_t slice_id = (size_t)jd * sd3 + l[3];
  const int site = l[0] + sd0 * (l[1] + sd1 * l[2]);
  for (int mu = 0; mu < 4; ++mu) {
    __half2* dst = l16 + slice_id * 4 * S * CS_LINK_H2 + ((size_t)mu * S + site) * CS_LINK_H2;
    for (int e = 0; e < 9; ++e) {
      const double2 v = u64[(((size_t)((dom * 4 + mu) * 9 + e)) << g.logvd) + s];
      dst[e] = __floats2half2_rn((float)v.x, (float)v.y);
    }
    dst[9] = __floats2half2_rn(0.f, 0.f);
  }
  __half2* h = c16 + (slice_id * S + site) * (CS_CLOV_U4 * 4);
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 18; ++k) {
      const double2 v = cinv64[(((size_t)(dom * 36 + 18 * b + k)) << g.logvd) + s];
      h[18 * b + k] = __floats2half2_rn((float)v.x, (float)v.y);
    }
}

// a domain whose time slices fit the cluster kernel: at most CS_MAX_K
// slices of at most CS_MAX_SLICE sites
bool sap_cluster_fits(const int d[4]) {
  const long long S = (long long)d[0] * d[1] * d[2];
  return d[3] >= 1 && d[3] <= CS_MAX_K && S >= 1 && S <= CS_MAX_SLICE;
}

bool sap_cluster_eligible(const qcd_ctx* ctx, int sap_prec) {
  if (!ctx->sap_general || sap_prec != QCD_PREC_HALF_GAUGE) return false;
  return sap_cluster_fits(ctx->sap_dom);
}

// build (or rebuild after a new clover term or domain) the staging copy
static void cluster_staging(qcd_ctx* ctx, cudaStream_t st) {
  const int* d = ctx->sap_dom;
  bool same = ctx->cl_gen == ctx->clover_gen && ctx->cl_link && ctx->cl_clov;
  for (int mu = 0; mu < 4; ++mu) same = same && ctx->cl_dom[mu] == d[mu];
  if (same) return;
  const Geom& g = ctx->geom;
  if (!ctx->cl_link) {
    QCD_CUDA_CHECK(cudaMalloc(&ctx->cl_link, (size_t)g.vol * 4 * CS_LINK_H2 * sizeof(__half2)));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->cl_clov, (size_t)g.vol * CS_CLOV_U4 * 16));
  }
  LaunchScope ls(ctx, QCD_KC_OTHER, st);
  build_cluster_stage_kernel<<<grid_for(g.vol, 128), 128, 0, st>>>(
      g, d[0], d[1], d[2], d[3], g.L[0] / d[0], g.L[1] / d[1], g.L[2] / d[2], ctx->u64, ctx->cinv64,
      (__half2*)ctx->cl_link, (__half2*)ctx->cl_clov);
  check_launch();
  for (int mu = 0; mu < 4; ++mu) ctx->cl_dom[mu] = d[mu];
  ctx->cl_gen = ctx->clover_gen;
}

// M_SAP with one cluster per domain, nrhs stacked float32 fields
void sap_cluster_apply(qcd_ctx* ctx, float4* x, const float4* b, int nrhs, int n_sap, int n_jac, void* ws_s,
                       cudaStream_t st) {
  cluster_staging(ctx, st);
  ClusterSapArgs a;
  a.g = ctx->geom;
  long long nsd = 1;
  for (int mu = 0; mu < 4; ++mu) {
    a.sd[mu] = ctx->sap_dom[mu];
    a.snd[mu] = a.g.L[mu] / a.sd[mu];
    nsd *= a.snd[mu];
  }
  a.slice = a.sd[0] * a.sd[1] * a.sd[2];
  a.n_jac = n_jac;
  a.kappa = (float)ctx->kappa;
  a.U16 = LinkPtrHalf{ctx->u16};
  a.links = (const unsigned char*)ctx->cl_link;
  a.clov = (const unsigned char*)ctx->cl_clov;
  a.status = ctx->d_status;
  // test hook: wait for 16 bytes that no copy brings, so that the bounded
  // wait gives up (in every CTA of every cluster) and reports QCD_ERR_TIMEOUT
  a.extra_tx = ctx->inject == QCD_INJECT_STAGING_WAIT ? 16 : 0;
  const int K = a.sd[3];
  const int threads = (a.slice + 31) / 32 * 32;
  const size_t smem = (size_t)CS_BYTES_PER_SITE * a.slice + 16;
  QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)CS_BYTES_PER_SITE * CS_MAX_SLICE + 16)));
  const size_t v4 = (size_t)a.g.vol * 6;
  for (int r = 0; r < nrhs; ++r) {
    a.b = F32Spinor{(float4*)b + r * v4};
    a.x = F32Spinor{x + r * v4};
    a.s_out = F32Spinor{(float4*)ws_s + r * v4};
    for (int sweep = 0; sweep <= n_sap; ++sweep) {
      a.s_in = sweep == 0 ? a.b : a.s_out;
      a.do_update = sweep == n_sap ? 0 : 1;
      for (int colour = 0; colour < 2; ++colour) {
        a.colour = colour;
        a.do_surface = (sweep == 0 && colour == 0) ? 0 : 1;
        LaunchScope ls(ctx, QCD_KC_SAP_BLOCK, st);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nsd / 2 * K));
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        QCD_CUDA_CHECK(cudaLaunchKernelEx(&cfg, sap_cluster_kernel, a));
        check_launch();
      }
    }
  }
}

}  // namespace qcd
