// SAP preconditioner (Sec. 3 of arXiv:2109.10687, Algorithms 1 and 2) on
// domains of any extents, such as the paper's 16x6x4x3 domains (Sec. 4.3,
// Tables 2-3), independent of the power-of-two blocking the fields are
// stored in.
//
// One CTA per SAP domain of the colour being swept, 384 threads, each
// thread the sites l = tid, tid + 384, tid + 768 of the domain's local
// numbering l = x + d0 (y + d1 (z + d2 t)).  A site's storage position
// (storage domain, site) follows from its global coordinates.  Shared
// memory holds the domain's source s (after the surface term) and its
// Jacobi iterate x, float32, 96 bytes per site each: up to 1152 sites
// (221 KB).  Links and C_inv are read through L1/L2 from the context's
// internal layouts.  Per launch:
//   1. surface term: s <- s + kappa C_inv H_{c c'} x_{c'}, the hops that
//      leave the domain reading the other colour's x from memory;
//   2. n_jac Jacobi sweeps x_k = s + kappa C_inv H_cc x_{k-1} (x_0 = s),
//      each computing every site's new x in registers before one barrier
//      and the store (the old x stays intact while neighbours read it);
//   3. the residual update s <- s + b - x + kappa C_inv H_cc x (skipped in
//      the closing sweep);
//   4. x of this colour written back to memory.
// The hops that stay inside the domain branch on the local coordinate (the
// domain's sites are spread over the warps without regard to direction).

#include <cstdio>

#include "qcd_internal.cuh"

namespace qcd {

constexpr int GS_THREADS = 384;
constexpr int GS_SPT = 3;
constexpr int GS_MAX_SITES = GS_THREADS * GS_SPT;  // 1152

template <typename LP, typename CP>
struct GenSapArgs {
  Geom g;         // storage geometry
  int sd[4];      // SAP domain extents
  int snd[4];     // SAP domains per direction
  int svol;       // sites per SAP domain
  int colour, n_jac, do_surface, do_update;
  float kappa;
  F32Spinor s_in, s_out, x, b;
  LP U;
  CP cinv;
};

// x in shared memory: float4 [6][svol] (component group k of local site l at k svol + l)
__device__ __forceinline__ void gs_load(const float4* sm, int svol, int l, Spinor<float>& a) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = sm[k * svol + l];
    a.v[(2 * k) / 3][(2 * k) % 3] = make_cx(v.x, v.y);
    a.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v.z, v.w);
  }
}
__device__ __forceinline__ void gs_store(float4* sm, int svol, int l, const Spinor<float>& a) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const cx<float> a0 = a.v[(2 * k) / 3][(2 * k) % 3], a1 = a.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
    sm[k * svol + l] = make_float4(a0.re, a0.im, a1.re, a1.im);
  }
}

// storage position of global coordinates x (each already in [0, L))
__device__ __forceinline__ void gs_storage(const Geom& g, const int x[4], int& dom, int& s) {
  coords_to_internal(g, x, dom, s);
}

// acc += the hop of direction MU, sign PM (-1 forward: (1 - gamma) U(n) x(n+mu),
// +1 backward: (1 + gamma) U(n-mu)^dag x(n-mu)), operand p, link at storage (ldom, ls)
template <int MU, int PM, typename LP>
__device__ __forceinline__ void gs_hop(const Geom& g, const LP& U, int ldom, int ls, const Spinor<float>& p,
                                       float sign, Spinor<float>& acc) {
  HalfSpinor<float> h, uh;
  project<MU, PM>(p, h);
  SU3<float> u;
  U.load(g, ldom, MU, ls, u);
  if (PM < 0) su3_mul(u, h, uh);
  else su3_dag_mul(u, h, uh);
  accumulate<MU, PM>(acc, uh, sign);
}

// The hops of direction MU of site (global X, local lc, storage dom/s):
// INTRA: those that stay in the domain (operand from shared memory), else
// those that leave it (operand x from memory, boundary sign in t).
template <int MU, bool INTRA, typename LP, typename CP>
__device__ __forceinline__ void gs_dir(const GenSapArgs<LP, CP>& a, const float4* sx, const int X[4],
                                       const int D[4], int l, int dom, int s, Spinor<float>& acc) {
  const Geom& g = a.g;
  int stride = 1;
#pragma unroll
  for (int nu = 0; nu < MU; ++nu) stride *= a.sd[nu];
  const int lc = X[MU] - D[MU] * a.sd[MU];  // local coordinate
  const bool fwd_in = lc < a.sd[MU] - 1, bwd_in = lc > 0;
  int Y[4] = {X[0], X[1], X[2], X[3]};
  if (INTRA ? fwd_in : !fwd_in) {
    Spinor<float> p;
    float sign = 1.f;
    if (INTRA) {
      gs_load(sx, a.svol, l + stride, p);
    } else {
      Y[MU] = X[MU] + 1 == g.L[MU] ? 0 : X[MU] + 1;
      if (MU == 3 && X[3] + 1 == g.L[3]) sign = (float)g.bc_t;
      int nd, ns;
      gs_storage(g, Y, nd, ns);
      a.x.load(g, nd, ns, p);
      Y[MU] = X[MU];
    }
    gs_hop<MU, -1>(g, a.U, dom, s, p, sign, acc);
  }
  if (INTRA ? bwd_in : !bwd_in) {
    Spinor<float> p;
    float sign = 1.f;
    Y[MU] = X[MU] == 0 ? g.L[MU] - 1 : X[MU] - 1;
    if (!INTRA && MU == 3 && X[3] == 0) sign = (float)g.bc_t;
    int nd, ns;
    gs_storage(g, Y, nd, ns);
    if (INTRA) gs_load(sx, a.svol, l - stride, p);
    else a.x.load(g, nd, ns, p);
    gs_hop<MU, +1>(g, a.U, nd, ns, p, sign, acc);
  }
}

template <bool INTRA, typename LP, typename CP>
__device__ __forceinline__ void gs_hops(const GenSapArgs<LP, CP>& a, const float4* sx, const int X[4],
                                        const int D[4], int l, int dom, int s, Spinor<float>& acc) {
  gs_dir<0, INTRA>(a, sx, X, D, l, dom, s, acc);
  gs_dir<1, INTRA>(a, sx, X, D, l, dom, s, acc);
  gs_dir<2, INTRA>(a, sx, X, D, l, dom, s, acc);
  gs_dir<3, INTRA>(a, sx, X, D, l, dom, s, acc);
}

template <typename LP, typename CP, typename CB>
__global__ void __launch_bounds__(GS_THREADS, 1) sap_general_kernel(GenSapArgs<LP, CP> a) {
  extern __shared__ __align__(16) float4 gsm[];
  float4* sx = gsm;                  // x iterate
  float4* ss = gsm + 6 * a.svol;     // source after the surface term
  const Geom& g = a.g;
  if (loop_idle(g)) return;
  // this CTA's domain: the blockIdx.x-th domain of colour a.colour; with an
  // even number of domains along x, every row of domains along x holds
  // snd[0] / 2 domains of each colour
  int D[4];
  {
    const int per = a.snd[0] / 2, k = blockIdx.x;
    const int row = k / per, i = k - row * per;
    D[1] = row % a.snd[1];
    D[2] = (row / a.snd[1]) % a.snd[2];
    D[3] = row / (a.snd[1] * a.snd[2]);
    D[0] = 2 * i + ((a.colour + D[1] + D[2] + D[3]) & 1);
  }
  const int tid = threadIdx.x;
  int X[GS_SPT][4], dom[GS_SPT], st[GS_SPT];
#pragma unroll
  for (int j = 0; j < GS_SPT; ++j) {
    const int l = tid + j * GS_THREADS;
    int r = l < a.svol ? l : 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int lc = mu < 3 ? r % a.sd[mu] : r;
      r = mu < 3 ? r / a.sd[mu] : 0;
      X[j][mu] = D[mu] * a.sd[mu] + lc;
    }
    gs_storage(g, X[j], dom[j], st[j]);
  }
  // 1. source and surface term
#pragma unroll
  for (int j = 0; j < GS_SPT; ++j) {
    const int l = tid + j * GS_THREADS;
    if (l >= a.svol) continue;
    Spinor<float> src;
    a.s_in.load(g, dom[j], st[j], src);
    if (a.do_surface) {
      Spinor<float> acc;
      zero(acc);
      gs_hops<false>(a, sx, X[j], D, l, dom[j], st[j], acc);
      clover_mul<float, CP, CB>(a.cinv, g, dom[j], st[j], acc);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          src.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, src.v[sp][c].re);
          src.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, src.v[sp][c].im);
        }
    }
    gs_store(ss, a.svol, l, src);
    gs_store(sx, a.svol, l, src);
  }
  __syncthreads();
  // 2.-3. Jacobi sweeps, then one more application of H_cc for the update
  const int napp = a.n_jac + (a.do_update ? 1 : 0);
  for (int it = 0; it < napp; ++it) {
    Spinor<float> xn[GS_SPT];
#pragma unroll
    for (int j = 0; j < GS_SPT; ++j) {
      const int l = tid + j * GS_THREADS;
      if (l >= a.svol) continue;
      Spinor<float> acc;
      zero(acc);
      gs_hops<true>(a, sx, X[j], D, l, dom[j], st[j], acc);
      clover_mul<float, CP, CB>(a.cinv, g, dom[j], st[j], acc);
      Spinor<float> src;
      gs_load(ss, a.svol, l, src);
      if (it < a.n_jac) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            xn[j].v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, src.v[sp][c].re);
            xn[j].v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, src.v[sp][c].im);
          }
      } else {
        // s + b - x + kappa C_inv H_cc x
        Spinor<float> b, xc;
        a.b.load(g, dom[j], st[j], b);
        gs_load(sx, a.svol, l, xc);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float re = src.v[sp][c].re + b.v[sp][c].re - xc.v[sp][c].re;
            const float im = src.v[sp][c].im + b.v[sp][c].im - xc.v[sp][c].im;
            acc.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, re);
            acc.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, im);
          }
        a.s_out.store(g, dom[j], st[j], acc);
      }
    }
    if (it < a.n_jac) {
      __syncthreads();  // every neighbour read of the old x is done
#pragma unroll
      for (int j = 0; j < GS_SPT; ++j) {
        const int l = tid + j * GS_THREADS;
        if (l < a.svol) gs_store(sx, a.svol, l, xn[j]);
      }
      __syncthreads();
    }
  }
  // 4. this colour's x
#pragma unroll
  for (int j = 0; j < GS_SPT; ++j) {
    const int l = tid + j * GS_THREADS;
    if (l >= a.svol) continue;
    Spinor<float> xc;
    gs_load(sx, a.svol, l, xc);
    a.x.store(g, dom[j], st[j], xc);
  }
}

template <typename LP, typename CP, typename CB>
static void general_sequence(qcd_ctx* ctx, F32Spinor s_first_in, F32Spinor s, F32Spinor x, F32Spinor b, LP U,
                             CP cinv, int n_sap, int n_jac, cudaStream_t st) {
  GenSapArgs<LP, CP> a;
  a.g = ctx->geom;
  long long nsd = 1;
  a.svol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    a.sd[mu] = ctx->sap_dom[mu];
    a.snd[mu] = a.g.L[mu] / a.sd[mu];
    a.svol *= a.sd[mu];
    nsd *= a.snd[mu];
  }
  a.n_jac = n_jac;
  a.kappa = (float)ctx->kappa;
  a.b = b;
  a.x = x;
  a.s_out = s;
  a.U = U;
  a.cinv = cinv;
  const size_t smem = (size_t)12 * a.svol * sizeof(float4);
  QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_general_kernel<LP, CP, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)12 * GS_MAX_SITES * sizeof(float4))));
  for (int sweep = 0; sweep <= n_sap; ++sweep) {
    a.s_in = sweep == 0 ? s_first_in : s;
    a.do_update = sweep == n_sap ? 0 : 1;
    for (int colour = 0; colour < 2; ++colour) {
      a.colour = colour;
      a.do_surface = (sweep == 0 && colour == 0) ? 0 : 1;
      LaunchScope ls(ctx, QCD_KC_SAP_BLOCK, st);
      sap_general_kernel<LP, CP, CB><<<(unsigned)(nsd / 2), GS_THREADS, smem, st>>>(a);
      check_launch();
    }
  }
}

bool sap_general_fits(const int sdom[4]) {
  return (long long)sdom[0] * sdom[1] * sdom[2] * sdom[3] <= GS_MAX_SITES;
}

// every extent divides the lattice into an even number of domains, and the
// domain fits the one-CTA kernel or the cluster kernel
bool sap_domain_valid(const int dims[4], const int sdom[4]) {
  for (int mu = 0; mu < 4; ++mu)
    if (sdom[mu] < 1 || dims[mu] % (2 * sdom[mu])) return false;
  return sap_general_fits(sdom) || sap_cluster_fits(sdom);
}

// M_SAP for nrhs stacked float32 fields with the context's general SAP
// domains; float32 (sap_prec SINGLE) or float16 links and C_inv with float32
// vectors (HALF_GAUGE).  ws_s holds s (float32), one field per rhs.  With
// float16 links and C_inv and domains whose time slices fit a CTA, the
// cluster kernel (sap_cluster.cu, shape 0) and this one (shape 1) are both
// available and the autotuner picks one; otherwise this kernel runs.
static const char* const kGeneralShapes[] = {"cluster_per_domain", "cta_per_domain"};

void sap_general_apply(qcd_ctx* ctx, float4* x, const float4* b, int nrhs, int n_sap, int n_jac, int sap_prec,
                       void* ws_s, cudaStream_t st) {
  QCD_REQUIRE(sap_prec == QCD_PREC_SINGLE || sap_prec == QCD_PREC_HALF_GAUGE, QCD_ERR_ARG,
              "SAP on general domains: sap_prec must be SINGLE or HALF_GAUGE");
  const bool can_cluster = sap_cluster_eligible(ctx, sap_prec);
  const bool can_cta = sap_general_fits(ctx->sap_dom);
  QCD_REQUIRE(can_cta || can_cluster, QCD_ERR_ARG,
              "SAP on general domains: domains above 1152 sites run on the cluster kernel only (sap_prec HALF_GAUGE)");
  QCD_REQUIRE(can_cta || ctx->sap_shape <= 0, QCD_ERR_ARG,
              "SAP on general domains: domains above 1152 sites need the cluster shape (0 or autotuned)");
  const size_t v4 = (size_t)ctx->geom.vol * 6;
  auto run = [&](int v) {
    if (v == 0 && can_cluster) {
      sap_cluster_apply(ctx, x, b, nrhs, n_sap, n_jac, ws_s, st);
      return;
    }
    for (int r = 0; r < nrhs; ++r) {
      F32Spinor xs{x + r * v4}, bs{(float4*)b + r * v4}, ss{(float4*)ws_s + r * v4};
      if (sap_prec == QCD_PREC_SINGLE)
        general_sequence<LinkPtr<float>, CloverPtrF32, CloverBlockF32>(ctx, bs, ss, xs, bs, LinkPtr<float>{ctx->u32},
                                                                       CloverPtrF32{ctx->cinv32}, n_sap, n_jac, st);
      else
        general_sequence<LinkPtrHalf, CloverPtrF16, CloverBlockF32>(ctx, bs, ss, xs, bs, LinkPtrHalf{ctx->u16},
                                                                     CloverPtrF16{ctx->cinv16}, n_sap, n_jac, st);
    }
  };
  int v = ctx->sap_shape;
  if (v < 0 && !can_cta) v = 0;
  if (v < 0) {
    if (can_cluster) {
      const Geom& g = ctx->geom;
      char key[160];
      std::snprintf(key, sizeof key, "sap_general_f16gauge L%dx%dx%dx%d dom%dx%dx%dx%d nrhs%d n_sap%d n_jac%d", g.L[0],
                    g.L[1], g.L[2], g.L[3], ctx->sap_dom[0], ctx->sap_dom[1], ctx->sap_dom[2], ctx->sap_dom[3], nrhs,
                    n_sap, n_jac);
      v = tune_pick(ctx, key, 2, kGeneralShapes, run, st);
    } else {
      v = 1;
    }
  }
  run(v);
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_set_sap_domain(qcd_ctx* ctx, const int sdom[4]) {
  if (!ctx) return QCD_ERR_ARG;
  workspace_reset_graphs(ctx);
  if (!sdom) {
    ctx->sap_general = false;
    return QCD_OK;
  }
  if (!sap_domain_valid(ctx->geom.L, sdom)) {
    ctx->err = "qcd_set_sap_domain: every L_mu must be a multiple of 2 d_mu, and a domain at most 1152 sites or "
               "at most 8 time slices of at most 448 sites";
    return QCD_ERR_ARG;
  }
  for (int mu = 0; mu < 4; ++mu) ctx->sap_dom[mu] = sdom[mu];
  ctx->sap_general = true;
  return QCD_OK;
}
