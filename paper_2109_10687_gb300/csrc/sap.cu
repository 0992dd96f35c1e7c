// SAP preconditioner with Jacobi domain inverses (Sec. 3 of
// arXiv:2109.10687: Eq. Msap, Algorithms 1-3).
//
// One kernel launch performs one half-sweep of Algorithm 1 on every domain
// of one colour c (E = 0, O = 1), one CTA per 256/vd domains, one thread per
// site:
//
//   1. surface term (skipped in the first E half-sweep, where x_O = 0):
//        s_c <- s_c - A_{c,c'} x_{c'} = s_c + kappa C_inv H_{c c'} x_{c'}
//      reading the neighbouring domains' x straight from memory (the GPU
//      counterpart of the halo exchange of Sec. 4.1);
//   2. Jacobi domain inverse (Algorithm 2) with the iterate kept in shared
//      memory:  x_0 = s_c,  x_k = s_c + kappa C_inv H_cc x_{k-1}, k = 1..n_jac.
//      This is Algorithm 2 written without the cancelling terms
//      (x + b - (x - kappa C_inv H x) = b + kappa C_inv H x), so
//      x_{n_jac} = sum_{j=0}^{n_jac} (I - A_cc)^j s_c;
//   3. residual update of Algorithm 1 (skipped in the closing sweep):
//        s_c <- s_c + b_c - A_cc x_c = s_c + b_c - x_c + kappa C_inv H_cc x_c.
//
// The whole preconditioner is 2 (n_sap + 1) such launches; A M_SAP adds one
// application of A to the result (Algorithm 3 as A (M_SAP b)).

#include "qcd_internal.cuh"

namespace qcd {

constexpr int SAP_THREADS = 256;

// x in shared memory: float4 [6][SAP_THREADS]
__device__ __forceinline__ void smem_load(const float4* sx, int slot, Spinor<float>& a) {
  float f[24];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = sx[k * SAP_THREADS + slot];
    f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
  }
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) a.v[sp][c] = make_cx(f[(sp * 3 + c) * 2], f[(sp * 3 + c) * 2 + 1]);
}
__device__ __forceinline__ void smem_store(float4* sx, int slot, const Spinor<float>& a) {
  float f[24];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) { f[(sp * 3 + c) * 2] = a.v[sp][c].re; f[(sp * 3 + c) * 2 + 1] = a.v[sp][c].im; }
#pragma unroll
  for (int k = 0; k < 6; ++k) sx[k * SAP_THREADS + slot] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// acc += hops of direction MU that stay inside the domain, operand from smem
template <int MU, typename LP>
__device__ __forceinline__ void intra_dir(const Geom& g, const float4* sx, int slot0, const LP& U, int dom, int s,
                                          Spinor<float>& acc) {
  const int c = (s >> g.shift[MU]) & (g.d[MU] - 1);
  const int step = 1 << g.shift[MU];
  if (c < g.d[MU] - 1) {
    Spinor<float> p;
    smem_load(sx, slot0 + s + step, p);
    HalfSpinor<float> h, uh;
    project<MU, -1>(p, h);
    SU3<float> u;
    U.load(g, dom, MU, s, u);
    su3_mul(u, h, uh);
    accumulate<MU, -1>(acc, uh);
  }
  if (c > 0) {
    Spinor<float> p;
    smem_load(sx, slot0 + s - step, p);
    HalfSpinor<float> h, uh;
    project<MU, +1>(p, h);
    SU3<float> u;
    U.load(g, dom, MU, s - step, u);
    su3_dag_mul(u, h, uh);
    accumulate<MU, +1>(acc, uh);
  }
}

// acc += hops of direction MU that leave the domain, operand x from memory
template <int MU, typename SIO, typename LP>
__device__ __forceinline__ void inter_dir(const Geom& g, const SIO& x, const LP& U, int dom, int s,
                                          Spinor<float>& acc) {
  const int c = (s >> g.shift[MU]) & (g.d[MU] - 1);
  if (c == g.d[MU] - 1) {
    int nd, ns;
    const int sign = nbr_site(g, dom, s, MU, true, nd, ns);
    Spinor<float> p;
    x.load(g, nd, ns, p);
    HalfSpinor<float> h, uh;
    project<MU, -1>(p, h);
    SU3<float> u;
    U.load(g, dom, MU, s, u);
    su3_mul(u, h, uh);
    if (sign < 0) scale_half(uh, -1.0f);
    accumulate<MU, -1>(acc, uh);
  }
  if (c == 0) {
    int nd, ns;
    const int sign = nbr_site(g, dom, s, MU, false, nd, ns);
    Spinor<float> p;
    x.load(g, nd, ns, p);
    HalfSpinor<float> h, uh;
    project<MU, +1>(p, h);
    SU3<float> u;
    U.load(g, nd, MU, ns, u);
    su3_dag_mul(u, h, uh);
    if (sign < 0) scale_half(uh, -1.0f);
    accumulate<MU, +1>(acc, uh);
  }
}

template <typename SIO, typename LP, typename CP>
struct SapArgs {
  Geom g;
  int colour;
  int n_jac;
  int do_surface;
  int do_update;
  float kappa;
  SIO s_in;       // s before this half-sweep (may be the source b in the first sweep)
  SIO s_out;      // s after the residual update
  SIO x;          // x of both colours (read: other colour, written: this colour)
  F32Spinor b;    // source of M_SAP
  LP U;
  CP cinv;
};

template <typename SIO, typename LP, typename CP, typename CB>
__global__ void __launch_bounds__(SAP_THREADS) sap_block_kernel(SapArgs<SIO, LP, CP> a) {
  __shared__ float4 sx[6 * SAP_THREADS];
  const Geom& g = a.g;
  if (loop_idle(g)) return;
  const int t = threadIdx.x;
  const int per_cta = SAP_THREADS >> g.logvd;           // domains per CTA
  const int local = t >> g.logvd;
  const int s = t & (g.vd - 1);
  const int k = blockIdx.x * per_cta + local;             // domain index within the colour
  const bool active = k < g.nhalf;
  const int dom = a.colour * g.nhalf + (active ? k : 0);
  const int slot0 = local << g.logvd;

  Spinor<float> src;  // s_c after the surface term
  if (active) {
    a.s_in.load(g, dom, s, src);
    if (a.do_surface) {
      Spinor<float> acc;
      zero(acc);
      inter_dir<0>(g, a.x, a.U, dom, s, acc);
      inter_dir<1>(g, a.x, a.U, dom, s, acc);
      inter_dir<2>(g, a.x, a.U, dom, s, acc);
      inter_dir<3>(g, a.x, a.U, dom, s, acc);
      clover_mul<float, CP, CB>(a.cinv, g, dom, s, acc);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          src.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, src.v[sp][c].re);
          src.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, src.v[sp][c].im);
        }
    }
    smem_store(sx, t, src);
  }
  __syncthreads();

  // Jacobi sweeps (plus one more application of H_cc for the residual update)
  Spinor<float> xk = src;
  const int napp = a.n_jac + (a.do_update ? 1 : 0);
  for (int it = 0; it < napp; ++it) {
    Spinor<float> acc;
    zero(acc);
    if (active) {
      intra_dir<0>(g, sx, slot0, a.U, dom, s, acc);
      intra_dir<1>(g, sx, slot0, a.U, dom, s, acc);
      intra_dir<2>(g, sx, slot0, a.U, dom, s, acc);
      intra_dir<3>(g, sx, slot0, a.U, dom, s, acc);
      clover_mul<float, CP, CB>(a.cinv, g, dom, s, acc);
    }
    if (it < a.n_jac) {
      // x_{k} = s_c + kappa C_inv H_cc x_{k-1}
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xk.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, src.v[sp][c].re);
          xk.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, src.v[sp][c].im);
        }
      __syncthreads();
      if (active) smem_store(sx, t, xk);
      __syncthreads();
    } else if (active) {
      // s_c + b_c - x_c + kappa C_inv H_cc x_c
      Spinor<float> b;
      a.b.load(g, dom, s, b);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float re = src.v[sp][c].re + b.v[sp][c].re - xk.v[sp][c].re;
          float im = src.v[sp][c].im + b.v[sp][c].im - xk.v[sp][c].im;
          acc.v[sp][c].re = fmaf(a.kappa, acc.v[sp][c].re, re);
          acc.v[sp][c].im = fmaf(a.kappa, acc.v[sp][c].im, im);
        }
      a.s_out.store(g, dom, s, acc);
    }
  }
  if (active) a.x.store(g, dom, s, xk);
}

// float32 <-> float16 field conversion (internal layouts, same site order;
// blockIdx.y selects the right-hand side)
__global__ void f32_to_f16_kernel(Geom g, F16Spinor out, F32Spinor in) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol || loop_idle(g)) return;
  const int dom = (int)(gid >> g.logvd) + blockIdx.y * g.ndom, s = (int)(gid & (g.vd - 1));
  Spinor<float> a;
  in.load(g, dom, s, a);
  out.store(g, dom, s, a);
}
__global__ void f16_to_f32_kernel(Geom g, F32Spinor out, F16Spinor in) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol || loop_idle(g)) return;
  const int dom = (int)(gid >> g.logvd) + blockIdx.y * g.ndom, s = (int)(gid & (g.vd - 1));
  Spinor<float> a;
  in.load(g, dom, s, a);
  out.store(g, dom, s, a);
}

template <typename SIO, typename LP, typename CP, typename CB>
static void launch_half_sweep(qcd_ctx* ctx, SapArgs<SIO, LP, CP> a, cudaStream_t st) {
  const Geom& g = ctx->geom;
  const int per_cta = SAP_THREADS >> g.logvd;
  const int grid = (g.nhalf + per_cta - 1) / per_cta;
  LaunchScope ls(ctx, QCD_KC_SAP_BLOCK, st);
  sap_block_kernel<SIO, LP, CP, CB><<<grid, SAP_THREADS, 0, st>>>(a);
  check_launch();
}

// The sweep sequence of Algorithm 1 for any storage type.
template <typename SIO, typename LP, typename CP, typename CB>
static void sap_sequence(qcd_ctx* ctx, SIO s_first_in, SIO s, SIO x, F32Spinor b, LP U, CP cinv, int n_sap,
                         int n_jac, cudaStream_t st) {
  SapArgs<SIO, LP, CP> a;
  a.g = ctx->geom;
  a.n_jac = n_jac;
  a.kappa = (float)ctx->kappa;
  a.b = b;
  a.U = U;
  a.cinv = cinv;
  a.x = x;
  a.s_out = s;
  for (int sweep = 0; sweep <= n_sap; ++sweep) {
    const bool last = sweep == n_sap;
    a.s_in = sweep == 0 ? s_first_in : s;
    a.do_update = last ? 0 : 1;
    a.colour = 0;
    a.do_surface = sweep == 0 ? 0 : 1;
    launch_half_sweep<SIO, LP, CP, CB>(ctx, a, st);
    a.colour = 1;
    a.do_surface = 1;
    launch_half_sweep<SIO, LP, CP, CB>(ctx, a, st);
  }
}

// x = M_SAP b for nrhs stacked float32 fields.  ws_s holds s (float32 or
// float16), ws_x16 / ws_b16 the float16 x and source of the generic kernel
// (sap_prec == HALF); ws_x16 is also the shared-memory kernel's face halo
// (96 bytes per site).  All three are sized for nrhs right-hand sides.  With the shared-memory kernel
// all right-hand sides go through each launch and share its staged links and
// C_inv; the generic kernel runs them one after the other.
void sap_apply_launch(qcd_ctx* ctx, float4* x, const float4* b, int nrhs, int n_sap, int n_jac, int sap_prec,
                      void* ws_s, void* ws_x16, void* ws_b16, cudaStream_t st) {
  if (ctx->sap_general) {
    sap_general_apply(ctx, x, b, nrhs, n_sap, n_jac, sap_prec, ws_s, st);
    return;
  }
  const Geom& g = ctx->geom;
  const bool staged = sap_staged_available(ctx) && !ctx->force_generic_sap;
  const size_t v = (size_t)g.vol;
  const size_t v4 = v * 6;
  if (sap_prec == QCD_PREC_HALF_GAUGE) {
    // float16 links and C_inv, float32 vectors
    if (staged) {
      F32Spinor xs{x}, bs{(float4*)b}, ss{(float4*)ws_s};
      sap_staged_sequence_h16g(ctx, bs, ss, xs, bs, (float4*)ws_x16, nrhs, n_sap, n_jac, st);
    } else {
      for (int r = 0; r < nrhs; ++r) {
        F32Spinor xs{x + r * v4}, bs{(float4*)b + r * v4}, ss{(float4*)ws_s + r * v4};
        sap_sequence<F32Spinor, LinkPtrHalf, CloverPtrF16, CloverBlockF32>(
            ctx, bs, ss, xs, bs, LinkPtrHalf{ctx->u16}, CloverPtrF16{ctx->cinv16}, n_sap, n_jac, st);
      }
    }
    return;
  }
  if (sap_prec == QCD_PREC_SINGLE) {
    if (staged) {
      F32Spinor xs{x}, bs{(float4*)b}, ss{(float4*)ws_s};
      sap_staged_sequence_f32(ctx, bs, ss, xs, bs, (float4*)ws_x16, nrhs, n_sap, n_jac, st);
    } else {
      for (int r = 0; r < nrhs; ++r) {
        F32Spinor xs{x + r * v4}, bs{(float4*)b + r * v4}, ss{(float4*)ws_s + r * v4};
        sap_sequence<F32Spinor, LinkPtr<float>, CloverPtrF32, CloverBlockF32>(
            ctx, bs, ss, xs, bs, LinkPtr<float>{ctx->u32}, CloverPtrF32{ctx->cinv32}, n_sap, n_jac, st);
      }
    }
    return;
  }
  const size_t nv = v * nrhs;
  F16Spinor s16{(uint4*)ws_s, (float*)((uint4*)ws_s + 3 * nv)};
  F16Spinor x16{(uint4*)ws_x16, (float*)((uint4*)ws_x16 + 3 * nv)};
  F16Spinor b16{(uint4*)ws_b16, (float*)((uint4*)ws_b16 + 3 * nv)};
  const dim3 cgrid(grid_for(g.vol, 256), nrhs);
  if (staged) {
    // the first sweep reads the float32 source and the last one writes the
    // float32 result: no conversion launches
    sap_staged_sequence_f16(ctx, F32Spinor{(float4*)b}, s16, F32Spinor{(float4*)b}, F32Spinor{x}, (float4*)ws_x16,
                            nrhs, n_sap, n_jac, st);
    return;
  }
  {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    f32_to_f16_kernel<<<cgrid, 256, 0, st>>>(g, b16, F32Spinor{(float4*)b});
    check_launch();
  }
  for (int r = 0; r < nrhs; ++r) {
    F16Spinor sr{s16.p + 3 * v * r, s16.nrm + v * r};
    F16Spinor xr{x16.p + 3 * v * r, x16.nrm + v * r};
    F16Spinor br{b16.p + 3 * v * r, b16.nrm + v * r};
    sap_sequence<F16Spinor, LinkPtrHalf, CloverPtrF16, CloverBlockF32>(
        ctx, br, sr, xr, F32Spinor{(float4*)b + r * v4}, LinkPtrHalf{ctx->u16}, CloverPtrF16{ctx->cinv16}, n_sap,
        n_jac, st);
  }
  {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    f16_to_f32_kernel<<<cgrid, 256, 0, st>>>(g, F32Spinor{x}, x16);
    check_launch();
  }
}

}  // namespace qcd
