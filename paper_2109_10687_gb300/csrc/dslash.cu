// Clover-Wilson operator kernels: D, D^dag, A = C_inv D, the clover
// multiply and the domain blocks A_EE / A_EO of Sec. 3 (arXiv:2109.10687,
// App. A for D; Sec. 3 Eq. hoppingmat for A).
//
// One thread per site.  Each of the eight hops is spin-projected to a half
// spinor (two spin rows), multiplied by the link (or its adjoint) and
// rebuilt into the accumulator: 168 flop per hop, 1320 for the hopping term,
// plus the clover block multiply.

#include <cstdio>

#include "qcd_internal.cuh"

namespace qcd {

template <typename R>
struct Prec;
template <>
struct Prec<float> {
  using SIO = F32Spinor;
  using LP = LinkPtr<float>;
  using CP = CloverPtrF32;
  using CB = CloverBlockF32;
};
template <>
struct Prec<double> {
  using SIO = F64Spinor;
  using LP = LinkPtr<double>;
  using CP = CloverPtrF64;
  using CB = CloverBlockF64;
};
template <>
struct Prec<df64> {
  using SIO = DF64Spinor;
  using LP = LinkPtr<df64>;
  using CP = CloverPtrDF64;
  using CB = CloverBlockDF64;
};

__global__ void __launch_bounds__(192, 4) dslash_df64_split_kernel(Geom g, DF64Spinor out, DF64Spinor in,
                                                                LinkPtr<df64> U, CloverPtrDF64 clov, df64 kappa,
                                                                int nrhs);

// acc += hop in direction MU (both orientations); PMF / PMB are the projector
// signs of the forward and backward hop.  FILTER: 0 all hops, 1 only hops
// inside the domain, 2 only hops that leave the domain.
template <int MU, int PMF, int PMB, int FILTER, typename R, typename SIO, typename LP>
__device__ __forceinline__ void hop_dir(const Geom& g, const SIO& in, const LP& U, int dom, int s, int rhs_off,
                                        Spinor<R>& acc) {
  {
    const bool intra = hop_is_intra(g, s, MU, true);
    if (FILTER == 0 || (FILTER == 1 && intra) || (FILTER == 2 && !intra)) {
      int nd, ns;
      const int sign = nbr_site(g, dom, s, MU, true, nd, ns);
      Spinor<R> p;
      in.load(g, nd + rhs_off, ns, p);
      HalfSpinor<R> h, uh;
      project<MU, PMF>(p, h);
      SU3<R> u;
      U.load(g, dom, MU, s, u);
      su3_mul(u, h, uh);
      if (sign < 0) scale_half(uh, R(-1.0f));
      accumulate<MU, PMF>(acc, uh);
    }
  }
  {
    const bool intra = hop_is_intra(g, s, MU, false);
    if (FILTER == 0 || (FILTER == 1 && intra) || (FILTER == 2 && !intra)) {
      int nd, ns;
      const int sign = nbr_site(g, dom, s, MU, false, nd, ns);
      Spinor<R> p;
      in.load(g, nd + rhs_off, ns, p);
      HalfSpinor<R> h, uh;
      project<MU, PMB>(p, h);
      SU3<R> u;
      U.load(g, nd, MU, ns, u);
      su3_dag_mul(u, h, uh);
      if (sign < 0) scale_half(uh, R(-1.0f));
      accumulate<MU, PMB>(acc, uh);
    }
  }
}

// Both hops of direction MU without branches: the neighbour (domain, site)
// and the boundary sign are selected, not branched on, so that the loads of
// all eight hops are independent straight-line code the compiler can issue
// early (the operator is bound by how many loads are in flight).  nb holds
// the eight neighbour domains of dom, tf its boundary-sign flags.
template <int MU, int PMF, int PMB, bool FIRST, typename R, typename SIO, typename LP>
__device__ __forceinline__ void hop_dir_bf(const Geom& g, const SIO& in, const LP& U, int dom, int s, int rhs_off,
                                           const int nb[8], int tf, Spinor<R>& acc) {
  static_assert(!FIRST || MU < 3, "the first hop must carry no boundary sign");
  const int c = (s >> g.shift[MU]) & (g.d[MU] - 1);
  const int step = 1 << g.shift[MU];
  const int span = (g.d[MU] - 1) * step;
  {
    const bool inside = c < g.d[MU] - 1;
    const int nd = inside ? dom : nb[2 * MU];
    const int ns = inside ? s + step : s - span;
    const R f = (!inside && ((tf >> (2 * MU)) & 1)) ? R(g.bc_t) : R(1.0f);
    Spinor<R> p;
    in.load(g, nd + rhs_off, ns, p);
    HalfSpinor<R> h, uh;
    project<MU, PMF>(p, h);
    SU3<R> u;
    U.load(g, dom, MU, s, u);
    su3_mul(u, h, uh);
    if (FIRST) rebuild<MU, PMF>(acc, uh);  // f = 1: the sign is for t hops only
    else accumulate<MU, PMF>(acc, uh, f);
  }
  {
    const bool inside = c > 0;
    const int nd = inside ? dom : nb[2 * MU + 1];
    const int ns = inside ? s - step : s + span;
    const R f = (!inside && ((tf >> (2 * MU + 1)) & 1)) ? R(g.bc_t) : R(1.0f);
    Spinor<R> p;
    in.load(g, nd + rhs_off, ns, p);
    HalfSpinor<R> h, uh;
    project<MU, PMB>(p, h);
    SU3<R> u;
    U.load(g, nd, MU, ns, u);
    su3_dag_mul(u, h, uh);
    accumulate<MU, PMB>(acc, uh, f);
  }
}

template <int PMF, int PMB, typename R, typename SIO, typename LP>
__device__ __forceinline__ void hopping_bf(const Geom& g, const SIO& in, const LP& U, int dom, int s, int rhs_off,
                                           Spinor<R>& acc) {
  int nb[8];
  const int4 n0 = __ldg(reinterpret_cast<const int4*>(g.nbr) + 2 * dom);
  const int4 n1 = __ldg(reinterpret_cast<const int4*>(g.nbr) + 2 * dom + 1);
  nb[0] = n0.x; nb[1] = n0.y; nb[2] = n0.z; nb[3] = n0.w;
  nb[4] = n1.x; nb[5] = n1.y; nb[6] = n1.z; nb[7] = n1.w;
  const int tf = __ldg(g.tflag + dom);
  hop_dir_bf<0, PMF, PMB, true>(g, in, U, dom, s, rhs_off, nb, tf, acc);  // starts the sum
  hop_dir_bf<1, PMF, PMB, false>(g, in, U, dom, s, rhs_off, nb, tf, acc);
  hop_dir_bf<2, PMF, PMB, false>(g, in, U, dom, s, rhs_off, nb, tf, acc);
  hop_dir_bf<3, PMF, PMB, false>(g, in, U, dom, s, rhs_off, nb, tf, acc);
}

template <int PMF, int PMB, int FILTER, typename R, typename SIO, typename LP>
__device__ __forceinline__ void hopping(const Geom& g, const SIO& in, const LP& U, int dom, int s, int rhs_off,
                                        Spinor<R>& acc) {
  zero(acc);
  hop_dir<0, PMF, PMB, FILTER>(g, in, U, dom, s, rhs_off, acc);
  hop_dir<1, PMF, PMB, FILTER>(g, in, U, dom, s, rhs_off, acc);
  hop_dir<2, PMF, PMB, FILTER>(g, in, U, dom, s, rhs_off, acc);
  hop_dir<3, PMF, PMB, FILTER>(g, in, U, dom, s, rhs_off, acc);
}

// D:    out = (1 + C) x - kappa H x
// D^dag: out = (1 + C) x - kappa H^dag x   (gamma_5 H gamma_5 swaps the projectors)
// A:    out = x - kappa C_inv H x
//
// Launch shape: THREADS per block, at least MINB blocks per SM (a register
// budget); the autotuner picks among the instantiated shapes.  Blocks are
// numbered rhs-fastest, so the nrhs blocks that share a tile of sites (and
// its links and clover) run back to back and reuse them from L2.
// One site (lexicographic-domain index gid) of one right-hand side.
template <typename R, int MODE, bool HINT = false, typename LP = typename Prec<R>::LP>
__device__ __forceinline__ void dslash_site(const Geom& g, const typename Prec<R>::SIO& out,
                                            const typename Prec<R>::SIO& in, const LP& U,
                                            const typename Prec<R>::CP& clov, R kappa, long long gid, int rhs) {
  // domains are visited in lexicographic order, so that the neighbouring
  // domains whose surface spinors a domain reads are processed at about the
  // same time and their data is still in L2
  const int dom = __ldg(g.lex2dom + (int)(gid >> g.logvd));
  const int s = (int)(gid & (g.vd - 1));
  const int rhs_off = rhs * g.ndom;
  Spinor<R> acc;
  if (MODE == MODE_DDAG) hopping_bf<+1, -1>(g, in, U, dom, s, rhs_off, acc);
  else hopping_bf<-1, +1>(g, in, U, dom, s, rhs_off, acc);
  Spinor<R> x;
  in.load(g, dom + rhs_off, s, x);
  if constexpr (HINT) {
    const CloverPtrF32Stream cs{clov.p};
    clover_mul<R, CloverPtrF32Stream, typename Prec<R>::CB>(cs, g, dom, s, MODE == MODE_A ? acc : x);
  } else if (MODE == MODE_A) {
    clover_mul<R, typename Prec<R>::CP, typename Prec<R>::CB>(clov, g, dom, s, acc);
  } else {
    clover_mul<R, typename Prec<R>::CP, typename Prec<R>::CB>(clov, g, dom, s, x);
  }
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.v[sp][c].re = fma(-kappa, acc.v[sp][c].re, x.v[sp][c].re);
      x.v[sp][c].im = fma(-kappa, acc.v[sp][c].im, x.v[sp][c].im);
    }
  if constexpr (HINT) out.store_stream(g, dom + rhs_off, s, x);
  else out.store(g, dom + rhs_off, s, x);
}

// HINT: the clover rows and the output, touched once per application, are
// read and written with the streaming (evict-first) cache operators, so
// that L2 keeps the spinor and link lines that neighbouring sites read
// again.  float32 only.  LP: the links' storage (LinkPtr12: the first two
// rows of SU(3) links, float32 only).
template <typename R, int MODE, int THREADS, int MINB, bool HINT, typename LP = typename Prec<R>::LP>
__global__ void __launch_bounds__(THREADS, MINB)
    dslash_kernel(Geom g, typename Prec<R>::SIO out, typename Prec<R>::SIO in, LP U, typename Prec<R>::CP clov,
                  R kappa, int nrhs) {
  const int rhs = blockIdx.x % nrhs;
  const long long gid = (blockIdx.x / nrhs) * (long long)THREADS + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (gid >= g.vol || loop_idle(g)) return;
  dslash_site<R, MODE, HINT, LP>(g, out, in, U, clov, kappa, gid, rhs);
}

// Ragged batch: one launch over several lattices of different sizes.  Block
// b belongs to lattice block_lat[b] (a table built once per batch); the
// block copies that lattice's descriptor (geometry, field pointers, kappa)
// to shared memory, so the geometry is read from there rather than from
// global memory on every index computation.
template <int MODE>
__global__ void __launch_bounds__(128, 4) dslash_batch_kernel(const BatchDesc* __restrict__ desc,
                                                              const int* __restrict__ block_lat) {
  __shared__ BatchDesc sd;
  {
    const int i = __ldg(block_lat + blockIdx.x);
    const int* src = reinterpret_cast<const int*>(desc + i);
    int* dst = reinterpret_cast<int*>(&sd);
    for (int k = threadIdx.x; k < (int)(sizeof(BatchDesc) / sizeof(int)); k += blockDim.x) dst[k] = __ldg(src + k);
  }
  __syncthreads();
  const long long gid = ((long long)blockIdx.x - sd.block_begin) * 128 + threadIdx.x;
  if (gid >= sd.g.vol) return;
  const F32Spinor out{sd.out}, in{(float4*)sd.in};
  const CloverPtrF32 clov{sd.clov};
  if (sd.u12)  // this lattice's links as 12 reals (uniform over the block)
    dslash_site<float, MODE, true, LinkPtr12>(sd.g, out, in, LinkPtr12{sd.u12}, clov, sd.kappa, gid, 0);
  else
    dslash_site<float, MODE, true>(sd.g, out, in, LinkPtr<float>{sd.u}, clov, sd.kappa, gid, 0);
}

void dslash_batch_launch(const BatchDesc* d_desc, const int* d_block_lat, long long total_blocks, int dagger,
                         cudaStream_t st) {
  QCD_REQUIRE(total_blocks < (1LL << 31), QCD_ERR_ARG, "batch too large for one launch");
  if (dagger) dslash_batch_kernel<MODE_DDAG><<<(unsigned)total_blocks, 128, 0, st>>>(d_desc, d_block_lat);
  else dslash_batch_kernel<MODE_D><<<(unsigned)total_blocks, 128, 0, st>>>(d_desc, d_block_lat);
  check_launch();
}

// Ragged batch solve: the float32 A of A M_SAP for every lattice in one
// launch (which 0: q = A zp, 1: t = A zr; lattices that have stopped
// iterating return at once), and the float64 D of Algorithm 4 (which 2:
// r64 = D x64, every lattice).  Block b belongs to lattice block_lat[b],
// whose descriptor the block copies to shared memory.
__device__ __forceinline__ void copy_lat_desc(const LatDesc* __restrict__ desc, int lat, LatDesc& sd) {
  const int* src = reinterpret_cast<const int*>(desc + lat);
  int* dst = reinterpret_cast<int*>(&sd);
  for (int k = threadIdx.x; k < (int)(sizeof(LatDesc) / sizeof(int)); k += blockDim.x) dst[k] = __ldg(src + k);
}
__global__ void __launch_bounds__(128, 3) lat_dslash_a_kernel(const LatDesc* __restrict__ desc,
                                                              const int* __restrict__ block_lat, int which) {
  __shared__ LatDesc sd;
  copy_lat_desc(desc, __ldg(block_lat + blockIdx.x), sd);
  __syncthreads();
  if (loop_idle(sd.g) || *(volatile const int*)sd.done) return;
  const long long gid = ((long long)blockIdx.x - sd.block_begin) * 128 + threadIdx.x;
  if (gid >= sd.g.vol) return;
  const CloverPtrF32 cinv{sd.cinv32};
  const F32Spinor o{which == 0 ? sd.q : sd.t}, i{which == 0 ? sd.zp : sd.zr};
  if (sd.u32c) {  // this lattice's links as 12 reals (uniform over the block)
    dslash_site<float, MODE_A, true, LinkPtr12>(sd.g, o, i, LinkPtr12{sd.u32c}, cinv, sd.kappa, gid, 0);
  } else {
    dslash_site<float, MODE_A, true>(sd.g, o, i, LinkPtr<float>{sd.u32}, cinv, sd.kappa, gid, 0);
  }
}
__global__ void __launch_bounds__(128) lat_dslash64_kernel(const LatDesc* __restrict__ desc,
                                                           const int* __restrict__ block_lat) {
  __shared__ LatDesc sd;
  copy_lat_desc(desc, __ldg(block_lat + blockIdx.x), sd);
  __syncthreads();
  const long long gid = ((long long)blockIdx.x - sd.block_begin) * 128 + threadIdx.x;
  if (gid >= sd.g.vol) return;
  dslash_site<double, MODE_D>(sd.g, F64Spinor{sd.r64}, F64Spinor{sd.x64}, LinkPtr<double>{sd.u64},
                              CloverPtrF64{sd.clov64}, sd.kappa64, gid, 0);
}

void lat_dslash_launch(const LatDesc* d_lat, const int* d_block_lat, long long blocks, int which, cudaStream_t st) {
  static_assert(sizeof(LatDesc) % sizeof(int) == 0, "descriptor is copied as ints");
  QCD_REQUIRE(blocks < (1LL << 31), QCD_ERR_ARG, "batch too large for one launch");
  if (which == 2) lat_dslash64_kernel<<<(unsigned)blocks, 128, 0, st>>>(d_lat, d_block_lat);
  else lat_dslash_a_kernel<<<(unsigned)blocks, 128, 0, st>>>(d_lat, d_block_lat, which);
  check_launch();
}

template <typename R>
__global__ void clover_apply_kernel(Geom g, typename Prec<R>::SIO out, typename Prec<R>::SIO in,
                                    typename Prec<R>::CP clov) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int dom = (int)(gid >> g.logvd);
  const int s = (int)(gid & (g.vd - 1));
  const int rhs_off = blockIdx.y * g.ndom;
  Spinor<R> x;
  in.load(g, dom + rhs_off, s, x);
  clover_mul<R, typename Prec<R>::CP, typename Prec<R>::CB>(clov, g, dom, s, x);
  out.store(g, dom + rhs_off, s, x);
}

// A_rc of Sec. 3: rows of colour `row`, columns of colour `col`.
__global__ void __launch_bounds__(128) ablock_kernel(Geom g, F32Spinor out, F32Spinor in, LinkPtr<float> U,
                                                     CloverPtrF32 cinv, float kappa, int row, int col) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int dom = (int)(gid >> g.logvd);
  const int s = (int)(gid & (g.vd - 1));
  const int colour = dom >= g.nhalf;
  Spinor<float> res;
  zero(res);
  if (colour == row) {
    Spinor<float> acc;
    if (row == col) hopping<-1, +1, 1>(g, in, U, dom, s, 0, acc);
    else hopping<-1, +1, 2>(g, in, U, dom, s, 0, acc);
    clover_mul<float, CloverPtrF32, CloverBlockF32>(cinv, g, dom, s, acc);
    if (row == col) in.load(g, dom, s, res);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        res.v[sp][c].re = fmaf(-kappa, acc.v[sp][c].re, res.v[sp][c].re);
        res.v[sp][c].im = fmaf(-kappa, acc.v[sp][c].im, res.v[sp][c].im);
      }
  }
  out.store(g, dom, s, res);
}

template <typename R, int MODE, int THREADS, int MINB, bool HINT = false, typename LP = typename Prec<R>::LP>
static void launch_dslash_shape(const Geom& g, void* out, const void* in, const void* U, const void* clov, R kappa,
                                int nrhs, cudaStream_t st, bool pdl) {
  using P = Prec<R>;
  const long long blocks = (long long)grid_for(g.vol, THREADS) * nrhs;
  QCD_REQUIRE(blocks < (1LL << 31), QCD_ERR_ARG, "lattice too large for one launch");
  const typename P::SIO o{(decltype(P::SIO::p))out}, i{(decltype(P::SIO::p))in};
  const LP u{(decltype(LP::p))U};
  const typename P::CP c{(decltype(P::CP::p))clov};
  if (pdl)
    launch_pdl(dslash_kernel<R, MODE, THREADS, MINB, HINT, LP>, dim3((unsigned)blocks), dim3(THREADS), 0, st, g, o, i, u,
               c, kappa, nrhs);
  else
    dslash_kernel<R, MODE, THREADS, MINB, HINT, LP><<<(unsigned)blocks, THREADS, 0, st>>>(g, o, i, u, c, kappa, nrhs);
}

// float32 launch shapes the autotuner chooses from: threads and blocks per
// SM and streaming cache operators (h); variants 8-15 (c) are the same
// shapes with the links read as their first two rows (SU(3) links)
template <int MODE>
static void launch_dslash_f32(int variant, const Geom& g, void* out, const void* in, const void* U, const void* U12,
                              const void* clov, float kappa, int nrhs, cudaStream_t st, bool pdl) {
  switch (variant) {
    case 0: launch_dslash_shape<float, MODE, 128, 4>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 1: launch_dslash_shape<float, MODE, 128, 5>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 2: launch_dslash_shape<float, MODE, 128, 6>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 3: launch_dslash_shape<float, MODE, 256, 2>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 4: launch_dslash_shape<float, MODE, 128, 4, true>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 5: launch_dslash_shape<float, MODE, 128, 5, true>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 6: launch_dslash_shape<float, MODE, 128, 6, true>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 7: launch_dslash_shape<float, MODE, 256, 2, true>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 8: launch_dslash_shape<float, MODE, 128, 4, false, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    case 9: launch_dslash_shape<float, MODE, 128, 5, false, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    case 10: launch_dslash_shape<float, MODE, 128, 6, false, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    case 11: launch_dslash_shape<float, MODE, 256, 2, false, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    case 12: launch_dslash_shape<float, MODE, 128, 4, true, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    case 13: launch_dslash_shape<float, MODE, 128, 5, true, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    case 14: launch_dslash_shape<float, MODE, 128, 6, true, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
    default: launch_dslash_shape<float, MODE, 256, 2, true, LinkPtr12>(g, out, in, U12, clov, kappa, nrhs, st, pdl); break;
  }
}
// float64 launch shapes (register budget against resident warps)
template <int MODE>
static void launch_dslash_f64(int variant, const Geom& g, void* out, const void* in, const void* U, const void* clov,
                              double kappa, int nrhs, cudaStream_t st, bool pdl) {
  switch (variant) {
    case 0: launch_dslash_shape<double, MODE, 128, 1>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 1: launch_dslash_shape<double, MODE, 128, 2>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    case 2: launch_dslash_shape<double, MODE, 128, 3>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
    default: launch_dslash_shape<double, MODE, 128, 4>(g, out, in, U, clov, kappa, nrhs, st, pdl); break;
  }
}
static const char* kDslashShapes64[] = {"128x1", "128x2", "128x3", "128x4"};
constexpr int kNumDslashShapes64 = 4;

static const char* kDslashShapes[] = {"128x4",   "128x5",   "128x6",   "256x2",   "128x4h",   "128x5h",
                                      "128x6h",  "256x2h",  "128x4c",  "128x5c",  "128x6c",   "256x2c",
                                      "128x4hc", "128x5hc", "128x6hc", "256x2hc"};
constexpr int kNumDslashShapes = 8;  // shapes per link format

void dslash_launch(qcd_ctx* ctx, void* out, const void* in, int prec, int mode, int nrhs, cudaStream_t st,
                   bool pdl) {
  const Geom& g = ctx->geom;
  if (prec == PREC_DF64) {
    QCD_REQUIRE(mode == MODE_D, QCD_ERR_ARG, "the double-float operator provides D only");
    QCD_REQUIRE(ctx->udf && ctx->clovdf, QCD_ERR_STATE, "double-float copies not built");
    LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
    const long long blocks = (long long)((g.vol + 63) / 64) * nrhs;
    QCD_REQUIRE(blocks < (1LL << 31), QCD_ERR_ARG, "lattice too large for one launch");
    dslash_df64_split_kernel<<<(unsigned)blocks, dim3(32, 3, 2), 0, st>>>(
        g, DF64Spinor{(float4*)out}, DF64Spinor{(float4*)in}, LinkPtr<df64>{ctx->udf}, CloverPtrDF64{ctx->clovdf},
        df64(ctx->kappa), nrhs);
    check_launch();
  } else if (prec == QCD_PREC_DOUBLE) {
    QCD_REQUIRE(mode != MODE_A, QCD_ERR_ARG, "A is provided in float32 only");
    auto run = [&](int v) {
      if (mode == MODE_D) launch_dslash_f64<MODE_D>(v, g, out, in, ctx->u64, ctx->clov64, ctx->kappa, nrhs, st, pdl);
      else launch_dslash_f64<MODE_DDAG>(v, g, out, in, ctx->u64, ctx->clov64, ctx->kappa, nrhs, st, pdl);
      check_launch();
    };
    char key[64];
    std::snprintf(key, sizeof key, "dslash_f64_mode%d_nrhs%d", mode, nrhs);
    const int v = tune_pick(ctx, key, kNumDslashShapes64, kDslashShapes64, run, st);
    LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
    run(v);
  } else if (prec == QCD_PREC_SINGLE) {
    const float k = (float)ctx->kappa;
    const void* clov = mode == MODE_A ? (const void*)ctx->cinv32 : (const void*)ctx->clov32;
    auto run = [&](int v) {
      if (mode == MODE_A) launch_dslash_f32<MODE_A>(v, g, out, in, ctx->u32, ctx->u32c, clov, k, nrhs, st, pdl);
      else if (mode == MODE_D) launch_dslash_f32<MODE_D>(v, g, out, in, ctx->u32, ctx->u32c, clov, k, nrhs, st, pdl);
      else launch_dslash_f32<MODE_DDAG>(v, g, out, in, ctx->u32, ctx->u32c, clov, k, nrhs, st, pdl);
      check_launch();
    };
    // The link format is not the tuner's to choose, since it changes the
    // arithmetic (the rebuilt row differs from the stored one by float32
    // rounding) and the tuner's choices may change scheduling only: 12-real
    // links whenever the links are SU(3), unless qcd_set_link_compression
    // says otherwise; the tuner picks among that format's launch shapes.
    QCD_REQUIRE(ctx->link12 != 1 || ctx->su3_links, QCD_ERR_STATE,
                "float32 D with 12-real links: the links are not SU(3) to 1e-9");
    const bool use12 = uses_links12(ctx);
    const int base = use12 ? kNumDslashShapes : 0;
    char key[64];
    std::snprintf(key, sizeof key, "dslash_f32_mode%d_nrhs%d%s", mode, nrhs, use12 ? "_links12" : "");
    const int v = base + tune_pick(ctx, key, kNumDslashShapes, kDslashShapes + base, [&](int c) { run(base + c); }, st);
    LaunchScope ls(ctx, QCD_KC_DSLASH, st);
    run(v);
  } else {
    throw Error{QCD_ERR_ARG, "operator precision must be DOUBLE or SINGLE"};
  }
}

void clover_apply_launch(qcd_ctx* ctx, void* out, const void* in, int prec, int inverse, int nrhs,
                         cudaStream_t st) {
  const Geom& g = ctx->geom;
  dim3 grid(grid_for(g.vol, 128), nrhs);
  if (prec == QCD_PREC_DOUBLE) {
    LaunchScope ls(ctx, QCD_KC_DOUBLE, st);
    F64Spinor o{(double2*)out}, i{(double2*)in};
    CloverPtrF64 c{inverse ? ctx->cinv64 : ctx->clov64};
    clover_apply_kernel<double><<<grid, 128, 0, st>>>(g, o, i, c);
  } else if (prec == QCD_PREC_SINGLE) {
    LaunchScope ls(ctx, QCD_KC_BLAS, st);
    F32Spinor o{(float4*)out}, i{(float4*)in};
    CloverPtrF32 c{inverse ? ctx->cinv32 : ctx->clov32};
    clover_apply_kernel<float><<<grid, 128, 0, st>>>(g, o, i, c);
  } else {
    throw Error{QCD_ERR_ARG, "clover precision must be DOUBLE or SINGLE"};
  }
  check_launch();
}

void ablock_launch(qcd_ctx* ctx, float4* out, const float4* in, int row, int col, cudaStream_t st) {
  const Geom& g = ctx->geom;
  LaunchScope ls(ctx, QCD_KC_DSLASH, st);
  ablock_kernel<<<grid_for(g.vol, 128), 128, 0, st>>>(g, F32Spinor{out}, F32Spinor{(float4*)in},
                                                      LinkPtr<float>{ctx->u32}, CloverPtrF32{ctx->cinv32},
                                                      (float)ctx->kappa, row, col);
  check_launch();
}

// ---------------------------------------------------------------------------
// D in double-float with the work of a site split over its three colour rows
// ---------------------------------------------------------------------------
// Thread (site, a) owns colour a of the site.  Phase 1: for each of the eight
// hops it loads colour a of the neighbour spinor (four spins), projects it to
// the two spin rows of that colour and leaves them in shared memory.
// Phase 2: for each hop it reads the projected rows of all three colours,
// forms row a of U h (or U^dag h) and rebuilds its four spins.  Each
// projection is done once (not once per colour thread), and a thread loads
// a third of every neighbour spinor.  Block (32, 3, 2): warps of 32
// consecutive sites share one colour; 64 sites per block.
constexpr int DF_SITES = 64;

// Code size matters more than anything else here: written out for all
// eight hops and three colour rows, a thread's double-float arithmetic is
// several thousand instructions that the instruction cache cannot hold, and
// the warps wait on instruction fetch.  So the hops run in a loop: the
// neighbour lookup, the loads and the complex multiply-adds are one piece
// of code for every hop, and only the spin projection and reconstruction,
// which differ by direction, go through a switch to their fixed forms; the
// clover rows read their entries by a row index known at run time.  The
// arithmetic and its order are those of the fully written-out form.

// neighbour (domain, site, sign) of hop (mu, fwd), selected without branches
__device__ __forceinline__ void df_nbr(const Geom& g, int mu, bool fwd, int dom, int s, const int nb[8], int tf,
                                       int& nd, int& ns, bool& neg) {
  const int c = (s >> g.shift[mu]) & (g.d[mu] - 1);
  const int step = 1 << g.shift[mu];
  const int span = (g.d[mu] - 1) * step;
  const bool inside = fwd ? c < g.d[mu] - 1 : c > 0;
  const int k = 2 * mu + (fwd ? 0 : 1);
  nd = inside ? dom : nb[k];
  ns = inside ? (fwd ? s + step : s - step) : (fwd ? s - span : s + span);
  neg = !inside && ((tf >> k) & 1) && g.bc_t < 0;
}

__device__ __forceinline__ float4 df_pack(cx<df64> v) { return make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }
__device__ __forceinline__ cx<df64> df_unpack(float4 v) { return make_cx(df64(v.x, v.y), df64(v.z, v.w)); }

// the projection of hop (MU, FWD): its fixed spin pattern
template <int MU, bool FWD>
__device__ __forceinline__ void df_proj(const cx<df64> q[4], cx<df64>& h0, cx<df64>& h1) {
  project1<MU, FWD ? -1 : +1>(q[0], q[1], q[2], q[3], h0, h1);
}

// phase 1 loads: colour a of the four spins of hop's neighbour, and its sign
__device__ __forceinline__ void df_project_load(const Geom& g, const DF64Spinor& in, int hop, int dom, int s, int a,
                                                const int nb[8], int tf, float4 q[4], bool& neg) {
  int nd, ns;
  df_nbr(g, hop >> 1, !(hop & 1), dom, s, nb, tf, nd, ns, neg);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) q[sp] = __ldg(in.p + in.idx(g, nd, sp * 3 + a, ns));
}

// phase 1: rows (h0, h1) of colour a of the projected neighbour, signed
__device__ __forceinline__ void df_project(int hop, int a, const float4 qv[4], bool neg, float4* sh, int sl) {
  cx<df64> q[4];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) q[sp] = df_unpack(qv[sp]);
  cx<df64> h0, h1;
  switch (hop) {
    case 0: df_proj<0, true>(q, h0, h1); break;
    case 1: df_proj<0, false>(q, h0, h1); break;
    case 2: df_proj<1, true>(q, h0, h1); break;
    case 3: df_proj<1, false>(q, h0, h1); break;
    case 4: df_proj<2, true>(q, h0, h1); break;
    case 5: df_proj<2, false>(q, h0, h1); break;
    case 6: df_proj<3, true>(q, h0, h1); break;
    default: df_proj<3, false>(q, h0, h1); break;
  }
  if (neg) {  // exact: a sign flip of both parts
    h0 = make_cx(-h0.re, -h0.im);
    h1 = make_cx(-h1.re, -h1.im);
  }
  sh[((hop * 2 + 0) * 3 + a) * DF_SITES + sl] = df_pack(h0);
  sh[((hop * 2 + 1) * 3 + a) * DF_SITES + sl] = df_pack(h1);
}

// the reconstruction of hop (MU, FWD) into the four spins of one colour
// (the rules of accumulate())
template <int MU, bool FWD>
__device__ __forceinline__ void df_rebuild(cx<df64> h0, cx<df64> h1, cx<df64> acc[4]) {
  constexpr int PM = FWD ? -1 : +1;
  acc[0] = acc[0] + h0;
  acc[1] = acc[1] + h1;
  if (MU == 0) {
    if (PM < 0) { acc[2] = acc[2] + times_mi(h1); acc[3] = acc[3] + times_mi(h0); }
    else        { acc[2] = acc[2] + times_i(h1);  acc[3] = acc[3] + times_i(h0); }
  } else if (MU == 1) {
    if (PM < 0) { acc[2] = acc[2] - h1; acc[3] = acc[3] + h0; }
    else        { acc[2] = acc[2] + h1; acc[3] = acc[3] - h0; }
  } else if (MU == 2) {
    if (PM < 0) { acc[2] = acc[2] + times_mi(h0); acc[3] = acc[3] + times_i(h1); }
    else        { acc[2] = acc[2] + times_i(h0);  acc[3] = acc[3] + times_mi(h1); }
  } else {
    if (PM < 0) { acc[2] = acc[2] - h0; acc[3] = acc[3] - h1; }
    else        { acc[2] = acc[2] + h0; acc[3] = acc[3] + h1; }
  }
}

// phase 2 loads: row a (forward) or column a (backward) of hop's link
__device__ __forceinline__ void df_link_load(const Geom& g, const LinkPtr<df64>& U, int hop, int dom, int s, int a,
                                             const int nb[8], int tf, float4 v[3]) {
  const int mu = hop >> 1;
  const bool fwd = !(hop & 1);
  int nd, ns;
  bool neg;
  df_nbr(g, mu, fwd, dom, s, nb, tf, nd, ns, neg);
  const size_t base = ((size_t)(((fwd ? dom : nd) * 4 + mu) * 9)) << g.logvd;
  const int site = fwd ? s : ns;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int e = fwd ? a * 3 + b : b * 3 + a;
    v[b] = __ldg(U.p + base + ((size_t)e << g.logvd) + site);
  }
}

// phase 2: row a of U h (forward) or U^dag h (backward), rebuilt into colour a
__device__ __forceinline__ void df_mul_acc(int hop, const float4 v[3], const float4* sh, int sl, cx<df64> acc[4]) {
  const bool fwd = !(hop & 1);
  cx<df64> row[3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
    row[b] = fwd ? make_cx(df64(v[b].x, v[b].y), df64(v[b].z, v[b].w))
                 : make_cx(df64(v[b].x, v[b].y), -df64(v[b].z, v[b].w));
  cx<df64> uh[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    cx<df64> t = row[0] * df_unpack(sh[((hop * 2 + r) * 3 + 0) * DF_SITES + sl]);
    t = cmac(t, row[1], df_unpack(sh[((hop * 2 + r) * 3 + 1) * DF_SITES + sl]));
    t = cmac(t, row[2], df_unpack(sh[((hop * 2 + r) * 3 + 2) * DF_SITES + sl]));
    uh[r] = t;
  }
  switch (hop) {
    case 0: df_rebuild<0, true>(uh[0], uh[1], acc); break;
    case 1: df_rebuild<0, false>(uh[0], uh[1], acc); break;
    case 2: df_rebuild<1, true>(uh[0], uh[1], acc); break;
    case 3: df_rebuild<1, false>(uh[0], uh[1], acc); break;
    case 4: df_rebuild<2, true>(uh[0], uh[1], acc); break;
    case 5: df_rebuild<2, false>(uh[0], uh[1], acc); break;
    case 6: df_rebuild<3, true>(uh[0], uh[1], acc); break;
    default: df_rebuild<3, false>(uh[0], uh[1], acc); break;
  }
}

// (1 + C) x, row i of block b (i = 3 r + a, known at run time): the block's
// packed reals come straight from memory, the diagonal one as a real
// factor and the off-diagonal ones conjugated below the diagonal; the loads
// of column j + 1 are issued before the arithmetic of column j
__device__ __forceinline__ float4 df_clover_entry(const float4* cp, int logvd, int i, int j) {
  const int k = j == i ? (i >> 1) : 3 + (j > i ? herm_off(i, j) : herm_off(j, i));
  return __ldg(cp + ((size_t)k << logvd));
}
__device__ __forceinline__ cx<df64> df_clover_row(const Geom& g, const DF64Spinor& in, const CloverPtrDF64& clov,
                                                  int dom, int s, int b, int i) {
  const float4* cp = clov.p + (((size_t)(dom * 36 + 18 * b)) << g.logvd) + s;
  cx<df64> y = make_cx(df64(0.f), df64(0.f));
  float4 xn = __ldg(in.p + in.idx(g, dom, (2 * b) * 3, s));
  float4 cn = df_clover_entry(cp, g.logvd, i, 0);
#pragma unroll 1
  for (int j = 0; j < 6; ++j) {
    const float4 xv = xn, cv = cn;
    if (j < 5) {
      xn = __ldg(in.p + in.idx(g, dom, (2 * b + (j + 1) / 3) * 3 + (j + 1) % 3, s));
      cn = df_clover_entry(cp, g.logvd, i, j + 1);
    }
    const cx<df64> xj = df_unpack(xv);
    if (j == i) {
      const df64 d = (i & 1) ? df64(cv.z, cv.w) : df64(cv.x, cv.y);
      y = make_cx(fma(d, xj.re, y.re), fma(d, xj.im, y.im));
    } else {
      const cx<df64> c = df_unpack(cv);
      y = j > i ? cmac(y, c, xj) : cmacc(y, c, xj);
    }
  }
  return y;
}

// One tile of DF_SITES sites from site0 (lexicographic-domain order) of the
// field `in` (one right-hand side); every thread of the block takes part.
// store(dom, comp, s, value) writes one colour row of the result.
template <typename Store>
__device__ __forceinline__ void df64_tile(const Geom& g, const DF64Spinor& inr, const LinkPtr<df64>& U,
                                          const CloverPtrDF64& clov, df64 kappa, long long site0, float4* sh,
                                          const Store& store) {
  const int a = threadIdx.y;  // colour row
  const int sl = threadIdx.z * 32 + threadIdx.x;
  const long long gid = site0 + sl;
  // every thread takes part in the barrier; sites past the end compute on
  // site 0 of the block's range and store nothing
  const bool live = gid < g.vol;
  const long long gq = live ? gid : site0;
  const int dom = __ldg(g.lex2dom + (int)(gq >> g.logvd));
  const int s = (int)(gq & (g.vd - 1));
  int nb[8];
  {
    const int4 n0 = __ldg(reinterpret_cast<const int4*>(g.nbr) + 2 * dom);
    const int4 n1 = __ldg(reinterpret_cast<const int4*>(g.nbr) + 2 * dom + 1);
    nb[0] = n0.x; nb[1] = n0.y; nb[2] = n0.z; nb[3] = n0.w;
    nb[4] = n1.x; nb[5] = n1.y; nb[6] = n1.z; nb[7] = n1.w;
  }
  const int tf = __ldg(g.tflag + dom);
  // each loop issues the next hop's loads before this hop's arithmetic
  {
    float4 qn[4];
    bool negn;
    df_project_load(g, inr, 0, dom, s, a, nb, tf, qn, negn);
#pragma unroll 1
    for (int hop = 0; hop < 8; ++hop) {
      float4 q[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] = qn[k];
      const bool neg = negn;
      if (hop < 7) df_project_load(g, inr, hop + 1, dom, s, a, nb, tf, qn, negn);
      df_project(hop, a, q, neg, sh, sl);
    }
  }
  __syncthreads();
  cx<df64> acc[4];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) acc[sp] = make_cx(df64(0.f), df64(0.f));
  {
    float4 vn[3];
    df_link_load(g, U, 0, dom, s, a, nb, tf, vn);
#pragma unroll 1
    for (int hop = 0; hop < 8; ++hop) {
      float4 v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = vn[k];
      if (hop < 7) df_link_load(g, U, hop + 1, dom, s, a, nb, tf, vn);
      df_mul_acc(hop, v, sh, sl, acc);
    }
  }
  if (!live) return;
  // (1 + C) x, rows (block b, spin-in-block r, colour a): index i = 3 r + a
  cx<df64> res[4];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int r = 0; r < 2; ++r) res[2 * b + r] = df_clover_row(g, inr, clov, dom, s, b, 3 * r + a);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
    store(dom, sp * 3 + a, s, make_cx(fma(-kappa, acc[sp].re, res[sp].re), fma(-kappa, acc[sp].im, res[sp].im)));
}

__global__ void __launch_bounds__(192, 4) dslash_df64_split_kernel(Geom g, DF64Spinor out, DF64Spinor in,
                                                                LinkPtr<df64> U, CloverPtrDF64 clov, df64 kappa,
                                                                int nrhs) {
  __shared__ float4 sh[8 * 2 * 3 * DF_SITES];  // projected rows [hop][row][colour][site], 48 KB
  const int rhs = blockIdx.x % nrhs;
  const int rhs_off = rhs * g.ndom;
  const DF64Spinor inr{in.p + ((size_t)rhs_off * 12 << g.logvd)};
  df64_tile(g, inr, U, clov, kappa, (blockIdx.x / nrhs) * (long long)DF_SITES, sh,
            [&](int dom, int comp, int s, cx<df64> o) { out.p[out.idx(g, dom + rhs_off, comp, s)] = df_pack(o); });
}

// Ragged batch: the double-float D of Algorithm 4 (r64 = D x, read from the
// scaled double-float copy xdf, written to float64 unscaled) over every
// lattice in one launch.  Tile b of DF_SITES sites belongs to lattice
// tile_lat[b]; the lattice's descriptor is copied to shared memory.
__global__ void __launch_bounds__(192, 4) lat_dslash_df64_kernel(const LatDesc* __restrict__ desc,
                                                                const int* __restrict__ tile_lat,
                                                                const double* __restrict__ b2) {
  extern __shared__ float4 dsh[];  // projected rows, 48 KB, then the descriptor
  LatDesc& sd = *reinterpret_cast<LatDesc*>(dsh + 8 * 2 * 3 * DF_SITES);
  const int lat = __ldg(tile_lat + blockIdx.x);
  {
    const int* src = reinterpret_cast<const int*>(desc + lat);
    int* dst = reinterpret_cast<int*>(&sd);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    for (int k = t; k < (int)(sizeof(LatDesc) / sizeof(int)); k += nt) dst[k] = __ldg(src + k);
  }
  __syncthreads();
  const int kexp = df_scale_exp(b2[lat], (size_t)sd.g.vol * 12);
  const F64Spinor out{sd.r64};
  const Geom& g = sd.g;
  df64_tile(g, DF64Spinor{sd.xdf}, LinkPtr<df64>{sd.udf}, CloverPtrDF64{sd.clovdf}, df64(sd.kappa64),
            ((long long)blockIdx.x - sd.df_tile_begin) * DF_SITES, dsh, [&](int dom, int comp, int s, cx<df64> o) {
              out.p[out.idx(g, dom, comp, s)] =
                  make_double2(df64_to_double_scaled(o.re, kexp), df64_to_double_scaled(o.im, kexp));
            });
}

void lat_dslash_df64_launch(const LatDesc* d_lat, const int* d_tile_lat, long long tiles, const double* d_b2,
                            cudaStream_t st) {
  QCD_REQUIRE(tiles < (1LL << 31), QCD_ERR_ARG, "batch too large for one launch");
  const int smem = (int)(sizeof(float4) * 8 * 2 * 3 * DF_SITES + sizeof(LatDesc));
  static const bool attr = [smem] {
    QCD_CUDA_CHECK(cudaFuncSetAttribute(lat_dslash_df64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return true;
  }();
  (void)attr;
  lat_dslash_df64_kernel<<<(unsigned)tiles, dim3(32, 3, 2), smem, st>>>(d_lat, d_tile_lat, d_b2);
  check_launch();
}

// float64 (double2) fields -> double-float (float4) copies, elementwise, by
// integer operations on the bits (links and clover entries are far inside
// float32's range)
__global__ void f64_to_df64_kernel(const double2* __restrict__ in, float4* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    const df64 re = df64_from_double_scaled(v.x, 0), im = df64_from_double_scaled(v.y, 0);
    out[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

void build_df64_copies(qcd_ctx* ctx, bool links, bool clover, cudaStream_t st) {
  const Geom& g = ctx->geom;
  if (links) {
    const size_t n = (size_t)g.vol * 36;
    if (!ctx->udf) QCD_CUDA_CHECK(cudaMalloc(&ctx->udf, n * sizeof(float4)));
    LaunchScope ls(ctx, QCD_KC_OTHER, st);
    f64_to_df64_kernel<<<1024, 256, 0, st>>>(ctx->u64, ctx->udf, n);
    check_launch();
  }
  if (clover) {
    const size_t n = (size_t)g.vol * 36;
    if (!ctx->clovdf) QCD_CUDA_CHECK(cudaMalloc(&ctx->clovdf, n * sizeof(float4)));
    LaunchScope ls(ctx, QCD_KC_OTHER, st);
    f64_to_df64_kernel<<<1024, 256, 0, st>>>(ctx->clov64, ctx->clovdf, n);
    check_launch();
  }
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

extern "C" int qcd_apply_D(qcd_ctx* ctx, void* out, const void* in, int prec, int dagger, int nrhs, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  require_operator(ctx);
  QCD_REQUIRE(out && in && out != in && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_apply_D: bad arguments");
  dslash_launch(ctx, out, in, prec, dagger ? MODE_DDAG : MODE_D, nrhs, (cudaStream_t)stream, true);
  API_END(ctx)
}

extern "C" int qcd_apply_A(qcd_ctx* ctx, void* out, const void* in, int nrhs, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  require_operator(ctx);
  QCD_REQUIRE(out && in && out != in && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_apply_A: bad arguments");
  dslash_launch(ctx, out, in, QCD_PREC_SINGLE, MODE_A, nrhs, (cudaStream_t)stream, true);
  API_END(ctx)
}

extern "C" int qcd_apply_clover(qcd_ctx* ctx, void* out, const void* in, int prec, int inverse, int nrhs,
                                void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  require_operator(ctx);
  QCD_REQUIRE(out && in && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_apply_clover: bad arguments");
  clover_apply_launch(ctx, out, in, prec, inverse, nrhs, (cudaStream_t)stream);
  API_END(ctx)
}

extern "C" int qcd_apply_A_block(qcd_ctx* ctx, void* out, const void* in, int row, int col, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  API_BEGIN
  require_operator(ctx);
  QCD_REQUIRE(out && in && out != in && (row == 0 || row == 1) && (col == 0 || col == 1), QCD_ERR_ARG,
              "qcd_apply_A_block: bad arguments");
  ablock_launch(ctx, (float4*)out, (const float4*)in, row, col, (cudaStream_t)stream);
  API_END(ctx)
}
