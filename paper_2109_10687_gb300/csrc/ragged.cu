// Ragged batch solve in shared launches: many lattices of different sizes,
// gauge fields and kappa solved together, D x_i = b_i for every lattice i, by
// the method of qcd_solve (Algorithm 4 in float64 around Algorithm 5 on
// A M_SAP, arXiv:2109.10687 Sec. 3), with every step of an iteration one
// launch over all lattices:
//   - the SAP half-sweeps (Algorithm 1): one launch per half-sweep over the
//     domains of that colour of every lattice (sap_batch_run);
//   - A z (float32) and D x (float64): one launch over the sites of every
//     lattice (lat_dslash_launch);
//   - the fused BLAS-1 kernels of Algorithm 5 and the float64 vector kernels
//     of Algorithm 4: grid (blocks, lattice), each lattice's segment of the
//     batch's ragged buffers (Seg) and its own scalar record (Scal).
// The inner loop is one CUDA graph with a conditional while node, driven by
// the number of lattices still iterating; a lattice that has converged stops
// there (its SAP domains and operator blocks return at once) while the
// others continue.  The outer loop (Algorithm 4) runs on the host, one
// residual per lattice per step; lattices that have met the tolerance get a
// zero inner right-hand side, so their inner solve stops at once and their x
// is left unchanged.
//
// Every lattice must have 4^4 domains (the shared-memory SAP kernel);
// buffers are allocated once per batch, on the first solve.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "blas.cuh"

namespace qcd {

struct RaggedWS {
  int n = 0;
  size_t v4tot = 0, n2tot = 0, vtot = 0;   // float4, double2 and sites over all lattices
  std::vector<size_t> v4off, v4len, n2off, n2len, voff;
  size_t *d_v4off = nullptr, *d_v4len = nullptr, *d_n2off = nullptr, *d_n2len = nullptr;
  float4 *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *t = nullptr, *zp = nullptr, *zr = nullptr,
         *rt = nullptr, *b32 = nullptr, *sap_s = nullptr, *halo = nullptr;
  double2 *x64 = nullptr, *r64 = nullptr, *b64 = nullptr;
  float4* xdf = nullptr;   // scaled double-float copy of x64 (residual_prec 0)
  double* partials = nullptr;
  unsigned* counters = nullptr;
  Scal* scal = nullptr;
  Scal* h_scal = nullptr;  // pinned
  int* ctrl = nullptr;     // [0] lattices iterating, [1] iterations, [2] iteration limit
  int* h_ctrl = nullptr;   // pinned
  double* dres = nullptr;  // [0, n) |b|^2, [n, 2n) |r|^2, [2n, 3n) per-lattice scale
  double* h_res = nullptr; // pinned copy
  int* d_status = nullptr; // QCD_ERR_TIMEOUT from a bounded wait in a SAP launch
  int nblocks = 0;
  LatDesc* d_lat = nullptr;
  int* d_site_lat = nullptr;
  long long site_blocks = 0;
  int* d_tile_lat = nullptr;  // lattice of every 64-site double-float tile
  long long df_tiles = 0;
  SapBatchPlan* plan_p = nullptr;  // M_SAP p -> zp
  SapBatchPlan* plan_r = nullptr;  // M_SAP r -> zr
  int plan_prec = -1, plan_nsap = -1, plan_njac = -1;
  cudaGraphExec_t loop = nullptr;
  long long nloop = 0;
  cudaStream_t st = nullptr;
  std::vector<int> clover_gen;  // each lattice's clover build the descriptors were made from
  std::vector<bool> links12;    // and each lattice's float32 link format
};

void ragged_free(RaggedWS* w) {
  if (!w) return;
  void* ptrs[] = {w->d_v4off, w->d_v4len, w->d_n2off, w->d_n2len, w->x, w->r, w->p, w->q, w->t, w->zp, w->zr,
                  w->rt, w->b32, w->sap_s, w->halo, w->x64, w->r64, w->b64, w->partials, w->counters, w->scal,
                  w->ctrl, w->dres, w->d_status, w->d_lat, w->d_site_lat, w->xdf, w->d_tile_lat};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (w->h_scal) cudaFreeHost(w->h_scal);
  if (w->h_ctrl) cudaFreeHost(w->h_ctrl);
  if (w->h_res) cudaFreeHost(w->h_res);
  sap_batch_free(w->plan_p);
  sap_batch_free(w->plan_r);
  if (w->loop) cudaGraphExecDestroy(w->loop);
  if (w->st) cudaStreamDestroy(w->st);
  delete w;
}

bool ragged_eligible(const std::vector<qcd_ctx*>& ctx, const qcd_solve_params& P) {
  if (P.outer_restart != 0) return false;  // the residual is float64 here whatever residual_prec says
  for (const qcd_ctx* c : ctx)
    if (!c->have_gauge || !c->have_clover || !sap_staged_available(c) || c->sap_general) return false;
  return true;
}

// ---------------------------------------------------------------------------
// kernels of the float64 outer loop over every lattice
// ---------------------------------------------------------------------------
// out[k] = |a_k|^2 for every lattice k (grid (blocks, lattices))
__global__ void k_rg_norm2_f64(const double2* __restrict__ a, Seg seg, double* out, double* partials,
                               unsigned* counters) {
  const int k = blockIdx.y;
  const size_t off = seg.at(k), n = seg.size(k);
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = a[off + i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, partials + (size_t)k * MAX_RED_OUT * gridDim.x, counters + k, tot) && threadIdx.x == 0)
    out[k] = tot[0];
}

// r_k = b_k - r_k (r holds D x on entry); out[k] = |r_k|^2
__global__ void k_rg_residual_f64(const double2* __restrict__ b, double2* r, Seg seg, double* out, double* partials,
                                  unsigned* counters) {
  const int k = blockIdx.y;
  const size_t off = seg.at(k), n = seg.size(k);
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = b[off + i], dv = r[off + i];
    const double2 v = make_double2(bv.x - dv.x, bv.y - dv.y);
    r[off + i] = v;
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce<1>(v, partials + (size_t)k * MAX_RED_OUT * gridDim.x, counters + k, tot) && threadIdx.x == 0)
    out[k] = tot[0];
}

// xdf_k = x64_k 2^e_k in double-float, e_k from lattice k's |b|^2 (b2)
__global__ void k_rg_to_df(const double2* __restrict__ x, float4* xdf, Seg seg, const double* b2) {
  const int k = blockIdx.y;
  const size_t off = seg.at(k), n = seg.size(k);
  const int e = df_scale_exp(b2[k], n);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = x[off + i];
    const df64 re = df64_from_double_scaled(v.x, e), im = df64_from_double_scaled(v.y, e);
    xdf[off + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

__device__ __forceinline__ bool rg_site(const LatDesc* __restrict__ desc, const int* __restrict__ site_lat,
                                        LatDesc& sd, int& lat, int& dom, int& s) {
  lat = __ldg(site_lat + blockIdx.x);
  {
    const int* src = reinterpret_cast<const int*>(desc + lat);
    int* dst = reinterpret_cast<int*>(&sd);
    for (int k = threadIdx.x; k < (int)(sizeof(LatDesc) / sizeof(int)); k += blockDim.x) dst[k] = __ldg(src + k);
  }
  __syncthreads();
  const long long gid = ((long long)blockIdx.x - sd.block_begin) * blockDim.x + threadIdx.x;
  if (gid >= sd.g.vol) return false;
  dom = (int)(gid >> sd.g.logvd);
  s = (int)(gid & (sd.g.vd - 1));
  return true;
}

// inner right-hand side of every lattice: b32 = C_inv R_SP(scale r64)
// (Algorithm 4's p = R_SP(r / err), and A q = C_inv p is the system solved)
__global__ void __launch_bounds__(128) k_rg_prep(const LatDesc* __restrict__ desc, const int* __restrict__ site_lat,
                                                 const double* __restrict__ scale) {
  __shared__ LatDesc sd;
  int lat, dom, s;
  if (!rg_site(desc, site_lat, sd, lat, dom, s)) return;
  const double f = scale[lat];
  Spinor<double> r;
  F64Spinor{sd.r64}.load(sd.g, dom, s, r);
  Spinor<float> p;
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) p.v[sp][c] = make_cx((float)(r.v[sp][c].re * f), (float)(r.v[sp][c].im * f));
  clover_mul<float, CloverPtrF32, CloverBlockF32>(CloverPtrF32{sd.cinv32}, sd.g, dom, s, p);
  F32Spinor{sd.b32}.store(sd.g, dom, s, p);
}

// x64 += scale P_DP(x32) for every lattice (Algorithm 4's x += err P_DP(q))
__global__ void __launch_bounds__(128) k_rg_axpy(const LatDesc* __restrict__ desc, const int* __restrict__ site_lat,
                                                 const double* __restrict__ scale) {
  __shared__ LatDesc sd;
  int lat, dom, s;
  if (!rg_site(desc, site_lat, sd, lat, dom, s)) return;
  const double f = scale[lat];
  if (f == 0.0) return;
  Spinor<float> q;
  F32Spinor{sd.x}.load(sd.g, dom, s, q);
  Spinor<double> x;
  const F64Spinor xs{sd.x64};
  xs.load(sd.g, dom, s, x);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.v[sp][c].re = fma(f, (double)q.v[sp][c].re, x.v[sp][c].re);
      x.v[sp][c].im = fma(f, (double)q.v[sp][c].im, x.v[sp][c].im);
    }
  xs.store(sd.g, dom, s, x);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static RaggedWS* ragged_ws(const std::vector<qcd_ctx*>& ctx, RaggedWS*& wp) {
  if (wp) {
    // descriptors and SAP plans hold kappa and pointers taken at the first
    // solve: rebuild them after any lattice's clover term was rebuilt or its
    // link format changed
    bool same = true;
    for (size_t i = 0; i < ctx.size(); ++i)
      same = same && wp->clover_gen[i] == ctx[i]->clover_gen && wp->links12[i] == uses_links12(ctx[i]);
    if (same) return wp;
    QCD_CUDA_CHECK(cudaDeviceSynchronize());
    ragged_free(wp);
    wp = nullptr;
  }
  RaggedWS* w = new RaggedWS();
  try {
    const int n = (int)ctx.size();
    w->n = n;
    std::vector<LatDesc> lat(n);
    std::vector<int> site_lat, tile_lat;
    for (int i = 0; i < n; ++i) {
      const Geom& g = ctx[i]->geom;
      w->voff.push_back(w->vtot);
      w->v4off.push_back(w->v4tot);
      w->v4len.push_back((size_t)g.vol * 6);
      w->n2off.push_back(w->n2tot);
      w->n2len.push_back((size_t)g.vol * 12);
      w->vtot += g.vol;
      w->v4tot += (size_t)g.vol * 6;
      w->n2tot += (size_t)g.vol * 12;
      lat[i].block_begin = (long long)site_lat.size();
      for (long long b = 0; b < (g.vol + 127) / 128; ++b) site_lat.push_back(i);
      lat[i].df_tile_begin = (long long)tile_lat.size();
      for (long long b = 0; b < (g.vol + 63) / 64; ++b) tile_lat.push_back(i);
    }
    w->site_blocks = (long long)site_lat.size();
    w->df_tiles = (long long)tile_lat.size();
    auto upload = [](size_t** d, const std::vector<size_t>& h) {
      QCD_CUDA_CHECK(cudaMalloc(d, sizeof(size_t) * h.size()));
      QCD_CUDA_CHECK(cudaMemcpy(*d, h.data(), sizeof(size_t) * h.size(), cudaMemcpyHostToDevice));
    };
    upload(&w->d_v4off, w->v4off);
    upload(&w->d_v4len, w->v4len);
    upload(&w->d_n2off, w->n2off);
    upload(&w->d_n2len, w->n2len);
    float4** v32[] = {&w->x, &w->r, &w->p, &w->q, &w->t, &w->zp, &w->zr, &w->rt, &w->b32, &w->sap_s, &w->halo};
    for (auto v : v32) QCD_CUDA_CHECK(cudaMalloc(v, sizeof(float4) * w->v4tot));
    double2** v64[] = {&w->x64, &w->r64, &w->b64};
    for (auto v : v64) QCD_CUDA_CHECK(cudaMalloc(v, sizeof(double2) * w->n2tot));
    QCD_CUDA_CHECK(cudaMalloc(&w->xdf, sizeof(float4) * w->n2tot));
    int dev = 0, sms = 0;
    QCD_CUDA_CHECK(cudaGetDevice(&dev));
    QCD_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t vmax = *std::max_element(w->v4len.begin(), w->v4len.end());
    w->nblocks = std::max(1, std::min(2 * sms, (int)((vmax + RED_THREADS - 1) / RED_THREADS)));
    QCD_CUDA_CHECK(cudaMalloc(&w->partials, sizeof(double) * MAX_RED_OUT * w->nblocks * n));
    QCD_CUDA_CHECK(cudaMalloc(&w->counters, sizeof(unsigned) * n));
    QCD_CUDA_CHECK(cudaMemset(w->counters, 0, sizeof(unsigned) * n));
    QCD_CUDA_CHECK(cudaMalloc(&w->scal, sizeof(Scal) * n));
    QCD_CUDA_CHECK(cudaMemset(w->scal, 0, sizeof(Scal) * n));
    QCD_CUDA_CHECK(cudaMallocHost(&w->h_scal, sizeof(Scal) * n));
    QCD_CUDA_CHECK(cudaMalloc(&w->ctrl, sizeof(int) * 4));
    QCD_CUDA_CHECK(cudaMemset(w->ctrl, 0, sizeof(int) * 4));
    QCD_CUDA_CHECK(cudaMallocHost(&w->h_ctrl, sizeof(int) * 4));
    QCD_CUDA_CHECK(cudaMalloc(&w->dres, sizeof(double) * 3 * n));
    QCD_CUDA_CHECK(cudaMallocHost(&w->h_res, sizeof(double) * 3 * n));
    QCD_CUDA_CHECK(cudaMalloc(&w->d_status, sizeof(int)));
    QCD_CUDA_CHECK(cudaMemset(w->d_status, 0, sizeof(int)));
    for (int i = 0; i < n; ++i) {
      const qcd_ctx* c = ctx[i];
      LatDesc& d = lat[i];
      d.g = c->geom;
      d.g.run_flag = w->ctrl;  // operator kernels inside the loop return at once when nothing iterates
      d.kappa = (float)c->kappa;
      d.kappa64 = c->kappa;
      d.u32 = c->u32;
      QCD_REQUIRE(c->link12 != 1 || c->su3_links, QCD_ERR_STATE,
                  "batch solve with 12-real links: a lattice's links are not SU(3) to 1e-9");
      d.u32c = uses_links12(c) ? c->u32c : nullptr;
      d.cinv32 = c->cinv32;
      d.u64 = c->u64;
      d.clov64 = c->clov64;
      d.x = w->x + w->v4off[i];
      d.q = w->q + w->v4off[i];
      d.t = w->t + w->v4off[i];
      d.zp = w->zp + w->v4off[i];
      d.zr = w->zr + w->v4off[i];
      d.b32 = w->b32 + w->v4off[i];
      d.x64 = w->x64 + w->n2off[i];
      d.r64 = w->r64 + w->n2off[i];
      d.b64 = w->b64 + w->n2off[i];
      d.udf = c->udf;
      d.clovdf = c->clovdf;
      d.xdf = w->xdf + w->n2off[i];
      d.done = &w->scal[i].done;
    }
    QCD_CUDA_CHECK(cudaMalloc(&w->d_lat, sizeof(LatDesc) * n));
    QCD_CUDA_CHECK(cudaMemcpy(w->d_lat, lat.data(), sizeof(LatDesc) * n, cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaMalloc(&w->d_site_lat, sizeof(int) * site_lat.size()));
    QCD_CUDA_CHECK(cudaMemcpy(w->d_site_lat, site_lat.data(), sizeof(int) * site_lat.size(), cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaMalloc(&w->d_tile_lat, sizeof(int) * tile_lat.size()));
    QCD_CUDA_CHECK(cudaMemcpy(w->d_tile_lat, tile_lat.data(), sizeof(int) * tile_lat.size(), cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking));
    for (const qcd_ctx* c : ctx) {
      w->clover_gen.push_back(c->clover_gen);
      w->links12.push_back(uses_links12(c));
    }
  } catch (...) {
    ragged_free(w);
    throw;
  }
  wp = w;
  return w;
}

// the SAP plans for (precision, n_sap, n_jac); a change drops the captured loop
static void ragged_plans(const std::vector<qcd_ctx*>& ctx, RaggedWS* w, const qcd_solve_params& P) {
  if (w->plan_p && w->plan_prec == P.sap_prec && w->plan_nsap == P.n_sap && w->plan_njac == P.n_jac) return;
  sap_batch_free(w->plan_p);
  sap_batch_free(w->plan_r);
  w->plan_p = w->plan_r = nullptr;
  if (w->loop) cudaGraphExecDestroy(w->loop);
  w->loop = nullptr;
  std::vector<SapLat> lp(w->n), lr(w->n);
  const size_t nv = w->vtot;
  for (int i = 0; i < w->n; ++i) {
    SapLat a;
    a.ctx = ctx[i];
    a.s32 = w->sap_s + w->v4off[i];
    a.s16 = reinterpret_cast<uint4*>(w->sap_s) + 3 * w->voff[i];
    a.s16n = reinterpret_cast<float*>(reinterpret_cast<uint4*>(w->sap_s) + 3 * nv) + w->voff[i];
    a.halo = w->halo + w->v4off[i];
    a.skip = &w->scal[i].done;
    a.in = F32Spinor{w->p + w->v4off[i]};
    a.out = F32Spinor{w->zp + w->v4off[i]};
    lp[i] = a;
    a.in = F32Spinor{w->r + w->v4off[i]};
    a.out = F32Spinor{w->zr + w->v4off[i]};
    lr[i] = a;
  }
  w->plan_p = sap_batch_plan(lp, P.sap_prec, P.n_sap, P.n_jac, w->d_status, w->ctrl);
  w->plan_r = sap_batch_plan(lr, P.sap_prec, P.n_sap, P.n_jac, w->d_status, w->ctrl);
  w->plan_prec = P.sap_prec;
  w->plan_nsap = P.n_sap;
  w->plan_njac = P.n_jac;
}

static void rg_half1(qcd_ctx* c0, RaggedWS* w, cudaStream_t st) {
  const dim3 grid(w->nblocks, w->n);
  const Seg seg{0, w->d_v4off, w->d_v4len};
  sap_batch_run(w->plan_p, c0, st);
  {
    LaunchScope ls(c0, QCD_KC_DSLASH, st);
    lat_dslash_launch(w->d_lat, w->d_site_lat, w->site_blocks, 0, st);
  }
  LaunchScope ls(c0, QCD_KC_BLAS, st);
  k_alpha<<<grid, RED_THREADS, 0, st>>>(w->rt, w->q, seg, w->scal, w->partials, w->counters, w->ctrl);
  k_update1<<<grid, RED_THREADS, 0, st>>>(w->x, w->r, w->zp, w->q, seg, w->scal, w->partials, w->counters, w->ctrl);
  c0->launches++;
  check_launch();
}
static void rg_half2(qcd_ctx* c0, RaggedWS* w, cudaStream_t st) {
  const dim3 grid(w->nblocks, w->n);
  const Seg seg{0, w->d_v4off, w->d_v4len};
  sap_batch_run(w->plan_r, c0, st);
  {
    LaunchScope ls(c0, QCD_KC_DSLASH, st);
    lat_dslash_launch(w->d_lat, w->d_site_lat, w->site_blocks, 1, st);
  }
  LaunchScope ls(c0, QCD_KC_BLAS, st);
  k_omega<<<grid, RED_THREADS, 0, st>>>(w->t, w->r, seg, w->scal, w->partials, w->counters, w->ctrl);
  k_update2<<<grid, RED_THREADS, 0, st>>>(w->x, w->r, w->zp, w->zr, w->t, w->rt, seg, w->scal, w->partials,
                                         w->counters, w->ctrl);
  k_update_p<<<grid, RED_THREADS, 0, st>>>(w->p, w->r, w->q, seg, w->scal);
  c0->launches += 2;
  check_launch();
}

// the solution share x += alpha z_p of a lattice whose iteration stopped
// after the first half (k_update1)
static void rg_xfinal(qcd_ctx* c0, RaggedWS* w, cudaStream_t st) {
  LaunchScope ls(c0, QCD_KC_BLAS, st);
  k_xfinal<<<dim3(w->nblocks, w->n), RED_THREADS, 0, st>>>(w->x, w->zp, Seg{0, w->d_v4off, w->d_v4len}, w->scal);
  check_launch();
}

static bool rg_all_done(RaggedWS* w, cudaStream_t st) {
  QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(Scal) * w->n, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  for (int i = 0; i < w->n; ++i)
    if (!w->h_scal[i].done) return false;
  return true;
}

// Algorithm 5 for every lattice on A M_SAP z = b32; solutions in w->x.
// use_graph 2: the loop is one graph with a conditional while node;
// otherwise kernels are launched one by one with host checks after each
// half-iteration.  Fills w->h_scal.
static void rg_bicgstab(qcd_ctx* c0, RaggedWS* w, const qcd_solve_params& P, cudaStream_t st) {
  const dim3 grid(w->nblocks, w->n);
  const Seg seg{0, w->d_v4off, w->d_v4len};
  w->h_ctrl[0] = 0;
  w->h_ctrl[1] = 0;
  w->h_ctrl[2] = P.max_inner;
  QCD_CUDA_CHECK(cudaMemcpyAsync(w->ctrl, w->h_ctrl, sizeof(int) * 3, cudaMemcpyHostToDevice, st));
  {
    LaunchScope ls(c0, QCD_KC_BLAS, st);
    k_init<<<grid, RED_THREADS, 0, st>>>(w->b32, w->x, w->r, w->p, w->rt, seg, P.inner_tol * P.inner_tol, w->scal,
                                         w->partials, w->counters, w->ctrl);
    check_launch();
  }
  if (P.use_graph == 2) {
    if (!w->loop) {
      cudaGraph_t gr;
      const long long c_start = c0->launches;
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
      QCD_CUDA_CHECK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      rg_half1(c0, w, st);
      rg_half2(c0, w, st);
      k_loop_cond<<<1, 1, 0, st>>>(handle, w->ctrl);
      c0->launches++;
      QCD_CUDA_CHECK(cudaStreamEndCapture(st, &body));
      QCD_CUDA_CHECK(cudaGraphInstantiate(&w->loop, gr, 0));
      cudaGraphDestroy(gr);
      w->nloop = c0->launches - c_start;
      c0->launches = c_start;  // captured kernels are counted when replayed
    }
    QCD_CUDA_CHECK(cudaGraphLaunch(w->loop, st));
    rg_xfinal(c0, w, st);
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_ctrl, w->ctrl, sizeof(int) * 3, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(Scal) * w->n, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    c0->launches += (long long)w->h_ctrl[1] * w->nloop;
    return;
  }
  int it = 0;
  bool finished = rg_all_done(w, st);
  while (!finished && it < P.max_inner) {
    ++it;
    rg_half1(c0, w, st);
    if (rg_all_done(w, st)) break;
    rg_half2(c0, w, st);
    finished = rg_all_done(w, st);
  }
  rg_xfinal(c0, w, st);
  QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(Scal) * w->n, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
}

int ragged_solve(const std::vector<qcd_ctx*>& ctx, RaggedWS*& wp, double* const* x, const double* const* b,
                 int on_device, const qcd_solve_params& P, qcd_solve_info* infos, cudaStream_t user_st,
                 std::string& err) {
  const auto t0 = std::chrono::steady_clock::now();
  RaggedWS* w = ragged_ws(ctx, wp);
  ragged_plans(ctx, w, P);
  const int n = w->n;
  qcd_ctx* c0 = ctx[0];
  cudaStream_t st = w->st;
  QCD_CUDA_CHECK(cudaStreamSynchronize(user_st));  // inputs ready
  const dim3 rgrid(w->nblocks, n);
  const Seg seg64{0, w->d_n2off, w->d_n2len};
  for (int i = 0; i < n; ++i) {
    int rc = qcd_import_spinor(ctx[i], w->b64 + w->n2off[i], b[i], QCD_PREC_DOUBLE, 1, on_device, (void*)st);
    if (rc != QCD_OK) throw Error{rc, "lattice " + std::to_string(i) + ": " + ctx[i]->err};
  }
  QCD_CUDA_CHECK(cudaMemsetAsync(w->d_status, 0, sizeof(int), st));
  {
    LaunchScope ls(c0, QCD_KC_DOUBLE, st);
    k_rg_norm2_f64<<<rgrid, RED_THREADS, 0, st>>>(w->b64, seg64, w->dres, w->partials, w->counters);
    check_launch();
  }
  // D x in double-float (residual_prec 0: from a copy of x scaled by the
  // power of two of each lattice's |b|^2, written back to float64) or in
  // float64; x, r and b stay float64 either way
  auto residual = [&]() {
    if (P.residual_prec == 0) {
      LaunchScope ls(c0, QCD_KC_DOUBLE, st);
      k_rg_to_df<<<rgrid, 256, 0, st>>>(w->x64, w->xdf, seg64, w->dres);
      check_launch();
      lat_dslash_df64_launch(w->d_lat, w->d_tile_lat, w->df_tiles, w->dres, st);
    } else {
      LaunchScope ls(c0, QCD_KC_DOUBLE, st);
      lat_dslash_launch(w->d_lat, w->d_site_lat, w->site_blocks, 2, st);
    }
    LaunchScope ls(c0, QCD_KC_DOUBLE, st);
    k_rg_residual_f64<<<rgrid, RED_THREADS, 0, st>>>(w->b64, w->r64, seg64, w->dres + n, w->partials, w->counters);
    check_launch();
  };
  if (P.x_is_guess) {
    for (int i = 0; i < n; ++i) {
      int rc = qcd_import_spinor(ctx[i], w->x64 + w->n2off[i], x[i], QCD_PREC_DOUBLE, 1, on_device, (void*)st);
      if (rc != QCD_OK) throw Error{rc, "lattice " + std::to_string(i) + ": " + ctx[i]->err};
    }
    residual();
  } else {
    QCD_CUDA_CHECK(cudaMemsetAsync(w->x64, 0, sizeof(double2) * w->n2tot, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->r64, w->b64, sizeof(double2) * w->n2tot, cudaMemcpyDeviceToDevice, st));
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->dres + n, w->dres, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  }
  QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_res, w->dres, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  std::vector<double> b2(w->h_res, w->h_res + n), r2(w->h_res + n, w->h_res + 2 * n);
  std::vector<int> outer(n, 0), inner(n, 0), status(n, QCD_OK), last_inner(n, QCD_OK);
  std::vector<char> active(n, 0);
  auto rel = [&](int i) { return b2[i] > 0 ? std::sqrt(r2[i] / b2[i]) : 0.0; };
  int dev_status = QCD_OK, steps = 0;
  for (;;) {
    int nactive = 0;
    for (int i = 0; i < n; ++i) {
      active[i] = 0;
      if (status[i] != QCD_OK) continue;
      if (!std::isfinite(r2[i])) {
        status[i] = QCD_ERR_NONFINITE;
        continue;
      }
      if (rel(i) < P.tol) continue;
      if (outer[i] >= P.max_outer) {
        status[i] = last_inner[i] == QCD_ERR_BREAKDOWN ? QCD_ERR_BREAKDOWN : QCD_ERR_NOT_CONVERGED;
        continue;
      }
      active[i] = 1;
      ++nactive;
    }
    if (nactive == 0) break;
    ++steps;
    // p = R_SP(r / err) per lattice (zero for lattices that have stopped)
    for (int i = 0; i < n; ++i) w->h_res[2 * n + i] = active[i] ? 1.0 / std::sqrt(r2[i]) : 0.0;
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->dres + 2 * n, w->h_res + 2 * n, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls(c0, QCD_KC_BLAS, st);
      k_rg_prep<<<(unsigned)w->site_blocks, 128, 0, st>>>(w->d_lat, w->d_site_lat, w->dres + 2 * n);
      check_launch();
    }
    rg_bicgstab(c0, w, P, st);
    int ds = QCD_OK;
    QCD_CUDA_CHECK(cudaMemcpyAsync(&ds, w->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    if (ds == QCD_ERR_TIMEOUT) {
      dev_status = ds;
      break;
    }
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      ++outer[i];
      inner[i] += w->h_scal[i].iters;
      last_inner[i] = w->h_scal[i].status;
    }
    // x += err P_DP(q) per lattice, then r = b - D x in float64
    for (int i = 0; i < n; ++i) w->h_res[2 * n + i] = active[i] ? std::sqrt(r2[i]) : 0.0;
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->dres + 2 * n, w->h_res + 2 * n, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls(c0, QCD_KC_DOUBLE, st);
      k_rg_axpy<<<(unsigned)w->site_blocks, 128, 0, st>>>(w->d_lat, w->d_site_lat, w->dres + 2 * n);
      check_launch();
    }
    residual();
    QCD_CUDA_CHECK(cudaMemcpyAsync(w->h_res + n, w->dres + n, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) r2[i] = w->h_res[n + i];
  }
  for (int i = 0; i < n; ++i) {
    int rc = qcd_export_spinor(ctx[i], x[i], w->x64 + w->n2off[i], QCD_PREC_DOUBLE, 1, on_device, (void*)st);
    if (rc != QCD_OK) throw Error{rc, "lattice " + std::to_string(i) + ": " + ctx[i]->err};
  }
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = QCD_OK;
  for (int i = 0; i < n; ++i) {
    if (dev_status != QCD_OK) status[i] = dev_status;
    if (infos) {
      infos[i].outer_iters = outer[i];
      infos[i].inner_iters = inner[i];
      infos[i].status = status[i];
      infos[i].true_resid = rel(i);
      infos[i].seconds = secs;
    }
    if (status[i] != QCD_OK && worst == QCD_OK) {
      worst = status[i];
      err = "lattice " + std::to_string(i) + ": " +
            (status[i] == QCD_ERR_NOT_CONVERGED ? "tolerance not reached"
             : status[i] == QCD_ERR_BREAKDOWN   ? "BiCGStab breakdown"
             : status[i] == QCD_ERR_TIMEOUT     ? "a bounded device-side wait gave up"
                                                : "non-finite residual");
    }
  }
  (void)steps;
  return worst;
}

}  // namespace qcd
