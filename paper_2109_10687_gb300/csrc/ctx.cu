// Context, geometry, layout conversion and instrumentation of libqcd_gb300.
//
// The geometry follows the red/black domain decomposition of Sec. 3 of
// arXiv:2109.10687: domains coloured by the parity of the sum of their
// indices, each domain stored contiguously (see qcd_internal.cuh).

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "qcd_internal.cuh"

namespace qcd {

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
struct Profiler {
  bool enabled = false;
  struct Pending {
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending[QCD_KC_COUNT];
  std::vector<cudaEvent_t> pool;
  long long launches[QCD_KC_COUNT] = {0};
  double ms[QCD_KC_COUNT] = {0};
  cudaEvent_t cur_a[QCD_KC_COUNT] = {nullptr};

  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      QCD_CUDA_CHECK(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  void drain(int kc) {
    for (auto& p : pending[kc]) {
      QCD_CUDA_CHECK(cudaEventSynchronize(p.b));
      float t = 0.f;
      QCD_CUDA_CHECK(cudaEventElapsedTime(&t, p.a, p.b));
      ms[kc] += t;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending[kc].clear();
  }
  ~Profiler() {
    for (int k = 0; k < QCD_KC_COUNT; ++k)
      for (auto& p : pending[k]) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
      }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cs != cudaStreamCaptureStatusNone;
}

// Kernels captured into a graph are not bracketed by events (the events would
// be recorded once, at capture); their device time is not attributed.
void launch_begin(qcd_ctx* ctx, int kc, cudaStream_t st) {
  ctx->launches++;
  Profiler* p = ctx->prof;
  if (p && p->enabled && !capturing(st)) {
    p->cur_a[kc] = p->get();
    QCD_CUDA_CHECK(cudaEventRecord(p->cur_a[kc], st));
  }
}

void launch_end(qcd_ctx* ctx, int kc, cudaStream_t st) {
  Profiler* p = ctx->prof;
  if (p && p->enabled && p->cur_a[kc]) {
    cudaEvent_t b = p->get();
    cudaEventRecord(b, st);
    p->pending[kc].push_back({p->cur_a[kc], b});
    p->cur_a[kc] = nullptr;
    p->launches[kc]++;
  }
}

void workspace_free(qcd_ctx* ctx);  // solver.cu

// ---------------------------------------------------------------------------
// layout conversion kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void paper_to_chiral(cx<double> p[4], cx<double> q[4]) {
  // S = (1/sqrt 2) [[1, 1], [1, -1]] on (upper, lower) spin pairs; S^2 = 1
  const double r = 0.70710678118654752440;
  q[0] = r * (p[0] + p[2]);
  q[1] = r * (p[1] + p[3]);
  q[2] = r * (p[0] - p[2]);
  q[3] = r * (p[1] - p[3]);
}

// The canonical side of both conversions is moved through shared memory: a
// block's 128 sites are 24 KB of consecutive canonical data, read or written
// one double per thread by consecutive threads (the canonical buffer is only
// guaranteed 8-byte alignment).  Every access is fully coalesced, which
// matters most when the canonical buffer is page-locked host memory reached
// over the host link.  An odd row stride (25 doubles per site) keeps the
// per-site shared-memory accesses free of bank conflicts.
constexpr int CONV_THREADS = 128;
constexpr int CONV_STRIDE = 25;

template <int PREC>
__global__ void __launch_bounds__(CONV_THREADS) import_spinor_kernel(Geom g, void* dst, const double* __restrict__ src,
                                                                     int nrhs, int paper_basis) {
  __shared__ double buf[CONV_THREADS * CONV_STRIDE];
  const long long n0 = blockIdx.x * (long long)CONV_THREADS;
  const long long n = n0 + threadIdx.x;
  const int rhs = blockIdx.y;
  const int nsites = (int)min((long long)CONV_THREADS, g.vol - n0);
  const double* in = src + ((size_t)rhs * g.vol + n0) * 24;
  for (int i = threadIdx.x; i < nsites * 24; i += CONV_THREADS) buf[(i / 24) * CONV_STRIDE + i % 24] = in[i];
  __syncthreads();
  if (n >= g.vol) return;
  int x[4];
  site_coords(g, n, x);
  int dom, s;
  coords_to_internal(g, x, dom, s);
  const double* mine = buf + threadIdx.x * CONV_STRIDE;
  Spinor<double> a;
  for (int c = 0; c < 3; ++c) {
    cx<double> p[4], q[4];
    for (int sp = 0; sp < 4; ++sp) p[sp] = make_cx(mine[(c * 4 + sp) * 2], mine[(c * 4 + sp) * 2 + 1]);
    if (paper_basis) paper_to_chiral(p, q);
    else
      for (int sp = 0; sp < 4; ++sp) q[sp] = p[sp];
    for (int sp = 0; sp < 4; ++sp) a.v[sp][c] = q[sp];
  }
  const int domr = dom + rhs * g.ndom;  // stacked right-hand sides
  if (PREC == QCD_PREC_DOUBLE) {
    F64Spinor o{(double2*)dst};
    o.store(g, domr, s, a);
  } else {
    Spinor<float> f;
    for (int sp = 0; sp < 4; ++sp)
      for (int c = 0; c < 3; ++c) f.v[sp][c] = make_cx((float)a.v[sp][c].re, (float)a.v[sp][c].im);
    if (PREC == QCD_PREC_SINGLE) {
      F32Spinor o{(float4*)dst};
      o.store(g, domr, s, f);
    } else {
      const size_t nv = (size_t)g.vol * nrhs;
      F16Spinor o{(uint4*)dst, (float*)((uint4*)dst + 3 * nv)};
      o.store(g, domr, s, f);
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(CONV_THREADS) export_spinor_kernel(Geom g, double* __restrict__ dst, const void* src,
                                                                     int nrhs, int paper_basis) {
  __shared__ double buf[CONV_THREADS * CONV_STRIDE];
  const long long n0 = blockIdx.x * (long long)CONV_THREADS;
  const long long n = n0 + threadIdx.x;
  const int rhs = blockIdx.y;
  const int nsites = (int)min((long long)CONV_THREADS, g.vol - n0);
  if (n < g.vol) {
    int x[4];
    site_coords(g, n, x);
    int dom, s;
    coords_to_internal(g, x, dom, s);
    const int domr = dom + rhs * g.ndom;
    Spinor<double> a;
    if (PREC == QCD_PREC_DOUBLE) {
      F64Spinor i{(double2*)src};
      i.load(g, domr, s, a);
    } else {
      Spinor<float> f;
      if (PREC == QCD_PREC_SINGLE) {
        F32Spinor i{(float4*)src};
        i.load(g, domr, s, f);
      } else {
        const size_t nv = (size_t)g.vol * nrhs;
        F16Spinor i{(uint4*)src, (float*)((uint4*)src + 3 * nv)};
        i.load(g, domr, s, f);
      }
      for (int sp = 0; sp < 4; ++sp)
        for (int c = 0; c < 3; ++c) a.v[sp][c] = make_cx((double)f.v[sp][c].re, (double)f.v[sp][c].im);
    }
    double* mine = buf + threadIdx.x * CONV_STRIDE;
    for (int c = 0; c < 3; ++c) {
      cx<double> p[4], q[4];
      for (int sp = 0; sp < 4; ++sp) p[sp] = a.v[sp][c];
      if (paper_basis) paper_to_chiral(p, q);  // S is its own inverse
      else
        for (int sp = 0; sp < 4; ++sp) q[sp] = p[sp];
      for (int sp = 0; sp < 4; ++sp) {
        mine[(c * 4 + sp) * 2] = q[sp].re;
        mine[(c * 4 + sp) * 2 + 1] = q[sp].im;
      }
    }
  }
  __syncthreads();
  double* out = dst + ((size_t)rhs * g.vol + n0) * 24;
  for (int i = threadIdx.x; i < nsites * 24; i += CONV_THREADS) out[i] = buf[(i / 24) * CONV_STRIDE + i % 24];
}

// canonical gauge field -> internal float64 / float32 / float16 links, with
// an optional SU(3) check that records the worst deviation in *bad (as the
// bit pattern of a non-negative double, so integer atomicMax orders it).
__global__ void gauge_import_kernel(Geom g, const double* __restrict__ src, double2* u64, float2* u32,
                                    __half2* u16, float4* u32c, unsigned long long* bad) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.vol) return;
  int x[4];
  site_coords(g, n, x);
  int dom, s;
  coords_to_internal(g, x, dom, s);
  double worst = 0.0;
  for (int mu = 0; mu < 4; ++mu) {
    const double* in = src + (n * 4 + mu) * 18;
    cx<double> m[3][3];
    for (int e = 0; e < 9; ++e) m[e / 3][e % 3] = make_cx(in[2 * e], in[2 * e + 1]);
    const size_t base = ((size_t)((dom * 4 + mu) * 9)) << g.logvd;
    for (int e = 0; e < 9; ++e) {
      const size_t k = base + ((size_t)e << g.logvd) + s;
      u64[k] = make_double2(m[e / 3][e % 3].re, m[e / 3][e % 3].im);
      u32[k] = make_float2((float)m[e / 3][e % 3].re, (float)m[e / 3][e % 3].im);
      u16[k] = __floats2half2_rn((float)m[e / 3][e % 3].re, (float)m[e / 3][e % 3].im);
    }
    // the first two rows, three float4
    const size_t cbase = ((size_t)((dom * 4 + mu) * 3)) << g.logvd;
    for (int q = 0; q < 3; ++q) {
      const cx<double> a = m[(2 * q) / 3][(2 * q) % 3], b = m[(2 * q + 1) / 3][(2 * q + 1) % 3];
      u32c[cbase + ((size_t)q << g.logvd) + s] = make_float4((float)a.re, (float)a.im, (float)b.re, (float)b.im);
    }
    // |U^dag U - 1| and |det U - 1|
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        cx<double> acc = make_cx(0.0, 0.0);
        for (int k = 0; k < 3; ++k) acc = cmacc(acc, m[k][i], m[k][j]);
        if (i == j) acc.re -= 1.0;
        worst = fmax(worst, fabs(acc.re) + fabs(acc.im));
      }
    cx<double> det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                     m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                     m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    worst = fmax(worst, fabs(det.re - 1.0) + fabs(det.im));
  }
  if (!(worst == worst)) worst = 1e300;  // NaN
  atomicMax(bad, (unsigned long long)__double_as_longlong(worst));
}

}  // namespace qcd

using namespace qcd;

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
static thread_local std::string g_create_error;  // per calling thread

#define QCD_API_BEGIN(ctx) \
  try {
#define QCD_API_END(ctx)                                          \
  }                                                               \
  catch (const qcd::Error& e) {                                   \
    if (ctx) (ctx)->err = e.msg;                                  \
    return e.code;                                                \
  }                                                               \
  catch (const std::exception& e) {                               \
    if (ctx) (ctx)->err = e.what();                               \
    return QCD_ERR_CUDA;                                          \
  }                                                               \
  catch (...) {                                                   \
    if (ctx) (ctx)->err = "unknown error";                        \
    return QCD_ERR_CUDA;                                          \
  }                                                               \
  return QCD_OK;

static int ilog2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

extern "C" const char* qcd_version(void) { return "qcd_gb300 1.0"; }

extern "C" const char* qcd_last_error(const qcd_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" int qcd_create(const int dims[4], const int domain[4], int bc_t, int basis, qcd_ctx** out) {
  if (!out || !dims) {
    g_create_error = "qcd_create: null argument";
    return QCD_ERR_ARG;
  }
  *out = nullptr;
  qcd_ctx* ctx = new qcd_ctx();
  try {
    Geom& g = ctx->geom;
    const int defd[4] = {4, 4, 4, 4};
    const int* dd = domain ? domain : defd;
    g.vd = 1;
    int sh = 0;
    for (int mu = 0; mu < 4; ++mu) {
      g.L[mu] = dims[mu];
      g.d[mu] = dd[mu];
      QCD_REQUIRE(g.L[mu] > 0 && g.d[mu] > 0, QCD_ERR_ARG, "lattice and domain extents must be positive");
      g.logd[mu] = ilog2_exact(g.d[mu]);
      QCD_REQUIRE(g.logd[mu] >= 0, QCD_ERR_ARG, "domain extents must be powers of two");
      QCD_REQUIRE(g.L[mu] % (2 * g.d[mu]) == 0, QCD_ERR_ARG,
                  "every lattice extent must be a multiple of twice the domain extent");
      g.nd[mu] = g.L[mu] / g.d[mu];
      g.shift[mu] = sh;
      sh += g.logd[mu];
      g.vd *= g.d[mu];
    }
    QCD_REQUIRE(g.vd <= 256, QCD_ERR_ARG, "at most 256 sites per domain");
    QCD_REQUIRE(bc_t == 1 || bc_t == -1, QCD_ERR_ARG, "bc_t must be +1 or -1");
    QCD_REQUIRE(basis == QCD_BASIS_CHIRAL || basis == QCD_BASIS_PAPER, QCD_ERR_ARG, "unknown basis");
    g.logvd = sh;
    g.vol = (long long)g.L[0] * g.L[1] * g.L[2] * g.L[3];
    QCD_REQUIRE(g.vol * 24LL * 16LL < (1LL << 62), QCD_ERR_ARG, "lattice too large");
    g.ndom = (int)(g.vol / g.vd);
    g.nhalf = g.ndom / 2;
    g.bc_t = bc_t;
    ctx->basis = basis;
    QCD_CUDA_CHECK(cudaGetDevice(&ctx->device));

    // domain neighbour table, colour-major domain numbering
    std::vector<int> id_of_lex(g.ndom), nbr((size_t)g.ndom * 8);
    std::vector<unsigned char> tflag(g.ndom, 0);
    std::vector<int> lex_of_id(g.ndom);
    for (int lex = 0; lex < g.ndom; ++lex) {
      int r = lex, dc[4];
      for (int mu = 0; mu < 4; ++mu) {
        dc[mu] = r % g.nd[mu];
        r /= g.nd[mu];
      }
      const int colour = (dc[0] + dc[1] + dc[2] + dc[3]) & 1;
      const int id = colour * g.nhalf + (lex >> 1);
      id_of_lex[lex] = id;
      lex_of_id[id] = lex;
    }
    for (int id = 0; id < g.ndom; ++id) {
      int r = lex_of_id[id], dc[4];
      for (int mu = 0; mu < 4; ++mu) {
        dc[mu] = r % g.nd[mu];
        r /= g.nd[mu];
      }
      for (int mu = 0; mu < 4; ++mu)
        for (int dir = 0; dir < 2; ++dir) {
          int e[4] = {dc[0], dc[1], dc[2], dc[3]};
          e[mu] = (e[mu] + (dir == 0 ? 1 : g.nd[mu] - 1)) % g.nd[mu];
          const int lex = ((e[3] * g.nd[2] + e[2]) * g.nd[1] + e[1]) * g.nd[0] + e[0];
          nbr[(size_t)id * 8 + 2 * mu + dir] = id_of_lex[lex];
        }
      if (dc[3] == g.nd[3] - 1) tflag[id] |= 1 << 6;
      if (dc[3] == 0) tflag[id] |= 1 << 7;
    }
    QCD_CUDA_CHECK(cudaMalloc(&ctx->d_nbr, nbr.size() * sizeof(int)));
    QCD_CUDA_CHECK(cudaMemcpy(ctx->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->d_lex2dom, id_of_lex.size() * sizeof(int)));
    QCD_CUDA_CHECK(cudaMemcpy(ctx->d_lex2dom, id_of_lex.data(), id_of_lex.size() * sizeof(int),
                              cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->d_tflag, tflag.size()));
    QCD_CUDA_CHECK(cudaMemcpy(ctx->d_tflag, tflag.data(), tflag.size(), cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->d_status, 64));
    QCD_CUDA_CHECK(cudaMemset(ctx->d_status, 0, 64));
    g.nbr = ctx->d_nbr;
    g.tflag = ctx->d_tflag;
    g.lex2dom = ctx->d_lex2dom;
    g.run_flag = nullptr;
    ctx->prof = new Profiler();
  } catch (const qcd::Error& e) {
    g_create_error = e.msg;
    qcd_destroy(ctx);
    return e.code;
  }
  *out = ctx;
  return QCD_OK;
}

extern "C" int qcd_destroy(qcd_ctx* ctx) {
  if (!ctx) return QCD_OK;
  workspace_free(ctx);
  tuner_free(ctx);
  void* ptrs[] = {ctx->d_nbr, ctx->d_lex2dom, ctx->d_tflag, ctx->u64, ctx->u32, ctx->u16, ctx->clov64,
                  ctx->clov32, ctx->cinv64, ctx->cinv32, ctx->cinv16, ctx->d_status,
                  ctx->st_link16, ctx->st_link32, ctx->st_clov16, ctx->st_clov32, ctx->udf, ctx->clovdf,
                  ctx->cl_link, ctx->cl_clov, ctx->flow_state, ctx->u32c};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  delete ctx->prof;
  delete ctx;
  return QCD_OK;
}

static void ensure_alloc(void** p, size_t bytes) {
  if (!*p) QCD_CUDA_CHECK(cudaMalloc(p, bytes));
}

extern "C" int qcd_set_gauge(qcd_ctx* ctx, const double* U, int on_device, double check_tol, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  QCD_REQUIRE(U, QCD_ERR_ARG, "qcd_set_gauge: null U");
  const Geom& g = ctx->geom;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nlink = (size_t)g.vol * 4 * 9;
  ensure_alloc((void**)&ctx->u64, nlink * sizeof(double2));
  ensure_alloc((void**)&ctx->u32, nlink * sizeof(float2));
  ensure_alloc((void**)&ctx->u16, nlink * sizeof(__half2));
  ensure_alloc((void**)&ctx->u32c, (size_t)g.vol * 4 * 3 * sizeof(float4));
  const double* src = U;
  double* tmp = nullptr;
  if (!on_device) {
    QCD_CUDA_CHECK(cudaMalloc(&tmp, nlink * 2 * sizeof(double)));
    QCD_CUDA_CHECK(cudaMemcpyAsync(tmp, U, nlink * 2 * sizeof(double), cudaMemcpyHostToDevice, st));
    src = tmp;
  }
  unsigned long long* bad = (unsigned long long*)ctx->d_status + 1;
  QCD_CUDA_CHECK(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st));
  {
    LaunchScope ls(ctx, QCD_KC_OTHER, st);
    gauge_import_kernel<<<grid_for(g.vol, 128), 128, 0, st>>>(g, src, ctx->u64, ctx->u32, ctx->u16, ctx->u32c, bad);
    check_launch();
  }
  unsigned long long hbad = 0;
  QCD_CUDA_CHECK(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  if (tmp) cudaFree(tmp);
  double worst;
  std::memcpy(&worst, &hbad, sizeof(worst));
  ctx->have_gauge = true;
  ctx->have_clover = false;
  ctx->su3_links = worst <= 1e-9;
  if (check_tol > 0 && !(worst <= check_tol)) {
    ctx->have_gauge = false;
    char buf[160];
    std::snprintf(buf, sizeof buf, "qcd_set_gauge: links deviate from SU(3) by %.3e > %.3e", worst, check_tol);
    throw qcd::Error{QCD_ERR_ARG, buf};
  }
  QCD_API_END(ctx)
}

extern "C" int qcd_set_params(qcd_ctx* ctx, double kappa, double csw) {
  if (!ctx) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  QCD_REQUIRE(std::isfinite(kappa) && std::isfinite(csw), QCD_ERR_ARG, "kappa and csw must be finite");
  ctx->kappa = kappa;
  ctx->csw = csw;
  ctx->have_clover = false;
  QCD_API_END(ctx)
}

extern "C" int qcd_build_clover(qcd_ctx* ctx, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  QCD_REQUIRE(ctx->have_gauge, QCD_ERR_STATE, "qcd_build_clover: no gauge field set");
  const Geom& g = ctx->geom;
  const size_t v = (size_t)g.vol;
  ensure_alloc((void**)&ctx->clov64, v * 36 * sizeof(double2));
  ensure_alloc((void**)&ctx->cinv64, v * 36 * sizeof(double2));
  ensure_alloc((void**)&ctx->clov32, v * 18 * sizeof(float4));
  ensure_alloc((void**)&ctx->cinv32, v * 18 * sizeof(float4));
  ensure_alloc((void**)&ctx->cinv16, v * 36 * sizeof(__half2));
  cudaStream_t st = (cudaStream_t)stream;
  QCD_CUDA_CHECK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  build_clover_launch(ctx, st);
  build_sap_staging(ctx, st);
  build_df64_copies(ctx, true, true, st);
  int hs = 0;
  QCD_CUDA_CHECK(cudaMemcpyAsync(&hs, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  QCD_REQUIRE(hs == 0, QCD_ERR_NONFINITE, "qcd_build_clover: singular or non-finite clover block");
  ctx->have_clover = true;
  ++ctx->clover_gen;
  QCD_API_END(ctx)
}

extern "C" int qcd_field_bytes(const qcd_ctx* ctx, int prec, int nrhs, size_t* bytes) {
  if (!ctx || !bytes || nrhs < 1 || prec < 0 || prec > 2) return QCD_ERR_ARG;
  *bytes = spinor_bytes(ctx->geom, prec) * (size_t)nrhs;
  return QCD_OK;
}

// Device address through which kernels can read or write a page-locked host
// buffer directly (mapped pinned memory; null for pageable memory).  Host
// data in a pinned buffer then crosses the host link once, inside the
// import or export kernel, with no staging copy in device memory.
static const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();  // clear the (non-sticky) error left by the query
    return nullptr;
  }
  return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

extern "C" int qcd_import_spinor(qcd_ctx* ctx, void* dst, const double* src, int prec, int nrhs,
                                 int src_on_device, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  QCD_REQUIRE(dst && src && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_import_spinor: bad arguments");
  QCD_REQUIRE(prec >= 0 && prec <= 2, QCD_ERR_ARG, "qcd_import_spinor: bad precision");
  const Geom& g = ctx->geom;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)g.vol * 24 * sizeof(double) * nrhs;
  const double* s = src;
  double* tmp = nullptr;
  if (!src_on_device) {
    if (const void* m = mapped_host_ptr(src)) {
      s = static_cast<const double*>(m);
    } else {
      QCD_CUDA_CHECK(cudaMalloc(&tmp, bytes));
      QCD_CUDA_CHECK(cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, st));
      s = tmp;
    }
  }
  dim3 grid(grid_for(g.vol, CONV_THREADS), nrhs);
  {
    LaunchScope ls(ctx, QCD_KC_OTHER, st);
    const int pb = ctx->basis == QCD_BASIS_PAPER;
    if (prec == QCD_PREC_DOUBLE)
      import_spinor_kernel<QCD_PREC_DOUBLE><<<grid, CONV_THREADS, 0, st>>>(g, dst, s, nrhs, pb);
    else if (prec == QCD_PREC_SINGLE)
      import_spinor_kernel<QCD_PREC_SINGLE><<<grid, CONV_THREADS, 0, st>>>(g, dst, s, nrhs, pb);
    else
      import_spinor_kernel<QCD_PREC_HALF><<<grid, CONV_THREADS, 0, st>>>(g, dst, s, nrhs, pb);
    check_launch();
  }
  if (!src_on_device) {
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));  // the host buffer may be reused on return
    if (tmp) cudaFree(tmp);
  }
  QCD_API_END(ctx)
}

extern "C" int qcd_export_spinor(qcd_ctx* ctx, double* dst, const void* src, int prec, int nrhs,
                                 int dst_on_device, void* stream) {
  if (!ctx) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  QCD_REQUIRE(dst && src && nrhs >= 1 && nrhs <= 65535, QCD_ERR_ARG, "qcd_export_spinor: bad arguments");
  QCD_REQUIRE(prec >= 0 && prec <= 2, QCD_ERR_ARG, "qcd_export_spinor: bad precision");
  const Geom& g = ctx->geom;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)g.vol * 24 * sizeof(double) * nrhs;
  double* d = dst;
  double* tmp = nullptr;
  if (!dst_on_device) {
    if (const void* m = mapped_host_ptr(dst)) {
      d = static_cast<double*>(const_cast<void*>(m));
    } else {
      QCD_CUDA_CHECK(cudaMalloc(&tmp, bytes));
      d = tmp;
    }
  }
  dim3 grid(grid_for(g.vol, CONV_THREADS), nrhs);
  {
    LaunchScope ls(ctx, QCD_KC_OTHER, st);
    const int pb = ctx->basis == QCD_BASIS_PAPER;
    if (prec == QCD_PREC_DOUBLE)
      export_spinor_kernel<QCD_PREC_DOUBLE><<<grid, CONV_THREADS, 0, st>>>(g, d, src, nrhs, pb);
    else if (prec == QCD_PREC_SINGLE)
      export_spinor_kernel<QCD_PREC_SINGLE><<<grid, CONV_THREADS, 0, st>>>(g, d, src, nrhs, pb);
    else
      export_spinor_kernel<QCD_PREC_HALF><<<grid, CONV_THREADS, 0, st>>>(g, d, src, nrhs, pb);
    check_launch();
  }
  if (tmp) {
    QCD_CUDA_CHECK(cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, st));
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));
    cudaFree(tmp);
  } else if (!dst_on_device) {
    QCD_CUDA_CHECK(cudaStreamSynchronize(st));  // the host buffer is complete on return
  }
  QCD_API_END(ctx)
}

extern "C" int qcd_profile_enable(qcd_ctx* ctx, int enable) {
  if (!ctx) return QCD_ERR_ARG;
  ctx->prof->enabled = enable != 0;
  return QCD_OK;
}

extern "C" int qcd_profile_read(qcd_ctx* ctx, int kc, long long* launches, double* ms, int reset) {
  if (!ctx || kc < 0 || kc >= QCD_KC_COUNT) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  ctx->prof->drain(kc);
  if (launches) *launches = ctx->prof->launches[kc];
  if (ms) *ms = ctx->prof->ms[kc];
  if (reset) {
    ctx->prof->launches[kc] = 0;
    ctx->prof->ms[kc] = 0;
  }
  QCD_API_END(ctx)
}

extern "C" int qcd_device_status(qcd_ctx* ctx, int* status, int reset, void* stream) {
  if (!ctx || !status) return QCD_ERR_ARG;
  QCD_API_BEGIN(ctx)
  cudaStream_t st = (cudaStream_t)stream;
  int hs = 0;
  QCD_CUDA_CHECK(cudaMemcpyAsync(&hs, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (reset) QCD_CUDA_CHECK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  QCD_CUDA_CHECK(cudaStreamSynchronize(st));
  *status = hs;
  QCD_API_END(ctx)
}

extern "C" int qcd_test_inject(qcd_ctx* ctx, int what) {
  if (!ctx || what < QCD_INJECT_NONE || what > QCD_INJECT_HALO_WAIT) return QCD_ERR_ARG;
  ctx->inject = what;
  return QCD_OK;
}

extern "C" int qcd_launch_count(const qcd_ctx* ctx, long long* count) {
  if (!ctx || !count) return QCD_ERR_ARG;
  *count = ctx->launches;
  return QCD_OK;
}
