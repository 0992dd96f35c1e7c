// Ragged batches of lattices: several contexts (lattices of different sizes,
// gauge fields, kappa and c_SW) handled together.
//
// qcd_batch_apply_D applies every lattice's float32 operator in one kernel
// launch through a work list: each lattice owns a contiguous range of blocks
// and its descriptor (geometry, field pointers, kappa).  qcd_batch_solve
// solves every lattice in shared launches (ragged.cu): each SAP half-sweep,
// operator application and BLAS-1 step of an iteration is one launch over
// all lattices.  Batches the shared launches do not cover (a lattice without
// 4^4 domains, the flexible GMRES outer solver, the double-float residual)
// run the lattices' solves concurrently instead, one host thread and one
// stream per lattice.

#include <thread>
#include <vector>

#include "qcd_internal.cuh"

struct qcd_batch {
  std::vector<qcd_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  qcd::BatchDesc* d_desc = nullptr;
  qcd::BatchDesc* h_desc = nullptr;  // pinned staging of the descriptors
  cudaEvent_t desc_free = nullptr;   // the previous descriptor copy has completed
  int* d_block_lat = nullptr;        // lattice of every block of the one-launch D
  long long nblocks = 0;
  qcd::RaggedWS* rws = nullptr;      // buffers of the shared-launch solve
  bool shared = true;                // solve in shared launches where supported
  std::string err;
};

using namespace qcd;

extern "C" int qcd_batch_create(int n, qcd_ctx* const* ctxs, qcd_batch** out) {
  if (!out || n < 1 || !ctxs) return QCD_ERR_ARG;
  *out = nullptr;
  qcd_batch* b = new qcd_batch();
  try {
    int dev0 = -1;
    for (int i = 0; i < n; ++i) {
      QCD_REQUIRE(ctxs[i], QCD_ERR_ARG, "qcd_batch_create: null context");
      if (i == 0) dev0 = ctxs[i]->device;
      QCD_REQUIRE(ctxs[i]->device == dev0, QCD_ERR_ARG, "qcd_batch_create: contexts on different devices");
      for (int j = 0; j < i; ++j) QCD_REQUIRE(ctxs[j] != ctxs[i], QCD_ERR_ARG, "qcd_batch_create: repeated context");
      b->ctx.push_back(ctxs[i]);
      cudaStream_t s;
      QCD_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      b->streams.push_back(s);
    }
    QCD_CUDA_CHECK(cudaMalloc(&b->d_desc, sizeof(BatchDesc) * n));
    QCD_CUDA_CHECK(cudaMallocHost(&b->h_desc, sizeof(BatchDesc) * n));
    QCD_CUDA_CHECK(cudaEventCreateWithFlags(&b->desc_free, cudaEventDisableTiming));
    QCD_CUDA_CHECK(cudaEventRecord(b->desc_free, 0));
  } catch (const qcd::Error& e) {
    qcd_batch_destroy(b);
    return e.code;
  }
  *out = b;
  return QCD_OK;
}

extern "C" int qcd_batch_destroy(qcd_batch* b) {
  if (!b) return QCD_OK;
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->h_desc) cudaFreeHost(b->h_desc);
  if (b->desc_free) cudaEventDestroy(b->desc_free);
  if (b->d_block_lat) cudaFree(b->d_block_lat);
  qcd::ragged_free(b->rws);
  delete b;
  return QCD_OK;
}

extern "C" int qcd_batch_set_shared(qcd_batch* b, int enable) {
  if (!b) return QCD_ERR_ARG;
  b->shared = enable != 0;
  return QCD_OK;
}

extern "C" const char* qcd_batch_last_error(const qcd_batch* b) { return b ? b->err.c_str() : ""; }

extern "C" int qcd_batch_apply_D(qcd_batch* b, void* const* out, const void* const* in, int dagger, void* stream) {
  if (!b) return QCD_ERR_ARG;
  try {
    QCD_REQUIRE(out && in, QCD_ERR_ARG, "qcd_batch_apply_D: null arrays");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->ctx.size();
    // the pinned staging may still feed the previous call's copy
    QCD_CUDA_CHECK(cudaEventSynchronize(b->desc_free));
    long long blocks = 0;
    for (int i = 0; i < n; ++i) {
      qcd_ctx* c = b->ctx[i];
      QCD_REQUIRE(c->have_gauge && c->have_clover, QCD_ERR_STATE, "qcd_batch_apply_D: a lattice has no operator");
      QCD_REQUIRE(out[i] && in[i] && out[i] != in[i], QCD_ERR_ARG, "qcd_batch_apply_D: bad field pointers");
      BatchDesc& d = b->h_desc[i];
      d.g = c->geom;
      d.out = (float4*)out[i];
      d.in = (const float4*)in[i];
      d.u = c->u32;
      QCD_REQUIRE(c->link12 != 1 || c->su3_links, QCD_ERR_STATE,
                  "batched D with 12-real links: a lattice's links are not SU(3) to 1e-9");
      d.u12 = uses_links12(c) ? c->u32c : nullptr;
      d.clov = c->clov32;
      d.kappa = (float)c->kappa;
      d.block_begin = blocks;
      blocks += (c->geom.vol + 127) / 128;
    }
    if (!b->d_block_lat) {
      // the geometries are fixed for the batch's lifetime: build the table once
      std::vector<int> lat((size_t)blocks);
      for (int i = 0; i < n; ++i) {
        const long long end = i + 1 < n ? b->h_desc[i + 1].block_begin : blocks;
        for (long long k = b->h_desc[i].block_begin; k < end; ++k) lat[(size_t)k] = i;
      }
      QCD_CUDA_CHECK(cudaMalloc(&b->d_block_lat, sizeof(int) * lat.size()));
      QCD_CUDA_CHECK(cudaMemcpy(b->d_block_lat, lat.data(), sizeof(int) * lat.size(), cudaMemcpyHostToDevice));
      b->nblocks = blocks;
    }
    QCD_REQUIRE(b->nblocks == blocks, QCD_ERR_STATE, "qcd_batch_apply_D: lattice sizes changed");
    QCD_CUDA_CHECK(cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(BatchDesc) * n, cudaMemcpyHostToDevice, st));
    QCD_CUDA_CHECK(cudaEventRecord(b->desc_free, st));
    {
      LaunchScope ls(b->ctx[0], QCD_KC_DSLASH, st);
      dslash_batch_launch(b->d_desc, b->d_block_lat, blocks, dagger, st);
    }
  } catch (const qcd::Error& e) {
    b->err = e.msg;
    return e.code;
  }
  return QCD_OK;
}

extern "C" int qcd_batch_solve(qcd_batch* b, double* const* x, const double* const* rhs, int on_device,
                               const qcd_solve_params* params, qcd_solve_info* infos, void* stream) {
  if (!b) return QCD_ERR_ARG;
  try {
    QCD_REQUIRE(x && rhs, QCD_ERR_ARG, "qcd_batch_solve: null arrays");
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i) QCD_REQUIRE(x[i] && rhs[i], QCD_ERR_ARG, "qcd_batch_solve: null field pointer");
    qcd_solve_params P;
    if (params) P = *params;
    else qcd_solve_params_default(&P);
    QCD_REQUIRE(P.tol > 0 && P.inner_tol > 0 && P.max_outer >= 1 && P.max_inner >= 1 && P.n_sap >= 0 && P.n_jac >= 1,
                QCD_ERR_ARG, "qcd_batch_solve: bad parameters");
    QCD_REQUIRE(P.sap_prec == QCD_PREC_SINGLE || P.sap_prec == QCD_PREC_HALF || P.sap_prec == QCD_PREC_HALF_GAUGE,
                QCD_ERR_ARG, "qcd_batch_solve: sap_prec must be SINGLE, HALF or HALF_GAUGE");
    if (b->shared && ragged_eligible(b->ctx, P)) {
      const int rc = ragged_solve(b->ctx, b->rws, x, rhs, on_device, P, infos, (cudaStream_t)stream, b->err);
      return rc;
    }
    QCD_CUDA_CHECK(cudaStreamSynchronize((cudaStream_t)stream));  // inputs ready before the lattices start
    std::vector<int> rc(n, QCD_OK);
    std::vector<qcd_solve_info> info(n);
    int dev = b->ctx[0]->device;
    std::vector<std::thread> th;
    th.reserve(n);
    for (int i = 0; i < n; ++i)
      th.emplace_back([&, i]() {
        cudaSetDevice(dev);
        rc[i] = qcd_solve(b->ctx[i], x[i], rhs[i], 1, on_device, params, &info[i], (void*)b->streams[i]);
      });
    for (auto& t : th) t.join();
    int worst = QCD_OK;
    for (int i = 0; i < n; ++i) {
      if (infos) infos[i] = info[i];
      if (rc[i] != QCD_OK && worst == QCD_OK) {
        worst = rc[i];
        b->err = "lattice " + std::to_string(i) + ": " + b->ctx[i]->err;
      }
    }
    return worst;
  } catch (const qcd::Error& e) {
    b->err = e.msg;
    return e.code;
  } catch (...) {
    b->err = "qcd_batch_solve: unknown error";
    return QCD_ERR_CUDA;
  }
}
