// Launch-shape autotuner: for kernels with several compiled launch shapes
// (threads per block, register budget, blocks per SM) the first launch with
// a given key times each shape on the real arguments with CUDA events and
// keeps the fastest.  The shapes differ only in scheduling, never in the
// arithmetic each site performs.

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdlib>
#include <vector>
#include <cstdio>
#include <map>
#include <string>

#include "qcd_internal.cuh"

namespace qcd {

struct Tuner {
  bool enabled = true;
  struct Entry {
    int variant;
    float ms;
    std::string name;
    std::string all;  // every shape tried: "name ms, ..."
  };
  std::map<std::string, Entry> best;
};

static Tuner* tuner_of(qcd_ctx* ctx) {
  if (!ctx->tuner) ctx->tuner = new Tuner();
  return ctx->tuner;
}

void tuner_free(qcd_ctx* ctx) {
  delete ctx->tuner;
  ctx->tuner = nullptr;
}

int tune_pick(qcd_ctx* ctx, const char* key, int nvariants, const char* const* names,
              const std::function<void(int)>& run, cudaStream_t st) {
  Tuner* t = tuner_of(ctx);
  auto it = t->best.find(key);
  if (it != t->best.end()) return it->second.variant;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (!t->enabled || cs != cudaStreamCaptureStatusNone || nvariants <= 1) return 0;
  cudaEvent_t a, b;
  QCD_CUDA_CHECK(cudaEventCreate(&a));
  QCD_CUDA_CHECK(cudaEventCreate(&b));
  int best_v = 0;
  float best_ms = 1e30f;
  std::string all;
  for (int v = 0; v < nvariants; ++v) {
    run(v);  // warm-up
    QCD_CUDA_CHECK(cudaEventRecord(a, st));
    for (int r = 0; r < 3; ++r) run(v);
    QCD_CUDA_CHECK(cudaEventRecord(b, st));
    QCD_CUDA_CHECK(cudaEventSynchronize(b));
    float ms = 0.f;
    QCD_CUDA_CHECK(cudaEventElapsedTime(&ms, a, b));
    ms /= 3.f;
    char item[96];
    std::snprintf(item, sizeof item, "%s%s %.4f", v ? ", " : "", names ? names[v] : std::to_string(v).c_str(), ms);
    all += item;
    if (ms < best_ms) {
      best_ms = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->launches += 4LL * nvariants;
  t->best[key] = {best_v, best_ms, names ? names[best_v] : std::to_string(best_v), all};
  return best_v;
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_set_tuning(qcd_ctx* ctx, int enable) {
  if (!ctx) return QCD_ERR_ARG;
  tuner_of(ctx)->enabled = enable != 0;
  if (!enable) tuner_of(ctx)->best.clear();
  return QCD_OK;
}

// ---------------------------------------------------------------------------
// domain-shape autotuner (time to solution)
// ---------------------------------------------------------------------------
// The SAP domain fixes the context's field layout, so each candidate shape
// gets a temporary context: gauge field, parameters and clover term set up,
// one solve to warm it (allocations and the kernel tuners), then one timed
// solve.  A candidate that does not fit the lattice, or whose solve misses
// the tolerance, is skipped (seconds = -1).
static std::vector<std::array<int, 4>> default_domains() {
  return {{4, 4, 4, 4}, {8, 4, 4, 2}, {2, 4, 4, 8}, {4, 4, 2, 4}, {8, 8, 2, 2}, {4, 4, 4, 2}, {2, 2, 2, 2}};
}

extern "C" int qcd_tune_domain(const int dims[4], int bc_t, int basis, const double* U, const double* b,
                               int on_device, double kappa, double csw, const qcd_solve_params* params,
                               const int* candidates, int n, int best_domain[4], double* seconds) {
  if (!dims || !U || !b || !best_domain || n < 0 || (n > 0 && !candidates)) return QCD_ERR_ARG;
  std::vector<std::array<int, 4>> cand;
  if (n > 0) {
    for (int k = 0; k < n; ++k)
      cand.push_back({candidates[4 * k], candidates[4 * k + 1], candidates[4 * k + 2], candidates[4 * k + 3]});
  } else {
    cand = default_domains();
  }
  qcd_solve_params P;
  if (params) P = *params;
  else qcd_solve_params_default(&P);
  long long vol = 1;
  for (int mu = 0; mu < 4; ++mu) vol *= dims[mu];
  const size_t bytes = (size_t)vol * 24 * sizeof(double);
  double* x = nullptr;
  if (on_device) {
    if (cudaMalloc(&x, bytes) != cudaSuccess) return QCD_ERR_OOM;
  } else {
    x = static_cast<double*>(std::malloc(bytes));
    if (!x) return QCD_ERR_OOM;
  }
  double best = -1.0;
  int result = QCD_ERR_ARG;  // until some candidate succeeds
  for (size_t k = 0; k < cand.size(); ++k) {
    double t = -1.0;
    qcd_ctx* c = nullptr;
    if (qcd_create(dims, cand[k].data(), bc_t, basis, &c) == QCD_OK) {
      int rc = qcd_set_gauge(c, U, on_device, 0.0, nullptr);
      if (rc == QCD_OK) rc = qcd_set_params(c, kappa, csw);
      if (rc == QCD_OK) rc = qcd_build_clover(c, nullptr);
      qcd_solve_info info;
      if (rc == QCD_OK) rc = qcd_solve(c, x, b, 1, on_device, &P, &info, nullptr);
      if (rc == QCD_OK) {
        const auto t0 = std::chrono::steady_clock::now();
        rc = qcd_solve(c, x, b, 1, on_device, &P, &info, nullptr);
        if (rc == QCD_OK) t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      }
      qcd_destroy(c);
    }
    if (seconds && k < (size_t)(n > 0 ? n : (int)cand.size())) seconds[k] = t;
    if (t >= 0.0 && (best < 0.0 || t < best)) {
      best = t;
      for (int mu = 0; mu < 4; ++mu) best_domain[mu] = cand[k][mu];
      result = QCD_OK;
    }
  }
  if (on_device) cudaFree(x);
  else std::free(x);
  cudaGetLastError();  // a rejected candidate leaves no error behind
  return result;
}

extern "C" int qcd_tune_domain_default_count(void) { return (int)default_domains().size(); }

extern "C" int qcd_set_link_compression(qcd_ctx* ctx, int mode) {
  if (!ctx || mode < -1 || mode > 1) return QCD_ERR_ARG;
  ctx->link12 = mode;
  workspace_reset_graphs(ctx);
  return QCD_OK;
}

extern "C" int qcd_link_format(const qcd_ctx* ctx, int* reals) {
  if (!ctx || !reals) return QCD_ERR_ARG;
  *reals = uses_links12(ctx) ? 12 : 18;
  return QCD_OK;
}

extern "C" int qcd_set_sap_shape(qcd_ctx* ctx, int shape) {
  if (!ctx || shape < -1 || shape > 4) return QCD_ERR_ARG;
  ctx->sap_shape = shape;
  return QCD_OK;
}

extern "C" int qcd_tuning_report(qcd_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return QCD_ERR_ARG;
  std::string out;
  for (auto& kv : tuner_of(ctx)->best) {
    char line[256];
    std::snprintf(line, sizeof line, "%s %s %.4f ms", kv.first.c_str(), kv.second.name.c_str(), kv.second.ms);
    out += line;
    out += " [" + kv.second.all + "]\n";
  }
  std::snprintf(buf, len, "%s", out.c_str());
  return QCD_OK;
}

// ---------------------------------------------------------------------------
// float32 FMA throughput (measurement utility)
// ---------------------------------------------------------------------------
namespace qcd {
constexpr int FMA_CHAINS = 8;
constexpr int FMA_UNROLL = 32;

// each thread runs FMA_CHAINS independent chains x <- x a + b; with a < 1
// and b > 0 the values stay in a normal range.  The result is stored only
// if it equals a value it cannot reach, which keeps the work live.
__global__ void __launch_bounds__(256) fma_peak_kernel(float* out, int iters, float a, float b) {
  float x[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) x[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < FMA_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
  }
  float sum = 0.f;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) sum += x[c];
  if (sum == -1.0f) out[blockIdx.x] = sum;
}
}  // namespace qcd

extern "C" int qcd_measure_fp32_peak(qcd_ctx* ctx, double* tflops, void* stream) {
  if (!ctx || !tflops) return QCD_ERR_ARG;
  try {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    QCD_CUDA_CHECK(cudaGetDevice(&dev));
    QCD_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * 8, threads = 256, iters = 2048;
    float* out = nullptr;
    QCD_CUDA_CHECK(cudaMalloc(&out, sizeof(float) * blocks));
    cudaEvent_t e0, e1;
    QCD_CUDA_CHECK(cudaEventCreate(&e0));
    QCD_CUDA_CHECK(cudaEventCreate(&e1));
    fma_peak_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999f, 1e-3f);
    double best = 0.0;
    for (int r = 0; r < 3; ++r) {
      QCD_CUDA_CHECK(cudaEventRecord(e0, st));
      fma_peak_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999f, 1e-3f);
      QCD_CUDA_CHECK(cudaEventRecord(e1, st));
      QCD_CUDA_CHECK(cudaEventSynchronize(e1));
      float ms = 0.f;
      QCD_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
      const double flop = 2.0 * blocks * threads * (double)iters * FMA_UNROLL * FMA_CHAINS;
      if (ms > 0.f) best = std::max(best, flop / (ms * 1e-3) / 1e12);
    }
    ctx->launches += 4;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    check_launch();
    *tflops = best;
  } catch (const Error& e) {
    ctx->err = e.msg;
    return e.code;
  } catch (...) {
    ctx->err = "unknown error";
    return QCD_ERR_CUDA;
  }
  return QCD_OK;
}
