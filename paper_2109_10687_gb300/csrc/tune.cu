// Launch-shape autotuner: for kernels with several compiled launch shapes
// (threads per block, register budget, blocks per SM) the first launch with
// a given key times each shape on the real arguments with CUDA events and
// keeps the fastest.  The shapes differ only in scheduling, never in the
// arithmetic each site performs.

#include <algorithm>
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

extern "C" int qcd_set_sap_shape(qcd_ctx* ctx, int shape) {
  if (!ctx || shape < -1 || shape > 1) return QCD_ERR_ARG;
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
