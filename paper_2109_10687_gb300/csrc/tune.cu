// Launch-shape autotuner: for kernels with several compiled launch shapes
// (threads per block, register budget, blocks per SM) the first launch with
// a given key times each shape on the real arguments with CUDA events and
// keeps the fastest.  The shapes differ only in scheduling, never in the
// arithmetic each site performs.

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
  for (int v = 0; v < nvariants; ++v) {
    run(v);  // warm-up
    QCD_CUDA_CHECK(cudaEventRecord(a, st));
    for (int r = 0; r < 3; ++r) run(v);
    QCD_CUDA_CHECK(cudaEventRecord(b, st));
    QCD_CUDA_CHECK(cudaEventSynchronize(b));
    float ms = 0.f;
    QCD_CUDA_CHECK(cudaEventElapsedTime(&ms, a, b));
    ms /= 3.f;
    if (ms < best_ms) {
      best_ms = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->launches += 4LL * nvariants;
  t->best[key] = {best_v, best_ms, names ? names[best_v] : std::to_string(best_v)};
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

extern "C" int qcd_tuning_report(qcd_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return QCD_ERR_ARG;
  std::string out;
  for (auto& kv : tuner_of(ctx)->best) {
    char line[256];
    std::snprintf(line, sizeof line, "%s %s %.4f ms\n", kv.first.c_str(), kv.second.name.c_str(), kv.second.ms);
    out += line;
  }
  std::snprintf(buf, len, "%s", out.c_str());
  return QCD_OK;
}
