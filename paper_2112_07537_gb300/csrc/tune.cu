// tune.cu -- launch-shape autotuner.  A tunable launch names a key (kernel,
// wavelet, block size, precision, shell, mode) and its candidate CTA sizes;
// the first time a key is met on a grid with autotuning enabled, each
// candidate is launched on the grid's own data (once to warm up, then timed
// with CUDA events on the grid's stream) and the fastest is kept in a
// process-wide table that every later launch with that key reads.  Only
// launches that give the same result when repeated are tuned (they read
// their inputs and overwrite their outputs), so tuning changes no value:
// every kernel computes each output point with the same arithmetic whatever
// its CTA size.  One key (kid 6) chooses between the two FP32 stage kernels
// instead, which evaluate the same operations in the same order (equal up to
// where the compiler fuses a multiply-add differently).  Tuning is skipped
// while a step is being captured into a CUDA graph (the cached or first
// candidate is used).
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "mr_internal.cuh"

namespace mr {

namespace {

struct Entry {
  int threads;
  int ncand;
  int cand[4];
  float ms[4];
};

std::mutex g_mu;
std::map<TuneKey, Entry> g_table;

const char *tune_kernel_name(int kid) {
  static const char *names[] = {"k_fill_plain", "k_prep", "k_criterion", "k_fused", "k_interp", "k_merge",
                                "stage kernel (1 k_fused, 2 k_march)"};
  return kid >= 0 && kid < (int)(sizeof names / sizeof names[0]) ? names[kid] : "?";
}

}  // namespace

bool operator<(const TuneKey &a, const TuneKey &b) {
  const int x[7] = {a.kid, a.N, a.Nt, a.nb, a.tp, a.shell, a.mode};
  const int y[7] = {b.kid, b.N, b.Nt, b.nb, b.tp, b.shell, b.mode};
  for (int i = 0; i < 7; ++i)
    if (x[i] != y[i]) return x[i] < y[i];
  return false;
}

int tune_threads(mr_grid *g, const TuneKey &key, const int *cand, int ncand,
                 const std::function<void(int)> &launch) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(key);
    if (it != g_table.end()) return it->second.threads;
  }
  if (!g->autotune || g->capturing || ncand < 2) return cand[0];
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cand[0];
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cand[0];
  }
  Entry en{};
  en.ncand = ncand > 4 ? 4 : ncand;
  int best = 0;
  const int saved = g->profiling;
  g->profiling = 0;  // the tuning launches are not recorded
  bool ok = true;
  for (int c = 0; c < en.ncand && ok; ++c) {
    en.cand[c] = cand[c];
    launch(cand[c]);
    cudaEventRecord(e0, g->stream);
    launch(cand[c]);
    cudaEventRecord(e1, g->stream);
    ok = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    float ms = 0.f;
    if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    en.ms[c] = ms;
    if (ok && ms < en.ms[best]) best = c;
  }
  g->profiling = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return cand[0];
  en.threads = cand[best];
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[key] = en;
  return en.threads;
}

}  // namespace mr

extern "C" int mr_autotune(mr_grid *g, int enable) {
  if (!g) return MR_ERR_INVALID;
  g->autotune = enable ? 1 : 0;
  return MR_OK;
}

extern "C" int mr_set_stage_kernel(mr_grid *g, int which) {
  if (!g || which < 0 || which > 2) return MR_ERR_INVALID;
  g->stage_kernel = which;
  return MR_OK;
}

extern "C" int mr_autotune_table(char *buf, size_t len, int *nentries) {
  using namespace mr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (nentries) *nentries = (int)g_table.size();
  if (!buf || !len) return MR_OK;
  std::string out;
  char line[256];
  for (const auto &kv : g_table) {
    const TuneKey &k = kv.first;
    const Entry &e = kv.second;
    int n = snprintf(line, sizeof line, "%s N=%d.%d nb=%d %s shell=%d mode=%d -> %d %s (", tune_kernel_name(k.kid),
                     k.N, k.Nt, k.nb, k.tp == 8 ? "f64" : k.tp == 5 ? "f32->f64" : "f32", k.shell, k.mode,
                     e.threads, k.kid == 6 ? "variant" : "threads");
    out.append(line, n > 0 ? (size_t)n : 0);
    for (int c = 0; c < e.ncand; ++c) {
      n = snprintf(line, sizeof line, "%s%d: %.3f ms", c ? ", " : "", e.cand[c], e.ms[c]);
      out.append(line, n > 0 ? (size_t)n : 0);
    }
    out += ")\n";
  }
  snprintf(buf, len, "%s", out.c_str());
  return out.size() + 1 > len ? MR_ERR_NOMEM : MR_OK;
}

extern "C" int mr_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(mr::g_mu);
  mr::g_table.clear();
  return MR_OK;
}
