// Optional per-stage timing with CUDA events recorded on the launching stream, and a count of
// kernel launches.  Off by default; when off, a stage costs one integer add.
#include <mutex>
#include <string>
#include <vector>

#include "psfm_internal.h"

namespace psfm {
namespace {

struct Stage {
  std::string name;
  double ms = 0.0;
  long long launches = 0, calls = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

std::mutex g_mu;
bool g_on = false;
long long g_launches = 0;
std::vector<Stage> g_stages;

Stage& stage(const char* name) {
  for (auto& s : g_stages)
    if (s.name == name) return s;
  g_stages.push_back(Stage());
  g_stages.back().name = name;
  return g_stages.back();
}

void resolve(Stage& s) {
  for (auto& e : s.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(e.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess)
      s.ms += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  s.pending.clear();
}

thread_local cudaEvent_t t_begin = nullptr;

}  // namespace

bool capturing(cudaStream_t s);

// Work enqueued while a stream is being captured into a graph is not timed (its events would
// belong to the graph), only counted.
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

void prof_begin(const char* name, cudaStream_t s) {
  (void)name;
  t_begin = nullptr;
  if (!g_on || capturing(s)) return;
  if (cudaEventCreate(&t_begin) == cudaSuccess) cudaEventRecord(t_begin, s);
}

void prof_end(const char* name, cudaStream_t s, int n_launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_launches += n_launches;
  if (!g_on || !t_begin) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  Stage& st = stage(name);
  st.pending.emplace_back(t_begin, e);
  st.launches += n_launches;
  st.calls += 1;
  t_begin = nullptr;
}

// FP32 FMA throughput probe: every thread runs kProbeChains independent FMA chains, unrolled
// so that the loop costs two instructions per 8 * kProbeChains FMAs.  The chains' sum is
// written out so that nothing is eliminated.
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 8;

__global__ void __launch_bounds__(256) k_fma_probe(int iters, float* out) {
  float a[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) a[j] = 1e-3f * (threadIdx.x + j);
  const float b = 0.99999f, c = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kProbeChains; ++j) a[j] = fmaf(a[j], b, c);
    }
  }
  float t = 0.f;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) t += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace psfm

extern "C" {

psfm_status psfm_fma_probe(int32_t n_blocks, int32_t iters, float* out, double* flops,
                           psfm_stream stream) {
  if (n_blocks < 1 || iters < 1 || !out) return PSFM_ERR_BAD_ARG;
  psfm::k_fma_probe<<<n_blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(iters, out);
  if (flops)
    *flops = 2.0 * n_blocks * 256.0 * psfm::kProbeChains * psfm::kProbeUnroll * (double)iters;
  return cudaGetLastError() == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

void psfm_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(psfm::g_mu);
  for (auto& s : psfm::g_stages) psfm::resolve(s);
  psfm::g_stages.clear();
  psfm::g_on = on != 0;
}

long long psfm_launch_count(void) {
  std::lock_guard<std::mutex> lk(psfm::g_mu);
  return psfm::g_launches;
}

int32_t psfm_profile_count(void) {
  std::lock_guard<std::mutex> lk(psfm::g_mu);
  return (int32_t)psfm::g_stages.size();
}

int32_t psfm_profile_entry(int32_t i, char* name, int32_t name_cap, double* ms,
                           long long* launches, long long* calls) {
  std::lock_guard<std::mutex> lk(psfm::g_mu);
  if (i < 0 || i >= (int32_t)psfm::g_stages.size()) return -1;
  auto& s = psfm::g_stages[i];
  psfm::resolve(s);
  if (name && name_cap > 0) {
    const size_t n = s.name.size() < (size_t)(name_cap - 1) ? s.name.size() : (size_t)(name_cap - 1);
    s.name.copy(name, n);
    name[n] = 0;
  }
  if (ms) *ms = s.ms;
  if (launches) *launches = s.launches;
  if (calls) *calls = s.calls;
  return 0;
}

}  // extern "C"
