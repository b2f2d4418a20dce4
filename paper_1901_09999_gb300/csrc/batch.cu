// Batched subtraction: many chips (each with its own size, basis and spatial order) solved and
// convolved by one call, spread over several CUDA streams so that the latency-bound solve
// stages of one chip overlap the arithmetic-bound convolutions of others, and captured into a
// CUDA graph on the first call so that later calls with the same buffers replay it with a
// single launch.
//
// Each stream slot is a pair: solves run on a high-priority stream and the image, variance,
// mask and pseudo-matrix passes on a low-priority one, so that the small, latency-bound solve
// kernels get SMs as soon as any convolution CTA retires instead of queueing behind whole
// convolution grids.  The graph is instantiated with per-node priorities, which capture
// takes from the streams.
//
// Per chip the work is exactly psfm_subtract's (extractor, rejection loop, r_bad, image,
// variance, mask, pseudo-matrix), with the solution kept on the device; the per-chip tables
// are uploaded once, at creation, and every execution resets only the device state block.
#include <cstring>
#include <vector>

#include "host.h"
#include "psfm_internal.h"
#include "solve.h"

struct psfm_batch {
  int n = 0;
  std::vector<psfm::Plan> plans;
  std::vector<psfm::Head> heads;
  std::vector<psfm::ApplyBuffers> ab;
  std::vector<psfm::SolveBuffers> sb;
  std::vector<cudaStream_t> streams;     // solve streams (high priority)
  std::vector<cudaStream_t> streams_lo;  // apply streams (low priority)
  std::vector<cudaEvent_t> done, done_lo, solved;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;
  long long kernels_per_exec = 0;
};

namespace {

using namespace psfm;

size_t layout(int n, const psfm_shape* shapes, const psfm_basis_spec* bases,
              const psfm_config* cfg, psfm_batch* b, char* base, psfm_status* st) {
  Workspace ws;
  ws.base = base;
  ws.measuring = base == nullptr;
  *st = PSFM_OK;
  for (int i = 0; i < n; ++i) {
    Plan p;
    psfm_status s = make_plan(p, shapes[i], &bases[i], cfg, 0);
    if (s != PSFM_OK) {
      *st = s;
      return 0;
    }
    Head h;
    const size_t hb = head_layout(p, h);
    if (!ws.measuring) head_bind(h, base + ws.used, p);
    ws.used += hb;
    ApplyBuffers a;
    carve_apply(p, ws, a);
    SolveBuffers sv;
    carve_solve(p, ws, sv);
    if (b) {
      a.tab = bind_tables(h.tables, h.offs);
      a.st = h.st;
      a.dsol = h.dsol;
      b->plans.push_back(p);
      b->heads.push_back(std::move(h));
      b->ab.push_back(a);
      b->sb.push_back(sv);
    }
  }
  return ws.used;
}

psfm_status enqueue_chip(psfm_batch* b, int i, cudaStream_t s, cudaStream_t s_lo,
                         const float* img, const float* ref, const float* var_img,
                         const float* var_ref, const uint16_t* mask_img, const uint16_t* mask_ref,
                         float* diff, float* diff_var, uint16_t* diff_mask, double* cov_out) {
  const Plan& p = b->plans[i];
  const Head& h = b->heads[i];
  if (cudaMemsetAsync(h.st, 0, sizeof(DevState), s) != cudaSuccess) return PSFM_ERR_CUDA;
  psfm_status st = run_solve(p, b->ab[i].tab, h.st, h.dsol, b->sb[i], img, ref, var_img, var_ref,
                             mask_img, mask_ref, nullptr, s);
  if (st != PSFM_OK) return st;
  if (cudaEventRecord(b->solved[i], s) != cudaSuccess ||
      cudaStreamWaitEvent(s_lo, b->solved[i], 0) != cudaSuccess)
    return PSFM_ERR_CUDA;
  const int cw = 2 * p.w - 1;
  return run_apply(p, h, b->ab[i], ref, var_ref, mask_ref, img, var_img, mask_img, nullptr, 1,
                   nullptr, 1, diff, diff_var, diff_mask, cov_out, cw, cov_out != nullptr, s_lo);
}

}  // namespace

extern "C" {

size_t psfm_batch_workspace_size(int32_t n, const psfm_shape* shapes,
                                 const psfm_basis_spec* bases, const psfm_config* cfg) {
  if (n < 1 || !shapes || !bases || !cfg) return 0;
  psfm_status st;
  const size_t sz = layout(n, shapes, bases, cfg, nullptr, nullptr, &st);
  return st == PSFM_OK ? sz : 0;
}

psfm_status psfm_batch_create(int32_t n, const psfm_shape* shapes, const psfm_basis_spec* bases,
                              const psfm_config* cfg, int32_t n_streams, void* workspace,
                              size_t ws_bytes, psfm_batch** out) {
  using namespace psfm;
  if (n < 1 || !shapes || !bases || !cfg || !workspace || !out || n_streams < 1 || n_streams > 32)
    return PSFM_ERR_BAD_ARG;
  if (!aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  *out = nullptr;
  psfm_status st;
  const size_t need = layout(n, shapes, bases, cfg, nullptr, nullptr, &st);
  if (st != PSFM_OK) return st;
  if (need > ws_bytes) return PSFM_ERR_WORKSPACE;
  psfm_batch* b = new psfm_batch();
  b->n = n;
  layout(n, shapes, bases, cfg, b, static_cast<char*>(workspace), &st);
  // tables are uploaded once; each execution resets only the device state block
  for (int i = 0; i < n; ++i)
    if (upload_head(b->plans[i], b->heads[i], nullptr, 0, 0) != cudaSuccess) {
      delete b;
      return PSFM_ERR_CUDA;
    }
  if (cudaStreamSynchronize(0) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return PSFM_ERR_CUDA;
  }
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
    psfm_batch_destroy(b);
    return PSFM_ERR_CUDA;
  }
  for (int k = 0; k < n_streams; ++k) {
    cudaStream_t s = nullptr, s_lo = nullptr;
    cudaEvent_t e = nullptr, e_lo = nullptr;
    const bool ok =
        cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
        cudaStreamCreateWithPriority(&s_lo, cudaStreamNonBlocking, prio_lo) == cudaSuccess &&
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&e_lo, cudaEventDisableTiming) == cudaSuccess;
    if (s) b->streams.push_back(s);
    if (s_lo) b->streams_lo.push_back(s_lo);
    if (e) b->done.push_back(e);
    if (e_lo) b->done_lo.push_back(e_lo);
    if (!ok) {
      psfm_batch_destroy(b);
      return PSFM_ERR_CUDA;
    }
  }
  for (int i = 0; i < n; ++i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      psfm_batch_destroy(b);
      return PSFM_ERR_CUDA;
    }
    b->solved.push_back(e);
  }
  *out = b;
  return PSFM_OK;
}

void psfm_batch_destroy(psfm_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto s : b->streams_lo) cudaStreamDestroy(s);
  for (auto e : b->done) cudaEventDestroy(e);
  for (auto e : b->done_lo) cudaEventDestroy(e);
  for (auto e : b->solved) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

psfm_status psfm_batch_subtract(psfm_batch* b, const float* const* imgs, const float* const* refs,
                                const float* const* var_imgs, const float* const* var_refs,
                                const uint16_t* const* mask_imgs,
                                const uint16_t* const* mask_refs, float* const* diffs,
                                float* const* diff_vars, uint16_t* const* diff_masks,
                                double* const* cov_outs, psfm_stream stream) {
  if (!b || !imgs || !refs || !var_imgs || !var_refs || !mask_imgs || !mask_refs || !diffs)
    return PSFM_ERR_BAD_ARG;
  const int n = b->n;
  std::vector<const void*> key;
  key.reserve(11 * n);
  for (int i = 0; i < n; ++i) {
    if (!imgs[i] || !refs[i] || !var_imgs[i] || !var_refs[i] || !mask_imgs[i] || !mask_refs[i] ||
        !diffs[i])
      return PSFM_ERR_BAD_ARG;
    key.insert(key.end(), {imgs[i], refs[i], var_imgs[i], var_refs[i], mask_imgs[i],
                           mask_refs[i], diffs[i], diff_vars ? diff_vars[i] : nullptr,
                           diff_masks ? diff_masks[i] : nullptr,
                           cov_outs ? cov_outs[i] : nullptr});
  }
  cudaStream_t origin = reinterpret_cast<cudaStream_t>(stream);
  if (b->exec && key == b->key)
    return cudaGraphLaunch(b->exec, origin) == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
  const bool capture = origin != nullptr;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  if (capture && cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return PSFM_ERR_CUDA;
  const long long l0 = psfm_launch_count();
  psfm_status st = PSFM_OK;
  if (cudaEventRecord(b->fork, origin) != cudaSuccess) st = PSFM_ERR_CUDA;
  const int K = (int)b->streams.size();
  for (int k = 0; k < K && st == PSFM_OK; ++k)
    if (cudaStreamWaitEvent(b->streams[k], b->fork, 0) != cudaSuccess ||
        cudaStreamWaitEvent(b->streams_lo[k], b->fork, 0) != cudaSuccess)
      st = PSFM_ERR_CUDA;
  for (int i = 0; i < n && st == PSFM_OK; ++i)
    st = enqueue_chip(b, i, b->streams[i % K], b->streams_lo[i % K], imgs[i], refs[i],
                      var_imgs[i], var_refs[i], mask_imgs[i], mask_refs[i], diffs[i],
                      diff_vars ? diff_vars[i] : nullptr, diff_masks ? diff_masks[i] : nullptr,
                      cov_outs ? cov_outs[i] : nullptr);
  for (int k = 0; k < K; ++k) {
    if (cudaEventRecord(b->done[k], b->streams[k]) != cudaSuccess ||
        cudaEventRecord(b->done_lo[k], b->streams_lo[k]) != cudaSuccess ||
        cudaStreamWaitEvent(origin, b->done[k], 0) != cudaSuccess ||
        cudaStreamWaitEvent(origin, b->done_lo[k], 0) != cudaSuccess)
      st = PSFM_ERR_CUDA;
  }
  b->kernels_per_exec = psfm_launch_count() - l0;
  if (!capture) return st;
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(origin, &g);
  if (st != PSFM_OK || ec != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != PSFM_OK ? st : PSFM_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PSFM_ERR_CUDA;
  }
  b->graph = g;
  b->exec = ex;
  b->key = key;
  return cudaGraphLaunch(ex, origin) == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

long long psfm_batch_kernel_count(const psfm_batch* b) { return b ? b->kernels_per_exec : 0; }

psfm_status psfm_batch_solutions(psfm_batch* b, psfm_solution* sols, psfm_stream stream) {
  if (!b) return PSFM_ERR_BAD_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return PSFM_ERR_CUDA;
  psfm_status first = PSFM_OK;
  for (int i = 0; i < b->n; ++i) {
    psfm_status st;
    if (sols)
      st = psfm::fetch_solution(b->plans[i], b->heads[i].st, b->heads[i].dsol, b->sb[i], &sols[i], s);
    else
      st = psfm::sync_status(b->heads[i].st, s);
    if (st != PSFM_OK && first == PSFM_OK) first = st;
  }
  return first;
}

}  // extern "C"
