// PSF-homogenised stack with outlier rejection and the unconvolved companion stack (Sec. 5.1).
//
// Pass 1 matches every input to the fake target and keeps its convolved image, variance and
// mask (and its solution and statistics) in the workspace.  An outlier is then a usable
// convolved pixel, where at least 3 inputs are usable, that deviates from the median of the
// usable convolved inputs there by more than clip_nsigma * sqrt(V'_i + alpha |median|) (the
// chi^2 softening of Sec. 3.6).  The paper carries the outlier mask back to the unconvolved
// input with a matched filter (the kernel applied to the image); here the input pixels within
// the CONV.BAD box (Chebyshev radius r_bad of that input's kernel, Sec. 3.4) of an outlier are
// rejected.  Pass 2 masks the rejected input pixels (reject_bit), convolves the inputs again
// with their unchanged kernels and accumulates the convolved stack, and accumulates the
// unconvolved inputs with the same rejections into the companion stack; both use the pass-1
// weights w_i = 1 / mean(V'_i).
#include <vector>

#include "host.h"
#include "psfm_internal.h"
#include "solve.h"

namespace psfm {

constexpr int kMaxStackFull = PSFM_STACK_FULL_MAX;  // inputs (one outlier bit each per pixel)

namespace {

// Per pixel: the median of the usable convolved inputs and the outlier bit of each input.
__global__ void k_clip_outliers(int n, int W, int H, int64_t pitch, const float* const* conv,
                                const float* const* conv_var, const uint16_t* const* conv_m,
                                uint16_t okmask, double nsig, double alpha, uint32_t* rejbits,
                                int32_t* n_rej) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const int64_t o = (int64_t)y * pitch + x;
  float v[kMaxStackFull];
  int nu = 0;
  uint32_t usable = 0;
  for (int i = 0; i < n; ++i) {
    if (conv_m[i][o] & okmask) continue;
    usable |= 1u << i;
    // insertion into the sorted prefix
    const float c = conv[i][o];
    int j = nu++;
    while (j > 0 && v[j - 1] > c) {
      v[j] = v[j - 1];
      --j;
    }
    v[j] = c;
  }
  uint32_t bits = 0;
  if (nu >= 3) {
    const double med = (nu & 1) ? (double)v[nu / 2]
                                : 0.5 * ((double)v[nu / 2 - 1] + (double)v[nu / 2]);
    const double soft = alpha * fabs(med);
    for (int i = 0; i < n; ++i) {
      if (!(usable >> i & 1u)) continue;
      const double d = (double)conv[i][o] - med;
      const double e = (double)conv_var[i][o] + soft;
      if (d * d > nsig * nsig * e) {
        bits |= 1u << i;
        atomicAdd(&n_rej[i], 1);
      }
    }
  }
  rejbits[o] = bits;
}

// Chebyshev dilation of input i's outlier bit by its r_bad: horizontal max into tmp, then
// vertical max into bad; rows of `pitch`.
__global__ void k_dilate_h(const uint32_t* rejbits, int bit, int W, int H, int64_t pitch,
                           const DevState* st, uint8_t* tmp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const int r = st->r_bad;
  const int64_t row = (int64_t)y * pitch;
  uint8_t f = 0;
  for (int d = -r; d <= r && !f; ++d) {
    const int xx = x + d;
    if (xx >= 0 && xx < W && (rejbits[row + xx] >> bit & 1u)) f = 1;
  }
  tmp[row + x] = f;
}

__global__ void k_dilate_v_mask(const uint8_t* tmp, int W, int H, int64_t pitch,
                                const DevState* st, const uint16_t* mask, uint16_t reject_bit,
                                uint16_t* m2) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const int r = st->r_bad;
  uint8_t f = 0;
  for (int d = -r; d <= r && !f; ++d) {
    const int yy = y + d;
    if (yy >= 0 && yy < H && tmp[(int64_t)yy * pitch + x]) f = 1;
  }
  const int64_t o = (int64_t)y * pitch + x;
  m2[o] = f ? (uint16_t)(mask[o] | reject_bit) : mask[o];
}

}  // namespace

namespace {

struct FullLayout {
  StackBuffers kb;
  float* uacc_w = nullptr;    // [H][pitch] unconvolved weight sums
  uint32_t* rejbits = nullptr;  // [H][pitch] outlier bit per input
  uint8_t* tmp = nullptr;     // [H][pitch] horizontal dilation
  uint16_t* m2 = nullptr;     // [H][pitch] input mask with rejected pixels
  int32_t* n_rej = nullptr;   // [n] outlier pixels per input
  const float** conv_p = nullptr;  // device arrays of the stored pass-1 planes
  const float** var_p = nullptr;
  const uint16_t** mask_p = nullptr;
  std::vector<float*> conv, var;
  std::vector<uint16_t*> cm;
  std::vector<Plan> plans;
  std::vector<Head> heads;
  size_t shared_off = 0;  // offset of the per-input apply/solve scratch (reused by each input)
};

// Lays out (base != nullptr) or measures the workspace; returns bytes or 0 on a bad plan.
size_t full_layout(int n, psfm_shape shape, const psfm_basis_spec* basis, const psfm_config* cfg,
                   int n_src_max, char* base, FullLayout* L, psfm_status* st) {
  Workspace ws;
  ws.base = base;
  ws.measuring = base == nullptr;
  *st = PSFM_OK;
  Plan p0;
  if ((*st = make_plan(p0, shape, &basis[0], cfg, 0)) != PSFM_OK) return 0;
  if (cfg->dual) {  // the inputs are matched to a noiseless rendered target
    *st = PSFM_ERR_UNSUPPORTED;
    return 0;
  }
  const size_t npx = (size_t)shape.height * shape.pitch;
  StackBuffers kb;
  carve_stack(p0, ws, kb, n_src_max);
  FullLayout tmpL;
  FullLayout& l = L ? *L : tmpL;
  l.kb = kb;
  l.uacc_w = ws.take<float>(npx);
  l.rejbits = ws.take<uint32_t>(npx);
  l.tmp = ws.take<uint8_t>(npx);
  l.m2 = ws.take<uint16_t>(npx);
  l.n_rej = ws.take<int32_t>(n);
  l.conv_p = ws.take<const float*>(n);
  l.var_p = ws.take<const float*>(n);
  l.mask_p = ws.take<const uint16_t*>(n);
  for (int i = 0; i < n; ++i) {
    Plan p;
    if ((*st = make_plan(p, shape, &basis[i], cfg, 0)) != PSFM_OK) return 0;
    l.conv.push_back(ws.take<float>(npx));
    l.var.push_back(ws.take<float>(npx));
    l.cm.push_back(ws.take<uint16_t>(npx));
    Head h;
    const size_t hb = head_layout(p, h);
    if (!ws.measuring) head_bind(h, base + ws.used, p);
    ws.used += hb;
    l.plans.push_back(p);
    l.heads.push_back(std::move(h));
  }
  l.shared_off = ws.used;
  size_t shared = 0;
  for (int i = 0; i < n; ++i) {
    Workspace w2;
    w2.measuring = true;
    ApplyBuffers b;
    carve_apply(l.plans[i], w2, b);
    SolveBuffers sb;
    carve_solve(l.plans[i], w2, sb);
    if (w2.used > shared) shared = w2.used;
  }
  return ws.used + shared;
}

psfm_status run_stack_full(int n, const float* const* imgs, const float* const* vars,
                           const uint16_t* const* masks, psfm_shape shape,
                           const double* const* src_xyf, const int32_t* n_src, double fwhm,
                           const psfm_basis_spec* basis, const psfm_config* cfg,
                           double clip_nsigma, uint16_t reject_bit, float* out, float* out_var,
                           uint16_t* out_mask, int32_t* out_count, float* uout,
                           float* uout_var, uint16_t* uout_mask, int32_t* uout_count,
                           int32_t* n_rejected, uint32_t* outliers, double* cov_out,
                           int cov_out_w, psfm_solution* sols, char* base, size_t ws_bytes,
                           cudaStream_t st) {
  int n_src_max = 1, wmax = 0;
  for (int i = 0; i < n; ++i) {
    if (!imgs[i] || !vars[i] || !masks[i] || n_src[i] < 0 || (n_src[i] > 0 && !src_xyf[i]))
      return PSFM_ERR_BAD_ARG;
    if (n_src[i] > n_src_max) n_src_max = n_src[i];
    const int wi = psfm_cov_width(&basis[i], 1, 0);
    if (wi < 0) return PSFM_ERR_BAD_ARG;
    if (wi > wmax) wmax = wi;
  }
  if (cov_out && cov_out_w != wmax) return PSFM_ERR_BAD_ARG;
  FullLayout L;
  psfm_status s;
  const size_t need = full_layout(n, shape, basis, cfg, n_src_max, base, &L, &s);
  if (s != PSFM_OK) return s;
  if (need > ws_bytes) return PSFM_ERR_WORKSPACE;
  const Plan& p0 = L.plans[0];
  const StackBuffers& kb = L.kb;
  const size_t npx = (size_t)shape.height * shape.pitch;
  bool ok = true;
  auto zero = [&](void* ptr, size_t bytes) {
    ok = ok && cudaMemsetAsync(ptr, 0, bytes, st) == cudaSuccess;
  };
  zero(out, sizeof(float) * npx);
  zero(out_var, sizeof(float) * npx);
  zero(out_count, sizeof(int32_t) * npx);
  zero(kb.acc_w, sizeof(float) * npx);
  zero(uout, sizeof(float) * npx);
  zero(uout_var, sizeof(float) * npx);
  zero(uout_count, sizeof(int32_t) * npx);
  zero(L.uacc_w, sizeof(float) * npx);
  zero(kb.zero_var, sizeof(float) * npx);
  zero(kb.zero_m, sizeof(uint16_t) * npx);
  zero(kb.pm_acc, sizeof(double) * kMaxCovOut * kMaxCovOut);
  zero(kb.wsum, sizeof(double) * 2);
  zero(L.n_rej, sizeof(int32_t) * n);
  if (!ok) return PSFM_ERR_CUDA;
  std::vector<const float*> hc(L.conv.begin(), L.conv.end()), hv(L.var.begin(), L.var.end());
  std::vector<const uint16_t*> hm(L.cm.begin(), L.cm.end());
  if (cudaMemcpyAsync(L.conv_p, hc.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(L.var_p, hv.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(L.mask_p, hm.data(), sizeof(uint16_t*) * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return PSFM_ERR_CUDA;
  char* shared = base + L.shared_off;
  auto buffers = [&](int i, ApplyBuffers& b, SolveBuffers& sb) {
    Workspace w2;
    w2.base = shared;
    carve_apply(L.plans[i], w2, b);
    carve_solve(L.plans[i], w2, sb);
    b.tab = bind_tables(L.heads[i].tables, L.heads[i].offs);
    b.st = L.heads[i].st;
    b.dsol = L.heads[i].dsol;
  };
  // ---- pass 1: solve every input against its target, keep the convolved planes
  for (int i = 0; i < n; ++i) {
    const Plan& p = L.plans[i];
    Head& h = L.heads[i];
    ApplyBuffers b;
    SolveBuffers sb;
    buffers(i, b, sb);
    if (cudaMemsetAsync(kb.target, 0, sizeof(float) * npx, st) != cudaSuccess) return PSFM_ERR_CUDA;
    if (n_src[i] > 0 &&
        cudaMemcpyAsync(kb.src, src_xyf[i], sizeof(double) * 3 * n_src[i], cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return PSFM_ERR_CUDA;
    prof_begin("stack_target", st);
    if (launch_render_target(p, kb.src, n_src[i], fwhm, kb.target, st) != cudaSuccess)
      return PSFM_ERR_CUDA;
    prof_end("stack_target", st, n_src[i] > 0 ? 1 : 0);
    if (upload_head(p, h, nullptr, 0, st) != cudaSuccess) return PSFM_ERR_CUDA;
    s = run_solve(p, b.tab, h.st, h.dsol, sb, kb.target, imgs[i], kb.zero_var, vars[i], kb.zero_m,
                  masks[i], nullptr, st);
    if (s != PSFM_OK) return s;
    const int ni = 2 * p.w - 1;
    s = run_apply(p, h, b, imgs[i], vars[i], masks[i], nullptr, nullptr, nullptr, nullptr, 1,
                  nullptr, 0, L.conv[i], L.var[i], L.cm[i], cov_out ? kb.pm : nullptr, ni, true,
                  st);
    if (s != PSFM_OK) return s;
    if (cov_out &&
        launch_stack_cov_accum(kb.pm, ni, cov_out_w, h.st, kb.pm_acc, kb.wsum, st) != cudaSuccess)
      return PSFM_ERR_CUDA;
    s = sols ? fetch_solution(p, h.st, h.dsol, sb, &sols[i], st) : sync_status(h.st, st);
    if (s != PSFM_OK) return s;
  }
  // ---- outliers against the per-pixel median of the convolved inputs
  const dim3 blk(256), grid((shape.width + 255) / 256, shape.height);
  prof_begin("stack_clip", st);
  k_clip_outliers<<<grid, blk, 0, st>>>(n, shape.width, shape.height, shape.pitch, L.conv_p,
                                         L.var_p, L.mask_p,
                                         (uint16_t)(cfg->badmask | cfg->conv_bad), clip_nsigma,
                                         cfg->soften_alpha, L.rejbits, L.n_rej);
  if (cudaGetLastError() != cudaSuccess) return PSFM_ERR_CUDA;
  if (outliers && cudaMemcpyAsync(outliers, L.rejbits, sizeof(uint32_t) * npx,
                                  cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return PSFM_ERR_CUDA;
  prof_end("stack_clip", st, 1);
  // ---- pass 2: reject, convolve again, accumulate both stacks
  for (int i = 0; i < n; ++i) {
    Plan p2 = L.plans[i];
    p2.cfg.badmask = (uint16_t)(p2.cfg.badmask | reject_bit);
    const Head& h = L.heads[i];
    ApplyBuffers b;
    SolveBuffers sb;
    buffers(i, b, sb);
    prof_begin("stack_reject", st);
    k_dilate_h<<<grid, blk, 0, st>>>(L.rejbits, i, shape.width, shape.height, shape.pitch, h.st,
                                     L.tmp);
    k_dilate_v_mask<<<grid, blk, 0, st>>>(L.tmp, shape.width, shape.height, shape.pitch, h.st,
                                          masks[i], reject_bit, L.m2);
    if (cudaGetLastError() != cudaSuccess) return PSFM_ERR_CUDA;
    prof_end("stack_reject", st, 2);
    s = run_apply(p2, h, b, imgs[i], vars[i], L.m2, nullptr, nullptr, nullptr, nullptr, 1,
                  nullptr, 0, kb.conv, kb.conv_var, kb.conv_m, nullptr, 0, false, st);
    if (s != PSFM_OK) return s;
    prof_begin("stack_accum", st);
    if (launch_stack_accum(p2, kb.conv, kb.conv_var, kb.conv_m, h.st, out, out_var, kb.acc_w,
                           out_count, st) != cudaSuccess ||
        launch_stack_accum(p2, imgs[i], vars[i], L.m2, h.st, uout, uout_var, L.uacc_w,
                           uout_count, st) != cudaSuccess)
      return PSFM_ERR_CUDA;
    prof_end("stack_accum", st, 2);
  }
  prof_begin("stack_final", st);
  if (launch_stack_final(p0, out, out_var, out_mask, kb.acc_w, out_count, kb.pm_acc, kb.wsum,
                         cov_out, cov_out_w, st) != cudaSuccess ||
      launch_stack_final(p0, uout, uout_var, uout_mask, L.uacc_w, uout_count, nullptr, nullptr,
                         nullptr, 0, st) != cudaSuccess)
    return PSFM_ERR_CUDA;
  prof_end("stack_final", st, cov_out ? 3 : 2);
  if (n_rejected &&
      cudaMemcpyAsync(n_rejected, L.n_rej, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
    return PSFM_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

}  // namespace
}  // namespace psfm

extern "C" {

size_t psfm_stack_full_workspace_size(int32_t n, psfm_shape shape, const psfm_basis_spec* basis,
                                      const psfm_config* cfg, int32_t n_src_max) {
  if (n < 1 || n > psfm::kMaxStackFull || !basis || !cfg) return 0;
  psfm_status st;
  const size_t sz =
      psfm::full_layout(n, shape, basis, cfg, n_src_max > 0 ? n_src_max : 1, nullptr, nullptr, &st);
  return st == PSFM_OK ? sz : 0;
}

psfm_status psfm_stack_full(int32_t n, const float* const* imgs, const float* const* vars,
                            const uint16_t* const* masks, psfm_shape shape,
                            const double* const* src_xyf, const int32_t* n_src,
                            double target_fwhm, const psfm_basis_spec* basis,
                            const psfm_config* cfg, double clip_nsigma, uint16_t reject_bit,
                            float* out, float* out_var, uint16_t* out_mask, int32_t* out_count,
                            float* uout, float* uout_var, uint16_t* uout_mask,
                            int32_t* uout_count, int32_t* n_rejected, uint32_t* outliers,
                            double* cov_out, int32_t cov_out_w, psfm_solution* sols,
                            void* workspace, size_t ws_bytes, psfm_stream stream) {
  if (n < 1 || n > psfm::kMaxStackFull || !imgs || !vars || !masks || !src_xyf || !n_src ||
      !basis || !cfg || !out || !out_var || !out_mask || !out_count || !uout || !uout_var ||
      !uout_mask || !uout_count || !workspace)
    return PSFM_ERR_BAD_ARG;
  if (!(target_fwhm > 0.0) || !(clip_nsigma > 0.0)) return PSFM_ERR_BAD_ARG;
  if (reject_bit == 0 || (reject_bit & (cfg->badmask | cfg->conv_bad | cfg->conv_poor)) != 0)
    return PSFM_ERR_BAD_ARG;
  if (!psfm::aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  return psfm::run_stack_full(n, imgs, vars, masks, shape, src_xyf, n_src, target_fwhm, basis,
                              cfg, clip_nsigma, reject_bit, out, out_var, out_mask, out_count,
                              uout, uout_var, uout_mask, uout_count, n_rejected, outliers,
                              cov_out, cov_out_w, sols, static_cast<char*>(workspace), ws_bytes,
                              reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
