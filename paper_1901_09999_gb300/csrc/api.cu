// C ABI entry points of libpsfm (see include/psfm.h for the contract of each call).
//
// Every call validates its arguments on the host, carves the caller's workspace into the
// buffers it needs, uploads one small blob (device state, solution, basis tables) and
// enqueues kernels on the caller's stream.  Nothing here computes image data on the host.
#include <cmath>
#include <cstring>
#include <vector>

#include "host.h"
#include "psfm_internal.h"
#include "solve.h"

using namespace psfm;

namespace psfm {

size_t head_layout(const Plan& p, Head& h) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  pack_tables(p, h.blob, h.offs);
  size_t o = al(sizeof(DevState));
  const size_t o_dsol = o;
  o = al(o + sizeof(double) * (2 + p.ncoef + 2 + 2 * (2 + p.Nb * p.Ns)));
  const size_t o_tab = o;
  o = al(o + h.blob.size());
  h.bytes = o;
  (void)o_dsol;
  (void)o_tab;
  return o;
}

void head_bind(Head& h, char* base, const Plan& p) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  h.st = reinterpret_cast<DevState*>(base);
  size_t o = al(sizeof(DevState));
  h.dsol = reinterpret_cast<double*>(base + o);
  h.dsol2 = h.dsol + (2 + p.ncoef + 2);
  h.dsol3 = h.dsol2 + (2 + p.Nb * p.Ns);
  o = al(o + sizeof(double) * (2 + p.ncoef + 2 + 2 * (2 + p.Nb * p.Ns)));
  h.tables = base + o;
}

DevTables bind_tables(char* t, const size_t offs[7]) {
  DevTables d;
  d.f1d = reinterpret_cast<float*>(t + offs[0]);
  d.f1d64 = reinterpret_cast<double*>(t + offs[1]);
  d.psi = reinterpret_cast<double*>(t + offs[2]);
  d.sk = reinterpret_cast<double*>(t + offs[3]);
  d.term = reinterpret_cast<int32_t*>(t + offs[4]);
  d.spat = reinterpret_cast<int32_t*>(t + offs[5]);
  d.pen = reinterpret_cast<double*>(t + offs[6]);
  return d;
}

// Apply-path buffers after the head.
void carve_apply(const Plan& p, Workspace& ws, ApplyBuffers& b) {
  const int nwords = (p.W + 31) / 32;
  b.bits = ws.take<uint32_t>((size_t)p.H * nwords);
  b.hb_bad = ws.take<uint32_t>((size_t)p.H * nwords);
  b.hb_poor = ws.take<uint32_t>((size_t)p.H * nwords);
  b.mask_tmp = ws.take<uint16_t>((size_t)p.H * p.pitch);
  const int ns = p.cfg.cov_grid * p.cfg.cov_grid;
  const int wt = p.w + kMaxCovIn - 1;
  const int nconv = 2 * p.w + kMaxCovIn - 2;
  b.kern = ws.take<double>((size_t)ns * p.w * p.w);
  b.kern_t = ws.take<double>((size_t)ns * wt * wt);
  b.kern_s2 = ws.take<double>(ns);
  b.kern_f = ws.take<float2>((size_t)ns * p.w * p.w);
  b.kern_tf = ws.take<float2>((size_t)ns * wt * wt);
  b.cov_acc = ws.take<double>((size_t)ns * nconv * nconv);
  b.cov_tmp = ws.take<double>((size_t)(2 * p.w - 1) * (2 * p.w - 1));
  const size_t npatch =
      (size_t)((p.W + kVarTile - 1) / kVarTile) * (size_t)((p.H + kVarTile - 1) / kVarTile);
  b.var_part = ws.take<double>(3 * npatch);
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

// Upload the head: device state (zeroed, r_bad given), solution and tables.
cudaError_t upload_head(const Plan& p, Head& h, const double* sol_vals, int r_bad,
                        cudaStream_t st) {
  std::vector<char> host(h.bytes, 0);
  DevState ds;
  std::memset(&ds, 0, sizeof(ds));
  ds.r_bad = r_bad;
  std::memcpy(host.data(), &ds, sizeof(ds));
  const size_t o_dsol = reinterpret_cast<char*>(h.dsol) - reinterpret_cast<char*>(h.st);
  const size_t o_tab = h.tables - reinterpret_cast<char*>(h.st);
  if (sol_vals) std::memcpy(host.data() + o_dsol, sol_vals, sizeof(double) * (2 + p.ncoef));
  std::memcpy(host.data() + o_tab, h.blob.data(), h.blob.size());
  return cudaMemcpyAsync(h.st, host.data(), h.bytes, cudaMemcpyHostToDevice, st);
}

psfm_status check_cov(const Plan& p, const double* cov_ref, int cov_ref_w, bool diff,
                      const double* cov_img, int cov_img_w, const double* cov_out, int cov_out_w,
                      int* c_ref, int* c_img) {
  *c_ref = cov_ref ? cov_ref_w : 1;
  *c_img = diff ? (cov_img ? cov_img_w : 1) : 0;
  if (cov_ref && (cov_ref_w < 1 || cov_ref_w % 2 == 0 || cov_ref_w > kMaxCovIn))
    return PSFM_ERR_BAD_ARG;
  if (cov_img && (!diff || cov_img_w < 1 || cov_img_w % 2 == 0)) return PSFM_ERR_BAD_ARG;
  if (cov_out) {
    const int n = 2 * p.w + *c_ref - 2;
    const int want = n > *c_img ? n : *c_img;
    if (cov_out_w != want) return PSFM_ERR_BAD_ARG;
  }
  return PSFM_OK;
}

// The apply path (Eq. 12-13, Sec. 3.4, Sec. 4.3-4.4) given the head already uploaded or
// computed on the device.  r_bad is read from the device state.
namespace {

// Dual kernel (Eq. 2): from the solution (b0, d0, b terms, c terms) the views (0, 0, c), the
// terms applied to I2, and (1, 0, -c), the kernel K2 = delta - sum c_k B_k of the difference.
__global__ void k_dual_split(const double* dsol, int nbs, double* dsol2, double* dsol3) {
  for (int i = threadIdx.x; i < 2 + nbs; i += blockDim.x) {
    const double c = i >= 2 ? dsol[2 + nbs + (i - 2)] : 0.0;
    dsol2[i] = c;
    dsol3[i] = i == 0 ? 1.0 : (i == 1 ? 0.0 : -c);
  }
}

// D = K2 (x) I2 - K1 (x) I1 - d0, its variance sum K1^2 (x) V1 + sum K2^2 (x) V2 (per patch),
// the mask of both convolutions and the pseudo-matrices of K1 and K2 averaged with the mean
// variances of the two parts as weights (Sec. 4.4).  White inputs only.
psfm_status run_apply_dual(const Plan& p, const Head& h, const ApplyBuffers& b,
                           const DevTables& t, const float* ref, const float* var_ref,
                           const uint16_t* mask_ref, const float* img, const float* var_img,
                           const uint16_t* mask_img, float* out, float* out_var,
                           uint16_t* out_mask, double* cov_out, int cov_out_w, bool stats,
                           cudaStream_t st) {
  uint16_t* mask_dst = out_mask ? out_mask : (stats ? b.mask_tmp : nullptr);
  k_dual_split<<<1, 256, 0, st>>>(h.dsol, p.Nb * p.Ns, h.dsol2, h.dsol3);
  cudaError_t e = launch_rbad(p, t, h.dsol3, h.st, st, true);
  if (e != cudaSuccess) return PSFM_ERR_CUDA;
  if (mask_dst) {
    prof_begin("mask", st);
    e = launch_mask(p, b, mask_ref, mask_img, mask_dst, st, 1);
    if (e == cudaSuccess) e = launch_mask(p, b, mask_ref, mask_img, mask_dst, st, 2);
    prof_end("mask", st, 6);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  prof_begin("conv_image", st);
  e = launch_conv_image(p, t, h.dsol, ref, mask_ref, img, out, st);
  if (e == cudaSuccess) e = launch_conv_image(p, t, h.dsol2, img, mask_img, out, out, st);
  prof_end("conv_image", st, 2);
  if (e != cudaSuccess) return PSFM_ERR_CUDA;
  if (out_var || stats) {
    prof_begin("variance", st);
    e = launch_variance(p, t, h.dsol, var_ref, mask_ref, nullptr, nullptr, 1, nullptr, out_var,
                        h.st, nullptr, st);
    if (e == cudaSuccess)
      e = launch_variance(p, t, h.dsol3, var_img, mask_img, out_var, nullptr, 1,
                          stats ? mask_dst : nullptr, out_var, h.st, b.var_part, st);
    prof_end("variance", st, 2);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  if (cov_out) {
    prof_begin("covariance", st);
    const int w1 = 2 * p.w - 1;
    e = launch_cov(p, b, nullptr, 1, nullptr, 0, b.cov_tmp, w1, st);
    if (e == cudaSuccess) {
      ApplyBuffers b3 = b;
      b3.dsol = h.dsol3;
      e = launch_cov(p, b3, nullptr, 1, b.cov_tmp, w1, cov_out, cov_out_w, st);
    }
    prof_end("covariance", st, 6);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  return PSFM_OK;
}

}  // namespace

psfm_status run_apply(const Plan& p, const Head& h, const ApplyBuffers& b, const float* ref,
                      const float* var_ref, const uint16_t* mask_ref, const float* img,
                      const float* var_img, const uint16_t* mask_img, const double* cov_ref,
                      int c_ref, const double* cov_img, int c_img, float* out, float* out_var,
                      uint16_t* out_mask, double* cov_out, int cov_out_w, bool stats,
                      cudaStream_t st) {
  const DevTables t = bind_tables(h.tables, h.offs);
  if (p.cfg.dual) {
    // the dual kernel convolves I2 as well, so it needs the science image; white inputs
    if (!img || !var_img || !mask_img) return PSFM_ERR_BAD_ARG;
    if (cov_ref || cov_img || (out_var && !var_ref)) return PSFM_ERR_UNSUPPORTED;
    return run_apply_dual(p, h, b, t, ref, var_ref, mask_ref, img, var_img, mask_img, out,
                          out_var, out_mask, cov_out, cov_out_w, stats, st);
  }
  const bool diff = img != nullptr;
  uint16_t* mask_dst = out_mask ? out_mask : (stats ? b.mask_tmp : nullptr);
  cudaError_t e = cudaSuccess;
  if (mask_dst) {
    prof_begin("mask", st);
    e = launch_mask(p, b, mask_ref, diff ? mask_img : nullptr, mask_dst, st);
    prof_end("mask", st, 3);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  prof_begin("conv_image", st);
  e = launch_conv_image(p, t, h.dsol, ref, mask_ref, img, out, st);
  prof_end("conv_image", st, 1);
  if (e != cudaSuccess) return PSFM_ERR_CUDA;
  if (out_var || stats) {
    prof_begin("variance", st);
    e = launch_variance(p, t, h.dsol, var_ref, mask_ref, diff ? var_img : nullptr,
                        cov_ref, c_ref, stats ? mask_dst : nullptr, out_var, h.st, b.var_part,
                        st);
    prof_end("variance", st, 1);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  if (cov_out) {
    prof_begin("covariance", st);
    e = launch_cov(p, b, cov_ref, c_ref, cov_img, c_img, cov_out, cov_out_w, st);
    prof_end("covariance", st, 3);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  return PSFM_OK;
}


// Stacking (Sec. 5.1-5.2): per input, render the target, solve, convolve with statistics,
// accumulate.  The stack accumulators sit at the start of the workspace; each input's
// solve and apply buffers follow.
psfm_status run_stack_impl(int n, const float* const* imgs, const float* const* vars,
                           const uint16_t* const* masks, psfm_shape shape,
                           const double* const* src_xyf, const int32_t* n_src, double fwhm,
                           const psfm_basis_spec* basis, const psfm_config* cfg, float* out,
                           float* out_var, uint16_t* out_mask, int32_t* out_count,
                           double* cov_out, int cov_out_w, psfm_solution* sols, char* base,
                           size_t ws_bytes, cudaStream_t st) {
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
  Plan p0;
  psfm_status s = make_plan(p0, shape, &basis[0], cfg, 0);
  if (s != PSFM_OK) return s;
  // each input is matched to the rendered target, which has no noise to convolve
  if (cfg->dual) return PSFM_ERR_UNSUPPORTED;
  Workspace ws;
  ws.base = base;
  ws.size = ws_bytes;
  StackBuffers kb;
  carve_stack(p0, ws, kb, n_src_max);
  const size_t stack_bytes = ws.used;
  if (stack_bytes > ws_bytes) return PSFM_ERR_WORKSPACE;
  const size_t npx = (size_t)shape.height * shape.pitch;
  if (cudaMemsetAsync(out, 0, sizeof(float) * npx, st) != cudaSuccess ||
      cudaMemsetAsync(out_var, 0, sizeof(float) * npx, st) != cudaSuccess ||
      cudaMemsetAsync(out_count, 0, sizeof(int32_t) * npx, st) != cudaSuccess ||
      cudaMemsetAsync(kb.acc_w, 0, sizeof(float) * npx, st) != cudaSuccess ||
      cudaMemsetAsync(kb.zero_var, 0, sizeof(float) * npx, st) != cudaSuccess ||
      cudaMemsetAsync(kb.zero_m, 0, sizeof(uint16_t) * npx, st) != cudaSuccess ||
      cudaMemsetAsync(kb.pm_acc, 0, sizeof(double) * kMaxCovOut * kMaxCovOut, st) !=
          cudaSuccess ||
      cudaMemsetAsync(kb.wsum, 0, sizeof(double) * 2, st) != cudaSuccess)
    return PSFM_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    Plan p;
    s = make_plan(p, shape, &basis[i], cfg, 0);
    if (s != PSFM_OK) return s;
    Workspace w2;
    w2.base = base + stack_bytes;
    w2.size = ws_bytes - stack_bytes;
    Head h;
    w2.used = head_layout(p, h);
    head_bind(h, w2.base, p);
    ApplyBuffers b;
    carve_apply(p, w2, b);
    SolveBuffers sb;
    carve_solve(p, w2, sb);
    if (stack_bytes + w2.used > ws_bytes) return PSFM_ERR_WORKSPACE;
    b.tab = bind_tables(h.tables, h.offs);
    b.st = h.st;
    b.dsol = h.dsol;
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
                  nullptr, 0, kb.conv, kb.conv_var, kb.conv_m, cov_out ? kb.pm : nullptr, ni, true,
                  st);
    if (s != PSFM_OK) return s;
    prof_begin("stack_accum", st);
    if (launch_stack_accum(p, kb.conv, kb.conv_var, kb.conv_m, h.st, out, out_var, kb.acc_w,
                           out_count, st) != cudaSuccess)
      return PSFM_ERR_CUDA;
    if (cov_out &&
        launch_stack_cov_accum(kb.pm, ni, cov_out_w, h.st, kb.pm_acc, kb.wsum, st) != cudaSuccess)
      return PSFM_ERR_CUDA;
    prof_end("stack_accum", st, cov_out ? 2 : 1);
    if (sols)
      s = fetch_solution(p, h.st, h.dsol, sb, &sols[i], st);
    else
      s = sync_status(h.st, st);
    if (s != PSFM_OK) return s;
  }
  prof_begin("stack_final", st);
  if (launch_stack_final(p0, out, out_var, out_mask, kb.acc_w, out_count, kb.pm_acc, kb.wsum,
                         cov_out, cov_out_w, st) != cudaSuccess)
    return PSFM_ERR_CUDA;
  prof_end("stack_final", st, cov_out ? 2 : 1);
  return cudaStreamSynchronize(st) == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

psfm_status run_stack(int n, const float* const* imgs, const float* const* vars,
                      const uint16_t* const* masks, psfm_shape shape,
                      const double* const* src_xyf, const int32_t* n_src, double target_fwhm,
                      const psfm_basis_spec* basis, const psfm_config* cfg, float* out,
                      float* out_var, uint16_t* out_mask, int32_t* out_count, double* cov_out,
                      int cov_out_w, psfm_solution* sols, char* ws, size_t ws_bytes,
                      cudaStream_t s) {
  return run_stack_impl(n, imgs, vars, masks, shape, src_xyf, n_src, target_fwhm, basis, cfg,
                        out, out_var, out_mask, out_count, cov_out, cov_out_w, sols, ws,
                        ws_bytes, s);
}

}  // namespace psfm

extern "C" {

void psfm_config_default(psfm_config* c) {
  if (!c) return;
  c->grid_nx = 6;
  c->grid_ny = 5;
  c->stamp_half = -1;
  c->max_cand = 8;
  c->thresh_nsigma = 5.0;
  c->reject_nsigma = 3.0;
  c->soften_alpha = 0.1;
  c->bad_frac = 0.2;
  c->max_iter = 5;
  c->var_tile = 64;
  c->cov_grid = 5;
  c->norm_mode = PSFM_NORM_SEPARATE;
  c->precision = PSFM_PREC_FP64;
  c->badmask = 0x00FF;
  c->conv_bad = (uint16_t)(1u << 14);
  c->conv_poor = (uint16_t)(1u << 15);
  c->nodata = 1;
  c->dual = 0;
  c->penalty = 1e-2;
}

const char* psfm_status_string(psfm_status s) {
  switch (s) {
    case PSFM_OK: return "ok";
    case PSFM_ERR_BAD_ARG: return "bad argument";
    case PSFM_ERR_TOO_FEW_STAMPS: return "fewer than 3 usable stamps";
    case PSFM_ERR_SINGULAR: return "normal equations singular";
    case PSFM_ERR_NONFINITE: return "non-finite input pixel";
    case PSFM_ERR_CUDA: return "CUDA error";
    case PSFM_ERR_TIMEOUT: return "device wait timed out";
    case PSFM_ERR_WORKSPACE: return "workspace too small or table overflow";
    case PSFM_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int32_t psfm_basis_size(const psfm_basis_spec* b) {
  if (!b || b->n_gauss < 1 || b->n_gauss > PSFM_MAX_GAUSS) return -1;
  int n = 0;
  for (int g = 0; g < b->n_gauss; ++g) {
    if (b->degree[g] < 0 || b->degree[g] > PSFM_MAX_DEGREE) return -1;
    n += (b->degree[g] + 1) * (b->degree[g] + 2) / 2;
  }
  return n;
}

int32_t psfm_spatial_size(const psfm_basis_spec* b) {
  if (!b || b->spatial_order < 0 || b->spatial_order > PSFM_MAX_SPATIAL_ORDER) return -1;
  return (b->spatial_order + 1) * (b->spatial_order + 2) / 2;
}

int32_t psfm_cov_width(const psfm_basis_spec* b, int32_t cov_in_w, int32_t cov_img_w) {
  if (!b || b->half_width < 1 || b->half_width > PSFM_MAX_HALF_WIDTH) return -1;
  if (cov_in_w < 1 || cov_in_w % 2 == 0 || cov_in_w > kMaxCovIn) return -1;
  if (cov_img_w < 0 || (cov_img_w > 0 && cov_img_w % 2 == 0)) return -1;
  const int n = 2 * (2 * b->half_width + 1) + cov_in_w - 2;
  return n > cov_img_w ? n : cov_img_w;
}

size_t psfm_workspace_size(int32_t op, psfm_shape shape, const psfm_basis_spec* basis,
                           const psfm_config* cfg, int32_t n_stamps) {
  if (op < PSFM_OP_SOLVE || op > PSFM_OP_STACK) return 0;
  Plan p;
  if (make_plan(p, shape, basis, cfg, op == PSFM_OP_STACK ? 0 : n_stamps) != PSFM_OK) return 0;
  Workspace ws;
  ws.measuring = true;
  if (op == PSFM_OP_STACK) {
    StackBuffers kb;
    carve_stack(p, ws, kb, n_stamps);
  }
  Head h;
  ws.used += head_layout(p, h);
  if (op == PSFM_OP_CONVOLVE || op == PSFM_OP_SUBTRACT || op == PSFM_OP_STACK) {
    ApplyBuffers b;
    carve_apply(p, ws, b);
  }
  if (op == PSFM_OP_SOLVE || op == PSFM_OP_SUBTRACT || op == PSFM_OP_STACK) {
    SolveBuffers sb;
    carve_solve(p, ws, sb);
  }
  return ws.used;
}

psfm_status psfm_convolve(const float* ref, const float* var_ref, const uint16_t* mask_ref,
                          const float* img, const float* var_img, const uint16_t* mask_img,
                          psfm_shape shape, const psfm_basis_spec* basis,
                          const psfm_config* cfg, const psfm_solution* sol,
                          const double* cov_ref, int32_t cov_ref_w, const double* cov_img,
                          int32_t cov_img_w, float* out, float* out_var, uint16_t* out_mask,
                          double* cov_out, int32_t cov_out_w, void* workspace,
                          size_t ws_bytes, psfm_stream stream) {
  Plan p;
  psfm_status s = make_plan(p, shape, basis, cfg, 0);
  if (s != PSFM_OK) return s;
  const bool diff = img != nullptr;
  if (!ref || !mask_ref || !out || !sol || !workspace) return PSFM_ERR_BAD_ARG;
  if (out_var && !var_ref) return PSFM_ERR_BAD_ARG;
  if (diff && (!mask_img || (out_var && !var_img))) return PSFM_ERR_BAD_ARG;
  if (!diff && (var_img || mask_img || cov_img)) return PSFM_ERR_BAD_ARG;
  if (cov_out && diff && !var_ref) return PSFM_ERR_BAD_ARG;
  if (cov_out && diff && !var_img) return PSFM_ERR_BAD_ARG;
  if (!sol->coeff || sol->n_coeff < p.ncoef) return PSFM_ERR_BAD_ARG;
  if (sol->r_bad < 0 || sol->r_bad > p.h) return PSFM_ERR_BAD_ARG;
  if (!aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  int c_ref = 1, c_img = 0;
  s = check_cov(p, cov_ref, cov_ref_w, diff, cov_img, cov_img_w, cov_out, cov_out_w, &c_ref,
                &c_img);
  if (s != PSFM_OK) return s;

  Head h;
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = ws_bytes;
  ws.used = head_layout(p, h);
  head_bind(h, ws.base, p);
  ApplyBuffers b;
  carve_apply(p, ws, b);
  if (ws.used > ws_bytes) return PSFM_ERR_WORKSPACE;
  b.tab = bind_tables(h.tables, h.offs);
  b.st = h.st;
  b.dsol = h.dsol;

  std::vector<double> vals(2 + p.ncoef);
  vals[0] = sol->b0;
  vals[1] = sol->d0;
  for (int i = 0; i < p.ncoef; ++i) vals[2 + i] = sol->coeff[i];
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (upload_head(p, h, vals.data(), sol->r_bad, st) != cudaSuccess) return PSFM_ERR_CUDA;
  return run_apply(p, h, b, ref, var_ref, mask_ref, img, var_img, mask_img, cov_ref, c_ref,
                   cov_img, c_img, out, out_var, out_mask, cov_out, cov_out_w,
                   cov_out != nullptr && diff, st);
}

psfm_status psfm_solve_kernel(const float* img, const float* ref, const float* var_img,
                              const float* var_ref, const uint16_t* mask_img,
                              const uint16_t* mask_ref, psfm_shape shape,
                              const psfm_stamp* stamps, int32_t n_stamps,
                              const psfm_basis_spec* basis, const psfm_config* cfg,
                              psfm_solution* out, void* workspace, size_t ws_bytes,
                              psfm_stream stream) {
  Plan p;
  psfm_status s = make_plan(p, shape, basis, cfg, n_stamps);
  if (s != PSFM_OK) return s;
  if (!img || !ref || !var_img || !var_ref || !mask_img || !mask_ref || !out || !workspace)
    return PSFM_ERR_BAD_ARG;
  if (n_stamps > 0 && !stamps) return PSFM_ERR_BAD_ARG;
  if (!aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  Head h;
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = ws_bytes;
  ws.used = head_layout(p, h);
  head_bind(h, ws.base, p);
  SolveBuffers sb;
  carve_solve(p, ws, sb);
  if (ws.used > ws_bytes) return PSFM_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (upload_head(p, h, nullptr, 0, st) != cudaSuccess) return PSFM_ERR_CUDA;
  const DevTables t = bind_tables(h.tables, h.offs);
  s = run_solve(p, t, h.st, h.dsol, sb, img, ref, var_img, var_ref, mask_img, mask_ref, stamps,
                st);
  if (s != PSFM_OK) return s;
  return fetch_solution(p, h.st, h.dsol, sb, out, st);
}

psfm_status psfm_subtract(const float* img, const float* ref, const float* var_img,
                          const float* var_ref, const uint16_t* mask_img,
                          const uint16_t* mask_ref, psfm_shape shape,
                          const psfm_stamp* stamps, int32_t n_stamps,
                          const psfm_basis_spec* basis, const psfm_config* cfg,
                          const double* cov_ref, int32_t cov_ref_w, const double* cov_img,
                          int32_t cov_img_w, float* diff, float* diff_var,
                          uint16_t* diff_mask, double* cov_out, int32_t cov_out_w,
                          psfm_solution* out, void* workspace, size_t ws_bytes,
                          psfm_stream stream) {
  Plan p;
  psfm_status s = make_plan(p, shape, basis, cfg, n_stamps);
  if (s != PSFM_OK) return s;
  if (!img || !ref || !var_img || !var_ref || !mask_img || !mask_ref || !diff || !workspace)
    return PSFM_ERR_BAD_ARG;
  if (n_stamps > 0 && !stamps) return PSFM_ERR_BAD_ARG;
  if (!aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  int c_ref = 1, c_img = 0;
  s = check_cov(p, cov_ref, cov_ref_w, true, cov_img, cov_img_w, cov_out, cov_out_w, &c_ref,
                &c_img);
  if (s != PSFM_OK) return s;
  Head h;
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = ws_bytes;
  ws.used = head_layout(p, h);
  head_bind(h, ws.base, p);
  ApplyBuffers b;
  carve_apply(p, ws, b);
  SolveBuffers sb;
  carve_solve(p, ws, sb);
  if (ws.used > ws_bytes) return PSFM_ERR_WORKSPACE;
  b.tab = bind_tables(h.tables, h.offs);
  b.st = h.st;
  b.dsol = h.dsol;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (upload_head(p, h, nullptr, 0, st) != cudaSuccess) return PSFM_ERR_CUDA;
  s = run_solve(p, b.tab, h.st, h.dsol, sb, img, ref, var_img, var_ref, mask_img, mask_ref,
                stamps, st);
  if (s != PSFM_OK) return s;
  s = run_apply(p, h, b, ref, var_ref, mask_ref, img, var_img, mask_img, cov_ref, c_ref, cov_img,
                c_img, diff, diff_var, diff_mask, cov_out, cov_out_w, cov_out != nullptr, st);
  if (s != PSFM_OK) return s;
  if (out) return fetch_solution(p, h.st, h.dsol, sb, out, st);
  return sync_status(h.st, st);
}

psfm_status psfm_stack(int32_t n, const float* const* imgs, const float* const* vars,
                       const uint16_t* const* masks, psfm_shape shape,
                       const double* const* src_xyf, const int32_t* n_src, double target_fwhm,
                       const psfm_basis_spec* basis, const psfm_config* cfg, float* out,
                       float* out_var, uint16_t* out_mask, int32_t* out_count,
                       double* cov_out, int32_t cov_out_w, psfm_solution* sols,
                       void* workspace, size_t ws_bytes, psfm_stream stream) {
  if (n < 1 || !imgs || !vars || !masks || !src_xyf || !n_src || !basis || !cfg || !out ||
      !out_var || !out_mask || !out_count || !workspace)
    return PSFM_ERR_BAD_ARG;
  if (!(target_fwhm > 0.0)) return PSFM_ERR_BAD_ARG;
  if (!aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return run_stack(n, imgs, vars, masks, shape, src_xyf, n_src, target_fwhm, basis, cfg, out,
                   out_var, out_mask, out_count, cov_out, cov_out_w, sols,
                   static_cast<char*>(workspace), ws_bytes, st);
}

}  // extern "C"
