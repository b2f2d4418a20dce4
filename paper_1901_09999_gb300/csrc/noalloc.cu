// psfm_convolve_noalloc: the image / variance / mask part of psfm_convolve for callers that
// cannot allocate device memory and cannot hand the library a workspace.
//
// Some hosts of this library cannot call cudaMalloc: plugins loaded into a pipeline whose
// device memory pool is owned by the host application, and real-time schedulers that ban
// allocation once they have started.  This entry point needs no workspace: its scratch lives
// in a file-scope device array of fixed size, created when the library is loaded on each GPU
// and kept until the process exits.
//
// Limits and behaviour:
//   * images of at most 4096 x 4096 pixels (PSFM_ERR_WORKSPACE beyond that);
//   * no covariance pseudo-matrix (white input noise is assumed for the per-patch covariance
//     factor, f_t = 1);
//   * the first call on each device looks up the device address of the scratch array with
//     cudaGetSymbolAddress while that device is current; make that first call before any
//     stream capture;
//   * every call uploads its coefficients and tables from host memory with cudaMemcpyAsync
//     on the caller's stream;
//   * every call shares the one array: calls that overlap on the GPU (different streams, or
//     host threads without ordering) race on it and give undefined results.  Calls on one
//     stream are ordered and safe.  Each call rewrites every byte it later reads (the device
//     state block is re-uploaded and zeroed; the bit planes are rebuilt in full), so nothing
//     carries over from the previous call.
#include <cstring>
#include <mutex>
#include <vector>

#include "psfm_internal.h"

namespace {

constexpr int kNoAllocMaxW = 4096;
constexpr int kNoAllocMaxH = 4096;
constexpr size_t kHeadBytes = 64 * 1024;
constexpr size_t kPlaneBytes = (size_t)kNoAllocMaxH * (kNoAllocMaxW / 32) * sizeof(uint32_t);
constexpr size_t kScratchBytes = kHeadBytes + 3 * kPlaneBytes;  // 6.1 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
char* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
psfm_status scratch_address(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PSFM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PSFM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PSFM_ERR_CUDA;
    g_dev_ptr[dev] = static_cast<char*>(p);
  }
  *out = g_dev_ptr[dev];
  return PSFM_OK;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" psfm_status psfm_convolve_noalloc(
    const float* ref, const float* var_ref, const uint16_t* mask_ref, const float* img,
    const float* var_img, const uint16_t* mask_img, psfm_shape shape,
    const psfm_basis_spec* basis, const psfm_config* cfg, const psfm_solution* sol, float* out,
    float* out_var, uint16_t* out_mask, psfm_stream stream) {
  using namespace psfm;
  Plan p;
  psfm_status s = make_plan(p, shape, basis, cfg, 0);
  if (s != PSFM_OK) return s;
  if (cfg->dual) return PSFM_ERR_UNSUPPORTED;  // the dual kernel's passes need a workspace
  const bool diff = img != nullptr;
  if (!ref || !mask_ref || !out || !sol) return PSFM_ERR_BAD_ARG;
  if (out_var && !var_ref) return PSFM_ERR_BAD_ARG;
  if (diff && (!mask_img || (out_var && !var_img))) return PSFM_ERR_BAD_ARG;
  if (!diff && (var_img || mask_img)) return PSFM_ERR_BAD_ARG;
  if (!sol->coeff || sol->n_coeff < p.ncoef) return PSFM_ERR_BAD_ARG;
  if (sol->r_bad < 0 || sol->r_bad > p.h) return PSFM_ERR_BAD_ARG;
  if (p.W > kNoAllocMaxW || p.H > kNoAllocMaxH) return PSFM_ERR_WORKSPACE;

  // head: [DevState][b0, d0, coeff][tables], as in the workspace of psfm_convolve
  std::vector<char> blob;
  size_t offs[7];
  pack_tables(p, blob, offs);
  const size_t o_dsol = al256(sizeof(DevState));
  const size_t o_tab = al256(o_dsol + sizeof(double) * (2 + p.ncoef));
  const size_t head = al256(o_tab + blob.size());
  if (head > kHeadBytes) return PSFM_ERR_WORKSPACE;

  char* base = nullptr;
  s = scratch_address(&base);
  if (s != PSFM_OK) return s;

  std::vector<char> host(head, 0);
  DevState ds = {};
  ds.r_bad = sol->r_bad;
  std::memcpy(host.data(), &ds, sizeof(ds));
  double* hv = reinterpret_cast<double*>(host.data() + o_dsol);
  hv[0] = sol->b0;
  hv[1] = sol->d0;
  for (int i = 0; i < p.ncoef; ++i) hv[2 + i] = sol->coeff[i];
  std::memcpy(host.data() + o_tab, blob.data(), blob.size());
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(base, host.data(), head, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PSFM_ERR_CUDA;

  char* t = base + o_tab;
  DevTables tab;
  tab.f1d = reinterpret_cast<float*>(t + offs[0]);
  tab.f1d64 = reinterpret_cast<double*>(t + offs[1]);
  tab.psi = reinterpret_cast<double*>(t + offs[2]);
  tab.sk = reinterpret_cast<double*>(t + offs[3]);
  tab.term = reinterpret_cast<int32_t*>(t + offs[4]);
  tab.spat = reinterpret_cast<int32_t*>(t + offs[5]);
  tab.pen = reinterpret_cast<double*>(t + offs[6]);
  DevState* dst = reinterpret_cast<DevState*>(base);
  const double* dsol = reinterpret_cast<const double*>(base + o_dsol);

  ApplyBuffers b = {};
  b.tab = tab;
  b.st = dst;
  b.dsol = const_cast<double*>(dsol);
  b.bits = reinterpret_cast<uint32_t*>(base + kHeadBytes);
  b.hb_bad = reinterpret_cast<uint32_t*>(base + kHeadBytes + kPlaneBytes);
  b.hb_poor = reinterpret_cast<uint32_t*>(base + kHeadBytes + 2 * kPlaneBytes);

  if (out_mask) {
    prof_begin("mask", st);
    const cudaError_t e = launch_mask(p, b, mask_ref, diff ? mask_img : nullptr, out_mask, st);
    prof_end("mask", st, 3);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  prof_begin("conv_image", st);
  cudaError_t e = launch_conv_image(p, tab, dsol, ref, mask_ref, img, out, st);
  prof_end("conv_image", st, 1);
  if (e != cudaSuccess) return PSFM_ERR_CUDA;
  if (out_var) {
    prof_begin("variance", st);
    e = launch_variance(p, tab, dsol, var_ref, mask_ref, diff ? var_img : nullptr, nullptr, 1,
                        nullptr, out_var, dst, nullptr, st);
    prof_end("variance", st, 1);
    if (e != cudaSuccess) return PSFM_ERR_CUDA;
  }
  return PSFM_OK;
}
