// Image convolution entry (Eq. 12): fills the launch parameters and dispatches on the kernel
// half width to the unit that instantiates it (k_conv.cuh holds the kernel), with the launch
// shape (tile height) of the tuning table for the basis class, and the autotuner that fills
// the table by timing every shape on a synthetic image.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "host.h"
#include "k_conv.cuh"

namespace psfm {
namespace {

std::mutex g_tmu;
std::vector<psfm_tune_entry> g_tune;

bool same_class(const psfm_tune_entry& e, int h, int S, int ng, const int* deg) {
  if (e.half_width != h || e.spatial_order != S || e.n_gauss != ng) return false;
  for (int g = 0; g < ng; ++g)
    if (e.degree[g] != deg[g]) return false;
  return true;
}

conv::ConvParams conv_params(const Plan& p, const DevTables& t, const double* dsol,
                             const float* ref, const uint16_t* mref, const float* img,
                             float* out) {
  conv::ConvParams P;
  P.b = basis_dev(p);
  P.g = ImgGeom{p.W, p.H, p.pitch};
  P.ref = ref;
  P.mref = mref;
  P.img = img;
  P.out = out;
  P.f1d = t.f1d;
  P.psi = t.psi;
  P.sk = t.sk;
  P.dsol = dsol;
  P.xscale = p.W > 1 ? (float)(2.0 / (p.W - 1)) : 0.f;
  P.yscale = p.H > 1 ? (float)(2.0 / (p.H - 1)) : 0.f;
  P.badmask = p.cfg.badmask;
  P.ty = kConvTY;
  return P;
}

cudaError_t dispatch(int h, const conv::ConvParams& P, cudaStream_t st) {
  if (h >= 1 && h <= 6) return conv::launch_range_1_6(h, P, st);
  if (h >= 7 && h <= 10) return conv::launch_range_7_10(h, P, st);
  if (h >= 11 && h <= 13) return conv::launch_range_11_13(h, P, st);
  if (h >= 14 && h <= 15) return conv::launch_range_14_15(h, P, st);
  if (h >= 16 && h <= 17) return conv::launch_range_16_17(h, P, st);
  if (h >= 18 && h <= 19) return conv::launch_range_18_19(h, P, st);
  if (h >= 20 && h <= 21) return conv::launch_range_20_21(h, P, st);
  if (h >= 22 && h <= 24) return conv::launch_range_22_24(h, P, st);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_conv_image(const Plan& p, const DevTables& t, const double* dsol,
                              const float* ref, const uint16_t* mref, const float* img,
                              float* out, cudaStream_t st) {
  conv::ConvParams P = conv_params(p, t, dsol, ref, mref, img, out);
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (const auto& e : g_tune)
      if (same_class(e, p.h, p.S, p.ng, p.deg)) {
        P.ty = e.tile_rows;
        break;
      }
  }
  return dispatch(p.h, P, st);
}

// Synthetic tuning images: a sky-like reference with a hashed texture, about 2 % of the pixels
// masked, and a science image for the difference mode.
__global__ void k_tune_fill(int W, int H, int64_t pitch, float* ref, float* img, uint16_t* mask) {
  const int64_t n = (int64_t)H * pitch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = (uint32_t)i * 2654435761u;
    v ^= v >> 15;
    v *= 2246822519u;
    v ^= v >> 13;
    ref[i] = 500.f + (float)(v & 1023);
    img[i] = 510.f + (float)((v >> 10) & 1023);
    mask[i] = (v >> 24) < 5 ? (uint16_t)1 : (uint16_t)0;
  }
}

}  // namespace psfm

namespace {

struct TuneLayout {
  size_t ref = 0, img = 0, mask = 0, out = 0, dsol = 0, tab = 0, total = 0;
};

TuneLayout tune_layout(const psfm::Plan& p, size_t blob) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  TuneLayout L;
  const size_t npx = (size_t)p.H * p.pitch;
  L.ref = 0;
  L.img = al(L.ref + sizeof(float) * npx);
  L.mask = al(L.img + sizeof(float) * npx);
  L.out = al(L.mask + sizeof(uint16_t) * npx);
  L.dsol = al(L.out + sizeof(float) * npx);
  L.tab = al(L.dsol + sizeof(double) * (2 + p.ncoef));
  L.total = al(L.tab + blob);
  return L;
}

}  // namespace

extern "C" {

size_t psfm_tune_conv_workspace_size(int32_t width, int32_t height,
                                     const psfm_basis_spec* basis) {
  psfm_config c;
  psfm_config_default(&c);
  psfm::Plan p;
  if (!basis || psfm::make_plan(p, psfm_shape{width, height, width}, basis, &c, 0) != PSFM_OK)
    return 0;
  std::vector<char> blob;
  size_t offs[7];
  psfm::pack_tables(p, blob, offs);
  return tune_layout(p, blob.size()).total;
}

psfm_status psfm_tune_conv(int32_t width, int32_t height, const psfm_basis_spec* basis,
                           void* workspace, size_t ws_bytes, psfm_stream stream,
                           psfm_tune_entry* out) {
  using namespace psfm;
  psfm_config c;
  psfm_config_default(&c);
  Plan p;
  if (!basis || !workspace) return PSFM_ERR_BAD_ARG;
  psfm_status s = make_plan(p, psfm_shape{width, height, width}, basis, &c, 0);
  if (s != PSFM_OK) return s;
  if (!aligned256(workspace)) return PSFM_ERR_BAD_ARG;
  std::vector<char> blob;
  size_t offs[7];
  pack_tables(p, blob, offs);
  const TuneLayout L = tune_layout(p, blob.size());
  if (ws_bytes < L.total) return PSFM_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  // synthetic reference and science images with a few masked pixels (difference mode, as in
  // a subtraction) and a solution with every coefficient non-zero
  std::vector<double> sol(2 + p.ncoef);
  sol[0] = 1.0;
  sol[1] = 0.5;
  for (int i = 0; i < p.ncoef; ++i) sol[2 + i] = 0.01 * ((i * 7919) % 13 - 6);
  const size_t npx = (size_t)p.H * p.pitch;
  k_tune_fill<<<1024, 256, 0, st>>>(p.W, p.H, p.pitch, reinterpret_cast<float*>(base + L.ref),
                                    reinterpret_cast<float*>(base + L.img),
                                    reinterpret_cast<uint16_t*>(base + L.mask));
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(base + L.dsol, sol.data(), sizeof(double) * sol.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + L.tab, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PSFM_ERR_CUDA;
  const DevTables t = bind_tables(base + L.tab, offs);
  conv::ConvParams P = conv_params(p, t, reinterpret_cast<const double*>(base + L.dsol),
                                   reinterpret_cast<const float*>(base + L.ref),
                                   reinterpret_cast<const uint16_t*>(base + L.mask),
                                   reinterpret_cast<const float*>(base + L.img),
                                   reinterpret_cast<float*>(base + L.out));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PSFM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PSFM_ERR_CUDA;
  }
  psfm_tune_entry best = {};
  best.ms = -1.f;
  s = PSFM_OK;
  for (int ty : {64, 128}) {
    {
      P.ty = ty;
      if (dispatch(p.h, P, st) != cudaSuccess) {  // shape not legal for this basis
        cudaGetLastError();
        continue;
      }
      float t3[3];
      for (int r = 0; r < 3 && s == PSFM_OK; ++r) {
        if (cudaEventRecord(e0, st) != cudaSuccess || dispatch(p.h, P, st) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t3[r], e0, e1) != cudaSuccess)
          s = PSFM_ERR_CUDA;
      }
      if (s != PSFM_OK) break;
      std::sort(t3, t3 + 3);
      if (best.ms < 0.f || t3[1] < best.ms) {
        best.ms = t3[1];
        best.tile_rows = ty;
        best.plane_chunk = conv::kMaxChunk;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PSFM_OK) return s;
  if (best.ms < 0.f) return PSFM_ERR_UNSUPPORTED;
  best.half_width = p.h;
  best.spatial_order = p.S;
  best.n_gauss = p.ng;
  for (int g = 0; g < PSFM_MAX_GAUSS; ++g) best.degree[g] = g < p.ng ? p.deg[g] : 0;
  s = psfm_tune_set(&best);
  if (s == PSFM_OK && out) *out = best;
  return s;
}

int32_t psfm_tune_count(void) {
  std::lock_guard<std::mutex> lk(psfm::g_tmu);
  return (int32_t)psfm::g_tune.size();
}

psfm_status psfm_tune_get(int32_t i, psfm_tune_entry* out) {
  std::lock_guard<std::mutex> lk(psfm::g_tmu);
  if (!out || i < 0 || i >= (int32_t)psfm::g_tune.size()) return PSFM_ERR_BAD_ARG;
  *out = psfm::g_tune[i];
  return PSFM_OK;
}

psfm_status psfm_tune_set(const psfm_tune_entry* e) {
  if (!e || e->half_width < 1 || e->half_width > PSFM_MAX_HALF_WIDTH || e->n_gauss < 1 ||
      e->n_gauss > PSFM_MAX_GAUSS || e->spatial_order < 0 ||
      e->spatial_order > PSFM_MAX_SPATIAL_ORDER ||
      (e->tile_rows != 64 && e->tile_rows != 128) ||
      (e->plane_chunk != 0 && e->plane_chunk != psfm::conv::kMaxChunk))
    return PSFM_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lk(psfm::g_tmu);
  for (auto& x : psfm::g_tune)
    if (psfm::same_class(x, e->half_width, e->spatial_order, e->n_gauss, e->degree)) {
      x = *e;
      return PSFM_OK;
    }
  psfm::g_tune.push_back(*e);
  return PSFM_OK;
}

void psfm_tune_clear(void) {
  std::lock_guard<std::mutex> lk(psfm::g_tmu);
  psfm::g_tune.clear();
}

}  // extern "C"
