// Host-side planning: validates a basis and configuration, enumerates basis and spatial terms
// in canonical order, and computes in FP64 the separable 1-D factors, the L2 normalisation
// psi_k and the zero-sum offsets s_k of the ISIS basis (Eq. 7 and the zero-sum requirement of
// Sec. 2).
#include <cmath>
#include <cstring>

#include "psfm_internal.h"

namespace psfm {

BasisDev basis_dev(const Plan& p) {
  BasisDev b;
  b.h = p.h;
  b.w = p.w;
  b.wpad = p.wpad;
  b.ng = p.ng;
  b.S = p.S;
  b.Ns = p.Ns;
  b.Nb = p.Nb;
  b.NH = p.NH;
  b.dmax = p.dmax;
  for (int g = 0; g < PSFM_MAX_GAUSS; ++g) {
    b.deg[g] = p.deg[g];
    b.plane_base[g] = p.plane_base[g];
    b.kbase[g] = p.kbase[g];
  }
  return b;
}

psfm_status make_plan(Plan& p, psfm_shape shape, const psfm_basis_spec* b, const psfm_config* c,
                      int n_stamps) {
  if (!b || !c) return PSFM_ERR_BAD_ARG;
  if (shape.width < 1 || shape.height < 1 || shape.pitch < shape.width) return PSFM_ERR_BAD_ARG;
  if (shape.width > (1 << 24) || shape.height > (1 << 24)) return PSFM_ERR_BAD_ARG;
  if (b->n_gauss < 1 || b->n_gauss > PSFM_MAX_GAUSS) return PSFM_ERR_BAD_ARG;
  if (b->half_width < 1 || b->half_width > PSFM_MAX_HALF_WIDTH) return PSFM_ERR_BAD_ARG;
  if (b->spatial_order < 0 || b->spatial_order > PSFM_MAX_SPATIAL_ORDER) return PSFM_ERR_BAD_ARG;
  if (b->bg_order != 0) return PSFM_ERR_UNSUPPORTED;
  p.W = shape.width;
  p.H = shape.height;
  p.pitch = shape.pitch;
  p.h = b->half_width;
  p.w = 2 * p.h + 1;
  p.wpad = (p.w + 3) / 4 * 4;
  p.ng = b->n_gauss;
  p.S = b->spatial_order;
  p.Ns = (p.S + 1) * (p.S + 2) / 2;
  p.Nb = 0;
  p.NH = 0;
  p.dmax = 0;
  for (int g = 0; g < PSFM_MAX_GAUSS; ++g) {
    p.deg[g] = 0;
    p.sigma[g] = 0;
    p.plane_base[g] = 0;
    p.kbase[g] = 0;
  }
  for (int g = 0; g < p.ng; ++g) {
    const int d = b->degree[g];
    const double s = b->sigma[g];
    if (d < 0 || d > PSFM_MAX_DEGREE || !(s > 0.0) || !std::isfinite(s)) return PSFM_ERR_BAD_ARG;
    p.deg[g] = d;
    p.sigma[g] = s;
    p.plane_base[g] = p.NH;
    p.kbase[g] = p.Nb;
    for (int pp = 0; pp <= d; ++pp)
      for (int q = 0; q <= d - pp; ++q) {
        p.tg[p.Nb] = g;
        p.tp[p.Nb] = pp;
        p.tq[p.Nb] = q;
        ++p.Nb;
      }
    p.NH += d + 1;
    if (d > p.dmax) p.dmax = d;
  }
  int si = 0;
  for (int l = 0; l <= p.S; ++l)
    for (int m = 0; m <= p.S - l; ++m) {
      p.sl[si] = l;
      p.sm[si] = m;
      ++si;
    }
  p.Nd = c->dual ? 2 * p.Nb : p.Nb;
  p.ncoef = p.Nd * p.Ns;
  // 1-D factors f_{g,n}(t) = t^n exp(-t^2 / (2 sigma_g^2)), the Gaussian of Eq. 7 with the
  // decaying sign
  p.f1d.assign((size_t)p.NH * p.w, 0.0);
  for (int g = 0; g < p.ng; ++g)
    for (int n = 0; n <= p.deg[g]; ++n)
      for (int t = -p.h; t <= p.h; ++t) {
        const double G = std::exp(-(double)t * t / (2.0 * p.sigma[g] * p.sigma[g]));
        p.f1d[(size_t)(p.plane_base[g] + n) * p.w + (t + p.h)] = std::pow((double)t, n) * G;
      }
  // psi_k: unit L2 norm of psi f_p(u) f_q(v) (separable); s_k = sum of the normalised term
  // for p, q both even (the others sum to zero by symmetry)
  for (int k = 0; k < p.Nb; ++k) {
    const double* fp = &p.f1d[(size_t)(p.plane_base[p.tg[k]] + p.tp[k]) * p.w];
    const double* fq = &p.f1d[(size_t)(p.plane_base[p.tg[k]] + p.tq[k]) * p.w];
    double np = 0, nq = 0, sp = 0, sq = 0;
    for (int t = 0; t < p.w; ++t) {
      np += fp[t] * fp[t];
      nq += fq[t] * fq[t];
      sp += fp[t];
      sq += fq[t];
    }
    p.psi[k] = 1.0 / std::sqrt(np * nq);
    p.sk[k] = (p.tp[k] % 2 == 0 && p.tq[k] % 2 == 0) ? p.psi[k] * sp * sq : 0.0;
    // penalty p_k = sum_{u,v} (u^2 + v^2)^2 k_k(u, v)^2 (Sec. 2); the delta of the zero-sum
    // correction sits at u = v = 0 where the weight vanishes
    double pen = 0.0;
    for (int a = 0; a < p.w; ++a)
      for (int b2 = 0; b2 < p.w; ++b2) {
        const double u = a - p.h, v = b2 - p.h, r2 = u * u + v * v;
        const double kv = p.psi[k] * fp[a] * fq[b2];
        pen += r2 * r2 * kv * kv;
      }
    p.pen[k] = pen;
  }
  // configuration
  p.cfg = *c;
  if (c->grid_nx < 1 || c->grid_ny < 1 || c->grid_nx * c->grid_ny > 65536) return PSFM_ERR_BAD_ARG;
  if (c->max_cand < 1 || c->max_cand > 16) return PSFM_ERR_BAD_ARG;
  if (c->max_iter < 1 || c->max_iter > 16) return PSFM_ERR_BAD_ARG;
  if (c->cov_grid < 1 || c->cov_grid > 8) return PSFM_ERR_BAD_ARG;
  if (c->var_tile != kVarTile) return PSFM_ERR_UNSUPPORTED;
  if (c->norm_mode != PSFM_NORM_SEPARATE && c->norm_mode != PSFM_NORM_JOINT)
    return PSFM_ERR_BAD_ARG;
  if (c->dual != 0 && c->dual != 1) return PSFM_ERR_BAD_ARG;
  if (c->dual && (!(c->penalty >= 0.0) || !std::isfinite(c->penalty))) return PSFM_ERR_BAD_ARG;
  // the dual kernel is built on the double-float design and Gram
  if (c->dual && c->precision != PSFM_PREC_F32X2) return PSFM_ERR_UNSUPPORTED;
  if (c->precision != PSFM_PREC_FP64 && c->precision != PSFM_PREC_FP32 &&
      c->precision != PSFM_PREC_F32X2 && c->precision != PSFM_PREC_TF32 &&
      c->precision != PSFM_PREC_BF16X3 && c->precision != PSFM_PREC_BF16X6)
    return PSFM_ERR_BAD_ARG;
  if (!(c->thresh_nsigma >= 0.0) || !(c->reject_nsigma > 0.0) || !(c->soften_alpha >= 0.0) ||
      !(c->bad_frac >= 0.0 && c->bad_frac <= 1.0))
    return PSFM_ERR_BAD_ARG;
  p.s = c->stamp_half < 0 ? p.h : c->stamp_half;
  if (p.s > 32) return PSFM_ERR_BAD_ARG;
  p.sw = 2 * p.s + 1;
  p.P = p.sw * p.sw;
  p.foot = p.sw + 2 * p.h;
  p.n_stamps = n_stamps;
  if (n_stamps < 0) return PSFM_ERR_BAD_ARG;
  if (n_stamps > 0) {
    p.nreg = n_stamps;
    p.max_cand = 1;
  } else {
    p.nreg = c->grid_nx * c->grid_ny;
    p.max_cand = c->max_cand;
  }
  p.Nsys = p.ncoef + (c->norm_mode == PSFM_NORM_JOINT ? 2 : 0);
  p.Nc = p.Nd + 3;
  // the tensor-core Gram holds the augmented block in one 128-lane accumulator tile
  if ((c->precision == PSFM_PREC_TF32 || c->precision == PSFM_PREC_BF16X3) && p.Nc > 128)
    return PSFM_ERR_UNSUPPORTED;
  // (PSFM_PREC_BF16X6: the split-product Gram holds one N = 64 tile; a basis with more
  // augmented columns takes the double-float Gram, with the same double-float design)
  return PSFM_OK;
}

void pack_tables(const Plan& p, std::vector<char>& blob, size_t offs[7]) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t o = 0;
  offs[0] = o;  // f1d fp32 [NH][wpad]
  o = al(o + sizeof(float) * p.NH * p.wpad);
  offs[1] = o;  // f1d fp64 [NH][w]
  o = al(o + sizeof(double) * p.NH * p.w);
  offs[2] = o;  // psi
  o = al(o + sizeof(double) * p.Nb);
  offs[3] = o;  // sk
  o = al(o + sizeof(double) * p.Nb);
  offs[4] = o;  // term
  o = al(o + sizeof(int32_t) * p.Nb);
  offs[5] = o;  // spatial
  o = al(o + sizeof(int32_t) * p.Ns);
  offs[6] = o;  // penalty p_k
  o = al(o + sizeof(double) * p.Nb);
  blob.assign(o, 0);
  float* f32 = reinterpret_cast<float*>(blob.data() + offs[0]);
  double* f64 = reinterpret_cast<double*>(blob.data() + offs[1]);
  for (int pl = 0; pl < p.NH; ++pl)
    for (int t = 0; t < p.w; ++t) {
      f32[pl * p.wpad + t] = (float)p.f1d[(size_t)pl * p.w + t];
      f64[pl * p.w + t] = p.f1d[(size_t)pl * p.w + t];
    }
  std::memcpy(blob.data() + offs[2], p.psi, sizeof(double) * p.Nb);
  std::memcpy(blob.data() + offs[3], p.sk, sizeof(double) * p.Nb);
  int32_t* term = reinterpret_cast<int32_t*>(blob.data() + offs[4]);
  for (int k = 0; k < p.Nb; ++k) term[k] = p.tg[k] | (p.tp[k] << 8) | (p.tq[k] << 16);
  int32_t* sp = reinterpret_cast<int32_t*>(blob.data() + offs[5]);
  for (int s = 0; s < p.Ns; ++s) sp[s] = p.sl[s] | (p.sm[s] << 8);
  std::memcpy(blob.data() + offs[6], p.pen, sizeof(double) * p.Nb);
}

}  // namespace psfm
