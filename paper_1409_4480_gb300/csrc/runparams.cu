// Checking run parameters and building the device job description (host code).
#include <algorithm>

#include "runparams.h"

namespace colt {

int camera_axis(const double d[3], int* axis, int* sgn) {
  int nz = 0, ax = -1;
  for (int a = 0; a < 3; ++a) {
    if (d[a] != 0.0) { ++nz; ax = a; }
  }
  if (nz != 1 || std::fabs(d[ax]) != 1.0) return -1;
  *axis = ax;
  *sgn = d[ax] > 0 ? 1 : -1;
  return 0;
}

const char* check_run_params(const colt_run_params* p, bool has_luminosity) {
  if (!p) return "params is NULL";
  if (p->core_skip != COLT_SKIP_OFF && p->core_skip != COLT_SKIP_CELL_NL && p->core_skip != COLT_SKIP_JEANS)
    return "bad core_skip mode";
  if (p->source != COLT_SOURCE_POINT && p->source != COLT_SOURCE_CELLS) return "bad source";
  if (p->source == COLT_SOURCE_CELLS && !has_luminosity)
    return "COLT_SOURCE_CELLS needs colt_set_cell_luminosity on the grid";
  if (p->spec_nbins <= 0 || !(p->spec_hi > p->spec_lo)) return "bad escape-spectrum bins";
  if (p->n_cam < 0 || p->n_cam > kMaxCams) return "n_cam must be in [0, 8]";
  if (p->n_cam > 0) {
    if (!p->cams) return "cams is NULL";
    if (p->cam_nbins <= 0 || !(p->cam_hi > p->cam_lo)) return "bad camera bins";
    for (int i = 0; i < p->n_cam; ++i) {
      int ax, s;
      if (camera_axis(p->cams[i].dir, &ax, &s)) return "camera direction must be a coordinate axis";
      if (p->cams[i].npix < 0 || p->cams[i].npix > 65536) return "bad npix";
    }
  }
  if (p->precision != COLT_PLAIN && p->precision != COLT_MIXED) return "bad precision";
  if (p->phase != COLT_PHASE_DIPOLE && p->phase != COLT_PHASE_ISOTROPIC) return "bad phase";
  if (p->emission != COLT_EMIT_LINE_CENTRE && p->emission != COLT_EMIT_NATURAL_THERMAL)
    return "bad emission mode";
  if (p->spec_units != COLT_UNITS_X && p->spec_units != COLT_UNITS_DV_KMS) return "bad spec_units";
  if (p->n_cam > 0 && p->cam_units != COLT_UNITS_X && p->cam_units != COLT_UNITS_DV_KMS) return "bad cam_units";
  if ((p->spec_units == COLT_UNITS_X || (p->n_cam > 0 && p->cam_units == COLT_UNITS_X)) && !(p->T_ref > 0))
    return "T_ref must be > 0 for x units";
  if (!(p->tau_esc_max > 0)) return "tau_esc_max must be > 0";
  if (!(p->albedo >= 0 && p->albedo <= 1)) return "albedo must be in [0,1]";
  if (!(p->src_sigma >= 0)) return "src_sigma must be >= 0";
  if (p->n_sources < 0 || p->n_sources > kMaxSources) return "n_sources must be in [0, 16]";
  if (p->n_sources > 0) {
    if (!p->sources) return "sources is NULL";
    if (p->source != COLT_SOURCE_POINT) return "sources[] needs COLT_SOURCE_POINT";
    double wmax = 0;
    for (int i = 0; i < p->n_sources; ++i) {
      const colt_source& q = p->sources[i];
      if (!(q.sigma >= 0) || !std::isfinite(q.sigma)) return "source sigma must be >= 0";
      if (!(q.weight >= 0) || !std::isfinite(q.weight)) return "source weight must be >= 0";
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(q.pos[a])) return "source position must be finite";
      wmax = std::max(wmax, q.weight);
    }
    if (!(wmax > 0)) return "some source weight must be > 0";
  }
  return nullptr;
}

RunDev make_run_dev(const double lo[3], const double hi[3], const colt_run_params* p) {
  RunDev r;
  r.n_packets = p->n_packets;
  r.pid_offset = p->pid_offset;
  r.rng = Rng{uint32_t(p->seed), uint32_t(p->seed >> 32)};
  for (int a = 0; a < 3; ++a) r.src[a] = p->src_pos[a];
  r.src_sigma = p->src_sigma;
  if (p->n_sources > 0) {
    // integer weights floor(2^(63 - b) w / max w), 2^b >= n + 1: they sum below 2^63
    const int n = p->n_sources;
    double wmax = 0;
    for (int i = 0; i < n; ++i) wmax = std::max(wmax, p->sources[i].weight);
    int b = 0;
    while (b < 63 && (1ull << b) < (unsigned long long)n + 1) ++b;
    r.n_src = n;
    for (int i = 0; i < n; ++i) {
      for (int a = 0; a < 3; ++a) r.src_pos[i][a] = p->sources[i].pos[a];
      r.src_sig[i] = p->sources[i].sigma;
      r.src_total += (unsigned long long)std::floor(std::ldexp(p->sources[i].weight / wmax, 63 - b));
      r.src_cum[i] = r.src_total;
    }
  }
  r.core_skip = p->core_skip;
  r.recoil = p->recoil ? 1 : 0;
  r.phase = p->phase;
  r.emission = p->emission;
  r.source = p->source;
  r.jeans_c = jeans_coefficient();
  r.jeans_cf = (float)r.jeans_c;
  r.tau_max = p->tau_esc_max;
  r.albedo = p->albedo;
  r.max_scatter = p->max_scatter;
  const double vref = p->T_ref > 0 ? vth_kms(p->T_ref) : 1.0;
  r.spec_scale = p->spec_units == COLT_UNITS_X ? 1.0 / vref : -1.0;
  r.spec_lo = p->spec_lo;
  r.spec_hi = p->spec_hi;
  r.spec_nb = p->spec_nbins;
  r.n_cam = p->n_cam;
  int64_t off = 0;
  for (int i = 0; i < p->n_cam; ++i) {
    camera_axis(p->cams[i].dir, &r.cam[i].axis, &r.cam[i].sgn);
    r.cam[i].npix = p->cams[i].npix;
    r.cam[i].img_off = off;
    off += (int64_t)p->cams[i].npix * p->cams[i].npix * p->cam_nbins;
  }
  r.cam_scale = p->cam_units == COLT_UNITS_X ? 1.0 / vref : -1.0;
  r.cam_lo = p->cam_lo;
  r.cam_hi = p->cam_hi;
  r.cam_nb = p->cam_nbins > 0 ? p->cam_nbins : 1;
  double fov = 0;
  for (int a = 0; a < 3; ++a) {
    r.centre[a] = 0.5 * (lo[a] + hi[a]);
    fov = std::max(fov, 0.5 * (hi[a] - lo[a]));
  }
  r.fov_half = p->fov_half > 0 ? p->fov_half : fov;
  r.pix_scale = 0.5 / r.fov_half;
  r.cam_inv_width = p->cam_hi > p->cam_lo ? (double)r.cam_nb / (p->cam_hi - p->cam_lo) : 1.0;
  fill_f32(r);
  return r;
}

}  // namespace colt
