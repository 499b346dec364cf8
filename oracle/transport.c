/*
 * Oracle (test infrastructure only): the packet loop, in FP64.
 *
 *   Sec. 3.1.1, Eq. init_freq : emission (x_i = 0 at line centre, Sec. 3.1.1
 *                               allows it for optically thick media)
 *   Sec. 3.1.2, Eq. lnR       : tau_event = -ln R, cell-by-cell walk, Eq. tauH
 *   Sec. 3.1.3                : scattering (see scatter.c)
 *   Sec. 3.2.4                : a tau_0 = a tau_cell + a tau_NL, Eq. atau0min,
 *                               or the Jeans estimate a tau_J, Eq. atau0J
 *   Sec. 3.1.1                : diffuse emission from the gas: a cell drawn
 *                               with probability proportional to its
 *                               (quantised) luminosity, a uniform position in it
 *   Sec. 6.1, Eq. SB          : next-event (peel-off) estimator, sum of
 *                               W(theta) exp(-tau_esc), traced only while
 *                               tau_esc <= tau_esc_max (50 in the paper)
 *
 * Readings taken here (the paper is silent on them):
 *   - dust (absent from the paper) is grey with opacity k_d per cell; an
 *     interaction is dust with probability k_d / (k_HI H + k_d); dust absorbs
 *     with probability 1 - A, else scatters isotropically with the comoving
 *     frequency unchanged;
 *   - the emission event itself is peeled off with weight exp(-tau_esc);
 *     dust scatterings peel off with W = 1;
 *   - the peel-off weight is W(mu) = (1 + RQ mu^2) / (1 + RQ/3) (isotropic
 *     scattering = 1), with the R/Q drawn for the actual scattering;
 *   - the escape frequency is the lab-frame x_lab = x + k.u of the last cell,
 *     reported either as x relative to the Doppler width at T_ref or as
 *     Delta v = -x_lab v_th (red = positive Delta v);
 *   - cameras are distant observers along coordinate axes; the image axes of
 *     a camera along +/-e_a are (+/-e_{a+1}, e_{a+2}) (indices mod 3), the
 *     image plane is centred on the box with half-width fov_half; peel-off
 *     rays along a periodic axis have no observer and contribute nothing;
 *   - spectral bins are half-open [lo, hi); escapes outside the range are
 *     counted as under/overflow;
 *   - a flight that visits more than 2^24 cells (only possible on periodic
 *     grids with empty cells) ends the packet as capped.
 * RNG: event 0 is the emission (block 0: mu, phi, tau_event; block 1: source
 * Gaussian, or for diffuse emission words 0-1 as one 64-bit number choosing
 * the cell; block 3: the position in that cell); event e >= 1 is the e-th
 * interaction, blocks as in scatter.c.
 */
#include "grid.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#include <unistd.h>

#define O_PI 3.14159265358979323846
#define O_MAX_TRIALS 1000000
#define IMG_BUF 8192
/* A flight visiting more cells than this (possible only on periodic grids
 * with empty cells) ends the packet as capped. */
#define O_MAX_FLIGHT_VISITS (1u << 24)

typedef struct {
  const o_grid* g;
  const o_params* p;
  o_result* res;
  uint32_t key[2];
  double vth_ref;
  int tid, nthreads;
  pthread_mutex_t* img_lock;
  /* private tallies */
  uint64_t n_emitted, n_escaped, n_absorbed, n_capped, n_scat, n_scat_hi, n_cell, n_peel;
  uint64_t under, over;
  uint64_t* spec;
  double* cam_spec;
  double* cam_spec2;
  double* cam_total;
  int64_t img_n;
  int64_t* img_idx;
  double* img_w;
  /* diffuse emission: inclusive prefix sums of the cell weights, and their total */
  const uint64_t* lum_cum;
  uint64_t lum_total;
} worker;

/* H(a,x): App. A1's approximation, or the quadrature in the exact-physics mode */
static double H_of(const o_params* p, double a, double x) {
  return p->exact ? o_H_exact(a, x) : o_H_approx(a, x);
}

static void draw_block(const uint32_t key[2], uint64_t pid, uint32_t event, uint32_t blk, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), event, blk};
  uint32_t r[4];
  o_philox4x32_10(ctr, key, r);
  for (int i = 0; i < 4; ++i) u[i] = o_uniform(r[i]);
}

static double dot3(const double p[3], const double q[3]) {
  return p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
}

static void flush_image(worker* w) {
  if (w->img_n == 0) return;
  pthread_mutex_lock(w->img_lock);
  for (int64_t i = 0; i < w->img_n; ++i) w->res->cam_image[w->img_idx[i]] += w->img_w[i];
  pthread_mutex_unlock(w->img_lock);
  w->img_n = 0;
}

static int camera_axis(const double d[3], int* sgn) {
  int a = 0;
  if (fabs(d[1]) > fabs(d[a])) a = 1;
  if (fabs(d[2]) > fabs(d[a])) a = 2;
  *sgn = d[a] > 0.0 ? 1 : -1;
  return a;
}

static double spectral_coord(int units, double x_lab, double vth, double vth_ref) {
  return units == 0 ? x_lab * vth / vth_ref : -x_lab * vth;
}

static int bin_of(double s, double lo, double hi, int nb) {
  if (!(s >= lo) || !(s < hi)) return -1;
  int b = (int)floor((s - lo) * (double)nb / (hi - lo));
  if (b < 0 || b >= nb) return -1;
  return b;
}

/* Sec. 6.1: one peel-off ray from position r in cell c, comoving frequency
 * x_c there, towards camera cam, with phase weight W. */
static void peel(worker* w, int cam, const double r0[3], int64_t c0, double x_c, double W) {
  const o_grid* g = w->g;
  const o_params* p = w->p;
  const double* k = p->cams[cam].dir;
  int sgn;
  int cax = camera_axis(k, &sgn);
  if (g->periodic_xy && cax < 2) return;
  double r[3] = {r0[0], r0[1], r0[2]};
  int64_t c = c0;
  double x = x_c;
  double tau = 0.0;
  for (;;) {
    double clo[3], chi[3];
    o_cell_bounds(g, c, clo, chi);
    int ax;
    double l = o_exit_distance(clo, chi, r, k, &ax);
    double H = H_of(p, g->a[c], x);
    tau += (g->kHI[c] * H + g->kd[c]) * l;
    w->n_peel++;
    if (tau > p->tau_esc_max) return;
    for (int i = 0; i < 3; ++i) r[i] += l * k[i];
    int64_t nx = o_next_cell(g, c, ax, r, k);
    if (nx < 0) break;
    /* Sec. 3.1.2: frequency in the new cell's comoving frame */
    x = (x + dot3(k, &g->u[3 * c])) * (g->vth[c] / g->vth[nx]) - dot3(k, &g->u[3 * nx]);
    c = nx;
  }
  double x_lab = x + dot3(k, &g->u[3 * c]);
  double s = spectral_coord(p->cam_units, x_lab, g->vth[c], w->vth_ref);
  double wt = W * exp(-tau);
  if (w->cam_total) w->cam_total[cam] += wt;
  int b = bin_of(s, p->cam_lo, p->cam_hi, p->cam_nbins);
  if (b < 0) return;
  if (w->cam_spec) w->cam_spec[(size_t)cam * p->cam_nbins + b] += wt;
  if (w->cam_spec2) w->cam_spec2[(size_t)cam * p->cam_nbins + b] += wt * wt;
  int npix = p->cams[cam].npix;
  if (npix > 0 && w->res->cam_image) {
    /* image plane axes of this camera */
    int au = (cax + 1) % 3, av = (cax + 2) % 3;
    double cu = 0.5 * (g->lo[au] + g->hi[au]), cv = 0.5 * (g->lo[av] + g->hi[av]);
    double pu = sgn * (r0[au] - cu), pv = r0[av] - cv;
    double fu = (pu + p->fov_half) / (2.0 * p->fov_half) * npix;
    double fv = (pv + p->fov_half) / (2.0 * p->fov_half) * npix;
    if (fu >= 0.0 && fu < npix && fv >= 0.0 && fv < npix) {
      int64_t iu = (int64_t)floor(fu), iv = (int64_t)floor(fv);
      /* offset of this camera's cube within the image buffer */
      int64_t off = 0;
      for (int q = 0; q < cam; ++q) off += (int64_t)p->cams[q].npix * p->cams[q].npix * p->cam_nbins;
      int64_t idx = off + ((iv * npix + iu) * p->cam_nbins) + b;
      w->img_idx[w->img_n] = idx;
      w->img_w[w->img_n] = wt;
      if (++w->img_n == IMG_BUF) flush_image(w);
    }
  }
}

static void peel_all_hi(worker* w, const double r[3], int64_t c, double x, const double ki[3],
                        const double u_atom[3], double g, double RQ) {
  for (int cam = 0; cam < w->p->n_cam; ++cam) {
    const double* kc = w->p->cams[cam].dir;
    double mu_c = dot3(ki, kc);
    double W = (1.0 + RQ * mu_c * mu_c) / (1.0 + RQ / 3.0);
    double dk[3] = {kc[0] - ki[0], kc[1] - ki[1], kc[2] - ki[2]};
    double x_c = x + dot3(dk, u_atom) + g * (mu_c - 1.0);
    peel(w, cam, r, c, x_c, W);
  }
}

static void peel_all_iso(worker* w, const double r[3], int64_t c, double x) {
  for (int cam = 0; cam < w->p->n_cam; ++cam) peel(w, cam, r, c, x, 1.0);
}

static void run_packet(worker* w, uint64_t idx) {
  const uint64_t pid = w->p->pid0 + idx;
  const o_grid* g = w->g;
  const o_params* p = w->p;
  double B0[4], B1[4];
  w->n_emitted++;
  /* emission, event 0 */
  draw_block(w->key, pid, 0, 0, B0);
  double mu = 2.0 * B0[0] - 1.0, phi = 2.0 * O_PI * B0[1];
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double k[3] = {st * cos(phi), st * sin(phi), mu};
  double tau = -log(B0[2]);
  double r[3] = {p->src_pos[0], p->src_pos[1], p->src_pos[2]};
  int64_t c;
  if (p->source == 1) {
    /* diffuse emission: t uniform on [0, W) from the 64-bit word (block 1,
     * words 0 and 1) as floor(word W / 2^64); the cell is the first whose
     * inclusive prefix weight exceeds t; the position is uniform inside it */
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), 0u, 1u}, q[4];
    o_philox4x32_10(ctr, w->key, q);
    uint64_t word = ((uint64_t)q[1] << 32) | q[0];
    uint64_t t = (uint64_t)(((unsigned __int128)word * w->lum_total) >> 64);
    int64_t lo = 0, hi = g->n_cells - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (w->lum_cum[mid] > t) hi = mid; else lo = mid + 1;
    }
    c = lo;
    double B3[4], clo[3], chi[3];
    draw_block(w->key, pid, 0, 3, B3);
    o_cell_bounds(g, c, clo, chi);
    for (int i = 0; i < 3; ++i) r[i] = clo[i] + B3[i] * (chi[i] - clo[i]);
  } else {
    double sigma = p->src_sigma;
    if (p->n_sources > 0) {
      /* several point sources, chosen with probability proportional to their
       * weights: integer weights w_s = floor(2^(63-b) weight_s / max weight),
       * b the least integer with 2^b >= n + 1; t = floor(word W / 2^64) from
       * the 64-bit word of event-0 block 4 (words 0 and 1); the source is the
       * first whose inclusive prefix weight exceeds t */
      int n = p->n_sources, b = 0;
      double wmax = 0.0;
      for (int i = 0; i < n; ++i) if (p->sources[5 * i + 4] > wmax) wmax = p->sources[5 * i + 4];
      while (b < 63 && ((uint64_t)1 << b) < (uint64_t)n + 1) ++b;
      uint64_t W = 0;
      for (int i = 0; i < n; ++i) W += (uint64_t)floor(ldexp(p->sources[5 * i + 4] / wmax, 63 - b));
      uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), 0u, 4u}, q[4];
      o_philox4x32_10(ctr, w->key, q);
      uint64_t word = ((uint64_t)q[1] << 32) | q[0];
      uint64_t t = (uint64_t)(((unsigned __int128)word * W) >> 64);
      uint64_t cum = 0;
      int s = 0;
      for (; s < n; ++s) {
        cum += (uint64_t)floor(ldexp(p->sources[5 * s + 4] / wmax, 63 - b));
        if (cum > t) break;
      }
      for (int i = 0; i < 3; ++i) r[i] = p->sources[5 * s + i];
      sigma = p->sources[5 * s + 3];
    }
    if (sigma > 0.0) {
      draw_block(w->key, pid, 0, 1, B1);
      double rho1 = sqrt(-2.0 * log(B1[0])), rho2 = sqrt(-2.0 * log(B1[2]));
      r[0] += sigma * rho1 * cos(2.0 * O_PI * B1[1]);
      r[1] += sigma * rho1 * sin(2.0 * O_PI * B1[1]);
      r[2] += sigma * rho2 * cos(2.0 * O_PI * B1[3]);
    }
    c = o_locate_cell(g, r, k);
  }
  double x = 0.0;
  uint64_t nscat = 0;
  int status = 0;
  double s_esc = 0.0;
  if (c < 0) {
    /* source outside the domain: leaves at once, at line centre */
    status = 1;
    s_esc = 0.0;
  } else if (p->emission == 1) {
    /* Sec. 3.1.1: x_i = x_nat + k_i.u_atom in the source cell's frame, x_nat
     * from the natural (Lorentzian) profile a / (pi (x^2 + a^2)) and each atom
     * velocity component (in units of v_th) Gaussian of variance 1/2.  Draws:
     * block 0 word 3 (x_nat), block 2 (Box-Muller: u_x, u_y from words 0-1,
     * u_z from words 2-3).  The emission is isotropic in the atom's frame, so
     * the photon sent towards a camera has x_nat + k_c.u_atom (W = 1). */
    double B2[4];
    draw_block(w->key, pid, 0, 2, B2);
    double rho1 = sqrt(-log(B2[0])), rho2 = sqrt(-log(B2[2]));
    double ua[3] = {rho1 * cos(2.0 * O_PI * B2[1]), rho1 * sin(2.0 * O_PI * B2[1]), rho2 * cos(2.0 * O_PI * B2[3])};
    x = g->a[c] * tan(O_PI * (B0[3] - 0.5)) + dot3(k, ua);
    peel_all_hi(w, r, c, x, k, ua, 0.0, 0.0);
  } else {
    peel_all_iso(w, r, c, x);
  }
  uint32_t event = 0;
  while (status == 0) {
    /* Sec. 3.1.2: march until tau_event is spent or the packet leaves */
    int interact = 0;
    uint32_t visits = 0;
    for (;;) {
      if (++visits > O_MAX_FLIGHT_VISITS) { status = 3; break; }
      double clo[3], chi[3];
      o_cell_bounds(g, c, clo, chi);
      int ax;
      double l = o_exit_distance(clo, chi, r, k, &ax);
      double ktot = g->kHI[c] * H_of(p, g->a[c], x) + g->kd[c];
      double tau_cell = ktot * l;
      w->n_cell++;
      if (tau <= tau_cell) {
        double le = tau / ktot;
        for (int i = 0; i < 3; ++i) r[i] += le * k[i];
        interact = 1;
        break;
      }
      tau -= tau_cell;
      for (int i = 0; i < 3; ++i) r[i] += l * k[i];
      int64_t nx = o_next_cell(g, c, ax, r, k);
      if (nx < 0) break;
      x = (x + dot3(k, &g->u[3 * c])) * (g->vth[c] / g->vth[nx]) - dot3(k, &g->u[3 * nx]);
      c = nx;
    }
    if (status == 3) break;
    if (!interact) {
      double x_lab = x + dot3(k, &g->u[3 * c]);
      s_esc = spectral_coord(p->spec_units, x_lab, g->vth[c], w->vth_ref);
      status = 1;
      break;
    }
    /* interaction, event e */
    ++event;
    draw_block(w->key, pid, event, 0, B0);
    double H = H_of(p, g->a[c], x);
    double ktot = g->kHI[c] * H + g->kd[c];
    if (B0[0] * ktot < g->kd[c]) {
      /* dust */
      if (B0[1] >= p->albedo) { status = 2; break; }
      draw_block(w->key, pid, event, 1, B1);
      double m = 2.0 * B1[2] - 1.0, f = 2.0 * O_PI * B1[3];
      double sm = sqrt(fmax(0.0, 1.0 - m * m));
      k[0] = sm * cos(f); k[1] = sm * sin(f); k[2] = m;
      nscat++;
      peel_all_iso(w, r, c, x);
    } else {
      o_scatter_io s;
      memset(&s, 0, sizeof(s));
      s.x = x;
      for (int i = 0; i < 3; ++i) s.k[i] = k[i];
      s.a = g->a[c];
      s.g = p->recoil ? g->g[c] : 0.0;
      if (p->core_skip == 2)
        s.atau0 = o_atau_jeans(g->T[c], g->nHI[c]);
      else if (p->core_skip)
        s.atau0 = g->a[c] * g->kHI[c] * o_min_face_distance(g, c, r) + g->atau_nl[c];
      else
        s.atau0 = -1.0;
      s.phase = p->phase;
      s.exact = p->exact;
      s.pid = pid;
      s.event = event;
      o_scatter_hi(&s, w->key);
      if (s.n_trials > O_MAX_TRIALS) { status = 3; break; }
      nscat++;
      w->n_scat_hi++;
      peel_all_hi(w, r, c, x, k, s.u_atom, s.g, s.RQ);
      for (int i = 0; i < 3; ++i) k[i] = s.k_f[i];
      x = s.x_f;
    }
    if (nscat >= p->max_scatter) {
      /* capped by the scattering limit: report the lab-frame frequency the
       * packet has at that moment */
      double x_lab = x + dot3(k, &g->u[3 * c]);
      s_esc = spectral_coord(p->spec_units, x_lab, g->vth[c], w->vth_ref);
      status = 3;
      break;
    }
    tau = -log(B0[2]);
  }
  w->n_scat += nscat;
  if (status == 1) {
    w->n_escaped++;
    int b = bin_of(s_esc, p->spec_lo, p->spec_hi, p->spec_nbins);
    if (b >= 0) w->spec[b]++;
    else if (s_esc < p->spec_lo) w->under++;
    else w->over++;
  } else if (status == 2) {
    w->n_absorbed++;
  } else {
    w->n_capped++;
  }
  if (p->pk_status) p->pk_status[idx] = status;
  if (p->pk_nscat) p->pk_nscat[idx] = nscat;
  if (p->pk_freq) p->pk_freq[idx] = (status == 1 || status == 3) ? s_esc : 0.0;
}

#define CHUNK 16

static void* worker_main(void* arg) {
  worker* w = (worker*)arg;
  uint64_t n = w->p->n_packets;
  for (uint64_t ch = (uint64_t)w->tid; ch * CHUNK < n; ch += (uint64_t)w->nthreads) {
    uint64_t end = (ch + 1) * CHUNK;
    if (end > n) end = n;
    for (uint64_t pid = ch * CHUNK; pid < end; ++pid) run_packet(w, pid);
  }
  flush_image(w);
  return NULL;
}

/* A derived grid (cell quantities, a tau_NL when core_skip == 1, the
 * luminosity weights when source == 1), reusable by several runs whose
 * parameters agree on core_skip, f_nl and source. */
struct o_prepared {
  o_grid g;
  int core_skip, source;
  double f_nl;
  uint64_t* lum_cum;
  uint64_t lum_total;
  double seconds;
};

o_prepared* o_prepare(const o_grid_in* gin, const o_params* p) {
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  o_prepared* pg = (o_prepared*)calloc(1, sizeof(o_prepared));
  if (!pg) return NULL;
  if (o_grid_build(gin, &pg->g)) { free(pg); return NULL; }
  pg->core_skip = p->core_skip;
  pg->source = p->source;
  pg->f_nl = p->f_nl;
  if (p->core_skip == 1) o_atau_nl_grid(&pg->g, p->f_nl);
  /* diffuse emission: integer weights w_c = floor(2^s L_c / max L) with
   * s = 63 - b, b the least integer with 2^b >= n_cells + 1 (the weights then
   * sum below 2^63), and their inclusive prefix sums */
  if (p->source == 1) {
    int64_t n = pg->g.n_cells;
    double lmax = 0.0;
    int ok = gin->lum != NULL;
    for (int64_t i = 0; ok && i < n; ++i) {
      if (!(gin->lum[i] >= 0.0) || !isfinite(gin->lum[i])) ok = 0;
      else if (gin->lum[i] > lmax) lmax = gin->lum[i];
    }
    if (!ok || !(lmax > 0.0)) { o_prepared_free(pg); return NULL; }
    int b = 0;
    while (b < 63 && ((uint64_t)1 << b) < (uint64_t)n + 1) ++b;
    pg->lum_cum = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i) {
      pg->lum_total += (uint64_t)floor(ldexp(gin->lum[i] / lmax, 63 - b));
      pg->lum_cum[i] = pg->lum_total;
    }
  } else if (p->source != 0) {
    o_prepared_free(pg);
    return NULL;
  }
  clock_gettime(CLOCK_MONOTONIC, &t1);
  pg->seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
  return pg;
}

void o_prepared_free(o_prepared* pg) {
  if (!pg) return;
  free(pg->lum_cum);
  o_grid_free(&pg->g);
  free(pg);
}

int o_run_prepared(const o_prepared* pg, const o_params* p, o_result* res) {
  if (p->spec_nbins <= 0 || !(p->spec_hi > p->spec_lo) || !res->spec) return -1;
  if (p->n_cam < 0 || (p->n_cam > 0 && (!p->cams || p->cam_nbins <= 0 || !(p->cam_hi > p->cam_lo)))) return -1;
  if (p->source != pg->source || (p->core_skip == 1) != (pg->core_skip == 1) ||
      (p->core_skip == 1 && p->f_nl != pg->f_nl))
    return -1;
  const o_grid* gp = &pg->g;
  struct timespec tm, t1;
  clock_gettime(CLOCK_MONOTONIC, &tm);
  int nt = p->n_threads;
  if (nt <= 0) nt = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nt < 1) nt = 1;
  pthread_mutex_t lock;
  pthread_mutex_init(&lock, NULL);
  worker* ws = (worker*)calloc((size_t)nt, sizeof(worker));
  pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
  size_t ncs = (size_t)(p->n_cam > 0 ? p->n_cam : 0) * (size_t)(p->cam_nbins > 0 ? p->cam_nbins : 0);
  for (int t = 0; t < nt; ++t) {
    worker* w = &ws[t];
    w->g = gp; w->p = p; w->res = res;
    w->key[0] = (uint32_t)p->seed; w->key[1] = (uint32_t)(p->seed >> 32);
    w->vth_ref = o_vth_kms(p->T_ref > 0.0 ? p->T_ref : 1.0e4);
    w->tid = t; w->nthreads = nt; w->img_lock = &lock;
    w->lum_cum = pg->lum_cum; w->lum_total = pg->lum_total;
    w->spec = (uint64_t*)calloc((size_t)p->spec_nbins, sizeof(uint64_t));
    if (ncs) {
      w->cam_spec = (double*)calloc(ncs, sizeof(double));
      w->cam_spec2 = (double*)calloc(ncs, sizeof(double));
      w->cam_total = (double*)calloc((size_t)p->n_cam, sizeof(double));
    }
    w->img_idx = (int64_t*)malloc(IMG_BUF * sizeof(int64_t));
    w->img_w = (double*)malloc(IMG_BUF * sizeof(double));
  }
  if (res->cam_image) {
    size_t nimg = 0;
    for (int q = 0; q < p->n_cam; ++q) nimg += (size_t)p->cams[q].npix * p->cams[q].npix * p->cam_nbins;
    memset(res->cam_image, 0, nimg * sizeof(double));
  }
  for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, worker_main, &ws[t]);
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  /* merge in thread order */
  memset(res->spec, 0, (size_t)p->spec_nbins * sizeof(uint64_t));
  res->n_emitted = res->n_escaped = res->n_absorbed = res->n_capped = 0;
  res->n_scat = res->n_scat_hi = res->n_cell_visits = res->n_peel_visits = 0;
  res->spec_under = res->spec_over = 0;
  if (res->cam_spec) memset(res->cam_spec, 0, ncs * sizeof(double));
  if (res->cam_spec2) memset(res->cam_spec2, 0, ncs * sizeof(double));
  if (res->cam_total) memset(res->cam_total, 0, (size_t)p->n_cam * sizeof(double));
  for (int t = 0; t < nt; ++t) {
    worker* w = &ws[t];
    res->n_emitted += w->n_emitted; res->n_escaped += w->n_escaped;
    res->n_absorbed += w->n_absorbed; res->n_capped += w->n_capped;
    res->n_scat += w->n_scat; res->n_scat_hi += w->n_scat_hi;
    res->n_cell_visits += w->n_cell; res->n_peel_visits += w->n_peel;
    res->spec_under += w->under; res->spec_over += w->over;
    for (int b = 0; b < p->spec_nbins; ++b) res->spec[b] += w->spec[b];
    for (size_t i = 0; i < ncs; ++i) {
      if (res->cam_spec) res->cam_spec[i] += w->cam_spec[i];
      if (res->cam_spec2) res->cam_spec2[i] += w->cam_spec2[i];
    }
    if (res->cam_total) for (int q = 0; q < p->n_cam; ++q) res->cam_total[q] += w->cam_total[q];
    free(w->spec); free(w->cam_spec); free(w->cam_spec2); free(w->cam_total);
    free(w->img_idx); free(w->img_w);
  }
  free(ws); free(th);
  pthread_mutex_destroy(&lock);
  clock_gettime(CLOCK_MONOTONIC, &t1);
  res->n_threads_used = nt;
  res->transport_seconds = (double)(t1.tv_sec - tm.tv_sec) + 1e-9 * (double)(t1.tv_nsec - tm.tv_nsec);
  res->seconds = res->transport_seconds;
  return 0;
}

int o_run(const o_grid_in* gin, const o_params* p, o_result* res) {
  if (p->spec_nbins <= 0 || !(p->spec_hi > p->spec_lo) || !res->spec) return -1;
  if (p->n_cam < 0 || (p->n_cam > 0 && (!p->cams || p->cam_nbins <= 0 || !(p->cam_hi > p->cam_lo)))) return -1;
  o_prepared* pg = o_prepare(gin, p);
  if (!pg) return -1;
  int rc = o_run_prepared(pg, p, res);
  if (rc == 0) res->seconds = pg->seconds + res->transport_seconds;
  o_prepared_free(pg);
  return rc;
}
