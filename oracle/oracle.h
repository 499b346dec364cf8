/*
 * FP64 CPU oracle for the Lyman-alpha Monte-Carlo radiative-transfer
 * packet loop of Smith, Safranek-Shrader, Bromm & Milosavljevic (2014),
 * "The Lyman-alpha signature of the first galaxies" (the COLT method).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is double precision.  Each function names the passage of the
 * paper it follows (section / equation / appendix).  Where the paper is
 * silent, the reading taken is stated at the function.
 */
#ifndef COLT_ORACLE_H
#define COLT_ORACLE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- units -- */
/* Sec. 2: line constants as functions of T4 = T / 1e4 K. */
double o_vth_kms(double T);      /* v_th = 12.85 T4^(1/2) km/s            */
double o_damping_a(double T);    /* a    = 4.702e-4 T4^(-1/2)             */
double o_sigma0(double T);       /* sigma_0 = 5.898e-14 T4^(-1/2) cm^2    */
double o_recoil_g(double T);     /* g    = 2.536e-4 T4^(-1/2)  (Eq. recoil) */

/* --------------------------------------------------------------- Voigt -- */
double o_H_exact(double a, double x);   /* Sec. 2 integral, adaptive quadrature */
double o_H_approx(double a, double x);  /* App. A1, Eq. AB + Table AB            */
void   o_H_approx_many(const double* a, const double* x, double* H, size_t n);
void   o_H_exact_many(const double* a, const double* x, double* H, size_t n);
double o_x_cw_fit(double a);            /* Sec. 3.2.2, Eq. xcw (rational fit)    */
double o_x_cw_lambert(double a);        /* Sec. 3.2.2, Eq. xcw (W_{-1} solution) */
double o_x_crit(double atau0);          /* Sec. 3.2.4, Eq. xcrit                 */
double o_atau_jeans(double T, double n_HI);  /* Sec. 3.2.4, Eq. atau0J (n in cm^-3) */

/* ----------------------------------------------------------------- RNG -- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), counter-based. */
void     o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   o_uniform(uint32_t r);         /* ((r>>8)|1) * 2^-24, strictly in (0,1) */
void     o_philox_many(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n);

/* ------------------------------------------------------------ sampling -- */
typedef struct {
  /* inputs */
  double x;          /* incoming comoving frequency (cell Doppler units)       */
  double k[3];       /* incoming direction k_i (unit)                          */
  double a;          /* damping parameter of the cell                          */
  double g;          /* recoil parameter (0 = off)                             */
  double atau0;      /* a*tau_0 used for x_crit (core-skip); <0 => skipping off */
  int    phase;      /* 0 = dipole/anisotropic (Eq. phaseW), 1 = isotropic     */
  uint64_t pid;      /* packet id (RNG counter words 0,1)                      */
  uint32_t event;    /* event index (RNG counter word 2)                       */
  /* outputs */
  double x_f;        /* outgoing comoving frequency, Eq. x_f                   */
  double k_f[3];     /* outgoing direction                                     */
  double u_atom[3];  /* atom velocity (thermal units), u_par k_i + u_perp      */
  double u_par;      /* parallel component                                     */
  double x_crit;     /* critical frequency used                                */
  double RQ;         /* R/Q drawn for the phase function                       */
  double mu;         /* cos(theta) between k_i and k_f                         */
  int    n_trials;   /* rejection trials used for u_par                        */
  /* in */
  int    exact;      /* exact-physics mode: |x| >= 9 by numeric inversion      */
} o_scatter_io;

/* One resonant (HI) scattering, Sec. 3.1.3 + 3.2.3 + 3.2.4, with the RNG
 * counter layout shared (by specification, not code) with the CUDA path. */
void o_scatter_hi(o_scatter_io* s, const uint32_t key[2]);
void o_scatter_many(o_scatter_io* s, size_t n, const uint32_t key[2]);

/* Standalone u_par sampler on its own stream (for distribution pins). */
double o_sample_upar(double x, double a, uint64_t pid, uint32_t event,
                     const uint32_t key[2], int* n_trials);

/* Phase-function mu sampler by CDF inversion (for distribution pins). */
double o_sample_mu(double RQ, double u);
void   o_sample_upar_many(double x, double a, uint64_t pid0, uint32_t event,
                          const uint32_t key[2], double* out, int32_t* ntr, size_t n);
void   o_sample_upar_many_ex(double x, double a, uint64_t pid0, uint32_t event, const uint32_t key[2],
                             double* out, int32_t* ntr, size_t n, int exact);
void   o_sample_mu_many(double RQ, const double* u, double* mu, size_t n);

/* ---------------------------------------------------------------- grid -- */
typedef struct {
  int kind;                 /* 0 = Cartesian, 1 = octree                       */
  int nx, ny, nz;           /* Cartesian cell counts                           */
  double lo[3], hi[3];      /* box (cm)                                        */
  int periodic_xy;          /* 1: periodic in x and y (slab)                   */
  /* per-cell inputs (FP32 as supplied by the caller), length n_cells          */
  const float* n_HI;        /* cm^-3                                           */
  const float* T;           /* K (>0)                                          */
  const float* vx; const float* vy; const float* vz;  /* km/s                  */
  const float* k_dust;      /* cm^-1 (may be NULL = 0)                         */
  /* octree leaves (kind == 1): level and integer coordinates at that level   */
  int64_t n_leaves;
  const uint8_t*  leaf_level;
  const uint32_t* leaf_ijk;  /* 3 per leaf */
  /* per-cell luminosity for diffuse emission (source = 1), may be NULL       */
  const double* lum;
} o_grid_in;

typedef struct {
  double dir[3];            /* camera direction (unit, coordinate axis)        */
  int    npix;              /* image pixels per side (0 = spectrum only)       */
} o_camera;

typedef struct {
  uint64_t n_packets;
  uint64_t seed;
  double   src_pos[3];      /* cm */
  double   src_sigma;       /* Gaussian spread of the source (cm), 0 = point   */
  int      core_skip;       /* Sec. 3.2.4: 0 off, 1 a tau_cell + a tau_NL,
                               2 a tau_J of the scattering cell (Eq. atau0J)   */
  int      recoil;          /* Eq. recoil on/off                               */
  int      phase;           /* 0 dipole (Eq. phaseW), 1 isotropic              */
  double   f_nl;            /* non-local threshold, Eq. atauNL                 */
  double   tau_esc_max;     /* peel-off cutoff (Sec. 6.1), default 50          */
  double   albedo;          /* dust albedo A                                   */
  uint64_t max_scatter;     /* per-packet cap                                  */
  /* angle-averaged escape spectrum */
  int      spec_units;      /* 0 = x relative to T_ref, 1 = Delta v (km/s)     */
  double   T_ref;
  double   spec_lo, spec_hi;
  int      spec_nbins;
  /* cameras (peel-off, Sec. 6.1) */
  int      n_cam;
  const o_camera* cams;
  int      cam_units;       /* 0 = x (T_ref), 1 = Delta v                      */
  double   cam_lo, cam_hi;
  int      cam_nbins;
  double   fov_half;        /* half-width of the image plane (cm), centred on box */
  int      n_threads;       /* host threads (0 = all)                          */
  /* optional per-packet records (length n_packets), may be NULL */
  int32_t*  pk_status;      /* 1 escaped, 2 absorbed, 3 capped                 */
  uint64_t* pk_nscat;
  double*   pk_freq;        /* escape spectral coordinate; for packets capped by
                               max_scatter the lab frequency at the cap        */
  uint64_t  pid0;           /* packets are ids pid0 .. pid0 + n_packets - 1     */
  int       emission;       /* 0 line centre (x = 0), 1 natural + thermal        */
  int       source;         /* 0 point (src_pos, src_sigma), 1 cells by luminosity */
  int       n_sources;      /* 0: the one source src_pos / src_sigma; else n point
                               sources, 5 doubles each in `sources` (x, y, z, sigma,
                               weight); each packet draws its source by weight from
                               the 64-bit word of event-0 block 4 (integer weights as
                               for diffuse emission)                                  */
  const double* sources;
  int       exact;          /* exact-physics mode, for measuring the bias of the
                               approximations: H(a,x) by quadrature instead of
                               H_approx, and u_par at |x| >= 9 by numeric
                               inversion instead of the Gaussian (core-skipping
                               and recoil are the run's own switches)        */
} o_params;

typedef struct {
  uint64_t n_emitted, n_escaped, n_absorbed, n_capped;
  uint64_t n_scat;          /* executed scatterings (HI + dust)                */
  uint64_t n_scat_hi;
  uint64_t n_cell_visits;   /* main-march cell visits                          */
  uint64_t n_peel_visits;   /* peel-off cell visits                            */
  uint64_t spec_under, spec_over;
  uint64_t* spec;           /* [spec_nbins] escape counts (caller-allocated)   */
  double*   cam_spec;       /* [n_cam][cam_nbins]                 (nullable)   */
  double*   cam_spec2;      /* [n_cam][cam_nbins] sum of w^2      (nullable)   */
  double*   cam_image;      /* [n_cam][npix][npix][cam_nbins]     (nullable)   */
  double*   cam_total;      /* [n_cam] sum of all peel-off weights (nullable)  */
  int       n_threads_used;
  double    seconds;            /* whole call: grid derivation, a tau_NL, packets */
  double    transport_seconds;  /* the packet loop alone                          */
} o_result;

/* Non-local a*tau estimate per cell (Eq. atauNL); out has n_cells entries. */
int  o_atau_nl(const o_grid_in* g, double f_nl, double* out);

/* Full packet loop (Sec. 3.1 + 3.2 + 6.1). Returns 0 or a negative code. */
int  o_run(const o_grid_in* g, const o_params* p, o_result* r);

/* The same in two steps, so that several runs share one grid derivation:
 * o_prepare derives the cell quantities (plus a tau_NL when p->core_skip == 1
 * and the luminosity weights when p->source == 1; NULL on bad input), and
 * o_run_prepared runs p's packets on it (p must agree with the prepared
 * core_skip, f_nl and source; several calls may run at once on one prepared
 * grid, which they only read). */
typedef struct o_prepared o_prepared;
o_prepared* o_prepare(const o_grid_in* g, const o_params* p);
int  o_run_prepared(const o_prepared* pg, const o_params* p, o_result* r);
void o_prepared_free(o_prepared* pg);

/* Octree helpers exposed for parity tests of the walk (kind == 1 grids). */
int64_t o_octree_locate(const o_grid_in* g, const double pos[3], const double dir[3]);

#ifdef __cplusplus
}
#endif
#endif
