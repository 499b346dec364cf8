/*
 * libcolt -- GB300 (sm_103a) Lyman-alpha Monte-Carlo radiative transfer.
 *
 * The packet transport loop of Smith, Safranek-Shrader, Bromm & Milosavljevic
 * (2014), "The Lyman-alpha signature of the first galaxies" (COLT): emission
 * (Sec. 3.1.1), optical-depth draws and the cell-by-cell march (Sec. 3.1.2,
 * Eq. lnR, Eq. tauH), resonant scattering with the u_par rejection sampler,
 * core-skipping, dipole phase function and recoil (Sec. 3.1.3, 3.2.1-3.2.4),
 * grey dust, and next-event (peel-off) camera tallies (Sec. 6.1, Eq. SB).
 *
 * Conventions for every call:
 *   - Return value: COLT_OK (0) or a negative colt_status.  No exception or
 *     abort crosses this boundary.  colt_last_error() gives a message.
 *   - Host pointers are read/written synchronously unless stated otherwise;
 *     device pointers are read on the context's stream.
 *   - The library owns every device buffer it allocates; callers keep
 *     ownership of everything they pass in.
 *   - One context per process and device.  All calls on a context are
 *     serialised by an internal mutex.
 *   - Units: lengths in cm, velocities in km/s, temperatures in K, densities
 *     in cm^-3, dust opacity in cm^-1.  Frequencies are the paper's
 *     x = (nu - nu_0) / Delta nu_D (Sec. 2) or Doppler velocity
 *     Delta v = -x v_th in km/s (red = positive).
 */
#ifndef COLT_H
#define COLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct colt_ctx colt_ctx;
typedef uint64_t colt_grid;   /* grid handle, 0 is never valid    */
typedef uint64_t colt_req;    /* request handle, 0 is never valid */

typedef enum {
  COLT_OK = 0,
  COLT_EINVAL = -1,     /* bad argument                                   */
  COLT_ENOMEM = -2,     /* would exceed the memory budget / allocation    */
  COLT_EAGAIN = -3,     /* not admitted yet (serving); retry later        */
  COLT_ETIMEOUT = -4,   /* a bounded wait ran out                         */
  COLT_ECUDA = -5,      /* a CUDA runtime call failed                     */
  COLT_ENOTFOUND = -6,  /* unknown handle                                 */
  COLT_EDEVICE = -7     /* a kernel raised its device-side error flag     */
} colt_status;

enum { COLT_CARTESIAN = 0, COLT_OCTREE = 1 };
enum { COLT_MEM_HOST = 0, COLT_MEM_DEVICE = 1 };
enum { COLT_PLAIN = 0, COLT_MIXED = 1 };          /* arithmetic of the transport */
enum { COLT_PHASE_DIPOLE = 0, COLT_PHASE_ISOTROPIC = 1 };
enum { COLT_UNITS_X = 0, COLT_UNITS_DV_KMS = 1 };
enum { COLT_EMIT_LINE_CENTRE = 0, COLT_EMIT_NATURAL_THERMAL = 1 };   /* Sec. 3.1.1 */
/* a tau_0 for the core-skipping cutoff x_crit (Sec. 3.2.4, Eq. xcrit):
 *   COLT_SKIP_CELL_NL  a tau_cell + a tau_NL (Eqs. atau0min, atauNL);
 *   COLT_SKIP_JEANS    the Jeans estimate of the scattering cell,
 *                      a tau_J = 6.428e4 T_4^(-1/2) (n_HI / cm^-3)^(1/2) (Eq. atau0J). */
enum { COLT_SKIP_OFF = 0, COLT_SKIP_CELL_NL = 1, COLT_SKIP_JEANS = 2 };
/* where packets are born (Sec. 3.1.1): a point (optionally Gaussian-spread)
 * source, or the gas itself with a per-cell luminosity (colt_set_cell_luminosity) */
enum { COLT_SOURCE_POINT = 0, COLT_SOURCE_CELLS = 1 };

/* ------------------------------------------------------------- context -- */
/* Create a context on CUDA device `device`.  mem_budget_bytes bounds what the
 * serving admission may hold resident (0 = 90% of free device memory).
 * cuda_stream (a cudaStream_t, may be NULL) is the stream all work runs on;
 * NULL makes the library create its own non-blocking stream.
 * Fails with COLT_ECUDA when no usable device exists. */
int colt_init(colt_ctx** ctx, int device, size_t mem_budget_bytes, void* cuda_stream);
void colt_finalize(colt_ctx* ctx);
const char* colt_last_error(colt_ctx* ctx);
/* SM count, L2 bytes and library build info (for reports). */
int colt_device_info(colt_ctx* ctx, int* sm_count, size_t* l2_bytes, int* cc_major, int* cc_minor);

/* ---------------------------------------------------------------- grids -- */
/* Per-cell inputs as the paper reads them (Sec. 3, first paragraph): density,
 * temperature and bulk velocity per cell, plus grey dust opacity.
 *   Cartesian: nx*ny*nz cells, x fastest, spanning the box [lo, hi).
 *   Octree: n_cells leaves; leaf i has refinement level leaf_level[i] (0 =
 *   root, at most 24) and integer coordinates leaf_ijk[3i..3i+2] at that
 *   level, i.e. it spans lo + ijk (hi-lo) 2^-level .. lo + (ijk+1) (hi-lo)
 *   2^-level.  The leaves must tile the box exactly, with fewer than 2^26 tree
 *   nodes (checked: COLT_EINVAL otherwise).  leaf_level / leaf_ijk are host
 *   arrays; the library builds a node table and per-leaf face neighbours
 *   (4 + 24 bytes per leaf beside the 32-byte record).
 * Field arrays (n_cells FP32 each) are host or device memory per fields_mem;
 * k_dust may be NULL (no dust).  T must be > 0 everywhere (empty cells carry
 * any positive temperature).
 * periodic_xy (Cartesian only): the box wraps in x and y (infinite slab).
 * f_nl: threshold of the non-local a*tau estimate (Sec. 3.2.4, Eq. atauNL),
 * computed once here on the device for every cell; 0 disables it.
 * The library copies the fields into its own packed device records. */
typedef struct {
  int kind;
  int nx, ny, nz;
  double lo[3], hi[3];
  int periodic_xy;
  int64_t n_cells;
  const uint8_t* leaf_level;
  const uint32_t* leaf_ijk;
  const float* n_HI;
  const float* T;
  const float* vx;
  const float* vy;
  const float* vz;
  const float* k_dust;
  int fields_mem;
  double f_nl;
} colt_grid_desc;

int colt_create_grid(colt_ctx* ctx, const colt_grid_desc* desc, colt_grid* out);
int colt_destroy_grid(colt_ctx* ctx, colt_grid grid);
/* Copy the packed per-cell records back to the host: 8 floats per cell,
 * (k_HI = n_HI sigma_0 [cm^-1], a, k_dust [cm^-1], 1/v_th [s/km],
 *  u_x, u_y, u_z [v/v_th], a tau_NL).  n_floats must be 8 * n_cells. */
int colt_read_cells(colt_ctx* ctx, colt_grid grid, float* out, size_t n_floats);
/* Diffuse emission (Sec. 3.1.1: recombination and collisional excitation in the
 * gas; the collisional emissivity of Sec. 5.3): lum[n_cells] is each cell's luminosity (FP64,
 * any unit; finite, >= 0, not all zero) in host or device memory per mem.  A
 * packet of a COLT_SOURCE_CELLS run starts in cell c with probability
 * w_c / sum(w), where w_c = floor(2^s lum_c / max(lum)) and
 * s = 63 - ceil(log2(n_cells + 1)) (so the weights sum below 2^63 and a cell
 * below 2^-s of the brightest does not emit), at a uniform position inside it
 * and an isotropic direction.  The cell is chosen exactly: t = floor(r w_tot
 * 2^-64) from a 64-bit Philox word r, then the first c whose inclusive prefix
 * sum of w exceeds t.  The library keeps the prefix sums on the device
 * (8 bytes per cell, plus 12 per leaf of an octree); a second call replaces
 * the first.  COLT_EINVAL for bad values, COLT_ENOMEM over the budget. */
int colt_set_cell_luminosity(colt_ctx* ctx, colt_grid grid, const double* lum, int mem);

/* ------------------------------------------------------------------ runs -- */
/* A distant observer along a coordinate axis (Sec. 6.1: six axis cameras).
 * dir must be +-e_x, +-e_y or +-e_z.  The image axes of a camera along +-e_a
 * are (+-e_{a+1}, e_{a+2}) (indices mod 3); npix = 0 gives a spectrum only. */
typedef struct {
  double dir[3];
  int npix;
} colt_camera;

/* One of several point sources of a solve (colt_run_params.sources). */
typedef struct {
  double pos[3];            /* position (cm)                                          */
  double sigma;             /* Gaussian spread (cm), 0 = point                        */
  double weight;            /* relative luminosity, >= 0 (not all 0)                  */
} colt_source;

typedef struct {
  uint64_t n_packets;
  uint64_t seed;            /* Philox key; results depend only on (seed, packet id) */
  double src_pos[3];        /* point source position (cm), when n_sources = 0         */
  double src_sigma;         /* Gaussian spread of the source (cm), 0 = point          */
  int core_skip;            /* COLT_SKIP_* (Sec. 3.2.4); any other nonzero value is
                               rejected                                             */
  int recoil;               /* Eq. recoil                                             */
  int phase;                /* COLT_PHASE_DIPOLE (Eq. phaseW) or _ISOTROPIC           */
  double tau_esc_max;       /* peel-off cutoff, 50 in Sec. 6.1                        */
  double albedo;            /* dust albedo A                                          */
  uint64_t max_scatter;     /* per-packet cap on scatterings (0 = none)               */
  /* angle-averaged escape spectrum: bins [lo, hi) in spec_units */
  int spec_units;           /* COLT_UNITS_X (x at T_ref) or COLT_UNITS_DV_KMS         */
  double T_ref;
  double spec_lo, spec_hi;
  int spec_nbins;
  /* peel-off cameras */
  int n_cam;
  const colt_camera* cams;  /* host array of n_cam                                    */
  int cam_units;
  double cam_lo, cam_hi;
  int cam_nbins;
  double fov_half;          /* image half-width (cm) about the box centre; 0 = box    */
  int precision;            /* COLT_PLAIN (FP64 arithmetic) or COLT_MIXED             */
  int block_size;           /* 0 = library default (autotuned)                        */
  int blocks_per_sm;        /* 0 = library default                                    */
  uint64_t pid_offset;      /* packets are ids pid_offset .. pid_offset + n_packets-1
                               (random streams are keyed by id, so a job split into
                               id ranges -- batches, replicas -- sums to the same
                               tallies); per-packet outputs are indexed from 0      */
  int emission;             /* COLT_EMIT_LINE_CENTRE: x = 0 in the source cell's frame;
                               COLT_EMIT_NATURAL_THERMAL: x = x_nat + k.u_atom with a
                               Lorentzian x_nat (width a) and a Maxwellian atom velocity
                               of the source cell (Sec. 3.1.1)                      */
  int source;               /* COLT_SOURCE_POINT (src_pos, src_sigma, or sources) or
                               COLT_SOURCE_CELLS (the grid's cell luminosities;
                               src_pos, src_sigma and sources unused)               */
  int n_sources;            /* 0: the one source src_pos / src_sigma; 1..16: each
                               packet starts at sources[s] (plus its Gaussian spread)
                               with probability weight_s / sum of weights, drawn
                               exactly from integer weights floor(2^(63-b) w_s /
                               max w), b the least integer with 2^b >= n_sources + 1,
                               by the 64-bit word of its emission's Philox block 4   */
  const colt_source* sources; /* host array of n_sources (copied by the call)         */
} colt_run_params;

/* Outputs of a run.  Counters are always filled; every array pointer may be
 * NULL (not wanted).  Arrays are HOST memory of the stated lengths:
 *   spec       [spec_nbins]                       escaped packets per bin
 *   cam_spec   [n_cam * cam_nbins]                sum of W exp(-tau_esc) (Eq. SB)
 *   cam_spec2  [n_cam * cam_nbins]                sum of squared weights
 *   cam_image  [sum_c npix_c^2 * cam_nbins]       per camera [v][u][bin]
 *   pk_status  [n_packets] 1 escaped, 2 absorbed, 3 capped
 *   pk_nscat   [n_packets] executed scatterings of each packet
 *   pk_freq    [n_packets] escape frequency (spec_units) of escaped packets;
 *                          for packets stopped by max_scatter, the lab-frame
 *                          frequency at that moment; 0 otherwise */
typedef struct {
  uint64_t n_emitted, n_escaped, n_absorbed, n_capped;
  uint64_t n_scat, n_scat_hi;
  uint64_t n_cell_visits, n_peel_visits, n_peel_rays;
  uint64_t spec_under, spec_over;
  double kernel_ms;         /* device time of the transport kernel (CUDA events) */
  uint64_t* spec;
  double* cam_spec;
  double* cam_spec2;
  double* cam_image;
  int32_t* pk_status;
  uint64_t* pk_nscat;
  double* pk_freq;
} colt_result;

/* Blocking solve: all packets of p on grid.  Results as above.
 * COLT_EDEVICE if the kernel's bounds checks fired (results then invalid). */
int colt_run(colt_ctx* ctx, colt_grid grid, const colt_run_params* p, colt_result* out);

/* Blocking batched solve: n (1..256) independent solves -- each with its own
 * grid, parameters and results (arrays of n) -- share one persistent launch,
 * so short and long solves fill the GPU together.  params[i].precision and
 * the grid kind (Cartesian / octree) must be equal for all i (COLT_EINVAL).
 * The launch starts the solves whose grids have shown the longest histories
 * first.  out[i].kernel_ms is the shared launch's time. */
int colt_run_batch(colt_ctx* ctx, int n, const colt_grid* grids, const colt_run_params* params,
                   colt_result* out);

/* ------------------------------------------------------------ autotune -- */
/* Launch configuration of the persistent transport kernel:
 *   variant         register variant (0: the compiler's allocation; 1 / 2:
 *                   registers capped so that four / three 256-thread CTAs fit
 *                   on an SM, FP32 only)
 *   blocks_per_sm   resident CTAs per SM (0 = as many as fit)
 *   warps_per_block 8 (4 and 16 also exist for the FP32 variant 0; 0 = 8)
 *   refill_min      a warp takes new packets once this many of its 32 lanes
 *                   are idle, or when all are (1 = every round; 0 = 1)
 * Each lane carries one packet (32 packets per warp).  The library default is
 * {0, 0, 0, 8, 1}.  Results never depend on the configuration (packets are
 * keyed by id), up to the summation order of the peel-off tallies. */
typedef struct {
  int variant;
  int blocks_per_sm;
  double scatterings_per_s;  /* measured by colt_autotune */
  int warps_per_block;
  int refill_min;
} colt_launch_config;

/* Tune the launch configuration on the solve (grid, *params) -- at most 2^20
 * packets, no images, the same packet ids each time -- by a coordinate search:
 * every register variant x resident CTAs per SM, then warps per CTA, then the
 * refill threshold (1, 4, 12), one solve per configuration.  The fastest is
 * kept for params->precision and the grid's kind (every later launch of that
 * pair with blocks_per_sm = 0 uses it, served launches included) and reported
 * in *out (may be NULL).  Blocking; ten solves for FP32, four for FP64. */
int colt_autotune(colt_ctx* ctx, colt_grid grid, const colt_run_params* params, colt_launch_config* out);

/* Set the launch configuration used for `precision` (COLT_PLAIN / COLT_MIXED)
 * and grid kind `kind` (COLT_CARTESIAN / COLT_OCTREE) without tuning;
 * COLT_EINVAL for a variant, block size or refill threshold (1..32) the build
 * does not offer.  blocks_per_sm = 0 means as many CTAs as fit. */
int colt_set_launch_config(colt_ctx* ctx, int precision, int kind, const colt_launch_config* cfg);

/* Same solve with HOST input fields: builds a temporary grid from desc, runs,
 * copies results back and frees the grid (one call for an end-to-end user). */
int colt_solve(colt_ctx* ctx, const colt_grid_desc* desc, const colt_run_params* p, colt_result* out);

/* ------------------------------------------------------------- serving -- */
/* Continuous batching.  colt_submit enqueues a solve (non-blocking); requests
 * are admitted as memory (mem_budget_bytes) allows, and the packets of all
 * admitted requests share persistent launches (up to six in flight, each of
 * at most 256 requests and 2^20 packets, one precision and one grid kind;
 * longest expected histories first, a request passed over four times first).
 * A request is done as soon as all its own packets have finished, whatever
 * else its launches still run.  Returns COLT_EAGAIN when the request cannot
 * be queued now (queue full).  The grid must stay alive until the request is
 * released.  Results of a request are identical to colt_run of the same
 * (grid, params) up to floating-point summation order of the peel-off
 * tallies. */
typedef struct {
  int done;                 /* 1 when all packets are finished                   */
  int admitted;
  uint64_t packets_done, packets_total;
  double submit_to_done_ms; /* latency, valid when done                          */
  uint64_t ctx_launches;    /* transport kernel launches this context has issued */
  int cancelled;            /* 1 after colt_cancel: the tallies cover packets_done
                               packets (those that had started), not packets_total */
  uint64_t ctx_timed_launches; /* finished transport launches of this context ...     */
  double ctx_kernel_ms;     /* ... and their summed device time (CUDA events around
                               each kernel on its own stream)                      */
  uint64_t longest_history; /* most scatterings of one packet of the request, over
                               the launches of it that have ended (a request can be
                               done before its last launch ends)                   */
  uint64_t ctx_cell_visits; /* flight cell visits and peel-off cell visits of the  */
  uint64_t ctx_peel_visits; /* context's finished, timed launches                  */
} colt_stats;

int colt_submit(colt_ctx* ctx, colt_grid grid, const colt_run_params* p, colt_req* out);
/* Submit n requests at once (grids[i], params[i]) -> out[i] (the serving API
 * has no counterpart in the paper).  Every request is checked first and none
 * is queued if one fails (the error of the first that fails); then all are
 * queued in order and the scheduler takes one step, so a batch fills shared
 * launches together instead of the first ones each taking a launch slot of
 * their own (colt_submit schedules after every request).  Admission,
 * completion and results are those of colt_submit of the same requests in the
 * same order.  COLT_EAGAIN when the queue cannot hold all n. */
int colt_submit_many(colt_ctx* ctx, int n, const colt_grid* grids, const colt_run_params* params,
                     colt_req* out);
/* Drives the scheduler one step (collects finished launches, admits queued
 * requests, refills free launch slots) and reports the request's state;
 * never blocks on the device.  The scheduler advances only inside colt_submit,
 * colt_poll and colt_wait. */
int colt_poll(colt_ctx* ctx, colt_req req, int* done, colt_stats* st);
/* Block until req is done or timeout_ms (< 0: no limit) elapses
 * (COLT_ETIMEOUT; the request keeps running).  While waiting it sleeps until
 * any in-flight launch finishes and then refills the free slot, so other
 * requests keep the GPU busy; it re-polls every millisecond, so a request
 * whose own packets finish inside a running launch is seen done promptly. */
int colt_wait(colt_ctx* ctx, colt_req req, double timeout_ms);
/* camera = -1: the angle-averaged escape spectrum (as doubles); else the
 * camera's peel-off spectrum.  nbins must match the request's bin count. */
int colt_read_spectrum(colt_ctx* ctx, colt_req req, int camera, double* buf, size_t nbins);
/* The peel-off image cube of camera `camera` (0 <= camera < n_cam, npix > 0),
 * laid out [v][u][bin] (npix x npix x cam_nbins doubles, Sec. 6.1 surface
 * brightness per pixel and bin before unit conversion); n must equal that
 * size (COLT_EINVAL otherwise). */
int colt_read_image(colt_ctx* ctx, colt_req req, int camera, double* buf, size_t n);
int colt_read_result(colt_ctx* ctx, colt_req req, colt_result* out);
/* Stop a request early.  A queued request is dropped at once (done, no
 * tallies: reading its results gives zero counters).  An admitted one hands
 * out no further packets: the packets already in a launch finish (a serving
 * launch carries at most 2^20 packets), then the request is done with the
 * tallies of those packets (colt_stats.cancelled = 1, packets_done < packets_total
 * when it was cut short).  A done request is left as it is.  Never blocks. */
int colt_cancel(colt_ctx* ctx, colt_req req);
/* Free a finished or queued request's results (COLT_EAGAIN while it runs:
 * colt_cancel first, then wait). */
int colt_release(colt_ctx* ctx, colt_req req);

/* --------------------------------------------- solve without allocating -- */
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code that runs under a device-memory
 * budget owned by another allocator, or a library that must not call
 * cudaMalloc on its user's behalf.  It performs the blocking batched solve of
 * colt_run_batch with caller-owned inputs and outputs and calls no
 * cudaMalloc, cudaFree or allocating routine, and needs no context.
 *
 * Inputs: n solves (1 <= n <= 8; larger n returns COLT_EINVAL), each a
 * Cartesian grid given by its geometry and its DEVICE array of packed cell
 * records (8 floats per cell, the layout colt_read_cells returns, including
 * a tau_NL), and its run parameters (host; source must be COLT_SOURCE_POINT,
 * since a grid view has no luminosity table).  Outputs: per solve, DEVICE
 * tallies the caller allocated: spec [spec_nbins] and counters [8] (emitted,
 * escaped, absorbed, capped, scatterings, HI scatterings, underflow,
 * overflow) as unsigned 64-bit, cam_spec / cam_spec2 [n_cam * cam_nbins]
 * (when n_cam > 0) and cam_image (when a camera has npix > 0) as doubles.
 * The call zeroes these outputs, runs, and synchronises cuda_stream (NULL is
 * the legacy default stream) before returning.  Returns COLT_EINVAL for bad
 * sizes or parameters, COLT_ECUDA for a failed CUDA call, COLT_EDEVICE when
 * the kernel's bounds checks fired.
 *
 * The launch header, job table and counters live in one static device array
 * of 16 KB that every GPU loading the library keeps until process exit.  The
 * first call on a device looks up that array's device address with the
 * device current; make that first call before any stream capture.  The
 * address is kept for the life of the process, so do not use this entry
 * point across a device reset (or a release and re-creation of the primary
 * context).  The solves run in the caller's order (colt_run_batch starts the
 * grids with the longest past histories first; this call keeps no such
 * per-grid record).  All calls
 * share the array, which keeps the last call's contents: calls that overlap
 * on the GPU (from several threads or streams) race, so serialise them. */
typedef struct {
  int nx, ny, nz;
  double lo[3], hi[3];
  int periodic_xy;
  const float* records;     /* device, 8 floats per cell */
} colt_grid_view;

typedef struct {
  unsigned long long* spec;
  unsigned long long* counters;
  double* cam_spec;
  double* cam_spec2;
  double* cam_image;
} colt_device_tallies;

int colt_run_noalloc(int n, const colt_grid_view* grids, const colt_run_params* params,
                     const colt_device_tallies* tallies, void* cuda_stream);

/* ------------------------------------------------------ parity helpers -- */
/* App. A1, Eq. AB: H_approx(a, x) for n pairs.  mem says where a, x, H live.
 * precision COLT_MIXED evaluates in FP32 on float arrays; COLT_PLAIN in FP64
 * on double arrays. */
int colt_voigt(colt_ctx* ctx, const void* a, const void* x, void* H, size_t n, int precision, int mem);

/* One resonant scattering per element (Sec. 3.1.3, 3.2.3, 3.2.4), with the
 * transport kernel's own device code and RNG layout:
 * Philox4x32-10 key (seed lo, seed hi), counter (pid lo, pid hi, event, block).
 * Inputs and outputs are in FP64 here; the arithmetic is the precision's. */
typedef struct {
  double x;          /* incoming comoving frequency                            */
  double k[3];       /* incoming direction                                     */
  double a;          /* damping parameter                                      */
  double g;          /* recoil parameter (0 = off)                             */
  double atau0;      /* a tau_0 for x_crit (Eq. xcrit); < 0: core-skipping off */
  int32_t phase;     /* COLT_PHASE_*                                           */
  uint64_t pid;
  uint32_t event;
  double x_f;        /* outputs                                                */
  double k_f[3];
  double u_atom[3];
  double u_par;
  double x_crit;
  double RQ;
  double mu;
  int32_t n_trials;
} colt_scatter_io;

int colt_scatter(colt_ctx* ctx, colt_scatter_io* io, size_t n, uint64_t seed, int precision);

#ifdef __cplusplus
}
#endif
#endif
