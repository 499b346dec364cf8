// Internal structures shared by the library's translation units (not part of
// the public ABI; see include/colt.h for that).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace colt {

constexpr int kMaxCams = 8;
constexpr int kMaxSources = 16;

// Per-cell record, two float4 (32 bytes, one DRAM/L2 sector):
//   r0 = (k_HI = n_HI sigma_0 [1/cm], a, k_dust [1/cm], 1/v_th [s/km])
//   r1 = (u_x, u_y, u_z [v/v_th], a tau_NL)
// Cartesian cells are stored x-fastest; octree leaves in input order.
// Octree (kind 1): leaf i of level L and integer coordinates ijk spans
// lo + ijk h 2^-L .. lo + (ijk + 1) h 2^-L, h = hi - lo (the root size).
//   node[v] >= 0 : v is internal, its 8 children are node[v] + (bx | by<<1 | bz<<2)
//   node[v] <  0 : v is leaf -1 - node[v]
//   nbr[6 i + 2 a + (0: +a face, 1: -a face)] = the node across that face at
//     the leaf's level or the coarser leaf covering it, packed as
//     id | level << 27; when that node is a leaf, id is the leaf's index and
//     bit 26 (kLeafFlag) is set, so a walk needs no node-table load to find
//     it; kNoNbr when the face is on the box boundary.
constexpr uint32_t kNoNbr = 0xFFFFFFFFu;
constexpr uint32_t kLeafFlag = 1u << 26;
constexpr uint32_t kNodeMask = (1u << 26) - 1u;
constexpr int kMaxOctLevel = 24;

// Eq. atau0J, a tau_J = 6.428e4 T_4^(-1/2) (n_HI / cm^-3)^(1/2), in terms of the
// cell record: with a = 4.702e-4 T_4^(-1/2) and k_HI = n_HI 5.898e-14 T_4^(-1/2) cm^-1
// (Sec. 2), a k_HI = 4.702e-4 x 5.898e-14 T_4^-1 n_HI, so a tau_J = C sqrt(a k_HI)
// with C = 6.428e4 / sqrt(4.702e-4 x 5.898e-14) (cm^1/2).
inline double jeans_coefficient() { return 6.428e4 / std::sqrt(4.702e-4 * 5.898e-14); }

struct GridDev {
  const float4* rec = nullptr;
  int kind = 0;
  int n[3] = {0, 0, 0};
  int64_t stride[3] = {1, 0, 0};
  // Cartesian: h = cell size; octree: h = root size (a leaf of level L: h 2^-L)
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, h[3] = {0, 0, 0};
  float hf[3] = {0, 0, 0};             // h in FP32 (fill_f32)
  float halff[3] = {0, 0, 0};          // half the box size in FP32
  int periodic_xy = 0;
  int64_t n_cells = 0;
  // octree (kind == 1)
  const int32_t* node = nullptr;
  const uint32_t* nbr = nullptr;
  int max_level = 0;
  // diffuse emission: inclusive prefix sums of the integer cell weights and
  // their total; octree: per leaf (i | level << 24, j, k)
  const unsigned long long* lum_cum = nullptr;
  unsigned long long lum_total = 0;
  const uint32_t* leaf_loc = nullptr;
};

struct CamDev {
  int axis = 0;      // 0,1,2
  int sgn = 1;       // +1 / -1
  int npix = 0;
  int64_t img_off = 0;
};

struct Tallies {
  unsigned long long* spec = nullptr;       // [spec_nb]
  unsigned long long* counters = nullptr;   // [kNumCounters] (per job)
  double* cam_spec = nullptr;               // [n_cam * cam_nb]
  double* cam_spec2 = nullptr;
  double* cam_image = nullptr;              // optional
  int32_t* pk_status = nullptr;             // optional [n_packets]
  uint64_t* pk_nscat = nullptr;
  double* pk_freq = nullptr;
};

// per-job counters (packet outcomes)
enum Counter {
  kEmitted = 0, kEscaped, kAbsorbed, kCapped, kScat, kScatHI, kUnder, kOver, kNumCounters
};
// per-launch diagnostic counters
enum LaunchCounter { kCellVisits = 0, kPeelVisits, kPeelRays, kNumLaunchCounters };

// FP32 copies of the run parameters that the FP32 path reads per event and
// per peel-off ray: a double -> float conversion issues on the FP64 pipe,
// which GB300 runs at 1/64 of the FP32 rate.
struct RunF {
  float tau_max = 50.f, albedo = 0.f, cam_scale = 1.f, cam_lo = 0.f, cam_hi = 1.f, cam_inv_width = 1.f,
        fov_half = 1.f, pix_scale = 0.5f;
};

struct RunDev {
  uint64_t n_packets = 0;
  uint64_t pid_offset = 0;    // packet ids are pid_offset + [0, n_packets)
  Rng rng{0, 0};
  double src[3] = {0, 0, 0};
  double src_sigma = 0;
  // several point sources: positions, spreads and inclusive prefix sums of
  // the integer weights (n_src = 0: the one source above)
  int n_src = 0;
  double src_pos[kMaxSources][3] = {};
  double src_sig[kMaxSources] = {};
  unsigned long long src_cum[kMaxSources] = {};
  unsigned long long src_total = 0;
  int core_skip = 1, recoil = 1, phase = 0;   // core_skip: COLT_SKIP_*
  int emission = 0;           // 0 line centre, 1 natural + thermal (Sec. 3.1.1)
  int source = 0;             // COLT_SOURCE_POINT / COLT_SOURCE_CELLS
  // a tau_J = jeans_c sqrt(a k_HI) (Eq. atau0J rewritten with a and sigma_0 of
  // the cell record), in FP64 and FP32
  double jeans_c = 0;
  float jeans_cf = 0;
  double tau_max = 50.0;
  double albedo = 0.0;
  uint64_t max_scatter = ~0ull;
  double spec_scale = 1.0;    // spectral coordinate = (lab Doppler velocity [km/s]) * scale
  double spec_lo = 0, spec_hi = 1;
  int spec_nb = 1;
  int n_cam = 0;
  CamDev cam[kMaxCams];
  double cam_scale = 1.0;
  double cam_lo = 0, cam_hi = 1;
  double cam_inv_width = 1.0;  // cam_nb / (cam_hi - cam_lo)
  int cam_nb = 1;
  double fov_half = 1.0;
  double pix_scale = 0.5;      // 1 / (2 fov_half)
  double centre[3] = {0, 0, 0};
  RunF f;
  Tallies t;
};

// Host: refresh the FP32 copies after the double fields are set.
inline void fill_f32(GridDev& g) {
  for (int a = 0; a < 3; ++a) {
    g.hf[a] = (float)g.h[a];
    g.halff[a] = (float)(0.5 * (g.hi[a] - g.lo[a]));
  }
}
inline void fill_f32(RunDev& r) {
  r.f.tau_max = (float)r.tau_max;
  r.f.albedo = (float)r.albedo;
  r.f.cam_scale = (float)r.cam_scale;
  r.f.cam_lo = (float)r.cam_lo;
  r.f.cam_hi = (float)r.cam_hi;
  r.f.cam_inv_width = (float)r.cam_inv_width;
  r.f.fov_half = (float)r.fov_half;
  r.f.pix_scale = (float)r.pix_scale;
}

// A parameter in the transport precision R: the double field in the FP64
// path, its FP32 copy in the FP32 path.
template <typename R>
__device__ __forceinline__ R prm(double d, float f);
template <>
__device__ __forceinline__ float prm<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double prm<double>(double d, float) { return d; }

// One solve inside a launch: its grid, its parameters and its tallies.
struct Job {
  GridDev g;
  RunDev p;
};

// A persistent launch over n_jobs jobs.  Packet slots are numbered 0..total-1
// across jobs; job j owns [job_end[j-1], job_end[j]).
struct LaunchDev {
  const Job* jobs = nullptr;
  const unsigned long long* job_end = nullptr;
  int n_jobs = 0;
  unsigned long long total = 0;
  unsigned long long* next = nullptr;        // work counter
  unsigned long long* counters = nullptr;    // [kNumLaunchCounters]
  int* error = nullptr;                      // device-side error flag
  unsigned long long* job_max = nullptr;     // [n_jobs] longest history (scatterings), or null
  int refill_min = 1;                        // a warp refills once this many lanes wait (or all idle)
  unsigned long long* job_done = nullptr;    // [n_jobs] finished packets, mapped host memory, or null
};

// launchers (transport.cu)
// L is a DEVICE pointer to the launch header (so a captured graph can replay it).
// All jobs of a launch share one grid kind (COLT_CARTESIAN / COLT_OCTREE).
// variant: 0 = the compiler's register allocation, 1 / 2 = registers capped
// for four / three CTAs per SM (FP32 only; transport_variants gives the count);
// blocks_per_sm 0 = as many CTAs as fit.  extras: some job uses diffuse
// emission or the Jeans core-skipping estimate (their kernel instantiation,
// register variant 0).
// warps: warps per CTA, 8 for every variant; the FP32 variant 0 is also built
// with 4 and 16 (transport_has_warps).
cudaError_t launch_transport(const LaunchDev* L, int precision, int kind, int variant, int blocks_per_sm,
                             int sm_count, cudaStream_t s, bool extras, int warps = 8);
// true when a job needs the extras instantiation
inline bool run_needs_extras(const RunDev& r) { return r.source == 1 || r.core_skip == 2; }
int transport_variants(int precision);
bool transport_has_warps(int precision, int variant, int warps);
// resident CTAs per SM of a variant and block size
int transport_occupancy(int precision, int kind, int variant, int warps = 8);
// grid preparation (grid.cu)
cudaError_t launch_atau_nl(const GridDev& g, const float* n_hi, double f_nl, float4* rec_mut, cudaStream_t s);
// octree grids: lev / ijk are the device copies of the leaves' levels and coordinates
cudaError_t launch_atau_nl_oct(const GridDev& g, const float* n_hi, const uint8_t* lev, const uint32_t* ijk,
                               double f_nl, float4* rec_mut, cudaStream_t s);
// parity helpers (parity.cu)
cudaError_t launch_voigt(const void* a, const void* x, void* H, size_t n, int precision, cudaStream_t s);
struct ScatterIODev;
cudaError_t launch_scatter(void* io, size_t n, uint64_t seed, int precision, cudaStream_t s);

}  // namespace colt
