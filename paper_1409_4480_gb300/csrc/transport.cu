// Persistent photon-packet transport kernel (Cartesian and octree grids).
//
// Paper mapping:
//   emission           Sec. 3.1.1 (isotropic k_i, x_i = 0 in the source cell, or
//                      natural + thermal; a point source, or diffuse emission from
//                      cells drawn by luminosity)
//   tau_event = -ln R  Sec. 3.1.2, Eq. lnR
//   cell march         Sec. 3.1.2 (tau_cell = (n sigma_0 H(a,x) + k_dust) l_cell,
//                      x' = (x + k.u) sqrt(T/T') - k.u' at every face)
//   scattering         Sec. 3.1.3 + 3.2.3 + 3.2.4 (device.cuh: scatter_hi); a tau_0
//                      for x_crit from the cell and non-local terms or from the
//                      Jeans estimate (Eq. atau0J)
//   peel-off           Sec. 6.1, Eq. SB (W(theta) exp(-tau_esc), stop at tau_esc > 50)
//
// GB300 design:
//   * One packet per lane; lanes whose packet finished take the next packet
//     slot from a global counter at the top of every round (one warp-aggregated
//     atomic per refill), so warps never idle on short packets.  Slots are
//     numbered across all jobs of the launch (a job = one solve: grid, params,
//     tallies), so one persistent launch runs many heterogeneous requests.
//   * A round advances every live lane by one flight + one interaction; the
//     march is per lane in cell-local coordinates (FP32 in the mixed path), with
//     the remaining optical depth in FP64.
//   * Peel-off rays run along coordinate axes.  Their cell sequence is known in
//     advance and the lab-frame frequency (x + k.u) v_th is invariant along a
//     ray, so the whole warp marches one ray at a time, 32 cells per step
//     (coalesced 32-byte records), with a butterfly sum of the cell optical
//     depths and an early exit once tau_esc exceeds the cutoff.
//   * Tally atomics are staged one per lane and issued 32 at a time.
#include <cstdio>

#include "internal.h"
#include "octree.cuh"

namespace colt {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kMaxFlightVisits = 1u << 24;
// peel-off cells a lane marches on its own (after the event cell) before the
// warp takes the ray over
constexpr int kLanePeel = 3;
// recoil parameter over damping parameter: 2.536e-4 / 4.702e-4 (Sec. 2, Eq. recoil)
constexpr double kGoverA = 2.536e-4 / 4.702e-4;

template <typename R>
struct PeelEv {
  R rel[3];     // event position relative to the box centre (cm), for image pixels
  int64_t cell;
  int ijk[3];
  int lvl;      // octree leaf level (0 on Cartesian grids)
  int job;
  R xi[3];      // position in the event cell (cell units)
  R xt[3];      // 1 - xi, formed from the exact position
  R x;          // comoving frequency at the event (before the scattering)
  R k[3];       // incoming direction (HI scattering)
  R ua[3];      // atom velocity (HI scattering)
  R upar, g, RQ;
  R vth, wn;    // the cell's v_th (km/s) and the phase weight's normaliser 1 / (1 + RQ/3)
  R u[3];
  R kHI, a, kd; // the event cell's opacity record (first cell of every peel-off ray)
  int type;     // 0: isotropic with W = 1 and x unchanged (emission, dust); 1: HI
};

__device__ __forceinline__ int bin_of(double s, double lo, double hi, int nb) {
  if (!(s >= lo) || !(s < hi)) return -1;
  int b = (int)floor((s - lo) * (double)nb / (hi - lo));
  return (b >= 0 && b < nb) ? b : -1;
}

// bin of a peel-off frequency, in the transport precision
template <typename R>
__device__ __forceinline__ int bin_of_r(R s, R lo, R hi, R inv_width, int nb) {
  if (!(s >= lo) || !(s < hi)) return -1;
  const int b = (int)floor((s - lo) * inv_width);
  return (b >= 0 && b < nb) ? b : -1;
}

// Remaining optical depth of a flight (Sec. 3.1.2: tau_event = -ln R, less
// the depth of every cell crossed).  The FP64 path keeps it in FP64.  The FP32
// path keeps it as an unevaluated float pair hi + lo, updated with Knuth's
// two-sum, so that many small cell depths subtract with ~48-bit accuracy on
// the FP32 pipe (GB300's FP64 pipe issues 1/64 of the FP32 rate).
template <typename R>
struct TauLeft {
  double v;
  __device__ __forceinline__ void set(R t) { v = (double)t; }
  __device__ __forceinline__ R value() const { return R(v); }
  // true (state kept) when the remaining depth is at most c; else subtract c
  __device__ __forceinline__ bool reached(R c) {
    if (v <= (double)c) return true;
    v -= (double)c;
    return false;
  }
};

template <>
struct TauLeft<float> {
  float hi, lo;
  __device__ __forceinline__ void set(float t) { hi = t; lo = 0.f; }
  __device__ __forceinline__ float value() const { return hi + lo; }
  __device__ __forceinline__ bool reached(float c) {
    const float s = __fsub_rn(hi, c);          // two-sum: s + e == hi - c exactly
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(-c, bb));
    const float t = __fadd_rn(e, lo);
    if (__fadd_rn(s, t) <= 0.f) return true;
    hi = __fadd_rn(s, t);                      // renormalise (fast two-sum)
    lo = __fsub_rn(t, __fsub_rn(hi, s));
    return false;
  }
};

__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ int64_t cell_index(const GridDev& G, const int c3[3]) {
  return (int64_t)c3[0] + G.stride[1] * c3[1] + G.stride[2] * c3[2];
}

// Diffuse emission (Sec. 3.1.1): the cell is the first whose inclusive prefix
// weight exceeds t = floor(r w_tot 2^-64), r the 64-bit word of event-0 block 1;
// the position is uniform in the cell (event-0 block 3, words 0-2).  Runs once
// per packet: kept out of line so that the transport loop's code stays compact.
struct EmitCell {
  int64_t cell;
  int ci[3];
  int lvl;
  double f[3];
};

__device__ __noinline__ EmitCell pick_emission_cell(const GridDev& G, const Rng& rng, uint64_t rpid) {
  EmitCell out;
  const u4 q1 = rng.block(rpid, 0, 1);
  const unsigned long long t = __umul64hi(((unsigned long long)q1.y << 32) | q1.x, G.lum_total);
  int64_t lo = 0, hi = G.n_cells - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(G.lum_cum + mid) > t) hi = mid; else lo = mid + 1;
  }
  out.cell = lo;
  if (G.kind == 1) {
    const uint32_t w0 = __ldg(G.leaf_loc + 3 * lo);
    out.lvl = (int)(w0 >> 24);
    out.ci[0] = (int)(w0 & 0xFFFFFFu);
    out.ci[1] = (int)__ldg(G.leaf_loc + 3 * lo + 1);
    out.ci[2] = (int)__ldg(G.leaf_loc + 3 * lo + 2);
  } else {
    const int64_t nxy = (int64_t)G.n[0] * G.n[1];
    out.lvl = 0;
    out.ci[2] = (int)(lo / nxy);
    out.ci[1] = (int)((lo - out.ci[2] * nxy) / G.n[0]);
    out.ci[0] = (int)(lo - out.ci[2] * nxy - (int64_t)out.ci[1] * G.n[0]);
  }
  const U4<double> q3 = uniforms<double>(rng, rpid, 0, 3);
  out.f[0] = q3.v[0];
  out.f[1] = q3.v[1];
  out.f[2] = q3.v[2];
  return out;
}

// kMinBlocks: resident CTAs per SM the register allocation must allow (1: the
// compiler's choice; 3: at most 85 registers; 4: at most 64)
// kX: the instantiation that also holds diffuse emission and the Jeans
// core-skipping estimate (launched only when a job of the launch uses them;
// the common instantiation leaves their code out of the loop entirely).
template <typename R, int kWarps, bool kOct, int kMinBlocks, bool kX>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
k_transport(const LaunchDev* __restrict__ Lp) {
  const LaunchDev L = *Lp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PeelEv<R>* sev = reinterpret_cast<PeelEv<R>*>(smem_raw) + (threadIdx.x >> 5) * 32;
  // lanes of the warp's events in ballot order (peel-off pair -> event)
  int* sidx = reinterpret_cast<int*>(smem_raw + sizeof(PeelEv<R>) * 32 * kWarps) + (threadIdx.x >> 5) * 32;
  // per lane: the damping parameter of the last resonant scattering and its
  // x_cw (Eq. xcw depends on the cell temperature only; a packet scatters
  // many times in one cell)
  R* sxcw = reinterpret_cast<R*>(smem_raw + (sizeof(PeelEv<R>) + sizeof(int)) * 32 * kWarps) + 2 * threadIdx.x;
  sxcw[0] = R(-1);
  const int lane = threadIdx.x & 31;

  unsigned long long lc[kNumLaunchCounters] = {0, 0, 0};

  // lane packet state
  bool alive = false, done = false;
  bool pend_done = false;   // the lane's packet finished this round: count it once its tallies are out
  int pend_job = 0;
  int jb = 0;
  const Job* J = L.jobs;
  uint64_t pid = 0;
  uint32_t event = 0, nscat = 0, nscat_hi = 0;
  int ci[3] = {0, 0, 0};
  int lvl = 0;            // octree leaf level
  int64_t leaf = 0;       // octree leaf index
  CellPos<R> xi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) xi[a].set(R(0));
  R k[3] = {0, 0, 1};
  R x = 0;
  TauLeft<R> tau;
  tau.set(R(0));

  // one peel-off contribution W exp(-tau_esc) into the camera spectrum (and
  // its square) and, inside the field of view, the image cube (Eq. SB)
  auto peel_tally = [&](const RunDev& P, const PeelEv<R>& e, int cam, int ax, int s, int bin, R wr) {
    const int64_t si = (int64_t)cam * P.cam_nb + bin;
    const double w = (double)wr;
    atomicAdd(P.t.cam_spec + si, w);
    atomicAdd(P.t.cam_spec2 + si, (double)(wr * wr));
    const int np = P.cam[cam].npix;
    if (np > 0 && P.t.cam_image) {
      const int au = (ax + 1) % 3, av = (ax + 2) % 3;
      const R pix = prm<R>(P.pix_scale, P.f.pix_scale) * R(np);         // pixels per cm
      const R fu = (R(s) * e.rel[au] + prm<R>(P.fov_half, P.f.fov_half)) * pix;
      const R fv = (e.rel[av] + prm<R>(P.fov_half, P.f.fov_half)) * pix;
      if (fu >= R(0) && fu < R(np) && fv >= R(0) && fv < R(np)) {
        const int64_t iu = (int64_t)floor(fu), iv = (int64_t)floor(fv);
        atomicAdd(P.t.cam_image + P.cam[cam].img_off + (iv * np + iu) * P.cam_nb + bin, w);
      }
    }
  };

  auto finish = [&](int status, double sfreq) {
    const RunDev& P = J->p;
    unsigned long long* C = P.t.counters;
    atomicAdd(C + kEmitted, 1ull);
    if (status == 1) {
      atomicAdd(C + kEscaped, 1ull);
      const int b = bin_of(sfreq, P.spec_lo, P.spec_hi, P.spec_nb);
      if (b >= 0) atomicAdd(P.t.spec + b, 1ull);
      else if (sfreq < P.spec_lo) atomicAdd(C + kUnder, 1ull);
      else atomicAdd(C + kOver, 1ull);
    } else if (status == 2) {
      atomicAdd(C + kAbsorbed, 1ull);
    } else {
      atomicAdd(C + kCapped, 1ull);
    }
    if (nscat) atomicAdd(C + kScat, (unsigned long long)nscat);
    if (L.job_max && nscat) atomicMax(L.job_max + jb, (unsigned long long)nscat);
    if (nscat_hi) atomicAdd(C + kScatHI, (unsigned long long)nscat_hi);
    if (P.t.pk_status) {
      P.t.pk_status[pid] = status;
      P.t.pk_nscat[pid] = nscat;
      P.t.pk_freq[pid] = sfreq;   // escape frequency; at the cap for max_scatter caps; else 0
    }
    pend_done = true;
    pend_job = jb;
    alive = false;
  };

  auto fill_event = [&](int type, const R* kin, const R* ua, R upar, R g, R RQ, R xin, const float4& r0,
                        const float4& r1) {
    const GridDev& G = J->g;
    PeelEv<R>& e = sev[lane];
    e.type = type;
    e.job = jb;
    const R lsc = kOct ? pow2neg<R>(lvl) : R(1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      e.ijk[a] = ci[a];
      e.xi[a] = xi[a].val();
      e.xt[a] = xi[a].from_top();
      e.rel[a] = (R(ci[a]) + e.xi[a]) * (prm<R>(G.h[a], G.hf[a]) * lsc) - prm<R>(0.5 * (G.hi[a] - G.lo[a]), G.halff[a]);
      e.k[a] = kin ? kin[a] : R(0);
      e.ua[a] = ua ? ua[a] : R(0);
    }
    e.lvl = lvl;
    e.cell = kOct ? leaf : cell_index(G, ci);
    e.x = xin;
    e.upar = upar;
    e.g = g;
    e.RQ = RQ;
    e.vth = m_div(R(1), R(r0.w));
    e.wn = m_div(R(1), R(1) + RQ * R(1.0 / 3.0));
    e.u[0] = r1.x; e.u[1] = r1.y; e.u[2] = r1.z;
    e.kHI = r0.x;
    e.a = r0.y;
    e.kd = r0.z;
  };

  // Next-event estimator cut (Sec. 6.1): a ray whose optical depth exceeds
  // tau_esc_max adds nothing.  Every axis ray starts in the event's own cell;
  // H(a, x) decreases with |x|, so (k_HI H(a, max_c |x_c|) + k_d) l_min bounds
  // each ray's first-cell depth from below (x_c: the frequency the event sends
  // towards camera c, over all six axis directions; l_min: the distance to the
  // nearest face).  When the bound exceeds twice the cutoff (a margin far above
  // H_approx's departures from monotonicity) no ray can contribute and the
  // event is not peeled off; otherwise every ray is traced as usual.
  auto peel_open = [&](int type, const R* kin, const R* ua, R upar, R g, R xin, const float4& rr0,
                       const R hc[3]) -> bool {
    const RunDev& P = J->p;
    R xmax = fabs(xin);
    if (type == 1) {
      xmax = R(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const R base = xin - upar - g;
        xmax = fmax(xmax, fabs(base + ua[q] + g * kin[q]));
        xmax = fmax(xmax, fabs(base - ua[q] - g * kin[q]));
      }
    }
    R lmin = R(3.0e38);
#pragma unroll
    for (int q = 0; q < 3; ++q) lmin = fmin(lmin, fmin(xi[q].val(), xi[q].from_top()) * hc[q]);
    lmin = fmax(lmin, R(0));
    const R tau_lb = (R(rr0.x) * voigt<R>(R(rr0.y), xmax) + R(rr0.z)) * lmin;
    return !(tau_lb > R(2) * prm<R>(P.tau_max, P.f.tau_max));
  };

#ifdef COLT_PHASE_CLOCKS
  // opt-in profiling build: SM cycles per phase of a round, printed per warp
  // (the lane maximum of each phase, exact for a warp with one live packet):
  // 0 refill, 1 rest of the interaction, 2 peel-off, 3 rounds, 4 flight,
  // 5 the event's draws, 6 the resonant scattering
  unsigned long long ph[7] = {0, 0, 0, 0, 0, 0, 0};
  long long t_mark = clock64();
#define COLT_PHASE(i)                                  \
  do {                                                 \
    __syncwarp();                                      \
    const long long t_now = clock64();                 \
    ph[i] += (unsigned long long)(t_now - t_mark);     \
    t_mark = t_now;                                    \
  } while (0)
#define COLT_MARK(i)                                   \
  do {                                                 \
    const long long t_now = clock64();                 \
    ph[i] += (unsigned long long)(t_now - t_mark);     \
    t_mark = t_now;                                    \
  } while (0)
#else
#define COLT_PHASE(i) \
  do {                \
  } while (0)
#define COLT_MARK(i) \
  do {               \
  } while (0)
#endif

  for (;;) {
    bool has_peel = false;
    // ---------------------------------------------------------- refill --
    // lanes without a packet take new ones when at least refill_min of them
    // wait (one atomic serves them all), or when the whole warp is idle
    const unsigned want = __ballot_sync(kFull, !alive && !done);
    const unsigned need = (want && (__popc(want) >= L.refill_min || __ballot_sync(kFull, alive) == 0u)) ? want : 0u;
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(L.next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (!alive && !done) {
        const unsigned long long slot = base + __popc(need & ((1u << lane) - 1u));
        if (slot < L.total) {
          // job owning this slot
          int lo = 0, hi = L.n_jobs - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (slot < L.job_end[mid]) hi = mid; else lo = mid + 1;
          }
          jb = lo;
          J = L.jobs + jb;
          const GridDev& G = J->g;
          const RunDev& P = J->p;
          // ---------------------------------------- emission, event 0 --
          pid = slot - (jb ? L.job_end[jb - 1] : 0ull);
          event = 0;
          nscat = 0;
          nscat_hi = 0;
          const uint64_t rpid = pid + P.pid_offset;
          U4<R> b0 = uniforms<R>(P.rng, rpid, 0, 0);
          const R mu = R(2) * b0.v[0] - R(1);
          R sp, cp;
          m_sincospi(R(2) * b0.v[1], &sp, &cp);
          const R st = m_sqrt(fmax(R(0), R(1) - mu * mu));
          k[0] = st * cp; k[1] = st * sp; k[2] = mu;
          tau.set(-m_log(b0.v[2]));
          bool inside = true;
          if (kX && P.source == 1) {
            const EmitCell ec = pick_emission_cell(G, P.rng, rpid);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              ci[a] = ec.ci[a];
              xi[a].set_d(ec.f[a]);
            }
            if constexpr (kOct) {
              lvl = ec.lvl;
              leaf = ec.cell;
            }
          } else {
            double r[3] = {P.src[0], P.src[1], P.src[2]};
            double sig = P.src_sigma;
            if (P.n_src > 0) {
              // several sources: the first whose inclusive prefix weight exceeds
              // t = floor(word W / 2^64), word the 64 bits of event-0 block 4
              const u4 q4 = P.rng.block(rpid, 0, 4);
              const unsigned long long t = __umul64hi(((unsigned long long)q4.y << 32) | q4.x, P.src_total);
              int si = 0;
              while (si < P.n_src - 1 && !(P.src_cum[si] > t)) ++si;
              r[0] = P.src_pos[si][0];
              r[1] = P.src_pos[si][1];
              r[2] = P.src_pos[si][2];
              sig = P.src_sig[si];
            }
            if (sig > 0.0) {
              U4<double> b1 = uniforms<double>(P.rng, rpid, 0, 1);
              const double rho1 = sqrt(-2.0 * log(b1.v[0])), rho2 = sqrt(-2.0 * log(b1.v[2]));
              double s1, c1, s2, c2;
              sincospi(2.0 * b1.v[1], &s1, &c1);
              sincospi(2.0 * b1.v[3], &s2, &c2);
              r[0] += sig * rho1 * c1;
              r[1] += sig * rho1 * s1;
              r[2] += sig * rho2 * c2;
            }
            if constexpr (kOct) {
              // descend from the root, split planes lo + (2i + 1) h 2^-d
  #pragma unroll
              for (int a = 0; a < 3; ++a) {
                if (!(r[a] >= G.lo[a] && r[a] <= G.hi[a]) || (r[a] == G.lo[a] && k[a] < R(0)) ||
                    (r[a] == G.hi[a] && !(k[a] < R(0))))
                  inside = false;
                ci[a] = 0;
              }
              lvl = 0;
              if (inside) {
                int32_t ch;
                uint32_t v = 0;
                while ((ch = __ldg(G.node + v)) >= 0 && lvl < kMaxOctLevel) {
                  ++lvl;
                  int cidx = 0;
  #pragma unroll
                  for (int a = 0; a < 3; ++a) {
                    // rounded product, then rounded sum (no fused multiply-add):
                    // the same number as the leaf faces lying in this plane
                    const double mid =
                        __dadd_rn(G.lo[a], __dmul_rn((double)(2 * ci[a] + 1), G.h[a] * pow2neg<double>(lvl)));
                    const int up = (r[a] > mid) || (r[a] == mid && !(k[a] < R(0)));
                    ci[a] = 2 * ci[a] + up;
                    cidx |= up << a;
                  }
                  v = (uint32_t)ch + (uint32_t)cidx;
                }
                leaf = -1 - (int64_t)__ldg(G.node + v);
                if (leaf < 0 || leaf >= G.n_cells) { atomicExch(L.error, 1); inside = false; leaf = 0; }
  #pragma unroll
                for (int a = 0; a < 3; ++a) {
                  const double hl = G.h[a] * pow2neg<double>(lvl);
                  xi[a].set_d((r[a] - __dadd_rn(G.lo[a], __dmul_rn((double)ci[a], hl))) / hl);
                }
              }
            } else {
  #pragma unroll
              for (int a = 0; a < 3; ++a) {
                const double t = (r[a] - G.lo[a]) / G.h[a];
                const double f = floor(t);
                int i = 0;
                double loc = 0.0;
                const bool in_range = f >= -1.0 && f <= (double)G.n[a];
                if (in_range) {
                  i = (int)f;
                  loc = t - f;
                  if (t == f && k[a] < R(0)) { i -= 1; loc = 1.0; }
                }
                if (!in_range || i < 0 || i >= G.n[a]) { inside = false; i = 0; }
                ci[a] = i;
                xi[a].set_d(loc);
              }
            }
          }
          x = R(0);
          alive = true;
          if (!inside) {
            finish(1, 0.0);     // source outside the box: leaves at line centre
          } else {
            const int64_t c = kOct ? leaf : cell_index(G, ci);
            const float4 e0 = __ldg(G.rec + 2 * c);
            R ua[3] = {R(0), R(0), R(0)};
            R upar = R(0);
            if (P.emission == 1) {
              // Sec. 3.1.1: x = x_nat + k.u_atom, x_nat Lorentzian of width a (block
              // 0 word 3), u_atom Maxwellian, variance 1/2 per component (block 2,
              // Box-Muller pairs); the peel-off sends x_nat + k_c.u_atom, W = 1
              const U4<R> b2 = uniforms<R>(P.rng, rpid, 0, 2);
              R s1, c1, s2, c2, sl, cl;
              m_sincospi(R(2) * b2.v[1], &s1, &c1);
              m_sincospi(R(2) * b2.v[3], &s2, &c2);
              m_sincospi(b0.v[3] - R(0.5), &sl, &cl);
              const R rho1 = m_sqrt(-m_log(b2.v[0])), rho2 = m_sqrt(-m_log(b2.v[2]));
              ua[0] = rho1 * c1;
              ua[1] = rho1 * s1;
              ua[2] = rho2 * c2;
              upar = k[0] * ua[0] + k[1] * ua[1] + k[2] * ua[2];
              x = R(e0.y) * m_div(sl, cl) + upar;
            }
            if (P.n_cam > 0) {
              R hc[3];
#pragma unroll
              for (int a = 0; a < 3; ++a) hc[a] = prm<R>(G.h[a], G.hf[a]) * (kOct ? pow2neg<R>(lvl) : R(1));
              const int ty = P.emission == 1 ? 1 : 0;
              if (peel_open(ty, k, ua, upar, R(0), x, e0, hc)) {
                fill_event(ty, ty ? k : nullptr, ty ? ua : nullptr, upar, R(0), R(0), x, e0, __ldg(G.rec + 2 * c + 1));
                has_peel = true;
              }
            }
          }
        } else {
          done = true;
        }
      }
    }
    if (__all_sync(kFull, done)) break;
    COLT_PHASE(0);

    // ------------------------------------------------ flight + interaction --
    // (a packet emitted this round makes its first flight next round)
    if (alive && !(need & (1u << lane))) {
      const GridDev& G = J->g;
      const RunDev& P = J->p;
      const float4* __restrict__ rec = G.rec;
      const uint64_t rpid = pid + P.pid_offset;
      // per flight: cell size, inverse direction, direction in cell units
      // (octree: of a root-sized cell, scaled by 2^-level at each crossing)
      R hh[3], ik[3], kh[3], h0[3], kh0[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h0[a] = prm<R>(G.h[a], G.hf[a]);
        ik[a] = k[a] != R(0) ? m_div(R(1), k[a]) : R(0);
        kh0[a] = m_div(k[a], h0[a]);
        hh[a] = h0[a];
        kh[a] = kh0[a];
      }
      if constexpr (kOct) {
        const R sc = pow2neg<R>(lvl);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          hh[a] = h0[a] * sc;
          kh[a] = kh0[a] * pow2neg<R>(-lvl);   // exact: 1 / sc
        }
      }
      int64_t c = kOct ? leaf : cell_index(G, ci);
      float4 r0 = __ldg(rec + 2 * c), r1 = __ldg(rec + 2 * c + 1);
      R ktot = 0;
      bool interact = false, escaped = false;
      int status = 0;
      uint32_t visits = 0;
      for (;;) {
        if (++visits > kMaxFlightVisits) { status = 3; break; }
        // distance to the exit face (cm): geometry only, so it comes first
        R tmin = R(3.0e38);
        int ax = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (k[a] != R(0)) {
            R d = (k[a] > R(0) ? xi[a].from_top() : -xi[a].val()) * hh[a] * ik[a];
            if (d < R(0)) d = R(0);
            if (d < tmin) { tmin = d; ax = a; }
          }
        }
        // octree: the exit face's neighbour entry, in flight during the Voigt
        // evaluation (unused when the packet interacts in this leaf)
        const uint32_t nbf = kOct ? oct_face_entry(G, c, ax, k[ax] > R(0) ? 1 : -1) : 0u;
        const R H = voigt<R>(R(r0.y), x);
        ktot = R(r0.x) * H + R(r0.z);
        if (tau.reached(ktot * tmin)) {
          const R le = m_div(tau.value(), ktot);
#pragma unroll
          for (int a = 0; a < 3; ++a) xi[a].add(le * kh[a]);
          interact = true;
          break;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) if (a != ax) xi[a].add(tmin * kh[a]);
        // cross the face on axis ax
        const int sgn = k[ax] > R(0) ? 1 : -1;
        if constexpr (kOct) {
          xi[ax].set(sgn > 0 ? R(1) : R(0));
          const int lvl_old = lvl;
          const int64_t nl = oct_cross_entry<R>(G, nbf, ax, sgn, k, ci, &lvl, xi);
          if (nl < 0) {
            escaped = true;
            break;
          }
          leaf = nl;
          if (lvl != lvl_old) {
            const R sc = pow2neg<R>(lvl);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              hh[a] = h0[a] * sc;
              kh[a] = kh0[a] * pow2neg<R>(-lvl);   // exact: 1 / sc
            }
          }
        } else {
          int ni = ci[ax] + sgn;
          xi[ax].set(sgn > 0 ? R(0) : R(1));
          if (ni < 0 || ni >= G.n[ax]) {
            if (G.periodic_xy && ax < 2) {
              ni = ni < 0 ? G.n[ax] - 1 : 0;
            } else {
              escaped = true;
              break;
            }
          }
          ci[ax] = ni;
        }
        const R ku_old = k[0] * R(r1.x) + k[1] * R(r1.y) + k[2] * R(r1.z);
        const R ivth_old = R(r0.w);
        c = kOct ? leaf : cell_index(G, ci);
        if (c < 0 || c >= G.n_cells) { atomicExch(L.error, 1); status = 3; break; }
        r0 = __ldg(rec + 2 * c);
        r1 = __ldg(rec + 2 * c + 1);
        const R ku_new = k[0] * R(r1.x) + k[1] * R(r1.y) + k[2] * R(r1.z);
        x = (x + ku_old) * m_div(R(r0.w), ivth_old) - ku_new;
      }
      lc[kCellVisits] += visits;
      COLT_MARK(4);
      if (status == 3) {
        finish(3, 0.0);
      } else if (escaped) {
        // lab-frame escape frequency in FP64: Doppler velocity (x + k.u) v_th
        const double ku = (double)k[0] * r1.x + (double)k[1] * r1.y + (double)k[2] * r1.z;
        const double V = ((double)x + ku) / (double)r0.w;
        if (isfinite(V) && isfinite((double)tau.value())) {
          finish(1, V * P.spec_scale);
        } else {
          // only non-finite cell records (device records the host never
          // checked) lead here: raise the device error flag, end as capped
          atomicExch(L.error, 1);
          finish(3, 0.0);
        }
      } else if (interact) {
        ++event;
        // the event's first three draw blocks are independent: compute them
        // together (block 2 is the first u_par trial of a resonant scattering)
        const U4<R> b0 = uniforms<R>(P.rng, rpid, event, 0);
        const U4<R> b1 = uniforms<R>(P.rng, rpid, event, 1);
        const U4<R> b2 = uniforms<R>(P.rng, rpid, event, 2);
        COLT_MARK(5);
        const R a = R(r0.y);
        bool cont = true;
        if (b0.v[0] * ktot < R(r0.z)) {
          // dust: absorb with probability 1 - A, else isotropic scattering
          if (b0.v[1] >= prm<R>(P.albedo, P.f.albedo)) {
            finish(2, 0.0);
            cont = false;
          } else {
            if (P.n_cam > 0 && peel_open(0, nullptr, nullptr, R(0), R(0), x, r0, hh)) {
              fill_event(0, nullptr, nullptr, R(0), R(0), R(0), x, r0, r1);
              has_peel = true;
            }
            const R m = R(2) * b1.v[2] - R(1);
            R sp, cp;
            m_sincospi(R(2) * b1.v[3], &sp, &cp);
            const R sm = m_sqrt(fmax(R(0), R(1) - m * m));
            k[0] = sm * cp; k[1] = sm * sp; k[2] = m;
            ++nscat;
          }
        } else {
          R atau0 = R(-1);
          if (kX && P.core_skip == 2) {
            // Eq. atau0J: the Jeans estimate of the scattering cell
            atau0 = prm<R>(P.jeans_c, P.jeans_cf) * m_sqrt(a * R(r0.x));
          } else if (P.core_skip) {
            R lmin = R(3.0e38);
#pragma unroll
            for (int q = 0; q < 3; ++q) lmin = fmin(lmin, fmin(xi[q].val(), xi[q].from_top()) * hh[q]);
            lmin = fmax(lmin, R(0));
            atau0 = a * R(r0.x) * lmin + R(r1.w);
          }
          const R g = P.recoil ? R(kGoverA) * a : R(0);
          R xcw;
          if (sxcw[0] == a) {
            xcw = sxcw[1];
          } else {
            xcw = x_cw_fit<R>(a);
            sxcw[0] = a;
            sxcw[1] = xcw;
          }
          ScatterOut<R> so = scatter_hi<R>(x, k, a, g, atau0, P.phase, P.rng, rpid, event, b0.v[3], b1, b2, xcw);
          COLT_MARK(6);
          if (so.n_trials > kMaxTrials) {
            finish(3, 0.0);
            cont = false;
          } else {
            ++nscat;
            ++nscat_hi;
            if (P.n_cam > 0 && peel_open(1, k, so.u_atom, so.u_par, g, x, r0, hh)) {
              fill_event(1, k, so.u_atom, so.u_par, g, so.RQ, x, r0, r1);
              has_peel = true;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) k[q] = so.k_f[q];
            x = so.x_f;
          }
        }
        if (cont) {
          if (P.max_scatter && nscat >= P.max_scatter) {
            // capped by the scattering limit: report the lab frequency at the cap
            const double ku = (double)k[0] * r1.x + (double)k[1] * r1.y + (double)k[2] * r1.z;
            finish(3, ((double)x + ku) / (double)r0.w * P.spec_scale);
          } else {
            tau.set(-m_log(b0.v[2]));
          }
        }
      }
    }

    // ------------------------------------------------------------ peel-off --
    // Phase 1 (per lane): the first cell of every camera ray is the event's own
    //   cell, whose record the lane holds, so its optical depth costs no memory
    //   access; a core photon's rays almost always pass tau_esc_max right there.
    // Phase 2 (per lane): up to kLanePeel further cells, one lane per ray.
    // Phase 3 (warp): rays still alive are marched by the whole warp, 32 cells
    //   per step (coalesced records, butterfly sum, exit once tau > cutoff).
    __syncwarp();
    {
      // (event, camera) pairs are spread over the lanes: a full warp gives each
      // lane the rays of one event, a warp with few events (the tail of long
      // histories) marches their rays on many lanes at once
      COLT_PHASE(1);
      const unsigned pm = __ballot_sync(kFull, has_peel);
      if (pm) {   // no event in the warp this round: nothing to peel off
      const int ncl = has_peel ? L.jobs[sev[lane].job].p.n_cam : 0;
      const int ncam_max = (int)__reduce_max_sync(kFull, (unsigned)ncl);
      const int n_pairs = __popc(pm) * ncam_max;
      if (has_peel) sidx[__popc(pm & ((1u << lane) - 1u))] = lane;
      __syncwarp();
      // q / ncam_max for q < 2^20, ncam_max <= 8: (q + 1/2) / n lies >= 1/16 from an integer
      const float inv_nc = n_pairs ? 1.0f / (float)ncam_max : 0.0f;
      for (int pbase = 0; pbase < n_pairs; pbase += 32) {
        const int q = pbase + lane;
        bool act = q < n_pairs;
        int src = __ffs(pm) - 1, cam = 0;
        if (act) {
          const int k = (int)(((float)q + 0.5f) * inv_nc);
          cam = q - k * ncam_max;
          src = sidx[k];
        }
        const PeelEv<R>& e = sev[src];
        const Job* JE = L.jobs + e.job;
        const GridDev& G = JE->g;
        const RunDev& P = JE->p;
        if (act && cam >= P.n_cam) act = false;
        int ax = 0, s = 1, bin = -1, remaining = 0;
        R W = R(1), Vr = R(0);
        R tau_acc = R(0);   // per-ray tau in the transport precision until the warp march
        int64_t cellp = 0, step = 0;
        if (act) {
          ax = P.cam[cam].axis;
          s = P.cam[cam].sgn;
          if (G.periodic_xy && ax < 2) act = false;   // no observer along a periodic axis
        }
        if (act) {
          R xc = e.x;
          if (e.type == 1) {
            const R mu_c = s > 0 ? e.k[ax] : -e.k[ax];
            W = (R(1) + e.RQ * mu_c * mu_c) * e.wn;
            const R kcu = s > 0 ? e.ua[ax] : -e.ua[ax];
            xc = e.x + kcu - e.upar + e.g * (mu_c - R(1));
          }
          const R us = s > 0 ? e.u[ax] : -e.u[ax];
          // lab-frame Doppler velocity (km/s), invariant along the ray
          Vr = (xc + us) * e.vth;
          bin = bin_of_r<R>(Vr * prm<R>(P.cam_scale, P.f.cam_scale), prm<R>(P.cam_lo, P.f.cam_lo), prm<R>(P.cam_hi, P.f.cam_hi), prm<R>(P.cam_inv_width, P.f.cam_inv_width), P.cam_nb);
          if (bin < 0) {
            act = false;
          } else {
            const R hax = prm<R>(G.h[ax], G.hf[ax]) * (kOct ? pow2neg<R>(e.lvl) : R(1));
            const R l0 = (s > 0 ? e.xt[ax] : e.xi[ax]) * hax;
            lc[kPeelRays]++;
            lc[kPeelVisits]++;
            // octree: the event leaf's face entry, loaded before the first
            // cell's Voigt so that the two overlap
            uint32_t nbe = kOct ? oct_face_entry(G, e.cell, ax, s) : 0u;
            tau_acc = (e.kHI * voigt<R>(e.a, xc) + e.kd) * l0;
            if constexpr (kOct) {
              // octree: this lane walks the ray leaf by leaf to the cutoff or
              // the box edge.  The next leaf depends on the last one; each
              // step loads the leaf's record and its next face entry together,
              // so one memory latency (not two) separates the steps.
              const float4* __restrict__ rec = G.rec;
              const R tmax = prm<R>(P.tau_max, P.f.tau_max);
              const R h0ax = prm<R>(G.h[ax], G.hf[ax]);
              R kr[3] = {R(0), R(0), R(0)};
              kr[ax] = R(s);
              int cj[3] = {e.ijk[0], e.ijk[1], e.ijk[2]};
              CellPos<R> xj[3];
#pragma unroll
              for (int a = 0; a < 3; ++a) xj[a].set(e.xi[a]);
              int lv = e.lvl;
              for (uint32_t guard = 0; tau_acc <= tmax && guard < kMaxFlightVisits; ++guard) {
                xj[ax].set(s > 0 ? R(1) : R(0));
                const int64_t nx = oct_cross_entry<R>(G, nbe, ax, s, kr, cj, &lv, xj);
                if (nx < 0) break;
                if (nx >= G.n_cells) { atomicExch(L.error, 1); tau_acc = R(3.0e38); break; }
                nbe = oct_face_entry(G, nx, ax, s);
                const float4 q0 = __ldg(rec + 2 * nx);
                const float uq = __ldg(reinterpret_cast<const float*>(rec + 2 * nx + 1) + ax);
                const R xcell = Vr * R(q0.w) - (s > 0 ? R(uq) : R(-uq));
                tau_acc += (R(q0.x) * voigt<R>(R(q0.y), xcell) + R(q0.z)) * (h0ax * pow2neg<R>(lv));
                lc[kPeelVisits]++;
              }
              remaining = 0;
            } else {
            const int start = e.ijk[ax];
            remaining = (s > 0 ? G.n[ax] - start : start + 1) - 1;
            step = (int64_t)s * G.stride[ax];
            cellp = e.cell + step;
            if (tau_acc <= prm<R>(P.tau_max, P.f.tau_max)) {
              const float4* __restrict__ rec = G.rec;
              for (int j = 0; j < kLanePeel && remaining > 0; ++j) {
                const float4 q0 = __ldg(rec + 2 * cellp);
                const float uq = __ldg(reinterpret_cast<const float*>(rec + 2 * cellp + 1) + ax);
                const R xcell = Vr * R(q0.w) - (s > 0 ? R(uq) : R(-uq));
                tau_acc += (R(q0.x) * voigt<R>(R(q0.y), xcell) + R(q0.z)) * hax;
                lc[kPeelVisits]++;
                cellp += step;
                --remaining;
                if (tau_acc > prm<R>(P.tau_max, P.f.tau_max)) break;
              }
            }
            }
            if (tau_acc > prm<R>(P.tau_max, P.f.tau_max)) {
              act = false;
            } else if (remaining == 0) {
              peel_tally(P, e, cam, ax, s, bin, W * m_exp(-R(tau_acc)));
              act = false;
            }
          }
        }
        unsigned coop = __ballot_sync(kFull, act);
        while (coop) {
          const int own = __ffs(coop) - 1;
          coop &= coop - 1;
          const int64_t c0 = __shfl_sync(kFull, cellp, own);
          const int64_t st = __shfl_sync(kFull, step, own);
          const int rem = __shfl_sync(kFull, remaining, own);
          const int axs = __shfl_sync(kFull, ax, own);
          const int ss = __shfl_sync(kFull, s, own);
          const R vv = __shfl_sync(kFull, Vr, own);
          R tacc = __shfl_sync(kFull, tau_acc, own);
          const Job* JS = L.jobs + __shfl_sync(kFull, e.job, own);
          const float4* __restrict__ rec = JS->g.rec;
          const R hs = prm<R>(JS->g.h[axs], JS->g.hf[axs]);
          const R tmax = prm<R>(JS->p.tau_max, JS->p.f.tau_max);
          bool cut = false;
          for (int base = 0; base < rem; base += 32) {
            const int m = base + lane;
            R tc = R(0);
            if (m < rem) {
              const int64_t c = c0 + st * m;
              const float4 q0 = __ldg(rec + 2 * c);
              const float uq = __ldg(reinterpret_cast<const float*>(rec + 2 * c + 1) + axs);
              const R xcell = vv * R(q0.w) - (ss > 0 ? R(uq) : R(-uq));
              tc = (R(q0.x) * voigt<R>(R(q0.y), xcell) + R(q0.z)) * hs;
              lc[kPeelVisits]++;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tc += __shfl_xor_sync(kFull, tc, o);
            tacc += __shfl_sync(kFull, tc, 0);
            if (tacc > tmax) { cut = true; break; }
          }
          if (lane == own && !cut) peel_tally(P, e, cam, ax, s, bin, W * m_exp(-tacc));
        }
      }
      }
    }
    __syncwarp();
    // packets that finished this round (their last peel-off, e.g. at a
    // scattering cap, tallied just above by some lane of the warp) are counted
    // to their jobs after a system-scope fence, so that a host which sees a
    // job's count complete finds its tallies complete.  One lane fences for
    // the warp (the warp barrier orders every lane's tally writes before it).
    if (L.job_done) {
      const unsigned fin = __ballot_sync(kFull, pend_done);
      if (fin) {
        if (lane == __ffs(fin) - 1) __threadfence_system();
        __syncwarp();
        if (pend_done) atomicAdd_system(L.job_done + pend_job, 1ull);
      }
    }
    pend_done = false;
    COLT_PHASE(2);
#ifdef COLT_PHASE_CLOCKS
    ph[3] += 1;
#endif
  }

#pragma unroll
  for (int i = 0; i < kNumLaunchCounters; ++i) {
    const unsigned long long v = warp_sum_ull(lc[i]);
    if (lane == 0 && v) atomicAdd(L.counters + i, v);
  }
#ifdef COLT_PHASE_CLOCKS
  for (int i = 0; i < 7; ++i)
    for (int o = 16; o > 0; o >>= 1) ph[i] = max(ph[i], __shfl_xor_sync(kFull, ph[i], o));
  if (lane == 0 && ph[3] > 64) {
    const double r = (double)ph[3];
    printf("phase cycles per round: refill %.0f  flight %.0f  draws %.0f  scatter %.0f  interaction-rest %.0f  "
           "peel %.0f  (rounds %llu)\n",
           ph[0] / r, ph[4] / r, ph[5] / r, ph[6] / r, ph[1] / r, ph[2] / r, ph[3]);
  }
#endif
#undef COLT_PHASE
#undef COLT_MARK
}

template <typename R, int kWarps>
constexpr size_t transport_smem() {
  return (sizeof(PeelEv<R>) + sizeof(int) + 2 * sizeof(R)) * 32 * kWarps;
}

template <typename R, bool kOct, int kMinBlocks, bool kX = false, int kWarps = 8>
static cudaError_t launch_t(const LaunchDev* L, int bps, int sm_count, cudaStream_t s) {
  const size_t smem = transport_smem<R, kWarps>();
  auto kern = k_transport<R, kWarps, kOct, kMinBlocks, kX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (bps > 0 && bps < occ) occ = bps;
  kern<<<sm_count * occ, kWarps * 32, smem, s>>>(L);
  return cudaGetLastError();
}

template <typename R, bool kOct, int kMinBlocks, int kWarps = 8>
static int occupancy_t() {
  auto kern = k_transport<R, kWarps, kOct, kMinBlocks, false>;
  constexpr size_t smem = transport_smem<R, kWarps>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 1;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
  return occ < 1 ? 1 : occ;
}

int transport_variants(int precision) { return precision == 0 ? 1 : 3; }

bool transport_has_warps(int precision, int variant, int warps) {
  return warps == 8 || (precision == 1 && variant == 0 && (warps == 4 || warps == 16));
}

cudaError_t launch_transport(const LaunchDev* L, int precision, int kind, int variant, int blocks_per_sm,
                             int sm_count, cudaStream_t s, bool extras, int warps) {
  if (!extras && precision == 1 && variant == 0 && warps == 4)
    return kind == 1 ? launch_t<float, true, 1, false, 4>(L, blocks_per_sm, sm_count, s)
                     : launch_t<float, false, 1, false, 4>(L, blocks_per_sm, sm_count, s);
  if (!extras && precision == 1 && variant == 0 && warps == 16)
    return kind == 1 ? launch_t<float, true, 1, false, 16>(L, blocks_per_sm, sm_count, s)
                     : launch_t<float, false, 1, false, 16>(L, blocks_per_sm, sm_count, s);
  if (extras) {
    // diffuse emission / Jeans estimate: the compiler's register allocation
    if (precision == 0)
      return kind == 1 ? launch_t<double, true, 1, true>(L, blocks_per_sm, sm_count, s)
                       : launch_t<double, false, 1, true>(L, blocks_per_sm, sm_count, s);
    return kind == 1 ? launch_t<float, true, 1, true>(L, blocks_per_sm, sm_count, s)
                     : launch_t<float, false, 1, true>(L, blocks_per_sm, sm_count, s);
  }
  if (precision == 0) {
    return kind == 1 ? launch_t<double, true, 1>(L, blocks_per_sm, sm_count, s)
                     : launch_t<double, false, 1>(L, blocks_per_sm, sm_count, s);
  }
  if (variant == 1)
    return kind == 1 ? launch_t<float, true, 4>(L, blocks_per_sm, sm_count, s)
                     : launch_t<float, false, 4>(L, blocks_per_sm, sm_count, s);
  if (variant == 2)
    return kind == 1 ? launch_t<float, true, 3>(L, blocks_per_sm, sm_count, s)
                     : launch_t<float, false, 3>(L, blocks_per_sm, sm_count, s);
  return kind == 1 ? launch_t<float, true, 1>(L, blocks_per_sm, sm_count, s)
                   : launch_t<float, false, 1>(L, blocks_per_sm, sm_count, s);
}

int transport_occupancy(int precision, int kind, int variant, int warps) {
  if (precision == 1 && variant == 0 && warps == 4)
    return kind == 1 ? occupancy_t<float, true, 1, 4>() : occupancy_t<float, false, 1, 4>();
  if (precision == 1 && variant == 0 && warps == 16)
    return kind == 1 ? occupancy_t<float, true, 1, 16>() : occupancy_t<float, false, 1, 16>();
  if (precision == 0) return kind == 1 ? occupancy_t<double, true, 1>() : occupancy_t<double, false, 1>();
  if (variant == 1) return kind == 1 ? occupancy_t<float, true, 4>() : occupancy_t<float, false, 4>();
  if (variant == 2) return kind == 1 ? occupancy_t<float, true, 3>() : occupancy_t<float, false, 3>();
  return kind == 1 ? occupancy_t<float, true, 1>() : occupancy_t<float, false, 1>();
}

}  // namespace colt
