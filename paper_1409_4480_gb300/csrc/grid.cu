// Per-grid pre-computation: the non-local core-skipping estimate
// a tau_NL = min over paths of sum a tau_0 (Sec. 3.2.4, Eq. atauNL), computed
// once per grid (the paper computes it "once for each cell as the initial
// conditions are read in").
//
// Paths run along the six coordinate axes from the cell's faces outward,
// through whole cells, while the HI density stays within f_NL of the cell's
// own density (|n_i - n| < f_NL n); a path ends at the domain edge, and along a
// periodic axis after one period.  One thread per cell walks all six paths;
// neighbouring threads walk neighbouring rows, so the x-paths read coalesced.
// On octrees a path starts at the centre of the leaf's face, crosses whole
// leaves (each contributing a k_HI times its own size along the axis) and is
// walked with the transport's face-crossing routine in FP64.
#include "internal.h"
#include "octree.cuh"

namespace colt {

__global__ void k_atau_nl_cart(const GridDev G, const float* __restrict__ n_hi, double f_nl, float4* rec) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.n_cells) return;
  const float nref = n_hi[c];
  float best = 0.0f;
  if (nref > 0.0f && f_nl > 0.0) {
    const int i0 = (int)(c % G.n[0]);
    const int j0 = (int)((c / G.n[0]) % G.n[1]);
    const int k0 = (int)(c / ((int64_t)G.n[0] * G.n[1]));
    const int id0[3] = {i0, j0, k0};
    double dbest = 1e300;
    for (int dir = 0; dir < 6; ++dir) {
      const int ax = dir >> 1;
      const int s = (dir & 1) ? -1 : 1;
      const bool periodic = G.periodic_xy && ax < 2;
      const int limit = G.n[ax] - 1;
      double sum = 0.0;
      int idx = id0[ax];
      for (int step = 0; step < limit; ++step) {
        idx += s;
        if (idx < 0 || idx >= G.n[ax]) {
          if (!periodic) break;
          idx = idx < 0 ? G.n[ax] - 1 : 0;
        }
        const int64_t cc = c + (int64_t)(idx - id0[ax]) * G.stride[ax];
        const double ni = n_hi[cc];
        if (!(fabs(ni - (double)nref) < (double)f_nl * (double)nref)) break;
        const float4 r0 = rec[2 * cc];
        sum += (double)r0.y * (double)r0.x * G.h[ax];
      }
      dbest = fmin(dbest, sum);
    }
    best = (float)dbest;
  }
  rec[2 * c + 1].w = best;
}

__global__ void k_atau_nl_oct(const GridDev G, const float* __restrict__ n_hi, const uint8_t* __restrict__ lev,
                              const uint32_t* __restrict__ ijk, double f_nl, float4* rec) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.n_cells) return;
  const float nref = n_hi[c];
  float best = 0.0f;
  if (nref > 0.0f && f_nl > 0.0) {
    double dbest = 1e300;
    for (int dir = 0; dir < 6; ++dir) {
      const int ax = dir >> 1;
      const int s = (dir & 1) ? -1 : 1;
      double k[3] = {0.0, 0.0, 0.0};
      k[ax] = (double)s;
      int ci[3] = {(int)ijk[3 * c], (int)ijk[3 * c + 1], (int)ijk[3 * c + 2]};
      int lv = lev[c];
      CellPos<double> xi[3];
      for (int a = 0; a < 3; ++a) xi[a].set(0.5);
      int64_t cur = c;
      double sum = 0.0;
      for (int guard = 0; guard < (1 << 26); ++guard) {
        xi[ax].set(s > 0 ? 1.0 : 0.0);
        const int64_t nx = oct_cross<double>(G, cur, ax, s, k, ci, &lv, xi);
        if (nx < 0 || nx == c || nx >= G.n_cells) break;
        const double ni = n_hi[nx];
        if (!(fabs(ni - (double)nref) < f_nl * (double)nref)) break;
        const float4 r0 = rec[2 * nx];
        sum += (double)r0.y * (double)r0.x * (G.h[ax] * pow2neg<double>(lv));
        cur = nx;
      }
      dbest = fmin(dbest, sum);
    }
    best = (float)dbest;
  }
  rec[2 * c + 1].w = best;
}

cudaError_t launch_atau_nl(const GridDev& g, const float* n_hi, double f_nl, float4* rec_mut, cudaStream_t s) {
  if (g.n_cells == 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (g.n_cells + block - 1) / block;
  k_atau_nl_cart<<<(unsigned)grid, block, 0, s>>>(g, n_hi, f_nl, rec_mut);
  return cudaGetLastError();
}

cudaError_t launch_atau_nl_oct(const GridDev& g, const float* n_hi, const uint8_t* lev, const uint32_t* ijk,
                               double f_nl, float4* rec_mut, cudaStream_t s) {
  if (g.n_cells == 0) return cudaSuccess;
  const int block = 128;
  const int64_t grid = (g.n_cells + block - 1) / block;
  k_atau_nl_oct<<<(unsigned)grid, block, 0, s>>>(g, n_hi, lev, ijk, f_nl, rec_mut);
  return cudaGetLastError();
}

}  // namespace colt
