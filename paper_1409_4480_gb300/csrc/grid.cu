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
#include "internal.h"

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

cudaError_t launch_atau_nl(const GridDev& g, const float* n_hi, double f_nl, float4* rec_mut, cudaStream_t s) {
  if (g.n_cells == 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (g.n_cells + block - 1) / block;
  k_atau_nl_cart<<<(unsigned)grid, block, 0, s>>>(g, n_hi, f_nl, rec_mut);
  return cudaGetLastError();
}

}  // namespace colt
