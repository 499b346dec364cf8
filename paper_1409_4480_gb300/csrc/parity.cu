// Parity entry points: the transport kernel's own device functions applied
// element-wise, so that tests can compare them with the FP64 oracle on
// identical inputs and identical Philox counters.
//   colt_voigt   -> voigt<R>        (App. A1, Eq. AB)
//   colt_scatter -> scatter_hi<R>   (Sec. 3.1.3, 3.2.3, 3.2.4)
#include "internal.h"
#include "colt.h"

namespace colt {

template <typename R>
__global__ void k_voigt(const R* __restrict__ a, const R* __restrict__ x, R* __restrict__ H, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    H[i] = voigt<R>(a[i], x[i]);
}

cudaError_t launch_voigt(const void* a, const void* x, void* H, size_t n, int precision, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  const size_t want = (n + block - 1) / block;
  const unsigned grid = (unsigned)(want < 65535 * 8 ? want : 65535 * 8);
  if (precision == COLT_PLAIN)
    k_voigt<double><<<grid, block, 0, s>>>((const double*)a, (const double*)x, (double*)H, n);
  else
    k_voigt<float><<<grid, block, 0, s>>>((const float*)a, (const float*)x, (float*)H, n);
  return cudaGetLastError();
}

template <typename R>
__global__ void k_scatter(colt_scatter_io* io, size_t n, Rng rng) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  colt_scatter_io v = io[i];
  const R k[3] = {R(v.k[0]), R(v.k[1]), R(v.k[2])};
  // the interaction's block 0 carries the core R/Q choice in its last word
  const U4<R> b0 = uniforms<R>(rng, v.pid, v.event, 0);
  const U4<R> b1 = uniforms<R>(rng, v.pid, v.event, 1);
  const U4<R> b2 = uniforms<R>(rng, v.pid, v.event, 2);
  const ScatterOut<R> o = scatter_hi<R>(R(v.x), k, R(v.a), R(v.g), R(v.atau0), v.phase, rng, v.pid, v.event,
                                        b0.v[3], b1, b2, x_cw_fit<R>(R(v.a)));
  v.x_f = o.x_f;
  for (int q = 0; q < 3; ++q) {
    v.k_f[q] = o.k_f[q];
    v.u_atom[q] = o.u_atom[q];
  }
  v.u_par = o.u_par;
  v.x_crit = o.x_crit;
  v.RQ = o.RQ;
  v.mu = o.mu;
  v.n_trials = o.n_trials;
  io[i] = v;
}

cudaError_t launch_scatter(void* io, size_t n, uint64_t seed, int precision, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const Rng rng{uint32_t(seed), uint32_t(seed >> 32)};
  const int block = 128;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  if (precision == COLT_PLAIN)
    k_scatter<double><<<grid, block, 0, s>>>((colt_scatter_io*)io, n, rng);
  else
    k_scatter<float><<<grid, block, 0, s>>>((colt_scatter_io*)io, n, rng);
  return cudaGetLastError();
}

}  // namespace colt
