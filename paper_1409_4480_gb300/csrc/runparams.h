// Run parameters -> device job description, shared by every entry point that
// builds a job (colt_run / colt_run_batch / colt_submit in api.cu and the
// allocation-free colt_run_noalloc in noalloc.cu), so that all of them accept
// the same parameters and give the same spectral scale.
#pragma once
#include <cmath>

#include "colt.h"
#include "internal.h"

namespace colt {

// Sec. 2 line constants, T4 = T / 1e4 K: thermal velocity (km/s), damping
// parameter and line-centre cross-section (cm^2).
inline double vth_kms(double T) { return 12.85 * std::sqrt(T / 1.0e4); }
inline double damping_a(double T) { return 4.702e-4 / std::sqrt(T / 1.0e4); }
inline double sigma0(double T) { return 5.898e-14 / std::sqrt(T / 1.0e4); }

// A camera direction must be +-e_axis: 0 and its axis / sign, else -1.
int camera_axis(const double d[3], int* axis, int* sgn);

// nullptr when *p is a valid parameter set, else a message naming the first
// bad field.  has_luminosity: the grid carries a cell-luminosity table (needed
// by COLT_SOURCE_CELLS).
const char* check_run_params(const colt_run_params* p, bool has_luminosity);

// The job description of *p (already checked) on a grid spanning lo..hi;
// the tally pointers are left null for the caller to attach.
RunDev make_run_dev(const double lo[3], const double hi[3], const colt_run_params* p);

}  // namespace colt
