// colt_run_noalloc: the blocking batched solve for callers that cannot
// allocate device memory -- code running under a fixed memory budget owned by
// another allocator, a host application whose device memory is carved up in
// advance, or a library that must not call cudaMalloc on its user's behalf.
// The caller supplies the cell records and the output tallies; the only device
// memory this entry point needs beyond them -- the launch header, the job
// table, the work counter, the launch counters and the error flag of the
// persistent transport kernel -- lives in a file-scope __device__ array below,
// which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "colt.h"
#include "internal.h"
#include "runparams.h"

using namespace colt;

namespace {

constexpr int kNoAllocMaxJobs = 8;                 // solves per call
constexpr size_t kScratchBytes = 16384;            // size of the static scratch
constexpr size_t kOffEnd = 256;                    // job_end[kNoAllocMaxJobs]
constexpr size_t kOffJobs = 512;                   // Job[kNoAllocMaxJobs]
constexpr size_t kOffWork = kOffJobs + sizeof(Job) * kNoAllocMaxJobs;  // next + launch counters
constexpr size_t kOffWorkAligned = (kOffWork + 255) & ~size_t(255);
constexpr size_t kOffError = kOffWorkAligned + 8 * sizeof(unsigned long long);
static_assert(sizeof(LaunchDev) <= kOffEnd, "launch header slot too small");
static_assert(kOffEnd + 8 * kNoAllocMaxJobs <= kOffJobs, "job_end slot too small");
static_assert(kOffError + sizeof(int) <= kScratchBytes, "scratch array too small");

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and kept for the life of the process: a
// device reset, or a release and re-creation of the primary context, may move
// the symbol, so this entry point must not be used across either.
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return COLT_EINVAL;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return COLT_ECUDA;
    g_scratch_dev[device] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[device];
  return COLT_OK;
}

}  // namespace

extern "C" int colt_run_noalloc(int n, const colt_grid_view* grids, const colt_run_params* params,
                                const colt_device_tallies* tallies, void* cuda_stream) {
  if (n < 1 || n > kNoAllocMaxJobs) return COLT_EINVAL;   // beyond the scratch's job table
  if (!grids || !params || !tallies) return COLT_EINVAL;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return COLT_ECUDA;
  unsigned char* scratch = nullptr;
  int rc = scratch_address(device, &scratch);
  if (rc) return rc;
  int sm_count = 0;
  if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return COLT_ECUDA;

  // host image of the launch header and job table (stack memory)
  alignas(16) unsigned char host[kOffJobs + sizeof(Job) * kNoAllocMaxJobs];
  std::memset(host, 0, sizeof(host));
  LaunchDev* hdr = reinterpret_cast<LaunchDev*>(host);
  unsigned long long* job_end = reinterpret_cast<unsigned long long*>(host + kOffEnd);
  Job* jobs = reinterpret_cast<Job*>(host + kOffJobs);
  const int precision = params[0].precision;
  unsigned long long total = 0;
  bool extras = false;
  for (int i = 0; i < n; ++i) {
    const colt_grid_view& gv = grids[i];
    const colt_run_params& p = params[i];
    const colt_device_tallies& t = tallies[i];
    if (!gv.records || gv.nx <= 0 || gv.ny <= 0 || gv.nz <= 0) return COLT_EINVAL;
    // the same parameter checks as colt_run, plus the limits of a grid view
    if (check_run_params(&p, false) != nullptr || p.precision != precision) return COLT_EINVAL;
    if (!t.spec || !t.counters) return COLT_EINVAL;
    if (p.n_cam > 0 && (!t.cam_spec || !t.cam_spec2)) return COLT_EINVAL;
    for (int c = 0; c < p.n_cam; ++c)
      if (p.cams[c].npix > 0 && !t.cam_image) return COLT_EINVAL;
    GridDev& G = jobs[i].g;
    G = GridDev{};
    G.rec = reinterpret_cast<const float4*>(gv.records);
    G.kind = COLT_CARTESIAN;
    G.n[0] = gv.nx; G.n[1] = gv.ny; G.n[2] = gv.nz;
    G.stride[0] = 1; G.stride[1] = gv.nx; G.stride[2] = (int64_t)gv.nx * gv.ny;
    for (int a = 0; a < 3; ++a) {
      if (!(gv.hi[a] > gv.lo[a])) return COLT_EINVAL;
      G.lo[a] = gv.lo[a];
      G.hi[a] = gv.hi[a];
      G.h[a] = (gv.hi[a] - gv.lo[a]) / G.n[a];
    }
    fill_f32(G);
    G.periodic_xy = gv.periodic_xy ? 1 : 0;
    G.n_cells = (int64_t)gv.nx * gv.ny * gv.nz;
    RunDev& r = jobs[i].p;
    r = make_run_dev(G.lo, G.hi, &p);
    extras = extras || run_needs_extras(r);
    r.t.spec = t.spec;
    r.t.counters = t.counters;
    r.t.cam_spec = t.cam_spec;
    r.t.cam_spec2 = t.cam_spec2;
    r.t.cam_image = t.cam_image;
    total += p.n_packets;
    job_end[i] = total;
  }
  hdr->jobs = reinterpret_cast<const Job*>(scratch + kOffJobs);
  hdr->job_end = reinterpret_cast<const unsigned long long*>(scratch + kOffEnd);
  hdr->n_jobs = n;
  hdr->total = total;
  hdr->next = reinterpret_cast<unsigned long long*>(scratch + kOffWorkAligned);
  hdr->counters = hdr->next + 1;
  hdr->error = reinterpret_cast<int*>(scratch + kOffError);

  // the outputs start at zero, and so do the work counter and error flag
  for (int i = 0; i < n; ++i) {
    const colt_run_params& p = params[i];
    const colt_device_tallies& t = tallies[i];
    if (cudaMemsetAsync(t.spec, 0, sizeof(unsigned long long) * p.spec_nbins, stream) != cudaSuccess ||
        cudaMemsetAsync(t.counters, 0, sizeof(unsigned long long) * kNumCounters, stream) != cudaSuccess)
      return COLT_ECUDA;
    if (p.n_cam > 0) {
      const size_t ns = sizeof(double) * (size_t)p.n_cam * p.cam_nbins;
      if (cudaMemsetAsync(t.cam_spec, 0, ns, stream) != cudaSuccess ||
          cudaMemsetAsync(t.cam_spec2, 0, ns, stream) != cudaSuccess)
        return COLT_ECUDA;
      size_t img = 0;
      for (int c = 0; c < p.n_cam; ++c) img += (size_t)p.cams[c].npix * p.cams[c].npix * p.cam_nbins;
      if (img && cudaMemsetAsync(t.cam_image, 0, sizeof(double) * img, stream) != cudaSuccess) return COLT_ECUDA;
    }
  }
  if (cudaMemsetAsync(scratch + kOffWorkAligned, 0, kOffError + sizeof(int) - kOffWorkAligned, stream) != cudaSuccess)
    return COLT_ECUDA;
  if (cudaMemcpyAsync(scratch, host, kOffJobs + sizeof(Job) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return COLT_ECUDA;
  if (total > 0 && launch_transport(reinterpret_cast<const LaunchDev*>(scratch), precision, COLT_CARTESIAN, 0,
                                    params[0].blocks_per_sm, sm_count, stream, extras) != cudaSuccess)
    return COLT_ECUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return COLT_ECUDA;
  int flag = 0;
  if (cudaMemcpy(&flag, scratch + kOffError, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return COLT_ECUDA;
  return flag ? COLT_EDEVICE : COLT_OK;
}
