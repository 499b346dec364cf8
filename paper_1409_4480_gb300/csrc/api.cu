// C ABI of libcolt (declared and documented in include/colt.h): contexts,
// grids, blocking runs, the continuous-batching scheduler and the parity
// helpers.  Host-side runtime in C++17; all compute is in the CUDA kernels.
//
// Launch slots: a persistent launch needs a header + job table in device
// memory (staged from pinned host memory) and a work counter.  The context
// owns kSlots of them, each with its own stream, so the serving scheduler can
// keep several launches in flight: the GPU's block scheduler hands SMs freed
// by one launch's finished CTAs to the next launch, so a launch's tail of
// long histories overlaps new work.  Slot 0 runs on the context stream and
// also serves the blocking calls.  Every launch counts each job's finished
// packets in mapped host memory, so a served request completes with its own
// packets; tally set-up, grid building and result copies run on an
// auxiliary stream, never behind a launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "colt.h"
#include "internal.h"
#include "runparams.h"

using namespace colt;

namespace {

constexpr int kMaxJobs = 256;                  // solves per persistent launch
constexpr int kSlots = 6;                      // launches in flight (serving)
constexpr uint64_t kStepPackets = 1ull << 20;  // packet budget of one serving launch
constexpr size_t kMaxQueued = 4096;             // requests waiting for admission
constexpr int kWorkWords = 8;                  // work counter + launch counters (+ phase clocks)
constexpr int kMaxPassed = 4;                  // launches a ready request may be passed over

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct GridObj {
  GridDev dev;
  float4* rec = nullptr;
  int32_t* node = nullptr;              // octree: node table (device)
  uint32_t* nbr = nullptr;              // octree: face neighbours (device)
  unsigned long long* lum_cum = nullptr;  // diffuse emission: prefix sums of the cell weights (device)
  uint32_t* leaf_loc = nullptr;         // octree + diffuse emission: leaf level and coordinates (device)
  size_t lum_bytes = 0;
  std::vector<uint8_t> leaf_level;      // octree leaves (host copies)
  std::vector<uint32_t> leaf_ijk;
  size_t bytes = 0;
  // longest history (scatterings) any finished solve on this grid has had
  uint64_t longest = 0;
  bool measured = false;
};

// Longest-expected-first ordering of the jobs of a launch: the persistent
// kernel hands out packets in job order, so a job whose histories can be very
// long should start first, letting its longest packet overlap the rest of the
// launch instead of running alone at the end (LPT scheduling).  A grid that
// has never run sorts first.
uint64_t grid_cost(const GridObj& g) { return g.measured ? g.longest : ~0ull; }


// Device + pinned staging for one persistent launch: header, job_end, jobs.
struct LaunchBuf {
  unsigned char* host = nullptr;        // pinned
  unsigned char* dev = nullptr;
  size_t bytes = 0;
  unsigned long long* work = nullptr;   // device: next counter + launch counters, then job_max
  unsigned long long* work_h = nullptr; // pinned copy of work after the launch ...
  unsigned long long* jmax_h = nullptr; // ... and its job_max part
  unsigned long long* jdone_h = nullptr; // pinned, mapped: packets of each job finished (written by the kernel)
  unsigned long long* jdone_d = nullptr; // its device address
  int* error = nullptr;
  LaunchDev* hdr_h() { return reinterpret_cast<LaunchDev*>(host); }
  unsigned long long* end_h() { return reinterpret_cast<unsigned long long*>(host + 256); }
  Job* jobs_h() { return reinterpret_cast<Job*>(host + 256 + 8 * kMaxJobs); }
  size_t off_end() const { return 256; }
  size_t off_jobs() const { return 256 + 8 * kMaxJobs; }
};

struct Slot {
  LaunchBuf lb;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t done = nullptr;
  cudaEvent_t k0 = nullptr, k1 = nullptr;   // around the transport kernel (timing)
  bool timed = false;                       // k0/k1 hold a launch not yet accounted
  bool in_flight = false;
  std::vector<std::pair<uint64_t, uint64_t>> jobs;  // (request id, packets)
  std::vector<char> credited;                       // job's packets already counted to its request
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [precision][grid kind]
  int graph_cfg[2][2] = {{-1, -1}, {-1, -1}};                               // launch configuration captured
};

struct Tally {
  unsigned long long* spec = nullptr;
  unsigned long long* counters = nullptr;
  double* cam_spec = nullptr;
  double* cam_spec2 = nullptr;
  double* cam_image = nullptr;
  int32_t* pk_status = nullptr;
  uint64_t* pk_nscat = nullptr;
  double* pk_freq = nullptr;
  size_t bytes = 0;
  void* block = nullptr;                // one allocation holds everything
  cudaStream_t stream = nullptr;        // stream-ordered pool allocation
};

enum ReqState { kQueued = 0, kAdmitted = 1, kDone = 2 };

struct Req {
  uint64_t id = 0;
  colt_grid grid = 0;
  colt_run_params p{};
  std::vector<colt_camera> cams;
  std::vector<colt_source> srcs;
  RunDev run;                           // tally pointers filled at admission
  Tally tally;
  int state = kQueued;
  int passed = 0;                       // launches built while it was ready but left out
  uint64_t next_local = 0;              // packets handed to launches
  uint64_t done_packets = 0;
  uint64_t target = 0;                  // packets the request will run (n_packets, less after colt_cancel)
  bool cancelled = false;
  double t_submit = 0, t_done = 0;
  size_t need_bytes = 0;
  uint64_t longest = 0;                 // most scatterings of one packet, over its ended launches
};

}  // namespace

struct colt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  size_t used = 0;
  int sm_count = 0;
  size_t l2 = 0;
  int cc_major = 0, cc_minor = 0;
  std::recursive_mutex mu;
  std::string err;
  uint64_t next_handle = 1;
  std::map<uint64_t, GridObj> grids;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::deque<uint64_t> queue;           // queued request ids (FIFO)
  Slot slots[kSlots];
  // library-internal stream for tally set-up, grid building and result
  // copies, so that none of them queues behind a launch on the context stream
  cudaStream_t aux = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_alloc = nullptr;
  uint64_t launches = 0;                // transport kernel launches issued
  uint64_t timed_launches = 0;          // ... of them completed and timed
  double kernel_ms = 0.0;               // their summed device time (CUDA events on their streams)
  uint64_t cell_visits = 0;             // ... and their flight cell and peel-off visits
  uint64_t peel_visits = 0;
  // completion signal of serving launches: a host function enqueued behind
  // each launch bumps done_seq, so colt_wait wakes when ANY slot finishes
  std::mutex cv_mu;
  std::condition_variable cv;
  uint64_t done_seq = 0;
  // launch configuration per [precision][grid kind] (colt_autotune)
  colt_launch_config cfg[2][2] = {{{0, 0, 0.0, 8, 1}, {0, 0, 0.0, 8, 1}}, {{0, 0, 0.0, 8, 1}, {0, 0, 0.0, 8, 1}}};
};

namespace {

int fail(colt_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(colt_ctx* c, cudaError_t e, const char* where) {
  return fail(c, COLT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CU(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int validate_params(colt_ctx* ctx, const colt_run_params* p, const GridObj& g) {
  const char* msg = check_run_params(p, g.lum_cum != nullptr);
  return msg ? fail(ctx, COLT_EINVAL, msg) : COLT_OK;
}

size_t tally_bytes(const colt_run_params* p, bool per_packet) {
  auto r = [](size_t n) { return (n + 255) & ~size_t(255); };
  size_t b = 0;
  b += r(sizeof(unsigned long long) * (size_t)p->spec_nbins);
  b += r(sizeof(unsigned long long) * kNumCounters);
  if (p->n_cam > 0) {
    b += 2 * r(sizeof(double) * (size_t)p->n_cam * p->cam_nbins);
    size_t img = 0;
    for (int i = 0; i < p->n_cam; ++i) img += (size_t)p->cams[i].npix * p->cams[i].npix * p->cam_nbins;
    if (img) b += r(sizeof(double) * img);
  }
  if (per_packet)
    b += r(sizeof(int32_t) * p->n_packets) + r(sizeof(uint64_t) * p->n_packets) + r(sizeof(double) * p->n_packets);
  return b;
}

// Allocate and zero one solve's tallies (stream-ordered pool on the context stream).
int alloc_tally(colt_ctx* ctx, const colt_run_params* p, bool per_packet, Tally* t) {
  t->bytes = tally_bytes(p, per_packet) + 256;
  t->stream = ctx->aux;
  CU(cudaMallocAsync(&t->block, t->bytes, ctx->aux));
  CU(cudaMemsetAsync(t->block, 0, t->bytes, ctx->aux));
  unsigned char* q = static_cast<unsigned char*>(t->block);
  auto take = [&](size_t n) {
    unsigned char* r = q;
    q += (n + 255) & ~size_t(255);
    return r;
  };
  t->counters = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * kNumCounters));
  t->spec = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * p->spec_nbins));
  if (p->n_cam > 0) {
    t->cam_spec = reinterpret_cast<double*>(take(sizeof(double) * p->n_cam * p->cam_nbins));
    t->cam_spec2 = reinterpret_cast<double*>(take(sizeof(double) * p->n_cam * p->cam_nbins));
    size_t img = 0;
    for (int i = 0; i < p->n_cam; ++i) img += (size_t)p->cams[i].npix * p->cams[i].npix * p->cam_nbins;
    if (img) t->cam_image = reinterpret_cast<double*>(take(sizeof(double) * img));
  }
  if (per_packet) {
    t->pk_status = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * p->n_packets));
    t->pk_nscat = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * p->n_packets));
    t->pk_freq = reinterpret_cast<double*>(take(sizeof(double) * p->n_packets));
  }
  return COLT_OK;
}

void free_tally(Tally* t) {
  if (t->block) cudaFreeAsync(t->block, t->stream);
  *t = Tally{};
}

// Job description from a grid and parameters (tally pointers attached later).
RunDev make_run(const GridObj& g, const colt_run_params* p) { return make_run_dev(g.dev.lo, g.dev.hi, p); }

void attach_tally(RunDev* r, const Tally& t) {
  r->t.spec = t.spec;
  r->t.counters = t.counters;
  r->t.cam_spec = t.cam_spec;
  r->t.cam_spec2 = t.cam_spec2;
  r->t.cam_image = t.cam_image;
  r->t.pk_status = t.pk_status;
  r->t.pk_nscat = t.pk_nscat;
  r->t.pk_freq = t.pk_freq;
}

int ensure_slot(colt_ctx* ctx, int si) {
  Slot& sl = ctx->slots[si];
  LaunchBuf& lb = sl.lb;
  if (lb.host) return COLT_OK;
  if (si == 0) {
    sl.stream = ctx->stream;
  } else {
    CU(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
    sl.own_stream = true;
  }
  CU(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  CU(cudaEventCreate(&sl.k0));
  CU(cudaEventCreate(&sl.k1));
  lb.bytes = lb.off_jobs() + sizeof(Job) * kMaxJobs;
  CU(cudaMallocHost(&lb.host, lb.bytes));
  CU(cudaMalloc(&lb.dev, lb.bytes));
  CU(cudaMalloc(&lb.work, sizeof(unsigned long long) * (kWorkWords + kMaxJobs)));
  CU(cudaMallocHost(&lb.work_h, sizeof(unsigned long long) * (kWorkWords + kMaxJobs)));
  std::memset(lb.work_h, 0, sizeof(unsigned long long) * (kWorkWords + kMaxJobs));
  lb.jmax_h = lb.work_h + kWorkWords;
  CU(cudaHostAlloc(&lb.jdone_h, sizeof(unsigned long long) * kMaxJobs, cudaHostAllocMapped));
  std::memset(lb.jdone_h, 0, sizeof(unsigned long long) * kMaxJobs);
  CU(cudaMalloc(&lb.error, sizeof(int)));
  CU(cudaMemset(lb.error, 0, sizeof(int)));
  std::memset(lb.host, 0, lb.bytes);
  LaunchDev* h = lb.hdr_h();
  h->jobs = reinterpret_cast<const Job*>(lb.dev + lb.off_jobs());
  h->job_end = reinterpret_cast<const unsigned long long*>(lb.dev + lb.off_end());
  h->next = lb.work;
  h->counters = lb.work + 1;
  h->error = lb.error;
  h->job_max = lb.work + kWorkWords;
  // finished-packet counts per job (set per launch: serving launches only)
  CU(cudaHostGetDevicePointer(reinterpret_cast<void**>(&lb.jdone_d), lb.jdone_h, 0));
  return COLT_OK;
}

// Enqueue one persistent launch over the jobs staged in the slot's host
// buffer: header/job-table copy, counter reset, kernel.  Recorded once per
// (slot, precision) as a CUDA graph and replayed.
int enqueue_launch(colt_ctx* ctx, int si, int precision, int kind, int blocks_per_sm, bool extras) {
  Slot& sl = ctx->slots[si];
  LaunchBuf& lb = sl.lb;
  const int gi = precision == COLT_PLAIN ? 0 : 1;
  const int gk = kind == COLT_OCTREE ? 1 : 0;
  const colt_launch_config& cfg = ctx->cfg[gi][gk];
  const int warps = cfg.warps_per_block > 0 && transport_has_warps(precision, cfg.variant, cfg.warps_per_block)
                        ? cfg.warps_per_block : 8;
  lb.hdr_h()->refill_min = std::max(1, cfg.refill_min);
  // the slot's previous launch has ended: nothing writes the counts now
  std::memset(lb.jdone_h, 0, sizeof(unsigned long long) * kMaxJobs);
  ++ctx->launches;
  if (blocks_per_sm > 0) {
    CU(cudaMemcpyAsync(lb.dev, lb.host, lb.bytes, cudaMemcpyHostToDevice, sl.stream));
    CU(cudaMemsetAsync(lb.work, 0, sizeof(unsigned long long) * (kWorkWords + kMaxJobs), sl.stream));
    CU(cudaEventRecord(sl.k0, sl.stream));
    CU(launch_transport(reinterpret_cast<const LaunchDev*>(lb.dev), precision, kind, cfg.variant, blocks_per_sm,
                        ctx->sm_count, sl.stream, extras, warps));
    CU(cudaEventRecord(sl.k1, sl.stream));
    sl.timed = true;
    CU(cudaMemcpyAsync(lb.work_h, lb.work, sizeof(unsigned long long) * (kWorkWords + kMaxJobs),
                       cudaMemcpyDeviceToHost, sl.stream));
    return COLT_OK;
  }
  const int code = cfg.variant * 64 + cfg.blocks_per_sm + (extras ? 4096 : 0) + warps * 8192;
  if (sl.graph[gi][gk] && sl.graph_cfg[gi][gk] != code) {
    cudaGraphExecDestroy(sl.graph[gi][gk]);
    sl.graph[gi][gk] = nullptr;
  }
  if (!sl.graph[gi][gk]) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(lb.dev, lb.host, lb.bytes, cudaMemcpyHostToDevice, sl.stream);
    cudaMemsetAsync(lb.work, 0, sizeof(unsigned long long) * (kWorkWords + kMaxJobs), sl.stream);
    cudaError_t le = launch_transport(reinterpret_cast<const LaunchDev*>(lb.dev), precision, kind, cfg.variant,
                                      cfg.blocks_per_sm, ctx->sm_count, sl.stream, extras, warps);
    cudaMemcpyAsync(lb.work_h, lb.work, sizeof(unsigned long long) * (kWorkWords + kMaxJobs),
                    cudaMemcpyDeviceToHost, sl.stream);
    cudaError_t ce = cudaStreamEndCapture(sl.stream, &g);
    if (le != cudaSuccess) return cuda_fail(ctx, le, "transport launch (capture)");
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&sl.graph[gi][gk], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(ctx, ie, "cudaGraphInstantiate");
    sl.graph_cfg[gi][gk] = code;
  }
  // the graph holds the header copy and counter reset before the kernel and
  // one small copy after it: its time is the kernel's to within those
  CU(cudaEventRecord(sl.k0, sl.stream));
  CU(cudaGraphLaunch(sl.graph[gi][gk], sl.stream));
  CU(cudaEventRecord(sl.k1, sl.stream));
  sl.timed = true;
  return COLT_OK;
}

// After the slot's launch completed: device-side error flag.
int check_device_error(colt_ctx* ctx, int si) {
  Slot& sl = ctx->slots[si];
  int h = 0;
  if (!sl.lb.error) return COLT_OK;
  CU(cudaMemcpyAsync(&h, sl.lb.error, sizeof(int), cudaMemcpyDeviceToHost, sl.stream));
  CU(cudaStreamSynchronize(sl.stream));
  if (h) {
    CU(cudaMemsetAsync(sl.lb.error, 0, sizeof(int), sl.stream));
    return fail(ctx, COLT_EDEVICE, "transport kernel raised its error flag (cell index out of range)");
  }
  return COLT_OK;
}

// Copy a solve's tallies into a caller's colt_result.
int copy_result(colt_ctx* ctx, const colt_run_params* p, const Tally& t, colt_result* out, bool per_packet) {
  unsigned long long cnt[kNumCounters];
  CU(cudaMemcpyAsync(cnt, t.counters, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->aux));
  if (out->spec)
    CU(cudaMemcpyAsync(out->spec, t.spec, sizeof(uint64_t) * p->spec_nbins, cudaMemcpyDeviceToHost, ctx->aux));
  if (p->n_cam > 0) {
    const size_t ns = (size_t)p->n_cam * p->cam_nbins;
    if (out->cam_spec) CU(cudaMemcpyAsync(out->cam_spec, t.cam_spec, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->aux));
    if (out->cam_spec2) CU(cudaMemcpyAsync(out->cam_spec2, t.cam_spec2, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->aux));
    if (out->cam_image && t.cam_image) {
      size_t img = 0;
      for (int i = 0; i < p->n_cam; ++i) img += (size_t)p->cams[i].npix * p->cams[i].npix * p->cam_nbins;
      CU(cudaMemcpyAsync(out->cam_image, t.cam_image, sizeof(double) * img, cudaMemcpyDeviceToHost, ctx->aux));
    }
  }
  if (per_packet) {
    if (out->pk_status) CU(cudaMemcpyAsync(out->pk_status, t.pk_status, sizeof(int32_t) * p->n_packets, cudaMemcpyDeviceToHost, ctx->aux));
    if (out->pk_nscat) CU(cudaMemcpyAsync(out->pk_nscat, t.pk_nscat, sizeof(uint64_t) * p->n_packets, cudaMemcpyDeviceToHost, ctx->aux));
    if (out->pk_freq) CU(cudaMemcpyAsync(out->pk_freq, t.pk_freq, sizeof(double) * p->n_packets, cudaMemcpyDeviceToHost, ctx->aux));
  }
  CU(cudaStreamSynchronize(ctx->aux));
  out->n_emitted = cnt[kEmitted];
  out->n_escaped = cnt[kEscaped];
  out->n_absorbed = cnt[kAbsorbed];
  out->n_capped = cnt[kCapped];
  out->n_scat = cnt[kScat];
  out->n_scat_hi = cnt[kScatHI];
  out->spec_under = cnt[kUnder];
  out->spec_over = cnt[kOver];
  return COLT_OK;
}

// Octree tables from the leaves (host): node[v] >= 0 is the first of v's 8
// children, node[v] < 0 marks leaf -1 - node[v]; the leaves must tile the box
// (every internal node has 8 children, no leaf overlaps another).
constexpr int32_t kUnset = INT32_MIN;

int build_octree_tables(colt_ctx* ctx, int64_t n, const uint8_t* lev, const uint32_t* ijk,
                        std::vector<int32_t>* node_out, std::vector<uint32_t>* nbr_out, int* max_level) {
  std::vector<int32_t>& node = *node_out;
  if (n > (int64_t)kNodeMask) return fail(ctx, COLT_EINVAL, "octree has too many leaves");
  node.assign(1, kUnset);
  int maxl = 0;
  for (int64_t l = 0; l < n; ++l) {
    const int L = lev[l];
    if (L > kMaxOctLevel) return fail(ctx, COLT_EINVAL, "octree level above the supported maximum");
    maxl = std::max(maxl, L);
    for (int a = 0; a < 3; ++a)
      if ((uint64_t)ijk[3 * l + a] >= (1ull << L)) return fail(ctx, COLT_EINVAL, "leaf coordinate outside its level");
    size_t v = 0;
    for (int t = 1; t <= L; ++t) {
      if (node[v] != kUnset && node[v] < 0) return fail(ctx, COLT_EINVAL, "octree leaves overlap");
      if (node[v] == kUnset) {
        if (node.size() + 8 > (size_t)kNodeMask) return fail(ctx, COLT_EINVAL, "octree has too many nodes");
        node[v] = (int32_t)node.size();
        node.resize(node.size() + 8, kUnset);
      }
      int cidx = 0;
      for (int a = 0; a < 3; ++a) cidx |= (int)((ijk[3 * l + a] >> (L - t)) & 1u) << a;
      v = (size_t)node[v] + cidx;
    }
    if (node[v] != kUnset) return fail(ctx, COLT_EINVAL, "octree leaves overlap");
    node[v] = -1 - (int32_t)l;
  }
  for (int32_t v : node)
    if (v == kUnset) return fail(ctx, COLT_EINVAL, "octree leaves do not tile the box");
  // face neighbours: the node across each face at the leaf's level, or the
  // coarser leaf that covers it
  std::vector<uint32_t>& nbr = *nbr_out;
  nbr.assign(6 * (size_t)n, kNoNbr);
  auto work = [&](int64_t l0, int64_t l1) {
    for (int64_t l = l0; l < l1; ++l) {
      const int L = lev[l];
      for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1;
        int64_t adj[3] = {ijk[3 * l], ijk[3 * l + 1], ijk[3 * l + 2]};
        adj[ax] += (f & 1) ? -1 : 1;
        if (adj[ax] < 0 || adj[ax] >= (int64_t)1 << L) continue;
        size_t v = 0;
        int t = 0;
        while (t < L && node[v] >= 0) {
          ++t;
          int cidx = 0;
          for (int a = 0; a < 3; ++a) cidx |= (int)((adj[a] >> (L - t)) & 1) << a;
          v = (size_t)node[v] + cidx;
        }
        nbr[6 * l + f] = node[v] < 0 ? ((uint32_t)(-1 - node[v]) | kLeafFlag | ((uint32_t)t << 27))
                                     : ((uint32_t)v | ((uint32_t)t << 27));
      }
    }
  };
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(16, n / 65536));
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) th.emplace_back(work, n * i / nt, n * (i + 1) / nt);
  for (auto& t : th) t.join();
  *max_level = maxl;
  return COLT_OK;
}

int build_grid(colt_ctx* ctx, const colt_grid_desc* d, GridObj* g) {
  if (!d) return fail(ctx, COLT_EINVAL, "desc is NULL");
  const bool oct = d->kind == COLT_OCTREE;
  if (!oct && d->kind != COLT_CARTESIAN) return fail(ctx, COLT_EINVAL, "unknown grid kind");
  int64_t n = 0;
  if (oct) {
    if (d->n_cells <= 0 || !d->leaf_level || !d->leaf_ijk) return fail(ctx, COLT_EINVAL, "octree needs leaves");
    if (d->periodic_xy) return fail(ctx, COLT_EINVAL, "periodic boundaries need a Cartesian grid");
    n = d->n_cells;
  } else {
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return fail(ctx, COLT_EINVAL, "cell counts must be positive");
    n = (int64_t)d->nx * d->ny * d->nz;
  }
  if (n >= ((int64_t)1 << 31) - 1) return fail(ctx, COLT_EINVAL, "too many cells");
  for (int a = 0; a < 3; ++a)
    if (!(d->hi[a] > d->lo[a]) || !std::isfinite(d->lo[a]) || !std::isfinite(d->hi[a]))
      return fail(ctx, COLT_EINVAL, "box must have hi > lo");
  if (!d->n_HI || !d->T || !d->vx || !d->vy || !d->vz) return fail(ctx, COLT_EINVAL, "missing field array");
  if (!(d->f_nl >= 0)) return fail(ctx, COLT_EINVAL, "f_nl must be >= 0");
  // fields to host
  std::vector<float> hf[6];
  const float* src[6] = {d->n_HI, d->T, d->vx, d->vy, d->vz, d->k_dust};
  const float* f[6];
  for (int i = 0; i < 6; ++i) {
    if (!src[i]) { f[i] = nullptr; continue; }
    if (d->fields_mem == COLT_MEM_DEVICE) {
      hf[i].resize(n);
      CU(cudaMemcpyAsync(hf[i].data(), src[i], sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->aux));
      f[i] = hf[i].data();
    } else {
      f[i] = src[i];
    }
  }
  CU(cudaStreamSynchronize(ctx->aux));
  std::vector<int32_t> node;
  std::vector<uint32_t> nbr;
  int max_level = 0;
  if (oct) {
    int rc = build_octree_tables(ctx, n, d->leaf_level, d->leaf_ijk, &node, &nbr, &max_level);
    if (rc) return rc;
    g->leaf_level.assign(d->leaf_level, d->leaf_level + n);
    g->leaf_ijk.assign(d->leaf_ijk, d->leaf_ijk + 3 * n);
  }
  const size_t bytes = sizeof(float4) * 2 * (size_t)n + sizeof(int32_t) * node.size() + sizeof(uint32_t) * nbr.size();
  if (ctx->used + bytes > ctx->budget) return fail(ctx, COLT_ENOMEM, "grid exceeds the memory budget");
  std::vector<float4> rec(2 * (size_t)n);
  for (int64_t c = 0; c < n; ++c) {
    const double T = f[1][c], nh = f[0][c];
    if (!(T > 0) || !std::isfinite(T) || !(nh >= 0) || !std::isfinite(nh))
      return fail(ctx, COLT_EINVAL, "T must be > 0 and n_HI >= 0 (finite) in every cell");
    const double vth = vth_kms(T);
    const double kd = f[5] ? (double)f[5][c] : 0.0;
    if (!(kd >= 0) || !std::isfinite(kd)) return fail(ctx, COLT_EINVAL, "k_dust must be >= 0");
    rec[2 * c] = make_float4((float)(nh * sigma0(T)), (float)damping_a(T), (float)kd, (float)(1.0 / vth));
    rec[2 * c + 1] = make_float4((float)(f[2][c] / vth), (float)(f[3][c] / vth), (float)(f[4][c] / vth), 0.0f);
  }
  GridDev& G = g->dev;
  G.kind = oct ? COLT_OCTREE : COLT_CARTESIAN;
  if (!oct) {
    G.n[0] = d->nx; G.n[1] = d->ny; G.n[2] = d->nz;
    G.stride[0] = 1; G.stride[1] = d->nx; G.stride[2] = (int64_t)d->nx * d->ny;
  }
  for (int a = 0; a < 3; ++a) {
    G.lo[a] = d->lo[a];
    G.hi[a] = d->hi[a];
    G.h[a] = oct ? (d->hi[a] - d->lo[a]) : (d->hi[a] - d->lo[a]) / G.n[a];
  }
  fill_f32(G);
  G.periodic_xy = (!oct && d->periodic_xy) ? 1 : 0;
  G.n_cells = n;
  G.max_level = max_level;
  CU(cudaMalloc(&g->rec, sizeof(float4) * 2 * (size_t)n));
  CU(cudaMemcpyAsync(g->rec, rec.data(), sizeof(float4) * 2 * (size_t)n, cudaMemcpyHostToDevice, ctx->aux));
  G.rec = g->rec;
  if (oct) {
    CU(cudaMalloc(&g->node, sizeof(int32_t) * node.size()));
    CU(cudaMalloc(&g->nbr, sizeof(uint32_t) * nbr.size()));
    CU(cudaMemcpyAsync(g->node, node.data(), sizeof(int32_t) * node.size(), cudaMemcpyHostToDevice, ctx->aux));
    CU(cudaMemcpyAsync(g->nbr, nbr.data(), sizeof(uint32_t) * nbr.size(), cudaMemcpyHostToDevice, ctx->aux));
    G.node = g->node;
    G.nbr = g->nbr;
  }
  // non-local a tau (Eq. atauNL), once per grid
  float* dn = nullptr;
  CU(cudaMallocAsync(&dn, sizeof(float) * n, ctx->aux));
  CU(cudaMemcpyAsync(dn, f[0], sizeof(float) * n, cudaMemcpyHostToDevice, ctx->aux));
  cudaError_t e = cudaSuccess;
  if (oct) {
    uint8_t* dlev = nullptr;
    uint32_t* dijk = nullptr;
    CU(cudaMallocAsync(&dlev, (size_t)n, ctx->aux));
    CU(cudaMallocAsync(&dijk, sizeof(uint32_t) * 3 * (size_t)n, ctx->aux));
    CU(cudaMemcpyAsync(dlev, d->leaf_level, (size_t)n, cudaMemcpyHostToDevice, ctx->aux));
    CU(cudaMemcpyAsync(dijk, d->leaf_ijk, sizeof(uint32_t) * 3 * (size_t)n, cudaMemcpyHostToDevice, ctx->aux));
    e = launch_atau_nl_oct(G, dn, dlev, dijk, d->f_nl, g->rec, ctx->aux);
    cudaFreeAsync(dlev, ctx->aux);
    cudaFreeAsync(dijk, ctx->aux);
  } else {
    e = launch_atau_nl(G, dn, d->f_nl, g->rec, ctx->aux);
  }
  cudaFreeAsync(dn, ctx->aux);
  cudaError_t e2 = cudaStreamSynchronize(ctx->aux);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "atau_nl kernel");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "atau_nl sync");
  g->bytes = bytes;
  return COLT_OK;
}

void free_grid(GridObj& g) {
  if (g.rec) cudaFree(g.rec);
  if (g.node) cudaFree(g.node);
  if (g.nbr) cudaFree(g.nbr);
  if (g.lum_cum) cudaFree(g.lum_cum);
  if (g.leaf_loc) cudaFree(g.leaf_loc);
  g.rec = nullptr;
  g.node = nullptr;
  g.nbr = nullptr;
  g.lum_cum = nullptr;
  g.leaf_loc = nullptr;
}

// Record the longest history a finished job saw on its grid.
void learn_cost(colt_ctx* ctx, colt_grid grid, uint64_t longest) {
  auto g = ctx->grids.find(grid);
  if (g == ctx->grids.end()) return;
  g->second.longest = std::max(g->second.longest, longest);
  g->second.measured = true;
}

// Count the packets of a slot's jobs to their requests: every job once the
// launch has ended (all), else the jobs whose packets have all finished
// (the kernel bumps the job's count in mapped host memory after a fence, so
// the job's tallies are complete when the count is).  A request is done when
// all its packets are.
void credit_jobs(colt_ctx* ctx, int si, bool all) {
  Slot& sl = ctx->slots[si];
  const volatile unsigned long long* done = sl.lb.jdone_h;
  const double t = now_ms();
  for (size_t j = 0; j < sl.jobs.size(); ++j) {
    if (sl.credited[j]) continue;
    const auto& jp = sl.jobs[j];
    if (!all && done[j] < jp.second) continue;
    sl.credited[j] = 1;
    auto it = ctx->reqs.find(jp.first);
    if (it == ctx->reqs.end()) continue;
    Req& r = *it->second;
    r.done_packets += jp.second;
    if (r.done_packets >= r.target && r.state == kAdmitted) {
      r.state = kDone;
      r.t_done = t;
    }
  }
}

// Add a finished launch's device time and its cell and peel-off visits (the
// launch counters, copied back after the kernel) to the context's totals.
void account_launch(colt_ctx* ctx, Slot& sl) {
  if (!sl.timed) return;
  float ms = 0;
  if (cudaEventElapsedTime(&ms, sl.k0, sl.k1) == cudaSuccess) {
    ctx->kernel_ms += ms;
    ++ctx->timed_launches;
  }
  ctx->cell_visits += sl.lb.work_h[1 + kCellVisits];
  ctx->peel_visits += sl.lb.work_h[1 + kPeelVisits];
  sl.timed = false;
}

int complete_slot(colt_ctx* ctx, int si) {
  Slot& sl = ctx->slots[si];
  sl.in_flight = false;
  account_launch(ctx, sl);
  for (size_t j = 0; j < sl.jobs.size(); ++j) {
    auto it = ctx->reqs.find(sl.jobs[j].first);
    if (it == ctx->reqs.end()) continue;
    learn_cost(ctx, it->second->grid, sl.lb.jmax_h[j]);
    it->second->longest = std::max<uint64_t>(it->second->longest, sl.lb.jmax_h[j]);
  }
  credit_jobs(ctx, si, true);
  sl.jobs.clear();
  sl.credited.clear();
  return check_device_error(ctx, si);
}

// Wait for every in-flight launch (used before blocking calls).
int drain_slots(colt_ctx* ctx) {
  for (int si = 0; si < kSlots; ++si) {
    if (!ctx->slots[si].in_flight) continue;
    CU(cudaEventSynchronize(ctx->slots[si].done));
    int rc = complete_slot(ctx, si);
    if (rc) return rc;
  }
  return COLT_OK;
}

int serve_admit(colt_ctx* ctx) {
  int admitted = 0;
  while (!ctx->queue.empty()) {
    int active = 0;
    for (auto& kv : ctx->reqs) active += kv.second->state == kAdmitted;
    if (active >= kMaxJobs * kSlots) break;
    const uint64_t id = ctx->queue.front();
    auto it = ctx->reqs.find(id);
    if (it == ctx->reqs.end()) { ctx->queue.pop_front(); continue; }
    Req& r = *it->second;
    if (ctx->used + r.need_bytes > ctx->budget) break;   // FIFO: wait for memory
    int rc = alloc_tally(ctx, &r.p, false, &r.tally);
    if (rc) return rc;
    ctx->used += r.tally.bytes;
    attach_tally(&r.run, r.tally);
    r.state = kAdmitted;
    ctx->queue.pop_front();
    ++admitted;
  }
  if (admitted) CU(cudaEventRecord(ctx->ev_alloc, ctx->aux));
  return admitted;
}

// Host function behind every serving launch (runs on a CUDA driver thread,
// makes no CUDA calls).
void CUDART_CB slot_done_cb(void* arg) {
  colt_ctx* ctx = static_cast<colt_ctx*>(arg);
  {
    std::lock_guard<std::mutex> g(ctx->cv_mu);
    ++ctx->done_seq;
  }
  ctx->cv.notify_all();
}

// Build and enqueue one batched launch on a free slot over admitted requests
// with packets not yet handed out (oldest first), sharing a packet budget;
// all jobs of a launch share one precision.  Returns 1 if launched.
int serve_launch(colt_ctx* ctx, int si) {
  std::vector<Req*> act;
  for (auto& kv : ctx->reqs)
    if (kv.second->state == kAdmitted && kv.second->next_local < kv.second->target)
      act.push_back(kv.second.get());
  if (act.empty()) return 0;
  // requests passed over kMaxPassed times first (oldest first), then
  // longest-expected-first, then oldest first
  auto cost = [&](const Req* r) {
    auto g = ctx->grids.find(r->grid);
    return g == ctx->grids.end() ? 0ull : grid_cost(g->second);
  };
  std::sort(act.begin(), act.end(), [&](const Req* a, const Req* b) {
    const bool aa = a->passed >= kMaxPassed, ab = b->passed >= kMaxPassed;
    if (aa != ab) return aa;
    if (!aa) {
      const uint64_t ca = cost(a), cb = cost(b);
      if (ca != cb) return ca > cb;
    }
    return a->id < b->id;
  });
  // all jobs of a launch share one precision and one grid kind
  auto kind_of = [&](const Req* r) {
    auto g = ctx->grids.find(r->grid);
    return g == ctx->grids.end() ? COLT_CARTESIAN : g->second.dev.kind;
  };
  const int prec = act.front()->p.precision;
  const int kind = kind_of(act.front());
  std::vector<Req*> sel;
  for (Req* r : act)
    if (r->p.precision == prec && kind_of(r) == kind && (int)sel.size() < kMaxJobs) sel.push_back(r);
  int rc = ensure_slot(ctx, si);
  if (rc) return rc;
  Slot& sl = ctx->slots[si];
  LaunchBuf& lb = sl.lb;
  uint64_t left = kStepPackets;
  unsigned long long total = 0;
  int nj = 0;
  bool extras = false;
  sl.jobs.clear();
  sl.credited.clear();
  for (size_t i = 0; i < sel.size() && left > 0; ++i) {
    Req* r = sel[i];
    const uint64_t rem = r->target - r->next_local;
    const uint64_t fair = std::max<uint64_t>(1, left / (sel.size() - i));
    const uint64_t take = std::min<uint64_t>(rem, std::max<uint64_t>(fair, std::min<uint64_t>(rem, left)));
    if (take == 0) continue;
    const GridObj& g = ctx->grids.at(r->grid);
    Job& J = lb.jobs_h()[nj];
    J.g = g.dev;
    J.p = r->run;
    J.p.n_packets = take;
    J.p.pid_offset = r->run.pid_offset + r->next_local;
    extras = extras || run_needs_extras(J.p);
    total += take;
    lb.end_h()[nj] = total;
    r->next_local += take;
    sl.jobs.push_back({r->id, take});
    sl.credited.push_back(0);
    left = left > take ? left - take : 0;
    ++nj;
  }
  if (nj == 0) return 0;
  for (Req* r : act)
    if (std::none_of(sl.jobs.begin(), sl.jobs.end(), [&](const std::pair<uint64_t, uint64_t>& j) {
          return j.first == r->id;
        }))
      ++r->passed;
  LaunchDev* h = lb.hdr_h();
  h->n_jobs = nj;
  h->total = total;
  // served requests complete with their own packets: count them per job
  h->job_done = lb.jdone_d;
  // tallies were allocated and zeroed on the context stream
  CU(cudaStreamWaitEvent(sl.stream, ctx->ev_alloc, 0));
  rc = enqueue_launch(ctx, si, prec, kind, 0, extras);
  if (rc) return rc;
  CU(cudaLaunchHostFunc(sl.stream, slot_done_cb, ctx));
  CU(cudaEventRecord(sl.done, sl.stream));
  sl.in_flight = true;
  return 1;
}

// Advance the scheduler without blocking on the device.
int serve_pump(colt_ctx* ctx) {
  for (int si = 0; si < kSlots; ++si) {
    Slot& sl = ctx->slots[si];
    if (!sl.in_flight) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) {
      credit_jobs(ctx, si, false);
      continue;
    }
    if (q != cudaSuccess) return cuda_fail(ctx, q, "serving launch");
    int rc = complete_slot(ctx, si);
    if (rc) return rc;
  }
  int rc = serve_admit(ctx);
  if (rc < 0) return rc;
  for (int si = 0; si < kSlots; ++si) {
    if (ctx->slots[si].in_flight) continue;
    rc = serve_launch(ctx, si);
    if (rc < 0) return rc;
    if (rc == 0) break;
  }
  return COLT_OK;
}

}  // namespace

// ====================================================================== ABI ==
extern "C" {

int colt_init(colt_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream) {
  if (!out) return COLT_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0 || device < 0 || device >= n) return COLT_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return COLT_ECUDA;
  auto* ctx = new colt_ctx();
  ctx->device = device;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete ctx; return COLT_ECUDA; }
  ctx->sm_count = prop.multiProcessorCount;
  ctx->l2 = prop.l2CacheSize;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.9 * (double)fr);
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return COLT_ECUDA; }
    ctx->own_stream = true;
  }
  // keep freed tally blocks cached in the device's default pool
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return COLT_ECUDA;
  }
  cudaEventCreate(&ctx->ev0);
  cudaEventCreate(&ctx->ev1);
  cudaEventCreateWithFlags(&ctx->ev_alloc, cudaEventDisableTiming);
  *out = ctx;
  return COLT_OK;
}

void colt_finalize(colt_ctx* ctx) {
  if (!ctx) return;
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    for (auto& sl : ctx->slots)
      if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaStreamSynchronize(ctx->stream);
    cudaStreamSynchronize(ctx->aux);
    for (auto& kv : ctx->reqs) free_tally(&kv.second->tally);
    for (auto& kv : ctx->grids) free_grid(kv.second);
    cudaStreamSynchronize(ctx->aux);
    cudaStreamSynchronize(ctx->stream);
    for (auto& sl : ctx->slots) {
      for (auto& gp : sl.graph)
        for (auto& g : gp) if (g) cudaGraphExecDestroy(g);
      if (sl.lb.host) cudaFreeHost(sl.lb.host);
      if (sl.lb.dev) cudaFree(sl.lb.dev);
      if (sl.lb.work) cudaFree(sl.lb.work);
      if (sl.lb.work_h) cudaFreeHost(sl.lb.work_h);
      if (sl.lb.jdone_h) cudaFreeHost(sl.lb.jdone_h);
      if (sl.lb.error) cudaFree(sl.lb.error);
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.k0) cudaEventDestroy(sl.k0);
      if (sl.k1) cudaEventDestroy(sl.k1);
      if (sl.own_stream) cudaStreamDestroy(sl.stream);
    }
    cudaEventDestroy(ctx->ev0);
    cudaEventDestroy(ctx->ev1);
    cudaEventDestroy(ctx->ev_alloc);
    cudaStreamDestroy(ctx->aux);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
}

const char* colt_last_error(colt_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int colt_device_info(colt_ctx* ctx, int* sm_count, size_t* l2_bytes, int* cc_major, int* cc_minor) {
  if (!ctx) return COLT_EINVAL;
  if (sm_count) *sm_count = ctx->sm_count;
  if (l2_bytes) *l2_bytes = ctx->l2;
  if (cc_major) *cc_major = ctx->cc_major;
  if (cc_minor) *cc_minor = ctx->cc_minor;
  return COLT_OK;
}

int colt_create_grid(colt_ctx* ctx, const colt_grid_desc* desc, colt_grid* out) {
  if (!ctx || !out) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  GridObj g;
  int rc = build_grid(ctx, desc, &g);
  if (rc) {
    cudaStreamSynchronize(ctx->aux);
    free_grid(g);
    return rc;
  }
  const uint64_t h = ctx->next_handle++;
  ctx->grids[h] = g;
  ctx->used += g.bytes;
  *out = h;
  return COLT_OK;
}

int colt_destroy_grid(colt_ctx* ctx, colt_grid grid) {
  if (!ctx) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->grids.find(grid);
  if (it == ctx->grids.end()) return fail(ctx, COLT_ENOTFOUND, "unknown grid");
  for (auto& kv : ctx->reqs)
    if (kv.second->grid == grid && kv.second->state != kDone)
      return fail(ctx, COLT_EINVAL, "grid is in use by an unfinished request");
  cudaStreamSynchronize(ctx->aux);
  free_grid(it->second);
  ctx->used -= it->second.bytes;
  ctx->grids.erase(it);
  return COLT_OK;
}

int colt_read_cells(colt_ctx* ctx, colt_grid grid, float* out, size_t n_floats) {
  if (!ctx || !out) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->grids.find(grid);
  if (it == ctx->grids.end()) return fail(ctx, COLT_ENOTFOUND, "unknown grid");
  if (n_floats != 8 * (size_t)it->second.dev.n_cells) return fail(ctx, COLT_EINVAL, "n_floats must be 8 * n_cells");
  CU(cudaMemcpyAsync(out, it->second.rec, sizeof(float) * n_floats, cudaMemcpyDeviceToHost, ctx->aux));
  CU(cudaStreamSynchronize(ctx->aux));
  return COLT_OK;
}

int colt_set_cell_luminosity(colt_ctx* ctx, colt_grid grid, const double* lum, int mem) {
  if (!ctx || !lum) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  auto it = ctx->grids.find(grid);
  if (it == ctx->grids.end()) return fail(ctx, COLT_ENOTFOUND, "unknown grid");
  if (mem != COLT_MEM_HOST && mem != COLT_MEM_DEVICE) return fail(ctx, COLT_EINVAL, "bad mem");
  for (auto& kv : ctx->reqs)
    if (kv.second->grid == grid && kv.second->state != kDone)
      return fail(ctx, COLT_EINVAL, "grid is in use by an unfinished request");
  GridObj& g = it->second;
  const int64_t n = g.dev.n_cells;
  const bool oct = g.dev.kind == COLT_OCTREE;
  std::vector<double> hl;
  const double* L = lum;
  if (mem == COLT_MEM_DEVICE) {
    hl.resize(n);
    CU(cudaMemcpyAsync(hl.data(), lum, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->aux));
    CU(cudaStreamSynchronize(ctx->aux));
    L = hl.data();
  }
  // integer weights w_c = floor(2^s lum_c / max lum), s = 63 - ceil(log2(n + 1)):
  // their sum stays below 2^63 and the prefix sums are exact in any order
  double lmax = 0.0;
  for (int64_t c = 0; c < n; ++c) {
    if (!(L[c] >= 0) || !std::isfinite(L[c])) return fail(ctx, COLT_EINVAL, "cell luminosities must be finite and >= 0");
    lmax = std::max(lmax, L[c]);
  }
  if (!(lmax > 0)) return fail(ctx, COLT_EINVAL, "no cell has a positive luminosity");
  int bits = 0;
  while (bits < 63 && ((uint64_t)1 << bits) < (uint64_t)n + 1) ++bits;
  const int s = 63 - bits;
  std::vector<unsigned long long> cum(n);
  unsigned long long acc = 0;
  for (int64_t c = 0; c < n; ++c) {
    acc += (unsigned long long)std::floor(std::ldexp(L[c] / lmax, s));
    cum[c] = acc;
  }
  const size_t bytes = sizeof(unsigned long long) * (size_t)n + (oct ? sizeof(uint32_t) * 3 * (size_t)n : 0);
  if (ctx->used - g.lum_bytes + bytes > ctx->budget) return fail(ctx, COLT_ENOMEM, "luminosity table exceeds the memory budget");
  std::vector<uint32_t> loc;
  if (oct) {
    loc.resize(3 * (size_t)n);
    for (int64_t c = 0; c < n; ++c) {
      loc[3 * c] = g.leaf_ijk[3 * c] | ((uint32_t)g.leaf_level[c] << 24);
      loc[3 * c + 1] = g.leaf_ijk[3 * c + 1];
      loc[3 * c + 2] = g.leaf_ijk[3 * c + 2];
    }
  }
  // the new table is complete on the device before the old one is released,
  // so a failure leaves the grid as it was
  unsigned long long* cum_d = nullptr;
  uint32_t* loc_d = nullptr;
  auto release_new = [&]() {
    if (cum_d) cudaFree(cum_d);
    if (loc_d) cudaFree(loc_d);
  };
  cudaError_t e = cudaMalloc(&cum_d, sizeof(unsigned long long) * (size_t)n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cum_d, cum.data(), sizeof(unsigned long long) * (size_t)n, cudaMemcpyHostToDevice, ctx->aux);
  if (e == cudaSuccess && oct) e = cudaMalloc(&loc_d, sizeof(uint32_t) * 3 * (size_t)n);
  if (e == cudaSuccess && oct)
    e = cudaMemcpyAsync(loc_d, loc.data(), sizeof(uint32_t) * 3 * (size_t)n, cudaMemcpyHostToDevice, ctx->aux);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->aux);
  if (e != cudaSuccess) {
    release_new();
    return cuda_fail(ctx, e, "luminosity table");
  }
  if (g.lum_cum) cudaFree(g.lum_cum);
  if (g.leaf_loc) cudaFree(g.leaf_loc);
  ctx->used -= g.lum_bytes;
  g.bytes -= g.lum_bytes;
  g.lum_cum = cum_d;
  g.leaf_loc = loc_d;
  g.dev.lum_cum = g.lum_cum;
  g.dev.leaf_loc = g.leaf_loc;
  g.dev.lum_total = acc;
  g.lum_bytes = bytes;
  g.bytes += bytes;
  ctx->used += bytes;
  return COLT_OK;
}

int colt_run_batch(colt_ctx* ctx, int n, const colt_grid* grids, const colt_run_params* params,
                   colt_result* out) {
  if (!ctx || !grids || !params || !out || n < 1 || n > kMaxJobs) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const int prec = params[0].precision;
  std::vector<const GridObj*> gs(n);
  int kind = COLT_CARTESIAN;
  for (int i = 0; i < n; ++i) {
    auto it = ctx->grids.find(grids[i]);
    if (it == ctx->grids.end()) return fail(ctx, COLT_ENOTFOUND, "unknown grid");
    gs[i] = &it->second;
    int rc = validate_params(ctx, &params[i], *gs[i]);
    if (rc) return rc;
    if (params[i].precision != prec) return fail(ctx, COLT_EINVAL, "all solves of a batch need one precision");
    if (gs[i]->dev.kind != gs[0]->dev.kind) return fail(ctx, COLT_EINVAL, "all solves of a batch need one grid kind");
  }
  kind = gs[0]->dev.kind;
  // a blocking run waits for in-flight serving launches first
  int rc = drain_slots(ctx);
  if (rc) return rc;
  std::vector<bool> per_packet(n);
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    per_packet[i] = out[i].pk_status || out[i].pk_nscat || out[i].pk_freq;
    need += tally_bytes(&params[i], per_packet[i]) + 256;
  }
  if (ctx->used + need > ctx->budget) return fail(ctx, COLT_ENOMEM, "tallies exceed the memory budget");
  std::vector<Tally> ts(n);
  auto free_all = [&]() { for (auto& t : ts) free_tally(&t); };
  rc = ensure_slot(ctx, 0);
  if (rc) return rc;
  LaunchBuf& lb = ctx->slots[0].lb;
  // job table in longest-expected-first order; results stay indexed by i
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return grid_cost(*gs[a]) > grid_cost(*gs[b]); });
  unsigned long long total = 0;
  bool extras = false;
  for (int q = 0; q < n; ++q) {
    const int i = ord[q];
    rc = alloc_tally(ctx, &params[i], per_packet[i], &ts[i]);
    if (rc) { free_all(); return rc; }
    Job& J = lb.jobs_h()[q];
    J.g = gs[i]->dev;
    J.p = make_run(*gs[i], &params[i]);
    extras = extras || run_needs_extras(J.p);
    attach_tally(&J.p, ts[i]);
    total += params[i].n_packets;
    lb.end_h()[q] = total;
  }
  LaunchDev* h = lb.hdr_h();
  h->n_jobs = n;
  h->total = total;
  h->job_done = nullptr;     // a blocking run completes with its launch
  unsigned long long lcnt[kNumLaunchCounters] = {0, 0, 0};
  float ms = 0;
  // the tallies were set up on the auxiliary stream
  CU(cudaEventRecord(ctx->ev_alloc, ctx->aux));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_alloc, 0));
  if (total > 0) {
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    rc = enqueue_launch(ctx, 0, prec, kind, params[0].blocks_per_sm, extras);
    if (rc) { free_all(); return rc; }
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    CU(cudaMemcpyAsync(lcnt, lb.work + 1, sizeof(lcnt), cudaMemcpyDeviceToHost, ctx->stream));
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    if (se != cudaSuccess) { free_all(); return cuda_fail(ctx, se, "transport kernel"); }
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  }
  if (total > 0) account_launch(ctx, ctx->slots[0]);
  rc = check_device_error(ctx, 0);
  if (total > 0 && !rc)
    for (int q = 0; q < n; ++q) learn_cost(ctx, grids[ord[q]], lb.jmax_h[q]);
  for (int i = 0; i < n && !rc; ++i) {
    rc = copy_result(ctx, &params[i], ts[i], &out[i], per_packet[i]);
    out[i].kernel_ms = ms;
    out[i].n_cell_visits = lcnt[kCellVisits];
    out[i].n_peel_visits = lcnt[kPeelVisits];
    out[i].n_peel_rays = lcnt[kPeelRays];
  }
  free_all();
  return rc;
}

int colt_run(colt_ctx* ctx, colt_grid grid, const colt_run_params* p, colt_result* out) {
  if (!ctx || !out || !p) return COLT_EINVAL;
  return colt_run_batch(ctx, 1, &grid, p, out);
}

int colt_autotune(colt_ctx* ctx, colt_grid grid, const colt_run_params* params, colt_launch_config* out) {
  if (!ctx || !params) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  auto it = ctx->grids.find(grid);
  if (it == ctx->grids.end()) return fail(ctx, COLT_ENOTFOUND, "unknown grid");
  int rc = validate_params(ctx, params, it->second);
  if (rc) return rc;
  const int prec = params->precision;
  const int kind = it->second.dev.kind;
  const int gi = prec == COLT_PLAIN ? 0 : 1, gk = kind == COLT_OCTREE ? 1 : 0;
  // calibration: the request itself (at most 2^20 packets, no images), once
  // per configuration on the same packet ids.  Both what the configuration
  // trades -- throughput of full warps and the latency of the last, longest
  // histories -- enter its time, so a heavy-tailed workload is tuned for its
  // tail and a uniform one for throughput.
  colt_run_params q = *params;
  std::vector<colt_camera> cams(params->cams, params->cams + params->n_cam);
  for (auto& c : cams) c.npix = 0;
  q.cams = cams.data();
  q.blocks_per_sm = 0;
  q.n_packets = std::min<uint64_t>(q.n_packets, 1ull << 20);
  std::vector<uint64_t> spec(q.spec_nbins);
  std::vector<double> cs((size_t)std::max(1, q.n_cam) * q.cam_nbins), cs2(cs.size());
  auto time_cfg = [&](const colt_launch_config& c, double* rate) -> int {
    ctx->cfg[gi][gk] = c;
    colt_result r{};
    r.spec = spec.data();
    if (q.n_cam > 0) {
      r.cam_spec = cs.data();
      r.cam_spec2 = cs2.data();
    }
    const int e = colt_run_batch(ctx, 1, &grid, &q, &r);
    if (e) {
      ctx->cfg[gi][gk] = colt_launch_config{0, 0, 0.0, 8, 1};
      return e;
    }
    *rate = r.kernel_ms > 0 ? (double)r.n_scat / (r.kernel_ms * 1e-3) : 0.0;
    return COLT_OK;
  };
  colt_launch_config best{0, 0, -1.0, 8, 1};
  // 1. register variant x resident CTAs per SM (8 warps, refill every round)
  for (int v = 0; v < transport_variants(prec); ++v) {
    const int occ = transport_occupancy(prec, kind, v, 8);
    for (int b = occ; b >= std::max(1, occ - 1); --b) {
      double rate = 0.0;
      rc = time_cfg(colt_launch_config{v, b, 0.0, 8, 1}, &rate);
      if (rc) return rc;
      if (rate > best.scatterings_per_s) best = colt_launch_config{v, b, rate, 8, 1};
    }
  }
  // 2. warps per CTA, at the most CTAs per SM that fit
  for (int w : {4, 16}) {
    if (!transport_has_warps(prec, best.variant, w)) continue;
    const int occ = transport_occupancy(prec, kind, best.variant, w);
    double rate = 0.0;
    rc = time_cfg(colt_launch_config{best.variant, occ, 0.0, w, 1}, &rate);
    if (rc) return rc;
    if (rate > best.scatterings_per_s) best = colt_launch_config{best.variant, occ, rate, w, 1};
  }
  // 3. refill threshold
  for (int m : {4, 12}) {
    double rate = 0.0;
    colt_launch_config c = best;
    c.refill_min = m;
    rc = time_cfg(c, &rate);
    if (rc) return rc;
    if (rate > best.scatterings_per_s) {
      best = c;
      best.scatterings_per_s = rate;
    }
  }
  ctx->cfg[gi][gk] = best;
  if (out) *out = best;
  return COLT_OK;
}

int colt_set_launch_config(colt_ctx* ctx, int precision, int kind, const colt_launch_config* cfg) {
  if (!ctx || !cfg) return COLT_EINVAL;
  if (precision != COLT_PLAIN && precision != COLT_MIXED) return fail(ctx, COLT_EINVAL, "bad precision");
  if (kind != COLT_CARTESIAN && kind != COLT_OCTREE) return fail(ctx, COLT_EINVAL, "bad grid kind");
  const int w = cfg->warps_per_block > 0 ? cfg->warps_per_block : 8;
  if (cfg->variant < 0 || cfg->variant >= transport_variants(precision) || !transport_has_warps(precision, cfg->variant, w))
    return fail(ctx, COLT_EINVAL, "this build has no such kernel variant / block size");
  if (cfg->blocks_per_sm < 0 || cfg->refill_min < 0 || cfg->refill_min > 32)
    return fail(ctx, COLT_EINVAL, "bad blocks_per_sm or refill_min");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  colt_launch_config c = *cfg;
  c.warps_per_block = w;
  c.refill_min = std::max(1, cfg->refill_min);
  ctx->cfg[precision == COLT_PLAIN ? 0 : 1][kind == COLT_OCTREE ? 1 : 0] = c;
  return COLT_OK;
}

int colt_solve(colt_ctx* ctx, const colt_grid_desc* desc, const colt_run_params* p, colt_result* out) {
  if (!ctx) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  colt_grid g = 0;
  int rc = colt_create_grid(ctx, desc, &g);
  if (rc) return rc;
  rc = colt_run(ctx, g, p, out);
  colt_destroy_grid(ctx, g);
  return rc;
}

// A request that colt_submit would queue (the grid exists, the parameters are
// valid, the request fits the memory budget alone); its tally bytes in *need.
static int check_request(colt_ctx* ctx, colt_grid grid, const colt_run_params* p, size_t* need) {
  if (!p) return COLT_EINVAL;
  auto it = ctx->grids.find(grid);
  if (it == ctx->grids.end()) return fail(ctx, COLT_ENOTFOUND, "unknown grid");
  int rc = validate_params(ctx, p, it->second);
  if (rc) return rc;
  *need = tally_bytes(p, false) + 256;
  size_t grids_bytes = 0;
  for (auto& kv : ctx->grids) grids_bytes += kv.second.bytes;
  if (grids_bytes + *need > ctx->budget)
    return fail(ctx, COLT_ENOMEM, "request can never fit in the memory budget");
  return COLT_OK;
}

// Queue a checked request (no scheduling step); returns its handle.
static colt_req enqueue_request(colt_ctx* ctx, colt_grid grid, const colt_run_params* p, size_t need) {
  auto r = std::make_unique<Req>();
  r->id = ctx->next_handle++;
  r->grid = grid;
  r->p = *p;
  r->cams.assign(p->cams, p->cams + p->n_cam);
  r->p.cams = r->cams.data();
  if (p->n_sources > 0) r->srcs.assign(p->sources, p->sources + p->n_sources);
  r->p.sources = r->srcs.data();
  r->need_bytes = need;
  r->run = make_run(ctx->grids.at(grid), &r->p);
  r->target = r->p.n_packets;
  r->t_submit = now_ms();
  if (r->p.n_packets == 0) {
    r->state = kDone;
    r->t_done = r->t_submit;
  } else {
    ctx->queue.push_back(r->id);
  }
  const colt_req id = r->id;
  ctx->reqs[id] = std::move(r);
  return id;
}

int colt_submit(colt_ctx* ctx, colt_grid grid, const colt_run_params* p, colt_req* out) {
  if (!ctx || !out) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  size_t need = 0;
  int rc = check_request(ctx, grid, p, &need);
  if (rc) return rc;
  if (ctx->queue.size() >= kMaxQueued) return fail(ctx, COLT_EAGAIN, "request queue full");
  *out = enqueue_request(ctx, grid, p, need);
  return serve_pump(ctx);
}

int colt_submit_many(colt_ctx* ctx, int n, const colt_grid* grids, const colt_run_params* params,
                     colt_req* out) {
  if (!ctx || n < 0 || (n > 0 && (!grids || !params || !out))) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  // every request is checked before any is queued: all or none
  std::vector<size_t> need(n);
  for (int i = 0; i < n; ++i) {
    int rc = check_request(ctx, grids[i], params + i, &need[i]);
    if (rc) return rc;
  }
  if (ctx->queue.size() + (size_t)n > kMaxQueued) return fail(ctx, COLT_EAGAIN, "request queue full");
  for (int i = 0; i < n; ++i) out[i] = enqueue_request(ctx, grids[i], params + i, need[i]);
  // one scheduling step for the whole batch: the requests share launches
  return serve_pump(ctx);
}

int colt_poll(colt_ctx* ctx, colt_req req, int* done, colt_stats* st) {
  if (!ctx) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  int rc = serve_pump(ctx);
  if (rc) return rc;
  auto it = ctx->reqs.find(req);
  if (it == ctx->reqs.end()) return fail(ctx, COLT_ENOTFOUND, "unknown request");
  const Req& r = *it->second;
  if (done) *done = r.state == kDone;
  if (st) {
    st->done = r.state == kDone;
    st->admitted = r.state != kQueued;
    st->packets_done = r.done_packets;
    st->packets_total = r.p.n_packets;
    st->submit_to_done_ms = r.state == kDone ? r.t_done - r.t_submit : 0.0;
    st->ctx_launches = ctx->launches;
    st->cancelled = r.cancelled ? 1 : 0;
    st->ctx_timed_launches = ctx->timed_launches;
    st->ctx_kernel_ms = ctx->kernel_ms;
    st->longest_history = r.longest;
    st->ctx_cell_visits = ctx->cell_visits;
    st->ctx_peel_visits = ctx->peel_visits;
  }
  return COLT_OK;
}

int colt_cancel(colt_ctx* ctx, colt_req req) {
  if (!ctx) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->reqs.find(req);
  if (it == ctx->reqs.end()) return fail(ctx, COLT_ENOTFOUND, "unknown request");
  Req& r = *it->second;
  if (r.state == kDone) return COLT_OK;
  r.cancelled = true;
  if (r.state == kQueued) {
    // never admitted: no tallies, nothing on the device
    ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), req), ctx->queue.end());
    r.target = 0;
    r.state = kDone;
    r.t_done = now_ms();
    return COLT_OK;
  }
  // admitted: packets already handed to launches finish; no more start
  r.target = r.next_local;
  if (r.done_packets >= r.target) {
    r.state = kDone;
    r.t_done = now_ms();
  }
  return COLT_OK;
}

int colt_wait(colt_ctx* ctx, colt_req req, double timeout_ms) {
  if (!ctx) return COLT_EINVAL;
  const double t0 = now_ms();
  for (;;) {
    uint64_t seq;
    {
      std::lock_guard<std::mutex> g(ctx->cv_mu);
      seq = ctx->done_seq;
    }
    {
      std::lock_guard<std::recursive_mutex> lk(ctx->mu);
      int done = 0;
      int rc = colt_poll(ctx, req, &done, nullptr);
      if (rc) return rc;
      if (done) return COLT_OK;
    }
    // re-poll at least this often: a request can finish inside a running
    // launch (its own packets done), and a queued one may wait on memory
    double wait_ms = 1.0;
    if (timeout_ms >= 0) {
      const double left = timeout_ms - (now_ms() - t0);
      if (left <= 0) return fail(ctx, COLT_ETIMEOUT, "colt_wait timed out");
      wait_ms = std::min(wait_ms, left);
    }
    // sleep until any in-flight launch finishes (its host function bumps done_seq)
    std::unique_lock<std::mutex> l(ctx->cv_mu);
    ctx->cv.wait_for(l, std::chrono::duration<double, std::milli>(wait_ms),
                     [&] { return ctx->done_seq != seq; });
  }
}

int colt_read_result(colt_ctx* ctx, colt_req req, colt_result* out) {
  if (!ctx || !out) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->reqs.find(req);
  if (it == ctx->reqs.end()) return fail(ctx, COLT_ENOTFOUND, "unknown request");
  Req& r = *it->second;
  if (r.state != kDone) return fail(ctx, COLT_EAGAIN, "request not done");
  if (!r.tally.block) {  // zero-packet request
    uint64_t* spec = out->spec;
    *out = colt_result{};
    if (spec) {
      std::memset(spec, 0, sizeof(uint64_t) * r.p.spec_nbins);
      out->spec = spec;
    }
    return COLT_OK;
  }
  out->pk_status = nullptr;
  out->pk_nscat = nullptr;
  out->pk_freq = nullptr;
  int rc = copy_result(ctx, &r.p, r.tally, out, false);
  out->kernel_ms = 0;
  out->n_cell_visits = out->n_peel_visits = out->n_peel_rays = 0;
  return rc;
}

int colt_read_spectrum(colt_ctx* ctx, colt_req req, int camera, double* buf, size_t nbins) {
  if (!ctx || !buf) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->reqs.find(req);
  if (it == ctx->reqs.end()) return fail(ctx, COLT_ENOTFOUND, "unknown request");
  Req& r = *it->second;
  if (r.state != kDone) return fail(ctx, COLT_EAGAIN, "request not done");
  if (camera < -1 || camera >= r.p.n_cam) return fail(ctx, COLT_EINVAL, "bad camera index");
  if (camera == -1) {
    if (nbins != (size_t)r.p.spec_nbins) return fail(ctx, COLT_EINVAL, "nbins mismatch");
    std::vector<uint64_t> h(nbins, 0);
    if (r.tally.block) {
      CU(cudaMemcpyAsync(h.data(), r.tally.spec, sizeof(uint64_t) * nbins, cudaMemcpyDeviceToHost, ctx->aux));
      CU(cudaStreamSynchronize(ctx->aux));
    }
    for (size_t i = 0; i < nbins; ++i) buf[i] = (double)h[i];
  } else {
    if (nbins != (size_t)r.p.cam_nbins) return fail(ctx, COLT_EINVAL, "nbins mismatch");
    if (!r.tally.block) { std::memset(buf, 0, sizeof(double) * nbins); return COLT_OK; }
    CU(cudaMemcpyAsync(buf, r.tally.cam_spec + (size_t)camera * r.p.cam_nbins, sizeof(double) * nbins,
                       cudaMemcpyDeviceToHost, ctx->aux));
    CU(cudaStreamSynchronize(ctx->aux));
  }
  return COLT_OK;
}

int colt_read_image(colt_ctx* ctx, colt_req req, int camera, double* buf, size_t n) {
  if (!ctx || !buf) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->reqs.find(req);
  if (it == ctx->reqs.end()) return fail(ctx, COLT_ENOTFOUND, "unknown request");
  Req& r = *it->second;
  if (r.state != kDone) return fail(ctx, COLT_EAGAIN, "request not done");
  if (camera < 0 || camera >= r.p.n_cam) return fail(ctx, COLT_EINVAL, "bad camera index");
  const int np = r.p.cams[camera].npix;
  if (np <= 0) return fail(ctx, COLT_EINVAL, "camera has no image");
  if (n != (size_t)np * np * r.p.cam_nbins) return fail(ctx, COLT_EINVAL, "image size mismatch");
  if (!r.tally.block || !r.tally.cam_image) { std::memset(buf, 0, sizeof(double) * n); return COLT_OK; }
  CU(cudaMemcpyAsync(buf, r.tally.cam_image + r.run.cam[camera].img_off, sizeof(double) * n, cudaMemcpyDeviceToHost,
                     ctx->aux));
  CU(cudaStreamSynchronize(ctx->aux));
  return COLT_OK;
}

int colt_release(colt_ctx* ctx, colt_req req) {
  if (!ctx) return COLT_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto it = ctx->reqs.find(req);
  if (it == ctx->reqs.end()) return fail(ctx, COLT_ENOTFOUND, "unknown request");
  Req& r = *it->second;
  if (r.state == kAdmitted) return fail(ctx, COLT_EAGAIN, "request still running");
  if (r.state == kQueued) {
    ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), req), ctx->queue.end());
  }
  if (r.tally.block) {
    ctx->used -= r.tally.bytes;
    free_tally(&r.tally);
  }
  ctx->reqs.erase(it);
  return COLT_OK;
}

int colt_voigt(colt_ctx* ctx, const void* a, const void* x, void* H, size_t n, int precision, int mem) {
  if (!ctx || (n && (!a || !x || !H))) return COLT_EINVAL;
  if (precision != COLT_PLAIN && precision != COLT_MIXED) return fail(ctx, COLT_EINVAL, "bad precision");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const size_t es = precision == COLT_PLAIN ? sizeof(double) : sizeof(float);
  if (mem == COLT_MEM_DEVICE) {
    CU(launch_voigt(a, x, H, n, precision, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return COLT_OK;
  }
  void *da = nullptr, *dx = nullptr, *dh = nullptr;
  CU(cudaMallocAsync(&da, es * n + 1, ctx->stream));
  CU(cudaMallocAsync(&dx, es * n + 1, ctx->stream));
  CU(cudaMallocAsync(&dh, es * n + 1, ctx->stream));
  cudaMemcpyAsync(da, a, es * n, cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(dx, x, es * n, cudaMemcpyHostToDevice, ctx->stream);
  cudaError_t e = launch_voigt(da, dx, dh, n, precision, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(H, dh, es * n, cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(da, ctx->stream);
  cudaFreeAsync(dx, ctx->stream);
  cudaFreeAsync(dh, ctx->stream);
  cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "voigt kernel");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "voigt sync");
  return COLT_OK;
}

int colt_scatter(colt_ctx* ctx, colt_scatter_io* io, size_t n, uint64_t seed, int precision) {
  if (!ctx || (n && !io)) return COLT_EINVAL;
  if (precision != COLT_PLAIN && precision != COLT_MIXED) return fail(ctx, COLT_EINVAL, "bad precision");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  if (n == 0) return COLT_OK;
  void* d = nullptr;
  CU(cudaMallocAsync(&d, sizeof(colt_scatter_io) * n, ctx->stream));
  cudaMemcpyAsync(d, io, sizeof(colt_scatter_io) * n, cudaMemcpyHostToDevice, ctx->stream);
  cudaError_t e = launch_scatter(d, n, seed, precision, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(io, d, sizeof(colt_scatter_io) * n, cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(d, ctx->stream);
  cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scatter kernel");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "scatter sync");
  return COLT_OK;
}

}  // extern "C"
