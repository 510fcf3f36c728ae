// C ABI of the chemistry library: handles, argument checks, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/rde_chem.h"
#include "../../include/rde_chem_selftest.h"
#include "chem_launch.h"
#include "fastmath.cuh"
#include "jit.h"
#include "mech_host.h"

struct rde_mech_s {
  int device = 0;
  int K = 0, R = 0;
  int num_sms = 0;
  unsigned char* d_mech = nullptr;
  int mech_bytes = 0;
  int fit = 1;  // queue CTAs per SM
  bool small_ok = false;    // a thread-per-cell kernel serves K (generic or specialised)
  bool generic_ok = false;  // a precompiled thread-per-cell kernel exists for K
  bool jit_ok = false;      // kernels specialised to this mechanism are loaded
  rde::JitKernels jit;
  bool jit_adj_tried = false, jit_adj_ok = false;   // specialised adjoint kernels (built on first use)
  rde::JitAdjKernels jadj;
  bool jit_ros2_tried = false, jit_ros2_ok = false; // specialised ROS2 kernels (built when selected)
  bool large_adj_tried = false, large_adj_ok = false;  // CTA-per-cell adjoint (set up on first use)
  rde::JitKernels jit_ros2;
  bool jit_extrap_tried = false, jit_extrap_ok = false;  // specialised extrapolation kernels
  rde::JitKernels jit_extrap;
  double* d_jscratch = nullptr;   // the extrapolation method's Jacobian scratch (allocated when selected)
  int jscratch_ctas = 0;
  bool jit_wide_tried = false;    // the wide queue kernel (built on the first call that asks for it)
  double* d_park = nullptr;       // its park area: [4 (K+1)][park_lanes]
  long long park_lanes = 0;
  bool large_ok = false;    // the CTA-per-cell kernel fits this mechanism
  int large_fit = 1;        // its CTAs per SM
  size_t plan_offset = 0;   // gather plan behind the image in d_mech
  std::vector<unsigned char> image;  // host copy of the device tables
  std::vector<double> E_J;           // activation energies as given (J/mol)
  // device scratch: [0] work-queue counter, [1..8) statistics
  unsigned long long* d_scratch = nullptr;
  rde_chem_options opt{};
};

namespace {

thread_local std::string g_msg;

int fail(int code, const std::string& msg) {
  g_msg = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(RDE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

int check_options(const rde_chem_options* o) {
  if (!(o->rtol > 0) || !(o->atol >= 0) || !(o->h_min > 0) || !(o->facmin > 0) || !(o->facmin <= 1) ||
      !(o->facmax >= 1) || !(o->safety > 0) || !(o->safety <= 1) || o->max_substeps < 1 ||
      !std::isfinite(o->rtol) || !std::isfinite(o->atol) || !std::isfinite(o->facmax))
    return fail(RDE_ERR_ARG, "invalid integrator options");
  if (o->method != RDE_METHOD_RODAS3 && o->method != RDE_METHOD_ROS2 && o->method != RDE_METHOD_EXTRAP)
    return fail(RDE_ERR_ARG, "unknown method");
  return RDE_OK;
}

int check_block(const rde_block& b, int K) {
  if (b.n < 0) return fail(RDE_ERR_ARG, "n_cells < 0");
  if (b.n == 0) return RDE_OK;
  if (!b.p || !b.T || !b.Y) return fail(RDE_ERR_NULL, "p, T and Y are required");
  if (b.ldY < b.n) return fail(RDE_ERR_ARG, "ldY < n_cells");
  const void* ptrs[] = {b.p, b.T, b.Y, b.h_hint};
  for (const void* q : ptrs)
    if (q && !aligned8(q)) return fail(RDE_ERR_ALIGN, "double arrays must be 8-byte aligned");
  if (b.cycles && !aligned8(b.cycles)) return fail(RDE_ERR_ALIGN, "cycles must be 8-byte aligned");
  const void* iptrs[] = {b.status, b.n_acc, b.n_rej};
  for (const void* q : iptrs)
    if (q && (reinterpret_cast<uintptr_t>(q) & 3u)) return fail(RDE_ERR_ALIGN, "int32 arrays must be 4-byte aligned");
  (void)K;
  return RDE_OK;
}

}  // namespace

// ---- allocation-free variant: scratch in a static device array ----------------
// The queue counter (word 0) and the statistics (words 1..7) of a no-alloc call.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[RDE_NOALLOC_SCRATCH_BYTES / 8];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned long long* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per device.
int noalloc_scratch(int dev, unsigned long long** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(RDE_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return RDE_OK;
}

}  // namespace

extern "C" {

const char* rde_strerror(int code) {
  switch (code) {
    case RDE_OK: return "success";
    case RDE_ERR_NULL: return "required pointer is NULL";
    case RDE_ERR_ARG: return "invalid argument";
    case RDE_ERR_PARSE: return "mechanism text malformed";
    case RDE_ERR_INVALID: return "mechanism inconsistent";
    case RDE_ERR_CUDA: return "CUDA runtime error";
    case RDE_ERR_UNSUPPORTED: return "mechanism size not supported by the compiled kernels";
    case RDE_ERR_ALIGN: return "pointer not aligned";
    case RDE_ERR_WORKSPACE: return "workspace too small";
    case RDE_ERR_NOMEM: return "allocation failed";
    case RDE_ERR_COMPILE: return "run-time compilation of a specialised kernel failed";
    default: return "unknown error code";
  }
}

const char* rde_last_error_message(void) { return g_msg.c_str(); }

int rde_chem_default_options(rde_chem_options* o) {
  if (!o) return fail(RDE_ERR_NULL, "options pointer is NULL");
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-8;
  o->atol = 1e-12;
  o->h_min = 1e-30;
  o->facmax = 5.0;
  o->facmin = 0.2;
  o->safety = 0.9;
  o->max_substeps = 100000;
  return RDE_OK;
}

int rde_mech_load(const char* text, size_t len, int flags, rde_mech_t* out) {
  g_msg.clear();
  if (!text || !out) return fail(RDE_ERR_NULL, "text and out are required");
  if (flags & ~(int)(RDE_LOAD_GENERIC | RDE_LOAD_REQUIRE_SPECIALIZED)) return fail(RDE_ERR_ARG, "unknown flags");
  if ((flags & RDE_LOAD_GENERIC) && (flags & RDE_LOAD_REQUIRE_SPECIALIZED))
    return fail(RDE_ERR_ARG, "RDE_LOAD_GENERIC and RDE_LOAD_REQUIRE_SPECIALIZED exclude each other");
  std::vector<unsigned char> image;
  std::vector<double> E_J;
  std::string err;
  int rc = rde::pack_mechanism(text, len, &image, &err, &E_J);
  if (rc == -1) return fail(RDE_ERR_PARSE, err);
  if (rc != 0) return fail(RDE_ERR_INVALID, err);
  const rde::MechHeader* hdr = reinterpret_cast<const rde::MechHeader*>(image.data());
  std::vector<unsigned char> plan;
  rde::build_large_plan(image.data(), &plan);
  rde_mech_s* h = new (std::nothrow) rde_mech_s();
  if (!h) return fail(RDE_ERR_NOMEM, "host allocation failed");
  h->plan_offset = (image.size() + 255) / 256 * 256;
  h->generic_ok = rde::kernel_supports(hdr->K);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_mech, h->plan_offset + plan.size());
  if (e == cudaSuccess) e = cudaMemcpy(h->d_mech, image.data(), image.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_mech + h->plan_offset, plan.data(), plan.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_scratch, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(h->d_scratch, 0, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess && h->generic_ok) e = rde::prepare_advance(hdr->K, (int)image.size(), &h->fit);
  std::string jit_log;
  if (e == cudaSuccess && !(flags & RDE_LOAD_GENERIC)) {
    h->jit_ok = rde::jit_build(image.data(), (int)image.size(), &h->jit, &jit_log) == 0;
    if (!h->jit_ok) cudaGetLastError();   // a failed attempt leaves no error for later calls
    if (!h->jit_ok && (flags & RDE_LOAD_REQUIRE_SPECIALIZED)) {
      cudaFree(h->d_mech);
      cudaFree(h->d_scratch);
      delete h;
      return fail(RDE_ERR_COMPILE, "specialised kernel: " + jit_log);
    }
  }
  h->small_ok = h->generic_ok || h->jit_ok;
  if (e == cudaSuccess) {
    // the CTA-per-cell kernel serves every K whose per-cell arrays fit in shared memory
    const cudaError_t el = rde::prepare_large(hdr->K, hdr->R, &h->large_fit);
    h->large_ok = (el == cudaSuccess);
    if (el != cudaSuccess && el != cudaErrorInvalidConfiguration) e = el;
    if (e == cudaSuccess && !h->small_ok && !h->large_ok) {
      cudaFree(h->d_mech);
      cudaFree(h->d_scratch);
      delete h;
      return fail(RDE_ERR_UNSUPPORTED, "mechanism with " + std::to_string(hdr->K) + " species and " +
                                           std::to_string(hdr->R) + " reactions exceeds shared memory per CTA");
    }
  }
  if (e != cudaSuccess) {
    if (h->d_mech) cudaFree(h->d_mech);
    if (h->d_scratch) cudaFree(h->d_scratch);
    if (h->d_park) cudaFree(h->d_park);
    delete h;
    return cuda_fail(e, "rde_mech_load");
  }
  h->K = hdr->K;
  h->R = hdr->R;
  h->mech_bytes = (int)image.size();
  h->image = image;
  h->E_J = E_J;
  rde_chem_default_options(&h->opt);
  *out = h;
  return RDE_OK;
}

int rde_mech_free(rde_mech_t h) {
  if (!h) return RDE_OK;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->d_mech);
  cudaFree(h->d_scratch);
  if (h->d_jscratch) cudaFree(h->d_jscratch);
  if (h->d_park) cudaFree(h->d_park);
  delete h;
  return RDE_OK;
}

int rde_mech_info(rde_mech_t h, int* n_species, int* n_reactions) {
  if (!h) return fail(RDE_ERR_NULL, "handle is NULL");
  if (n_species) *n_species = h->K;
  if (n_reactions) *n_reactions = h->R;
  return RDE_OK;
}

int rde_chem_set_options(rde_mech_t h, const rde_chem_options* o) {
  if (!h || !o) return fail(RDE_ERR_NULL, "handle and options are required");
  int rc = check_options(o);
  if (rc) return rc;
  if (o->method == RDE_METHOD_ROS2 && h->jit_ok && !h->jit_ros2_tried) {
    // a specialised handle selecting ROS2: compile its ROS2 kernels now (host, synchronous)
    h->jit_ros2_tried = true;
    std::string log;
    DeviceGuard g(h->device);
    h->jit_ros2_ok = rde::jit_build(h->image.data(), h->mech_bytes, &h->jit_ros2, &log, RDE_METHOD_ROS2) == 0;
    if (!h->jit_ros2_ok) cudaGetLastError();
  }
  if (o->method == RDE_METHOD_ROS2 && !h->jit_ros2_ok && !h->generic_ok)
    return fail(RDE_ERR_UNSUPPORTED, "no ROS2 kernel for this mechanism (precompiled for 2, 3 and 9 species)");
  if (o->method == RDE_METHOD_EXTRAP) {
    DeviceGuard g(h->device);
    if (h->jit_ok && !h->jit_extrap_tried) {
      h->jit_extrap_tried = true;
      std::string log;
      h->jit_extrap_ok = rde::jit_build(h->image.data(), h->mech_bytes, &h->jit_extrap, &log, RDE_METHOD_EXTRAP) == 0;
      if (!h->jit_extrap_ok) cudaGetLastError();
    }
    if (!h->jit_extrap_ok && !h->generic_ok)
      return fail(RDE_ERR_UNSUPPORTED, "no extrapolation kernel for this mechanism");
    if (!h->d_jscratch) {
      // one lane per thread of the persistent queue grid: CTAs per SM x SMs x 128 lanes
      const int fit = h->jit_extrap_ok ? h->jit_extrap.fit : h->fit;
      const int ctas = h->num_sms * (fit > 0 ? fit : 1);
      const size_t N = (size_t)h->K + 1;
      cudaError_t e = cudaMalloc(&h->d_jscratch, sizeof(double) * N * N * (size_t)ctas * 128);
      if (e != cudaSuccess) {
        h->d_jscratch = nullptr;
        return cuda_fail(e, "allocate the extrapolation scratch");
      }
      h->jscratch_ctas = ctas;
    }
  }
  h->opt = *o;
  return RDE_OK;
}

int rde_chem_get_options(rde_mech_t h, rde_chem_options* o) {
  if (!h || !o) return fail(RDE_ERR_NULL, "handle and options are required");
  *o = h->opt;
  return RDE_OK;
}

namespace {
// Picks the kernel for a call: the thread-per-cell kernel when one is compiled for K
// (PLAIN / QUEUE / AUTO), else, or on RDE_SCHED_BLOCK, the CTA-per-cell kernel.
int pick_kernel(const rde_mech_s* h, int schedule, bool* large) {
  const bool ros2 = h->opt.method == RDE_METHOD_ROS2, extrap = h->opt.method == RDE_METHOD_EXTRAP;
  // a thread-per-cell kernel for the handle's method: specialised, else precompiled
  const bool thread_cell = ros2 ? (h->jit_ros2_ok || h->generic_ok)
                                : extrap ? (h->jit_extrap_ok || h->generic_ok) : h->small_ok;
  *large = (schedule == RDE_SCHED_BLOCK) || !thread_cell;
  if (*large && (ros2 || extrap))
    return fail(RDE_ERR_UNSUPPORTED, "the CTA-per-cell kernel integrates with RODAS3 only");
  if (extrap && schedule == RDE_SCHED_PLAIN)
    return fail(RDE_ERR_UNSUPPORTED, "the extrapolation method runs on the queue schedule only");
  if (*large && !h->large_ok) return fail(RDE_ERR_UNSUPPORTED, "no kernel for this mechanism and schedule");
  return RDE_OK;
}

// The wide queue kernel and its park area (one lane per thread of its persistent grid),
// built on the first call that asks for it (host, synchronous: not inside a capture).
void build_wide(rde_mech_s* h) {
  if (h->jit_wide_tried || !h->jit_ok || h->opt.method != RDE_METHOD_RODAS3) return;
  h->jit_wide_tried = true;
  DeviceGuard g(h->device);
  std::string log;
  if (rde::jit_build_wide(h->image.data(), h->mech_bytes, &h->jit, &log) != 0) {
    cudaGetLastError();
    h->jit.queue_w = nullptr;
    return;
  }
  const long long lanes = (long long)h->num_sms * (h->jit.fit_w > 0 ? h->jit.fit_w : 1) * 256;
  if (cudaMalloc(&h->d_park, sizeof(double) * 4 * (size_t)(h->K + 1) * (size_t)lanes) != cudaSuccess) {
    cudaGetLastError();
    h->d_park = nullptr;
    h->jit.queue_w = nullptr;
    return;
  }
  h->park_lanes = lanes;
}

// threads_per_cta of a call: 0 or 128 (the 128-thread kernels) or 256 (the wide queue
// kernel, specialised RODAS3 only)
int check_threads(const rde_mech_s* h, const rde_chem_call* c, bool large) {
  if (c->threads_per_cta != 0 && c->threads_per_cta != 128 && c->threads_per_cta != 256)
    return fail(RDE_ERR_ARG, "threads_per_cta must be 0, 128 or 256");
  if (c->threads_per_cta == 256 &&
      (large || c->schedule == RDE_SCHED_PLAIN || h->opt.method != RDE_METHOD_RODAS3 || !h->jit_ok ||
       !h->jit.queue_w || !h->d_park))
    return fail(RDE_ERR_UNSUPPORTED, "threads_per_cta = 256 needs the wide queue kernel (specialised RODAS3)");
  return RDE_OK;
}

cudaError_t launch_cells(const rde_mech_s* h, rde::LaunchArgs& a, bool large, cudaStream_t s) {
  a.plan = h->d_mech + h->plan_offset;
  a.R = h->R;
  a.large_fit = h->large_fit;
  if (large) return rde::launch_large(a, s);
  if (h->opt.method == RDE_METHOD_ROS2)
    return h->jit_ros2_ok ? rde::jit_launch(h->jit_ros2, a, s) : rde::launch_advance(a, s);
  if (h->opt.method == RDE_METHOD_EXTRAP) {
    a.jscratch = h->d_jscratch;
    a.jscratch_ctas = h->jscratch_ctas;
    return h->jit_extrap_ok ? rde::jit_launch(h->jit_extrap, a, s) : rde::launch_advance(a, s);
  }
  a.park = h->d_park;
  a.park_lanes = h->park_lanes;
  return h->jit_ok ? rde::jit_launch(h->jit, a, s) : rde::launch_advance(a, s);
}
}  // namespace

int rde_chem_advance_ex(rde_mech_t h, const rde_chem_call* c, void* stream) {
  if (!h || !c) return fail(RDE_ERR_NULL, "handle and call are required");
  if (!(c->dt > 0) || !std::isfinite(c->dt)) return fail(RDE_ERR_ARG, "dt must be finite and > 0");
  if (c->schedule != RDE_SCHED_AUTO && c->schedule != RDE_SCHED_PLAIN && c->schedule != RDE_SCHED_QUEUE &&
      c->schedule != RDE_SCHED_BLOCK)
    return fail(RDE_ERR_ARG, "unknown schedule");
  bool large = false;
  if (int prc = pick_kernel(h, c->schedule, &large)) return prc;
  if (c->threads_per_cta == 256 && c->schedule != RDE_SCHED_PLAIN && !large) build_wide(h);
  if (int trc = check_threads(h, c, large)) return trc;
  if (c->ctas_per_sm < 0 || c->ctas_per_sm > 32) return fail(RDE_ERR_ARG, "ctas_per_sm out of range");
  long long n_total;
  if (c->blocks) {
    if (c->n_blocks < 1 || c->n_blocks > 1024) return fail(RDE_ERR_ARG, "n_blocks must be 1..1024");
    if (c->n_total < 0) return fail(RDE_ERR_ARG, "n_total < 0");
    if (!aligned8(c->blocks)) return fail(RDE_ERR_ALIGN, "block table must be 8-byte aligned");
    n_total = c->n_total;
  } else {
    int rc = check_block(c->cells, h->K);
    if (rc) return rc;
    n_total = c->cells.n;
  }
  if (c->order && !aligned8(c->order)) return fail(RDE_ERR_ALIGN, "order must be 8-byte aligned");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(h->d_scratch, 0, 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "reset scratch");
  if (n_total == 0) return RDE_OK;
  rde::LaunchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.mech = h->d_mech;
  a.mech_bytes = h->mech_bytes;
  a.K = h->K;
  a.cells = c->cells;
  a.blocks = c->blocks;
  a.n_blocks = c->blocks ? c->n_blocks : 0;
  a.n_total = n_total;
  a.order = reinterpret_cast<const long long*>(c->order);
  a.dt = c->dt;
  a.opt = h->opt;
  a.queue = h->d_scratch;
  a.stats = reinterpret_cast<long long*>(h->d_scratch + 1);
  a.schedule = (c->schedule == RDE_SCHED_PLAIN) ? RDE_SCHED_PLAIN : RDE_SCHED_QUEUE;
  a.threads = c->threads_per_cta;
  a.ctas_per_sm = c->ctas_per_sm;
  a.num_sms = h->num_sms;
  a.fit = h->fit;
  e = launch_cells(h, a, large, s);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return RDE_OK;
}

int rde_chem_advance(rde_mech_t h, int64_t n_cells, const double* p, double* T, double* Y, double dt,
                     void* stream) {
  rde_chem_call c;
  std::memset(&c, 0, sizeof(c));
  c.cells.p = p;
  c.cells.T = T;
  c.cells.Y = Y;
  c.cells.n = n_cells;
  c.cells.ldY = n_cells;
  c.dt = dt;
  c.schedule = RDE_SCHED_AUTO;
  return rde_chem_advance_ex(h, &c, stream);
}

int rde_chem_kernel_info(rde_mech_t h, int* threads_per_cta, int* max_ctas_per_sm, size_t* shared_bytes) {
  if (!h) return fail(RDE_ERR_NULL, "handle is NULL");
  // the kernel of the AUTO schedule
  if (threads_per_cta) *threads_per_cta = h->small_ok ? rde::kernel_threads() : rde::large_threads();
  if (max_ctas_per_sm) *max_ctas_per_sm = h->jit_ok ? h->jit.fit : (h->small_ok ? h->fit : h->large_fit);
  if (shared_bytes)
    *shared_bytes = h->small_ok ? rde::thread_cell_shared_bytes(h->K, h->mech_bytes, 0)
                                : rde::large_shared_bytes(h->K, h->R, 0);
  return RDE_OK;
}

int rde_chem_kernel_variant(rde_mech_t h, int* variant, double* compile_seconds) {
  if (!h) return fail(RDE_ERR_NULL, "handle is NULL");
  if (variant) *variant = h->jit_ok ? RDE_KERNEL_SPECIALIZED : (h->generic_ok ? RDE_KERNEL_GENERIC : RDE_KERNEL_BLOCK);
  if (compile_seconds) *compile_seconds = h->jit_ok ? h->jit.compile_s : 0.0;
  return RDE_OK;
}

int rde_chem_get_stats(rde_mech_t h, void* stream, rde_chem_stats* out) {
  if (!h || !out) return fail(RDE_ERR_NULL, "handle and out are required");
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  unsigned long long v[8];
  e = cudaMemcpy(v, h->d_scratch, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read statistics");
  std::memset(out, 0, sizeof(*out));
  out->cells = (int64_t)v[1];
  out->accepted = (int64_t)v[2];
  out->rejected = (int64_t)v[3];
  out->failed = (int64_t)v[4];
  out->max_attempts = (int64_t)v[5];
  return RDE_OK;
}

int rde_chem_status(rde_mech_t h, void* stream, int64_t* n_failed) {
  if (!n_failed) return fail(RDE_ERR_NULL, "n_failed is NULL");
  rde_chem_stats st;
  int rc = rde_chem_get_stats(h, stream, &st);
  if (rc) return rc;
  *n_failed = st.failed;
  return RDE_OK;
}

int rde_selftest_jit_compile(const char* text, size_t len, int part, char* source, size_t source_len, char* log,
                             size_t log_len, double* seconds, size_t* cubin_bytes) {
  g_msg.clear();
  if (!text) return fail(RDE_ERR_NULL, "text is required");
  std::vector<unsigned char> image;
  std::string err;
  int rc = rde::pack_mechanism(text, len, &image, &err);
  if (rc == -1) return fail(RDE_ERR_PARSE, err);
  if (rc != 0) return fail(RDE_ERR_INVALID, err);
  auto copy_out = [](const std::string& s, char* dst, size_t cap) {
    if (!dst || cap == 0) return;
    const size_t n = s.size() < cap - 1 ? s.size() : cap - 1;
    std::memcpy(dst, s.data(), n);
    dst[n] = '\0';
  };
  if (part < 0 || part > 3) return fail(RDE_ERR_ARG, "part must be 0, 1, 2 or 3");
  copy_out(part == 1   ? rde::jit_adjoint_source(image.data())
           : part == 3 ? rde::jit_wide_source(image.data())
                       : rde::jit_source(image.data(), part == 2 ? RDE_METHOD_ROS2 : RDE_METHOD_RODAS3),
           source, source_len);
  std::string jlog;
  if (rde::jit_compile_only(image.data(), part, &jlog, seconds, cubin_bytes) != 0) {
    copy_out(jlog, log, log_len);
    return fail(RDE_ERR_COMPILE, jlog.substr(0, 2000));
  }
  copy_out(jlog, log, log_len);   // empty unless a verbose compilation was asked for
  return RDE_OK;
}

int rde_selftest_batched_lu(int dmma, int64_t batch, int n, double* A, int32_t* piv, int32_t* info, void* stream) {
  g_msg.clear();
  if (dmma != 0 && dmma != 1) return fail(RDE_ERR_ARG, "dmma must be 0 or 1");
  if (batch < 0) return fail(RDE_ERR_ARG, "batch < 0");
  if (n < 1 || n > rde::lu_compare_max_order()) return fail(RDE_ERR_ARG, "n must be 1..56");
  if (batch == 0) return RDE_OK;
  if (!A || !piv) return fail(RDE_ERR_NULL, "A and piv are required");
  if (!aligned8(A)) return fail(RDE_ERR_ALIGN, "A must be 8-byte aligned");
  cudaError_t e = rde::launch_batched_lu(dmma, batch, n, A, piv, info, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "batched LU");
  return RDE_OK;
}

int rde_selftest_math(int fn, int64_t n, const double* x, double* y, int on_device, void* stream) {
  if (fn != 0 && fn != 1) return fail(RDE_ERR_ARG, "fn must be 0 (exp) or 1 (log)");
  if (on_device != 0 && on_device != 1) return fail(RDE_ERR_ARG, "on_device must be 0 or 1");
  if (n < 0) return fail(RDE_ERR_ARG, "n < 0");
  if (n == 0) return RDE_OK;
  if (!x || !y) return fail(RDE_ERR_NULL, "x and y are required");
  const double* et = rde::exp2_table_host();
  const double* lt = rde::log_table_host();
  if (!on_device) {
    for (int64_t i = 0; i < n; ++i) y[i] = fn == 0 ? rde::exp_tab(x[i], et) : rde::log_tab(x[i], lt);
    return RDE_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t tb = sizeof(double) * (rde::kExpTabSize + 2 * rde::kLogTabSize);
  double* d_tab = nullptr;
  cudaError_t e = cudaMalloc(&d_tab, tb);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, et, sizeof(double) * rde::kExpTabSize, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tab + rde::kExpTabSize, lt, sizeof(double) * 2 * rde::kLogTabSize, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = rde::launch_selftest_math(fn, (long long)n, x, y, d_tab, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_tab) cudaFree(d_tab);
  if (e != cudaSuccess) return cuda_fail(e, "rde_selftest_math");
  return RDE_OK;
}

int rde_chem_advance_noalloc(rde_mech_t h, const rde_chem_call* c, void* stream) {
  if (!h || !c) return fail(RDE_ERR_NULL, "handle and call are required");
  if (!(c->dt > 0) || !std::isfinite(c->dt)) return fail(RDE_ERR_ARG, "dt must be finite and > 0");
  if (c->schedule != RDE_SCHED_AUTO && c->schedule != RDE_SCHED_PLAIN && c->schedule != RDE_SCHED_QUEUE &&
      c->schedule != RDE_SCHED_BLOCK)
    return fail(RDE_ERR_ARG, "unknown schedule");
  bool large = false;
  if (int prc = pick_kernel(h, c->schedule, &large)) return prc;
  if (int trc = check_threads(h, c, large)) return trc;
  if (c->ctas_per_sm < 0 || c->ctas_per_sm > 32) return fail(RDE_ERR_ARG, "ctas_per_sm out of range");
  // scratch this call needs: the queue counter and seven statistics words
  const size_t needed = 8 * sizeof(unsigned long long);
  if (needed > RDE_NOALLOC_SCRATCH_BYTES)
    return fail(RDE_ERR_WORKSPACE, "call needs " + std::to_string(needed) + " scratch bytes, more than the " +
                                       std::to_string(RDE_NOALLOC_SCRATCH_BYTES) + "-byte static array");
  long long n_total;
  if (c->blocks) {
    if (c->n_blocks < 1 || c->n_blocks > 1024) return fail(RDE_ERR_ARG, "n_blocks must be 1..1024");
    if (c->n_total < 0) return fail(RDE_ERR_ARG, "n_total < 0");
    if (!aligned8(c->blocks)) return fail(RDE_ERR_ALIGN, "block table must be 8-byte aligned");
    n_total = c->n_total;
  } else {
    int rc = check_block(c->cells, h->K);
    if (rc) return rc;
    n_total = c->cells.n;
  }
  if (c->order && !aligned8(c->order)) return fail(RDE_ERR_ALIGN, "order must be 8-byte aligned");
  DeviceGuard g(h->device);
  unsigned long long* scratch = nullptr;
  int rc = noalloc_scratch(h->device, &scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, needed, s);
  if (e != cudaSuccess) return cuda_fail(e, "clear no-alloc scratch");
  if (n_total == 0) return RDE_OK;
  rde::LaunchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.mech = h->d_mech;
  a.mech_bytes = h->mech_bytes;
  a.K = h->K;
  a.cells = c->cells;
  a.blocks = c->blocks;
  a.n_blocks = c->blocks ? c->n_blocks : 0;
  a.n_total = n_total;
  a.order = reinterpret_cast<const long long*>(c->order);
  a.dt = c->dt;
  a.opt = h->opt;
  a.queue = scratch;
  a.stats = reinterpret_cast<long long*>(scratch + 1);
  a.schedule = (c->schedule == RDE_SCHED_PLAIN) ? RDE_SCHED_PLAIN : RDE_SCHED_QUEUE;
  a.threads = c->threads_per_cta;
  a.ctas_per_sm = c->ctas_per_sm;
  a.num_sms = h->num_sms;
  a.fit = h->fit;
  e = launch_cells(h, a, large, s);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return RDE_OK;
}

struct rde_graph_s {
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

int rde_chem_graph_create(rde_mech_t h, const rde_chem_call* c, int n_steps, void** out) {
  if (!h || !c || !out) return fail(RDE_ERR_NULL, "handle, call and out are required");
  if (n_steps < 1 || n_steps > 100000) return fail(RDE_ERR_ARG, "n_steps must be 1..100000");
  DeviceGuard g(h->device);
  if (c->threads_per_cta == 256 && c->schedule != RDE_SCHED_PLAIN && c->schedule != RDE_SCHED_BLOCK)
    build_wide(h);   // before the capture begins
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "create capture stream");
  cudaGraph_t graph = nullptr;
  int rc = RDE_OK;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    return cuda_fail(e, "begin capture");
  }
  for (int i = 0; i < n_steps && rc == RDE_OK; ++i) rc = rde_chem_advance_ex(h, c, s);
  e = cudaStreamEndCapture(s, &graph);
  cudaStreamDestroy(s);
  if (rc != RDE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  rde_graph_s* gr = new (std::nothrow) rde_graph_s();
  if (!gr) {
    cudaGraphDestroy(graph);
    return fail(RDE_ERR_NOMEM, "host allocation failed");
  }
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    delete gr;
    return cuda_fail(e, "instantiate graph");
  }
  gr->device = h->device;
  *out = gr;
  return RDE_OK;
}

int rde_chem_graph_launch(void* graph, void* stream) {
  if (!graph) return fail(RDE_ERR_NULL, "graph is NULL");
  rde_graph_s* gr = static_cast<rde_graph_s*>(graph);
  DeviceGuard g(gr->device);
  cudaError_t e = cudaGraphLaunch(gr->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return RDE_OK;
}

int rde_chem_graph_destroy(void* graph) {
  if (!graph) return RDE_OK;
  rde_graph_s* gr = static_cast<rde_graph_s*>(graph);
  DeviceGuard g(gr->device);
  cudaGraphExecDestroy(gr->exec);
  delete gr;
  return RDE_OK;
}

// ---- discrete adjoint ----------------------------------------------------------
namespace {
constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct AdjLayout {
  size_t offsets, order, rec, pool, lanes, rows, queue, stages, ckpt, seg, replay, total;
  int S, seg_max;   // self-checkpointing mode only
};

// Workspace regions; with `stages` the stage checkpoints of every accepted step follow.
// The lane scratch serves the thread-per-cell reverse kernel only.
AdjLayout adj_layout(const rde_mech_s* h, long long n, long long total_steps, bool stages) {
  const bool thread_cell = h->generic_ok || h->jit_ok;
  const int N = h->K + 1, R = h->R;
  AdjLayout L{};
  size_t o = 0;
  L.offsets = o;  o = align_up(o + sizeof(long long) * (n + 1));
  L.order = o;    o = align_up(o + sizeof(long long) * n);
  L.rec = o;      o = align_up(o + sizeof(int) * n);
  L.pool = o;     o = align_up(o + sizeof(double) * (size_t)total_steps * (N + 1));
  L.lanes = o;
  if (thread_cell) o = align_up(o + sizeof(double) * (size_t)(8 * N + 2 * R) * rde::adjoint_lanes(h->num_sms));
  L.rows = o;     o = align_up(o + sizeof(double) * (size_t)(2 * R) * n);
  L.queue = o;    o = align_up(o + 2 * sizeof(unsigned long long));
  L.stages = o;
  if (stages) o = align_up(o + sizeof(double) * (size_t)total_steps * (size_t)rde::adjoint_stage_doubles(h->K));
  L.total = o;
  return L;
}

// Self-checkpointing workspace (no step counts known): S checkpoints of N + 3 doubles per
// cell (thread per cell) or per CTA (CTA per cell), a segment buffer of seg_max steps and
// the replay state per reverse lane (or per CTA), the parameter rows and the counters.
AdjLayout adj_layout_self(const rde_mech_s* h, long long n, int S, bool large) {
  const int N = h->K + 1, R = h->R;
  const long long lanes = rde::adjoint_lanes(h->num_sms);
  const long long owners = large ? (long long)h->num_sms : n;   // who holds S checkpoints
  const long long segs = large ? (long long)h->num_sms : lanes;
  AdjLayout L{};
  L.S = S;
  L.seg_max = rde::ckpt_seg_max(h->opt.max_substeps, S);
  size_t o = 0;
  L.order = o;    o = align_up(o + sizeof(long long) * n);
  L.rec = o;      o = align_up(o + sizeof(int) * n);
  L.ckpt = o;     o = align_up(o + sizeof(double) * (size_t)owners * S * (N + 3));
  L.seg = o;      o = align_up(o + sizeof(double) * (size_t)segs * L.seg_max * (N + 1));
  L.lanes = o;
  L.replay = o;
  if (!large) {
    o = align_up(o + sizeof(double) * (size_t)(8 * N + 2 * R) * lanes);
    L.replay = o;
    o = align_up(o + sizeof(double) * (size_t)(N + 6) * lanes);
  }
  L.rows = o;     o = align_up(o + sizeof(double) * (size_t)(2 * R) * n);
  L.queue = o;    o = align_up(o + 2 * sizeof(unsigned long long));
  L.offsets = L.pool = L.stages = 0;
  L.total = o;
  return L;
}

// Checkpoints per owner of the self-checkpointing mode: the default of the workspace
// query, and the bounds a given workspace is fitted between.
int ckpt_default(bool large) { return large ? 4096 : rde::kCkptDefault; }
int ckpt_max(bool large) { return large ? 4096 : rde::kCkptMax; }
}  // namespace

size_t rde_chem_adjoint_workspace_steps(rde_mech_t h, int64_t n_cells, int64_t total_steps) {
  if (!h || n_cells < 0 || total_steps < 0) return 0;
  return adj_layout(h, n_cells, total_steps, false).total;
}

size_t rde_chem_adjoint_workspace_checkpointed(rde_mech_t h, int64_t n_cells, int64_t total_steps) {
  if (!h || n_cells < 0 || total_steps < 0) return 0;
  // only the thread-per-cell adjoint keeps stage checkpoints
  const bool thread_cell = h->generic_ok || h->jit_ok;
  return adj_layout(h, n_cells, total_steps, thread_cell).total;
}

size_t rde_chem_adjoint_workspace(rde_mech_t h, int64_t n_cells, double dt) {
  if (!h || n_cells < 0 || !(dt > 0) || !std::isfinite(dt)) return 0;
  // the AUTO schedule takes the thread-per-cell adjoint where a kernel serves the
  // mechanism; its layout is the larger of the two.  The thread-per-cell layout holds
  // S checkpoints per cell and a replay segment of max_substeps / S steps per lane, so
  // for few cells the larger S can take less memory: take the smaller of the default S
  // and the largest one (the call then uses the largest S that fits)
  const bool thread_cell = h->generic_ok || h->jit_ok;
  size_t a = adj_layout_self(h, n_cells, ckpt_default(!thread_cell), !thread_cell).total;
  const size_t a2 = adj_layout_self(h, n_cells, ckpt_max(!thread_cell), !thread_cell).total;
  if (a2 < a) a = a2;
  const size_t b = adj_layout_self(h, n_cells, ckpt_default(true), true).total;
  return a > b ? a : b;
}

int rde_chem_advance_adjoint_ex(rde_mech_t h, const rde_adjoint_call* c, void* stream) {
  if (!h || !c) return fail(RDE_ERR_NULL, "handle and call are required");
  if (h->opt.method != RDE_METHOD_RODAS3)
    return fail(RDE_ERR_UNSUPPORTED, "the adjoint differentiates RODAS3 steps only");
  if (c->schedule != RDE_SCHED_AUTO && c->schedule != RDE_SCHED_BLOCK)
    return fail(RDE_ERR_ARG, "adjoint schedule must be RDE_SCHED_AUTO or RDE_SCHED_BLOCK");
  if (c->schedule == RDE_SCHED_AUTO && h->jit_ok && !h->jit_adj_tried) {
    // first adjoint call of a specialised handle: compile the specialised adjoint kernels
    h->jit_adj_tried = true;
    std::string log;
    DeviceGuard g(h->device);
    h->jit_adj_ok = rde::jit_build_adjoint(h->image.data(), h->mech_bytes, &h->jadj, &log) == 0;
    if (!h->jit_adj_ok) cudaGetLastError();
  }
  const bool large = c->schedule == RDE_SCHED_BLOCK || (!h->generic_ok && !h->jit_adj_ok);
  if (large && h->large_ok && !h->large_adj_tried) {
    h->large_adj_tried = true;
    DeviceGuard g(h->device);
    h->large_adj_ok = rde::prepare_large_adjoint(h->K, h->R) == cudaSuccess;
    if (!h->large_adj_ok) cudaGetLastError();
  }
  if (large && !h->large_adj_ok)
    return fail(RDE_ERR_UNSUPPORTED, "no adjoint kernel fits this mechanism");
  if (c->n < 0) return fail(RDE_ERR_ARG, "n < 0");
  if (!(c->dt > 0) || !std::isfinite(c->dt)) return fail(RDE_ERR_ARG, "dt must be finite and > 0");
  const bool self = c->n_steps == nullptr;
  if (!self && c->total_steps < 0) return fail(RDE_ERR_ARG, "total_steps < 0");
  if (!c->g_lnA || !c->g_E) return fail(RDE_ERR_NULL, "g_lnA and g_E are required");
  if (c->n > 0) {
    if (!c->p || !c->T0 || !c->Y0 || !c->gT || !c->gY || !c->gT0 || !c->gY0)
      return fail(RDE_ERR_NULL, "p, T0, Y0, gT, gY, gT0 and gY0 are required");
    if (c->ldY < c->n) return fail(RDE_ERR_ARG, "ldY < n");
    const void* dp[] = {c->p, c->T0, c->Y0, c->gT, c->gY, c->gT0, c->gY0, c->g_lnA, c->g_E};
    for (const void* q : dp)
      if (!aligned8(q)) return fail(RDE_ERR_ALIGN, "double arrays must be 8-byte aligned");
  }
  AdjLayout lay;
  bool use_stages = false;
  if (self) {
    // self-checkpointing: the most checkpoints per owner (a power of two) the workspace holds
    int S = ckpt_max(large);
    while (S > rde::kCkptMin && adj_layout_self(h, c->n, S, large).total > c->workspace_bytes) S >>= 1;
    lay = adj_layout_self(h, c->n, S, large);
    if (!c->workspace || c->workspace_bytes < lay.total)
      return fail(RDE_ERR_WORKSPACE, "adjoint workspace needs at least " + std::to_string(lay.total) + " bytes");
  } else {
    // stage checkpoints when the workspace holds them, else recompute the stages
    const AdjLayout full = adj_layout(h, c->n, c->total_steps, true);
    use_stages = !large && c->workspace_bytes >= full.total;
    lay = use_stages ? full : adj_layout(h, c->n, c->total_steps, false);
    if (!c->workspace || c->workspace_bytes < lay.total)
      return fail(RDE_ERR_WORKSPACE, "adjoint workspace needs " + std::to_string(lay.total) + " bytes");
  }
  if ((reinterpret_cast<uintptr_t>(c->workspace) & (kAlign - 1)) != 0)
    return fail(RDE_ERR_ALIGN, "workspace must be 256-byte aligned");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(c->workspace);
  cudaError_t e = cudaMemsetAsync(ws + lay.queue, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->g_lnA, 0, sizeof(double) * h->R, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->g_E, 0, sizeof(double) * h->R, s);
  if (e != cudaSuccess) return cuda_fail(e, "clear adjoint workspace");
  if (c->n == 0) return RDE_OK;
  rde::AdjointLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.mech = h->d_mech;
  a.plan = h->d_mech + h->plan_offset;
  a.large = large;
  a.mech_bytes = h->mech_bytes;
  a.K = h->K;
  a.R = h->R;
  a.n = c->n;
  a.p = c->p;
  a.T0 = c->T0;
  a.Y0 = c->Y0;
  a.ldY = c->ldY;
  a.dt = c->dt;
  a.opt = h->opt;
  a.n_steps = c->n_steps;
  a.total_steps = c->total_steps;
  a.offsets = self ? nullptr : reinterpret_cast<long long*>(ws + lay.offsets);
  a.order = reinterpret_cast<long long*>(ws + lay.order);
  a.rec = reinterpret_cast<int*>(ws + lay.rec);
  a.pool = self ? nullptr : reinterpret_cast<double*>(ws + lay.pool);
  a.stages = use_stages ? reinterpret_cast<double*>(ws + lay.stages) : nullptr;
  if (self) {
    a.n_steps = nullptr;
    a.total_steps = 0;
    a.ckpt_S = lay.S;
    a.seg_max = lay.seg_max;
    a.ckpt = reinterpret_cast<double*>(ws + lay.ckpt);
    a.seg = reinterpret_cast<double*>(ws + lay.seg);
    a.replay = large ? nullptr : reinterpret_cast<double*>(ws + lay.replay);
  }
  a.lane_scratch = reinterpret_cast<double*>(ws + lay.lanes);
  a.rows = reinterpret_cast<double*>(ws + lay.rows);
  a.queue = reinterpret_cast<unsigned long long*>(ws + lay.queue);
  a.gT = c->gT;
  a.gY = c->gY;
  a.gT0 = c->gT0;
  a.gY0 = c->gY0;
  a.g_lnA = c->g_lnA;
  a.g_E = c->g_E;
  a.status = c->status;
  a.num_sms = h->num_sms;
  if (!large && h->jit_adj_ok) {
    a.jit_record = reinterpret_cast<const void*>(h->jadj.record);
    a.jit_reverse = reinterpret_cast<const void*>(h->jadj.reverse);
    a.jit_reverse_self = reinterpret_cast<const void*>(h->jadj.reverse_self);
    a.jit_fit_record = h->jadj.fit_record;
  }
  e = rde::launch_adjoint(a, s);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  return RDE_OK;
}

size_t rde_selftest_adjoint_self_workspace(void* hv, int64_t n_cells, int S, int block) {
  rde_mech_t h = static_cast<rde_mech_t>(hv);
  if (!h || n_cells < 0 || S < rde::kCkptMin || S > 4096 || (S & (S - 1))) return 0;
  return adj_layout_self(h, n_cells, S, block != 0).total;
}

int rde_chem_advance_adjoint(rde_mech_t h, int64_t n_cells, const double* p, const double* T0, const double* Y0,
                             double dt, const double* gT, const double* gY, double* gT0, double* gY0, double* g_lnA,
                             double* g_E, void* workspace, size_t ws_bytes, void* stream) {
  rde_adjoint_call c;
  std::memset(&c, 0, sizeof(c));
  c.n = n_cells;
  c.p = p;
  c.T0 = T0;
  c.Y0 = Y0;
  c.ldY = n_cells;
  c.dt = dt;
  c.n_steps = nullptr;   // the library finds each cell's steps itself
  c.gT = gT;
  c.gY = gY;
  c.gT0 = gT0;
  c.gY0 = gY0;
  c.g_lnA = g_lnA;
  c.g_E = g_E;
  c.workspace = workspace;
  c.workspace_bytes = ws_bytes;
  c.schedule = RDE_SCHED_AUTO;
  return rde_chem_advance_adjoint_ex(h, &c, stream);
}

int rde_mech_get_arrhenius(rde_mech_t h, double* lnA, double* E) {
  if (!h || !lnA || !E) return fail(RDE_ERR_NULL, "handle, lnA and E are required");
  const rde::MechView v = rde::mech_view(h->image.data());
  for (int r = 0; r < h->R; ++r) {
    lnA[r] = v.rx[r].lnA;
    E[r] = h->E_J[r];
  }
  return RDE_OK;
}

int rde_mech_set_arrhenius(rde_mech_t h, const double* lnA, const double* E) {
  if (!h || !lnA || !E) return fail(RDE_ERR_NULL, "handle, lnA and E are required");
  for (int r = 0; r < h->R; ++r)
    if (!std::isfinite(lnA[r]) || !std::isfinite(E[r])) return fail(RDE_ERR_ARG, "non-finite parameter");
  rde::MechView v = rde::mech_view(h->image.data());
  rde::RxnPacked* rx = const_cast<rde::RxnPacked*>(v.rx);
  for (int r = 0; r < h->R; ++r) {
    rx[r].lnA = lnA[r];
    rx[r].EaR = E[r] / rde::kRuHost;   // as the parser computes it from E in J/mol
    h->E_J[r] = E[r];
  }
  std::vector<unsigned char> plan;   // the CTA-per-cell kernel reads ln A and E/R from the plan
  rde::build_large_plan(h->image.data(), &plan);
  DeviceGuard g(h->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h->d_mech, h->image.data(), h->image.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_mech + h->plan_offset, plan.data(), plan.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "upload parameters");
  return RDE_OK;
}

}  // extern "C"
