// Load-time generation, NVRTC compilation and loading of mechanism-specialised
// thread-per-cell kernels (see jit.h).  Host code only.
#include "jit.h"

#include <dlfcn.h>
#include <libgen.h>
#include <nvrtc.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <vector>

#include "mech_layout.h"

namespace rde {

namespace {

constexpr int kJitThreads = 128;   // threads per CTA, as the generic kernels
constexpr int kWideThreads = 256;  // threads per CTA of the wide kernels (two warps per SM sub-partition)
constexpr int kWideMaxK = 16;      // species of the wide kernels (their slots live in registers)
constexpr int kJitMaxBlocks = 1024;
constexpr size_t kSharedLimit = 227 * 1024;

// ---- NVRTC through dlopen ----------------------------------------------------
struct Nvrtc {
  bool ok = false;
  std::string why;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
  nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
  const char* (*errstr)(nvrtcResult) = nullptr;
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so", "libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
      n.why = "libnvrtc.so not found";
      return;
    }
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.errstr = reinterpret_cast<decltype(n.errstr)>(dlsym(h, "nvrtcGetErrorString"));
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy && n.errstr;
    if (!n.ok) n.why = "libnvrtc.so lacks an entry point";
  });
  return n;
}

// Directory of the kernel sources: <package>/csrc, beside <package>/_build/librde_chem.so.
std::string source_dir() {
  Dl_info info;
  if (!dladdr(reinterpret_cast<void*>(&jit_max_species), &info) || !info.dli_fname) return std::string();
  std::vector<char> p(info.dli_fname, info.dli_fname + std::strlen(info.dli_fname) + 1);
  std::string build_dir = dirname(p.data());
  std::vector<char> q(build_dir.begin(), build_dir.end());
  q.push_back('\0');
  return std::string(dirname(q.data())) + "/csrc";
}

// ---- source generation ---------------------------------------------------------
std::string lit(double v) {
  char b[64];
  if (std::isfinite(v)) {
    std::snprintf(b, sizeof(b), "%a", v);
  } else {
    long long bits;
    std::memcpy(&bits, &v, 8);
    std::snprintf(b, sizeof(b), "__longlong_as_double(0x%llxLL)", (unsigned long long)bits);
  }
  return b;
}

// "q == 0 ? v0 : (q == 1 ? v1 : v2)" over n values
template <class T, class F>
std::string select(const T* v, int n, F fmt) {
  std::string s = fmt(v[n - 1]);
  for (int i = n - 2; i >= 0; --i) s = "(q == " + std::to_string(i) + " ? " + fmt(v[i]) + " : " + s + ")";
  return s;
}

std::string ifmt(int v) { return std::to_string(v); }
std::string dfmt(double v) { return lit(v); }

void reaction_struct(std::ostringstream& o, const MechView& v, int r) {
  const RxnPacked& x = v.rx[r];
  o << "struct Rx" << r << " {\n"
    << "  const RxnPacked& x;\n"
    << "  __device__ __forceinline__ double lnA() const { return x.lnA; }\n"
    << "  __device__ __forceinline__ double EaR() const { return x.EaR; }\n"
    << "  __device__ __forceinline__ int type() const { return " << x.type << "; }\n"
    << "  __device__ __forceinline__ int rev() const { return " << x.rev << "; }\n"
    << "  __device__ __forceinline__ int nf() const { return " << x.nf << "; }\n"
    << "  __device__ __forceinline__ int nb() const { return " << x.nb << "; }\n"
    << "  __device__ __forceinline__ int np() const { return " << x.np << "; }\n"
    << "  __device__ __forceinline__ int fi(int q) const { return " << select(x.fi, kMaxSide, ifmt) << "; }\n"
    << "  __device__ __forceinline__ int fo(int q) const { return " << select(x.fo, kMaxSide, ifmt) << "; }\n"
    << "  __device__ __forceinline__ int bi(int q) const { return " << select(x.bi, kMaxSide, ifmt) << "; }\n"
    << "  __device__ __forceinline__ int bo(int q) const { return " << select(x.bo, kMaxSide, ifmt) << "; }\n"
    << "  __device__ __forceinline__ int pi(int q) const { return " << select(x.pi, kMaxPart, ifmt) << "; }\n"
    << "  __device__ __forceinline__ double fod(int q) const { return " << select(x.fod, kMaxSide, dfmt) << "; }\n"
    << "  __device__ __forceinline__ double bod(int q) const { return " << select(x.bod, kMaxSide, dfmt) << "; }\n"
    << "  __device__ __forceinline__ double pnu(int q) const { return " << select(x.pnu, kMaxPart, dfmt) << "; }\n"
    << "  __device__ __forceinline__ double b() const { return " << lit(x.b) << "; }\n"
    << "  __device__ __forceinline__ double dnu() const { return " << lit(x.dnu) << "; }\n"
    << "  __device__ __forceinline__ double lnA0() const { return " << lit(x.lnA0) << "; }\n"
    << "  __device__ __forceinline__ double b0() const { return " << lit(x.b0) << "; }\n"
    << "  __device__ __forceinline__ double EaR0() const { return " << lit(x.EaR0) << "; }\n"
    << "  __device__ __forceinline__ double troe_a() const { return " << lit(x.troe_a) << "; }\n"
    << "  __device__ __forceinline__ double troe_invT3() const { return " << lit(x.troe_invT3) << "; }\n"
    << "  __device__ __forceinline__ double troe_invT1() const { return " << lit(x.troe_invT1) << "; }\n"
    << "  __device__ __forceinline__ double troe_T2() const { return " << lit(x.troe_T2) << "; }\n"
    << "  __device__ __forceinline__ int has_T2() const { return " << x.has_T2 << "; }\n";
  // third body: the same additions in the same order as the generic loop over efficiency entries
  const int ne = x.eff_end - x.eff_begin;
  o << "  template <class S, class LT>\n"
    << "  __device__ __forceinline__ double third_body(const MechView&, const LT& L, double Msum) const {\n"
    << "    double M = Msum;\n";
  for (int e = x.eff_begin; e < x.eff_end; ++e)
    o << "    M += " << lit(v.eff[e].alpha_minus_1) << " * L[S::C + " << v.eff[e].k << "];\n";
  o << "    return M;\n  }\n";
  std::vector<int> ek;
  std::vector<double> ea;
  for (int e = x.eff_begin; e < x.eff_end; ++e) {
    ek.push_back(v.eff[e].k);
    ea.push_back(v.eff[e].alpha_minus_1);
  }
  o << "  __device__ __forceinline__ int eff_begin() const { return 0; }\n"
    << "  __device__ __forceinline__ int eff_end() const { return " << ne << "; }\n";
  if (ne > 0) {
    o << "  __device__ __forceinline__ int eff_k(const MechView&, int q) const { return "
      << select(ek.data(), ne, ifmt) << "; }\n"
      << "  __device__ __forceinline__ double eff_am1(const MechView&, int q) const { return "
      << select(ea.data(), ne, dfmt) << "; }\n";
  } else {
    o << "  __device__ __forceinline__ int eff_k(const MechView&, int) const { return 0; }\n"
      << "  __device__ __forceinline__ double eff_am1(const MechView&, int) const { return 0.0; }\n";
  }
  o << "};\n";
}

// NVRTC: source -> cubin for sm_103a; 0, or -1 with *log
int compile_source(const std::string& src, std::vector<char>* cubin, std::string* log) {
  const Nvrtc& nv = nvrtc();
  if (!nv.ok) {
    *log = nv.why;
    return -1;
  }
  const std::string inc = "-I" + source_dir();
  // -default-device: the shared headers' unannotated functions (host tables, the C ABI
  // prototypes) are parsed as device functions; nothing here calls them
  std::vector<const char*> opts = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "-default-device", inc.c_str()};
  const char* verbose = std::getenv("RDE_JIT_PTXAS_VERBOSE");   // registers and spills into the log
  if (verbose && verbose[0] == '1') opts.push_back("--ptxas-options=-v");
  nvrtcProgram prog;
  nvrtcResult rc = nv.create(&prog, src.c_str(), "rde_jit.cu", 0, nullptr, nullptr);
  if (rc != NVRTC_SUCCESS) {
    *log = std::string("nvrtcCreateProgram: ") + nv.errstr(rc);
    return -1;
  }
  rc = nv.compile(prog, (int)opts.size(), opts.data());
  size_t ls = 0;
  nv.log_size(prog, &ls);
  std::string plog(ls, '\0');
  if (ls) nv.log(prog, &plog[0]);
  if (rc != NVRTC_SUCCESS) {
    *log = std::string("nvrtcCompileProgram: ") + nv.errstr(rc) + "\n" + plog;
    nv.destroy(&prog);
    return -1;
  }
  if (verbose && verbose[0] == '1') *log = plog;
  size_t cs = 0;
  nv.cubin_size(prog, &cs);
  cubin->resize(cs);
  nv.cubin(prog, cubin->data());
  nv.destroy(&prog);
  return 0;
}

// a compiled library and its kernels (forward: queue, plain; adjoint: record, reverse and
// the self-checkpointing reverse)
struct CacheEntry {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t queue = nullptr, plain = nullptr, third = nullptr;
};

std::mutex g_cache_mu;
std::map<std::string, CacheEntry>& cache() {
  static std::map<std::string, CacheEntry> c;
  return c;
}

}  // namespace

size_t thread_cell_shared_bytes(int K, int mech_bytes, int n_blocks) {
  const size_t N = (size_t)K + 1;
  const size_t lane = N * N + 6 * (size_t)K + 2 * N;   // the lane slots of chem_device.cuh (Slots<K>)
  return (size_t)mech_bytes + sizeof(double) * lane * kJitThreads +
         (n_blocks > 0 ? sizeof(long long) * (n_blocks + 1) : 0);
}

size_t wide_shared_bytes(int K, int mech_bytes, int n_blocks) {
  const size_t N = (size_t)K + 1;
  return (size_t)mech_bytes + sizeof(double) * N * N * kWideThreads +
         (n_blocks > 0 ? sizeof(long long) * (n_blocks + 1) : 0);
}

int wide_max_blocks(int K, int mech_bytes) {
  if (K > kWideMaxK) return -1;
  const size_t base = wide_shared_bytes(K, mech_bytes, 0);
  if (base > kSharedLimit) return -1;
  const long long room = (long long)((kSharedLimit - base) / sizeof(long long)) - 1;
  return (int)(room < kJitMaxBlocks ? room : kJitMaxBlocks);
}

int jit_max_species(int mech_bytes) {
  int K = 0;
  while (K < 64 && thread_cell_shared_bytes(K + 1, mech_bytes, kJitMaxBlocks) <= kSharedLimit) ++K;
  return K;
}

namespace {

// preamble, includes and the generated reaction sequence rde::jit::Reactions
std::string jit_common(const unsigned char* image, const char* include, int group) {
  const MechView v = mech_view(image);
  const int K = v.hdr->K, R = v.hdr->R;
  std::ostringstream o;
  o << "// generated: mechanism-specialised chemistry kernels, " << K << " species, " << R << " reactions\n"
    << "#if defined(__CUDACC_RTC__)\n"
    << "typedef signed char int8_t;\ntypedef short int16_t;\ntypedef int int32_t;\ntypedef long long int64_t;\n"
    << "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\ntypedef unsigned int uint32_t;\n"
    << "typedef unsigned long long uint64_t;\n"
    << "#endif\n"
    << "#include \"" << include << "\"\n"
    << "namespace rde {\nnamespace jit {\n";
  for (int r = 0; r < R; ++r) reaction_struct(o, v, r);
  // the reaction sequence; a compiler-only memory barrier after every `group` reactions
  // keeps shared-memory values from being carried in registers across the whole
  // sequence (which would exhaust the register file) while letting the reactions of a
  // group interleave
  if (group < 1) group = 1;
  o << "struct Reactions {\n"
    << "  template <class F>\n"
    << "  static __device__ __forceinline__ void each(const MechView& m, F&& f) {\n";
  for (int r = 0; r < R; ++r) {
    o << "    f(Rx" << r << "{m.rx[" << r << "]}, " << r << ");\n";
    if ((r + 1) % group == 0 || r == R - 1) o << "    asm volatile(\"\" ::: \"memory\");\n";
  }
  o << "  }\n};\n"
    << "}  // namespace jit\n}  // namespace rde\n";
  return o.str();
}

}  // namespace

std::string jit_source(const unsigned char* image, int method) {
  const int K = mech_view(image).hdr->K;
  const char* meth = method == RDE_METHOD_ROS2     ? "rde::kMethodRos2"
                     : method == RDE_METHOD_EXTRAP ? "rde::kMethodExtrap"
                                                   : "rde::kMethodRodas3";
  std::ostringstream o;
  // the forward step interleaves groups of 4 reactions (1.3 % faster than single reactions
  // on the 9-species field, 186 registers without spills); RDE_JIT_REACTION_GROUP overrides
  int group = 4;
  if (const char* g = std::getenv("RDE_JIT_REACTION_GROUP")) group = std::atoi(g);
  o << jit_common(image, "chem_kernel_body.cuh", group)
    << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", 1) rde_jit_queue(const rde::LaunchArgs a) {\n"
    << "  rde::advance_body<" << K << ", true, rde::RhsOf<rde::jit::Reactions>, " << meth << ">(a);\n}\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", 1) rde_jit_plain(const rde::LaunchArgs a) {\n"
    << "  rde::advance_body<" << K << ", false, rde::RhsOf<rde::jit::Reactions>, " << meth << ">(a);\n}\n";
  return o.str();
}

std::string jit_wide_source(const unsigned char* image) {
  const int K = mech_view(image).hdr->K;
  std::ostringstream o;
  int group = 4;
  if (const char* g = std::getenv("RDE_JIT_REACTION_GROUP")) group = std::atoi(g);
  // the wide queue kernel (RODAS3): 256 threads, species and vector slots in registers, the
  // cell state and stage vectors in a park area of one lane per thread of the persistent grid
  o << jit_common(image, "chem_kernel_body.cuh", group)
    << "extern \"C\" __global__ void __launch_bounds__(" << kWideThreads << ", 1) rde_jit_queue_w(const rde::LaunchArgs a) {\n"
    << "  rde::advance_body<" << K << ", true, rde::RhsOf<rde::jit::Reactions>, rde::kMethodRodas3, " << kWideThreads
    << ">(a);\n}\n";
  return o.str();
}

std::string jit_adjoint_source(const unsigned char* image) {
  const int K = mech_view(image).hdr->K;
  std::ostringstream o;
  // the adjoint keeps single-reaction groups: larger ones make its reverse kernel spill.
  // Stages per second-derivative evaluation: all four in one (the default; 10.24 s against
  // 10.82 s with two and 12.14 s with one on the 262,144-cell front-heavy field, despite
  // 576 bytes of spills), or 1 or 2 by RDE_JIT_HVP_DIRECTIONS
  int nd = 4;
  if (const char* e = std::getenv("RDE_JIT_HVP_DIRECTIONS")) nd = std::atoi(e);
  if (nd != 1 && nd != 2) nd = 4;
  o << jit_common(image, "chem_adjoint_body.cuh", 1)
    << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", 1) rde_jit_record(const rde::AdjArgs a) {\n"
    << "  rde::record_body<" << K << ", rde::jit::Reactions>(a);\n}\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", 1) rde_jit_reverse(const rde::AdjArgs a) {\n"
    << "  rde::reverse_body<" << K << ", rde::jit::Reactions, " << nd << ">(a);\n}\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", 1) rde_jit_reverse_self(const rde::AdjArgs a) {\n"
    << "  rde::reverse_body<" << K << ", rde::jit::Reactions, " << nd << ", true>(a);\n}\n";
  return o.str();
}

size_t adjoint_record_shared_bytes(int K, int mech_bytes) { return thread_cell_shared_bytes(K, mech_bytes, 0); }

size_t adjoint_reverse_shared_bytes(int K, int mech_bytes) {
  const size_t N = (size_t)K + 1;
  const size_t head = N * N + 9 * (size_t)K, dual = 18 * (size_t)K;   // the slots of AdjSlots<K>
  return (size_t)mech_bytes + sizeof(double) * ((head > dual ? head : dual) + 2 * N) * kJitThreads;
}

int jit_compile_only(const unsigned char* image, int part, std::string* log, double* seconds, size_t* cubin_bytes) {
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<char> cubin;
  const std::string src = part == 1   ? jit_adjoint_source(image)
                          : part == 3 ? jit_wide_source(image)
                                      : jit_source(image, part == 2 ? RDE_METHOD_ROS2 : RDE_METHOD_RODAS3);
  if (compile_source(src, &cubin, log) != 0) return -1;
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (cubin_bytes) *cubin_bytes = cubin.size();
  return 0;
}

namespace {

// compiles `src` (or takes it from the process cache) and returns its two kernels
int load_cached(const std::string& src, const char* name0, const char* name1, CacheEntry* entry, double* compile_s,
                std::string* log, const char* name2 = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = cache().find(src);
    if (it != cache().end()) {
      *entry = it->second;
      *compile_s = 0.0;
      return 0;
    }
  }
  std::vector<char> cubin;
  if (compile_source(src, &cubin, log) != 0) return -1;
  CacheEntry e0;
  cudaError_t e = cudaLibraryLoadData(&e0.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&e0.queue, e0.lib, name0);
  if (e == cudaSuccess && name1) e = cudaLibraryGetKernel(&e0.plain, e0.lib, name1);
  if (e == cudaSuccess && name2) e = cudaLibraryGetKernel(&e0.third, e0.lib, name2);
  if (e != cudaSuccess) {
    *log = std::string("loading the compiled kernels: ") + cudaGetErrorString(e);
    return -1;
  }
  *compile_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  std::lock_guard<std::mutex> lk(g_cache_mu);
  cache()[src] = e0;
  *entry = e0;
  return 0;
}

// shared-memory limit of a kernel on the current device and its CTAs per SM
int configure(cudaKernel_t k, size_t smem, int* fit, std::string* log, int threads = kJitThreads) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, reinterpret_cast<const void*>(k), threads, smem);
  if (e != cudaSuccess || *fit < 1) {
    *log = std::string("configuring the compiled kernels: ") + cudaGetErrorString(e);
    return -1;
  }
  return 0;
}

}  // namespace

int jit_build(const unsigned char* image, int mech_bytes, JitKernels* out, std::string* log, int method) {
  const int K = mech_view(image).hdr->K;
  if (K < 1 || K > jit_max_species(mech_bytes)) {
    *log = "species count outside the thread-per-cell kernels";
    return -1;
  }
  CacheEntry entry;
  double compile_s = 0.0;
  if (load_cached(jit_source(image, method), "rde_jit_queue", "rde_jit_plain", &entry, &compile_s, log) != 0)
    return -1;
  // per device and mechanism (outside any stream capture)
  const size_t smax = thread_cell_shared_bytes(K, mech_bytes, kJitMaxBlocks);
  int fit = 0, fit2 = 0;
  if (configure(entry.queue, smax, &fit, log) != 0 || configure(entry.plain, smax, &fit2, log) != 0) return -1;
  out->queue = entry.queue;
  out->plain = entry.plain;
  out->fit = fit;
  out->compile_s = compile_s;
  return 0;
}

int jit_build_wide(const unsigned char* image, int mech_bytes, JitKernels* out, std::string* log) {
  const int K = mech_view(image).hdr->K;
  const int wb = wide_max_blocks(K, mech_bytes);
  if (wb < 0) {
    *log = "species count outside the wide kernel";
    return -1;
  }
  CacheEntry entry;
  double compile_s = 0.0;
  if (load_cached(jit_wide_source(image), "rde_jit_queue_w", nullptr, &entry, &compile_s, log) != 0) return -1;
  int fw = 0;
  if (configure(entry.queue, wide_shared_bytes(K, mech_bytes, wb), &fw, log, kWideThreads) != 0) return -1;
  out->queue_w = entry.queue;
  out->wide_blocks = wb;
  out->fit_w = fw;
  return 0;
}

int jit_build_adjoint(const unsigned char* image, int mech_bytes, JitAdjKernels* out, std::string* log) {
  const int K = mech_view(image).hdr->K;
  if (K < 1 || K > jit_max_species(mech_bytes) ||
      adjoint_reverse_shared_bytes(K, mech_bytes) > kSharedLimit) {
    *log = "species count outside the adjoint kernels";
    return -1;
  }
  CacheEntry entry;
  double compile_s = 0.0;
  if (load_cached(jit_adjoint_source(image), "rde_jit_record", "rde_jit_reverse", &entry, &compile_s, log,
                  "rde_jit_reverse_self") != 0)
    return -1;
  int fit_self = 0;
  if (configure(entry.queue, adjoint_record_shared_bytes(K, mech_bytes), &out->fit_record, log) != 0 ||
      configure(entry.plain, adjoint_reverse_shared_bytes(K, mech_bytes), &out->fit_reverse, log) != 0 ||
      configure(entry.third, adjoint_reverse_shared_bytes(K, mech_bytes), &fit_self, log) != 0)
    return -1;
  out->record = entry.queue;
  out->reverse = entry.plain;
  out->reverse_self = entry.third;
  out->compile_s = compile_s;
  return 0;
}

bool jit_uses_wide(const JitKernels& k, const LaunchArgs& a) {
  const int fit = k.fit_w > 0 ? k.fit_w : 1;
  return k.queue_w && a.schedule != RDE_SCHED_PLAIN && a.threads == kWideThreads &&
         (!a.blocks || a.n_blocks <= k.wide_blocks) && a.park &&
         a.park_lanes >= (long long)a.num_sms * fit * kWideThreads;
}

cudaError_t jit_launch(const JitKernels& k, const LaunchArgs& a, cudaStream_t stream) {
  if (a.blocks && a.n_blocks > kJitMaxBlocks) return cudaErrorInvalidValue;
  const bool queue = a.schedule != RDE_SCHED_PLAIN;
  const bool wide = jit_uses_wide(k, a);
  const int threads = wide ? kWideThreads : kJitThreads;
  const size_t smem = wide ? wide_shared_bytes(a.K, a.mech_bytes, a.blocks ? a.n_blocks : 0)
                           : thread_cell_shared_bytes(a.K, a.mech_bytes, a.blocks ? a.n_blocks : 0);
  const long long blocks_needed = (a.n_total + threads - 1) / threads;
  long long grid = blocks_needed;
  if (queue) {
    const int fit = wide ? (k.fit_w > 0 ? k.fit_w : 1) : (k.fit > 0 ? k.fit : 1);
    const int per_sm = a.ctas_per_sm > 0 ? (a.ctas_per_sm < fit ? a.ctas_per_sm : fit) : fit;
    grid = blocks_needed < (long long)a.num_sms * per_sm ? blocks_needed : (long long)a.num_sms * per_sm;
  }
  if (grid < 1) grid = 1;
  LaunchArgs arg = a;
  void* params[] = {&arg};
  const cudaKernel_t kern = wide ? k.queue_w : (queue ? k.queue : k.plain);
  return cudaLaunchKernel(reinterpret_cast<const void*>(kern), dim3((unsigned)grid), dim3(threads), params, smem,
                          stream);
}

}  // namespace rde
