// Mechanism-specialised thread-per-cell kernels, compiled at load time.
//
// The generic kernels read every reaction's structure (species, orders, type,
// efficiencies, falloff constants) from the mechanism image inside a loop over
// reactions, which costs table loads, index arithmetic and branches per reaction.
// For a given mechanism the library can instead generate one descriptor type per
// reaction whose structure is a set of compile-time constants, and compile the
// same kernel body (chem_kernel_body.cuh) over the unrolled sequence of reactions
// with NVRTC for sm_103a.  ln A and E/R are still read from the image at run time,
// so rde_mech_set_arrhenius needs no recompilation.  NVRTC is opened with dlopen;
// without it (or if compilation fails) the handle keeps the precompiled kernels.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "chem_launch.h"

namespace rde {

struct JitKernels {
  cudaKernel_t queue = nullptr;
  cudaKernel_t plain = nullptr;
  int fit = 0;          // queue CTAs per SM
  double compile_s = 0; // wall time of the compilation (0 when taken from the process cache)
  // The wide queue kernel (RODAS3; jit_build_wide): 256 threads per CTA, only the N x N
  // matrix in shared memory (the species and vector slots in registers, the cell state
  // and stage vectors in a global park area), so that two warps share each SM
  // sub-partition.  A call selects it with threads = 256 (QUEUE schedule, block table of
  // at most wide_blocks entries, park area given).
  cudaKernel_t queue_w = nullptr;
  int fit_w = 0;
  int wide_blocks = -1;
};

// The adjoint's record and reverse kernels specialised to a mechanism (compiled on the
// first adjoint call of a handle).
struct JitAdjKernels {
  cudaKernel_t record = nullptr;
  cudaKernel_t reverse = nullptr;
  cudaKernel_t reverse_self = nullptr;   // the reverse sweep of the self-checkpointing mode
  int fit_record = 0, fit_reverse = 0;
  double compile_s = 0;
};

// Largest species count of a thread-per-cell kernel (its lane slots fit in shared memory).
int jit_max_species(int mech_bytes);

// Source of the specialised kernels for a packed image and integration method
// (RDE_METHOD_*; exposed for tests and inspection).
std::string jit_source(const unsigned char* image, int method = RDE_METHOD_RODAS3);

// Generates, compiles and loads the kernels for `image` on the current device (a process-wide
// cache keyed by the source avoids recompiling a mechanism); returns 0, or -1 with *log set.
int jit_build(const unsigned char* image, int mech_bytes, JitKernels* out, std::string* log,
              int method = RDE_METHOD_RODAS3);

// Source of the wide queue kernel (RODAS3, 256 threads per CTA).
std::string jit_wide_source(const unsigned char* image);

// Compiles and loads the wide queue kernel into out->queue_w (fit_w, wide_blocks); 0, or
// -1 with *log (K > 16, or the matrix slots do not fit shared memory).
int jit_build_wide(const unsigned char* image, int mech_bytes, JitKernels* out, std::string* log);

// Source of the specialised adjoint kernels.
std::string jit_adjoint_source(const unsigned char* image);

// As jit_build, for the adjoint kernels.
int jit_build_adjoint(const unsigned char* image, int mech_bytes, JitAdjKernels* out, std::string* log);

// Generates and compiles only (no device needed) the forward (part 0) or adjoint (part 1)
// kernels: 0, or -1 with *log; *seconds and *cubin_bytes describe the compilation.
int jit_compile_only(const unsigned char* image, int part, std::string* log, double* seconds, size_t* cubin_bytes);

// Dynamic shared bytes of the adjoint's record and reverse kernels for K species.
size_t adjoint_record_shared_bytes(int K, int mech_bytes);
size_t adjoint_reverse_shared_bytes(int K, int mech_bytes);

// Launches like launch_advance (same LaunchArgs, same schedules) on `stream`.
cudaError_t jit_launch(const JitKernels& k, const LaunchArgs& a, cudaStream_t stream);

// Whether jit_launch serves the call `a` with the wide kernels.
bool jit_uses_wide(const JitKernels& k, const LaunchArgs& a);

// Dynamic shared bytes of a wide kernel for K species.
size_t wide_shared_bytes(int K, int mech_bytes, int n_blocks);

// Dynamic shared bytes of a thread-per-cell kernel for K species (n_blocks = 0: no block table).
size_t thread_cell_shared_bytes(int K, int mech_bytes, int n_blocks);

}  // namespace rde
