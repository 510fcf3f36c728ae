/*
 * rde_chem_selftest.h - test hooks of the chemistry library (not part of the
 * chemistry step itself).
 *
 * The step evaluates its Arrhenius rates and equilibrium constants with the
 * library's own table-driven FP64 exp and ln T with its own table-driven log
 * (Tang's table-driven method); this entry point exposes those two functions
 * so that tests can bound their error and check that host and device agree.
 */
#ifndef RDE_CHEM_SELFTEST_H
#define RDE_CHEM_SELFTEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y[i] = f(x[i]) for i < n, f = exp (fn == 0) or natural log (fn == 1).
 *   on_device == 0: x, y are host arrays, evaluated on the host (synchronous);
 *   on_device == 1: x, y are device arrays, evaluated by a kernel on `stream`
 *                   (a cudaStream_t as void*); the call synchronises the stream.
 * Errors: RDE_ERR_NULL (x or y NULL with n > 0), RDE_ERR_ARG (n < 0, fn or
 * on_device out of range), RDE_ERR_CUDA. */
int rde_selftest_math(int fn, int64_t n, const double* x, double* y, int on_device, void* stream);

/* Generates the mechanism-specialised kernel source for an RDEMECH 1 text and
 * compiles it with NVRTC for sm_103a, without loading it (no GPU needed).
 *   part                0: the RODAS3 forward kernels, 1: the adjoint's record and reverse
 *                       kernels, 2: the ROS2 forward kernels, 3: the wide (256-thread)
 *                       RODAS3 queue kernel
 *   source, source_len  optional: receives the generated source (NUL-terminated,
 *                       truncated to source_len - 1 characters)
 *   log, log_len        optional: receives the compiler log on failure
 *   seconds, cubin_bytes optional: compilation wall time and cubin size
 * Errors: RDE_ERR_NULL, RDE_ERR_ARG (part), RDE_ERR_PARSE, RDE_ERR_INVALID, RDE_ERR_COMPILE. */
int rde_selftest_jit_compile(const char* text, size_t len, int part, char* source, size_t source_len, char* log,
                             size_t log_len, double* seconds, size_t* cubin_bytes);

/* Batched LU with partial pivoting of `batch` row-major n x n matrices (n <= 56),
 * in place: P A = L U with unit lower L below the diagonal and U on and above it;
 * piv[b*n + j] is the row swapped with row j at step j (0-based), info[b] the first
 * zero pivot (1-based, 0 if none).  A blocked right-looking factorisation, one warp
 * per matrix, whose trailing update runs on the FP64 tensor cores (dmma = 1: DMMA,
 * mma.sync m8n8k4) or the CUDA cores (dmma = 0: DFMA); everything else is the same
 * code.  It exists to compare the two paths for the 54 x 54 systems of a
 * 53-species mechanism.  A, piv, info: device memory; asynchronous on `stream`.
 * Errors: RDE_ERR_NULL, RDE_ERR_ARG (n outside 1..56, batch < 0, dmma not 0/1),
 * RDE_ERR_CUDA. */
int rde_selftest_batched_lu(int dmma, int64_t batch, int n, double* A, int32_t* piv, int32_t* info, void* stream);

/* Workspace (bytes) of the self-checkpointing adjoint (rde_chem_advance_adjoint, or
 * rde_chem_advance_adjoint_ex without n_steps) laid out for exactly S checkpoints
 * per cell (per CTA when block != 0: the CTA-per-cell adjoint), so that tests can
 * make the adjoint replay segments.  A call given exactly these bytes uses S.
 * rde_mech_t is passed as void*.  0 for a NULL handle, n_cells < 0 or S not a
 * power of two in [16, 4096]. */
size_t rde_selftest_adjoint_self_workspace(void* h, int64_t n_cells, int S, int block);

#ifdef __cplusplus
}
#endif
#endif /* RDE_CHEM_SELFTEST_H */
