/*
 * rde_chem.h - C ABI of the GB300 (sm_103a) per-cell chemistry step.
 *
 * The operation.  The paper's reacting-flow solver (Section 2.1) splits the
 * chemistry from the flow: inside the energy and species solve of each PIMPLE
 * iteration, the "detailed chemistry model" supplies the species source terms
 * omega_dot_i of Eq. 21 and the heat release Q_dot of Eq. 20 (Appendix A).
 * This library advances every cell's (T, Y_k) at its fixed pressure p over one
 * flow time step dt as a closed, adiabatic, constant-pressure reactor:
 *
 *     dY_k/dt = W_k omega_dot_k / rho,     dT/dt = -sum_k H_k omega_dot_k / (rho c_p)
 *
 * with Arrhenius forward rates, reverse rates from NASA-7 equilibrium constants,
 * three-body and Lindemann/Troe falloff terms, an analytic Jacobian, a dense LU
 * with partial pivoting and adaptive L-stable Rosenbrock substeps (RODAS3, four
 * stages, order 3 with an embedded order-2 error estimate) under per-cell error
 * control.  Chemistry cost is uneven across cells: the paper notes that
 * convergence of chemical reactions takes longer where combustion occurs
 * (Section 1) and balances its CPU ranks on measured time rather than cell
 * count (Section 3.3.1); the queue schedule below is the single-GPU analogue.
 *
 * Conventions for every call.
 *   - Return 0 (RDE_OK) on success, a negative RDE_ERR_* code on an argument,
 *     parse or CUDA error.  Argument errors are detected on the host before
 *     anything is launched; rde_strerror() names a code and
 *     rde_last_error_message() gives the detail of the calling thread's last
 *     error.
 *   - Device pointers are caller-owned CUDA device memory (for example torch
 *     tensors); the library never frees them.  Pointers to doubles must be
 *     8-byte aligned.  The handle owns the mechanism's device tables and a small
 *     device scratch area (work-queue counter and statistics).
 *   - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Compute calls are asynchronous on that stream.
 *   - Per-cell integration failures never fail a call: they are reported in
 *     the optional per-cell status array and counted in the handle's
 *     statistics.  A failed cell keeps its last accepted state.
 *   - Identical inputs give bitwise identical outputs (no floating-point
 *     atomics); the PLAIN and QUEUE schedules give identical per-cell results.
 *   - A handle's statistics and work-queue counter are shared by its calls:
 *     calls on one handle must not run concurrently on different streams.
 */
#ifndef RDE_CHEM_H
#define RDE_CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes --------------------------------------------------------- */
#define RDE_OK 0
#define RDE_ERR_NULL (-1)         /* a required pointer is NULL */
#define RDE_ERR_ARG (-2)          /* bad size, time step, option or layout */
#define RDE_ERR_PARSE (-3)        /* mechanism text malformed */
#define RDE_ERR_INVALID (-4)      /* mechanism inconsistent (element balance, ranges, ...) */
#define RDE_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define RDE_ERR_UNSUPPORTED (-6)  /* mechanism size outside the compiled kernels */
#define RDE_ERR_ALIGN (-7)        /* a pointer is not 8-byte aligned */
#define RDE_ERR_WORKSPACE (-8)    /* caller workspace too small */
#define RDE_ERR_NOMEM (-9)        /* host or device allocation failed */

/* ---- per-cell status (optional status[] output) -------------------------- */
#define RDE_CELL_OK 0
#define RDE_CELL_MAX_SUBSTEPS 1   /* attempts (accepted + rejected) reached max_substeps */
#define RDE_CELL_H_UNDERFLOW 2    /* step size fell below h_min */
#define RDE_CELL_BAD_STATE 3      /* input T, p or Y non-finite, or T <= 0 or p <= 0; untouched */
#define RDE_CELL_LU_SINGULAR 4    /* zero pivot in the LU of I/(h gamma) - J */

/* ---- schedules ----------------------------------------------------------- */
#define RDE_SCHED_AUTO 0          /* library choice (currently QUEUE) */
#define RDE_SCHED_PLAIN 1         /* one thread per cell, one launch-wide pass */
#define RDE_SCHED_QUEUE 2         /* persistent CTAs; a lane whose cell finishes takes the next
                                     cell from a device work queue (substep-granular refill) */

typedef struct rde_mech_s* rde_mech_t;

/* Integrator options.  Defaults: rtol 1e-8, atol 1e-12, h_min 1e-30 s,
 * facmax 5, facmin 0.2, safety 0.9, max_substeps 100000.
 * Error norm: RMS over the K+1 unknowns of e_i / (atol + rtol max(|y_i|, |y_new,i|)).
 * Accept if <= 1; h <- h min(facmax', max(facmin, safety err^(-1/3))), facmax' = 1
 * right after a rejection; a non-finite estimate is a rejection with facmin. */
typedef struct {
  double rtol, atol, h_min, facmax, facmin, safety;
  int32_t max_substeps;
  int32_t reserved;
} rde_chem_options;

/* One block of cells in structure-of-arrays layout.  All arrays are DEVICE memory.
 *   p      [n]        pressure in Pa, read only (constant over dt)
 *   T      [n]        temperature in K, in/out
 *   Y      [K][ldY]   mass fractions, species-major (Y[k*ldY + i]), in/out
 *   h_hint [n]        optional in/out: first substep size (min(dt, h_hint) if > 0,
 *                     else dt) and, on return, the controller's next proposed size
 *   status [n]        optional out: RDE_CELL_* code
 *   n_acc, n_rej [n]  optional out: accepted / rejected substeps
 *   n                 number of cells (>= 0), ldY >= n                              */
typedef struct {
  const double* p;
  double* T;
  double* Y;
  double* h_hint;
  int32_t* status;
  int32_t* n_acc;
  int32_t* n_rej;
  int64_t n;
  int64_t ldY;
} rde_block;

/* Extended call.  Either `cells` describes one block (blocks == NULL), or
 * `blocks` is a DEVICE array of n_blocks (1..1024) descriptors whose n sum to
 * n_total; all blocks are advanced in one launch.  `order`, if not NULL, is a
 * DEVICE array [n_total] of int64 global cell indices (a permutation) giving
 * the order in which the queue hands cells out, e.g. most expensive first. */
typedef struct {
  rde_block cells;
  const rde_block* blocks;
  int32_t n_blocks;
  int32_t schedule;
  int64_t n_total;
  double dt;
  const int64_t* order;
  int32_t threads_per_cta;  /* 0: default (128) */
  int32_t ctas_per_sm;      /* 0: default; QUEUE schedule only */
} rde_chem_call;

/* Counters of the most recent compute call on the handle. */
typedef struct {
  int64_t cells;            /* cells processed */
  int64_t accepted;         /* accepted substeps, all cells */
  int64_t rejected;         /* rejected substeps, all cells */
  int64_t failed;           /* cells with status != RDE_CELL_OK */
  int64_t max_attempts;     /* largest accepted + rejected count of one cell */
  int64_t reserved[3];
} rde_chem_stats;

/* Parse, validate and upload a mechanism written in the RDEMECH 1 text format
 * (ELEMENTS / SPECIES with NASA-7 fits / REACTIONS with ELEM, THREEBODY,
 * LINDEMANN or TROE records; A in mol-cm-s, E in kJ/mol, W in g/mol).  The
 * paper's mechanism (Section 2.1) is a detailed H2/air set read the same way.
 *   text, len  the file contents (need not be NUL-terminated)
 *   flags      0 (reserved)
 *   out        receives the handle on success; untouched on error
 * Host call, synchronous with respect to the current CUDA device, which the
 * handle is bound to.  Errors: RDE_ERR_NULL, RDE_ERR_PARSE, RDE_ERR_INVALID
 * (unbalanced elements, unknown species, bad NASA ranges, order > 3, ...),
 * RDE_ERR_UNSUPPORTED (species count without a compiled kernel), RDE_ERR_CUDA,
 * RDE_ERR_NOMEM. */
int rde_mech_load(const char* text, size_t len, int flags, rde_mech_t* out);

/* Release the handle and its device memory (synchronises its device). NULL is a no-op. */
int rde_mech_free(rde_mech_t h);

/* Species and reaction counts of a loaded mechanism. */
int rde_mech_info(rde_mech_t h, int* n_species, int* n_reactions);

int rde_chem_default_options(rde_chem_options* o);
/* Replace / read the handle's integrator options.  RDE_ERR_ARG unless
 * 0 < rtol, 0 <= atol, 0 < h_min, 0 < facmin <= 1 <= facmax, 0 < safety <= 1,
 * max_substeps >= 1. */
int rde_chem_set_options(rde_mech_t h, const rde_chem_options* o);
int rde_chem_get_options(rde_mech_t h, rde_chem_options* o);

/* Advance n_cells cells over dt (seconds) with the default QUEUE schedule.
 *   p [n], T [n], Y [K][n] as in rde_block with ldY = n (device memory).
 * Errors: RDE_ERR_NULL (handle or, with n > 0, an array), RDE_ERR_ARG (n < 0,
 * dt <= 0 or non-finite), RDE_ERR_ALIGN, RDE_ERR_CUDA (launch failure).
 * n_cells == 0 returns RDE_OK without launching. */
int rde_chem_advance(rde_mech_t h, int64_t n_cells, const double* p, double* T, double* Y, double dt,
                     void* stream);

/* Advance with optional outputs, block tables, schedule and launch shape. */
int rde_chem_advance_ex(rde_mech_t h, const rde_chem_call* c, void* stream);

/* Same step as rde_chem_advance_ex, for callers that must not allocate device
 * memory during the call: code running while a CUDA stream is being captured
 * into a graph, real-time or latency-critical loops that forbid allocator
 * calls, and hosts whose device memory is owned by another allocator (for
 * example a framework's caching allocator that must see every allocation).
 * The paper has no counterpart; it is a deployment convenience.
 *
 * The work-queue counter and the per-call statistics, which the other entry
 * points keep in a small buffer that rde_mech_load allocates for the handle,
 * live here in one library-wide static device array of 256 bytes
 * (RDE_NOALLOC_SCRATCH_BYTES), present on every GPU that loads the library
 * until the process exits.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  The caller still passes the cells
 * (c, as in rde_chem_advance_ex) and the mechanism handle.
 *   - The first call on each device looks up the array's device address and
 *     caches it; make that first call before any stream capture begins.
 *   - The array is shared by every call and keeps the last call's contents;
 *     the call clears the counters it needs (an asynchronous memset on
 *     `stream`).  Calls whose kernels overlap on the GPU (on different streams
 *     or threads) race on it and must be serialised by the caller.
 *   - Statistics of this call are not kept: pass status / n_acc / n_rej arrays
 *     in c to observe per-cell outcomes.  rde_chem_get_stats does not see it.
 * Errors: as rde_chem_advance_ex, plus RDE_ERR_WORKSPACE if the call would need
 * more scratch than RDE_NOALLOC_SCRATCH_BYTES, and RDE_ERR_CUDA if the address
 * lookup fails. */
#define RDE_NOALLOC_SCRATCH_BYTES 256
int rde_chem_advance_noalloc(rde_mech_t h, const rde_chem_call* c, void* stream);

/* Synchronise `stream` and read the counters of the handle's last compute call. */
int rde_chem_get_stats(rde_mech_t h, void* stream, rde_chem_stats* out);

/* Synchronise `stream` and return the number of failed cells of the last call. */
int rde_chem_status(rde_mech_t h, void* stream, int64_t* n_failed);

/* Static description of a code. */
const char* rde_strerror(int code);

/* Detail of the calling thread's most recent error (empty if none). */
const char* rde_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* RDE_CHEM_H */
