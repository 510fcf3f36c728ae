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

#if !defined(__CUDACC_RTC__)  /* run-time compiled kernels get these types from the compiler preamble */
#include <stddef.h>
#include <stdint.h>
#endif

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
#define RDE_ERR_UNSUPPORTED (-6)  /* mechanism size or call outside the compiled kernels */
#define RDE_ERR_ALIGN (-7)        /* a pointer is not 8-byte aligned */
#define RDE_ERR_WORKSPACE (-8)    /* caller workspace too small */
#define RDE_ERR_NOMEM (-9)        /* host or device allocation failed */
#define RDE_ERR_COMPILE (-10)     /* run-time compilation of a specialised kernel failed
                                     (only with RDE_LOAD_REQUIRE_SPECIALIZED) */

/* ---- rde_mech_load flags ------------------------------------------------------
 * By default a mechanism whose per-lane arrays fit a thread-per-cell kernel (up to
 * 9 species) gets kernels specialised to it at load time: the reactions become
 * straight-line code with their structure (species, orders, type, efficiencies,
 * falloff constants) as compile-time constants, compiled by NVRTC for sm_103a
 * (seconds, once per mechanism and process).  ln A and E stay run-time data, so
 * rde_mech_set_arrhenius needs no recompilation.  Without NVRTC, or if the
 * compilation fails, the handle uses the precompiled kernels.
 *
 * A call with threads_per_cta = 256 (QUEUE or AUTO schedule, RODAS3, K <= 16)
 * runs a wide specialised queue kernel instead: 256 threads per CTA, only each
 * lane's (K+1)^2 matrix in shared memory, its species and vector slots in
 * registers and its cell state and stage vectors in a park area of 4 (K+1)
 * doubles per lane of the persistent grid (12.5 MB at 9 species on a 152-SM GPU).
 * The handle's first such call compiles the kernel and allocates the park area
 * (host, synchronous; make it outside any stream capture; rde_chem_graph_create
 * does it before its capture).  It runs the operations of the 128-thread kernels
 * in the same order, but the compiler fuses multiply-adds differently when the
 * slots live in registers, so the two agree to rounding, not bitwise (each is
 * bitwise reproducible).  Its warps pass one CTA-wide barrier per attempt, so
 * they run the same stretch of code together.  Calls whose block table does not
 * fit beside its shared memory use the 128-thread kernels.  On the 9-species
 * field it is about 1.26x faster than the 128-thread kernel; AUTO (0) keeps the
 * 128-thread kernels, whose arithmetic the recorded-mode adjoint retraces and
 * which need no second compilation or park area. */
#define RDE_LOAD_GENERIC 1u                /* use only the precompiled kernels */
#define RDE_LOAD_REQUIRE_SPECIALIZED 2u    /* fail (RDE_ERR_COMPILE) rather than fall back */

/* ---- kernel variants (rde_chem_kernel_variant) ---------------------------- */
#define RDE_KERNEL_GENERIC 0       /* precompiled thread-per-cell kernel (2, 3 or 9 species) */
#define RDE_KERNEL_SPECIALIZED 1   /* thread-per-cell kernel compiled for this mechanism */
#define RDE_KERNEL_BLOCK 2         /* CTA-per-cell kernel */

/* ---- per-cell status (optional status[] output) -------------------------- */
#define RDE_CELL_OK 0
#define RDE_CELL_MAX_SUBSTEPS 1   /* attempts (accepted + rejected) reached max_substeps */
#define RDE_CELL_H_UNDERFLOW 2    /* step size fell below h_min */
#define RDE_CELL_BAD_STATE 3      /* input T, p or Y non-finite, or T <= 0 or p <= 0; untouched */
#define RDE_CELL_LU_SINGULAR 4    /* zero pivot in the LU of I/(h gamma) - J */
#define RDE_CELL_ADJ_MISMATCH 5   /* adjoint: the recorded integration did not take n_steps accepted steps */

/* ---- schedules ----------------------------------------------------------- */
#define RDE_SCHED_AUTO 0          /* library choice: QUEUE when a thread-per-cell kernel is compiled
                                     for the species count (2, 3, 9), else BLOCK */
#define RDE_SCHED_PLAIN 1         /* one launch-wide pass: one thread per cell (one CTA per cell
                                     when only the CTA-per-cell kernel serves the mechanism) */
#define RDE_SCHED_QUEUE 2         /* persistent CTAs; a lane whose cell finishes takes the next
                                     cell from a device work queue (substep-granular refill) */
#define RDE_SCHED_BLOCK 3         /* CTA-per-cell kernel for any species count: 128 threads share
                                     one cell's matrix, reactions and LU in shared memory;
                                     persistent CTAs take cells from the work queue.  The
                                     per-cell results agree with the thread-per-cell kernels to
                                     rounding (sums run in another fixed order). */

typedef struct rde_mech_s* rde_mech_t;

/* Integration methods (rde_chem_options.method).  The paper names no integrator.
 * Two L-stable Rosenbrock methods in the transformed Hairer-Wanner form with an
 * embedded error estimate (Hairer and Wanner, Solving ODEs II, Section IV.7):
 *   RODAS3  4 stages, order 3, embedded order 2 (Sandu et al. 1997); the default
 *   ROS2    2 stages, order 2, embedded order 1 (y + k1); gamma = 1 - 1/sqrt(2)
 * and a method of another family for comparison:
 *   EXTRAP  linearly implicit Euler extrapolation of fixed order 3 (the SEULEX
 *           family; Deuflhard, and Hairer and Wanner, Section IV.9): n = 1, 2, 3
 *           substeps of (I/h_n - J)(y_{i+1} - y_i) = f(y_i) with one J, extrapolated
 *           (Aitken-Neville, expansion in powers of h) to order 3; the error estimate
 *           is the difference to the order-2 entry.  The thread-per-cell kernels on
 *           the QUEUE (or AUTO) schedule only: the handle allocates a Jacobian scratch
 *           of (K+1)^2 doubles per resident lane (16 MB at 9 species) when the method
 *           is selected.
 * The adjoint and the CTA-per-cell kernel (RDE_SCHED_BLOCK) integrate RODAS3 only. */
#define RDE_METHOD_RODAS3 0
#define RDE_METHOD_ROS2 1
#define RDE_METHOD_EXTRAP 2

/* Integrator options.  Defaults: rtol 1e-8, atol 1e-12, h_min 1e-30 s,
 * facmax 5, facmin 0.2, safety 0.9, max_substeps 100000, method RODAS3.
 * Error norm: RMS over the K+1 unknowns of e_i / (atol + rtol max(|y_i|, |y_new,i|)).
 * Accept if <= 1; h <- h min(facmax', max(facmin, safety err^(-1/(q+1)))), with
 * q the order of the embedded estimate (2 for RODAS3 and EXTRAP, 1 for ROS2), facmax' = 1
 * right after a rejection; a non-finite estimate is a rejection with facmin. */
typedef struct {
  double rtol, atol, h_min, facmax, facmin, safety;
  int32_t max_substeps;
  int32_t method;           /* RDE_METHOD_RODAS3, RDE_METHOD_ROS2 or RDE_METHOD_EXTRAP */
} rde_chem_options;

/* One block of cells in structure-of-arrays layout.  All arrays are DEVICE memory.
 *   p      [n]        pressure in Pa, read only (constant over dt)
 *   T      [n]        temperature in K, in/out
 *   Y      [K][ldY]   mass fractions, species-major (Y[k*ldY + i]), in/out
 *   h_hint [n]        optional in/out: first substep size (min(dt, h_hint) if > 0,
 *                     else dt) and, on return, the controller's next proposed size
 *   status [n]        optional out: RDE_CELL_* code
 *   n_acc, n_rej [n]  optional out: accepted / rejected substeps
 *   n                 number of cells (>= 0), ldY >= n
 *   cycles [n]        optional out: the cell's measured cost, SM clock cycles from
 *                     the moment its lane (or CTA) takes the cell to the moment it
 *                     stores the result (clock64; the time the warp spent on it,
 *                     which includes waiting for the other lanes' attempts).  Cycles
 *                     of different SMs are not synchronised; each value is a
 *                     difference on one SM.  This is the per-cell load measure a
 *                     time-weighted partition of cells across ranks uses, as the
 *                     paper balances its ranks on measured time (Section 3.3.1). */
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
  int64_t* cycles;
} rde_block;

/* Extended call.  Either `cells` describes one block (blocks == NULL), or
 * `blocks` is a DEVICE array of n_blocks (1..1024) descriptors whose n sum to
 * n_total; all blocks are advanced in one launch.  `order`, if not NULL, is a
 * DEVICE array [n_total] of int64 global cell indices (a permutation) giving
 * the order in which the queue hands cells out, e.g. most expensive first.
 * The kernels read a device block table without the host checking it: a block
 * whose n is negative is treated as empty, and positions beyond the table's
 * total are never handed out. */
typedef struct {
  rde_block cells;
  const rde_block* blocks;
  int32_t n_blocks;
  int32_t schedule;
  int64_t n_total;
  double dt;
  const int64_t* order;
  int32_t threads_per_cta;  /* 0 or 128: the 128-thread kernels; 256: the wide queue
                               kernel (specialised RODAS3, QUEUE/AUTO schedule, else
                               RDE_ERR_UNSUPPORTED; rde_chem_advance_noalloc only after
                               an rde_chem_advance_ex call has built it) */
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
 *   flags      0, or RDE_LOAD_GENERIC / RDE_LOAD_REQUIRE_SPECIALIZED (see above)
 *   out        receives the handle on success; untouched on error
 * Host call, synchronous with respect to the current CUDA device, which the
 * handle is bound to.  Errors: RDE_ERR_NULL, RDE_ERR_PARSE, RDE_ERR_INVALID
 * (unbalanced elements, unknown species, bad NASA ranges, order > 3, ...),
 * RDE_ERR_UNSUPPORTED (more than 63 species, or a cell's arrays exceed the shared
 * memory of one CTA: (K+1)^2 + 11R doubles and more, about 100 KB for 53 species
 * and 325 reactions),
 * RDE_ERR_ARG (unknown flags), RDE_ERR_COMPILE, RDE_ERR_CUDA,
 * RDE_ERR_NOMEM. */
int rde_mech_load(const char* text, size_t len, int flags, rde_mech_t* out);

/* The kernel the AUTO schedule uses for this handle (RDE_KERNEL_*) and, for a
 * specialised kernel, the seconds its compilation took in this process (0 when it
 * came from the process-wide cache of compiled mechanisms).  Either pointer may be NULL. */
int rde_chem_kernel_variant(rde_mech_t h, int* variant, double* compile_seconds);

/* Release the handle and its device memory (synchronises its device). NULL is a no-op. */
int rde_mech_free(rde_mech_t h);

/* Species and reaction counts of a loaded mechanism. */
int rde_mech_info(rde_mech_t h, int* n_species, int* n_reactions);

int rde_chem_default_options(rde_chem_options* o);
/* Replace / read the handle's integrator options.  RDE_ERR_ARG unless
 * 0 < rtol, 0 <= atol, 0 < h_min, 0 < facmin <= 1 <= facmax, 0 < safety <= 1,
 * max_substeps >= 1 and method is one of RDE_METHOD_*.  Selecting ROS2 on a
 * handle with specialised kernels compiles its ROS2 kernels in this call (host,
 * synchronous; do it before any stream capture); RDE_ERR_UNSUPPORTED when no
 * thread-per-cell kernel exists for ROS2 (neither specialised nor precompiled for
 * 2, 3 or 9 species), in which case the options are left unchanged. */
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
 *     caches it for the rest of the process; make that first call before any
 *     stream capture begins.  The cached address assumes that the device's
 *     primary context lives until exit: after a cudaDeviceReset the library's
 *     module may load at another address, so do not call this entry point
 *     again in a process that has reset the device.
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

/* CUDA graph of n_steps consecutive steps of the same cells (state, and h_hint
 * if given, carried from step to step), for time loops such as the paper's 500 us
 * of simulated time split into flow steps (Section 3.2.2).  The call is captured
 * on an internal stream; the graph holds, per step, a memset of the handle's
 * scratch and one kernel launch, so replaying it costs one host call.
 *   c        the call to repeat (device arrays, block table, schedule, as in
 *            rde_chem_advance_ex); captured by value: the arrays it points to must
 *            stay valid while the graph exists
 *   n_steps  1..100000
 *   out      receives an opaque executable-graph handle
 * Errors: as rde_chem_advance_ex, RDE_ERR_ARG for n_steps, RDE_ERR_CUDA. */
int rde_chem_graph_create(rde_mech_t h, const rde_chem_call* c, int n_steps, void** out);
/* Replay the graph on `stream` (asynchronous). */
int rde_chem_graph_launch(void* graph, void* stream);
/* Destroy the graph (NULL is a no-op). */
int rde_chem_graph_destroy(void* graph);

/* Launch shape of the kernel that serves the handle's AUTO schedule (with
 * threads_per_cta = 0): threads per CTA, queue CTAs that fit per SM, and dynamic
 * shared memory per CTA (bytes, without a block table).  Any argument may be
 * NULL. */
int rde_chem_kernel_info(rde_mech_t h, int* threads_per_cta, int* max_ctas_per_sm, size_t* shared_bytes);

/* ---- discrete adjoint ------------------------------------------------------
 * Gradients of a loss through the chemistry step: given the cotangents gT, gY
 * of the final state, the step returns d loss / d(T0, Y0) per cell and
 * d loss / d(ln A_r), d loss / d(E_r) summed over cells, for mechanism
 * calibration and sensitivity studies of the source terms of Eqs. 20-21.  The
 * derivative is that of the discrete map the integrator computes, with each
 * cell's sequence of accepted step sizes held fixed (the step-size controller is
 * not differentiated).  ln A_r is that of k_inf for falloff reactions; E_r is in
 * J/mol.  The adjoint re-integrates each cell from (T0, Y0) with the forward
 * step's arithmetic (no h_hint: the first step is dt), recording its accepted
 * steps, and sweeps them backwards.  Kernels: thread per cell where a
 * thread-per-cell kernel serves the mechanism (precompiled for 2, 3 and 9
 * species, or specialised at load time), else, or with schedule =
 * RDE_SCHED_BLOCK, one CTA of 128 threads per cell for any K + 1 <= 64 (the
 * 53-species stress mechanism), which always recomputes the stages.
 *
 * rde_chem_advance_adjoint (below) is self-contained: it needs only the step's
 * input state, dt and the cotangents, and a workspace of
 * rde_chem_adjoint_workspace(h, n_cells, dt) bytes.  It runs in the
 * self-checkpointing mode: the re-integration keeps S checkpoints per cell
 * (thread per cell; per CTA for the CTA-per-cell adjoint), each the state, time,
 * proposed and accepted step size of one accepted step, at every s-th step
 * where s is the smallest power of two with (steps of the cell) <= S s: when
 * the S entries are full, every other one is dropped and s doubles.  The
 * reverse sweep then reads each step from its checkpoint (s = 1) or replays
 * the s steps of a segment from the segment's checkpoint with the same
 * arithmetic (checked bit for bit against the next checkpoint; a cell whose
 * replay does not retrace its steps gets RDE_CELL_ADJ_MISMATCH and zero
 * gradients) and recomputes each step's stages.  S is the largest power of two
 * up to 1024 (4096 per CTA) whose layout the workspace holds, at least 16; the
 * query sizes for S = 512, or 1024 where that layout is smaller (few cells), and
 * 4096 per CTA.  A cell of at most S steps costs no replay.
 *
 * rde_chem_advance_adjoint_ex takes the same arguments as a struct and, when the
 * caller passes the forward pass's accepted step counts (n_acc of
 * rde_chem_advance_ex with the same options and parameters, no h_hint), the
 * recorded mode: the re-integration writes y_n and h_n of every accepted step
 * into a pool at per-cell offsets, in two memory modes chosen by the workspace:
 *   - step checkpoints (rde_chem_adjoint_workspace_steps bytes): the reverse
 *     sweep recomputes each step's Jacobian, LU factors and stages from y_n;
 *   - stage checkpoints (rde_chem_adjoint_workspace_checkpointed bytes or more):
 *     the re-integration also stores each accepted step's LU factors and stage
 *     vectors, (N^2 + 4N + 1) doubles a step with N = K + 1, and the reverse sweep
 *     reads them instead of recomputing (about 1.1 KB a step at 9 species).
 * All modes give the gradient of the same discrete map; they differ by rounding
 * only (recomputed stages are not bitwise those of the re-integration).  The
 * CTA-per-cell adjoint re-integrates with the CTA-per-cell step, so its n_steps
 * must come from a forward pass with RDE_SCHED_BLOCK (which is what AUTO takes for
 * such a mechanism).  The thread-per-cell adjoint re-integrates with the
 * arithmetic of the 128-thread kernels: take n_steps from a forward call with
 * threads_per_cta = 0 or 128.  The wide 256-thread queue kernel rounds differently
 * (its slots live in registers, so the compiler fuses operations differently);
 * its counts agree except where rounding flips a step decision, and such a cell
 * gets RDE_CELL_ADJ_MISMATCH. */
typedef struct {
  int64_t n;                 /* cells (single block) */
  const double* p;           /* [n] Pa */
  const double* T0;          /* [n] K, the step's input state */
  const double* Y0;          /* [K][ldY] */
  int64_t ldY;
  double dt;
  const int32_t* n_steps;    /* [n] accepted steps of each cell's forward integration, or
                                NULL: self-checkpointing mode (total_steps is ignored) */
  int64_t total_steps;       /* sum of n_steps (sizes the workspace); a cell whose records
                                would end beyond it gets RDE_CELL_ADJ_MISMATCH */
  const double* gT;          /* [n] cotangent of the final T */
  const double* gY;          /* [K][ldY] cotangent of the final Y */
  double* gT0;               /* [n] out */
  double* gY0;               /* [K][ldY] out */
  double* g_lnA;             /* [R] out, summed over cells */
  double* g_E;               /* [R] out, per J/mol, summed over cells */
  int32_t* status;           /* optional [n] out: RDE_CELL_* (failed cells get zero gradients) */
  void* workspace;           /* device memory, 256-byte aligned: see the workspace queries */
  size_t workspace_bytes;
  int32_t schedule;          /* RDE_SCHED_AUTO (0), or RDE_SCHED_BLOCK for the CTA-per-cell
                                adjoint */
} rde_adjoint_call;

/* Device workspace (bytes) of rde_chem_advance_adjoint for n_cells cells of this
 * handle (its mechanism and options: a cell takes at most max_substeps steps) in
 * the self-checkpointing mode: about n_cells * 512 * (K + 4) * 8 bytes for the
 * thread-per-cell adjoint (27 MB per 1,000 cells at 9 species) plus per-lane
 * scratch.  dt must be finite and > 0; it does not change the size.  0 for a NULL
 * handle, n_cells < 0 or a bad dt. */
size_t rde_chem_adjoint_workspace(rde_mech_t h, int64_t n_cells, double dt);

/* The adjoint of one step as the survey of the method's boundary states it:
 * self-contained (self-checkpointing mode, AUTO schedule, no per-cell status).
 *   p [n], T0 [n], Y0 [K][n] (ldY = n): the step's input, device memory
 *   gT [n], gY [K][n]: cotangents of the step's output
 *   gT0 [n], gY0 [K][n], g_lnA [R], g_E [R]: outputs (device memory)
 *   workspace, ws_bytes: device memory, 256-byte aligned; the call takes the
 *                        largest S (a power of two, 16 .. 1024) whose layout fits,
 *                        RDE_ERR_WORKSPACE if none does (the per-lane replay
 *                        segment holds max_substeps / S steps, so a small S needs a
 *                        large segment)
 * Asynchronous on `stream` (the first call of a handle with specialised kernels
 * compiles its adjoint kernels on the host first).  Errors as
 * rde_chem_advance_adjoint_ex. */
int rde_chem_advance_adjoint(rde_mech_t h, int64_t n_cells, const double* p, const double* T0, const double* Y0,
                             double dt, const double* gT, const double* gY, double* gT0, double* gY0, double* g_lnA,
                             double* g_E, void* workspace, size_t ws_bytes, void* stream);

/* Device workspace (bytes) of the recorded mode of rde_chem_advance_adjoint_ex for
 * n_cells cells with total_steps accepted steps (step checkpoints; the stages are
 * recomputed). 0 for a NULL handle or negative sizes. */
size_t rde_chem_adjoint_workspace_steps(rde_mech_t h, int64_t n_cells, int64_t total_steps);

/* Device workspace (bytes) of the same adjoint with stage checkpoints: the above plus
 * total_steps * (N^2 + 4N + 1) doubles; the plain size where only the CTA-per-cell
 * adjoint serves the mechanism.  The paper keeps no adjoint; stage checkpointing
 * trades this memory for the reverse sweep's recomputation. */
size_t rde_chem_adjoint_workspace_checkpointed(rde_mech_t h, int64_t n_cells, int64_t total_steps);

/* The adjoint with the arguments of rde_adjoint_call; asynchronous on `stream`
 * (the first call of a handle with specialised kernels compiles the mechanism's
 * adjoint kernels on the host first: do it before any stream capture).
 * Errors: RDE_ERR_NULL, RDE_ERR_ARG (n < 0, dt, ldY < n, total_steps < 0),
 * RDE_ERR_ALIGN, RDE_ERR_WORKSPACE (workspace smaller than required),
 * RDE_ERR_UNSUPPORTED (no adjoint kernel fits the mechanism, or method ROS2),
 * RDE_ERR_CUDA. */
int rde_chem_advance_adjoint_ex(rde_mech_t h, const rde_adjoint_call* c, void* stream);

/* Read or replace the Arrhenius parameters of every reaction: ln A in SI units
 * (of k_inf for falloff reactions) and E in J/mol.  Host arrays of R values;
 * replacing re-uploads the mechanism tables (synchronous). */
int rde_mech_get_arrhenius(rde_mech_t h, double* lnA, double* E);
int rde_mech_set_arrhenius(rde_mech_t h, const double* lnA, const double* E);

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
