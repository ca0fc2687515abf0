/*
 * flups_gpu.h -- C ABI of the GB300 Fourier Poisson solver (FLUPS method,
 * arXiv 2211.07777).
 *
 * The library solves lap(phi) = f (Section "Methodology", eq. poisson) and the
 * Biot-Savart variant lap(u) = curl(f) (Section "Application: the
 * Biot-Savart solver", eq. biotsavart) on a uniform 3D grid, each face of
 * each direction being periodic, even, odd or unbounded, with cell- or
 * node-centred data (Section 2.1).  The solution is u = G * f computed as
 * u^ = G^ f^ after a sequence of 1D transforms, one direction at a time.
 *
 * Conventions common to every entry point:
 *   - Every function returns FLUPS_OK (0) on success or a negative
 *     flups_status; none aborts, exits or throws across the ABI.
 *   - Field arrays live in device memory, are contiguous and x-fastest: value
 *     (i, j, k) is at i + n[0] * (j + n[1] * k).  A vector field (ncomp = 3)
 *     is its 3 components back to back.  Element type: float (FLUPS_F32) or
 *     double (FLUPS_F64), per the topology.
 *   - Sizes per direction: N = L / h cells (given through h and L, must be
 *     an integer).  Cell-centred data hold N values (x_j = (j + 1/2) h);
 *     node-centred data hold N + 1 values (x_j = j h), except that a
 *     node-centred periodic direction may also hold N values (the duplicate
 *     f_N omitted).  N must be of the form 2^a 3^b with N >= 4; the
 *     transform length (N, 2N or 4N per direction type) must not exceed 4096.
 *   - Streams are `cudaStream_t` passed as `void*` (NULL = legacy default).
 *   - Not thread safe per solver: one solver is used by one host thread and
 *     one stream at a time.  Distinct solvers are independent.
 */
#ifndef FLUPS_GPU_H
#define FLUPS_GPU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  FLUPS_OK = 0,
  FLUPS_EINVAL = -1,   /* null pointer, bad enum, bad argument value */
  FLUPS_EBC = -2,      /* inadmissible boundary conditions (periodic on one face only, mismatched vector BCs) */
  FLUPS_ESIZE = -3,    /* unsupported grid size (not 2^a 3^b, too large, too small) */
  FLUPS_ENOMEM = -4,   /* device or host allocation failed */
  FLUPS_ECUDA = -5,    /* a CUDA runtime call failed (see flups_last_cuda_error) */
  FLUPS_EGREEN = -6,   /* Green kernel not available for these boundary conditions */
  FLUPS_ESTATE = -7,   /* call out of order (e.g. solve before setup) */
  FLUPS_EDEVICE = -8   /* a kernel's bounded wait gave up (see flups_solver_check): the result is not valid */
} flups_status;

/* Face conditions (Section 2.2, 2.3). */
typedef enum { FLUPS_EVEN = 0, FLUPS_ODD = 1, FLUPS_PER = 3, FLUPS_UNB = 4 } flups_bc;
/* Data layout (Section 2.1). */
typedef enum { FLUPS_CELL = 0, FLUPS_NODE = 1 } flups_center;
/* Arithmetic of the transforms.  FLUPS_F64E: FP64 arrays (as FLUPS_F64) with
 * the transforms in double-float arithmetic on the FP32 units (about 48
 * significant bits, error within the FP64 path's 1e-12 bound); every size,
 * boundary condition, kernel and operator of the other paths. */
typedef enum { FLUPS_F32 = 0, FLUPS_F64 = 1, FLUPS_F64E = 2 } flups_prec;
/* Operator. */
typedef enum { FLUPS_POISSON = 0, FLUPS_BIOT_SAVART = 1 } flups_op;
/* Green kernels (Section "Validation").  SPECTRAL is -1/|k|^2 with the zero
 * mode set to 0 (spectral/periodic BCs only).  HEJ2..HEJ10: regularised of
 * order 2m, eps = eps_over_h * max(h), with any boundary conditions.
 * HEJ0: spectral truncation at pi/h, every direction unbounded or semi-unbounded.  LGF2: lattice
 * Green's function, spectral BCs only. */
typedef enum {
  FLUPS_SPECTRAL = 0, FLUPS_HEJ0 = 1, FLUPS_HEJ2 = 2, FLUPS_HEJ4 = 4, FLUPS_HEJ6 = 6,
  FLUPS_HEJ8 = 8, FLUPS_HEJ10 = 10, FLUPS_LGF2 = 100
} flups_green;
/* Derivative used in the spectral curl (Section "Application: the Biot-Savart solver"). */
typedef enum { FLUPS_DIFF_SPECTRAL = 0, FLUPS_DIFF_FD2 = 2, FLUPS_DIFF_FD4 = 4, FLUPS_DIFF_FD6 = 6 } flups_diff;

typedef struct flups_topo_s* flups_topo;
typedef struct flups_solver_s* flups_solver;

/* Grid topology.  n[3] = number of values per direction as stored by the
 * caller (see the size conventions above); center = FLUPS_CELL/FLUPS_NODE;
 * ncomp = 1 (scalar) or 3 (vector); prec = FLUPS_F32/FLUPS_F64.
 * Host-only; allocates a small host object owned by the caller (free with
 * flups_topo_free after the solvers built on it are cleaned up). */
int flups_init_topo(const int n[3], int center, int ncomp, int prec, flups_topo* out);
int flups_topo_free(flups_topo t);

/* Solver.  bc = ncomp * 3 * 2 ints, [comp][dir][face], face 0 = left (x = 0),
 * 1 = right (x = L); for FLUPS_POISSON with ncomp = 3 every component is
 * solved independently with its own BCs.  For FLUPS_BIOT_SAVART (ncomp = 3)
 * the BCs are those of the source f; the result u has in every direction the
 * conditions of the curl (even and odd swapped along the differentiated
 * direction).  h[3], L[3]: spacing and length per direction (h = L/N).
 * green: flups_green.  eps_over_h: regularisation length in units of max(h)
 * (2.0 in the paper's validation).  op: flups_op.  diff: flups_diff (ignored
 * for FLUPS_POISSON).  Host-only; validates everything that does not need the
 * device and returns FLUPS_EBC / FLUPS_ESIZE / FLUPS_EGREEN on violations. */
int flups_init_solver(flups_topo t, const int* bc, const double h[3], const double L[3], int green,
                      double eps_over_h, int op, int diff, flups_solver* out);

/* Setup: plans the transforms (direction order by cost, Section 1),
 * allocates the device workspace, builds twiddle tables (FP64, rounded once)
 * and, with any unbounded direction, the Green's function spectrum (FP64 on
 * the device, stored in the path precision).  Enqueued on `stream` and
 * synchronised before returning.  *workspace_bytes (may be NULL) receives the
 * device bytes the solver holds.  Calling it twice is a no-op. */
int flups_setup(flups_solver s, void* stream, size_t* workspace_bytes);

/* Solve: phi = G * rhs, both device arrays of the topology's shape (for the
 * Biot-Savart operator, 3 components each).  phi == rhs is allowed (in
 * place).  Enqueued on `stream`; returns without synchronising.  rhs is
 * read-only unless phi == rhs. */
int flups_solve(flups_solver s, void* phi, const void* rhs, void* stream);

/* Same solve with HOST arrays, on `stream`, synchronised before returning.
 * A pinned array (cudaHostAlloc / cudaHostRegister, mapped into the unified
 * address space; flups_host_mapped says so) is used in place: the first pass
 * loads rhs, and the last pass stores phi, over the host link, so the
 * transfers overlap those two passes.  A pageable array goes through a device
 * staging copy (allocated on first use, kept with the solver).  phi_host ==
 * rhs_host is allowed. */
int flups_solve_host(flups_solver s, void* phi_host, const void* rhs_host, void* stream);

/* 1 if the host range [host, host + bytes) is pinned memory that the device
 * addresses directly (what flups_solve_host uses in place), else 0. */
int flups_host_mapped(const void* host, size_t bytes);

/* Releases the plan, the Green spectrum and the workspace (twiddle tables
 * are shared by all solvers of the process and kept until exit).  The
 * caller's arrays are never freed.  Safe on NULL.  flups_cleanup frees
 * synchronously; flups_cleanup_async frees in stream order on `stream`
 * without synchronising the device, and requires that no work using the
 * solver is still pending on other streams. */
int flups_cleanup(flups_solver s);
int flups_cleanup_async(flups_solver s, void* stream);

/* The planner's transform order (host-only, any time after flups_init_solver):
 * order[i] = the direction (0 x, 1 y, 2 z) transformed i-th, by cost class
 * (Section 1: symmetric, then semi-unbounded, then periodic, then unbounded),
 * ties in x, y, z order; the first periodic or unbounded direction in that
 * order takes the real-to-complex transform. */
int flups_solver_order(flups_solver s, int order[3]);

/* Introspection (host-only, after flups_setup): number of kernel launches per
 * solve; transform order (3 direction indices); algorithmic bytes moved per
 * solve by the 5-pass model (each pass reads and writes its arrays once plus
 * one read of the stored Green spectrum). */
int flups_solver_info(flups_solver s, int* launches_per_solve, int order[3], double* model_bytes,
                      double* green_bytes);

/* Launch only pass i (0 <= i < launches_per_solve) of the solve on `stream`:
 * the solve is exactly passes 0, 1, ... in order (pass 0 reads rhs, the last
 * pass writes phi; the passes in between use the solver's workspace).  Lets a
 * caller time each kernel with events on its own stream. */
int flups_solve_pass(flups_solver s, int i, void* phi, const void* rhs, void* stream);
/* The whole solve with a CUDA event recorded before every pass and after the
 * last one: events = launches_per_solve + 1 cudaEvent_t handles (passed as
 * void*), owned by the caller.  For timing each kernel on its own stream. */
int flups_solve_events(flups_solver s, void* phi, const void* rhs, void* stream, void* const* events);
/* Pass i: kernel kind (0 forward real, 1 inverse real, 2 forward C2C,
 * 3 inverse C2C, 4 fused real, 5 fused C2C), transform axis, FFT length,
 * algorithmic bytes (arrays read and written once, Green spectrum read once)
 * and nominal flops (5 P log2 P per complex FFT of length P). */
int flups_pass_info(flups_solver s, int i, int* kind, int* axis, int* fft_len, double* bytes, double* flops);
/* How pass i runs (bit flags): 1 compile-time tile engine, 2 Green slice staged in shared memory
 * ahead of the multiply, 4 that slice copied by TMA (tensor map + mbarrier), 8 doubled transform
 * pruned to its nonzero half, 16 input tile copied by TMA (tensor map + mbarrier), 32 x pass on the
 * column kernels' register-chained stages, 64 input rows staged by one bulk copy.  Introspection
 * only; no counterpart in the paper. */
int flups_pass_features(flups_solver s, int i, int* flags);

/* Allocation-free fully periodic solve (the paper has no counterpart; this is
 * an integration convenience).  For callers that must not allocate device
 * memory: a host application whose own pool allocator owns the whole device,
 * or a latency-critical loop that cannot pay the implicit device
 * synchronisation of cudaMalloc/cudaFree.  It computes the same result as
 * flups_solve for a cell-centred, periodic-on-all-faces, FP64 problem with
 * the FLUPS_SPECTRAL kernel (-1/|k|^2, zero mean): phi and rhs are device
 * arrays of n[0] x n[1] x n[2] doubles (x fastest, phi == rhs allowed), L the
 * domain lengths.  Each n must be 2^a 3^b, 4 <= n <= 4096.
 *
 * Its whole workspace lives in one static device array of 48 MiB
 * (FLUPS_NOALLOC_SCRATCH_BYTES) that every GPU loading the library holds
 * until the process exits; sizes whose workspace exceeds it return
 * FLUPS_ESIZE (2 (n0/2 + 1) n1 n2 complex doubles plus small tables: up to
 * about 128^3).  It calls no cudaMalloc, cudaFree or allocating library
 * routine.  The first call on a device looks up the array's device address
 * with that device current (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls on a device share the one array and
 * nothing in it needs to start at zero (every read follows a write of the same
 * call); calls that overlap on the GPU (different streams, or different host
 * threads) race on it and must be serialised by the caller.  Enqueued on
 * `stream`; returns without synchronising. */
int flups_solve_periodic_noalloc(double* phi, const double* rhs, const int n[3], const double L[3], void* stream);

/* Plans shared by several concurrent solves (the serving runtime uses these).
 * flups_setup_shared: like flups_setup but allocates no workspace; solves then
 * go through flups_solve_ws with a caller-owned device workspace of
 * flups_workspace_size bytes (256-byte aligned), so one plan (twiddles, Green
 * spectrum) serves any number of solves in flight on different streams, each
 * with its own workspace.  flups_solver_memory (host-only, after
 * flups_init_solver): device bytes the plan keeps resident, the transient
 * peak of its setup, and the workspace of one solve.
 *
 * Device status of a workspace solve: the int at byte offset
 * flups_workspace_status(s) of the workspace is zeroed at the start of each
 * flups_solve_ws (stream-ordered) and set to a nonzero code by a kernel whose
 * bounded wait gave up (codes as in flups_solver_check); read it after the
 * solve has completed, e.g. with a stream-ordered copy to the host.  Each
 * workspace thus reports the status of its own solve. */
int flups_setup_shared(flups_solver s, void* stream);
int flups_workspace_size(flups_solver s, size_t* bytes);
int flups_workspace_status(flups_solver s, size_t* offset);
int flups_solve_ws(flups_solver s, void* phi, const void* rhs, void* workspace, void* stream);
int flups_solver_memory(flups_solver s, size_t* resident, size_t* transient, size_t* workspace);

/* ---- Serving: continuous batching of independent solves -------------------
 * A request describes one solve (same fields as flups_init_topo/init_solver;
 * scalar problems use bc[0]).  Its host arrays are read (rhs) and written
 * (phi) asynchronously: they must stay valid, and pinned for full copy
 * bandwidth, until the request's ticket is reported done.  Requests are
 * admitted as slots and memory free up within the device-memory budget given
 * at creation; admitted requests run concurrently on `nstreams` streams.
 * Plans (Green spectra, twiddles) are cached per problem and evicted least
 * recently used when memory is needed.  Not thread safe: one host thread
 * drives a server. */
typedef struct {
  int n[3];
  int center, prec, op, diff;
  int bc[3][3][2];
  double h[3], L[3];
  int green;
  double eps_over_h;
} flups_request;

typedef struct {
  long long submitted, admitted, completed, rejected, failed, queued_max;
  long long plan_hits, plan_misses, slots_created, evictions, plans_cached;
  size_t hbm_in_use, hbm_peak;
  /* host seconds spent, summed: plan setups on the setup workers (Green spectrum and
   * twiddles, enqueue to completion), and slot creation on the serving thread (device
   * arrays and the CUDA graph of the solve) */
  double setup_seconds, slot_seconds;
} flups_server_stats;

typedef struct flups_server_s* flups_server;

int flups_server_create(size_t hbm_budget_bytes, int nstreams, flups_server* out);
/* Queues the request and admits what fits.  Returns FLUPS_EBC/ESIZE/EGREEN/
 * EINVAL for an invalid request and FLUPS_ENOMEM if it cannot fit the budget
 * even alone (nothing is queued then). */
int flups_server_submit(flups_server sv, const flups_request* rq, const void* rhs_host, void* phi_host,
                        long long* ticket);
/* Completed tickets since the last call (up to max): latency from submission
 * to the end of the result's copy to the host, in seconds, and the status
 * (FLUPS_OK, or an error with latency -1; FLUPS_EDEVICE when a kernel of that
 * request's own solve reported a bounded wait that gave up, so its phi is not
 * valid).  poll never blocks; wait blocks until at least one ticket completes
 * or nothing is left. */
int flups_server_poll(flups_server sv, long long* tickets, double* latency_s, int* status, int max, int* n_done);
int flups_server_wait(flups_server sv, long long* tickets, double* latency_s, int* status, int max, int* n_done);
int flups_server_pending(flups_server sv, int* queued, int* running);
int flups_server_get_stats(flups_server sv, flups_server_stats* out);
/* Waits for the requests in flight, then frees every plan, slot and stream. */
int flups_server_destroy(flups_server sv);

/* Measured fused multiply-add rate of the current device (measurement support;
 * the paper has no counterpart): prec = FLUPS_F32 or FLUPS_F64; one launch of
 * 8 CTAs per SM, 256 threads each running 8 independent FMA chains for
 * 16 * iters steps, timed with CUDA events after a warm-up launch.
 * *tflops = 2 * FMAs / time (TFLOP/s), *ms (may be NULL) = the timed launch.
 * Allocates and frees a small device buffer; synchronous. */
int flups_measure_fma_peak(int prec, int iters, double* tflops, double* ms);

/* Text of a status code (static storage). */
const char* flups_strerror(int status);
/* Text of the last CUDA error seen by the library in this process (static storage). */
const char* flups_last_cuda_error(void);

/* Opt in, before flups_setup, to sharing the stored Green spectrum with other
 * solvers of the process that store the same data (same device, precision,
 * kernel, eps and per-direction sampling).  The last sharing solver released
 * frees it, stream-ordered on its release stream: release a sharing solver
 * only when no solve of any solver sharing its spectrum is still in flight
 * (the serving runtime releases idle plans only).  No counterpart in the paper. */
int flups_solver_share_green(flups_solver s);

/* Device-side status of the solver's kernels (solves on its own workspace)
 * since the last call: *code = 0, or the nonzero code a kernel left when one
 * of its bounded waits gave up: 1 the TMA copy of the Green slice in the fused
 * pass, 2 the TMA copy of a column pass's input tile did not complete within
 * 1 s.  A kernel whose wait gave up waits at most 0.1 s more for its copies in
 * flight and then writes none of its tile's results, so the solve's result is
 * not valid (undefined).  The first code recorded is kept.  Until the code is
 * read here, later bounded waits of the solver's kernels give their copies
 * 1 ms instead of 1 s.  Synchronises the device, resets the code.  No
 * counterpart in the paper (device-side failure reporting). */
int flups_solver_check(flups_solver s, int* code);

/* Test hook for the precision of the stored Green spectrum: samples (n values)
 * receives the FP64 real-space samples G(k_s, r_u) the setup transforms, the
 * Green index x fastest over the extents of every direction (unbounded-like:
 * r = g h, g = 0..M; spectral: the folded mode), and spectrum (n values) the
 * stored spectrum as the fused pass reads it, converted to double (the
 * double-float path stores hi + lo float pairs): the
 * samples' DCT-I along each unbounded-like direction (Section 2.3: the kernel
 * symmetrised on the extended domain, transformed there; computed in
 * double-float arithmetic on the FP32 units) times prod(h_u)/(P1 P2 P3).
 * n must be the product of the extents.  Only for solvers with a stored
 * spectrum (some direction unbounded or semi-unbounded; else FLUPS_ESTATE).
 * Synchronous; allocates a temporary device buffer.  No counterpart in the paper. */
int flups_debug_green(flups_solver s, double* samples, double* spectrum, long long n);

/* Test hook for that failure path: mask bit 0 (code 1) and bit 1 (code 2)
 * make the corresponding bounded waits of this solver's later solves give up
 * at once, as if their copies had not arrived in time (the copies do arrive:
 * the drain waits for them, so no copy is left in flight).  The solve's result
 * is then not valid and the code is reported.  mask = 0 restores normal
 * solves.  Host-only.  No counterpart in the paper. */
int flups_debug_wait_limit(flups_solver s, int mask);

/* Test hook: evaluate the device FP64 special functions used by the Green's
 * function generation at n points (device arrays x, y, out): which = 0 E1(x),
 * 1 Si(x), 2 HEJ2 one-unbounded kernel G(k = x, z = y), 3 two-unbounded
 * kernel G(k = x, r = y), 4 three-unbounded kernel G(r = y), 10 d_u + m
 * (d_u = 1..3, m = 2..5) the terms that turn the HEJ2 kernel with d_u unbounded
 * directions into HEJ2m, at k_s = x, r = y.  Synchronous. */
int flups_debug_special(int which, const double* x, const double* y, double* out, int n, double eps);

#ifdef __cplusplus
}
#endif

#endif /* FLUPS_GPU_H */
