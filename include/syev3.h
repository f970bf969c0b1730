/* syev3.h -- C ABI of the GB300 batched 3x3 real symmetric eigensolver.
 *
 * The method is C. F. Borges, "Solving the 3x3 Real Symmetric Eigenproblem"
 * (arXiv 1806.06698): an ordered Jacobi rotation in the (1,2)-plane reduces
 * each matrix to an arrow (Sec. 1); the arrow is tested for beta-, combo- and
 * numerical deflation and deflated arrows go to a 2x2 solve (Sec. 1.1);
 * otherwise the Borges-Gragg zero finder (Sec. 1.4.1) gives the shifted
 * extreme eigenvalues mu and nu, the middle one follows from the trace and
 * the eigenvectors from closed forms (Sec. 1.2).
 *
 * Conventions shared by every entry point:
 *  - A matrix is passed as its packed upper triangle, 6 values in the order
 *    (a11, a22, a33, a12, a13, a23); n matrices are n consecutive records
 *    (array of structures, no padding).
 *  - Eigenvalues: 3 per matrix, ascending.
 *  - Eigenvectors: a row-major 3x3 per matrix whose column k is the unit
 *    eigenvector of eigenvalue k (the torch.linalg.eigh convention); each
 *    column's largest-magnitude component is positive (first one on ties).
 *  - Pointers named d_* / device buffers are CUDA device memory (or managed
 *    memory) on the current device, allocated and owned by the caller; the
 *    library never frees or keeps them.  Buffers must be 8-byte aligned
 *    (FP64) or 4-byte aligned (FP32); 16-byte alignment selects the bulk-copy
 *    (TMA) input path and vector stores.
 *  - Calls are asynchronous on `stream` (NULL = the legacy default stream)
 *    unless stated otherwise; errors detected on the host are returned
 *    before anything is launched.
 *  - A record with a NaN or Inf entry yields NaN eigenvalues and vectors.
 *  - The zero finder is capped at 64 steps; a capped lane keeps its best
 *    iterate (it never traps) and is counted when counters are supplied.
 */
#ifndef SYEV3_H
#define SYEV3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t. */
typedef struct CUstream_st* syev3_stream_t;

/* Element type of every floating-point buffer of a call. */
typedef enum {
  SYEV3_F64 = 0,             /* binary64 in and out */
  SYEV3_F32 = 1,             /* binary32 in and out, plain FP32 arithmetic */
  SYEV3_F32_COMPENSATED = 2  /* binary32 in and out; compensated FP32 with FP64 refinement of flagged lanes */
} syev3_dtype;

typedef enum {
  SYEV3_OK = 0,
  SYEV3_EINVAL = 1,  /* bad argument: nothing was launched */
  SYEV3_ECUDA = 2,   /* a CUDA call failed (syev3_last_cuda_error() has the code) */
  SYEV3_ENOCONV = 3, /* reserved: reported through counters, never returned by a launch */
  SYEV3_ETIMEOUT = 4 /* a device-side wait ran out (see syev3_device_flags) */
} syev3_status;    /* (and SYEV3_EAGAIN, below with the server) */

/* Library ABI version (this header: 2). */
int syev3_abi_version(void);

/* Human-readable name of a status code (static string). */
const char* syev3_status_string(int status);

/* The cudaError_t of the most recent SYEV3_ECUDA on this host thread. */
int syev3_last_cuda_error(void);

/* syev3_batched -- eigenvalues and eigenvectors of n packed symmetric 3x3
 * matrices (Borges Secs. 1-1.4.1).
 *   A_packed6 : device, n x 6 of `dtype`, read only.
 *   n         : number of matrices, >= 0; n == 0 is a no-op returning SYEV3_OK.
 *   lambda    : device, n x 3 of `dtype`, written (ascending eigenvalues).
 *   U         : device, n x 9 of `dtype`, written (eigenvector columns), or
 *               NULL to compute eigenvalues only.
 *   dtype     : a syev3_dtype.
 *   stream    : CUDA stream the work is ordered on.
 * Returns SYEV3_EINVAL (NULL A or lambda, n < 0, bad dtype, misaligned or
 * overlapping buffers) or SYEV3_ECUDA (launch failure); SYEV3_OK otherwise.
 * syev3_batched allocates no device memory and uses none beyond its
 * arguments: the FP64 refinement of the compensated FP32 form works on a
 * shared-memory list inside the kernel (syev3_batched_ws takes a scratch
 * workspace from the caller instead).
 */
int syev3_batched(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype,
                  syev3_stream_t stream);

/* syev3_batched_ex -- syev3_batched with optional counters.
 *   d_counters : device, 4 x uint64, or NULL.  When given, the kernels add
 *                [0] lanes whose zero finder hit the step cap,
 *                [1] lanes with a non-finite input entry,
 *                [2] lanes refined in FP64 (SYEV3_F32_COMPENSATED only),
 *                [3] refined lanes whose FP64 residual ||A u - lambda u||
 *                    exceeded 16 eps32 ||A||_F (SYEV3_F32_COMPENSATED only).
 *                The caller zeroes them; they accumulate across calls.
 */
int syev3_batched_ex(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype,
                     uint64_t* d_counters, syev3_stream_t stream);

/* syev3_batched_ws -- syev3_batched_ex with a caller-provided device
 * workspace.  For SYEV3_F32_COMPENSATED the FP64 refinement of flagged lanes
 * (not in the paper: see SYEV3_F32_COMPENSATED) then runs as a second kernel
 * over a list of those lanes kept in the workspace, so the FP32 kernel holds
 * no FP64 code (fewer registers, more resident warps): the faster path when
 * few lanes are flagged (syev3_batched refines them in the FP32 kernel, in
 * whole warps gathered across tiles, and is the faster one when many are).
 * Results equal those of syev3_batched up to rounding.  From 2^21 matrices
 * on, the FP32 solve runs in 8 runs on `stream` and each run's refinement
 * on a side stream beside the next run's solve (events order them; `stream`
 * waits for the side stream before anything queued after the call); the
 * side stream and its events are created by the library on the first such
 * call for a device and kept, and calls from several host threads enqueue
 * their work one after the other.
 * Other dtypes ignore the workspace (it may be NULL).
 *   d_workspace     : device, at least syev3_workspace_bytes(n, dtype) bytes,
 *                     256-byte aligned, caller-owned; must not overlap the
 *                     inputs or outputs; contents need not be initialised
 *                     (the library clears what must start at zero on
 *                     `stream`).  Calls that share a workspace must be
 *                     ordered (same stream or synchronised).
 *   workspace_bytes : its size.
 * Returns SYEV3_EINVAL as syev3_batched_ex, and for a missing, misaligned,
 * too small, host-pageable or overlapping workspace. */
size_t syev3_workspace_bytes(int64_t n, int dtype);

int syev3_batched_ws(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype, uint64_t* d_counters,
                     void* d_workspace, size_t workspace_bytes, syev3_stream_t stream);

/* syev3_batched_static_ws -- syev3_batched_ws for SYEV3_F32_COMPENSATED
 * with the scratch list in the library's static device memory (a file-scope
 * __device__ array of SYEV3_STATIC_MAX_N records, 12.6 MB), so that the call
 * allocates nothing and needs no workspace from the caller.  Not in the
 * paper (which has no counterpart to any of the memory management here):
 * for callers that cannot pass a workspace -- a C caller without a device
 * allocator of its own, or code that must not call cudaMalloc/cudaFree on
 * this path (they synchronise the device and can fail under memory
 * pressure).
 *   A_packed6, lambda, U, d_counters, stream: as syev3_batched_ex with
 *   dtype SYEV3_F32_COMPENSATED (float32 buffers).
 *   n : 0 <= n <= SYEV3_STATIC_MAX_N, else SYEV3_EINVAL (nothing launched).
 * The array is shared by every call on a device: calls that overlap in time
 * (other streams or host threads) race on it and must be ordered by the
 * caller.  The first call on a device resolves the array's address
 * (cudaGetSymbolAddress, with that device current); it must come before any
 * stream capture begins on that device.  The address is kept for the life
 * of the process: do not use this entry point on a device after
 * cudaDeviceReset (the new context may place the array elsewhere).  Errors
 * as syev3_batched_ws. */
#define SYEV3_STATIC_MAX_N 262144

int syev3_batched_static_ws(const void* A_packed6, int64_t n, void* lambda, void* U, uint64_t* d_counters,
                            syev3_stream_t stream);

/* syev3_batched_method -- syev3_batched (FP64 only) with the variants of
 * the method the paper also describes, for studying them against the
 * production path:
 *   zero_finder    : SYEV3_ZF_PRODUCTION -- the path of syev3_batched (FP32
 *                    Borges-Gragg seeds, one FP64 step and the stopping test);
 *                    SYEV3_ZF_BORGES_GRAGG -- the Borges-Gragg iteration of
 *                    Sec. 1.4.1 in FP64 from the start of Eq. (7);
 *                    SYEV3_ZF_NEWTON -- Newton's method of Sec. 1.4.2 in FP64,
 *                    started left of the zero, stopped when |f| < 2 eps x.
 *   deflation_test : SYEV3_DEFLATION_SIMPLIFIED -- the test the paper adopts,
 *                    |abar b1 b2| <= eps |a1 + a2| h^2 (Sec. 1.1);
 *                    SYEV3_DEFLATION_EISPACK -- the EISPACK-style test it is
 *                    derived from, |abar b1 b2| <= eps (|a1 b2^2 + a2 b1^2| +
 *                    |a1 b1^2 + a2 b2^2|).
 *   d_stats        : device, SYEV3_METHOD_STATS x uint64, or NULL; the
 *                    kernel adds [0] lanes whose zero finder hit the 64-step
 *                    cap, [1] non-finite lanes, [2] diagonal, [3] deflated and
 *                    [4] reduced arrows, [5] zero-finder steps taken by the
 *                    full FP64 iteration, [6] roots it solved, [7] the FP64
 *                    lane-slots its warps spent (32 x the longest iteration of
 *                    each warp; [5]/[7] is the iteration's SIMT efficiency).
 *                    With SYEV3_ZF_PRODUCTION, [5]-[7] cover only the roots the
 *                    seeded step leaves to the full iteration.  The caller
 *                    zeroes them; they accumulate.
 * Arguments and errors otherwise as syev3_batched; SYEV3_EINVAL also for a
 * dtype other than SYEV3_F64, a NULL method or an unknown variant. */
typedef enum {
  SYEV3_ZF_PRODUCTION = 0,
  SYEV3_ZF_BORGES_GRAGG = 1,
  SYEV3_ZF_NEWTON = 2
} syev3_zero_finder;

typedef enum {
  SYEV3_DEFLATION_SIMPLIFIED = 0,
  SYEV3_DEFLATION_EISPACK = 1
} syev3_deflation_test;

#define SYEV3_METHOD_STATS 8

typedef struct {
  int zero_finder;    /* a syev3_zero_finder */
  int deflation_test; /* a syev3_deflation_test */
} syev3_method;

int syev3_batched_method(const void* A_packed6, int64_t n, void* lambda, void* U, int dtype,
                         const syev3_method* method, uint64_t* d_stats, syev3_stream_t stream);

/* syev3_batched_bwd -- gradient of a loss through syev3_batched, packed.
 * Not in the paper: the standard derivative of simple eigenpairs,
 *   Abar = U (diag(g_lambda) + F o (U^T g_U)) U^T,
 *   F_ij = 1/(lambda_j - lambda_i) for i != j, and F_ij = 0 where
 *   |lambda_i - lambda_j| < gap_tau * ||A||_F (||A||_F = ||lambda||_2);
 * g_A_packed6 receives (Abar_11, Abar_22, Abar_33, Abar_12 + Abar_21,
 * Abar_13 + Abar_31, Abar_23 + Abar_32): the gradient with respect to the
 * packed entries (a11, a22, a33, a12, a13, a23).
 *   lambda, U   : device, the outputs of syev3_batched (n x 3, n x 9).
 *   g_lambda    : device, n x 3, gradient of the loss with respect to lambda.
 *   g_U         : device, n x 9, gradient with respect to U, or NULL (zero).
 *   n           : >= 0.
 *   g_A_packed6 : device, n x 6, written; must not overlap the inputs.
 *   gap_tau     : >= 0; eigenvector coupling of closer pairs is dropped.
 *   dtype       : SYEV3_F64, or SYEV3_F32 / SYEV3_F32_COMPENSATED (FP32).
 * Returns SYEV3_EINVAL (NULL required buffer, n < 0, negative or
 * non-finite gap_tau, misaligned, overlapping or host-pageable buffers) or
 * SYEV3_ECUDA; SYEV3_OK otherwise.  Asynchronous on `stream`. */
int syev3_batched_bwd(const void* lambda, const void* U, const void* g_lambda, const void* g_U, int64_t n,
                      void* g_A_packed6, double gap_tau, int dtype, syev3_stream_t stream);

/* syev3_batched_host -- syev3_batched for buffers in host memory
 * (blocking).  The batch is cut into chunks of `chunk` matrices; with
 * chunk <= 0 the library's schedule, 2^16 matrices first and each next
 * chunk a quarter longer up to 2^20 (the first results start back early).
 * Each chunk is copied in, solved and copied out on one of three library
 * streams, so copies overlap the solves of neighbouring chunks.
 *   A_host      : host, n x 6 of dtype (page-locked memory lets the copies
 *                 run asynchronously; pageable memory works, slower).
 *   lambda_host : host, n x 3, written.  U_host: host, n x 9, or NULL.
 *   stream      : the pipeline starts after the work queued on it.
 * Device staging buffers (3 x the largest chunk) are allocated by the library
 * on the first call for a device and kept for later calls; they grow when
 * a larger chunk is asked for.  Calls for the same device from several host
 * threads are serialised.  Returns when the host outputs are written. */
int syev3_batched_host(const void* A_host, int64_t n, void* lambda_host, void* U_host, int dtype, int64_t chunk,
                       syev3_stream_t stream);

/* Device-side status bits of the current device, OR-ed over all launches
 * since the last call, then cleared (synchronises the device).
 *   bit 0: a bulk-copy wait timed out (SYEV3_ETIMEOUT).  Every wait of the
 *   kernels on a bulk copy is bounded (1 s of the GPU's global timer); a CTA
 *   whose wait runs out records this bit, lets its copies in flight land and
 *   exits, so the context stays usable. */
int syev3_device_flags(uint32_t* flags);

/* syev3_selftest_wait_limit -- exercises that failure path: launches one CTA
 * that waits on an mbarrier nothing completes; after the wait limit (about
 * 1 s) it sets bit 0 of the device flags and exits.  For tests of the
 * failure handling; not in the paper.  Asynchronous on `stream`. */
int syev3_selftest_wait_limit(syev3_stream_t stream);

/* syev3_selftest_arith -- the kernels' own approximate arithmetic, applied
 * elementwise, so tests can hold it to the error bounds the solver relies
 * on.  Not in the paper.
 *   op : SYEV3_ARITH_RCP64  -- 1/x in FP64: the hardware's reciprocal
 *                              estimate refined by one third-order
 *                              Newton-Raphson step (within 1 ulp of 1/x for
 *                              2^-1000 < |x| < 2^1000);
 *        SYEV3_ARITH_RCP32, SYEV3_ARITH_SQRT32, SYEV3_ARITH_RSQRT32 -- the
 *                              FP32 hardware approximations 1/x, sqrt(x),
 *                              1/sqrt(x) (flush-to-zero) used by the FP32
 *                              zero finder;
 *        SYEV3_ARITH_F2D, SYEV3_ARITH_D2F -- float to double (exact) and
 *                              double to float (round to nearest even),
 *                              computed on the integer pipes by the FP64
 *                              kernels and the FP64 refinement; the IEEE
 *                              results bit for bit.
 *   x  : device, n elements (double for RCP64 and D2F, float otherwise),
 *        read.
 *   y  : device, n elements (double for RCP64 and F2D, float otherwise),
 *        written; may not overlap x.
 *   n  : >= 0.
 * Returns SYEV3_EINVAL (bad op, n < 0, NULL or misaligned buffers) or
 * SYEV3_ECUDA; asynchronous on `stream`. */
#define SYEV3_ARITH_RCP64 0
#define SYEV3_ARITH_RCP32 1
#define SYEV3_ARITH_SQRT32 2
#define SYEV3_ARITH_RSQRT32 3
#define SYEV3_ARITH_F2D 4
#define SYEV3_ARITH_D2F 5

int syev3_selftest_arith(int op, const void* x, void* y, int64_t n, syev3_stream_t stream);

/* syev3_probe_dfma -- launches one kernel that issues only FP64 fused
 * multiply-adds (independent chains on every resident thread of every SM)
 * and stores in *dfma_count the number it executes, so that the caller,
 * timing the launch on `stream`, obtains the device's FP64 operation rate:
 * the peak against which the FP64 solver's roofline is reported.  Not in
 * the paper.
 *   iters      : iterations per chain, >= 1 (10^5 takes about 10 ms).
 *   d_sink     : device, 1 double (never written in practice; keeps the
 *                chains from being optimised away).
 *   dfma_count : host, written before the launch.
 * Returns SYEV3_EINVAL or SYEV3_ECUDA on failure. */
int syev3_probe_dfma(int64_t iters, double* d_sink, int64_t* dfma_count, syev3_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request server (not in the paper; each
 * request's matrices go through the method of Secs. 1-1.4.1).
 *
 * Requests reference packed matrices already in device memory.  The queues,
 * the admission state and the results live on the device: a ring of
 * SYEV3_SERVER_SLOTS request slots, a FIFO admission over them against an
 * arena of fixed size (the memory budget, allocated once by
 * syev3_server_create) that receives every request's eigenvalues and
 * eigenvectors, and per round the list of work the device chose.  The
 * library's host thread passes new requests and releases to the device and
 * launches rounds while there is work; in each round the device
 *  - frees released requests and admits waiting ones in arrival order as far
 *    as the arena has room,
 *  - gives every admitted request with work left up to `chunk` matrices
 *    (round-robin, `round_matrices` in all), and solves them as one ragged
 *    batch per element type, so requests that arrive while others run share
 *    the device from their first round on,
 *  - marks finished requests done, with a device timestamp.
 * Results stay in the arena until syev3_server_release.
 * ------------------------------------------------------------------------ */
typedef struct syev3_server_s syev3_server;

/* Requests submitted and not yet released, at most. */
#define SYEV3_SERVER_SLOTS 16384

/* Returned by syev3_server_submit when SYEV3_SERVER_SLOTS requests are
 * outstanding (not yet released): release some and submit again. */
#define SYEV3_EAGAIN 5

typedef struct {
  size_t memory_budget_bytes; /* device arena for results; 0 = 16 GiB */
  int64_t chunk;              /* matrices of one request per round; 0 = 2^18 */
  int64_t round_matrices;     /* matrices per round over all requests, <= 2^27; 0 = 2^21 */
  int max_rounds_in_flight;   /* rounds queued on the device at once, 1..4; 0 = 2 */
} syev3_server_config;

typedef struct {
  int state;        /* 0 waiting for memory, 1 admitted, 2 done, 3 failed */
  int dtype;
  int64_t n;
  void* d_lambda;   /* device, n x 3 (valid once admitted; final when done) */
  void* d_U;        /* device, n x 9, or NULL when vectors were not asked for */
  int64_t t_submit_ns, t_admit_ns, t_done_ns; /* host steady clock (admission
                                                 and completion: the device's
                                                 timer, mapped to it) */
} syev3_request_info;

typedef struct {
  int64_t completed, matrices, chunks, waiting; /* chunks: work items issued */
  size_t arena_bytes, arena_used, arena_peak;
  int error;        /* first failure status, or SYEV3_OK */
  int64_t rounds;   /* rounds completed on the device */
  int64_t launches; /* kernels launched by the server */
} syev3_server_stats;

/* Creates a server on the current device; cfg may be NULL (defaults).
 * Allocates the arena and the device queues with cudaMalloc and a mailbox
 * in mapped host memory: SYEV3_ECUDA if that fails (nothing is kept);
 * SYEV3_EINVAL for a budget below 256 bytes or max_rounds_in_flight > 4. */
int syev3_server_create(const syev3_server_config* cfg, syev3_server** out);

/* Stops launching, waits for the rounds on the device, frees everything. */
int syev3_server_destroy(syev3_server* srv);

/* Queues a request: n >= 1 packed matrices at d_A (device, dtype as in
 * syev3_batched, must stay valid and unchanged until the request is done).
 * Returns at once with a ticket; SYEV3_EINVAL if the outputs could never fit
 * the arena, SYEV3_EAGAIN when SYEV3_SERVER_SLOTS requests are outstanding,
 * or the server's error after a failure. */
int syev3_server_submit(syev3_server* srv, int dtype, const void* d_A, int64_t n, int vectors,
                        uint64_t* ticket);

/* State, result pointers and timestamps of a request (non-blocking). */
int syev3_server_query(syev3_server* srv, uint64_t ticket, syev3_request_info* info);

/* Blocks until the request is done (SYEV3_OK), failed (the server's error)
 * or timeout_s passed (SYEV3_ETIMEOUT). */
int syev3_server_wait(syev3_server* srv, uint64_t ticket, double timeout_s);

/* Ends a done (or failed) request: its results are freed on the device in
 * the next round.  SYEV3_EINVAL if it is unknown or not finished.  After a
 * failure the server keeps its device memory (its device state is not
 * trusted) and accepts only destroy. */
int syev3_server_release(syev3_server* srv, uint64_t ticket);

int syev3_server_get_stats(syev3_server* srv, syev3_server_stats* stats);

/* Failure handling, exercised without a device fault: the next round the
 * server would launch is not launched, and the server fails as if that
 * launch had returned `status` (not SYEV3_OK): requests not yet done fail
 * with it, later submits return it, releases free nothing.  For tests. */
int syev3_server_inject_failure(syev3_server* srv, int status);

#ifdef __cplusplus
}
#endif

#endif /* SYEV3_H */
