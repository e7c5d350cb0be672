/*
 * rg.h -- C ABI of the GB300 rank-Greville recursive least-squares library (librg.so).
 *
 * The method (Staub & Steinmann, "Efficient Recursive Least Squares Solver for
 * Rank-Deficient Matrices", arXiv 2106.11594) keeps a full-rank factorization
 * A_n = B_n C_n of the n x m observation matrix (Section 2.1, Eq. label_eq_mat_prod):
 * C_n (r x m) holds r linearly independent observed rows, Ct_n = (C_n C_n^T)^-1 C_n is
 * its dual basis, and P_n^-1 = (B_n^T B_n)^-1 is r x r. For every new observation
 * (Gamma, y) it projects Gamma onto span(C_n) (gamma = Ct_n Gamma), forms the rejection
 * Gamma_r = Gamma - C_n^T gamma, runs the rank test of Eq. label_eq_eps, then either
 * appends a basis row (Theorem 6, independent case) or applies the rank-preserving
 * Sherman-Morrison update of P^-1 (Theorem 6, dependent case), and refreshes the
 * minimum-norm least-squares solution X = A^+ Y (Theorems 4 and 5; Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Every matrix is row-major. A block of k observations is a k x m array whose row i
 *    is Gamma_i^T; targets are a length-k array.
 *  - Pointers documented as "device" must be CUDA device (or managed) memory on the
 *    device that was current when the state was created; "host" pointers are ordinary
 *    CPU memory. The caller owns every buffer it passes; the library owns the state.
 *  - Calls are asynchronous on the state's CUDA stream unless documented as
 *    synchronising. Arguments are validated on the host before anything is enqueued:
 *    a bad argument returns RG_EINVAL and enqueues nothing.
 *  - Errors found on the device (non-finite rows, rank capacity exceeded, a bounded
 *    wait that ran out) are recorded in a device status word and returned by the next
 *    synchronising call (rg_solution, rg_rank, rg_sync). The row that raised the error
 *    and every later row of the same call are not applied; the state stays as it was
 *    after the last applied row; rg_rows_seen reports how many rows were applied.
 *  - rg_last_error() returns a thread-local message describing the last failure.
 *  - Nothing here falls back to the CPU: without a usable CUDA device every call that
 *    needs one returns RG_ECUDA.
 */
#ifndef RG_H
#define RG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rg_state rg_state; /* one recursive least-squares stream (opaque)   */
typedef struct rg_batch rg_batch; /* many independent streams of uneven shape       */

typedef enum {
  RG_OK = 0,
  RG_EINVAL = 1,      /* invalid argument (checked on the host, nothing enqueued)   */
  RG_ENOMEM = 2,      /* device or host allocation failed                           */
  RG_ECUDA = 3,       /* a CUDA runtime call failed (message in rg_last_error)       */
  RG_ECAPACITY = 4,   /* an independent row arrived while rank == r_max              */
  RG_ENONFINITE = 5,  /* a row or target contained NaN or Inf                        */
  RG_ETIMEOUT = 6     /* a bounded device-side wait gave up (state must be reset)     */
} rg_status;

/* Flags of rg_init / rg_batch_init (OR them together). */
enum {
  RG_FP64 = 0,        /* all arithmetic in FP64                                      */
  RG_MIXED = 1,       /* projections in FP32; rank test, denominators, P^-1 and w in
                         FP64; candidate rows are re-decided in FP64 (see rg_init)   */
  RG_TEST_REL = 0,    /* independent iff ||Gamma_r|| > eps ||Gamma||                  */
  RG_TEST_PAPER = 2,  /* dependent iff ||Gamma_r|| < eps or ||Gamma_r|| < eps ||Gamma||
                         (Eq. label_eq_eps, both clauses)                            */
  RG_ORTHONORMAL = 4, /* keep the orthonormal variant of Section 2.2 (alpha_{n+1} =
                         1/||Gamma_r||: the basis rows are orthonormal and serve as their
                         own dual basis) instead of Algorithm 1's raw rows and dual basis.
                         RG_MIXED always uses it; with RG_FP64 it is opt-in (rg_init,
                         rg_solve_noalloc and rg_batch_init)                         */
  RG_ORTHOGONAL = 8   /* keep the orthogonal variant of Section 2.2 (alpha_{n+1} = 1: the
                         basis rows are the raw rejections Gamma_r, mutually orthogonal, and
                         the dual rows are Gamma_r / ||Gamma_r||^2; appends leave the older
                         rows unchanged). FP64 only: excludes RG_MIXED and
                         RG_ORTHONORMAL (RG_EINVAL)                                  */
};

/*
 * rg_init -- create an empty stream (rank 0, X = 0) for observations of length m.
 *   out        host; receives the new state.
 *   m          number of regressors (columns), >= 1.
 *   tol        rank-test threshold eps of Eq. label_eq_eps. tol <= 0 selects the
 *              paper's default (m^2 r + m r + m) eps_M, r the rank before the row.
 *              Must not be NaN.
 *   flags      RG_FP64 or RG_MIXED, OR-ed with RG_TEST_REL or RG_TEST_PAPER and
 *              optionally RG_ORTHONORMAL or (FP64 only) RG_ORTHOGONAL. In RG_MIXED mode a row whose FP32 relative rejection
 *              ||Gamma_r|| / ||Gamma|| exceeds 1e-5 is recomputed and decided in FP64;
 *              rows below that floor are taken as dependent.
 *   r_max      capacity of the basis (maximum rank), 1..m; <= 0 means m.
 *   cuda_stream  cudaStream_t on which all work of this state is enqueued (NULL: the
 *              legacy default stream). Device memory is allocated here, once.
 * Returns RG_OK, RG_EINVAL, RG_ENOMEM or RG_ECUDA.
 */
rg_status rg_init(rg_state** out, int64_t m, double tol, int flags, int64_t r_max,
                  void* cuda_stream);

/*
 * rg_add_rows -- apply Algorithm 1 to k new observations, in order.
 *   Gamma      device, k x m row-major FP64 (row i = Gamma_i^T).
 *   y          device, k FP64 targets.
 *   k          number of rows, >= 0 (0 is a no-op).
 *   indep_out  device, k bytes, may be NULL: indep_out[i] = 1 if row i grew the rank,
 *              0 if it was dependent (rows not applied because of an error keep 0xFF).
 * The result equals k sequential single-row updates in exact arithmetic (the rows are
 * projected as one block and the rank changes inside the block are applied in order).
 * Asynchronous; device errors surface at the next synchronising call.
 */
rg_status rg_add_rows(rg_state* st, const double* Gamma, const double* y, int64_t k,
                      uint8_t* indep_out);

/*
 * rg_add_rows_host -- same as rg_add_rows for HOST buffers: the rows are copied to the
 * device inside the call (in chunks through two library-owned staging slots, on a copy
 * stream of the library, so that a chunk's copy overlaps the previous update) and the call
 * returns once the host buffers may be reused; the update itself stays asynchronous
 * (device errors surface at the next synchronising call). indep_out is host memory (may be
 * NULL); when given, the call also waits for the update.
 */
rg_status rg_add_rows_host(rg_state* st, const double* Gamma, const double* y, int64_t k,
                           uint8_t* indep_out);

/*
 * rg_solution -- materialise X = A^+ Y (length m) into device memory X.
 *   rank_out   host, may be NULL: receives the current rank (this synchronises).
 * Synchronising when rank_out != NULL; returns any pending device error.
 */
rg_status rg_solution(rg_state* st, double* X, int64_t* rank_out);

/*
 * rg_adjoint -- gradient of a loss L(X) through X = A^+ y, from the state's final
 * factorization. The paper has no counterpart: it is the classical derivative of the
 * pseudoinverse on the manifold of fixed-rank matrices (from the Penrose equations of
 * Section 1), evaluated with A^+ = Ct^T P^-1 B^T (Section 2.1):
 *   dL/dy = h = A^+T g,   dL/dA = -h X^T + rho (A^+ h)^T + (A^+T X) g_perp^T,
 *   rho = y - A X,        g_perp = (I - A^+ A) g.
 *   A     device FP64, n x m row-major: exactly the rows fed since init/reset, in order
 *         (the library does not keep them).
 *   y     device FP64, n: their targets.
 *   g     device FP64, m: dL/dX.
 *   gA    device FP64, n x m (output);  gy  device FP64, n (output).
 *   X     device FP64, m, may be NULL: receives X.
 * FP64 throughout, in both modes. Uses a stream-ordered workspace (cudaMallocAsync) of
 * about 8 (4m + 7 r_max + 3n + 4 m ceil(n/256)) bytes. Asynchronous.
 */
rg_status rg_adjoint(rg_state* st, const double* A, const double* y, int64_t n, const double* g,
                     double* gA, double* gy, double* X);

/*
 * rg_pinv -- the pseudoinverse A_n^+ (m x n) of the n rows the stream has taken since
 * rg_init / rg_reset. Theorems label_th_pinv_indep and label_th_pinv_lindep update A^+ row
 * by row (A^+ <- [A^+ - K b^T, K]); the library forms the same matrix after any call from
 * the factorization it keeps, A^+ = D^T P^-1 B^T with B = A D^T (Section 2.1; D = Ct, or
 * Q in the orthonormal variant), in 4 m n r FP64 flops.
 *   A      device, n x m row-major: the rows fed, in order (the caller keeps them; the
 *          result is only A^+ when they are exactly those rows).
 *   n      number of rows fed, >= 0.
 *   Apinv  device, m x n written with row stride ld: Apinv[c * ld + i] is entry (c, i) of
 *          A^+ (coefficient c, observation i), so that X = A^+ y.
 *   ld     row stride of Apinv, >= n.
 * Reads the rank (synchronising), then runs asynchronously on the state's stream with a
 * stream-ordered workspace of (m + n) r doubles. Ranks above 2048 give RG_EINVAL. A stream
 * stopped by RG_ECAPACITY or RG_ENONFINITE still yields the pseudoinverse of the rows
 * it applied (pass those rows).
 */
rg_status rg_pinv(rg_state* st, const double* A, int64_t n, double* Apinv, int64_t ld);

/* rg_solution_host -- rg_solution into HOST memory X (m doubles). Synchronising. */
rg_status rg_solution_host(rg_state* st, double* X, int64_t* rank_out);

/*
 * rg_set_screen -- mixed mode only: floor tau_lo of the FP32 screen (default 1e-5). A row
 * whose FP32 relative rejection ||Gamma_r|| / ||Gamma|| is at most max(tau_lo, tol / 2) is
 * declared dependent without an FP64 decision; rows above it are re-decided in FP64 against
 * tol. Lowering it catches rejections between tol and the default floor (ill-conditioned
 * inputs, Section 4.2's stability discussion) at the price of more FP64 decisions; below
 * the FP32 noise of the projections (~1e-7 relative) every row is decided in FP64.
 * 0 < tau_lo < 1, else RG_EINVAL. Host-side only; applies from the next call.
 */
rg_status rg_set_screen(rg_state* st, double tau_lo);

/* rg_rank -- current rank r into *rank_out (host). Synchronising. */
rg_status rg_rank(rg_state* st, int64_t* rank_out);

/* rg_rows_seen -- number of rows applied since init/reset into *rows_out (host).
 * Synchronising. */
rg_status rg_rows_seen(rg_state* st, int64_t* rows_out);

/* rg_sync -- wait for the state's stream and return any pending device error
 * (the error is cleared once returned). */
rg_status rg_sync(rg_state* st);

/* rg_reset -- return to the empty state (rank 0, X = 0) without reallocating.
 * Asynchronous. */
rg_status rg_reset(rg_state* st);

/*
 * rg_export -- copy the factorization for inspection. Device pointers, each may be NULL:
 *   C (r x m), Ct (r x m), Pinv (r x r), w (r; X = Ct^T w), basis_rows (r int64: the
 *   0-based index, counted from init/reset, of the input row stored in each row of C).
 *   capacity   number of rows each of C/Ct/w/basis_rows can hold (>= current rank,
 *              else RG_EINVAL); Pinv must hold capacity x capacity and is written with
 *              row stride r.
 *   rank_out   host, receives r. Synchronising.
 */
rg_status rg_export(rg_state* st, double* C, double* Ct, double* Pinv, double* w,
                    int64_t* basis_rows, int64_t capacity, int64_t* rank_out);

/*
 * Snapshots of the factorization: checkpoint / resume of a stream, and the factor
 * snapshots that gradients through intermediate solutions X_n need. The paper has no
 * counterpart; the state copied is exactly what Algorithm 1 carries from one row to the
 * next (the basis, its dual basis, the r x r state and the solution coordinates, Section
 * 2.1), so that restoring a snapshot taken after n rows and feeding rows n+1.. gives the
 * same results as never having stopped.
 *
 * rg_snapshot_size -- bytes of a snapshot of this state (host; fixed by m, r_max and the
 *   flags given to rg_init: about 8 r_max (2m + r_max) bytes in FP64 mode).
 */
rg_status rg_snapshot_size(rg_state* st, int64_t* bytes_out);

/*
 * rg_snapshot -- copy the state into buf: the basis C (or Q), the dual basis Ct (general
 * variant), the FP32 copy of Q (mixed mode), the leading r x r block of P = B^T B, the
 * solution coordinates w_b and u, the basis-row indices, the rank, the rows seen and the
 * internal block size. A deferred update of the previous call is folded into the state
 * first. The rank is read on the device; only rows below it are copied.
 *   buf    device, 256-byte aligned, at least rg_snapshot_size bytes; owned by the caller.
 * Asynchronous; the snapshot is complete when the state's stream reaches this point.
 */
rg_status rg_snapshot(rg_state* st, void* buf, int64_t bytes);

/*
 * rg_restore -- make the state equal to a snapshot taken from a state with the same m,
 * r_max and flags (this state or another); the next rows continue from it. A buffer
 * whose header does not match (another shape or variant, or not a snapshot) leaves the
 * state unchanged and returns RG_EINVAL at the next synchronising call. Clears the status
 * word. Asynchronous.
 */
rg_status rg_restore(rg_state* st, const void* buf, int64_t bytes);

/* rg_set_stream -- enqueue later work of this state on another cudaStream_t. */
rg_status rg_set_stream(rg_state* st, void* cuda_stream);

/* rg_free -- release the state (synchronises its stream first). NULL is a no-op. */
rg_status rg_free(rg_state* st);

/* ------------------------------------------------------------------------------------
 * Batched form: B independent streams of uneven (n_b, m_b) in one persistent kernel.
 * Packed layout: instance b's rows are Gamma_packed[elem_offsets[b] .. elem_offsets[b+1])
 * viewed as n_b x m_b row-major, with n_b = row_offsets[b+1] - row_offsets[b];
 * its targets are y_packed[row_offsets[b] .. row_offsets[b+1]).
 * ------------------------------------------------------------------------------------ */

/*
 * rg_batch_init -- create B empty streams.
 *   m       host, B column counts (each >= 1).
 *   r_max   host, B capacities (NULL: r_max[b] = m[b]).
 *   tol, flags, cuda_stream: as rg_init (shared by all instances).
 */
rg_status rg_batch_init(rg_batch** out, int64_t B, const int64_t* m, double tol, int flags,
                        const int64_t* r_max, void* cuda_stream);

/*
 * rg_batch_add_rows -- append a block of rows to every instance (n_b may be 0).
 *   Gamma_packed, y_packed  device FP64, packed as above.
 *   row_offsets, elem_offsets  device int64, B+1 entries each; elem_offsets[b+1] -
 *              elem_offsets[b] must equal n_b m_b (checked on the device: a mismatch
 *              sets RG_EINVAL in the status word and skips the instance).
 *   indep_out  device, sum(n_b) bytes in row order, may be NULL.
 * Instances are scheduled longest-first (by n_b m_b r_max_b) over persistent CTAs.
 */
rg_status rg_batch_add_rows(rg_batch* bt, const double* Gamma_packed,
                            const int64_t* row_offsets, const int64_t* elem_offsets,
                            const double* y_packed, uint8_t* indep_out);

/*
 * rg_batch_solution -- X_packed[x_offsets[b] .. + m_b) = X of instance b.
 *   X_packed   device FP64.
 *   x_offsets  device int64, B+1 entries (NULL: packed back to back by m_b).
 *   ranks_out  device int64, B entries, may be NULL.
 * Asynchronous.
 */
rg_status rg_batch_solution(rg_batch* bt, double* X_packed, const int64_t* x_offsets,
                            int64_t* ranks_out);

/*
 * rg_batch_adjoint -- rg_adjoint for every instance, one launch. The rows, offsets and
 * targets are laid out as in rg_batch_add_rows and must be all rows fed since
 * init/reset; total_rows (host) is row_offsets[B]. g_packed holds dL/dX of instance b at
 * x_offsets[b] (NULL: packed by m_b); gA_packed is laid out like Gamma_packed, gy_packed
 * like y_packed. Inconsistent offsets set RG_EINVAL on the instance (reported by the next
 * rg_batch_sync). FP64 throughout. Asynchronous.
 */
rg_status rg_batch_adjoint(rg_batch* bt, const double* Gamma_packed, const int64_t* row_offsets,
                           const int64_t* elem_offsets, const double* y_packed, int64_t total_rows,
                           const double* g_packed, const int64_t* x_offsets, double* gA_packed,
                           double* gy_packed);

/* rg_batch_set_screen -- rg_set_screen for every instance of the batch. */
rg_status rg_batch_set_screen(rg_batch* bt, double tau_lo);

/* rg_batch_set_stream -- issue later batch calls on cuda_stream (synchronises the old
 * stream first). Lets a caller capture the batch calls into a CUDA graph. */
rg_status rg_batch_set_stream(rg_batch* bt, void* cuda_stream);

/*
 * rg_batch_set_block_rows -- cap on the rows an instance takes per internal block (the
 * block grows from 64 rows after a rank change up to this cap while rows stay dependent;
 * Section 3's block of observations). rows > 0 sets it (32 <= rows <= the capacity laid
 * out at init, which depends on the largest r_max; otherwise RG_EINVAL); rows <= 0 only
 * queries. rows_out (host, may be NULL) receives the cap in force. Host-side only; takes
 * effect at the next rg_batch_add_rows. Used by the autotuner.
 */
rg_status rg_batch_set_block_rows(rg_batch* bt, int64_t rows, int64_t* rows_out);

/*
 * rg_batch_set_tc_group -- mixed mode's tensor-core block projection (the products of
 * Section 3's block of observations against the block-start basis, 3xTF32): how many
 * 64-column slices of the second product (the rejections Gamma - G Q) are issued back to
 * back into their own tensor-memory accumulators before one wait. group > 0 sets it
 * (1 <= group <= 6, otherwise RG_EINVAL); group <= 0 only queries. group_out (host, may be
 * NULL) receives the value in force (default 6). Host-side only; takes effect at the next
 * rg_batch_add_rows; no effect in FP64 mode. Results do not depend on it. Used by the
 * autotuner.
 */
rg_status rg_batch_set_tc_group(rg_batch* bt, int64_t group, int64_t* group_out);

/* rg_batch_sync -- wait and return any pending device error of the batch. */
rg_status rg_batch_sync(rg_batch* bt);

/* rg_batch_reset -- every instance back to the empty state. Asynchronous. */
rg_status rg_batch_reset(rg_batch* bt);

/* rg_batch_free -- release (synchronises first). NULL is a no-op. */
rg_status rg_batch_free(rg_batch* bt);

/*
 * rg_solve_noalloc -- solve one stream from scratch, as rg_init + rg_add_rows + rg_solution
 * would, WITHOUT allocating any memory. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc, for example a latency-critical loop that
 * cannot accept cudaMalloc's implicit device synchronisation, or a host application whose
 * device memory is owned entirely by its own allocator.
 *   Gamma      device, n x m row-major FP64;  y  device, n FP64 targets;  n >= 0.
 *   m, tol, flags, r_max: as rg_init.
 *   X          device, m FP64: receives the minimum-norm least-squares solution.
 *   rank_out   host, may be NULL. When given, the call synchronises the stream, stores the
 *              rank and returns any device-side error (non-finite row, capacity). When NULL
 *              the call is asynchronous and device-side errors of this call cannot be read
 *              at all (the next call clears the status word). Pass NULL while the stream is
 *              being captured: the synchronisation is not allowed during a capture.
 *   cuda_stream  cudaStream_t for all work (NULL: legacy default stream).
 * State and scratch live in one fixed file-scope device array of 8 MiB that every GPU
 * loading the library holds until the process exits; a problem whose state and scratch do
 * not fit is rejected with RG_EINVAL and a message. With r_max = m the limits are m <= 494
 * in FP64, m <= 568 in FP64 with RG_ORTHONORMAL (no dual basis to keep) and m <= 528 in
 * mixed mode; a smaller r_max raises them.
 * Every call shares that array and clears what must start at zero itself; calls that
 * overlap on the GPU (different streams or host threads) race on it and must be
 * serialised by the caller. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.
 */
rg_status rg_solve_noalloc(const double* Gamma, const double* y, int64_t n, int64_t m,
                           double tol, int flags, int64_t r_max, double* X, int64_t* rank_out,
                           void* cuda_stream);

/* Thread-local description of the last error returned on this thread ("" if none). */
const char* rg_last_error(void);

/* Library version string. */
const char* rg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RG_H */
