/*
 * sttsm.h — C ABI of the GB300 (sm_103a) library for the symmetric tensor
 * times same matrix operation on Blocked Compact Symmetric Storage.
 *
 * Paper: M. D. Schatz, T. M. Low, R. A. van de Geijn, T. G. Kolda,
 * "Exploiting Symmetry in Tensors for High Performance: Multiplication with
 * Symmetric Tensors", arXiv 1301.7744.
 *
 * Operation (eq. (cob), Sec. 2.5):  C := [A; X, ..., X] = A x_0 X x_1 ... x_{m-1} X,
 *   gamma_{j_0..j_{m-1}} = sum_{i in [0,n)^m} alpha_{i_0..i_{m-1}} prod_k chi_{j_k, i_k},
 * with A an order-m symmetric tensor of dimension n, X a p x n matrix and C
 * an order-m symmetric tensor of dimension p.
 *
 * Conventions used by every entry point:
 *   - Indices are 0-based (Sec. 2.1).
 *   - Dense tensors are in dimensional order (App. A): entry (i_0..i_{m-1})
 *     at offset sum_k i_k n^k, mode 0 fastest.
 *   - X is p x n, column-major: chi_{j,i} at X[j + i*p] (the libflame
 *     convention the paper follows, Sec. 3.3).
 *   - BCSS (Sec. 3.3, 4.3, 5.3; Tbl. 1): a tensor of dimension n is cut
 *     into blocks of b^m entries, nbar = ceil(n/b) blocks per mode (App. B).
 *     Only blocks with sorted block indices ibar_0 <= ... <= ibar_{m-1}
 *     are stored: C(nbar+m-1, m) blocks.  Stored block with indices
 *     (ibar_0..ibar_{m-1}) has rank sum_k C(ibar_k + k, k + 1) (colex order:
 *     the last block index varies slowest, the order of the paper's loops;
 *     for m = 2, b = 1 it is the element order pictured in Sec. 3.3).  A
 *     block is a dense b^m array in dimensional order.  Block entries that
 *     fall at an index >= n are padding and are zero.  Diagonal blocks are
 *     stored in full (Sec. 3.3); by default every entry of them is computed,
 *     and sttsm_set_inblock_symmetry computes their canonical entries only.
 *   - Device pointers unless stated otherwise.  The caller owns every
 *     buffer; the library never frees caller memory.  The library owns
 *     only small per-shape plans (tile lists) it caches in device memory.
 *   - Every call returns an sttsm_status (or a count); nothing throws
 *     across the ABI.  Arguments are validated before any launch.  Work is
 *     enqueued on `stream` (a cudaStream_t; 0 = legacy default stream).
 *   - A and C must hold symmetric data; the library does not check it.
 */
#ifndef STTSM_H
#define STTSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STTSM_OK = 0,
    STTSM_ERR_ARG = -1,          /* invalid argument (size, pointer, alignment) */
    STTSM_ERR_UNSUPPORTED = -2,  /* valid but not implemented (e.g. m > 8, TF32X3) */
    STTSM_ERR_NOMEM = -3,        /* workspace too small / plan allocation failed */
    STTSM_ERR_TIMEOUT = -4,      /* a device-side bounded wait ran out (status word set) */
    STTSM_ERR_CUDA = -5,         /* a CUDA runtime call failed */
    STTSM_ERR_BUSY = -6          /* serving queue full */
} sttsm_status;

/* Arithmetic of the mode products.
 *   STTSM_FP64:  A, X, C in FP64; FP64 FMAs on the CUDA cores.
 *   STTSM_BF16X6: A, X, C in FP32; every FP32 operand is split into three
 *                 BF16 pieces (hi, mid, lo) and the six piece products whose
 *                 piece orders sum to <= 2 run on the tcgen05 tensor cores
 *                 with FP32 accumulation in tensor memory.
 *   STTSM_BF16X3: as BF16X6 with two pieces and three products (about 2^-16
 *                 relative error per product: cheaper, less accurate).
 *   STTSM_TF32X3: reserved; returns STTSM_ERR_UNSUPPORTED.
 *   STTSM_BF16X6_R64, STTSM_BF16X3_R64: as BF16X6 / BF16X3, with the final
 *                 C-block reduction in FP64 (Fig. 5's last level, C = sum over
 *                 ibar_0 of T^(1) blocks x_0 X blocks): the FP32 partial sums
 *                 of that level — per contraction group of <= 128 indices on
 *                 the tensor cores, per block of b indices on the CUDA-core
 *                 kernel of short contractions — are added in FP64 registers
 *                 and C is rounded to FP32 once.  The last level's tiles are
 *                 then at most 128 columns wide (more launches' worth of
 *                 epilogue work); the other levels are unchanged. */
typedef enum { STTSM_FP64 = 0, STTSM_BF16X6 = 1, STTSM_TF32X3 = 2, STTSM_BF16X3 = 3, STTSM_BF16X6_R64 = 4,
               STTSM_BF16X3_R64 = 5 } sttsm_prec;

/* Element types for bcss_pack / bcss_unpack. */
typedef enum { STTSM_DTYPE_F64 = 0, STTSM_DTYPE_F32 = 1 } sttsm_dtype;

/* ------------------------------------------------------------------ BCSS indexing (host) */

/* Number of stored blocks, C(nbar + m - 1, m) (Tbl. 1).  -1 on bad arguments. */
int64_t bcss_num_blocks(int m, int64_t n, int b);

/* Number of stored entries, b^m C(nbar + m - 1, m) (Tbl. 1).  -1 on bad arguments. */
int64_t bcss_num_elems(int m, int64_t n, int b);

/* Colex rank of a non-decreasing block-index tuple (m entries), i.e. the
 * position of that block in BCSS storage.  -1 if the tuple is not sorted or
 * has a negative entry. */
int64_t bcss_block_rank(int m, const int32_t* sorted_blk_idx);

/* Inverse of bcss_block_rank: writes the sorted tuple of the block stored
 * at `rank` into blk_idx_out[0..m-1].  STTSM_ERR_ARG if rank < 0. */
int bcss_block_unrank(int m, int64_t rank, int32_t* blk_idx_out);

/* Flops of the algorithm-by-blocks with partially symmetric temporaries,
 * Tbl. 4 (MinCosts), BCSS computation row with b_A = b_C = b:
 *   2 nbar b^{m+1} sum_{d=0}^{m-1} C(pbar+d, d+1) C(nbar+m-d-2, m-d-1).
 * This is the useful-flop count that throughput figures are quoted in. */
double sttsm_flops(int m, int64_t n, int64_t p, int b);

/* ------------------------------------------------------------------ BCSS packing (device) */

/* Dense (n^m, dimensional order) -> BCSS.  Reads, for every stored block,
 * the dense entries at its block indices; writes zeros at padding entries.
 * dense: n^m elements; bcss: bcss_num_elems(m,n,b) elements; dtype as
 * sttsm_dtype.  The copy is bit-exact.  1 <= m <= 8, n >= 1, b >= 1. */
int bcss_pack(const void* dense, void* bcss, int m, int64_t n, int b, int dtype, void* stream);

/* BCSS -> dense.  Entry (i_0..i_{m-1}) is read from the block of the sorted
 * block indices at the sorted in-block indices (the canonical entry), so
 * the dense result is exactly symmetric even where the stored diagonal
 * blocks carry rounding asymmetry (Sec. 5.4 mentions this asymmetry and a
 * post-processing step; this is that step).  Bit-exact copy. */
int bcss_unpack(const void* bcss, void* dense, int m, int64_t n, int b, int dtype, void* stream);

/* ------------------------------------------------------------------ sttsm (device) */

/* Bytes of device workspace sttsm_bcss needs: the two ping-pong buffers
 * holding the unique blocks of the partially symmetric temporaries
 * T^(m-1) ... T^(1) (Thm. 1; Tbl. 4 "All temporaries"), one level at a time,
 * plus the split pieces of X for the tensor-core precisions. */
int sttsm_workspace_size(int m, int64_t n, int64_t p, int b, int prec, size_t* bytes);

/* C := [A; X, ..., X] on BCSS (Sec. 5.4 algorithm-by-blocks, Fig. 5, with
 * Thm. 1's partial symmetry exploited in every temporary, Sec. 6.3).
 *   A_bcss: bcss_num_elems(m, n, b) elements (FP64 for STTSM_FP64, else FP32).
 *   X:      p x n column-major, same element type.
 *   C_bcss: bcss_num_elems(m, p, b) elements, written in full (padding
 *           entries become zero).
 *   workspace: >= sttsm_workspace_size bytes, 256-byte aligned.
 * 1 <= m <= 8; b^{m-1} < 2^31; all pointers 16-byte aligned (a 32-byte
 * aligned C_bcss lets the last level of the tensor-core path write whole
 * 32-byte sectors; the result is the same bits either way).  Asynchronous
 * on `stream`.  Returns STTSM_ERR_TIMEOUT if a previous launch on this
 * device recorded a bounded-wait timeout (the status word is then cleared). */
int sttsm_bcss(const void* A_bcss, const void* X, int m, int64_t n, int64_t p, int b,
               void* C_bcss, int prec, void* workspace, size_t ws_bytes, void* stream);

/* Multiplication in all modes but one, the related operation Sec. 2.5 names:
 * B := A x_1 X x_2 ... x_{m-1} X with mode 0 left untransformed, so B is
 * n x p x ... x p and symmetric in its last m-1 modes (Sec. 2.3).  B is the
 * temporary T^(1) of the algorithm-by-blocks (levels 0 .. m-2 of Fig. 5 with
 * Thm. 1), returned in its partially symmetric block storage:
 *   T: sttsm_all_but_one_elems(m, n, p, b) elements (FP64 for STTSM_FP64,
 *      else FP32), laid out [node][ib][b^m]:
 *        node = colex rank of the sorted block tuple (jb_1 <= ... <= jb_{m-1})
 *               of the transformed modes, C(pbar+m-2, m-1) nodes;
 *        ib   = block index of mode 0, nbar blocks per node;
 *        in-block offset i_0 + sum_{t=1}^{m-1} j_t b^t (local indices; mode t
 *               holds the t-th smallest block index of the tuple).
 *      Entries past n (mode 0) or p (modes 1..m-1) are zero.
 *   A_bcss, X, prec, workspace (>= sttsm_workspace_size(m, n, p, b, prec)
 *   bytes) and errors as sttsm_bcss.  2 <= m <= 8 (STTSM_ERR_ARG otherwise). */
int sttsm_bcss_all_but_one(const void* A_bcss, const void* X, int m, int64_t n, int64_t p, int b,
                           void* T, int prec, void* workspace, size_t ws_bytes, void* stream);

/* Elements of the all-but-one result: C(pbar+m-2, m-1) * nbar * b^m; -1 on
 * invalid arguments (m < 2). */
int64_t sttsm_all_but_one_elems(int m, int64_t n, int64_t p, int b);

/* Useful flops of the all-but-one result: the Tbl. 4 sum of sttsm_flops over
 * levels d = 0 .. m-2 only. */
double sttsm_all_but_one_flops(int m, int64_t n, int64_t p, int b);

/* End-to-end variant on HOST buffers: copies A_bcss and X (host, ideally
 * pinned) to the device buffers dA and dX, runs sttsm_bcss, copies C back
 * to the host buffer C_bcss, all enqueued on `stream` (synchronise the
 * stream before reading C_bcss). dA, dX, dC, workspace are device buffers
 * of the sizes sttsm_bcss needs. */
int sttsm_bcss_host(const void* A_bcss, const void* X, int m, int64_t n, int64_t p, int b,
                    void* C_bcss, int prec, void* dA, void* dX, void* dC,
                    void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ batches (device) */

/* One sttsm instance of a batch: device pointers to A (BCSS, block size b),
 * X (p x n column-major) and C (BCSS), in the element type of the batch's
 * precision. */
typedef struct {
    const void* A;
    const void* X;
    void* C;
    int m;
    int64_t n, p;
    int b;
} sttsm_desc;

/* Block size for one instance: the candidate whose tile plan the cost model
 * rates cheapest (split precisions: per-stage MMA time vs gather latency plus
 * a per-tile overhead, summed over every tile of every level; FP64: the
 * Tbl. 4 flop count).  Returns the chosen b (> 0) or an sttsm_status. */
int sttsm_autotune_b(int m, int64_t n, int64_t p, int prec, const int* cands, int ncand);

/* Block size by measurement: for every candidate b the call allocates device
 * buffers of that shape (A, X, C, workspace), fills A and X with a
 * deterministic non-zero pattern, runs sttsm_bcss once to warm up and `reps`
 * times under CUDA events, and keeps the candidate with the smallest median.
 * Candidates that are invalid or do not fit in 90 % of the free device memory
 * are skipped (times_ms entry -1).  The choice is cached per (device, m, n,
 * p, prec, candidate list); with times_ms == NULL a cached choice is returned
 * without measuring, with times_ms (ncand entries) every candidate is
 * measured again and its median (ms) written.  Synchronises the device and
 * allocates (cudaMalloc) for the duration of the call.  Returns the chosen b
 * or an sttsm_status (STTSM_ERR_UNSUPPORTED if no candidate ran). */
int sttsm_autotune_b_measured(int m, int64_t n, int64_t p, int prec, const int* cands, int ncand, int reps,
                              double* times_ms);

/* Batch plan: many independent instances (different m, n, p, b) run as one
 * sequence of launches — per wave, one X-split launch and one launch per
 * level d covering the level-d tiles of every instance with m > d (Fig. 5's
 * levels, with each instance's own plan).  Instances are grouped into
 * waves whose workspaces fit ws_budget bytes (0 = one wave).  The plan owns
 * its tile lists and descriptor tables (device memory).  The descriptors'
 * pointers are captured: the buffers must stay valid while the plan lives.
 * STTSM_ERR_NOMEM if one instance alone exceeds the budget. */
int sttsm_batch_plan_create(const sttsm_desc* d, int count, int prec, size_t ws_budget, void** plan);
int sttsm_batch_workspace_size(const void* plan, size_t* bytes);
int sttsm_batch_info(const void* plan, int* waves, double* useful_flops);

/* Runs the plan on `stream`.  The first run for a given workspace captures
 * the whole launch sequence into a CUDA graph (on an internal stream); later
 * runs replay it with one cudaGraphLaunch.  Every instance's C is written in
 * full, bit-identical to sttsm_bcss on that instance alone. */
int sttsm_batch_run(void* plan, void* workspace, size_t ws_bytes, void* stream);
int sttsm_batch_plan_destroy(void* plan);

/* One-shot batch: plan, run, synchronise `stream`, destroy. */
int sttsm_batch(const sttsm_desc* d, int count, int prec, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ serving (device) */

/* Continuous-batching server for sttsm requests (split precisions only).
 * The handle owns an HBM arena of hbm_budget_bytes for the workspaces of
 * admitted requests, a CUDA stream and a scheduler thread.  Requests wait in
 * a FIFO queue (at most queue_cap) until their workspace fits in the arena;
 * each admitted request advances one level of Fig. 5 per step, and one step
 * covers every active request at its own level in shared launches, so
 * requests arriving while others run overlap with them on the device.
 * A, X and C stay where the caller put them (device memory, BCSS); the
 * caller keeps them valid until the request is done. */
int sttsm_serve_create(size_t hbm_budget_bytes, int prec, int queue_cap, void** handle);

/* Queues one request.  STTSM_ERR_BUSY if the queue is full, STTSM_ERR_NOMEM
 * if its workspace alone exceeds the budget. */
int sttsm_serve_submit(void* handle, const sttsm_desc* d, uint64_t* ticket);

/* done = 1 once C is complete; latency_ms = completion (seen by the
 * scheduler) minus submission, host clock.  Returns STTSM_ERR_TIMEOUT if a
 * device-side wait timed out, or the scheduler's error. */
int sttsm_serve_poll(void* handle, uint64_t ticket, int* done, double* latency_ms);

/* out[6]: submitted, admitted, completed, queued, active, arena bytes in use. */
int sttsm_serve_stats(void* handle, uint64_t* out);

/* Stops the scheduler, waits for the stream, frees the handle.  Requests not
 * yet done are dropped (their C is undefined). */
int sttsm_serve_destroy(void* handle);

/* Allocation-free variant of sttsm_bcss.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * where they call it — code under a fixed, pre-reserved memory budget
 * (embedded and real-time services), plug-ins hosted by a framework that
 * owns every device allocation, and paths where an allocation could stall
 * or fail at an unpredictable moment.  It takes only the inputs and the
 * output; it calls no cudaMalloc, cudaFree or other allocating routine.
 *   Workspace: one file-scope device array of STTSM_NOALLOC_SCRATCH_BYTES
 *   (64 MiB) that every GPU loading the library holds until the process
 *   exits.  It carries the split X pieces, the temporaries and the level
 *   plans.  Shapes that need more return STTSM_ERR_NOMEM before any launch
 *   (m = 3, n = p = 128, b = 32 fits; use sttsm_bcss with a caller
 *   workspace beyond that).
 *   Set-up: the first call on each device looks up the array's device
 *   address (cudaGetSymbolAddress) and page-locks and maps a static host
 *   status word for that device (cudaHostRegister: no allocation); make
 *   that first call before any stream capture.
 *   Errors: a bounded wait that runs out in this entry point's kernels
 *   raises its status word; the next sttsm_bcss_noalloc call on that device
 *   returns STTSM_ERR_TIMEOUT before launching anything and clears it (the C
 *   of the call that timed out is undefined).  sttsm_device_status does not
 *   see this word.
 *   Plans: the level plans of the last shape (m, n, p, b, prec) stay in the
 *   array; a call with another shape rebuilds them on the host and copies
 *   them in on `stream`.  That copy is refused with STTSM_ERR_UNSUPPORTED
 *   while `stream` is capturing.  Work already enqueued or recorded for the
 *   earlier shape must not run after a call with another shape.
 *   Sharing: every call uses the same array and finds the previous call's
 *   contents there.  Calls that overlap on the GPU (several streams or host
 *   threads) race on it and corrupt each other: serialise them.
 * Arguments, layouts and results are those of sttsm_bcss. */
#define STTSM_NOALLOC_SCRATCH_BYTES (64u << 20)
int sttsm_bcss_noalloc(const void* A_bcss, const void* X, int m, int64_t n, int64_t p, int b,
                       void* C_bcss, int prec, void* stream);

/* Self-test of the failure path of sttsm_bcss_noalloc: sets that entry
 * point up on the current device if needed, launches one kernel whose
 * thread waits on an mbarrier nothing arrives on, bounded by limit_ms
 * (0 < limit_ms <= 1000), through the bounded wait the level kernels use,
 * and synchronises the device.  The wait runs out and raises the entry
 * point's status word, which the next sttsm_bcss_noalloc call reports as
 * STTSM_ERR_TIMEOUT.  Returns STTSM_OK, or STTSM_ERR_ARG for an
 * out-of-range limit. */
int sttsm_noalloc_selftest_wait_timeout(double limit_ms);

/* Kernel for short contractions (n̄ b <= 64) under the split precisions:
 * 0 (default) = FP32 FMAs on the CUDA cores, one thread per output row (at
 * least as accurate as BF16X6; tiles of <= 64 columns and <= 64 contraction
 * indices are latency-bound on the tensor cores); 1 = the tcgen05 small-tile
 * kernel.  Process-wide; affects later calls and later batch-plan runs. */
int sttsm_set_small_kernel(int kind);

/* Last two levels of short contractions (the FP32 kernel, n̄ b <= 64 and
 * p̄ b <= 64): one launch that keeps the partially symmetric temporary T^(1)
 * in shared memory (Fig. 5, levels m-2 and m-1: for fixed trailing indices
 * they are the m = 2 product X_{jb0} S X_{jb1}^T of Sec. 3.2 on a slice S of
 * T^(2)), or two launches through T^(1) in the workspace.  Both give the same
 * bits.  mode 0 = two launches everywhere; 1 (default) = one launch in
 * sttsm_bcss (one launch fewer per call), two in batch plans and serving
 * (measured faster there: with many instances per launch the one-level
 * kernel's larger tiles keep the SMs busier than the fused kernel's units);
 * 2 = one launch everywhere.  Process-wide; affects later calls, requests
 * submitted later and batch plans created later.  STTSM_ERR_ARG otherwise. */
int sttsm_set_fused_tail(int mode);

/* Symmetry inside diagonal blocks (Sec. 3.3 and 5.3 store blocks with
 * repeated block indices in full and compute all their entries).  With on = 1,
 * split-precision levels of short contractions of order m <= 5 (n̄ b <= 64,
 * run by the FP32 kernel) compute only the canonical entries of each stored
 * block of T^(k):
 * those whose full indices are non-decreasing within the k leading and
 * within the m - k trailing modes, the modes among which T^(k) is symmetric.
 * The temporaries (in the workspace) hold only those, and the next level reads
 * each operand entry at its canonical position; the level that writes the
 * result copies each canonical entry to every position of its block that
 * equals it by symmetry, so C (or T^(1) of sttsm_bcss_all_but_one) keeps the
 * BCSS layout with full blocks, every diagonal block exactly symmetric.  When b divides n and p the entries
 * computed per level are C(n+k-1, k) C(p+m-k-1, m-k), the minimum flop count
 * of Sec. 6 ("analysis relative to minimum"); the columns of the diagonal
 * child block past the canonical ones are still multiplied and dropped.
 * Canonical rows are not contiguous in memory, so loads and stores coalesce
 * less than in the full computation: on GB300 the mode is faster only where
 * blocks are large and few per mode (m = 5, n = 64, b = 16), slower on small b.
 * Results agree with on = 0 to within rounding (different entries of a
 * diagonal block come from the same sum instead of sums in different orders).
 * The fused last two levels (sttsm_set_fused_tail) are not used while it is
 * on.  Affects later sttsm_bcss calls, batch plans created later and requests
 * submitted later; the allocation-free entry point sttsm_bcss_noalloc always
 * computes every entry.  Default 0.  STTSM_ERR_ARG unless on is 0 or 1. */
int sttsm_set_inblock_symmetry(int on);

/* Device status word: 0 = fine; otherwise the code of the last device-side
 * failure (1 = bounded wait timed out).  Reading clears it. */
int sttsm_device_status(void);

/* Self-test of the failure path: launches one kernel whose thread waits on an
 * mbarrier nothing arrives on, through the same bounded wait the level
 * kernels use but limited to limit_ms (0 < limit_ms <= 1000); the wait runs
 * out, the kernel raises the status word and leaves, and the call returns
 * STTSM_ERR_TIMEOUT with the status cleared (the context stays usable).
 * Synchronises the device.  STTSM_ERR_ARG for an out-of-range limit. */
int sttsm_selftest_wait_timeout(double limit_ms);

/* ------------------------------------------------------------------ diagnostics (host) */

/* The plan sttsm_bcss runs at level d (0 <= d < m; level d reads T^(m-d) and
 * writes T^(m-1-d), Fig. 5) for precision `prec` (which fixes the tile
 * shape).  Host buffers; pass NULL buffers to query the sizes.
 *   tiles:  ntiles x 8 int32 (inst, parent node, first child node, first row,
 *           first column, columns, pad0, pad1), capacity tiles_cap tiles;
 *           pad0 = 1 for TMA-fed tiles of 16 fastest x 8 next rows; in the
 *           in-block-symmetry mode pad0 = 2 | tie pattern of the parent's
 *           blocks << 8 | its first block << 16, pad1 = the parent's canonical
 *           rows, and "first row" counts canonical rows (sttsm_plan_sym_rows);
 *           else 0, 0;
 *   G:      P_out x nbar int32 gather table, (rank << 3) | q, capacity G_cap;
 *   info:   9 int64: k, P_parent, P_out, rows per parent, parent nodes,
 *           child nodes, rows per block R = b^(m-1), b^m, tile rows BM.
 * Returns STTSM_ERR_NOMEM if a capacity is too small. */
int sttsm_plan_level(int m, int64_t n, int64_t p, int b, int prec, int d, int32_t* tiles, int64_t tiles_cap,
                     int32_t* G, int64_t G_cap, int64_t* ntiles_out, int64_t* nG_out, int64_t* info);

/* The canonical-row map of the in-block-symmetry mode (sttsm_set_inblock_symmetry)
 * at level d for parent node `parent` (colex rank of its sorted tuple of d
 * p-blocks; 0 at level 0): for rho = rho0 .. rho0 + count - 1, g_out[i] = the
 * row pr * b^(m-1) + rr (the row map of sttsm_plan_level) of canonical row rho,
 * or -1 past the parent's canonical rows, and tie_out[i] bit a set where modes
 * a and a + 1 of that row hold the same block within one symmetric group.
 * *rows_out = the parent's canonical rows.  Host buffers (any may be NULL).
 * STTSM_ERR_UNSUPPORTED unless m <= 5, n̄ b <= 64 and p̄ < 65536; STTSM_ERR_ARG for an
 * out-of-range level, parent or range. */
int sttsm_plan_sym_rows(int m, int64_t n, int64_t p, int b, int d, int64_t parent, int64_t rho0, int64_t count,
                        int64_t* g_out, uint32_t* tie_out, int64_t* rows_out);

/* The units of the fused launch of levels m-2 and m-1 (sttsm_set_fused_tail)
 * for a short-contraction shape: ntiles x 8 int32 (0, parent node J of level
 * m-2, 0, first trailing local index tuple s0, children of J, tuples in the
 * unit, colex-rank term of J among the C nodes, 0); *group_out = tuples per
 * unit.  Host buffers; NULL tiles queries the count.  STTSM_ERR_UNSUPPORTED if
 * the shape does not take the fused launch, STTSM_ERR_NOMEM if tiles_cap is
 * too small. */
int sttsm_plan_pair(int m, int64_t n, int64_t p, int b, int32_t* tiles, int64_t tiles_cap, int64_t* ntiles_out,
                    int32_t* group_out);

/* Per-launch timing of the library's kernels (diagnostics).  While enabled,
 * every kernel sttsm_bcss launches is bracketed by CUDA events on its
 * stream.  sttsm_profile_enable(1) clears earlier records; (0) stops.
 * sttsm_profile_read waits for the recorded events and copies up to `max`
 * records: kind (0 = FP64 level, 1 = tensor-core level with gathered A,
 * 2 = operand split, 3 = tensor-core level with TMA-fed A, 4 = levels m-2
 * and m-1 fused),
 * level d, useful flops of that launch (Tbl. 4 terms of level d; 0 for the
 * split), and its duration in ms.  *count receives the number of records. */
int sttsm_profile_enable(int on);
int sttsm_profile_read(int max, int* kind, int* level, double* useful_flops, float* ms, int* count);

#ifdef __cplusplus
}
#endif

#endif
