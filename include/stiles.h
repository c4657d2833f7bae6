/*
 * stiles.h -- C ABI of the GB300 (sm_103a) selected-inversion library.
 *
 * Computes, for a symmetric positive definite block-arrowhead matrix A,
 *   (1) the tiled Cholesky factor A = L L^T restricted to the band-plus-arrow
 *       tile pattern (Sec. III of the sTiles selected-inversion paper,
 *       arXiv 2504.19171: POTRF / TRSM / SYRK / GEMM on the structurally
 *       non-zero tiles), and
 *   (2) the selected inverse Sigma = A^{-1} on exactly the tiles of L
 *       (Sec. III-B, Fig. 2 case 7: the selection equals L's pattern), by the
 *       two-phase method: phase 1 (Algorithm 2) inverts each diagonal tile of
 *       L and scales the off-diagonal tiles, phase 2 (Algorithm 3, with the
 *       tile recurrences of Sec. III-A) sweeps the tile columns backwards,
 *   (3) logdet(A) = 2 * sum log diag(L).
 *
 * Matrix model. nt band tile columns of order b, lower bandwidth `band`
 * tiles (w), and an arrow tile row of height `arrow` (a, tile index nt):
 *   struct(k) = { k+1 .. min(k+w, nt-1) }  U  { nt   if a > 0 },
 * tile (i,k) is in the pattern iff i == k or i in struct(k). n = nt*b + a.
 * a = 0 gives a pure block-banded matrix; w = 0 a block-diagonal one.
 *
 * Tile layout (the same for A, L and Sigma; "packed band+arrow layout").
 * Every tile is a dense column-major array whose leading dimension is its
 * row count (b, or a for arrow tiles). Tile column k < nt occupies the
 * fixed-stride slot
 *     colstride = (1 + w) * b * b + a * b            doubles
 * starting at k * colstride:
 *     (k,k)       at k*colstride                     b x b
 *     (k+d,k)     at k*colstride + d*b*b,  1<=d<=w    b x b
 *     (nt,k)      at k*colstride + (1+w)*b*b          a x b
 * and the corner (nt,nt) (a x a) sits at nt*colstride. Total doubles:
 *     stiles_layout_doubles = nt*colstride + a*a.
 * Sub-diagonal slots with k+d > nt-1 exist but are never read or written.
 * Input A: only the lower triangle of diagonal tiles is read.
 * Output L: lower triangle of diagonal tiles; their strict upper triangle
 * is written as zero. Output Sigma: every entry of every pattern tile,
 * diagonal tiles full and exactly symmetric.
 *
 * Memory ownership. All device buffers (A, L, Sigma, scratch) belong to the
 * caller (e.g. torch.empty(..., device="cuda")). The handle owns host
 * metadata, a read-only device task table built at create time, and a small
 * device status block (status word, logdet partial sums). Launches are
 * asynchronous on the caller's stream; one handle runs one launch at a time
 * (its status block and the caller's scratch are per launch).
 *
 * Precision. STILES_FP64 computes everything in IEEE binary64 on the FP64
 * pipe (GB300's tcgen05 tensor cores have no FP64 kind); STILES_EMU64 and
 * STILES_FP32X lower only the off-diagonal bulk products (see
 * stiles_precision).
 *
 * Errors. Every function returns STILES_OK (0) or a negative code. Launch
 * functions only report argument and CUDA launch errors; numerical status
 * (NOT_SPD, TIMEOUT) is read with stiles_status / stiles_logdet, which wait
 * for the last launch of the handle to finish.
 */
#ifndef STILES_H
#define STILES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stiles_handle *stiles_t;

enum stiles_status_code {
  STILES_OK = 0,
  STILES_ERR_INVALID_ARG = -1, /* bad shape, null pointer, wrong handle state */
  STILES_ERR_NOT_SPD = -2,     /* a pivot of POTRF was not positive (or NaN) */
  STILES_ERR_TIMEOUT = -3,     /* a bounded dependency wait on the device expired */
  STILES_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  STILES_ERR_OOM = -5,         /* host or device allocation for the handle failed */
  STILES_ERR_UNSUPPORTED = -6, /* precision or option not available */
  STILES_ERR_PLAN = -7,        /* a task table failed its consistency check */
  STILES_ERR_TOO_LARGE = -8,   /* the shape's scratch does not fit the fixed no-allocation array */
  STILES_ERR_BUSY = -9         /* request server: no memory or slot free now (retry after a release) */
};

/* Precision of the off-diagonal bulk products (the factor's GEMM/SYRK
 * updates, the TRMM of phase 1, and the products of phase 2). The diagonal
 * POTRF, TRSM, TRTRI, LAUUM and the Sigma_ii assembly (subtract, mirror)
 * always run in FP64.
 *   STILES_FP64   IEEE binary64 on the FP64 pipe.
 *   STILES_EMU64  emulated FP64: every operand is split, per row / column of
 *                 its panel, into seven 8-bit integer digits (56-bit fixed
 *                 point, the entry's sign on each) held exactly in bf16;
 *                 digit products run on the tensor cores with exact FP32
 *                 accumulation per K chunk, move into int32 level sums and
 *                 are recombined exactly in 128-bit integers, then rounded to
 *                 FP64 (split-precision scheme of Ozaki, Ogita, Oishi and
 *                 Rump). Error of a product term about 8 x 2^-56 of
 *                 (max |row| x max |column|).
 *   STILES_FP32X  FP32-class: operands rounded to FP32, FP32 FMA accumulation. */
enum stiles_precision { STILES_FP64 = 0, STILES_EMU64 = 1, STILES_FP32X = 2 };

/* Create a handle for one matrix shape.
 *   nt >= 1 band tile columns, b >= 1 tile order, band = w >= 0 lower tile
 *   bandwidth (clipped to nt-1), arrow = a >= 0 arrow width,
 *   precision = STILES_FP64, STILES_EMU64 or STILES_FP32X.
 * Builds the task DAG of the factorization, of the selected inversion and of
 * both fused (host, C++), orders each by a critical-path list schedule, and
 * uploads the tables. Returns STILES_ERR_INVALID_ARG for a bad shape,
 * STILES_ERR_UNSUPPORTED for another precision, STILES_ERR_OOM /
 * STILES_ERR_CUDA if the tables cannot be placed on the current device.
 * On success *out owns the handle; release it with stiles_destroy. */
int stiles_create(int nt, int b, int band, int arrow, int precision, stiles_t *out);

/* Same as stiles_create with a tuning code (0 = the defaults; the project's
 * autotuner picks one per (b, band, arrow blocks, precision)). Bits 0-5
 * change only how the work is cut into tasks: bits 2-5 split output blocks
 * among CTAs differently (bit-identical results); bits 0-1 group the
 * factor's update terms differently (results equal up to rounding). Bit 6
 * changes which products a reduced-precision handle lowers:
 *   bits 0-1  factor: source block columns per update task for tile columns
 *             older than k-1 (0: 8, 1: 4, 2: 16, 3: 32)
 *   bits 2-3  phase 2: parts of an off-diagonal Sigma block task
 *             (0: four 32 x 32 quadrants, 1: two 32-row halves, 2: whole)
 *   bits 4-5  factor: parts of the newest update of an off-diagonal block
 *             (0: four quadrants, 1: whole)
 *   bit 6     STILES_EMU64 / STILES_FP32X: also lower the block updates inside
 *             each diagonal tile (its POTRF's own SYRK / GEMM steps); with 0
 *             the whole diagonal-tile POTRF runs in true FP64
 * Other codes return STILES_ERR_INVALID_ARG. */
int stiles_create_tuned(int nt, int b, int band, int arrow, int precision, int tuning, stiles_t *out);

/* General selections (Sec. III-B, Fig. 2). Sigma tile (j, i) depends only on
 * Sigma of tile columns after i (the recurrences of Sec. III-A run from the
 * last column backwards), so any set of requested entries (r, c) of Sigma is
 * served by computing tile columns >= first_column = min over the set of
 * min(r, c) / b (arrow rows and columns: tile nt); those columns' phase-1 and
 * phase-2 tasks are all that is kept (the factorization is always complete).
 * This handle computes Sigma on L's pattern for tile columns >= first_column
 * and writes no Sigma tile of earlier columns. 0 <= first_column <= nt (< nt
 * without an arrow). The full inverse (Fig. 2 case 6) is the pattern with
 * band = nt - 1: pack the tiles outside A's own band as zeros.
 * Task cutting: the fused plan of every column (first_column 0) applies the
 * factor's far update terms in runs of several block columns, for
 * throughput; the factor-only plan and the fused plans with first_column > 0
 * apply them one block column at a time, for the shortest critical path. The
 * two cuttings give L, logdet and Sigma that agree up to rounding. */
int stiles_create_selected(int nt, int b, int band, int arrow, int precision, int first_column, stiles_t *out);

/* Doubles of one packed A / L / Sigma buffer (see the layout above). */
int stiles_layout_doubles(stiles_t h, size_t *doubles);

/* Bytes the caller must provide: L and Sigma buffers (equal to the packed
 * size * 8) and a scratch buffer (device, 256-byte aligned) that holds
 * L_ii^{-1}, the scaled off-diagonal tiles L_ki L_ii^{-1} and the device
 * scheduler's state (dependency counters and ready queues). Any pointer may
 * be NULL to skip it. */
int stiles_workspace_bytes(stiles_t h, size_t *L_bytes, size_t *sigma_bytes, size_t *scratch_bytes);

/* Tiled Cholesky (Sec. III): reads A_tiles (device, packed layout), writes
 * L_tiles (device, packed layout). A_tiles and L_tiles may be the same
 * buffer (in-place factorization). scratch: device, >= scratch_bytes.
 * One persistent kernel launch on `stream` (a cudaStream_t, NULL = legacy
 * default stream). Asynchronous: a non-SPD matrix is reported by
 * stiles_status / stiles_logdet as STILES_ERR_NOT_SPD with the LAPACK-style
 * 1-based global column of the first failing pivot. */
int stiles_factor(stiles_t h, const double *A_tiles, double *L_tiles, void *scratch, void *stream);

/* Selected inversion (Algorithms 2 and 3): reads L_tiles (device, output of
 * stiles_factor, complete before this launch in stream order), writes
 * Sigma_tiles (device, packed layout; must not alias L_tiles or scratch).
 * One persistent kernel launch on `stream`; asynchronous. */
int stiles_selinv(stiles_t h, const double *L_tiles, double *Sigma_tiles, void *scratch, void *stream);

/* Factorization and selected inversion in ONE persistent launch: the phase-1
 * work of tile column i starts as soon as column i of L is final, while
 * later columns are still being factored. Same buffers and rules as the two
 * calls above (A_tiles may alias L_tiles; Sigma_tiles must not alias
 * either). Asynchronous. */
int stiles_factor_selinv(stiles_t h, const double *A_tiles, double *L_tiles, double *Sigma_tiles, void *scratch,
                         void *stream);

/* End-to-end form of stiles_factor_selinv for callers whose matrix lives in
 * host memory: A_host (stiles_layout_doubles doubles, the packed tile layout)
 * in, Sigma_host (same layout) out, the fused factor + selected inversion in
 * between, all on `stream`. Two ways, chosen per call:
 *   - A_host and Sigma_host page-locked and mapped into the device's address
 *     space (cudaHostAlloc, cudaHostRegister with cudaHostRegisterMapped, or
 *     torch pin_memory on a unified-addressing system; each buffer inside one
 *     such allocation) and not overlapping: the kernel reads each block of A
 *     over the host link when its first factor task needs it, and writes
 *     every final Sigma block to Sigma_host as well as to Sigma_dev, so both
 *     transfers overlap the computation. A_dev is not used (not written).
 *     Entries of Sigma_host outside the computed tiles keep their values.
 *   - otherwise: copy A_host into A_dev, run the fused call, copy Sigma_dev
 *     back into Sigma_host (page-locked buffers make the copies asynchronous;
 *     A_host and Sigma_host may then be the same buffer).
 * Host buffers must stay valid, A_host unchanged and Sigma_host unread, until
 * the stream reaches the end of the call.
 * Device buffers follow the rules of stiles_factor_selinv (A_dev may alias
 * L_dev; Sigma_dev holds the full result in both ways). Asynchronous: read
 * the status / logdet afterwards as usual. */
int stiles_factor_selinv_host(stiles_t h, const double *A_host, double *Sigma_host, double *A_dev, double *L_dev,
                              double *Sigma_dev, void *scratch, void *stream);

/* Allocation-free variant of stiles_factor_selinv (the paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory when they run the factorization, such as services whose device
 * memory is reserved once at start-up by their own allocator and may not grow
 * while serving, or code that must not call cudaMalloc at that point).
 * Same arguments as stiles_factor_selinv minus `scratch`: instead of a
 * caller buffer it uses a fixed array of STILES_NOALLOC_SCRATCH_BYTES
 * (64 MiB) defined in the library (a file-scope __device__ array, so every
 * GPU that loads the library holds it until the process exits). The call
 * allocates nothing. The handle must already exist (stiles_create allocates
 * its task tables when it is created, not here).
 *   - Shapes whose scratch (stiles_workspace_bytes) exceeds the array return
 *     STILES_ERR_TOO_LARGE and launch nothing.
 *   - A call whose stream is not capturing looks up the array's device
 *     address (cudaGetSymbolAddress, with the handle's device current) and
 *     remembers it; a call made during stream capture uses the address the
 *     last uncaptured call on that device remembered, and returns
 *     STILES_ERR_INVALID_ARG if there was none. So make one uncaptured call
 *     on a device before capturing this entry point into a graph, and again
 *     after a device reset (cudaDeviceReset, or a reset of the primary
 *     context by another library), which unloads the array.
 *   - Every call, from every handle, shares the one array and leaves its
 *     contents behind; each call re-initialises the part that must start from
 *     a known state (the scheduler state) on its stream before the launch.
 *     Calls whose launches overlap on the GPU (other streams, other threads)
 *     race on the array: serialise them.
 * Status and logdet are read as usual with stiles_status / stiles_logdet. */
#define STILES_NOALLOC_SCRATCH_BYTES (64ull << 20)
int stiles_factor_selinv_noalloc(stiles_t h, const double *A_tiles, double *L_tiles, double *Sigma_tiles, void *stream);

/* logdet(A) = 2 * sum log diag(L) from the last factorization of this handle
 * (stiles_factor or stiles_factor_selinv; a later stiles_selinv does not
 * change it). Waits for the handle's last launch. Returns that
 * factorization's status code (STILES_OK, STILES_ERR_NOT_SPD,
 * STILES_ERR_TIMEOUT), or STILES_ERR_INVALID_ARG if the handle has not
 * factorized yet; *out_host is written only on STILES_OK. */
int stiles_logdet(stiles_t h, double *out_host);

/* Device status of the last launch (check it after stiles_factor before
 * calling stiles_selinv: a selected inversion of a failed factor returns
 * meaningless values with an OK status). Waits for it, then writes *code (a
 * stiles_status_code), *info (NOT_SPD: 1-based global column of the first
 * failing pivot; TIMEOUT: index of the task whose wait expired; else 0) and
 * *tasks_done (tasks that completed). Any output pointer may be NULL.
 * Returns STILES_OK if the status could be read. */
int stiles_status(stiles_t h, int *code, long long *info, long long *tasks_done);

/* Options. STILES_OPT_WAIT_BUDGET_NS: bound of one device dependency wait in
 * nanoseconds (default 20 s); when it expires the launch stops with
 * STILES_ERR_TIMEOUT instead of hanging. STILES_OPT_GRID: persistent CTAs per
 * launch (0 = the default, two per SM). STILES_OPT_TRACE: 1 allocates a
 * device trace buffer (32 bytes per task) and makes every later launch record
 * per-part %globaltimer stamps (read with stiles_trace); 0 frees it (default
 * off: tracing costs a few extra stores per part). Returns STILES_ERR_INVALID_ARG
 * for an unknown option or value. */
enum stiles_option { STILES_OPT_WAIT_BUDGET_NS = 1, STILES_OPT_GRID = 2, STILES_OPT_TRACE = 3 };
int stiles_set_option(stiles_t h, int option, long long value);

/* Per-part trace of the last launch (tracing must be on). Waits for the
 * launch. *n_tasks receives the task count of that launch; if out_host is not
 * NULL it must hold capacity >= 16 * n_tasks words and receives 4 records of
 * 4 words per task (one per possible part, in list-schedule order; records of
 * parts a task does not have are zero): time the worker started looking for
 * work, time it got this part, end time (ns of the GPU's global timer), and
 * (sm << 32 | cta << 12 | precision << 10 | last part << 9 | urgent << 8 | op). */
int stiles_trace(stiles_t h, unsigned long long *out_host, size_t capacity, size_t *n_tasks);

/* Plan statistics for a shape, computed on the host (no GPU, no handle).
 * which: 0 = factor plan, 1 = selinv plan, 2 = fused plan, plus 16 x the
 * stiles_precision of the plan (e.g. 2 + 16 * STILES_EMU64), plus 256 x a
 * tuning code (stiles_create_tuned), plus 65536 x a first selected column
 * (stiles_create_selected); workers = number
 * of persistent workers the list schedule assumes (e.g. the SM count).
 * stats[0] tasks, [1] segments, [2] waits, [3] counters,
 * [4] algorithmic flops of the tile operations (POTRF, TRTRI, LAUUM m^3/3;
 *     TRSM, TRMM m k^2; SYRK and the symmetric Sigma_ii update m^2 k;
 *     GEMM 2 m n k),
 * [5] phase-2 tile GEMMs: (tile, tile) products accumulated into Sigma tiles
 *     (the count of the GEMM-count table of Sec. III-E and Appendix A),
 * [6] critical path and [7] list-schedule makespan, in estimated ns,
 * [8] the part of [4] that runs as block products in the plan's reduced
 *     precision (0 for STILES_FP64; the rest stays on the FP64 pipe),
 * [9] successor edges of the dependency graph (each costs one device atomic
 *     when its source task completes).
 * Returns STILES_ERR_INVALID_ARG for a bad shape, STILES_ERR_PLAN if the
 * table fails its consistency check. */
int stiles_plan_stats(int nt, int b, int band, int arrow, int which, int workers, long long stats[10]);

/* Test hook: CTAs of the persistent kernel that can be resident on one SM of
 * the current device with the shared memory of an FP64 plan (tensor_parts =
 * 0) or of a plan with tensor-core parts (1); the kernel is designed for 2.
 * Returns STILES_ERR_CUDA if the query fails. */
int stiles_debug_occupancy(int tensor_parts, int *blocks_per_sm);

/* Test hook: build the plan `which` (as in stiles_plan_stats) for a shape and
 * emulate one launch of it on the host: every memory access of every task
 * part stays inside its buffer, every queue stays inside its capacity, and
 * every task is released exactly once. Returns STILES_OK or STILES_ERR_PLAN
 * (the first problem is printed to stderr). Host only. */
int stiles_debug_validate(int nt, int b, int band, int arrow, int which);

/* Test hook: build the plan `which` for a shape, corrupt its dependency table
 * on the host (mode 1: one wait names a counter beyond the table; mode 2: one
 * wait needs one more signal than exists; mode 3: a wait on a task later in
 * claim order) and return the consistency check's result (expected
 * STILES_ERR_PLAN). Host only. */
int stiles_debug_check_corrupted(int nt, int b, int band, int arrow, int which, int mode);

/* Test hook: build the plan `which` (as in stiles_plan_stats) and check it
 * for races on the host: the table is replayed in its order and every two
 * task parts that touch the same element of A, L, Sigma or the scratch
 * tiles, one of them writing it, must be ordered by the dependency graph
 * (parts of one task run side by side and must not conflict at all). The
 * accesses follow the kernel's: operand regions of each segment, the input
 * sub-block, the lower triangle of a triangular block, the output sub-block,
 * SYMUPD's mirror, the rows a ZERO task clears. plant = 1 removes every
 * predecessor of the last POTRF that has some before the check; plant = 2
 * removes every edge into the first column-join task of a fused plan (its
 * tile column's phase 1 then no longer follows that column of L). Both are
 * planted races, expected to be found. Returns STILES_OK, STILES_ERR_PLAN
 * (the first race printed to stderr) or STILES_ERR_INVALID_ARG (bad
 * arguments, plant = 2 on a plan without a join task, or a plan of more
 * than 16384 tasks). Host only; memory grows with the buffers
 * (12 bytes per element) -- meant for small shapes. */
int stiles_debug_race_check(int nt, int b, int band, int arrow, int which, int plant);

/* Test hook: the same race check for the request-server template of a shape
 * (precision and tuning as in stiles_server_create): a served request's A is
 * built in place in L by the template's PREP tasks, so A references alias L
 * and each PREP task writes its whole tile column of L. plant as above.
 * Returns STILES_OK, STILES_ERR_PLAN (first race on stderr) or
 * STILES_ERR_INVALID_ARG. Host only; small shapes. */
int stiles_debug_race_check_serve(int nt, int b, int band, int arrow, int precision, int tuning, int plant);

/* Test hook: the same race check for the merged table of a batch (shapes
 * and tuning codes as in stiles_debug_validate_batch; each matrix at its own
 * offset in the shared buffers): conflicts inside a matrix and across
 * matrices (an offset that lets two matrices overlap) are both reported.
 * plant as in stiles_debug_race_check. Host only; small batches. */
int stiles_debug_race_check_batch(int count, const int *nt, const int *b, const int *band, const int *arrow,
                                  int precision, const int *tuning, int plant);

/* Test hook: make the handle's plan `which` unsatisfiable on the device (one
 * task waits for one more predecessor than it has) without the host check,
 * so that a launch must end with STILES_ERR_TIMEOUT once the wait budget
 * expires. Used to test that a stuck dependency ends the kernel cleanly. */
int stiles_debug_break_plan(stiles_t h, int which);

/* Release the handle (waits for its last launch). Accepts NULL. */
int stiles_destroy(stiles_t h);

/* Human-readable name of a status code. */
/* ---------------------------------------------------------------- batch --
 * Many independent matrices of different shapes factored and inverted in ONE
 * persistent launch (no counterpart in the paper, which treats one matrix at
 * a time). Their task tables are merged into one table and ordered by one
 * critical-path list schedule, so the small matrices fill the GPU beside the
 * sequential factorization chains of the large ones.
 *
 * Layout. Matrix m occupies doubles [off[m], off[m] + stiles_layout_doubles
 * of its shape) of each batch buffer (A, L, Sigma), in the packed band+arrow
 * layout of its own shape; off[] (multiples of 32 doubles) comes from
 * stiles_batch_offsets. A, L and Sigma are separate caller buffers of
 * off[count] doubles each (A may alias L); the scratch buffer holds every
 * matrix's L^-1 / U tiles at the same offsets plus the scheduler state.
 *
 * Launch. stiles_batch_factor_selinv enqueues a CUDA graph (built on the first
 * call for a given set of buffer pointers, re-used while they stay the same)
 * whose nodes reset the scheduler state and the status blocks and run the
 * persistent kernel: one graph launch per batch. Asynchronous; one launch at
 * a time per batch handle.
 *
 * Status. Per matrix: STILES_OK, STILES_ERR_NOT_SPD with the 1-based global
 * column of its first failing pivot, or the launch-wide STILES_ERR_TIMEOUT /
 * STILES_ERR_PLAN (a timeout stops every matrix). */
typedef struct stiles_batch *stiles_batch_t;

/* count >= 1 shapes (nt[m], b[m], band[m], arrow[m], as for stiles_create),
 * one precision for the whole batch, tuning[m] as for stiles_create_tuned
 * (NULL: all 0). Returns the codes of stiles_create. */
int stiles_batch_create(int count, const int *nt, const int *b, const int *band, const int *arrow, int precision,
                        const int *tuning, stiles_batch_t *out);

/* off[0 .. count]: offset (doubles) of each matrix in the batch buffers;
 * off[count] = doubles of each of the A, L and Sigma buffers. */
int stiles_batch_offsets(stiles_batch_t h, size_t *off);

/* Bytes of each of A, L, Sigma (off[count] doubles) and of the scratch. */
int stiles_batch_workspace_bytes(stiles_batch_t h, size_t *buffer_bytes, size_t *scratch_bytes);

/* Fused factor + selected inversion of every matrix of the batch in one graph
 * launch on `stream` (a cudaStream_t, or NULL for the default stream).
 * scratch must be 256-byte aligned. */
int stiles_batch_factor_selinv(stiles_batch_t h, const double *A, double *L, double *Sigma, void *scratch,
                               void *stream);

/* Status of matrix `index` after the last launch (waits for it): *code as
 * above, *info = 1-based failing column for NOT_SPD, else 0. */
int stiles_batch_status(stiles_batch_t h, int index, int *code, long long *info);

/* logdet of every matrix (out_host[count]); waits for the last launch.
 * Entries of matrices whose status is not STILES_OK are NaN. Returns the
 * launch-wide error (TIMEOUT / PLAN) if there was one, else STILES_OK. */
int stiles_batch_logdet(stiles_batch_t h, double *out_host);

/* STILES_OPT_WAIT_BUDGET_NS and STILES_OPT_GRID, as for a single handle. */
int stiles_batch_set_option(stiles_batch_t h, int option, long long value);

/* Plan statistics of the merged table (same fields as stiles_plan_stats). */
int stiles_batch_stats(stiles_batch_t h, long long stats[9]);

/* --------------------------------------------------------------- server --
 * Request server with continuous batching (no counterpart in the paper; its
 * use case is the hyperparameter sweep of INLA-type models, where many
 * selected inversions of matrices with a fixed pattern and varying values are
 * needed). One persistent kernel keeps running; requests are admitted while
 * others execute and their tasks share the GPU with them.
 *
 * A request names a pool shape and two value parameters: its matrix is the
 * shape's base matrix B (set once) rescaled as
 *     A = rho * (band entries of B) + (arrow entries of B),
 *     diag(A)_i = tau + rho * rb_i + ra_i,
 * with rb / ra the caller's band / arrow absolute row sums of B (so A stays
 * strictly diagonally dominant for every tau > 0, rho > 0 when B's diagonal
 * is). The kernel builds A in the request's own memory (one task per tile
 * column), factors it in place and computes Sigma on L's pattern.
 *
 * Memory. stiles_server_create allocates everything once: base values of
 * every shape, a data arena of data_bytes from which each request takes its
 * L, Sigma and scratch (3 x stiles_layout_doubles of its shape, rounded up to
 * 32 doubles; stiles_server_request_bytes), task-table arenas for
 * max(4, max_requests) copies of the largest shape, ready rings and a pinned,
 * host-mapped control block. stiles_server_submit returns STILES_ERR_BUSY if
 * the request does not fit now (admission by HBM footprint): retry after a
 * stiles_server_release.
 *
 * Threading: the functions of one server are called from one host thread. */
typedef struct stiles_server *stiles_server_t;

/* Pool of nshapes shapes (as for stiles_create), one precision, optional
 * per-shape tuning codes, data arena bytes, request slots (1 .. 1024). */
int stiles_server_create(int nshapes, const int *nt, const int *b, const int *band, const int *arrow, int precision,
                         const int *tuning, size_t data_bytes, int max_requests, stiles_server_t *out);

/* Packed-layout doubles and matrix order n of a pool shape. */
int stiles_server_shape_doubles(stiles_server_t h, int shape, size_t *doubles, size_t *n);

/* Base matrix of a shape (packed layout, stiles_server_shape_doubles
 * doubles) and its band / arrow absolute row sums (n doubles each); host or
 * device pointers. Every shape needs one before stiles_server_start. */
int stiles_server_set_base(stiles_server_t h, int shape, const double *base, const double *rb, const double *ra);

/* Launch the server kernel (on the server's own stream). Idle workers give up
 * window_s seconds after the launch (STILES_ERR_TIMEOUT from
 * stiles_server_stop): a bound, so that a host that never stops the server
 * cannot keep the GPU. */
int stiles_server_start(stiles_server_t h, double window_s);

/* Admit a request of pool shape `shape` with (tau, rho); `tag` is returned by
 * stiles_server_poll. On STILES_OK *request is its slot. STILES_ERR_BUSY if
 * no memory or slot is free now. */
int stiles_server_submit(stiles_server_t h, int shape, double tau, double rho, long long tag, int *request);

/* Admit a request of pool shape `shape` with explicit values: A_host (host
 * memory, the shape's packed layout, stiles_server_shape_doubles doubles) is
 * copied into the request's memory before it joins the kernel, instead of
 * being built from the base matrix. Same results and errors as
 * stiles_server_submit. */
int stiles_server_submit_values(stiles_server_t h, int shape, const double *A_host, long long tag, int *request);

/* Requests completed since the last poll, each reported once (up to max). */
int stiles_server_poll(stiles_server_t h, int max, int *requests, long long *tags, int *n_out);

/* Status (STILES_OK / STILES_ERR_NOT_SPD with the 1-based failing column in
 * *info) and logdet (NaN unless OK) of a completed request. */
int stiles_server_result(stiles_server_t h, int request, int *code, long long *info, double *logdet);

/* Sigma of a completed request (packed layout of its shape): copied to
 * host_out (host memory while the server runs: a device-side copy could need
 * an SM, which the running kernel holds) if not NULL, and/or its device
 * address in *device_ptr (valid until the request is released). */
int stiles_server_sigma(stiles_server_t h, int request, double *host_out, const double **device_ptr);

/* Free a completed request's memory, tables and slot. */
int stiles_server_release(stiles_server_t h, int request);

/* Status of the server kernel read while it runs: *code STILES_OK, or
 * STILES_ERR_TIMEOUT once a wait (or the window) expired; *info the first
 * error's detail; *tasks_done tasks completed since the start. */
int stiles_server_status(stiles_server_t h, int *code, long long *info, long long *tasks_done);

/* Data-arena bytes a request of `shape` takes. */
int stiles_server_request_bytes(stiles_server_t h, int shape, size_t *bytes);

/* Ask the kernel to stop once idle (call after every request completed) and
 * wait for it. STILES_OK, or STILES_ERR_TIMEOUT if the window ran out. */
int stiles_server_stop(stiles_server_t h);

/* Stops the kernel if running, frees everything. */
int stiles_server_destroy(stiles_server_t h);

/* Test hook (host only, no device): build the merged table of a batch and
 * emulate a launch of it (bounds of every access within the batch buffers,
 * queue capacities, every task released once). Returns STILES_OK or
 * STILES_ERR_PLAN. */
int stiles_debug_validate_batch(int count, const int *nt, const int *b, const int *band, const int *arrow,
                                int precision, const int *tuning);

/* Test hook (host only): build the request-server table of one shape and
 * emulate a launch of it (as stiles_debug_validate). */
int stiles_debug_validate_serve(int nt, int b, int band, int arrow, int precision, int tuning);

/* Waits for the last launch, frees the tables, the graph and the handle. */
int stiles_batch_destroy(stiles_batch_t h);

const char *stiles_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* STILES_H */
