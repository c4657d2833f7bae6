// Task tables shared by the host planner (plan.cpp) and the persistent
// kernel (stiles_kernel.cu).
//
// A plan is a flat list of fine-block tasks in claim order. Every task writes
// one output block of at most FB x FB doubles:
//     acc = sum over its segments  op(A_s) * op(B_s)          (FP64)
// followed by an epilogue (Op) that combines acc with an input block and, for
// POTRF / TRSM / TRTRI, a triangular solve in shared memory. The paper's tile
// operations (Sec. III-A; Algorithms 2 and 3) are split into such tasks over
// FB x FB sub-blocks of the b x b tiles.
//
// Dependencies are counters in device memory: a task lists (counter, need)
// pairs to wait for and the counters it increments when done (the producer /
// consumer flags of Algorithm 3, one per block or block panel instead of one
// per tile).
#pragma once
#include <stdint.h>

namespace stiles {

constexpr int FB = 64;  // fine block order (rows and columns of one task's output)
constexpr int kCtasPerSm = 2;  // persistent CTAs (workers) per SM

// Buffer ids, stored in the top bits of a 64-bit element offset.
enum Buf : int { BUF_A = 0, BUF_L = 1, BUF_S = 2, BUF_W = 3 };
constexpr int BUF_SHIFT = 60;
constexpr int64_t OFF_MASK = (int64_t(1) << BUF_SHIFT) - 1;
inline int64_t mkref(int buf, int64_t off) { return (int64_t(buf) << BUF_SHIFT) | off; }

enum Op : uint8_t {
  OP_UPD = 0,       // out = cin - acc
  OP_POTRF = 1,     // out = chol(cin - acc)           (square, lower; zero above the diagonal)
  OP_TRSM_RLT = 2,  // out = (cin - acc) * T^{-T}      (T = aux, lower n x n)
  OP_TRTRI = 3,     // out = T^{-1}                    (T = aux, lower m x m; zero above)
  OP_TRSM_LLN = 4,  // out = -T^{-1} * acc             (T = aux, lower m x m)
  OP_STORE = 5,     // out = acc
  OP_NEG = 6,       // out = -acc
  OP_SYMUPD = 7,    // out = cin - acc and its transpose into the mirror block (aux)
  OP_PREP = 8,      // served requests: one tile column of A from the shape's base values and the
                    // request's (rho, tau): band entries x rho, arrow entries as they are,
                    // diagonal tau + rho rb[i] + ra[i] (rb / ra = band / arrow absolute row sums)
  OP_ZERO = 9,      // the zrows x n block above out (L's strict upper part in a diagonal tile's
                    // block column) set to zero; off the factorization's critical path
  OP_JOIN = 10,     // no work: one dependency point for many waiters (a tile column of L final)
};

// How a task's output block is divided among CTAs (each part runs as its own
// queue entry; the last part to finish releases the task's successors).
enum PartMode : uint8_t {
  PM_FULL = 0,   // one part: the whole block
  PM_ROWS2 = 1,  // rows [0,32) and [32,64)
  PM_QUAD4 = 2,  // the four 32 x 32 quadrants
  PM_TRI3 = 3,   // quadrants (0,0), (1,0), (1,1): a diagonal block's lower part
  PM_ROWS4 = 4,  // rows [0,16), [16,32), [32,48), [48,64)
  PM_TILE32 = 5, // a grid of at most 2 x 2 sub-tiles of at most 32 x 32 (parts = row tiles x column tiles)
  PM_ROWS8 = 6,  // rows [0,8), [8,16), [16,24), [24,32) of a block of at most 32 rows
  PM_TRI16 = 7,  // quadrants (0,0), (1,0), (1,1) of 16 x 16: the lower part of a square block of at most 32
  PM_QUAD16 = 8, // the 16 x 16 quadrants (0,0), (0,1), (1,0), (1,1) of a block of at most 32 x 32
};

// Arithmetic of a task's block products (its epilogue is always FP64).
enum Precision : uint8_t {
  PREC_FP64 = 0,   // FP64 FMA pipe
  PREC_EMU64 = 1,  // split-precision emulated FP64: 8 fixed-point digits of 8 bits per operand (bf16
                   // planes) against per-row / per-column exponents, products on the tensor cores
  PREC_FP32X = 2,  // FP32-class: each operand's FP32 value as three bf16 pieces, products on the
                   // tensor cores with FP32 sums
};

// Task flags.
enum TaskFlag : uint8_t {
  TF_SYM_DIAG = 1,  // OP_SYMUPD on a diagonal block (mirror inside the block)
  TF_URGENT = 2,    // on the critical path: queued ahead of the buckets
  TF_CORNER = 4,    // OP_PREP of the arrow corner column
};

struct Seg {       // acc += op(A) (m x k) * op(B) (k x n)
  int64_t a, b;    // buffer refs (mkref) of element (0,0) of the stored operands
  int32_t lda, ldb;
  int32_t k;       // inner length
  int32_t trans;   // bit 0: op(A) = A^T ; bit 1: op(B) = B^T
};

struct Wait {
  int32_t ctr;
  int32_t need;    // wait until counter >= need
};

struct Task {        // 64 bytes
  int64_t out;       // ref of the output block
  int64_t cin;       // ref of the input block (OP_UPD/POTRF/TRSM_RLT/SYMUPD) or -1
  int64_t aux;       // ref of the triangular block (TRSM/TRTRI) or the mirror block (SYMUPD) or -1
  int32_t ldo, ldc, ldx;
  int16_t m, n;      // output rows / columns (<= FB)
  int32_t seg0, nseg;
  int32_t wait0, nwait;
  int32_t sig0;      // signals: sig[sig0 .. sig0+nsig)
  int16_t nsig;
  uint8_t op;
  uint8_t flags;     // TaskFlag bits
  int32_t diag;      // POTRF: index of its logdet partial sum
  int32_t zrows;     // ZERO: rows above the block in its tile column to zero (L's strict upper part)
  int32_t gcol;      // POTRF: 0-based global column of the block's first pivot
  uint8_t parts;     // 1..4 queue entries (see PartMode)
  uint8_t pmode;
  uint8_t prec;      // Precision of the block products
};
static_assert(sizeof(Task) == 80, "task layout");

}  // namespace stiles

#ifndef __CUDACC_RTC__
#include <vector>

namespace stiles {

enum PlanKind : int { PLAN_FACTOR = 0, PLAN_SELINV = 1, PLAN_FUSED = 2 };

// Tuning code of a plan (bit fields; 0 = the defaults). It changes how work is
// cut into tasks, never what is computed: bits 2-5 only re-partition output
// blocks among CTAs (bit-identical results), bits 0-1 regroup the factor's
// update terms (the same sums, rounded at other points).
//   bits 0-1  factor: source block columns per update task for tile columns
//             older than k-1 (0: 8, 1: 4, 2: 16, 3: 32)
//   bits 2-3  phase 2: parts of an off-diagonal Sigma block task
//             (0: four 32 x 32 quadrants, 1: two 32-row halves, 2: whole block)
//   bits 4-5  factor: parts of the newest update of an off-diagonal block
//             (0: four quadrants, 1: whole block)
//   bit 6     reduced-precision plans: the block updates inside a diagonal
//             tile (the SYRK / GEMM steps of that tile's POTRF) also run in
//             the reduced precision (0: they stay FP64, so that the whole
//             diagonal-tile POTRF is true FP64). This one changes rounding.
enum : int { kTuneBits = 7 };
inline int tune_chunk_old(int t) { const int v[4] = {8, 4, 16, 32}; return v[t & 3]; }
inline int tune_p2_split(int t) { return (t >> 2) & 3; }
inline int tune_upd_split(int t) { return (t >> 4) & 3; }
inline bool tune_lower_diag(int t) { return (t >> 6) & 1; }
inline bool tune_valid(int t) { return t >= 0 && t < (1 << kTuneBits) && tune_p2_split(t) <= 2 && tune_upd_split(t) <= 1; }

struct Shape {
  int nt, b, w, a;  // w already clipped to nt-1
  int prec = PREC_FP64;  // precision of the off-diagonal bulk products (Precision)
  int tune = 0;          // tuning code (see above)
  int sel0 = 0;          // selected inversion of tile columns >= sel0 only (their phase 1 and 2)
};

// Dynamic schedule: a task becomes ready when its last predecessor finishes
// (device counter rem[t], initialised to indeg[t]) and is pushed into the
// bucket of its expected start time in the list schedule; workers pop from the
// earliest non-empty bucket. Buckets hold kTasksPerBucket consecutive tasks of
// the list-schedule order.
constexpr int kTasksPerBucket = 64;
constexpr int kSlotsPerBucket = 4 * kTasksPerBucket;  // up to 4 parts per task

struct Plan {
  std::vector<Task> tasks;  // in list-schedule order
  std::vector<Seg> segs;
  std::vector<Wait> waits;  // counter form of the dependencies (host checks)
  std::vector<int32_t> sigs;
  std::vector<int32_t> indeg;     // predecessors per task
  std::vector<int32_t> succ_off;  // successors: succ[succ_off[t] .. succ_off[t+1])
  std::vector<int32_t> succ;
  std::vector<int32_t> slots0;    // initial bucket slots: ready tasks at the front, -1 elsewhere
  std::vector<int32_t> tail0;     // initial ready parts per bucket
  std::vector<int32_t> bcap;      // parts per bucket (a bucket is finished when all were popped)
  std::vector<int32_t> uslots0;   // initial urgent queue (ready urgent parts first, -1 elsewhere)
  int32_t urgent_parts = 0;       // capacity of the urgent queue
  int32_t urgent_tail0 = 0;
  int32_t nbuckets = 0;
  int32_t nctr = 0;         // dependency counters used
  int32_t ndiag = 0;        // logdet partial sums (one per POTRF task)
  double flops = 0;         // algorithmic flops (tile-operation convention)
  double flops_lowered = 0; // the part of them run as block products in the plan's reduced precision
  long long tile_gemms = 0; // phase-2 (tile, tile) products
  double cp_ns = 0;         // critical path of the estimated task graph
  double makespan_ns = 0;   // list-schedule makespan on `workers` workers
};

// Packed band+arrow layout (see include/stiles.h).
struct Layout {
  int nt, b, w, a;
  int64_t colstride;
  explicit Layout(const Shape& s)
      : nt(s.nt), b(s.b), w(s.w), a(s.a), colstride((int64_t)(1 + s.w) * s.b * s.b + (int64_t)s.a * s.b) {}
  int rows(int i) const { return i == nt ? a : b; }
  int last() const { return a > 0 ? nt : nt - 1; }
  int nsub(int k) const { return k >= nt ? 0 : (nt - 1 - k < w ? nt - 1 - k : w); }
  int64_t doubles() const { return (int64_t)nt * colstride + (int64_t)a * a; }
  int64_t tile(int i, int k) const {
    if (k == nt) return (int64_t)nt * colstride;
    if (i == nt) return (int64_t)k * colstride + (int64_t)(1 + w) * b * b;
    return (int64_t)k * colstride + (int64_t)(i - k) * b * b;
  }
  int nblk(int i) const { return (rows(i) + FB - 1) / FB; }
  int bdim(int i, int r) const { int m = rows(i) - r * FB; return m < FB ? m : FB; }
  int64_t blk(int i, int k, int r, int c) const { return tile(i, k) + (int64_t)r * FB + (int64_t)c * FB * rows(i); }
  void structure(int k, std::vector<int>& out) const {
    out.clear();
    if (k >= nt) return;
    for (int i = k + 1; i <= k + nsub(k); ++i) out.push_back(i);
    if (a > 0) out.push_back(nt);
  }
};

// Build the task table of one plan kind, ordered by a list schedule on
// `workers` persistent workers. Returns 0 or a negative stiles status code.
int build_plan(const Shape& s, PlanKind kind, int workers, Plan* out);

// Consistency check of a task table: every wait names an existing counter
// that enough tasks signal, and every such producer precedes the waiter in
// claim order (the condition under which claim-order execution cannot
// deadlock). Returns 0 or STILES_ERR_PLAN.
int check_plan(const Plan& p);

// Host emulation of a launch of the plan (bounds of every access, queue
// capacities, every task released once). Returns 0 or STILES_ERR_PLAN.
int validate_plan(const Plan& p, const Shape& s, int kind);
// The same with an explicit buffer length (doubles in each of A, L, Sigma and
// the scratch's packed part), for batch plans.
int validate_plan_len(const Plan& p, int64_t buf_doubles, int kind);
// Host race check of a plan (see plan.cpp); plant = 1 plants a race first.
int race_check_plan(const Plan& p, int64_t buf_doubles, int plant, bool serve = false);

// Fused task table of one shape for the request server: as the fused plan,
// plus one OP_PREP task per tile column that writes the request's A (in the
// L buffer) from the shape's base values; every task that reads a block of A
// waits for the PREP of its tile column, and the PREP tasks are the only
// roots. PREP fields: out = tile column slot (BUF_L), cin = the same slot of
// the base values (BUF_A), aux = rb of the column's first row (BUF_A; ra
// follows rb at distance gcol = n), ldo = b, ldc = a, ldx = present
// sub-diagonal tiles, zrows = w, diag = first row of the column.
int build_serve_template(const Shape& s, int workers, Plan* out);

// One fused (factor + selected inversion) task table for a batch of
// independent matrices: matrix m's tiles live at offset base[m] (doubles) of
// each of the shared A, L, Sigma and scratch buffers; its tasks, counters and
// logdet slots are renumbered into one table and ordered by one list
// schedule over all of them, so the small matrices fill the GPU beside the
// critical paths of the large ones. diag_base[m] .. diag_base[m+1] are the
// logdet / pivot slots of matrix m. Returns 0 or a negative status code.
int build_batch_plan(const std::vector<Shape>& shapes, const std::vector<int64_t>& base, int workers, Plan* out,
                     std::vector<int32_t>* diag_base);

}  // namespace stiles
#endif
