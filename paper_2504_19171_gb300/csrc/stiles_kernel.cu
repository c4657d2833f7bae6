// Persistent dependency-driven FP64 kernel for tiled Cholesky and two-phase
// selected inversion on GB300 (sm_103a).
//
// Two CTAs per SM (each 4 warps) claim tasks in the planner's list-schedule order with an
// atomic counter, waits (bounded by %globaltimer) until the counters its task
// depends on reach their targets, runs the task, then signals. A task only
// waits on tasks claimed before it, by CTAs that are already running, so the
// claim order cannot deadlock whatever the number of resident CTAs. These
// counters play the role of the producer/consumer flags of Algorithm 3
// ("WaitForTile / SignalTileReady"), kept on the device.
//
// FP64 has no tensor-core path on GB300 (tcgen05 has no f64 kind), so the
// block products run on the FP64 FMA pipe: 2 DFMA per clock per SM, reached
// with 4 warps. Each task stages FB x KC panels of its operands in shared
// memory (L2-only loads, so data published by other SMs is never read from a
// stale L1 line) and accumulates a 64 x 64 block in registers (4 x 8 per
// thread).
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"
#include "stiles_device.h"

namespace stiles {

constexpr int KC = 32;         // K chunk staged in shared memory
constexpr int LDS = FB + 1;    // padded shared-memory row length (doubles)
constexpr int NTHREADS = 128;  // 4 warps: one per SM sub-partition

__device__ __forceinline__ double* resolve(const KParams& p, int64_t ref) {
  return p.buf[ref >> BUF_SHIFT] + (ref & OFF_MASK);
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int load_relaxed_flag(int* a) {
  return cuda::atomic_ref<int, cuda::thread_scope_device>(*a).load(cuda::memory_order_relaxed);
}

__device__ __forceinline__ int load_acquire_i(const int* a) {
  return cuda::atomic_ref<int, cuda::thread_scope_device>(*const_cast<int*>(a)).load(cuda::memory_order_acquire);
}

__device__ __forceinline__ void store_release_i(int* a, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_device>(*a).store(v, cuda::memory_order_release);
}

// Record a TIMEOUT (first error wins) and stop every worker.
__device__ void raise_timeout(const KParams& p, long long where) {
  if (atomicCAS(&p.st->code, 0, STILES_DEV_TIMEOUT) == 0) p.st->info = (unsigned long long)where;
  atomicExch(&p.st->abort, 1);
}

#ifdef STILES_CHECKED
// Self-checking build: record the first violation (what, task, part) and stop.
__device__ void check_fail(const KParams& p, int what, long long t, int q) {
  if (atomicCAS(&p.st->code, 0, STILES_DEV_CHECK) == 0)
    p.st->info = ((unsigned long long)(t & 0xffffffffll) << 16) | ((unsigned long long)q << 8) | (unsigned)what;
  atomicExch(&p.st->abort, 1);
}
#define STILES_CHECK(cond, what, t, q) \
  do {                                  \
    if (!(cond)) check_fail(p, what, t, q); \
  } while (0)
#else
#define STILES_CHECK(cond, what, t, q) \
  do {                                  \
  } while (0)
#endif

// Push a ready task into the bucket of its list-schedule position: one slot
// per part (value 4 t + part), so that the parts run on different CTAs.
__device__ __forceinline__ void push_task(const KParams& p, int t) {
  const int parts = p.tasks[t].parts;
  if (p.tasks[t].flags & TF_URGENT) {
    const int pos = atomicAdd(p.q.lo + 8, parts);
    STILES_CHECK(pos + parts <= p.ucap, 1, t, 0);
    for (int q = 0; q < parts; ++q) store_release_i(p.q.uslots + pos + q, 4 * t + q);
    return;
  }
  const int b = t / kTasksPerBucket;
  STILES_CHECK(b < p.nbuckets && t >= 0, 2, t, 0);
  const int pos = atomicAdd(p.q.tail + b, parts);
  STILES_CHECK(pos + parts <= p.bcap[b], 3, t, 0);
  for (int q = 0; q < parts; ++q) store_release_i(p.q.slots + (size_t)b * kSlotsPerBucket + pos + q, 4 * t + q);
  atomicAdd(p.q.gcnt + (b >> 5), parts);
}

// Lane 0 of warp 0 pops the ready task part of the earliest bucket
// (list-schedule order), after the urgent queue. Returns 4 * task + part, or
// -1 when every part has been popped, the launch was aborted, or this call
// exceeded the wait budget (TIMEOUT; every path of the loop checks it).
__device__ int pop_lane0(const KParams& p) {
  const int nb = p.nbuckets, ngroups = (nb + 31) / 32;
  const unsigned long long start = gtimer();
  for (;;) {
    if (load_relaxed_flag(&p.st->abort)) return -1;
    if (gtimer() - start > (unsigned long long)p.budget_ns) {
      raise_timeout(p, (long long)load_relaxed_flag(p.q.lo) * kTasksPerBucket);
      return -1;
    }
    int* slot = nullptr;
    // urgent queue first (critical-path tasks of the factorization)
    if (p.ucap > 0) {
      const int uh = load_relaxed_flag(p.q.lo + 16);
      if (uh < load_acquire_i(p.q.lo + 8)) {
        if (atomicCAS(p.q.lo + 16, uh, uh + 1) != uh) continue;  // taken by another worker
        STILES_CHECK(uh < p.ucap, 4, uh, 0);
        slot = p.q.uslots + uh;
      }
    }
    if (!slot) {
      const int l = load_relaxed_flag(p.q.lo);
      if (l >= nb) {
        if (load_relaxed_flag(p.q.lo + 16) >= p.ucap) return -1;  // every part popped
        __nanosleep(200);
        continue;
      }
      // move lo past finished buckets (finished is permanent: atomicMax is safe)
      int f = l;
      while (f < nb && f < l + 64 && load_relaxed_flag(p.q.head + f) >= p.bcap[f]) ++f;
      if (f > l) {
        atomicMax(p.q.lo, f);
        continue;
      }
      bool raced = false;
      for (int g = l >> 5; g < ngroups && !slot && !raced; ++g) {
        if (load_relaxed_flag(p.q.gcnt + g) <= 0) continue;
        const int b1 = min(nb, 32 * g + 32);
        for (int b = max(l, 32 * g); b < b1; ++b) {
          const int h = load_relaxed_flag(p.q.head + b);
          if (h >= load_acquire_i(p.q.tail + b)) continue;
          if (atomicCAS(p.q.head + b, h, h + 1) != h) {
            raced = true;  // another worker took it: rescan from lo
            break;
          }
          atomicSub(p.q.gcnt + g, 1);
          STILES_CHECK(h < p.bcap[b], 5, b, 0);
          slot = p.q.slots + (size_t)b * kSlotsPerBucket + h;
          break;
        }
      }
      if (!slot) {
        if (!raced) __nanosleep(200);
        continue;
      }
    }
    // the pusher reserved this slot before storing it: wait for the store
    int t = load_acquire_i(slot);
    while (t < 0) {
      if (load_relaxed_flag(&p.st->abort)) return -1;
      if (gtimer() - start > (unsigned long long)p.budget_ns) {
        raise_timeout(p, -1);
        return -1;
      }
      __nanosleep(32);
      t = load_acquire_i(slot);
    }
    return t;
  }
}

// Warp 0: lane 0 pops, every lane gets the result.
__device__ __forceinline__ int pop_task(const KParams& p) {
  int v = -1;
  if ((threadIdx.x & 31) == 0) v = pop_lane0(p);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Warp 0, after task t finished and its writes were fenced: release the
// successors whose last predecessor this was.
__device__ void complete_task(const KParams& p, int t) {
  const int lane = threadIdx.x & 31;
  const int s0 = p.succ_off[t], s1 = p.succ_off[t + 1];
  for (int q = s0 + lane; q < s1; q += 32) {
    const int s = p.succ[q];
    STILES_CHECK(s >= 0 && s < p.ntasks, 6, t, 0);
    const int left = cuda::atomic_ref<int, cuda::thread_scope_device>(p.q.rem[s]).fetch_sub(1, cuda::memory_order_acq_rel);
    if (left == 1) push_task(p, s);
  }
}

// Sub-tile of a task's output block computed by one part (rows r0 .. r0+rm,
// columns c0 .. c0+cn; rm or cn <= 0: nothing to do for this part).
struct Sub {
  int r0, c0, rm, cn;
};

__device__ __forceinline__ Sub sub_of(const Task& tk, int q) {
  Sub sb{0, 0, tk.m, tk.n};
  switch (tk.pmode) {
    case PM_ROWS2: sb.r0 = 32 * q; sb.rm = min(32, tk.m - sb.r0); break;
    case PM_ROWS4: sb.r0 = 16 * q; sb.rm = min(16, tk.m - sb.r0); break;
    case PM_QUAD4: sb.r0 = 32 * (q & 1); sb.c0 = 32 * (q >> 1); break;
    case PM_TRI3: sb.r0 = q == 0 ? 0 : 32; sb.c0 = q == 2 ? 32 : 0; break;
    default: break;
  }
  if (tk.pmode == PM_QUAD4 || tk.pmode == PM_TRI3) {
    sb.rm = min(32, tk.m - sb.r0);
    sb.cn = min(32, tk.n - sb.c0);
  }
  return sb;
}

// acc[i][j] += sum over the task's segments of op(A)[r0 + tx + 16 i, :] op(B)[:, c0 + ty + 8 j]
// with 128 threads as a 16 x 8 grid (tx = tid % 16, ty = tid / 16): a
// (16 TM) x (8 TN) sub-tile, staged KC columns of K at a time in shared
// memory through L2-only loads.
template <int TM, int TN>
__device__ __forceinline__ void accumulate(const KParams& p, const Task& tk, const Sub& sb, double (&acc)[TM][TN],
                                           double* As, double* Bs) {
  constexpr int RM = 16 * TM, CN = 8 * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int s = 0; s < tk.nseg; ++s) {
    const Seg g = p.segs[tk.seg0 + s];
    const bool ta = g.trans & 1, tb = g.trans & 2;
    // op(A)[r0 + i, k] and op(B)[k, c0 + j]
    const double* A = resolve(p, g.a) + (ta ? (int64_t)sb.r0 * g.lda : (int64_t)sb.r0);
    const double* B = resolve(p, g.b) + (tb ? (int64_t)sb.c0 : (int64_t)sb.c0 * g.ldb);
    for (int k0 = 0; k0 < g.k; k0 += KC) {
      const int kc = min(KC, g.k - k0);
#pragma unroll 4
      for (int e = tid; e < RM * KC; e += NTHREADS) {
        int i, kk;
        if (!ta) { i = e % RM; kk = e / RM; } else { kk = e % KC; i = e / KC; }
        double v = 0.0;
        if (i < sb.rm && kk < kc)
          v = __ldcg(ta ? A + (int64_t)(k0 + kk) + (int64_t)i * g.lda : A + (int64_t)i + (int64_t)(k0 + kk) * g.lda);
        As[kk * LDS + i] = v;
      }
#pragma unroll 4
      for (int e = tid; e < CN * KC; e += NTHREADS) {
        int j, kk;
        if (tb) { j = e % CN; kk = e / CN; } else { kk = e % KC; j = e / KC; }
        double v = 0.0;
        if (j < sb.cn && kk < kc)
          v = __ldcg(tb ? B + (int64_t)j + (int64_t)(k0 + kk) * g.ldb : B + (int64_t)(k0 + kk) + (int64_t)j * g.ldb);
        Bs[kk * LDS + j] = v;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        double a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk * LDS + tx + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk * LDS + ty + 8 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
}

// X[rl][cl] = sign * acc (or cin - acc) over the whole (16 TM) x (8 TN) sub-tile
// (rows / columns beyond the sub-tile get -acc = 0 or are ignored later).
template <int TM, int TN>
__device__ __forceinline__ void acc_to_smem(const KParams& p, const Task& tk, const Sub& sb, const double (&acc)[TM][TN],
                                            double* X, bool sub_cin, double sign) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double* C = sub_cin ? resolve(p, tk.cin) + sb.r0 + (int64_t)sb.c0 * tk.ldc : nullptr;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int r = tx + 16 * i, c = ty + 8 * j;
      double v = sign * acc[i][j];
      if (sub_cin && r < sb.rm && c < sb.cn) v = __ldcg(C + r + (int64_t)c * tk.ldc) - acc[i][j];
      X[r * LDS + c] = v;
    }
}

__device__ __forceinline__ void load_tri(const KParams& p, const Task& tk, int dim, double* T) {
  const double* S = resolve(p, tk.aux);
  for (int e = threadIdx.x; e < dim * dim; e += NTHREADS) {
    const int r = e % dim, c = e / dim;
    T[r * LDS + c] = (r >= c) ? __ldcg(S + r + (int64_t)c * tk.ldx) : 0.0;
  }
}

// out[r0 + r][c0 + c] = X[r][c] for the sub-tile (zero above the diagonal if lower_only)
__device__ __forceinline__ void store_sub(const KParams& p, const Task& tk, const Sub& sb, const double* X,
                                          bool lower_only) {
  double* O = resolve(p, tk.out) + sb.r0 + (int64_t)sb.c0 * tk.ldo;
  for (int e = threadIdx.x; e < sb.rm * sb.cn; e += NTHREADS) {
    const int r = e % sb.rm, c = e / sb.rm;
    O[r + (int64_t)c * tk.ldo] = (lower_only && r + sb.r0 < c + sb.c0) ? 0.0 : X[r * LDS + c];
  }
}

// ---- triangular sweeps on blocks in shared memory (row length LDS) -------
// FP64 runs at 1/64 of the FP32 rate on GB300, so these avoid block-wide
// barriers in their inner loops: independent rows (or columns) are owned by
// one warp and stepped with __syncwarp only.

// X (m x n) <- X T^{-T}, T lower n x n, rcp[j*LDS] = 1 / T[j][j].
// Rows are independent: warp w owns rows RPW w .. RPW w + RPW - 1 (RPW = 16,
// 8 when m <= 32, 4 when m <= 16), its lanes split the columns of each step.
__device__ __forceinline__ void trsm_rows_lt(double* X, const double* T, const double* rcp, int m, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpw = m > 32 ? 16 : m > 16 ? 8 : 4, phases = 32 / rpw;
  const int r = warp * rpw + lane % rpw, ph = lane / rpw;
  const bool own = r < m;
  for (int j = 0; j < n; ++j) {
    if (own && ph == 0) X[r * LDS + j] *= rcp[j * LDS];
    __syncwarp();
    if (own) {
      const double xj = X[r * LDS + j];
      for (int c = j + 1 + ph; c < n; c += phases) X[r * LDS + c] -= xj * T[c * LDS + j];
    }
    __syncwarp();
  }
}

// X (m x n) <- T^{-1} X, T lower m x m, rcp[j*LDS] = 1 / T[j][j]. Columns are
// independent; warp w owns columns 4q + w (interleaved, so that the
// triangular work of an inverse is balanced). `lower` skips the columns c > j
// that stay zero when X starts as the identity.
__device__ __forceinline__ void trsm_cols_ln(double* X, const double* T, const double* rcp, int m, int n, bool lower) {
  const int lane = threadIdx.x & 31, c = 4 * (lane & 15) + (threadIdx.x >> 5), half = lane >> 4;
  const bool own = c < n;
  for (int j = 0; j < m; ++j) {
    const bool act = own && (!lower || c <= j);
    if (act && half == 0) X[j * LDS + c] *= rcp[j * LDS];
    __syncwarp();
    if (act) {
      const double xj = X[j * LDS + c];
      for (int r = j + 1 + half; r < m; r += 2) X[r * LDS + c] -= T[r * LDS + j] * xj;
    }
    __syncwarp();
  }
}

// In-place lower Cholesky of the n x n block X (n <= FB), right-looking in
// panels of 16 columns: warp 0 factors the 16 x 16 diagonal part, all threads
// solve the panel below it (a column sweep: rows in parallel) and update the
// trailing lower triangle. A pivot d gives r = rsqrt(d) (one dependent FP64
// chain instead of sqrt then a divide; dependent FP64 operations cost about
// 64 cycles each on GB300), L_jj = d r and the column is scaled by r.
// `rcp` is a scratch column of at least FB doubles (stride LDS). Returns the
// first column (0-based) whose pivot was not positive, or -1.
__device__ int potrf_smem(double* X, int n, double* rcp) {
  const int tid = threadIdx.x, lane = tid & 31;
  __shared__ int s_bad;
  if (tid == 0) s_bad = -1;
  for (int p0 = 0; p0 < n; p0 += 16) {
    const int pw = min(16, n - p0);
    if (tid < 32) {
      for (int j = 0; j < pw; ++j) {
        const int cj = p0 + j;
        const double d = X[cj * LDS + cj];
        const double rl = rsqrt(d);
        __syncwarp();
        if (lane == 0) {
          if (!(d > 0.0) && s_bad < 0) s_bad = cj;
          X[cj * LDS + cj] = d * rl;
          rcp[cj * LDS] = rl;
        }
        if (lane > j && lane < pw) X[(p0 + lane) * LDS + cj] *= rl;
        __syncwarp();
        const int w = pw - j - 1;
        for (int e = lane; e < w * w; e += 32) {
          const int r = j + 1 + e % w, c = j + 1 + e / w;
          if (c <= r) X[(p0 + r) * LDS + p0 + c] -= X[(p0 + r) * LDS + cj] * X[(p0 + c) * LDS + cj];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // rows below the panel: X[r][p0:p0+pw] <- X[r][p0:p0+pw] D^{-T} (rows in parallel)
    const int t0 = p0 + pw, w = n - t0;
    for (int j = 0; j < pw; ++j) {
      for (int r = t0 + tid; r < n; r += NTHREADS) X[r * LDS + p0 + j] *= rcp[(p0 + j) * LDS];
      __syncthreads();
      for (int e = tid; e < w * (pw - j - 1); e += NTHREADS) {
        const int r = t0 + e % w, c = p0 + j + 1 + e / w;
        X[r * LDS + c] -= X[r * LDS + p0 + j] * X[c * LDS + p0 + j];
      }
      __syncthreads();
    }
    // trailing lower triangle: X[r][c] -= sum_k X[r][p0+k] X[c][p0+k]
    for (int e = tid; e < w * w; e += NTHREADS) {
      const int r = t0 + e % w, c = t0 + e / w;
      if (c <= r) {
        double sacc = 0.0;
        for (int k = 0; k < pw; ++k) sacc = fma(X[r * LDS + p0 + k], X[c * LDS + p0 + k], sacc);
        X[r * LDS + c] -= sacc;
      }
    }
    __syncthreads();
  }
  return s_bad;
}

template <int TM, int TN>
__device__ void run_sub(const KParams& p, const Task& tk, const Sub& sb, double* smem) {
  double* As = smem;             // KC x LDS
  double* Bs = smem + KC * LDS;  // KC x LDS
  double* T = smem;              // FB x LDS, reuses As/Bs after the K-loop
  double* X = smem + 2 * KC * LDS;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m = tk.m, n = tk.n;
  double acc[TM][TN];
  if (tk.op != OP_TRTRI) accumulate<TM, TN>(p, tk, sb, acc, As, Bs);

  switch (tk.op) {
    case OP_UPD:
    case OP_STORE:
    case OP_NEG: {
      double* O = resolve(p, tk.out) + sb.r0 + (int64_t)sb.c0 * tk.ldo;
      const double* C = tk.op == OP_UPD ? resolve(p, tk.cin) + sb.r0 + (int64_t)sb.c0 * tk.ldc : nullptr;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int r = tx + 16 * i, c = ty + 8 * j;
          if (r < sb.rm && c < sb.cn) {
            double v = acc[i][j];
            if (tk.op == OP_UPD) v = __ldcg(C + r + (int64_t)c * tk.ldc) - v;
            else if (tk.op == OP_NEG) v = -v;
            O[r + (int64_t)c * tk.ldo] = v;
          }
        }
      break;
    }
    case OP_SYMUPD: {
      acc_to_smem<TM, TN>(p, tk, sb, acc, X, true, 1.0);
      __syncthreads();
      double* O = resolve(p, tk.out);
      if ((tk.flags & TF_SYM_DIAG) && sb.r0 == sb.c0) {  // diagonal sub-block: keep its lower triangle, mirror it
        double* D = O + sb.r0 + (int64_t)sb.c0 * tk.ldo;
        for (int e = tid; e < sb.rm * sb.cn; e += NTHREADS) {
          const int r = e % sb.rm, c = e / sb.rm;
          D[r + (int64_t)c * tk.ldo] = r >= c ? X[r * LDS + c] : X[c * LDS + r];
        }
      } else {
        // this sub-block, and its transpose into the mirror position: inside the
        // same block for a diagonal block, else the mirror block (aux)
        double* D = O + sb.r0 + (int64_t)sb.c0 * tk.ldo;
        const bool dblk = tk.flags & TF_SYM_DIAG;
        double* M = dblk ? O + sb.c0 + (int64_t)sb.r0 * tk.ldo : resolve(p, tk.aux) + sb.c0 + (int64_t)sb.r0 * tk.ldx;
        const int ldm = dblk ? tk.ldo : tk.ldx;
        for (int e = tid; e < sb.rm * sb.cn; e += NTHREADS) {
          const int r = e % sb.rm, c = e / sb.rm;
          D[r + (int64_t)c * tk.ldo] = X[r * LDS + c];
        }
        for (int e = tid; e < sb.rm * sb.cn; e += NTHREADS) {
          const int c = e % sb.cn, r = e / sb.cn;
          M[c + (int64_t)r * ldm] = X[r * LDS + c];
        }
      }
      break;
    }
    case OP_TRSM_RLT: {  // X = (C - acc) T^{-T}, T lower n x n: rows are independent
      acc_to_smem<TM, TN>(p, tk, sb, acc, X, true, 1.0);
      load_tri(p, tk, n, T);
      __syncthreads();
      double* rcp = T + FB;  // column FB of T's padded rows is free: rcp[j * LDS]
      if (tid < n) rcp[tid * LDS] = 1.0 / T[tid * LDS + tid];
      __syncthreads();
      trsm_rows_lt(X, T, rcp, sb.rm, n);
      __syncthreads();
      store_sub(p, tk, sb, X, false);
      break;
    }
    default:
      if constexpr (TM == 4 && TN == 8) {
        switch (tk.op) {
          case OP_POTRF: {
            acc_to_smem<TM, TN>(p, tk, sb, acc, X, true, 1.0);
            __syncthreads();
            const int bad = potrf_smem(X, n, T);
            store_sub(p, tk, sb, X, true);
            if (tk.zrows > 0) {  // strict upper part of L's diagonal tile in this block column
              double* Z = resolve(p, tk.out) - tk.zrows;
              for (int e = tid; e < tk.zrows * n; e += NTHREADS)
                Z[e % tk.zrows + (int64_t)(e / tk.zrows) * tk.ldo] = 0.0;
            }
            // log of the pivots, summed in a fixed tree order
            double lg = tid < n ? log(X[tid * LDS + tid]) : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lg += __shfl_down_sync(0xffffffffu, lg, o);
            __shared__ double s_lg[NTHREADS / 32];
            if ((tid & 31) == 0) s_lg[tid >> 5] = lg;
            __syncthreads();
            if (tid == 0) {
              p.logdet_part[tk.diag] = (s_lg[0] + s_lg[1]) + (s_lg[2] + s_lg[3]);
              if (bad >= 0) {
                atomicCAS(&p.st->code, 0, STILES_DEV_NOT_SPD);
                atomicMin(&p.st->spd_col, (unsigned long long)tk.gcol + (unsigned long long)bad);
              }
            }
            break;
          }
          case OP_TRSM_LLN: {  // X = -T^{-1} acc, T lower m x m: columns are independent
            acc_to_smem<TM, TN>(p, tk, sb, acc, X, false, -1.0);
            load_tri(p, tk, m, T);
            __syncthreads();
            double* rcp = T + FB;
            if (tid < m) rcp[tid * LDS] = 1.0 / T[tid * LDS + tid];
            __syncthreads();
            trsm_cols_ln(X, T, rcp, m, n, false);
            __syncthreads();
            store_sub(p, tk, sb, X, false);
            break;
          }
          case OP_TRTRI: {  // X = T^{-1}, T lower m x m: solve T X = I column by column
            load_tri(p, tk, m, T);
            for (int e = tid; e < FB * FB; e += NTHREADS) {
              const int r = e % FB, c = e / FB;
              X[r * LDS + c] = r == c ? 1.0 : 0.0;
            }
            __syncthreads();
            double* rcp = T + FB;
            if (tid < m) rcp[tid * LDS] = 1.0 / T[tid * LDS + tid];
            __syncthreads();
            trsm_cols_ln(X, T, rcp, m, m, true);
            __syncthreads();
            store_sub(p, tk, sb, X, true);
            break;
          }
          default:
            break;
        }
      }
      break;
  }
}

// Run part q of task tk (the planner only splits operations whose parts are
// independent: products, the row-wise TRSM and the mirrored Sigma_ii store).
#ifdef STILES_CHECKED
// [ref + lo, ref + hi] inside its buffer
__device__ bool ref_ok(const KParams& p, int64_t ref, int64_t lo, int64_t hi) {
  if (ref < 0) return false;
  const int buf = (int)(ref >> BUF_SHIFT);
  const int64_t off = ref & OFF_MASK;
  return buf >= 0 && buf < 4 && p.buf[buf] != nullptr && off + lo >= 0 && off + hi < p.buf_len;
}

__device__ bool task_part_ok(const KParams& p, const Task& tk, const Sub& sb) {
  const int r0 = sb.r0, c0 = sb.c0, r1 = sb.r0 + sb.rm - 1, c1 = sb.c0 + sb.cn - 1;
  if (tk.m < 1 || tk.n < 1 || tk.m > FB || tk.n > FB || tk.op > OP_SYMUPD) return false;
  for (int s = 0; s < tk.nseg; ++s) {
    const Seg g = p.segs[tk.seg0 + s];
    const int64_t amax = (g.trans & 1) ? (g.k - 1) + (int64_t)r1 * g.lda : r1 + (int64_t)(g.k - 1) * g.lda;
    const int64_t amin = (g.trans & 1) ? (int64_t)r0 * g.lda : r0;
    const int64_t bmax = (g.trans & 2) ? c1 + (int64_t)(g.k - 1) * g.ldb : (g.k - 1) + (int64_t)c1 * g.ldb;
    const int64_t bmin = (g.trans & 2) ? c0 : (int64_t)c0 * g.ldb;
    if (g.k < 1 || !ref_ok(p, g.a, amin, amax) || !ref_ok(p, g.b, bmin, bmax)) return false;
  }
  if (!ref_ok(p, tk.out, r0 + (int64_t)c0 * tk.ldo, r1 + (int64_t)c1 * tk.ldo)) return false;
  const bool cin = tk.op == OP_UPD || tk.op == OP_POTRF || tk.op == OP_TRSM_RLT || tk.op == OP_SYMUPD;
  if (cin && !ref_ok(p, tk.cin, r0 + (int64_t)c0 * tk.ldc, r1 + (int64_t)c1 * tk.ldc)) return false;
  if (tk.op == OP_TRSM_RLT && !ref_ok(p, tk.aux, 0, (tk.n - 1) + (int64_t)(tk.n - 1) * tk.ldx)) return false;
  if ((tk.op == OP_TRSM_LLN || tk.op == OP_TRTRI) && !ref_ok(p, tk.aux, 0, (tk.m - 1) + (int64_t)(tk.m - 1) * tk.ldx))
    return false;
  if (tk.op == OP_SYMUPD && !(tk.flags & TF_SYM_DIAG) && !ref_ok(p, tk.aux, c0 + (int64_t)r0 * tk.ldx, c1 + (int64_t)r1 * tk.ldx))
    return false;
  if (tk.op == OP_POTRF && tk.zrows > 0 && !ref_ok(p, tk.out, -(int64_t)tk.zrows, (int64_t)(tk.n - 1) * tk.ldo))
    return false;
  return true;
}
#endif

__device__ void run_task(const KParams& p, const Task& tk, int t, int q, double* smem) {
  const Sub sb = sub_of(tk, q);
  if (sb.rm <= 0 || sb.cn <= 0) return;
#ifdef STILES_CHECKED
  if (!task_part_ok(p, tk, sb)) {
    if (threadIdx.x == 0) check_fail(p, 7, t, q);
    return;
  }
#endif
  switch (tk.pmode) {
    case PM_ROWS2: run_sub<2, 8>(p, tk, sb, smem); break;
    case PM_ROWS4: run_sub<1, 8>(p, tk, sb, smem); break;
    case PM_QUAD4:
    case PM_TRI3: run_sub<2, 4>(p, tk, sb, smem); break;
    default: run_sub<4, 8>(p, tk, sb, smem); break;
  }
}

__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

__global__ void __launch_bounds__(NTHREADS, 2) persistent_kernel(KParams p) {
  extern __shared__ double smem[];
  __shared__ int s_item, s_last;
  for (;;) {
    unsigned long long t_claim = 0;
    if (threadIdx.x < 32) {
      if (p.trace && threadIdx.x == 0) t_claim = gtimer();
      const int v = pop_task(p);
      if (threadIdx.x == 0) s_item = v;
    }
    __syncthreads();
    const int v = s_item;
    if (v < 0) break;
    const int t = v >> 2, q = v & 3;
#ifdef STILES_CHECKED
    if (t >= p.ntasks || q >= p.tasks[t].parts) {
      if (threadIdx.x == 0) check_fail(p, 8, t, q);
      break;
    }
#endif
    unsigned long long t_ready = 0;
    if (p.trace && threadIdx.x == 0) t_ready = gtimer();
    __threadfence();
    const Task tk = p.tasks[t];
    run_task(p, tk, t, q, smem);
    __threadfence();
    __syncthreads();
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) {
        s_last = tk.parts <= 1 ||
                 cuda::atomic_ref<int, cuda::thread_scope_device>(p.q.pdone[t]).fetch_add(1, cuda::memory_order_acq_rel) ==
                     tk.parts - 1;
      }
      __syncwarp();
      if (s_last) {
        complete_task(p, t);
        if (threadIdx.x == 0) {
          atomicAdd(&p.st->done, 1ull);
          if (p.trace) {
            unsigned long long* tr = p.trace + 4 * (size_t)t;
            tr[0] = t_claim;
            tr[1] = t_ready;
            tr[2] = gtimer();
            tr[3] = ((unsigned long long)smid() << 32) | ((unsigned long long)blockIdx.x << 8) | tk.op;
          }
        }
      }
    }
  }
}

size_t kernel_smem_bytes() { return sizeof(double) * (size_t)(2 * KC * LDS + FB * LDS); }

cudaError_t launch_persistent(const KParams& p, int grid, cudaStream_t stream) {
  static bool configured = false;
  const size_t smem = kernel_smem_bytes();
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  persistent_kernel<<<grid, NTHREADS, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace stiles
