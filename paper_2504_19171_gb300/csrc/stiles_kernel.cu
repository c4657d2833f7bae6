// Persistent dependency-driven kernel for tiled Cholesky and two-phase
// selected inversion on GB300 (sm_103a).
//
// Two CTAs per SM (each 4 warps) run task parts until every part of the plan
// has been executed. A task becomes ready when its last predecessor finishes
// (per-task predecessor counters, decremented by the finishing task: the
// device form of Algorithm 3's "WaitForTile / SignalTileReady" flags); the
// finisher pushes its parts into a queue, and idle workers claim parts with
// fetch-and-add on availability counters. Static plans queue parts in
// buckets of the host's list-schedule order behind an urgent FIFO for the
// factorization's frontier; the request server (serve mode) uses three FIFO
// rings and activates new requests from a host-mapped inbox while it runs.
// Every wait is bounded by %globaltimer and ends the launch with a TIMEOUT
// status instead of hanging.
//
// FP64 has no tensor-core path on GB300 (tcgen05 has no f64 kind), so the
// FP64 block products run on the FP64 FMA pipe: 2 DFMA per clock per SM,
// reached with 4 warps. Each task stages FB x KC panels of its operands in
// shared memory (L2-only loads, so data published by other SMs is never read
// from a stale L1 line) and accumulates up to a 64 x 64 block in registers
// (4 x 8 per thread). The reduced-precision modes replace the products of
// the bulk tasks by split-precision digit products on the tensor cores
// (tcgen05 MMAs from shared memory into tensor memory): 8 digits per operand
// for emulated FP64, 4 for the FP32-class mode. In the end-to-end call the matrix may live in
// page-locked host memory (read over the host link by the tasks that first
// load each block) and every final Sigma write is repeated into a host
// buffer, so the transfers overlap the computation.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "plan.h"
#include "stiles_device.h"
#include "tcgen05.cuh"

namespace stiles {

constexpr int KC = 32;         // K chunk staged in shared memory
constexpr int LDS = FB + 1;    // padded shared-memory row length (doubles)
constexpr int NTHREADS = 128;  // 4 warps: one per SM sub-partition

__device__ __forceinline__ double* resolve(const KParams& p, int64_t ref) {
  return p.buf[ref >> BUF_SHIFT] + (ref & OFF_MASK);
}

// Task-table reads. A request server rewrites table ranges (copy engine)
// while the kernel runs; a worker reads a task only after the acquire load of
// the queue slot that delivered it, which is ordered after the host's
// publication (system-scope release / acquire on the inbox, then release /
// acquire through the queues), so plain loads see the new rows. (Loading
// whole rows with L2-only vector loads instead costs registers the block
// products need.)
__device__ __forceinline__ Task load_task(const KParams& p, int t) { return p.tasks[t]; }

__device__ __forceinline__ Seg load_seg(const KParams& p, int g) { return p.segs[g]; }

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

// Host-mapped memory (request server control block).
__device__ __forceinline__ int load_acquire_sys(const int* a) {
  return cuda::atomic_ref<int, cuda::thread_scope_system>(*const_cast<int*>(a)).load(cuda::memory_order_acquire);
}

__device__ __forceinline__ void store_release_sys(unsigned* a, unsigned v) {
  cuda::atomic_ref<unsigned, cuda::thread_scope_system>(*a).store(v, cuda::memory_order_release);
}

// Record a TIMEOUT (first error wins) and stop every worker.
__device__ void raise_timeout(const KParams& p, long long where) {
  if (atomicCAS(&p.st->code, 0, STILES_DEV_TIMEOUT) == 0) p.st->info = (unsigned long long)where;
  atomicExch(&p.st->abort, 1);
}

// Record the first violation of a table or queue invariant (what, task,
// part) and stop every worker (STILES_DEV_CHECK, reported as a plan error).
__device__ void check_fail(const KParams& p, int what, long long t, int q) {
  if (atomicCAS(&p.st->code, 0, STILES_DEV_CHECK) == 0)
    p.st->info = ((unsigned long long)(t & 0xffffffffll) << 16) | ((unsigned long long)q << 8) | (unsigned)what;
  atomicExch(&p.st->abort, 1);
}

#ifdef STILES_CHECKED
// Self-checking build: every invariant below is checked.
#define STILES_CHECK(cond, what, t, q) \
  do {                                  \
    if (!(cond)) check_fail(p, what, t, q); \
  } while (0)
#else
#define STILES_CHECK(cond, what, t, q) \
  do {                                  \
  } while (0)
#endif

// Push a ready task into the bucket of its queue position: one slot per part
// (value 4 t + part), so that the parts run on different CTAs. The slots are
// reserved (tail), stored, and only then counted as available.
__device__ void serve_push(const KParams& p, int t);

__device__ __forceinline__ void push_task(const KParams& p, int t) {
  if (p.serve) {
    serve_push(p, t);
    return;
  }
  const Task tk = load_task(p, t);
  const int parts = tk.parts;
  // The queue capacities are checked in every build (one compare on an
  // atomic path): a table that would overflow a queue stops the launch with
  // a check failure instead of writing past the slots.
  if (tk.flags & TF_URGENT) {
    const int pos = atomicAdd(p.q.lo + 8, parts);
    if (pos + parts > p.ucap) {
      check_fail(p, 1, t, 0);
      return;
    }
    for (int q = 0; q < parts; ++q) store_release_i(p.q.uslots + pos + q, 4 * t + q);
    atomicAdd(p.q.lo + 24, parts);
    return;
  }
  const int b = t / kTasksPerBucket;
  if (b >= p.nbuckets || t < 0) {
    check_fail(p, 2, t, 0);
    return;
  }
  const int pos = atomicAdd(p.q.tail + b, parts);
  if (pos + parts > p.bcap[b]) {
    check_fail(p, 3, t, 0);
    return;
  }
  for (int q = 0; q < parts; ++q) store_release_i(p.q.slots + (size_t)b * kSlotsPerBucket + pos + q, 4 * t + q);
  atomicAdd(p.q.avail + b, parts);
  atomicAdd(p.q.gcnt + (b >> 5), parts);
  atomicAdd(p.q.scnt + (b >> 10), parts);
}

// Lane 0: wait for the store of a claimed queue slot (its pusher reserved it
// before counting it available, and stores it right after). Returns the
// item, or -1 on abort / budget expiry.
__device__ int wait_slot(const KParams& p, int* slot, unsigned long long start) {
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

// Lane 0: claim one available part of a queue (avail / head pair) without a
// compare-and-swap retry loop: many idle workers contending for the same
// bucket each cost two fetch-and-adds, not a round trip per lost race.
// Returns the claimed slot index, or -1 if nothing was available.
__device__ __forceinline__ int claim(int* avail, int* head) {
  if (load_relaxed_flag(avail) <= 0) return -1;
  if (atomicSub(avail, 1) <= 0) {
    atomicAdd(avail, 1);
    return -1;
  }
  return atomicAdd(head, 1);
}

// ---- request server: three FIFO rings (urgent, other factor tasks, rest) ---
// Ring entries are reserved (tail), stored, then counted available, like the
// buckets; a popped entry is reset to -1 so the ring can wrap (its capacity
// exceeds the parts that can be ready at once).
__device__ void serve_push(const KParams& p, int t) {
  const Task tk = load_task(p, t);
  const int parts = tk.parts;
  const bool factor = tk.op == OP_UPD || tk.op == OP_POTRF || tk.op == OP_TRSM_RLT || tk.op == OP_PREP;
  const ServeRing& R = p.sv.ring[(tk.flags & TF_URGENT) ? 0 : factor ? 1 : 2];
  const unsigned pos = (unsigned)atomicAdd(R.ctr, parts);
  for (int q = 0; q < parts; ++q) {
    int* slot = R.slots + ((pos + q) & R.mask);
    const unsigned long long start = gtimer();
    while (load_acquire_i(slot) != -1) {  // the previous lap's entry not yet taken: bounded wait
      if (load_relaxed_flag(&p.st->abort)) return;
      if (gtimer() - start > (unsigned long long)p.budget_ns) {
        raise_timeout(p, t);
        return;
      }
      __nanosleep(64);
    }
    store_release_i(slot, 4 * t + q);
  }
  atomicAdd(R.ctr + 16, parts);
}

// Lane 0 of an idle worker: a ready part of the highest non-empty ring
// (>= 0), a new request to activate (-4 - record index), -1 to stop, or -3.
__device__ int serve_try_lane0(const KParams& p, unsigned long long deadline) {
  if (load_relaxed_flag(&p.st->abort)) return -1;
  for (int r = 0; r < 3; ++r) {
    const ServeRing& R = p.sv.ring[r];
    const int h = claim(R.ctr + 16, R.ctr + 8);
    if (h >= 0) {
      int* slot = R.slots + ((unsigned)h & R.mask);
      const int v = wait_slot(p, slot, gtimer());
      if (v >= 0) cuda::atomic_ref<int, cuda::thread_scope_device>(*slot).store(-1, cuda::memory_order_relaxed);
      return v;
    }
  }
  const int seen = load_relaxed_flag(p.sv.inbox_seen);
  if (seen < load_acquire_sys(&p.sv.ctl->inbox_count)) {
    if (atomicCAS(p.sv.inbox_seen, seen, seen + 1) == seen) return -4 - seen;
    return -3;
  }
  if (load_acquire_sys(&p.sv.ctl->stop)) return -1;
  if (gtimer() > deadline) {
    raise_timeout(p, -2);
    return -1;
  }
  return -3;
}

// Warp 0: activate inbox record `idx`: its value parameters, then its root
// tasks into the rings (lanes in parallel).
__device__ void serve_activate(const KParams& p, int idx) {
  const int lane = threadIdx.x & 31;
  const ServeRec* rec = &p.sv.ctl->inbox[idx % kServeInbox];
  int slot = 0, root0 = 0, nroots = 0;
  if (lane == 0) {
    const volatile ServeRec* vr = rec;
    slot = vr->slot;
    root0 = vr->root0;
    nroots = vr->nroots;
    p.sv.req_param[2 * slot] = vr->rho;
    p.sv.req_param[2 * slot + 1] = vr->tau;
    p.sv.req_seq[slot] = vr->seq;
    __threadfence();
  }
  root0 = __shfl_sync(0xffffffffu, root0, 0);
  nroots = __shfl_sync(0xffffffffu, nroots, 0);
  __syncwarp();
  for (int i = lane; i < nroots; i += 32) push_task(p, __ldcg(p.sv.roots + root0 + i));
}

__device__ int serve_pop(const KParams& p, unsigned long long deadline) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (;;) {
    int r = -3;
    if (lane == 0) r = serve_try_lane0(p, deadline);
    r = __shfl_sync(FULL, r, 0);
    if (r >= -1) return r;
    if (r <= -4) {
      serve_activate(p, -4 - r);
      continue;
    }
    __nanosleep(400);
  }
}

// Lane 0: abort / budget check, then one attempt on the urgent queue.
// Returns an item (>= 0), -1 to stop, or -3 when no urgent part is ready.
__device__ int pop_urgent_lane0(const KParams& p, unsigned long long start) {
  if (load_relaxed_flag(&p.st->abort)) return -1;
  if (gtimer() - start > (unsigned long long)p.budget_ns) {
    raise_timeout(p, (long long)load_relaxed_flag(p.q.lo) * kTasksPerBucket);
    return -1;
  }
  if (p.ucap <= 0) return -3;
  const int uh = claim(p.q.lo + 24, p.q.lo + 16);
  if (uh < 0) return -3;
  if (uh >= p.ucap) {  // claimed past the urgent queue (checked in every build)
    check_fail(p, 4, uh, 0);
    return -1;
  }
  return wait_slot(p, p.q.uslots + uh, start);
}

// Warp 0 pops a ready task part: the urgent queue first, then the earliest
// bucket (queue order) with an available part. Lane 0 takes every decision
// and broadcasts it, the other lanes only help to scan 32 super-groups /
// groups / buckets per load round, so the warp stays uniform. Returns
// 4 * task + part, or -1 when every part has been popped, the launch was
// aborted, or the wait budget of this call expired (TIMEOUT; checked on
// every pass of the loop).
__device__ int pop_task(const KParams& p, unsigned long long deadline) {
  if (p.serve) return serve_pop(p, deadline);
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nb = p.nbuckets, ngroups = (nb + 31) / 32, nsuper = (ngroups + 31) / 32;
  const unsigned long long start = lane == 0 ? gtimer() : 0ull;
  for (;;) {
    int r = -3;
    if (lane == 0) r = pop_urgent_lane0(p, start);
    r = __shfl_sync(FULL, r, 0);
    if (r != -3) return r;
    int l = 0;
    if (lane == 0) l = load_relaxed_flag(p.q.lo);
    l = __shfl_sync(FULL, l, 0);
    // scan from lo: super-groups of 32 groups, groups of 32 buckets, buckets
    int got = -3;  // -3: nothing found, -1: stop, >= 0: item
    const int g_lo = l >> 5;
    for (int sbase = l >> 10; sbase < nsuper && got == -3; sbase += 32) {
      const int sg = sbase + lane;
      unsigned sm = __ballot_sync(FULL, sg < nsuper && load_relaxed_flag(p.q.scnt + sg) > 0);
      while (sm && got == -3) {
        const int si = sbase + __ffs(sm) - 1;
        sm &= sm - 1;
        const int g = si * 32 + lane;
        unsigned gm = __ballot_sync(FULL, g < ngroups && g >= g_lo && load_relaxed_flag(p.q.gcnt + g) > 0);
        while (gm && got == -3) {
          const int gi = si * 32 + __ffs(gm) - 1;
          gm &= gm - 1;
          const int b = gi * 32 + lane;
          unsigned rm = __ballot_sync(FULL, b < nb && b >= l && load_relaxed_flag(p.q.avail + b) > 0);
          while (rm && got == -3) {  // try the ready buckets in order
            const int bb = gi * 32 + __ffs(rm) - 1;
            rm &= rm - 1;
            if (lane == 0) {
              const int h = claim(p.q.avail + bb, p.q.head + bb);
              if (h >= 0) {
                atomicSub(p.q.gcnt + gi, 1);
                atomicSub(p.q.scnt + (gi >> 5), 1);
                if (h >= p.bcap[bb]) {  // claimed past the bucket (checked in every build)
                  check_fail(p, 5, bb, 0);
                  got = -1;
                } else {
                  got = wait_slot(p, p.q.slots + (size_t)bb * kSlotsPerBucket + h, start);
                }
              }
            }
            got = __shfl_sync(FULL, got, 0);
          }
        }
      }
    }
    if (got != -3) return got;
    // nothing claimed: move lo past finished buckets (finished is permanent,
    // so atomicMax is safe), stop once every part was popped, else back off
    if (l >= nb) {
      int done = 0;
      if (lane == 0) done = load_relaxed_flag(p.q.lo + 16) >= p.ucap;
      if (__shfl_sync(FULL, done, 0)) return -1;
    } else {
      const int b = l + lane;
      const bool fin = b >= nb || load_relaxed_flag(p.q.head + b) >= p.bcap[b];
      const unsigned unf = __ballot_sync(FULL, !fin);
      const int nfin = unf ? __ffs(unf) - 1 : 32;
      if (nfin > 0) {
        if (lane == 0) atomicMax(p.q.lo, l + nfin);
        continue;
      }
    }
    __nanosleep(200);
  }
}

// Warp 0, after task t finished and its writes were fenced: release the
// successors whose last predecessor this was.
__device__ void complete_task(const KParams& p, int t) {
  const int lane = threadIdx.x & 31;
  const int s0 = __ldcg(p.succ_off + t), s1 = __ldcg(p.succ_off + t + 1);
  for (int q = s0 + lane; q < s1; q += 32) {
    const int s = __ldcg(p.succ + q);
    STILES_CHECK(s >= 0 && s < p.ntasks, 6, t, 0);
    const int left = cuda::atomic_ref<int, cuda::thread_scope_device>(p.q.rem[s]).fetch_sub(1, cuda::memory_order_acq_rel);
    if (left == 1) push_task(p, s);
  }
  if (p.serve) {  // request accounting: the last task of a request signals the host
    __syncwarp();
    if (lane == 0) {
      const int slot = __ldcg(p.sv.treq + t);
      if (atomicSub(p.sv.req_left + slot, 1) == 1) {
        __threadfence_system();
        store_release_sys(&p.sv.ctl->done_seq[slot], __ldcg(p.sv.req_seq + slot));
      }
    }
  }
}

// OP_PREP (request server): tile column of A from the shape's base values and
// the request's (rho, tau): band entries x rho, arrow entries unchanged,
// diagonal tau + rho rb[i] + ra[i]. Every output element is written once.
__device__ void run_prep(const KParams& p, const Task& tk, int t) {
  const int slot = __ldcg(p.sv.treq + t);
  const double rho = __ldcg(p.sv.req_param + 2 * slot), tau = __ldcg(p.sv.req_param + 2 * slot + 1);
  if (rho != rho) return;  // a request with explicit values: its A was copied into place
  double* O = resolve(p, tk.out);
  const double* B = resolve(p, tk.cin);
  const double* rb = resolve(p, tk.aux);
  const double* ra = rb + tk.gcol;
  const int b = tk.ldo, a = tk.ldc;
  if (tk.flags & TF_CORNER) {  // arrow x arrow: entries unchanged, diagonal rebuilt
    for (int e = threadIdx.x; e < a * a; e += NTHREADS) {
      const int r = e % a, c = e / a;
      O[e] = r == c ? tau + rho * rb[r] + ra[r] : __ldg(B + e);
    }
    return;
  }
  const int64_t bb = (int64_t)b * b, band = (1 + (int64_t)tk.ldx) * bb;
  for (int64_t e = threadIdx.x; e < band; e += NTHREADS) {  // diagonal tile, then the sub-diagonal tiles
    const int r = (int)(e % b);
    const bool dg = e < bb && r == (int)(e / b);
    O[e] = dg ? tau + rho * rb[r] + ra[r] : rho * __ldg(B + e);
  }
  const int64_t arrow0 = (1 + (int64_t)tk.zrows) * bb;  // the arrow tile (a x b) is copied
  for (int64_t e = threadIdx.x; e < (int64_t)a * b; e += NTHREADS) O[arrow0 + e] = __ldg(B + arrow0 + e);
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
    case PM_TILE32: {
      const int pr = tk.m > 32 ? 2 : 1;
      sb.r0 = 32 * (q % pr);
      sb.c0 = 32 * (q / pr);
      break;
    }
    case PM_ROWS8: sb.r0 = 8 * q; sb.rm = min(8, tk.m - sb.r0); break;
    case PM_TRI16: sb.r0 = q == 0 ? 0 : 16; sb.c0 = q == 2 ? 16 : 0; break;
    case PM_QUAD16: sb.r0 = 16 * (q >> 1); sb.c0 = 16 * (q & 1); break;
    default: break;
  }
  if (tk.pmode == PM_QUAD4 || tk.pmode == PM_TRI3 || tk.pmode == PM_TILE32) {
    sb.rm = min(32, tk.m - sb.r0);
    sb.cn = min(32, tk.n - sb.c0);
  } else if (tk.pmode == PM_TRI16 || tk.pmode == PM_QUAD16) {
    sb.rm = min(16, tk.m - sb.r0);
    sb.cn = min(16, tk.n - sb.c0);
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
    const Seg g = load_seg(p, tk.seg0 + s);
    const bool ta = g.trans & 1, tb = g.trans & 2;
    // op(A)[r0 + i, k] and op(B)[k, c0 + j]
    const double* A = resolve(p, g.a) + (ta ? (int64_t)sb.r0 * g.lda : (int64_t)sb.r0);
    const double* B = resolve(p, g.b) + (tb ? (int64_t)sb.c0 : (int64_t)sb.c0 * g.ldb);
    for (int k0 = 0; k0 < g.k; k0 += KC) {
      const int kc = min(KC, g.k - k0);
      // each batch of loads is in flight before its shared-memory stores
      constexpr int NA = RM * KC / NTHREADS, NB = CN * KC / NTHREADS;
      constexpr int BA = NA < 8 ? NA : 8, BB = NB < 8 ? NB : 8;
#pragma unroll
      for (int u0 = 0; u0 < NA; u0 += BA) {
        double v[BA];
#pragma unroll
        for (int u = 0; u < BA; ++u) {
          const int e = tid + (u0 + u) * NTHREADS;
          int i, kk;
          if (!ta) { i = e % RM; kk = e / RM; } else { kk = e % KC; i = e / KC; }
          v[u] = (i < sb.rm && kk < kc)
                     ? __ldcg(ta ? A + (int64_t)(k0 + kk) + (int64_t)i * g.lda : A + (int64_t)i + (int64_t)(k0 + kk) * g.lda)
                     : 0.0;
        }
#pragma unroll
        for (int u = 0; u < BA; ++u) {
          const int e = tid + (u0 + u) * NTHREADS;
          int i, kk;
          if (!ta) { i = e % RM; kk = e / RM; } else { kk = e % KC; i = e / KC; }
          As[kk * LDS + i] = v[u];
        }
      }
#pragma unroll
      for (int u0 = 0; u0 < NB; u0 += BB) {
        double v[BB];
#pragma unroll
        for (int u = 0; u < BB; ++u) {
          const int e = tid + (u0 + u) * NTHREADS;
          int j, kk;
          if (tb) { j = e % CN; kk = e / CN; } else { kk = e % KC; j = e / KC; }
          v[u] = (j < sb.cn && kk < kc)
                     ? __ldcg(tb ? B + (int64_t)j + (int64_t)(k0 + kk) * g.ldb : B + (int64_t)(k0 + kk) + (int64_t)j * g.ldb)
                     : 0.0;
        }
#pragma unroll
        for (int u = 0; u < BB; ++u) {
          const int e = tid + (u0 + u) * NTHREADS;
          int j, kk;
          if (tb) { j = e % CN; kk = e / CN; } else { kk = e % KC; j = e / KC; }
          Bs[kk * LDS + j] = v[u];
        }
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

// ---- split-precision block products on the tensor cores (tcgen05) -------
//
// Error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump. For one
// task part (at most 32 x 32 outputs) every row i of op(A) gets the biased
// exponent E_i of its largest entry over all the task's segments and every
// column j of op(B) the exponent F_j. Each entry becomes a signed fixed-point
// integer X relative to that exponent, |X| < 2^(DB S - 2) (the largest entry
// of the row keeps its 53-bit significand in the emulated-FP64 mode; the
// others are rounded to the same unit), written as S balanced base-2^DB
// digits d_t in [-2^(DB-1), 2^(DB-1)), X = sum_t d_t 2^(DB (S-1-t)), which
// bf16 holds exactly. A digit product is an integer of magnitude at most
// 2^(2 DB - 2); products of levels L = t + u <= S - 1 are kept. Emulated FP64
// uses S = 8 digits of DB = 8 bits (|X| < 2^62: entries down to 2^-9 of their
// row maximum keep all 53 bits, the dropped levels weigh below 2^-56 of the
// leading product). The FP32-class mode uses no shared exponent: every entry
// becomes its FP32 value (rounded to nearest) written as three bf16 pieces
// that keep their own exponents (piece_pairs), in the same four-plane layout
// with a zero fourth plane; its cells hold ordinary FP32 sums.
//
// Tensor-core layout. D has M = 128 rows, made from a 32-row part by
// stacking four digit planes of A: stack g (g < G = S / 4) holds plane
// g + G p in rows 32 p + i (p = 0..3). The B planes are concatenated along
// N ([B_0 | B_1 | ... | B_{S-1}], 32 columns each). Stack g is multiplied by
// the first 32 (S - g) columns of that concatenation into TMEM columns from
// 32 g on, so TMEM cell (lane block p, column block c) collects the plane
// pairs (g + G p, c - g), all of one level L = G p + c. A cell receives at
// most G pairs per K step: in the emulated-FP64 mode its FP32 sums are
// integers of magnitude at most 2^24, hence exact, for up to
// 2^24 / (G 2^14) = 512 of K.
// Before that much K has been accumulated (or at the end of the task) the
// cells of levels <= S - 1 are read -- warp p reads lane block p -- and
// combined per output: exactly in two 64-bit halves for emulated FP64, then
// scaled by 2^(E_i + F_j - bias); summed in FP32 for the FP32-class mode. The
// result is added to the part's FP64 value.
// Non-finite operands make their row or column NaN (emulated FP64: biased
// exponent 0x7ff; FP32-class: NaN pieces, also for values beyond the FP32
// range).

constexpr int TC_KS = 32;           // K per staging buffer (two MMA K steps)
constexpr uint32_t TC_COLS = 256;   // TMEM columns per CTA (two CTAs per SM share 512)
constexpr int TC_STAGE_BYTES_MAX = 2 * 32 * 8 * TC_KS * 2;  // A and B digit planes of S = 8
// shared memory of a tensor part: two staging buffers, the row / column
// exponents, then the part's FP64 result (32 x 33 doubles)
constexpr int TC_EXP_OFF = 2 * TC_STAGE_BYTES_MAX;
constexpr int TC_RES_OFF = TC_EXP_OFF + 64 * 4;
constexpr int TC_SMEM_BYTES = TC_RES_OFF + 32 * 33 * 8;

// Per-CTA state of the tensor path (static shared memory of the kernel).
struct TcShared {
  uint64_t mbar[2];      // completion barriers of the two staging buffers
  uint32_t ncommit[2];   // commits issued to each barrier so far (this launch)
  uint32_t tmem;         // TMEM base address of this CTA's TC_COLS columns
};

__device__ __forceinline__ int biased_exp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

// out[i] = max(out[i], largest biased exponent over k < K of element (i, k))
// of a panel of n <= 32 vectors: element (i, k) sits at P[i + k ld] when
// `along_i` (the vectors' index is the contiguous one), else at P[k + i ld].
// Loads follow the contiguous dimension, 16 independent ones in flight per
// thread. Ends with a block barrier.
__device__ __forceinline__ void max_exp_into(const double* P, int ld, bool along_i, int n, int K, int* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int U = 16;
  if (along_i) {  // lanes over i, warps over k (k = warp + 4 u)
    int mx = 0;
    if (lane < n)
      for (int k0 = warp; k0 < K; k0 += 4 * U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = k0 + 4 * u < K ? __ldcg(P + lane + (int64_t)(k0 + 4 * u) * ld) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) mx = max(mx, biased_exp(v[u]));
      }
    __shared__ int part[4][32];
    part[warp][lane] = mx;
    __syncthreads();
    if (warp == 0) out[lane] = max(out[lane], max(max(part[0][lane], part[1][lane]), max(part[2][lane], part[3][lane])));
  } else {  // lanes over k; warp w takes vectors w, w + 4, ..., w + 28 at once (two k per lane)
    int mx[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) mx[v] = 0;
    for (int k0 = lane; k0 < K; k0 += 64) {
      double x[8][2];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const int i = warp + 4 * v;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = k0 + 32 * h;
          x[v][h] = (i < n && k < K) ? __ldcg(P + k + (int64_t)i * ld) : 0.0;
        }
      }
#pragma unroll
      for (int v = 0; v < 8; ++v) mx[v] = max(mx[v], max(biased_exp(x[v][0]), biased_exp(x[v][1])));
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx[v] = max(mx[v], __shfl_xor_sync(0xffffffffu, mx[v], o));
      if (lane == 0) out[warp + 4 * v] = max(out[warp + 4 * v], mx[v]);
    }
  }
  __syncthreads();
}

// Signed fixed-point value of v relative to the biased exponent emax of its
// row or column (emax >= its own), rounded to nearest: the row maximum maps
// to [2^(BITS-1), 2^BITS).
template <int BITS>
__device__ __forceinline__ long long fixed_point(double v, int emax) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7ff);
  const long long m = (long long)((bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull));
  const int sh = max(emax, 1) - max(e, 1) + 53 - BITS;  // >= 53 - BITS
  long long X;
  if (sh < 0) X = m << -sh;
  else if (sh == 0) X = m;
  else if (sh < 63) X = (m + (1ll << (sh - 1))) >> sh;
  else X = 0;
  return (bits >> 63) ? -X : X;
}

// C = sum_{t < S} 2^(DB-1) 2^(DB t): X + C has base-2^DB digits d_t + 2^(DB-1).
template <int S, int DB>
__host__ __device__ constexpr unsigned long long digit_bias() {
  unsigned long long c = 0;
  for (int t = 0; t < S; ++t) c |= 1ull << (DB * t + DB - 1);
  return c;
}

// The S digits (DB bits each, balanced) of a pair of K-adjacent values (v0
// at k, v1 at k + 1) as packed bf16 pairs: w[t] = bf16(d_t(v0)) | bf16(d_t(v1)) << 16.
template <int S, int DB>
__device__ __forceinline__ void digit_pairs(double v0, double v1, int emax, uint32_t (&w)[S]) {
  constexpr int BITS = DB * S - 2;
  constexpr unsigned long long C = digit_bias<S, DB>();
  constexpr float kMagic = 8388608.0f + (float)(1 << (DB - 1));  // 2^23 + 2^(DB-1)
  // in unsigned arithmetic: with DB S = 64 the bias C is above 2^63
  const unsigned long long y0 = (unsigned long long)fixed_point<BITS>(v0, emax) + C;
  const unsigned long long y1 = (unsigned long long)fixed_point<BITS>(v1, emax) + C;
  static_assert(DB == 8 && S <= 8, "byte digits of a 64-bit value");
  // digit t is byte S - 1 - t of y: one byte permute puts it under the
  // exponent of 2^23 (bytes 0x00, 0x00, 0x4B above it); the float minus
  // 2^23 + 2^(DB-1) is the digit exactly, and its bf16 is its upper half
  const uint32_t h0[2] = {(uint32_t)y0, (uint32_t)(y0 >> 32)}, h1[2] = {(uint32_t)y1, (uint32_t)(y1 >> 32)};
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const int bi = S - 1 - t;
    const uint32_t sel = 0x7540u | (uint32_t)(bi & 3);
    const float f0 = __uint_as_float(__byte_perm(h0[bi >> 2], 0x4B000000u, sel)) - kMagic;
    const float f1 = __uint_as_float(__byte_perm(h1[bi >> 2], 0x4B000000u, sel)) - kMagic;
    w[t] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
  }
}

// FP32-class operands: the value rounded to nearest FP32 (ties away from
// zero), built from the double's bits without an FP64 instruction: half a
// unit of the 23rd fraction bit is added to the bit pattern (a carry moves
// into the exponent as it should), then sign, exponent rebiased and the top
// 23 fraction bits are taken. Below the FP32 normal range it is zero, above
// it infinity; an infinity or NaN in gives NaN.
__device__ __forceinline__ uint32_t fp32_bits_of(double v) {
  const unsigned long long b0 = (unsigned long long)__double_as_longlong(v);
  if (((b0 >> 52) & 0x7ff) == 0x7ff) return 0x7fc00000u;
  const unsigned long long b = b0 + (1ull << 28);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const int e = (int)((hi >> 20) & 0x7ff);
  const uint32_t sgn = hi & 0x80000000u;
  if (e < 1023 - 126) return sgn;
  if (e > 1023 + 127) return sgn | 0x7f800000u;
  return sgn | ((uint32_t)(e - 1023 + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
}

// The FP32 values of a pair of K-adjacent operands (v0 at k, v1 at k + 1) as
// three bf16 pieces each, packed in pairs like digit_pairs: piece t is the
// value left after pieces < t, truncated to its top 8 significant bits, so
// the three pieces sum to the FP32 value exactly and each keeps its own
// exponent. The fourth plane is zero.
__device__ __forceinline__ void piece_pairs(double v0, double v1, uint32_t (&w)[4]) {
  float r0 = __uint_as_float(fp32_bits_of(v0)), r1 = __uint_as_float(fp32_bits_of(v1));
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t p0 = __float_as_uint(r0) & 0xffff0000u, p1 = __float_as_uint(r1) & 0xffff0000u;
    w[t] = (p0 >> 16) | p1;
    r0 -= __uint_as_float(p0);
    r1 -= __uint_as_float(p1);
  }
  w[3] = 0u;
}

// Byte offset of element (row, k) (k even: a packed pair) in a staging
// operand of canonical K-major core matrices: 8 rows x 8 K per 128 bytes,
// TC_KS / 8 core matrices along K per 8-row group.
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
  return (uint32_t)((((row >> 3) * (TC_KS / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}
constexpr uint32_t TC_LBO = 128;                 // K-adjacent core matrices
constexpr uint32_t TC_SBO = (TC_KS / 8) * 128;   // 8-row groups

// Panel element owned by slot q (0..3) of this thread, for a stage of 32
// vectors x TC_KS: vector index `vi` and the even K offset `kk` of its pair.
// Warp w takes the 8-vector group w, slot q the K core matrix q, and lane
// (r, kp) = (lane % 8, lane / 8) the vector 8 w + r and K pair kp of it: the
// warp's 32 packed-pair stores then fill the 32 words of one core matrix
// (no shared-memory bank conflict), and its loads read 8 x 64 contiguous
// bytes whichever dimension of the operand is the contiguous one.
__device__ __forceinline__ void tc_slot(int q, int& vi, int& kk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  vi = 8 * warp + (lane & 7);
  kk = 8 * q + 2 * (lane >> 3);
}

// Bounded wait for phase `parity` of a staging barrier (all threads).
__device__ bool tc_wait(const KParams& p, uint32_t mbar, uint32_t parity) {
  if (tc::mbar_test(mbar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!tc::mbar_test(mbar, parity)) {
    if (gtimer() - t0 > (unsigned long long)p.budget_ns) {
      raise_timeout(p, -3);
      return false;
    }
  }
  return true;
}

// Raw values of one stage (TC_KS of K from k0) of the part's operands, as
// this thread's four K-adjacent pairs of op(A) and of op(B) (zero outside
// the part or the segment).
__device__ __forceinline__ void tc_load(const double* A, const double* B, const Seg& gs, const Sub& sb, int k0,
                                        double (&va)[8], double (&vb)[8]) {
  const bool ta = gs.trans & 1, tb = gs.trans & 2;
  const int kc = min(TC_KS, gs.k - k0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int i, kk;
    tc_slot(q, i, kk);
    const double* P = ta ? A + (int64_t)(k0 + kk) + (int64_t)i * gs.lda : A + (int64_t)i + (int64_t)(k0 + kk) * gs.lda;
    const int64_t step = ta ? 1 : gs.lda;
    va[2 * q] = (i < sb.rm && kk < kc) ? __ldcg(P) : 0.0;
    va[2 * q + 1] = (i < sb.rm && kk + 1 < kc) ? __ldcg(P + step) : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int j, kk;
    tc_slot(q, j, kk);
    const double* P = tb ? B + (int64_t)j + (int64_t)(k0 + kk) * gs.ldb : B + (int64_t)(k0 + kk) + (int64_t)j * gs.ldb;
    const int64_t step = tb ? gs.ldb : 1;
    vb[2 * q] = (j < sb.cn && kk < kc) ? __ldcg(P) : 0.0;
    vb[2 * q + 1] = (j < sb.cn && kk + 1 < kc) ? __ldcg(P + step) : 0.0;
  }
}

// acc (accumulate<2,4> thread mapping: rows tx + 16 i, columns ty + 8 jj) =
// sum over the task's segments of op(A) op(B) for the sub-tile sb (<= 32 x
// 32), through S-digit products on the tensor cores (see above). The next
// stage's operands are loaded while the current one is split into digits.
template <int S, int DB>
__device__ void accumulate_tc(const KParams& p, const Task& tk, const Sub& sb, double (&acc)[2][4], double* smem,
                              TcShared& ts) {
  // FP32-class parts (S = 4) take per-element FP32 pieces (piece_pairs): no
  // shared exponents, so no exponent pre-pass and no scaling at the drain
  constexpr bool FLT = S == 4;
  constexpr int G = S / 4;                 // stacks of four A planes
  constexpr int BITS = DB * S - 2;
  // K accumulated in a TMEM cell before it is read: exactly (integers of
  // magnitude at most 2^24, at most G products of 2^(2 DB - 2) per K step)
  // for emulated FP64;
  // the FP32-class mode only needs FP32 accumulation
  constexpr int KMAX = S == 8 ? (1 << 24) / (G << (2 * DB - 2)) : 4096;
  constexpr int ROWS = 32 * S;             // rows of the A stacks and of the B concatenation
  constexpr uint32_t OPB = ROWS * TC_KS * 2;  // bytes of one operand in a stage
  // k2 = E_i + F_j - kScale: X_a X_b summed over the kept levels is
  // 2^(DB (S - 1)) V with V = sum_L S_L 2^(DB (S - 1 - L))
  constexpr int kScale = 2044 + 2 * BITS - DB * (S - 1);
  static_assert((S == 8 || S == 4) && DB == 8, "digit formats of the two modes");
  static_assert(S == 4 || KMAX >= TC_KS, "exact chunk");
  static_assert(32 * 4 * 32 * 16 <= 2 * TC_STAGE_BYTES_MAX, "drain buffer fits the staging region");
  uint8_t* stage = reinterpret_cast<uint8_t*>(smem);
  int* rexp = reinterpret_cast<int*>(stage + TC_EXP_OFF);
  int* cexp = rexp + 32;
  // the part's result, row lane, column 4 js + warp owned by thread (warp, lane)
  double* R = reinterpret_cast<double*>(stage + TC_RES_OFF);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // A part whose whole K is two stages (one segment of at most 2 TC_KS: the
  // factor's one-block-column updates) takes the exact row / column exponents
  // from the two stages' values in registers (in the segment loop below),
  // read back to back, instead of a pass of its own.
  bool small = false;
  if constexpr (!FLT) small = tk.nseg == 1 && load_seg(p, tk.seg0).k <= 2 * TC_KS;
  if constexpr (!FLT) if (!small) {
    if (tid < 64) rexp[tid] = 0;
    __syncthreads();
    for (int s = 0; s < tk.nseg; ++s) {
      const Seg gs = load_seg(p, tk.seg0 + s);
      const bool ta = gs.trans & 1, tb = gs.trans & 2;
      const double* A = resolve(p, gs.a) + (ta ? (int64_t)sb.r0 * gs.lda : (int64_t)sb.r0);
      const double* B = resolve(p, gs.b) + (tb ? (int64_t)sb.c0 : (int64_t)sb.c0 * gs.ldb);
      max_exp_into(A, gs.lda, !ta, sb.rm, gs.k, rexp);
      max_exp_into(B, gs.ldb, tb, sb.cn, gs.k, cexp);
    }
  }
#pragma unroll
  for (int js = 0; js < 8; ++js) R[lane * 33 + 4 * js + warp] = 0.0;
  int nstage = 0, kacc = 0;
  const uint32_t mb0 = tc::smem_addr(&ts.mbar[0]), mb1 = tc::smem_addr(&ts.mbar[1]);
  for (int s = 0; s < tk.nseg; ++s) {
    const Seg gs = load_seg(p, tk.seg0 + s);
    const bool ta = gs.trans & 1, tb = gs.trans & 2;
    const double* A = resolve(p, gs.a) + (ta ? (int64_t)sb.r0 * gs.lda : (int64_t)sb.r0);
    const double* B = resolve(p, gs.b) + (tb ? (int64_t)sb.c0 : (int64_t)sb.c0 * gs.ldb);
    double na[8], nb[8];  // the next stage's values, in flight
    tc_load(A, B, gs, sb, 0, na, nb);
    if (small) {
      // this thread holds row 8 warp + lane % 8 of op(A) and column 8 warp +
      // lane % 8 of op(B) at 8 of each stage's K; lanes lane % 8 + 8 m hold the
      // rest. The second stage is read here for its exponents only (the loop
      // reads it again as its prefetch, from L2).
      int ea = 0, eb = 0;
      if (gs.k > TC_KS) {
        double xa[8], xb[8];
        tc_load(A, B, gs, sb, TC_KS, xa, xb);
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          ea = max(ea, biased_exp(xa[x]));
          eb = max(eb, biased_exp(xb[x]));
        }
      }
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        ea = max(ea, biased_exp(na[x]));
        eb = max(eb, biased_exp(nb[x]));
      }
#pragma unroll
      for (int o = 8; o < 32; o <<= 1) {
        ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
        eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
      }
      if (lane < 8) {
        rexp[8 * warp + lane] = ea;
        cexp[8 * warp + lane] = eb;
      }
      __syncthreads();
    }
    for (int k0 = 0; k0 < gs.k; k0 += TC_KS) {
      double ca[8], cb[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        ca[x] = na[x];
        cb[x] = nb[x];
      }
      if (k0 + TC_KS < gs.k) tc_load(A, B, gs, sb, k0 + TC_KS, na, nb);
      const int buf = nstage & 1;
      uint8_t* sa = stage + buf * TC_STAGE_BYTES_MAX;
      uint8_t* sbuf = sa + OPB;
      // the MMAs that last read this buffer (two stages ago) must be done
      // (a wait that runs out of budget ends the part on every thread at the barrier below)
      const bool ok = nstage < 2 || tc_wait(p, buf ? mb1 : mb0, (ts.ncommit[buf] - 1) & 1);
      if (ok) {
        // op(A) rows: digit t of row i goes to stack row 128 (t % G) + 32 (t / G) + i
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i, kk;
          tc_slot(q, i, kk);
          uint32_t w[S];
          if constexpr (FLT) piece_pairs(ca[2 * q], ca[2 * q + 1], w);
          else digit_pairs<S, DB>(ca[2 * q], ca[2 * q + 1], rexp[i], w);
#pragma unroll
          for (int t = 0; t < S; ++t)
            *reinterpret_cast<uint32_t*>(sa + tc_off(128 * (t % G) + 32 * (t / G) + i, kk)) = w[t];
        }
        // op(B) columns: digit u of column j goes to row 32 u + j
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int j, kk;
          tc_slot(q, j, kk);
          uint32_t w[S];
          if constexpr (FLT) piece_pairs(cb[2 * q], cb[2 * q + 1], w);
          else digit_pairs<S, DB>(cb[2 * q], cb[2 * q + 1], cexp[j], w);
#pragma unroll
          for (int t = 0; t < S; ++t) *reinterpret_cast<uint32_t*>(sbuf + tc_off(32 * t + j, kk)) = w[t];
        }
      }
      tc::fence_smem_to_async();
      if (__syncthreads_or(!ok)) return;
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_addr(sa), b0 = tc::smem_addr(sbuf);
#pragma unroll
        for (int ks = 0; ks < TC_KS / 16; ++ks)
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const uint64_t ad = tc::smem_desc(a0 + g * (128 / 8) * TC_SBO + ks * 2 * TC_LBO, TC_LBO, TC_SBO);
            const uint64_t bd = tc::smem_desc(b0 + ks * 2 * TC_LBO, TC_LBO, TC_SBO);
            tc::mma_bf16(ts.tmem + 32 * g, ad, bd, tc::idesc_bf16_f32(128, 32 * (S - g)),
                         (kacc == 0 && ks == 0 && g == 0) ? 0u : 1u);
          }
        tc::commit(buf ? mb1 : mb0);
        ts.ncommit[buf] += 1;
      }
      ++nstage;
      kacc += TC_KS;
      const bool last = (s == tk.nseg - 1) && (k0 + TC_KS >= gs.k);
      if (!last && kacc + TC_KS <= KMAX) continue;
      // ---- drain: every MMA done, cells -> exact sums -> FP64
      __syncthreads();  // ncommit of the last stage visible
      const bool done = (ts.ncommit[0] == 0 || tc_wait(p, mb0, (ts.ncommit[0] - 1) & 1)) &&
                        (ts.ncommit[1] == 0 || tc_wait(p, mb1, (ts.ncommit[1] - 1) & 1));
      if (__syncthreads_or(!done)) return;
      tc::fence_after_sync();
      kacc = 0;
      // lane block p (= warp) reads its cells, four columns at a time, and
      // leaves its partial sums for every (column, row) in the staging region
      long long* part = reinterpret_cast<long long*>(stage);  // [32 j][4 p][32 i] x (hi, lo)
      float* partf = reinterpret_cast<float*>(stage);          // [32 j][4 p][32 i]
      const uint32_t trow = ts.tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
      for (int js = 0; js < 8; ++js) {
        uint32_t cell[S][4];  // every column block is read; blocks of levels >= S are not used
        tc::ld_cells(trow + 4 * js, cell);
        if constexpr (S == 8) {
          long long hi[4], lo[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) hi[x] = lo[x] = 0;
#pragma unroll
          for (int c = 0; c < S; ++c) {
            const int L = G * warp + c;
            if (L <= S - 1) {
#pragma unroll
              for (int x = 0; x < 4; ++x) {
                const long long v = (long long)__float2int_rn(__uint_as_float(cell[c][x]));
                if (L <= 3) hi[x] += v << (DB * (3 - L));
                else lo[x] += v << (DB * (7 - L));
              }
            }
          }
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int e = ((4 * js + x) * 4 + warp) * 32 + lane;
            part[2 * e] = hi[x];
            part[2 * e + 1] = lo[x];
          }
        } else {
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            float v = 0.0f;
#pragma unroll
            for (int c = 0; c < S; ++c) {
              const int L = G * warp + c;
              if (L <= S - 1) v = FLT ? v + __uint_as_float(cell[c][x]) : fmaf(__uint_as_float(cell[c][x]), (float)(1 << (DB * (3 - L))), v);
            }
            partf[((4 * js + x) * 4 + warp) * 32 + lane] = v;
          }
        }
      }
      __syncthreads();
      // thread (warp, lane): outputs (row lane, column 4 js + warp)
#pragma unroll 2
      for (int js = 0; js < 8; ++js) {
        const int j = 4 * js + warp;
        double V;
        if constexpr (S == 8) {
          long long H = 0, Lo = 0;
#pragma unroll
          for (int pb = 0; pb < 4; ++pb) {
            const int e = (j * 4 + pb) * 32 + lane;
            H += part[2 * e];
            Lo += part[2 * e + 1];
          }
          V = fma((double)H, (double)(1ll << (4 * DB)), (double)Lo);  // H 2^(4 DB) + Lo, one rounding
        } else {
          float f = 0.0f;
#pragma unroll
          for (int pb = 0; pb < 4; ++pb) f += partf[(j * 4 + pb) * 32 + lane];
          V = (double)f;
        }
        double& r = R[lane * 33 + j];
        if constexpr (FLT) {
          r += V;
        } else {
          const int er = rexp[lane], ec = cexp[j];
          const int k2 = max(er, 1) + max(ec, 1) - kScale;
          const double sc =
              (k2 >= -1022 && k2 <= 1023) ? __longlong_as_double((long long)(k2 + 1023) << 52) : ldexp(1.0, k2);
          r = (er == 0x7ff || ec == 0x7ff) ? __longlong_as_double(0x7ff8000000000000ll) : fma(V, sc, r);
        }
      }
      tc::fence_before_sync();
      __syncthreads();  // TMEM reads done before the next MMAs; staging free again
    }
  }
  // to the accumulate<2,4> mapping
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = R[(tx + 16 * i) * 33 + ty + 8 * jj];
  __syncthreads();
}

// X[rl][cl] = sign * acc (or cin - acc) over the whole (16 TM) x (8 TN) sub-tile
// (rows / columns beyond the sub-tile get -acc = 0 or are ignored later).
template <int TM, int TN>
__device__ __forceinline__ void acc_to_smem(const KParams& p, const Task& tk, const Sub& sb, const double (&acc)[TM][TN],
                                            double* X, bool sub_cin, double sign) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double* C = sub_cin ? resolve(p, tk.cin) + sb.r0 + (int64_t)sb.c0 * tk.ldc : nullptr;
  // every load is issued before the first shared-memory store (a store
  // through a generic pointer would otherwise order the loads one by one)
  double v[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int r = tx + 16 * i, c = ty + 8 * j;
      v[i][j] = (sub_cin && r < sb.rm && c < sb.cn) ? __ldcg(C + r + (int64_t)c * tk.ldc) : 0.0;
    }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int r = tx + 16 * i, c = ty + 8 * j;
      const bool in = sub_cin && r < sb.rm && c < sb.cn;
      X[r * LDS + c] = in ? v[i][j] - acc[i][j] : sign * acc[i][j];
    }
}

// T[r][c] = lower triangle of the dim x dim block at tk.aux (zero above):
// thread t reads rows t % 64 of columns t / 64, +2, +4, ... in batches of 8
// loads in flight before their shared-memory stores.
__device__ __forceinline__ void load_tri(const KParams& p, const Task& tk, int dim, double* T) {
  const double* S = resolve(p, tk.aux);
  const int r = threadIdx.x & (FB - 1), c0 = threadIdx.x / FB;
  constexpr int kStep = NTHREADS / FB, kBatch = 8;
  for (int cb = c0; cb < FB; cb += kStep * kBatch) {
    double v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int c = cb + u * kStep;
      v[u] = (r < dim && c < dim && r >= c) ? __ldcg(S + r + (int64_t)c * tk.ldx) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int c = cb + u * kStep;
      if (r < dim && c < dim) T[r * LDS + c] = v[u];
    }
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

// X (m x n, m <= 16) <- X T^{-T} with the row values in registers: T lower
// n x n with its strict lower part already divided by the pivot of its column
// (Tn[c][j] = T[c][j] / T[j][j]), rcp[j*LDS] = 1 / T[j][j]. Warp w owns rows
// 4w .. 4w+3; the 8 lanes of a row hold its columns ph, ph+8, ... (ph = lane /
// 4). Step j takes the finished (not yet scaled) value y_j of each row from
// the lane that holds it (a shuffle) and subtracts y_j Tn[c][j] from the
// columns c > j; x = y / diag(T) at the end. No shared-memory round trip and
// no one-lane scaling between two steps.
__device__ __forceinline__ void trsm_rows_lt16(double* X, const double* Tn, const double* rcp, int m, int n) {
  static_assert(FB == 64, "8 lanes x 8 columns per row");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = warp * 4 + (lane & 3), ph = lane >> 2;
  const bool own = r < m;
  double y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = ph + 8 * q;
    y[q] = own && c < n ? X[r * LDS + c] : 0.0;
  }
#pragma unroll
  for (int j = 0; j < FB; ++j) {
    if (j >= n) break;
    const double yj = __shfl_sync(0xffffffffu, y[j >> 3], (lane & 3) + 4 * (j & 7));
#pragma unroll
    for (int q = j >> 3; q < 8; ++q) {
      const int c = ph + 8 * q;
      if (c > j) y[q] = fma(-yj, Tn[c * LDS + j], y[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = ph + 8 * q;
    if (own && c < n) X[r * LDS + c] = y[q] * rcp[c * LDS];
  }
}

// The same for m <= 8 (the parts of a row-split block on the factorization's
// critical path): two rows per warp, 16 lanes per row, so that a lane applies
// at most four columns per step.
__device__ __forceinline__ void trsm_rows_lt8(double* X, const double* Tn, const double* rcp, int m, int n) {
  static_assert(FB == 64, "16 lanes x 4 columns per row");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = warp * 2 + (lane & 1), ph = lane >> 1;
  const bool own = r < m;
  double y[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = ph + 16 * q;
    y[q] = own && c < n ? X[r * LDS + c] : 0.0;
  }
#pragma unroll
  for (int j = 0; j < FB; ++j) {
    if (j >= n) break;
    const double yj = __shfl_sync(0xffffffffu, y[j >> 4], (lane & 1) + 2 * (j & 15));
#pragma unroll
    for (int q = j >> 4; q < 4; ++q) {
      const int c = ph + 16 * q;
      if (c > j) y[q] = fma(-yj, Tn[c * LDS + j], y[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = ph + 16 * q;
    if (own && c < n) X[r * LDS + c] = y[q] * rcp[c * LDS];
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

// Trailing rank-1 update of the block POTRF, one batch of B elements per
// thread: element e of the packed lower triangle (width w, row pairs
// (a, w-1-a) of w+1 elements) maps to X[c0+a][c0+b] and is updated by column
// k. fetch() loads a batch (indices past ne are marked -1) and advances the
// (i, kk) walk; apply() writes it.
struct Rank1Walk {
  int c0, w, w1, k, ne, nt, di, dk, i, kk;
};
template <int B>
__device__ __forceinline__ void rank1_fetch(const double* X, Rank1Walk& s, int e, int (&id)[B], double (&xr)[B],
                                            double (&lr)[B], double (&lc)[B]) {
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int a = s.kk <= s.i ? s.i : s.w - 1 - s.i, b = s.kk <= s.i ? s.kk : s.kk - s.i - 1;
    id[u] = e + u * s.nt < s.ne ? (s.c0 + a) * LDS + s.c0 + b : -1;
    if (id[u] >= 0) {
      xr[u] = X[id[u]];
      lr[u] = X[(s.c0 + a) * LDS + s.k];
      lc[u] = X[(s.c0 + b) * LDS + s.k];
    }
    s.kk += s.dk;
    s.i += s.di;
    if (s.kk >= s.w1) {
      s.kk -= s.w1;
      ++s.i;
    }
  }
}
template <int B>
__device__ __forceinline__ void rank1_apply(double* X, const int (&id)[B], const double (&xr)[B],
                                            const double (&lr)[B], const double (&lc)[B]) {
#pragma unroll
  for (int u = 0; u < B; ++u)
    if (id[u] >= 0) X[id[u]] = fma(-lr[u], lc[u], xr[u]);
}

// In-place lower Cholesky of the n x n block X (n <= FB), one column per
// step with a two-column lookahead, so that a step has one block barrier:
//   warp 0, step j: pivot d = X[j][j], r = rsqrt(d) (one dependent FP64
//     chain instead of sqrt then a divide), column j scaled by r, then
//     column j+1 updated by columns j-1 and j (it is pivot j+1 next); the
//     column j-1 term does not depend on r and is applied while r is formed,
//     lane 0's scaled row j+1 is broadcast by a shuffle;
//   warps 1-3, step j: columns j+2 .. n-1 (lower part) updated by column j-1,
//     walking the lower triangle of width w as w/2 row pairs (a, w-1-a) of
//     w+1 elements each (no lane idles), in batches of six.
// Every column thus receives the updates of the columns before it in
// ascending order, and only warp 0's pivot chain is on the critical path.
// X[j][j] keeps the pivot d until the end (nothing reads it after step j);
// r is kept in the row's padding slot X[j][FB], and L_jj = d r and the pivot
// check are done for all columns at once after the loop.
// Returns the first column (0-based) whose pivot was not positive, or -1.
__device__ int potrf_smem(double* X, int n) {
  static_assert(FB <= 64 && LDS > FB, "two rows per lane of warp 0; a padding column per row");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_bad;
  if (tid == 0) s_bad = n;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      const int j1 = j + 1;
      const double d = X[j * LDS + j];
      const double l0 = j > 0 && j1 < n ? X[j1 * LDS + j - 1] : 0.0;
      double xj[2] = {0.0, 0.0}, x1[2] = {0.0, 0.0}, lj[2] = {0.0, 0.0};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = j1 + lane + 32 * u;
        if (r < n) {
          xj[u] = X[r * LDS + j];
          x1[u] = X[r * LDS + j1];
          if (j > 0) x1[u] = fma(-X[r * LDS + j - 1], l0, x1[u]);
        }
      }
      const double rr = rsqrt(d);
      if (lane == 0) X[j * LDS + FB] = rr;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = j1 + lane + 32 * u;
        if (r < n) {
          lj[u] = xj[u] * rr;
          X[r * LDS + j] = lj[u];
        }
      }
      const double l1 = __shfl_sync(0xffffffffu, lj[0], 0);  // L[j+1][j], row j+1 is lane 0's
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = j1 + lane + 32 * u;
        if (r < n) X[r * LDS + j1] = fma(-lj[u], l1, x1[u]);
      }
    } else if (j > 0 && j + 2 < n) {
      Rank1Walk s;
      s.c0 = j + 2;
      s.w = n - s.c0;
      s.w1 = s.w + 1;
      s.k = j - 1;
      s.ne = s.w * s.w1 / 2;
      s.nt = NTHREADS - 32;
      s.di = s.nt / s.w1;
      s.dk = s.nt % s.w1;
      const int t = tid - 32;
      s.i = t / s.w1;
      s.kk = t % s.w1;
      constexpr int B = 6;  // elements per batch: their loads are issued before their stores
      int id[B];
      double xr[B], lr[B], lc[B];
      for (int e = t; e < s.ne; e += B * s.nt) {
        rank1_fetch<B>(X, s, e, id, xr, lr, lc);
        rank1_apply<B>(X, id, xr, lr, lc);
      }
    }
    __syncthreads();
  }
  if (tid < n) {
    const double d = X[tid * LDS + tid];
    if (!(d > 0.0)) atomicMin(&s_bad, tid);
    X[tid * LDS + tid] = d * X[tid * LDS + FB];
  }
  __syncthreads();
  return s_bad < n ? s_bad : -1;
}

template <bool TC, int TM, int TN>
__device__ void run_sub(const KParams& p, const Task& tk, const Sub& sb, double* smem, TcShared* ts) {
  double* As = smem;             // KC x LDS
  double* Bs = smem + KC * LDS;  // KC x LDS
  double* T = smem;              // FB x LDS, reuses As/Bs after the K-loop
  double* X = smem + 2 * KC * LDS;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m = tk.m, n = tk.n;
  double acc[TM][TN];
  if (tk.op != OP_TRTRI) {
    if constexpr (TC && TM == 2 && TN == 4) {  // reduced-precision parts are <= 32 x 32 sub-tiles
      if (tk.prec == PREC_EMU64) accumulate_tc<8, 8>(p, tk, sb, acc, smem, *ts);
      else if (tk.prec == PREC_FP32X) accumulate_tc<4, 8>(p, tk, sb, acc, smem, *ts);
      else accumulate<TM, TN>(p, tk, sb, acc, As, Bs);
    } else {
      accumulate<TM, TN>(p, tk, sb, acc, As, Bs);
    }
  }

  switch (tk.op) {
    case OP_UPD:
    case OP_STORE:
    case OP_NEG: {
      double* O = resolve(p, tk.out) + sb.r0 + (int64_t)sb.c0 * tk.ldo;
      const double* C = tk.op == OP_UPD ? resolve(p, tk.cin) + sb.r0 + (int64_t)sb.c0 * tk.ldc : nullptr;
      // an off-diagonal Sigma block is final when its NEG task writes it (the
      // planner emits NEG and SYMUPD tasks only with outputs, and SYMUPD
      // mirror blocks, in the Sigma buffer, so the offsets below stay inside it)
      double* Om = tk.op == OP_NEG && p.smirror ? p.smirror + (O - p.buf[BUF_S]) : nullptr;
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
            if (Om) Om[r + (int64_t)c * tk.ldo] = v;
          }
        }
      break;
    }
    case OP_SYMUPD: {
      acc_to_smem<TM, TN>(p, tk, sb, acc, X, true, 1.0);
      __syncthreads();
      double* O = resolve(p, tk.out);
      // the diagonal tile's Sigma blocks are final when their SYMUPD writes them
      if ((tk.flags & TF_SYM_DIAG) && sb.r0 == sb.c0) {  // diagonal sub-block: keep its lower triangle, mirror it
        double* D = O + sb.r0 + (int64_t)sb.c0 * tk.ldo;
        double* Dm = p.smirror ? p.smirror + (D - p.buf[BUF_S]) : nullptr;
        for (int e = tid; e < sb.rm * sb.cn; e += NTHREADS) {
          const int r = e % sb.rm, c = e / sb.rm;
          const double v = r >= c ? X[r * LDS + c] : X[c * LDS + r];
          D[r + (int64_t)c * tk.ldo] = v;
          if (Dm) Dm[r + (int64_t)c * tk.ldo] = v;
        }
      } else {
        // this sub-block, and its transpose into the mirror position: inside the
        // same block for a diagonal block, else the mirror block (aux)
        double* D = O + sb.r0 + (int64_t)sb.c0 * tk.ldo;
        const bool dblk = tk.flags & TF_SYM_DIAG;
        double* M = dblk ? O + sb.c0 + (int64_t)sb.r0 * tk.ldo : resolve(p, tk.aux) + sb.c0 + (int64_t)sb.r0 * tk.ldx;
        const int ldm = dblk ? tk.ldo : tk.ldx;
        double* Dm = p.smirror ? p.smirror + (D - p.buf[BUF_S]) : nullptr;
        double* Mm = p.smirror ? p.smirror + (M - p.buf[BUF_S]) : nullptr;
        for (int e = tid; e < sb.rm * sb.cn; e += NTHREADS) {
          const int r = e % sb.rm, c = e / sb.rm;
          D[r + (int64_t)c * tk.ldo] = X[r * LDS + c];
          if (Dm) Dm[r + (int64_t)c * tk.ldo] = X[r * LDS + c];
        }
        for (int e = tid; e < sb.rm * sb.cn; e += NTHREADS) {
          const int c = e % sb.cn, r = e / sb.cn;
          M[c + (int64_t)r * ldm] = X[r * LDS + c];
          if (Mm) Mm[c + (int64_t)r * ldm] = X[r * LDS + c];
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
      if (sb.rm <= 16) {  // every part of a row-split block
        const int warp = tid >> 5, lane = tid & 31;
        for (int c = warp + 1; c < n; c += NTHREADS / 32)
          for (int j = lane; j < c; j += 32) T[c * LDS + j] *= rcp[j * LDS];
        __syncthreads();
        if (sb.rm <= 8) trsm_rows_lt8(X, T, rcp, sb.rm, n);
        else trsm_rows_lt16(X, T, rcp, sb.rm, n);
      } else {
        trsm_rows_lt(X, T, rcp, sb.rm, n);
      }
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
            const int bad = potrf_smem(X, n);
            store_sub(p, tk, sb, X, true);
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
                if (p.badpiv) p.badpiv[tk.diag] = bad;
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
    const Seg g = load_seg(p, tk.seg0 + s);
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
  return true;
}
#endif

// OP_ZERO: the zrows x n block above the task's output block (column-major,
// leading dimension ldo) set to zero.
__device__ void run_zero(const KParams& p, const Task& tk, int t) {
#ifdef STILES_CHECKED
  if (tk.zrows < 1 || tk.n < 1 || !ref_ok(p, tk.out, -(int64_t)tk.zrows, (int64_t)(tk.n - 1) * tk.ldo)) {
    if (threadIdx.x == 0) check_fail(p, 7, t, 0);
    return;
  }
#endif
  double* Z = resolve(p, tk.out) - tk.zrows;
  for (int e = threadIdx.x; e < tk.zrows * tk.n; e += NTHREADS) Z[e % tk.zrows + (int64_t)(e / tk.zrows) * tk.ldo] = 0.0;
}

template <bool TC>
__device__ void run_task(const KParams& p, const Task& tk, int t, int q, double* smem, TcShared* ts) {
  if (tk.op == OP_PREP) {
    run_prep(p, tk, t);
    return;
  }
  if (tk.op == OP_ZERO) {
    run_zero(p, tk, t);
    return;
  }
  if (tk.op == OP_JOIN) return;  // a dependency point only
  const Sub sb = sub_of(tk, q);
  if (sb.rm <= 0 || sb.cn <= 0) return;
#ifdef STILES_CHECKED
  if (!task_part_ok(p, tk, sb)) {
    if (threadIdx.x == 0) check_fail(p, 7, t, q);
    return;
  }
#endif
  switch (tk.pmode) {
    case PM_ROWS2: run_sub<TC, 2, 8>(p, tk, sb, smem, ts); break;
    case PM_ROWS4:
    case PM_ROWS8: run_sub<TC, 1, 8>(p, tk, sb, smem, ts); break;
    case PM_TRI16:
    case PM_QUAD16: run_sub<TC, 1, 2>(p, tk, sb, smem, ts); break;
    case PM_QUAD4:
    case PM_TRI3:
    case PM_TILE32: run_sub<TC, 2, 4>(p, tk, sb, smem, ts); break;
    default: run_sub<TC, 4, 8>(p, tk, sb, smem, ts); break;
  }
}

__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// Per-CTA state of the tensor path, in static shared memory of the kernel
// instance that has one.
template <bool TC>
__device__ __forceinline__ TcShared* tc_shared() {
  if constexpr (TC) {
    __shared__ TcShared ts;
    return &ts;
  } else {
    return nullptr;
  }
}

// Two instances: TC = false for plans whose products are all FP64 (no
// tensor-core code at all), TC = true for plans with reduced-precision parts.
template <bool TC>
__global__ void __launch_bounds__(NTHREADS, 2) persistent_kernel(KParams p) {
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_item, s_last;
  TcShared* ts = tc_shared<TC>();
  // plans with reduced-precision products hold TC_COLS TMEM columns and two
  // completion barriers for the kernel's lifetime (two CTAs per SM: 512)
  if constexpr (TC) {
    if (threadIdx.x < 32) tc::tmem_alloc<TC_COLS>(&ts->tmem);
    if (threadIdx.x == 0) {
      tc::mbar_init(tc::smem_addr(&ts->mbar[0]), 1);
      tc::mbar_init(tc::smem_addr(&ts->mbar[1]), 1);
      tc::fence_mbar_init();
      ts->ncommit[0] = ts->ncommit[1] = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  // request server: idle workers give up this long after the kernel started
  const unsigned long long deadline = p.serve ? gtimer() + p.sv.deadline : 0ull;
  for (;;) {
    unsigned long long t_claim = 0;
    if (threadIdx.x < 32) {
      if (p.trace && threadIdx.x == 0) t_claim = gtimer();
      const int v = pop_task(p, deadline);
      if (threadIdx.x == 0) s_item = v;
    }
    __syncthreads();
    const int v = s_item;
    if (v < 0) break;
    const int t = v >> 2, q = v & 3;
#ifdef STILES_CHECKED
    if (t >= p.ntasks || q >= load_task(p, t).parts) {
      if (threadIdx.x == 0) check_fail(p, 8, t, q);
      break;
    }
#endif
    unsigned long long t_ready = 0;
    if (p.trace && threadIdx.x == 0) t_ready = gtimer();
    __threadfence();
    const Task tk = load_task(p, t);
    run_task<TC>(p, tk, t, q, smem, ts);
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
        if (threadIdx.x == 0) atomicAdd(&p.st->done, 1ull);
      }
      if (p.trace && threadIdx.x == 0) {  // one record per task part
        unsigned long long* tr = p.trace + 4 * (4 * (size_t)t + q);
        tr[0] = t_claim;
        tr[1] = t_ready;
        tr[2] = gtimer();
        tr[3] = ((unsigned long long)smid() << 32) | ((unsigned long long)blockIdx.x << 12) |
                ((unsigned long long)tk.prec << 10) | ((unsigned long long)s_last << 9) |
                ((unsigned long long)(tk.flags & TF_URGENT) << 7) | tk.op;
      }
    }
  }
  if constexpr (TC) {  // every part waited for its MMAs before it returned
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
      tc::fence_after_sync();
      tc::tmem_dealloc<TC_COLS>(ts->tmem);
    }
    if (threadIdx.x == 0) {
      tc::mbar_inval(tc::smem_addr(&ts->mbar[0]));
      tc::mbar_inval(tc::smem_addr(&ts->mbar[1]));
    }
  }
}

// Dynamic shared memory of a launch: the FP64 tasks' staging and block
// regions, or more when the plan has tensor-core parts.
size_t kernel_smem_bytes(bool use_tc) {
  const size_t fp64 = sizeof(double) * (size_t)(2 * KC * LDS + FB * LDS);
  return use_tc && (size_t)TC_SMEM_BYTES > fp64 ? (size_t)TC_SMEM_BYTES : fp64;
}

int kernel_threads() { return NTHREADS; }

const void* persistent_kernel_ptr(bool use_tc) {
  return use_tc ? (const void*)persistent_kernel<true> : (const void*)persistent_kernel<false>;
}

// The shared-memory limit is a per-device attribute of each kernel instance:
// it is set once for every device the process launches on (the current one).
cudaError_t configure_persistent() {
  constexpr int kMaxDevices = 64;
  static std::atomic<bool> configured[kMaxDevices];
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kMaxDevices;
  if (cached && configured[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  if (cached && configured[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(persistent_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kernel_smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(persistent_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem_bytes(true));
  if (e == cudaSuccess && cached) configured[dev].store(true, std::memory_order_release);
  return e;
}

cudaError_t kernel_occupancy(bool use_tc, int* blocks_per_sm) {
  cudaError_t e = configure_persistent();
  if (e != cudaSuccess) return e;
  return use_tc ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persistent_kernel<true>, NTHREADS,
                                                                kernel_smem_bytes(true))
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persistent_kernel<false>, NTHREADS,
                                                                kernel_smem_bytes(false));
}

cudaError_t launch_persistent(const KParams& p, int grid, cudaStream_t stream) {
  cudaError_t e = configure_persistent();
  if (e != cudaSuccess) return e;
  if (p.use_tc)
    persistent_kernel<true><<<grid, NTHREADS, kernel_smem_bytes(true), stream>>>(p);
  else
    persistent_kernel<false><<<grid, NTHREADS, kernel_smem_bytes(false), stream>>>(p);
  return cudaGetLastError();
}

}  // namespace stiles
