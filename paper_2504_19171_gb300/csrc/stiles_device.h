// Launch parameters and device status block of the persistent kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"

namespace stiles {

// Device status codes (the host maps them to stiles_status_code).
enum : int { STILES_DEV_OK = 0, STILES_DEV_NOT_SPD = 1, STILES_DEV_TIMEOUT = 2, STILES_DEV_CHECK = 3 };

struct DevStatus {
  int code;                    // first error (STILES_DEV_*)
  int abort;                   // set on TIMEOUT: every CTA stops claiming / waiting
  unsigned long long done;     // tasks completed
  unsigned long long info;     // TIMEOUT: index of the task whose wait expired
  unsigned long long spd_col;  // NOT_SPD: smallest failing global column (0-based); ~0 if none
};

// Per-launch scheduler state, one contiguous int32 block in the caller's
// scratch, reset before every launch from a device image built at create:
//   rem[ntasks]      predecessors not yet finished (image: indeg)
//   pdone[ntasks]    parts of the task finished so far
//   slots[nb*kSlotsPerBucket]  bucket b owns slots [b*kSlotsPerBucket, +kSlotsPerBucket)
//   tail[nbuckets]   slots reserved by pushes into the bucket so far
//   head[nbuckets]   slots claimed by pops so far
//   avail[nbuckets]  parts pushed and not yet claimed (a pop claims one by
//                    decrementing it while positive, then takes head++)
//   gcnt[ngroups]    ready parts per group of 32 buckets (a scan hint)
//   scnt[nsuper]     ready parts per super-group of 32 groups (a scan hint)
//   uslots[ucap]     urgent queue (critical-path tasks), popped before any bucket
//   lo[32]           lo[0]: every bucket below it is finished (all popped);
//                    lo[8]: urgent tail, lo[16]: urgent head, lo[24]: urgent avail
struct SchedState {
  int* rem;
  int* pdone;
  int* slots;
  int* tail;
  int* head;
  int* avail;
  int* gcnt;
  int* scnt;
  int* uslots;
  int* lo;
};

inline size_t sched_state_ints(int ntasks, int nbuckets, int ucap) {
  const int ngroups = (nbuckets + 31) / 32, nsuper = (ngroups + 31) / 32;
  return 2 * (size_t)ntasks + (size_t)nbuckets * kSlotsPerBucket + 3 * (size_t)nbuckets + (size_t)ngroups +
         (size_t)nsuper + (size_t)(ucap > 0 ? ucap : 1) + 32;
}

inline SchedState sched_state_at(int* base, int ntasks, int nbuckets, int ucap) {
  SchedState s;
  s.rem = base;
  s.pdone = s.rem + ntasks;
  s.slots = s.pdone + ntasks;
  s.tail = s.slots + (size_t)nbuckets * kSlotsPerBucket;
  s.head = s.tail + nbuckets;
  s.avail = s.head + nbuckets;
  s.gcnt = s.avail + nbuckets;
  s.scnt = s.gcnt + (nbuckets + 31) / 32;
  s.uslots = s.scnt + ((nbuckets + 31) / 32 + 31) / 32;
  s.lo = s.uslots + (ucap > 0 ? ucap : 1);
  return s;
}

// ---- request server (continuous batching in one running kernel) ----------
constexpr int kServeInbox = 4096;  // records in the host inbox ring (>= request slots)
constexpr int kServeMaxReq = 1024; // request slots

struct ServeRec {  // one activation, written by the host
  int slot;        // request slot
  int root0;       // its root tasks: roots[root0 .. root0 + nroots)
  int nroots;
  unsigned seq;    // sequence number, echoed in done_seq[slot] when the request completes
  double rho, tau; // value parameters of the request (OP_PREP)
};

struct ServeCtl {  // host-mapped (pinned) control block
  int inbox_count; // records published by the host
  int stop;        // 1: workers exit once idle
  int pad[30];
  ServeRec inbox[kServeInbox];
  unsigned done_seq[kServeMaxReq];  // written by the device (system-scope release)
};

struct ServeRing {  // ready parts of one priority class
  int* slots;       // capacity mask + 1 entries, -1 when free
  int* ctr;         // ctr[0] tail (reserved), ctr[8] head (claimed), ctr[16] available
  unsigned mask;
};

struct ServeDev {
  ServeRing ring[3];           // urgent, other factor tasks, the rest
  ServeCtl* ctl;               // device address of the host-mapped control block
  int* inbox_seen;             // records activated so far
  int32_t* treq;               // task -> request slot
  int32_t* req_left;           // per slot: tasks not yet finished
  unsigned* req_seq;           // per slot: sequence number of the request it holds
  double* req_param;           // per slot: rho, tau
  int32_t* roots;              // root task lists (global task indices)
  unsigned long long deadline; // %globaltimer value after which idle workers stop
};

struct KParams {
  const Task* tasks;
  const Seg* segs;
  const int32_t* succ_off;  // successors in schedule order
  const int32_t* succ;
  const int32_t* bcap;  // parts per bucket
  int ntasks;
  int nbuckets;
  int ucap;             // urgent queue capacity
  SchedState q;         // mutable scheduler state
  DevStatus* st;        // status block (reset before the launch)
  double* logdet_part;  // one partial sum of log diag(L) per POTRF task
  double* buf[4];       // BUF_A, BUF_L, BUF_S, BUF_W base pointers
  double* smirror;      // optional: second copy of every final Sigma write, same layout as buf[BUF_S]
                        // (a host buffer mapped into the device's address space), or null
  long long budget_ns;  // bound of one dependency wait
  int32_t* badpiv;     // optional: per POTRF task, first failing pivot (0-based in its block) or -1
  unsigned long long* trace;  // optional: 4 words per task (claim, ready, end ns; sm/cta/op), or null
  long long buf_len;          // doubles in each of buf[0..3] (self-checking builds)
  int serve;                  // 1: request server (rings and inbox instead of the static buckets)
  int use_tc;                 // 1: the plan has reduced-precision products (tensor memory and barriers held)
  ServeDev sv;
};

size_t kernel_smem_bytes(bool use_tc);  // dynamic shared memory of a launch
int kernel_threads();
// Sets the kernel's dynamic shared-memory limit on the current device (once per device).
cudaError_t configure_persistent();
const void* persistent_kernel_ptr(bool use_tc);  // the kernel instance a plan launches
cudaError_t launch_persistent(const KParams& p, int grid, cudaStream_t stream);
// Resident CTAs of the persistent kernel per SM at the launch's shared memory.
cudaError_t kernel_occupancy(bool use_tc, int* blocks_per_sm);

}  // namespace stiles
