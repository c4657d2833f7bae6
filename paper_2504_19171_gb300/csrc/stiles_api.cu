// C ABI of the selected-inversion library (declared in include/stiles.h):
// handle creation (planning on the host, one upload of the task tables),
// launches on the caller's stream, status and logdet read-back.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/stiles.h"
#include "plan.h"
#include "stiles_device.h"

using namespace stiles;
using stiles::sched_state_at;

namespace {

struct DevPlan {
  Task* tasks = nullptr;
  Seg* segs = nullptr;
  int32_t* succ_off = nullptr;
  int32_t* succ = nullptr;
  int32_t* bcap = nullptr;
  int32_t* image = nullptr;  // initial scheduler state (copied to scratch before each launch)
  size_t image_ints = 0;
  int ntasks = 0;
  int nbuckets = 0;
  int ucap = 0;
};

// Initial scheduler state of a plan: rem = indeg, slots = slots0, tail = tail0,
// head = 0, gcnt = ready tasks per group of 32 buckets, lo = 0.
std::vector<int32_t> sched_image(const Plan& p) {
  const int nt = (int)p.tasks.size(), nb = p.nbuckets;
  std::vector<int32_t> img(sched_state_ints(nt, nb, p.urgent_parts), 0);
  SchedState q = sched_state_at(img.data(), nt, nb, p.urgent_parts);
  for (int t = 0; t < nt; ++t) q.rem[t] = p.indeg[t];
  for (size_t i = 0; i < p.slots0.size(); ++i) q.slots[i] = p.slots0[i];
  for (int b = 0; b < nb; ++b) {
    q.tail[b] = p.tail0[b];
    q.avail[b] = p.tail0[b];
    q.gcnt[b >> 5] += p.tail0[b];
    q.scnt[b >> 10] += p.tail0[b];
  }
  for (size_t i = 0; i < p.uslots0.size(); ++i) q.uslots[i] = p.uslots0[i];
  q.lo[8] = p.urgent_tail0;
  q.lo[24] = p.urgent_tail0;
  return img;
}

template <typename T>
int upload(const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return 0;
  if (cudaMalloc((void**)out, v.size() * sizeof(T)) != cudaSuccess) return STILES_ERR_OOM;
  if (cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return STILES_ERR_CUDA;
  return 0;
}

}  // namespace

struct stiles_handle {
  Shape s;
  int device = 0;
  int sms = 0;
  int grid = 0;
  long long budget_ns = 20LL * 1000 * 1000 * 1000;
  Plan plans[3];
  DevPlan dev[3];
  DevStatus* dstatus = nullptr;  // one block per plan kind
  double* dlogdet = nullptr;
  int ndiag = 0;
  size_t state_ints_max = 0;
  size_t w_bytes = 0;        // scratch: L^{-1} and U tiles (packed layout)
  size_t ctr_offset = 0;     // scratch: scheduler state start (bytes)
  size_t scratch_bytes = 0;
  unsigned long long* dtrace = nullptr;  // optional per-task trace (STILES_OPT_TRACE)
  size_t trace_tasks = 0;
  cudaStream_t last_stream = nullptr;
  bool launched = false;
  int last_kind = -1;         // plan kind of the last launch
  int last_factor_kind = -1;  // plan kind of the last launch that factorized
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static void free_handle(stiles_handle* h) {
  if (!h) return;
  for (auto& d : h->dev) {
    cudaFree(d.tasks);
    cudaFree(d.segs);
    cudaFree(d.succ_off);
    cudaFree(d.succ);
    cudaFree(d.bcap);
    cudaFree(d.image);
  }
  cudaFree(h->dstatus);
  cudaFree(h->dlogdet);
  cudaFree(h->dtrace);
  delete h;
}

extern "C" int stiles_create(int nt, int b, int band, int arrow, int precision, stiles_t* out) {
  if (!out) return STILES_ERR_INVALID_ARG;
  *out = nullptr;
  if (nt < 1 || b < 1 || band < 0 || arrow < 0) return STILES_ERR_INVALID_ARG;
  if (precision != STILES_FP64 && precision != STILES_EMU64 && precision != STILES_FP32X) return STILES_ERR_UNSUPPORTED;
  stiles_handle* h = new (std::nothrow) stiles_handle();
  if (!h) return STILES_ERR_OOM;
  h->s = Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow, precision};
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return STILES_ERR_CUDA;
  }
  h->grid = h->sms * kCtasPerSm;
  for (int k = 0; k < 3; ++k) {
    int rc = build_plan(h->s, (PlanKind)k, h->grid, &h->plans[k]);
    if (rc) {
      delete h;
      return rc;
    }
  }
  int rc = 0;
  for (int k = 0; k < 3 && !rc; ++k) {
    Plan& p = h->plans[k];
    rc = upload(p.tasks, &h->dev[k].tasks);
    if (!rc) rc = upload(p.segs, &h->dev[k].segs);
    if (!rc) rc = upload(p.succ_off, &h->dev[k].succ_off);
    if (!rc) rc = upload(p.succ, &h->dev[k].succ);
    if (!rc) rc = upload(p.bcap, &h->dev[k].bcap);
    std::vector<int32_t> img = sched_image(p);
    if (!rc) rc = upload(img, &h->dev[k].image);
    h->dev[k].image_ints = img.size();
    h->dev[k].ntasks = (int)p.tasks.size();
    h->dev[k].nbuckets = p.nbuckets;
    h->dev[k].ucap = p.urgent_parts;
    if (img.size() > h->state_ints_max) h->state_ints_max = img.size();
    if (p.ndiag > h->ndiag) h->ndiag = p.ndiag;
  }
  if (!rc && cudaMalloc((void**)&h->dstatus, 3 * sizeof(DevStatus)) != cudaSuccess) rc = STILES_ERR_OOM;
  if (!rc && cudaMalloc((void**)&h->dlogdet, sizeof(double) * (h->ndiag > 0 ? h->ndiag : 1)) != cudaSuccess)
    rc = STILES_ERR_OOM;
  if (rc) {
    free_handle(h);
    return rc;
  }
  Layout L(h->s);
  h->w_bytes = align_up((size_t)L.doubles() * sizeof(double), 256);
  h->ctr_offset = h->w_bytes;
  h->scratch_bytes = align_up(h->ctr_offset + sizeof(int) * h->state_ints_max, 256);
  *out = h;
  return STILES_OK;
}

extern "C" int stiles_layout_doubles(stiles_t h, size_t* doubles) {
  if (!h || !doubles) return STILES_ERR_INVALID_ARG;
  *doubles = (size_t)Layout(h->s).doubles();
  return STILES_OK;
}

extern "C" int stiles_workspace_bytes(stiles_t h, size_t* L_bytes, size_t* sigma_bytes, size_t* scratch_bytes) {
  if (!h) return STILES_ERR_INVALID_ARG;
  const size_t bytes = (size_t)Layout(h->s).doubles() * sizeof(double);
  if (L_bytes) *L_bytes = bytes;
  if (sigma_bytes) *sigma_bytes = bytes;
  if (scratch_bytes) *scratch_bytes = h->scratch_bytes;
  return STILES_OK;
}

static int launch(stiles_t h, int kind, const double* A, double* L, double* S, void* scratch, void* stream) {
  if (!h || !scratch) return STILES_ERR_INVALID_ARG;
  if (((uintptr_t)scratch) % 256 != 0) return STILES_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const DevPlan& d = h->dev[kind];
  char* scr = (char*)scratch;
  int* state = (int*)(scr + h->ctr_offset);
  if (d.image_ints &&
      cudaMemcpyAsync(state, d.image, sizeof(int) * d.image_ints, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return STILES_ERR_CUDA;
  DevStatus* ds = h->dstatus + kind;
  if (cudaMemsetAsync(ds, 0, sizeof(DevStatus), st) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaMemsetAsync(&ds->spd_col, 0xff, sizeof(unsigned long long), st) != cudaSuccess) return STILES_ERR_CUDA;
  KParams p{};
  p.tasks = d.tasks;
  p.segs = d.segs;
  p.succ_off = d.succ_off;
  p.succ = d.succ;
  p.bcap = d.bcap;
  p.ntasks = d.ntasks;
  p.nbuckets = d.nbuckets;
  p.ucap = d.ucap;
  p.q = sched_state_at(state, d.ntasks, d.nbuckets, d.ucap);
  p.st = ds;
  p.logdet_part = h->dlogdet;
  p.buf[BUF_A] = const_cast<double*>(A);
  p.buf[BUF_L] = L;
  p.buf[BUF_S] = S;
  p.buf[BUF_W] = (double*)scr;
  p.budget_ns = h->budget_ns;
  p.trace = h->dtrace;
  if (h->dtrace && cudaMemsetAsync(h->dtrace, 0, 16 * sizeof(unsigned long long) * h->trace_tasks, st) != cudaSuccess)
    return STILES_ERR_CUDA;
  p.buf_len = Layout(h->s).doubles();
  h->last_stream = st;
  h->launched = true;
  h->last_kind = kind;
  if (kind != PLAN_SELINV) h->last_factor_kind = kind;
  if (d.ntasks == 0) return STILES_OK;
  if (launch_persistent(p, h->grid, st) != cudaSuccess) return STILES_ERR_CUDA;
  return STILES_OK;
}

extern "C" int stiles_factor(stiles_t h, const double* A, double* L, void* scratch, void* stream) {
  if (!A || !L) return STILES_ERR_INVALID_ARG;
  return launch(h, PLAN_FACTOR, A, L, nullptr, scratch, stream);
}

extern "C" int stiles_selinv(stiles_t h, const double* L, double* S, void* scratch, void* stream) {
  if (!L || !S || (const double*)S == L || (void*)S == scratch) return STILES_ERR_INVALID_ARG;
  return launch(h, PLAN_SELINV, nullptr, const_cast<double*>(L), S, scratch, stream);
}

extern "C" int stiles_factor_selinv(stiles_t h, const double* A, double* L, double* S, void* scratch, void* stream) {
  if (!A || !L || !S || S == L || (const double*)S == A || (void*)S == scratch) return STILES_ERR_INVALID_ARG;
  return launch(h, PLAN_FUSED, A, L, S, scratch, stream);
}

extern "C" int stiles_factor_selinv_host(stiles_t h, const double* A_host, double* S_host, double* A_dev,
                                         double* L_dev, double* S_dev, void* scratch, void* stream) {
  if (!h || !A_host || !S_host || !A_dev || !L_dev || !S_dev || S_dev == L_dev || S_dev == A_dev ||
      (void*)S_dev == scratch)
    return STILES_ERR_INVALID_ARG;
  const size_t bytes = (size_t)Layout(h->s).doubles() * sizeof(double);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(A_dev, A_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return STILES_ERR_CUDA;
  const int rc = launch(h, PLAN_FUSED, A_dev, L_dev, S_dev, scratch, stream);
  if (rc != STILES_OK) return rc;
  if (cudaMemcpyAsync(S_host, S_dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return STILES_ERR_CUDA;
  return STILES_OK;
}

// Scratch of stiles_factor_selinv_noalloc: one fixed array per device that
// loads the library, shared by every call (see include/stiles.h).
static __device__ __align__(256) unsigned char g_noalloc_scratch[STILES_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Device address of the array on `device` (which must be current). Looked up
// once per device; the host-side name of the array is not a device address.
int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return STILES_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return STILES_ERR_CUDA;
    g_noalloc_ptr[device] = ptr;
  }
  *out = g_noalloc_ptr[device];
  return STILES_OK;
}
}  // namespace

extern "C" int stiles_factor_selinv_noalloc(stiles_t h, const double* A, double* L, double* S, void* stream) {
  if (!h || !A || !L || !S || S == L || (const double*)S == A) return STILES_ERR_INVALID_ARG;
  if (h->scratch_bytes > STILES_NOALLOC_SCRATCH_BYTES) return STILES_ERR_TOO_LARGE;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  void* scratch = nullptr;
  const int rc = noalloc_scratch(h->device, &scratch);
  if (rc) return rc;
  return launch(h, PLAN_FUSED, A, L, S, scratch, stream);
}

static int read_status(stiles_t h, int kind, DevStatus* ds) {
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaMemcpy(ds, h->dstatus + kind, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess)
    return STILES_ERR_CUDA;
  return STILES_OK;
}

static int code_of(const DevStatus& ds) {
  if (ds.code == STILES_DEV_NOT_SPD) return STILES_ERR_NOT_SPD;
  if (ds.code == STILES_DEV_TIMEOUT) return STILES_ERR_TIMEOUT;
  if (ds.code == STILES_DEV_CHECK) return STILES_ERR_PLAN;
  return STILES_OK;
}

extern "C" int stiles_status(stiles_t h, int* code, long long* info, long long* tasks_done) {
  if (!h) return STILES_ERR_INVALID_ARG;
  if (!h->launched) {
    if (code) *code = STILES_OK;
    if (info) *info = 0;
    if (tasks_done) *tasks_done = 0;
    return STILES_OK;
  }
  DevStatus ds;
  int rc = read_status(h, h->last_kind, &ds);
  if (rc) return rc;
  const int c = code_of(ds);
  if (code) *code = c;
  if (info) *info = c == STILES_ERR_NOT_SPD ? (long long)ds.spd_col + 1 : c != STILES_OK ? (long long)ds.info : 0;
  if (tasks_done) *tasks_done = (long long)ds.done;
  return STILES_OK;
}

extern "C" int stiles_logdet(stiles_t h, double* out_host) {
  if (!h || !out_host) return STILES_ERR_INVALID_ARG;
  if (h->last_factor_kind < 0) return STILES_ERR_INVALID_ARG;
  DevStatus ds;
  int rc = read_status(h, h->last_factor_kind, &ds);
  if (rc) return rc;
  const int c = code_of(ds);
  if (c != STILES_OK) return c;
  std::vector<double> part(h->ndiag);
  if (h->ndiag > 0 &&
      cudaMemcpy(part.data(), h->dlogdet, sizeof(double) * h->ndiag, cudaMemcpyDeviceToHost) != cudaSuccess)
    return STILES_ERR_CUDA;
  double acc = 0.0;
  for (double v : part) acc += v;  // fixed order: tile column, then block
  *out_host = 2.0 * acc;
  return STILES_OK;
}

extern "C" int stiles_set_option(stiles_t h, int option, long long value) {
  if (!h) return STILES_ERR_INVALID_ARG;
  switch (option) {
    case STILES_OPT_WAIT_BUDGET_NS:
      if (value <= 0) return STILES_ERR_INVALID_ARG;
      h->budget_ns = value;
      return STILES_OK;
    case STILES_OPT_GRID:
      if (value < 0 || value > 65535) return STILES_ERR_INVALID_ARG;
      h->grid = value == 0 ? h->sms * kCtasPerSm : (int)value;
      return STILES_OK;
    case STILES_OPT_TRACE: {
      if (value != 0 && value != 1) return STILES_ERR_INVALID_ARG;
      if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
      if (h->launched && cudaStreamSynchronize(h->last_stream) != cudaSuccess) return STILES_ERR_CUDA;
      cudaFree(h->dtrace);
      h->dtrace = nullptr;
      h->trace_tasks = 0;
      if (value) {
        size_t n = 0;
        for (auto& d : h->dev) n = (size_t)d.ntasks > n ? (size_t)d.ntasks : n;
        if (cudaMalloc((void**)&h->dtrace, 16 * sizeof(unsigned long long) * (n ? n : 1)) != cudaSuccess)
          return STILES_ERR_OOM;
        h->trace_tasks = n;
      }
      return STILES_OK;
    }
    default:
      return STILES_ERR_INVALID_ARG;
  }
}

extern "C" int stiles_plan_stats(int nt, int b, int band, int arrow, int which, int workers, long long stats[8]) {
  const int kind = which & 15, prec = which >> 4;
  if (!stats || kind < 0 || kind > 2 || prec < 0 || prec > PREC_FP32X || workers < 1) return STILES_ERR_INVALID_ARG;
  if (nt < 1 || b < 1 || band < 0 || arrow < 0) return STILES_ERR_INVALID_ARG;
  Plan p;
  int rc = build_plan(Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow, prec}, (PlanKind)kind, workers, &p);
  if (rc) return rc;
  stats[0] = (long long)p.tasks.size();
  stats[1] = (long long)p.segs.size();
  stats[2] = (long long)p.waits.size();
  stats[3] = p.nctr;
  stats[4] = (long long)p.flops;
  stats[5] = p.tile_gemms;
  stats[6] = (long long)p.cp_ns;
  stats[7] = (long long)p.makespan_ns;
  return STILES_OK;
}

extern "C" int stiles_debug_validate(int nt, int b, int band, int arrow, int which) {
  const int kind = which & 15, prec = which >> 4;
  if (kind < 0 || kind > 2 || prec < 0 || prec > PREC_FP32X || nt < 1 || b < 1 || band < 0 || arrow < 0)
    return STILES_ERR_INVALID_ARG;
  const Shape sh{nt, b, band < nt - 1 ? band : nt - 1, arrow, prec};
  Plan p;
  int rc = build_plan(sh, (PlanKind)kind, 304, &p);
  return rc ? rc : validate_plan(p, sh, kind);
}

extern "C" int stiles_debug_check_corrupted(int nt, int b, int band, int arrow, int which, int mode) {
  if (which < 0 || which > 2 || nt < 1 || b < 1 || band < 0 || arrow < 0) return STILES_ERR_INVALID_ARG;
  Plan p;
  int rc = build_plan(Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow}, (PlanKind)which, 16, &p);
  if (rc) return rc;
  if (p.waits.empty() || p.tasks.size() < 2) return STILES_ERR_INVALID_ARG;
  switch (mode) {
    case 1: p.waits.back().ctr = p.nctr; break;
    case 2: p.waits.back().need += 1000000; break;
    case 3: {  // make the first task that waits depend on the last task's signal
      const Task& last = p.tasks.back();
      if (last.nsig < 1) return STILES_ERR_INVALID_ARG;
      for (Task& t : p.tasks)
        if (t.nwait > 0) {
          p.waits[t.wait0] = Wait{p.sigs[last.sig0], 1 << 20};
          break;
        }
      break;
    }
    default: return STILES_ERR_INVALID_ARG;
  }
  return check_plan(p);
}

extern "C" int stiles_debug_break_plan(stiles_t h, int which) {
  if (!h || which < 0 || which > 2) return STILES_ERR_INVALID_ARG;
  Plan& p = h->plans[which];
  // the first task with a predecessor now waits for one more that never comes
  for (size_t t = 0; t < p.tasks.size(); ++t)
    if (p.indeg[t] > 0) {
      const int32_t v = p.indeg[t] + 1;
      if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
      if (cudaMemcpy(h->dev[which].image + t, &v, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return STILES_ERR_CUDA;
      p.indeg[t] = v;
      return STILES_OK;
    }
  return STILES_ERR_INVALID_ARG;
}

extern "C" int stiles_trace(stiles_t h, unsigned long long* out_host, size_t capacity, size_t* n_tasks) {
  if (!h || !n_tasks) return STILES_ERR_INVALID_ARG;
  if (!h->dtrace || !h->launched) return STILES_ERR_INVALID_ARG;
  const size_t n = (size_t)h->dev[h->last_kind].ntasks;
  *n_tasks = n;
  if (!out_host) return STILES_OK;
  if (capacity < 16 * n) return STILES_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return STILES_ERR_CUDA;
  if (n && cudaMemcpy(out_host, h->dtrace, 16 * sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return STILES_ERR_CUDA;
  return STILES_OK;
}

extern "C" int stiles_destroy(stiles_t h) {
  if (!h) return STILES_OK;
  if (h->launched) {
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->last_stream);
  }
  free_handle(h);
  return STILES_OK;
}

extern "C" const char* stiles_strerror(int code) {
  switch (code) {
    case STILES_OK: return "ok";
    case STILES_ERR_INVALID_ARG: return "invalid argument";
    case STILES_ERR_NOT_SPD: return "matrix is not symmetric positive definite";
    case STILES_ERR_TIMEOUT: return "a device dependency wait timed out";
    case STILES_ERR_CUDA: return "CUDA runtime error";
    case STILES_ERR_OOM: return "out of memory";
    case STILES_ERR_UNSUPPORTED: return "unsupported option";
    case STILES_ERR_PLAN: return "task table failed its consistency check";
    case STILES_ERR_TOO_LARGE: return "shape too large for the fixed no-allocation scratch";
    default: return "unknown status";
  }
}
