// C ABI of the selected-inversion library (declared in include/stiles.h):
// handle creation (planning on the host, one upload of the task tables),
// launches on the caller's stream, status and logdet read-back.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stiles.h"
#include "plan.h"
#include "stiles_device.h"

using namespace stiles;

namespace {

struct DevPlan {
  Task* tasks = nullptr;
  Seg* segs = nullptr;
  Wait* waits = nullptr;
  int32_t* sigs = nullptr;
  int ntasks = 0;
  int nctr = 0;
};

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
  int nctr_max = 0;
  size_t w_bytes = 0;        // scratch: L^{-1} and U tiles (packed layout)
  size_t ctr_offset = 0;     // scratch: counters start (bytes)
  size_t scratch_bytes = 0;
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
    cudaFree(d.waits);
    cudaFree(d.sigs);
  }
  cudaFree(h->dstatus);
  cudaFree(h->dlogdet);
  delete h;
}

extern "C" int stiles_create(int nt, int b, int band, int arrow, int precision, stiles_t* out) {
  if (!out) return STILES_ERR_INVALID_ARG;
  *out = nullptr;
  if (nt < 1 || b < 1 || band < 0 || arrow < 0) return STILES_ERR_INVALID_ARG;
  if (precision != STILES_FP64) return STILES_ERR_UNSUPPORTED;
  stiles_handle* h = new (std::nothrow) stiles_handle();
  if (!h) return STILES_ERR_OOM;
  h->s = Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow};
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return STILES_ERR_CUDA;
  }
  h->grid = h->sms;
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
    if (!rc) rc = upload(p.waits, &h->dev[k].waits);
    if (!rc) rc = upload(p.sigs, &h->dev[k].sigs);
    h->dev[k].ntasks = (int)p.tasks.size();
    h->dev[k].nctr = p.nctr;
    if (p.nctr > h->nctr_max) h->nctr_max = p.nctr;
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
  h->scratch_bytes = align_up(h->ctr_offset + sizeof(int) * ((size_t)h->nctr_max + 1), 256);
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
  int* ctr = (int*)(scr + h->ctr_offset);
  int* claim = ctr + h->nctr_max;
  if (cudaMemsetAsync(ctr, 0, sizeof(int) * ((size_t)d.nctr), st) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaMemsetAsync(claim, 0, sizeof(int), st) != cudaSuccess) return STILES_ERR_CUDA;
  DevStatus* ds = h->dstatus + kind;
  if (cudaMemsetAsync(ds, 0, sizeof(DevStatus), st) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaMemsetAsync(&ds->spd_col, 0xff, sizeof(unsigned long long), st) != cudaSuccess) return STILES_ERR_CUDA;
  KParams p{};
  p.tasks = d.tasks;
  p.segs = d.segs;
  p.waits = d.waits;
  p.sigs = d.sigs;
  p.ntasks = d.ntasks;
  p.ctr = ctr;
  p.claim = claim;
  p.st = ds;
  p.logdet_part = h->dlogdet;
  p.buf[BUF_A] = const_cast<double*>(A);
  p.buf[BUF_L] = L;
  p.buf[BUF_S] = S;
  p.buf[BUF_W] = (double*)scr;
  p.budget_ns = h->budget_ns;
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
  if (info) *info = c == STILES_ERR_NOT_SPD ? (long long)ds.spd_col + 1 : c == STILES_ERR_TIMEOUT ? (long long)ds.info : 0;
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
      h->grid = value == 0 ? h->sms : (int)value;
      return STILES_OK;
    default:
      return STILES_ERR_INVALID_ARG;
  }
}

extern "C" int stiles_plan_stats(int nt, int b, int band, int arrow, int which, int workers, long long stats[8]) {
  if (!stats || which < 0 || which > 2 || workers < 1) return STILES_ERR_INVALID_ARG;
  if (nt < 1 || b < 1 || band < 0 || arrow < 0) return STILES_ERR_INVALID_ARG;
  Plan p;
  int rc = build_plan(Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow}, (PlanKind)which, workers, &p);
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
  if (p.tasks.empty() || p.waits.empty()) return STILES_ERR_INVALID_ARG;
  // the first task with a wait now needs a signal count no task provides
  for (size_t t = 0; t < p.tasks.size(); ++t)
    if (p.tasks[t].nwait > 0) {
      Wait w = p.waits[p.tasks[t].wait0];
      w.need = 1 << 30;
      if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
      if (cudaMemcpy(h->dev[which].waits + p.tasks[t].wait0, &w, sizeof(Wait), cudaMemcpyHostToDevice) != cudaSuccess)
        return STILES_ERR_CUDA;
      p.waits[p.tasks[t].wait0] = w;
      return STILES_OK;
    }
  return STILES_ERR_INVALID_ARG;
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
    default: return "unknown status";
  }
}
