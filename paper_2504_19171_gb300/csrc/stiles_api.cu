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

// cudaMalloc that leaves no error behind when it fails: the failure is
// reported as STILES_ERR_OOM, and the runtime's last-error slot is cleared so
// that a later launch check does not pick it up.
int dev_malloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) == cudaSuccess) return 0;
  *p = nullptr;
  cudaGetLastError();
  return STILES_ERR_OOM;
}

template <typename T>
int upload(const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return 0;
  if (dev_malloc((void**)out, v.size() * sizeof(T))) return STILES_ERR_OOM;
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
  bool mirror_ok = false;     // fused plan: every final Sigma write (NEG, SYMUPD) lands in the Sigma buffer
};

// The kernel mirrors the writes of the fused plan's NEG and SYMUPD tasks to a
// host buffer at their offset in the Sigma buffer: allowed only when every
// such write (output block, and the mirror block of an off-diagonal SYMUPD)
// is in the Sigma buffer.
static bool sigma_writes_in_sigma(const Plan& p) {
  for (const Task& t : p.tasks) {
    if (t.op != OP_NEG && t.op != OP_SYMUPD) continue;
    if ((t.out >> BUF_SHIFT) != BUF_S) return false;
    if (t.op == OP_SYMUPD && !(t.flags & TF_SYM_DIAG) && (t.aux >> BUF_SHIFT) != BUF_S) return false;
  }
  return true;
}

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

static int create_handle(int nt, int b, int band, int arrow, int precision, int tuning, int first_column,
                         stiles_t* out);

extern "C" int stiles_create(int nt, int b, int band, int arrow, int precision, stiles_t* out) {
  return create_handle(nt, b, band, arrow, precision, 0, 0, out);
}

extern "C" int stiles_create_tuned(int nt, int b, int band, int arrow, int precision, int tuning, stiles_t* out) {
  return create_handle(nt, b, band, arrow, precision, tuning, 0, out);
}

extern "C" int stiles_create_selected(int nt, int b, int band, int arrow, int precision, int first_column,
                                      stiles_t* out) {
  return create_handle(nt, b, band, arrow, precision, 0, first_column, out);
}

static int create_handle(int nt, int b, int band, int arrow, int precision, int tuning, int first_column,
                         stiles_t* out) {
  if (!out) return STILES_ERR_INVALID_ARG;
  *out = nullptr;
  if (nt < 1 || b < 1 || band < 0 || arrow < 0 || !tune_valid(tuning)) return STILES_ERR_INVALID_ARG;
  if (first_column < 0 || first_column > (arrow > 0 ? nt : nt - 1)) return STILES_ERR_INVALID_ARG;
  if (precision != STILES_FP64 && precision != STILES_EMU64 && precision != STILES_FP32X) return STILES_ERR_UNSUPPORTED;
  stiles_handle* h = new (std::nothrow) stiles_handle();
  if (!h) return STILES_ERR_OOM;
  h->s = Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow, precision, tuning, first_column};
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
  if (!rc) rc = dev_malloc((void**)&h->dstatus, 3 * sizeof(DevStatus));
  if (!rc) rc = dev_malloc((void**)&h->dlogdet, sizeof(double) * (h->ndiag > 0 ? h->ndiag : 1));
  if (rc) {
    free_handle(h);
    return rc;
  }
  h->mirror_ok = sigma_writes_in_sigma(h->plans[PLAN_FUSED]);
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

static int launch(stiles_t h, int kind, const double* A, double* L, double* S, void* scratch, void* stream,
                  double* smirror = nullptr) {
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
  p.smirror = smirror;
  p.budget_ns = h->budget_ns;
  p.use_tc = h->s.prec != PREC_FP64;
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

// Device address of the `bytes`-long host buffer at `ptr` when it is
// page-locked and mapped into the current device's address space (both of
// its ends resolve into one mapping), else null: pageable memory, device
// memory, or a buffer that runs past its page-locked allocation.
static const char* mapped_host(const void* ptr, size_t bytes) {
  cudaPointerAttributes first{}, last{};
  if (cudaPointerGetAttributes(&first, ptr) != cudaSuccess ||
      cudaPointerGetAttributes(&last, (const char*)ptr + bytes - 1) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer is an answer here, not an error
    return nullptr;
  }
  if (first.type != cudaMemoryTypeHost || last.type != cudaMemoryTypeHost || !first.devicePointer ||
      (const char*)last.devicePointer != (const char*)first.devicePointer + bytes - 1)
    return nullptr;
  return (const char*)first.devicePointer;
}

extern "C" int stiles_factor_selinv_host(stiles_t h, const double* A_host, double* S_host, double* A_dev,
                                         double* L_dev, double* S_dev, void* scratch, void* stream) {
  if (!h || !A_host || !S_host || !A_dev || !L_dev || !S_dev || S_dev == L_dev || S_dev == A_dev ||
      (void*)S_dev == scratch)
    return STILES_ERR_INVALID_ARG;
  const size_t bytes = (size_t)Layout(h->s).doubles() * sizeof(double);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  // Page-locked, separate host buffers: the kernel reads A over the host link
  // as its factor tasks first need each block, and writes every final Sigma
  // block to the host buffer as well as to S_dev, so both transfers overlap
  // the computation instead of preceding and following it.
  const double* A_map = (const double*)mapped_host(A_host, bytes);
  double* S_map = (double*)mapped_host(S_host, bytes);
  const char *a0 = (const char*)A_host, *s0 = (const char*)S_host;
  const bool apart = a0 + bytes <= s0 || s0 + bytes <= a0;
  if (A_map && S_map && apart && h->mirror_ok)
    return launch(h, PLAN_FUSED, A_map, L_dev, S_dev, scratch, stream, S_map);
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

// Device address of the array on `device` (which must be current). The
// host-side name of the array is not a device address. Outside stream capture
// it is looked up on every call (an address kept from before a device or
// primary-context reset would be stale) and remembered; a call made while
// `stream` is capturing uses the address remembered by the last uncaptured
// call on that device, so no runtime lookup is made during capture.
int noalloc_scratch(int device, cudaStream_t stream, void** out) {
  if (device < 0 || device >= kMaxDevices) return STILES_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return STILES_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return STILES_ERR_CUDA;
    g_noalloc_ptr[device] = ptr;
  }
  if (!g_noalloc_ptr[device]) return STILES_ERR_INVALID_ARG;  // first call on this device is being captured
  *out = g_noalloc_ptr[device];
  return STILES_OK;
}
}  // namespace

extern "C" int stiles_factor_selinv_noalloc(stiles_t h, const double* A, double* L, double* S, void* stream) {
  if (!h || !A || !L || !S || S == L || (const double*)S == A) return STILES_ERR_INVALID_ARG;
  if (h->scratch_bytes > STILES_NOALLOC_SCRATCH_BYTES) return STILES_ERR_TOO_LARGE;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  void* scratch = nullptr;
  const int rc = noalloc_scratch(h->device, (cudaStream_t)stream, &scratch);
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
        if (dev_malloc((void**)&h->dtrace, 16 * sizeof(unsigned long long) * (n ? n : 1))) return STILES_ERR_OOM;
        h->trace_tasks = n;
      }
      return STILES_OK;
    }
    default:
      return STILES_ERR_INVALID_ARG;
  }
}

extern "C" int stiles_plan_stats(int nt, int b, int band, int arrow, int which, int workers, long long stats[10]) {
  const int kind = which & 15, prec = (which >> 4) & 15, tune = (which >> 8) & 255, sel0 = which >> 16;
  if (!stats || kind < 0 || kind > 2 || prec > PREC_FP32X || workers < 1 || !tune_valid(tune))
    return STILES_ERR_INVALID_ARG;
  if (nt < 1 || b < 1 || band < 0 || arrow < 0) return STILES_ERR_INVALID_ARG;
  Plan p;
  int rc = build_plan(Shape{nt, b, band < nt - 1 ? band : nt - 1, arrow, prec, tune, sel0}, (PlanKind)kind, workers,
                      &p);
  if (rc) return rc;
  stats[0] = (long long)p.tasks.size();
  stats[1] = (long long)p.segs.size();
  stats[2] = (long long)p.waits.size();
  stats[3] = p.nctr;
  stats[4] = (long long)p.flops;
  stats[5] = p.tile_gemms;
  stats[6] = (long long)p.cp_ns;
  stats[7] = (long long)p.makespan_ns;
  stats[8] = (long long)p.flops_lowered;
  stats[9] = (long long)p.succ.size();
  return STILES_OK;
}

extern "C" int stiles_debug_occupancy(int tensor_parts, int* blocks_per_sm) {
  if (!blocks_per_sm) return STILES_ERR_INVALID_ARG;
  return kernel_occupancy(tensor_parts != 0, blocks_per_sm) == cudaSuccess ? STILES_OK : STILES_ERR_CUDA;
}

extern "C" int stiles_debug_validate(int nt, int b, int band, int arrow, int which) {
  const int kind = which & 15, prec = (which >> 4) & 15, tune = (which >> 8) & 255, sel0 = which >> 16;
  if (kind < 0 || kind > 2 || prec > PREC_FP32X || !tune_valid(tune) || nt < 1 || b < 1 || band < 0 || arrow < 0)
    return STILES_ERR_INVALID_ARG;
  const Shape sh{nt, b, band < nt - 1 ? band : nt - 1, arrow, prec, tune, sel0};
  Plan p;
  int rc = build_plan(sh, (PlanKind)kind, 304, &p);
  return rc ? rc : validate_plan(p, sh, kind);
}

// Planted race of the race-check hook (plant = 2): every successor edge into
// the first column-join task of the table removed, so that the join -- and
// the phase-1 tasks that wait on it -- no longer follow the L blocks of their
// tile column. Returns false if the table has no join task.
static bool plant_unjoined_column(Plan& p) {
  const int n = (int)p.tasks.size();
  int join = -1;
  for (int t = 0; t < n && join < 0; ++t)
    if (p.tasks[t].op == OP_JOIN) join = t;
  if (join < 0) return false;
  std::vector<int32_t> off(n + 1, 0), succ;
  succ.reserve(p.succ.size());
  for (int t = 0; t < n; ++t) {
    off[t] = (int32_t)succ.size();
    for (int e = p.succ_off[t]; e < p.succ_off[t + 1]; ++e)
      if (p.succ[e] != join) succ.push_back(p.succ[e]);
  }
  off[n] = (int32_t)succ.size();
  p.succ_off.swap(off);
  p.succ.swap(succ);
  p.indeg[join] = 0;
  return true;
}

extern "C" int stiles_debug_race_check(int nt, int b, int band, int arrow, int which, int plant) {
  const int kind = which & 15, prec = (which >> 4) & 15, tune = (which >> 8) & 255, sel0 = which >> 16;
  if (kind < 0 || kind > 2 || prec > PREC_FP32X || !tune_valid(tune) || nt < 1 || b < 1 || band < 0 || arrow < 0 ||
      plant < 0 || plant > 2)
    return STILES_ERR_INVALID_ARG;
  const Shape sh{nt, b, band < nt - 1 ? band : nt - 1, arrow, prec, tune, sel0};
  Plan p;
  const int rc = build_plan(sh, (PlanKind)kind, 304, &p);
  if (rc) return rc;
  if (plant == 2) {
    if (!plant_unjoined_column(p)) return STILES_ERR_INVALID_ARG;
    return race_check_plan(p, Layout(sh).doubles(), 0);
  }
  return race_check_plan(p, Layout(sh).doubles(), plant);
}

extern "C" int stiles_debug_race_check_serve(int nt, int b, int band, int arrow, int precision, int tuning, int plant) {
  if (nt < 1 || b < 1 || band < 0 || arrow < 0 || precision < 0 || precision > PREC_FP32X || !tune_valid(tuning) ||
      plant < 0 || plant > 1)
    return STILES_ERR_INVALID_ARG;
  const Shape sh{nt, b, band < nt - 1 ? band : nt - 1, arrow, precision, tuning};
  Plan p;
  const int rc = build_serve_template(sh, 304, &p);
  return rc ? rc : race_check_plan(p, Layout(sh).doubles(), plant, true);
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

// ------------------------------------------------------------------ batch --

struct stiles_batch {
  int count = 0;
  int device = 0;
  int sms = 0;
  int grid = 0;
  int prec = 0;
  long long budget_ns = 60LL * 1000 * 1000 * 1000;
  std::vector<Shape> shapes;
  std::vector<int64_t> off;        // count + 1 offsets (doubles)
  std::vector<int32_t> diag_base;  // count + 1 POTRF slot ranges
  std::vector<int64_t> slot_gcol;  // per POTRF slot: global column of its block's first pivot
  Plan plan;
  DevPlan dev;
  DevStatus* dstatus = nullptr;
  double* dlogdet = nullptr;
  int32_t* dbad = nullptr;
  int ndiag = 0;
  size_t w_bytes = 0, ctr_offset = 0, scratch_bytes = 0;
  cudaStream_t last_stream = nullptr;
  bool launched = false;
  // graph of one launch, valid for the buffer pointers it was built with
  KParams kp{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[6] = {};
};

static void free_batch(stiles_batch* h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  cudaFree(h->dev.tasks);
  cudaFree(h->dev.segs);
  cudaFree(h->dev.succ_off);
  cudaFree(h->dev.succ);
  cudaFree(h->dev.bcap);
  cudaFree(h->dev.image);
  cudaFree(h->dstatus);
  cudaFree(h->dlogdet);
  cudaFree(h->dbad);
  delete h;
}

extern "C" int stiles_batch_create(int count, const int* nt, const int* b, const int* band, const int* arrow,
                                   int precision, const int* tuning, stiles_batch_t* out) {
  if (!out) return STILES_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !nt || !b || !band || !arrow) return STILES_ERR_INVALID_ARG;
  if (precision != STILES_FP64 && precision != STILES_EMU64 && precision != STILES_FP32X) return STILES_ERR_UNSUPPORTED;
  stiles_batch* h = new (std::nothrow) stiles_batch();
  if (!h) return STILES_ERR_OOM;
  h->count = count;
  h->prec = precision;
  h->off.assign(count + 1, 0);
  for (int m = 0; m < count; ++m) {
    const int tune = tuning ? tuning[m] : 0;
    if (nt[m] < 1 || b[m] < 1 || band[m] < 0 || arrow[m] < 0 || !tune_valid(tune)) {
      delete h;
      return STILES_ERR_INVALID_ARG;
    }
    const Shape s{nt[m], b[m], band[m] < nt[m] - 1 ? band[m] : nt[m] - 1, arrow[m], precision, tune};
    h->shapes.push_back(s);
    h->off[m + 1] = (int64_t)align_up((size_t)(h->off[m] + Layout(s).doubles()), 32);
  }
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return STILES_ERR_CUDA;
  }
  h->grid = h->sms * kCtasPerSm;
  std::vector<int64_t> base(h->off.begin(), h->off.end() - 1);
  int rc = build_batch_plan(h->shapes, base, h->grid, &h->plan, &h->diag_base);
  if (rc) {
    delete h;
    return rc;
  }
  Plan& p = h->plan;
  rc = upload(p.tasks, &h->dev.tasks);
  if (!rc) rc = upload(p.segs, &h->dev.segs);
  if (!rc) rc = upload(p.succ_off, &h->dev.succ_off);
  if (!rc) rc = upload(p.succ, &h->dev.succ);
  if (!rc) rc = upload(p.bcap, &h->dev.bcap);
  {
    std::vector<int32_t> img = sched_image(p);
    if (!rc) rc = upload(img, &h->dev.image);
    h->dev.image_ints = img.size();
  }
  h->dev.ntasks = (int)p.tasks.size();
  h->dev.nbuckets = p.nbuckets;
  h->dev.ucap = p.urgent_parts;
  h->ndiag = p.ndiag;
  if (!rc) rc = dev_malloc((void**)&h->dstatus, sizeof(DevStatus));
  if (!rc) rc = dev_malloc((void**)&h->dlogdet, sizeof(double) * (h->ndiag > 0 ? h->ndiag : 1));
  if (!rc) rc = dev_malloc((void**)&h->dbad, sizeof(int32_t) * (h->ndiag > 0 ? h->ndiag : 1));
  if (!rc && configure_persistent() != cudaSuccess) rc = STILES_ERR_CUDA;
  if (rc) {
    free_batch(h);
    return rc;
  }
  h->slot_gcol.assign(h->ndiag, 0);
  for (const Task& tk : p.tasks)
    if (tk.op == OP_POTRF && tk.diag >= 0 && tk.diag < h->ndiag) h->slot_gcol[tk.diag] = tk.gcol;
  // the task table is on the device; keep only what the host reads later
  p.tasks.clear(); p.tasks.shrink_to_fit();
  p.segs.clear(); p.segs.shrink_to_fit();
  p.waits.clear(); p.waits.shrink_to_fit();
  p.sigs.clear(); p.sigs.shrink_to_fit();
  p.succ.clear(); p.succ.shrink_to_fit();
  p.succ_off.clear(); p.succ_off.shrink_to_fit();
  p.slots0.clear(); p.slots0.shrink_to_fit();
  h->w_bytes = align_up((size_t)h->off[count] * sizeof(double), 256);
  h->ctr_offset = h->w_bytes;
  h->scratch_bytes = align_up(h->ctr_offset + sizeof(int) * h->dev.image_ints, 256);
  *out = h;
  return STILES_OK;
}

extern "C" int stiles_batch_offsets(stiles_batch_t h, size_t* off) {
  if (!h || !off) return STILES_ERR_INVALID_ARG;
  for (int m = 0; m <= h->count; ++m) off[m] = (size_t)h->off[m];
  return STILES_OK;
}

extern "C" int stiles_batch_workspace_bytes(stiles_batch_t h, size_t* buffer_bytes, size_t* scratch_bytes) {
  if (!h) return STILES_ERR_INVALID_ARG;
  if (buffer_bytes) *buffer_bytes = (size_t)h->off[h->count] * sizeof(double);
  if (scratch_bytes) *scratch_bytes = h->scratch_bytes;
  return STILES_OK;
}

// Graph of one batch launch: reset the scheduler state (copy of the initial
// image), the status block (zero, then "no failing column") and the pivot
// slots (-1), then the persistent kernel.
static int build_batch_graph(stiles_batch* h, const double* A, double* L, double* S, void* scratch) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  char* scr = (char*)scratch;
  int* state = (int*)(scr + h->ctr_offset);
  KParams& p = h->kp;
  p = KParams{};
  p.tasks = h->dev.tasks;
  p.segs = h->dev.segs;
  p.succ_off = h->dev.succ_off;
  p.succ = h->dev.succ;
  p.bcap = h->dev.bcap;
  p.ntasks = h->dev.ntasks;
  p.nbuckets = h->dev.nbuckets;
  p.ucap = h->dev.ucap;
  p.q = sched_state_at(state, h->dev.ntasks, h->dev.nbuckets, h->dev.ucap);
  p.st = h->dstatus;
  p.logdet_part = h->dlogdet;
  p.badpiv = h->dbad;
  p.buf[BUF_A] = const_cast<double*>(A);
  p.buf[BUF_L] = L;
  p.buf[BUF_S] = S;
  p.buf[BUF_W] = (double*)scr;
  p.budget_ns = h->budget_ns;
  p.use_tc = h->prec != PREC_FP64;
  p.trace = nullptr;
  p.buf_len = h->off[h->count];
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return STILES_ERR_CUDA;
  std::vector<cudaGraphNode_t> deps;
  cudaGraphNode_t n = nullptr;
  bool ok = true;
  if (h->dev.image_ints) {
    ok = ok && cudaGraphAddMemcpyNode1D(&n, g, nullptr, 0, state, h->dev.image, sizeof(int) * h->dev.image_ints,
                                        cudaMemcpyDeviceToDevice) == cudaSuccess;
    deps.push_back(n);
  }
  cudaMemsetParams ms{};
  ms.dst = h->dstatus;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = sizeof(DevStatus) / 4;
  ms.height = 1;
  cudaGraphNode_t n_status = nullptr;
  ok = ok && cudaGraphAddMemsetNode(&n_status, g, nullptr, 0, &ms) == cudaSuccess;
  cudaMemsetParams ms2{};
  ms2.dst = &h->dstatus->spd_col;
  ms2.value = 0xffffffffu;
  ms2.elementSize = 4;
  ms2.width = sizeof(unsigned long long) / 4;
  ms2.height = 1;
  ok = ok && cudaGraphAddMemsetNode(&n, g, &n_status, 1, &ms2) == cudaSuccess;
  deps.push_back(n);
  if (h->ndiag > 0) {
    cudaMemsetParams ms3{};
    ms3.dst = h->dbad;
    ms3.value = 0xffffffffu;
    ms3.elementSize = 4;
    ms3.width = (size_t)h->ndiag;
    ms3.height = 1;
    ok = ok && cudaGraphAddMemsetNode(&n, g, nullptr, 0, &ms3) == cudaSuccess;
    deps.push_back(n);
  }
  if (h->dev.ntasks > 0) {
    void* args[1] = {&h->kp};
    cudaKernelNodeParams kn{};
    kn.func = const_cast<void*>(persistent_kernel_ptr(h->kp.use_tc != 0));
    kn.gridDim = dim3((unsigned)h->grid);
    kn.blockDim = dim3((unsigned)kernel_threads());
    kn.sharedMemBytes = (unsigned)kernel_smem_bytes(h->kp.use_tc != 0);
    kn.kernelParams = args;
    ok = ok && cudaGraphAddKernelNode(&n, g, deps.data(), deps.size(), &kn) == cudaSuccess;
  }
  cudaGraphExec_t ex = nullptr;
  ok = ok && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (!ok) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    return STILES_ERR_CUDA;
  }
  h->graph = g;
  h->gexec = ex;
  return STILES_OK;
}

extern "C" int stiles_batch_factor_selinv(stiles_batch_t h, const double* A, double* L, double* S, void* scratch,
                                          void* stream) {
  if (!h || !A || !L || !S || !scratch || S == L || (const double*)S == A || (void*)S == scratch)
    return STILES_ERR_INVALID_ARG;
  if (((uintptr_t)scratch) % 256 != 0) return STILES_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  const void* key[6] = {A, L, S, scratch, (const void*)(intptr_t)h->grid, (const void*)(intptr_t)h->budget_ns};
  if (!h->gexec || memcmp(key, h->gkey, sizeof(key)) != 0) {
    const int rc = build_batch_graph(h, A, L, S, scratch);
    if (rc) return rc;
    memcpy(h->gkey, key, sizeof(key));
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaGraphLaunch(h->gexec, st) != cudaSuccess) return STILES_ERR_CUDA;
  h->last_stream = st;
  h->launched = true;
  return STILES_OK;
}

static int batch_sync(stiles_batch_t h, DevStatus* ds) {
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return STILES_ERR_CUDA;
  if (cudaMemcpy(ds, h->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess) return STILES_ERR_CUDA;
  return STILES_OK;
}

// First failing global column (0-based) of matrix m, or -1.
static long long batch_bad_column(stiles_batch_t h, const std::vector<int32_t>& bad, int m) {
  long long best = -1;
  for (int q = h->diag_base[m]; q < h->diag_base[m + 1]; ++q)
    if (bad[q] >= 0) {
      const long long col = h->slot_gcol[q] + bad[q];
      if (best < 0 || col < best) best = col;
    }
  return best;
}

extern "C" int stiles_batch_status(stiles_batch_t h, int index, int* code, long long* info) {
  if (!h || index < 0 || index >= h->count) return STILES_ERR_INVALID_ARG;
  if (!h->launched) {
    if (code) *code = STILES_OK;
    if (info) *info = 0;
    return STILES_OK;
  }
  DevStatus ds;
  int rc = batch_sync(h, &ds);
  if (rc) return rc;
  int c = code_of(ds);
  long long inf = c == STILES_OK || c == STILES_ERR_NOT_SPD ? 0 : (long long)ds.info;
  if (c == STILES_OK || c == STILES_ERR_NOT_SPD) {
    const int n = h->diag_base[index + 1] - h->diag_base[index];
    std::vector<int32_t> bad(h->ndiag, -1);
    if (n > 0 && cudaMemcpy(bad.data() + h->diag_base[index], h->dbad + h->diag_base[index], sizeof(int32_t) * n,
                            cudaMemcpyDeviceToHost) != cudaSuccess)
      return STILES_ERR_CUDA;
    const long long col = batch_bad_column(h, bad, index);
    c = col >= 0 ? STILES_ERR_NOT_SPD : STILES_OK;
    inf = col >= 0 ? col + 1 : 0;
  }
  if (code) *code = c;
  if (info) *info = inf;
  return STILES_OK;
}

extern "C" int stiles_batch_logdet(stiles_batch_t h, double* out_host) {
  if (!h || !out_host || !h->launched) return STILES_ERR_INVALID_ARG;
  DevStatus ds;
  int rc = batch_sync(h, &ds);
  if (rc) return rc;
  const int c = code_of(ds);
  if (c != STILES_OK && c != STILES_ERR_NOT_SPD) return c;
  std::vector<double> part(h->ndiag > 0 ? h->ndiag : 1);
  std::vector<int32_t> bad(h->ndiag > 0 ? h->ndiag : 1, -1);
  if (h->ndiag > 0 &&
      (cudaMemcpy(part.data(), h->dlogdet, sizeof(double) * h->ndiag, cudaMemcpyDeviceToHost) != cudaSuccess ||
       cudaMemcpy(bad.data(), h->dbad, sizeof(int32_t) * h->ndiag, cudaMemcpyDeviceToHost) != cudaSuccess))
    return STILES_ERR_CUDA;
  for (int m = 0; m < h->count; ++m) {
    double acc = 0.0;
    bool spd = true;
    for (int q = h->diag_base[m]; q < h->diag_base[m + 1]; ++q) {
      acc += part[q];  // fixed order: tile column, then block (as for one matrix)
      spd = spd && bad[q] < 0;
    }
    out_host[m] = spd ? 2.0 * acc : __builtin_nan("");
  }
  return STILES_OK;
}

extern "C" int stiles_batch_set_option(stiles_batch_t h, int option, long long value) {
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
    default:
      return STILES_ERR_INVALID_ARG;
  }
}

extern "C" int stiles_batch_stats(stiles_batch_t h, long long stats[9]) {
  if (!h || !stats) return STILES_ERR_INVALID_ARG;
  stats[0] = h->dev.ntasks;
  stats[1] = 0;
  stats[2] = 0;
  stats[3] = h->plan.nctr;
  stats[4] = (long long)h->plan.flops;
  stats[5] = h->plan.tile_gemms;
  stats[6] = (long long)h->plan.cp_ns;
  stats[7] = (long long)h->plan.makespan_ns;
  stats[8] = (long long)h->plan.flops_lowered;
  return STILES_OK;
}

extern "C" int stiles_batch_destroy(stiles_batch_t h) {
  if (!h) return STILES_ERR_INVALID_ARG;
  if (h->launched) {
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->last_stream);
  }
  free_batch(h);
  return STILES_OK;
}

extern "C" int stiles_debug_validate_batch(int count, const int* nt, const int* b, const int* band, const int* arrow,
                                           int precision, const int* tuning) {
  if (count < 1 || !nt || !b || !band || !arrow || precision < 0 || precision > PREC_FP32X) return STILES_ERR_INVALID_ARG;
  std::vector<Shape> shapes;
  std::vector<int64_t> base;
  int64_t off = 0;
  for (int m = 0; m < count; ++m) {
    const int tune = tuning ? tuning[m] : 0;
    if (nt[m] < 1 || b[m] < 1 || band[m] < 0 || arrow[m] < 0 || !tune_valid(tune)) return STILES_ERR_INVALID_ARG;
    shapes.push_back(Shape{nt[m], b[m], band[m] < nt[m] - 1 ? band[m] : nt[m] - 1, arrow[m], precision, tune});
    base.push_back(off);
    off = (int64_t)align_up((size_t)(off + Layout(shapes.back()).doubles()), 32);
  }
  Plan p;
  std::vector<int32_t> diag_base;
  const int rc = build_batch_plan(shapes, base, 304, &p, &diag_base);
  return rc ? rc : validate_plan_len(p, off, PLAN_FUSED);
}

extern "C" int stiles_debug_race_check_batch(int count, const int* nt, const int* b, const int* band, const int* arrow,
                                             int precision, const int* tuning, int plant) {
  if (count < 1 || !nt || !b || !band || !arrow || precision < 0 || precision > PREC_FP32X || plant < 0 || plant > 1)
    return STILES_ERR_INVALID_ARG;
  std::vector<Shape> shapes;
  std::vector<int64_t> base;
  int64_t off = 0;
  for (int m = 0; m < count; ++m) {
    const int tune = tuning ? tuning[m] : 0;
    if (nt[m] < 1 || b[m] < 1 || band[m] < 0 || arrow[m] < 0 || !tune_valid(tune)) return STILES_ERR_INVALID_ARG;
    shapes.push_back(Shape{nt[m], b[m], band[m] < nt[m] - 1 ? band[m] : nt[m] - 1, arrow[m], precision, tune});
    base.push_back(off);
    off = (int64_t)align_up((size_t)(off + Layout(shapes.back()).doubles()), 32);
  }
  Plan p;
  std::vector<int32_t> diag_base;
  const int rc = build_batch_plan(shapes, base, 304, &p, &diag_base);
  return rc ? rc : race_check_plan(p, off, plant);
}

extern "C" int stiles_debug_validate_serve(int nt, int b, int band, int arrow, int precision, int tuning) {
  if (nt < 1 || b < 1 || band < 0 || arrow < 0 || precision < 0 || precision > PREC_FP32X || !tune_valid(tuning))
    return STILES_ERR_INVALID_ARG;
  const Shape sh{nt, b, band < nt - 1 ? band : nt - 1, arrow, precision, tuning};
  Plan p;
  const int rc = build_serve_template(sh, 304, &p);
  if (rc) return rc;
  int roots_prep = 0, roots = 0;
  for (size_t t = 0; t < p.tasks.size(); ++t)
    if (p.indeg[t] == 0) {
      ++roots;
      roots_prep += p.tasks[t].op == OP_PREP;
    }
  if (roots == 0 || roots != roots_prep) return STILES_ERR_PLAN;  // the PREP tasks are the only roots
  return validate_plan_len(p, Layout(sh).doubles(), PLAN_FUSED);
}
