// Request server (include/stiles.h, "server"): one persistent kernel keeps
// running while requests of different shapes arrive. Each request gets device
// memory for its L (A is built in place), Sigma and scratch from a first-fit
// arena (admission by HBM footprint), a relocated copy of its shape's task
// table, and a request slot; the host then posts an activation record in a
// host-mapped inbox, and an idle worker of the running kernel pushes the
// request's root tasks into the shared ready rings. Requests admitted while
// others run therefore share the GPU task by task (continuous batching). The
// last task of a request writes the request's sequence number to host-mapped
// memory; the host reads the results with copies on a second stream while the
// kernel keeps running. While the kernel runs, every transfer is a plain
// host<->device copy (copy engine): nothing may need an SM.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/stiles.h"
#include "plan.h"
#include "stiles_device.h"

using namespace stiles;

namespace {

// First-fit allocator over [0, cap) (units of the arena's element).
class FirstFit {
 public:
  void reset(int64_t cap) {
    free_.clear();
    if (cap > 0) free_[0] = cap;
  }
  int64_t alloc(int64_t n, int64_t align) {
    if (n <= 0) n = 1;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      const int64_t start = (it->first + align - 1) / align * align;
      const int64_t end = it->first + it->second;
      if (start + n <= end) {
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (start > off) free_[off] = start - off;
        if (start + n < end) free_[start + n] = end - (start + n);
        return start;
      }
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    if (n <= 0) n = 1;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<int64_t, int64_t> free_;
};

struct ShapeT {
  Shape s;
  Plan plan;
  int64_t doubles = 0;  // packed layout
  int64_t n = 0;        // matrix order
  std::vector<int32_t> roots;
  int64_t base_off = 0;  // in the base arena: values, then rb (n), ra (n)
  bool base_set = false;
};

struct Req {
  bool live = false, done = false;
  int shape = -1;
  long long tag = 0;
  unsigned seq = 0;
  int64_t dL = -1, dS = -1, dW = -1;  // data arena offsets (doubles)
  int64_t t0 = -1, g0 = -1, s0 = -1, d0 = -1, r0 = -1;
  int64_t nt = 0, ng = 0, ns = 0, nd = 0, nr = 0;
};

// A failed allocation is reported as STILES_ERR_OOM and its error cleared
// from the runtime's last-error slot (a later launch check must not see it).
template <typename T>
int dmalloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  if (cudaMalloc((void**)p, sizeof(T) * (size_t)n) == cudaSuccess) return 0;
  *p = nullptr;
  cudaGetLastError();
  return STILES_ERR_OOM;
}

inline int host_alloc(void** p, size_t bytes, unsigned flags) {
  if (cudaHostAlloc(p, bytes, flags) == cudaSuccess) return 0;
  *p = nullptr;
  cudaGetLastError();
  return STILES_ERR_OOM;
}

inline int64_t reloc(int64_t ref, int64_t add) { return ref < 0 ? ref : ref + add; }
inline int64_t rebuf(int64_t ref, int buf, int64_t add) {
  return ref < 0 ? ref : mkref(buf, (ref & OFF_MASK) + add);
}

}  // namespace

struct stiles_server {
  int device = 0, sms = 0, grid = 0, prec = 0;
  std::vector<ShapeT> shapes;
  // device arenas
  double* base = nullptr;
  int64_t base_doubles = 0;
  double* data = nullptr;
  int64_t data_doubles = 0;
  Task* tasks = nullptr;
  int32_t *succ_off = nullptr, *rem = nullptr, *pdone = nullptr, *treq = nullptr;
  int64_t task_cap = 0;
  Seg* segs = nullptr;
  int64_t seg_cap = 0;
  int32_t* succ = nullptr;
  int64_t succ_cap = 0;
  double* logdet = nullptr;
  int32_t* badpiv = nullptr;
  int64_t diag_cap = 0;
  int32_t* roots = nullptr;
  int64_t root_cap = 0;
  int32_t* req_left = nullptr;
  unsigned* req_seq = nullptr;
  double* req_param = nullptr;
  int* inbox_seen = nullptr;
  int* ring_slots = nullptr;
  int* ring_ctr = nullptr;
  unsigned ring_mask = 0;
  DevStatus* dstatus = nullptr;
  ServeCtl* ctl_host = nullptr;
  ServeCtl* ctl_dev = nullptr;
  FirstFit data_ff, task_ff, seg_ff, succ_ff, diag_ff, root_ff;
  std::vector<Req> reqs;
  std::vector<int> free_slots;
  int max_req = 0;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  bool running = false;
  unsigned next_seq = 1;
  int posted = 0;
  long long budget_ns = 20LL * 1000 * 1000 * 1000;
  // pinned staging of one request's relocated tables
  char* stage = nullptr;
  size_t stage_bytes = 0;
};

static void free_server(stiles_server* h) {
  if (!h) return;
  cudaFree(h->base);
  cudaFree(h->data);
  cudaFree(h->tasks);
  cudaFree(h->succ_off);
  cudaFree(h->rem);
  cudaFree(h->pdone);
  cudaFree(h->treq);
  cudaFree(h->segs);
  cudaFree(h->succ);
  cudaFree(h->logdet);
  cudaFree(h->badpiv);
  cudaFree(h->roots);
  cudaFree(h->req_left);
  cudaFree(h->req_seq);
  cudaFree(h->req_param);
  cudaFree(h->inbox_seen);
  cudaFree(h->ring_slots);
  cudaFree(h->ring_ctr);
  cudaFree(h->dstatus);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->stage) cudaFreeHost(h->stage);
  if (h->kstream) cudaStreamDestroy(h->kstream);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  delete h;
}

extern "C" int stiles_server_create(int nshapes, const int* nt, const int* b, const int* band, const int* arrow,
                                    int precision, const int* tuning, size_t data_bytes, int max_requests,
                                    stiles_server_t* out) {
  if (!out) return STILES_ERR_INVALID_ARG;
  *out = nullptr;
  if (nshapes < 1 || !nt || !b || !band || !arrow || max_requests < 1 || max_requests > kServeMaxReq)
    return STILES_ERR_INVALID_ARG;
  if (precision != STILES_FP64 && precision != STILES_EMU64 && precision != STILES_FP32X) return STILES_ERR_UNSUPPORTED;
  stiles_server* h = new (std::nothrow) stiles_server();
  if (!h) return STILES_ERR_OOM;
  h->prec = precision;
  h->max_req = max_requests;
  int64_t max_tasks = 0, max_segs = 0, max_succ = 0, max_diag = 0, max_roots = 0;
  for (int m = 0; m < nshapes; ++m) {
    const int tune = tuning ? tuning[m] : 0;
    if (nt[m] < 1 || b[m] < 1 || band[m] < 0 || arrow[m] < 0 || !tune_valid(tune)) {
      delete h;
      return STILES_ERR_INVALID_ARG;
    }
    ShapeT T;
    T.s = Shape{nt[m], b[m], band[m] < nt[m] - 1 ? band[m] : nt[m] - 1, arrow[m], precision, tune};
    int rc = build_serve_template(T.s, 304, &T.plan);
    if (rc) {
      delete h;
      return rc;
    }
    T.doubles = Layout(T.s).doubles();
    T.n = (int64_t)nt[m] * b[m] + arrow[m];
    for (size_t t = 0; t < T.plan.tasks.size(); ++t)
      if (T.plan.indeg[t] == 0) T.roots.push_back((int32_t)t);
    T.base_off = h->base_doubles;
    h->base_doubles += (T.doubles + 2 * T.n + 31) / 32 * 32;
    max_tasks = std::max<int64_t>(max_tasks, (int64_t)T.plan.tasks.size() + 1);
    max_segs = std::max<int64_t>(max_segs, (int64_t)T.plan.segs.size());
    max_succ = std::max<int64_t>(max_succ, (int64_t)T.plan.succ.size());
    max_diag = std::max<int64_t>(max_diag, (int64_t)T.plan.ndiag);
    max_roots = std::max<int64_t>(max_roots, (int64_t)T.roots.size());
    h->shapes.push_back(std::move(T));
  }
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return STILES_ERR_CUDA;
  }
  h->grid = h->sms * kCtasPerSm;
  // table arenas: room for max_requests of the largest shape, capped by 4 of them at least
  const int64_t k = std::max(4, max_requests);
  h->task_cap = std::min<int64_t>(k * max_tasks, (int64_t)1 << 28);
  h->seg_cap = k * std::max<int64_t>(max_segs, 1);
  h->succ_cap = k * std::max<int64_t>(max_succ, 1);
  h->diag_cap = k * std::max<int64_t>(max_diag, 1);
  h->root_cap = k * std::max<int64_t>(max_roots, 1);
  h->data_doubles = (int64_t)(data_bytes / sizeof(double));
  unsigned ring = 1;
  while ((int64_t)ring < 4 * h->task_cap && ring < (1u << 30)) ring <<= 1;
  h->ring_mask = ring - 1;
  int rc = 0;
  if (!rc) rc = dmalloc(&h->base, h->base_doubles);
  if (!rc) rc = dmalloc(&h->data, h->data_doubles);
  if (!rc) rc = dmalloc(&h->tasks, h->task_cap);
  if (!rc) rc = dmalloc(&h->succ_off, h->task_cap);
  if (!rc) rc = dmalloc(&h->rem, h->task_cap);
  if (!rc) rc = dmalloc(&h->pdone, h->task_cap);
  if (!rc) rc = dmalloc(&h->treq, h->task_cap);
  if (!rc) rc = dmalloc(&h->segs, h->seg_cap);
  if (!rc) rc = dmalloc(&h->succ, h->succ_cap);
  if (!rc) rc = dmalloc(&h->logdet, h->diag_cap);
  if (!rc) rc = dmalloc(&h->badpiv, h->diag_cap);
  if (!rc) rc = dmalloc(&h->roots, h->root_cap);
  if (!rc) rc = dmalloc(&h->req_left, kServeMaxReq);
  if (!rc) rc = dmalloc(&h->req_seq, kServeMaxReq);
  if (!rc) rc = dmalloc(&h->req_param, 2 * kServeMaxReq);
  if (!rc) rc = dmalloc(&h->inbox_seen, 1);
  if (!rc) rc = dmalloc(&h->ring_slots, 3 * (int64_t)ring);
  if (!rc) rc = dmalloc(&h->ring_ctr, 3 * 32);
  if (!rc) rc = dmalloc(&h->dstatus, 1);
  if (!rc) rc = host_alloc((void**)&h->ctl_host, sizeof(ServeCtl), cudaHostAllocMapped);
  if (!rc && cudaHostGetDevicePointer((void**)&h->ctl_dev, h->ctl_host, 0) != cudaSuccess) rc = STILES_ERR_CUDA;
  if (!rc) {
    h->stage_bytes = (size_t)max_tasks * (sizeof(Task) + 5 * sizeof(int32_t) + 4) + (size_t)max_segs * sizeof(Seg) +
                     (size_t)max_succ * sizeof(int32_t) + (size_t)max_roots * sizeof(int32_t) +
                     (size_t)max_diag * sizeof(int32_t) + 4096;
    rc = host_alloc((void**)&h->stage, h->stage_bytes, cudaHostAllocDefault);
  }
  if (!rc && (cudaStreamCreateWithFlags(&h->kstream, cudaStreamNonBlocking) != cudaSuccess ||
              cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) != cudaSuccess))
    rc = STILES_ERR_CUDA;
  if (!rc && configure_persistent() != cudaSuccess) rc = STILES_ERR_CUDA;
  if (rc) {
    free_server(h);
    return rc;
  }
  memset(h->ctl_host, 0, sizeof(ServeCtl));
  h->data_ff.reset(h->data_doubles);
  h->task_ff.reset(h->task_cap);
  h->seg_ff.reset(h->seg_cap);
  h->succ_ff.reset(h->succ_cap);
  h->diag_ff.reset(h->diag_cap);
  h->root_ff.reset(h->root_cap);
  h->reqs.assign(max_requests, Req{});
  for (int q = max_requests - 1; q >= 0; --q) h->free_slots.push_back(q);
  *out = h;
  return STILES_OK;
}

extern "C" int stiles_server_shape_doubles(stiles_server_t h, int shape, size_t* doubles, size_t* n) {
  if (!h || shape < 0 || shape >= (int)h->shapes.size()) return STILES_ERR_INVALID_ARG;
  if (doubles) *doubles = (size_t)h->shapes[shape].doubles;
  if (n) *n = (size_t)h->shapes[shape].n;
  return STILES_OK;
}

extern "C" int stiles_server_set_base(stiles_server_t h, int shape, const double* base, const double* rb,
                                      const double* ra) {
  if (!h || shape < 0 || shape >= (int)h->shapes.size() || !base || !rb || !ra) return STILES_ERR_INVALID_ARG;
  ShapeT& T = h->shapes[shape];
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  double* dst = h->base + T.base_off;
  if (cudaMemcpyAsync(dst, base, sizeof(double) * T.doubles, cudaMemcpyDefault, h->cstream) != cudaSuccess ||
      cudaMemcpyAsync(dst + T.doubles, rb, sizeof(double) * T.n, cudaMemcpyDefault, h->cstream) != cudaSuccess ||
      cudaMemcpyAsync(dst + T.doubles + T.n, ra, sizeof(double) * T.n, cudaMemcpyDefault, h->cstream) != cudaSuccess ||
      cudaStreamSynchronize(h->cstream) != cudaSuccess)
    return STILES_ERR_CUDA;
  T.base_set = true;
  return STILES_OK;
}

extern "C" int stiles_server_start(stiles_server_t h, double window_s) {
  if (!h || h->running || !(window_s > 0)) return STILES_ERR_INVALID_ARG;
  for (const ShapeT& T : h->shapes)
    if (!T.base_set) return STILES_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  cudaStream_t cs = h->cstream;
  const unsigned ring = h->ring_mask + 1;
  if (cudaMemsetAsync(h->ring_slots, 0xff, sizeof(int) * 3 * (size_t)ring, cs) != cudaSuccess ||
      cudaMemsetAsync(h->ring_ctr, 0, sizeof(int) * 3 * 32, cs) != cudaSuccess ||
      cudaMemsetAsync(h->inbox_seen, 0, sizeof(int), cs) != cudaSuccess ||
      cudaMemsetAsync(h->dstatus, 0, sizeof(DevStatus), cs) != cudaSuccess ||
      cudaMemsetAsync(&h->dstatus->spd_col, 0xff, sizeof(unsigned long long), cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return STILES_ERR_CUDA;
  h->ctl_host->stop = 0;
  h->ctl_host->inbox_count = 0;
  h->posted = 0;
  KParams p{};
  p.tasks = h->tasks;
  p.succ_off = h->succ_off;
  p.succ = h->succ;
  p.segs = h->segs;
  p.ntasks = (int)h->task_cap;
  p.q.rem = h->rem;
  p.q.pdone = h->pdone;
  p.st = h->dstatus;
  p.logdet_part = h->logdet;
  p.badpiv = h->badpiv;
  p.buf[BUF_A] = h->base;
  p.buf[BUF_L] = h->data;
  p.buf[BUF_S] = h->data;
  p.buf[BUF_W] = h->data;
  p.budget_ns = h->budget_ns;
  p.buf_len = h->data_doubles;
  p.serve = 1;
  p.use_tc = h->prec != PREC_FP64;
  for (int r = 0; r < 3; ++r) {
    p.sv.ring[r].slots = h->ring_slots + (size_t)r * ring;
    p.sv.ring[r].ctr = h->ring_ctr + 32 * r;
    p.sv.ring[r].mask = h->ring_mask;
  }
  p.sv.ctl = h->ctl_dev;
  p.sv.inbox_seen = h->inbox_seen;
  p.sv.treq = h->treq;
  p.sv.req_left = h->req_left;
  p.sv.req_seq = h->req_seq;
  p.sv.req_param = h->req_param;
  p.sv.roots = h->roots;
  // the window is measured on the device clock from each worker's start
  p.sv.deadline = (unsigned long long)(window_s * 1e9);
  if (launch_persistent(p, h->grid, h->kstream) != cudaSuccess) return STILES_ERR_CUDA;
  h->running = true;
  return STILES_OK;
}

static int submit_impl(stiles_server_t h, int shape, double tau, double rho, const double* A_host, long long tag,
                       int* request);

// Admission and activation of one request (see the file comment).
extern "C" int stiles_server_submit(stiles_server_t h, int shape, double tau, double rho, long long tag,
                                    int* request) {
  if (!(rho == rho) || !(tau == tau)) return STILES_ERR_INVALID_ARG;
  return submit_impl(h, shape, tau, rho, nullptr, tag, request);
}

// A request with explicit values: A_host (host memory, the shape's packed
// layout) is copied into the request's L before activation, and its PREP
// tasks leave it as it is (rho = NaN marks the request).
extern "C" int stiles_server_submit_values(stiles_server_t h, int shape, const double* A_host, long long tag,
                                           int* request) {
  if (!A_host) return STILES_ERR_INVALID_ARG;
  return submit_impl(h, shape, 0.0, __builtin_nan(""), A_host, tag, request);
}

static int submit_impl(stiles_server_t h, int shape, double tau, double rho, const double* A_host, long long tag,
                       int* request) {
  if (!h || !request || shape < 0 || shape >= (int)h->shapes.size()) return STILES_ERR_INVALID_ARG;
  if (!h->running) return STILES_ERR_INVALID_ARG;
  const ShapeT& T = h->shapes[shape];
  const Plan& P = T.plan;
  if (h->free_slots.empty()) return STILES_ERR_BUSY;
  Req R;
  R.shape = shape;
  R.tag = tag;
  R.nt = (int64_t)P.tasks.size() + 1;
  R.ng = (int64_t)P.segs.size();
  R.ns = (int64_t)P.succ.size();
  R.nd = P.ndiag;
  R.nr = (int64_t)T.roots.size();
  const int64_t dbl = (T.doubles + 31) / 32 * 32;
  bool ok = true;
  auto take = [&](FirstFit& ff, int64_t n, int64_t align, int64_t& off) {
    if (!ok) return;
    off = ff.alloc(n, align);
    if (off < 0) ok = false;
  };
  take(h->data_ff, dbl, 32, R.dL);
  take(h->data_ff, dbl, 32, R.dS);
  take(h->data_ff, dbl, 32, R.dW);
  take(h->task_ff, R.nt, 1, R.t0);
  take(h->seg_ff, R.ng, 1, R.g0);
  take(h->succ_ff, R.ns, 1, R.s0);
  take(h->diag_ff, R.nd, 1, R.d0);
  take(h->root_ff, R.nr, 1, R.r0);
  if (!ok) {  // give back what was taken: not admitted now
    if (R.dL >= 0) h->data_ff.release(R.dL, dbl);
    if (R.dS >= 0) h->data_ff.release(R.dS, dbl);
    if (R.dW >= 0) h->data_ff.release(R.dW, dbl);
    if (R.t0 >= 0) h->task_ff.release(R.t0, R.nt);
    if (R.g0 >= 0) h->seg_ff.release(R.g0, R.ng);
    if (R.s0 >= 0) h->succ_ff.release(R.s0, R.ns);
    if (R.d0 >= 0) h->diag_ff.release(R.d0, R.nd);
    if (R.r0 >= 0) h->root_ff.release(R.r0, R.nr);
    return STILES_ERR_BUSY;
  }
  const int slot = h->free_slots.back();
  h->free_slots.pop_back();
  R.seq = h->next_seq++;
  R.live = true;
  // relocated tables in the pinned staging area
  const int64_t n = (int64_t)P.tasks.size();
  char* st = h->stage;
  Task* tk = (Task*)st;
  st += sizeof(Task) * n;
  Seg* sg = (Seg*)st;
  st += sizeof(Seg) * R.ng;
  int32_t* so = (int32_t*)st;
  st += sizeof(int32_t) * (n + 1);
  int32_t* sc = (int32_t*)st;
  st += sizeof(int32_t) * R.ns;
  int32_t* rm = (int32_t*)st;
  st += sizeof(int32_t) * n;
  int32_t* tq = (int32_t*)st;
  st += sizeof(int32_t) * n;
  int32_t* rt = (int32_t*)st;
  st += sizeof(int32_t) * R.nr;
  int32_t* zero = (int32_t*)st;  // pdone
  st += sizeof(int32_t) * n;
  int32_t* minus1 = (int32_t*)st;  // pivot slots
  st += sizeof(int32_t) * R.nd;
  int32_t* left = (int32_t*)st;
  memset(zero, 0, sizeof(int32_t) * n);
  for (int64_t q = 0; q < R.nd; ++q) minus1[q] = -1;
  const int64_t base = T.base_off;
  for (int64_t t = 0; t < n; ++t) {
    Task x = P.tasks[t];
    if (x.op == OP_PREP) {
      x.out = reloc(x.out, R.dL);
      x.cin = reloc(x.cin, base);
      x.aux = reloc(x.aux, base);
    } else {
      auto fix = [&](int64_t ref) {
        if (ref < 0) return ref;
        switch ((int)(ref >> BUF_SHIFT)) {
          case BUF_A: return rebuf(ref, BUF_L, R.dL);  // A is built in place in L
          case BUF_L: return reloc(ref, R.dL);
          case BUF_S: return reloc(ref, R.dS);
          default: return reloc(ref, R.dW);
        }
      };
      x.out = fix(x.out);
      x.cin = fix(x.cin);
      x.aux = fix(x.aux);
      if (x.diag >= 0) x.diag += (int32_t)R.d0;
    }
    x.seg0 += (int32_t)R.g0;
    tk[t] = x;
    so[t] = P.succ_off[t] + (int32_t)R.s0;
    rm[t] = P.indeg[t];
    tq[t] = slot;
  }
  so[n] = P.succ_off[n] + (int32_t)R.s0;
  for (int64_t g = 0; g < R.ng; ++g) {
    Seg x = P.segs[g];
    auto fix = [&](int64_t ref) {
      switch ((int)(ref >> BUF_SHIFT)) {
        case BUF_A: return rebuf(ref, BUF_L, R.dL);
        case BUF_L: return reloc(ref, R.dL);
        case BUF_S: return reloc(ref, R.dS);
        default: return reloc(ref, R.dW);
      }
    };
    x.a = fix(x.a);
    x.b = fix(x.b);
    sg[g] = x;
  }
  for (int64_t e = 0; e < R.ns; ++e) sc[e] = P.succ[e] + (int32_t)R.t0;
  for (int64_t r = 0; r < R.nr; ++r) rt[r] = T.roots[r] + (int32_t)R.t0;
  *left = (int32_t)n;
  cudaStream_t cs = h->cstream;
  bool cok = cudaSetDevice(h->device) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->tasks + R.t0, tk, sizeof(Task) * n, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  if (R.ng) cok = cok && cudaMemcpyAsync(h->segs + R.g0, sg, sizeof(Seg) * R.ng, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->succ_off + R.t0, so, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, cs) == cudaSuccess;
  if (R.ns) cok = cok && cudaMemcpyAsync(h->succ + R.s0, sc, sizeof(int32_t) * R.ns, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->rem + R.t0, rm, sizeof(int32_t) * n, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  // copy-engine transfers only: a memset may run as a kernel, which would
  // wait behind the running server kernel
  cok = cok && cudaMemcpyAsync(h->pdone + R.t0, zero, sizeof(int32_t) * n, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->treq + R.t0, tq, sizeof(int32_t) * n, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->roots + R.r0, rt, sizeof(int32_t) * R.nr, cudaMemcpyHostToDevice, cs) == cudaSuccess;
  if (R.nd)
    cok = cok && cudaMemcpyAsync(h->badpiv + R.d0, minus1, sizeof(int32_t) * R.nd, cudaMemcpyHostToDevice, cs) ==
                     cudaSuccess;
  cok = cok && cudaMemcpyAsync(h->req_left + slot, left, sizeof(int32_t), cudaMemcpyHostToDevice, cs) == cudaSuccess;
  if (A_host)
    cok = cok && cudaMemcpyAsync(h->data + R.dL, A_host, sizeof(double) * T.doubles, cudaMemcpyHostToDevice, cs) ==
                     cudaSuccess;
  cok = cok && cudaStreamSynchronize(cs) == cudaSuccess;
  if (!cok) return STILES_ERR_CUDA;
  // publish the activation record (the kernel reads it after an acquire of inbox_count)
  ServeRec& rec = h->ctl_host->inbox[h->posted % kServeInbox];
  rec.slot = slot;
  rec.root0 = (int)R.r0;
  rec.nroots = (int)R.nr;
  rec.seq = R.seq;
  rec.rho = rho;
  rec.tau = tau;
  std::atomic_thread_fence(std::memory_order_release);
  __atomic_store_n(&h->ctl_host->inbox_count, ++h->posted, __ATOMIC_RELEASE);
  h->reqs[slot] = R;
  *request = slot;
  return STILES_OK;
}

// Completed requests since the last poll (each reported once).
extern "C" int stiles_server_poll(stiles_server_t h, int max, int* requests, long long* tags, int* n_out) {
  if (!h || !n_out || max < 0 || (max > 0 && (!requests || !tags))) return STILES_ERR_INVALID_ARG;
  int n = 0;
  for (int q = 0; q < h->max_req && n < max; ++q) {
    Req& R = h->reqs[q];
    if (!R.live || R.done) continue;
    const unsigned v = __atomic_load_n(&h->ctl_host->done_seq[q], __ATOMIC_ACQUIRE);
    if (v == R.seq) {
      R.done = true;
      requests[n] = q;
      tags[n] = R.tag;
      ++n;
    }
  }
  *n_out = n;
  return STILES_OK;
}

// Status and logdet of a completed request (copies on the server's copy
// stream; the kernel keeps running).
extern "C" int stiles_server_result(stiles_server_t h, int request, int* code, long long* info, double* logdet) {
  if (!h || request < 0 || request >= h->max_req || !h->reqs[request].live || !h->reqs[request].done)
    return STILES_ERR_INVALID_ARG;
  const Req& R = h->reqs[request];
  std::vector<double> part(R.nd > 0 ? R.nd : 1);
  std::vector<int32_t> bad(R.nd > 0 ? R.nd : 1, -1);
  if (cudaSetDevice(h->device) != cudaSuccess) return STILES_ERR_CUDA;
  if (R.nd > 0 &&
      (cudaMemcpyAsync(part.data(), h->logdet + R.d0, sizeof(double) * R.nd, cudaMemcpyDeviceToHost, h->cstream) !=
           cudaSuccess ||
       cudaMemcpyAsync(bad.data(), h->badpiv + R.d0, sizeof(int32_t) * R.nd, cudaMemcpyDeviceToHost, h->cstream) !=
           cudaSuccess ||
       cudaStreamSynchronize(h->cstream) != cudaSuccess))
    return STILES_ERR_CUDA;
  // first failing column: POTRF slots in emission order of the template
  const ShapeT& T = h->shapes[R.shape];
  long long col = -1;
  double acc = 0.0;
  for (const Task& x : T.plan.tasks)
    if (x.op == OP_POTRF && x.diag >= 0 && x.diag < R.nd && bad[x.diag] >= 0) {
      const long long c = (long long)x.gcol + bad[x.diag];
      if (col < 0 || c < col) col = c;
    }
  for (int64_t q = 0; q < R.nd; ++q) acc += part[q];
  if (code) *code = col >= 0 ? STILES_ERR_NOT_SPD : STILES_OK;
  if (info) *info = col >= 0 ? col + 1 : 0;
  if (logdet) *logdet = col >= 0 ? __builtin_nan("") : 2.0 * acc;
  return STILES_OK;
}

// Sigma of a completed request in the packed layout of its shape: copied to
// host_out (host or device memory), or its device address in *device_ptr.
extern "C" int stiles_server_sigma(stiles_server_t h, int request, double* host_out, const double** device_ptr) {
  if (!h || request < 0 || request >= h->max_req || !h->reqs[request].live || !h->reqs[request].done)
    return STILES_ERR_INVALID_ARG;
  const Req& R = h->reqs[request];
  const double* src = h->data + R.dS;
  if (device_ptr) *device_ptr = src;
  if (host_out) {
    if (cudaSetDevice(h->device) != cudaSuccess ||
        cudaMemcpyAsync(host_out, src, sizeof(double) * h->shapes[R.shape].doubles, cudaMemcpyDefault, h->cstream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->cstream) != cudaSuccess)
      return STILES_ERR_CUDA;
  }
  return STILES_OK;
}

// Frees a completed request's memory, tables and slot.
extern "C" int stiles_server_release(stiles_server_t h, int request) {
  if (!h || request < 0 || request >= h->max_req || !h->reqs[request].live || !h->reqs[request].done)
    return STILES_ERR_INVALID_ARG;
  Req& R = h->reqs[request];
  const int64_t dbl = (h->shapes[R.shape].doubles + 31) / 32 * 32;
  h->data_ff.release(R.dL, dbl);
  h->data_ff.release(R.dS, dbl);
  h->data_ff.release(R.dW, dbl);
  h->task_ff.release(R.t0, R.nt);
  h->seg_ff.release(R.g0, R.ng);
  h->succ_ff.release(R.s0, R.ns);
  h->diag_ff.release(R.d0, R.nd);
  h->root_ff.release(R.r0, R.nr);
  R = Req{};
  h->free_slots.push_back(request);
  return STILES_OK;
}

// Bytes of data memory a request of `shape` takes (L, Sigma, scratch).
extern "C" int stiles_server_request_bytes(stiles_server_t h, int shape, size_t* bytes) {
  if (!h || !bytes || shape < 0 || shape >= (int)h->shapes.size()) return STILES_ERR_INVALID_ARG;
  *bytes = 3 * (size_t)((h->shapes[shape].doubles + 31) / 32 * 32) * sizeof(double);
  return STILES_OK;
}

// Device status of the running (or last) server kernel, read without
// waiting for it: code (STILES_OK / STILES_ERR_TIMEOUT / STILES_ERR_PLAN),
// info of the first error, tasks completed so far.
extern "C" int stiles_server_status(stiles_server_t h, int* code, long long* info, long long* tasks_done) {
  if (!h) return STILES_ERR_INVALID_ARG;
  DevStatus ds;
  if (cudaSetDevice(h->device) != cudaSuccess ||
      cudaMemcpyAsync(&ds, h->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->cstream) != cudaSuccess ||
      cudaStreamSynchronize(h->cstream) != cudaSuccess)
    return STILES_ERR_CUDA;
  if (code) *code = ds.code == STILES_DEV_TIMEOUT ? STILES_ERR_TIMEOUT : ds.code == STILES_DEV_CHECK ? STILES_ERR_PLAN : STILES_OK;
  if (info) *info = (long long)ds.info;
  if (tasks_done) *tasks_done = (long long)ds.done;
  return STILES_OK;
}

// Asks the kernel to stop once idle and waits for it. Returns its status:
// STILES_OK, or STILES_ERR_TIMEOUT if the window ran out (or a wait expired).
extern "C" int stiles_server_stop(stiles_server_t h) {
  if (!h || !h->running) return STILES_ERR_INVALID_ARG;
  __atomic_store_n(&h->ctl_host->stop, 1, __ATOMIC_RELEASE);
  if (cudaSetDevice(h->device) != cudaSuccess || cudaStreamSynchronize(h->kstream) != cudaSuccess)
    return STILES_ERR_CUDA;
  h->running = false;
  DevStatus ds;
  if (cudaMemcpy(&ds, h->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess) return STILES_ERR_CUDA;
  if (ds.code == STILES_DEV_TIMEOUT) return STILES_ERR_TIMEOUT;
  if (ds.code == STILES_DEV_CHECK) return STILES_ERR_PLAN;
  return STILES_OK;
}

extern "C" int stiles_server_destroy(stiles_server_t h) {
  if (!h) return STILES_ERR_INVALID_ARG;
  if (h->running) stiles_server_stop(h);
  free_server(h);
  return STILES_OK;
}
