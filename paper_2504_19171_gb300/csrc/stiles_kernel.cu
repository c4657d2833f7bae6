// Persistent dependency-driven FP64 kernel for tiled Cholesky and two-phase
// selected inversion on GB300 (sm_103a).
//
// One CTA per SM claims tasks in the planner's list-schedule order with an
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

__device__ __forceinline__ int load_acquire(int* a) {
  return cuda::atomic_ref<int, cuda::thread_scope_device>(*a).load(cuda::memory_order_acquire);
}

__device__ __forceinline__ int load_relaxed_flag(int* a) {
  return cuda::atomic_ref<int, cuda::thread_scope_device>(*a).load(cuda::memory_order_relaxed);
}

// Warp 0 waits until every (counter, need) of the task holds. Returns 1, or
// 0 if the launch was aborted or this wait exceeded its time budget.
__device__ int wait_deps(const KParams& p, const Task& tk, int tindex) {
  const int lane = threadIdx.x & 31;
  unsigned long long t0 = 0;
  for (int base = 0; base < tk.nwait; base += 32) {
    const int q = base + lane;
    int ctr = -1, need = 0;
    if (q < tk.nwait) {
      const Wait w = p.waits[tk.wait0 + q];
      ctr = w.ctr;
      need = w.need;
    }
    for (;;) {
      const bool ok = ctr < 0 || load_acquire(p.ctr + ctr) >= need;
      if (__all_sync(0xffffffffu, ok)) break;
      // lane 0 decides for the whole warp, so every lane leaves together
      int stop = 0;
      if (lane == 0) {
        stop = load_relaxed_flag(&p.st->abort);
        const unsigned long long now = gtimer();
        if (t0 == 0) {
          t0 = now;
        } else if (!stop && now - t0 > (unsigned long long)p.budget_ns) {
          if (atomicCAS(&p.st->code, 0, STILES_DEV_TIMEOUT) == 0) p.st->info = (unsigned long long)tindex;
          atomicExch(&p.st->abort, 1);
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return 0;
      __nanosleep(256);
    }
  }
  return 1;
}

// acc[i][j] holds output (row tx + 16 i, column ty + 8 j).
struct Acc {
  double v[4][8];
};

__device__ __forceinline__ void accumulate(const KParams& p, const Task& tk, Acc& acc, double* As, double* Bs) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc.v[i][j] = 0.0;
  const int m = tk.m, n = tk.n;
  for (int s = 0; s < tk.nseg; ++s) {
    const Seg g = p.segs[tk.seg0 + s];
    const double* A = resolve(p, g.a);
    const double* B = resolve(p, g.b);
    const bool ta = g.trans & 1, tb = g.trans & 2;
    for (int k0 = 0; k0 < g.k; k0 += KC) {
      const int kc = min(KC, g.k - k0);
      // stage op(A)[0:m, k0:k0+kc] as As[kk][i] and op(B)[k0:k0+kc, 0:n] as Bs[kk][j]
#pragma unroll 4
      for (int e = tid; e < FB * KC; e += NTHREADS) {
        int i, kk;
        if (!ta) { i = e & (FB - 1); kk = e / FB; } else { kk = e & (KC - 1); i = e / KC; }
        double v = 0.0;
        if (i < m && kk < kc)
          v = __ldcg(ta ? A + (int64_t)(k0 + kk) + (int64_t)i * g.lda : A + (int64_t)i + (int64_t)(k0 + kk) * g.lda);
        As[kk * LDS + i] = v;
      }
#pragma unroll 4
      for (int e = tid; e < FB * KC; e += NTHREADS) {
        int j, kk;
        if (tb) { j = e & (FB - 1); kk = e / FB; } else { kk = e & (KC - 1); j = e / KC; }
        double v = 0.0;
        if (j < n && kk < kc)
          v = __ldcg(tb ? B + (int64_t)j + (int64_t)(k0 + kk) * g.ldb : B + (int64_t)(k0 + kk) + (int64_t)j * g.ldb);
        Bs[kk * LDS + j] = v;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        double a[4], b[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk * LDS + tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = Bs[kk * LDS + ty + 8 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc.v[i][j] = fma(a[i], b[j], acc.v[i][j]);
      }
      __syncthreads();
    }
  }
}

// X[r][c] (r, c < FB) in shared memory with row length LDS.
__device__ __forceinline__ void acc_to_smem(const KParams& p, const Task& tk, const Acc& acc, double* X, bool sub_cin,
                                            double sign) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double* C = sub_cin ? resolve(p, tk.cin) : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = tx + 16 * i, c = ty + 8 * j;
      double v = sign * acc.v[i][j];
      if (sub_cin && r < tk.m && c < tk.n) v = __ldcg(C + r + (int64_t)c * tk.ldc) - acc.v[i][j];
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

__device__ __forceinline__ void store_block(const KParams& p, const Task& tk, const double* X, bool lower_only) {
  double* O = resolve(p, tk.out);
  for (int e = threadIdx.x; e < tk.m * tk.n; e += NTHREADS) {
    const int r = e % tk.m, c = e / tk.m;
    O[r + (int64_t)c * tk.ldo] = (lower_only && r < c) ? 0.0 : X[r * LDS + c];
  }
}

__device__ void run_task(const KParams& p, const Task& tk, double* smem) {
  double* As = smem;            // KC x LDS
  double* Bs = smem + KC * LDS;  // KC x LDS
  double* T = smem;              // FB x LDS, reuses As/Bs after the K-loop
  double* X = smem + 2 * KC * LDS;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m = tk.m, n = tk.n;
  Acc acc;
  if (tk.op != OP_TRTRI) accumulate(p, tk, acc, As, Bs);

  switch (tk.op) {
    case OP_UPD:
    case OP_STORE:
    case OP_NEG: {
      double* O = resolve(p, tk.out);
      const double* C = tk.op == OP_UPD ? resolve(p, tk.cin) : nullptr;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = tx + 16 * i, c = ty + 8 * j;
          if (r < m && c < n) {
            double v = acc.v[i][j];
            if (tk.op == OP_UPD) v = __ldcg(C + r + (int64_t)c * tk.ldc) - v;
            else if (tk.op == OP_NEG) v = -v;
            O[r + (int64_t)c * tk.ldo] = v;
          }
        }
      break;
    }
    case OP_SYMUPD: {
      acc_to_smem(p, tk, acc, X, true, 1.0);
      __syncthreads();
      double* O = resolve(p, tk.out);
      if (tk.flags & 1) {  // diagonal block: keep the lower triangle, mirror it
        for (int e = tid; e < m * n; e += NTHREADS) {
          const int r = e % m, c = e / m;
          O[r + (int64_t)c * tk.ldo] = r >= c ? X[r * LDS + c] : X[c * LDS + r];
        }
      } else {
        double* M = resolve(p, tk.aux);  // mirror block (c, r): n x m
        for (int e = tid; e < m * n; e += NTHREADS) {
          const int r = e % m, c = e / m;
          O[r + (int64_t)c * tk.ldo] = X[r * LDS + c];
        }
        for (int e = tid; e < m * n; e += NTHREADS) {
          const int c = e % n, r = e / n;
          M[c + (int64_t)r * tk.ldx] = X[r * LDS + c];
        }
      }
      break;
    }
    case OP_POTRF: {
      __shared__ double s_dinv;
      __shared__ int s_bad;
      acc_to_smem(p, tk, acc, X, true, 1.0);
      if (tid == 0) s_bad = -1;
      double logsum = 0.0;
      __syncthreads();
      for (int j = 0; j < n; ++j) {
        if (tid == 0) {
          double d = X[j * LDS + j];
          if (!(d > 0.0) && s_bad < 0) s_bad = j;
          d = sqrt(d);
          X[j * LDS + j] = d;
          logsum += log(d);
          s_dinv = 1.0 / d;
        }
        __syncthreads();
        const double dinv = s_dinv;
        for (int r = j + 1 + tid; r < n; r += NTHREADS) X[r * LDS + j] *= dinv;
        __syncthreads();
        const int w = n - j - 1;
        for (int e = tid; e < w * w; e += NTHREADS) {
          const int r = j + 1 + e % w, c = j + 1 + e / w;
          if (c <= r) X[r * LDS + c] -= X[r * LDS + j] * X[c * LDS + j];
        }
        __syncthreads();
      }
      store_block(p, tk, X, true);
      if (tk.zrows > 0) {  // strict upper part of L's diagonal tile in this block column
        double* Z = resolve(p, tk.out) - tk.zrows;
        for (int e = tid; e < tk.zrows * n; e += NTHREADS) Z[e % tk.zrows + (int64_t)(e / tk.zrows) * tk.ldo] = 0.0;
      }
      if (tid == 0) {
        p.logdet_part[tk.diag] = logsum;
        if (s_bad >= 0) {
          atomicCAS(&p.st->code, 0, STILES_DEV_NOT_SPD);
          atomicMin(&p.st->spd_col, (unsigned long long)tk.gcol + (unsigned long long)s_bad);
        }
      }
      break;
    }
    case OP_TRSM_RLT: {  // X = (C - acc) T^{-T}, T lower n x n: solve X T^T = B row-wise
      acc_to_smem(p, tk, acc, X, true, 1.0);
      load_tri(p, tk, n, T);
      __syncthreads();
      for (int j = 0; j < n; ++j) {
        const double dinv = 1.0 / T[j * LDS + j];
        for (int r = tid; r < m; r += NTHREADS) X[r * LDS + j] *= dinv;
        __syncthreads();
        const int w = n - j - 1;
        for (int e = tid; e < m * w; e += NTHREADS) {
          const int r = e % m, c = j + 1 + e / m;
          X[r * LDS + c] -= X[r * LDS + j] * T[c * LDS + j];
        }
        __syncthreads();
      }
      store_block(p, tk, X, false);
      break;
    }
    case OP_TRSM_LLN: {  // X = -T^{-1} acc, T lower m x m
      acc_to_smem(p, tk, acc, X, false, -1.0);
      load_tri(p, tk, m, T);
      __syncthreads();
      for (int j = 0; j < m; ++j) {
        const double dinv = 1.0 / T[j * LDS + j];
        for (int c = tid; c < n; c += NTHREADS) X[j * LDS + c] *= dinv;
        __syncthreads();
        const int w = m - j - 1;
        for (int e = tid; e < n * w; e += NTHREADS) {
          const int c = e % n, r = j + 1 + e / n;
          X[r * LDS + c] -= T[r * LDS + j] * X[j * LDS + c];
        }
        __syncthreads();
      }
      store_block(p, tk, X, false);
      break;
    }
    case OP_TRTRI: {  // X = T^{-1}, T lower m x m: solve T X = I
      load_tri(p, tk, m, T);
      for (int e = tid; e < FB * FB; e += NTHREADS) {
        const int r = e % FB, c = e / FB;
        X[r * LDS + c] = r == c ? 1.0 : 0.0;
      }
      __syncthreads();
      for (int j = 0; j < m; ++j) {
        const double dinv = 1.0 / T[j * LDS + j];
        for (int c = tid; c <= j; c += NTHREADS) X[j * LDS + c] *= dinv;
        __syncthreads();
        const int w = m - j - 1, cw = j + 1;
        for (int e = tid; e < cw * w; e += NTHREADS) {
          const int c = e % cw, r = j + 1 + e / cw;
          X[r * LDS + c] -= T[r * LDS + j] * X[j * LDS + c];
        }
        __syncthreads();
      }
      store_block(p, tk, X, true);
      break;
    }
    default:
      break;
  }
}

__global__ void __launch_bounds__(NTHREADS, 1) persistent_kernel(KParams p) {
  extern __shared__ double smem[];
  __shared__ int s_task, s_ok;
  for (;;) {
    if (threadIdx.x == 0) {
      s_task = load_relaxed_flag(&p.st->abort) ? p.ntasks : atomicAdd(p.claim, 1);
    }
    __syncthreads();
    const int t = s_task;
    if (t >= p.ntasks) break;
    const Task tk = p.tasks[t];
    if (threadIdx.x < 32) {
      const int ok = wait_deps(p, tk, t);
      if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    __threadfence();
    run_task(p, tk, smem);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < tk.nsig; ++q) atomicAdd(p.ctr + p.sigs[tk.sig0 + q], 1);
      atomicAdd(&p.st->done, 1ull);
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
