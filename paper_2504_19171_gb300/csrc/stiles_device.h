// Launch parameters and device status block of the persistent kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"

namespace stiles {

// Device status codes (the host maps them to stiles_status_code).
enum : int { STILES_DEV_OK = 0, STILES_DEV_NOT_SPD = 1, STILES_DEV_TIMEOUT = 2 };

struct DevStatus {
  int code;                    // first error (STILES_DEV_*)
  int abort;                   // set on TIMEOUT: every CTA stops claiming / waiting
  unsigned long long done;     // tasks completed
  unsigned long long info;     // TIMEOUT: index of the task whose wait expired
  unsigned long long spd_col;  // NOT_SPD: smallest failing global column (0-based); ~0 if none
};

struct KParams {
  const Task* tasks;
  const Seg* segs;
  const Wait* waits;
  const int32_t* sigs;
  int ntasks;
  int* ctr;             // dependency counters (zeroed before the launch)
  int* claim;           // next task to claim (zeroed before the launch)
  DevStatus* st;        // status block (reset before the launch)
  double* logdet_part;  // one partial sum of log diag(L) per POTRF task
  double* buf[4];       // BUF_A, BUF_L, BUF_S, BUF_W base pointers
  long long budget_ns;  // bound of one dependency wait
};

size_t kernel_smem_bytes();
cudaError_t launch_persistent(const KParams& p, int grid, cudaStream_t stream);

}  // namespace stiles
