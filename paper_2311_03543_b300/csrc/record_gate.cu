// Gate for recorded calls: device times that do not include host gaps.
//
// A recorded call is timed by two events around its launches.  When the GPU
// is idle, the launches of a call with several kernels (pre-pass, GEMM,
// reduce) reach it one by one as the host issues them, and the idle time in
// between would be counted as the call's time.  The recording path therefore
// enqueues this one-thread kernel first: it waits until the host, having
// enqueued the whole call, writes the call's ticket into a host-mapped word
// (or until a short budget runs out, after which the call simply runs), so
// the call's kernels then run back to back between the two events.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.h"

namespace compar {
namespace {

__global__ void record_gate_kernel(const unsigned int* flag, unsigned int ticket,
                                   unsigned long long budget_ns) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    unsigned int v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (static_cast<int>(v - ticket) >= 0) return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > budget_ns) return;  // the host is late: run the call anyway
    __nanosleep(256);
  }
}

}  // namespace

int launch_record_gate(const unsigned int* flag_dev, unsigned int ticket, cudaStream_t s) {
  record_gate_kernel<<<1, 1, 0, s>>>(flag_dev, ticket, 2000000ull);  // 2 ms at most
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

}  // namespace compar
