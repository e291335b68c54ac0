// selftest.cu -- exercises the failure path of the bounded waits used by the
// bulk-copy passes, without faulting or hanging the GPU: one block waits on an
// mbarrier that nothing ever arrives at, the wait runs out after the given
// limit, and the kernel records the same error code a stalled copy would.
#include "gfc_internal.h"
#include "tma.cuh"

namespace {

__global__ void k_wait_selftest(int* err, unsigned long long timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) gfc::mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = gfc::mbar_wait(&bar, 0, timeout_ns);  // no arrival is ever made
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, gfc::kErrBulkWait);
}

}  // namespace

extern "C" gfc_status gfc_plan_selftest_wait(gfc_plan* plan, int timeout_ms) {
  gfc::clear_error();
  if (!plan) return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_plan_selftest_wait: null plan");
  if (timeout_ms < 1 || timeout_ms > 2000)
    return gfc::fail(GFC_ERR_INVALID_ARG, "gfc_plan_selftest_wait: timeout_ms=%d (1..2000)", timeout_ms);
  k_wait_selftest<<<1, 32, 0, plan->stream>>>(plan->dev_err, (unsigned long long)timeout_ms * 1000000ull);
  GFC_CUDA_TRY(cudaGetLastError());
  return GFC_OK;
}
