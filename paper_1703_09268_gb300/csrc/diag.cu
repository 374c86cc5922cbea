// Diagnostic entry point for the failure reporting of bounded device waits.
#include "common.cuh"
#include "tma.cuh"

namespace helm {

namespace {

__device__ int g_wait_gave_up;

// One thread waits on an mbarrier phase that nothing completes, with the
// same bounded wait the streamed kernels use, and records that it gave up.
__global__ void k_unsatisfied_wait() {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  g_wait_gave_up = mbar_wait_bounded(&bar, 0u) ? 0 : 1;
}

}  // namespace

}  // namespace helm

extern "C" int helm_check_bounded_wait(helm_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(helm::g_wait_gave_up, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return HELM_E_CUDA;
  helm::k_unsatisfied_wait<<<1, 32, 0, st>>>();
  helm::count_launch();
  int gave_up = 0;
  if (cudaMemcpyFromSymbolAsync(&gave_up, helm::g_wait_gave_up, sizeof(int), 0, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return HELM_E_CUDA;
  return gave_up ? HELM_E_TIMEOUT : HELM_OK;
}
