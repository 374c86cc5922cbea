// helm_apply_noalloc: the operator apply of helm_apply without a
// caller-provided workspace.
//
// helm_apply needs scratch device memory for the extended model (FP64 and
// FP32 copies), the damping-layer coefficient tables and the per-field slot
// lists; normally the caller allocates it and passes it in.  Some callers
// cannot allocate device memory at the point where they apply the operator:
// code embedded in a host framework that owns every device allocation
// through its own pool and forbids raw cudaMalloc, and latency-critical
// serving loops that must not allocate per request.  For them this file
// keeps the scratch in one file-scope device array of fixed size, so a call
// allocates nothing.  The call is not meant for stream capture: like
// helm_apply it copies small host arrays to the device and synchronises its
// stream before returning.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Every call shares it, and it keeps whatever the last call wrote, so
// two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "solver.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[HELM_NOALLOC_SCRATCH_BYTES];

namespace helm {
namespace {

// Device address of g_noalloc_scratch per device ordinal, looked up once per
// device (the host-side symbol is only a stand-in, never a device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HELM_E_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HELM_E_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return HELM_OK;
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" int helm_apply_noalloc(helm_plan* P, const double* m_phys, double freq_hz, int adjoint,
                                  int precision, const void* x, void* y, int nrhs, helm_stream_t stream) {
  if (!P || !m_phys || !x || !y || nrhs < 1 || !(freq_hz > 0.0) || !std::isfinite(freq_hz)) return HELM_E_INVAL;
  if (precision != HELM_FP64 && precision != HELM_MIXED) return HELM_E_INVAL;
  const size_t need = layout(*P, HELM_CALL_APPLY, 1, nrhs, 0, nullptr, nullptr);
  if (need > (size_t)HELM_NOALLOC_SCRATCH_BYTES) return HELM_E_NOMEM;
  void* ws = nullptr;
  int st = scratch_address(&ws);
  if (st != HELM_OK) return st;
  Ctx c;
  layout(*P, HELM_CALL_APPLY, 1, nrhs, 0, (char*)ws, &c);
  c.st = (cudaStream_t)stream;
  // setup_operator clears the error counters and rewrites every other piece of
  // scratch this call reads (model copies, tables, frequency data, slot lists).
  if ((st = setup_operator(c, m_phys, &freq_hz)) != HELM_OK) return st;
  std::vector<int> g(nrhs);
  for (int i = 0; i < nrhs; ++i) g[i] = i;
  if ((st = set_batch(c, g)) != HELM_OK) return st;
  const int dir = adjoint ? 1 : 0;
  // no shape tuning here (it would create timing events): a grid tuned by an earlier call keeps its
  // shape, any other takes the first one -- the results are the same either way
  if (precision == HELM_FP64) {
    launch_stencil<double>(op_view<double>(c, 0, dir), c.slot_f, c.act, c.na, (const double2*)x, Scale<double>{},
                           nullptr, Scale<double>{}, (double2*)y, c.st, nullptr, nullptr, 0, 0, false);
  } else {
    launch_stencil<float>(op_view<float>(c, 0, dir), c.slot_f, c.act, c.na, (const float2*)x, Scale<float>{},
                          nullptr, Scale<float>{}, (float2*)y, c.st, nullptr, nullptr, 0, 0, false);
  }
  return sync_check(c);
}
