// Work queue over models: helm_misfit_and_gradient_batch.
//
// Every item is a complete misfit_and_gradient request (its own plan, model,
// acquisition, workspace and stream).  Host workers take items from a shared
// atomic counter in order; each worker blocks only on its own stream, so the
// solves of different models overlap on the GPU and small models fill the
// SMs that one large model alone would leave idle.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "helm.h"

static int worst_status(int a, int b) {
  const int order[] = {HELM_E_CUDA, HELM_E_TIMEOUT, HELM_E_INVAL, HELM_E_NOMEM, HELM_E_NONFINITE, HELM_E_NOCONV};
  for (int s : order)
    if (a == s || b == s) return s;
  return HELM_OK;
}

extern "C" int helm_misfit_and_gradient_batch(helm_batch_item* items, int nitems, int nworkers) {
  if (!items || nitems < 0 || nworkers < 1) return HELM_E_INVAL;
  if (nitems == 0) return HELM_OK;
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int i = next.fetch_add(1); i < nitems; i = next.fetch_add(1)) {
      helm_batch_item& it = items[i];
      it.status = misfit_and_gradient(it.plan, it.m_phys, it.freqs_hz, it.nfreq, it.src_idx, it.n_srcloc, it.Q,
                                      it.nsrc, it.wavelet, it.rec_idx, it.nrec, it.d_obs, it.mask, it.f_out, it.g_out,
                                      it.workspace, it.ws_bytes, it.reports, it.stream);
    }
  };
  const int nw = std::min(nworkers, nitems);
  std::vector<std::thread> pool;
  pool.reserve(nw - 1);
  for (int w = 1; w < nw; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  int st = HELM_OK;
  for (int i = 0; i < nitems; ++i) st = worst_status(st, items[i].status);
  return st;
}
