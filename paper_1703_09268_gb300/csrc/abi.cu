// The extern "C" entry points of include/helm.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "solver.h"

namespace helm {

std::atomic<uint64_t> g_launches{0};

// ---------------------------------------------------------------------------
// Per-class launch timing
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
  int cls;
  double bytes;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<cudaEvent_t> g_ev_pool;
std::vector<ProfRec> g_recs;
uint64_t g_prof_n[PC_COUNT];
double g_prof_ms[PC_COUNT];
double g_prof_bytes[PC_COUNT];

cudaEvent_t take_event() {
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_records() {
  for (ProfRec& r : g_recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    g_prof_n[r.cls] += 1;
    g_prof_ms[r.cls] += ms;
    g_prof_bytes[r.cls] += r.bytes;
    g_ev_pool.push_back(r.a);
    g_ev_pool.push_back(r.b);
  }
  g_recs.clear();
}
}  // namespace

ProfScope::ProfScope(int c, double by, cudaStream_t s) : cls(c), bytes(by), st(s), slot(-1) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_recs.size() >= 200000) drain_records();
  ProfRec r{c, by, take_event(), take_event()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  slot = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_recs.size()) cudaEventRecord(g_recs[slot].b, st);
}

// ---------------------------------------------------------------------------
// Plan construction
// ---------------------------------------------------------------------------
static int build_plan(const helm_grid* g, const helm_solve_opts* o, helm_plan* P) {
  if (!g || !o) return HELM_E_INVAL;
  if (g->dim != 2 && g->dim != 3) return HELM_E_INVAL;
  if (!(g->h > 0.0) || !std::isfinite(g->h)) return HELM_E_INVAL;
  if (g->levels < 1 || g->levels > MAX_LEVELS) return HELM_E_INVAL;
  for (int d = 0; d < 3; ++d) {
    if (g->npml[d] < 0 || g->n[d] < 1) return HELM_E_INVAL;
    if (g->sigma_max[d] < 0.0 || !std::isfinite(g->sigma_max[d])) return HELM_E_INVAL;
  }
  if (g->dim == 2 && (g->n[1] != 1 || g->npml[1] != 0)) return HELM_E_INVAL;
  const int active[3] = {1, g->dim == 3 ? 1 : 0, 1};
  for (int d = 0; d < 3; ++d)
    if (active[d] && g->n[d] < 2) return HELM_E_INVAL;
  bool need_vref = false;
  for (int d = 0; d < 3; ++d)
    if (g->npml[d] > 0 && g->sigma_max[d] == 0.0) need_vref = true;
  if (need_vref && !(g->v_ref > 0.0)) return HELM_E_INVAL;
  // options
  if (o->precision != HELM_FP64 && o->precision != HELM_MIXED) return HELM_E_INVAL;
  if (o->precond < HELM_PRECOND_NONE || o->precond > HELM_PRECOND_MLGMRES) return HELM_E_INVAL;
  if (o->k_inner < 1 || o->k_inner > KMAX || o->max_cycles < 1) return HELM_E_INVAL;
  if (!(o->tol > 0.0) || !(o->tol < 1.0)) return HELM_E_INVAL;
  if (o->precision == HELM_MIXED && (!(o->tol_inner > 0.0) || !(o->tol_inner < 1.0) || o->max_refine < 1))
    return HELM_E_INVAL;
  if (o->precond == HELM_PRECOND_MLGMRES) {
    if (o->k_so < 1 || o->k_si < 1 || o->k_si > KMAX || o->k_co < 1 || o->k_ci < 1 || o->k_ci > KMAX)
      return HELM_E_INVAL;
    if (g->levels < 2) return HELM_E_INVAL;
  }
  if (o->precond == HELM_PRECOND_JACOBI && (!(o->jacobi_omega > 0.0) || o->jacobi_sweeps < 1))
    return HELM_E_INVAL;
  if (o->max_batch < 0) return HELM_E_INVAL;
  if (o->reorth != 0 && o->reorth != 1) return HELM_E_INVAL;
  if (o->sstep != 0 && o->sstep != 1) return HELM_E_INVAL;

  std::memset(P, 0, sizeof(*P));
  P->g = *g;
  P->o = *o;
  P->L = o->precond == HELM_PRECOND_MLGMRES ? g->levels : 1;
  const int q = 1 << (g->levels - 1);
  for (int d = 0; d < 3; ++d) {
    if (!active[d]) {
      P->pad[d] = 0;
    } else {
      const int base = g->n[d] + 2 * g->npml[d];
      P->pad[d] = ((-(base + 1)) % q + q) % q;
    }
    if (g->sigma_max[d] > 0.0)
      P->smax[d] = g->sigma_max[d];
    else
      P->smax[d] = g->npml[d] > 0 ? 3.0 * g->v_ref * std::log(1000.0) / (2.0 * g->npml[d] * g->h) : 0.0;
  }
  P->n_phys = (size_t)g->n[0] * g->n[1] * g->n[2];
  for (int l = 0; l < MAX_LEVELS; ++l) {
    LevelGeom& L = P->lev[l];
    for (int d = 0; d < 3; ++d) {
      if (l == 0)
        L.N[d] = active[d] ? g->n[d] + 2 * g->npml[d] + P->pad[d] : 1;
      else
        L.N[d] = active[d] ? (P->lev[l - 1].N[d] - 1) / 2 : 1;
    }
    if (g->dim == 3) {
      L.K[0] = L.N[0]; L.K[1] = L.N[1]; L.K[2] = L.N[2];
    } else {
      // 2D: x, a unit axis, z -- the stencil's flattened plane is one x row and it marches in z
      L.K[0] = L.N[0]; L.K[1] = 1; L.K[2] = L.N[2];
    }
    L.n = (size_t)L.N[0] * L.N[1] * L.N[2];
    L.Nmax = std::max(L.K[0], std::max(L.K[1], L.K[2]));
    L.h = g->h * (double)(1 << l);
    if (l < P->L)
      for (int d = 0; d < 3; ++d)
        if (active[d] && L.N[d] < 3) return HELM_E_INVAL;
  }
  return HELM_OK;
}

static bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

// Bind a workspace to a Ctx after checking its size.
static int bind(helm_plan* P, int call, int nfreq, int nsrc, int nrec, void* ws, size_t ws_bytes,
                helm_stream_t stream, Ctx& c) {
  const size_t need = layout(*P, call, nfreq, nsrc, nrec, nullptr, nullptr);
  if (!ws || ws_bytes < need) return HELM_E_NOMEM;
  if (!aligned256(ws)) return HELM_E_INVAL;
  layout(*P, call, nfreq, nsrc, nrec, (char*)ws, &c);
  c.st = (cudaStream_t)stream;
  return arm_guards(c);
}

static int read_err(Ctx& c, int* h) {
  cudaMemcpyAsync(h, c.err, 4 * sizeof(int), cudaMemcpyDeviceToHost, c.st);
  return sync_check(c);
}

static void fill_reports(helm_rhs_report* reports, const std::vector<int>& g,
                         const std::vector<SlotReport>& rep) {
  if (!reports) return;
  for (size_t a = 0; a < g.size(); ++a) {
    helm_rhs_report& r = reports[g[a]];
    r.status = rep[a].status;
    r.iters = rep[a].iters;
    r.refinements = rep[a].refine;
    r.rel_resid = rep[a].rel;
  }
}

static int worst(int a, int b) {
  if (a == HELM_E_CUDA || b == HELM_E_CUDA) return HELM_E_CUDA;
  if (a == HELM_E_TIMEOUT || b == HELM_E_TIMEOUT) return HELM_E_TIMEOUT;
  if (a == HELM_E_NONFINITE || b == HELM_E_NONFINITE) return HELM_E_NONFINITE;
  if (a == HELM_E_NOCONV || b == HELM_E_NOCONV) return HELM_E_NOCONV;
  return a != HELM_OK ? a : b;
}

}  // namespace helm

using namespace helm;

extern "C" {

int helm_default_opts(helm_solve_opts* o) {
  if (!o) return HELM_E_INVAL;
  std::memset(o, 0, sizeof(*o));
  o->precision = HELM_MIXED;
  o->precond = HELM_PRECOND_MLGMRES;
  o->k_inner = 10;
  o->max_cycles = 200;
  o->tol = 1e-10;
  o->tol_inner = 0.1;
  o->max_refine = 60;
  o->k_so = 3;
  o->k_si = 5;
  o->k_co = 3;
  o->k_ci = 5;
  o->jacobi_omega = 0.6;
  o->jacobi_sweeps = 1;
  o->max_batch = 0;
  o->reorth = 1;
  o->sstep = 1;
  return HELM_OK;
}

int helm_plan_create(const helm_grid* grid, const helm_solve_opts* opts, helm_plan** plan) {
  if (!plan) return HELM_E_INVAL;
  *plan = nullptr;
  helm_plan* P = new (std::nothrow) helm_plan;
  if (!P) return HELM_E_NOMEM;
  const int st = build_plan(grid, opts, P);
  if (st != HELM_OK) {
    delete P;
    return st;
  }
  *plan = P;
  return HELM_OK;
}

void helm_plan_destroy(helm_plan* plan) { delete plan; }

int helm_plan_dims(const helm_plan* P, int N[3], size_t* n_comp, size_t* n_phys) {
  if (!P) return HELM_E_INVAL;
  if (N)
    for (int d = 0; d < 3; ++d) N[d] = P->lev[0].N[d];
  if (n_comp) *n_comp = P->lev[0].n;
  if (n_phys) *n_phys = P->n_phys;
  return HELM_OK;
}

int helm_workspace_size(const helm_plan* P, int call, int nfreq, int nsrc, int nrec, size_t* bytes) {
  if (!P || !bytes || nfreq < 1 || nsrc < 1 || nrec < 0) return HELM_E_INVAL;
  if (call < HELM_CALL_APPLY || call > HELM_CALL_WRI) return HELM_E_INVAL;
  *bytes = layout(*P, call, nfreq, nsrc, nrec, nullptr, nullptr);
  return HELM_OK;
}

int helm_apply(helm_plan* P, const double* m_phys, double freq_hz, int adjoint, int precision,
               const void* x, void* y, int nrhs, void* ws, size_t ws_bytes, helm_stream_t stream) {
  NvtxRange nvtx("helm_apply");
  if (!P || !m_phys || !x || !y || nrhs < 1 || !(freq_hz > 0.0) || !std::isfinite(freq_hz))
    return HELM_E_INVAL;
  if (precision != HELM_FP64 && precision != HELM_MIXED) return HELM_E_INVAL;
  Ctx c;
  int st = bind(P, HELM_CALL_APPLY, 1, nrhs, 0, ws, ws_bytes, stream, c);
  if (st != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, &freq_hz)) != HELM_OK) return st;
  std::vector<int> g(nrhs);
  for (int i = 0; i < nrhs; ++i) g[i] = i;
  if ((st = set_batch(c, g)) != HELM_OK) return st;
  const int dir = adjoint ? 1 : 0;
  if (precision == HELM_FP64) {
    launch_stencil<double>(op_view<double>(c, 0, dir), c.slot_f, c.act, c.na, (const double2*)x,
                           Scale<double>{}, nullptr, Scale<double>{}, (double2*)y, c.st);
  } else {
    launch_stencil<float>(op_view<float>(c, 0, dir), c.slot_f, c.act, c.na, (const float2*)x,
                          Scale<float>{}, nullptr, Scale<float>{}, (float2*)y, c.st);
  }
  return final_check(c);
}

int helm_precond_apply(helm_plan* P, const double* m_phys, double freq_hz, int adjoint, const void* x, void* z,
                       int nrhs, void* ws, size_t ws_bytes, helm_stream_t stream) {
  NvtxRange nvtx("helm_precond_apply");
  if (!P || !m_phys || !x || !z || nrhs < 1 || !(freq_hz > 0.0) || !std::isfinite(freq_hz)) return HELM_E_INVAL;
  Ctx c;
  int st = bind(P, HELM_CALL_PRECOND, 1, nrhs, 0, ws, ws_bytes, stream, c);
  if (st != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, &freq_hz)) != HELM_OK) return st;
  const size_t n = P->lev[0].n;
  const size_t esz = P->o.precision == HELM_MIXED ? sizeof(float2) : sizeof(double2);
  for (int start = 0; start < nrhs; start += c.B) {
    const int nb = std::min(c.B, nrhs - start);
    std::vector<int> g(nb);
    for (int a = 0; a < nb; ++a) g[a] = start + a;
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    st = precond_apply(c, adjoint ? 1 : 0, (const char*)x + (size_t)start * n * esz, (char*)z + (size_t)start * n * esz);
    if (st != HELM_OK) return st;
  }
  return final_check(c);
}

static int check_common(helm_plan* P, const double* m_phys, const double* freqs, int nfreq, int nsrc) {
  if (!P || !m_phys || !freqs || nfreq < 1 || nsrc < 1) return HELM_E_INVAL;
  for (int k = 0; k < nfreq; ++k)
    if (!(freqs[k] > 0.0) || !std::isfinite(freqs[k])) return HELM_E_INVAL;
  return HELM_OK;
}

static int check_indices(Ctx& c, const int32_t* src, int nsrcloc, const int32_t* rec, int nrec) {
  if (src) launch_check_idx(*c.P, src, nsrcloc, c.err, c.st);
  if (rec) launch_check_idx(*c.P, rec, nrec, c.err, c.st);
  int h[4] = {0, 0, 0, 0};
  if (read_err(c, h) != HELM_OK) return HELM_E_CUDA;
  return h[0] == 0 ? HELM_OK : HELM_E_INVAL;
}

int helm_forward(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq,
                 const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                 const int32_t* rec_idx, int nrec, const void* U0, void* U_out, void* D_out, void* ws,
                 size_t ws_bytes, helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx("helm_forward");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!src_idx || n_srcloc < 1 || !Q || nrec < 0 || (nrec > 0 && !rec_idx)) return HELM_E_INVAL;
  if (D_out && nrec < 1) return HELM_E_INVAL;
  Ctx c;
  if ((st = bind(P, HELM_CALL_FORWARD, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, src_idx, n_srcloc, nrec > 0 ? rec_idx : nullptr, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  int result = HELM_OK;
  for (int start = 0; start < nrhs; start += c.B) {
    const int nb = std::min(c.B, nrhs - start);
    std::vector<int> g(nb);
    for (int a = 0; a < nb; ++a) g[a] = start + a;
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_sources(*P, src_idx, n_srcloc, (const double2*)Q, nsrc, (const double2*)wavelet, c.slot_f,
                   c.slot_s, nb, c.q, c.err + 1, c.st);
    // warm start: the caller's initial fields of this batch's pairs
    if (U0) launch_copy_fields((const double2*)U0, c.u, c.slot_g, nb, c.ident, n, c.st);
    std::vector<SlotReport> rep;
    st = solve_batch(c, 0, c.q, c.u, nb, rep, nullptr, U0 != nullptr);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    for (auto& r : rep) result = worst(result, r.status);
    if (U_out) launch_copy_fields(c.u, (double2*)U_out, c.ident, nb, c.slot_g, n, c.st);
    if (D_out) launch_receivers(*P, c.u, rec_idx, nrec, c.slot_g, nb, (double2*)D_out, nrec, c.st);
    fill_reports(reports, g, rep);
  }
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

int helm_adjoint(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq,
                 const int32_t* rec_idx, int nrec, const void* R_in, int nsrc, void* V_out, void* ws,
                 size_t ws_bytes, helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx("helm_adjoint");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!rec_idx || nrec < 1 || !R_in || !V_out) return HELM_E_INVAL;
  Ctx c;
  if ((st = bind(P, HELM_CALL_ADJOINT, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, nullptr, 0, rec_idx, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  int result = HELM_OK;
  for (int start = 0; start < nrhs; start += c.B) {
    const int nb = std::min(c.B, nrhs - start);
    std::vector<int> g(nb);
    for (int a = 0; a < nb; ++a) g[a] = start + a;
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_spread(*P, (const double2*)R_in, nrec, rec_idx, nrec, 1.0, c.slot_g, nb, c.q, c.st);
    std::vector<SlotReport> rep;
    st = solve_batch(c, 1, c.q, c.v, nb, rep);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    for (auto& r : rep) result = worst(result, r.status);
    launch_copy_fields(c.v, (double2*)V_out, c.ident, nb, c.slot_g, n, c.st);
    fill_reports(reports, g, rep);
  }
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

int misfit_and_gradient(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq,
                        const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                        const int32_t* rec_idx, int nrec, const void* d_obs, const uint8_t* mask,
                        double* f_out, double* g_out, void* ws, size_t ws_bytes, helm_rhs_report* reports,
                        helm_stream_t stream) {
  NvtxRange nvtx("misfit_and_gradient");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!src_idx || n_srcloc < 1 || !Q || !rec_idx || nrec < 1 || !d_obs || !f_out || !g_out)
    return HELM_E_INVAL;
  Ctx c;
  if ((st = bind(P, HELM_CALL_MISFIT_GRAD, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, src_idx, n_srcloc, rec_idx, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  // (k, s) pairs to evaluate
  std::vector<int> todo;
  if (mask) {
    std::vector<uint8_t> mh(nrhs);
    cudaMemcpyAsync(mh.data(), mask, nrhs, cudaMemcpyDeviceToHost, c.st);
    if (const int sc = sync_check(c); sc != HELM_OK) return sc;
    for (int i = 0; i < nrhs; ++i)
      if (mh[i]) todo.push_back(i);
  } else {
    for (int i = 0; i < nrhs; ++i) todo.push_back(i);
  }
  if (reports)
    for (int i = 0; i < nrhs; ++i) reports[i] = helm_rhs_report{HELM_OK, 0, 0, 0.0};
  cudaMemsetAsync(c.gcomp, 0, sizeof(double) * n, c.st);
  cudaMemsetAsync(f_out, 0, sizeof(double), c.st);
  int result = HELM_OK;
  for (size_t start = 0; start < todo.size(); start += c.B) {
    const int nb = (int)std::min<size_t>(c.B, todo.size() - start);
    std::vector<int> g(todo.begin() + start, todo.begin() + start + nb);
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    // state: u = H^{-1} q
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_sources(*P, src_idx, n_srcloc, (const double2*)Q, nsrc, (const double2*)wavelet, c.slot_f,
                   c.slot_s, nb, c.q, c.err + 1, c.st);
    std::vector<SlotReport> rf, ra;
    st = solve_batch(c, 0, c.q, c.u, nb, rf);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    // misfit and adjoint source -P_r^T (P_r u - d)
    launch_residual_misfit(*P, c.u, rec_idx, nrec, (const double2*)d_obs, c.slot_f, c.slot_s, nsrc, c.ident,
                           nb, c.res, c.f_slot, c.st);
    launch_sum_f(c.f_slot, c.ident, nb, f_out, 1, c.st);
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_spread(*P, c.res, nrec, rec_idx, nrec, -1.0, c.ident, nb, c.q, c.st);
    // adjoint state v = H^{-H} b
    st = solve_batch(c, 1, c.q, c.v, nb, ra);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    // g += w^2 Re(conj(u) v)
    launch_grad_accum(c.u, nullptr, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
    for (int a = 0; a < nb; ++a) {
      SlotReport r = rf[a];
      r.iters += ra[a].iters;
      r.refine += ra[a].refine;
      r.rel = std::max(rf[a].rel, ra[a].rel);
      r.status = worst(rf[a].status, ra[a].status);
      result = worst(result, r.status);
      rf[a] = r;
    }
    fill_reports(reports, g, rf);
  }
  launch_extend_adjoint(*P, c.gcomp, g_out, c.st);
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

// (k, s) pairs selected by an optional device mask, in (frequency, source) order.
static int mask_list(Ctx& c, const uint8_t* mask, int nrhs, std::vector<int>& todo) {
  todo.clear();
  if (!mask) {
    for (int i = 0; i < nrhs; ++i) todo.push_back(i);
    return HELM_OK;
  }
  std::vector<uint8_t> mh(nrhs);
  cudaMemcpyAsync(mh.data(), mask, nrhs, cudaMemcpyDeviceToHost, c.st);
  if (const int sc = sync_check(c); sc != HELM_OK) return sc;
  for (int i = 0; i < nrhs; ++i)
    if (mh[i]) todo.push_back(i);
  return HELM_OK;
}

// Per-pair report of several solves: iterations added, the worst residual and status.
static void merge_reports(std::vector<SlotReport>& acc, const std::vector<SlotReport>& add) {
  for (size_t a = 0; a < acc.size(); ++a) {
    acc[a].iters += add[a].iters;
    acc[a].refine += add[a].refine;
    acc[a].rel = std::max(acc[a].rel, add[a].rel);
    acc[a].status = worst(acc[a].status, add[a].status);
  }
}

// The linearised calls (Appendix A): kind 0 = J dm, 1 = J^T dD, 2 = J^T J dm,
// 3 = full Hessian of the misfit times dm (dD_in then holds d_obs).
static int linearised(int kind, helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq,
                      const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                      const int32_t* rec_idx, int nrec, const double* dm_phys, const void* dD_in,
                      const uint8_t* mask, void* dD_out, double* g_out, void* ws, size_t ws_bytes,
                      helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx(kind == 0 ? "helm_born" : kind == 1 ? "helm_born_adjoint" : kind == 2 ? "helm_gn_hessvec" : "helm_hessvec");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!src_idx || n_srcloc < 1 || !Q || !rec_idx || nrec < 1) return HELM_E_INVAL;
  if ((kind != 1 && !dm_phys) || ((kind == 1 || kind == 3) && !dD_in) || (kind == 0 && !dD_out) ||
      (kind != 0 && !g_out))
    return HELM_E_INVAL;
  const int call = kind == 0   ? HELM_CALL_BORN
                   : kind == 1 ? HELM_CALL_BORN_ADJOINT
                   : kind == 2 ? HELM_CALL_GN_HESSVEC
                               : HELM_CALL_HESSVEC;
  Ctx c;
  if ((st = bind(P, call, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, src_idx, n_srcloc, rec_idx, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  std::vector<int> todo;
  if ((st = mask_list(c, mask, nrhs, todo)) != HELM_OK) return st;
  if (reports)
    for (int i = 0; i < nrhs; ++i) reports[i] = helm_rhs_report{HELM_OK, 0, 0, 0.0};
  if (kind == 0) cudaMemsetAsync(dD_out, 0, sizeof(double2) * (size_t)nrhs * nrec, c.st);
  if (kind != 0) cudaMemsetAsync(c.gcomp, 0, sizeof(double) * n, c.st);
  if (kind != 1) launch_extend(*P, dm_phys, c.dmc, nullptr, c.st);
  int result = HELM_OK;
  for (size_t start = 0; start < todo.size(); start += c.B) {
    const int nb = (int)std::min<size_t>(c.B, todo.size() - start);
    std::vector<int> g(todo.begin() + start, todo.begin() + start + nb);
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    // state u = H^{-1} q
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_sources(*P, src_idx, n_srcloc, (const double2*)Q, nsrc, (const double2*)wavelet, c.slot_f,
                   c.slot_s, nb, c.q, c.err + 1, c.st);
    std::vector<SlotReport> rep, r2;
    st = solve_batch(c, 0, c.q, c.u, nb, rep);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    if (kind == 3) {
      auto solve = [&](int dir, double2* out) {
        st = solve_batch(c, dir, c.q, out, nb, r2);
        if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return false;
        result = worst(result, st);
        merge_reports(rep, r2);
        return true;
      };
      // adjoint state v = -H^{-H} P_r^T (P_r u - d)
      launch_residual_misfit(*P, c.u, rec_idx, nrec, (const double2*)dD_in, c.slot_f, c.slot_s, nsrc, c.ident, nb,
                             c.res, c.f_slot, c.st);
      cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
      launch_spread(*P, c.res, nrec, rec_idx, nrec, -1.0, c.ident, nb, c.q, c.st);
      if (!solve(1, c.v)) return st;
      // linearised state du = -H^{-1} w^2 (E dm) u, then the DT^*[dm, du] v term
      launch_born_source(c.u, c.dmc, c.w2_64, c.slot_f, nb, n, c.q, c.st);
      if (!solve(0, c.du)) return st;
      launch_grad_accum(c.du, nullptr, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
      // dv = H^{-H}(-w^2 (E dm) v - P_r^T P_r du), then the T^* dv term
      launch_born_source(c.v, c.dmc, c.w2_64, c.slot_f, nb, n, c.q, c.st);
      launch_receivers(*P, c.du, rec_idx, nrec, c.ident, nb, c.res, nrec, c.st);
      launch_spread(*P, c.res, nrec, rec_idx, nrec, -1.0, c.ident, nb, c.q, c.st);
      if (!solve(1, c.du)) return st;
      launch_grad_accum(c.u, nullptr, c.du, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
      for (auto& r : rep) result = worst(result, r.status);
      fill_reports(reports, g, rep);
      continue;
    }
    if (kind != 1) {
      // linearised state du = H^{-1}(-T dm), data dD = P_r du
      launch_born_source(c.u, c.dmc, c.w2_64, c.slot_f, nb, n, c.q, c.st);
      st = solve_batch(c, 0, c.q, c.v, nb, r2);
      if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
      result = worst(result, st);
      merge_reports(rep, r2);
      if (kind == 0)
        launch_receivers(*P, c.v, rec_idx, nrec, c.slot_g, nb, (double2*)dD_out, nrec, c.st);
      else
        launch_receivers(*P, c.v, rec_idx, nrec, c.ident, nb, c.res, nrec, c.st);
    }
    if (kind != 0) {
      // adjoint state v = -H^{-H} P_r^T dD, then g += w^2 Re(conj(u) v)
      cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
      if (kind == 1)
        launch_spread(*P, (const double2*)dD_in, nrec, rec_idx, nrec, -1.0, c.slot_g, nb, c.q, c.st);
      else
        launch_spread(*P, c.res, nrec, rec_idx, nrec, -1.0, c.ident, nb, c.q, c.st);
      st = solve_batch(c, 1, c.q, c.v, nb, r2);
      if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
      result = worst(result, st);
      merge_reports(rep, r2);
      launch_grad_accum(c.u, nullptr, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
    }
    for (auto& r : rep) result = worst(result, r.status);
    fill_reports(reports, g, rep);
  }
  if (kind != 0) launch_extend_adjoint(*P, c.gcomp, g_out, c.st);
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

int helm_born(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq, const int32_t* src_idx,
              int n_srcloc, const void* Q, int nsrc, const void* wavelet, const int32_t* rec_idx, int nrec,
              const double* dm_phys, const uint8_t* mask, void* dD_out, void* ws, size_t ws_bytes,
              helm_rhs_report* reports, helm_stream_t stream) {
  return linearised(0, P, m_phys, freqs_hz, nfreq, src_idx, n_srcloc, Q, nsrc, wavelet, rec_idx, nrec, dm_phys,
                    nullptr, mask, dD_out, nullptr, ws, ws_bytes, reports, stream);
}

int helm_born_adjoint(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq, const int32_t* src_idx,
                      int n_srcloc, const void* Q, int nsrc, const void* wavelet, const int32_t* rec_idx, int nrec,
                      const void* dD_in, const uint8_t* mask, double* g_out, void* ws, size_t ws_bytes,
                      helm_rhs_report* reports, helm_stream_t stream) {
  return linearised(1, P, m_phys, freqs_hz, nfreq, src_idx, n_srcloc, Q, nsrc, wavelet, rec_idx, nrec, nullptr,
                    dD_in, mask, nullptr, g_out, ws, ws_bytes, reports, stream);
}

int helm_misfit_and_gradient_25d(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq,
                                 const double* ky, const double* ck, int nk, const int32_t* src_idx, int n_srcloc,
                                 const void* Q, int nsrc, const void* wavelet, const int32_t* rec_idx, int nrec,
                                 const void* d_obs, double* f_out, double* g_out, void* ws, size_t ws_bytes,
                                 helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx("helm_misfit_and_gradient_25d");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (P->g.dim != 2 || !ky || !ck || nk < 1 || !src_idx || n_srcloc < 1 || !Q || !rec_idx || nrec < 1 || !d_obs ||
      !f_out || !g_out)
    return HELM_E_INVAL;
  for (int i = 0; i < nk; ++i)
    if (!std::isfinite(ky[i]) || !std::isfinite(ck[i])) return HELM_E_INVAL;
  // virtual frequencies v = j*nk + i: (w_j, k_i)
  const int nv = nfreq * nk;
  Ctx c;
  if ((st = bind(P, HELM_CALL_MISFIT_GRAD_25D, nv, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  const int gmax = c.B / nk;  // whole groups of nk slots per batch
  if (gmax < 1) return HELM_E_INVAL;
  std::vector<double> fv(nv), sv(nv), cv(nv);
  for (int j = 0; j < nfreq; ++j)
    for (int i = 0; i < nk; ++i) {
      fv[j * nk + i] = freqs_hz[j];
      sv[j * nk + i] = ky[i] * ky[i];
      cv[j * nk + i] = ck[i];
    }
  cudaMemcpyAsync(c.shift, sv.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.ck, cv.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, c.st);
  if (wavelet)
    for (int v = 0; v < nv; ++v)
      cudaMemcpyAsync(c.wav + v, (const double2*)wavelet + v / nk, sizeof(double2), cudaMemcpyDeviceToDevice, c.st);
  if ((st = setup_operator(c, m_phys, fv.data())) != HELM_OK) return st;
  if ((st = check_indices(c, src_idx, n_srcloc, rec_idx, nrec)) != HELM_OK) return st;
  const size_t n = P->lev[0].n;
  if (reports)
    for (int i = 0; i < nv * nsrc; ++i) reports[i] = helm_rhs_report{HELM_OK, 0, 0, 0.0};
  cudaMemsetAsync(c.gcomp, 0, sizeof(double) * n, c.st);
  cudaMemsetAsync(f_out, 0, sizeof(double), c.st);
  const int ngroups_all = nfreq * nsrc;
  int result = HELM_OK;
  for (int g0 = 0; g0 < ngroups_all; g0 += gmax) {
    const int ng = std::min(gmax, ngroups_all - g0);
    const int nb = ng * nk;
    std::vector<int> gl(nb), fl(nb), sl(nb);
    for (int a = 0; a < ng; ++a) {
      const int j = (g0 + a) / nsrc, s = (g0 + a) % nsrc;
      for (int i = 0; i < nk; ++i) {
        gl[a * nk + i] = (j * nsrc + s) * nk + i;
        fl[a * nk + i] = j * nk + i;
        sl[a * nk + i] = s;
      }
    }
    if ((st = set_batch_fs(c, gl, fl, sl)) != HELM_OK) return st;
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_sources(*P, src_idx, n_srcloc, (const double2*)Q, nsrc, wavelet ? c.wav : nullptr, c.slot_f, c.slot_s,
                   nb, c.q, c.err + 1, c.st);
    std::vector<SlotReport> rep, ra;
    st = solve_batch(c, 0, c.q, c.u, nb, rep);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    // r = sum_i c_i P_r u_i - d per (frequency, source) group, f += 1/2 ||r||^2
    launch_residual_25d(*P, c.u, rec_idx, nrec, (const double2*)d_obs, c.ck, c.slot_f, c.slot_s, nsrc, nk, ng, c.res,
                        c.f_slot, c.st);
    launch_sum_f(c.f_slot, c.ident, ng, f_out, 1, c.st);
    // v_i = -H(k_i)^{-H} P_r^T (c_i r), g += w^2 Re(conj(u_i) v_i)
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_spread_25d(*P, c.res, rec_idx, nrec, c.ck, c.slot_f, nk, nb, c.q, c.st);
    st = solve_batch(c, 1, c.q, c.v, nb, ra);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    merge_reports(rep, ra);
    launch_grad_accum(c.u, nullptr, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
    for (auto& r : rep) result = worst(result, r.status);
    fill_reports(reports, gl, rep);
  }
  launch_extend_adjoint(*P, c.gcomp, g_out, c.st);
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

int helm_wri_misfit_and_gradient(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq,
                                 const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                                 const int32_t* rec_idx, int nrec, const void* d_obs, double lambda, double cg_tol,
                                 int cg_maxit, double* f_out, double* g_out, void* ws, size_t ws_bytes,
                                 helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx("helm_wri_misfit_and_gradient");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!src_idx || n_srcloc < 1 || !Q || !rec_idx || nrec < 1 || !d_obs || !f_out || !g_out) return HELM_E_INVAL;
  if (!(lambda > 0.0) || !std::isfinite(lambda) || !(cg_tol > 0.0) || !std::isfinite(cg_tol) || cg_maxit < 1)
    return HELM_E_INVAL;
  Ctx c;
  if ((st = bind(P, HELM_CALL_WRI, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, src_idx, n_srcloc, rec_idx, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  const double inv_l2 = 1.0 / (lambda * lambda);
  if (reports)
    for (int i = 0; i < nrhs; ++i) reports[i] = helm_rhs_report{HELM_OK, 0, 0, 0.0};
  cudaMemsetAsync(c.gcomp, 0, sizeof(double) * n, c.st);
  cudaMemsetAsync(f_out, 0, sizeof(double), c.st);
  int result = HELM_OK;
  for (int start = 0; start < nrhs; start += c.B) {
    const int nb = std::min(c.B, nrhs - start);
    std::vector<int> g(nb);
    for (int a = 0; a < nb; ++a) g[a] = start + a;
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    std::vector<SlotReport> rep, r2;
    // slots whose conjugate gradients still run (all in the first iteration, so
    // every slot's correction field is defined; converged slots then stop
    // taking solves and their reports stop changing)
    std::vector<int> live(nb);
    for (int a = 0; a < nb; ++a) live[a] = a;
    auto solve = [&](int dir, const double2* rhs, double2* out) {
      st = solve_batch(c, dir, rhs, out, nb, r2, &live);
      if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return false;
      result = worst(result, st);
      merge_reports(rep, r2);
      return true;
    };
    auto sources = [&]() {
      cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
      launch_sources(*P, src_idx, n_srcloc, (const double2*)Q, nsrc, (const double2*)wavelet, c.slot_f, c.slot_s,
                     nb, c.q, c.err + 1, c.st);
    };
    // u0 = H^{-1} q; receiver residual r0 = d - P_r u0
    sources();
    st = solve_batch(c, 0, c.q, c.u, nb, rep);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    launch_residual_misfit(*P, c.u, rec_idx, nrec, (const double2*)d_obs, c.slot_f, c.slot_s, nsrc, c.ident, nb,
                           c.res, c.f_slot, c.st);
    launch_wri_init(c.res, nrec, nb, c.cgR, c.cgP, c.rho, c.rho0, c.st);
    cudaMemsetAsync(c.acc, 0, sizeof(double2) * nb * n, c.st);
    // conjugate gradients on (I + lambda^-2 P_r H^{-1} H^{-H} P_r^T) z = r0; the field
    // correction H^{-1} H^{-H} P_r^T z accumulates from the same steps
    const double thr2 = cg_tol * cg_tol;
    std::vector<double> rh(nb), r0h(nb);
    bool converged = false;
    for (int it = 0; it < cg_maxit && !converged; ++it) {
      cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
      launch_spread(*P, c.cgP, nrec, rec_idx, nrec, 1.0, c.ident, nb, c.q, c.st);
      if (!solve(1, c.q, c.v)) return st;   // w = H^{-H} P_r^T p
      if (!solve(0, c.v, c.du)) return st;  // v = H^{-1} w
      launch_wri_ap(*P, c.du, rec_idx, nrec, inv_l2, c.cgP, c.cgAP, c.rho, c.rho0, thr2, c.alpha, nb, c.st);
      launch_axpy_slots(c.du, c.alpha, 0.0, n, nb, c.acc, c.st);
      launch_wri_step(nrec, nb, c.cgR, c.cgP, c.cgAP, c.alpha, c.rho, c.st);
      cudaMemcpyAsync(rh.data(), c.rho, sizeof(double) * nb, cudaMemcpyDeviceToHost, c.st);
      cudaMemcpyAsync(r0h.data(), c.rho0, sizeof(double) * nb, cudaMemcpyDeviceToHost, c.st);
      if (const int sc = sync_check(c); sc != HELM_OK) return sc;
      live.clear();
      for (int a = 0; a < nb; ++a) {
        if (!std::isfinite(rh[a])) return HELM_E_NONFINITE;
        if (rh[a] > thr2 * r0h[a]) live.push_back(a);
      }
      converged = live.empty();
    }
    for (int a = 0; a < nb; ++a)
      if (rh[a] > thr2 * r0h[a] && r0h[a] > 0.0) rep[a].status = worst(rep[a].status, HELM_E_NOCONV);
    // u = u0 + lambda^-2 acc; y = q - H u (FP64); f and g
    launch_axpy_slots(c.acc, nullptr, inv_l2, n, nb, c.u, c.st);
    sources();
    std::vector<int> all(nb);
    for (int a = 0; a < nb; ++a) all[a] = a;
    set_active(c, all);
    launch_stencil<double>(op_view<double>(c, 0, 0), c.slot_f, c.act, c.na, c.u, Scale<double>{}, c.q,
                           Scale<double>{}, c.v, c.st);
    launch_sqnorm(c.v, n, nb, c.partial, c.sq, c.st);
    launch_residual_misfit(*P, c.u, rec_idx, nrec, (const double2*)d_obs, c.slot_f, c.slot_s, nsrc, c.ident, nb,
                           c.res, c.f_slot, c.st);
    launch_wri_f(c.f_slot, c.sq, nb, lambda * lambda, f_out, c.st);
    // H u - q = -y:  g += lambda^2 w^2 Re(conj(u) (H u - q))
    launch_grad_accum(c.u, nullptr, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st, -lambda * lambda);
    for (auto& r : rep) result = worst(result, r.status);
    fill_reports(reports, g, rep);
  }
  launch_extend_adjoint(*P, c.gcomp, g_out, c.st);
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

int helm_hessvec(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq, const int32_t* src_idx,
                 int n_srcloc, const void* Q, int nsrc, const void* wavelet, const int32_t* rec_idx, int nrec,
                 const void* d_obs, const double* dm_phys, const uint8_t* mask, double* Hdm_out, void* ws,
                 size_t ws_bytes, helm_rhs_report* reports, helm_stream_t stream) {
  return linearised(3, P, m_phys, freqs_hz, nfreq, src_idx, n_srcloc, Q, nsrc, wavelet, rec_idx, nrec, dm_phys,
                    d_obs, mask, nullptr, Hdm_out, ws, ws_bytes, reports, stream);
}

int helm_gn_hessvec(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq, const int32_t* src_idx,
                    int n_srcloc, const void* Q, int nsrc, const void* wavelet, const int32_t* rec_idx, int nrec,
                    const double* dm_phys, const uint8_t* mask, double* Hdm_out, void* ws, size_t ws_bytes,
                    helm_rhs_report* reports, helm_stream_t stream) {
  return linearised(2, P, m_phys, freqs_hz, nfreq, src_idx, n_srcloc, Q, nsrc, wavelet, rec_idx, nrec, dm_phys,
                    nullptr, mask, nullptr, Hdm_out, ws, ws_bytes, reports, stream);
}

int helm_misfit(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq, const int32_t* src_idx,
                int n_srcloc, const void* Q, int nsrc, const void* wavelet, const int32_t* rec_idx, int nrec,
                const void* d_obs, const uint8_t* mask, double* f_out, void* R_out, void* U_out, int u_type,
                void* ws, size_t ws_bytes, helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx("helm_misfit");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!src_idx || n_srcloc < 1 || !Q || !rec_idx || nrec < 1 || !d_obs || !f_out) return HELM_E_INVAL;
  if (u_type != HELM_FIELD_C128 && u_type != HELM_FIELD_C64) return HELM_E_INVAL;
  Ctx c;
  if ((st = bind(P, HELM_CALL_MISFIT, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, src_idx, n_srcloc, rec_idx, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  std::vector<int> todo;
  if ((st = mask_list(c, mask, nrhs, todo)) != HELM_OK) return st;
  if (reports)
    for (int i = 0; i < nrhs; ++i) reports[i] = helm_rhs_report{HELM_OK, 0, 0, 0.0};
  cudaMemsetAsync(f_out, 0, sizeof(double), c.st);
  if (R_out) cudaMemsetAsync(R_out, 0, sizeof(double2) * (size_t)nrhs * nrec, c.st);
  int result = HELM_OK;
  for (size_t start = 0; start < todo.size(); start += c.B) {
    const int nb = (int)std::min<size_t>(c.B, todo.size() - start);
    std::vector<int> g(todo.begin() + start, todo.begin() + start + nb);
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_sources(*P, src_idx, n_srcloc, (const double2*)Q, nsrc, (const double2*)wavelet, c.slot_f, c.slot_s, nb,
                   c.q, c.err + 1, c.st);
    std::vector<SlotReport> rep;
    st = solve_batch(c, 0, c.q, c.u, nb, rep);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    for (auto& r : rep) result = worst(result, r.status);
    launch_residual_misfit(*P, c.u, rec_idx, nrec, (const double2*)d_obs, c.slot_f, c.slot_s, nsrc, c.ident, nb,
                           c.res, c.f_slot, c.st);
    launch_sum_f(c.f_slot, c.ident, nb, f_out, 1, c.st);
    if (R_out) launch_copy_fields(c.res, (double2*)R_out, c.ident, nb, c.slot_g, (size_t)nrec, c.st);
    if (U_out && u_type == HELM_FIELD_C64)
      launch_copy_fields(c.u, (float2*)U_out, c.ident, nb, c.slot_g, n, c.st);
    else if (U_out)
      launch_copy_fields(c.u, (double2*)U_out, c.ident, nb, c.slot_g, n, c.st);
    fill_reports(reports, g, rep);
  }
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

int helm_gradient(helm_plan* P, const double* m_phys, const double* freqs_hz, int nfreq, const int32_t* rec_idx,
                  int nrec, const void* R_in, int nsrc, const void* U_in, int u_type, const uint8_t* mask,
                  double* g_out, void* ws, size_t ws_bytes, helm_rhs_report* reports, helm_stream_t stream) {
  NvtxRange nvtx("helm_gradient");
  int st = check_common(P, m_phys, freqs_hz, nfreq, nsrc);
  if (st != HELM_OK) return st;
  if (!rec_idx || nrec < 1 || !R_in || !U_in || !g_out) return HELM_E_INVAL;
  if (u_type != HELM_FIELD_C128 && u_type != HELM_FIELD_C64) return HELM_E_INVAL;
  Ctx c;
  if ((st = bind(P, HELM_CALL_GRADIENT, nfreq, nsrc, nrec, ws, ws_bytes, stream, c)) != HELM_OK) return st;
  if ((st = setup_operator(c, m_phys, freqs_hz)) != HELM_OK) return st;
  if ((st = check_indices(c, nullptr, 0, rec_idx, nrec)) != HELM_OK) return st;
  const int nrhs = nfreq * nsrc;
  const size_t n = P->lev[0].n;
  std::vector<int> todo;
  if ((st = mask_list(c, mask, nrhs, todo)) != HELM_OK) return st;
  if (reports)
    for (int i = 0; i < nrhs; ++i) reports[i] = helm_rhs_report{HELM_OK, 0, 0, 0.0};
  cudaMemsetAsync(c.gcomp, 0, sizeof(double) * n, c.st);
  int result = HELM_OK;
  for (size_t start = 0; start < todo.size(); start += c.B) {
    const int nb = (int)std::min<size_t>(c.B, todo.size() - start);
    std::vector<int> g(todo.begin() + start, todo.begin() + start + nb);
    if ((st = set_batch(c, g)) != HELM_OK) return st;
    // adjoint source -P_r^T R and the adjoint state v = H^{-H}(-P_r^T R)
    cudaMemsetAsync(c.q, 0, sizeof(double2) * nb * n, c.st);
    launch_spread(*P, (const double2*)R_in, nrec, rec_idx, nrec, -1.0, c.slot_g, nb, c.q, c.st);
    std::vector<SlotReport> rep;
    st = solve_batch(c, 1, c.q, c.v, nb, rep);
    if (st == HELM_E_CUDA || st == HELM_E_TIMEOUT) return st;
    result = worst(result, st);
    for (auto& r : rep) result = worst(result, r.status);
    if (u_type == HELM_FIELD_C64)
      launch_grad_accum((const float2*)U_in, c.slot_g, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
    else
      launch_grad_accum((const double2*)U_in, c.slot_g, c.v, c.w2_64, c.slot_f, c.ident, nb, n, c.gcomp, c.st);
    fill_reports(reports, g, rep);
  }
  launch_extend_adjoint(*P, c.gcomp, g_out, c.st);
  if (const int sc = final_check(c); sc != HELM_OK) return sc;
  return result;
}

#ifdef HELM_DEBUG
int helm_debug_guard_selftest(helm_plan* P, void* ws, size_t ws_bytes, helm_stream_t stream) {
  if (!P) return HELM_E_INVAL;
  Ctx c;
  int st = bind(P, HELM_CALL_APPLY, 1, 1, 0, ws, ws_bytes, stream, c);
  if (st != HELM_OK) return st;
  cudaMemsetAsync(c.err, 0, 8 * sizeof(int), c.st);  // no operator set-up here to clear the counters
  if ((st = final_check(c)) != HELM_OK) return st;  // freshly armed guards are intact
  if (c.guards.empty()) return HELM_E_CUDA;
  // a stray one-byte write just past the first array, from the host API
  const unsigned char stray = 0x5A;
  if (cudaMemcpyAsync(c.ws_base + c.guards[0], &stray, 1, cudaMemcpyHostToDevice, c.st) != cudaSuccess)
    return HELM_E_CUDA;
  return final_check(c);
}
#endif

const char* helm_status_string(int s) {
  switch (s) {
    case HELM_OK: return "ok";
    case HELM_E_INVAL: return "invalid argument";
    case HELM_E_NOMEM: return "workspace too small";
    case HELM_E_CUDA: return "CUDA error";
    case HELM_E_NOCONV: return "solve did not reach its tolerance";
    case HELM_E_NONFINITE: return "non-finite residual";
    case HELM_E_TIMEOUT: return "device wait timed out";
    case HELM_E_BOUNDS: return "debug build: write outside a workspace array or slot index out of range";
    default: return "unknown status";
  }
}

uint64_t helm_kernel_launch_count(void) { return g_launches.load(); }

int helm_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  drain_records();
  for (int i = 0; i < PC_COUNT; ++i) {
    g_prof_n[i] = 0;
    g_prof_ms[i] = 0.0;
    g_prof_bytes[i] = 0.0;
  }
  g_prof_on = on != 0;
  return HELM_OK;
}

int helm_profile_read(int cls, uint64_t* launches, double* ms, double* bytes) {
  if (cls < 0 || cls >= PC_COUNT) return HELM_E_INVAL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  drain_records();
  if (launches) *launches = g_prof_n[cls];
  if (ms) *ms = g_prof_ms[cls];
  if (bytes) *bytes = g_prof_bytes[cls];
  return HELM_OK;
}

}  // extern "C"
