// Host orchestration of the batched Helmholtz solves.
//
//  * krylov():  restarted GMRES / FGMRES (Saad & Schultz 1986; Saad 1993),
//               Arnoldi with CGS2, right preconditioning, per-slot residual
//               tracking.  Tolerance-driven solves read per-slot residuals
//               once per restart cycle and drop converged right-hand sides
//               from the active list (the per-RHS convergence mask).
//  * vcycle():  the ML-GMRES preconditioner of Sec. 4 (Alg. vcycle, Fig.
//               mlgmres): GMRES(k_so, k_si) smoothing with identity
//               preconditioner, residual, full-weighting restriction, coarse
//               FGMRES(k_co, k_ci) recursively preconditioned by the same
//               cycle (plain GMRES on the last level), linear prolongation,
//               post-smoothing.  The cycle starts from a zero guess.
//  * damped Jacobi as the plain alternative preconditioner.
//  * solve_batch(): FP64 solves, or complex64 inner solves inside FP64
//               iterative refinement (outer residual r = q - H u and the
//               update u += e in FP64).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "reduce.cuh"
#include "solver.h"

// 1: the first Gram-Schmidt pass of each Arnoldi step is folded into the
// stencil launch; 0: it runs as its own streaming pass.
#ifndef HELM_FUSE_DOTS
#define HELM_FUSE_DOTS 1
#endif

namespace helm {

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------

template <typename R>
static void layout_krylov(Bump& bp, KInst<R>& I, int level, int k, bool flex, int B, size_t n) {
  I.level = level;
  I.k = k;
  I.flex = flex;
  I.V = bp.take<cplx<R>>((size_t)(k + 1) * B * n);
  I.Z = flex ? bp.take<cplx<R>>((size_t)k * B * n) : nullptr;
  I.w = bp.take<cplx<R>>((size_t)B * n);
  const size_t K1 = KMAX + 1;
  I.ks.H = bp.take<double2>((size_t)B * K1 * KMAX);
  I.ks.cs = bp.take<double2>((size_t)B * KMAX);
  I.ks.sn = bp.take<double2>((size_t)B * KMAX);
  I.ks.g = bp.take<double2>((size_t)B * K1);
  I.ks.hcol = bp.take<double2>((size_t)B * K1);
  I.ks.scale = bp.take<double>((size_t)B * K1);
  I.ks.bnorm = bp.take<double>(B);
  I.ks.rnorm = bp.take<double>(B);
  I.ks.est = bp.take<double>(B);
  I.ks.coef = bp.take<cplx<R>>((size_t)B * K1);
  I.ks.scale_r = bp.take<R>((size_t)B * K1);
}

template <typename R>
static void layout_hierarchy(Bump& bp, const helm_plan& P, Hierarchy<R>& H, int B, bool outer = true) {
  const helm_solve_opts& o = P.o;
  const size_t n0 = P.lev[0].n;
  const bool flex0 = o.precond != HELM_PRECOND_NONE;
  if (outer) layout_krylov<R>(bp, H.inst[0], 0, o.k_inner, flex0, B, n0);
  if (o.precond == HELM_PRECOND_JACOBI) {
    H.r[0] = bp.take<cplx<R>>((size_t)B * n0);
  } else if (o.precond == HELM_PRECOND_MLGMRES) {
    // inst 1: smoother on level 0; inst 2: coarse solver on level 1;
    // inst 3: smoother on level 1; inst 4: coarse solver on level 2.
    layout_krylov<R>(bp, H.inst[1], 0, o.k_si, false, B, n0);
    H.r[0] = bp.take<cplx<R>>((size_t)B * n0);
    const size_t n1 = P.lev[1].n;
    layout_krylov<R>(bp, H.inst[2], 1, o.k_ci, P.L > 2, B, n1);
    H.b[1] = bp.take<cplx<R>>((size_t)B * n1);
    H.x[1] = bp.take<cplx<R>>((size_t)B * n1);
    if (P.L > 2) {
      const size_t n2 = P.lev[2].n;
      layout_krylov<R>(bp, H.inst[3], 1, o.k_si, false, B, n1);
      H.r[1] = bp.take<cplx<R>>((size_t)B * n1);
      layout_krylov<R>(bp, H.inst[4], 2, o.k_ci, false, B, n2);
      H.b[2] = bp.take<cplx<R>>((size_t)B * n2);
      H.x[2] = bp.take<cplx<R>>((size_t)B * n2);
    }
  }
}

static size_t layout_body(const helm_plan& P, int call, int nfreq, int nsrc, int nrec, Bump& bp, Ctx& C);

size_t layout(const helm_plan& P, int call, int nfreq, int nsrc, int nrec, char* base, Ctx* c) {
  Ctx local;
  Ctx& C = c ? *c : local;
  Bump bp;
  bp.base = base;
  C.guards.clear();
  bp.guards = &C.guards;
  layout_body(P, call, nfreq, nsrc, nrec, bp, C);
#ifdef HELM_DEBUG
  // the device copy of the guard list (its own band is not in the list)
  const size_t ng = C.guards.size();
  C.guards_dev = bp.take<size_t>(ng > 0 ? ng : 1);
  C.guards.resize(ng);
#endif
  C.ws_base = base;
  return bp.off;
}

static size_t layout_body(const helm_plan& P, int call, int nfreq, int nsrc, int nrec, Bump& bp, Ctx& C) {
  const int nrhs = nfreq * nsrc;
  int B = nrhs;
  if (call != HELM_CALL_APPLY && P.o.max_batch > 0 && P.o.max_batch < B) B = P.o.max_batch;
  if (B < 1) B = 1;
  C.P = &P;
  C.call = call;
  C.nfreq = nfreq;
  C.nsrc = nsrc;
  C.nrec = nrec;
  C.B = B;
  C.mixed = P.o.precision == HELM_MIXED;
  const int L = (call == HELM_CALL_APPLY) ? 1 : P.L;
  for (int l = 0; l < L; ++l) {
    const size_t n = P.lev[l].n;
    const size_t tn = (size_t)nfreq * 9 * P.lev[l].Nmax;
    C.m64[l] = bp.take<double>(n);
    C.m32[l] = bp.take<float>(n);
    for (int d = 0; d < 2; ++d) {
      C.tab64[l][d] = bp.take<double2>(tn);
      C.tab32[l][d] = bp.take<float2>(tn);
    }
  }
  C.omega = bp.take<double>(nfreq);
  C.w2_64 = bp.take<double>(nfreq);
  C.w2_32 = bp.take<float>(nfreq);
  C.slot_f = bp.take<int>(B);
  C.slot_s = bp.take<int>(B);
  C.slot_g = bp.take<int>(B);
  C.act = bp.take<int>(B);
  C.ident = bp.take<int>(B);
  C.err = bp.take<int>(8);
  if (call == HELM_CALL_APPLY) return bp.off;
  // partial rows: at most max(RED_BLOCKS_MAX, B) rows of at most max(2(KMAX+1), Gram) values
  C.partial = bp.take<double>((size_t)std::max(RED_BLOCKS_MAX, B) *
                              std::max(2 * (KMAX + 1), gram_nvals(SSTEP_MAX)));
  C.counter = bp.take<unsigned>(B);
  if (call == HELM_CALL_PRECOND) {
    // the preconditioner's own levels only (no outer basis, no FP64 fields)
    if (C.mixed) layout_hierarchy<float>(bp, P, C.h32, B, false);
    else layout_hierarchy<double>(bp, P, C.h64, B, false);
    return bp.off;
  }
  const size_t n0 = P.lev[0].n;
  C.q = bp.take<double2>((size_t)B * n0);
  C.u = bp.take<double2>((size_t)B * n0);
  const bool born = call == HELM_CALL_BORN || call == HELM_CALL_BORN_ADJOINT || call == HELM_CALL_GN_HESSVEC ||
                    call == HELM_CALL_HESSVEC || call == HELM_CALL_MISFIT_GRAD_25D || call == HELM_CALL_WRI;
  if (call == HELM_CALL_ADJOINT || call == HELM_CALL_MISFIT_GRAD || call == HELM_CALL_GRADIENT || born)
    C.v = bp.take<double2>((size_t)B * n0);
  C.nrm = bp.take<double>(B);
  C.qn = bp.take<double>(B);
  if (C.mixed) {
    C.r64 = bp.take<double2>((size_t)B * n0);
    C.b32 = bp.take<float2>((size_t)B * n0);
    C.x32 = bp.take<float2>((size_t)B * n0);
    layout_hierarchy<float>(bp, P, C.h32, B);
  } else {
    layout_hierarchy<double>(bp, P, C.h64, B);
  }
  if (call == HELM_CALL_MISFIT_GRAD_25D) {
    C.shift = bp.take<double>(nfreq);
    C.ck = bp.take<double>(nfreq);
    C.wav = bp.take<double2>(nfreq);
  }
  if (call == HELM_CALL_MISFIT_GRAD || call == HELM_CALL_MISFIT || call == HELM_CALL_HESSVEC ||
      call == HELM_CALL_MISFIT_GRAD_25D || call == HELM_CALL_WRI) {
    C.res = bp.take<double2>((size_t)B * (nrec > 0 ? nrec : 1));
    C.f_slot = bp.take<double>(B);
  }
  if (call == HELM_CALL_HESSVEC || call == HELM_CALL_WRI) C.du = bp.take<double2>((size_t)B * n0);
  if (call == HELM_CALL_WRI) {
    const size_t nr = (size_t)B * (nrec > 0 ? nrec : 1);
    C.acc = bp.take<double2>((size_t)B * n0);
    C.cgR = bp.take<double2>(nr);
    C.cgP = bp.take<double2>(nr);
    C.cgAP = bp.take<double2>(nr);
    C.rho = bp.take<double>(B);
    C.rho0 = bp.take<double>(B);
    C.alpha = bp.take<double>(B);
    C.sq = bp.take<double>(B);
  }
  if (call == HELM_CALL_MISFIT_GRAD || call == HELM_CALL_GRADIENT || call == HELM_CALL_BORN_ADJOINT ||
      call == HELM_CALL_GN_HESSVEC || call == HELM_CALL_HESSVEC || call == HELM_CALL_MISFIT_GRAD_25D ||
      call == HELM_CALL_WRI)
    C.gcomp = bp.take<double>(n0);
  if (call == HELM_CALL_GN_HESSVEC) C.res = bp.take<double2>((size_t)B * (nrec > 0 ? nrec : 1));
  if (call == HELM_CALL_BORN || call == HELM_CALL_GN_HESSVEC || call == HELM_CALL_HESSVEC)
    C.dmc = bp.take<double>(n0);
  return bp.off;
}

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------

template <typename R> OpView<R> op_view(const Ctx& c, int level, int dir);
template <> OpView<float> op_view<float>(const Ctx& c, int level, int dir) {
  const LevelGeom& L = c.P->lev[level];
  OpView<float> v;
  v.tab = c.tab32[level][dir];
  v.m = c.m32[level];
  v.w2 = c.w2_32;
  for (int d = 0; d < 3; ++d) v.K[d] = L.K[d];
  v.n = L.n;
  v.Nmax = L.Nmax;
  return v;
}
template <> OpView<double> op_view<double>(const Ctx& c, int level, int dir) {
  const LevelGeom& L = c.P->lev[level];
  OpView<double> v;
  v.tab = c.tab64[level][dir];
  v.m = c.m64[level];
  v.w2 = c.w2_64;
  for (int d = 0; d < 3; ++d) v.K[d] = L.K[d];
  v.n = L.n;
  v.Nmax = L.Nmax;
  return v;
}

int sync_check(Ctx& c) {
  cudaError_t e = cudaStreamSynchronize(c.st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return HELM_E_CUDA;
  if (c.err) {
    // err[3]: a kernel gave up on a bounded wait (results of the call are void)
    int gave_up = 0;
    if (cudaMemcpyAsync(&gave_up, c.err + 3, sizeof(int), cudaMemcpyDeviceToHost, c.st) != cudaSuccess ||
        cudaStreamSynchronize(c.st) != cudaSuccess)
      return HELM_E_CUDA;
    if (gave_up) return HELM_E_TIMEOUT;
  }
  return HELM_OK;
}

#ifdef HELM_DEBUG
// One block per guard band: any byte that is not the guard pattern marks err[2].
__global__ void k_check_guards(const unsigned char* __restrict__ base, const size_t* __restrict__ guards,
                               int* __restrict__ bad) {
  const unsigned char* g = base + guards[blockIdx.x];
  for (unsigned i = threadIdx.x; i < kGuardBytes; i += blockDim.x)
    if (g[i] != kGuardByte) atomicOr(bad, 1);
}
#endif

int arm_guards(Ctx& c) {
#ifdef HELM_DEBUG
  if (!c.ws_base) return HELM_OK;
  for (size_t off : c.guards) cudaMemsetAsync(c.ws_base + off, kGuardByte, kGuardBytes, c.st);
  if (!c.guards.empty())
    cudaMemcpyAsync(c.guards_dev, c.guards.data(), sizeof(size_t) * c.guards.size(), cudaMemcpyHostToDevice, c.st);
  c.host_fault = false;
  return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_E_CUDA;
#else
  (void)c;
  return HELM_OK;
#endif
}

int final_check(Ctx& c) {
  int st = sync_check(c);
  if (st != HELM_OK) return st;
#ifdef HELM_DEBUG
  if (c.ws_base && !c.guards.empty()) {
    cudaMemsetAsync(c.err + 2, 0, sizeof(int), c.st);
    k_check_guards<<<(unsigned)c.guards.size(), 64, 0, c.st>>>((const unsigned char*)c.ws_base, c.guards_dev,
                                                              c.err + 2);
    count_launch();
    int bad = 0;
    if (cudaMemcpyAsync(&bad, c.err + 2, sizeof(int), cudaMemcpyDeviceToHost, c.st) != cudaSuccess ||
        cudaStreamSynchronize(c.st) != cudaSuccess)
      return HELM_E_CUDA;
    if (bad) return HELM_E_BOUNDS;
  }
  if (c.host_fault) return HELM_E_BOUNDS;
#endif
  return HELM_OK;
}

void set_active(Ctx& c, const std::vector<int>& a) {
#ifdef HELM_DEBUG
  for (int s : a)
    if (s < 0 || s >= c.B) c.host_fault = true;
#endif
  c.act_h = a;
  c.na = (int)a.size();
  if (c.na > 0)
    cudaMemcpyAsync(c.act, a.data(), sizeof(int) * a.size(), cudaMemcpyHostToDevice, c.st);
}

int setup_operator(Ctx& c, const double* m_phys, const double* freqs_hz) {
  const helm_plan& P = *c.P;
  const int L = c.call == HELM_CALL_APPLY ? 1 : P.L;
  std::vector<double> om(c.nfreq), w2(c.nfreq);
  std::vector<float> w2f(c.nfreq);
  for (int k = 0; k < c.nfreq; ++k) {
    om[k] = 2.0 * M_PI * freqs_hz[k];
    w2[k] = om[k] * om[k];
    w2f[k] = (float)w2[k];
  }
  cudaMemcpyAsync(c.omega, om.data(), sizeof(double) * c.nfreq, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.w2_64, w2.data(), sizeof(double) * c.nfreq, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.w2_32, w2f.data(), sizeof(float) * c.nfreq, cudaMemcpyHostToDevice, c.st);
  std::vector<int> id(c.B);
  for (int i = 0; i < c.B; ++i) id[i] = i;
  cudaMemcpyAsync(c.ident, id.data(), sizeof(int) * c.B, cudaMemcpyHostToDevice, c.st);
  cudaMemsetAsync(c.err, 0, 8 * sizeof(int), c.st);
  if (c.counter) cudaMemsetAsync(c.counter, 0, sizeof(unsigned) * c.B, c.st);
  launch_extend(P, m_phys, c.m64[0], c.m32[0], c.st);
  for (int l = 1; l < L; ++l) {
    launch_restrict_model(c.m64[l - 1], P.lev[l - 1], c.m64[l], P.lev[l], c.st);
    launch_copy_m32(c.m64[l], c.m32[l], P.lev[l].n, c.st);
  }
  for (int l = 0; l < L; ++l)
    launch_tables(P, l, c.omega, c.nfreq, c.tab64[l][0], c.tab64[l][1], c.tab32[l][0], c.tab32[l][1], c.st,
                  c.shift);
  return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_E_CUDA;
}

int set_batch_fs(Ctx& c, const std::vector<int>& g, const std::vector<int>& f, const std::vector<int>& s) {
  const int nb = (int)g.size();
#ifdef HELM_DEBUG
  if (nb > c.B) c.host_fault = true;
  for (int a = 0; a < nb; ++a)
    if (f[a] < 0 || f[a] >= c.nfreq || s[a] < 0 || s[a] >= c.nsrc) c.host_fault = true;
#endif
  cudaMemcpyAsync(c.slot_f, f.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.slot_s, s.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.slot_g, g.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.st);
  std::vector<int> a(nb);
  for (int i = 0; i < nb; ++i) a[i] = i;
  set_active(c, a);
  return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_E_CUDA;
}

int set_batch(Ctx& c, const std::vector<int>& g) {
  const int nb = (int)g.size();
#ifdef HELM_DEBUG
  if (nb > c.B) c.host_fault = true;
  for (int v : g)
    if (v < 0 || v >= c.nfreq * c.nsrc) c.host_fault = true;
#endif
  std::vector<int> f(nb), s(nb);
  for (int a = 0; a < nb; ++a) {
    f[a] = g[a] / c.nsrc;
    s[a] = g[a] % c.nsrc;
  }
  cudaMemcpyAsync(c.slot_f, f.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.slot_s, s.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.st);
  cudaMemcpyAsync(c.slot_g, g.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.st);
  std::vector<int> a(nb);
  for (int i = 0; i < nb; ++i) a[i] = i;
  set_active(c, a);
  return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_E_CUDA;
}

template <typename R> static Hierarchy<R>& hier(Ctx& c);
template <> Hierarchy<float>& hier<float>(Ctx& c) { return c.h32; }
template <> Hierarchy<double>& hier<double>(Ctx& c) { return c.h64; }


static Epi make_epi(Ctx& c, int kind, const KState* ks = nullptr) {
  Epi e;
  e.kind = kind;
  if (ks) e.ks = *ks;
  e.counter = c.counter;
  e.partial = c.partial;
  e.fault = c.err ? c.err + 3 : nullptr;
  return e;
}

// ||bs*b|| of every active slot into out[slot]
template <typename R>
static void norms(Ctx& c, const cplx<R>* b, Scale<R> bs, size_t n, double* out) {
  Epi e = make_epi(c, EPI_NORM);
  e.out = out;
  launch_gs<R>(GS_SUB_STORE_NORM, nullptr, 0, 0, nullptr, b, bs, nullptr, c.act, c.na, n, e, c.st);
}

using Prec32 = std::function<void(const cplx<float>*, Scale<float>, cplx<float>*)>;
using Prec64 = std::function<void(const cplx<double>*, Scale<double>, cplx<double>*)>;
template <typename R> struct PrecT;
template <> struct PrecT<float> { using T = Prec32; };
template <> struct PrecT<double> { using T = Prec64; };

struct KrylovOut {
  std::vector<int> iters;  // per slot
  int cycles = 0;
};

// Restarted (F)GMRES on level I.level for the active slots:
// solves H x = bs*b.  tol > 0: tolerance-driven (host reads residuals each
// cycle and narrows the active list; the caller's list is restored on exit);
// tol == 0: exactly `cycles` cycles without host synchronisation.
template <typename R>
static int krylov(Ctx& c, KInst<R>& I, const cplx<R>* b, Scale<R> bs, cplx<R>* x, bool x0_zero,
                  int cycles, double tol, const typename PrecT<R>::T* prec, KrylovOut* out,
                  bool final_resid = false) {
  const OpView<R> op = op_view<R>(c, I.level, c.dir);
  const size_t n = op.n;
  const size_t vs = (size_t)c.B * n;  // stride between basis vectors
  const int K1 = KMAX + 1;
  const std::vector<int> saved = c.act_h;
  const bool reorth = c.P->o.reorth != 0;
  int status = HELM_OK;
  if (x0_zero) launch_zero<R>(x, c.act, c.na, n, c.st);
  if (tol > 0.0 && !x0_zero) norms<R>(c, b, bs, n, I.ks.bnorm);
  std::vector<double> rn(c.B), bn(c.B);
  const bool flex = I.flex && prec;
  for (int cyc = 0; cyc < cycles && c.na > 0; ++cyc) {
    // start vector V_0 = bs*b - H x (a plain copy while x is zero) and beta = ||V_0||
    Epi es = make_epi(c, EPI_START, &I.ks);
    es.set_bnorm = (tol > 0.0 && cyc == 0 && x0_zero) ? 1 : 0;
    if (cyc == 0 && x0_zero)
      launch_gs<R>(GS_SUB_STORE_NORM, nullptr, 0, 0, nullptr, b, bs, I.V, c.act, c.na, n, es, c.st);
    else
      launch_stencil<R>(op, c.slot_f, c.act, c.na, x, Scale<R>{}, b, bs, I.V, c.st, &es);
    if (tol > 0.0) {
      cudaMemcpyAsync(rn.data(), I.ks.rnorm, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st);
      cudaMemcpyAsync(bn.data(), I.ks.bnorm, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st);
      if (const int sc = sync_check(c); sc != HELM_OK) return sc;
      std::vector<int> keep;
      for (int s : c.act_h) {
        if (!std::isfinite(rn[s])) { status = HELM_E_NONFINITE; continue; }
        if (rn[s] > tol * bn[s]) keep.push_back(s);
      }
      if (keep.size() != c.act_h.size()) set_active(c, keep);
      if (c.na == 0) break;
    }
    const cplx<R>* coef = (const cplx<R>*)I.ks.coef;
    for (int j = 0; j < I.k; ++j) {
      cplx<R>* Vj = I.V + (size_t)j * vs;
      const cplx<R>* zin = Vj;
      Scale<R> zs{(const R*)I.ks.scale_r + j, K1};
      if (flex) {
        cplx<R>* Zj = I.Z + (size_t)j * vs;
        (*prec)(Vj, zs, Zj);
        zin = Zj;
        zs = Scale<R>{};
      }
      // w = H z_j and the first Gram-Schmidt pass h = V^H w (folded into the
      // stencil, or as a separate streaming pass)
      Epi ed = make_epi(c, EPI_DOTS, &I.ks);
      ed.nv = j + 1;
      if (HELM_FUSE_DOTS) {
        launch_stencil<R>(op, c.slot_f, c.act, c.na, zin, zs, nullptr, Scale<R>{}, I.w, c.st, &ed, I.V, vs, j + 1);
      } else {
        launch_stencil<R>(op, c.slot_f, c.act, c.na, zin, zs, nullptr, Scale<R>{}, I.w, c.st);
        launch_gs<R>(GS_DOT, I.V, vs, j + 1, nullptr, I.w, Scale<R>{}, nullptr, c.act, c.na, n, ed, c.st);
      }
      if (reorth) {
        Epi e2 = make_epi(c, EPI_DOTS, &I.ks);
        e2.nv = j + 1;
        e2.accumulate = 1;
        launch_gs<R>(GS_SUB_DOT, I.V, vs, j + 1, coef, I.w, Scale<R>{}, nullptr, c.act, c.na, n, e2, c.st);
      }
      // v_{j+1} = w - V h, its norm, the Givens update (and the small solve after the last column)
      Epi ea = make_epi(c, EPI_ARNOLDI, &I.ks);
      ea.j = j;
      ea.ksolve = I.k;
      ea.flex = flex ? 1 : 0;
      launch_gs<R>(GS_SUB_STORE_NORM, I.V, vs, j + 1, coef, I.w, Scale<R>{}, I.V + (size_t)(j + 1) * vs, c.act,
                   c.na, n, ea, c.st);
    }
    launch_gs<R>(GS_ADD_STORE, flex ? I.Z : I.V, vs, I.k, coef, x, Scale<R>{}, x, c.act, c.na, n, Epi{}, c.st);
    if (out) {
      for (int s : c.act_h) out->iters[s] += I.k;
      out->cycles++;
    }
  }
  if (tol > 0.0) {
    set_active(c, saved);
    if (final_resid) {
      // final true residual norm for the caller's slots
      Epi en = make_epi(c, EPI_NORM);
      en.out = I.ks.rnorm;
      launch_stencil<R>(op, c.slot_f, c.act, c.na, x, Scale<R>{}, b, bs, I.w, c.st, &en);
    }
  }
  return status;
}

// s-step GMRES cycles (the same minimal-residual step as GMRES(k) from x, over
// the same Krylov space): W_0 = r = bs*b - H x, W_i = H W_{i-1} for i = 1..k,
// one Gram pass over W_0..W_k, the k x k normal equations in FP64 (diagonally
// scaled, so the basis needs no normalisation), x += sum_i y_i W_i.  A cycle
// streams k+3 passes instead of the ~k^2 of Gram-Schmidt.  Between cycles the
// next residual comes by recurrence, r = W_0 - sum_i y_i W_{i+1}, in the same
// pass as the update of x, so only the first cycle applies the stencil to x.
// With want_resid the last cycle also leaves that residual in W_0 and the
// function returns it (nullptr otherwise).
template <typename R>
static const cplx<R>* sstep(Ctx& c, KInst<R>& I, const cplx<R>* b, Scale<R> bs, cplx<R>* x, bool x0_zero,
                            int cycles, bool want_resid) {
  const OpView<R> op = op_view<R>(c, I.level, c.dir);
  const size_t n = op.n;
  const size_t vs = (size_t)c.B * n;
  const int S = I.k;
  if (cycles <= 0) {
    if (x0_zero) launch_zero<R>(x, c.act, c.na, n, c.st);
    return nullptr;
  }
  for (int cyc = 0; cyc < cycles && c.na > 0; ++cyc) {
    if (cyc == 0 && x0_zero) {
      // x = 0: the residual is bs*b itself; the first image is H(bs*b)
      launch_gs<R>(GS_ADD_STORE, nullptr, 0, 0, nullptr, b, bs, I.V, c.act, c.na, n, Epi{}, c.st);
    } else if (cyc == 0) {
      launch_stencil<R>(op, c.slot_f, c.act, c.na, x, Scale<R>{}, b, bs, I.V, c.st);
    }
    for (int i = 1; i <= S; ++i)
      launch_stencil<R>(op, c.slot_f, c.act, c.na, I.V + (size_t)(i - 1) * vs, Scale<R>{}, nullptr, Scale<R>{},
                        I.V + (size_t)i * vs, c.st);
    Epi eg = make_epi(c, EPI_GRAM, &I.ks);
    eg.idx = S;
    launch_gram<R>(I.V, vs, S, c.act, c.na, n, eg, c.st);
    const bool recur = cyc + 1 < cycles || want_resid;
    launch_sstep_update<R>(I.V, vs, S, (const cplx<R>*)I.ks.coef, x, c.act, c.na, n, recur ? 1 : 0,
                           (cyc == 0 && x0_zero) ? 1 : 0, c.st);
  }
  return want_resid ? I.V : nullptr;
}

// A fixed-cycle solve without preconditioner (smoother or last-level coarse
// solve): s-step cycles when enabled, Arnoldi otherwise.  With want_resid the
// s-step path returns the residual bs*b - H x it carries (nullptr when the
// caller has to form it).
template <typename R>
static const cplx<R>* fixed_solve(Ctx& c, KInst<R>& I, const cplx<R>* b, Scale<R> bs, cplx<R>* x, bool x0_zero,
                                  int cycles, bool want_resid = false) {
  if (c.P->o.sstep && I.k <= SSTEP_MAX) return sstep<R>(c, I, b, bs, x, x0_zero, cycles, want_resid);
  krylov<R>(c, I, b, bs, x, x0_zero, cycles, 0.0, nullptr, nullptr);
  return nullptr;
}

// ML-GMRES V-cycle at `level`: out = M^{-1}(ins*in), zero initial guess.
template <typename R>
static void vcycle(Ctx& c, int level, const cplx<R>* in, Scale<R> ins, cplx<R>* out) {
  const helm_plan& P = *c.P;
  const helm_solve_opts& o = P.o;
  Hierarchy<R>& H = hier<R>(c);
  KInst<R>& smooth = H.inst[level == 0 ? 1 : 3];
  KInst<R>& coarse = H.inst[level == 0 ? 2 : 4];
  const OpView<R> op = op_view<R>(c, level, c.dir);
  // pre-smoothing from zero; the residual (carried by the s-step smoother, or
  // formed here) is restricted to the next level
  const cplx<R>* r = fixed_solve<R>(c, smooth, in, ins, out, true, o.k_so, true);
  if (!r) {
    launch_stencil<R>(op, c.slot_f, c.act, c.na, out, Scale<R>{}, in, ins, H.r[level], c.st);
    r = H.r[level];
  }
  launch_restrict<R>(r, P.lev[level], H.b[level + 1], P.lev[level + 1], c.act, c.na, c.st);
  // coarse solve, recursively preconditioned except on the last level
  if (level + 1 < P.L - 1) {
    typename PrecT<R>::T pc = [&c, level](const cplx<R>* i2, Scale<R> s2, cplx<R>* o2) {
      vcycle<R>(c, level + 1, i2, s2, o2);
    };
    krylov<R>(c, coarse, H.b[level + 1], Scale<R>{}, H.x[level + 1], true, o.k_co, 0.0, &pc, nullptr);
  } else {
    fixed_solve<R>(c, coarse, H.b[level + 1], Scale<R>{}, H.x[level + 1], true, o.k_co);
  }
  launch_prolong_add<R>(H.x[level + 1], P.lev[level + 1], out, P.lev[level], c.act, c.na, c.st);
  // post-smoothing from the corrected guess
  fixed_solve<R>(c, smooth, in, ins, out, false, o.k_so);
}

// Damped Jacobi: sweeps of z += omega D^{-1}(ins*in - H z), from z = 0.
template <typename R>
static void jacobi(Ctx& c, const cplx<R>* in, Scale<R> ins, cplx<R>* out) {
  const helm_solve_opts& o = c.P->o;
  Hierarchy<R>& H = hier<R>(c);
  const OpView<R> op = op_view<R>(c, 0, c.dir);
  const R w = (R)o.jacobi_omega;
  launch_jacobi_first<R>(op, c.slot_f, c.act, c.na, in, ins, w, out, c.st);
  for (int sw = 1; sw < o.jacobi_sweeps; ++sw) {
    launch_stencil<R>(op, c.slot_f, c.act, c.na, out, Scale<R>{}, in, ins, H.r[0], c.st);
    launch_jacobi_update<R>(op, c.slot_f, c.act, c.na, H.r[0], w, out, c.st);
  }
}

// Outer tolerance-driven solve in precision R of H x = b (b, x in R), from
// x = 0 or (warm) from the x given.
template <typename R>
static int outer_solve(Ctx& c, const cplx<R>* b, cplx<R>* x, double tol, KrylovOut* ko, bool final_resid,
                       bool warm = false) {
  const helm_solve_opts& o = c.P->o;
  Hierarchy<R>& H = hier<R>(c);
  typename PrecT<R>::T pc;
  const typename PrecT<R>::T* pp = nullptr;
  if (o.precond == HELM_PRECOND_MLGMRES) {
    pc = [&c](const cplx<R>* i, Scale<R> s, cplx<R>* z) { vcycle<R>(c, 0, i, s, z); };
    pp = &pc;
  } else if (o.precond == HELM_PRECOND_JACOBI) {
    pc = [&c](const cplx<R>* i, Scale<R> s, cplx<R>* z) { jacobi<R>(c, i, s, z); };
    pp = &pc;
  }
  return krylov<R>(c, H.inst[0], b, Scale<R>{}, x, !warm, o.max_cycles, tol, pp, ko, final_resid);
}

template <typename R>
static void precond_apply_t(Ctx& c, const cplx<R>* x, cplx<R>* z) {
  const helm_solve_opts& o = c.P->o;
  if (o.precond == HELM_PRECOND_MLGMRES) {
    vcycle<R>(c, 0, x, Scale<R>{}, z);
  } else if (o.precond == HELM_PRECOND_JACOBI) {
    jacobi<R>(c, x, Scale<R>{}, z);
  } else {
    cudaMemcpyAsync(z, x, sizeof(cplx<R>) * (size_t)c.na * c.P->lev[0].n, cudaMemcpyDeviceToDevice, c.st);
  }
}

int precond_apply(Ctx& c, int dir, const void* x, void* z) {
  c.dir = dir;
  if (c.mixed)
    precond_apply_t<float>(c, (const float2*)x, (float2*)z);
  else
    precond_apply_t<double>(c, (const double2*)x, (double2*)z);
  return sync_check(c);
}

int solve_batch(Ctx& c, int dir, const double2* q, double2* u, int nb, std::vector<SlotReport>& rep,
                const std::vector<int>* only, bool warm) {
  NvtxRange nvtx(dir ? "adjoint solves" : "forward solves");
  const helm_plan& P = *c.P;
  const helm_solve_opts& o = P.o;
  c.dir = dir;
  const size_t n = P.lev[0].n;
  rep.assign(nb, SlotReport{});
  std::vector<int> all;
  if (only) {
    all = *only;
  } else {
    all.resize(nb);
    for (int i = 0; i < nb; ++i) all[i] = i;
  }
  const std::vector<int> solved = all;
  set_active(c, all);
  if (c.na == 0) return HELM_OK;
  KrylovOut ko;
  ko.iters.assign(c.B, 0);
  int st = HELM_OK;
  std::vector<double> rn(c.B, 0.0), qn(c.B, 0.0);
  const OpView<double> op64 = op_view<double>(c, 0, dir);
  norms<double>(c, q, Scale<double>{}, n, c.qn);
  if (!c.mixed) {
    st = outer_solve<double>(c, q, u, o.tol, &ko, true, warm);
    cudaMemcpyAsync(rn.data(), c.h64.inst[0].ks.rnorm, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st);
    cudaMemcpyAsync(qn.data(), c.qn, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st);
    for (int a : solved) rep[a].refine = 1;
  } else {
    // FP64 iterative refinement around complex64 inner solves:
    //   r = q - H u (FP64), e = H^{-1}(r/||r||) (complex64), u += ||r|| e (FP64)
    if (warm) {
      Epi e0 = make_epi(c, EPI_NORM);
      e0.out = c.nrm;
      launch_stencil<double>(op64, c.slot_f, c.act, c.na, u, Scale<double>{}, q, Scale<double>{}, c.r64, c.st, &e0);
    } else {
      launch_zero<double>(u, c.act, c.na, n, c.st);
      cudaMemcpyAsync(c.r64, q, sizeof(double2) * (size_t)nb * n, cudaMemcpyDeviceToDevice, c.st);
      cudaMemcpyAsync(c.nrm, c.qn, sizeof(double) * nb, cudaMemcpyDeviceToDevice, c.st);
    }
    for (int it = 0; it <= o.max_refine; ++it) {
      cudaMemcpyAsync(rn.data(), c.nrm, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st);
      cudaMemcpyAsync(qn.data(), c.qn, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st);
      if (const int sc = sync_check(c); sc != HELM_OK) return sc;
      std::vector<int> keep;
      for (int s : c.act_h) {
        if (!std::isfinite(rn[s])) { st = HELM_E_NONFINITE; continue; }
        if (rn[s] > o.tol * qn[s]) keep.push_back(s);
      }
      if (keep.size() != c.act_h.size()) set_active(c, keep);
      if (c.na == 0 || it == o.max_refine) break;
      // inner tolerance: the reduction the strictest active slot still needs
      // (with a safety factor), but no tighter than tol_inner
      double need = 1.0;
      for (int s : c.act_h) {
        rep[s].refine++;
        need = std::min(need, o.tol * qn[s] / rn[s]);
      }
      const double itol = std::min(0.5, std::max(o.tol_inner, 0.5 * need));
      launch_to32_scaled(c.r64, c.nrm, c.b32, c.act, c.na, n, c.st);
      int s2 = outer_solve<float>(c, c.b32, c.x32, itol, &ko, false);
      if (s2 == HELM_E_NONFINITE) st = s2;
      launch_axpy_up(c.x32, c.nrm, u, c.act, c.na, n, c.st);
      Epi en = make_epi(c, EPI_NORM);
      en.out = c.nrm;
      launch_stencil<double>(op64, c.slot_f, c.act, c.na, u, Scale<double>{}, q, Scale<double>{}, c.r64, c.st, &en);
    }
  }
  if (const int sc = sync_check(c); sc != HELM_OK) return sc;
  for (int a : solved) {
    rep[a].iters = ko.iters[a];
    rep[a].rel = qn[a] > 0.0 ? rn[a] / qn[a] : 0.0;
    if (!std::isfinite(rep[a].rel)) rep[a].status = HELM_E_NONFINITE;
    else if (rep[a].rel > o.tol) rep[a].status = HELM_E_NOCONV;
  }
  return st;
}

template OpView<float> op_view<float>(const Ctx&, int, int);
template OpView<double> op_view<double>(const Ctx&, int, int);

}  // namespace helm
