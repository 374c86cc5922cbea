// Host-side solver orchestration and workspace layout (internal).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <functional>
#include <vector>

#include "common.cuh"

namespace helm {

// A named NVTX range for the lifetime of the object (calls and solves show up
// as ranges in NVTX-aware profilers; without one attached it costs a branch).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Bytes of the guard band a debug build (HELM_DEBUG) leaves after every
// workspace array; bind() fills them with kGuardByte and the end of each call
// checks that no kernel wrote into one.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

// Sub-allocates the caller's workspace; with base == nullptr it only sizes.
struct Bump {
  char* base = nullptr;
  size_t off = 0;
  std::vector<size_t>* guards = nullptr;  // debug build: offsets of the guard bands
  template <typename T> T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
#ifdef HELM_DEBUG
    off = (off + 255) & ~(size_t)255;
    if (guards) guards->push_back(off);
    off += kGuardBytes;
#endif
    return p;
  }
};

template <typename R> struct KInst {
  int level = 0;
  int k = 0;
  bool flex = false;
  cplx<R>* V = nullptr;  // (k+1) sets of B fields
  cplx<R>* Z = nullptr;  // k sets (flexible only)
  cplx<R>* w = nullptr;  // 1 set
  KState ks{};
};

template <typename R> struct Hierarchy {
  KInst<R> inst[MAX_KINST];
  cplx<R>* r[MAX_LEVELS] = {};   // V-cycle residual per level
  cplx<R>* b[MAX_LEVELS] = {};   // restricted right-hand side per level
  cplx<R>* x[MAX_LEVELS] = {};   // coarse solution per level
};

// Everything one call needs on the device.
struct Ctx {
  const helm_plan* P = nullptr;
  cudaStream_t st = nullptr;
  int call = 0;
  int nfreq = 0, nsrc = 0, nrec = 0;
  int B = 0;      // slots per batch
  int dir = 0;    // 0: H, 1: H^H
  bool mixed = false;
  // model and tables per level
  double* m64[MAX_LEVELS] = {};
  float* m32[MAX_LEVELS] = {};
  double2* tab64[MAX_LEVELS][2] = {};
  float2* tab32[MAX_LEVELS][2] = {};
  double* omega = nullptr;
  double* w2_64 = nullptr;
  float* w2_32 = nullptr;
  // slots
  int* slot_f = nullptr;
  int* slot_s = nullptr;
  int* slot_g = nullptr;   // global (k, s) index of each slot
  int* act = nullptr;      // device active list
  int* ident = nullptr;    // 0..B-1
  int* err = nullptr;      // [4] device error counters
  double* partial = nullptr;
  unsigned* counter = nullptr;  // [B] arrival tickets of the fused reductions
  // FP64 fields
  double2* q = nullptr;    // right-hand side
  double2* u = nullptr;    // solution (forward field)
  double2* v = nullptr;    // adjoint field
  double2* r64 = nullptr;  // refinement residual
  float2* b32 = nullptr;   // complex64 inner right-hand side r/||r||
  float2* x32 = nullptr;   // complex64 inner solution
  double* nrm = nullptr;   // [B] residual norms
  double* qn = nullptr;    // [B] right-hand side norms
  double2* res = nullptr;  // [B][nrec] receiver residuals
  double* f_slot = nullptr;
  double* gcomp = nullptr;
  double* dmc = nullptr;   // extended model perturbation E dm (linearised calls)
  double2* du = nullptr;   // linearised state / adjoint (full Hessian product)
  double* shift = nullptr; // [nfreq] diagonal shift per (virtual) frequency (2.5D: k_y^2), or null
  double* ck = nullptr;    // [nfreq] 2.5D quadrature weight per virtual frequency
  double2* wav = nullptr;  // [nfreq] 2.5D wavelet per virtual frequency
  // WRI: field accumulator and receiver-space conjugate-gradient state
  double2* acc = nullptr;  // [B][n]
  double2* cgR = nullptr;  // [B][nrec] residual
  double2* cgP = nullptr;  // [B][nrec] search direction
  double2* cgAP = nullptr; // [B][nrec] A times the direction
  double* rho = nullptr;   // [B] ||R||^2
  double* rho0 = nullptr;  // [B] initial ||R||^2
  double* alpha = nullptr; // [B] step length
  double* sq = nullptr;    // [B] ||H u - q||^2
  // Krylov hierarchies
  Hierarchy<float> h32;
  Hierarchy<double> h64;
  KState ks64{};           // FP64 bookkeeping for refinement norms
  // host state
  std::vector<int> act_h;
  int na = 0;
  // debug build: workspace base, guard-band offsets (host list and device copy), host-side index faults
  char* ws_base = nullptr;
  std::vector<size_t> guards;
  size_t* guards_dev = nullptr;
  bool host_fault = false;
};

size_t layout(const helm_plan& P, int call, int nfreq, int nsrc, int nrec, char* base, Ctx* c);

// Per-slot outcome of one batched solve.
struct SlotReport {
  int status = HELM_OK;
  int iters = 0;
  int refine = 0;
  double rel = 0.0;
};

// One-time per-call device setup: extended model on every level, tables, w^2.
int setup_operator(Ctx& c, const double* m_phys, const double* freqs_hz);
// Set the current batch: slots 0..nb-1 take global (k, s) indices g[0..nb-1].
int set_batch(Ctx& c, const std::vector<int>& g);
// The same with explicit (frequency, source) per slot; g are the report indices.
int set_batch_fs(Ctx& c, const std::vector<int>& g, const std::vector<int>& f, const std::vector<int>& s);
void set_active(Ctx& c, const std::vector<int>& a);
// Solve H u = q (dir 0) or H^H u = q (dir 1) for all slots of the batch, or
// only for the slots listed in `only`; q and u are FP64 batch arrays.  Fills
// rep[0..nb-1] (slots left out keep an empty report and their u untouched).
// With `warm` the solves start from the u they are given (a slot whose
// initial residual already meets the tolerance takes no iteration), else
// from zero.
int solve_batch(Ctx& c, int dir, const double2* q, double2* u, int nb, std::vector<SlotReport>& rep,
                const std::vector<int>* only = nullptr, bool warm = false);
int sync_check(Ctx& c);
// sync_check, then (debug build) the guard bands and host-side index checks:
// HELM_E_BOUNDS when a kernel wrote past the end of a workspace array or a
// slot index was out of range.  Called at the end of every entry point.
int final_check(Ctx& c);
// Debug build: write the guard pattern and the guard list after layout().
int arm_guards(Ctx& c);
// z = M^{-1} x for the active slots (the plan's preconditioner, the plan's
// precision; dir 1 uses the adjoint operator H^H).
int precond_apply(Ctx& c, int dir, const void* x, void* z);

template <typename R> OpView<R> op_view(const Ctx& c, int level, int dir);

}  // namespace helm
