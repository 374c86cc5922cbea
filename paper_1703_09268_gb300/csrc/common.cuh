// Internal declarations shared by the CUDA translation units of libhelm.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include "helm.h"

namespace helm {

// ---------------------------------------------------------------------------
// Complex arithmetic on interleaved float2 / double2
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };
template <typename R> using cplx = typename CT<R>::T;

__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}
// acc + conj(a)*b
template <typename C> __device__ __forceinline__ C cfmac(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
  return acc;
}
// acc - a*b
template <typename C> __device__ __forceinline__ C cfms(C a, C b, C acc) {
  acc.x = fma(-a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(-a.x, b.y, fma(-a.y, b.x, acc.y));
  return acc;
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return mkc(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Limits and launch accounting
// ---------------------------------------------------------------------------
constexpr int KMAX = 32;          // longest Krylov cycle
constexpr int MAX_LEVELS = 3;     // multigrid levels
constexpr int MAX_KINST = 5;      // nested Krylov solver instances (see solver.cu)
constexpr int RED_BLOCKS_MAX = 4096;  // total blocks of one reduction launch

extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Optional per-kernel-class timing: when enabled (helm_profile_enable), every
// launch in a class is bracketed by CUDA events on its stream and its
// algorithmic bytes are accumulated.
enum ProfClass {
  PC_STENCIL32 = 0, PC_STENCIL64, PC_GS32, PC_GS64, PC_SMALL, PC_TRANSFER, PC_FWI, PC_MISC,
  PC_STENCIL32_COARSE, PC_GS32_COARSE, PC_GRAM32, PC_UPDATE32, PC_COUNT
};
// Launches on grids below this many nodes per field are booked to the coarse classes.
constexpr size_t PROF_COARSE_N = 200000;
template <typename R> inline int prof_stencil_class(size_t n) {
  return sizeof(R) == 8 ? PC_STENCIL64 : (n < PROF_COARSE_N ? PC_STENCIL32_COARSE : PC_STENCIL32);
}
template <typename R> inline int prof_gs_class(size_t n, int fine_class = PC_GS32) {
  return sizeof(R) == 8 ? PC_GS64 : (n < PROF_COARSE_N ? PC_GS32_COARSE : fine_class);
}
struct ProfScope {
  ProfScope(int cls, double bytes, cudaStream_t st);
  ~ProfScope();
  int cls;
  double bytes;
  cudaStream_t st;
  int slot;
};

// ---------------------------------------------------------------------------
// Plan: host-side geometry of every grid level
// ---------------------------------------------------------------------------
struct LevelGeom {
  int N[3];        // computational nodes per physical axis (x, y, z)
  int K[3];        // the same sizes in kernel order (2D: x, 1, z)
  size_t n;        // nodes of one field
  int Nmax;        // table row length
  double h;        // spacing at this level
};

}  // namespace helm

struct helm_plan {
  helm_grid g;
  helm_solve_opts o;
  int L;                    // grid levels used by the solver
  int pad[3];               // extra high-side layer cells
  double smax[3];           // sigma_max per physical axis
  helm::LevelGeom lev[helm::MAX_LEVELS];
  size_t n_phys;
};

namespace helm {

// ---------------------------------------------------------------------------
// Device views used by launches
// ---------------------------------------------------------------------------

// One level of the operator in precision R, for one direction (forward or
// adjoint).  Tables are [nfreq][axis 0..2][cm, cd, cp][Nmax] in kernel-axis
// order; w2[f] = omega_f^2.
template <typename R> struct OpView {
  const cplx<R>* tab;
  const R* m;
  const R* w2;
  int K[3];
  size_t n;
  int Nmax;
};

// Per-slot scale vector with stride (scale of slot s = p[s * stride]).
template <typename R> struct Scale {
  const R* p = nullptr;
  int stride = 0;
};

// Per-solver-instance small state, one entry per right-hand-side slot.
struct KState {
  double2* H;      // [B][KMAX+1][KMAX] Hessenberg, rotated in place
  double2* cs;     // [B][KMAX]
  double2* sn;     // [B][KMAX]
  double2* g;      // [B][KMAX+1] rotated right-hand side of the least-squares problem
  double2* hcol;   // [B][KMAX+1] current Arnoldi column
  double* scale;   // [B][KMAX+1] 1/||.|| of each stored basis vector
  double* bnorm;   // [B] ||b|| of the system being solved
  double* rnorm;   // [B] last true residual norm
  double* est;     // [B] current Arnoldi residual estimate
  void* coef;      // [B][KMAX+1] cplx<R>: coefficients of the next vector pass
  void* scale_r;   // [B][KMAX+1] R copy of `scale`
};

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------

struct Epi;  // fused reduction + per-slot epilogue (reduce.cuh)

// y = bs*b - xs*H x   (b == nullptr: y = xs*H x), for the active slots.  With an
// epilogue the kernel also reduces y: the norm (EPI_NORM / EPI_START) or the
// dots with basis vectors V_0..V_{nv-1} (EPI_DOTS).  The plain apply picks
// its tile shape per grid, timing the shapes on first use unless may_tune is
// false (then a grid not tuned yet takes the first shape).
template <typename R>
void launch_stencil(const OpView<R>& op, const int* slot_f, const int* act, int na,
                    const cplx<R>* x, Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y,
                    cudaStream_t st, const Epi* epi = nullptr, const cplx<R>* V = nullptr,
                    size_t vstride = 0, int nv = 0, bool may_tune = true);

// Damped Jacobi: z = z + omega D^{-1}(bs*b - H z) (first sweep with z = 0 gives omega D^{-1} bs*b).
template <typename R>
void launch_jacobi_first(const OpView<R>& op, const int* slot_f, const int* act, int na,
                         const cplx<R>* b, Scale<R> bs, R omega, cplx<R>* z, cudaStream_t st);
template <typename R>
void launch_jacobi_update(const OpView<R>& op, const int* slot_f, const int* act, int na,
                          const cplx<R>* r, R omega, cplx<R>* z, cudaStream_t st);

// Vector passes over basis vectors V_0..V_{nv-1} (V_i of slot s at V + i*vstride + s*n),
// each with its reduction folded into an epilogue.
enum GsMode { GS_DOT = 0, GS_SUB_DOT = 1, GS_SUB_STORE_NORM = 2, GS_ADD_STORE = 3 };
template <typename R>
void launch_gs(int mode, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* coef,
               const cplx<R>* w, Scale<R> ws, cplx<R>* out, const int* act, int na, size_t n,
               const Epi& e, cudaStream_t st);
int reduction_blocks(int na, size_t n, int threads);
// End of an s-step cycle: x += sum_{i<s} c_i W_i (x = ... when xzero) and, with
// recur, W_0 <- W_0 - sum_{i<s} c_i W_{i+1} in the same pass.
template <typename R>
void launch_sstep_update(cplx<R>* V, size_t vstride, int s, const cplx<R>* coef, cplx<R>* x, const int* act, int na,
                         size_t n, int recur, int xzero, cudaStream_t st);
// Gram pass of an s-step cycle over W_0..W_s (EPI_GRAM epilogue).
template <typename R>
void launch_gram(const cplx<R>* V, size_t vstride, int s, const int* act, int na, size_t n, const Epi& e,
                 cudaStream_t st);

// Precision conversions and refinement helpers (slot-batched).
void launch_to32_scaled(const double2* r, const double* rnorm, float2* out, const int* act, int na,
                        size_t n, cudaStream_t st);
void launch_axpy_up(const float2* e, const double* rnorm, double2* u, const int* act, int na,
                    size_t n, cudaStream_t st);
template <typename R>
void launch_zero(cplx<R>* x, const int* act, int na, size_t n, cudaStream_t st);

// Inter-grid transfers: coarse = R fine (full weighting), fine += P coarse.
template <typename R>
void launch_restrict(const cplx<R>* fine, const LevelGeom& f, cplx<R>* coarse, const LevelGeom& c,
                     const int* act, int na, cudaStream_t st);
template <typename R>
void launch_prolong_add(const cplx<R>* coarse, const LevelGeom& c, cplx<R>* fine, const LevelGeom& f,
                        const int* act, int na, cudaStream_t st);
void launch_restrict_model(const double* mf, const LevelGeom& f, double* mc, const LevelGeom& c,
                           cudaStream_t st);

// Model extension, tables, sources, receivers, misfit and gradient.
void launch_extend(const helm_plan& P, const double* m_phys, double* m64, float* m32, cudaStream_t st);
void launch_tables(const helm_plan& P, int level, const double* freqs_dev, int nfreq,
                   double2* tab64_fwd, double2* tab64_adj, float2* tab32_fwd, float2* tab32_adj,
                   cudaStream_t st, const double* shift = nullptr);
void launch_copy_m32(const double* m64, float* m32, size_t n, cudaStream_t st);
void launch_sources(const helm_plan& P, const int32_t* src_idx, int n_srcloc, const double2* Q,
                    int nsrc, const double2* wavelet, const int* slot_f, const int* slot_s,
                    int nslots, double2* q, int* bad, cudaStream_t st);
void launch_check_idx(const helm_plan& P, const int32_t* idx, int cnt, int* bad, cudaStream_t st);
void launch_receivers(const helm_plan& P, const double2* u, const int32_t* rec_idx, int nrec,
                      const int* slots, int nslots, double2* d_out, size_t d_stride, cudaStream_t st);
void launch_residual_misfit(const helm_plan& P, const double2* u, const int32_t* rec_idx, int nrec,
                            const double2* d_obs, const int* slot_f, const int* slot_s, int nsrc,
                            const int* slots, int nslots, double2* res, double* f_slot,
                            cudaStream_t st);
void launch_spread(const helm_plan& P, const double2* r, size_t r_stride, const int32_t* rec_idx,
                   int nrec, double sign, const int* slots, int nslots, double2* b, cudaStream_t st);
void launch_grad_accum(const double2* u, const int* u_idx, const double2* v, const double* w2, const int* slot_f,
                       const int* slots, int nslots, size_t n, double* gcomp, cudaStream_t st, double scale = 1.0);
// the same with complex64 forward fields
void launch_grad_accum(const float2* u, const int* u_idx, const double2* v, const double* w2, const int* slot_f,
                       const int* slots, int nslots, size_t n, double* gcomp, cudaStream_t st, double scale = 1.0);
// WRI: receiver-space conjugate gradients (one slot per block) and helpers
void launch_wri_init(const double2* res, int nrec, int nslots, double2* R, double2* Pd, double* rho, double* rho0,
                     cudaStream_t st);
void launch_wri_ap(const helm_plan& P, const double2* du, const int32_t* rec_idx, int nrec, double inv_l2,
                   const double2* Pd, double2* AP, const double* rho, const double* rho0, double thr2, double* alpha,
                   int nslots, cudaStream_t st);
void launch_wri_step(int nrec, int nslots, double2* R, double2* Pd, const double2* AP, const double* alpha,
                     double* rho, cudaStream_t st);
void launch_axpy_slots(const double2* x, const double* c, double c0, size_t n, int nslots, double2* y,
                       cudaStream_t st);
void launch_sqnorm(const double2* x, size_t n, int nslots, double* part, double* sq, cudaStream_t st);
void launch_wri_f(const double* f_slot, const double* sq, int nslots, double lam2, double* f, cudaStream_t st);
// b_s = -w_f^2 dmc u_s for slots 0..nslots-1 (linearised state right-hand side)
void launch_born_source(const double2* u, const double* dmc, const double* w2, const int* slot_f, int nslots,
                        size_t n, double2* b, cudaStream_t st);
// 2.5D: residual per group of nk slots (one per k_y node) and the weighted adjoint sources
void launch_residual_25d(const helm_plan& P, const double2* u, const int32_t* rec_idx, int nrec, const double2* d_obs,
                         const double* ck, const int* slot_f, const int* slot_s, int nsrc, int nk, int ngroups,
                         double2* res, double* f_grp, cudaStream_t st);
void launch_spread_25d(const helm_plan& P, const double2* res, const int32_t* rec_idx, int nrec, const double* ck,
                       const int* slot_f, int nk, int nslots, double2* b, cudaStream_t st);
void launch_extend_adjoint(const helm_plan& P, const double* gcomp, double* g_phys, cudaStream_t st);
void launch_sum_f(const double* f_slot, const int* slots, int nslots, double* f_out, int accumulate,
                  cudaStream_t st);
void launch_copy_fields(const double2* src, double2* dst, const int* slots, int nslots,
                        const int* dst_index, size_t n, cudaStream_t st);
// complex128 fields rounded to complex64
void launch_copy_fields(const double2* src, float2* dst, const int* slots, int nslots,
                        const int* dst_index, size_t n, cudaStream_t st);
void launch_check_finite(const double* vals, const int* act, int na, int* bad, cudaStream_t st);

}  // namespace helm
