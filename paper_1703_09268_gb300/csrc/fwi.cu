// Model extension, damping-layer tables, source injection, receiver
// restriction, least-squares misfit, adjoint sources and the adjoint-state
// gradient (Sec. 2; Appendix A eqs. (dU2), (dH), (dHadj); Listing pdefunc).
#include <cmath>

#include <algorithm>

#include "common.cuh"

namespace helm {

namespace {

struct GeomArgs {
  int n[3];     // physical nodes
  int N[3];     // computational nodes
  int lo[3];    // layer cells on the low side (= npml)
};

GeomArgs geom(const helm_plan& P) {
  GeomArgs g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = P.g.n[d];
    g.N[d] = P.lev[0].N[d];
    g.lo[d] = P.g.npml[d];
  }
  return g;
}

__device__ __forceinline__ bool phys_to_comp(const GeomArgs& g, long long idx, size_t* out) {
  const long long np = (long long)g.n[0] * g.n[1] * g.n[2];
  if (idx < 0 || idx >= np) return false;
  const long long ix = idx % g.n[0];
  const long long iy = (idx / g.n[0]) % g.n[1];
  const long long iz = idx / ((long long)g.n[0] * g.n[1]);
  *out = (size_t)(ix + g.lo[0]) + (size_t)g.N[0] * ((size_t)(iy + g.lo[1]) + (size_t)g.N[1] * (size_t)(iz + g.lo[2]));
  return true;
}

// E m: every computational node copies the nearest physical node along each axis.
__global__ void k_extend(GeomArgs g, const double* __restrict__ mp, double* __restrict__ m64,
                         float* __restrict__ m32) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)g.N[0] * g.N[1] * g.N[2];
  if (i >= n) return;
  int c[3];
  c[0] = (int)(i % g.N[0]);
  c[1] = (int)((i / g.N[0]) % g.N[1]);
  c[2] = (int)(i / ((size_t)g.N[0] * g.N[1]));
  int q[3];
  for (int d = 0; d < 3; ++d) q[d] = min(max(c[d] - g.lo[d], 0), g.n[d] - 1);
  const double v = mp[(size_t)q[0] + (size_t)g.n[0] * ((size_t)q[1] + (size_t)g.n[1] * q[2])];
  m64[i] = v;
  if (m32) m32[i] = (float)v;
}

__global__ void k_copy_m32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Damping-layer tables of one level.  Kernel axis ka maps to physical axis
// pax[ka] (or -1 for the unit middle axis of 2D problems).
struct TabArgs {
  int pax[3];
  int N[3];          // level sizes per kernel axis
  int lo[3], hi[3];  // physical box in level-0 cells, per kernel axis
  int wlo[3], whi[3];// layer widths in level-0 cells, per kernel axis
  double smax[3];
  int stride0;       // 2^level: level node j sits at level-0 coordinate (j+1)*stride0 - 1
  double h;          // spacing at this level
  int Nmax;
};

__device__ double sigma_at(const TabArgs& A, int ka, double t0) {
  if (t0 < A.lo[ka]) {
    if (A.wlo[ka] <= 0) return 0.0;
    const double r = (A.lo[ka] - t0) / (double)A.wlo[ka];
    return A.smax[ka] * r * r;
  }
  if (t0 > A.hi[ka]) {
    if (A.whi[ka] <= 0) return 0.0;
    const double r = (t0 - A.hi[ka]) / (double)A.whi[ka];
    return A.smax[ka] * r * r;
  }
  return 0.0;
}

// 1/eta with eta = 1 + i sigma / omega
__device__ double2 inv_eta(const TabArgs& A, int ka, double t0, double omega) {
  const double s = sigma_at(A, ka, t0) / omega;
  const double den = 1.0 + s * s;
  return make_double2(1.0 / den, -s / den);
}

__device__ double2 mulc(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ double2 conjc(double2 a) { return make_double2(a.x, -a.y); }

__global__ void k_tables(TabArgs A, const double* __restrict__ omega, const double* __restrict__ shift, int nfreq,
                         double2* __restrict__ t64f, double2* __restrict__ t64a,
                         float2* __restrict__ t32f, float2* __restrict__ t32a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int ka = blockIdx.y;
  const int f = blockIdx.z;
  if (i >= A.Nmax || f >= nfreq) return;
  double2 cm = make_double2(0, 0), cd = make_double2(0, 0), cp = make_double2(0, 0);
  double2 am = make_double2(0, 0), ad = make_double2(0, 0), ap = make_double2(0, 0);
  if (A.pax[ka] >= 0 && i < A.N[ka]) {
    const double w = omega[f];
    const double s0 = (double)A.stride0;
    const double h2 = A.h * A.h;
    auto at = [&](double j) { return (j + 1.0) * s0 - 1.0; };  // level-0 coordinate of level node j
    const double2 a_i = inv_eta(A, ka, at(i), w);
    const double2 b_m = inv_eta(A, ka, at(i - 0.5), w);
    const double2 b_p = inv_eta(A, ka, at(i + 0.5), w);
    cm = mulc(a_i, b_m); cm.x /= h2; cm.y /= h2;
    cp = mulc(a_i, b_p); cp.x /= h2; cp.y /= h2;
    cd = make_double2(-(cm.x + cp.x), -(cm.y + cp.y));
    // a constant diagonal shift (2.5D: -k_y^2) rides on the first axis' diagonal
    if (shift && ka == 0) cd.x -= shift[f];
    // H^H: coefficient of x_{i-1} is conj(cp[i-1]), of x_{i+1} is conj(cm[i+1])
    if (i > 0) {
      const double2 a_l = inv_eta(A, ka, at(i - 1), w);
      am = conjc(mulc(a_l, b_m)); am.x /= h2; am.y /= h2;
    }
    if (i + 1 < A.N[ka]) {
      const double2 a_r = inv_eta(A, ka, at(i + 1), w);
      ap = conjc(mulc(a_r, b_p)); ap.x /= h2; ap.y /= h2;
    }
    ad = conjc(cd);
  }
  const size_t base = ((size_t)f * 3 + ka) * 3 * A.Nmax + i;
  const size_t N = A.Nmax;
  t64f[base] = cm; t64f[base + N] = cd; t64f[base + 2 * N] = cp;
  t64a[base] = am; t64a[base + N] = ad; t64a[base + 2 * N] = ap;
  t32f[base] = make_float2((float)cm.x, (float)cm.y);
  t32f[base + N] = make_float2((float)cd.x, (float)cd.y);
  t32f[base + 2 * N] = make_float2((float)cp.x, (float)cp.y);
  t32a[base] = make_float2((float)am.x, (float)am.y);
  t32a[base + N] = make_float2((float)ad.x, (float)ad.y);
  t32a[base + 2 * N] = make_float2((float)ap.x, (float)ap.y);
}

// q[slot] += wavelet[f] * Q[k, s] / h^dim at the node of src_idx[k].
__global__ void k_sources(GeomArgs g, const int32_t* __restrict__ src_idx, int n_srcloc,
                          const double2* __restrict__ Q, int nsrc, const double2* __restrict__ wavelet,
                          const int* __restrict__ slot_f, const int* __restrict__ slot_s, int nslots,
                          double inv_hd, double2* q, size_t n, int* bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = blockIdx.y;
  if (k >= n_srcloc || slot >= nslots) return;
  size_t c;
  if (!phys_to_comp(g, src_idx[k], &c)) {
    if (slot == 0) atomicAdd(bad, 1);
    return;
  }
  const int f = slot_f[slot], s = slot_s[slot];
  const double2 w = wavelet ? wavelet[f] : make_double2(1.0, 0.0);
  double2 v = mulc(w, Q[(size_t)k * nsrc + s]);
  double* dst = (double*)(q + (size_t)slot * n + c);
  atomicAdd(dst, v.x * inv_hd);
  atomicAdd(dst + 1, v.y * inv_hd);
}

__global__ void k_check_idx(GeomArgs g, const int32_t* __restrict__ idx, int cnt, int* bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  size_t c;
  if (!phys_to_comp(g, idx[k], &c)) atomicAdd(bad, 1);
}

// d_out[dst(slot)][k] = u[slot][rec_k]
__global__ void k_receivers(GeomArgs g, const double2* __restrict__ u, size_t n,
                            const int32_t* __restrict__ rec_idx, int nrec, const int* __restrict__ slots,
                            int nslots, double2* __restrict__ d_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (k >= nrec || a >= nslots) return;
  size_t c;
  double2 v = make_double2(0, 0);
  if (phys_to_comp(g, rec_idx[k], &c)) v = u[(size_t)a * n + c];
  d_out[(size_t)slots[a] * nrec + k] = v;
}

// res[slot][k] = u[slot][rec_k] - d_obs[f][s][k]; f_slot[slot] = 1/2 sum |res|^2
__global__ void k_residual_misfit(GeomArgs g, const double2* __restrict__ u, size_t n,
                                  const int32_t* __restrict__ rec_idx, int nrec,
                                  const double2* __restrict__ d_obs, const int* __restrict__ slot_f,
                                  const int* __restrict__ slot_s, int nsrc, int nslots,
                                  double2* __restrict__ res, double* __restrict__ f_slot) {
  __shared__ double sh[256];
  const int slot = blockIdx.x;
  if (slot >= nslots) return;
  const size_t drow = ((size_t)slot_f[slot] * nsrc + slot_s[slot]) * nrec;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    size_t c;
    double2 v = make_double2(0, 0);
    if (phys_to_comp(g, rec_idx[k], &c)) v = u[(size_t)slot * n + c];
    const double2 d = d_obs[drow + k];
    const double2 r = make_double2(v.x - d.x, v.y - d.y);
    res[(size_t)slot * nrec + k] = r;
    acc += r.x * r.x + r.y * r.y;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) f_slot[slot] = 0.5 * sh[0];
}

// b[slot] += sign * P_r^T r[slot]   (b zeroed beforehand)
__global__ void k_spread(GeomArgs g, const double2* __restrict__ r, size_t r_stride,
                         const int32_t* __restrict__ rec_idx, int nrec, double sign,
                         const int* __restrict__ slots, int nslots, double2* b, size_t n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (k >= nrec || a >= nslots) return;
  size_t c;
  if (!phys_to_comp(g, rec_idx[k], &c)) return;
  const double2 v = r[(size_t)slots[a] * r_stride + k];
  double* dst = (double*)(b + (size_t)a * n + c);
  atomicAdd(dst, sign * v.x);
  atomicAdd(dst + 1, sign * v.y);
}

// gcomp[p] += sum_slots w_f^2 Re(conj(u) v), slots summed in order.  The
// field u of slot s is u[u_idx[s]] when u_idx is given (fields stored by the
// caller in (frequency, source) order), else u[s].
// U is complex128, or complex64 for forward fields stored at half the bytes
// (promoted to FP64 before the product).
template <typename CU>
__global__ void k_grad_accum(const CU* __restrict__ u, const int* __restrict__ u_idx,
                             const double2* __restrict__ v, const double* __restrict__ w2,
                             const int* __restrict__ slot_f, const int* __restrict__ slots, int nslots,
                             size_t n, double scale, double* __restrict__ gcomp) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double acc = gcomp[p];
  for (int a = 0; a < nslots; ++a) {
    const int s = slots[a];
    const CU uu = u[(size_t)(u_idx ? u_idx[s] : s) * n + p];
    const double2 vv = v[(size_t)s * n + p];
    acc += scale * w2[slot_f[s]] * ((double)uu.x * vv.x + (double)uu.y * vv.y);
  }
  gcomp[p] = acc;
}

// ---- WRI (penalty method): conjugate gradients in the receiver space ----
// A z = r0 with A = I + lambda^-2 P_r H^{-1} H^{-H} P_r^T (Hermitian positive
// definite), one slot per block, fixed-order reductions.

__device__ __forceinline__ double block_sum_256(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// R = -(P u0 - d) = d - P u0, Pd = R, rho = rho0 = ||R||^2
__global__ void k_wri_init(const double2* __restrict__ res, int nrec, double2* __restrict__ R,
                           double2* __restrict__ Pd, double* __restrict__ rho, double* __restrict__ rho0) {
  __shared__ double sh[256];
  const int a = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    const double2 r = res[(size_t)a * nrec + k];
    const double2 v = make_double2(-r.x, -r.y);
    R[(size_t)a * nrec + k] = v;
    Pd[(size_t)a * nrec + k] = v;
    acc += v.x * v.x + v.y * v.y;
  }
  const double t = block_sum_256(acc, sh);
  if (threadIdx.x == 0) {
    rho[a] = t;
    rho0[a] = t;
  }
}

// AP = Pd + lambda^-2 P_r du;  alpha = rho / Re<Pd, AP> (0 once the slot has converged)
__global__ void k_wri_ap(GeomArgs g, const double2* __restrict__ du, size_t n, const int32_t* __restrict__ rec_idx,
                         int nrec, double inv_l2, const double2* __restrict__ Pd, double2* __restrict__ AP,
                         const double* __restrict__ rho, const double* __restrict__ rho0, double thr2,
                         double* __restrict__ alpha) {
  __shared__ double sh[256];
  const int a = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    size_t c;
    double2 v = make_double2(0, 0);
    if (phys_to_comp(g, rec_idx[k], &c)) v = du[(size_t)a * n + c];
    const double2 pk = Pd[(size_t)a * nrec + k];
    const double2 ap = make_double2(pk.x + inv_l2 * v.x, pk.y + inv_l2 * v.y);
    AP[(size_t)a * nrec + k] = ap;
    acc += pk.x * ap.x + pk.y * ap.y;
  }
  const double pap = block_sum_256(acc, sh);
  if (threadIdx.x == 0) {
    const bool live = rho[a] > thr2 * rho0[a] && pap > 0.0 && isfinite(pap);
    alpha[a] = live ? rho[a] / pap : 0.0;
  }
}

// R -= alpha AP;  rho' = ||R||^2;  Pd = R + (rho'/rho) Pd;  rho = rho'
__global__ void k_wri_step(int nrec, double2* __restrict__ R, double2* __restrict__ Pd,
                           const double2* __restrict__ AP, const double* __restrict__ alpha,
                           double* __restrict__ rho) {
  __shared__ double sh[256];
  const int a = blockIdx.x;
  const double al = alpha[a];
  if (al == 0.0) return;  // converged slot: the whole block leaves together
  double acc = 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    double2 r = R[(size_t)a * nrec + k];
    const double2 ap = AP[(size_t)a * nrec + k];
    r.x -= al * ap.x;
    r.y -= al * ap.y;
    R[(size_t)a * nrec + k] = r;
    acc += r.x * r.x + r.y * r.y;
  }
  const double rn = block_sum_256(acc, sh);
  const double beta = rho[a] > 0.0 ? rn / rho[a] : 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    const double2 r = R[(size_t)a * nrec + k];
    const double2 pk = Pd[(size_t)a * nrec + k];
    Pd[(size_t)a * nrec + k] = make_double2(r.x + beta * pk.x, r.y + beta * pk.y);
  }
  __syncthreads();
  if (threadIdx.x == 0) rho[a] = rn;
}

// y_s += c_s x_s for slots 0..nslots-1 (c per slot, or the constant c0 when c is null)
__global__ void k_axpy_slots(const double2* __restrict__ x, const double* __restrict__ c, double c0, size_t n,
                             double2* __restrict__ y) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int a = blockIdx.y;
  const double w = c ? c[a] : c0;
  if (w == 0.0) return;
  const double2 v = x[(size_t)a * n + p];
  double2 t = y[(size_t)a * n + p];
  t.x = fma(w, v.x, t.x);
  t.y = fma(w, v.y, t.y);
  y[(size_t)a * n + p] = t;
}

// sq[a] = ||x_a||^2: per-block partial sums, then one block per slot adds them in order
__global__ void k_sqnorm_partial(const double2* __restrict__ x, size_t n, int nblk, double* __restrict__ part) {
  __shared__ double sh[256];
  const int a = blockIdx.y;
  double acc = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)nblk * blockDim.x) {
    const double2 v = x[(size_t)a * n + p];
    acc += v.x * v.x + v.y * v.y;
  }
  const double t = block_sum_256(acc, sh);
  if (threadIdx.x == 0) part[(size_t)a * nblk + blockIdx.x] = t;
}
__global__ void k_sqnorm_fold(const double* __restrict__ part, int nblk, int nslots, double* __restrict__ sq) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nslots) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += part[(size_t)a * nblk + b];
  sq[a] = t;
}

// f += sum_a f_slot[a] + lam2/2 sum_a sq[a]  (slots in order)
__global__ void k_wri_f(const double* __restrict__ f_slot, const double* __restrict__ sq, int nslots, double lam2,
                        double* __restrict__ f) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = f[0];
  for (int a = 0; a < nslots; ++a) t += f_slot[a] + 0.5 * lam2 * sq[a];
  f[0] = t;
}

// Right-hand side of the linearised state equation (Appendix A, eq. (dU2)
// with A = I): b = -T dm = -w^2 (E dm) u, per slot.
__global__ void k_born_source(const double2* __restrict__ u, const double* __restrict__ dmc,
                              const double* __restrict__ w2, const int* __restrict__ slot_f, size_t n,
                              double2* __restrict__ b) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int s = blockIdx.y;
  const double c = -w2[slot_f[s]] * dmc[p];
  const double2 uu = u[(size_t)s * n + p];
  b[(size_t)s * n + p] = make_double2(c * uu.x, c * uu.y);
}

// 2.5D residual of group a (slots a*nk .. a*nk+nk-1, one per k_y node):
// r = sum_i c_i P_r u_i - d, with c indexed by the slot's virtual frequency;
// f_grp[a] = 1/2 ||r||^2.
__global__ void k_residual_25d(GeomArgs g, const double2* __restrict__ u, size_t n,
                               const int32_t* __restrict__ rec_idx, int nrec, const double2* __restrict__ d_obs,
                               const double* __restrict__ ck, const int* __restrict__ slot_f,
                               const int* __restrict__ slot_s, int nsrc, int nk, double2* __restrict__ res,
                               double* __restrict__ f_grp) {
  __shared__ double sh[256];
  const int a = blockIdx.x;
  const int s0 = a * nk;
  const int j = slot_f[s0] / nk;
  const size_t drow = ((size_t)j * nsrc + slot_s[s0]) * nrec;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    size_t c;
    double2 v = make_double2(0, 0);
    if (phys_to_comp(g, rec_idx[k], &c)) {
      for (int i = 0; i < nk; ++i) {
        const double w = ck[slot_f[s0 + i]];
        const double2 ui = u[(size_t)(s0 + i) * n + c];
        v.x += w * ui.x;
        v.y += w * ui.y;
      }
    }
    const double2 d = d_obs[drow + k];
    const double2 r = make_double2(v.x - d.x, v.y - d.y);
    res[(size_t)a * nrec + k] = r;
    acc += r.x * r.x + r.y * r.y;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) f_grp[a] = 0.5 * sh[0];
}

// b_slot += -c_i P_r^T r_group for every slot (its group is slot / nk).
__global__ void k_spread_25d(GeomArgs g, const double2* __restrict__ res, const int32_t* __restrict__ rec_idx,
                             int nrec, const double* __restrict__ ck, const int* __restrict__ slot_f, int nk,
                             int nslots, double2* b, size_t n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (k >= nrec || a >= nslots) return;
  size_t c;
  if (!phys_to_comp(g, rec_idx[k], &c)) return;
  const double w = -ck[slot_f[a]];
  const double2 r = res[(size_t)(a / nk) * nrec + k];
  double* dst = (double*)(b + (size_t)a * n + c);
  atomicAdd(dst, w * r.x);
  atomicAdd(dst + 1, w * r.y);
}

// g_phys = E^T gcomp: each physical node sums the computational nodes copying it.
__global__ void k_extend_adjoint(GeomArgs g, const double* __restrict__ gc, double* __restrict__ gp) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t np = (size_t)g.n[0] * g.n[1] * g.n[2];
  if (i >= np) return;
  int q[3];
  q[0] = (int)(i % g.n[0]);
  q[1] = (int)((i / g.n[0]) % g.n[1]);
  q[2] = (int)(i / ((size_t)g.n[0] * g.n[1]));
  int a[3], b[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = q[d] == 0 ? 0 : q[d] + g.lo[d];
    b[d] = q[d] == g.n[d] - 1 ? g.N[d] - 1 : q[d] + g.lo[d];
  }
  double acc = 0.0;
  for (int z = a[2]; z <= b[2]; ++z)
    for (int y = a[1]; y <= b[1]; ++y)
      for (int x = a[0]; x <= b[0]; ++x)
        acc += gc[(size_t)x + (size_t)g.N[0] * ((size_t)y + (size_t)g.N[1] * z)];
  gp[i] = acc;
}

__global__ void k_sum_f(const double* __restrict__ f_slot, const int* __restrict__ slots, int nslots,
                        double* f_out, int accumulate) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double acc = accumulate ? *f_out : 0.0;
  for (int a = 0; a < nslots; ++a) acc += f_slot[slots[a]];
  *f_out = acc;
}

// dst complex128 (a copy) or complex64 (each part rounded to nearest)
template <typename CD>
__global__ void k_copy_fields(const double2* __restrict__ src, CD* __restrict__ dst,
                              const int* __restrict__ slots, const int* __restrict__ dst_index,
                              size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = blockIdx.y;
  const double2 v = src[(size_t)slots[a] * n + i];
  CD o;
  o.x = v.x;
  o.y = v.y;
  dst[(size_t)dst_index[a] * n + i] = o;
}

}  // namespace

void launch_extend(const helm_plan& P, const double* m_phys, double* m64, float* m32, cudaStream_t st) {
  const size_t n = P.lev[0].n;
  k_extend<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(geom(P), m_phys, m64, m32);
  count_launch();
}

void launch_copy_m32(const double* m64, float* m32, size_t n, cudaStream_t st) {
  k_copy_m32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m64, m32, n);
  count_launch();
}

void launch_tables(const helm_plan& P, int level, const double* omega_dev, int nfreq,
                   double2* t64f, double2* t64a, float2* t32f, float2* t32a, cudaStream_t st,
                   const double* shift) {
  const LevelGeom& L = P.lev[level];
  TabArgs A;
  const int map3[3] = {0, 1, 2}, map2[3] = {0, -1, 2};
  for (int ka = 0; ka < 3; ++ka) {
    const int pa = P.g.dim == 3 ? map3[ka] : map2[ka];
    A.pax[ka] = pa;
    A.N[ka] = L.K[ka];
    if (pa >= 0) {
      A.lo[ka] = P.g.npml[pa];
      A.hi[ka] = P.g.npml[pa] + P.g.n[pa] - 1;
      A.wlo[ka] = P.g.npml[pa];
      A.whi[ka] = P.g.npml[pa] + P.pad[pa];
      A.smax[ka] = P.smax[pa];
    } else {
      A.lo[ka] = A.hi[ka] = A.wlo[ka] = A.whi[ka] = 0;
      A.smax[ka] = 0.0;
    }
  }
  A.stride0 = 1 << level;
  A.h = L.h;
  A.Nmax = L.Nmax;
  dim3 grd((L.Nmax + 127) / 128, 3, nfreq);
  k_tables<<<grd, 128, 0, st>>>(A, omega_dev, shift, nfreq, t64f, t64a, t32f, t32a);
  count_launch();
}

void launch_sources(const helm_plan& P, const int32_t* src_idx, int n_srcloc, const double2* Q,
                    int nsrc, const double2* wavelet, const int* slot_f, const int* slot_s,
                    int nslots, double2* q, int* bad, cudaStream_t st) {
  if (n_srcloc <= 0 || nslots <= 0) return;
  const double inv_hd = 1.0 / std::pow(P.g.h, (double)P.g.dim);
  dim3 grd((n_srcloc + 127) / 128, nslots);
  k_sources<<<grd, 128, 0, st>>>(geom(P), src_idx, n_srcloc, Q, nsrc, wavelet, slot_f, slot_s, nslots,
                                 inv_hd, q, P.lev[0].n, bad);
  count_launch();
}

void launch_check_idx(const helm_plan& P, const int32_t* idx, int cnt, int* bad, cudaStream_t st) {
  if (cnt <= 0) return;
  k_check_idx<<<(cnt + 255) / 256, 256, 0, st>>>(geom(P), idx, cnt, bad);
  count_launch();
}

void launch_receivers(const helm_plan& P, const double2* u, const int32_t* rec_idx, int nrec,
                      const int* slots, int nslots, double2* d_out, size_t d_stride, cudaStream_t st) {
  (void)d_stride;
  if (nrec <= 0 || nslots <= 0) return;
  dim3 grd((nrec + 255) / 256, nslots);
  k_receivers<<<grd, 256, 0, st>>>(geom(P), u, P.lev[0].n, rec_idx, nrec, slots, nslots, d_out);
  count_launch();
}

void launch_residual_misfit(const helm_plan& P, const double2* u, const int32_t* rec_idx, int nrec,
                            const double2* d_obs, const int* slot_f, const int* slot_s, int nsrc,
                            const int* slots, int nslots, double2* res, double* f_slot,
                            cudaStream_t st) {
  (void)slots;
  if (nslots <= 0) return;
  k_residual_misfit<<<nslots, 256, 0, st>>>(geom(P), u, P.lev[0].n, rec_idx, nrec, d_obs, slot_f, slot_s,
                                            nsrc, nslots, res, f_slot);
  count_launch();
}

void launch_spread(const helm_plan& P, const double2* r, size_t r_stride, const int32_t* rec_idx,
                   int nrec, double sign, const int* slots, int nslots, double2* b, cudaStream_t st) {
  if (nrec <= 0 || nslots <= 0) return;
  dim3 grd((nrec + 255) / 256, nslots);
  k_spread<<<grd, 256, 0, st>>>(geom(P), r, r_stride, rec_idx, nrec, sign, slots, nslots, b, P.lev[0].n);
  count_launch();
}

void launch_grad_accum(const double2* u, const int* u_idx, const double2* v, const double* w2, const int* slot_f,
                       const int* slots, int nslots, size_t n, double* gcomp, cudaStream_t st, double scale) {
  if (nslots <= 0) return;
  ProfScope ps(PC_FWI, (double)nslots * n * 2 * sizeof(double2) + (double)n * 2 * sizeof(double), st);
  k_grad_accum<double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(u, u_idx, v, w2, slot_f, slots, nslots, n,
                                                                     scale, gcomp);
  count_launch();
}

void launch_grad_accum(const float2* u, const int* u_idx, const double2* v, const double* w2, const int* slot_f,
                       const int* slots, int nslots, size_t n, double* gcomp, cudaStream_t st, double scale) {
  if (nslots <= 0) return;
  ProfScope ps(PC_FWI, (double)nslots * n * (sizeof(float2) + sizeof(double2)) + (double)n * 2 * sizeof(double), st);
  k_grad_accum<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(u, u_idx, v, w2, slot_f, slots, nslots, n,
                                                                    scale, gcomp);
  count_launch();
}

void launch_wri_init(const double2* res, int nrec, int nslots, double2* R, double2* Pd, double* rho, double* rho0,
                     cudaStream_t st) {
  if (nslots <= 0) return;
  k_wri_init<<<nslots, 256, 0, st>>>(res, nrec, R, Pd, rho, rho0);
  count_launch();
}

void launch_wri_ap(const helm_plan& P, const double2* du, const int32_t* rec_idx, int nrec, double inv_l2,
                   const double2* Pd, double2* AP, const double* rho, const double* rho0, double thr2, double* alpha,
                   int nslots, cudaStream_t st) {
  if (nslots <= 0) return;
  k_wri_ap<<<nslots, 256, 0, st>>>(geom(P), du, P.lev[0].n, rec_idx, nrec, inv_l2, Pd, AP, rho, rho0, thr2, alpha);
  count_launch();
}

void launch_wri_step(int nrec, int nslots, double2* R, double2* Pd, const double2* AP, const double* alpha,
                     double* rho, cudaStream_t st) {
  if (nslots <= 0) return;
  k_wri_step<<<nslots, 256, 0, st>>>(nrec, R, Pd, AP, alpha, rho);
  count_launch();
}

void launch_axpy_slots(const double2* x, const double* c, double c0, size_t n, int nslots, double2* y,
                       cudaStream_t st) {
  if (nslots <= 0) return;
  dim3 grd((unsigned)((n + 255) / 256), nslots);
  k_axpy_slots<<<grd, 256, 0, st>>>(x, c, c0, n, y);
  count_launch();
}

void launch_sqnorm(const double2* x, size_t n, int nslots, double* part, double* sq, cudaStream_t st) {
  if (nslots <= 0) return;
  const int nblk = (int)std::max<size_t>(1, std::min<size_t>(32, (n + 255) / 256));
  dim3 grd(nblk, nslots);
  k_sqnorm_partial<<<grd, 256, 0, st>>>(x, n, nblk, part);
  k_sqnorm_fold<<<(nslots + 127) / 128, 128, 0, st>>>(part, nblk, nslots, sq);
  count_launch(2);
}

void launch_wri_f(const double* f_slot, const double* sq, int nslots, double lam2, double* f, cudaStream_t st) {
  k_wri_f<<<1, 32, 0, st>>>(f_slot, sq, nslots, lam2, f);
  count_launch();
}

void launch_born_source(const double2* u, const double* dmc, const double* w2, const int* slot_f, int nslots,
                        size_t n, double2* b, cudaStream_t st) {
  if (nslots <= 0) return;
  ProfScope ps(PC_FWI, (double)nslots * n * 2 * sizeof(double2) + (double)n * sizeof(double), st);
  dim3 grd((unsigned)((n + 255) / 256), nslots);
  k_born_source<<<grd, 256, 0, st>>>(u, dmc, w2, slot_f, n, b);
  count_launch();
}

void launch_residual_25d(const helm_plan& P, const double2* u, const int32_t* rec_idx, int nrec, const double2* d_obs,
                         const double* ck, const int* slot_f, const int* slot_s, int nsrc, int nk, int ngroups,
                         double2* res, double* f_grp, cudaStream_t st) {
  if (ngroups <= 0) return;
  k_residual_25d<<<ngroups, 256, 0, st>>>(geom(P), u, P.lev[0].n, rec_idx, nrec, d_obs, ck, slot_f, slot_s, nsrc, nk,
                                          res, f_grp);
  count_launch();
}

void launch_spread_25d(const helm_plan& P, const double2* res, const int32_t* rec_idx, int nrec, const double* ck,
                       const int* slot_f, int nk, int nslots, double2* b, cudaStream_t st) {
  if (nslots <= 0) return;
  dim3 grd((unsigned)((nrec + 127) / 128), nslots);
  k_spread_25d<<<grd, 128, 0, st>>>(geom(P), res, rec_idx, nrec, ck, slot_f, nk, nslots, b, P.lev[0].n);
  count_launch();
}

void launch_extend_adjoint(const helm_plan& P, const double* gcomp, double* g_phys, cudaStream_t st) {
  const size_t np = P.n_phys;
  k_extend_adjoint<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(geom(P), gcomp, g_phys);
  count_launch();
}

void launch_sum_f(const double* f_slot, const int* slots, int nslots, double* f_out, int accumulate,
                  cudaStream_t st) {
  k_sum_f<<<1, 1, 0, st>>>(f_slot, slots, nslots, f_out, accumulate);
  count_launch();
}

void launch_copy_fields(const double2* src, double2* dst, const int* slots, int nslots,
                        const int* dst_index, size_t n, cudaStream_t st) {
  if (nslots <= 0) return;
  dim3 grd((unsigned)((n + 255) / 256), nslots);
  k_copy_fields<double2><<<grd, 256, 0, st>>>(src, dst, slots, dst_index, n);
  count_launch();
}

void launch_copy_fields(const double2* src, float2* dst, const int* slots, int nslots, const int* dst_index, size_t n,
                        cudaStream_t st) {
  if (nslots <= 0) return;
  dim3 grd((unsigned)((n + 255) / 256), nslots);
  k_copy_fields<float2><<<grd, 256, 0, st>>>(src, dst, slots, dst_index, n);
  count_launch();
}

}  // namespace helm
