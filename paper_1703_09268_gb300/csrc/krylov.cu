// Batched Krylov vector kernels and per-right-hand-side bookkeeping.
//
// Arnoldi with classical Gram-Schmidt and one re-orthogonalisation pass
// (CGS2) for GMRES / FGMRES (Sec. 4 uses GMRES as smoother and FGMRES as
// outer and coarse solver).  Basis vectors are stored unnormalised with a
// per-slot scale s_i = 1/||v_i|| applied by every consumer, so no separate
// normalisation pass is needed.  Every reduction is two-stage and
// deterministic: fixed per-block partials (warp shuffles, then shared memory)
// summed in a fixed order in FP64 by a per-slot kernel.
#include <cmath>

#include "common.cuh"

namespace helm {

namespace {

constexpr int GS_THREADS = 256;
constexpr int GS_WARPS = GS_THREADS / 32;

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce `nvals` per-thread values (vals[k]) and write one partial row.
template <typename R, int NV>
__device__ __forceinline__ void block_partials(R (&vals)[NV], int nvals, double* out) {
  __shared__ double sh[GS_WARPS][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    if (k < nvals) {
      R v = warp_sum<R>(vals[k]);
      if (lane == 0) sh[wid][k] = (double)v;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nvals; k += blockDim.x) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < GS_WARPS; ++w) t += sh[w][k];
    out[k] = t;
  }
}

template <typename R, int MODE, int KM>
__global__ void __launch_bounds__(GS_THREADS)
k_gs(const cplx<R>* __restrict__ V, size_t vstride, int nv, const cplx<R>* __restrict__ coef,
     const cplx<R>* w, const R* __restrict__ wsc, int wss, cplx<R>* out,
     const int* __restrict__ act, size_t n, size_t chunk, double* __restrict__ partial) {
  using C = cplx<R>;
  const int a = blockIdx.y;
  const int s = act[a];
  const size_t beg = (size_t)blockIdx.x * chunk;
  const size_t end = min(n, beg + chunk);
  const C* Vs = V + (size_t)s * n;
  const C* W = w + (size_t)s * n;
  C* O = out ? out + (size_t)s * n : nullptr;
  const R sw = wsc ? wsc[(size_t)s * wss] : R(1);
  C cf[KM];
#pragma unroll
  for (int i = 0; i < KM; ++i)
    cf[i] = (MODE != GS_DOT && i < nv) ? coef[(size_t)s * (KMAX + 1) + i] : mkc(R(0), R(0));
  constexpr bool DOTS = (MODE == GS_DOT || MODE == GS_SUB_DOT);
  constexpr int NVAL = DOTS ? 2 * KM : 1;
  R acc[NVAL];
#pragma unroll
  for (int k = 0; k < NVAL; ++k) acc[k] = R(0);
  for (size_t p = beg + threadIdx.x; p < end; p += GS_THREADS) {
    C t = W[p];
    t = mkc(t.x * sw, t.y * sw);
    C v[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i)
      if (i < nv) v[i] = Vs[i * vstride + p];
    if (MODE == GS_SUB_DOT || MODE == GS_SUB_STORE_NORM) {
#pragma unroll
      for (int i = 0; i < KM; ++i)
        if (i < nv) t = cfms(cf[i], v[i], t);
    }
    if (MODE == GS_ADD_STORE) {
#pragma unroll
      for (int i = 0; i < KM; ++i)
        if (i < nv) t = cfma(cf[i], v[i], t);
      O[p] = t;
    }
    if (DOTS) {
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        if (i < nv) {
          acc[2 * i] = fma(v[i].x, t.x, fma(v[i].y, t.y, acc[2 * i]));
          acc[2 * i + 1] = fma(v[i].x, t.y, fma(-v[i].y, t.x, acc[2 * i + 1]));
        }
      }
    }
    if (MODE == GS_SUB_STORE_NORM) {
      if (O) O[p] = t;
      acc[0] = fma(t.x, t.x, fma(t.y, t.y, acc[0]));
    }
  }
  if (MODE == GS_ADD_STORE) return;
  const int nvals = DOTS ? 2 * nv : 1;
  block_partials<R, NVAL>(acc, nvals, partial + ((size_t)a * gridDim.x + blockIdx.x) * nvals);
}

template <typename R, int MODE, int KM>
void gs_go(dim3 grd, cudaStream_t st, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* coef,
           const cplx<R>* w, Scale<R> ws, cplx<R>* out, const int* act, size_t n, size_t chunk,
           double* partial) {
  k_gs<R, MODE, KM><<<grd, GS_THREADS, 0, st>>>(V, vstride, nv, coef, w, ws.p, ws.stride, out, act,
                                                n, chunk, partial);
}

template <typename R, int MODE>
void gs_pick(int nv, dim3 grd, cudaStream_t st, const cplx<R>* V, size_t vstride,
             const cplx<R>* coef, const cplx<R>* w, Scale<R> ws, cplx<R>* out, const int* act,
             size_t n, size_t chunk, double* partial) {
  if (nv <= 1)
    gs_go<R, MODE, 1>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, partial);
  else if (nv <= 4)
    gs_go<R, MODE, 4>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, partial);
  else if (nv <= 8)
    gs_go<R, MODE, 8>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, partial);
  else if (nv <= 16)
    gs_go<R, MODE, 16>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, partial);
  else
    gs_go<R, MODE, KMAX + 1>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, partial);
}

// ---- per-slot bookkeeping (one thread block per active slot) -------------

__device__ double sum_partials(const double* partial, int a, int nblk, int nvals, int k) {
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += partial[((size_t)a * nblk + b) * nvals + k];
  return t;
}

template <typename R>
__global__ void k_red_dots(const double* __restrict__ partial, int nblk, int nv,
                           const int* __restrict__ act, KState ks, int accumulate) {
  __shared__ double sh[2 * (KMAX + 1)];
  const int a = blockIdx.x;
  const int s = act[a];
  const int nvals = 2 * nv;
  for (int k = threadIdx.x; k < nvals; k += blockDim.x) sh[k] = sum_partials(partial, a, nblk, nvals, k);
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double sc = ks.scale[(size_t)s * (KMAX + 1) + i];
    double2 h = make_double2(sh[2 * i] * sc, sh[2 * i + 1] * sc);
    double2* hc = ks.hcol + (size_t)s * (KMAX + 1) + i;
    if (accumulate) h = make_double2(hc->x + h.x, hc->y + h.y);
    *hc = h;
    cplx<R>* cf = (cplx<R>*)ks.coef + (size_t)s * (KMAX + 1) + i;
    *cf = mkc((R)(h.x * sc), (R)(h.y * sc));
  }
}

template <typename R>
__global__ void k_red_norm_arnoldi(const double* __restrict__ partial, int nblk,
                                   const int* __restrict__ act, int na, KState ks, int j) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int s = act[a];
  const double nrm2 = sum_partials(partial, a, nblk, 1, 0);
  const double hn = sqrt(nrm2);
  const size_t so = (size_t)s * (KMAX + 1);
  const double inv = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
  ks.scale[so + j + 1] = inv;
  ((R*)ks.scale_r)[so + j + 1] = (R)inv;
  double2 col[KMAX + 1];
  for (int i = 0; i <= j; ++i) col[i] = ks.hcol[so + i];
  col[j + 1] = make_double2(hn, 0.0);
  double2* cs = ks.cs + (size_t)s * KMAX;
  double2* sn = ks.sn + (size_t)s * KMAX;
  // previous rotations G_i = [[c, s], [-conj(s), conj(c)]]
  for (int i = 0; i < j; ++i) {
    const double2 c = cs[i], z = sn[i], h0 = col[i], h1 = col[i + 1];
    col[i] = make_double2(c.x * h0.x - c.y * h0.y + z.x * h1.x - z.y * h1.y,
                          c.x * h0.y + c.y * h0.x + z.x * h1.y + z.y * h1.x);
    col[i + 1] = make_double2(-(z.x * h0.x + z.y * h0.y) + (c.x * h1.x + c.y * h1.y),
                              -(z.x * h0.y - z.y * h0.x) + (c.x * h1.y - c.y * h1.x));
  }
  // new rotation mapping (col[j], col[j+1]) to (rho, 0)
  const double2 p = col[j], q = col[j + 1];
  const double rho = hypot(hypot(p.x, p.y), hypot(q.x, q.y));
  double2 c, z;
  if (rho == 0.0) {
    c = make_double2(1.0, 0.0);
    z = make_double2(0.0, 0.0);
  } else {
    c = make_double2(p.x / rho, -p.y / rho);  // conj(p)/rho
    z = make_double2(q.x / rho, -q.y / rho);  // conj(q)/rho
  }
  cs[j] = c;
  sn[j] = z;
  col[j] = make_double2(rho, 0.0);
  col[j + 1] = make_double2(0.0, 0.0);
  double2* H = ks.H + (size_t)s * (KMAX + 1) * KMAX;
  for (int i = 0; i <= j; ++i) H[i * KMAX + j] = col[i];
  double2* g = ks.g + so;
  const double2 gj = g[j];
  g[j] = make_double2(c.x * gj.x - c.y * gj.y, c.x * gj.y + c.y * gj.x);
  g[j + 1] = make_double2(-(z.x * gj.x + z.y * gj.y), -(z.x * gj.y - z.y * gj.x));
  ks.est[s] = hypot(g[j + 1].x, g[j + 1].y);
}

template <typename R>
__global__ void k_red_start(const double* __restrict__ partial, int nblk, const int* __restrict__ act,
                            int na, KState ks, int set_bnorm) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int s = act[a];
  const double beta = sqrt(sum_partials(partial, a, nblk, 1, 0));
  const size_t so = (size_t)s * (KMAX + 1);
  const double inv = (beta > 0.0 && isfinite(beta)) ? 1.0 / beta : 0.0;
  ks.scale[so] = inv;
  ((R*)ks.scale_r)[so] = (R)inv;
  ks.g[so] = make_double2(beta, 0.0);
  for (int i = 1; i <= KMAX; ++i) ks.g[so + i] = make_double2(0.0, 0.0);
  ks.rnorm[s] = beta;
  ks.est[s] = beta;
  if (set_bnorm) ks.bnorm[s] = beta;
}

__global__ void k_red_norm(const double* __restrict__ partial, int nblk, const int* __restrict__ act,
                           int na, double* out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  out[act[a]] = sqrt(sum_partials(partial, a, nblk, 1, 0));
}

template <typename R>
__global__ void k_small_solve(const int* __restrict__ act, int na, KState ks, int k, int flexible) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int s = act[a];
  const size_t so = (size_t)s * (KMAX + 1);
  const double2* H = ks.H + (size_t)s * (KMAX + 1) * KMAX;
  const double2* g = ks.g + so;
  double2 y[KMAX];
  for (int i = k - 1; i >= 0; --i) {
    double2 t = g[i];
    for (int l = i + 1; l < k; ++l) {
      const double2 h = H[i * KMAX + l];
      t.x -= h.x * y[l].x - h.y * y[l].y;
      t.y -= h.x * y[l].y + h.y * y[l].x;
    }
    const double2 d = H[i * KMAX + i];
    const double den = d.x * d.x + d.y * d.y;
    if (den > 0.0 && isfinite(den)) {
      y[i] = make_double2((t.x * d.x + t.y * d.y) / den, (t.y * d.x - t.x * d.y) / den);
    } else {
      y[i] = make_double2(0.0, 0.0);
    }
  }
  cplx<R>* cf = (cplx<R>*)ks.coef + so;
  for (int i = 0; i < k; ++i) {
    const double sc = flexible ? 1.0 : ks.scale[so + i];
    cf[i] = mkc((R)(y[i].x * sc), (R)(y[i].y * sc));
  }
}

__global__ void k_to32_scaled(const double2* __restrict__ r, const double* __restrict__ rnorm,
                              float2* __restrict__ out, const int* __restrict__ act, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = act[blockIdx.y];
  const double rn = rnorm[s];
  const double inv = (rn > 0.0 && isfinite(rn)) ? 1.0 / rn : 0.0;
  const double2 v = r[(size_t)s * n + i];
  out[(size_t)s * n + i] = make_float2((float)(v.x * inv), (float)(v.y * inv));
}

__global__ void k_axpy_up(const float2* __restrict__ e, const double* __restrict__ rnorm,
                          double2* __restrict__ u, const int* __restrict__ act, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = act[blockIdx.y];
  const double rn = rnorm[s];
  const float2 v = e[(size_t)s * n + i];
  double2 t = u[(size_t)s * n + i];
  t.x = fma(rn, (double)v.x, t.x);
  t.y = fma(rn, (double)v.y, t.y);
  u[(size_t)s * n + i] = t;
}

template <typename R>
__global__ void k_zero(cplx<R>* __restrict__ x, const int* __restrict__ act, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[(size_t)act[blockIdx.y] * n + i] = mkc(R(0), R(0));
}

__global__ void k_check_finite(const double* __restrict__ vals, const int* __restrict__ act, int na,
                               int* bad) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  if (!isfinite(vals[act[a]])) atomicAdd(bad, 1);
}

}  // namespace

template <typename R>
int launch_gs(int mode, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* coef,
              const cplx<R>* w, Scale<R> ws, cplx<R>* out, const int* act, int na, size_t n,
              double* partial, cudaStream_t st) {
  if (na <= 0) return 0;
  int target = (152 * 8 + na - 1) / na;
  int maxb = (int)((n + GS_THREADS - 1) / GS_THREADS);
  int nblk = target < maxb ? target : maxb;
  if (nblk < 1) nblk = 1;
  // partial rows available: max(RED_BLOCKS_MAX, na) (see the workspace layout)
  if ((size_t)nblk * na > (size_t)RED_BLOCKS_MAX) nblk = RED_BLOCKS_MAX / na > 0 ? RED_BLOCKS_MAX / na : 1;
  const size_t chunk = (n + nblk - 1) / nblk;
  dim3 grd(nblk, na);
  double vecs = nv + 1;                        // V_0..V_{nv-1} and w read once
  if (mode == GS_SUB_STORE_NORM && out) vecs += 1;  // plus the stored result
  if (mode == GS_ADD_STORE) vecs += 1;         // x read and written
  ProfScope ps(sizeof(R) == 4 ? PC_GS32 : PC_GS64, vecs * na * n * sizeof(cplx<R>), st);
  switch (mode) {
    case GS_DOT: gs_pick<R, GS_DOT>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, partial); break;
    case GS_SUB_DOT: gs_pick<R, GS_SUB_DOT>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, partial); break;
    case GS_SUB_STORE_NORM: gs_pick<R, GS_SUB_STORE_NORM>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, partial); break;
    default: gs_pick<R, GS_ADD_STORE>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, partial); break;
  }
  count_launch();
  return nblk;
}

void launch_red_dots(const double* partial, int nblk, int nv, const int* act, int na, KState ks,
                     int accumulate, int rbytes, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_SMALL, 0.0, st);
  if (rbytes == 4)
    k_red_dots<float><<<na, 64, 0, st>>>(partial, nblk, nv, act, ks, accumulate);
  else
    k_red_dots<double><<<na, 64, 0, st>>>(partial, nblk, nv, act, ks, accumulate);
  count_launch();
}

void launch_red_norm_arnoldi(const double* partial, int nblk, const int* act, int na, KState ks,
                             int j, int rbytes, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_SMALL, 0.0, st);
  const int th = 64, bl = (na + th - 1) / th;
  if (rbytes == 4)
    k_red_norm_arnoldi<float><<<bl, th, 0, st>>>(partial, nblk, act, na, ks, j);
  else
    k_red_norm_arnoldi<double><<<bl, th, 0, st>>>(partial, nblk, act, na, ks, j);
  count_launch();
}

void launch_red_start(const double* partial, int nblk, const int* act, int na, KState ks,
                      int set_bnorm, int rbytes, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_SMALL, 0.0, st);
  const int th = 64, bl = (na + th - 1) / th;
  if (rbytes == 4)
    k_red_start<float><<<bl, th, 0, st>>>(partial, nblk, act, na, ks, set_bnorm);
  else
    k_red_start<double><<<bl, th, 0, st>>>(partial, nblk, act, na, ks, set_bnorm);
  count_launch();
}

void launch_red_norm(const double* partial, int nblk, const int* act, int na, double* out,
                     cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_SMALL, 0.0, st);
  const int th = 64, bl = (na + th - 1) / th;
  k_red_norm<<<bl, th, 0, st>>>(partial, nblk, act, na, out);
  count_launch();
}

void launch_small_solve(const int* act, int na, KState ks, int k, int flexible, int rbytes,
                        cudaStream_t st) {
  if (na <= 0 || k <= 0) return;
  ProfScope ps(PC_SMALL, 0.0, st);
  const int th = 32, bl = (na + th - 1) / th;
  if (rbytes == 4)
    k_small_solve<float><<<bl, th, 0, st>>>(act, na, ks, k, flexible);
  else
    k_small_solve<double><<<bl, th, 0, st>>>(act, na, ks, k, flexible);
  count_launch();
}

void launch_to32_scaled(const double2* r, const double* rnorm, float2* out, const int* act, int na,
                        size_t n, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * n * (16 + 8), st);
  dim3 grd((unsigned)((n + 255) / 256), na);
  k_to32_scaled<<<grd, 256, 0, st>>>(r, rnorm, out, act, n);
  count_launch();
}

void launch_axpy_up(const float2* e, const double* rnorm, double2* u, const int* act, int na,
                    size_t n, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * n * (8 + 16 + 16), st);
  dim3 grd((unsigned)((n + 255) / 256), na);
  k_axpy_up<<<grd, 256, 0, st>>>(e, rnorm, u, act, n);
  count_launch();
}

template <typename R>
void launch_zero(cplx<R>* x, const int* act, int na, size_t n, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * n * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((n + 255) / 256), na);
  k_zero<R><<<grd, 256, 0, st>>>(x, act, n);
  count_launch();
}

void launch_check_finite(const double* vals, const int* act, int na, int* bad, cudaStream_t st) {
  if (na <= 0) return;
  k_check_finite<<<(na + 63) / 64, 64, 0, st>>>(vals, act, na, bad);
  count_launch();
}

template int launch_gs<float>(int, const float2*, size_t, int, const float2*, const float2*,
                              Scale<float>, float2*, const int*, int, size_t, double*, cudaStream_t);
template int launch_gs<double>(int, const double2*, size_t, int, const double2*, const double2*,
                               Scale<double>, double2*, const int*, int, size_t, double*, cudaStream_t);
template void launch_zero<float>(float2*, const int*, int, size_t, cudaStream_t);
template void launch_zero<double>(double2*, const int*, int, size_t, cudaStream_t);

}  // namespace helm
