// Batched Krylov vector kernels.
//
// Arnoldi with classical Gram-Schmidt, optionally with one
// re-orthogonalisation pass (CGS2), for GMRES / FGMRES (Sec. 4 uses GMRES as
// smoother and FGMRES as outer and coarse solver).  Basis vectors are stored
// unnormalised with a per-slot scale s_i = 1/||v_i|| applied by every
// consumer, so no normalisation pass is needed.  Each pass carries its own
// deterministic reduction and per-slot epilogue (reduce.cuh).
#include <cmath>
#include <cstdint>

#include "reduce.cuh"
#include "tma.cuh"

namespace helm {

namespace {

constexpr int GS_THREADS = 256;

template <typename R, int MODE, int KM>
__global__ void __launch_bounds__(GS_THREADS)
k_gs(const cplx<R>* __restrict__ V, size_t vstride, int nv, const cplx<R>* __restrict__ coef,
     const cplx<R>* w, const R* __restrict__ wsc, int wss, cplx<R>* out, const int* __restrict__ act,
     size_t n, size_t chunk, Epi e) {
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
  if (MODE == GS_ADD_STORE || e.kind == EPI_NONE) return;
  const int nvals = DOTS ? 2 * nv : 1;
  block_partial_row<R, NVAL, GS_THREADS / 32>(acc, nvals, e.partial + ((size_t)a * gridDim.x + blockIdx.x) * nvals);
  epi_arrive<R>(e, a, s, gridDim.x, nvals);
}

template <typename R, int MODE, int KM>
void gs_go(dim3 grd, cudaStream_t st, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* coef,
           const cplx<R>* w, Scale<R> ws, cplx<R>* out, const int* act, size_t n, size_t chunk, const Epi& e) {
  k_gs<R, MODE, KM><<<grd, GS_THREADS, 0, st>>>(V, vstride, nv, coef, w, ws.p, ws.stride, out, act, n, chunk, e);
}

template <typename R, int MODE>
void gs_pick(int nv, dim3 grd, cudaStream_t st, const cplx<R>* V, size_t vstride, const cplx<R>* coef,
             const cplx<R>* w, Scale<R> ws, cplx<R>* out, const int* act, size_t n, size_t chunk, const Epi& e) {
  if (nv <= 1)
    gs_go<R, MODE, 1>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, e);
  else if (nv <= 4)
    gs_go<R, MODE, 4>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, e);
  else if (nv <= 8)
    gs_go<R, MODE, 8>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, e);
  else if (nv <= 16)
    gs_go<R, MODE, 16>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, e);
  else
    gs_go<R, MODE, KMAX + 1>(grd, st, V, vstride, nv, coef, w, ws, out, act, n, chunk, e);
}

// Elements p and p+1 of a complex field whose global index p is even: one
// 16-byte access in single precision, two in double.
template <typename R> __device__ __forceinline__ void ld_pair(const cplx<R>* q, cplx<R>& a, cplx<R>& b) {
  if constexpr (sizeof(R) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(q);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
  } else {
    a = q[0];
    b = q[1];
  }
}
template <typename R> __device__ __forceinline__ void st_pair(cplx<R>* q, cplx<R> a, cplx<R> b) {
  if constexpr (sizeof(R) == 4) {
    *reinterpret_cast<float4*>(q) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    q[0] = a;
    q[1] = b;
  }
}

// Paired traversal of one slot's field: with VEC the points are visited in
// pairs (p, p+1) starting at the first even global index, and the odd head /
// tail points (at most one each) are returned separately.
struct PairSplit {
  int head;        // 1 when the slot's first point has an odd global index
  size_t npair;    // pairs after the head
  bool tail;       // one point left after the pairs
};
__device__ __forceinline__ PairSplit pair_split(size_t slot_base, size_t n) {
  PairSplit ps;
  ps.head = (int)(slot_base & 1) && n > 0 ? 1 : 0;
  ps.npair = (n - ps.head) >> 1;
  ps.tail = ((n - ps.head) & 1) != 0;
  return ps;
}

// Gram sums of one point: <W_i, W_j> (1 <= i <= j <= S), <W_i, W_0>, ||W_0||^2.
template <typename R, int S>
__device__ __forceinline__ void gram_point(const cplx<R>* w, R* acc) {
  int k = 0;
#pragma unroll
  for (int i = 1; i <= S; ++i) {
#pragma unroll
    for (int j = i; j <= S; ++j, ++k) {
      acc[2 * k] = fma(w[i].x, w[j].x, fma(w[i].y, w[j].y, acc[2 * k]));
      acc[2 * k + 1] = fma(w[i].x, w[j].y, fma(-w[i].y, w[j].x, acc[2 * k + 1]));
    }
  }
#pragma unroll
  for (int i = 1; i <= S; ++i, ++k) {
    acc[2 * k] = fma(w[i].x, w[0].x, fma(w[i].y, w[0].y, acc[2 * k]));
    acc[2 * k + 1] = fma(w[i].x, w[0].y, fma(-w[i].y, w[0].x, acc[2 * k + 1]));
  }
  acc[2 * k] = fma(w[0].x, w[0].x, fma(w[0].y, w[0].y, acc[2 * k]));
}

// Gram pass of an s-step cycle: raw <W_i, W_j> (1 <= i <= j <= S) and
// <W_i, W_0> over the stored basis W_0..W_S, folded into EPI_GRAM.  Block b of
// a slot covers units [b*chunk, (b+1)*chunk), a unit being a point (VEC false)
// or a pair of points (VEC true).
template <typename R, int S, bool VEC>
__global__ void __launch_bounds__(GS_THREADS, VEC ? 2 : (sizeof(R) == 4 ? 3 : 2))
k_gram(const cplx<R>* __restrict__ V, size_t vstride, const int* __restrict__ act, size_t n, size_t chunk, Epi e) {
  using C = cplx<R>;
  constexpr int NV = gram_nvals(S);
  const int a = blockIdx.y;
  const int s = act[a];
  const C* Vs = V + (size_t)s * n;
  R acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = R(0);
  if (VEC) {
    const PairSplit sp = pair_split((size_t)s * n, n);
    const size_t beg = (size_t)blockIdx.x * chunk;
    const size_t end = min(sp.npair, beg + chunk);
    for (size_t q = beg + threadIdx.x; q < end; q += GS_THREADS) {
      const size_t p = sp.head + 2 * q;
      C wa[S + 1], wb[S + 1];
#pragma unroll
      for (int i = 0; i <= S; ++i) ld_pair<R>(Vs + i * vstride + p, wa[i], wb[i]);
      gram_point<R, S>(wa, acc);
      gram_point<R, S>(wb, acc);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      C w[S + 1];
      if (sp.head) {
#pragma unroll
        for (int i = 0; i <= S; ++i) w[i] = Vs[i * vstride];
        gram_point<R, S>(w, acc);
      }
      if (sp.tail) {
#pragma unroll
        for (int i = 0; i <= S; ++i) w[i] = Vs[i * vstride + n - 1];
        gram_point<R, S>(w, acc);
      }
    }
  } else {
    const size_t beg = (size_t)blockIdx.x * chunk;
    const size_t end = min(n, beg + chunk);
    for (size_t p = beg + threadIdx.x; p < end; p += GS_THREADS) {
      C w[S + 1];
#pragma unroll
      for (int i = 0; i <= S; ++i) w[i] = Vs[i * vstride + p];
      gram_point<R, S>(w, acc);
    }
  }
  block_partial_row<R, NV, GS_THREADS / 32>(acc, NV, e.partial + ((size_t)a * gridDim.x + blockIdx.x) * NV);
  epi_arrive<R>(e, a, s, gridDim.x, NV);
}

// Gram pass with the basis streamed into shared memory by bulk asynchronous
// copies (TMA): a ring of GRAM_STAGES tiles of GS_THREADS point pairs per
// vector, each tile announced on its own mbarrier.  Thread 0 keeps the ring
// full while all threads reduce the tile in front; memory traffic and the
// arithmetic (about 4.5 flops per byte) overlap instead of alternating.
// Single precision, pairs of points (the same layout conditions as the paired
// kernels).  A wait that gives up sets e.fault and the block stops streaming
// (its sums are void; the call reports HELM_E_TIMEOUT).
template <int S> __host__ __device__ constexpr int gram_stages() {
  return (S + 1) * 4096 * 4 <= 100 * 1024 ? 4 : (S + 1) * 4096 * 3 <= 100 * 1024 ? 3 : 2;
}
template <int S> __host__ __device__ constexpr size_t gram_tma_smem() { return (size_t)gram_stages<S>() * (S + 1) * GS_THREADS * 16; }

template <int S>
__global__ void __launch_bounds__(GS_THREADS, 2)
k_gram_tma(const float2* __restrict__ V, size_t vstride, const int* __restrict__ act, size_t n, size_t chunk,
           Epi e) {
  constexpr int NV = gram_nvals(S);
  constexpr int ST = gram_stages<S>();
  constexpr int TP = GS_THREADS;
  extern __shared__ __align__(128) float4 ring[];  // [ST][S+1][TP]
  __shared__ __align__(8) uint64_t full[ST];
  const int a = blockIdx.y;
  const int s = act[a];
  const int tid = threadIdx.x;
  const float2* Vs = V + (size_t)s * n;
  const PairSplit sp = pair_split((size_t)s * n, n);
  const size_t beg = min(sp.npair, (size_t)blockIdx.x * chunk);
  const size_t end = min(sp.npair, beg + chunk);
  const int ntile = (int)((end - beg + TP - 1) / TP);
  if (tid == 0) {
    for (int st = 0; st < ST; ++st) mbar_init(&full[st], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int t) {  // thread 0: tile t into stage t % ST
    const int st = t % ST;
    const size_t q0 = beg + (size_t)t * TP;
    const uint32_t bytes = (uint32_t)min((size_t)TP, end - q0) * 16u;
    mbar_arrive_expect_tx(&full[st], bytes * (S + 1));
#pragma unroll
    for (int i = 0; i <= S; ++i)
      bulk_g2s(ring + ((size_t)st * (S + 1) + i) * TP, Vs + i * vstride + sp.head + 2 * q0, bytes, &full[st]);
  };
  if (tid == 0)
    for (int t = 0; t < min(ST, ntile); ++t) issue(t);
  float acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.f;
  int done = 0;  // tiles consumed
  bool failed = false;
  for (int t = 0; t < ntile; ++t) {
    const int st = t % ST;
    const bool ok = mbar_wait_bounded(&full[st], (uint32_t)(t / ST) & 1u);
    // one barrier per tile: everyone has left tile t-1 (its stage may be
    // refilled) and agrees on whether tile t arrived
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0 && t >= 1 && t - 1 + ST < ntile) issue(t - 1 + ST);
    const size_t q0 = beg + (size_t)t * TP;
    if (q0 + tid < end) {
      float2 wa[S + 1], wb[S + 1];
#pragma unroll
      for (int i = 0; i <= S; ++i) {
        const float4 v = ring[((size_t)st * (S + 1) + i) * TP + tid];
        wa[i] = make_float2(v.x, v.y);
        wb[i] = make_float2(v.z, v.w);
      }
      gram_point<float, S>(wa, acc);
      gram_point<float, S>(wb, acc);
    }
    done = t + 1;
  }
  if (failed && tid == 0) {
    if (e.fault) atomicExch(e.fault, 1);
    // let the copies already issued land (bounded) before the block exits
    const int issued = min(ntile, max(ST, done + ST - 1));
    for (int t = done; t < issued; ++t) (void)mbar_wait_bounded(&full[t % ST], (uint32_t)(t / ST) & 1u);
  }
  if (blockIdx.x == 0 && tid == 0) {
    float2 w[S + 1];
    if (sp.head) {
#pragma unroll
      for (int i = 0; i <= S; ++i) w[i] = Vs[i * vstride];
      gram_point<float, S>(w, acc);
    }
    if (sp.tail) {
#pragma unroll
      for (int i = 0; i <= S; ++i) w[i] = Vs[i * vstride + n - 1];
      gram_point<float, S>(w, acc);
    }
  }
  block_partial_row<float, NV, GS_THREADS / 32>(acc, NV, e.partial + ((size_t)a * gridDim.x + blockIdx.x) * NV);
  epi_arrive<float>(e, a, s, gridDim.x, NV);
}

// End of an s-step cycle: x += sum_{i<S} y_i W_i (x = sum_i y_i W_i when
// xzero), and with recur the next residual by recurrence in the same pass,
// W_0 <- W_0 - sum_{i<S} y_i W_{i+1} (= b - H x_new since W_{i+1} = H W_i).
template <typename R, int S>
__device__ __forceinline__ void sstep_point(const cplx<R>* cf, const cplx<R>* w, cplx<R>& xv, cplx<R>& r,
                                            bool recur) {
  r = w[0];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    xv = cfma(cf[i], w[i], xv);
    if (recur) r = cfms(cf[i], w[i + 1], r);
  }
}

template <typename R, int S, bool VEC>
__global__ void __launch_bounds__(GS_THREADS)
k_sstep_update(cplx<R>* V, size_t vstride, const cplx<R>* __restrict__ coef, cplx<R>* x,
               const int* __restrict__ act, size_t n, int recur, int xzero) {
  using C = cplx<R>;
  const int s = act[blockIdx.y];
  C cf[S];
#pragma unroll
  for (int i = 0; i < S; ++i) cf[i] = coef[(size_t)s * (KMAX + 1) + i];
  C* Vs = V + (size_t)s * n;
  C* X = x + (size_t)s * n;
  const int nw = recur ? S + 1 : S;  // W_S only feeds the recurrence
  const C zero = mkc(R(0), R(0));
  auto one = [&](size_t p) {
    C w[S + 1];
#pragma unroll
    for (int i = 0; i <= S; ++i) w[i] = i < nw ? Vs[i * vstride + p] : zero;
    C xv = xzero ? zero : X[p], r;
    sstep_point<R, S>(cf, w, xv, r, recur);
    X[p] = xv;
    if (recur) Vs[p] = r;
  };
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if (VEC) {
    const PairSplit sp = pair_split((size_t)s * n, n);
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < sp.npair; q += stride) {
      const size_t p = sp.head + 2 * q;
      C wa[S + 1], wb[S + 1];
#pragma unroll
      for (int i = 0; i <= S; ++i) {
        if (i < nw) ld_pair<R>(Vs + i * vstride + p, wa[i], wb[i]);
        else wa[i] = wb[i] = zero;
      }
      C xa = zero, xb = zero, ra, rb;
      if (!xzero) ld_pair<R>(X + p, xa, xb);
      sstep_point<R, S>(cf, wa, xa, ra, recur);
      sstep_point<R, S>(cf, wb, xb, rb, recur);
      st_pair<R>(X + p, xa, xb);
      if (recur) st_pair<R>(Vs + p, ra, rb);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (sp.head) one(0);
      if (sp.tail) one(n - 1);
    }
  } else {
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) one(p);
  }
}

template <typename R, int S, bool VEC>
void sup_go(dim3 grd, cudaStream_t st, cplx<R>* V, size_t vstride, const cplx<R>* coef, cplx<R>* x, const int* act,
            size_t n, int recur, int xzero) {
  k_sstep_update<R, S, VEC><<<grd, GS_THREADS, 0, st>>>(V, vstride, coef, x, act, n, recur, xzero);
}

template <typename R, int S, bool VEC>
void gram_go(dim3 grd, cudaStream_t st, const cplx<R>* V, size_t vstride, const int* act, size_t n, size_t chunk,
             const Epi& e) {
  k_gram<R, S, VEC><<<grd, GS_THREADS, 0, st>>>(V, vstride, act, n, chunk, e);
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

}  // namespace

int reduction_blocks(int na, size_t n, int threads) {
  int target = (152 * 8 + na - 1) / na;
  int maxb = (int)((n + threads - 1) / threads);
  int nblk = target < maxb ? target : maxb;
  if (nblk < 1) nblk = 1;
  // partial rows available: max(RED_BLOCKS_MAX, na) (see the workspace layout)
  if ((size_t)nblk * na > (size_t)RED_BLOCKS_MAX) nblk = RED_BLOCKS_MAX / na > 0 ? RED_BLOCKS_MAX / na : 1;
  return nblk;
}

template <typename R>
void launch_gs(int mode, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* coef, const cplx<R>* w,
               Scale<R> ws, cplx<R>* out, const int* act, int na, size_t n, const Epi& e, cudaStream_t st) {
  if (na <= 0) return;
  const int nblk = reduction_blocks(na, n, GS_THREADS);
  const size_t chunk = (n + nblk - 1) / nblk;
  dim3 grd(nblk, na);
  double vecs = nv + 1;                             // V_0..V_{nv-1} and w read once
  if (mode == GS_SUB_STORE_NORM && out) vecs += 1;  // plus the stored result
  if (mode == GS_ADD_STORE) vecs += 1;              // x read and written
  ProfScope ps(prof_gs_class<R>(n, mode == GS_ADD_STORE ? PC_UPDATE32 : PC_GS32), vecs * na * n * sizeof(cplx<R>),
               st);
  switch (mode) {
    case GS_DOT: gs_pick<R, GS_DOT>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, e); break;
    case GS_SUB_DOT: gs_pick<R, GS_SUB_DOT>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, e); break;
    case GS_SUB_STORE_NORM:
      gs_pick<R, GS_SUB_STORE_NORM>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, e);
      break;
    default: gs_pick<R, GS_ADD_STORE>(nv, grd, st, V, vstride, coef, w, ws, out, act, n, chunk, e); break;
  }
  count_launch();
}

// Paired 16-byte accesses need every basis vector of a slot to start at the
// same parity (even vstride) and 16-byte aligned bases; single precision only.
template <typename R>
static bool use_pairs(const void* V, size_t vstride, const void* x) {
  return sizeof(R) == 4 && vstride % 2 == 0 && ((uintptr_t)V & 15) == 0 && ((uintptr_t)x & 15) == 0;
}

template <typename R, template <typename, int, bool> class F, typename... A>
static void s_dispatch(int s, bool vec, A&&... args) {
  switch (s * 2 + (vec ? 1 : 0)) {
#define HELM_S_CASE(S)                                       \
  case 2 * S: F<R, S, false>::go(args...); break;            \
  case 2 * S + 1: F<R, S, true>::go(args...); break;
    HELM_S_CASE(1) HELM_S_CASE(2) HELM_S_CASE(3) HELM_S_CASE(4)
    HELM_S_CASE(5) HELM_S_CASE(6) HELM_S_CASE(7) HELM_S_CASE(8)
#undef HELM_S_CASE
    default: break;
  }
}
template <typename R, int S, bool VEC> struct GramGo {
  static void go(dim3 grd, cudaStream_t st, const cplx<R>* V, size_t vstride, const int* act, size_t n, size_t chunk,
                 const Epi& e) {
    if constexpr (VEC && sizeof(R) == 4) {
      // dynamic shared memory above 48 KB is opt-in, once per kernel and device
      static std::atomic<bool> attr[64];
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64 || !attr[dev].load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(k_gram_tma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tma_smem<S>());
        if (dev >= 0 && dev < 64) attr[dev].store(true, std::memory_order_release);
      }
      k_gram_tma<S><<<grd, GS_THREADS, gram_tma_smem<S>(), st>>>((const float2*)V, vstride, act, n, chunk, e);
    } else {
      gram_go<R, S, false>(grd, st, V, vstride, act, n, chunk, e);
    }
  }
};
template <typename R, int S, bool VEC> struct SupGo {
  static void go(dim3 grd, cudaStream_t st, cplx<R>* V, size_t vstride, const cplx<R>* coef, cplx<R>* x,
                 const int* act, size_t n, int recur, int xzero) {
    sup_go<R, S, VEC && sizeof(R) == 4>(grd, st, V, vstride, coef, x, act, n, recur, xzero);
  }
};

template <typename R>
void launch_gram(const cplx<R>* V, size_t vstride, int s, const int* act, int na, size_t n, const Epi& e,
                 cudaStream_t st) {
  if (na <= 0 || s < 1 || s > SSTEP_MAX) return;
  const bool vec = use_pairs<R>(V, vstride, V);
  const size_t units = vec ? n / 2 : n;
  // the streamed (paired) kernel holds two blocks per SM: one wave of them
  int nblk = vec ? std::max(1, std::min((int)((units + GS_THREADS - 1) / GS_THREADS), 2 * 152 / na))
                 : reduction_blocks(na, n, GS_THREADS);
  if ((size_t)nblk * na > (size_t)RED_BLOCKS_MAX) nblk = std::max(1, RED_BLOCKS_MAX / na);
  const size_t chunk = (units + nblk - 1) / nblk;
  dim3 grd(nblk, na);
  ProfScope ps(prof_gs_class<R>(n, PC_GRAM32), (double)(s + 1) * na * n * sizeof(cplx<R>), st);
  s_dispatch<R, GramGo>(s, vec, grd, st, V, vstride, act, n, chunk, e);
  count_launch();
}

template <typename R>
void launch_sstep_update(cplx<R>* V, size_t vstride, int s, const cplx<R>* coef, cplx<R>* x, const int* act, int na,
                         size_t n, int recur, int xzero, cudaStream_t st) {
  if (na <= 0 || s < 1 || s > SSTEP_MAX) return;
  const bool vec = use_pairs<R>(V, vstride, x);
  const size_t units = vec ? n / 2 + 1 : n;
  const int per_slot = std::max(1, std::min((int)((units + GS_THREADS - 1) / GS_THREADS), (152 * 8 + na - 1) / na));
  dim3 grd(per_slot, na);
  // bytes: W_0..W_{s-1} (and W_s) read, x read unless zero, x written (and W_0)
  const double vecs = s + (recur ? 2 : 0) + (xzero ? 1 : 2);
  ProfScope ps(prof_gs_class<R>(n, PC_UPDATE32), vecs * na * n * sizeof(cplx<R>), st);
  s_dispatch<R, SupGo>(s, vec, grd, st, V, vstride, coef, x, act, n, recur, xzero);
  count_launch();
}

void launch_to32_scaled(const double2* r, const double* rnorm, float2* out, const int* act, int na, size_t n,
                        cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * n * (16 + 8), st);
  dim3 grd((unsigned)((n + 255) / 256), na);
  k_to32_scaled<<<grd, 256, 0, st>>>(r, rnorm, out, act, n);
  count_launch();
}

void launch_axpy_up(const float2* e, const double* rnorm, double2* u, const int* act, int na, size_t n,
                    cudaStream_t st) {
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

template void launch_gs<float>(int, const float2*, size_t, int, const float2*, const float2*, Scale<float>, float2*,
                               const int*, int, size_t, const Epi&, cudaStream_t);
template void launch_gs<double>(int, const double2*, size_t, int, const double2*, const double2*, Scale<double>,
                                double2*, const int*, int, size_t, const Epi&, cudaStream_t);
template void launch_sstep_update<float>(float2*, size_t, int, const float2*, float2*, const int*, int, size_t,
                                         int, int, cudaStream_t);
template void launch_sstep_update<double>(double2*, size_t, int, const double2*, double2*, const int*, int, size_t,
                                          int, int, cudaStream_t);
template void launch_gram<float>(const float2*, size_t, int, const int*, int, size_t, const Epi&, cudaStream_t);
template void launch_gram<double>(const double2*, size_t, int, const int*, int, size_t, const Epi&, cudaStream_t);
template void launch_zero<float>(float2*, const int*, int, size_t, cudaStream_t);
template void launch_zero<double>(double2*, const int*, int, size_t, cudaStream_t);

}  // namespace helm
