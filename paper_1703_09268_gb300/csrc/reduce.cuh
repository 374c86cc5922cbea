// Deterministic per-right-hand-side reductions folded into the producing
// kernel, and the Arnoldi bookkeeping that consumes them.
//
// Every block of a slot writes one row of FP64 partial sums; the last block
// to arrive (atomic ticket after a fence) sums the rows in block order and
// runs the epilogue for that slot: Gram-Schmidt coefficients, the Givens
// update of the Hessenberg column (and, after the last column of a cycle, the
// small triangular solve), a restart norm, or a plain norm.  The result does
// not depend on block scheduling.
#pragma once

#include "common.cuh"

namespace helm {

enum EpiKind { EPI_NONE = 0, EPI_DOTS = 1, EPI_ARNOLDI = 2, EPI_START = 3, EPI_NORM = 4, EPI_GRAM = 5 };

constexpr int SSTEP_MAX = 8;  // longest s-step basis (s+1 stored vectors)
// Gram pass values: <W_i, W_j> for 1 <= i <= j <= s, <W_i, W_0> for 1 <= i <= s, and ||W_0||^2 (complex pairs)
__host__ __device__ constexpr int gram_nvals(int s) { return 2 * (s * (s + 1) / 2 + s + 1); }

struct Epi {
  int kind = EPI_NONE;
  int nv = 0;             // EPI_DOTS: number of basis vectors
  int accumulate = 0;     // EPI_DOTS: add to the current column (second Gram-Schmidt pass)
  int j = 0;              // EPI_ARNOLDI: column index
  int ksolve = 0;         // EPI_ARNOLDI: solve the least-squares problem after column ksolve-1
  int flex = 0;           // EPI_ARNOLDI: update coefficients for Z (flexible) or scaled V
  int set_bnorm = 0;      // EPI_START: also record ||b||
  int idx = 0;            // EPI_GRAM: s (the basis has s+1 stored vectors)
  KState ks{};
  double* out = nullptr;       // EPI_NORM: out[slot] = sqrt(sum)
  unsigned* counter = nullptr; // [B] arrival tickets, zero between launches
  double* partial = nullptr;   // [rows][nvals]
  int* fault = nullptr;        // set to 1 by a kernel that gave up on a bounded wait
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce vals[0..nvals) (every thread of the block calls this) and write
// the block's partial row.
template <typename R, int NV, int MAXW>
__device__ __forceinline__ void block_partial_row(R (&vals)[NV], int nvals, double* row) {
  __shared__ double sh[MAXW][NV];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    if (k < nvals) {
      const R v = warp_sum<R>(vals[k]);
      if (lane == 0) sh[wid][k] = (double)v;
    }
  }
  __syncthreads();
  for (int k = tid; k < nvals; k += nthr) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[w][k];
    row[k] = t;
  }
}

__device__ __forceinline__ double2 shfl_d2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
// a - b * c
__device__ __forceinline__ double2 d2_fms(double2 a, double2 b, double2 c) {
  return make_double2(a.x - (b.x * c.x - b.y * c.y), a.y - (b.x * c.y + b.y * c.x));
}
// a - conj(b) * c
__device__ __forceinline__ double2 d2_fmsc(double2 a, double2 b, double2 c) {
  return make_double2(a.x - (b.x * c.x + b.y * c.y), a.y - (b.x * c.y - b.y * c.x));
}

// Per-slot epilogue, run by the 32 lanes of the first warp of the block that
// folded the slot's sums (in shared memory).  The small dense algebra is
// spread over the lanes so that its dependency chains are O(k) rather than
// O(k^2) or O(k^3) long: FP64 is a narrow pipe on this part and one thread
// walking a k^3 loop would idle the GPU for tens of microseconds.
template <typename R>
__device__ __noinline__ void epilogue(const Epi& e, int s, const double* sums, int lane) {
  const KState& ks = e.ks;
  const size_t so = (size_t)s * (KMAX + 1);
  if (e.kind == EPI_NORM) {
    if (lane == 0) e.out[s] = sqrt(sums[0]);
    return;
  }
  if (e.kind == EPI_GRAM) {
    // s-step minimal-residual update.  The basis is W_0 = r0, W_{i+1} = H W_i
    // (unnormalised; the diagonal scaling below takes care of magnitudes).
    // Minimise ||r0 - sum_i y_i W_{i+1}|| through the normal equations
    // G y = c, G_ij = <W_{i+1}, W_{j+1}>, c_i = <W_{i+1}, r0>, scaled to unit
    // diagonal and solved by a Cholesky factorisation that drops directions
    // with a negligible pivot; then x += sum_i y_i W_i.
    __shared__ double2 sG[SSTEP_MAX][SSTEP_MAX];
    __shared__ double ssg[SSTEP_MAX], sinv[SSTEP_MAX];
    const int S = e.idx;
    const int KS = S * (S + 1) / 2;
    // packed upper triangle: (a, b), a <= b, at a*S - a(a-1)/2 + (b - a)
    for (int q = lane; q < S * S; q += 32) {
      const int i = q / S, j = q % S;
      const int a = min(i, j), b = max(i, j);
      const int k = a * S - a * (a - 1) / 2 + (b - a);
      sG[i][j] = make_double2(sums[2 * k], i <= j ? sums[2 * k + 1] : -sums[2 * k + 1]);
    }
    const double r0sq = sums[2 * (KS + S)];
    double2 ci = make_double2(0.0, 0.0);
    double sgl = 0.0;
    if (lane < S) {
      const double d = sums[2 * (lane * S - lane * (lane - 1) / 2)];
      sgl = (d > 0.0 && isfinite(d)) ? 1.0 / sqrt(d) : 0.0;
      ssg[lane] = sgl;
      ci = make_double2(sums[2 * (KS + lane)] * sgl, sums[2 * (KS + lane) + 1] * sgl);
    }
    __syncwarp();
    for (int q = lane; q < S * S; q += 32) {
      const int i = q / S, j = q % S;
      const double f = ssg[i] * ssg[j];
      sG[i][j] = make_double2(sG[i][j].x * f, sG[i][j].y * f);
    }
    __syncwarp();
    // right-looking Cholesky G = L L^H (lower triangle in place); a pivot at
    // or below the threshold drops its direction (column of L set to zero)
    const double thr = sizeof(R) == 4 ? 1e-6 : 1e-12;
    for (int j = 0; j < S; ++j) {
      if (lane == 0) {
        const double d = sG[j][j].x;
        const bool live = d > thr && isfinite(d);
        const double r = live ? sqrt(d) : 0.0;
        sG[j][j] = make_double2(r, 0.0);
        sinv[j] = live ? 1.0 / r : 0.0;
      }
      __syncwarp();
      const double iv = sinv[j];
      if (lane > j && lane < S) sG[lane][j] = make_double2(sG[lane][j].x * iv, sG[lane][j].y * iv);
      __syncwarp();
      for (int q = lane; q < S * S; q += 32) {
        const int i = q / S, k = q % S;
        if (k > j && k <= i) sG[i][k] = d2_fms(sG[i][k], sG[i][j], make_double2(sG[k][j].x, -sG[k][j].y));
      }
      __syncwarp();
    }
    // L w = c (column sweep; lane i holds row i), then L^H z = w
    double2 t = ci, wz = make_double2(0.0, 0.0);
    for (int j = 0; j < S; ++j) {
      const double2 tj = shfl_d2(t, j);
      const double2 wj = make_double2(tj.x * sinv[j], tj.y * sinv[j]);
      if (lane > j && lane < S) t = d2_fms(t, sG[lane][j], wj);
      if (lane == j) wz = wj;
    }
    t = wz;
    for (int i = S - 1; i >= 0; --i) {
      const double2 ti = shfl_d2(t, i);
      const double2 zi = make_double2(ti.x * sinv[i], ti.y * sinv[i]);
      if (lane < i) t = d2_fmsc(t, sG[i][lane], zi);
      if (lane == i) wz = zi;
    }
    // Re(c^H z) in scaled variables: the squared residual reduction
    double red = lane < S ? ci.x * wz.x + ci.y * wz.y : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) red += __shfl_xor_sync(0xffffffffu, red, o);
    // y_i = sg_i z_i multiplies W_i in the update
    if (lane < S) ((cplx<R>*)ks.coef)[so + lane] = mkc((R)(wz.x * sgl), (R)(wz.y * sgl));
    if (lane == 0) {
      ks.rnorm[s] = sqrt(r0sq);
      ks.est[s] = sqrt(fmax(0.0, r0sq - red));
    }
    __syncwarp();
    return;
  }
  if (e.kind == EPI_START) {
    const double beta = sqrt(sums[0]);
    if (lane == 0) {
      const double inv = (beta > 0.0 && isfinite(beta)) ? 1.0 / beta : 0.0;
      ks.scale[so] = inv;
      ((R*)ks.scale_r)[so] = (R)inv;
      ks.g[so] = make_double2(beta, 0.0);
      ks.rnorm[s] = beta;
      ks.est[s] = beta;
      if (e.set_bnorm) ks.bnorm[s] = beta;
    }
    for (int i = 1 + lane; i <= KMAX; i += 32) ks.g[so + i] = make_double2(0.0, 0.0);
    return;
  }
  if (e.kind == EPI_DOTS) {
    for (int i = lane; i < e.nv; i += 32) {
      const double sc = ks.scale[so + i];
      double2 h = make_double2(sums[2 * i] * sc, sums[2 * i + 1] * sc);
      if (e.accumulate) {
        const double2 o = ks.hcol[so + i];
        h = make_double2(o.x + h.x, o.y + h.y);
      }
      ks.hcol[so + i] = h;
      ((cplx<R>*)ks.coef)[so + i] = mkc((R)(h.x * sc), (R)(h.y * sc));
    }
    return;
  }
  // EPI_ARNOLDI: new column hcol[0..j], h_{j+1,j} = sqrt(sum)
  const int j = e.j;
  const double hn = sqrt(sums[0]);
  double2* cs = ks.cs + (size_t)s * KMAX;
  double2* sn = ks.sn + (size_t)s * KMAX;
  double2* H = ks.H + (size_t)s * (KMAX + 1) * KMAX;
  double2* g = ks.g + so;
  if (lane == 0) {
    const double inv = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
    ks.scale[so + j + 1] = inv;
    ((R*)ks.scale_r)[so + j + 1] = (R)inv;
  }
  // apply the previous rotations G_i = [[c, z], [-conj(z), conj(c)]] to the
  // column: lane i holds rotation i and entry i+1; the chain itself is serial
  const double2 zero = make_double2(0.0, 0.0);
  const double2 cl = lane < j ? cs[lane] : zero;
  const double2 zl = lane < j ? sn[lane] : zero;
  const double2 hl = lane < j ? ks.hcol[so + lane + 1] : zero;
  double2 prev = ks.hcol[so];
  double2 mine = zero;
  for (int i = 0; i < j; ++i) {
    const double2 c = shfl_d2(cl, i), z = shfl_d2(zl, i), h1 = shfl_d2(hl, i), h0 = prev;
    if (lane == i)
      mine = make_double2(c.x * h0.x - c.y * h0.y + z.x * h1.x - z.y * h1.y,
                          c.x * h0.y + c.y * h0.x + z.x * h1.y + z.y * h1.x);
    prev = make_double2(-(z.x * h0.x + z.y * h0.y) + (c.x * h1.x + c.y * h1.y),
                        -(z.x * h0.y - z.y * h0.x) + (c.x * h1.y - c.y * h1.x));
  }
  if (lane < j) H[lane * KMAX + j] = mine;
  if (lane == 0) {
    // new rotation mapping (prev, hn) to (rho, 0)
    const double rho = hypot(hypot(prev.x, prev.y), hn);
    double2 c, z;
    if (rho == 0.0 || !isfinite(rho)) {
      c = make_double2(1.0, 0.0);
      z = make_double2(0.0, 0.0);
    } else {
      c = make_double2(prev.x / rho, -prev.y / rho);
      z = make_double2(hn / rho, 0.0);
    }
    cs[j] = c;
    sn[j] = z;
    H[j * KMAX + j] = make_double2(isfinite(rho) ? rho : 0.0, 0.0);
    const double2 gj = g[j];
    g[j] = make_double2(c.x * gj.x - c.y * gj.y, c.x * gj.y + c.y * gj.x);
    g[j + 1] = make_double2(-(z.x * gj.x + z.y * gj.y), -(z.x * gj.y - z.y * gj.x));
    ks.est[s] = hypot(g[j + 1].x, g[j + 1].y);
  }
  __syncwarp();
  if (j + 1 != e.ksolve) return;
  // least-squares solution of the rotated (upper triangular) system by a
  // column sweep (lane l holds row l; the next column is loaded while the
  // current one is applied), then the coefficients of the solution update
  // x += sum y_i z_i (z_i = s_i v_i unless flexible)
  const int k = e.ksolve;
  double2 t = lane < k ? g[lane] : zero, y = zero;
  double2 hc = lane < k - 1 ? H[lane * KMAX + (k - 1)] : zero;
  double2 dc = H[(k - 1) * KMAX + (k - 1)];
  for (int i = k - 1; i >= 0; --i) {
    const double2 hnx = (i > 0 && lane < i - 1) ? H[lane * KMAX + (i - 1)] : zero;
    const double2 dnx = i > 0 ? H[(i - 1) * KMAX + (i - 1)] : zero;
    const double2 ti = shfl_d2(t, i);
    const double den = dc.x * dc.x + dc.y * dc.y;
    const double2 yi = (den > 0.0 && isfinite(den))
                           ? make_double2((ti.x * dc.x + ti.y * dc.y) / den, (ti.y * dc.x - ti.x * dc.y) / den)
                           : zero;
    if (lane < i) t = d2_fms(t, hc, yi);
    if (lane == i) y = yi;
    hc = hnx;
    dc = dnx;
  }
  if (lane < k) {
    const double sc = e.flex ? 1.0 : ks.scale[so + lane];
    ((cplx<R>*)ks.coef)[so + lane] = mkc((R)(y.x * sc), (R)(y.y * sc));
  }
}

// Called by every thread of a block after its partial row is written.
template <typename R>
__device__ __forceinline__ void epi_arrive(const Epi& e, int a, int s, int nblk, int nvals) {
  __shared__ int s_last;
  __shared__ double s_sum[2 * (KMAX + 1) > gram_nvals(SSTEP_MAX) ? 2 * (KMAX + 1) : gram_nvals(SSTEP_MAX)];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&e.counter[s], 1u) == (unsigned)(nblk - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // Fold the rows: thread t sums value k = t % nvals over the rows of group
  // t / nvals (rows b = group, group + ngroups, ...); groups are then added in
  // group order.  The order of every addition is fixed.
  __shared__ double s_grp[256];
  const int ngroups = nvals <= nthr ? min(nthr / nvals, 256 / nvals) : 1;
  const double* base = e.partial + (size_t)a * nblk * nvals;
  for (int t = tid; t < nvals * ngroups; t += nthr) {
    const int k = t % nvals, grp = t / nvals;
    double acc = 0.0;
    for (int b = grp; b < nblk; b += ngroups) acc += __ldcg(base + (size_t)b * nvals + k);
    if (ngroups > 1) s_grp[t] = acc; else s_sum[k] = acc;
  }
  __syncthreads();
  if (ngroups > 1) {
    for (int k = tid; k < nvals; k += nthr) {
      double acc = 0.0;
      for (int grp = 0; grp < ngroups; ++grp) acc += s_grp[grp * nvals + k];
      s_sum[k] = acc;
    }
    __syncthreads();
  }
  if (tid < 32) {
    if (tid == 0) e.counter[s] = 0u;
    epilogue<R>(e, s, s_sum, tid);
  }
}

}  // namespace helm
