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
};

__device__ __forceinline__ int epi_nvals(const Epi& e) { return e.kind == EPI_DOTS ? 2 * e.nv : 1; }

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

template <typename R>
__device__ __noinline__ void epilogue(const Epi& e, int s, const double* sums) {
  const KState& ks = e.ks;
  const size_t so = (size_t)s * (KMAX + 1);
  if (e.kind == EPI_NORM) {
    e.out[s] = sqrt(sums[0]);
    return;
  }
  if (e.kind == EPI_GRAM) {
    // s-step minimal-residual update.  The basis is W_0 = r0, W_{i+1} = H W_i
    // (unnormalised; the diagonal scaling below takes care of magnitudes).
    // Minimise ||r0 - sum_i y_i W_{i+1}|| through the normal equations
    // G y = c, G_ij = <W_{i+1}, W_{j+1}>, c_i = <W_{i+1}, r0>, scaled to unit
    // diagonal and solved by a Cholesky factorisation that drops directions
    // with a negligible pivot; then x += sum_i y_i W_i.
    const int S = e.idx;
    double2 G[SSTEP_MAX][SSTEP_MAX];
    double2 c[SSTEP_MAX];
    double sg[SSTEP_MAX];
    int k = 0;
    for (int i = 0; i < S; ++i)
      for (int j = i; j < S; ++j, ++k) {
        G[i][j] = make_double2(sums[2 * k], sums[2 * k + 1]);
        G[j][i] = make_double2(sums[2 * k], -sums[2 * k + 1]);
      }
    for (int i = 0; i < S; ++i, ++k) c[i] = make_double2(sums[2 * k], sums[2 * k + 1]);
    const double r0sq = sums[2 * k];
    ks.rnorm[s] = sqrt(r0sq);
    for (int i = 0; i < S; ++i) {
      const double d = G[i][i].x;
      sg[i] = (d > 0.0 && isfinite(d)) ? 1.0 / sqrt(d) : 0.0;
    }
    for (int i = 0; i < S; ++i) {
      for (int j = 0; j < S; ++j) G[i][j] = make_double2(G[i][j].x * sg[i] * sg[j], G[i][j].y * sg[i] * sg[j]);
      c[i] = make_double2(c[i].x * sg[i], c[i].y * sg[i]);
    }
    // in-place Cholesky G = L L^H (lower triangle), forward and back substitution
    bool live[SSTEP_MAX];
    for (int j = 0; j < S; ++j) {
      double d = G[j][j].x;
      for (int l = 0; l < j; ++l)
        if (live[l]) d -= G[j][l].x * G[j][l].x + G[j][l].y * G[j][l].y;
      live[j] = d > (sizeof(R) == 4 ? 1e-6 : 1e-12) && isfinite(d);
      const double r = live[j] ? sqrt(d) : 0.0;
      G[j][j] = make_double2(r, 0.0);
      for (int i = j + 1; i < S; ++i) {
        double2 t = G[i][j];
        for (int l = 0; l < j; ++l) {
          if (!live[l]) continue;
          const double2 a = G[i][l], b = G[j][l];  // t -= a * conj(b)
          t.x -= a.x * b.x + a.y * b.y;
          t.y -= a.y * b.x - a.x * b.y;
        }
        G[i][j] = live[j] ? make_double2(t.x / r, t.y / r) : make_double2(0.0, 0.0);
      }
    }
    double2 w[SSTEP_MAX], z[SSTEP_MAX];
    for (int i = 0; i < S; ++i) {  // L w = c
      double2 t = c[i];
      for (int l = 0; l < i; ++l) {
        const double2 a = G[i][l];
        t.x -= a.x * w[l].x - a.y * w[l].y;
        t.y -= a.x * w[l].y + a.y * w[l].x;
      }
      w[i] = live[i] ? make_double2(t.x / G[i][i].x, t.y / G[i][i].x) : make_double2(0.0, 0.0);
    }
    for (int i = S - 1; i >= 0; --i) {  // L^H z = w
      double2 t = w[i];
      for (int l = i + 1; l < S; ++l) {
        const double2 a = G[l][i];  // (L^H)_{il} = conj(L_li)
        t.x -= a.x * z[l].x + a.y * z[l].y;
        t.y -= a.x * z[l].y - a.y * z[l].x;
      }
      z[i] = live[i] ? make_double2(t.x / G[i][i].x, t.y / G[i][i].x) : make_double2(0.0, 0.0);
    }
    double red = 0.0;
    for (int i = 0; i < S; ++i) red += c[i].x * z[i].x + c[i].y * z[i].y;  // Re(c^H z) in scaled variables
    ks.est[s] = sqrt(fmax(0.0, r0sq - red));
    // y_i = sg_i z_i multiplies W_i in the update
    cplx<R>* cf = (cplx<R>*)ks.coef + so;
    for (int i = 0; i < S; ++i) cf[i] = mkc((R)(z[i].x * sg[i]), (R)(z[i].y * sg[i]));
    return;
  }
  if (e.kind == EPI_START) {
    const double beta = sqrt(sums[0]);
    const double inv = (beta > 0.0 && isfinite(beta)) ? 1.0 / beta : 0.0;
    ks.scale[so] = inv;
    ((R*)ks.scale_r)[so] = (R)inv;
    ks.g[so] = make_double2(beta, 0.0);
    for (int i = 1; i <= KMAX; ++i) ks.g[so + i] = make_double2(0.0, 0.0);
    ks.rnorm[s] = beta;
    ks.est[s] = beta;
    if (e.set_bnorm) ks.bnorm[s] = beta;
    return;
  }
  if (e.kind == EPI_DOTS) {
    for (int i = 0; i < e.nv; ++i) {
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
  const double inv = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
  ks.scale[so + j + 1] = inv;
  ((R*)ks.scale_r)[so + j + 1] = (R)inv;
  double2* cs = ks.cs + (size_t)s * KMAX;
  double2* sn = ks.sn + (size_t)s * KMAX;
  double2* H = ks.H + (size_t)s * (KMAX + 1) * KMAX;
  double2* g = ks.g + so;
  double2 prev = ks.hcol[so];
  // apply the previous rotations G_i = [[c, z], [-conj(z), conj(c)]] while streaming the column
  for (int i = 0; i < j; ++i) {
    const double2 c = cs[i], z = sn[i], h0 = prev, h1 = ks.hcol[so + i + 1];
    H[i * KMAX + j] = make_double2(c.x * h0.x - c.y * h0.y + z.x * h1.x - z.y * h1.y,
                                   c.x * h0.y + c.y * h0.x + z.x * h1.y + z.y * h1.x);
    prev = make_double2(-(z.x * h0.x + z.y * h0.y) + (c.x * h1.x + c.y * h1.y),
                        -(z.x * h0.y - z.y * h0.x) + (c.x * h1.y - c.y * h1.x));
  }
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
  if (j + 1 != e.ksolve) return;
  // least-squares solution of the rotated (upper triangular) system, then the
  // coefficients of the solution update x += sum y_i z_i (z_i = s_i v_i unless flexible)
  const int k = e.ksolve;
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
    y[i] = (den > 0.0 && isfinite(den)) ? make_double2((t.x * d.x + t.y * d.y) / den, (t.y * d.x - t.x * d.y) / den)
                                        : make_double2(0.0, 0.0);
  }
  cplx<R>* cf = (cplx<R>*)ks.coef + so;
  for (int i = 0; i < k; ++i) {
    const double sc = e.flex ? 1.0 : ks.scale[so + i];
    cf[i] = mkc((R)(y[i].x * sc), (R)(y[i].y * sc));
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
  if (tid == 0) {
    e.counter[s] = 0u;
    epilogue<R>(e, s, s_sum);
  }
}

}  // namespace helm
