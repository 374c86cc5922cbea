// 7-point (5-point in 2D) complex Helmholtz stencil with damping-layer
// coefficients, its adjoint, the fused residual and damped Jacobi.
//
// The operator (Sec. 2, extended-domain Helmholtz equation; Appendix A,
// eq. (dH) with A = I) is, per kernel axis d with node coefficient tables,
//
//   (H x)_p = sum_d [ cm_d(i_d) x_{p-e_d} + cd_d(i_d) x_p + cp_d(i_d) x_{p+e_d} ] + w^2 m_p x_p,
//
// zero beyond the outer walls.  The adjoint H^H has the same shape with the
// transposed, conjugated tables, so one kernel serves both directions.
//
// Layout: fields are x-fastest [Nz][Ny][Nx] per right-hand-side slot, slots
// n apart.  Thread (ix, iy) marches over a run of z-planes and keeps the
// z-1 / z / z+1 values in registers; x and y neighbours come through L1.
#include "common.cuh"

namespace helm {

namespace {

constexpr int SBX = 32;   // block extent along x (one warp: coalesced rows)
constexpr int SBY = 4;    // block extent along y
constexpr int ZRUN = 16;  // z-planes per thread

template <typename R, bool RESID>
__global__ void __launch_bounds__(SBX * SBY)
k_stencil(const cplx<R>* __restrict__ x, const R* __restrict__ xs, int xss,
          const cplx<R>* __restrict__ b, const R* __restrict__ bs, int bss,
          cplx<R>* __restrict__ y, const cplx<R>* __restrict__ tab, const R* __restrict__ m,
          const R* __restrict__ w2, const int* __restrict__ slot_f, const int* __restrict__ act,
          int K0, int K1, int K2, size_t n, int Nmax, int nzc) {
  using C = cplx<R>;
  const int ix = blockIdx.x * SBX + threadIdx.x;
  const int iy = blockIdx.y * SBY + threadIdx.y;
  const int a = blockIdx.z / nzc;
  const int zc = blockIdx.z - a * nzc;
  if (ix >= K0 || iy >= K1) return;
  const int s = act[a];
  const int f = slot_f[s];
  const C* T = tab + (size_t)f * 9 * Nmax;
  const C xm = T[ix], xd = T[Nmax + ix], xp = T[2 * Nmax + ix];
  const C ym = T[3 * Nmax + iy], yd = T[4 * Nmax + iy], yp = T[5 * Nmax + iy];
  const C* Tz = T + 6 * Nmax;
  const R om2 = w2[f];
  const R sx = xs ? xs[(size_t)s * xss] : R(1);
  R sb = R(0);
  if (RESID) sb = bs ? bs[(size_t)s * bss] : R(1);
  const C* X = x + (size_t)s * n;
  C* Y = y + (size_t)s * n;
  const C* Bv = RESID ? b + (size_t)s * n : nullptr;
  const size_t plane = (size_t)K0 * K1;
  const int z0 = zc * ZRUN;
  const int z1 = min(z0 + ZRUN, K2);
  size_t p = (size_t)ix + (size_t)K0 * iy + plane * z0;
  const C zero = mkc(R(0), R(0));
  const bool hw = ix > 0, he = ix + 1 < K0, hs = iy > 0, hn = iy + 1 < K1;
  C prev = z0 > 0 ? X[p - plane] : zero;
  C cur = X[p];
  const R dxy_re = xd.x + yd.x, dxy_im = xd.y + yd.y;
  for (int z = z0; z < z1; ++z, p += plane) {
    const C next = (z + 1 < K2) ? X[p + plane] : zero;
    const C w = hw ? X[p - 1] : zero;
    const C e = he ? X[p + 1] : zero;
    const C so = hs ? X[p - K0] : zero;
    const C no = hn ? X[p + K0] : zero;
    const C zm = Tz[z], zd = Tz[Nmax + z], zp = Tz[2 * Nmax + z];
    const C diag = mkc(dxy_re + zd.x + om2 * m[p], dxy_im + zd.y);
    C acc = cmul(diag, cur);
    acc = cfma(xm, w, acc);
    acc = cfma(xp, e, acc);
    acc = cfma(ym, so, acc);
    acc = cfma(yp, no, acc);
    acc = cfma(zm, prev, acc);
    acc = cfma(zp, next, acc);
    C out;
    if (RESID) {
      const C bv = Bv ? Bv[p] : zero;
      out = mkc(sb * bv.x - sx * acc.x, sb * bv.y - sx * acc.y);
    } else {
      out = mkc(sx * acc.x, sx * acc.y);
    }
    Y[p] = out;
    prev = cur;
    cur = next;
  }
}

// Diagonal of H at p: sum of the three cd tables and w^2 m.
template <typename R>
__device__ __forceinline__ cplx<R> diag_at(const cplx<R>* T, int Nmax, int ix, int iy, int iz, R om2, R mp) {
  const cplx<R> a = T[Nmax + ix], b = T[4 * Nmax + iy], c = T[7 * Nmax + iz];
  return mkc(a.x + b.x + c.x + om2 * mp, a.y + b.y + c.y);
}

template <typename R>
__device__ __forceinline__ cplx<R> cdiv(cplx<R> a, cplx<R> d) {
  const R den = d.x * d.x + d.y * d.y;
  const R inv = R(1) / den;
  return mkc((a.x * d.x + a.y * d.y) * inv, (a.y * d.x - a.x * d.y) * inv);
}

// z = omega D^{-1} (bs * b): the first damped-Jacobi sweep from a zero guess.
template <typename R>
__global__ void k_jacobi_first(const cplx<R>* __restrict__ b, const R* __restrict__ bs, int bss,
                               cplx<R>* __restrict__ z, const cplx<R>* __restrict__ tab,
                               const R* __restrict__ m, const R* __restrict__ w2,
                               const int* __restrict__ slot_f, const int* __restrict__ act, int K0,
                               int K1, int K2, size_t n, int Nmax, R omega) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = act[blockIdx.y];
  const int f = slot_f[s];
  const int ix = (int)(i % K0);
  const int iy = (int)((i / K0) % K1);
  const int iz = (int)(i / ((size_t)K0 * K1));
  const cplx<R>* T = tab + (size_t)f * 9 * Nmax;
  const cplx<R> d = diag_at<R>(T, Nmax, ix, iy, iz, w2[f], m[i]);
  const R sb = bs ? bs[(size_t)s * bss] : R(1);
  const cplx<R> bv = b[(size_t)s * n + i];
  const cplx<R> q = cdiv<R>(mkc(omega * sb * bv.x, omega * sb * bv.y), d);
  z[(size_t)s * n + i] = q;
}

// z += omega D^{-1} r
template <typename R>
__global__ void k_jacobi_update(const cplx<R>* __restrict__ r, cplx<R>* __restrict__ z,
                                const cplx<R>* __restrict__ tab, const R* __restrict__ m,
                                const R* __restrict__ w2, const int* __restrict__ slot_f,
                                const int* __restrict__ act, int K0, int K1, int K2, size_t n,
                                int Nmax, R omega) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = act[blockIdx.y];
  const int f = slot_f[s];
  const int ix = (int)(i % K0);
  const int iy = (int)((i / K0) % K1);
  const int iz = (int)(i / ((size_t)K0 * K1));
  const cplx<R>* T = tab + (size_t)f * 9 * Nmax;
  const cplx<R> d = diag_at<R>(T, Nmax, ix, iy, iz, w2[f], m[i]);
  const cplx<R> rv = r[(size_t)s * n + i];
  const cplx<R> q = cdiv<R>(mkc(omega * rv.x, omega * rv.y), d);
  cplx<R> zv = z[(size_t)s * n + i];
  z[(size_t)s * n + i] = mkc(zv.x + q.x, zv.y + q.y);
}

}  // namespace

template <typename R>
void launch_stencil(const OpView<R>& op, const int* slot_f, const int* act, int na,
                    const cplx<R>* x, Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y,
                    cudaStream_t st) {
  if (na <= 0) return;
  const double by = (double)na * op.n * ((b || bs.p) ? 3 : 2) * sizeof(cplx<R>) + (double)op.n * sizeof(R);
  ProfScope ps(sizeof(R) == 4 ? PC_STENCIL32 : PC_STENCIL64, by, st);
  const int nzc = (op.K[2] + ZRUN - 1) / ZRUN;
  dim3 blk(SBX, SBY);
  dim3 grd((op.K[0] + SBX - 1) / SBX, (op.K[1] + SBY - 1) / SBY, nzc * na);
  if (b || bs.p) {
    k_stencil<R, true><<<grd, blk, 0, st>>>(x, xs.p, xs.stride, b, bs.p, bs.stride, y, op.tab, op.m,
                                            op.w2, slot_f, act, op.K[0], op.K[1], op.K[2], op.n,
                                            op.Nmax, nzc);
  } else {
    k_stencil<R, false><<<grd, blk, 0, st>>>(x, xs.p, xs.stride, nullptr, nullptr, 0, y, op.tab, op.m,
                                             op.w2, slot_f, act, op.K[0], op.K[1], op.K[2], op.n,
                                             op.Nmax, nzc);
  }
  count_launch();
}

template <typename R>
void launch_jacobi_first(const OpView<R>& op, const int* slot_f, const int* act, int na,
                         const cplx<R>* b, Scale<R> bs, R omega, cplx<R>* z, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * op.n * 2 * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((op.n + 255) / 256), na);
  k_jacobi_first<R><<<grd, 256, 0, st>>>(b, bs.p, bs.stride, z, op.tab, op.m, op.w2, slot_f, act,
                                         op.K[0], op.K[1], op.K[2], op.n, op.Nmax, omega);
  count_launch();
}

template <typename R>
void launch_jacobi_update(const OpView<R>& op, const int* slot_f, const int* act, int na,
                          const cplx<R>* r, R omega, cplx<R>* z, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * op.n * 3 * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((op.n + 255) / 256), na);
  k_jacobi_update<R><<<grd, 256, 0, st>>>(r, z, op.tab, op.m, op.w2, slot_f, act, op.K[0], op.K[1],
                                          op.K[2], op.n, op.Nmax, omega);
  count_launch();
}

#define INST(R)                                                                                      \
  template void launch_stencil<R>(const OpView<R>&, const int*, const int*, int, const cplx<R>*,     \
                                  Scale<R>, const cplx<R>*, Scale<R>, cplx<R>*, cudaStream_t);       \
  template void launch_jacobi_first<R>(const OpView<R>&, const int*, const int*, int,               \
                                       const cplx<R>*, Scale<R>, R, cplx<R>*, cudaStream_t);        \
  template void launch_jacobi_update<R>(const OpView<R>&, const int*, const int*, int,              \
                                        const cplx<R>*, R, cplx<R>*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace helm
