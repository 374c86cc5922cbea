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
// n apart.  A tile is a run of consecutive (x, y) columns of a plane
// (flattened, so no lanes idle at ragged row ends) by a run of z-planes; each
// thread marches its column in z, keeps the z-1 / z / z+1 values in registers
// and issues the loads of the next plane before computing the current one; x
// and y neighbours come through L1.  The plain apply has several tile shapes
// and picks one per grid by timing them on first use (or takes the one
// helm_stencil_select forces).  The reducing apply loops its blocks over tiles
// so the number of blocks per slot is bounded, which lets the kernel also
// reduce its output: dot products with Krylov basis vectors (the first
// Gram-Schmidt pass of an Arnoldi step) or the norm of a residual
// (reduce.cuh).
#include <array>
#include <map>
#include <mutex>

#include "reduce.cuh"
#include "tma.cuh"

namespace helm {

namespace {

constexpr int STPB = 128;  // threads per block = consecutive (x, y) columns of a plane
constexpr int ZRUN = 16;   // z-planes per tile

struct TileGeom {
  int K0, K1, K2;
  int nseg, nzc, ntiles;  // plane segments of STPB columns, z-chunks, tiles per slot
  size_t n;
  int Nmax;
};

// Plain apply (no reduction): one tile of TPB consecutive (x, y) columns by
// ZR planes per block, on a 1D grid whose block index runs over the active
// slots fastest, so the blocks that share a tile of m (and of the damping
// tables) run back to back and m is fetched from HBM about once per launch
// rather than once per slot.  The tile's z coefficients sit in shared memory
// and, in single precision, the z march is fully unrolled (no register
// rotation between planes).  With PF > 0 (x 16-byte aligned) thread 0
// bulk-prefetches into L2, one plane at a time, the tile's window of x PF
// planes ahead of the march: the bytes in flight no longer depend on
// registers.  TPB, ZR and MINB (blocks per SM the register budget is sized
// for) are the variants the launch-time tuner chooses between.
template <typename R, bool RESID, int PF, int TPB, int ZR, int MINB>
__global__ void __launch_bounds__(TPB, MINB)
k_stencil_plain(const cplx<R>* __restrict__ x, const R* __restrict__ xs, int xss, const cplx<R>* __restrict__ b,
                const R* __restrict__ bs, int bss, cplx<R>* __restrict__ y, const cplx<R>* __restrict__ tab,
                const R* __restrict__ m, const R* __restrict__ w2, const int* __restrict__ slot_f,
                const int* __restrict__ act, int na, TileGeom G) {
  using C = cplx<R>;
  __shared__ C stz[3][ZR];
  const int planei = G.K0 * G.K1;
  const int a = (int)(blockIdx.x % (unsigned)na);
  const int tile = (int)(blockIdx.x / (unsigned)na);
  const int seg = tile % G.nseg;
  const int zc = tile / G.nseg;
  const int p2 = seg * TPB + threadIdx.x;
  const int s = act[a];
  const int f = slot_f[s];
  const C* T = tab + (size_t)f * 9 * G.Nmax;
  const C* Tz = T + 6 * G.Nmax;
  const int z0 = zc * ZR;
  const int z1 = min(z0 + ZR, G.K2);
  for (int i = threadIdx.x; i < 3 * ZR; i += TPB) {
    const int k = i / ZR, zz = i % ZR;
    stz[k][zz] = z0 + zz < G.K2 ? Tz[k * G.Nmax + z0 + zz] : mkc(R(0), R(0));
  }
  __syncthreads();
  if (p2 >= planei) return;
  const R om2 = w2[f];
  const C* X = x + (size_t)s * G.n;
  C* Y = y + (size_t)s * G.n;
  const int ix = p2 % G.K0;
  const int iy = p2 / G.K0;
  const C xm = T[ix], xd = T[G.Nmax + ix], xp = T[2 * G.Nmax + ix];
  const C ym = T[3 * G.Nmax + iy], yd = T[4 * G.Nmax + iy], yp = T[5 * G.Nmax + iy];
  const R dre = xd.x + yd.x, dim = xd.y + yd.y;
  // pointer stepping: xq/yq/mq address plane z of this column; neighbours are
  // fixed offsets from xq
  const int P = planei;
  const int K0 = G.K0;
  const size_t p0 = (size_t)p2 + (size_t)P * z0;
  const C* xq = X + p0;
  C* yq = Y + p0;
  const R* mq = m + p0;
  const C* bq = RESID ? b + (size_t)s * G.n + p0 : nullptr;
  const R sx = xs ? xs[(size_t)s * xss] : R(1);
  const R sb = (RESID && bs) ? bs[(size_t)s * bss] : R(1);
  const C zero = mkc(R(0), R(0));
  const bool hw = ix > 0, he = ix + 1 < K0, hs = iy > 0, hn = iy + 1 < G.K1;
  C prev = z0 > 0 ? xq[-P] : zero;
  C cur = xq[0];
  C next = (z0 + 1 < G.K2) ? xq[P] : zero;
  C w = hw ? xq[-1] : zero, ea = he ? xq[1] : zero, so = hs ? xq[-K0] : zero, no = hn ? xq[K0] : zero;
  R mm = mq[0];
#pragma unroll(sizeof(R) == 4 ? ZR : 1)
  for (int zz = 0; zz < ZR; ++zz) {
    const int z = z0 + zz;
    if (z >= z1) break;
    const C* xn = xq + P;  // plane z+1
    C next2 = zero, w2n = zero, e2n = zero, s2n = zero, n2n = zero;
    R m2 = R(0);
    if (z + 1 < z1) {
      next2 = (z + 2 < G.K2) ? xn[P] : zero;
      w2n = hw ? xn[-1] : zero;
      e2n = he ? xn[1] : zero;
      s2n = hs ? xn[-K0] : zero;
      n2n = hn ? xn[K0] : zero;
      m2 = mq[P];
    }
    if (PF > 0 && threadIdx.x == 0 && z + PF < G.K2) {
      // plane z+PF, columns [seg*TPB - K0, seg*TPB + TPB + K0) clipped to the plane, rounded out
      // to 16-byte bounds without leaving this slot's field (the element before an odd-aligned
      // field start belongs to the previous slot, or the start is even)
      const size_t fb = (size_t)s * G.n, pz = fb + (size_t)(z + PF) * P;
      const size_t lo = pz + (size_t)max(0, seg * TPB - K0);
      const size_t hi = pz + (size_t)min(P, seg * TPB + TPB + K0);
      const size_t a0 = lo & ~(size_t)1;
      size_t a1 = (hi + 1) & ~(size_t)1;
      if (a1 > fb + G.n) a1 -= 2;
      if (a1 > a0) bulk_prefetch_l2(x + a0, (uint32_t)((a1 - a0) * sizeof(C)));
    }
    const C zm = stz[0][zz], zd = stz[1][zz], zp = stz[2][zz];
    const C diag = mkc(dre + zd.x + om2 * mm, dim + zd.y);
    C h = cmul(diag, cur);
    h = cfma(xm, w, h);
    h = cfma(xp, ea, h);
    h = cfma(ym, so, h);
    h = cfma(yp, no, h);
    h = cfma(zm, prev, h);
    h = cfma(zp, next, h);
    if (RESID) {
      const C bv = bq[0];
      yq[0] = mkc(sb * bv.x - sx * h.x, sb * bv.y - sx * h.y);
      bq += P;
    } else {
      yq[0] = mkc(sx * h.x, sx * h.y);
    }
    xq = xn;
    yq += P;
    mq += P;
    prev = cur;
    cur = next;
    next = next2;
    w = w2n;
    ea = e2n;
    so = s2n;
    no = n2n;
    mm = m2;
  }
}

// RED: 0 no reduction, -1 norm of the output, KM > 0 dots of the output with up to KM basis vectors
template <typename R, bool RESID, int RED>
__global__ void __launch_bounds__(STPB)
k_stencil(const cplx<R>* __restrict__ x, const R* __restrict__ xs, int xss, const cplx<R>* __restrict__ b,
          const R* __restrict__ bs, int bss, cplx<R>* __restrict__ y, const cplx<R>* __restrict__ tab,
          const R* __restrict__ m, const R* __restrict__ w2, const int* __restrict__ slot_f,
          const int* __restrict__ act, int na, TileGeom G, const cplx<R>* __restrict__ V, size_t vstride, int nv,
          Epi e) {
  using C = cplx<R>;
  constexpr int KM = RED > 0 ? RED : 1;
  constexpr int NVAL = RED > 0 ? 2 * RED : 1;
  // 1D grid, slots fastest: block j of every slot works on the same tiles at the same time, so the
  // tiles of m are shared through L2; nb blocks per slot, each with its own partial row
  const int a = (int)(blockIdx.x % (unsigned)na);
  const int jb = (int)(blockIdx.x / (unsigned)na);
  const int nb = (int)(gridDim.x / (unsigned)na);
  const int s = act[a];
  const int f = slot_f[s];
  const C* T = tab + (size_t)f * 9 * G.Nmax;
  const C* Tz = T + 6 * G.Nmax;
  const R om2 = w2[f];
  const R sx = xs ? xs[(size_t)s * xss] : R(1);
  const R sb = (RESID && bs) ? bs[(size_t)s * bss] : R(1);
  const C* X = x + (size_t)s * G.n;
  C* Y = y + (size_t)s * G.n;
  const C* Bv = RESID ? b + (size_t)s * G.n : nullptr;
  const C* Vs = RED > 0 ? V + (size_t)s * G.n : nullptr;
  const size_t plane = (size_t)G.K0 * G.K1;
  const C zero = mkc(R(0), R(0));
  R acc[NVAL];
#pragma unroll
  for (int k = 0; k < NVAL; ++k) acc[k] = R(0);
  const int planei = G.K0 * G.K1;
  for (int tile = jb; tile < G.ntiles; tile += nb) {
    const int seg = tile % G.nseg;
    const int zc = tile / G.nseg;
    const int p2 = seg * STPB + threadIdx.x;
    if (p2 >= planei) continue;
    const int ix = p2 % G.K0;
    const int iy = p2 / G.K0;
    const C xm = T[ix], xd = T[G.Nmax + ix], xp = T[2 * G.Nmax + ix];
    const C ym = T[3 * G.Nmax + iy], yd = T[4 * G.Nmax + iy], yp = T[5 * G.Nmax + iy];
    const R dxy_re = xd.x + yd.x, dxy_im = xd.y + yd.y;
    const int z0 = zc * ZRUN;
    const int z1 = min(z0 + ZRUN, G.K2);
    const bool hw = ix > 0, he = ix + 1 < G.K0, hs = iy > 0, hn = iy + 1 < G.K1;
    size_t p = (size_t)p2 + plane * z0;
    // register pipeline: the loads of plane z+1 are issued before plane z is computed
    C prev = z0 > 0 ? X[p - plane] : zero;
    C cur = X[p];
    C next = (z0 + 1 < G.K2) ? X[p + plane] : zero;
    C w = hw ? X[p - 1] : zero, ea = he ? X[p + 1] : zero;
    C so = hs ? X[p - G.K0] : zero, no = hn ? X[p + G.K0] : zero;
    R mm = m[p];
    for (int z = z0; z < z1; ++z, p += plane) {
      const size_t q = p + plane;
      const bool more = z + 1 < z1;
      C next2 = zero, w2n = zero, e2n = zero, s2n = zero, n2n = zero;
      R m2 = R(0);
      if (more) {
        next2 = (z + 2 < G.K2) ? X[q + plane] : zero;
        w2n = hw ? X[q - 1] : zero;
        e2n = he ? X[q + 1] : zero;
        s2n = hs ? X[q - G.K0] : zero;
        n2n = hn ? X[q + G.K0] : zero;
        m2 = m[q];
      }
      const C zm = Tz[z], zd = Tz[G.Nmax + z], zp = Tz[2 * G.Nmax + z];
      const C diag = mkc(dxy_re + zd.x + om2 * mm, dxy_im + zd.y);
      C h = cmul(diag, cur);
      h = cfma(xm, w, h);
      h = cfma(xp, ea, h);
      h = cfma(ym, so, h);
      h = cfma(yp, no, h);
      h = cfma(zm, prev, h);
      h = cfma(zp, next, h);
      C out;
      if (RESID) {
        const C bv = Bv[p];
        out = mkc(sb * bv.x - sx * h.x, sb * bv.y - sx * h.y);
      } else {
        out = mkc(sx * h.x, sx * h.y);
      }
      Y[p] = out;
      if (RED < 0) acc[0] = fma(out.x, out.x, fma(out.y, out.y, acc[0]));
      if (RED > 0) {
#pragma unroll
        for (int i = 0; i < KM; ++i) {
          if (i < nv) {
            const C v = Vs[i * vstride + p];
            acc[2 * i] = fma(v.x, out.x, fma(v.y, out.y, acc[2 * i]));
            acc[2 * i + 1] = fma(v.x, out.y, fma(-v.y, out.x, acc[2 * i + 1]));
          }
        }
      }
      prev = cur;
      cur = next;
      next = next2;
      w = w2n;
      ea = e2n;
      so = s2n;
      no = n2n;
      mm = m2;
    }
  }
  if (RED == 0) return;
  const int nvals = RED > 0 ? 2 * nv : 1;
  block_partial_row<R, NVAL, STPB / 32>(acc, nvals, e.partial + ((size_t)a * nb + jb) * nvals);
  epi_arrive<R>(e, a, s, nb, nvals);
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
                               cplx<R>* __restrict__ z, const cplx<R>* __restrict__ tab, const R* __restrict__ m,
                               const R* __restrict__ w2, const int* __restrict__ slot_f,
                               const int* __restrict__ act, int K0, int K1, int K2, size_t n, int Nmax, R omega) {
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
  z[(size_t)s * n + i] = cdiv<R>(mkc(omega * sb * bv.x, omega * sb * bv.y), d);
}

// z += omega D^{-1} r
template <typename R>
__global__ void k_jacobi_update(const cplx<R>* __restrict__ r, cplx<R>* __restrict__ z,
                                const cplx<R>* __restrict__ tab, const R* __restrict__ m, const R* __restrict__ w2,
                                const int* __restrict__ slot_f, const int* __restrict__ act, int K0, int K1, int K2,
                                size_t n, int Nmax, R omega) {
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
  const cplx<R> zv = z[(size_t)s * n + i];
  z[(size_t)s * n + i] = mkc(zv.x + q.x, zv.y + q.y);
}

template <typename R, bool RESID, int RED>
void stencil_go(dim3 grd, cudaStream_t st, const OpView<R>& op, const int* slot_f, const int* act,
                const cplx<R>* x, Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y, const TileGeom& G,
                const cplx<R>* V, size_t vstride, int nv, const Epi& e) {
  // grd = (blocks per slot, slots): launched as one dimension with the slots fastest
  k_stencil<R, RESID, RED><<<grd.x * grd.y, STPB, 0, st>>>(x, xs.p, xs.stride, b, bs.p, bs.stride, y, op.tab, op.m,
                                                            op.w2, slot_f, act, (int)grd.y, G, V, vstride, nv, e);
}

template <typename R, bool RESID>
void stencil_red(dim3 grd, cudaStream_t st, const OpView<R>& op, const int* slot_f, const int* act,
                 const cplx<R>* x, Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y, const TileGeom& G,
                 const cplx<R>* V, size_t vstride, int nv, const Epi& e) {
  if (e.kind == EPI_NONE)
    stencil_go<R, RESID, 0>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  else if (e.kind != EPI_DOTS)
    stencil_go<R, RESID, -1>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  else if (nv <= 4)
    stencil_go<R, RESID, 4>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  else if (nv <= 8)
    stencil_go<R, RESID, 8>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  else if (nv <= 16)
    stencil_go<R, RESID, 16>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  else
    stencil_go<R, RESID, KMAX + 1>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
}

// Shapes of the plain apply the tuner chooses between: threads per block
// (consecutive columns of a plane), z-planes per tile, blocks per SM the
// register budget is sized for.
struct PlainShape {
  int tpb, zr, minb;
};
constexpr PlainShape kPlain[] = {{128, 16, 6}, {128, 16, 8}, {128, 32, 6}, {256, 16, 3},
                                 {128, 8, 8},  {256, 8, 4},  {128, 32, 8}, {64, 32, 16}};
constexpr int kNumPlain = (int)(sizeof(kPlain) / sizeof(kPlain[0]));

std::atomic<int> g_plain_forced{-1};  // >= 0: every plain apply uses this shape
std::mutex g_tune_mu;
struct TuneRec {
  int variant;
  float us;
};
std::map<std::array<int, 5>, TuneRec> g_plain_choice;  // (K0, K1, K2, residual, prefetch) -> choice

template <typename R, bool RESID, int PF, int TPB, int ZR, int MINB>
void plain_go(cudaStream_t st, const OpView<R>& op, const int* slot_f, const int* act, int na, const cplx<R>* x,
              Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y) {
  TileGeom G;
  G.K0 = op.K[0];
  G.K1 = op.K[1];
  G.K2 = op.K[2];
  G.nseg = (int)(((size_t)G.K0 * G.K1 + TPB - 1) / TPB);
  G.nzc = (G.K2 + ZR - 1) / ZR;
  G.ntiles = G.nseg * G.nzc;
  G.n = op.n;
  G.Nmax = op.Nmax;
  const unsigned nblk = (unsigned)G.ntiles * (unsigned)na;
  k_stencil_plain<R, RESID, PF, TPB, ZR, MINB><<<nblk, TPB, 0, st>>>(x, xs.p, xs.stride, b, bs.p, bs.stride, y, op.tab,
                                                                      op.m, op.w2, slot_f, act, na, G);
  count_launch();
}

template <typename R, bool RESID, int PF>
void plain_variant(int v, cudaStream_t st, const OpView<R>& op, const int* slot_f, const int* act, int na,
                   const cplx<R>* x, Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y) {
  if (sizeof(R) == 8) v = 0;  // the FP64 apply is bound by the FP64 pipe: one shape
  switch (v) {
    case 1: plain_go<R, RESID, PF, 128, 16, 8>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    case 2: plain_go<R, RESID, PF, 128, 32, 6>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    case 3: plain_go<R, RESID, PF, 256, 16, 3>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    case 4: plain_go<R, RESID, PF, 128, 8, 8>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    case 5: plain_go<R, RESID, PF, 256, 8, 4>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    case 6: plain_go<R, RESID, PF, 128, 32, 8>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    case 7: plain_go<R, RESID, PF, 64, 32, 16>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
    default: plain_go<R, RESID, PF, 128, 16, 6>(st, op, slot_f, act, na, x, xs, b, bs, y); break;
  }
}

// The shape for this grid: the forced one, else the tuned one, tuning on first
// use.  Tuning launches every shape on the call's own fields (each launch
// writes the same y: every shape computes every point with the same
// arithmetic, so the results are bitwise identical) and keeps the fastest of
// three timed launches per shape; it synchronises the stream once per grid.
template <typename R, bool RESID, int PF>
int plain_choose(cudaStream_t st, const OpView<R>& op, const int* slot_f, const int* act, int na, const cplx<R>* x,
                 Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y, bool may_tune) {
  const int forced = g_plain_forced.load();
  if (forced >= 0) return forced;
  if (sizeof(R) == 8 || op.n < PROF_COARSE_N) return 0;  // FP64, or grids that sit in L2: no tuning
  const std::array<int, 5> key{op.K[0], op.K[1], op.K[2], RESID ? 1 : 0, PF};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_plain_choice.find(key);
  if (it != g_plain_choice.end()) return it->second.variant;
  if (!may_tune) return 0;  // the caller may not create the timing events: the first shape
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return 0;
  }
  int best = 0;
  float best_ms = 1e30f;
  for (int v = 0; v < kNumPlain; ++v) {
    plain_variant<R, RESID, PF>(v, st, op, slot_f, act, na, x, xs, b, bs, y);  // warm
    float tmin = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, st);
      plain_variant<R, RESID, PF>(v, st, op, slot_f, act, na, x, xs, b, bs, y);
      cudaEventRecord(e1, st);
      float ms = 1e30f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        tmin = std::min(tmin, ms);
    }
    if (tmin < best_ms) {
      best_ms = tmin;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_plain_choice[key] = TuneRec{best, 1e3f * best_ms};
  return best;
}

}  // namespace

template <typename R>
void launch_stencil(const OpView<R>& op, const int* slot_f, const int* act, int na, const cplx<R>* x,
                    Scale<R> xs, const cplx<R>* b, Scale<R> bs, cplx<R>* y, cudaStream_t st, const Epi* epi,
                    const cplx<R>* V, size_t vstride, int nv, bool may_tune) {
  if (na <= 0) return;
  Epi e = epi ? *epi : Epi{};
  double by = (double)na * op.n * (b ? 3 : 2) * sizeof(cplx<R>) + (double)op.n * sizeof(R);
  if (e.kind == EPI_DOTS) by += (double)na * op.n * nv * sizeof(cplx<R>);
  if (e.kind == EPI_NONE) {
    // L2 prefetch 4 planes ahead: single precision (the FP64 stencil is ALU-bound), 16-byte aligned x,
    // grids that do not sit in L2 anyway.  The shape is chosen (tuned on first use) outside the timed scope.
    const bool pf = sizeof(R) == 4 && ((uintptr_t)x & 15) == 0 && op.n >= PROF_COARSE_N;
    int v;
    if (b && pf) v = plain_choose<R, true, 4>(st, op, slot_f, act, na, x, xs, b, bs, y, may_tune);
    else if (b) v = plain_choose<R, true, 0>(st, op, slot_f, act, na, x, xs, b, bs, y, may_tune);
    else if (pf) v = plain_choose<R, false, 4>(st, op, slot_f, act, na, x, xs, b, bs, y, may_tune);
    else v = plain_choose<R, false, 0>(st, op, slot_f, act, na, x, xs, b, bs, y, may_tune);
    ProfScope ps(prof_stencil_class<R>(op.n), by, st);
    if (b && pf) plain_variant<R, true, 4>(v, st, op, slot_f, act, na, x, xs, b, bs, y);
    else if (b) plain_variant<R, true, 0>(v, st, op, slot_f, act, na, x, xs, b, bs, y);
    else if (pf) plain_variant<R, false, 4>(v, st, op, slot_f, act, na, x, xs, b, bs, y);
    else plain_variant<R, false, 0>(v, st, op, slot_f, act, na, x, xs, b, bs, y);
    return;
  }
  ProfScope ps(prof_stencil_class<R>(op.n), by, st);
  TileGeom G;
  G.K0 = op.K[0];
  G.K1 = op.K[1];
  G.K2 = op.K[2];
  G.nseg = (int)(((size_t)G.K0 * G.K1 + STPB - 1) / STPB);
  G.nzc = (G.K2 + ZRUN - 1) / ZRUN;
  G.ntiles = G.nseg * G.nzc;
  G.n = op.n;
  G.Nmax = op.Nmax;
  // bounded blocks per slot: every block reduces into one partial row
  const int target = (152 * 12 + na - 1) / na;
  int nblk = std::min(G.ntiles, std::max(1, target));
  const int rows = std::max(RED_BLOCKS_MAX, na);
  if ((long long)nblk * na > rows) nblk = std::max(1, rows / na);
  dim3 grd(nblk, na);
  if (b) {
    stencil_red<R, true>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  } else {
    stencil_red<R, false>(grd, st, op, slot_f, act, x, xs, b, bs, y, G, V, vstride, nv, e);
  }
  count_launch();
}

template <typename R>
void launch_jacobi_first(const OpView<R>& op, const int* slot_f, const int* act, int na, const cplx<R>* b,
                         Scale<R> bs, R omega, cplx<R>* z, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * op.n * 2 * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((op.n + 255) / 256), na);
  k_jacobi_first<R><<<grd, 256, 0, st>>>(b, bs.p, bs.stride, z, op.tab, op.m, op.w2, slot_f, act, op.K[0], op.K[1],
                                         op.K[2], op.n, op.Nmax, omega);
  count_launch();
}

template <typename R>
void launch_jacobi_update(const OpView<R>& op, const int* slot_f, const int* act, int na, const cplx<R>* r,
                          R omega, cplx<R>* z, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_MISC, (double)na * op.n * 3 * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((op.n + 255) / 256), na);
  k_jacobi_update<R><<<grd, 256, 0, st>>>(r, z, op.tab, op.m, op.w2, slot_f, act, op.K[0], op.K[1], op.K[2], op.n,
                                          op.Nmax, omega);
  count_launch();
}

#define INST(R)                                                                                                 \
  template void launch_stencil<R>(const OpView<R>&, const int*, const int*, int, const cplx<R>*, Scale<R>,      \
                                  const cplx<R>*, Scale<R>, cplx<R>*, cudaStream_t, const Epi*, const cplx<R>*, \
                                  size_t, int, bool);                                                           \
  template void launch_jacobi_first<R>(const OpView<R>&, const int*, const int*, int, const cplx<R>*, Scale<R>, \
                                       R, cplx<R>*, cudaStream_t);                                              \
  template void launch_jacobi_update<R>(const OpView<R>&, const int*, const int*, int, const cplx<R>*, R,        \
                                        cplx<R>*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace helm

using namespace helm;

extern "C" {

int helm_stencil_variant_count(void) { return kNumPlain; }

int helm_stencil_variant_info(int variant, int* threads, int* zplanes, int* min_blocks) {
  if (variant < 0 || variant >= kNumPlain) return HELM_E_INVAL;
  if (threads) *threads = kPlain[variant].tpb;
  if (zplanes) *zplanes = kPlain[variant].zr;
  if (min_blocks) *min_blocks = kPlain[variant].minb;
  return HELM_OK;
}

int helm_stencil_select(int variant) {
  if (variant < -1 || variant >= kNumPlain) return HELM_E_INVAL;
  g_plain_forced.store(variant);
  return HELM_OK;
}

int helm_stencil_tuned(const helm_plan* plan, int level, int residual, int* variant, double* us) {
  if (!plan || level < 0 || level >= MAX_LEVELS || !variant) return HELM_E_INVAL;
  const LevelGeom& L = plan->lev[level];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int pf : {4, 0}) {
    auto it = g_plain_choice.find(std::array<int, 5>{L.K[0], L.K[1], L.K[2], residual ? 1 : 0, pf});
    if (it != g_plain_choice.end()) {
      *variant = it->second.variant;
      if (us) *us = it->second.us;
      return HELM_OK;
    }
  }
  return HELM_E_INVAL;
}

}  // extern "C"
