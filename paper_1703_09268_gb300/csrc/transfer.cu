// Inter-grid transfers of the multigrid V-cycle (Sec. 4, Alg. vcycle):
// linear interpolation P (coarse node j sits on fine node 2j+1; even fine
// nodes average their two coarse neighbours, zero beyond the walls) and the
// full-weighting restriction R = 2^-dim P^T (1D weights 1/4, 1/2, 1/4).
// A kernel axis of size 1 (the middle axis of 2D problems) is not coarsened.
#include "common.cuh"

namespace helm {

namespace {

__device__ __forceinline__ double2 axpy(double2 acc, double w, double2 v) {
  return make_double2(fma(w, v.x, acc.x), fma(w, v.y, acc.y));
}
__device__ __forceinline__ float2 axpy(float2 acc, float w, float2 v) {
  return make_float2(fma(w, v.x, acc.x), fma(w, v.y, acc.y));
}
__device__ __forceinline__ double axpy(double acc, double w, double v) { return fma(w, v, acc); }

template <typename T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ double2 zero_of<double2>() { return make_double2(0, 0); }
template <> __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0, 0); }
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <typename T> __device__ __forceinline__ T add(T a, T b);
template <> __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
template <> __device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

struct Dims { int f[3]; int c[3]; };

// Grid of both kernels: (plane segments of 256 points, planes, slots); all
// index arithmetic in 32 bits within a plane.

// coarse = R fine for one slot per blockIdx.z (act list) or a single field (act == nullptr)
template <typename T, typename W>
__global__ void __launch_bounds__(256) k_restrict(const T* __restrict__ fine, T* __restrict__ coarse, Dims D,
                                                  const int* __restrict__ act, size_t nf, size_t nc) {
  const int Pc = D.c[0] * D.c[1];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Pc) return;
  const int jz = blockIdx.y;
  const int s = act ? act[blockIdx.z] : 0;
  const int jx = q % D.c[0], jy = q / D.c[0];
  const bool cx = D.f[0] != D.c[0], cy = D.f[1] != D.c[1], cz = D.f[2] != D.c[2];
  const int fx = cx ? 2 * jx + 1 : jx, fy = cy ? 2 * jy + 1 : jy, fz = cz ? 2 * jz + 1 : jz;
  const int Pf = D.f[0] * D.f[1];
  const T* F = fine + (size_t)s * nf;
  T acc = zero_of<T>();
  const W w1[3] = {W(0.25), W(0.5), W(0.25)};
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    if (!cz && dz != 0) continue;
    const W wz = cz ? w1[dz + 1] : W(1);
    const T* Fz = F + (size_t)(fz + dz) * Pf;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      if (!cy && dy != 0) continue;
      const W wy = cy ? w1[dy + 1] : W(1);
      const T* row = Fz + (fy + dy) * D.f[0] + fx;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!cx && dx != 0) continue;
        const W wx = cx ? w1[dx + 1] : W(1);
        acc = axpy(acc, wx * wy * wz, row[dx]);
      }
    }
  }
  coarse[(size_t)s * nc + (size_t)jz * Pc + q] = acc;
}

// fine += P coarse.  Every fine node takes two taps per coarsened axis (the
// odd node's single parent appears once with weight 1, an even node's two
// parents with 1/2 each, a missing parent beyond a wall with weight 0), so
// lanes of a warp follow one path.
template <typename T, typename W>
__global__ void __launch_bounds__(256) k_prolong_add(const T* __restrict__ coarse, T* __restrict__ fine, Dims D,
                                                     const int* __restrict__ act, size_t nf, size_t nc) {
  const int Pf = D.f[0] * D.f[1];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Pf) return;
  const int s = act[blockIdx.z];
  const int fc[3] = {p % D.f[0], p / D.f[0], (int)blockIdx.y};
  int i0[3], i1[3];
  W w0[3], w1[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int f = fc[d];
    if (D.f[d] == D.c[d]) {
      i0[d] = i1[d] = f;
      w0[d] = W(1);
      w1[d] = W(0);
    } else if (f & 1) {
      i0[d] = i1[d] = (f - 1) >> 1;
      w0[d] = W(1);
      w1[d] = W(0);
    } else {
      const int j = f >> 1;  // parents j-1 and j
      i0[d] = j - 1 >= 0 ? j - 1 : 0;
      i1[d] = j < D.c[d] ? j : D.c[d] - 1;
      w0[d] = j - 1 >= 0 ? W(0.5) : W(0);
      w1[d] = j < D.c[d] ? W(0.5) : W(0);
    }
  }
  const T* Cs = coarse + (size_t)s * nc;
  const int Pc = D.c[0] * D.c[1];
  T acc = zero_of<T>();
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const W wz = a ? w1[2] : w0[2];
    const T* Cz = Cs + (size_t)(a ? i1[2] : i0[2]) * Pc;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const W wzy = wz * (b ? w1[1] : w0[1]);
      const T* row = Cz + (b ? i1[1] : i0[1]) * D.c[0];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const W w = wzy * (c ? w1[0] : w0[0]);
        if (w != W(0)) acc = axpy(acc, w, row[c ? i1[0] : i0[0]]);
      }
    }
  }
  T* Fs = fine + (size_t)s * nf + (size_t)blockIdx.y * Pf + p;
  *Fs = add(*Fs, acc);
}

Dims dims(const LevelGeom& f, const LevelGeom& c) {
  Dims D;
  for (int d = 0; d < 3; ++d) { D.f[d] = f.K[d]; D.c[d] = c.K[d]; }
  return D;
}

}  // namespace

template <typename R>
void launch_restrict(const cplx<R>* fine, const LevelGeom& f, cplx<R>* coarse, const LevelGeom& c,
                     const int* act, int na, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_TRANSFER, (double)na * (f.n + c.n) * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((c.K[0] * c.K[1] + 255) / 256), c.K[2], na);
  k_restrict<cplx<R>, R><<<grd, 256, 0, st>>>(fine, coarse, dims(f, c), act, f.n, c.n);
  count_launch();
}

template <typename R>
void launch_prolong_add(const cplx<R>* coarse, const LevelGeom& c, cplx<R>* fine, const LevelGeom& f,
                        const int* act, int na, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_TRANSFER, (double)na * (c.n + 2 * f.n) * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((f.K[0] * f.K[1] + 255) / 256), f.K[2], na);
  k_prolong_add<cplx<R>, R><<<grd, 256, 0, st>>>(coarse, fine, dims(f, c), act, f.n, c.n);
  count_launch();
}

void launch_restrict_model(const double* mf, const LevelGeom& f, double* mc, const LevelGeom& c,
                           cudaStream_t st) {
  dim3 grd((unsigned)((c.K[0] * c.K[1] + 255) / 256), c.K[2], 1);
  k_restrict<double, double><<<grd, 256, 0, st>>>(mf, mc, dims(f, c), nullptr, f.n, c.n);
  count_launch();
}

template void launch_restrict<float>(const float2*, const LevelGeom&, float2*, const LevelGeom&,
                                     const int*, int, cudaStream_t);
template void launch_restrict<double>(const double2*, const LevelGeom&, double2*, const LevelGeom&,
                                      const int*, int, cudaStream_t);
template void launch_prolong_add<float>(const float2*, const LevelGeom&, float2*, const LevelGeom&,
                                        const int*, int, cudaStream_t);
template void launch_prolong_add<double>(const double2*, const LevelGeom&, double2*, const LevelGeom&,
                                         const int*, int, cudaStream_t);

}  // namespace helm
