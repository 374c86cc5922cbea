// Inter-grid transfers of the multigrid V-cycle (Sec. 4, Alg. vcycle):
// linear interpolation P (coarse node j sits on fine node 2j+1; even fine
// nodes average their two coarse neighbours, zero beyond the walls) and the
// full-weighting restriction R = 2^-dim P^T (1D weights 1/4, 1/2, 1/4).
// A kernel axis of size 1 (the third axis of 2D problems) is not coarsened.
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

// coarse = R fine for one slot per blockIdx.y (act list) or a single field (act == nullptr)
template <typename T, typename W>
__global__ void k_restrict(const T* __restrict__ fine, T* __restrict__ coarse, Dims D,
                           const int* __restrict__ act, size_t nf, size_t nc) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int s = act ? act[blockIdx.y] : 0;
  const int jx = (int)(i % D.c[0]);
  const int jy = (int)((i / D.c[0]) % D.c[1]);
  const int jz = (int)(i / ((size_t)D.c[0] * D.c[1]));
  const T* F = fine + (size_t)s * nf;
  const bool cx = D.f[0] != D.c[0], cy = D.f[1] != D.c[1], cz = D.f[2] != D.c[2];
  const int fx = cx ? 2 * jx + 1 : jx, fy = cy ? 2 * jy + 1 : jy, fz = cz ? 2 * jz + 1 : jz;
  T acc = zero_of<T>();
  const W w1[3] = {W(0.25), W(0.5), W(0.25)};
  for (int dz = cz ? -1 : 0; dz <= (cz ? 1 : 0); ++dz) {
    const W wz = cz ? w1[dz + 1] : W(1);
    for (int dy = cy ? -1 : 0; dy <= (cy ? 1 : 0); ++dy) {
      const W wy = cy ? w1[dy + 1] : W(1);
      const size_t row = (size_t)D.f[0] * ((size_t)(fy + dy) + (size_t)D.f[1] * (size_t)(fz + dz));
      for (int dx = cx ? -1 : 0; dx <= (cx ? 1 : 0); ++dx) {
        const W wx = cx ? w1[dx + 1] : W(1);
        acc = axpy(acc, wx * wy * wz, F[row + fx + dx]);
      }
    }
  }
  coarse[(size_t)s * nc + i] = acc;
}

// fine += P coarse
template <typename T, typename W>
__global__ void k_prolong_add(const T* __restrict__ coarse, T* __restrict__ fine, Dims D,
                              const int* __restrict__ act, size_t nf, size_t nc) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const int s = act[blockIdx.y];
  int f[3];
  f[0] = (int)(i % D.f[0]);
  f[1] = (int)((i / D.f[0]) % D.f[1]);
  f[2] = (int)(i / ((size_t)D.f[0] * D.f[1]));
  int idx[3][2];
  W wt[3][2];
  int cnt[3];
  for (int d = 0; d < 3; ++d) {
    if (D.f[d] == D.c[d]) {
      cnt[d] = 1; idx[d][0] = f[d]; wt[d][0] = W(1);
    } else if (f[d] & 1) {
      cnt[d] = 1; idx[d][0] = (f[d] - 1) >> 1; wt[d][0] = W(1);
    } else {
      cnt[d] = 0;
      const int j = f[d] >> 1;  // neighbours j-1 and j
      if (j - 1 >= 0) { idx[d][cnt[d]] = j - 1; wt[d][cnt[d]] = W(0.5); ++cnt[d]; }
      if (j < D.c[d]) { idx[d][cnt[d]] = j; wt[d][cnt[d]] = W(0.5); ++cnt[d]; }
    }
  }
  const T* Cs = coarse + (size_t)s * nc;
  T acc = zero_of<T>();
  for (int a = 0; a < cnt[2]; ++a)
    for (int b = 0; b < cnt[1]; ++b)
      for (int c = 0; c < cnt[0]; ++c)
        acc = axpy(acc, wt[0][c] * wt[1][b] * wt[2][a],
                   Cs[(size_t)idx[0][c] + (size_t)D.c[0] * ((size_t)idx[1][b] + (size_t)D.c[1] * idx[2][a])]);
  T* Fs = fine + (size_t)s * nf;
  Fs[i] = add(Fs[i], acc);
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
  dim3 grd((unsigned)((c.n + 255) / 256), na);
  k_restrict<cplx<R>, R><<<grd, 256, 0, st>>>(fine, coarse, dims(f, c), act, f.n, c.n);
  count_launch();
}

template <typename R>
void launch_prolong_add(const cplx<R>* coarse, const LevelGeom& c, cplx<R>* fine, const LevelGeom& f,
                        const int* act, int na, cudaStream_t st) {
  if (na <= 0) return;
  ProfScope ps(PC_TRANSFER, (double)na * (c.n + 2 * f.n) * sizeof(cplx<R>), st);
  dim3 grd((unsigned)((f.n + 255) / 256), na);
  k_prolong_add<cplx<R>, R><<<grd, 256, 0, st>>>(coarse, fine, dims(f, c), act, f.n, c.n);
  count_launch();
}

void launch_restrict_model(const double* mf, const LevelGeom& f, double* mc, const LevelGeom& c,
                           cudaStream_t st) {
  dim3 grd((unsigned)((c.n + 255) / 256), 1);
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
