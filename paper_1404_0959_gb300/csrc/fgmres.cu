// fgmres.cu -- vector kernels of flexible GMRES(m) (declarations and the
// algorithm they serve in fgmres.cuh).  Plain grid-stride kernels over the N^3
// cells of one box: these passes are far cheaper than the network application
// each direction may carry, so they are written for clarity (coalesced
// scalar accesses, one 256-thread block per chunk of the grid).
#include "fe_internal.cuh"
#include "fgmres.cuh"

namespace fe {

constexpr int kGmThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGmThreads) k_gm_dots(const T* __restrict__ V, long n, int nv,
                                                        const T* __restrict__ w, double* __restrict__ part) {
  DotAcc<T> acc[kGmMax + 1], ww;
  for (long c = blockIdx.x * (long)kGmThreads + threadIdx.x; c < n; c += (long)gridDim.x * kGmThreads) {
    const T wc = w[c];
#pragma unroll
    for (int i = 0; i < kGmMax + 1; ++i)
      if (i < nv) acc[i].add(V[(long)i * n + c], wc);
    ww.add(wc, wc);
  }
  // block tree in FP64: warp shuffles, then the warps in order
  __shared__ double red[kGmThreads / 32][kGmPart];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kGmMax + 1; ++i) {
    double s = acc[i].value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][i] = s;
  }
  {
    double s = ww.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][kGmMax + 1] = s;
  }
  __syncthreads();
  if (threadIdx.x < kGmPart) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kGmThreads / 32; ++q) s += red[q][threadIdx.x];
    part[(long)blockIdx.x * kGmPart + threadIdx.x] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGmThreads) k_gm_combine(T* out, const T* a, double sa, const T* __restrict__ V,
                                                           long n, int nv, GmCoef h) {
  const T s = (T)sa;
  for (long c = blockIdx.x * (long)kGmThreads + threadIdx.x; c < n; c += (long)gridDim.x * kGmThreads) {
    T v = a ? s * a[c] : T(0);
#pragma unroll 4
    for (int i = 0; i < nv; ++i) v += (T)h.h[i] * V[(long)i * n + c];
    out[c] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGmThreads) k_gm_jacobi(T* __restrict__ z, const T* __restrict__ v,
                                                          const T* __restrict__ dinv, long n) {
  for (long c = blockIdx.x * (long)kGmThreads + threadIdx.x; c < n; c += (long)gridDim.x * kGmThreads)
    z[c] = v[c] * dinv[c];
}

// z = v dinv + sc[SC_NSCALE] y: the residual-form direction of the network
// output y for the unit Arnoldi vector v; block partial sums of ||z||^2
template <typename T>
__global__ void __launch_bounds__(kGmThreads) k_gm_from_net(T* __restrict__ z, const T* __restrict__ v,
                                                            const T* __restrict__ dinv, const float* __restrict__ net,
                                                            const double* __restrict__ sc, long n,
                                                            double* __restrict__ part) {
  __shared__ double red[kGmThreads / 32];
  const T scale = (T)sc[SC_NSCALE];
  double s = 0.0;
  for (long c = blockIdx.x * (long)kGmThreads + threadIdx.x; c < n; c += (long)gridDim.x * kGmThreads) {
    const T zc = v[c] * dinv[c] + scale * (T)net[c];
    z[c] = zc;
    s += (double)zc * (double)zc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kGmThreads / 32; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

__global__ void k_gm_set(double* sc, int slot, double v) { sc[slot] = v; }

__global__ void k_gm_finish(double* sc, int* active, double iters, double rr, int conv) {
  sc[SC_ITERS] = iters;
  sc[SC_RR] = rr;
  if (sc[SC_ODONE] == 0.0) sc[SC_CONV] = conv ? 1.0 : 0.0;
  if (sc[SC_DONE] == 0.0) {
    sc[SC_DONE] = 1.0;
    atomicSub(active, 1);
  }
}

template <typename T>
void gm_dots(const T* V, long n, int nv, const T* w, double* part, int nblk, cudaStream_t st) {
  k_gm_dots<T><<<nblk, kGmThreads, 0, st>>>(V, n, nv, w, part);
}
template <typename T>
void gm_combine(T* out, const T* a, double sa, const T* V, long n, int nv, const GmCoef& h, int nblk,
                cudaStream_t st) {
  k_gm_combine<T><<<nblk, kGmThreads, 0, st>>>(out, a, sa, V, n, nv, h);
}
template <typename T>
void gm_jacobi(T* z, const T* v, const T* dinv, long n, int nblk, cudaStream_t st) {
  k_gm_jacobi<T><<<nblk, kGmThreads, 0, st>>>(z, v, dinv, n);
}
template <typename T>
void gm_from_net(T* z, const T* v, const T* dinv, const float* net, const double* sc, long n, double* part, int nblk,
                 cudaStream_t st) {
  k_gm_from_net<T><<<nblk, kGmThreads, 0, st>>>(z, v, dinv, net, sc, n, part);
}
void gm_set_scalar(double* sc, int slot, double v, cudaStream_t st) { k_gm_set<<<1, 1, 0, st>>>(sc, slot, v); }
void gm_finish(double* sc, int* active, double iters, double rr, int conv, cudaStream_t st) {
  k_gm_finish<<<1, 1, 0, st>>>(sc, active, iters, rr, conv);
}

#define INST(T)                                                                                        \
  template void gm_dots<T>(const T*, long, int, const T*, double*, int, cudaStream_t);                 \
  template void gm_combine<T>(T*, const T*, double, const T*, long, int, const GmCoef&, int, cudaStream_t); \
  template void gm_jacobi<T>(T*, const T*, const T*, long, int, cudaStream_t);                          \
  template void gm_from_net<T>(T*, const T*, const T*, const float*, const double*, long, double*, int, cudaStream_t);
INST(double)
INST(float)

}  // namespace fe
