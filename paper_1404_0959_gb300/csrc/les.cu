// les.cu -- a-priori analysis of the sub-grid stress for large-eddy simulation
// (the paper's Sec. 1 names LES of the plume as the goal of its DNS, Sec. 2
// the a-priori use of the DNS database; neither names a filter or a model).
//
// Filter: top-hat of width Delta = 2 m h per axis by the trapezoidal rule
// (end points at half weight), applied as a tensor product.  Favre filtering:
// rho_bar = bar(rho), u~_i = bar(rho u_i) / rho_bar; sub-grid stress
// tau_ij = bar(rho u_i u_j) - bar(rho u_i) bar(rho u_j) / rho_bar.  Resolved
// strain from the Gauss cell gradient of u~ (the method's own Gc, in the
// compact form (f_{i-2} - 10 f_{i-1} + 10 f_{i+1} - f_{i+2}) / 16h), model
// slot: Smagorinsky B_ij = -2 rho_bar Delta^2 |S| S^d_ij.  Statistics: means
// of tau_kk / 2, -tau^d:S, tau^d:B, B:B, tau^d:tau^d and B:S.
//
// Passes over HBM (N^3 words each): x pass reads rho, u (4) and writes the ten
// x-filtered quantities (rho, rho u_i, rho u_i u_j); y and z passes read ten
// and write ten (each thread eight consecutive outputs from a register window
// when N is a multiple of eight and m <= 4); the Favre velocity reads four and
// writes three; the statistics pass reads thirteen.  74 words per cell in all.
#include <cmath>
#include <cstring>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

constexpr int LES_NF = 10;       // rho, rho u (3), rho u u (6: 00 01 02 11 12 22)
constexpr int LES_THREADS = 256;

template <typename T>
struct LesPtrs {
  T* f[LES_NF];
};

__device__ __forceinline__ long les_wrap(long i, long N) { return i < 0 ? i + N : (i >= N ? i - N : i); }

// trapezoidal top-hat weight of offset o in -m..m
template <typename T>
__device__ __forceinline__ T les_w(int o, int m) {
  const T w = T(1) / T(2 * m);
  return (o == -m || o == m) ? T(0.5) * w : w;
}

// x pass: products formed on the fly, filtered along x
template <typename T>
__global__ void __launch_bounds__(LES_THREADS) k_les_x(const T* __restrict__ rho, const T* __restrict__ u0,
                                                       const T* __restrict__ u1, const T* __restrict__ u2, int N,
                                                       int m, LesPtrs<T> out) {
  const long n = (long)N * N * N;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const long i = c % N, row = c - i;
    T acc[LES_NF];
#pragma unroll
    for (int q = 0; q < LES_NF; ++q) acc[q] = T(0);
    for (int o = -m; o <= m; ++o) {
      const long s = row + les_wrap(i + o, N);
      const T w = les_w<T>(o, m);
      const T r = rho[s], a = u0[s], b = u1[s], d = u2[s];
      const T ra = r * a, rb = r * b, rd = r * d;
      acc[0] += w * r;
      acc[1] += w * ra;
      acc[2] += w * rb;
      acc[3] += w * rd;
      acc[4] += w * (ra * a);
      acc[5] += w * (ra * b);
      acc[6] += w * (ra * d);
      acc[7] += w * (rb * b);
      acc[8] += w * (rb * d);
      acc[9] += w * (rd * d);
    }
#pragma unroll
    for (int q = 0; q < LES_NF; ++q) out.f[q][c] = acc[q];
  }
}

// y (axis 1) or z (axis 2) pass over the ten fields
template <typename T>
__global__ void __launch_bounds__(LES_THREADS) k_les_line(LesPtrs<T> in, LesPtrs<T> out, int N, int m, int axis) {
  const long n = (long)N * N * N;
  const long stride = axis == 1 ? N : (long)N * N;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const long pos = (c / stride) % N;
    const long base = c - pos * stride;
    T acc[LES_NF];
#pragma unroll
    for (int q = 0; q < LES_NF; ++q) acc[q] = T(0);
    for (int o = -m; o <= m; ++o) {
      const long s = base + les_wrap(pos + o, N) * stride;
      const T w = les_w<T>(o, m);
#pragma unroll
      for (int q = 0; q < LES_NF; ++q) acc[q] += w * in.f[q][s];
    }
#pragma unroll
    for (int q = 0; q < LES_NF; ++q) out.f[q][c] = acc[q];
  }
}

// y (axis 1) or z (axis 2) pass with a register window: each thread makes LES_OUTS consecutive outputs
// along the axis from LES_OUTS + 2M loads per field (N a multiple of LES_OUTS); the weighted sum of
// each output runs over the offsets -M..M in order, as in k_les_line.
constexpr int LES_OUTS = 8;
template <typename T, int M>
__global__ void __launch_bounds__(LES_THREADS) k_les_win(LesPtrs<T> in, LesPtrs<T> out, int N, int axis) {
  const long nb = (long)N * N * (N / LES_OUTS);
  const long stride = axis == 1 ? N : (long)N * N;
  const T w = T(1) / T(2 * M), we = T(0.5) * w;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < nb; q += (long)gridDim.x * blockDim.x) {
    // q = i + N (a + N b) with a in [0, N), b in [0, N / LES_OUTS): axis 1: (i, k = a, block of j = b);
    // axis 2: (i, j = a, block of k = b); the outputs are p0 .. p0 + LES_OUTS - 1 < N along the axis
    const long i = q % N, a = (q / N) % N, b = q / ((long)N * N);
    const long base = axis == 1 ? i + (long)N * (long)N * a : i + (long)N * a;
    const long p0 = b * LES_OUTS;
#pragma unroll
    for (int f = 0; f < LES_NF; ++f) {  // unrolled: the field pointers stay in registers
      const T* src = in.f[f];
      T win[LES_OUTS + 2 * M];
#pragma unroll
      for (int t = 0; t < LES_OUTS + 2 * M; ++t) win[t] = src[base + les_wrap(p0 - M + t, N) * stride];
      T* dst = out.f[f];
#pragma unroll
      for (int o = 0; o < LES_OUTS; ++o) {
        T acc = T(0);
#pragma unroll
        for (int t = 0; t <= 2 * M; ++t) acc += ((t == 0 || t == 2 * M) ? we : w) * win[o + t];
        dst[base + (p0 + o) * stride] = acc;
      }
    }
  }
}

// u~_i = bar(rho u_i) / rho_bar
template <typename T>
__global__ void __launch_bounds__(LES_THREADS) k_les_favre(LesPtrs<T> F, T* __restrict__ ut0, T* __restrict__ ut1,
                                                           T* __restrict__ ut2, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const T ir = T(1) / F.f[0][c];
    ut0[c] = F.f[1][c] * ir;
    ut1[c] = F.f[2][c] * ir;
    ut2[c] = F.f[3][c] * ir;
  }
}

// Gauss cell gradient along d of a cell field (h * Gc), compact form
template <typename T>
__device__ __forceinline__ T les_gc_h(const T* __restrict__ f, long i, long j, long k, int N, int d) {
  auto at = [&](int s) -> T {
    long ii = i, jj = j, kk = k;
    if (d == 0) ii = les_wrap(i + s, N);
    else if (d == 1) jj = les_wrap(j + s, N);
    else kk = les_wrap(k + s, N);
    return f[ii + (long)N * (jj + (long)N * kk)];
  };
  return ((at(-2) - at(2)) + T(10) * (at(1) - at(-1))) * T(0.0625);
}

// symmetric tensors in the order 00 01 02 11 12 22
template <typename T>
__device__ __forceinline__ T les_contract(const T (&a)[6], const T (&b)[6]) {
  return a[0] * b[0] + a[3] * b[3] + a[5] * b[5] + T(2) * (a[1] * b[1] + a[2] * b[2] + a[4] * b[4]);
}

template <typename T>
__device__ __forceinline__ void les_dev(T (&a)[6]) {
  const T tr = (a[0] + a[3] + a[5]) * T(1.0 / 3.0);
  a[0] -= tr;
  a[3] -= tr;
  a[5] -= tr;
}

constexpr int LES_NS = 6;  // sums: tr tau, tau^d:S, tau^d:B, B:B, tau^d:tau^d, B:S

// statistics; optional output (rho_bar, u~ (3), tau (6)) as ten N^3 arrays
template <typename T>
__global__ void __launch_bounds__(LES_THREADS) k_les_stats(LesPtrs<T> F, const T* __restrict__ ut0,
                                                           const T* __restrict__ ut1, const T* __restrict__ ut2,
                                                           int N, double ih, double delta, double* part, T* out) {
  const long n = (long)N * N * N;
  const T* ut[3] = {ut0, ut1, ut2};
  const T ihT = (T)ih, d2 = (T)(delta * delta);
  T acc[LES_NS];
#pragma unroll
  for (int q = 0; q < LES_NS; ++q) acc[q] = T(0);
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const long i = c % N, j = (c / N) % N, k = c / ((long)N * N);
    const T rb = F.f[0][c];
    const T ir = T(1) / rb;
    const T ru[3] = {F.f[1][c], F.f[2][c], F.f[3][c]};
    T tau[6];
    tau[0] = F.f[4][c] - ru[0] * ru[0] * ir;
    tau[1] = F.f[5][c] - ru[0] * ru[1] * ir;
    tau[2] = F.f[6][c] - ru[0] * ru[2] * ir;
    tau[3] = F.f[7][c] - ru[1] * ru[1] * ir;
    tau[4] = F.f[8][c] - ru[1] * ru[2] * ir;
    tau[5] = F.f[9][c] - ru[2] * ru[2] * ir;
    // g[a][b] = Gc_b u~_a
    T g[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) g[a][b] = les_gc_h<T>(ut[a], i, j, k, N, b) * ihT;
    T S[6] = {g[0][0], T(0.5) * (g[0][1] + g[1][0]), T(0.5) * (g[0][2] + g[2][0]), g[1][1],
              T(0.5) * (g[1][2] + g[2][1]), g[2][2]};
    const T mag = sqrt(T(2) * les_contract<T>(S, S));
    T Sd[6] = {S[0], S[1], S[2], S[3], S[4], S[5]};
    les_dev<T>(Sd);
    T B[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) B[q] = T(-2) * rb * d2 * mag * Sd[q];
    T td[6] = {tau[0], tau[1], tau[2], tau[3], tau[4], tau[5]};
    les_dev<T>(td);
    acc[0] += tau[0] + tau[3] + tau[5];
    acc[1] += les_contract<T>(td, S);
    acc[2] += les_contract<T>(td, B);
    acc[3] += les_contract<T>(B, B);
    acc[4] += les_contract<T>(td, td);
    acc[5] += les_contract<T>(B, S);
    if (out) {
      out[c] = rb;
      out[n + c] = ru[0] * ir;
      out[2 * n + c] = ru[1] * ir;
      out[3 * n + c] = ru[2] * ir;
#pragma unroll
      for (int q = 0; q < 6; ++q) out[(4 + q) * n + c] = tau[q];
    }
  }
  // block tree in double (fixed order); the host adds the block partials in order
  __shared__ double red[LES_THREADS / 32][LES_NS];
#pragma unroll
  for (int q = 0; q < LES_NS; ++q) {
    double v = (double)acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < LES_NS) {
    double s = 0.0;
    for (int w = 0; w < LES_THREADS / 32; ++w) s += red[w][threadIdx.x];
    part[(long)blockIdx.x * LES_NS + threadIdx.x] = s;
  }
}

static int les_grid(long n, int nsm) {
  const long g = (n + LES_THREADS - 1) / LES_THREADS;
  const long cap = (long)nsm * 8;
  return (int)(g < cap ? g : cap);
}

// work: 23 N^3 arrays of T (x/z output set, y output set, u~); part: les_grid
// blocks x LES_NS doubles.  Statistics in stats[0..5]: delta, k_sgs, pi_sgs,
// cs2_opt, corr, pi_model (fixed-order sums).
template <typename T>
int les_apriori(const T* rho, const T* u0, const T* u1, const T* u2, int N, int m, double cs, T* work, double* part,
                double* hpart, int nsm, T* out, double* stats, cudaStream_t st) {
  const long n = (long)N * N * N;
  LesPtrs<T> A, Bp;
  for (int q = 0; q < LES_NF; ++q) {
    A.f[q] = work + q * n;
    Bp.f[q] = work + (LES_NF + q) * n;
  }
  T* ut = work + 2 * LES_NF * n;
  const int grid = les_grid(n, nsm);
  k_les_x<T><<<grid, LES_THREADS, 0, st>>>(rho, u0, u1, u2, N, m, A);
  if (N % LES_OUTS == 0 && m <= 4) {
    const int gw = les_grid(n / LES_OUTS, nsm);
    for (int axis = 1; axis <= 2; ++axis) {
      const LesPtrs<T>& src = axis == 1 ? A : Bp;
      const LesPtrs<T>& dst = axis == 1 ? Bp : A;
      switch (m) {
        case 1: k_les_win<T, 1><<<gw, LES_THREADS, 0, st>>>(src, dst, N, axis); break;
        case 2: k_les_win<T, 2><<<gw, LES_THREADS, 0, st>>>(src, dst, N, axis); break;
        case 3: k_les_win<T, 3><<<gw, LES_THREADS, 0, st>>>(src, dst, N, axis); break;
        default: k_les_win<T, 4><<<gw, LES_THREADS, 0, st>>>(src, dst, N, axis); break;
      }
    }
  } else {
    k_les_line<T><<<grid, LES_THREADS, 0, st>>>(A, Bp, N, m, 1);
    k_les_line<T><<<grid, LES_THREADS, 0, st>>>(Bp, A, N, m, 2);
  }
  k_les_favre<T><<<grid, LES_THREADS, 0, st>>>(A, ut, ut + n, ut + 2 * n, n);
  const double h = 2.0 * M_PI / N, delta = 2.0 * m * h;
  k_les_stats<T><<<grid, LES_THREADS, 0, st>>>(A, ut, ut + n, ut + 2 * n, N, 1.0 / h, delta, part, out);
  if (cudaMemcpyAsync(hpart, part, (size_t)grid * LES_NS * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return FE_ERR_CUDA;
  double s[LES_NS] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < grid; ++b)
    for (int q = 0; q < LES_NS; ++q) s[q] += hpart[(long)b * LES_NS + q];
  for (int q = 0; q < LES_NS; ++q) s[q] /= (double)n;
  stats[0] = delta;
  stats[1] = 0.5 * s[0];
  stats[2] = -s[1];
  stats[3] = s[3] > 0.0 ? s[2] / s[3] : 0.0;
  stats[4] = (s[3] > 0.0 && s[4] > 0.0) ? s[2] / std::sqrt(s[3] * s[4]) : 0.0;
  stats[5] = -cs * cs * s[5];
  return FE_OK;
}

int les_max_blocks(int nsm) { return nsm * 8; }

template int les_apriori<double>(const double*, const double*, const double*, const double*, int, int, double,
                                 double*, double*, double*, int, double*, double*, cudaStream_t);
template int les_apriori<float>(const float*, const float*, const float*, const float*, int, int, double, float*,
                                double*, double*, int, float*, double*, cudaStream_t);

}  // namespace fe
