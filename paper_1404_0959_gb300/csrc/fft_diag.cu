// fft_diag.cu -- spectral initial condition, turbulence diagnostics, Q field.
//
// Sec. 1 of arXiv:1404.0959: freely decaying homogeneous isotropic turbulence
// at r.m.s. Mach 0.2 / 0.5.  Sec. 2 par. 1: energy spectrum, enstrophy, kinetic
// energy and Taylor microscale; Fig. 1: density r.m.s.; Fig. 3: Q iso-surfaces.
//
// The 3D DFT is done as 1D transforms of every grid line, one thread block per
// line, with a mixed-radix (4, 2, 3) Stockham autosort FFT in shared memory
// (FP64).  N = 2^a 3^b, N <= 512.  None of this is on the per-step hot path.
#include <cuComplex.h>

#include "fe_internal.cuh"

namespace fe {

template <typename T>
__device__ __forceinline__ T* F(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

// ---- FFT -------------------------------------------------------------------------------
constexpr int FFT_THREADS = 256;
constexpr int FFT_MAXN = 512;

struct Radices {
  int n, r[12];
};

// One Stockham stage set for a line held in shared memory.  sign = -1 forward,
// +1 inverse (unnormalised).
__global__ void __launch_bounds__(FFT_THREADS) k_fft_lines(double2* data, int N, int axis, int sign, Radices rad) {
  __shared__ double2 buf[2][FFT_MAXN];
  const int l = blockIdx.x;
  long base, stride;
  const long NN = (long)N * N;
  if (axis == 0) {
    base = (long)N * l;  // (j, k) row
    stride = 1;
  } else if (axis == 1) {
    base = (long)(l % N) + NN * (l / N);
    stride = N;
  } else {
    base = (long)(l % N) + (long)N * (l / N);
    stride = NN;
  }
  for (int q = threadIdx.x; q < N; q += blockDim.x) buf[0][q] = data[base + stride * q];
  __syncthreads();
  int cur = 0;
  int n = N, s = 1;
  for (int st = 0; st < rad.n; ++st) {
    const int r = rad.r[st];
    const int m = n / r;
    const double2* X = buf[cur];
    double2* Y = buf[cur ^ 1];
    for (int w = threadIdx.x; w < m * s; w += blockDim.x) {
      const int p = w / s, q = w % s;
      double2 a[4];
      for (int t = 0; t < r; ++t) a[t] = X[q + s * (p + t * m)];
      for (int tp = 0; tp < r; ++tp) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < r; ++t) {
          double sn, cs;
          sincospi(2.0 * (double)((t * tp) % r) / (double)r, &sn, &cs);
          sn *= sign;
          re += a[t].x * cs - a[t].y * sn;
          im += a[t].x * sn + a[t].y * cs;
        }
        double sn, cs;
        sincospi(2.0 * (double)(p * tp) / (double)n, &sn, &cs);
        sn *= sign;
        Y[q + s * (r * p + tp)] = make_double2(re * cs - im * sn, re * sn + im * cs);
      }
    }
    __syncthreads();
    cur ^= 1;
    n = m;
    s *= r;
  }
  for (int q = threadIdx.x; q < N; q += blockDim.x) data[base + stride * q] = buf[cur][q];
}

static Radices radices_of(int N) {
  Radices R;
  R.n = 0;
  while (N % 4 == 0) { R.r[R.n++] = 4; N /= 4; }
  while (N % 2 == 0) { R.r[R.n++] = 2; N /= 2; }
  while (N % 3 == 0) { R.r[R.n++] = 3; N /= 3; }
  if (N != 1) R.n = -1;
  return R;
}

bool fft_supported(int N) { return N >= 2 && N <= FFT_MAXN && radices_of(N).n >= 0; }

void fft3d(double2* data, int N, int sign, cudaStream_t st) {
  Radices R = radices_of(N);
  for (int ax = 0; ax < 3; ++ax) k_fft_lines<<<N * N, FFT_THREADS, 0, st>>>(data, N, ax, sign, R);
}

// ---- spectral initial condition ---------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014): output m of the stream seeded with s is
// mix(s + (m+1) * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t m) {
  uint64_t z = seed + (m + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t z) { return (double)((z >> 11) + 1ull) * 0x1.0p-53; }

__global__ void k_ic_modes(double2* uh0, double2* uh1, double2* uh2, int N, uint64_t seed, double k0) {
  const long NNN = (long)N * N * N;
  for (long f = blockIdx.x * (long)blockDim.x + threadIdx.x; f < NNN; f += (long)gridDim.x * blockDim.x) {
    int i = (int)(f % N), j = (int)((f / N) % N), k = (int)(f / ((long)N * N));
    double kv[3] = {(double)(i < (N + 1) / 2 ? i : i - N), (double)(j < (N + 1) / 2 ? j : j - N),
                    (double)(k < (N + 1) / 2 ? k : k - N)};
    double2 g[3];
    for (int c = 0; c < 3; ++c) {
      uint64_t m0 = 2ull * (3ull * (uint64_t)f + (uint64_t)c);
      double a = u01(splitmix64_at(seed, m0)), b = u01(splitmix64_at(seed, m0 + 1ull));
      double r = sqrt(-2.0 * log(a));
      double sn, cs;
      sincospi(2.0 * b, &sn, &cs);
      g[c] = make_double2(r * cs * M_SQRT1_2, r * sn * M_SQRT1_2);
    }
    double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
    bool keep = k2 > 0.0;
    if (N % 2 == 0) {
      double nyq = -(double)(N / 2);
      keep = keep && kv[0] != nyq && kv[1] != nyq && kv[2] != nyq;
    }
    double2* out[3] = {uh0, uh1, uh2};
    if (!keep) {
      for (int c = 0; c < 3; ++c) out[c][f] = make_double2(0.0, 0.0);
      continue;
    }
    double kd_re = kv[0] * g[0].x + kv[1] * g[1].x + kv[2] * g[2].x;
    double kd_im = kv[0] * g[0].y + kv[1] * g[1].y + kv[2] * g[2].y;
    double km = sqrt(k2);
    double E = k2 * k2 * exp(-2.0 * (km / k0) * (km / k0));
    double amp = sqrt(E / (4.0 * M_PI * k2));
    for (int c = 0; c < 3; ++c) {
      double re = (g[c].x - kv[c] * kd_re / k2) * amp;
      double im = (g[c].y - kv[c] * kd_im / k2) * amp;
      out[c][f] = make_double2(re, im);
    }
  }
}

// partial sums of |Re u|^2 per block (fixed order), for the Mach rescaling
__global__ void k_sumsq_real(const double2* a, const double2* b, const double2* c, long n, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    s += a[q].x * a[q].x + b[q].x * b[q].x + c[q].x * c[q].x;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <typename T>
__global__ void k_ic_store(const double2* uh, T* u, long n, double scale) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    u[q] = (T)(uh[q].x * scale);
}

template <typename T>
__global__ void k_fill(T* a, long n, double v) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) a[q] = (T)v;
}

template <typename T>
__global__ void k_to_complex(const T* a, double2* z, long n) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    z[q] = make_double2((double)a[q], 0.0);
}

// shell binning of |z|^2 / (2 N^6)
__global__ void k_shell(const double2* z, int N, double* bins, int nbins) {
  const long NNN = (long)N * N * N;
  const double norm = 1.0 / (2.0 * (double)N * N * N * (double)N * N * N);
  for (long f = blockIdx.x * (long)blockDim.x + threadIdx.x; f < NNN; f += (long)gridDim.x * blockDim.x) {
    int i = (int)(f % N), j = (int)((f / N) % N), k = (int)(f / ((long)N * N));
    double kx = i < (N + 1) / 2 ? i : i - N, ky = j < (N + 1) / 2 ? j : j - N, kz = k < (N + 1) / 2 ? k : k - N;
    int sh = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
    if (sh < nbins) atomicAdd(&bins[sh], (z[f].x * z[f].x + z[f].y * z[f].y) * norm);
  }
}

// ---- cell diagnostics --------------------------------------------------------------------
// Per-block partial sums, 8 + nd values: rho|u|^2, |u|^2, |w|^2, sum_d (Gc_d u_d)^2,
// rho, (rho - mean)^2, energy density, rho Y_j ...
constexpr int NDIAG = 7 + MAXD;

template <typename T>
__global__ void __launch_bounds__(NTHR) k_diag(const BoxDev* boxes, const int2* work, double* part, int box, int s,
                                                double rho_mean) {
  Tile t = tile_of(boxes, work);
  if (t.box != box) return;
  const BoxDev& B = boxes[t.box];
  const T* rho = F<T>(B, S(s, F_RHO));
  const T* u[3] = {F<T>(B, S(s, F_U0)), F<T>(B, S(s, F_U1)), F<T>(B, S(s, F_U2))};
  const double ih = B.ih;
  double acc[NDIAG];
  for (int q = 0; q < NDIAG; ++q) acc[q] = 0.0;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      const int c = n(0, 0, 0);
      double g[3][3];  // g[m][l] = Gc_m u_l
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int l = 0; l < 3; ++l) g[m][l] = Gc_h<double>(u[l], n, m, 0, 0, 0) * ih;
      double w0 = g[1][2] - g[2][1], w1 = g[2][0] - g[0][2], w2 = g[0][1] - g[1][0];
      double r = (double)rho[c];
      double uu = 0.0;
      for (int l = 0; l < 3; ++l) uu += (double)u[l][c] * (double)u[l][c];
      acc[0] += r * uu;
      acc[1] += uu;
      acc[2] += w0 * w0 + w1 * w1 + w2 * w2;
      acc[3] += g[0][0] * g[0][0] + g[1][1] * g[1][1] + g[2][2] * g[2][2];
      acc[4] += r;
      acc[5] += (r - rho_mean) * (r - rho_mean);
      if (B.closure == FE_FOURIER)
        acc[6] += r * (B.cv * (double)F<T>(B, S(s, F_T))[c] + 0.5 * uu);
      else
        acc[6] += 0.5 * r * uu;
      for (int j = 0; j < B.nd; ++j) acc[7 + j] += r * (double)F<T>(B, S(s, F_Y0 + j))[c];
    }
  }
  // plain block tree (fixed order); partials stay per block for the host to add
  __shared__ double red[NDIAG][NTHR / 32];
  const int tid = threadIdx.x + TX * threadIdx.y, lane = tid & 31, warp = tid >> 5;
  for (int q = 0; q < NDIAG; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (tid < NDIAG) {
    double v = 0.0;
    for (int w = 0; w < NTHR / 32; ++w) v += red[tid][w];
    part[(size_t)(blockIdx.x - B.tile0) * NDIAG + tid] = v;
  }
}

// Q = (|Omega|^2 - |S|^2) / 2 from the Gauss velocity gradient.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_qcrit(const BoxDev* boxes, const int2* work, int box, int s, T* q) {
  Tile t = tile_of(boxes, work);
  if (t.box != box || !t.active) return;
  const BoxDev& B = boxes[t.box];
  const T* u[3] = {F<T>(B, S(s, F_U0)), F<T>(B, S(s, F_U1)), F<T>(B, S(s, F_U2))};
  const double ih = B.ih;
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    double g[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int l = 0; l < 3; ++l) g[m][l] = Gc_h<double>(u[l], n, m, 0, 0, 0) * ih;
    double s2 = 0.0, w2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double sv = 0.5 * (g[j][i] + g[i][j]), wv = 0.5 * (g[j][i] - g[i][j]);
        s2 += sv * sv;
        w2 += wv * wv;
      }
    q[n(0, 0, 0)] = (T)(0.5 * (w2 - s2));
  }
}

// ---- host-side drivers (called from fe_api.cu) -------------------------------------------
static int ew_grid(long n) {
  long g = (n + 255) / 256;
  return (int)(g < 152L * 16 ? g : 152L * 16);
}

template <typename T>
int ic_spectral(T* u0, T* u1, T* u2, int N, uint64_t seed, double k0, double mach, cudaStream_t st) {
  const long n = (long)N * N * N;
  double2* buf = nullptr;
  if (cudaMalloc(&buf, 3 * n * sizeof(double2)) != cudaSuccess) return FE_ERR_OOM;
  double* part = nullptr;
  const int nb = ew_grid(n);
  if (cudaMalloc(&part, nb * sizeof(double)) != cudaSuccess) {
    cudaFree(buf);
    return FE_ERR_OOM;
  }
  k_ic_modes<<<ew_grid(n), 256, 0, st>>>(buf, buf + n, buf + 2 * n, N, seed, k0);
  for (int c = 0; c < 3; ++c) fft3d(buf + c * n, N, +1, st);
  k_sumsq_real<<<nb, 256, 0, st>>>(buf, buf + n, buf + 2 * n, n, part);
  double* hp = (double*)malloc(nb * sizeof(double));
  cudaMemcpyAsync(hp, part, nb * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double ss = 0.0;
  for (int b = 0; b < nb; ++b) ss += hp[b];
  free(hp);
  double ms = ss / (double)n;
  double scale = ms > 0.0 ? mach / sqrt(ms) : 0.0;
  T* out[3] = {u0, u1, u2};
  for (int c = 0; c < 3; ++c) k_ic_store<T><<<ew_grid(n), 256, 0, st>>>(buf + c * n, out[c], n, scale);
  cudaStreamSynchronize(st);
  cudaFree(part);
  cudaFree(buf);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

template <typename T>
void fill(T* a, long n, double v, cudaStream_t st) {
  k_fill<T><<<ew_grid(n), 256, 0, st>>>(a, n, v);
}

template <typename T>
int spectrum(const T* u0, const T* u1, const T* u2, int N, double* host_bins, int nbins, cudaStream_t st) {
  const long n = (long)N * N * N;
  double2* buf = nullptr;
  double* bins = nullptr;
  if (cudaMalloc(&buf, n * sizeof(double2)) != cudaSuccess) return FE_ERR_OOM;
  if (cudaMalloc(&bins, nbins * sizeof(double)) != cudaSuccess) {
    cudaFree(buf);
    return FE_ERR_OOM;
  }
  cudaMemsetAsync(bins, 0, nbins * sizeof(double), st);
  const T* u[3] = {u0, u1, u2};
  for (int c = 0; c < 3; ++c) {
    k_to_complex<T><<<ew_grid(n), 256, 0, st>>>(u[c], buf, n);
    fft3d(buf, N, -1, st);
    k_shell<<<ew_grid(n), 256, 0, st>>>(buf, N, bins, nbins);
  }
  cudaMemcpyAsync(host_bins, bins, nbins * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFree(bins);
  cudaFree(buf);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

// Sums of the cell diagnostics of one box: out[NDIAG] (two passes for the rms).
template <typename T>
int diag_sums(const Launch& L, const BoxDev& hb, int box, int s, double* out) {
  double* part = nullptr;
  if (cudaMalloc(&part, (size_t)hb.ntiles * NDIAG * sizeof(double)) != cudaSuccess) return FE_ERR_OOM;
  double* hp = (double*)malloc((size_t)hb.ntiles * NDIAG * sizeof(double));
  const double n = (double)hb.N * hb.N * hb.N;
  double mean = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    k_diag<T><<<L.nblocks, dim3(TX, TY), 0, L.st>>>(L.boxes, L.work, part, box, s, mean);
    cudaMemcpyAsync(hp, part, (size_t)hb.ntiles * NDIAG * sizeof(double), cudaMemcpyDeviceToHost, L.st);
    cudaStreamSynchronize(L.st);
    for (int q = 0; q < NDIAG; ++q) {
      double v = 0.0;
      for (int b = 0; b < hb.ntiles; ++b) v += hp[(size_t)b * NDIAG + q];
      out[q] = v;
    }
    mean = out[4] / n;
  }
  free(hp);
  cudaFree(part);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

template <typename T>
void qcrit(const Launch& L, int box, int s, T* q) {
  k_qcrit<T><<<L.nblocks, dim3(TX, TY), 0, L.st>>>(L.boxes, L.work, box, s, q);
}

#define INST(T)                                                                                   \
  template int ic_spectral<T>(T*, T*, T*, int, uint64_t, double, double, cudaStream_t);           \
  template void fill<T>(T*, long, double, cudaStream_t);                                          \
  template int spectrum<T>(const T*, const T*, const T*, int, double*, int, cudaStream_t);        \
  template int diag_sums<T>(const Launch&, const BoxDev&, int, int, double*);                     \
  template void qcrit<T>(const Launch&, int, int, T*);
INST(double)
INST(float)

}  // namespace fe
