// isosurface.cu -- iso-surfaces of a cell field (the paper's Fig. 3 shows
// iso-surfaces of the Q criterion) and their orthographic depth image, in
// CUDA, with no graphics API.
//
// Extraction: marching tetrahedra.  The cube whose corners are cells
// (i + dx, j + dy, k + dz) (values with periodic wrap, coordinates unwrapped,
// corner b = dx + 2 dy + 4 dz at ((i + dx + 1/2) h, ...)) is split into the six
// tetrahedra of the Freudenthal triangulation (paths 0 -> e_a -> e_a + e_b -> 7),
// the same split in every cube, so the surface is closed.  A corner is inside
// when f > iso; a tetrahedron with one corner apart gives one triangle, two
// and two give two (the fixed vertex orders below).  Edge points are the
// linear zero of f - iso from the edge's lower corner.  Triangles are written
// cube by cube in flat cube order: a count pass, a scan of the block totals on
// the host, and an emit pass that scans its block in shared memory.
//
// Rasterisation: view along +z, W x W pixel centres ((p + 1/2) L / W), a pixel
// is covered when its three edge functions share a sign, depth by barycentric
// weights, z-buffer min through a 64-bit atomicMin on the bits of z >= 0.
//
// Every floating-point step is a single rounded IEEE operation in a fixed
// order (no contraction into FMAs), in double precision for either field type,
// so the results are those of the same arithmetic done step by step.
#include <cmath>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

constexpr int ISO_THREADS = 256;
constexpr int ISO_PER_THREAD = 16;
constexpr int ISO_CH = ISO_THREADS * ISO_PER_THREAD;  // cubes per emit block

__constant__ int kTet[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

template <typename T>
__device__ __forceinline__ void cube_values(const T* f, int N, long c, double (&v)[8], int& i, int& j, int& k) {
  i = (int)(c % N);
  j = (int)((c / N) % N);
  k = (int)(c / ((long)N * N));
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    int ii = i + (b & 1), jj = j + ((b >> 1) & 1), kk = k + ((b >> 2) & 1);
    ii -= ii >= N ? N : 0;
    jj -= jj >= N ? N : 0;
    kk -= kk >= N ? N : 0;
    v[b] = (double)f[ii + (long)N * (jj + (long)N * kk)];
  }
}

__device__ __forceinline__ int tet_count(const double (&v)[8], int t, double iso) {
  int n = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) n += v[kTet[t][q]] > iso ? 1 : 0;
  return (n == 1 || n == 3) ? 1 : (n == 2 ? 2 : 0);
}

// edge point between corners a and b, from the lower one
__device__ __forceinline__ void edge_pt(const double (&v)[8], int i, int j, int k, double h, double iso, int a,
                                        int b, double* p) {
  if (b < a) {
    const int s = a;
    a = b;
    b = s;
  }
  const double t = (iso - v[a]) / sub(v[b], v[a]);
  const int ia[3] = {i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1)};
  const int ib[3] = {i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double pa = mul((double)ia[q] + 0.5, h), pb = mul((double)ib[q] + 0.5, h);
    p[q] = add(pa, mul(t, sub(pb, pa)));
  }
}

__device__ __forceinline__ double tri_area(const double* p) {
  const double e1[3] = {p[3] - p[0], p[4] - p[1], p[5] - p[2]};
  const double e2[3] = {p[6] - p[0], p[7] - p[1], p[8] - p[2]};
  const double c0 = e1[1] * e2[2] - e1[2] * e2[1];
  const double c1 = e1[2] * e2[0] - e1[0] * e2[2];
  const double c2 = e1[0] * e2[1] - e1[1] * e2[0];
  return 0.5 * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

template <typename T>
__global__ void __launch_bounds__(ISO_THREADS) k_iso_count(const T* __restrict__ f, int N, double iso,
                                                           int* __restrict__ counts) {
  const long n = (long)N * N * N;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    double v[8];
    int i, j, k;
    cube_values<T>(f, N, c, v, i, j, k);
    int s = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) s += tet_count(v, t, iso);
    counts[c] = s;
  }
}

// block b: the sum of counts[b * ISO_CH, (b + 1) * ISO_CH)
__global__ void __launch_bounds__(ISO_THREADS) k_iso_blocksum(const int* __restrict__ counts, long n,
                                                              long long* __restrict__ bsum) {
  __shared__ long long red[ISO_THREADS];
  const long base = (long)blockIdx.x * ISO_CH;
  long long s = 0;
  for (int q = threadIdx.x; q < ISO_CH; q += ISO_THREADS) {
    const long c = base + q;
    if (c < n) s += counts[c];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = ISO_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

// Emit: thread t of block b owns cubes b*ISO_CH + t*ISO_PER_THREAD + [0, ISO_PER_THREAD)
// (consecutive), so a block scan of the thread totals orders the triangles by cube.
template <typename T>
__global__ void __launch_bounds__(ISO_THREADS) k_iso_emit(const T* __restrict__ f, int N, double iso, double h,
                                                          const int* __restrict__ counts,
                                                          const long long* __restrict__ boff,
                                                          double* __restrict__ tri, long long max_tri,
                                                          double* __restrict__ apart) {
  __shared__ long long scan[ISO_THREADS];
  __shared__ double red[ISO_THREADS];
  const long n = (long)N * N * N;
  const long c0 = (long)blockIdx.x * ISO_CH + (long)threadIdx.x * ISO_PER_THREAD;
  long long mine = 0;
  for (int q = 0; q < ISO_PER_THREAD; ++q)
    if (c0 + q < n) mine += counts[c0 + q];
  scan[threadIdx.x] = mine;
  __syncthreads();
  // inclusive Hillis-Steele scan of the thread totals
  for (int o = 1; o < ISO_THREADS; o <<= 1) {
    const long long add_o = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += add_o;
    __syncthreads();
  }
  long long off = boff[blockIdx.x] + scan[threadIdx.x] - mine;
  double area = 0.0;
  for (int q = 0; q < ISO_PER_THREAD; ++q) {
    const long c = c0 + q;
    if (c >= n || counts[c] == 0) continue;
    double v[8];
    int i, j, k;
    cube_values<T>(f, N, c, v, i, j, k);
    for (int t = 0; t < 6; ++t) {
      int ins[4], outs[4], ni = 0, no = 0;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const int b = kTet[t][qq];
        if (v[b] > iso) ins[ni++] = b;
        else outs[no++] = b;
      }
      double p[2][9];
      int nt = 0;
      if (ni == 1 || ni == 3) {
        const int lone = ni == 1 ? ins[0] : outs[0];
        int rest[3], nr = 0;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
          if (kTet[t][qq] != lone) rest[nr++] = kTet[t][qq];
        edge_pt(v, i, j, k, h, iso, lone, rest[0], p[0]);
        edge_pt(v, i, j, k, h, iso, lone, rest[1], p[0] + 3);
        edge_pt(v, i, j, k, h, iso, lone, rest[2], p[0] + 6);
        nt = 1;
      } else if (ni == 2) {
        const int a = ins[0], b = ins[1], cc = outs[0], d = outs[1];
        edge_pt(v, i, j, k, h, iso, a, cc, p[0]);
        edge_pt(v, i, j, k, h, iso, a, d, p[0] + 3);
        edge_pt(v, i, j, k, h, iso, b, d, p[0] + 6);
        edge_pt(v, i, j, k, h, iso, a, cc, p[1]);
        edge_pt(v, i, j, k, h, iso, b, d, p[1] + 3);
        edge_pt(v, i, j, k, h, iso, b, cc, p[1] + 6);
        nt = 2;
      }
      for (int e = 0; e < nt; ++e) {
        area += tri_area(p[e]);
        if (tri && off < max_tri)
          for (int qq = 0; qq < 9; ++qq) tri[off * 9 + qq] = p[e][qq];
        ++off;
      }
    }
  }
  red[threadIdx.x] = area;
  __syncthreads();
  for (int o = ISO_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) apart[blockIdx.x] = red[0];
}

__device__ __forceinline__ double edge_fn(double xa, double ya, double xb, double yb, double px, double py) {
  return sub(mul(sub(xb, xa), sub(py, ya)), mul(sub(yb, ya), sub(px, xa)));
}

__global__ void k_fill_u64(unsigned long long* a, long n, unsigned long long v) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) a[q] = v;
}

// one thread per triangle; depth bits of z >= 0 are ordered like z
__global__ void __launch_bounds__(ISO_THREADS) k_raster(const double* __restrict__ tri, long long ntri, int W,
                                                        double step, unsigned long long* __restrict__ depth) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ntri;
       q += (long long)gridDim.x * blockDim.x) {
    const double* p = tri + q * 9;
    const double x0 = p[0], y0 = p[1], z0 = p[2], x1 = p[3], y1 = p[4], z1 = p[5], x2 = p[6], y2 = p[7], z2 = p[8];
    if (edge_fn(x0, y0, x1, y1, x2, y2) == 0.0) continue;
    const int lo_x = max((int)floor(fmin(x0, fmin(x1, x2)) / step - 0.5) - 1, 0);
    const int hi_x = min((int)ceil(fmax(x0, fmax(x1, x2)) / step - 0.5) + 1, W - 1);
    const int lo_y = max((int)floor(fmin(y0, fmin(y1, y2)) / step - 0.5) - 1, 0);
    const int hi_y = min((int)ceil(fmax(y0, fmax(y1, y2)) / step - 0.5) + 1, W - 1);
    for (int py = lo_y; py <= hi_y; ++py) {
      const double cy = mul((double)py + 0.5, step);
      for (int px = lo_x; px <= hi_x; ++px) {
        const double cx = mul((double)px + 0.5, step);
        const double e12 = edge_fn(x1, y1, x2, y2, cx, cy);
        const double e20 = edge_fn(x2, y2, x0, y0, cx, cy);
        const double e01 = edge_fn(x0, y0, x1, y1, cx, cy);
        if ((e12 >= 0.0 && e20 >= 0.0 && e01 >= 0.0) || (e12 <= 0.0 && e20 <= 0.0 && e01 <= 0.0)) {
          const double num = add(add(mul(e12, z0), mul(e20, z1)), mul(e01, z2));
          const double z = num / add(add(e12, e20), e01);
          if (z >= 0.0) atomicMin(&depth[(long)py * W + px], (unsigned long long)__double_as_longlong(z));
        }
      }
    }
  }
}

static int iso_grid(long n, int nsm) {
  const long g = (n + ISO_THREADS - 1) / ISO_THREADS;
  const long cap = (long)nsm * 8;
  return (int)(g < cap ? g : cap);
}

long iso_blocks(long n) { return (n + ISO_CH - 1) / ISO_CH; }

// counts: n ints; bsum/boff/apart: iso_blocks(n) entries (device); hb: host scratch of 2 iso_blocks(n) doubles
template <typename T>
int isosurface(const T* f, int N, double iso, double* tri, long long max_tri, int* counts, long long* bsum,
               long long* boff, double* apart, std::vector<double>& hscratch, int nsm, long long* ntri,
               double* area, cudaStream_t st) {
  const long n = (long)N * N * N;
  const long nb = iso_blocks(n);
  const double h = 2.0 * M_PI / N;
  k_iso_count<T><<<iso_grid(n, nsm), ISO_THREADS, 0, st>>>(f, N, iso, counts);
  k_iso_blocksum<<<(unsigned)nb, ISO_THREADS, 0, st>>>(counts, n, bsum);
  std::vector<long long> hs(nb), ho(nb);
  if (cudaMemcpyAsync(hs.data(), bsum, nb * sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FE_ERR_CUDA;
  long long run = 0;
  for (long b = 0; b < nb; ++b) {
    ho[b] = run;
    run += hs[b];
  }
  if (cudaMemcpyAsync(boff, ho.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FE_ERR_CUDA;
  k_iso_emit<T><<<(unsigned)nb, ISO_THREADS, 0, st>>>(f, N, iso, h, counts, boff, tri, max_tri, apart);
  hscratch.resize(nb);
  if (cudaMemcpyAsync(hscratch.data(), apart, nb * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return FE_ERR_CUDA;
  double a = 0.0;
  for (long b = 0; b < nb; ++b) a += hscratch[b];
  *ntri = run;
  *area = a;
  return FE_OK;
}

int raster_depth(const double* tri, long long ntri, int W, double extent, double* depth, int nsm, cudaStream_t st) {
  const long npx = (long)W * W;
  k_fill_u64<<<iso_grid(npx, nsm), ISO_THREADS, 0, st>>>((unsigned long long*)depth, npx, 0x7FF0000000000000ull);
  if (ntri > 0)
    k_raster<<<iso_grid((long)ntri, nsm), ISO_THREADS, 0, st>>>(tri, ntri, W, extent / W,
                                                                 (unsigned long long*)depth);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

template int isosurface<double>(const double*, int, double, double*, long long, int*, long long*, long long*,
                                double*, std::vector<double>&, int, long long*, double*, cudaStream_t);
template int isosurface<float>(const float*, int, double, double*, long long, int*, long long*, long long*,
                               double*, std::vector<double>&, int, long long*, double*, cudaStream_t);

}  // namespace fe
