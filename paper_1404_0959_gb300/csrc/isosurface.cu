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
// Rasterisation in single precision: view along +z, W x W pixel centres
// ((p + 1/2) L / W, in double), coordinates relative to each triangle's first
// corner rounded to FP32, edge functions and barycentric depth in FP32, a
// pixel covered when its three edge functions share a sign, z-buffer min
// through a 32-bit atomicMin on the bits of z >= 0.
//
// Every floating-point step is a single rounded IEEE operation in a fixed
// order (no contraction into FMAs): double precision for the extraction (for
// either field type), single precision for the image, so the results are those
// of the same arithmetic done step by step.  The extraction first lists the
// cut cubes (a second scan, of cut flags) so that its double-precision work
// runs on full warps.
#include <cmath>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

constexpr int ISO_THREADS = 256;
constexpr int ISO_CH = ISO_THREADS;  // cubes per scan block

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

template <int A, int B, int C, int D>
__device__ __forceinline__ int tet_count(const double (&v)[8], double iso) {
  const int n = (v[A] > iso) + (v[B] > iso) + (v[C] > iso) + (v[D] > iso);
  return (n == 1 || n == 3) ? 1 : (n == 2 ? 2 : 0);
}

__device__ __forceinline__ int cube_count(const double (&v)[8], double iso) {
  return tet_count<0, 1, 3, 7>(v, iso) + tet_count<0, 1, 5, 7>(v, iso) + tet_count<0, 2, 3, 7>(v, iso) +
         tet_count<0, 2, 6, 7>(v, iso) + tet_count<0, 4, 5, 7>(v, iso) + tet_count<0, 4, 6, 7>(v, iso);
}

// edge point between corners a and b (values fa, fb), from the lower one
__device__ __forceinline__ void edge_pt(double fa, double fb, int i, int j, int k, double h, double iso, int a, int b,
                                        double& px, double& py, double& pz) {
  if (b < a) {
    const int s = a;
    a = b;
    b = s;
    const double t = fa;
    fa = fb;
    fb = t;
  }
  const double t = (iso - fa) / sub(fb, fa);
  const double ax = mul((double)(i + (a & 1)) + 0.5, h), bx = mul((double)(i + (b & 1)) + 0.5, h);
  const double ay = mul((double)(j + ((a >> 1) & 1)) + 0.5, h), by = mul((double)(j + ((b >> 1) & 1)) + 0.5, h);
  const double az = mul((double)(k + ((a >> 2) & 1)) + 0.5, h), bz = mul((double)(k + ((b >> 2) & 1)) + 0.5, h);
  px = add(ax, mul(t, sub(bx, ax)));
  py = add(ay, mul(t, sub(by, ay)));
  pz = add(az, mul(t, sub(bz, az)));
}

__device__ __forceinline__ double tri_area(const double (&p)[9]) {
  const double e1[3] = {p[3] - p[0], p[4] - p[1], p[5] - p[2]};
  const double e2[3] = {p[6] - p[0], p[7] - p[1], p[8] - p[2]};
  const double c0 = e1[1] * e2[2] - e1[2] * e2[1];
  const double c1 = e1[2] * e2[0] - e1[0] * e2[2];
  const double c2 = e1[0] * e2[1] - e1[1] * e2[0];
  return 0.5 * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

__device__ __forceinline__ void put_tri(const double (&p)[9], double* tri, long long& off, long long max_tri,
                                        double& area) {
  area += tri_area(p);
  if (tri && off < max_tri) {
#pragma unroll
    for (int q = 0; q < 9; ++q) tri[off * 9 + q] = p[q];
  }
  ++off;
}

// value and corner bit of tetrahedron corner q (0..3), selected without indexing
template <int A, int B, int C, int D>
__device__ __forceinline__ double tv(const double (&v)[8], int q) {
  return q == 0 ? v[A] : (q == 1 ? v[B] : (q == 2 ? v[C] : v[D]));
}
template <int A, int B, int C, int D>
__device__ __forceinline__ int tb(int q) {
  return q == 0 ? A : (q == 1 ? B : (q == 2 ? C : D));
}

// the triangles of one tetrahedron (corners A, B, C, D in order), as defined above
template <int A, int B, int C, int D>
__device__ __forceinline__ void tet_emit(const double (&v)[8], int i, int j, int k, double h, double iso,
                                         double* tri, long long& off, long long max_tri, double& area) {
  const int in0 = v[A] > iso, in1 = v[B] > iso, in2 = v[C] > iso, in3 = v[D] > iso;
  const int n = in0 + in1 + in2 + in3;
  if (n == 0 || n == 4) return;
  const int ins = in0 | (in1 << 1) | (in2 << 2) | (in3 << 3);
  double p[9];
  auto P = [&](int qa, int qb, int slot) {
    edge_pt(tv<A, B, C, D>(v, qa), tv<A, B, C, D>(v, qb), i, j, k, h, iso, tb<A, B, C, D>(qa), tb<A, B, C, D>(qb),
            p[3 * slot], p[3 * slot + 1], p[3 * slot + 2]);
  };
  if (n == 1 || n == 3) {
    const int lonemask = n == 1 ? ins : (~ins & 15);
    const int lone = __ffs(lonemask) - 1;
    // the other three corners in tetrahedron order
    const int r0 = lone == 0 ? 1 : 0, r1 = lone <= 1 ? 2 : 1, r2 = lone <= 2 ? 3 : 2;
    P(lone, r0, 0);
    P(lone, r1, 1);
    P(lone, r2, 2);
    put_tri(p, tri, off, max_tri, area);
  } else {
    const int a = __ffs(ins) - 1, b = __ffs(ins & ~(1 << a)) - 1;
    const int outm = ~ins & 15;
    const int c = __ffs(outm) - 1, d = __ffs(outm & ~(1 << c)) - 1;
    P(a, c, 0);
    P(a, d, 1);
    P(b, d, 2);
    put_tri(p, tri, off, max_tri, area);
    P(a, c, 0);
    P(b, d, 1);
    P(b, c, 2);
    put_tri(p, tri, off, max_tri, area);
  }
}

template <typename T>
__global__ void __launch_bounds__(ISO_THREADS) k_iso_count(const T* __restrict__ f, int N, double iso,
                                                           int* __restrict__ counts) {
  const long n = (long)N * N * N;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    double v[8];
    int i, j, k;
    cube_values<T>(f, N, c, v, i, j, k);
    counts[c] = cube_count(v, iso);
  }
}

// block b: the sums of counts[b * ISO_CH, (b + 1) * ISO_CH) and of the cut flags (count > 0)
__global__ void __launch_bounds__(ISO_THREADS) k_iso_blocksum(const int* __restrict__ counts, long n,
                                                              long long* __restrict__ bsum,
                                                              long long* __restrict__ bcut) {
  __shared__ long long red[ISO_THREADS], redc[ISO_THREADS];
  const long base = (long)blockIdx.x * ISO_CH;
  long long s = 0, sc = 0;
  for (int q = threadIdx.x; q < ISO_CH; q += ISO_THREADS) {
    const long c = base + q;
    if (c < n) {
      s += counts[c];
      sc += counts[c] > 0 ? 1 : 0;
    }
  }
  red[threadIdx.x] = s;
  redc[threadIdx.x] = sc;
  __syncthreads();
  for (int o = ISO_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      redc[threadIdx.x] += redc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = red[0];
    bcut[blockIdx.x] = redc[0];
  }
}

// List of the cut cubes in flat order with the offset of their first triangle
// (one cube per thread; block scans of the counts and of the cut flags).
__global__ void __launch_bounds__(ISO_THREADS) k_iso_compact(const int* __restrict__ counts, long n,
                                                             const long long* __restrict__ boff,
                                                             const long long* __restrict__ bcoff,
                                                             int* __restrict__ list, long long* __restrict__ loff) {
  __shared__ long long sc[ISO_THREADS], sf[ISO_THREADS];
  const long c = (long)blockIdx.x * ISO_CH + threadIdx.x;
  const int mine = c < n ? counts[c] : 0;
  sc[threadIdx.x] = mine;
  sf[threadIdx.x] = mine > 0 ? 1 : 0;
  __syncthreads();
  for (int o = 1; o < ISO_THREADS; o <<= 1) {
    const long long a = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
    const long long b = threadIdx.x >= o ? sf[threadIdx.x - o] : 0;
    __syncthreads();
    sc[threadIdx.x] += a;
    sf[threadIdx.x] += b;
    __syncthreads();
  }
  if (mine > 0) {
    const long long e = bcoff[blockIdx.x] + sf[threadIdx.x] - 1;
    list[e] = (int)c;
    loff[e] = boff[blockIdx.x] + sc[threadIdx.x] - mine;
  }
}

// Emit: one thread per cut cube of the list, its triangles from the listed offset.
template <typename T>
__global__ void __launch_bounds__(ISO_THREADS) k_iso_emit(const T* __restrict__ f, int N, double iso, double h,
                                                          const int* __restrict__ list,
                                                          const long long* __restrict__ loff, long long ncut,
                                                          double* __restrict__ tri, long long max_tri,
                                                          double* __restrict__ apart) {
  __shared__ double red[ISO_THREADS];
  const long long e = (long long)blockIdx.x * ISO_THREADS + threadIdx.x;
  double area = 0.0;
  if (e < ncut) {
    const long c = list[e];
    long long off = loff[e];
    double v[8];
    int i, j, k;
    cube_values<T>(f, N, c, v, i, j, k);
    tet_emit<0, 1, 3, 7>(v, i, j, k, h, iso, tri, off, max_tri, area);
    tet_emit<0, 1, 5, 7>(v, i, j, k, h, iso, tri, off, max_tri, area);
    tet_emit<0, 2, 3, 7>(v, i, j, k, h, iso, tri, off, max_tri, area);
    tet_emit<0, 2, 6, 7>(v, i, j, k, h, iso, tri, off, max_tri, area);
    tet_emit<0, 4, 5, 7>(v, i, j, k, h, iso, tri, off, max_tri, area);
    tet_emit<0, 4, 6, 7>(v, i, j, k, h, iso, tri, off, max_tri, area);
  }
  red[threadIdx.x] = area;
  __syncthreads();
  for (int o = ISO_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) apart[blockIdx.x] = red[0];
}

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }

__device__ __forceinline__ float edge_fn(float xa, float ya, float xb, float yb, float px, float py) {
  return fsub(fmul(fsub(xb, xa), fsub(py, ya)), fmul(fsub(yb, ya), fsub(px, xa)));
}

__global__ void k_fill_u32(unsigned* a, long n, unsigned v) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) a[q] = v;
}

// one thread per triangle; the bits of a float z >= 0 are ordered like z
__global__ void __launch_bounds__(ISO_THREADS) k_raster(const double* __restrict__ tri, long long ntri, int W,
                                                        double step, unsigned* __restrict__ depth) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ntri;
       q += (long long)gridDim.x * blockDim.x) {
    const double* p = tri + q * 9;
    const double x0 = p[0], y0 = p[1];
    const float X1 = (float)(p[3] - x0), Y1 = (float)(p[4] - y0), X2 = (float)(p[6] - x0), Y2 = (float)(p[7] - y0);
    const float Z0 = (float)p[2], Z1 = (float)p[5], Z2 = (float)p[8];
    if (fsub(fmul(X1, Y2), fmul(Y1, X2)) == 0.f) continue;
    const int lo_x = max((int)floor(fmin(x0, fmin(p[3], p[6])) / step - 0.5) - 1, 0);
    const int hi_x = min((int)ceil(fmax(x0, fmax(p[3], p[6])) / step - 0.5) + 1, W - 1);
    const int lo_y = max((int)floor(fmin(y0, fmin(p[4], p[7])) / step - 0.5) - 1, 0);
    const int hi_y = min((int)ceil(fmax(y0, fmax(p[4], p[7])) / step - 0.5) + 1, W - 1);
    for (int py = lo_y; py <= hi_y; ++py) {
      const float CY = (float)__dsub_rn(__dmul_rn((double)py + 0.5, step), y0);
      for (int px = lo_x; px <= hi_x; ++px) {
        const float CX = (float)__dsub_rn(__dmul_rn((double)px + 0.5, step), x0);
        const float e12 = edge_fn(X1, Y1, X2, Y2, CX, CY);
        const float e20 = edge_fn(X2, Y2, 0.f, 0.f, CX, CY);
        const float e01 = edge_fn(0.f, 0.f, X1, Y1, CX, CY);
        if ((e12 >= 0.f && e20 >= 0.f && e01 >= 0.f) || (e12 <= 0.f && e20 <= 0.f && e01 <= 0.f)) {
          const float num = fadd(fadd(fmul(e12, Z0), fmul(e20, Z1)), fmul(e01, Z2));
          const float z = __fdiv_rn(num, fadd(fadd(e12, e20), e01));
          // the depth only decreases, so a read that is already <= z (even an older value) means the
          // atomic would change nothing: most covered pixels of a many-layered surface skip it
          unsigned* d = &depth[(long)py * W + px];
          const unsigned zb = __float_as_uint(z);
          if (z >= 0.f && zb < *d) atomicMin(d, zb);
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

// work: counts (n ints), list (n ints), loff (n long longs), bsum, bcut, boff, bcoff (nb long longs each),
// apart (nb doubles): see iso_work_bytes
size_t iso_work_bytes(long n) {
  const long nb = iso_blocks(n);
  return (size_t)n * (2 * sizeof(int) + sizeof(long long)) + (size_t)nb * (4 * sizeof(long long) + sizeof(double)) +
         1024;
}

template <typename T>
int isosurface(const T* f, int N, double iso, double* tri, long long max_tri, void* work,
               std::vector<double>& hscratch, int nsm, long long* ntri, double* area, cudaStream_t st) {
  const long n = (long)N * N * N;
  const long nb = iso_blocks(n);
  const double h = 2.0 * M_PI / N;
  long long* bsum = (long long*)work;
  long long* bcut = bsum + nb;
  long long* boff = bcut + nb;
  long long* bcoff = boff + nb;
  double* apart = (double*)(bcoff + nb);
  long long* loff = (long long*)(apart + nb);
  int* counts = (int*)(loff + n);
  int* list = counts + n;
  k_iso_count<T><<<iso_grid(n, nsm), ISO_THREADS, 0, st>>>(f, N, iso, counts);
  k_iso_blocksum<<<(unsigned)nb, ISO_THREADS, 0, st>>>(counts, n, bsum, bcut);
  std::vector<long long> hs(2 * nb), ho(2 * nb);
  if (cudaMemcpyAsync(hs.data(), bsum, 2 * nb * sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FE_ERR_CUDA;
  long long run = 0, runc = 0;
  for (long b = 0; b < nb; ++b) {
    ho[b] = run;
    ho[nb + b] = runc;
    run += hs[b];
    runc += hs[nb + b];
  }
  if (cudaMemcpyAsync(boff, ho.data(), 2 * nb * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FE_ERR_CUDA;
  double a = 0.0;
  if (runc > 0) {
    k_iso_compact<<<(unsigned)nb, ISO_THREADS, 0, st>>>(counts, n, boff, bcoff, list, loff);
    const long ne = (long)((runc + ISO_THREADS - 1) / ISO_THREADS);
    k_iso_emit<T><<<(unsigned)ne, ISO_THREADS, 0, st>>>(f, N, iso, h, list, loff, runc, tri, max_tri, apart);
    hscratch.resize(ne);
    if (cudaMemcpyAsync(hscratch.data(), apart, ne * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FE_ERR_CUDA;
    for (long b = 0; b < ne; ++b) a += hscratch[b];
  }
  if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
  *ntri = run;
  *area = a;
  return FE_OK;
}

int raster_depth(const double* tri, long long ntri, int W, double extent, float* depth, int nsm, cudaStream_t st) {
  const long npx = (long)W * W;
  k_fill_u32<<<iso_grid(npx, nsm), ISO_THREADS, 0, st>>>((unsigned*)depth, npx, 0x7F800000u);
  if (ntri > 0)
    k_raster<<<iso_grid((long)ntri, nsm), ISO_THREADS, 0, st>>>(tri, ntri, W, extent / W, (unsigned*)depth);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

template int isosurface<double>(const double*, int, double, double*, long long, void*, std::vector<double>&, int,
                                long long*, double*, cudaStream_t);
template int isosurface<float>(const float*, int, double, double*, long long, void*, std::vector<double>&, int,
                               long long*, double*, cudaStream_t);

}  // namespace fe
