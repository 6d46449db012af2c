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
constexpr int ISO_PER_THREAD = 1;
constexpr int ISO_CH = ISO_THREADS * ISO_PER_THREAD;  // cubes per emit block

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

__device__ __forceinline__ double edge_fn(double xa, double ya, double xb, double yb, double px, double py) {
  return sub(mul(sub(xb, xa), sub(py, ya)), mul(sub(yb, ya), sub(px, xa)));
}

__global__ void k_fill_u64(unsigned long long* a, long n, unsigned long long v) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) a[q] = v;
}

// Edge function in FP32 from coordinates relative to the triangle's first
// corner (shifted in FP64, then rounded to FP32, so every value has the size
// of the triangle), with a bound on its distance from the exact edge function:
// each shifted coordinate carries one FP32 rounding (relative 2^-24 of at most
// S, the largest of them), each difference adds one, each product one and the
// final subtraction one; 8 * 2^-24 (S (|d1| + |d2|) over both products + |p1|
// + |p2|) covers them with room, and the FP64 shift adds far less.
__device__ __forceinline__ float edge_fn32(float xa, float ya, float xb, float yb, float px, float py, float S,
                                           float& bound) {
  const float d1 = xb - xa, d2 = py - ya, d3 = yb - ya, d4 = px - xa;
  const float p1 = d1 * d2, p2 = d3 * d4;
  bound = 4.76837158203125e-07f * (S * (fabsf(d1) + fabsf(d2) + fabsf(d3) + fabsf(d4)) + fabsf(p1) + fabsf(p2)) +
          1e-30f;
  return p1 - p2;
}

// sign of a filtered edge function: +1 / -1 when certain, 0 when the exact test decides
__device__ __forceinline__ int certain_sign(float e, float bound) {
  return e > 2.f * bound ? 1 : (e < -2.f * bound ? -1 : 0);
}

// one thread per triangle; depth bits of z >= 0 are ordered like z.  Every
// coverage decision equals the exact-rounding FP64 test: FP32 decides only
// when all three signs are certain (covered: one sign; not covered: two
// opposite certain signs), otherwise the FP64 edge functions decide.
__global__ void __launch_bounds__(ISO_THREADS) k_raster(const double* __restrict__ tri, long long ntri, int W,
                                                        double step, unsigned long long* __restrict__ depth) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ntri;
       q += (long long)gridDim.x * blockDim.x) {
    const double* p = tri + q * 9;
    const double x0 = p[0], y0 = p[1], z0 = p[2], x1 = p[3], y1 = p[4], z1 = p[5], x2 = p[6], y2 = p[7], z2 = p[8];
    if (edge_fn(x0, y0, x1, y1, x2, y2) == 0.0) continue;
    // FP32 copies relative to corner 0 (the shift itself in FP64)
    const float fx0 = 0.f, fy0 = 0.f, fx1 = (float)(x1 - x0), fy1 = (float)(y1 - y0), fx2 = (float)(x2 - x0),
                fy2 = (float)(y2 - y0);
    // a lower bound of any depth the barycentric formula can give inside the triangle (a convex
    // combination of the corners, a few roundings below its smallest corner at most)
    const double zlow = fmin(z0, fmin(z1, z2)) - 1e-12 * fmax(z0, fmax(z1, z2));
    const int lo_x = max((int)floor(fmin(x0, fmin(x1, x2)) / step - 0.5) - 1, 0);
    const int hi_x = min((int)ceil(fmax(x0, fmax(x1, x2)) / step - 0.5) + 1, W - 1);
    const int lo_y = max((int)floor(fmin(y0, fmin(y1, y2)) / step - 0.5) - 1, 0);
    const int hi_y = min((int)ceil(fmax(y0, fmax(y1, y2)) / step - 0.5) + 1, W - 1);
    for (int py = lo_y; py <= hi_y; ++py) {
      const double cy = mul((double)py + 0.5, step);
      const float fcy = (float)(cy - y0);
      for (int px = lo_x; px <= hi_x; ++px) {
        const double cx = mul((double)px + 0.5, step);
        const float fcx = (float)(cx - x0);
        const float S = fmaxf(fmaxf(fmaxf(fabsf(fx1), fabsf(fy1)), fmaxf(fabsf(fx2), fabsf(fy2))),
                              fmaxf(fabsf(fcx), fabsf(fcy)));
        float b12, b20, b01;
        const int s12 = certain_sign(edge_fn32(fx1, fy1, fx2, fy2, fcx, fcy, S, b12), b12);
        const int s20 = certain_sign(edge_fn32(fx2, fy2, fx0, fy0, fcx, fcy, S, b20), b20);
        const int s01 = certain_sign(edge_fn32(fx0, fy0, fx1, fy1, fcx, fcy, S, b01), b01);
        const bool pos = s12 > 0 || s20 > 0 || s01 > 0, neg = s12 < 0 || s20 < 0 || s01 < 0;
        if (pos && neg) continue;  // certainly outside
        double e12 = 0.0, e20 = 0.0, e01 = 0.0;
        if (s12 == 0 || s20 == 0 || s01 == 0) {  // a near-tie: the exact-rounding test decides
          e12 = edge_fn(x1, y1, x2, y2, cx, cy);
          e20 = edge_fn(x2, y2, x0, y0, cx, cy);
          e01 = edge_fn(x0, y0, x1, y1, cx, cy);
          if (!((e12 >= 0.0 && e20 >= 0.0 && e01 >= 0.0) || (e12 <= 0.0 && e20 <= 0.0 && e01 <= 0.0))) continue;
        } else {
          e12 = edge_fn(x1, y1, x2, y2, cx, cy);
          e20 = edge_fn(x2, y2, x0, y0, cx, cy);
          e01 = edge_fn(x0, y0, x1, y1, cx, cy);
        }
        // a triangle whose nearest corner is behind the stored depth cannot lower it
        unsigned long long* slot = &depth[(long)py * W + px];
        const double cur = __longlong_as_double((long long)*((volatile unsigned long long*)slot));
        if (zlow > cur) continue;
        const double num = add(add(mul(e12, z0), mul(e20, z1)), mul(e01, z2));
        const double z = num / add(add(e12, e20), e01);
        if (z >= 0.0 && z < cur) atomicMin(slot, (unsigned long long)__double_as_longlong(z));
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
