// unet.cu -- learned preconditioner for the pressure-correction solve.
//
// The paper (arXiv:1404.0959, Sec. 2 par. 1) solves a pressure-correction
// equation in every PISO corrector; this file adds a 3-level 3D-conv U-Net
// whose output serves as a search direction of flexible CG (the Jacobi
// direction remains the fallback).  Layers (3x3x3 kernels, periodic, ReLU
// after all but the last):
//   e1a 16->16, e1b 16->16 (N), d1 16->32 stride 2, e2 32->32 (N/2),
//   d2 32->64 stride 2, e3 64->64 (N/4), u2 [up2(e3), e2] 96->32 (N/2),
//   u1 [up2(u2), e1b] 48->16 (N), out 16->16 (N; channel 0 is the output).
// The first layer's input has 16 channels of which 2 carry data (the
// normalised residual and psi - 1), the last layer's 16 outputs of which 1 is
// used; the padding channels have zero inputs / zero loss and stay inert
// (16-wide channel groups keep every K step of the tensor-core GEMM full).
//
// Activations are channels-last BF16 (voxel-major, channels contiguous).
// Convolutions are implicit GEMMs on the tensor cores (mma.sync m16n8k16,
// BF16 x BF16 -> FP32): rows = voxels gathered per tap, K = input channels,
// columns = output channels.  The same gather kernel serves the forward pass
// and the data gradient (transposed weights, negated taps); the weight
// gradient is a GEMM over voxels with FP32 atomics per CTA.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

typedef __nv_bfloat16 bf16;

// ---- gather modes -------------------------------------------------------------------
enum Gather {
  G_SAME = 0,    // input on the output grid, position p + t
  G_DOWN = 1,    // input on the grid twice as fine (stride-2 conv), position 2p + t
  G_UP = 2,      // input on the grid half as fine, read at (p + t) / 2 (nearest upsampling)
  G_SAME_T = 3,  // data gradient of a stride-1 conv: position p - t
  G_DOWN_T = 4,  // data gradient of a stride-2 conv: output grid fine, input coarse, (p - t)/2 if even
};

struct Src {
  const bf16* ptr;
  int C;      // channels of this source (multiple of 16)
  int mode;   // Gather
  int n;      // cells per side of the source grid
};

struct ConvArgs {
  Src s0, s1;          // channels [0, s0.C) then [s0.C, s0.C + s1.C)
  int Cin;             // s0.C + s1.C
  int Cout;            // multiple of 8
  int No;              // cells per side of the output grid
  const bf16* W;       // [27][Cout][Cin] (k = ci contiguous)
  const float* bias;   // [Cout] or null
  bf16* out;           // [No^3][Cout] or null
  float* out32;        // [No^3][Cout] or null (fp32 copy)
  int out32_ch;        // channels written to out32 (1: channel 0 only, else Cout)
  int relu;
  int accumulate;      // out32 += result
};

__device__ __forceinline__ int wrapn(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Source voxel index of output position (x, y, z) for tap t, or -1 (zero).
__device__ __forceinline__ int gather_index(const Src& s, int x, int y, int z, int dx, int dy, int dz, int No) {
  int px, py, pz;
  switch (s.mode) {
    case G_SAME:
      px = wrapn(x + dx, s.n); py = wrapn(y + dy, s.n); pz = wrapn(z + dz, s.n);
      break;
    case G_DOWN:
      px = wrapn(2 * x + dx, s.n); py = wrapn(2 * y + dy, s.n); pz = wrapn(2 * z + dz, s.n);
      break;
    case G_UP:
      px = wrapn(x + dx, No) >> 1; py = wrapn(y + dy, No) >> 1; pz = wrapn(z + dz, No) >> 1;
      break;
    case G_SAME_T:
      px = wrapn(x - dx, s.n); py = wrapn(y - dy, s.n); pz = wrapn(z - dz, s.n);
      break;
    default: {  // G_DOWN_T: fine output grid No = 2 n
      int qx = wrapn(x - dx, No), qy = wrapn(y - dy, No), qz = wrapn(z - dz, No);
      if ((qx | qy | qz) & 1) return -1;
      px = qx >> 1; py = qy >> 1; pz = qz >> 1;
    }
  }
  return px + s.n * (py + s.n * pz);
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int CONV_WARPS = 4;
constexpr int CONV_MT = 2;  // 16-voxel m-tiles per warp

// Gather convolution: each warp computes 32 output voxels x all Cout (NT
// n-tiles of 8).  A fragments come straight from the channels-last source
// (two adjacent channels per 32-bit load), B fragments from the weights.
template <int NT>
__global__ void __launch_bounds__(CONV_WARPS * 32) k_conv(ConvArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const long nvox = (long)a.No * a.No * a.No;
  const long vbase = ((long)blockIdx.x * CONV_WARPS + warp) * (16 * CONV_MT);
  if (vbase >= nvox) return;
  // the two rows (voxels) of each m-tile this thread feeds
  int rx[CONV_MT][2], ry[CONV_MT][2], rz[CONV_MT][2];
  bool rv[CONV_MT][2];
#pragma unroll
  for (int m = 0; m < CONV_MT; ++m)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      long v = vbase + 16 * m + g + 8 * h;
      rv[m][h] = v < nvox;
      if (!rv[m][h]) v = 0;
      rx[m][h] = (int)(v % a.No);
      ry[m][h] = (int)((v / a.No) % a.No);
      rz[m][h] = (int)(v / ((long)a.No * a.No));
    }
  float acc[CONV_MT][NT][4];
#pragma unroll
  for (int m = 0; m < CONV_MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;

  for (int t = 0; t < 27; ++t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
#pragma unroll
    for (int sidx = 0; sidx < 2; ++sidx) {
      const Src& s = sidx == 0 ? a.s0 : a.s1;
      if (s.C == 0) continue;
      const int cofs = sidx == 0 ? 0 : a.s0.C;
      int idx[CONV_MT][2];
#pragma unroll
      for (int m = 0; m < CONV_MT; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          idx[m][h] = rv[m][h] ? gather_index(s, rx[m][h], ry[m][h], rz[m][h], dx, dy, dz, a.No) : -1;
      for (int c0 = 0; c0 < s.C; c0 += 16) {
        uint32_t af[CONV_MT][4];
#pragma unroll
        for (int m = 0; m < CONV_MT; ++m) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int id = idx[m][h];
            const bf16* p = s.ptr + (long)(id < 0 ? 0 : id) * s.C + c0 + 2 * tig;
            uint32_t lo = id < 0 ? 0u : ld_pair(p), hi = id < 0 ? 0u : ld_pair(p + 8);
            af[m][h] = lo;      // a0 (row g) / a1 (row g+8)
            af[m][2 + h] = hi;  // a2 / a3: columns + 8
          }
        }
        const bf16* wt = a.W + ((long)t * a.Cout) * a.Cin + cofs + c0 + 2 * tig;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const bf16* wp = wt + (long)(8 * n + g) * a.Cin;
          uint32_t bfr[2] = {ld_pair(wp), ld_pair(wp + 8)};
#pragma unroll
          for (int m = 0; m < CONV_MT; ++m) mma_bf16(acc[m][n], af[m], bfr);
        }
      }
    }
  }
  // epilogue: bias, ReLU, store
#pragma unroll
  for (int m = 0; m < CONV_MT; ++m)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!rv[m][h]) continue;
      const long v = vbase + 16 * m + g + 8 * h;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int co = 8 * n + 2 * tig;
        float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[co];
          v1 += a.bias[co + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.out) {
          __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
          *reinterpret_cast<__nv_bfloat162*>(a.out + v * a.Cout + co) = pr;
        }
        if (a.out32) {
          if (a.out32_ch == 1) {
            if (co == 0) a.out32[v] = a.accumulate ? a.out32[v] + v0 : v0;
          } else {
            float* o = a.out32 + v * a.Cout + co;
            if (a.accumulate) {
              o[0] += v0;
              o[1] += v1;
            } else {
              o[0] = v0;
              o[1] = v1;
            }
          }
        }
      }
    }
}

// Weight gradient: dW[t][co][ci] += sum_v dpre(v)[co] * in(v, t)[ci] over a
// chunk of voxels, for one tap, one 16-wide co block and one 32-wide ci
// block per CTA; the 4 warps split the chunk and are reduced in shared
// memory before one FP32 atomic add per weight.
struct WgradArgs {
  Src s0, s1;
  int Cin, Cout, No;
  const bf16* dpre;  // [No^3][Cout]
  float* dW;         // [27][Cout][Cin]
  long chunk;        // voxels per CTA
};

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(CONV_WARPS * 32) k_wgrad(WgradArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int t = blockIdx.y;
  const int co0 = 16 * (blockIdx.z % (a.Cout / 16 > 0 ? a.Cout / 16 : 1));
  const int ci0 = 32 * (blockIdx.z / (a.Cout / 16 > 0 ? a.Cout / 16 : 1));
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const long nvox = (long)a.No * a.No * a.No;
  const long v0 = (long)blockIdx.x * a.chunk;
  const long v1 = v0 + a.chunk < nvox ? v0 + a.chunk : nvox;
  const int ncb = a.Cin - ci0 < 32 ? (a.Cin - ci0) / 8 : 4;  // n-tiles in this ci block
  const bool row0 = co0 + g < a.Cout, row1 = co0 + g + 8 < a.Cout;
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[n][e] = 0.f;
  // warp w takes k-steps w, w + 4, ...
  for (long kb = v0 + 16 * warp; kb < v1; kb += 16 * CONV_WARPS) {
    // this thread's 4 voxels: kb + 2 tig + {0, 1, 8, 9}
    long vv[4] = {kb + 2 * tig, kb + 2 * tig + 1, kb + 2 * tig + 8, kb + 2 * tig + 9};
    bf16 dp[2][4];  // rows co0 + g, co0 + g + 8
    int gi0[4], gi1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool ok = vv[q] < v1;
      const long v = ok ? vv[q] : v0;
      const int x = (int)(v % a.No), y = (int)((v / a.No) % a.No), z = (int)(v / ((long)a.No * a.No));
      gi0[q] = ok ? gather_index(a.s0, x, y, z, dx, dy, dz, a.No) : -1;
      gi1[q] = ok && a.s1.C ? gather_index(a.s1, x, y, z, dx, dy, dz, a.No) : -1;
      const bf16 zero = __float2bfloat16(0.f);
      dp[0][q] = ok && row0 ? a.dpre[v * a.Cout + co0 + g] : zero;
      dp[1][q] = ok && row1 ? a.dpre[v * a.Cout + co0 + g + 8] : zero;
    }
    // A (16 co x 16 voxels): a0 = (g, 2tig..+1), a1 = (g+8, ..), a2 = (g, 2tig+8..+9), a3 = (g+8, ..)
    uint32_t af[4] = {pack2(dp[0][0], dp[0][1]), pack2(dp[1][0], dp[1][1]), pack2(dp[0][2], dp[0][3]),
                      pack2(dp[1][2], dp[1][3])};
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      if (n >= ncb) break;
      const int ci = ci0 + 8 * n + g;
      const bool in0 = ci < a.s0.C;
      bf16 b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int id = in0 ? gi0[q] : gi1[q];
        const Src& s = in0 ? a.s0 : a.s1;
        const int cc = in0 ? ci : ci - a.s0.C;
        b[q] = id < 0 ? __float2bfloat16(0.f) : s.ptr[(long)id * s.C + cc];
      }
      uint32_t bfr[2] = {pack2(b[0], b[1]), pack2(b[2], b[3])};
      mma_bf16(acc[n], af, bfr);
    }
  }
  // reduce the 4 warps in shared memory, then one atomic per weight
  __shared__ float red[CONV_WARPS][16][32];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int col = 8 * n + 2 * tig;
    red[warp][g][col] = acc[n][0];
    red[warp][g][col + 1] = acc[n][1];
    red[warp][g + 8][col] = acc[n][2];
    red[warp][g + 8][col + 1] = acc[n][3];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 16 * 32; e += CONV_WARPS * 32) {
    const int r = e / 32, col = e % 32;
    if (col >= 8 * ncb || co0 + r >= a.Cout) continue;
    const float s = red[0][r][col] + red[1][r][col] + red[2][r][col] + red[3][r][col];
    atomicAdd(&a.dW[((long)t * a.Cout + co0 + r) * a.Cin + ci0 + col], s);
  }
}

// bias gradient: db[co] += sum_v dpre(v)[co] (one block per chunk)
__global__ void k_bgrad(const bf16* dpre, long nvox, int Cout, float* db) {
  __shared__ float red[256];
  for (int co = 0; co < Cout; ++co) {
    float s = 0.f;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox; v += (long)gridDim.x * blockDim.x)
      s += __bfloat162float(dpre[v * Cout + co]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&db[co], red[0]);
    __syncthreads();
  }
}

// dpre = bf16(d * (act > 0))  (act null: no mask), optional second addend
__global__ void k_mask(const float* d, const float* d2, const bf16* act, long n, bf16* out) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    float v = d[q] + (d2 ? d2[q] : 0.f);
    if (act && !(__bfloat162float(act[q]) > 0.f)) v = 0.f;
    out[q] = __float2bfloat16(v);
  }
}

// sum over the 8 fine children of channels [0, Cc) of a fine [n^3][Cf] fp32 tensor -> coarse [(n/2)^3][Cc]
__global__ void k_up2_back(const float* fine, int nf, int Cf, int Cc, float* coarse) {
  const int nc = nf / 2;
  const long total = (long)nc * nc * nc * Cc;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    const int c = (int)(q % Cc);
    const long u = q / Cc;
    const int x = (int)(u % nc), y = (int)((u / nc) % nc), z = (int)(u / ((long)nc * nc));
    float s = 0.f;
    for (int oz = 0; oz < 2; ++oz)
      for (int oy = 0; oy < 2; ++oy)
        for (int ox = 0; ox < 2; ++ox) {
          const long v = (2 * x + ox) + (long)nf * ((2 * y + oy) + (long)nf * (2 * z + oz));
          s += fine[v * Cf + c];
        }
    coarse[q] = s;
  }
}

// copy channels [c0, c0 + C) of a [n][Cf] fp32 tensor into a dense [n][C]
__global__ void k_slice(const float* src, long n, int Cf, int c0, int C, float* dst) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n * C; q += (long)gridDim.x * blockDim.x)
    dst[q] = src[(q / C) * Cf + c0 + q % C];
}

// Network input of the residual-form preconditioner, for a residual r of the
// operator M = diag(psi/dt) - dt/2 D(G2 .) with Jacobi inverse dinv = 1/d,
// d = psi/dt + 3 dt/h^2: channel 0 = (r dinv) / (rms(r) d0) with d0 the
// Jacobi inverse at psi = 1, channel 1 = (3 dt/h^2) dinv (the Laplacian's
// share of the diagonal, which carries dt and psi), channels 2..15 = 0.  The
// direction is z = r dinv + rms(r) d0 y for the network output y.
// 16-channel input voxel: (c0, c1, 0, ..., 0) in two 16-byte stores
__device__ __forceinline__ void pack_voxel(bf16* o, float c0, float c1) {
  __nv_bfloat162 p = __floats2bfloat162_rn(c0, c1);
  uint4 a;
  a.x = *reinterpret_cast<uint32_t*>(&p);
  a.y = a.z = a.w = 0u;
  reinterpret_cast<uint4*>(o)[0] = a;
  reinterpret_cast<uint4*>(o)[1] = make_uint4(0u, 0u, 0u, 0u);
}

// a = 1 / (rms(r) d0), w = 3 dt / h^2
template <typename T>
__global__ void k_pack_input(const T* r, const T* dinv, long n, double a, double w, bf16* in16) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const double dq = (double)dinv[q];
    pack_voxel(in16 + q * 16, (float)((double)r[q] * dq * a), (float)(dq * w));
  }
}

// z = r dinv + scale y (the residual-form direction, FP32)
template <typename T>
__global__ void k_direction(const T* r, const T* dinv, const float* y, double scale, long n, float* z) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    z[q] = (float)((double)r[q] * (double)dinv[q] + scale * (double)y[q]);
}

// training target t = (e - r dinv) * inv_scale into tgt; block partial sums of t^2
template <typename T>
__global__ void k_target(const T* r, const T* e, const T* dinv, long n, double inv_scale, float* tgt, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const float t = (float)(((double)e[q] - (double)r[q] * (double)dinv[q]) * inv_scale);
    tgt[q] = t;
    s += (double)t * (double)t;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam (Kingma and Ba 2015) on the FP32 master weights; refreshes the BF16
// forward copy [27][Cout][Cin] and the transposed copy [27][Cin][Cout].
__global__ void k_adam(float* w, const float* g, float* m, float* v, long n, float lr, float b1, float b2, float eps,
                       float c1, float c2, int taps, int Cout, int Cin, bf16* wf, bf16* wt, int mask_ci, int mask_co) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    float gq = g[q];
    float mq = b1 * m[q] + (1.f - b1) * gq;
    float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    if (taps > 0) {
      const int ci = (int)(q % Cin);
      const int co = (int)((q / Cin) % Cout);
      const int t = (int)(q / ((long)Cin * Cout));
      if (ci >= mask_ci || co >= mask_co) wq = 0.f;  // padding channels stay inert
      wf[q] = __float2bfloat16(wq);
      wt[((long)t * Cin + ci) * Cout + co] = __float2bfloat16(wq);
    }
    w[q] = wq;
  }
}

__global__ void k_cast_weights(const float* w, long n, int Cout, int Cin, bf16* wf, bf16* wt) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int ci = (int)(q % Cin);
    const int co = (int)((q / Cin) % Cout);
    const int t = (int)(q / ((long)Cin * Cout));
    wf[q] = __float2bfloat16(w[q]);
    wt[((long)t * Cin + ci) * Cout + co] = __float2bfloat16(w[q]);
  }
}

// loss = ||y - t||^2 / ||t||^2 partial sums (y: channel 0 of out32) and dy in the 16-channel layout
__global__ void k_loss_grad(const float* y, const float* tgt, long n, double inv_tt, float* dy8, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const double d = (double)y[q] - (double)tgt[q];
    s += d * d;
    float* o = dy8 + q * 16;
    o[0] = (float)(2.0 * d * inv_tt);
    for (int c = 1; c < 16; ++c) o[c] = 0.f;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---- host side ----------------------------------------------------------------------------
struct Layer {
  const char* name;
  int cin, cout, cin_real, cout_real, level_out, stride;
  float* w;  // fp32 master [27][cout][cin]
  float* b;
  float* gw;
  float* gb;
  float* mw;
  float* vw;
  float* mb;
  float* vb;
  bf16* wf;
  bf16* wt;
};

static const int kNL = 9;
// name, cin, cout, cin_real, cout_real, level of the output, stride
static const int kDims[kNL][6] = {{16, 16, 2, 16, 0, 1},  {16, 16, 16, 16, 0, 1}, {16, 32, 16, 32, 1, 2},
                                  {32, 32, 32, 32, 1, 1}, {32, 64, 32, 64, 2, 2}, {64, 64, 64, 64, 2, 1},
                                  {96, 32, 96, 32, 1, 1}, {48, 16, 48, 16, 0, 1}, {16, 16, 16, 1, 0, 1}};
static const char* kNames[kNL] = {"e1a", "e1b", "d1", "e2", "d2", "e3", "u2", "u1", "out"};

struct UNet {
  int N = 0;  // finest grid
  Layer L[kNL];
  void* wslab = nullptr;
  // activations (bf16 channels-last)
  bf16 *in16 = nullptr, *e1a = nullptr, *e1b = nullptr, *d1 = nullptr, *e2 = nullptr, *d2 = nullptr,
       *e3 = nullptr, *u2 = nullptr, *u1 = nullptr;
  float* out32 = nullptr;  // [N^3] channel 0
  // training buffers
  float *g0 = nullptr, *g1 = nullptr, *g2 = nullptr, *gsk0 = nullptr, *gsk1 = nullptr, *dy8 = nullptr;
  bf16* dpre = nullptr;
  double* part = nullptr;
  int adam_step = 0;
  std::vector<void*> allocs;
  bool trained = false;
  int use_tc = 1;      // stride-1 layers on the fifth-generation tensor cores where they fit
  int* err = nullptr;  // device flag: a tensor-core convolution gave up a bounded wait
  int nsm = 152;
};

struct TcConvArgs {
  const bf16* s0;
  const bf16* s1;
  int c0, c1, m0, m1;
  int No;
  const bf16* W;
  const float* bias;
  bf16* out;
  float* out32;
  int relu;
  int* err;
};
int conv_tc(const TcConvArgs& a, int Cout, int nsm, cudaStream_t st);

static long cube(long n) { return n * n * n; }

static int unet_alloc(UNet& U, int N, bool training) {
  U.N = N;
  const long n0 = cube(N), n1 = cube(N / 2), n2 = cube(N / 4);
  auto A = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    U.allocs.push_back(p);
    return p;
  };
  U.in16 = (bf16*)A(n0 * 16 * 2);
  U.e1a = (bf16*)A(n0 * 16 * 2);
  U.e1b = (bf16*)A(n0 * 16 * 2);
  U.d1 = (bf16*)A(n1 * 32 * 2);
  U.e2 = (bf16*)A(n1 * 32 * 2);
  U.d2 = (bf16*)A(n2 * 64 * 2);
  U.e3 = (bf16*)A(n2 * 64 * 2);
  U.u2 = (bf16*)A(n1 * 32 * 2);
  U.u1 = (bf16*)A(n0 * 16 * 2);
  U.out32 = (float*)A(n0 * 4);
  U.err = (int*)A(sizeof(int));
  if (U.err) cudaMemset(U.err, 0, sizeof(int));
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      U.nsm = nsm;
  }
  if (!U.in16 || !U.e1a || !U.e1b || !U.d1 || !U.e2 || !U.d2 || !U.e3 || !U.u2 || !U.u1 || !U.out32 || !U.err)
    return FE_ERR_OOM;
  size_t wtotal = 0;
  for (int l = 0; l < kNL; ++l) {
    const long nw = 27L * kDims[l][0] * kDims[l][1];
    wtotal += (nw * 4 * 4 + kDims[l][1] * 4 * 4 + nw * 2 * 2 + 10 * 256);  // 10 slices, each 256-aligned
  }
  char* ws = (char*)A(wtotal);
  if (!ws) return FE_ERR_OOM;
  cudaMemset(ws, 0, wtotal);
  for (int l = 0; l < kNL; ++l) {
    Layer& y = U.L[l];
    y.name = kNames[l];
    y.cin = kDims[l][0];
    y.cout = kDims[l][1];
    y.cin_real = kDims[l][2];
    y.cout_real = kDims[l][3];
    y.level_out = kDims[l][4];
    y.stride = kDims[l][5];
    const long nw = 27L * y.cin * y.cout;
    auto take = [&](size_t bytes) {
      void* p = ws;
      ws += (bytes + 255) & ~(size_t)255;
      return p;
    };
    y.w = (float*)take(nw * 4);
    y.gw = (float*)take(nw * 4);
    y.mw = (float*)take(nw * 4);
    y.vw = (float*)take(nw * 4);
    y.b = (float*)take(y.cout * 4);
    y.gb = (float*)take(y.cout * 4);
    y.mb = (float*)take(y.cout * 4);
    y.vb = (float*)take(y.cout * 4);
    y.wf = (bf16*)take(nw * 2);
    y.wt = (bf16*)take(nw * 2);
  }
  if (training) {
    U.g0 = (float*)A(n0 * 48 * 4);
    U.g1 = (float*)A(n1 * 96 * 4);
    U.g2 = (float*)A(n2 * 64 * 4);
    U.gsk0 = (float*)A(n0 * 16 * 4);
    U.gsk1 = (float*)A(n1 * 32 * 4);
    U.dy8 = (float*)A(n0 * 16 * 4);
    U.dpre = (bf16*)A(n0 * 64 * 2 > n1 * 96 * 2 ? n0 * 64 * 2 : n1 * 96 * 2);
    U.part = (double*)A(4096 * 8);
    if (!U.g0 || !U.g1 || !U.g2 || !U.gsk0 || !U.gsk1 || !U.dy8 || !U.dpre || !U.part) return FE_ERR_OOM;
  }
  return FE_OK;
}

static void unet_free(UNet& U) {
  for (void* p : U.allocs) cudaFree(p);
  U.allocs.clear();
}

static int ew(long n) {
  long g = (n + 255) / 256;
  return (int)(g < 152L * 8 ? g : 152L * 8);
}

static void launch_conv(const UNet& U, const ConvArgs& a, cudaStream_t st) {
  // stride-1 gathers (same grid, nearest upsampling) go to the tensor-memory kernel when it fits
  auto tc_mode = [&](const Src& s, int& m) {
    if (s.C == 0) return true;
    if (s.mode == G_SAME && s.n == a.No) return (m = 0, true);
    if (s.mode == G_UP && 2 * s.n == a.No) return (m = 1, true);
    return false;
  };
  int m0 = 0, m1 = 0;
  if (U.use_tc && !a.accumulate && (a.out32 == nullptr || a.out32_ch == 1) && tc_mode(a.s0, m0) &&
      tc_mode(a.s1, m1)) {
    TcConvArgs t{a.s0.ptr, a.s1.ptr, a.s0.C, a.s1.C, m0, m1, a.No, a.W, a.bias, a.out, a.out32, a.relu, U.err};
    if (conv_tc(t, a.Cout, U.nsm, st)) return;
  }
  const long nvox = cube(a.No);
  const int grid = (int)((nvox + 16 * CONV_MT * CONV_WARPS - 1) / (16 * CONV_MT * CONV_WARPS));
  switch (a.Cout / 8) {
    case 1: k_conv<1><<<grid, CONV_WARPS * 32, 0, st>>>(a); break;
    case 2: k_conv<2><<<grid, CONV_WARPS * 32, 0, st>>>(a); break;
    case 4: k_conv<4><<<grid, CONV_WARPS * 32, 0, st>>>(a); break;
    case 6: k_conv<6><<<grid, CONV_WARPS * 32, 0, st>>>(a); break;
    case 8: k_conv<8><<<grid, CONV_WARPS * 32, 0, st>>>(a); break;
    case 12: k_conv<12><<<grid, CONV_WARPS * 32, 0, st>>>(a); break;
  }
}

static Src src(const bf16* p, int C, int mode, int n) { return Src{p, C, mode, n}; }

// forward conv of layer l
static void fwd(UNet& U, int l, Src s0, Src s1, bf16* out, float* out32, int relu, cudaStream_t st) {
  Layer& y = U.L[l];
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.s0 = s0;
  a.s1 = s1;
  a.Cin = s0.C + s1.C;
  a.Cout = y.cout;
  a.No = U.N >> y.level_out;
  a.W = y.wf;
  a.bias = y.b;
  a.out = out;
  a.out32 = out32;
  a.out32_ch = 1;
  a.relu = relu;
  launch_conv(U, a, st);
}

// Forward pass on the packed input; output channel 0 in U.out32.
static void unet_forward(UNet& U, cudaStream_t st) {
  const int n0 = U.N, n1 = U.N / 2, n2 = U.N / 4;
  Src none = src(nullptr, 0, G_SAME, 0);
  fwd(U, 0, src(U.in16, 16, G_SAME, n0), none, U.e1a, nullptr, 1, st);
  fwd(U, 1, src(U.e1a, 16, G_SAME, n0), none, U.e1b, nullptr, 1, st);
  fwd(U, 2, src(U.e1b, 16, G_DOWN, n0), none, U.d1, nullptr, 1, st);
  fwd(U, 3, src(U.d1, 32, G_SAME, n1), none, U.e2, nullptr, 1, st);
  fwd(U, 4, src(U.e2, 32, G_DOWN, n1), none, U.d2, nullptr, 1, st);
  fwd(U, 5, src(U.d2, 64, G_SAME, n2), none, U.e3, nullptr, 1, st);
  fwd(U, 6, src(U.e3, 64, G_UP, n2), src(U.e2, 32, G_SAME, n1), U.u2, nullptr, 1, st);
  fwd(U, 7, src(U.u2, 32, G_UP, n1), src(U.e1b, 16, G_SAME, n0), U.u1, nullptr, 1, st);
  fwd(U, 8, src(U.u1, 16, G_SAME, n0), none, nullptr, U.out32, 0, st);
}

// Data gradient of layer l: dIn (fp32, [n_in^3][Cin]) from dpre ([n_out^3][Cout] bf16).
static void bwd_data(UNet& U, int l, int n_in, float* dIn, cudaStream_t st) {
  Layer& y = U.L[l];
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  const int n_out = U.N >> y.level_out;
  a.s0 = src(U.dpre, y.cout, y.stride == 2 ? G_DOWN_T : G_SAME_T, n_out);
  a.s1 = src(nullptr, 0, G_SAME, 0);
  a.Cin = y.cout;
  a.Cout = y.cin;
  a.No = n_in;
  a.W = y.wt;  // [27][cin][cout]: rows = input channels, k = output channels
  a.out32 = dIn;
  a.out32_ch = y.cin;
  launch_conv(U, a, st);
}

static void wgrad(UNet& U, int l, Src s0, Src s1, cudaStream_t st) {
  Layer& y = U.L[l];
  WgradArgs a;
  a.s0 = s0;
  a.s1 = s1;
  a.Cin = y.cin;
  a.Cout = y.cout;
  a.No = U.N >> y.level_out;
  a.dpre = U.dpre;
  a.dW = y.gw;
  const long nvox = cube(a.No);
  const int coblocks = y.cout >= 16 ? y.cout / 16 : 1;
  const int ciblocks = (y.cin + 31) / 32;
  long nchunk = 64;
  a.chunk = (nvox + nchunk - 1) / nchunk;
  a.chunk = (a.chunk + 15) / 16 * 16;
  nchunk = (nvox + a.chunk - 1) / a.chunk;
  dim3 grid((unsigned)nchunk, 27, coblocks * ciblocks);
  k_wgrad<<<grid, CONV_WARPS * 32, 0, st>>>(a);
  k_bgrad<<<64, 256, 0, st>>>(U.dpre, nvox, y.cout, y.gb);
}

}  // namespace fe

namespace fe {

// Network input for the current residual of a solve: rms(r)^2 = rr / n with
// rr read from the box scalar rr_slot, dt from SC_KDT (the solve's operator);
// the output scale rms(r) d0 of the direction goes to SC_NSCALE.
template <typename T>
__global__ void k_pack_fcg(const T* r, const T* dinv, long n, double* sc, int rr_slot, double ih, bf16* in16) {
  const double rr = sc[rr_slot], dt = sc[SC_KDT];
  const double c3 = 3.0 * dt * ih * ih, d0 = 1.0 / (1.0 / dt + c3);
  const double rms = rr > 0.0 ? sqrt(rr / (double)n) : 0.0;
  const double a = rms > 0.0 ? 1.0 / (rms * d0) : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[SC_NSCALE] = rms * d0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const double dq = (double)dinv[q];
    pack_voxel(in16 + q * 16, (float)((double)r[q] * dq * a), (float)(dq * c3));
  }
}

// mean-square of a field (two-level, fixed order): part[block] partial sums
template <typename T>
__global__ void k_sumsq(const T* a, long n, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    s += (double)a[q] * (double)a[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <typename T>
__global__ void k_scale_to_f32(const T* a, long n, double s, float* out) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    out[q] = (float)((double)a[q] * s);
}

static double host_sum(const double* dpart, int nb, cudaStream_t st) {
  std::vector<double> h(nb);
  cudaMemcpyAsync(h.data(), dpart, nb * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += h[b];
  return s;
}

UNet* unet_create(int N, bool training, int* rc) {
  UNet* U = new UNet();
  *rc = unet_alloc(*U, N, training);
  if (*rc != FE_OK) {
    unet_free(*U);
    delete U;
    return nullptr;
  }
  return U;
}

void unet_destroy(UNet* U) {
  if (!U) return;
  unet_free(*U);
  delete U;
}

long unet_param_count() {
  long n = 0;
  for (int l = 0; l < kNL; ++l) n += 27L * kDims[l][2] * kDims[l][3] + kDims[l][3];
  return n;
}

// host layout per layer: W[27][cin_real][cout_real] then b[cout_real]
int unet_set_weights(UNet* U, const float* host, cudaStream_t st) {
  long off = 0;
  for (int l = 0; l < kNL; ++l) {
    Layer& y = U->L[l];
    const long nw = 27L * y.cin * y.cout;
    std::vector<float> w(nw, 0.f), b(y.cout, 0.f);
    for (int t = 0; t < 27; ++t)
      for (int ci = 0; ci < y.cin_real; ++ci)
        for (int co = 0; co < y.cout_real; ++co)
          w[((long)t * y.cout + co) * y.cin + ci] = host[off + ((long)t * y.cin_real + ci) * y.cout_real + co];
    off += 27L * y.cin_real * y.cout_real;
    for (int co = 0; co < y.cout_real; ++co) b[co] = host[off + co];
    off += y.cout_real;
    cudaMemcpyAsync(y.w, w.data(), nw * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(y.b, b.data(), y.cout * 4, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(y.mw, 0, nw * 4, st);
    cudaMemsetAsync(y.vw, 0, nw * 4, st);
    cudaMemsetAsync(y.mb, 0, y.cout * 4, st);
    cudaMemsetAsync(y.vb, 0, y.cout * 4, st);
    k_cast_weights<<<ew(nw), 256, 0, st>>>(y.w, nw, y.cout, y.cin, y.wf, y.wt);
    cudaStreamSynchronize(st);  // host vectors go out of scope
  }
  U->adam_step = 0;
  U->trained = true;
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

// which = 0: weights and biases, 1: their gradients
int unet_get_weights(UNet* U, float* host, int which, cudaStream_t st) {
  long off = 0;
  for (int l = 0; l < kNL; ++l) {
    Layer& y = U->L[l];
    const long nw = 27L * y.cin * y.cout;
    std::vector<float> w(nw), b(y.cout);
    cudaMemcpyAsync(w.data(), which ? y.gw : y.w, nw * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(b.data(), which ? y.gb : y.b, y.cout * 4, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (int t = 0; t < 27; ++t)
      for (int ci = 0; ci < y.cin_real; ++ci)
        for (int co = 0; co < y.cout_real; ++co)
          host[off + ((long)t * y.cin_real + ci) * y.cout_real + co] = w[((long)t * y.cout + co) * y.cin + ci];
    off += 27L * y.cin_real * y.cout_real;
    for (int co = 0; co < y.cout_real; ++co) host[off + co] = b[co];
    off += y.cout_real;
  }
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

// Network pass for the current residual of a solve (input as k_pack_fcg);
// the output y stays in U->out32 and its scale in sc[SC_NSCALE].
template <typename T>
void unet_apply_sc(UNet* U, const T* r, const T* dinv, double* sc, int rr_slot, double ih, cudaStream_t st) {
  const long n = cube(U->N);
  k_pack_fcg<T><<<ew(n), 256, 0, st>>>(r, dinv, n, sc, rr_slot, ih, U->in16);
  unet_forward(*U, st);
}

// Preconditioner scales of a residual: rms(r) from a fixed-order reduction, d0 from dt.
template <typename T>
static void precond_scales(UNet* U, const T* r, double dt, double ih, cudaStream_t st, double* rms, double* d0) {
  const long n = cube(U->N);
  const int nb = ew(n);
  k_sumsq<T><<<nb, 256, 0, st>>>(r, n, U->part);
  const double rr = host_sum(U->part, nb, st);
  *rms = rr > 0.0 ? sqrt(rr / (double)n) : 0.0;
  *d0 = 1.0 / (1.0 / dt + 3.0 * dt * ih * ih);
}

// z = r dinv + rms(r) d0 net(input): the residual-form direction.
template <typename T>
int unet_apply(UNet* U, const T* r, const T* dinv, double dt, double ih, float* z, cudaStream_t st) {
  const long n = cube(U->N);
  if (!U->part) return FE_ERR_UNSUPPORTED;
  double rms, d0;
  precond_scales<T>(U, r, dt, ih, st, &rms, &d0);
  k_pack_input<T><<<ew(n), 256, 0, st>>>(r, dinv, n, rms > 0.0 ? 1.0 / (rms * d0) : 0.0, 3.0 * dt * ih * ih,
                                         U->in16);
  unet_forward(*U, st);
  k_direction<T><<<ew(n), 256, 0, st>>>(r, dinv, U->out32, rms * d0, n, z);
  int herr = 0;
  cudaMemcpyAsync(&herr, U->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (herr) {
    cudaMemsetAsync(U->err, 0, sizeof(int), st);
    return FE_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

// One training step on the pair (r, e) with M e = r (M of this dt): input as
// unet_apply, target t = (e - r dinv) / (rms(r) d0), loss ||y - t||^2 /
// ||t||^2, backward through every layer, Adam.  lr <= 0: gradients only.
template <typename T>
int unet_train_step(UNet* U, const T* r, const T* e, const T* dinv, double dt, double ih, double lr, double* loss,
                    cudaStream_t st) {
  if (!U->g0) return FE_ERR_UNSUPPORTED;
  const int n0 = U->N, n1 = U->N / 2, n2 = U->N / 4;
  const long v0 = cube(n0), v1 = cube(n1), v2 = cube(n2);
  const int nb = ew(v0);
  double rms, d0;
  precond_scales<T>(U, r, dt, ih, st, &rms, &d0);
  if (!(rms > 0.0)) return FE_ERR_INVALID_ARG;
  k_pack_input<T><<<ew(v0), 256, 0, st>>>(r, dinv, v0, 1.0 / (rms * d0), 3.0 * dt * ih * ih, U->in16);
  unet_forward(*U, st);
  // target into gsk0 (fp32 scratch), its norm, then loss and dL/dy
  float* tgt = U->gsk0;
  k_target<T><<<nb, 256, 0, st>>>(r, e, dinv, v0, 1.0 / (rms * d0), tgt, U->part);
  const double tt = host_sum(U->part, nb, st);
  if (!(tt > 0.0)) return FE_ERR_INVALID_ARG;
  k_loss_grad<<<nb, 256, 0, st>>>(U->out32, tgt, v0, 1.0 / tt, U->dy8, U->part);
  *loss = host_sum(U->part, nb, st) / tt;
  for (int l = 0; l < kNL; ++l) {
    cudaMemsetAsync(U->L[l].gw, 0, 27L * U->L[l].cin * U->L[l].cout * 4, st);
    cudaMemsetAsync(U->L[l].gb, 0, U->L[l].cout * 4, st);
  }
  Src none = src(nullptr, 0, G_SAME, 0);
  // out (linear)
  k_mask<<<ew(v0 * 16), 256, 0, st>>>(U->dy8, nullptr, nullptr, v0 * 16, U->dpre);
  wgrad(*U, 8, src(U->u1, 16, G_SAME, n0), none, st);
  bwd_data(*U, 8, n0, U->g0, st);
  // u1
  k_mask<<<ew(v0 * 16), 256, 0, st>>>(U->g0, nullptr, U->u1, v0 * 16, U->dpre);
  wgrad(*U, 7, src(U->u2, 32, G_UP, n1), src(U->e1b, 16, G_SAME, n0), st);
  bwd_data(*U, 7, n0, U->g0, st);
  k_up2_back<<<ew(v1 * 32), 256, 0, st>>>(U->g0, n0, 48, 32, U->g1);
  k_slice<<<ew(v0 * 16), 256, 0, st>>>(U->g0, v0, 48, 32, 16, U->gsk0);
  // u2
  k_mask<<<ew(v1 * 32), 256, 0, st>>>(U->g1, nullptr, U->u2, v1 * 32, U->dpre);
  wgrad(*U, 6, src(U->e3, 64, G_UP, n2), src(U->e2, 32, G_SAME, n1), st);
  bwd_data(*U, 6, n1, U->g1, st);
  k_up2_back<<<ew(v2 * 64), 256, 0, st>>>(U->g1, n1, 96, 64, U->g2);
  k_slice<<<ew(v1 * 32), 256, 0, st>>>(U->g1, v1, 96, 64, 32, U->gsk1);
  // e3
  k_mask<<<ew(v2 * 64), 256, 0, st>>>(U->g2, nullptr, U->e3, v2 * 64, U->dpre);
  wgrad(*U, 5, src(U->d2, 64, G_SAME, n2), none, st);
  bwd_data(*U, 5, n2, U->g2, st);
  // d2
  k_mask<<<ew(v2 * 64), 256, 0, st>>>(U->g2, nullptr, U->d2, v2 * 64, U->dpre);
  wgrad(*U, 4, src(U->e2, 32, G_DOWN, n1), none, st);
  bwd_data(*U, 4, n1, U->g1, st);
  // e2 (+ skip from u2)
  k_mask<<<ew(v1 * 32), 256, 0, st>>>(U->g1, U->gsk1, U->e2, v1 * 32, U->dpre);
  wgrad(*U, 3, src(U->d1, 32, G_SAME, n1), none, st);
  bwd_data(*U, 3, n1, U->g1, st);
  // d1
  k_mask<<<ew(v1 * 32), 256, 0, st>>>(U->g1, nullptr, U->d1, v1 * 32, U->dpre);
  wgrad(*U, 2, src(U->e1b, 16, G_DOWN, n0), none, st);
  bwd_data(*U, 2, n0, U->g0, st);
  // e1b (+ skip from u1)
  k_mask<<<ew(v0 * 16), 256, 0, st>>>(U->g0, U->gsk0, U->e1b, v0 * 16, U->dpre);
  wgrad(*U, 1, src(U->e1a, 16, G_SAME, n0), none, st);
  bwd_data(*U, 1, n0, U->g0, st);
  // e1a
  k_mask<<<ew(v0 * 16), 256, 0, st>>>(U->g0, nullptr, U->e1a, v0 * 16, U->dpre);
  wgrad(*U, 0, src(U->in16, 16, G_SAME, n0), none, st);
  if (lr > 0.0) {
    U->adam_step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)U->adam_step), c2 = 1.f - powf(b2, (float)U->adam_step);
    for (int l = 0; l < kNL; ++l) {
      Layer& y = U->L[l];
      const long nw = 27L * y.cin * y.cout;
      k_adam<<<ew(nw), 256, 0, st>>>(y.w, y.gw, y.mw, y.vw, nw, (float)lr, b1, b2, 1e-8f, c1, c2, 27, y.cout, y.cin,
                                     y.wf, y.wt, y.cin_real, y.cout_real);
      k_adam<<<1, 256, 0, st>>>(y.b, y.gb, y.mb, y.vb, y.cout, (float)lr, b1, b2, 1e-8f, c1, c2, 0, y.cout, 1,
                                nullptr, nullptr, 1, y.cout_real);
    }
  }
  cudaStreamSynchronize(st);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

float* unet_output(UNet* U) { return U->out32; }
int unet_N(const UNet* U) { return U->N; }
void unet_set_kernels(UNet* U, int tc) { U->use_tc = tc; }

#define INST(T)                                                                                         \
  template void unet_apply_sc<T>(UNet*, const T*, const T*, double*, int, double, cudaStream_t);         \
  template int unet_apply<T>(UNet*, const T*, const T*, double, double, float*, cudaStream_t);          \
  template int unet_train_step<T>(UNet*, const T*, const T*, const T*, double, double, double, double*, \
                                  cudaStream_t);
INST(double)
INST(float)

}  // namespace fe

namespace fe {
__global__ void k_bf16_to_f32(const bf16* a, long n, float* out) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    out[q] = __bfloat162float(a[q]);
}

// Activation of layer l (0..8; 9 = packed input) after the last forward pass,
// channels-last, as floats: count = n_l^3 * C_l.
int unet_activation(UNet* U, int l, float* host, long count, cudaStream_t st) {
  const int n0 = U->N, n1 = U->N / 2, n2 = U->N / 4;
  const bf16* p = nullptr;
  long n = 0;
  switch (l) {
    case 0: p = U->e1a; n = cube(n0) * 16; break;
    case 1: p = U->e1b; n = cube(n0) * 16; break;
    case 2: p = U->d1; n = cube(n1) * 32; break;
    case 3: p = U->e2; n = cube(n1) * 32; break;
    case 4: p = U->d2; n = cube(n2) * 64; break;
    case 5: p = U->e3; n = cube(n2) * 64; break;
    case 6: p = U->u2; n = cube(n1) * 32; break;
    case 7: p = U->u1; n = cube(n0) * 16; break;
    case 8:
      if (count != cube(n0)) return FE_ERR_INVALID_ARG;
      cudaMemcpyAsync(host, U->out32, cube(n0) * 4, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      return FE_OK;
    case 9: p = U->in16; n = cube(n0) * 16; break;
    default: return FE_ERR_INVALID_ARG;
  }
  if (count != n) return FE_ERR_INVALID_ARG;
  float* d = nullptr;
  if (cudaMalloc(&d, n * 4) != cudaSuccess) return FE_ERR_OOM;
  k_bf16_to_f32<<<ew(n), 256, 0, st>>>(p, n, d);
  cudaMemcpyAsync(host, d, n * 4, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFree(d);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
}  // namespace fe
