// zmarch.cuh -- z-marching star-stencil machinery for the step kernels.
//
// A 32 x 8 thread block owns a 32 x 8 column tile and walks tz z-planes.  For
// every field read with a star stencil of radius R (offsets along one axis at
// a time) each thread keeps its column's values at z-offsets -R..R in a
// register queue (one new global load per plane), and the block stages the
// current plane of the field with an R-wide x/y halo in shared memory (one
// interior store per thread plus (4 R TY + 4 R TX) / (TX TY) halo loads per
// cell).  The tile is "wrapped": thread columns beyond the box edge hold the
// periodic continuation, so ragged tiles and N < 32 need no special cases;
// only threads inside the box store results.
#pragma once
#include "fe_internal.cuh"

namespace fe {

template <int R>
struct ZGeom {
  static constexpr int W = TX + 2 * R, H = TY + 2 * R;
  int N, NN;
  int col;         // flat (x, y) index of this thread's column
  int csm;         // its smem position
  int hcol, hsm;   // halo cell this thread stages (hcol < 0: none)
  bool active;     // column inside the box
  __device__ __forceinline__ ZGeom(int x0, int y0, int N_) {
    N = N_;
    NN = N * N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
    const int gx = (x0 + tx) % N, gy = (y0 + ty) % N;
    active = (x0 + tx < N) && (y0 + ty < N);
    col = gx + N * gy;
    csm = (ty + R) * W + tx + R;
    hcol = -1;
    hsm = 0;
    int lx = 0, ly = 0;
    if (tid < 2 * R * TY) {  // x halo: 2R cells on each of TY rows
      const int row = tid / (2 * R), k = tid % (2 * R);
      lx = k < R ? k - R : TX + (k - R);
      ly = row;
      hcol = 0;
    } else if (tid < 2 * R * TY + 2 * R * TX) {  // y halo: 2R rows of TX cells
      const int q = tid - 2 * R * TY;
      const int rowi = q / TX, cx = q % TX;
      lx = cx;
      ly = rowi < R ? rowi - R : TY + (rowi - R);
      hcol = 0;
    }
    if (hcol == 0) {
      const int hx = ((x0 + lx) % N + N) % N, hy = ((y0 + ly) % N + N) % N;
      hcol = hx + N * hy;
      hsm = (ly + R) * W + lx + R;
    }
  }
  __device__ __forceinline__ int plane(int k) const { return NN * k; }
  __device__ __forceinline__ int wrapz(int k) const { return k < 0 ? k + N : (k >= N ? k - N : k); }
};

// One field read with a radius-R star stencil.  Loads run PF planes ahead:
// the z-queue values and the halo values needed at planes k + 1 .. k + PF are
// in flight while plane k is computed.
template <typename T, int R, int PF = 1>
struct ZField {
  const T* __restrict__ g;
  T q[2 * R + 1];  // q[R + s] = value at z-offset s of the current plane
  T nq[PF];        // pending queue entries (planes k + R + 1 .. k + R + PF)
  T nh[PF];        // pending halo values (planes k + 1 .. k + PF)
  T* sm;           // shared plane (H x W)
  __device__ __forceinline__ void init(const T* gp, T* smem, const ZGeom<R>& G, int k0) {
    g = gp;
    sm = smem;
#pragma unroll
    for (int s = -R; s < R; ++s) q[R + s + 1] = __ldg(&g[G.col + G.plane(G.wrapz(k0 + s))]);
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      nq[j] = __ldg(&g[G.col + G.plane(G.wrapz(k0 + R + j))]);
      nh[j] = G.hcol >= 0 ? __ldg(&g[G.hcol + G.plane(G.wrapz(k0 + j))]) : T{};
    }
  }
  // move to plane k: shift the queue in, request plane k + R + PF
  __device__ __forceinline__ void advance(const ZGeom<R>& G, int k) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) q[s] = q[s + 1];
    q[2 * R] = nq[0];
#pragma unroll
    for (int j = 0; j + 1 < PF; ++j) nq[j] = nq[j + 1];
    nq[PF - 1] = __ldg(&g[G.col + G.plane(G.wrapz(k + R + PF))]);
  }
  // stage the current plane (call between two __syncthreads), request halo plane k + PF
  __device__ __forceinline__ void stage(const ZGeom<R>& G, int k) {
    sm[G.csm] = q[R];
    if (G.hcol >= 0) {
      sm[G.hsm] = nh[0];
#pragma unroll
      for (int j = 0; j + 1 < PF; ++j) nh[j] = nh[j + 1];
      nh[PF - 1] = __ldg(&g[G.hcol + G.plane(G.wrapz(k + PF))]);
    }
  }
  // value at offset s along axis d from this thread's cell
  __device__ __forceinline__ T at(const ZGeom<R>& G, int d, int s) const {
    if (d == 2) return q[R + s];
    return d == 0 ? sm[G.csm + s] : sm[G.csm + s * ZGeom<R>::W];
  }
  __device__ __forceinline__ T c() const { return q[R]; }
};

// A field read at this thread's own cell only, PF planes ahead.
template <typename T, int PF>
struct ZStream {
  const T* __restrict__ g;
  T v[PF];  // planes k .. k + PF - 1
  template <int R>
  __device__ __forceinline__ void init(const T* gp, const ZGeom<R>& G, int k0) {
    g = gp;
#pragma unroll
    for (int j = 0; j < PF; ++j) v[j] = __ldg(&g[G.col + G.plane(G.wrapz(k0 + j))]);
  }
  // value at plane k; requests plane k + PF
  template <int R>
  __device__ __forceinline__ T next(const ZGeom<R>& G, int k) {
    const T out = v[0];
#pragma unroll
    for (int j = 0; j + 1 < PF; ++j) v[j] = v[j + 1];
    v[PF - 1] = __ldg(&g[G.col + G.plane(G.wrapz(k + PF))]);
    return out;
  }
};

// Tile origin of this block's (box, tile) work item.
struct TileXYZ {
  int box, x0, y0, k0, kend;
};
__device__ __forceinline__ TileXYZ tile_xyz(const BoxDev* boxes, const int2* work) {
  const int2 w = work[blockIdx.x];
  const BoxDev& B = boxes[w.x];
  TileXYZ t;
  t.box = w.x;
  const int tx = w.y % B.tnx, r = w.y / B.tnx, ty = r % B.tny, tzb = r / B.tny;
  t.x0 = tx * TX;
  t.y0 = ty * TY;
  t.k0 = tzb * B.tz;
  t.kend = min(t.k0 + B.tz, B.N);
  return t;
}

// ---- star stencils on a staged field (same arithmetic as the global-memory helpers) ----
// FV: any view with at(G, d, s) and c() (ZField, ZView, ZView2).
template <typename FV, typename GT>
__device__ __forceinline__ auto zI4(const FV& f, const GT& G, int d, int o) -> decltype(f.c()) {
  using T = decltype(f.c());
  return (T(9) * (f.at(G, d, o) + f.at(G, d, o + 1)) - (f.at(G, d, o - 1) + f.at(G, d, o + 2))) * T(0.0625);
}
template <typename FV, typename GT>
__device__ __forceinline__ auto zGc_h(const FV& f, const GT& G, int d) -> decltype(f.c()) {
  using T = decltype(f.c());
  return (T(10) * (f.at(G, d, 1) - f.at(G, d, -1)) - (f.at(G, d, 2) - f.at(G, d, -2))) * T(0.0625);
}
template <typename FV, typename GT>
__device__ __forceinline__ auto zDG4_h2(const FV& f, const GT& G, int d) -> decltype(f.c()) {
  using T = decltype(f.c());
  return (T(28) * (f.at(G, d, -1) + f.at(G, d, 1)) - T(54) * f.c() - (f.at(G, d, -2) + f.at(G, d, 2))) *
         T(1.0 / 24.0);
}

// L_m = -D(phi I4 u_m) + mu (sum_d D G4_d u_m + Gc_m(div)/3), and the viscous part
template <typename T, typename FV, typename GT>
__device__ __forceinline__ void zeval_L(const FV (&u)[3], const FV& div, const T (&php)[3], const T (&phm)[3],
                                        const GT& G, T ih, T mu, T (&L)[3], T (&visc)[3]) {
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    T conv = T(0), lap = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      conv += php[d] * zI4(u[m], G, d, 0) - phm[d] * zI4(u[m], G, d, -1);
      lap += zDG4_h2(u[m], G, d);
    }
    visc[m] = mu * (lap * ih * ih + zGc_h(div, G, m) * ih * T(1.0 / 3.0));
    L[m] = visc[m] - conv * ih;
  }
}

}  // namespace fe
