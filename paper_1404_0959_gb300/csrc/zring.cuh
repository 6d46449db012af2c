// zring.cuh -- z-marching with asynchronous copies into shared-memory rings.
//
// Same 32 x 8 column tiles and radius-2 halo geometry as zmarch.cuh (ZGeom<2>),
// but every streamed plane -- the z-neighbours included -- lives in a shared
// ring filled by cp.async (global -> shared without registers), A planes ahead
// of the plane being computed.  Three ring kinds:
//   stencil field  planes k-2 .. k+2 in use           (5 + A slots, tile + halo)
//   face array     planes k-1 .. k (own, x-1, y-1)    (2 + A slots, tile + halo)
//   centre field   plane k, own cells                  (1 + A slots, tile only)
// One group of copies per plane; before plane k a thread waits until its own
// copies of plane k (+2 for stencils) have landed, then one barrier makes
// all threads' copies visible and frees the slots of plane k - 3 for reuse.
#pragma once
#include "zbulk.cuh"
#include "zmarch.cuh"

namespace fe {

template <typename T>
__device__ __forceinline__ void cp_async(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int kZHW = ZGeom<2>::H * ZGeom<2>::W;  // tile + radius-2 halo, elements

// Plane m of a tile-with-halo field into a ring slot.
template <typename T>
__device__ __forceinline__ void zr_issue_halo(const ZGeom<2>& G, const T* g, T* slot, int m) {
  const int pl = G.plane(m);
  cp_async(slot + G.csm, g + G.col + pl);
  if (G.hcol >= 0) cp_async(slot + G.hsm, g + G.hcol + pl);
}
// Plane m of a centre-only field (own cells) into a ring slot.
template <typename T>
__device__ __forceinline__ void zr_issue_centre(const ZGeom<2>& G, const T* g, T* slot, int tid, int m) {
  cp_async(slot + tid, g + G.col + G.plane(m));
}

// Stencil view of one field at plane k: five ring slots k-2 .. k+2.
template <typename T>
struct ZView {
  const T* p[5];
  int csm;
  __device__ __forceinline__ T at(const ZGeom<2>&, int d, int s) const {
    if (d == 2) return p[2 + s][csm];
    return d == 0 ? p[2][csm + s] : p[2][csm + s * ZGeom<2>::W];
  }
  __device__ __forceinline__ T c() const { return p[2][csm]; }
};
// Sum of two stencil views (a + b per cell, the same rounding as staging the sum).
template <typename T>
struct ZView2 {
  ZView<T> a, b;
  __device__ __forceinline__ T at(const ZGeom<2>& G, int d, int s) const { return a.at(G, d, s) + b.at(G, d, s); }
  __device__ __forceinline__ T c() const { return a.c() + b.c(); }
};

// Ring slot bookkeeping of one tile: stencil slots (5 + A), face slots (2 + A),
// centre slots (1 + A), indexed from the tile's first plane k0.
template <int A>
struct ZSlots {
  static constexpr int NS = 5 + A, NF = 2 + A, NC = 1 + A;
  int k0;
  __device__ __forceinline__ int s(int m) const { return (m - k0 + 2) % NS; }  // stencil plane m
  __device__ __forceinline__ int f(int m) const { return (m - k0 + 1) % NF; }  // face plane m
  __device__ __forceinline__ int c(int m) const { return (m - k0) % NC; }      // centre plane m
};

// Ring plan of one kernel: NSF stencil fields, NFF face arrays, NCF centre
// fields, A planes of lookahead.  Global pointers are set by the kernel
// (gs/gf/gc); smem is carved from the dynamic shared allocation.
template <typename T, int A, int NSF, int NFF, int NCF>
struct RingPlan {
  using SL = ZSlots<A>;
  static constexpr int elems = NSF * SL::NS * kZHW + NFF * SL::NF * kZHW + NCF * SL::NC * NTHR;
  static constexpr int bytes = (elems > 0 ? elems : 1) * (int)sizeof(T);
  T* rs;
  T* rf;
  T* rc;
  const T* gs[NSF > 0 ? NSF : 1];
  const T* gf[NFF > 0 ? NFF : 1];
  const T* gc[NCF > 0 ? NCF : 1];
  SL sl;
  int k0, kend;
  int ncf = NCF;  // centre fields copied (the first ncf of gc)
  __device__ __forceinline__ void init(unsigned char* smem, int k0_, int kend_) {
    rs = reinterpret_cast<T*>(smem);
    rf = rs + NSF * SL::NS * kZHW;
    rc = rf + NFF * SL::NF * kZHW;
    k0 = k0_;
    kend = kend_;
    sl.k0 = k0_;
  }
  __device__ __forceinline__ void stencil_plane(const ZGeom<2>& G, int m) {
    const int w = G.wrapz(m);
#pragma unroll
    for (int f = 0; f < NSF; ++f) zr_issue_halo(G, gs[f], rs + (f * SL::NS + sl.s(m)) * kZHW, w);
  }
  __device__ __forceinline__ void face_plane(const ZGeom<2>& G, int m) {
    const int w = G.wrapz(m);
#pragma unroll
    for (int f = 0; f < NFF; ++f) zr_issue_halo(G, gf[f], rf + (f * SL::NF + sl.f(m)) * kZHW, w);
  }
  __device__ __forceinline__ void centre_plane(const ZGeom<2>& G, int tid, int m) {
#pragma unroll
    for (int f = 0; f < NCF; ++f)
      if (f < ncf) zr_issue_centre(G, gc[f], rc + (f * SL::NC + sl.c(m)) * NTHR, tid, m);
  }
  // group q >= 1: stencil plane k0+2+q, face and centre planes k0+q (skipped beyond the tile)
  __device__ __forceinline__ void issue(const ZGeom<2>& G, int tid, int q) {
    if (k0 + 2 + q <= kend + 1) stencil_plane(G, k0 + 2 + q);
    if (k0 + q < kend) {
      face_plane(G, k0 + q);
      centre_plane(G, tid, k0 + q);
    }
  }
  // group 0 (stencil k0-2..k0+2, faces k0-1..k0, centre k0) and groups 1..A-1
  __device__ __forceinline__ void prologue(const ZGeom<2>& G, int tid) {
    for (int m = k0 - 2; m <= k0 + 2; ++m) stencil_plane(G, m);
    face_plane(G, k0 - 1);
    face_plane(G, k0);
    centre_plane(G, tid, k0);
    cp_async_commit();
#pragma unroll
    for (int q = 1; q < A; ++q) {
      issue(G, tid, q);
      cp_async_commit();
    }
  }
  // before plane k = k0 + i: wait for its copies, make them visible, start plane group A + i
  __device__ __forceinline__ void next(const ZGeom<2>& G, int tid, int i) {
    cp_async_wait<A - 1>();
    __syncthreads();
    issue(G, tid, A + i);
    cp_async_commit();
  }
  __device__ __forceinline__ ZView<T> view(int f, int k, const ZGeom<2>& G) const {
    ZView<T> v;
    v.csm = G.csm;
#pragma unroll
    for (int j = 0; j < 5; ++j) v.p[j] = rs + (f * SL::NS + sl.s(k - 2 + j)) * kZHW;
    return v;
  }
  // faces f0, f0+1, f0+2 (x, y, z arrays): values at the +1/2 and -1/2 faces of the cell
  __device__ __forceinline__ void faces(int f0, int k, const ZGeom<2>& G, T (&plus)[3], T (&minus)[3]) const {
    const T* fx = rf + (f0 * SL::NF + sl.f(k)) * kZHW;
    const T* fy = rf + ((f0 + 1) * SL::NF + sl.f(k)) * kZHW;
    const T* fz = rf + ((f0 + 2) * SL::NF + sl.f(k)) * kZHW;
    const T* fzm = rf + ((f0 + 2) * SL::NF + sl.f(k - 1)) * kZHW;
    plus[0] = fx[G.csm];
    minus[0] = fx[G.csm - 1];
    plus[1] = fy[G.csm];
    minus[1] = fy[G.csm - ZGeom<2>::W];
    plus[2] = fz[G.csm];
    minus[2] = fzm[G.csm];
  }
  __device__ __forceinline__ T cen(int f, int k, int tid) const { return rc[(f * SL::NC + sl.c(k)) * NTHR + tid]; }
};

}  // namespace fe
