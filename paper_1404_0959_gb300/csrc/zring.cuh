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

}  // namespace fe
