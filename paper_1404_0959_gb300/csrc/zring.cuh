// zring.cuh -- z-marching with asynchronous copies into shared-memory rings.
//
// A block of 16 x 8 threads owns a 32 x 8 column tile and walks its z-planes;
// each thread computes the two x-neighbouring cells (x, x+1) of its column
// pair, so every shared-memory read, copy, slot computation and loop step
// serves two cells, and the x-neighbours of both cells come from three
// 8-byte (16-byte in FP64) pair reads.  Every streamed plane lives in a
// shared ring filled by 16-byte cp.async chunks (global -> shared without
// registers), A planes ahead of the plane being computed.  Three ring kinds:
//   stencil field  planes k .. k+2 in use               (3 + A slots, tile + halo)
//   face array     planes k-1 .. k (own, x-1, y-1)      (2 + A slots, tile + halo)
//   centre field   plane k, own cells                    (1 + A slots, tile only)
// The z-neighbours of a stencil field come from a per-thread register queue
// (planes k-2 .. k+2 of the own column pair): each plane is read from shared
// memory once for the queue, when it is two planes ahead, and once per x/y
// neighbour while it is the current plane.  One group of copies per plane;
// before plane k a thread waits until its own copies of plane k (+2 for
// stencils) have landed, then one barrier makes all threads' copies visible
// and frees the slots of plane k - 1 for reuse.
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

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Threads of a ring block: 16 column pairs x 8 rows.
constexpr int RTX = TX / 2, RNT = RTX * TY;

// Two neighbouring cells of one field (x, x+1).
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
template <typename T>
using P2 = typename Pair<T>::type;
template <typename T>
__device__ __forceinline__ T pc(const P2<T>& v, int r) {
  return r ? v.y : v.x;
}
template <typename T>
__device__ __forceinline__ P2<T> ldp(const T* p) {
  return *reinterpret_cast<const P2<T>*>(p);
}
// the same from global memory through the read-only path
template <typename T>
__device__ __forceinline__ P2<T> ldg2(const T* p) {
  return __ldg(reinterpret_cast<const P2<T>*>(p));
}
template <typename T>
__device__ __forceinline__ void stp(T* p, T a, T b) {
  P2<T> v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<P2<T>*>(p) = v;
}

// Tile geometry of the ring kernels: 32 x 8 columns, y-halo 2, x-halo XH (2
// cells rounded up to one 16-byte chunk), copied in 16-byte chunks: at most
// two chunks per thread and field for the tile with its star halo (corners
// are not needed), at most one per thread for a centre-only plane.  Needs
// N % CE == 0 so no chunk straddles the periodic seam (and N even, so a
// column pair is inside the box or outside it as a whole); wrapped columns
// beyond a ragged box edge hold the periodic continuation as in ZGeom.
template <typename T>
struct RGeom {
  static constexpr int CE = 16 / (int)sizeof(T);  // cells per chunk
  static constexpr int XH = CE > 2 ? CE : 2;      // x-halo
  static constexpr int W = TX + 2 * XH, H = TY + 4, HW = H * W;
  static constexpr int ROWC = W / CE, MIDC = TX / CE;
  static constexpr int NCH = TY * ROWC + 4 * MIDC;  // chunks of a tile-with-halo plane
  static constexpr int NCC = TX * TY / CE;          // chunks of a centre plane
  static_assert(NCH <= 2 * RNT && NCC <= RNT, "two halo chunks and one centre chunk per thread");
  int N, NN, col, csm;
  bool active;
  int ch_g[2], ch_s[2];  // this thread's halo-plane chunks: global column (-1: none), shared offset
  int cc_g, cc_s;        // this thread's centre-plane chunk
  __device__ __forceinline__ static int wrap(int v, int n) { return ((v % n) + n) % n; }
  __device__ __forceinline__ RGeom(int x0, int y0, int N_) {
    N = N_;
    NN = N * N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + RTX * ty;
    active = (x0 + 2 * tx < N) && (y0 + ty < N);
    col = wrap(x0 + 2 * tx, N) + N * wrap(y0 + ty, N);
    csm = (ty + 2) * W + 2 * tx + XH;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int ch = tid + j * RNT;
      ch_g[j] = -1;
      ch_s[j] = 0;
      if (ch < NCH) {
        int lx, ly;
        if (ch < TY * ROWC) {
          ly = ch / ROWC;
          lx = (ch % ROWC) * CE - XH;
        } else {
          const int h = ch - TY * ROWC, hr = h / MIDC;
          ly = hr < 2 ? hr - 2 : TY + hr - 2;
          lx = (h % MIDC) * CE;
        }
        ch_g[j] = wrap(x0 + lx, N) + N * wrap(y0 + ly, N);
        ch_s[j] = (ly + 2) * W + lx + XH;
      }
    }
    cc_g = -1;
    cc_s = 0;
    if (tid < NCC) {
      const int row = tid / (TX / CE), x = (tid % (TX / CE)) * CE;
      cc_g = wrap(x0 + x, N) + N * wrap(y0 + row, N);
      cc_s = row * TX + x;
    }
  }
  __device__ __forceinline__ int plane(int k) const { return NN * k; }
  __device__ __forceinline__ int wrapz(int k) const { return k < 0 ? k + N : (k >= N ? k - N : k); }
};

// Plane m of a tile-with-halo field / of a centre-only field into a ring slot.
template <typename T>
__device__ __forceinline__ void zr_issue_halo(const RGeom<T>& G, const T* g, T* slot, int m) {
#pragma unroll
  for (int j = 0; j < 2; ++j)
    if (G.ch_g[j] >= 0) cp_async16(slot + G.ch_s[j], g + G.ch_g[j] + G.plane(m));
}
template <typename T>
__device__ __forceinline__ void zr_issue_centre(const RGeom<T>& G, const T* g, T* slot, int m) {
  if (G.cc_g >= 0) cp_async16(slot + G.cc_s, g + G.cc_g + G.plane(m));
}

// Stencil view of one field at plane k for cell r (0: x, 1: x+1) of the
// thread's pair: the current ring slot (x/y neighbours, read as pairs) and the
// register queue (z-neighbours and the cell itself).
template <typename T>
struct ZView {
  const T* p;
  P2<T> z[5];  // own column pair, planes k-2 .. k+2
  int csm, r;
  template <typename GT>
  __device__ __forceinline__ T at(const GT&, int d, int s) const {
    if (d == 2) return pc<T>(z[2 + s], r);
    if (d == 1) return pc<T>(ldp(p + csm + s * RGeom<T>::W), r);
    const int o = r + s;  // -2 .. 3: pair (o >> 1), component (o & 1)
    return pc<T>(ldp(p + csm + 2 * (o >> 1)), o & 1);
  }
  __device__ __forceinline__ T c() const { return pc<T>(z[2], r); }
};
// Sum of two stencil views (a + b per cell, the same rounding as staging the sum).
template <typename T>
struct ZView2 {
  ZView<T> a, b;
  template <typename GT>
  __device__ __forceinline__ T at(const GT& G, int d, int s) const { return a.at(G, d, s) + b.at(G, d, s); }
  __device__ __forceinline__ T c() const { return a.c() + b.c(); }
};

// Ring slot bookkeeping of one tile: stencil slots (3 + A, from plane k0),
// face slots (2 + A, from plane k0 - 1), centre slots (1 + A, from plane k0).
template <int A>
struct ZSlots {
  static constexpr int NS = 3 + A, NF = 2 + A, NC = 1 + A;
  int k0;
  __device__ __forceinline__ int s(int m) const { return (m - k0) % NS; }      // stencil plane m
  __device__ __forceinline__ int f(int m) const { return (m - k0 + 1) % NF; }  // face plane m
  __device__ __forceinline__ int c(int m) const { return (m - k0) % NC; }      // centre plane m
};

// Ring plan of one kernel: NSF stencil fields, NFF face arrays, NCF centre
// fields, A planes of lookahead.  Global pointers are set by the kernel
// (gs/gf/gc); smem is carved from the dynamic shared allocation.
template <typename T, int A, int NSF, int NFF, int NCF>
struct RingPlan {
  using SL = ZSlots<A>;
  using G_ = RGeom<T>;
  static constexpr int HW = G_::HW;
  static constexpr int elems = NSF * SL::NS * HW + NFF * SL::NF * HW + NCF * SL::NC * NTHR;
  static constexpr int bytes = (elems > 0 ? elems : 1) * (int)sizeof(T);
  T* rs;
  T* rf;
  T* rc;
  const T* gs[NSF > 0 ? NSF : 1];
  const T* gf[NFF > 0 ? NFF : 1];
  const T* gc[NCF > 0 ? NCF : 1];
  P2<T> zq[NSF > 0 ? NSF : 1][5];  // z-queues of the stencil fields (own pair, planes k-2 .. k+2)
  SL sl;
  int k0, kend;
  int ncf = NCF;  // centre fields copied (the first ncf of gc)
  __device__ __forceinline__ void init(unsigned char* smem, int k0_, int kend_) {
    rs = reinterpret_cast<T*>(smem);
    rf = rs + NSF * SL::NS * HW;
    rc = rf + NFF * SL::NF * HW;
    k0 = k0_;
    kend = kend_;
    sl.k0 = k0_;
  }
  __device__ __forceinline__ const T* sslot(int f, int m) const { return rs + (f * SL::NS + sl.s(m)) * HW; }
  __device__ __forceinline__ void stencil_plane(const G_& G, int m) {
    const int w = G.wrapz(m);
#pragma unroll
    for (int f = 0; f < NSF; ++f) zr_issue_halo(G, gs[f], rs + (f * SL::NS + sl.s(m)) * HW, w);
  }
  __device__ __forceinline__ void face_plane(const G_& G, int m) {
    const int w = G.wrapz(m);
#pragma unroll
    for (int f = 0; f < NFF; ++f) zr_issue_halo(G, gf[f], rf + (f * SL::NF + sl.f(m)) * HW, w);
  }
  __device__ __forceinline__ void centre_plane(const G_& G, int m) {
#pragma unroll
    for (int f = 0; f < NCF; ++f)
      if (f < ncf) zr_issue_centre(G, gc[f], rc + (f * SL::NC + sl.c(m)) * NTHR, m);
  }
  // group q >= 1: stencil plane k0+2+q, face and centre planes k0+q (skipped beyond the tile)
  __device__ __forceinline__ void issue(const G_& G, int q) {
    if (k0 + 2 + q <= kend + 1) stencil_plane(G, k0 + 2 + q);
    if (k0 + q < kend) {
      face_plane(G, k0 + q);
      centre_plane(G, k0 + q);
    }
  }
  // group 0 (stencil k0..k0+2, faces k0-1..k0, centre k0) and groups 1..A-1;
  // the queue entries below the tile (planes k0-2, k0-1) straight from global memory
  __device__ __forceinline__ void prologue(const G_& G) {
    for (int m = k0; m <= k0 + 2; ++m) stencil_plane(G, m);
    face_plane(G, k0 - 1);
    face_plane(G, k0);
    centre_plane(G, k0);
    cp_async_commit();
#pragma unroll
    for (int q = 1; q < A; ++q) {
      issue(G, q);
      cp_async_commit();
    }
    const int m2 = G.plane(G.wrapz(k0 - 2)), m1 = G.plane(G.wrapz(k0 - 1));
#pragma unroll
    for (int f = 0; f < NSF; ++f) {
      zq[f][0] = ldp(gs[f] + G.col + m2);
      zq[f][1] = ldp(gs[f] + G.col + m1);
    }
  }
  // before plane k = k0 + i: wait for its copies, make them visible, start plane group
  // A + i, and move the z-queues to plane k (plane k+2 read from its slot)
  __device__ __forceinline__ void next(const G_& G, int i) {
    cp_async_wait<A - 1>();
    __syncthreads();
    issue(G, A + i);
    cp_async_commit();
    const int k = k0 + i;
    if (i == 0) {
#pragma unroll
      for (int f = 0; f < NSF; ++f) {
        zq[f][2] = ldp(sslot(f, k) + G.csm);
        zq[f][3] = ldp(sslot(f, k + 1) + G.csm);
      }
    } else {
#pragma unroll
      for (int f = 0; f < NSF; ++f) {
#pragma unroll
        for (int j = 0; j < 4; ++j) zq[f][j] = zq[f][j + 1];
      }
    }
#pragma unroll
    for (int f = 0; f < NSF; ++f) zq[f][4] = ldp(sslot(f, k + 2) + G.csm);
  }
  __device__ __forceinline__ ZView<T> view(int f, int k, const G_& G, int r) const {
    ZView<T> v;
    v.csm = G.csm;
    v.r = r;
    v.p = sslot(f, k);
#pragma unroll
    for (int j = 0; j < 5; ++j) v.z[j] = zq[f][j];
    return v;
  }
  // faces f0, f0+1, f0+2 (x, y, z arrays) of cell r: values at its +1/2 and -1/2 faces
  __device__ __forceinline__ void faces(int f0, int k, const G_& G, int r, T (&plus)[3], T (&minus)[3]) const {
    const T* fx = rf + (f0 * SL::NF + sl.f(k)) * HW;
    const T* fy = rf + ((f0 + 1) * SL::NF + sl.f(k)) * HW;
    const T* fz = rf + ((f0 + 2) * SL::NF + sl.f(k)) * HW;
    const T* fzm = rf + ((f0 + 2) * SL::NF + sl.f(k - 1)) * HW;
    const P2<T> xc = ldp(fx + G.csm), xl = ldp(fx + G.csm - 2);
    plus[0] = pc<T>(xc, r);
    minus[0] = r ? xc.x : xl.y;
    plus[1] = pc<T>(ldp(fy + G.csm), r);
    minus[1] = pc<T>(ldp(fy + G.csm - G_::W), r);
    plus[2] = pc<T>(ldp(fz + G.csm), r);
    minus[2] = pc<T>(ldp(fzm + G.csm), r);
  }
  // the same for both cells at once: plus[d][r], minus[d][r]
  __device__ __forceinline__ void faces2(int f0, int k, const G_& G, T (&plus)[3][2], T (&minus)[3][2]) const {
    const T* fx = rf + (f0 * SL::NF + sl.f(k)) * HW;
    const T* fy = rf + ((f0 + 1) * SL::NF + sl.f(k)) * HW;
    const T* fz = rf + ((f0 + 2) * SL::NF + sl.f(k)) * HW;
    const T* fzm = rf + ((f0 + 2) * SL::NF + sl.f(k - 1)) * HW;
    const P2<T> xc = ldp(fx + G.csm), xl = ldp(fx + G.csm - 2);
    const P2<T> yc = ldp(fy + G.csm), yl = ldp(fy + G.csm - G_::W);
    const P2<T> zc = ldp(fz + G.csm), zl = ldp(fzm + G.csm);
    plus[0][0] = xc.x, plus[0][1] = xc.y, minus[0][0] = xl.y, minus[0][1] = xc.x;
    plus[1][0] = yc.x, plus[1][1] = yc.y, minus[1][0] = yl.x, minus[1][1] = yl.y;
    plus[2][0] = zc.x, plus[2][1] = zc.y, minus[2][0] = zl.x, minus[2][1] = zl.y;
  }
  // centre field f at plane k, both cells of the pair
  __device__ __forceinline__ P2<T> cen(int f, int k, int tid) const {
    return ldp(rc + (f * SL::NC + sl.c(k)) * NTHR + 2 * tid);
  }
};

// The neighbours at distance 1 and 2 along axis d of both cells (index r) of the thread's pair, for
// stencil field f of a ring plan at plane k: two pair reads along x (the pairs left and right of the
// own one, which is the queue's centre), four along y, none along z (the queue).  Loading a line once
// and evaluating both cells from registers replaces the per-cell, per-stencil reads of ZView.
template <typename T>
struct Line2 {
  T m2[2], m1[2], p1[2], p2[2];
};
template <typename T, typename Plan>
__device__ __forceinline__ Line2<T> ring_line(const Plan& R, int f, int k, const RGeom<T>& G, int d) {
  Line2<T> L;
  const P2<T> c = R.zq[f][2];
  if (d == 2) {
    const P2<T> a = R.zq[f][0], b = R.zq[f][1], e = R.zq[f][3], g = R.zq[f][4];
    L.m2[0] = a.x, L.m2[1] = a.y, L.m1[0] = b.x, L.m1[1] = b.y;
    L.p1[0] = e.x, L.p1[1] = e.y, L.p2[0] = g.x, L.p2[1] = g.y;
    return L;
  }
  const T* p = R.sslot(f, k) + G.csm;
  if (d == 1) {
    constexpr int W = RGeom<T>::W;
    const P2<T> a = ldp(p - 2 * W), b = ldp(p - W), e = ldp(p + W), g = ldp(p + 2 * W);
    L.m2[0] = a.x, L.m2[1] = a.y, L.m1[0] = b.x, L.m1[1] = b.y;
    L.p1[0] = e.x, L.p1[1] = e.y, L.p2[0] = g.x, L.p2[1] = g.y;
    return L;
  }
  const P2<T> l = ldp(p - 2), r = ldp(p + 2);  // cells x-2, x-1 and x+2, x+3
  L.m2[0] = l.x, L.m1[0] = l.y, L.p1[0] = c.y, L.p2[0] = r.x;
  L.m2[1] = l.y, L.m1[1] = c.x, L.p1[1] = r.x, L.p2[1] = r.y;
  return L;
}
// Only the neighbours at distance 1 (m1, p1; m2, p2 left unset): two reads along x, two along y.
template <typename T, typename Plan>
__device__ __forceinline__ Line2<T> ring_line1(const Plan& R, int f, int k, const RGeom<T>& G, int d) {
  Line2<T> L;
  const P2<T> c = R.zq[f][2];
  if (d == 2) {
    const P2<T> b = R.zq[f][1], e = R.zq[f][3];
    L.m1[0] = b.x, L.m1[1] = b.y, L.p1[0] = e.x, L.p1[1] = e.y;
    return L;
  }
  const T* p = R.sslot(f, k) + G.csm;
  if (d == 1) {
    constexpr int W = RGeom<T>::W;
    const P2<T> b = ldp(p - W), e = ldp(p + W);
    L.m1[0] = b.x, L.m1[1] = b.y, L.p1[0] = e.x, L.p1[1] = e.y;
    return L;
  }
  const P2<T> l = ldp(p - 2), r = ldp(p + 2);
  L.m1[0] = l.y, L.p1[0] = c.y, L.m1[1] = c.x, L.p1[1] = r.x;
  return L;
}
// 16 x the fourth-order face values I4 at the +1/2 and -1/2 faces of cell r along a line (centre value c)
template <typename T>
__device__ __forceinline__ T i4p16(const Line2<T>& L, T c, int r) {
  return fma(T(9), c + L.p1[r], -(L.m1[r] + L.p2[r]));
}
template <typename T>
__device__ __forceinline__ T i4m16(const Line2<T>& L, T c, int r) {
  return fma(T(9), L.m1[r] + c, -(L.m2[r] + L.p1[r]));
}
// 16 h x the centred fourth-order derivative Gc of cell r along a line
template <typename T>
__device__ __forceinline__ T gc16(const Line2<T>& L, int r) {
  return fma(T(10), L.p1[r] - L.m1[r], -(L.p2[r] - L.m2[r]));
}

}  // namespace fe
