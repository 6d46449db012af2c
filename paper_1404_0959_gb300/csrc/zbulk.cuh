// zbulk.cuh -- plane streaming through the bulk-copy (TMA) engine.
//
// A block owns "row groups" of R = kBulkCells / N full x-rows (four
// consecutive x-cells per thread and row it handles) and walks a contiguous
// range of (row group, z-plane) pairs in group-major order, so every block of
// a persistent grid gets the same number of planes (+-1).  Each plane of each
// streamed field arrives in shared memory by cp.async.bulk: the R rows of the
// group are one contiguous run of memory, and the y-halo rows above and below
// (periodic wrap) are one row each, so no tensor map is needed and the x
// direction is complete in every row (x-neighbours wrap inside the row).
// Completion is tracked by one mbarrier per ring stage (expect-tx bytes); one
// thread issues the copies S - 1 planes ahead of the plane being computed.
//
// Raw plane sequence of one segment (row group g, output planes k0..k0+len-1):
// k0-1, k0, ..., k0+len (the z-halo planes at both ends are read too).
#pragma once
#include "fe_internal.cuh"

namespace fe {

// ---- PTX wrappers ----------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy completing on `bar` (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after `cap` polls (each try_wait itself blocks for a
// hardware-defined time slice), so a lost copy cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int cap = 1 << 22) {
  for (int i = 0; i < cap; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---- geometry and plane sequence ------------------------------------------------
// A block of kBulkThreads threads covers kBulkCells cells of each plane:
// kBulkRows rows of four x-consecutive cells per thread.
#ifndef FE_BULK_THREADS
#define FE_BULK_THREADS 256
#endif
constexpr int kBulkThreads = FE_BULK_THREADS;
// Two block sizes: kBulkCells for the Jacobi iteration (its stage of five
// streams), kBulkCellsPoly for the polynomial iteration where the box edge
// lets a group of that many cells fit (fewer, larger plane steps).
#ifndef FE_BULK_CELLS
#define FE_BULK_CELLS 2048
#endif
#ifndef FE_BULK_CELLS_POLY
#define FE_BULK_CELLS_POLY 4096
#endif
constexpr int kBulkCells = FE_BULK_CELLS;
constexpr int kBulkCellsPoly = FE_BULK_CELLS_POLY;
// rows of four cells per thread for a block of `cells` cells per plane
template <int CELLS>
__host__ __device__ constexpr int bulk_rows() {
  return CELLS / (4 * kBulkThreads);
}
static_assert(bulk_rows<kBulkCells>() >= 1 && 4 * kBulkThreads * bulk_rows<kBulkCells>() == kBulkCells,
              "bulk block shape");
static_assert(bulk_rows<kBulkCellsPoly>() >= 1 && 4 * kBulkThreads * bulk_rows<kBulkCellsPoly>() == kBulkCellsPoly,
              "bulk block shape (polynomial iteration)");

struct BulkGeom {
  int N, R, G, Q;  // box edge, rows per group, row groups, threads per row (N / 4)
  int lgN;         // log2 N (streamed boxes have power-of-two edges)
  int a, b;        // this block's range of (group, plane) pairs, group-major
  __device__ __forceinline__ BulkGeom(int N_, int blk, int nblk, int cells) {
    N = N_;
    lgN = __ffs(N) - 1;
    R = cells / N;
    G = N / R;
    Q = N / 4;
    const long tot = (long)G * N;
    a = (int)(tot * blk / nblk);
    b = (int)(tot * (blk + 1) / nblk);
  }
  // raw planes of this block's sequence
  __device__ __forceinline__ int count() const {
    if (b <= a) return 0;
    const int g0 = a / N, g1 = (b - 1) / N;
    return (b - a) + 2 * (g1 - g0 + 1);
  }
};

// Position i of the raw sequence: row group g, plane m (wrapped), position in
// its segment pos (0 = lower z-halo plane, len + 1 = upper one) and the
// segment's output-plane count len.
struct BulkPos {
  int g, m, pos, len;
};
__device__ __forceinline__ BulkPos bulk_pos(const BulkGeom& Gm, int i) {
  int s = Gm.a;
  while (true) {
    const int g = s >> Gm.lgN, k0 = s & (Gm.N - 1);
    const int e = min(Gm.b, (g + 1) * Gm.N);
    const int len = e - s;
    if (i < len + 2) {
      int m = k0 - 1 + i;
      m += m < 0 ? Gm.N : 0;
      m -= m >= Gm.N ? Gm.N : 0;
      return BulkPos{g, m, i, len};
    }
    i -= len + 2;
    s = e;
  }
}

}  // namespace fe
