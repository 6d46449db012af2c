// unet_tc.cu -- 3x3x3 convolutions of the U-Net preconditioner on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Implicit GEMM: D[voxel][co] = sum_{tap, ci} A_tap[voxel][ci] W[tap][co][ci].
// A CTA computes tiles of kR = 4 output rows of 128 voxels (x-runs at fixed
// z, rows y0..y0+3).  For each 16-channel slice of the input it stages the
// (kR + 2) x 3 input rows the tile touches (periodic wrap; nearest upsampling
// of a half-resolution source is applied while staging) in shared memory in
// the no-swizzle K-major core-matrix layout
//   [8-channel half][voxel][8 channels]   (16 bytes per voxel and half)
// so the A operand of every tap is the staged row shifted by whole voxels
// (one descriptor, no im2col copy).  An input row feeds up to three output
// rows (dy = +1, 0, -1), so the weights of one (dz, dx) are stacked along N
// ([W(dy=+1); W(dy=0); W(dy=-1)], 3 Cout rows) and one MMA with N up to
// 3 Cout updates those three rows at once: measured on this part the cost
// of an M = 128, K = 16 MMA is set by reading A from shared memory and does
// not grow with N up to 128, so wider N means fewer MMAs per voxel.
// One elected thread issues the MMAs and commits to mbarriers that release
// the staging buffers and hand finished accumulators to the epilogue
// (tcgen05.ld, bias, ReLU, BF16 stores).  Staging uses cp.async (16-byte
// chunks; the gather wraps per chunk).
#include <cuda_bf16.h>

#include "zbulk.cuh"
#include "zring.cuh"

namespace fe {

typedef __nv_bfloat16 bf16;

struct TcConvArgs {
  const bf16* s0;  // source 0 (channels-last), channels c0, mode 0 = same grid, 1 = half grid (upsampled)
  const bf16* s1;
  int c0, c1, m0, m1;
  int No;          // output grid side (multiple of 128)
  const bf16* W;   // [27][Cout][Cin], Cin = c0 + c1
  const float* bias;
  bf16* out;       // [No^3][Cout] or null
  float* out32;    // [No^3] channel 0, or null
  int relu;
  int* err;        // set when a bounded wait gave up
};

namespace tc {

constexpr int kR = 4;                             // output rows per tile
constexpr int kRowVox = 130;                      // 128 + halo of 1 on each side
constexpr int kRowBytes = 2 * kRowVox * 16;       // two 8-channel halves
constexpr int kRows = (kR + 2) * 3;               // input rows: kR + 2 in y, 3 in z
constexpr int kInBytes = kRows * kRowBytes;       // input slice of one stage
constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  // no-swizzle shared-memory matrix descriptor: start, leading and stride byte
  // offsets in 16-byte units, descriptor version 1 (bits 46-47), layout 0
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[NC]);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t t, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(t));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t t, float (&v)[32]) {
  float a[16], b[16];
  tmem_ld<16>(t, a);
  tmem_ld<16>(t + 16, b);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = a[i];
    v[16 + i] = b[i];
  }
}
template <>
__device__ __forceinline__ void tmem_ld<64>(uint32_t t, float (&v)[64]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float a[16];
    tmem_ld<16>(t + 16 * q, a);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[16 * q + i] = a[i];
  }
}

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

}  // namespace tc

// Shared memory: [barriers 128 B][weights: resident all slices, or per stage][NS stages of input (+ weights)]
// [unused guard of FE_TC_GUARD bytes]
#ifndef FE_TC_GUARD
#define FE_TC_GUARD 0
#endif
template <int COUT, bool WRES, int NSTAGE>
struct TcPlan {
  static constexpr int NS = NSTAGE;
  static constexpr int wslice = 27 * COUT * 32;      // weights of one 16-channel slice (9 stacked blocks)
  static constexpr int wblock = 3 * COUT * 32;       // one (dz, dx) block: 3 Cout rows x K = 16
  static constexpr int zbytes = tc::kR * COUT * 32;  // zero B operand that clears an accumulator
  static constexpr int stage_bytes = tc::kInBytes + (WRES ? 0 : wslice);
  static int bytes(int cin) {
    return 128 + zbytes + (WRES ? (cin / 16) * wslice : 0) + NS * stage_bytes + FE_TC_GUARD;
  }
};

// offset of W[t][co][8 h .. 8 h + 7] of one slice in the stacked layout
template <int COUT>
__device__ __forceinline__ int wofs(int t, int co, int h) {
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int blk = (dz + 1) * 3 + (dx + 1), n = (1 - dy) * COUT + co;
  return blk * (3 * COUT * 32) + h * (3 * COUT * 16) + n * 16;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-specialised pipeline.  Warp 0 (one lane) issues the MMAs; warps 1-7
// stage input slices (cp.async, kLook steps ahead) and publish them on
// full[stage]; the MMA warp releases a stage with a tcgen05.commit on
// empty[stage] and hands a finished tile to the epilogue warps (4-7) on
// acc_full[buf]; they free the accumulator on acc_empty[buf].
template <int COUT, bool WRES, int NSTAGE>
__global__ void __launch_bounds__(tc::kThreads, 1) k_conv_tc(TcConvArgs a) {
  using P = TcPlan<COUT, WRES, NSTAGE>;
  constexpr int NS = P::NS, LOOK = NS - 1, NPROD = tc::kThreads - 32, NEPI = 128;
  extern __shared__ __align__(1024) unsigned char sm[];
  static_assert(NS >= 2 && NS <= 4, "2 to 4 stages");
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);  // NS (<= 4)
  uint64_t* empty = full + 4;                        // NS
  uint64_t* acc_full = full + 8;                     // 2
  uint64_t* acc_empty = full + 10;                   // 2
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + 96);
  int* abort_flag = reinterpret_cast<int*>(sm + 100);
  const int Cin = a.c0 + a.c1, nsl = Cin / 16;
  constexpr int R = tc::kR;
  unsigned char* zb = sm + 128;
  unsigned char* wres = zb + P::zbytes;
  unsigned char* stage0 = wres + (WRES ? nsl * P::wslice : 0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int No = a.No, nseg = No / 128;
  const long ntiles = (long)nseg * (No / R) * No;
  const long t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int ntile = (int)(t1 - t0), nsteps = ntile * nsl;
  constexpr int TCOLS = 2 * R * COUT;  // two tiles x kR rows x COUT fp32 columns (a power of two)
  static_assert((TCOLS & (TCOLS - 1)) == 0 && TCOLS >= 32 && TCOLS <= 512, "tensor memory columns");

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(full + q, NPROD);
      mbar_init(empty + q, 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(acc_full + q, 1);
      mbar_init(acc_empty + q, NEPI);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  for (int q = tid; q < P::zbytes / 16; q += tc::kThreads) reinterpret_cast<uint4*>(zb)[q] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  // tiles march in z for a fixed (x segment, row group): consecutive tiles of
  // a CTA share two of their three z-planes of input rows, so the re-reads hit L2
  auto tile_of = [&](int i, int& x0, int& y0, int& z) {
    const long t = t0 + i;
    z = (int)(t % No);
    const long r = t / No;
    x0 = 128 * (int)(r % nseg);
    y0 = R * (int)(r / nseg);
  };
  auto fail = [&]() { atomicExch(abort_flag, 1); };
  auto aborted = [&]() { return *(volatile int*)abort_flag != 0; };

  if (warp == 0) {
    // ---------------- MMA issuer (the warp waits together, lane 0 issues) ----------------
    constexpr uint32_t id1 = tc::idesc(128, COUT), id2 = tc::idesc(128, 2 * COUT), id3 = tc::idesc(128, 3 * COUT),
                       idz = tc::idesc(128, R * COUT);
    int s = 0;
    for (; s < nsteps; ++s) {
      const int i = s / nsl, sl = s % nsl;
      bool w = true;
      if (sl == 0 && i >= 2) w = mbar_wait(acc_empty + (i & 1), (unsigned)(((i - 2) >> 1) & 1));
      if (w) w = mbar_wait(full + (s % NS), (unsigned)((s / NS) & 1));
      if (!__all_sync(0xffffffffu, w && !aborted())) break;  // warp-uniform decision
      tc::fence_after();
      if (lane == 0) {
        const unsigned st = smem_u32(stage0 + (s % NS) * P::stage_bytes);
        const unsigned wb = WRES ? smem_u32(wres + sl * P::wslice) : st + tc::kInBytes;
        const uint64_t abase = tc::desc(st, tc::kRowVox * 16, 128), bbase = tc::desc(wb, 3 * COUT * 16, 128);
        const uint32_t d0 = tmem + (uint32_t)((i & 1) * R * COUT);
        if (sl == 0) tc::mma(d0, abase, tc::desc(smem_u32(zb), R * COUT * 16, 128), idz, 0);  // D = 0
#pragma unroll
        for (int yy = 0; yy < R + 2; ++yy)
#pragma unroll
          for (int zz = 0; zz < 3; ++zz)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              // output rows fed by input row yy: j = yy-2 .. yy (dy = +1, 0, -1) inside [0, R)
              const int jlo = yy - 2 < 0 ? 0 : yy - 2, jhi = yy > R - 1 ? R - 1 : yy;
              const int n = jhi - jlo + 1, dyi0 = jlo - (yy - 2);  // first stacked block row used
              const uint64_t aoff = (uint64_t)(((yy * 3 + zz) * tc::kRowBytes + dx * 16) >> 4);
              const uint64_t boff = (uint64_t)(((zz * 3 + dx) * (3 * COUT * 32) + dyi0 * COUT * 16) >> 4);
              const uint32_t dc = d0 + (uint32_t)(jlo * COUT);
              tc::mma(dc, abase + aoff, bbase + boff, n == 3 ? id3 : (n == 2 ? id2 : id1), 1);
            }
        tc::commit(empty + (s % NS));
        if (sl == nsl - 1) tc::commit(acc_full + (i & 1));
      }
      __syncwarp();
    }
    if (s < nsteps && lane == 0) fail();
    // every MMA issued has completed before the accumulator memory is released
    if (s > 0) mbar_wait(empty + ((s - 1) % NS), (unsigned)(((s - 1) / NS) & 1));
    __syncwarp();
  } else {
    // ---------------- producers (warps 1-7) and epilogue (warps 4-7) ----------------
    const int ptid = tid - 32;
    auto stage = [&](int s) {
      const int i = s / nsl, sl = s % nsl;
      int x0, y0, z;
      tile_of(i, x0, y0, z);
      unsigned char* st = stage0 + (s % NS) * P::stage_bytes;
      for (int q = ptid; q < tc::kRows * tc::kRowVox * 2; q += NPROD) {
        const int r = q / (tc::kRowVox * 2), rem = q - r * (tc::kRowVox * 2), v = rem >> 1, h = rem & 1;
        const int yy = tc::wrapc(y0 - 1 + r / 3, No), zz = tc::wrapc(z - 1 + r % 3, No),
                  xx = tc::wrapc(x0 - 1 + v, No);  // row r = yy * 3 + zz of the stage
        const int ch = 16 * sl + 8 * h;
        const bf16* src;
        if (ch < a.c0) {
          const int n = a.m0 ? No / 2 : No, sh = a.m0;
          src = a.s0 + ((long)(xx >> sh) + (long)n * ((yy >> sh) + (long)n * (zz >> sh))) * a.c0 + ch;
        } else {
          const int n = a.m1 ? No / 2 : No, sh = a.m1;
          src = a.s1 + ((long)(xx >> sh) + (long)n * ((yy >> sh) + (long)n * (zz >> sh))) * a.c1 + (ch - a.c0);
        }
        tc::cp16(st + r * tc::kRowBytes + h * (tc::kRowVox * 16) + v * 16, src);
      }
      if (!WRES) {
        unsigned char* wst = st + tc::kInBytes;
        for (int q = ptid; q < 27 * COUT * 2; q += NPROD) {
          const int h = q & 1, co = (q >> 1) % COUT, t = (q >> 1) / COUT;
          tc::cp16(wst + wofs<COUT>(t, co, h), a.W + ((long)t * COUT + co) * Cin + 16 * sl + 8 * h);
        }
      }
    };
    auto epilogue = [&](int i) -> bool {
      if (!__all_sync(0xffffffffu, mbar_wait(acc_full + (i & 1), (unsigned)((i >> 1) & 1)))) return false;
      tc::fence_after();
      int x0, y0, z;
      tile_of(i, x0, y0, z);
      const int sub = warp & 3;
      const int x = x0 + 32 * sub + lane;
#pragma unroll 1
      for (int j = 0; j < R; ++j) {
        float v[COUT];
        tc::tmem_ld<COUT>(tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)((i & 1) * R * COUT + j * COUT), v);
        const long vox = (long)x + (long)No * ((y0 + j) + (long)No * z);
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
          const float u = v[c] + (a.bias ? a.bias[c] : 0.f);
          v[c] = a.relu ? fmaxf(u, 0.f) : u;
        }
        if (a.out) {
          uint4* o = reinterpret_cast<uint4*>(a.out + vox * COUT);
#pragma unroll
          for (int q = 0; q < COUT / 8; ++q) {
            __nv_bfloat162 p0 = __floats2bfloat162_rn(v[8 * q], v[8 * q + 1]);
            __nv_bfloat162 p1 = __floats2bfloat162_rn(v[8 * q + 2], v[8 * q + 3]);
            __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * q + 4], v[8 * q + 5]);
            __nv_bfloat162 p3 = __floats2bfloat162_rn(v[8 * q + 6], v[8 * q + 7]);
            uint4 u;
            u.x = *reinterpret_cast<uint32_t*>(&p0);
            u.y = *reinterpret_cast<uint32_t*>(&p1);
            u.z = *reinterpret_cast<uint32_t*>(&p2);
            u.w = *reinterpret_cast<uint32_t*>(&p3);
            o[q] = u;
          }
        }
        if (a.out32) a.out32[vox] = v[0];
      }
      tc::fence_before();
      mbar_arrive(acc_empty + (i & 1));
      return true;
    };
    const bool epi = warp >= 4;
    if (WRES) {  // resident weights: [slice][tap][half][co][8], part of the first group
      const int n = nsl * 27 * COUT * 2;
      for (int q = ptid; q < n; q += NPROD) {
        const int h = q & 1, co = (q >> 1) % COUT, r2 = (q >> 1) / COUT, t = r2 % 27, sl = r2 / 27;
        tc::cp16(wres + sl * P::wslice + wofs<COUT>(t, co, h), a.W + ((long)t * COUT + co) * Cin + 16 * sl + 8 * h);
      }
    }
    for (int q = 0; q < LOOK; ++q) {
      if (q < nsteps) stage(q);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    bool ok = true;
    for (int s = 0; s < nsteps && ok; ++s) {
      // publish step s (its group is the oldest of the LOOK outstanding ones)
      asm volatile("cp.async.wait_group %0;" ::"n"(LOOK - 1) : "memory");
      tc::fence_proxy_async();
      mbar_arrive(full + (s % NS));
      // refill: step s + LOOK reuses the stage of step s + LOOK - NS = s - 1
      const int s2 = s + LOOK;
      if (s2 < nsteps) {
        if (s2 >= NS) ok = mbar_wait(empty + (s2 % NS), (unsigned)(((s2 - NS) / NS) & 1));
        if (ok) stage(s2);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      const int i = s / nsl;
      if (ok && epi && s % nsl == 0 && i > 0) ok = epilogue(i - 1);
      if (aborted()) ok = false;
    }
    if (ok && epi && ntile > 0) ok = epilogue(ntile - 1);
    if (!ok) fail();
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

// ---- host ----------------------------------------------------------------------------------------
// Launch if the layer fits (stride 1, output grid a multiple of 128, Cout in
// {16, 32, 64}, source channels multiples of 16); returns 0 otherwise.  The
// deepest staging ring that fits in shared memory is used, weights resident
// when they fit.
template <int COUT, bool WRES, int NS>
static int tc_launch(const TcConvArgs& a, int nsm, cudaStream_t st) {
  const int bytes = TcPlan<COUT, WRES, NS>::bytes(a.c0 + a.c1);
  if (bytes > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(k_conv_tc<COUT, WRES, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const long ntiles = (long)(a.No / 128) * (a.No / tc::kR) * a.No;
  const int grid = (int)(ntiles < nsm ? ntiles : nsm);
  k_conv_tc<COUT, WRES, NS><<<grid, tc::kThreads, bytes, st>>>(a);
  return 1;
}

template <int COUT>
static int tc_dispatch(const TcConvArgs& a, int nsm, cudaStream_t st) {
  const int cin = a.c0 + a.c1;
  constexpr int lim = 227 * 1024;
  if (TcPlan<COUT, true, 3>::bytes(cin) <= lim) return tc_launch<COUT, true, 3>(a, nsm, st);
  if (TcPlan<COUT, true, 2>::bytes(cin) <= lim) return tc_launch<COUT, true, 2>(a, nsm, st);
  if (TcPlan<COUT, false, 3>::bytes(cin) <= lim) return tc_launch<COUT, false, 3>(a, nsm, st);
  return tc_launch<COUT, false, 2>(a, nsm, st);
}

int conv_tc(const TcConvArgs& a, int Cout, int nsm, cudaStream_t st) {
  const int cin = a.c0 + a.c1;
  if (a.No < 128 || a.No % 128 || (a.c0 % 16) || (a.c1 % 16) || cin == 0 || !a.err) return 0;
  if (2 * tc::kR * Cout > 512) return 0;
  switch (Cout) {
    case 16: return tc_dispatch<16>(a, nsm, st);
    case 32: return tc_dispatch<32>(a, nsm, st);
    case 64: return tc_dispatch<64>(a, nsm, st);
  }
  return 0;
}

}  // namespace fe
