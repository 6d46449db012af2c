// step_rkernels.cu -- the PISO stencil kernels on asynchronous-copy rings
// (zring.cuh): every streamed plane reaches shared memory by cp.async A
// planes ahead, so no register holds data in flight and the z-neighbours are
// read from the ring.  Same per-cell arithmetic as step_zkernels.cu (and as
// the general kernels of step_kernels.cu, which carry the formulas of Sec. 2
// of arXiv:1404.0959).
#include "zring.cuh"

namespace fe {

template <typename T>
__device__ __forceinline__ T* Fr(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

// Dynamic shared-memory limits are set once per device by rprepare<T>()
// (outside any stream capture); the launchers run a ring kernel only on a
// prepared device.
constexpr int kMaxDev = 64;
template <typename T>
struct RingReady {
  static bool ok[kMaxDev];
};
template <typename T>
bool RingReady<T>::ok[kMaxDev] = {};
static int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
  return dev;
}
template <typename T>
static bool ring_ready() {
  const int dev = current_device();
  return dev >= 0 && RingReady<T>::ok[dev];
}
template <typename K>
static bool set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

// ---- correction (symmetric operator) ----------------------------------------------------------
// p^k = p^{k-1} + x staged as the sum of two rings; fluxes phi^k = phi* - dt G2 x,
// u^k = HbyA - dt/rho^{k-1} Gc p^k, rho^k = rho^n - dt/2 (div phi^n + D phi^k);
// FP64 path: ||b - M x||^2 for the reported residual.
constexpr int kCorrA = 2;
template <typename T, bool MIXED>
struct CorrRing {
  static constexpr int A = kCorrA, NCEN = MIXED ? 6 : 8;
  static constexpr int elems = 2 * ZSlots<A>::NS * kZHW + 3 * ZSlots<A>::NF * kZHW + NCEN * ZSlots<A>::NC * NTHR;
  static constexpr int bytes = elems * (int)sizeof(T);
};

template <typename T, bool MIXED>
__global__ void __launch_bounds__(NTHR) kr_corr(const BoxDev* boxes, const int2* work, double* part, int s, int rhop,
                                                int pp, int pnew, int kset, int kidx) {
  using CR = CorrRing<T, MIXED>;
  constexpr int A = CR::A;
  using SL = ZSlots<A>;
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  const int tid = threadIdx.x + TX * threadIdx.y;
  extern __shared__ __align__(16) unsigned char rsm[];
  T* base = reinterpret_cast<T*>(rsm);
  T* r_pp = base;
  T* r_x = r_pp + SL::NS * kZHW;
  T* r_ps = r_x + SL::NS * kZHW;  // 3 face rings
  T* r_c = r_ps + 3 * SL::NF * kZHW;  // centre rings: rho, rk, hb0..2, divphi [, psi, b]
  const T* g_pp = Fr<T>(B, pp);
  const T* g_x = Fr<T>(B, K_X);
  const T* g_ps[3] = {Fr<T>(B, W_PS0), Fr<T>(B, W_PS1), Fr<T>(B, W_PS2)};
  const T* g_c[8] = {Fr<T>(B, S(s, F_RHO)), Fr<T>(B, rhop), Fr<T>(B, W_HB0), Fr<T>(B, W_HB1),
                     Fr<T>(B, W_HB2),      Fr<T>(B, W_DIVPHI), Fr<T>(B, W_PSI), Fr<T>(B, K_B)};
  T* rk = Fr<T>(B, rhop);
  T* __restrict__ pn = Fr<T>(B, pnew);
  T* __restrict__ phk[3] = {Fr<T>(B, S(kset, F_PHI0)), Fr<T>(B, S(kset, F_PHI1)), Fr<T>(B, S(kset, F_PHI2))};
  T* __restrict__ uk[3] = {Fr<T>(B, S(kset, F_U0)), Fr<T>(B, S(kset, F_U1)), Fr<T>(B, S(kset, F_U2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], idt = T(1) / dt;
  const SL sl{t.k0};
  const int nk = t.kend - t.k0;
  // copies of the planes needed first: stencil k0-2..k0+2, faces k0-1..k0, centre k0
  auto issue = [&](int q) {  // group q >= 1: stencil k0+2+q, face k0+q, centre k0+q (within range)
    const int ms = t.k0 + 2 + q, mf = t.k0 + q, mc = t.k0 + q;
    if (ms <= t.kend + 1) {
      const int w = G.wrapz(ms);
      zr_issue_halo(G, g_pp, r_pp + sl.s(ms) * kZHW, w);
      zr_issue_halo(G, g_x, r_x + sl.s(ms) * kZHW, w);
    }
    if (mf < t.kend) {
#pragma unroll
      for (int d = 0; d < 3; ++d) zr_issue_halo(G, g_ps[d], r_ps + (d * SL::NF + sl.f(mf)) * kZHW, mf);
    }
    if (mc < t.kend) {
#pragma unroll
      for (int j = 0; j < CR::NCEN; ++j) zr_issue_centre(G, g_c[j], r_c + (j * SL::NC + sl.c(mc)) * NTHR, tid, mc);
    }
  };
  for (int m = t.k0 - 2; m <= t.k0 + 2; ++m) {
    const int w = G.wrapz(m);
    zr_issue_halo(G, g_pp, r_pp + sl.s(m) * kZHW, w);
    zr_issue_halo(G, g_x, r_x + sl.s(m) * kZHW, w);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    zr_issue_halo(G, g_ps[d], r_ps + (d * SL::NF + sl.f(t.k0 - 1)) * kZHW, G.wrapz(t.k0 - 1));
    zr_issue_halo(G, g_ps[d], r_ps + (d * SL::NF + sl.f(t.k0)) * kZHW, t.k0);
  }
#pragma unroll
  for (int j = 0; j < CR::NCEN; ++j) zr_issue_centre(G, g_c[j], r_c + (j * SL::NC + sl.c(t.k0)) * NTHR, tid, t.k0);
  cp_async_commit();
#pragma unroll
  for (int q = 1; q < A; ++q) {
    issue(q);
    cp_async_commit();
  }
  double rr = 0.0;
  for (int i = 0; i < nk; ++i) {
    const int k = t.k0 + i;
    cp_async_wait<A - 1>();
    __syncthreads();
    issue(A + i);
    cp_async_commit();
    if (!G.active) continue;
    ZView<T> vp, vx;
    vp.csm = vx.csm = G.csm;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      vp.p[j] = r_pp + sl.s(k - 2 + j) * kZHW;
      vx.p[j] = r_x + sl.s(k - 2 + j) * kZHW;
    }
    const ZView2<T> pk{vp, vx};
    T psp[3], psm[3];
    {
      const T* f0 = r_ps + (0 * SL::NF + sl.f(k)) * kZHW;
      const T* f1 = r_ps + (1 * SL::NF + sl.f(k)) * kZHW;
      const T* f2 = r_ps + (2 * SL::NF + sl.f(k)) * kZHW;
      const T* f2m = r_ps + (2 * SL::NF + sl.f(k - 1)) * kZHW;
      psp[0] = f0[G.csm];
      psm[0] = f0[G.csm - 1];
      psp[1] = f1[G.csm];
      psm[1] = f1[G.csm - ZGeom<2>::W];
      psp[2] = f2[G.csm];
      psm[2] = f2m[G.csm];
    }
    auto cen = [&](int j) { return r_c[(j * SL::NC + sl.c(k)) * NTHR + tid]; };
    const int c = G.col + G.plane(k);
    const T xc = vx.c();
    T dsum = T(0), lap = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T xp = vx.at(G, d, 1), xm = vx.at(G, d, -1);
      const T fp = psp[d] - dt * (xp - xc) * ih;
      const T fm = psm[d] - dt * (xc - xm) * ih;
      lap += (xp - xc) - (xc - xm);
      phk[d][c] = fp;
      dsum += fp - fm;
    }
    const T dtr = dt / cen(1);
    pn[c] = pk.c();
#pragma unroll
    for (int m = 0; m < 3; ++m) uk[m][c] = cen(2 + m) - dtr * (zGc_h(pk, G, m) * ih);
    rk[c] = cen(0) - T(0.5) * dt * (cen(5) + dsum * ih);
    if (!MIXED) {
      const T Mx = cen(6) * xc * idt - T(0.5) * dt * lap * ih * ih;
      const double r = (double)cen(7) - (double)Mx;
      rr += r * r;
    }
  }
  cp_async_wait<0>();
  Red<T> v[1] = {MIXED ? Red<T>{} : red_from<T>(rr)};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      if (MIXED) {
        B.sc[SC_RES0 + kidx] = B.sc[SC_ORES];
        B.sc[SC_IT0 + kidx] = B.sc[SC_ITSUM];
      } else {
        const double bb = B.sc[SC_BB];
        B.sc[SC_RES0 + kidx] = bb > 0.0 ? sqrt(res[0] / bb) : 0.0;
        B.sc[SC_IT0 + kidx] = B.sc[SC_ITERS];
      }
    }
  }
}

// ---- launchers (0: the ring kernel could not be prepared) --------------------------------------
#define RGRID(bytes) L.nblocks, dim3(TX, TY), (bytes), L.st
template <typename T>
int rlaunch_corr(const Launch& L, int s, int rhop, int pp, int pnew, int kset, int kidx, int mixed) {
  if (!ring_ready<T>()) return 0;
  constexpr int bm = CorrRing<T, true>::bytes, bf = CorrRing<T, false>::bytes;
  if (mixed)
    FE_LAUNCH(L, KID_CORR, (kr_corr<T, true><<<RGRID(bm)>>>(L.boxes, L.work, L.part, s, rhop, pp, pnew, kset, kidx)));
  else
    FE_LAUNCH(L, KID_CORR, (kr_corr<T, false><<<RGRID(bf)>>>(L.boxes, L.work, L.part, s, rhop, pp, pnew, kset, kidx)));
  return 1;
}

template <typename T>
int rprepare() {
  const int dev = current_device();
  if (dev < 0) return 0;
  bool ok = set_smem(kr_corr<T, true>, CorrRing<T, true>::bytes) && set_smem(kr_corr<T, false>, CorrRing<T, false>::bytes);
  RingReady<T>::ok[dev] = ok;
  return ok ? 1 : 0;
}

#define RINST(T)                                                                \
  template int rlaunch_corr<T>(const Launch&, int, int, int, int, int, int, int); \
  template int rprepare<T>();
RINST(double)
RINST(float)

}  // namespace fe
