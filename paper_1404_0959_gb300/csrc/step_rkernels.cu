// step_rkernels.cu -- the PISO stencil kernels on asynchronous-copy rings
// (zring.cuh): every streamed plane reaches shared memory by cp.async A
// planes ahead, so no register holds data in flight; the z-neighbours come
// from per-thread register queues fed from the ring.  Same per-cell
// arithmetic as step_zkernels.cu (and as
// the general kernels of step_kernels.cu, which carry the formulas of Sec. 2
// of arXiv:1404.0959).
#include "zring.cuh"

namespace fe {

// Lookahead planes of each ring kernel (shared memory per block grows with
// it; measured at 256^3 FP32 with column-pair threads: the corrector, the
// predictor, Du/Dt, the divergence, the right-hand side and the n-level flux
// divergences run best with two planes, the assembly and the dust kernels with
// one), and the predictor's
// register cap (three resident blocks per SM in FP32: its 174-register build
// left it at two and ran 25 % slower).
#ifndef FE_RING_A
#define FE_RING_A 2
#endif
#ifndef FE_RING_A_LIGHT
#define FE_RING_A_LIGHT 1
#endif
#ifndef FE_RING_MINB
#define FE_RING_MINB 1  // minimum resident blocks per SM asked of the register allocator
#endif
#ifndef FE_RING_MINB_PRED
#define FE_RING_MINB_PRED 3
#endif
#ifndef FE_RING_OFF
#define FE_RING_OFF 0u  // ring kernels left out (bits of RingKernel): their z-marching versions run
#endif
#ifndef FE_RING_A_RHS
#define FE_RING_A_RHS 3
#endif
#ifndef FE_RING_A_DIV
#define FE_RING_A_DIV 3
#endif
constexpr int kA = FE_RING_A, kA1 = FE_RING_A_LIGHT;
// Lookahead of the right-hand side and the divergence: three planes in flight.  The right-hand side is
// held to three resident blocks by its registers whatever its rings take, and the divergence keeps six
// blocks of its small rings (seven with two planes), so both gain bytes in flight per SM (measured at
// 256^3: divergence 0.277 -> 0.248 ms, right-hand side 0.360 -> 0.346 ms per step; four planes for the
// divergence 0.255).
constexpr int kArhs = FE_RING_A_RHS, kAdiv = FE_RING_A_DIV;

template <typename T>
__device__ __forceinline__ T* Fr(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

// Dynamic shared-memory limits are set once per device by rprepare<T>()
// (outside any stream capture); the launchers run a ring kernel only on a
// prepared device.
constexpr int kMaxDev = 64;
// per device, one bit per ring kernel (set when its shared-memory limit was accepted)
enum RingKernel { RK_CORR_M, RK_CORR_F, RK_PRED, RK_ASM, RK_ACCEL, RK_FLUX1, RK_FLUX2, RK_FLUX3, RK_DUST1, RK_DUST2,
                  RK_DUST3, RK_DIV, RK_RHS, RK_PRED_TW, RK_ASM_TW, RK_ACCEL_TW, RK_DUST1F, RK_DUST2F, RK_DUST3F,
                  RK_FECELL, RK_FEFACE };
template <typename T>
struct RingReady {
  static unsigned ok[kMaxDev];
};
template <typename T>
unsigned RingReady<T>::ok[kMaxDev] = {};
static int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
  return dev;
}
template <typename T>
static bool ring_ready(int kernel) {
  const int dev = current_device();
  return dev >= 0 && (RingReady<T>::ok[dev] >> kernel & 1u);
}
template <typename K>
static bool set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

template <typename P>
struct Unparen;
template <typename P>
struct Unparen<void(P)> {
  using type = P;
};
#define RING_PROLOGUE(P)                                   \
  const TileXYZ t = tile_xyz(boxes, work);                 \
  const BoxDev& B = boxes[t.box];                          \
  const RGeom<T> G(t.x0, t.y0, B.N);                       \
  const int tid = threadIdx.x + RTX * threadIdx.y;         \
  extern __shared__ __align__(16) unsigned char rsm[];     \
  typename Unparen<void(P)>::type R;                       \
  R.init(rsm, t.k0, t.kend)

// ---- correction (symmetric operator) ----------------------------------------------------------
// p^k = p^{k-1} + x staged as the sum of two rings; fluxes phi^k = phi* - dt G2 x,
// u^k = HbyA - dt/rho^{k-1} Gc p^k, rho^k = rho^n - dt/2 (div phi^n + D phi^k);
// FP64 path: ||b - M x||^2 for the reported residual.
template <typename T, bool MIXED>
using CorrPlan = RingPlan<T, kA, 2, 3, MIXED ? 6 : 8>;  // p^{k-1}, x | phi* | rho^n, rho^{k-1}, HbyA0..2, D phi^n [, psi, b]

template <typename T, bool MIXED>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_corr(const BoxDev* boxes, const int2* work, double* part, int s, int rhop,
                                                int pp, int pnew, int kset, int kidx, int xslot) {
  constexpr int NC = MIXED ? 6 : 8;
  RING_PROLOGUE((CorrPlan<T, MIXED>));
  R.gs[0] = Fr<T>(B, pp);
  R.gs[1] = Fr<T>(B, xslot);  // the pressure correction (FP32 solution, or the high parts of its pairs)
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = Fr<T>(B, W_PS0 + d);
  R.gc[0] = Fr<T>(B, S(s, F_RHO));
  R.gc[1] = Fr<T>(B, rhop);
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[2 + m] = Fr<T>(B, W_HB0 + m);
  R.gc[5] = Fr<T>(B, W_DIVPHI);
  if (NC == 8) {
    R.gc[6 % NC] = Fr<T>(B, W_PSI);
    R.gc[7 % NC] = Fr<T>(B, K_B);
  }
  T* rk = Fr<T>(B, rhop);  // rho^{k-1} in (through the ring), rho^k out (own cells only)
  T* __restrict__ pn = Fr<T>(B, pnew);
  T* __restrict__ phk[3] = {Fr<T>(B, S(kset, F_PHI0)), Fr<T>(B, S(kset, F_PHI1)), Fr<T>(B, S(kset, F_PHI2))};
  T* __restrict__ uk[3] = {Fr<T>(B, S(kset, F_U0)), Fr<T>(B, S(kset, F_U1)), Fr<T>(B, S(kset, F_U2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], idt = T(1) / dt;
  double rr = 0.0;
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crn = R.cen(0, k, tid), crp = R.cen(1, k, tid), cdp = R.cen(5, k, tid);
    const P2<T> chb[3] = {R.cen(2, k, tid), R.cen(3, k, tid), R.cen(4, k, tid)};
    T oph[3][2], opn[2], ou[3][2], ork[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const ZView<T> vp = R.view(0, k, G, r), vx = R.view(1, k, G, r);
      const ZView2<T> pk{vp, vx};
      T psp[3], psm[3];
      R.faces(0, k, G, r, psp, psm);
      const T xc = vx.c();
      T dsum = T(0), lap = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T xp = vx.at(G, d, 1), xm = vx.at(G, d, -1);
        const T fp = psp[d] - dt * (xp - xc) * ih;
        const T fm = psm[d] - dt * (xc - xm) * ih;
        lap += (xp - xc) - (xc - xm);
        oph[d][r] = fp;
        dsum += fp - fm;
      }
      const T dtr = dt / pc<T>(crp, r);
      opn[r] = pk.c();
#pragma unroll
      for (int m = 0; m < 3; ++m) ou[m][r] = pc<T>(chb[m], r) - dtr * (zGc_h(pk, G, m) * ih);
      ork[r] = pc<T>(crn, r) - T(0.5) * dt * (pc<T>(cdp, r) + dsum * ih);
      if (!MIXED) {
        const T Mx = pc<T>(R.cen(6 % NC, k, tid), r) * xc * idt - T(0.5) * dt * lap * ih * ih;
        const double e = (double)pc<T>(R.cen(7 % NC, k, tid), r) - (double)Mx;
        rr += e * e;
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) stp(phk[d] + c, oph[d][0], oph[d][1]);
    stp(pn + c, opn[0], opn[1]);
#pragma unroll
    for (int m = 0; m < 3; ++m) stp(uk[m] + c, ou[m][0], ou[m][1]);
    stp(rk + c, ork[0], ork[1]);
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

// L_m = -D(phi I4 u_m) + mu (lap u_m + Gc_m(div) / 3) and its viscous part for both cells of the pair
// (u0..2, div: stencil fields 0..3 of the plan; face fluxes phm / php of both cells), from one line of
// u_m per axis and one of div along m: the convection from the unscaled 16 I4 at both faces, the compact
// Laplacian as (28 S1 - 162 u - S2) / 24 (S1, S2: the six neighbours at distance 1 and 2), Gc unscaled;
// cl = mu / (24 h^2), cd = mu / (48 h), cc = 1 / (16 h).
template <typename T, typename Plan>
__device__ __forceinline__ void ring_L(const Plan& R, int k, const RGeom<T>& G, const T (&php)[3][2],
                                       const T (&phm)[3][2], T cl, T cd, T cc, T (&L)[3][2], T (&visc)[3][2]) {
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    T conv[2], lap[2];
    {
      const Line2<T> l[3] = {ring_line(R, m, k, G, 0), ring_line(R, m, k, G, 1), ring_line(R, m, k, G, 2)};
      const P2<T> uc = R.zq[m][2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T u = pc<T>(uc, r);
        T cv = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) cv += php[d][r] * i4p16(l[d], u, r) - phm[d][r] * i4m16(l[d], u, r);
        conv[r] = cv;
        const T s1 = (l[0].m1[r] + l[0].p1[r]) + (l[1].m1[r] + l[1].p1[r]) + (l[2].m1[r] + l[2].p1[r]);
        const T s2 = (l[0].m2[r] + l[0].p2[r]) + (l[1].m2[r] + l[1].p2[r]) + (l[2].m2[r] + l[2].p2[r]);
        lap[r] = fma(T(28), s1, -fma(T(162), u, s2));
      }
    }
    const Line2<T> ld = ring_line(R, 3, k, G, m);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      visc[m][r] = fma(cl, lap[r], cd * gc16(ld, r));
      L[m][r] = visc[m][r] - cc * conv[r];
    }
  }
}

// two-way: Ysum as a second centre field with one plane of lookahead, so that three blocks per
// multiprocessor still fit in FP32
template <typename T, bool TW = false>
using PredPlan = RingPlan<T, TW ? kA1 : kA, 5, 3, TW ? 2 : 1>;  // u0..2, div, p | phi | rho [, Ysum]
// TW: two-way coupling (a with the inertia rho (1 + Ysum), R^n with the reaction -(rho Ysum) a)
template <typename T, bool TW>
__global__ void __launch_bounds__(RNT, sizeof(T) == 4 ? FE_RING_MINB_PRED : FE_RING_MINB) kr_pred(const BoxDev* boxes, const int2* work, int s, int kset, int ysl) {
  RING_PROLOGUE((PredPlan<T, TW>));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[m] = Fr<T>(B, S(s, F_U0 + m));
  R.gs[3] = Fr<T>(B, W_DIV);
  R.gs[4] = Fr<T>(B, S(s, F_P));
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = Fr<T>(B, S(s, F_PHI0 + d));
  R.gc[0] = Fr<T>(B, S(s, F_RHO));
  if (TW) R.gc[TW ? 1 : 0] = Fr<T>(B, ysl);
  T* __restrict__ divphi = Fr<T>(B, W_DIVPHI);
  T* __restrict__ Rn[3] = {Fr<T>(B, W_RN0), Fr<T>(B, W_RN1), Fr<T>(B, W_RN2)};
  T* __restrict__ An[3] = {Fr<T>(B, W_AN0), Fr<T>(B, W_AN1), Fr<T>(B, W_AN2)};
  T* __restrict__ psi = Fr<T>(B, W_PSI);
  T* __restrict__ dinv = Fr<T>(B, W_DINV);
  T* __restrict__ rho0 = Fr<T>(B, S(kset, F_RHO));
  T* __restrict__ us[3] = {Fr<T>(B, S(kset, F_U0)), Fr<T>(B, S(kset, F_U1)), Fr<T>(B, S(kset, F_U2))};
  const T ih = (T)B.ih, mu = (T)B.mu, dt = (T)B.sc[SC_DT], gam = (T)B.gamma;
  const T cl = mu * ih * ih * T(1.0 / 24.0), cd = mu * ih * T(1.0 / 48.0), cc = ih * T(0.0625);
  const JacobiDiag<T> jd(B.sc[SC_DT], B.ih);
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crho = R.cen(0, k, tid);
    P2<T> ys2;
    if (TW) ys2 = R.cen(TW ? 1 : 0, k, tid);
    T ous[3][2], oRn[3][2], oAn[3][2], ops[2], odi[2], odp[2], or0[2];
    T php[3][2], phm[3][2];
    R.faces2(0, k, G, php, phm);
    T L[3][2], visc[3][2];
    ring_L(R, k, G, php, phm, cl, cd, cc, L, visc);
    T gp[3][2];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const Line2<T> lp = ring_line(R, 4, k, G, m);
      gp[m][0] = cc * gc16(lp, 0);
      gp[m][1] = cc * gc16(lp, 1);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T dph = ((php[0][r] - phm[0][r]) + (php[1][r] - phm[1][r]) + (php[2][r] - phm[2][r])) * ih;
      const T rc = pc<T>(crho, r);
      const T r0 = rc - dt * dph;
      const T ir0 = rcp_rn(r0), ir = rcp_rn(rc);
      if (TW) {
        const T ys = pc<T>(ys2, r);
        const T ia = rcp_rn(rc * (T(1) + ys)), w = rc * ys;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const T a = (visc[m][r] - gp[m][r]) * ia;
          const T Rf = L[m][r] - w * a;
          ous[m][r] = (rc * pc<T>(R.zq[m][2], r) + dt * (Rf - gp[m][r])) * ir0;
          oRn[m][r] = Rf;
          oAn[m][r] = a;
        }
      } else {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          ous[m][r] = (rc * pc<T>(R.zq[m][2], r) + dt * (L[m][r] - gp[m][r])) * ir0;
          oRn[m][r] = L[m][r];
          oAn[m][r] = (visc[m][r] - gp[m][r]) * ir;
        }
      }
      const T ps = rc / (gam * pc<T>(R.zq[4][2], r));
      ops[r] = ps;
      odi[r] = jd.inv(ps);
      odp[r] = dph;
      or0[r] = r0;
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      stp(us[m] + c, ous[m][0], ous[m][1]);
      stp(Rn[m] + c, oRn[m][0], oRn[m][1]);
      stp(An[m] + c, oAn[m][0], oAn[m][1]);
    }
    stp(psi + c, ops[0], ops[1]);
    stp(dinv + c, odi[0], odi[1]);
    stp(divphi + c, odp[0], odp[1]);
    stp(rho0 + c, or0[0], or0[1]);
  }
  cp_async_wait<0>();
}

// ---- corrector assembly ------------------------------------------------------------------------------
template <typename T, bool TW = false>
using AsmPlan = RingPlan<T, kA1, 4, 3, TW ? 12 : 8>;  // u0..2 (level k-1), div | phi | rho, un0..2, rho', Rn0..2
                                                       // [, Ysum, a0..2]
// TW: two-way coupling, L^{k-1} - (rho^{k-1} Ysum) a with a the latest Du/Dt (read per cell pair)
template <typename T, bool TW>
__global__ void __launch_bounds__(RNT, sizeof(T) == 4 && TW ? 3 : FE_RING_MINB) kr_asm(const BoxDev* boxes, const int2* work,
                                                                                   int s, int up0, int php0, int rhop,
                                                                                   int ysl) {
  RING_PROLOGUE((AsmPlan<T, TW>));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[m] = Fr<T>(B, up0 + m);
  R.gs[3] = Fr<T>(B, W_DIV);
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = Fr<T>(B, php0 + d);
  R.gc[0] = Fr<T>(B, S(s, F_RHO));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[1 + m] = Fr<T>(B, S(s, F_U0 + m));
  R.gc[4] = Fr<T>(B, rhop);
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[5 + m] = Fr<T>(B, W_RN0 + m);
  if (TW) {
    R.gc[TW ? 8 : 0] = Fr<T>(B, ysl);
#pragma unroll
    for (int m = 0; m < 3; ++m) R.gc[TW ? 9 + m : 0] = Fr<T>(B, W_AN0 + m);
  }
  T* __restrict__ hb[3] = {Fr<T>(B, W_HB0), Fr<T>(B, W_HB1), Fr<T>(B, W_HB2)};
  const T ih = (T)B.ih, mu = (T)B.mu, dt = (T)B.sc[SC_DT];
  const T cl = mu * ih * ih * T(1.0 / 24.0), cd = mu * ih * T(1.0 / 48.0), cc = ih * T(0.0625);
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crho = R.cen(0, k, tid), crp = R.cen(4, k, tid);
    T ohb[3][2];
    T php[3][2], phm[3][2];
    R.faces2(0, k, G, php, phm);
    T L[3][2], visc[3][2];
    ring_L(R, k, G, php, phm, cl, cd, cc, L, visc);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T rc = pc<T>(crho, r);
      const T irp = rcp_rn(pc<T>(crp, r));
      if (TW) {
        const T w = pc<T>(crp, r) * pc<T>(R.cen(TW ? 8 : 0, k, tid), r);
#pragma unroll
        for (int m = 0; m < 3; ++m) L[m][r] = L[m][r] - w * pc<T>(R.cen(TW ? 9 + m : 0, k, tid), r);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const T Rm = T(0.5) * (pc<T>(R.cen(5 + m, k, tid), r) + L[m][r]);
        ohb[m][r] = (rc * pc<T>(R.cen(1 + m, k, tid), r) + dt * Rm) * irp;
      }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) stp(hb[m] + c, ohb[m][0], ohb[m][1]);
  }
  cp_async_wait<0>();
}

// ---- Du/Dt at level k -----------------------------------------------------------------------------------
template <typename T, bool TW = false>
using AccelPlan = RingPlan<T, kA, 5, 0, TW ? 2 : 1>;  // u0..2, div, p | | rho [, Ysum]
// TW: two-way coupling, inertia rho (1 + Ysum) with Ysum from slot ysl (a centre field of the ring)
template <typename T, bool TW>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_accel(const BoxDev* boxes, const int2* work, int kset, int pk,
                                                              int ysl) {
  RING_PROLOGUE((AccelPlan<T, TW>));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[m] = Fr<T>(B, S(kset, F_U0 + m));
  R.gs[3] = Fr<T>(B, W_DIV);
  R.gs[4] = Fr<T>(B, pk);
  R.gc[0] = Fr<T>(B, S(kset, F_RHO));
  if (TW) R.gc[TW ? 1 : 0] = Fr<T>(B, ysl);
  T* __restrict__ a[3] = {Fr<T>(B, W_AN0), Fr<T>(B, W_AN1), Fr<T>(B, W_AN2)};
  const T ih = (T)B.ih, mu = (T)B.mu;
  // a_m = (mu (lap u_m + Gc_m(div) / 3) - Gc_m p) / rho with the compact fourth-order Laplacian
  // sum_d D G4_d = (28 S1 - 162 u - S2) / (24 h^2) (S1, S2: sums of the six neighbours at distance 1
  // and 2) and Gc_m = (10 (f_+1 - f_-1) - (f_+2 - f_-2)) / (16 h); the constant factors are folded
  const T cl = mu * ih * ih * T(1.0 / 24.0), cd = mu * ih * T(1.0 / 48.0), cg = ih * T(0.0625);
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crho = R.cen(0, k, tid);
    P2<T> ys2;
    if (TW) ys2 = R.cen(TW ? 1 : 0, k, tid);
    T ir[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
      ir[r] = TW ? rcp_rn(pc<T>(crho, r) * (T(1) + pc<T>(ys2, r))) : rcp_rn(pc<T>(crho, r));
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      T lap[2];
      {
        const Line2<T> lx = ring_line(R, m, k, G, 0), ly = ring_line(R, m, k, G, 1), lz = ring_line(R, m, k, G, 2);
        const P2<T> uc = R.zq[m][2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const T s1 = (lx.m1[r] + lx.p1[r]) + (ly.m1[r] + ly.p1[r]) + (lz.m1[r] + lz.p1[r]);
          const T s2 = (lx.m2[r] + lx.p2[r]) + (ly.m2[r] + ly.p2[r]) + (lz.m2[r] + lz.p2[r]);
          lap[r] = fma(T(28), s1, -fma(T(162), pc<T>(uc, r), s2));
        }
      }
      const Line2<T> ld = ring_line(R, 3, k, G, m), lp = ring_line(R, 4, k, G, m);
      T oa[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T gd = fma(T(10), ld.p1[r] - ld.m1[r], -(ld.p2[r] - ld.m2[r]));
        const T gp = fma(T(10), lp.p1[r] - lp.m1[r], -(lp.p2[r] - lp.m2[r]));
        oa[r] = (fma(cl, lap[r], cd * gd) - cg * gp) * ir[r];
      }
      stp(a[m] + c, oa[0], oa[1]);
    }
  }
  cp_async_wait<0>();
}

// ---- dust: n-level flux divergences FYN_j = D(phi_p^n I4 Y_j^n) --------------------------------------------
// h D(phi_p I4 Y_j) for both cells of the pair and every class: phi_p = phi - tau_j I4(rho) I4(a_d) at each
// face (rho, a0..2, Y_j: stencil fields 0, 1..3, 4 + j of the plan; phi: face arrays 0..2).  Lines of rho
// and a_d along d, and of Y_j along d, each read once; 16 I4 evaluated unscaled, the factors folded.
template <typename T, int ND, typename Plan>
__device__ __forceinline__ void ring_particle_flux(const Plan& R, int k, const RGeom<T>& G, const T (&taup)[ND],
                                                   T (&fl)[ND][2]) {
  T php[3][2], phm[3][2];
  R.faces2(0, k, G, php, phm);
  const P2<T> rc = R.zq[0][2];
#pragma unroll
  for (int j = 0; j < ND; ++j) fl[j][0] = fl[j][1] = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T rap[2], ram[2];
    {
      const Line2<T> lr = ring_line(R, 0, k, G, d), la = ring_line(R, 1 + d, k, G, d);
      const P2<T> ac = R.zq[1 + d][2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        rap[r] = i4p16(lr, pc<T>(rc, r), r) * i4p16(la, pc<T>(ac, r), r);
        ram[r] = i4m16(lr, pc<T>(rc, r), r) * i4m16(la, pc<T>(ac, r), r);
      }
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const T tq = taup[j] * T(1.0 / 256.0);
      const Line2<T> ly = ring_line(R, 4 + j, k, G, d);
      const P2<T> yc = R.zq[4 + j][2];
#pragma unroll
      for (int r = 0; r < 2; ++r)
        fl[j][r] += fma(-tq, rap[r], php[d][r]) * i4p16(ly, pc<T>(yc, r), r) -
                    fma(-tq, ram[r], phm[d][r]) * i4m16(ly, pc<T>(yc, r), r);
    }
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) fl[j][0] *= T(0.0625), fl[j][1] *= T(0.0625);
}

template <typename T, int ND>
using FluxPlan = RingPlan<T, kA, 4 + ND, 3, 0>;  // rho, a0..2, Y_j | phi (two planes ahead: measured)
template <typename T, int ND>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_fluxn(const BoxDev* boxes, const int2* work, int s) {
  RING_PROLOGUE((FluxPlan<T, ND>));
  (void)tid;  // no centre fields
  R.gs[0] = Fr<T>(B, S(s, F_RHO));
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gs[1 + d] = Fr<T>(B, W_AN0 + d);
#pragma unroll
  for (int j = 0; j < ND; ++j) R.gs[4 + j] = Fr<T>(B, S(s, F_Y0 + j));
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = Fr<T>(B, S(s, F_PHI0 + d));
  const T ih = (T)B.ih;
  T taup[ND];
  T* fyn[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    taup[j] = (T)B.tau_p[j];
    fyn[j] = Fr<T>(B, W_FYN0 + j);
  }
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    T fl[ND][2];
    ring_particle_flux<T, ND>(R, k, G, taup, fl);
#pragma unroll
    for (int j = 0; j < ND; ++j) stp(fyn[j] + c, fl[j][0] * ih, fl[j][1] * ih);
  }
  cp_async_wait<0>();
}

// ---- dust: level k, (rho Y)^k and Y^k; on the last corrector the barotropic closure and totals -----------------
// FR: Fourier closure -- also E^k = (rho^n E^n - dt/2 (D F_E^n + D F_E^k)) / rho^k (E^n, D F_E^n and
// D F_E^k as centre fields, k_fe_cell / k_fe_div), and on the last corrector T = (E - |u|^2/2) / c_v,
// p = rho R T and the total energy sum rho E (the general k_dust<T, true>'s expressions)
template <typename T, int ND, bool FR = false>
using DustPlan = RingPlan<T, kA1, 4 + ND, 3, 4 + 2 * ND + (FR ? 3 : 0)>;  // rho^k, a0..2, Y_j^{k-1} | phi^k |
                                                                         // rho^n, Y^n, FYN, [E^n, DFE^n, DFE^k,] u0..2
template <typename T, int ND, bool FR>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_dust(const BoxDev* boxes, const int2* work, double* part, int s, int kset,
                                                int yp0, int yn0, int last, int enew) {
  RING_PROLOGUE((DustPlan<T, ND, FR>));
  constexpr int EB = 1 + 2 * ND, UB = EB + (FR ? 3 : 0);  // centre indices of E^n (FR) and of u^k
  R.gs[0] = Fr<T>(B, S(kset, F_RHO));
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gs[1 + d] = Fr<T>(B, W_AN0 + d);
#pragma unroll
  for (int j = 0; j < ND; ++j) R.gs[4 + j] = Fr<T>(B, yp0 + j);
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = Fr<T>(B, S(kset, F_PHI0 + d));
  R.gc[0] = Fr<T>(B, S(s, F_RHO));
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    R.gc[1 + j] = Fr<T>(B, S(s, F_Y0 + j));
    R.gc[1 + ND + j] = Fr<T>(B, W_FYN0 + j);
  }
  if (FR) {
    R.gc[FR ? EB : 0] = Fr<T>(B, W_EN);
    R.gc[FR ? EB + 1 : 0] = Fr<T>(B, W_FEN);
    R.gc[FR ? EB + 2 : 0] = Fr<T>(B, W_FED);
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[UB + m] = Fr<T>(B, S(kset, F_U0 + m));
  if (!last) R.ncf = UB;  // u^k is read on the last corrector only
  T* __restrict__ eout = FR && enew >= 0 ? Fr<T>(B, enew) : nullptr;
  T* __restrict__ tout = FR ? Fr<T>(B, S(kset, F_T)) : nullptr;
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], gam = (T)B.gamma;
  T taup[ND];
  T* ynew[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    taup[j] = (T)B.tau_p[j];
    ynew[j] = Fr<T>(B, yn0 + j);
  }
  T* __restrict__ pout = Fr<T>(B, S(kset, F_P));
  SumAcc<T> amass, abad;
  DotAcc<T> aen, ady[ND];
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crn = R.cen(0, k, tid);
    T oy[ND][2], op[2], oe[2], ot[2];
    T flx[ND][2];
    ring_particle_flux<T, ND>(R, k, G, taup, flx);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T rk = pc<T>(R.zq[0][2], r);
      const T irk = rcp_rn(rk);
      const T rn = pc<T>(crn, r);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const T fl = flx[j][r];
        const T rY = rn * pc<T>(R.cen(1 + j, k, tid), r) - T(0.5) * dt * (pc<T>(R.cen(1 + ND + j, k, tid), r) + fl * ih);
        const T Yk = rY * irk;
        oy[j][r] = Yk;
        if (last) {
          ady[j].add(rk, Yk);
          if (!isfinite(Yk)) abad.add(T(1));
        }
      }
      T Ek = T(0);
      if (FR) {
        const T rE = rn * pc<T>(R.cen(FR ? EB : 0, k, tid), r) -
                     T(0.5) * dt * (pc<T>(R.cen(FR ? EB + 1 : 0, k, tid), r) + pc<T>(R.cen(FR ? EB + 2 : 0, k, tid), r));
        Ek = rE * irk;
        oe[r] = Ek;
      }
      op[r] = T(0);
      ot[r] = T(0);
      if (last) {
        const T u0 = pc<T>(R.cen(UB, k, tid), r), u1 = pc<T>(R.cen(UB + 1, k, tid), r),
                u2 = pc<T>(R.cen(UB + 2, k, tid), r);
        const T uu = u0 * u0 + u1 * u1 + u2 * u2;
        T pf;
        if (FR) {
          const T Tk = (Ek - T(0.5) * uu) / (T)B.cv;
          ot[r] = Tk;
          pf = rk * (T)B.R * Tk;
          aen.add(rk, Ek);
        } else {
          pf = pow(rk, gam) / gam;
          aen.add(rk, uu);
        }
        op[r] = pf;
        amass.add(rk);
        if (!(isfinite(rk) && isfinite(uu) && isfinite(pf))) abad.add(T(1));
      }
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) stp(ynew[j] + c, oy[j][0], oy[j][1]);
    if (eout) stp(eout + c, oe[0], oe[1]);
    if (last) {
      stp(pout + c, op[0], op[1]);
      if (FR) stp(tout + c, ot[0], ot[1]);
    }
  }
  cp_async_wait<0>();
  if (!last) return;
  Red<T> acc[3 + ND];
  acc[0] = amass.red();
  acc[1] = aen.red();
  acc[2] = abad.red();
#pragma unroll
  for (int j = 0; j < ND; ++j) acc[3 + j] = ady[j].red();
  __shared__ double res[3 + ND];
  if (block_sum_last<3 + ND>(acc, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_MASS] = res[0];
      B.sc[SC_ENERGY] = FR ? res[1] : 0.5 * res[1];
      B.sc[SC_BAD] = res[2];
      for (int j = 0; j < MAXD; ++j) B.sc[SC_DUST0 + j] = j < ND ? res[3 + j] : 0.0;
    }
  }
}

// ---- Fourier closure: per cell H = E + p/rho, T and the nine Gauss gradients h Gc_m u_l ------------------
// (the fields the energy face fluxes k_fe_face read; k_fe_cell's expressions).  es >= 0: E from slot es
// (tmode 1); es < 0: the level-n energy E^n = c_v T^n + |u^n|^2 / 2 from T^n and u^n, also stored in W_EN.
// tmode 0: T = T^n, 1: T = p / (rho R).  The gradients from line loads of u_l along m, both cells.
template <typename T>
using FeCellPlan = RingPlan<T, kA, 3, 0, 6>;  // u0..2 | | rho, p, E or T^n, u^n_0..2
template <typename T>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_fe_cell(const BoxDev* boxes, const int2* work, int s, int u0,
                                                                int rhos, int ps, int es, int tmode) {
  RING_PROLOGUE(FeCellPlan<T>);
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[m] = Fr<T>(B, u0 + m);
  R.gc[0] = Fr<T>(B, rhos);
  R.gc[1] = Fr<T>(B, ps);
  R.gc[2] = Fr<T>(B, es >= 0 ? es : S(s, F_T));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[3 + m] = Fr<T>(B, S(s, F_U0 + m));
  R.ncf = es >= 0 ? 3 : 6;  // u^n only for E^n
  T* __restrict__ Hc = Fr<T>(B, W_FEH);
  T* __restrict__ Tc = Fr<T>(B, W_FET);
  T* __restrict__ En = Fr<T>(B, W_EN);
  const T cv = (T)B.cv, Rg = (T)B.R;
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crho = R.cen(0, k, tid), cp = R.cen(1, k, tid), cx = R.cen(2, k, tid);
    T oh[2], ot[2], oe[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T rc = pc<T>(crho, r), p = pc<T>(cp, r), x = pc<T>(cx, r);
      T e = x;
      if (es < 0) {
        const T a = pc<T>(R.cen(3, k, tid), r), b = pc<T>(R.cen(4, k, tid), r), d = pc<T>(R.cen(5, k, tid), r);
        e = cv * x + T(0.5) * (a * a + b * b + d * d);
        oe[r] = e;
      }
      oh[r] = e + p / rc;
      ot[r] = tmode ? p / (rc * Rg) : x;
    }
    stp(Hc + c, oh[0], oh[1]);
    stp(Tc + c, ot[0], ot[1]);
    if (es < 0) stp(En + c, oe[0], oe[1]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const Line2<T> ln = ring_line(R, l, k, G, m);
        stp(Fr<T>(B, W_FEG0 + 3 * m + l) + c, gc16(ln, 0) * T(0.0625), gc16(ln, 1) * T(0.0625));
      }
    }
  }
  cp_async_wait<0>();
}

// The three +1/2 face fluxes F_E = phi I4(H) - sum_m tau_dm I4(u_m) - kappa G4(T) of every cell
// (k_fe_face's expressions): lines of H, T, u0..2 and div along each axis from the ring, the gradient
// fields h Gc_m u_d (needed only along d, at offsets -1..2) by pair loads through the read-only path.
template <typename T>
using FeFacePlan = RingPlan<T, kA1, 6, 0, 3>;  // H, T, u0..2, div | | phi0..2
template <typename T>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_fe_face(const BoxDev* boxes, const int2* work, int u0, int phi0) {
  RING_PROLOGUE(FeFacePlan<T>);
  R.gs[0] = Fr<T>(B, W_FEH);
  R.gs[1] = Fr<T>(B, W_FET);
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[2 + m] = Fr<T>(B, u0 + m);
  R.gs[5] = Fr<T>(B, W_DIV);
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gc[d] = Fr<T>(B, phi0 + d);
  const T ih = (T)B.ih, mu = (T)B.mu, kappa = (T)B.kappa;
  const int N = B.N, NN = N * N;
  // own pair (x, x+1) and its neighbours for the gradient loads (N even: pairs never straddle the seam)
  const int xg = RGeom<T>::wrap(t.x0 + 2 * threadIdx.x, N), yg = RGeom<T>::wrap(t.y0 + threadIdx.y, N);
  const int xl = xg == 0 ? N - 2 : xg - 2, xr = xg + 2 == N ? 0 : xg + 2;
  int yrow[4];  // rows y-1 .. y+2
#pragma unroll
  for (int q = 0; q < 4; ++q) yrow[q] = RGeom<T>::wrap(yg + q - 1, N) * N;
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
#pragma unroll
    for (int d = 0; d < 3; ++d) {  // unrolled: the axis selects the line loads at compile time
      const Line2<T> lh = ring_line(R, 0, k, G, d), lt = ring_line(R, 1, k, G, d);
      const P2<T> hc = R.zq[0][2], tc = R.zq[1][2];
      const P2<T> ph = R.cen(d, k, tid);
      T work[2] = {T(0), T(0)}, of[2];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const Line2<T> lu = ring_line(R, 2 + m, k, G, d);
        const P2<T> uc = R.zq[2 + m][2];
        // g = h Gc_m u_d at offsets -1..2 along d of both cells
        const T* g = Fr<T>(B, W_FEG0 + 3 * m + d);
        T gv[2][4];
        if (d == 0) {
          const int row = yrow[1] + k * NN;
          const P2<T> a = ldg2(g + row + xl), b = ldg2(g + row + xg), e = ldg2(g + row + xr);
          gv[0][0] = a.y, gv[0][1] = b.x, gv[0][2] = b.y, gv[0][3] = e.x;
          gv[1][0] = b.x, gv[1][1] = b.y, gv[1][2] = e.x, gv[1][3] = e.y;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int o = d == 1 ? yrow[q] + k * NN : yrow[1] + G.wrapz(k + q - 1) * NN;
            const P2<T> v = ldg2(g + o + xg);
            gv[0][q] = v.x, gv[1][q] = v.y;
          }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const T u = pc<T>(uc, r);
          const T ig = (T(9) * (gv[r][1] + gv[r][2]) - (gv[r][0] + gv[r][3])) * T(0.0625);
          const T g4u = (T(27) * (lu.p1[r] - u) - (lu.p2[r] - lu.m1[r])) * T(1.0 / 24.0);
          T tau = (g4u + ig) * ih;
          if (d == m) {
            const Line2<T> ld = ring_line(R, 5, k, G, d);
            tau -= T(2.0 / 3.0) * (i4p16(ld, pc<T>(R.zq[5][2], r), r) * T(0.0625));
          }
          work[r] += (mu * tau) * (i4p16(lu, u, r) * T(0.0625));
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T IH = i4p16(lh, pc<T>(hc, r), r) * T(0.0625);
        const T G4T = (T(27) * (lt.p1[r] - pc<T>(tc, r)) - (lt.p2[r] - lt.m1[r])) * T(1.0 / 24.0) * ih;
        of[r] = pc<T>(ph, r) * IH - work[r] - kappa * G4T;
      }
      stp(Fr<T>(B, W_FEF0 + d) + c, of[0], of[1]);
    }
  }
  cp_async_wait<0>();
}

// ---- velocity divergence div = sum_m Gc_m(u_m) --------------------------------------------------------
template <typename T>
using DivPlan = RingPlan<T, kAdiv, 3, 0, 0>;  // u0..2
// with_dt: also max_i sum_d |u_d| over the box and the adaptive time step
// from it (the first divergence of a step reads u^n, the field k_dt reads).
template <typename T>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_div(const BoxDev* boxes, const int2* work, int u0,
                                                            double* part, int with_dt) {
  RING_PROLOGUE(DivPlan<T>);
  (void)tid;  // no centre fields
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[m] = Fr<T>(B, u0 + m);
  T* __restrict__ div = Fr<T>(B, W_DIV);
  const T ih16 = (T)B.ih * T(0.0625);
  T umax = T(0);
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    T od[2];
    const Line2<T> l0 = ring_line(R, 0, k, G, 0), l1 = ring_line(R, 1, k, G, 1), l2 = ring_line(R, 2, k, G, 2);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      od[r] = ((gc16(l0, r) + gc16(l1, r)) + gc16(l2, r)) * ih16;
      if (with_dt)
        umax = fmax(umax, fabs(pc<T>(R.zq[0][2], r)) + fabs(pc<T>(R.zq[1][2], r)) + fabs(pc<T>(R.zq[2][2], r)));
    }
    stp(div + G.col + G.plane(k), od[0], od[1]);
  }
  cp_async_wait<0>();
  if (!with_dt) return;
  __shared__ double res;
  if (block_max_last((double)umax, B, part, &res, B.tile0, B.ntiles))
    if (threadIdx.x == 0 && threadIdx.y == 0) finish_dt(B, res);
}

// ---- phi* and the pressure right-hand side --------------------------------------------------------------
// With rstart (mixed-precision plain CG) b goes straight to the refinement's
// copy (K_AUX) and to the first inner right-hand side (K_R), and the kernel
// starts the refined solve: ||b||^2 and <b, D^{-1} b> into the refinement and
// CG scalars (the solution pairs start as zero by the outer-step count).
template <typename T>
using RhsPlan = RingPlan<T, kArhs, 5, 0, 3>;  // rho', HbyA0..2, p | | rho^n, D phi^n [, D^{-1}]
template <typename T>
__global__ void __launch_bounds__(RNT, FE_RING_MINB) kr_rhs(const BoxDev* boxes, const int2* work, int s, int rhop,
                                                            int pp, double* part, int* rstart, int* active, int poly) {
  RING_PROLOGUE(RhsPlan<T>);
  R.gs[0] = Fr<T>(B, rhop);
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gs[1 + d] = Fr<T>(B, W_HB0 + d);
  R.gs[4] = Fr<T>(B, pp);
  R.gc[0] = Fr<T>(B, S(s, F_RHO));
  R.gc[1] = Fr<T>(B, W_DIVPHI);
  R.gc[2] = Fr<T>(B, W_DINV);
  const bool start = rstart != nullptr;
  if (!start || poly) R.ncf = 2;  // D^{-1} only for <b, D^{-1} b> of a Jacobi start
  T* __restrict__ ps[3] = {Fr<T>(B, W_PS0), Fr<T>(B, W_PS1), Fr<T>(B, W_PS2)};
  T* __restrict__ b = Fr<T>(B, start ? K_AUX : K_B);
  T* __restrict__ r0 = Fr<T>(B, K_R);
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], idt = T(1) / dt, dih = dt * ih;
  DotAcc<T> abb, abz;
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crho = R.cen(0, k, tid), cdp = R.cen(1, k, tid);
    // phi* at the +1/2 faces and D phi* from lines of rho', HbyA_d and p along d (16 I4 unscaled)
    T ops[3][2], ob[2], dsum[2] = {T(0), T(0)};
    const P2<T> rpc = R.zq[0][2], pcc = R.zq[4][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const Line2<T> lr = ring_line(R, 0, k, G, d), lh = ring_line(R, 1 + d, k, G, d);
      const Line2<T> lp = ring_line1(R, 4, k, G, d);
      const P2<T> hc = R.zq[1 + d][2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T rc = pc<T>(rpc, r), h = pc<T>(hc, r), p = pc<T>(pcc, r);
        const T fp = i4p16(lr, rc, r) * i4p16(lh, h, r) * T(1.0 / 256.0) - dih * (lp.p1[r] - p);
        const T fm = i4m16(lr, rc, r) * i4m16(lh, h, r) * T(1.0 / 256.0) - dih * (p - lp.m1[r]);
        ops[d][r] = fp;
        dsum[r] += fp - fm;
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
      ob[r] = -((pc<T>(rpc, r) - pc<T>(crho, r)) * idt + T(0.5) * pc<T>(cdp, r) + T(0.5) * dsum[r] * ih);
#pragma unroll
    for (int d = 0; d < 3; ++d) stp(ps[d] + c, ops[d][0], ops[d][1]);
    stp(b + c, ob[0], ob[1]);
    if (start) {
      const P2<T> cd = poly ? P2<T>{} : R.cen(2, k, tid);
      stp(r0 + c, ob[0], ob[1]);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        abb.add(ob[r], ob[r]);
        if (!poly) abz.add(ob[r], ob[r] * pc<T>(cd, r));
      }
    }
  }
  cp_async_wait<0>();
  if (!start) return;
  Red<T> v[2] = {abb.red(), abz.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      mix_finish_scalars(B, res[0], 1, rstart);
      cg_start_scalars(B, res[1], res[0], active);
    }
  }
}

// ---- launchers (0: the ring kernel could not be prepared) --------------------------------------
#define RGRID(bytes) L.nblocks, dim3(RTX, TY), (bytes), L.st
template <typename T>
int rlaunch_corr(const Launch& L, int s, int rhop, int pp, int pnew, int kset, int kidx, int mixed) {
  if (!L.ring_ok || !ring_ready<T>(mixed ? RK_CORR_M : RK_CORR_F)) return 0;
  constexpr int bm = CorrPlan<T, true>::bytes, bf = CorrPlan<T, false>::bytes;
  if (mixed)
    FE_LAUNCH(L, KID_CORR, (kr_corr<T, true><<<RGRID(bm)>>>(L.boxes, L.work, L.part, s, rhop, pp, pnew, kset, kidx,
                                                             mixed == 2 ? K_XH : K_X)));
  else
    FE_LAUNCH(L, KID_CORR, (kr_corr<T, false><<<RGRID(bf)>>>(L.boxes, L.work, L.part, s, rhop, pp, pnew, kset, kidx,
                                                              K_X)));
  return 1;
}

template <typename T>
int rlaunch_pred(const Launch& L, int s, int kset) {
  const bool tw = L.ysum >= 0;
  if (!L.ring_ok || !ring_ready<T>(tw ? RK_PRED_TW : RK_PRED)) return 0;
  if (tw)
    FE_LAUNCH(L, KID_PRED, (kr_pred<T, true><<<RGRID((PredPlan<T, true>::bytes))>>>(L.boxes, L.work, s, kset, L.ysum)));
  else
    FE_LAUNCH(L, KID_PRED, (kr_pred<T, false><<<RGRID(PredPlan<T>::bytes)>>>(L.boxes, L.work, s, kset, -1)));
  return 1;
}
template <typename T>
int rlaunch_asm(const Launch& L, int s, int up0, int php0, int rhop) {
  const bool tw = L.ysum >= 0;
  if (!L.ring_ok || !ring_ready<T>(tw ? RK_ASM_TW : RK_ASM)) return 0;
  if (tw)
    FE_LAUNCH(L, KID_ASM,
              (kr_asm<T, true><<<RGRID((AsmPlan<T, true>::bytes))>>>(L.boxes, L.work, s, up0, php0, rhop, L.ysum)));
  else
    FE_LAUNCH(L, KID_ASM, (kr_asm<T, false><<<RGRID(AsmPlan<T>::bytes)>>>(L.boxes, L.work, s, up0, php0, rhop, -1)));
  return 1;
}
template <typename T>
int rlaunch_accel(const Launch& L, int kset, int pk) {
  const bool tw = L.ysum >= 0;
  if (!L.ring_ok || !ring_ready<T>(tw ? RK_ACCEL_TW : RK_ACCEL)) return 0;
  if (tw)
    FE_LAUNCH(L, KID_ACCEL, (kr_accel<T, true><<<RGRID((AccelPlan<T, true>::bytes))>>>(L.boxes, L.work, kset, pk, L.ysum)));
  else
    FE_LAUNCH(L, KID_ACCEL, (kr_accel<T, false><<<RGRID(AccelPlan<T>::bytes)>>>(L.boxes, L.work, kset, pk, -1)));
  return 1;
}
template <typename T>
int rlaunch_fluxn(const Launch& L, int s, int nd) {
  if (nd < 1 || nd > 3 || !L.ring_ok || !ring_ready<T>(RK_FLUX1 + nd - 1)) return 0;
  switch (nd) {
    case 1: FE_LAUNCH(L, KID_FLUXN, (kr_fluxn<T, 1><<<RGRID((FluxPlan<T, 1>::bytes))>>>(L.boxes, L.work, s))); break;
    case 2: FE_LAUNCH(L, KID_FLUXN, (kr_fluxn<T, 2><<<RGRID((FluxPlan<T, 2>::bytes))>>>(L.boxes, L.work, s))); break;
    case 3: FE_LAUNCH(L, KID_FLUXN, (kr_fluxn<T, 3><<<RGRID((FluxPlan<T, 3>::bytes))>>>(L.boxes, L.work, s))); break;
    default: return 0;
  }
  return 1;
}
template <typename T, bool FR>
static int rlaunch_dust_any(const Launch& L, int s, int kset, int yp0, int yn0, int last, int nd, int enew) {
  if (nd < 1 || nd > 3 || !L.ring_ok || !ring_ready<T>((FR ? RK_DUST1F : RK_DUST1) + nd - 1)) return 0;
  switch (nd) {
    case 1:
      FE_LAUNCH(L, KID_DUST, (kr_dust<T, 1, FR><<<RGRID((DustPlan<T, 1, FR>::bytes))>>>(L.boxes, L.work, L.part, s, kset,
                                                                                         yp0, yn0, last, enew)));
      break;
    case 2:
      FE_LAUNCH(L, KID_DUST, (kr_dust<T, 2, FR><<<RGRID((DustPlan<T, 2, FR>::bytes))>>>(L.boxes, L.work, L.part, s, kset,
                                                                                         yp0, yn0, last, enew)));
      break;
    case 3:
      FE_LAUNCH(L, KID_DUST, (kr_dust<T, 3, FR><<<RGRID((DustPlan<T, 3, FR>::bytes))>>>(L.boxes, L.work, L.part, s, kset,
                                                                                         yp0, yn0, last, enew)));
      break;
    default: return 0;
  }
  return 1;
}
template <typename T>
int rlaunch_dust(const Launch& L, int s, int kset, int yp0, int yn0, int last, int nd) {
  return rlaunch_dust_any<T, false>(L, s, kset, yp0, yn0, last, nd, -1);
}
template <typename T>
int rlaunch_dust_fourier(const Launch& L, int s, int kset, int yp0, int yn0, int enew, int last, int nd) {
  return rlaunch_dust_any<T, true>(L, s, kset, yp0, yn0, last, nd, enew);
}

template <typename T>
int rlaunch_div(const Launch& L, int u0, int with_dt) {
  if (!L.ring_ok || !ring_ready<T>(RK_DIV)) return 0;
  FE_LAUNCH(L, KID_DIV, (kr_div<T><<<RGRID(DivPlan<T>::bytes)>>>(L.boxes, L.work, u0, L.part, with_dt)));
  return 1;
}
template <typename T>
int rlaunch_fe_cell(const Launch& L, int s, int u0, int rhos, int ps, int es, int tmode) {
  if (!L.ring_ok || !ring_ready<T>(RK_FECELL)) return 0;
  FE_LAUNCH(L, KID_FE_CELL, (kr_fe_cell<T><<<RGRID(FeCellPlan<T>::bytes)>>>(L.boxes, L.work, s, u0, rhos, ps, es,
                                                                             tmode)));
  return 1;
}
template <typename T>
int rlaunch_fe_face(const Launch& L, int u0, int phi0) {
  if (!L.ring_ok || !ring_ready<T>(RK_FEFACE)) return 0;
  FE_LAUNCH(L, KID_FE_FACE, (kr_fe_face<T><<<RGRID(FeFacePlan<T>::bytes)>>>(L.boxes, L.work, u0, phi0)));
  return 1;
}
template <typename T>
int rlaunch_rhs(const Launch& L, int s, int rhop, int pp) {
  if (!L.ring_ok || !ring_ready<T>(RK_RHS)) return 0;
  FE_LAUNCH(L, KID_RHS,
            (kr_rhs<T><<<RGRID(RhsPlan<T>::bytes)>>>(L.boxes, L.work, s, rhop, pp, L.part, L.rstart, L.active,
                                                     L.poly)));
  return 1;
}

template <typename T>
int rprepare() {
  const int dev = current_device();
  if (dev < 0) return 0;
  unsigned ok = 0;
  auto set = [&](int bit, bool accepted) { ok |= accepted ? 1u << bit : 0u; };
  set(RK_CORR_M, set_smem(kr_corr<T, true>, CorrPlan<T, true>::bytes));
  set(RK_CORR_F, set_smem(kr_corr<T, false>, CorrPlan<T, false>::bytes));
  set(RK_PRED, set_smem(kr_pred<T, false>, PredPlan<T>::bytes));
  set(RK_ASM, set_smem(kr_asm<T, false>, AsmPlan<T>::bytes));
  set(RK_ACCEL, set_smem(kr_accel<T, false>, AccelPlan<T>::bytes));
  set(RK_PRED_TW, set_smem(kr_pred<T, true>, PredPlan<T, true>::bytes));
  set(RK_ASM_TW, set_smem(kr_asm<T, true>, AsmPlan<T, true>::bytes));
  set(RK_ACCEL_TW, set_smem(kr_accel<T, true>, AccelPlan<T, true>::bytes));
  set(RK_FLUX1, set_smem(kr_fluxn<T, 1>, FluxPlan<T, 1>::bytes));
  set(RK_FLUX2, set_smem(kr_fluxn<T, 2>, FluxPlan<T, 2>::bytes));
  set(RK_FLUX3, set_smem(kr_fluxn<T, 3>, FluxPlan<T, 3>::bytes));
  set(RK_DUST1, set_smem(kr_dust<T, 1, false>, DustPlan<T, 1>::bytes));
  set(RK_DUST2, set_smem(kr_dust<T, 2, false>, DustPlan<T, 2>::bytes));
  set(RK_DUST3, set_smem(kr_dust<T, 3, false>, DustPlan<T, 3>::bytes));
  set(RK_DUST1F, set_smem(kr_dust<T, 1, true>, DustPlan<T, 1, true>::bytes));
  set(RK_DUST2F, set_smem(kr_dust<T, 2, true>, DustPlan<T, 2, true>::bytes));
  set(RK_DUST3F, set_smem(kr_dust<T, 3, true>, DustPlan<T, 3, true>::bytes));
  set(RK_DIV, set_smem(kr_div<T>, DivPlan<T>::bytes));
  set(RK_RHS, set_smem(kr_rhs<T>, RhsPlan<T>::bytes));
  set(RK_FECELL, set_smem(kr_fe_cell<T>, FeCellPlan<T>::bytes));
  set(RK_FEFACE, set_smem(kr_fe_face<T>, FeFacePlan<T>::bytes));
  cudaGetLastError();  // a refused limit is not an error of the context
  ok &= ~(unsigned)(FE_RING_OFF);
  RingReady<T>::ok[dev] = ok;
  return ok != 0;
}

#define RINST(T)                                                                \
  template int rlaunch_corr<T>(const Launch&, int, int, int, int, int, int, int); \
  template int rlaunch_pred<T>(const Launch&, int, int);                          \
  template int rlaunch_asm<T>(const Launch&, int, int, int, int);                 \
  template int rlaunch_accel<T>(const Launch&, int, int);                         \
  template int rlaunch_fluxn<T>(const Launch&, int, int);                         \
  template int rlaunch_dust<T>(const Launch&, int, int, int, int, int, int);      \
  template int rlaunch_dust_fourier<T>(const Launch&, int, int, int, int, int, int, int); \
  template int rlaunch_div<T>(const Launch&, int, int);                           \
  template int rlaunch_rhs<T>(const Launch&, int, int, int);                      \
  template int rlaunch_fe_cell<T>(const Launch&, int, int, int, int, int, int);   \
  template int rlaunch_fe_face<T>(const Launch&, int, int);                       \
  template int rprepare<T>();
RINST(double)
RINST(float)

}  // namespace fe
