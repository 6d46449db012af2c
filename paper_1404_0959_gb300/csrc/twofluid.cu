// twofluid.cu -- Eulerian two-fluid dust phase (the paper's Sec. 2 par. 2
// contrasts its Equilibrium-Eulerian model with the full Eulerian two-phase
// model, where the particle phase carries its own momentum).  Reading: dilute,
// pressureless, one-way coupled; per class j with bulk density sigma = rho Y
// and velocity V:
//     d sigma/dt + div(sigma V) = 0,  d(sigma V)/dt + div(sigma V V) = sigma (u - V)/tau_p.
// After the gas step n -> n+1 (the gas does not depend on the dust):
//   face flux of the carrier mass  phi_v,d = phi_d + I4_d(rho) I4_d(V_d - u_d),
//   dust mass flux F_d = phi_v,d I4_d(Y), momentum flux G_dm = F_d I4_d(V_m);
//   predictor sigma* = sigma^n - dt D(F^n), m* = sigma^n V^n - dt D(G^n);
//   corrector from the gas at n+1 and the predicted dust (Heun):
//   sigma = sigma^n - dt/2 [D(F^n) + D(F*)], m likewise;
//   backward-Euler drag after each stage: V = u^{n+1} + (m/sigma - u^{n+1}) tau/(tau + dt),
//   Y = sigma / rho^{n+1}.
// Two forms: the ring kernels (every box's N a multiple of the 16-byte chunk;
// one class per launch, its planes and the gas planes arriving in shared-memory
// rings by asynchronous copies, zring.cuh) and the general kernels (one thread
// walks the z-planes of a column; neighbours through the read-only cache with
// periodic wrap).  Both evaluate the same expressions in the same order.
#include "zring.cuh"

namespace fe {

__device__ __forceinline__ int tfx(int d) { return d == 0 ? -1 : 0; }
__device__ __forceinline__ int tfy(int d) { return d == 1 ? -1 : 0; }
__device__ __forceinline__ int tfz(int d) { return d == 2 ? -1 : 0; }

template <typename T>
__device__ __forceinline__ T* TF(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

// Five values of f along d around the cell (offsets -2..2)
template <typename T>
__device__ __forceinline__ void tf_win(const T* f, const Nbr& n, int d, T (&w)[5]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) w[q] = __ldg(&f[n.at(d, 0, 0, 0, q - 2)]);
}

// fourth-order interpolation to the face between window entries a+1 and a+2 (a = 0: minus face,
// a = 1: plus face), the same formula as I4f
template <typename T>
__device__ __forceinline__ T tf_i4(const T (&w)[5], int a) {
  return (T(9) * (w[a + 1] + w[a + 2]) - (w[a] + w[a + 3])) * T(0.0625);
}

// D(F) and D(G_m) of one class at one cell: gas (rho, u, phi), dust (Y, V).  Per direction one
// five-point window of each field gives both faces.
template <typename T>
__device__ __forceinline__ void tf_div(const T* rho, const T* const (&u)[3], const T* const (&phi)[3], const T* Y,
                                       const T* const (&V)[3], const Nbr& n, T ih, T& DF, T (&DG)[3]) {
  DF = T(0);
  DG[0] = DG[1] = DG[2] = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T wr[5], wu[5], wy[5], wv[3][5];
    tf_win<T>(rho, n, d, wr);
    tf_win<T>(u[d], n, d, wu);
    tf_win<T>(Y, n, d, wy);
#pragma unroll
    for (int m = 0; m < 3; ++m) tf_win<T>(V[m], n, d, wv[m]);
    const T php = __ldg(&phi[d][n(0, 0, 0)]);
    const T phm = __ldg(&phi[d][n(tfx(d), tfy(d), tfz(d))]);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int a = side ? 0 : 1;  // plus face: entries 1..4, minus face: 0..3
      const T sgn = side ? T(-1) : T(1);
      const T slip = tf_i4<T>(wv[d], a) - tf_i4<T>(wu, a);
      const T F = ((side ? phm : php) + tf_i4<T>(wr, a) * slip) * tf_i4<T>(wy, a);
      DF += sgn * F;
#pragma unroll
      for (int m = 0; m < 3; ++m) DG[m] += sgn * F * tf_i4<T>(wv[m], a);
    }
  }
  DF *= ih;
#pragma unroll
  for (int m = 0; m < 3; ++m) DG[m] *= ih;
}

// Predictor: n-level divergences into W_TFN (D(F), D(G_0..2)), predicted Y*, V* into W_TFS.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_tf_pred(const BoxDev* boxes, const int2* work, int s, int ks) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (!t.active) return;
  const T* rho = TF<T>(B, S(s, F_RHO));
  const T* u[3] = {TF<T>(B, S(s, F_U0)), TF<T>(B, S(s, F_U1)), TF<T>(B, S(s, F_U2))};
  const T* phi[3] = {TF<T>(B, S(s, F_PHI0)), TF<T>(B, S(s, F_PHI1)), TF<T>(B, S(s, F_PHI2))};
  const T* rho1 = TF<T>(B, S(ks, F_RHO));
  const T* u1[3] = {TF<T>(B, S(ks, F_U0)), TF<T>(B, S(ks, F_U1)), TF<T>(B, S(ks, F_U2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT];
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    const int c = n(0, 0, 0);
    const T rn = __ldg(&rho[c]), ir1 = T(1) / __ldg(&rho1[c]);
    for (int j = 0; j < B.nd; ++j) {
      const T* Y = TF<T>(B, S(s, F_Y0 + j));
      const T* V[3] = {TF<T>(B, S(s, F_V0 + 3 * j)), TF<T>(B, S(s, F_V0 + 3 * j + 1)),
                       TF<T>(B, S(s, F_V0 + 3 * j + 2))};
      T DF, DG[3];
      tf_div<T>(rho, u, phi, Y, V, n, ih, DF, DG);
      const T sig_n = rn * __ldg(&Y[c]);
      const T sig = sig_n - dt * DF;
      const T isig = T(1) / sig;
      const T tau = (T)B.tau_p[j];
      const T r = tau / (tau + dt);
      TF<T>(B, W_TFN0 + 4 * j)[c] = DF;
      TF<T>(B, W_TFS0 + 4 * j)[c] = sig * ir1;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        TF<T>(B, W_TFN0 + 4 * j + 1 + m)[c] = DG[m];
        const T mom = sig_n * __ldg(&V[m][c]) - dt * DG[m];
        const T um = __ldg(&u1[m][c]);
        TF<T>(B, W_TFS0 + 4 * j + 1 + m)[c] = um + (mom * isig - um) * r;
      }
    }
  }
}

// Corrector: Y^{n+1}, V^{n+1} into state set ks; dust-mass totals and the
// non-finite count (added to the gas step's) of the box.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_tf_corr(const BoxDev* boxes, const int2* work, double* part, int s,
                                                  int ks) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  const T* rhon = TF<T>(B, S(s, F_RHO));
  const T* rho1 = TF<T>(B, S(ks, F_RHO));
  const T* u1[3] = {TF<T>(B, S(ks, F_U0)), TF<T>(B, S(ks, F_U1)), TF<T>(B, S(ks, F_U2))};
  const T* phi1[3] = {TF<T>(B, S(ks, F_PHI0)), TF<T>(B, S(ks, F_PHI1)), TF<T>(B, S(ks, F_PHI2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], hdt = T(0.5) * dt;
  DotAcc<T> ady[MAXD];
  SumAcc<T> abad;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      const int c = n(0, 0, 0);
      const T rn = __ldg(&rhon[c]), r1 = __ldg(&rho1[c]);
      for (int j = 0; j < B.nd; ++j) {
        const T* Ys = TF<T>(B, W_TFS0 + 4 * j);
        const T* Vs[3] = {TF<T>(B, W_TFS0 + 4 * j + 1), TF<T>(B, W_TFS0 + 4 * j + 2), TF<T>(B, W_TFS0 + 4 * j + 3)};
        T DF, DG[3];
        tf_div<T>(rho1, u1, phi1, Ys, Vs, n, ih, DF, DG);
        const T sig_n = rn * __ldg(&TF<T>(B, S(s, F_Y0 + j))[c]);
        const T sig = sig_n - hdt * (__ldg(&TF<T>(B, W_TFN0 + 4 * j)[c]) + DF);
        const T isig = T(1) / sig;
        const T tau = (T)B.tau_p[j];
        const T r = tau / (tau + dt);
        const T Yk = sig / r1;
        TF<T>(B, S(ks, F_Y0 + j))[c] = Yk;
        ady[j].add(r1, Yk);
        bool bad = !isfinite(Yk);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const T mom = sig_n * __ldg(&TF<T>(B, S(s, F_V0 + 3 * j + m))[c]) -
                        hdt * (__ldg(&TF<T>(B, W_TFN0 + 4 * j + 1 + m)[c]) + DG[m]);
          const T um = __ldg(&u1[m][c]);
          const T Vm = um + (mom * isig - um) * r;
          TF<T>(B, S(ks, F_V0 + 3 * j + m))[c] = Vm;
          bad = bad || !isfinite(Vm);
        }
        if (bad) abad.add(T(1));
      }
    }
  }
  Red<T> acc[1 + MAXD];
  acc[0] = abad.red();
#pragma unroll
  for (int j = 0; j < MAXD; ++j) acc[1 + j] = ady[j].red();
  __shared__ double res[1 + MAXD];
  if (block_sum_last<1 + MAXD>(acc, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_BAD] += res[0];
      for (int j = 0; j < B.nd; ++j) B.sc[SC_DUST0 + j] = res[1 + j];
    }
  }
}

// ---- ring forms (one class j per launch) --------------------------------------------------------
// D(F) and D(G_m) of both cells of the pair from the carrier density, the carrier velocity, the class's
// Y and V (stencil fields 0, 1..3, 4, 5..7) and the carrier face fluxes: the expressions of tf_div
// (I4 to the +1/2 face from offsets -1..2, to the -1/2 face from -2..1), with the lines of the six
// fields along each axis read once and 16 I4 evaluated unscaled, the factors folded.
template <typename T, typename RP, typename GT>
__device__ __forceinline__ void tfr_div(const RP& R, const GT& G, int k, T ih, T (&DF)[2], T (&DG)[3][2]) {
  T php[3][2], phm[3][2];
  R.faces2(0, k, G, php, phm);
  T dg[3][2] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}}, df[2] = {T(0), T(0)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const Line2<T> lr = ring_line(R, 0, k, G, d), ly = ring_line(R, 4, k, G, d), lu = ring_line(R, 1 + d, k, G, d);
    const Line2<T> lv[3] = {ring_line(R, 5, k, G, d), ring_line(R, 6, k, G, d), ring_line(R, 7, k, G, d)};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T rc = pc<T>(R.zq[0][2], r), yc = pc<T>(R.zq[4][2], r), uc = pc<T>(R.zq[1 + d][2], r);
      T vc[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) vc[m] = pc<T>(R.zq[5 + m][2], r);
      const T sp = i4p16(lv[d], vc[d], r) - i4p16(lu, uc, r), sm = i4m16(lv[d], vc[d], r) - i4m16(lu, uc, r);
      const T Fp = fma(i4p16(lr, rc, r) * T(1.0 / 256.0), sp, php[d][r]) * i4p16(ly, yc, r);
      const T Fm = fma(i4m16(lr, rc, r) * T(1.0 / 256.0), sm, phm[d][r]) * i4m16(ly, yc, r);
      df[r] += Fp - Fm;
#pragma unroll
      for (int m = 0; m < 3; ++m) dg[m][r] += Fp * i4p16(lv[m], vc[m], r) - Fm * i4m16(lv[m], vc[m], r);
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    DF[r] = df[r] * (ih * T(0.0625));
#pragma unroll
    for (int m = 0; m < 3; ++m) DG[m][r] = dg[m][r] * (ih * T(1.0 / 256.0));
  }
}

#define TF_RING_PROLOGUE(P)                              \
  const TileXYZ t = tile_xyz(boxes, work);               \
  const BoxDev& B = boxes[t.box];                        \
  const RGeom<T> G(t.x0, t.y0, B.N);                     \
  const int tid = threadIdx.x + RTX * threadIdx.y;       \
  extern __shared__ __align__(16) unsigned char rsm[];   \
  P R;                                                   \
  R.init(rsm, t.k0, t.kend)

// predictor: rho^n, u^n (3), Y^n_j, V^n_j (3) | phi^n | rho^{n+1}, u^{n+1} (3)
template <typename T>
using TfPredPlan = RingPlan<T, 1, 8, 3, 4>;
template <typename T>
__global__ void __launch_bounds__(RNT) kr_tf_pred(const BoxDev* boxes, const int2* work, int s, int ks, int j) {
  TF_RING_PROLOGUE(TfPredPlan<T>);
  R.gs[0] = TF<T>(B, S(s, F_RHO));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[1 + m] = TF<T>(B, S(s, F_U0 + m));
  R.gs[4] = TF<T>(B, S(s, F_Y0 + j));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[5 + m] = TF<T>(B, S(s, F_V0 + 3 * j + m));
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = TF<T>(B, S(s, F_PHI0 + d));
  R.gc[0] = TF<T>(B, S(ks, F_RHO));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[1 + m] = TF<T>(B, S(ks, F_U0 + m));
  T* __restrict__ tfn = TF<T>(B, W_TFN0 + 4 * j);
  T* __restrict__ tfs = TF<T>(B, W_TFS0 + 4 * j);
  T* __restrict__ tfn_m[3] = {TF<T>(B, W_TFN0 + 4 * j + 1), TF<T>(B, W_TFN0 + 4 * j + 2), TF<T>(B, W_TFN0 + 4 * j + 3)};
  T* __restrict__ tfs_m[3] = {TF<T>(B, W_TFS0 + 4 * j + 1), TF<T>(B, W_TFS0 + 4 * j + 2), TF<T>(B, W_TFS0 + 4 * j + 3)};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT];
  const T tau = (T)B.tau_p[j];
  const T rr = tau / (tau + dt);
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> cr1 = R.cen(0, k, tid);
    const P2<T> cu1[3] = {R.cen(1, k, tid), R.cen(2, k, tid), R.cen(3, k, tid)};
    T oDF[2], oDG[3][2], oY[2], oV[3][2];
    T DF[2], DG[3][2];
    tfr_div<T>(R, G, k, ih, DF, DG);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T rn = pc<T>(R.zq[0][2], r), ir1 = T(1) / pc<T>(cr1, r);
      const T sig_n = rn * pc<T>(R.zq[4][2], r);
      const T sig = sig_n - dt * DF[r];
      const T isig = T(1) / sig;
      oDF[r] = DF[r];
      oY[r] = sig * ir1;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        oDG[m][r] = DG[m][r];
        const T mom = sig_n * pc<T>(R.zq[5 + m][2], r) - dt * DG[m][r];
        const T um = pc<T>(cu1[m], r);
        oV[m][r] = um + (mom * isig - um) * rr;
      }
    }
    stp(tfn + c, oDF[0], oDF[1]);
    stp(tfs + c, oY[0], oY[1]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      stp(tfn_m[m] + c, oDG[m][0], oDG[m][1]);
      stp(tfs_m[m] + c, oV[m][0], oV[m][1]);
    }
  }
  cp_async_wait<0>();
}

// corrector: rho^{n+1}, u^{n+1} (3), Y*_j, V*_j (3) | phi^{n+1} | rho^n, Y^n_j, D(F^n), D(G^n) (3), V^n_j (3)
template <typename T>
using TfCorrPlan = RingPlan<T, 1, 8, 3, 9>;
template <typename T>
__global__ void __launch_bounds__(RNT) kr_tf_corr(const BoxDev* boxes, const int2* work, double* part, int s, int ks,
                                                  int j) {
  TF_RING_PROLOGUE(TfCorrPlan<T>);
  R.gs[0] = TF<T>(B, S(ks, F_RHO));
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gs[1 + m] = TF<T>(B, S(ks, F_U0 + m));
#pragma unroll
  for (int q = 0; q < 4; ++q) R.gs[4 + q] = TF<T>(B, W_TFS0 + 4 * j + q);
#pragma unroll
  for (int d = 0; d < 3; ++d) R.gf[d] = TF<T>(B, S(ks, F_PHI0 + d));
  R.gc[0] = TF<T>(B, S(s, F_RHO));
  R.gc[1] = TF<T>(B, S(s, F_Y0 + j));
#pragma unroll
  for (int q = 0; q < 4; ++q) R.gc[2 + q] = TF<T>(B, W_TFN0 + 4 * j + q);
#pragma unroll
  for (int m = 0; m < 3; ++m) R.gc[6 + m] = TF<T>(B, S(s, F_V0 + 3 * j + m));
  T* __restrict__ yo = TF<T>(B, S(ks, F_Y0 + j));
  T* __restrict__ vo[3] = {TF<T>(B, S(ks, F_V0 + 3 * j)), TF<T>(B, S(ks, F_V0 + 3 * j + 1)),
                           TF<T>(B, S(ks, F_V0 + 3 * j + 2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], hdt = T(0.5) * dt;
  const T tau = (T)B.tau_p[j];
  const T rr = tau / (tau + dt);
  DotAcc<T> ady;
  SumAcc<T> abad;
  R.prologue(G);
  for (int i = 0; i < t.kend - t.k0; ++i) {
    const int k = t.k0 + i;
    R.next(G, i);
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const P2<T> crn = R.cen(0, k, tid), cyn = R.cen(1, k, tid), cfn = R.cen(2, k, tid);
    const P2<T> cgn[3] = {R.cen(3, k, tid), R.cen(4, k, tid), R.cen(5, k, tid)};
    const P2<T> cvn[3] = {R.cen(6, k, tid), R.cen(7, k, tid), R.cen(8, k, tid)};
    T oY[2], oV[3][2];
    T DF[2], DG[3][2];
    tfr_div<T>(R, G, k, ih, DF, DG);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T rn = pc<T>(crn, r), r1 = pc<T>(R.zq[0][2], r);
      const T sig_n = rn * pc<T>(cyn, r);
      const T sig = sig_n - hdt * (pc<T>(cfn, r) + DF[r]);
      const T isig = T(1) / sig;
      const T Yk = sig / r1;
      oY[r] = Yk;
      ady.add(r1, Yk);
      bool bad = !isfinite(Yk);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const T mom = sig_n * pc<T>(cvn[m], r) - hdt * (pc<T>(cgn[m], r) + DG[m][r]);
        const T um = pc<T>(R.zq[1 + m][2], r);
        const T Vm = um + (mom * isig - um) * rr;
        oV[m][r] = Vm;
        bad = bad || !isfinite(Vm);
      }
      if (bad) abad.add(T(1));
    }
    stp(yo + c, oY[0], oY[1]);
#pragma unroll
    for (int m = 0; m < 3; ++m) stp(vo[m] + c, oV[m][0], oV[m][1]);
  }
  cp_async_wait<0>();
  Red<T> acc[2] = {abad.red(), ady.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(acc, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_BAD] += res[0];
      B.sc[SC_DUST0 + j] = res[1];
    }
  }
}

// Dynamic shared-memory limits of the ring forms, set once per device outside any capture.
constexpr int kTfMaxDev = 64;
template <typename T>
struct TfReady {
  static int ok[kTfMaxDev];
};
template <typename T>
int TfReady<T>::ok[kTfMaxDev] = {};
template <typename T>
int tfprepare() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTfMaxDev) return 0;
  const bool a = cudaFuncSetAttribute(kr_tf_pred<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TfPredPlan<T>::bytes) == cudaSuccess;
  const bool b = cudaFuncSetAttribute(kr_tf_corr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TfCorrPlan<T>::bytes) == cudaSuccess;
  cudaGetLastError();  // a refused limit is not an error of the context
  TfReady<T>::ok[dev] = a && b ? 1 : -1;
  return a && b;
}
template <typename T>
static bool tf_ring_ready() {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kTfMaxDev && TfReady<T>::ok[dev] == 1;
}

// V = u (every class) in state set s: the dust starts with the gas velocity
template <typename T>
__global__ void __launch_bounds__(NTHR) k_tf_init(const BoxDev* boxes, const int2* work, int s, int only_box) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (!t.active || (only_box >= 0 && t.box != only_box)) return;
  for (int k = t.k0; k < t.kend; ++k) {
    const int c = t.i + B.N * (t.j + B.N * k);
    for (int j = 0; j < B.nd; ++j)
#pragma unroll
      for (int m = 0; m < 3; ++m) TF<T>(B, S(s, F_V0 + 3 * j + m))[c] = TF<T>(B, S(s, F_U0 + m))[c];
  }
}

#define TF_GRID L.nblocks, dim3(TX, TY), 0, L.st
template <typename T>
void launch_two_fluid(const Launch& L, int s, int ks) {
  if (L.ring_ok && tf_ring_ready<T>()) {  // one class per launch; predictor of every class first
    for (int j = 0; j < L.nd; ++j)
      FE_LAUNCH(L, KID_TF_PRED,
                (kr_tf_pred<T><<<L.nblocks, dim3(RTX, TY), TfPredPlan<T>::bytes, L.st>>>(L.boxes, L.work, s, ks, j)));
    for (int j = 0; j < L.nd; ++j)
      FE_LAUNCH(L, KID_TF_CORR, (kr_tf_corr<T><<<L.nblocks, dim3(RTX, TY), TfCorrPlan<T>::bytes, L.st>>>(
                                    L.boxes, L.work, L.part, s, ks, j)));
    return;
  }
  FE_LAUNCH(L, KID_TF_PRED, (k_tf_pred<T><<<TF_GRID>>>(L.boxes, L.work, s, ks)));
  FE_LAUNCH(L, KID_TF_CORR, (k_tf_corr<T><<<TF_GRID>>>(L.boxes, L.work, L.part, s, ks)));
}
template <typename T>
void launch_two_fluid_init(const Launch& L, int s, int box) {
  FE_LAUNCH(L, KID_OTHER, (k_tf_init<T><<<TF_GRID>>>(L.boxes, L.work, s, box)));
}
template void launch_two_fluid<double>(const Launch&, int, int);
template void launch_two_fluid<float>(const Launch&, int, int);
template void launch_two_fluid_init<double>(const Launch&, int, int);
template void launch_two_fluid_init<float>(const Launch&, int, int);
template int tfprepare<double>();
template int tfprepare<float>();

}  // namespace fe
