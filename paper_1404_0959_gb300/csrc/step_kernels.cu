// step_kernels.cu -- the PISO step stencils (Sec. 2 par. 1 of arXiv:1404.0959:
// PISO, fourth-order central interpolation, adaptive dt; Sec. 2 par. 2:
// Equilibrium-Eulerian dust, Fourier / barotropic closure).
//
// The general kernels: the time-step maximum, the dust-loading sum, the
// Fourier closure's flux divergences and dust/energy update (and any number of
// dust classes), the transonic corrector and the derived initial fields; the
// other stages run the ring and z-marching kernels (step_rkernels.cu,
// step_zkernels.cu).  One thread owns one (i, j) column of a tile and walks its
// z-planes; every neighbour value is read through the read-only cache with
// periodic wrap.
// The viscous term uses the identity D tau(u)_m = mu (sum_d D G4_d u_m +
// Gc_m(div u)/3), which holds exactly for the stencils here because the Gauss
// gradients along different axes commute on the periodic grid; the face
// stress itself is formed only where the energy equation needs it.
#include "fe_internal.cuh"

namespace fe {

// z-marching shared-memory variants (step_zkernels.cu)
template <typename T> void zlaunch_div(const Launch& L, int u0);
template <typename T> void zlaunch_pred(const Launch& L, int s, int k);
template <typename T> void zlaunch_asm(const Launch& L, int s, int up0, int php0, int rhop);
template <typename T> void zlaunch_rhs(const Launch& L, int s, int rhop, int pp);
template <typename T> void zlaunch_corr(const Launch& L, int s, int rhop, int pp, int pnew, int kset, int kidx,
                                        int mixed);
template <typename T> void zlaunch_accel(const Launch& L, int kset, int pk);
template <typename T> void zlaunch_fluxn(const Launch& L, int s, int nd);
template <typename T> void zlaunch_dust(const Launch& L, int s, int kset, int yp0, int yn0, int last, int nd);

template <typename T>
__device__ __forceinline__ T* F(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

// offsets of "one cell back along d"
__device__ __forceinline__ int bx(int d) { return d == 0 ? -1 : 0; }
__device__ __forceinline__ int by(int d) { return d == 1 ? -1 : 0; }
__device__ __forceinline__ int bz(int d) { return d == 2 ? -1 : 0; }

// ---- Fourier closure: the total-energy face flux in two passes -------------------------------
// F_E = phi I4(H) - sum_m tau_dm I4(u_m) - kappa G4(T) on a d-face reads H and T at four cells
// along d and the Gauss gradients h Gc_m u_d at four cells along d for every face; evaluated inside
// the dust kernels it cost each face twice (from both of its cells) and hundreds of neighbour loads
// per cell.  Here (1) every cell's H = E + p/rho, T and h Gc_m u_l (nine) are formed once, (2) every
// cell's three +1/2 face fluxes once from star stencils of those, and the dust kernels difference
// the face arrays.  face stress tau_dm = mu (G4_d u_m + I4_d(Gc_m u_d) - 2/3 delta_dm I4_d(div u)).
//
// k_fe_cell: velocity slots u0..u0+2, density and pressure slots; E from slot es, or (es < 0) the
// level-n energy c_v T^n + |u^n|^2/2 of set s; T = T^n of set s (tmode 0) or p/(rho R) (tmode 1).
template <typename T>
__global__ void __launch_bounds__(NTHR) k_fe_cell(const BoxDev* boxes, const int2* work, int s, int u0, int rhos,
                                                  int ps, int es, int tmode) {
  Tile t = tile_of(boxes, work);
  if (!t.active) return;
  const BoxDev& B = boxes[t.box];
  const T* u[3] = {F<T>(B, u0), F<T>(B, u0 + 1), F<T>(B, u0 + 2)};
  const T* un[3] = {F<T>(B, S(s, F_U0)), F<T>(B, S(s, F_U1)), F<T>(B, S(s, F_U2))};
  const T* Tn = F<T>(B, S(s, F_T));
  const T* rho = F<T>(B, rhos);
  const T* p = F<T>(B, ps);
  const T* E = es >= 0 ? F<T>(B, es) : nullptr;
  T* __restrict__ Hc = F<T>(B, W_FEH);
  T* __restrict__ Tc = F<T>(B, W_FET);
  const T cv = (T)B.cv, Rg = (T)B.R;
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    const int c = n(0, 0, 0);
    T e;
    if (E) {
      e = __ldg(&E[c]);
    } else {  // the level-n energy, kept for the dust kernels (W_EN)
      const T uu = __ldg(&un[0][c]) * __ldg(&un[0][c]) + __ldg(&un[1][c]) * __ldg(&un[1][c]) +
                   __ldg(&un[2][c]) * __ldg(&un[2][c]);
      e = cv * __ldg(&Tn[c]) + T(0.5) * uu;
      F<T>(B, W_EN)[c] = e;
    }
    const T pc = __ldg(&p[c]), rc = __ldg(&rho[c]);
    Hc[c] = e + pc / rc;
    Tc[c] = tmode ? pc / (rc * Rg) : __ldg(&Tn[c]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int l = 0; l < 3; ++l) F<T>(B, W_FEG0 + 3 * m + l)[c] = Gc_h<T>(u[l], n, m, 0, 0, 0);
  }
}

// D(F_E) * (1/h) from the face arrays into slot out (the same sum as the dust kernels form)
template <typename T>
__global__ void __launch_bounds__(NTHR) k_fe_div(const BoxDev* boxes, const int2* work, int out) {
  Tile t = tile_of(boxes, work);
  if (!t.active) return;
  const BoxDev& B = boxes[t.box];
  const T ih = (T)B.ih;
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    const int c = n(0, 0, 0);
    T acc = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* fe = F<T>(B, W_FEF0 + d);
      acc += __ldg(&fe[c]) - __ldg(&fe[n(bx(d), by(d), bz(d))]);
    }
    F<T>(B, out)[c] = acc * ih;
  }
}

// k_fe_face: the three +1/2 face fluxes of every cell (face d of cell c between c and c + e_d) from
// k_fe_cell's fields, the velocity u0..u0+2, the face mass fluxes phi0..phi0+2 and W_DIV (div u).
template <typename T>
__global__ void __launch_bounds__(NTHR) k_fe_face(const BoxDev* boxes, const int2* work, int u0, int phi0) {
  Tile t = tile_of(boxes, work);
  if (!t.active) return;
  const BoxDev& B = boxes[t.box];
  const T* u[3] = {F<T>(B, u0), F<T>(B, u0 + 1), F<T>(B, u0 + 2)};
  const T* Hc = F<T>(B, W_FEH);
  const T* Tc = F<T>(B, W_FET);
  const T* div = F<T>(B, W_DIV);
  const T ih = (T)B.ih, mu = (T)B.mu, kappa = (T)B.kappa;
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    const int c = n(0, 0, 0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T hq[4], tq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = n.at(d, 0, 0, 0, q - 1);
        hq[q] = __ldg(&Hc[a]);
        tq[q] = __ldg(&Tc[a]);
      }
      const T IH = (T(9) * (hq[1] + hq[2]) - (hq[0] + hq[3])) * T(0.0625);
      const T G4T = (T(27) * (tq[2] - tq[1]) - (tq[3] - tq[0])) * T(1.0 / 24.0) * ih;
      T work = T(0);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const T* gmd = F<T>(B, W_FEG0 + 3 * m + d);  // h Gc_m u_d
        T g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) g[q] = __ldg(&gmd[n.at(d, 0, 0, 0, q - 1)]);
        const T ig = (T(9) * (g[1] + g[2]) - (g[0] + g[3])) * T(0.0625);
        T tau = (G4f_h<T>(u[m], n, d, 0, 0, 0) + ig) * ih;
        if (d == m) tau -= T(2.0 / 3.0) * I4f<T>(div, n, d, 0, 0, 0);
        work += (mu * tau) * I4f<T>(u[m], n, d, 0, 0, 0);
      }
      const T ph = __ldg(&F<T>(B, phi0 + d)[c]);
      F<T>(B, W_FEF0 + d)[c] = ph * IH - work - kappa * G4T;
    }
  }
}

// ---------------------------------------------------------------------------------
// a1: adaptive time step from max_i sum_d |u_d| of state s.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_dt(const BoxDev* boxes, const int2* ework, double* part, int s) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  const T* __restrict__ u0 = F<T>(B, S(s, F_U0));
  const T* __restrict__ u1 = F<T>(B, S(s, F_U1));
  const T* __restrict__ u2 = F<T>(B, S(s, F_U2));
  const int tid = threadIdx.x + TX * threadIdx.y;
  T m = T(0);
  for (int q0 = ch.begin + 4 * tid; q0 < ch.end; q0 += 4 * NTHR) {
    if (q0 + 4 <= ch.end) {
      V4<T> a = ld4(u0 + q0), b = ld4(u1 + q0), c = ld4(u2 + q0);
#pragma unroll
      for (int e = 0; e < 4; ++e) m = fmax(m, fabs(a.v[e]) + fabs(b.v[e]) + fabs(c.v[e]));
    } else {
      for (int c = q0; c < ch.end; ++c) m = fmax(m, fabs(u0[c]) + fabs(u1[c]) + fabs(u2[c]));
    }
  }
  __shared__ double res;
  if (block_max_last((double)m, B, part, &res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) finish_dt(B, res);
  }
}

// two-way coupling with several dust classes: W_YSUM = sum_j Y_j of set s, in class order
template <typename T>
__global__ void __launch_bounds__(NTHR) k_ysum(const BoxDev* boxes, const int2* ework, int s) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  T* __restrict__ out = F<T>(B, W_YSUM);
  const int tid = threadIdx.x + TX * threadIdx.y;
  for (int c = ch.begin + tid; c < ch.end; c += NTHR) {
    T v = F<T>(B, S(s, F_Y0))[c];
    for (int j = 1; j < B.nd; ++j) v = v + F<T>(B, S(s, F_Y0 + j))[c];
    out[c] = v;
  }
}

// n-level dust flux divergences D(phi_p^n I4 Y^n) and, Fourier, D(F_E^n).
template <typename T, bool FOURIER>
__global__ void __launch_bounds__(NTHR, FOURIER ? 1 : 2) k_fluxn(const BoxDev* boxes, const int2* work, int s) {
  Tile t = tile_of(boxes, work);
  if (!t.active) return;
  const BoxDev& B = boxes[t.box];
  const T* rho = F<T>(B, S(s, F_RHO));
  const T* u[3] = {F<T>(B, S(s, F_U0)), F<T>(B, S(s, F_U1)), F<T>(B, S(s, F_U2))};
  const T* phi[3] = {F<T>(B, S(s, F_PHI0)), F<T>(B, S(s, F_PHI1)), F<T>(B, S(s, F_PHI2))};
  const T* a[3] = {F<T>(B, W_AN0), F<T>(B, W_AN1), F<T>(B, W_AN2)};
  const T ih = (T)B.ih;
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    const int c = n(0, 0, 0);
    // mass-flux factor I4(rho) I4(a_d) per face, shared by all classes
    T ra_p[3], ra_m[3], ph_p[3], ph_m[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ra_p[d] = I4f<T>(rho, n, d, 0, 0, 0) * I4f<T>(a[d], n, d, 0, 0, 0);
      ra_m[d] = I4f<T>(rho, n, d, bx(d), by(d), bz(d)) * I4f<T>(a[d], n, d, bx(d), by(d), bz(d));
      ph_p[d] = __ldg(&phi[d][c]);
      ph_m[d] = __ldg(&phi[d][n(bx(d), by(d), bz(d))]);
    }
    for (int j = 0; j < B.nd; ++j) {
      const T* Y = F<T>(B, S(s, F_Y0 + j));
      const T tp = (T)B.tau_p[j];
      T acc = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T fp = (ph_p[d] - tp * ra_p[d]) * I4f<T>(Y, n, d, 0, 0, 0);
        T fm = (ph_m[d] - tp * ra_m[d]) * I4f<T>(Y, n, d, bx(d), by(d), bz(d));
        acc += fp - fm;
      }
      F<T>(B, W_FYN0 + j)[c] = acc * ih;
    }
    if (FOURIER) {  // D(F_E^n) from the face fluxes of k_fe_face
      T acc = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T* fe = F<T>(B, W_FEF0 + d);
        acc += __ldg(&fe[c]) - __ldg(&fe[n(bx(d), by(d), bz(d))]);
      }
      F<T>(B, W_FEN)[c] = acc * ih;
    }
  }
}

// a6: p^k, phi^k, u^k, rho^k from the correction x = p'; the true residual
// ||b - M x||^2 of the solve is accumulated on the way (same stencil reads).
template <typename T>
__global__ void __launch_bounds__(NTHR, 2) k_corr(const BoxDev* boxes, const int2* work, double* part, int s,
                                                int rhop, int pp, int pnew, int kset, int kidx, int mixed) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  const T* rho = F<T>(B, S(s, F_RHO));
  T* rk = F<T>(B, rhop);  // rho^{k-1} in, rho^k out (own cell only)
  const T* p = F<T>(B, pp);
  T* pn = F<T>(B, pnew);
  const T* x = F<T>(B, K_X);
  const T* b = F<T>(B, K_B);
  const T* psi = F<T>(B, W_PSI);
  const T* hb[3] = {F<T>(B, W_HB0), F<T>(B, W_HB1), F<T>(B, W_HB2)};
  const T* ps[3] = {F<T>(B, W_PS0), F<T>(B, W_PS1), F<T>(B, W_PS2)};
  const T* divphi = F<T>(B, W_DIVPHI);
  T* phk[3] = {F<T>(B, S(kset, F_PHI0)), F<T>(B, S(kset, F_PHI1)), F<T>(B, S(kset, F_PHI2))};
  T* uk[3] = {F<T>(B, S(kset, F_U0)), F<T>(B, S(kset, F_U1)), F<T>(B, S(kset, F_U2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], idt = T(1) / dt;
  const bool tr = B.transonic != 0;
  double rr = 0.0;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      const int c = n(0, 0, 0);
      const T xc = __ldg(&x[c]);
      const T psic = __ldg(&psi[c]);
      T dsum = T(0), lap = T(0), trd = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T xp = __ldg(&x[n.at(d, 0, 0, 0, 1)]), xm = __ldg(&x[n.at(d, 0, 0, 0, -1)]);
        T fp = __ldg(&ps[d][c]) - dt * (xp - xc) * ih;
        T fm = __ldg(&ps[d][n(bx(d), by(d), bz(d))]) - dt * (xc - xm) * ih;
        lap += (xp - xc) - (xc - xm);
        if (tr) {
          auto I4px = [&](int ox, int oy, int oz) {
            T v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              int id = n.at(d, ox, oy, oz, q - 1);
              v[q] = __ldg(&psi[id]) * __ldg(&x[id]);
            }
            return (T(9) * (v[1] + v[2]) - (v[0] + v[3])) * T(0.0625);
          };
          T tp = I4px(0, 0, 0) * I4f<T>(hb[d], n, d, 0, 0, 0);
          T tm = I4px(bx(d), by(d), bz(d)) * I4f<T>(hb[d], n, d, bx(d), by(d), bz(d));
          fp += tp;
          fm += tm;
          trd += tp - tm;
        }
        phk[d][c] = fp;
        dsum += fp - fm;
      }
      const T dtr = dt / rk[c];
      pn[c] = __ldg(&p[c]) + xc;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        T g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int sft = q < 2 ? q - 2 : q - 1;  // -2, -1, +1, +2
          int id = n.at(m, 0, 0, 0, sft);
          g[q] = __ldg(&p[id]) + __ldg(&x[id]);
        }
        T gp = (T(10) * (g[2] - g[1]) - (g[3] - g[0])) * T(0.0625) * ih;
        uk[m][c] = __ldg(&hb[m][c]) - dtr * gp;
      }
      rk[c] = __ldg(&rho[c]) - T(0.5) * dt * (__ldg(&divphi[c]) + dsum * ih);
      if (!mixed) {
        T Mx = psic * xc * idt - T(0.5) * dt * lap * ih * ih + T(0.5) * trd * ih;
        double r = (double)__ldg(&b[c]) - (double)Mx;
        rr += r * r;
      }
    }
  }
  Red<T> v[1] = {mixed ? Red<T>{} : red_from<T>(rr)};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      if (mixed) {  // FP64 refinement residual and total inner iterations
        B.sc[SC_RES0 + kidx] = B.sc[SC_ORES];
        B.sc[SC_IT0 + kidx] = B.sc[SC_ITSUM];
      } else {
        double bb = B.sc[SC_BB];
        B.sc[SC_RES0 + kidx] = bb > 0.0 ? sqrt(res[0] / bb) : 0.0;
        B.sc[SC_IT0 + kidx] = B.sc[SC_ITERS];
      }
    }
  }
}

// a7/a8: dust transport at level k, Fourier energy, and on the last
// corrector the closure plus the conserved totals and a non-finite count.
// eprev < 0: E^{k-1} = E^n from state s; enew < 0: last corrector (write T, p).
template <typename T, bool FOURIER>
__global__ void __launch_bounds__(NTHR, FOURIER ? 1 : 2) k_dust(const BoxDev* boxes, const int2* work, double* part, int s,
                                                int kset, int pk, int yp0, int yn0, int eprev, int enew,
                                                int last) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  const T* rhon = F<T>(B, S(s, F_RHO));
  const T* rho = F<T>(B, S(kset, F_RHO));
  const T* u[3] = {F<T>(B, S(kset, F_U0)), F<T>(B, S(kset, F_U1)), F<T>(B, S(kset, F_U2))};
  const T* phi[3] = {F<T>(B, S(kset, F_PHI0)), F<T>(B, S(kset, F_PHI1)), F<T>(B, S(kset, F_PHI2))};
  const T* a[3] = {F<T>(B, W_AN0), F<T>(B, W_AN1), F<T>(B, W_AN2)};
  const T* p = F<T>(B, pk);
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT];
  constexpr bool fourier = FOURIER;
  // totals of the last corrector: mass, energy (barotropic: 2 x kinetic),
  // non-finite count, dust mass per class
  SumAcc<T> amass, abad;
  DotAcc<T> aen, ady[MAXD];
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      const int c = n(0, 0, 0);
      const T rk = __ldg(&rho[c]);
      const T irk = T(1) / rk;
      const T rn = __ldg(&rhon[c]);
      T ra_p[3], ra_m[3], ph_p[3], ph_m[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ra_p[d] = I4f<T>(rho, n, d, 0, 0, 0) * I4f<T>(a[d], n, d, 0, 0, 0);
        ra_m[d] = I4f<T>(rho, n, d, bx(d), by(d), bz(d)) * I4f<T>(a[d], n, d, bx(d), by(d), bz(d));
        ph_p[d] = __ldg(&phi[d][c]);
        ph_m[d] = __ldg(&phi[d][n(bx(d), by(d), bz(d))]);
      }
      for (int j = 0; j < B.nd; ++j) {
        const T* Yp = F<T>(B, yp0 + j);
        const T tp = (T)B.tau_p[j];
        T fl = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          T fp = (ph_p[d] - tp * ra_p[d]) * I4f<T>(Yp, n, d, 0, 0, 0);
          T fm = (ph_m[d] - tp * ra_m[d]) * I4f<T>(Yp, n, d, bx(d), by(d), bz(d));
          fl += fp - fm;
        }
        T rY = rn * __ldg(&F<T>(B, S(s, F_Y0 + j))[c]) - T(0.5) * dt * (__ldg(&F<T>(B, W_FYN0 + j)[c]) + fl * ih);
        T Yk = rY * irk;
        F<T>(B, yn0 + j)[c] = Yk;
        if (last) {
          ady[j].add(rk, Yk);
          if (!isfinite(Yk)) abad.add(T(1));
        }
      }
      T Ek = T(0);
      if (fourier) {
        const T cv = (T)B.cv;
        const T* un[3] = {F<T>(B, S(s, F_U0)), F<T>(B, S(s, F_U1)), F<T>(B, S(s, F_U2))};
        const T* Tn = F<T>(B, S(s, F_T));
        auto En_at = [&](int q) {
          T uu = __ldg(&un[0][q]) * __ldg(&un[0][q]) + __ldg(&un[1][q]) * __ldg(&un[1][q]) +
                 __ldg(&un[2][q]) * __ldg(&un[2][q]);
          return cv * __ldg(&Tn[q]) + T(0.5) * uu;
        };
        T fl = T(0);  // D(F_E^k) from the face fluxes of k_fe_face
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T* fe = F<T>(B, W_FEF0 + d);
          fl += __ldg(&fe[c]) - __ldg(&fe[n(bx(d), by(d), bz(d))]);
        }
        T rE = rn * En_at(c) - T(0.5) * dt * (__ldg(&F<T>(B, W_FEN)[c]) + fl * ih);
        Ek = rE * irk;
        if (enew >= 0) F<T>(B, enew)[c] = Ek;
      }
      if (last) {
        T u0 = __ldg(&u[0][c]), u1 = __ldg(&u[1][c]), u2 = __ldg(&u[2][c]);
        T uu = u0 * u0 + u1 * u1 + u2 * u2;
        T pf;
        if (fourier) {
          T Tk = (Ek - T(0.5) * uu) / (T)B.cv;
          F<T>(B, S(kset, F_T))[c] = Tk;
          pf = rk * (T)B.R * Tk;
          aen.add(rk, Ek);
        } else {
          pf = pow(rk, (T)B.gamma) / (T)B.gamma;
          aen.add(rk, uu);
        }
        F<T>(B, S(kset, F_P))[c] = pf;
        amass.add(rk);
        if (!(isfinite(rk) && isfinite(uu) && isfinite(pf))) abad.add(T(1));
      }
    }
  }
  if (!last) return;
  Red<T> acc[3 + MAXD];
  acc[0] = amass.red();
  acc[1] = aen.red();
  acc[2] = abad.red();
#pragma unroll
  for (int j = 0; j < MAXD; ++j) acc[3 + j] = ady[j].red();
  __shared__ double res[3 + MAXD];
  if (block_sum_last<3 + MAXD>(acc, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_MASS] = res[0];
      B.sc[SC_ENERGY] = fourier ? res[1] : 0.5 * res[1];
      B.sc[SC_BAD] = res[2];
      for (int j = 0; j < MAXD; ++j) B.sc[SC_DUST0 + j] = res[3 + j];
    }
  }
}

// p from the closure and phi = I4(rho) I4(u_d) for state set s.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_derive(const BoxDev* boxes, const int2* work, int s, int only_box) {
  Tile t = tile_of(boxes, work);
  if (!t.active || (only_box >= 0 && t.box != only_box)) return;
  const BoxDev& B = boxes[t.box];
  const T* rho = F<T>(B, S(s, F_RHO));
  const T* u[3] = {F<T>(B, S(s, F_U0)), F<T>(B, S(s, F_U1)), F<T>(B, S(s, F_U2))};
  T* phi[3] = {F<T>(B, S(s, F_PHI0)), F<T>(B, S(s, F_PHI1)), F<T>(B, S(s, F_PHI2))};
  T* p = F<T>(B, S(s, F_P));
  for (int k = t.k0; k < t.kend; ++k) {
    Nbr n(t.i, t.j, k, B.N);
    const int c = n(0, 0, 0);
    const T r = __ldg(&rho[c]);
    if (B.closure == FE_FOURIER)
      p[c] = r * (T)B.R * __ldg(&F<T>(B, S(s, F_T))[c]);
    else
      p[c] = pow(r, (T)B.gamma) / (T)B.gamma;
#pragma unroll
    for (int d = 0; d < 3; ++d) phi[d][c] = I4f<T>(rho, n, d, 0, 0, 0) * I4f<T>(u[d], n, d, 0, 0, 0);
  }
}

// ---- launchers --------------------------------------------------------------------
#define GRID L.nblocks, dim3(TX, TY), 0, L.st
template <typename T> void launch_dt(const Launch& L, int s, int) {
  FE_LAUNCH(L, KID_DT, (k_dt<T><<<L.neblocks, dim3(TX, TY), 0, L.st>>>(L.boxes, L.ework, L.part, s)));
}
template <typename T> void launch_div(const Launch& L, int u0) { zlaunch_div<T>(L, u0); }
template <typename T> void launch_dt_div(const Launch& L, int s) {
  if (rlaunch_div<T>(L, S(s, F_U0), 1)) return;  // the ring divergence also takes the max for dt
  launch_dt<T>(L, s, 0);
  launch_div<T>(L, S(s, F_U0));
}
template <typename T> void launch_pred(const Launch& L, int s, int k) { zlaunch_pred<T>(L, s, k); }
// Fourier closure: the energy face fluxes of a level (k_fe_cell, then k_fe_face)
template <typename T> static void launch_fe_faces(const Launch& L, int s, int u0, int rhos, int ps, int es, int tmode,
                                                  int phi0) {
  if (!rlaunch_fe_cell<T>(L, s, u0, rhos, ps, es, tmode))
    FE_LAUNCH(L, KID_FE_CELL, (k_fe_cell<T><<<GRID>>>(L.boxes, L.work, s, u0, rhos, ps, es, tmode)));
  if (!rlaunch_fe_face<T>(L, u0, phi0)) FE_LAUNCH(L, KID_FE_FACE, (k_fe_face<T><<<GRID>>>(L.boxes, L.work, u0, phi0)));
}
template <typename T> void launch_fluxn(const Launch& L, int s) {
  if (!L.fourier && L.nd >= 1 && L.nd <= 3) {
    zlaunch_fluxn<T>(L, s, L.nd);
  } else if (L.fourier) {  // level n: E^n = c_v T^n + |u^n|^2/2, T^n stored
    launch_fe_faces<T>(L, s, S(s, F_U0), S(s, F_RHO), S(s, F_P), -1, 0, S(s, F_PHI0));
    if (L.nd >= 1 && L.nd <= 3) {  // D(F_E^n), then the dust flux divergences as in the barotropic step
      FE_LAUNCH(L, KID_FE_FACE, (k_fe_div<T><<<GRID>>>(L.boxes, L.work, W_FEN)));
      zlaunch_fluxn<T>(L, s, L.nd);
    } else {
      FE_LAUNCH(L, KID_FLUXN, (k_fluxn<T, true><<<GRID>>>(L.boxes, L.work, s)));
    }
  } else {
    FE_LAUNCH(L, KID_FLUXN, (k_fluxn<T, false><<<GRID>>>(L.boxes, L.work, s)));
  }
}
template <typename T> void launch_asm(const Launch& L, int s, int up0, int php0, int rhop) {
  zlaunch_asm<T>(L, s, up0, php0, rhop);
}
template <typename T> void launch_rhs(const Launch& L, int s, int rhop, int pp) { zlaunch_rhs<T>(L, s, rhop, pp); }
template <typename T> void launch_corr(const Launch& L, int s, int rhop, int pp, int pnew, int kset, int kidx,
                                       int mixed) {
  if (!L.transonic) zlaunch_corr<T>(L, s, rhop, pp, pnew, kset, kidx, mixed);
  else FE_LAUNCH(L, KID_CORR, (k_corr<T><<<GRID>>>(L.boxes, L.work, L.part, s, rhop, pp, pnew, kset, kidx, mixed)));
}
template <typename T> void launch_accel(const Launch& L, int kset, int pk) { zlaunch_accel<T>(L, kset, pk); }
template <typename T> void launch_dust(const Launch& L, int s, int kset, int pk, int yp0, int yn0, int eprev, int enew,
                                       int last, int) {
  if (!L.fourier && L.nd >= 1 && L.nd <= 3)
    zlaunch_dust<T>(L, s, kset, yp0, yn0, last, L.nd);
  else if (L.fourier) {  // level k: E^{k-1} (E^n in the first corrector), T = p^k / (rho^k R)
    launch_fe_faces<T>(L, s, S(kset, F_U0), S(kset, F_RHO), pk, eprev, 1, S(kset, F_PHI0));
    if (L.nd >= 1 && L.nd <= 3 && L.ring_ok) {  // D(F_E^k), then the ring kernel (when it can run)
      FE_LAUNCH(L, KID_FE_FACE, (k_fe_div<T><<<GRID>>>(L.boxes, L.work, W_FED)));
      if (rlaunch_dust_fourier<T>(L, s, kset, yp0, yn0, enew, last, L.nd)) return;
    }
    FE_LAUNCH(L, KID_DUST, (k_dust<T, true><<<GRID>>>(L.boxes, L.work, L.part, s, kset, pk, yp0, yn0, eprev, enew, last)));
  }
  else
    FE_LAUNCH(L, KID_DUST, (k_dust<T, false><<<GRID>>>(L.boxes, L.work, L.part, s, kset, pk, yp0, yn0, eprev, enew, last)));
}
template <typename T> void launch_ysum(const Launch& L, int s) {
  FE_LAUNCH(L, KID_OTHER, (k_ysum<T><<<L.neblocks, dim3(TX, TY), 0, L.st>>>(L.boxes, L.ework, s)));
}
template <typename T> void launch_derive_box(const Launch& L, int s, int box) {
  FE_LAUNCH(L, KID_DERIVE, (k_derive<T><<<GRID>>>(L.boxes, L.work, s, box)));
}

#define INST(T)                                                                              \
  template void launch_dt<T>(const Launch&, int, int);                                       \
  template void launch_div<T>(const Launch&, int);                                           \
  template void launch_dt_div<T>(const Launch&, int);                                        \
  template void launch_pred<T>(const Launch&, int, int);                                     \
  template void launch_fluxn<T>(const Launch&, int);                                         \
  template void launch_asm<T>(const Launch&, int, int, int, int);                            \
  template void launch_rhs<T>(const Launch&, int, int, int);                                 \
  template void launch_corr<T>(const Launch&, int, int, int, int, int, int, int);            \
  template void launch_accel<T>(const Launch&, int, int);                                    \
  template void launch_dust<T>(const Launch&, int, int, int, int, int, int, int, int, int);  \
  template void launch_derive_box<T>(const Launch&, int, int);                                \
  template void launch_ysum<T>(const Launch&, int);
INST(double)
INST(float)

}  // namespace fe
