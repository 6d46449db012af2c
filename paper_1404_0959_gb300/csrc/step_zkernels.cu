// step_zkernels.cu -- z-marching shared-memory versions of the PISO stencil
// kernels (barotropic closure, symmetric pressure operator, up to 3 dust
// classes).  Same arithmetic as step_kernels.cu, which keeps the general
// versions (Fourier closure, transonic correction, more classes); see that
// file for the formulas (Sec. 2 of arXiv:1404.0959: PISO, fourth-order
// central interpolation, Equilibrium-Eulerian dust, barotropic closure).
#include "zmarch.cuh"

namespace fe {

template <typename T>
__device__ __forceinline__ T* Fz(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

// Face values of a face array at this cell's +1/2 face and at its -1/2 face
// (the neighbour's +1/2 face) along x, y, z; the z one is carried over planes.
template <typename T>
struct FaceBack {
  const T* __restrict__ f[3];
  int colxm, colym;  // flat (x-1, y) and (x, y-1) columns
  T zprev;           // f_z at (k-1) of the current column
  __device__ __forceinline__ void init(const T* fx, const T* fy, const T* fz, const ZGeom<2>& G, int k0) {
    f[0] = fx;
    f[1] = fy;
    f[2] = fz;
    const int gx = G.col % G.N, gy = G.col / G.N;
    colxm = (gx == 0 ? G.N - 1 : gx - 1) + G.N * gy;
    colym = gx + G.N * (gy == 0 ? G.N - 1 : gy - 1);
    zprev = __ldg(&f[2][G.col + G.plane(G.wrapz(k0 - 1))]);
  }
  // plus[d] = face value at +1/2, minus[d] at -1/2 for plane k
  __device__ __forceinline__ void get(const ZGeom<2>& G, int k, T (&plus)[3], T (&minus)[3]) {
    const int pk = G.plane(k);
    plus[0] = __ldg(&f[0][G.col + pk]);
    minus[0] = __ldg(&f[0][colxm + pk]);
    plus[1] = __ldg(&f[1][G.col + pk]);
    minus[1] = __ldg(&f[1][colym + pk]);
    plus[2] = __ldg(&f[2][G.col + pk]);
    minus[2] = zprev;
    zprev = plus[2];
  }
};

// ---- div -----------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_div(const BoxDev* boxes, const int2* work, int u0) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[3][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> u[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m].init(Fz<T>(B, u0 + m), sm[m], G, t.k0);
  T* __restrict__ div = Fz<T>(B, W_DIV);
  const T ih = (T)B.ih;
  for (int k = t.k0; k < t.kend; ++k) {
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].advance(G, k);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].stage(G, k);
    __syncthreads();
    if (G.active) div[G.col + G.plane(k)] = (zGc_h(u[0], G, 0) + zGc_h(u[1], G, 1) + zGc_h(u[2], G, 2)) * ih;
  }
}

// ---- predictor ------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_pred(const BoxDev* boxes, const int2* work, int s, int kset, int ysl) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[5][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> u[3], div, p;
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m].init(Fz<T>(B, S(s, F_U0 + m)), sm[m], G, t.k0);
  div.init(Fz<T>(B, W_DIV), sm[3], G, t.k0);
  p.init(Fz<T>(B, S(s, F_P)), sm[4], G, t.k0);
  FaceBack<T> phi;
  phi.init(Fz<T>(B, S(s, F_PHI0)), Fz<T>(B, S(s, F_PHI1)), Fz<T>(B, S(s, F_PHI2)), G, t.k0);
  const T* __restrict__ rho = Fz<T>(B, S(s, F_RHO));
  T* __restrict__ divphi = Fz<T>(B, W_DIVPHI);
  T* __restrict__ Rn[3] = {Fz<T>(B, W_RN0), Fz<T>(B, W_RN1), Fz<T>(B, W_RN2)};
  T* __restrict__ An[3] = {Fz<T>(B, W_AN0), Fz<T>(B, W_AN1), Fz<T>(B, W_AN2)};
  T* __restrict__ psi = Fz<T>(B, W_PSI);
  T* __restrict__ dinv = Fz<T>(B, W_DINV);
  T* __restrict__ rho0 = Fz<T>(B, S(kset, F_RHO));
  T* __restrict__ us[3] = {Fz<T>(B, S(kset, F_U0)), Fz<T>(B, S(kset, F_U1)), Fz<T>(B, S(kset, F_U2))};
  const T* __restrict__ ysum = ysl >= 0 ? Fz<T>(B, ysl) : nullptr;
  const T ih = (T)B.ih, mu = (T)B.mu, dt = (T)B.sc[SC_DT], gam = (T)B.gamma;
  const JacobiDiag<T> jd(B.sc[SC_DT], B.ih);
  for (int k = t.k0; k < t.kend; ++k) {
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].advance(G, k);
    div.advance(G, k);
    p.advance(G, k);
    T php[3], phm[3];
    phi.get(G, k, php, phm);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].stage(G, k);
    div.stage(G, k);
    p.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const T dph = ((php[0] - phm[0]) + (php[1] - phm[1]) + (php[2] - phm[2])) * ih;
    const T r = __ldg(&rho[c]);
    const T r0 = r - dt * dph;
    const T ir0 = rcp_rn(r0), ir = rcp_rn(r);
    T L[3], visc[3];
    zeval_L<T>(u, div, php, phm, G, ih, mu, L, visc);
    if (ysum) {  // two-way: a = (D tau - Gc p) / (rho (1 + Ysum)), R^n = L - (rho Ysum) a
      const T ys = __ldg(&ysum[c]);
      const T ia = rcp_rn(r * (T(1) + ys)), w = r * ys;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const T gp = zGc_h(p, G, m) * ih;
        const T a = (visc[m] - gp) * ia;
        const T Rf = L[m] - w * a;
        us[m][c] = (r * u[m].c() + dt * (Rf - gp)) * ir0;
        Rn[m][c] = Rf;
        An[m][c] = a;
      }
    } else {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const T gp = zGc_h(p, G, m) * ih;
        us[m][c] = (r * u[m].c() + dt * (L[m] - gp)) * ir0;
        Rn[m][c] = L[m];
        An[m][c] = (visc[m] - gp) * ir;
      }
    }
    const T ps = r / (gam * p.c());
    psi[c] = ps;
    dinv[c] = jd.inv(ps);
    divphi[c] = dph;
    rho0[c] = r0;
  }
}

// ---- corrector assembly ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_asm(const BoxDev* boxes, const int2* work, int s, int up0, int php0,
                                                int rhop, int ysl) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[4][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> u[3], div;
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m].init(Fz<T>(B, up0 + m), sm[m], G, t.k0);
  div.init(Fz<T>(B, W_DIV), sm[3], G, t.k0);
  FaceBack<T> phi;
  phi.init(Fz<T>(B, php0), Fz<T>(B, php0 + 1), Fz<T>(B, php0 + 2), G, t.k0);
  const T* __restrict__ rho = Fz<T>(B, S(s, F_RHO));
  const T* __restrict__ un[3] = {Fz<T>(B, S(s, F_U0)), Fz<T>(B, S(s, F_U1)), Fz<T>(B, S(s, F_U2))};
  const T* __restrict__ rp = Fz<T>(B, rhop);
  const T* __restrict__ Rn[3] = {Fz<T>(B, W_RN0), Fz<T>(B, W_RN1), Fz<T>(B, W_RN2)};
  T* __restrict__ hb[3] = {Fz<T>(B, W_HB0), Fz<T>(B, W_HB1), Fz<T>(B, W_HB2)};
  const T* __restrict__ ysum = ysl >= 0 ? Fz<T>(B, ysl) : nullptr;
  const T* __restrict__ An[3] = {Fz<T>(B, W_AN0), Fz<T>(B, W_AN1), Fz<T>(B, W_AN2)};
  const T ih = (T)B.ih, mu = (T)B.mu, dt = (T)B.sc[SC_DT];
  for (int k = t.k0; k < t.kend; ++k) {
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].advance(G, k);
    div.advance(G, k);
    T php[3], phm[3];
    phi.get(G, k, php, phm);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].stage(G, k);
    div.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    T L[3], visc[3];
    zeval_L<T>(u, div, php, phm, G, ih, mu, L, visc);
    const T r = __ldg(&rho[c]);
    const T rpv = __ldg(&rp[c]);
    const T irp = rcp_rn(rpv);
    if (ysum) {  // two-way: L^{k-1} - (rho^{k-1} Ysum) a, a the latest Du/Dt
      const T w = rpv * __ldg(&ysum[c]);
#pragma unroll
      for (int m = 0; m < 3; ++m) L[m] = L[m] - w * __ldg(&An[m][c]);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const T R = T(0.5) * (__ldg(&Rn[m][c]) + L[m]);
      hb[m][c] = (r * __ldg(&un[m][c]) + dt * R) * irp;
    }
  }
}

// ---- phi*, right-hand side ---------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_rhs(const BoxDev* boxes, const int2* work, int s, int rhop, int pp,
                                                double* part, int* rstart, int* active) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[5][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> rp, hb[3], p;
  rp.init(Fz<T>(B, rhop), sm[0], G, t.k0);
#pragma unroll
  for (int d = 0; d < 3; ++d) hb[d].init(Fz<T>(B, W_HB0 + d), sm[1 + d], G, t.k0);
  p.init(Fz<T>(B, pp), sm[4], G, t.k0);
  const T* __restrict__ rho = Fz<T>(B, S(s, F_RHO));
  const T* __restrict__ divphi = Fz<T>(B, W_DIVPHI);
  T* __restrict__ ps[3] = {Fz<T>(B, W_PS0), Fz<T>(B, W_PS1), Fz<T>(B, W_PS2)};
  // rstart: b to the refinement's copy and the first inner right-hand side, and the
  // refined solve started (as in kr_rhs)
  const bool start = rstart != nullptr;
  T* __restrict__ b = Fz<T>(B, start ? K_AUX : K_B);
  T* __restrict__ r0 = Fz<T>(B, K_R);
  const T* __restrict__ dinv = Fz<T>(B, W_DINV);
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], idt = T(1) / dt;
  DotAcc<T> abb, abz;
  for (int k = t.k0; k < t.kend; ++k) {
    rp.advance(G, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) hb[d].advance(G, k);
    p.advance(G, k);
    __syncthreads();
    rp.stage(G, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) hb[d].stage(G, k);
    p.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    T dsum = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T fp = zI4(rp, G, d, 0) * zI4(hb[d], G, d, 0) - dt * (p.at(G, d, 1) - p.c()) * ih;
      const T fm = zI4(rp, G, d, -1) * zI4(hb[d], G, d, -1) - dt * (p.c() - p.at(G, d, -1)) * ih;
      ps[d][c] = fp;
      dsum += fp - fm;
    }
    const T bc = -((rp.c() - __ldg(&rho[c])) * idt + T(0.5) * __ldg(&divphi[c]) + T(0.5) * dsum * ih);
    b[c] = bc;
    if (start) {
      r0[c] = bc;
      abb.add(bc, bc);
      abz.add(bc, bc * __ldg(&dinv[c]));
    }
  }
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

// ---- correction (symmetric operator) ---------------------------------------------------------
// The staged field "pk" holds p^{k-1} + x (so Gc reads p^k directly).
template <typename T>
struct ZSum2 {
  ZField<T, 2> f;
  const T* __restrict__ g2;
  __device__ __forceinline__ T ld(int q) const { return __ldg(&f.g[q]) + __ldg(&g2[q]); }
  __device__ __forceinline__ void init(const T* a, const T* b2, T* smem, const ZGeom<2>& G, int k0) {
    f.g = a;
    f.sm = smem;
    g2 = b2;
#pragma unroll
    for (int s = -2; s < 2; ++s) f.q[2 + s + 1] = ld(G.col + G.plane(G.wrapz(k0 + s)));
    f.nq[0] = ld(G.col + G.plane(G.wrapz(k0 + 2)));
    f.nh[0] = G.hcol >= 0 ? ld(G.hcol + G.plane(k0)) : T(0);
  }
  __device__ __forceinline__ void advance(const ZGeom<2>& G, int k) {
#pragma unroll
    for (int s = 0; s < 4; ++s) f.q[s] = f.q[s + 1];
    f.q[4] = f.nq[0];
    f.nq[0] = ld(G.col + G.plane(G.wrapz(k + 3)));
  }
  __device__ __forceinline__ void stage(const ZGeom<2>& G, int k) {
    f.sm[G.csm] = f.q[2];
    if (G.hcol >= 0) {
      f.sm[G.hsm] = f.nh[0];
      f.nh[0] = ld(G.hcol + G.plane(G.wrapz(k + 1)));
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(NTHR, 2) kz_corr(const BoxDev* boxes, const int2* work, double* part, int s,
                                                   int rhop, int pp, int pnew, int kset, int kidx, int mixed) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[2][ZGeom<2>::H * ZGeom<2>::W];
  ZSum2<T> pk;
  ZField<T, 2> x;
  const int xs = mixed == 2 ? K_XH : K_X;  // the pressure correction (or the high parts of its pairs)
  pk.init(Fz<T>(B, pp), Fz<T>(B, xs), sm[0], G, t.k0);
  x.init(Fz<T>(B, xs), sm[1], G, t.k0);
  FaceBack<T> ps;
  ps.init(Fz<T>(B, W_PS0), Fz<T>(B, W_PS1), Fz<T>(B, W_PS2), G, t.k0);
  const T* __restrict__ rho = Fz<T>(B, S(s, F_RHO));
  T* rk = Fz<T>(B, rhop);  // rho^{k-1} in, rho^k out (own cell only)
  T* __restrict__ pn = Fz<T>(B, pnew);
  const T* __restrict__ b = Fz<T>(B, K_B);
  const T* __restrict__ psi = Fz<T>(B, W_PSI);
  const T* __restrict__ hb[3] = {Fz<T>(B, W_HB0), Fz<T>(B, W_HB1), Fz<T>(B, W_HB2)};
  const T* __restrict__ divphi = Fz<T>(B, W_DIVPHI);
  T* __restrict__ phk[3] = {Fz<T>(B, S(kset, F_PHI0)), Fz<T>(B, S(kset, F_PHI1)), Fz<T>(B, S(kset, F_PHI2))};
  T* __restrict__ uk[3] = {Fz<T>(B, S(kset, F_U0)), Fz<T>(B, S(kset, F_U1)), Fz<T>(B, S(kset, F_U2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], idt = T(1) / dt;
  double rr = 0.0;
  for (int k = t.k0; k < t.kend; ++k) {
    pk.advance(G, k);
    x.advance(G, k);
    T psp[3], psm[3];
    ps.get(G, k, psp, psm);
    __syncthreads();
    pk.stage(G, k);
    x.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const T xc = x.c();
    T dsum = T(0), lap = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T xp = x.at(G, d, 1), xm = x.at(G, d, -1);
      const T fp = psp[d] - dt * (xp - xc) * ih;
      const T fm = psm[d] - dt * (xc - xm) * ih;
      lap += (xp - xc) - (xc - xm);
      phk[d][c] = fp;
      dsum += fp - fm;
    }
    const T dtr = dt / rk[c];
    pn[c] = pk.f.c();
#pragma unroll
    for (int m = 0; m < 3; ++m) uk[m][c] = __ldg(&hb[m][c]) - dtr * (zGc_h(pk.f, G, m) * ih);
    rk[c] = __ldg(&rho[c]) - T(0.5) * dt * (__ldg(&divphi[c]) + dsum * ih);
    if (!mixed) {
      const T Mx = __ldg(&psi[c]) * xc * idt - T(0.5) * dt * lap * ih * ih;
      const double r = (double)__ldg(&b[c]) - (double)Mx;
      rr += r * r;
    }
  }
  Red<T> v[1] = {mixed ? Red<T>{} : red_from<T>(rr)};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      if (mixed) {
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

// ---- Du/Dt at level k ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_accel(const BoxDev* boxes, const int2* work, int kset, int pk, int ysl) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[5][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> u[3], div, p;
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m].init(Fz<T>(B, S(kset, F_U0 + m)), sm[m], G, t.k0);
  div.init(Fz<T>(B, W_DIV), sm[3], G, t.k0);
  p.init(Fz<T>(B, pk), sm[4], G, t.k0);
  const T* __restrict__ rho = Fz<T>(B, S(kset, F_RHO));
  T* __restrict__ a[3] = {Fz<T>(B, W_AN0), Fz<T>(B, W_AN1), Fz<T>(B, W_AN2)};
  const T* __restrict__ ysum = ysl >= 0 ? Fz<T>(B, ysl) : nullptr;
  const T ih = (T)B.ih, mu = (T)B.mu;
  for (int k = t.k0; k < t.kend; ++k) {
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].advance(G, k);
    div.advance(G, k);
    p.advance(G, k);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m].stage(G, k);
    div.stage(G, k);
    p.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    // inertia rho, or rho (1 + Ysum) with the dust's reaction (two-way)
    const T ir = ysum ? rcp_rn(__ldg(&rho[c]) * (T(1) + __ldg(&ysum[c]))) : rcp_rn(__ldg(&rho[c]));
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const T lap = zDG4_h2(u[m], G, 0) + zDG4_h2(u[m], G, 1) + zDG4_h2(u[m], G, 2);
      const T visc = mu * (lap * ih * ih + zGc_h(div, G, m) * ih * T(1.0 / 3.0));
      a[m][c] = (visc - zGc_h(p, G, m) * ih) * ir;
    }
  }
}

// ---- dust flux divergences and transport (ND classes, barotropic) ---------------------------
// n-level: FYN_j = D(phi_p^n I4 Y_j^n)
template <typename T, int ND>
__global__ void __launch_bounds__(NTHR) kz_fluxn(const BoxDev* boxes, const int2* work, int s) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[4 + ND][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> rho, a[3], Y[ND];
  rho.init(Fz<T>(B, S(s, F_RHO)), sm[0], G, t.k0);
#pragma unroll
  for (int d = 0; d < 3; ++d) a[d].init(Fz<T>(B, W_AN0 + d), sm[1 + d], G, t.k0);
#pragma unroll
  for (int j = 0; j < ND; ++j) Y[j].init(Fz<T>(B, S(s, F_Y0 + j)), sm[4 + j], G, t.k0);
  FaceBack<T> phi;
  phi.init(Fz<T>(B, S(s, F_PHI0)), Fz<T>(B, S(s, F_PHI1)), Fz<T>(B, S(s, F_PHI2)), G, t.k0);
  const T ih = (T)B.ih;
  T taup[ND];
  T* fyn[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    taup[j] = (T)B.tau_p[j];
    fyn[j] = Fz<T>(B, W_FYN0 + j);
  }
  for (int k = t.k0; k < t.kend; ++k) {
    rho.advance(G, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d].advance(G, k);
#pragma unroll
    for (int j = 0; j < ND; ++j) Y[j].advance(G, k);
    T php[3], phm[3];
    phi.get(G, k, php, phm);
    __syncthreads();
    rho.stage(G, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d].stage(G, k);
#pragma unroll
    for (int j = 0; j < ND; ++j) Y[j].stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    T ra_p[3], ra_m[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ra_p[d] = zI4(rho, G, d, 0) * zI4(a[d], G, d, 0);
      ra_m[d] = zI4(rho, G, d, -1) * zI4(a[d], G, d, -1);
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const T tp = taup[j];
      T acc = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d)
        acc += (php[d] - tp * ra_p[d]) * zI4(Y[j], G, d, 0) - (phm[d] - tp * ra_m[d]) * zI4(Y[j], G, d, -1);
      fyn[j][c] = acc * ih;
    }
  }
}

// level k: (rho Y)^k and Y^k; on the last corrector the barotropic closure,
// the FP64 totals and a non-finite count
template <typename T, int ND>
__global__ void __launch_bounds__(NTHR, 2) kz_dust(const BoxDev* boxes, const int2* work, double* part, int s,
                                                   int kset, int yp0, int yn0, int last) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<2> G(t.x0, t.y0, B.N);
  __shared__ T sm[4 + ND][ZGeom<2>::H * ZGeom<2>::W];
  ZField<T, 2> rho, a[3], Y[ND];
  rho.init(Fz<T>(B, S(kset, F_RHO)), sm[0], G, t.k0);
#pragma unroll
  for (int d = 0; d < 3; ++d) a[d].init(Fz<T>(B, W_AN0 + d), sm[1 + d], G, t.k0);
#pragma unroll
  for (int j = 0; j < ND; ++j) Y[j].init(Fz<T>(B, yp0 + j), sm[4 + j], G, t.k0);
  FaceBack<T> phi;
  phi.init(Fz<T>(B, S(kset, F_PHI0)), Fz<T>(B, S(kset, F_PHI1)), Fz<T>(B, S(kset, F_PHI2)), G, t.k0);
  const T* __restrict__ rhon = Fz<T>(B, S(s, F_RHO));
  const T* __restrict__ u[3] = {Fz<T>(B, S(kset, F_U0)), Fz<T>(B, S(kset, F_U1)), Fz<T>(B, S(kset, F_U2))};
  const T ih = (T)B.ih, dt = (T)B.sc[SC_DT], gam = (T)B.gamma;
  T taup[ND];
  const T* yold[ND];
  const T* fyn[ND];
  T* ynew[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    taup[j] = (T)B.tau_p[j];
    yold[j] = Fz<T>(B, S(s, F_Y0 + j));
    fyn[j] = Fz<T>(B, W_FYN0 + j);
    ynew[j] = Fz<T>(B, yn0 + j);
  }
  T* __restrict__ pout = Fz<T>(B, S(kset, F_P));
  // totals of the last corrector: mass, 2 x kinetic energy, non-finite count,
  // dust mass per class
  SumAcc<T> amass, abad;
  DotAcc<T> aen, ady[ND];
  for (int k = t.k0; k < t.kend; ++k) {
    rho.advance(G, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d].advance(G, k);
#pragma unroll
    for (int j = 0; j < ND; ++j) Y[j].advance(G, k);
    T php[3], phm[3];
    phi.get(G, k, php, phm);
    __syncthreads();
    rho.stage(G, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d].stage(G, k);
#pragma unroll
    for (int j = 0; j < ND; ++j) Y[j].stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    const T rk = rho.c();
    const T irk = rcp_rn(rk);
    const T rn = __ldg(&rhon[c]);
    T ra_p[3], ra_m[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ra_p[d] = zI4(rho, G, d, 0) * zI4(a[d], G, d, 0);
      ra_m[d] = zI4(rho, G, d, -1) * zI4(a[d], G, d, -1);
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const T tp = taup[j];
      T fl = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d)
        fl += (php[d] - tp * ra_p[d]) * zI4(Y[j], G, d, 0) - (phm[d] - tp * ra_m[d]) * zI4(Y[j], G, d, -1);
      const T rY = rn * __ldg(&yold[j][c]) - T(0.5) * dt * (__ldg(&fyn[j][c]) + fl * ih);
      const T Yk = rY * irk;
      ynew[j][c] = Yk;
      if (last) {
        ady[j].add(rk, Yk);
        if (!isfinite(Yk)) abad.add(T(1));
      }
    }
    if (last) {
      const T u0 = __ldg(&u[0][c]), u1 = __ldg(&u[1][c]), u2 = __ldg(&u[2][c]);
      const T uu = u0 * u0 + u1 * u1 + u2 * u2;
      const T pf = pow(rk, gam) / gam;
      pout[c] = pf;
      amass.add(rk);
      aen.add(rk, uu);
      if (!(isfinite(rk) && isfinite(uu) && isfinite(pf))) abad.add(T(1));
    }
  }
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
      B.sc[SC_ENERGY] = 0.5 * res[1];
      B.sc[SC_BAD] = res[2];
      for (int j = 0; j < MAXD; ++j) B.sc[SC_DUST0 + j] = j < ND ? res[3 + j] : 0.0;
    }
  }
}

// ---- launchers ---------------------------------------------------------------------------------
#define ZGRID L.nblocks, dim3(TX, TY), 0, L.st
template <typename T> void zlaunch_div(const Launch& L, int u0) {
  if (rlaunch_div<T>(L, u0)) return;
  FE_LAUNCH(L, KID_DIV, (kz_div<T><<<ZGRID>>>(L.boxes, L.work, u0)));
}
template <typename T> void zlaunch_pred(const Launch& L, int s, int k) {
  if (rlaunch_pred<T>(L, s, k)) return;
  FE_LAUNCH(L, KID_PRED, (kz_pred<T><<<ZGRID>>>(L.boxes, L.work, s, k, L.ysum)));
}
template <typename T> void zlaunch_asm(const Launch& L, int s, int up0, int php0, int rhop) {
  if (rlaunch_asm<T>(L, s, up0, php0, rhop)) return;
  FE_LAUNCH(L, KID_ASM, (kz_asm<T><<<ZGRID>>>(L.boxes, L.work, s, up0, php0, rhop, L.ysum)));
}
template <typename T> void zlaunch_rhs(const Launch& L, int s, int rhop, int pp) {
  if (rlaunch_rhs<T>(L, s, rhop, pp)) return;
  FE_LAUNCH(L, KID_RHS, (kz_rhs<T><<<ZGRID>>>(L.boxes, L.work, s, rhop, pp, L.part, L.rstart, L.active)));
}
template <typename T> void zlaunch_corr(const Launch& L, int s, int rhop, int pp, int pnew, int kset, int kidx,
                                        int mixed) {
  if (rlaunch_corr<T>(L, s, rhop, pp, pnew, kset, kidx, mixed)) return;
  FE_LAUNCH(L, KID_CORR, (kz_corr<T><<<ZGRID>>>(L.boxes, L.work, L.part, s, rhop, pp, pnew, kset, kidx, mixed)));
}
template <typename T> void zlaunch_accel(const Launch& L, int kset, int pk) {
  if (rlaunch_accel<T>(L, kset, pk)) return;
  FE_LAUNCH(L, KID_ACCEL, (kz_accel<T><<<ZGRID>>>(L.boxes, L.work, kset, pk, L.ysum)));
}
template <typename T> void zlaunch_fluxn(const Launch& L, int s, int nd) {
  if (rlaunch_fluxn<T>(L, s, nd)) return;
  switch (nd) {
    case 1: FE_LAUNCH(L, KID_FLUXN, (kz_fluxn<T, 1><<<ZGRID>>>(L.boxes, L.work, s))); break;
    case 2: FE_LAUNCH(L, KID_FLUXN, (kz_fluxn<T, 2><<<ZGRID>>>(L.boxes, L.work, s))); break;
    case 3: FE_LAUNCH(L, KID_FLUXN, (kz_fluxn<T, 3><<<ZGRID>>>(L.boxes, L.work, s))); break;
  }
}
template <typename T> void zlaunch_dust(const Launch& L, int s, int kset, int yp0, int yn0, int last, int nd) {
  if (rlaunch_dust<T>(L, s, kset, yp0, yn0, last, nd)) return;
  switch (nd) {
    case 1: FE_LAUNCH(L, KID_DUST, (kz_dust<T, 1><<<ZGRID>>>(L.boxes, L.work, L.part, s, kset, yp0, yn0, last))); break;
    case 2: FE_LAUNCH(L, KID_DUST, (kz_dust<T, 2><<<ZGRID>>>(L.boxes, L.work, L.part, s, kset, yp0, yn0, last))); break;
    case 3: FE_LAUNCH(L, KID_DUST, (kz_dust<T, 3><<<ZGRID>>>(L.boxes, L.work, L.part, s, kset, yp0, yn0, last))); break;
  }
}

#define ZINST(T)                                                                            \
  template void zlaunch_div<T>(const Launch&, int);                                         \
  template void zlaunch_pred<T>(const Launch&, int, int);                                   \
  template void zlaunch_asm<T>(const Launch&, int, int, int, int);                          \
  template void zlaunch_rhs<T>(const Launch&, int, int, int);                               \
  template void zlaunch_corr<T>(const Launch&, int, int, int, int, int, int, int);          \
  template void zlaunch_accel<T>(const Launch&, int, int);                                  \
  template void zlaunch_fluxn<T>(const Launch&, int, int);                                  \
  template void zlaunch_dust<T>(const Launch&, int, int, int, int, int, int);
ZINST(double)
ZINST(float)

}  // namespace fe
