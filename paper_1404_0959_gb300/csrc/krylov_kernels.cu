// krylov_kernels.cu -- matrix-free Krylov solvers for the pressure-correction
// equation of the PISO corrector (Sec. 2 par. 1 of arXiv:1404.0959 uses PISO;
// the paper does not name the linear solver).
//
//   M x = psi x / dt - dt/2 D(G2 x)  [+ 1/2 D(I4(psi x) I4(HbyA))  transonic]
//
// Jacobi-preconditioned CG (Hestenes-Stiefel) for the symmetric form and
// Jacobi-preconditioned BiCGStab (van der Vorst 1992) for any form.  Vectors
// have the field precision; every inner product is accumulated in double
// (per-thread, then a fixed-order warp/block tree, then the box's last block
// adds the block partials in order).  A box whose solve has finished skips
// every later launch, so one launch serves all boxes of an ensemble.
#include "fe_internal.cuh"

namespace fe {

template <typename T>
__device__ __forceinline__ T* F(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

__device__ __forceinline__ bool box_done(const BoxDev& B) { return B.sc[SC_DONE] != 0.0; }

// (M v)_c.  `scale` multiplies v element-wise first (the Jacobi
// preconditioner applied on the fly: pass inverse-diagonal mode).
template <typename T, bool PRE>
__device__ __forceinline__ T applyM(const BoxDev& B, const T* v, const Nbr& n, T dt, T ih) {
  const T* psi = F<T>(B, W_PSI);
  const T c3 = T(3) * dt * ih * ih;
  auto val = [&](int q) {
    T x = __ldg(&v[q]);
    if (PRE) x /= __ldg(&psi[q]) / dt + c3;
    return x;
  };
  const int c = n(0, 0, 0);
  const T vc = val(c);
  T lap = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) lap += (val(n.at(d, 0, 0, 0, 1)) - vc) - (vc - val(n.at(d, 0, 0, 0, -1)));
  T y = __ldg(&psi[c]) * vc / dt - T(0.5) * dt * lap * ih * ih;
  if (B.transonic) {
    T trd = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* hb = F<T>(B, W_HB0 + d);
      auto I4pv = [&](int ox, int oy, int oz) {
        T w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int id = n.at(d, ox, oy, oz, q - 1);
          w[q] = __ldg(&psi[id]) * val(id);
        }
        return (T(9) * (w[1] + w[2]) - (w[0] + w[3])) * T(0.0625);
      };
      T tp = I4pv(0, 0, 0) * I4f<T>(hb, n, d, 0, 0, 0);
      T tm = I4pv(d == 0 ? -1 : 0, d == 1 ? -1 : 0, d == 2 ? -1 : 0) *
             I4f<T>(hb, n, d, d == 0 ? -1 : 0, d == 1 ? -1 : 0, d == 2 ? -1 : 0);
      trd += tp - tm;
    }
    y += T(0.5) * trd * ih;
  }
  return y;
}

template <typename T>
__device__ __forceinline__ T jacobi_diag(const BoxDev& B, T psic, T dt) {
  return psic / dt + T(3) * dt * (T)B.ih * (T)B.ih;
}

// ---- CG ------------------------------------------------------------------------------
// r = b, x = 0, pd = z = b / diag; rz = <r, z>, bb = <b, b>.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_init(const BoxDev* boxes, const int2* work, double* part, int* active) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  const T* b = F<T>(B, K_B);
  const T* psi = F<T>(B, W_PSI);
  T* r = F<T>(B, K_R);
  T* x = F<T>(B, K_X);
  T* pd = F<T>(B, K_PD);
  const T dt = (T)B.sc[SC_KDT];
  double v[2] = {0.0, 0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      T bc = b[c];
      T z = bc / jacobi_diag<T>(B, psi[c], dt);
      r[c] = bc;
      x[c] = T(0);
      pd[c] = z;
      v[0] += (double)bc * (double)z;
      v[1] += (double)bc * (double)bc;
    }
  }
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_RZ] = res[0];
      B.sc[SC_BB] = res[1];
      B.sc[SC_ITERS] = 0.0;
      bool zero = !(res[1] > 0.0);
      B.sc[SC_DONE] = zero ? 1.0 : 0.0;
      B.sc[SC_CONV] = zero ? 1.0 : 0.0;
      if (!zero) atomicAdd(active, 1);
    }
  }
}

// q = M pd; alpha = rz / <pd, q>
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_matvec(const BoxDev* boxes, const int2* work, double* part) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* pd = F<T>(B, K_PD);
  T* q = F<T>(B, K_Q);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih;
  double v[1] = {0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      T y = applyM<T, false>(B, pd, n, dt, ih);
      q[c] = y;
      v[0] += (double)__ldg(&pd[c]) * (double)y;
    }
  }
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_PQ] = res[0];
      B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
    }
  }
}

// x += alpha pd; r -= alpha q; z = r / diag; convergence test on ||r||.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_update(const BoxDev* boxes, const int2* work, double* part, int* active) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* pd = F<T>(B, K_PD);
  const T* q = F<T>(B, K_Q);
  const T* psi = F<T>(B, W_PSI);
  T* x = F<T>(B, K_X);
  T* r = F<T>(B, K_R);
  const T dt = (T)B.sc[SC_KDT];
  const T alpha = (T)B.sc[SC_ALPHA];
  double v[2] = {0.0, 0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      x[c] = x[c] + alpha * pd[c];
      T rc = r[c] - alpha * q[c];
      r[c] = rc;
      T z = rc / jacobi_diag<T>(B, psi[c], dt);
      v[0] += (double)rc * (double)z;
      v[1] += (double)rc * (double)rc;
    }
  }
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double it = B.sc[SC_ITERS] + 1.0;
      B.sc[SC_ITERS] = it;
      B.sc[SC_RR] = res[1];
      if (sqrt(res[1]) <= B.sc[SC_TOL] * sqrt(B.sc[SC_BB])) {
        B.sc[SC_DONE] = 1.0;
        B.sc[SC_CONV] = 1.0;
        atomicSub(active, 1);
      } else if (it >= B.sc[SC_MAXIT]) {
        B.sc[SC_DONE] = 1.0;
        B.sc[SC_CONV] = 0.0;
        atomicSub(active, 1);
      } else {
        B.sc[SC_BETA] = res[0] / B.sc[SC_RZ];
        B.sc[SC_RZ] = res[0];
      }
    }
  }
}

// pd = r / diag + beta pd
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_dir(const BoxDev* boxes, const int2* work) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B) || !t.active) return;
  const T* r = F<T>(B, K_R);
  const T* psi = F<T>(B, W_PSI);
  T* pd = F<T>(B, K_PD);
  const T dt = (T)B.sc[SC_KDT];
  const T beta = (T)B.sc[SC_BETA];
  for (int k = t.k0; k < t.kend; ++k) {
    int c = t.i + B.N * (t.j + B.N * k);
    pd[c] = r[c] / jacobi_diag<T>(B, psi[c], dt) + beta * pd[c];
  }
}

// ||b - M x||^2 -> SC_TRUE_RR (x in slot xs)
template <typename T>
__global__ void __launch_bounds__(NTHR) k_true_res(const BoxDev* boxes, const int2* work, double* part, int xs) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  const T* x = F<T>(B, xs);
  const T* b = F<T>(B, K_B);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih;
  double v[1] = {0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      double r = (double)b[c] - (double)applyM<T, false>(B, x, n, dt, ih);
      v[0] += r * r;
    }
  }
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) B.sc[SC_TRUE_RR] = res[0];
  }
}

// ---- BiCGStab (right Jacobi preconditioning) -----------------------------------------
// r = rhat = b, x = p = v = 0; rho = <rhat, r> = bb; rho_old = alpha = omega = 1.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_bicg_init(const BoxDev* boxes, const int2* work, double* part, int* active) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  const T* b = F<T>(B, K_B);
  T* r = F<T>(B, K_R);
  T* rh = F<T>(B, K_RHAT);
  T* x = F<T>(B, K_X);
  T* p = F<T>(B, K_PD);
  T* v = F<T>(B, K_V);
  double a[1] = {0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      T bc = b[c];
      r[c] = bc;
      rh[c] = bc;
      x[c] = T(0);
      p[c] = T(0);
      v[c] = T(0);
      a[0] += (double)bc * (double)bc;
    }
  }
  __shared__ double res[1];
  if (block_sum_last<1>(a, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_BB] = res[0];
      B.sc[SC_RZ] = res[0];  // rho_i
      B.sc[SC_RHO_OLD] = 1.0;
      B.sc[SC_ALPHA] = 1.0;
      B.sc[SC_OMEGA] = 1.0;
      B.sc[SC_ITERS] = 0.0;
      bool zero = !(res[0] > 0.0);
      B.sc[SC_DONE] = zero ? 1.0 : 0.0;
      B.sc[SC_CONV] = zero ? 1.0 : 0.0;
      if (!zero) atomicAdd(active, 1);
    }
  }
}

// p = r + beta (p - omega v), beta = (rho / rho_old)(alpha / omega)
template <typename T>
__global__ void __launch_bounds__(NTHR) k_bicg_p(const BoxDev* boxes, const int2* work) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B) || !t.active) return;
  const T* r = F<T>(B, K_R);
  const T* v = F<T>(B, K_V);
  T* p = F<T>(B, K_PD);
  const double beta = (B.sc[SC_RZ] / B.sc[SC_RHO_OLD]) * (B.sc[SC_ALPHA] / B.sc[SC_OMEGA]);
  const T bt = (T)beta, om = (T)B.sc[SC_OMEGA];
  for (int k = t.k0; k < t.kend; ++k) {
    int c = t.i + B.N * (t.j + B.N * k);
    p[c] = r[c] + bt * (p[c] - om * v[c]);
  }
}

// v = M (p / diag); alpha = rho / <rhat, v>
template <typename T>
__global__ void __launch_bounds__(NTHR) k_bicg_v(const BoxDev* boxes, const int2* work, double* part) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* p = F<T>(B, K_PD);
  const T* rh = F<T>(B, K_RHAT);
  T* v = F<T>(B, K_V);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih;
  double a[1] = {0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      T y = applyM<T, true>(B, p, n, dt, ih);
      v[c] = y;
      a[0] += (double)rh[c] * (double)y;
    }
  }
  __shared__ double res[1];
  if (block_sum_last<1>(a, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_RV] = res[0];
      B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
    }
  }
}

// s = r - alpha v (stored), t = M (s / diag); omega = <t, s> / <t, t>
template <typename T>
__global__ void __launch_bounds__(NTHR) k_bicg_s(const BoxDev* boxes, const int2* work) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B) || !t.active) return;
  const T* r = F<T>(B, K_R);
  const T* v = F<T>(B, K_V);
  T* s = F<T>(B, K_S);
  const T alpha = (T)B.sc[SC_ALPHA];
  for (int k = t.k0; k < t.kend; ++k) {
    int c = t.i + B.N * (t.j + B.N * k);
    s[c] = r[c] - alpha * v[c];
  }
}

template <typename T>
__global__ void __launch_bounds__(NTHR) k_bicg_t(const BoxDev* boxes, const int2* work, double* part) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* s = F<T>(B, K_S);
  T* tv = F<T>(B, K_T);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih;
  double a[2] = {0.0, 0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      T y = applyM<T, true>(B, s, n, dt, ih);
      tv[c] = y;
      a[0] += (double)y * (double)__ldg(&s[c]);
      a[1] += (double)y * (double)y;
    }
  }
  __shared__ double res[2];
  if (block_sum_last<2>(a, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_TS] = res[0];
      B.sc[SC_TT] = res[1];
      B.sc[SC_OMEGA] = res[0] / res[1];
    }
  }
}

// x += alpha p/diag + omega s/diag; r = s - omega t; rho_old = rho, rho = <rhat, r>
template <typename T>
__global__ void __launch_bounds__(NTHR) k_bicg_x(const BoxDev* boxes, const int2* work, double* part, int* active) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* p = F<T>(B, K_PD);
  const T* s = F<T>(B, K_S);
  const T* tv = F<T>(B, K_T);
  const T* rh = F<T>(B, K_RHAT);
  const T* psi = F<T>(B, W_PSI);
  T* x = F<T>(B, K_X);
  T* r = F<T>(B, K_R);
  const T dt = (T)B.sc[SC_KDT];
  const T alpha = (T)B.sc[SC_ALPHA], om = (T)B.sc[SC_OMEGA];
  double a[2] = {0.0, 0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      T dg = jacobi_diag<T>(B, psi[c], dt);
      T sc = s[c];
      x[c] = x[c] + alpha * (p[c] / dg) + om * (sc / dg);
      T rc = sc - om * tv[c];
      r[c] = rc;
      a[0] += (double)rc * (double)rc;
      a[1] += (double)rh[c] * (double)rc;
    }
  }
  __shared__ double res[2];
  if (block_sum_last<2>(a, B, part, res)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double it = B.sc[SC_ITERS] + 1.0;
      B.sc[SC_ITERS] = it;
      B.sc[SC_RR] = res[0];
      B.sc[SC_RHO_OLD] = B.sc[SC_RZ];
      B.sc[SC_RZ] = res[1];
      if (sqrt(res[0]) <= B.sc[SC_TOL] * sqrt(B.sc[SC_BB])) {
        B.sc[SC_DONE] = 1.0;
        B.sc[SC_CONV] = 1.0;
        atomicSub(active, 1);
      } else if (it >= B.sc[SC_MAXIT]) {
        B.sc[SC_DONE] = 1.0;
        B.sc[SC_CONV] = 0.0;
        atomicSub(active, 1);
      }
    }
  }
}

// ---- launchers ------------------------------------------------------------------------
#define GRID L.nblocks, dim3(TX, TY), 0, L.st
template <typename T> void launch_cg_init(const Launch& L, double) {
  FE_LAUNCH(L, KID_CG_INIT, (k_cg_init<T><<<GRID>>>(L.boxes, L.work, L.part, L.active)));
}
template <typename T> void launch_cg_matvec(const Launch& L) {
  FE_LAUNCH(L, KID_CG_MATVEC, (k_cg_matvec<T><<<GRID>>>(L.boxes, L.work, L.part)));
}
template <typename T> void launch_cg_update(const Launch& L) {
  FE_LAUNCH(L, KID_CG_UPDATE, (k_cg_update<T><<<GRID>>>(L.boxes, L.work, L.part, L.active)));
}
template <typename T> void launch_cg_dir(const Launch& L) {
  FE_LAUNCH(L, KID_CG_DIR, (k_cg_dir<T><<<GRID>>>(L.boxes, L.work)));
}
template <typename T> void launch_true_res(const Launch& L, int xs) {
  FE_LAUNCH(L, KID_TRUE_RES, (k_true_res<T><<<GRID>>>(L.boxes, L.work, L.part, xs)));
}
template <typename T> void launch_bicg_init(const Launch& L) {
  FE_LAUNCH(L, KID_BICG_INIT, (k_bicg_init<T><<<GRID>>>(L.boxes, L.work, L.part, L.active)));
}
template <typename T> void launch_bicg_p(const Launch& L) {
  FE_LAUNCH(L, KID_BICG_P, (k_bicg_p<T><<<GRID>>>(L.boxes, L.work)));
}
template <typename T> void launch_bicg_v(const Launch& L) {
  FE_LAUNCH(L, KID_BICG_V, (k_bicg_v<T><<<GRID>>>(L.boxes, L.work, L.part)));
}
template <typename T> void launch_bicg_s(const Launch& L) {
  FE_LAUNCH(L, KID_BICG_S, (k_bicg_s<T><<<GRID>>>(L.boxes, L.work)));
  FE_LAUNCH(L, KID_BICG_T, (k_bicg_t<T><<<GRID>>>(L.boxes, L.work, L.part)));
}
template <typename T> void launch_bicg_x(const Launch& L) {
  FE_LAUNCH(L, KID_BICG_X, (k_bicg_x<T><<<GRID>>>(L.boxes, L.work, L.part, L.active)));
}

#define INST(T)                                                  \
  template void launch_cg_init<T>(const Launch&, double);        \
  template void launch_cg_matvec<T>(const Launch&);              \
  template void launch_cg_update<T>(const Launch&);              \
  template void launch_cg_dir<T>(const Launch&);                 \
  template void launch_true_res<T>(const Launch&, int);          \
  template void launch_bicg_init<T>(const Launch&);              \
  template void launch_bicg_p<T>(const Launch&);                 \
  template void launch_bicg_v<T>(const Launch&);                 \
  template void launch_bicg_s<T>(const Launch&);                 \
  template void launch_bicg_x<T>(const Launch&);
INST(double)
INST(float)

}  // namespace fe
