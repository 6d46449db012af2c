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
#include "zbulk.cuh"
#include "zmarch.cuh"
#include "zring.cuh"

namespace fe {

template <typename T>
__device__ __forceinline__ T* F(const BoxDev& B, int slot) {
  return reinterpret_cast<T*>(B.f[slot]);
}

__device__ __forceinline__ bool box_done(const BoxDev& B) { return B.sc[SC_DONE] != 0.0; }

// (M v)_c with v read through `val` (PRE: v scaled by the inverse Jacobi
// diagonal first, i.e. M D^{-1} v for right preconditioning).
template <typename T, bool PRE>
__device__ __forceinline__ T applyM(const BoxDev& B, const T* v, const Nbr& n, T dt, T ih) {
  const T* psi = F<T>(B, W_PSI);
  const T* dinv = F<T>(B, W_DINV);
  auto val = [&](int q) {
    T x = __ldg(&v[q]);
    if (PRE) x *= __ldg(&dinv[q]);
    return x;
  };
  const T idt = T(1) / dt;
  const int c = n(0, 0, 0);
  const T vc = val(c);
  T lap = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) lap += (val(n.at(d, 0, 0, 0, 1)) - vc) - (vc - val(n.at(d, 0, 0, 0, -1)));
  T y = __ldg(&psi[c]) * vc * idt - T(0.5) * dt * lap * ih * ih;
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

// The operator in FP64 on the double-float correction (transonic refinement residuals).
template <typename T>
__device__ __forceinline__ double applyM64_pairs(const BoxDev& B, const float2* xs, const Nbr& n, double dt) {
  const T* psi = F<T>(B, W_PSI);
  const double ih = B.ih, idt = 1.0 / dt;
  auto v = [&](int q) {
    const float2 a = xs[q];
    return (double)a.x + (double)a.y;
  };
  const int c = n(0, 0, 0);
  const double vc = v(c);
  double lap = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) lap += (v(n.at(d, 0, 0, 0, 1)) - vc) - (vc - v(n.at(d, 0, 0, 0, -1)));
  double y = (double)__ldg(&psi[c]) * vc * idt - 0.5 * dt * lap * ih * ih;
  if (B.transonic) {
    double trd = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* hb = F<T>(B, W_HB0 + d);
      auto I4pv = [&](int ox, int oy, int oz) {
        double w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int id = n.at(d, ox, oy, oz, q - 1);
          w[q] = (double)__ldg(&psi[id]) * v(id);
        }
        return (9.0 * (w[1] + w[2]) - (w[0] + w[3])) * 0.0625;
      };
      double tp = I4pv(0, 0, 0) * I4f<double>(hb, n, d, 0, 0, 0);
      double tm = I4pv(d == 0 ? -1 : 0, d == 1 ? -1 : 0, d == 2 ? -1 : 0) *
                  I4f<double>(hb, n, d, d == 0 ? -1 : 0, d == 1 ? -1 : 0, d == 2 ? -1 : 0);
      trd += tp - tm;
    }
    y += 0.5 * trd * ih;
  }
  return y;
}

// ---- CG ------------------------------------------------------------------------------
// Element-wise CG kernels walk a flat chunk of the box with 16-byte accesses;
// each thread keeps two vectors of four cells in flight.
template <typename F4, typename F1>
__device__ __forceinline__ void chunk_loop(const Chunk& ch, int tid, F4 f4, F1 f1) {
  for (int q0 = ch.begin + 4 * tid; q0 < ch.end; q0 += 4 * NTHR) {
    if (q0 + 4 <= ch.end) {
      f4(q0);
    } else {
      for (int c = q0; c < ch.end; ++c) f1(c);
    }
  }
}

// r = b, x = 0, pd = z = b / diag; rz = <r, z>, bb = <b, b>.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_init(const BoxDev* boxes, const int2* work, double* part, int* active) {
  const Chunk ch = chunk_of(boxes, work);
  const BoxDev& B = boxes[ch.box];
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ b = F<T>(B, K_B);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ r = F<T>(B, K_R);
  T* __restrict__ x = F<T>(B, K_X);
  T* __restrict__ pd = F<T>(B, K_PD);
  const T keep = B.sc[SC_ODONE] != 0.0 ? T(0) : T(1);  // refinement already converged for this box
  DotAcc<T> a0, a1;
  chunk_loop(
      ch, tid,
      [&](int q0) {
        V4<T> bv = ld4(b + q0), dv = ld4(dinv + q0), zv, zero{{T(0), T(0), T(0), T(0)}};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          bv.v[e] *= keep;
          zv.v[e] = bv.v[e] * dv.v[e];
          a0.add(bv.v[e], zv.v[e]);
          a1.add(bv.v[e], bv.v[e]);
        }
        st4(r + q0, bv);
        st4(x + q0, zero);
        st4(pd + q0, zv);
      },
      [&](int c) {
        T bc = b[c] * keep;
        T z = bc * dinv[c];
        r[c] = bc;
        x[c] = T(0);
        pd[c] = z;
        a0.add(bc, z);
        a1.add(bc, bc);
      });
  Red<T> v[2] = {a0.red(), a1.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_RZ] = res[0];
      B.sc[SC_BB] = res[1];
      B.sc[SC_ITERS] = 0.0;
      B.sc[SC_ALPHA] = 0.0;
      B.sc[SC_BETA] = 0.0;
      bool zero = !(res[1] > 0.0);
      B.sc[SC_DONE] = zero ? 1.0 : 0.0;
      if (B.sc[SC_ODONE] == 0.0) B.sc[SC_CONV] = zero ? 1.0 : 0.0;  // a finished refinement keeps its verdict
      if (!zero) atomicAdd(active, 1);
    }
  }
}

// q = M pd; alpha = rz / <pd, q>.  Symmetric operator: each thread walks its
// (i, j) column through the tile's z-planes keeping pd at k-1, k, k+1 in
// registers; x and y neighbours come through the read-only cache.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_matvec(const BoxDev* boxes, const int2* work, double* part) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* __restrict__ pd = F<T>(B, K_PD);
  const T* __restrict__ psi = F<T>(B, W_PSI);
  T* __restrict__ q = F<T>(B, K_Q);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih, idt = T(1) / dt;
  const T lapc = T(0.5) * dt * ih * ih;
  DotAcc<T> a0;
  if (t.active) {
    const int N = B.N, NN = N * N;
    if (!B.transonic) {
      const int col = t.i + N * t.j;
      const int xm = (t.i == 0 ? N - 1 : t.i - 1) + N * t.j - col;
      const int xp = (t.i == N - 1 ? 0 : t.i + 1) + N * t.j - col;
      const int ym = t.i + N * (t.j == 0 ? N - 1 : t.j - 1) - col;
      const int yp = t.i + N * (t.j == N - 1 ? 0 : t.j + 1) - col;
      int km = t.k0 == 0 ? N - 1 : t.k0 - 1;
      T vm = __ldg(&pd[col + NN * km]);
      T vc = __ldg(&pd[col + NN * t.k0]);
#pragma unroll 2
      for (int k = t.k0; k < t.kend; ++k) {
        const int kp = k == N - 1 ? 0 : k + 1;
        const int c = col + NN * k;
        const T vp = __ldg(&pd[col + NN * kp]);
        const T nb = (__ldg(&pd[c + xm]) + __ldg(&pd[c + xp])) + (__ldg(&pd[c + ym]) + __ldg(&pd[c + yp])) + (vm + vp);
        const T y = __ldg(&psi[c]) * vc * idt - lapc * (nb - T(6) * vc);
        q[c] = y;
        a0.add(vc, y);
        vm = vc;
        vc = vp;
      }
    } else {
      for (int k = t.k0; k < t.kend; ++k) {
        Nbr n(t.i, t.j, k, N);
        int c = n(0, 0, 0);
        T y = applyM<T, false>(B, pd, n, dt, ih);
        q[c] = y;
        a0.add(__ldg(&pd[c]), y);
      }
    }
  }
  Red<T> v[1] = {a0.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_PQ] = res[0];
      B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
    }
  }
}

// Planes requested ahead by the z-marching Krylov kernels, minimum resident
// blocks per SM of the fused CG kernel (FP32), shared-memory plane buffers
// (2: the next plane is staged while the current one is read, one barrier per
// plane), and minimum resident blocks per SM of the column-pair refinement
// boundary (5: 96 registers instead of 122, one more block of four warps per
// SM to cover its global-load latency).
#ifndef FE_KPF
#define FE_KPF 2
#endif
#ifndef FE_DM_MINB
#define FE_DM_MINB 4
#endif
#ifndef FE_DM_NBUF
#define FE_DM_NBUF 2
#endif
#ifndef FE_REFINE_MINB
#define FE_REFINE_MINB 5
#endif
constexpr int KPF = FE_KPF;
constexpr int kDmBuf = FE_DM_NBUF;

// q = M pd; alpha = rz / <pd, q> (symmetric operator): z-marching form, pd
// staged per plane in shared memory with a 1-cell halo, z-neighbours in
// registers, loads issued KPF planes ahead.
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_cg_matvec(const BoxDev* boxes, const int2* work, double* part) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const ZGeom<1> G(t.x0, t.y0, B.N);
  __shared__ T sm[ZGeom<1>::H * ZGeom<1>::W];
  ZField<T, 1, KPF> p;
  p.init(F<T>(B, K_PD), sm, G, t.k0);
  ZStream<T, KPF> psi;
  psi.init(F<T>(B, W_PSI), G, t.k0);
  T* __restrict__ q = F<T>(B, K_Q);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih, idt = T(1) / dt;
  const T lapc = T(0.5) * dt * ih * ih;
  DotAcc<T> a0;
  for (int k = t.k0; k < t.kend; ++k) {
    p.advance(G, k);
    const T ps = psi.next(G, k);
    __syncthreads();
    p.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    const T vc = p.c();
    const T nb = (p.at(G, 0, -1) + p.at(G, 0, 1)) + (p.at(G, 1, -1) + p.at(G, 1, 1)) + (p.at(G, 2, -1) + p.at(G, 2, 1));
    const T y = ps * vc * idt - lapc * (nb - T(6) * vc);
    q[G.col + G.plane(k)] = y;
    a0.add(vc, y);
  }
  Red<T> v[1] = {a0.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_PQ] = res[0];
      B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
    }
  }
}

// One CG iteration's direction and operator in one pass (symmetric operator):
//   pd_new = D^{-1} r + beta pd_old,  x += alpha pd_old,  q = M pd_new,
//   alpha = rz / <pd_new, q>.
// x therefore lags one direction behind; k_cg_xfinal adds the last one.
// pd_old and pd_new alternate between slots K_PD and K_PP with the parity of
// the iteration counter (neighbouring tiles still read pd_old as halo).  At
// iteration 0 alpha = beta = 0 (set by k_cg_init) and pd_new = D^{-1} b.
// POLY: pd_new = z + beta pd_old with z = P r from kz_cg_rpoly (the first-order Neumann
// polynomial preconditioner), z read in place of r and D^{-1}.
template <typename T, bool POLY>
__global__ void __launch_bounds__(NTHR, sizeof(T) == 4 ? FE_DM_MINB : 2) kz_cg_dirmatvec(const BoxDev* boxes, const int2* work, double* part) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const ZGeom<1> G(t.x0, t.y0, B.N);
  __shared__ T smb[kDmBuf][ZGeom<1>::H * ZGeom<1>::W];
  const int odd = ((int)B.sc[SC_ITERS]) & 1;
  const T* __restrict__ po = F<T>(B, odd ? K_PP : K_PD);
  T* __restrict__ pn = F<T>(B, odd ? K_PD : K_PP);
  const T* __restrict__ r = F<T>(B, POLY ? K_Z : K_R);  // POLY: z
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ x = F<T>(B, K_X);
  T* __restrict__ q = F<T>(B, K_Q);
  const T alpha = (T)B.sc[SC_ALPHA], beta = (T)B.sc[SC_BETA];
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih, idt = T(1) / dt;
  const T lapc = T(0.5) * dt * ih * ih;
  // first iteration of a solve: pd_new = D^{-1} r (POLY: z) and x = 0 whatever pd_old and x hold
  const bool first = B.sc[SC_ITERS] == 0.0;
  auto dir = [&](T rv, T dv, T pv) {
    if (POLY) return first ? rv : rv + beta * pv;
    return first ? rv * dv : rv * dv + beta * pv;
  };
  auto ld = [&](const T* f, int col, int k) { return __ldg(&f[col + G.plane(G.wrapz(k))]); };
  // D^{-1} is not read in the polynomial form
  auto ldd = [&](int col, int k) { return POLY ? T(1) : ld(dinv, col, k); };
  // centre column: r, dinv, pd_old for planes k + 1 .. k + KPF in flight
  T cr[KPF], cd[KPF], cp[KPF];
  // halo cell: r, dinv, pd_old for planes k .. k + KPF - 1
  T hr[KPF], hd[KPF], hp[KPF];
  ZStream<T, KPF> psi, xs;
  psi.init(F<T>(B, W_PSI), G, t.k0);
  xs.init(x, G, t.k0);
#pragma unroll
  for (int j = 0; j < KPF; ++j) {
    cr[j] = ld(r, G.col, t.k0 + 1 + j);
    cd[j] = ldd(G.col, t.k0 + 1 + j);
    cp[j] = ld(po, G.col, t.k0 + 1 + j);
    if (G.hcol >= 0) {
      hr[j] = ld(r, G.hcol, t.k0 + j);
      hd[j] = ldd(G.hcol, t.k0 + j);
      hp[j] = ld(po, G.hcol, t.k0 + j);
    }
  }
  // z-queue of pd_new at k - 1, k; pd_old at k (for the x update)
  T zm = dir(ld(r, G.col, t.k0 - 1), ldd(G.col, t.k0 - 1), ld(po, G.col, t.k0 - 1));
  T oc = ld(po, G.col, t.k0);
  T zc = dir(ld(r, G.col, t.k0), ldd(G.col, t.k0), oc);
  DotAcc<T> a0;
  for (int k = t.k0; k < t.kend; ++k) {
    const T op = cp[0];
    const T zp = dir(cr[0], cd[0], cp[0]);
#pragma unroll
    for (int j = 0; j + 1 < KPF; ++j) {
      cr[j] = cr[j + 1];
      cd[j] = cd[j + 1];
      cp[j] = cp[j + 1];
    }
    cr[KPF - 1] = ld(r, G.col, k + 1 + KPF);
    cd[KPF - 1] = ldd(G.col, k + 1 + KPF);
    cp[KPF - 1] = ld(po, G.col, k + 1 + KPF);
    const T ps = psi.next(G, k);
    const T xv = xs.next(G, k);
    T* sm = smb[kDmBuf == 2 ? (k & 1) : 0];
    if (kDmBuf == 1) __syncthreads();
    sm[G.csm] = zc;
    if (G.hcol >= 0) {
      sm[G.hsm] = dir(hr[0], hd[0], hp[0]);
#pragma unroll
      for (int j = 0; j + 1 < KPF; ++j) {
        hr[j] = hr[j + 1];
        hd[j] = hd[j + 1];
        hp[j] = hp[j + 1];
      }
      hr[KPF - 1] = ld(r, G.hcol, k + KPF);
      hd[KPF - 1] = ldd(G.hcol, k + KPF);
      hp[KPF - 1] = ld(po, G.hcol, k + KPF);
    }
    __syncthreads();
    if (G.active) {
      const int c = G.col + G.plane(k);
      const T* s = sm + G.csm;
      const T nb = (s[-1] + s[1]) + (s[-ZGeom<1>::W] + s[ZGeom<1>::W]) + (zm + zp);
      const T y = ps * zc * idt - lapc * (nb - T(6) * zc);
      q[c] = y;
      pn[c] = zc;
      x[c] = first ? T(0) : xv + alpha * oc;
      a0.add(zc, y);
    }
    zm = zc;
    zc = zp;
    oc = op;
  }
  Red<T> v[1] = {a0.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_PQ] = res[0];
      B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
    }
  }
}

// ---- kz_cg_dirmatvec on streamed planes --------------------------------------------
// The same iteration (identical per-cell arithmetic) for boxes with N in
// {64, 128, 256, 512}: raw planes of r, D^{-1}, pd_old (with y-halo rows),
// psi and x (own rows) arrive by bulk copy in a ring of kBulkStages stages;
// pd_new of each plane (own and halo rows) goes to a 4-slot ring, and the
// operator is applied one plane behind, once pd_new of the plane above is
// there.  One barrier per plane.
#ifndef FE_BULK_STAGES
#define FE_BULK_STAGES 2
#endif
constexpr int kBulkStages = FE_BULK_STAGES;

// One ring stage of a kernel: nh streams with their two y-halo rows and no
// own-row-only streams, for blocks of `cells` cells per plane of edge N.
__host__ __device__ constexpr int bulk_stage_elems(int N, int cells, int nh, int no) {
  return nh * (cells + 2 * N) + no * cells;
}
__host__ __device__ constexpr int bulk_ring_elems(int N, int cells) {
  return 4 * (cells + 2 * N);
}
// Dynamic shared memory of the streamed CG kernels of one solver for edge N:
// the largest stage among them (Jacobi: kb_cg_dirmatvec<T, false>, three halo
// streams and two own; polynomial: kb_cg_rpoly<T, false>, three and one).
template <typename T>
int bulk_smem_bytes(int N, int cells, bool poly) {
  const int se = poly ? bulk_stage_elems(N, cells, 3, 1) : bulk_stage_elems(N, cells, 3, 2);
  return 128 + (kBulkStages * se + bulk_ring_elems(N, cells)) * (int)sizeof(T);
}

// POLY: the direction is pd_new = z + beta pd_old with z = P r from kb_cg_rpoly (first-order Neumann
// polynomial preconditioner), streamed with y-halo rows in place of r and D^{-1}.
template <typename T, bool POLY, int CELLS>
__global__ void __launch_bounds__(kBulkThreads) kb_cg_dirmatvec(const BoxDev* boxes, const int2* bwork, double* part) {
  constexpr int kBulkRows = bulk_rows<CELLS>();
  const int2 w = bwork[blockIdx.x];
  const BoxDev& B = boxes[w.x];
  if (box_done(B)) return;
  extern __shared__ __align__(128) unsigned char zsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(zsm);
  const int N = B.N;
  const BulkGeom Gm(N, w.y, B.bntiles, CELLS);
  const int R = Gm.R, RN = R * N, HN = (R + 2) * N;
  T* stage0 = reinterpret_cast<T*>(zsm + 128);
  constexpr int NHS = POLY ? 2 : 3;  // streams with y-halo rows
  const int SE = bulk_stage_elems(N, CELLS, NHS, 2);
  T* ring = stage0 + kBulkStages * SE;
  const int tid = threadIdx.x;
  const int odd = ((int)B.sc[SC_ITERS]) & 1;
  const T* __restrict__ po = F<T>(B, odd ? K_PP : K_PD);
  T* __restrict__ pn = F<T>(B, odd ? K_PD : K_PP);
  const T* __restrict__ r = F<T>(B, POLY ? K_Z : K_R);  // POLY: z
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  const T* __restrict__ psi = F<T>(B, W_PSI);
  T* __restrict__ x = F<T>(B, K_X);
  T* __restrict__ q = F<T>(B, K_Q);
  const T alpha = (T)B.sc[SC_ALPHA], beta = (T)B.sc[SC_BETA];
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih, idt = T(1) / dt;
  const T lapc = T(0.5) * dt * ih * ih;
  const bool first = B.sc[SC_ITERS] == 0.0;  // pd_new = D^{-1} r (POLY: z), x = 0 whatever pd_old and x hold
  const int nseq = Gm.count();
  const size_t NN = (size_t)N * N;

  // stage layout: r | dinv | pd_old (POLY: z | pd_old) (R + 2 rows each, halo rows first and last) | psi | x (R rows)
  auto issue = [&](int j) {
    const BulkPos P = bulk_pos(Gm, j);
    T* st = stage0 + (j % kBulkStages) * SE;
    uint64_t* bj = bar + (j % kBulkStages);
    const int y0 = P.g * R;
    const int ym = y0 == 0 ? N - 1 : y0 - 1;
    const size_t pl = (size_t)P.m * NN;
    const bool comp = P.pos >= 1 && P.pos <= P.len;
    const unsigned row = (unsigned)(N * sizeof(T)), rows = (unsigned)(RN * sizeof(T));
    // the first iteration of a solve reads neither pd_old (the last halo stream) nor x
    const int nh = first ? NHS - 1 : NHS;
    mbar_expect_tx(bj, nh * (rows + 2 * row) + (comp ? (first ? 1 : 2) * rows : 0));
    const T* src[3] = {r, POLY ? po : dinv, po};
    // rows ym .. ym + R + 1 of each stream: one copy, two where they wrap in y
    const int n0 = min(R + 2, N - ym);
#pragma unroll
    for (int f = 0; f < NHS; ++f) {
      if (f >= nh) break;
      T* d = st + f * HN;
      bulk_g2s(d, src[f] + pl + (size_t)ym * N, (unsigned)n0 * row, bj);
      if (n0 < R + 2) bulk_g2s(d + n0 * N, src[f] + pl, (unsigned)(R + 2 - n0) * row, bj);
    }
    if (comp) {
      bulk_g2s(st + NHS * HN, psi + pl + (size_t)y0 * N, rows, bj);
      if (!first) bulk_g2s(st + NHS * HN + RN, x + pl + (size_t)y0 * N, rows, bj);
    }
  };

  if (tid == 0) {
    for (int s = 0; s < kBulkStages; ++s) mbar_init(bar + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < kBulkStages && j < nseq; ++j) issue(j);

  const int Q = Gm.Q;
  const int x4 = (tid % Q) * 4;                                // first x of this thread
  const int RS = R / kBulkRows;                                // own rows: tid / Q + RS * u
  const int hr = tid < Q ? 0 : R + 1;                          // halo row handled (tid < 2Q)
  const bool halo = tid < 2 * Q;
  const int xm1 = x4 == 0 ? N - 1 : x4 - 1, xp4 = x4 + 4 == N ? 0 : x4 + 4;
  V4<T> sv_psi[kBulkRows], sv_x[kBulkRows], sv_po[kBulkRows], cu_psi[kBulkRows], cu_x[kBulkRows], cu_po[kBulkRows];
  DotAcc<T> a0;
  bool failed = false;
  for (int i = 0; i < nseq; ++i) {
    const BulkPos P = bulk_pos(Gm, i);
    const bool ok = mbar_wait(bar + (i % kBulkStages), (unsigned)((i / kBulkStages) & 1));
    const T* st = stage0 + (i % kBulkStages) * SE;
    T* slot = ring + (i & 3) * HN;
    if (ok) {
#pragma unroll
      for (int u = 0; u < kBulkRows; ++u) {  // own rows: pd_new, and the centre values needed one plane later
        const int jr = tid / Q + RS * u;
        const int o = (jr + 1) * N + x4;
        V4<T> nv, pv = {};
        if (POLY) {
          const V4<T> zv = ld4(st + o);
          if (!first) pv = ld4(st + HN + o);
#pragma unroll
          for (int e = 0; e < 4; ++e) nv.v[e] = first ? zv.v[e] : zv.v[e] + beta * pv.v[e];
        } else {
          const V4<T> rv = ld4(st + o), dv = ld4(st + HN + o);
          if (!first) pv = ld4(st + 2 * HN + o);
#pragma unroll
          for (int e = 0; e < 4; ++e) nv.v[e] = first ? rv.v[e] * dv.v[e] : rv.v[e] * dv.v[e] + beta * pv.v[e];
        }
        st4(slot + o, nv);
        cu_po[u] = pv;
        if (P.pos >= 1 && P.pos <= P.len) {
          cu_psi[u] = ld4(st + NHS * HN + jr * N + x4);
          cu_x[u] = first ? V4<T>{} : ld4(st + NHS * HN + RN + jr * N + x4);
        }
      }
      if (halo) {
        const int o = hr * N + x4;
        V4<T> nv;
        if (POLY) {
          const V4<T> zv = ld4(st + o), pv = first ? V4<T>{} : ld4(st + HN + o);
#pragma unroll
          for (int e = 0; e < 4; ++e) nv.v[e] = first ? zv.v[e] : zv.v[e] + beta * pv.v[e];
        } else {
          const V4<T> rv = ld4(st + o), dv = ld4(st + HN + o), pv = first ? V4<T>{} : ld4(st + 2 * HN + o);
#pragma unroll
          for (int e = 0; e < 4; ++e) nv.v[e] = first ? rv.v[e] * dv.v[e] : rv.v[e] * dv.v[e] + beta * pv.v[e];
        }
        st4(slot + o, nv);
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0 && i + kBulkStages < nseq) issue(i + kBulkStages);
    if (P.pos >= 2) {  // operator for the plane below (pos - 1 in 1..len)
      const int mo = P.m == 0 ? N - 1 : P.m - 1;
      const T* c = ring + ((i - 1) & 3) * HN;
      const T* zm = ring + ((i - 2) & 3) * HN;
      const T* zp = slot;
#pragma unroll
      for (int u = 0; u < kBulkRows; ++u) {
        const int jr = tid / Q + RS * u;
        const int o = (jr + 1) * N;
        const size_t gbase = (size_t)mo * NN + (size_t)(P.g * R + jr) * N + x4;
        const V4<T> cc = ld4(c + o + x4), cs = ld4(c + o - N + x4), cn = ld4(c + o + N + x4);
        const V4<T> cb = ld4(zm + o + x4), ca = ld4(zp + o + x4);
        const T left = c[o + xm1], right = c[o + xp4];
        V4<T> yv, xn;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T vc = cc.v[e];
          const T vxm = e == 0 ? left : cc.v[e == 0 ? 0 : e - 1];
          const T vxp = e == 3 ? right : cc.v[e == 3 ? 3 : e + 1];
          const T nb = (vxm + vxp) + (cs.v[e] + cn.v[e]) + (cb.v[e] + ca.v[e]);
          const T y = sv_psi[u].v[e] * vc * idt - lapc * (nb - T(6) * vc);
          yv.v[e] = y;
          xn.v[e] = first ? T(0) : sv_x[u].v[e] + alpha * sv_po[u].v[e];
          a0.add(vc, y);
        }
        st4(q + gbase, yv);
        st4(pn + gbase, cc);
        st4(x + gbase, xn);
      }
    }
#pragma unroll
    for (int u = 0; u < kBulkRows; ++u) {
      sv_psi[u] = cu_psi[u];
      sv_x[u] = cu_x[u];
      sv_po[u] = cu_po[u];
    }
  }
  if (failed) {
    // drain the copies still in flight (bounded), record the failure, leave
    if (tid == 0) {
      for (int s = 0; s < kBulkStages; ++s) mbar_wait(bar + s, 0u, 1 << 16), mbar_wait(bar + s, 1u, 1 << 16);
      B.sc[SC_KERR] = 1.0;
    }
    return;
  }
  Red<T> v[1] = {a0.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.btile0, B.bntiles)) {
    if (tid == 0) {
      B.sc[SC_PQ] = res[0];
      B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
    }
  }
}

// x += alpha pd for the direction of the last iteration (after kz_cg_dirmatvec).
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_xfinal(const BoxDev* boxes, const int2* work) {
  const Chunk ch = chunk_of(boxes, work);
  const BoxDev& B = boxes[ch.box];
  const int it = (int)B.sc[SC_ITERS];
  if (it == 0) return;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ pd = F<T>(B, (it & 1) ? K_PP : K_PD);
  T* __restrict__ x = F<T>(B, K_X);
  const T alpha = (T)B.sc[SC_ALPHA];
  chunk_loop(
      ch, tid,
      [&](int q0) {
        V4<T> xv = ld4(x + q0), pv = ld4(pd + q0);
#pragma unroll
        for (int e = 0; e < 4; ++e) xv.v[e] += alpha * pv.v[e];
        st4(x + q0, xv);
      },
      [&](int c) { x[c] = x[c] + alpha * pd[c]; });
}

// Iteration count, convergence test on ||r|| and the next beta (last block of
// a CG update).
__device__ void cg_update_scalars(const BoxDev& B, double rz, double rr, int* active) {
  double it = B.sc[SC_ITERS] + 1.0;
  B.sc[SC_ITERS] = it;
  B.sc[SC_RR] = rr;
  if (sqrt(rr) <= B.sc[SC_TOL] * sqrt(B.sc[SC_BB])) {
    B.sc[SC_DONE] = 1.0;
    B.sc[SC_CONV] = 1.0;
    atomicSub(active, 1);
  } else if (it >= B.sc[SC_MAXIT]) {
    B.sc[SC_DONE] = 1.0;
    B.sc[SC_CONV] = 0.0;
    atomicSub(active, 1);
  } else {
    B.sc[SC_BETA] = rz / B.sc[SC_RZ];
    B.sc[SC_RZ] = rz;
  }
}

// r -= alpha q; rz = <r, D^{-1} r>; convergence test on ||r|| (the update of
// the fused iteration: x is advanced by kz_cg_dirmatvec).
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_rupdate(const BoxDev* boxes, const int2* work, double* part, int* active) {
  const Chunk ch = chunk_of(boxes, work);
  const BoxDev& B = boxes[ch.box];
  if (box_done(B)) return;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ qv = F<T>(B, K_Q);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ r = F<T>(B, K_R);
  const T alpha = (T)B.sc[SC_ALPHA];
  DotAcc<T> a0, a1;
  chunk_loop(
      ch, tid,
      [&](int q0) {
        V4<T> rv = ld4(r + q0), qq = ld4(qv + q0), dv = ld4(dinv + q0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          rv.v[e] -= alpha * qq.v[e];
          a0.add(rv.v[e], rv.v[e] * dv.v[e]);
          a1.add(rv.v[e], rv.v[e]);
        }
        st4(r + q0, rv);
      },
      [&](int c) {
        T rc = r[c] - alpha * qv[c];
        r[c] = rc;
        a0.add(rc, rc * dinv[c]);
        a1.add(rc, rc);
      });
  Red<T> v[2] = {a0.red(), a1.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) cg_update_scalars(B, res[0], res[1], active);
  }
}

// Residual update with the polynomial-preconditioned residual, on streamed planes (the step after
// kb_cg_dirmatvec<T, true>): r_new = r - alpha q and w = D^{-1} r_new on the own and y-halo rows, then,
// one plane behind, z = D^{-1} (2 r_new - M w), i.e. z = P r_new with the first-order Neumann polynomial
// P = D^{-1} (2 I - M D^{-1}) (Dubois, Greenbaum and Rodrigue 1979; symmetric, and positive definite
// because the eigenvalues of D^{-1} M lie in (0, 2) for this diagonally dominant operator), <r_new, z>,
// ||r_new||^2 and the CG bookkeeping.  r alternates between K_R and K_RB by the parity of the iteration
// count (neighbouring blocks read the old residual as halo).  START: the first residual of an inner
// solve (alpha = 0, r stays in K_R): z and <r, z> only, no iteration counted.
template <typename T, bool START, int CELLS>
__global__ void __launch_bounds__(kBulkThreads) kb_cg_rpoly(const BoxDev* boxes, const int2* bwork, double* part, int* active) {
  constexpr int kBulkRows = bulk_rows<CELLS>();
  const int2 w = bwork[blockIdx.x];
  const BoxDev& B = boxes[w.x];
  if (box_done(B)) return;
  extern __shared__ __align__(128) unsigned char zsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(zsm);
  const int N = B.N;
  const BulkGeom Gm(N, w.y, B.bntiles, CELLS);
  const int R = Gm.R, HN = (R + 2) * N, RN = R * N;
  T* stage0 = reinterpret_cast<T*>(zsm + 128);
  constexpr int NHS = START ? 2 : 3;  // streams with y-halo rows: r, D^{-1} (and q)
  const int SE = bulk_stage_elems(N, CELLS, NHS, 1);
  T* ring = stage0 + kBulkStages * SE;
  const int tid = threadIdx.x;
  const int odd = START ? 0 : ((int)B.sc[SC_ITERS]) & 1;  // iterations before this one
  const T* __restrict__ ro = F<T>(B, odd ? K_RB : K_R);
  T* __restrict__ rn = F<T>(B, odd ? K_R : K_RB);
  const T* __restrict__ qv = F<T>(B, K_Q);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  const T* __restrict__ psi = F<T>(B, W_PSI);
  T* __restrict__ z = F<T>(B, K_Z);
  const T alpha = START ? T(0) : (T)B.sc[SC_ALPHA];
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih, idt = T(1) / dt;
  const T lapc = T(0.5) * dt * ih * ih;
  const int nseq = Gm.count();
  const size_t NN = (size_t)N * N;
  constexpr int FD = NHS - 1;         // stage index of D^{-1}

  // stage layout: r | q | D^{-1} (START: r | D^{-1}) (R + 2 rows each) | psi (R rows)
  auto issue = [&](int j) {
    const BulkPos P = bulk_pos(Gm, j);
    T* st = stage0 + (j % kBulkStages) * SE;
    uint64_t* bj = bar + (j % kBulkStages);
    const int y0 = P.g * R;
    const int ym = y0 == 0 ? N - 1 : y0 - 1;
    const size_t pl = (size_t)P.m * NN;
    const bool comp = P.pos >= 1 && P.pos <= P.len;
    const unsigned row = (unsigned)(N * sizeof(T)), rows = (unsigned)(RN * sizeof(T));
    mbar_expect_tx(bj, NHS * (rows + 2 * row) + (comp ? rows : 0));
    const T* src[3] = {ro, START ? dinv : qv, dinv};
    const int n0 = min(R + 2, N - ym);
#pragma unroll
    for (int f = 0; f < NHS; ++f) {
      T* d = st + f * HN;
      bulk_g2s(d, src[f] + pl + (size_t)ym * N, (unsigned)n0 * row, bj);
      if (n0 < R + 2) bulk_g2s(d + n0 * N, src[f] + pl, (unsigned)(R + 2 - n0) * row, bj);
    }
    if (comp) bulk_g2s(st + NHS * HN, psi + pl + (size_t)y0 * N, rows, bj);
  };

  if (tid == 0) {
    for (int s = 0; s < kBulkStages; ++s) mbar_init(bar + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < kBulkStages && j < nseq; ++j) issue(j);

  const int Q = Gm.Q;
  const int x4 = (tid % Q) * 4;
  const int RS = R / kBulkRows;
  const int hr = tid < Q ? 0 : R + 1;
  const bool halo = tid < 2 * Q;
  const int xm1 = x4 == 0 ? N - 1 : x4 - 1, xp4 = x4 + 4 == N ? 0 : x4 + 4;
  V4<T> sv_psi[kBulkRows], sv_r[kBulkRows], sv_d[kBulkRows], cu_psi[kBulkRows], cu_r[kBulkRows], cu_d[kBulkRows];
  DotAcc<T> a0, a1;
  bool failed = false;
  for (int i = 0; i < nseq; ++i) {
    const BulkPos P = bulk_pos(Gm, i);
    const bool ok = mbar_wait(bar + (i % kBulkStages), (unsigned)((i / kBulkStages) & 1));
    const T* st = stage0 + (i % kBulkStages) * SE;
    T* slot = ring + (i & 3) * HN;
    if (ok) {
#pragma unroll
      for (int u = 0; u < kBulkRows; ++u) {  // own rows: w = D^{-1} r_new, and r_new, D^{-1}, psi kept for the operator
        const int jr = tid / Q + RS * u;
        const int o = (jr + 1) * N + x4;
        const V4<T> rv = ld4(st + o), dv = ld4(st + FD * HN + o);
        V4<T> nr, wv;
        if (START) {
          nr = rv;
        } else {
          const V4<T> qq = ld4(st + HN + o);
#pragma unroll
          for (int e = 0; e < 4; ++e) nr.v[e] = rv.v[e] - alpha * qq.v[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) wv.v[e] = nr.v[e] * dv.v[e];
        st4(slot + o, wv);
        cu_r[u] = nr;
        cu_d[u] = dv;
        if (P.pos >= 1 && P.pos <= P.len) cu_psi[u] = ld4(st + NHS * HN + jr * N + x4);
      }
      if (halo) {
        const int o = hr * N + x4;
        const V4<T> rv = ld4(st + o), dv = ld4(st + FD * HN + o);
        V4<T> wv;
        if (START) {
#pragma unroll
          for (int e = 0; e < 4; ++e) wv.v[e] = rv.v[e] * dv.v[e];
        } else {
          const V4<T> qq = ld4(st + HN + o);
#pragma unroll
          for (int e = 0; e < 4; ++e) wv.v[e] = (rv.v[e] - alpha * qq.v[e]) * dv.v[e];
        }
        st4(slot + o, wv);
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0 && i + kBulkStages < nseq) issue(i + kBulkStages);
    if (P.pos >= 2) {  // the plane below (pos - 1 in 1..len): z = D^{-1} (2 r_new - M w)
      const int mo = P.m == 0 ? N - 1 : P.m - 1;
      const T* c = ring + ((i - 1) & 3) * HN;
      const T* zm = ring + ((i - 2) & 3) * HN;
      const T* zp = slot;
#pragma unroll
      for (int u = 0; u < kBulkRows; ++u) {
        const int jr = tid / Q + RS * u;
        const int o = (jr + 1) * N;
        const size_t gbase = (size_t)mo * NN + (size_t)(P.g * R + jr) * N + x4;
        const V4<T> cc = ld4(c + o + x4), cs = ld4(c + o - N + x4), cn = ld4(c + o + N + x4);
        const V4<T> cb = ld4(zm + o + x4), ca = ld4(zp + o + x4);
        const T left = c[o + xm1], right = c[o + xp4];
        V4<T> zv;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T vc = cc.v[e];
          const T vxm = e == 0 ? left : cc.v[e == 0 ? 0 : e - 1];
          const T vxp = e == 3 ? right : cc.v[e == 3 ? 3 : e + 1];
          const T nb = (vxm + vxp) + (cs.v[e] + cn.v[e]) + (cb.v[e] + ca.v[e]);
          const T mw = sv_psi[u].v[e] * vc * idt - lapc * (nb - T(6) * vc);
          const T ze = sv_d[u].v[e] * (T(2) * sv_r[u].v[e] - mw);
          zv.v[e] = ze;
          a0.add(sv_r[u].v[e], ze);
          if (!START) a1.add(sv_r[u].v[e], sv_r[u].v[e]);  // START: the boundary measured ||r||
        }
        st4(z + gbase, zv);
        if (!START) st4(rn + gbase, sv_r[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kBulkRows; ++u) {
      sv_psi[u] = cu_psi[u];
      sv_r[u] = cu_r[u];
      sv_d[u] = cu_d[u];
    }
  }
  if (failed) {
    if (tid == 0) {
      for (int s = 0; s < kBulkStages; ++s) mbar_wait(bar + s, 0u, 1 << 16), mbar_wait(bar + s, 1u, 1 << 16);
      B.sc[SC_KERR] = 1.0;
    }
    return;
  }
  Red<T> v[2] = {a0.red(), a1.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.btile0, B.bntiles)) {
    if (tid == 0) {
      if (START) B.sc[SC_RZ] = res[0];
      else cg_update_scalars(B, res[0], res[1], active);
    }
  }
}

// kb_cg_rpoly in z-marching form (boxes whose planes are not streamed): r_new = r - alpha q and
// w = D^{-1} r_new at the tile's cells and their one-cell x/y halo (staged per plane in shared memory,
// z-neighbours of w in registers), z = D^{-1} (2 r_new - M w) at the own cells, <r_new, z>, ||r_new||^2
// and the CG bookkeeping; r alternates between K_R and K_RB by the parity of the iteration count.
// START: the first z of an inner solve (alpha = 0, r in K_R).
template <typename T, bool START>
__global__ void __launch_bounds__(NTHR, sizeof(T) == 4 ? FE_DM_MINB : 2) kz_cg_rpoly(const BoxDev* boxes, const int2* work,
                                                                                     double* part, int* active) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const ZGeom<1> G(t.x0, t.y0, B.N);
  __shared__ T smb[kDmBuf][ZGeom<1>::H * ZGeom<1>::W];
  const int odd = START ? 0 : ((int)B.sc[SC_ITERS]) & 1;
  const T* __restrict__ ro = F<T>(B, odd ? K_RB : K_R);
  T* __restrict__ rn = F<T>(B, odd ? K_R : K_RB);
  const T* __restrict__ qv = F<T>(B, K_Q);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ z = F<T>(B, K_Z);
  const T alpha = START ? T(0) : (T)B.sc[SC_ALPHA];
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih, idt = T(1) / dt;
  const T lapc = T(0.5) * dt * ih * ih;
  auto ld = [&](const T* f, int col, int k) { return __ldg(&f[col + G.plane(G.wrapz(k))]); };
  auto ldq = [&](int col, int k) { return START ? T(0) : ld(qv, col, k); };
  auto res = [&](T rv, T qq) { return START ? rv : rv - alpha * qq; };
  // centre column: r, q, D^{-1} for planes k + 1 .. k + KPF in flight; halo cell: planes k .. k + KPF - 1
  T cr[KPF], cq[KPF], cd[KPF], hr[KPF], hq[KPF], hd[KPF];
  ZStream<T, KPF> psi;
  psi.init(F<T>(B, W_PSI), G, t.k0);
#pragma unroll
  for (int j = 0; j < KPF; ++j) {
    cr[j] = ld(ro, G.col, t.k0 + 1 + j);
    cq[j] = ldq(G.col, t.k0 + 1 + j);
    cd[j] = ld(dinv, G.col, t.k0 + 1 + j);
    if (G.hcol >= 0) {
      hr[j] = ld(ro, G.hcol, t.k0 + j);
      hq[j] = ldq(G.hcol, t.k0 + j);
      hd[j] = ld(dinv, G.hcol, t.k0 + j);
    }
  }
  // z-queue of w at k - 1, k; r_new and D^{-1} at k
  T wm = res(ld(ro, G.col, t.k0 - 1), ldq(G.col, t.k0 - 1)) * ld(dinv, G.col, t.k0 - 1);
  T rc = res(ld(ro, G.col, t.k0), ldq(G.col, t.k0)), dc = ld(dinv, G.col, t.k0);
  T wc = rc * dc;
  DotAcc<T> a0, a1;
  for (int k = t.k0; k < t.kend; ++k) {
    const T r1 = res(cr[0], cq[0]), d1 = cd[0];
    const T wp = r1 * d1;
#pragma unroll
    for (int j = 0; j + 1 < KPF; ++j) {
      cr[j] = cr[j + 1];
      cq[j] = cq[j + 1];
      cd[j] = cd[j + 1];
    }
    cr[KPF - 1] = ld(ro, G.col, k + 1 + KPF);
    cq[KPF - 1] = ldq(G.col, k + 1 + KPF);
    cd[KPF - 1] = ld(dinv, G.col, k + 1 + KPF);
    const T ps = psi.next(G, k);
    T* sm = smb[kDmBuf == 2 ? (k & 1) : 0];
    if (kDmBuf == 1) __syncthreads();
    sm[G.csm] = wc;
    if (G.hcol >= 0) {
      sm[G.hsm] = res(hr[0], hq[0]) * hd[0];
#pragma unroll
      for (int j = 0; j + 1 < KPF; ++j) {
        hr[j] = hr[j + 1];
        hq[j] = hq[j + 1];
        hd[j] = hd[j + 1];
      }
      hr[KPF - 1] = ld(ro, G.hcol, k + KPF);
      hq[KPF - 1] = ldq(G.hcol, k + KPF);
      hd[KPF - 1] = ld(dinv, G.hcol, k + KPF);
    }
    __syncthreads();
    if (G.active) {
      const int c = G.col + G.plane(k);
      const T* s = sm + G.csm;
      const T nb = (s[-1] + s[1]) + (s[-ZGeom<1>::W] + s[ZGeom<1>::W]) + (wm + wp);
      const T mw = ps * wc * idt - lapc * (nb - T(6) * wc);
      const T zv = dc * (T(2) * rc - mw);
      z[c] = zv;
      if (!START) rn[c] = rc;
      a0.add(rc, zv);
      if (!START) a1.add(rc, rc);  // START: the boundary measured ||r||
    }
    wm = wc;
    wc = wp;
    rc = r1;
    dc = d1;
  }
  Red<T> v[2] = {a0.red(), a1.red()};
  __shared__ double sres[2];
  if (block_sum_last<2>(v, B, part, sres, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      if (START) B.sc[SC_RZ] = sres[0];
      else cg_update_scalars(B, sres[0], sres[1], active);
    }
  }
}

// x += alpha pd; r -= alpha q; rz = <r, D^{-1} r>; convergence test on ||r||.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_update(const BoxDev* boxes, const int2* work, double* part, int* active) {
  const Chunk ch = chunk_of(boxes, work);
  const BoxDev& B = boxes[ch.box];
  if (box_done(B)) return;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ pd = F<T>(B, K_PD);
  const T* __restrict__ qv = F<T>(B, K_Q);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ x = F<T>(B, K_X);
  T* __restrict__ r = F<T>(B, K_R);
  const T alpha = (T)B.sc[SC_ALPHA];
  DotAcc<T> a0, a1;
  chunk_loop(
      ch, tid,
      [&](int q0) {
        V4<T> rv = ld4(r + q0), qq = ld4(qv + q0), dv = ld4(dinv + q0);
        V4<T> xv = ld4(x + q0), pv = ld4(pd + q0);
#pragma unroll
        for (int e = 0; e < 4; ++e) xv.v[e] += alpha * pv.v[e];
        st4(x + q0, xv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          rv.v[e] -= alpha * qq.v[e];
          a0.add(rv.v[e], rv.v[e] * dv.v[e]);
          a1.add(rv.v[e], rv.v[e]);
        }
        st4(r + q0, rv);
      },
      [&](int c) {
        x[c] = x[c] + alpha * pd[c];
        T rc = r[c] - alpha * qv[c];
        r[c] = rc;
        a0.add(rc, rc * dinv[c]);
        a1.add(rc, rc);
      });
  Red<T> v[2] = {a0.red(), a1.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) cg_update_scalars(B, res[0], res[1], active);
  }
}

// pd = r / diag + beta pd
template <typename T>
__global__ void __launch_bounds__(NTHR) k_cg_dir(const BoxDev* boxes, const int2* work) {
  const Chunk ch = chunk_of(boxes, work);
  const BoxDev& B = boxes[ch.box];
  if (box_done(B)) return;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ r = F<T>(B, K_R);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ pd = F<T>(B, K_PD);
  const T beta = (T)B.sc[SC_BETA];
  chunk_loop(
      ch, tid,
      [&](int q0) {
        V4<T> rv = ld4(r + q0), dv = ld4(dinv + q0), pv = ld4(pd + q0);
#pragma unroll
        for (int e = 0; e < 4; ++e) pv.v[e] = rv.v[e] * dv.v[e] + beta * pv.v[e];
        st4(pd + q0, pv);
      },
      [&](int c) { pd[c] = r[c] * dinv[c] + beta * pd[c]; });
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
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
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
  DotAcc<T> acc;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      T bc = b[c];
      r[c] = bc;
      rh[c] = bc;
      x[c] = T(0);
      p[c] = T(0);
      v[c] = T(0);
      acc.add(bc, bc);
    }
  }
  Red<T> a[1] = {acc.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(a, B, part, res, B.tile0, B.ntiles)) {
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
  DotAcc<T> acc;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      T y = applyM<T, true>(B, p, n, dt, ih);
      v[c] = y;
      acc.add(rh[c], y);
    }
  }
  Red<T> a[1] = {acc.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(a, B, part, res, B.tile0, B.ntiles)) {
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
  DotAcc<T> acc0, acc1;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      T y = applyM<T, true>(B, s, n, dt, ih);
      tv[c] = y;
      acc0.add(y, __ldg(&s[c]));
      acc1.add(y, y);
    }
  }
  Red<T> a[2] = {acc0.red(), acc1.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(a, B, part, res, B.tile0, B.ntiles)) {
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
  const T* dinv = F<T>(B, W_DINV);
  T* x = F<T>(B, K_X);
  T* r = F<T>(B, K_R);
  const T alpha = (T)B.sc[SC_ALPHA], om = (T)B.sc[SC_OMEGA];
  DotAcc<T> acc0, acc1;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      T di = dinv[c];
      T sc = s[c];
      x[c] = x[c] + alpha * (p[c] * di) + om * (sc * di);
      T rc = sc - om * tv[c];
      r[c] = rc;
      acc0.add(rc, rc);
      acc1.add(rh[c], rc);
    }
  }
  Red<T> a[2] = {acc0.red(), acc1.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(a, B, part, res, B.tile0, B.ntiles)) {
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

// ---- mixed precision: iterative refinement around the field-precision solve -----------
// The accumulated correction x is kept as a double-float pair per cell (slot
// K_X64, 8 bytes).  first: keep b in K_AUX, x = 0, ||b||^2.  Otherwise the
// residual r = b - M x in double-float arithmetic (FP64 for the transonic
// operator), stored in K_B as the next inner right-hand side.  The last block
// records the residual, the convergence of the box and the inner tolerance
// that the next inner solve needs (just enough to reach the target).
template <typename T>
__device__ __forceinline__ DF residual_df(const BoxDev& B, const float2* __restrict__ xs, const T* __restrict__ psi,
                                          T bc, const Nbr& n, DF idt, DF kl, DF k6) {
  const int c = n(0, 0, 0);
  auto X = [&](int q) {
    const float2 v = xs[q];
    return DF{v.x, v.y};
  };
  DF nb = df_add(X(n(1, 0, 0)), X(n(-1, 0, 0)));
  nb = df_add(nb, df_add(X(n(0, 1, 0)), X(n(0, -1, 0))));
  nb = df_add(nb, df_add(X(n(0, 0, 1)), X(n(0, 0, -1))));
  // a_c = psi_c / dt + 6 k,  M x = a_c x_c - k sum_nb
  const DF a = df_add(df_mul(idt, DF{(float)psi[c], 0.f}), k6);
  const DF mx = df_add(df_mul(a, X(c)), df_neg(df_mul(kl, nb)));
  return df_add(DF{(float)bc, 0.f}, df_neg(mx));
}

// Box bookkeeping after a refinement residual: convergence, counters, the FP64
// residual report and the next inner tolerance.

// First refinement step (element-wise): keep b in K_AUX, x pairs = 0, ||b||^2.
template <typename T>
__global__ void __launch_bounds__(NTHR) k_mix_first(const BoxDev* boxes, const int2* ework, double* part,
                                                    int* outer_active) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ b = F<T>(B, K_B);
  T* __restrict__ borig = F<T>(B, K_AUX);
  float2* __restrict__ xs = F<float2>(B, K_X64);
  DotAcc<float> acc;
  chunk_loop(
      ch, tid,
      [&](int q0) {
        const V4<T> bv = ld4(b + q0);
        st4(borig + q0, bv);
        reinterpret_cast<float4*>(xs + q0)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(xs + q0)[1] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc.add((float)bv.v[e], (float)bv.v[e]);
      },
      [&](int c) {
        const T bc = b[c];
        borig[c] = bc;
        xs[c] = make_float2(0.f, 0.f);
        acc.add((float)bc, (float)bc);
      });
  DF v[1] = {acc.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) mix_finish_scalars(B, res[0], 1, outer_active);
  }
}

// Refinement residual r = b - M x (x as double-float pairs) for the symmetric
// operator, z-marching form (pairs staged with a 1-cell halo).
template <typename T>
__global__ void __launch_bounds__(NTHR) kz_mix_residual(const BoxDev* boxes, const int2* work, double* part,
                                                        int* outer_active) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  const ZGeom<1> G(t.x0, t.y0, B.N);
  __shared__ float2 sm[ZGeom<1>::H * ZGeom<1>::W];
  ZField<float2, 1, KPF> xs;
  xs.init(F<float2>(B, K_X64), sm, G, t.k0);
  ZStream<T, KPF> borig, psi;
  borig.init(F<T>(B, K_AUX), G, t.k0);
  psi.init(F<T>(B, W_PSI), G, t.k0);
  T* __restrict__ b = F<T>(B, K_B);
  const double dt = B.sc[SC_KDT];
  const DF idt = df_from_double(1.0 / dt), kl = df_from_double(0.5 * dt * B.ih * B.ih),
           k6 = df_from_double(3.0 * dt * B.ih * B.ih);
  DotAcc<float> acc;
  auto X = [&](const float2 v) { return DF{v.x, v.y}; };
  for (int k = t.k0; k < t.kend; ++k) {
    xs.advance(G, k);
    const T bc = borig.next(G, k), pc = psi.next(G, k);
    __syncthreads();
    xs.stage(G, k);
    __syncthreads();
    if (!G.active) continue;
    // neighbour sum: hi parts by a TwoSum chain (error terms kept), lo parts plainly
    const float2 n0 = xs.at(G, 0, 1), n1 = xs.at(G, 0, -1), n2 = xs.at(G, 1, 1), n3 = xs.at(G, 1, -1),
                 n4 = xs.at(G, 2, 1), n5 = xs.at(G, 2, -1);
    DF nb = df_two_sum(n0.x, n1.x);
    {
      const float h[4] = {n2.x, n3.x, n4.x, n5.x};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const DF u = df_two_sum(nb.hi, h[j]);
        nb.hi = u.hi;
        nb.lo = __fadd_rn(nb.lo, u.lo);
      }
      nb.lo = __fadd_rn(nb.lo, __fadd_rn(__fadd_rn(__fadd_rn(n0.y, n1.y), __fadd_rn(n2.y, n3.y)), __fadd_rn(n4.y, n5.y)));
      nb = df_fast_two_sum(nb.hi, nb.lo);
    }
    const DF a = df_add_same_sign(df_mul(idt, DF{(float)pc, 0.f}), k6);
    const DF mx = df_add(df_mul(a, X(xs.c())), df_neg(df_mul(kl, nb)));
    const DF r = df_add(DF{(float)bc, 0.f}, df_neg(mx));
    b[G.col + G.plane(k)] = (T)r.hi;
    acc.add(r.hi, r.hi);
  }
  DF v[1] = {acc.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) mix_finish_scalars(B, res[0], 0, outer_active);
  }
}

// ---- fused refinement of the plain-CG mixed-precision solve -----------------------------------


// Start of a refined solve whose right-hand side is in K_B (the standalone
// pressure solve; in a step the right-hand-side kernel does this itself):
// b to K_AUX and to the first inner right-hand side K_R, ||b||^2 and
// <b, D^{-1} b> into the refinement and CG scalars.  The solution pairs start
// as zero by the outer-step count (nothing is written to them).
template <typename T>
__global__ void __launch_bounds__(NTHR) k_refine_start(const BoxDev* boxes, const int2* ework, double* part,
                                                       int* outer_active, int* active) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ b = F<T>(B, K_B);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ borig = F<T>(B, K_AUX);
  T* __restrict__ r = F<T>(B, K_R);
  DotAcc<T> arr, arz;
  chunk_loop(
      ch, tid,
      [&](int q0) {
        const V4<T> bv = ld4(b + q0), dv = ld4(dinv + q0);
        st4(borig + q0, bv);
        st4(r + q0, bv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          arr.add(bv.v[e], bv.v[e]);
          arz.add(bv.v[e], bv.v[e] * dv.v[e]);
        }
      },
      [&](int c) {
        const T bc = b[c];
        borig[c] = bc;
        r[c] = bc;
        arr.add(bc, bc);
        arz.add(bc, bc * dinv[c]);
      });
  Red<T> v[2] = {arr.red(), arz.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      mix_finish_scalars(B, res[0], 1, outer_active);
      cg_start_scalars(B, res[1], res[0], active);
    }
  }
}

// Boundary between inner solves, one pass: x pairs' = x pairs + (x + alpha pd)
// (the last direction the fused iteration has not added yet; nothing when the
// solve did not iterate), r = b - M x pairs' in double-float arithmetic, the
// refinement bookkeeping, and the start of the next inner solve from r.  The
// pairs ping-pong between K_X64 and K_X64B with the parity of the outer step
// (neighbouring tiles read the old pairs as halo).  Symmetric operator.
// Loads run KPF planes ahead, halo cells included.  kp_refine is the same
// pass on column pairs (two x-neighbouring cells per thread, vector loads).
template <typename T>
struct PairRaw {
  float2 a;  // old pair
  T x, p;    // FP32 iterate and last direction (zero when the solve did not move)
};
template <typename T>
struct PairSrc {
  const float2* __restrict__ xo;
  const T* __restrict__ x;
  const T* __restrict__ pd;
  T alpha;
  bool moved, fresh;
  __device__ __forceinline__ PairRaw<T> load(int q) const {
    PairRaw<T> v;
    v.a = fresh ? make_float2(0.f, 0.f) : __ldg(&xo[q]);
    v.x = moved ? __ldg(&x[q]) : T(0);
    v.p = moved ? __ldg(&pd[q]) : T(0);
    return v;
  }
  // pair + (x + alpha pd) as a pair (the FP32 sum rounds as the field update would)
  __device__ __forceinline__ float2 make(const PairRaw<T>& v) const {
    if (!moved) return v.a;
    const float d = (float)(v.x + alpha * v.p);
    const DF s = df_two_sum(v.a.x, d);
    const DF t = df_fast_two_sum(s.hi, __fadd_rn(s.lo, v.a.y));
    return make_float2(t.hi, t.lo);
  }
};

// One cell of r = b - M x for x as double-float pairs (symmetric operator):
// r = b - (psi/dt) x - kl (6 x - sum of the six neighbours n0..n5),
// kl = dt/(2 h^2).  The neighbour sum of the high parts is exact (TwoSum),
// 6 x and the two products are split exactly by FMA (TwoProduct), and the
// three large terms meet in two TwoSums, so the cancellation between them
// loses nothing; every low-order part is carried in plain FP32 (its rounding
// is about 2^-48 of the terms).
__device__ __forceinline__ float refine_residual(float2 zc, float2 n0, float2 n1, float2 n2, float2 n3, float2 n4,
                                                 float2 n5, float bc, float pc, DF idt, DF kl) {
  const DF s01 = df_two_sum(n0.x, n1.x), s23 = df_two_sum(n2.x, n3.x), s45 = df_two_sum(n4.x, n5.x);
  const DF u = df_two_sum(s01.hi, s23.hi), v = df_two_sum(u.hi, s45.hi);
  const float nlo = __fadd_rn(__fadd_rn(__fadd_rn(s01.lo, s23.lo), __fadd_rn(s45.lo, u.lo)),
                              __fadd_rn(v.lo, __fadd_rn(__fadd_rn(__fadd_rn(n0.y, n1.y), __fadd_rn(n2.y, n3.y)),
                                                        __fadd_rn(n4.y, n5.y))));
  const float p6 = __fmul_rn(6.f, zc.x), e6 = __fmaf_rn(6.f, zc.x, -p6);
  const DF sh = df_two_sum(p6, -v.hi);
  const float slo = __fadd_rn(__fadd_rn(sh.lo, e6), __fsub_rn(__fmul_rn(6.f, zc.y), nlo));
  const float kp = __fmul_rn(kl.hi, sh.hi);
  const float ke = __fmaf_rn(kl.lo, sh.hi, __fmaf_rn(kl.hi, slo, __fmaf_rn(kl.hi, sh.hi, -kp)));
  const float wp = __fmul_rn(idt.hi, pc);
  const float we = __fmaf_rn(idt.lo, pc, __fmaf_rn(idt.hi, pc, -wp));
  const float ap = __fmul_rn(wp, zc.x);
  const float ae = __fmaf_rn(we, zc.x, __fmaf_rn(wp, zc.y, __fmaf_rn(wp, zc.x, -ap)));
  const DF t1 = df_two_sum(bc, -ap), t2 = df_two_sum(t1.hi, -kp);
  return __fadd_rn(t2.hi, __fsub_rn(__fadd_rn(t2.lo, t1.lo), __fadd_rn(ae, ke)));
}

template <typename T>
__global__ void __launch_bounds__(NTHR) kz_refine(const BoxDev* boxes, const int2* work, double* part,
                                                  int* outer_active, int* active, int poly) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (B.sc[SC_ODONE] != 0.0) return;
  const ZGeom<1> G(t.x0, t.y0, B.N);
  __shared__ float2 sm[ZGeom<1>::H * ZGeom<1>::W];
  const int par = ((int)B.sc[SC_OUTER]) & 1, it = (int)B.sc[SC_ITERS];
  PairSrc<T> src;
  src.fresh = B.sc[SC_OUTER] == 0.0;  // first boundary: the pairs start as zero
  src.xo = F<float2>(B, par ? K_X64B : K_X64);
  src.x = F<T>(B, K_X);
  src.pd = F<T>(B, (it & 1) ? K_PP : K_PD);
  src.alpha = (T)B.sc[SC_ALPHA];
  src.moved = it > 0;
  float2* __restrict__ xn = F<float2>(B, par ? K_X64 : K_X64B);
  T* __restrict__ xh = F<T>(B, K_XH);
  T* __restrict__ r = F<T>(B, K_R);
  const double dt = B.sc[SC_KDT];
  const DF idt = df_from_double(1.0 / dt), kl = df_from_double(0.5 * dt * B.ih * B.ih);
  // pairs at planes k-1, k, k+1 of the own column; raw loads of later planes
  auto cq = [&](int k) { return G.col + G.plane(G.wrapz(k)); };
  auto hq = [&](int k) { return G.hcol + G.plane(G.wrapz(k)); };
  float2 zm, zc = src.make(src.load(cq(t.k0 - 1))), zp = src.make(src.load(cq(t.k0)));
  PairRaw<T> nq[KPF], nh[KPF];  // own column planes k+2.., halo planes k..
#pragma unroll
  for (int j = 0; j < KPF; ++j) {
    nq[j] = src.load(cq(t.k0 + 1 + j));
    if (G.hcol >= 0) nh[j] = src.load(hq(t.k0 + j));
  }
  ZStream<T, KPF> borig, psi, dinv;
  borig.init(F<T>(B, K_AUX), G, t.k0);
  psi.init(F<T>(B, W_PSI), G, t.k0);
  dinv.init(F<T>(B, W_DINV), G, t.k0);
  DotAcc<float> arr, arz;
  for (int k = t.k0; k < t.kend; ++k) {
    zm = zc;
    zc = zp;
    zp = src.make(nq[0]);
#pragma unroll
    for (int j = 0; j + 1 < KPF; ++j) nq[j] = nq[j + 1];
    nq[KPF - 1] = src.load(cq(k + 2 + KPF - 1));
    const T bc = borig.next(G, k), pc = psi.next(G, k), dc = dinv.next(G, k);
    __syncthreads();
    sm[G.csm] = zc;
    if (G.hcol >= 0) {
      sm[G.hsm] = src.make(nh[0]);
#pragma unroll
      for (int j = 0; j + 1 < KPF; ++j) nh[j] = nh[j + 1];
      nh[KPF - 1] = src.load(hq(k + KPF));
    }
    __syncthreads();
    if (!G.active) continue;
    const int c = G.col + G.plane(k);
    xn[c] = zc;
    xh[c] = (T)zc.x;  // the high part is the pair rounded to FP32
    const float2* s = sm + G.csm;
    const float rv = refine_residual(zc, s[1], s[-1], s[ZGeom<1>::W], s[-ZGeom<1>::W], zp, zm, (float)bc, (float)pc,
                                     idt, kl);
    r[c] = (T)rv;
    arr.add(rv, rv);
    if (!poly) arz.add(rv, (float)((T)rv * dc));  // poly: the next solve's start pass forms <r, z>
  }
  DF v[2] = {arr.red(), arz.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      mix_finish_scalars(B, res[0], 0, outer_active);
      cg_start_scalars(B, res[1], res[0], active);
    }
  }
}

// kz_refine on column pairs: 16 x 8 threads per 32 x 8 tile, each thread the
// cells (x, x+1) of its column pair (N even), pair loads and stores; the
// inner x-neighbours come from registers, the outer ones and the y-neighbours
// from the staged plane of updated pairs.  poly: the next inner solve starts
// with the polynomial preconditioner's own pass (kb/kz_cg_rpoly<T, true>), so
// D^{-1} is not read and <r, D^{-1} r> not formed.
template <typename T>
__global__ void __launch_bounds__(RNT, FE_REFINE_MINB) kp_refine(const BoxDev* boxes, const int2* work, double* part,
                                                 int* outer_active, int* active, int poly) {
  const TileXYZ t = tile_xyz(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (B.sc[SC_ODONE] != 0.0) return;
  constexpr int SW = TX + 2, SH = TY + 2;  // staged plane: tile + one-cell halo
  __shared__ __align__(16) float2 sm[SH * SW];
  const int N = B.N, NN = N * N;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + RTX * ty;
  auto wrap = [&](int v) { return ((v % N) + N) % N; };  // tiles wider than a small box wrap more than once
  const bool act = (t.x0 + 2 * tx < N) && (t.y0 + ty < N);
  const int col = wrap(t.x0 + 2 * tx) + N * wrap(t.y0 + ty);
  const int csm = (ty + 1) * SW + 2 * tx + 1;
  int hcol = -1, hsm = 0;  // the halo cell this thread stages (80 of them: x-halo 2 x 8, y-halo 2 x 32)
  if (tid < 2 * TY + 2 * TX) {
    int lx, ly;
    if (tid < 2 * TY) {
      ly = tid >> 1;
      lx = (tid & 1) ? TX : -1;
    } else {
      const int h = tid - 2 * TY;
      ly = h < TX ? -1 : TY;
      lx = h % TX;
    }
    hcol = wrap(t.x0 + lx) + N * wrap(t.y0 + ly);
    hsm = (ly + 1) * SW + lx + 1;
  }
  auto plane = [&](int k) { return NN * (k < 0 ? k + N : (k >= N ? k - N : k)); };
  const int par = ((int)B.sc[SC_OUTER]) & 1, it = (int)B.sc[SC_ITERS];
  PairSrc<T> src;
  src.fresh = B.sc[SC_OUTER] == 0.0;
  src.xo = F<float2>(B, par ? K_X64B : K_X64);
  src.x = F<T>(B, K_X);
  src.pd = F<T>(B, (it & 1) ? K_PP : K_PD);
  src.alpha = (T)B.sc[SC_ALPHA];
  src.moved = it > 0;
  float2* __restrict__ xn = F<float2>(B, par ? K_X64 : K_X64B);
  T* __restrict__ xh = F<T>(B, K_XH);
  T* __restrict__ r = F<T>(B, K_R);
  const T* __restrict__ borig = F<T>(B, K_AUX);
  const T* __restrict__ psi = F<T>(B, W_PSI);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  const double dt = B.sc[SC_KDT];
  const DF idt = df_from_double(1.0 / dt), kl = df_from_double(0.5 * dt * B.ih * B.ih);
  // raw values of the own pair at one plane
  struct Raw2 {
    float4 a;  // old pairs of both cells
    P2<T> x, p;
  };
  auto load2 = [&](int q) {
    Raw2 v;
    v.a = src.fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(reinterpret_cast<const float4*>(src.xo + q));
    if (src.moved) {
      v.x = ldp(src.x + q);
      v.p = ldp(src.pd + q);
    } else {
      v.x.x = v.x.y = v.p.x = v.p.y = T(0);
    }
    return v;
  };
  auto make2 = [&](const Raw2& v, float2& c0, float2& c1) {
    c0 = src.make(PairRaw<T>{make_float2(v.a.x, v.a.y), v.x.x, v.p.x});
    c1 = src.make(PairRaw<T>{make_float2(v.a.z, v.a.w), v.x.y, v.p.y});
  };
  float2 zm[2], zc[2], zp[2];
  make2(load2(col + plane(t.k0 - 1)), zc[0], zc[1]);
  make2(load2(col + plane(t.k0)), zp[0], zp[1]);
  Raw2 nq[KPF];            // own pair, planes k+2 ..
  PairRaw<T> nh[KPF];      // halo cell, planes k ..
  P2<T> nb_[KPF], np_[KPF], nd_[KPF];  // b, psi, D^{-1} of the own pair, planes k ..
#pragma unroll
  for (int j = 0; j < KPF; ++j) {
    nq[j] = load2(col + plane(t.k0 + 1 + j));
    if (hcol >= 0) nh[j] = src.load(hcol + plane(t.k0 + j));
    const int q = col + plane(t.k0 + j);
    nb_[j] = ldp(borig + q);
    np_[j] = ldp(psi + q);
    if (!poly) nd_[j] = ldp(dinv + q);
  }
  DotAcc<float> arr, arz;
  for (int k = t.k0; k < t.kend; ++k) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      zm[e] = zc[e];
      zc[e] = zp[e];
    }
    make2(nq[0], zp[0], zp[1]);
    const P2<T> bc = nb_[0], pcv = np_[0], dc = nd_[0];
#pragma unroll
    for (int j = 0; j + 1 < KPF; ++j) {
      nq[j] = nq[j + 1];
      nb_[j] = nb_[j + 1];
      np_[j] = np_[j + 1];
      nd_[j] = nd_[j + 1];
    }
    nq[KPF - 1] = load2(col + plane(k + 1 + KPF));
    {
      const int q = col + plane(k + KPF);
      nb_[KPF - 1] = ldp(borig + q);
      np_[KPF - 1] = ldp(psi + q);
      if (!poly) nd_[KPF - 1] = ldp(dinv + q);
    }
    __syncthreads();
    sm[csm] = zc[0];
    sm[csm + 1] = zc[1];
    if (hcol >= 0) {
      sm[hsm] = src.make(nh[0]);
#pragma unroll
      for (int j = 0; j + 1 < KPF; ++j) nh[j] = nh[j + 1];
      nh[KPF - 1] = src.load(hcol + plane(k + KPF));
    }
    __syncthreads();
    if (!act) continue;
    const int c = col + NN * k;
    *reinterpret_cast<float4*>(xn + c) = make_float4(zc[0].x, zc[0].y, zc[1].x, zc[1].y);
    stp(xh + c, (T)zc[0].x, (T)zc[1].x);  // the high parts are the pairs rounded to FP32
    const float r0 = refine_residual(zc[0], zc[1], sm[csm - 1], sm[csm + SW], sm[csm - SW], zp[0], zm[0],
                                     (float)bc.x, (float)pcv.x, idt, kl);
    const float r1 = refine_residual(zc[1], sm[csm + 2], zc[0], sm[csm + 1 + SW], sm[csm + 1 - SW], zp[1], zm[1],
                                     (float)bc.y, (float)pcv.y, idt, kl);
    stp(r + c, (T)r0, (T)r1);
    arr.add(r0, r0);
    arr.add(r1, r1);
    if (!poly) {
      arz.add(r0, (float)((T)r0 * dc.x));
      arz.add(r1, (float)((T)r1 * dc.y));
    }
  }
  DF v[2] = {arr.red(), arz.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      mix_finish_scalars(B, res[0], 0, outer_active);
      cg_start_scalars(B, res[1], res[0], active);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NTHR) k_mix_residual(const BoxDev* boxes, const int2* work, double* part, int first,
                                                       int* outer_active) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  T* __restrict__ b = F<T>(B, K_B);
  T* __restrict__ borig = F<T>(B, K_AUX);
  float2* __restrict__ xs = F<float2>(B, K_X64);
  const T* __restrict__ psi = F<T>(B, W_PSI);
  const double dt = B.sc[SC_KDT];
  const DF idt = df_from_double(1.0 / dt), kl = df_from_double(0.5 * dt * B.ih * B.ih),
           k6 = df_from_double(3.0 * dt * B.ih * B.ih);
  DotAcc<float> acc;
  double acc64 = 0.0;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      const int c = n(0, 0, 0);
      if (first) {
        T bc = b[c];
        borig[c] = bc;
        xs[c] = make_float2(0.f, 0.f);
        acc.add((float)bc, (float)bc);
      } else if (!B.transonic) {
        DF r = residual_df<T>(B, xs, psi, borig[c], n, idt, kl, k6);
        b[c] = (T)r.hi;
        acc.add(r.hi, r.hi);
      } else {
        // transonic operator: FP64 on the pair values
        double r = (double)borig[c] - applyM64_pairs<T>(B, xs, n, dt);
        b[c] = (T)r;
        acc64 += r * r;
      }
    }
  }
  DF v[1] = {B.transonic ? df_add(acc.red(), df_from_double(acc64)) : acc.red()};
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) mix_finish_scalars(B, res[0], first, outer_active);
  }
}

// x (double-float pair) += inner correction
template <typename T>
__global__ void __launch_bounds__(NTHR) k_mix_accum(const BoxDev* boxes, const int2* ework) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ x = F<T>(B, K_X);
  float2* __restrict__ xs = F<float2>(B, K_X64);
  for (int c = ch.begin + tid; c < ch.end; c += NTHR) {
    const float2 a = xs[c];
    const DF s = df_add(DF{a.x, a.y}, DF{(float)x[c], 0.f});
    xs[c] = make_float2(s.hi, s.lo);
  }
}

// x = the pair rounded to the field precision
template <typename T>
__global__ void __launch_bounds__(NTHR) k_mix_finish(const BoxDev* boxes, const int2* ework, int pingpong) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  const int tid = threadIdx.x + TX * threadIdx.y;
  T* __restrict__ x = F<T>(B, K_X);
  if (pingpong) {
    // fused refinement: every boundary pass wrote the high parts (the pairs rounded to
    // FP32) to K_XH; only a solve that never reached a boundary (b = 0) leaves zero there
    if (B.sc[SC_OUTER] != 0.0) return;
    T* __restrict__ xh = F<T>(B, K_XH);
    for (int c = ch.begin + tid; c < ch.end; c += NTHR) xh[c] = T(0);
    return;
  }
  const float2* __restrict__ xs = F<float2>(B, K_X64);
  for (int c = ch.begin + tid; c < ch.end; c += NTHR) {
    const float2 a = xs[c];
    x[c] = (T)__fadd_rn(a.x, a.y);
  }
}

// ---- flexible CG (learned preconditioner) ------------------------------------------------
// Direction candidates: the residual-form network direction
// z = r dinv + sc[SC_NSCALE] y (y the network output, FP32) or the Jacobi
// direction r dinv when <z, r> <= 0 or without a network output.
// p = z' - beta p_prev with beta = <z', q_prev> / <p_prev, q_prev>
// (Notay 2000, truncation 1).
template <typename T>
__global__ void __launch_bounds__(NTHR) k_fcg_dots(const BoxDev* boxes, const int2* ework, double* part,
                                                   const float* z) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  if (box_done(B)) return;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ r = F<T>(B, K_R);
  const T* __restrict__ q = F<T>(B, K_Q);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  const T zs = z ? (T)B.sc[SC_NSCALE] : T(0);
  DotAcc<T> zr, zq, dq;
  for (int c = ch.begin + tid; c < ch.end; c += NTHR) {
    const T rc = r[c], qc = q[c], rd = rc * dinv[c];
    const T zc = z ? rd + zs * (T)z[c] : rd;  // no network output: Jacobi direction
    zr.add(zc, rc);
    zq.add(zc, qc);
    dq.add(rd, qc);
  }
  Red<T> v[3] = {zr.red(), zq.red(), dq.red()};
  __shared__ double res[3];
  if (block_sum_last<3>(v, B, part, res, B.etile0, B.entiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const bool fb = !(res[0] > 0.0);
      B.sc[SC_FB] = fb ? 1.0 : 0.0;
      if (fb) B.sc[SC_NFB] += 1.0;
      const double pq = B.sc[SC_PQ];
      B.sc[SC_BETA] = (B.sc[SC_ITERS] == 0.0 || !(pq != 0.0)) ? 0.0 : (fb ? res[2] : res[1]) / pq;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NTHR) k_fcg_dir(const BoxDev* boxes, const int2* ework, const float* z) {
  const Chunk ch = chunk_of(boxes, ework);
  const BoxDev& B = boxes[ch.box];
  if (box_done(B)) return;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const T* __restrict__ r = F<T>(B, K_R);
  const T* __restrict__ dinv = F<T>(B, W_DINV);
  T* __restrict__ p = F<T>(B, K_PD);
  const bool fb = B.sc[SC_FB] != 0.0;
  const T beta = (T)B.sc[SC_BETA];
  const T zs = z ? (T)B.sc[SC_NSCALE] : T(0);
  for (int c = ch.begin + tid; c < ch.end; c += NTHR) {
    const T rd = r[c] * dinv[c];
    const T zc = (fb || !z) ? rd : rd + zs * (T)z[c];
    p[c] = zc - beta * p[c];
  }
}

// q = M p; alpha = <p, r> / <p, q>
template <typename T>
__global__ void __launch_bounds__(NTHR) k_fcg_matvec(const BoxDev* boxes, const int2* work, double* part) {
  Tile t = tile_of(boxes, work);
  const BoxDev& B = boxes[t.box];
  if (box_done(B)) return;
  const T* __restrict__ p = F<T>(B, K_PD);
  const T* __restrict__ r = F<T>(B, K_R);
  T* __restrict__ q = F<T>(B, K_Q);
  const T dt = (T)B.sc[SC_KDT], ih = (T)B.ih;
  DotAcc<T> pq, pr;
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      const int c = n(0, 0, 0);
      const T y = applyM<T, false>(B, p, n, dt, ih);
      q[c] = y;
      pq.add(p[c], y);
      pr.add(p[c], r[c]);
    }
  }
  Red<T> v[2] = {pq.red(), pr.red()};
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_PQ] = res[0];
      B.sc[SC_ALPHA] = res[1] / res[0];
    }
  }
}

// ---- launchers ------------------------------------------------------------------------
#define GRID L.nblocks, dim3(TX, TY), 0, L.st
#define EGRID L.neblocks, dim3(TX, TY), 0, L.st
template <typename T> void launch_cg_init(const Launch& L, double) {
  FE_LAUNCH(L, KID_CG_INIT, (k_cg_init<T><<<EGRID>>>(L.boxes, L.ework, L.part, L.active)));
}
template <typename T> void launch_cg_matvec(const Launch& L) {
  if (L.transonic) FE_LAUNCH(L, KID_CG_MATVEC, (k_cg_matvec<T><<<GRID>>>(L.boxes, L.work, L.part)));
  else FE_LAUNCH(L, KID_CG_MATVEC, (kz_cg_matvec<T><<<GRID>>>(L.boxes, L.work, L.part)));
}
template <typename T> void launch_cg_update(const Launch& L) {
  FE_LAUNCH(L, KID_CG_UPDATE, (k_cg_update<T><<<EGRID>>>(L.boxes, L.ework, L.part, L.active)));
}
template <typename T> void launch_cg_fused(const Launch& L) {
  if (L.poly) {  // polynomial preconditioner: direction from z, residual update forms the next z
    if (L.bwork && L.bcells == kBulkCellsPoly) {
      FE_LAUNCH(L, KID_CG_DIRMATVEC, (kb_cg_dirmatvec<T, true, kBulkCellsPoly><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                         L.boxes, L.bwork, L.part)));
      FE_LAUNCH(L, KID_CG_RUPDATE, (kb_cg_rpoly<T, false, kBulkCellsPoly><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                       L.boxes, L.bwork, L.part, L.active)));
    } else if (L.bwork) {
      FE_LAUNCH(L, KID_CG_DIRMATVEC, (kb_cg_dirmatvec<T, true, kBulkCells><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                         L.boxes, L.bwork, L.part)));
      FE_LAUNCH(L, KID_CG_RUPDATE, (kb_cg_rpoly<T, false, kBulkCells><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                       L.boxes, L.bwork, L.part, L.active)));
    } else {
      FE_LAUNCH(L, KID_CG_DIRMATVEC, (kz_cg_dirmatvec<T, true><<<GRID>>>(L.boxes, L.work, L.part)));
      FE_LAUNCH(L, KID_CG_RUPDATE, (kz_cg_rpoly<T, false><<<GRID>>>(L.boxes, L.work, L.part, L.active)));
    }
    return;
  }
  if (L.bwork)
    FE_LAUNCH(L, KID_CG_DIRMATVEC, (kb_cg_dirmatvec<T, false, kBulkCells><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                       L.boxes, L.bwork, L.part)));
  else
    FE_LAUNCH(L, KID_CG_DIRMATVEC, (kz_cg_dirmatvec<T, false><<<GRID>>>(L.boxes, L.work, L.part)));
  FE_LAUNCH(L, KID_CG_RUPDATE, (k_cg_rupdate<T><<<EGRID>>>(L.boxes, L.ework, L.part, L.active)));
}
// First polynomial-preconditioned residual z = P r of an inner solve and <r, z> (nothing without it)
template <typename T> void launch_cg_start(const Launch& L) {
  if (!L.poly) return;
  if (L.bwork && L.bcells == kBulkCellsPoly)
    FE_LAUNCH(L, KID_CG_START, (kb_cg_rpoly<T, true, kBulkCellsPoly><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                   L.boxes, L.bwork, L.part, L.active)));
  else if (L.bwork)
    FE_LAUNCH(L, KID_CG_START, (kb_cg_rpoly<T, true, kBulkCells><<<L.nbblocks, kBulkThreads, L.bsmem, L.st>>>(
                                   L.boxes, L.bwork, L.part, L.active)));
  else
    FE_LAUNCH(L, KID_CG_START, (kz_cg_rpoly<T, true><<<GRID>>>(L.boxes, L.work, L.part, L.active)));
}
template <typename T> void launch_cg_xfinal(const Launch& L) {
  FE_LAUNCH(L, KID_CG_XFINAL, (k_cg_xfinal<T><<<EGRID>>>(L.boxes, L.ework)));
}
template <typename T> void launch_cg_dir(const Launch& L) {
  FE_LAUNCH(L, KID_CG_DIR, (k_cg_dir<T><<<EGRID>>>(L.boxes, L.ework)));
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
template <typename T> void launch_fcg(const Launch& L, const float* z) {
  FE_LAUNCH(L, KID_FCG_DOTS, (k_fcg_dots<T><<<EGRID>>>(L.boxes, L.ework, L.part, z)));
  FE_LAUNCH(L, KID_FCG_DIR, (k_fcg_dir<T><<<EGRID>>>(L.boxes, L.ework, z)));
  FE_LAUNCH(L, KID_FCG_MATVEC, (k_fcg_matvec<T><<<GRID>>>(L.boxes, L.work, L.part)));
  FE_LAUNCH(L, KID_CG_UPDATE, (k_cg_update<T><<<EGRID>>>(L.boxes, L.ework, L.part, L.active)));
}
template <typename T> void launch_mix_residual(const Launch& L, int first, int* outer_active) {
  if (first)
    FE_LAUNCH(L, KID_MIX_RES, (k_mix_first<T><<<EGRID>>>(L.boxes, L.ework, L.part, outer_active)));
  else if (L.transonic)
    FE_LAUNCH(L, KID_MIX_RES, (k_mix_residual<T><<<GRID>>>(L.boxes, L.work, L.part, first, outer_active)));
  else
    FE_LAUNCH(L, KID_MIX_RES, (kz_mix_residual<T><<<GRID>>>(L.boxes, L.work, L.part, outer_active)));
}
template <typename T> void launch_refine_start(const Launch& L, int* outer_active) {
  FE_LAUNCH(L, KID_MIX_RES, (k_refine_start<T><<<EGRID>>>(L.boxes, L.ework, L.part, outer_active, L.active)));
  launch_cg_start<T>(L);
}
template <typename T> void launch_refine(const Launch& L, int* outer_active) {
  if (L.ring_ok)  // every box's N a multiple of the 16-byte chunk, so even: column pairs
    FE_LAUNCH(L, KID_REFINE,
              (kp_refine<T><<<L.nblocks, dim3(RTX, TY), 0, L.st>>>(L.boxes, L.work, L.part, outer_active, L.active,
                                                                     L.poly)));
  else
    FE_LAUNCH(L, KID_REFINE, (kz_refine<T><<<GRID>>>(L.boxes, L.work, L.part, outer_active, L.active, L.poly)));
  launch_cg_start<T>(L);
}
template <typename T> void launch_mix_finish_pp(const Launch& L) {
  FE_LAUNCH(L, KID_MIX_FIN, (k_mix_finish<T><<<EGRID>>>(L.boxes, L.ework, 1)));
}
template <typename T> void launch_mix_accum(const Launch& L) {
  FE_LAUNCH(L, KID_MIX_ACC, (k_mix_accum<T><<<EGRID>>>(L.boxes, L.ework)));
}
template <typename T> void launch_mix_finish(const Launch& L) {
  FE_LAUNCH(L, KID_MIX_FIN, (k_mix_finish<T><<<EGRID>>>(L.boxes, L.ework, 0)));
}

// Cells per block of the streamed CG kernels of one solver for the box edges
// minN..maxN: the larger polynomial block where every box has at least
// sixteen row groups (enough (group, plane) pairs per block that the two
// z-halo planes of each segment stay a small share) and its shared memory
// fits, else kBulkCells.
#ifndef FE_BULK_POLY_MIN_GROUPS
#define FE_BULK_POLY_MIN_GROUPS 16
#endif
template <typename T>
int bulk_cg_cells(int minN, int maxN, bool poly) {
  if (poly && kBulkCellsPoly != kBulkCells && minN * minN >= FE_BULK_POLY_MIN_GROUPS * kBulkCellsPoly &&
      bulk_smem_bytes<T>(maxN, kBulkCellsPoly, true) <= 227 * 1024)
    return kBulkCellsPoly;
  return kBulkCells;
}
template <typename T, int CELLS>
static bool bulk_set_smem(int bytes) {
  return cudaFuncSetAttribute(kb_cg_dirmatvec<T, false, CELLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(kb_cg_dirmatvec<T, true, CELLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(kb_cg_rpoly<T, false, CELLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess &&
         cudaFuncSetAttribute(kb_cg_rpoly<T, true, CELLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
             cudaSuccess;
}
// Dynamic shared memory of the streamed CG kernels of one solver for edge N
// and `cells` per block (sets the kernels' opt-in limit); 0 if it does not fit.
template <typename T>
int bulk_cg_prepare(int N, int cells, bool poly) {
  const int bytes = bulk_smem_bytes<T>(N, cells, poly);
  if (bytes > 227 * 1024) return 0;
  const bool ok = cells == kBulkCellsPoly ? bulk_set_smem<T, kBulkCellsPoly>(bytes) : bulk_set_smem<T, kBulkCells>(bytes);
  return ok ? bytes : 0;
}
// (row group, plane) pairs of an N^3 box
int bulk_cg_pairs(int N, int cells) { return N * (N / (cells / N)); }
template <typename T>
int bulk_cg_blocks_per_sm(int bytes, int cells) {
  int nb = 0;
  const cudaError_t e =
      cells == kBulkCellsPoly
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kb_cg_rpoly<T, false, kBulkCellsPoly>, kBulkThreads, bytes)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kb_cg_dirmatvec<T, false, kBulkCells>, kBulkThreads, bytes);
  return e == cudaSuccess ? nb : 0;
}

#define INST(T)                                                  \
  template void launch_cg_init<T>(const Launch&, double);        \
  template void launch_cg_matvec<T>(const Launch&);              \
  template void launch_cg_update<T>(const Launch&);              \
  template void launch_cg_fused<T>(const Launch&);               \
  template void launch_cg_xfinal<T>(const Launch&);              \
  template int bulk_cg_prepare<T>(int, int, bool);              \
  template int bulk_cg_cells<T>(int, int, bool);                 \
  template int bulk_cg_blocks_per_sm<T>(int, int);               \
  template void launch_cg_dir<T>(const Launch&);                 \
  template void launch_true_res<T>(const Launch&, int);          \
  template void launch_bicg_init<T>(const Launch&);              \
  template void launch_bicg_p<T>(const Launch&);                 \
  template void launch_bicg_v<T>(const Launch&);                 \
  template void launch_bicg_s<T>(const Launch&);                 \
  template void launch_bicg_x<T>(const Launch&);                 \
  template void launch_mix_residual<T>(const Launch&, int, int*); \
  template void launch_mix_accum<T>(const Launch&);              \
  template void launch_refine<T>(const Launch&, int*);           \
  template void launch_refine_start<T>(const Launch&, int*);     \
  template void launch_cg_start<T>(const Launch&);               \
  template void launch_mix_finish_pp<T>(const Launch&);          \
  template void launch_mix_finish<T>(const Launch&);              \
  template void launch_fcg<T>(const Launch&, const float*);
INST(double)
INST(float)

}  // namespace fe
