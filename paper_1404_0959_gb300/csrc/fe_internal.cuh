// fe_internal.cuh -- device-side data model, stencils and reductions of libfe.
//
// Data model (one context = n_boxes independent periodic boxes):
//  * every field of a box is an N^3 SoA array, x fastest; a face array of
//    direction d stores at cell c the value on the face between c and c+e_d;
//  * a box descriptor (BoxDev) holds the box constants and a table of field
//    pointers indexed by slot; kernels name fields by slot so the host can
//    swap time levels without moving data;
//  * every stencil kernel is launched once for all boxes over a work list of
//    (box, tile) pairs; a tile is 32 (x) x 8 (y) cells times tz z-planes and
//    is processed by a 32 x 8 thread block that walks the z-planes;
//  * reductions are deterministic: each block writes its partial sums to a
//    fixed slot, the last block of a box (found with one atomic counter, no
//    waiting) adds the partials in index order and updates the box scalars.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fe.h"

namespace fe {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NTHR = TX * TY;
constexpr int MAXD = FE_MAX_DUST;
constexpr int MAXP = 16;  // partial sums per block

// ---- field slots -----------------------------------------------------------
// state set s (0 or 1): base s * NSF
// F_V0 + 3 j + m: velocity component m of dust class j (two-fluid dust model only)
enum StateField { F_RHO = 0, F_U0, F_U1, F_U2, F_PHI0, F_PHI1, F_PHI2, F_P, F_T, F_Y0, F_V0 = F_Y0 + MAXD,
                  NSF = F_V0 + 3 * MAXD };
__host__ __device__ constexpr int S(int set, int f) { return set * NSF + f; }
enum WorkSlot {
  W_BASE = 2 * NSF,
  W_DIV = W_BASE,  // cell divergence of the velocity last differentiated
  W_DIVPHI,        // D(phi^n)
  W_RN0, W_RN1, W_RN2,    // R^n
  W_AN0, W_AN1, W_AN2,    // Du/Dt (level n, then level k)
  W_PSI,                  // rho^n / (gamma p^n)
  W_DINV,                 // 1 / Jacobi diagonal (psi/dt + 3 dt/h^2)
  W_HB0, W_HB1, W_HB2,    // HbyA
  W_PS0, W_PS1, W_PS2,    // phi*
  W_PW0, W_PW1,           // p^k ping-pong
  W_EW0, W_EW1,           // E^k ping-pong (Fourier)
  W_FEN,                  // D(F_E^n) (Fourier)
  W_FYN0,                 // D(phi_p^n I4 Y^n), MAXD slots
  W_YW0 = W_FYN0 + MAXD,  // Y^k ping 0, MAXD slots
  W_YW1 = W_YW0 + MAXD,   // Y^k ping 1, MAXD slots
  W_TFN0 = W_YW1 + MAXD,  // two-fluid dust: D(F^n), D(G^n_0..2) per class, 4 MAXD slots
  W_TFS0 = W_TFN0 + 4 * MAXD,  // two-fluid dust: predicted Y*, V*_0..2 per class, 4 MAXD slots
  // Krylov vectors
  K_B = W_TFS0 + 4 * MAXD, K_X, K_R, K_PD, K_Q,
  K_RHAT, K_V, K_S, K_T,  // BiCGStab
  K_Z, K_PP, K_QP,        // flexible CG: preconditioned r, previous direction and its image
  K_RB,                   // polynomial-preconditioned CG: residual ping-pong partner of K_R
  K_X64,                  // double accumulator (mixed precision refinement)
  K_X64B,                 // its ping-pong partner (fused refinement of plain CG)
  K_XH,                   // fused refinement: high parts of the pairs = the FP32 solution the corrector reads
  K_B64,                  // double right-hand side (mixed precision refinement)
  K_AUX,                  // scratch (diagnostics, user solve)
  W_YSUM,                 // two-way coupling with several classes: sum_j Y_j^n of the step
  // Fourier closure, total-energy flux: per cell H = E + p/rho, T and the Gauss gradients h Gc_m u_l
  // (m, l = 0..2: slot W_FEG0 + 3 m + l); the +1/2 face fluxes F_E along x, y, z
  W_FEH, W_FET, W_FEG0, W_FEF0 = W_FEG0 + 9,
  W_EN = W_FEF0 + 3,  // Fourier: E^n = c_v T^n + |u^n|^2 / 2 of the step (ring dust kernel)
  W_FED,              // Fourier: D(F_E^k) of the current corrector (ring dust kernel)
  NSLOT
};

// ---- per-box scalars (double) ---------------------------------------------
enum Scalar {
  SC_DT = 0, SC_DTPREV, SC_TIME, SC_UMAX,
  SC_RZ, SC_ALPHA, SC_BETA, SC_PQ, SC_BB, SC_RR, SC_DONE, SC_ITERS, SC_CONV, SC_TRUE_RR,
  SC_RHO_OLD, SC_OMEGA, SC_RV, SC_TS, SC_TT, SC_RHAT_R,  // BiCGStab
  SC_ZQ, SC_PR,                                           // flexible CG
  SC_TOL, SC_MAXIT, SC_KDT,   // Krylov tolerance, cap and the dt of its operator
  SC_IT0, SC_IT1, SC_IT2, SC_IT3, SC_RES0, SC_RES1, SC_RES2, SC_RES3,
  SC_ODONE, SC_OBB, SC_ORR, SC_ORES, SC_ITSUM, SC_OTOL, SC_OUTER,  // mixed-precision refinement
  SC_FB, SC_NFB,                                                    // flexible CG: Jacobi fallback flag, count
  SC_NSCALE,  // learned preconditioner: scale rms(r) d0 of the network's correction of the Jacobi direction
  SC_KERR,  // a kernel gave up a bounded wait (bulk-copy completion)
  SC_MASS, SC_ENERGY, SC_BAD, SC_DUST0,
  NSC = SC_DUST0 + MAXD + 4
};

struct BoxDev {
  int N, nd, closure, transonic;
  int tnx, tny, tnz, tz;   // tile grid and planes per tile
  int tile0, ntiles;       // this box's blocks in the stencil work list
  int etile0, entiles;     // this box's blocks in the element-wise work list
  int echunk;              // cells per element-wise block (multiple of 4 * NTHR)
  int btile0, bntiles;     // this box's blocks in the plane-streaming work list (0: not streamed)
  double h, ih, mu, gamma, R, cv, kappa, cfl, growth, dtmax;
  double tau_p[MAXD];
  void* f[NSLOT];
  double* sc;   // NSC scalars
  int* cnt;     // reduction counter (reset by the last block)
};

// ---- indexing ----------------------------------------------------------------
__device__ __forceinline__ int wrapi(int v, int N) {
  v += (v < 0) ? N : 0;
  v -= (v >= N) ? N : 0;
  return v;
}

// Wrapped flat offsets of the cells at -4..+4 along each axis.
struct Nbr {
  int x[9], y[9], z[9];
  __device__ __forceinline__ Nbr(int i, int j, int k, int N) {
#pragma unroll
    for (int s = -4; s <= 4; ++s) {
      x[s + 4] = wrapi(i + s, N);
      y[s + 4] = wrapi(j + s, N) * N;
      z[s + 4] = wrapi(k + s, N) * N * N;
    }
  }
  __device__ __forceinline__ int operator()(int dx, int dy, int dz) const { return x[dx + 4] + y[dy + 4] + z[dz + 4]; }
  // cell at offset o (given as a triple) shifted by s along d
  __device__ __forceinline__ int at(int d, int ox, int oy, int oz, int s) const {
    return (*this)(ox + (d == 0 ? s : 0), oy + (d == 1 ? s : 0), oz + (d == 2 ? s : 0));
  }
};

// ---- stencils (value type T, arrays of type A) --------------------------------
// I4 along d on the face between cell o and o+e_d
template <typename T, typename A>
__device__ __forceinline__ T I4f(const A* f, const Nbr& n, int d, int ox, int oy, int oz) {
  T a = (T)f[n.at(d, ox, oy, oz, -1)], b = (T)f[n.at(d, ox, oy, oz, 0)];
  T c = (T)f[n.at(d, ox, oy, oz, 1)], e = (T)f[n.at(d, ox, oy, oz, 2)];
  return (T(9) * (b + c) - (a + e)) * T(0.0625);
}
// G4 along d on the face between o and o+e_d (times h: caller multiplies by ih)
template <typename T, typename A>
__device__ __forceinline__ T G4f_h(const A* f, const Nbr& n, int d, int ox, int oy, int oz) {
  T a = (T)f[n.at(d, ox, oy, oz, -1)], b = (T)f[n.at(d, ox, oy, oz, 0)];
  T c = (T)f[n.at(d, ox, oy, oz, 1)], e = (T)f[n.at(d, ox, oy, oz, 2)];
  return (T(27) * (c - b) - (e - a)) * T(1.0 / 24.0);
}
// Gauss cell gradient along d at cell o (times h)
template <typename T, typename A>
__device__ __forceinline__ T Gc_h(const A* f, const Nbr& n, int d, int ox, int oy, int oz) {
  T m2 = (T)f[n.at(d, ox, oy, oz, -2)], m1 = (T)f[n.at(d, ox, oy, oz, -1)];
  T p1 = (T)f[n.at(d, ox, oy, oz, 1)], p2 = (T)f[n.at(d, ox, oy, oz, 2)];
  return (T(10) * (p1 - m1) - (p2 - m2)) * T(0.0625);
}
// D o G4 along d at cell o (times h^2)
template <typename T, typename A>
__device__ __forceinline__ T DG4_h2(const A* f, const Nbr& n, int d, int ox, int oy, int oz) {
  T m2 = (T)f[n.at(d, ox, oy, oz, -2)], m1 = (T)f[n.at(d, ox, oy, oz, -1)];
  T c0 = (T)f[n.at(d, ox, oy, oz, 0)];
  T p1 = (T)f[n.at(d, ox, oy, oz, 1)], p2 = (T)f[n.at(d, ox, oy, oz, 2)];
  return (T(28) * (m1 + p1) - T(54) * c0 - (m2 + p2)) * T(1.0 / 24.0);
}

// ---- double-float arithmetic ---------------------------------------------------
// An unevaluated pair hi + lo of floats (about 48 significant bits), with the
// error-free TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and FMA-based TwoProduct, and
// the pair addition and multiplication built on them (Dekker 1971).  Used for
// the refinement residual b - M x of the mixed-precision pressure solve: on
// this GPU the FP32 pipe is far wider than the FP64 pipe.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  DF t = df_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}
// Pair addition without the second TwoSum (Dekker's original): accurate to
// about 2^-44 relative to |a| + |b|, for operands of one sign.
__device__ __forceinline__ DF df_add_same_sign(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_from_double(double d) {
  const float hi = (float)d;
  return DF{hi, (float)(d - (double)hi)};
}

// Correctly rounded reciprocal: the value of 1 / v in IEEE division, without
// the general division sequence.
__device__ __forceinline__ float rcp_rn(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp_rn(double v) { return __drcp_rn(v); }

// ---- Jacobi preconditioner ---------------------------------------------------------
// 1 / diag(M) = 1 / (psi/dt + 3 dt/h^2) in the field precision, with one fused
// multiply-add: every kernel that stores it and every kernel that forms it on
// the fly gets the same bits.
template <typename T>
struct JacobiDiag {
  T idt, c3;
  __device__ __forceinline__ JacobiDiag(double dt, double ih) {
    const T d = (T)dt, h = (T)ih;
    idt = T(1) / d;
    c3 = T(3) * d * h * h;
  }
  __device__ __forceinline__ T inv(T psi) const { return rcp_rn(fma(psi, idt, c3)); }
};

// ---- inner-product accumulation ----------------------------------------------------
// double vectors: FP64 fused multiply-add.  float vectors: the compensated
// "Dot2" scheme of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005): each product is split exactly into
// rounded product + error with one FMA (TwoProduct) and added to a float
// pair with Knuth's error-free TwoSum, so the pair carries about 48
// significant bits -- FP64-class accuracy computed on the FP32 pipe, which on
// this GPU is far wider than the FP64 pipe.  The pairs stay pairs through the
// warp and block trees (double-float additions) and become a double once per
// block: on this GPU even a few FP64 additions per thread cost more than the
// block's memory traffic.  The _rn intrinsics keep the compiler from
// contracting the error-free steps.  red() gives the value to reduce (a double
// or a float pair).
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ double red() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float z = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ DF red() const { return DF{hi, lo}; }
};

// Plain sums with the same accuracy: FP64, or a float pair with TwoSum.
template <typename T>
struct SumAcc;
template <>
struct SumAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a) { s += a; }
  __device__ __forceinline__ double red() const { return s; }
};
template <>
struct SumAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a) {
    const DF t = df_two_sum(hi, a);
    hi = t.hi;
    lo = __fadd_rn(lo, t.lo);
  }
  __device__ __forceinline__ DF red() const { return DF{hi, lo}; }
};

// The reduced type of a field precision: double for FP64 fields, a float pair
// for FP32 fields.
template <typename T>
struct RedSel {
  using type = double;
};
template <>
struct RedSel<float> {
  using type = DF;
};
template <typename T>
using Red = typename RedSel<T>::type;
template <typename T>
__device__ __forceinline__ Red<T> red_from(double v);
template <>
__device__ __forceinline__ double red_from<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ DF red_from<float>(double v) {
  return df_from_double(v);
}

// ---- mixed-precision refinement and CG start bookkeeping (last block of a reduction) ----
// Refinement scalars after a residual evaluation, ||r||^2 = rr (first: of the
// right-hand side itself), and the tolerance of the next inner solve: the
// outer target with a safety margin, never below what an FP32 Krylov
// recurrence resolves.
#ifndef FE_INNER_MARGIN
#define FE_INNER_MARGIN 0.5
#endif
#ifndef FE_INNER_FLOOR
#define FE_INNER_FLOOR 1e-6
#endif
__device__ inline void mix_finish_scalars(const BoxDev& B, double rr, int first, int* outer_active) {
  double* sc = B.sc;
  if (first) {
    sc[SC_OBB] = rr;
    sc[SC_ITSUM] = 0.0;
    sc[SC_OUTER] = 0.0;
    bool zero = !(rr > 0.0);
    sc[SC_ODONE] = zero ? 1.0 : 0.0;
    sc[SC_CONV] = zero ? 1.0 : 0.0;
    if (!zero) atomicAdd(outer_active, 1);
  } else if (sc[SC_ODONE] == 0.0) {
    sc[SC_ITSUM] += sc[SC_ITERS];
    sc[SC_OUTER] += 1.0;
    if (sqrt(rr) <= sc[SC_OTOL] * sqrt(sc[SC_OBB])) {
      sc[SC_ODONE] = 1.0;
      sc[SC_CONV] = 1.0;
      atomicSub(outer_active, 1);
    } else if (sc[SC_OUTER] >= 8.0) {
      sc[SC_ODONE] = 1.0;
      sc[SC_CONV] = 0.0;
      atomicSub(outer_active, 1);
    }
  }
  sc[SC_ORR] = rr;
  sc[SC_ORES] = sc[SC_OBB] > 0.0 ? sqrt(rr / sc[SC_OBB]) : 0.0;
  // inner tolerance: reach the outer target with a factor 2 margin, within FP32 reach
  double need = rr > 0.0 ? FE_INNER_MARGIN * sc[SC_OTOL] * sqrt(sc[SC_OBB] / rr) : 0.5;
  sc[SC_TOL] = fmin(0.5, fmax(need, FE_INNER_FLOOR));
}

// The CG scalars of a new inner solve from its right-hand side r: rz, ||r||^2,
// counters, and whether it runs (not for a box whose refinement has converged).
__device__ inline void cg_start_scalars(const BoxDev& B, double rz, double rr, int* active) {
  double* sc = B.sc;
  sc[SC_ITERS] = 0.0;
  sc[SC_ALPHA] = 0.0;
  sc[SC_BETA] = 0.0;
  sc[SC_RZ] = rz;
  sc[SC_BB] = rr;
  const bool run = sc[SC_ODONE] == 0.0 && rr > 0.0;
  sc[SC_DONE] = run ? 0.0 : 1.0;
  if (run) atomicAdd(active, 1);
  else if (sc[SC_ODONE] == 0.0) sc[SC_CONV] = 1.0;  // a finished refinement keeps its verdict
}

// Adaptive time step from the box's max_i sum_d |u_d| (last block of the max
// reduction): CFL rule, growth limit against the previous step, cap.
__device__ inline void finish_dt(const BoxDev& B, double umax) {
  double dt = umax > 0.0 ? B.cfl * B.h / umax : HUGE_VAL;
  const double prev = B.sc[SC_DTPREV];
  if (prev > 0.0) dt = fmin(dt, B.growth * prev);
  dt = fmin(dt, B.dtmax);
  B.sc[SC_UMAX] = umax;
  B.sc[SC_DT] = dt;
  B.sc[SC_KDT] = dt;
}

// ---- block prologue -----------------------------------------------------------
struct Tile {
  int box, i, j, k0, kend;
  bool active;
};
__device__ __forceinline__ Tile tile_of(const BoxDev* boxes, const int2* work) {
  int2 w = work[blockIdx.x];
  const BoxDev& B = boxes[w.x];
  Tile t;
  t.box = w.x;
  int tx = w.y % B.tnx;
  int r = w.y / B.tnx;
  int ty = r % B.tny;
  int tzb = r / B.tny;
  t.i = tx * TX + threadIdx.x;
  t.j = ty * TY + threadIdx.y;
  t.k0 = tzb * B.tz;
  t.kend = min(t.k0 + B.tz, B.N);
  t.active = (t.i < B.N) && (t.j < B.N);
  return t;
}

// Element-wise kernels ignore the tile geometry: block w.y of a box takes the
// w.y-th of ntiles equal chunks of its N^3 cells (chunk length a multiple of
// 4 so that 16-byte vector accesses stay aligned).
struct Chunk {
  int box;
  int begin, end;
};
__device__ __forceinline__ Chunk chunk_of(const BoxDev* boxes, const int2* ework) {
  int2 w = ework[blockIdx.x];
  const BoxDev& B = boxes[w.x];
  const int n = B.N * B.N * B.N;
  Chunk c;
  c.box = w.x;
  c.begin = min(w.y * B.echunk, n);
  c.end = min(c.begin + B.echunk, n);
  return c;
}

// four consecutive elements as one (float4) or two (double2) 16-byte accesses
template <typename T>
struct V4 {
  T v[4];
};
__device__ __forceinline__ V4<float> ld4(const float* p) {
  float4 a = *reinterpret_cast<const float4*>(p);
  return V4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return V4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& a) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a.v[0], a.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(a.v[2], a.v[3]);
}

// ---- deterministic reductions ----------------------------------------------------
// Last-block phase of the block sums: the box's last block to finish adds the
// partials of all its blocks in block order.  Blocks of up to 32 warps
// (a multiple of 32 threads), 1-D or 2-D.
constexpr int kMaxWarps = 32;
template <int K>
__device__ bool sum_partials_last(const BoxDev& B, double* part, double* res, int tile0, int ntiles) {
  __shared__ double red[K][kMaxWarps];
  __shared__ int last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    __threadfence();
    int prev = atomicAdd(B.cnt, 1);
    last = (prev == ntiles - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = 0.0;
    for (int b = tid; b < ntiles; b += nt) s += __ldcg(&part[(size_t)(tile0 + b) * MAXP + q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[q][warp] = s;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = 0.0;
      for (int w = 0; w < nt / 32; ++w) s += red[q][w];
      res[q] = s;
    }
    *B.cnt = 0;
  }
  __syncthreads();
  return true;
}

// Block-sum K values (fixed tree), write this block's partials, and report
// whether this is the box's last block; if so `res` (shared) holds the box
// totals (partials added in block order).  Must be called by all threads.
// tile0/ntiles: the box's block range in the work list of this launch.
template <int K>
__device__ bool block_sum_last(double (&v)[K], const BoxDev& B, double* part, double* res, int tile0, int ntiles) {
  __shared__ double red[K][kMaxWarps];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[q][warp] = s;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = 0.0;
      for (int w = 0; w < nt / 32; ++w) s += red[q][w];
      part[(size_t)blockIdx.x * MAXP + q] = s;
    }
  }
  return sum_partials_last<K>(B, part, res, tile0, ntiles);
}
// Float-pair values: the warp and block trees add pairs on the FP32 pipe.
template <int K>
__device__ bool block_sum_last(DF (&v)[K], const BoxDev& B, double* part, double* res, int tile0, int ntiles) {
  __shared__ DF red[K][kMaxWarps];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    DF s = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const DF t{__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o)};
      s = df_add(s, t);
    }
    if (lane == 0) red[q][warp] = s;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      DF s = red[q][0];
      for (int w = 1; w < nt / 32; ++w) s = df_add(s, red[q][w]);
      part[(size_t)blockIdx.x * MAXP + q] = (double)s.hi + (double)s.lo;
    }
  }
  return sum_partials_last<K>(B, part, res, tile0, ntiles);
}

// Same for a maximum of one value.
__device__ __forceinline__ bool block_max_last(double v, const BoxDev& B, double* part, double* res, int tile0,
                                               int ntiles) {
  __shared__ double red[kMaxWarps];
  __shared__ int last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
  double s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (tid == 0) {
    double m = red[0];
    for (int w = 1; w < nt / 32; ++w) m = fmax(m, red[w]);
    part[(size_t)blockIdx.x * MAXP] = m;
    __threadfence();
    int prev = atomicAdd(B.cnt, 1);
    last = (prev == ntiles - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  s = 0.0;
  for (int b = tid; b < ntiles; b += nt) s = fmax(s, __ldcg(&part[(size_t)(tile0 + b) * MAXP]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (tid == 0) {
    double m = red[0];
    for (int w = 1; w < nt / 32; ++w) m = fmax(m, red[w]);
    *res = m;
    *B.cnt = 0;
  }
  __syncthreads();
  return true;
}

// ---- launch plumbing ------------------------------------------------------------
// Kernel ids (instrumentation: launch counts and CUDA-event timing of one id).
enum KernelId {
  KID_DT = 0, KID_DIV, KID_PRED, KID_FLUXN, KID_ASM, KID_RHS, KID_CORR, KID_ACCEL, KID_DUST, KID_DERIVE,
  KID_CG_INIT, KID_CG_MATVEC, KID_CG_UPDATE, KID_CG_DIR, KID_TRUE_RES,
  KID_BICG_INIT, KID_BICG_P, KID_BICG_V, KID_BICG_S, KID_BICG_T, KID_BICG_X,
  KID_COMMIT, KID_DINV, KID_MIX_RES, KID_MIX_ACC, KID_MIX_FIN, KID_FCG_DOTS, KID_FCG_DIR, KID_FCG_MATVEC,
  KID_CG_DIRMATVEC, KID_CG_RUPDATE, KID_CG_XFINAL, KID_REFINE, KID_UNET, KID_TF_PRED, KID_TF_CORR, KID_FE_CELL,
  KID_FE_FACE, KID_CG_START, KID_OTHER,
  KID_COUNT
};

struct Prof;  // defined in fe_api.cu
void prof_begin(Prof* p, int kid, cudaStream_t st);
void prof_end(Prof* p, int kid, cudaStream_t st);

struct Launch {
  const BoxDev* boxes;
  const int2* work;   // stencil tiles (box, tile)
  int nblocks;
  const int2* ework;  // element-wise chunks (box, chunk)
  int neblocks;
  double* part;
  int* active;  // number of boxes whose Krylov solve is running
  cudaStream_t st;
  Prof* prof;
  int fourier;    // closure of the context (selects kernel variants)
  int transonic;  // transonic pressure operator
  int nd;         // dust classes
  int ring_ok;        // every box's N is a multiple of the 16-byte chunk (ring kernels usable)
  const int2* bwork;  // plane-streaming blocks (box, block of box); null: z-marching kernels
  int nbblocks;
  int bsmem;          // dynamic shared memory of the streamed CG kernel
  int* rstart = nullptr;  // right-hand-side kernels: also start the refined solve (outer counter)
  int ysum = -1;          // two-way coupling: slot of the dust loading sum_j Y_j^n (-1: one-way)
  int poly = 0;           // streamed CG with the Neumann polynomial preconditioner (needs bwork)
  int bcells = 0;         // cells per block of the streamed CG kernels (kBulkCells or kBulkCellsPoly)
};

// Launch `call` (a kernel launch statement) under instrumentation id kid.
#define FE_LAUNCH(L, kid, call)          \
  do {                                   \
    prof_begin((L).prof, (kid), (L).st); \
    call;                                \
    prof_end((L).prof, (kid), (L).st);   \
  } while (0)

// Two-fluid dust phase after the gas step s -> ks (twofluid.cu); V = u in set s.
template <typename T> void launch_two_fluid(const Launch& L, int s, int ks);
template <typename T> void launch_two_fluid_init(const Launch& L, int s, int box);
template <typename T> int tfprepare();  // shared-memory limits of the two-fluid ring kernels (before any capture)

// Step kernels (step_kernels.cu); T = field type.
template <typename T> void launch_dt(const Launch& L, int s, int first);
template <typename T> void launch_div(const Launch& L, int uslot0);
template <typename T> void launch_dt_div(const Launch& L, int s);  // adaptive dt and div u^n (one pass where it can)
template <typename T> void launch_pred(const Launch& L, int s, int k);
template <typename T> void launch_fluxn(const Launch& L, int s);
template <typename T> void launch_asm(const Launch& L, int s, int uprev0, int phiprev0, int rhoprev);
template <typename T> void launch_rhs(const Launch& L, int s, int rhoprev, int pprev);
template <typename T> void launch_corr(const Launch& L, int s, int rhoprev, int pprev, int pnew, int kset, int kidx,
                                      int mixed);
template <typename T> void launch_accel(const Launch& L, int kset, int pk);
template <typename T> void launch_dust(const Launch& L, int s, int kset, int pk, int yprev0, int ynew0, int eprev,
                                      int enew, int last, int first);
template <typename T> void launch_derive_box(const Launch& L, int s, int box);
template <typename T> void launch_ysum(const Launch& L, int s);  // W_YSUM = sum_j Y_j of set s
// Krylov kernels (krylov_kernels.cu); V = vector type.
template <typename V> void launch_cg_init(const Launch& L, double dt_override);
template <typename V> void launch_cg_matvec(const Launch& L);
template <typename V> void launch_cg_update(const Launch& L);
template <typename V> void launch_cg_fused(const Launch& L);   // symmetric operator: dir + matvec, then update
template <typename V> void launch_cg_xfinal(const Launch& L);  // after launch_cg_fused iterations
template <typename V> void launch_refine_start(const Launch& L, int* outer_active);  // fused refinement: start from K_B
template <typename V> void launch_refine(const Launch& L, int* outer_active);          // fused refinement: boundary
template <typename V> void launch_cg_start(const Launch& L);  // polynomial-preconditioned CG: first z = P r
template <typename V> void launch_mix_finish_pp(const Launch& L);  // final x from the ping-ponged pairs
// PISO kernels on asynchronous-copy rings (return 0: not launched, use the z-marching kernel)
template <typename V> int rprepare();  // shared-memory limits of the ring kernels on the current device
template <typename V> int rlaunch_corr(const Launch& L, int s, int rhop, int pp, int pnew, int kset, int kidx, int mixed);
template <typename V> int rlaunch_pred(const Launch& L, int s, int kset);
template <typename V> int rlaunch_asm(const Launch& L, int s, int up0, int php0, int rhop);
template <typename V> int rlaunch_accel(const Launch& L, int kset, int pk);
template <typename V> int rlaunch_fluxn(const Launch& L, int s, int nd);
template <typename V> int rlaunch_dust(const Launch& L, int s, int kset, int yp0, int yn0, int last, int nd);
// Fourier closure: dust, energy E^k (to slot enew unless negative) and, last, T, p and totals
template <typename V> int rlaunch_dust_fourier(const Launch& L, int s, int kset, int yp0, int yn0, int enew, int last,
                                               int nd);
template <typename V> int rlaunch_div(const Launch& L, int u0, int with_dt = 0);
template <typename V> int rlaunch_fe_cell(const Launch& L, int s, int u0, int rhos, int ps, int es, int tmode);
template <typename V> int rlaunch_fe_face(const Launch& L, int u0, int phi0);
template <typename V> int rlaunch_rhs(const Launch& L, int s, int rhop, int pp);
template <typename V> int bulk_cg_cells(int minN, int maxN, bool poly);  // cells per block of the streamed CG kernels
template <typename V> int bulk_cg_prepare(int N, int cells, bool poly);  // their dynamic smem (0: unusable)
template <typename V> int bulk_cg_blocks_per_sm(int smem_bytes, int cells);
int bulk_cg_pairs(int N, int cells);  // (row group, plane) pairs of the streamed CG kernels for an N^3 box
template <typename V> void launch_cg_dir(const Launch& L);
template <typename V> void launch_true_res(const Launch& L, int xslot);
template <typename V> void launch_bicg_init(const Launch& L);
template <typename V> void launch_bicg_p(const Launch& L);
template <typename V> void launch_bicg_v(const Launch& L);
template <typename V> void launch_bicg_s(const Launch& L);
template <typename V> void launch_bicg_x(const Launch& L);
template <typename V> void launch_mix_residual(const Launch& L, int first, int* outer_active);
template <typename V> void launch_mix_accum(const Launch& L);
template <typename V> void launch_mix_finish(const Launch& L);
template <typename V> void launch_fcg(const Launch& L, const float* z);

}  // namespace fe
