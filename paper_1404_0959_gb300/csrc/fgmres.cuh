// fgmres.cuh -- vector kernels of flexible GMRES(m) (Saad, "A flexible
// inner-outer preconditioned GMRES algorithm", SIAM J. Sci. Comput. 14, 1993)
// for the pressure-correction equation of one box: multi-vector dot products
// with FP64-class accumulation (block partial sums, added by the host in block
// order), linear combinations of basis vectors, the Jacobi direction and the
// conversion of the network output.  The operator is the library's own matvec
// kernel; the Arnoldi bookkeeping (Hessenberg matrix, Givens rotations,
// least-squares update) runs on the host in FP64.
#pragma once
#include <cuda_runtime.h>

namespace fe {

constexpr int kGmMax = 32;         // largest restart length
constexpr int kGmPart = kGmMax + 2;  // partial sums per block: <v_i, w> for i < kGmMax + 1, then <w, w>

#ifndef FE_FGMRES_M
#define FE_FGMRES_M 20
#endif
constexpr int kGmRestart = FE_FGMRES_M;
// A network direction is kept only if its Arnoldi column shrinks the
// least-squares residual to at most this fraction of its previous value
// (|sin| of the new Givens rotation); otherwise the Jacobi direction replaces it.
constexpr double kGmNetKeep = 0.9;
// ... and only if its image M z has a new component of at least this fraction
// of its norm (not already in the span of the basis).
constexpr double kGmNetFresh = 1e-5;
static_assert(kGmRestart >= 1 && kGmRestart <= kGmMax, "restart length within the kernels' bound");

// Coefficients of a linear combination, passed by value.
struct GmCoef {
  double h[kGmMax + 1];
};

// part[b * kGmPart + i] = block b's share of <V_i, w> (i < nv, V_i = V + i n)
// and part[b * kGmPart + kGmMax + 1] = of <w, w>.  nv <= kGmMax + 1.
template <typename T>
void gm_dots(const T* V, long n, int nv, const T* w, double* part, int nblk, cudaStream_t st);
// out = sa a + sum_{i < nv} h_i V_i (out may alias a; nv <= kGmMax + 1).
template <typename T>
void gm_combine(T* out, const T* a, double sa, const T* V, long n, int nv, const GmCoef& h, int nblk,
                cudaStream_t st);
// z = dinv v.
template <typename T>
void gm_jacobi(T* z, const T* v, const T* dinv, long n, int nblk, cudaStream_t st);
// z = dinv v + sc[SC_NSCALE] net (residual-form network direction for v); part[b] = block b's
// share of ||z||^2 (not finite if any net value is not).
template <typename T>
void gm_from_net(T* z, const T* v, const T* dinv, const float* net, const double* sc, long n, double* part, int nblk,
                 cudaStream_t st);
// sc[slot] = v (one thread).
void gm_set_scalar(double* sc, int slot, double v, cudaStream_t st);
// End of a solve: iteration count, squared residual, verdict; marks the box
// done and leaves the running-solve counter.
void gm_finish(double* sc, int* active, double iters, double rr, int conv, cudaStream_t st);

}  // namespace fe
