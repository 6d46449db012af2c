// noalloc.cu -- an allocation-free variant of the Jacobi-PCG pressure solve.
//
// Some callers cannot allocate device memory: code that runs while another
// framework owns the device allocator, real-time loops where an allocation
// could stall, or hosts that reserve all memory up front.  For them
// fe_solve_pressure_noalloc solves the same pressure-correction equation as
// fe_solve_pressure (Jacobi-preconditioned CG on
// psi x/dt - dt/2 D(G2 x) = b) without any context and without allocating:
// its Krylov vectors, block partial sums and scalars live in one file-scope
// device array of fixed size, sized for grids up to FE_NOALLOC_MAX_N^3.
//
// The array exists once per device that loads this library and stays
// allocated until the process exits.  Every call on a device reuses it and
// it keeps the previous call's contents, so a call clears the parts that
// must start at zero (reduction counter, convergence flags).  Calls that run
// at the same time on one device (different streams or threads) share the
// array and race; serialise them.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the entry point looks up the device address
// with cudaGetSymbolAddress while the caller's device is current and caches
// it per CUDA context: a context that is destroyed and created again (after
// cudaDeviceReset, for instance) loads the module afresh, and its address is
// looked up again.
//
// The solve is driven from the host: it reads the convergence flag back
// every few iterations and waits for the stream, so it cannot be recorded
// into a CUDA graph.  A call on a stream that is being captured returns
// FE_ERR_UNSUPPORTED before it enqueues anything.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fe_internal.cuh"

namespace fe {

constexpr int NA_MAX_N = FE_NOALLOC_MAX_N;
constexpr long NA_MAX_CELLS = (long)NA_MAX_N * NA_MAX_N * NA_MAX_N;
constexpr int NA_TZ = 4;
constexpr int NA_MAX_BLOCKS = ((NA_MAX_N + TX - 1) / TX) * ((NA_MAX_N + TY - 1) / TY) * ((NA_MAX_N + NA_TZ - 1) / NA_TZ);
// layout in doubles: r | pd | q | block partials | scalars | counter
constexpr long NA_OFF_PART = 3 * NA_MAX_CELLS;
constexpr long NA_OFF_SC = NA_OFF_PART + (long)NA_MAX_BLOCKS * MAXP;
constexpr long NA_OFF_CNT = NA_OFF_SC + NSC;
constexpr long NA_TOTAL = NA_OFF_CNT + 8;

static __device__ __align__(256) double fe_noalloc_scratch[NA_TOTAL];

__device__ __forceinline__ Tile na_tile(const BoxDev& B) {
  Tile t;
  t.box = 0;
  int q = blockIdx.x;
  int tx = q % B.tnx;
  int r = q / B.tnx;
  int ty = r % B.tny;
  int tzb = r / B.tny;
  t.i = tx * TX + threadIdx.x;
  t.j = ty * TY + threadIdx.y;
  t.k0 = tzb * B.tz;
  t.kend = min(t.k0 + B.tz, B.N);
  t.active = (t.i < B.N) && (t.j < B.N);
  return t;
}

__device__ __forceinline__ double na_diag(const BoxDev& B, double psic, double dt) {
  return psic / dt + 3.0 * dt * B.ih * B.ih;
}

__global__ void __launch_bounds__(NTHR) na_init(BoxDev B) {
  Tile t = na_tile(B);
  const double* b = (const double*)B.f[K_B];
  const double* psi = (const double*)B.f[W_PSI];
  double* r = (double*)B.f[K_R];
  double* x = (double*)B.f[K_X];
  double* pd = (double*)B.f[K_PD];
  double* part = (double*)B.f[K_AUX];
  const double dt = B.sc[SC_KDT];
  double v[2] = {0.0, 0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      double bc = b[c];
      double z = bc / na_diag(B, psi[c], dt);
      r[c] = bc;
      x[c] = 0.0;
      pd[c] = z;
      v[0] += bc * z;
      v[1] += bc * bc;
    }
  }
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.sc[SC_RZ] = res[0];
      B.sc[SC_BB] = res[1];
      B.sc[SC_ITERS] = 0.0;
      bool zero = !(res[1] > 0.0);
      B.sc[SC_DONE] = zero ? 1.0 : 0.0;
      B.sc[SC_CONV] = zero ? 1.0 : 0.0;
    }
  }
}

__device__ __forceinline__ double na_applyM(const BoxDev& B, const double* v, const Nbr& n, double dt) {
  const double* psi = (const double*)B.f[W_PSI];
  const int c = n(0, 0, 0);
  const double vc = v[c];
  double lap = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) lap += (v[n.at(d, 0, 0, 0, 1)] - vc) - (vc - v[n.at(d, 0, 0, 0, -1)]);
  return psi[c] * vc / dt - 0.5 * dt * lap * B.ih * B.ih;
}

__global__ void __launch_bounds__(NTHR) na_matvec(BoxDev B) {
  if (B.sc[SC_DONE] != 0.0) return;
  Tile t = na_tile(B);
  const double* pd = (const double*)B.f[K_PD];
  double* q = (double*)B.f[K_Q];
  double* part = (double*)B.f[K_AUX];
  const double dt = B.sc[SC_KDT];
  double v[1] = {0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      int c = n(0, 0, 0);
      double y = na_applyM(B, pd, n, dt);
      q[c] = y;
      v[0] += pd[c] * y;
    }
  }
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) B.sc[SC_ALPHA] = B.sc[SC_RZ] / res[0];
  }
}

__global__ void __launch_bounds__(NTHR) na_update(BoxDev B) {
  if (B.sc[SC_DONE] != 0.0) return;
  Tile t = na_tile(B);
  const double* pd = (const double*)B.f[K_PD];
  const double* q = (const double*)B.f[K_Q];
  const double* psi = (const double*)B.f[W_PSI];
  double* x = (double*)B.f[K_X];
  double* r = (double*)B.f[K_R];
  double* part = (double*)B.f[K_AUX];
  const double dt = B.sc[SC_KDT], alpha = B.sc[SC_ALPHA];
  double v[2] = {0.0, 0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      int c = t.i + B.N * (t.j + B.N * k);
      x[c] = x[c] + alpha * pd[c];
      double rc = r[c] - alpha * q[c];
      r[c] = rc;
      double z = rc / na_diag(B, psi[c], dt);
      v[0] += rc * z;
      v[1] += rc * rc;
    }
  }
  __shared__ double res[2];
  if (block_sum_last<2>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double it = B.sc[SC_ITERS] + 1.0;
      B.sc[SC_ITERS] = it;
      if (sqrt(res[1]) <= B.sc[SC_TOL] * sqrt(B.sc[SC_BB])) {
        B.sc[SC_DONE] = 1.0;
        B.sc[SC_CONV] = 1.0;
      } else if (it >= B.sc[SC_MAXIT]) {
        B.sc[SC_DONE] = 1.0;
        B.sc[SC_CONV] = 0.0;
      } else {
        B.sc[SC_BETA] = res[0] / B.sc[SC_RZ];
        B.sc[SC_RZ] = res[0];
      }
    }
  }
}

__global__ void __launch_bounds__(NTHR) na_dir(BoxDev B) {
  if (B.sc[SC_DONE] != 0.0) return;
  Tile t = na_tile(B);
  if (!t.active) return;
  const double* r = (const double*)B.f[K_R];
  const double* psi = (const double*)B.f[W_PSI];
  double* pd = (double*)B.f[K_PD];
  const double dt = B.sc[SC_KDT], beta = B.sc[SC_BETA];
  for (int k = t.k0; k < t.kend; ++k) {
    int c = t.i + B.N * (t.j + B.N * k);
    pd[c] = r[c] / na_diag(B, psi[c], dt) + beta * pd[c];
  }
}

__global__ void __launch_bounds__(NTHR) na_true_res(BoxDev B) {
  Tile t = na_tile(B);
  const double* x = (const double*)B.f[K_X];
  const double* b = (const double*)B.f[K_B];
  double* part = (double*)B.f[K_AUX];
  const double dt = B.sc[SC_KDT];
  double v[1] = {0.0};
  if (t.active) {
    for (int k = t.k0; k < t.kend; ++k) {
      Nbr n(t.i, t.j, k, B.N);
      double r = b[n(0, 0, 0)] - na_applyM(B, x, n, dt);
      v[0] += r * r;
    }
  }
  __shared__ double res[1];
  if (block_sum_last<1>(v, B, part, res, B.tile0, B.ntiles)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) B.sc[SC_TRUE_RR] = res[0];
  }
}

// Cache of the scratch array's device address, keyed by (device, context id).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

struct NaSlot {
  int dev;
  unsigned long long ctx;
  double* ptr;
};
static std::mutex g_na_mutex;
static NaSlot g_na_cache[16];
static int g_na_used = 0;

// Unique id of the context current on this thread (0 if it cannot be told).
static unsigned long long na_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_cur = (CtxGetCurrentFn)f1;
      get_id = (CtxGetIdFn)f2;
    }
  }
  if (!get_cur || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

static int na_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return FE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  const unsigned long long ctx = na_context_id();
  if (ctx != 0)
    for (int q = 0; q < g_na_used; ++q)
      if (g_na_cache[q].dev == dev && g_na_cache[q].ctx == ctx) {
        *out = g_na_cache[q].ptr;
        return FE_OK;
      }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, fe_noalloc_scratch) != cudaSuccess || !p) return FE_ERR_CUDA;
  if (ctx != 0) {  // without a context id the address is looked up on every call
    const int q = g_na_used < 16 ? g_na_used++ : (int)(ctx % 16);
    g_na_cache[q] = NaSlot{dev, ctx, (double*)p};
  }
  *out = (double*)p;
  return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" int fe_solve_pressure_noalloc(int N, const double* psi, const double* b, double* x, double dt, double tol,
                                         int maxit, void* stream, fe_solve_info* info) {
  if (N > FE_NOALLOC_MAX_N) return FE_ERR_TOO_LARGE;
  if (N < 8 || !psi || !b || !x || !(dt > 0.0) || !(tol > 0.0) || maxit < 1) return FE_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // a stale launch error left by earlier, unrelated work is not this call's
  (void)cudaGetLastError();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return FE_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return FE_ERR_UNSUPPORTED;  // host-polled: cannot be captured
  double* base = nullptr;
  int rc = na_scratch(&base);
  if (rc != FE_OK) return rc;
  BoxDev B;
  memset(&B, 0, sizeof(B));
  B.N = N;
  B.tz = NA_TZ;
  B.tnx = (N + TX - 1) / TX;
  B.tny = (N + TY - 1) / TY;
  B.tnz = (N + NA_TZ - 1) / NA_TZ;
  B.ntiles = B.tnx * B.tny * B.tnz;
  B.tile0 = 0;
  B.h = 2.0 * M_PI / N;
  B.ih = 1.0 / B.h;
  B.f[K_R] = base;
  B.f[K_PD] = base + NA_MAX_CELLS;
  B.f[K_Q] = base + 2 * NA_MAX_CELLS;
  B.f[K_AUX] = base + NA_OFF_PART;
  B.f[W_PSI] = (void*)psi;
  B.f[K_B] = (void*)b;
  B.f[K_X] = x;
  B.sc = base + NA_OFF_SC;
  B.cnt = (int*)(base + NA_OFF_CNT);
  // clear what must start at zero: scalars (flags) and the reduction counter
  if (cudaMemsetAsync(B.sc, 0, (NSC + 8) * sizeof(double), st) != cudaSuccess) return FE_ERR_CUDA;
  double hs[3] = {tol, (double)maxit, dt};
  if (cudaMemcpyAsync(B.sc + SC_TOL, hs, sizeof(hs), cudaMemcpyHostToDevice, st) != cudaSuccess) return FE_ERR_CUDA;
  const dim3 blk(TX, TY);
  na_init<<<B.ntiles, blk, 0, st>>>(B);
  if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
  const int poll = 4;
  double done = 0.0;
  for (int it = 0; it < maxit;) {
    if (cudaMemcpyAsync(&done, B.sc + SC_DONE, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FE_ERR_CUDA;
    if (done != 0.0) break;
    for (int q = 0; q < poll && it < maxit; ++q, ++it) {
      na_matvec<<<B.ntiles, blk, 0, st>>>(B);
      na_update<<<B.ntiles, blk, 0, st>>>(B);
      na_dir<<<B.ntiles, blk, 0, st>>>(B);
    }
    if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
  }
  na_true_res<<<B.ntiles, blk, 0, st>>>(B);
  if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
  double sc[NSC];
  if (cudaMemcpyAsync(sc, B.sc, NSC * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FE_ERR_CUDA;
  if (info) {
    info->iters = (int)sc[SC_ITERS];
    info->rel_res_true = sc[SC_BB] > 0.0 ? sqrt(sc[SC_TRUE_RR] / sc[SC_BB]) : 0.0;
  }
  return sc[SC_CONV] != 0.0 ? FE_OK : FE_ERR_NOT_CONVERGED;
}
