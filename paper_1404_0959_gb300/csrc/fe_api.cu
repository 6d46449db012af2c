// fe_api.cu -- the C ABI of libfe (include/fe.h): context, memory plan, the
// PISO step driver (Sec. 2 par. 1 of arXiv:1404.0959) and the solve /
// diagnostics entry points.  All device memory of a context is allocated in
// fe_create (one slab per box) and freed in fe_destroy; the step itself
// allocates nothing.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "fe_internal.cuh"
#include "fgmres.cuh"

using namespace fe;

namespace fe {
bool fft_supported(int N);
template <typename T> int ic_spectral(T*, T*, T*, int, uint64_t, double, double, cudaStream_t);
template <typename T> void fill(T*, long, double, cudaStream_t);
template <typename T> int spectrum(const T*, const T*, const T*, int, double*, int, cudaStream_t);
template <typename T> int diag_sums(const Launch&, const BoxDev&, int, int, double*);
template <typename T> void qcrit(const Launch&, int, int, T*);
struct UNet;
template <typename T>
int les_apriori(const T* rho, const T* u0, const T* u1, const T* u2, int N, int m, double cs, T* work, double* part,
                double* hpart, int nsm, T* out, double* stats, cudaStream_t st);
int les_max_blocks(int nsm);
template <typename T>
int isosurface(const T* f, int N, double iso, double* tri, long long max_tri, void* work,
               std::vector<double>& hscratch, int nsm, long long* ntri, double* area, cudaStream_t st);
size_t iso_work_bytes(long n);
int raster_depth(const double* tri, long long ntri, int W, double extent, float* depth, int nsm, cudaStream_t st);
UNet* unet_create(int N, bool training, int* rc);
void unet_destroy(UNet* U);
long unet_param_count();
int unet_set_weights(UNet* U, const float* host, cudaStream_t st);
int unet_get_weights(UNet* U, float* host, int which, cudaStream_t st);
template <typename T> void unet_apply_sc(UNet*, const T*, const T*, double*, int, double, cudaStream_t);
template <typename T> int unet_apply(UNet*, const T*, const T*, double, double, float*, cudaStream_t);
template <typename T>
int unet_train_step(UNet*, const T*, const T*, const T*, double, double, double, double*, cudaStream_t);
float* unet_output(UNet* U);
int unet_activation(UNet* U, int l, float* host, long count, cudaStream_t st);
void unet_set_kernels(UNet* U, int tc);
}  // namespace fe

namespace fe {
struct Prof {
  bool on = false;
  int target = -1;
  long long count[KID_COUNT] = {};
  std::vector<cudaEvent_t> ev;  // start/stop pairs of the target kernel
  size_t used = 0;
  bool failed = false;
};
void prof_begin(Prof* p, int kid, cudaStream_t st) {
  if (!p || !p->on) return;
  p->count[kid]++;
  if (kid != p->target) return;
  while (p->ev.size() < 2 * (p->used + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      p->failed = true;
      return;
    }
    p->ev.push_back(e);
  }
  cudaEventRecord(p->ev[2 * p->used], st);
}
void prof_end(Prof* p, int kid, cudaStream_t st) {
  if (!p || !p->on || kid != p->target || p->failed) return;
  cudaEventRecord(p->ev[2 * p->used + 1], st);
  p->used++;
}
}  // namespace fe

static const char* kKernelNames[] = {
    "dt",      "div",       "pred",      "fluxn",  "asm",      "rhs",       "corr",    "accel",
    "dust",    "derive",    "cg_init",   "cg_matvec", "cg_update", "cg_dir", "true_res", "bicg_init",
    "bicg_p",  "bicg_v",    "bicg_s",    "bicg_t", "bicg_x",   "commit",    "dinv",
    "mix_residual", "mix_accum", "mix_finish", "fcg_dots", "fcg_dir", "fcg_matvec",
    "cg_dirmatvec", "cg_rupdate", "cg_xfinal", "refine", "unet", "tf_pred", "tf_corr", "fe_cell", "fe_face", "cg_start",
    "other"};
static_assert(sizeof(kKernelNames) / sizeof(kKernelNames[0]) == KID_COUNT, "kernel name table");
static_assert(KID_COUNT <= FE_PROFILE_MAX_KERNELS, "profile counters");

struct fe_ctx {
  fe_params prm;
  std::vector<int32_t> N;
  std::vector<double> nu, tau_p, Y0, mach, k0;
  std::vector<uint64_t> seed;
  cudaStream_t st = nullptr;
  int nb = 0;
  bool fp64 = true;
  std::vector<BoxDev> hbox;
  std::vector<void*> slabs;
  BoxDev* dbox = nullptr;
  int2* dwork = nullptr;
  int nblocks = 0;
  int2* dework = nullptr;
  int2* dbwork = nullptr;   // plane-streaming blocks (box, block of box)
  int nbblocks = 0, bsmem = 0, bcells = 0, npart = 0;
  int ring_ok = 0;          // all N multiples of the 16-byte chunk of the ring kernels
  bool use_bulk = true;     // streamed CG kernel where the boxes allow it
  int unet_tc = 1;          // U-Net stride-1 layers on tcgen05 (1) or warp-level MMA (0)
  int neblocks = 0;
  std::vector<int> tzb;    // tile depth per box (0: default for its N)
  int nsm = 152;           // multiprocessors of the device
  double* dpart = nullptr;
  double* dsc = nullptr;
  int* dcnt = nullptr;
  int* dactive = nullptr;
  int* douter = nullptr;   // boxes whose refinement loop is running
  int* hactive = nullptr;  // pinned
  double* hsc = nullptr;   // pinned copy of all box scalars
  int cur = 0;             // state set holding the current state
  int hint[16] = {};       // iterations of the previous Krylov solve, per solve key
  UNet* unet = nullptr;    // learned preconditioner (FE_FCG_LEARNED, FE_FGMRES_LEARNED)
  void* gm_basis = nullptr;   // FE_FGMRES_LEARNED: Arnoldi basis V (m + 1 vectors), directions Z (m)
  double* gm_part = nullptr;  // its block partial sums (device) ...
  double* gm_hpart = nullptr; // ... and their pinned host copy
  int gm_blocks = 0;
  bool use_graphs = false;           // step as one CUDA graph with WHILE nodes for the solves
  cudaGraphExec_t gexec[2] = {};     // per parity of the current state set
  cudaStream_t cap[3] = {};          // capture streams (loop nesting levels)
  int* dloop = nullptr;              // loop iteration counters
  bool unet_ready = false;
  void* const* harvest_b = nullptr;  // fe_harvest_pressure: per-corrector copies of b and x
  void* const* harvest_x = nullptr;
  int harvest_max = 0, harvest_n = 0;
  Prof prof;
  void* les_work = nullptr;   // fe_les_apriori: 23 N^3 arrays of the largest box (allocated on first use)
  size_t les_bytes = 0;
  double* les_part = nullptr;  // its block partial sums (device) and their pinned host copy
  double* les_hpart = nullptr;
  void* iso_work = nullptr;     // fe_isosurface: per-cube counts and block scan (allocated on first use)
  size_t iso_bytes = 0;
  std::vector<double> iso_host;
  Launch L() {
    Launch l{dbox,           dwork,         nblocks,       dework, neblocks, dpart, dactive, st, &prof,
             prm.closure == FE_FOURIER, prm.transonic, prm.n_dust, ring_ok, use_bulk && nbblocks > 0 ? dbwork : nullptr,
             nbblocks, bsmem};
    l.poly = prm.solver == FE_PCG_POLY && !fp64;  // FP64 contexts run Jacobi-PCG
    l.bcells = bcells;
    return l;
  }
};

static void drop_graphs(fe_ctx* c);

#define CK(x)                                     \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return FE_ERR_CUDA;    \
  } while (0)

static size_t slot_bytes(int N, size_t esz) {
  size_t b = (size_t)N * N * N * esz;
  return (b + 255) & ~(size_t)255;
}

// Which slots a box needs and their element sizes.
static void slot_plan(const fe_ctx* c, std::vector<std::pair<int, size_t>>& plan) {
  const size_t e = c->fp64 ? 8 : 4;
  const int nd = c->prm.n_dust;
  const bool fourier = c->prm.closure == FE_FOURIER;
  const bool two_fluid = c->prm.dust_model == FE_DUST_TWO_FLUID;
  for (int set = 0; set < 2; ++set) {
    for (int f = F_RHO; f <= F_P; ++f) plan.push_back({S(set, f), e});
    if (fourier) plan.push_back({S(set, F_T), e});
    for (int j = 0; j < nd; ++j) plan.push_back({S(set, F_Y0 + j), e});
    if (two_fluid)
      for (int q = 0; q < 3 * nd; ++q) plan.push_back({S(set, F_V0 + q), e});
  }
  if (two_fluid)
    for (int q = 0; q < 4 * nd; ++q) {
      plan.push_back({W_TFN0 + q, e});
      plan.push_back({W_TFS0 + q, e});
    }
  int w[] = {W_DIV, W_DIVPHI, W_RN0, W_RN1, W_RN2, W_AN0, W_AN1, W_AN2, W_PSI, W_DINV, W_HB0, W_HB1, W_HB2,
             W_PS0, W_PS1, W_PS2, W_PW0, W_PW1, K_B, K_X, K_R, K_PD, K_Q, K_AUX};
  for (int s : w) plan.push_back({s, e});
  if (fourier) {
    for (int s : {(int)W_EW0, (int)W_EW1, (int)W_FEN, (int)W_FEH, (int)W_FET}) plan.push_back({s, e});
    for (int q = 0; q < 9; ++q) plan.push_back({W_FEG0 + q, e});
    for (int q = 0; q < 3; ++q) plan.push_back({W_FEF0 + q, e});
    plan.push_back({W_EN, e});
    plan.push_back({W_FED, e});
  }
  for (int j = 0; j < nd; ++j) {
    plan.push_back({W_FYN0 + j, e});
    plan.push_back({W_YW0 + j, e});
    plan.push_back({W_YW1 + j, e});
  }
  if (c->prm.coupling == FE_COUPLING_TWO_WAY && nd > 1) plan.push_back({W_YSUM, e});
  // BiCGStab vectors: its own solver, and the harvest of a transonic flexible-GMRES context (which
  // generates its training pairs with BiCGStab)
  if (c->prm.solver == FE_BICGSTAB_JACOBI || (c->prm.solver == FE_FGMRES_LEARNED && c->prm.transonic))
    for (int s : {K_RHAT, K_V, K_S, K_T}) plan.push_back({s, e});
  // second CG direction buffer (the learned solver's harvest runs plain CG)
  if (c->prm.solver != FE_BICGSTAB_JACOBI) plan.push_back({K_PP, e});
  if (c->prm.solver == FE_PCG_POLY && !c->fp64) {  // z = P r and the residual ping-pong of the streamed CG
    plan.push_back({K_Z, e});
    plan.push_back({K_RB, e});
  }
  if (!c->fp64) plan.push_back({K_X64, 8});
  if (!c->fp64 && c->prm.solver != FE_BICGSTAB_JACOBI) {
    plan.push_back({K_X64B, 8});
    plan.push_back({K_XH, e});
  }
}

static int validate(const fe_params* p) {
  if (!p || p->n_boxes < 1 || !p->N || !p->nu || !p->mach_rms || !p->k0 || !p->seed) return FE_ERR_INVALID_ARG;
  if (p->precision != FE_FP64 && p->precision != FE_FP32_MIXED) return FE_ERR_INVALID_ARG;
  if (p->closure != FE_BAROTROPIC && p->closure != FE_FOURIER) return FE_ERR_INVALID_ARG;
  if (p->n_dust < 0 || p->n_dust > FE_MAX_DUST) return FE_ERR_INVALID_ARG;
  if (p->n_dust > 0 && (!p->tau_p || !p->Y0)) return FE_ERR_INVALID_ARG;
  if (p->n_corr < 1 || p->n_corr > 4) return FE_ERR_INVALID_ARG;
  if (p->dust_model != FE_DUST_EQUILIBRIUM && p->dust_model != FE_DUST_TWO_FLUID) return FE_ERR_INVALID_ARG;
  if (p->dust_model == FE_DUST_TWO_FLUID)
    for (int q = 0; q < p->n_boxes * p->n_dust; ++q)
      if (!(p->tau_p[q] > 0.0)) return FE_ERR_INVALID_ARG;
  if (p->coupling != FE_COUPLING_ONE_WAY && p->coupling != FE_COUPLING_TWO_WAY) return FE_ERR_INVALID_ARG;
  if (p->coupling == FE_COUPLING_TWO_WAY && (p->closure != FE_BAROTROPIC || p->dust_model != FE_DUST_EQUILIBRIUM))
    return FE_ERR_UNSUPPORTED;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->p_tol > 0.0) || p->p_maxit < 1) return FE_ERR_INVALID_ARG;
  if (p->closure == FE_FOURIER && !(p->Pr > 0.0)) return FE_ERR_INVALID_ARG;
  if (p->solver != FE_PCG_JACOBI && p->solver != FE_BICGSTAB_JACOBI && p->solver != FE_FCG_LEARNED &&
      p->solver != FE_FGMRES_LEARNED && p->solver != FE_PCG_POLY)
    return FE_ERR_INVALID_ARG;
  if (p->transonic && (p->solver == FE_PCG_JACOBI || p->solver == FE_PCG_POLY)) return FE_ERR_INVALID_ARG;
  if (p->solver == FE_FCG_LEARNED && (p->n_boxes != 1 || p->N[0] % 4 != 0 || p->transonic))
    return FE_ERR_UNSUPPORTED;
  if (p->solver == FE_FGMRES_LEARNED && (p->n_boxes != 1 || p->N[0] % 4 != 0)) return FE_ERR_UNSUPPORTED;
  if (p->learned_every < 0) return FE_ERR_INVALID_ARG;
  for (int b = 0; b < p->n_boxes; ++b)
    if (p->N[b] < 8 || p->N[b] > 512 || !(p->nu[b] >= 0.0)) return FE_ERR_INVALID_ARG;
  return FE_OK;
}

// Element-wise kernels: chunks per SM over all boxes (each block one chunk).
#ifndef FE_ECHUNKS
#define FE_ECHUNKS 8  // one wave of eight 256-thread blocks per SM (measured: the residual update 57 -> 54 us at 256^3)
#endif
static int tz_for(int N) { return N >= 128 ? 8 : 4; }

// (Re)build both work lists for tile depth tz (0: default per N) and upload the
// descriptors.  Grows the partial-sum buffer when needed.
// tzb[b]: tile depth of box b (0: the default for its N)
static int set_tiling(fe_ctx* c, const std::vector<int>& tzb) {
  std::vector<int2> work, ework;
  // element-wise chunk: about two waves of 8 blocks per SM over all boxes, so
  // the per-block reduction tail (fence + counter) is paid rarely
  long total = 0;
  for (int b = 0; b < c->nb; ++b) total += (long)c->hbox[b].N * c->hbox[b].N * c->hbox[b].N;
  const long quantum = 4L * NTHR;
  long chunk = (total + (long)FE_ECHUNKS * c->nsm - 1) / ((long)FE_ECHUNKS * c->nsm);
  chunk = std::max(quantum, (chunk + quantum - 1) / quantum * quantum);
  for (int b = 0; b < c->nb; ++b) {
    BoxDev& B = c->hbox[b];
    const int N = B.N;
    const int tz = tzb[b];
    B.tz = tz > 0 ? (tz < N ? tz : N) : tz_for(N);
    B.tnx = (N + TX - 1) / TX;
    B.tny = (N + TY - 1) / TY;
    B.tnz = (N + B.tz - 1) / B.tz;
    B.ntiles = B.tnx * B.tny * B.tnz;
    B.tile0 = (int)work.size();
    for (int q = 0; q < B.ntiles; ++q) work.push_back(make_int2(b, q));
    const long n = (long)N * N * N;
    B.echunk = (int)chunk;
    B.entiles = (int)((n + chunk - 1) / chunk);
    B.etile0 = (int)ework.size();
    for (int q = 0; q < B.entiles; ++q) ework.push_back(make_int2(b, q));
  }
  c->ring_ok = 1;
  for (int b = 0; b < c->nb; ++b)
    if (c->hbox[b].N % (c->fp64 ? 2 : 4)) c->ring_ok = 0;
  // plane-streaming blocks (FP32 fields; FP64 contexts are bound by the FP64
  // pipe and keep the z-marching kernel): every box with N in {64, 128, 256,
  // 512}, a persistent grid of the resident blocks per SM x SMs shared out by cells
  std::vector<int2> bwork;
  int bsmem = 0;
  bool stream = !c->prm.transonic && !c->fp64;
  long scells = 0;
  for (int b = 0; b < c->nb && stream; ++b) {
    const int N = c->hbox[b].N;
    stream = N >= 64 && N <= 512 && (N & (N - 1)) == 0;
    scells += (long)N * N * N;
  }
  int bcells = 0;
  if (stream) {
    int maxN = 0, minN = 1 << 30;
    for (int b = 0; b < c->nb; ++b) maxN = std::max(maxN, c->hbox[b].N), minN = std::min(minN, c->hbox[b].N);
    const bool poly = c->prm.solver == FE_PCG_POLY;
    bcells = c->fp64 ? bulk_cg_cells<double>(minN, maxN, poly) : bulk_cg_cells<float>(minN, maxN, poly);
    bsmem = c->fp64 ? bulk_cg_prepare<double>(maxN, bcells, poly) : bulk_cg_prepare<float>(maxN, bcells, poly);
    const int per_sm = bsmem <= 0 ? 0
                       : c->fp64 ? bulk_cg_blocks_per_sm<double>(bsmem, bcells)
                                 : bulk_cg_blocks_per_sm<float>(bsmem, bcells);
    stream = per_sm > 0;
    const long grid = (long)per_sm * c->nsm;
    for (int b = 0; b < c->nb && stream; ++b) {
      BoxDev& B = c->hbox[b];
      const long N = B.N, planes = bulk_cg_pairs(B.N, bcells);
      long nb = (grid * N * N * N + scells - 1) / scells;
      nb = std::max(1L, std::min(nb, planes / 4));
      B.btile0 = (int)bwork.size();
      B.bntiles = (int)nb;
      for (int q = 0; q < B.bntiles; ++q) bwork.push_back(make_int2(b, q));
    }
  }
  if (!stream) {
    bwork.clear();
    bsmem = 0;
    bcells = 0;
    for (int b = 0; b < c->nb; ++b) c->hbox[b].btile0 = c->hbox[b].bntiles = 0;
  }
  CK(cudaStreamSynchronize(c->st));
  const int need = (int)std::max(std::max(work.size(), ework.size()), bwork.size());
  cudaFree(c->dbwork);
  c->dbwork = nullptr;
  if (!bwork.empty() && cudaMalloc(&c->dbwork, bwork.size() * sizeof(int2)) != cudaSuccess) return FE_ERR_OOM;
  if (!bwork.empty())
    CK(cudaMemcpyAsync(c->dbwork, bwork.data(), bwork.size() * sizeof(int2), cudaMemcpyHostToDevice, c->st));
  c->nbblocks = (int)bwork.size();
  c->bsmem = bsmem;
  c->bcells = bcells;
  if ((int)work.size() != c->nblocks || (int)ework.size() != c->neblocks || !c->dpart || need > c->npart) {
    cudaFree(c->dwork);
    cudaFree(c->dework);
    cudaFree(c->dpart);
    c->dwork = c->dework = nullptr;
    c->dpart = nullptr;
    c->npart = 0;
    if (cudaMalloc(&c->dwork, work.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&c->dework, ework.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&c->dpart, (size_t)need * MAXP * sizeof(double)) != cudaSuccess)
      return FE_ERR_OOM;
    c->npart = need;
  }
  c->nblocks = (int)work.size();
  c->neblocks = (int)ework.size();
  c->tzb = tzb;
  drop_graphs(c);
  CK(cudaMemcpyAsync(c->dwork, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->dework, ework.data(), ework.size() * sizeof(int2), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->dbox, c->hbox.data(), c->nb * sizeof(BoxDev), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

static int set_tiling(fe_ctx* c, int tz) { return set_tiling(c, std::vector<int>(c->nb, tz)); }

extern "C" int fe_create(const fe_params* prm, void* stream, fe_ctx** out) {
  if (!out) return FE_ERR_INVALID_ARG;
  *out = nullptr;
  int v = validate(prm);
  if (v != FE_OK) return v;
  fe_ctx* c = new (std::nothrow) fe_ctx();
  if (!c) return FE_ERR_OOM;
  c->prm = *prm;
  c->nb = prm->n_boxes;
  c->fp64 = prm->precision == FE_FP64;
  c->st = (cudaStream_t)stream;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      c->nsm = nsm;
    // ring kernels need their shared-memory limits set before any capture (else z-marching kernels run)
    if (c->fp64) rprepare<double>();
    else rprepare<float>();
    if (prm->dust_model == FE_DUST_TWO_FLUID) {
      if (c->fp64) tfprepare<double>();
      else tfprepare<float>();
    }
  }
  const int nb = c->nb, nd = prm->n_dust;
  c->N.assign(prm->N, prm->N + nb);
  c->nu.assign(prm->nu, prm->nu + nb);
  c->mach.assign(prm->mach_rms, prm->mach_rms + nb);
  c->k0.assign(prm->k0, prm->k0 + nb);
  c->seed.assign(prm->seed, prm->seed + nb);
  if (nd > 0) {
    c->tau_p.assign(prm->tau_p, prm->tau_p + (size_t)nb * nd);
    c->Y0.assign(prm->Y0, prm->Y0 + (size_t)nb * nd);
  }
  c->prm.N = c->N.data();
  c->prm.nu = c->nu.data();
  c->prm.mach_rms = c->mach.data();
  c->prm.k0 = c->k0.data();
  c->prm.seed = c->seed.data();
  c->prm.tau_p = nd ? c->tau_p.data() : nullptr;
  c->prm.Y0 = nd ? c->Y0.data() : nullptr;

  // descriptors (work lists are built by set_tiling)
  c->hbox.resize(nb);
  std::vector<std::pair<int, size_t>> plan;
  slot_plan(c, plan);
  int rc = FE_OK;
  for (int b = 0; b < nb && rc == FE_OK; ++b) {
    BoxDev& B = c->hbox[b];
    memset(&B, 0, sizeof(B));
    const int N = c->N[b];
    B.N = N;
    B.nd = nd;
    B.closure = prm->closure;
    B.transonic = prm->transonic;
    B.h = 2.0 * M_PI / N;
    B.ih = 1.0 / B.h;
    B.mu = c->nu[b];
    B.gamma = prm->gamma;
    B.R = 1.0 / prm->gamma;
    B.cv = B.R / (prm->gamma - 1.0);
    B.kappa = prm->closure == FE_FOURIER ? B.mu * prm->gamma * B.cv / prm->Pr : 0.0;
    B.cfl = prm->cfl;
    B.growth = prm->dt_growth_max > 0 ? prm->dt_growth_max : HUGE_VAL;
    B.dtmax = prm->dt_max > 0 ? prm->dt_max : HUGE_VAL;
    for (int j = 0; j < nd; ++j) B.tau_p[j] = c->tau_p[(size_t)b * nd + j];
    size_t total = 0;
    for (auto& s : plan) total += slot_bytes(N, s.second);
    void* slab = nullptr;
    if (cudaMalloc(&slab, total) != cudaSuccess) {
      rc = FE_ERR_OOM;
      break;
    }
    c->slabs.push_back(slab);
    cudaMemsetAsync(slab, 0, total, c->st);
    size_t off = 0;
    for (auto& s : plan) {
      B.f[s.first] = (char*)slab + off;
      off += slot_bytes(N, s.second);
    }
  }
  if (rc == FE_OK) {
    if (cudaMalloc(&c->dbox, nb * sizeof(BoxDev)) != cudaSuccess ||
        cudaMalloc(&c->dsc, (size_t)nb * NSC * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->dcnt, nb * sizeof(int)) != cudaSuccess || cudaMalloc(&c->dactive, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->douter, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->hactive, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->hsc, (size_t)nb * NSC * sizeof(double)) != cudaSuccess)
      rc = FE_ERR_OOM;
  }
  if (rc == FE_OK) {
    memset(c->hsc, 0, (size_t)nb * NSC * sizeof(double));
    for (int b = 0; b < nb; ++b) {
      c->hbox[b].sc = c->dsc + (size_t)b * NSC;
      c->hbox[b].cnt = c->dcnt + b;
      double* s = c->hsc + (size_t)b * NSC;
      s[SC_TOL] = prm->p_tol;
      s[SC_OTOL] = prm->p_tol;
      s[SC_MAXIT] = prm->p_maxit;
      s[SC_DONE] = 1.0;
    }
    cudaMemcpyAsync(c->dsc, c->hsc, (size_t)nb * NSC * sizeof(double), cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(c->dcnt, 0, nb * sizeof(int), c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) rc = FE_ERR_CUDA;
  }
  if (rc == FE_OK && prm->solver == FE_FGMRES_LEARNED) {
    const long n = (long)c->hbox[0].N * c->hbox[0].N * c->hbox[0].N;
    const size_t esz = c->fp64 ? 8 : 4;
    c->gm_blocks = (int)std::min<long>((n + 255) / 256, 8L * c->nsm);
    const size_t parts = std::max<size_t>((size_t)c->gm_blocks * kGmPart, NSC);
    if (cudaMalloc(&c->gm_basis, (size_t)(2 * kGmRestart + 1) * n * esz) != cudaSuccess ||
        cudaMalloc(&c->gm_part, parts * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->gm_hpart, parts * sizeof(double)) != cudaSuccess)
      rc = FE_ERR_OOM;
  }
  if (rc == FE_OK) rc = set_tiling(c, 0);
  if (rc != FE_OK) {
    fe_destroy(c);
    return rc;
  }
  *out = c;
  return FE_OK;
}

extern "C" void fe_destroy(fe_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  for (void* s : c->slabs) cudaFree(s);
  for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
  drop_graphs(c);
  for (int q = 0; q < 3; ++q)
    if (c->cap[q]) cudaStreamDestroy(c->cap[q]);
  cudaFree(c->dloop);
  unet_destroy(c->unet);
  cudaFree(c->dbox);
  cudaFree(c->dwork);
  cudaFree(c->dework);
  cudaFree(c->dbwork);
  cudaFree(c->dpart);
  cudaFree(c->dsc);
  cudaFree(c->dcnt);
  cudaFree(c->dactive);
  cudaFree(c->douter);
  cudaFree(c->gm_basis);
  cudaFree(c->gm_part);
  cudaFree(c->les_work);
  cudaFree(c->iso_work);
  cudaFree(c->les_part);
  if (c->les_hpart) cudaFreeHost(c->les_hpart);
  if (c->gm_hpart) cudaFreeHost(c->gm_hpart);
  if (c->hactive) cudaFreeHost(c->hactive);
  if (c->hsc) cudaFreeHost(c->hsc);
  delete c;
}

extern "C" const char* fe_strerror(int code) {
  switch (code) {
    case FE_OK: return "ok";
    case FE_ERR_INVALID_ARG: return "invalid argument";
    case FE_ERR_CUDA: return "CUDA error";
    case FE_ERR_NOT_CONVERGED: return "pressure solve did not converge";
    case FE_ERR_NONFINITE: return "non-finite value in the new state";
    case FE_ERR_OOM: return "out of device memory";
    case FE_ERR_UNSUPPORTED: return "unsupported configuration";
    case FE_ERR_TOO_LARGE: return "grid larger than the fixed static buffer of the allocation-free entry point";
    default: return "unknown error";
  }
}

// ---- helpers ---------------------------------------------------------------------------------
static int field_slot(const fe_ctx* c, int field, int set) {
  if (field >= FE_RHO && field <= FE_UZ) return S(set, F_RHO + field);  // RHO, U0..2 line up
  if (field == FE_P) return S(set, F_P);
  if (field == FE_T) return c->prm.closure == FE_FOURIER ? S(set, F_T) : -1;
  if (field >= FE_PHIX && field <= FE_PHIZ) return S(set, F_PHI0 + (field - FE_PHIX));
  if (field >= FE_Y0 && field < FE_Y0 + c->prm.n_dust) return S(set, F_Y0 + (field - FE_Y0));
  if (c->prm.dust_model == FE_DUST_TWO_FLUID && field >= FE_V0 && field < FE_V0 + 3 * c->prm.n_dust)
    return S(set, F_V0 + (field - FE_V0));
  return -1;
}

static int pull_scalars(fe_ctx* c) {
  CK(cudaMemcpyAsync(c->hsc, c->dsc, (size_t)c->nb * NSC * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

static int push_scalar(fe_ctx* c, int box, int idx, double v) {
  c->hsc[(size_t)box * NSC + idx] = v;
  CK(cudaMemcpyAsync(c->dsc + (size_t)box * NSC + idx, c->hsc + (size_t)box * NSC + idx, sizeof(double),
                     cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

// Krylov driver for all boxes: operator/psi/dt already in place, rhs in K_B.
// y = a - y (harvested snapshot targets)
template <typename T>
__global__ void k_sub_from(const T* a, T* y, long n) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) y[q] = a[q] - y[q];
}

// The host reads the number of running solves only after `batch` iterations
// have been queued: the first batch is one less than the iteration count of
// the previous solve with the same key (boxes that finish early skip the
// surplus launches on the device), later batches are single iterations.
template <typename T>
static int krylov(fe_ctx* c, int maxit, int key) {
  Launch L = c->L();
  CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), c->st));
  const bool bicg = c->prm.solver == FE_BICGSTAB_JACOBI;
  if (bicg) launch_bicg_init<T>(L);
  else launch_cg_init<T>(L, 0.0);
  int it = 0;
  int batch = c->hint[key] > 1 ? c->hint[key] - 1 : 1;
  // harvesting: snapshots (r_k, x_k) of box 0 after iterations 2 and 5 of the first solve
  const bool snap = c->harvest_b && key <= 1;
  const bool fused = !bicg && !snap && c->hbox[0].f[K_PP] != nullptr;
  const int snap_at[2] = {2, 5};
  int nsnap = 0, snap_slot[2] = {-1, -1};
  if (snap) batch = 1;
  while (true) {
    if (it > 0 || batch == 1) {
      CK(cudaMemcpyAsync(c->hactive, c->dactive, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (*c->hactive == 0 || it >= maxit) break;
    }
    // snapshots only of a solve that is still running: the iterate at which the
    // solve stops is x* itself and would give the degenerate pair (r*, 0)
    if (snap && nsnap < 2 && it == snap_at[nsnap] && c->harvest_n < c->harvest_max) {
      const size_t bytes = (size_t)c->hbox[0].N * c->hbox[0].N * c->hbox[0].N * sizeof(T);
      CK(cudaMemcpyAsync(c->harvest_b[c->harvest_n], c->hbox[0].f[K_R], bytes, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(c->harvest_x[c->harvest_n], c->hbox[0].f[K_X], bytes, cudaMemcpyDeviceToDevice, c->st));
      snap_slot[nsnap++] = c->harvest_n++;
    }
    const int n = it == 0 ? batch : 1;
    for (int q = 0; q < n && it < maxit; ++q, ++it) {
      if (bicg) {
        launch_bicg_p<T>(L);
        launch_bicg_v<T>(L);
        launch_bicg_s<T>(L);
        launch_bicg_x<T>(L);
      } else if (fused) {
        launch_cg_fused<T>(L);
      } else {
        launch_cg_matvec<T>(L);
        launch_cg_update<T>(L);
        launch_cg_dir<T>(L);
      }
    }
  }
  if (fused) launch_cg_xfinal<T>(L);
  c->hint[key] = it;
  // snapshot targets: e_k = x* - x_k
  for (int q = 0; q < nsnap; ++q) {
    const long n = (long)c->hbox[0].N * c->hbox[0].N * c->hbox[0].N;
    k_sub_from<T><<<(int)std::min<long>((n + 255) / 256, 4096), 256, 0, c->st>>>(
        (const T*)c->hbox[0].f[K_X], (T*)c->harvest_x[snap_slot[q]], n);
  }
  CK(cudaGetLastError());
  return FE_OK;
}

// Flexible CG with the network direction (box 0; one network application per
// iteration).  The host polls convergence after every iteration: each one
// already costs a full network pass.  allow_net = false: Jacobi directions
// only (a later refinement solve of a corrector with learned_every = 0).
template <typename T>
static int fcg_learned(fe_ctx* c, int maxit, bool allow_net) {
  Launch L = c->L();
  BoxDev& B = c->hbox[0];
  CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), c->st));
  launch_cg_init<T>(L, 0.0);
  for (int it = 0; it < maxit; ++it) {
    CK(cudaMemcpyAsync(c->hactive, c->dactive, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (*c->hactive == 0) break;
    const int every = c->prm.learned_every;
    const bool net = allow_net && (every > 0 ? (it % every == 0) : (it == 0));
    if (net)
      FE_LAUNCH(L, KID_UNET,
                (unet_apply_sc<T>(c->unet, (const T*)B.f[K_R], (const T*)B.f[W_DINV], B.sc,
                                  it == 0 ? SC_BB : SC_RR, B.ih, c->st)));
    launch_fcg<T>(L, net ? unet_output(c->unet) : nullptr);
  }
  CK(cudaGetLastError());
  return FE_OK;
}

// Block partial sums of the FGMRES kernels, added on the host in block order.
static int gm_sums(fe_ctx* c, int stride, double* out) {
  const size_t cnt = (size_t)c->gm_blocks * stride;
  CK(cudaMemcpyAsync(c->gm_hpart, c->gm_part, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i < stride; ++i) out[i] = 0.0;
  for (int bl = 0; bl < c->gm_blocks; ++bl)
    for (int i = 0; i < stride; ++i) out[i] += c->gm_hpart[(size_t)bl * stride + i];
  return FE_OK;
}

// Flexible GMRES(m) (Saad 1993) on box 0, any operator: right
// preconditioning with the network direction (learned_every as for flexible
// CG) or the Jacobi one (no network loaded, or a network output that is not
// finite or is zero), Arnoldi by classical Gram-Schmidt with one
// reorthogonalisation, Givens rotations and the least-squares update in FP64
// on the host, restart after kGmRestart directions from the true residual.
// Stops when the least-squares residual meets SC_TOL ||b|| or at the
// iteration cap; x0 = 0 (the refinement's correction starts from zero).
template <typename T>
static int fgmres_learned(fe_ctx* c, int maxit, bool allow_net) {
  Launch L = c->L();
  BoxDev& B = c->hbox[0];
  cudaStream_t st = c->st;
  const long n = (long)B.N * B.N * B.N;
  const int m = kGmRestart, nb = c->gm_blocks;
  CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), st));
  launch_cg_init<T>(L, 0.0);  // x = 0, r = b, ||b||^2, the solve's scalars and counter
  double* hs = c->gm_hpart;
  CK(cudaMemcpyAsync(hs, B.sc, NSC * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hs[SC_DONE] != 0.0) return FE_OK;  // zero right-hand side, or the refinement has converged
  const double bnorm = std::sqrt(hs[SC_BB]), tol = hs[SC_TOL];
  const int cap = std::min(maxit, (int)hs[SC_MAXIT]);
  T* V = (T*)c->gm_basis;
  T* Z = V + (size_t)(m + 1) * n;
  const T* b = (const T*)B.f[K_B];
  T* r = (T*)B.f[K_R];
  T* x = (T*)B.f[K_X];
  T* pd = (T*)B.f[K_PD];
  const T* q = (const T*)B.f[K_Q];
  const T* dinv = (const T*)B.f[W_DINV];
  const T* psi = (const T*)B.f[W_PSI];
  const int every = c->prm.learned_every;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  double d[kGmPart], e[kGmPart];
  GmCoef co{};
  int it = 0, rc = FE_OK;
  double res = bnorm;
  bool conv = false;
  while (true) {
    gm_dots<T>(V, n, 0, r, c->gm_part, nb, st);  // ||r||^2
    if ((rc = gm_sums(c, kGmPart, d)) != FE_OK) return rc;
    const double beta = std::sqrt(d[kGmMax + 1]);
    if (!(beta > tol * bnorm)) {  // the restart's true residual already meets the tolerance
      res = beta;
      conv = true;
      break;
    }
    gm_combine<T>(V, r, 1.0 / beta, nullptr, n, 0, co, nb, st);  // v_0 = r / beta
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      T* vj = V + (size_t)j * n;
      T* vn = V + (size_t)(j + 1) * n;
      // Arnoldi column of the direction in pd: q = M z, w = q - V h twice
      // (classical Gram-Schmidt with one reorthogonalisation) into vn,
      // col[j + 1] = ||w||, col[0..j] = h after the previous rotations
      double col[kGmMax + 2], qn = 0.0;
      auto column = [&]() -> int {
        launch_cg_matvec<T>(L);
        gm_dots<T>(V, n, j + 1, q, c->gm_part, nb, st);
        int e1 = gm_sums(c, kGmPart, d);
        if (e1 != FE_OK) return e1;
        qn = std::sqrt(d[kGmMax + 1]);
        for (int i = 0; i <= j; ++i) co.h[i] = -d[i];
        gm_combine<T>(vn, q, 1.0, V, n, j + 1, co, nb, st);
        gm_dots<T>(V, n, j + 1, vn, c->gm_part, nb, st);
        if ((e1 = gm_sums(c, kGmPart, e)) != FE_OK) return e1;
        for (int i = 0; i <= j; ++i) {
          co.h[i] = -e[i];
          col[i] = d[i] + e[i];
        }
        gm_combine<T>(vn, vn, 1.0, V, n, j + 1, co, nb, st);
        gm_dots<T>(V, n, 0, vn, c->gm_part, nb, st);
        if ((e1 = gm_sums(c, kGmPart, d)) != FE_OK) return e1;
        col[j + 1] = std::sqrt(d[kGmMax + 1]);
        for (int i = 0; i < j; ++i) {
          const double a0 = col[i], a1 = col[i + 1];
          col[i] = cs[i] * a0 + sn[i] * a1;
          col[i + 1] = -sn[i] * a0 + cs[i] * a1;
        }
        return FE_OK;
      };
      // the network's direction for v_j, kept if finite and non-zero, if its
      // image is not (to kGmNetFresh of its norm) in the span of the basis (a
      // singular Hessenberg matrix would fake convergence), and if it shrinks
      // the least-squares residual to at most kGmNetKeep of its value;
      // otherwise (or without a network) the Jacobi direction
      bool have = false;
      if (allow_net && c->unet_ready && (every > 0 ? it % every == 0 : it == 0)) {
        gm_set_scalar(B.sc, SC_PR, 1.0, st);  // ||v_j||^2 = 1: the input scale of the unit vector v_j
        FE_LAUNCH(L, KID_UNET, (unet_apply_sc<T>(c->unet, vj, dinv, B.sc, SC_PR, B.ih, st)));
        gm_from_net<T>(pd, vj, dinv, unet_output(c->unet), B.sc, n, c->gm_part, nb, st);
        double zz = 0.0;
        if ((rc = gm_sums(c, 1, &zz)) != FE_OK) return rc;
        if (std::isfinite(zz) && zz > 0.0) {
          if ((rc = column()) != FE_OK) return rc;
          const double hyp = std::hypot(col[j], col[j + 1]);
          have = std::isfinite(hyp) && hyp > kGmNetFresh * qn && std::fabs(col[j + 1] / hyp) <= kGmNetKeep;
        }
      }
      if (!have) {
        gm_jacobi<T>(pd, vj, dinv, n, nb, st);
        if ((rc = column()) != FE_OK) return rc;
      }
      CK(cudaMemcpyAsync(Z + (size_t)j * n, pd, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
      const double hn = col[j + 1];
      if (hn > 0.0) gm_combine<T>(vn, vn, 1.0 / hn, nullptr, n, 0, co, nb, st);
      for (int i = 0; i <= j + 1; ++i) Hij(i, j) = col[i];
      // the rotation that zeroes H(j+1, j)
      const double a0 = Hij(j, j), a1 = Hij(j + 1, j), hyp = std::hypot(a0, a1);
      cs[j] = a1 == 0.0 ? 1.0 : a0 / hyp;
      sn[j] = a1 == 0.0 ? 0.0 : a1 / hyp;
      Hij(j, j) = cs[j] * a0 + sn[j] * a1;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      k = j + 1;
      res = std::fabs(g[j + 1]);
      if (res <= tol * bnorm) {
        conv = true;
        stop = true;
        break;
      }
      if (it >= cap || !(hn > 0.0)) {
        stop = true;
        break;
      }
    }
    // y from the rotated upper triangle; x += Z y
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
      y[i] = Hij(i, i) != 0.0 ? t / Hij(i, i) : 0.0;
    }
    for (int i = 0; i < k; ++i) co.h[i] = y[i];
    gm_combine<T>(x, x, 1.0, Z, n, k, co, nb, st);
    if (stop) break;
    // restart from the true residual r = b - M x
    CK(cudaMemcpyAsync(pd, x, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    launch_cg_matvec<T>(L);
    co.h[0] = -1.0;
    gm_combine<T>(r, b, 1.0, q, n, 1, co, nb, st);
  }
  gm_finish(B.sc, c->dactive, (double)it, res * res, conv ? 1 : 0, st);
  CK(cudaGetLastError());
  return FE_OK;
}

// outer: index of the refinement solve within the corrector (0 in FP64).  With
// learned_every = 0 the network gives only the first direction of the
// corrector's first solve: once per corrector, not once per refinement step.
template <typename T>
static int inner_solve(fe_ctx* c, int maxit, int key, int outer = 0) {
  const bool allow_net = c->prm.learned_every != 0 || outer == 0;
  if (c->prm.solver == FE_FCG_LEARNED) {
    if (!c->unet_ready) return FE_ERR_UNSUPPORTED;
    return fcg_learned<T>(c, maxit, allow_net);
  }
  if (c->prm.solver == FE_FGMRES_LEARNED) return fgmres_learned<T>(c, maxit, allow_net);
  return krylov<T>(c, maxit, key);
}

// Pressure solve of every box with the right-hand side in K_B: one Krylov
// solve in FP64 mode; in mixed mode FP64 iterative refinement (residual
// b - M x64 in FP64, inner solves in FP32, x64 += x) until the FP64 residual
// meets the tolerance, then x = (float) x64.
// Mixed precision with the fused plain-CG iteration: the refinement boundary
// (last direction, pair accumulation, double-float residual, next start) is
// one kernel.
static bool fused_refine(const fe_ctx* c) {
  return !c->fp64 && (c->prm.solver == FE_PCG_JACOBI || c->prm.solver == FE_PCG_POLY) && !c->prm.transonic &&
         !c->harvest_b &&
         c->hbox[0].f[K_PP] != nullptr && c->hbox[0].f[K_X64B] != nullptr;
}

// Fused CG iterations of an already started solve (host-driven, batched as in krylov()).
template <typename T>
static int cg_iterate(fe_ctx* c, int maxit, int key) {
  Launch L = c->L();
  int it = 0;
  const int batch = c->hint[key] > 1 ? c->hint[key] - 1 : 1;
  while (true) {
    if (it > 0 || batch == 1) {
      CK(cudaMemcpyAsync(c->hactive, c->dactive, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (*c->hactive == 0 || it >= maxit) break;
    }
    const int n = it == 0 ? batch : 1;
    for (int q = 0; q < n && it < maxit; ++q, ++it) launch_cg_fused<T>(L);
  }
  c->hint[key] = it;
  return FE_OK;
}

// started: the right-hand-side kernel of the step already started the refined
// solve (K_AUX, K_R and the scalars); otherwise start it from K_B here.
template <typename T>
static int refine_solve(fe_ctx* c, bool started) {
  Launch L = c->L();
  if (!started) {
    CK(cudaMemsetAsync(c->douter, 0, sizeof(int), c->st));
    CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), c->st));
    launch_refine_start<T>(L, c->douter);
  }
  for (int outer = 0; outer < 8; ++outer) {
    CK(cudaMemcpyAsync(c->hactive, c->douter, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (*c->hactive == 0) break;
    int rc = cg_iterate<T>(c, c->prm.p_maxit, 1 + outer);
    if (rc != FE_OK) return rc;
    CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), c->st));
    launch_refine<T>(L, c->douter);
  }
  launch_mix_finish_pp<T>(L);
  CK(cudaGetLastError());
  return FE_OK;
}

template <typename T>
static int pressure_solve(fe_ctx* c, bool started = false) {
  if (c->fp64) return inner_solve<T>(c, c->prm.p_maxit, 0);
  if (fused_refine(c)) return refine_solve<T>(c, started);
  Launch L = c->L();
  CK(cudaMemsetAsync(c->douter, 0, sizeof(int), c->st));
  launch_mix_residual<T>(L, 1, c->douter);
  for (int outer = 0; outer < 8; ++outer) {
    CK(cudaMemcpyAsync(c->hactive, c->douter, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (*c->hactive == 0) break;
    int rc = inner_solve<T>(c, c->prm.p_maxit, 1 + outer, outer);
    if (rc != FE_OK) return rc;
    launch_mix_accum<T>(L);
    launch_mix_residual<T>(L, 0, c->douter);
  }
  launch_mix_finish<T>(L);
  CK(cudaGetLastError());
  return FE_OK;
}

__global__ void k_commit(double* sc, int nb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double* s = sc + (size_t)b * NSC;
  s[SC_TIME] += s[SC_DT];
  s[SC_DTPREV] = s[SC_DT];
}

// ---- CUDA-graph form of the pressure solves --------------------------------------------------
// A Krylov loop becomes a conditional WHILE node whose body ends with a
// one-thread kernel that keeps the loop alive while some box is still
// iterating and an iteration counter is below its cap, so the graph always
// terminates on its own.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* active, int* counter, int cap) {
  const int n = ++(*counter);
  cudaGraphSetConditional(h, (*active > 0 && n < cap) ? 1u : 0u);
}

__global__ void k_cond_set(cudaGraphConditionalHandle h, unsigned v) { cudaGraphSetConditional(h, v); }

// Open a WHILE node at the capture point of `cs`; its body is captured on `bs`.
// The condition is set to 1 right before the node (a handle's default value
// applies only at graph launch, which would skip a nested loop's later passes).
static int while_begin(cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus stt;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, &deps, nullptr, &nd));
  CK(cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault));
  k_cond_set<<<1, 1, 0, cs>>>(*h, 1u);
  CK(cudaGetLastError());
  CK(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = *h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamBeginCaptureToGraph(bs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  return FE_OK;
}

static int while_end(cudaStream_t bs) {
  cudaGraph_t body;
  CK(cudaStreamEndCapture(bs, &body));
  return FE_OK;
}

// Krylov solve of every box captured on stream level `lev` (loop body on lev + 1).
template <typename T>
static int krylov_graph(fe_ctx* c, int lev) {
  cudaStream_t cs = c->cap[lev], bs = c->cap[lev + 1];
  Launch L = c->L();
  L.st = cs;
  const int maxit = c->prm.p_maxit;
  CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), cs));
  const bool bicg = c->prm.solver == FE_BICGSTAB_JACOBI;
  const bool learned = c->prm.solver == FE_FCG_LEARNED;
  BoxDev& B0 = c->hbox[0];
  if (bicg) launch_bicg_init<T>(L);
  else launch_cg_init<T>(L, 0.0);
  if (learned) {  // first iteration with the network direction
    unet_apply_sc<T>(c->unet, (const T*)B0.f[K_R], (const T*)B0.f[W_DINV], B0.sc, SC_BB, B0.ih, cs);
    launch_fcg<T>(L, unet_output(c->unet));
  }
  CK(cudaMemsetAsync(c->dloop + lev, 0, sizeof(int), cs));
  cudaGraphConditionalHandle h;
  int rc = while_begin(cs, bs, &h);
  if (rc != FE_OK) return rc;
  Launch Lb = L;
  Lb.st = bs;
  if (bicg) {
    launch_bicg_p<T>(Lb);
    launch_bicg_v<T>(Lb);
    launch_bicg_s<T>(Lb);
    launch_bicg_x<T>(Lb);
  } else if (learned) {
    if (c->prm.learned_every == 1)
      unet_apply_sc<T>(c->unet, (const T*)B0.f[K_R], (const T*)B0.f[W_DINV], B0.sc, SC_RR, B0.ih, bs);
    launch_fcg<T>(Lb, c->prm.learned_every == 1 ? unet_output(c->unet) : nullptr);
  } else {
    launch_cg_fused<T>(Lb);
  }
  k_loop_cond<<<1, 1, 0, bs>>>(h, c->dactive, c->dloop + lev, maxit + 1);
  rc = while_end(bs);
  if (rc == FE_OK && !bicg && !learned) launch_cg_xfinal<T>(L);
  return rc;
}

// Pressure solve captured on stream level 0 (mixed precision adds the
// refinement loop as an outer WHILE node).
template <typename T>
static int pressure_graph(fe_ctx* c) {
  if (c->fp64) return krylov_graph<T>(c, 0);
  cudaStream_t cs = c->cap[0], bs = c->cap[1];
  Launch L = c->L();
  L.st = cs;
  if (fused_refine(c)) {  // the right-hand-side kernel started the refined solve
    CK(cudaMemsetAsync(c->dloop + 3, 0, sizeof(int), cs));
    cudaGraphConditionalHandle ho, hi;
    int rc = while_begin(cs, bs, &ho);  // refinement steps
    if (rc != FE_OK) return rc;
    cudaStream_t is = c->cap[2];
    CK(cudaMemsetAsync(c->dloop + 1, 0, sizeof(int), bs));
    rc = while_begin(bs, is, &hi);  // fused CG iterations of one inner solve
    if (rc != FE_OK) return rc;
    Launch Li = L;
    Li.st = is;
    launch_cg_fused<T>(Li);
    k_loop_cond<<<1, 1, 0, is>>>(hi, c->dactive, c->dloop + 1, c->prm.p_maxit + 1);
    rc = while_end(is);
    if (rc != FE_OK) return rc;
    Launch Lb = L;
    Lb.st = bs;
    CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), bs));
    launch_refine<T>(Lb, c->douter);
    k_loop_cond<<<1, 1, 0, bs>>>(ho, c->douter, c->dloop + 3, 8);
    rc = while_end(bs);
    if (rc != FE_OK) return rc;
    launch_mix_finish_pp<T>(L);
    return FE_OK;
  }
  CK(cudaMemsetAsync(c->douter, 0, sizeof(int), cs));
  launch_mix_residual<T>(L, 1, c->douter);
  CK(cudaMemsetAsync(c->dloop + 3, 0, sizeof(int), cs));
  cudaGraphConditionalHandle h;
  int rc = while_begin(cs, bs, &h);
  if (rc != FE_OK) return rc;
  rc = krylov_graph<T>(c, 1);
  if (rc != FE_OK) return rc;
  Launch Lb = L;
  Lb.st = bs;
  launch_mix_accum<T>(Lb);
  launch_mix_residual<T>(Lb, 0, c->douter);
  k_loop_cond<<<1, 1, 0, bs>>>(h, c->douter, c->dloop + 3, 8);
  rc = while_end(bs);
  if (rc != FE_OK) return rc;
  launch_mix_finish<T>(L);
  return FE_OK;
}

// The kernel sequence of one PISO step (state set s -> 1 - s).  graph = true:
// issued into the capture on stream level 0 with the solves as WHILE nodes.
template <typename T>
static int issue_step(fe_ctx* c, int s, bool graph) {
  Launch L = c->L();
  if (graph) L.st = c->cap[0];
  const int ks = 1 - s, nc = c->prm.n_corr;
  if (c->prm.coupling == FE_COUPLING_TWO_WAY && c->prm.n_dust > 0) {  // the loading sum_j Y_j^n of the step
    L.ysum = c->prm.n_dust == 1 ? S(s, F_Y0) : W_YSUM;
    if (c->prm.n_dust > 1) launch_ysum<T>(L, s);
  }
  launch_dt_div<T>(L, s);
  launch_pred<T>(L, s, ks);
  launch_fluxn<T>(L, s);
  for (int kk = 0; kk < nc; ++kk) {
    const int rhop = S(ks, F_RHO);
    const int up0 = S(ks, F_U0);
    const int php0 = kk == 0 ? S(s, F_PHI0) : S(ks, F_PHI0);
    const int pp = kk == 0 ? S(s, F_P) : W_PW0 + ((kk - 1) & 1);
    const int pn = W_PW0 + (kk & 1);
    if (kk == 0) launch_div<T>(L, up0);
    launch_asm<T>(L, s, up0, php0, rhop);
    if (fused_refine(c)) {  // b, the first inner right-hand side and the solve's start in one pass
      CK(cudaMemsetAsync(c->douter, 0, sizeof(int), L.st));
      CK(cudaMemsetAsync(c->dactive, 0, sizeof(int), L.st));
      Launch Lr = L;
      Lr.rstart = c->douter;
      launch_rhs<T>(Lr, s, rhop, pp);
      launch_cg_start<T>(L);
    } else {
      launch_rhs<T>(L, s, rhop, pp);
    }
    int rc = graph ? pressure_graph<T>(c) : pressure_solve<T>(c, true);
    if (rc != FE_OK) return rc;
    if (!graph && c->harvest_b && c->harvest_n < c->harvest_max) {
      const size_t bytes = (size_t)c->hbox[0].N * c->hbox[0].N * c->hbox[0].N * sizeof(T);
      CK(cudaMemcpyAsync(c->harvest_b[c->harvest_n], c->hbox[0].f[c->fp64 ? K_B : K_AUX], bytes,
                         cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(c->harvest_x[c->harvest_n], c->hbox[0].f[K_X], bytes, cudaMemcpyDeviceToDevice, c->st));
      c->harvest_n++;
    }
    launch_corr<T>(L, s, rhop, pp, pn, ks, kk, c->fp64 ? 0 : (fused_refine(c) ? 2 : 1));
    launch_div<T>(L, S(ks, F_U0));
    launch_accel<T>(L, ks, pn);
    const bool last = kk == nc - 1;
    const int yp0 = kk == 0 ? S(s, F_Y0) : W_YW0 + ((kk - 1) & 1) * MAXD;
    const int yn0 = last ? S(ks, F_Y0) : W_YW0 + (kk & 1) * MAXD;
    const int ep = kk == 0 ? -1 : W_EW0 + ((kk - 1) & 1);
    const int en = last ? -1 : W_EW0 + (kk & 1);
    launch_dust<T>(L, s, ks, pn, yp0, yn0, ep, en, last ? 1 : 0, kk == 0 ? 1 : 0);
  }
  // two-fluid dust: its own transport and drag after the gas step (it overwrites the
  // classes' Y of the new level and their totals)
  if (c->prm.dust_model == FE_DUST_TWO_FLUID && c->prm.n_dust > 0) launch_two_fluid<T>(L, s, ks);
  CK(cudaGetLastError());
  return FE_OK;
}

static void drop_graphs(fe_ctx* c) {
  for (int q = 0; q < 2; ++q)
    if (c->gexec[q]) {
      cudaGraphExecDestroy(c->gexec[q]);
      c->gexec[q] = nullptr;
    }
}

template <typename T>
static int build_graph(fe_ctx* c, int s) {
  for (int q = 0; q < 3; ++q)
    if (!c->cap[q]) CK(cudaStreamCreateWithFlags(&c->cap[q], cudaStreamNonBlocking));
  if (!c->dloop) CK(cudaMalloc(&c->dloop, 8 * sizeof(int)));
  CK(cudaStreamBeginCapture(c->cap[0], cudaStreamCaptureModeRelaxed));
  int rc = issue_step<T>(c, s, true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap[0], &g);
  if (rc != FE_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != FE_OK ? rc : FE_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&c->gexec[s], g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

static bool graph_ok(const fe_ctx* c) {
  if (!c->use_graphs || c->harvest_b || c->prof.on) return false;
  if (c->prm.solver == FE_FCG_LEARNED && (!c->unet_ready || c->prm.learned_every > 1)) return false;
  // mixed precision, network once per corrector: host-driven (the refinement
  // loop's later solves skip the network, which the graph's loop body cannot)
  if (c->prm.solver == FE_FCG_LEARNED && !c->fp64 && c->prm.learned_every == 0) return false;
  if (c->prm.solver == FE_FGMRES_LEARNED) return false;  // host-driven: the Arnoldi step reads its dots
  return true;
}

// One PISO step of every box.  commit = false runs a trial step (autotuning):
// the new state is computed into the other state set but not adopted.
template <typename T>
static int step_once(fe_ctx* c, bool commit = true) {
  const int s = c->cur, ks = 1 - s, nc = c->prm.n_corr;
  if (graph_ok(c)) {
    if (!c->gexec[s]) {
      int rc = build_graph<T>(c, s);
      if (rc != FE_OK) return rc;
    }
    CK(cudaGraphLaunch(c->gexec[s], c->st));
  } else {
    int rc = issue_step<T>(c, s, false);
    if (rc != FE_OK) return rc;
  }
  if (!commit) return FE_OK;
  int rc = pull_scalars(c);
  if (rc != FE_OK) return rc;
  for (int b = 0; b < c->nb; ++b) {
    const double* sc = c->hsc + (size_t)b * NSC;
    if (sc[SC_KERR] != 0.0) return FE_ERR_CUDA;
    if (sc[SC_BAD] > 0.0 || !std::isfinite(sc[SC_DT])) return FE_ERR_NONFINITE;
    for (int kk = 0; kk < nc; ++kk)
      if (!(sc[SC_RES0 + kk] <= c->prm.p_tol * (1.0 + 1e-3))) return FE_ERR_NOT_CONVERGED;
  }
  {
    Launch L2 = c->L();
    FE_LAUNCH(L2, KID_COMMIT, (k_commit<<<(c->nb + 127) / 128, 128, 0, c->st>>>(c->dsc, c->nb)));
  }
  CK(cudaGetLastError());
  c->cur = ks;
  return FE_OK;
}

extern "C" int fe_step(fe_ctx* c, int nsteps, fe_step_info* info) {
  if (!c || nsteps < 0) return FE_ERR_INVALID_ARG;
  for (int n = 0; n < nsteps; ++n) {
    int rc = c->fp64 ? step_once<double>(c) : step_once<float>(c);
    if (rc != FE_OK) return rc;
  }
  if (info) {
    int rc = pull_scalars(c);
    if (rc != FE_OK) return rc;
    for (int b = 0; b < c->nb; ++b) {
      const double* sc = c->hsc + (size_t)b * NSC;
      info[b].t = sc[SC_TIME];
      info[b].dt = sc[SC_DTPREV];
      for (int k = 0; k < 4; ++k) {
        info[b].iters[k] = k < c->prm.n_corr ? (int)sc[SC_IT0 + k] : 0;
        info[b].rel_res[k] = k < c->prm.n_corr ? sc[SC_RES0 + k] : 0.0;
      }
    }
  }
  return FE_OK;
}

extern "C" int fe_set_field(fe_ctx* c, int box, int field, const void* src, int is_dev) {
  if (!c || !src || box < 0 || box >= c->nb) return FE_ERR_INVALID_ARG;
  int slot = field_slot(c, field, c->cur);
  if (slot < 0) return FE_ERR_INVALID_ARG;
  const int N = c->N[box];
  size_t bytes = (size_t)N * N * N * (c->fp64 ? 8 : 4);
  CK(cudaMemcpyAsync(c->hbox[box].f[slot], src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

extern "C" int fe_get_field(fe_ctx* c, int box, int field, void* dst, int is_dev) {
  if (!c || !dst || box < 0 || box >= c->nb) return FE_ERR_INVALID_ARG;
  int slot = field_slot(c, field, c->cur);
  if (slot < 0) return FE_ERR_INVALID_ARG;
  const int N = c->N[box];
  size_t bytes = (size_t)N * N * N * (c->fp64 ? 8 : 4);
  CK(cudaMemcpyAsync(dst, c->hbox[box].f[slot], bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

// Several fields in one call: every copy queued on the context stream, one
// synchronisation at the end (all arguments are checked before any copy).  Measured on the GB300
// box: about 200 GB/s each way from page-locked memory whether the copies run on one stream, on
// four streams, or as a kernel that loads the host memory directly: the host link is the limit.
static int copy_fields(fe_ctx* c, int box, int n, const int* fields, void* const* ptrs, int is_dev, bool in) {
  if (!c || box < 0 || box >= c->nb || n < 0 || (n > 0 && (!fields || !ptrs))) return FE_ERR_INVALID_ARG;
  for (int q = 0; q < n; ++q)
    if (!ptrs[q] || field_slot(c, fields[q], c->cur) < 0) return FE_ERR_INVALID_ARG;
  const int N = c->N[box];
  const size_t bytes = (size_t)N * N * N * (c->fp64 ? 8 : 4);
  for (int q = 0; q < n; ++q) {
    void* dev = c->hbox[box].f[field_slot(c, fields[q], c->cur)];
    if (in)
      CK(cudaMemcpyAsync(dev, ptrs[q], bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
    else
      CK(cudaMemcpyAsync(ptrs[q], dev, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

extern "C" int fe_set_fields(fe_ctx* c, int box, int n, const int* fields, const void* const* src, int is_dev) {
  return copy_fields(c, box, n, fields, const_cast<void* const*>(src), is_dev, true);
}

extern "C" int fe_get_fields(fe_ctx* c, int box, int n, const int* fields, void* const* dst, int is_dev) {
  return copy_fields(c, box, n, fields, dst, is_dev, false);
}

extern "C" int fe_set_clock(fe_ctx* c, int box, double t, double dt_prev) {
  if (!c || box < 0 || box >= c->nb) return FE_ERR_INVALID_ARG;
  int rc = push_scalar(c, box, SC_TIME, t);
  if (rc != FE_OK) return rc;
  return push_scalar(c, box, SC_DTPREV, dt_prev > 0.0 ? dt_prev : 0.0);
}

template <typename T>
static int init_box(fe_ctx* c, int b, int mode) {
  BoxDev& B = c->hbox[b];
  const int s = c->cur;
  const long n = (long)B.N * B.N * B.N;
  if (mode == FE_INIT_SPECTRAL) {
    if (!fft_supported(B.N)) return FE_ERR_UNSUPPORTED;
    int rc = ic_spectral<T>((T*)B.f[S(s, F_U0)], (T*)B.f[S(s, F_U1)], (T*)B.f[S(s, F_U2)], B.N, c->seed[b], c->k0[b],
                            c->mach[b], c->st);
    if (rc != FE_OK) return rc;
    fill<T>((T*)B.f[S(s, F_RHO)], n, 1.0, c->st);
    if (c->prm.closure == FE_FOURIER) fill<T>((T*)B.f[S(s, F_T)], n, 1.0, c->st);
    for (int j = 0; j < B.nd; ++j) fill<T>((T*)B.f[S(s, F_Y0 + j)], n, c->Y0[(size_t)b * B.nd + j], c->st);
  }
  launch_derive_box<T>(c->L(), s, b);
  if (c->prm.dust_model == FE_DUST_TWO_FLUID && B.nd > 0) launch_two_fluid_init<T>(c->L(), s, b);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  int rc = push_scalar(c, b, SC_TIME, 0.0);
  if (rc != FE_OK) return rc;
  return push_scalar(c, b, SC_DTPREV, 0.0);
}

extern "C" int fe_init_state(fe_ctx* c, int box, int mode) {
  if (!c || box < -1 || box >= c->nb || (mode != FE_INIT_SPECTRAL && mode != FE_INIT_DERIVE))
    return FE_ERR_INVALID_ARG;
  for (int b = (box < 0 ? 0 : box); b < (box < 0 ? c->nb : box + 1); ++b) {
    int rc = c->fp64 ? init_box<double>(c, b, mode) : init_box<float>(c, b, mode);
    if (rc != FE_OK) return rc;
  }
  return FE_OK;
}

template <typename T>
__global__ void k_psi_box(const BoxDev* boxes, int box, int s, double dt) {
  const BoxDev& B = boxes[box];
  T* dinv = (T*)B.f[W_DINV];
  const JacobiDiag<T> jd(dt, B.ih);
  const long n = (long)B.N * B.N * B.N;
  const T* rho = (const T*)B.f[S(s, F_RHO)];
  const T* p = (const T*)B.f[S(s, F_P)];
  T* psi = (T*)B.f[W_PSI];
  T* hb[3] = {(T*)B.f[W_HB0], (T*)B.f[W_HB1], (T*)B.f[W_HB2]};
  const T* u[3] = {(const T*)B.f[S(s, F_U0)], (const T*)B.f[S(s, F_U1)], (const T*)B.f[S(s, F_U2)]};
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    T ps = rho[q] / ((T)B.gamma * p[q]);
    psi[q] = ps;
    dinv[q] = jd.inv(ps);
    for (int d = 0; d < 3; ++d) hb[d][q] = u[d][q];
  }
}

template <typename T>
static int solve_box(fe_ctx* c, int box, const void* b, void* x, double dt, double tol, int maxit,
                     fe_solve_info* info) {
  BoxDev& B = c->hbox[box];
  const size_t bytes = (size_t)B.N * B.N * B.N * sizeof(T);
  // other boxes stay idle: mark them done for this solve
  int rc = pull_scalars(c);
  if (rc != FE_OK) return rc;
  std::vector<double> saved((size_t)c->nb * NSC);
  memcpy(saved.data(), c->hsc, saved.size() * sizeof(double));
  k_psi_box<T><<<1024, 256, 0, c->st>>>(c->dbox, box, c->cur, dt);
  CK(cudaMemcpyAsync(B.f[K_B], b, bytes, cudaMemcpyDeviceToDevice, c->st));
  for (int q = 0; q < c->nb; ++q) {
    double* s = c->hsc + (size_t)q * NSC;
    s[SC_KDT] = dt;
    s[SC_TOL] = tol;
    s[SC_OTOL] = tol;
    s[SC_MAXIT] = maxit;
  }
  CK(cudaMemcpyAsync(c->dsc, c->hsc, (size_t)c->nb * NSC * sizeof(double), cudaMemcpyHostToDevice, c->st));
  // zero rhs of the other boxes so their solves end at once
  for (int q = 0; q < c->nb; ++q)
    if (q != box) CK(cudaMemsetAsync(c->hbox[q].f[K_B], 0, (size_t)c->N[q] * c->N[q] * c->N[q] * sizeof(T), c->st));
  const int save_maxit = c->prm.p_maxit;
  c->prm.p_maxit = maxit;
  rc = pressure_solve<T>(c);
  c->prm.p_maxit = save_maxit;
  if (rc != FE_OK) return rc;
  if (c->fp64) launch_true_res<T>(c->L(), K_X);
  CK(cudaMemcpyAsync(x, B.f[fused_refine(c) ? K_XH : K_X], bytes, cudaMemcpyDeviceToDevice, c->st));
  rc = pull_scalars(c);
  if (rc != FE_OK) return rc;
  const double* s = c->hsc + (size_t)box * NSC;
  fe_solve_info inf;
  if (c->fp64) {
    inf.iters = (int)s[SC_ITERS];
    inf.rel_res_true = s[SC_BB] > 0 ? sqrt(s[SC_TRUE_RR] / s[SC_BB]) : 0.0;
  } else {
    inf.iters = (int)s[SC_ITSUM];
    inf.rel_res_true = s[SC_ORES];
  }
  bool conv = s[SC_CONV] != 0.0;
  if (info) *info = inf;
  // restore the step scalars (tolerance, cap, dt) of every box
  memcpy(c->hsc, saved.data(), saved.size() * sizeof(double));
  CK(cudaMemcpyAsync(c->dsc, c->hsc, (size_t)c->nb * NSC * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return conv ? FE_OK : FE_ERR_NOT_CONVERGED;
}

extern "C" int fe_solve_pressure(fe_ctx* c, int box, const void* b, void* x, double dt, double tol, int maxit,
                                 fe_solve_info* info) {
  if (!c || !b || !x || box < 0 || box >= c->nb || !(dt > 0.0) || !(tol > 0.0) || maxit < 1)
    return FE_ERR_INVALID_ARG;
  return c->fp64 ? solve_box<double>(c, box, b, x, dt, tol, maxit, info)
                 : solve_box<float>(c, box, b, x, dt, tol, maxit, info);
}

template <typename T>
static int diag_box(fe_ctx* c, int box, fe_diag* out, double* spec, int nbins) {
  BoxDev& B = c->hbox[box];
  double sums[7 + MAXD];
  int rc = diag_sums<T>(c->L(), B, box, c->cur, sums);
  if (rc != FE_OK) return rc;
  const double n = (double)B.N * B.N * B.N, vol = B.h * B.h * B.h;
  memset(out, 0, sizeof(*out));
  out->ke = 0.5 * sums[0] / n;
  out->ke_u = 0.5 * sums[1] / n;
  out->enstrophy = 0.5 * sums[2] / n;
  out->taylor = sums[3] > 0 ? sqrt(sums[1] / sums[3]) : 0.0;
  out->rho_rms = sqrt(sums[5] / n);
  out->mass = vol * sums[4];
  out->energy = vol * sums[6];
  for (int j = 0; j < B.nd; ++j) out->dust_mass[j] = vol * sums[7 + j];
  rc = pull_scalars(c);
  if (rc != FE_OK) return rc;
  out->t = c->hsc[(size_t)box * NSC + SC_TIME];
  out->dt_prev = c->hsc[(size_t)box * NSC + SC_DTPREV];
  if (spec && nbins > 0) {
    if (!fft_supported(B.N)) return FE_ERR_UNSUPPORTED;
    const int s = c->cur;
    rc = spectrum<T>((const T*)B.f[S(s, F_U0)], (const T*)B.f[S(s, F_U1)], (const T*)B.f[S(s, F_U2)], B.N, spec, nbins,
                     c->st);
    if (rc != FE_OK) return rc;
  }
  return FE_OK;
}

extern "C" int fe_diagnostics(fe_ctx* c, int box, fe_diag* out, double* spectrum_host, int nbins) {
  if (!c || !out || box < 0 || box >= c->nb || nbins < 0 || (nbins > 0 && !spectrum_host)) return FE_ERR_INVALID_ARG;
  return c->fp64 ? diag_box<double>(c, box, out, spectrum_host, nbins)
                 : diag_box<float>(c, box, out, spectrum_host, nbins);
}

extern "C" int fe_q_criterion(fe_ctx* c, int box, void* q) {
  if (!c || !q || box < 0 || box >= c->nb) return FE_ERR_INVALID_ARG;
  if (c->fp64) qcrit<double>(c->L(), box, c->cur, (double*)q);
  else qcrit<float>(c->L(), box, c->cur, (float*)q);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

extern "C" int fe_profile_start(fe_ctx* c, int kernel_id) {
  if (!c || kernel_id < -1 || kernel_id >= KID_COUNT) return FE_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->st));
  c->prof.on = true;
  c->prof.target = kernel_id;
  c->prof.used = 0;
  c->prof.failed = false;
  for (int k = 0; k < KID_COUNT; ++k) c->prof.count[k] = 0;
  return FE_OK;
}

extern "C" int fe_profile_stop(fe_ctx* c, fe_profile_info* out) {
  if (!c || !out) return FE_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->st));
  memset(out, 0, sizeof(*out));
  double ms = 0.0;
  for (size_t i = 0; i < c->prof.used; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->prof.ev[2 * i], c->prof.ev[2 * i + 1]));
    ms += t;
  }
  long long tot = 0;
  for (int k = 0; k < KID_COUNT; ++k) {
    tot += c->prof.count[k];
    if (k < FE_PROFILE_MAX_KERNELS) out->counts[k] = c->prof.count[k];
  }
  out->launches = tot;
  out->target_launches = (int64_t)c->prof.used;
  out->target_ms = ms;
  c->prof.on = false;
  return c->prof.failed ? FE_ERR_CUDA : FE_OK;
}

extern "C" int fe_kernel_count(void) { return KID_COUNT; }

extern "C" const char* fe_kernel_name(int id) {
  if (id < 0 || id >= KID_COUNT) return "";
  return kKernelNames[id];
}

extern "C" int fe_set_tiling(fe_ctx* c, int tz) {
  if (!c || tz < 0 || tz > 512) return FE_ERR_INVALID_ARG;
  return set_tiling(c, tz);
}

extern "C" int fe_set_box_tiling(fe_ctx* c, int box, int tz) {
  if (!c || box < 0 || box >= c->nb || tz < 0 || tz > 512) return FE_ERR_INVALID_ARG;
  std::vector<int> t = c->tzb;
  t[box] = tz;
  return set_tiling(c, t);
}

// Time of `trials` trial steps (after one untimed) with the tiling tzb; the state is not committed.
static int time_tiling(fe_ctx* c, const std::vector<int>& tzb, int trials, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  int rc = set_tiling(c, tzb);
  if (rc != FE_OK) return rc;
  rc = c->fp64 ? step_once<double>(c, false) : step_once<float>(c, false);
  if (rc != FE_OK) return rc;
  CK(cudaEventRecord(e0, c->st));
  for (int t = 0; t < trials && rc == FE_OK; ++t) rc = c->fp64 ? step_once<double>(c, false) : step_once<float>(c, false);
  CK(cudaEventRecord(e1, c->st));
  if (rc != FE_OK) return rc;
  CK(cudaEventSynchronize(e1));
  CK(cudaEventElapsedTime(ms, e0, e1));
  return FE_OK;
}

extern "C" int fe_autotune(fe_ctx* c, int trials, int* best_tz) {
  if (!c || trials < 1) return FE_ERR_INVALID_ARG;
  int rc = pull_scalars(c);
  if (rc != FE_OK) return rc;
  std::vector<double> saved(c->hsc, c->hsc + (size_t)c->nb * NSC);
  const int cand[] = {4, 8, 16, 24, 32, 48, 64};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // one depth for every box first, then, in an ensemble of several box sizes, each size in turn
  // (largest boxes first) while the others keep theirs
  std::vector<int> best(c->nb, 0);
  float best_ms = 1e30f;
  for (int tz : cand) {
    std::vector<int> t(c->nb, tz);
    float ms = 0.f;
    rc = time_tiling(c, t, trials, e0, e1, &ms);
    if (rc != FE_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  std::vector<int> sizes = c->N;
  std::sort(sizes.begin(), sizes.end(), std::greater<int>());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  for (size_t q = 0; q < sizes.size() && sizes.size() > 1 && rc == FE_OK; ++q) {
    for (int tz : cand) {
      std::vector<int> t = best;
      bool changed = false;
      for (int b = 0; b < c->nb; ++b)
        if (c->N[b] == sizes[q] && t[b] != tz) {
          t[b] = tz;
          changed = true;
        }
      if (!changed) continue;
      float ms = 0.f;
      rc = time_tiling(c, t, trials, e0, e1, &ms);
      if (rc != FE_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc2 = set_tiling(c, best);
  memcpy(c->hsc, saved.data(), saved.size() * sizeof(double));
  CK(cudaMemcpyAsync(c->dsc, c->hsc, saved.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (best_tz) {  // the depth of the largest box
    int bmax = 0;
    for (int b = 1; b < c->nb; ++b)
      if (c->N[b] > c->N[bmax]) bmax = b;
    *best_tz = best[bmax];
  }
  return rc != FE_OK ? rc : rc2;
}

// ---- a-priori LES analysis ----------------------------------------------------------------
extern "C" int fe_les_apriori(fe_ctx* c, int box, int m, double cs, fe_les_stats* out, void* fields) {
  if (!c || !out || box < 0 || box >= c->nb || m < 1 || m > FE_LES_MAX_M || !(cs >= 0.0)) return FE_ERR_INVALID_ARG;
  const int N = c->N[box];
  if (2 * m + 1 > N) return FE_ERR_INVALID_ARG;
  const size_t w = c->fp64 ? 8 : 4;
  const size_t need = (size_t)23 * N * N * N * w;
  if (c->les_bytes < need) {
    cudaFree(c->les_work);
  cudaFree(c->iso_work);
    c->les_work = nullptr;
    c->les_bytes = 0;
    if (cudaMalloc(&c->les_work, need) != cudaSuccess) {
      cudaGetLastError();
      return FE_ERR_OOM;
    }
    c->les_bytes = need;
  }
  const int nbl = les_max_blocks(c->nsm);
  if (!c->les_part) {
    if (cudaMalloc(&c->les_part, (size_t)nbl * 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->les_hpart, (size_t)nbl * 8 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return FE_ERR_OOM;
    }
  }
  const BoxDev& B = c->hbox[box];
  const int s = c->cur;
  double st[6];
  int rc;
  if (c->fp64)
    rc = les_apriori<double>((const double*)B.f[S(s, F_RHO)], (const double*)B.f[S(s, F_U0)],
                             (const double*)B.f[S(s, F_U1)], (const double*)B.f[S(s, F_U2)], N, m, cs,
                             (double*)c->les_work, c->les_part, c->les_hpart, c->nsm, (double*)fields, st, c->st);
  else
    rc = les_apriori<float>((const float*)B.f[S(s, F_RHO)], (const float*)B.f[S(s, F_U0)],
                            (const float*)B.f[S(s, F_U1)], (const float*)B.f[S(s, F_U2)], N, m, cs,
                            (float*)c->les_work, c->les_part, c->les_hpart, c->nsm, (float*)fields, st, c->st);
  if (rc != FE_OK) return rc;
  out->delta = st[0];
  out->k_sgs = st[1];
  out->pi_sgs = st[2];
  out->cs2_opt = st[3];
  out->corr = st[4];
  out->pi_model = st[5];
  return FE_OK;
}

// ---- iso-surfaces and their depth image -------------------------------------------------
extern "C" int fe_isosurface(fe_ctx* c, int box, const void* field, double iso, double* tri, long long max_tri,
                             long long* ntri, double* area) {
  if (!c || !field || !ntri || !area || box < 0 || box >= c->nb || max_tri < 0 || (max_tri > 0 && !tri) ||
      !std::isfinite(iso))
    return FE_ERR_INVALID_ARG;
  const int N = c->N[box];
  const long n = (long)N * N * N;
  const size_t need = iso_work_bytes(n);
  if (c->iso_bytes < need) {
    cudaFree(c->iso_work);
    c->iso_work = nullptr;
    c->iso_bytes = 0;
    if (cudaMalloc(&c->iso_work, need) != cudaSuccess) {
      cudaGetLastError();
      return FE_ERR_OOM;
    }
    c->iso_bytes = need;
  }
  if (c->fp64)
    return isosurface<double>((const double*)field, N, iso, tri, max_tri, c->iso_work, c->iso_host, c->nsm, ntri, area,
                              c->st);
  return isosurface<float>((const float*)field, N, iso, tri, max_tri, c->iso_work, c->iso_host, c->nsm, ntri, area,
                           c->st);
}

extern "C" int fe_raster_depth(fe_ctx* c, const double* tri, long long ntri, int width, double extent,
                               float* depth) {
  if (!c || !depth || width < 1 || width > 65536 || ntri < 0 || (ntri > 0 && !tri) || !(extent > 0.0))
    return FE_ERR_INVALID_ARG;
  int rc = raster_depth(tri, ntri, width, extent, depth, c->nsm, c->st);
  if (rc != FE_OK) return rc;
  CK(cudaStreamSynchronize(c->st));
  return FE_OK;
}

// ---- learned preconditioner --------------------------------------------------------------
extern "C" long fe_preconditioner_size(void) { return unet_param_count(); }

extern "C" int fe_load_preconditioner(fe_ctx* c, const float* w, size_t count) {
  if (!c || !w || (long)count != unet_param_count()) return FE_ERR_INVALID_ARG;
  if (c->hbox[0].N % 4 != 0) return FE_ERR_UNSUPPORTED;
  if (!c->unet) {
    int rc = FE_OK;
    c->unet = unet_create(c->hbox[0].N, true, &rc);
    if (c->unet) unet_set_kernels(c->unet, c->unet_tc);
    if (!c->unet) return rc;
  }
  int rc = unet_set_weights(c->unet, w, c->st);
  c->unet_ready = rc == FE_OK;
  drop_graphs(c);
  return rc;
}

extern "C" int fe_get_preconditioner(fe_ctx* c, float* w, size_t count, int gradients) {
  if (!c || !w || (long)count != unet_param_count()) return FE_ERR_INVALID_ARG;
  if (!c->unet_ready) return FE_ERR_UNSUPPORTED;
  return unet_get_weights(c->unet, w, gradients ? 1 : 0, c->st);
}

extern "C" int fe_precond_apply(fe_ctx* c, int box, const void* r, double dt, float* z) {
  if (!c || box != 0 || !r || !z || !(dt > 0.0)) return FE_ERR_INVALID_ARG;
  if (!c->unet_ready) return FE_ERR_UNSUPPORTED;
  BoxDev& B = c->hbox[0];
  // psi of the current state and the Jacobi inverse of the operator with this dt
  if (c->fp64) k_psi_box<double><<<1024, 256, 0, c->st>>>(c->dbox, 0, c->cur, dt);
  else k_psi_box<float><<<1024, 256, 0, c->st>>>(c->dbox, 0, c->cur, dt);
  if (c->fp64)
    return unet_apply<double>(c->unet, (const double*)r, (const double*)B.f[W_DINV], dt, B.ih, z, c->st);
  return unet_apply<float>(c->unet, (const float*)r, (const float*)B.f[W_DINV], dt, B.ih, z, c->st);
}

extern "C" int fe_precond_train_step(fe_ctx* c, int box, const void* r, const void* e, double dt, double lr,
                                     double* loss) {
  if (!c || box != 0 || !r || !e || !loss || !(dt > 0.0)) return FE_ERR_INVALID_ARG;
  if (!c->unet_ready) return FE_ERR_UNSUPPORTED;
  BoxDev& B = c->hbox[0];
  if (c->fp64) k_psi_box<double><<<1024, 256, 0, c->st>>>(c->dbox, 0, c->cur, dt);
  else k_psi_box<float><<<1024, 256, 0, c->st>>>(c->dbox, 0, c->cur, dt);
  if (c->fp64)
    return unet_train_step<double>(c->unet, (const double*)r, (const double*)e, (const double*)B.f[W_DINV], dt, B.ih,
                                   lr, loss, c->st);
  return unet_train_step<float>(c->unet, (const float*)r, (const float*)e, (const float*)B.f[W_DINV], dt, B.ih, lr,
                                loss, c->st);
}

extern "C" int fe_harvest_pressure(fe_ctx* c, void* const* b_out, void* const* x_out, int max_pairs, int* npairs) {
  if (!c || !b_out || !x_out || max_pairs < 1 || !npairs) return FE_ERR_INVALID_ARG;
  const int solver = c->prm.solver;
  const int plain = c->prm.transonic ? FE_BICGSTAB_JACOBI : FE_PCG_JACOBI;
  if (plain == FE_BICGSTAB_JACOBI && !c->hbox[0].f[K_RHAT]) return FE_ERR_UNSUPPORTED;  // no BiCGStab vectors
  c->prm.solver = plain;
  c->harvest_b = b_out;
  c->harvest_x = x_out;
  c->harvest_max = max_pairs;
  c->harvest_n = 0;
  int rc = c->fp64 ? step_once<double>(c) : step_once<float>(c);
  c->prm.solver = solver;
  c->harvest_b = c->harvest_x = nullptr;
  *npairs = c->harvest_n;
  if (rc == FE_OK) CK(cudaStreamSynchronize(c->st));
  return rc;
}

extern "C" int fe_precond_activation(fe_ctx* c, int layer, float* out, size_t count) {
  if (!c || !out) return FE_ERR_INVALID_ARG;
  if (!c->unet_ready) return FE_ERR_UNSUPPORTED;
  return unet_activation(c->unet, layer, out, (long)count, c->st);
}

extern "C" int fe_precond_kernels(fe_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 1) return FE_ERR_INVALID_ARG;
  c->unet_tc = mode;
  if (c->unet) unet_set_kernels(c->unet, mode);
  drop_graphs(c);
  return FE_OK;
}

extern "C" int fe_use_plane_streaming(fe_ctx* c, int on) {
  if (!c) return FE_ERR_INVALID_ARG;
  if (c->use_bulk != (on != 0)) drop_graphs(c);
  c->use_bulk = on != 0;
  return FE_OK;
}

extern "C" int fe_plane_streaming_active(const fe_ctx* c) {
  if (!c) return FE_ERR_INVALID_ARG;
  return c->use_bulk && c->nbblocks > 0 ? 1 : 0;
}

extern "C" int fe_use_graphs(fe_ctx* c, int on) {
  if (!c) return FE_ERR_INVALID_ARG;
  c->use_graphs = on != 0;
  if (!c->use_graphs) drop_graphs(c);
  return FE_OK;
}
