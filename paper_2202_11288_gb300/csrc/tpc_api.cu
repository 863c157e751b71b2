// C ABI (include/tpcamg.h): device hierarchy, launch plans, V-cycle and solve loop.
//
// Two device hierarchies may exist per handle: FP64 (always; the outer residual, tpc_apply,
// tpc_vcycle) and FP32 (precision = TPC_MIXED: the inner V-cycles). The FP32 spectra are the
// FP64 spectra rounded once.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tpc_internal.h"
#include "tpc_kernels.cuh"
#include "tpc_f32.cuh"
#include "tpc_box.cuh"
#include "tpc_krylov.cuh"

namespace tpc {
void set_host_error(const std::string& s);
const char* host_error();

// One block does the whole product for m <= 2^LOG_WHOLE: FP64 (bound by the FP64 pipe, one
// SM is slow) only for small m; FP32 up to the 4096 points one block holds.
template <typename T> constexpr int log_whole() { return sizeof(T) == 8 ? 9 : 12; }
constexpr int LOG_R1_MAX = 11;    // strided pass: at most 2048 rows
constexpr int LOG_TILE_MAX = 13;  // strided tile: at most 8192 complex entries
constexpr int NORM_BLOCKS = 304;  // 2 x 152 SMs

template <typename T> struct DevLevel {
  int k = 0;
  long long N = 0, n = 0, m = 0;
  int logm = 0, logR1 = 0, logL = 0, logC = 0;
  int fwd_blocks = 0, mid_blocks = 0;
  size_t smem_strided = 0, smem_mid = 0;
  T* sA = nullptr;
  T* sD = nullptr;
  c2<T>* sB = nullptr;
  c2<T>* sC = nullptr;
  T* p = nullptr;
  T* q = nullptr;
  T* xi = nullptr;
  T* zeta = nullptr;
  T o = 0, wA_pre = 0, wO_pre = 0, wD_pre = 0, wA_post = 0, wO_post = 0, wD_post = 0;
  // support of the Cross vectors: q, zeta vanish from index nq on, p, xi from np on (the
  // couplings to the middle unknown reach only about r points, scaled per level)
  long long nq = 0, np = 0;
  // weakly singular model only: tridiagonal band (entries (i, i-1), (i, i), (i, i+1)) and the
  // per-entry damped Jacobi weights omega / a_ii (the diagonal is not constant per segment)
  T* bl = nullptr;
  T* bd = nullptr;
  T* bu = nullptr;
  T* wpre = nullptr;
  T* wpost = nullptr;
  c2<T>* twm = nullptr;
  // FP32 levels with m = 2^20 .. 2^23 (no band): the register-resident kernels of tpc_f32.cuh
  // with four columns per strided tile
  bool f32reg = false;
};

// Smallest s with v[i] == 0 for every i >= s (over the union of two vectors).
inline long long support2(const std::vector<double>& a, const std::vector<double>& b) {
  long long s = (long long)a.size();
  while (s > 0 && a[s - 1] == 0.0 && b[s - 1] == 0.0) --s;
  return s;
}

// Device hierarchy in one precision.
template <typename T> struct Hier {
  std::vector<DevLevel<T>> lev;  // lev[i] = level K - i
  std::vector<T*> f, e, t;       // per level vectors (n_k)
  c2<T>* z = nullptr;            // complex work array (m_K)
  T* partials = nullptr;
  c2<T>* twL = nullptr;          // W_4096^j, j < 4096 (FP32 kernels copy j <= 512)
  c2<T>* tws = nullptr;          // FP32: step twiddle tables (f32p::STEP_TW_ENTRIES)
  T* coarse_inv = nullptr;
  BottomPlan<T>* bottom = nullptr;  // single-block V-cycle bottom (FP32, V(1,1)), or null
  int bottom_li = -1;               // level index where it takes over
  size_t bottom_smem = 0;
  int geo = 0;                      // transfer (tpc_params.transfer)
};

}  // namespace tpc

using namespace tpc;

struct tpc_handle {
  tpc_params prm{};
  int K = 0, kc = 0, r = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;            // created here when the caller passed NULL
  HostHierarchy host;
  Hier<double> d;                     // FP64 hierarchy
  Hier<float> s;                      // FP32 hierarchy (TPC_MIXED only)
  double* u = nullptr;                // finest solution
  double* b = nullptr;                // finest right-hand side (copy)
  double* r0 = nullptr;               // finest residual
  float* res32 = nullptr;             // TPC_MIXED: inner residual and accumulated correction
  float* acc32 = nullptr;
  double* sumsq_part = nullptr;
  double* sumsq = nullptr;            // device scalar ||r||^2
  double* sumsq_host = nullptr;       // pinned
  double* hb = nullptr;               // device staging for tpc_solve_host (b, x)
  double* hx = nullptr;
  // one outer iteration as a CUDA graph per count of inner FP32 cycles (the index; FP64: 1
  // only), all captured at set-up
  cudaGraphExec_t iter_exec[33] = {};
  long long iter_nodes[33] = {};      // kernel nodes of iter_exec[c]
  cudaEvent_t ev = nullptr;           // marks the latest ||r||^2 read-back
  long long launches = 0;             // kernels launched so far (see tpc_kernel_launches)
  int last_cycles = 0;                // V-cycles of the latest solve (tpc_last_solve_cycles)
  // finest residual from prefix sums (tpc_params.box_residual, piecewise-constant generators):
  // the arguments with the work arrays filled in (operand, right-hand side, result per call)
  bool box_on = false;
  box::BoxArgs box_args{};
  // TPC_OUTER_FGMRES: basis vectors v_0..v_S and z_0..z_{S-1} (S = inner_cycles; FP32 in
  // TPC_MIXED, FP64 else; kld apart), the cycle's scalars and the dot products' partial sums
  float* kv32 = nullptr;
  float* kz32 = nullptr;
  double* kv64 = nullptr;
  double* kz64 = nullptr;
  long long kld = 0;
  krylov::KState* ks = nullptr;
  double* kpart = nullptr;
  std::string err;
  std::vector<void*> dev_allocs;
  size_t dev_bytes = 0;               // device memory held by the handle
};

namespace {

// NVTX ranges (header-only NVTX3: no cost unless a profiler is attached) mark set-up phases,
// solves and outer iterations on the host timeline.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

int cuda_fail(tpc_handle* H, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  if (H) H->err = msg;
  set_host_error(msg);
  return TPC_ECUDA;
}

#define TPC_CUDA(H, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(H, e_, #call);  \
  } while (0)

#define TPC_TRY(x)                   \
  do {                               \
    int rc_ = (x);                   \
    if (rc_ != TPC_OK) return rc_;   \
  } while (0)

// Device allocations of a handle come from the device's stream-ordered memory pool (fast to
// take and return when many handles are set up and destroyed, e.g. by a batch or a server).
template <typename P>
int dalloc(tpc_handle* H, P** ptr, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMallocAsync(&v, count * sizeof(P) + 16, H->stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    H->err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
    set_host_error(H->err);
    return (e == cudaErrorMemoryAllocation) ? TPC_ENOMEM : TPC_ECUDA;
  }
  H->dev_allocs.push_back(v);
  H->dev_bytes += count * sizeof(P) + 16;
  *ptr = reinterpret_cast<P*>(v);
  if (H->prm.poison) {  // all bits set: NaN in FP32 and FP64
    e = cudaMemsetAsync(v, 0xFF, count * sizeof(P) + 16, H->stream);
    if (e != cudaSuccess) return cuda_fail(H, e, "cudaMemsetAsync (poison)");
  }
  return TPC_OK;
}

// Copy FP64 host values to a device array of T (rounded once when T is float).
template <typename T>
int upload(tpc_handle* H, T* dst, const std::vector<double>& src) {
  if (sizeof(T) == sizeof(double)) {
    TPC_CUDA(H, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double),
                                cudaMemcpyHostToDevice, H->stream));
  } else {
    std::vector<T> tmp(src.begin(), src.end());
    TPC_CUDA(H, cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice,
                                H->stream));
  }
  TPC_CUDA(H, cudaStreamSynchronize(H->stream));  // the source may go out of scope
  return TPC_OK;
}

int grid_for(long long n) {
  long long g = (n + NTHREADS - 1) / NTHREADS;
  if (g > 4 * 152) g = 4 * 152;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
void plan_level(DevLevel<T>& L) {
  L.logm = L.k + 1;
  if (L.logm <= log_whole<T>()) {
    L.logR1 = 0;
    L.logL = L.logm;
    L.logC = 0;
    L.fwd_blocks = 0;
    L.mid_blocks = 1;
  } else {
    int logL = (L.logm + 1) / 2;
    if (logL > LOG_LMAX) logL = LOG_LMAX;
    L.logL = logL;
    L.logR1 = L.logm - logL;
    int logC = 4;
    if (logC > LOG_TILE_MAX - L.logR1) logC = LOG_TILE_MAX - L.logR1;
    int want = logL - 9;  // keep >= 512 column blocks when the level is large enough
    if (want < 0) want = 0;
    if (logC > want) logC = want;
    if (logC < 0) logC = 0;
    L.logC = logC;
    L.fwd_blocks = 1 << (logL - logC);
    L.mid_blocks = (1 << (L.logm - logL - 1)) + 1;
  }
  L.smem_strided =
      L.logR1 ? sizeof(c2<T>) * (size_t)(tw_slots<T>() + padded_size(1 << (L.logR1 + L.logC))) : 0;
  L.smem_mid =
      sizeof(c2<T>) * (size_t)(tw_slots<T>() + padded_size(1 << (L.logL + (L.logR1 ? 1 : 0))));
}

// The plan of a three-pass level for the factorisation m = R1 x L with L = 2^logL: the
// register-resident FP32 kernels where they apply (reg), else the general kernels with tile
// width 2^logC (logC < 0: the rule of plan_level).
template <typename T>
void apply_split(DevLevel<T>& L, int logL, int logC, bool reg) {
  L.logL = logL;
  L.logR1 = L.logm - logL;
  L.mid_blocks = (1 << (L.logm - logL - 1)) + 1;
  L.f32reg = reg;
  if (reg) {
    L.logC = f32p::LOG_CT;
    L.fwd_blocks = 1 << (logL - f32p::LOG_CT);
    L.smem_strided = f32p::strided_smem(L.logR1);
    L.smem_mid = f32p::mid_smem(logL);
    return;
  }
  if (logC < 0) {
    logC = 4;
    if (logC > LOG_TILE_MAX - L.logR1) logC = LOG_TILE_MAX - L.logR1;
    const int want = logL - 9 > 0 ? logL - 9 : 0;  // >= 512 column blocks on large levels
    if (logC > want) logC = want;
    if (logC < 0) logC = 0;
  }
  L.logC = logC;
  L.fwd_blocks = 1 << (logL - logC);
  L.smem_strided = sizeof(c2<T>) * (size_t)(tw_slots<T>() + padded_size(1 << (L.logR1 + logC)));
  L.smem_mid = sizeof(c2<T>) * (size_t)(tw_slots<T>() + padded_size(1 << (logL + 1)));
}

template <typename T>
LevelArgs<T> level_args(const Hier<T>& G, const DevLevel<T>& L) {
  LevelArgs<T> a{};
  a.N = (int)L.N;  // levels have m <= 2^23
  a.logm = L.logm;
  a.logR1 = L.logR1;
  a.logL = L.logL;
  a.logC = L.logC;
  a.sA = L.sA;
  a.sD = L.sD;
  a.sB = L.sB;
  a.sC = L.sC;
  a.p = L.p;
  a.q = L.q;
  a.xi = L.xi;
  a.zeta = L.zeta;
  a.nq = (int)L.nq;
  a.np = (int)L.np;
  a.bl = L.bl;
  a.bd = L.bd;
  a.bu = L.bu;
  a.pvec = L.wpre;
  a.wvec = L.wpre;
  a.o = L.o;
  a.twm = L.twm;
  a.twL = G.twL;
  a.tws = G.tws;
  a.z = G.z;
  a.partials = G.partials;
  a.nparts = L.fwd_blocks;
  a.geo = G.geo;
  return a;
}

// How the operand of a product is formed while it is loaded (see Pro in tpc_kernels.cuh).
template <typename T> struct Prologue {
  int mode = PRO_NONE;
  T* xout = nullptr;        // operand stored here (PRO_SMOOTH / RESTRICT / PROLONG)
  T* fout = nullptr;        // restricted right-hand side stored here (PRO_RESTRICT)
  const T* rfine = nullptr;
  const T* ec = nullptr;
};

// The arguments of one product y = epilogue(A_k u) (u = x or formed by the prologue).
template <typename T>
LevelArgs<T> stage_args(const Hier<T>& G, const DevLevel<T>& L, const T* x, const T* f, T* y,
                        int epi, bool post, const Prologue<T>& pro) {
  LevelArgs<T> a = level_args<T>(G, L);
  a.x = x;
  a.f = f;
  a.y = y;
  a.epi = epi;
  a.wA = post ? L.wA_post : L.wA_pre;
  a.wO = post ? L.wO_post : L.wO_pre;
  a.wD = post ? L.wD_post : L.wD_pre;
  a.wvec = post ? L.wpost : L.wpre;
  a.pro = pro.mode;
  a.pA = L.wA_pre;
  a.pO = L.wO_pre;
  a.pD = L.wD_pre;
  a.xout = pro.xout;
  a.fout = pro.fout;
  a.rfine = pro.rfine;
  a.ec = pro.ec;
  return a;
}

// y = epilogue(A_k u) for one level on the handle's stream, u = x or formed by the prologue.
template <typename T, bool NS>
void launch_matvec(tpc_handle* H, const Hier<T>& G, const DevLevel<T>& L, const T* x,
                   const T* f, T* y, int epi, bool post, const Prologue<T>& pro) {
  const LevelArgs<T> a = stage_args<T>(G, L, x, f, y, epi, post, pro);
  cudaStream_t s = H->stream;
  if (L.logR1 == 0) {
    launch_k(k_mid_whole<T, NS>, 1, fft_threads<T>(), L.smem_mid, s, a);
    H->launches += 1;
    return;
  }
  H->launches += 3;
  if constexpr (sizeof(T) == 4) {
    if (L.f32reg) {
      f32p::launch_fwd(a, L.fwd_blocks, s);
      f32p::launch_mid<NS>(a, L.mid_blocks, s);
      f32p::launch_inv(a, L.fwd_blocks, s);
      return;
    }
  }
  launch_fwd_strided<T>(a, L.fwd_blocks, L.smem_strided, s);
  launch_mid_pair<T, NS>(a, L.mid_blocks, L.smem_mid, s);
  launch_inv_strided<T>(a, L.fwd_blocks, L.smem_strided, s);
}

template <typename T>
void matvec(tpc_handle* H, const Hier<T>& G, int li, const T* x, const T* f, T* y, int epi,
            bool post, const Prologue<T>& pro = Prologue<T>()) {
  if (H->prm.variant != TPC_SPD)
    launch_matvec<T, true>(H, G, G.lev[li], x, f, y, epi, post, pro);
  else
    launch_matvec<T, false>(H, G, G.lev[li], x, f, y, epi, post, pro);
}

// Algorithm 2 on level index li (level K - li). The right-hand side is f_top (top level) or
// the restriction of rfine, the residual of the finer level (stored in G.f[li] on the way).
// Returns the buffer that holds B_k f: G.e[li] or G.t[li].
//   pre-smoothing:  the first sweep from 0 is the prologue of the first product
//                   (u = omega D^{-1} f, after restricting f when the level is not the top);
//   residual:       epilogue of the last pre-smoothing product (f - A u), restricted by the
//                   next level's prologue;
//   correction:     prologue of the first post-smoothing product (u + I_{k-1}^k e_c).
template <typename T>
T* enqueue_vcycle(tpc_handle* H, Hier<T>& G, int li, const T* f_top, const T* rfine) {
  const DevLevel<T>& L = G.lev[li];
  cudaStream_t s = H->stream;
  T* e = G.e[li];
  T* t = G.t[li];
  const T* f = rfine ? G.f[li] : f_top;
  if constexpr (sizeof(T) == 4) {  // the single-block bottom exists in FP32 only
    if (G.bottom && li == G.bottom_li && rfine) {
      if (H->prm.variant != TPC_SPD)
        launch_k(k_vcycle_bottom<T, true>, 1, fft_threads<T>(), G.bottom_smem, s, G.bottom);
      else
        launch_k(k_vcycle_bottom<T, false>, 1, fft_threads<T>(), G.bottom_smem, s, G.bottom);
      H->launches += 1;
      return t;  // the last post-smoothing product of level li writes G.t[li]
    }
  }
  if (L.k == H->kc) {
    if (rfine) {
      launch_k(k_coarse_solve<T>, 1, 256, 0, s, G.coarse_inv, G.f[li], rfine, e, (int)L.n, G.geo);
    } else {
      launch_k(k_coarse_solve<T>, 1, 256, 0, s, G.coarse_inv, const_cast<T*>(f_top), nullptr, e,
               (int)L.n, G.geo);
    }
    H->launches += 1;
    return e;
  }
  Prologue<T> first;
  first.mode = rfine ? PRO_RESTRICT : PRO_SMOOTH;
  first.xout = e;
  first.fout = G.f[li];
  first.rfine = rfine;
  for (int l = 1; l < H->prm.m1; ++l) {
    matvec<T>(H, G, li, e, f, t, EPI_JACOBI, false, first);
    first = Prologue<T>();
    std::swap(e, t);
  }
  matvec<T>(H, G, li, e, f, t, EPI_RESID, false, first);
  const T* ec = enqueue_vcycle<T>(H, G, li + 1, nullptr, t);
  if (H->prm.m2 == 0) {
    launch_k(k_prolong_add<T>, grid_for(L.n), NTHREADS, 0, s, e, ec, L.n, G.geo);
    H->launches += 1;
    return e;
  }
  Prologue<T> corr;
  corr.mode = PRO_PROLONG;
  corr.xout = e;
  corr.ec = ec;
  for (int l = 0; l < H->prm.m2; ++l) {
    matvec<T>(H, G, li, e, f, t, EPI_JACOBI, true, corr);
    corr = Prologue<T>();
    std::swap(e, t);
  }
  return e;
}

// r = b - A_K x on the finest level (the outer residual): from prefix sums when the handle
// uses the box form, else the FFT product with its residual epilogue.
void enqueue_finest_residual(tpc_handle* H, const double* x, const double* b, double* r) {
  if (!H->box_on) {
    matvec<double>(H, H->d, 0, x, b, r, EPI_RESID, false);
    return;
  }
  box::BoxArgs a = H->box_args;
  a.x = x;
  a.b = b;
  a.r = r;
  cudaStream_t s = H->stream;
  launch_k(box::k_box_local, 2 * a.nblk, box::NT, 0, s, a);
  launch_k(box::k_box_offsets, 1, 1024, 0, s, a);
  const int gx = (int)std::min<long long>((a.N + box::NT - 1) / box::NT, 4 * 152);
  launch_k(box::k_box_resid, dim3(gx, 2), box::NT, 0, s, a);
  H->launches += 3;
}

// Runs of equal nonzero values of a generator t[d + N - 1] (d = -(N-1)..N-1); -1 if there are
// more than maxr.
int generator_runs(const std::vector<double>& t, long long N, box::Run* out, int maxr) {
  int n = 0;
  long long d = -(N - 1);
  while (d <= N - 1) {
    const double v = t[(size_t)(d + N - 1)];
    long long e = d;
    while (e + 1 <= N - 1 && t[(size_t)(e + 1 + N - 1)] == v) ++e;
    if (v != 0.0) {
      if (n == maxr) return -1;
      out[n].lo = (int)d;
      out[n].hi = (int)e;
      out[n].val = v;
      ++n;
    }
    d = e + 1;
  }
  return n;
}

// Sets up the box form of the finest residual when the finest generators have few runs.
int setup_box(tpc_handle* H) {
  H->box_on = false;
  if (!H->prm.box_residual) return TPC_OK;
  const LevelForm& F = H->host.lev[0];
  const DevLevel<double>& L = H->d.lev[0];
  if (F.has_band() || !L.p) return TPC_OK;
  box::BoxArgs a{};
  const std::vector<double>* gens[4] = {&F.tA, &F.tB, &F.tC, &F.tD};
  for (int g = 0; g < 4; ++g) {
    a.nrun[g] = generator_runs(*gens[g], F.N, a.run[g], box::MAXR);
    if (a.nrun[g] < 0) return TPC_OK;  // not piecewise constant enough: FFT residual
  }
  a.N = (int)F.N;
  a.nblk = (int)((F.N + 1 + box::BLK - 1) / box::BLK);
  TPC_TRY(dalloc(H, &a.loc, 2 * (size_t)(F.N + 1)));
  TPC_TRY(dalloc(H, &a.bsum, 2 * (size_t)a.nblk));
  TPC_TRY(dalloc(H, &a.off, 2 * (size_t)a.nblk));
  TPC_TRY(dalloc(H, &a.part, 2 * (size_t)a.nblk));
  TPC_TRY(dalloc(H, &a.dot, 1));
  a.p = L.p;
  a.q = L.q;
  a.xi = L.xi;
  a.zeta = L.zeta;
  a.o = L.o;
  a.nq = (int)L.nq;
  a.np = (int)L.np;
  H->box_args = a;
  H->box_on = true;
  return TPC_OK;
}

void enqueue_sumsq(tpc_handle* H, const double* r, long long n) {
  H->launches += 2;
  launch_k(k_sumsq_partial<double>, NORM_BLOCKS, NTHREADS, 0, H->stream, r, n, H->sumsq_part);
  launch_k(k_sumsq_final, 1, 32, 0, H->stream, H->sumsq_part, NORM_BLOCKS, H->sumsq);
}

// One restart cycle of flexible GMRES with `steps` steps (tpc_krylov.cuh) on the FP64 residual
// r0 of n unknowns (its squared norm in sumsq): basis vectors V (steps + 1) and Z (steps), ld
// apart, of the V-cycles' precision T; vcycle(v) enqueues one V-cycle on right-hand side v and
// returns where its result is, matvec(x, y) enqueues y = A x; u += Z y. Shared by the 1-D and
// 2-D solvers.
template <typename T, typename VC, typename MV>
long long fgmres_cycle(cudaStream_t s, long long n, long long ld, const double* r0,
                       const double* sumsq, double* u, T* V, T* Z, krylov::KState* ks,
                       double* kpart, int steps, VC vcycle, MV matvec) {
  using namespace krylov;
  const int g = grid_for(n);
  long long launches = 0;
  launch_k(k_kry_start<T>, g, NTHREADS, 0, s, r0, V, n, sumsq, ks);
  ++launches;
  for (int j = 0; j < steps; ++j) {
    T* vj = V + (size_t)j * ld;
    T* w = V + (size_t)(j + 1) * ld;
    T* zj = Z + (size_t)j * ld;
    const T* ec = vcycle(vj);
    launch_k(k_copy<T>, g, NTHREADS, 0, s, ec, zj, n);
    matvec(zj, w);
    for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
      launch_k(k_kry_dot_partial<T>, dim3(KNB, j + 1), 256, 0, s, V, ld, w, n, kpart);
      launch_k(k_kry_dot_final, j + 1, 32, 0, s, kpart, KNB, ks, j, pass);
      launch_k(k_kry_axpy<T>, g, NTHREADS, 0, s, w, V, ld, j + 1, ks, n);
    }
    launch_k(k_kry_sumsq_partial<T>, KNB, 256, 0, s, w, n, kpart);
    launch_k(k_kry_rotate, 1, 32, 0, s, kpart, KNB, ks, j);
    launch_k(k_kry_scale<T>, g, NTHREADS, 0, s, w, n, ks);
    launches += 11;
  }
  launch_k(k_kry_solve, 1, 32, 0, s, ks, steps);
  launch_k(k_kry_update<T>, g, NTHREADS, 0, s, u, Z, ld, steps, ks, n);
  return launches + 2;
}

template <typename T>
void enqueue_fgmres_cycle(tpc_handle* H, Hier<T>& G, T* V, T* Z, int steps) {
  const long long n = H->d.lev[0].n;
  H->launches += fgmres_cycle<T>(
      H->stream, n, H->kld, H->r0, H->sumsq, H->u, V, Z, H->ks, H->kpart, steps,
      [&](const T* v) -> const T* { return enqueue_vcycle<T>(H, G, 0, v, nullptr); },
      [&](const T* x, T* y) { matvec<T>(H, G, 0, x, nullptr, y, EPI_APPLY, false); });
}

// One outer iteration.
//   FGMRES: one restart cycle of `cycles` steps (above); r = b - A u; ||r||^2.
//   FP64:  u += B_K r; r = b - A u; ||r||^2.
//   mixed: f = s r in FP32 (s = sqrt(n) / ||r||); `cycles` FP32 iterations
//          e <- e + B_K (f - A e) from e = 0; u += e / s; then the FP64 residual and norm.
void enqueue_iteration(tpc_handle* H, int cycles) {
  const long long n = H->d.lev[0].n;
  const int g = grid_for(n);
  if (H->prm.outer == TPC_OUTER_FGMRES) {
    if (H->prm.precision == TPC_MIXED) enqueue_fgmres_cycle<float>(H, H->s, H->kv32, H->kz32, cycles);
    else enqueue_fgmres_cycle<double>(H, H->d, H->kv64, H->kz64, cycles);
  } else if (H->prm.precision == TPC_MIXED) {
    Hier<float>& S = H->s;
    launch_k(k_to_f32_scaled, g, NTHREADS, 0, H->stream, H->r0, S.f[0], n, H->sumsq);
    H->launches += 1;
    const float* ec = enqueue_vcycle<float>(H, S, 0, S.f[0], nullptr);
    launch_k(k_copy<float>, g, NTHREADS, 0, H->stream, ec, H->acc32, n);
    H->launches += 1;
    for (int c = 1; c < cycles; ++c) {
      matvec<float>(H, S, 0, H->acc32, S.f[0], H->res32, EPI_RESID, false);
      ec = enqueue_vcycle<float>(H, S, 0, H->res32, nullptr);
      launch_k(k_axpy<float>, g, NTHREADS, 0, H->stream, H->acc32, ec, n);
      H->launches += 1;
    }
    launch_k(k_axpy_f32_scaled, g, NTHREADS, 0, H->stream, H->u, H->acc32, n, H->sumsq);
    H->launches += 1;
  } else {
    double* e = enqueue_vcycle<double>(H, H->d, 0, H->r0, nullptr);
    launch_k(k_axpy<double>, g, NTHREADS, 0, H->stream, H->u, e, n);
    H->launches += 1;
  }
  enqueue_finest_residual(H, H->u, H->b, H->r0);
  enqueue_sumsq(H, H->r0, n);
}

int full_cycles(const tpc_handle* H) {
  return (H->prm.precision == TPC_MIXED || H->prm.outer == TPC_OUTER_FGMRES) ? H->prm.inner_cycles
                                                                               : 1;
}

// Captures and instantiates the iteration graph with `cycles` inner cycles unless it exists.
int iter_graph(tpc_handle* H, int cycles) {
  if (cycles < 1 || cycles > 32) return TPC_EINVAL;
  if (H->iter_exec[cycles]) return TPC_OK;
  cudaGraph_t graph = nullptr;
  TPC_CUDA(H, cudaStreamBeginCapture(H->stream, cudaStreamCaptureModeThreadLocal));
  const long long before = H->launches;
  enqueue_iteration(H, cycles);
  const long long nodes = H->launches - before;
  H->launches = before;
  cudaError_t ce = cudaStreamEndCapture(H->stream, &graph);
  if (ce != cudaSuccess) return cuda_fail(H, ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&H->iter_exec[cycles], graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    H->iter_exec[cycles] = nullptr;
    return cuda_fail(H, ce, "cudaGraphInstantiate");
  }
  H->iter_nodes[cycles] = nodes;
  return TPC_OK;
}

template <typename T, bool NS>
cudaError_t set_smem_attrs() {
  const int big = 150 * 1024;  // largest: (520 + 8704) x 16 B = 144 KB
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = strided_smem_attrs<T>(big)) != cudaSuccess) return e;
  if ((e = mid_pair_smem_attrs<T, NS>(big)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_mid_whole<T, NS>, A, big)) != cudaSuccess) return e;
  if constexpr (sizeof(T) == 8) {  // the generator spectra are transformed in FP64 only
    if ((e = cudaFuncSetAttribute(k_fwd_strided<T, IN_REAL, PRO_NONE>, A, big)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_mid_fwd<T>, A, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_mid_fwd_real<T>, A, big)) != cudaSuccess) return e;
  } else {  // the single-block V-cycle bottom and the register-resident kernels: FP32 only
    if ((e = cudaFuncSetAttribute(k_vcycle_bottom<T, NS>, A, big)) != cudaSuccess) return e;
    if ((e = f32p::set_attrs()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Circulant first column of an N x N Toeplitz generator, embedded in length m (eq. (3.4)):
// c[d] = t_d, c[m - d] = t_{-d} for 1 <= d <= N - 1, zero elsewhere.
void circulant_column(const std::vector<double>& t, long long N, long long m,
                      std::vector<double>& c) {
  c.assign((size_t)m, 0.0);
  c[0] = t[N - 1];
  for (long long d = 1; d <= N - 1; ++d) {
    c[d] = t[d + N - 1];
    c[m - d] = t[-d + N - 1];
  }
}

// Forward transform (FP64) of a real length-m column into G.z (bit-reversed order).
int forward_real(tpc_handle* H, const Hier<double>& G, const DevLevel<double>& L,
                 const double* real_dev) {
  LevelArgs<double> a = level_args<double>(G, L);
  a.real_in = real_dev;
  cudaStream_t s = H->stream;
  H->launches += L.logR1 ? 2 : 1;
  if (L.logR1 == 0) {
    k_mid_fwd_real<double><<<1, FFT_THREADS, L.smem_mid, s>>>(a);
  } else {
    k_fwd_strided<double, IN_REAL, PRO_NONE><<<L.fwd_blocks, FFT_THREADS, L.smem_strided, s>>>(a);
    k_mid_fwd<double><<<1 << L.logR1, FFT_THREADS,
                        sizeof(double2) * (size_t)(tw_slots<double>() + padded_size(1 << L.logL)), s>>>(a);
  }
  TPC_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

// Step twiddles of the register-resident FP32 kernels: for S = 2^s, s = 5..12, the entries
// W_S^{c bitrev_16(t)} (t < 16, c < S / 16) at complex offset (S - 32) + t (S / 16) + c.
void step_twiddle_tables(std::vector<double>& out) {
  out.assign(2 * (size_t)f32p::STEP_TW_ENTRIES, 0.0);
  std::vector<double> w;
  for (int ls = 5; ls <= 12; ++ls) {
    const long long S = 1LL << ls, cols = S / 16;
    twiddles(S, S, w);
    for (int t = 0; t < 16; ++t) {
      const long long bt = (long long)(((t & 1) << 3) | ((t & 2) << 1) | ((t & 4) >> 1) | ((t & 8) >> 3));
      for (long long c = 0; c < cols; ++c) {
        const long long e = (c * bt) % S;
        const size_t o = (size_t)(f32p::steptw_off(ls) + t * cols + c);
        out[2 * o] = w[2 * e];
        out[2 * o + 1] = w[2 * e + 1];
      }
    }
  }
}

// Level data (plan, Cross, diagonal weights, twiddles, vectors) of hierarchy G.
template <typename T>
int alloc_levels(tpc_handle* H, Hier<T>& G) {
  const HostHierarchy& HH = H->host;
  const int nlev = (int)HH.lev.size();
  G.lev.resize(nlev);
  G.geo = H->prm.transfer == TPC_TRANSFER_GEOMETRIC ? 1 : 0;
  std::vector<double> tw;
  twiddles(1LL << LOG_LMAX, 1LL << LOG_LMAX, tw);  // W_4096^j, j < 4096
  TPC_TRY(dalloc(H, &G.twL, (size_t)1 << LOG_LMAX));
  TPC_TRY(upload<T>(H, reinterpret_cast<T*>(G.twL), tw));
  if (sizeof(T) == 4) {
    std::vector<double> st;
    step_twiddle_tables(st);
    TPC_TRY(dalloc(H, &G.tws, (size_t)f32p::STEP_TW_ENTRIES));
    TPC_TRY(upload<T>(H, reinterpret_cast<T*>(G.tws), st));
  }
  long long max_m = 0;
  int max_parts = 1;
  for (int i = 0; i < nlev; ++i) {
    const LevelForm& F = HH.lev[i];
    DevLevel<T>& L = G.lev[i];
    L.k = F.k;
    L.N = F.N;
    L.n = 2 * F.N + 1;
    L.m = 2 * F.N + 2;
    plan_level(L);
    if (sizeof(T) == 4 && f32p::eligible(L.logm, L.logR1, L.logL, F.has_band())) {
      L.f32reg = true;
      L.logC = f32p::LOG_CT;
      L.fwd_blocks = 1 << (L.logL - f32p::LOG_CT);
      L.smem_strided = f32p::strided_smem(L.logR1);
      L.smem_mid = f32p::mid_smem(L.logL);
    }
    if (L.logR1 > LOG_R1_MAX) {
      H->err = "level too large for this build (m > 2^23)";
      return TPC_ENOTSUP;
    }
    if (L.m > max_m) max_m = L.m;
    if (L.fwd_blocks > max_parts) max_parts = L.fwd_blocks;
    const double dA = F.tA[F.N - 1], dO = F.o, dD = F.tD[F.N - 1];
    const double wpre = H->prm.omega_pre, wpost = H->prm.omega_post;
    L.o = (T)F.o;
    L.wA_pre = (T)(wpre / dA);
    L.wO_pre = (T)(wpre / dO);
    L.wD_pre = (T)(wpre / dD);
    L.wA_post = (T)(wpost / dA);
    L.wO_post = (T)(wpost / dO);
    L.wD_post = (T)(wpost / dD);
    // the coarsest level only needs its inverse, unless it is also the finest (its product
    // then gives the outer residual)
    if (L.k == H->kc && i != 0) continue;
    TPC_TRY(dalloc(H, &L.p, L.N));
    TPC_TRY(dalloc(H, &L.q, L.N));
    TPC_TRY(dalloc(H, &L.xi, L.N));
    TPC_TRY(dalloc(H, &L.zeta, L.N));
    TPC_TRY(upload<T>(H, L.p, F.p));
    TPC_TRY(upload<T>(H, L.q, F.q));
    TPC_TRY(upload<T>(H, L.xi, F.xi));
    TPC_TRY(upload<T>(H, L.zeta, F.zeta));
    L.nq = support2(F.q, F.zeta);
    L.np = support2(F.p, F.xi);
    if (F.has_band()) {
      const long long n = L.n;
      TPC_TRY(dalloc(H, &L.bl, n));
      TPC_TRY(dalloc(H, &L.bd, n));
      TPC_TRY(dalloc(H, &L.bu, n));
      TPC_TRY(upload<T>(H, L.bl, F.bl));
      TPC_TRY(upload<T>(H, L.bd, F.bd));
      TPC_TRY(upload<T>(H, L.bu, F.bu));
      std::vector<double> wp((size_t)n), wq((size_t)n);
      for (long long i = 0; i < n; ++i) {
        const double t = (i < F.N) ? F.tA[F.N - 1] : (i == F.N ? F.o : F.tD[F.N - 1]);
        const double aii = t + F.bd[i];
        wp[i] = H->prm.omega_pre / aii;
        wq[i] = H->prm.omega_post / aii;
      }
      TPC_TRY(dalloc(H, &L.wpre, n));
      TPC_TRY(dalloc(H, &L.wpost, n));
      TPC_TRY(upload<T>(H, L.wpre, wp));
      TPC_TRY(upload<T>(H, L.wpost, wq));
    }
    if (L.logR1 && sizeof(T) == sizeof(double)) {  // FP32 computes these (inter_tw)
      std::vector<double> twm;
      twiddles(L.m, L.m, twm);  // W_m^j, j < m
      TPC_TRY(dalloc(H, &L.twm, L.m));
      TPC_TRY(upload<T>(H, reinterpret_cast<T*>(L.twm), twm));
    }
    TPC_TRY(dalloc(H, &L.sA, L.m));
    TPC_TRY(dalloc(H, &L.sD, L.m));
    TPC_TRY(dalloc(H, &L.sB, L.m));
    if (H->prm.variant != TPC_SPD) TPC_TRY(dalloc(H, &L.sC, L.m));
  }
  TPC_TRY(dalloc(H, &G.z, max_m));
  (void)max_parts;  // the autotuner may choose down to one column per block
  TPC_TRY(dalloc(H, &G.partials, (size_t)1 << LOG_LMAX));
  const long long nc = 2 * HH.lev.back().N + 1;
  TPC_TRY(dalloc(H, &G.coarse_inv, (size_t)(nc * nc)));
  TPC_TRY(upload<T>(H, G.coarse_inv, HH.coarse_inv));
  G.f.resize(nlev);
  G.e.resize(nlev);
  G.t.resize(nlev);
  for (int i = 0; i < nlev; ++i) {
    TPC_TRY(dalloc(H, &G.f[i], G.lev[i].n));
    TPC_TRY(dalloc(H, &G.e[i], G.lev[i].n));
    TPC_TRY(dalloc(H, &G.t[i], G.lev[i].n));
  }
  return TPC_OK;
}

// The single-block bottom of the FP32 V(1,1) cycle: levels li0..(coarsest-1) all use the
// one-block plan; li0 > 0 (the level above passes its residual down).
template <typename T>
int build_bottom(tpc_handle* H, Hier<T>& G) {
  const int nlev = (int)G.lev.size();
  const int ic = nlev - 1;  // coarsest
  if (H->prm.m1 != 1 || H->prm.m2 != 1 || nlev < 3) return TPC_OK;
  int li0 = ic;
  while (li0 - 1 >= 1 && G.lev[li0 - 1].logR1 == 0) --li0;
  const int np = ic - li0;  // product levels in the bottom
  if (np < 1 || np > BOTTOM_MAX_LEVELS) return TPC_OK;
  BottomPlan<T> bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.nlev = np;
  for (int j = 0; j < np; ++j) {
    const int li = li0 + j;
    const DevLevel<T>& L = G.lev[li];
    LevelArgs<T> a = level_args<T>(G, L);
    a.pA = L.wA_pre;
    a.pO = L.wO_pre;
    a.pD = L.wD_pre;
    // descent: restriction of the finer residual + first sweep, residual
    a.pro = PRO_RESTRICT;
    a.rfine = G.t[li - 1];
    a.fout = G.f[li];
    a.xout = G.e[li];
    a.x = G.e[li];
    a.f = G.f[li];
    a.y = G.t[li];
    a.epi = EPI_RESID;
    a.wA = L.wA_pre;
    a.wO = L.wO_pre;
    a.wD = L.wD_pre;
    bp.pre[j] = a;
    // ascent: coarse correction + one post-smoothing sweep, result in t
    a.pro = PRO_PROLONG;
    a.rfine = nullptr;
    a.fout = nullptr;
    a.ec = (li + 1 == ic) ? G.e[ic] : G.t[li + 1];
    a.epi = EPI_JACOBI;
    a.wA = L.wA_post;
    a.wO = L.wO_post;
    a.wD = L.wD_post;
    a.wvec = L.wpost;
    bp.post[j] = a;
  }
  bp.cinv = G.coarse_inv;
  bp.geo = G.geo;
  bp.nc = (int)G.lev[ic].n;
  // shared-memory layout of the bottom's vectors (16-byte aligned each)
  bp.tr_elems = padded_size(1 << G.lev[li0].logm);
  long long off = 0;
  auto take = [&off](long long n) {
    const long long o = off;
    off += (n + 3) / 4 * 4;
    return (int)o;
  };
  for (int j = 0; j < np; ++j) {
    const long long n = G.lev[li0 + j].n;
    bp.off_e[j] = take(n);
    bp.off_f[j] = take(n);
    bp.off_t[j] = take(n);
  }
  bp.off_fc = take(bp.nc);
  bp.off_ec = take(bp.nc);
  const size_t smem = sizeof(c2<T>) * (size_t)(tw_slots<T>() + bp.tr_elems) + sizeof(T) * (size_t)off;
  if (smem > 150 * 1024) return TPC_OK;  // beyond the kernels' shared-memory limit: no bottom
  TPC_TRY(dalloc(H, &G.bottom, 1));
  TPC_CUDA(H, cudaMemcpyAsync(G.bottom, &bp, sizeof(bp), cudaMemcpyHostToDevice, H->stream));
  TPC_CUDA(H, cudaStreamSynchronize(H->stream));
  G.bottom_li = li0;
  G.bottom_smem = smem;
  return TPC_OK;
}

std::mutex g_tune_mu;
// (sizeof(T), log2 m) -> the chosen factorisation and tile width, shared by every handle of
// the process so that a solve alone, in a batch and in the server computes the same
struct TunedLevel {
  int logL, logC;
  bool reg;
};
std::map<std::pair<int, int>, TunedLevel> g_tuned;

// Mean time of `reps` launches of the level's product (after one warm-up), or of its two
// strided passes only (passes_only), on zeroed level buffers; < 0 on a CUDA error.
template <typename T>
float time_product(tpc_handle* H, Hier<T>& G, int li, bool passes_only, cudaEvent_t* ev) {
  const DevLevel<T>& L = G.lev[li];
  cudaStream_t s = H->stream;
  LevelArgs<T> a = level_args<T>(G, L);
  a.x = G.e[li];
  a.f = G.f[li];
  a.y = G.t[li];
  a.pro = PRO_NONE;
  a.epi = EPI_RESID;
  const bool ns = H->prm.variant != TPC_SPD;
  const int reps = 3;
  for (int rep = 0; rep <= reps; ++rep) {
    if (rep == 1) cudaEventRecord(ev[0], s);
    if constexpr (sizeof(T) == 4) {
      if (L.f32reg) {
        f32p::launch_fwd(a, L.fwd_blocks, s);
        if (!passes_only) {
          if (ns) f32p::launch_mid<true>(a, L.mid_blocks, s);
          else f32p::launch_mid<false>(a, L.mid_blocks, s);
        }
        f32p::launch_inv(a, L.fwd_blocks, s);
        continue;
      }
    }
    launch_fwd_strided<T>(a, L.fwd_blocks, L.smem_strided, s);
    if (!passes_only) {
      if (ns) launch_mid_pair<T, true>(a, L.mid_blocks, L.smem_mid, s);
      else launch_mid_pair<T, false>(a, L.mid_blocks, L.smem_mid, s);
    }
    launch_inv_strided<T>(a, L.fwd_blocks, L.smem_strided, s);
  }
  cudaEventRecord(ev[1], s);
  float t = -1.0f;
  if (cudaEventSynchronize(ev[1]) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
      cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess)
    return -1.0f;
  H->launches += 3 * (reps + 1);
  return t / reps;
}

// Set-up autotuner of the three-pass levels (tpc_params.autotune). Candidates: the
// factorisations m = R1 x L with log2 L the rule's value or one off it (2^7 <= L <= 2^12,
// 2^6 <= R1 <= 2^11) and, for the general kernels, every tile width of the strided passes
// (1 to 16 columns, tile <= 8192 entries); an FP32 factorisation the register-resident
// kernels take uses them. The width is chosen on the two strided passes, the factorisation on
// the whole product; the rule's choice stays unless another is more than 3 % faster.
template <typename T>
int autotune_levels(tpc_handle* H, Hier<T>& G, bool only_finest) {
  cudaStream_t s = H->stream;
  cudaEvent_t ev[2];
  TPC_CUDA(H, cudaEventCreate(&ev[0]));
  TPC_CUDA(H, cudaEventCreate(&ev[1]));
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int rc = TPC_OK;
  for (size_t li = 0; li < G.lev.size() && rc == TPC_OK; ++li) {
    if (only_finest && li > 0) break;
    DevLevel<T>& L = G.lev[li];
    if (L.logR1 == 0 || !L.sA) continue;
    const bool band = L.bd != nullptr;
    const std::pair<int, int> key((int)sizeof(T), L.logm);
    const auto hit = g_tuned.find(key);
    if (hit != g_tuned.end()) {
      const TunedLevel& t = hit->second;
      if (t.reg && (band || sizeof(T) != 4)) apply_split<T>(L, t.logL, -1, false);
      else apply_split<T>(L, t.logL, t.logC, t.reg);
      continue;
    }
    for (T* v : {G.e[li], G.f[li], G.t[li]})
      if (cudaMemsetAsync(v, 0, (size_t)L.n * sizeof(T), s) != cudaSuccess) rc = TPC_ECUDA;
    const int rule_logL = L.logL;
    TunedLevel best{L.logL, L.logC, L.f32reg}, rule = best;
    float best_t = -1.0f, rule_t = -1.0f;
    for (int d : {0, 1, -1}) {
      const int logL = rule_logL + d, logR1 = L.logm - logL;
      if (rc != TPC_OK) break;
      if (d != 0 && (logL < 7 || logL > LOG_LMAX || logR1 < 6 || logR1 > LOG_R1_MAX)) continue;
      const bool reg = sizeof(T) == 4 && f32p::eligible(L.logm, logR1, logL, band);
      int logC = f32p::LOG_CT;
      if (!reg) {
        // the tile width on the strided passes: the rule's unless another is 3 % faster
        apply_split<T>(L, logL, -1, false);
        const int keep = L.logC;
        float tw[5] = {-1.0f, -1.0f, -1.0f, -1.0f, -1.0f};
        for (int c = 0; c <= 4 && logR1 + c <= LOG_TILE_MAX && c <= logL; ++c) {
          apply_split<T>(L, logL, c, false);
          tw[c] = time_product<T>(H, G, li, true, ev);
          if (tw[c] < 0.0f) rc = TPC_ECUDA;
        }
        logC = keep;
        for (int c = 0; c < 5; ++c)
          if (tw[c] >= 0.0f && (tw[logC] < 0.0f || tw[c] < tw[logC])) logC = c;
        if (tw[keep] >= 0.0f && tw[keep] <= 1.03f * tw[logC]) logC = keep;
      }
      apply_split<T>(L, logL, logC, reg);
      const float t = time_product<T>(H, G, li, false, ev);
      if (t < 0.0f) {
        rc = TPC_ECUDA;
        break;
      }
      if (d == 0) {
        rule_t = t;
        rule = TunedLevel{logL, logC, reg};
      }
      if (best_t < 0.0f || t < best_t) {
        best_t = t;
        best = TunedLevel{logL, logC, reg};
      }
    }
    // the rule's factorisation (with its tuned width) unless another is more than 3 % faster
    if (rule_t >= 0.0f && best.logL != rule_logL && best_t > rule_t / 1.03f) best = rule;
    if (rc == TPC_OK) {
      apply_split<T>(L, best.logL, best.logC, best.reg);
      g_tuned[key] = TunedLevel{L.logL, L.logC, L.f32reg};
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc != TPC_OK) return cuda_fail(H, cudaGetLastError(), "autotune");
  return TPC_OK;
}

int setup_device(tpc_handle* H) {
  NvtxScope range("tpc_setup: device levels, spectra, autotune, graphs");
  const HostHierarchy& HH = H->host;
  const int nlev = (int)HH.lev.size();
  const bool mixed = H->prm.precision == TPC_MIXED;
  cudaError_t ae;
  if ((ae = set_smem_attrs<double, false>()) != cudaSuccess) return cuda_fail(H, ae, "cudaFuncSetAttribute");
  if ((ae = set_smem_attrs<double, true>()) != cudaSuccess) return cuda_fail(H, ae, "cudaFuncSetAttribute");
  if ((ae = set_smem_attrs<float, false>()) != cudaSuccess) return cuda_fail(H, ae, "cudaFuncSetAttribute");
  if ((ae = set_smem_attrs<float, true>()) != cudaSuccess) return cuda_fail(H, ae, "cudaFuncSetAttribute");
  TPC_TRY(alloc_levels<double>(H, H->d));
  if (mixed) {
    TPC_TRY(alloc_levels<float>(H, H->s));
    TPC_TRY(build_bottom<float>(H, H->s));
  }
  double* staging = nullptr;
  TPC_TRY(dalloc(H, &staging, (size_t)H->d.lev[0].m));
  // spectra of the Toeplitz blocks, divided by 2m (the 1/m of the inverse transform and the
  // 1/2 of the two-real-in-one-complex unpacking); FP32 copies are the FP64 values rounded
  std::vector<double> col;
  for (int i = 0; i < nlev; ++i) {
    const LevelForm& F = HH.lev[i];
    DevLevel<double>& L = H->d.lev[i];
    if (!L.sA) continue;
    const double scale = 1.0 / (2.0 * (double)L.m);
    const int g = (int)((L.m + 255) / 256);
    const std::vector<double>* gens[4] = {&F.tA, &F.tB, &F.tC, &F.tD};
    for (int blk = 0; blk < 4; ++blk) {
      if (blk == 2 && !L.sC) continue;
      circulant_column(*gens[blk], L.N, L.m, col);
      TPC_CUDA(H, cudaMemcpyAsync(staging, col.data(), L.m * sizeof(double),
                                  cudaMemcpyHostToDevice, H->stream));
      TPC_TRY(forward_real(H, H->d, L, staging));
      if (blk == 0) k_extract_real<double><<<g, 256, 0, H->stream>>>(H->d.z, L.sA, L.m, scale);
      if (blk == 3) k_extract_real<double><<<g, 256, 0, H->stream>>>(H->d.z, L.sD, L.m, scale);
      if (blk == 1) k_extract_cplx<double><<<g, 256, 0, H->stream>>>(H->d.z, L.sB, L.m, scale);
      if (blk == 2) k_extract_cplx<double><<<g, 256, 0, H->stream>>>(H->d.z, L.sC, L.m, scale);
      H->launches += 1;
      TPC_CUDA(H, cudaGetLastError());
      TPC_CUDA(H, cudaStreamSynchronize(H->stream));  // col is reused
    }
    if (mixed) {
      DevLevel<float>& Ls = H->s.lev[i];
      const int g2 = (int)((2 * L.m + 255) / 256);
      k_round_f32<<<g, 256, 0, H->stream>>>(L.sA, Ls.sA, L.m);
      k_round_f32<<<g, 256, 0, H->stream>>>(L.sD, Ls.sD, L.m);
      k_round_f32<<<g2, 256, 0, H->stream>>>(reinterpret_cast<const double*>(L.sB),
                                             reinterpret_cast<float*>(Ls.sB), 2 * L.m);
      H->launches += 3;
      if (L.sC) {
        k_round_f32<<<g2, 256, 0, H->stream>>>(reinterpret_cast<const double*>(L.sC),
                                               reinterpret_cast<float*>(Ls.sC), 2 * L.m);
        H->launches += 1;
      }
      TPC_CUDA(H, cudaGetLastError());
    }
  }
  if (H->prm.autotune) {
    NvtxScope tune("tpc_setup: autotune");
    if (mixed) {
      TPC_TRY(autotune_levels<float>(H, H->s, false));
      TPC_TRY(autotune_levels<double>(H, H->d, true));
    } else {
      TPC_TRY(autotune_levels<double>(H, H->d, false));
    }
  }
  TPC_TRY(setup_box(H));
  const long long nK = H->d.lev[0].n;
  TPC_TRY(dalloc(H, &H->u, nK));
  TPC_TRY(dalloc(H, &H->b, nK));
  TPC_TRY(dalloc(H, &H->r0, nK));
  if (mixed) {
    TPC_TRY(dalloc(H, &H->res32, nK));
    TPC_TRY(dalloc(H, &H->acc32, nK));
  }
  if (H->prm.outer == TPC_OUTER_FGMRES) {
    const int S = H->prm.inner_cycles;
    H->kld = (nK + 63) / 64 * 64;
    if (mixed) {
      TPC_TRY(dalloc(H, &H->kv32, (size_t)(S + 1) * H->kld));
      TPC_TRY(dalloc(H, &H->kz32, (size_t)S * H->kld));
    } else {
      TPC_TRY(dalloc(H, &H->kv64, (size_t)(S + 1) * H->kld));
      TPC_TRY(dalloc(H, &H->kz64, (size_t)S * H->kld));
    }
    TPC_TRY(dalloc(H, &H->ks, 1));
    TPC_TRY(dalloc(H, &H->kpart, (size_t)(krylov::MAXS + 1) * krylov::KNB));
  }
  TPC_TRY(dalloc(H, &H->sumsq_part, NORM_BLOCKS));
  TPC_TRY(dalloc(H, &H->sumsq, 1));
  TPC_CUDA(H, cudaMallocHost(&H->sumsq_host, sizeof(double)));
  TPC_CUDA(H, cudaEventCreateWithFlags(&H->ev, cudaEventDisableTiming));
  TPC_CUDA(H, cudaStreamSynchronize(H->stream));
  // every count the solve may choose, so that solves allocate nothing
  NvtxScope graphs("tpc_setup: iteration graphs");
  for (int c = 1; c <= full_cycles(H); ++c) TPC_TRY(iter_graph(H, c));
  return TPC_OK;
}

void release(tpc_handle* H) {
  if (!H) return;
  for (cudaGraphExec_t g : H->iter_exec)
    if (g) cudaGraphExecDestroy(g);
  if (H->stream) cudaStreamSynchronize(H->stream);
  if (H->ev) cudaEventDestroy(H->ev);
  for (void* p : H->dev_allocs) cudaFreeAsync(p, H->stream);
  if (H->stream) cudaStreamSynchronize(H->stream);
  if (H->sumsq_host) cudaFreeHost(H->sumsq_host);
  if (H->own_stream && H->stream) cudaStreamDestroy(H->stream);
  (void)cudaGetLastError();
  delete H;
}

int level_index(const tpc_handle* H, int level) {
  if (!H || level < H->kc || level > H->K) return -1;
  return H->K - level;
}

// One solve as a small state machine, so that tpc_solve (one instance) and tpc_solve_batch
// (several instances, each on its handle's stream, serviced round-robin) run the same steps:
//   begin:   b copied in, u = 0 (or x0), r = b - A u, ||r||^2 read back asynchronously;
//   step:    after the read-back arrives: test the stopping rule, else launch one iteration
//            graph and read ||r||^2 back again;
//   finish:  u copied to x.
struct SolveState {
  tpc_handle* H = nullptr;
  double* x_dev = nullptr;
  double tol = 0.0, r0 = 0.0, rel = 0.0;
  double rel_prev = 0.0;  // relative residual before the latest iteration
  int cycles = 0;         // inner cycles of the latest iteration
  int it = 0, status = TPC_OK;
  bool started = false, done = false;
  nvtxRangeId_t iter_range = 0;  // NVTX range of the iteration in flight (0: none)
};

// Inner FP32 cycles of the next mixed-precision iteration: the full count first; then the
// fewest that reach tol / 4 if the residual keeps falling at the rate per cycle observed in
// the previous iteration (the FP64 residuals measure it; a rate slowed by FP32 rounding only
// asks for more cycles). Fewer cycles in the last iteration save whole V-cycles; a miss costs
// one more iteration. FP64 solves of the stationary iteration run one V-cycle per iteration;
// FGMRES restart cycles (either precision) take their step counts by the same rule.
int next_cycles(const SolveState& st) {
  const int full = full_cycles(st.H);
  if (full <= 1 || st.it == 0 || st.cycles < 1) return full;
  const double red = st.rel / st.rel_prev;
  if (!(red > 0.0 && red < 1.0)) return full;
  const double rho = std::pow(red, 1.0 / st.cycles);
  const double need = st.tol / (4.0 * st.rel);
  if (!(rho > 0.0 && rho < 1.0) || !(need > 0.0 && need < 1.0)) return full;
  const double c = std::ceil(std::log(need) / std::log(rho));
  return c < 1.0 ? 1 : (c > full ? full : (int)c);
}

int solve_begin(SolveState& st, const double* b_dev, double* x_dev, double tol, int use_x0) {
  tpc_handle* H = st.H;
  const long long n = H->d.lev[0].n;
  const size_t bytes = (size_t)n * sizeof(double);
  cudaStream_t s = H->stream;
  st.x_dev = x_dev;
  st.tol = tol;
  st.it = 0;
  st.status = TPC_OK;
  st.started = false;
  st.done = false;
  H->last_cycles = 0;
  TPC_CUDA(H, cudaMemcpyAsync(H->b, b_dev, bytes, cudaMemcpyDeviceToDevice, s));
  if (use_x0) {
    TPC_CUDA(H, cudaMemcpyAsync(H->u, x_dev, bytes, cudaMemcpyDeviceToDevice, s));
    enqueue_finest_residual(H, H->u, H->b, H->r0);
  } else {
    TPC_CUDA(H, cudaMemsetAsync(H->u, 0, bytes, s));
    TPC_CUDA(H, cudaMemcpyAsync(H->r0, H->b, bytes, cudaMemcpyDeviceToDevice, s));
  }
  enqueue_sumsq(H, H->r0, n);
  TPC_CUDA(H, cudaGetLastError());
  TPC_CUDA(H, cudaMemcpyAsync(H->sumsq_host, H->sumsq, sizeof(double), cudaMemcpyDeviceToHost, s));
  TPC_CUDA(H, cudaEventRecord(H->ev, s));
  return TPC_OK;
}

// Call when H->ev has completed. Decides and, if the solve goes on, enqueues one iteration.
int solve_step(SolveState& st) {
  tpc_handle* H = st.H;
  if (st.iter_range) {
    nvtxRangeEnd(st.iter_range);
    st.iter_range = 0;
  }
  cudaStream_t s = H->stream;
  const double ss = *H->sumsq_host;
  if (!st.started) {
    st.started = true;
    st.r0 = std::sqrt(ss);
    st.rel = (st.r0 > 0.0) ? 1.0 : 0.0;
    if (!std::isfinite(st.r0)) {
      H->err = "right-hand side or initial residual is not finite";
      st.status = TPC_EINVAL;
      st.done = true;
      return TPC_OK;
    }
  } else {
    ++st.it;
    st.rel = std::sqrt(ss) / st.r0;
    if (!std::isfinite(st.rel)) {
      H->err = "residual became non-finite";
      st.status = TPC_EDIVERGED;
      st.done = true;
      return TPC_OK;
    }
  }
  if (!(st.rel >= st.tol && st.r0 > 0.0)) {
    st.done = true;
    return TPC_OK;
  }
  if (st.it >= H->prm.max_iters) {
    st.status = TPC_ENOTCONV;
    st.done = true;
    return TPC_OK;
  }
  const int c = next_cycles(st);
  if (!H->iter_exec[c]) return TPC_EINVAL;  // every count 1..full is captured at set-up
  st.rel_prev = st.rel;
  st.cycles = c;
  nvtxEventAttributes_t ea{};
  ea.version = NVTX_VERSION;
  ea.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  ea.messageType = NVTX_MESSAGE_TYPE_ASCII;
  ea.message.ascii = "tpc outer iteration (payload: inner cycles)";
  ea.payloadType = NVTX_PAYLOAD_TYPE_INT32;
  ea.payload.iValue = c;
  st.iter_range = nvtxRangeStartEx(&ea);
  TPC_CUDA(H, cudaGraphLaunch(H->iter_exec[c], s));
  H->launches += H->iter_nodes[c];
  H->last_cycles += c;
  TPC_CUDA(H, cudaMemcpyAsync(H->sumsq_host, H->sumsq, sizeof(double), cudaMemcpyDeviceToHost, s));
  TPC_CUDA(H, cudaEventRecord(H->ev, s));
  return TPC_OK;
}

int solve_finish(SolveState& st) {
  tpc_handle* H = st.H;
  if (st.iter_range) {
    nvtxRangeEnd(st.iter_range);
    st.iter_range = 0;
  }
  const size_t bytes = (size_t)H->d.lev[0].n * sizeof(double);
  if (st.status != TPC_EINVAL)
    TPC_CUDA(H, cudaMemcpyAsync(st.x_dev, H->u, bytes, cudaMemcpyDeviceToDevice, H->stream));
  return TPC_OK;
}

int solve_impl(tpc_handle* H, const double* b_dev, double* x_dev, double tol, int use_x0,
               int* iters_out, double* relres_out) {
  NvtxScope range("tpc_solve");
  SolveState st;
  st.H = H;
  TPC_TRY(solve_begin(st, b_dev, x_dev, tol, use_x0));
  while (!st.done) {
    TPC_CUDA(H, cudaEventSynchronize(H->ev));
    TPC_TRY(solve_step(st));
  }
  TPC_TRY(solve_finish(st));
  TPC_CUDA(H, cudaStreamSynchronize(H->stream));
  if (iters_out) *iters_out = st.it;
  if (relres_out) *relres_out = st.rel;
  return st.status;
}

template <typename T>
int apply_impl(tpc_handle* H, Hier<T>& G, int level, const T* x_dev, T* y_dev) {
  const int li = level_index(H, level);
  if (li < 0 || !x_dev || !y_dev || (const void*)x_dev == (const void*)y_dev) {
    H->err = "bad argument to tpc_apply";
    return TPC_EINVAL;
  }
  if (G.lev.empty() || !G.lev[li].sA) {
    H->err = "no product on this level (the coarsest level is held as an inverse, or the "
             "FP32 hierarchy was not built)";
    return TPC_EINVAL;
  }
  matvec<T>(H, G, li, x_dev, nullptr, y_dev, EPI_APPLY, false);
  TPC_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

}  // namespace

// Asynchronous solve with host buffers, driven by polling (used by the request server):
// the right-hand side is copied to the handle's staging buffer, the solve runs as in
// tpc_solve, and the solution is copied back into the caller's host buffer.
namespace tpc {
struct AsyncSolve {
  SolveState st;
  double* x_host = nullptr;
  bool copying_out = false;
  bool complete = false;
};

int async_begin_host(tpc_handle* H, const double* b_host, double* x_host, double tol,
                     AsyncSolve** out) {
  const long long n = H->d.lev[0].n;
  const size_t bytes = (size_t)n * sizeof(double);
  if (!H->hb) {
    TPC_TRY(dalloc(H, &H->hb, n));
    TPC_TRY(dalloc(H, &H->hx, n));
  }
  AsyncSolve* a = new (std::nothrow) AsyncSolve();
  if (!a) return TPC_ENOMEM;
  a->st.H = H;
  a->x_host = x_host;
  cudaError_t e = cudaMemcpyAsync(H->hb, b_host, bytes, cudaMemcpyHostToDevice, H->stream);
  if (e != cudaSuccess) {
    delete a;
    return cuda_fail(H, e, "cudaMemcpyAsync");
  }
  const int rc = solve_begin(a->st, H->hb, H->hx, tol, 0);
  if (rc != TPC_OK) {
    delete a;
    return rc;
  }
  *out = a;
  return TPC_OK;
}

// Non-blocking: advances the solve if its last read-back arrived. *done = 1 once the
// solution is in the caller's host buffer.
int async_poll(AsyncSolve* a, int* done) {
  tpc_handle* H = a->st.H;
  *done = 0;
  if (a->complete) {
    *done = 1;
    return TPC_OK;
  }
  const cudaError_t q = cudaEventQuery(H->ev);
  if (q == cudaErrorNotReady) return TPC_OK;
  if (q != cudaSuccess) return cuda_fail(H, q, "cudaEventQuery");
  if (a->copying_out) {
    a->complete = true;
    *done = 1;
    return TPC_OK;
  }
  TPC_TRY(solve_step(a->st));
  if (a->st.done) {
    TPC_TRY(solve_finish(a->st));
    const size_t bytes = (size_t)H->d.lev[0].n * sizeof(double);
    if (a->st.status != TPC_EINVAL)
      TPC_CUDA(H, cudaMemcpyAsync(a->x_host, H->hx, bytes, cudaMemcpyDeviceToHost, H->stream));
    TPC_CUDA(H, cudaEventRecord(H->ev, H->stream));
    a->copying_out = true;
  }
  return TPC_OK;
}

void async_result(const AsyncSolve* a, int* status, int* iters, double* relres) {
  *status = a->st.status;
  *iters = a->st.it;
  *relres = a->st.rel;
}

void async_free(AsyncSolve* a) { delete a; }

size_t handle_device_bytes(const tpc_handle* H) { return H ? H->dev_bytes : 0; }

}  // namespace tpc

// Times the three transform kernels of one level (residual epilogue), reps launches each after
// one warm-up launch, with CUDA events on the handle's stream.
template <typename T>
int time_level(tpc_handle* H, const Hier<T>& G, int level, int reps, const T* x_dev,
               const T* f_dev, T* y_dev, double* ms_out) {
  const int li = level_index(H, level);
  if (li < 0 || reps < 1 || !x_dev || !f_dev || !y_dev || !ms_out || x_dev == y_dev ||
      (int)G.lev.size() <= li || !G.lev[li].sA) {
    H->err = "bad argument to tpc_time_level_kernels";
    return TPC_EINVAL;
  }
  const DevLevel<T>& L = G.lev[li];
  const bool ns = H->prm.variant != TPC_SPD;
  LevelArgs<T> a = level_args<T>(G, L);
  a.x = x_dev;
  a.f = f_dev;
  a.y = y_dev;
  a.epi = EPI_RESID;
  const int nt = fft_threads<T>();
  cudaStream_t s = H->stream;
  cudaEvent_t ev[2];
  TPC_CUDA(H, cudaEventCreate(&ev[0]));
  TPC_CUDA(H, cudaEventCreate(&ev[1]));
  for (int which = 0; which < 3; ++which) {
    ms_out[which] = 0.0;
    if (L.logR1 == 0 && which != 1) continue;
    for (int rep = 0; rep <= reps; ++rep) {
      if (rep == 1) cudaEventRecord(ev[0], s);
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (L.f32reg) {
          if (which == 0) f32p::launch_fwd(a, L.fwd_blocks, s);
          else if (which == 2) f32p::launch_inv(a, L.fwd_blocks, s);
          else if (ns) f32p::launch_mid<true>(a, L.mid_blocks, s);
          else f32p::launch_mid<false>(a, L.mid_blocks, s);
          done = true;
        }
      }
      if (done) {
      } else if (which == 0) {
        launch_fwd_strided<T>(a, L.fwd_blocks, L.smem_strided, s);
      } else if (which == 2) {
        launch_inv_strided<T>(a, L.fwd_blocks, L.smem_strided, s);
      } else if (L.logR1 == 0) {
        if (ns) k_mid_whole<T, true><<<1, nt, L.smem_mid, s>>>(a);
        else k_mid_whole<T, false><<<1, nt, L.smem_mid, s>>>(a);
      } else {
        if (ns) launch_mid_pair<T, true>(a, L.mid_blocks, L.smem_mid, s);
        else launch_mid_pair<T, false>(a, L.mid_blocks, L.smem_mid, s);
      }
      H->launches += 1;
    }
    cudaEventRecord(ev[1], s);
    TPC_CUDA(H, cudaEventSynchronize(ev[1]));
    float ms = 0.0f;
    TPC_CUDA(H, cudaEventElapsedTime(&ms, ev[0], ev[1]));
    ms_out[which] = (double)ms / reps;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  TPC_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

extern "C" {

int tpc_setup(const tpc_params* p, double delta, double h, int levels, void* cuda_stream,
              tpc_handle** out) {
  if (!out || !p) {
    set_host_error("NULL argument");
    return TPC_EINVAL;
  }
  *out = nullptr;
  if (p->precision != TPC_FP64 && p->precision != TPC_MIXED) {
    set_host_error("precision must be TPC_FP64 or TPC_MIXED");
    return TPC_EINVAL;
  }
  if ((p->precision == TPC_MIXED || p->outer == TPC_OUTER_FGMRES) &&
      (p->inner_cycles < 1 || p->inner_cycles > 32)) {
    set_host_error("inner_cycles must be in 1..32");
    return TPC_EINVAL;
  }
  tpc_handle* H = new (std::nothrow) tpc_handle();
  if (!H) {
    set_host_error("host allocation failed");
    return TPC_ENOMEM;
  }
  H->prm = *p;
  if (H->prm.max_iters < 0) H->prm.max_iters = 0;
  std::string err;
  int rc;
  {
    NvtxScope range("tpc_setup: host hierarchy");
    rc = build_host_hierarchy(*p, delta, h, levels, H->host, err);
  }
  if (rc != TPC_OK) {
    set_host_error(err);
    delete H;
    return rc;
  }
  H->K = H->host.K;
  H->kc = H->host.kc;
  H->r = H->host.r;
  H->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev_count = 0;
  cudaError_t ce = cudaGetDeviceCount(&dev_count);
  if (ce != cudaSuccess || dev_count == 0) {
    (void)cudaGetLastError();
    set_host_error(std::string("no CUDA device: ") + cudaGetErrorString(ce));
    delete H;
    return TPC_ECUDA;
  }
  if (!H->stream) {
    // Work is captured into CUDA graphs, which the legacy default stream does not allow; a
    // blocking stream keeps the default stream's ordering with the caller's other work.
    ce = cudaStreamCreate(&H->stream);
    if (ce != cudaSuccess) {
      set_host_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(ce));
      delete H;
      return TPC_ECUDA;
    }
    H->own_stream = true;
  }
  rc = setup_device(H);
  if (rc != TPC_OK) {
    set_host_error(H->err);
    release(H);
    return rc;
  }
  *out = H;
  return TPC_OK;
}

int tpc_solve(tpc_handle* H, const double* b_dev, double* x_dev, double tol, int use_x0,
              int* iters_out, double* relres_out) {
  if (!H || !b_dev || !x_dev || !(tol >= 0.0)) {
    if (H) H->err = "bad argument to tpc_solve";
    return TPC_EINVAL;
  }
  return solve_impl(H, b_dev, x_dev, tol, use_x0, iters_out, relres_out);
}

int tpc_bdf4_step(tpc_handle* H, const double* u1, const double* u2, const double* u3,
                  const double* u4, double hist_scale, const double* g, double g_scale,
                  double tol, double* u_out, int* iters_out, double* relres_out) {
  if (!H || !u1 || !u2 || !u3 || !u4 || !u_out || !(tol >= 0.0) || !std::isfinite(hist_scale) ||
      !std::isfinite(g_scale)) {
    if (H) H->err = "bad argument to tpc_bdf4_step";
    return TPC_EINVAL;
  }
  const long long n = H->d.lev[0].n;
  cudaStream_t s = H->stream;
  // the right-hand side goes to the residual buffer, which the solve copies before reuse
  k_bdf4_rhs<<<grid_for(n), NTHREADS, 0, s>>>(H->r0, u1, u2, u3, u4, hist_scale, g, g_scale, n);
  H->launches += 1;
  TPC_CUDA(H, cudaGetLastError());
  if (u_out != u1)  // initial guess: the previous level
    TPC_CUDA(H, cudaMemcpyAsync(u_out, u1, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return solve_impl(H, H->r0, u_out, tol, 1, iters_out, relres_out);
}

int tpc_solve_batch(tpc_handle* const* hs, int count, const double* const* b_dev,
                    double* const* x_dev, double tol, int* iters_out, double* relres_out,
                    int* status_out) {
  if (count < 0 || (count > 0 && (!hs || !b_dev || !x_dev)) || !(tol >= 0.0)) {
    set_host_error("bad argument to tpc_solve_batch");
    return TPC_EINVAL;
  }
  std::vector<tpc_handle*> sorted(hs, hs + count);
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b_dev[i] || !x_dev[i]) {
      set_host_error("tpc_solve_batch: NULL handle or vector");
      return TPC_EINVAL;
    }
  }
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    set_host_error("tpc_solve_batch: a handle appears twice (each instance needs its own)");
    return TPC_EINVAL;
  }
  NvtxScope range("tpc_solve_batch");
  std::vector<SolveState> st(count);
  for (int i = 0; i < count; ++i) {
    st[i].H = hs[i];
    const int rc = solve_begin(st[i], b_dev[i], x_dev[i], tol, 0);
    if (rc != TPC_OK) {
      set_host_error(hs[i]->err);
      return rc;
    }
  }
  int active = count;
  while (active > 0) {
    for (int i = 0; i < count; ++i) {
      if (st[i].done) continue;
      tpc_handle* H = st[i].H;
      TPC_CUDA(H, cudaEventSynchronize(H->ev));
      const int rc = solve_step(st[i]);
      if (rc != TPC_OK) {
        set_host_error(H->err);
        return rc;
      }
      if (st[i].done) {
        TPC_TRY(solve_finish(st[i]));
        --active;
      }
    }
  }
  int worst = TPC_OK;
  for (int i = 0; i < count; ++i) {
    tpc_handle* H = st[i].H;
    TPC_CUDA(H, cudaStreamSynchronize(H->stream));
    if (iters_out) iters_out[i] = st[i].it;
    if (relres_out) relres_out[i] = st[i].rel;
    if (status_out) status_out[i] = st[i].status;
    if (st[i].status < worst || (worst == TPC_OK && st[i].status != TPC_OK)) worst = st[i].status;
  }
  return worst;
}

int tpc_solve_host(tpc_handle* H, const double* b_host, double* x_host, double tol, int use_x0,
                   int* iters_out, double* relres_out) {
  NvtxScope range("tpc_solve_host");
  if (!H || !b_host || !x_host || !(tol >= 0.0)) {
    if (H) H->err = "bad argument to tpc_solve_host";
    return TPC_EINVAL;
  }
  const long long n = H->d.lev[0].n;
  const size_t bytes = (size_t)n * sizeof(double);
  if (!H->hb) {
    TPC_TRY(dalloc(H, &H->hb, n));
    TPC_TRY(dalloc(H, &H->hx, n));
  }
  TPC_CUDA(H, cudaMemcpyAsync(H->hb, b_host, bytes, cudaMemcpyHostToDevice, H->stream));
  if (use_x0) TPC_CUDA(H, cudaMemcpyAsync(H->hx, x_host, bytes, cudaMemcpyHostToDevice, H->stream));
  const int rc = solve_impl(H, H->hb, H->hx, tol, use_x0, iters_out, relres_out);
  if (rc < 0) return rc;
  TPC_CUDA(H, cudaMemcpyAsync(x_host, H->hx, bytes, cudaMemcpyDeviceToHost, H->stream));
  TPC_CUDA(H, cudaStreamSynchronize(H->stream));
  return rc;
}

int tpc_apply(tpc_handle* H, int level, const double* x_dev, double* y_dev) {
  if (!H) return TPC_EINVAL;
  return apply_impl<double>(H, H->d, level, x_dev, y_dev);
}

int tpc_apply_f32(tpc_handle* H, int level, const float* x_dev, float* y_dev) {
  if (!H) return TPC_EINVAL;
  return apply_impl<float>(H, H->s, level, x_dev, y_dev);
}

int tpc_vcycle(tpc_handle* H, const double* r_dev, double* e_dev) {
  if (!H || !r_dev || !e_dev || r_dev == e_dev) {
    if (H) H->err = "bad argument to tpc_vcycle";
    return TPC_EINVAL;
  }
  const double* res = enqueue_vcycle<double>(H, H->d, 0, r_dev, nullptr);
  TPC_CUDA(H, cudaMemcpyAsync(e_dev, res, (size_t)H->d.lev[0].n * sizeof(double),
                              cudaMemcpyDeviceToDevice, H->stream));
  TPC_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

long long tpc_level_size(const tpc_handle* H, int level) {
  const int li = level_index(H, level);
  return li < 0 ? 0 : H->d.lev[li].n;
}
int tpc_finest_level(const tpc_handle* H) { return H ? H->K : -1; }
int tpc_coarsest_level(const tpc_handle* H) { return H ? H->kc : -1; }

int tpc_export_level(const tpc_handle* H, int level, double* host_buf, size_t cap,
                     size_t* need) {
  const int li = level_index(H, level);
  if (li < 0 || !need) return TPC_EINVAL;
  const LevelForm& F = H->host.lev[li];
  *need = export_count(F.N);
  if (!host_buf) return TPC_OK;
  if (cap < *need) return TPC_EINVAL;
  export_level(F, host_buf);
  return TPC_OK;
}

int tpc_tune_get(int word, int logm, int* logL, int* logC, int* reg) {
  if ((word != 4 && word != 8) || !logL || !logC || !reg) return TPC_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto hit = g_tuned.find(std::make_pair(word, logm));
  if (hit == g_tuned.end()) return 0;
  *logL = hit->second.logL;
  *logC = hit->second.logC;
  *reg = hit->second.reg ? 1 : 0;
  return 1;
}

int tpc_tune_set(int word, int logm, int logL, int logC, int reg) {
  const int logR1 = logm - logL;
  if ((word != 4 && word != 8) || logm < 13 || logm > 23 || logL < 7 || logL > LOG_LMAX ||
      logR1 < 6 || logR1 > LOG_R1_MAX || (reg != 0 && reg != 1)) {
    set_host_error("tpc_tune_set: factorisation out of range");
    return TPC_EINVAL;
  }
  if (reg) {
    if (word != 4 || !f32p::eligible(logm, logR1, logL, false)) {
      set_host_error("tpc_tune_set: the register-resident kernels do not take this factorisation");
      return TPC_EINVAL;
    }
    logC = f32p::LOG_CT;
  } else if (logC < 0 || logC > 4 || logR1 + logC > LOG_TILE_MAX || logC > logL) {
    set_host_error("tpc_tune_set: tile width out of range");
    return TPC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[std::make_pair(word, logm)] = TunedLevel{logL, logC, reg != 0};
  return TPC_OK;
}

void tpc_tune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
}

int tpc_time_level_kernels(tpc_handle* H, int level, int reps, const double* x_dev,
                           const double* f_dev, double* y_dev, double* ms_out) {
  if (!H) return TPC_EINVAL;
  return time_level<double>(H, H->d, level, reps, x_dev, f_dev, y_dev, ms_out);
}

int tpc_time_level_kernels_f32(tpc_handle* H, int level, int reps, const float* x_dev,
                               const float* f_dev, float* y_dev, double* ms_out) {
  if (!H) return TPC_EINVAL;
  return time_level<float>(H, H->s, level, reps, x_dev, f_dev, y_dev, ms_out);
}

long long tpc_kernel_launches(const tpc_handle* H) { return H ? H->launches : 0; }

int tpc_last_solve_cycles(const tpc_handle* H) { return H ? H->last_cycles : -1; }

int tpc_residual(tpc_handle* H, const double* x_dev, const double* b_dev, double* r_dev) {
  if (!H) return TPC_EINVAL;
  if (!x_dev || !b_dev || !r_dev || (const void*)r_dev == (const void*)x_dev ||
      (const void*)r_dev == (const void*)b_dev) {
    H->err = "bad argument to tpc_residual";
    return TPC_EINVAL;
  }
  enqueue_finest_residual(H, x_dev, b_dev, r_dev);
  TPC_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

int tpc_uses_box_residual(const tpc_handle* H) { return H ? (H->box_on ? 1 : 0) : -1; }

void tpc_destroy(tpc_handle* H) { release(H); }

const char* tpc_last_error(const tpc_handle* H) {
  if (H) return H->err.c_str();
  return host_error();
}

}  // extern "C"

// The 2-D system (tensor-product reading of section 2.2), built on the 1-D hierarchy above.
#include "tpc_2d.cuh"

// Stage-batched solves of many instances, built on the handles above.
#include "tpc_batch.cuh"
