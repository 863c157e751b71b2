// tpc_apply_noalloc: the Toeplitz-plus-Cross product of one level for callers that cannot
// allocate device memory.
//
// Who needs it: code that must not call cudaMalloc / cudaFree while it runs -- for example work
// recorded while a CUDA graph is being captured in a mode that forbids allocation, a plugin
// or service whose host application owns every device allocation (fixed memory pools, strict
// per-tenant budgets), or a hot path that must never synchronise the device, which
// cudaMalloc/cudaFree can do. tpc_apply needs a handle whose tpc_setup allocated the work
// arrays; this entry point takes the level's generators and Cross vectors from the caller and
// keeps all of its own work memory (transform work array, block spectra, twiddles, partial
// sums) in one file-scope static device array of fixed size.
//
// Limits and sharing rules:
//   * N = 2^k - 1 with 1 <= k <= 15, i.e. circulant length m = 2N + 2 <= 65536
//     (NOALLOC_MAX_M); larger N is rejected with TPC_EINVAL.
//   * the static array (about 5.7 MB) is held by every GPU that loads the library until the
//     process exits;
//   * all calls share it and it keeps the last call's contents: two calls whose work overlaps
//     on the GPU (different streams, or different host threads) race and corrupt each other;
//     calls must be ordered (same stream, or synchronised);
//   * the first call on a device does a one-time set-up on that device (the array's device
//     address via cudaGetSymbolAddress, shared-memory limits of the kernels) and synchronises
//     it; make that first call before any stream capture. Every call looks the address up
//     again and repeats the set-up if it changed (the device was reset and the module loaded
//     anew), and writes the 4096-point twiddle table on its own stream, so nothing of an
//     earlier context is trusted.
//   * only Toeplitz-plus-Cross levels (TPC_SPD, TPC_NONSYM): the tridiagonal band of the
//     weakly singular model (section 2.1) is not part of the generator-plus-Cross layout and
//     is not applied.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "tpc_internal.h"
#include "tpc_kernels.cuh"

namespace tpc {
void set_host_error(const std::string& s);
}

namespace {

using namespace tpc;

constexpr long long NOALLOC_MAX_M = 1LL << 16;
constexpr int NOALLOC_MAX_DEV = 64;
constexpr int NA_LOG_WHOLE = 9;     // same plan rules as the handle-based path
constexpr int NA_LOG_TILE_MAX = 13;
constexpr int NA_MAX_PARTS = 4096;

// Byte offsets inside the static array (every part 256-byte aligned).
constexpr size_t OFF_STAGE = 0;                                          // m doubles
constexpr size_t OFF_Z = OFF_STAGE + NOALLOC_MAX_M * 8;                  // m complex
constexpr size_t OFF_SA = OFF_Z + NOALLOC_MAX_M * 16;                    // m doubles
constexpr size_t OFF_SD = OFF_SA + NOALLOC_MAX_M * 8;                    // m doubles
constexpr size_t OFF_SB = OFF_SD + NOALLOC_MAX_M * 8;                    // m complex
constexpr size_t OFF_SC = OFF_SB + NOALLOC_MAX_M * 16;                   // m complex
constexpr size_t OFF_TWM = OFF_SC + NOALLOC_MAX_M * 16;                  // m complex
constexpr size_t OFF_TWL = OFF_TWM + NOALLOC_MAX_M * 16;                 // 4096 complex
constexpr size_t OFF_PART = OFF_TWL + (size_t(1) << LOG_LMAX) * 16;      // partial sums
constexpr size_t NOALLOC_BYTES = OFF_PART + NA_MAX_PARTS * 8;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Per device: the address the last set-up found (nullptr: not set up), guarded by g_mu.
unsigned char* g_dev_ptr[NOALLOC_MAX_DEV] = {nullptr};
std::mutex g_mu;

// W_n^j = exp(-2 pi i j / n), j < count (n a power of two), from sincospi.
__global__ void k_na_twiddles(double2* out, long long n, long long count) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j < count) {
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    out[j] = make_double2(c, -s);
  }
}

// Circulant first column of an N x N Toeplitz generator t (t[d + N - 1] = T(i, j), d = i - j),
// embedded in length m (eq. (3.4)); every entry is written (the zeros included).
__global__ void k_na_circulant(const double* t, long long N, long long m, double* c) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  double v = 0.0;
  if (i < N) v = t[i + N - 1];              // c[d] = t_d, 0 <= d <= N - 1
  else if (i > m - N) v = t[(i - m) + N - 1];  // c[m - d] = t_{-d}, 1 <= d <= N - 1
  c[i] = v;
}

int fail(int code, const char* msg) {
  set_host_error(msg);
  return code;
}

// The static array's device address on the current device (looked up on every call, which
// allocates nothing), and the kernels' shared-memory limits, set once per address.
int setup_device(int dev, unsigned char** base) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    (void)cudaGetLastError();
    return fail(TPC_ECUDA, "tpc_apply_noalloc: cudaGetSymbolAddress failed");
  }
  unsigned char* b = static_cast<unsigned char*>(p);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev_ptr[dev] == b) {
    *base = b;
    return TPC_OK;
  }
  const int big = 150 * 1024;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(k_fwd_strided<double, IN_PACK, PRO_NONE>, A, big) != cudaSuccess ||
      cudaFuncSetAttribute(k_fwd_strided<double, IN_REAL, PRO_NONE>, A, big) != cudaSuccess ||
      cudaFuncSetAttribute(k_mid_pair<double, true>, A, big) != cudaSuccess ||
      cudaFuncSetAttribute(k_mid_whole<double, true>, A, big) != cudaSuccess ||
      cudaFuncSetAttribute(k_mid_fwd<double>, A, big) != cudaSuccess ||
      cudaFuncSetAttribute(k_mid_fwd_real<double>, A, big) != cudaSuccess ||
      cudaFuncSetAttribute(k_inv_strided<double, EPI_APPLY>, A, big) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(TPC_ECUDA, "tpc_apply_noalloc: cudaFuncSetAttribute failed");
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(TPC_ECUDA, "tpc_apply_noalloc: device set-up failed");
  g_dev_ptr[dev] = b;
  *base = b;
  return TPC_OK;
}

}  // namespace

extern "C" int tpc_apply_noalloc(long long N, const double* tA, const double* tB,
                                 const double* tC, const double* tD, const double* p,
                                 const double* q, const double* xi, const double* zeta, double o,
                                 const double* x_dev, double* y_dev, void* cuda_stream) {
  if (!tA || !tB || !tC || !tD || !p || !q || !xi || !zeta || !x_dev || !y_dev ||
      x_dev == y_dev)
    return fail(TPC_EINVAL, "tpc_apply_noalloc: NULL or aliasing pointer");
  if (N < 1 || ((N + 1) & N) != 0)
    return fail(TPC_EINVAL, "tpc_apply_noalloc: N must be 2^k - 1");
  const long long m = 2 * N + 2;
  if (m > NOALLOC_MAX_M)
    return fail(TPC_EINVAL,
                "tpc_apply_noalloc: N too large (2N + 2 must be <= 65536, i.e. N <= 32767)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEV) {
    (void)cudaGetLastError();
    return fail(TPC_ECUDA, "tpc_apply_noalloc: no usable CUDA device");
  }
  unsigned char* base = nullptr;
  const int rc = setup_device(dev, &base);
  if (rc != TPC_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

  // plan (same rules as the handle-based path)
  int logm = 0;
  while ((1LL << logm) < m) ++logm;
  int logR1 = 0, logL = logm, logC = 0, fwd_blocks = 0, mid_blocks = 1;
  if (logm > NA_LOG_WHOLE) {
    logL = (logm + 1) / 2;
    if (logL > LOG_LMAX) logL = LOG_LMAX;
    logR1 = logm - logL;
    logC = 4;
    if (logC > NA_LOG_TILE_MAX - logR1) logC = NA_LOG_TILE_MAX - logR1;
    int want = logL - 9;
    if (want < 0) want = 0;
    if (logC > want) logC = want;
    if (logC < 0) logC = 0;
    fwd_blocks = 1 << (logL - logC);
    mid_blocks = (1 << (logm - logL - 1)) + 1;
  }
  const size_t smem_strided =
      logR1 ? sizeof(double2) * (size_t)(tw_slots<double>() + padded_size(1 << (logR1 + logC))) : 0;
  const size_t smem_mid = sizeof(double2) * (size_t)(tw_slots<double>() + padded_size(1 << (logL + (logR1 ? 1 : 0))));
  const size_t smem_fwd_blk = sizeof(double2) * (size_t)(tw_slots<double>() + padded_size(1 << logL));

  double* stage = reinterpret_cast<double*>(base + OFF_STAGE);
  double2* z = reinterpret_cast<double2*>(base + OFF_Z);
  double* sA = reinterpret_cast<double*>(base + OFF_SA);
  double* sD = reinterpret_cast<double*>(base + OFF_SD);
  double2* sB = reinterpret_cast<double2*>(base + OFF_SB);
  double2* sC = reinterpret_cast<double2*>(base + OFF_SC);
  double2* twm = reinterpret_cast<double2*>(base + OFF_TWM);
  double2* twL = reinterpret_cast<double2*>(base + OFF_TWL);
  double* parts = reinterpret_cast<double*>(base + OFF_PART);

  LevelArgs<double> a{};
  a.N = (int)N;  // N <= 32767 (checked above)
  a.logm = logm;
  a.logR1 = logR1;
  a.logL = logL;
  a.logC = logC;
  a.sA = sA;
  a.sD = sD;
  a.sB = sB;
  a.sC = sC;
  a.p = p;
  a.q = q;
  a.xi = xi;
  a.zeta = zeta;
  a.nq = (int)N;  // full support (the caller's vectors are not scanned)
  a.np = (int)N;
  a.o = o;
  a.twm = twm;
  a.twL = twL;
  a.z = z;
  a.partials = parts;
  a.nparts = fwd_blocks;
  const unsigned gm = (unsigned)((m + 255) / 256);
  const long long nl = 1LL << LOG_LMAX;
  k_na_twiddles<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(twL, nl, nl);
  if (logR1) k_na_twiddles<<<gm, 256, 0, s>>>(twm, m, m);

  // spectra of the four Toeplitz blocks, divided by 2m, in bit-reversed order
  const double scale = 1.0 / (2.0 * (double)m);
  const double* gens[4] = {tA, tB, tC, tD};
  for (int blk = 0; blk < 4; ++blk) {
    k_na_circulant<<<gm, 256, 0, s>>>(gens[blk], N, m, stage);
    a.real_in = stage;
    if (logR1 == 0) {
      k_mid_fwd_real<double><<<1, FFT_THREADS, smem_mid, s>>>(a);
    } else {
      k_fwd_strided<double, IN_REAL, PRO_NONE><<<fwd_blocks, FFT_THREADS, smem_strided, s>>>(a);
      k_mid_fwd<double><<<1 << logR1, FFT_THREADS, smem_fwd_blk, s>>>(a);
    }
    if (blk == 0) k_extract_real<double><<<gm, 256, 0, s>>>(z, sA, m, scale);
    if (blk == 1) k_extract_cplx<double><<<gm, 256, 0, s>>>(z, sB, m, scale);
    if (blk == 2) k_extract_cplx<double><<<gm, 256, 0, s>>>(z, sC, m, scale);
    if (blk == 3) k_extract_real<double><<<gm, 256, 0, s>>>(z, sD, m, scale);
  }

  // the product y = A x (eq. (3.7) and the product formula after it)
  a.real_in = nullptr;
  a.x = x_dev;
  a.y = y_dev;
  a.epi = EPI_APPLY;
  a.pro = PRO_NONE;
  if (logR1 == 0) {
    k_mid_whole<double, true><<<1, FFT_THREADS, smem_mid, s>>>(a);
  } else {
    k_fwd_strided<double, IN_PACK, PRO_NONE><<<fwd_blocks, FFT_THREADS, smem_strided, s>>>(a);
    k_mid_pair<double, true><<<mid_blocks, FFT_THREADS, smem_mid, s>>>(a);
    k_inv_strided<double, EPI_APPLY><<<fwd_blocks, FFT_THREADS, smem_strided, s>>>(a);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TPC_ECUDA, cudaGetErrorString(e));
  return TPC_OK;
}
