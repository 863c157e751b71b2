// 2-D Toeplitz-like-plus-Cross systems: the constant kernel on the unit square with a square
// horizon [-delta, delta]^2 and tensor-product quadratic collocation (the paper defines the 1-D
// systems of section 2.2 only; this is the tensor-product reading). With the 1-D level matrix A
// and d = 12 r the finest matrix is A2 = A (x) I + I (x) A - (A (x) A) / d. The transfers are the
// section 3.1 full weighting on each axis (R (x) R, P (x) P), so every Galerkin level (eq. (3.2))
// keeps the form
//     A2_k = A_k (x) Q_k + Q_k (x) A_k - (A_k (x) A_k) / d,
// A_k the 1-D Galerkin levels (generator-plus-Cross form with spectra, eq. (3.7)) and Q_k the 1-D
// Galerkin levels of the identity, which stay tridiagonal Toeplitz on the concatenated index:
// q0' = (6 q0 + 8 q1) / 8, q1' = (q0 + 4 q1) / 8 from q0 = 1, q1 = 0.
//
// Unknowns: U[i][j] at (x_i, y_j), i, j over the 1-D unknowns [v; w_o; w_bar] of a level (n of
// them), stored row by row. For (X (x) Y) vec(U) = vec(X U Y^T) the product is
//     V = U A^T (A on every row),  T = U Q^T - V / d,   Y = A T + Q V (A, Q on every column),
// done as: batched single-block FFT products on the rows of U; one tiled transpose that forms T
// and V transposed; batched products on the rows of T^T; one tiled transpose that adds Q V and
// applies the epilogue (product, residual or damped Jacobi with the diagonal of A2_k).
//
// This file is included by tpc_api.cu (it uses the 1-D hierarchy of an internal handle).
#pragma once

namespace tpc {
namespace twod {

constexpr int LOG_M_MAX = LOG_LMAX;  // a 1-D level's product fits one block: m <= 4096

template <typename T> struct Lev2 {
  int n = 0;                 // 1-D unknowns of the level
  long long nn = 0;          // n^2
  T* f = nullptr;            // right-hand side (restricted), iterate e, scratch t
  T* e = nullptr;
  T* t = nullptr;
  T wtab[9] = {};            // pre-smoothing omega / diag(A2) by (segment of i, segment of j)
  T wpost[9] = {};
};

template <typename T> struct Hier2 {
  std::vector<Lev2<T>> lev;  // lev[li] = level K - li
  T* V = nullptr;            // work arrays of the product (nn of the finest level)
  T* Tt = nullptr;
  T* Vt = nullptr;
  T* Zt = nullptr;
  T* cinv = nullptr;         // coarsest inverse
};

// Segment of a 1-D index: 0 nodes v, 1 the middle unknown w_o, 2 midpoints w_bar.
__device__ __forceinline__ int seg(int i, int N) { return i < N ? 0 : (i == N ? 1 : 2); }

// Batched 1-D products y_row = A_k x_row over the rows of an n x n array, one row per block
// (every level here has m <= 4096, which one block transforms).
// 256 threads in both precisions (FP64: no spills at this size; two blocks per SM).
constexpr int ROW_THREADS = 256;
template <typename T, bool NS>
__global__ void __launch_bounds__(ROW_THREADS, 1) k2d_rows(LevelArgs<T> a, const T* U, T* Y,
                                                           int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<T>* tab = reinterpret_cast<c2<T>*>(smem_raw);
  c2<T>* s = tab + tw_slots<T>();
  __shared__ T red[FFT_THREADS / 32];
  __shared__ __align__(16) LevelArgs<T> la;
  const c2<T>* tw = step_table<T>(tab, a.twL);
  for (int row = blockIdx.x; row < n; row += gridDim.x) {
    if (threadIdx.x == 0) {
      la = a;
      la.x = U + (size_t)row * n;
      la.y = Y + (size_t)row * n;
    }
    __syncthreads();
    mid_core<T, MID_WHOLE, NS, 0, 0, PRO_NONE, EPI_APPLY, 2>(la, tw, s, red, 0, 0);
    __syncthreads();
  }
}

// Tt = (U Q^T - V / d)^T and Vt = V^T, 32 x 32 tiles.
template <typename T>
__global__ void __launch_bounds__(256) k2d_mid_transpose(const T* __restrict__ U,
                                                         const T* __restrict__ V, T* Tt, T* Vt,
                                                         int n, T q0, T q1, T dinv) {
  __shared__ T ts[32][33];
  __shared__ T vs[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int i = i0 + k, j = j0 + threadIdx.x;
    if (i < n && j < n) {
      const size_t o = (size_t)i * n + j;
      const T u = U[o];
      const T ul = (j > 0) ? U[o - 1] : (T)0;
      const T ur = (j + 1 < n) ? U[o + 1] : (T)0;
      const T v = V[o];
      ts[k][threadIdx.x] = fma(q0, u, fma(q1, ul + ur, -dinv * v));
      vs[k][threadIdx.x] = v;
    }
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int j = j0 + k, i = i0 + threadIdx.x;
    if (i < n && j < n) {
      const size_t o = (size_t)j * n + i;
      Tt[o] = ts[threadIdx.x][k];
      Vt[o] = vs[threadIdx.x][k];
    }
  }
}

// Y[i][j] = Zt[j][i] + (Q V)[i][j] with (Q V)[i][j] = q0 Vt[j][i] + q1 (Vt[j][i-1] + Vt[j][i+1]),
// then the epilogue: EPI_APPLY y = Y; EPI_RESID y = f - Y; EPI_JACOBI y = x + w (f - Y), w from
// the 3 x 3 table by segments.
template <typename T>
struct Wtab {
  T w[9];
};
template <typename T>
__global__ void __launch_bounds__(256) k2d_final(const T* __restrict__ Zt, const T* __restrict__ Vt,
                                                 int n, int N, T q0, T q1, int epi,
                                                 const T* __restrict__ f, const T* __restrict__ x,
                                                 T* y, Wtab<T> wt) {
  __shared__ T zs[32][33];
  __shared__ T vs[32][35];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  // transposed tiles: rows j of Zt / Vt, columns i (with a one-column halo for Vt)
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int j = j0 + k;
    if (j >= n) continue;
    const int i = i0 + threadIdx.x;
    const size_t o = (size_t)j * n;
    if (i < n) {
      zs[k][threadIdx.x] = Zt[o + i];
      vs[k][threadIdx.x + 1] = Vt[o + i];
    }
    if (threadIdx.x == 0) vs[k][0] = (i0 > 0) ? Vt[o + i0 - 1] : (T)0;
    if (threadIdx.x == 1) vs[k][33] = (i0 + 32 < n) ? Vt[o + i0 + 32] : (T)0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int i = i0 + k, j = j0 + threadIdx.x;
    if (i >= n || j >= n) continue;
    const T vm = (i + 1 < n) ? vs[threadIdx.x][k + 2] : (T)0;
    const T Y = zs[threadIdx.x][k] + fma(q0, vs[threadIdx.x][k + 1], q1 * (vs[threadIdx.x][k] + vm));
    const size_t o = (size_t)i * n + j;
    if (epi == EPI_APPLY) {
      y[o] = Y;
    } else if (epi == EPI_RESID) {
      y[o] = f[o] - Y;
    } else {
      y[o] = fma(wt.w[3 * seg(i, N) + seg(j, N)], f[o] - Y, x[o]);
    }
  }
}

// First damped Jacobi sweep from zero: e = omega D^{-1} f.
template <typename T>
__global__ void k2d_jacobi0(const T* __restrict__ f, T* e, int n, int N, Wtab<T> wt) {
  const long long nn = (long long)n * n;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nn;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o / n), j = (int)(o % n);
    e[o] = wt.w[3 * seg(i, N) + seg(j, N)] * f[o];
  }
}

// Restriction R (x) R (section 3.1 on each axis): fc[I][J] = sum_{a,b} w_a w_b rf[2I+a][2J+b],
// w = (1/4, 1/2, 1/4).
template <typename T>
__global__ void k2d_restrict(const T* __restrict__ rf, int nf, T* fc, int nc) {
  const long long ncc = (long long)nc * nc;
  const T w[3] = {(T)0.25, (T)0.5, (T)0.25};
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < ncc;
       o += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(o / nc), J = (int)(o % nc);
    T acc = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* row = rf + (size_t)(2 * I + a) * nf + 2 * J;
      acc = fma(w[a], fma(w[0], row[0], fma(w[1], row[1], w[2] * row[2])), acc);
    }
    fc[o] = acc;
  }
}

// The 1-D prolongation P = 2 R^T at fine index i: coarse indices and weights (one or two terms).
__device__ __forceinline__ int prolong_terms(int i, int nc, int* I, float* w) {
  if (i & 1) {
    I[0] = (i - 1) / 2;
    w[0] = 1.0f;
    return 1;
  }
  const int c = i / 2;
  int k = 0;
  if (c >= 1) {
    I[k] = c - 1;
    w[k++] = 0.5f;
  }
  if (c < nc) {
    I[k] = c;
    w[k++] = 0.5f;
  }
  return k;
}

// u += (P (x) P) ec.
template <typename T>
__global__ void k2d_prolong_add(T* u, const T* __restrict__ ec, int nf, int nc) {
  const long long nn = (long long)nf * nf;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nn;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o / nf), j = (int)(o % nf);
    int Ii[2], Jj[2];
    float wi[2], wj[2];
    const int ni = prolong_terms(i, nc, Ii, wi), nj = prolong_terms(j, nc, Jj, wj);
    T acc = 0;
    for (int a = 0; a < ni; ++a)
      for (int b = 0; b < nj; ++b)
        acc = fma((T)(wi[a] * wj[b]), ec[(size_t)Ii[a] * nc + Jj[b]], acc);
    u[o] += acc;
  }
}

}  // namespace twod
}  // namespace tpc

// ----------------------------------------------------------------------------------------------
// Host side: the 2-D handle, V-cycle, outer loop and the C ABI.
// ----------------------------------------------------------------------------------------------
struct tpc2d_handle {
  tpc_params prm{};
  tpc_handle* h1 = nullptr;           // 1-D hierarchy: levels A_k with spectra, FP64 (+ FP32)
  int K = 0, kc = 0;
  double d = 0.0;                     // 12 r
  std::vector<double> q0, q1;         // Q_k = tridiag(q1, q0, q1) per level index
  cudaStream_t stream = nullptr;
  tpc::twod::Hier2<double> D;
  tpc::twod::Hier2<float> S;
  double* u = nullptr;                // finest iterate, right-hand side copy, residual
  double* b = nullptr;
  double* r0 = nullptr;
  float* res32 = nullptr;             // TPC_MIXED: inner residual and accumulated correction
  float* acc32 = nullptr;
  double* sumsq_part = nullptr;
  double* sumsq = nullptr;
  double* sumsq_host = nullptr;       // pinned
  cudaGraphExec_t iter_exec[33] = {};
  cudaEvent_t ev = nullptr;
  double* hb = nullptr;               // staging buffers of solves with host buffers (on demand)
  double* hx = nullptr;
  // TPC_OUTER_FGMRES: the Krylov basis (FP32 in TPC_MIXED, else FP64), scalars, partial sums
  float* kv32 = nullptr;
  float* kz32 = nullptr;
  double* kv64 = nullptr;
  double* kz64 = nullptr;
  long long kld = 0;
  tpc::krylov::KState* ks = nullptr;
  double* kpart = nullptr;
  long long launches = 0;
  int last_cycles = 0;
  std::vector<void*> allocs;
  size_t dev_bytes = 0;               // device memory of allocs
  std::string err;
};

namespace tpc {
namespace twod {

int fail2(tpc2d_handle* H, cudaError_t e, const char* what) {
  H->err = std::string(what) + ": " + cudaGetErrorString(e);
  set_host_error(H->err);
  return TPC_ECUDA;
}

#define TPC2_CUDA(H, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return fail2(H, e_, #call);      \
  } while (0)

template <typename P>
int alloc2(tpc2d_handle* H, P** ptr, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMallocAsync(&v, count * sizeof(P) + 16, H->stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    H->err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
    set_host_error(H->err);
    return e == cudaErrorMemoryAllocation ? TPC_ENOMEM : TPC_ECUDA;
  }
  H->allocs.push_back(v);
  H->dev_bytes += count * sizeof(P) + 16;
  *ptr = reinterpret_cast<P*>(v);
  if (H->prm.poison) TPC2_CUDA(H, cudaMemsetAsync(v, 0xFF, count * sizeof(P) + 16, H->stream));
  return TPC_OK;
}

template <typename T> Hier<T>& hier1(tpc2d_handle* H);
template <> Hier<double>& hier1<double>(tpc2d_handle* H) { return H->h1->d; }
template <> Hier<float>& hier1<float>(tpc2d_handle* H) { return H->h1->s; }
template <typename T> Hier2<T>& hier2(tpc2d_handle* H);
template <> Hier2<double>& hier2<double>(tpc2d_handle* H) { return H->D; }
template <> Hier2<float>& hier2<float>(tpc2d_handle* H) { return H->S; }

template <typename T>
size_t rows_smem(const DevLevel<T>& L) {
  return sizeof(c2<T>) * (size_t)(tw_slots<T>() + padded_size(1 << L.logm));
}

// y = epilogue(A2_k x) on level index li (see k2d_final for the epilogues).
template <typename T>
void matvec2(tpc2d_handle* H, int li, const T* x, const T* f, T* y, int epi, const T* w9) {
  Hier<T>& G1 = hier1<T>(H);
  Hier2<T>& G2 = hier2<T>(H);
  const DevLevel<T>& L = G1.lev[li];
  const int n = G2.lev[li].n;
  LevelArgs<T> a = level_args<T>(G1, L);
  a.logR1 = 0;
  a.logL = L.logm;
  a.logC = 0;
  const size_t sm = rows_smem(L);
  cudaStream_t s = H->stream;
  const dim3 tg((n + 31) / 32, (n + 31) / 32), tb(32, 8);
  const T q0 = (T)H->q0[li], q1 = (T)H->q1[li];
  Wtab<T> wt{};
  if (w9)
    for (int k = 0; k < 9; ++k) wt.w[k] = w9[k];
  const bool ns = H->prm.variant != TPC_SPD;
  if (ns) k2d_rows<T, true><<<n, ROW_THREADS, sm, s>>>(a, x, G2.V, n);
  else k2d_rows<T, false><<<n, ROW_THREADS, sm, s>>>(a, x, G2.V, n);
  k2d_mid_transpose<T><<<tg, tb, 0, s>>>(x, G2.V, G2.Tt, G2.Vt, n, q0, q1, (T)(1.0 / H->d));
  if (ns) k2d_rows<T, true><<<n, ROW_THREADS, sm, s>>>(a, G2.Tt, G2.Zt, n);
  else k2d_rows<T, false><<<n, ROW_THREADS, sm, s>>>(a, G2.Tt, G2.Zt, n);
  k2d_final<T><<<tg, tb, 0, s>>>(G2.Zt, G2.Vt, n, (int)L.N, q0, q1, epi, f, x, y, wt);
  H->launches += 4;
}

int grid2(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, 4 * 152));
}

// Algorithm 2 on the 2-D level li with the right-hand side f_top (top) or the restriction of the
// finer level's residual rfine; returns the buffer holding B_k f.
template <typename T>
T* vcycle2(tpc2d_handle* H, int li, const T* f_top, const T* rfine) {
  Hier2<T>& G2 = hier2<T>(H);
  Lev2<T>& P = G2.lev[li];
  cudaStream_t s = H->stream;
  const T* f = f_top;
  if (rfine) {
    k2d_restrict<T><<<grid2(P.nn), 256, 0, s>>>(rfine, G2.lev[li - 1].n, P.f, P.n);
    H->launches += 1;
    f = P.f;
  }
  const int nlev = (int)G2.lev.size();
  if (li == nlev - 1) {
    k_coarse_solve<T><<<1, 256, 0, s>>>(G2.cinv, const_cast<T*>(f), nullptr, P.e, (int)P.nn, 0);
    H->launches += 1;
    return P.e;
  }
  const int N = (P.n - 1) / 2;
  T* e = P.e;
  T* t = P.t;
  Wtab<T> w0{};
  for (int k = 0; k < 9; ++k) w0.w[k] = P.wtab[k];
  k2d_jacobi0<T><<<grid2(P.nn), 256, 0, s>>>(f, e, P.n, N, w0);
  H->launches += 1;
  for (int l = 1; l < H->prm.m1; ++l) {
    matvec2<T>(H, li, e, f, t, EPI_JACOBI, P.wtab);
    std::swap(e, t);
  }
  matvec2<T>(H, li, e, f, t, EPI_RESID, nullptr);
  const T* ec = vcycle2<T>(H, li + 1, nullptr, t);
  k2d_prolong_add<T><<<grid2(P.nn), 256, 0, s>>>(e, ec, P.n, G2.lev[li + 1].n);
  H->launches += 1;
  for (int l = 0; l < H->prm.m2; ++l) {
    matvec2<T>(H, li, e, f, t, EPI_JACOBI, P.wpost);
    std::swap(e, t);
  }
  return e;
}

void sumsq2(tpc2d_handle* H, const double* r, long long n) {
  k_sumsq_partial<double><<<NORM_BLOCKS, NTHREADS, 0, H->stream>>>(r, n, H->sumsq_part);
  k_sumsq_final<<<1, 32, 0, H->stream>>>(H->sumsq_part, NORM_BLOCKS, H->sumsq);
  H->launches += 2;
}

// One outer iteration: FP64 u += B r, or `cycles` FP32 iterations on the scaled residual
// (as the 1-D mixed solve); then r = b - A2 u in FP64 and ||r||^2.
void iteration2(tpc2d_handle* H, int cycles) {
  const long long nn = H->D.lev[0].nn;
  const int g = grid2(nn);
  cudaStream_t s = H->stream;
  if (H->prm.outer == TPC_OUTER_FGMRES) {
    // one restart cycle of flexible GMRES, V-cycles as the preconditioner (as the 1-D solver)
    if (H->prm.precision == TPC_MIXED) {
      H->launches += fgmres_cycle<float>(
          s, nn, H->kld, H->r0, H->sumsq, H->u, H->kv32, H->kz32, H->ks, H->kpart, cycles,
          [&](const float* v) -> const float* { return vcycle2<float>(H, 0, v, nullptr); },
          [&](const float* x, float* y) { matvec2<float>(H, 0, x, nullptr, y, EPI_APPLY, nullptr); });
    } else {
      H->launches += fgmres_cycle<double>(
          s, nn, H->kld, H->r0, H->sumsq, H->u, H->kv64, H->kz64, H->ks, H->kpart, cycles,
          [&](const double* v) -> const double* { return vcycle2<double>(H, 0, v, nullptr); },
          [&](const double* x, double* y) { matvec2<double>(H, 0, x, nullptr, y, EPI_APPLY, nullptr); });
    }
  } else if (H->prm.precision == TPC_MIXED) {
    float* f32 = H->S.lev[0].f;
    k_to_f32_scaled<<<g, NTHREADS, 0, s>>>(H->r0, f32, nn, H->sumsq);
    const float* ec = vcycle2<float>(H, 0, f32, nullptr);
    k_copy<float><<<g, NTHREADS, 0, s>>>(ec, H->acc32, nn);
    H->launches += 2;
    for (int c = 1; c < cycles; ++c) {
      matvec2<float>(H, 0, H->acc32, f32, H->res32, EPI_RESID, nullptr);
      ec = vcycle2<float>(H, 0, H->res32, nullptr);
      k_axpy<float><<<g, NTHREADS, 0, s>>>(H->acc32, ec, nn);
      H->launches += 1;
    }
    k_axpy_f32_scaled<<<g, NTHREADS, 0, s>>>(H->u, H->acc32, nn, H->sumsq);
    H->launches += 1;
  } else {
    const double* e = vcycle2<double>(H, 0, H->r0, nullptr);
    k_axpy<double><<<g, NTHREADS, 0, s>>>(H->u, e, nn);
    H->launches += 1;
  }
  matvec2<double>(H, 0, H->u, H->b, H->r0, EPI_RESID, nullptr);
  sumsq2(H, H->r0, nn);
}

int graph2(tpc2d_handle* H, int cycles) {
  if (H->iter_exec[cycles]) return TPC_OK;
  cudaGraph_t graph = nullptr;
  TPC2_CUDA(H, cudaStreamBeginCapture(H->stream, cudaStreamCaptureModeThreadLocal));
  const long long before = H->launches;
  iteration2(H, cycles);
  H->launches = before;
  cudaError_t ce = cudaStreamEndCapture(H->stream, &graph);
  if (ce != cudaSuccess) return fail2(H, ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&H->iter_exec[cycles], graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    H->iter_exec[cycles] = nullptr;
    return fail2(H, ce, "cudaGraphInstantiate");
  }
  return TPC_OK;
}

template <typename T>
int alloc_hier2(tpc2d_handle* H, Hier2<T>& G) {
  const HostHierarchy& HH = H->h1->host;
  const int nlev = (int)HH.lev.size();
  G.lev.resize(nlev);
  for (int li = 0; li < nlev; ++li) {
    const LevelForm& F = HH.lev[li];
    Lev2<T>& P = G.lev[li];
    P.n = (int)(2 * F.N + 1);
    P.nn = (long long)P.n * P.n;
    TPC_TRY(alloc2(H, &P.f, (size_t)P.nn));
    TPC_TRY(alloc2(H, &P.e, (size_t)P.nn));
    TPC_TRY(alloc2(H, &P.t, (size_t)P.nn));
    const double a[3] = {F.tA[F.N - 1], F.o, F.tD[F.N - 1]};  // diagonal of A_k by segment
    for (int si = 0; si < 3; ++si)
      for (int sj = 0; sj < 3; ++sj) {
        const double dg = H->q0[li] * (a[si] + a[sj]) - a[si] * a[sj] / H->d;
        P.wtab[3 * si + sj] = (T)(H->prm.omega_pre / dg);
        P.wpost[3 * si + sj] = (T)(H->prm.omega_post / dg);
      }
  }
  const long long nn = G.lev[0].nn;
  TPC_TRY(alloc2(H, &G.V, (size_t)nn));
  TPC_TRY(alloc2(H, &G.Tt, (size_t)nn));
  TPC_TRY(alloc2(H, &G.Vt, (size_t)nn));
  TPC_TRY(alloc2(H, &G.Zt, (size_t)nn));
  std::vector<double> inv;
  const LevelForm& Fc = HH.lev.back();
  if (coarse_inverse_2d(Fc, H->q0[nlev - 1], H->q1[nlev - 1], H->d, inv) != TPC_OK) {
    H->err = "coarsest 2-D matrix is singular";
    return TPC_ESINGULAR;
  }
  TPC_TRY(alloc2(H, &G.cinv, inv.size()));
  std::vector<T> tmp(inv.begin(), inv.end());
  TPC2_CUDA(H, cudaMemcpyAsync(G.cinv, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice,
                               H->stream));
  TPC2_CUDA(H, cudaStreamSynchronize(H->stream));
  return TPC_OK;
}

template <typename T>
cudaError_t rows_attrs() {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int big = 150 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k2d_rows<T, true>, A, big);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k2d_rows<T, false>, A, big);
}

void release2(tpc2d_handle* H) {
  if (!H) return;
  for (cudaGraphExec_t g : H->iter_exec)
    if (g) cudaGraphExecDestroy(g);
  if (H->stream) cudaStreamSynchronize(H->stream);
  if (H->ev) cudaEventDestroy(H->ev);
  for (void* p : H->allocs) cudaFreeAsync(p, H->stream);
  if (H->stream) cudaStreamSynchronize(H->stream);
  if (H->sumsq_host) cudaFreeHost(H->sumsq_host);
  if (H->h1) tpc_destroy(H->h1);
  (void)cudaGetLastError();
  delete H;
}

// The outer iteration of a 2-D solve as a state machine: solve2_begin enqueues the initial
// residual norm, each solve2_step (called once the handle's event has completed) reads the
// latest norm, decides, and enqueues the next iteration's graph and norm read-back, and
// solve2_finish enqueues the copy of the iterate. tpc2d_solve drives it synchronously, the
// request server by polling.
struct Solve2State {
  tpc2d_handle* H = nullptr;
  double* x_dev = nullptr;
  double tol = 0.0, r0 = 0.0, rel = 0.0, rel_prev = 0.0;
  int it = 0, cycles = 0, status = TPC_OK;
  bool started = false, done = false;
};

int solve2_begin(Solve2State& st, const double* b_dev, double* x_dev, double tol, int use_x0) {
  tpc2d_handle* H = st.H;
  const long long nn = H->D.lev[0].nn;
  const size_t bytes = (size_t)nn * sizeof(double);
  cudaStream_t s = H->stream;
  st.x_dev = x_dev;
  st.tol = tol;
  TPC2_CUDA(H, cudaMemcpyAsync(H->b, b_dev, bytes, cudaMemcpyDeviceToDevice, s));
  if (use_x0) {
    TPC2_CUDA(H, cudaMemcpyAsync(H->u, x_dev, bytes, cudaMemcpyDeviceToDevice, s));
    matvec2<double>(H, 0, H->u, H->b, H->r0, EPI_RESID, nullptr);
  } else {
    TPC2_CUDA(H, cudaMemsetAsync(H->u, 0, bytes, s));
    TPC2_CUDA(H, cudaMemcpyAsync(H->r0, H->b, bytes, cudaMemcpyDeviceToDevice, s));
  }
  sumsq2(H, H->r0, nn);
  TPC2_CUDA(H, cudaMemcpyAsync(H->sumsq_host, H->sumsq, sizeof(double), cudaMemcpyDeviceToHost, s));
  TPC2_CUDA(H, cudaEventRecord(H->ev, s));
  H->last_cycles = 0;
  return TPC_OK;
}

int solve2_step(Solve2State& st) {
  tpc2d_handle* H = st.H;
  const double ss = *H->sumsq_host;
  if (!st.started) {
    st.started = true;
    st.r0 = std::sqrt(ss);
    st.rel = st.r0 > 0.0 ? 1.0 : 0.0;
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
  // inner cycles: the full count first, then the fewest expected to reach tol / 4 at the rate
  // per cycle measured by the previous iteration (as the 1-D mixed solve)
  const int full = (H->prm.precision == TPC_MIXED || H->prm.outer == TPC_OUTER_FGMRES)
                       ? H->prm.inner_cycles
                       : 1;
  int c = full;
  if (full > 1 && st.it > 0 && st.cycles > 0) {
    const double red = st.rel / st.rel_prev;
    const double rho = std::pow(red, 1.0 / st.cycles), need = st.tol / (4.0 * st.rel);
    if (red > 0.0 && red < 1.0 && rho > 0.0 && rho < 1.0 && need > 0.0 && need < 1.0) {
      const double cc = std::ceil(std::log(need) / std::log(rho));
      c = cc < 1.0 ? 1 : (cc > full ? full : (int)cc);
    }
  }
  cudaStream_t s = H->stream;
  TPC2_CUDA(H, cudaGraphLaunch(H->iter_exec[c], s));
  TPC2_CUDA(H, cudaMemcpyAsync(H->sumsq_host, H->sumsq, sizeof(double), cudaMemcpyDeviceToHost, s));
  TPC2_CUDA(H, cudaEventRecord(H->ev, s));
  H->last_cycles += c;
  st.rel_prev = st.rel;
  st.cycles = c;
  return TPC_OK;
}

int solve2_finish(Solve2State& st) {
  tpc2d_handle* H = st.H;
  const size_t bytes = (size_t)H->D.lev[0].nn * sizeof(double);
  TPC2_CUDA(H, cudaMemcpyAsync(st.x_dev, H->u, bytes, cudaMemcpyDeviceToDevice, H->stream));
  return TPC_OK;
}

int level_index2(const tpc2d_handle* H, int level) {
  if (!H || level < H->kc || level > H->K) return -1;
  return H->K - level;
}

}  // namespace twod
}  // namespace tpc

extern "C" {

int tpc2d_setup(const tpc_params* p, double delta, double h, void* cuda_stream,
                tpc2d_handle** out) {
  using namespace tpc::twod;
  if (!p || !out) {
    set_host_error("NULL argument");
    return TPC_EINVAL;
  }
  *out = nullptr;
  if (p->variant != TPC_SPD && p->variant != TPC_NONSYM) {
    set_host_error("the 2-D system needs variant TPC_SPD or TPC_NONSYM");
    return TPC_EINVAL;
  }
  if (p->kernel != 0 || p->transfer != TPC_TRANSFER_PAPER) {
    set_host_error("the 2-D system is built for the constant kernel and the paper's transfer");
    return TPC_ENOTSUP;
  }
  if (p->coarsest_level > 3) {
    set_host_error("the 2-D system needs coarsest_level <= 3 (dense solve of <= 225 unknowns)");
    return TPC_EINVAL;
  }
  tpc2d_handle* H = new (std::nothrow) tpc2d_handle();
  if (!H) {
    set_host_error("host allocation failed");
    return TPC_ENOMEM;
  }
  H->prm = *p;
  if (H->prm.max_iters < 0) H->prm.max_iters = 0;
  tpc_params p1 = *p;
  p1.autotune = 0;
  p1.box_residual = 0;
  p1.outer = TPC_OUTER_VCYCLE;  // the internal 1-D handle only holds the 1-D levels
  if ((p->outer != TPC_OUTER_VCYCLE && p->outer != TPC_OUTER_FGMRES) ||
      (p->outer == TPC_OUTER_FGMRES && (p->inner_cycles < 1 || p->inner_cycles > 32))) {
    set_host_error("outer must be TPC_OUTER_VCYCLE or TPC_OUTER_FGMRES (inner_cycles 1..32)");
    delete H;
    return TPC_EINVAL;
  }
  int rc = tpc_setup(&p1, delta, h, 0, cuda_stream, &H->h1);
  if (rc != TPC_OK) {
    delete H;
    return rc;
  }
  if (H->h1->K > LOG_M_MAX - 1) {
    set_host_error("the 2-D system needs h = 2^-K with K <= 11 (each axis' product in one block)");
    release2(H);
    return TPC_EINVAL;
  }
  H->stream = H->h1->stream;
  H->K = H->h1->K;
  H->kc = H->h1->kc;
  H->d = 12.0 * H->h1->r;
  const int nlev = (int)H->h1->host.lev.size();
  H->q0.assign(nlev, 1.0);
  H->q1.assign(nlev, 0.0);
  for (int li = 1; li < nlev; ++li) {  // Galerkin levels of the identity (Toeplitz rule)
    H->q0[li] = (6.0 * H->q0[li - 1] + 8.0 * H->q1[li - 1]) / 8.0;
    H->q1[li] = (H->q0[li - 1] + 4.0 * H->q1[li - 1]) / 8.0;
  }
  cudaError_t ae;
  if ((ae = rows_attrs<double>()) != cudaSuccess || (ae = rows_attrs<float>()) != cudaSuccess) {
    rc = fail2(H, ae, "cudaFuncSetAttribute");
    release2(H);
    return rc;
  }
  const bool mixed = p->precision == TPC_MIXED;
  auto setup = [&]() -> int {
    TPC_TRY(alloc_hier2<double>(H, H->D));
    if (mixed) TPC_TRY(alloc_hier2<float>(H, H->S));
    const long long nn = H->D.lev[0].nn;
    TPC_TRY(alloc2(H, &H->u, (size_t)nn));
    TPC_TRY(alloc2(H, &H->b, (size_t)nn));
    TPC_TRY(alloc2(H, &H->r0, (size_t)nn));
    if (mixed) {
      TPC_TRY(alloc2(H, &H->res32, (size_t)nn));
      TPC_TRY(alloc2(H, &H->acc32, (size_t)nn));
    }
    if (H->prm.outer == TPC_OUTER_FGMRES) {
      const int S = H->prm.inner_cycles;
      H->kld = (nn + 63) / 64 * 64;
      if (mixed) {
        TPC_TRY(alloc2(H, &H->kv32, (size_t)(S + 1) * H->kld));
        TPC_TRY(alloc2(H, &H->kz32, (size_t)S * H->kld));
      } else {
        TPC_TRY(alloc2(H, &H->kv64, (size_t)(S + 1) * H->kld));
        TPC_TRY(alloc2(H, &H->kz64, (size_t)S * H->kld));
      }
      TPC_TRY(alloc2(H, &H->ks, 1));
      TPC_TRY(alloc2(H, &H->kpart, (size_t)(tpc::krylov::MAXS + 1) * tpc::krylov::KNB));
    }
    TPC_TRY(alloc2(H, &H->sumsq_part, NORM_BLOCKS));
    TPC_TRY(alloc2(H, &H->sumsq, 1));
    TPC2_CUDA(H, cudaMallocHost(&H->sumsq_host, sizeof(double)));
    TPC2_CUDA(H, cudaEventCreateWithFlags(&H->ev, cudaEventDisableTiming));
    TPC2_CUDA(H, cudaStreamSynchronize(H->stream));
    const bool many = mixed || H->prm.outer == TPC_OUTER_FGMRES;
    for (int c = 1; c <= (many ? H->prm.inner_cycles : 1); ++c) TPC_TRY(graph2(H, c));
    return TPC_OK;
  };
  rc = setup();
  if (rc != TPC_OK) {
    set_host_error(H->err);
    release2(H);
    return rc;
  }
  *out = H;
  return TPC_OK;
}

int tpc2d_solve(tpc2d_handle* H, const double* b_dev, double* x_dev, double tol, int use_x0,
                int* iters_out, double* relres_out) {
  using namespace tpc::twod;
  if (!H || !b_dev || !x_dev || !(tol >= 0.0)) {
    if (H) H->err = "bad argument to tpc2d_solve";
    return TPC_EINVAL;
  }
  Solve2State st;
  st.H = H;
  TPC_TRY(solve2_begin(st, b_dev, x_dev, tol, use_x0));
  while (!st.done) {
    TPC2_CUDA(H, cudaEventSynchronize(H->ev));
    TPC_TRY(solve2_step(st));
  }
  if (st.status == TPC_EINVAL) return TPC_EINVAL;  // non-finite right-hand side: x untouched
  TPC_TRY(solve2_finish(st));
  TPC2_CUDA(H, cudaStreamSynchronize(H->stream));
  if (iters_out) *iters_out = st.it;
  if (relres_out) *relres_out = st.rel;
  return st.status;
}

int tpc2d_apply(tpc2d_handle* H, int level, const double* x_dev, double* y_dev) {
  using namespace tpc::twod;
  const int li = level_index2(H, level);
  if (li < 0 || !x_dev || !y_dev || (const void*)x_dev == (const void*)y_dev ||
      li == (int)H->D.lev.size() - 1) {
    if (H) H->err = "bad argument to tpc2d_apply (levels above the coarsest)";
    return TPC_EINVAL;
  }
  matvec2<double>(H, li, x_dev, nullptr, y_dev, EPI_APPLY, nullptr);
  TPC2_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

int tpc2d_apply_f32(tpc2d_handle* H, int level, const float* x_dev, float* y_dev) {
  using namespace tpc::twod;
  const int li = level_index2(H, level);
  if (li < 0 || !x_dev || !y_dev || (const void*)x_dev == (const void*)y_dev ||
      H->prm.precision != TPC_MIXED || li == (int)H->S.lev.size() - 1) {
    if (H) H->err = "bad argument to tpc2d_apply_f32 (TPC_MIXED handles, levels above the coarsest)";
    return TPC_EINVAL;
  }
  matvec2<float>(H, li, x_dev, nullptr, y_dev, EPI_APPLY, nullptr);
  TPC2_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

int tpc2d_vcycle(tpc2d_handle* H, const double* r_dev, double* e_dev) {
  using namespace tpc::twod;
  if (!H || !r_dev || !e_dev || r_dev == e_dev) {
    if (H) H->err = "bad argument to tpc2d_vcycle";
    return TPC_EINVAL;
  }
  const double* e = vcycle2<double>(H, 0, r_dev, nullptr);
  TPC2_CUDA(H, cudaMemcpyAsync(e_dev, e, (size_t)H->D.lev[0].nn * sizeof(double),
                               cudaMemcpyDeviceToDevice, H->stream));
  TPC2_CUDA(H, cudaGetLastError());
  return TPC_OK;
}

long long tpc2d_level_size(const tpc2d_handle* H, int level) {
  const int li = tpc::twod::level_index2(H, level);
  return li < 0 ? 0 : H->D.lev[li].nn;
}
int tpc2d_finest_level(const tpc2d_handle* H) { return H ? H->K : -1; }
int tpc2d_coarsest_level(const tpc2d_handle* H) { return H ? H->kc : -1; }
int tpc2d_last_solve_cycles(const tpc2d_handle* H) { return H ? H->last_cycles : -1; }
long long tpc2d_kernel_launches(const tpc2d_handle* H) { return H ? H->launches : 0; }
void tpc2d_destroy(tpc2d_handle* H) { tpc::twod::release2(H); }
const char* tpc2d_last_error(const tpc2d_handle* H) {
  if (H) return H->err.c_str();
  return tpc::host_error();
}

}  // extern "C"

// Polled 2-D solve with host buffers (the request server's 2-D requests): as async_begin_host
// and async_poll of the 1-D solver, on the state machine above.
namespace tpc {
struct AsyncSolve2 {
  twod::Solve2State st;
  double* x_host = nullptr;
  bool copying_out = false;
  bool complete = false;
};

int async2d_begin_host(tpc2d_handle* H, const double* b_host, double* x_host, double tol,
                       AsyncSolve2** out) {
  using namespace twod;
  const long long nn = H->D.lev[0].nn;
  if (!H->hb) {
    TPC_TRY(alloc2(H, &H->hb, (size_t)nn));
    TPC_TRY(alloc2(H, &H->hx, (size_t)nn));
  }
  AsyncSolve2* a = new (std::nothrow) AsyncSolve2();
  if (!a) return TPC_ENOMEM;
  a->st.H = H;
  a->x_host = x_host;
  cudaError_t e = cudaMemcpyAsync(H->hb, b_host, (size_t)nn * sizeof(double),
                                  cudaMemcpyHostToDevice, H->stream);
  if (e != cudaSuccess) {
    delete a;
    return fail2(H, e, "cudaMemcpyAsync");
  }
  const int rc = solve2_begin(a->st, H->hb, H->hx, tol, 0);
  if (rc != TPC_OK) {
    delete a;
    return rc;
  }
  *out = a;
  return TPC_OK;
}

int async2d_poll(AsyncSolve2* a, int* done) {
  using namespace twod;
  tpc2d_handle* H = a->st.H;
  *done = 0;
  if (a->complete) {
    *done = 1;
    return TPC_OK;
  }
  const cudaError_t q = cudaEventQuery(H->ev);
  if (q == cudaErrorNotReady) return TPC_OK;
  if (q != cudaSuccess) return fail2(H, q, "cudaEventQuery");
  if (a->copying_out) {
    a->complete = true;
    *done = 1;
    return TPC_OK;
  }
  TPC_TRY(solve2_step(a->st));
  if (a->st.done) {
    if (a->st.status != TPC_EINVAL) {
      TPC_TRY(solve2_finish(a->st));
      TPC2_CUDA(H, cudaMemcpyAsync(a->x_host, H->hx, (size_t)H->D.lev[0].nn * sizeof(double),
                                   cudaMemcpyDeviceToHost, H->stream));
    }
    TPC2_CUDA(H, cudaEventRecord(H->ev, H->stream));
    a->copying_out = true;
  }
  return TPC_OK;
}

void async2d_result(const AsyncSolve2* a, int* status, int* iters, double* relres) {
  *status = a->st.status;
  *iters = a->st.it;
  *relres = a->st.rel;
}

void async2d_free(AsyncSolve2* a) { delete a; }

size_t handle2d_device_bytes(const tpc2d_handle* H) {
  return H ? H->dev_bytes + handle_device_bytes(H->h1) : 0;
}

}  // namespace tpc
