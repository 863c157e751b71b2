// Flexible GMRES outer iteration (tpc_params.outer = TPC_OUTER_FGMRES; not the paper's, whose
// outer iteration is the stationary u <- u + B (b - A u) of section 5).
//
// One outer iteration is one restart cycle of right-preconditioned flexible GMRES with `steps`
// steps (Saad's FGMRES): from the FP64 residual r = b - A u,
//   v_0 = r / ||r||;  for j < steps: z_j = B v_j (one V-cycle of Algorithm 2), w = A z_j,
//   classical Gram-Schmidt of w against v_0..v_j done twice, h_{j+1,j} = ||w||,
//   v_{j+1} = w / h_{j+1,j};  Givens rotations reduce the Hessenberg matrix to R and
//   beta e_1 to g;  y = R^{-1} g;  u += Z y;
// then the FP64 residual and its norm as in every outer iteration. In TPC_MIXED the vectors
// v_j, z_j, the V-cycles and the products are FP32, and so is the element-wise arithmetic on
// them (each thread's share of a dot product is summed in FP32, about a hundred terms at the
// largest sizes, the shares in FP64; the Hessenberg matrix, the rotations and y are FP64, and
// the FP32 correction sum_j y_j z_j is added to the FP64 iterate): on this GPU an FP64
// operation per element costs more than the memory traffic of the step. In TPC_FP64
// everything is FP64. The small least-squares problem lives on the device, so an outer
// iteration stays one CUDA graph.
//
// This file is included by tpc_api.cu.
#pragma once

namespace tpc {
namespace krylov {

constexpr int MAXS = 32;       // restart length limit (= the inner-cycle limit)
constexpr int LDH = MAXS + 1;  // leading dimension of the Hessenberg matrix
constexpr int KNB = 304;       // partial-sum blocks of the dot products (2 x 152 SMs)

// Scalars of one restart cycle (device memory).
struct KState {
  double R[LDH * MAXS];  // column j at R + j LDH: Hessenberg column, then rotated into R
  double cs[MAXS], sn[MAXS];
  double g[MAXS + 1];    // rotated beta e_1
  double y[MAXS];
  double h[MAXS + 1];    // coefficients of the current Gram-Schmidt pass
  double inv;            // 1 / h_{j+1,j} of the current step (0 at a breakdown)
};

// v_0 = r / ||r|| (r FP64, v_0 of type T); g = beta e_1.
template <typename T>
__global__ void k_kry_start(const double* __restrict__ r, T* __restrict__ v0, long long n,
                            const double* __restrict__ sumsq, KState* ks) {
  pdl_wait();
  const double beta = sqrt(sumsq[0]);
  const double s = beta > 0.0 ? 1.0 / beta : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v0[i] = (T)(r[i] * s);
  if (blockIdx.x == 0 && threadIdx.x == 0) ks->g[0] = beta;
}

// Partial dot products of w with v_0..v_{nv-1} (vectors ld apart): grid (KNB, nv), FP64 sums
// over a fixed grid-stride partition (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) k_kry_dot_partial(const T* __restrict__ V, long long ld,
                                                         const T* __restrict__ w, long long n,
                                                         double* __restrict__ part) {
  pdl_wait();
  __shared__ double red[8];
  const T* v = V + (size_t)blockIdx.y * ld;
  T acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = fma(v[i], w[i], acc);
  const double s = block_sum<double>((double)acc, red);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// h_i = sum of the partials of vector i (one warp per vector, fixed order); column j of the
// Hessenberg matrix gets h (first pass) or h added (second pass).
__global__ void k_kry_dot_final(const double* __restrict__ part, int np, KState* ks, int j,
                                int accumulate) {
  pdl_wait();
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += 32) acc += part[(size_t)i * np + k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) {
    ks->h[i] = acc;
    double* col = ks->R + (size_t)j * LDH;
    col[i] = accumulate ? col[i] + acc : acc;
  }
}

// w -= sum_i h_i v_i, i < nv (in T).
template <typename T>
__global__ void k_kry_axpy(T* __restrict__ w, const T* __restrict__ V, long long ld, int nv,
                           const KState* __restrict__ ks, long long n) {
  pdl_wait();
  __shared__ T hs[MAXS + 1];
  if (threadIdx.x < nv) hs[threadIdx.x] = (T)ks->h[threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    T acc = w[i];
    for (int k = 0; k < nv; ++k) acc = fma(-hs[k], V[(size_t)k * ld + i], acc);
    w[i] = acc;
  }
}

// Partial sums of squares of w (each thread's share in T, the shares in FP64).
template <typename T>
__global__ void __launch_bounds__(256) k_kry_sumsq_partial(const T* __restrict__ w, long long n,
                                                           double* __restrict__ part) {
  pdl_wait();
  __shared__ double red[8];
  T acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = fma(w[i], w[i], acc);
  const double s = block_sum<double>((double)acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// h_{j+1,j} = ||w|| from the partial sums of squares, then the rotations of column j: the
// earlier ones, and a new one that zeroes h_{j+1,j} (cs = 1, sn = 0 when both entries are 0);
// g follows the new rotation.
__global__ void k_kry_rotate(const double* __restrict__ part, int np, KState* ks, int j) {
  pdl_wait();
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += 32) acc += part[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x != 0) return;
  double* col = ks->R + (size_t)j * LDH;
  const double hn = sqrt(acc);
  col[j + 1] = hn;
  ks->inv = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {
    const double t = ks->cs[i] * col[i] + ks->sn[i] * col[i + 1];
    col[i + 1] = -ks->sn[i] * col[i] + ks->cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double rr = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (rr != 0.0) {
    c = a / rr;
    s = b / rr;
  }
  ks->cs[j] = c;
  ks->sn[j] = s;
  col[j] = rr;
  col[j + 1] = 0.0;
  ks->g[j + 1] = -s * ks->g[j];
  ks->g[j] = c * ks->g[j];
}

// v_{j+1} = w / h_{j+1,j} (0 at a breakdown).
template <typename T>
__global__ void k_kry_scale(T* __restrict__ w, long long n, const KState* __restrict__ ks) {
  pdl_wait();
  const T s = (T)ks->inv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] *= s;
}

// y = R^{-1} g by back substitution (a zero pivot gives y_i = 0).
__global__ void k_kry_solve(KState* ks, int steps) {
  pdl_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = steps - 1; i >= 0; --i) {
    double s = ks->g[i];
    for (int k = i + 1; k < steps; ++k) s -= ks->R[(size_t)k * LDH + i] * ks->y[k];
    const double piv = ks->R[(size_t)i * LDH + i];
    ks->y[i] = piv != 0.0 ? s / piv : 0.0;
  }
}

// u += sum_j y_j z_j (the sum in T, added to the FP64 iterate).
template <typename T>
__global__ void k_kry_update(double* __restrict__ u, const T* __restrict__ Z, long long ld,
                             int steps, const KState* __restrict__ ks, long long n) {
  pdl_wait();
  __shared__ T ys[MAXS];
  if (threadIdx.x < steps) ys[threadIdx.x] = (T)ks->y[threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    T acc = 0;
    for (int k = 0; k < steps; ++k) acc = fma(ys[k], Z[(size_t)k * ld + i], acc);
    u[i] += (double)acc;
  }
}

}  // namespace krylov
}  // namespace tpc
