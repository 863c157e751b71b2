// Finest-level residual r = b - A u without transforms, for levels whose Toeplitz generators are
// piecewise constant (the constant kernel of section 2.2: the printed coefficients of eq. (2.9)
// and eq. (2.11) are constant over ranges of the distance; a shift sigma only changes t_0).
//
// A Toeplitz block T(i, j) = t_{i-j} whose generator is constant, t_d = c, on a run lo <= d <= hi
// contributes c * sum_{j = i - hi}^{i - lo} x_j = c (P(i - lo + 1) - P(i - hi)) to (T x)_i, with P
// the exclusive prefix sum of x (x_j = 0 outside 0 <= j < N, so P(k) = P(0) = 0 for k <= 0 and
// P(k) = P(N) for k >= N). The product is then O(runs) per output instead of two FFTs.
//
// Accuracy. P(k) = Off(k / 2048) + Loc(k): Loc is the prefix inside a block of 2048 entries (plain
// FP64, magnitude at most 2048 max|x|), Off the prefix of the block totals kept as a double-double
// (hi, lo). A box sum P(a) - P(b) = (Off_hi(qa) - Off_hi(qb)) + (Off_lo(qa) - Off_lo(qb)) +
// (Loc(a) - Loc(b)) then carries rounding errors of the size of the box and of one block, not of
// the whole prefix (whose magnitude reaches N max|x|): the errors of the block totals before b
// cancel exactly in the difference.
//
// The Cross parts (eq. (3.7)) are applied as in the transform kernels: p, xi times w_o, and the
// middle row q.v + o w_o + zeta.w_bar.
#pragma once

#include <cuda_runtime.h>

namespace tpc {
namespace box {

constexpr int LB = 11;         // scan block: 2048 entries
constexpr int BLK = 1 << LB;
constexpr int MAXR = 16;       // runs per generator
constexpr int NT = 256;

struct Run {
  int lo, hi;                  // generator index range d in [lo, hi], T(i, j) = t_{i - j}
  double val;
};

struct BoxArgs {
  int N;                       // N_K
  int nblk;                    // scan blocks per segment: prefix indices k = 0..N
  const double* x;             // operand u, 2N + 1 (v, w_o, w_bar)
  const double* b;             // right-hand side
  double* r;                   // residual out (may alias nothing above)
  double* loc;                 // 2 (N + 1): in-block exclusive prefix of v, then of w_bar
  double* bsum;                // 2 nblk: block totals
  double2* off;                // 2 nblk: exclusive prefix of the block totals, (hi, lo)
  double* part;                // 2 nblk: partial Cross dots (q.v per block, zeta.w_bar per block)
  double* dot;                 // q.v + zeta.w_bar
  const double* p;
  const double* q;
  const double* xi;
  const double* zeta;
  double o;
  int nq, np;                  // q, zeta vanish from nq on; p, xi from np on
  int nrun[4];                 // runs of A (acts on v), B_bar (w_bar), C_bar (v), D_bar (w_bar)
  Run run[4][MAXR];
};

// Local prefix of each 2048-entry block of v (blocks 0..nblk-1) and of w_bar (nblk..2 nblk-1),
// the block totals and the block's share of the Cross dot.
__device__ __forceinline__ void box_local_body(const BoxArgs& a, int blk) {
  __shared__ double wsum[NT / 32];
  __shared__ double wdot[NT / 32];
  const int s = blk >= a.nblk;
  const int qb = blk - s * a.nblk;
  const int N = a.N;
  const double* xs = a.x + (s ? N + 1 : 0);
  const double* cr = s ? a.zeta : a.q;
  const int k0 = qb * BLK + 8 * threadIdx.x;
  double v[8];
  double dot = 0.0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = k0 + e;
    v[e] = (k < N) ? xs[k] : 0.0;
    if (k < a.nq) dot = fma(cr[k], v[e], dot);
  }
  double pre[8];
  double run = 0.0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    pre[e] = run;
    run += v[e];
  }
  // exclusive scan of the thread totals over the block (warp shuffles, then the warp totals)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  double dsum = dot;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
  if (lane == 31) wsum[wid] = inc;
  if (lane == 0) wdot[wid] = dsum;
  __syncthreads();
  double wpre = 0.0;
  for (int w = 0; w < wid; ++w) wpre += wsum[w];
  const double excl = wpre + (inc - run);
  double* loc = a.loc + (size_t)s * (N + 1);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = k0 + e;
    if (k <= N) loc[k] = excl + pre[e];
  }
  if (threadIdx.x == 0) {
    double tot = 0.0, dt = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      tot += wsum[w];
      dt += wdot[w];
    }
    a.bsum[blk] = tot;
    a.part[blk] = dt;
  }
}
__global__ void __launch_bounds__(NT) k_box_local(BoxArgs a) {
  pdl_wait();
  box_local_body(a, (int)blockIdx.x);
}

// Double-double addition (Knuth's two-sum on the high parts, then the low parts).
__device__ __forceinline__ double2 dd_add(double2 x, double2 y) {
  const double s = x.x + y.x;
  const double bb = s - x.x;
  const double err = (x.x - (s - bb)) + (y.x - bb);
  const double lo = err + x.y + y.y;
  const double hi = s + lo;
  return make_double2(hi, lo - (hi - s));
}

// Exclusive double-double prefix of the block totals of both segments, and the Cross dot (a
// fixed-order tree sum of the block shares). One block of 1024 threads.
__device__ __forceinline__ void box_offsets_body(const BoxArgs& a) {
  __shared__ double2 sc[1024];
  __shared__ double red[1024];
  const int t = threadIdx.x;
  const int nb = a.nblk;
  const int per = (nb + 1023) / 1024;  // blocks per thread
  for (int s = 0; s < 2; ++s) {
    const double* bs = a.bsum + s * nb;
    double2 mine = make_double2(0.0, 0.0);
    for (int j = 0; j < per; ++j) {
      const int q = t * per + j;
      if (q < nb) mine = dd_add(mine, make_double2(bs[q], 0.0));
    }
    sc[t] = mine;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan of the thread sums
      const double2 y = (t >= o) ? sc[t - o] : make_double2(0.0, 0.0);
      __syncthreads();
      if (t >= o) sc[t] = dd_add(sc[t], y);
      __syncthreads();
    }
    double2 run = (t > 0) ? sc[t - 1] : make_double2(0.0, 0.0);
    for (int j = 0; j < per; ++j) {
      const int q = t * per + j;
      if (q < nb) {
        a.off[s * nb + q] = run;
        run = dd_add(run, make_double2(bs[q], 0.0));
      }
    }
    __syncthreads();
  }
  double d = 0.0;
  for (int q = t; q < 2 * nb; q += 1024) d += a.part[q];
  red[t] = d;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) a.dot[0] = red[0];
}
__global__ void __launch_bounds__(1024) k_box_offsets(BoxArgs a) {
  pdl_wait();
  box_offsets_body(a);
}

// P(a) - P(b) of segment s (a, b already clamped to [0, N]).
__device__ __forceinline__ double box_sum(const BoxArgs& a, int s, int ka, int kb) {
  const double* loc = a.loc + (size_t)s * (a.N + 1);
  const double2 oa = a.off[s * a.nblk + (ka >> LB)];
  const double2 ob = a.off[s * a.nblk + (kb >> LB)];
  return ((oa.x - ob.x) + (oa.y - ob.y)) + (loc[ka] - loc[kb]);
}

// (T x_s)_i for the runs (in shared memory) of one generator acting on segment s.
__device__ __forceinline__ double toeplitz_runs(const BoxArgs& a, const Run* runs, int nrun,
                                                int s, int i) {
  const int N = a.N;
  const double* xs = a.x + (s ? N + 1 : 0);
  double acc = 0.0;
  for (int u = 0; u < nrun; ++u) {
    const Run R = runs[u];
    if (R.lo == R.hi) {
      const int j = i - R.lo;
      if (j >= 0 && j < N) acc = fma(R.val, xs[j], acc);
    } else {
      const int ka = min(max(i - R.lo + 1, 0), N);
      const int kb = min(max(i - R.hi, 0), N);
      if (ka > kb) acc = fma(R.val, box_sum(a, s, ka, kb), acc);
    }
  }
  return acc;
}

// r = b - A u for the node rows (blockIdx.y = 0: A v + B_bar w_bar + p w_o) and the midpoint
// rows (1: C_bar v + D_bar w_bar + xi w_o); block (0, 0) also forms the middle row.
// Block bx of gx (grid-stride over the rows), half 0 / 1 (node / midpoint rows).
__device__ __forceinline__ void box_resid_body(const BoxArgs& a, int bx, int gx, int half) {
  __shared__ int nr[4];
  __shared__ Run sr[4][MAXR];
  if (threadIdx.x < 4) nr[threadIdx.x] = a.nrun[threadIdx.x];
  if (threadIdx.x < 4 * MAXR) sr[threadIdx.x / MAXR][threadIdx.x % MAXR] =
      a.run[threadIdx.x / MAXR][threadIdx.x % MAXR];
  __syncthreads();
  const int N = a.N;
  const double w_o = a.x[N];
  const int g1 = half ? 2 : 0, g2 = half ? 3 : 1;
  for (int i = bx * NT + threadIdx.x; i < N; i += gx * NT) {
    double y = toeplitz_runs(a, sr[g1], nr[g1], 0, i) + toeplitz_runs(a, sr[g2], nr[g2], 1, i);
    if (i < a.np) y = fma(half ? a.xi[i] : a.p[i], w_o, y);
    const int row = half ? N + 1 + i : i;
    a.r[row] = a.b[row] - y;
  }
  if (bx == 0 && half == 0 && threadIdx.x == 0) a.r[N] = a.b[N] - fma(a.o, w_o, a.dot[0]);
}
__global__ void __launch_bounds__(NT) k_box_resid(BoxArgs a) {
  pdl_wait();
  box_resid_body(a, (int)blockIdx.x, (int)gridDim.x, (int)blockIdx.y);
}

}  // namespace box
}  // namespace tpc
