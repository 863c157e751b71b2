// Kernels of one Toeplitz-plus-Cross level and of the V-cycle (Algorithm 2).
//
// Level k (section 3.2.2): u = [v (N); w_o (1); w_bar (N)], N = N_k = 2^k - 1, m = 2N + 2.
// y = A_k u is computed as (eq. (3.7) and the product formula after it)
//   [A v + B_bar w_bar ; q.v + o w_o + zeta.w_bar ; C_bar v + D_bar w_bar]
//   + [p w_o ; 0 ; xi w_o],
// with the four Toeplitz products done through one circulant embedding of length m
// (eq. (3.4)): z = pad(v) + i pad(w_bar) is transformed once, the 2x2 block product
// [Y1; Y2] = [A^ B^; C^ D^] [V^; W^] is formed per frequency pair (j, m-j) (V^, W^ are the
// transforms of v and w_bar, unpacked from Z_j and conj(Z_{m-j})), and Y1 + i Y2 is
// transformed back: the real part is A v + B_bar w_bar, the imaginary part C_bar v + D_bar w_bar.
//
// Pipelines for one product (forward DIF, inverse DIT, see tpc_fft.cuh):
//   m <= 2^LOG_WHOLE : k_mid<MID_WHOLE>: one CTA does pack, FFT, spectral product, inverse
//                      FFT and the epilogue.
//   larger m         : m = R1 * L. k_fwd_strided (R1-point DIF on each of the L columns of
//                      stride L, then the twiddle W_m^{c k}: the first log2 R1 stages),
//                      k_mid<MID_PAIR> (remaining log2 L stages on contiguous blocks, the
//                      spectral product across the mirror block, the first log2 L inverse
//                      stages), k_inv_strided (twiddle, R1-point DIT, epilogue).
// Bit-reversed position p holds frequency j = bitrev(p); its partner m - j sits at
// p' = 3 * 2^h - 1 - p inside the same octave [2^h, 2^{h+1}) (p' = p for p = 0, 1). In
// blocks of L positions, block b >= 2 pairs with b' = 3 * 2^g - 1 - b (g = octave of b);
// blocks 0 and 1 pair with themselves.
#pragma once

#include <cstdlib>
#include <cstring>

#include "tpc_fft.cuh"

namespace tpc {

// Programmatic dependent launch. The kernels of a solve run back to back on one stream, most
// of them short (the coarse levels). Launched with the programmatic-serialisation attribute
// (launch_k), a kernel may be scheduled before its predecessor has finished; it calls
// pdl_wait() before it touches global memory, which returns once the predecessor has
// completed and its memory is visible, so the results are those of ordinary stream order and
// only the launch latency overlaps. The kernels do not signal their successors early: that
// lets a successor's blocks be scheduled while the predecessor's last blocks run, which
// measured faster for batches of small solves but slower for the largest single solve.
// Without the attribute pdl_wait() is a no-op. TPC_PDL=0 in the environment launches without it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("TPC_PDL");
    return !(e && std::strcmp(e, "0") == 0);
  }();
  return on;
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

constexpr int LOG_LMAX = 12;        // longest in-shared-memory sub-transform (4096 points)
constexpr int NTHREADS = 256;       // elementwise kernels
constexpr int FFT_THREADS = 512;    // upper bound of the transform kernels' block size
// Transform kernels: FP64 is bound by the FP64 pipe -> 512 threads (one radix-16 task per
// thread for 8192 points, 16 warps on the SM's single resident block); FP32 -> 256 threads,
// 2 resident blocks per SM for the strided passes (their prologue / epilogue need the
// registers) and 3 for the contiguous-block kernels (measured best for each).
#ifndef TPC_F32_THREADS
#define TPC_F32_THREADS 256
#endif
#ifndef TPC_F32_MIN_BLOCKS
#define TPC_F32_MIN_BLOCKS 2
#endif
#ifndef TPC_F32_MID_MIN_BLOCKS
#define TPC_F32_MID_MIN_BLOCKS 3
#endif
template <typename T> constexpr int fft_threads() { return sizeof(T) == 8 ? 512 : TPC_F32_THREADS; }
// strided passes (register-heavier prologue / epilogue)
template <typename T> constexpr int fft_min_blocks() {
  return sizeof(T) == 8 ? 1 : TPC_F32_MIN_BLOCKS;
}
// FP32 strided passes of levels up to m = 2^LOG_M_HIGH_OCC: instances held to three resident
// blocks per SM (at most 85 registers a thread, none spilled) instead of two. Alone a level
// runs as fast either way (these levels are latency-bound); beside other solves (batches,
// the server) the third slot per SM lets more of their blocks run at once. The largest
// levels keep two (their radix-16 steps slow down under the register cap).
#ifndef TPC_LOG_M_HIGH_OCC
#define TPC_LOG_M_HIGH_OCC 18
#endif
constexpr int LOG_M_HIGH_OCC = TPC_LOG_M_HIGH_OCC;
constexpr int F32_HIGH_OCC_BLOCKS = 3;
// contiguous-block kernels
template <typename T> constexpr int mid_min_blocks() {
  return sizeof(T) == 8 ? 1 : TPC_F32_MID_MIN_BLOCKS;
}

enum Epi { EPI_APPLY = 0, EPI_RESID = 1, EPI_JACOBI = 2 };
// Prologue: how the operand u of the product is formed while it is loaded.
//   PRO_NONE:     u = x
//   PRO_SMOOTH:   u = omega D^{-1} f                  (first pre-smoothing sweep from 0), stored
//   PRO_RESTRICT: f = I_k^{k-1} r_fine, u = omega D^{-1} f (restriction + first sweep), both stored
//   PRO_PROLONG:  u = x + I_{k-1}^k e_coarse          (coarse-grid correction), stored
enum Pro { PRO_NONE = 0, PRO_SMOOTH = 1, PRO_RESTRICT = 2, PRO_PROLONG = 3 };
enum MidMode { MID_PAIR = 0, MID_WHOLE = 1, MID_FWD = 2, MID_FWD_REAL = 3 };
enum InMode { IN_PACK = 0, IN_REAL = 1 };

// Element indices inside a level's product are 32-bit: m <= 2^23 (the strided passes take
// R1 <= 2^11 rows of L <= 2^12 columns), so every index of z, the vectors and the tables is
// below 2^24.
template <typename T> struct LevelArgs {
  int N;                 // N_k
  int logm, logR1, logL, logC;
  const T* sA;           // spectra at bit-reversed positions, already divided by 2m
  const T* sD;
  const c2<T>* sB;
  const c2<T>* sC;       // nullptr for the SPD system (C_bar = B_bar^T, C^ = conj B^)
  const T* p;
  const T* q;
  const T* xi;
  const T* zeta;
  T o;
  int nq, np;            // q, zeta are zero from index nq on; p, xi from index np on
  // weakly singular model (else null): tridiagonal band of the concatenated index and the
  // per-entry Jacobi weights (pvec: pre-smoothing, for the prologue; wvec: this product's)
  const T* bl;
  const T* bd;
  const T* bu;
  const T* pvec;
  const T* wvec;
  T wA, wO, wD;          // omega / diagonal, per segment (damped Jacobi, eq. (3.3))
  const c2<T>* twm;      // strided pipelines only: W_m^j, j < m (FP64); two-level (FP32)
  const c2<T>* twL;      // W_{4096}^j, j < 4096 (FP32 copies the octant j <= 512 to shared)
  const c2<T>* tws;      // FP32: step twiddle tables of the register-resident kernels (tpc_f32.cuh)
  // per call
  int pro;               // Pro
  T pA, pO, pD;          // pre-smoothing omega / diagonal per segment (PRO_SMOOTH, PRO_RESTRICT)
  T* xout;               // where the formed operand is stored (PRO_SMOOTH/RESTRICT/PROLONG)
  T* fout;               // where the restricted right-hand side is stored (PRO_RESTRICT)
  const T* rfine;        // residual of the finer level (PRO_RESTRICT)
  const T* ec;           // correction from the coarser level (PRO_PROLONG)
  const T* x;            // operand u (n_k)
  const T* f;            // right-hand side for EPI_RESID / EPI_JACOBI
  T* y;                  // result (n_k); must not alias x
  const T* real_in;      // IN_REAL / MID_FWD_REAL input (m reals)
  int epi;
  c2<T>* z;              // complex work array (m)
  T* partials;           // per-CTA partial dots of the forward strided pass
  int nparts;
  int geo;               // transfer: 0 the paper's (concatenated vector), 1 geometric
};

// Twiddle W_m^e of the strided passes, e < m. FP64 (whose kernels are bound by the FP64 pipe)
// reads one table of m entries; FP32 (bound by memory latency) computes it (w_f32).
// FP32 W_m^e = exp(-2 pi i e / m) without tables or FP64: the exact quadrant / octant symmetries
// of sine and cosine reduce the angle to theta = 2 pi s / m in [0, pi/4] (s integer), then the
// Taylor series of sin and cos, truncated after the x^9 / x^10 terms (remainder below 2e-9 for
// |x| <= pi/4, far under the FP32 epsilon), are evaluated by Horner's rule.
__device__ __forceinline__ float2 w_f32(int e, int logm) {
  const int q4 = 1 << (logm - 2), q8 = q4 >> 1;
  const int quad = e >> (logm - 2);
  int r = e & (q4 - 1);
  const bool swap = r > q8;
  if (swap) r = q4 - r;
  // 32-bit integer conversions only (64-bit ones would run on the FP64 pipe); 2^-logm exactly
  const float x = (float)r * (6.283185307179586f * __int_as_float((127 - logm) << 23));
  const float x2 = x * x;
  const float sn = x * fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 362880.0f, -1.0f / 5040.0f),
                                              1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
  const float cs = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 3628800.0f,
                                                             1.0f / 40320.0f), -1.0f / 720.0f),
                                          1.0f / 24.0f), -0.5f), 1.0f);
  const float c0 = swap ? sn : cs, s0 = swap ? cs : sn;  // cos, sin of 2 pi (e mod m/4) / m
  // exp(-i (quad pi/2 + phi)) = (-i)^quad (c0 - i s0)
  const float re = (quad == 0) ? c0 : (quad == 1) ? -s0 : (quad == 2) ? -c0 : s0;
  const float im = (quad == 0) ? -s0 : (quad == 1) ? -c0 : (quad == 2) ? s0 : c0;
  return make_float2(re, im);
}

// FP32 twiddles of the strided passes, factored per thread. Thread tid of a block of nt
// threads (C = 2^logC columns, tile = R1 C entries, tile >= 2 nt) holds the entries
// e = tid + nt j, j < J = tile / nt: column c = c0 + (tid mod C) and row t = t0 + (nt / C) j with
// t0 = tid / C < nt / C. The row bits of t0 and of (nt / C) j do not overlap, so
// bitrev(t) = bitrev(t0) + bitrev_J(j) (bit reversal over log2 R1 and log2 J bits) and
// W_m^{c bitrev(t)} = W_m^{c bitrev(t0)} * W_m^{c bitrev_J(j)}: one value per thread times an
// entry of a C x J table built once per block (at most 512 entries).
struct InterTw32 {
  float2 base;   // W_m^{c bitrev(t0)}
  int row;       // first table entry of this thread's column
  int logJ;
};
__device__ __forceinline__ InterTw32 inter_tw32_setup(float2* tab, long long c0, int logC,
                                                      int logR1, int logm) {
  const int nt = blockDim.x, C = 1 << logC;
  const int logJ = logR1 + logC - (31 - __clz(nt));
  const int J = 1 << logJ;
  for (int i = threadIdx.x; i < (C << logJ); i += nt)
    tab[i] = w_f32((int)((c0 + (i >> logJ)) * (i & (J - 1))), logm);
  InterTw32 r;
  const int cc = threadIdx.x & (C - 1), t0 = threadIdx.x >> logC;
  r.base = w_f32((int)((c0 + cc) * (long long)brev_bits((unsigned)t0, logR1)), logm);
  r.row = cc << logJ;
  r.logJ = logJ;
  return r;
}
__device__ __forceinline__ float2 inter_tw32(const InterTw32& it, const float2* tab, int j) {
  return cmul<float>(it.base, tab[it.row + (int)(__brev((unsigned)j) >> (32 - it.logJ))]);
}

template <typename T>
__device__ __forceinline__ c2<T> inter_tw(const c2<T>* __restrict__ twm, int e, int logm) {
  if constexpr (sizeof(T) == 8) {
    return __ldg(twm + e);
  } else {
    return w_f32(e, logm);  // e < m <= 2^23
  }
}

// Fine indices (concatenated, 0-based) of the three restricted values of coarse index I, with
// weights 1/4, 1/2, 1/4. The paper's transfer (section 3.1): 2I, 2I+1, 2I+2. The geometric
// one (an option, not the paper's): the coarse unknown at position t h (t = 2(I+1) for a node
// I < Nc, t = 2(I-Nc)+1 for a midpoint) takes the fine midpoint, node and midpoint at
// (t - 1/2) h, t h, (t + 1/2) h, i.e. w_t, v_t, w_{t+1} (Nf = 2 Nc + 1 fine nodes).
__device__ __forceinline__ void restrict_idx(int I, int Nc, int geo, int& i0, int& i1, int& i2) {
  if (!geo) {
    i0 = 2 * I;
    i1 = 2 * I + 1;
    i2 = 2 * I + 2;
    return;
  }
  const int t = (I < Nc) ? 2 * (I + 1) : 2 * (I - Nc) + 1;
  const int Nf = 2 * Nc + 1;
  i0 = Nf + t - 1;
  i1 = t - 1;
  i2 = Nf + t;
}
// Restriction at coarse index I of a level with Nc nodes.
template <typename T>
__device__ __forceinline__ T restrict_at(const T* __restrict__ r, int I, int Nc, int geo) {
  int i0, i1, i2;
  restrict_idx(I, Nc, geo, i0, i1, i2);
  return (T)0.25 * r[i0] + (T)0.5 * r[i1] + (T)0.25 * r[i2];
}
// Coarse index (concatenated, 0-based) of the coarse unknown at position t h (geometric
// transfer), t = 1..Nf: a coarse node for even t, a coarse midpoint for odd t.
__device__ __forceinline__ int coarse_of_position(int t, int Nc) {
  return (t & 1) ? Nc + (t - 1) / 2 : t / 2 - 1;
}
// Operand entry j of the product (concatenated index), formed by the prologue; w is the
// pre-smoothing weight of j's segment. Split into the loads (issued in batches, so that many
// loads are in flight per thread) and the arithmetic and stores that follow them.
template <typename T> struct Raw {
  T a0, a1, a2;
};
// The coarse-correction values of PRO_PROLONG at fine index j (a1, a2 of Raw).
template <typename T>
__device__ __forceinline__ void prolong_load(const LevelArgs<T>& a, int j, Raw<T>& r) {
  if (a.geo) {
    // P = 2 R^T of the geometric transfer: node v_t (j = t - 1) takes the coarse value at
    // t h; midpoint w_u (j = N + u - 1) half of those at (u - 1) h and u h (0 outside 1..N).
    // Laid out for operand_finish, which adds a1 at odd j and (a1 + a2) / 2 at even j.
    const int N = a.N, Nc = (N - 1) / 2;
    if (j < N) {
      r.a1 = a.ec[coarse_of_position(j + 1, Nc)];
      r.a2 = r.a1;
    } else {
      const int u = j - N + 1;
      const T lo = (u >= 2) ? a.ec[coarse_of_position(u - 1, Nc)] : (T)0;
      const T hi = (u <= N) ? a.ec[coarse_of_position(u, Nc)] : (T)0;
      if (j & 1) {
        r.a1 = (T)0.5 * (lo + hi);
      } else {
        r.a1 = lo;
        r.a2 = hi;
      }
    }
    return;
  }
  if (j & 1) {
    r.a1 = a.ec[(j - 1) / 2];
  } else {
    const int I = j / 2;
    r.a1 = (I >= 1) ? a.ec[I - 1] : (T)0;
    r.a2 = (I < a.N) ? a.ec[I] : (T)0;  // coarse size n_{k-1} = N_k
  }
}
template <typename T>
__device__ __forceinline__ Raw<T> operand_load(const LevelArgs<T>& a, int j, int pro) {
  Raw<T> r{0, 0, 0};
  if (pro == PRO_NONE) {
    r.a0 = a.x[j];
  } else if (pro == PRO_SMOOTH) {
    r.a0 = a.f[j];
  } else if (pro == PRO_RESTRICT) {
    int i0, i1, i2;
    restrict_idx(j, a.N, a.geo, i0, i1, i2);
    r.a0 = a.rfine[i0];
    r.a1 = a.rfine[i1];
    r.a2 = a.rfine[i2];
  } else {
    r.a0 = a.x[j];
    prolong_load<T>(a, j, r);
  }
  return r;
}
template <typename T>
__device__ __forceinline__ T operand_finish(const LevelArgs<T>& a, int j, const Raw<T>& r,
                                            T w, int pro) {
  if (pro == PRO_NONE) return r.a0;
  if ((pro == PRO_SMOOTH || pro == PRO_RESTRICT) && a.pvec) w = a.pvec[j];
  if (pro == PRO_SMOOTH) {
    const T v = w * r.a0;
    a.xout[j] = v;
    return v;
  }
  if (pro == PRO_RESTRICT) {
    const T fv = (T)0.25 * r.a0 + (T)0.5 * r.a1 + (T)0.25 * r.a2;  // restriction, section 3.1
    a.fout[j] = fv;
    const T v = w * fv;
    a.xout[j] = v;
    return v;
  }
  const T v = r.a0 + ((j & 1) ? r.a1 : (T)0.5 * (r.a1 + r.a2));  // prolongation, P = 2 R^T
  a.xout[j] = v;
  return v;
}
template <typename T>
__device__ __forceinline__ T operand(const LevelArgs<T>& a, int j, T w, int pro) {
  return operand_finish<T>(a, j, operand_load<T>(a, j, pro), w, pro);
}

#ifndef TPC_UNROLL
#define TPC_UNROLL 4
#endif
constexpr int UNROLL = TPC_UNROLL;  // elements per thread whose loads are issued together

// Asynchronous global -> shared copies (4 or 8 bytes, both addresses aligned to the size): a
// thread issues all of its copies for a tile without holding registers for them, then waits.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}
// Waits for this thread's copies (others' copies need a barrier as well).
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  return s;  // valid in thread 0
}

// Epilogue for output index i < N: ax_v, ax_w are the Toeplitz parts of (A u)_v[i] and
// (A u)_{w_bar}[i]; the Cross column p, xi times w_o is added here. Loads first (batched by
// the callers), then arithmetic and stores.
template <typename T> struct EpiRaw {
  T p, xi, fv, fw, xv, xw;
  T bv, bw;  // band products (B x)_i, (B x)_{iw} (weakly singular model, else 0)
  T wv, ww;  // per-entry Jacobi weights (weakly singular model)
};
// (B x)_j of the tridiagonal band at concatenated index j (0 <= j < n).
template <typename T>
__device__ __forceinline__ T band_at(const LevelArgs<T>& a, int j) {
  const int n = 2 * a.N + 1;
  T s = a.bd[j] * a.x[j];
  if (j > 0) s = fma(a.bl[j], a.x[j - 1], s);
  if (j + 1 < n) s = fma(a.bu[j], a.x[j + 1], s);
  return s;
}
template <typename T>
__device__ __forceinline__ EpiRaw<T> epi_load(const LevelArgs<T>& a, int i, int epi) {
  EpiRaw<T> r{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int iw = a.N + 1 + i;
  if (a.bd) {
    r.bv = band_at<T>(a, i);
    r.bw = band_at<T>(a, iw);
    if (epi == EPI_JACOBI) {
      r.wv = a.wvec[i];
      r.ww = a.wvec[iw];
    }
  }
  if (i < a.np) {
    r.p = a.p[i];
    r.xi = a.xi[i];
  }
  if (epi != EPI_APPLY) {
    r.fv = a.f[i];
    r.fw = a.f[iw];
  }
  if (epi == EPI_JACOBI) {
    r.xv = a.x[i];
    r.xw = a.x[iw];
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void epi_store(const LevelArgs<T>& a, int i, const EpiRaw<T>& r,
                                          T ax_v, T ax_w, T w_o, int epi) {
  const T yv = fma(r.p, w_o, ax_v) + r.bv;
  const T yw = fma(r.xi, w_o, ax_w) + r.bw;
  const int iw = a.N + 1 + i;
  if (epi == EPI_APPLY) {
    a.y[i] = yv;
    a.y[iw] = yw;
  } else if (epi == EPI_RESID) {
    a.y[i] = r.fv - yv;
    a.y[iw] = r.fw - yw;
  } else {
    a.y[i] = fma(a.bd ? r.wv : a.wA, r.fv - yv, r.xv);
    a.y[iw] = fma(a.bd ? r.ww : a.wD, r.fw - yw, r.xw);
  }
}

template <typename T>
__device__ __forceinline__ void epi_middle(const LevelArgs<T>& a, T dot, T w_o, int epi) {
  const int im = a.N;
  const T ym = fma(a.o, w_o, dot) + (a.bd ? band_at<T>(a, im) : (T)0);
  if (epi == EPI_APPLY)
    a.y[im] = ym;
  else if (epi == EPI_RESID)
    a.y[im] = a.f[im] - ym;
  else
    a.y[im] = fma(a.bd ? a.wvec[im] : a.wO, a.f[im] - ym, a.x[im]);
}

// Spectral 2x2 block product for the frequency pair held at positions (lower, upper).
// Spectra of the lower member (bit-reversed position P): loaded first, applied after.
template <typename T> struct Spec {
  T sa, sd;
  c2<T> sb, sc;
};
template <typename T, bool NS>
__device__ __forceinline__ Spec<T> spec_load(const LevelArgs<T>& a, int P) {
  Spec<T> r;
  r.sa = a.sA[P];
  r.sd = a.sD[P];
  r.sb = a.sB[P];
  if (NS) {
    r.sc = a.sC[P];
  } else {
    r.sc.x = r.sb.x;
    r.sc.y = -r.sb.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void mac_pair(const Spec<T>& sp, c2<T>* zl, c2<T>* zu) {
  const c2<T> Zp = *zl, Zq = *zu;
  // 2 V^ = Z_p + conj Z_q ; 2 W^ = (Z_p - conj Z_q) / i, from Z_p + Z_q and Z_p - Z_q
  const c2<T> S = cadd<T>(Zp, Zq), D = csub<T>(Zp, Zq);
  const T vr = S.x, vi = D.y;
  const T wr = S.y, wi = -D.x;
  const T y1r = fma(sp.sa, vr, fma(sp.sb.x, wr, -sp.sb.y * wi));
  const T y1i = fma(sp.sa, vi, fma(sp.sb.x, wi, sp.sb.y * wr));
  const T y2r = fma(sp.sd, wr, fma(sp.sc.x, vr, -sp.sc.y * vi));
  const T y2i = fma(sp.sd, wi, fma(sp.sc.x, vi, sp.sc.y * vr));
  *zl = mk<T>(y1r - y2i, y1i + y2r);
  if (zu != zl) *zu = mk<T>(y1r + y2i, y2r - y1i);
}

// Pair tasks of the self-paired block 0 (positions [0, L)): task q -> (p, p').
__device__ __forceinline__ void block0_pair(int q, int& p, int& pp) {
  if (q < 2) {
    p = pp = q;
    return;
  }
  const int qq = q - 1;
  const int g = 31 - __clz(qq);
  p = qq + (1 << g);
  pp = 3 * (2 << g) - 1 - p;
}

// ------------------------------------------------------------------------------------
// Forward strided pass: the first log2(R1) DIF stages as R1-point transforms of the L
// columns (stride L), each followed by the twiddle W_m^{c k}. One CTA: 2^logC columns.
// ------------------------------------------------------------------------------------
// PRO: the prologue, fixed at compile time (the launch selects the instance from a.pro).
// Body of the pass for column block blk (the kernel's block index, or a batched kernel's tile).
template <typename T, int IN, int PRO>
__device__ __forceinline__ void fwd_strided_body(const LevelArgs<T>& a, int blk) {
  constexpr int pro = PRO;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<T>* tab = reinterpret_cast<c2<T>*>(smem_raw);
  c2<T>* s = tab + tw_slots<T>();
  __shared__ T red[FFT_THREADS / 32];
  const int logR1 = a.logR1, logC = a.logC, logL = a.logL;
  const c2<T>* tw = step_table_issue<T>(tab, a.twL);  // in flight with the tile's copies
  const int C = 1 << logC;
  const int tile = 1 << (logR1 + logC);
  const int c0 = blk << logC;
  const int half = 1 << (logR1 - 1);
  T dot = 0;
  // FP32 (bound by memory latency): the raw operand values and the Cross rows q, zeta arrive by
  // asynchronous copies, all of a thread's copies in flight at once: the operand pair (v, w_bar)
  // into the slot of its row t < R1/2, (q, zeta) into the slot of row t + R1/2 (the zero
  // padding, cleared once read). The restriction prologue (three fine values per entry) keeps
  // the register path.
  constexpr bool ASYNC = sizeof(T) == 4 && IN == IN_PACK && PRO != PRO_RESTRICT;
  if constexpr (ASYNC) {
    const int ht = tile >> 1;
    const T* src = (PRO == PRO_SMOOTH) ? a.f : a.x;
    for (int e = threadIdx.x; e < ht; e += blockDim.x) {
      const int t = e >> logC, cc = e & (C - 1);
      const int P = c0 + cc + (t << logL);
      c2<T>* lo = s + pad16(e);
      c2<T>* hi = s + pad16(e + ht);
      if (P < a.N) {
        cp_async4(&lo->x, src + P);
        cp_async4(&lo->y, src + a.N + 1 + P);
        if (P < a.nq) {
          cp_async4(&hi->x, a.q + P);
          cp_async4(&hi->y, a.zeta + P);
        } else {
          *hi = mk<T>(0, 0);
        }
      } else {
        *lo = mk<T>(0, 0);
        *hi = mk<T>(0, 0);
      }
    }
    cp_async_wait_all();
    for (int e0 = threadIdx.x; e0 < ht; e0 += UNROLL * blockDim.x) {
      Raw<T> rv[UNROLL], rw[UNROLL];
      if constexpr (PRO == PRO_PROLONG) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
          const int e = e0 + u * blockDim.x;
          const int t = e >> logC, cc = e & (C - 1);
          const int P = c0 + cc + (t << logL);
          if (e < ht && P < a.N) {
            prolong_load<T>(a, P, rv[u]);
            prolong_load<T>(a, a.N + 1 + P, rw[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= ht) continue;
        const int t = e >> logC, cc = e & (C - 1);
        const int P = c0 + cc + (t << logL);
        c2<T>* lo = s + pad16(e);
        c2<T>* hi = s + pad16(e + ht);
        if (P < a.N) {
          const c2<T> raw = *lo, qz = *hi;
          rv[u].a0 = raw.x;
          rw[u].a0 = raw.y;
          const T xv = operand_finish<T>(a, P, rv[u], a.pA, pro);
          const T xw = operand_finish<T>(a, a.N + 1 + P, rw[u], a.pD, pro);
          *lo = mk<T>(xv, xw);
          dot = fma(qz.x, xv, fma(qz.y, xw, dot));
        }
        *hi = mk<T>(0, 0);
      }
    }
  } else if (IN == IN_PACK) {
    // rows t >= R1/2 are the zero padding of the embedding
    for (int e = threadIdx.x + (tile >> 1); e < tile; e += blockDim.x) s[pad16(e)] = mk<T>(0, 0);
    for (int e0 = threadIdx.x; e0 < (tile >> 1); e0 += UNROLL * blockDim.x) {
      Raw<T> rv[UNROLL], rw[UNROLL];
      T qv[UNROLL], zv[UNROLL];
      bool ok[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        const int t = e >> logC, cc = e & (C - 1);
        const int P = c0 + cc + (t << logL);
        ok[u] = (e < (tile >> 1)) && P < a.N;
        if (ok[u]) {
          rv[u] = operand_load<T>(a, P, pro);
          rw[u] = operand_load<T>(a, a.N + 1 + P, pro);
          qv[u] = (P < a.nq) ? a.q[P] : (T)0;
          zv[u] = (P < a.nq) ? a.zeta[P] : (T)0;
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= (tile >> 1)) continue;
        const int t = e >> logC, cc = e & (C - 1);
        const int P = c0 + cc + (t << logL);
        c2<T> v = mk<T>(0, 0);
        if (ok[u]) {
          const T xv = operand_finish<T>(a, P, rv[u], a.pA, pro);
          const T xw = operand_finish<T>(a, a.N + 1 + P, rw[u], a.pD, pro);
          v = mk<T>(xv, xw);
          dot = fma(qv[u], xv, fma(zv[u], xw, dot));
        }
        s[pad16(e)] = v;
      }
    }
  } else {
    for (int e0 = threadIdx.x; e0 < tile; e0 += UNROLL * blockDim.x) {
      T rv[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        const int t = e >> logC, cc = e & (C - 1);
        if (e < tile) rv[u] = a.real_in[c0 + cc + (t << logL)];
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < tile) s[pad16(e)] = mk<T>(rv[u], 0);
      }
    }
  }
  (void)half;
  if constexpr (sizeof(T) == 4) cp_async_wait_all();  // the step table
  __syncthreads();
  smem_dif<T, true>(s, logR1, logC, C, 1, tw, LOG_LMAX);
  if (sizeof(T) == 4 && tile >= 2 * (int)blockDim.x &&
      (long long)tile * C <= (long long)TW_TAB * blockDim.x) {
    // the step-twiddle table is no longer needed: its slots take the factored twiddles
    float2* t2 = reinterpret_cast<float2*>(tab);
    const InterTw32 it = inter_tw32_setup(t2, c0, logC, logR1, a.logm);
    __syncthreads();
    int j = 0;
    for (int e = threadIdx.x; e < tile; e += blockDim.x, ++j) {
      const int t = e >> logC, cc = e & (C - 1);
      const int P = c0 + cc + (t << logL);
      const float2 w = inter_tw32(it, t2, j);
      a.z[P] = cmul<T>(s[pad16(e)], mk<T>((T)w.x, (T)w.y));
    }
  } else {
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int t = e >> logC, cc = e & (C - 1);
      const int c = c0 + cc;
      const int P = c + (t << logL);
      const int kb = (int)brev_bits((unsigned)t, logR1);
      a.z[P] = cmul<T>(s[pad16(e)], inter_tw<T>(a.twm, c * kb, a.logm));
    }
  }
  if (IN == IN_PACK) {
    const T tot = block_sum<T>(dot, red);
    if (threadIdx.x == 0) {
      a.partials[blk] = tot;
      if (blk == 0 && pro != PRO_NONE) (void)operand<T>(a, a.N, a.pO, pro);  // middle w_o
    }
  }
}

template <typename T, int IN, int PRO, int MINB = fft_min_blocks<T>()>
__global__ void __launch_bounds__(fft_threads<T>(), MINB) k_fwd_strided(LevelArgs<T> a) {
  pdl_wait();
  fwd_strided_body<T, IN, PRO>(a, (int)blockIdx.x);
}

// ------------------------------------------------------------------------------------
// Contiguous blocks of L points: DIF, spectral product with the mirror block, DIT.
// ------------------------------------------------------------------------------------
// Body of the contiguous-block kernels on blocks (b, b2) with the step twiddles tw, the padded
// data area s and the reduction scratch red in shared memory.
// LOGL_CT, NSEQ_CT: when nonzero, log2 L and the number of blocks (1 or 2) as compile-time
// constants, so that every step's strides, task counts and radix are folded into the code.
template <typename T, int MODE, bool NS, int LOGL_CT = 0, int NSEQ_CT = 0, int PRO_CT = -1,
          int EPI_CT = -1, int UNR = UNROLL>
__device__ __forceinline__ void mid_core(const LevelArgs<T>& a, const c2<T>* tw, c2<T>* s,
                                         T* red, int b, int b2) {
  const int pro = PRO_CT >= 0 ? PRO_CT : a.pro;
  const int epi = EPI_CT >= 0 ? EPI_CT : a.epi;
  const int logL = LOGL_CT ? LOGL_CT : a.logL;
  const int L = 1 << logL;
  const int nseq = NSEQ_CT ? NSEQ_CT : ((b != b2) ? 2 : 1);
  const int total = nseq << logL;
  T dot = 0;
  if constexpr (MODE == MID_WHOLE) {
    for (int e0 = threadIdx.x; e0 < total; e0 += UNR * blockDim.x) {
      Raw<T> rv[UNR], rw[UNR];
      T qv[UNR], zv[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int i = e0 + u * blockDim.x;
        if (i < a.N) {
          rv[u] = operand_load<T>(a, i, pro);
          rw[u] = operand_load<T>(a, a.N + 1 + i, pro);
          qv[u] = (i < a.nq) ? a.q[i] : (T)0;
          zv[u] = (i < a.nq) ? a.zeta[i] : (T)0;
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int i = e0 + u * blockDim.x;
        if (i >= total) continue;
        c2<T> v = mk<T>(0, 0);
        if (i < a.N) {
          const T xv = operand_finish<T>(a, i, rv[u], a.pA, pro);
          const T xw = operand_finish<T>(a, a.N + 1 + i, rw[u], a.pD, pro);
          v = mk<T>(xv, xw);
          dot = fma(qv[u], xv, fma(zv[u], xw, dot));
        }
        s[pad16(i)] = v;
      }
    }
  } else if (sizeof(T) == 4 && MODE == MID_PAIR) {
    // FP32: asynchronous copies, all of a thread's copies in flight at once
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int sq = e >> logL, i = e & (L - 1);
      cp_async8(s + pad16(e), a.z + (sq ? b2 : b) * L + i);
    }
    cp_async_wait_all();
  } else {
    for (int e0 = threadIdx.x; e0 < total; e0 += 2 * UNR * blockDim.x) {
      c2<T> v[2 * UNR];
#pragma unroll
      for (int u = 0; u < 2 * UNR; ++u) {
        const int e = e0 + u * blockDim.x;
        const int sq = e >> logL, i = e & (L - 1);
        const int P = (sq ? b2 : b) * L + i;
        if (e < total) {
          if constexpr (MODE == MID_FWD_REAL) v[u] = mk<T>(a.real_in[P], 0);
          else v[u] = a.z[P];
        }
      }
#pragma unroll
      for (int u = 0; u < 2 * UNR; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) s[pad16(e)] = v[u];
      }
    }
  }
  T dot_total = 0;
  if (MODE == MID_WHOLE) {
    if (threadIdx.x == 0 && pro != PRO_NONE) (void)operand<T>(a, a.N, a.pO, pro);  // middle w_o
    dot_total = block_sum<T>(dot, red);
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();  // the step table
  __syncthreads();
  smem_dif<T, false>(s, logL, nseq - 1, 1, L, tw, LOG_LMAX);
  if constexpr (MODE == MID_FWD || MODE == MID_FWD_REAL) {
    for (int e = threadIdx.x; e < L; e += blockDim.x) a.z[b * L + e] = s[pad16(e)];
    return;
  }
  // spectral product: ntask frequency pairs; task i -> (lower, upper) shared-memory slots and
  // the bit-reversed position of the lower member
  const int ntask = (b != b2) ? L : ((b == 1) ? (L >> 1) : (L >> 1) + 1);
  for (int i0 = threadIdx.x; i0 < ntask; i0 += UNR * blockDim.x) {
    Spec<T> sp[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < ntask) {
        int p = i, pp;
        if (b == 0) block0_pair(i, p, pp);
        sp[u] = spec_load<T, NS>(a, b * L + p);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i >= ntask) continue;
      int lo, hi;
      if (b != b2) {
        lo = i;
        hi = L + (L - 1 - i);
      } else if (b == 1) {
        lo = i;
        hi = L - 1 - i;
      } else {
        block0_pair(i, lo, hi);
      }
      mac_pair<T>(sp[u], s + pad16(lo), s + pad16(hi));
    }
  }
  __syncthreads();
  smem_dit<T, false>(s, logL, nseq - 1, 1, L, tw, LOG_LMAX);
  if constexpr (MODE == MID_WHOLE) {
    const T w_o = a.x[a.N];
    for (int i0 = threadIdx.x; i0 < a.N; i0 += UNR * blockDim.x) {
      EpiRaw<T> er[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < a.N) er[u] = epi_load<T>(a, i, epi);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < a.N) {
          const c2<T> y = s[pad16(i)];
          epi_store<T>(a, i, er[u], y.x, y.y, w_o, epi);
        }
      }
    }
    if (threadIdx.x == 0) epi_middle<T>(a, dot_total, w_o, epi);
  } else {
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int sq = e >> logL, i = e & (L - 1);
      a.z[(sq ? b2 : b) * L + i] = s[pad16(e)];
    }
  }
}

template <typename T, int MODE, bool NS, int LOGL_CT = 0>
__device__ __forceinline__ void mid_body(const LevelArgs<T>& a, int blk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<T>* tab = reinterpret_cast<c2<T>*>(smem_raw);
  c2<T>* s = tab + tw_slots<T>();
  __shared__ T red[FFT_THREADS / 32];
  const c2<T>* tw = step_table_issue<T>(tab, a.twL);  // in flight with the tile's copies
  int b, b2;
  if (MODE == MID_FWD || MODE == MID_FWD_REAL || MODE == MID_WHOLE) {
    b = b2 = blk;
  } else {
    const int cta = blk;
    if (cta < 2) {
      b = b2 = cta;
    } else {
      const int j = cta - 1;
      const int g = 31 - __clz(j);
      b = j + (1 << g);
      b2 = 3 * (2 << g) - 1 - b;
    }
  }
  if constexpr (LOGL_CT > 0) {
    if (b != b2) mid_core<T, MODE, NS, LOGL_CT, 2>(a, tw, s, red, b, b2);
    else mid_core<T, MODE, NS, LOGL_CT, 1>(a, tw, s, red, b, b2);
  } else {
    mid_core<T, MODE, NS>(a, tw, s, red, b, b2);
  }
}

// One kernel name per mode (so profilers can select them).
// LOGL_CT: 0 for any L, or log2 L fixed at compile time (the launch picks the instance).
template <typename T, bool NS, int LOGL_CT = 0>
__global__ void __launch_bounds__(fft_threads<T>(), mid_min_blocks<T>()) k_mid_pair(LevelArgs<T> a) {
  pdl_wait();
  mid_body<T, MID_PAIR, NS, LOGL_CT>(a, (int)blockIdx.x);
}
template <typename T, bool NS>
__global__ void __launch_bounds__(fft_threads<T>(), mid_min_blocks<T>()) k_mid_whole(LevelArgs<T> a) {
  pdl_wait();
  mid_body<T, MID_WHOLE, NS>(a, (int)blockIdx.x);
}
template <typename T>
__global__ void __launch_bounds__(fft_threads<T>(), mid_min_blocks<T>()) k_mid_fwd(LevelArgs<T> a) {
  mid_body<T, MID_FWD, false>(a, (int)blockIdx.x);
}
template <typename T>
__global__ void __launch_bounds__(fft_threads<T>(), mid_min_blocks<T>()) k_mid_fwd_real(LevelArgs<T> a) {
  mid_body<T, MID_FWD_REAL, false>(a, (int)blockIdx.x);
}

// ------------------------------------------------------------------------------------
// Inverse strided pass: twiddle conj(W_m^{c k}), R1-point DIT per column, epilogue.
// ------------------------------------------------------------------------------------
// EPI: the epilogue, fixed at compile time (the launch selects the instance from a.epi).
template <typename T, int EPI>
__device__ __forceinline__ void inv_strided_body(const LevelArgs<T>& a, int blk) {
  constexpr int epi = EPI;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<T>* tab = reinterpret_cast<c2<T>*>(smem_raw);
  c2<T>* s = tab + tw_slots<T>();
  const int logR1 = a.logR1, logC = a.logC, logL = a.logL;
  const int C = 1 << logC;
  const int tile = 1 << (logR1 + logC);
  const int c0 = blk << logC;
  const bool fact = sizeof(T) == 4 && tile >= 2 * (int)blockDim.x &&
                    (long long)tile * C <= (long long)TW_TAB * blockDim.x;
  const TabRegs<T> tr = step_table_load<T>(a.twL);  // in flight with the tile's copies
  InterTw32 it{};
  const float2* t2 = reinterpret_cast<const float2*>(tab);
  if (fact) {
    // factored twiddles in the step-table slots until the transform needs them
    it = inter_tw32_setup(reinterpret_cast<float2*>(tab), c0, logC, logR1, a.logm);
    __syncthreads();
  }
  if constexpr (sizeof(T) == 4) {
    // asynchronous copies of the tile, then the twiddle in place (each thread its own slots)
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int t = e >> logC, cc = e & (C - 1);
      cp_async8(s + pad16(e), a.z + c0 + cc + (t << logL));
    }
    cp_async_wait_all();
    int j = 0;
    for (int e = threadIdx.x; e < tile; e += blockDim.x, ++j) {
      c2<T> w;
      if (fact) {
        const float2 wf = inter_tw32(it, t2, j);
        w = mk<T>((T)wf.x, (T)wf.y);
      } else {
        const int t = e >> logC, cc = e & (C - 1);
        const int kb = (int)brev_bits((unsigned)t, logR1);
        w = inter_tw<T>(a.twm, (c0 + cc) * kb, a.logm);
      }
      s[pad16(e)] = cmulc<T>(s[pad16(e)], w);
    }
  } else {
    for (int e0 = threadIdx.x; e0 < tile; e0 += 2 * UNROLL * blockDim.x) {
      c2<T> v[2 * UNROLL];
#pragma unroll
      for (int u = 0; u < 2 * UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        const int t = e >> logC, cc = e & (C - 1);
        if (e < tile) v[u] = a.z[c0 + cc + (t << logL)];
      }
#pragma unroll
      for (int u = 0; u < 2 * UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e >= tile) continue;
        const int t = e >> logC, cc = e & (C - 1);
        const int kb = (int)brev_bits((unsigned)t, logR1);
        s[pad16(e)] = cmulc<T>(v[u], inter_tw<T>(a.twm, (c0 + cc) * kb, a.logm));
      }
    }
  }
  __syncthreads();  // the factored twiddles' slots are free
  const c2<T>* tw = step_table_store<T>(tab, a.twL, tr);
  if constexpr (sizeof(T) == 4) __syncthreads();
  smem_dit<T, true>(s, logR1, logC, C, 1, tw, LOG_LMAX);
  const T w_o = a.x[a.N];
  const int half = 1 << (logR1 - 1);
  const int nout = half << logC;
  // FP32: the right-hand side pair (f_v, f_w) of each output arrives by asynchronous copies
  // into the slot of row t + R1/2 (the rows the embedding discards, free after the transform)
  constexpr bool ASYNC_F = sizeof(T) == 4 && EPI != EPI_APPLY;
  if constexpr (ASYNC_F) {
    for (int e = threadIdx.x; e < nout; e += blockDim.x) {
      const int t = e >> logC, cc = e & (C - 1);
      const int P = c0 + cc + (t << logL);
      if (P < a.N) {
        c2<T>* hi = s + pad16(e + nout);
        cp_async4(&hi->x, a.f + P);
        cp_async4(&hi->y, a.f + a.N + 1 + P);
      }
    }
    cp_async_wait_all();
  }
  for (int e0 = threadIdx.x; e0 < nout; e0 += UNROLL * blockDim.x) {
    EpiRaw<T> er[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int e = e0 + u * blockDim.x;
      const int t = e >> logC, cc = e & (C - 1);
      const int P = c0 + cc + (t << logL);
      if (e < nout && P < a.N) {
        if constexpr (ASYNC_F) {
          er[u] = epi_load<T>(a, P, EPI_APPLY);  // p, xi only
          const c2<T> fp = s[pad16(e + nout)];
          er[u].fv = fp.x;
          er[u].fw = fp.y;
          if (EPI == EPI_JACOBI) {
            er[u].xv = a.x[P];
            er[u].xw = a.x[a.N + 1 + P];
            if (a.bd) {
              er[u].wv = a.wvec[P];
              er[u].ww = a.wvec[a.N + 1 + P];
            }
          }
        } else {
          er[u] = epi_load<T>(a, P, epi);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int e = e0 + u * blockDim.x;
      const int t = e >> logC, cc = e & (C - 1);
      const int P = c0 + cc + (t << logL);
      if (e < nout && P < a.N) {
        const c2<T> y = s[pad16(e)];
        epi_store<T>(a, P, er[u], y.x, y.y, w_o, epi);
      }
    }
  }
  if (blk == 0 && threadIdx.x < 32) {
    T acc = 0;
    for (int i = threadIdx.x; i < a.nparts; i += 32) acc += a.partials[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) epi_middle<T>(a, acc, w_o, epi);
  }
}

template <typename T, int EPI, int MINB = fft_min_blocks<T>()>
__global__ void __launch_bounds__(fft_threads<T>(), MINB) k_inv_strided(LevelArgs<T> a) {
  pdl_wait();
  inv_strided_body<T, EPI>(a, (int)blockIdx.x);
}

// ------------------------------------------------------------------------------------
// The bottom of a V(1,1) cycle in one block: every level whose product fits one block
// (m <= 4096), from the level below the strided ones down to the coarsest and back up.
// Descent, level i: u = omega D^{-1} (restriction of the finer residual), r = f - A u
// (PRO_RESTRICT + EPI_RESID); coarsest: f = restriction, e = A^{-1} f; ascent: u + P e_c then
// one damped Jacobi sweep (PRO_PROLONG + EPI_JACOBI). Same arithmetic, buffers and order as
// the per-level launches, without one launch per product; the two modes are compile-time
// constants of the two loops, and two elements' loads per thread are batched instead of four
// (fewer registers; faster on these small levels).
// ------------------------------------------------------------------------------------
constexpr int BOTTOM_MAX_LEVELS = 12;
template <typename T> struct BottomPlan {
  int nlev;                              // product levels, finest first
  LevelArgs<T> pre[BOTTOM_MAX_LEVELS];
  LevelArgs<T> post[BOTTOM_MAX_LEVELS];
  const T* cinv;                         // coarsest inverse (nc x nc)
  int geo;                               // transfer (see LevelArgs)
  int nc;                                // coarsest unknowns
  // The bottom levels' vectors e, f, t and the coarsest f, e live in shared memory (element
  // offsets past the transform area of tr_elems complex values); only the input (the residual
  // of the level above, pre[0].rfine) and the output (post[0].y) are global.
  int tr_elems;
  int off_e[BOTTOM_MAX_LEVELS], off_f[BOTTOM_MAX_LEVELS], off_t[BOTTOM_MAX_LEVELS];
  int off_fc, off_ec;
};

template <typename T>
__device__ __forceinline__ void copy_args(LevelArgs<T>* dst, const LevelArgs<T>* src) {
  const int n = (int)(sizeof(LevelArgs<T>) / sizeof(int));
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    reinterpret_cast<int*>(dst)[i] = reinterpret_cast<const int*>(src)[i];
  __syncthreads();
}

template <typename T, bool NS>
__device__ __forceinline__ void vcycle_bottom_body(const BottomPlan<T>* bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<T>* tab = reinterpret_cast<c2<T>*>(smem_raw);
  c2<T>* s = tab + tw_slots<T>();
  __shared__ T red[FFT_THREADS / 32];
  __shared__ __align__(16) LevelArgs<T> la;
  const int nlev = bp->nlev;
  T* vec = reinterpret_cast<T*>(s + bp->tr_elems);
  const c2<T>* tw = step_table<T>(tab, bp->pre[0].twL);
  for (int i = 0; i < nlev; ++i) {
    copy_args<T>(&la, &bp->pre[i]);
    if (threadIdx.x == 0) {
      T* e = vec + bp->off_e[i];
      T* f = vec + bp->off_f[i];
      if (i > 0) la.rfine = vec + bp->off_t[i - 1];
      la.fout = f;
      la.xout = e;
      la.x = e;
      la.f = f;
      la.y = vec + bp->off_t[i];
    }
    __syncthreads();
    mid_core<T, MID_WHOLE, NS, 0, 0, PRO_RESTRICT, EPI_RESID, 2>(la, tw, s, red, 0, 0);
    __syncthreads();
  }
  {
    T* fs = vec + bp->off_fc;
    T* es = vec + bp->off_ec;
    const T* rc = vec + bp->off_t[nlev - 1];
    const int nc = bp->nc;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) fs[i] = restrict_at<T>(rc, i, (nc - 1) / 2, bp->geo);
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      T acc = 0;
      for (int j = 0; j < nc; ++j) acc = fma(bp->cinv[(long long)i * nc + j], fs[j], acc);
      es[i] = acc;
    }
    __syncthreads();
  }
  for (int i = nlev - 1; i >= 0; --i) {
    copy_args<T>(&la, &bp->post[i]);
    if (threadIdx.x == 0) {
      T* e = vec + bp->off_e[i];
      la.x = e;
      la.xout = e;
      la.f = vec + bp->off_f[i];
      la.ec = (i + 1 == nlev) ? vec + bp->off_ec : vec + bp->off_t[i + 1];
      if (i > 0) la.y = vec + bp->off_t[i];  // post[0].y: the global t of the top bottom level
    }
    __syncthreads();
    mid_core<T, MID_WHOLE, NS, 0, 0, PRO_PROLONG, EPI_JACOBI, 2>(la, tw, s, red, 0, 0);
    __syncthreads();
  }
}

template <typename T, bool NS>
__global__ void __launch_bounds__(fft_threads<T>(), 1) k_vcycle_bottom(const BottomPlan<T>* bp) {
  pdl_wait();
  vcycle_bottom_body<T, NS>(bp);
}

// ------------------------------------------------------------------------------------
// Spectra: stored value = (transform of the circulant column) / (2m) at every position.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_extract_real(const c2<T>* z, T* out, long long m, T scale) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < m) out[i] = z[i].x * scale;
}
template <typename T>
__global__ void k_extract_cplx(const c2<T>* z, c2<T>* out, long long m, T scale) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < m) out[i] = mk<T>(z[i].x * scale, z[i].y * scale);
}

// ------------------------------------------------------------------------------------
// V-cycle pieces (Algorithm 2)
// ------------------------------------------------------------------------------------
// Correction with P = 2 (I_k^{k-1})^T: e[2I+1] += ec[I], e[2I], e[2I+2] += ec[I] / 2.
template <typename T>
__global__ void k_prolong_add(T* e, const T* ec, long long nf, int geo) {
  pdl_wait();
  const long long nc = (nf - 1) / 2;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nf;
       j += (long long)gridDim.x * blockDim.x) {
    T add;
    if (geo) {  // geometric transfer: see prolong_load
      const int N = (int)nc, Nc = (N - 1) / 2;
      if (j < N) {
        add = ec[coarse_of_position((int)j + 1, Nc)];
      } else {
        const int u = (int)j - N + 1;
        const T lo = (u >= 2) ? ec[coarse_of_position(u - 1, Nc)] : (T)0;
        const T hi = (u <= N) ? ec[coarse_of_position(u, Nc)] : (T)0;
        add = (T)0.5 * (lo + hi);
      }
    } else if (j & 1) {
      add = ec[(j - 1) / 2];
    } else {
      const long long I = j / 2;
      const T lo = (I - 1 >= 0) ? ec[I - 1] : (T)0;
      const T hi = (I < nc) ? ec[I] : (T)0;
      add = (T)0.5 * (lo + hi);
    }
    e[j] += add;
  }
}

// Coarsest level: e = A_kc^{-1} f with the inverse formed on the host (n <= 255). With
// rfine != nullptr the right-hand side is first restricted from the finer residual (and
// stored in f).
template <typename T>
__global__ void k_coarse_solve(const T* inv, T* f, const T* rfine, T* e, int n, int geo) {
  __shared__ T fs[256];
  pdl_wait();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (rfine) {
      fs[i] = restrict_at<T>(rfine, i, (n - 1) / 2, geo);
      f[i] = fs[i];
    } else {
      fs[i] = f[i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T acc = 0;
    for (int j = 0; j < n; ++j) acc = fma(inv[(long long)i * n + j], fs[j], acc);
    e[i] = acc;
  }
}

template <typename T>
__global__ void k_axpy(T* u, const T* e, long long n) {
  pdl_wait();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    u[i] += e[i];
}

// Right-hand side of one step of eq. (5.1) for the shifted system (sigma I + A) U^k = b:
// b = hs (4 u1 - 3 u2 + 4/3 u3 - 1/4 u4) + gs g  (u_j = U^{k-j}).
static __global__ void k_bdf4_rhs(double* b, const double* u1, const double* u2, const double* u3,
                           const double* u4, double hs, const double* g, double gs, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double hist = 4.0 * u1[i] - 3.0 * u2[i] + (4.0 / 3.0) * u3[i] - 0.25 * u4[i];
    b[i] = hs * hist + (g ? gs * g[i] : 0.0);
  }
}

template <typename T>
__global__ void k_copy(const T* src, T* dst, long long n) {
  pdl_wait();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Mixed precision: the FP64 residual r enters the FP32 V-cycles scaled to unit RMS,
// f = r * sqrt(n / ||r||^2), and the FP32 correction e comes back as u += e / that scale.
static __global__ void k_to_f32_scaled(const double* r, float* f, long long n, const double* sumsq) {
  pdl_wait();
  const double ss = sumsq[0];
  const double s = (ss > 0.0) ? sqrt((double)n / ss) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    f[i] = (float)(r[i] * s);
}
static __global__ void k_axpy_f32_scaled(double* u, const float* e, long long n, const double* sumsq) {
  pdl_wait();
  const double inv = sqrt(sumsq[0] / (double)n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = fma((double)e[i], inv, u[i]);
}
static __global__ void k_round_f32(const double* in, float* out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// Deterministic two-stage sum of squares: fixed grid, fixed order.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_sumsq_partial(const T* r, long long n,
                                                            double* part) {
  __shared__ double red[NTHREADS / 32];
  pdl_wait();
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)r[i];
    acc = fma(v, v, acc);
  }
  const double s = block_sum<double>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
static __global__ void k_sumsq_final(const double* part, int np, double* out) {
  pdl_wait();
  double acc = 0;
  for (int i = threadIdx.x; i < np; i += 32) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) out[0] = acc;
}

// Launches of the strided passes with the prologue / epilogue instance chosen from the
// arguments' runtime mode, and (FP32) the occupancy instance from the level size.
template <typename T, int MB>
inline void launch_fwd_strided_mb(const LevelArgs<T>& a, int blocks, size_t smem, cudaStream_t s) {
  const int nt = fft_threads<T>();
  switch (a.pro) {
    case PRO_SMOOTH: launch_k(k_fwd_strided<T, IN_PACK, PRO_SMOOTH, MB>, blocks, nt, smem, s, a); break;
    case PRO_RESTRICT: launch_k(k_fwd_strided<T, IN_PACK, PRO_RESTRICT, MB>, blocks, nt, smem, s, a); break;
    case PRO_PROLONG: launch_k(k_fwd_strided<T, IN_PACK, PRO_PROLONG, MB>, blocks, nt, smem, s, a); break;
    default: launch_k(k_fwd_strided<T, IN_PACK, PRO_NONE, MB>, blocks, nt, smem, s, a); break;
  }
}
template <typename T>
inline void launch_fwd_strided(const LevelArgs<T>& a, int blocks, size_t smem, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.logm <= LOG_M_HIGH_OCC) {
      launch_fwd_strided_mb<T, F32_HIGH_OCC_BLOCKS>(a, blocks, smem, s);
      return;
    }
  }
  launch_fwd_strided_mb<T, fft_min_blocks<T>()>(a, blocks, smem, s);
}
template <typename T, int MB>
inline void launch_inv_strided_mb(const LevelArgs<T>& a, int blocks, size_t smem, cudaStream_t s) {
  const int nt = fft_threads<T>();
  switch (a.epi) {
    case EPI_RESID: launch_k(k_inv_strided<T, EPI_RESID, MB>, blocks, nt, smem, s, a); break;
    case EPI_JACOBI: launch_k(k_inv_strided<T, EPI_JACOBI, MB>, blocks, nt, smem, s, a); break;
    default: launch_k(k_inv_strided<T, EPI_APPLY, MB>, blocks, nt, smem, s, a); break;
  }
}
template <typename T>
inline void launch_inv_strided(const LevelArgs<T>& a, int blocks, size_t smem, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.logm <= LOG_M_HIGH_OCC) {
      launch_inv_strided_mb<T, F32_HIGH_OCC_BLOCKS>(a, blocks, smem, s);
      return;
    }
  }
  launch_inv_strided_mb<T, fft_min_blocks<T>()>(a, blocks, smem, s);
}
// The contiguous-block kernel: the instance with L fixed at compile time for the FP32 levels
// with L = 2^10 .. 2^12 (the largest ones), the general one otherwise.
template <typename T, bool NS>
inline void launch_mid_pair(const LevelArgs<T>& a, int blocks, size_t smem, cudaStream_t s) {
  const int nt = fft_threads<T>();
  if (sizeof(T) == 4 && a.logL == 12) launch_k(k_mid_pair<T, NS, 12>, blocks, nt, smem, s, a);
  else if (sizeof(T) == 4 && a.logL == 11) launch_k(k_mid_pair<T, NS, 11>, blocks, nt, smem, s, a);
  else if (sizeof(T) == 4 && a.logL == 10) launch_k(k_mid_pair<T, NS, 10>, blocks, nt, smem, s, a);
  else launch_k(k_mid_pair<T, NS>, blocks, nt, smem, s, a);
}
template <typename T, bool NS>
inline cudaError_t mid_pair_smem_attrs(int bytes) {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if constexpr (sizeof(T) == 4) {
    if ((e = cudaFuncSetAttribute(k_mid_pair<T, NS, 12>, A, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_mid_pair<T, NS, 11>, A, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_mid_pair<T, NS, 10>, A, bytes)) != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_mid_pair<T, NS>, A, bytes);
}

// Raise the dynamic shared-memory limit of every strided-pass instance.
template <typename T, int MB>
inline cudaError_t strided_smem_attrs_mb(int bytes) {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_fwd_strided<T, IN_PACK, PRO_NONE, MB>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_strided<T, IN_PACK, PRO_SMOOTH, MB>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_strided<T, IN_PACK, PRO_RESTRICT, MB>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_strided<T, IN_PACK, PRO_PROLONG, MB>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_inv_strided<T, EPI_APPLY, MB>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_inv_strided<T, EPI_RESID, MB>, A, bytes)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_inv_strided<T, EPI_JACOBI, MB>, A, bytes);
}
template <typename T>
inline cudaError_t strided_smem_attrs(int bytes) {
  if constexpr (sizeof(T) == 4) {
    const cudaError_t e = strided_smem_attrs_mb<T, F32_HIGH_OCC_BLOCKS>(bytes);
    if (e != cudaSuccess) return e;
  }
  return strided_smem_attrs_mb<T, fft_min_blocks<T>()>(bytes);
}

}  // namespace tpc
