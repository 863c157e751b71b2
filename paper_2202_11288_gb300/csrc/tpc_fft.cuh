// Device building blocks: complex arithmetic and in-shared-memory FFTs built from radix-16
// (and smaller) register butterflies.
//
// Transform convention (section 3.2): forward F x = sum_j x_j W^{jk}, W = exp(-2 pi i / m),
// computed decimation-in-frequency (natural order in, bit-reversed order out); the inverse is
// decimation-in-time with conjugate twiddles (bit-reversed in, natural out) and no 1/m factor
// (the 1/m is folded into the stored spectra). The product C x = ifft(fft(c) .* fft(x)) of a
// circulant embedding (eq. (3.4)) never needs the bit-reversal permutation: spectra are
// stored in the same bit-reversed order as the forward output.
//
// A DIF step of radix R on sub-blocks of length S treats each sub-block as R rows of S/R
// columns: for column c it takes the R entries c + t S/R, applies the R-point DIF network
// (result slot t holds frequency bitrev_R(t)) and multiplies slot t by W_S^{c bitrev_R(t)};
// this equals log2(R) consecutive radix-2 DIF stages. The DIT step is its exact transpose.
#pragma once

#include <cuda_runtime.h>

namespace tpc {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };
template <typename T> using c2 = typename V2<T>::t;

template <typename T> __device__ __forceinline__ c2<T> mk(T a, T b) {
  c2<T> r;
  r.x = a;
  r.y = b;
  return r;
}
// Complex add / subtract. FP32 uses the packed two-lane instructions (add and fma on a pair of
// floats in one instruction; a - b is fma(b, -1, a), the same rounding as the subtraction).
template <typename T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) {
  if constexpr (sizeof(T) == 4) return __fadd2_rn(a, b);
  else return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) {
  if constexpr (sizeof(T) == 4) return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
  else return mk<T>(a.x - b.x, a.y - b.y);
}
// a * b
template <typename T> __device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __device__ __forceinline__ c2<T> cmulc(c2<T> a, c2<T> b) {
  return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Shared-memory index with one padding slot every 16 entries (keeps the strided accesses of
// the butterfly steps on distinct banks).
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_size(int n) { return n + (n >> 4); }

// x * exp(-2 pi i e / 16) for a compile-time e in [0, 16). The constants are cos and sin of
// multiples of pi/8: cos(pi/8) = sqrt(2 + sqrt 2) / 2, sin(pi/8) = sqrt(2 - sqrt 2) / 2,
// cos(pi/4) = sqrt(2) / 2.
template <typename T, int E>
__device__ __forceinline__ c2<T> mul_w16(c2<T> x) {
  constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173;
  constexpr double H = 0.70710678118654752440;
  if constexpr (E == 0) return x;
  else if constexpr (E == 4) return mk<T>(x.y, -x.x);           // * (-i)
  else if constexpr (E == 8) return mk<T>(-x.x, -x.y);          // * (-1)
  else if constexpr (E == 12) return mk<T>(-x.y, x.x);          // * (+i)
  else if constexpr (E == 2) return mk<T>((T)H * (x.x + x.y), (T)H * (x.y - x.x));
  else if constexpr (E == 6) return mk<T>((T)H * (x.y - x.x), -(T)H * (x.x + x.y));
  else if constexpr (E == 10) return mk<T>(-(T)H * (x.x + x.y), (T)H * (x.x - x.y));
  else if constexpr (E == 14) return mk<T>((T)H * (x.x - x.y), (T)H * (x.x + x.y));
  else {
    // general angle: w = (cos, -sin) of 2 pi E / 16
    constexpr double wr = (E == 1) ? C1 : (E == 3) ? S1 : (E == 5) ? -S1 : (E == 7) ? -C1
                        : (E == 9) ? -C1 : (E == 11) ? -S1 : (E == 13) ? S1 : C1;
    constexpr double wi = (E == 1) ? -S1 : (E == 3) ? -C1 : (E == 5) ? -C1 : (E == 7) ? -S1
                        : (E == 9) ? S1 : (E == 11) ? C1 : (E == 13) ? C1 : S1;
    return cmul<T>(x, mk<T>((T)wr, (T)wi));
  }
}

// R-point DIF network on registers: natural order in, slot t = frequency bitrev_R(t) out.
// Butterfly (B + I, B + I + H) of the stage with half-size H uses W_{2H}^I = W_16^{8 I / H}.
template <typename T, int H, int B, int I>
__device__ __forceinline__ void dif_bfly(c2<T>* v) {
  if constexpr (I < H) {
    const c2<T> u = v[B + I], w = v[B + I + H];
    v[B + I] = cadd<T>(u, w);
    v[B + I + H] = mul_w16<T, (8 * I) / H>(csub<T>(u, w));
    dif_bfly<T, H, B, I + 1>(v);
  }
}
template <typename T, int R, int H, int B>
__device__ __forceinline__ void dif_blocks(c2<T>* v) {
  if constexpr (B < R) {
    dif_bfly<T, H, B, 0>(v);
    dif_blocks<T, R, H, B + 2 * H>(v);
  }
}
template <typename T, int R, int H = R / 2>
__device__ __forceinline__ void reg_dif_stage(c2<T>* v) {
  if constexpr (H >= 1) {
    dif_blocks<T, R, H, 0>(v);
    reg_dif_stage<T, R, H / 2>(v);
  }
}

// Transposed network: slot t = frequency bitrev_R(t) in, natural order out, conjugate
// twiddles (the inverse up to a factor R).
template <typename T, int H, int B, int I>
__device__ __forceinline__ void dit_bfly(c2<T>* v) {
  if constexpr (I < H) {
    const c2<T> u = v[B + I];
    const c2<T> w = mul_w16<T, (16 - (8 * I) / H) % 16>(v[B + I + H]);
    v[B + I] = cadd<T>(u, w);
    v[B + I + H] = csub<T>(u, w);
    dit_bfly<T, H, B, I + 1>(v);
  }
}
template <typename T, int R, int H, int B>
__device__ __forceinline__ void dit_blocks(c2<T>* v) {
  if constexpr (B < R) {
    dit_bfly<T, H, B, 0>(v);
    dit_blocks<T, R, H, B + 2 * H>(v);
  }
}
template <typename T, int R, int H = 1>
__device__ __forceinline__ void reg_dit_stage(c2<T>* v) {
  if constexpr (H < R) {
    dit_blocks<T, R, H, 0>(v);
    reg_dit_stage<T, R, H * 2>(v);
  }
}

// Twiddles of the in-shared-memory steps: W_4096^e = exp(-2 pi i e / 4096) for e < 4096 from
// an octant table tab[j] = W_4096^j, j <= 512, held in shared memory, using the exact
// symmetries W^{1024 q + r} = (-i)^q W^r and W^r = -i conj(W^{1024 - r}).
constexpr int TW_TAB = 520;  // octant table slots (513 entries, rounded for alignment)
// Shared-memory slots reserved for the step twiddles ahead of the data: FP32 keeps the octant
// table there; FP64 reads its table from global memory and reserves nothing.
template <typename T> __host__ __device__ constexpr int tw_slots() {
  return sizeof(T) == 8 ? 0 : TW_TAB;
}
template <typename T>
__device__ __forceinline__ c2<T> tw4096(const c2<T>* __restrict__ tab, int e) {
  const int q = (e >> 10) & 3, r = e & 1023;
  const bool flip = r > 512;
  const c2<T> t = tab[flip ? 1024 - r : r];
  const T a = flip ? -t.y : t.x, b = flip ? -t.x : t.y;  // W^r
  // times (-i)^q
  const T re = (q == 0) ? a : (q == 1) ? b : (q == 2) ? -a : -b;
  const T im = (q == 0) ? b : (q == 1) ? -a : (q == 2) ? -b : a;
  return mk<T>(re, im);
}
// The twiddle table the steps use: FP32 copies the octant of the global W_4096 table into
// shared memory (all threads; ends with a barrier); FP64 uses the global table directly.
template <typename T>
__device__ __forceinline__ const c2<T>* step_table(c2<T>* tab, const c2<T>* __restrict__ g) {
  if constexpr (sizeof(T) == 8) {
    return g;
  } else {
    for (int j = threadIdx.x; j <= 512; j += blockDim.x) tab[j] = g[j];
    __syncthreads();
    return tab;
  }
}

// FP32: the same copy as asynchronous copies issued together with a tile's, no barrier; the
// caller waits for its copies (cp.async.wait_all) and passes a barrier before the first step.
template <typename T>
__device__ __forceinline__ const c2<T>* step_table_issue(c2<T>* tab, const c2<T>* __restrict__ g) {
  if constexpr (sizeof(T) == 8) {
    return g;
  } else {
    for (int j = threadIdx.x; j <= 512; j += blockDim.x) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(tab + j);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d),
                   "l"(__cvta_generic_to_global(g + j))
                   : "memory");
    }
    return tab;
  }
}
// FP32: a thread's share of the table (entries threadIdx.x + k * blockDim.x), read early into
// registers while the slots still hold something else, stored by step_table_store.
constexpr int TW_PER_THREAD = (513 + 255) / 256;  // blockDim.x >= 256
template <typename T> struct TabRegs { c2<T> v[TW_PER_THREAD]; };
template <typename T>
__device__ __forceinline__ TabRegs<T> step_table_load(const c2<T>* __restrict__ g) {
  TabRegs<T> r{};
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < TW_PER_THREAD; ++k) {
      const int j = threadIdx.x + k * blockDim.x;
      if (j <= 512) r.v[k] = g[j];
    }
  }
  return r;
}
// Stores the loaded share (no barrier: the caller passes one before the first step).
template <typename T>
__device__ __forceinline__ const c2<T>* step_table_store(c2<T>* tab, const c2<T>* __restrict__ g,
                                                         const TabRegs<T>& r) {
  if constexpr (sizeof(T) == 8) {
    return g;
  } else {
#pragma unroll
    for (int k = 0; k < TW_PER_THREAD; ++k) {
      const int j = threadIdx.x + k * blockDim.x;
      if (j <= 512) tab[j] = r.v[k];
    }
    return tab;
  }
}

template <int R> __device__ __forceinline__ int brev_r(int t) {
  return (int)(__brev((unsigned)t) >> (32 - (R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1)));
}

// One radix-R step on all sub-blocks of length 2^logS of 2^logCount sequences of length
// 2^logL held in shared memory (element t of sequence q at pad16(q * qs + t * ts)).
// tw: the full W_4096 table in global memory (FP64) or the octant table in shared memory
// (FP32), see step_tw; 2^logLmax = 4096. QFAST: consecutive threads take
// consecutive sequences first (interleaved column tiles), else consecutive columns.
// W_4096^e for the in-shared-memory steps: FP64 (bound by the FP64 pipe, L1 mostly free)
// reads the full 4096-entry table from global memory through L1; FP32 reads the octant table
// in shared memory (a full table there is read at bank-conflicting strides, W^{c k} with c
// varying across the lanes).
template <typename T>
__device__ __forceinline__ c2<T> step_tw(const c2<T>* __restrict__ tw, int e) {
  if constexpr (sizeof(T) == 8) return __ldg(tw + e);
  else return tw4096<T>(tw, e);  // octant table in shared memory
}

// Twiddles W^{c k}, k = 1..R-1, of one task. FP64: one exact table read each. FP32: exact
// reads of W^c, W^{2c}, W^{4c}, W^{8c} and the other powers as products of those (at most three
// roundings), which keeps the FP32 steps' instruction count and table reads low.
template <typename T, int R>
__device__ __forceinline__ void task_twiddles(const c2<T>* __restrict__ tw, int c, int twsh,
                                              c2<T>* pw) {
  const int ec = c << twsh;
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int k = 1; k < R; ++k) pw[k] = step_tw<T>(tw, ec * k);
  } else {
#pragma unroll
    for (int k = 1; k < R; k <<= 1) pw[k] = step_tw<T>(tw, ec * k);
#pragma unroll
    for (int k = 3; k < R; ++k) {
      if ((k & (k - 1)) == 0) continue;
      const int hb = 1 << (31 - __clz(k));
      pw[k] = cmul<T>(pw[k - hb], pw[hb]);
    }
  }
}

template <typename T, int R, bool QFAST, bool INV>
__device__ __forceinline__ void fft_step(c2<T>* s, int logS, int logL, int logCount, int ts,
                                         int qs, const c2<T>* __restrict__ tw, int logLmax) {
  constexpr int logR = (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1;
  const int logCols = logS - logR;
  const int logSb = logL - logS;
  const int ntask = 1 << (logCount + logSb + logCols);
  const int twsh = logLmax - logS;
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    int q, c, sb;
    if (QFAST) {
      q = task & ((1 << logCount) - 1);
      const int rest = task >> logCount;
      c = rest & ((1 << logCols) - 1);
      sb = rest >> logCols;
    } else {
      c = task & ((1 << logCols) - 1);
      const int rest = task >> logCols;
      sb = rest & ((1 << logSb) - 1);
      q = rest >> logSb;
    }
    const int base = q * qs + ((sb << logS) + c) * ts;
    const int step = ts << logCols;
    // pad16(base + t step) = pad16(base) + t pstep when step is a multiple of 16 (pstep =
    // step + step / 16) or when all R entries lie in one group of 16 slots (pstep = step);
    // otherwise each index is padded on its own. The test is uniform over a step's tasks
    // except in the last case, and the two loops keep the fast one free of the general form.
    const int pb = pad16(base);
    int pstep = -1;
    if ((step & 15) == 0) pstep = step + (step >> 4);
    else if ((base & 15) + (R - 1) * step < 16) pstep = step;
    c2<T> v[R];
    if (pstep >= 0) {
#pragma unroll
      for (int t = 0; t < R; ++t) v[t] = s[pb + t * pstep];
    } else {
#pragma unroll
      for (int t = 0; t < R; ++t) v[t] = s[pad16(base + t * step)];
    }
    if (INV) {
      if (logCols > 0) {
        c2<T> pw[R];
        task_twiddles<T, R>(tw, c, twsh, pw);
#pragma unroll
        for (int t = 1; t < R; ++t) v[t] = cmulc<T>(v[t], pw[brev_r<R>(t)]);
      }
      reg_dit_stage<T, R>(v);
    } else {
      reg_dif_stage<T, R>(v);
      if (logCols > 0) {
        c2<T> pw[R];
        task_twiddles<T, R>(tw, c, twsh, pw);
#pragma unroll
        for (int t = 1; t < R; ++t) v[t] = cmul<T>(v[t], pw[brev_r<R>(t)]);
      }
    }
    if (pstep >= 0) {
#pragma unroll
      for (int t = 0; t < R; ++t) s[pb + t * pstep] = v[t];
    } else {
#pragma unroll
      for (int t = 0; t < R; ++t) s[pad16(base + t * step)] = v[t];
    }
  }
}

// Radices of the steps of a 2^logL transform: as many of the largest radix (2^TPC_LOG_RMAX,
// default 16) as fit, then the remainder.
#ifndef TPC_LOG_RMAX
#define TPC_LOG_RMAX 4
#endif
__device__ __forceinline__ int step_radix_log(int logL, int idx) {
  const int nfull = logL / TPC_LOG_RMAX;
  return idx < nfull ? TPC_LOG_RMAX : (logL % TPC_LOG_RMAX);
}
__device__ __forceinline__ int num_steps(int logL) {
  return logL / TPC_LOG_RMAX + ((logL % TPC_LOG_RMAX) ? 1 : 0);
}

template <typename T, bool QFAST, bool INV>
__device__ __forceinline__ void dispatch_step(int r, c2<T>* s, int logS, int logL, int logCount,
                                              int ts, int qs, const c2<T>* tw, int logLmax) {
  switch (r) {
    case 4: fft_step<T, 16, QFAST, INV>(s, logS, logL, logCount, ts, qs, tw, logLmax); break;
    case 3: fft_step<T, 8, QFAST, INV>(s, logS, logL, logCount, ts, qs, tw, logLmax); break;
    case 2: fft_step<T, 4, QFAST, INV>(s, logS, logL, logCount, ts, qs, tw, logLmax); break;
    default: fft_step<T, 2, QFAST, INV>(s, logS, logL, logCount, ts, qs, tw, logLmax); break;
  }
}

// Forward DIF of length 2^logL on 2^logCount sequences in shared memory (natural in,
// bit-reversed out). Ends with __syncthreads().
template <typename T, bool QFAST>
__device__ __forceinline__ void smem_dif(c2<T>* s, int logL, int logCount, int ts, int qs,
                                         const c2<T>* __restrict__ tw, int logLmax) {
  int logS = logL;
  const int ns = num_steps(logL);
  for (int k = 0; k < ns; ++k) {
    const int r = step_radix_log(logL, k);
    dispatch_step<T, QFAST, false>(r, s, logS, logL, logCount, ts, qs, tw, logLmax);
    __syncthreads();
    logS -= r;
  }
}

// Inverse: the DIF steps transposed, in reverse order (bit-reversed in, natural out,
// unnormalised). Ends with __syncthreads().
template <typename T, bool QFAST>
__device__ __forceinline__ void smem_dit(c2<T>* s, int logL, int logCount, int ts, int qs,
                                         const c2<T>* __restrict__ tw, int logLmax) {
  const int ns = num_steps(logL);
  int logS = 0;
  for (int k = ns - 1; k >= 0; --k) {
    const int r = step_radix_log(logL, k);
    logS += r;
    dispatch_step<T, QFAST, true>(r, s, logS, logL, logCount, ts, qs, tw, logLmax);
    __syncthreads();
  }
}

// Bit reversal of the low `bits` bits (bits >= 1).
__device__ __forceinline__ unsigned brev_bits(unsigned x, int bits) {
  return __brev(x) >> (32 - bits);
}

}  // namespace tpc
