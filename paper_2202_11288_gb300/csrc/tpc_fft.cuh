// Device building blocks: complex arithmetic and in-shared-memory radix-2 FFT stages.
//
// Transform convention (section 3.2): forward F x = sum_j x_j W^{jk}, W = exp(-2 pi i / m),
// computed decimation-in-frequency (natural order in, bit-reversed order out); the inverse is
// decimation-in-time with conjugate twiddles (bit-reversed in, natural out) and no 1/m factor
// (the 1/m is folded into the stored spectra). The product C x = ifft(fft(c) .* fft(x)) of a
// circulant embedding (eq. ccs3.4) never needs the bit-reversal permutation: spectra are
// stored in the same bit-reversed order as the forward output.
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
template <typename T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
// a * b
template <typename T> __device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __device__ __forceinline__ c2<T> cmulc(c2<T> a, c2<T> b) {
  return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Radix-2 DIF stages of length 2^logL on 2^logCount independent sequences held in shared
// memory: element t of sequence q lives at s[q * qs + t * ts]. tw[j] = exp(-2 pi i j / Lmax),
// j < Lmax / 2, Lmax = 2^logLmax >= 2^logL. QFAST: consecutive threads take consecutive
// sequences (for tiles whose sequences are interleaved columns); otherwise consecutive
// butterflies of one sequence. Ends with __syncthreads().
template <typename T, bool QFAST>
__device__ __forceinline__ void smem_dif(c2<T>* s, int logL, int logCount, int ts, int qs,
                                         const c2<T>* __restrict__ tw, int logLmax) {
  if (logL == 0) return;
  const int nbf = 1 << (logL - 1 + logCount);
  const int qmask = (1 << logCount) - 1;
  const int bmask = (1 << (logL - 1)) - 1;
  for (int logh = logL - 1; logh >= 0; --logh) {
    const int hh = 1 << logh;
    const int tsh = logLmax - logh - 1;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
      int q, bb;
      if (QFAST) {
        q = b & qmask;
        bb = b >> logCount;
      } else {
        bb = b & bmask;
        q = b >> (logL - 1);
      }
      const int i = bb & (hh - 1);
      const int t0 = ((bb >> logh) << (logh + 1)) + i;
      c2<T>* p0 = s + q * qs + t0 * ts;
      c2<T>* p1 = p0 + hh * ts;
      const c2<T> u = *p0, v = *p1;
      const c2<T> w = __ldg(tw + (i << tsh));
      *p0 = cadd<T>(u, v);
      *p1 = cmul<T>(csub<T>(u, v), w);
    }
    __syncthreads();
  }
}

// The transposed (inverse) network: radix-2 DIT stages with conjugate twiddles,
// bit-reversed in, natural out, unnormalised. Ends with __syncthreads().
template <typename T, bool QFAST>
__device__ __forceinline__ void smem_dit(c2<T>* s, int logL, int logCount, int ts, int qs,
                                         const c2<T>* __restrict__ tw, int logLmax) {
  if (logL == 0) return;
  const int nbf = 1 << (logL - 1 + logCount);
  const int qmask = (1 << logCount) - 1;
  const int bmask = (1 << (logL - 1)) - 1;
  for (int logh = 0; logh < logL; ++logh) {
    const int hh = 1 << logh;
    const int tsh = logLmax - logh - 1;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
      int q, bb;
      if (QFAST) {
        q = b & qmask;
        bb = b >> logCount;
      } else {
        bb = b & bmask;
        q = b >> (logL - 1);
      }
      const int i = bb & (hh - 1);
      const int t0 = ((bb >> logh) << (logh + 1)) + i;
      c2<T>* p0 = s + q * qs + t0 * ts;
      c2<T>* p1 = p0 + hh * ts;
      const c2<T> u = *p0;
      const c2<T> v = cmulc<T>(*p1, __ldg(tw + (i << tsh)));
      *p0 = cadd<T>(u, v);
      *p1 = csub<T>(u, v);
    }
    __syncthreads();
  }
}

// Bit reversal of the low `bits` bits (bits >= 1).
__device__ __forceinline__ unsigned brev_bits(unsigned x, int bits) {
  return __brev(x) >> (32 - bits);
}

}  // namespace tpc
