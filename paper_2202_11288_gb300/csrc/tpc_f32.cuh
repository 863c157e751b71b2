// FP32 product of the largest levels (m = 2^20 .. 2^23) with register-resident transform steps.
//
// Same mathematics and data layout as the general kernels of tpc_kernels.cuh (m = R1 * L;
// forward: R1-point DIF of each column, twiddle W_m^{c bitrev(t)}, L-point DIF of each row block;
// the 2x2 spectral product of eq. (3.7) per frequency pair; the transposed inverse), so the
// spectra, the work array z and the results are interchangeable with theirs. What differs is
// where the data lives between the radix steps:
//   * the first step of a pass works on values loaded from global memory into registers and
//     the last step writes its results from registers to global memory: a pass moves its tile
//     through shared memory twice instead of four or five times;
//   * step twiddles W_S^{c bitrev_16(t)} come from one precomputed FP32 table (rounded once from
//     FP64) laid out [t][c], so the lanes of a warp read consecutive entries;
//   * in the contiguous-block kernel a thread holds a group of the last forward step and the
//     group of its mirror block that holds the partners of the group's frequencies, so the
//     spectral product and the first inverse step run in registers;
//   * the forward pass stores, and the inverse pass loads, whole 32-byte rows of its four
//     columns (two 16-byte accesses per row).
// Radix steps: L = 16 * 16 * r_s and R1 = 16 * 16 * r_s' with r_s, r_s' in {4, 8, 16}: two
// radix-16 steps, then radix r_s on groups of r_s consecutive positions.
#pragma once

#include "tpc_kernels.cuh"

namespace tpc {
namespace f32p {

constexpr int NT_STRIDED = 256;  // threads of the strided passes
// Resident blocks per SM the strided passes are compiled for, and whether a row moves as one
// 32-byte access (1) or as two 16-byte ones (0).
#ifndef TPC_F32_STRIDED_MINB
#define TPC_F32_STRIDED_MINB 2
#endif
#ifndef TPC_F32_ROW_V8
#define TPC_F32_ROW_V8 1
#endif
constexpr int CT = 4;            // columns per strided tile
constexpr int LOG_CT = 2;

// Step twiddle table: for S = 2^s, s = 5..12, entries T_S[t][c] = W_S^{c bitrev_16(t)},
// t < 16, c < S / 16, at offset (S - 32) + t (S / 16) + c. 8160 complex values.
constexpr int STEP_TW_ENTRIES = 8160;
__host__ __device__ constexpr int steptw_off(int logS) { return (1 << logS) - 32; }

// Shared-memory index of position i of a contiguous block: 16 bytes of padding after every 16
// complex values (keeps 16-byte alignment; conflict-free for the access patterns below).
__device__ __forceinline__ int pidx(int i) { return i + 2 * (i >> 4); }
__host__ __device__ constexpr int pblock(int n) { return n + 2 * (n >> 4); }

// Strided tile (float2 units): row-major, the four columns of a row side by side, 16 bytes of
// padding after every group of RS rows (RS = R1 / 256, the radix of the last step). The radix-16
// steps then touch 256 contiguous bytes per warp access and the last step's 16-byte accesses
// (one group per lane) fall on distinct banks.
template <int LRS>
__device__ __forceinline__ int tidx(int row, int cc) { return 4 * row + cc + 2 * (row >> LRS); }
// R1 / RS = 256 groups, so a tile holds 4 R1 + 512 float2.
__host__ __device__ constexpr int tile_size(int R1) { return 4 * R1 + 512; }

// 32-byte row of four complex values (one full sector) to / from global memory in one access;
// the address must be 32-byte aligned.
__device__ __forceinline__ void st_row(float2* dst, float2 a, float2 b, float2 c, float2 d) {
#if !TPC_F32_ROW_V8
  reinterpret_cast<float4*>(dst)[0] = make_float4(a.x, a.y, b.x, b.y);
  reinterpret_cast<float4*>(dst)[1] = make_float4(c.x, c.y, d.x, d.y);
  return;
#endif
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "f"(a.x),
               "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
               : "memory");
}
__device__ __forceinline__ void ld_row(const float2* src, float2& a, float2& b, float2& c,
                                       float2& d) {
#if !TPC_F32_ROW_V8
  const float4 t0 = reinterpret_cast<const float4*>(src)[0], t1 = reinterpret_cast<const float4*>(src)[1];
  a = make_float2(t0.x, t0.y);
  b = make_float2(t0.z, t0.w);
  c = make_float2(t1.x, t1.y);
  d = make_float2(t1.z, t1.w);
  return;
#endif
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y), "=f"(c.x), "=f"(c.y), "=f"(d.x),
                 "=f"(d.y)
               : "l"(src));
}

// R-point DIF / DIT register networks (tpc_fft.cuh), R in {4, 8, 16}.
template <int R>
__device__ __forceinline__ void dif(float2* v) { reg_dif_stage<float, R>(v); }
template <int R>
__device__ __forceinline__ void dit(float2* v) { reg_dit_stage<float, R>(v); }

// 16-point DIF whose inputs 8..15 are zero (the zero half of the circulant embedding): the
// first radix-2 stage reduces to v[i + 8] = W_16^i v[i].
__device__ __forceinline__ void dif16_zero_upper(float2* v) {
  v[15] = mul_w16<float, 7>(v[7]);
  v[14] = mul_w16<float, 6>(v[6]);
  v[13] = mul_w16<float, 5>(v[5]);
  v[12] = mul_w16<float, 4>(v[4]);
  v[11] = mul_w16<float, 3>(v[3]);
  v[10] = mul_w16<float, 2>(v[2]);
  v[9] = mul_w16<float, 1>(v[1]);
  v[8] = v[0];
  dif_blocks<float, 16, 4, 0>(v);
  dif_blocks<float, 16, 2, 0>(v);
  dif_blocks<float, 16, 1, 0>(v);
}

// 16-point DIT of which only outputs 0..7 are kept (the rows the embedding keeps): the last
// radix-2 stage computes the sums only.
__device__ __forceinline__ void dit16_lower_half(float2* v) {
  dit_blocks<float, 16, 1, 0>(v);
  dit_blocks<float, 16, 2, 0>(v);
  dit_blocks<float, 16, 4, 0>(v);
  v[0] = cadd<float>(v[0], v[8]);
  v[1] = cadd<float>(v[1], mul_w16<float, 15>(v[9]));
  v[2] = cadd<float>(v[2], mul_w16<float, 14>(v[10]));
  v[3] = cadd<float>(v[3], mul_w16<float, 13>(v[11]));
  v[4] = cadd<float>(v[4], mul_w16<float, 12>(v[12]));
  v[5] = cadd<float>(v[5], mul_w16<float, 11>(v[13]));
  v[6] = cadd<float>(v[6], mul_w16<float, 10>(v[14]));
  v[7] = cadd<float>(v[7], mul_w16<float, 9>(v[15]));
}

// The 15 step twiddles of column c of a radix-16 step on sub-blocks of 2^LOGS points.
template <int LOGS>
__device__ __forceinline__ void load_tw(const float2* __restrict__ tws, int c, float2* w) {
  const float2* t = tws + steptw_off(LOGS) + c;
#pragma unroll
  for (int j = 1; j < 16; ++j) w[j] = __ldg(t + j * (1 << (LOGS - 4)));
}
__device__ __forceinline__ void apply_tw(float2* v, const float2* w) {
#pragma unroll
  for (int j = 1; j < 16; ++j) v[j] = cmul<float>(v[j], w[j]);
}
__device__ __forceinline__ void apply_twc(float2* v, const float2* w) {
#pragma unroll
  for (int j = 1; j < 16; ++j) v[j] = cmulc<float>(v[j], w[j]);
}

template <int R> __device__ __forceinline__ int brev_small(int s) {
  return (int)(__brev((unsigned)s) >> (32 - (R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1)));
}

// Lower-member spectra of one frequency pair and the 2x2 block product on registers (the same
// arithmetic as mac_pair in tpc_kernels.cuh).
__device__ __forceinline__ void mac_reg(float sa, float sd, float2 sb, float2 sc, float2& zl,
                                        float2& zu) {
  const float2 Zp = zl, Zq = zu;
  const float2 S = cadd<float>(Zp, Zq), D = csub<float>(Zp, Zq);
  const float vr = S.x, vi = D.y;
  const float wr = S.y, wi = -D.x;
  const float y1r = fmaf(sa, vr, fmaf(sb.x, wr, -sb.y * wi));
  const float y1i = fmaf(sa, vi, fmaf(sb.x, wi, sb.y * wr));
  const float y2r = fmaf(sd, wr, fmaf(sc.x, vr, -sc.y * vi));
  const float y2i = fmaf(sd, wi, fmaf(sc.x, vi, sc.y * vr));
  zl = make_float2(y1r - y2i, y1i + y2r);
  zu = make_float2(y1r + y2i, y2r - y1i);
}

// ------------------------------------------------------------------------------------------
// Forward strided pass: columns c0 .. c0 + 3 (c0 = 4 blockIdx.x) of the R1 x L view of the
// packed operand z = pad(v) + i pad(w_bar); R1-point DIF of each column, twiddle
// W_m^{c bitrev_R1(t)}, result to z. The prologue forms the operand while it is loaded.
// ------------------------------------------------------------------------------------------
template <int LR1, int PRO>
__global__ void __launch_bounds__(NT_STRIDED, TPC_F32_STRIDED_MINB) k32_fwd(LevelArgs<float> a) {
  pdl_wait();
  constexpr int R1 = 1 << LR1;
  constexpr int RS = R1 >> 8;                   // radix of the last step (4 or 8)
  constexpr int LRS = LR1 - 8;
  constexpr int ST1 = R1 / 16;                  // stride of the first step
  constexpr int TASKS = CT * R1 / 16;           // tasks of the radix-16 steps per tile
  static_assert(TASKS % NT_STRIDED == 0, "tile / threads");
  static_assert(tile_size(R1) == 4 * R1 + 2 * (R1 / RS), "tile size");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  float2* wc = s + tile_size(R1);               // W_{L RS}^{(c0 + cc) k}, [cc][k]
  __shared__ float red[NT_STRIDED / 32];
  const int tid = threadIdx.x;
  const int L = 1 << a.logL;
  const int c0 = blockIdx.x * CT;
  const int N = a.N;
  if (tid < CT * RS) {
    const int cc = tid / RS, k = tid % RS;
    wc[tid] = w_f32((c0 + cc) * k, a.logL + LRS);
  }
  float dot = 0.0f;
  // step 1: radix 16 on stride R1 / 16, inputs rows c1 + (R1/16) j, j < 8 (rows >= R1/2 are
  // the zero padding)
#pragma unroll 1
  for (int q = tid; q < TASKS; q += NT_STRIDED) {
    const int cc = q & (CT - 1), c1 = q >> LOG_CT;
    float2 v[16];
    // all eight operand rows' loads issued before any is formed (measured 5 % faster than
    // four at a time at m = 2^23, no spills)
    constexpr int FR = 8;
#pragma unroll
    for (int h = 0; h < 8; h += FR) {
      Raw<float> rv[FR], rw[FR];
      float qv[FR], zv[FR];
#pragma unroll
      for (int j = 0; j < FR; ++j) {
        const int P = c0 + cc + (c1 + ST1 * (h + j)) * L;
        rv[j] = Raw<float>{0, 0, 0};
        rw[j] = Raw<float>{0, 0, 0};
        qv[j] = 0.0f;
        zv[j] = 0.0f;
        if (P < N) {
          rv[j] = operand_load<float>(a, P, PRO);
          rw[j] = operand_load<float>(a, N + 1 + P, PRO);
          if (P < a.nq) {
            qv[j] = __ldg(a.q + P);
            zv[j] = __ldg(a.zeta + P);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < FR; ++j) {
        const int P = c0 + cc + (c1 + ST1 * (h + j)) * L;
        float xv = 0.0f, xw = 0.0f;
        if (P < N) {
          xv = operand_finish<float>(a, P, rv[j], a.pA, PRO);
          xw = operand_finish<float>(a, N + 1 + P, rw[j], a.pD, PRO);
          dot = fmaf(qv[j], xv, fmaf(zv[j], xw, dot));
        }
        v[h + j] = make_float2(xv, xw);
      }
    }
    float2 w[16];
    load_tw<LR1>(a.tws, c1, w);
    dif16_zero_upper(v);
    apply_tw(v, w);
#pragma unroll
    for (int j = 0; j < 16; ++j) s[tidx<LRS>(c1 + ST1 * j, cc)] = v[j];
  }
  __syncthreads();
  // step 2: radix 16 on sub-blocks of 16 RS rows, stride RS
#pragma unroll 1
  for (int q = tid; q < TASKS; q += NT_STRIDED) {
    const int c2 = q & (RS - 1);
    const int cc = (q >> LRS) & (CT - 1);
    const int sb = q >> (LRS + LOG_CT);
    float2 v[16], w[16];
    const int r0 = sb * 16 * RS + c2;
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = s[tidx<LRS>(r0 + RS * j, cc)];
    load_tw<LRS + 4>(a.tws, c2, w);
    dif<16>(v);
    apply_tw(v, w);
#pragma unroll
    for (int j = 0; j < 16; ++j) s[tidx<LRS>(r0 + RS * j, cc)] = v[j];
  }
  __syncthreads();
  // step 3: radix RS on groups of RS consecutive rows, all four columns per thread; inter-pass
  // twiddle W_m^{c bitrev_R1(t)} = W_m^{c bitrev_8(g)} W_{L RS}^{c bitrev_RS(s)} (t = RS g + s);
  // whole rows (four columns, 32 bytes) to z
  {
    const int g = tid;  // 256 groups
    float2 v[CT][RS];
    {
      const float4* src = reinterpret_cast<const float4*>(s + tidx<LRS>(RS * g, 0));
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const float4 t0 = src[2 * k], t1 = src[2 * k + 1];
        v[0][k] = make_float2(t0.x, t0.y);
        v[1][k] = make_float2(t0.z, t0.w);
        v[2][k] = make_float2(t1.x, t1.y);
        v[3][k] = make_float2(t1.z, t1.w);
      }
    }
    const int bg = (int)(__brev((unsigned)g) >> 24);
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
      dif<RS>(v[cc]);
      const float2 base = w_f32((c0 + cc) * bg, a.logm);
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const float2 tw = (k == 0) ? base : cmul<float>(base, wc[cc * RS + brev_small<RS>(k)]);
        v[cc][k] = cmul<float>(v[cc][k], tw);
      }
    }
#pragma unroll
    for (int k = 0; k < RS; ++k) st_row(a.z + c0 + (RS * g + k) * L, v[0][k], v[1][k], v[2][k], v[3][k]);
  }
  const float tot = block_sum<float>(dot, red);
  if (tid == 0) {
    a.partials[blockIdx.x] = tot;
    if (blockIdx.x == 0 && PRO != PRO_NONE) (void)operand<float>(a, N, a.pO, PRO);  // w_o
  }
}

// ------------------------------------------------------------------------------------------
// Contiguous blocks: L-point DIF of block b (and of its mirror b2), the spectral product of
// every frequency pair, L-point DIT, in place in z. NT = L / 16 threads.
// ------------------------------------------------------------------------------------------
template <int LL, bool NS>
__global__ void __launch_bounds__(1 << (LL - 4), 1 << (13 - LL)) k32_mid(LevelArgs<float> a) {
  pdl_wait();
  constexpr int L = 1 << LL;
  constexpr int NT = L / 16;
  constexpr int RS = L >> 8;       // radix of the last step: 4, 8, 16
  constexpr int LRS = LL - 8;
  constexpr int NG = 256;          // groups of the last step per block
  constexpr int GPT = NG / NT;     // groups per thread
  constexpr int PB = pblock(L);    // padded block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x;
  int b, b2;
  {
    const int cta = blockIdx.x;
    if (cta < 2) {
      b = b2 = cta;
    } else {
      const int j = cta - 1;
      const int gq = 31 - __clz(j);
      b = j + (1 << gq);
      b2 = 3 * (2 << gq) - 1 - b;
    }
  }
  const bool pair = b != b2;
  const int nseq = pair ? 2 : 1;
  // step A: radix 16 on the whole block, stride NT: column c = tid
  {
    float2 w[16];
    load_tw<LL>(a.tws, tid, w);
#pragma unroll 1
    for (int sq = 0; sq < nseq; ++sq) {
      const float2* src = a.z + (size_t)(sq ? b2 : b) * L + tid;
      float2 v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = src[j * NT];
      dif<16>(v);
      apply_tw(v, w);
      float2* d = s + sq * PB;
#pragma unroll
      for (int j = 0; j < 16; ++j) d[pidx(tid + j * NT)] = v[j];
    }
  }
  __syncthreads();
  // step B: radix 16 on sub-blocks of 16 RS points, stride RS
  {
    const int c2 = tid & (RS - 1), sb = tid >> LRS;
    const int r0 = sb * 16 * RS + c2;
    float2 w[16];
    load_tw<LRS + 4>(a.tws, c2, w);
#pragma unroll 1
    for (int sq = 0; sq < nseq; ++sq) {
      float2* d = s + sq * PB;
      float2 v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = d[pidx(r0 + RS * j)];
      dif<16>(v);
      apply_tw(v, w);
#pragma unroll
      for (int j = 0; j < 16; ++j) d[pidx(r0 + RS * j)] = v[j];
    }
  }
  __syncthreads();
  if (pair) {
    // step C (radix RS, group G of b and group NG-1-G of b2), the spectral product of the pairs
    // (b, G, k) / (b2, NG-1-G, RS-1-k) with the spectra of the lower member (in b), and the
    // first inverse step, all in registers
#pragma unroll 1
    for (int gq = 0; gq < GPT; ++gq) {
      const int G = tid + NT * gq;
      const int G2 = NG - 1 - G;
      float2 u[RS], x[RS];
      {
        const float4* s1 = reinterpret_cast<const float4*>(s + pidx(G * RS));
        const float4* s2 = reinterpret_cast<const float4*>(s + PB + pidx(G2 * RS));
#pragma unroll
        for (int k = 0; k < RS / 2; ++k) {
          const float4 t1 = s1[k], t2 = s2[k];
          u[2 * k] = make_float2(t1.x, t1.y);
          u[2 * k + 1] = make_float2(t1.z, t1.w);
          x[2 * k] = make_float2(t2.x, t2.y);
          x[2 * k + 1] = make_float2(t2.z, t2.w);
        }
      }
      dif<RS>(u);
      dif<RS>(x);
      const int P0 = b * L + G * RS;
#pragma unroll
      for (int k0 = 0; k0 < RS; k0 += 4) {
        const float4 sa4 = __ldg(reinterpret_cast<const float4*>(a.sA + P0 + k0));
        const float4 sd4 = __ldg(reinterpret_cast<const float4*>(a.sD + P0 + k0));
        const float4 sb01 = __ldg(reinterpret_cast<const float4*>(a.sB + P0 + k0));
        const float4 sb23 = __ldg(reinterpret_cast<const float4*>(a.sB + P0 + k0 + 2));
        float sa[4] = {sa4.x, sa4.y, sa4.z, sa4.w};
        float sd[4] = {sd4.x, sd4.y, sd4.z, sd4.w};
        float2 sbv[4] = {make_float2(sb01.x, sb01.y), make_float2(sb01.z, sb01.w),
                         make_float2(sb23.x, sb23.y), make_float2(sb23.z, sb23.w)};
        float2 scv[4];
        if constexpr (NS) {
          const float4 sc01 = __ldg(reinterpret_cast<const float4*>(a.sC + P0 + k0));
          const float4 sc23 = __ldg(reinterpret_cast<const float4*>(a.sC + P0 + k0 + 2));
          scv[0] = make_float2(sc01.x, sc01.y);
          scv[1] = make_float2(sc01.z, sc01.w);
          scv[2] = make_float2(sc23.x, sc23.y);
          scv[3] = make_float2(sc23.z, sc23.w);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) scv[i] = make_float2(sbv[i].x, -sbv[i].y);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          mac_reg(sa[i], sd[i], sbv[i], scv[i], u[k0 + i], x[RS - 1 - k0 - i]);
      }
      dit<RS>(u);
      dit<RS>(x);
      {
        float4* s1 = reinterpret_cast<float4*>(s + pidx(G * RS));
        float4* s2 = reinterpret_cast<float4*>(s + PB + pidx(G2 * RS));
#pragma unroll
        for (int k = 0; k < RS / 2; ++k) {
          s1[k] = make_float4(u[2 * k].x, u[2 * k].y, u[2 * k + 1].x, u[2 * k + 1].y);
          s2[k] = make_float4(x[2 * k].x, x[2 * k].y, x[2 * k + 1].x, x[2 * k + 1].y);
        }
      }
    }
  } else {
    // self-paired blocks 0 and 1 (two CTAs of the grid): step C through shared memory, the
    // spectral product as in the general kernel, the first inverse step
#pragma unroll 1
    for (int gq = 0; gq < GPT; ++gq) {
      float4* sp = reinterpret_cast<float4*>(s + pidx((tid + NT * gq) * RS));
      float2 u[RS];
#pragma unroll
      for (int k = 0; k < RS / 2; ++k) {
        const float4 t1 = sp[k];
        u[2 * k] = make_float2(t1.x, t1.y);
        u[2 * k + 1] = make_float2(t1.z, t1.w);
      }
      dif<RS>(u);
#pragma unroll
      for (int k = 0; k < RS / 2; ++k)
        sp[k] = make_float4(u[2 * k].x, u[2 * k].y, u[2 * k + 1].x, u[2 * k + 1].y);
    }
    __syncthreads();
    const int ntask = (b == 1) ? (L >> 1) : (L >> 1) + 1;
    for (int i = tid; i < ntask; i += NT) {
      int lo, hi;
      if (b == 1) {
        lo = i;
        hi = L - 1 - i;
      } else {
        block0_pair(i, lo, hi);
      }
      const Spec<float> sp = spec_load<float, NS>(a, b * L + lo);
      mac_pair<float>(sp, s + pidx(lo), s + pidx(hi));
    }
    __syncthreads();
#pragma unroll 1
    for (int gq = 0; gq < GPT; ++gq) {
      float4* sp = reinterpret_cast<float4*>(s + pidx((tid + NT * gq) * RS));
      float2 u[RS];
#pragma unroll
      for (int k = 0; k < RS / 2; ++k) {
        const float4 t1 = sp[k];
        u[2 * k] = make_float2(t1.x, t1.y);
        u[2 * k + 1] = make_float2(t1.z, t1.w);
      }
      dit<RS>(u);
#pragma unroll
      for (int k = 0; k < RS / 2; ++k)
        sp[k] = make_float4(u[2 * k].x, u[2 * k].y, u[2 * k + 1].x, u[2 * k + 1].y);
    }
  }
  __syncthreads();
  // inverse step B
  {
    const int c2 = tid & (RS - 1), sb = tid >> LRS;
    const int r0 = sb * 16 * RS + c2;
    float2 w[16];
    load_tw<LRS + 4>(a.tws, c2, w);
#pragma unroll 1
    for (int sq = 0; sq < nseq; ++sq) {
      float2* d = s + sq * PB;
      float2 v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = d[pidx(r0 + RS * j)];
      apply_twc(v, w);
      dit<16>(v);
#pragma unroll
      for (int j = 0; j < 16; ++j) d[pidx(r0 + RS * j)] = v[j];
    }
  }
  __syncthreads();
  // inverse step A, results to z
  {
    float2 w[16];
    load_tw<LL>(a.tws, tid, w);
#pragma unroll 1
    for (int sq = 0; sq < nseq; ++sq) {
      const float2* d = s + sq * PB;
      float2 v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = d[pidx(tid + j * NT)];
      apply_twc(v, w);
      dit<16>(v);
      float2* dst = a.z + (size_t)(sq ? b2 : b) * L + tid;
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[j * NT] = v[j];
    }
  }
}

// ------------------------------------------------------------------------------------------
// Inverse strided pass: twiddle conj W_m^{c bitrev_R1(t)}, R1-point DIT of each of the four
// columns, epilogue on the rows t < R1/2 (the first N outputs of each half).
// ------------------------------------------------------------------------------------------
template <int LR1, int EPI>
__global__ void __launch_bounds__(NT_STRIDED, TPC_F32_STRIDED_MINB) k32_inv(LevelArgs<float> a) {
  pdl_wait();
  constexpr int R1 = 1 << LR1;
  constexpr int RS = R1 >> 8;
  constexpr int LRS = LR1 - 8;
  constexpr int ST1 = R1 / 16;
  constexpr int TASKS = CT * R1 / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  float2* wc = s + tile_size(R1);
  const int tid = threadIdx.x;
  const int L = 1 << a.logL;
  const int c0 = blockIdx.x * CT;
  const int N = a.N;
  if (tid < CT * RS) {
    const int cc = tid / RS, k = tid % RS;
    wc[tid] = w_f32((c0 + cc) * k, a.logL + LRS);
  }
  // whole rows of the four columns from z, conj twiddle, first DIT step (radix RS)
  {
    const int g = tid;
    float2 v[CT][RS];
#pragma unroll
    for (int k = 0; k < RS; ++k)
      ld_row(a.z + c0 + (RS * g + k) * L, v[0][k], v[1][k], v[2][k], v[3][k]);
    __syncthreads();  // the W_{L RS} table
    const int bg = (int)(__brev((unsigned)g) >> 24);
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
      const float2 base = w_f32((c0 + cc) * bg, a.logm);
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const float2 tw = (k == 0) ? base : cmul<float>(base, wc[cc * RS + brev_small<RS>(k)]);
        v[cc][k] = cmulc<float>(v[cc][k], tw);
      }
      dit<RS>(v[cc]);
    }
    float4* dst = reinterpret_cast<float4*>(s + tidx<LRS>(RS * g, 0));
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      dst[2 * k] = make_float4(v[0][k].x, v[0][k].y, v[1][k].x, v[1][k].y);
      dst[2 * k + 1] = make_float4(v[2][k].x, v[2][k].y, v[3][k].x, v[3][k].y);
    }
  }
  __syncthreads();
  // DIT radix 16 on sub-blocks of 16 RS rows, stride RS
#pragma unroll 1
  for (int q = tid; q < TASKS; q += NT_STRIDED) {
    const int c2 = q & (RS - 1);
    const int cc = (q >> LRS) & (CT - 1);
    const int sb = q >> (LRS + LOG_CT);
    float2 v[16], w[16];
    const int r0 = sb * 16 * RS + c2;
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = s[tidx<LRS>(r0 + RS * j, cc)];
    load_tw<LRS + 4>(a.tws, c2, w);
    apply_twc(v, w);
    dit<16>(v);
#pragma unroll
    for (int j = 0; j < 16; ++j) s[tidx<LRS>(r0 + RS * j, cc)] = v[j];
  }
  __syncthreads();
  // last DIT step (radix 16, stride R1/16), rows c1 + (R1/16) j for j < 8, and the epilogue
  const float w_o = a.x[N];
#pragma unroll 1
  for (int q = tid; q < TASKS; q += NT_STRIDED) {
    const int cc = q & (CT - 1), c1 = q >> LOG_CT;
    float2 v[16];
    {
      float2 w[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = s[tidx<LRS>(c1 + ST1 * j, cc)];
      load_tw<LR1>(a.tws, c1, w);
      apply_twc(v, w);
    }
    dit16_lower_half(v);
    // the epilogue (no band on these levels), all eight rows' loads first (measured faster than
    // four at a time): Cross column p, xi below its support, right-hand side f (residual,
    // Jacobi), current iterate x (Jacobi)
    constexpr int ER = 8;
#pragma unroll
    for (int h = 0; h < 8; h += ER) {
      float pv[ER], xiv[ER], fv[ER], fw[ER], xv[ER], xw[ER];
#pragma unroll
      for (int j = 0; j < ER; ++j) {
        const int P = c0 + cc + (c1 + ST1 * (h + j)) * L;
        pv[j] = xiv[j] = fv[j] = fw[j] = xv[j] = xw[j] = 0.0f;
        if (P < N) {
          if (P < a.np) {
            pv[j] = __ldg(a.p + P);
            xiv[j] = __ldg(a.xi + P);
          }
          if (EPI != EPI_APPLY) {
            fv[j] = __ldg(a.f + P);
            fw[j] = __ldg(a.f + N + 1 + P);
          }
          if (EPI == EPI_JACOBI) {
            xv[j] = a.x[P];
            xw[j] = a.x[N + 1 + P];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < ER; ++j) {
        const int P = c0 + cc + (c1 + ST1 * (h + j)) * L;
        if (P < N) {
          const float yv = fmaf(pv[j], w_o, v[h + j].x);
          const float yw = fmaf(xiv[j], w_o, v[h + j].y);
          if (EPI == EPI_APPLY) {
            a.y[P] = yv;
            a.y[N + 1 + P] = yw;
          } else if (EPI == EPI_RESID) {
            a.y[P] = fv[j] - yv;
            a.y[N + 1 + P] = fw[j] - yw;
          } else {
            a.y[P] = fmaf(a.wA, fv[j] - yv, xv[j]);
            a.y[N + 1 + P] = fmaf(a.wD, fw[j] - yw, xw[j]);
          }
        }
      }
    }
  }
  if (blockIdx.x == 0 && tid < 32) {
    float acc = 0;
    for (int i = tid; i < a.nparts; i += 32) acc += a.partials[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (tid == 0) epi_middle<float>(a, acc, w_o, EPI);
  }
}

// Dynamic shared memory of the kernels.
inline size_t strided_smem(int logR1) {
  const int R1 = 1 << logR1;
  return sizeof(float2) * (size_t)(tile_size(R1) + CT * (R1 >> 8));
}
inline size_t mid_smem(int logL) { return sizeof(float2) * (size_t)(2 * pblock(1 << logL)); }

// Levels the register-resident kernels take: m = 2^20 .. 2^23 (R1 = 2^10, 2^11; L = 2^10 .. 2^12)
// without the banded part of the weakly singular model.
inline bool eligible(int logm, int logR1, int logL, bool band) {
  return !band && logm >= 20 && logm <= 23 && (logR1 == 10 || logR1 == 11) && logL >= 10 &&
         logL <= 12;
}

template <int LR1>
inline void launch_fwd_lr(const LevelArgs<float>& a, int blocks, cudaStream_t st) {
  const size_t sm = strided_smem(LR1);
  switch (a.pro) {
    case PRO_SMOOTH: launch_k(k32_fwd<LR1, PRO_SMOOTH>, blocks, NT_STRIDED, sm, st, a); break;
    case PRO_RESTRICT: launch_k(k32_fwd<LR1, PRO_RESTRICT>, blocks, NT_STRIDED, sm, st, a); break;
    case PRO_PROLONG: launch_k(k32_fwd<LR1, PRO_PROLONG>, blocks, NT_STRIDED, sm, st, a); break;
    default: launch_k(k32_fwd<LR1, PRO_NONE>, blocks, NT_STRIDED, sm, st, a); break;
  }
}
template <int LR1>
inline void launch_inv_lr(const LevelArgs<float>& a, int blocks, cudaStream_t st) {
  const size_t sm = strided_smem(LR1);
  switch (a.epi) {
    case EPI_RESID: launch_k(k32_inv<LR1, EPI_RESID>, blocks, NT_STRIDED, sm, st, a); break;
    case EPI_JACOBI: launch_k(k32_inv<LR1, EPI_JACOBI>, blocks, NT_STRIDED, sm, st, a); break;
    default: launch_k(k32_inv<LR1, EPI_APPLY>, blocks, NT_STRIDED, sm, st, a); break;
  }
}
inline void launch_fwd(const LevelArgs<float>& a, int blocks, cudaStream_t st) {
  if (a.logR1 == 11) launch_fwd_lr<11>(a, blocks, st);
  else launch_fwd_lr<10>(a, blocks, st);
}
inline void launch_inv(const LevelArgs<float>& a, int blocks, cudaStream_t st) {
  if (a.logR1 == 11) launch_inv_lr<11>(a, blocks, st);
  else launch_inv_lr<10>(a, blocks, st);
}
template <bool NS>
inline void launch_mid(const LevelArgs<float>& a, int blocks, cudaStream_t st) {
  const size_t sm = mid_smem(a.logL);
  if (a.logL == 12) launch_k(k32_mid<12, NS>, blocks, 256, sm, st, a);
  else if (a.logL == 11) launch_k(k32_mid<11, NS>, blocks, 128, sm, st, a);
  else launch_k(k32_mid<10, NS>, blocks, 64, sm, st, a);
}

template <int LR1>
inline cudaError_t strided_attrs_lr() {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int sm = (int)strided_smem(LR1);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k32_fwd<LR1, PRO_NONE>, A, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k32_fwd<LR1, PRO_SMOOTH>, A, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k32_fwd<LR1, PRO_RESTRICT>, A, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k32_fwd<LR1, PRO_PROLONG>, A, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k32_inv<LR1, EPI_APPLY>, A, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k32_inv<LR1, EPI_RESID>, A, sm)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k32_inv<LR1, EPI_JACOBI>, A, sm);
}
template <bool NS>
inline cudaError_t mid_attrs() {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k32_mid<12, NS>, A, (int)mid_smem(12))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k32_mid<11, NS>, A, (int)mid_smem(11))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k32_mid<10, NS>, A, (int)mid_smem(10));
}
inline cudaError_t set_attrs() {
  cudaError_t e;
  if ((e = strided_attrs_lr<10>()) != cudaSuccess) return e;
  if ((e = strided_attrs_lr<11>()) != cudaSuccess) return e;
  if ((e = mid_attrs<false>()) != cudaSuccess) return e;
  return mid_attrs<true>();
}

}  // namespace f32p
}  // namespace tpc
