// Stage-batched solves of many independent 1-D instances (the batched configuration).
//
// Instances whose level structure is identical (same finest level K, coarsest level, system,
// inner-cycle count; mixed precision with V(1,1) cycles, the single-block V-cycle bottom and the
// prefix-sum residual) form a group. For a group, every stage of an outer iteration -- each
// product of the V-cycle (Algorithm 2), the single-block bottom, the element-wise steps of the
// FP64 refinement, the prefix-sum residual and the norm -- is ONE launch over all instances of
// the group: a grid dimension runs over the instances, each block reading its instance's
// arguments from a device array. A three-pass product (forward strided pass, contiguous blocks,
// inverse strided pass) is either one persistent cooperative launch whose blocks take the tiles
// of all instances pass by pass, separated by grid-wide barriers on a device counter -- a
// barrier's wait gives up after a bounded number of polls, raises an error flag the host reads,
// and the kernel returns (no hang) -- or three launches, one per pass, over the tiles of all
// instances (the default: measured faster on every level of these kernels). Every instance runs exactly the kernels' bodies, arguments and tile
// decomposition of its lone solve, so its iterates are bitwise those of tpc_solve; instances
// that have converged, or that take fewer inner cycles in an iteration, are masked per stage.
// One iteration of a group is captured once per inner-cycle count as a CUDA graph.
//
// This file is included by tpc_api.cu (it uses the handles' hierarchies).
#pragma once

namespace tpc {
namespace batch {

// Wait limit of a barrier: polls of the counter, each followed by a 256 ns sleep (about a second).
constexpr unsigned MAX_POLLS = 1u << 22;

// Grid-wide barrier of a cooperative launch (all blocks resident): each block adds one arrival
// to *count and waits until `target` arrivals are counted. The wait gives up after max_polls
// polls (or as soon as another block has given up) and sets *err = 1; returns false then.
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned target, int* err,
                                          unsigned max_polls) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    int good = 1;
    unsigned polls = 0;
    while (*reinterpret_cast<volatile unsigned*>(count) < target) {
      if (*reinterpret_cast<volatile int*>(err) != 0) {
        good = 0;
        break;
      }
      if (++polls > max_polls) {
        atomicExch(err, 1);
        good = 0;
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// The contiguous-block body of the persistent kernel: the general instance, which the lone
// launch (launch_mid_pair) also runs for log2 L <= 9; levels with larger L (compile-time
// instances) take the three-launch form (use_coop).
template <typename T, bool NS>
__device__ __forceinline__ void mid_pair_dispatch(const LevelArgs<T>& a, int blk) {
  mid_body<T, MID_PAIR, NS>(a, blk);
}

// One three-pass product of every live instance: work item w = instance * blocks + tile.
template <typename T, bool NS, int PRO, int EPI>
__global__ void __launch_bounds__(fft_threads<T>(), 2)
    k_batch_product(const LevelArgs<T>* __restrict__ args, const int* __restrict__ live, int ninst,
                    int fwd_blocks, int mid_blocks, unsigned* sync, int* err, unsigned max_polls) {
  __shared__ __align__(16) LevelArgs<T> la;
  for (int w = blockIdx.x; w < ninst * fwd_blocks; w += gridDim.x) {
    const int inst = w / fwd_blocks;
    if (!live[inst]) continue;
    copy_args<T>(&la, &args[inst]);
    fwd_strided_body<T, IN_PACK, PRO>(la, w - inst * fwd_blocks);
    __syncthreads();
  }
  if (!grid_sync(sync, gridDim.x, err, max_polls)) return;
  for (int w = blockIdx.x; w < ninst * mid_blocks; w += gridDim.x) {
    const int inst = w / mid_blocks;
    if (!live[inst]) continue;
    copy_args<T>(&la, &args[inst]);
    mid_pair_dispatch<T, NS>(la, w - inst * mid_blocks);
    __syncthreads();
  }
  if (!grid_sync(sync, 2 * gridDim.x, err, max_polls)) return;
  for (int w = blockIdx.x; w < ninst * fwd_blocks; w += gridDim.x) {
    const int inst = w / fwd_blocks;
    if (!live[inst]) continue;
    copy_args<T>(&la, &args[inst]);
    inv_strided_body<T, EPI>(la, w - inst * fwd_blocks);
    __syncthreads();
  }
}

// The same product as three launches over all live instances, grid (tiles, instances): the
// lone kernels' bodies and resident-block counts, no grid barrier (the launch boundaries order
// the passes).
template <typename T, int PRO, int MINB>
__global__ void __launch_bounds__(fft_threads<T>(), MINB)
    k_batch_fwd(const LevelArgs<T>* __restrict__ args, const int* __restrict__ live) {
  __shared__ __align__(16) LevelArgs<T> la;
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  copy_args<T>(&la, &args[inst]);
  fwd_strided_body<T, IN_PACK, PRO>(la, (int)blockIdx.x);
}
// LOGL_CT as launch_mid_pair picks it (the FP32 instances with log2 L = 10..12, else 0).
template <typename T, bool NS, int LOGL_CT>
__global__ void __launch_bounds__(fft_threads<T>(), mid_min_blocks<T>())
    k_batch_mid(const LevelArgs<T>* __restrict__ args, const int* __restrict__ live) {
  __shared__ __align__(16) LevelArgs<T> la;
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  copy_args<T>(&la, &args[inst]);
  mid_body<T, MID_PAIR, NS, LOGL_CT>(la, (int)blockIdx.x);
}
template <typename T, int EPI, int MINB>
__global__ void __launch_bounds__(fft_threads<T>(), MINB)
    k_batch_inv(const LevelArgs<T>* __restrict__ args, const int* __restrict__ live) {
  __shared__ __align__(16) LevelArgs<T> la;
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  copy_args<T>(&la, &args[inst]);
  inv_strided_body<T, EPI>(la, (int)blockIdx.x);
}

// Single-block products (levels with m <= 4096), one block per instance.
template <typename T, bool NS>
__global__ void __launch_bounds__(fft_threads<T>(), 1)
    k_batch_whole(const LevelArgs<T>* __restrict__ args, const int* __restrict__ live) {
  __shared__ __align__(16) LevelArgs<T> la;
  const int inst = blockIdx.x;
  if (!live[inst]) return;
  copy_args<T>(&la, &args[inst]);
  mid_body<T, MID_WHOLE, NS>(la, 0);
}

// The single-block V-cycle bottom of every live instance, one block each.
template <typename T, bool NS>
__global__ void __launch_bounds__(fft_threads<T>(), 1)
    k_batch_bottom(const BottomPlan<T>* const* __restrict__ plans, const int* __restrict__ live) {
  const int inst = blockIdx.x;
  if (!live[inst]) return;
  vcycle_bottom_body<T, NS>(plans[inst]);
}

// Buffers of one instance's outer iteration (mixed precision).
struct IterPtrs {
  const double* r0;   // FP64 residual
  double* u;          // iterate
  double* sumsq;      // ||r||^2 (device scalar of the handle)
  float* f32;         // scaled residual (right-hand side of the first FP32 cycle)
  float* acc32;       // accumulated FP32 correction
  const float* ec;    // result of the FP32 V-cycle (the top level's buffer it returns)
};

// The element-wise kernels of the iteration, grid (blocks, instances), same arithmetic as
// k_to_f32_scaled, k_copy, k_axpy and k_axpy_f32_scaled.
__global__ void k_batch_to_f32(const IterPtrs* __restrict__ p, const int* __restrict__ live,
                               long long n) {
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  const IterPtrs q = p[inst];
  const double ss = q.sumsq[0];
  const double s = (ss > 0.0) ? sqrt((double)n / ss) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    q.f32[i] = (float)(q.r0[i] * s);
}
__global__ void k_batch_copy(const IterPtrs* __restrict__ p, const int* __restrict__ live,
                             long long n) {
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  const IterPtrs q = p[inst];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    q.acc32[i] = q.ec[i];
}
__global__ void k_batch_axpy(const IterPtrs* __restrict__ p, const int* __restrict__ live,
                             long long n) {
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  const IterPtrs q = p[inst];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    q.acc32[i] += q.ec[i];
}
__global__ void k_batch_axpy_scaled(const IterPtrs* __restrict__ p, const int* __restrict__ live,
                                    long long n) {
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  const IterPtrs q = p[inst];
  const double inv = sqrt(q.sumsq[0] / (double)n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    q.u[i] = fma((double)q.acc32[i], inv, q.u[i]);
}

// The prefix-sum residual of every live instance (grids as the lone kernels' times instances).
__global__ void __launch_bounds__(box::NT) k_batch_box_local(const box::BoxArgs* __restrict__ a,
                                                            const int* __restrict__ live) {
  if (!live[blockIdx.y]) return;
  box::box_local_body(a[blockIdx.y], (int)blockIdx.x);
}
__global__ void __launch_bounds__(1024) k_batch_box_offsets(const box::BoxArgs* __restrict__ a,
                                                           const int* __restrict__ live) {
  if (!live[blockIdx.x]) return;
  box::box_offsets_body(a[blockIdx.x]);
}
__global__ void __launch_bounds__(box::NT) k_batch_box_resid(const box::BoxArgs* __restrict__ a,
                                                            const int* __restrict__ live) {
  if (!live[blockIdx.z]) return;
  box::box_resid_body(a[blockIdx.z], (int)blockIdx.x, (int)gridDim.x, (int)blockIdx.y);
}

// ||r||^2 of every live instance: the partial sums of k_sumsq_partial (same grid of
// NORM_BLOCKS blocks per instance, same order), then the final sum into the handle's scalar and
// into out[inst] for the host.
__global__ void __launch_bounds__(NTHREADS) k_batch_sumsq_partial(const IterPtrs* __restrict__ p,
                                                                 const int* __restrict__ live,
                                                                 long long n, double* part) {
  __shared__ double red[NTHREADS / 32];
  const int inst = blockIdx.y;
  if (!live[inst]) return;
  const double* r = p[inst].r0;
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = r[i];
    acc = fma(v, v, acc);
  }
  const double s = block_sum<double>(acc, red);
  if (threadIdx.x == 0) part[(size_t)inst * gridDim.x + blockIdx.x] = s;
}
__global__ void k_batch_sumsq_final(const IterPtrs* __restrict__ p, const int* __restrict__ live,
                                    const double* part, int np, double* out) {
  const int inst = blockIdx.x;
  if (!live[inst]) return;
  double acc = 0;
  for (int i = threadIdx.x; i < np; i += 32) acc += part[(size_t)inst * np + i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) {
    p[inst].sumsq[0] = acc;
    out[inst] = acc;
  }
}

// A barrier no block can pass (its target exceeds the grid): the wait must give up and report.
__global__ void k_grid_wait_selftest(unsigned* sync, int* err, unsigned max_polls, int* passed) {
  if (grid_sync(sync, gridDim.x + 1, err, max_polls) && threadIdx.x == 0) atomicAdd(passed, 1);
}

}  // namespace batch
}  // namespace tpc

// ----------------------------------------------------------------------------------------------
// Host side: groups, their stage arguments, one iteration as a graph, the solve loop.
// ----------------------------------------------------------------------------------------------
struct tpc_batch {
  struct Group {
    std::vector<int> idx;          // members (indices into hs)
    int ninst = 0;
    bool ns = false;
    int nl = 0;                    // levels with products above the single-block bottom
    std::vector<const DevLevel<float>*> lev;  // plan of each such level (the first member's)
    size_t bottom_smem = 0;
    long long n = 0;               // finest unknowns
    int box_nblk = 0, box_gx = 0;
    cudaStream_t stream = nullptr;
    LevelArgs<float>* pre = nullptr;     // [nl][ninst], first cycle (right-hand side f_32)
    LevelArgs<float>* post = nullptr;    // [nl][ninst]
    LevelArgs<float>* pre_r = nullptr;   // [ninst], level 0 of later cycles (right-hand side res32)
    LevelArgs<float>* post_r = nullptr;  // [ninst]
    LevelArgs<float>* resid = nullptr;   // [ninst], residual product of later cycles
    BottomPlan<float>** plans = nullptr;
    tpc::batch::IterPtrs* iter = nullptr;
    tpc::box::BoxArgs* boxa = nullptr;
    int* live = nullptr;                 // [33][ninst]: row 0 the active instances, row c >= 1
                                         // those that run inner cycle c + 1
    int* live_host = nullptr;            // pinned copy
    double* part = nullptr;              // [ninst][NORM_BLOCKS]
    double* out = nullptr;               // [ninst] ||r||^2 after the iteration
    double* out_host = nullptr;          // pinned
    unsigned* sync = nullptr;            // barrier counter of the cooperative launches
    int* err = nullptr;                  // set when a barrier's wait gave up
    int* err_host = nullptr;             // pinned
    cudaGraphExec_t exec[33] = {};
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
  };
  std::vector<tpc_handle*> hs;
  std::vector<tpc2d_handle*> hs2;        // 2-D instances, solved beside the groups
  std::vector<Group> groups;
  std::vector<int> solo;                 // instances solved with their own iteration graphs
  int product_mode = TPC_BATCH_AUTO;     // how the three-pass products are launched
  std::vector<void*> dev, pinned;
  std::string err;
};

namespace tpc {
namespace batch {

int bfail(tpc_batch* B, cudaError_t e, const char* what) {
  B->err = std::string(what) + ": " + cudaGetErrorString(e);
  set_host_error(B->err);
  return TPC_ECUDA;
}
#define TPCB_CUDA(B, call)                               \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bfail(B, e_, #call);   \
  } while (0)

template <typename P>
int balloc(tpc_batch* B, P** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(P) + 16);
  if (e != cudaSuccess) return bfail(B, e, "cudaMalloc");
  B->dev.push_back(v);
  *p = reinterpret_cast<P*>(v);
  return TPC_OK;
}
template <typename P>
int bpinned(tpc_batch* B, P** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMallocHost(&v, count * sizeof(P) + 16);
  if (e != cudaSuccess) return bfail(B, e, "cudaMallocHost");
  B->pinned.push_back(v);
  *p = reinterpret_cast<P*>(v);
  return TPC_OK;
}
template <typename P>
int upload_vec(tpc_batch* B, P* dst, const std::vector<P>& src, cudaStream_t s) {
  TPCB_CUDA(B, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(P), cudaMemcpyHostToDevice, s));
  TPCB_CUDA(B, cudaStreamSynchronize(s));
  return TPC_OK;
}

// Whether an instance can run stage-batched (mixed precision, V(1,1), single-block bottom,
// prefix-sum residual, levels of the general FP32 kernels), and its group key.
bool eligible(const tpc_handle* H) {
  if (H->prm.precision != TPC_MIXED || H->prm.outer != TPC_OUTER_VCYCLE || H->prm.m1 != 1 ||
      H->prm.m2 != 1 || !H->box_on)
    return false;
  const Hier<float>& S = H->s;
  if (!S.bottom || S.bottom_li < 1) return false;
  for (int li = 0; li < S.bottom_li; ++li) {
    const DevLevel<float>& L = S.lev[li];
    if (L.f32reg || L.bd || !L.sA) return false;
  }
  return true;
}
std::vector<long long> group_key(const tpc_handle* H) {
  const Hier<float>& S = H->s;
  std::vector<long long> k = {H->K, H->kc, H->prm.variant != TPC_SPD, H->prm.inner_cycles,
                              S.bottom_li, (long long)S.bottom_smem};
  for (int li = 0; li < S.bottom_li; ++li) {
    const DevLevel<float>& L = S.lev[li];
    k.insert(k.end(), {L.logm, L.logR1, L.logL, L.logC, L.fwd_blocks, L.mid_blocks,
                       (long long)L.smem_strided, (long long)L.smem_mid});
  }
  return k;
}

template <bool NS, int PRO, int EPI>
int coop_product(tpc_batch* B, tpc_batch::Group& g, int li, const LevelArgs<float>* args,
                 const int* live) {
  const DevLevel<float>& L = *g.lev[li];
  auto kern = k_batch_product<float, NS, PRO, EPI>;
  const size_t smem = std::max(L.smem_strided, L.smem_mid);
  const int nt = fft_threads<float>();
  TPCB_CUDA(B, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 150 * 1024));
  int per_sm = 0;
  TPCB_CUDA(B, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
  int dev = 0, nsm = 0;
  TPCB_CUDA(B, cudaGetDevice(&dev));
  TPCB_CUDA(B, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) {
    B->err = "batched product does not fit one block per SM";
    return TPC_ENOTSUP;
  }
  const long long work = (long long)g.ninst * std::max(L.fwd_blocks, L.mid_blocks);
  const int grid = (int)std::max<long long>(1, std::min<long long>(work, (long long)per_sm * nsm));
  TPCB_CUDA(B, cudaMemsetAsync(g.sync, 0, sizeof(unsigned), g.stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = g.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TPCB_CUDA(B, cudaLaunchKernelEx(&cfg, kern, args, live, g.ninst, (int)L.fwd_blocks,
                                  (int)L.mid_blocks, g.sync, g.err, MAX_POLLS));
  return TPC_OK;
}

template <int PRO, int EPI, int MB, bool NS>
int three_pass_mb(tpc_batch* B, tpc_batch::Group& g, const DevLevel<float>& L,
                  const LevelArgs<float>* args, const int* live) {
  const int nt = fft_threads<float>();
  // the limit of each kernel is raised once to the largest any level asks (never lowered: a
  // graph captured for another group may launch the same kernel with more)
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int lim = 150 * 1024;
  auto kf = k_batch_fwd<float, PRO, MB>;
  auto km = L.logL == 12 ? k_batch_mid<float, NS, 12>
            : L.logL == 11 ? k_batch_mid<float, NS, 11>
            : L.logL == 10 ? k_batch_mid<float, NS, 10> : k_batch_mid<float, NS, 0>;
  auto ki = k_batch_inv<float, EPI, MB>;
  TPCB_CUDA(B, cudaFuncSetAttribute(kf, A, lim));
  TPCB_CUDA(B, cudaFuncSetAttribute(km, A, lim));
  TPCB_CUDA(B, cudaFuncSetAttribute(ki, A, lim));
  kf<<<dim3(L.fwd_blocks, g.ninst), nt, L.smem_strided, g.stream>>>(args, live);
  km<<<dim3(L.mid_blocks, g.ninst), nt, L.smem_mid, g.stream>>>(args, live);
  ki<<<dim3(L.fwd_blocks, g.ninst), nt, L.smem_strided, g.stream>>>(args, live);
  TPCB_CUDA(B, cudaGetLastError());
  return TPC_OK;
}
// Resident blocks of the strided passes as the lone launch picks them (launch_fwd_strided).
template <int PRO, int EPI, bool NS>
int three_pass(tpc_batch* B, tpc_batch::Group& g, int li, const LevelArgs<float>* args,
               const int* live) {
  const DevLevel<float>& L = *g.lev[li];
  if (L.logm <= LOG_M_HIGH_OCC)
    return three_pass_mb<PRO, EPI, F32_HIGH_OCC_BLOCKS, NS>(B, g, L, args, live);
  return three_pass_mb<PRO, EPI, fft_min_blocks<float>(), NS>(B, g, L, args, live);
}

// Whether level li of the group runs its products as one cooperative launch (else three).
bool use_coop(const tpc_batch* B, const tpc_batch::Group& g, int li) {
  // the persistent kernel holds the general contiguous-block body only (log2 L <= 9)
  if (g.lev[li]->logL > 9) return false;
  if (B->product_mode == TPC_BATCH_COOPERATIVE) return true;
  return false;
}

template <int PRO, int EPI, bool NS>
int product_kind(tpc_batch* B, tpc_batch::Group& g, int li, const LevelArgs<float>* args,
                 const int* live) {
  if (use_coop(B, g, li)) return coop_product<NS, PRO, EPI>(B, g, li, args, live);
  return three_pass<PRO, EPI, NS>(B, g, li, args, live);
}

// One product stage of level li over the group (prologue / epilogue as in the lone V-cycle).
int product(tpc_batch* B, tpc_batch::Group& g, int li, const LevelArgs<float>* args, int pro,
            int epi, const int* live) {
  const DevLevel<float>& L = *g.lev[li];
  if (L.logR1 == 0) {
    if (g.ns) k_batch_whole<float, true><<<g.ninst, fft_threads<float>(), L.smem_mid, g.stream>>>(args, live);
    else k_batch_whole<float, false><<<g.ninst, fft_threads<float>(), L.smem_mid, g.stream>>>(args, live);
    TPCB_CUDA(B, cudaGetLastError());
    return TPC_OK;
  }
  const int kind = pro * 4 + epi;
  if (g.ns) {
    switch (kind) {
      case PRO_SMOOTH * 4 + EPI_RESID: return product_kind<PRO_SMOOTH, EPI_RESID, true>(B, g, li, args, live);
      case PRO_RESTRICT * 4 + EPI_RESID: return product_kind<PRO_RESTRICT, EPI_RESID, true>(B, g, li, args, live);
      case PRO_PROLONG * 4 + EPI_JACOBI: return product_kind<PRO_PROLONG, EPI_JACOBI, true>(B, g, li, args, live);
      default: return product_kind<PRO_NONE, EPI_RESID, true>(B, g, li, args, live);
    }
  }
  switch (kind) {
    case PRO_SMOOTH * 4 + EPI_RESID: return product_kind<PRO_SMOOTH, EPI_RESID, false>(B, g, li, args, live);
    case PRO_RESTRICT * 4 + EPI_RESID: return product_kind<PRO_RESTRICT, EPI_RESID, false>(B, g, li, args, live);
    case PRO_PROLONG * 4 + EPI_JACOBI: return product_kind<PRO_PROLONG, EPI_JACOBI, false>(B, g, li, args, live);
    default: return product_kind<PRO_NONE, EPI_RESID, false>(B, g, li, args, live);
  }
}

// The FP32 V-cycle of the group from the top (first: right-hand side f_32, else res32).
int vcycle(tpc_batch* B, tpc_batch::Group& g, bool first, const int* live) {
  for (int li = 0; li < g.nl; ++li) {
    const LevelArgs<float>* a = (li == 0 && !first) ? g.pre_r : g.pre + (size_t)li * g.ninst;
    TPC_TRY(product(B, g, li, a, li == 0 ? PRO_SMOOTH : PRO_RESTRICT, EPI_RESID, live));
  }
  if (g.ns) k_batch_bottom<float, true><<<g.ninst, fft_threads<float>(), g.bottom_smem, g.stream>>>(g.plans, live);
  else k_batch_bottom<float, false><<<g.ninst, fft_threads<float>(), g.bottom_smem, g.stream>>>(g.plans, live);
  TPCB_CUDA(B, cudaGetLastError());
  for (int li = g.nl - 1; li >= 0; --li) {
    const LevelArgs<float>* a = (li == 0 && !first) ? g.post_r : g.post + (size_t)li * g.ninst;
    TPC_TRY(product(B, g, li, a, PRO_PROLONG, EPI_JACOBI, live));
  }
  return TPC_OK;
}

// One outer iteration of the group with `cycles` inner cycles (mirrors enqueue_iteration).
int iteration(tpc_batch* B, tpc_batch::Group& g, int cycles) {
  const int ni = g.ninst;
  const int* live0 = g.live;
  const dim3 eg(grid_for(g.n), ni);
  cudaStream_t s = g.stream;
  k_batch_to_f32<<<eg, NTHREADS, 0, s>>>(g.iter, live0, g.n);
  TPC_TRY(vcycle(B, g, true, live0));
  k_batch_copy<<<eg, NTHREADS, 0, s>>>(g.iter, live0, g.n);
  for (int c = 1; c < cycles; ++c) {
    const int* lc = g.live + (size_t)c * ni;
    TPC_TRY(product(B, g, 0, g.resid, PRO_NONE, EPI_RESID, lc));
    TPC_TRY(vcycle(B, g, false, lc));
    k_batch_axpy<<<eg, NTHREADS, 0, s>>>(g.iter, lc, g.n);
  }
  k_batch_axpy_scaled<<<eg, NTHREADS, 0, s>>>(g.iter, live0, g.n);
  k_batch_box_local<<<dim3(2 * g.box_nblk, ni), box::NT, 0, s>>>(g.boxa, live0);
  k_batch_box_offsets<<<ni, 1024, 0, s>>>(g.boxa, live0);
  k_batch_box_resid<<<dim3(g.box_gx, 2, ni), box::NT, 0, s>>>(g.boxa, live0);
  k_batch_sumsq_partial<<<dim3(NORM_BLOCKS, ni), NTHREADS, 0, s>>>(g.iter, live0, g.n, g.part);
  k_batch_sumsq_final<<<ni, 32, 0, s>>>(g.iter, live0, g.part, NORM_BLOCKS, g.out);
  TPCB_CUDA(B, cudaGetLastError());
  return TPC_OK;
}

int graph(tpc_batch* B, tpc_batch::Group& g, int cycles) {
  if (g.exec[cycles]) return TPC_OK;
  cudaGraph_t gr = nullptr;
  TPCB_CUDA(B, cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal));
  const int rc = iteration(B, g, cycles);
  cudaError_t ce = cudaStreamEndCapture(g.stream, &gr);
  if (rc != TPC_OK) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  if (ce != cudaSuccess) return bfail(B, ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&g.exec[cycles], gr, 0);
  cudaGraphDestroy(gr);
  if (ce != cudaSuccess) {
    g.exec[cycles] = nullptr;
    return bfail(B, ce, "cudaGraphInstantiate");
  }
  return TPC_OK;
}

// Device arrays of a group: every member's stage arguments, built with stage_args exactly as
// its lone V-cycle builds them.
int build_group(tpc_batch* B, tpc_batch::Group& g) {
  const int ni = g.ninst;
  tpc_handle* H0 = B->hs[g.idx[0]];
  const Hier<float>& S0 = H0->s;
  g.ns = H0->prm.variant != TPC_SPD;
  g.nl = S0.bottom_li;
  g.bottom_smem = S0.bottom_smem;
  TPCB_CUDA(B, cudaFuncSetAttribute(k_batch_bottom<float, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 150 * 1024));
  TPCB_CUDA(B, cudaFuncSetAttribute(k_batch_bottom<float, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 150 * 1024));
  g.n = H0->d.lev[0].n;
  g.box_nblk = H0->box_args.nblk;
  g.box_gx = (int)std::min<long long>((H0->box_args.N + box::NT - 1) / box::NT, 4 * 152);
  for (int li = 0; li < g.nl; ++li) g.lev.push_back(&S0.lev[li]);
  TPCB_CUDA(B, cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
  TPCB_CUDA(B, cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming));
  std::vector<LevelArgs<float>> pre((size_t)g.nl * ni), post((size_t)g.nl * ni), pre_r(ni),
      post_r(ni), resid(ni);
  std::vector<BottomPlan<float>*> plans(ni);
  std::vector<IterPtrs> iter(ni);
  std::vector<box::BoxArgs> boxa(ni);
  for (int j = 0; j < ni; ++j) {
    tpc_handle* H = B->hs[g.idx[j]];
    const Hier<float>& S = H->s;
    for (int li = 0; li < g.nl; ++li) {
      const DevLevel<float>& L = S.lev[li];
      float* e = S.e[li];
      float* t = S.t[li];
      Prologue<float> first;
      first.mode = li == 0 ? PRO_SMOOTH : PRO_RESTRICT;
      first.xout = e;
      first.fout = S.f[li];
      first.rfine = li == 0 ? nullptr : S.t[li - 1];
      Prologue<float> corr;
      corr.mode = PRO_PROLONG;
      corr.xout = e;
      corr.ec = S.t[li + 1];
      const float* f = li == 0 ? S.f[0] : S.f[li];
      pre[(size_t)li * ni + j] = stage_args<float>(S, L, e, f, t, EPI_RESID, false, first);
      post[(size_t)li * ni + j] = stage_args<float>(S, L, e, f, t, EPI_JACOBI, true, corr);
      if (li == 0) {
        pre_r[j] = stage_args<float>(S, L, e, H->res32, t, EPI_RESID, false, first);
        post_r[j] = stage_args<float>(S, L, e, H->res32, t, EPI_JACOBI, true, corr);
        resid[j] = stage_args<float>(S, L, H->acc32, S.f[0], H->res32, EPI_RESID, false,
                                     Prologue<float>());
      }
    }
    plans[j] = S.bottom;
    iter[j] = IterPtrs{H->r0, H->u, H->sumsq, S.f[0], H->acc32, S.t[0]};
    boxa[j] = H->box_args;
    boxa[j].x = H->u;
    boxa[j].b = H->b;
    boxa[j].r = H->r0;
  }
  TPC_TRY(balloc(B, &g.pre, pre.size()));
  TPC_TRY(balloc(B, &g.post, post.size()));
  TPC_TRY(balloc(B, &g.pre_r, (size_t)ni));
  TPC_TRY(balloc(B, &g.post_r, (size_t)ni));
  TPC_TRY(balloc(B, &g.resid, (size_t)ni));
  TPC_TRY(balloc(B, &g.plans, (size_t)ni));
  TPC_TRY(balloc(B, &g.iter, (size_t)ni));
  TPC_TRY(balloc(B, &g.boxa, (size_t)ni));
  TPC_TRY(balloc(B, &g.live, (size_t)33 * ni));
  TPC_TRY(bpinned(B, &g.live_host, (size_t)33 * ni));
  TPC_TRY(balloc(B, &g.part, (size_t)ni * NORM_BLOCKS));
  TPC_TRY(balloc(B, &g.out, (size_t)ni));
  TPC_TRY(bpinned(B, &g.out_host, (size_t)ni));
  TPC_TRY(balloc(B, &g.sync, 1));
  TPC_TRY(balloc(B, &g.err, 1));
  TPC_TRY(bpinned(B, &g.err_host, 1));
  TPC_TRY(upload_vec(B, g.pre, pre, g.stream));
  TPC_TRY(upload_vec(B, g.post, post, g.stream));
  TPC_TRY(upload_vec(B, g.pre_r, pre_r, g.stream));
  TPC_TRY(upload_vec(B, g.post_r, post_r, g.stream));
  TPC_TRY(upload_vec(B, g.resid, resid, g.stream));
  TPC_TRY(upload_vec(B, g.plans, plans, g.stream));
  TPC_TRY(upload_vec(B, g.iter, iter, g.stream));
  TPC_TRY(upload_vec(B, g.boxa, boxa, g.stream));
  TPCB_CUDA(B, cudaMemsetAsync(g.err, 0, sizeof(int), g.stream));
  TPCB_CUDA(B, cudaStreamSynchronize(g.stream));
  return TPC_OK;
}

void destroy(tpc_batch* B) {
  if (!B) return;
  for (auto& g : B->groups) {
    for (cudaGraphExec_t e : g.exec)
      if (e) cudaGraphExecDestroy(e);
    if (g.stream) cudaStreamSynchronize(g.stream);
    if (g.ev) cudaEventDestroy(g.ev);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  for (void* p : B->dev) cudaFree(p);
  for (void* p : B->pinned) cudaFreeHost(p);
  (void)cudaGetLastError();
  delete B;
}

// solve_step's bookkeeping for a stage-batched instance, given its new ||r||^2: the next
// iteration's inner-cycle count, or 0 when the solve is over.
int decide(SolveState& st, double ss) {
  tpc_handle* H = st.H;
  if (!st.started) {
    st.started = true;
    st.r0 = std::sqrt(ss);
    st.rel = (st.r0 > 0.0) ? 1.0 : 0.0;
    if (!std::isfinite(st.r0)) {
      H->err = "right-hand side or initial residual is not finite";
      st.status = TPC_EINVAL;
      st.done = true;
      return 0;
    }
  } else {
    ++st.it;
    st.rel = std::sqrt(ss) / st.r0;
    if (!std::isfinite(st.rel)) {
      H->err = "residual became non-finite";
      st.status = TPC_EDIVERGED;
      st.done = true;
      return 0;
    }
  }
  if (!(st.rel >= st.tol && st.r0 > 0.0)) {
    st.done = true;
    return 0;
  }
  if (st.it >= H->prm.max_iters) {
    st.status = TPC_ENOTCONV;
    st.done = true;
    return 0;
  }
  const int c = next_cycles(st);
  st.rel_prev = st.rel;
  st.cycles = c;
  H->last_cycles += c;
  return c;
}

}  // namespace batch
}  // namespace tpc

extern "C" {

int tpc_batch_create(tpc_handle* const* hs, int count, tpc_batch** out) {
  return tpc_batch_create_2d(hs, count, nullptr, 0, out);
}

int tpc_batch_create_2d(tpc_handle* const* hs, int count, tpc2d_handle* const* hs2, int count2,
                        tpc_batch** out) {
  using namespace tpc::batch;
  if (!out || count < 0 || (count > 0 && !hs) || count2 < 0 || (count2 > 0 && !hs2)) {
    set_host_error("bad argument to tpc_batch_create");
    return TPC_EINVAL;
  }
  *out = nullptr;
  std::vector<tpc2d_handle*> sorted2(hs2, hs2 + count2);
  for (tpc2d_handle* H : sorted2)
    if (!H) {
      set_host_error("tpc_batch_create: NULL 2-D handle");
      return TPC_EINVAL;
    }
  std::sort(sorted2.begin(), sorted2.end());
  if (std::adjacent_find(sorted2.begin(), sorted2.end()) != sorted2.end()) {
    set_host_error("tpc_batch_create: a 2-D handle appears twice (each instance needs its own)");
    return TPC_EINVAL;
  }
  std::vector<tpc_handle*> sorted(hs, hs + count);
  for (tpc_handle* H : sorted)
    if (!H) {
      set_host_error("tpc_batch_create: NULL handle");
      return TPC_EINVAL;
    }
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    set_host_error("tpc_batch_create: a handle appears twice (each instance needs its own)");
    return TPC_EINVAL;
  }
  tpc_batch* B = new (std::nothrow) tpc_batch();
  if (!B) return TPC_ENOMEM;
  B->hs.assign(hs, hs + count);
  B->hs2.assign(hs2, hs2 + count2);
  std::map<std::vector<long long>, std::vector<int>> keyed;
  for (int i = 0; i < count; ++i) {
    if (eligible(B->hs[i])) keyed[group_key(B->hs[i])].push_back(i);
    else B->solo.push_back(i);
  }
  for (auto& kv : keyed) {
    B->groups.emplace_back();
    tpc_batch::Group& g = B->groups.back();
    g.idx = kv.second;
    g.ninst = (int)g.idx.size();
  }
  for (auto& g : B->groups) {
    const int rc = build_group(B, g);
    if (rc != TPC_OK) {
      set_host_error(B->err);
      destroy(B);
      return rc;
    }
  }
  *out = B;
  return TPC_OK;
}

int tpc_batch_solve(tpc_batch* B, const double* const* b_dev, double* const* x_dev, double tol,
                    int* iters_out, double* relres_out, int* status_out) {
  using namespace tpc::batch;
  const int count = B ? (int)B->hs.size() : 0;
  const int count2 = B ? (int)B->hs2.size() : 0;
  if (!B || !(tol >= 0.0) || (count + count2 > 0 && (!b_dev || !x_dev))) {
    set_host_error("bad argument to tpc_batch_solve");
    return TPC_EINVAL;
  }
  for (int i = 0; i < count + count2; ++i)
    if (!b_dev[i] || !x_dev[i]) {
      set_host_error("tpc_batch_solve: NULL vector");
      return TPC_EINVAL;
    }
  NvtxScope range("tpc_batch_solve");
  std::vector<SolveState> st(count);
  for (int i = 0; i < count; ++i) {
    st[i].H = B->hs[i];
    const int rc = solve_begin(st[i], b_dev[i], x_dev[i], tol, 0);
    if (rc != TPC_OK) {
      set_host_error(B->hs[i]->err);
      return rc;
    }
  }
  // the 2-D instances: their own iteration graphs on their own streams, advanced by polling
  std::vector<tpc::twod::Solve2State> st2(count2);
  for (int i = 0; i < count2; ++i) {
    st2[i].H = B->hs2[i];
    const int rc = tpc::twod::solve2_begin(st2[i], b_dev[count + i], x_dev[count + i], tol, 0);
    if (rc != TPC_OK) {
      set_host_error(B->hs2[i]->err);
      return rc;
    }
  }
  int active2 = count2;
  // the grouped instances' first decisions need their initial norms on the host
  for (auto& g : B->groups)
    for (int j : g.idx) TPCB_CUDA(B, cudaEventSynchronize(B->hs[j]->ev));
  std::vector<int> cyc(count, 0);
  for (auto& g : B->groups)
    for (int j : g.idx) cyc[j] = decide(st[j], *B->hs[j]->sumsq_host);
  int active_solo = (int)B->solo.size();
  // a group's next iteration, with every member that still iterates (none: the group is done)
  auto launch = [&](tpc_batch::Group& g) -> int {
    int cmax = 0;
    for (int jj = 0; jj < g.ninst; ++jj) cmax = std::max(cmax, cyc[g.idx[jj]]);
    if (cmax == 0) return TPC_OK;
    for (int c = 0; c < cmax; ++c)
      for (int jj = 0; jj < g.ninst; ++jj) {
        const int ci = cyc[g.idx[jj]];
        g.live_host[(size_t)c * g.ninst + jj] = (c == 0) ? (ci > 0) : (ci > c);
      }
    TPC_TRY(graph(B, g, cmax));
    TPCB_CUDA(B, cudaMemcpyAsync(g.live, g.live_host, sizeof(int) * (size_t)cmax * g.ninst,
                                 cudaMemcpyHostToDevice, g.stream));
    TPCB_CUDA(B, cudaGraphLaunch(g.exec[cmax], g.stream));
    TPCB_CUDA(B, cudaMemcpyAsync(g.out_host, g.out, sizeof(double) * g.ninst,
                                 cudaMemcpyDeviceToHost, g.stream));
    TPCB_CUDA(B, cudaMemcpyAsync(g.err_host, g.err, sizeof(int), cudaMemcpyDeviceToHost, g.stream));
    TPCB_CUDA(B, cudaEventRecord(g.ev, g.stream));
    g.in_flight = true;
    return TPC_OK;
  };
  for (auto& g : B->groups) TPC_TRY(launch(g));
  // every group, lone instance and 2-D instance advances as soon as its own latest read-back
  // has arrived
  for (;;) {
    bool any = false;
    for (auto& g : B->groups) {
      if (!g.in_flight) continue;
      any = true;
      const cudaError_t q = cudaEventQuery(g.ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return bfail(B, q, "cudaEventQuery");
      g.in_flight = false;
      if (*g.err_host) {
        B->err = "a device-side wait of a batched product gave up (grid barrier not reached)";
        set_host_error(B->err);
        return TPC_ESYNC;
      }
      for (int jj = 0; jj < g.ninst; ++jj) {
        const int j = g.idx[jj];
        if (cyc[j] == 0) continue;
        *B->hs[j]->sumsq_host = g.out_host[jj];
        cyc[j] = decide(st[j], g.out_host[jj]);
        B->hs[j]->launches += 1;
      }
      TPC_TRY(launch(g));
    }
    // instances outside the groups: their own iteration graphs
    if (active_solo > 0) {
      any = true;
      for (int i : B->solo) {
        if (st[i].done) continue;
        const cudaError_t q = cudaEventQuery(B->hs[i]->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return bfail(B, q, "cudaEventQuery");
        const int rc = solve_step(st[i]);
        if (rc != TPC_OK) {
          set_host_error(B->hs[i]->err);
          return rc;
        }
        if (st[i].done) {
          TPC_TRY(solve_finish(st[i]));
          --active_solo;
        }
      }
    }
    if (active2 > 0) {
      any = true;
      for (int i = 0; i < count2; ++i) {
        if (st2[i].done) continue;
        tpc2d_handle* H2 = B->hs2[i];
        const cudaError_t q = cudaEventQuery(H2->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return bfail(B, q, "cudaEventQuery");
        const int rc = tpc::twod::solve2_step(st2[i]);
        if (rc != TPC_OK) {
          set_host_error(H2->err);
          return rc;
        }
        if (st2[i].done) {
          if (st2[i].status != TPC_EINVAL) TPC_TRY(tpc::twod::solve2_finish(st2[i]));
          --active2;
        }
      }
    }
    if (!any) break;
  }
  int worst = TPC_OK;
  for (int i = 0; i < count2; ++i) {
    TPCB_CUDA(B, cudaStreamSynchronize(B->hs2[i]->stream));
    const int j = count + i;
    if (iters_out) iters_out[j] = st2[i].it;
    if (relres_out) relres_out[j] = st2[i].rel;
    if (status_out) status_out[j] = st2[i].status;
    if (st2[i].status < worst || (worst == TPC_OK && st2[i].status != TPC_OK)) worst = st2[i].status;
  }
  for (int i = 0; i < count; ++i) {
    tpc_handle* H = B->hs[i];
    if (std::find(B->solo.begin(), B->solo.end(), i) == B->solo.end()) TPC_TRY(solve_finish(st[i]));
    TPCB_CUDA(B, cudaStreamSynchronize(H->stream));
    if (iters_out) iters_out[i] = st[i].it;
    if (relres_out) relres_out[i] = st[i].rel;
    if (status_out) status_out[i] = st[i].status;
    if (st[i].status < worst || (worst == TPC_OK && st[i].status != TPC_OK)) worst = st[i].status;
  }
  return worst;
}

int tpc_batch_set_product_mode(tpc_batch* B, int mode) {
  if (!B || mode < TPC_BATCH_AUTO || mode > TPC_BATCH_THREE_PASS) {
    set_host_error("bad argument to tpc_batch_set_product_mode");
    return TPC_EINVAL;
  }
  if (mode == B->product_mode) return TPC_OK;
  for (auto& g : B->groups) {
    if (g.stream) cudaStreamSynchronize(g.stream);
    for (cudaGraphExec_t& e : g.exec)
      if (e) {
        cudaGraphExecDestroy(e);
        e = nullptr;
      }
  }
  B->product_mode = mode;
  return TPC_OK;
}

int tpc_batch_groups(const tpc_batch* B) { return B ? (int)B->groups.size() : -1; }

int tpc_batch_grouped_instances(const tpc_batch* B) {
  return B ? (int)(B->hs.size() - B->solo.size()) : -1;
}

void tpc_batch_destroy(tpc_batch* B) { tpc::batch::destroy(B); }

int tpc_grid_wait_selftest(unsigned max_polls, int* gave_up, int* passed) {
  if (!gave_up || !passed) return TPC_EINVAL;
  unsigned* sync = nullptr;
  int* flags = nullptr;
  cudaError_t e = cudaMalloc(&sync, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&flags, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(sync, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(flags, 0, 2 * sizeof(int));
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4);
    cfg.blockDim = dim3(32);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, tpc::batch::k_grid_wait_selftest, sync, flags, max_polls,
                           flags + 1);
  }
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, flags, sizeof(h), cudaMemcpyDeviceToHost);
  if (sync) cudaFree(sync);
  if (flags) cudaFree(flags);
  if (e != cudaSuccess) {
    set_host_error(std::string("tpc_grid_wait_selftest: ") + cudaGetErrorString(e));
    return TPC_ECUDA;
  }
  *gave_up = h[0];
  *passed = h[1];
  return TPC_OK;
}

}  // extern "C"
