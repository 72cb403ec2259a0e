// Sequential SL time stepping u_{n+1} = S_n u_n (eq. (one-step) with g = 0) by one thread-block cluster.
//
// The time loop is inherently serial, so the work of one step (nx gathers) is what a single launch can
// spread.  The slice is split into C contiguous chunks, one per CTA of a cluster (C <= 16), kept in each
// CTA's shared memory (double buffered).  A gather near a chunk edge reads the neighbouring CTA's chunk
// through distributed shared memory, and one cluster barrier per step orders the writes of step n
// before the reads of step n+1.  The step arithmetic is the one of the single-CTA kernel (same weights,
// same summation order), so both give identical results.
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace mgrit {

namespace {

constexpr int kClusterThreads = 256;

template <int P, typename R, int PPT>
struct StepRegs;

template <int P, int PPT>
struct StepRegs<P, float, PPT> {
  float eps[PPT];
  int base[PPT];
};

template <int P, int PPT>
struct StepRegs<P, double, PPT> {
  double w[PPT][P + 1];
  int base[PPT];
};

template <int P, typename R, int PPT>
__device__ __forceinline__ void load_step(StepRegs<P, R, PPT>& s, const LevelTables& T, int n, int lo, int ppt) {
  const int nx = T.nx;
#pragma unroll
  for (int t = 0; t < PPT; ++t) {
    if (t >= ppt) break;
    const int i = lo + threadIdx.x + t * kClusterThreads;
    s.base[t] = i + (int)__ldg(T.shift + (size_t)n * nx + i);
    if constexpr (std::is_same<R, float>::value) {
      s.eps[t] = __ldg(T.eps32 + (size_t)n * nx + i);
    } else {
      const double* wr = T.w64 + (size_t)n * (P + 1) * nx + i;
#pragma unroll
      for (int a = 0; a <= P; ++a) s.w[t][a] = __ldg(wr + (size_t)a * nx);
    }
  }
}

// u0: [nx] (NULL = zero); out: store_all ? [(N+1)][nx] (row 0 = u0) : [nx] (the final slice).
// chunk = nx / C is a power of two and a multiple of the block size; ppt = chunk / blockDim.x <= PPT.
template <int P, typename R, int PPT>
__global__ void __launch_bounds__(kClusterThreads) k_sequential_cluster_1d(LevelTables T, int N,
                                                                           const R* __restrict__ u0,
                                                                           R* __restrict__ out, int store_all,
                                                                           int log2_chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int nx = T.nx, chunk = 1 << log2_chunk, lo = rank * chunk;
  const int ppt = chunk / kClusterThreads;
  R* buf0 = reinterpret_cast<R*>(smem_raw);
  R* buf1 = buf0 + chunk;
  for (int q = threadIdx.x; q < chunk; q += kClusterThreads) {
    const R v = u0 ? u0[lo + q] : (R)0;
    buf0[q] = v;
    if (store_all) out[lo + q] = v;
  }
  StepRegs<P, R, PPT> cur, nxt;
  if (N > 0) load_step<P, R, PPT>(nxt, T, 0, lo, ppt);
  cl.sync();
  for (int n = 0; n < N; ++n) {
    cur = nxt;
    if (n + 1 < N) load_step<P, R, PPT>(nxt, T, n + 1, lo, ppt);
    const R* src = (n & 1) ? buf1 : buf0;
    R* dst = (n & 1) ? buf0 : buf1;
    R* orow = store_all ? out + (size_t)(n + 1) * nx : (n == N - 1 ? out : nullptr);
#pragma unroll
    for (int t = 0; t < PPT; ++t) {
      if (t >= ppt) break;
      R w[P + 1];
      if constexpr (std::is_same<R, float>::value) {
        lagrange_weights<P, float>(cur.eps[t], w);
      } else {
#pragma unroll
        for (int a = 0; a <= P; ++a) w[a] = cur.w[t][a];
      }
      R v[P + 1];
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int idx = wrap_pow2(cur.base[t] + a, nx);
        const int owner = idx >> log2_chunk, off = idx & (chunk - 1);
        const R* p = owner == rank ? src : cl.map_shared_rank(src, (unsigned)owner);
        v[a] = p[off];
      }
      R acc = w[0] * v[0];
#pragma unroll
      for (int a = 1; a <= P; ++a) acc += w[a] * v[a];
      const int q = threadIdx.x + t * kClusterThreads;
      dst[q] = acc;
      if (orow) orow[lo + q] = acc;
    }
    cl.sync();
  }
}

template <int P, typename R, int PPT>
cudaError_t launch_cluster(const LevelTables& T, int N, const R* u0, R* out, int store_all, int C, int log2_chunk,
                           cudaStream_t st) {
  auto kern = k_sequential_cluster_1d<P, R, PPT>;
  const size_t smem = 2 * ((size_t)1 << log2_chunk) * sizeof(R);
  cudaError_t e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  e = cudaLaunchKernelEx(&cfg, kern, T, N, u0, out, store_all, log2_chunk);
  return e;
}

template <typename R, int PPT>
cudaError_t dispatch_p(const LevelTables& T, int N, const R* u0, R* out, int store_all, int C, int l2,
                       cudaStream_t st) {
  if (T.p == 1) return launch_cluster<1, R, PPT>(T, N, u0, out, store_all, C, l2, st);
  if (T.p == 3) return launch_cluster<3, R, PPT>(T, N, u0, out, store_all, C, l2, st);
  return launch_cluster<5, R, PPT>(T, N, u0, out, store_all, C, l2, st);
}

template <typename R>
cudaError_t sequential_cluster(const LevelTables& T, int N, const R* u0, R* out, int store_all, cudaStream_t st) {
  const int nx = T.nx;
  // one 256-point chunk per CTA, at most 16 CTAs (two chunks per thread with 8 when 16 is refused)
  for (int C : {16, 8}) {
    int c = nx / kClusterThreads;
    if (c > C) c = C;
    if (c < 1 || nx % (c * kClusterThreads) != 0) return cudaErrorNotSupported;
    const int chunk = nx / c;
    int l2 = 0;
    while ((1 << l2) < chunk) ++l2;
    const int ppt = chunk / kClusterThreads;
    cudaError_t e = cudaErrorNotSupported;
    if (ppt == 1) e = dispatch_p<R, 1>(T, N, u0, out, store_all, c, l2, st);
    else if (ppt == 2) e = dispatch_p<R, 2>(T, N, u0, out, store_all, c, l2, st);
    if (e != cudaErrorNotSupported) return e;
  }
  return cudaErrorNotSupported;
}

}  // namespace

cudaError_t launch_sequential_cluster_1d(const LevelTables& T, int N, const void* u0, void* out, int store_all,
                                         int is_double, cudaStream_t st) {
  if (T.solver != nullptr || T.trans) return cudaErrorNotSupported;
  if (is_double) return sequential_cluster<double>(T, N, (const double*)u0, (double*)out, store_all, st);
  return sequential_cluster<float>(T, N, (const float*)u0, (float*)out, store_all, st);
}

}  // namespace mgrit
