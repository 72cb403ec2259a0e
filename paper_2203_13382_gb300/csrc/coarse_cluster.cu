// FP64 coarse-level relaxation split over a thread-block cluster per coarse interval.
//
// On coarse levels with few intervals (J of 4 or 32 on the 1D workload) one CTA per interval would
// occupy J SMs, and on GB300 a CTA's FP64 steps are bound by its own SM's FP64 pipe (2 FMA a clock).
// Here the slice of interval j is cut into C contiguous chunks, one per CTA of a cluster (C <= 16), so
// C SMs share each step.  A step is the one of relax_kernels.cu (gather with the FP64 weights of the
// w64 table, then the partitioned periodic banded solve with the stored factorisation of
// solver_layout.cuh) with the same operations in the same order, so the results are identical to the
// single-CTA kernel; the gather reads other chunks and the solve reads neighbouring partitions through
// distributed shared memory, with cluster barriers where the single-CTA kernel has block barriers.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "solver_layout.cuh"

namespace cg = cooperative_groups;

namespace mgrit {

namespace {

constexpr int kClusterRelaxThreads = 256;

template <int P>
__global__ void __launch_bounds__(kClusterRelaxThreads, P <= 3 ? 2 : 1) k_relax_cluster_1d(LevelTables T, RelaxArgs a,
                                                                           int log2_chunk) {
  constexpr int B = (P + 1) / 2, Q = kPartRows - B, BB = B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int j = (int)blockIdx.x / C;
  const int nx = T.nx, chunk = 1 << log2_chunk, lo = rank * chunk;
  const int Pc = chunk / kPartRows, log2_pc = log2_chunk - 3;  // partitions of this CTA
  const SolverGeom G = solver_geom(nx, P);
  const int Pall = G.P;
  double* src = reinterpret_cast<double*>(smem_raw);
  double* dst = src + chunk;
  double* ytail = dst + chunk;  // [Pc][B] each
  double* gb0 = ytail + Pc * B;
  double* gb1 = gb0 + Pc * B;
  double* xsb = gb1 + Pc * B;
  // the B values of global partition kk in exchange buffer buf (this CTA's or another's)
  auto part = [&](double* buf, int kk) -> const double* {
    const int owner = kk >> log2_pc;
    double* b = owner == rank ? buf : cl.map_shared_rank(buf, (unsigned)owner);
    return b + (kk & (Pc - 1)) * B;
  };
  {
    const double* st = a.start ? (const double*)a.start + (size_t)j * a.start_stride + lo : nullptr;
    const double* co = a.corr ? (const double*)a.corr + (size_t)j * a.corr_stride + lo : nullptr;
    double* wb = a.start_wb ? (double*)a.start_wb + (size_t)j * a.wb_stride + lo : nullptr;
    for (int q = threadIdx.x; q < chunk; q += kClusterRelaxThreads) {
      double v = st ? st[q] : 0.0;
      if (co) v += co[q];
      src[q] = v;
      if (wb) wb[q] = v;
    }
  }
  if (j >= a.J) return;  // the extra cluster: only the correction of the last C-point (whole cluster)
  cl.sync();
  const int kl = threadIdx.x;  // local partition of this thread
  const bool act = kl < Pc;
  const int k = rank * Pc + kl;  // global partition
  const int g0 = kl * kPartRows;
  for (int s = 0; s < a.nsteps; ++s) {
    const int n = j * a.m + s;
    // gather: dst[i] = sum_a w_a src[i + shift + a] over this chunk's points
    {
      const double* __restrict__ wrow = T.w64 + (size_t)n * (P + 1) * nx;
      const uint16_t* __restrict__ shrow = T.shift + (size_t)n * nx;
#pragma unroll 1
      for (int q = threadIdx.x; q < chunk; q += kClusterRelaxThreads) {
        const int i = lo + q;
        double w[P + 1];
#pragma unroll
        for (int e = 0; e <= P; ++e) w[e] = __ldg(wrow + (size_t)e * nx + i);
        const int b = i + (int)__ldg(shrow + i);
        double v[P + 1];
#pragma unroll
        for (int e = 0; e <= P; ++e) {
          const int idx = wrap_pow2(b + e, nx);
          const int owner = idx >> log2_chunk;
          const double* p = owner == rank ? src : cl.map_shared_rank(src, (unsigned)owner);
          v[e] = p[idx & (chunk - 1)];
        }
        double acc = w[0] * v[0];
#pragma unroll
        for (int e = 1; e <= P; ++e) acc += w[e] * v[e];
        dst[q] = acc;
      }
    }
    __syncthreads();
    // correction solve x <- M^{-1} x on this chunk's partitions (stored factorisation of step n); the
    // factor loads of each phase are issued before the cluster barrier that precedes their use
    const double* data = (const double*)T.solver + (size_t)n * T.solver_stride;
    const double* pcr_src = data + G.pcr_off;
    double y[Q], g[B], hd[B];
    if (act) {
#pragma unroll
      for (int r = 0; r < B; ++r) hd[r] = dst[g0 + r];
#pragma unroll
      for (int r = 0; r < Q; ++r) y[r] = dst[g0 + B + r];
      auto LU = [&](int r, int f) -> double { return __ldg(data + (size_t)rec_lu(B, r, f) * Pall + k); };
#pragma unroll
      for (int r = 0; r < Q; ++r)
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r - t >= 0) y[r] -= LU(r, t - 1) * y[r - t];
#pragma unroll
      for (int r = Q - 1; r >= 0; --r) {
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r + t < Q) y[r] -= LU(r, B + t) * y[r + t];
        y[r] *= LU(r, B);
      }
#pragma unroll
      for (int e = 0; e < B; ++e) ytail[kl * B + e] = y[Q - B + e];
    }
    double ct[BB], ch[BB];
    if (act) {
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        ct[e] = __ldg(data + (size_t)rec_ct(B, Q, 0, e) * Pall + k);
        ch[e] = __ldg(data + (size_t)rec_ch(B, Q, 0, e) * Pall + k);
      }
    }
    cl.sync();
    if (act) {
      const double* yt = part(ytail, (k + Pall - 1) & (Pall - 1));
#pragma unroll
      for (int e = 0; e < B; ++e) {
        double v = hd[e];
#pragma unroll
        for (int c = 0; c < B; ++c) v -= ct[e * B + c] * yt[c] + ch[e * B + c] * y[c];
        g[e] = v;
      }
    }
    // block parallel cyclic reduction on the separators, one cluster barrier a level
    double fin[BB];
    for (int t = 0; t < G.T; ++t) {
      double* buf = (t & 1) ? gb1 : gb0;
      double cf[2 * BB];
      if (act) {
#pragma unroll
        for (int e = 0; e < B; ++e) buf[kl * B + e] = g[e];
        const double* lv = pcr_src + (size_t)t * 2 * BB * Pall;
#pragma unroll
        for (int e = 0; e < 2 * BB; ++e) cf[e] = lv[(size_t)e * Pall + k];
        if (t == G.T - 1) {
#pragma unroll
          for (int e = 0; e < BB; ++e) fin[e] = pcr_src[(G.fin_off - G.pcr_off) + (size_t)e * Pall + k];
        }
      }
      cl.sync();
      if (act) {
        const int d = 1 << t;
        const double* pm = part(buf, (k - d) & (Pall - 1));
        const double* pp = part(buf, (k + d) & (Pall - 1));
        double gm[B], gp[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
          gm[e] = pm[e];
          gp[e] = pp[e];
        }
#pragma unroll
        for (int e = 0; e < B; ++e) {
          double v = g[e];
#pragma unroll
          for (int c = 0; c < B; ++c) v += cf[e * B + c] * gm[c] + cf[BB + e * B + c] * gp[c];
          g[e] = v;
        }
      }
    }
    double xs[B];
    if (act) {
#pragma unroll
      for (int e = 0; e < B; ++e) {
        double v = 0.0;
#pragma unroll
        for (int c = 0; c < B; ++c) v += fin[e * B + c] * g[c];
        xs[e] = v;
        xsb[kl * B + e] = v;
      }
    }
    cl.sync();
    if (act) {
      const double* pn = part(xsb, (k + 1) & (Pall - 1));
      double xn[B];
#pragma unroll
      for (int e = 0; e < B; ++e) {
        xn[e] = pn[e];
        dst[g0 + e] = xs[e];
      }
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        double v = y[r];
#pragma unroll
        for (int c = 0; c < B; ++c) {
          v -= __ldg(data + (size_t)rec_v(B, Q, r, c) * Pall + k) * xs[c];
          v -= __ldg(data + (size_t)rec_w(B, Q, r, c) * Pall + k) * xn[c];
        }
        dst[g0 + B + r] = v;
      }
    }
    __syncthreads();
    // right-hand side, F-point store, C-point output (this chunk's points)
    const bool last = (s == a.m - 1);
    const double* gr = a.g ? (const double*)a.g + (size_t)(n + 1) * nx + lo : nullptr;
    if (!last) {
      double* fs = a.fstore ? (double*)a.fstore + (size_t)(n + 1) * nx + lo : nullptr;
      if (gr || fs) {
        for (int q = threadIdx.x; q < chunk; q += kClusterRelaxThreads) {
          double v = dst[q];
          if (gr) v += gr[q];
          dst[q] = v;
          if (fs) fs[q] = v;
        }
      }
    } else if (a.mode == MODE_FC) {
      double* co = (double*)a.cout + (size_t)(j + 1) * a.c_stride + lo;
      for (int q = threadIdx.x; q < chunk; q += kClusterRelaxThreads) {
        double v = dst[q];
        if (gr) v += gr[q];
        co[q] = v;
      }
    } else {  // MODE_RES (no residual norm on coarse levels)
      const double* ci = a.cin ? (const double*)a.cin + (size_t)(j + 1) * a.c_stride + lo : nullptr;
      const double* cc = a.cin_corr ? (const double*)a.cin_corr + (size_t)(j + 1) * a.corr_stride + lo : nullptr;
      double* ro = (double*)a.rout + (size_t)(j + 1) * a.r_stride + lo;
      float* ro32 = a.rout32 ? a.rout32 + (size_t)(j + 1) * a.r_stride + lo : nullptr;
      for (int q = threadIdx.x; q < chunk; q += kClusterRelaxThreads) {
        double v = dst[q];
        if (gr && a.g_at_c) v += gr[q];
        if (cc) v -= (ci ? ci[q] : 0.0) + cc[q];
        else if (ci) v -= ci[q];
        ro[q] = v;
        if (ro32) ro32[q] = (float)v;
      }
    }
    cl.sync();  // every chunk of this step is final before the next gather reads it
    double* t = src;
    src = dst;
    dst = t;
  }
}

template <int P>
cudaError_t launch_cluster_relax(const LevelTables& T, const RelaxArgs& a, int C, cudaStream_t st) {
  auto kern = k_relax_cluster_1d<P>;
  const int chunk = T.nx / C;
  int l2 = 0;
  while ((1 << l2) < chunk) ++l2;
  constexpr int B = (P + 1) / 2;
  const size_t smem = (2 * (size_t)chunk + 4 * (size_t)(chunk / kPartRows) * B) * sizeof(double);
  cudaError_t e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((a.J + (a.extra_cta ? 1 : 0)) * C));
  cfg.blockDim = dim3(kClusterRelaxThreads);
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
  return cudaLaunchKernelEx(&cfg, kern, T, a, l2);
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 1;
  }
  return n;
}

}  // namespace

int cluster_relax_size(const LevelTables& T, const RelaxArgs& a) {
  if (T.cluster <= 0 || !T.solver || T.otf || T.trans || T.w64 == nullptr || a.norm_partial || a.J <= 0) return 1;
  int C = 1;
  if (T.cluster >= 2) {  // a fixed size
    while (C < 16 && 2 * C <= T.cluster) C *= 2;
  } else {  // the largest size whose J * C CTAs are resident at once (two a SM for p <= 3)
    const int slots = sm_count() * (T.p <= 3 ? 2 : 1);
    while (C < 16 && 2 * C * a.J <= slots) C *= 2;
  }
  // at most 256 partitions and at least one per CTA
  while (C > 1 && T.nx / C < kPartRows) C /= 2;
  if (C < 2 || T.nx / C > kClusterRelaxThreads * kPartRows) return 1;
  return C;
}

cudaError_t launch_relax_cluster_1d(const LevelTables& T, const RelaxArgs& a, int C, cudaStream_t st) {
  if (C < 2 || (C & (C - 1)) != 0 || C > 16 || T.nx % C != 0) return cudaErrorNotSupported;
  for (int c = C; c >= 2; c /= 2) {
    if (T.nx / c > kClusterRelaxThreads * kPartRows) break;
    cudaError_t e;
    if (T.p == 1) e = launch_cluster_relax<1>(T, a, c, st);
    else if (T.p == 3) e = launch_cluster_relax<3>(T, a, c, st);
    else e = launch_cluster_relax<5>(T, a, c, st);
    if (e != cudaErrorNotSupported) return e;
  }
  return cudaErrorNotSupported;
}

}  // namespace mgrit
