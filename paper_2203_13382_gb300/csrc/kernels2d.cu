// Two-dimensional kernels (Sec. 4 of the paper): the tensor-product SL step (eq. (SL2D_char1-2) and the
// interpolation of Sec. 4.1) over all coarse intervals at once, and the corrected coarse operator
// [I - diag(sigma_x)(I (x) D) - diag(sigma_y)(D (x) I)]^{-1} S (eq. (BEOper_2D)) with the paper's inexact
// solve: GMRES from a zero guess, stopped at relative residual rtol or after kmax iterations (Sec. 4.3).
//
// A 2D slice (nx * nx values) does not fit in shared memory, so a relaxation pass is a sequence of
// launches, one per step index k of the intervals, each updating every interval's slice in global memory.
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mgrit {

namespace {

constexpr int kThreads2d = 256;

// Coefficient of the centred stencil (delta^2)^B at offset o: (-1)^{B+o} C(2B, B+o) (compile time).
template <int B>
constexpr int dstencil_int(int o) {
  int c = 1;
  for (int t = 1; t <= B + o; ++t) c = c * (2 * B - (B + o) + t) / t;
  return ((B + o) & 1) ? -c : c;
}
constexpr int kThreadsGmres = 1024;  // one CTA per system: more loads in flight per SM

// FP64 systems keep ten FP64 projection sums a thread: 512 threads (128 registers) instead of 1024.
template <typename R>
constexpr int gmres_threads() {
  return std::is_same<R, double>::value ? 512 : kThreadsGmres;
}

// Weights of one axis for element pt of step row n.  FP32: from the stored eps; FP64: the weight table
// (or, without one, from the offset).
template <int P, typename R>
__device__ __forceinline__ void axis_weights(const LevelTables& T, int comp, int n, long long pt, R (&w)[P + 1]) {
  const long long off = ((long long)comp * T.nt + n) * T.npts + pt;
  if constexpr (std::is_same<R, float>::value) {
    lagrange_weights<P, float>(__ldg(T.eps32 + off), w);
  } else if (T.w64) {  // table [comp][n][a][pt]
    const double* wr = T.w64 + ((size_t)comp * T.nt + n) * (P + 1) * T.npts + pt;
#pragma unroll
    for (int a = 0; a <= P; ++a) w[a] = __ldg(wr + (size_t)a * T.npts);
  } else {
    const double s = __ldg(T.s64 + off);
    double e = s - floor(s);
    if (e >= 1.0) e -= 1.0;
    lagrange_weights<P, double>(e, w);
  }
}

// dst[j] = S_{n(j)} src[j] (+ g[n(j)+1]) for every interval j (blockIdx.y), n(j) = j*m + k (or the
// single step n0 when m == 0).
template <int P, typename R>
__global__ void __launch_bounds__(kThreads2d) k_step2d(LevelTables T, const R* __restrict__ src, R* __restrict__ dst,
                                                       int m, int k, int n0, const R* __restrict__ g, int add_g,
                                                       R* __restrict__ fstore) {
  const int j = blockIdx.y;
  const long long N = T.npts;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  const int n = m > 0 ? j * m + k : n0;
  const int nx = T.nx;
  int i, jj;
  split_pow2(pt, nx, i, jj);
  R wx[P + 1], wy[P + 1];
  axis_weights<P, R>(T, 0, n, pt, wx);
  axis_weights<P, R>(T, 1, n, pt, wy);
  const int bx = i + (int)__ldg(T.shift + (long long)n * N + pt);
  const int by = jj + (int)__ldg(T.shift + ((long long)T.nt + n) * N + pt);
  const R* s = src + (size_t)j * N;
  R acc = (R)0;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const R* row = s + (size_t)wrap_pow2(by + b, nx) * nx;
    R ra = wx[0] * __ldg(row + wrap_pow2(bx, nx));
#pragma unroll
    for (int a = 1; a <= P; ++a) ra += wx[a] * __ldg(row + wrap_pow2(bx + a, nx));
    acc += wy[b] * ra;
  }
  if (add_g && g) acc += g[(size_t)(n + 1) * N + pt];
  dst[(size_t)j * N + pt] = acc;
  if (fstore) fstore[(size_t)(n + 1) * N + pt] = acc;
}

// 1D: dst[j] = S_{n(j)} src[j] (+ g[n(j)+1]) on slices in global memory (the coarse passes that solve the
// correction by GMRES, solve_mode 1).  FP64 weights from the table, FP32 from eps; the summation order of
// the shared-memory gather (apply_gather), so both give the same values.
template <int P, typename R>
__global__ void __launch_bounds__(kThreads2d) k_step1d_g(LevelTables T, const R* __restrict__ src, R* __restrict__ dst,
                                                         int m, int k, int n0, const R* __restrict__ g, int add_g,
                                                         R* __restrict__ fstore) {
  const int j = blockIdx.y;
  const int nx = T.nx;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const int n = m > 0 ? j * m + k : n0;
  R w[P + 1];
  if constexpr (std::is_same<R, float>::value) {
    lagrange_weights<P, float>(__ldg(T.eps32 + (size_t)n * nx + i), w);
  } else {
    const double* wr = T.w64 + (size_t)n * (P + 1) * nx + i;
#pragma unroll
    for (int a = 0; a <= P; ++a) w[a] = __ldg(wr + (size_t)a * nx);
  }
  const int b = i + (int)__ldg(T.shift + (size_t)n * nx + i);
  const R* s = src + (size_t)j * nx;
  R acc = w[0] * s[wrap_pow2(b, nx)];
#pragma unroll
  for (int a = 1; a <= P; ++a) acc += w[a] * s[wrap_pow2(b + a, nx)];
  if (add_g && g) acc += g[(size_t)(n + 1) * nx + i];
  dst[(size_t)j * nx + i] = acc;
  if (fstore) fstore[(size_t)(n + 1) * nx + i] = acc;
}

// Transposed step dst[j] = S_row^T src[j] (+ g[n(j)+1]), FP64, row = nt-1-n(j) when T.reverse.  Target
// node (X, Y) receives w_a(eps_i) w_b(nu_i) src_i from every arrival point i whose stencil base node
// is (X - a, Y - b); the arrival points of each base node are read from the sorted buckets, so the sum
// has a fixed order (a deterministic scatter-add).
template <int P>
__global__ void __launch_bounds__(kThreads2d) k_step2d_T(LevelTables T, const double* __restrict__ src,
                                                         double* __restrict__ dst, int m, int k, int n0,
                                                         const double* __restrict__ g, double* __restrict__ fstore) {
  const int j = blockIdx.y;
  const long long N = T.npts;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  const int n = m > 0 ? j * m + k : n0;
  const int row = T.reverse ? T.nt - 1 - n : n;
  const int nx = T.nx, mask = nx - 1;
  int X, Y;
  split_pow2(pt, nx, X, Y);
  const int* bs = T.bstart + (size_t)row * (N + 1);
  const int* bp = T.bperm + (size_t)row * N;
  const double* sx = T.s64 + (size_t)row * N;
  const double* sy = T.s64 + ((size_t)T.nt + row) * N;
  // weight tables of the two axes ([comp][n][a][pt]); without them the weights follow from the offsets
  const double* wx = T.w64 ? T.w64 + (size_t)row * (P + 1) * N : nullptr;
  const double* wy = T.w64 ? T.w64 + ((size_t)T.nt + row) * (P + 1) * N : nullptr;
  const double* s = src + (size_t)j * N;
  double acc = 0.0;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int rowkey = ((Y - b) & mask) * nx;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int key = rowkey + ((X - a) & mask);
      const int q1 = __ldg(bs + key + 1);
      for (int q = __ldg(bs + key); q < q1; ++q) {
        const int i = __ldg(bp + q);
        double wa, wb;
        if (wx) {
          wa = __ldg(wx + (size_t)a * N + i);
          wb = __ldg(wy + (size_t)b * N + i);
        } else {
          double ex = __ldg(sx + i), ey = __ldg(sy + i);
          ex -= floor(ex);
          if (ex >= 1.0) ex -= 1.0;
          ey -= floor(ey);
          if (ey >= 1.0) ey -= 1.0;
          wa = lagrange_basis<P>(ex, a);
          wb = lagrange_basis<P>(ey, b);
        }
        acc += wa * wb * __ldg(s + i);
      }
    }
  }
  if (g) acc += g[(size_t)(n + 1) * N + pt];
  dst[(size_t)j * N + pt] = acc;
  if (fstore) fstore[(size_t)(n + 1) * N + pt] = acc;
}

// y = M x with M = I - diag(sx) (I (x) D) - diag(sy) (D (x) I), D = (delta^2)^B (periodic).
template <int B, typename R>
__device__ __forceinline__ R apply_M(const R* x, const R* sx, const R* sy, long long pt, int nx) {
  int i, jj;
  split_pow2(pt, nx, i, jj);
  const R* row = x + (size_t)jj * nx;
  R dxv = (R)0, dyv = (R)0;
#pragma unroll
  for (int o = -B; o <= B; ++o) {
    const R d = (R)dstencil_int<B>(o);
    dxv += d * row[wrap_pow2(i + o, nx)];
    dyv += d * x[(size_t)wrap_pow2(jj + o, nx) * nx + i];
  }
  return x[pt] - sx[pt] * dxv - sy[pt] * dyv;
}

// 1D (the paper's solve on 1D coarse levels, solve_mode 1): y = M x with M = I - diag(s) D, and
// y = M^T x = x - D diag(s) x (D is symmetric).
template <int B, typename R>
__device__ __forceinline__ R apply_M1d(const R* x, const R* sg, long long pt, int nx) {
  const int i = (int)pt;
  R dv = (R)0;
#pragma unroll
  for (int o = -B; o <= B; ++o) dv += (R)dstencil_int<B>(o) * x[wrap_pow2(i + o, nx)];
  return x[pt] - sg[pt] * dv;
}
template <int B, typename R>
__device__ __forceinline__ R apply_MT1d(const R* x, const R* sg, long long pt, int nx) {
  const int i = (int)pt;
  R dv = (R)0;
#pragma unroll
  for (int o = -B; o <= B; ++o) {
    const int q = wrap_pow2(i + o, nx);
    dv += (R)dstencil_int<B>(o) * sg[q] * x[q];
  }
  return x[pt] - dv;
}

// y = M^T x = x - (I (x) D) diag(sx) x - (D (x) I) diag(sy) x (D is symmetric).
template <int B, typename R>
__device__ __forceinline__ R apply_MT(const R* x, const R* sx, const R* sy, long long pt, int nx) {
  int i, jj;
  split_pow2(pt, nx, i, jj);
  R dxv = (R)0, dyv = (R)0;
#pragma unroll
  for (int o = -B; o <= B; ++o) {
    const R d = (R)dstencil_int<B>(o);
    const long long px = (long long)jj * nx + wrap_pow2(i + o, nx);
    const long long py = (long long)wrap_pow2(jj + o, nx) * nx + i;
    dxv += d * sx[px] * x[px];
    dyv += d * sy[py] * x[py];
  }
  return x[pt] - dxv - dyv;
}

// CTA-wide dot product; each thread accumulates its strided share in R and the warps reduce in R (FP32
// systems stay off the narrow FP64 pipe), the warp partials are summed in FP64.
template <typename R>
__device__ __forceinline__ double cta_dot(const R* a, const R* b, long long N, double* red) {
  R s = (R)0;
  for (long long q = threadIdx.x; q < N; q += blockDim.x) s += a[q] * b[q];
  double t = block_sum_r<R>(s, red);
  __syncthreads();
  if (threadIdx.x == 0) red[32] = t;
  __syncthreads();
  t = red[32];
  __syncthreads();
  return t;
}

// Arnoldi step with an unnormalised basis: the stored vectors are u_t with v_t = s_t u_t.  Pass A forms
// w = s_k M u_k row by row (M^T for TRANS; DIM = 1: the 1D operator with sigma sx), stores it, and
// accumulates the raw projections <u_t, w>, t = 0..k, in R per thread and warp, the warp partials summed
// in FP64 into hsum[0..k] (all threads see them).  Rows [lo, hi).
template <int B, typename R, bool TRANS, int DIM = 2>
__device__ __forceinline__ void cta_apply_project(const R* uk, const R* sx, const R* sy, int nx, const R* V, long long N,
                                                  R* w, int kk, long long lo, long long hi, R sk,
                                                  double (*wpart)[11], double* hsum) {
  R acc[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) acc[t] = (R)0;
  for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
    R mq;
    if constexpr (DIM == 1) mq = TRANS ? apply_MT1d<B, R>(uk, sx, q, nx) : apply_M1d<B, R>(uk, sx, q, nx);
    else mq = TRANS ? apply_MT<B, R>(uk, sx, sy, q, nx) : apply_M<B, R>(uk, sx, sy, q, nx);
    const R wq = sk * mq;
    w[q] = wq;
#pragma unroll
    for (int t = 0; t < 10; ++t)
      if (t <= kk) acc[t] += V[(size_t)t * N + q] * wq;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 10; ++t) {
    if (t > kk) break;
    R v = acc[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wpart[warp][t] = (double)v;
  }
  __syncthreads();
  if ((int)threadIdx.x <= kk) {
    double v = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) v += wpart[k][threadIdx.x];
    hsum[threadIdx.x] = v;
  }
  __syncthreads();
}

// Pass B: w -= sum_t c_t u_t over the rows [lo, hi) and the sum of squares of the result (this CTA's
// rows, valid in thread 0).
template <typename R>
__device__ __forceinline__ double cta_subtract_sumsq(const R* V, long long N, R* w, int kk, long long lo, long long hi,
                                                     const double* c, double* red) {
  R cr[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) cr[t] = t <= kk ? (R)c[t] : (R)0;
  R nn = (R)0;
  for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
    R v = w[q];
#pragma unroll
    for (int t = 0; t < 10; ++t)
      if (t <= kk) v -= cr[t] * V[(size_t)t * N + q];
    w[q] = v;
    nn += v * v;
  }
  return block_sum_r<R>(nn, red);
}

// One CTA per interval j: b (= rhs, in place -> solution) of the system of step n(j) = n0 + j*m
// (row nt_rev - 1 - n(j) when nt_rev > 0; TRANS solves with M^T).  basis: [J][kmax + 1][N] scratch
// ([J][kmax + 2][N] with restarts > 1).  DIM = 1: the 1D system I - diag(sigma_x) D of nx unknowns
// (sigma_y unused).  GMRES (Arnoldi with classical Gram-Schmidt: the projections on all basis vectors in
// one pass over w, then one update pass; Givens rotations), zero initial guess, stop when the
// least-squares residual <= rtol ||b|| or after kmax iterations.  restarts > 1 (the exact solves of
// solve_mode 2): up to that many GMRES(kmax) cycles, each from the residual b - M x of the solution
// accumulated so far (the extra scratch vector), until the true residual is <= rtol ||b||.
template <int B, typename R, bool TRANS, int DIM = 2>
__global__ void __launch_bounds__(gmres_threads<R>()) k_gmres2d(const R* __restrict__ sigma_x,
                                                        const R* __restrict__ sigma_y, int nx, int n0, int m,
                                                        int nt_rev, R* __restrict__ bx_all, R* __restrict__ basis,
                                                        int kmax, double rtol, int restarts = 1) {
  __shared__ double red[40];
  __shared__ double H[11][10];
  __shared__ double cs[10], sn[10], gv[11], yv[10];
  __shared__ double wpart[32][11];
  __shared__ double hsum[11];
  const long long N = DIM == 1 ? (long long)nx : (long long)nx * nx;
  const int j = blockIdx.x;
  const int n = nt_rev > 0 ? nt_rev - 1 - (n0 + j * m) : n0 + j * m;
  const R* sx = sigma_x + (size_t)n * N;
  const R* sy = sigma_y + (size_t)n * N;
  R* b = bx_all + (size_t)j * N;
  const int nvec = restarts > 1 ? kmax + 2 : kmax + 1;
  R* V = basis + (size_t)j * nvec * N;
  R* xacc = restarts > 1 ? V + (size_t)(kmax + 1) * N : nullptr;  // the accumulated solution
  const double beta0 = sqrt(cta_dot<R>(b, b, N, red));
  if (beta0 == 0.0) return;  // x = 0
  const double target = rtol * beta0;
  __shared__ double sc[11], cf[10];  // v_t = sc[t] u_t; projection coefficients of the update pass
  for (long long q = threadIdx.x; q < N; q += blockDim.x) {
    V[q] = b[q];  // u_0 = b, v_0 = b / beta
    if (xacc) xacc[q] = (R)0;
  }
  double beta = beta0;
  for (int cyc = 0; cyc < restarts; ++cyc) {
  if (cyc > 0) {  // restart from the true residual of the accumulated solution
    __syncthreads();
    R rr = (R)0;
    for (long long q = threadIdx.x; q < N; q += blockDim.x) {
      R mq;
      if constexpr (DIM == 1) mq = TRANS ? apply_MT1d<B, R>(xacc, sx, q, nx) : apply_M1d<B, R>(xacc, sx, q, nx);
      else mq = TRANS ? apply_MT<B, R>(xacc, sx, sy, q, nx) : apply_M<B, R>(xacc, sx, sy, q, nx);
      const R r = b[q] - mq;
      V[q] = r;
      rr += r * r;
    }
    const double t = block_sum_r<R>(rr, red);
    if (threadIdx.x == 0) red[34] = t;
    __syncthreads();
    beta = sqrt(red[34]);
    if (!(beta > target)) break;  // converged (or a non-finite residual: stop)
  }
  if (threadIdx.x == 0) {
    gv[0] = beta;
    for (int t = 1; t <= kmax; ++t) gv[t] = 0.0;
    sc[0] = 1.0 / beta;
  }
  __syncthreads();
  int kused = 0;
  for (int kk = 0; kk < kmax; ++kk) {
    R* uk = V + (size_t)kk * N;
    R* w = V + (size_t)(kk + 1) * N;
    // classical Gram-Schmidt in two passes: w = M v_k with the projections on all basis vectors, then
    // the update with the norm of the result
    cta_apply_project<B, R, TRANS, DIM>(uk, sx, sy, nx, V, N, w, kk, 0, N, (R)sc[kk], wpart, hsum);
    if ((int)threadIdx.x <= kk) {
      const double h = sc[threadIdx.x] * hsum[threadIdx.x];
      H[threadIdx.x][kk] = h;
      cf[threadIdx.x] = h * sc[threadIdx.x];
    }
    __syncthreads();
    double nn = cta_subtract_sumsq<R>(V, N, w, kk, 0, N, cf, red);
    if (threadIdx.x == 0) red[33] = nn;
    __syncthreads();
    const double hn = sqrt(red[33]);
    if (threadIdx.x == 0) {
      H[kk + 1][kk] = hn;
      for (int t = 0; t < kk; ++t) {  // previous rotations
        const double a = H[t][kk], c = H[t + 1][kk];
        H[t][kk] = cs[t] * a + sn[t] * c;
        H[t + 1][kk] = -sn[t] * a + cs[t] * c;
      }
      const double a = H[kk][kk], c = H[kk + 1][kk];
      const double r = sqrt(a * a + c * c);
      cs[kk] = r > 0.0 ? a / r : 1.0;
      sn[kk] = r > 0.0 ? c / r : 0.0;
      H[kk][kk] = r;
      H[kk + 1][kk] = 0.0;
      gv[kk + 1] = -sn[kk] * gv[kk];
      gv[kk] = cs[kk] * gv[kk];
      red[36] = fabs(gv[kk + 1]);
      sc[kk + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
    __syncthreads();
    kused = kk + 1;
    if (red[36] <= target || !(hn > 0.0)) break;
  }
  if (threadIdx.x == 0) {  // back substitution R y = g
    for (int t = kused - 1; t >= 0; --t) {
      double v = gv[t];
      for (int c = t + 1; c < kused; ++c) v -= H[t][c] * yv[c];
      yv[t] = v / H[t][t];
    }
  }
  __syncthreads();
  R yr[10];
  for (int t = 0; t < kused; ++t) yr[t] = (R)(yv[t] * sc[t]);
  for (long long q = threadIdx.x; q < N; q += blockDim.x) {
    R x = (R)0;
    for (int t = 0; t < kused; ++t) x += yr[t] * V[(size_t)t * N + q];
    if (xacc) xacc[q] += x;
    else b[q] = x;
  }
  if (!xacc) return;
  }
  __syncthreads();
  for (long long q = threadIdx.x; q < N; q += blockDim.x) b[q] = xacc[q];
}

// The same GMRES with one system spread over a thread-block cluster of C CTAs (C = gridDim / J): CTA
// rank r owns the rows [r N / C, (r + 1) N / C) of every vector.  Dot products are reduced across the
// cluster through distributed shared memory; every CTA adds the C partial sums in rank order, so all
// of them hold the same value and take the same Givens rotations and stopping decision.  A cluster
// barrier orders the writes of each new basis vector before M reads neighbouring rows of it.
template <int B, typename R, bool TRANS>
__global__ void __launch_bounds__(gmres_threads<R>()) k_gmres2d_cluster(const R* __restrict__ sigma_x,
                                                                   const R* __restrict__ sigma_y, int nx, int n0,
                                                                   int m, int nt_rev, R* __restrict__ bx_all,
                                                                   R* __restrict__ basis, int kmax, double rtol) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double red[40];
  __shared__ double part[2];
  __shared__ double mpart[2][11];
  __shared__ double H[11][10];
  __shared__ double cs[10], sn[10], gv[11], yv[10];
  __shared__ double wpart[32][11];
  __shared__ double hsum[11];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const long long N = (long long)nx * nx;
  const long long lo = N * rank / C, hi = N * (rank + 1) / C;
  const int j = blockIdx.x / C;
  const int n = nt_rev > 0 ? nt_rev - 1 - (n0 + j * m) : n0 + j * m;
  const R* sx = sigma_x + (size_t)n * N;
  const R* sy = sigma_y + (size_t)n * N;
  R* b = bx_all + (size_t)j * N;
  R* V = basis + (size_t)j * (kmax + 1) * N;
  int slot = 0;
  // cluster-wide dot product of rows [lo, hi)
  auto dot = [&](const R* x, const R* y) -> double {
    R sacc = (R)0;
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) sacc += x[q] * y[q];
    const double t = block_sum_r<R>(sacc, red);
    if (threadIdx.x == 0) part[slot] = t;
    cl.sync();
    double tot = 0.0;
    for (int r = 0; r < C; ++r) tot += *cl.map_shared_rank(&part[slot], (unsigned)r);
    slot ^= 1;
    return tot;
  };
  const double beta = sqrt(dot(b, b));
  if (beta == 0.0) {  // the same decision in every CTA; wait until no CTA reads this one's partials
    cl.sync();
    return;
  }
  __shared__ double sc[11], cf[10];  // v_t = sc[t] u_t; projection coefficients of the update pass
  for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) V[q] = b[q];  // u_0 = b, v_0 = b / beta
  if (threadIdx.x == 0) {
    gv[0] = beta;
    for (int t = 1; t <= kmax; ++t) gv[t] = 0.0;
    sc[0] = 1.0 / beta;
  }
  int kused = 0;
  for (int kk = 0; kk < kmax; ++kk) {
    R* uk = V + (size_t)kk * N;
    R* w = V + (size_t)(kk + 1) * N;
    cl.sync();  // u_k complete in every CTA before M reads its neighbouring rows
    // classical Gram-Schmidt in two passes: w = M v_k with this CTA's raw projections on all basis
    // vectors (one cluster reduction), then the update with the sum of squares (one cluster reduction)
    cta_apply_project<B, R, TRANS>(uk, sx, sy, nx, V, N, w, kk, lo, hi, (R)sc[kk], wpart, hsum);
    if ((int)threadIdx.x <= kk) mpart[slot][threadIdx.x] = hsum[threadIdx.x];
    cl.sync();
    if ((int)threadIdx.x <= kk) {
      double v = 0.0;
      for (int r = 0; r < C; ++r) v += cl.map_shared_rank(&mpart[slot][0], (unsigned)r)[threadIdx.x];
      const double h = sc[threadIdx.x] * v;
      H[threadIdx.x][kk] = h;
      cf[threadIdx.x] = h * sc[threadIdx.x];
    }
    slot ^= 1;
    __syncthreads();
    const double nn = cta_subtract_sumsq<R>(V, N, w, kk, lo, hi, cf, red);
    if (threadIdx.x == 0) part[slot] = nn;
    cl.sync();
    double tot = 0.0;
    for (int r = 0; r < C; ++r) tot += *cl.map_shared_rank(&part[slot], (unsigned)r);
    slot ^= 1;
    const double hn = sqrt(tot);
    if (threadIdx.x == 0) {
      H[kk + 1][kk] = hn;
      for (int t = 0; t < kk; ++t) {
        const double a = H[t][kk], c = H[t + 1][kk];
        H[t][kk] = cs[t] * a + sn[t] * c;
        H[t + 1][kk] = -sn[t] * a + cs[t] * c;
      }
      const double a = H[kk][kk], c = H[kk + 1][kk];
      const double r = sqrt(a * a + c * c);
      cs[kk] = r > 0.0 ? a / r : 1.0;
      sn[kk] = r > 0.0 ? c / r : 0.0;
      H[kk][kk] = r;
      H[kk + 1][kk] = 0.0;
      gv[kk + 1] = -sn[kk] * gv[kk];
      gv[kk] = cs[kk] * gv[kk];
      red[36] = fabs(gv[kk + 1]);
      sc[kk + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
    __syncthreads();
    kused = kk + 1;
    if (red[36] <= rtol * beta || !(hn > 0.0)) break;
  }
  if (threadIdx.x == 0) {
    for (int t = kused - 1; t >= 0; --t) {
      double v = gv[t];
      for (int c = t + 1; c < kused; ++c) v -= H[t][c] * yv[c];
      yv[t] = v / H[t][t];
    }
  }
  __syncthreads();
  R yr[10];
  for (int t = 0; t < kused; ++t) yr[t] = (R)(yv[t] * sc[t]);
  for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
    R x = (R)0;
    for (int t = 0; t < kused; ++t) x += yr[t] * V[(size_t)t * N + q];
    b[q] = x;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// J systems of step index n0 (+ j m): one CTA each, or, when J leaves SMs idle, a cluster of CTAs each
// (2D).  DIM = 1: the 1D systems, one CTA each (sig holds sigma only, [nt][nx]).
template <int B, typename R, bool TRANS, int DIM = 2>
cudaError_t launch_gmres(const R* sig, long long N, int nt, int nx, int n0, int m, int ntr, R* b, R* basis,
                         int kmax, double rtol, int J, cudaStream_t st, int restarts = 1) {
  if (DIM == 1 || restarts > 1) {  // one CTA per system (restarted solves keep their solution in scratch)
    k_gmres2d<B, R, TRANS, DIM><<<J, gmres_threads<R>(), 0, st>>>(sig, DIM == 1 ? sig : sig + (size_t)nt * N, nx, n0, m,
                                                                   ntr, b, basis, kmax, rtol, restarts);
    return cudaGetLastError();
  }
  int C = 1;
  while (C < 16 && J * C * 2 <= 152) C *= 2;
  if (C > 1) {
    auto kern = k_gmres2d_cluster<B, R, TRANS>;
    cudaError_t e = C > 8 ? cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)
                          : cudaSuccess;
    for (; C > 1 && e == cudaSuccess; C /= 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(J * C));
      cfg.blockDim = dim3(gmres_threads<R>());
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        continue;  // try a smaller cluster
      }
      return cudaLaunchKernelEx(&cfg, kern, sig, sig + (size_t)nt * N, nx, n0, m, ntr, b, basis, kmax, rtol);
    }
    cudaGetLastError();
  }
  k_gmres2d<B, R, TRANS><<<J, gmres_threads<R>(), 0, st>>>(sig, sig + (size_t)nt * N, nx, n0, m, ntr, b, basis,
                                                             kmax, rtol);
  return cudaGetLastError();
}

template <typename R>
__global__ void k_add_rows(R* __restrict__ dst, const R* __restrict__ g, int m, int k, int n0, long long N,
                           R* __restrict__ fstore) {
  const int j = blockIdx.y;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  const int n = m > 0 ? j * m + k : n0;
  R v = dst[(size_t)j * N + pt];
  if (g) v += g[(size_t)(n + 1) * N + pt];
  dst[(size_t)j * N + pt] = v;
  if (fstore) fstore[(size_t)(n + 1) * N + pt] = v;
}

// cur[j] = start[j] (+ corr[j]) for j = 0 .. count-1; optional write-back.
template <typename R>
__global__ void k_load_start(const R* __restrict__ start, long long sstride, const R* __restrict__ corr,
                             long long cstride, R* __restrict__ wb, long long wbstride, R* __restrict__ cur,
                             long long N, int J) {
  const int j = blockIdx.y;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  R v = start ? start[(size_t)j * sstride + pt] : (R)0;
  if (corr) v += corr[(size_t)j * cstride + pt];
  if (wb) wb[(size_t)j * wbstride + pt] = v;
  if (j < J) cur[(size_t)j * N + pt] = v;
}

// FC: cout[j+1] = cur[j] (+ g).  RES: rout[j+1] = cur[j] (+ gC) - cin[j+1]; per-interval sum of squares.
template <typename R>
__global__ void __launch_bounds__(kThreads2d) k_finish2d(const R* __restrict__ cur, RelaxArgs a, long long N,
                                                         double* __restrict__ partial, int chunks) {
  __shared__ double red[33];
  const int j = blockIdx.y;
  R sq = (R)0;  // FP32 levels: the per-thread and per-warp sums in FP32
  const int nC = (j + 1) * a.m;
  const R* gr = a.g ? (const R*)a.g + (size_t)nC * N : nullptr;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < N; pt += (long long)gridDim.x * blockDim.x) {
    R v = cur[(size_t)j * N + pt];
    if (a.mode == MODE_FC) {
      if (gr) v += gr[pt];
      ((R*)a.cout)[(size_t)(j + 1) * a.c_stride + pt] = v;
    } else {
      if (gr && a.g_at_c) v += gr[pt];
      const R ci = a.cin ? ((const R*)a.cin)[(size_t)(j + 1) * a.c_stride + pt] : (R)0;
      if (a.cin_corr) v -= ci + ((const R*)a.cin_corr)[(size_t)(j + 1) * a.corr_stride + pt];
      else if (a.cin) v -= ci;
      if (a.rout_f64) ((double*)a.rout)[(size_t)(j + 1) * a.r_stride + pt] = (double)v;
      else ((R*)a.rout)[(size_t)(j + 1) * a.r_stride + pt] = v;
      if (a.rout32) a.rout32[(size_t)(j + 1) * a.r_stride + pt] = (float)v;
      sq += v * v;
    }
  }
  if (a.mode == MODE_RES && partial) {
    const double t = block_sum_r<R>(sq, red);
    if (threadIdx.x == 0) partial[(size_t)j * chunks + blockIdx.x] = t;
  }
}

__global__ void k_sum_chunks(const double* __restrict__ partial, int chunks, int J, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += partial[(size_t)j * chunks + c];
  out[j] = s;
}

template <typename R>
cudaError_t step_all(const LevelTables& T, const Scratch2d& S, R* src, R* dst, int m, int k, int n0, int J,
                     const R* g, R* fstore, cudaStream_t st) {
  const long long N = T.npts;
  dim3 grid((unsigned)((N + kThreads2d - 1) / kThreads2d), (unsigned)J);
  const bool coarse = T.solver != nullptr;
  const int addg_in_step = coarse ? 0 : 1;
  const int n_first = m > 0 ? k : n0;
  if (T.npts == T.nx) {  // 1D coarse levels solved by GMRES (solve_mode 1)
    if (T.trans) return cudaErrorNotSupported;
#define MGRIT_STEP1D(PP) k_step1d_g<PP, R><<<grid, kThreads2d, 0, st>>>(T, src, dst, m, k, n0, g, addg_in_step, coarse ? nullptr : fstore)
    if (T.p == 1) MGRIT_STEP1D(1);
    else if (T.p == 3) MGRIT_STEP1D(3);
    else MGRIT_STEP1D(5);
#undef MGRIT_STEP1D
    if (coarse) {
      const R* sig = (const R*)T.solver;  // sigma [nt][nx]
      const int B = (T.p + 1) / 2;
      cudaError_t e;
      if (B == 1) e = launch_gmres<1, R, false, 1>(sig, N, T.nt, T.nx, n_first, m, 0, dst, (R*)S.basis, S.kmax, S.rtol, J, st, S.restarts);
      else if (B == 2) e = launch_gmres<2, R, false, 1>(sig, N, T.nt, T.nx, n_first, m, 0, dst, (R*)S.basis, S.kmax, S.rtol, J, st, S.restarts);
      else e = launch_gmres<3, R, false, 1>(sig, N, T.nt, T.nx, n_first, m, 0, dst, (R*)S.basis, S.kmax, S.rtol, J, st, S.restarts);
      if (e != cudaSuccess) return e;
      k_add_rows<R><<<grid, kThreads2d, 0, st>>>(dst, g, m, k, n0, N, fstore);
    }
    return cudaGetLastError();
  }
  if (T.trans) {  // Phi^T = S^T M^{-T}: the correction solve (in place on src), then the transposed step
    if constexpr (std::is_same<R, double>::value) {
      if (coarse) {
        const double* sig = (const double*)T.solver;  // FP64 (the adjoint is FP64)
        const int B = (T.p + 1) / 2, ntr = T.reverse ? T.nt : 0;
        cudaError_t e;
        if (B == 1)
          e = launch_gmres<1, double, true>(sig, N, T.nt, T.nx, n_first, m, ntr, src, (double*)S.basis, S.kmax, S.rtol,
                                            J, st, S.restarts);
        else if (B == 2)
          e = launch_gmres<2, double, true>(sig, N, T.nt, T.nx, n_first, m, ntr, src, (double*)S.basis, S.kmax, S.rtol,
                                            J, st, S.restarts);
        else
          e = launch_gmres<3, double, true>(sig, N, T.nt, T.nx, n_first, m, ntr, src, (double*)S.basis, S.kmax, S.rtol,
                                            J, st, S.restarts);
        if (e != cudaSuccess) return e;
      }
      if (T.p == 1) k_step2d_T<1><<<grid, kThreads2d, 0, st>>>(T, src, dst, m, k, n0, g, fstore);
      else if (T.p == 3) k_step2d_T<3><<<grid, kThreads2d, 0, st>>>(T, src, dst, m, k, n0, g, fstore);
      else k_step2d_T<5><<<grid, kThreads2d, 0, st>>>(T, src, dst, m, k, n0, g, fstore);
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }
#define MGRIT_STEP2D(PP) k_step2d<PP, R><<<grid, kThreads2d, 0, st>>>(T, src, dst, m, k, n0, g, addg_in_step, coarse ? nullptr : fstore)
  if (T.p == 1) MGRIT_STEP2D(1);
  else if (T.p == 3) MGRIT_STEP2D(3);
  else MGRIT_STEP2D(5);
#undef MGRIT_STEP2D
  if (coarse) {
    // sigma_x block then sigma_y block, [nt][N] each, in the level's precision
    const R* sig = (const R*)T.solver;
    const int B = (T.p + 1) / 2;
    cudaError_t e;
    if (B == 1) e = launch_gmres<1, R, false>(sig, N, T.nt, T.nx, n_first, m, 0, dst, (R*)S.basis, S.kmax, S.rtol, J, st, S.restarts);
    else if (B == 2) e = launch_gmres<2, R, false>(sig, N, T.nt, T.nx, n_first, m, 0, dst, (R*)S.basis, S.kmax, S.rtol, J, st, S.restarts);
    else e = launch_gmres<3, R, false>(sig, N, T.nt, T.nx, n_first, m, 0, dst, (R*)S.basis, S.kmax, S.rtol, J, st, S.restarts);
    if (e != cudaSuccess) return e;
    k_add_rows<R><<<grid, kThreads2d, 0, st>>>(dst, g, m, k, n0, N, fstore);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t relax2d(const LevelTables& T, const RelaxArgs& a, const Scratch2d& S, cudaStream_t st) {
  const long long N = T.npts;
  const int J = a.J;
  R* cur = (R*)S.cur;
  R* nxt = (R*)S.nxt;
  dim3 g1((unsigned)((N + kThreads2d - 1) / kThreads2d), (unsigned)(J + (a.extra_cta ? 1 : 0)));
  k_load_start<R><<<g1, kThreads2d, 0, st>>>((const R*)a.start, a.start_stride, (const R*)a.corr, a.corr_stride,
                                             (R*)a.start_wb, a.wb_stride, cur, N, J);
  for (int k = 0; k < a.nsteps; ++k) {
    const bool last = (k == a.m - 1);
    cudaError_t e = step_all<R>(T, S, cur, nxt, a.m, k, 0, J, last ? nullptr : (const R*)a.g,
                                last ? nullptr : (R*)a.fstore, st);
    if (e != cudaSuccess) return e;
    R* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (a.mode == MODE_FC || a.mode == MODE_RES) {
    const int chunks = 64;
    dim3 g2(chunks, (unsigned)J);
    k_finish2d<R><<<g2, kThreads2d, 0, st>>>(cur, a, N, S.partial, chunks);
    if (a.mode == MODE_RES && a.norm_partial)
      k_sum_chunks<<<(J + 255) / 256, 256, 0, st>>>(S.partial, chunks, J, a.norm_partial);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t sequential2d(const LevelTables& T, int Nst, const R* g, const R* u0, R* out, int store_all,
                         const Scratch2d& S, cudaStream_t st) {
  const long long N = T.npts;
  R* cur = (R*)S.cur;
  R* nxt = (R*)S.nxt;
  dim3 g1((unsigned)((N + kThreads2d - 1) / kThreads2d), 1u);
  k_load_start<R><<<g1, kThreads2d, 0, st>>>(u0, 0, nullptr, 0, store_all ? out : nullptr, 0, cur, N, 1);
  for (int n = 0; n < Nst; ++n) {
    R* fs = store_all ? out : nullptr;
    cudaError_t e = step_all<R>(T, S, cur, nxt, 0, 0, n, 1, g, fs, st);
    if (e != cudaSuccess) return e;
    R* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (!store_all) cudaMemcpyAsync(out, cur, (size_t)N * sizeof(R), cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}


// ---- 2D adjoint support -----------------------------------------------------------------------------

// Base node of the stencil of arrival point pt in step row n: ((i + shift_x) mod nx, (j + shift_y) mod nx).
__device__ __forceinline__ int base_key(const uint16_t* __restrict__ shift, int nt, int n, long long N, int nx,
                                        long long pt) {
  const int mask = nx - 1;
  int i, jj;
  split_pow2(pt, nx, i, jj);
  const int bx = (i + (int)shift[(size_t)n * N + pt]) & mask;
  const int by = (jj + (int)shift[((size_t)nt + n) * N + pt]) & mask;
  return by * nx + bx;
}

// counts[n][1 + key] += 1 (counts zeroed before).
__global__ void k_bucket_count(const uint16_t* __restrict__ shift, int nt, int nx, int* __restrict__ counts) {
  const long long N = (long long)nx * nx;
  const int n = blockIdx.y;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  atomicAdd(counts + (size_t)n * (N + 1) + 1 + base_key(shift, nt, n, N, nx, pt), 1);
}

// In-place inclusive scan of each row of length len (one CTA of 1024 threads per row).
__global__ void __launch_bounds__(1024) k_scan_rows(int* __restrict__ v, long long len) {
  __shared__ int part[1024];
  int* row = v + (size_t)blockIdx.x * len;
  const long long chunk = (len + blockDim.x - 1) / blockDim.x;
  const long long lo = threadIdx.x * chunk, hi = lo + chunk < len ? lo + chunk : len;
  int s = 0;
  for (long long q = lo; q < hi; ++q) s += row[q];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // Hillis-Steele inclusive scan of the chunk sums
    const int t = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  int run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
  for (long long q = lo; q < hi; ++q) {
    run += row[q];
    row[q] = run;
  }
}

// perm[n][cursor[n][key]++] = pt (cursor starts as a copy of bstart's first npts entries of the row).
__global__ void k_bucket_fill(const uint16_t* __restrict__ shift, int nt, int nx, int* __restrict__ cursor,
                              int* __restrict__ perm) {
  const long long N = (long long)nx * nx;
  const int n = blockIdx.y;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  const int slot = atomicAdd(cursor + (size_t)n * N + base_key(shift, nt, n, N, nx, pt), 1);
  perm[(size_t)n * N + slot] = (int)pt;
}

// Sorts every bucket (insertion sort; buckets hold a few points) so that the order is independent of
// the order of the atomic slot claims.
__global__ void k_bucket_sort(const int* __restrict__ bstart, int nx, int* __restrict__ perm) {
  const long long N = (long long)nx * nx;
  const int n = blockIdx.y;
  const long long key = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (key >= N) return;
  const int* bs = bstart + (size_t)n * (N + 1);
  int* pp = perm + (size_t)n * N;
  const int lo = bs[key], hi = bs[key + 1];
  for (int a = lo + 1; a < hi; ++a) {
    const int v = pp[a];
    int b = a - 1;
    while (b >= lo && pp[b] > v) {
      pp[b + 1] = pp[b];
      --b;
    }
    pp[b + 1] = v;
  }
}

__global__ void k_copy_starts(const int* __restrict__ bstart, long long N, int* __restrict__ cursor) {
  const int n = blockIdx.y;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < N) cursor[(size_t)n * N + q] = bstart[(size_t)n * (N + 1) + q];
}

// partial[j][chunk] += sum over the chunk's points of lambda_{n+1} (dPhi_n/da) u_n, n = j m + k, u_n = cur[j].
template <int P>
__global__ void __launch_bounds__(kThreads2d) k_grad2d(LevelTables T, const double* __restrict__ ds,
                                                       const double* __restrict__ cur, const double* __restrict__ mu,
                                                       int nt, int m, int k, double* __restrict__ partial,
                                                       int chunks) {
  __shared__ double red[33];
  const int j = blockIdx.y;
  const int n = j * m + k;
  const long long N = T.npts;
  const int nx = T.nx;
  const double* lam = mu + (size_t)(nt - n - 1) * N;
  const double* u = cur + (size_t)j * N;
  double acc = 0.0;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < N; pt += (long long)gridDim.x * blockDim.x) {
    const size_t ox = (size_t)n * N + pt, oy = ((size_t)T.nt + n) * N + pt;
    double ex = T.s64[ox], ey = T.s64[oy];
    ex -= floor(ex);
    if (ex >= 1.0) ex -= 1.0;
    ey -= floor(ey);
    if (ey >= 1.0) ey -= 1.0;
    double wx[P + 1], wy[P + 1], dwx[P + 1], dwy[P + 1];
    lagrange_weights<P, double>(ex, wx);
    lagrange_weights<P, double>(ey, wy);
    lagrange_weights_deps<P>(ex, dwx);
    lagrange_weights_deps<P>(ey, dwy);
    int i, jj;
    split_pow2(pt, nx, i, jj);
    const int bx = i + (int)T.shift[ox], by = jj + (int)T.shift[oy];
    const double dsx = ds[ox], dsy = ds[oy];
    double val = 0.0;
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const double* row = u + (size_t)wrap_pow2(by + b, nx) * nx;
      double rx = 0.0, rdx = 0.0;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const double v = row[wrap_pow2(bx + a, nx)];
        rx += wx[a] * v;
        rdx += dwx[a] * v;
      }
      val += wy[b] * dsx * rdx + dwy[b] * dsy * rx;
    }
    acc += lam[pt] * val;
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) partial[(size_t)j * chunks + blockIdx.x] += t;
}

}  // namespace

cudaError_t launch_relax_2d(const LevelTables& T, const RelaxArgs& a, const Scratch2d& S, int is_double,
                            cudaStream_t st) {
  return is_double ? relax2d<double>(T, a, S, st) : relax2d<float>(T, a, S, st);
}

cudaError_t launch_sequential_2d(const LevelTables& T, int N, const void* g, const void* u0, void* out, int store_all,
                                 const Scratch2d& S, int is_double, cudaStream_t st) {
  if (is_double)
    return sequential2d<double>(T, N, (const double*)g, (const double*)u0, (double*)out, store_all, S, st);
  return sequential2d<float>(T, N, (const float*)g, (const float*)u0, (float*)out, store_all, S, st);
}

cudaError_t launch_apply_steps_2d(const LevelTables& T, int n0, int count, const void* in, void* out,
                                  const Scratch2d& S, int is_double, cudaStream_t st) {
  for (int c = 0; c < count; ++c) {
    const long long N = T.npts;
    cudaError_t e;
    if (is_double)
      e = step_all<double>(T, S, (double*)in + (size_t)c * N, (double*)out + (size_t)c * N, 0, 0, n0 + c, 1,
                           nullptr, nullptr, st);
    else
      e = step_all<float>(T, S, (float*)in + (size_t)c * N, (float*)out + (size_t)c * N, 0, 0, n0 + c, 1, nullptr,
                          nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_bucket_build(const uint16_t* shift, int nt, int nx, int* bstart, int* bperm, cudaStream_t st) {
  const long long N = (long long)nx * nx;
  const int bs = 256;
  dim3 grid((unsigned)((N + bs - 1) / bs), (unsigned)nt);
  cudaError_t e = cudaMemsetAsync(bstart, 0, (size_t)nt * (N + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_bucket_count<<<grid, bs, 0, st>>>(shift, nt, nx, bstart);
  k_scan_rows<<<nt, 1024, 0, st>>>(bstart, N + 1);
  int* cursor = nullptr;
  e = cudaMallocAsync((void**)&cursor, (size_t)nt * N * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_copy_starts<<<grid, bs, 0, st>>>(bstart, N, cursor);
  k_bucket_fill<<<grid, bs, 0, st>>>(shift, nt, nx, cursor, bperm);
  k_bucket_sort<<<grid, bs, 0, st>>>(bstart, nx, bperm);
  cudaFreeAsync(cursor, st);
  return cudaGetLastError();
}

cudaError_t launch_gradient_a_2d(const LevelTables& T, const double* ds, const double* C, const double* mu, int nt,
                                 int m, int J, const Scratch2d& S, double* out, cudaStream_t st) {
  const long long N = T.npts;
  const int chunks = 64;
  double* cur = (double*)S.cur;
  double* nxt = (double*)S.nxt;
  dim3 g1((unsigned)((N + kThreads2d - 1) / kThreads2d), (unsigned)J);
  k_load_start<double><<<g1, kThreads2d, 0, st>>>(C, N, nullptr, 0, nullptr, 0, cur, N, J);
  cudaError_t e = cudaMemsetAsync(S.partial, 0, (size_t)J * chunks * sizeof(double), st);
  if (e != cudaSuccess) return e;
  LevelTables F = T;  // forward fine steps
  F.solver = nullptr;
  F.trans = 0;
  F.reverse = 0;
  dim3 g2(chunks, (unsigned)J);
  for (int k = 0; k < m; ++k) {
    if (T.p == 1) k_grad2d<1><<<g2, kThreads2d, 0, st>>>(T, ds, cur, mu, nt, m, k, S.partial, chunks);
    else if (T.p == 3) k_grad2d<3><<<g2, kThreads2d, 0, st>>>(T, ds, cur, mu, nt, m, k, S.partial, chunks);
    else k_grad2d<5><<<g2, kThreads2d, 0, st>>>(T, ds, cur, mu, nt, m, k, S.partial, chunks);
    if (k + 1 < m) {
      e = step_all<double>(F, S, cur, nxt, m, k, 0, J, nullptr, nullptr, st);
      if (e != cudaSuccess) return e;
      double* t = cur;
      cur = nxt;
      nxt = t;
    }
  }
  k_sum_chunks<<<(J + 255) / 256, 256, 0, st>>>(S.partial, chunks, J, out);
  return cudaGetLastError();
}

}  // namespace mgrit
