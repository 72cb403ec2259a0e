// Relaxation kernels of the MGRIT cycle for 1D problems (Sec. 2.2).
//
// One CTA owns one coarse interval j and keeps the current time slice in shared memory across the
// m steps of the interval, so HBM sees only the per-step gather tables, the interval's start slice
// and the interval's output.  A step is either the fine SL step Phi (Sec. 2.1: gather with Lagrange
// weights of degree P) or the coarse operator Psi = [I - diag(sigma) D_{P+1}]^{-1} S (eq.
// (Phi_multilevel)): the same gather followed by a partitioned periodic banded solve in shared memory.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mgrit {

namespace {

template <typename R>
struct SolverViewC {
  const R* lu;
  const R* vw;
  const R* sinv;
  const R* ctail;
  const R* chead;
};

template <typename R>
__device__ __forceinline__ SolverViewC<R> solver_view_c(const R* base, int nx, int b, int P) {
  const int s = nx / P, q = s - b;
  SolverViewC<R> v;
  v.lu = base;
  v.vw = v.lu + (size_t)(2 * b + 1) * q * P;
  v.sinv = v.vw + (size_t)2 * b * nx;
  v.ctail = v.sinv + (size_t)(b * P) * (b * P);
  v.chead = v.ctail + (size_t)P * b * b;
  return v;
}

// dst[i] = sum_a w_a(eps_i) src[(i + shift_i + a) mod nx]  -- the SL gather of step row n.
template <int P, typename R>
__device__ __forceinline__ void gather_step(const R* __restrict__ src, R* __restrict__ dst, const LevelTables& T,
                                            int n) {
  const int nx = T.nx;
  const uint16_t* __restrict__ sh = T.shift + (size_t)n * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const int base = i + (int)__ldg(sh + i);
    R w[P + 1];
    if constexpr (std::is_same<R, double>::value) {
      const double* __restrict__ wr = T.w64 + (size_t)n * (P + 1) * nx + i;
#pragma unroll
      for (int a = 0; a <= P; ++a) w[a] = __ldg(wr + (size_t)a * nx);
    } else {
      lagrange_weights<P, float>(__ldg(T.eps32 + (size_t)n * nx + i), w);
    }
    R acc = w[0] * src[wrap_pow2(base, nx)];
#pragma unroll
    for (int a = 1; a <= P; ++a) acc += w[a] * src[wrap_pow2(base + a, nx)];
    dst[i] = acc;
  }
}

// x <- M^{-1} x for M = I - diag(sigma) D_{2B} of one step (data: factorisation, see setup_kernels.cu).
// scr: shared scratch of at least q (P + 1) + 2 B P reals (may alias the consumed gather source).
template <int B, typename R>
__device__ __forceinline__ void corr_solve(R* __restrict__ x, R* __restrict__ scr, const R* __restrict__ data, int nx,
                                           int P) {
  const int s = nx / P, q = s - B, nb = B * P, ld = P + 1;
  const SolverViewC<R> V = solver_view_c<R>(data, nx, B, P);
  R* yt = scr;           // interior values, transposed [r][k] with leading dimension P + 1
  R* gS = scr + q * ld;  // separator right-hand sides
  R* xS = gS + nb;       // separator solution
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const int k = i / s, r = i - k * s - B;
    if (r >= 0) yt[r * ld + k] = x[i];
  }
  __syncthreads();
  if ((int)threadIdx.x < P) {  // banded forward / backward substitution of each interior block
    const int k = threadIdx.x;
    R y[B];
#pragma unroll
    for (int t = 0; t < B; ++t) y[t] = (R)0;  // y[t] = value of row r-1-t
    for (int r = 0; r < q; ++r) {
      R v = yt[r * ld + k];
#pragma unroll
      for (int t = 1; t <= B; ++t)
        if (r - t >= 0) v -= V.lu[((size_t)(t - 1) * q + r) * P + k] * y[t - 1];
      yt[r * ld + k] = v;
#pragma unroll
      for (int t = B - 1; t >= 1; --t) y[t] = y[t - 1];
      y[0] = v;
    }
#pragma unroll
    for (int t = 0; t < B; ++t) y[t] = (R)0;  // y[t] = value of row r+1+t
    for (int r = q - 1; r >= 0; --r) {
      R v = yt[r * ld + k];
#pragma unroll
      for (int t = 1; t <= B; ++t)
        if (r + t < q) v -= V.lu[((size_t)(B + t) * q + r) * P + k] * y[t - 1];
      v *= V.lu[((size_t)B * q + r) * P + k];
      yt[r * ld + k] = v;
#pragma unroll
      for (int t = B - 1; t >= 1; --t) y[t] = y[t - 1];
      y[0] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb; e += blockDim.x) {  // separator right-hand sides
    const int k = e / B, a = e - k * B, km = (k + P - 1) % P;
    R v = x[k * s + a];
#pragma unroll
    for (int c = 0; c < B; ++c) {
      v -= V.ctail[(k * B + a) * B + c] * yt[(q - B + c) * ld + km];
      v -= V.chead[(k * B + a) * B + c] * yt[c * ld + k];
    }
    gS[e] = v;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {  // separators: inverse of the Schur complement
    R acc = (R)0;
    for (int c = 0; c < nb; ++c) acc += V.sinv[(size_t)c * nb + r] * gS[c];
    xS[r] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {  // back-substitute the spikes
    const int k = i / s, r = i - k * s - B;
    if (r < 0) {
      x[i] = xS[k * B + r + B];
    } else {
      const int kp = (k + 1 == P) ? 0 : k + 1;
      R v = yt[r * ld + k];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        v -= V.vw[(size_t)c * nx + i] * xS[k * B + c];
        v -= V.vw[(size_t)(B + c) * nx + i] * xS[kp * B + c];
      }
      x[i] = v;
    }
  }
  __syncthreads();
}

template <int P, typename R, bool COARSE>
__device__ __forceinline__ void full_step(R*& src, R*& dst, const LevelTables& T, int n) {
  gather_step<P, R>(src, dst, T, n);
  __syncthreads();
  if constexpr (COARSE) {
    constexpr int B = (P + 1) / 2;
    corr_solve<B, R>(dst, src, (const R*)T.solver + (size_t)n * T.solver_stride, T.nx, T.P);
  }
}

template <int P, typename R, bool COARSE>
__global__ void __launch_bounds__(kSliceThreads) k_relax_1d(LevelTables T, RelaxArgs a, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* src = reinterpret_cast<R*>(smem_raw);
  R* dst = src + buf;
  double* red = reinterpret_cast<double*>(dst + buf);
  const int nx = T.nx;
  const int j = blockIdx.x;
  {
    const R* st = a.start ? (const R*)a.start + (size_t)j * a.start_stride : nullptr;
    const R* co = a.corr ? (const R*)a.corr + (size_t)j * a.corr_stride : nullptr;
    R* wb = a.start_wb ? (R*)a.start_wb + (size_t)j * a.wb_stride : nullptr;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      R v = st ? st[i] : (R)0;
      if (co) v += co[i];
      src[i] = v;
      if (wb) wb[i] = v;
    }
  }
  __syncthreads();
  if (j >= a.J) return;  // extra CTA: only the correction of the last C-point
  double sq = 0.0;
  for (int k = 0; k < a.nsteps; ++k) {
    const int n = j * a.m + k;
    full_step<P, R, COARSE>(src, dst, T, n);
    const R* gr = a.g ? (const R*)a.g + (size_t)(n + 1) * nx : nullptr;
    const bool last = (k == a.m - 1);
    if (!last) {
      R* fs = a.fstore ? (R*)a.fstore + (size_t)(n + 1) * nx : nullptr;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        R v = dst[i];
        if (gr) v += gr[i];
        dst[i] = v;
        if (fs) fs[i] = v;
      }
    } else if (a.mode == MODE_FC) {
      R* co = (R*)a.cout + (size_t)(j + 1) * a.c_stride;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        R v = dst[i];
        if (gr) v += gr[i];
        co[i] = v;
      }
    } else {  // MODE_RES
      const R* ci = a.cin ? (const R*)a.cin + (size_t)(j + 1) * a.c_stride : nullptr;
      R* ro = (R*)a.rout + (size_t)(j + 1) * a.r_stride;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        R v = dst[i];
        if (gr && a.g_at_c) v += gr[i];
        if (ci) v -= ci[i];
        ro[i] = v;
        sq += (double)v * (double)v;
      }
    }
    __syncthreads();
    R* t = src;
    src = dst;
    dst = t;
  }
  if (a.mode == MODE_RES && a.norm_partial) {
    const double tot = block_sum(sq, red);
    if (threadIdx.x == 0) a.norm_partial[j] = tot;
  }
}

// u0: [nx] start slice; out: store_all ? [(N+1)][nx] (row 0 = u0) : [nx] (the final slice).
template <int P, typename R, bool COARSE>
__global__ void __launch_bounds__(kSliceThreads) k_sequential_1d(LevelTables T, int N, const R* g, const R* u0,
                                                                 R* out_all, int store_all, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* src = reinterpret_cast<R*>(smem_raw);
  R* dst = src + buf;
  const int nx = T.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const R v = u0 ? u0[i] : (R)0;
    src[i] = v;
    if (store_all) out_all[i] = v;
  }
  __syncthreads();
  for (int n = 0; n < N; ++n) {
    full_step<P, R, COARSE>(src, dst, T, n);
    const R* gr = g ? g + (size_t)(n + 1) * nx : nullptr;
    R* out = store_all ? out_all + (size_t)(n + 1) * nx : (n == N - 1 ? out_all : nullptr);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      R v = dst[i];
      if (gr) v += gr[i];
      dst[i] = v;
      if (out) out[i] = v;
    }
    __syncthreads();
    R* t = src;
    src = dst;
    dst = t;
  }
}

template <int P, typename R, bool COARSE>
__global__ void __launch_bounds__(kSliceThreads) k_apply_1d(LevelTables T, int n0, const R* in, R* out, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* src = reinterpret_cast<R*>(smem_raw);
  R* dst = src + buf;
  const int nx = T.nx, c = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) src[i] = in[(size_t)c * nx + i];
  __syncthreads();
  full_step<P, R, COARSE>(src, dst, T, n0 + c);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) out[(size_t)c * nx + i] = dst[i];
}

int buffer_elems(const LevelTables& T, bool coarse) {
  int e = T.nx;
  if (coarse) {
    const int b = (T.p + 1) / 2;
    const int s = T.nx / T.P, q = s - b;
    const int need = q * (T.P + 1) + 2 * b * T.P;
    if (need > e) e = need;
  }
  return (e + 31) & ~31;
}

template <typename R>
size_t smem_bytes(int buf) {
  return 2 * (size_t)buf * sizeof(R) + 64 * sizeof(double);
}

template <typename R, bool COARSE>
cudaError_t relax_dispatch(const LevelTables& T, const RelaxArgs& a, cudaStream_t st) {
  const int buf = buffer_elems(T, COARSE);
  const size_t sm = smem_bytes<R>(buf);
  const int grid = a.J + (a.extra_cta ? 1 : 0);
  if (grid <= 0) return cudaSuccess;
#define MGRIT_LAUNCH_RELAX(PP)                                                                             \
  {                                                                                                        \
    auto kern = k_relax_1d<PP, R, COARSE>;                                                                 \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
    if (e != cudaSuccess) return e;                                                                        \
    kern<<<grid, kSliceThreads, sm, st>>>(T, a, buf);                                                      \
    return cudaGetLastError();                                                                             \
  }
  if (T.p == 1) MGRIT_LAUNCH_RELAX(1)
  if (T.p == 3) MGRIT_LAUNCH_RELAX(3)
  MGRIT_LAUNCH_RELAX(5)
#undef MGRIT_LAUNCH_RELAX
}

template <typename R, bool COARSE>
cudaError_t sequential_dispatch(const LevelTables& T, int N, const void* g, const void* u0, void* u, int store_all,
                                cudaStream_t st) {
  const int buf = buffer_elems(T, COARSE);
  const size_t sm = smem_bytes<R>(buf);
#define MGRIT_LAUNCH_SEQ(PP)                                                                               \
  {                                                                                                        \
    auto kern = k_sequential_1d<PP, R, COARSE>;                                                            \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
    if (e != cudaSuccess) return e;                                                                        \
    kern<<<1, kSliceThreads, sm, st>>>(T, N, (const R*)g, (const R*)u0, (R*)u, store_all, buf);            \
    return cudaGetLastError();                                                                             \
  }
  if (T.p == 1) MGRIT_LAUNCH_SEQ(1)
  if (T.p == 3) MGRIT_LAUNCH_SEQ(3)
  MGRIT_LAUNCH_SEQ(5)
#undef MGRIT_LAUNCH_SEQ
}

template <typename R, bool COARSE>
cudaError_t apply_dispatch(const LevelTables& T, int n0, int count, const void* in, void* out, cudaStream_t st) {
  const int buf = buffer_elems(T, COARSE);
  const size_t sm = smem_bytes<R>(buf);
#define MGRIT_LAUNCH_APPLY(PP)                                                                             \
  {                                                                                                        \
    auto kern = k_apply_1d<PP, R, COARSE>;                                                                 \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
    if (e != cudaSuccess) return e;                                                                        \
    kern<<<count, kSliceThreads, sm, st>>>(T, n0, (const R*)in, (R*)out, buf);                             \
    return cudaGetLastError();                                                                             \
  }
  if (T.p == 1) MGRIT_LAUNCH_APPLY(1)
  if (T.p == 3) MGRIT_LAUNCH_APPLY(3)
  MGRIT_LAUNCH_APPLY(5)
#undef MGRIT_LAUNCH_APPLY
}

__global__ void k_sum(const double* __restrict__ v, int count, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += v[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) out[0] = t;
}

__global__ void k_axpy_convert(int kind, const void* __restrict__ x, void* __restrict__ y, const void* __restrict__ z,
                               long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  switch (kind) {
    case 0: ((double*)y)[i] = ((const double*)x)[i]; break;
    case 1: ((float*)y)[i] = (float)((const double*)x)[i]; break;
    case 2: ((double*)y)[i] += (double)((const float*)x)[i]; break;
    case 3: ((double*)y)[i] = (double)((const float*)x)[i]; break;
    case 4: ((double*)y)[i] += ((const double*)x)[i]; break;
    default: ((double*)y)[i] += ((const double*)x)[i] + (double)((const float*)z)[i]; break;
  }
}

}  // namespace

cudaError_t launch_relax_1d(const LevelTables& T, const RelaxArgs& a, int is_double, cudaStream_t st) {
  const bool coarse = T.solver != nullptr;
  if (is_double) return coarse ? relax_dispatch<double, true>(T, a, st) : relax_dispatch<double, false>(T, a, st);
  return coarse ? relax_dispatch<float, true>(T, a, st) : relax_dispatch<float, false>(T, a, st);
}

cudaError_t launch_sequential_1d(const LevelTables& T, int N, const void* g, const void* u0, void* u, int store_all,
                                 int is_double, cudaStream_t st) {
  const bool coarse = T.solver != nullptr;
  if (is_double)
    return coarse ? sequential_dispatch<double, true>(T, N, g, u0, u, store_all, st)
                  : sequential_dispatch<double, false>(T, N, g, u0, u, store_all, st);
  return coarse ? sequential_dispatch<float, true>(T, N, g, u0, u, store_all, st)
                : sequential_dispatch<float, false>(T, N, g, u0, u, store_all, st);
}

cudaError_t launch_apply_steps_1d(const LevelTables& T, int n0, int count, const void* in, void* out, int is_double,
                                  cudaStream_t st) {
  const bool coarse = T.solver != nullptr;
  if (count <= 0) return cudaSuccess;
  if (is_double)
    return coarse ? apply_dispatch<double, true>(T, n0, count, in, out, st)
                  : apply_dispatch<double, false>(T, n0, count, in, out, st);
  return coarse ? apply_dispatch<float, true>(T, n0, count, in, out, st)
                : apply_dispatch<float, false>(T, n0, count, in, out, st);
}

void launch_sum(const double* v, int count, double* out, cudaStream_t st) { k_sum<<<1, 1024, 0, st>>>(v, count, out); }

void launch_axpy_convert(int kind, const void* x, void* y, const void* z, long long n, cudaStream_t st) {
  if (n <= 0) return;
  const int bs = 256;
  k_axpy_convert<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(kind, x, y, z, n);
}

void launch_fill_zero(void* y, long long bytes, cudaStream_t st) { cudaMemsetAsync(y, 0, (size_t)bytes, st); }

}  // namespace mgrit
