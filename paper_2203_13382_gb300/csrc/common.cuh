// Shared device/host helpers for the MGRIT semi-Lagrangian kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#define MGRIT_HD __host__ __device__ __forceinline__
#define MGRIT_D __device__ __forceinline__

namespace mgrit {

constexpr int kMaxOrder = 5;  // odd interpolation degree p <= 5
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.1415926535897932384626433832795;

// Number of threads for the slice-resident kernels.
constexpr int kSliceThreads = 512;

MGRIT_HD int wrap_pow2(int idx, int nx) { return idx & (nx - 1); }

// Column i and row j of element pt of an nx x nx slice, nx a power of two (shifts, not a 64-bit divide).
MGRIT_D void split_pow2(long long pt, int nx, int& i, int& j) {
  i = (int)(pt & (nx - 1));
  j = (int)(pt >> (__ffs(nx) - 1));
}

// Coefficient 1 / prod_{q != j} (j - q) of the Lagrange basis polynomial of node j = a - (P+1)/2,
// a = 0..P, on the unit-spaced nodes -(P+1)/2 .. (P-1)/2: equals (-1)^{P-a} / (a! (P-a)!).
template <int P>
MGRIT_HD double lagrange_denominator_inv(int a) {
  double f = 1.0;
  for (int b = 2; b <= a; ++b) f *= b;
  double g = 1.0;
  for (int b = 2; b <= P - a; ++b) g *= b;
  return (((P - a) & 1) ? -1.0 : 1.0) / (f * g);
}

// Monomial coefficients of the Lagrange basis polynomials of lagrange_weights: c[a][d] is the
// coefficient of eps^d in w_a(eps) = prod_{b != a} (-eps - j_b) / prod_{b != a} (j_a - j_b), j_b = b - L.
// Formed at compile time in FP64 (the products have integer coefficients; one rounding by the
// denominator).
template <int P>
struct LagrangeCoef {
  double c[P + 1][P + 1];
  constexpr LagrangeCoef() : c{} {
    constexpr int L = (P + 1) / 2;
    for (int a = 0; a <= P; ++a) {
      double poly[P + 1] = {};
      poly[0] = 1.0;
      int deg = 0;
      for (int b = 0; b <= P; ++b) {
        if (b == a) continue;
        const double q = -(double)(b - L);  // factor (q - eps)
        for (int d = deg + 1; d >= 1; --d) poly[d] = q * poly[d] - poly[d - 1];
        poly[0] = q * poly[0];
        ++deg;
      }
      double den = 1.0;  // prod_{b != a} (a - b) = (-1)^{P-a} a! (P-a)!
      for (int b = 0; b <= P; ++b)
        if (b != a) den *= (double)(a - b);
      for (int d = 0; d <= P; ++d) c[a][d] = poly[d] / den;
    }
  }
};

// Lagrange weights w_a(eps), a = 0..P, for interpolation at the point -eps relative to the east
// node, with nodes j = a - (P+1)/2 (Sec. 2.1), each by Horner's rule on its monomial coefficients
// (P multiply-adds a weight).
template <int P, typename R>
MGRIT_D void lagrange_weights(R eps, R (&w)[P + 1]) {
  constexpr LagrangeCoef<P> k{};
#pragma unroll
  for (int a = 0; a <= P; ++a) {
    R v = (R)k.c[a][P];
#pragma unroll
    for (int d = P - 1; d >= 0; --d) v = v * eps + (R)k.c[a][d];
    w[a] = v;
  }
}

// d w_a / d eps of lagrange_weights (product rule over the factors (-eps - j)).
template <int P>
MGRIT_D void lagrange_weights_deps(double eps, double (&dw)[P + 1]) {
  constexpr int L = (P + 1) / 2;
  double f[P + 1];
#pragma unroll
  for (int a = 0; a <= P; ++a) f[a] = -eps - (double)(a - L);
#pragma unroll
  for (int a = 0; a <= P; ++a) {
    double tot = 0.0;
#pragma unroll
    for (int skip = 0; skip <= P; ++skip) {
      if (skip == a) continue;
      double term = 1.0;
#pragma unroll
      for (int q = 0; q <= P; ++q)
        if (q != a && q != skip) term *= f[q];
      tot += term;
    }
    dw[a] = -tot * lagrange_denominator_inv<P>(a);
  }
}

// The single weight w_a(eps) of lagrange_weights (one factor of a 2D tensor-product weight).
template <int P>
MGRIT_D double lagrange_basis(double eps, int a) {
  constexpr int L = (P + 1) / 2;
  double w = lagrange_denominator_inv<P>(a);
#pragma unroll
  for (int c = 0; c <= P; ++c)
    if (c != a) w *= -eps - (double)(c - L);
  return w;
}

// Deterministic block sum of one double per thread (all threads must call).
MGRIT_D double block_sum(double v, double* smem_scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) smem_scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) t += smem_scratch[k];
  }
  return t;  // valid in thread 0
}

// Deterministic block sum of one R per thread: the warp sums in R (FP32 values stay off the FP64 pipe,
// which GB300 runs at 2 operations a clock per SM), the warp partials in FP64 (result in thread 0).
template <typename R>
MGRIT_D double block_sum_r(R v, double* smem_scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) smem_scratch[warp] = (double)v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) t += smem_scratch[k];
  }
  return t;  // valid in thread 0
}

// ---- TMA bulk copies into shared memory, completed on an mbarrier (sm_90+ PTX) ---------------------

MGRIT_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

MGRIT_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive on the barrier and announce `bytes` of transaction (the bulk copy that completes it).
MGRIT_D void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
MGRIT_D void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Programmatic dependent launch (sm_90+).  A kernel launched with programmatic stream serialization may
// start while the kernel before it on the stream is still running: it does its independent prologue
// (barrier set-up, bulk copies of set-up tables) and then waits in pdl_wait until that kernel has finished
// and its writes are visible; nothing that kernel writes, or reads, is touched before the wait.
// pdl_trigger lets the next kernel start once every CTA of this one has called it.  Both are no-ops for a
// kernel launched without the attribute.
MGRIT_D void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
MGRIT_D void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asks for [src, src + bytes) to be brought into L2 (a hint: nothing to wait for, no shared memory).
// Issued only for 16-byte aligned addresses and sizes that are a multiple of 16.
MGRIT_D void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  if (((reinterpret_cast<uintptr_t>(src) | bytes) & 15u) == 0 && bytes > 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy ones.
MGRIT_D void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

MGRIT_D bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the barrier phase with the given parity, giving up after about `limit_cycles` SM cycles.
MGRIT_D bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_cycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit_cycles) return false;
  return true;
}

constexpr long long kWaitLimitCycles = 2000000000LL;  // about one second at 2 GHz

}  // namespace mgrit
