// Relaxation kernels of the MGRIT cycle for 1D problems (Sec. 2.2).
//
// One CTA owns one coarse interval j and keeps the current time slice in shared memory across the
// m steps of the interval, so HBM sees only the per-step gather tables, the interval's start slice
// and the interval's output.  A step is either the fine SL step Phi (Sec. 2.1: gather with Lagrange
// weights of degree P) or the coarse operator Psi = [I - diag(sigma) D_{P+1}]^{-1} S (eq.
// (Phi_multilevel)): the same gather followed by a partitioned periodic banded solve in shared memory.
#include <type_traits>

#include "common.cuh"
#include "df32.cuh"
#include "kernels.h"
#include "solver_layout.cuh"

namespace mgrit {

namespace {

// ---- gather tables of one step, loaded into registers ahead of use (software pipelining) ----------
constexpr int kPts = 8;  // points per thread: nx <= kPts * threads (4096 for 512-thread CTAs)

// Threads of the slice-resident kernels (one CTA per interval).  Measured on the 4096-point coarse
// levels: 512 threads at one CTA per SM beat 256 threads at two (longer per-thread gathers and
// register spills of the on-the-fly solve outweigh the second CTA).
template <int P, typename R, int COARSE>
constexpr int slice_threads() {
  return kSliceThreads;
}

template <int P, typename R>
struct GatherRegs;

template <int P>
struct GatherRegs<P, double> {  // FP64 streams its table loads inside the gather (register pressure)
  int n;
};

template <int P>
struct GatherRegs<P, float> {};  // FP32 reads its tables from shared memory (staged by TMA)

template <int P, typename R>
__device__ __forceinline__ void load_gather(GatherRegs<P, R>& g, const LevelTables& T, int n) {
  if constexpr (std::is_same<R, double>::value) g.n = n;
  (void)T;
}

// dst[i] = sum_a w_a(eps_i) src[(i + shift_i + a) mod nx]  -- the SL gather (Sec. 2.1), FP64 weights
// from the w64 table.
template <int P>
__device__ __forceinline__ void apply_gather(const GatherRegs<P, double>& g, const LevelTables& T,
                                             const double* __restrict__ src, double* __restrict__ dst) {
  const int nx = T.nx;
#pragma unroll 2
  for (int q = 0; q < kPts; ++q) {
    const int i = threadIdx.x + q * kSliceThreads;
    if (i < nx) {
      double w[P + 1];
      const double* __restrict__ wr = T.w64 + (size_t)g.n * (P + 1) * nx + i;
#pragma unroll
      for (int a = 0; a <= P; ++a) w[a] = __ldg(wr + (size_t)a * nx);
      const int b = i + (int)__ldg(T.shift + (size_t)g.n * nx + i);
      double acc = w[0] * src[wrap_pow2(b, nx)];
#pragma unroll
      for (int a = 1; a <= P; ++a) acc += w[a] * src[wrap_pow2(b + a, nx)];
      dst[i] = acc;
    }
  }
}

// The same gather in FP32 with the step's eps / shift rows in shared memory; the weights are formed
// from eps in registers.  src carries the periodic halo src[nx + t] = src[t], t < kMaxOrder, so a
// stencil is P + 1 consecutive elements from its wrapped first node.
template <int P, int NT>
__device__ __forceinline__ void apply_gather_staged(const float* __restrict__ eps, const uint16_t* __restrict__ sh,
                                                    const float* __restrict__ src, float* __restrict__ dst, int nx) {
#pragma unroll 2
  for (int q = 0; q < kPts; ++q) {
    const int i = threadIdx.x + q * NT;
    if (i < nx) {
      float w[P + 1];
      lagrange_weights<P, float>(eps[i], w);
      const float* s = src + wrap_pow2(i + (int)sh[i], nx);
      float acc = w[0] * s[0];
#pragma unroll
      for (int a = 1; a <= P; ++a) acc += w[a] * s[a];
      dst[i] = acc;
    }
  }
}

// Thread t < kMaxOrder: the periodic halo of slice s (its element t already final and visible to t).
template <typename R>
__device__ __forceinline__ void write_halo(R* s, int nx) {
  if (threadIdx.x < kMaxOrder) s[nx + threadIdx.x] = s[threadIdx.x];
}

// ---- correction solve x <- M^{-1} x, M = I - diag(sigma) D_{2B} (layout: solver_layout.cuh) ----------

// The 8 values of one partition (8-aligned) in shared memory, moved as vectors (fewer bank conflicts).
template <typename R>
__device__ __forceinline__ void load_part(const R* p, R (&v)[kPartRows]) {
  if constexpr (std::is_same<R, float>::value) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double2 a = reinterpret_cast<const double2*>(p)[c];
      v[2 * c] = a.x;
      v[2 * c + 1] = a.y;
    }
  }
}
template <typename R>
__device__ __forceinline__ void store_part(R* p, const R (&v)[kPartRows]) {
  if constexpr (std::is_same<R, float>::value) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) reinterpret_cast<double2*>(p)[c] = make_double2(v[2 * c], v[2 * c + 1]);
  }
}

// xch: shared scratch of 4 * P * B reals (may alias the consumed gather source).
// pcr_src: the coefficient block [pcr_off, total) of this step, either in global memory (data +
// pcr_off) or staged in shared memory.
template <int B, typename R>
__device__ __forceinline__ void corr_solve(R* __restrict__ x, R* __restrict__ xch, const R* __restrict__ data,
                                           const R* pcr_src, int nx) {
  constexpr int Q = kPartRows - B;
  constexpr int BB = B * B;
  const SolverGeom G = solver_geom(nx, 2 * B - 1);
  const int P = G.P;
  const int k = threadIdx.x;
  const bool act = k < P;
  const int g0 = k * kPartRows;
  R* ytail = xch;
  R* gb0 = xch + P * B;
  R* gb1 = gb0 + P * B;
  R* xsb = gb1 + P * B;
  R y[Q], g[B], ct[BB], ch[BB], xp[kPartRows];
  if (act) {
    load_part<R>(x + g0, xp);
#pragma unroll
    for (int e = 0; e < BB; ++e) {
      ct[e] = __ldg(data + (size_t)rec_ct(B, Q, 0, e) * P + k);
      ch[e] = __ldg(data + (size_t)rec_ch(B, Q, 0, e) * P + k);
    }
    auto LU = [&](int r, int f) -> R { return __ldg(data + (size_t)rec_lu(B, r, f) * P + k); };
#pragma unroll
    for (int r = 0; r < Q; ++r) y[r] = xp[B + r];
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
    for (int a = 0; a < B; ++a) ytail[k * B + a] = y[Q - B + a];
  }
  __syncthreads();
  R cf[2 * BB], fin[BB];
  if (act) {
    const int km = (k + P - 1) & (P - 1);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      R v = xp[a];
#pragma unroll
      for (int c = 0; c < B; ++c) v -= ct[a * B + c] * ytail[km * B + c] + ch[a * B + c] * y[c];
      g[a] = v;
    }
    if (G.T > 0) {
#pragma unroll
      for (int e = 0; e < 2 * BB; ++e) cf[e] = pcr_src[(size_t)e * P + k];
    }
#pragma unroll
    for (int e = 0; e < BB; ++e) fin[e] = pcr_src[(G.fin_off - G.pcr_off) + (size_t)e * P + k];
  }
  // block parallel cyclic reduction on the separators
  for (int t = 0; t < G.T; ++t) {
    R cfn[2 * BB];
    if (act && t + 1 < G.T) {
      const R* lv = pcr_src + (size_t)(t + 1) * 2 * BB * P;
#pragma unroll
      for (int e = 0; e < 2 * BB; ++e) cfn[e] = lv[(size_t)e * P + k];
    }
    R* buf = (t & 1) ? gb1 : gb0;
    if (act) {
#pragma unroll
      for (int a = 0; a < B; ++a) buf[k * B + a] = g[a];
    }
    __syncthreads();
    if (act) {
      const int d = 1 << t;
      const int km = (k - d) & (P - 1), kp = (k + d) & (P - 1);
      R gm[B], gp[B];
#pragma unroll
      for (int a = 0; a < B; ++a) {
        gm[a] = buf[km * B + a];
        gp[a] = buf[kp * B + a];
      }
#pragma unroll
      for (int a = 0; a < B; ++a) {
        R v = g[a];
#pragma unroll
        for (int c = 0; c < B; ++c) v += cf[a * B + c] * gm[c] + cf[BB + a * B + c] * gp[c];
        g[a] = v;
      }
#pragma unroll
      for (int e = 0; e < 2 * BB; ++e) cf[e] = cfn[e];
    }
  }
  R xs[B];
  if (act) {
#pragma unroll
    for (int a = 0; a < B; ++a) {
      R v = (R)0;
#pragma unroll
      for (int c = 0; c < B; ++c) v += fin[a * B + c] * g[c];
      xs[a] = v;
      xsb[k * B + a] = v;
    }
  }
  __syncthreads();
  if (act) {
    const int kp = (k + 1) & (P - 1);
    R xn[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      xn[a] = xsb[kp * B + a];
      xp[a] = xs[a];
    }
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      R v = y[r];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        v -= __ldg(data + (size_t)rec_v(B, Q, r, c) * P + k) * xs[c];
        v -= __ldg(data + (size_t)rec_w(B, Q, r, c) * P + k) * xn[c];
      }
      xp[B + r] = v;
    }
    store_part<R>(x + g0, xp);
  }
  __syncthreads();
}

// ---- on-the-fly correction solve (FP32 coarse levels) ---------------------------------------------
//
// x <- M^{-1} x for M = I - diag(sigma) D_{2B}, factorised in every application from the sigma row:
// the same partitioned algorithm as the stored factorisation (solver_layout.cuh: 8-row partitions,
// interior banded LU, spikes, separator Schur blocks, block PCR), with the PCR reducing the matrix
// blocks in lockstep with the right-hand side.  Reads 4 bytes (sigma) per row instead of the stored
// record; all arithmetic FP32.  X: shared exchange area of (3 B^2 + B) * P floats.

// Coefficient of the centred stencil (delta^2)^B at offset o: (-1)^{B+o} C(2B, B+o).
template <int B>
constexpr float dcoef(int o) {
  int c = 1;
  for (int t = 1; t <= B + o; ++t) c = c * (2 * B - (B + o) + t) / t;
  return (o < -B || o > B) ? 0.f : (((B + o) & 1) ? -(float)c : (float)c);
}

template <int B>
__device__ __forceinline__ void inv_small(const float (&A)[B * B], float (&R)[B * B]) {
  if constexpr (B == 1) {
    R[0] = __frcp_rn(A[0]);
  } else if constexpr (B == 2) {
    const float id = __frcp_rn(A[0] * A[3] - A[1] * A[2]);
    R[0] = A[3] * id;
    R[1] = -A[1] * id;
    R[2] = -A[2] * id;
    R[3] = A[0] * id;
  } else {  // adjugate / determinant
    const float c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const float id = __frcp_rn(A[0] * c00 + A[1] * c01 + A[2] * c02);
    R[0] = c00 * id;
    R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    R[3] = c01 * id;
    R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    R[6] = c02 * id;
    R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  }
}

// C = A * B (B x B, row-major); acc: C += A * B.
template <int B>
__device__ __forceinline__ void mm_small(const float (&A)[B * B], const float (&Bm)[B * B], float (&C)[B * B]) {
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float v = 0.f;
#pragma unroll
      for (int e = 0; e < B; ++e) v += A[a * B + e] * Bm[e * B + c];
      C[a * B + c] = v;
    }
}

template <int B, int PR>
__device__ __forceinline__ void corr_solve_otf(float* __restrict__ x, const float* __restrict__ sig,
                                               float* __restrict__ X, int nx) {
  constexpr int Q = PR - B, BB = B * B;
  const int P = nx / PR;
  const int T = __ffs(P) - 1;  // P is a power of two
  const int k = threadIdx.x;
  const bool act = k < P;
  const int g0 = k * PR;
  float xp[PR], sg[PR] = {};  // sg is read only by the partition threads, after their loads
  float y[Q], V[Q][B], W[Q][B];
  float Lk[BB], Dk[BB], Uk[BB], gk[B];
  // M[g0 + rr, g0 + rr + o] for |o| <= B
  auto M = [&](int rr, int o) -> float { return (o == 0 ? 1.f : 0.f) - sg[rr] * dcoef<B>(o); };
  if (act) {
#pragma unroll
    for (int c = 0; c < PR / kPartRows; ++c) {
      load_part<float>(x + g0 + c * kPartRows, *reinterpret_cast<float(*)[kPartRows]>(xp + c * kPartRows));
      load_part<float>(sig + g0 + c * kPartRows, *reinterpret_cast<float(*)[kPartRows]>(sg + c * kPartRows));
    }
    // 1) banded LU of the interior rows g0 + B + r (no pivoting, as the stored factorisation)
    float l[Q][B], U[Q][B + 1], piv[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float a[2 * B + 1];
#pragma unroll
      for (int c = -B; c <= B; ++c) a[c + B] = (r + c >= 0 && r + c < Q) ? M(B + r, c) : 0.f;
#pragma unroll
      for (int t = B; t >= 1; --t) {
        if (r - t < 0) continue;
        const float lt = a[B - t] * piv[r - t];
        l[r][t - 1] = lt;
#pragma unroll
        for (int c = 1; c <= B; ++c)
          if (-t + c <= B) a[-t + c + B] -= lt * U[r - t][c];
      }
      piv[r] = __frcp_rn(a[B]);
#pragma unroll
      for (int c = 0; c <= B; ++c) U[r][c] = a[B + c];
    }
    auto solve = [&](float (&v)[Q]) {
#pragma unroll
      for (int r = 0; r < Q; ++r)
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r - t >= 0) v[r] -= l[r][t - 1] * v[r - t];
#pragma unroll
      for (int r = Q - 1; r >= 0; --r) {
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r + t < Q) v[r] -= U[r][t] * v[r + t];
        v[r] *= piv[r];
      }
    };
#pragma unroll
    for (int r = 0; r < Q; ++r) y[r] = xp[B + r];
    solve(y);
    // 2) spikes V = A^{-1} M[I_k, S_k], W = A^{-1} M[I_k, S_{k+1}]
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float v[Q], w[Q];
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const int ov = c - B - r, ow = Q - r + c;
        v[r] = ov >= -B ? M(B + r, ov) : 0.f;
        w[r] = ow <= B ? M(B + r, ow) : 0.f;
      }
      solve(v);
      solve(w);
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        V[r][c] = v[r];
        W[r][c] = w[r];
      }
    }
    // tails of V, W, y for partition k + 1
#pragma unroll
    for (int a = 0; a < B; ++a) {
#pragma unroll
      for (int c = 0; c < B; ++c) {
        X[(size_t)(a * B + c) * P + k] = V[Q - B + a][c];
        X[(size_t)(BB + a * B + c) * P + k] = W[Q - B + a][c];
      }
      X[(size_t)(2 * BB + a) * P + k] = y[Q - B + a];
    }
  }
  __syncthreads();
  if (act) {
    // 3) separator row a: ctail (tail of I_{k-1}), Mss (S_k), chead (head of I_k); Schur blocks
    const int km = (k + P - 1) & (P - 1);
    float Vt[BB], Wt[BB], yt[B];
#pragma unroll
    for (int e = 0; e < BB; ++e) {
      Vt[e] = X[(size_t)e * P + km];
      Wt[e] = X[(size_t)(BB + e) * P + km];
    }
#pragma unroll
    for (int a = 0; a < B; ++a) yt[a] = X[(size_t)(2 * BB + a) * P + km];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      float g = xp[a];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float lv = 0.f, dv = M(a, c - a), uv = 0.f;
#pragma unroll
        for (int c2 = 0; c2 < B; ++c2) {
          const float ct = c2 >= a ? M(a, c2 - B - a) : 0.f;
          const float ch = c2 <= a ? M(a, B + c2 - a) : 0.f;
          lv -= ct * Vt[c2 * B + c];
          dv -= ct * Wt[c2 * B + c] + ch * V[c2][c];
          uv -= ch * W[c2][c];
        }
        Lk[a * B + c] = lv;
        Dk[a * B + c] = dv;
        Uk[a * B + c] = uv;
        const float ct = c >= a ? M(a, c - B - a) : 0.f;
        const float ch = c <= a ? M(a, B + c - a) : 0.f;
        g -= ct * yt[c] + ch * y[c];
      }
      gk[a] = g;
    }
  }
  __syncthreads();
  // 4) block PCR on (L, D, U | g); exchange per level: D^{-1}, L, U, g of every partition
  for (int t = 0; t < T; ++t) {
    const int d = 1 << t;
    if (act) {
      float Di[BB];
      inv_small<B>(Dk, Di);
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        X[(size_t)e * P + k] = Di[e];
        X[(size_t)(BB + e) * P + k] = Lk[e];
        X[(size_t)(2 * BB + e) * P + k] = Uk[e];
      }
#pragma unroll
      for (int a = 0; a < B; ++a) X[(size_t)(3 * BB + a) * P + k] = gk[a];
    }
    __syncthreads();
    if (act) {
      const int km = (k - d) & (P - 1), kp = (k + d) & (P - 1);
      float Dm[BB], Dp[BB], al[BB], ga[BB], tmp[BB], tmp2[BB];
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        Dm[e] = X[(size_t)e * P + km];
        Dp[e] = X[(size_t)e * P + kp];
      }
      mm_small<B>(Lk, Dm, al);
      mm_small<B>(Uk, Dp, ga);
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        al[e] = -al[e];
        ga[e] = -ga[e];
      }
#pragma unroll
      for (int a = 0; a < B; ++a) {
        float v = gk[a];
#pragma unroll
        for (int c = 0; c < B; ++c)
          v += al[a * B + c] * X[(size_t)(3 * BB + c) * P + km] + ga[a * B + c] * X[(size_t)(3 * BB + c) * P + kp];
        gk[a] = v;
      }
      // D += al U_{k-d} + ga L_{k+d};  L = al L_{k-d};  U = ga U_{k+d}
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        tmp[e] = X[(size_t)(2 * BB + e) * P + km];   // U_{k-d}
        tmp2[e] = X[(size_t)(BB + e) * P + kp];      // L_{k+d}
      }
      float n1[BB], n2[BB];
      mm_small<B>(al, tmp, n1);
      mm_small<B>(ga, tmp2, n2);
#pragma unroll
      for (int e = 0; e < BB; ++e) Dk[e] += n1[e] + n2[e];
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        tmp[e] = X[(size_t)(BB + e) * P + km];       // L_{k-d}
        tmp2[e] = X[(size_t)(2 * BB + e) * P + kp];  // U_{k+d}
      }
      mm_small<B>(al, tmp, Lk);
      mm_small<B>(ga, tmp2, Uk);
    }
    __syncthreads();
  }
  // 5) separators x_S = (L + D + U)^{-1} g, then the interiors
  float xs[B];
  if (act) {
    float F[BB], Fi[BB];
#pragma unroll
    for (int e = 0; e < BB; ++e) F[e] = Lk[e] + Dk[e] + Uk[e];
    inv_small<B>(F, Fi);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < B; ++c) v += Fi[a * B + c] * gk[c];
      xs[a] = v;
      X[(size_t)a * P + k] = v;
    }
  }
  __syncthreads();
  if (act) {
    const int kp = (k + 1) & (P - 1);
    float xn[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      xn[a] = X[(size_t)a * P + kp];
      xp[a] = xs[a];
    }
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float v = y[r];
#pragma unroll
      for (int c = 0; c < B; ++c) v -= V[r][c] * xs[c] + W[r][c] * xn[c];
      xp[B + r] = v;
    }
#pragma unroll
    for (int c = 0; c < PR / kPartRows; ++c)
      store_part<float>(x + g0 + c * kPartRows, *reinterpret_cast<const float(*)[kPartRows]>(xp + c * kPartRows));
  }
  __syncthreads();
}

// ---- precomputed reduction coefficients of the on-the-fly solve (FP32 coarse levels, B <= 2) --------
//
// Only the right-hand side of the block PCR changes between applications of M^{-1}: the coefficients
// alpha_t = -L_k D_{k-d}^{-1}, gamma_t = -U_k D_{k+d}^{-1} of every level t and the final (L+D+U)^{-1}
// depend on sigma alone.  They are formed once per step (the same FP32 arithmetic as corr_solve_otf)
// and stored as [t][alpha | gamma][B*B][P] then fin [B*B][P], partition fastest, padded to 16 bytes;
// the solve stages the record of each step into shared memory by TMA and runs the PCR on g only.

MGRIT_HD unsigned pcr_record_floats(int nx, int p) {
  const int B = (p + 1) / 2, PR = B <= 2 ? 16 : 8, P = nx / PR;
  int T = 0;
  while ((1 << T) < P) ++T;
  const unsigned n = (unsigned)((2 * T + 1) * B * B * P);
  return (n + 3u) & ~3u;
}

// One CTA per step row (P threads): the matrix part of corr_solve_otf, storing the coefficients.
template <int B, int PR>
__global__ void __launch_bounds__(512) k_pcr_coef(const float* __restrict__ sig_all, int nx, float* __restrict__ out_all,
                                                  unsigned stride) {
  constexpr int Q = PR - B, BB = B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* X = reinterpret_cast<float*>(smem_raw);
  const int P = nx / PR;
  const int T = __ffs(P) - 1;  // P is a power of two
  const int k = threadIdx.x;
  const bool act = k < P;
  const int g0 = k * PR;
  const float* sig = sig_all + (size_t)blockIdx.x * nx;
  float* out = out_all + (size_t)blockIdx.x * stride;
  float sg[PR] = {};  // read only by the partition threads, after their loads
  float V[Q][B], W[Q][B];
  float Lk[BB], Dk[BB], Uk[BB];
  auto M = [&](int rr, int o) -> float { return (o == 0 ? 1.f : 0.f) - sg[rr] * dcoef<B>(o); };
  if (act) {
#pragma unroll
    for (int c = 0; c < PR / kPartRows; ++c)
      load_part<float>(sig + g0 + c * kPartRows, *reinterpret_cast<float(*)[kPartRows]>(sg + c * kPartRows));
    float l[Q][B], U[Q][B + 1], piv[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float a[2 * B + 1];
#pragma unroll
      for (int c = -B; c <= B; ++c) a[c + B] = (r + c >= 0 && r + c < Q) ? M(B + r, c) : 0.f;
#pragma unroll
      for (int t = B; t >= 1; --t) {
        if (r - t < 0) continue;
        const float lt = a[B - t] * piv[r - t];
        l[r][t - 1] = lt;
#pragma unroll
        for (int c = 1; c <= B; ++c)
          if (-t + c <= B) a[-t + c + B] -= lt * U[r - t][c];
      }
      piv[r] = __frcp_rn(a[B]);
#pragma unroll
      for (int c = 0; c <= B; ++c) U[r][c] = a[B + c];
    }
    auto solve = [&](float (&v)[Q]) {
#pragma unroll
      for (int r = 0; r < Q; ++r)
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r - t >= 0) v[r] -= l[r][t - 1] * v[r - t];
#pragma unroll
      for (int r = Q - 1; r >= 0; --r) {
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r + t < Q) v[r] -= U[r][t] * v[r + t];
        v[r] *= piv[r];
      }
    };
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float v[Q], w[Q];
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const int ov = c - B - r, ow = Q - r + c;
        v[r] = ov >= -B ? M(B + r, ov) : 0.f;
        w[r] = ow <= B ? M(B + r, ow) : 0.f;
      }
      solve(v);
      solve(w);
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        V[r][c] = v[r];
        W[r][c] = w[r];
      }
    }
#pragma unroll
    for (int a = 0; a < B; ++a)
#pragma unroll
      for (int c = 0; c < B; ++c) {
        X[(size_t)(a * B + c) * P + k] = V[Q - B + a][c];
        X[(size_t)(BB + a * B + c) * P + k] = W[Q - B + a][c];
      }
  }
  __syncthreads();
  if (act) {
    const int km = (k + P - 1) & (P - 1);
    float Vt[BB], Wt[BB];
#pragma unroll
    for (int e = 0; e < BB; ++e) {
      Vt[e] = X[(size_t)e * P + km];
      Wt[e] = X[(size_t)(BB + e) * P + km];
    }
#pragma unroll
    for (int a = 0; a < B; ++a)
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float lv = 0.f, dv = M(a, c - a), uv = 0.f;
#pragma unroll
        for (int c2 = 0; c2 < B; ++c2) {
          const float ct = c2 >= a ? M(a, c2 - B - a) : 0.f;
          const float ch = c2 <= a ? M(a, B + c2 - a) : 0.f;
          lv -= ct * Vt[c2 * B + c];
          dv -= ct * Wt[c2 * B + c] + ch * V[c2][c];
          uv -= ch * W[c2][c];
        }
        Lk[a * B + c] = lv;
        Dk[a * B + c] = dv;
        Uk[a * B + c] = uv;
      }
  }
  __syncthreads();
  for (int t = 0; t < T; ++t) {
    const int d = 1 << t;
    if (act) {
      float Di[BB];
      inv_small<B>(Dk, Di);
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        X[(size_t)e * P + k] = Di[e];
        X[(size_t)(BB + e) * P + k] = Lk[e];
        X[(size_t)(2 * BB + e) * P + k] = Uk[e];
      }
    }
    __syncthreads();
    if (act) {
      const int km = (k - d) & (P - 1), kp = (k + d) & (P - 1);
      float Dm[BB], Dp[BB], al[BB], ga[BB], tmp[BB], tmp2[BB], n1[BB], n2[BB];
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        Dm[e] = X[(size_t)e * P + km];
        Dp[e] = X[(size_t)e * P + kp];
      }
      mm_small<B>(Lk, Dm, al);
      mm_small<B>(Uk, Dp, ga);
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        al[e] = -al[e];
        ga[e] = -ga[e];
        out[((size_t)(2 * t) * BB + e) * P + k] = al[e];
        out[((size_t)(2 * t + 1) * BB + e) * P + k] = ga[e];
      }
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        tmp[e] = X[(size_t)(2 * BB + e) * P + km];  // U_{k-d}
        tmp2[e] = X[(size_t)(BB + e) * P + kp];     // L_{k+d}
      }
      mm_small<B>(al, tmp, n1);
      mm_small<B>(ga, tmp2, n2);
#pragma unroll
      for (int e = 0; e < BB; ++e) Dk[e] += n1[e] + n2[e];
#pragma unroll
      for (int e = 0; e < BB; ++e) {
        tmp[e] = X[(size_t)(BB + e) * P + km];       // L_{k-d}
        tmp2[e] = X[(size_t)(2 * BB + e) * P + kp];  // U_{k+d}
      }
      mm_small<B>(al, tmp, Lk);
      mm_small<B>(ga, tmp2, Uk);
    }
    __syncthreads();
  }
  if (act) {
    float F[BB], Fi[BB];
#pragma unroll
    for (int e = 0; e < BB; ++e) F[e] = Lk[e] + Dk[e] + Uk[e];
    inv_small<B>(F, Fi);
#pragma unroll
    for (int e = 0; e < BB; ++e) out[((size_t)(2 * T) * BB + e) * P + k] = Fi[e];
  }
}

// The solve with the stored coefficients `cf` (in shared memory): x <- M^{-1} x.  The interior rows are
// solved twice with the banded LU formed from sigma: first with their own right-hand side (y, which
// gives the separator right-hand side g), then, once the separators are known, with the separator
// couplings moved to the right-hand side (the spikes of the stored factorisation are not needed).
// The PCR updates g only.  X: exchange area of at least 3 B P floats.
// `cf` is being filled by a bulk copy that completes on cf_bar (phase parity cf_par): the first interior
// solve needs no coefficient, so the wait comes after it, on the barrier that publishes its tails.  Once
// every thread has read the last coefficient, thread 0 calls issue_next() (the next step's copy into the
// same buffer).  Returns false (all threads) if the bounded wait gave up.
template <int B, int PR, typename IssueNext>
__device__ __forceinline__ bool corr_solve_coef(float* __restrict__ x, const float* __restrict__ sig,
                                                const float* __restrict__ cf, float* __restrict__ X, int nx,
                                                uint64_t* cf_bar, uint32_t cf_par, IssueNext issue_next) {
  constexpr int Q = PR - B, BB = B * B;
  const int P = nx / PR;
  const int T = __ffs(P) - 1;  // P is a power of two
  const int k = threadIdx.x;
  const bool act = k < P;
  const int g0 = k * PR;
  float xp[PR], sg[PR] = {};  // sg is read only by the partition threads, after their loads
  float gk[B];
  auto M = [&](int rr, int o) -> float { return (o == 0 ? 1.f : 0.f) - sg[rr] * dcoef<B>(o); };
  // v <- A^{-1} v for the interior block A (banded LU without pivoting, formed from sigma)
  auto interior_solve = [&](float (&v)[Q]) {
    float l[Q][B], U[Q][B + 1], piv[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float a[2 * B + 1];
#pragma unroll
      for (int c = -B; c <= B; ++c) a[c + B] = (r + c >= 0 && r + c < Q) ? M(B + r, c) : 0.f;
#pragma unroll
      for (int t = B; t >= 1; --t) {
        if (r - t < 0) continue;
        const float lt = a[B - t] * piv[r - t];
        l[r][t - 1] = lt;
#pragma unroll
        for (int c = 1; c <= B; ++c)
          if (-t + c <= B) a[-t + c + B] -= lt * U[r - t][c];
      }
      piv[r] = __frcp_rn(a[B]);
#pragma unroll
      for (int c = 0; c <= B; ++c) U[r][c] = a[B + c];
      // forward substitution of this row as soon as it is eliminated
#pragma unroll
      for (int t = 1; t <= B; ++t)
        if (r - t >= 0) v[r] -= l[r][t - 1] * v[r - t];
    }
#pragma unroll
    for (int r = Q - 1; r >= 0; --r) {
#pragma unroll
      for (int t = 1; t <= B; ++t)
        if (r + t < Q) v[r] -= U[r][t] * v[r + t];
      v[r] *= piv[r];
    }
  };
  if (act) {
#pragma unroll
    for (int c = 0; c < PR / kPartRows; ++c) {
      load_part<float>(x + g0 + c * kPartRows, *reinterpret_cast<float(*)[kPartRows]>(xp + c * kPartRows));
      load_part<float>(sig + g0 + c * kPartRows, *reinterpret_cast<float(*)[kPartRows]>(sg + c * kPartRows));
    }
    float y[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) y[r] = xp[B + r];
    interior_solve(y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      X[(size_t)a * P + k] = y[Q - B + a];
      gk[a] = y[a];  // head of y, used below
    }
  }
  const bool cf_ok = mbar_wait_bounded(cf_bar, cf_par, kWaitLimitCycles);
  if (__syncthreads_or(!cf_ok)) return false;
  if (act) {
    const int km = (k + P - 1) & (P - 1);
    float g[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      float v = xp[a];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const float ct = c >= a ? M(a, c - B - a) : 0.f;
        const float ch = c <= a ? M(a, B + c - a) : 0.f;
        v -= ct * X[(size_t)c * P + km] + ch * gk[c];
      }
      g[a] = v;
    }
#pragma unroll
    for (int a = 0; a < B; ++a) gk[a] = g[a];
  }
  // block PCR on g with the stored alpha / gamma (double-buffered exchange: one barrier a level)
  for (int t = 0; t < T; ++t) {
    float* gb = X + (size_t)(((t & 1) + 1) * B) * P;
    if (act) {
#pragma unroll
      for (int a = 0; a < B; ++a) gb[(size_t)a * P + k] = gk[a];
    }
    __syncthreads();
    if (act) {
      const int d = 1 << t;
      const int km = (k - d) & (P - 1), kp = (k + d) & (P - 1);
      float gm[B], gp[B];
#pragma unroll
      for (int a = 0; a < B; ++a) {
        gm[a] = gb[(size_t)a * P + km];
        gp[a] = gb[(size_t)a * P + kp];
      }
      const float* al = cf + (size_t)(2 * t) * BB * P + k;
      const float* ga = cf + (size_t)(2 * t + 1) * BB * P + k;
#pragma unroll
      for (int a = 0; a < B; ++a) {
        float v = gk[a];
#pragma unroll
        for (int c = 0; c < B; ++c) v += al[(size_t)(a * B + c) * P] * gm[c] + ga[(size_t)(a * B + c) * P] * gp[c];
        gk[a] = v;
      }
    }
  }
  float xs[B];
  if (act) {
    const float* fi = cf + (size_t)(2 * T) * BB * P + k;
#pragma unroll
    for (int a = 0; a < B; ++a) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < B; ++c) v += fi[(size_t)(a * B + c) * P] * gk[c];
      xs[a] = v;
    }
  }
  // the separators go to the area of the y tails, which every thread last read before the first PCR
  // barrier (P = 1: no PCR level, and the one partition thread reads back its own values)
  if (act) {
#pragma unroll
    for (int a = 0; a < B; ++a) X[(size_t)a * P + k] = xs[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) issue_next();  // every coefficient of this step has been read
  if (act) {
    const int kp = (k + 1) & (P - 1);
    float xn[B];
#pragma unroll
    for (int a = 0; a < B; ++a) xn[a] = X[(size_t)a * P + kp];
    // interior: A x_I = b_I - M[I, S_k] x_S(k) - M[I, S_{k+1}] x_S(k+1)
    float v[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float w = xp[B + r];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const int ov = c - B - r, ow = Q - r + c;
        if (ov >= -B) w -= M(B + r, ov) * xs[c];
        if (ow <= B) w -= M(B + r, ow) * xn[c];
      }
      v[r] = w;
    }
    interior_solve(v);
#pragma unroll
    for (int a = 0; a < B; ++a) xp[a] = xs[a];
#pragma unroll
    for (int r = 0; r < Q; ++r) xp[B + r] = v[r];
#pragma unroll
    for (int c = 0; c < PR / kPartRows; ++c)
      store_part<float>(x + g0 + c * kPartRows, *reinterpret_cast<const float(*)[kPartRows]>(xp + c * kPartRows));
  }
  __syncthreads();
  return true;
}

// ---- banded separator inverse (FP32 coarse levels) --------------------------------------------------
//
// With 8-row partitions (one per thread, B separator rows first, Q = 8 - B interior rows) the separator
// unknowns satisfy the Schur system S x_S = g, and S^{-1} is the separator block of M^{-1}, whose entries
// decay exponentially away from the diagonal (M = I - diag(sigma) D is close to a diagonally dominant
// M-matrix on the coarse levels).  Where S^{-1} is below kBandTolerance of its diagonal blocks beyond a few
// partitions, it is stored as a band of half-width W <= kBandMax partitions (setup: k_sep_band probes
// it), and the separator solve is one banded product instead of the block cyclic reduction: two block
// barriers instead of one per reduction level, every thread a partition.

constexpr int kBandMax = kBandMaxHalfWidth;  // largest stored half-bandwidth, in partitions

// Floats of one band row (one offset d: B*B blocks for every partition), padded to 16 bytes, and of a
// whole step record (offsets -kBandMax .. kBandMax; layout [d][a * B + c][partition]).
MGRIT_HD unsigned band_row_floats(int nx, int p) {
  const int B = (p + 1) / 2;
  return ((unsigned)(B * B * (nx / 8)) + 3u) & ~3u;
}
MGRIT_HD unsigned band_record_floats(int nx, int p) { return (2 * kBandMax + 1) * band_row_floats(nx, p); }

// x <- M^{-1} x with 8-row partitions: the interior rows solved from sigma (banded LU, no pivoting), the
// separator right-hand sides g_k, x_S(k) = sum_{|d| <= W} Sinv[k][d] g_{k+d} (band `bd`: the W-trimmed
// record, [d + W][a * B + c][k], rows of `row` floats), then the interiors again with the separators
// known.  X: exchange area of 2 B P floats.  The band is being filled by a bulk copy that completes on
// cf_bar (parity cf_par); the wait comes after the first interior solve.  Once every thread has read
// the band, thread 0 calls issue_next().  Returns false (all threads) if the bounded wait gave up.
template <int B, typename IssueNext>
__device__ __forceinline__ bool corr_solve_band(float* __restrict__ x, const float* __restrict__ sig,
                                                const float* __restrict__ bd, int W, unsigned row,
                                                float* __restrict__ X, int nx, uint64_t* cf_bar, uint32_t cf_par,
                                                IssueNext issue_next) {
  constexpr int PR = kPartRows, Q = PR - B;
  const int P = nx / PR;
  const int k = threadIdx.x;
  const bool act = k < P;
  const int g0 = k * PR;
  float xp[PR], sg[PR] = {};  // sg is read only by the partition threads, after their loads
  float gk[B];
  auto M = [&](int rr, int o) -> float { return (o == 0 ? 1.f : 0.f) - sg[rr] * dcoef<B>(o); };
  auto interior_solve = [&](float (&v)[Q]) {
    float l[Q][B], U[Q][B + 1], piv[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float a[2 * B + 1];
#pragma unroll
      for (int c = -B; c <= B; ++c) a[c + B] = (r + c >= 0 && r + c < Q) ? M(B + r, c) : 0.f;
#pragma unroll
      for (int t = B; t >= 1; --t) {
        if (r - t < 0) continue;
        const float lt = a[B - t] * piv[r - t];
        l[r][t - 1] = lt;
#pragma unroll
        for (int c = 1; c <= B; ++c)
          if (-t + c <= B) a[-t + c + B] -= lt * U[r - t][c];
      }
      piv[r] = __frcp_rn(a[B]);
#pragma unroll
      for (int c = 0; c <= B; ++c) U[r][c] = a[B + c];
#pragma unroll
      for (int t = 1; t <= B; ++t)
        if (r - t >= 0) v[r] -= l[r][t - 1] * v[r - t];
    }
#pragma unroll
    for (int r = Q - 1; r >= 0; --r) {
#pragma unroll
      for (int t = 1; t <= B; ++t)
        if (r + t < Q) v[r] -= U[r][t] * v[r + t];
      v[r] *= piv[r];
    }
  };
  float* G = X + (size_t)B * P;  // separator right-hand sides of every partition
  if (act) {
    load_part<float>(x + g0, xp);
    load_part<float>(sig + g0, sg);
    float y[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) y[r] = xp[B + r];
    interior_solve(y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      X[(size_t)a * P + k] = y[Q - B + a];  // tail of y, read by partition k + 1
      gk[a] = y[a];                          // head of y, used below
    }
  }
  const bool cf_ok = mbar_wait_bounded(cf_bar, cf_par, kWaitLimitCycles);
  if (__syncthreads_or(!cf_ok)) return false;
  if (act) {
    const int km = (k + P - 1) & (P - 1);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      float v = xp[a];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const float ct = c >= a ? M(a, c - B - a) : 0.f;
        const float ch = c <= a ? M(a, B + c - a) : 0.f;
        v -= ct * X[(size_t)c * P + km] + ch * gk[c];
      }
      G[(size_t)a * P + k] = v;
    }
  }
  __syncthreads();
  float xs[B];
  if (act) {
#pragma unroll
    for (int a = 0; a < B; ++a) xs[a] = 0.f;
    for (int d = -W; d <= W; ++d) {
      const int kd = (k + d) & (P - 1);
      const float* br = bd + (size_t)(d + W) * row + k;
      float gv[B];
#pragma unroll
      for (int c = 0; c < B; ++c) gv[c] = G[(size_t)c * P + kd];
#pragma unroll
      for (int a = 0; a < B; ++a)
#pragma unroll
        for (int c = 0; c < B; ++c) xs[a] += br[(size_t)(a * B + c) * P] * gv[c];
    }
    // the separators go to the area of the y tails, which every thread last read before the barrier above
#pragma unroll
    for (int a = 0; a < B; ++a) X[(size_t)a * P + k] = xs[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) issue_next();  // every band entry of this step has been read
  if (act) {
    const int kp = (k + 1) & (P - 1);
    float xn[B];
#pragma unroll
    for (int a = 0; a < B; ++a) xn[a] = X[(size_t)a * P + kp];
    // interior: A x_I = b_I - M[I, S_k] x_S(k) - M[I, S_{k+1}] x_S(k+1)
    float v[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float w = xp[B + r];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const int ov = c - B - r, ow = Q - r + c;
        if (ov >= -B) w -= M(B + r, ov) * xs[c];
        if (ow <= B) w -= M(B + r, ow) * xn[c];
      }
      v[r] = w;
    }
    interior_solve(v);
#pragma unroll
    for (int a = 0; a < B; ++a) xp[a] = xs[a];
#pragma unroll
    for (int r = 0; r < Q; ++r) xp[B + r] = v[r];
    store_part<float>(x + g0, xp);
  }
  __syncthreads();
  return true;
}

// Setup, one CTA per step row of an FP32 coarse level (P = nx / 8 partitions, 16 <= P <= 512, one thread
// each): the band of S^{-1}, the inverse of the separator Schur system S x_S = g of the 8-row partitions.
// Each thread forms the Schur blocks (L_k, D_k, U_k) of its separator from sigma (the interior LU and the
// spikes, as corr_solve_otf does), then S is reduced by block cyclic reduction with all probe right-hand
// sides at once: e = 1 on separator component c of every partition k == col (mod NC), for the NC colours
// (8 or 16) and B components (in groups of G colours).  The value at partition k' is
// Sinv[(k', a), (k' + d, c)] of the probe partition k' + d, d in [1 - NC/2, NC/2], nearest to it (the other
// probe partitions are NC or more away).  Entries |d| <= min(NC/2 - 1, kBandMax) go to the record;
// ind[t], t = 1..NC/2, is raised to the largest |Sinv[k'][d]|, |d| = t, over the largest diagonal block
// entry (at t = NC/2 the two probes k' +- NC/2 are summed: an upper bound of the tail), by atomicMax on the
// bits of non-negative floats.
template <int B>
constexpr int band_group() { return B <= 2 ? 8 : 2; }

template <int B, int NC>
__global__ void __launch_bounds__(512) k_sep_band(const float* __restrict__ sig_all, int nx, float* __restrict__ rec_all,
                                                  unsigned rec_stride, unsigned row, float* __restrict__ ind) {
  constexpr int RMAX = (NC / 2 - 1) < kBandMax ? (NC / 2 - 1) : kBandMax;  // recorded offsets
  constexpr int PR = kPartRows, Q = PR - B, BB = B * B;
  constexpr int G = band_group<B>(), R = G * B;  // colours and right-hand sides of one reduction pass
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* X = reinterpret_cast<float*>(smem_raw);  // [3 BB][P] matrix exchange
  const int P = nx / PR;
  float* Xg = X + (size_t)3 * BB * P;             // [R B][P] right-hand side exchange
  const int T = __ffs(P) - 1;
  const int k = threadIdx.x;
  const bool act = k < P;
  const float* sgrow = sig_all + (size_t)blockIdx.x * nx;
  float* rec = rec_all + (size_t)blockIdx.x * rec_stride;
  float sg[PR] = {};
  float L0[BB], D0[BB], U0[BB];
  auto M = [&](int rr, int o) -> float { return (o == 0 ? 1.f : 0.f) - sg[rr] * dcoef<B>(o); };
  float V[Q][B], W[Q][B];
  if (act) {
    load_part<float>(sgrow + (size_t)k * PR, sg);
    // interior LU (rows B .. PR-1 of the partition, no pivoting) and the spikes V = A^{-1} M[I, S_k],
    // W = A^{-1} M[I, S_{k+1}]
    float l[Q][B], U[Q][B + 1], piv[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      float a[2 * B + 1];
#pragma unroll
      for (int c = -B; c <= B; ++c) a[c + B] = (r + c >= 0 && r + c < Q) ? M(B + r, c) : 0.f;
#pragma unroll
      for (int t = B; t >= 1; --t) {
        if (r - t < 0) continue;
        const float lt = a[B - t] * piv[r - t];
        l[r][t - 1] = lt;
#pragma unroll
        for (int c = 1; c <= B; ++c)
          if (-t + c <= B) a[-t + c + B] -= lt * U[r - t][c];
      }
      piv[r] = __frcp_rn(a[B]);
#pragma unroll
      for (int c = 0; c <= B; ++c) U[r][c] = a[B + c];
    }
    auto solve = [&](float (&v)[Q]) {
#pragma unroll
      for (int r = 0; r < Q; ++r)
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r - t >= 0) v[r] -= l[r][t - 1] * v[r - t];
#pragma unroll
      for (int r = Q - 1; r >= 0; --r) {
#pragma unroll
        for (int t = 1; t <= B; ++t)
          if (r + t < Q) v[r] -= U[r][t] * v[r + t];
        v[r] *= piv[r];
      }
    };
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float v[Q], w[Q];
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const int ov = c - B - r, ow = Q - r + c;
        v[r] = ov >= -B ? M(B + r, ov) : 0.f;
        w[r] = ow <= B ? M(B + r, ow) : 0.f;
      }
      solve(v);
      solve(w);
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        V[r][c] = v[r];
        W[r][c] = w[r];
      }
    }
#pragma unroll
    for (int a = 0; a < B; ++a)
#pragma unroll
      for (int c = 0; c < B; ++c) {
        X[(size_t)(a * B + c) * P + k] = V[Q - B + a][c];
        X[(size_t)(BB + a * B + c) * P + k] = W[Q - B + a][c];
      }
  }
  __syncthreads();
  if (act) {  // the Schur blocks of separator k: couplings to S_{k-1}, S_k, S_{k+1}
    const int km = (k + P - 1) & (P - 1);
    float Vt[BB], Wt[BB];
#pragma unroll
    for (int e = 0; e < BB; ++e) {
      Vt[e] = X[(size_t)e * P + km];
      Wt[e] = X[(size_t)(BB + e) * P + km];
    }
#pragma unroll
    for (int a = 0; a < B; ++a)
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float lv = 0.f, dv = M(a, c - a), uv = 0.f;
#pragma unroll
        for (int c2 = 0; c2 < B; ++c2) {
          const float ct = c2 >= a ? M(a, c2 - B - a) : 0.f;
          const float ch = c2 <= a ? M(a, B + c2 - a) : 0.f;
          lv -= ct * Vt[c2 * B + c];
          dv -= ct * Wt[c2 * B + c] + ch * V[c2][c];
          uv -= ch * W[c2][c];
        }
        L0[a * B + c] = lv;
        D0[a * B + c] = dv;
        U0[a * B + c] = uv;
      }
  }
  float dmax = 0.f, tmax[NC / 2 + 1] = {};
  for (int col0 = 0; col0 < NC; col0 += G) {
    float Lk[BB], Dk[BB], Uk[BB], gk[R][B];
#pragma unroll
    for (int e = 0; e < BB; ++e) {
      Lk[e] = L0[e];
      Dk[e] = D0[e];
      Uk[e] = U0[e];
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int a = 0; a < B; ++a) gk[r][a] = (act && (k & (NC - 1)) == col0 + r / B && a == r % B) ? 1.f : 0.f;
    for (int t = 0; t < T; ++t) {
      __syncthreads();  // the previous level's (or pass's) reads of the exchange are done
      if (act) {
        float Di[BB];
        inv_small<B>(Dk, Di);
#pragma unroll
        for (int e = 0; e < BB; ++e) {
          X[(size_t)e * P + k] = Di[e];
          X[(size_t)(BB + e) * P + k] = Lk[e];
          X[(size_t)(2 * BB + e) * P + k] = Uk[e];
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int a = 0; a < B; ++a) Xg[(size_t)(r * B + a) * P + k] = gk[r][a];
      }
      __syncthreads();
      if (act) {
        const int d = 1 << t;
        const int km = (k - d) & (P - 1), kp = (k + d) & (P - 1);
        float Dm[BB], Dp[BB], al[BB], ga[BB], tmp[BB], tmp2[BB], n1[BB], n2[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) {
          Dm[e] = X[(size_t)e * P + km];
          Dp[e] = X[(size_t)e * P + kp];
        }
        mm_small<B>(Lk, Dm, al);
        mm_small<B>(Uk, Dp, ga);
#pragma unroll
        for (int e = 0; e < BB; ++e) {
          al[e] = -al[e];
          ga[e] = -ga[e];
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int a = 0; a < B; ++a) {
            float v = gk[r][a];
#pragma unroll
            for (int c = 0; c < B; ++c)
              v += al[a * B + c] * Xg[(size_t)(r * B + c) * P + km] + ga[a * B + c] * Xg[(size_t)(r * B + c) * P + kp];
            gk[r][a] = v;
          }
#pragma unroll
        for (int e = 0; e < BB; ++e) {
          tmp[e] = X[(size_t)(2 * BB + e) * P + km];  // U_{k-d}
          tmp2[e] = X[(size_t)(BB + e) * P + kp];     // L_{k+d}
        }
        mm_small<B>(al, tmp, n1);
        mm_small<B>(ga, tmp2, n2);
#pragma unroll
        for (int e = 0; e < BB; ++e) Dk[e] += n1[e] + n2[e];
#pragma unroll
        for (int e = 0; e < BB; ++e) {
          tmp[e] = X[(size_t)(BB + e) * P + km];       // L_{k-d}
          tmp2[e] = X[(size_t)(2 * BB + e) * P + kp];  // U_{k+d}
        }
        mm_small<B>(al, tmp, Lk);
        mm_small<B>(ga, tmp2, Uk);
      }
    }
    if (act) {  // x = (L + D + U)^{-1} g: the columns of S^{-1} on this separator
      float F[BB], Fi[BB];
#pragma unroll
      for (int e = 0; e < BB; ++e) F[e] = Lk[e] + Dk[e] + Uk[e];
      inv_small<B>(F, Fi);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r % B;
        int d = (col0 + r / B - k) & (NC - 1);  // probe partition k + d, d in [1 - NC/2, NC/2]
        if (d > NC / 2) d -= NC;
        const int ad = d < 0 ? -d : d;
#pragma unroll
        for (int a = 0; a < B; ++a) {
          float v = 0.f;
#pragma unroll
          for (int c2 = 0; c2 < B; ++c2) v += Fi[a * B + c2] * gk[r][c2];
          if (ad <= RMAX) rec[(size_t)(d + kBandMax) * row + (size_t)(a * B + c) * P + k] = v;
          if (ad == 0) dmax = fmaxf(dmax, fabsf(v));
          else tmax[ad] = fmaxf(tmax[ad], fabsf(v));
        }
      }
    }
  }
  if (act && dmax > 0.f) {
#pragma unroll
    for (int t = 1; t <= NC / 2; ++t) atomicMax(reinterpret_cast<int*>(ind) + t, __float_as_int(tmax[t] / dmax));
  }
}

// Rows per partition of the on-the-fly solve: 16 for B <= 2 (half the partitions of the stored layout,
// so one PCR level less and half the reduction work), 8 for B = 3 (register budget).
template <int B>
constexpr int otf_rows() { return B <= 2 ? 16 : 8; }

// dst = S^T src for table row `row` (FP64): target k sums, in increasing arrival index i, the weight
// w_a(eps_i) src[i] of every arrival point i whose stencil node a lands on k.  The candidates form the
// window i in [k + fmin + L - P, k + fmax + L] (fmin/fmax: range of floor(s) on this step), so the
// transposed gather is a deterministic gather, not an atomic scatter.
template <int P>
__device__ __forceinline__ void apply_gather_T(const LevelTables& T, int row, const double* __restrict__ src,
                                               double* __restrict__ dst) {
  constexpr int L = (P + 1) / 2;
  const int nx = T.nx;
  const uint16_t* __restrict__ sh = T.shift + (size_t)row * nx;
  const double* __restrict__ w = T.w64 + (size_t)row * (P + 1) * nx;
  const int2 fr = T.frange[row];
  int Wn = P + 1 + (fr.y - fr.x);
  if (Wn > nx) Wn = nx;
  for (int k = threadIdx.x; k < nx; k += blockDim.x) {
    const int start = k + fr.x + L - P;
    double acc = 0.0;
    for (int t = 0; t < Wn; ++t) {
      const int i = wrap_pow2(start + t, nx);
      const int a = wrap_pow2(k - i - (int)__ldg(sh + i), nx);
      if (a <= P) acc += __ldg(w + (size_t)a * nx + i) * src[i];
    }
    dst[k] = acc;
  }
}

// FP32 levels stage each step's tables into shared memory: a double buffer of (eps row, shift row and a
// third row: sigma for coarse levels factorised on the fly, eps_lo for the FP32-pair passes), each buffer
// filled one step ahead by TMA bulk copies that complete on its mbarrier; then, on coarse levels, the
// exchange area of the solve.  Byte offsets from the 128-aligned start of the region: buffer b starts at
// b * per_buf with eps at +0, shift at +e, the third row at +e+h; the barriers at `bars`.
struct StageLayout {
  unsigned e, h, per_buf, cf, bars, xch, total, tx;  // tx: table bytes copied per step
};
MGRIT_HD StageLayout stage_layout(int nx, int p, int otf, unsigned cf_floats, int df = 0, int band = 0) {
  StageLayout o;
  o.e = ((unsigned)nx * 4u + 127u) & ~127u;
  o.h = ((unsigned)nx * 2u + 127u) & ~127u;
  o.per_buf = o.e + o.h + ((otf || df) ? o.e : 0u);
  o.cf = 2 * o.per_buf;  // one buffer of block-PCR coefficients (otf levels with stored coefficients)
  o.bars = o.cf + ((cf_floats * 4u + 127u) & ~127u);
  o.xch = o.bars + 128;
  const int B = (p + 1) / 2, P = nx / (B <= 2 ? 16 : 8);  // partitions of the on-the-fly solve
  const unsigned x_otf = (unsigned)((3 * B * B + B) * P * 4), x_band = (unsigned)(2 * B * (nx / 8) * 4);
  o.total = o.xch + (otf ? (band ? x_band : (x_otf > x_band ? x_otf : x_band)) : 0u);
  o.tx = (unsigned)nx * ((otf || df) ? 10u : 6u);
  return o;
}

// Per-CTA state of the table prefetch (scalars only, so it stays in registers): buffer `cur` holds (or
// receives) the current step's rows; bit b of `phase` is the parity of buffer b's next completion.
struct Stage {
  unsigned char* base;
  StageLayout lay;
  uint32_t phase;
  int cur;
  int pending;     // step row whose copy into buffer `cur` is in flight (-1: none)
  int cf_pending;  // step row whose coefficient record is in flight (-1: none)
  bool ready;      // buffer `cur` has been waited for (stage_wait_ahead)
  int test_wait;   // > 0: the next stage_acquire waits on bar(3), which nothing completes (timeout test)
  MGRIT_D uint64_t* bar(int b) const { return reinterpret_cast<uint64_t*>(base + lay.bars) + b; }
  MGRIT_D unsigned char* buf(int b) const { return base + (size_t)b * lay.per_buf; }
  MGRIT_D const float* eps(int b) const { return reinterpret_cast<const float*>(buf(b)); }
  MGRIT_D const uint16_t* sh(int b) const { return reinterpret_cast<const uint16_t*>(buf(b) + lay.e); }
  MGRIT_D const float* sig(int b) const { return reinterpret_cast<const float*>(buf(b) + lay.e + lay.h); }
  MGRIT_D float* xch() const { return reinterpret_cast<float*>(base + lay.xch); }
  MGRIT_D float* cf() const { return reinterpret_cast<float*>(base + lay.cf); }
};

// Carves the region out of dynamic shared memory after `used` bytes and initialises the barriers
// (all threads must call; includes a barrier).  Inactive (base null) unless T.gather_stage.
__device__ __forceinline__ Stage stage_init(unsigned char* smem, size_t used, const LevelTables& T, bool coarse) {
  Stage s;
  s.base = nullptr;
  s.phase = 0;
  s.cur = 0;
  s.pending = -1;
  s.cf_pending = -1;
  s.ready = false;
  s.test_wait = 0;
  if (!T.gather_stage) return s;
  s.test_wait = T.test_wait;
  s.lay = stage_layout(T.nx, T.p, coarse && T.otf, coarse && T.otf ? T.cf_floats : 0u, T.df, coarse && T.otf && T.band > 0);
  s.base = smem + ((used + 127) & ~(size_t)127);
  if (threadIdx.x == 0) {
    mbar_init(s.bar(0), 1);
    mbar_init(s.bar(1), 1);
    mbar_init(s.bar(2), 1);
    mbar_init(s.bar(3), 1);  // never arrived on: the barrier of the timeout test
  }
  __syncthreads();
  return s;
}

// Thread 0: bulk copies of the rows of step `row` into buffer b (all complete on bar(b)).
__device__ __forceinline__ void stage_issue(const Stage& s, const LevelTables& T, int row, int b, bool otf) {
  const unsigned nx = (unsigned)T.nx;
  unsigned char* d = s.buf(b);
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(s.bar(b), s.lay.tx);
  bulk_copy_g2s(d, T.eps32 + (size_t)row * T.table_stride, nx * 4u, s.bar(b));
  bulk_copy_g2s(d + s.lay.e, T.shift + (size_t)row * T.table_stride, nx * 2u, s.bar(b));
  if (otf)
    bulk_copy_g2s(d + s.lay.e + s.lay.h, (const float*)T.solver + (size_t)row * T.solver_stride, nx * 4u, s.bar(b));
  else if (T.df)
    bulk_copy_g2s(d + s.lay.e + s.lay.h, T.eps_lo + (size_t)row * T.table_stride, nx * 4u, s.bar(b));
}

// Thread 0: bulk copy of the coefficient record of step `row` (the banded separator inverse or the
// block-PCR coefficients; completes on bar(2)).
__device__ __forceinline__ void stage_issue_cf(const Stage& s, const LevelTables& T, int row) {
  const unsigned bytes = T.cf_floats * 4u;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(s.bar(2), bytes);
  bulk_copy_g2s(s.cf(), T.cf_src + (size_t)row * T.cf_stride, bytes, s.bar(2));
}

// Thread 0 issues the copies of a CTA's first step n right after stage_init, so that they overlap the
// load of the start slice (FP32 levels; coarse levels with stored coefficients also the record).
template <int P, int COARSE>
__device__ __forceinline__ void stage_prefetch_first(Stage& s, const LevelTables& T, int n) {
  if (!s.base || n < 0) return;
  if (threadIdx.x == 0) {
    stage_issue(s, T, n, s.cur, COARSE);
    if (COARSE && T.cf_floats) stage_issue_cf(s, T, n);
  }
  s.pending = n;
  if (COARSE && T.cf_floats) s.cf_pending = n;
}

// Issues the next step's copies (and this step's if it was not prefetched), then waits for buffer
// `cur` unless stage_wait_ahead already did; false if the bounded wait gave up (T.err set; thread 0 lets
// the copies in flight land first).
__device__ __forceinline__ bool stage_acquire(Stage& s, const LevelTables& T, int n, int next_n, bool otf) {
  const int b = s.cur;
  if (threadIdx.x == 0) {
    if (s.pending != n) stage_issue(s, T, n, b, otf);
    if (next_n >= 0) stage_issue(s, T, next_n, b ^ 1, otf);
  }
  if (s.ready) {
    s.ready = false;
    return true;
  }
  const uint32_t par = (s.phase >> b) & 1u;
  bool ok;
  if (s.test_wait > 0) {  // timeout test: a wait that runs out; the copies are drained below
    ok = mbar_wait_bounded(s.bar(3), 0u, s.test_wait);
    s.test_wait = 0;
  } else {
    ok = mbar_wait_bounded(s.bar(b), par, kWaitLimitCycles);
  }
  s.phase ^= 1u << b;
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicExch(T.err, 1);
      mbar_wait_bounded(s.bar(b), par, kWaitLimitCycles);
      if (next_n >= 0) mbar_wait_bounded(s.bar(b ^ 1), (s.phase >> (b ^ 1)) & 1u, kWaitLimitCycles);
    }
    return false;
  }
  return true;
}

// At the end of a step: this thread waits for buffer `cur` (the next step's rows, copied since the start
// of the step), so that the caller's end-of-step barrier also agrees on the outcome; the next
// stage_acquire then skips its wait.  On false the caller's barrier reports the failure and the CTA
// stops through stage_abandon.
__device__ __forceinline__ bool stage_wait_ahead(Stage& s) {
  const int b = s.cur;
  const bool ok = mbar_wait_bounded(s.bar(b), (s.phase >> b) & 1u, kWaitLimitCycles);
  s.phase ^= 1u << b;
  s.ready = true;
  return ok;
}

// After a failed stage_wait_ahead: thread 0 sets T.err and lets the copies still in flight (the next
// step's rows and, with stored coefficients, its record) land before the CTA returns.
__device__ __forceinline__ void stage_abandon(const Stage& s, const LevelTables& T, bool record) {
  if (threadIdx.x != 0) return;
  atomicExch(T.err, 1);
  const int b = s.cur;
  mbar_wait_bounded(s.bar(b), ((s.phase >> b) & 1u) ^ 1u, kWaitLimitCycles);
  if (record && s.cf_pending >= 0) mbar_wait_bounded(s.bar(2), (s.phase >> 2) & 1u, kWaitLimitCycles);
}

// One full step src -> dst (Phi, or Psi with the correction solve), given the prefetched gather table.
// next_n: the step this CTA takes after this one (-1: none), whose sigma row is prefetched.
// Returns false if a bounded wait gave up (the caller then stops; the flag T.err is set).
template <int P, typename R, int COARSE, bool TRANS, int NT>
__device__ __forceinline__ bool full_step(const GatherRegs<P, R>& gr, R* src, R* dst, const LevelTables& T, int n,
                                          Stage& stg, int next_n) {
  constexpr int B = (P + 1) / 2;
  if constexpr (TRANS) {  // Phi^T (FP64): coarse levels first solve with M^T in place, then S^T
    const int row = T.reverse ? T.nt - 1 - n : n;
    if constexpr (COARSE) {
      const double* data = (const double*)T.solver + (size_t)row * T.solver_stride;
      const SolverGeom G = solver_geom(T.nx, T.p);
      corr_solve<B, double>((double*)src, (double*)dst, data, data + G.pcr_off, T.nx);
    }
    apply_gather_T<P>(T, row, (const double*)src, (double*)dst);
    __syncthreads();
    (void)gr;
    (void)stg;
    (void)next_n;
    return true;
  }
  if constexpr (std::is_same<R, float>::value) {  // tables staged by TMA; coarse: factorised on the fly
    // a staged coefficient record: the banded separator inverse (COARSE == 2) or, p <= 3, the block-PCR
    // coefficients; without one (p = 5 levels without a band) the matrix is factorised on the fly
    constexpr bool coef = COARSE == 2 || (COARSE == 1 && B <= 2);
    if (coef && threadIdx.x == 0 && stg.cf_pending != n) stage_issue_cf(stg, T, n);
    if (!stage_acquire(stg, T, n, next_n, COARSE)) {
      if (coef && threadIdx.x == 0) mbar_wait_bounded(stg.bar(2), (stg.phase >> 2) & 1u, kWaitLimitCycles);
      return false;
    }
    const int b = stg.cur;
    apply_gather_staged<P, NT>(stg.eps(b), stg.sh(b), (const float*)src, (float*)dst, T.nx);
    __syncthreads();
    if constexpr (COARSE) {
      if constexpr (coef) {
        const uint32_t par = (stg.phase >> 2) & 1u;
        stg.phase ^= 4u;
        auto issue_next = [&]() {
          if (next_n >= 0) stage_issue_cf(stg, T, next_n);
        };
        bool ok;
        if constexpr (COARSE == 2) {  // the banded separator inverse
          ok = corr_solve_band<B>((float*)dst, stg.sig(b), stg.cf(), T.band, band_row_floats(T.nx, T.p), stg.xch(),
                                  T.nx, stg.bar(2), par, issue_next);
        } else {
          ok = corr_solve_coef<B, otf_rows<B>()>((float*)dst, stg.sig(b), stg.cf(), stg.xch(), T.nx, stg.bar(2), par,
                                                 issue_next);
        }
        if (!ok) {  // nothing of the next step's record was issued; the current one may still land
          if (threadIdx.x == 0) {
            atomicExch(T.err, 1);
            mbar_wait_bounded(stg.bar(2), par, kWaitLimitCycles);
            if (next_n >= 0) mbar_wait_bounded(stg.bar(b ^ 1), (stg.phase >> (b ^ 1)) & 1u, kWaitLimitCycles);
          }
          return false;
        }
        stg.cf_pending = next_n;
      } else {
        corr_solve_otf<B, otf_rows<B>()>((float*)dst, stg.sig(b), stg.xch(), T.nx);
      }
    }
    stg.cur ^= 1;
    stg.pending = next_n;
    (void)gr;
    return true;
  } else {
    (void)stg;
    (void)next_n;
    apply_gather<P>(gr, T, src, dst);
    __syncthreads();
    if constexpr (COARSE) {
      const R* data = (const R*)T.solver + (size_t)n * T.solver_stride;
      const SolverGeom G = solver_geom(T.nx, T.p);
      corr_solve<B, R>(dst, src, data, data + G.pcr_off, T.nx);
    }
    return true;
  }
}

// Fine-level kernels keep two (FP32: shared memory of the staged tables) or three (FP64) CTAs per SM.
// The pass of interval j (one CTA); also the body of the batched kernel.
template <int P, typename R, int COARSE, bool TRANS, int NT>
__device__ __forceinline__ void relax_body(const LevelTables& T, const RelaxArgs& a, int j, int buf,
                                           unsigned char* smem_raw) {
  constexpr int kP = kPts;  // points per thread (nx <= kPts * NT)
  R* src = reinterpret_cast<R*>(smem_raw);
  R* dst = src + buf;
  double* red = reinterpret_cast<double*>(dst + buf);
  const int nx = T.nx;
  Stage stg = stage_init(smem_raw, 2 * (size_t)buf * sizeof(R) + 64 * sizeof(double), T, COARSE);
  if constexpr (std::is_same<R, float>::value)
    stage_prefetch_first<P, COARSE>(stg, T, (j < a.J && a.nsteps > 0) ? j * a.m : -1);
  pdl_trigger();
  pdl_wait();  // the set-up tables above are read-only; everything below depends on the previous kernel
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
  if constexpr (std::is_same<R, float>::value) write_halo(src, nx);
  __syncthreads();
  if (j >= a.J) return;  // extra CTA: only the correction of the last C-point
  double sq = 0.0;
  // FP32: the next step's gather table is loaded during the current step; FP64 (ALU bound, and short
  // of registers for two tables) loads it at the start of its step.
  constexpr bool kPipe = std::is_same<R, float>::value;
  GatherRegs<P, R> gcur, gnext;
  if (kPipe && a.nsteps > 0) load_gather<P, R>(gnext, T, j * a.m);
  for (int k = 0; k < a.nsteps; ++k) {
    const int n = j * a.m + k;
    if constexpr (kPipe) {
      gcur = gnext;
      if (k + 1 < a.nsteps) load_gather<P, R>(gnext, T, n + 1);
    } else {
      load_gather<P, R>(gcur, T, n);
    }
    const R* gr = a.g ? (const R*)a.g + (size_t)(n + 1) * nx : nullptr;
    // FP32: the right-hand side of this step is loaded before the step so its latency is hidden
    R gpre[kP];
    if constexpr (kPipe) {
      if (gr) {
#pragma unroll
        for (int q = 0; q < kP; ++q) {
          const int i = threadIdx.x + q * NT;
          gpre[q] = (i < nx) ? gr[i] : (R)0;
        }
      }
    }
    if (!full_step<P, R, COARSE, TRANS, NT>(gcur, src, dst, T, n, stg, k + 1 < a.nsteps ? n + 1 : -1)) return;
    const bool last = (k == a.m - 1);
    R* fs = a.fstore ? (R*)a.fstore + (size_t)(n + 1) * nx : nullptr;
    if (!last) {
      if (gr || fs) {  // F-point: add the right-hand side and / or store it
#pragma unroll
        for (int q = 0; q < kP; ++q) {
          const int i = threadIdx.x + q * NT;
          if (i >= nx) continue;
          R v = dst[i];
          if (gr) {
            if constexpr (kPipe) v += gpre[q];
            else v += gr[i];
          }
          dst[i] = v;
          if (fs) fs[i] = v;
        }
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
      const R* cc = a.cin_corr ? (const R*)a.cin_corr + (size_t)(j + 1) * a.corr_stride : nullptr;
      R* ro = a.rout_f64 ? nullptr : (R*)a.rout + (size_t)(j + 1) * a.r_stride;
      double* ro64 = a.rout_f64 ? (double*)a.rout + (size_t)(j + 1) * a.r_stride : nullptr;
      float* ro32 = a.rout32 ? a.rout32 + (size_t)(j + 1) * a.r_stride : nullptr;
      R sqt = (R)0;  // FP32 levels accumulate their (FP32) residual in FP32 per thread
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        R v = dst[i];
        if (gr && a.g_at_c) v += gr[i];
        if (cc) v -= (ci ? ci[i] : (R)0) + cc[i];  // the corrected C value, rounded as it is stored
        else if (ci) v -= ci[i];
        if (ro64) ro64[i] = (double)v;
        else ro[i] = v;
        if (ro32) ro32[i] = (float)v;
        if (a.norm_partial) sqt += v * v;
      }
      sq += (double)sqt;
    }
    if constexpr (kPipe) {  // FP32: halo of the next step's source; the wait for its rows joins the barrier
      bool ahead_ok = true;
      if (k + 1 < a.nsteps) {
        write_halo(dst, nx);
        ahead_ok = stage_wait_ahead(stg);
      }
      if (__syncthreads_or(!ahead_ok)) {
        stage_abandon(stg, T, COARSE && T.cf_floats > 0);
        return;
      }
    } else {
      __syncthreads();
    }
    R* t = src;
    src = dst;
    dst = t;
  }
  if (a.mode == MODE_RES && a.norm_partial) {
    const double tot = block_sum(sq, red);
    if (threadIdx.x == 0) a.norm_partial[j] = tot;
  }
}

template <int P, typename R, int COARSE, bool TRANS>
__global__ void __launch_bounds__(slice_threads<P, R, COARSE>(),
                                  COARSE ? (slice_threads<P, R, COARSE>() == 256 ? 2 : 1)
                                         : (std::is_same<R, float>::value ? 2 : 3))
    k_relax_1d(LevelTables T, RelaxArgs a, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  relax_body<P, R, COARSE, TRANS, slice_threads<P, R, COARSE>()>(T, a, blockIdx.x, buf, smem_raw);
}

// ---- level-0 FP64 passes of the FP32-bulk cycle in FP32 pairs --------------------------------------
//
// The exact C-point residual of the FP64 iterate (MODE_RES), and the final post F-relaxation into the
// FP64 solution (MODE_POST), with the fine SL step of Sec. 2.1 evaluated in FP32 pairs (df32.cuh, about
// 48 bits): the slice lives in shared memory as (hi, lo) pairs and the Lagrange weights are formed in
// registers from the step's eps (hi, lo) and shift rows, which are read straight from global memory
// (coalesced); with the slices alone in shared memory and at most 64 registers a thread, two 512-thread
// CTAs share an SM, whose warps hide the loads.  FP64 appears only where the interval meets FP64 data:
// the start slice, the C-point residual, the F-point stores.  Level 0 adds no right-hand side (g = 0).

// dst[i] = (S_n src)_i for the points of this thread, src with its periodic halo (src[nx + t] = src[t]).
// All of the thread's table loads are issued before the first interpolation, so a warp waits for the
// step's rows once rather than once per point.
template <int P, int NT>
__device__ __forceinline__ void apply_gather_df(const float* __restrict__ eh, const float* __restrict__ el,
                                                const uint16_t* __restrict__ sh, const float2* __restrict__ src,
                                                float2* __restrict__ dst, int nx) {
  float h[kPts], l[kPts];
  int s[kPts];
#pragma unroll
  for (int q = 0; q < kPts; ++q) {
    const int i = threadIdx.x + q * NT;
    h[q] = 0.f;
    l[q] = 0.f;
    s[q] = 0;
    if (i < nx) {
      h[q] = __ldg(eh + i);
      l[q] = __ldg(el + i);
      s[q] = (int)__ldg(sh + i);
    }
  }
#pragma unroll
  for (int q = 0; q < kPts; ++q) {
    const int i = threadIdx.x + q * NT;
    if (i < nx) {
      const df32 v = df_interp<P>(df32{h[q], l[q]}, src + wrap_pow2(i + s[q], nx));
      dst[i] = make_float2(v.h, v.l);
    }
  }
}

template <int P, int NT>
__device__ __forceinline__ void relax_body_df(const LevelTables& T, const RelaxArgs& a, int j, int buf,
                                              unsigned char* smem_raw) {
  float2* src = reinterpret_cast<float2*>(smem_raw);
  float2* dst = src + buf;
  double* red = reinterpret_cast<double*>(dst + buf);
  const int nx = T.nx;
  // the table rows of a step are read once, straight from global memory: they are asked into L2 two
  // steps ahead (three bulk prefetches a step, one thread each), so the gather's loads hit L2
  auto prefetch_rows = [&](int k) {
    if (k >= a.nsteps || threadIdx.x >= 96 || (threadIdx.x & 31)) return;
    const size_t row = (size_t)(j * a.m + k) * T.table_stride;
    const int w = threadIdx.x >> 5;
    if (w == 0) bulk_prefetch_l2(T.eps32 + row, (uint32_t)nx * 4u);
    else if (w == 1) bulk_prefetch_l2(T.eps_lo + row, (uint32_t)nx * 4u);
    else bulk_prefetch_l2(T.shift + row, (uint32_t)nx * 2u);
  };
  if (j < a.J) {
    prefetch_rows(0);
    prefetch_rows(1);
  }
  pdl_trigger();
  pdl_wait();  // the tables are read-only; the slices and C-point arrays come from the previous kernel
  {
    const double* st = a.start ? (const double*)a.start + (size_t)j * a.start_stride : nullptr;
    const double* co = a.corr ? (const double*)a.corr + (size_t)j * a.corr_stride : nullptr;
    double* wb = a.start_wb ? (double*)a.start_wb + (size_t)j * a.wb_stride : nullptr;
    for (int i = threadIdx.x; i < nx; i += NT) {
      double v = st ? st[i] : 0.0;
      if (co) v += co[i];
      const df32 d = df_from_double(v);
      src[i] = make_float2(d.h, d.l);
      if (wb) wb[i] = v;
    }
  }
  write_halo(src, nx);
  __syncthreads();
  if (j >= a.J) return;  // extra CTA: only the correction of the last C-point
  double sq = 0.0;
  for (int k = 0; k < a.nsteps; ++k) {
    const int n = j * a.m + k;
    const size_t row = (size_t)n * T.table_stride;
    prefetch_rows(k + 2);
    apply_gather_df<P, NT>(T.eps32 + row, T.eps_lo + row, T.shift + row, src, dst, nx);
    __syncthreads();
    const bool last = (k == a.m - 1);
    if (!last) {
      if (a.fstore) {  // F-point of the FP64 solution
        double* fs = (double*)a.fstore + (size_t)(n + 1) * nx;
        for (int i = threadIdx.x; i < nx; i += NT) {
          const float2 v = dst[i];
          fs[i] = df_to_double_bits(df32{v.x, v.y});
        }
      }
    } else if (a.mode == MODE_FC) {
      double* co = (double*)a.cout + (size_t)(j + 1) * a.c_stride;
      for (int i = threadIdx.x; i < nx; i += NT) {
        const float2 v = dst[i];
        co[i] = df_to_double(df32{v.x, v.y});
      }
    } else {  // MODE_RES: r = S^m u_C(j) - u_C(j+1), in FP64 from the pair
      const double* ci = a.cin ? (const double*)a.cin + (size_t)(j + 1) * a.c_stride : nullptr;
      const double* cc = a.cin_corr ? (const double*)a.cin_corr + (size_t)(j + 1) * a.corr_stride : nullptr;
      double* ro = a.rout ? (double*)a.rout + (size_t)(j + 1) * a.r_stride : nullptr;
      float* ro32 = a.rout32 ? a.rout32 + (size_t)(j + 1) * a.r_stride : nullptr;
      for (int i = threadIdx.x; i < nx; i += NT) {
        const float2 d = dst[i];
        const double pv = df_to_double(df32{d.x, d.y});
        double v = pv;
        if (cc) v -= (ci ? ci[i] : 0.0) + cc[i];
        else if (ci) v -= ci[i];
        if (ro) ro[i] = a.rout_value ? pv : v;
        if (ro32) ro32[i] = (float)v;
        if (a.norm_partial) sq += v * v;
      }
    }
    if (k + 1 < a.nsteps) write_halo(dst, nx);
    __syncthreads();
    float2* t = src;
    src = dst;
    dst = t;
  }
  if (a.mode == MODE_RES && a.norm_partial) {
    const double tot = block_sum(sq, red);
    if (threadIdx.x == 0) a.norm_partial[j] = tot;
  }
}

template <int P>
__global__ void __launch_bounds__(kSliceThreads, 2) k_relax_df_1d(LevelTables T, RelaxArgs a, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  relax_body_df<P, kSliceThreads>(T, a, blockIdx.x, buf, smem_raw);
}

// u0: [nx] start slice; out: store_all ? [(N+1)][nx] (row 0 = u0) : [nx] (the final slice).
template <int P, typename R, int COARSE, bool TRANS, int NT>
__device__ __forceinline__ void sequential_body(const LevelTables& T, int N, const R* g, const R* u0, R* out_all,
                                                int store_all, int buf, unsigned char* smem_raw) {
  R* src = reinterpret_cast<R*>(smem_raw);
  R* dst = src + buf;
  const int nx = T.nx;
  Stage stg = stage_init(smem_raw, 2 * (size_t)buf * sizeof(R) + 64 * sizeof(double), T, COARSE);
  if constexpr (std::is_same<R, float>::value) stage_prefetch_first<P, COARSE>(stg, T, N > 0 ? 0 : -1);
  pdl_trigger();
  pdl_wait();  // u0 and g come from the previous kernel
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const R v = u0 ? u0[i] : (R)0;
    src[i] = v;
    if (store_all) out_all[i] = v;
  }
  if constexpr (std::is_same<R, float>::value) write_halo(src, nx);
  __syncthreads();
  constexpr bool kPipe = std::is_same<R, float>::value;
  GatherRegs<P, R> gcur, gnext;
  if (kPipe && N > 0) load_gather<P, R>(gnext, T, 0);
  for (int n = 0; n < N; ++n) {
    if constexpr (kPipe) {
      gcur = gnext;
      if (n + 1 < N) load_gather<P, R>(gnext, T, n + 1);
    } else {
      load_gather<P, R>(gcur, T, n);
    }
    if (!full_step<P, R, COARSE, TRANS, NT>(gcur, src, dst, T, n, stg, n + 1 < N ? n + 1 : -1)) return;
    const R* gr = g ? g + (size_t)(n + 1) * nx : nullptr;
    R* out = store_all ? out_all + (size_t)(n + 1) * nx : (n == N - 1 ? out_all : nullptr);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      R v = dst[i];
      if (gr) v += gr[i];
      dst[i] = v;
      if (out) out[i] = v;
    }
    if constexpr (kPipe) write_halo(dst, nx);
    __syncthreads();
    R* t = src;
    src = dst;
    dst = t;
  }
}

template <int P, typename R, int COARSE, bool TRANS>
__global__ void __launch_bounds__(slice_threads<P, R, COARSE>()) k_sequential_1d(LevelTables T, int N, const R* g,
                                                                                 const R* u0, R* out_all,
                                                                                 int store_all, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sequential_body<P, R, COARSE, TRANS, slice_threads<P, R, COARSE>()>(T, N, g, u0, out_all, store_all, buf,
                                                                       smem_raw);
}

// ---- batched problems: one launch per cycle phase over (problem, interval) tiles --------------------

// NT threads a CTA (FP32 tiles of slices up to kPts * NT points; FP64 tiles use 512): a smaller CTA for
// the problems with shorter slices, so that more of their intervals are resident on an SM at once.  The
// minimum CTAs per SM scale with 512 / NT, keeping the register budget a thread of the 512-thread kernel.
template <typename R, int COARSE, int NT>
__global__ void __launch_bounds__(NT, (COARSE ? 1 : (std::is_same<R, float>::value ? 2 : 3)) * (kSliceThreads / NT))
    k_relax_batched(const LevelTables* __restrict__ tabs, const RelaxArgs* __restrict__ args,
                    const BatchTile* __restrict__ tiles, const int* __restrict__ active, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchTile t = tiles[blockIdx.x];
  if (active && !active[t.problem]) return;
  const LevelTables T = tabs[t.table];
  const RelaxArgs a = args[t.args];
  switch (T.p) {
    case 1: relax_body<1, R, COARSE, false, NT>(T, a, t.j, buf, smem_raw); break;
    case 3: relax_body<3, R, COARSE, false, NT>(T, a, t.j, buf, smem_raw); break;
    default: relax_body<5, R, COARSE, false, NT>(T, a, t.j, buf, smem_raw); break;
  }
}

// The FP32-pair level-0 passes of every problem of a batch (one tile per interval), NT threads a CTA
// (slices of at most kPts * NT points), as the FP32 batched passes.
template <int NT>
__global__ void __launch_bounds__(NT, 2 * kSliceThreads / NT)
    k_relax_batched_df(const LevelTables* __restrict__ tabs, const RelaxArgs* __restrict__ args,
                       const BatchTile* __restrict__ tiles, const int* __restrict__ active, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchTile t = tiles[blockIdx.x];
  if (active && !active[t.problem]) return;
  const LevelTables T = tabs[t.table];
  const RelaxArgs a = args[t.args];
  switch (T.p) {
    case 1: relax_body_df<1, NT>(T, a, t.j, buf, smem_raw); break;
    case 3: relax_body_df<3, NT>(T, a, t.j, buf, smem_raw); break;
    default: relax_body_df<5, NT>(T, a, t.j, buf, smem_raw); break;
  }
}

template <typename R, int COARSE>
__global__ void __launch_bounds__(kSliceThreads, 1) k_sequential_batched(const LevelTables* __restrict__ tabs,
                                                                         const SeqArgs* __restrict__ args,
                                                                         const BatchTile* __restrict__ tiles,
                                                                         const int* __restrict__ active, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchTile t = tiles[blockIdx.x];
  if (active && !active[t.problem]) return;
  const LevelTables T = tabs[t.table];
  const SeqArgs a = args[t.args];
  switch (T.p) {
    case 1: sequential_body<1, R, COARSE, false, kSliceThreads>(T, a.N, (const R*)a.g, (const R*)a.u0, (R*)a.out, a.store_all, buf, smem_raw); break;
    case 3: sequential_body<3, R, COARSE, false, kSliceThreads>(T, a.N, (const R*)a.g, (const R*)a.u0, (R*)a.out, a.store_all, buf, smem_raw); break;
    default: sequential_body<5, R, COARSE, false, kSliceThreads>(T, a.N, (const R*)a.g, (const R*)a.u0, (R*)a.out, a.store_all, buf, smem_raw); break;
  }
}

template <int P, typename R, int COARSE, bool TRANS>
__global__ void __launch_bounds__(slice_threads<P, R, COARSE>()) k_apply_1d(LevelTables T, int n0, const R* in,
                                                                            R* out, int buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* src = reinterpret_cast<R*>(smem_raw);
  R* dst = src + buf;
  const int nx = T.nx, c = blockIdx.x;
  Stage stg = stage_init(smem_raw, 2 * (size_t)buf * sizeof(R) + 64 * sizeof(double), T, COARSE);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) src[i] = in[(size_t)c * nx + i];
  if constexpr (std::is_same<R, float>::value) write_halo(src, nx);
  __syncthreads();
  GatherRegs<P, R> gr;
  load_gather<P, R>(gr, T, n0 + c);
  if (!full_step<P, R, COARSE, TRANS, slice_threads<P, R, COARSE>()>(gr, src, dst, T, n0 + c, stg, -1)) return;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) out[(size_t)c * nx + i] = dst[i];
}

int buffer_elems(const LevelTables& T, bool coarse) {
  int e = T.nx + kMaxOrder;  // the slice and the periodic halo of the FP32 gather
  if (coarse && !T.otf) {  // the stored-factor solve uses the consumed gather source as exchange area
    const int need = 4 * (T.nx / kPartRows) * ((T.p + 1) / 2);
    if (need > e) e = need;
  }
  return (e + 31) & ~31;
}

// Shared bytes for slice buffers of `buf` elements of type R plus the coarse region of T.
template <typename R>
size_t smem_bytes(int buf, const LevelTables& T, bool coarse) {
  size_t b = 2 * (size_t)buf * sizeof(R) + 64 * sizeof(double);
  if (T.gather_stage)
    b = ((b + 127) & ~(size_t)127) +
        stage_layout(T.nx, T.p, coarse && T.otf, coarse && T.otf ? T.cf_floats : 0u, T.df, coarse && T.otf && T.band > 0).total;
  return b;
}

// Launches kern with programmatic stream serialization (see pdl_wait): it may begin its prologue while the
// previous kernel on the stream finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename R, int COARSE, bool TR>
cudaError_t relax_dispatch(const LevelTables& T, const RelaxArgs& a, cudaStream_t st) {
  const int buf = buffer_elems(T, COARSE);
  const size_t sm = smem_bytes<R>(buf, T, COARSE);
  const int grid = a.J + (a.extra_cta ? 1 : 0);
  if (grid <= 0) return cudaSuccess;
#define MGRIT_LAUNCH_RELAX(PP)                                                                             \
  {                                                                                                        \
    auto kern = k_relax_1d<PP, R, COARSE, TR>;                                                                 \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
    if (e != cudaSuccess) return e;                                                                        \
    e = launch_pdl(kern, (unsigned)grid, (unsigned)slice_threads<PP, R, COARSE>(), sm, st, T, a, buf);      \
    return e != cudaSuccess ? e : cudaGetLastError();                                                      \
  }
  if (T.p == 1) MGRIT_LAUNCH_RELAX(1)
  if (T.p == 3) MGRIT_LAUNCH_RELAX(3)
  MGRIT_LAUNCH_RELAX(5)
#undef MGRIT_LAUNCH_RELAX
}

cudaError_t relax_df_dispatch(const LevelTables& T, const RelaxArgs& a, cudaStream_t st) {
  const int buf = buffer_elems(T, false);
  const size_t sm = smem_bytes<float2>(buf, T, false);
  const int grid = a.J + (a.extra_cta ? 1 : 0);
  if (grid <= 0) return cudaSuccess;
#define MGRIT_LAUNCH_DF(PP)                                                                                \
  {                                                                                                        \
    cudaError_t e = cudaFuncSetAttribute(k_relax_df_1d<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                         (int)sm);                                                         \
    if (e != cudaSuccess) return e;                                                                        \
    e = launch_pdl(k_relax_df_1d<PP>, (unsigned)grid, (unsigned)kSliceThreads, sm, st, T, a, buf);         \
    return e != cudaSuccess ? e : cudaGetLastError();                                                      \
  }
  if (T.p == 1) MGRIT_LAUNCH_DF(1)
  if (T.p == 3) MGRIT_LAUNCH_DF(3)
  MGRIT_LAUNCH_DF(5)
#undef MGRIT_LAUNCH_DF
}

template <typename R, int COARSE, bool TR>
cudaError_t sequential_dispatch(const LevelTables& T, int N, const void* g, const void* u0, void* u, int store_all,
                                cudaStream_t st) {
  const int buf = buffer_elems(T, COARSE);
  const size_t sm = smem_bytes<R>(buf, T, COARSE);
#define MGRIT_LAUNCH_SEQ(PP)                                                                               \
  {                                                                                                        \
    auto kern = k_sequential_1d<PP, R, COARSE, TR>;                                                            \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
    if (e != cudaSuccess) return e;                                                                        \
    e = launch_pdl(kern, 1u, (unsigned)slice_threads<PP, R, COARSE>(), sm, st, T, N, (const R*)g, (const R*)u0, \
                   (R*)u, store_all, buf);                                                                 \
    return e != cudaSuccess ? e : cudaGetLastError();                                                      \
  }
  if (T.p == 1) MGRIT_LAUNCH_SEQ(1)
  if (T.p == 3) MGRIT_LAUNCH_SEQ(3)
  MGRIT_LAUNCH_SEQ(5)
#undef MGRIT_LAUNCH_SEQ
}

template <typename R, int COARSE, bool TR>
cudaError_t apply_dispatch(const LevelTables& T, int n0, int count, const void* in, void* out, cudaStream_t st) {
  const int buf = buffer_elems(T, COARSE);
  const size_t sm = smem_bytes<R>(buf, T, COARSE);
#define MGRIT_LAUNCH_APPLY(PP)                                                                             \
  {                                                                                                        \
    auto kern = k_apply_1d<PP, R, COARSE, TR>;                                                                 \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
    if (e != cudaSuccess) return e;                                                                        \
    kern<<<count, slice_threads<PP, R, COARSE>(), sm, st>>>(T, n0, (const R*)in, (R*)out, buf);                             \
    return cudaGetLastError();                                                                             \
  }
  if (T.p == 1) MGRIT_LAUNCH_APPLY(1)
  if (T.p == 3) MGRIT_LAUNCH_APPLY(3)
  MGRIT_LAUNCH_APPLY(5)
#undef MGRIT_LAUNCH_APPLY
}

template <int P>
__global__ void __launch_bounds__(kSliceThreads) k_gradient_a_1d(LevelTables T, const double* __restrict__ s64,
                                                                 const double* __restrict__ ds,
                                                                 const double* __restrict__ C,
                                                                 const double* __restrict__ mu, int nt, int m,
                                                                 double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* u = reinterpret_cast<double*>(smem_raw);
  double* v = u + T.nx;
  double* red = v + T.nx;
  const int nx = T.nx, j = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) u[i] = C[(size_t)j * nx + i];
  __syncthreads();
  double acc = 0.0;
  for (int k = 0; k < m; ++k) {
    const int n = j * m + k;
    const double* lam = mu + (size_t)(nt - n - 1) * nx;  // lambda_{n+1}
    const uint16_t* sh = T.shift + (size_t)n * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double sv = s64[(size_t)n * nx + i];
      double eps = sv - floor(sv);
      if (eps >= 1.0) eps -= 1.0;
      double dw[P + 1];
      lagrange_weights_deps<P>(eps, dw);
      const int b = i + (int)sh[i];
      double t = 0.0;
#pragma unroll
      for (int a = 0; a <= P; ++a) t += dw[a] * u[wrap_pow2(b + a, nx)];
      acc += lam[i] * ds[(size_t)n * nx + i] * t;
    }
    GatherRegs<P, double> gr;
    load_gather<P, double>(gr, T, n);
    apply_gather<P>(gr, T, u, v);
    __syncthreads();
    double* t = u;
    u = v;
    v = t;
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) partial[j] = tot;
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
    case 5: ((double*)y)[i] += ((const double*)x)[i] + (double)((const float*)z)[i]; break;
    case 7: ((double*)y)[i] += ((const double*)x)[i] + ((const double*)z)[i]; break;
    case 8: ((double*)y)[i] = ((const double*)x)[i] + float_to_double_bits(((const float*)z)[i]); break;
    case 9: ((double*)y)[i] = ((const double*)x)[i] + ((const double*)z)[i]; break;
    default: ((double*)y)[i] = ((const double*)x)[i] - ((const double*)z)[i]; break;
  }
}

}  // namespace

cudaError_t launch_relax_1d(const LevelTables& T, const RelaxArgs& a, int is_double, cudaStream_t st) {
  const bool coarse = T.solver != nullptr;
  if (T.df) {  // level-0 FP64 pass of an FP32-bulk handle: FP32 pairs
    if (!is_double || coarse || T.trans || !T.eps_lo) return cudaErrorInvalidValue;
    return relax_df_dispatch(T, a, st);
  }
  if (T.trans) {
    if (!is_double) return cudaErrorInvalidValue;
    return coarse ? relax_dispatch<double, 1, true>(T, a, st) : relax_dispatch<double, 0, true>(T, a, st);
  }
  if (is_double && coarse && T.cluster) {
    const int C = cluster_relax_size(T, a);
    if (C > 1) {
      const cudaError_t e = launch_relax_cluster_1d(T, a, C, st);
      if (e != cudaErrorNotSupported) return e;
      cudaGetLastError();
    }
  }
  if (is_double)
    return coarse ? relax_dispatch<double, 1, false>(T, a, st) : relax_dispatch<double, 0, false>(T, a, st);
  if (coarse) return T.band ? relax_dispatch<float, 2, false>(T, a, st) : relax_dispatch<float, 1, false>(T, a, st);
  return relax_dispatch<float, 0, false>(T, a, st);
}

cudaError_t launch_sequential_1d(const LevelTables& T, int N, const void* g, const void* u0, void* u, int store_all,
                                 int is_double, cudaStream_t st) {
  const bool coarse = T.solver != nullptr;
  if (T.trans) {
    if (!is_double) return cudaErrorInvalidValue;
    return coarse ? sequential_dispatch<double, 1, true>(T, N, g, u0, u, store_all, st)
                  : sequential_dispatch<double, 0, true>(T, N, g, u0, u, store_all, st);
  }
  if (is_double)
    return coarse ? sequential_dispatch<double, 1, false>(T, N, g, u0, u, store_all, st)
                  : sequential_dispatch<double, 0, false>(T, N, g, u0, u, store_all, st);
  if (coarse)
    return T.band ? sequential_dispatch<float, 2, false>(T, N, g, u0, u, store_all, st)
                  : sequential_dispatch<float, 1, false>(T, N, g, u0, u, store_all, st);
  return sequential_dispatch<float, 0, false>(T, N, g, u0, u, store_all, st);
}

cudaError_t launch_apply_steps_1d(const LevelTables& T, int n0, int count, const void* in, void* out, int is_double,
                                  cudaStream_t st) {
  const bool coarse = T.solver != nullptr;
  if (count <= 0) return cudaSuccess;
  if (T.trans) {
    if (!is_double) return cudaErrorInvalidValue;
    return coarse ? apply_dispatch<double, 1, true>(T, n0, count, in, out, st)
                  : apply_dispatch<double, 0, true>(T, n0, count, in, out, st);
  }
  if (is_double)
    return coarse ? apply_dispatch<double, 1, false>(T, n0, count, in, out, st)
                  : apply_dispatch<double, 0, false>(T, n0, count, in, out, st);
  if (coarse)
    return T.band ? apply_dispatch<float, 2, false>(T, n0, count, in, out, st)
                  : apply_dispatch<float, 1, false>(T, n0, count, in, out, st);
  return apply_dispatch<float, 0, false>(T, n0, count, in, out, st);
}

void launch_sum(const double* v, int count, double* out, cudaStream_t st) { k_sum<<<1, 1024, 0, st>>>(v, count, out); }

namespace {

// out = sum_i (a[i] + b[i] - ref[i])^2 (b optional), one CTA, fixed summation order.
__global__ void k_dist2(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ ref,
                        long long n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double e = (b ? a[i] + b[i] : a[i]) - ref[i];
    s += e * e;
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) out[0] = t;
}

}  // namespace

void launch_dist2(const double* a, const double* b, const double* ref, long long n, double* out, cudaStream_t st) {
  k_dist2<<<1, 1024, 0, st>>>(a, b, ref, n, out);
}

namespace {

__global__ void k_axpy_batched(int kind, const Segment* __restrict__ seg) {
  const Segment sg = seg[blockIdx.y];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < sg.n; i += (long long)gridDim.x * blockDim.x) {
    switch (kind) {
      case 1: ((float*)sg.y)[i] = (float)((const double*)sg.x)[i]; break;
      case 3: ((double*)sg.y)[i] = (double)((const float*)sg.x)[i]; break;
      case 5: ((double*)sg.y)[i] += ((const double*)sg.x)[i] + (double)((const float*)sg.z)[i]; break;
      case 8: ((double*)sg.y)[i] = ((const double*)sg.x)[i] + float_to_double_bits(((const float*)sg.z)[i]); break;
      default: ((double*)sg.y)[i] = ((const double*)sg.x)[i]; break;
    }
  }
}

__global__ void k_sum_batched(const Segment* __restrict__ seg) {
  __shared__ double red[32];
  const Segment sg = seg[blockIdx.x];
  double s = 0.0;
  for (long long i = threadIdx.x; i < sg.n; i += blockDim.x) s += ((const double*)sg.x)[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0 && sg.n > 0) *(double*)sg.y = t;
}

}  // namespace

void relax_smem_need(const LevelTables& T, int is_double, int* buf, size_t* smem, size_t* region) {
  const bool coarse = T.solver != nullptr;
  const int b = buffer_elems(T, coarse);
  *buf = b;
  *smem = is_double ? smem_bytes<double>(b, T, coarse) : smem_bytes<float>(b, T, coarse);
  *region = T.gather_stage
                ? stage_layout(T.nx, T.p, coarse && T.otf, coarse && T.otf ? T.cf_floats : 0u, T.df, coarse && T.otf && T.band > 0).total
                : 0;
}

namespace {

template <typename R, int CC, int NT>
cudaError_t launch_batched_nt(const LevelTables* d_tabs, const RelaxArgs* d_args, const BatchTile* d_tiles, int ntiles,
                              const int* d_active, int buf, size_t smem, cudaStream_t st) {
  auto kern = k_relax_batched<R, CC, NT>;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ntiles, NT, smem, st>>>(d_tabs, d_args, d_tiles, d_active, buf);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_batched_df(const LevelTables* d_tabs, const RelaxArgs* d_args, const BatchTile* d_tiles, int ntiles,
                              const int* d_active, int buf, size_t smem, cudaStream_t st) {
  const cudaError_t e =
      cudaFuncSetAttribute(k_relax_batched_df<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_relax_batched_df<NT><<<ntiles, NT, smem, st>>>(d_tabs, d_args, d_tiles, d_active, buf);
  return cudaGetLastError();
}

template <int CC>
cudaError_t launch_batched_f32(const LevelTables* d_tabs, const RelaxArgs* d_args, const BatchTile* d_tiles, int ntiles,
                               const int* d_active, int buf, size_t smem, int threads, cudaStream_t st) {
  switch (threads) {
    case 32: return launch_batched_nt<float, CC, 32>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
    case 64: return launch_batched_nt<float, CC, 64>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
    case 128: return launch_batched_nt<float, CC, 128>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
    case 256: return launch_batched_nt<float, CC, 256>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
    default: return launch_batched_nt<float, CC, kSliceThreads>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
  }
}

}  // namespace

cudaError_t launch_relax_batched(const LevelTables* d_tabs, const RelaxArgs* d_args, const BatchTile* d_tiles,
                                 int ntiles, const int* d_active, int is_double, int coarse, int buf, size_t smem,
                                 int threads, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (is_double == 2) {  // FP32-pair level-0 passes
    if (coarse) return cudaErrorInvalidValue;
    switch (threads) {
      case 32: return launch_batched_df<32>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
      case 64: return launch_batched_df<64>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
      case 128: return launch_batched_df<128>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
      case 256: return launch_batched_df<256>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
      default: return launch_batched_df<kSliceThreads>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
    }
  }
  if (is_double) {
    if (coarse) return launch_batched_nt<double, 1, kSliceThreads>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
    return launch_batched_nt<double, 0, kSliceThreads>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, st);
  }
  if (coarse == 2) return launch_batched_f32<2>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, threads, st);
  if (coarse) return launch_batched_f32<1>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, threads, st);
  return launch_batched_f32<0>(d_tabs, d_args, d_tiles, ntiles, d_active, buf, smem, threads, st);
}

cudaError_t launch_sequential_batched(const LevelTables* d_tabs, const SeqArgs* d_args, const BatchTile* d_tiles,
                                      int ntiles, const int* d_active, int is_double, int coarse, int buf,
                                      size_t smem, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
#define MGRIT_BSEQ(RR, CC)                                                                                         \
  {                                                                                                                \
    cudaError_t e = cudaFuncSetAttribute(k_sequential_batched<RR, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                                               \
    if (e != cudaSuccess) return e;                                                                                \
    k_sequential_batched<RR, CC><<<ntiles, kSliceThreads, smem, st>>>(d_tabs, d_args, d_tiles, d_active, buf);      \
    return cudaGetLastError();                                                                                     \
  }
  if (is_double) {
    if (coarse) MGRIT_BSEQ(double, 1)
    MGRIT_BSEQ(double, 0)
  }
  if (coarse == 2) MGRIT_BSEQ(float, 2)
  if (coarse) MGRIT_BSEQ(float, 1)
  MGRIT_BSEQ(float, 0)
#undef MGRIT_BSEQ
}

void launch_axpy_batched(int kind, const Segment* d_seg, int nseg, long long maxn, cudaStream_t st) {
  if (nseg <= 0 || maxn <= 0) return;
  long long blocks = (maxn + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  dim3 grid((unsigned)blocks, (unsigned)nseg);
  k_axpy_batched<<<grid, 256, 0, st>>>(kind, d_seg);
}

void launch_sum_batched(const Segment* d_seg, int nseg, cudaStream_t st) {
  if (nseg <= 0) return;
  k_sum_batched<<<nseg, 256, 0, st>>>(d_seg);
}

cudaError_t launch_gradient_a_1d(const LevelTables& T, const double* s64, const double* ds, const double* C,
                                 const double* mu, int nt, int m, double* partial, cudaStream_t st) {
  const size_t sm = 2 * (size_t)T.nx * sizeof(double) + 64 * sizeof(double);
  const int J = nt / m;
#define MGRIT_LAUNCH_GRAD(PP)                                                                            \
  {                                                                                                      \
    cudaError_t e = cudaFuncSetAttribute(k_gradient_a_1d<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)sm);                                                       \
    if (e != cudaSuccess) return e;                                                                      \
    k_gradient_a_1d<PP><<<J, kSliceThreads, sm, st>>>(T, s64, ds, C, mu, nt, m, partial);                 \
    return cudaGetLastError();                                                                           \
  }
  if (T.p == 1) MGRIT_LAUNCH_GRAD(1)
  if (T.p == 3) MGRIT_LAUNCH_GRAD(3)
  MGRIT_LAUNCH_GRAD(5)
#undef MGRIT_LAUNCH_GRAD
}

unsigned pcr_record_size(int nx, int p) { return pcr_record_floats(nx, p); }
unsigned band_record_size(int nx, int p) { return band_record_floats(nx, p); }
unsigned band_row_size(int nx, int p) { return band_row_floats(nx, p); }

cudaError_t launch_sep_band(const float* sig32, int nt, int nx, int p, int colours, float* rec, float* ind,
                            cudaStream_t st) {
  const int B = (p + 1) / 2, P = nx / kPartRows;
  if (P < 16 || P > 512 || (colours != 8 && colours != 16)) return cudaErrorInvalidValue;
  const int R = (B <= 2 ? 8 : 2) * B;
  const size_t smem = (size_t)(3 * B * B + R * B) * P * sizeof(float);
  const unsigned stride = band_record_floats(nx, p), row = band_row_floats(nx, p);
  cudaError_t e = cudaSuccess;
#define MGRIT_BAND(BB, NCC)                                                                                \
  {                                                                                                        \
    e = cudaFuncSetAttribute(k_sep_band<BB, NCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                        \
    k_sep_band<BB, NCC><<<nt, P, smem, st>>>(sig32, nx, rec, stride, row, ind);                            \
  }
  if (colours == 8) {
    if (B == 1) MGRIT_BAND(1, 8)
    else if (B == 2) MGRIT_BAND(2, 8)
    else MGRIT_BAND(3, 8)
  } else {
    if (B == 1) MGRIT_BAND(1, 16)
    else if (B == 2) MGRIT_BAND(2, 16)
    else MGRIT_BAND(3, 16)
  }
#undef MGRIT_BAND
  return cudaGetLastError();
}

cudaError_t launch_pcr_coef(const float* sig32, int nt, int nx, int p, float* out, cudaStream_t st) {
  const int B = (p + 1) / 2;
  if (B > 2) return cudaErrorInvalidValue;
  const int P = nx / 16;
  const unsigned stride = pcr_record_floats(nx, p);
  const size_t smem = (size_t)3 * B * B * P * sizeof(float);
  const int threads = ((P + 31) / 32) * 32;
  if (B == 1) k_pcr_coef<1, 16><<<nt, threads, smem, st>>>(sig32, nx, out, stride);
  else k_pcr_coef<2, 16><<<nt, threads, smem, st>>>(sig32, nx, out, stride);
  return cudaGetLastError();
}

void launch_axpy_convert(int kind, const void* x, void* y, const void* z, long long n, cudaStream_t st) {
  if (n <= 0) return;
  const int bs = 256;
  k_axpy_convert<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(kind, x, y, z, n);
}

void launch_fill_zero(void* y, long long bytes, cudaStream_t st) { cudaMemsetAsync(y, 0, (size_t)bytes, st); }

}  // namespace mgrit
