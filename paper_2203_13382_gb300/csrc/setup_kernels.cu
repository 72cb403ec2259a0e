// Setup kernels: departure points, backtracking with phi/sigma, gather tables, and the factorisation
// of the periodic banded correction matrices.  All arithmetic here is FP64.
#include <climits>

#include "common.cuh"
#include "df32.cuh"
#include "kernels.h"
#include "physics.cuh"
#include "solver_layout.cuh"

namespace mgrit {

// ------------------------------------------------------------------------------------------------
// K1: fine departure offsets (Sec. 2.1 eq. (depart_ODE); Sec. 4.1 eq. (SL2D_char1-2))
// ------------------------------------------------------------------------------------------------

// sin and cos of a small angle: Taylor polynomials, else sincos.  |t| < 2^-7 (the stage offsets of the
// fine steps): sin to t^5, cos to t^6, truncation below 5e-17 relative; |t| < 1/8: sin to t^9, cos to
// t^10, truncation below 3e-19.
MGRIT_D void small_sincos(double t, double& st, double& ct) {
  const double at = fabs(t);
  if (at < 0.0078125) {
    const double t2 = t * t;
    st = t * (1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120)));
    ct = 1.0 + t2 * (-0.5 + t2 * (1.0 / 24 + t2 * (-1.0 / 720)));
  } else if (at < 0.125) {
    const double t2 = t * t;
    st = t * (1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880)))));
    ct = 1.0 + t2 * (-0.5 + t2 * (1.0 / 24 + t2 * (-1.0 / 720 + t2 * (1.0 / 40320 + t2 * (-1.0 / 3628800)))));
  } else {
    sincos(t, &st, &ct);
  }
}

// Coefficients of the order-R tableau as compile-time constants (the same tableaux as make_tableau).
template <int R>
struct ErkTab {
  static constexpr int S = R == 1 ? 1 : (R == 3 ? 3 : 6);
  static constexpr double a(int s, int j) {
    if (R == 3) return (s == 1 && j == 0) ? 0.5 : (s == 2 && j == 0) ? -1.0 : (s == 2 && j == 1) ? 2.0 : 0.0;
    if (R == 5) {
      constexpr double t[6][6] = {{0, 0, 0, 0, 0, 0},
                                  {0.25, 0, 0, 0, 0, 0},
                                  {0.125, 0.125, 0, 0, 0, 0},
                                  {0, -0.5, 1.0, 0, 0, 0},
                                  {3.0 / 16.0, 0, 0, 9.0 / 16.0, 0, 0},
                                  {-3.0 / 7.0, 2.0 / 7.0, 12.0 / 7.0, -12.0 / 7.0, 8.0 / 7.0, 0}};
      return t[s][j];
    }
    return 0.0;
  }
  static constexpr double b(int s) {
    if (R == 1) return 1.0;
    if (R == 3) return s == 1 ? 2.0 / 3.0 : 1.0 / 6.0;
    constexpr double t[6] = {7.0 / 90.0, 0.0, 32.0 / 90.0, 12.0 / 90.0, 32.0 / 90.0, 7.0 / 90.0};
    return t[s];
  }
  static constexpr double c(int s) {
    if (R == 3) return s == 0 ? 0.0 : (s == 1 ? 0.5 : 1.0);
    if (R == 5) {
      constexpr double t[6] = {0.0, 0.25, 0.25, 0.5, 0.75, 1.0};
      return t[s];
    }
    return 0.0;
  }
};

constexpr int kDepSteps = 16;  // time steps per thread of k_departure_1d

// Arrival node i of the steps n0 .. n0 + kDepSteps - 1 (blockIdx.y): the node's sin / cos of the
// spatial phase are formed once; the spatial factor at a stage point x_i - d is sin / cos(phase - kw d)
// by the angle-addition formula with a small-angle series (d is a fraction of dt), and the time
// factors cos(2 pi t) of the stages are shared by the block.
template <int R>
__global__ void __launch_bounds__(256) k_departure_1d(WaveParams w, int nx, int nt, double xmin, double h,
                                                      double dt, double* __restrict__ s) {
  using Tb = ErkTab<R>;
  constexpr int S = Tb::S;
  // tf[nb][st]: the time factor of stage st of step n0 + nb (kind 3: a cos(2 pi t), else cos(2 pi t))
  __shared__ double tf[kDepSteps][S];
  const int n0 = blockIdx.y * kDepSteps;
  for (int q = threadIdx.x; q < kDepSteps * S; q += blockDim.x) {
    const int nb = q / S, st = q % S;
    const double c = cos(kTwoPi * ((n0 + nb + 1) * dt - Tb::c(st) * dt));
    tf[nb][st] = w.kind == 3 ? w.a * c : c;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const double x = xmin + h * i;
  const double kw = (w.kind == 3) ? kTwoPi * w.k : kTwoPi;  // spatial wavenumber
  double Sx = 0.0, Cx = 1.0;
  if (w.kind >= 2) sincos(kw * x, &Sx, &Cx);
  // stage offsets in units of the phase: kw (x - stage point) = sum_j pa[st][j] k_j; the offset in
  // grid units s = sum_st pb[st] k_st
  double pa[S][S], pb[S];
#pragma unroll
  for (int st = 0; st < S; ++st) {
#pragma unroll
    for (int j = 0; j < S; ++j) pa[st][j] = kw * dt * Tb::a(st, j);
    pb[st] = Tb::b(st) * dt / h;
  }
  const int nend = min(kDepSteps, nt - n0);
  for (int nb = 0; nb < nend; ++nb) {
    double k[S];
#pragma unroll
    for (int st = 0; st < S; ++st) {
      double a;
      if (w.kind == 0) {
        a = w.a;
      } else if (w.kind == 1) {
        a = tf[nb][st];
      } else if (st == 0) {  // the first stage point is the arrival node itself
        if (w.kind == 2) a = tf[nb][0] * Cx;
        else a = 1.0 + tf[nb][0] * Sx;
      } else {
        double ph = 0.0;  // kw (x - stage point)
#pragma unroll
        for (int j = 0; j < st; ++j)
          if (Tb::a(st, j) != 0.0) ph = ph + pa[st][j] * k[j];
        double sth, cth;
        small_sincos(ph, sth, cth);
        if (w.kind == 2) a = tf[nb][st] * (Cx * cth + Sx * sth);  // cos(2 pi t) cos(2 pi (x - d))
        else a = 1.0 + tf[nb][st] * (Sx * cth - Cx * sth);  // 1 + a sin(2 pi k (x - d)) cos(2 pi t)
      }
      k[st] = a;
    }
    double sv = 0.0;
#pragma unroll
    for (int st = 0; st < S; ++st)
      if (Tb::b(st) != 0.0) sv = sv + pb[st] * k[st];
    s[(size_t)(n0 + nb) * nx + i] = sv;
  }
}

// ---- the same departure points in FP32 pairs (FP32-bulk handles, the spatially varying 1D speeds) ----
//
// GB300 runs FP64 at 1/64 of the FP32 rate, and the ERK stages above are FP64-bound.  Here every stage
// runs on the FP32 pipes in FP32 pairs (df32.cuh: Dekker's product, Knuth's TwoSum), about 46 significant
// bits after the rounding of a few dozen operations -- far inside the 1e-11 to which departure offsets are
// checked, and of the order of the FP32-pair level-0 residual these handles use anyway.  FP64 remains
// where a value enters once per node or row: sin / cos of the node's spatial phase, the stage time factors
// and the offset stored.

// a + b, renormalised (TwoSum of the high parts, the low parts added to its error).
MGRIT_D df32 dep_add(df32 a, df32 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return df_norm(s, __fadd_rn(err, __fadd_rn(a.l, b.l)));
}

// a * b renormalised.
MGRIT_D df32 dep_mul(df32 a, df32 b) {
  const df32 p = df_mul(a, b);
  return df_norm(p.h, p.l);
}

// sin t, cos t of a pair |t| < 2^-7: sin t = t (1 + t^2 (-1/6 + t^2/120)) with the t^3 term in pairs, and
// cos t = 1 - t^2/2 + t^4 (1/24 - t^2/720) with t^2/2 in pairs; the parts left in FP32 (t^5/120, t^4/24 and
// beyond) and the truncated terms are below 1e-17.
MGRIT_D void dep_small_sincos(df32 t, df32& st, df32& ct) {
  constexpr float m6h = (float)(-1.0 / 6.0);
  constexpr float m6l = (float)(-1.0 / 6.0 - (double)(float)(-1.0 / 6.0));
  const df32 t2 = dep_mul(t, t);
  const float q = t2.h;
  const df32 c1 = dep_add(df32{m6h, m6l}, df32{__fmul_rn(q, 1.f / 120.f), 0.f});
  st = dep_add(t, dep_mul(t, dep_mul(t2, c1)));
  const float cc = __fmul_rn(__fmul_rn(q, q), __fmaf_rn(q, -1.f / 720.f, 1.f / 24.f));
  ct = dep_add(df32{1.f, 0.f}, dep_add(df32{-0.5f * t2.h, -0.5f * t2.l}, df32{cc, 0.f}));
}

template <int R>
__global__ void __launch_bounds__(256) k_departure_1d_df(WaveParams w, int nx, int nt, double xmin, double h,
                                                         double dt, double* __restrict__ s) {
  using Tb = ErkTab<R>;
  constexpr int S = Tb::S;
  __shared__ float2 tf[kDepSteps][S];  // the stage time factors as pairs (kind 3: a cos(2 pi t))
  const int n0 = blockIdx.y * kDepSteps;
  for (int q = threadIdx.x; q < kDepSteps * S; q += blockDim.x) {
    const int nb = q / S, st = q % S;
    const double c = cos(kTwoPi * ((n0 + nb + 1) * dt - Tb::c(st) * dt));
    const df32 v = df_from_double(w.kind == 3 ? w.a * c : c);
    tf[nb][st] = make_float2(v.h, v.l);
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const double x = xmin + h * i;
  const double kw = (w.kind == 3) ? kTwoPi * w.k : kTwoPi;
  double Sx64, Cx64;
  sincos(kw * x, &Sx64, &Cx64);
  const df32 Sx = df_from_double(Sx64), Cx = df_from_double(Cx64);
  df32 pa[S][S], pb[S];
#pragma unroll
  for (int st = 0; st < S; ++st) {
#pragma unroll
    for (int j = 0; j < S; ++j) pa[st][j] = df_from_double(kw * dt * Tb::a(st, j));
    pb[st] = df_from_double(Tb::b(st) * dt / h);
  }
  const int nend = min(kDepSteps, nt - n0);
  for (int nb = 0; nb < nend; ++nb) {
    df32 k[S];
#pragma unroll
    for (int st = 0; st < S; ++st) {
      const float2 t2 = tf[nb][st];
      const df32 tfp{t2.x, t2.y};
      df32 a;
      if (st == 0) {  // the first stage point is the arrival node itself
        a = w.kind == 2 ? dep_mul(tfp, Cx) : dep_add(df32{1.f, 0.f}, dep_mul(tfp, Sx));
      } else {
        df32 ph{0.f, 0.f};  // kw (x - stage point)
#pragma unroll
        for (int j = 0; j < st; ++j)
          if (Tb::a(st, j) != 0.0) ph = dep_add(ph, dep_mul(pa[st][j], k[j]));
        df32 sth, cth;
        if (fabsf(ph.h) < 0.0078125f) {
          dep_small_sincos(ph, sth, cth);
        } else {  // large phase steps (coarse grids): FP64
          double s64, c64;
          small_sincos(df_to_double(ph), s64, c64);
          sth = df_from_double(s64);
          cth = df_from_double(c64);
        }
        if (w.kind == 2) {  // cos(2 pi t) cos(2 pi (x - d))
          a = dep_mul(tfp, dep_add(dep_mul(Cx, cth), dep_mul(Sx, sth)));
        } else {  // 1 + a sin(2 pi k (x - d)) cos(2 pi t)
          const df32 cs = dep_mul(Cx, sth);
          a = dep_add(df32{1.f, 0.f}, dep_mul(tfp, dep_add(dep_mul(Sx, cth), df32{-cs.h, -cs.l})));
        }
      }
      k[st] = a;
    }
    df32 sv{0.f, 0.f};
#pragma unroll
    for (int st = 0; st < S; ++st)
      if (Tb::b(st) != 0.0) sv = dep_add(sv, dep_mul(pb[st], k[st]));
    s[(size_t)(n0 + nb) * nx + i] = df_to_double(sv);
  }
}

// 2D: arrival node (i, j) of the steps n0 .. n0 + kDepSteps - 1 (blockIdx.y).  The node's sin / cos of
// the spatial phases are formed once; at a stage point (x - dx, y - dy) they follow by angle addition with
// a small-angle series, and the time factors of the stages are shared by the block.
template <int R>
__global__ void __launch_bounds__(256) k_departure_2d(WaveParams w, int nx, int log2nx, int nt, double xmin, double h,
                                                      double dt, double* __restrict__ sx, double* __restrict__ sy) {
  using Tb = ErkTab<R>;
  constexpr int S = Tb::S;
  __shared__ double tc[kDepSteps][S], ts[kDepSteps][S];
  const int n0 = blockIdx.y * kDepSteps;
  for (int q = threadIdx.x; q < kDepSteps * S; q += blockDim.x) {
    const int nb = q / S, st = q % S;
    const double t = (n0 + nb + 1) * dt - Tb::c(st) * dt;
    const double ph = w.kind == 11 ? kTwoPi * t / 3.4 : kTwoPi * t;
    double sn, cs;
    sincos(ph, &sn, &cs);
    tc[nb][st] = cs;
    ts[nb][st] = sn;
  }
  __syncthreads();
  const long long npts = (long long)nx * nx;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  const int i = (int)(pt & (nx - 1)), j = (int)(pt >> log2nx);
  const double x = xmin + h * i, y = xmin + h * j;
  // spatial wavenumber: 2 pi (kind 12) or pi (kind 11, sin^2 / cos^2 of pi x)
  const double kw = w.kind == 11 ? kPi : kTwoPi;
  double Sx = 0.0, Cx = 1.0, Sy = 0.0, Cy = 1.0;
  if (w.kind != 10) {
    sincos(kw * x, &Sx, &Cx);
    sincos(kw * y, &Sy, &Cy);
  }
  const double inv_h = 1.0 / h;
  const int nend = min(kDepSteps, nt - n0);
  for (int nb = 0; nb < nend; ++nb) {
    double kx[S], ky[S];
#pragma unroll
    for (int st = 0; st < S; ++st) {
      double dx = 0.0, dy = 0.0;  // (x, y) - (stage point)
#pragma unroll
      for (int q = 0; q < st; ++q)
        if (Tb::a(st, q) != 0.0) {
          dx = dx + dt * Tb::a(st, q) * kx[q];
          dy = dy + dt * Tb::a(st, q) * ky[q];
        }
      double vx, vy;
      if (w.kind == 10) {
        vx = w.a;
        vy = w.a2;
      } else {
        double sdx = 0.0, cdx = 1.0, sdy = 0.0, cdy = 1.0;
        if (st > 0) {
          small_sincos(kw * dx, sdx, cdx);
          small_sincos(kw * dy, sdy, cdy);
        }
        const double sys = Sy * cdy - Cy * sdy;  // sin(kw (y - dy))
        const double cxs = Cx * cdx + Sx * sdx;  // cos(kw (x - dx))
        if (w.kind == 11) {
          vx = sys * sys * tc[nb][st];
          vy = -cxs * cxs * tc[nb][st];
        } else {
          vx = 1.0 + w.a * sys * tc[nb][st];
          vy = 1.0 + w.a * cxs * ts[nb][st];
        }
      }
      kx[st] = vx;
      ky[st] = vy;
    }
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int st = 0; st < S; ++st)
      if (Tb::b(st) != 0.0) {
        ax = ax + Tb::b(st) * kx[st];
        ay = ay + Tb::b(st) * ky[st];
      }
    const size_t o = (size_t)(n0 + nb) * npts + pt;
    sx[o] = dt * ax * inv_h;
    sy[o] = dt * ay * inv_h;
  }
}

void launch_departure_1d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* s,
                         bool pairs, cudaStream_t st) {
  const int bs = 256;
  dim3 grid((unsigned)((nx + bs - 1) / bs), (unsigned)((nt + kDepSteps - 1) / kDepSteps));
  if (pairs && (w.kind == 2 || w.kind == 3)) {
    if (r == 1) k_departure_1d_df<1><<<grid, bs, 0, st>>>(w, nx, nt, xmin, h, dt, s);
    else if (r == 3) k_departure_1d_df<3><<<grid, bs, 0, st>>>(w, nx, nt, xmin, h, dt, s);
    else k_departure_1d_df<5><<<grid, bs, 0, st>>>(w, nx, nt, xmin, h, dt, s);
    return;
  }
  if (r == 1) k_departure_1d<1><<<grid, bs, 0, st>>>(w, nx, nt, xmin, h, dt, s);
  else if (r == 3) k_departure_1d<3><<<grid, bs, 0, st>>>(w, nx, nt, xmin, h, dt, s);
  else k_departure_1d<5><<<grid, bs, 0, st>>>(w, nx, nt, xmin, h, dt, s);
}

void launch_departure_2d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* sx,
                         double* sy, cudaStream_t st) {
  const long long npts = (long long)nx * nx;
  const int bs = 256;
  int l2 = 0;
  while ((1 << l2) < nx) ++l2;
  dim3 grid((unsigned)((npts + bs - 1) / bs), (unsigned)((nt + kDepSteps - 1) / kDepSteps));
  if (r == 1) k_departure_2d<1><<<grid, bs, 0, st>>>(w, nx, l2, nt, xmin, h, dt, sx, sy);
  else if (r == 3) k_departure_2d<3><<<grid, bs, 0, st>>>(w, nx, l2, nt, xmin, h, dt, sx, sy);
  else k_departure_2d<5><<<grid, bs, 0, st>>>(w, nx, l2, nt, xmin, h, dt, sx, sy);
}

// Per step: range [min, max] of floor(s) over the arrival points (window of the transposed gather).
__global__ void k_floor_range(const double* __restrict__ s, int nx, int2* __restrict__ out) {
  __shared__ int mn[32], mx[32];
  const double* row = s + (size_t)blockIdx.x * nx;
  int lo = INT_MAX, hi = INT_MIN;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = row[i];
    double f = floor(v);
    if (v - f >= 1.0) f += 1.0;
    const int fi = (int)f;
    lo = min(lo, fi);
    hi = max(hi, fi);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    mn[threadIdx.x >> 5] = lo;
    mx[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = min(lo, mn[w]);
      hi = max(hi, mx[w]);
    }
    out[blockIdx.x] = make_int2(lo, hi);
  }
}

void launch_floor_range(const double* s, int nt, int nx, int2* out, cudaStream_t st) {
  k_floor_range<<<nt, 256, 0, st>>>(s, nx, out);
}

// d s / d a by the tangent-linear ERK step (a = the amplitude parameter of the wave speed).
__global__ void k_departure_da_1d(WaveParams w, Tableau T, int nx, double xmin, double h, double dt,
                                  double* __restrict__ ds) {
  const int n = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const double x = xmin + h * i;
  const double t1 = (n + 1) * dt;
  double k[6], dk[6];
  for (int st = 0; st < T.stages; ++st) {
    double xs = x, dxs = 0.0;
    for (int j = 0; j < st; ++j)
      if (T.A[st][j] != 0.0) {
        xs = xs - dt * T.A[st][j] * k[j];
        dxs = dxs - dt * T.A[st][j] * dk[j];
      }
    const double ts = t1 - T.c[st] * dt;
    double da = 0.0, dx = 0.0;
    if (w.kind == 0) {
      da = 1.0;
    } else if (w.kind == 2) {
      dx = -kTwoPi * cos(kTwoPi * ts) * sin(kTwoPi * xs);
    } else if (w.kind == 3) {
      const double ct = cos(kTwoPi * ts);
      da = sin(kTwoPi * w.k * xs) * ct;
      dx = w.a * kTwoPi * w.k * cos(kTwoPi * w.k * xs) * ct;
    }
    k[st] = alpha_1d(w, xs, ts);
    dk[st] = da + dx * dxs;
  }
  double d = 0.0;
  for (int st = 0; st < T.stages; ++st)
    if (T.b[st] != 0.0) d = d + T.b[st] * dk[st];
  ds[(size_t)n * nx + i] = dt * d / h;
}

void launch_departure_da_1d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* ds,
                            cudaStream_t st) {
  const int bs = 256;
  dim3 grid((unsigned)((nx + bs - 1) / bs), (unsigned)nt);
  k_departure_da_1d<<<grid, bs, 0, st>>>(w, make_tableau(r), nx, xmin, h, dt, ds);
}

// Derivatives of the 2D velocity: (dvx/da, dvx/dx, dvx/dy) and (dvy/da, dvy/dx, dvy/dy).  The parameter
// a is the amplitude of kind 12 (both components) and the x speed of kind 10; kind 11 has none.
MGRIT_D void dvelocity_2d(const WaveParams& w, double x, double y, double t, double (&gx)[3], double (&gy)[3]) {
  gx[0] = gx[1] = gx[2] = gy[0] = gy[1] = gy[2] = 0.0;
  if (w.kind == 10) {
    gx[0] = 1.0;
  } else if (w.kind == 11) {
    const double ct = cos(kTwoPi * t / 3.4);
    gx[2] = 2.0 * kPi * sin(kPi * y) * cos(kPi * y) * ct;
    gy[1] = 2.0 * kPi * cos(kPi * x) * sin(kPi * x) * ct;
  } else {
    const double ct = cos(kTwoPi * t), st = sin(kTwoPi * t);
    gx[0] = sin(kTwoPi * y) * ct;
    gx[2] = w.a * kTwoPi * cos(kTwoPi * y) * ct;
    gy[0] = cos(kTwoPi * x) * st;
    gy[1] = -w.a * kTwoPi * sin(kTwoPi * x) * st;
  }
}

// (d sx / d a, d sy / d a): the stages of erk_displacement_2d differentiated (tangent-linear ERK).
__global__ void k_departure_da_2d(WaveParams w, Tableau T, int nx, int nt, double xmin, double h, double dt,
                                  double* __restrict__ dsx, double* __restrict__ dsy) {
  const long long npts = (long long)nx * nx;
  const int n = blockIdx.y;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  int i, j;
  split_pow2(pt, nx, i, j);
  const double x = xmin + h * i, y = xmin + h * j;
  const double t1 = (n + 1) * dt;
  double kx[6], ky[6], dkx[6], dky[6];
  for (int st = 0; st < T.stages; ++st) {
    double xs = x, ys = y, dxs = 0.0, dys = 0.0;
    for (int q = 0; q < st; ++q)
      if (T.A[st][q] != 0.0) {
        xs = xs - dt * T.A[st][q] * kx[q];
        ys = ys - dt * T.A[st][q] * ky[q];
        dxs = dxs - dt * T.A[st][q] * dkx[q];
        dys = dys - dt * T.A[st][q] * dky[q];
      }
    const double ts = t1 - T.c[st] * dt;
    double gx[3], gy[3];
    velocity_2d(w, xs, ys, ts, kx[st], ky[st]);
    dvelocity_2d(w, xs, ys, ts, gx, gy);
    dkx[st] = gx[0] + gx[1] * dxs + gx[2] * dys;
    dky[st] = gy[0] + gy[1] * dxs + gy[2] * dys;
  }
  double ax = 0.0, ay = 0.0;
  for (int st = 0; st < T.stages; ++st)
    if (T.b[st] != 0.0) {
      ax = ax + T.b[st] * dkx[st];
      ay = ay + T.b[st] * dky[st];
    }
  const size_t o = (size_t)n * npts + pt;
  dsx[o] = dt * ax / h;
  dsy[o] = dt * ay / h;
}

void launch_departure_da_2d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* dsx,
                            double* dsy, cudaStream_t st) {
  const int bs = 256;
  const long long npts = (long long)nx * nx;
  dim3 grid((unsigned)((npts + bs - 1) / bs), (unsigned)nt);
  k_departure_da_2d<<<grid, bs, 0, st>>>(w, make_tableau(r), nx, nt, xmin, h, dt, dsx, dsy);
}

// ------------------------------------------------------------------------------------------------
// K2: backtracking (Sec. 3.3.1 eq. (coarse_depart_interp); Sec. SM6) and phi / sigma (eq. (nu_p_def))
// ------------------------------------------------------------------------------------------------

// floor(s) and eps = s - floor(s) as an FP32 pair (eh = eps rounded to nearest-even at 24 bits, el = the
// rest rounded the same way), from the bit pattern of s with integer operations only (GB300 runs FP64,
// conversions included, at 1/64 of the FP32 rate).  With E the unbiased exponent of s and m its 53-bit
// significand, eps = G 2^-k: for 1 <= |s| < 2^30 the k = 52 - E fraction bits of m (complemented to
// 2^k when s < 0), for 0 < s < 1 all of m with k = 52 - E.  Then eh takes the top 24 bits of G with the
// rounding carry and el the signed remainder.  Every case the function accepts gives the values of the
// FP64 route (eps is exact in FP64 there); it returns false for the rest (-1 < s < 0, |s| >= 2^30,
// 0 < eps < 2^-74), which take the FP64 route.
MGRIT_D bool split_offset_int(double s, int& fl, float& eh, float& el) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  const int e = (int)((b >> 52) & 0x7ff);
  const bool neg = (b >> 63) != 0;
  if (e == 0) {
    if (neg) return false;
    fl = 0;  // +0 or a positive subnormal: eps below 2^-1022, taken as 0
    eh = el = 0.f;
    return true;
  }
  const int E = e - 1023;
  if (E >= 30) return false;
  const unsigned long long m = (b & 0xfffffffffffffULL) | (1ULL << 52);
  const int k = 52 - E;
  unsigned long long G;
  if (E >= 0) {
    const long long I = (long long)(m >> k);
    G = m & ((1ULL << k) - 1);
    if (!neg) {
      fl = (int)I;
    } else if (G) {
      fl = -(int)I - 1;
      G = (1ULL << k) - G;
    } else {
      fl = -(int)I;
    }
  } else {
    if (neg) return false;
    fl = 0;
    G = m;
  }
  if (G == 0) {
    eh = el = 0.f;
    return true;
  }
  const int lead = 63 - __clzll((long long)G);
  int ex = lead - k;  // eps in [2^ex, 2^(ex+1))
  if (ex < -74) return false;
  unsigned hm;
  int r = 0;  // G = hm 2^d + r
  int d = lead - 23;
  if (d <= 0) {
    hm = (unsigned)(G << (-d));
    d = 0;
  } else {
    hm = (unsigned)(G >> d);
    const unsigned long long rem = G & ((1ULL << d) - 1);
    const unsigned long long half = 1ULL << (d - 1);
    long long rr = (long long)rem;
    if (rem > half || (rem == half && (hm & 1u))) {
      ++hm;
      rr -= 1LL << d;
    }
    r = (int)rr;
    if (hm == (1u << 24)) {
      hm >>= 1;
      ++ex;
    }
  }
  eh = __uint_as_float(((unsigned)(ex + 127) << 23) | (hm & 0x7fffffu));
  // el = r 2^-k: r has at most 29 bits, so its conversion rounds as the FP64 route does, and 2^-k is a
  // normal FP32 power of two (k = lead - ex <= 52 + 74)
  el = r == 0 ? 0.f : __fmul_rn(__int2float_rn(r), __uint_as_float((unsigned)(127 - k) << 23));
  return true;
}

// eps = s - floor(s) in [0, 1) (east-neighbour distance, eq. (depart_decompose)).
MGRIT_D double frac_eps(double s) {
  double e = s - floor(s);
  if (e >= 1.0) e -= 1.0;
  return e;
}

// prod_{q=-(p+1)/2}^{(p-1)/2} (q + z) = (p+1)! f_{p+1}(z)  (eq. (fpoly_def) without its constant factor).
// prod_{q=-L}^{L-1} (q + z), L = (P+1)/2, evaluated as its monic polynomial in z by Horner's rule
// (integer coefficients, exact; P + 1 multiply-adds instead of P + 1 adds and P multiplies).
template <int P>
struct FProdCoef {
  double c[P + 2];  // c[d]: coefficient of z^d
  constexpr FProdCoef() : c{} {
    constexpr int L = (P + 1) / 2;
    c[0] = 1.0;
    int deg = 0;
    for (int q = -L; q <= L - 1; ++q) {  // multiply by (z + q)
      for (int d = deg + 1; d >= 1; --d) c[d] = c[d - 1] + q * c[d];
      c[0] = q * c[0];
      ++deg;
    }
  }
};

template <int P>
MGRIT_D double f_prod(double z) {
  constexpr FProdCoef<P> k{};
  double out = 1.0;
#pragma unroll
  for (int d = P; d >= 0; --d) out = out * z + k.c[d];
  return out;
}

// f_prod of an FP32 pair z (about 44 significant bits): Horner's rule on the integer coefficients with
// pair products (Dekker) and the constant added by TwoSum, renormalised every step (df32.cuh).
template <int P>
MGRIT_D df32 f_prod_df(df32 z) {
  constexpr FProdCoef<P> k{};
  df32 out{1.f, 0.f};
#pragma unroll
  for (int d = P; d >= 0; --d) {
    const df32 t = df_mul(out, z);
    const float c = (float)k.c[d];
    const float s = __fadd_rn(t.h, c);
    const float bb = __fsub_rn(s, t.h);
    const float err = __fadd_rn(__fsub_rn(t.h, __fsub_rn(s, bb)), __fsub_rn(c, bb));
    out = df_norm(s, __fadd_rn(err, t.l));
  }
  return out;
}

// s = fl + eps with eps as an FP32 pair: the integer route where it applies, else FP64.
MGRIT_D void offset_parts(double s, int& fl, df32& eps) {
  float eh, el;
  if (split_offset_int(s, fl, eh, el)) {
    eps = df32{eh, el};
    return;
  }
  double f = floor(s), e = s - f;
  if (e >= 1.0) {
    e -= 1.0;
    f += 1.0;
  }
  fl = (int)f;
  eps = df_from_double(e);
}

// a - e for an integer a (|a| < 2^24) and a pair 0 <= e < 1, renormalised.
MGRIT_D df32 int_minus_pair(int a, df32 e) {
  const float c = (float)a;
  const float s = __fsub_rn(c, e.h);
  const float bb = __fsub_rn(s, c);
  const float err = __fsub_rn(__fsub_rn(c, __fsub_rn(s, bb)), __fadd_rn(e.h, bb));
  return df_norm(s, __fsub_rn(err, e.l));
}

// One coarse step row n (blockIdx.y) of arrival nodes i.  pairs (FP32-bulk handles): the composition of
// the fine maps and the sum of f over the m fine steps are formed in FP32 pairs on the FP32 pipes, each
// fine offset split into its integer floor and its eps pair by integer operations (GB300 runs FP64 at
// 1/64 of the FP32 rate); the coarse offset keeps about 46 bits (1e-11 of a 650-cell offset on the
// deepest level of the 4096 x 16384 workload).  Otherwise FP64 throughout.  eh_prev / el_prev (or null):
// the fine level's eps pair rows where that level keeps them (level 0 of the FP32-bulk mode).
template <int P>
__global__ void k_backtrack_1d(const double* __restrict__ s_prev, const double* __restrict__ sig_prev,
                               const float* __restrict__ eh_prev, const float* __restrict__ el_prev, int pairs,
                               int m, int nx, double* __restrict__ s_out, double* __restrict__ sig_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const int n = blockIdx.y;
  const size_t base = (size_t)m * n * nx;
  // position of the coarse characteristic relative to x_i in grid units; c^{(m-1)} = f^{(m-1)}
  double sc;
  if (pairs) {
    int fl;
    df32 e;
    offset_parts(s_prev[base + (size_t)(m - 1) * nx + i], fl, e);
    df32 c = int_minus_pair(-fl, e);  // -(fl + eps)
    for (int k = m - 2; k >= 0; --k) {
      const double* row = s_prev + base + (size_t)k * nx;
      // east node of c (the node itself if c lies on one): ceil of the high part unless c sits just above
      // an integer high part
      float ce = ceilf(c.h);
      if (ce == c.h && c.l > 0.f) ce += 1.f;
      const int xE = (int)ce;
      const int E = i + xE;
      int fE_i, fW_i;
      df32 eE, eW;
      offset_parts(row[wrap_pow2(E, nx)], fE_i, eE);
      offset_parts(row[wrap_pow2(E - 1, nx)], fW_i, eW);
      const df32 fE = int_minus_pair(xE - fE_i, eE);      // xE - s[E]
      const df32 fW = int_minus_pair(xE - 1 - fW_i, eW);  // (xE - 1) - s[E - 1]
      const df32 slope = dep_add(fE, df32{-fW.h, -fW.l});
      const df32 t = dep_add(c, df32{-ce, 0.f});           // c - xE
      c = dep_add(dep_mul(slope, t), fE);
    }
    sc = -df_to_double(c);
  } else {
    double c = -s_prev[base + (size_t)(m - 1) * nx + i];
    for (int k = m - 2; k >= 0; --k) {
      const double* row = s_prev + base + (size_t)k * nx;
      const double xE = ceil(c);  // east node of c (the node itself if c lies on one)
      const int E = i + (int)xE;
      const double fE = xE - row[wrap_pow2(E, nx)];
      const double fW = (xE - 1.0) - row[wrap_pow2(E - 1, nx)];
      c = (fE - fW) * (c - xE) + fE;
    }
    sc = -c;
  }
  const size_t idx = (size_t)n * nx + i;
  s_out[idx] = sc;
  double ff = 0.0, gs = 0.0;
  if (eh_prev || pairs) {
    float fh = 0.f, fq = 0.f;
    for (int k = 0; k < m; ++k) {
      const size_t q = base + (size_t)k * nx + i;
      df32 e;
      if (eh_prev) {
        e = df32{eh_prev[q], el_prev[q]};
      } else {
        int fl;
        offset_parts(s_prev[q], fl, e);
      }
      df_acc(fh, fq, f_prod_df<P>(e));
    }
    ff = (double)fh + (double)fq;
  } else {
    for (int k = 0; k < m; ++k) ff += f_prod<P>(frac_eps(s_prev[base + (size_t)k * nx + i]));
  }
  if (sig_prev)
    for (int k = 0; k < m; ++k) gs += sig_prev[base + (size_t)k * nx + i];
  double inv_fact = 1.0;
#pragma unroll
  for (int b = 2; b <= P + 1; ++b) inv_fact /= b;
  const double phi = ((P + 1) & 1 ? -1.0 : 1.0) * (f_prod<P>(frac_eps(sc)) - ff) * inv_fact;
  sig_out[idx] = sig_prev ? gs + phi : phi;
}

void launch_backtrack_1d(const double* s_prev, const double* sigma_prev, const float* eh_prev, const float* el_prev,
                         bool pairs, int m, int ntc, int nx, int p, double* s_out, double* sigma_out,
                         cudaStream_t st) {
  const int bs = 256;
  for (int r0 = 0; r0 < ntc; r0 += 65535) {
    const int rows = min(65535, ntc - r0);
    dim3 g((unsigned)((nx + bs - 1) / bs), (unsigned)rows);
    const double* sp = s_prev + (size_t)m * r0 * nx;
    const double* gp = sigma_prev ? sigma_prev + (size_t)m * r0 * nx : nullptr;
    const float* eh = (eh_prev && el_prev) ? eh_prev + (size_t)m * r0 * nx : nullptr;
    const float* el = (eh_prev && el_prev) ? el_prev + (size_t)m * r0 * nx : nullptr;
    double* so = s_out + (size_t)r0 * nx;
    double* go = sigma_out + (size_t)r0 * nx;
    if (p == 1) k_backtrack_1d<1><<<g, bs, 0, st>>>(sp, gp, eh, el, pairs ? 1 : 0, m, nx, so, go);
    else if (p == 3) k_backtrack_1d<3><<<g, bs, 0, st>>>(sp, gp, eh, el, pairs ? 1 : 0, m, nx, so, go);
    else k_backtrack_1d<5><<<g, bs, 0, st>>>(sp, gp, eh, el, pairs ? 1 : 0, m, nx, so, go);
  }
}

// Bilinear fit p2d of Sec. SM6 in grid units relative to the arrival node.
MGRIT_D double p2d(double x, double y, double xE, double yN, double rNE, double rNW, double rSE, double rSW) {
  const double pN = (rNE - rNW) * (x - xE) + rNE;
  const double pS = (rSE - rSW) * (x - xE) + rSE;
  return (pN - pS) * (y - yN) + pN;
}

template <int P>
__global__ void k_backtrack_2d(const double* __restrict__ sx_prev, const double* __restrict__ sy_prev,
                               const double* __restrict__ gx_prev, const double* __restrict__ gy_prev, int m, int nx,
                               int log2nx, double* __restrict__ sx_out, double* __restrict__ sy_out,
                               double* __restrict__ gx_out, double* __restrict__ gy_out) {
  const long long npts = (long long)nx * nx;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  const int n = blockIdx.y;
  const int i = (int)(pt & (nx - 1)), j = (int)(pt >> log2nx);
  const size_t base = (size_t)m * n * npts;
  double c = -sx_prev[base + (size_t)(m - 1) * npts + pt];
  double d = -sy_prev[base + (size_t)(m - 1) * npts + pt];
  for (int k = m - 2; k >= 0; --k) {
    const double* kx = sx_prev + base + (size_t)k * npts;
    const double* ky = sy_prev + base + (size_t)k * npts;
    const double xE = ceil(c), yN = ceil(d);
    const int E = wrap_pow2(i + (int)xE, nx), W = wrap_pow2(i + (int)xE - 1, nx);
    const int N = wrap_pow2(j + (int)yN, nx), S = wrap_pow2(j + (int)yN - 1, nx);
    const double xW = xE - 1.0, yS = yN - 1.0;
    const size_t NE = ((size_t)N << log2nx) + E, NW = ((size_t)N << log2nx) + W;
    const size_t SE = ((size_t)S << log2nx) + E, SW = ((size_t)S << log2nx) + W;
    const double cx = p2d(c, d, xE, yN, xE - kx[NE], xW - kx[NW], xE - kx[SE], xW - kx[SW]);
    const double cy = p2d(c, d, xE, yN, yN - ky[NE], yN - ky[NW], yS - ky[SE], yS - ky[SW]);
    c = cx;
    d = cy;
  }
  const size_t idx = (size_t)n * npts + pt;
  sx_out[idx] = -c;
  sy_out[idx] = -d;
  double fx = 0.0, fy = 0.0, sgx = 0.0, sgy = 0.0;
  for (int k = 0; k < m; ++k) {
    const size_t q = base + (size_t)k * npts + pt;
    fx += f_prod<P>(frac_eps(sx_prev[q]));
    fy += f_prod<P>(frac_eps(sy_prev[q]));
    if (gx_prev) {
      sgx += gx_prev[q];
      sgy += gy_prev[q];
    }
  }
  double inv_fact = 1.0;
#pragma unroll
  for (int b = 2; b <= P + 1; ++b) inv_fact /= b;
  const double sgn = ((P + 1) & 1) ? -1.0 : 1.0;
  const double phx = sgn * (f_prod<P>(frac_eps(-c)) - fx) * inv_fact;
  const double phy = sgn * (f_prod<P>(frac_eps(-d)) - fy) * inv_fact;
  gx_out[idx] = gx_prev ? sgx + phx : phx;
  gy_out[idx] = gy_prev ? sgy + phy : phy;
}

void launch_backtrack_2d(const double* sx_prev, const double* sy_prev, const double* gx_prev, const double* gy_prev,
                         int m, int ntc, int nx, int p, double* sx_out, double* sy_out, double* gx_out, double* gy_out,
                         cudaStream_t st) {
  const long long npts = (long long)nx * nx;
  const int bs = 256;
  int l2 = 0;
  while ((1 << l2) < nx) ++l2;
  dim3 g((unsigned)((npts + bs - 1) / bs), (unsigned)ntc);
  if (p == 1)
    k_backtrack_2d<1><<<g, bs, 0, st>>>(sx_prev, sy_prev, gx_prev, gy_prev, m, nx, l2, sx_out, sy_out, gx_out, gy_out);
  else if (p == 3)
    k_backtrack_2d<3><<<g, bs, 0, st>>>(sx_prev, sy_prev, gx_prev, gy_prev, m, nx, l2, sx_out, sy_out, gx_out, gy_out);
  else
    k_backtrack_2d<5><<<g, bs, 0, st>>>(sx_prev, sy_prev, gx_prev, gy_prev, m, nx, l2, sx_out, sy_out, gx_out, gy_out);
}

// ------------------------------------------------------------------------------------------------
// Gather tables
// ------------------------------------------------------------------------------------------------

// One step row (blockIdx.y) of one level: shift, and the FP64 weights and / or the FP32 distance.
template <int P>
__global__ void k_build_tables(const double* __restrict__ s, int nx, int npts_row, uint16_t* __restrict__ shift,
                               double* __restrict__ w64, float* __restrict__ eps32, float* __restrict__ eps_lo) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts_row) return;
  const size_t row = blockIdx.y, idx = row * npts_row + pt;
  const double sv = s[idx];
  constexpr int L = (P + 1) / 2;
  if (!w64) {  // FP32 tables: floor and the eps pair by integer operations where they apply
    int fl;
    float eh, el;
    if (split_offset_int(sv, fl, eh, el)) {
      shift[idx] = (uint16_t)((-fl - L) & (nx - 1));
      eps32[idx] = eh;
      if (eps_lo) eps_lo[idx] = el;
      return;
    }
  }
  double fl = floor(sv);
  double eps = sv - fl;
  if (eps >= 1.0) {
    eps -= 1.0;
    fl += 1.0;
  }
  // first stencil node E - L with E = i - floor(s); stored as an offset from i, modulo nx (a power of two)
  const int fli = (int)fl;
  shift[idx] = (uint16_t)((-fli - L) & (nx - 1));
  if (eps32) eps32[idx] = (float)eps;
  if (eps_lo) eps_lo[idx] = (float)(eps - (double)(float)eps);
  if (w64) {
    double w[P + 1];
    lagrange_weights<P, double>(eps, w);
#pragma unroll
    for (int a = 0; a <= P; ++a) w64[(row * (P + 1) + a) * npts_row + pt] = w[a];
  }
}

void launch_build_tables(const double* s, int nt, int nx, int npts_row, int p, uint16_t* shift, double* w64,
                         float* eps32, float* eps_lo, cudaStream_t st) {
  const int bs = 256;
  // rows in chunks of 65535 (grid y limit)
  for (int r0 = 0; r0 < nt; r0 += 65535) {
    const int rows = min(65535, nt - r0);
    const size_t o = (size_t)r0 * npts_row;
    dim3 g((unsigned)((npts_row + bs - 1) / bs), (unsigned)rows);
    double* w = w64 ? w64 + o * (p + 1) : nullptr;
    float* e = eps32 ? eps32 + o : nullptr;
    float* el = eps_lo ? eps_lo + o : nullptr;
    if (p == 1) k_build_tables<1><<<g, bs, 0, st>>>(s + o, nx, npts_row, shift + o, w, e, el);
    else if (p == 3) k_build_tables<3><<<g, bs, 0, st>>>(s + o, nx, npts_row, shift + o, w, e, el);
    else k_build_tables<5><<<g, bs, 0, st>>>(s + o, nx, npts_row, shift + o, w, e, el);
  }
}

// ------------------------------------------------------------------------------------------------
// K3: factorisation of M = I - diag(sigma) D_{p+1} for every step of a level (eq. (Bp_def),
// (Phi_multilevel)); layout and algorithm in solver_layout.cuh.  FP64 arithmetic, stored as R.
// ------------------------------------------------------------------------------------------------

MGRIT_HD double dstencil(int b, int j) {
  // coefficient of the centred stencil (delta^2)^b at offset j: (-1)^{b+j} C(2b, b+j)
  if (j < -b || j > b) return 0.0;
  double c = 1.0;
  const int n = 2 * b, k = b + j;
  for (int t = 1; t <= k; ++t) c = c * (n - k + t) / t;
  return ((b + j) & 1) ? -c : c;
}

size_t solver_reals(int nx, int p) { return solver_geom(nx, p).total; }

// In-place inverse of a B x B matrix (row-major) by Gauss-Jordan with partial pivoting; false if singular.
template <int B>
__device__ bool small_inverse(double (&A)[B][B]) {
  int perm[B];
  for (int kk = 0; kk < B; ++kk) {
    int pr = kk;
    for (int r = kk + 1; r < B; ++r)
      if (fabs(A[r][kk]) > fabs(A[pr][kk])) pr = r;
    perm[kk] = pr;
    if (!(fabs(A[pr][kk]) > 1e-300)) return false;
    if (pr != kk)
      for (int c = 0; c < B; ++c) {
        const double t = A[kk][c];
        A[kk][c] = A[pr][c];
        A[pr][c] = t;
      }
    const double pv = A[kk][kk];
    A[kk][kk] = 1.0;
    for (int c = 0; c < B; ++c) A[kk][c] /= pv;
    for (int r = 0; r < B; ++r) {
      if (r == kk) continue;
      const double f = A[r][kk];
      A[r][kk] = 0.0;
      for (int c = 0; c < B; ++c) A[r][c] -= f * A[kk][c];
    }
  }
  for (int kk = B - 1; kk >= 0; --kk)
    if (perm[kk] != kk)
      for (int r = 0; r < B; ++r) {
        const double t = A[r][kk];
        A[r][kk] = A[r][perm[kk]];
        A[r][perm[kk]] = t;
      }
  return true;
}

template <int B>
__device__ void mat_mul(const double (&X)[B][B], const double (&Y)[B][B], double (&Z)[B][B]) {
  for (int a = 0; a < B; ++a)
    for (int c = 0; c < B; ++c) {
      double v = 0.0;
      for (int e = 0; e < B; ++e) v += X[a][e] * Y[e][c];
      Z[a][c] = v;
    }
}

// One CTA per step, one thread per partition k < P.
// TRANS: factorise M^T = I - D_{p+1} diag(sigma) instead (entry (row, row+off) uses sigma[row+off]).
template <int B, typename R, bool TRANS>
__global__ void __launch_bounds__(512) k_factor_1d(const double* __restrict__ sigma_all, int nx, R* __restrict__ out_all, size_t stride,
                            int* flag) {
  constexpr int Q = kPartRows - B;
  const SolverGeom G = solver_geom(nx, 2 * B - 1);
  const int P = G.P;
  const double* sigma = sigma_all + (size_t)blockIdx.x * nx;
  R* out = out_all + (size_t)blockIdx.x * stride;
  extern __shared__ double sh[];  // exchange: 3 blocks of B x B per partition
  const int k = threadIdx.x;
  const bool active = k < P;
  const int g0 = k * kPartRows;
  auto Mval = [&](int row, int off) -> double {  // M[row, row + off] (or M^T), |off| <= B
    const int src = TRANS ? row + off : row;
    const int rr = ((src % nx) + nx) % nx;
    return (off == 0 ? 1.0 : 0.0) - sigma[rr] * dstencil(B, off);
  };
  double Lb[B][B] = {}, Db[B][B] = {}, Ub[B][B] = {};  // ctail / Mss / chead, then the Schur blocks
  double Vh[B][B] = {}, Wh[B][B] = {};                  // head rows of the spikes
  bool ok = true;
  if (active) {
    // 1) banded LU of the interior block (rows g0 + B + r)
    double l[Q][B], U[Q][B + 1];
    for (int r = 0; r < Q; ++r) {
      double a[2 * B + 1];
      for (int c = -B; c <= B; ++c) a[c + B] = (r + c >= 0 && r + c < Q) ? Mval(g0 + B + r, c) : 0.0;
      for (int t = B; t >= 1; --t) {
        if (r - t < 0) {
          l[r][t - 1] = 0.0;
          continue;
        }
        const double lt = a[B - t] / U[r - t][0];
        l[r][t - 1] = lt;
        for (int c = 1; c <= B; ++c) {
          const int col = -t + c;
          if (col <= B) a[col + B] -= lt * U[r - t][c];
        }
      }
      if (!(fabs(a[B]) > 1e-13)) ok = false;
      for (int c = 0; c <= B; ++c) U[r][c] = a[B + c];
    }
    auto solve = [&](double (&x)[Q]) {
      for (int r = 0; r < Q; ++r)
        for (int t = 1; t <= B; ++t)
          if (r - t >= 0) x[r] -= l[r][t - 1] * x[r - t];
      for (int r = Q - 1; r >= 0; --r) {
        for (int t = 1; t <= B; ++t)
          if (r + t < Q) x[r] -= U[r][t] * x[r + t];
        x[r] /= U[r][0];
      }
    };
    // 2) spikes V = A^{-1} M[I_k, S_k], W = A^{-1} M[I_k, S_{k+1}]
    double V[Q][B], W[Q][B];
    for (int c = 0; c < B; ++c) {
      double xv[Q], xw[Q];
      for (int r = 0; r < Q; ++r) {
        const int ov = c - B - r;  // column g0 + c of S_k
        const int ow = Q - r + c;  // column g0 + 8 + c of S_{k+1}
        xv[r] = (ov >= -B) ? Mval(g0 + B + r, ov) : 0.0;
        xw[r] = (ow <= B) ? Mval(g0 + B + r, ow) : 0.0;
      }
      solve(xv);
      solve(xw);
      for (int r = 0; r < Q; ++r) {
        V[r][c] = xv[r];
        W[r][c] = xw[r];
      }
    }
    // 3) couplings of the separator rows
    for (int a = 0; a < B; ++a)
      for (int c = 0; c < B; ++c) {
        Lb[a][c] = (c >= a) ? Mval(g0 + a, c - B - a) : 0.0;  // ctail
        Ub[a][c] = (c <= a) ? Mval(g0 + a, B + c - a) : 0.0;  // chead
        Db[a][c] = Mval(g0 + a, c - a);                       // M[S_k, S_k]
        Vh[a][c] = V[a][c];
        Wh[a][c] = W[a][c];
      }
    for (int r = 0; r < Q; ++r) {
      for (int t = 0; t < B; ++t) out[(size_t)rec_lu(B, r, t) * P + k] = (R)l[r][t];
      out[(size_t)rec_lu(B, r, B) * P + k] = (R)(1.0 / U[r][0]);
      for (int t = 1; t <= B; ++t) out[(size_t)rec_lu(B, r, B + t) * P + k] = (R)U[r][t];
      for (int c = 0; c < B; ++c) {
        out[(size_t)rec_v(B, Q, r, c) * P + k] = (R)V[r][c];
        out[(size_t)rec_w(B, Q, r, c) * P + k] = (R)W[r][c];
      }
    }
    for (int a = 0; a < B; ++a)
      for (int c = 0; c < B; ++c) {
        out[(size_t)rec_ct(B, Q, a, c) * P + k] = (R)Lb[a][c];
        out[(size_t)rec_ch(B, Q, a, c) * P + k] = (R)Ub[a][c];
        // tail rows of V and W go to partition k + 1
        sh[((size_t)k * 2 + 0) * B * B + a * B + c] = V[Q - B + a][c];
        sh[((size_t)k * 2 + 1) * B * B + a * B + c] = W[Q - B + a][c];
      }
  }
  __syncthreads();
  if (active) {
    // 4) Schur complement blocks: L_k (x_{S_{k-1}}), D_k (x_{S_k}), U_k (x_{S_{k+1}})
    const int km = (k + P - 1) % P;
    double Ln[B][B], Dn[B][B], Un[B][B];
    for (int a = 0; a < B; ++a)
      for (int c = 0; c < B; ++c) {
        double lv = 0.0, dv = Db[a][c], uv = 0.0;
        for (int c2 = 0; c2 < B; ++c2) {
          const double vt = sh[((size_t)km * 2 + 0) * B * B + c2 * B + c];
          const double wt = sh[((size_t)km * 2 + 1) * B * B + c2 * B + c];
          lv -= Lb[a][c2] * vt;
          dv -= Lb[a][c2] * wt;
          dv -= Ub[a][c2] * Vh[c2][c];
          uv -= Ub[a][c2] * Wh[c2][c];
        }
        Ln[a][c] = lv;
        Dn[a][c] = dv;
        Un[a][c] = uv;
      }
    for (int a = 0; a < B; ++a)
      for (int c = 0; c < B; ++c) {
        Lb[a][c] = Ln[a][c];
        Db[a][c] = Dn[a][c];
        Ub[a][c] = Un[a][c];
      }
  }
  __syncthreads();
  // 5) block PCR factorisation
  for (int t = 0; t < G.T; ++t) {
    const int d = 1 << t;
    if (active)
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) {
          sh[((size_t)k * 3 + 0) * B * B + a * B + c] = Lb[a][c];
          sh[((size_t)k * 3 + 1) * B * B + a * B + c] = Db[a][c];
          sh[((size_t)k * 3 + 2) * B * B + a * B + c] = Ub[a][c];
        }
    __syncthreads();
    double Lm[B][B], Dm[B][B], Um[B][B], Lp[B][B], Dp[B][B], Up[B][B];
    if (active) {
      const int km = ((k - d) % P + P) % P, kp = (k + d) % P;
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) {
          Lm[a][c] = sh[((size_t)km * 3 + 0) * B * B + a * B + c];
          Dm[a][c] = sh[((size_t)km * 3 + 1) * B * B + a * B + c];
          Um[a][c] = sh[((size_t)km * 3 + 2) * B * B + a * B + c];
          Lp[a][c] = sh[((size_t)kp * 3 + 0) * B * B + a * B + c];
          Dp[a][c] = sh[((size_t)kp * 3 + 1) * B * B + a * B + c];
          Up[a][c] = sh[((size_t)kp * 3 + 2) * B * B + a * B + c];
        }
    }
    __syncthreads();
    if (active) {
      ok = ok && small_inverse<B>(Dm) && small_inverse<B>(Dp);
      double al[B][B], ga[B][B], t1[B][B];
      mat_mul<B>(Lb, Dm, al);
      mat_mul<B>(Ub, Dp, ga);
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) {
          al[a][c] = -al[a][c];
          ga[a][c] = -ga[a][c];
        }
      R* pc = out + G.pcr_off + (size_t)t * 2 * B * B * P;
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) {
          pc[(size_t)(a * B + c) * P + k] = (R)al[a][c];
          pc[(size_t)(B * B + a * B + c) * P + k] = (R)ga[a][c];
        }
      double nD[B][B];
      mat_mul<B>(al, Um, t1);
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) nD[a][c] = Db[a][c] + t1[a][c];
      mat_mul<B>(ga, Lp, t1);
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) nD[a][c] += t1[a][c];
      mat_mul<B>(al, Lm, t1);
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) Lb[a][c] = t1[a][c];
      mat_mul<B>(ga, Up, t1);
      for (int a = 0; a < B; ++a)
        for (int c = 0; c < B; ++c) {
          Ub[a][c] = t1[a][c];
          Db[a][c] = nD[a][c];
        }
    }
  }
  if (active) {
    double F[B][B];
    for (int a = 0; a < B; ++a)
      for (int c = 0; c < B; ++c) F[a][c] = Lb[a][c] + Db[a][c] + Ub[a][c];
    ok = ok && small_inverse<B>(F);
    for (int a = 0; a < B; ++a)
      for (int c = 0; c < B; ++c) out[G.fin_off + (size_t)(a * B + c) * P + k] = (R)F[a][c];
    if (!ok) atomicExch(flag, 1);
  }
}

int launch_factor_1d(const double* sigma, int nt, int nx, int p, double* out, int* flag, cudaStream_t st,
                     int transpose) {
  const SolverGeom G = solver_geom(nx, p);
  const int threads = ((G.P + 31) / 32) * 32;
  const size_t smem = (size_t)G.P * 3 * G.B * G.B * sizeof(double);
  const size_t stride = G.total;
#define MGRIT_FACTOR(BB)                                                                                         \
  if (transpose) {                                                                                               \
    cudaFuncSetAttribute(k_factor_1d<BB, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
    k_factor_1d<BB, double, true><<<nt, threads, smem, st>>>(sigma, nx, out, stride, flag);                      \
  } else {                                                                                                       \
    cudaFuncSetAttribute(k_factor_1d<BB, double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k_factor_1d<BB, double, false><<<nt, threads, smem, st>>>(sigma, nx, out, stride, flag);                     \
  }
  if (G.B == 1) {
    MGRIT_FACTOR(1)
  } else if (G.B == 2) {
    MGRIT_FACTOR(2)
  } else {
    MGRIT_FACTOR(3)
  }
#undef MGRIT_FACTOR
  return 1;
}

}  // namespace mgrit
