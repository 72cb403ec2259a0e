// Setup kernels: departure points, backtracking with phi/sigma, gather tables, and the factorisation
// of the periodic banded correction matrices.  All arithmetic here is FP64.
#include "common.cuh"
#include "kernels.h"
#include "physics.cuh"

namespace mgrit {

// ------------------------------------------------------------------------------------------------
// K1: fine departure offsets (Sec. 2.1 eq. (depart_ODE); Sec. 4.1 eq. (SL2D_char1-2))
// ------------------------------------------------------------------------------------------------

__global__ void k_departure_1d(WaveParams w, Tableau T, int nx, int nt, double xmin, double h, double dt,
                               double* __restrict__ s) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nx * nt) return;
  const int n = (int)(idx / nx), i = (int)(idx % nx);
  const double x = xmin + h * i;
  const double t1 = (n + 1) * dt;
  s[idx] = erk_displacement_1d(w, T, x, t1, dt) / h;
}

__global__ void k_departure_2d(WaveParams w, Tableau T, int nx, int nt, double xmin, double h, double dt,
                               double* __restrict__ sx, double* __restrict__ sy) {
  const long long npts = (long long)nx * nx;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npts * nt) return;
  const int n = (int)(idx / npts);
  const long long pt = idx % npts;
  const int j = (int)(pt / nx), i = (int)(pt % nx);
  const double x = xmin + h * i, y = xmin + h * j;
  double dx, dy;
  erk_displacement_2d(w, T, x, y, (n + 1) * dt, dt, dx, dy);
  sx[idx] = dx / h;
  sy[idx] = dy / h;
}

void launch_departure_1d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* s,
                         cudaStream_t st) {
  const long long tot = (long long)nx * nt;
  const int bs = 256;
  k_departure_1d<<<(unsigned)((tot + bs - 1) / bs), bs, 0, st>>>(w, make_tableau(r), nx, nt, xmin, h, dt, s);
}

void launch_departure_2d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* sx,
                         double* sy, cudaStream_t st) {
  const long long tot = (long long)nx * nx * nt;
  const int bs = 256;
  k_departure_2d<<<(unsigned)((tot + bs - 1) / bs), bs, 0, st>>>(w, make_tableau(r), nx, nt, xmin, h, dt, sx, sy);
}

// ------------------------------------------------------------------------------------------------
// K2: backtracking (Sec. 3.3.1 eq. (coarse_depart_interp); Sec. SM6) and phi / sigma (eq. (nu_p_def))
// ------------------------------------------------------------------------------------------------

// eps = s - floor(s) in [0, 1) (east-neighbour distance, eq. (depart_decompose)).
MGRIT_D double frac_eps(double s) {
  double e = s - floor(s);
  if (e >= 1.0) e -= 1.0;
  return e;
}

// f_{p+1}(z) = prod_{q=-(p+1)/2}^{(p-1)/2} (q + z) / (p+1)!  (eq. (fpoly_def)).
MGRIT_D double f_poly(double z, int p) {
  const int L = (p + 1) / 2;
  double out = 1.0, fact = 1.0;
  for (int q = -L; q <= L - 1; ++q) out = out * (q + z);
  for (int b = 2; b <= p + 1; ++b) fact *= b;
  return out / fact;
}

__global__ void k_backtrack_1d(const double* __restrict__ s_prev, const double* __restrict__ sig_prev, int m, int ntc,
                               int nx, int p, double* __restrict__ s_out, double* __restrict__ sig_out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ntc * nx) return;
  const int n = (int)(idx / nx), i = (int)(idx % nx);
  const long long base = (long long)m * n * nx;
  // position of the coarse characteristic relative to x_i in grid units; c^{(m-1)} = f^{(m-1)}
  double c = -s_prev[base + (long long)(m - 1) * nx + i];
  for (int k = m - 2; k >= 0; --k) {
    const double* row = s_prev + base + (long long)k * nx;
    const double xE = ceil(c);  // east node of c (the node itself if c lies on one)
    const int E = i + (int)xE;
    const double fE = xE - row[wrap_pow2(E, nx)];
    const double fW = (xE - 1.0) - row[wrap_pow2(E - 1, nx)];
    c = (fE - fW) * (c - xE) + fE;
  }
  const double sc = -c;
  s_out[idx] = sc;
  double ff = 0.0, gs = 0.0;
  for (int k = 0; k < m; ++k) {
    ff += f_poly(frac_eps(s_prev[base + (long long)k * nx + i]), p);
    if (sig_prev) gs += sig_prev[base + (long long)k * nx + i];
  }
  const double phi = ((p + 1) & 1 ? -1.0 : 1.0) * (f_poly(frac_eps(sc), p) - ff);
  sig_out[idx] = sig_prev ? gs + phi : phi;
}

void launch_backtrack_1d(const double* s_prev, const double* sigma_prev, int m, int ntc, int nx, int p, double* s_out,
                         double* sigma_out, cudaStream_t st) {
  const long long tot = (long long)nx * ntc;
  const int bs = 256;
  k_backtrack_1d<<<(unsigned)((tot + bs - 1) / bs), bs, 0, st>>>(s_prev, sigma_prev, m, ntc, nx, p, s_out, sigma_out);
}

// Bilinear fit p2d of Sec. SM6 in grid units relative to the arrival node.
MGRIT_D double p2d(double x, double y, double xE, double yN, double rNE, double rNW, double rSE, double rSW) {
  const double pN = (rNE - rNW) * (x - xE) + rNE;
  const double pS = (rSE - rSW) * (x - xE) + rSE;
  return (pN - pS) * (y - yN) + pN;
}

__global__ void k_backtrack_2d(const double* __restrict__ sx_prev, const double* __restrict__ sy_prev,
                               const double* __restrict__ gx_prev, const double* __restrict__ gy_prev, int m, int ntc,
                               int nx, int p, double* __restrict__ sx_out, double* __restrict__ sy_out,
                               double* __restrict__ gx_out, double* __restrict__ gy_out) {
  const long long npts = (long long)nx * nx;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ntc * npts) return;
  const int n = (int)(idx / npts);
  const long long pt = idx % npts;
  const int j = (int)(pt / nx), i = (int)(pt % nx);
  const long long base = (long long)m * n * npts;
  double c = -sx_prev[base + (long long)(m - 1) * npts + pt];
  double d = -sy_prev[base + (long long)(m - 1) * npts + pt];
  for (int k = m - 2; k >= 0; --k) {
    const double* kx = sx_prev + base + (long long)k * npts;
    const double* ky = sy_prev + base + (long long)k * npts;
    const double xE = ceil(c), yN = ceil(d);
    const int E = wrap_pow2(i + (int)xE, nx), W = wrap_pow2(i + (int)xE - 1, nx);
    const int N = wrap_pow2(j + (int)yN, nx), S = wrap_pow2(j + (int)yN - 1, nx);
    const double xW = xE - 1.0, yS = yN - 1.0;
    const long long NE = (long long)N * nx + E, NW = (long long)N * nx + W;
    const long long SE = (long long)S * nx + E, SW = (long long)S * nx + W;
    const double cx = p2d(c, d, xE, yN, xE - kx[NE], xW - kx[NW], xE - kx[SE], xW - kx[SW]);
    const double cy = p2d(c, d, xE, yN, yN - ky[NE], yN - ky[NW], yS - ky[SE], yS - ky[SW]);
    c = cx;
    d = cy;
  }
  sx_out[idx] = -c;
  sy_out[idx] = -d;
  double fx = 0.0, fy = 0.0, sgx = 0.0, sgy = 0.0;
  for (int k = 0; k < m; ++k) {
    const long long q = base + (long long)k * npts + pt;
    fx += f_poly(frac_eps(sx_prev[q]), p);
    fy += f_poly(frac_eps(sy_prev[q]), p);
    if (gx_prev) {
      sgx += gx_prev[q];
      sgy += gy_prev[q];
    }
  }
  const double sgn = ((p + 1) & 1) ? -1.0 : 1.0;
  const double phx = sgn * (f_poly(frac_eps(-c), p) - fx);
  const double phy = sgn * (f_poly(frac_eps(-d), p) - fy);
  gx_out[idx] = gx_prev ? sgx + phx : phx;
  gy_out[idx] = gy_prev ? sgy + phy : phy;
}

void launch_backtrack_2d(const double* sx_prev, const double* sy_prev, const double* gx_prev, const double* gy_prev,
                         int m, int ntc, int nx, int p, double* sx_out, double* sy_out, double* gx_out, double* gy_out,
                         cudaStream_t st) {
  const long long tot = (long long)nx * nx * ntc;
  const int bs = 256;
  k_backtrack_2d<<<(unsigned)((tot + bs - 1) / bs), bs, 0, st>>>(sx_prev, sy_prev, gx_prev, gy_prev, m, ntc, nx, p,
                                                                  sx_out, sy_out, gx_out, gy_out);
}

// ------------------------------------------------------------------------------------------------
// Gather tables
// ------------------------------------------------------------------------------------------------

template <int P>
__global__ void k_build_tables(const double* __restrict__ s, long long total, int nx, int npts_row,
                               uint16_t* __restrict__ shift, double* __restrict__ w64, float* __restrict__ eps32) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const double sv = s[idx];
  double fl = floor(sv);
  double eps = sv - fl;
  if (eps >= 1.0) {
    eps -= 1.0;
    fl += 1.0;
  }
  constexpr int L = (P + 1) / 2;
  // first stencil node E - L with E = i - floor(s); stored as an offset from i, modulo nx
  const long long fli = (long long)fl;
  shift[idx] = (uint16_t)(((-fli - L) % nx + nx) % nx);
  if (eps32) eps32[idx] = (float)eps;
  if (w64) {
    double w[P + 1];
    lagrange_weights<P, double>(eps, w);
    const long long row = idx / npts_row, pt = idx % npts_row;
#pragma unroll
    for (int a = 0; a <= P; ++a) w64[(row * (P + 1) + a) * npts_row + pt] = w[a];
  }
}

void launch_build_tables(const double* s, int nt, int nx, int npts_row, int p, uint16_t* shift, double* w64,
                         float* eps32, cudaStream_t st) {
  const long long tot = (long long)nt * npts_row;
  const int bs = 256;
  const unsigned g = (unsigned)((tot + bs - 1) / bs);
  if (p == 1) k_build_tables<1><<<g, bs, 0, st>>>(s, tot, nx, npts_row, shift, w64, eps32);
  else if (p == 3) k_build_tables<3><<<g, bs, 0, st>>>(s, tot, nx, npts_row, shift, w64, eps32);
  else k_build_tables<5><<<g, bs, 0, st>>>(s, tot, nx, npts_row, shift, w64, eps32);
}

// ------------------------------------------------------------------------------------------------
// K3: partitioned factorisation of M = I - diag(sigma) D_{p+1} (eq. (Bp_def), (Phi_multilevel))
//
// The periodic system is split into P partitions of s = nx/P rows.  The first b rows of each
// partition are separators S_k, the other q = s - b rows the interior I_k, which couples only to
// S_k and S_{k+1}.  Per step we store: the banded LU of each interior block (no pivoting), the
// spikes V_k = A_k^{-1} M[I_k, S_k] and W_k = A_k^{-1} M[I_k, S_{k+1}], the separator couplings to
// the neighbouring interiors, and the inverse of the (periodic block-tridiagonal) Schur complement
// on the separators.  Layout (reals) per step:
//   lu    [(2b+1)][q][P]   rows t < b: L multipliers l_{t+1}; t = b: 1/U_rr; t > b: U_{r, r+t-b}
//   vw    [2b][nx]         V columns then W columns, indexed by the interior point's global index
//   sinv  [bP][bP]         column-major inverse of the Schur complement
//   ctail [P][b][b]        M[S_k + a, (k s - b + c) mod nx]   (couples to the tail of I_{k-1})
//   chead [P][b][b]        M[S_k + a, k s + b + c]           (couples to the head of I_k)
// ------------------------------------------------------------------------------------------------

MGRIT_HD double dstencil(int b, int j) {
  // coefficient of the centred stencil (delta^2)^b at offset j: (-1)^{b+j} C(2b, b+j)
  if (j < -b || j > b) return 0.0;
  double c = 1.0;
  const int n = 2 * b, k = b + j;
  for (int t = 1; t <= k; ++t) c = c * (n - k + t) / t;
  return ((b + j) & 1) ? -c : c;
}

size_t solver_reals(int nx, int p, int P) {
  const int b = (p + 1) / 2;
  const int s = nx / P, q = s - b;
  return (size_t)(2 * b + 1) * q * P + (size_t)2 * b * nx + (size_t)(b * P) * (b * P) + (size_t)2 * P * b * b;
}

int solver_partitions(int nx, int p) {
  const int b = (p + 1) / 2;
  int P = 32;
  while (P > 1 && (nx % P != 0 || nx / P < 2 * b + 1)) P >>= 1;
  return P;
}

template <typename R>
struct SolverView {
  R* lu;
  R* vw;
  R* sinv;
  R* ctail;
  R* chead;
};

template <typename R>
MGRIT_HD SolverView<R> solver_view(R* base, int nx, int b, int P) {
  const int s = nx / P, q = s - b;
  SolverView<R> v;
  v.lu = base;
  v.vw = v.lu + (size_t)(2 * b + 1) * q * P;
  v.sinv = v.vw + (size_t)2 * b * nx;
  v.ctail = v.sinv + (size_t)(b * P) * (b * P);
  v.chead = v.ctail + (size_t)P * b * b;
  return v;
}

constexpr int kFactorThreads = 256;
constexpr int kMaxSchur = 96;  // b * P <= 3 * 32

// Solve A_k x = rhs in place (interior block of partition k) using the stored LU (FP64 copy).
__device__ void interior_solve_fp64(const double* lu, int b, int q, int P, int k, double* x /*len q, stride 1*/) {
  for (int r = 0; r < q; ++r) {
    double v = x[r];
    for (int t = 1; t <= b && r - t >= 0; ++t) v -= lu[((size_t)(t - 1) * q + r) * P + k] * x[r - t];
    x[r] = v;
  }
  for (int r = q - 1; r >= 0; --r) {
    double v = x[r];
    for (int t = 1; t <= b && r + t < q; ++t) v -= lu[((size_t)(b + t) * q + r) * P + k] * x[r + t];
    x[r] = v * lu[((size_t)b * q + r) * P + k];
  }
}

template <typename R>
__global__ void __launch_bounds__(kFactorThreads) k_factor_1d(const double* __restrict__ sigma_all, int nx, int p,
                                                              int P, R* __restrict__ out_all, size_t stride,
                                                              double* __restrict__ scratch_all, int* flag) {
  const int n = blockIdx.x;
  const int b = (p + 1) / 2;
  const int s = nx / P, q = s - b;
  const int nb = b * P;
  const double* sigma = sigma_all + (size_t)n * nx;
  R* out = out_all + (size_t)n * stride;  // (chunk-relative step n)
  SolverView<R> V = solver_view<R>(out, nx, b, P);
  // FP64 working copies in global scratch: lu [(2b+1)][q][P], spikes [2b][nx]
  double* lu = scratch_all + (size_t)blockIdx.x * ((size_t)(2 * b + 1) * q * P + (size_t)2 * b * nx);
  double* sp = lu + (size_t)(2 * b + 1) * q * P;
  extern __shared__ double S[];  // [nb][nb] row-major Schur complement
  __shared__ int perm[kMaxSchur];
  __shared__ double piv_s;
  __shared__ int piv_row;

  auto Mval = [&](int row, int col) -> double {  // entry M[row, col] (indices mod nx)
    int off = col - row;
    off = ((off % nx) + nx) % nx;
    if (off > nx / 2) off -= nx;
    const double dv = dstencil(b, off);
    return (off == 0 ? 1.0 : 0.0) - sigma[((row % nx) + nx) % nx] * dv;
  };

  // 1) banded LU of each interior block (one thread per partition)
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const int g0 = k * s + b;
    double Uw[3][4];  // last b rows of U: Uw[t][c] = U[r-1-t][r-1-t+c], c = 0..b
    for (int r = 0; r < q; ++r) {
      double a[7];  // a[c + b] = A[r][r + c], c = -b..b
      for (int c = -b; c <= b; ++c) a[c + b] = (r + c >= 0 && r + c < q) ? Mval(g0 + r, g0 + r + c) : 0.0;
      for (int t = b; t >= 1; --t) {  // eliminate columns r-t (left to right)
        if (r - t < 0) {
          lu[((size_t)(t - 1) * q + r) * P + k] = 0.0;
          continue;
        }
        const double* Ur = Uw[t - 1];  // row r - t of U
        const double l = a[b - t] / Ur[0];
        lu[((size_t)(t - 1) * q + r) * P + k] = l;
        for (int c = 1; c <= b; ++c) {  // columns r - t + c
          const int col = -t + c;
          if (col <= b) a[col + b] -= l * Ur[c];
        }
      }
      const double diag = a[b];
      if (!(fabs(diag) > 1e-13)) atomicExch(flag, 1);
      lu[((size_t)b * q + r) * P + k] = 1.0 / diag;
      for (int t = 1; t <= b; ++t) lu[((size_t)(b + t) * q + r) * P + k] = a[b + t];
      for (int t = b - 1; t >= 1; --t)
        for (int c = 0; c <= b; ++c) Uw[t][c] = Uw[t - 1][c];
      for (int c = 0; c <= b; ++c) Uw[0][c] = a[b + c];
    }
  }
  __syncthreads();
  // 2) spikes V (columns of S_k) and W (columns of S_{k+1})
  for (int task = threadIdx.x; task < P * 2 * b; task += blockDim.x) {
    const int k = task % P, col = task / P;  // col < b: V column col; else W column col - b
    const int g0 = k * s + b;
    double* dst = sp + (size_t)col * nx;
    // build rhs in dst at the interior points of partition k
    for (int r = 0; r < q; ++r) {
      double v = 0.0;
      if (col < b) {
        const int off = (k * s + col) - (g0 + r);  // column in S_k
        if (off >= -b) v = -sigma[g0 + r] * dstencil(b, off);
      } else {
        const int cc = col - b;
        const int off = q - r + cc;  // column (k+1) s + cc relative to g0 + r
        if (off <= b) v = -sigma[g0 + r] * dstencil(b, off);
      }
      dst[g0 + r] = v;
    }
    // forward / backward substitution along the contiguous interior range of dst
    for (int r = 0; r < q; ++r) {
      double v = dst[g0 + r];
      for (int t = 1; t <= b && r - t >= 0; ++t) v -= lu[((size_t)(t - 1) * q + r) * P + k] * dst[g0 + r - t];
      dst[g0 + r] = v;
    }
    for (int r = q - 1; r >= 0; --r) {
      double v = dst[g0 + r];
      for (int t = 1; t <= b && r + t < q; ++t) v -= lu[((size_t)(b + t) * q + r) * P + k] * dst[g0 + r + t];
      dst[g0 + r] = v * lu[((size_t)b * q + r) * P + k];
    }
    // separator slots of this column: zero
    if (k == 0) {
      for (int kk = 0; kk < P; ++kk)
        for (int a = 0; a < b; ++a) dst[kk * s + a] = 0.0;
    }
  }
  __syncthreads();
  // 3) couplings and the Schur complement on the separators
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) S[e] = 0.0;
  __syncthreads();
  for (int task = threadIdx.x; task < P * b; task += blockDim.x) {
    const int k = task / b, a = task % b;
    const int row = k * s + a;
    const int km = (k + P - 1) % P, kp = (k + 1) % P;
    double ct[3], ch[3];
    for (int c = 0; c < b; ++c) {
      ct[c] = Mval(row, k * s - b + c);  // tail of I_{k-1} (wraps for k = 0)
      ch[c] = Mval(row, k * s + b + c);  // head of I_k
      V.ctail[((size_t)k * b + a) * b + c] = (R)ct[c];
      V.chead[((size_t)k * b + a) * b + c] = (R)ch[c];
    }
    for (int c = 0; c < b; ++c) {
      // x_{S_{k-1}} coefficient: -ctail * V_{k-1}(tail rows)
      double Lc = 0.0, Dc = Mval(row, k * s + c), Uc = 0.0;
      for (int c2 = 0; c2 < b; ++c2) {
        const int tail = km * s + b + (q - b + c2);  // global index of tail row c2 of I_{k-1}
        const int head = k * s + b + c2;             // head row c2 of I_k
        Lc -= ct[c2] * sp[(size_t)c * nx + tail];
        Dc -= ct[c2] * sp[(size_t)(b + c) * nx + tail];
        Dc -= ch[c2] * sp[(size_t)c * nx + head];
        Uc -= ch[c2] * sp[(size_t)(b + c) * nx + head];
      }
      atomicAdd(&S[(size_t)(k * b + a) * nb + km * b + c], Lc);
      atomicAdd(&S[(size_t)(k * b + a) * nb + k * b + c], Dc);
      atomicAdd(&S[(size_t)(k * b + a) * nb + kp * b + c], Uc);
    }
  }
  __syncthreads();
  // 4) in-place Gauss-Jordan inversion of S (row-major in smem) with partial pivoting
  for (int kk = 0; kk < nb; ++kk) {
    if (threadIdx.x == 0) {
      int pr = kk;
      double best = fabs(S[(size_t)kk * nb + kk]);
      for (int r = kk + 1; r < nb; ++r) {
        const double v = fabs(S[(size_t)r * nb + kk]);
        if (v > best) {
          best = v;
          pr = r;
        }
      }
      piv_row = pr;
      perm[kk] = pr;
      if (!(best > 1e-300)) atomicExch(flag, 1);
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != kk)
      for (int c = threadIdx.x; c < nb; c += blockDim.x) {
        const double t = S[(size_t)kk * nb + c];
        S[(size_t)kk * nb + c] = S[(size_t)pr * nb + c];
        S[(size_t)pr * nb + c] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) piv_s = S[(size_t)kk * nb + kk];
    __syncthreads();
    const double pv = piv_s;
    for (int c = threadIdx.x; c < nb; c += blockDim.x)
      S[(size_t)kk * nb + c] = (c == kk ? 1.0 : S[(size_t)kk * nb + c]) / pv;
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int r = e / nb, c = e % nb;
      if (r == kk) continue;
      const double f = S[(size_t)r * nb + kk];
      if (c == kk) continue;
      S[e] -= f * S[(size_t)kk * nb + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      if (r == kk) continue;
      S[(size_t)r * nb + kk] = -S[(size_t)r * nb + kk] * S[(size_t)kk * nb + kk];
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int kk = nb - 1; kk >= 0; --kk) {
    const int pr = perm[kk];
    if (pr != kk)
      for (int r = threadIdx.x; r < nb; r += blockDim.x) {
        const double t = S[(size_t)r * nb + kk];
        S[(size_t)r * nb + kk] = S[(size_t)r * nb + pr];
        S[(size_t)r * nb + pr] = t;
      }
    __syncthreads();
  }
  // 5) write out: LU, spikes (global point layout), Schur inverse (column-major)
  for (size_t e = threadIdx.x; e < (size_t)(2 * b + 1) * q * P; e += blockDim.x) V.lu[e] = (R)lu[e];
  for (size_t e = threadIdx.x; e < (size_t)2 * b * nx; e += blockDim.x) V.vw[e] = (R)sp[e];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    V.sinv[(size_t)c * nb + r] = (R)S[e];
  }
}

int launch_factor_1d(const double* sigma, int nt, int nx, int p, int P, void* out, int is_double, int* flag,
                     cudaStream_t st) {
  const int b = (p + 1) / 2;
  const int s = nx / P, q = s - b;
  const size_t per = (size_t)(2 * b + 1) * q * P + (size_t)2 * b * nx;
  const size_t stride = solver_reals(nx, p, P);
  const int nb = b * P;
  const size_t smem = (size_t)nb * nb * sizeof(double);
  cudaFuncSetAttribute(k_factor_1d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_factor_1d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // process in chunks to bound the FP64 scratch
  const int chunk = 256;
  double* scratch = nullptr;
  const int nchunk = nt < chunk ? nt : chunk;
  if (cudaMallocAsync((void**)&scratch, per * nchunk * sizeof(double), st) != cudaSuccess) return 0;
  int launches = 0;
  for (int n0 = 0; n0 < nt; n0 += chunk, ++launches) {
    const int cnt = (nt - n0) < chunk ? (nt - n0) : chunk;
    if (is_double)
      k_factor_1d<double><<<cnt, kFactorThreads, smem, st>>>(sigma + (size_t)n0 * nx, nx, p, P,
                                                          (double*)out + (size_t)n0 * stride, stride, scratch, flag);
    else
      k_factor_1d<float><<<cnt, kFactorThreads, smem, st>>>(sigma + (size_t)n0 * nx, nx, p, P,
                                                         (float*)out + (size_t)n0 * stride, stride, scratch, flag);
  }
  cudaFreeAsync(scratch, st);
  return launches;
}

}  // namespace mgrit
