// Storage layout of the factorised correction matrices M = I - diag(sigma) D_{p+1} (one per coarse step).
//
// The periodic banded system (half-bandwidth B = (p+1)/2) is cut into P = nx / 8 partitions of 8 rows,
// one per thread.  The first B rows of partition k are its separators S_k; the other q = 8 - B rows, the
// interior I_k, couple only to S_k and S_{k+1}.  Eliminating the interiors leaves a periodic block-
// tridiagonal system for the separators (B x B blocks L_k, D_k, U_k), solved by block parallel cyclic
// reduction (PCR): at level t (stride 2^t) row k eliminates rows k -/+ 2^t with alpha_k = -L_k D_{k-s}^{-1},
// gamma_k = -U_k D_{k+s}^{-1}; after log2(P) levels the rows decouple and x_k = (L_k + D_k + U_k)^{-1} g_k.
//
// Per step (reals of type R), all arrays "structure of arrays" with the partition index k fastest:
//   rec[e][k], e < rec_e: for interior row r: l_1..l_B (multipliers of y_{r-1..r-B}), 1/U_rr,
//                         U_{r,r+1..r+B};  then V[r][c] (q x B), W[r][c] (q x B), ctail[a][c], chead[a][c]
//   pcr[t][e][k], e < 2 B^2: alpha (B x B, row-major) then gamma, for t = 0 .. T-1 (T = log2 P)
//   fin[e][k], e < B^2: (L + D + U)^{-1} of the last level
// V = A_k^{-1} M[I_k, S_k], W = A_k^{-1} M[I_k, S_{k+1}] (the spikes); ctail[a][c] = M[S_k + a, k*8 - B + c]
// couples to the tail of I_{k-1}, chead[a][c] = M[S_k + a, k*8 + B + c] to the head of I_k.
#pragma once

#include "common.cuh"

namespace mgrit {

constexpr int kPartRows = 8;

struct SolverGeom {
  int P, B, q, T, rec_e;
  size_t pcr_off, fin_off, total;
};

MGRIT_HD SolverGeom solver_geom(int nx, int p) {
  SolverGeom g;
  g.B = (p + 1) / 2;
  g.P = nx / kPartRows;
  g.q = kPartRows - g.B;
  g.T = 0;
  while ((1 << g.T) < g.P) ++g.T;
  g.rec_e = g.q * (2 * g.B + 1) + 2 * g.q * g.B + 2 * g.B * g.B;
  g.pcr_off = (size_t)g.rec_e * g.P;
  g.fin_off = g.pcr_off + (size_t)g.T * 2 * g.B * g.B * g.P;
  g.total = g.fin_off + (size_t)g.B * g.B * g.P;
  return g;
}

// offsets inside rec (element index e)
MGRIT_HD int rec_lu(int B, int r, int f) { return r * (2 * B + 1) + f; }
MGRIT_HD int rec_v(int B, int q, int r, int c) { return q * (2 * B + 1) + r * B + c; }
MGRIT_HD int rec_w(int B, int q, int r, int c) { return q * (2 * B + 1) + q * B + r * B + c; }
MGRIT_HD int rec_ct(int B, int q, int a, int c) { return q * (2 * B + 1) + 2 * q * B + a * B + c; }
MGRIT_HD int rec_ch(int B, int q, int a, int c) { return q * (2 * B + 1) + 2 * q * B + B * B + a * B + c; }

}  // namespace mgrit
