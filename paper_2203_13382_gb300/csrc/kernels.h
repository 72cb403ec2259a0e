// Internal launch interface between the host runtime and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "physics.cuh"

namespace mgrit {

// ---- setup (setup_kernels.cu) ------------------------------------------------------------------

// Fine departure offsets s[n][i] = (x_i - xi) / h, one backward ERK-r step (Sec. 2.1); pairs: the
// spatially varying speeds evaluated in FP32 pairs (FP32-bulk handles), else FP64.
void launch_departure_1d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* s,
                         bool pairs, cudaStream_t st);
// 2D: sx, sy each [nt][nx*nx], row-major (y slow).
void launch_departure_2d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* sx,
                         double* sy, cudaStream_t st);

// Coarse offsets by backtracking (eq. (coarse_depart_interp)) plus phi / sigma (eq. (nu_p_def)).
// s_prev [m*ntc][nx], sigma_prev [m*ntc][nx] or NULL (level 1); eh_prev / el_prev [m*ntc][nx]: the fine
// level's eps as FP32 pairs, or NULL (the sum of f over the fine steps then comes from s_prev in FP64);
// outputs [ntc][nx].
// pairs: FP32-pair arithmetic for the composition and the sum of f (FP32-bulk handles), else FP64.
void launch_backtrack_1d(const double* s_prev, const double* sigma_prev, const float* eh_prev, const float* el_prev,
                         bool pairs, int m, int ntc, int nx, int p, double* s_out, double* sigma_out,
                         cudaStream_t st);
// 2D bilinear backtracking (Sec. SM6); sigma_x / sigma_y per component.
void launch_backtrack_2d(const double* sx_prev, const double* sy_prev, const double* gx_prev, const double* gy_prev,
                         int m, int ntc, int nx, int p, double* sx_out, double* sy_out, double* gx_out, double* gy_out,
                         cudaStream_t st);

// Gather tables of one level from its offsets: shift[n][i] = (E - (p+1)/2 - i) mod nx, and any of the
// FP64 Lagrange weights w64[n][a][i] (a = 0..p), the FP32 distance eps32[n][i] and the rest
// eps_lo[n][i] = eps - eps32 rounded to FP32 (NULL: not written).
void launch_build_tables(const double* s, int nt, int nx, int npts_row, int p, uint16_t* shift, double* w64,
                         float* eps32, float* eps_lo, cudaStream_t st);

// Block-PCR coefficients of the on-the-fly FP32 correction solve (p <= 3): per step, from the FP32 sigma
// rows [nt][nx], record_floats(nx, p) floats into out [nt][record].
unsigned pcr_record_size(int nx, int p);
cudaError_t launch_pcr_coef(const float* sig32, int nt, int nx, int p, float* out, cudaStream_t st);

// The banded separator inverse of the FP32 correction solves (8-row partitions, nx / 8 in 16 .. 512):
// per step a record of band_record_size floats, offsets -kBandMaxHalfWidth .. kBandMaxHalfWidth in rows of
// band_row_size floats, probed from the FP32 sigma rows [nt][nx] with 8 colours (offsets up to 3 stored;
// ind[t], t = 1..4) or 16 colours (offsets up to 6; ind[t], t = 1..8): ind[t] is raised to the largest
// entry at partition distance t relative to the diagonal blocks (ind zeroed before).
constexpr int kBandMaxHalfWidth = 6;
// Entries of the separator inverse below this fraction of its diagonal blocks are left out of the band:
// below the unit roundoff of the FP32 solve that applies it (2^-24 = 6e-8), so the truncation adds less
// than the solve's own rounding.
constexpr float kBandTolerance = 1e-8f;
unsigned band_record_size(int nx, int p);
unsigned band_row_size(int nx, int p);
cudaError_t launch_sep_band(const float* sig32, int nt, int nx, int p, int colours, float* rec, float* ind,
                            cudaStream_t st);

// Factorisation of M = I - diag(sigma) D_{p+1} (periodic, half-bandwidth b = (p+1)/2) for each of nt
// steps (layout: solver_layout.cuh), FP64, solver_reals(nx, p) values per step (FP64 coarse levels and
// the adjoint's M^T; FP32 levels use launch_pcr_coef).  flag (device int) is set to 1 if a pivot is too
// small.  Returns the number of kernel launches issued.
size_t solver_reals(int nx, int p);
int launch_factor_1d(const double* sigma, int nt, int nx, int p, double* out, int* flag, cudaStream_t st,
                     int transpose = 0);

// Adjoint support: per step the range of floor(s) (window of the transposed gather), and d s / d a by
// the tangent-linear ERK step.
void launch_floor_range(const double* s, int nt, int nx, int2* out, cudaStream_t st);
void launch_departure_da_1d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* ds,
                            cudaStream_t st);
// 2D: dsx, dsy each [nt][nx*nx].
void launch_departure_da_2d(const WaveParams& w, int r, int nx, int nt, double xmin, double h, double dt, double* dsx,
                            double* dsy, cudaStream_t st);

// ---- relaxation (relax_kernels.cu) ---------------------------------------------------------------

// One pass over the coarse intervals of a level (one CTA per interval j = 0..J-1).  The CTA loads
// its start slice, takes `nsteps` steps n = j*m + k (k = 0..nsteps-1) of Phi (fine SL step) or
// Psi (gather + correction solve), adding g[n+1] when g is given, and then, by `mode`:
//   MODE_FC   : cout[j+1] = result                      (F- then C-relaxation)
//   MODE_RES  : rout[j+1] = result + gC - cin[j+1]      (F-relaxation + C-point residual)
//   MODE_POST : F-points stored, nothing at the C-point (post F-relaxation, nsteps = m-1)
// F-point results are stored to fstore (full level array) when fstore != NULL.
enum RelaxMode { MODE_FC = 0, MODE_RES = 1, MODE_POST = 2 };

struct LevelTables {
  int nx;
  int npts;  // nx (1D) or nx*nx (2D)
  int p;
  const uint16_t* shift;  // [nt][npts] (2D: x then y blocks)
  const double* w64;      // [nt][p+1][npts] or NULL
  const float* eps32;     // [nt][npts] or NULL (2D: x then y blocks)
  const float* eps_lo;    // level 0 of FP32-bulk handles: eps - eps32 rounded to FP32 ([nt][npts]) or NULL
  // df = 1: a level-0 FP64 pass of the FP32-bulk cycle, run in FP32 pairs from (eps32, eps_lo) instead of
  // FP64 weights (df32.cuh), reading its tables straight from global memory
  int df;
  long long table_stride; // elements per step row of shift / eps32 (npts)
  int nt;                 // steps on this level (for 2D block offsets)
  // correction solver (coarse levels, corrected operator); NULL for the plain SL step
  const void* solver;
  size_t solver_stride;  // reals per step
  // gather_stage = 1 (FP32 1D levels): each step's eps32 and shift rows (and sigma on otf levels) are
  // prefetched into shared memory by TMA bulk copies, one step ahead.  otf = 1 (FP32 coarse levels):
  // `solver` holds sigma as FP32 rows [nt][nx] (solver_stride = nx) and the correction matrix is
  // factorised on the fly in every application; otf = 0: `solver` holds the stored factorisation
  // (solver_layout.cuh).  err: device flag set to 1 if a bounded wait gave up.
  int gather_stage;
  int otf;
  int* err;
  // otf levels with p <= 3: the block-PCR coefficients of every step (relax_kernels.cu
  // pcr_record_floats floats a step, FP32), staged per step into shared memory; NULL: formed on the fly
  const float* pcr;
  unsigned pcr_floats;
  // otf levels: the coefficient record staged per step, cf_floats floats from cf_src + row * cf_stride
  // (0: none).  band > 0: the banded separator inverse of half-width `band` partitions (8-row partitions,
  // relax_kernels.cu corr_solve_band); band = 0 with a record: the block-PCR coefficients above.
  int band;
  const float* cf_src;
  unsigned cf_stride;
  unsigned cf_floats;
  // adjoint: trans = 1 applies Phi^T (coarse: (M^{-1} S)^T = S^T M^{-T}, `solver` then holds the
  // factorisation of M^T); reverse = 1 maps step n to table row nt - 1 - n; frange[row] = floor range.
  int trans;
  int reverse;
  const int2* frange;
  // 2D: FP64 offsets (x block then y block, [2][nt][npts]) for the on-the-fly FP64 weights; on coarse
  // levels `solver` then points at sigma ([2][nt][npts], FP64) of the corrected operator.
  const double* s64;
  // 2D adjoint: arrival points grouped by the base node of their stencil, per step row:
  // bperm[row][bstart[row][key] .. bstart[row][key+1]) lists them in increasing order.
  const int* bstart;  // [nt][npts + 1]
  const int* bperm;   // [nt][npts]
  // 1D FP64 coarse levels: 0 = one CTA per interval; 1 = passes over few intervals split each interval
  // over a thread-block cluster sized automatically; 2..16 = that cluster size (coarse_cluster.cu;
  // identical results)
  int cluster;
  // testing the timeout path only (mgrit_options.test_wait_cycles): > 0 makes the first bounded wait of
  // every CTA of a staged FP32 pass wait, with this limit in SM cycles, on a barrier nothing completes
  int test_wait;
};



struct RelaxArgs {
  int m;          // interval length on this level
  int J;          // intervals
  int nsteps;     // steps per CTA
  int mode;
  const void* start;   // start slice j at start + j * start_stride
  long long start_stride;
  const void* corr;    // optional: added to the start slice (stride corr_stride)
  long long corr_stride;
  void* start_wb;      // optional: corrected start written back (stride wb_stride)
  long long wb_stride;
  int extra_cta;       // launch one more CTA (j = J) that only loads / corrects / writes back its start
  const void* g;       // optional RHS, full level array [(N+1)][npts]
  void* fstore;        // optional F-point store, full level array [(N+1)][npts]
  void* cout;          // MODE_FC output (stride c_stride)
  const void* cin;     // MODE_RES: current C value (stride c_stride)
  const void* cin_corr;  // MODE_RES: optional correction added to cin (stride corr_stride)
  void* rout;          // MODE_RES: residual output (stride r_stride)
  float* rout32;       // MODE_RES, FP64 passes: optional FP32 copy of the residual (stride r_stride)
  int rout_f64;        // MODE_RES, FP32 passes: rout holds doubles (an FP64 coarse level's right-hand side)
  int rout_value;      // MODE_RES, FP32-pair passes: rout receives the propagated C value S^m u_C(j) (the
                       // C-relaxed value, residual + current value) instead of the residual
  long long c_stride;
  long long r_stride;
  int g_at_c;          // MODE_RES: add g at the C-point
  double* norm_partial;  // MODE_RES: per-interval sum of squares [J] (NULL: not needed)
};

// is_double selects FP64 (tables w64) or FP32 (tables eps32) arithmetic and storage.
cudaError_t launch_relax_1d(const LevelTables& T, const RelaxArgs& a, int is_double, cudaStream_t st);

// FP64 coarse passes split over a cluster of C CTAs per interval (coarse_cluster.cu).  cluster_relax_size
// returns the cluster size for this pass (1: use the one-CTA-per-interval kernel); the launch returns
// cudaErrorNotSupported when no cluster of that size (or a smaller power of two) can be formed.
int cluster_relax_size(const LevelTables& T, const RelaxArgs& a);
cudaError_t launch_relax_cluster_1d(const LevelTables& T, const RelaxArgs& a, int C, cudaStream_t st);

// Sequential stepping over all steps of a level: u[n+1] = Phi_n u[n] + g[n+1], n = 0..N-1 (coarsest
// level solve, and the fine-level comparator), from u0 ([npts]; NULL = zero).  store_all = 1: out is
// [(N+1)][npts] with row 0 = u0; store_all = 0: out is [npts] and receives u[N] only.
cudaError_t launch_sequential_1d(const LevelTables& T, int N, const void* g, const void* u0, void* out, int store_all,
                                 int is_double, cudaStream_t st);

// Fine-level sequential stepping (g = 0, plain SL step) by one thread-block cluster holding the slice in
// the shared memory of its CTAs (seq_cluster.cu); nx >= 256.  Same arguments and results as
// launch_sequential_1d; cudaErrorNotSupported when the cluster cannot be formed (the caller then uses
// the single-CTA kernel).
cudaError_t launch_sequential_cluster_1d(const LevelTables& T, int N, const void* u0, void* out, int store_all,
                                         int is_double, cudaStream_t st);

// Applies count steps n0..n0+count-1 to independent slices: out[c] = Phi_{n0+c} in[c].
cudaError_t launch_apply_steps_1d(const LevelTables& T, int n0, int count, const void* in, void* out, int is_double,
                                  cudaStream_t st);

// dJ/da contributions of the intervals of level 0 (FP64): CTA j recomputes u_n, n = j m .. j m + m - 1,
// from the checkpoint C[j] and adds lambda_{n+1}^T (dPhi_n/da) u_n with lambda_{n+1} = mu[nt - n - 1].
cudaError_t launch_gradient_a_1d(const LevelTables& T, const double* s64, const double* ds, const double* C,
                                 const double* mu, int nt, int m, double* partial, cudaStream_t st);

// ---- batched problems (one launch per cycle phase) ------------------------------------------------
struct BatchTile {
  int table;    // index into the LevelTables array of the launch
  int args;     // index into the RelaxArgs / SeqArgs array
  int j;        // interval
  int problem;  // problem index (for the active mask)
};
struct SeqArgs {
  int N;
  const void* g;
  const void* u0;
  void* out;
  int store_all;
};
struct Segment {
  const void* x;
  void* y;
  const void* z;
  long long n;
};
// Shared-memory bytes and slice-buffer length a tile of this level needs, and the bytes of its coarse
// region placed (128-aligned) after the slice buffers; a launch over several tiles takes the largest
// buffer and the largest region.
void relax_smem_need(const LevelTables& T, int is_double, int* buf, size_t* smem, size_t* region);
// threads: CTA size of FP32 launches (32 .. 512, every tile's slice at most 8 * threads points); FP64
// launches use 512.
cudaError_t launch_relax_batched(const LevelTables* d_tabs, const RelaxArgs* d_args, const BatchTile* d_tiles,
                                 int ntiles, const int* d_active, int is_double, int coarse, int buf, size_t smem,
                                 int threads, cudaStream_t st);
cudaError_t launch_sequential_batched(const LevelTables* d_tabs, const SeqArgs* d_args, const BatchTile* d_tiles,
                                      int ntiles, const int* d_active, int is_double, int coarse, int buf,
                                      size_t smem, cudaStream_t st);
// launch_axpy_convert over many segments in one launch (kinds 1, 3, 5, 8 and 0 = copy); segments of
// inactive problems have n = 0.
void launch_axpy_batched(int kind, const Segment* d_seg, int nseg, long long maxn, cudaStream_t st);
// out = sum of seg.x[0 .. n) (doubles, fixed order) written to *(double*)seg.y, one CTA per segment.
void launch_sum_batched(const Segment* d_seg, int nseg, cudaStream_t st);

// Deterministic sum of `count` doubles (fixed order): out[0] = sum.
void launch_sum(const double* v, int count, double* out, cudaStream_t st);
// out[0] = sum_i (a[i] + b[i] - ref[i])^2 over n values (b may be NULL), fixed order.
void launch_dist2(const double* a, const double* b, const double* ref, long long n, double* out, cudaStream_t st);
// Elementwise update with type conversion: kind 0: y = x (d); 1: y(f) = x(d); 2: y(d) += x(f);
// 3: y(d) = x(f); 4: y(d) += x(d); 5: y(d) += x(d) + z(f); 6: y(d) = x(d) - z(d); 7: y(d) += x(d) + z(d);
// 8: y(d) = x(d) + z(f); 9: y(d) = x(d) + z(d).
void launch_axpy_convert(int kind, const void* x, void* y, const void* z, long long n, cudaStream_t st);
// zero fill
void launch_fill_zero(void* y, long long bytes, cudaStream_t st);

// Work buffers of the 2D passes (one slice per interval, the GMRES basis, reduction partials).
struct Scratch2d {
  void* cur;
  void* nxt;
  void* basis;     // [J][kmax + 1][npts] ([J][kmax + 2][npts] with restarts > 1)
  int kmax;        // GMRES iterations at most (<= 10)
  double rtol;     // GMRES relative residual
  double* partial; // [J][64]
  int restarts;    // 1: one GMRES(kmax) cycle (the paper's inexact solve); > 1: restarted cycles to rtol
};

// 2D passes with the same semantics as launch_relax_1d / launch_sequential_1d / launch_apply_steps_1d
// (kernels2d.cu); coarse steps solve the correction system by GMRES (the paper's inexact solve).
cudaError_t launch_relax_2d(const LevelTables& T, const RelaxArgs& a, const Scratch2d& S, int is_double,
                            cudaStream_t st);
cudaError_t launch_sequential_2d(const LevelTables& T, int N, const void* g, const void* u0, void* out, int store_all,
                                 const Scratch2d& S, int is_double, cudaStream_t st);
cudaError_t launch_apply_steps_2d(const LevelTables& T, int n0, int count, const void* in, void* out,
                                  const Scratch2d& S, int is_double, cudaStream_t st);

// 2D adjoint.  Groups the arrival points of every step row by the base node of their stencil
// (shift: [2][nt][npts] as in LevelTables) into bstart / bperm; deterministic (sorted buckets).
cudaError_t launch_bucket_build(const uint16_t* shift, int nt, int nx, int* bstart, int* bperm, cudaStream_t st);
// dJ/da contributions per interval of level 0 (FP64): u_n recomputed from the checkpoints C[j] by fine
// steps; out[j] = sum_n lambda_{n+1} . (dPhi_n/da) u_n with lambda_{n+1} = mu[nt - n - 1].
cudaError_t launch_gradient_a_2d(const LevelTables& T, const double* ds, const double* C, const double* mu, int nt,
                                 int m, int J, const Scratch2d& S, double* out, cudaStream_t st);

}  // namespace mgrit
