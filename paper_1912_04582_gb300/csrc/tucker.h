// Tucker-format device structures and launchers (internal).
#pragma once

#include <cstddef>
#include <cstdint>

#include "dvm_internal.h"

namespace dvm {

// One set of Tucker tensors, one per cell, FP64, capacity R per mode.
struct TuckerDev {
  double *core;   // [nc][R*R*R], compact r1 x r2 x r3 (k3 fastest)
  double *fac[3]; // [nc][N_a*R], row i at offset i*R, first r_a columns used
  int *rank;      // [nc][3]
};

// per-cell parameters of the assembly: n, u (3), T, q (3), dt nu, the Shakhov
// coefficient, the Maxwellian amplitude
constexpr int kCellPar = 12;

struct TuckerStepParams {
  TuckerDev cur;         // state at t^n (read)
  TuckerDev nxt;         // state at t^{n+1} (written)
  const double *sums;    // [nc][kSums] moment sums of cur
  const SlotDev *slot;   // [nc][6]
  const double *ghostf;  // [nghost][3][Nmax] rank-1 ghost Maxwellian factors
  const float *ghostf32; // the same in FP32
  const double *xi[3];
  const double *finit;   // mode 1: [nc][N^3] tensors to compress
  double *err;           // [nc] relative truncation error of the last rounding (may be null)
  long long *phase;      // [32] optional per-phase cycle counters (null: off)
  const double *cellpar; // [nc][kCellPar] per-cell parameters of the assembly (null: the
                         // assembly forms them from the sums)
  int *flag;
  void *scratch;         // per-CTA work space
  size_t scratch_stride; // elements (of the kernel's scalar type) per CTA
  int64_t nc;
  int N1, N2, N3, R, Nmax;
  int mode;              // 0 = time step, 1 = compress finit
  int tc_gram;           // phase-major mixed path: first-mode Gram on the tensor cores
  int gemm_asm;          // phase-major mixed path: assembly as one GEMM per cell (all faces on
                         // coordinate planes)
  double w, dt, Pr, omega, delta, tol;
};

// Work buffers of the phase-major step for a chunk of cells [c0, c0 + cn)
struct TuckerSplitBufs {
  void *X;       // [cn][N1*N2*N3] f^{n+1} before rounding (working precision)
  void *Y1;      // [cn][R*N2*N3] after the first-mode projection
  void *Y2;      // [cn][R*R*N3]  after the second-mode projection
  double *C;     // [cn][Nmax*Nmax] Gram matrix of the current mode
  double *e;     // [cn] ||X||^2
  double *disc;  // [cn] energy left out so far
  void *T2all;   // [nc][R][N2 N3] mode-2/3 contraction of every cell (working precision)
  void *U1all;   // [nc][R][padN(N1)] first-mode factors, transposed, zero-padded
  void *t2;      // assembly staging, t2_stride elements per assembly CTA
  size_t t2_stride;
  int asm_grid;  // assembly CTAs (persistent over the chunk)
  int64_t c0, cn;  // cells [c0, c0 + cn) of this launch
  int64_t joff;    // their first buffer index (buffers hold one chunk)
  float *rowmax;   // [cn][Nmax] largest |X| per first-mode row (mixed path; may be null)
  double *cellpar; // [nc][kCellPar] per-cell parameters, formed at the start of the step
  double *macro;   // [nc][8] macroparameters of the current state (may be null)
};

// Extra streams and fork / join events of the phase-major step (optional):
// the cells of a chunk are split into `ways` ranges, one per stream (the
// caller's stream and ways - 1 of these)
constexpr int kMaxWays = 4;
struct SplitStreams {
  int ways;
  cudaStream_t sx[kMaxWays - 1];
  cudaEvent_t fork, join[kMaxWays - 1];
};

// Kernel classes of the optional per-launch event timing (dvm_set_kernel_timing)
enum KernelClass : int {
  kKFullStep = 0,   // full-grid step kernel
  kKFusedStep = 1,  // fused Tucker step kernel
  kKAsm = 2,        // phase-major: assembly
  kKGram0 = 3,      // phase-major: first-mode Gram matrices
  kKGram12 = 4,     // phase-major: second / third-mode Gram matrices
  kKEig = 5,        // phase-major: eigen-solves
  kKProj = 6,       // phase-major: projections and cores
  kKMoments = 7,    // moments (and macroparameters) of the new state
  kKContract = 8,   // phase-major: mode-2/3 contraction of every cell
  kKClasses = 9
};

// Event marks around launches (null: no timing)
struct LaunchTimer {
  void (*mark)(void *self, int cls, bool begin, cudaStream_t s);
  void *self;
  void operator()(int cls, bool begin, cudaStream_t s) const {
    if (mark) mark(self, cls, begin, s);
  }
};

struct TuckerMomentParams {
  TuckerDev T;
  const double *uref;    // reference velocity, uref[c*uref_stride + k] (may be null)
  int uref_stride;
  const SlotDev *slot;
  const double *xi[3];
  double *sums;          // [nc][kSums] out
  const double *sums_prev;  // [nc][kSums] of the previous state (residual) or null
  double *respart;       // [nc][2] or null
  const double *vol;
  int *flag;
  int64_t nc;            // cells [c0, nc) are processed
  int64_t c0;
  int N1, N2, N3, R;
  double w;
  int stage;             // set by launch_tucker_moments: factors (1) / core (2) to shared memory
};

// Tensor-core Gram matrices (gram_tc.cu): plan of the MMA groups for n rows
constexpr int kTcSlices = 5;     // integer slices per FP32 value
constexpr int kTcMaxGroups = 4;  // MMA groups per K-chunk
struct GramTcPlan {
  int n, sp;                     // rows, rows per slice in shared memory
  int ngroups;                   // 0: no plan
  int a0[kTcMaxGroups];          // first slice of the A operand (128 rows)
  int b0[kTcMaxGroups];          // first slice of the B operand
  int nb[kTcMaxGroups];          // slices in the B operand
  int N[kTcMaxGroups];           // MMA N (B rows, a multiple of 16)
  int col[kTcMaxGroups];         // first tensor-memory column of the group's accumulator
  int ncols;                     // tensor-memory columns allocated
  int buf_rows;                  // rows of one shared-memory stage
  int nstages;                   // shared-memory stages of sliced chunks (2 or 3)
  int ltri;                      // words of one level accumulator (the packed upper triangle)
  signed char own[kTcSlices * kTcSlices];  // group + 1 that owns product (k, l), else 0
};
GramTcPlan gram_tc_plan(int n);
bool gram_tc_supported(int n, int K);
// raise the kernel's shared-memory opt-in for n rows (outside stream captures); 0 ok
int gram_tc_prepare(int n);
// raise the GEMM-form assembly kernel's shared-memory opt-in (outside stream captures);
// 0 ok, else the form is not available for this size
int tucker_asm_gemm_prepare(int Nmax, int N1, int R);
// C (double-float pairs) or Cd (doubles), cstride elements per cell; disc[cell] = 0
// rowmax (optional, rstride floats per cell): each row's largest magnitude, known from
// the producer of X; without it the kernel reads X twice (row scales, then slicing)
int launch_gram_tc(const float *X, int64_t xstride, int64_t ncell, int n, int K, float2 *C,
                   double *Cd, int64_t cstride, double *disc, int *flag, cudaStream_t s,
                   const float *rowmax = nullptr, int64_t rstride = 0,
                   long long *phase = nullptr);

size_t tucker_scratch_elems(int N1, int N2, int N3, int R);
size_t tucker_smem_bytes(int Nmax, int R, bool fp64);
int tucker_step_blocks_per_sm(int Nmax, int R, bool fp64);
int launch_tucker_step(const TuckerStepParams &p, int grid, bool fp64, cudaStream_t s);
// phase-major step over chunks of `chunk` cells (buffers sized for one chunk)
// mp (optional): moments of the new state, launched per cell range at the end of
// its chain (cells [c0, nc) of mp are ignored; each range sets its own)
int launch_tucker_split_step(const TuckerStepParams &p, TuckerSplitBufs b, int64_t chunk,
                             bool fp64, cudaStream_t s, const LaunchTimer *lt = nullptr,
                             const SplitStreams *ss = nullptr,
                             const TuckerMomentParams *mp = nullptr);
// bytes of TuckerSplitBufs per cell (working precision fp64 or float)
size_t tucker_split_bytes_per_cell(int N1, int N2, int N3, int R, int Nmax, bool fp64);
// assembly CTAs per SM of the phase-major variant and their staging elements
int tucker_split_asm_per_sm();
size_t tucker_split_t2_elems(int N1, int N2, int N3, int R);
// bytes per cell of the all-cell contraction buffers (TuckerSplitBufs::T2all, U1all)
size_t tucker_split_t2all_bytes_per_cell(int N1, int N2, int N3, int R, bool fp64);
// raise the kernels' shared-memory opt-in for this size (outside stream
// captures); returns a mask of the launch variants whose kernels fit: 1 fused,
// 2 phase-major
int tucker_prepare_launch(int Nmax, int R, bool fp64);
int launch_tucker_expand(const TuckerDev &T, int64_t c0, int64_t ncell, int N1, int N2, int N3,
                         int R, int Nmax, void *scratch, size_t stride, double *out, int grid,
                         bool fp64, cudaStream_t s);
void launch_tucker_moments(const TuckerMomentParams &p, cudaStream_t s);
void launch_tucker_maxwellians(TuckerDev T, const double *n, const double *u, const double *Tc,
                               const double *xi0, const double *xi1, const double *xi2, int64_t nc,
                               int N1, int N2, int N3, int R, cudaStream_t s);

}  // namespace dvm
