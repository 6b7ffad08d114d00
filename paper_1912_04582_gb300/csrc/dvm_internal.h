// Internal declarations of the GB300 S-model DVM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dvm.h"

namespace dvm {

constexpr int kMaxGroups = 4096;
constexpr int kMaxN = 128;

// Per-cell moment sums written by the full-grid step epilogue / moments kernel.
// All sums are raw (without the quadrature weight) and taken about a per-cell
// reference velocity r (stored in the first three slots):
//   [0..2] r
//   [3]    S0  = sum f
//   [4..6] M_a = sum (xi_a - r_a) f
//   [7..12] S11 S22 S33 S12 S13 S23 = sum (xi_a - r_a)(xi_b - r_b) f
//   [13..15] Q_a = sum (xi_a - r_a) |xi - r|^2 f
//   [16..21] O_l = sum max(xi.e_l, 0) f  for wall slots l (0 elsewhere)
constexpr int kSums = 24;
constexpr int kRawSums = 19;  // entries 3..21 are reduced

enum SlotKind : int32_t {
  kInterior = 0,
  kZeroGrad = 1,
  kSymmetry = 2,
  kFreeStream = 3,
  kWall = 4,
};

// What the step kernel needs to know about one (cell, local face) slot.
struct SlotDev {
  double ce[3];     // c * e: c = dt |A| / |V| and e the outward unit normal
  double c;         // dt |A| / |V|
  double e[3];      // outward unit normal
  double wall_den;  // wall slots: sum over nodes with xi.e < 0 of (xi.e) fhat_w
  int32_t kind;     // SlotKind
  int32_t axis;     // 0,1,2 if e = +-unit axis exactly; -1 otherwise
  int32_t sgn;      // sign of e along `axis` (+1/-1)
  int32_t src;      // neighbour cell (interior) or ghost tensor index (free stream / wall)
  int32_t flip;     // symmetry: axis whose index is mirrored
  int32_t pad[3];
};
static_assert(sizeof(SlotDev) == 96, "SlotDev layout");

// Parameters of one full-grid launch.
struct FullParams {
  const double *f;       // [nc][nn] state at t^n
  double *fnew;          // [nc][nn] state at t^{n+1}
  const double *sums;    // [nc][kSums] moment sums of f
  double *sums_new;      // [nc][kSums] moment sums of fnew
  double *respart;       // [nc][2] residual numerator / denominator parts (may be null)
  const SlotDev *slot;   // [nc][6]
  const double *ghost;   // [nghost][nn] free-stream / unit wall Maxwellians
  const double *vol;     // [nc]
  const double *xi[3];   // nodes per axis
  int *flag;             // bit 0: non-physical n or T seen; bit 1: a bulk copy wait ran out
  int64_t nc;
  int N1, N2, N3;
  int all_axis;          // 1 if every face normal is a signed coordinate axis
  double w;              // quadrature weight
  double dt;
  double Pr, omega, delta;  // delta = sqrt(pi) / (2 Kn)
  double *dtnu;          // [nc] dt nu of f^n (written by the implicit step's right-hand side)
};

// One wavefront of an LU-SGS sweep of the implicit full-grid step.
struct LusgsParams {
  double *g;             // [nc][nn] dt R^n before the forward sweep, the increment after
                         // the backward sweep
  double *rD;            // [nc][nn] 1 / D~ (written by the forward sweep, read by the backward)
  const double *dtnu;    // [nc] dt nu of f^n
  const SlotDev *slot;   // [nc][6]
  const double *xi[3];
  const int32_t *cells;  // the cells of this wavefront
  int N1, N2, N3;
  int all_axis;
};

// moments-only launch (initialisation / reference velocity refresh)
struct MomentParams {
  const double *f;
  double *sums;          // [nc][kSums] output
  const double *uref;    // [nc][3] reference velocity (may be null = 0)
  const SlotDev *slot;
  const double *xi[3];
  int64_t nc;
  int N1, N2, N3;
};

void launch_full_step(const FullParams &p, cudaStream_t s);
// implicit step (LU-SGS): dt R^n into p.fnew and dt nu into p.dtnu; one sweep
// wavefront; f^{n+1} = f^n + df into p.fnew with the moment sums and residual parts
void launch_full_rhs(const FullParams &p, cudaStream_t s);
void launch_lusgs_sweep(const LusgsParams &p, int ncell, bool forward, cudaStream_t s);
void launch_lusgs_apply(const FullParams &p, cudaStream_t s);
void launch_full_moments(const MomentParams &p, cudaStream_t s);
void launch_macro_from_sums(const double *sums, double *macro, int64_t nc, double w,
                            cudaStream_t s);
void launch_residual_reduce(const double *respart, int64_t nc, double dt, double *out,
                            cudaStream_t s);
void launch_maxwellian_fill(double *out, const double *xi0, const double *xi1,
                            const double *xi2, int N1, int N2, int N3, double n,
                            const double u[3], double T, cudaStream_t s);
void launch_inflow_sum(const double *ghost, const double *xi0, const double *xi1,
                       const double *xi2, int N1, int N2, int N3, const double e[3],
                       double *out, cudaStream_t s);
void launch_cell_maxwellians(double *f, const double *n, const double *u, const double *T,
                             const double *xi0, const double *xi1, const double *xi2,
                             int64_t nc, int N1, int N2, int N3, cudaStream_t s);

// error plumbing
void set_error(const std::string &msg);

// host-side fault injection (faults.cu): true when the armed failure of that kind
// fires at this call
bool fault_alloc();
bool fault_timeout();
bool fault_admit();

}  // namespace dvm

#define DVM_CUDA_TRY(expr)                                                       \
  do {                                                                           \
    cudaError_t e__ = (expr);                                                    \
    if (e__ != cudaSuccess) {                                                    \
      dvm::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));       \
      return DVM_ERR_CUDA;                                                       \
    }                                                                            \
  } while (0)
