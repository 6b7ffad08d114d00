// Solver context shared by the C ABI and the format-specific drivers.
#pragma once

#include <array>
#include <cstdint>
#include <vector>

#include "dvm_internal.h"
#include "tucker.h"

struct TuckerState;  // tucker_step.cu

struct dvm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  dvm_vgrid vg{};
  dvm_gas gas{};
  dvm_opts opts{};
  int64_t nc = 0, nf = 0, nn = 0;
  int N[3] = {0, 0, 0};
  double w = 0.0, xi_max = 0.0;
  std::vector<double> xi[3];

  // topology and geometry (host)
  std::vector<int32_t> slot_nb;     // [nc*6] neighbour cell, -1 on the boundary
  std::vector<int32_t> slot_group;  // [nc*6] boundary group, -1 inside
  std::vector<int8_t> slot_owner;   // [nc*6] 1 if the cell owns the face
  std::vector<double> slot_A;       // [nc*6][3] outward area vector
  std::vector<double> vol;          // [nc]
  std::vector<int64_t> face_slot;   // [nf] owner slot of each face
  std::vector<int64_t> face_other;  // [nf] neighbour slot or -1

  // boundary conditions
  std::vector<int32_t> bc_type;                // [kMaxGroups], -1 = unset
  std::vector<std::array<double, 8>> bc_par;   // [kMaxGroups]
  std::vector<int32_t> group_ghost;            // [kMaxGroups] ghost tensor index or -1
  int nghost = 0;
  bool all_axis = true;
  std::vector<dvm::SlotDev> slot;  // [nc*6]

  // device memory
  double *d_xi[3] = {nullptr, nullptr, nullptr};
  dvm::SlotDev *d_slot = nullptr;
  double *d_ghost = nullptr;   // [nghost][nn]
  double *d_vol = nullptr;
  double *d_f[2] = {nullptr, nullptr};  // full format state
  double *d_sums[2] = {nullptr, nullptr};
  double *d_uref = nullptr;    // [nc][3]
  double *d_respart = nullptr; // [nc][2]
  double *d_res = nullptr;     // [1]
  double *d_macro = nullptr;   // [nc][8]
  int *d_flag = nullptr;
  int cur = 0;
  size_t bytes = 0;

  double dt = 0.0;
  int64_t steps = 0;
  bool prepared = false;
  bool initialized = false;

  TuckerState *tucker = nullptr;

  // implicit full-format step (LU-SGS): the cells of the forward sweep's
  // wavefronts, then the backward sweep's, in launch order; per-cell dt nu
  int32_t *d_wave = nullptr;         // [2][nc]
  std::vector<int64_t> wave_off[2];  // wavefront w of sweep s: [wave_off[s][w], wave_off[s][w+1])
  double *d_dtnu = nullptr;          // [nc]
  double *d_rD = nullptr;            // [nc][nn] 1 / D~ of the current step

  // optional per-launch event timing (dvm_set_kernel_timing)
  struct Timing {
    bool on = false;
    cudaEvent_t open[dvm::kKClasses] = {};
    std::vector<std::array<void *, 3>> pending;  // (class, start, end)
    double ms[dvm::kKClasses] = {};
    int64_t launches[dvm::kKClasses] = {};
  } timing;
  dvm::LaunchTimer timer() {
    return timing.on ? dvm::LaunchTimer{&ctx_timer_mark, this} : dvm::LaunchTimer{nullptr, nullptr};
  }
  static void ctx_timer_mark(void *self, int cls, bool begin, cudaStream_t s);
};

int ctx_collect_timing(dvm_ctx *C);

// context.cu
int ctx_alloc_state(dvm_ctx *C);
void ctx_free(dvm_ctx *C);
int ctx_prepare_boundaries(dvm_ctx *C);
int ctx_init_from_maxwellians(dvm_ctx *C, const double *n, const double *u, const double *T);
int ctx_init_from_full(dvm_ctx *C, const double *f, bool on_device);
int ctx_clear_flag(dvm_ctx *C);
int ctx_step(dvm_ctx *C, int32_t nsteps, double *residual_out);
int ctx_moments(dvm_ctx *C, double *out);
int ctx_get_f(dvm_ctx *C, int64_t cell0, int64_t ncell, double *out);
int ctx_get_ranks(dvm_ctx *C, int32_t *r);
int ctx_memory(dvm_ctx *C, size_t *f_bytes, size_t *total_bytes);
int ctx_save(dvm_ctx *C, const char *path);
int ctx_load(dvm_ctx *C, const char *path);
int ctx_malloc(dvm_ctx *C, void **p, size_t bytes);
int ctx_finalize_dt_from_macro(dvm_ctx *C, const std::vector<double> &macro);
// wavefronts of one LU-SGS sweep (see dvm_lusgs_wavefronts)
void lusgs_wavefronts(int64_t nc, const int32_t *nb, bool forward, int32_t *order,
                      std::vector<int64_t> &off);

namespace dvm {
int build_topology(dvm_ctx *C, const dvm_mesh *m);
}

// tucker_step.cu (Tucker format)
int tucker_alloc(dvm_ctx *C);
void tucker_free(dvm_ctx *C);
int tucker_init_from_full(dvm_ctx *C, const double *d_f_full);
int tucker_set_state(dvm_ctx *C, const int32_t *ranks, const double *core,
                     const double *const fac[3], bool on_device);
int tucker_get_state(dvm_ctx *C, int32_t *ranks, double *core, double *const fac[3]);
int tucker_init_maxwellians(dvm_ctx *C, const double *d_n, const double *d_u, const double *d_T);
int tucker_step(dvm_ctx *C, int32_t nsteps, double *residual_out);
int tucker_moments(dvm_ctx *C, double *d_macro);
int tucker_get_f(dvm_ctx *C, int64_t cell0, int64_t ncell, double *d_out);
int tucker_get_ranks(dvm_ctx *C, int32_t *r);
int tucker_memory(dvm_ctx *C, size_t *f_bytes);
int tucker_save(dvm_ctx *C, FILE *fp);
int tucker_load(dvm_ctx *C, FILE *fp);
int tucker_launch_info(dvm_ctx *C, int32_t *grid, float *tune_ms);
