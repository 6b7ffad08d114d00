// Context state management: device allocation, boundary set-up, initial state,
// time stepping dispatch (full grid here, Tucker in tucker_step.cu), moments
// and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dvm_context.h"

using namespace dvm;

namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr uint64_t kCkptMagic = 0x31304d5644475342ULL;  // "BSGDVM01"

bool is_unit_axis(const double e[3], int *axis, int *sgn) {
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, d = (a + 2) % 3;
    if (std::fabs(e[a]) == 1.0 && e[b] == 0.0 && e[d] == 0.0) {
      *axis = a;
      *sgn = e[a] > 0 ? 1 : -1;
      return true;
    }
  }
  return false;
}

int sync_and_check(dvm_ctx *C) {
  DVM_CUDA_TRY(cudaGetLastError());
  DVM_CUDA_TRY(cudaStreamSynchronize(C->stream));
  return DVM_OK;
}
}  // namespace

int ctx_malloc(dvm_ctx *C, void **p, size_t bytes) {
  if (fault_alloc()) {
    *p = nullptr;
    set_error("device allocation of " + std::to_string(bytes) +
              " bytes failed: out of memory (injected by dvm_fault_inject)");
    return DVM_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(p, bytes == 0 ? 16 : bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " +
              cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DVM_ERR_OOM : DVM_ERR_CUDA;
  }
  C->bytes += bytes;
  return DVM_OK;
}

#define CTX_MALLOC(ptr, bytes)                                          \
  do {                                                                  \
    int rc__ = ctx_malloc(C, reinterpret_cast<void **>(&(ptr)), (bytes)); \
    if (rc__ != DVM_OK) return rc__;                                    \
  } while (0)

int ctx_alloc_state(dvm_ctx *C) {
  const int64_t nc = C->nc;
  for (int a = 0; a < 3; ++a) {
    CTX_MALLOC(C->d_xi[a], sizeof(double) * C->N[a]);
    DVM_CUDA_TRY(cudaMemcpy(C->d_xi[a], C->xi[a].data(), sizeof(double) * C->N[a],
                            cudaMemcpyHostToDevice));
  }
  CTX_MALLOC(C->d_vol, sizeof(double) * nc);
  DVM_CUDA_TRY(cudaMemcpy(C->d_vol, C->vol.data(), sizeof(double) * nc, cudaMemcpyHostToDevice));
  CTX_MALLOC(C->d_slot, sizeof(SlotDev) * 6 * nc);
  for (int k = 0; k < 2; ++k) CTX_MALLOC(C->d_sums[k], sizeof(double) * kSums * nc);
  CTX_MALLOC(C->d_uref, sizeof(double) * 3 * nc);
  CTX_MALLOC(C->d_respart, sizeof(double) * 2 * nc);
  CTX_MALLOC(C->d_res, sizeof(double) * 4);
  CTX_MALLOC(C->d_macro, sizeof(double) * 8 * nc);
  CTX_MALLOC(C->d_flag, sizeof(int) * 4);
  DVM_CUDA_TRY(cudaMemset(C->d_flag, 0, sizeof(int) * 4));
  if (C->opts.format == DVM_FORMAT_FULL) {
    const size_t fb = sizeof(double) * (size_t)nc * (size_t)C->nn;
    for (int k = 0; k < 2; ++k) CTX_MALLOC(C->d_f[k], fb);
    if (C->opts.scheme == DVM_SCHEME_LUSGS) {
      std::vector<int32_t> order(2 * nc);
      for (int s = 0; s < 2; ++s)
        lusgs_wavefronts(nc, C->slot_nb.data(), s == 0, order.data() + s * nc, C->wave_off[s]);
      CTX_MALLOC(C->d_wave, sizeof(int32_t) * 2 * nc);
      DVM_CUDA_TRY(cudaMemcpy(C->d_wave, order.data(), sizeof(int32_t) * 2 * nc,
                              cudaMemcpyHostToDevice));
      CTX_MALLOC(C->d_dtnu, sizeof(double) * nc);
      CTX_MALLOC(C->d_rD, fb);
    }
  } else {
    int rc = tucker_alloc(C);
    if (rc != DVM_OK) return rc;
  }
  return DVM_OK;
}

// per-launch event timing: a begin mark records a fresh event, the matching end
// mark another, queued until ctx_collect_timing reads them
void dvm_ctx::ctx_timer_mark(void *self, int cls, bool begin, cudaStream_t s) {
  dvm_ctx *C = static_cast<dvm_ctx *>(self);
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaEventRecord(e, s);
  if (begin) {
    if (C->timing.open[cls]) cudaEventDestroy(C->timing.open[cls]);
    C->timing.open[cls] = e;
  } else if (C->timing.open[cls]) {
    C->timing.pending.push_back({reinterpret_cast<void *>((intptr_t)cls),
                                 static_cast<void *>(C->timing.open[cls]), static_cast<void *>(e)});
    C->timing.open[cls] = nullptr;
  } else {
    cudaEventDestroy(e);
  }
}

int ctx_collect_timing(dvm_ctx *C) {
  auto &T = C->timing;
  if (!T.pending.empty()) DVM_CUDA_TRY(cudaStreamSynchronize(C->stream));
  for (auto &p : T.pending) {
    const int cls = (int)reinterpret_cast<intptr_t>(p[0]);
    float ms = 0.f;
    cudaEvent_t a = static_cast<cudaEvent_t>(p[1]), b = static_cast<cudaEvent_t>(p[2]);
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
      T.ms[cls] += ms;
      T.launches[cls] += 1;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  T.pending.clear();
  cudaGetLastError();
  return DVM_OK;
}

void ctx_free(dvm_ctx *C) {
  ctx_collect_timing(C);
  for (auto &e : C->timing.open)
    if (e) cudaEventDestroy(e);
  if (C->tucker) tucker_free(C);
  void *ptrs[] = {C->d_xi[0], C->d_xi[1], C->d_xi[2], C->d_vol, C->d_slot, C->d_ghost,
                  C->d_f[0], C->d_f[1], C->d_sums[0], C->d_sums[1], C->d_uref, C->d_respart,
                  C->d_res, C->d_macro, C->d_flag, C->d_wave, C->d_dtnu, C->d_rD};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

// Validate boundary conditions, build ghost tensors and the per-slot table (the
// time-step dependent coefficient c is filled in once dt is known).
int ctx_prepare_boundaries(dvm_ctx *C) {
  if (C->prepared) return DVM_OK;
  const int64_t nc = C->nc;
  C->group_ghost.assign(kMaxGroups, -1);
  C->nghost = 0;
  for (int64_t s = 0; s < 6 * nc; ++s) {
    const int g = C->slot_group[s];
    if (g < 0) continue;
    if (C->bc_type[g] < 0) {
      set_error("boundary group " + std::to_string(g) + " has no boundary condition");
      return DVM_ERR_STATE;
    }
    if ((C->bc_type[g] == DVM_BC_FREESTREAM || C->bc_type[g] == DVM_BC_WALL) &&
        C->group_ghost[g] < 0)
      C->group_ghost[g] = C->nghost++;
  }
  if (C->nghost > 0) {
    CTX_MALLOC(C->d_ghost, sizeof(double) * (size_t)C->nghost * (size_t)C->nn);
    for (int g = 0; g < kMaxGroups; ++g) {
      const int k = C->group_ghost[g];
      if (k < 0) continue;
      const auto &p = C->bc_par[g];
      const double u[3] = {p[1], p[2], p[3]};
      const double n = C->bc_type[g] == DVM_BC_WALL ? 1.0 : p[0];
      launch_maxwellian_fill(C->d_ghost + (size_t)k * C->nn, C->d_xi[0], C->d_xi[1], C->d_xi[2],
                             C->N[0], C->N[1], C->N[2], n, u, p[4], C->stream);
    }
  }
  C->slot.assign(6 * nc, SlotDev{});
  C->all_axis = true;
  std::map<std::tuple<int, double, double, double>, double> den_cache;
  std::vector<std::pair<int64_t, std::tuple<int, double, double, double>>> need_den;
  for (int64_t s = 0; s < 6 * nc; ++s) {
    SlotDev &sd = C->slot[s];
    const double *A = &C->slot_A[3 * s];
    const double an = std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    for (int k = 0; k < 3; ++k) sd.e[k] = A[k] / an;
    int axis = -1, sgn = 1;
    if (!is_unit_axis(sd.e, &axis, &sgn)) {
      axis = -1;
      C->all_axis = false;
    }
    sd.axis = axis;
    sd.sgn = sgn;
    sd.flip = -1;
    sd.wall_den = 0.0;
    const int g = C->slot_group[s];
    if (g < 0) {
      sd.kind = kInterior;
      sd.src = C->slot_nb[s];
    } else {
      switch (C->bc_type[g]) {
        case DVM_BC_ZEROGRAD:
          sd.kind = kZeroGrad;
          sd.src = (int32_t)(s / 6);
          break;
        case DVM_BC_SYMMETRY: {
          int ax = -1;
          for (int a = 0; a < 3; ++a)
            if (std::fabs(std::fabs(sd.e[a]) - 1.0) < 1e-12) ax = a;
          if (ax < 0 || C->vg.lo[ax] != -C->vg.hi[ax]) {
            set_error("symmetry needs a coordinate-plane face and a velocity grid symmetric about 0");
            return DVM_ERR_UNSUPPORTED;
          }
          sd.kind = kSymmetry;
          sd.flip = ax;
          sd.src = (int32_t)(s / 6);
          break;
        }
        case DVM_BC_FREESTREAM:
          sd.kind = kFreeStream;
          sd.src = C->group_ghost[g];
          break;
        case DVM_BC_WALL: {
          sd.kind = kWall;
          sd.src = C->group_ghost[g];
          auto key = std::make_tuple(g, sd.e[0], sd.e[1], sd.e[2]);
          need_den.emplace_back(s, key);
          den_cache[key] = 0.0;
          break;
        }
      }
    }
  }
  if (!den_cache.empty()) {
    double *d_tmp = nullptr;
    CTX_MALLOC(d_tmp, sizeof(double) * den_cache.size());
    size_t i = 0;
    std::map<std::tuple<int, double, double, double>, size_t> pos;
    for (auto &kv : den_cache) {
      const int g = std::get<0>(kv.first);
      const double e[3] = {std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first)};
      launch_inflow_sum(C->d_ghost + (size_t)C->group_ghost[g] * C->nn, C->d_xi[0], C->d_xi[1],
                        C->d_xi[2], C->N[0], C->N[1], C->N[2], e, d_tmp + i, C->stream);
      pos[kv.first] = i++;
    }
    std::vector<double> h(den_cache.size());
    DVM_CUDA_TRY(cudaMemcpyAsync(h.data(), d_tmp, sizeof(double) * h.size(),
                                 cudaMemcpyDeviceToHost, C->stream));
    int rc = sync_and_check(C);
    cudaFree(d_tmp);
    C->bytes -= sizeof(double) * den_cache.size();
    if (rc != DVM_OK) return rc;
    for (auto &sk : need_den) {
      const double d = h[pos[sk.second]];
      if (!(d < 0.0)) {
        set_error("wall Maxwellian has no inflow on this velocity grid");
        return DVM_ERR_INVALID_ARG;
      }
      C->slot[sk.first].wall_den = d;
    }
  }
  DVM_CUDA_TRY(cudaMemcpyAsync(C->d_slot, C->slot.data(), sizeof(SlotDev) * 6 * nc,
                               cudaMemcpyHostToDevice, C->stream));
  C->prepared = true;
  return sync_and_check(C);
}

// dt from the CFL rule on the current macroparameters, then the slot
// coefficients c = dt |A| / |V|.
static int finalize_dt(dvm_ctx *C, const std::vector<double> &macro, bool keep_dt) {
  const int64_t nc = C->nc;
  if (!keep_dt) {
    if (C->opts.dt > 0.0) {
      C->dt = C->opts.dt;
    } else {
      const double delta = std::sqrt(kPi) / (2.0 * C->gas.Kn);
      double worst = 0.0;
      for (int64_t c = 0; c < nc; ++c) {
        const double n = macro[8 * c], T = macro[8 * c + 4];
        if (!(n > 0.0) || !(T > 0.0)) {
          set_error("non-physical initial state (n or T <= 0)");
          return DVM_ERR_NONPHYSICAL;
        }
        double s = 0.0;
        for (int l = 0; l < 6; ++l) {
          const double *A = &C->slot_A[3 * (6 * c + l)];
          s += std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
        }
        const double rate = delta * n * std::pow(T, 1.0 - C->gas.omega) + s * C->xi_max / (2.0 * C->vol[c]);
        worst = std::max(worst, rate);
      }
      C->dt = C->opts.cfl / worst;
    }
  }
  for (int64_t s = 0; s < 6 * nc; ++s) {
    SlotDev &sd = C->slot[s];
    const double *A = &C->slot_A[3 * s];
    const double an = std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    sd.c = C->dt * an / C->vol[s / 6];
    for (int k = 0; k < 3; ++k) sd.ce[k] = sd.c * sd.e[k];
  }
  DVM_CUDA_TRY(cudaMemcpyAsync(C->d_slot, C->slot.data(), sizeof(SlotDev) * 6 * nc,
                               cudaMemcpyHostToDevice, C->stream));
  return sync_and_check(C);
}

static MomentParams moment_params(dvm_ctx *C, const double *f, double *sums, const double *uref) {
  MomentParams mp{};
  mp.f = f;
  mp.sums = sums;
  mp.uref = uref;
  mp.slot = C->d_slot;
  for (int a = 0; a < 3; ++a) mp.xi[a] = C->d_xi[a];
  mp.nc = C->nc;
  mp.N1 = C->N[0];
  mp.N2 = C->N[1];
  mp.N3 = C->N[2];
  return mp;
}

// moments of the full state about its own velocity (two passes), macro to host
static int full_moments_two_pass(dvm_ctx *C, std::vector<double> &macro) {
  const int64_t nc = C->nc;
  double *f = C->d_f[C->cur];
  launch_full_moments(moment_params(C, f, C->d_sums[C->cur], nullptr), C->stream);
  launch_macro_from_sums(C->d_sums[C->cur], C->d_macro, nc, C->w, C->stream);
  macro.resize(8 * nc);
  DVM_CUDA_TRY(cudaMemcpyAsync(macro.data(), C->d_macro, sizeof(double) * 8 * nc,
                               cudaMemcpyDeviceToHost, C->stream));
  int rc = sync_and_check(C);
  if (rc != DVM_OK) return rc;
  std::vector<double> u(3 * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) u[3 * c + k] = macro[8 * c + 1 + k];
  DVM_CUDA_TRY(cudaMemcpyAsync(C->d_uref, u.data(), sizeof(double) * 3 * nc,
                               cudaMemcpyHostToDevice, C->stream));
  launch_full_moments(moment_params(C, f, C->d_sums[C->cur], C->d_uref), C->stream);
  launch_macro_from_sums(C->d_sums[C->cur], C->d_macro, nc, C->w, C->stream);
  DVM_CUDA_TRY(cudaMemcpyAsync(macro.data(), C->d_macro, sizeof(double) * 8 * nc,
                               cudaMemcpyDeviceToHost, C->stream));
  return sync_and_check(C);
}

int ctx_init_from_maxwellians(dvm_ctx *C, const double *n, const double *u, const double *T) {
  const int64_t nc = C->nc;
  double *d_in = nullptr;
  CTX_MALLOC(d_in, sizeof(double) * 5 * nc);
  DVM_CUDA_TRY(cudaMemcpyAsync(d_in, n, sizeof(double) * nc, cudaMemcpyHostToDevice, C->stream));
  DVM_CUDA_TRY(cudaMemcpyAsync(d_in + nc, u, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, C->stream));
  DVM_CUDA_TRY(cudaMemcpyAsync(d_in + 4 * nc, T, sizeof(double) * nc, cudaMemcpyHostToDevice, C->stream));
  int rc = DVM_OK;
  if (C->opts.format == DVM_FORMAT_FULL) {
    launch_cell_maxwellians(C->d_f[C->cur], d_in, d_in + nc, d_in + 4 * nc, C->d_xi[0], C->d_xi[1],
                            C->d_xi[2], nc, C->N[0], C->N[1], C->N[2], C->stream);
    rc = sync_and_check(C);
  } else {
    // a Maxwellian is exactly rank 1 in Tucker format (Section 5)
    rc = tucker_init_maxwellians(C, d_in, d_in + nc, d_in + 4 * nc);
  }
  cudaFree(d_in);
  C->bytes -= sizeof(double) * 5 * nc;
  if (rc != DVM_OK) return rc;
  if (C->opts.format == DVM_FORMAT_TUCKER) {
    C->initialized = true;
    return DVM_OK;
  }
  std::vector<double> macro;
  rc = full_moments_two_pass(C, macro);
  if (rc != DVM_OK) return rc;
  rc = finalize_dt(C, macro, false);
  if (rc != DVM_OK) return rc;
  C->steps = 0;
  C->initialized = true;
  return DVM_OK;
}

int ctx_init_from_full(dvm_ctx *C, const double *f, bool on_device) {
  const size_t fb = sizeof(double) * (size_t)C->nc * C->nn;
  if (C->opts.format == DVM_FORMAT_TUCKER) {
    const double *src = f;
    double *d_full = nullptr;
    if (!on_device) {
      int rc = ctx_malloc(C, reinterpret_cast<void **>(&d_full), fb);
      if (rc != DVM_OK) return rc;
      DVM_CUDA_TRY(cudaMemcpyAsync(d_full, f, fb, cudaMemcpyHostToDevice, C->stream));
      src = d_full;
    }
    int rc = sync_and_check(C);
    if (rc == DVM_OK) rc = tucker_init_from_full(C, src);
    if (d_full) {
      cudaFree(d_full);
      C->bytes -= fb;
    }
    if (rc == DVM_OK) C->initialized = true;
    return rc;
  }
  DVM_CUDA_TRY(cudaMemcpyAsync(C->d_f[C->cur], f, fb,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               C->stream));
  std::vector<double> macro;
  int rc = full_moments_two_pass(C, macro);
  if (rc != DVM_OK) return rc;
  rc = finalize_dt(C, macro, C->initialized);
  if (rc != DVM_OK) return rc;
  C->initialized = true;
  return DVM_OK;
}

// the Tucker driver reuses the CFL rule
int ctx_finalize_dt_from_macro(dvm_ctx *C, const std::vector<double> &macro) {
  return finalize_dt(C, macro, false);
}

static int read_residual(dvm_ctx *C, double *residual_out) {
  int flag = 0;
  if (residual_out) {
    launch_residual_reduce(C->d_respart, C->nc, C->dt, C->d_res, C->stream);
    DVM_CUDA_TRY(cudaMemcpyAsync(residual_out, C->d_res, sizeof(double), cudaMemcpyDeviceToHost,
                                 C->stream));
  }
  DVM_CUDA_TRY(cudaMemcpyAsync(&flag, C->d_flag, sizeof(int), cudaMemcpyDeviceToHost, C->stream));
  int rc = sync_and_check(C);
  if (rc != DVM_OK) return rc;
  if (flag & 1) {
    set_error("non-physical state: n <= 0 or T <= 0 in some cell");
    return DVM_ERR_NONPHYSICAL;
  }
  if (flag & 2) {  // blocks returned without writing their results
    set_error("a bulk shared-memory copy did not complete within its wait limit: the step "
              "failed and the solver state is undefined (initialise again or load a checkpoint)");
    return DVM_ERR_TIMEOUT;
  }
  return DVM_OK;
}

// Wavefronts of one LU-SGS sweep over the cells in increasing (forward) or
// decreasing (backward) index order: a cell's wavefront is one more than the
// largest wavefront of its neighbours that come before it in the sweep, so the
// cells of one wavefront depend only on earlier wavefronts and can be updated
// in parallel with the result of the sequential sweep.  order[] lists the cells
// by wavefront (increasing index within one), off[w] .. off[w+1] is wavefront w.
void lusgs_wavefronts(int64_t nc, const int32_t *nb, bool forward, int32_t *order,
                      std::vector<int64_t> &off) {
  std::vector<int32_t> wave(nc, 0);
  int32_t nw = 0;
  for (int64_t k = 0; k < nc; ++k) {
    const int64_t i = forward ? k : nc - 1 - k;
    int32_t w = 0;
    for (int l = 0; l < 6; ++l) {
      const int64_t j = nb[6 * i + l];
      if (j >= 0 && (forward ? j < i : j > i)) w = std::max(w, wave[j] + 1);
    }
    wave[i] = w;
    nw = std::max(nw, w + 1);
  }
  off.assign((size_t)nw + 1, 0);
  for (int64_t i = 0; i < nc; ++i) off[wave[i] + 1]++;
  for (int32_t w = 0; w < nw; ++w) off[w + 1] += off[w];
  std::vector<int64_t> pos(off.begin(), off.end() - 1);
  for (int64_t i = 0; i < nc; ++i) order[pos[wave[i]]++] = (int32_t)i;
}

// One implicit step (LU-SGS): right-hand side, forward and backward sweeps by
// wavefront, then f^{n+1} = f^n + df with its moment sums.
static void lusgs_step(dvm_ctx *C, FullParams &P) {
  const LaunchTimer lt = C->timer();
  lt(kKFullStep, true, C->stream);
  P.dtnu = C->d_dtnu;
  launch_full_rhs(P, C->stream);
  LusgsParams L{};
  L.g = P.fnew;
  L.rD = C->d_rD;
  L.dtnu = C->d_dtnu;
  L.slot = C->d_slot;
  for (int a = 0; a < 3; ++a) L.xi[a] = C->d_xi[a];
  L.N1 = C->N[0];
  L.N2 = C->N[1];
  L.N3 = C->N[2];
  L.all_axis = C->all_axis ? 1 : 0;
  for (int s = 0; s < 2; ++s) {
    const std::vector<int64_t> &off = C->wave_off[s];
    for (size_t w = 0; w + 1 < off.size(); ++w) {
      L.cells = C->d_wave + s * C->nc + off[w];
      launch_lusgs_sweep(L, (int)(off[w + 1] - off[w]), s == 0, C->stream);
    }
  }
  launch_lusgs_apply(P, C->stream);
  lt(kKFullStep, false, C->stream);
}

// A new state starts with no device error recorded (the flag is sticky until then).
int ctx_clear_flag(dvm_ctx *C) {
  DVM_CUDA_TRY(cudaMemsetAsync(C->d_flag, 0, sizeof(int) * 4, C->stream));
  return DVM_OK;
}

int ctx_step(dvm_ctx *C, int32_t nsteps, double *residual_out) {
  if (fault_timeout()) {  // the device flag as a timed-out bulk-copy wait leaves it
    static const int kTimedOut = 2;
    DVM_CUDA_TRY(cudaMemcpyAsync(C->d_flag, &kTimedOut, sizeof(int), cudaMemcpyHostToDevice,
                                 C->stream));
  }
  if (C->opts.format == DVM_FORMAT_TUCKER) {
    int rc = tucker_step(C, nsteps, residual_out);
    if (rc != DVM_OK) return rc;
    return residual_out ? read_residual(C, residual_out) : DVM_OK;
  }
  FullParams P{};
  P.respart = C->d_respart;
  P.slot = C->d_slot;
  P.ghost = C->d_ghost;
  P.vol = C->d_vol;
  for (int a = 0; a < 3; ++a) P.xi[a] = C->d_xi[a];
  P.flag = C->d_flag;
  P.nc = C->nc;
  P.N1 = C->N[0];
  P.N2 = C->N[1];
  P.N3 = C->N[2];
  P.all_axis = C->all_axis ? 1 : 0;
  P.w = C->w;
  P.dt = C->dt;
  P.Pr = C->gas.Pr;
  P.omega = C->gas.omega;
  P.delta = std::sqrt(kPi) / (2.0 * C->gas.Kn);
  for (int32_t s = 0; s < nsteps; ++s) {
    P.f = C->d_f[C->cur];
    P.fnew = C->d_f[1 - C->cur];
    P.sums = C->d_sums[C->cur];
    P.sums_new = C->d_sums[1 - C->cur];
    if (C->opts.scheme == DVM_SCHEME_LUSGS) {
      lusgs_step(C, P);
    } else {
      const LaunchTimer lt = C->timer();
      lt(kKFullStep, true, C->stream);
      launch_full_step(P, C->stream);
      lt(kKFullStep, false, C->stream);
    }
    C->cur = 1 - C->cur;
    C->steps++;
  }
  DVM_CUDA_TRY(cudaGetLastError());
  if (nsteps == 0 && residual_out) {
    *residual_out = 0.0;
    return DVM_OK;
  }
  return residual_out ? read_residual(C, residual_out) : DVM_OK;
}

int ctx_moments(dvm_ctx *C, double *out) {
  if (C->opts.format == DVM_FORMAT_TUCKER) {
    int rc = tucker_moments(C, C->d_macro);
    if (rc != DVM_OK) return rc;
  } else {
    launch_macro_from_sums(C->d_sums[C->cur], C->d_macro, C->nc, C->w, C->stream);
  }
  DVM_CUDA_TRY(cudaMemcpyAsync(out, C->d_macro, sizeof(double) * 8 * C->nc,
                               cudaMemcpyDeviceToHost, C->stream));
  return sync_and_check(C);
}

int ctx_get_f(dvm_ctx *C, int64_t cell0, int64_t ncell, double *out) {
  const size_t bytes = sizeof(double) * (size_t)ncell * C->nn;
  if (ncell == 0) return DVM_OK;
  if (C->opts.format == DVM_FORMAT_TUCKER) {
    double *d_tmp = nullptr;
    int rc = ctx_malloc(C, reinterpret_cast<void **>(&d_tmp), bytes);
    if (rc != DVM_OK) return rc;
    rc = tucker_get_f(C, cell0, ncell, d_tmp);
    if (rc == DVM_OK) {
      cudaError_t e = cudaMemcpyAsync(out, d_tmp, bytes, cudaMemcpyDeviceToHost, C->stream);
      rc = (e == cudaSuccess) ? sync_and_check(C) : DVM_ERR_CUDA;
    }
    cudaFree(d_tmp);
    C->bytes -= bytes;
    return rc;
  }
  DVM_CUDA_TRY(cudaMemcpyAsync(out, C->d_f[C->cur] + (size_t)cell0 * C->nn, bytes,
                               cudaMemcpyDeviceToHost, C->stream));
  return sync_and_check(C);
}

int ctx_get_ranks(dvm_ctx *C, int32_t *r) {
  if (C->opts.format == DVM_FORMAT_TUCKER) return tucker_get_ranks(C, r);
  for (int64_t c = 0; c < C->nc; ++c)
    for (int a = 0; a < 3; ++a) r[3 * c + a] = C->N[a];
  return DVM_OK;
}

int ctx_memory(dvm_ctx *C, size_t *f_bytes, size_t *total_bytes) {
  if (f_bytes) {
    if (C->opts.format == DVM_FORMAT_TUCKER) {
      int rc = tucker_memory(C, f_bytes);
      if (rc != DVM_OK) return rc;
    } else {
      *f_bytes = sizeof(double) * (size_t)C->nc * C->nn;
    }
  }
  if (total_bytes) *total_bytes = C->bytes;
  return DVM_OK;
}

namespace {
struct CkptHeader {
  uint64_t magic;
  int32_t format, N[3];
  int64_t nc, steps;
  double dt;
  int32_t cur_pad[2];
};
}  // namespace

int ctx_save(dvm_ctx *C, const char *path) {
  FILE *fp = std::fopen(path, "wb");
  if (!fp) {
    set_error(std::string("cannot open ") + path);
    return DVM_ERR_IO;
  }
  CkptHeader h{};
  h.magic = kCkptMagic;
  h.format = C->opts.format;
  for (int a = 0; a < 3; ++a) h.N[a] = C->N[a];
  h.nc = C->nc;
  h.steps = C->steps;
  h.dt = C->dt;
  int rc = DVM_OK;
  if (std::fwrite(&h, sizeof h, 1, fp) != 1) rc = DVM_ERR_IO;
  if (rc == DVM_OK && C->opts.format == DVM_FORMAT_FULL) {
    const size_t n1 = (size_t)C->nc * C->nn, n2 = (size_t)C->nc * kSums;
    std::vector<double> buf(n1 > n2 ? n1 : n2);
    if (cudaMemcpy(buf.data(), C->d_f[C->cur], sizeof(double) * n1, cudaMemcpyDeviceToHost) != cudaSuccess ||
        std::fwrite(buf.data(), sizeof(double), n1, fp) != n1)
      rc = DVM_ERR_IO;
    if (rc == DVM_OK &&
        (cudaMemcpy(buf.data(), C->d_sums[C->cur], sizeof(double) * n2, cudaMemcpyDeviceToHost) != cudaSuccess ||
         std::fwrite(buf.data(), sizeof(double), n2, fp) != n2))
      rc = DVM_ERR_IO;
  } else if (rc == DVM_OK) {
    rc = tucker_save(C, fp);
  }
  std::fclose(fp);
  if (rc != DVM_OK && dvm_last_error()[0] == 0) set_error("checkpoint write failed");
  return rc;
}

int ctx_load(dvm_ctx *C, const char *path) {
  FILE *fp = std::fopen(path, "rb");
  if (!fp) {
    set_error(std::string("cannot open ") + path);
    return DVM_ERR_IO;
  }
  CkptHeader h{};
  int rc = DVM_OK;
  if (std::fread(&h, sizeof h, 1, fp) != 1 || h.magic != kCkptMagic || h.format != C->opts.format ||
      h.nc != C->nc || h.N[0] != C->N[0] || h.N[1] != C->N[1] || h.N[2] != C->N[2]) {
    set_error("checkpoint does not match this context");
    std::fclose(fp);
    return DVM_ERR_IO;
  }
  C->dt = h.dt;
  C->steps = h.steps;
  if (C->opts.format == DVM_FORMAT_FULL) {
    const size_t n1 = (size_t)C->nc * C->nn, n2 = (size_t)C->nc * kSums;
    std::vector<double> buf(n1 > n2 ? n1 : n2);
    if (std::fread(buf.data(), sizeof(double), n1, fp) != n1 ||
        cudaMemcpy(C->d_f[C->cur], buf.data(), sizeof(double) * n1, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = DVM_ERR_IO;
    if (rc == DVM_OK && (std::fread(buf.data(), sizeof(double), n2, fp) != n2 ||
                         cudaMemcpy(C->d_sums[C->cur], buf.data(), sizeof(double) * n2,
                                    cudaMemcpyHostToDevice) != cudaSuccess))
      rc = DVM_ERR_IO;
  } else {
    rc = tucker_load(C, fp);
  }
  std::fclose(fp);
  if (rc != DVM_OK) {
    if (dvm_last_error()[0] == 0) set_error("checkpoint read failed");
    return rc;
  }
  std::vector<double> unused;
  rc = finalize_dt(C, unused, true);
  if (rc != DVM_OK) return rc;
  C->initialized = true;
  return DVM_OK;
}

// Enqueue the residual of the last step and the non-physical flag into
// pinned host memory (out[0] = residual, low bytes of out[1] = flag) on the
// context's stream, without synchronising.
int ctx_enqueue_residual(dvm_ctx *C, double *pinned_out) {
  launch_residual_reduce(C->d_respart, C->nc, C->dt, C->d_res, C->stream);
  DVM_CUDA_TRY(cudaMemcpyAsync(pinned_out, C->d_res, sizeof(double), cudaMemcpyDeviceToHost,
                               C->stream));
  DVM_CUDA_TRY(cudaMemcpyAsync(pinned_out + 1, C->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                               C->stream));
  return DVM_OK;
}
