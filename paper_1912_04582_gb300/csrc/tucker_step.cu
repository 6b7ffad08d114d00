// Tucker-format driver: state allocation, initialisation (rank-1 Maxwellians or
// HOSVD of full tensors), time stepping, moments, inspection and checkpoints.
// Kernels: tucker_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "dvm_context.h"
#include "tucker.h"

using namespace dvm;

struct TuckerState {
  TuckerDev buf[2]{};
  int cur = 0;
  int scur = 0;        // index of the moment-sum buffer of the current state
  int R = 0;
  int Nmax = 0;
  bool fp64 = true;
  void *scratch = nullptr;
  size_t stride = 0;   // scratch elements per CTA
  int grid = 0;
  double *ghostf = nullptr;  // [nghost][3][Nmax]
  float *ghostf32 = nullptr; // the same in FP32 (mixed-precision assembly)
  double *err = nullptr;     // [nc]
  long long *phase = nullptr;  // [16] per-phase cycles (DVM_TUCKER_PHASES set)
  int max_grid = 0;             // CTAs the scratch is sized for
  bool tuned = false;           // grid picked by the autotuner
  bool retuned = false;         // picked again once the state has developed
  int64_t tuned_step = 0;       // step counter at the first tuning
  float tune_ms[5] = {0, 0, 0, 0, 0};  // [0] phase-major step, [1..4] fused kernel per CTAs/SM
  bool split = false;                  // phase-major variant chosen
  bool gemm_asm = false;               // its assembly may take the GEMM form
  int fit = 3;                         // variants whose kernels fit: 1 fused, 2 phase-major
  TuckerSplitBufs sb{};                // its work buffers (one chunk of cells)
  int64_t chunk = 0;                   // cells per chunk
  void *split_mem = nullptr;
  size_t split_bytes = 0;
  SplitStreams ss{};                   // second stream of the phase-major step
  cudaGraphExec_t graph = nullptr;     // two steps (returns to the same buffer parity)
  int graph_parity = -1;               // S->cur / S->scur when the graph was captured
  cudaStream_t gstream = nullptr;      // private stream the graph is captured on / replayed on
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // hand-offs with the caller's stream
};

int ctx_finalize_dt_from_macro(dvm_ctx *C, const std::vector<double> &macro);

namespace {

// launch errors with the place they surfaced
int launch_check(const char *where) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return DVM_OK;
  set_error(std::string("Tucker step (") + where + "): " + cudaGetErrorString(e));
  return DVM_ERR_CUDA;
}

int sync_check(dvm_ctx *C) {
  DVM_CUDA_TRY(cudaGetLastError());
  DVM_CUDA_TRY(cudaStreamSynchronize(C->stream));
  return DVM_OK;
}

TuckerStepParams step_params(dvm_ctx *C) {
  TuckerState *S = C->tucker;
  TuckerStepParams p{};
  p.slot = C->d_slot;
  p.ghostf = S->ghostf;
  p.ghostf32 = S->ghostf32;
  for (int a = 0; a < 3; ++a) p.xi[a] = C->d_xi[a];
  p.err = S->err;
  p.phase = S->phase;
  p.flag = C->d_flag;
  p.scratch = S->scratch;
  p.scratch_stride = S->stride;
  p.nc = C->nc;
  p.N1 = C->N[0];
  p.N2 = C->N[1];
  p.N3 = C->N[2];
  p.R = S->R;
  p.Nmax = S->Nmax;
  p.w = C->w;
  p.dt = C->dt;
  p.Pr = C->gas.Pr;
  p.omega = C->gas.omega;
  p.delta = std::sqrt(3.14159265358979323846) / (2.0 * C->gas.Kn);
  p.tol = C->opts.tol;
  p.tc_gram = !S->fp64 && C->opts.engine == DVM_ENGINE_AUTO &&
              gram_tc_supported(C->N[0], C->N[1] * C->N[2]);
  p.gemm_asm = S->gemm_asm && C->all_axis;
  return p;
}

TuckerMomentParams moment_params(dvm_ctx *C, const TuckerDev &T, double *sums) {
  TuckerMomentParams m{};
  m.T = T;
  m.slot = C->d_slot;
  for (int a = 0; a < 3; ++a) m.xi[a] = C->d_xi[a];
  m.sums = sums;
  m.vol = C->d_vol;
  m.flag = C->d_flag;
  m.nc = C->nc;
  m.N1 = C->N[0];
  m.N2 = C->N[1];
  m.N3 = C->N[2];
  m.R = C->tucker->R;
  m.w = C->w;
  return m;
}

// moments of the current state about its own velocity: pass 1 about 0, pass 2
// about the pass-1 velocity; macro to host
int two_pass_moments(dvm_ctx *C, std::vector<double> &macro) {
  TuckerState *S = C->tucker;
  const int64_t nc = C->nc;
  TuckerMomentParams m = moment_params(C, S->buf[S->cur], C->d_sums[S->scur]);
  launch_tucker_moments(m, C->stream);
  launch_macro_from_sums(C->d_sums[S->scur], C->d_macro, nc, C->w, C->stream);
  m.uref = C->d_macro + 1;
  m.uref_stride = 8;
  m.sums = C->d_sums[1 - S->scur];
  launch_tucker_moments(m, C->stream);
  S->scur = 1 - S->scur;
  launch_macro_from_sums(C->d_sums[S->scur], C->d_macro, nc, C->w, C->stream);
  macro.resize(8 * nc);
  DVM_CUDA_TRY(cudaMemcpyAsync(macro.data(), C->d_macro, sizeof(double) * 8 * nc,
                               cudaMemcpyDeviceToHost, C->stream));
  return sync_check(C);
}

int build_ghost_factors(dvm_ctx *C) {
  TuckerState *S = C->tucker;
  if (S->ghostf) {
    cudaFree(S->ghostf);
    S->ghostf = nullptr;
  }
  const int ng = std::max(C->nghost, 1);
  std::vector<double> h((size_t)ng * 3 * S->Nmax, 0.0);
  const double pi = 3.14159265358979323846;
  for (int g = 0; g < kMaxGroups; ++g) {
    const int k = C->group_ghost.empty() ? -1 : C->group_ghost[g];
    if (k < 0) continue;
    const auto &p = C->bc_par[g];
    const double n = C->bc_type[g] == DVM_BC_WALL ? 1.0 : p[0];
    const double T = p[4];
    const double amp = std::cbrt(n) / std::sqrt(pi * T);
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < C->N[a]; ++i) {
        const double v = C->xi[a][i] - p[1 + a];
        h[((size_t)k * 3 + a) * S->Nmax + i] = amp * std::exp(-v * v / T);
      }
  }
  int rc = ctx_malloc(C, reinterpret_cast<void **>(&S->ghostf), sizeof(double) * h.size());
  if (rc != DVM_OK) return rc;
  DVM_CUDA_TRY(cudaMemcpyAsync(S->ghostf, h.data(), sizeof(double) * h.size(),
                               cudaMemcpyHostToDevice, C->stream));
  if (S->ghostf32) {
    cudaFree(S->ghostf32);
    S->ghostf32 = nullptr;
  }
  std::vector<float> h32(h.begin(), h.end());
  rc = ctx_malloc(C, reinterpret_cast<void **>(&S->ghostf32), sizeof(float) * h32.size());
  if (rc != DVM_OK) return rc;
  DVM_CUDA_TRY(cudaMemcpyAsync(S->ghostf32, h32.data(), sizeof(float) * h32.size(),
                               cudaMemcpyHostToDevice, C->stream));
  return sync_check(C);
}

int check_tucker_faces(dvm_ctx *C) {
  for (int64_t s = 0; s < 6 * C->nc; ++s)
    if (C->slot[s].kind == kWall && C->slot[s].axis < 0) {
      set_error("Tucker format: diffuse walls must lie on coordinate planes");
      return DVM_ERR_UNSUPPORTED;
    }
  return DVM_OK;
}

int finish_init(dvm_ctx *C) {
  int rc = check_tucker_faces(C);
  if (rc != DVM_OK) return rc;
  rc = build_ghost_factors(C);
  if (rc != DVM_OK) return rc;
  std::vector<double> macro;
  rc = two_pass_moments(C, macro);
  if (rc != DVM_OK) return rc;
  if (!C->initialized) {
    rc = ctx_finalize_dt_from_macro(C, macro);
    if (rc != DVM_OK) return rc;
    C->steps = 0;
  }
  for (int64_t c = 0; c < C->nc; ++c)
    if (!(macro[8 * c] > 0.0) || !(macro[8 * c + 4] > 0.0)) {
      set_error("non-physical initial state (n or T <= 0)");
      return DVM_ERR_NONPHYSICAL;
    }
  return DVM_OK;
}

}  // namespace

int tucker_alloc(dvm_ctx *C) {
  TuckerState *S = new TuckerState();
  C->tucker = S;
  S->R = C->opts.rank_cap;
  S->Nmax = std::max(C->N[0], std::max(C->N[1], C->N[2]));
  S->fp64 = C->opts.precision == DVM_PREC_FP64;
  if (S->Nmax > 64) {
    set_error("Tucker format supports at most 64 velocity nodes per axis");
    return DVM_ERR_UNSUPPORTED;
  }
  const int64_t nc = C->nc;
  const int R = S->R;
  for (int b = 0; b < 2; ++b) {
    TuckerDev &T = S->buf[b];
    int rc = ctx_malloc(C, reinterpret_cast<void **>(&T.core), sizeof(double) * nc * R * R * R);
    if (rc != DVM_OK) return rc;
    for (int a = 0; a < 3; ++a) {
      rc = ctx_malloc(C, reinterpret_cast<void **>(&T.fac[a]),
                      sizeof(double) * nc * (int64_t)C->N[a] * R);
      if (rc != DVM_OK) return rc;
      DVM_CUDA_TRY(cudaMemset(T.fac[a], 0, sizeof(double) * nc * (int64_t)C->N[a] * R));
    }
    rc = ctx_malloc(C, reinterpret_cast<void **>(&T.rank), sizeof(int) * 3 * nc);
    if (rc != DVM_OK) return rc;
    DVM_CUDA_TRY(cudaMemset(T.core, 0, sizeof(double) * nc * R * R * R));
    DVM_CUDA_TRY(cudaMemset(T.rank, 0, sizeof(int) * 3 * nc));
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C->device);
  const int per_sm = std::min(4, tucker_step_blocks_per_sm(S->Nmax, R, S->fp64));
  S->grid = (int)std::min<int64_t>(nc, (int64_t)sms * per_sm);
  S->max_grid = S->grid;
  S->stride = tucker_scratch_elems(C->N[0], C->N[1], C->N[2], R);
  S->stride = (S->stride + 63) & ~size_t(63);
  const size_t es = S->fp64 ? sizeof(double) : sizeof(float);
  int rc = ctx_malloc(C, &S->scratch, es * S->stride * S->grid);
  if (rc != DVM_OK) return rc;
  rc = ctx_malloc(C, reinterpret_cast<void **>(&S->err), sizeof(double) * nc);
  if (rc != DVM_OK) return rc;
  DVM_CUDA_TRY(cudaMemset(S->err, 0, sizeof(double) * nc));
  S->fit = tucker_prepare_launch(S->Nmax, R, S->fp64);
  // the assembly in GEMM form (used on meshes whose faces all lie on coordinate planes,
  // known once the boundaries are set up: each face weight then depends on one velocity
  // coordinate)
  S->gemm_asm = !S->fp64 && C->opts.engine == DVM_ENGINE_AUTO &&
                tucker_asm_gemm_prepare(S->Nmax, C->N[0], R) == 0;
  if (!S->fp64 && C->opts.engine == DVM_ENGINE_AUTO &&
      gram_tc_supported(C->N[0], C->N[1] * C->N[2]) && gram_tc_prepare(C->N[0]) != 0) {
    set_error("tensor-core Gram kernel: shared-memory opt-in refused by the device");
    return DVM_ERR_UNSUPPORTED;
  }
  const int need = C->opts.variant == DVM_VARIANT_FUSED ? 1 :
                   C->opts.variant == DVM_VARIANT_PHASED ? 2 : 3;
  if (!(S->fit & need)) {
    set_error("Tucker kernels of the requested launch variant need more shared memory than "
              "the device allows (lower the rank cap or use the other variant)");
    return DVM_ERR_UNSUPPORTED;
  }
  if (std::getenv("DVM_TUCKER_PHASES")) {
    rc = ctx_malloc(C, reinterpret_cast<void **>(&S->phase), sizeof(long long) * 32);
    if (rc != DVM_OK) return rc;
    DVM_CUDA_TRY(cudaMemset(S->phase, 0, sizeof(long long) * 32));
  }
  return DVM_OK;
}

void tucker_free(dvm_ctx *C) {
  TuckerState *S = C->tucker;
  if (!S) return;
  for (int b = 0; b < 2; ++b) {
    if (S->buf[b].core) cudaFree(S->buf[b].core);
    for (int a = 0; a < 3; ++a)
      if (S->buf[b].fac[a]) cudaFree(S->buf[b].fac[a]);
    if (S->buf[b].rank) cudaFree(S->buf[b].rank);
  }
  if (S->graph) cudaGraphExecDestroy(S->graph);
  if (S->gstream) cudaStreamDestroy(S->gstream);
  if (S->ev_in) cudaEventDestroy(S->ev_in);
  if (S->ev_out) cudaEventDestroy(S->ev_out);
  if (S->scratch) cudaFree(S->scratch);
  if (S->split_mem) cudaFree(S->split_mem);
  for (int w = 0; w < kMaxWays - 1; ++w) {
    if (S->ss.sx[w]) cudaStreamDestroy(S->ss.sx[w]);
    if (S->ss.join[w]) cudaEventDestroy(S->ss.join[w]);
  }
  if (S->ss.fork) cudaEventDestroy(S->ss.fork);
  if (S->ghostf) cudaFree(S->ghostf);
  if (S->ghostf32) cudaFree(S->ghostf32);
  if (S->err) cudaFree(S->err);
  if (S->phase) {
    long long h[32] = {0};
    if (cudaMemcpy(h, S->phase, sizeof h, cudaMemcpyDeviceToHost) == cudaSuccess) {
      // fused kernel / eigen-solve kernel; 16-26: the tensor-core Gram kernel's roles
      static const char *names[32] = {
          "prologue", "reseeds", "retries", "assemble|asm_terms", "energy|setup", "gram|asm_eq",
          "eig_init", "rank", "project|retry", "eig_cq32", "eig_orth32", "eig_cq64", "eig_orth64",
          "contract", "rayleigh", "sort", "gtc_tma_wait", "gtc_mma_wait_ready", "gtc_mma_issue",
          "gtc_mma_wait_readback", "gtc_slice_wait_load", "gtc_slice_wait_freed", "gtc_slice",
          "gtc_readback", "gtc_wait_accum", "gtc_cells", "gtc_total", "", "", "", "", ""};
      std::fprintf(stderr, "tucker phases (SM cycles summed over CTAs; reseeds, retries, cells: counts):");
      for (int i = 0; i < 27; ++i) std::fprintf(stderr, " %s=%lld", names[i], h[i]);
      std::fprintf(stderr, "\n");
    }
    cudaFree(S->phase);
  }
  delete S;
  C->tucker = nullptr;
}

int tucker_init_maxwellians(dvm_ctx *C, const double *d_n, const double *d_u, const double *d_T) {
  TuckerState *S = C->tucker;
  launch_tucker_maxwellians(S->buf[S->cur], d_n, d_u, d_T, C->d_xi[0], C->d_xi[1], C->d_xi[2],
                            C->nc, C->N[0], C->N[1], C->N[2], S->R, C->stream);
  int rc = sync_check(C);
  if (rc != DVM_OK) return rc;
  return finish_init(C);
}

// The Tucker state given directly (host or device arrays in the arena layout:
// ranks [nc][3], core [nc][R^3] with the r1 x r2 x r3 core at the front, factor
// a [nc][N_a][R] with the first r_a columns used).
int tucker_set_state(dvm_ctx *C, const int32_t *ranks, const double *core,
                     const double *const fac[3], bool on_device) {
  TuckerState *S = C->tucker;
  const int64_t nc = C->nc;
  const int R = S->R;
  std::vector<int32_t> r(3 * nc);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (on_device) {
    DVM_CUDA_TRY(cudaMemcpyAsync(r.data(), ranks, sizeof(int32_t) * 3 * nc,
                                 cudaMemcpyDeviceToHost, C->stream));
    int rc = sync_check(C);
    if (rc != DVM_OK) return rc;
  } else {
    std::copy(ranks, ranks + 3 * nc, r.begin());
  }
  for (int64_t i = 0; i < 3 * nc; ++i)
    if (r[i] < 1 || r[i] > R || r[i] > C->N[i % 3]) {
      set_error("dvm_init_tucker: ranks must lie in 1 .. min(N_a, rank cap)");
      return DVM_ERR_INVALID_ARG;
    }
  TuckerDev &T = S->buf[S->cur];
  DVM_CUDA_TRY(cudaMemcpyAsync(T.rank, ranks, sizeof(int32_t) * 3 * nc, kind, C->stream));
  DVM_CUDA_TRY(cudaMemcpyAsync(T.core, core, sizeof(double) * nc * R * R * R, kind, C->stream));
  for (int a = 0; a < 3; ++a)
    DVM_CUDA_TRY(cudaMemcpyAsync(T.fac[a], fac[a], sizeof(double) * nc * (int64_t)C->N[a] * R,
                                 kind, C->stream));
  int rc = sync_check(C);
  if (rc != DVM_OK) return rc;
  return finish_init(C);
}

int tucker_get_state(dvm_ctx *C, int32_t *ranks, double *core, double *const fac[3]) {
  TuckerState *S = C->tucker;
  const int64_t nc = C->nc;
  const int R = S->R;
  const TuckerDev &T = S->buf[S->cur];
  if (ranks)
    DVM_CUDA_TRY(cudaMemcpyAsync(ranks, T.rank, sizeof(int32_t) * 3 * nc, cudaMemcpyDeviceToHost,
                                 C->stream));
  if (core)
    DVM_CUDA_TRY(cudaMemcpyAsync(core, T.core, sizeof(double) * nc * R * R * R,
                                 cudaMemcpyDeviceToHost, C->stream));
  for (int a = 0; a < 3; ++a)
    if (fac[a])
      DVM_CUDA_TRY(cudaMemcpyAsync(fac[a], T.fac[a], sizeof(double) * nc * (int64_t)C->N[a] * R,
                                   cudaMemcpyDeviceToHost, C->stream));
  return sync_check(C);
}

int tucker_init_from_full(dvm_ctx *C, const double *d_f_full) {
  TuckerState *S = C->tucker;
  TuckerStepParams p = step_params(C);
  p.mode = 1;
  p.finit = d_f_full;
  p.nxt = S->buf[S->cur];
  if (launch_tucker_step(p, S->grid, S->fp64, C->stream) != 0) {
    set_error("Tucker kernel needs more shared memory than the device allows");
    return DVM_ERR_UNSUPPORTED;
  }
  int rc = sync_check(C);
  if (rc != DVM_OK) return rc;
  return finish_init(C);
}

namespace {

// one explicit step: step kernel (cur -> nxt), then the moments of the new
// state about the previous velocity (with the residual parts)
int enqueue_one_step(dvm_ctx *C, TuckerStepParams &p) {
  TuckerState *S = C->tucker;
  p.mode = 0;
  p.cur = S->buf[S->cur];
  p.nxt = S->buf[1 - S->cur];
  p.sums = C->d_sums[S->scur];
  const LaunchTimer lt = C->timer();
  // the moments of the new state are taken about the current state's velocity
  // (from the current sums, untouched by the step)
  TuckerMomentParams m = moment_params(C, p.nxt, C->d_sums[1 - S->scur]);
  m.uref = C->d_macro + 1;
  m.uref_stride = 8;
  m.sums_prev = C->d_sums[S->scur];
  m.respart = C->d_respart;
  int lrc;
  if (S->split) {  // the split step forms the macroparameters (S->sb.macro) first
    lrc = launch_tucker_split_step(p, S->sb, S->chunk, S->fp64, C->stream, &lt, &S->ss, &m);
  } else {
    lt(kKFusedStep, true, C->stream);
    lrc = launch_tucker_step(p, S->grid, S->fp64, C->stream);
    lt(kKFusedStep, false, C->stream);
    if (lrc == 0) {
      lt(kKMoments, true, C->stream);
      launch_macro_from_sums(C->d_sums[S->scur], C->d_macro, C->nc, C->w, C->stream);
      lt(kKMoments, false, C->stream);
      lt(kKMoments, true, C->stream);
      launch_tucker_moments(m, C->stream);
      lt(kKMoments, false, C->stream);
    }
  }
  if (lrc != 0) {
    set_error("Tucker kernel needs more shared memory than the device allows");
    return DVM_ERR_UNSUPPORTED;
  }
  S->cur = 1 - S->cur;
  S->scur = 1 - S->scur;
  return DVM_OK;
}

// Work buffers of the phase-major variant for a chunk of at most 1/8 of the
// free device memory (at most all cells).
int alloc_split(dvm_ctx *C) {
  TuckerState *S = C->tucker;
  size_t free_b = 0, total_b = 0;
  DVM_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const size_t es = S->fp64 ? sizeof(double) : sizeof(float);
  const size_t per =
      tucker_split_bytes_per_cell(C->N[0], C->N[1], C->N[2], S->R, S->Nmax, S->fp64) + 64;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C->device);
  const size_t t2_stride = (tucker_split_t2_elems(C->N[0], C->N[1], C->N[2], S->R) + 63) & ~size_t(63);
  int64_t chunk = std::min<int64_t>(C->nc, (int64_t)(free_b / 8 / per));
  if (C->opts.max_chunk > 0) chunk = std::min<int64_t>(chunk, C->opts.max_chunk);
  if (chunk < 1) {
    set_error("no device memory for the phase-major Tucker step buffers");
    return DVM_ERR_OOM;
  }
  (void)t2_stride;
  const int asm_grid = (int)std::min<int64_t>(chunk, (int64_t)sms * tucker_split_asm_per_sm());
  const size_t t2all = tucker_split_t2all_bytes_per_cell(C->N[0], C->N[1], C->N[2], S->R, S->fp64);
  const size_t bytes = per * chunk + t2all * C->nc + 512;
  void *mem = nullptr;
  int rc = ctx_malloc(C, &mem, bytes);
  if (rc != DVM_OK) return rc;
  char *q = static_cast<char *>(mem);
  TuckerSplitBufs b{};
  b.t2 = nullptr;  // the assembly reads the all-cell contractions instead
  b.t2_stride = 0;
  b.asm_grid = asm_grid;
  b.cellpar = reinterpret_cast<double *>(q);  // first: 8-byte aligned
  q += sizeof(double) * kCellPar * (size_t)C->nc;
  b.macro = C->d_macro;
  b.T2all = q;
  q += es * (size_t)C->nc * S->R * C->N[1] * C->N[2];
  b.U1all = q;
  q += t2all * C->nc - es * (size_t)C->nc * S->R * C->N[1] * C->N[2] -
       sizeof(double) * kCellPar * (size_t)C->nc;
  q = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(q) + 255) & ~uintptr_t(255));
  b.X = q;
  q += es * chunk * C->N[0] * C->N[1] * C->N[2];
  b.Y1 = q;
  q += es * chunk * S->R * C->N[1] * C->N[2];
  b.Y2 = q;
  q += es * chunk * S->R * S->R * C->N[2];
  q = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(q) + 255) & ~uintptr_t(255));
  b.C = reinterpret_cast<double *>(q);
  q += sizeof(double) * chunk * S->Nmax * S->Nmax;
  b.e = reinterpret_cast<double *>(q);
  q += sizeof(double) * chunk;
  b.disc = reinterpret_cast<double *>(q);
  q += sizeof(double) * chunk;
  // first-mode row maxima of X, for the tensor-core Gram matrices of the mixed path
  b.rowmax = (!S->fp64 && C->opts.engine == DVM_ENGINE_AUTO &&
              gram_tc_supported(C->N[0], C->N[1] * C->N[2]))
                 ? reinterpret_cast<float *>(q)
                 : nullptr;
  S->sb = b;
  S->chunk = chunk;
  S->split_mem = mem;
  S->split_bytes = bytes;
  if (!S->ss.fork) {
    DVM_CUDA_TRY(cudaEventCreateWithFlags(&S->ss.fork, cudaEventDisableTiming));
    for (int w = 0; w < kMaxWays - 1; ++w) {
      DVM_CUDA_TRY(cudaStreamCreateWithFlags(&S->ss.sx[w], cudaStreamNonBlocking));
      DVM_CUDA_TRY(cudaEventCreateWithFlags(&S->ss.join[w], cudaEventDisableTiming));
    }
    S->ss.ways = 2;  // measured on the cavity: 2, 3 and 4 ranges all within 1%
  }
  return DVM_OK;
}

void free_split(dvm_ctx *C) {
  TuckerState *S = C->tucker;
  if (!S->split_mem) return;
  cudaFree(S->split_mem);
  C->bytes -= std::min(C->bytes, S->split_bytes);
  S->split_mem = nullptr;
  S->chunk = 0;
}

constexpr int64_t kRetuneSteps = 16;

// Autotuner, on the first step: time the fused step kernel once for each
// resident-CTAs-per-SM choice the scratch allows and, unless the variant is
// fixed, the phase-major step; keep the fastest.  Tuning launches write into the
// spare buffer, so the state is untouched (a cell's arithmetic does not depend
// on which CTA or variant runs it).  Meshes with no more cells than SMs keep the
// fused kernel at one cell per CTA unless the phase-major variant is requested.
int autotune(dvm_ctx *C) {
  TuckerState *S = C->tucker;
  S->tuned = true;
  S->tuned_step = C->steps;
  const int variant = C->opts.variant;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C->device);
  const bool fused_fits = (S->fit & 1) != 0;
  const bool phased = variant == DVM_VARIANT_PHASED || !fused_fits;
  const bool small = C->nc <= sms || std::getenv("DVM_NO_AUTOTUNE") || !fused_fits;
  if (small && !phased) return DVM_OK;
  TuckerStepParams p = step_params(C);
  p.mode = 0;
  p.cur = S->buf[S->cur];
  p.nxt = S->buf[1 - S->cur];
  p.sums = C->d_sums[S->scur];
  p.phase = nullptr;
  cudaEvent_t e0, e1;
  DVM_CUDA_TRY(cudaEventCreate(&e0));
  DVM_CUDA_TRY(cudaEventCreate(&e1));
  auto timed = [&](auto &&launch) -> float {
    if (launch() != 0) return -1.f;  // warm-up
    cudaEventRecord(e0, C->stream);
    launch();
    cudaEventRecord(e1, C->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  float best = 1e30f;
  int best_grid = S->grid;
  for (int per_sm = 1; per_sm <= 4 && !small; ++per_sm) {
    const int grid = (int)std::min<int64_t>(C->nc, (int64_t)sms * per_sm);
    if (grid > S->max_grid) break;
    const float ms = timed([&] { return launch_tucker_step(p, grid, S->fp64, C->stream); });
    if (ms < 0.f) break;
    S->tune_ms[per_sm] = ms;
    if (ms < best) {
      best = ms;
      best_grid = grid;
    }
  }
  S->grid = best_grid;
  int rc = DVM_OK;
  if (variant != DVM_VARIANT_FUSED && (phased || !std::getenv("DVM_NO_SPLIT"))) {
    rc = S->split_mem ? DVM_OK : alloc_split(C);
    if (rc == DVM_OK) {
      const float ms = timed([&] {
        return launch_tucker_split_step(p, S->sb, S->chunk, S->fp64, C->stream, nullptr, &S->ss);
      });
      if (ms > 0.f) S->tune_ms[0] = ms;
      S->split = phased || (ms > 0.f && ms < best);
      if (!S->split) free_split(C);
    } else if (!phased) {
      rc = DVM_OK;  // no memory for the buffers: keep the fused kernel
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DVM_OK) return rc;
  DVM_CUDA_TRY(cudaGetLastError());
  return DVM_OK;
}

}  // namespace

int tucker_step(dvm_ctx *C, int32_t nsteps, double *residual_out) {
  (void)residual_out;
  TuckerState *S = C->tucker;
  // the variant is picked on the first step and once more after kRetuneSteps
  // steps, when the ranks (and with them the cost of each variant) have developed
  if (!S->tuned || (!S->retuned && C->steps >= S->tuned_step + kRetuneSteps)) {
    if (S->tuned) {
      S->retuned = true;
      if (S->graph) {  // re-captured with the variant chosen now
        DVM_CUDA_TRY(cudaStreamSynchronize(S->gstream));
        cudaGraphExecDestroy(S->graph);
        S->graph = nullptr;
      }
    }
    int rc = launch_check("before the autotuner");
    if (rc == DVM_OK) rc = autotune(C);
    if (rc == DVM_OK) rc = launch_check("autotuner");
    if (rc != DVM_OK) return rc;
  }
  TuckerStepParams p = step_params(C);
  int32_t s = 0;
  // pairs of steps replay a captured CUDA graph (launch overhead paid once per
  // pair); the graph is re-captured if the buffer parity differs
  const bool use_graph =
      nsteps >= 2 && !S->phase && !C->timing.on && !std::getenv("DVM_NO_GRAPH");
  if (use_graph) {
    if (!S->gstream) {
      DVM_CUDA_TRY(cudaStreamCreateWithFlags(&S->gstream, cudaStreamNonBlocking));
      DVM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
      DVM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming));
    }
    const int parity = S->cur * 2 + S->scur;
    if (!S->graph || S->graph_parity != parity) {
      if (S->graph) {
        cudaGraphExecDestroy(S->graph);
        S->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaStream_t user = C->stream;
      C->stream = S->gstream;  // capture the launches on the private stream
      DVM_CUDA_TRY(cudaStreamBeginCapture(S->gstream, cudaStreamCaptureModeThreadLocal));
      const int c0 = S->cur, s0 = S->scur;
      int rc = enqueue_one_step(C, p);
      if (rc == DVM_OK) rc = enqueue_one_step(C, p);
      if (rc == DVM_OK) rc = launch_check("graph capture");
      S->cur = c0;  // capture does not execute: restore the parity
      S->scur = s0;
      cudaError_t e = cudaStreamEndCapture(S->gstream, &g);
      C->stream = user;
      if (rc != DVM_OK) return rc;
      DVM_CUDA_TRY(e);
      e = cudaGraphInstantiate(&S->graph, g, 0);
      cudaGraphDestroy(g);
      DVM_CUDA_TRY(e);
      S->graph_parity = parity;
    }
    // the graph runs on the private stream, ordered after and before the
    // caller's stream by events
    DVM_CUDA_TRY(cudaEventRecord(S->ev_in, C->stream));
    DVM_CUDA_TRY(cudaStreamWaitEvent(S->gstream, S->ev_in, 0));
    for (; s + 2 <= nsteps; s += 2) {
      DVM_CUDA_TRY(cudaGraphLaunch(S->graph, S->gstream));
      C->steps += 2;
    }
    DVM_CUDA_TRY(cudaEventRecord(S->ev_out, S->gstream));
    DVM_CUDA_TRY(cudaStreamWaitEvent(C->stream, S->ev_out, 0));
  }
  for (; s < nsteps; ++s) {
    int rc = enqueue_one_step(C, p);
    if (rc != DVM_OK) return rc;
    C->steps++;
  }
  return launch_check(use_graph ? "graph replay / last step" : "step launches");
}

int tucker_launch_info(dvm_ctx *C, int32_t *grid, float *tune_ms) {
  TuckerState *S = C->tucker;
  if (grid) *grid = S->split ? -S->grid : S->grid;
  if (tune_ms)
    for (int i = 0; i < 5; ++i) tune_ms[i] = S->tune_ms[i];
  return DVM_OK;
}

int tucker_moments(dvm_ctx *C, double *d_macro) {
  launch_macro_from_sums(C->d_sums[C->tucker->scur], d_macro, C->nc, C->w, C->stream);
  DVM_CUDA_TRY(cudaGetLastError());
  return DVM_OK;
}

int tucker_get_f(dvm_ctx *C, int64_t cell0, int64_t ncell, double *d_out) {
  TuckerState *S = C->tucker;
  const int grid = (int)std::min<int64_t>(ncell, S->grid);
  if (launch_tucker_expand(S->buf[S->cur], cell0, ncell, C->N[0], C->N[1], C->N[2], S->R, S->Nmax,
                           S->scratch, S->stride, d_out, grid, S->fp64, C->stream) != 0) {
    set_error("Tucker kernel needs more shared memory than the device allows");
    return DVM_ERR_UNSUPPORTED;
  }
  DVM_CUDA_TRY(cudaGetLastError());
  return DVM_OK;
}

int tucker_get_ranks(dvm_ctx *C, int32_t *r) {
  TuckerState *S = C->tucker;
  DVM_CUDA_TRY(cudaMemcpyAsync(r, S->buf[S->cur].rank, sizeof(int) * 3 * C->nc,
                               cudaMemcpyDeviceToHost, C->stream));
  return sync_check(C);
}

int tucker_memory(dvm_ctx *C, size_t *f_bytes) {
  std::vector<int32_t> r(3 * C->nc);
  int rc = tucker_get_ranks(C, r.data());
  if (rc != DVM_OK) return rc;
  size_t vals = 0;
  for (int64_t c = 0; c < C->nc; ++c)
    vals += (size_t)r[3 * c] * r[3 * c + 1] * r[3 * c + 2] + (size_t)C->N[0] * r[3 * c] +
            (size_t)C->N[1] * r[3 * c + 1] + (size_t)C->N[2] * r[3 * c + 2];
  *f_bytes = vals * sizeof(double);
  return DVM_OK;
}

namespace {
template <typename T>
bool io_dev(FILE *fp, T *d, size_t n, bool write) {
  std::vector<T> h(n);
  if (write) {
    if (cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return std::fwrite(h.data(), sizeof(T), n, fp) == n;
  }
  if (std::fread(h.data(), sizeof(T), n, fp) != n) return false;
  return cudaMemcpy(d, h.data(), sizeof(T) * n, cudaMemcpyHostToDevice) == cudaSuccess;
}

bool io_state(dvm_ctx *C, FILE *fp, bool write) {
  TuckerState *S = C->tucker;
  const int64_t nc = C->nc;
  const int R = S->R;
  TuckerDev &T = S->buf[S->cur];
  if (!io_dev(fp, T.rank, 3 * nc, write)) return false;
  if (!io_dev(fp, T.core, (size_t)nc * R * R * R, write)) return false;
  for (int a = 0; a < 3; ++a)
    if (!io_dev(fp, T.fac[a], (size_t)nc * C->N[a] * R, write)) return false;
  return io_dev(fp, C->d_sums[S->scur], (size_t)nc * kSums, write);
}
}  // namespace

int tucker_save(dvm_ctx *C, FILE *fp) {
  int32_t R = C->tucker->R;
  if (std::fwrite(&R, sizeof R, 1, fp) != 1 || !io_state(C, fp, true)) {
    set_error("checkpoint write failed");
    return DVM_ERR_IO;
  }
  return DVM_OK;
}

int tucker_load(dvm_ctx *C, FILE *fp) {
  int32_t R = 0;
  if (std::fread(&R, sizeof R, 1, fp) != 1 || R != C->tucker->R) {
    set_error("checkpoint rank capacity does not match this context");
    return DVM_ERR_IO;
  }
  int rc = check_tucker_faces(C);
  if (rc != DVM_OK) return rc;
  rc = build_ghost_factors(C);
  if (rc != DVM_OK) return rc;
  if (!io_state(C, fp, false)) {
    set_error("checkpoint read failed");
    return DVM_ERR_IO;
  }
  return DVM_OK;
}
