// dvm_full_macro_noalloc: macroparameters of a batch of full velocity tensors
// that already live in device memory, computed without allocating any device
// memory.
//
// Who needs this: code that cannot call cudaMalloc at the point where it wants
// the moments — for example a host application whose device memory is handed
// out by its own pool allocator and that forbids any other allocation, or a
// pipeline that must not pay cudaMalloc's implicit device-wide synchronisation
// between kernels it has already queued.  Such a caller passes its own input
// (the tensors) and output (the macroparameters); the intermediate per-cell
// sums live in a fixed, file-scope device array instead of allocated scratch.
//
// The scratch array below is part of the library image: every GPU that loads
// the library holds it (kNoallocMaxCells * 8 doubles = 1 MiB) until the process
// exits.  All calls share it, so calls whose GPU work overlaps (different
// streams, or different host threads on one device) race on it and must be
// serialised by the caller.  Nothing in it needs to start at zero: the first
// pass writes every entry that the second pass reads, and a later call simply
// overwrites what the previous one left there.
#include <cuda.h>

#include <mutex>

#include "dvm_internal.h"

namespace {

constexpr int64_t kNoallocMaxCells = 16384;
constexpr int kNoallocStride = 8;  // per cell: S0, sum xi_1 f, sum xi_2 f, sum xi_3 f, 4 spare

static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxCells * kNoallocStride];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};  // context the address was looked up in

// Unique id of the calling thread's current CUDA context (0 if there is none or it
// cannot be queried), through the driver's entry points so that the library needs
// no link against the driver library.  A looked-up symbol address belongs to one
// context: after a device reset the next call finds a new id and looks it up again.
// Called with g_mu held.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void **>(&get_current),
                                         12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void **>(&get_id), 12000,
                                         cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      get_current = nullptr;
      get_id = nullptr;
    }
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// velocity node i of one axis: ((N-1-i) lo + i hi) / (N-1), without contraction
__device__ __forceinline__ double node(int i, int N, double lo, double hi) {
  return __ddiv_rn(__dadd_rn(__dmul_rn((double)(N - 1 - i), lo), __dmul_rn((double)i, hi)),
                   (double)(N - 1));
}

template <int B, int K>
__device__ void block_sum(double (&v)[K], double *s_red /* [B/32][K] */, double *s_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < K; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp * K + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int q = 0; q < B / 32; ++q) t += s_red[q * K + threadIdx.x];
    s_tot[threadIdx.x] = t;
  }
  __syncthreads();
}

struct Grid {
  int N1, N2, N3;
  double lo0, lo1, lo2, hi0, hi1, hi2;
};

// pass 1: S0 and sum xi_a f of each cell -> scratch
template <int B>
__global__ void __launch_bounds__(B) noalloc_pass1(const double *__restrict__ f, Grid g,
                                                   double *scratch) {
  __shared__ double s_red[(B / 32) * 4];
  __shared__ double s_tot[4];
  const int64_t c = blockIdx.x;
  const int NP = g.N2 * g.N3;
  const double *fc = f + c * (int64_t)g.N1 * NP;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int p = threadIdx.x; p < NP; p += B) {
    const int i2 = p / g.N3, i3 = p - i2 * g.N3;
    double s0 = 0.0, s1 = 0.0;
    for (int i1 = 0; i1 < g.N1; ++i1) {
      const double x = fc[(int64_t)i1 * NP + p];
      s0 += x;
      s1 = fma(node(i1, g.N1, g.lo0, g.hi0), x, s1);
    }
    v[0] += s0;
    v[1] += s1;
    v[2] = fma(node(i2, g.N2, g.lo1, g.hi1), s0, v[2]);
    v[3] = fma(node(i3, g.N3, g.lo2, g.hi2), s0, v[3]);
  }
  block_sum<B, 4>(v, s_red, s_tot);
  if (threadIdx.x < 4) scratch[c * kNoallocStride + threadIdx.x] = s_tot[threadIdx.x];
}

// pass 2: sums about the cell velocity u = (sum xi f)/(sum f) from scratch, then
// [n, u, T, q] (Section 2 definitions, R_g = 1/2, m = 1) -> macro
template <int B>
__global__ void __launch_bounds__(B) noalloc_pass2(const double *__restrict__ f, Grid g, double w,
                                                   const double *scratch, double *macro) {
  __shared__ double s_red[(B / 32) * 13];
  __shared__ double s_tot[13];
  const int64_t c = blockIdx.x;
  const int NP = g.N2 * g.N3;
  const double *fc = f + c * (int64_t)g.N1 * NP;
  const double *sc = scratch + c * kNoallocStride;
  const double r0 = sc[1] / sc[0], r1 = sc[2] / sc[0], r2 = sc[3] / sc[0];
  double v[13];
  for (int k = 0; k < 13; ++k) v[k] = 0.0;
  for (int p = threadIdx.x; p < NP; p += B) {
    const int i2 = p / g.N3, i3 = p - i2 * g.N3;
    const double b = node(i2, g.N2, g.lo1, g.hi1) - r1, d = node(i3, g.N3, g.lo2, g.hi2) - r2;
    double P0 = 0.0, P1 = 0.0, P2 = 0.0, P3 = 0.0;
    for (int i1 = 0; i1 < g.N1; ++i1) {
      const double a = node(i1, g.N1, g.lo0, g.hi0) - r0;
      const double x = fc[(int64_t)i1 * NP + p];
      P0 += x;
      P1 = fma(a, x, P1);
      P2 = fma(a * a, x, P2);
      P3 = fma(a * a * a, x, P3);
    }
    const double bb = b * b, dd = d * d, s = bb + dd;
    v[0] += P0;
    v[1] += P1;
    v[2] = fma(b, P0, v[2]);
    v[3] = fma(d, P0, v[3]);
    v[4] += P2;
    v[5] = fma(bb, P0, v[5]);
    v[6] = fma(dd, P0, v[6]);
    v[7] = fma(b, P1, v[7]);
    v[8] = fma(d, P1, v[8]);
    v[9] = fma(b * d, P0, v[9]);
    v[10] += fma(s, P1, P3);
    v[11] += fma(b, P2, b * s * P0);
    v[12] += fma(d, P2, d * s * P0);
  }
  block_sum<B, 13>(v, s_red, s_tot);
  if (threadIdx.x == 0) {
    const double *S = s_tot;
    const double S0 = S[0];
    const double m[3] = {S[1] / S0, S[2] / S0, S[3] / S0};
    const double Sab[3][3] = {{S[4], S[7], S[8]}, {S[7], S[5], S[9]}, {S[8], S[9], S[6]}};
    const double E = S[4] + S[5] + S[6];
    const double mm = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    const double mM = m[0] * S[1] + m[1] * S[2] + m[2] * S[3];
    double *o = macro + 8 * c;
    o[0] = w * S0;
    o[1] = r0 + m[0];
    o[2] = r1 + m[1];
    o[3] = r2 + m[2];
    o[4] = (2.0 / 3.0) * (E / S0 - mm);
    for (int a = 0; a < 3; ++a) {
      const double su = Sab[a][0] * m[0] + Sab[a][1] * m[1] + Sab[a][2] * m[2];
      o[5 + a] = 0.5 * w *
                 (S[10 + a] - 2.0 * su + mm * S[1 + a] - m[a] * E + 2.0 * m[a] * mM - m[a] * mm * S0);
    }
  }
}

template <int B>
void launch(const double *f, int64_t nc, Grid g, double w, double *scratch, double *macro,
            cudaStream_t s) {
  noalloc_pass1<B><<<(unsigned)nc, B, 0, s>>>(f, g, scratch);
  noalloc_pass2<B><<<(unsigned)nc, B, 0, s>>>(f, g, w, scratch, macro);
}

}  // namespace

extern "C" int dvm_full_macro_noalloc(const double *f, int64_t n_cell, const dvm_vgrid *vg,
                                      double *macro, void *cuda_stream) {
  if (!vg || n_cell < 0 || (n_cell > 0 && (!f || !macro))) {
    dvm::set_error("dvm_full_macro_noalloc: null argument or negative n_cell");
    return DVM_ERR_INVALID_ARG;
  }
  if (n_cell > kNoallocMaxCells) {
    dvm::set_error("dvm_full_macro_noalloc: n_cell = " + std::to_string(n_cell) +
                   " exceeds the fixed scratch capacity of " + std::to_string(kNoallocMaxCells) +
                   " cells; use dvm_moments on a context instead");
    return DVM_ERR_INVALID_ARG;
  }
  for (int a = 0; a < 3; ++a)
    if (vg->N[a] < 2 || vg->N[a] > dvm::kMaxN || !(vg->hi[a] > vg->lo[a])) {
      dvm::set_error("dvm_full_macro_noalloc: bad velocity grid");
      return DVM_ERR_INVALID_ARG;
    }
  if (n_cell == 0) return DVM_OK;
  int dev = 0;
  DVM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    dvm::set_error("dvm_full_macro_noalloc: device ordinal out of range");
    return DVM_ERR_UNSUPPORTED;
  }
  double *scratch = nullptr;
  {
    // set-up once per device (again if its context has changed, e.g. after a
    // device reset), with that device current: host code must not use
    // g_noalloc_scratch itself (on the host it names a stand-in, not device
    // memory), so look up its device address.
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_ctx_id();
    if (!g_scratch_ptr[dev] || id == 0 || id != g_ctx_id[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        g_scratch_ptr[dev] = nullptr;
        dvm::set_error(std::string("dvm_full_macro_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e));
        return DVM_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<double *>(p);
      g_ctx_id[dev] = current_ctx_id();  // the look-up has made the context current
    }
    scratch = g_scratch_ptr[dev];
  }
  Grid g{vg->N[0], vg->N[1], vg->N[2], vg->lo[0], vg->lo[1], vg->lo[2],
         vg->hi[0], vg->hi[1], vg->hi[2]};
  double w = 1.0;
  for (int a = 0; a < 3; ++a) w *= (vg->hi[a] - vg->lo[a]) / (double)(vg->N[a] - 1);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int NP = vg->N[1] * vg->N[2];
  if (NP >= 256)
    launch<256>(f, n_cell, g, w, scratch, macro, s);
  else if (NP > 64)
    launch<128>(f, n_cell, g, w, scratch, macro, s);
  else
    launch<64>(f, n_cell, g, w, scratch, macro, s);
  DVM_CUDA_TRY(cudaGetLastError());
  return DVM_OK;
}
