// Tucker-format kernels of the S-model DVM step (arXiv:1912.04582, Sections 4-5).
//
// State per cell: ranks (r1, r2, r3) <= R, core G (r1 x r2 x r3, compact), factors
// U_a (N_a x R, row-major, first r_a columns used, orthonormal after rounding),
// all FP64.
//
// One step per cell (one CTA, persistent over cells):
//   1. Moments of the Tucker tensor by weighted convolution (Section 4 item 5):
//      S_a^(p) = U_a^T (v_a^p) for p = 0..3, then core contractions
//      (tucker_moments_kernel, FP64).
//   2. Assembly of f^{n+1} (Section 5): the self term f_i o W with the
//      Lemma-1 weight W = 1 - dt nu - sum_l c_l (xi.e_l)^+, the equilibrium term
//      dt nu f^S (rank-1 Maxwellian factors times the cubic Shakhov polynomial,
//      Proposition 1), and one block per face, (-c_l (xi.e_l)^-) o f_nb(l).
//      Because the pre-rounding rank r0 = 2r + sum r_nb + 4 is at least N on
//      every workload of interest, the QR-of-factors route of Section 4 item 4
//      leaves an N1 x N2 x N3 core; this kernel therefore forms that tensor X
//      directly in scratch by mode products of each block (a dense
//      contraction), which also lets faces whose normal is not a coordinate
//      axis use the exact CIR weight (xi.e)^- pointwise.
//   3. Rounding (Section 4 items 1 and 4): sequentially truncated HOSVD of X —
//      per mode the Gram matrix of the unfolding, its eigen-decomposition by
//      cyclic Jacobi rotations, truncation to the smallest rank whose discarded
//      energy is <= (eps^2/3) ||X||^2 (capped), projection — giving the new
//      orthonormal factors and core.
// The heavy arithmetic (expansions, Gram matrices, Jacobi) is templated on the
// scalar type: double for the FP64 path, float for the mixed path; moments,
// macroparameters, rank decisions' energy sums and the stored state stay FP64.
#include <cfloat>
#include <cmath>

#include "dvm_device.cuh"
#include "dvm_internal.h"
#include "tucker.h"

namespace dvm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kTB = 256;   // threads per CTA for the step / rounding kernel
constexpr int kKC = 32;    // column chunk of the Gram (SYRK) tiles

template <typename Real>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double jacobi = 1e-15;
  static constexpr int sweeps = 24;
};
template <>
struct Eps<float> {
  static constexpr float jacobi = 3e-7f;
  static constexpr int sweeps = 16;
};

__device__ __forceinline__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  __syncthreads();
  return t;
}

// Shared-memory layout of the step / rounding kernel.
template <typename Real>
struct Smem {
  Real *fac[3];   // [Nmax * R] factor rows for the expansion in progress
  Real *A;        // [Nmax * Nmax] Gram / Jacobi matrix
  Real *V;        // [Nmax * Nmax] eigenvectors
  Real *tile;     // [Nmax * kKC] SYRK tile
  Real *cs;       // [Nmax + 2] Jacobi cosines / sines
  int *pairs;     // [Nmax + 2]
  int *perm;      // [Nmax]
  double *tab;    // [3][8][Nmax] per-axis tables
  double *par;    // [32] cell scalars
  double *red;    // [32]
};

template <typename Real>
__host__ __device__ inline size_t smem_bytes(int Nmax, int R) {
  size_t b = 0;
  b += sizeof(Real) * 3 * (size_t)Nmax * R;
  b += sizeof(Real) * 2 * (size_t)Nmax * Nmax;
  b += sizeof(Real) * (size_t)Nmax * kKC;
  b += sizeof(Real) * (Nmax + 2);
  b += sizeof(int) * (2 * Nmax + 2);
  b = (b + 15) & ~size_t(15);
  b += sizeof(double) * (24 * (size_t)Nmax + 64);
  return b + 64;
}

template <typename Real>
__device__ Smem<Real> carve(unsigned char *base, int Nmax, int R) {
  Smem<Real> s;
  // doubles first (8-byte alignment), then Real arrays, then ints
  size_t off = 0;
  s.tab = reinterpret_cast<double *>(base + off);
  off += sizeof(double) * 24 * (size_t)Nmax;
  s.par = reinterpret_cast<double *>(base + off);
  off += sizeof(double) * 32;
  s.red = reinterpret_cast<double *>(base + off);
  off += sizeof(double) * 32;
  for (int a = 0; a < 3; ++a) {
    s.fac[a] = reinterpret_cast<Real *>(base + off);
    off += sizeof(Real) * (size_t)Nmax * R;
  }
  s.A = reinterpret_cast<Real *>(base + off);
  off += sizeof(Real) * (size_t)Nmax * Nmax;
  s.V = reinterpret_cast<Real *>(base + off);
  off += sizeof(Real) * (size_t)Nmax * Nmax;
  s.tile = reinterpret_cast<Real *>(base + off);
  off += sizeof(Real) * (size_t)Nmax * kKC;
  s.cs = reinterpret_cast<Real *>(base + off);
  off += sizeof(Real) * (Nmax + 2);
  off = (off + 3) & ~size_t(3);
  s.pairs = reinterpret_cast<int *>(base + off);
  off += sizeof(int) * (Nmax + 2);
  s.perm = reinterpret_cast<int *>(base + off);
  return s;
}

// ---------------------------------------------------------------------------
// Expansion of one Tucker tensor (Section 4: A = G x1 U1 x2 U2 x3 U3) into a
// full N1 x N2 x N3 array.  The factors are first copied to shared memory in
// `Real`, optionally with their rows scaled (rowscale[a] != null).  The last
// mode product either assigns (acc == false) or accumulates weight(i) * value.
template <typename Real, typename Weight>
__device__ void expand(const TuckerDev &T, int64_t cell, const int N[3], int R,
                       const double *const rowscale[3], Smem<Real> &sm, Real *T1, Real *T2,
                       Real *out, bool acc, const Weight &weight) {
  const int tid = threadIdx.x;
  const int r1 = T.rank[3 * cell], r2 = T.rank[3 * cell + 1], r3 = T.rank[3 * cell + 2];
  const double *G = T.core + cell * (int64_t)R * R * R;
  for (int a = 0; a < 3; ++a) {
    const int ra = T.rank[3 * cell + a];
    const double *U = T.fac[a] + cell * (int64_t)N[a] * R;
    for (int idx = tid; idx < N[a] * ra; idx += blockDim.x) {
      const int i = idx / ra, k = idx - i * ra;
      double v = U[(int64_t)i * R + k];
      if (rowscale[a]) v *= rowscale[a][i];
      sm.fac[a][idx] = (Real)v;
    }
  }
  __syncthreads();
  const int N1 = N[0], N2 = N[1], N3 = N[2];
  // T1[k1][k2][i3] = sum_k3 G[k1][k2][k3] U3[i3][k3]
  for (int idx = tid; idx < r1 * r2 * N3; idx += blockDim.x) {
    const int i3 = idx % N3, k12 = idx / N3;
    const double *g = G + (int64_t)k12 * r3;
    const Real *u = sm.fac[2] + i3 * r3;
    Real s = 0;
    for (int k3 = 0; k3 < r3; ++k3) s += (Real)g[k3] * u[k3];
    T1[idx] = s;
  }
  __syncthreads();
  // T2[k1][i2][i3] = sum_k2 U2[i2][k2] T1[k1][k2][i3]
  for (int idx = tid; idx < r1 * N2 * N3; idx += blockDim.x) {
    const int i3 = idx % N3, t = idx / N3, i2 = t % N2, k1 = t / N2;
    const Real *u = sm.fac[1] + i2 * r2;
    const Real *src = T1 + (int64_t)k1 * r2 * N3 + i3;
    Real s = 0;
    for (int k2 = 0; k2 < r2; ++k2) s += u[k2] * src[(int64_t)k2 * N3];
    T2[idx] = s;
  }
  __syncthreads();
  // out[i1][p] (+)= w * sum_k1 U1[i1][k1] T2[k1][p]
  const int NP = N2 * N3;
  for (int p = tid; p < NP; p += blockDim.x) {
    const int i2 = p / N3, i3 = p - i2 * N3;
    for (int i0 = 0; i0 < N1; i0 += 8) {
      Real a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int k1 = 0; k1 < r1; ++k1) {
        const Real t = T2[(int64_t)k1 * NP + p];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (i0 + j < N1) a[j] += sm.fac[0][(i0 + j) * r1 + k1] * t;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i1 = i0 + j;
        if (i1 < N1) {
          const int64_t o = (int64_t)i1 * NP + p;
          if (acc)
            out[o] += (Real)weight(i1, i2, i3) * a[j];
          else
            out[o] = a[j];
        }
      }
    }
  }
  __syncthreads();
}

struct NoWeight {
  __device__ double operator()(int, int, int) const { return 1.0; }
};

// inflow weight of a face: -c min(xi.e, 0) * scale
struct FaceWeight {
  const double *x0, *x1, *x2;
  double c, e0, e1, e2, scale;
  __device__ double operator()(int i1, int i2, int i3) const {
    const double xn = e0 * x0[i1] + e1 * x1[i2] + e2 * x2[i3];
    return -c * fmin(xn, 0.0) * scale;
  }
};

// ---------------------------------------------------------------------------
// Gram matrix of the mode-m unfolding of a tensor with dims D (row-major):
// C[a][b] = sum_j T(a, j) T(b, j), into sm.A (n x n, n = D[m]).
template <typename Real>
__device__ void gram(const Real *T, const int D[3], int m, Smem<Real> &sm) {
  const int tid = threadIdx.x;
  const int n = D[m];
  const int cols = (D[0] * D[1] * D[2]) / n;
  const int nn = n * n;
  constexpr int Q = 16;  // outputs per thread (n <= 64 with 256 threads)
  Real acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = 0;
  for (int j0 = 0; j0 < cols; j0 += kKC) {
    for (int idx = tid; idx < n * kKC; idx += blockDim.x) {
      const int a = idx / kKC, jj = idx - a * kKC, j = j0 + jj;
      Real v = 0;
      if (j < cols) {
        int64_t addr;
        if (m == 0) {
          addr = (int64_t)a * cols + j;
        } else if (m == 1) {
          const int k = j / D[2], i = j - k * D[2];
          addr = ((int64_t)k * D[1] + a) * D[2] + i;
        } else {
          addr = (int64_t)j * D[2] + a;
        }
        v = T[addr];
      }
      sm.tile[idx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int o = tid + q * kTB;
      if (o < nn) {
        const int a = o / n, b = o - a * n;
        const Real *ta = sm.tile + a * kKC, *tb = sm.tile + b * kKC;
        Real s = acc[q];
#pragma unroll 8
        for (int k = 0; k < kKC; ++k) s += ta[k] * tb[k];
        acc[q] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int o = tid + q * kTB;
    if (o < nn) sm.A[o] = acc[q];
  }
  __syncthreads();
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix in sm.A
// (eigenvalues left on its diagonal, eigenvectors in the columns of sm.V).
// Disjoint rotation pairs of a round-robin schedule are applied together.
template <typename Real>
__device__ void jacobi(Smem<Real> &sm, int n) {
  const int tid = threadIdx.x;
  Real *A = sm.A, *V = sm.V;
  for (int i = tid; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? Real(1) : Real(0);
  const int m = (n + 1) & ~1;
  const int half = m / 2;
  for (int sweep = 0; sweep < Eps<Real>::sweeps; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = tid; i < n * n; i += blockDim.x) {
      const double a = (double)A[i];
      if (i / n == i % n) dia += a * a; else off += a * a;
    }
    off = block_sum_d(off, sm.red);
    dia = block_sum_d(dia, sm.red);
    if (off <= (double)Eps<Real>::jacobi * (double)Eps<Real>::jacobi * dia || dia == 0.0) break;
    for (int round = 0; round < m - 1; ++round) {
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = 0;
          q = 1 + round;
        } else {
          p = 1 + (round + tid) % (m - 1);
          q = 1 + (round - tid + (m - 1)) % (m - 1);
        }
        Real c = 1, s = 0;
        if (p < n && q < n) {
          const Real apq = A[p * n + q];
          if (apq != Real(0)) {
            const Real theta = (A[q * n + q] - A[p * n + p]) / (Real(2) * apq);
            const Real t = (theta >= Real(0) ? Real(1) : Real(-1)) /
                           (fabs(theta) + sqrt(theta * theta + Real(1)));
            c = Real(1) / sqrt(t * t + Real(1));
            s = t * c;
          }
        } else {
          p = q = -1;
        }
        sm.pairs[2 * tid] = p;
        sm.pairs[2 * tid + 1] = q;
        sm.cs[2 * tid] = c;
        sm.cs[2 * tid + 1] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += blockDim.x) {  // A <- A P, V <- V P
        const int k = idx / n, r = idx - k * n;
        const int p = sm.pairs[2 * k], q = sm.pairs[2 * k + 1];
        if (p < 0) continue;
        const Real c = sm.cs[2 * k], s = sm.cs[2 * k + 1];
        const Real ap = A[r * n + p], aq = A[r * n + q];
        A[r * n + p] = c * ap - s * aq;
        A[r * n + q] = s * ap + c * aq;
        const Real vp = V[r * n + p], vq = V[r * n + q];
        V[r * n + p] = c * vp - s * vq;
        V[r * n + q] = s * vp + c * vq;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += blockDim.x) {  // A <- P^T A
        const int k = idx / n, j = idx - k * n;
        const int p = sm.pairs[2 * k], q = sm.pairs[2 * k + 1];
        if (p < 0) continue;
        const Real c = sm.cs[2 * k], s = sm.cs[2 * k + 1];
        const Real bp = A[p * n + j], bq = A[q * n + j];
        A[p * n + j] = c * bp - s * bq;
        A[q * n + j] = s * bp + c * bq;
      }
      __syncthreads();
    }
  }
}

// Sort the eigenvalues (descending, into sm.perm) and pick the truncation rank:
// the smallest r whose discarded energy is <= thr, capped to [1, cap].
template <typename Real>
__device__ int choose_rank(Smem<Real> &sm, int n, double thr, int cap, double *discarded) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) sm.perm[i] = i;
    for (int i = 1; i < n; ++i) {  // insertion sort by eigenvalue, descending
      const int v = sm.perm[i];
      const double lv = (double)sm.A[v * n + v];
      int j = i - 1;
      while (j >= 0 && (double)sm.A[sm.perm[j] * n + sm.perm[j]] < lv) {
        sm.perm[j + 1] = sm.perm[j];
        --j;
      }
      sm.perm[j + 1] = v;
    }
    double tail = 0.0;
    int r = n;
    for (int k = n - 1; k >= 1 && thr > 0.0; --k) {  // eps = 0: no truncation
      const double l = fmax((double)sm.A[sm.perm[k] * n + sm.perm[k]], 0.0);
      if (tail + l > thr) break;
      tail += l;
      r = k;
    }
    if (r > cap) {
      tail = 0.0;
      for (int k = cap; k < n; ++k) tail += fmax((double)sm.A[sm.perm[k] * n + sm.perm[k]], 0.0);
      r = cap;
    }
    if (r < 1) r = 1;
    sm.par[30] = (double)r;
    sm.par[31] = tail;
  }
  __syncthreads();
  const int r = (int)sm.par[30];
  if (discarded) *discarded += sm.par[31];
  return r;
}

// out = T x_m Vsel^T : mode m of T (dims D) contracted with the first r sorted
// eigenvectors; result dims D with D[m] -> r.
template <typename Real>
__device__ void project(const Real *T, const int D[3], int m, int r, Smem<Real> &sm, Real *out) {
  const int n = D[m];
  int Do[3] = {D[0], D[1], D[2]};
  Do[m] = r;
  const int total = Do[0] * Do[1] * Do[2];
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int i2 = idx % Do[2], t = idx / Do[2], i1 = t % Do[1], i0 = t / Do[1];
    const int ii[3] = {i0, i1, i2};
    const int k = ii[m];
    const int col = sm.perm[k];
    int64_t base, stride;
    if (m == 0) {
      base = (int64_t)i1 * D[2] + i2;
      stride = (int64_t)D[1] * D[2];
    } else if (m == 1) {
      base = (int64_t)i0 * D[1] * D[2] + i2;
      stride = D[2];
    } else {
      base = ((int64_t)i0 * D[1] + i1) * D[2];
      stride = 1;
    }
    Real s = 0;
    for (int a = 0; a < n; ++a) s += sm.V[a * n + col] * T[base + a * stride];
    out[idx] = s;
  }
  __syncthreads();
}

// Truncated sequential HOSVD of X (N1 x N2 x N3 in scratch) into the Tucker
// slot `cell` of `out`.  Uses T2 (>= R*N2*N3) and T1 (>= R*R*N3) as work space.
template <typename Real>
__device__ void round_hosvd(Real *X, Real *T1, Real *T2, const int N[3], int R, double eps,
                            TuckerDev &out, int64_t cell, Smem<Real> &sm, double *err_out) {
  int D[3] = {N[0], N[1], N[2]};
  // total energy ||X||^2 (FP64 sums)
  double e = 0.0;
  const int NN = N[0] * N[1] * N[2];
  for (int i = threadIdx.x; i < NN; i += blockDim.x) e += (double)X[i] * (double)X[i];
  e = block_sum_d(e, sm.red);
  const double thr = eps * eps / 3.0 * e;
  double discarded = 0.0;
  int r[3];
  const Real *src = X;
  Real *dst[3] = {T2, T1, nullptr};
  for (int m = 0; m < 3; ++m) {
    gram<Real>(src, D, m, sm);
    jacobi<Real>(sm, D[m]);
    r[m] = choose_rank<Real>(sm, D[m], thr, R, &discarded);
    // factor U_m = first r sorted eigenvectors (FP64 state, row stride R)
    double *U = out.fac[m] + cell * (int64_t)N[m] * R;
    for (int idx = threadIdx.x; idx < N[m] * r[m]; idx += blockDim.x) {
      const int i = idx / r[m], k = idx - i * r[m];
      U[(int64_t)i * R + k] = (double)sm.V[i * D[m] + sm.perm[k]];
    }
    if (m < 2) {
      project<Real>(src, D, m, r[m], sm, dst[m]);
      D[m] = r[m];
      src = dst[m];
    } else {
      // core = Y2 x_3 V3^T, written compact in FP64
      int Do[3] = {D[0], D[1], r[2]};
      const int total = Do[0] * Do[1] * Do[2];
      double *G = out.core + cell * (int64_t)R * R * R;
      const int n = D[2];
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k3 = idx % Do[2], k12 = idx / Do[2];
        const int col = sm.perm[k3];
        const Real *y = src + (int64_t)k12 * n;
        double s = 0.0;
        for (int a = 0; a < n; ++a) s += (double)sm.V[a * n + col] * (double)y[a];
        G[idx] = s;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    out.rank[3 * cell] = r[0];
    out.rank[3 * cell + 1] = r[1];
    out.rank[3 * cell + 2] = r[2];
    if (err_out) err_out[cell] = e > 0.0 ? sqrt(discarded / e) : 0.0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kTB) tucker_step_kernel(TuckerStepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<Real> sm = carve<Real>(smem_raw, P.Nmax, P.R);
  __shared__ SlotDev s_slot[6];
  __shared__ double s_scale[6];
  const int N[3] = {P.N1, P.N2, P.N3};
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3, NP = N2 * N3;
  const int NN = N1 * NP;
  const int tid = threadIdx.x;
  Real *X = reinterpret_cast<Real *>(P.scratch) + (size_t)blockIdx.x * P.scratch_stride;
  Real *E = X + NN;
  Real *T2 = E + NN;
  Real *T1 = T2 + (size_t)P.R * NP;
  double *xt[3] = {sm.tab, sm.tab + P.Nmax, sm.tab + 2 * P.Nmax};  // nodes
  for (int a = 0; a < 3; ++a)
    for (int i = tid; i < N[a]; i += blockDim.x) xt[a][i] = P.xi[a][i];
  __syncthreads();

  for (int64_t c = blockIdx.x; c < P.nc; c += gridDim.x) {
    if (P.mode == 1) {  // compress a given full tensor
      const double *src = P.finit + c * (int64_t)NN;
      for (int i = tid; i < NN; i += blockDim.x) X[i] = (Real)src[i];
      __syncthreads();
      round_hosvd<Real>(X, T1, T2, N, P.R, P.tol, P.nxt, c, sm, P.err);
      continue;
    }
    // ---- prologue: macroparameters, wall densities
    const double *S = P.sums + c * kSums;
    if (tid < 6) {
      s_slot[tid] = P.slot[c * 6 + tid];
      s_scale[tid] = (s_slot[tid].kind == kWall) ? -S[16 + tid] / s_slot[tid].wall_den : 1.0;
    }
    if (tid == 0) {
      CellMacro m;
      macro_from_sums(S, P.w, m);
      if (m.bad) atomicOr(P.flag, 1);
      const double nu = P.delta * m.n * pow(m.T, 1.0 - P.omega);
      sm.par[0] = m.n;
      for (int a = 0; a < 3; ++a) {
        sm.par[1 + a] = m.u[a];
        sm.par[5 + a] = m.q[a];
      }
      sm.par[4] = m.T;
      sm.par[8] = P.dt * nu;
      sm.par[9] = 1.6 * (1.0 - P.Pr) / (m.n * m.T * m.T);
      sm.par[10] = cbrt(m.n) / sqrt(kPi * m.T);
    }
    __syncthreads();
    {
      const double T = sm.par[4], dtnu = sm.par[8], A = sm.par[9], amp = sm.par[10];
      for (int a = 0; a < 3; ++a)
        for (int i = tid; i < N[a]; i += blockDim.x) {
          const double v = xt[a][i] - sm.par[1 + a];
          double *tb = sm.tab + (3 + 3 * a) * P.Nmax;  // F, A q v, v^2/T per axis
          tb[i] = (a == 0 ? dtnu : 1.0) * amp * exp(-v * v / T);
          tb[P.Nmax + i] = A * sm.par[5 + a] * v;
          tb[2 * P.Nmax + i] = v * v / T;
        }
    }
    __syncthreads();
    // ---- own expansion into E
    const double *none[3] = {nullptr, nullptr, nullptr};
    expand<Real>(P.cur, c, N, P.R, none, sm, T1, T2, E, false, NoWeight{});
    // ---- pointwise part: c0 f + dt nu f^S + ghost / self-referencing faces
    {
      const double dtnu = sm.par[8];
      const double *F0 = sm.tab + 3 * P.Nmax, *F1 = sm.tab + 6 * P.Nmax, *F2 = sm.tab + 9 * P.Nmax;
      for (int idx = tid; idx < NN; idx += blockDim.x) {
        const int i3 = idx % N3, t = idx / N3, i2 = t % N2, i1 = t / N2;
        const double x1 = xt[0][i1], x2 = xt[1][i2], x3 = xt[2][i3];
        const double fM = F0[i1] * F1[i2] * F2[i3];
        const double aq = F0[P.Nmax + i1] + F1[P.Nmax + i2] + F2[P.Nmax + i3];
        const double tt = F0[2 * P.Nmax + i1] + F1[2 * P.Nmax + i2] + F2[2 * P.Nmax + i3] - 2.5;
        double val = fM * fma(aq, tt, 1.0);
        double c0 = 1.0 - dtnu;
        const double fe = (double)E[idx];
#pragma unroll
        for (int l = 0; l < 6; ++l) {
          const SlotDev &sl = s_slot[l];
          const double xn = sl.e[0] * x1 + sl.e[1] * x2 + sl.e[2] * x3;
          c0 -= sl.c * fmax(xn, 0.0);
          const double m = -sl.c * fmin(xn, 0.0);
          if (m == 0.0) continue;
          double g;
          switch (sl.kind) {
            case kInterior: continue;  // added by its block expansion below
            case kZeroGrad: g = fe; break;
            case kSymmetry: {
              int j1 = i1, j2 = i2, j3 = i3;
              if (sl.flip == 0) j1 = N1 - 1 - i1;
              else if (sl.flip == 1) j2 = N2 - 1 - i2;
              else j3 = N3 - 1 - i3;
              g = (double)E[((int64_t)j1 * N2 + j2) * N3 + j3];
              break;
            }
            default: {  // free stream / wall: rank-1 Maxwellian ghost
              const double *gf = P.ghostf + (int64_t)sl.src * 3 * P.Nmax;
              g = s_scale[l] * gf[i1] * gf[P.Nmax + i2] * gf[2 * P.Nmax + i3];
            }
          }
          val = fma(m, g, val);
        }
        X[idx] = (Real)fma(c0, fe, val);
      }
      __syncthreads();
    }
    // ---- one block per interior face: X += (-c (xi.e)^-) o f_nb
    for (int l = 0; l < 6; ++l) {
      const SlotDev sl = s_slot[l];
      if (sl.kind != kInterior) continue;
      FaceWeight fw{xt[0], xt[1], xt[2], sl.c, sl.e[0], sl.e[1], sl.e[2], 1.0};
      expand<Real>(P.cur, sl.src, N, P.R, none, sm, T1, T2, X, true, fw);
    }
    // ---- rounding
    round_hosvd<Real>(X, T1, T2, N, P.R, P.tol, P.nxt, c, sm, P.err);
  }
}

// Expansion of cells [c0, c0 + ncell) into full FP64 tensors (inspection).
template <typename Real>
__global__ void __launch_bounds__(kTB) tucker_expand_kernel(TuckerDev T, int64_t c0, int64_t ncell,
                                                            int N1, int N2, int N3, int R, int Nmax,
                                                            void *scratch, size_t stride, double *out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<Real> sm = carve<Real>(smem_raw, Nmax, R);
  const int N[3] = {N1, N2, N3};
  const int NN = N1 * N2 * N3;
  Real *E = reinterpret_cast<Real *>(scratch) + (size_t)blockIdx.x * stride;
  Real *T2 = E + NN;
  Real *T1 = T2 + (size_t)R * N2 * N3;
  const double *none[3] = {nullptr, nullptr, nullptr};
  for (int64_t j = blockIdx.x; j < ncell; j += gridDim.x) {
    expand<Real>(T, c0 + j, N, R, none, sm, T1, T2, E, false, NoWeight{});
    for (int i = threadIdx.x; i < NN; i += blockDim.x) out[j * NN + i] = (double)E[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Moments of each cell's Tucker tensor (Section 4 item 5) about the reference
// velocity r: the same 19 raw sums as the full-grid path plus the outflow sums
// of axis-aligned wall faces; FP64.
__global__ void __launch_bounds__(128) tucker_moments_kernel(TuckerMomentParams P) {
  extern __shared__ double msm[];  // [3][5][R] projections, [6][R] wall projections
  __shared__ double s_out[32];
  __shared__ SlotDev s_slot[6];
  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x;
  const int R = P.R;
  const int N[3] = {P.N1, P.N2, P.N3};
  const int r[3] = {P.T.rank[3 * c], P.T.rank[3 * c + 1], P.T.rank[3 * c + 2]};
  const int64_t us = P.uref_stride;
  const double ref[3] = {P.uref ? P.uref[us * c] : 0.0, P.uref ? P.uref[us * c + 1] : 0.0,
                         P.uref ? P.uref[us * c + 2] : 0.0};
  double *Sp = msm;            // [a][p][k], p = 0..3
  double *Sw = msm + 12 * R;   // [l][k] wall outflow projection for slot l
  if (tid < 6) s_slot[tid] = P.slot[c * 6 + tid];
  __syncthreads();
  // S_a^(p)[k] = sum_i U_a[i][k] (xi_a,i - r_a)^p
  for (int idx = tid; idx < 12 * R; idx += blockDim.x) {
    const int k = idx % R, ap = idx / R, p = ap % 4, a = ap / 4;
    double s = 0.0;
    if (k < r[a]) {
      const double *U = P.T.fac[a] + c * (int64_t)N[a] * R;
      for (int i = 0; i < N[a]; ++i) {
        const double v = P.xi[a][i] - ref[a];
        double w = 1.0;
        for (int e = 0; e < p; ++e) w *= v;
        s = fma(U[(int64_t)i * R + k], w, s);
      }
    }
    Sp[idx] = s;
  }
  for (int idx = tid; idx < 6 * R; idx += blockDim.x) {
    const int k = idx % R, l = idx / R;
    const SlotDev &sl = s_slot[l];
    double s = 0.0;
    if (sl.kind == kWall && sl.axis >= 0 && k < r[sl.axis]) {
      const int a = sl.axis;
      const double *U = P.T.fac[a] + c * (int64_t)N[a] * R;
      for (int i = 0; i < N[a]; ++i) s = fma(U[(int64_t)i * R + k], fmax(sl.sgn * P.xi[a][i], 0.0), s);
    }
    Sw[idx] = s;
  }
  __syncthreads();
  // monomials (a1, a2, a3) of the 19 sums; thread j < 19 computes sum j,
  // threads 19..24 the wall outflows
  const double *G = P.T.core + c * (int64_t)R * R * R;
  if (tid < 25) {
    const double *w0, *w1, *w2;
    const int mono[19][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0},
                             {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {3, 0, 0}, {1, 2, 0},
                             {1, 0, 2}, {2, 1, 0}, {0, 3, 0}, {0, 1, 2}, {2, 0, 1}, {0, 2, 1},
                             {0, 0, 3}};
    bool live = true;
    if (tid < 19) {
      w0 = Sp + (0 * 4 + mono[tid][0]) * R;
      w1 = Sp + (1 * 4 + mono[tid][1]) * R;
      w2 = Sp + (2 * 4 + mono[tid][2]) * R;
    } else {
      const int l = tid - 19;
      const SlotDev &sl = s_slot[l];
      live = sl.kind == kWall && sl.axis >= 0;
      w0 = (live && sl.axis == 0) ? Sw + l * R : Sp + 0 * 4 * R;
      w1 = (live && sl.axis == 1) ? Sw + l * R : Sp + 1 * 4 * R;
      w2 = (live && sl.axis == 2) ? Sw + l * R : Sp + 2 * 4 * R;
    }
    double s = 0.0;
    if (live) {
      for (int k1 = 0; k1 < r[0]; ++k1) {
        double s1 = 0.0;
        for (int k2 = 0; k2 < r[1]; ++k2) {
          const double *g = G + ((int64_t)k1 * r[1] + k2) * r[2];
          double s2 = 0.0;
          for (int k3 = 0; k3 < r[2]; ++k3) s2 = fma(g[k3], w2[k3], s2);
          s1 = fma(s2, w1[k2], s1);
        }
        s = fma(s1, w0[k1], s);
      }
    }
    s_out[tid] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double *Sn = P.sums + c * kSums;
    const double *o = s_out;
    Sn[0] = ref[0];
    Sn[1] = ref[1];
    Sn[2] = ref[2];
    for (int k = 0; k < 10; ++k) Sn[3 + k] = o[k];
    Sn[13] = o[10] + o[11] + o[12];
    Sn[14] = o[13] + o[14] + o[15];
    Sn[15] = o[16] + o[17] + o[18];
    for (int l = 0; l < 6; ++l) Sn[16 + l] = o[19 + l];
    Sn[22] = 0.0;
    Sn[23] = 0.0;
    CellMacro m;
    macro_from_sums(Sn, P.w, m);
    if (m.bad) atomicOr(P.flag, 1);
    if (P.respart && P.sums_prev) {
      double U0[5], U1[5];
      conserved_from_sums(P.sums_prev + c * kSums, P.w, U0);
      conserved_from_sums(Sn, P.w, U1);
      double num = 0.0, den = 0.0;
      for (int k = 0; k < 5; ++k) {
        num += (U1[k] - U0[k]) * (U1[k] - U0[k]);
        den += U0[k] * U0[k];
      }
      P.respart[2 * c] = P.vol[c] * num;
      P.respart[2 * c + 1] = P.vol[c] * den;
    }
  }
}

// Rank-1 Tucker Maxwellian per cell (Section 5): U_a(i) proportional to
// exp(-(xi_a,i - u_a)^2 / T), normalised; the core carries n (pi T)^{-3/2} and
// the three norms.
__global__ void tucker_maxwellian_kernel(TuckerDev Tk, const double *n, const double *u,
                                         const double *Tc, const double *xi0, const double *xi1,
                                         const double *xi2, int N1, int N2, int N3, int R) {
  __shared__ double s_norm[3];
  const int64_t c = blockIdx.x;
  const int N[3] = {N1, N2, N3};
  const double *xi[3] = {xi0, xi1, xi2};
  const double T = Tc[c];
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    double *U = Tk.fac[a] + c * (int64_t)N[a] * R;
    double s = 0.0;
    for (int i = 0; i < N[a]; ++i) {
      const double v = xi[a][i] - u[3 * c + a];
      const double g = exp(-v * v / T);
      U[(int64_t)i * R] = g;
      s += g * g;
    }
    const double nr = sqrt(s);
    for (int i = 0; i < N[a]; ++i) U[(int64_t)i * R] /= nr;
    s_norm[a] = nr;
    Tk.rank[3 * c + a] = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    Tk.core[c * (int64_t)R * R * R] = n[c] / pow(kPi * T, 1.5) * s_norm[0] * s_norm[1] * s_norm[2];
}

template <typename Real>
int launch_step_T(const TuckerStepParams &p, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes<Real>(p.Nmax, p.R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(tucker_step_kernel<Real>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
  }
  tucker_step_kernel<Real><<<grid, kTB, smem, s>>>(p);
  return 0;
}

template <typename Real>
int launch_expand_T(const TuckerDev &T, int64_t c0, int64_t ncell, int N1, int N2, int N3, int R,
                    int Nmax, void *scratch, size_t stride, double *out, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes<Real>(Nmax, R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(tucker_expand_kernel<Real>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
  }
  tucker_expand_kernel<Real><<<grid, kTB, smem, s>>>(T, c0, ncell, N1, N2, N3, R, Nmax, scratch,
                                                     stride, out);
  return 0;
}

}  // namespace

size_t tucker_scratch_elems(int N1, int N2, int N3, int R) {
  const size_t NN = (size_t)N1 * N2 * N3;
  return 2 * NN + (size_t)R * N2 * N3 + (size_t)R * R * N3 + 64;
}

size_t tucker_smem_bytes(int Nmax, int R, bool fp64) {
  return fp64 ? smem_bytes<double>(Nmax, R) : smem_bytes<float>(Nmax, R);
}

int launch_tucker_step(const TuckerStepParams &p, int grid, bool fp64, cudaStream_t s) {
  return fp64 ? launch_step_T<double>(p, grid, s) : launch_step_T<float>(p, grid, s);
}

int launch_tucker_expand(const TuckerDev &T, int64_t c0, int64_t ncell, int N1, int N2, int N3,
                         int R, int Nmax, void *scratch, size_t stride, double *out, int grid,
                         bool fp64, cudaStream_t s) {
  return fp64 ? launch_expand_T<double>(T, c0, ncell, N1, N2, N3, R, Nmax, scratch, stride, out,
                                        grid, s)
              : launch_expand_T<float>(T, c0, ncell, N1, N2, N3, R, Nmax, scratch, stride, out,
                                       grid, s);
}

void launch_tucker_maxwellians(TuckerDev T, const double *n, const double *u, const double *Tc,
                               const double *xi0, const double *xi1, const double *xi2, int64_t nc,
                               int N1, int N2, int N3, int R, cudaStream_t s) {
  tucker_maxwellian_kernel<<<(unsigned)nc, 32, 0, s>>>(T, n, u, Tc, xi0, xi1, xi2, N1, N2, N3, R);
}

void launch_tucker_moments(const TuckerMomentParams &p, cudaStream_t s) {
  const size_t smem = sizeof(double) * 18 * (size_t)p.R;
  tucker_moments_kernel<<<(unsigned)p.nc, 128, smem, s>>>(p);
}

}  // namespace dvm
