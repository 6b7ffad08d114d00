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
//   2. Assembly of f^{n+1} (Section 5): the self term f_i o W with the Lemma-1
//      weight W = 1 - dt nu - sum_l c_l (xi.e_l)^+, the equilibrium term
//      dt nu f^S (rank-1 Maxwellian factors times the cubic Shakhov
//      polynomial, Proposition 1), and one block per face,
//      (-c_l (xi.e_l)^-) o f_nb(l).  The pre-rounding rank
//      r0 = 2r + sum r_nb + 4 is at least N on every workload of interest, so
//      the QR-of-factors route of Section 4 item 4 leaves an N1 x N2 x N3 core;
//      this kernel forms that tensor X directly in scratch by mode products of
//      each block (dense contractions), which also lets faces whose normal is
//      not a coordinate axis use the exact CIR weight (xi.e)^- pointwise.
//   3. Rounding (Section 4 items 1 and 4): sequentially truncated HOSVD of X.
//      Per mode: the Gram matrix of the unfolding (FP64 accumulation on the FP64
//      path; exact FP32 products summed in double-FP32 on the mixed path, so
//      that eigenvalues far below sqrt(FP32 round-off) remain resolved), its
//      leading eigenvectors by orthogonal (block power) iteration — FP32 steps
//      on the mixed path, always finished by an FP64 step on the accurate Gram
//      matrix — and the truncation rank chosen from the energy the kept
//      orthonormal vectors capture exactly: the smallest r with
//      trace(C) - sum_{j<r} q_j^T C q_j <= (eps^2/3) ||X||^2, then capped.  The error bound ||X - X~|| <= eps ||X|| therefore holds by
//      construction whenever the cap is inactive.
// Expansions, assembly and projections run in the kernel's scalar type (double
// on the FP64 path, float on the mixed path); moments, macroparameters, Gram
// matrices, eigen-solves, energy sums and the stored state are FP64.
#include <cfloat>
#include <cmath>
#include <map>
#include <mutex>

#include "dvm_device.cuh"
#include "dvm_internal.h"
#include "tucker.h"

namespace dvm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kTB = 256;   // threads per CTA for the step / rounding kernel
constexpr int kKC = 32;    // column chunk of the Gram tiles
// tile row of gram_w32: a warp reads rows 4 apart from 8 adjacent columns; a
// stride of 2 mod 8 words puts those 4 rows on disjoint banks
constexpr int kKP2 = kKC + 2;
constexpr int kTileRow = kKP2 > kKC + 1 ? kKP2 : kKC + 1;  // row length of the tile buffers
constexpr int kExtra = 2;  // oversampling columns of the subspace iteration
constexpr int kPower = 3;     // orthogonal (power) iterations from a cold start
constexpr int kWarmIter = 1;  // orthogonal iterations from the previous step's factor
constexpr int kF32Passes = 2; // Cholesky-QR passes per FP32 orthogonal iteration
constexpr int kTabs = 21;  // per-axis tables of the assembly
constexpr int kTerms = 7;  // distinct Tucker tensors of one cell's assembly: itself + 6 faces
constexpr int kRows = 16;  // first-mode rows one thread assembles per pass

// table / first-mode row length padded to a multiple of kRows (zero-filled)
__host__ __device__ inline int padN(int n) { return (n + kRows - 1) / kRows * kRows; }

// p rounded up to a 16-byte boundary
template <typename T>
__device__ __forceinline__ T *align16(T *p) {
  return reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
}

// Optional per-phase cycle counters (thread 0 of every CTA adds clock64 deltas
// to P.phase[i] when P.phase is not null); no effect on the computation.
struct PhaseClock {
  long long *acc;
  long long t;
  __device__ PhaseClock(long long *a) {
    acc = a;
    t = a ? (long long)clock64() : 0;
  }
  __device__ void mark(int i) {
    if (acc && threadIdx.x == 0) {
      const long long now = (long long)clock64();
      atomicAdd(reinterpret_cast<unsigned long long *>(acc + i), (unsigned long long)(now - t));
      t = now;
    }
  }
  // event counts in slots 1 and 2 (re-seeding rounds, eigen-solver retries)
  __device__ void count(int i, int v) {
    if (acc && threadIdx.x == 0 && v > 0)
      atomicAdd(reinterpret_cast<unsigned long long *>(acc + i), (unsigned long long)v);
  }
};

__host__ __device__ inline int sub_k(int Nmax, int R) {
  const int k = Nmax < R + kExtra ? Nmax : R + kExtra;
  return k < 24 ? k : 24;
}

// Shared-memory layout of the step / rounding kernel.
template <typename Real>
struct Smem {
  int nmax;       // Nmax the layout was carved for
  int kdim;       // K: columns of the eigen-solver blocks
  int asm_space;  // doubles at sm.C usable as assembly staging space
  double *par;    // [32] cell scalars
  double *red;    // [32]
  double *C;      // [Nmax*Nmax] Gram matrix (FP64)
  const double *Cg;  // the Gram matrix the eigen-solver reads (sm.C or a global copy)
  Real *tile2;    // second Gram tile buffer (prefetch), or null
  int *cidx;      // first-mode Gram: indices of the columns kept (cidx_cap entries)
  int cidx_cap;
  double *Q;      // [Nmax*K] subspace basis
  double *W;      // [Nmax*K] C*Q, then the Ritz vectors
  double *B;      // [K*K] projected matrix
  double *Z;      // [K] sorted Rayleigh quotients
  double *cs;     // [K+2] Jacobi cosines / sines
  Real *rt;       // [kTabs][Nmax] assembly tables
  Real *fac[3];   // [Nmax*R] factor rows of the expansion in progress
  Real *u1;       // [kTerms+1][R][padN(Nmax)] first-mode factors of the assembly's terms,
                  // transposed (column k contiguous), zero-padded
  Real *tile;     // [Nmax*(kKC+1)] Gram tile
  Real *Vr;       // [Nmax*K] kept eigenvectors in the working precision
  float *Q32;     // [Nmax*K] (inside sm.W)
  float *W32;     // [Nmax*K] (inside sm.W)
  int *pairs;     // [K+2]
  int *perm;      // [K]
};

template <typename Real>
__host__ __device__ inline size_t smem_bytes(int Nmax, int R) {
  const int K = sub_k(Nmax, R);
  size_t b = sizeof(double) *
             (64 + (size_t)Nmax * Nmax + 2 * (size_t)Nmax * K + (size_t)K * K + 2 * K + 2);
  b += sizeof(Real) * ((size_t)kTabs * padN(Nmax) + 3 * (size_t)Nmax * R +
                       (kTerms + 1) * (size_t)R * padN(Nmax) +
                       (size_t)(Nmax > 32 ? Nmax : 32) * kTileRow +
                       (size_t)Nmax * K);
  b += sizeof(int) * (2 * (size_t)K + 2);
  return b + 64;
}

template <typename Real>
__device__ Smem<Real> carve(unsigned char *base, int Nmax, int R) {
  const int K = sub_k(Nmax, R);
  Smem<Real> s;
  s.nmax = Nmax;
  s.kdim = K;
  s.asm_space = Nmax * Nmax + 2 * Nmax * K;
  size_t off = 0;
  auto takeD = [&](size_t n) {
    double *p = reinterpret_cast<double *>(base + off);
    off += sizeof(double) * n;
    return p;
  };
  s.par = takeD(32);
  s.red = takeD(32);
  s.C = takeD((size_t)Nmax * Nmax);
  s.Cg = s.C;
  s.tile2 = nullptr;
  s.Q = takeD((size_t)Nmax * K);
  s.W = takeD((size_t)Nmax * K);
  s.B = takeD((size_t)K * K);
  s.Z = takeD((size_t)K);
  s.cs = takeD(K + 2);
  auto takeR = [&](size_t n) {
    Real *p = reinterpret_cast<Real *>(base + off);
    off += sizeof(Real) * n;
    return p;
  };
  off = (off + 15) & ~size_t(15);  // the tables and the first-mode rows are read
  s.rt = takeR((size_t)kTabs * padN(Nmax));  // by 16-byte loads
  for (int a = 0; a < 3; ++a) s.fac[a] = takeR((size_t)Nmax * R);
  off = (off + 15) & ~size_t(15);
  s.u1 = takeR((size_t)(kTerms + 1) * R * padN(Nmax));
  s.cidx = reinterpret_cast<int *>(s.u1);  // the assembly's rows are dead during rounding
  s.cidx_cap = (int)((size_t)(kTerms + 1) * R * padN(Nmax) * sizeof(Real) / sizeof(int));
  s.tile = takeR((size_t)(Nmax > 32 ? Nmax : 32) * kTileRow);
  s.Vr = takeR((size_t)Nmax * K);
  off = (off + 3) & ~size_t(3);
  // the FP32 iteration blocks live in sm.W (consumed before sm.W is written)
  s.Q32 = reinterpret_cast<float *>(s.W);
  s.W32 = s.Q32 + (size_t)Nmax * K;
  s.pairs = reinterpret_cast<int *>(base + off);
  off += sizeof(int) * (K + 2);
  s.perm = reinterpret_cast<int *>(base + off);
  return s;
}

// doubles at sm.C usable by the assembly as staging space
template <typename Real>
__device__ __forceinline__ int asm_space_doubles(const Smem<Real> &sm) {
  return sm.asm_space;
}

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

// Exclusive prefix sum of v over the block (thread order) and the total; uses
// red[0..32) as scratch (ints); ends with a barrier.
__device__ __forceinline__ int block_scan_excl(int v, int *red, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[warp] = x;
  __syncthreads();
  int base = 0, tot = 0;
  for (int q = 0; q < nw; ++q) {
    if (q < warp) base += red[q];
    tot += red[q];
  }
  __syncthreads();
  *total = tot;
  return base + x - v;
}

// ---------------------------------------------------------------------------
// Expansion of one Tucker tensor (Section 4: A = G x1 U1 x2 U2 x3 U3) into a
// full N1 x N2 x N3 array (inspection and check-pointing).
template <typename Real>
__device__ void expand(const TuckerDev &T, int64_t cell, const int N[3], int R, Smem<Real> &sm,
                       Real *T1, Real *T2, Real *out) {
  const int tid = threadIdx.x;
  const int r1 = T.rank[3 * cell], r2 = T.rank[3 * cell + 1], r3 = T.rank[3 * cell + 2];
  const double *G = T.core + cell * (int64_t)R * R * R;
  for (int a = 0; a < 3; ++a) {
    const int ra = T.rank[3 * cell + a];
    const double *U = T.fac[a] + cell * (int64_t)N[a] * R;
    for (int idx = tid; idx < N[a] * ra; idx += blockDim.x) {
      const int i = idx / ra, k = idx - i * ra;
      sm.fac[a][idx] = (Real)U[(int64_t)i * R + k];
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
        if (i1 < N1) out[(int64_t)i1 * NP + p] = a[j];
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Gram matrix of the mode-m unfolding of a tensor with dims D (row-major),
// C[a][b] = sum_j T(a, j) T(b, j), into sm.C (FP64).  For float data each
// product is formed exactly (p + e with e = fma(x, y, -p)) and accumulated in a
// (hi, lo) pair of floats (Knuth's two-sum), renormalised after every tile.
__device__ __forceinline__ void df_acc(float x, float y, float &hi, float &lo) {
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, pe));
}

constexpr int kKP = kKC + 1;  // padded tile row (no shared-memory bank conflicts)

// Storage of one Gram entry: FP64 on the FP64 path; on the mixed path the
// double-float accumulator itself, as a (hi, lo) pair of floats in the same 8 bytes
// (the eigen-solver's FP64-accuracy products read it without FP64 arithmetic).
template <typename Real>
__device__ __forceinline__ void gram_store(double *C, int idx, Real hi, Real lo) {
  if constexpr (sizeof(Real) == 8) {
    C[idx] = hi;
  } else {
    const float s = __fadd_rn(hi, lo);  // renormalised pair
    reinterpret_cast<float2 *>(C)[idx] = make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
  }
}

// One Gram entry as a double
template <typename Real>
__device__ __forceinline__ double gram_load(const double *C, int idx) {
  if constexpr (sizeof(Real) == 8) {
    return C[idx];
  } else {
    const float2 v = reinterpret_cast<const float2 *>(C)[idx];
    return (double)v.x + (double)v.y;
  }
}

// trace of the n x n Gram matrix at sm.Cg (thread 0 sums in order; all threads
// return it)
template <typename Real>
__device__ double gram_trace(Smem<Real> &sm, int n) {
  if (threadIdx.x < 32) {  // warp 0: a lane per diagonal entry, fixed shuffle tree
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) t += gram_load<Real>(sm.Cg, i * n + i);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sm.par[27] = t;
  }
  __syncthreads();
  const double tr = sm.par[27];
  __syncthreads();
  return tr;
}


// Double-float (hi, lo) += (h2, l2), renormalised (fast two-sum of the high parts)
__device__ __forceinline__ void df_add_into(float &hi, float &lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  const float t = __fadd_rn(__fadd_rn(lo, l2), err);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Gram matrix of the mode-m unfolding by TS x TS output blocks on or above the diagonal.
// The nb (nb + 1) / 2 blocks (nb = ceil(n / TS)) are numbered row by row; every block needs
// a thread (the callers launch at least as many threads as blocks); with fewer blocks than
// threads the columns of every staged chunk are split into S segments, thread t owning
// block t mod nblk and segment t / nblk; the segments' partial sums are then added into
// the result in segment order (a fixed order: the same sums in either launch variant).
// Each chunk's loop stops at the last real column.
template <typename Real, int TS>
__device__ void gram_tiled(const Real *T, const int D[3], int m, Smem<Real> &sm) {
  const int n = D[m];
  const int cols = (D[0] * D[1] * D[2]) / n;
  const int nb = (n + TS - 1) / TS, nblk = nb * (nb + 1) / 2;
  const int S = nblk >= (int)blockDim.x ? 1 : min(4, (int)blockDim.x / nblk);
  const int seg = threadIdx.x / nblk;
  int ta = 0, tb = 0;
  {
    int b = threadIdx.x - seg * nblk;
    while (ta < nb && b >= nb - ta) {
      b -= nb - ta;
      ++ta;
    }
    tb = ta + b;
  }
  const bool active = seg < S && ta < nb;
  Real hi[TS][TS], lo[TS][TS];
#pragma unroll
  for (int i = 0; i < TS; ++i)
#pragma unroll
    for (int j = 0; j < TS; ++j) hi[i][j] = lo[i][j] = 0;
  for (int j0 = 0; j0 < cols; j0 += kKC) {
    for (int idx = threadIdx.x; idx < n * kKC; idx += blockDim.x) {
      const int a = idx / kKC, jj = idx - a * kKC, j = j0 + jj;
      Real v = 0;
      if (j < cols) {
        int64_t addr;
        if (m == 0) {
          addr = (int64_t)a * cols + j;
        } else if (m == 1) {
          const int kk = j / D[2], i = j - kk * D[2];
          addr = ((int64_t)kk * D[1] + a) * D[2] + i;
        } else {
          addr = (int64_t)j * D[2] + a;
        }
        v = T[addr];
      }
      sm.tile[a * kKP + jj] = v;
    }
    __syncthreads();
    if (active) {
      const int len = min(kKC, cols - j0);
      const int k0 = seg * len / S, k1 = (seg + 1) * len / S;
#pragma unroll 4
      for (int kk = k0; kk < k1; ++kk) {
        Real xa[TS], xb[TS];
#pragma unroll
        for (int i = 0; i < TS; ++i) {
          const int ra = ta * TS + i, rb = tb * TS + i;
          xa[i] = ra < n ? sm.tile[ra * kKP + kk] : Real(0);
          xb[i] = rb < n ? sm.tile[rb * kKP + kk] : Real(0);
        }
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int j = 0; j < TS; ++j) {
            if constexpr (sizeof(Real) == 8) {
              hi[i][j] = fma(xa[i], xb[j], hi[i][j]);
            } else {
              df_acc(xa[i], xb[j], hi[i][j], lo[i][j]);
            }
          }
      }
      if constexpr (sizeof(Real) == 4) {
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int j = 0; j < TS; ++j) {  // renormalise (fast two-sum)
            const float sum = __fadd_rn(hi[i][j], lo[i][j]);
            lo[i][j] = __fsub_rn(lo[i][j], __fsub_rn(sum, hi[i][j]));
            hi[i][j] = sum;
          }
      }
    }
    __syncthreads();
  }
  for (int sg = 0; sg < S; ++sg) {  // the segments' partial sums, in order
    if (active && seg == sg) {
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) {
          const int a = ta * TS + i, b = tb * TS + j;
          // a diagonal block holds entry (a, b) twice, as (i, j) and (j, i): take it once
          if (a < n && b < n && (ta < tb || i <= j)) {
            Real h = hi[i][j], l = lo[i][j];
            if (sg > 0) {
              if constexpr (sizeof(Real) == 8) {
                h += sm.C[a * n + b];
              } else {
                const float2 c = reinterpret_cast<const float2 *>(sm.C)[a * n + b];
                df_add_into(h, l, c.x, c.y);
              }
            }
            gram_store<Real>(sm.C, a * n + b, h, l);
            gram_store<Real>(sm.C, b * n + a, h, l);
          }
        }
    }
    __syncthreads();
  }
}

// Double-float (hi, lo) sum of two pairs (Knuth's two-sum of the high parts,
// low parts added), renormalised.
__device__ __forceinline__ void df_add(float &hi, float &lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  const float t = __fadd_rn(__fadd_rn(lo, l2), err);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Gram matrix for n <= 32 with every thread of a 256-thread CTA busy: the upper
// triangle of the 8 x 8 grid of 4 x 4 blocks is 28 off-diagonal blocks plus 8
// diagonal ones, taken as 28 + 4 work items (a diagonal item is two diagonal
// blocks, 2 x 10 distinct entries); each item is split 8 ways over the
// columns of every tile (group g takes tile columns g, g + 8, ...).  The 8
// partial sums of an entry sit in 8 adjacent lanes and are combined by a fixed
// shuffle tree (double-float on the mixed path), so the result does not depend
// on scheduling.  Same precision contract as gram_tiled.
template <typename Real>
__device__ __noinline__ void gram_w32(const Real *T, const int D[3], int m, Smem<Real> &sm,
                                      double skip_rel) {
  constexpr bool f32 = sizeof(Real) == 4;
  const int n = D[m];
  const int cols_all = (D[0] * D[1] * D[2]) / n;
  // First mode: columns whose energy is at most skip_rel of the tensor's are left
  // out (their total, the "dropped" energy, is returned in sm.par[26] for the
  // caller's error budget); the kept columns are listed in order in sm.cidx.
  const bool select = m == 0 && skip_rel > 0.0 && sm.cidx && cols_all <= sm.cidx_cap &&
                      cols_all <= 4 * (int)blockDim.x;
  int cols = cols_all;
  if (select) {
    float e[4];
    double part = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * threadIdx.x + q;
      float s = 0.f;
      if (j < cols_all)
        for (int a = 0; a < n; ++a) {
          const float v = (float)T[(int64_t)a * cols_all + j];
          s = fmaf(v, v, s);
        }
      e[q] = s;
      part += (double)s;
    }
    const double total = block_sum_d(part, sm.red);
    const float cut = (float)(skip_rel * total);
    int keep = 0;
    double drop = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * threadIdx.x + q;
      if (j >= cols_all) continue;
      if (e[q] > cut) ++keep;
      else drop += (double)e[q];
    }
    int kept_total;
    int off = block_scan_excl(keep, reinterpret_cast<int *>(sm.red), &kept_total);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * threadIdx.x + q;
      if (j < cols_all && e[q] > cut) sm.cidx[off++] = j;
    }
    // FP32 column energies: the dropped total is raised by a relative 1e-5 so that
    // it bounds the exact one
    drop = block_sum_d(drop, sm.red) * (1.0 + 1e-5);
    if (threadIdx.x == 0) sm.par[26] = drop;
    cols = kept_total;
    __syncthreads();
  } else if (m == 0 && threadIdx.x == 0) {
    sm.par[26] = 0.0;
  }
  const int item = threadIdx.x >> 3, g = threadIdx.x & 7;
  const bool diag = item >= 28;
  int ta, tb;
  if (!diag) {  // item -> (ta < tb), row-major over the strict upper triangle
    int t = item;
    ta = 0;
    while (t >= 7 - ta) {
      t -= 7 - ta;
      ++ta;
    }
    tb = ta + 1 + t;
  } else {
    ta = item - 28;  // diagonal blocks ta and ta + 4
    tb = ta + 4;
  }
  Real hi[20], lo[20];
#pragma unroll
  for (int i = 0; i < 20; ++i) hi[i] = lo[i] = Real(0);
  // tiles of kKC columns; each thread stages 32 * kKC / 256 elements of the next
  // tile in registers while the current one is used (two buffers when
  // sm.tile2 is set: one barrier per tile)
  constexpr int kPer = 32 * kKC / 256;
  Real pre[kPer];
  auto fetch = [&](int j0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int idx = threadIdx.x + 256 * q;
      const int a = idx / kKC, jj = idx - a * kKC, j = j0 + jj;
      Real v = 0;
      if (a < n && j < cols) {
        int64_t addr;
        if (m == 0) {
          addr = (int64_t)a * cols_all + (select ? sm.cidx[j] : j);
        } else if (m == 1) {
          const int kk = j / D[2], i = j - kk * D[2];
          addr = ((int64_t)kk * D[1] + a) * D[2] + i;
        } else {
          addr = (int64_t)j * D[2] + a;
        }
        v = T[addr];
      }
      pre[q] = v;
    }
  };
  auto stage = [&](Real *buf) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int idx = threadIdx.x + 256 * q;
      const int a = idx / kKC, jj = idx - a * kKC;
      buf[a * kKP2 + jj] = pre[q];
    }
  };
  fetch(0);
  stage(sm.tile);
  __syncthreads();
  for (int j0 = 0, t = 0; j0 < cols; j0 += kKC, ++t) {
    const Real *cur = (sm.tile2 && (t & 1)) ? sm.tile2 : sm.tile;
    const bool more = j0 + kKC < cols;
    if (more) fetch(j0 + kKC);
#pragma unroll
    for (int q = 0; q < kKC / 8; ++q) {
      const int kk = g + 8 * q;
      Real xa[4], xb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xa[i] = cur[(4 * ta + i) * kKP2 + kk];
        xb[i] = cur[(4 * tb + i) * kKP2 + kk];
      }
      if (!diag) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if constexpr (f32) df_acc(xa[i], xb[j], hi[4 * i + j], lo[4 * i + j]);
            else hi[4 * i + j] = fma(xa[i], xb[j], hi[4 * i + j]);
          }
      } else {
        int e = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = i; j < 4; ++j, ++e) {
            if constexpr (f32) {
              df_acc(xa[i], xa[j], hi[e], lo[e]);
              df_acc(xb[i], xb[j], hi[10 + e], lo[10 + e]);
            } else {
              hi[e] = fma(xa[i], xa[j], hi[e]);
              hi[10 + e] = fma(xb[i], xb[j], hi[10 + e]);
            }
          }
      }
    }
    if constexpr (f32) {
      if ((t & 3) == 3 || !more) {  // renormalise (fast two-sum) every 4 tiles: the low
#pragma unroll                      // word takes at most 16 additions in between
        for (int i = 0; i < 20; ++i) {
          const float sum = __fadd_rn(hi[i], lo[i]);
          lo[i] = __fsub_rn(lo[i], __fsub_rn(sum, hi[i]));
          hi[i] = sum;
        }
      }
    }
    if (sm.tile2) {
      if (more) stage((t & 1) ? sm.tile : sm.tile2);
      __syncthreads();
    } else {
      __syncthreads();
      if (more) {
        stage(sm.tile);
        __syncthreads();
      }
    }
  }
  // combine the 8 column groups (lanes 8*item' + g of this warp)
#pragma unroll
  for (int i = 0; i < 20; ++i) {
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const Real h2 = __shfl_xor_sync(0xffffffffu, hi[i], o);
      if constexpr (f32) {
        const float l2 = __shfl_xor_sync(0xffffffffu, lo[i], o);
        df_add(hi[i], lo[i], h2, l2);
      } else {
        hi[i] = hi[i] + h2;
      }
    }
  }
  if (g == 0) {
    auto put = [&](int a, int b, Real h, Real l) {
      if (a < n && b < n) {
        gram_store<Real>(sm.C, a * n + b, h, l);
        gram_store<Real>(sm.C, b * n + a, h, l);
      }
    };
    if (!diag) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          put(4 * ta + i, 4 * tb + j, hi[4 * i + j], lo[4 * i + j]);
    } else {
      int e = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j, ++e) {
          put(4 * ta + i, 4 * ta + j, hi[e], lo[e]);
          put(4 * tb + i, 4 * tb + j, hi[10 + e], lo[10 + e]);
        }
    }
  }
  __syncthreads();
}

// Gram matrix of a second- or third-mode unfolding with n <= 32 rows by 256 threads:
// one thread per entry of the upper triangle (at most three each), each a sequential
// sum over the columns in order — double-float with exact products, renormalised
// every 16 products, on the mixed path; FP64 FMAs on the FP64 path — with the columns
// staged 32 at a time in sm.tile.  The result does not depend on the block size.  These
// unfoldings are small (r1 N3 or r1 r2 columns), and gram_w32's 40 register
// accumulators per thread would hold the kernel to two blocks per SM.
template <typename Real>
__device__ __noinline__ void gram_seq(const Real *T, const int D[3], int m, Smem<Real> &sm) {
  constexpr bool f32 = sizeof(Real) == 4;
  const int n = D[m];
  const int cols = (D[0] * D[1] * D[2]) / n;
  const int ne = n * (n + 1) / 2;
  int ea[3], eb[3];
  Real hi[3], lo[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = threadIdx.x + 256 * q;
    ea[q] = -1;
    eb[q] = -1;
    hi[q] = lo[q] = Real(0);
    if (e < ne) {
      int a = 0, t = e;  // e -> (a <= b), row-major over the upper triangle
      while (t >= n - a) {
        t -= n - a;
        ++a;
      }
      ea[q] = a;
      eb[q] = a + t;
    }
  }
  for (int j0 = 0; j0 < cols; j0 += kKC) {
    for (int idx = threadIdx.x; idx < n * kKC; idx += blockDim.x) {
      const int a = idx / kKC, jj = idx - a * kKC, j = j0 + jj;
      Real v = 0;
      if (j < cols) {
        int64_t addr;
        if (m == 1) {
          const int kk = j / D[2], i = j - kk * D[2];
          addr = ((int64_t)kk * D[1] + a) * D[2] + i;
        } else {
          addr = (int64_t)j * D[2] + a;
        }
        v = T[addr];
      }
      sm.tile[a * kKP2 + jj] = v;
    }
    __syncthreads();
    const int cn = cols - j0 < kKC ? cols - j0 : kKC;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (ea[q] < 0) continue;
      const Real *xa = sm.tile + ea[q] * kKP2, *xb = sm.tile + eb[q] * kKP2;
      for (int jj = 0; jj < cn; ++jj) {
        if constexpr (f32) {
          df_acc(xa[jj], xb[jj], hi[q], lo[q]);
          if ((jj & 15) == 15 || jj == cn - 1) {  // fast two-sum renormalisation
            const float sum = __fadd_rn(hi[q], lo[q]);
            lo[q] = __fsub_rn(lo[q], __fsub_rn(sum, hi[q]));
            hi[q] = sum;
          }
        } else {
          hi[q] = fma(xa[jj], xb[jj], hi[q]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (ea[q] < 0) continue;
    gram_store<Real>(sm.C, ea[q] * n + eb[q], hi[q], lo[q]);
    gram_store<Real>(sm.C, eb[q] * n + ea[q], hi[q], lo[q]);
  }
  __syncthreads();
}

// n <= 32 with 256 threads: gram_w32 (first mode) or gram_seq (second and third
// modes); otherwise the 16 x 16 thread grid (TS = 2 covers n <= 32, TS = 4 covers n <= 64)
template <typename Real, int TS>
__device__ void gram(const Real *T, const int D[3], int m, Smem<Real> &sm, double skip_rel = 0.0) {
  if (m >= 1 && D[m] <= 32 && blockDim.x == 256) {
    gram_seq<Real>(T, D, m, sm);
  } else if (D[m] <= 32 && blockDim.x == 256) {
    gram_w32<Real>(T, D, m, sm, skip_rel);
  } else {
    gram_tiled<Real, TS>(T, D, m, sm);
    if (m == 0 && threadIdx.x == 0) sm.par[26] = 0.0;
    __syncthreads();
  }
}

// relative energy below which a first-mode Gram column is left out: all such
// columns together hold at most 1e-3 of the first mode's truncation budget
// (eps^2/3 of the energy)
__host__ __device__ inline double gram_skip_rel(double eps, int cols) {
  return eps > 0.0 ? 1e-3 * (eps * eps / 3.0) / (double)cols : 0.0;
}

// ---------------------------------------------------------------------------
// Dense helpers on shared-memory matrices (row-major).

// W[n x k] = C[n x n] Q[n x k]
template <typename T>
__device__ void mat_cq(const T *__restrict__ C, const T *Q, T *W, int n, int k) {
  for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
    const int i = idx / k, j = idx - i * k;
    T s = 0;
    // C is stored exactly symmetric: C[i][t] is read as C[t][i], so the lanes of
    // a warp (consecutive i) touch consecutive words
    for (int t = 0; t < n; ++t) s = fma(C[t * n + i], Q[t * k + j], s);
    W[idx] = s;
  }
  __syncthreads();
}

// W = C_hi Q in FP32 (the mixed path's orthogonal iterations), C_hi the leading
// float of every double-float Gram entry, read by columns like mat_cq
__device__ void mat_cq_hi(const float2 *__restrict__ C, const float *Q, float *W, int n, int k) {
  // four columns of a row at a time (independent chains; each entry's sum in t order)
  const int ng = (k + 3) >> 2;
  for (int idx = threadIdx.x; idx < n * ng; idx += blockDim.x) {
    const int i = idx / ng, j0 = 4 * (idx - i * ng), nq = min(4, k - j0);
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < n; ++t) {
      const float c = C[t * n + i].x;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nq) s[q] = fmaf(c, Q[t * k + j0 + q], s[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) W[i * k + j0 + q] = s[q];
  }
  __syncthreads();
}

// One term of a double-float inner product sum_t (c_t.hi + c_t.lo) (vh_t + vl_t):
// (hi, lo) += (ct.x + ct.y) (h + l), the leading product exact (fma) and a two-sum
// accumulation: about 2^-48 relative over the sum.
__device__ __forceinline__ void df_mac(float2 ct, float h, float l, float &hi, float &lo) {
  const float p = __fmul_rn(ct.x, h);
  const float pe = __fmaf_rn(ct.x, h, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, __fmaf_rn(ct.x, l, __fmaf_rn(ct.y, h, pe))));
}

// Double-float inner products of row i of the symmetric double-float matrix C (n x n, read
// by columns: the lanes of a warp, one row each, read consecutive entries) with up to four
// columns j0 .. j0 + 3 of V (n x k, hi parts vh, lo parts vl or none) at once: each sum in
// t order by df_mac, four independent chains
__device__ __forceinline__ void df_dot4(const float2 *C, int n, int i, const float *vh,
                                        const float *vl, int k, int j0, double (&out)[4]) {
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
  const int nq = min(4, k - j0);
  for (int t = 0; t < n; ++t) {
    const float2 ct = C[t * n + i];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) df_mac(ct, vh[t * k + j0 + q], vl ? vl[t * k + j0 + q] : 0.f, hi[q], lo[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = (double)hi[q] + (double)lo[q];
}

constexpr int kOrthMax = 24;  // largest number of basis columns

// deterministic start vectors in [-1, 1)
__device__ __forceinline__ double start_value(int i, int j) {
  unsigned h = 0x9E3779B9u * (unsigned)(i + 1) ^ (0x85EBCA6Bu * (unsigned)(j + 7));
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (double)(h & 0xFFFFFF) / 8388608.0 - 1.0;
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// G = Q^T Q for the k columns of Q (n x k), accumulated in A, both triangles.
// With at most 16 entries (k <= 5) each entry's sum is split over two adjacent
// lanes (rows of one parity each) and combined by one shuffle, so a single warp
// is fully used; the split depends on k only (the same sums in any block size).
template <typename T, typename A>
__device__ void gram_cols(const T *Q, int n, int k, A *Gs) {
  const int ne = k * (k + 1) / 2;
  const int parts = ne <= 16 ? 2 : 1;
  for (int base = 0; base < ne * parts; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const int e = idx / parts, h = idx - e * parts;
    int a = 0, b = 0;
    A s = 0;
    if (e < ne) {
      int t = e;  // e -> (a <= b), row-major over the upper triangle
      while (t >= k - a) {
        t -= k - a;
        ++a;
      }
      b = a + t;
      for (int r = h; r < n; r += parts) s = fma((A)Q[r * k + a], (A)Q[r * k + b], s);
    }
    if (parts == 2) s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (e < ne && h == 0) {
      Gs[a * k + b] = s;
      Gs[b * k + a] = s;
    }
  }
}

// Cholesky factor of the k x k symmetric matrix Gs + shift I, by warp 0: lane i
// keeps row i in registers; right-looking, the pivot and the new column entries
// are broadcast by shuffles.  On exit the lower triangle of Gs holds L and
// dinv[j] = 1 / L_jj.  Column j is dependent when its pivot is not positive or
// not above rel * G_jj (the part of the column outside the span of the previous
// ones has lost all accurate digits): dinv[j] = 0, so the solve below zeroes
// it.  Returns the number of dependent columns (the same on every lane).
// Called by warp 0 only; KM >= k bounds the register arrays.
template <typename A, int KM>
__device__ __noinline__ int chol_warp(A *Gs, A *dinv, int k, A shift, A rel) {
  const int lane = threadIdx.x & 31;
  const A tiny = (A)(sizeof(A) == 8 ? 1e-300 : 1e-30);
  A g[KM];
  const A diag0 = lane < k ? Gs[lane * k + lane] : A(0);
  if (lane < k) Gs[lane * k + lane] = diag0 + shift;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < KM; ++c) g[c] = (lane < k && c < k) ? Gs[lane * k + c] : A(0);
  int ndep = 0;
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    if (j < k) {
      const A d = __shfl_sync(0xffffffffu, g[j], j);
      bool dep = !(d > tiny);
      if (rel > A(0)) dep = dep || !(d > rel * __shfl_sync(0xffffffffu, diag0, j));
      const A inv = dep ? A(0) : rsqrt_t(d);
      ndep += dep;
      const A lij = lane > j ? g[j] * inv : A(0);
#pragma unroll
      for (int c = j + 1; c < KM; ++c)
        if (c < k) g[c] = fma(-lij, __shfl_sync(0xffffffffu, lij, c), g[c]);
      if (lane == j) {
        g[j] = dep ? A(1) : d * inv;
        dinv[j] = inv;
      } else if (lane > j) {
        g[j] = lij;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < KM; ++c)
    if (lane < k && c <= lane) Gs[lane * k + c] = g[c];
  __syncwarp();
  return ndep;
}

// Q <- Q L^{-T}: every row x of Q solves y L^T = x (forward substitution, one
// thread per row, the row held in registers).
template <typename T, typename A, int KM>
__device__ __noinline__ void solve_rows(T *Q, int n, int k, const A *L, const A *dinv) {
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    A y[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) {
      if (j < k) {
        A v = (A)Q[r * k + j];
#pragma unroll
        for (int i = 0; i < j; ++i) v = fma(-y[i], L[j * k + i], v);
        y[j] = v * dinv[j];
      }
    }
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) Q[r * k + j] = (T)y[j];
  }
}

// Treatment of numerically dependent columns by orthonormalise()
constexpr int kDepNone = 0;    // no relative test (only breakdown zeroes a column)
constexpr int kDepZero = 1;    // relative test; dependent columns are zeroed
constexpr int kDepReseed = 2;  // relative test; dependent columns are re-seeded

// Orthonormalise the k <= n columns of Q (n x k, row-major) in place by
// Cholesky-QR repeated `passes` times: G = Q^T Q, its Cholesky factor L, then
// Q <- Q L^{-T}; arithmetic in A.  The first pass factors G + shift_rel *
// trace(G) I instead (shifted Cholesky-QR, Fukaya et al. 2020): the shift keeps
// the factorisation from breaking down on nearly dependent columns while leaving
// span(Q) unchanged, and the following unshifted passes restore orthonormality
// to the working precision.  With dep != kDepNone (the last step of an
// eigen-solve) the unshifted passes also flag columns that are numerically
// dependent (pivot <= 1e-10 G_jj: the part outside the span of the previous
// columns has no accurate digits left) and zero them, so the non-zero columns
// are orthonormal to round-off.  With kDepReseed (where the basis must keep full
// rank) flagged columns are then replaced by fresh start vectors and two more
// passes run (at most two such rounds).  Returns the number of non-zero columns;
// *reseeds (if given) receives the number of re-seeding rounds.  Gs (k x k) and
// dinv (k) are scratch in shared memory; ends with a barrier.
template <typename T, typename A>
__device__ __noinline__ int orthonormalise(T *Q, int n, int k, A *Gs, A *dinv, int passes,
                                           double shift_rel, int dep, int *reseeds = nullptr) {
  const bool reseed = dep == kDepReseed;
  __shared__ int s_dep;
  int round = 0;
  for (; round < 3; ++round) {
    for (int pass = 0; pass < passes; ++pass) {
      const bool shifted = round == 0 && pass == 0;
      gram_cols<T, A>(Q, n, k, Gs);
      __syncthreads();
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        A tr = lane < k ? Gs[lane * k + lane] : A(0);
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        const A shift = shifted ? (A)shift_rel * tr : A(0);
        const A rel = (dep != kDepNone && !shifted) ? A(1e-10) : A(0);
        // register arrays sized for k (the arithmetic does not depend on the size)
        const int ndep = k <= 8    ? chol_warp<A, 8>(Gs, dinv, k, shift, rel)
                         : k <= 16 ? chol_warp<A, 16>(Gs, dinv, k, shift, rel)
                                   : chol_warp<A, kOrthMax>(Gs, dinv, k, shift, rel);
        if (lane == 0) s_dep = ndep;
      }
      __syncthreads();
      if (k <= 8)
        solve_rows<T, A, 8>(Q, n, k, Gs, dinv);
      else if (k <= 16)
        solve_rows<T, A, 16>(Q, n, k, Gs, dinv);
      else
        solve_rows<T, A, kOrthMax>(Q, n, k, Gs, dinv);
      __syncthreads();
    }
    if (!reseed || s_dep == 0 || round == 2) break;
    for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
      const int j = idx % k;
      if (dinv[j] == A(0)) Q[idx] = (T)start_value(idx / k, j + 131 * (round + 1));
    }
    __syncthreads();
    passes = 2;
  }
  const int nz = k - s_dep;
  if (reseeds) *reseeds = round < 3 ? round : 2;
  __syncthreads();
  return nz;
}

// Leading eigenvectors of the n x n Gram matrix sm.Cg by orthogonal (block
// power) iteration with k basis columns: the start block is the warm basis
// (r_warm columns, row stride ldw: the previous step's orthonormal factor, which
// spans most of the new dominant subspace) completed by fixed start vectors.
// FP64 path: FP64 iterations.  Mixed path: FP32 iterations on the rounded Gram
// matrix, then one FP64 step on the accurate one.  Every path ends with an FP64
// shifted Cholesky-QR3, so the basis is orthonormal to FP64 round-off; columns it
// finds dependent are handled as dep_final says (zeroed on a first solve: the
// rank rule never keeps a zero column; re-seeded on a retry).  On exit
// sm.W holds the k columns ordered by their Rayleigh quotients (descending), sm.Z
// the sorted quotients, sm.par[29] the number of non-zero columns.  Returns k.
template <typename Real, typename WT>
__device__ __noinline__ int leading_eigs(Smem<Real> &sm, int n, int k, const WT *warm, int ldw, int r_warm,
                            PhaseClock &pc, int dep_final) {
  if (!warm) r_warm = 0;
  if (r_warm > k) r_warm = k;
  const int iters = r_warm > 0 ? kWarmIter : kPower;
  float *G32 = reinterpret_cast<float *>(sm.B), *d32 = reinterpret_cast<float *>(sm.cs);
  if (sizeof(Real) == 8) {
    for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
      const int i = idx / k, j = idx - i * k;
      sm.Q[idx] = j < r_warm ? (double)warm[(int64_t)i * ldw + j] : start_value(i, j);
    }
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
      mat_cq(sm.Cg, sm.Q, sm.W, n, k);
      for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) sm.Q[idx] = sm.W[idx];
      __syncthreads();
      pc.mark(11);
      const bool last = it == iters - 1;
      const int nz = orthonormalise<double, double>(sm.Q, n, k, sm.B, sm.cs, last ? 3 : 2,
                                                    last ? 1e-11 : 1e-12, last ? dep_final : kDepNone);
      if (threadIdx.x == 0) sm.par[29] = (double)nz;
      pc.mark(12);
    }
  } else {
    const float2 *Cdf = reinterpret_cast<const float2 *>(sm.Cg);
    for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
      const int i = idx / k, j = idx - i * k;
      sm.Q32[idx] = (float)(j < r_warm ? (double)warm[(int64_t)i * ldw + j] : start_value(i, j));
    }
    __syncthreads();
    pc.mark(6);
    for (int it = 0; it < iters; ++it) {
      mat_cq_hi(Cdf, sm.Q32, sm.W32, n, k);
      for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) sm.Q32[idx] = sm.W32[idx];
      __syncthreads();
      pc.mark(9);
      orthonormalise<float, float>(sm.Q32, n, k, G32, d32, kF32Passes, 1e-5, kDepNone);
      pc.mark(10);
    }
    // one power step with the accurate Gram matrix: Q = C Q32 in double-float (Q32, in
    // sm.W's space, is read in place: nothing writes sm.W before the Rayleigh quotients)
    const float *V = sm.Q32;
    const int ng = (k + 3) >> 2;  // groups of four columns
    for (int idx = threadIdx.x; idx < n * ng; idx += blockDim.x) {
      const int i = idx / ng, j0 = 4 * (idx - i * ng);
      double w[4];
      df_dot4(Cdf, n, i, V, nullptr, k, j0, w);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j0 + q < k) sm.Q[i * k + j0 + q] = w[q];
    }
    __syncthreads();
    pc.mark(11);
    int rounds = 0;
    const int nz = orthonormalise<double, double>(sm.Q, n, k, sm.B, sm.cs, 3, 1e-11, dep_final, &rounds);
    if (threadIdx.x == 0) sm.par[29] = (double)nz;
    pc.mark(12);
    pc.count(1, rounds);
  }
  // Rayleigh quotients d_j = q_j^T C q_j of the orthonormal columns (FP64
  // accuracy): any leading set of columns captures exactly the sum of its d_j, so
  // the columns are ordered by d_j and the rank rule reads them (sorted, in sm.Z).
  // One warp per column, a lane per row, a fixed shuffle tree.  A column the last
  // Cholesky-QR pass zeroed (sm.cs[j] = 1 / L_jj = 0) gets -1, so it sorts after
  // every non-zero column (its captured energy, 0, is what the rank rule adds).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (sizeof(Real) == 8) {
    mat_cq(sm.Cg, sm.Q, sm.W, n, k);
    for (int j = warp; j < k; j += nwarp) {
      double d = 0.0;
      for (int i = lane; i < n; i += 32) d = fma(sm.Q[i * k + j], sm.W[i * k + j], d);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) sm.cs[j] = sm.cs[j] == 0.0 ? -1.0 : d;  // zeroed columns sort last
    }
  } else {
    // (C q_j)_i in double-float with q split into float hi + lo parts (in sm.W)
    const float2 *Cdf = reinterpret_cast<const float2 *>(sm.Cg);
    float *qh = reinterpret_cast<float *>(sm.W), *ql = qh + n * k;
    for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
      const double q = sm.Q[idx];
      const float h = (float)q;
      qh[idx] = h;
      ql[idx] = (float)(q - (double)h);
    }
    __syncthreads();
    // four columns at a time (each lane's rows in order, then the shuffle tree: the same
    // sums as one column at a time)
    for (int j0 = 4 * warp; j0 < k; j0 += 4 * nwarp) {
      double d[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = lane; i < n; i += 32) {
        double w[4];
        df_dot4(Cdf, n, i, qh, ql, k, j0, w);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j0 + q < k) d[q] = fma(sm.Q[i * k + j0 + q], w[q], d[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
        if (lane == 0 && j0 + q < k) sm.cs[j0 + q] = sm.cs[j0 + q] == 0.0 ? -1.0 : d[q];
      }
    }
  }
  __syncthreads();
  pc.mark(14);
  if (warp == 0) {
    if (lane == 0) {  // order columns by quotient, descending
      for (int i = 0; i < k; ++i) sm.perm[i] = i;
      for (int i = 1; i < k; ++i) {
        const int v = sm.perm[i];
        const double lv = sm.cs[v];
        int j = i - 1;
        while (j >= 0 && sm.cs[sm.perm[j]] < lv) {
          sm.perm[j + 1] = sm.perm[j];
          --j;
        }
        sm.perm[j + 1] = v;
      }
      for (int j = 0; j < k; ++j) sm.Z[j] = sm.cs[sm.perm[j]];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
    const int i = idx / k, j = idx - i * k;
    sm.W[idx] = sm.Q[i * k + sm.perm[j]];
  }
  __syncthreads();
  pc.mark(15);
  return k;
}

// Truncation rank from the energy the first r basis vectors capture (tr =
// trace(C)): the smallest r with tr - sum_{j<r} d_j <= thr (thr > 0), else all k; then
// r <- min(r, cap, non-zero columns), r >= 1.  Returns r; *met tells whether
// the threshold was reached within the k columns, sm.par[31] holds the energy
// the r columns leave out.
template <typename Real>
__device__ int choose_rank(Smem<Real> &sm, int n, int k, double thr, int cap, bool *met,
                           double tr) {
  (void)n;
  if (threadIdx.x == 0) {
    double kept = 0.0;
    int r = k, found = 0;
    for (int j = 0; j < k && thr > 0.0; ++j) {
      kept += fmax(sm.Z[j], 0.0);
      if (tr - kept <= thr) {
        r = j + 1;
        found = 1;
        break;
      }
    }
    if (r > cap) r = cap;
    if (r > (int)sm.par[29]) r = (int)sm.par[29];  // never keep zeroed columns
    if (r < 1) r = 1;
    kept = 0.0;
    for (int j = 0; j < r; ++j) kept += fmax(sm.Z[j], 0.0);
    sm.par[28] = (double)found;
    sm.par[30] = (double)r;
    sm.par[31] = fmax(tr - kept, 0.0);
  }
  __syncthreads();
  *met = sm.par[28] != 0.0;
  return (int)sm.par[30];
}

// out = T x_m Vr^T : mode m of T (dims D) contracted with the first r kept
// eigenvectors (sm.Vr, n x k, column j = j-th vector); result dims D with D[m] -> r.
template <typename Real>
__device__ void project(const Real *T, const int D[3], int m, int r, int k, Smem<Real> &sm,
                        Real *out) {
  const int n = D[m];
  int Do[3] = {D[0], D[1], D[2]};
  Do[m] = r;
  const int total = Do[0] * Do[1] * Do[2];
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int i2 = idx % Do[2], t = idx / Do[2], i1 = t % Do[1], i0 = t / Do[1];
    const int ii[3] = {i0, i1, i2};
    const int kk = ii[m];
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
    for (int a = 0; a < n; ++a) s += sm.Vr[a * k + kk] * T[base + a * stride];
    out[idx] = s;
  }
  __syncthreads();
}

// Truncated sequential HOSVD of X (N1 x N2 x N3 in scratch) into the Tucker
// slot `cell` of `out`.  Uses T2 (>= R*N2*N3) and T1 (>= R*R*N3) as work space.
template <typename Real, int TS>
__device__ void round_hosvd(Real *X, Real *T1, Real *T2, const int N[3], int R, double eps,
                            TuckerDev &out, int64_t cell, Smem<Real> &sm, double *err_out,
                            PhaseClock &pc, const TuckerDev *warm) {
  int D[3] = {N[0], N[1], N[2]};
  double e = 0.0, thr = 0.0;  // ||X||^2 = trace of the first Gram matrix
  double discarded = 0.0;
  int r[3];
  pc.mark(4);
  const Real *src = X;
  Real *dst[2] = {T2, T1};
  for (int m = 0; m < 3; ++m) {
    const int n = D[m];
    gram<Real, TS>(src, D, m, sm, m == 0 ? gram_skip_rel(eps, D[1] * D[2]) : 0.0);
    const double tr = gram_trace<Real>(sm, n);
    double dropped = 0.0;  // energy of the columns the first Gram matrix left out
    if (m == 0) {
      dropped = sm.par[26];
      e = tr + dropped;
      thr = eps * eps / 3.0 * e;
    }
    pc.mark(5);
    const double *wU = warm ? warm->fac[m] + cell * (int64_t)N[m] * R : nullptr;
    const int wr = warm ? warm->rank[3 * cell + m] : 0;
    // basis size: the previous rank plus kExtra columns (ranks grow by at most
    // kExtra per step through this path); if the threshold is not reached
    // within them, the solve is repeated with the full basis, warm-started from
    // the columns just found
    int kmax = n < R + kExtra ? n : R + kExtra;
    if (kmax > kOrthMax) kmax = kOrthMax;
    int k = (wU && wr > 0 && thr > 0.0 && wr + kExtra < kmax) ? wr + kExtra : kmax;
    // truncating: dependent columns are zeroed (a zero column is never kept, and the
    // full solve below follows if the rest miss the threshold); exact (no threshold):
    // re-seeded, so the basis spans the whole space
    k = leading_eigs<Real, double>(sm, n, k, wU, R, wr, pc, thr - dropped > 0.0 ? kDepZero : kDepReseed);
    pc.mark(6);
    bool met;
    r[m] = choose_rank<Real>(sm, n, k, thr - dropped, R, &met, tr);
    if (!met && k < kmax) {
      // the k columns found start the full solve (kept in sm.Vr, which the
      // iteration does not touch)
      for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) sm.Vr[idx] = (Real)sm.W[idx];
      __syncthreads();
      k = leading_eigs<Real, Real>(sm, n, kmax, sm.Vr, k, k, pc, kDepReseed);
      pc.mark(6);
      r[m] = choose_rank<Real>(sm, n, k, thr - dropped, R, &met, tr);
    }
    discarded += sm.par[31] + dropped;
    double *U = out.fac[m] + cell * (int64_t)N[m] * R;
    for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
      const int i = idx / k, j = idx - i * k;
      const double v = sm.W[idx];
      sm.Vr[idx] = (Real)v;
      if (j < r[m]) U[(int64_t)i * R + j] = v;
    }
    __syncthreads();
    pc.mark(7);
    if (m < 2) {
      project<Real>(src, D, m, r[m], k, sm, dst[m]);
      D[m] = r[m];
      src = dst[m];
      pc.mark(8);
    } else {
      // core = Y2 x_3 V3^T (FP64 accumulation), compact r1 x r2 x r3
      const int total = D[0] * D[1] * r[2];
      double *G = out.core + cell * (int64_t)R * R * R;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k3 = idx % r[2], k12 = idx / r[2];
        const Real *y = src + (int64_t)k12 * n;
        double s = 0.0;
        for (int a = 0; a < n; ++a) s = fma(sm.W[a * k + k3], (double)y[a], s);
        G[idx] = s;
      }
      __syncthreads();
      pc.mark(8);
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
// Per-cell tables of the assembly (working precision), per axis a:
//   [a] nodes xi_a, [3+a] Maxwellian factor (dt nu folded into a = 0),
//   [6+a] A q_a v_a, [9+a] v_a^2/T, [12+a] self outflow weight
//   -sum_{faces normal to a} c max(s xi_a, 0); [15+l] inflow weight of face l
//   (faces normal to a coordinate axis; scaled by the wall density on walls).
template <typename Real>
__device__ __forceinline__ Real *tabp(Smem<Real> &sm, int Nmax, int t) {
  return sm.rt + t * padN(Nmax);
}

// kRows consecutive values from 16-byte aligned shared memory by 16-byte loads
// (the tables, the first-mode factor rows and row offsets are multiples of 16 bytes)
template <typename Real>
__device__ __forceinline__ void ld_rows(const Real *src, Real (&v)[kRows]) {
  if constexpr (sizeof(Real) == 4) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int q = 0; q < kRows / 4; ++q) {
      const float4 t = s4[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
#pragma unroll
    for (int q = 0; q < kRows / 2; ++q) {
      const double2 t = s2[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Fused assembly of f^{n+1} for one cell (Section 5, Lemma 1) into X, one pass.
//
// Every Tucker tensor the update needs (the cell's own f and the f of each
// interior neighbour) is first contracted over modes 2 and 3:
//   T2_t[k1][i2][i3] = sum_{k2,k3} G_t[k1][k2][k3] U2_t[i2][k2] U3_t[i3][k3]
// (global scratch, compact, one block per distinct tensor), and its first-mode
// rows U1_t are kept in shared memory.  Then one pass over the (i2, i3)
// columns, kRows first-mode rows per thread, forms
//   X = dt nu f^S + sum_{Maxwellian ghosts l} m_l g_l + W_self o f
//       + sum_{interior / symmetry faces l} m_l o f_src(l)
// with f = U1 T2 formed in registers, the Lemma-1 self weight
//   W_self = 1 - dt nu - sum_l c_l (xi.e_l)^+ + sum_{zero-gradient faces l} m_l
// and the inflow weights m_l = -c_l (xi.e_l)^- (times the wall density on
// walls).  A symmetry face reuses the cell's own T2 with the mirrored index
// (rows of U1 reversed, or the mirrored (i2, i3) column).  X is written once and
// its squared norm returned (FP64, block-reduced).
struct AsmTerm {
  int64_t off;  // T2 offset from the T2 base (elements)
  int r1;       // first-mode rank
  int u1;       // U1 row block in sm.u1 (elements)
  int rev;      // 1: first-mode index mirrored
  int reflect;  // 1 / 2: second / third-mode index mirrored; 0 none
  int face;     // weight: -1 the Lemma-1 self weight, else m of face `face`
};

template <typename Real>
__device__ __noinline__ void term_contract(const TuckerDev &T, int64_t cell, const int N[3], int R, int NP,
                              Smem<Real> &sm, Real *u1dst, Real *T2dst, int *r1_out) {
  const int tid = threadIdx.x;
  const int r1 = T.rank[3 * cell], r2 = T.rank[3 * cell + 1], r3 = T.rank[3 * cell + 2];
  const double *U1 = T.fac[0] + cell * (int64_t)N[0] * R;
  const double *U2 = T.fac[1] + cell * (int64_t)N[1] * R;
  const double *U3 = T.fac[2] + cell * (int64_t)N[2] * R;
  const int N1P = padN(N[0]);
  for (int idx = tid; idx < r1 * N1P; idx += blockDim.x) {
    const int k = idx / N1P, i = idx - k * N1P;
    u1dst[idx] = i < N[0] ? (Real)U1[(int64_t)i * R + k] : Real(0);
  }
  for (int idx = tid; idx < N[1] * r2; idx += blockDim.x) {
    const int i = idx / r2, k = idx - i * r2;
    sm.fac[1][idx] = (Real)U2[(int64_t)i * R + k];
  }
  for (int idx = tid; idx < N[2] * r3; idx += blockDim.x) {
    const int i = idx / r3, k = idx - i * r3;
    sm.fac[2][idx] = (Real)U3[(int64_t)i * R + k];
  }
  __syncthreads();
  // mode-3 then mode-2 contraction, a slab of first-mode indices at a time,
  // both stages in shared memory (the Gram / eigen-solver space, free during the
  // assembly): Gs = G[k1 slab], T1s[kk][k2][i3] = sum_k3 Gs[kk][k2][k3] U3[i3][k3],
  // T2[k1][i2][i3] = sum_k2 U2[i2][k2] T1s[kk][k2][i3]
  const double *G = T.core + cell * (int64_t)R * R * R;
  const int N2 = N[1], N3 = N[2];
  const int slabG = r2 * r3, slabT = r2 * N3;
  Real *Gs = reinterpret_cast<Real *>(sm.C);
  const int cap = (int)(asm_space_doubles(sm) * sizeof(double) / sizeof(Real));
  const int kc = max(1, cap / max(1, slabG + slabT));
  for (int k1a = 0; k1a < r1; k1a += kc) {
    const int kn = min(kc, r1 - k1a);
    Real *T1s = Gs + kn * slabG;
    for (int idx = tid; idx < kn * slabG; idx += blockDim.x) Gs[idx] = (Real)G[k1a * slabG + idx];
    __syncthreads();
    for (int idx = tid; idx < kn * slabT; idx += blockDim.x) {
      const int i3 = idx % N3, t = idx / N3;  // t = kk * r2 + k2
      const Real *g = Gs + t * r3;
      const Real *u3 = sm.fac[2] + i3 * r3;
      Real acc = 0;
      for (int k3 = 0; k3 < r3; ++k3) acc = fma(g[k3], u3[k3], acc);
      T1s[idx] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < kn * N2 * N3; idx += blockDim.x) {
      const int i3 = idx % N3, t = idx / N3, i2 = t % N2, kk = t / N2;
      const Real *u2 = sm.fac[1] + i2 * r2;
      const Real *t1 = T1s + kk * slabT + i3;
      Real acc = 0;
      for (int k2 = 0; k2 < r2; ++k2) acc = fma(u2[k2], t1[k2 * N3], acc);
      T2dst[(int64_t)(k1a + kk) * NP + i2 * N3 + i3] = acc;
    }
    __syncthreads();
  }
  if (tid == 0) *r1_out = r1;
  __syncthreads();
}

// The assembly pass proper (see above).  The mode-2/3 contractions come either
// from T2all / U1all (computed once per cell by tucker_t2_kernel: [cell][R][N2 N3]
// and [cell][R][padN(N1)]) or, when T2all is null, are formed here into T2buf.
// kRowMax: also write the largest magnitude of each first-mode row of X to rowmax[N1]
// (the row scales of the tensor-core Gram matrix), kept per thread while its items stay
// in one block of rows and combined by shared-memory atomics (non-negative floats order
// as their bit patterns)
template <typename Real, bool kRowMax = false>
__device__ __noinline__ void assemble(const TuckerStepParams &P, int64_t c, const int N[3],
                                      Smem<Real> &sm, const SlotDev *s_slot,
                                      const double *s_scale, Real *X, Real *T2buf,
                                      const Real *T2all, const Real *U1all, PhaseClock &pc,
                                      float *rowmax = nullptr) {
  __shared__ AsmTerm s_term[1 + 2 * 6];
  __shared__ int s_r1[kTerms];
  __shared__ unsigned s_rmax[kRowMax ? 64 : 1];
  const int tid = threadIdx.x;
  if (kRowMax && tid < 64) s_rmax[tid] = 0u;
  const int N1 = N[0], N2 = N[1], N3 = N[2], NP = N2 * N3, Nm = P.Nmax, R = P.R;
  const int N1P = padN(N1), u1slot = R * padN(Nm);
  int nsrc = 0;
  int64_t off = 0;
  int64_t src_off[kTerms];
  int src_r1[kTerms];
  bool mirror1 = false;  // a symmetry face mirrors the first-mode index
  for (int l = -1; l < 6; ++l) {
    if (l >= 0 && s_slot[l].kind == kSymmetry && s_slot[l].flip == 0) mirror1 = true;
    if (l >= 0 && s_slot[l].kind != kInterior) continue;
    const int64_t cell = l < 0 ? c : (int64_t)s_slot[l].src;
    if (T2all) {  // precomputed: first-mode rows to shared memory
      const int r1 = P.cur.rank[3 * cell];
      const Real *u = U1all + cell * (int64_t)R * N1P;
      Real *d = sm.u1 + nsrc * u1slot;
      for (int idx = tid; idx < r1 * N1P; idx += blockDim.x) d[idx] = u[idx];
      src_off[nsrc] = cell * (int64_t)R * NP;
      src_r1[nsrc] = r1;
    } else {  // contraction of the cell's own tensor / each interior neighbour here
      term_contract<Real>(P.cur, cell, N, R, NP, sm, sm.u1 + nsrc * u1slot, T2buf + off,
                          &s_r1[nsrc]);
      src_off[nsrc] = off;
      src_r1[nsrc] = s_r1[nsrc];
      off += (int64_t)s_r1[nsrc] * NP;
    }
    ++nsrc;
  }
  if (T2all) __syncthreads();
  const Real *T2base = T2all ? T2all : T2buf;
  if (mirror1) {  // the cell's own first-mode factor with rows reversed, in the spare slot
    Real *dst = sm.u1 + kTerms * u1slot;
    for (int idx = tid; idx < src_r1[0] * N1P; idx += blockDim.x) {
      const int k = idx / N1P, i = idx - k * N1P;
      dst[idx] = i < N1 ? sm.u1[k * N1P + N1 - 1 - i] : Real(0);
    }
  }
  // term list: self, interior faces, symmetry faces (the mirrored self)
  int nterm = 0;
  bool self_extra = false;  // faces that change the self weight pointwise
  {
    int q = 0;
    for (int l = -1; l < 6; ++l) {
      if (l >= 0) {
        const SlotDev &sl = s_slot[l];
        if (sl.axis < 0 || sl.kind == kZeroGrad) self_extra = true;
        if (sl.kind != kInterior && sl.kind != kSymmetry) continue;
      }
      AsmTerm tm;
      const bool sym = l >= 0 && s_slot[l].kind == kSymmetry;
      const int qs = (l < 0 || sym) ? 0 : ++q;
      tm.off = src_off[qs];
      tm.r1 = src_r1[qs];
      tm.rev = sym && s_slot[l].flip == 0;
      tm.u1 = tm.rev ? kTerms * u1slot : qs * u1slot;
      tm.reflect = sym ? (s_slot[l].flip == 1 ? 1 : (s_slot[l].flip == 2 ? 2 : 0)) : 0;
      tm.face = l;
      if (tid == 0) s_term[nterm] = tm;
      ++nterm;
    }
  }
  __syncthreads();
  pc.mark(13);
  // face coefficients in the working precision: e0, e1, e2, c, wall-density scale
  __shared__ Real s_fr[6 * 5];
  if (tid < 30) {
    const int l = tid / 5, q = tid - l * 5;
    const SlotDev &sl = s_slot[l];
    s_fr[tid] = (Real)(q < 3 ? sl.e[q] : (q == 3 ? sl.c : s_scale[l]));
  }
  __syncthreads();
  const Real *ghostR = sizeof(Real) == 8 ? reinterpret_cast<const Real *>(P.ghostf)
                                         : reinterpret_cast<const Real *>(P.ghostf32);
  const Real w0 = (Real)(1.0 - sm.par[8]);
  const Real *x0 = tabp(sm, Nm, 0), *x1 = tabp(sm, Nm, 1), *x2 = tabp(sm, Nm, 2);
  const Real *F0 = tabp(sm, Nm, 3), *F1 = tabp(sm, Nm, 4), *F2 = tabp(sm, Nm, 5);
  const Real *Q0 = tabp(sm, Nm, 6), *Q1 = tabp(sm, Nm, 7), *Q2 = tabp(sm, Nm, 8);
  const Real *V0 = tabp(sm, Nm, 9), *V1 = tabp(sm, Nm, 10), *V2 = tabp(sm, Nm, 11);
  const Real *G0 = tabp(sm, Nm, 12), *G1 = tabp(sm, Nm, 13), *G2 = tabp(sm, Nm, 14);
  const int nch = N1P / kRows;
  float rm[kRowMax ? kRows : 1];
  int rm_ch = -1;
  auto flush_rows = [&]() {
    if constexpr (kRowMax) {
      if (rm_ch >= 0) {
#pragma unroll
        for (int j = 0; j < kRows; ++j)
          if (rm_ch * kRows + j < N1) atomicMax(&s_rmax[rm_ch * kRows + j], __float_as_uint(rm[j]));
      }
    }
  };
  for (int item = tid; item < NP * nch; item += blockDim.x) {
    const int p = item % NP, ch = item / NP;
    if constexpr (kRowMax) {
      if (ch != rm_ch) {
        flush_rows();
        rm_ch = ch;
#pragma unroll
        for (int j = 0; j < kRows; ++j) rm[j] = 0.f;
      }
    }
    const int i2 = p / N3, i3 = p - i2 * N3;
    const int i10 = ch * kRows;  // rows i10 .. i10 + kRows - 1 (tables zero-padded)
    Real acc[kRows], sv[kRows];
    // equilibrium term dt nu f^S (Proposition 1: Maxwellian factors times the
    // cubic Shakhov polynomial)
    {
      const Real fM12 = F1[i2] * F2[i3], Qp = Q1[i2] + Q2[i3], Vp = V1[i2] + V2[i3] - Real(2.5);
      Real f0[kRows], q0[kRows], v0[kRows];
      ld_rows(F0 + i10, f0);
      ld_rows(Q0 + i10, q0);
      ld_rows(V0 + i10, v0);
#pragma unroll
      for (int j = 0; j < kRows; ++j) acc[j] = f0[j] * fM12 * (Real(1) + (q0[j] + Qp) * (v0[j] + Vp));
    }
    // rank-1 Maxwellian ghosts (free stream, diffuse wall)
    for (int l = 0; l < 6; ++l) {
      const SlotDev &sl = s_slot[l];
      if (sl.kind != kFreeStream && sl.kind != kWall) continue;
      const Real *gf = ghostR + (int64_t)sl.src * 3 * Nm;
      const Real g23 = gf[Nm + i2] * gf[2 * Nm + i3];
      const Real *tab = tabp(sm, Nm, 15 + l);
      const Real *fr = s_fr + 5 * l;
      const Real e0 = fr[0], cl = fr[3], sc = fr[4];
      const Real xn23 = fr[1] * x1[i2] + fr[2] * x2[i3];
      const Real m23 = sl.axis == 1 ? tab[i2] : (sl.axis == 2 ? tab[i3] : Real(0));
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        const int i1 = i10 + j;
        Real m;
        if (sl.axis == 0) m = tab[i1];
        else if (sl.axis > 0) m = m23;
        else m = -cl * fmin(e0 * x0[i1] + xn23, Real(0)) * sc;
        acc[j] = fma(m, gf[min(i1, N1 - 1)] * g23, acc[j]);
      }
    }
    pc.mark(5);
    // Tucker terms: f = U1 T2 in registers, then the weight
    for (int t = 0; t < nterm; ++t) {
      const AsmTerm tm = s_term[t];
      int pp = p;
      if (tm.reflect == 1) pp = (N2 - 1 - i2) * N3 + i3;
      else if (tm.reflect == 2) pp = i2 * N3 + (N3 - 1 - i3);
      const Real *t2 = T2base + tm.off + pp;
      const Real *u1 = sm.u1 + tm.u1 + i10;
#pragma unroll
      for (int j = 0; j < kRows; ++j) sv[j] = 0;
      for (int k1 = 0; k1 < tm.r1; k1 += 4) {  // four loads in flight
        Real tv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) tv[q] = k1 + q < tm.r1 ? t2[(int64_t)(k1 + q) * NP] : Real(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (k1 + q < tm.r1) {
            Real ur[kRows];
            ld_rows(u1 + (k1 + q) * N1P, ur);
#pragma unroll
            for (int j = 0; j < kRows; ++j) sv[j] = fma(ur[j], tv[q], sv[j]);
          }
        }
      }
      if (tm.face < 0) {  // Lemma-1 self weight
        const Real c0p = w0 + G1[i2] + G2[i3];
        Real g0[kRows];
        ld_rows(G0 + i10, g0);
#pragma unroll
        for (int j = 0; j < kRows; ++j) acc[j] = fma(c0p + g0[j], sv[j], acc[j]);
        // outflow of faces whose normal is not a coordinate axis, inflow of
        // zero-gradient faces (their ghost is the cell itself)
        for (int l = 0; self_extra && l < 6; ++l) {
          const SlotDev &sl = s_slot[l];
          const bool nonaxis = sl.axis < 0, zg = sl.kind == kZeroGrad;
          if (!nonaxis && !zg) continue;
          const Real *fr = s_fr + 5 * l;
          const Real e0 = fr[0], cl = fr[3], sc = fr[4];
          const Real *tab = tabp(sm, Nm, 15 + l);
          const Real xn23 = fr[1] * x1[i2] + fr[2] * x2[i3];
          const Real m23 = sl.axis == 1 ? tab[i2] : (sl.axis == 2 ? tab[i3] : Real(0));
#pragma unroll
          for (int j = 0; j < kRows; ++j) {
            const int i1 = i10 + j;
            Real wadd;
            if (nonaxis) {
              const Real xn = e0 * x0[i1] + xn23;
              wadd = -cl * fmax(xn, Real(0));
              if (zg) wadd -= cl * fmin(xn, Real(0)) * sc;
            } else {
              wadd = sl.axis == 0 ? tab[i1] : m23;
            }
            acc[j] = fma(wadd, sv[j], acc[j]);
          }
        }
      } else {
        const SlotDev &sl = s_slot[tm.face];
        const Real *tab = tabp(sm, Nm, 15 + tm.face);
        if (sl.axis == 0) {
          Real tr[kRows];
          ld_rows(tab + i10, tr);
#pragma unroll
          for (int j = 0; j < kRows; ++j) acc[j] = fma(tr[j], sv[j], acc[j]);
        } else if (sl.axis > 0) {
          const Real m = sl.axis == 1 ? tab[i2] : tab[i3];
#pragma unroll
          for (int j = 0; j < kRows; ++j) acc[j] = fma(m, sv[j], acc[j]);
        } else {
          const Real *fr = s_fr + 5 * tm.face;
          const Real e0 = fr[0], cl = fr[3], sc = fr[4];
          const Real xn23 = fr[1] * x1[i2] + fr[2] * x2[i3];
          const Real *xr = x0 + i10;
#pragma unroll
          for (int j = 0; j < kRows; ++j) {
            const Real xn = e0 * xr[j] + xn23;
            acc[j] = fma(-cl * fmin(xn, Real(0)) * sc, sv[j], acc[j]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const int i1 = i10 + j;
      if (i1 < N1) __stcs(X + (int64_t)i1 * NP + p, acc[j]);  // streamed past L2
      if constexpr (kRowMax) rm[j] = fmaxf(rm[j], fabsf((float)acc[j]));
    }
    pc.mark(3);
  }
  flush_rows();
  __syncthreads();
  if constexpr (kRowMax) {
    for (int i = tid; i < N1; i += blockDim.x) rowmax[i] = __uint_as_float(s_rmax[i]);
  }
}

// The cell's parameters from its moment sums (Section 4 item 5): n, u, T, q
// (out[0..7]), dt nu with nu = delta n T^(1 - omega) (out[8]), the Shakhov
// coefficient (8/5)(1 - Pr)/(n T^2) (out[9]) and the Maxwellian amplitude
// n^(1/3) / sqrt(pi T) of each per-axis factor (out[10]).  Sets bit 0 of *P.flag
// for a non-physical state.
template <typename Params>
__device__ void cell_params(const double *S, const Params &P, double *out) {
  CellMacro m;
  macro_from_sums(S, P.w, m);
  if (m.bad) atomicOr(P.flag, 1);
  const double nu = P.delta * m.n * pow(m.T, 1.0 - P.omega);
  out[0] = m.n;
  for (int a = 0; a < 3; ++a) {
    out[1 + a] = m.u[a];
    out[5 + a] = m.q[a];
  }
  out[4] = m.T;
  out[8] = P.dt * nu;
  out[9] = 1.6 * (1.0 - P.Pr) / (m.n * m.T * m.T);
  out[10] = cbrt(m.n) / sqrt(kPi * m.T);
}

// Per-cell parameters of every cell, one thread per cell, and (macro != null) the
// macroparameters [nc][8] (n, u, T, q) of the current state
__global__ void tucker_cellpar_kernel(TuckerStepParams P, double *cellpar, double *macro) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= P.nc) return;
  double par[kCellPar];
  cell_params(P.sums + c * kSums, P, par);
  par[11] = 0.0;
  for (int k = 0; k < kCellPar; ++k) cellpar[c * kCellPar + k] = par[k];
  if (macro)
    for (int k = 0; k < 8; ++k) macro[c * 8 + k] = par[k];
}

// Per-cell prologue of the assembly: slots, wall-density scales, the cell's
// macroparameters (moments of f^n, Section 4 item 5) and the per-axis tables of
// the Maxwellian, Shakhov and face weights (zero-padded to padN(Nmax)).
template <typename Real>
__device__ void cell_prologue(const TuckerStepParams &P, int64_t c, const int N[3], Smem<Real> &sm,
                              SlotDev *s_slot, double *s_scale) {
  const int tid = threadIdx.x;
  const int Nm = P.Nmax;
  // ---- prologue: macroparameters, wall densities
  const double *S = P.sums + c * kSums;
  if (tid < 6) {
    s_slot[tid] = P.slot[c * 6 + tid];
    s_scale[tid] = (s_slot[tid].kind == kWall) ? -S[16 + tid] / s_slot[tid].wall_den : 1.0;
  }
  if (P.cellpar) {  // formed for all cells at the start of the step
    if (tid < 11) sm.par[tid] = P.cellpar[c * kCellPar + tid];
  } else if (tid == 0) {
    cell_params(S, P, sm.par);
  }
  __syncthreads();
  {
    const double T = sm.par[4], dtnu = sm.par[8], A = sm.par[9], amp = sm.par[10];
    const int NmP = padN(Nm);
    for (int a = 0; a < 3; ++a)
      for (int i = tid; i < NmP; i += blockDim.x) {
        if (i >= N[a]) {  // zero padding up to a multiple of kRows
          for (int t = a; t < 15; t += 3) tabp(sm, Nm, t)[i] = Real(0);
          continue;
        }
        if constexpr (sizeof(Real) == 8) {
          const double x = P.xi[a][i];
          const double v = x - sm.par[1 + a];
          tabp(sm, Nm, 0 + a)[i] = x;
          tabp(sm, Nm, 3 + a)[i] = (a == 0 ? dtnu : 1.0) * amp * exp(-v * v / T);
          tabp(sm, Nm, 6 + a)[i] = A * sm.par[5 + a] * v;
          tabp(sm, Nm, 9 + a)[i] = v * v / T;
          double g = 0.0;
          for (int l = 0; l < 6; ++l) {
            const SlotDev &sl = s_slot[l];
            if (sl.axis == a) g -= sl.c * fmax(sl.sgn * x, 0.0);
          }
          tabp(sm, Nm, 12 + a)[i] = g;
        } else {  // the tables are FP32: evaluate them in FP32
          const float x = (float)P.xi[a][i];
          const float v = x - (float)sm.par[1 + a];
          const float iT = 1.0f / (float)T;
          tabp(sm, Nm, 0 + a)[i] = x;
          tabp(sm, Nm, 3 + a)[i] = (float)(a == 0 ? dtnu * amp : amp) * expf(-v * v * iT);
          tabp(sm, Nm, 6 + a)[i] = (float)(A * sm.par[5 + a]) * v;
          tabp(sm, Nm, 9 + a)[i] = v * v * iT;
          float g = 0.0f;
          for (int l = 0; l < 6; ++l) {
            const SlotDev &sl = s_slot[l];
            if (sl.axis == a) g -= (float)sl.c * fmaxf((float)sl.sgn * x, 0.0f);
          }
          tabp(sm, Nm, 12 + a)[i] = g;
        }
      }
    for (int l = 0; l < 6; ++l) {
      const SlotDev &sl = s_slot[l];
      if (sl.axis < 0) continue;
      for (int i = tid; i < NmP; i += blockDim.x)
        tabp(sm, Nm, 15 + l)[i] =
            i < N[sl.axis]
                ? (Real)(-sl.c * fmin(sl.sgn * P.xi[sl.axis][i], 0.0) * s_scale[l])
                : Real(0);
    }
  }
  __syncthreads();
}

// minimum resident CTAs per SM the register allocation must allow
template <typename Real>
struct MinBlocks {
  static constexpr int value = sizeof(Real) == 8 ? 2 : 4;
};

template <typename Real, int TS>
__global__ void __launch_bounds__(kTB, MinBlocks<Real>::value) tucker_step_kernel(TuckerStepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<Real> sm = carve<Real>(smem_raw, P.Nmax, P.R);
  __shared__ SlotDev s_slot[6];
  __shared__ double s_scale[6];
  const int N[3] = {P.N1, P.N2, P.N3};
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3, NP = N2 * N3;
  const int NN = N1 * NP;
  const int tid = threadIdx.x;
  Real *X = reinterpret_cast<Real *>(P.scratch) + (size_t)blockIdx.x * P.scratch_stride;
  Real *T2buf = X + NN;  // assembly: mode-2/3 contractions; rounding: its work space
  Real *T2 = T2buf;
  Real *T1 = T2 + (size_t)P.R * NP;

  PhaseClock pc(P.phase);
  for (int64_t c = blockIdx.x; c < P.nc; c += gridDim.x) {
    if (P.mode == 1) {  // compress a given full tensor
      const double *src = P.finit + c * (int64_t)NN;
      for (int i = tid; i < NN; i += blockDim.x) X[i] = (Real)src[i];
      __syncthreads();
      round_hosvd<Real, TS>(X, T1, T2, N, P.R, P.tol, P.nxt, c, sm, P.err, pc, nullptr);
      continue;
    }
    cell_prologue<Real>(P, c, N, sm, s_slot, s_scale);
    pc.mark(0);
    // ---- f^{n+1} before rounding, in one pass
    assemble<Real>(P, c, N, sm, s_slot, s_scale, X, T2buf, nullptr, nullptr, pc);
    pc.mark(3);
    // ---- rounding
    round_hosvd<Real, TS>(X, T1, T2, N, P.R, P.tol, P.nxt, c, sm, P.err, pc, &P.cur);
  }
}

// ---------------------------------------------------------------------------
// Phase-major variant of the step (same arithmetic as tucker_step_kernel, cell
// for cell): each phase runs for a chunk of cells before the next starts, so
// the short dependent chains of the eigen-solves (one warp per cell) overlap
// across many cells instead of a few.
//   asm      persistent CTAs: prologue + assembly -> X (global), ||X||^2
//   gram(m)  one CTA per cell: Gram matrix of the mode-m unfolding -> C
//   eig(m)   one warp per cell: basis, rank rule -> new factor U_m, rank
//   proj(m)  one CTA per cell: X x_1 U1^T -> Y1, Y1 x_2 U2^T -> Y2,
//            Y2 x_3 U3^T -> core (FP64 accumulation)

constexpr int kAsmTB = 128;  // threads per CTA of the phase-major assembly kernel

// Shared memory of the assembly kernel: cell scalars, the core staging space
// (one first-mode slab of G and of its mode-3 contraction), tables, factor rows.
template <typename Real>
__host__ __device__ inline size_t smem_asm_bytes(int Nmax, int R) {
  const size_t stage = ((size_t)R * (R + Nmax) * sizeof(Real) + 15) / 16 * 2;  // doubles
  return sizeof(double) * (64 + stage) +
         sizeof(Real) * ((size_t)kTabs * padN(Nmax) + 3 * (size_t)Nmax * R +
                         (kTerms + 1) * (size_t)R * padN(Nmax)) +
         64;
}

template <typename Real>
__device__ Smem<Real> carve_asm(unsigned char *base, int Nmax, int R) {
  Smem<Real> s{};
  // doubles; even, so that the tables start on a 16-byte boundary
  const int stage = (int)(((size_t)R * (R + Nmax) * sizeof(Real) + 15) / 16) * 2;
  s.nmax = Nmax;
  s.par = reinterpret_cast<double *>(base);
  s.red = s.par + 32;
  s.C = s.red + 32;
  s.asm_space = stage;
  Real *r = reinterpret_cast<Real *>(s.C + stage);
  s.rt = r;
  r += (size_t)kTabs * padN(Nmax);
  for (int a = 0; a < 3; ++a) {
    s.fac[a] = r;
    r += (size_t)Nmax * R;
  }
  s.u1 = align16(r);
  return s;
}

template <typename Real>
__global__ void __launch_bounds__(kAsmTB, sizeof(Real) == 8 ? 4 : 6)
    tucker_asm_kernel(TuckerStepParams P, TuckerSplitBufs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<Real> sm = carve_asm<Real>(smem_raw, P.Nmax, P.R);
  __shared__ SlotDev s_slot[6];
  __shared__ double s_scale[6];
  const int N[3] = {P.N1, P.N2, P.N3};
  const int64_t NN = (int64_t)P.N1 * P.N2 * P.N3;
  Real *T2buf = reinterpret_cast<Real *>(B.t2) + (size_t)blockIdx.x * B.t2_stride;
  PhaseClock pc(P.phase);
  for (int64_t j = blockIdx.x; j < B.cn; j += gridDim.x) {
    const int64_t c = B.c0 + j, jb = B.joff + j;
    cell_prologue<Real>(P, c, N, sm, s_slot, s_scale);
    pc.mark(0);
    Real *X = reinterpret_cast<Real *>(B.X) + jb * NN;
    if (sizeof(Real) == 4 && B.rowmax)
      assemble<Real, sizeof(Real) == 4>(P, c, N, sm, s_slot, s_scale, X, T2buf,
                                        reinterpret_cast<const Real *>(B.T2all),
                                        reinterpret_cast<const Real *>(B.U1all), pc,
                                        B.rowmax + jb * P.Nmax);
    else
      assemble<Real>(P, c, N, sm, s_slot, s_scale, X, T2buf,
                     reinterpret_cast<const Real *>(B.T2all),
                     reinterpret_cast<const Real *>(B.U1all), pc);
    pc.mark(3);
    if (threadIdx.x == 0) B.disc[jb] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Assembly of f^{n+1} in GEMM form (mixed path; meshes whose faces all lie on coordinate
// planes).  Every term of
//   X = dt nu f^S + sum_ghosts m_l g_l + W_self o f + sum_faces m_l o f_src(l)
// factors into (a vector over the first-mode index i1) x (a vector over the columns
// p = (i2, i3)), because every face weight then depends on one velocity coordinate:
// the self term (Lemma 1) is (w0 + G0(i1) + zero-gradient inflows along axis 0) U1 T2 +
// U1 (T2 o (G1(i2) + G2(i3) + zero-gradient inflows along axes 1, 2)); a face term is
// (m_l(i1) U1_src) T2_src or U1_src (T2_src o m_l(i2 or i3)) (a symmetry face: the
// cell's own tensor with one index mirrored); the Shakhov term (Proposition 1: f^M
// times a cubic polynomial) is four rank-one products; a ghost is one.  Hence
// X = A B^T with A [N1 x K] the row factors and B [NP x K] the column factors, K <=
// 4 + 8 R the cell's number of rank-one terms: one small GEMM per cell, its K-term sums
// in FP32 FMAs.  One CTA per cell: A in shared memory, then per tile of 256 columns the
// column factors staged 32 terms at a time (every thread one column, its gathers all
// issued before any is used) and a register tile of N1P / 4 rows x 4 columns per thread,
// A read as broadcast float4 and B as one float4 per term.  X is written once, column-
// coalesced, and each first-mode row's largest magnitude kept (the tensor-core Gram
// matrix's row scales).
constexpr int kAgThreads = 256;
constexpr int kAgCols = 256;  // columns of X per tile: 64 groups of four
constexpr int kAgKC = 32;     // terms per staged chunk of B

struct AgTerm {
  int64_t t2;  // Tucker terms: T2 row offset (elements), cell * R * NP + k * NP
  int64_t u1;  // Tucker terms: U1 row offset (elements), cell * R * padN(N1) + k * padN(N1)
  int kind;    // 0 Tucker term, 1-4 Shakhov parts, 5 ghost of face `face`
  int refl;    // 1 / 2: second / third-mode index mirrored
  int wsel;    // column weight: 0 none, 1 self (G1(i2) + G2(i3)), 2 face tab over i2, 3 over i3
  int face;
  int wa;      // row weight: 0 none, 1 self (w0 + G0(i1)), 2 face tab over i1
  int rev;     // first-mode index mirrored
};

__host__ __device__ inline int ag_max_terms(int R) { return 4 + 8 * R; }

// shared memory: cell scalars and tables, self weights, A [K][padN(N1)], the staged column
// factors B [kAgKC][kAgCols], term list, row maxima
__host__ __device__ inline size_t ag_smem_bytes(int Nmax, int N1, int R, int nbuf = 1) {
  const size_t NmP = padN(Nmax), K4 = (size_t)((ag_max_terms(R) + 3) & ~3);
  return sizeof(double) * 96 + sizeof(float) * ((size_t)kTabs * NmP + 3 * NmP) +
         sizeof(float) * K4 * padN(N1) + sizeof(float) * kAgKC * kAgCols * nbuf +
         sizeof(AgTerm) * K4 + sizeof(unsigned) * NmP + 64;
}

// B stages: two (the next unit's column factors copied in while the current one's FMAs
// run) where the four-column staging applies (N3 a multiple of four, tiles of at most 12
// rows) and two CTAs per SM still fit, else one
__host__ __device__ inline int ag_nbuf(int Nmax, int N1, int N3, int R) {
  return (padN(N1) <= 48 && (N3 & 3) == 0 &&
          2 * (ag_smem_bytes(Nmax, N1, R, 2) + 1024) <= 228 * 1024)
             ? 2
             : 1;
}

__device__ __forceinline__ void cp_async16(float *smem_dst, const float *gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// the column factor at (i2, i3) of a computed term: a Shakhov part (Proposition 1: the
// Maxwellian's (i2, i3) factor times 1, Vp, Qp or Qp Vp) or a ghost (its (i2, i3) factors,
// weighed by the face's inflow table when the face normal is axis 1 or 2)
__device__ __forceinline__ float ag_column(const AgTerm &tm, Smem<float> &sm, const SlotDev *s_slot,
                                           const float *ghostR, int Nm, int i2, int i3) {
  if (tm.kind == 5) {
    const SlotDev &sl = s_slot[tm.face];
    const float *gf = ghostR + (int64_t)sl.src * 3 * Nm;
    float x = gf[Nm + i2] * gf[2 * Nm + i3];
    if (sl.axis == 1) x *= tabp(sm, Nm, 15 + tm.face)[i2];
    else if (sl.axis == 2) x *= tabp(sm, Nm, 15 + tm.face)[i3];
    return x;
  }
  const float fM = tabp(sm, Nm, 4)[i2] * tabp(sm, Nm, 5)[i3];
  const float Qp = tabp(sm, Nm, 7)[i2] + tabp(sm, Nm, 8)[i3];
  const float Vp = tabp(sm, Nm, 10)[i2] + tabp(sm, Nm, 11)[i3] - 2.5f;
  return tm.kind == 1 ? fM : (tm.kind == 2 ? fM * Vp : (tm.kind == 3 ? fM * Qp : fM * Qp * Vp));
}

// X of one cell: thread (rg, cg) = (tid / 64, tid % 64) holds rows rg TR .. rg TR + TR - 1
// and columns 4 cg .. 4 cg + 3 of each 256-column tile (TR = padN(N1) / 4)
template <int TR>
__device__ __forceinline__ void ag_columns(const TuckerStepParams &P, const TuckerSplitBufs &B,
                                           int64_t jb, Smem<float> &sm, const SlotDev *s_slot,
                                           const float *A_s, float *B_s, const AgTerm *terms,
                                           int K, const float *colW2, const float *colW3,
                                           unsigned *s_rmax) {
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3, NP = N2 * N3, Nm = P.Nmax, N1P = padN(N1);
  const int tid = threadIdx.x, lane = tid & 31;
  const int rg = tid >> 6, cg = tid & 63, row0 = rg * TR;
  const float *T2all = reinterpret_cast<const float *>(B.T2all);
  const float *ghostR = P.ghostf32;
  float *Xc = reinterpret_cast<float *>(B.X) + jb * (int64_t)N1 * NP;
  // vector staging: four columns of one i2 row per thread (16-row tiles keep the scalar
  // staging, for registers)
  const bool vec = (NP & 3) == 0, vec4 = TR <= 12 && (N3 & 3) == 0;
  float rm[TR];
#pragma unroll
  for (int r = 0; r < TR; ++r) rm[r] = 0.f;
  for (int c0 = 0; c0 < NP; c0 += kAgCols) {
    float acc[TR][4];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kAgKC) {
      const int kn = min(kAgKC, K - k0), kn4 = (kn + 3) & ~3;
      if (vec4) {
        // N3 a multiple of four: thread (ts, cq) stages columns c0 + 4 cq .. + 3 (one i2
        // row) of terms ts, ts + 4, ..., ts + 28 of the chunk (dealt round robin, so the
        // four groups share a short chunk evenly): one float4 gather, weighing and store
        // per term, the gathers of a batch issued before any is used
        const int ts = tid >> 6, cq = tid & 63;
        const int p = c0 + 4 * cq;
        const bool pin = p < NP;  // all four columns or none (NP a multiple of four)
        const int pc = pin ? p : 0, i2 = pc / N3, i3 = pc - i2 * N3;
        const int pm2 = (N2 - 1 - i2) * N3 + i3, pm3 = i2 * N3 + (N3 - 4 - i3);
        constexpr int VG = TR >= 12 ? 4 : 8;  // gathers in flight (registers: the tile is live)
#pragma unroll
        for (int e0 = 0; e0 < 8; e0 += VG) {
          if (ts + 4 * e0 >= kn4) break;  // warp-uniform
          float4 g[VG];
#pragma unroll
          for (int e = 0; e < VG; ++e) {
            const int kk = ts + 4 * (e0 + e);
            g[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kk < kn && pin && terms[k0 + kk].kind == 0) {
              const int refl = terms[k0 + kk].refl;
              g[e] = __ldg(reinterpret_cast<const float4 *>(
                  T2all + terms[k0 + kk].t2 + (refl == 1 ? pm2 : (refl == 2 ? pm3 : pc))));
            }
          }
#pragma unroll
          for (int e = 0; e < VG; ++e) {
            const int kk = ts + 4 * (e0 + e);
            if (kk >= kn4) break;  // warp-uniform
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kk < kn && pin) {
              const AgTerm tm = terms[k0 + kk];
              if (tm.kind == 0) {
                x = tm.refl == 2 ? make_float4(g[e].w, g[e].z, g[e].y, g[e].x) : g[e];
                if (tm.wsel == 1) {
                  const float w2 = colW2[i2];
                  const float4 w3 = *reinterpret_cast<const float4 *>(colW3 + i3);
                  x = make_float4(x.x * (w2 + w3.x), x.y * (w2 + w3.y), x.z * (w2 + w3.z),
                                  x.w * (w2 + w3.w));
                } else if (tm.wsel == 2) {
                  const float w = tabp(sm, Nm, 15 + tm.face)[i2];
                  x = make_float4(x.x * w, x.y * w, x.z * w, x.w * w);
                } else if (tm.wsel == 3) {
                  const float4 w = *reinterpret_cast<const float4 *>(tabp(sm, Nm, 15 + tm.face) + i3);
                  x = make_float4(x.x * w.x, x.y * w.y, x.z * w.z, x.w * w.w);
                }
              } else {
                x = make_float4(ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3),
                                ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3 + 1),
                                ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3 + 2),
                                ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3 + 3));
              }
            }
            *reinterpret_cast<float4 *>(B_s + kk * kAgCols + 4 * cq) = x;
          }
        }
      } else {  // stage B[c0 + tid][k0 .. k0 + kn4): this thread's column, SH terms at a time
        constexpr int SH = TR > 12 ? 8 : 16;  // gathers in flight (registers: the tile is live)
        const int p = c0 + tid;
        const bool pin = p < NP;
        const int pc = pin ? p : 0, i2 = pc / N3, i3 = pc - i2 * N3;
        const int pm2 = (N2 - 1 - i2) * N3 + i3, pm3 = i2 * N3 + (N3 - 1 - i3);
#pragma unroll
        for (int h = 0; h < kAgKC; h += SH) {
          if (h >= kn4) break;  // uniform
          float g[SH];
#pragma unroll
          for (int e = 0; e < SH; ++e) {
            g[e] = 0.f;
            if (h + e < kn && pin && terms[k0 + h + e].kind == 0) {
              const int refl = terms[k0 + h + e].refl;
              g[e] = __ldg(T2all + terms[k0 + h + e].t2 + (refl == 1 ? pm2 : (refl == 2 ? pm3 : pc)));
            }
          }
#pragma unroll
          for (int e = 0; e < SH; ++e) {
            if (h + e >= kn4) break;  // uniform
            float x = 0.f;
            if (h + e < kn && pin) {
              const AgTerm tm = terms[k0 + h + e];
              if (tm.kind == 0) {
                x = g[e];
                if (tm.wsel == 1) x *= colW2[i2] + colW3[i3];
                else if (tm.wsel == 2) x *= tabp(sm, Nm, 15 + tm.face)[i2];
                else if (tm.wsel == 3) x *= tabp(sm, Nm, 15 + tm.face)[i3];
              } else {
                x = ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3);
              }
            }
            B_s[(h + e) * kAgCols + tid] = x;
          }
        }
      }
      __syncthreads();
      const float *a = A_s + (size_t)k0 * N1P + row0;
      const float *bp = B_s + 4 * cg;
#pragma unroll(TR > 12 ? 1 : 4)
      for (int e = 0; e < kn4; ++e) {
        float av[TR];
#pragma unroll
        for (int q = 0; q < TR / 4; ++q) {
          const float4 t = *reinterpret_cast<const float4 *>(a + (size_t)e * N1P + 4 * q);
          av[4 * q] = t.x;
          av[4 * q + 1] = t.y;
          av[4 * q + 2] = t.z;
          av[4 * q + 3] = t.w;
        }
        const float4 bv = *reinterpret_cast<const float4 *>(bp + e * kAgCols);
#pragma unroll
        for (int r = 0; r < TR; ++r) {
          acc[r][0] = fmaf(av[r], bv.x, acc[r][0]);
          acc[r][1] = fmaf(av[r], bv.y, acc[r][1]);
          acc[r][2] = fmaf(av[r], bv.z, acc[r][2]);
          acc[r][3] = fmaf(av[r], bv.w, acc[r][3]);
        }
      }
      __syncthreads();  // B_s is restaged next
    }
    // the tile of X (streamed past L2) and the row maxima
    const int cb = c0 + 4 * cg;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      const int row = row0 + r;
      if (row >= N1 || cb >= NP) continue;
      float *dst = Xc + (int64_t)row * NP + cb;
      if (vec) {  // NP a multiple of 4: the four columns are in range and 16-byte aligned
        __stcs(reinterpret_cast<float4 *>(dst), make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
        rm[r] = fmaxf(rm[r], fmaxf(fmaxf(fabsf(acc[r][0]), fabsf(acc[r][1])),
                                   fmaxf(fabsf(acc[r][2]), fabsf(acc[r][3]))));
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (cb + q < NP) {
            __stcs(dst + q, acc[r][q]);
            rm[r] = fmaxf(rm[r], fabsf(acc[r][q]));
          }
      }
    }
  }
  if (B.rowmax) {  // across the warp's 32 column groups (its rows are the same), then warps
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      float m = rm[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0 && row0 + r < N1) atomicMax(&s_rmax[row0 + r], __float_as_uint(m));
    }
  }
}

// ag_columns with two B stages (N3 a multiple of four, TR <= 12): the units (tile, chunk
// of 32 terms) run in order; the Tucker columns of unit u + 1 are copied from T2 straight
// into the other stage (16-byte asynchronous copies, thread (ts, cq) its four columns of
// terms ts, ts + 4, ...) while unit u's FMAs run, and each thread then weighs its own
// entries in place (the computed columns and the zero padding written there too): one
// barrier per unit.  The same sums as ag_columns.
template <int TR>
__device__ __forceinline__ void ag_columns_pipe(const TuckerStepParams &P, const TuckerSplitBufs &B,
                                                int64_t jb, Smem<float> &sm, const SlotDev *s_slot,
                                                const float *A_s, float *B_s, const AgTerm *terms,
                                                int K, const float *colW2, const float *colW3,
                                                unsigned *s_rmax) {
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3, NP = N2 * N3, Nm = P.Nmax, N1P = padN(N1);
  const int tid = threadIdx.x, lane = tid & 31;
  const int rg = tid >> 6, cg = tid & 63, row0 = rg * TR;
  const int ts = tid >> 6, cq = tid & 63;
  const float *T2all = reinterpret_cast<const float *>(B.T2all);
  const float *ghostR = P.ghostf32;
  float *Xc = reinterpret_cast<float *>(B.X) + jb * (int64_t)N1 * NP;
  const int nchunk = (K + kAgKC - 1) / kAgKC, ntile = (NP + kAgCols - 1) / kAgCols;
  const int nunit = nchunk * ntile;
  constexpr int kStage = kAgKC * kAgCols;
  // copies of unit u's Tucker columns into stage u & 1 (one commit group per unit)
  auto issue = [&](int u) {
    const int tile = u / nchunk, k0 = (u - tile * nchunk) * kAgKC, kn = min(kAgKC, K - k0);
    const int p = tile * kAgCols + 4 * cq;
    if (p < NP) {
      const int i2 = p / N3, i3 = p - i2 * N3;
      const int pm2 = (N2 - 1 - i2) * N3 + i3, pm3 = i2 * N3 + (N3 - 4 - i3);
      float *buf = B_s + (u & 1) * kStage + 4 * cq;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int kk = ts + 4 * e;
        if (kk >= kn) break;  // warp-uniform
        const AgTerm &tm = terms[k0 + kk];
        if (tm.kind == 0)
          cp_async16(buf + kk * kAgCols, T2all + tm.t2 + (tm.refl == 1 ? pm2 : (tm.refl == 2 ? pm3 : p)));
      }
    }
    cp_async_commit();
  };
  float rm[TR];
#pragma unroll
  for (int r = 0; r < TR; ++r) rm[r] = 0.f;
  float acc[TR][4];
  if (nunit > 0) issue(0);
  for (int u = 0; u < nunit; ++u) {
    const int tile = u / nchunk, ch = u - tile * nchunk, k0 = ch * kAgKC;
    const int kn = min(kAgKC, K - k0), kn4 = (kn + 3) & ~3, c0 = tile * kAgCols;
    float *buf = B_s + (u & 1) * kStage;
    cp_async_wait_all();  // this thread's copies of unit u have landed
    {  // weigh this thread's entries of unit u in place
      const int p = c0 + 4 * cq;
      const bool pin = p < NP;
      const int pc = pin ? p : 0, i2 = pc / N3, i3 = pc - i2 * N3;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int kk = ts + 4 * e;
        if (kk >= kn4) break;  // warp-uniform
        float4 *dst = reinterpret_cast<float4 *>(buf + kk * kAgCols + 4 * cq);
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kk < kn && pin) {
          const AgTerm tm = terms[k0 + kk];
          if (tm.kind == 0) {
            x = *dst;
            if (tm.refl == 2) x = make_float4(x.w, x.z, x.y, x.x);
            if (tm.wsel == 1) {
              const float w2 = colW2[i2];
              const float4 w3 = *reinterpret_cast<const float4 *>(colW3 + i3);
              x = make_float4(x.x * (w2 + w3.x), x.y * (w2 + w3.y), x.z * (w2 + w3.z), x.w * (w2 + w3.w));
            } else if (tm.wsel == 2) {
              const float w = tabp(sm, Nm, 15 + tm.face)[i2];
              x = make_float4(x.x * w, x.y * w, x.z * w, x.w * w);
            } else if (tm.wsel == 3) {
              const float4 w = *reinterpret_cast<const float4 *>(tabp(sm, Nm, 15 + tm.face) + i3);
              x = make_float4(x.x * w.x, x.y * w.y, x.z * w.z, x.w * w.w);
            }
          } else {
            x = make_float4(ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3),
                            ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3 + 1),
                            ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3 + 2),
                            ag_column(tm, sm, s_slot, ghostR, Nm, i2, i3 + 3));
          }
        }
        *dst = x;
      }
    }
    __syncthreads();  // unit u staged; every thread is past unit u - 1's FMAs
    if (u + 1 < nunit) issue(u + 1);
    if (ch == 0) {
#pragma unroll
      for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
    }
    const float *a = A_s + (size_t)k0 * N1P + row0;
    const float *bp = buf + 4 * cg;
#pragma unroll 4
    for (int e = 0; e < kn4; ++e) {
      float av[TR];
#pragma unroll
      for (int q = 0; q < TR / 4; ++q) {
        const float4 t = *reinterpret_cast<const float4 *>(a + (size_t)e * N1P + 4 * q);
        av[4 * q] = t.x;
        av[4 * q + 1] = t.y;
        av[4 * q + 2] = t.z;
        av[4 * q + 3] = t.w;
      }
      const float4 bv = *reinterpret_cast<const float4 *>(bp + e * kAgCols);
#pragma unroll
      for (int r = 0; r < TR; ++r) {
        acc[r][0] = fmaf(av[r], bv.x, acc[r][0]);
        acc[r][1] = fmaf(av[r], bv.y, acc[r][1]);
        acc[r][2] = fmaf(av[r], bv.z, acc[r][2]);
        acc[r][3] = fmaf(av[r], bv.w, acc[r][3]);
      }
    }
    if (ch + 1 == nchunk) {  // the tile of X (NP a multiple of four) and the row maxima
      const int cb = c0 + 4 * cg;
      if (cb < NP) {
#pragma unroll
        for (int r = 0; r < TR; ++r) {
          const int row = row0 + r;
          if (row >= N1) continue;
          __stcs(reinterpret_cast<float4 *>(Xc + (int64_t)row * NP + cb),
                 make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
          rm[r] = fmaxf(rm[r], fmaxf(fmaxf(fabsf(acc[r][0]), fabsf(acc[r][1])),
                                     fmaxf(fabsf(acc[r][2]), fabsf(acc[r][3]))));
        }
      }
    }
  }
  if (B.rowmax) {  // across the warp's 32 column groups (its rows are the same), then warps
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      float m = rm[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0 && row0 + r < N1) atomicMax(&s_rmax[row0 + r], __float_as_uint(m));
    }
  }
}

// TR rows of X per thread (padN(N1) / 4), kPipe: two B stages (ag_nbuf = 2)
template <int TR, bool kPipe>
__global__ void __launch_bounds__(kAgThreads, 2)
    tucker_asm_gemm_kernel(TuckerStepParams P, TuckerSplitBufs B) {
  extern __shared__ __align__(16) unsigned char ag_raw[];
  const int Nm = P.Nmax, N1 = P.N1, N2 = P.N2, N3 = P.N3, NmP = padN(Nm), NP = N2 * N3;
  const int N1P = padN(N1), R = P.R, Kmax = ag_max_terms(R), K4max = (Kmax + 3) & ~3;
  const int N[3] = {N1, N2, N3};
  Smem<float> sm{};
  sm.nmax = Nm;
  sm.par = reinterpret_cast<double *>(ag_raw);
  sm.red = sm.par + 32;
  sm.rt = reinterpret_cast<float *>(sm.par + 96);
  float *rowW = sm.rt + (size_t)kTabs * NmP;        // self weight over i1
  float *colW2 = rowW + NmP, *colW3 = colW2 + NmP;  // self weight parts over i2, i3
  float *A_s = colW3 + NmP;                         // [K][N1P]
  float *B_s = A_s + (size_t)K4max * N1P;           // [1 or 2][kAgKC][kAgCols]
  AgTerm *terms = reinterpret_cast<AgTerm *>(B_s + (kPipe ? 2 : 1) * kAgKC * kAgCols);
  unsigned *s_rmax = reinterpret_cast<unsigned *>(terms + K4max);
  __shared__ SlotDev s_slot[6];
  __shared__ double s_scale[6];
  __shared__ int s_K, s_rk[7];
  const float *U1all = reinterpret_cast<const float *>(B.U1all);
  const float *ghostR = P.ghostf32;
  const int tid = threadIdx.x;
  for (int64_t j = blockIdx.x; j < B.cn; j += gridDim.x) {
    const int64_t c = B.c0 + j, jb = B.joff + j;
    cell_prologue<float>(P, c, N, sm, s_slot, s_scale);
    // first-mode ranks of the cell and of each face's source, loaded side by side
    if (tid < 7) {
      const SlotDev *sl = tid > 0 ? &s_slot[tid - 1] : nullptr;
      s_rk[tid] = P.cur.rank[3 * ((sl && sl->kind == kInterior) ? (int64_t)sl->src : c)];
    }
    __syncthreads();
    // the cell's rank-one terms: Shakhov parts, ghosts, self (row weight), self (column
    // weight), then each interior / symmetry face
    if (tid == 0) {
      int n = 0;
      auto put = [&](const AgTerm &tm) {
        if (n < Kmax) terms[n] = tm;
        ++n;
      };
      for (int k = 1; k <= 4; ++k) put(AgTerm{0, 0, k, 0, 0, 0, 0, 0});
      for (int l = 0; l < 6; ++l)
        if (s_slot[l].kind == kFreeStream || s_slot[l].kind == kWall) put(AgTerm{0, 0, 5, 0, 0, l, 0, 0});
      const int r = s_rk[0];
      const int64_t oT = c * (int64_t)R * NP, oU = c * (int64_t)R * N1P;
      for (int k = 0; k < r; ++k) put(AgTerm{oT + (int64_t)k * NP, oU + (int64_t)k * N1P, 0, 0, 0, -1, 1, 0});
      for (int k = 0; k < r; ++k) put(AgTerm{oT + (int64_t)k * NP, oU + (int64_t)k * N1P, 0, 0, 1, -1, 0, 0});
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        if (sl.kind != kInterior && sl.kind != kSymmetry) continue;
        const bool sym = sl.kind == kSymmetry;
        const int64_t src = sym ? c : (int64_t)sl.src;
        const int rs = s_rk[l + 1];
        const int wa = sl.axis == 0 ? 2 : 0, ws = sl.axis == 1 ? 2 : (sl.axis == 2 ? 3 : 0);
        const int rev = sym && sl.flip == 0, refl = sym ? (sl.flip == 1 ? 1 : (sl.flip == 2 ? 2 : 0)) : 0;
        const int64_t sT = src * (int64_t)R * NP, sU = src * (int64_t)R * N1P;
        for (int k = 0; k < rs; ++k)
          put(AgTerm{sT + (int64_t)k * NP, sU + (int64_t)k * N1P, 0, refl, ws, l, wa, rev});
      }
      s_K = n;
    }
    // self weights (Lemma 1): w0 + G0(i1) | G1(i2) | G2(i3), plus zero-gradient inflows
    {
      const float w0 = (float)(1.0 - sm.par[8]);
      for (int i = tid; i < NmP; i += blockDim.x) {
        float a = i < N1 ? w0 + tabp(sm, Nm, 12)[i] : 0.f;
        float b2 = i < N2 ? tabp(sm, Nm, 13)[i] : 0.f, b3 = i < N3 ? tabp(sm, Nm, 14)[i] : 0.f;
        for (int l = 0; l < 6; ++l) {
          if (s_slot[l].kind != kZeroGrad) continue;
          const float *tab = tabp(sm, Nm, 15 + l);
          if (s_slot[l].axis == 0 && i < N1) a += tab[i];
          if (s_slot[l].axis == 1 && i < N2) b2 += tab[i];
          if (s_slot[l].axis == 2 && i < N3) b3 += tab[i];
        }
        rowW[i] = a;
        colW2[i] = b2;
        colW3[i] = b3;
        s_rmax[i] = 0u;
      }
    }
    __syncthreads();
    const int K = s_K;
    if (K > Kmax) {  // more terms than 4 + 8 R: a rank above the cap (state corrupt)
      if (tid == 0) atomicOr(P.flag, 2);
      break;
    }
    // A: the row factors, [term][row], zero past N1 and up to a multiple of four terms
    const int K4 = (K + 3) & ~3;
    for (int idx = tid; idx < K4 * N1P; idx += blockDim.x) {
      const int k = idx / N1P, row = idx - k * N1P;
      float x = 0.f;
      if (k < K && row < N1) {
        const AgTerm tm = terms[k];
        if (tm.kind == 0) {
          x = U1all[tm.u1 + (tm.rev ? N1 - 1 - row : row)];
          if (tm.wa == 1) x *= rowW[row];
          else if (tm.wa == 2) x *= tabp(sm, Nm, 15 + tm.face)[row];
        } else if (tm.kind == 5) {
          const SlotDev &sl = s_slot[tm.face];
          x = ghostR[(int64_t)sl.src * 3 * Nm + row];
          if (sl.axis == 0) x *= tabp(sm, Nm, 15 + tm.face)[row];
        } else {
          const float f0 = tabp(sm, Nm, 3)[row], q0 = tabp(sm, Nm, 6)[row], v0 = tabp(sm, Nm, 9)[row];
          x = tm.kind == 1 ? f0 * (1.f + q0 * v0) : (tm.kind == 2 ? f0 * q0 : (tm.kind == 3 ? f0 * v0 : f0));
        }
      }
      A_s[idx] = x;
    }
    __syncthreads();
    if constexpr (kPipe)
      ag_columns_pipe<TR>(P, B, jb, sm, s_slot, A_s, B_s, terms, K, colW2, colW3, s_rmax);
    else
      ag_columns<TR>(P, B, jb, sm, s_slot, A_s, B_s, terms, K, colW2, colW3, s_rmax);
    __syncthreads();
    if (B.rowmax)
      for (int i = tid; i < N1; i += blockDim.x) B.rowmax[jb * Nm + i] = __uint_as_float(s_rmax[i]);
    if (tid == 0) B.disc[jb] = 0.0;
  }
}

// the GEMM-form assembly kernel for a first mode padded to N1P rows and 1 or 2 B stages
using AgKernel = void (*)(TuckerStepParams, TuckerSplitBufs);
inline AgKernel ag_kernel(int N1P, int nbuf) {
  if (nbuf == 2) {
    if (N1P == 16) return tucker_asm_gemm_kernel<4, true>;
    if (N1P == 32) return tucker_asm_gemm_kernel<8, true>;
    return tucker_asm_gemm_kernel<12, true>;
  }
  if (N1P == 16) return tucker_asm_gemm_kernel<4, false>;
  if (N1P == 32) return tucker_asm_gemm_kernel<8, false>;
  if (N1P == 48) return tucker_asm_gemm_kernel<12, false>;
  return tucker_asm_gemm_kernel<16, false>;
}

// Mode-2/3 contraction T2 = G x2 U2 x3 U3 of every cell's current tensor and its
// first-mode factor in the working precision (transposed, zero-padded), once per
// step for all cells (each is used by the cell and its face neighbours).
template <typename Real>
__global__ void __launch_bounds__(kAsmTB) tucker_t2_kernel(TuckerStepParams P, TuckerSplitBufs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<Real> sm = carve_asm<Real>(smem_raw, P.Nmax, P.R);
  const int N[3] = {P.N1, P.N2, P.N3};
  const int NP = P.N2 * P.N3, R = P.R, N1P = padN(P.N1);
  __shared__ int s_r1;
  for (int64_t c = blockIdx.x; c < P.nc; c += gridDim.x) {
    term_contract<Real>(P.cur, c, N, R, NP, sm,
                        reinterpret_cast<Real *>(B.U1all) + c * (int64_t)R * N1P,
                        reinterpret_cast<Real *>(B.T2all) + c * (int64_t)R * NP, &s_r1);
  }
}

// dims of the tensor whose mode-m unfolding the Gram / projection of mode m use
__device__ __forceinline__ void split_dims(const TuckerSplitBufs &B, const TuckerDev &nxt,
                                           int64_t c, int m, const int N[3], int D[3]) {
  D[0] = m >= 1 ? nxt.rank[3 * c] : N[0];
  D[1] = m >= 2 ? nxt.rank[3 * c + 1] : N[1];
  D[2] = N[2];
}

template <typename Real>
__device__ __forceinline__ const Real *split_src(const TuckerSplitBufs &B, int64_t j, int m, int R,
                                                 const int N[3]) {
  if (m == 0) return reinterpret_cast<const Real *>(B.X) + j * (int64_t)N[0] * N[1] * N[2];
  if (m == 1) return reinterpret_cast<const Real *>(B.Y1) + j * (int64_t)R * N[1] * N[2];
  return reinterpret_cast<const Real *>(B.Y2) + j * (int64_t)R * R * N[2];
}

// Gram matrix of the mode-m unfolding of cell j's tensor, into B.C[j] (n x n)
template <typename Real, int TS>
__global__ void __launch_bounds__(kTB) tucker_gram_kernel(TuckerStepParams P, TuckerSplitBufs B,
                                                          int m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nm = P.Nmax;
  Smem<Real> sm{};
  sm.par = reinterpret_cast<double *>(smem_raw);
  sm.red = sm.par + 32;
  sm.C = sm.red + 32;
  sm.tile = reinterpret_cast<Real *>(sm.C + (size_t)Nm * Nm);
  sm.tile2 = sm.tile + (size_t)(Nm > 32 ? Nm : 32) * kTileRow;
  sm.cidx = reinterpret_cast<int *>(sm.tile2 + (size_t)(Nm > 32 ? Nm : 32) * kTileRow);
  sm.cidx_cap = 4 * kTB;
  const int N[3] = {P.N1, P.N2, P.N3};
  const int64_t j = blockIdx.x, c = B.c0 + j, jb = B.joff + j;
  int D[3];
  split_dims(B, P.nxt, c, m, N, D);
  gram<Real, TS>(split_src<Real>(B, jb, m, P.R, N), D, m, sm,
                 m == 0 ? gram_skip_rel(P.tol, D[1] * D[2]) : 0.0);
  if (m == 0 && threadIdx.x == 0) B.disc[jb] = sm.par[26];  // columns left out
  const int n = D[m];
  double *out = B.C + jb * (int64_t)Nm * Nm;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) out[i] = sm.C[i];
}

// Gram matrix of mode m >= 1 (second / third) of cell j's tensor when N_m <= 32, into
// B.C[j] (gram_seq: few registers, so many blocks per SM)
template <typename Real>
__global__ void __launch_bounds__(kTB, 4) tucker_gram_small_kernel(TuckerStepParams P,
                                                                    TuckerSplitBufs B, int m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nm = P.Nmax;
  Smem<Real> sm{};
  sm.par = reinterpret_cast<double *>(smem_raw);
  sm.red = sm.par + 32;
  sm.C = sm.red + 32;
  sm.tile = reinterpret_cast<Real *>(sm.C + (size_t)Nm * Nm);
  const int N[3] = {P.N1, P.N2, P.N3};
  const int64_t j = blockIdx.x, c = B.c0 + j, jb = B.joff + j;
  int D[3];
  split_dims(B, P.nxt, c, m, N, D);
  gram_seq<Real>(split_src<Real>(B, jb, m, P.R, N), D, m, sm);
  const int n = D[m];
  double *out = B.C + jb * (int64_t)Nm * Nm;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) out[i] = sm.C[i];
}

template <typename Real>
__host__ __device__ inline size_t smem_eig_bytes(int Nmax, int R) {
  const int K = sub_k(Nmax, R);
  size_t b = sizeof(double) * (64 + 2 * (size_t)Nmax * K + (size_t)K * K + 2 * K + 2);
  if (sizeof(Real) == 8) b += sizeof(Real) * (size_t)Nmax * K;  // the retry start (FP64 path)
  b += 16 + sizeof(int) * (2 * (size_t)K + 2);
  return b + 64;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

constexpr int kBulkWaitIters = 1 << 22;  // bound on the polls of a bulk copy's barrier

// One global -> shared copy of `bytes` bytes (a multiple of 8) for stage_to_shared
struct StagePiece {
  void *dst;
  const void *src;
  unsigned bytes;
};

__device__ __forceinline__ bool bulk_ok(const StagePiece &q) {
  return q.bytes > 0 && (q.bytes & 15u) == 0 &&
         ((reinterpret_cast<uintptr_t>(q.src) | reinterpret_cast<uintptr_t>(q.dst)) & 15) == 0;
}

__device__ __forceinline__ void plain_copy(const StagePiece &q) {
  double *d = static_cast<double *>(q.dst);
  const double *v = static_cast<const double *>(q.src);
  for (int i = threadIdx.x; i < (int)(q.bytes >> 3); i += blockDim.x) d[i] = v[i];
}

// Copy np pieces from global to shared memory.  Pieces whose addresses and size
// are multiples of 16 bytes go by bulk asynchronous copies (cp.async.bulk; thread 0
// issues them, completion is counted in bytes on one mbarrier, which every thread
// polls at most kBulkWaitIters times); the others, meanwhile, by plain loads of
// the block.  Returns true (in every thread) when all pieces are in place.  If the
// barrier has not completed within the limit, bit 1 of *flag is set, the block
// polls once more (again bounded) so that it does not give up shared memory with a
// copy still landing in it, and false is returned: the caller then returns at
// once, writes nothing, and the host reports the step as failed (DVM_ERR_TIMEOUT,
// the state undefined).  Called by every thread; ends with a barrier.
__device__ __forceinline__ unsigned poll_bulk(unsigned bar) {
  unsigned done = 0;
  for (int it = 0; it < kBulkWaitIters && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar)
        : "memory");
  return done;
}

template <int NP>
__device__ __noinline__ bool stage_to_shared(const StagePiece (&pc)[NP], int np, int *flag) {
  __shared__ __align__(8) unsigned long long s_bar;
  unsigned tx = 0;
  for (int q = 0; q < np; ++q)
    if (bulk_ok(pc[q])) tx += pc[q].bytes;
  const unsigned bar = smem_u32(&s_bar);
  if (tx > 0) {
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx)
                   : "memory");
      for (int q = 0; q < np; ++q)
        if (bulk_ok(pc[q]))
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
              "[%3];" ::"r"(smem_u32(pc[q].dst)),
              "l"(pc[q].src), "r"(pc[q].bytes), "r"(bar)
              : "memory");
    }
  }
  for (int q = 0; q < np; ++q)
    if (!bulk_ok(pc[q])) plain_copy(pc[q]);
  if (tx > 0 && !__syncthreads_and(poll_bulk(bar))) {
    if (threadIdx.x == 0) atomicOr(flag, 2);
    poll_bulk(bar);  // drain (bounded) before the block leaves
    __syncthreads();
    return false;
  }
  __syncthreads();
  return true;
}

// Eigen-solve and rank rule of mode m for cell j: one CTA per cell.  On exit
// nxt.fac[m] holds the kept orthonormal columns, nxt.rank the new rank; the
// energy left out accumulates in B.disc (the relative error is stored after
// mode 3).
// threads per eigen-solve CTA (one warp per cell).  The solver's loops are block-size
// generic (the fused kernel runs the same routines with 256 threads and gets the same
// sums); four warps per cell were measured 9% slower on the C3 cavity.  Up to 16 cells per
// SM (the mixed path's ~13 KB of shared memory a cell, 128 registers a thread).
constexpr int kEigTB = 32;

template <typename Real>
__global__ void __launch_bounds__(kEigTB, 16) tucker_eig_kernel(TuckerStepParams P, TuckerSplitBufs B,
                                                             int m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nm = P.Nmax, R = P.R, K = sub_k(Nm, R);
  Smem<Real> sm{};
  sm.nmax = Nm;
  sm.kdim = K;
  {
    size_t off = 0;
    auto takeD = [&](size_t n) {
      double *p = reinterpret_cast<double *>(smem_raw + off);
      off += sizeof(double) * n;
      return p;
    };
    sm.par = takeD(32);
    sm.red = takeD(32);
    sm.Q = takeD((size_t)Nm * K);
    sm.W = takeD((size_t)Nm * K);
    sm.B = takeD((size_t)K * K);
    sm.Z = takeD(K);
    sm.cs = takeD(K + 2);
    if (sizeof(Real) == 8) {  // the FP64 path's retry start (the mixed path starts from sm.Q)
      sm.Vr = reinterpret_cast<Real *>(smem_raw + off);
      off += sizeof(Real) * (size_t)Nm * K;
    } else {
      sm.Vr = nullptr;
    }
    off = (off + 15) & ~size_t(15);
    sm.Q32 = reinterpret_cast<float *>(sm.W);
    sm.W32 = sm.Q32 + (size_t)Nm * K;
    sm.pairs = reinterpret_cast<int *>(smem_raw + off);
    off += sizeof(int) * (K + 2);
    sm.perm = reinterpret_cast<int *>(smem_raw + off);
  }
  PhaseClock pc(P.phase);
  const int N[3] = {P.N1, P.N2, P.N3};
  const int64_t c = B.c0 + blockIdx.x, j = B.joff + blockIdx.x;  // j: buffer index
  const int n = N[m];
  // the previous factor (the warm start) to shared memory, into a block the eigen-solver
  // fills only after reading it (sm.Q on the mixed path, where the FP32 basis lives in
  // sm.W; sm.W on the FP64 path).  The Gram matrix is read where the Gram kernel left it
  // (L2 / L1): without a shared copy of it more cells fit on an SM at once.
  double *Ws = sizeof(Real) == 4 ? sm.Q : sm.W;
  {
    const StagePiece pcs[1] = {{Ws, P.cur.fac[m] + c * (int64_t)n * R, 8u * (unsigned)(n * R)}};
    if (!stage_to_shared(pcs, 1, P.flag)) return;  // timed out: step reported failed
  }
  sm.Cg = B.C + j * (int64_t)Nm * Nm;
  const double tr = gram_trace<Real>(sm, n);
  // ||X||^2 = trace of the first Gram matrix + the columns it left out (B.disc)
  if (m == 0 && threadIdx.x == 0) B.e[j] = tr + B.disc[j];
  __syncthreads();
  const double dropped = m == 0 ? B.disc[j] : 0.0;
  const double thr = P.tol * P.tol / 3.0 * B.e[j] - dropped;
  const double *wU = Ws;
  const int wr = P.cur.rank[3 * c + m];
  int kmax = n < R + kExtra ? n : R + kExtra;
  if (kmax > kOrthMax) kmax = kOrthMax;
  int k = (wr > 0 && thr > 0.0 && wr + kExtra < kmax) ? wr + kExtra : kmax;
  pc.mark(4);
  // truncating: dependent columns zeroed; exact: re-seeded (as in round_hosvd)
  k = leading_eigs<Real, double>(sm, n, k, wU, R, wr, pc, thr > 0.0 ? kDepZero : kDepReseed);
  bool met;
  int r = choose_rank<Real>(sm, n, k, thr, R, &met, tr);
  pc.mark(7);
  if (!met && k < kmax) {  // the k columns found start a solve with kmax columns
    if constexpr (sizeof(Real) == 4) {
      // mixed path: from sm.Q, which the solver reads into its FP32 basis (in sm.W's
      // space) before it writes sm.Q again
      for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) sm.Q[idx] = sm.W[idx];
      __syncthreads();
      k = leading_eigs<Real, double>(sm, n, kmax, sm.Q, k, k, pc, kDepReseed);
    } else {
      for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) sm.Vr[idx] = (Real)sm.W[idx];
      __syncthreads();
      k = leading_eigs<Real, Real>(sm, n, kmax, sm.Vr, k, k, pc, kDepReseed);
    }
    r = choose_rank<Real>(sm, n, k, thr, R, &met, tr);
    pc.mark(8);
    pc.count(2, 1);
  }
  double *U = P.nxt.fac[m] + c * (int64_t)n * R;
  for (int idx = threadIdx.x; idx < n * r; idx += blockDim.x) {
    const int i = idx / r, jj = idx - i * r;
    U[(int64_t)i * R + jj] = sm.W[i * k + jj];
  }
  if (threadIdx.x == 0) {
    P.nxt.rank[3 * c + m] = r;
    const double d = B.disc[j] + sm.par[31];
    B.disc[j] = d;
    if (m == 2 && P.err) P.err[c] = B.e[j] > 0.0 ? sqrt(d / B.e[j]) : 0.0;
  }
  pc.mark(7);
}

// out = T x_m V^T for m = 0, 1 (V: n x r, row-major): a thread takes one position of
// the other two indices and forms all r outputs there, so each input fibre is read
// once; each output is the same fma chain as project()'s (a = 0 .. n-1).  KM >= r
// bounds the accumulators; Exact (r == KM) drops the per-output guards, so that no
// predicated-off FP64 instruction takes a slot of the FP64 pipe.
template <typename Real, int KM, bool Exact>
__device__ void project_fibres(const Real *T, const int D[3], int m, int r, const Real *V,
                               Real *out) {
  if (Exact) r = KM;
  const int n = D[m];
  const int npos = m == 0 ? D[1] * D[2] : D[0] * D[2];
  const int64_t plane = (int64_t)D[1] * D[2];
  for (int pos = threadIdx.x; pos < npos; pos += blockDim.x) {
    int64_t base, stride, obase, ostride;
    if (m == 0) {
      base = pos;
      stride = plane;
      obase = pos;
      ostride = plane;
    } else {
      const int i0 = pos / D[2], i2 = pos - i0 * D[2];
      base = (int64_t)i0 * plane + i2;
      stride = D[2];
      obase = (int64_t)i0 * r * D[2] + i2;
      ostride = D[2];
    }
    Real s[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) s[k] = 0;
    for (int a = 0; a < n; ++a) {
      const Real x = T[base + a * stride];
      const Real *v = V + a * r;
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (Exact || k < r) s[k] = fma(v[k], x, s[k]);
    }
#pragma unroll
    for (int k = 0; k < KM; ++k)
      if (Exact || k < r) out[obase + k * ostride] = s[k];
  }
  __syncthreads();
}

// project_fibres with the accumulator count fixed to r for r <= 8
template <typename Real>
__device__ void project_fibres_r(const Real *T, const int D[3], int m, int r, const Real *V,
                                 Real *out) {
  switch (r) {
    case 1: project_fibres<Real, 1, true>(T, D, m, r, V, out); break;
    case 2: project_fibres<Real, 2, true>(T, D, m, r, V, out); break;
    case 3: project_fibres<Real, 3, true>(T, D, m, r, V, out); break;
    case 4: project_fibres<Real, 4, true>(T, D, m, r, V, out); break;
    case 5: project_fibres<Real, 5, true>(T, D, m, r, V, out); break;
    case 6: project_fibres<Real, 6, true>(T, D, m, r, V, out); break;
    case 7: project_fibres<Real, 7, true>(T, D, m, r, V, out); break;
    case 8: project_fibres<Real, 8, true>(T, D, m, r, V, out); break;
    default: project_fibres<Real, kOrthMax, false>(T, D, m, r, V, out); break;
  }
}

// Projection of mode m with the new factor: Y_{m+1} = Y_m x_m U_m^T (m = 0, 1,
// working precision), or the core G = Y_2 x_3 U_3^T (m = 2, FP64 accumulation)
template <typename Real>
__global__ void __launch_bounds__(kTB) tucker_proj_kernel(TuckerStepParams P, TuckerSplitBufs B,
                                                          int m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = P.R;
  const int N[3] = {P.N1, P.N2, P.N3};
  const int64_t c = B.c0 + blockIdx.x, j = B.joff + blockIdx.x;  // j: buffer index
  int D[3];
  split_dims(B, P.nxt, c, m, N, D);
  const int n = D[m], r = P.nxt.rank[3 * c + m];
  const double *U = P.nxt.fac[m] + c * (int64_t)n * R;
  const Real *src = split_src<Real>(B, j, m, R, N);
  if (m < 2) {
    Real *V = reinterpret_cast<Real *>(smem_raw);
    for (int idx = threadIdx.x; idx < n * r; idx += blockDim.x) {
      const int i = idx / r, k = idx - i * r;
      V[idx] = (Real)U[(int64_t)i * R + k];
    }
    __syncthreads();
    Real *dst = const_cast<Real *>(split_src<Real>(B, j, m + 1, R, N));
    project_fibres_r<Real>(src, D, m, r, V, dst);
  } else {
    double *Us = reinterpret_cast<double *>(smem_raw);
    for (int idx = threadIdx.x; idx < n * r; idx += blockDim.x) {
      const int i = idx / r, k = idx - i * r;
      Us[idx] = U[(int64_t)i * R + k];
    }
    __syncthreads();
    const int total = D[0] * D[1] * r;
    double *G = P.nxt.core + c * (int64_t)R * R * R;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int k3 = idx % r, k12 = idx / r;
      const Real *y = src + (int64_t)k12 * n;
      double s = 0.0;
      for (int a = 0; a < n; ++a) s = fma(Us[a * r + k3], (double)y[a], s);
      G[idx] = s;
    }
  }
}

// Expansion of cells [c0, c0 + ncell) into full FP64 tensors (inspection).
template <typename Real>
__global__ void __launch_bounds__(kTB) tucker_expand_kernel(TuckerDev T, int64_t c0, int64_t ncell,
                                                            int N1, int N2, int N3, int R, int Nmax,
                                                            void *scratch, size_t stride, double *out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<Real> sm{};  // expand() uses the factor rows only
  for (int a = 0; a < 3; ++a) sm.fac[a] = reinterpret_cast<Real *>(smem_raw) + (size_t)a * Nmax * R;
  const int N[3] = {N1, N2, N3};
  const int NN = N1 * N2 * N3;
  Real *E = reinterpret_cast<Real *>(scratch) + (size_t)blockIdx.x * stride;
  Real *T2 = E + NN;
  Real *T1 = T2 + (size_t)R * N2 * N3;
  for (int64_t j = blockIdx.x; j < ncell; j += gridDim.x) {
    expand<Real>(T, c0 + j, N, R, sm, T1, T2, E);
    for (int i = threadIdx.x; i < NN; i += blockDim.x) out[j * NN + i] = (double)E[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Moments of each cell's Tucker tensor (Section 4 item 5) about the reference
// velocity r: the same 19 raw sums as the full-grid path plus the outflow sums
// of axis-aligned wall faces; FP64.
__global__ void __launch_bounds__(128) tucker_moments_kernel(TuckerMomentParams P) {
  // [3][4][R] projections, [6][R] wall projections, [3][4][Nx] powers of the
  // velocities, then (P.stage) the cell's factors and core staged from global memory
  extern __shared__ __align__(16) double msm[];
  __shared__ double s_out[32];
  __shared__ SlotDev s_slot[6];
  const int64_t c = P.c0 + blockIdx.x;
  const int tid = threadIdx.x;
  const int R = P.R;
  const int N[3] = {P.N1, P.N2, P.N3};
  const int r[3] = {P.T.rank[3 * c], P.T.rank[3 * c + 1], P.T.rank[3 * c + 2]};
  const int64_t us = P.uref_stride;
  const double ref[3] = {P.uref ? P.uref[us * c] : 0.0, P.uref ? P.uref[us * c + 1] : 0.0,
                         P.uref ? P.uref[us * c + 2] : 0.0};
  double *Sp = msm;            // [a][p][k], p = 0..3
  double *Sw = msm + 12 * R;   // [l][k] wall outflow projection for slot l
  const double *Uc[3], *G = P.T.core + c * (int64_t)R * R * R;
  for (int a = 0; a < 3; ++a) Uc[a] = P.T.fac[a] + c * (int64_t)N[a] * R;
  const int Nx = max(N[0], max(N[1], N[2]));
  // (xi_a,i - r_a)^p for p = 0..3, formed once per cell (not once per column k)
  double *Pw = msm + ((18 * (size_t)R + 1) & ~size_t(1));  // [a][p][Nx]
  for (int idx = tid; idx < 12 * Nx; idx += blockDim.x) {
    const int i = idx % Nx, ap = idx / Nx, p = ap % 4, a = ap / 4;
    double w = 1.0;
    if (i < N[a]) {
      const double v = P.xi[a][i] - ref[a];
      for (int e = 0; e < p; ++e) w *= v;
    }
    Pw[idx] = w;
  }
  if (tid < 6) s_slot[tid] = P.slot[c * 6 + tid];
  if (P.stage) {  // bit 0: factors, bit 1: core (the leading r1 r2 r3 entries)
    StagePiece pcs[4];
    int np = 0;
    size_t off = ((18 * (size_t)R + 1) & ~size_t(1)) + 12 * (size_t)Nx;
    if (P.stage & 1)
      for (int a = 0; a < 3; ++a) {
        pcs[np++] = {msm + off, Uc[a], 8u * (unsigned)(N[a] * R)};
        Uc[a] = msm + off;
        off += ((size_t)N[a] * R + 1) & ~size_t(1);
      }
    if (P.stage & 2) {
      const int g = r[0] * r[1] * r[2];
      const int ge = (g & 1) && g < R * R * R ? g + 1 : g;  // 16-byte multiple when possible
      pcs[np++] = {msm + off, G, 8u * (unsigned)ge};
      G = msm + off;
    }
    if (!stage_to_shared(pcs, np, P.flag)) return;  // timed out: step reported failed
  } else {
    __syncthreads();
  }
  // S_a^(p)[k] = sum_i U_a[i][k] (xi_a,i - r_a)^p
  for (int idx = tid; idx < 12 * R; idx += blockDim.x) {
    const int k = idx % R, ap = idx / R, a = ap / 4;
    double s = 0.0;
    if (k < r[a]) {
      const double *U = Uc[a], *w = Pw + ap * Nx;
      for (int i = 0; i < N[a]; ++i) s = fma(U[(int64_t)i * R + k], w[i], s);
    }
    Sp[idx] = s;
  }
  for (int idx = tid; idx < 6 * R; idx += blockDim.x) {
    const int k = idx % R, l = idx / R;
    const SlotDev &sl = s_slot[l];
    double s = 0.0;
    if (sl.kind == kWall && sl.axis >= 0 && k < r[sl.axis]) {
      const int a = sl.axis;
      const double *U = Uc[a];
      for (int i = 0; i < N[a]; ++i) s = fma(U[(int64_t)i * R + k], fmax(sl.sgn * P.xi[a][i], 0.0), s);
    }
    Sw[idx] = s;
  }
  __syncthreads();
  // monomials (a1, a2, a3) of the 19 sums; thread j < 19 computes sum j,
  // threads 19..24 the wall outflows
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

// The kernels' dynamic shared-memory opt-in is a per-function setting shared by
// every context in the process: only ever raise it (to the largest size any
// context needs), and do so outside stream captures (tucker_prepare_launch is
// called when a context is created).  The sizes set so far are kept per kernel
// function (one kernel serves contexts of every size).
std::mutex g_optin_mu;
std::map<const void *, size_t> g_optin;

template <typename K>
int raise_smem_optin(K kernel, size_t smem) {
  std::lock_guard<std::mutex> lk(g_optin_mu);
  size_t &opted = g_optin[reinterpret_cast<const void *>(kernel)];
  if (smem <= opted) return 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  opted = smem;
  return 0;
}

template <typename Real, int TS>
int launch_step_TS(const TuckerStepParams &p, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes<Real>(p.Nmax, p.R);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap == cudaStreamCaptureStatusNone &&
      raise_smem_optin(tucker_step_kernel<Real, TS>, smem) != 0)
    return -1;
  tucker_step_kernel<Real, TS><<<grid, kTB, smem, s>>>(p);
  return 0;
}

template <typename Real>
int launch_step_T(const TuckerStepParams &p, int grid, cudaStream_t s) {
  return p.Nmax <= 32 ? launch_step_TS<Real, 2>(p, grid, s) : launch_step_TS<Real, 4>(p, grid, s);
}

template <typename Real, int TS>
struct SplitSmem {
  size_t asm_, gram, gram_small, eig, proj;
  SplitSmem(int Nmax, int R) {
    gram_small = sizeof(double) * (64 + (size_t)Nmax * Nmax) + sizeof(Real) * 32 * kTileRow + 64;
    asm_ = smem_asm_bytes<Real>(Nmax, R);
    gram = sizeof(double) * (64 + (size_t)Nmax * Nmax) +
           2 * sizeof(Real) * (size_t)(Nmax > 32 ? Nmax : 32) * kTileRow +
           sizeof(int) * 4 * kTB + 64;
    eig = smem_eig_bytes<Real>(Nmax, R);
    proj = sizeof(double) * (size_t)Nmax * R;
  }
};

template <typename Real, int TS>
// Raise the shared-memory opt-ins of both variants' kernels; returns a mask of
// the variants whose kernels fit: 1 fused, 2 phase-major.
int prepare_split_TS(int Nmax, int R) {
  const SplitSmem<Real, TS> z(Nmax, R);
  int mask = 0;
  if (raise_smem_optin(tucker_step_kernel<Real, TS>, smem_bytes<Real>(Nmax, R)) == 0) mask |= 1;
  if (sizeof(Real) == 4 && Nmax <= 64)  // GEMM-form assembly (used where the mesh allows)
    tucker_asm_gemm_prepare(Nmax, Nmax, R);
  if (raise_smem_optin(tucker_asm_kernel<Real>, z.asm_) == 0 &&
      raise_smem_optin(tucker_t2_kernel<Real>, z.asm_) == 0 &&
      raise_smem_optin(tucker_gram_kernel<Real, TS>, z.gram) == 0 &&
      raise_smem_optin(tucker_gram_small_kernel<Real>, z.gram_small) == 0 &&
      raise_smem_optin(tucker_eig_kernel<Real>, z.eig) == 0 &&
      raise_smem_optin(tucker_proj_kernel<Real>, z.proj) == 0)
    mask |= 2;
  return mask;
}

// The chain of one range of cells: assembly, then per mode Gram / eigen-solve /
// projection.
template <typename Real, int TS>
void split_chain(const TuckerStepParams &p, const TuckerSplitBufs &b, const SplitSmem<Real, TS> &z,
                 cudaStream_t s, const LaunchTimer &T, const TuckerMomentParams *mp) {
  const int ga = (int)(b.cn < b.asm_grid ? b.cn : b.asm_grid);
  T(kKAsm, true, s);
  if (sizeof(Real) == 4 && p.gemm_asm) {  // one small GEMM per cell of its rank-one terms
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int gg = (int)(b.cn < 2 * sms ? b.cn : 2 * sms);
    const int nbuf = ag_nbuf(p.Nmax, p.N1, p.N3, p.R);
    ag_kernel(padN(p.N1), nbuf)<<<gg, kAgThreads, ag_smem_bytes(p.Nmax, p.N1, p.R, nbuf), s>>>(p, b);
  } else {
    tucker_asm_kernel<Real><<<ga, kAsmTB, z.asm_, s>>>(p, b);
  }
  T(kKAsm, false, s);
  for (int m = 0; m < 3; ++m) {
    const int gc = m == 0 ? kKGram0 : kKGram12;
    T(gc, true, s);
    bool done = false;
    if constexpr (sizeof(Real) == 4) {
      if (m == 0 && p.tc_gram) {  // exact-split Gram on the tensor cores (gram_tc.cu)
        const int64_t NN = (int64_t)p.N1 * p.N2 * p.N3, NC = (int64_t)p.Nmax * p.Nmax;
        done = launch_gram_tc(reinterpret_cast<const float *>(b.X) + b.joff * NN, NN, b.cn, p.N1,
                              p.N2 * p.N3, reinterpret_cast<float2 *>(b.C + b.joff * NC), nullptr,
                              NC, b.disc + b.joff, p.flag, s,
                              b.rowmax ? b.rowmax + b.joff * p.Nmax : nullptr, p.Nmax,
                              p.phase) == 0;
      }
    }
    if (done) {
    } else if (m >= 1 && p.Nmax <= 32) {  // every cell's N_m <= 32: gram_seq in a light kernel
      tucker_gram_small_kernel<Real><<<(unsigned)b.cn, kTB, z.gram_small, s>>>(p, b, m);
    } else {
      // engine AUTO (mixed path): second/third modes with half the threads, so that twice
      // as many cells run per SM (their unfoldings have few columns), where every 4 x 4
      // output block still gets a thread (gram_tiled gives each thread one block: at most
      // 128 blocks, i.e. Nmax <= 60); the CUDA-core engine keeps the fused variant's block
      // size, and with it the same sums
      const int nbk = (p.Nmax + 3) / 4;
      const int tb = (m >= 1 && p.tc_gram && nbk * (nbk + 1) / 2 <= kTB / 2) ? kTB / 2 : kTB;
      tucker_gram_kernel<Real, TS><<<(unsigned)b.cn, tb, z.gram, s>>>(p, b, m);
    }
    T(gc, false, s);
    T(kKEig, true, s);
    tucker_eig_kernel<Real><<<(unsigned)b.cn, kEigTB, z.eig, s>>>(p, b, m);
    T(kKEig, false, s);
    T(kKProj, true, s);
    tucker_proj_kernel<Real><<<(unsigned)b.cn, kTB, z.proj, s>>>(p, b, m);
    T(kKProj, false, s);
  }
  if (mp) {  // moments of the new state of these cells
    TuckerMomentParams q = *mp;
    q.c0 = b.c0;
    q.nc = b.c0 + b.cn;
    T(kKMoments, true, s);
    launch_tucker_moments(q, s);
    T(kKMoments, false, s);
  }
}

template <typename Real, int TS>
int launch_split_TS(const TuckerStepParams &p, TuckerSplitBufs b, int64_t chunk, cudaStream_t s,
                    const LaunchTimer *lt, const SplitStreams *ss, const TuckerMomentParams *mp) {
  const LaunchTimer none{nullptr, nullptr};
  const LaunchTimer &T = lt ? *lt : none;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap == cudaStreamCaptureStatusNone && !(prepare_split_TS<Real, TS>(p.Nmax, p.R) & 2))
    return -1;
  const SplitSmem<Real, TS> z(p.Nmax, p.R);
  // per-cell parameters (and the macroparameters) of every cell, one thread each,
  // so that no assembly block forms them serially
  T(kKMoments, true, s);
  tucker_cellpar_kernel<<<(unsigned)((p.nc + 127) / 128), 128, 0, s>>>(p, b.cellpar, b.macro);
  T(kKMoments, false, s);
  TuckerStepParams q = p;
  q.cellpar = b.cellpar;
  T(kKContract, true, s);
  tucker_t2_kernel<Real><<<(unsigned)(p.nc < 65535 * 16 ? p.nc : 65535 * 16), kAsmTB, z.asm_, s>>>(q, b);
  T(kKContract, false, s);
  // with extra streams (and no per-launch timing), each chunk's cell ranges run
  // their chains concurrently: one range's FP64-bound eigen-solves overlap another
  // range's FP32-bound Gram / assembly kernels
  const int ways = (ss && !(lt && lt->mark)) ? (ss->ways < kMaxWays ? ss->ways : kMaxWays) : 1;
  auto fork = [&]() -> bool {
    if (cudaEventRecord(ss->fork, s) != cudaSuccess) return false;
    for (int w = 1; w < ways; ++w)
      if (cudaStreamWaitEvent(ss->sx[w - 1], ss->fork, 0) != cudaSuccess) return false;
    return true;
  };
  auto join = [&]() -> bool {
    for (int w = 1; w < ways; ++w) {
      if (cudaEventRecord(ss->join[w - 1], ss->sx[w - 1]) != cudaSuccess) return false;
      if (cudaStreamWaitEvent(s, ss->join[w - 1], 0) != cudaSuccess) return false;
    }
    return true;
  };
  if (ways > 1 && !fork()) return -1;
  for (int64_t c0 = 0; c0 < p.nc; c0 += chunk) {
    const int64_t cn = p.nc - c0 < chunk ? p.nc - c0 : chunk;
    const int wn = cn >= ways ? ways : 1;
    for (int w = 0; w < wn; ++w) {
      const int64_t a = cn * w / wn, e = cn * (w + 1) / wn;
      TuckerSplitBufs bw = b;
      bw.c0 = c0 + a;
      bw.cn = e - a;
      bw.joff = a;
      split_chain<Real, TS>(q, bw, z, w == 0 ? s : ss->sx[w - 1], T, mp);
    }
    // the next chunk reuses the buffers: every range must be done
    if (ways > 1 && c0 + chunk < p.nc && !(join() && fork())) return -1;
  }
  if (ways > 1 && !join()) return -1;
  return 0;
}

template <typename Real>
int launch_expand_T(const TuckerDev &T, int64_t c0, int64_t ncell, int N1, int N2, int N3, int R,
                    int Nmax, void *scratch, size_t stride, double *out, int grid, cudaStream_t s) {
  const size_t smem = sizeof(Real) * 3 * (size_t)Nmax * R;
  if (raise_smem_optin(tucker_expand_kernel<Real>, smem) != 0) return -1;
  tucker_expand_kernel<Real><<<grid, kTB, smem, s>>>(T, c0, ncell, N1, N2, N3, R, Nmax, scratch,
                                                     stride, out);
  return 0;
}

}  // namespace

size_t tucker_scratch_elems(int N1, int N2, int N3, int R) {
  // X, then the assembly's compact mode-2/3 contractions (at most kTerms blocks
  // of R x N2 x N3), which also hold the rounding's and the expansion's T2, T1
  const size_t NN = (size_t)N1 * N2 * N3;
  return NN + (size_t)kTerms * R * N2 * N3 + 64;
}

template <typename Real, int TS>
int blocks_per_sm_TS(int Nmax, int R) {
  const size_t smem = smem_bytes<Real>(Nmax, R);
  if (raise_smem_optin(tucker_step_kernel<Real, TS>, smem) != 0) return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tucker_step_kernel<Real, TS>, kTB, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb < 1 ? 1 : nb;
}

template <typename Real>
int blocks_per_sm_T(int Nmax, int R) {
  return Nmax <= 32 ? blocks_per_sm_TS<Real, 2>(Nmax, R) : blocks_per_sm_TS<Real, 4>(Nmax, R);
}

int tucker_step_blocks_per_sm(int Nmax, int R, bool fp64) {
  return fp64 ? blocks_per_sm_T<double>(Nmax, R) : blocks_per_sm_T<float>(Nmax, R);
}

size_t tucker_smem_bytes(int Nmax, int R, bool fp64) {
  return fp64 ? smem_bytes<double>(Nmax, R) : smem_bytes<float>(Nmax, R);
}

int launch_tucker_step(const TuckerStepParams &p, int grid, bool fp64, cudaStream_t s) {
  return fp64 ? launch_step_T<double>(p, grid, s) : launch_step_T<float>(p, grid, s);
}

int launch_tucker_split_step(const TuckerStepParams &p, TuckerSplitBufs b, int64_t chunk,
                             bool fp64, cudaStream_t s, const LaunchTimer *lt,
                             const SplitStreams *ss, const TuckerMomentParams *mp) {
  if (fp64)
    return p.Nmax <= 32 ? launch_split_TS<double, 2>(p, b, chunk, s, lt, ss, mp)
                        : launch_split_TS<double, 4>(p, b, chunk, s, lt, ss, mp);
  return p.Nmax <= 32 ? launch_split_TS<float, 2>(p, b, chunk, s, lt, ss, mp)
                      : launch_split_TS<float, 4>(p, b, chunk, s, lt, ss, mp);
}

int tucker_split_asm_per_sm() { return 6; }

size_t tucker_split_t2_elems(int N1, int N2, int N3, int R) {
  (void)N1;
  return (size_t)kTerms * R * N2 * N3 + 64;
}

int tucker_prepare_launch(int Nmax, int R, bool fp64) {
  if (fp64)
    return Nmax <= 32 ? prepare_split_TS<double, 2>(Nmax, R) : prepare_split_TS<double, 4>(Nmax, R);
  return Nmax <= 32 ? prepare_split_TS<float, 2>(Nmax, R) : prepare_split_TS<float, 4>(Nmax, R);
}

int tucker_asm_gemm_prepare(int Nmax, int N1, int R) {
  if (Nmax > 64 || N1 > 64) return -1;  // register tiles of at most 16 rows per thread
  for (int nbuf = 1; nbuf <= 2; ++nbuf) {
    const size_t smem = ag_smem_bytes(Nmax, N1, R, nbuf);
    if (nbuf == 2 && smem > 227 * 1024) break;  // then only one stage is ever used
    if (raise_smem_optin(ag_kernel(padN(N1), nbuf), smem) != 0) return -1;
  }
  return 0;
}

size_t tucker_split_bytes_per_cell(int N1, int N2, int N3, int R, int Nmax, bool fp64) {
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  return es * ((size_t)N1 * N2 * N3 + (size_t)R * N2 * N3 + (size_t)R * R * N3) +
         sizeof(double) * ((size_t)Nmax * Nmax + 2) + sizeof(float) * (size_t)Nmax;
}

size_t tucker_split_t2all_bytes_per_cell(int N1, int N2, int N3, int R, bool fp64) {
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  return es * (size_t)R * ((size_t)N2 * N3 + padN(N1)) + sizeof(double) * kCellPar;
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

// The cell's factors (and core) are staged in shared memory when they fit in the
// default 48 KB with the projections.
void launch_tucker_moments(const TuckerMomentParams &p, cudaStream_t s) {
  const int N[3] = {p.N1, p.N2, p.N3};
  const int Nx = std::max(N[0], std::max(N[1], N[2]));
  const size_t base = ((18 * (size_t)p.R + 1) & ~size_t(1)) + 12 * (size_t)Nx;
  size_t fac = 0;
  for (int a = 0; a < 3; ++a) fac += ((size_t)N[a] * p.R + 1) & ~size_t(1);
  const size_t core = (size_t)p.R * p.R * p.R + 1;
  constexpr size_t kLimit = 48 * 1024 / sizeof(double);
  TuckerMomentParams q = p;
  q.stage = base + fac + core <= kLimit ? 3 : (base + fac <= kLimit ? 1 : 0);
  const size_t smem =
      sizeof(double) * (q.stage == 3 ? base + fac + core : (q.stage == 1 ? base + fac : base));
  tucker_moments_kernel<<<(unsigned)(p.nc - p.c0), 128, smem, s>>>(q);
}

}  // namespace dvm
