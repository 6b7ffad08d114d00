// Full-grid FP64 kernels of the S-model DVM step (arXiv:1912.04582, Section 3).
//
// One CTA owns one spatial cell.  Thread t owns the velocity "columns"
// p = (i2, i3) = t, t + B, ... of the cell and walks i1 = 0..N1-1, so that for
// a fixed i1 a warp reads 32 consecutive doubles of f (i3 fastest): every load
// and store of f is a coalesced 256-byte transaction.  Per-cell data that
// depends on i1 only (the first Maxwellian factor, the Shakhov polynomial
// pieces, the upwind weights of faces normal to axis 1) sits in shared memory;
// data that depends on (i2, i3) only is kept in registers for the whole i1
// walk.  This makes the per-node work of the fused step
//   f^{n+1} = c0(xi) f + dt nu f^S + sum_l m_l(xi) g_l,
//   c0 = 1 - dt nu - sum_l c_l xi_n,l^+,   m_l = -c_l xi_n,l^-,   c_l = dt |A_l| / |V|
// (Algorithm 1 with Algorithm 2 inside, CIR flux written as
// xi_n^+ f_L + xi_n^- f_R, exact-flux equation) one FP64 FMA per face plus a
// handful of FMAs for f^S and the update, with no exp per node: f^M is the
// product of three 1D factors (Section 5, rank-1 Maxwellian).
//
// The epilogue accumulates the moment sums of f^{n+1} about the cell's current
// velocity u^n (so the heat flux of the next step needs no second pass and no
// large cancellation), plus the wall outflow sums that fix the wall density of
// the next step (impermeability condition, Section 2).
#include <algorithm>
#include <cmath>

#include "dvm_device.cuh"
#include "dvm_internal.h"

namespace dvm {
namespace {

constexpr double kPi = 3.14159265358979323846;

template <int B>
__device__ inline void warp_block_reduce(double (&v)[kRawSums], double (*s_red)[kRawSums],
                                         double *s_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRawSums; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kRawSums; ++k) s_red[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < kRawSums) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < B / 32; ++q) t += s_red[q][threadIdx.x];
    s_tot[threadIdx.x] = t;
  }
  __syncthreads();
}

// Fold the i1-walk partial sums P_k = sum_{i1} v1^k g (k = 0..3) of one column
// (i2, i3) into the 13 moment sums about r (v = xi - r).
__device__ __forceinline__ void fold_column(double (&acc)[kRawSums], double P0, double P1,
                                            double P2, double P3, double v2, double v3) {
  const double v22 = v2 * v2, v33 = v3 * v3, s23 = v22 + v33;
  acc[0] += P0;
  acc[1] += P1;
  acc[2] = fma(v2, P0, acc[2]);
  acc[3] = fma(v3, P0, acc[3]);
  acc[4] += P2;
  acc[5] = fma(v22, P0, acc[5]);
  acc[6] = fma(v33, P0, acc[6]);
  acc[7] = fma(v2, P1, acc[7]);
  acc[8] = fma(v3, P1, acc[8]);
  acc[9] = fma(v2 * v3, P0, acc[9]);
  acc[10] += fma(s23, P1, P3);
  acc[11] += fma(v2, P2, v2 * s23 * P0);
  acc[12] += fma(v3, P2, v3 * s23 * P0);
}

// ------------------------------------------------------------------------
// Fused explicit step: f^{n+1} and the moment sums of f^{n+1}.  With kIncr the
// kernel writes the increment dt R^n of the explicit scheme instead (the
// right-hand side of the implicit step) and the cell's dt nu, without moments.
template <int B, bool ALL_AXIS, bool kIncr>
__global__ void __launch_bounds__(B) full_step_kernel(const FullParams P) {
  extern __shared__ double tab[];
  __shared__ SlotDev s_slot[6];
  __shared__ double s_par[12];
  __shared__ double s_scale[6];
  __shared__ double s_red[B / 32][kRawSums];
  __shared__ double s_tot[kRawSums];

  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x;
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3;
  const int NP = N2 * N3;
  const int64_t nn = (int64_t)N1 * NP;

  double *tF1 = tab;           // dt nu n^{1/3} (pi T)^{-1/2} exp(-v1^2/T)
  double *tA1 = tF1 + N1;      // A q1 v1
  double *tT1 = tA1 + N1;      // v1^2 / T
  double *tV1 = tT1 + N1;      // v1
  double *tV2 = tV1 + N1;      // v1^2
  double *tV3 = tV2 + N1;      // v1^3
  double *tC1 = tV3 + N1;      // 1 - dt nu - sum_{axis-1 faces} c max(s xi1, 0)
  double *tX1 = tC1 + N1;      // xi1
  double *tM = tX1 + N1;       // [6][N1] inflow weight -c min(xi_n, 0) of axis-1 faces (x n_w)
  double *tO = tM + 6 * N1;    // [6][N1] wall outflow weight of axis-1 wall faces
  double *tF2 = tO + 6 * N1;   // n^{1/3} (pi T)^{-1/2} exp(-v2^2/T)
  double *tF3 = tF2 + N2;

  const double *S = P.sums + c * kSums;
  if (tid < 6) {
    s_slot[tid] = P.slot[c * 6 + tid];
    const SlotDev &sl = s_slot[tid];
    s_scale[tid] = (sl.kind == kWall) ? -S[16 + tid] / sl.wall_den : 1.0;
  }
  if (tid == 0) {
    CellMacro m;
    macro_from_sums(S, P.w, m);
    if (m.bad) atomicOr(P.flag, 1);
    const double nu = P.delta * m.n * pow(m.T, 1.0 - P.omega);
    s_par[0] = m.n;
    s_par[1] = m.u[0];
    s_par[2] = m.u[1];
    s_par[3] = m.u[2];
    s_par[4] = m.T;
    s_par[5] = m.q[0];
    s_par[6] = m.q[1];
    s_par[7] = m.q[2];
    s_par[8] = nu;
    s_par[9] = 1.6 * (1.0 - P.Pr) / (m.n * m.T * m.T);  // Shakhov A (R_g = 1/2, m = 1)
    s_par[10] = cbrt(m.n) / sqrt(kPi * m.T);            // per-axis Maxwellian amplitude
    s_par[11] = P.dt * nu;
    if (kIncr) P.dtnu[c] = s_par[11];
  }
  __syncthreads();

  const double T = s_par[4], invT = 1.0 / T, A = s_par[9], amp = s_par[10], dtnu = s_par[11];
  const double u0 = s_par[1], u1 = s_par[2], u2 = s_par[3];
  const double q0 = s_par[5], q1 = s_par[6], q2 = s_par[7];

  for (int i = tid; i < N1; i += B) {
    const double x = P.xi[0][i];
    const double v = x - u0;
    tF1[i] = dtnu * amp * exp(-v * v * invT);
    tA1[i] = A * q0 * v;
    tT1[i] = v * v * invT;
    tV1[i] = v;
    tV2[i] = v * v;
    tV3[i] = v * v * v;
    tX1[i] = x;
    double c0 = (kIncr ? 0.0 : 1.0) - dtnu;
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      const SlotDev &sl = s_slot[l];
      double m = 0.0, o = 0.0;
      if (sl.axis == 0) {
        const double sx = sl.sgn * x;
        c0 -= sl.c * fmax(sx, 0.0);
        m = -sl.c * fmin(sx, 0.0) * s_scale[l];  // inflow: -c xi_n^- (>= 0)
        o = sl.kind == kWall ? fmax(sx, 0.0) : 0.0;
      }
      tM[l * N1 + i] = m;
      tO[l * N1 + i] = o;
    }
    tC1[i] = c0;
  }
  for (int i = tid; i < N2; i += B) {
    const double v = P.xi[1][i] - u1;
    tF2[i] = amp * exp(-v * v * invT);
  }
  for (int i = tid; i < N3; i += B) {
    const double v = P.xi[2][i] - u2;
    tF3[i] = amp * exp(-v * v * invT);
  }
  __syncthreads();

  double acc[kRawSums];
#pragma unroll
  for (int k = 0; k < kRawSums; ++k) acc[k] = 0.0;

  const double *__restrict__ fown = P.f + c * nn;
  double *__restrict__ fout = P.fnew + c * nn;

  for (int p = tid; p < NP; p += B) {
    const int i2 = p / N3, i3 = p - i2 * N3;
    const double x2 = P.xi[1][i2], x3 = P.xi[2][i3];
    const double v2 = x2 - u1, v3 = x3 - u2;
    const double G = tF2[i2] * tF3[i3];
    const double bq = A * (q1 * v2 + q2 * v3);
    const double cp = (v2 * v2 + v3 * v3) * invT - 2.5;
    double C23 = 0.0;
    const double *src[6];
    double pf[6];   // axis-2/3 faces: upwind weight; generic faces: e2 xi2 + e3 xi3
    double ow[6];   // axis-2/3 wall faces: outflow weight
    int flip1 = 0;  // bit l: mirror i1 for face l
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      const SlotDev &sl = s_slot[l];
      pf[l] = 0.0;
      ow[l] = 0.0;
      if (sl.axis == 1 || sl.axis == 2) {
        const double sx = sl.sgn * (sl.axis == 1 ? x2 : x3);
        C23 -= sl.c * fmax(sx, 0.0);
        pf[l] = -sl.c * fmin(sx, 0.0) * s_scale[l];
        ow[l] = sl.kind == kWall ? fmax(sx, 0.0) : 0.0;
      } else if (!ALL_AXIS && sl.axis < 0) {
        pf[l] = sl.e[1] * x2 + sl.e[2] * x3;
      }
      int pp = p;
      const double *base;
      switch (sl.kind) {
        case kInterior: base = P.f + (int64_t)sl.src * nn; break;
        case kFreeStream:
        case kWall: base = P.ghost + (int64_t)sl.src * nn; break;
        case kSymmetry:
          base = fown;
          if (sl.flip == 0) flip1 |= 1 << l;
          else if (sl.flip == 1) pp = (N2 - 1 - i2) * N3 + i3;
          else pp = i2 * N3 + (N3 - 1 - i3);
          break;
        default: base = fown; break;  // zero gradient
      }
      src[l] = base + pp;
    }

    double P0 = 0.0, P1 = 0.0, P2 = 0.0, P3 = 0.0;
    double O[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
    for (int i1 = 0; i1 < N1; ++i1) {
      const int64_t off = (int64_t)i1 * NP;
      const int64_t offm = (int64_t)(N1 - 1 - i1) * NP;
      const double fc = __ldg(fown + off + p);
      const double fM = tF1[i1] * G;
      const double poly = fma(tA1[i1] + bq, tT1[i1] + cp, 1.0);
      double a = fM * poly;
      double c0 = tC1[i1] + C23;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        const double g = __ldg(src[l] + ((flip1 >> l) & 1 ? offm : off));
        if (sl.axis == 0) {
          a = fma(tM[l * N1 + i1], g, a);
        } else if (ALL_AXIS || sl.axis > 0) {
          a = fma(pf[l], g, a);
        } else {
          const double xu = fma(sl.e[0], tX1[i1], pf[l]);
          const double x = sl.c * xu;
          a = fma(-fmin(x, 0.0) * s_scale[l], g, a);
          c0 -= fmax(x, 0.0);
        }
      }
      const double fn = fma(c0, fc, a);
      fout[off + p] = fn;
      if (kIncr) continue;
      P0 += fn;
      P1 = fma(tV1[i1], fn, P1);
      P2 = fma(tV2[i1], fn, P2);
      P3 = fma(tV3[i1], fn, P3);
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        if (sl.kind == kWall) {
          if (sl.axis == 0) {
            O[l] = fma(tO[l * N1 + i1], fn, O[l]);
          } else if (!ALL_AXIS && sl.axis < 0) {
            O[l] = fma(fmax(fma(sl.e[0], tX1[i1], pf[l]), 0.0), fn, O[l]);
          }
        }
      }
    }
    if (kIncr) continue;
    fold_column(acc, P0, P1, P2, P3, v2, v3);
#pragma unroll
    for (int l = 0; l < 6; ++l) acc[13 + l] += O[l] + ow[l] * P0;
  }
  if (kIncr) return;

  warp_block_reduce<B>(acc, s_red, s_tot);

  if (tid == 0) {
    double *Sn = P.sums_new + c * kSums;
    Sn[0] = u0;
    Sn[1] = u1;
    Sn[2] = u2;
    for (int k = 0; k < kRawSums; ++k) Sn[3 + k] = s_tot[k];
    Sn[22] = 0.0;
    Sn[23] = 0.0;
    if (P.respart) {
      double U0[5], U1[5];
      conserved_from_sums(S, P.w, U0);
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

// ------------------------------------------------------------------------
// Moment sums of f about a reference velocity (no update).
template <int B>
__global__ void __launch_bounds__(B) full_moments_kernel(const MomentParams P) {
  extern __shared__ double tab[];
  __shared__ SlotDev s_slot[6];
  __shared__ double s_red[B / 32][kRawSums];
  __shared__ double s_tot[kRawSums];
  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x;
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3;
  const int NP = N2 * N3;
  const int64_t nn = (int64_t)N1 * NP;
  double *tV1 = tab, *tV2 = tV1 + N1, *tV3 = tV2 + N1, *tX1 = tV3 + N1;
  const double r0 = P.uref ? P.uref[3 * c] : 0.0;
  const double r1 = P.uref ? P.uref[3 * c + 1] : 0.0;
  const double r2 = P.uref ? P.uref[3 * c + 2] : 0.0;
  if (tid < 6) s_slot[tid] = P.slot[c * 6 + tid];
  for (int i = tid; i < N1; i += B) {
    const double x = P.xi[0][i], v = x - r0;
    tV1[i] = v;
    tV2[i] = v * v;
    tV3[i] = v * v * v;
    tX1[i] = x;
  }
  __syncthreads();
  double acc[kRawSums];
#pragma unroll
  for (int k = 0; k < kRawSums; ++k) acc[k] = 0.0;
  const double *fc = P.f + c * nn;
  for (int p = tid; p < NP; p += B) {
    const int i2 = p / N3, i3 = p - i2 * N3;
    const double x2 = P.xi[1][i2], x3 = P.xi[2][i3];
    double P0 = 0.0, P1 = 0.0, P2 = 0.0, P3 = 0.0;
    double O[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i1 = 0; i1 < N1; ++i1) {
      const double g = __ldg(fc + (int64_t)i1 * NP + p);
      P0 += g;
      P1 = fma(tV1[i1], g, P1);
      P2 = fma(tV2[i1], g, P2);
      P3 = fma(tV3[i1], g, P3);
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        if (sl.kind == kWall) {
          const double x = sl.e[0] * tX1[i1] + sl.e[1] * x2 + sl.e[2] * x3;
          O[l] = fma(fmax(x, 0.0), g, O[l]);
        }
      }
    }
    fold_column(acc, P0, P1, P2, P3, x2 - r1, x3 - r2);
#pragma unroll
    for (int l = 0; l < 6; ++l) acc[13 + l] += O[l];
  }
  warp_block_reduce<B>(acc, s_red, s_tot);
  if (tid == 0) {
    double *Sn = P.sums + c * kSums;
    Sn[0] = r0;
    Sn[1] = r1;
    Sn[2] = r2;
    for (int k = 0; k < kRawSums; ++k) Sn[3 + k] = s_tot[k];
    Sn[22] = 0.0;
    Sn[23] = 0.0;
  }
}

__global__ void macro_kernel(const double *sums, double *macro, int64_t nc, double w) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  CellMacro m;
  macro_from_sums(sums + c * kSums, w, m);
  double *o = macro + 8 * c;
  o[0] = m.n;
  o[1] = m.u[0];
  o[2] = m.u[1];
  o[3] = m.u[2];
  o[4] = m.T;
  o[5] = m.q[0];
  o[6] = m.q[1];
  o[7] = m.q[2];
}

__global__ void residual_reduce_kernel(const double *respart, int64_t nc, double dt,
                                       double *out) {
  __shared__ double s_a[1024], s_b[1024];
  double a = 0.0, b = 0.0;
  for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) {
    a += respart[2 * c];
    b += respart[2 * c + 1];
  }
  s_a[threadIdx.x] = a;
  s_b[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      s_a[threadIdx.x] += s_a[threadIdx.x + s];
      s_b[threadIdx.x] += s_b[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(s_a[0]) / (dt * sqrt(s_b[0]));
}

__global__ void maxwellian_fill_kernel(double *out, const double *xi0, const double *xi1,
                                       const double *xi2, int N1, int N2, int N3, double n,
                                       double ux, double uy, double uz, double T) {
  const int64_t nn = (int64_t)N1 * N2 * N3;
  const double cst = n / pow(kPi * T, 1.5);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(idx % N3);
    const int i2 = (int)((idx / N3) % N2);
    const int i1 = (int)(idx / ((int64_t)N2 * N3));
    const double v1 = xi0[i1] - ux, v2 = xi1[i2] - uy, v3 = xi2[i3] - uz;
    out[idx] = cst * exp(-(v1 * v1 + v2 * v2 + v3 * v3) / T);
  }
}

__global__ void cell_maxwellians_kernel(double *f, const double *n, const double *u,
                                        const double *T, const double *xi0, const double *xi1,
                                        const double *xi2, int N1, int N2, int N3) {
  const int64_t c = blockIdx.y;
  const int64_t nn = (int64_t)N1 * N2 * N3;
  const double Tc = T[c];
  const double cst = n[c] / pow(kPi * Tc, 1.5);
  const double ux = u[3 * c], uy = u[3 * c + 1], uz = u[3 * c + 2];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(idx % N3);
    const int i2 = (int)((idx / N3) % N2);
    const int i1 = (int)(idx / ((int64_t)N2 * N3));
    const double v1 = xi0[i1] - ux, v2 = xi1[i2] - uy, v3 = xi2[i3] - uz;
    f[c * nn + idx] = cst * exp(-(v1 * v1 + v2 * v2 + v3 * v3) / Tc);
  }
}

__global__ void inflow_sum_kernel(const double *g, const double *xi0, const double *xi1,
                                  const double *xi2, int N1, int N2, int N3, double e0,
                                  double e1, double e2, double *out) {
  __shared__ double s[256];
  const int64_t nn = (int64_t)N1 * N2 * N3;
  double a = 0.0;
  for (int64_t idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int i3 = (int)(idx % N3);
    const int i2 = (int)((idx / N3) % N2);
    const int i1 = (int)(idx / ((int64_t)N2 * N3));
    const double x = e0 * xi0[i1] + e1 * xi1[i2] + e2 * xi2[i3];
    if (x < 0.0) a = fma(x, g[idx], a);
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = s[0];
}

size_t step_smem_bytes(int N1, int N2, int N3) {
  return sizeof(double) * (size_t)(20 * N1 + N2 + N3);
}

template <int B>
void launch_step_B(const FullParams &p, bool all_axis, bool incr, cudaStream_t s) {
  const size_t smem = step_smem_bytes(p.N1, p.N2, p.N3);
  if (incr) {
    if (all_axis)
      full_step_kernel<B, true, true><<<(unsigned)p.nc, B, smem, s>>>(p);
    else
      full_step_kernel<B, false, true><<<(unsigned)p.nc, B, smem, s>>>(p);
  } else if (all_axis) {
    full_step_kernel<B, true, false><<<(unsigned)p.nc, B, smem, s>>>(p);
  } else {
    full_step_kernel<B, false, false><<<(unsigned)p.nc, B, smem, s>>>(p);
  }
}

// ------------------------------------------------------------------------
// LU-SGS sweeps of the implicit step (Section 3, linear-system equation),
// scaled by dt: with c_l = dt |A_l| / |V_i| and e_l outward from cell i,
//   D~_i(xi) = 1 + dt nu_i + sum_l c_l (xi.e_l)^+      (all six faces),
//   M~_l(xi) = c_l (xi.e_l)^-                           (interior face l to cell j),
//   forward : g_i  = (g_i - sum_{l: j<i} M~_l g_j) / D~_i   (g_i = dt R_i on entry)
//   backward: df_i = g_i - (sum_{l: j>i} M~_l df_j) / D~_i
// Every node is independent within a sweep: a CTA takes one row i1 of one cell
// of the wavefront (grid: cells x N1), its threads the columns (i2, i3) of that
// row with coalesced loads of the cell's and its neighbours' rows.  FP64 issue
// bounds the sweep, so on meshes whose faces all lie on coordinate planes the
// face weights are looked up, not recomputed per node: the axis-1 faces' weights
// are CTA scalars, the axis-2/3 faces' sit in shared-memory tables over i2 / i3,
// and D~ = d0(i1) + d2(i2) + d3(i3).  The forward sweep stores 1/D~ for the
// backward sweep.  Every neighbour a cell reads belongs to an earlier wavefront
// of the same sweep, so the launch order of the wavefronts reproduces the
// sequential sweep exactly.
template <int B, bool ALL_AXIS, bool FWD>
__global__ void __launch_bounds__(B) lusgs_sweep_kernel(const LusgsParams P) {
  extern __shared__ double tab[];
  __shared__ SlotDev s_slot[6];
  __shared__ double s_d0;     // 1 + dt nu + sum_{axis-1 faces} c max(s xi1, 0) at this row
  __shared__ double s_m0[6];  // axis-1 faces: c min(s xi1, 0) at this row
  const int64_t c = P.cells[blockIdx.x];
  const int i1 = blockIdx.y;
  const int tid = threadIdx.x;
  const int N2 = P.N2, N3 = P.N3;
  const int NP = N2 * N3;
  const int Nm = N2 > N3 ? N2 : N3;
  const int64_t nn = (int64_t)P.N1 * NP;
  double *tD = tab;            // [N2 + N3] axis-2 / axis-3 faces' sum of c max(s xi, 0)
  double *tM = tD + N2 + N3;   // [6][Nm] c min(s xi, 0) of face l over its axis
  if (tid < 6) s_slot[tid] = P.slot[c * 6 + tid];
  __syncthreads();
  const double x1 = P.xi[0][i1];
  if (tid == 0) {
    double d = 1.0 + P.dtnu[c];
    for (int l = 0; l < 6; ++l) {
      const SlotDev &sl = s_slot[l];
      s_m0[l] = 0.0;
      if (ALL_AXIS && sl.axis == 0) {
        const double sx = sl.sgn * x1;
        d = fma(sl.c, fmax(sx, 0.0), d);
        s_m0[l] = sl.c * fmin(sx, 0.0);
      }
    }
    s_d0 = d;
  }
  if (ALL_AXIS) {
    for (int k = tid; k < N2 + N3; k += B) {
      const int ax = k < N2 ? 1 : 2;
      const int i = k < N2 ? k : k - N2;
      const double x = (k < N2 ? P.xi[1] : P.xi[2])[i];
      double d = 0.0;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        if (sl.axis == ax) {
          const double sx = sl.sgn * x;
          d = fma(sl.c, fmax(sx, 0.0), d);
          tM[l * Nm + i] = sl.c * fmin(sx, 0.0);
        }
      }
      tD[k] = d;
    }
  }
  __syncthreads();
  const int64_t row = (int64_t)i1 * NP;
  const double *nbp[6];  // this row of the neighbour across face l, if face l couples
  int ax[6];             // on this sweep's side: the axis of face l, else -1
  double m0[6];
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    const SlotDev &sl = s_slot[l];
    const bool on = sl.kind == kInterior && (FWD ? (int64_t)sl.src < c : (int64_t)sl.src > c);
    nbp[l] = P.g + (on ? (int64_t)sl.src : c) * nn + row;
    ax[l] = on ? (ALL_AXIS ? sl.axis : 3) : -1;
    m0[l] = s_m0[l];
  }
  const double d0 = s_d0;
  double *__restrict__ gc = P.g + c * nn + row;
  double *__restrict__ rc = P.rD + c * nn + row;
  for (int p = tid; p < NP; p += B) {
    const int i2 = p / N3, i3 = p - i2 * N3;
    double D, S = 0.0;
    if (ALL_AXIS) {
      D = d0 + tD[i2] + tD[N2 + i3];
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if (ax[l] >= 0) {
          const double m = ax[l] == 0 ? m0[l] : tM[l * Nm + (ax[l] == 1 ? i2 : i3)];
          S = fma(m, nbp[l][p], S);
        }
      }
    } else {
      const double x2 = P.xi[1][i2], x3 = P.xi[2][i3];
      D = d0;
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        const double xn = sl.axis >= 0 ? sl.sgn * (sl.axis == 0 ? x1 : (sl.axis == 1 ? x2 : x3))
                                       : fma(sl.e[0], x1, fma(sl.e[1], x2, sl.e[2] * x3));
        const double x = sl.c * xn;
        D += fmax(x, 0.0);
        if (ax[l] >= 0) S = fma(fmin(x, 0.0), nbp[l][p], S);
      }
    }
    if (FWD) {
      const double r = 1.0 / D;
      rc[p] = r;
      gc[p] = (gc[p] - S) * r;
    } else {
      gc[p] = fma(-S, rc[p], gc[p]);
    }
  }
}

// f^{n+1} = f^n + df (in place over df) and the moment sums of f^{n+1} about the
// cell's velocity u^n, the wall outflow sums and the residual parts, as in the
// epilogue of the explicit step.
template <int B>
__global__ void __launch_bounds__(B) lusgs_apply_kernel(const FullParams P) {
  extern __shared__ double tab[];
  __shared__ SlotDev s_slot[6];
  __shared__ double s_red[B / 32][kRawSums];
  __shared__ double s_tot[kRawSums];
  __shared__ double s_u[3];
  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x;
  const int N1 = P.N1, N2 = P.N2, N3 = P.N3;
  const int NP = N2 * N3;
  const int64_t nn = (int64_t)N1 * NP;
  double *tV1 = tab, *tV2 = tV1 + N1, *tV3 = tV2 + N1, *tX1 = tV3 + N1;
  const double *S = P.sums + c * kSums;
  if (tid < 6) s_slot[tid] = P.slot[c * 6 + tid];
  if (tid == 0) {
    CellMacro m;
    macro_from_sums(S, P.w, m);
    s_u[0] = m.u[0];
    s_u[1] = m.u[1];
    s_u[2] = m.u[2];
  }
  __syncthreads();
  const double r0 = s_u[0], r1 = s_u[1], r2 = s_u[2];
  for (int i = tid; i < N1; i += B) {
    const double x = P.xi[0][i], v = x - r0;
    tV1[i] = v;
    tV2[i] = v * v;
    tV3[i] = v * v * v;
    tX1[i] = x;
  }
  __syncthreads();
  double acc[kRawSums];
#pragma unroll
  for (int k = 0; k < kRawSums; ++k) acc[k] = 0.0;
  const double *__restrict__ fc = P.f + c * nn;
  double *__restrict__ fo = P.fnew + c * nn;
  for (int p = tid; p < NP; p += B) {
    const int i2 = p / N3, i3 = p - i2 * N3;
    const double x2 = P.xi[1][i2], x3 = P.xi[2][i3];
    double P0 = 0.0, P1 = 0.0, P2 = 0.0, P3 = 0.0;
    double O[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i1 = 0; i1 < N1; ++i1) {
      const int64_t off = (int64_t)i1 * NP + p;
      const double g = __ldg(fc + off) + fo[off];
      fo[off] = g;
      P0 += g;
      P1 = fma(tV1[i1], g, P1);
      P2 = fma(tV2[i1], g, P2);
      P3 = fma(tV3[i1], g, P3);
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        const SlotDev &sl = s_slot[l];
        if (sl.kind == kWall) {
          const double x = sl.e[0] * tX1[i1] + sl.e[1] * x2 + sl.e[2] * x3;
          O[l] = fma(fmax(x, 0.0), g, O[l]);
        }
      }
    }
    fold_column(acc, P0, P1, P2, P3, x2 - r1, x3 - r2);
#pragma unroll
    for (int l = 0; l < 6; ++l) acc[13 + l] += O[l];
  }
  warp_block_reduce<B>(acc, s_red, s_tot);
  if (tid == 0) {
    double *Sn = P.sums_new + c * kSums;
    Sn[0] = r0;
    Sn[1] = r1;
    Sn[2] = r2;
    for (int k = 0; k < kRawSums; ++k) Sn[3 + k] = s_tot[k];
    Sn[22] = 0.0;
    Sn[23] = 0.0;
    if (P.respart) {
      double U0[5], U1[5];
      conserved_from_sums(S, P.w, U0);
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

}  // namespace

// block size: 256 threads, fewer for small velocity grids
static int pick_block(int NP) {
  if (NP >= 256) return 256;
  if (NP > 64) return 128;
  return 64;
}

void launch_full_step(const FullParams &p, cudaStream_t s) {
  const bool all_axis = p.all_axis != 0;
  switch (pick_block(p.N2 * p.N3)) {
    case 256: launch_step_B<256>(p, all_axis, false, s); break;
    case 128: launch_step_B<128>(p, all_axis, false, s); break;
    default: launch_step_B<64>(p, all_axis, false, s); break;
  }
}

void launch_full_rhs(const FullParams &p, cudaStream_t s) {
  const bool all_axis = p.all_axis != 0;
  switch (pick_block(p.N2 * p.N3)) {
    case 256: launch_step_B<256>(p, all_axis, true, s); break;
    case 128: launch_step_B<128>(p, all_axis, true, s); break;
    default: launch_step_B<64>(p, all_axis, true, s); break;
  }
}

template <int B, bool FWD>
static void launch_sweep_B(const LusgsParams &p, int ncell, cudaStream_t s) {
  const dim3 grid((unsigned)ncell, (unsigned)p.N1);
  const size_t smem = sizeof(double) * (size_t)(p.N2 + p.N3 + 6 * std::max(p.N2, p.N3));
  if (p.all_axis)
    lusgs_sweep_kernel<B, true, FWD><<<grid, B, smem, s>>>(p);
  else
    lusgs_sweep_kernel<B, false, FWD><<<grid, B, 0, s>>>(p);
}

void launch_lusgs_sweep(const LusgsParams &p, int ncell, bool forward, cudaStream_t s) {
  if (ncell <= 0) return;
  switch (pick_block(p.N2 * p.N3)) {
    case 256: forward ? launch_sweep_B<256, true>(p, ncell, s) : launch_sweep_B<256, false>(p, ncell, s); break;
    case 128: forward ? launch_sweep_B<128, true>(p, ncell, s) : launch_sweep_B<128, false>(p, ncell, s); break;
    default: forward ? launch_sweep_B<64, true>(p, ncell, s) : launch_sweep_B<64, false>(p, ncell, s); break;
  }
}

void launch_lusgs_apply(const FullParams &p, cudaStream_t s) {
  const size_t smem = sizeof(double) * 4 * (size_t)p.N1;
  switch (pick_block(p.N2 * p.N3)) {
    case 256: lusgs_apply_kernel<256><<<(unsigned)p.nc, 256, smem, s>>>(p); break;
    case 128: lusgs_apply_kernel<128><<<(unsigned)p.nc, 128, smem, s>>>(p); break;
    default: lusgs_apply_kernel<64><<<(unsigned)p.nc, 64, smem, s>>>(p); break;
  }
}

void launch_full_moments(const MomentParams &p, cudaStream_t s) {
  const int NP = p.N2 * p.N3;
  const size_t smem = sizeof(double) * 4 * (size_t)p.N1;
  switch (pick_block(NP)) {
    case 256: full_moments_kernel<256><<<(unsigned)p.nc, 256, smem, s>>>(p); break;
    case 128: full_moments_kernel<128><<<(unsigned)p.nc, 128, smem, s>>>(p); break;
    default: full_moments_kernel<64><<<(unsigned)p.nc, 64, smem, s>>>(p); break;
  }
}

void launch_macro_from_sums(const double *sums, double *macro, int64_t nc, double w,
                            cudaStream_t s) {
  const int B = 128;
  macro_kernel<<<(unsigned)((nc + B - 1) / B), B, 0, s>>>(sums, macro, nc, w);
}

void launch_residual_reduce(const double *respart, int64_t nc, double dt, double *out,
                            cudaStream_t s) {
  residual_reduce_kernel<<<1, 1024, 0, s>>>(respart, nc, dt, out);
}

void launch_maxwellian_fill(double *out, const double *xi0, const double *xi1,
                            const double *xi2, int N1, int N2, int N3, double n,
                            const double u[3], double T, cudaStream_t s) {
  const int64_t nn = (int64_t)N1 * N2 * N3;
  const int B = 256;
  const unsigned g = (unsigned)((nn + B - 1) / B);
  maxwellian_fill_kernel<<<g, B, 0, s>>>(out, xi0, xi1, xi2, N1, N2, N3, n, u[0], u[1], u[2],
                                         T);
}

void launch_cell_maxwellians(double *f, const double *n, const double *u, const double *T,
                             const double *xi0, const double *xi1, const double *xi2,
                             int64_t nc, int N1, int N2, int N3, cudaStream_t s) {
  const int64_t nn = (int64_t)N1 * N2 * N3;
  const int B = 256;
  dim3 grid((unsigned)((nn + B - 1) / B), (unsigned)nc);
  cell_maxwellians_kernel<<<grid, B, 0, s>>>(f, n, u, T, xi0, xi1, xi2, N1, N2, N3);
}

void launch_inflow_sum(const double *ghost, const double *xi0, const double *xi1,
                       const double *xi2, int N1, int N2, int N3, const double e[3],
                       double *out, cudaStream_t s) {
  inflow_sum_kernel<<<1, 256, 0, s>>>(ghost, xi0, xi1, xi2, N1, N2, N3, e[0], e[1], e[2], out);
}

}  // namespace dvm
