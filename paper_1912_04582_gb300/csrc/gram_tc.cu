// Gram matrices C = X X^T of many small row-major FP32 matrices X (n x K, n <= 64,
// K <= 4096) on the tcgen05 tensor cores, exact to FP64 rounding of the sliced input:
// the first-mode Gram matrices of the Tucker rounding (Section 4 item 4: the
// truncated SVD of the unfolding, taken here as the eigen-decomposition of its Gram
// matrix), which need entries accurate far below FP32 rounding (the rank rule at
// eps = 1e-6 compares discarded energies of ~1e-13 of the trace).
//
// Exact integer split (an Ozaki-type scheme).  Row a of X is scaled by 2^(6 - e_a),
// e_a the smallest integer with max_j |x_aj| <= 2^e_a, and split into S = 5 slices of
// signed integers,
//     x_aj = 2^(e_a - 6) (s0 + 2^-7 s1 + 2^-14 s2 + 2^-21 s3 + 2^-28 s4) + r_aj,
// each |s_k| <= 64 (round to nearest at each level), |r_aj| <= 2^-35 max_j |x_aj|.
// Every slice is an integer exactly representable in bf16, every product of two
// slices is an integer of magnitude <= 2^12, and a sum of K <= 4096 of them stays
// <= 2^24: the tensor cores (kind::f16, bf16 inputs, FP32 accumulators) add them
// without rounding.  Then
//     C_ab = 2^(e_a + e_b - 12) sum_{k,l} 2^(-7(k+l)) D^(k,l)_ab,
//     D^(k,l) = S_k S_l^T,
// formed in FP64 in a fixed order.  The pair (4, 4), of relative size 2^-56, is
// left out.  The result is the Gram matrix of the sliced tensor X - r to FP64
// rounding: a relative perturbation of X below 2^-35, far under the FP32 rounding
// the tensor already carries.
//
// Tensor-core mapping.  The slices of a K-chunk of 64 columns sit in shared memory
// one after the other, sp = n rounded up to 8 rows each, as a K-major 128-byte
// swizzled bf16 operand.  One MMA group takes 128 consecutive rows as A (the M = 128
// accumulator lanes hold several slices) and a run of rows as B (N up to 256
// columns hold several slices): a single instruction forms up to 4 x 5 slice
// products.  One to three groups cover every needed pair for n <= 64; their FP32
// accumulators live in tensor memory (TMEM).  Per CTA: 256 threads slice the next
// chunk (from a register prefetch) while the tensor cores work on the previous ones
// (three-stage ring, one mbarrier per stage signalled by tcgen05.commit); thread 0
// issues the MMAs.  After a cell's last chunk the accumulators are read back
// (tcgen05.ld) tile by tile and combined.  Every wait is bounded: on timeout the CTA
// sets bit 1 of *flag, drains, frees its tensor memory and returns.
#include <cstdint>
#include <mutex>

#include "dvm_internal.h"
#include "tucker.h"

namespace dvm {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcStages = 3;
constexpr int kTcKC = 64;              // columns per chunk: one 128-byte bf16 row
constexpr int kTcRowBytes = 128;
constexpr int kTcWaitIters = 1 << 24;  // bound on the polls of one mbarrier phase

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes
// apart; start address in 16-byte units (the leading-dimension offset is unused for
// swizzled K-major operands)
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: FP32 accumulator, bf16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ bool bar_poll(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kTcWaitIters && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// bf16 of a small integer held in a float (exact), two per 32-bit word
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

}  // namespace

// Plan of the MMA groups for one row count n (host-side; see GramTcPlan in tucker.h):
// the set of at most three groups (A = slices a0 .. a0 + na - 1 in the 128 accumulator
// lanes, B = slices b0 .. b0 + nb - 1 in at most 256 columns) that forms every needed
// slice product with the fewest tensor-memory columns (the MMA work is proportional to
// them), found by exhaustive search; each product is owned by the first group that
// forms it.
static GramTcPlan make_plan(int n) {
  GramTcPlan p{};
  if (n < 1 || n > 64) return p;
  const int sp = n <= 32 ? 32 : (n + 7) / 8 * 8;
  const int na = 128 / sp, nbmax = 256 / sp;
  auto needed = [](int k, int l) { return k + l <= 2 * kTcSlices - 3; };  // all but (4, 4)
  auto bit = [](int k, int l) { return 1u << (k < l ? k * kTcSlices + l : l * kTcSlices + k); };
  uint32_t need = 0;
  for (int k = 0; k < kTcSlices; ++k)
    for (int l = k; l < kTcSlices; ++l)
      if (needed(k, l)) need |= bit(k, l);
  struct Cand {
    int a0, b0, nb, N;
    uint32_t mask;
  };
  Cand c[kTcSlices * kTcSlices * kTcSlices];
  int nc = 0;
  for (int a0 = 0; a0 < kTcSlices; ++a0)
    for (int b0 = 0; b0 < kTcSlices; ++b0)
      for (int nb = 1; nb <= nbmax && b0 + nb <= kTcSlices; ++nb) {
        uint32_t m = 0;
        for (int i = 0; i < na && a0 + i < kTcSlices; ++i)
          for (int j = 0; j < nb; ++j)
            if (needed(a0 + i, b0 + j)) m |= bit(a0 + i, b0 + j);
        c[nc++] = {a0, b0, nb, (nb * sp + 15) / 16 * 16, m};
      }
  int best[3] = {-1, -1, -1}, best_cost = 1 << 30, best_n = 0;
  for (int i = 0; i < nc; ++i) {
    // fewest columns, then fewest groups (fewer MMA instructions per K-step)
    auto better = [&](int cost, int ng) {
      return cost < best_cost || (cost == best_cost && ng < best_n);
    };
    if (c[i].mask == need && better(c[i].N, 1)) {
      best_cost = c[i].N;
      best[0] = i;
      best_n = 1;
    }
    for (int j = i + 1; j < nc; ++j) {
      const int cj = c[i].N + c[j].N;
      if ((c[i].mask | c[j].mask) == need && cj <= 512 && better(cj, 2)) {
        best_cost = cj;
        best[0] = i;
        best[1] = j;
        best_n = 2;
      }
      for (int k = j + 1; k < nc; ++k) {
        const int ck = cj + c[k].N;
        if ((c[i].mask | c[j].mask | c[k].mask) == need && ck <= 512 && better(ck, 3)) {
          best_cost = ck;
          best[0] = i;
          best[1] = j;
          best[2] = k;
          best_n = 3;
        }
      }
    }
  }
  if (best_n == 0) return p;
  p.n = n;
  p.sp = sp;
  int col = 0;
  uint32_t owned = 0;
  for (int g = 0; g < best_n; ++g) {
    const Cand &q = c[best[g]];
    p.a0[g] = q.a0;
    p.b0[g] = q.b0;
    p.nb[g] = q.nb;
    p.N[g] = q.N;
    p.col[g] = col;
    col += q.N;
    for (int i = 0; i < na && q.a0 + i < kTcSlices; ++i)
      for (int j = 0; j < q.nb; ++j) {
        const int k = q.a0 + i, l = q.b0 + j;
        if (needed(k, l) && !(owned & bit(k, l))) {
          owned |= bit(k, l);
          p.own[k * kTcSlices + l] = (signed char)(g + 1);
        }
      }
  }
  p.ngroups = best_n;
  p.ncols = col <= 32 ? 32 : col <= 64 ? 64 : col <= 128 ? 128 : col <= 256 ? 256 : 512;
  int rows = kTcSlices * sp;
  for (int g = 0; g < p.ngroups; ++g) {
    const int ra = p.a0[g] * sp + 128, rb = p.b0[g] * sp + p.N[g];
    rows = ra > rows ? ra : rows;
    rows = rb > rows ? rb : rows;
  }
  p.buf_rows = (rows + 7) / 8 * 8;
  return p;
}

GramTcPlan gram_tc_plan(int n) {
  static GramTcPlan plans[65];
  static bool made[65] = {};
  static std::mutex mu;
  if (n < 1 || n > 64) return GramTcPlan{};
  std::lock_guard<std::mutex> lk(mu);
  if (!made[n]) {
    plans[n] = make_plan(n);
    made[n] = true;
  }
  return plans[n];
}

size_t gram_tc_smem_bytes(const GramTcPlan &p) {
  const size_t stages = (size_t)kTcStages * p.buf_rows * kTcRowBytes;
  const size_t acc = sizeof(double) * 64 * 65 / 2;  // upper triangle, n <= 64
  return 1024 + stages + acc + 64 * (sizeof(int) + sizeof(float)) + 64;
}

namespace {

struct TcArgs {
  const float *X;   // cell j: X + j * xstride, row-major n x K
  int64_t xstride;
  int64_t ncell;
  int K;
  float2 *C;        // cell j: C + j * cstride, n x n double-float pairs (hi, lo), or
  double *Cd;       // the same as doubles (exactly one of C, Cd is set)
  int64_t cstride;
  double *disc;     // [ncell] set to 0 (no columns left out), may be null
  int *flag;
  GramTcPlan plan;
};

__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel(TcArgs A) {
  extern __shared__ unsigned char tc_raw[];
  const GramTcPlan &P = A.plan;
  const int n = P.n, sp = P.sp, K = A.K;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  const size_t stage_bytes = (size_t)P.buf_rows * kTcRowBytes;
  unsigned char *stages = base;
  double *Sacc = reinterpret_cast<double *>(stages + kTcStages * stage_bytes);  // upper triangle
  int *rexp = reinterpret_cast<int *>(Sacc + 64 * 65 / 2);
  float *rinv = reinterpret_cast<float *>(rexp + 64);
  __shared__ __align__(8) unsigned long long s_bar[kTcStages];
  __shared__ uint32_t s_tmem;

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&s_tmem)),
                 "r"(P.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const int nchunk = (K + kTcKC - 1) / kTcKC;
  const int items = n * (kTcKC / 8);  // (row, 8-column piece) per chunk
  uint32_t issued = 0;                // chunks committed so far (all cells of this CTA)
  bool fail = false;

  for (int64_t cell = blockIdx.x; cell < A.ncell && !fail; cell += gridDim.x) {
    const float *X = A.X + cell * A.xstride;
    // pass 1: row scales (exponent of the row maximum)
    for (int a = warp; a < n; a += kTcThreads / 32) {
      float m = 0.f;
      for (int j = lane * 4; j < K; j += 32 * 4) {
        const float4 v = *reinterpret_cast<const float4 *>(X + (int64_t)a * K + j);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) {
        int e = m > 0.f ? ilogbf(m) + 1 : 0;
        e = e < -100 ? -100 : (e > 100 ? 100 : e);
        rexp[a] = e;
        rinv[a] = ldexpf(1.0f, 6 - e);
      }
    }
    for (int i = tid; i < n * (n + 1) / 2; i += kTcThreads) Sacc[i] = 0.0;
    __syncthreads();
    // register prefetch of a chunk's pieces (at most two per thread: n <= 64)
    float pre[2][8];
    auto fetch = [&](int ch) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int it = tid + q * kTcThreads;
        const int a = it >> 3, c = it & 7, j = ch * kTcKC + c * 8;
        if (it < items && j < K) {
          const float4 *src = reinterpret_cast<const float4 *>(X + (int64_t)a * K + j);
          const float4 u = src[0], w = src[1];
          pre[q][0] = u.x; pre[q][1] = u.y; pre[q][2] = u.z; pre[q][3] = u.w;
          pre[q][4] = w.x; pre[q][5] = w.y; pre[q][6] = w.z; pre[q][7] = w.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) pre[q][e] = 0.f;
        }
      }
    };
    fetch(0);
    for (int ch = 0; ch < nchunk; ++ch, ++issued) {
      const int st = (int)(issued % kTcStages);
      unsigned char *buf = stages + (size_t)st * stage_bytes;
      // the MMAs that last read this stage must be complete
      if (issued >= (uint32_t)kTcStages) {
        const uint32_t par = ((issued / kTcStages) - 1) & 1;
        const bool ok = bar_poll(smem_addr(&s_bar[st]), par);
        if (__syncthreads_or(!ok)) {
          fail = true;
          break;
        }
      }
      // slice the prefetched pieces into the stage (row k*sp + a of slice k)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int it = tid + q * kTcThreads;
        if (it < items) {
          const int a = it >> 3, c = it & 7;
          float y[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) y[e] = pre[q][e] * rinv[a];
#pragma unroll
          for (int k = 0; k < kTcSlices; ++k) {
            float s[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              s[e] = rintf(y[e]);
              y[e] = (y[e] - s[e]) * 128.0f;
            }
            const int row = k * sp + a;
            uint4 v;
            v.x = pack2(s[0], s[1]);
            v.y = pack2(s[2], s[3]);
            v.z = pack2(s[4], s[5]);
            v.w = pack2(s[6], s[7]);
            *reinterpret_cast<uint4 *>(buf + (size_t)row * kTcRowBytes + ((c ^ (row & 7)) << 4)) = v;
          }
        }
      }
      if (ch + 1 < nchunk) fetch(ch + 1);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        fence_after();
        const uint32_t b0 = smem_addr(buf);
        for (int g = 0; g < P.ngroups; ++g) {
          const uint32_t idesc = umma_idesc(128, P.N[g]);
          const uint32_t da = b0 + (uint32_t)(P.a0[g] * sp) * kTcRowBytes;
          const uint32_t db = b0 + (uint32_t)(P.b0[g] * sp) * kTcRowBytes;
#pragma unroll
          for (int kk = 0; kk < kTcKC / 16; ++kk)
            mma_bf16(tmem + (uint32_t)P.col[g], umma_desc(da + kk * 32), umma_desc(db + kk * 32),
                     idesc, (ch > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(smem_addr(&s_bar[st]));
      }
    }
    if (fail) break;
    // the cell's last commit (and with it all earlier MMAs) must be complete
    {
      const uint32_t last = issued - 1;
      const bool ok = bar_poll(smem_addr(&s_bar[last % kTcStages]), (last / kTcStages) & 1);
      if (__syncthreads_or(!ok)) {
        fail = true;
        break;
      }
    }
    fence_after();
    // combine: tile by tile (one B slice of one group at a time), accumulators to
    // shared memory as exact FP32 integers, then each upper-triangle entry adds its
    // owned products in a fixed order
    float *tile = reinterpret_cast<float *>(stages);  // [128][sp + 1]
    const int tw = sp + 1;
    for (int g = 0; g < P.ngroups; ++g) {
      for (int jb = 0; jb < P.nb[g]; ++jb) {
        const int l = P.b0[g] + jb;
        {
          const int q = warp & 3, half = warp >> 2;  // lanes 32q .. 32q + 31
          const int c0 = jb * sp + half * (sp / 2);
          for (int cc = 0; cc < sp / 2; cc += 4) {
            uint32_t r0, r1, r2, r3;
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(P.col[g] + c0 + cc);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
                "tcgen05.wait::ld.sync.aligned;"
                : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                : "r"(taddr)
                : "memory");
            float *t = tile + (32 * q + lane) * tw + half * (sp / 2) + cc;
            t[0] = __uint_as_float(r0);
            t[1] = __uint_as_float(r1);
            t[2] = __uint_as_float(r2);
            t[3] = __uint_as_float(r3);
          }
        }
        fence_before();
        __syncthreads();
        const int na = 128 / sp;
        for (int e = tid; e < n * (n + 1) / 2; e += kTcThreads) {
          int a = 0, t = e;  // e -> (a <= b), row-major over the upper triangle
          while (t >= n - a) {
            t -= n - a;
            ++a;
          }
          const int b = a + t;
          double s = Sacc[e];
          for (int i = 0; i < na; ++i) {
            const int k = P.a0[g] + i;
            if (k >= kTcSlices || P.own[k * kTcSlices + l] != g + 1) continue;
            const double w = __longlong_as_double((long long)(1023 - 7 * (k + l)) << 52);
            s += w * (double)tile[(i * sp + a) * tw + b];
            if (k != l) s += w * (double)tile[(i * sp + b) * tw + a];
          }
          Sacc[e] = s;
        }
        __syncthreads();
      }
    }
    // C_ab = 2^(e_a + e_b - 12) S_ab (as double-float pairs or doubles), both triangles
    for (int e = tid; e < n * (n + 1) / 2; e += kTcThreads) {
      int a = 0, t = e;
      while (t >= n - a) {
        t -= n - a;
        ++a;
      }
      const int b = a + t;
      const double v = ldexp(Sacc[e], rexp[a] + rexp[b] - 12);
      if (A.Cd) {
        double *C = A.Cd + cell * A.cstride;
        C[a * n + b] = v;
        C[b * n + a] = v;
      } else {
        float2 *C = A.C + cell * A.cstride;
        const float hi = (float)v;
        const float lo = (float)(v - (double)hi);
        C[a * n + b] = make_float2(hi, lo);
        C[b * n + a] = make_float2(hi, lo);
      }
    }
    if (tid == 0 && A.disc) A.disc[cell] = 0.0;
    fence_before();
    __syncthreads();  // the accumulators and the tile are free for the next cell
    fence_after();
  }
  if (fail) {
    if (tid == 0) atomicOr(A.flag, 2);
    // drain (bounded) every committed group before giving up the tensor memory
    if (issued > 0) {
      const uint32_t last = issued - 1;
      bar_poll(smem_addr(&s_bar[last % kTcStages]), (last / kTcStages) & 1);
    }
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.ncols)
                 : "memory");
}

}  // namespace

namespace {
size_t g_opted = 0;  // dynamic shared memory the kernel may use (process-wide)

// at least half the shared memory of an SM, so that two CTAs never share one SM's
// tensor memory (each may hold up to all 512 columns)
size_t launch_smem(const GramTcPlan &p) {
  const size_t smem = gram_tc_smem_bytes(p);
  return smem < 120 * 1024 ? 120 * 1024 : smem;
}
}  // namespace

int gram_tc_prepare(int n) {
  const GramTcPlan p = gram_tc_plan(n);
  if (p.ngroups == 0) return -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  const size_t smem = launch_smem(p);
  if (smem <= g_opted) return 0;
  if (cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  g_opted = smem;
  return 0;
}

bool gram_tc_supported(int n, int K) {
  if (n < 1 || n > 64 || K < 8 || K > 4096 || (K % 8) != 0) return false;
  return gram_tc_plan(n).ngroups > 0;
}

int launch_gram_tc(const float *X, int64_t xstride, int64_t ncell, int n, int K, float2 *C,
                   double *Cd, int64_t cstride, double *disc, int *flag, cudaStream_t s) {
  if (ncell <= 0) return 0;
  if (!gram_tc_supported(n, K) || (xstride % 4) != 0 ||
      (reinterpret_cast<uintptr_t>(X) & 15) != 0)
    return -1;
  TcArgs a{};
  a.X = X;
  a.xstride = xstride;
  a.ncell = ncell;
  a.K = K;
  a.C = C;
  a.Cd = Cd;
  a.cstride = cstride;
  a.disc = disc;
  a.flag = flag;
  a.plan = gram_tc_plan(n);
  const size_t smem = launch_smem(a.plan);
  if (smem > g_opted) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap != cudaStreamCaptureStatusNone || gram_tc_prepare(n) != 0) return -1;
  }
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(ncell < sms ? ncell : sms);
  gram_tc_kernel<<<grid, kTcThreads, launch_smem(a.plan), s>>>(a);
  return 0;
}

}  // namespace dvm

// Exported building block: see include/dvm.h.
extern "C" int dvm_gram_tc(const float *X, int64_t ncell, int32_t n, int32_t K, double *C,
                           int32_t *status, void *cuda_stream) {
  if (ncell < 0 || (ncell > 0 && (!X || !C || !status))) {
    dvm::set_error("dvm_gram_tc: null argument or negative ncell");
    return DVM_ERR_INVALID_ARG;
  }
  if (!dvm::gram_tc_supported(n, K)) {
    dvm::set_error("dvm_gram_tc: needs 1 <= n <= 64 and 8 <= K <= 4096 with K a multiple of 8");
    return DVM_ERR_INVALID_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) {
    dvm::set_error("dvm_gram_tc: X must be 16-byte aligned");
    return DVM_ERR_INVALID_ARG;
  }
  if (ncell == 0) return DVM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (dvm::launch_gram_tc(X, (int64_t)n * K, ncell, n, K, nullptr, C, (int64_t)n * n, nullptr,
                          status, s) != 0) {
    dvm::set_error("dvm_gram_tc: launch configuration not available on this device");
    return DVM_ERR_UNSUPPORTED;
  }
  DVM_CUDA_TRY(cudaGetLastError());
  return DVM_OK;
}
